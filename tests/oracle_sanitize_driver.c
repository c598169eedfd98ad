/*
 * Drives every function of the C oracle over seeded small graphs, for a build with
 * AddressSanitizer and UndefinedBehaviorSanitizer (tests/test_oracle_sanitize.py).  A
 * sanitizer report or a failed check ends the process with a non-zero status.
 *
 * Cases: all 8 option settings, weighted and unweighted, empty edge lists, N = 0 and 1,
 * self-loops, duplicate edges, unlabelled nodes, empty classes, and invalid inputs (which
 * must be reported without Z being written).
 */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

int oracle_validate(const int32_t *src, const int32_t *dst, const float *w, int64_t E, int32_t N,
                    const int32_t *y, int32_t K, uint32_t flags);
void oracle_label_counts(const int32_t *y, int32_t N, int32_t K, int64_t *nk);
void oracle_csr(const int32_t *src, const int32_t *dst, const float *w, int64_t E, int32_t N,
                int64_t *rowptr, int32_t *col, float *val);
void oracle_degrees(const int32_t *src, const float *w, int64_t E, int32_t N, uint32_t flags, double *deg);
void oracle_class_counts(const int32_t *src, const int32_t *dst, int64_t E, int32_t N, const int32_t *y,
                         int32_t K, int64_t *C);
int oracle_embed(const int32_t *src, const int32_t *dst, const float *w, int64_t E, int32_t N,
                 const int32_t *y, int32_t K, uint32_t flags, double *Z);
int oracle_embed_rows(const int32_t *src, const int32_t *dst, const float *w, int64_t E, int32_t N,
                      const int32_t *y, int32_t K, uint32_t flags, int threads, double *Z);
int oracle_embed_sparse(const int32_t *src, const int32_t *dst, const float *w, int64_t E, int32_t N,
                        const int32_t *y, int32_t K, uint32_t flags, int64_t *zrowptr, int32_t *zcol,
                        double *zval);

static uint64_t rng_state;

/* SplitMix64 (Steele, Lea and Flood, 2014) */
static uint64_t next_u64(void) {
    uint64_t z = (rng_state += 0x9e3779b97f4a7c15ull);
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

static int32_t below(int32_t n) { return (int32_t)(next_u64() % (uint64_t)n); }

static int failures = 0;

static void check(int ok, const char *what, int32_t N, int64_t E, uint32_t flags) {
    if (!ok) {
        fprintf(stderr, "check failed: %s (N=%d E=%lld flags=%u)\n", what, (int)N, (long long)E, flags);
        ++failures;
    }
}

static void run_case(int32_t N, int64_t E, int32_t K, int weighted) {
    /* one extra element so that N = 0 or E = 0 still gives valid pointers */
    int32_t *src = malloc(sizeof(int32_t) * (size_t)(E + 1));
    int32_t *dst = malloc(sizeof(int32_t) * (size_t)(E + 1));
    float *w = weighted ? malloc(sizeof(float) * (size_t)(E + 1)) : NULL;
    int32_t *y = malloc(sizeof(int32_t) * (size_t)(N + 1));
    for (int64_t e = 0; e < E; ++e) {
        src[e] = below(N);
        dst[e] = (e % 7 == 3) ? src[e] : below(N); /* some self-loops */
        if (e % 11 == 5 && e > 0) { src[e] = src[e - 1]; dst[e] = dst[e - 1]; } /* duplicates */
        if (w) w[e] = (float)(1.0 - (double)(next_u64() >> 11) * 0x1.0p-53);
    }
    /* every fifth node unlabelled; with K > 1, class K-1 stays empty */
    for (int32_t i = 0; i < N; ++i) y[i] = (i % 5 == 4) ? -1 : below(K > 1 ? K - 1 : 1);

    int64_t *nk = malloc(sizeof(int64_t) * (size_t)K);
    int64_t *rowptr = malloc(sizeof(int64_t) * (size_t)(N + 1));
    int32_t *col = malloc(sizeof(int32_t) * (size_t)(E + 1));
    float *val = malloc(sizeof(float) * (size_t)(E + 1));
    double *deg = malloc(sizeof(double) * (size_t)(N + 1));
    int64_t *C = malloc(sizeof(int64_t) * (size_t)(N + 1) * (size_t)K);
    double *Z = malloc(sizeof(double) * (size_t)(N + 1) * (size_t)K);
    double *Zr = malloc(sizeof(double) * (size_t)(N + 1) * (size_t)K);

    check(oracle_validate(src, dst, w, E, N, y, K, 7u) == 0, "valid input accepted", N, E, 7u);
    oracle_label_counts(y, N, K, nk);
    int64_t labelled = 0;
    for (int32_t k = 0; k < K; ++k) labelled += nk[k];
    check(labelled == N - N / 5, "class sizes add up to the labelled nodes", N, E, 0u);

    oracle_csr(src, dst, w, E, N, rowptr, col, val);
    check(rowptr[0] == 0 && rowptr[N] == E, "index pointers span the edge list", N, E, 0u);
    for (int32_t i = 0; i < N; ++i) check(rowptr[i] <= rowptr[i + 1], "index pointers ascend", N, E, 0u);

    oracle_class_counts(src, dst, E, N, y, K, C);
    for (uint32_t flags = 0; flags < 8; ++flags) {
        oracle_degrees(src, w, E, N, flags, deg);
        for (int32_t i = 0; i < N; ++i) check(deg[i] >= 0.0 && isfinite(deg[i]), "finite degrees", N, E, flags);
        check(oracle_embed(src, dst, w, E, N, y, K, flags, Z) == 0, "embedding runs", N, E, flags);
        for (int threads = 1; threads <= 5; threads += 2) {
            check(oracle_embed_rows(src, dst, w, E, N, y, K, flags, threads, Zr) == 0, "row-parallel form runs",
                  N, E, flags);
            check(memcmp(Z, Zr, sizeof(double) * (size_t)N * (size_t)K) == 0,
                  "row-parallel form is bit-identical", N, E, flags);
        }
        for (int64_t q = 0; q < (int64_t)N * K; ++q) check(isfinite(Z[q]), "finite Z", N, E, flags);
        {  /* the sparse form: every stored value is the dense entry, bit for bit */
            int64_t *zr = malloc(sizeof(int64_t) * (size_t)(N + 1));
            int32_t *zc = malloc(sizeof(int32_t) * (size_t)(E + N + 1));
            double *zv = malloc(sizeof(double) * (size_t)(E + N + 1));
            check(oracle_embed_sparse(src, dst, w, E, N, y, K, flags, zr, zc, zv) == 0, "sparse form runs", N, E,
                  flags);
            check(zr[0] == 0 && zr[N] <= E + N, "sparse index pointers", N, E, flags);
            for (int32_t i = 0; i < N; ++i)
                for (int64_t t = zr[i]; t < zr[i + 1]; ++t) {
                    check(zc[t] >= 0 && zc[t] < K && (t == zr[i] || zc[t - 1] < zc[t]), "sparse classes ascend", N, E,
                          flags);
                    check(zv[t] == Z[(int64_t)i * K + zc[t]], "sparse value is the dense entry", N, E, flags);
                }
            free(zv);
            free(zc);
            free(zr);
        }
        if (flags == 0 && !w)  /* Z n_k equals the class counts (Eq. 1 with one-hot W / n_k) */
            for (int64_t q = 0; q < (int64_t)N * K; ++q) {
                const double c = (double)C[q];
                check(fabs(Z[q] * (double)nk[q % K] - c) <= 1e-9 * (1.0 + c), "Z n_k = class counts", N, E, flags);
            }
        if (flags & 4u)
            for (int32_t i = 0; i < N; ++i) {
                double s = 0.0;
                for (int32_t k = 0; k < K; ++k) s += Z[(int64_t)i * K + k] * Z[(int64_t)i * K + k];
                check(s == 0.0 || fabs(s - 1.0) < 1e-12, "correlation rows have norm 1 or 0", N, E, flags);
            }
    }

    /* invalid inputs: reported, Z left as it was */
    if (N > 0 && E > 0) {
        for (int64_t q = 0; q < (int64_t)N * K; ++q) Z[q] = -7.0;
        int32_t keep = dst[0];
        dst[0] = N;
        check(oracle_embed(src, dst, w, E, N, y, K, 7u, Z) == 1, "index error reported", N, E, 7u);
        check(oracle_embed_rows(src, dst, w, E, N, y, K, 7u, 3, Z) == 1, "row-parallel index error", N, E, 7u);
        dst[0] = keep;
        keep = y[0];
        y[0] = K;
        check(oracle_embed(src, dst, w, E, N, y, K, 7u, Z) == 2, "label error reported", N, E, 7u);
        check(oracle_embed_rows(src, dst, w, E, N, y, K, 7u, 2, Z) == 2, "row-parallel label error", N, E, 7u);
        y[0] = keep;
        if (w) {
            float wk = w[0];
            w[0] = -1.0f;
            check(oracle_embed(src, dst, w, E, N, y, K, 2u, Z) == 4, "negative weight reported", N, E, 2u);
            check(oracle_embed(src, dst, w, E, N, y, K, 1u, Z) == 0, "negative weight fine without Laplacian", N, E, 1u);
            w[0] = wk;
            for (int64_t q = 0; q < (int64_t)N * K; ++q) Z[q] = -7.0;
        }
        int untouched = 1;
        for (int64_t q = 0; q < (int64_t)N * K; ++q) untouched &= Z[q] == -7.0;
        check(untouched, "Z not written on error", N, E, 7u);
    }
    check(oracle_validate(src, dst, w, E, N, y, 0, 0u) == 8, "K < 1 rejected", N, E, 0u);

    free(src); free(dst); free(w); free(y); free(nk); free(rowptr); free(col); free(val);
    free(deg); free(C); free(Z); free(Zr);
}

int main(void) {
    rng_state = 20240605ull;
    const int32_t Ns[] = {0, 1, 2, 17, 200};
    const int64_t Es[] = {0, 1, 9, 500};
    const int32_t Ks[] = {1, 3, 8};
    for (size_t a = 0; a < sizeof(Ns) / sizeof(Ns[0]); ++a)
        for (size_t b = 0; b < sizeof(Es) / sizeof(Es[0]); ++b)
            for (size_t c = 0; c < sizeof(Ks) / sizeof(Ks[0]); ++c)
                for (int weighted = 0; weighted < 2; ++weighted) {
                    if (Ns[a] == 0 && Es[b] > 0) continue;  /* no node to attach an edge to */
                    run_case(Ns[a], Es[b], Ks[c], weighted);
                }
    if (failures) {
        fprintf(stderr, "%d checks failed\n", failures);
        return 1;
    }
    printf("oracle sanitizer driver: all checks passed\n");
    return 0;
}
