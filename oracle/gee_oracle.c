/*
 * FP64 CPU oracle for sparse Graph Encoder Embedding (Qin & Shen, "Efficient Graph
 * Encoder Embedding for Large Sparse Graphs in Python").
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain reference that the CUDA path
 * is checked against.  Only the tests, the smoke check and the benchmark's CPU-baseline
 * leg may load it; the library never calls it.  It shares no code, header or table with
 * the CUDA path.
 *
 * Every function follows the paper's definitions directly, in the paper's order:
 *   - W (Section 2): row j of the N x K matrix W holds 1/n_k in column k = y_j, zero
 *     elsewhere; n_k is the number of nodes of class k.
 *   - Z = A W (Eq. 1), evaluated in the edge-list form of Section 2:
 *       Z_i^k = sum over neighbours j of i with y_j = k of e_ij * W_j^k,
 *     with e_ij = 1 when the edge list carries no weights.
 *   - Options (Section 2, Table 1): diagonal augmentation replaces A by A + I;
 *     Laplacian normalisation replaces A by D^-1/2 A D^-1/2 with D the degree matrix;
 *     correlation divides each row of Z by its 2-norm.
 *   - CSR (Section 3): col_indices / data / index_pointers with rows in order.
 *
 * Readings where the paper is silent (each is listed with its reason in the design notes):
 *   - the edge list is directed: an entry (i, j, e) adds e to A_ij only;
 *   - duplicate entries add up (A_ij is the sum of their weights);
 *   - when options are combined, D is taken from A + I and the order is
 *     D^-1/2 (A + I) D^-1/2, then W, then the row 2-norm;
 *   - D_ii is the row sum of A (+1 with augmentation); D_ii = 0 gives D_ii^-1/2 = 0;
 *   - a row of Z whose 2-norm is 0 is left at zero;
 *   - label -1 marks an unlabelled node: it is in no class, so it contributes nothing
 *     as a neighbour, but it still has a row of Z;
 *   - an empty class (n_k = 0) leaves column k at zero;
 *   - within a CSR row, entries keep their input order (stable by source).
 * Floating point: every sum, product and square root is in IEEE double; input weights
 * are float32 and are widened exactly.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_DIAG_AUG 1u
#define ORACLE_LAPLACIAN 2u
#define ORACLE_CORRELATION 4u

#define ORACLE_ERR_INDEX 1
#define ORACLE_ERR_LABEL 2
#define ORACLE_ERR_WEIGHT 4
#define ORACLE_ERR_ARG 8

/* Input checks: node ids in [0, N), labels in [-1, K), weights finite, and non-negative
 * when the Laplacian option is on (a negative degree has no real inverse square root). */
int oracle_validate(const int32_t *src, const int32_t *dst, const float *w, int64_t E,
                    int32_t N, const int32_t *y, int32_t K, uint32_t flags) {
    int err = 0;
    if (N < 0 || E < 0 || K < 1) return ORACLE_ERR_ARG;
    for (int64_t e = 0; e < E; ++e) {
        if (src[e] < 0 || src[e] >= N || dst[e] < 0 || dst[e] >= N) err |= ORACLE_ERR_INDEX;
        if (w) {
            double x = (double)w[e];
            if (!isfinite(x) || ((flags & ORACLE_LAPLACIAN) && x < 0.0)) err |= ORACLE_ERR_WEIGHT;
        }
    }
    for (int32_t i = 0; i < N; ++i)
        if (y[i] < -1 || y[i] >= K) err |= ORACLE_ERR_LABEL;
    return err;
}

/* An undirected edge list that lists each edge once, as the directed list of A: for every
 * edge (i, j, e) in input order, the entry (i, j, e) and then, if i != j, its reverse
 * (j, i, e) (a self-loop is one entry of A_ii).  out_* have room for 2E entries; returns
 * the number written.  w and out_w may be NULL (unweighted). */
int64_t oracle_symmetrize(const int32_t *src, const int32_t *dst, const float *w, int64_t E, int32_t *out_src,
                          int32_t *out_dst, float *out_w) {
    int64_t n = 0;
    for (int64_t e = 0; e < E; ++e) {
        out_src[n] = src[e];
        out_dst[n] = dst[e];
        if (w && out_w) out_w[n] = w[e];
        ++n;
        if (src[e] == dst[e]) continue;
        out_src[n] = dst[e];
        out_dst[n] = src[e];
        if (w && out_w) out_w[n] = w[e];
        ++n;
    }
    return n;
}

/* n_k = number of nodes j with y_j = k (Section 2, definition of W). */
void oracle_label_counts(const int32_t *y, int32_t N, int32_t K, int64_t *nk) {
    for (int32_t k = 0; k < K; ++k) nk[k] = 0;
    for (int32_t j = 0; j < N; ++j)
        if (y[j] >= 0 && y[j] < K) nk[y[j]] += 1;
}

/* W_j^k: 1/n_k in the column of j's own class, zero elsewhere (Section 2). */
static double weight_matrix_entry(const int32_t *y, const int64_t *nk, int32_t j, int32_t k) {
    if (y[j] != k || nk[k] == 0) return 0.0;
    return 1.0 / (double)nk[k];
}

/* CSR of A (Section 3): index_pointers[i] .. index_pointers[i+1] delimit row i in
 * col_indices and data; entries of a row keep the order of the edge list (a stable
 * counting sort by source).  val may be NULL for unweighted input. */
void oracle_csr(const int32_t *src, const int32_t *dst, const float *w, int64_t E, int32_t N,
                int64_t *rowptr, int32_t *col, float *val) {
    for (int32_t i = 0; i <= N; ++i) rowptr[i] = 0;
    for (int64_t e = 0; e < E; ++e) rowptr[src[e] + 1] += 1;
    for (int32_t i = 0; i < N; ++i) rowptr[i + 1] += rowptr[i];
    int64_t *next = (int64_t *)malloc(sizeof(int64_t) * (size_t)(N > 0 ? N : 1));
    for (int32_t i = 0; i < N; ++i) next[i] = rowptr[i];
    for (int64_t e = 0; e < E; ++e) {
        int64_t p = next[src[e]]++;
        col[p] = dst[e];
        if (val) val[p] = w ? w[e] : 1.0f;
    }
    free(next);
}

/* D_ii = sum_j A_ij, with A replaced by A + I under diagonal augmentation (Section 2):
 * the row sum of the (augmented) edge list, accumulated in double in edge order. */
void oracle_degrees(const int32_t *src, const float *w, int64_t E, int32_t N, uint32_t flags,
                    double *deg) {
    for (int32_t i = 0; i < N; ++i) deg[i] = 0.0;
    for (int64_t e = 0; e < E; ++e) deg[src[e]] += w ? (double)w[e] : 1.0;
    if (flags & ORACLE_DIAG_AUG)
        for (int32_t i = 0; i < N; ++i) deg[i] += 1.0;
}

/* Number of neighbours of i (counted with multiplicity) that carry label k:
 * C[i*K + k] = #{edges (i, j) : y_j = k}.  Without options and without weights,
 * Z_i^k * n_k equals this count exactly (Eq. 1 with W = one-hot / n_k). */
void oracle_class_counts(const int32_t *src, const int32_t *dst, int64_t E, int32_t N,
                         const int32_t *y, int32_t K, int64_t *C) {
    memset(C, 0, sizeof(int64_t) * (size_t)N * (size_t)K);
    for (int64_t e = 0; e < E; ++e) {
        int32_t k = y[dst[e]];
        if (k >= 0) C[(int64_t)src[e] * K + k] += 1;
    }
}

/* Z kept sparse (Section 3): for each row i, the classes that occur among the labels of
 * i's neighbours (and i's own class with augmentation, when i is labelled), ascending,
 * with their values of Eq. 1 and the Table 1 options: the structure of the sparse
 * product (A (+ I)) W.  Each row's terms are added in edge-list order, as in oracle_embed,
 * into a per-row accumulator over the K classes, so every stored value equals
 * oracle_embed's entry bit for bit.  zrowptr [N+1], zcol / zval with room for E + N
 * entries.  Returns the validation error bits; the outputs are only written when 0. */
int oracle_embed_sparse(const int32_t *src, const int32_t *dst, const float *w, int64_t E, int32_t N,
                        const int32_t *y, int32_t K, uint32_t flags, int64_t *zrowptr, int32_t *zcol,
                        double *zval) {
    int err = oracle_validate(src, dst, w, E, N, y, K, flags);
    if (err) return err;
    int64_t *nk = (int64_t *)malloc(sizeof(int64_t) * (size_t)K);
    oracle_label_counts(y, N, K, nk);
    double *dinv = NULL;
    if (flags & ORACLE_LAPLACIAN) {
        dinv = (double *)malloc(sizeof(double) * (size_t)(N > 0 ? N : 1));
        oracle_degrees(src, w, E, N, flags, dinv);
        for (int32_t i = 0; i < N; ++i) dinv[i] = dinv[i] > 0.0 ? 1.0 / sqrt(dinv[i]) : 0.0;
    }
    /* the edges of every row, in edge-list order */
    int64_t *start = (int64_t *)calloc((size_t)N + 1, sizeof(int64_t));
    int64_t *order = (int64_t *)malloc(sizeof(int64_t) * (size_t)(E > 0 ? E : 1));
    for (int64_t e = 0; e < E; ++e) start[src[e] + 1] += 1;
    for (int32_t i = 0; i < N; ++i) start[i + 1] += start[i];
    int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)(N > 0 ? N : 1));
    for (int32_t i = 0; i < N; ++i) fill[i] = start[i];
    for (int64_t e = 0; e < E; ++e) order[fill[src[e]]++] = e;
    double *acc = (double *)calloc((size_t)K, sizeof(double));
    char *seen = (char *)calloc((size_t)K, 1);
    int32_t *touched = (int32_t *)malloc(sizeof(int32_t) * (size_t)K);
    int64_t out = 0;
    for (int32_t i = 0; i < N; ++i) {
        int32_t nt = 0;
        for (int64_t t = start[i]; t < start[i + 1]; ++t) {
            const int64_t e = order[t];
            const int32_t j = dst[e], k = y[j];
            if (k < 0) continue;
            double a = w ? (double)w[e] : 1.0;
            if (dinv) a = dinv[i] * a * dinv[j];
            acc[k] += a * weight_matrix_entry(y, nk, j, k);
            if (!seen[k]) {
                seen[k] = 1;
                touched[nt++] = k;
            }
        }
        if ((flags & ORACLE_DIAG_AUG) && y[i] >= 0) {
            const int32_t k = y[i];
            double a = 1.0;
            if (dinv) a = dinv[i] * a * dinv[i];
            acc[k] += a * weight_matrix_entry(y, nk, i, k);
            if (!seen[k]) {
                seen[k] = 1;
                touched[nt++] = k;
            }
        }
        /* ascending classes (insertion sort: rows are short in the tests) */
        for (int32_t u = 1; u < nt; ++u) {
            const int32_t v = touched[u];
            int32_t q = u - 1;
            while (q >= 0 && touched[q] > v) {
                touched[q + 1] = touched[q];
                --q;
            }
            touched[q + 1] = v;
        }
        double r = 1.0;
        if (flags & ORACLE_CORRELATION) {
            double s2 = 0.0;
            for (int32_t u = 0; u < nt; ++u) s2 += acc[touched[u]] * acc[touched[u]];
            r = sqrt(s2);
        }
        zrowptr[i] = out;
        for (int32_t u = 0; u < nt; ++u) {
            const int32_t k = touched[u];
            zcol[out] = k;
            zval[out] = ((flags & ORACLE_CORRELATION) && r > 0.0) ? acc[k] / r : acc[k];
            ++out;
            acc[k] = 0.0;
            seen[k] = 0;
        }
    }
    zrowptr[N] = out;
    free(touched);
    free(seen);
    free(acc);
    free(fill);
    free(order);
    free(start);
    free(dinv);
    free(nk);
    return 0;
}

/* The embedding Z (N x K, row-major, double), edge-list form of Eq. 1 with the options
 * of Table 1.  Returns the validation error bits; Z is only written when they are 0. */
int oracle_embed(const int32_t *src, const int32_t *dst, const float *w, int64_t E, int32_t N,
                 const int32_t *y, int32_t K, uint32_t flags, double *Z) {
    int err = oracle_validate(src, dst, w, E, N, y, K, flags);
    if (err) return err;

    /* the class sizes n_k that define W */
    int64_t *nk = (int64_t *)malloc(sizeof(int64_t) * (size_t)K);
    oracle_label_counts(y, N, K, nk);

    /* Laplacian: D^-1/2 from the degrees of A (+ I) */
    double *dinv = NULL;
    if (flags & ORACLE_LAPLACIAN) {
        dinv = (double *)malloc(sizeof(double) * (size_t)(N > 0 ? N : 1));
        oracle_degrees(src, w, E, N, flags, dinv);
        for (int32_t i = 0; i < N; ++i) dinv[i] = dinv[i] > 0.0 ? 1.0 / sqrt(dinv[i]) : 0.0;
    }

    memset(Z, 0, sizeof(double) * (size_t)N * (size_t)K);

    /* Z_i^k += e_ij * W_j^k over the edge list, with e_ij rescaled to
     * D_ii^-1/2 e_ij D_jj^-1/2 under the Laplacian option */
    for (int64_t e = 0; e < E; ++e) {
        int32_t i = src[e], j = dst[e];
        int32_t k = y[j];
        if (k < 0) continue;
        double a = w ? (double)w[e] : 1.0;
        if (dinv) a = dinv[i] * a * dinv[j];
        Z[(int64_t)i * K + k] += a * weight_matrix_entry(y, nk, j, k);
    }

    /* diagonal augmentation: the extra edge (i, i, 1) of A + I for every node */
    if (flags & ORACLE_DIAG_AUG) {
        for (int32_t i = 0; i < N; ++i) {
            int32_t k = y[i];
            if (k < 0) continue;
            double a = 1.0;
            if (dinv) a = dinv[i] * a * dinv[i];
            Z[(int64_t)i * K + k] += a * weight_matrix_entry(y, nk, i, k);
        }
    }

    /* correlation: divide every row by its 2-norm; zero rows stay zero */
    if (flags & ORACLE_CORRELATION) {
        for (int32_t i = 0; i < N; ++i) {
            double s = 0.0;
            for (int32_t k = 0; k < K; ++k) s += Z[(int64_t)i * K + k] * Z[(int64_t)i * K + k];
            double r = sqrt(s);
            if (r > 0.0)
                for (int32_t k = 0; k < K; ++k) Z[(int64_t)i * K + k] /= r;
        }
    }

    free(dinv);
    free(nk);
    return 0;
}
