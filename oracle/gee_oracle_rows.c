/*
 * Row-parallel FP64 CPU oracle for sparse GEE: the same definitions as oracle_embed in
 * gee_oracle.c (Section 2 Eq. 1 and its per-entry form, Table 1 options, Section 3 CSR),
 * evaluated row by row on several host threads.
 *
 * TEST INFRASTRUCTURE AND CPU BASELINE ONLY.  Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg may load it; the library never calls it, and it shares no
 * code, header or table with the CUDA path (nor with gee_oracle.c: it is a separate
 * restatement, so that the plain oracle stays a single-threaded literal reading).
 *
 * Why its result is bit-identical to oracle_embed: every floating-point quantity of row
 * i (its degree, its row of Z, its 2-norm) is a sum over the edges whose source is i.
 * oracle_embed adds them in edge-list order.  Here the edges are first grouped by source
 * with a stable counting sort (Section 3 CSR, rows in input order), so row i sees the
 * same edges in the same order and performs the same IEEE double operations on them; the
 * augmentation term and the 2-norm follow in the same place as in oracle_embed.  Threads
 * only split the rows (and the edge list for the counting sort); no sum is split.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define RO_DIAG_AUG 1u
#define RO_LAPLACIAN 2u
#define RO_CORRELATION 4u

#define RO_ERR_INDEX 1
#define RO_ERR_LABEL 2
#define RO_ERR_WEIGHT 4
#define RO_ERR_ARG 8
#define RO_ERR_NOMEM 16

typedef struct {
    /* inputs */
    const int32_t *src, *dst, *y;
    const float *w;
    int64_t E;
    int32_t N, K;
    uint32_t flags;
    int T;
    /* shared state */
    uint32_t *hist;      /* [T][N] per-thread source counts, then per-thread start offsets */
    int64_t *rowptr;     /* [N + 1] */
    int32_t *col;        /* [E] */
    float *val;          /* [E] */
    const int64_t *nk;   /* [K] */
    double *dinv;        /* [N] D^-1/2 (only with the Laplacian) */
    double *Z;           /* [N][K] */
    int err[64];         /* per-thread validation bits */
} Job;

typedef struct {
    Job *job;
    int t;
    void (*fn)(Job *, int);
} Task;

static void *run_task(void *p) {
    Task *tk = (Task *)p;
    tk->fn(tk->job, tk->t);
    return NULL;
}

/* Run fn(job, t) for t = 0..T-1 on T threads (t = 0 on the calling thread). */
static void parallel(Job *job, void (*fn)(Job *, int)) {
    pthread_t th[64];
    Task tk[64];
    int started[64];
    for (int t = 0; t < job->T; ++t) {
        tk[t].job = job;
        tk[t].t = t;
        tk[t].fn = fn;
        started[t] = 0;
    }
    for (int t = 1; t < job->T; ++t) started[t] = pthread_create(&th[t], NULL, run_task, &tk[t]) == 0;
    fn(job, 0);
    for (int t = 1; t < job->T; ++t) {
        if (started[t]) pthread_join(th[t], NULL);
        else fn(job, t); /* could not start a thread: do its share here */
    }
}

static void span(int64_t n, int T, int t, int64_t *lo, int64_t *hi) {
    *lo = n * t / T;
    *hi = n * (t + 1) / T;
}

/* input checks of oracle_validate, split over the edges and nodes */
static void phase_validate(Job *j, int t) {
    int64_t lo, hi;
    int err = 0;
    span(j->E, j->T, t, &lo, &hi);
    for (int64_t e = lo; e < hi; ++e) {
        if (j->src[e] < 0 || j->src[e] >= j->N || j->dst[e] < 0 || j->dst[e] >= j->N) err |= RO_ERR_INDEX;
        if (j->w) {
            double x = (double)j->w[e];
            if (!isfinite(x) || ((j->flags & RO_LAPLACIAN) && x < 0.0)) err |= RO_ERR_WEIGHT;
        }
    }
    span(j->N, j->T, t, &lo, &hi);
    for (int64_t i = lo; i < hi; ++i)
        if (j->y[i] < -1 || j->y[i] >= j->K) err |= RO_ERR_LABEL;
    j->err[t] = err;
}

/* counting sort, step 1: each thread counts the sources of its slice of the edge list */
static void phase_count(Job *j, int t) {
    int64_t lo, hi;
    uint32_t *h = j->hist + (size_t)t * (size_t)j->N;
    memset(h, 0, sizeof(uint32_t) * (size_t)j->N);
    span(j->E, j->T, t, &lo, &hi);
    for (int64_t e = lo; e < hi; ++e) h[j->src[e]] += 1;
}

/* step 3: each row's start for each thread = row start + counts of earlier slices */
static void phase_offsets(Job *j, int t) {
    int64_t lo, hi;
    span(j->N, j->T, t, &lo, &hi);
    for (int64_t i = lo; i < hi; ++i) {
        int64_t run = j->rowptr[i];
        for (int s = 0; s < j->T; ++s) {
            uint32_t *h = j->hist + (size_t)s * (size_t)j->N + i;
            uint32_t c = *h;
            *h = (uint32_t)(run - j->rowptr[i]);
            run += c;
        }
    }
}

/* step 4: each thread places its slice in input order (stable) */
static void phase_scatter(Job *j, int t) {
    int64_t lo, hi;
    uint32_t *h = j->hist + (size_t)t * (size_t)j->N;
    span(j->E, j->T, t, &lo, &hi);
    for (int64_t e = lo; e < hi; ++e) {
        int32_t i = j->src[e];
        int64_t p = j->rowptr[i] + (int64_t)(h[i]++);
        j->col[p] = j->dst[e];
        j->val[p] = j->w ? j->w[e] : 1.0f;
    }
}

/* D_ii = row sum of A (+1 with augmentation), in row order, then D^-1/2 */
static void phase_degrees(Job *j, int t) {
    int64_t lo, hi;
    span(j->N, j->T, t, &lo, &hi);
    for (int64_t i = lo; i < hi; ++i) {
        double d = 0.0;
        for (int64_t p = j->rowptr[i]; p < j->rowptr[i + 1]; ++p) d += j->w ? (double)j->val[p] : 1.0;
        if (j->flags & RO_DIAG_AUG) d += 1.0;
        j->dinv[i] = d > 0.0 ? 1.0 / sqrt(d) : 0.0;
    }
}

/* W_j^k = 1 / n_k for k = y_j (Section 2) */
static double wentry(const Job *j, int32_t node, int32_t k) {
    if (j->y[node] != k || j->nk[k] == 0) return 0.0;
    return 1.0 / (double)j->nk[k];
}

/* rows of Z: the entries of the row in input order, then the augmentation term, then
 * the 2-norm, exactly as oracle_embed orders them for that row */
static void phase_rows(Job *j, int t) {
    int64_t lo, hi;
    const int32_t K = j->K;
    span(j->N, j->T, t, &lo, &hi);
    for (int64_t i = lo; i < hi; ++i) {
        double *z = j->Z + i * K;
        for (int32_t k = 0; k < K; ++k) z[k] = 0.0;
        for (int64_t p = j->rowptr[i]; p < j->rowptr[i + 1]; ++p) {
            int32_t nb = j->col[p];
            int32_t k = j->y[nb];
            if (k < 0) continue;
            double a = j->w ? (double)j->val[p] : 1.0;
            if (j->flags & RO_LAPLACIAN) a = j->dinv[i] * a * j->dinv[nb];
            z[k] += a * wentry(j, nb, k);
        }
        if (j->flags & RO_DIAG_AUG) {
            int32_t k = j->y[i];
            if (k >= 0) {
                double a = 1.0;
                if (j->flags & RO_LAPLACIAN) a = j->dinv[i] * a * j->dinv[i];
                z[k] += a * wentry(j, (int32_t)i, k);
            }
        }
        if (j->flags & RO_CORRELATION) {
            double s = 0.0;
            for (int32_t k = 0; k < K; ++k) s += z[k] * z[k];
            double r = sqrt(s);
            if (r > 0.0)
                for (int32_t k = 0; k < K; ++k) z[k] /= r;
        }
    }
}

/* Z (N x K, row-major, double) on `threads` threads (1..64).  Returns the validation
 * bits of oracle_validate (Z untouched), RO_ERR_NOMEM, or 0. */
int oracle_embed_rows(const int32_t *src, const int32_t *dst, const float *w, int64_t E, int32_t N,
                      const int32_t *y, int32_t K, uint32_t flags, int threads, double *Z) {
    if (N < 0 || E < 0 || K < 1) return RO_ERR_ARG;
    Job j;
    memset(&j, 0, sizeof(j));
    j.src = src;
    j.dst = dst;
    j.w = w;
    j.y = y;
    j.E = E;
    j.N = N;
    j.K = K;
    j.flags = flags;
    j.T = threads < 1 ? 1 : (threads > 64 ? 64 : threads);
    parallel(&j, phase_validate);
    int err = 0;
    for (int t = 0; t < j.T; ++t) err |= j.err[t];
    if (err) return err;
    if (N == 0) return 0;

    int64_t *nk = (int64_t *)calloc((size_t)K, sizeof(int64_t));
    j.hist = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)j.T * (size_t)N);
    j.rowptr = (int64_t *)malloc(sizeof(int64_t) * ((size_t)N + 1));
    j.col = (int32_t *)malloc(sizeof(int32_t) * (size_t)(E > 0 ? E : 1));
    j.val = (float *)malloc(sizeof(float) * (size_t)(E > 0 ? E : 1));
    j.dinv = (double *)malloc(sizeof(double) * (size_t)N);
    if (!nk || !j.hist || !j.rowptr || !j.col || !j.val || !j.dinv) {
        free(nk);
        free(j.hist);
        free(j.rowptr);
        free(j.col);
        free(j.val);
        free(j.dinv);
        return RO_ERR_NOMEM;
    }
    for (int32_t i = 0; i < N; ++i)
        if (y[i] >= 0) nk[y[i]] += 1;
    j.nk = nk;
    j.Z = Z;

    parallel(&j, phase_count);
    j.rowptr[0] = 0;
    for (int32_t i = 0; i < N; ++i) {
        int64_t c = 0;
        for (int t = 0; t < j.T; ++t) c += j.hist[(size_t)t * (size_t)N + i];
        j.rowptr[i + 1] = j.rowptr[i] + c;
    }
    parallel(&j, phase_offsets);
    parallel(&j, phase_scatter);
    if (flags & RO_LAPLACIAN) parallel(&j, phase_degrees);
    parallel(&j, phase_rows);

    free(nk);
    free(j.hist);
    free(j.rowptr);
    free(j.col);
    free(j.val);
    free(j.dinv);
    return 0;
}
