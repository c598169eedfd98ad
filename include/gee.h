/*
 * gee.h -- C ABI of the GB300 sparse Graph Encoder Embedding library (libgee.so).
 *
 * Method: Qin & Shen, "Efficient Graph Encoder Embedding for Large Sparse Graphs in
 * Python".  For a graph with N nodes, a directed edge list (i, j, e_ij) and labels
 * y_j in {0..K-1} (or -1 = unlabelled), the library computes the N x K embedding
 *
 *     Z = A W                                              (Section 2, Eq. 1)
 *     Z_i^k = sum_{j : y_j = k} e_ij / n_k                 (Section 2, per-entry form)
 *
 * where W_j = e_{y_j} / n_{y_j} is the normalised one-hot label matrix and n_k the class
 * size, with the three options of Section 2 / Table 1:
 *     GEE_DIAG_AUG     A -> A + I
 *     GEE_LAPLACIAN    A -> D^-1/2 A D^-1/2, D = diag(row sums), taken after A + I
 *     GEE_CORRELATION  Z_i -> Z_i / ||Z_i||_2 (rows with norm 0 stay 0)
 * The sparse matrices are held in CSR (Section 3) built on the device.
 *
 * Conventions for every entry point:
 *   - Pointers named d_* or documented "device" are device pointers (cudaMalloc / torch
 *     CUDA tensors) on the current device; the caller owns them.  The library allocates
 *     nothing: all scratch lives in the caller's workspace.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).  Device
 *     work is enqueued on it and the call returns without synchronising unless stated.
 *   - Return value: GEE_OK or a gee_error code for problems visible on the host (bad
 *     arguments, sizes, workspace, CUDA launch errors).  Problems that depend on the
 *     data (an id out of range, a bad label or weight) are reported as GEE_STATUS_* bits
 *     in a device word (`d_status`) once the stream reaches that point; outputs are then
 *     undefined but every memory access stays inside the caller's buffers.
 *   - Layouts: src/dst/labels int32, w float32, Z float32 row-major [N][K].
 *   - Limits: 0 <= N <= 2^21, 0 <= E < 2^30, 1 <= K <= 64.
 */
#ifndef GEE_H
#define GEE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Embedding options (Section 2, Table 1). */
#define GEE_DIAG_AUG 1u
#define GEE_LAPLACIAN 2u
#define GEE_CORRELATION 4u
#define GEE_ALL_OPTIONS 7u
/* Not an option of the method: gee_embed launches its kernels one by one instead of
 * replaying a cached CUDA graph (see gee_embed). */
#define GEE_NO_GRAPH_CACHE 0x100u
/* Input format, not an option of the method: the edge list is undirected and lists each
 * edge once.  Every listed edge (i, j, e) with i != j then adds e to both A_ij and A_ji (a
 * self-loop (i, i, e) adds e to A_ii once), without the caller storing both directions:
 * the reverse copies are made inside the CSR build, whose first radix pass reads the
 * input arrays once for both directions.  In the CSR, row i lists the edges that touch i
 * in input order: edge e = (i, j) gives the entry of column j and edge e = (j, i), j != i,
 * the entry of column j, each at the position of e in the list.  The CSR then holds up to
 * 2E entries (gee_build_csr: col/val need room for 2E; rowptr[N] is the count). */
#define GEE_SYMMETRIZE 0x200u

/* Supported sizes. */
#define GEE_MAX_N (1 << 21)
#define GEE_MAX_E ((int64_t)1 << 30)
#define GEE_MAX_K 64

/* Host-visible return codes. */
typedef enum gee_error {
    GEE_OK = 0,
    GEE_ERR_ARG = 1,       /* a NULL pointer where one is required, negative size, ... */
    GEE_ERR_TOO_LARGE = 2, /* N, E or K beyond the limits above */
    GEE_ERR_WORKSPACE = 3, /* workspace NULL, too small, or not 256-byte aligned */
    GEE_ERR_CUDA = 4,      /* a CUDA runtime call or kernel launch failed */
    GEE_ERR_DATA = 5,      /* (blocking calls only) the device reported GEE_STATUS_* bits */
    GEE_ERR_NOMEM = 6,     /* the server's memory budget cannot hold the request (or its pool) */
    GEE_PENDING = 7,       /* (server) the request has not completed yet */
    GEE_ERR_STATE = 8      /* (server) unknown ticket, or not allowed in the request's state */
} gee_error;

/* Device status bits, OR-ed into the status word of a call. */
#define GEE_STATUS_INDEX 1u   /* an edge endpoint outside [0, N) */
#define GEE_STATUS_LABEL 2u   /* a label outside [-1, K) */
#define GEE_STATUS_WEIGHT 4u  /* a non-finite weight, or a negative one with GEE_LAPLACIAN */
#define GEE_STATUS_TIMEOUT 8u /* a bounded wait for an asynchronous copy gave up (should never happen) */
#define GEE_STATUS_INTERNAL 16u /* an internal invariant failed: a scratch index out of range, a
                                   capacity exceeded (should never happen; indicates a library bug
                                   or a workspace overwritten during the call) */
#define GEE_STATUS_STALE 32u    /* gee_reembed: the workspace does not hold the CSR of a completed
                                   gee_embed with the same sizes, options and workspace */

/* Options.  Zero-initialise and set `flags`; the tuning fields select the kernel
 * shapes (0 = automatic) and never change which value is computed, only the order of
 * floating-point additions. */
typedef struct gee_opts {
    uint32_t flags;        /* GEE_DIAG_AUG | GEE_LAPLACIAN | GEE_CORRELATION */
    int32_t hub_threshold; /* rows with more entries are split into chunks of this many
                              entries across CTAs and merged; 0 = automatic */
    int32_t lanes_per_row; /* graph-level lanes per light row (1,2,...,32; 0 = auto from the
                              mean degree): sets the automatic threshold (256 x lanes) */
    int32_t rows_per_item; /* light rows a warp claims at once: 1,2,4,...,32; 0 = auto */
    int32_t vec_width;     /* 16-byte vectors of col (and data) each lane of the product kernel
                              keeps in flight: 2, 4 or 8; 0 = auto (the depth that keeps two or
                              more CTAs per SM with the least shared memory, leaving the most L1
                              for the node-table gathers).  Never changes the bits of Z (a
                              lane's entries are added in the same order) */
    int32_t short_len;     /* K > 8: light rows of at most this many entries are taken one lane
                              per row, longer ones by a whole warp: 8, 16, 32, 64, 128 or 256;
                              0 = auto (256).  Changes the order of additions of the rows
                              between the old and the new bound */
} gee_opts;

/*
 * gee_autotune -- chooses the tuning fields of gee_opts for one graph by running
 * gee_embed with a small set of candidates around the automatic values and timing
 * each with CUDA events on `stream` (the call waits for the stream).  The fastest
 * candidate goes to *best (flags copied from opts->flags; a tuning field of opts that
 * is already non-zero is kept fixed), its mean time in ms to *best_ms (may be NULL).
 * Arguments as for gee_embed; the workspace must hold
 * gee_autotune_workspace_size(...) bytes.  Z is overwritten (with a correct result).
 * The choice is cached per (device, N, E, K, weighted, flags, fixed fields): a repeated
 * call returns it without running anything.  Tuning changes only the order of
 * floating-point additions, never which value is computed.  Returns GEE_OK or an error.
 */
size_t gee_autotune_workspace_size(int64_t E, int32_t N, int32_t K, int weighted, const gee_opts *opts);
int gee_autotune(const int32_t *d_src, const int32_t *d_dst, const float *d_w, int64_t E, int32_t N,
                 const int32_t *d_labels, int32_t K, const gee_opts *opts, float *d_Z, void *d_workspace,
                 size_t workspace_bytes, void *stream, gee_opts *best, float *best_ms);

/*
 * The autotuner's choices persist across processes in a JSON file (one entry per line):
 * gee_tune_cache_save writes every cached choice with the name of the GPU it was measured
 * on; gee_tune_cache_load adds the file's entries measured on a GPU of the current
 * device's name (*loaded = how many, may be NULL), so a later gee_autotune on such a GPU
 * returns them without timing anything.  GEE_ERR_ARG for a missing or malformed file
 * (then nothing is loaded).  gee_tune_cache_clear forgets every cached choice.
 */
int gee_tune_cache_save(const char *path);
int gee_tune_cache_load(const char *path, int *loaded);
int gee_tune_cache_clear(void);

/* Bytes of device workspace gee_embed needs for a graph of this size.  `weighted` is
 * non-zero when a weight array will be passed.  opts may be NULL (defaults). */
size_t gee_workspace_size(int64_t E, int32_t N, int32_t K, int weighted, const gee_opts *opts);

/*
 * gee_embed -- Z = A W with the selected options (Eq. 1, Table 1), from an edge list.
 *
 *   d_src, d_dst  device int32 [E]: edge (d_src[e], d_dst[e]) adds its weight to
 *                 A[src][dst] only (store both directions for an undirected graph);
 *                 duplicates add up.  May be NULL when E == 0.
 *   d_w           device float32 [E] edge weights e_ij, or NULL for weight 1 (Section 2).
 *   E, N          edge and node counts.
 *   d_labels      device int32 [N], y_j in [0, K) or -1 (unlabelled: in no class, still
 *                 gets a row of Z).
 *   K             number of classes.
 *   opts          flags and tuning; NULL = no options, automatic tuning.
 *   d_Z           device float32 [N][K], fully written.
 *   d_workspace   device scratch of at least gee_workspace_size(...) bytes, 256-byte
 *                 aligned; its contents on entry are ignored.  Calls that run
 *                 concurrently need separate workspaces.
 *   stream        cudaStream_t (void*).
 *   d_status      device uint32, or NULL: receives the GEE_STATUS_* bits of this call
 *                 (0 = success) when the stream reaches the end of the call.
 *
 * Steps (all on the device, stream-ordered): label counts n_k and input checks; CSR of
 * A by a stable LSD radix sort on the source id (rows keep input order, Section 3);
 * degrees D (after A + I) and the node table s_j = D_jj^-1/2 / n_{y_j}; the label-gather
 * product with the augmentation term, the D_ii^-1/2 scaling and the row 2-norm fused
 * into its epilogue.  Deterministic: the same input gives bit-identical Z.
 *
 * Launch cache: the second call with the same arguments (device, every pointer, E, N,
 * K, opts, workspace_bytes) captures the call's kernel sequence into a CUDA graph, and
 * later such calls replay it with one launch instead of about a dozen, on `stream`.
 * The graph re-runs every kernel and reads the inputs afresh; only the host launch
 * work is saved.  The library keeps up to 16 graphs (least recently used goes first);
 * gee_graph_cache_clear() frees them.  GEE_NO_GRAPH_CACHE in opts->flags turns it off.
 */
int gee_embed(const int32_t *d_src, const int32_t *d_dst, const float *d_w, int64_t E, int32_t N,
              const int32_t *d_labels, int32_t K, const gee_opts *opts, float *d_Z,
              void *d_workspace, size_t workspace_bytes, void *stream, uint32_t *d_status);

/*
 * gee_reembed -- Z for NEW labels on a graph whose CSR is already built: the CSR of A,
 * the degrees D and the split and bucket plans do not depend on the labels (Section 2: W
 * is built from known or predicted labels, so an iterative or semi-supervised use embeds
 * the same graph again and again with updated labels).  Only the class sizes n_k, the
 * node table s_j = D_jj^-1/2 / n_{y_j} and the product with its epilogue run again.
 *
 *   d_labels      device int32 [N], the new y_j in [0, K) or -1.
 *   E, N, K, weighted, opts, d_workspace, workspace_bytes
 *                 exactly those of the last gee_embed (or gee_reembed) that used this
 *                 workspace; its contents must be unchanged since.  K may not change.
 *   d_Z, stream, d_status   as gee_embed.
 * The result is bit-identical to gee_embed with the new labels (same plan, same sums).
 * If the workspace does not hold such a build (checked on the device against a hash of
 * the plan and the workspace address), GEE_STATUS_STALE is set in d_status and Z is
 * undefined; every memory access still stays inside the buffers.  Repeated calls with the
 * same arguments replay a cached CUDA graph, as gee_embed does.
 */
int gee_reembed(const int32_t *d_labels, int64_t E, int32_t N, int32_t K, int weighted, const gee_opts *opts,
                float *d_Z, void *d_workspace, size_t workspace_bytes, void *stream, uint32_t *d_status);

/* Destroys the CUDA graphs cached by gee_embed (all devices).  Not to be called while
 * another thread is inside gee_embed.  Returns GEE_OK or GEE_ERR_CUDA. */
int gee_graph_cache_clear(void);

/* Number of argument sets the launch cache currently remembers (captured or seen once),
 * and in *captured (may be NULL) how many of them hold an instantiated CUDA graph. */
int gee_graph_cache_size(int *captured);

/*
 * gee_embed_timed -- gee_embed with CUDA events recorded on `stream` between its launch
 * phases; waits for the stream and stores the device time of each phase, in
 * milliseconds, into the HOST array phase_ms[GEE_NUM_PHASES] (-1 for a phase that
 * launched nothing).  For measurement only: the work and the result are those of
 * gee_embed, and it uses the same launch cache (the cached graph of a timed call holds
 * the events as event-record nodes, so replays are timed phase by phase too).  Phases,
 * in launch order:
 *   0 workspace memset, 1 k_prep (label counts, checks, first-digit histograms per
 *   range), 2 k_offsets (first pass), 3 k_scatter first pass (graphs with more than
 *   2^8 nodes), 4 k_count (final-digit histograms, row lengths), 5 k_offsets (final
 *   pass), 6 k_scatter final pass (writes the CSR), 7 k_rowscan (index_pointers,
 *   unweighted degrees, hub-row list and chunks), 8 k_wdeg (weighted degrees, hub
 *   chunks then light rows), 9 k_spmm (Z with the fused epilogue, hub chunks then
 *   light rows).
 */
#define GEE_NUM_PHASES 10
int gee_embed_timed(const int32_t *d_src, const int32_t *d_dst, const float *d_w, int64_t E, int32_t N,
                    const int32_t *d_labels, int32_t K, const gee_opts *opts, float *d_Z,
                    void *d_workspace, size_t workspace_bytes, void *stream, uint32_t *d_status,
                    float *phase_ms);

/*
 * gee_build_csr -- the sparse matrices gee_embed builds, copied out for inspection
 * (Section 3 CSR; Section 2 n_k and D).  Same inputs and workspace as gee_embed.
 *
 *   d_rowptr  device int32 [N+1]  index_pointers of A (rowptr[N] = E)
 *   d_col     device int32 [E]    col_indices, rows in input order ([2E] with GEE_SYMMETRIZE)
 *   d_val     device float32 [E]  data (1.0 for unweighted input), or NULL to skip ([2E] with
 *                                 GEE_SYMMETRIZE)
 *   d_nk      device int32 [K]    class sizes n_k, or NULL
 *   d_deg     device float32 [N]  D_ii (row sum, +1 with GEE_DIAG_AUG), or NULL
 * Integer outputs are exact.  For unweighted input d_deg holds exact integers for every
 * row with fewer than 2^24 entries (float32 represents every integer below 2^24); a
 * longer row's degree is its exact count rounded to float32 (relative error < 6e-8).
 */
int gee_build_csr(const int32_t *d_src, const int32_t *d_dst, const float *d_w, int64_t E, int32_t N,
                  const int32_t *d_labels, int32_t K, const gee_opts *opts, int32_t *d_rowptr,
                  int32_t *d_col, float *d_val, int32_t *d_nk, float *d_deg, void *d_workspace,
                  size_t workspace_bytes, void *stream, uint32_t *d_status);

/*
 * gee_class_counts -- per-class neighbour counts C[i][k] = #{entries j of row i with
 * y_j = k} from a CSR (Section 2: Z_i^k n_k for unweighted input without options).
 * d_rowptr [N+1], d_col [nnz], d_labels [N] device int32; d_C device int32 [N][K].
 * Exact integer arithmetic.  Labels outside [0, K) are ignored.
 */
int gee_class_counts(const int32_t *d_rowptr, const int32_t *d_col, int32_t N, const int32_t *d_labels,
                     int32_t K, int32_t *d_C, void *stream);

/*
 * gee_embed_host -- gee_embed on HOST buffers (pinned memory gives full copy speed):
 * copies src/dst/w/labels to the device workspace, embeds, copies Z back and waits for
 * the stream.  Returns GEE_ERR_DATA (and stores the bits in *status if non-NULL) when
 * the device reported bad data.  Workspace: gee_host_workspace_size(...) bytes.
 */
size_t gee_host_workspace_size(int64_t E, int32_t N, int32_t K, int weighted, const gee_opts *opts);
int gee_embed_host(const int32_t *src, const int32_t *dst, const float *w, int64_t E, int32_t N,
                   const int32_t *labels, int32_t K, const gee_opts *opts, float *Z,
                   void *d_workspace, size_t workspace_bytes, void *stream, uint32_t *status);

/*
 * gee_embed_static -- gee_embed without a workspace argument, for callers that cannot
 * allocate device memory.  The paper has no counterpart; this is an interface addition.
 *
 * Who needs it: code that is handed device pointers by another framework but has no
 * access to that framework's allocator, and latency-critical loops that must not call
 * cudaMalloc (it can synchronise the whole device).  Instead of a caller workspace the
 * call uses one scratch array of GEE_STATIC_WORKSPACE_BYTES (64 MiB) built into the
 * library; every GPU that loads the library holds that memory until the process exits.
 *
 *   Arguments   as gee_embed, minus d_workspace / workspace_bytes; the caller still owns
 *               and passes the inputs, d_Z and d_status.
 *   Limit       returns GEE_ERR_TOO_LARGE, launching nothing, when
 *               gee_workspace_size(E, N, K, d_w != NULL, opts) exceeds
 *               GEE_STATIC_WORKSPACE_BYTES (about 4 million weighted directed edges on a
 *               graph with more than 256 nodes, about 8 million with at most 256, about
 *               twice that unweighted), and beyond gee_embed's own limits.
 *   Allocation  none: no cudaMalloc, cudaFree or allocating library call.  The launch
 *               cache of gee_embed is bypassed (GEE_NO_GRAPH_CACHE is always set), so
 *               repeated calls never capture or instantiate a CUDA graph either.
 *   Set-up      every call looks up the array's device address (cudaGetSymbolAddress)
 *               with the calling thread's current device; the first call on a device can
 *               load the library's device code there, so make it before any stream
 *               capture.
 *   Sharing     all calls on a device use the same array, which keeps the last call's
 *               contents; each call clears what must start at zero itself.  Calls that
 *               overlap on the GPU (different streams, different host threads) race on
 *               the array and give wrong results: serialise them.
 */
#define GEE_STATIC_WORKSPACE_BYTES (64u << 20)
int gee_embed_static(const int32_t *d_src, const int32_t *d_dst, const float *d_w, int64_t E, int32_t N,
                     const int32_t *d_labels, int32_t K, const gee_opts *opts, float *d_Z, void *stream,
                     uint32_t *d_status);

/* ------------------------------------------------------------------------------------
 * Sparse Z for many classes.  Section 3 keeps the embedding as a sparse matrix; with
 * K >> 64 the dense [N][K] array would dominate the bytes.  Row i of Z holds one entry for
 * every class that occurs among the labels of i's neighbours (an unlabelled neighbour
 * counts in no class) and, with GEE_DIAG_AUG, for i's own class when i is labelled: the
 * structure of the sparse product (A (+ I)) W.  The values are those of Eq. 1 with the
 * Table 1 options, as in gee_embed (the 2-norm runs over the row's entries); an entry can
 * be 0 (weights that cancel, a degree of 0 under GEE_LAPLACIAN).
 *
 *   K                1 .. GEE_MAX_K_SPARSE classes (labels in [-1, K))
 *   d_zrowptr        device int32 [N+1] out: row i's entries are [zrowptr[i], zrowptr[i+1])
 *   d_zcol, d_zval   device int32 / float32 [zcap] out: classes (ascending within a row) and
 *                    values
 *   zcap             room in d_zcol/d_zval, at least E + N (2E + N with GEE_SYMMETRIZE):
 *                    the most entries Z can have (GEE_ERR_ARG otherwise)
 *   d_workspace      gee_sparse_workspace_size bytes, 256-byte aligned
 * A row's sums run in a fixed order for a given graph and options (the same bits on every
 * call); the order differs from gee_embed's, so the values agree with it to rounding.
 * Stream-ordered, no allocation; errors and status bits as gee_embed.  The tuning fields
 * of opts apply to the CSR build (hub_threshold) only.
 */
#define GEE_MAX_K_SPARSE (1 << 20)
size_t gee_sparse_workspace_size(int64_t E, int32_t N, int32_t K, int weighted, const gee_opts *opts);
int gee_embed_sparse(const int32_t *d_src, const int32_t *d_dst, const float *d_w, int64_t E, int32_t N,
                     const int32_t *d_labels, int32_t K, const gee_opts *opts, int32_t *d_zrowptr, int32_t *d_zcol,
                     float *d_zval, int64_t zcap, void *d_workspace, size_t workspace_bytes, void *stream,
                     uint32_t *d_status);

/* ------------------------------------------------------------------------------------
 * One graph split by source rows over several GPUs (one process per GPU).  Rows are
 * independent once the node table {y_j, s_j = D_jj^-1/2 / n_{y_j}} of every node is known
 * (Section 2: Z_i^k sums e_ij W_j^k over the row's own entries), so a rank that owns rows
 * [r0, r1) needs only the edges whose source is in that range.  Per rank:
 *   1. gee_shard_build   CSR of its rows and their degrees; its partial class sizes n_k
 *   2. (caller)          all-reduce (sum) of n_k over the ranks
 *   3. gee_shard_table   the node table entries of its rows, from the global n_k
 *   4. (caller)          all-gather of the entries into the table of all N nodes
 *   5. gee_shard_embed   Z of its rows, gathering the node table of any column
 * The library does no communication; the caller moves K int32 (step 2) and 8 bytes per
 * node (step 4), e.g. with NCCL.  All calls of one rank use the same arguments E, N, r0,
 * r1, K, weighted, opts and workspace; steps 3 and 5 read what step 1 left in the
 * workspace (step 5 checks it on the device, GEE_STATUS_STALE otherwise).  With the same
 * explicit tuning fields the rows' sums run exactly as in gee_embed of the whole graph.
 * GEE_SYMMETRIZE is refused (GEE_ERR_ARG; the size query returns 0): the reverse copy of a
 * rank's edge belongs to another rank's row, so each rank passes both directions of the
 * edges of its own rows.
 *
 *   d_src, d_dst, d_w  device [E]: the rank's edges; every d_src[e] in [r0, r1), every
 *                      d_dst[e] a global id in [0, N) (else GEE_STATUS_INDEX)
 *   d_labels           device int32 [r1 - r0]: labels of the rank's rows
 *   d_nk               device int32 [K]: out (build) the rank's class sizes; in (table) the
 *                      sizes summed over all ranks
 *   d_tab              device int32 [r1 - r0][2] (table, out: this rank's slice) or
 *                      [N][2] (embed, in: the gathered table); entry j = {y_j, bits of s_j}
 *   d_Z                device float32 [r1 - r0][K]: the rank's rows of Z
 */
size_t gee_shard_workspace_size(int64_t E, int32_t N, int32_t r0, int32_t r1, int32_t K, int weighted,
                                const gee_opts *opts);
int gee_shard_build(const int32_t *d_src, const int32_t *d_dst, const float *d_w, int64_t E, int32_t N, int32_t r0,
                    int32_t r1, const int32_t *d_labels, int32_t K, const gee_opts *opts, int32_t *d_nk,
                    void *d_workspace, size_t workspace_bytes, void *stream, uint32_t *d_status);
int gee_shard_table(int64_t E, int32_t N, int32_t r0, int32_t r1, const int32_t *d_labels, int32_t K, int weighted,
                    const gee_opts *opts, const int32_t *d_nk, int32_t *d_tab, void *d_workspace,
                    size_t workspace_bytes, void *stream);
int gee_shard_embed(int64_t E, int32_t N, int32_t r0, int32_t r1, const int32_t *d_labels, int32_t K, int weighted,
                    const gee_opts *opts, const int32_t *d_tab, float *d_Z, void *d_workspace,
                    size_t workspace_bytes, void *stream, uint32_t *d_status);

/* ------------------------------------------------------------------------------------
 * Many graphs at once.  The graphs of a batch are embedded by the same kernels in one
 * launch sequence (each kernel's work items span all graphs); each graph's Z is
 * bit-identical to what gee_embed gives for it alone.  All graphs share one option set.
 */
typedef struct gee_graph {
    const int32_t *src, *dst; /* device int32 [E] (NULL when E == 0) */
    const float *w;           /* device float32 [E] or NULL (unweighted) */
    const int32_t *labels;    /* device int32 [N] */
    float *Z;                 /* device float32 [N][K] */
    int64_t E;
    int32_t N, K;
} gee_graph;

/* Workspace bytes for a batch (0 if a graph is invalid).  `graphs` is a HOST array. */
size_t gee_batch_workspace_size(const gee_graph *graphs, int32_t G, const gee_opts *opts);

/* Embed G graphs (HOST array of descriptors).  Copies the per-graph plan (about 300
 * bytes per graph) into the workspace, then enqueues the kernels on `stream`.
 * d_status: device uint32 [G] receiving each graph's GEE_STATUS_* bits, or NULL. */
int gee_embed_batch(const gee_graph *graphs, int32_t G, const gee_opts *opts, void *d_workspace,
                    size_t workspace_bytes, void *stream, uint32_t *d_status);

/* A reusable batch plan: created once (plans, uploads the descriptors into the
 * workspace and waits for the copy), then launched any number of times on the same
 * inputs/outputs.  With use_graph != 0 the first launch captures the kernel sequence
 * in a CUDA graph and later launches replay it.  The workspace must outlive the plan. */
typedef struct gee_batch_plan gee_batch_plan;
int gee_batch_plan_create(const gee_graph *graphs, int32_t G, const gee_opts *opts, void *d_workspace,
                          size_t workspace_bytes, void *stream, gee_batch_plan **plan);
int gee_batch_plan_launch(gee_batch_plan *plan, void *stream, uint32_t *d_status, int use_graph);
/* The plan's launch sequence with CUDA events between phases (as gee_embed_timed): waits
 * and stores the device time of each phase, in ms, into HOST phase_ms[GEE_NUM_PHASES]. */
int gee_batch_plan_launch_timed(gee_batch_plan *plan, void *stream, float *phase_ms);
void gee_batch_plan_destroy(gee_batch_plan *plan);

/* The batch's tuning fields, chosen by timing whole batch launches (plans captured as CUDA
 * graphs, two replays per candidate): a coordinate search over vec_width {8, 4, 2},
 * short_len {256, 64, 128} and rows_per_item {auto, 4, 16, 32}, each field keeping its
 * fastest value.  In a batch the fields act by graph class: short_len on the graphs with
 * K > 8, rows_per_item on those with K <= 8, vec_width on the whole product launch; split
 * thresholds stay automatic per graph.  A field set in opts stays fixed.  The workspace
 * (gee_batch_autotune_workspace_size bytes) is overwritten, and so are the graphs' Z;
 * best receives the options (flags of opts), best_ms the mean time of its launch. */
size_t gee_batch_autotune_workspace_size(const gee_graph *graphs, int32_t G, const gee_opts *opts);
int gee_batch_autotune(const gee_graph *graphs, int32_t G, const gee_opts *opts, void *d_workspace,
                       size_t workspace_bytes, void *stream, gee_opts *best, float *best_ms);

/* ------------------------------------------------------------------------------------
 * Serving: continuous batching of embedding requests.
 *
 * The server owns one device memory pool of `hbm_budget` bytes (allocated once by
 * gee_server_create) and a worker thread.  Submitted requests are admitted first come,
 * first served, as soon as their inputs, Z and a workspace fit in the pool; admitted
 * requests are copied to the device on a copy stream
 * and gathered into batches that run through the batch path on `streams` compute
 * streams, so work admitted while other batches run overlaps with them.  A batch's
 * workspace (the CSR of its graphs) and each request's Z stay resident until the request
 * is released.  Each request's Z is bit-identical to gee_embed's for the same graph.
 * Latency = submission to completion of the request's batch on the device.
 */
typedef struct gee_server gee_server;

typedef struct gee_server_config {
    size_t hbm_budget; /* device bytes for inputs, workspaces and Z (>= 1 MiB) */
    int32_t max_batch; /* most graphs per launch; 0 = 1024 */
    int32_t streams;   /* concurrent compute streams; 0 = 2 */
    uint32_t flags;    /* embedding options for every request */
    int32_t reserved;  /* must be 0 */
} gee_server_config;

typedef struct gee_request {
    const int32_t *src, *dst; /* HOST int32 [E]; must stay valid until the request completes
                                 (pinned memory lets the copy overlap other work) */
    const float *w;           /* HOST float32 [E] or NULL */
    const int32_t *labels;    /* HOST int32 [N] */
    int64_t E;
    int32_t N, K;
} gee_request;

typedef struct gee_server_stats {
    int64_t submitted, completed, queued, running;
    int64_t launches, edges_done;
    uint64_t pool_bytes, bytes_in_use, peak_bytes_in_use; /* peak never exceeds pool_bytes */
    int32_t last_error;                                   /* last launch error (GEE_OK if none) */
    int32_t reserved;
} gee_server_stats;

/* Create a server on the current device.  GEE_ERR_NOMEM if the pool cannot be allocated. */
int gee_server_create(const gee_server_config *cfg, gee_server **server);
/* Queue a request; *ticket identifies it.  GEE_ERR_NOMEM if it could not fit in the pool
 * even alone (refused at once). */
int gee_server_submit(gee_server *server, const gee_request *req, int64_t *ticket);
/* GEE_OK once done (then *d_Z = its device Z [N][K], *status = its GEE_STATUS_* bits,
 * *latency_ms = submit-to-done time; each output pointer may be NULL), GEE_PENDING
 * before.  wait != 0 blocks until done, for at most 120 s (then GEE_PENDING).
 * GEE_ERR_CUDA if the request's batch failed on the device. */
int gee_server_poll(gee_server *server, int64_t ticket, int wait, const float **d_Z, uint32_t *status,
                    double *latency_ms);
/* Wait for the request and copy its Z to HOST Z_host [N][K]. */
int gee_server_fetch(gee_server *server, int64_t ticket, float *Z_host);
/* Drop a request that is still queued (admitted work always completes). */
int gee_server_cancel(gee_server *server, int64_t ticket);
/* Free a completed request's resident memory (its Z, and its batch's CSR once every
 * request of the batch is released). */
int gee_server_release(gee_server *server, int64_t ticket);
int gee_server_get_stats(gee_server *server, gee_server_stats *stats);
/* Stop the worker, wait for the device, free the pool. */
void gee_server_destroy(gee_server *server);

/* Human-readable text of a gee_error code. */
const char *gee_strerror(int code);

/* Library version: major * 10000 + minor * 100 + patch. */
int gee_version(void);

#ifdef __cplusplus
}
#endif

#endif /* GEE_H */
