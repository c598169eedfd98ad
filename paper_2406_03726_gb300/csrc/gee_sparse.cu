// Sparse Z for many classes (Section 3: the embedding is kept as a sparse matrix).
//
// Row i of Z has an entry for every class k that occurs among the labels of its
// neighbours (plus its own class with the diagonal augmentation): the structure of the
// sparse product A W (with A + I).  Its value is the same as in the dense path,
//   Z_ik = D_ii^-1/2 ( sum_{j in N(i), y_j = k} e_ij s_j  +  [aug, k = y_i] s_i ),
// scaled by 1 / ||Z_i|| with the correlation option; s_j = D_jj^-1/2 / n_{y_j} is the node
// table the CSR build leaves.  Output: zrowptr [N+1], zcol (classes, ascending within a
// row) and zval.
//
// The CSR, degrees and node table come from the usual build.  Then:
//   k_zs_wstart the first row of every window of kZsWin CSR positions.
//   k_zs_rows   one CTA per window takes the rows that start in it and have at most
//               kZsWin entries (at most 3 kZsWin - 1 entries with the augmentation terms):
//               it loads them with every thread, sorts each row's entries by (class,
//               position) in shared memory (a warp-level bitonic network per row), sums
//               each (row, class) run with a segmented scan (a fixed tree per window, so
//               the bits are reproducible), and writes each row's runs to its own slice of
//               the run buffer, at rowptr[i] + i.  Empty rows get their augmentation
//               term; longer rows are listed.
//   k_zs_long_* the listed rows' chunks of kZsChunk entries are sorted and summed the
//               same way by any CTA; then one CTA per row concatenates its chunk lists in
//               chunk order, sorts them by class with a stable radix sort and sums each
//               class's partial sums in chunk order (two-sum compensation).
//   k_zs_scan*  exclusive scan of the per-row run counts -> zrowptr.
//   k_zs_write  one warp per row: D_ii^-1/2, the row norm, and the stores.
#include "gee_internal.cuh"
#include "gee_sparse.cuh"

#include <algorithm>

namespace gee {
namespace {

constexpr int kZsWin = 1024;                  // window of CSR positions per k_zs_rows CTA
constexpr int kZsTile = 3 * kZsWin;           // entries a window can hold (at most 3 kZsWin - 1)
constexpr int kZsChunk = 4096;                // entries per chunk of a long row
constexpr int kZsScanTile = 2048;             // rows per tile of the count scan
constexpr uint32_t kZsNoClass = 0x1fffffu;    // class field of an unlabelled neighbour
constexpr uint64_t kZsPad = ~0ull;

__device__ __forceinline__ float2 two_sum2(float a, float b) {
    const float s = a + b;
    const float bb = s - a;
    const float e = (a - (s - bb)) + (b - bb);
    return make_float2(s, e);
}

// Exclusive scan of one value per thread over the CTA (256 threads); returns the prefix
// and writes the total.
__device__ __forceinline__ uint32_t zs_block_scan(uint32_t v, uint32_t *s_warp, uint32_t &total) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += t;
    }
    if (lane == 31) s_warp[w] = x;
    __syncthreads();
    uint32_t before = 0, tot = 0;
#pragma unroll
    for (int i = 0; i < kWarps; ++i) {
        const uint32_t s = s_warp[i];
        before += (i < w) ? s : 0u;
        tot += s;
    }
    __syncthreads();
    total = tot;
    return before + x - v;
}

// Exclusive scan of n <= kPer * 256 flags in place (t[0..n) -> prefix; t[n] = total).
template <int kPer = 16>
__device__ void zs_scan_array(uint32_t *t, int n, uint32_t *s_warp) {
    const int i0 = threadIdx.x * kPer;
    uint32_t loc[kPer];
    uint32_t sum = 0;
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
        loc[k] = (i0 + k < n) ? t[i0 + k] : 0u;
        sum += loc[k];
    }
    uint32_t total;
    uint32_t run = zs_block_scan(sum, s_warp, total);
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
        if (i0 + k < n) t[i0 + k] = run;
        run += loc[k];
    }
    if (threadIdx.x == 0) t[n] = total;
    __syncthreads();
}

// Bitonic sort of n (a power of two) keys with their values, ascending, in shared memory.
__device__ void zs_sort(uint64_t *key, float *val, int n) {
    for (int k = 2; k <= n; k <<= 1)
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < n; i += kThreads) {
                const int ixj = i ^ j;
                if (ixj > i) {
                    const uint64_t a = key[i], b = key[ixj];
                    const bool up = (i & k) == 0;
                    if ((a > b) == up) {
                        key[i] = b;
                        key[ixj] = a;
                        const float t = val[i];
                        val[i] = val[ixj];
                        val[ixj] = t;
                    }
                }
            }
            __syncthreads();
        }
}

// Sort key[0..L) ascending (with their values) by one warp, in place: the bitonic network
// in its all-ascending form (each merge first compares i with its mirror in the block,
// then half-cleaners), so every compare-exchange puts the smaller key at the lower index
// and positions at or past L, which act as +infinity, are never touched.
__device__ void zs_warp_sort(uint64_t *key, float *val, int L, int lane) {
    int P = 1;
    while (P < L) P <<= 1;
    auto ce = [&](int i, int j) {
        if (j < L) {
            const uint64_t a = key[i], b = key[j];
            if (a > b) {
                key[i] = b;
                key[j] = a;
                const float t = val[i];
                val[i] = val[j];
                val[j] = t;
            }
        }
    };
    for (int k = 2; k <= P; k <<= 1) {
        const int h = k >> 1;
        for (int t = lane; t < (P >> 1); t += 32) {
            const int b = t / h, o = t - b * h;
            ce(b * k + o, b * k + k - 1 - o);
        }
        __syncwarp();
        for (int d = k >> 2; d > 0; d >>= 1) {
            for (int t = lane; t < (P >> 1); t += 32) {
                const int i = (t / d) * 2 * d + (t % d);
                ce(i, i + d);
            }
            __syncwarp();
        }
    }
}

// Inclusive segmented sum of val[0..n) over runs of equal (key >> shift), in place
// (Hillis-Steele with segment flags: a fixed tree for a given run position, so the result
// is reproducible).  v2/f/f2 are scratch of n entries.
__device__ void zs_segsum(const uint64_t *key, float *val, float *v2, uint8_t *f, uint8_t *f2, int n, int shift) {
    for (int i = threadIdx.x; i < n; i += kThreads) f[i] = (i == 0 || (key[i] >> shift) != (key[i - 1] >> shift));
    __syncthreads();
    float *a = val, *b = v2;
    uint8_t *fa = f, *fb = f2;
    for (int d = 1; d < n; d <<= 1) {
        for (int i = threadIdx.x; i < n; i += kThreads) {
            if (i >= d && !fa[i]) {
                b[i] = a[i - d] + a[i];
                fb[i] = fa[i - d];
            } else {
                b[i] = a[i];
                fb[i] = fa[i];
            }
        }
        __syncthreads();
        float *t = a;
        a = b;
        b = t;
        uint8_t *tf = fa;
        fa = fb;
        fb = tf;
    }
    if (a != val) {
        for (int i = threadIdx.x; i < n; i += kThreads) val[i] = a[i];
        __syncthreads();
    }
}

__device__ __forceinline__ float node_s(const SparseArgs &a, int j) { return __int_as_float(__ldg(&a.tab[j]).y); }

// First row of every window: wstart[w] = the first row with rowptr >= w * kZsWin, for the
// windows 0 .. E / kZsWin + 1 (the last entry is N).
__global__ void __launch_bounds__(kThreads) k_zs_wstart(const __grid_constant__ SparseArgs a, int windows) {
    for (int64_t r = (int64_t)blockIdx.x * kThreads + threadIdx.x; r <= a.N; r += (int64_t)gridDim.x * kThreads) {
        // the windows (w_prev, w_r] start at row r; row N stands for the end
        const int64_t wr = r < a.N ? (int64_t)__ldg(a.rowptr + r) / kZsWin : (int64_t)windows;
        const int64_t wp = r > 0 ? (int64_t)__ldg(a.rowptr + r - 1) / kZsWin : -1;
        for (int64_t w = wp + 1; w <= wr && w <= windows; ++w) a.wstart[w] = (int32_t)r;
    }
}

// ---- k_zs_rows ----------------------------------------------------------------------------
struct ZsRowsSmem {
    uint64_t key[kZsTile];
    float val[kZsTile];
    union {                       // the segmented sum's scratch, then the tail flags and
        float v2[kZsTile + 1];    // their exclusive scan
        uint32_t t[kZsTile + 1];
    };
    uint8_t f[kZsTile], f2[kZsTile];
    int32_t rowid[kZsWin];        // rows of the window with 1..kZsWin entries, in order
    uint32_t roff[kZsWin + 1];    // their first tile position
    uint32_t s_warp[kWarps];
    int32_t s_range[2];
    uint32_t s_nm, s_ne;
};

__global__ void __launch_bounds__(kThreads) k_zs_rows(const __grid_constant__ SparseArgs a) {
    extern __shared__ __align__(16) unsigned char zs_smem[];
    ZsRowsSmem &S = *reinterpret_cast<ZsRowsSmem *>(zs_smem);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const bool aug = (a.flags & kOptAug) != 0;
    uint32_t err = 0;
    if (tid < 2) S.s_range[tid] = __ldcg(a.wstart + blockIdx.x + tid);  // rows [ra, rb) start in the window
    if (tid == 0) {
        S.s_nm = 0;
        S.s_ne = 0;
    }
    __syncthreads();
    const int ra = S.s_range[0], rb = S.s_range[1];
    // ---- classify the window's rows; lay out the short ones in the tile
    for (int r0 = ra; r0 < rb; r0 += kThreads) {
        const int r = r0 + tid;
        int len = 0;
        bool med = false, own = false;
        if (r < rb) {
            const int64_t p0 = __ldg(a.rowptr + r), p1 = __ldg(a.rowptr + r + 1);
            len = (int)(p1 - p0);
            const int yi = __ldg(a.y + r);
            own = aug && yi >= 0 && yi < a.K;
            if (len == 0) {  // only the augmentation term
                a.cnt[r] = own ? 1 : 0;
                if (own) a.runs_a[p0 + r] = make_int4(yi, __float_as_int(node_s(a, r)), 0, 0);
            } else if (len > kZsWin) {
                const uint32_t slot = atomicAdd(a.long_count, 1u);
                if (slot < a.long_cap) a.long_list[slot] = r;
                else err |= kStInternal;
            } else {
                med = true;
            }
        }
        uint32_t tot_m, tot_e;
        const uint32_t m = zs_block_scan(med ? 1u : 0u, S.s_warp, tot_m);
        const uint32_t e = zs_block_scan(med ? (uint32_t)(len + (own ? 1 : 0)) : 0u, S.s_warp, tot_e);
        if (med) {
            const uint32_t mi = S.s_nm + m;
            if (mi < (uint32_t)kZsWin) {
                S.rowid[mi] = r;
                S.roff[mi] = S.s_ne + e;
            } else {
                err |= kStInternal;
            }
        }
        __syncthreads();
        if (tid == 0) {
            S.s_nm += tot_m;
            S.s_ne += tot_e;
        }
        __syncthreads();
    }
    // the window bound (at most kZsWin rows of 1..kZsWin entries start in it) keeps both
    // within the tile; if it did not, the window is skipped and reported
    const bool over = S.s_nm > (uint32_t)kZsWin || S.s_ne > (uint32_t)kZsTile;
    if (over) err |= kStInternal;
    const int nm = over ? 0 : (int)S.s_nm;
    const int ne = over ? 0 : (int)S.s_ne;
    if (tid == 0) S.roff[nm] = (uint32_t)ne;
    __syncthreads();
    if (nm > 0) {
        const int n2 = ne;
        // ---- load the window's entries with every thread, 8 at a time, so that the column,
        // label and node-table reads of many entries are in flight together; entry p of
        // the tile belongs to the last short row with roff <= p
        constexpr int kBatch = 8;
        for (int p0b = 0; p0b < ne; p0b += kThreads * kBatch) {
            int mi[kBatch], e[kBatch], j[kBatch];
            int64_t q[kBatch];
#pragma unroll
            for (int u = 0; u < kBatch; ++u) {
                const int p = p0b + u * kThreads + tid;
                mi[u] = -1;
                e[u] = 0;
                j[u] = 0;
                q[u] = 0;
                if (p < ne) {
                    int lo = 0, hi = nm;  // last row with roff <= p
                    while (hi - lo > 1) {
                        const int mid = (lo + hi) >> 1;
                        if ((int)S.roff[mid] <= p) lo = mid;
                        else hi = mid;
                    }
                    mi[u] = lo;
                    e[u] = p - (int)S.roff[lo];
                    q[u] = (int64_t)__ldg(a.rowptr + S.rowid[lo]) + e[u];
                }
            }
#pragma unroll
            for (int u = 0; u < kBatch; ++u) {
                if (mi[u] < 0) continue;
                const int r = S.rowid[mi[u]];
                const int len = (int)(__ldg(a.rowptr + r + 1) - (q[u] - e[u]));
                j[u] = e[u] < len ? min(max(__ldg(a.col + q[u]), 0), a.N - 1) : -1 - r;  // -1 - r: the augmentation term
            }
#pragma unroll
            for (int u = 0; u < kBatch; ++u) {
                if (mi[u] < 0) continue;
                const int p = p0b + u * kThreads + tid;
                uint32_t cls;
                float v;
                if (j[u] >= 0) {
                    const int yj = __ldg(a.y + j[u]);
                    cls = (yj >= 0 && yj < a.K) ? (uint32_t)yj : kZsNoClass;
                    v = (a.val ? __ldg(a.val + q[u]) : 1.0f) * node_s(a, j[u]);
                } else {
                    const int r = -1 - j[u];
                    cls = (uint32_t)__ldg(a.y + r);
                    v = node_s(a, r);
                }
                S.key[p] = ((uint64_t)mi[u] << 33) | ((uint64_t)cls << 12) | (uint64_t)e[u];
                S.val[p] = v;
            }
        }
        __syncthreads();
        // ---- each row's entries by (class, position): one warp per row
        for (int m = warp; m < nm; m += kWarps) {
            const int o = (int)S.roff[m];
            zs_warp_sort(S.key + o, S.val + o, (int)S.roff[m + 1] - o, lane);
        }
        __syncthreads();
        zs_segsum(S.key, S.val, S.v2, S.f, S.f2, n2, 12);
        // ---- runs: the last entry of each (row, class) run holds its sum
        for (int i = tid; i < n2; i += kThreads) {
            const uint64_t k = S.key[i];
            const bool valid = k != kZsPad && ((k >> 12) & kZsNoClass) != kZsNoClass;
            const bool tail = valid && (i == n2 - 1 || (S.key[i + 1] >> 12) != (k >> 12));
            S.t[i] = tail ? 1u : 0u;
        }
        __syncthreads();
        zs_scan_array(S.t, n2, S.s_warp);
        for (int i = tid; i < n2; i += kThreads) {
            const uint64_t k = S.key[i];
            if (k == kZsPad) continue;
            const bool valid = ((k >> 12) & kZsNoClass) != kZsNoClass;
            const bool tail = valid && (i == n2 - 1 || (S.key[i + 1] >> 12) != (k >> 12));
            if (!tail) continue;
            const int mi = (int)(k >> 33);
            if (mi >= nm) {
                err |= kStInternal;
                continue;
            }
            const int r = S.rowid[mi];
            const uint32_t rank = S.t[i] - S.t[S.roff[mi]];
            const int64_t base = (int64_t)__ldg(a.rowptr + r) + r;
            a.runs_a[base + rank] = make_int4((int)((k >> 12) & kZsNoClass), __float_as_int(S.val[i]), 0, 0);
        }
        for (int mi = tid; mi < nm; mi += kThreads)
            a.cnt[S.rowid[mi]] = (int)(S.t[S.roff[mi + 1]] - S.t[S.roff[mi]]);
    }
    if (err) atomicOr(a.status, err);
}

// ---- long rows: chunks sorted in parallel, then merged row by row -----------------------
// A listed row of T = len (+1 augmentation term) entries has ceil(T / kZsChunk) chunks.
// k_zs_long_plan numbers the chunks of all listed rows; k_zs_long_sort sorts and sums each
// chunk (any CTA) into its sorted run list, stored in the row's slice of runs_b at
// c * kZsChunk; k_zs_long_merge combines a row's chunk lists (one CTA per row).

__device__ __forceinline__ int long_row_entries(const SparseArgs &a, int r, int64_t &p0) {
    p0 = __ldg(a.rowptr + r);
    const int len = (int)(__ldg(a.rowptr + r + 1) - p0);
    const int yi = __ldg(a.y + r);
    return len + (((a.flags & kOptAug) && yi >= 0 && yi < a.K) ? 1 : 0);
}

__global__ void __launch_bounds__(kThreads) k_zs_long_plan(const __grid_constant__ SparseArgs a) {
    __shared__ uint32_t s_warp[kWarps];
    const uint32_t n = min(__ldcg(a.long_count), a.long_cap);
    uint32_t run = 0;
    for (uint32_t b = 0; b < n; b += kThreads) {
        const uint32_t li = b + threadIdx.x;
        uint32_t m = 0;
        if (li < n) {
            const int r = min(max(__ldcg(a.long_list + li), 0), a.N - 1);
            int64_t p0;
            m = (uint32_t)((long_row_entries(a, r, p0) + kZsChunk - 1) / kZsChunk);
        }
        uint32_t tot;
        const uint32_t x = zs_block_scan(m, s_warp, tot);
        if (li < n) a.chunk_off[li] = run + x;
        run += tot;
    }
    if (threadIdx.x == 0) a.chunk_off[n] = min(run, a.chunk_cap);
    if (threadIdx.x == 0 && run > a.chunk_cap) atomicOr(a.status, kStInternal);
}

struct ZsLongSortSmem {
    uint64_t key[kZsChunk];
    float val[kZsChunk];
    union {                       // the segmented sum's scratch, then the tail flags and
        float v2[kZsChunk + 1];   // their exclusive scan
        uint32_t t[kZsChunk + 1];
    };
    uint8_t f[kZsChunk], f2[kZsChunk];
    uint32_t s_warp[kWarps];
    int32_t s_li;
};

struct ZsLongMergeSmem {
    uint32_t hist[kWarps][256];   // per-warp digit counts of a radix pass
    uint32_t wpre[kWarps][256];   // per tile: each warp's first place among a digit's elements
    uint16_t cnt[kWarps][256];    // per tile: each warp's elements of a digit so far
    uint32_t base[256];           // next place of each digit in the pass's output
    uint32_t s_warp[kWarps];
    int32_t s_li;
    uint32_t s_carry;
};

__global__ void __launch_bounds__(kThreads) k_zs_long_sort(const __grid_constant__ SparseArgs a) {
    extern __shared__ __align__(16) unsigned char zs_smem[];
    ZsLongSortSmem &S = *reinterpret_cast<ZsLongSortSmem *>(zs_smem);
    const int tid = threadIdx.x;
    const uint32_t n = min(__ldcg(a.long_count), a.long_cap);
    const uint32_t chunks = n ? __ldcg(a.chunk_off + n) : 0u;
    for (uint32_t gc = blockIdx.x; gc < chunks; gc += gridDim.x) {
        if (tid == 0) {  // the listed row of this chunk: last li with chunk_off[li] <= gc
            int lo = 0, hi = (int)n;
            while (hi - lo > 1) {
                const int mid = (lo + hi) >> 1;
                if (__ldcg(a.chunk_off + mid) <= gc) lo = mid;
                else hi = mid;
            }
            S.s_li = lo;
        }
        __syncthreads();
        const int li = S.s_li;
        const int r = min(max(__ldcg(a.long_list + li), 0), a.N - 1);
        int64_t p0;
        const int T = long_row_entries(a, r, p0);
        const int len = (int)(__ldg(a.rowptr + r + 1) - p0);
        const int c0 = (int)(gc - __ldcg(a.chunk_off + li)) * kZsChunk;
        const int nc = max(0, min(kZsChunk, T - c0));
        int n2 = 32;
        while (n2 < nc) n2 <<= 1;
        for (int i = tid; i < n2; i += kThreads) {
            uint64_t k = kZsPad;
            float v = 0.0f;
            if (i < nc) {
                const int e = c0 + i;
                if (e < len) {
                    const int j = min(max(__ldg(a.col + p0 + e), 0), a.N - 1);
                    const int yj = __ldg(a.y + j);
                    if (yj >= 0 && yj < a.K) {
                        k = ((uint64_t)yj << 32) | (uint64_t)e;
                        v = (a.val ? __ldg(a.val + p0 + e) : 1.0f) * node_s(a, j);
                    }
                } else {
                    k = ((uint64_t)__ldg(a.y + r) << 32) | (uint64_t)e;
                    v = node_s(a, r);
                }
            }
            S.key[i] = k;
            S.val[i] = v;
        }
        __syncthreads();
        zs_sort(S.key, S.val, n2);
        zs_segsum(S.key, S.val, S.v2, S.f, S.f2, n2, 32);
        for (int i = tid; i < n2; i += kThreads) {
            const uint64_t k = S.key[i];
            S.t[i] = (k != kZsPad && (i == n2 - 1 || (S.key[i + 1] >> 32) != (k >> 32))) ? 1u : 0u;
        }
        __syncthreads();
        zs_scan_array<kZsChunk / kThreads>(S.t, n2, S.s_warp);
        int4 *out = a.runs_b + p0 + r + c0;  // the chunk's own part of the row's slice
        for (int i = tid; i < n2; i += kThreads) {
            const uint64_t k = S.key[i];
            if (k != kZsPad && (i == n2 - 1 || (S.key[i + 1] >> 32) != (k >> 32)))
                out[S.t[i]] = make_int4((int)(k >> 32), __float_as_int(S.val[i]), 0, 0);
        }
        if (tid == 0) a.chunk_cnt[gc] = (int32_t)S.t[n2];
        __syncthreads();
    }
}

// One listed row per CTA (rows claimed one at a time): the row's chunk lists, each sorted by
// class, are concatenated in chunk order, sorted by class with a stable radix sort (8-bit
// digits; a class's entries stay in chunk order), and each run of one class is summed in
// that order with two-sum compensation.  Work and traffic are linear in the row's runs.
__global__ void __launch_bounds__(kThreads) k_zs_long_merge(const __grid_constant__ SparseArgs a) {
    extern __shared__ __align__(16) unsigned char zs_smem[];
    ZsLongMergeSmem &S = *reinterpret_cast<ZsLongMergeSmem *>(zs_smem);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const unsigned lt = (1u << lane) - 1u;
    const uint32_t n = min(__ldcg(a.long_count), a.long_cap);
    const int bits = 32 - __clz((unsigned)max(a.K - 1, 1));  // class bits
    for (;;) {
        if (tid == 0) S.s_li = (int32_t)atomicAdd(a.long_count + 1, 1u);  // rows claimed one at a time
        __syncthreads();
        const uint32_t li = (uint32_t)S.s_li;
        if (li >= n) break;
        const int r = min(max(__ldcg(a.long_list + li), 0), a.N - 1);
        int64_t p0;
        const int T = long_row_entries(a, r, p0);
        const uint32_t g0 = __ldcg(a.chunk_off + li), g1 = __ldcg(a.chunk_off + li + 1);
        int4 *const ra = a.runs_a + p0 + r, *const rb = a.runs_b + p0 + r;
        // chunk numbers beyond the capacity (reported by the plan) or more chunks than the
        // row's entries give: skip the row
        const bool ok = g0 <= g1 && g1 <= a.chunk_cap &&
                        (int64_t)(g1 - g0) <= ((int64_t)T + kZsChunk - 1) / kZsChunk;
        const int m = ok ? (int)(g1 - g0) : 0;
        // ---- the chunk lists, concatenated in chunk order, into runs_a
        int M = 0;
        for (int c = 0; c < m; ++c) {
            const int np = min(max(__ldcg(a.chunk_cnt + g0 + c), 0), kZsChunk);
            for (int t = tid; t < np; t += kThreads) ra[M + t] = __ldcg(rb + c * kZsChunk + t);
            M += np;
        }
        __syncthreads();
        // ---- stable radix sort by class, runs_a <-> runs_b
        int4 *src = ra, *dst = rb;
        for (int sh = 0; sh < bits; sh += 8) {
            for (int i = tid; i < kWarps * 256; i += kThreads) (&S.hist[0][0])[i] = 0u;
            __syncthreads();
            for (int i = tid; i < M; i += kThreads) atomicAdd(&S.hist[warp][(__ldcg(&src[i].x) >> sh) & 255], 1u);
            __syncthreads();
            {  // digit bases: exclusive scan of the digit totals (thread = digit)
                uint32_t tot = 0;
#pragma unroll
                for (int w = 0; w < kWarps; ++w) tot += S.hist[w][tid];
                uint32_t all;
                S.base[tid] = zs_block_scan(tot, S.s_warp, all);
            }
            __syncthreads();
            for (int t0 = 0; t0 < M; t0 += kThreads * 8) {
                for (int i = lane; i < 256; i += 32) S.cnt[warp][i] = 0;
                __syncwarp();
                int4 el[8];
                uint32_t dg[8], rk[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) {  // element t0 + 256 warp + 32 u + lane: tile order kept
                    const int idx = t0 + warp * 256 + u * 32 + lane;
                    const bool valid = idx < M;
                    el[u] = valid ? __ldcg(&src[idx]) : make_int4(0, 0, 0, 0);
                    dg[u] = valid ? ((uint32_t)el[u].x >> sh) & 255u : 256u + (uint32_t)lane;  // unique if invalid
                    const unsigned peers = __match_any_sync(0xffffffffu, dg[u]);
                    const uint32_t before = valid ? S.cnt[warp][dg[u]] : 0u;
                    __syncwarp();
                    if (valid && (peers & lt) == 0u) S.cnt[warp][dg[u]] = (uint16_t)(before + __popc(peers));
                    __syncwarp();
                    rk[u] = before + __popc(peers & lt);
                }
                __syncthreads();
                uint32_t tile_tot = 0;  // thread = digit: each warp's first place in the tile
#pragma unroll
                for (int w = 0; w < kWarps; ++w) {
                    S.wpre[w][tid] = tile_tot;
                    tile_tot += S.cnt[w][tid];
                }
                __syncthreads();
#pragma unroll
                for (int u = 0; u < 8; ++u)
                    if (dg[u] < 256u) dst[S.base[dg[u]] + S.wpre[warp][dg[u]] + rk[u]] = el[u];
                __syncthreads();
                S.base[tid] += tile_tot;
                __syncthreads();
            }
            int4 *tmp = src;
            src = dst;
            dst = tmp;
        }
        // ---- one run per class (in chunk order): its sum into dst, then dst -> runs_a
        if (tid == 0) S.s_carry = 0;
        __syncthreads();
        for (int t0 = 0; t0 < M; t0 += kThreads) {
            const int i = t0 + tid;
            const bool head = i < M && (i == 0 || __ldcg(&src[i].x) != __ldcg(&src[i - 1].x));
            uint32_t tot;
            const uint32_t x = zs_block_scan(head ? 1u : 0u, S.s_warp, tot);
            if (head) {
                const int4 h = __ldcg(&src[i]);
                float sum = __int_as_float(h.y), comp = __int_as_float(h.z);
                for (int j = i + 1; j < M; ++j) {
                    const int4 q = __ldcg(&src[j]);
                    if (q.x != h.x) break;
                    const float2 t = two_sum2(sum, __int_as_float(q.y));
                    sum = t.x;
                    comp += t.y + __int_as_float(q.z);
                }
                dst[S.s_carry + x] = make_int4(h.x, __float_as_int(sum), __float_as_int(comp), 0);
            }
            __syncthreads();
            if (tid == 0) S.s_carry += tot;
            __syncthreads();
        }
        const int na = (int)S.s_carry;
        if (dst != ra)
            for (int i = tid; i < na; i += kThreads) ra[i] = __ldcg(dst + i);
        if (tid == 0) a.cnt[r] = na;
        __syncthreads();
    }
}

// ---- the count scan ---------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads) k_zs_scan_tiles(const __grid_constant__ SparseArgs a) {
    __shared__ uint32_t t[kZsScanTile + 1];
    __shared__ uint32_t s_warp[kWarps];
    const int64_t r0 = (int64_t)blockIdx.x * kZsScanTile;
    const int n = (int)min((int64_t)kZsScanTile, (int64_t)a.N - r0);
    for (int i = threadIdx.x; i < kZsScanTile; i += kThreads) t[i] = i < n ? (uint32_t)a.cnt[r0 + i] : 0u;
    __syncthreads();
    zs_scan_array(t, kZsScanTile, s_warp);
    for (int i = threadIdx.x; i < n; i += kThreads) a.zrowptr[r0 + i] = (int32_t)t[i];
    if (threadIdx.x == 0) a.tile_sum[blockIdx.x] = t[kZsScanTile];
}

__global__ void __launch_bounds__(kThreads) k_zs_scan_top(const __grid_constant__ SparseArgs a, int tiles) {
    __shared__ uint32_t s_warp[kWarps];
    uint32_t run = 0;
    for (int b = 0; b < tiles; b += kThreads) {
        const int i = b + threadIdx.x;
        const uint32_t v = i < tiles ? a.tile_sum[i] : 0u;
        uint32_t tot;
        const uint32_t x = zs_block_scan(v, s_warp, tot);
        if (i < tiles) a.tile_sum[i] = run + x;
        run += tot;
    }
    if (threadIdx.x == 0) {
        a.tile_sum[tiles] = run;
        a.zrowptr[a.N] = (int32_t)run;
        if ((int64_t)run > a.zcap) atomicOr(a.status, kStInternal);
    }
}

// ---- k_zs_write: one warp per row -------------------------------------------------------
__global__ void __launch_bounds__(kThreads) k_zs_write(const __grid_constant__ SparseArgs a) {
    const int lane = threadIdx.x & 31;
    const bool lap = (a.flags & kOptLap) != 0, cor = (a.flags & kOptCor) != 0;
    for (int64_t r = ((int64_t)blockIdx.x * kThreads + threadIdx.x) >> 5; r < a.N;
         r += ((int64_t)gridDim.x * kThreads) >> 5) {
        const int32_t z0 = __ldcg(a.zrowptr + r) + (int32_t)__ldcg(a.tile_sum + (r / kZsScanTile));
        const int n = __ldcg(a.cnt + r);
        const int64_t base = (int64_t)__ldg(a.rowptr + r) + r;
        const float dv = lap ? __ldg(a.dinv + r) : 1.0f;
        const bool fits = (int64_t)z0 + n <= a.zcap;
        float ss = 0.0f;
        for (int t = lane; t < n; t += 32) {
            const int4 q = __ldcg(&a.runs_a[base + t]);
            const float v = (__int_as_float(q.y) + __int_as_float(q.z)) * dv;
            ss += v * v;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
        const float sc = (cor && ss > 0.0f) ? 1.0f / sqrtf(ss) : 1.0f;
        if (fits)
            for (int t = lane; t < n; t += 32) {
                const int4 q = __ldcg(&a.runs_a[base + t]);
                a.zcol[z0 + t] = q.x;
                a.zval[z0 + t] = (__int_as_float(q.y) + __int_as_float(q.z)) * dv * sc;
            }
        __syncwarp();
        if (lane == 0) {
            a.zrowptr[r] = z0;
            if (!fits) atomicOr(a.status, kStInternal);
        }
    }
}

}  // namespace


cudaError_t configure_sparse_kernels() {
    cudaError_t e = cudaFuncSetAttribute(k_zs_rows, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sizeof(ZsRowsSmem));
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_zs_long_sort, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sizeof(ZsLongSortSmem));
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_zs_long_merge, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)sizeof(ZsLongMergeSmem));
}

int sparse_scan_tiles(int32_t N) { return (int)(((int64_t)N + kZsScanTile - 1) / kZsScanTile); }
int64_t sparse_long_cap(int64_t E) { return E / (kZsWin + 1) + 1; }
int64_t sparse_windows(int64_t E) { return E / kZsWin + 1; }
int64_t sparse_chunk_cap(int64_t E) { return (E + sparse_long_cap(E)) / kZsChunk + sparse_long_cap(E) + 1; }

cudaError_t launch_sparse(const SparseArgs &a, int sms, cudaStream_t st) {
    if (a.N <= 0) return cudaSuccess;
    const int64_t windows = a.E / kZsWin + 1;
    k_zs_wstart<<<(unsigned)std::min<int64_t>(((int64_t)a.N + kThreads) / kThreads, (int64_t)sms * 16), kThreads, 0,
                  st>>>(a, (int)windows);
    k_zs_rows<<<(unsigned)windows, kThreads, sizeof(ZsRowsSmem), st>>>(a);
    k_zs_long_plan<<<1, kThreads, 0, st>>>(a);
    k_zs_long_sort<<<3 * sms, kThreads, sizeof(ZsLongSortSmem), st>>>(a);
    k_zs_long_merge<<<2 * sms, kThreads, sizeof(ZsLongMergeSmem), st>>>(a);
    const int tiles = sparse_scan_tiles(a.N);
    k_zs_scan_tiles<<<tiles, kThreads, 0, st>>>(a);
    k_zs_scan_top<<<1, kThreads, 0, st>>>(a, tiles);
    const int64_t warps = a.N;  // one warp per row
    const int blocks = (int)std::min<int64_t>((warps + kWarps - 1) / kWarps, (int64_t)1 << 30);
    k_zs_write<<<blocks, kThreads, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace gee
