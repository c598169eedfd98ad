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
//   k_zs_rows   one CTA per window of kZsWin CSR positions takes the rows that start in
//               it and have at most kZsWin entries (at most 3 kZsWin entries with the
//               augmentation terms): it sorts the entries by (row, class, position) in
//               shared memory (bitonic), sums each (row, class) run with a segmented scan
//               (a fixed tree per window, so the bits are reproducible), and writes each
//               row's runs to its own slice of the run buffer, at rowptr[i] + i.  Empty
//               rows get their augmentation term; longer rows are listed.
//   k_zs_long   one CTA per listed row: chunks of kZsChunk entries are sorted and summed
//               the same way, and merged into the row's sorted run list in chunk order
//               (sums with two-sum compensation).
//   k_zs_scan*  exclusive scan of the per-row run counts -> zrowptr.
//   k_zs_write  one warp per row: D_ii^-1/2, the row norm, and the stores.
#include "gee_internal.cuh"
#include "gee_sparse.cuh"

#include <algorithm>

namespace gee {
namespace {

constexpr int kZsWin = 1024;                  // window of CSR positions per k_zs_rows CTA
constexpr int kZsTile = 4096;                 // entries a window can hold (<= 3 kZsWin - 1)
constexpr int kZsChunk = 2048;                // entries per chunk of a long row
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

// Exclusive scan of n <= 16 * 256 flags in place (t[0..n) -> prefix; t[n] = total).
__device__ void zs_scan_array(uint32_t *t, int n, uint32_t *s_warp) {
    constexpr int kPer = 16;
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

// ---- k_zs_rows ----------------------------------------------------------------------------
struct ZsRowsSmem {
    uint64_t key[kZsTile];
    float val[kZsTile];
    float v2[kZsTile];
    uint32_t t[kZsTile + 1];      // tail flags, then their exclusive scan
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
    const int64_t w0 = (int64_t)blockIdx.x * kZsWin, w1 = w0 + kZsWin;
    uint32_t err = 0;
    if (tid < 2) {  // rows [ra, rb): the first rows with rowptr >= w0 and >= w1
        const int64_t target = tid == 0 ? w0 : w1;
        int lo = 0, hi = a.N;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if ((int64_t)__ldg(a.rowptr + mid) < target) lo = mid + 1;
            else hi = mid;
        }
        S.s_range[tid] = lo;
    }
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
        int n2 = 32;
        while (n2 < ne) n2 <<= 1;
        for (int i = ne + tid; i < n2; i += kThreads) {
            S.key[i] = kZsPad;
            S.val[i] = 0.0f;
        }
        // ---- load: one warp per row, lanes over its entries (and its augmentation term)
        for (int mi = warp; mi < nm; mi += kWarps) {
            const int r = S.rowid[mi];
            const int64_t p0 = __ldg(a.rowptr + r);
            const int o = (int)S.roff[mi];
            const int tot = (int)S.roff[mi + 1] - o;
            const int len = (int)(__ldg(a.rowptr + r + 1) - p0);
            for (int e = lane; e < tot; e += 32) {
                uint32_t cls;
                float v;
                if (e < len) {
                    const int j = min(max(__ldg(a.col + p0 + e), 0), a.N - 1);
                    const int yj = __ldg(a.y + j);
                    cls = (yj >= 0 && yj < a.K) ? (uint32_t)yj : kZsNoClass;
                    v = (a.val ? __ldg(a.val + p0 + e) : 1.0f) * node_s(a, j);
                } else {  // the augmentation term, after the row's entries
                    cls = (uint32_t)__ldg(a.y + r);
                    v = node_s(a, r);
                }
                S.key[o + e] = ((uint64_t)mi << 33) | ((uint64_t)cls << 12) | (uint64_t)e;
                S.val[o + e] = v;
            }
        }
        __syncthreads();
        zs_sort(S.key, S.val, n2);
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

// ---- k_zs_long ----------------------------------------------------------------------------
struct ZsLongSmem {
    uint64_t key[kZsChunk];
    float val[kZsChunk];
    float v2[kZsChunk];
    uint32_t t[kZsChunk + 1];     // tail flags / scan, then unmatched flags / scan
    uint8_t f[kZsChunk], f2[kZsChunk];
    int32_t pc[kZsChunk];         // the chunk's runs: class, sum
    float ps[kZsChunk];
    int32_t lba[kZsChunk];        // for each run: the runs of the list with a smaller class
    uint32_t s_warp[kWarps];
};

__device__ __forceinline__ int lower_bound_runs(const int4 *A, int n, int c) {
    int lo = 0, hi = n;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (__ldcg(&A[mid].x) < c) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

__global__ void __launch_bounds__(kThreads) k_zs_long(const __grid_constant__ SparseArgs a) {
    extern __shared__ __align__(16) unsigned char zs_smem[];
    ZsLongSmem &S = *reinterpret_cast<ZsLongSmem *>(zs_smem);
    const int tid = threadIdx.x;
    const bool aug = (a.flags & kOptAug) != 0;
    const uint32_t nlong = min(__ldcg(a.long_count), a.long_cap);
    uint32_t err = 0;
    for (uint32_t li = blockIdx.x; li < nlong; li += gridDim.x) {
        const int r = min(max(__ldcg(a.long_list + li), 0), a.N - 1);
        const int64_t p0 = __ldg(a.rowptr + r);
        const int len = (int)(__ldg(a.rowptr + r + 1) - p0);
        const int yi = __ldg(a.y + r);
        const bool own = aug && yi >= 0 && yi < a.K;
        const int T = len + (own ? 1 : 0);
        int4 *cur = a.runs_a + p0 + r, *nxt = a.runs_b + p0 + r;
        int na = 0;
        for (int c0 = 0; c0 < T; c0 += kZsChunk) {
            const int nc = min(kZsChunk, T - c0);
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
                        k = ((uint64_t)yi << 32) | (uint64_t)e;
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
            zs_scan_array(S.t, n2, S.s_warp);
            const int np = (int)S.t[n2];
            for (int i = tid; i < n2; i += kThreads) {
                const uint64_t k = S.key[i];
                if (k != kZsPad && (i == n2 - 1 || (S.key[i + 1] >> 32) != (k >> 32))) {
                    S.pc[S.t[i]] = (int)(k >> 32);
                    S.ps[S.t[i]] = S.val[i];
                }
            }
            __syncthreads();
            // ---- merge the chunk's runs into the row's list (classes ascending); a class in
            // both keeps its place in the list and adds the chunk's sum after the earlier ones
            for (int t = tid; t < np; t += kThreads) {
                const int lb = lower_bound_runs(cur, na, S.pc[t]);
                S.lba[t] = lb;
                S.t[t] = (lb < na && __ldcg(&cur[lb].x) == S.pc[t]) ? 0u : 1u;  // unmatched
            }
            __syncthreads();
            zs_scan_array(S.t, np, S.s_warp);
            const int nu = (int)S.t[np];
            for (int i = tid; i < na; i += kThreads) {
                const int4 ai = __ldcg(&cur[i]);
                int lo = 0, hi = np;  // chunk runs with a smaller class
                while (lo < hi) {
                    const int mid = (lo + hi) >> 1;
                    if (S.pc[mid] < ai.x) lo = mid + 1;
                    else hi = mid;
                }
                float s = __int_as_float(ai.y), comp = __int_as_float(ai.z);
                if (lo < np && S.pc[lo] == ai.x) {
                    const float2 q = two_sum2(s, S.ps[lo]);
                    s = q.x;
                    comp += q.y;
                }
                nxt[i + (int)S.t[lo]] = make_int4(ai.x, __float_as_int(s), __float_as_int(comp), 0);
            }
            for (int t = tid; t < np; t += kThreads)
                if (S.t[t + 1] != S.t[t]) nxt[S.lba[t] + (int)S.t[t]] = make_int4(S.pc[t], __float_as_int(S.ps[t]), 0, 0);
            __syncthreads();
            na += nu;
            int4 *tmp = cur;
            cur = nxt;
            nxt = tmp;
        }
        if (cur != a.runs_a + p0 + r) {
            for (int i = tid; i < na; i += kThreads) a.runs_a[p0 + r + i] = __ldcg(&cur[i]);
        }
        if (tid == 0) a.cnt[r] = na;
        __syncthreads();
    }
    if (err) atomicOr(a.status, err);
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

size_t sparse_smem_rows() { return sizeof(ZsRowsSmem); }
size_t sparse_smem_long() { return sizeof(ZsLongSmem); }

cudaError_t configure_sparse_kernels() {
    cudaError_t e = cudaFuncSetAttribute(k_zs_rows, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sizeof(ZsRowsSmem));
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_zs_long, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(ZsLongSmem));
}

int sparse_scan_tiles(int32_t N) { return (int)(((int64_t)N + kZsScanTile - 1) / kZsScanTile); }
int64_t sparse_long_cap(int64_t E) { return E / (kZsWin + 1) + 1; }

cudaError_t launch_sparse(const SparseArgs &a, int sms, cudaStream_t st) {
    if (a.N <= 0) return cudaSuccess;
    const int64_t windows = a.E / kZsWin + 1;
    k_zs_rows<<<(unsigned)windows, kThreads, sizeof(ZsRowsSmem), st>>>(a);
    k_zs_long<<<2 * sms, kThreads, sizeof(ZsLongSmem), st>>>(a);
    const int tiles = sparse_scan_tiles(a.N);
    k_zs_scan_tiles<<<tiles, kThreads, 0, st>>>(a);
    k_zs_scan_top<<<1, kThreads, 0, st>>>(a, tiles);
    const int64_t warps = a.N;
    const int blocks = (int)std::min<int64_t>((warps + kWarps - 1) / kWarps, (int64_t)sms * 8);
    k_zs_write<<<blocks, kThreads, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace gee
