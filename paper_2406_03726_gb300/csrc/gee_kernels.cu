// Device kernels of the sparse GEE path (Qin & Shen, Section 2 Eq. 1, Table 1, Section 3).
//
//   k_prep     label counts n_k (definition of W), input checks, per-range histograms of
//              the first radix digit of the source ids
//   k_offsets  per-range bucket offsets of a radix pass (prefix over digits and ranges)
//   k_scatter  one stable LSD radix pass over the edges, keyed by source id, one CTA per
//              range with TMA-staged tiles; the final pass writes the CSR (col_indices,
//              data)
//   k_count    (graphs with more than 2^8 nodes) final-digit histograms of the packed
//              first-pass output and the row lengths
//   k_rowscan  index_pointers from the last pass's bucket offsets and the row lengths;
//              unweighted degrees D_ii and the node table s_j = D_jj^-1/2 / n_{y_j};
//              hub-row list and (last CTA) the chunk offsets of the split rows
//   k_wdeg     weighted degrees: FP32 compensated sums on light rows, FP64 chunk
//              partials merged in FP64 on hub rows; then D^-1/2 and the node table
//   k_spmm     Z = D^-1/2 (A + I) D^-1/2 W as a label-gather over the CSR rows, with the
//              augmentation term, the D_ii^-1/2 scaling and the row 2-norm (correlation)
//              fused into the epilogue; hub rows are split across CTAs and merged with
//              two-sum compensation by the last CTA to finish
//
// Every copy wait is bounded (kSpinLimit) and records kStTimeout instead of hanging; a failed
// internal invariant records kStInternal;
// every global index derived from data is range-checked, so bad input cannot make a
// kernel touch memory outside its buffers.
#include "gee_internal.cuh"

#include <cuda_runtime.h>
#include <algorithm>
#include <cstdint>

namespace gee {

// ------------------------------------------------------------------------------------
// small device helpers

__host__ __device__ __forceinline__ int64_t min64(int64_t a, int64_t b) { return a < b ? a : b; }

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// streaming loads of data read exactly once (no L1 allocation)
__device__ __forceinline__ int32_t ld_stream(const int32_t *p) {
    int32_t v;
    asm("ld.global.nc.L1::no_allocate.s32 %0, [%1];" : "=r"(v) : "l"(p));
    return v;
}
__device__ __forceinline__ uint32_t ld_stream(const uint32_t *p) {
    uint32_t v;
    asm("ld.global.nc.L1::no_allocate.u32 %0, [%1];" : "=r"(v) : "l"(p));
    return v;
}
__device__ __forceinline__ float ld_stream(const float *p) {
    float v;
    asm("ld.global.nc.L1::no_allocate.f32 %0, [%1];" : "=f"(v) : "l"(p));
    return v;
}
__device__ __forceinline__ int4 ld_stream4(const int32_t *p) {
    int4 v;
    asm("ld.global.nc.L1::no_allocate.v4.s32 {%0,%1,%2,%3}, [%4];"
        : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
        : "l"(p));
    return v;
}
__device__ __forceinline__ float4 ld_stream4(const float *p) {
    float4 v;
    asm("ld.global.nc.L1::no_allocate.v4.f32 {%0,%1,%2,%3}, [%4];"
        : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
        : "l"(p));
    return v;
}

__device__ __forceinline__ int find_graph(const int32_t *prefix, int G, int item) {
    int lo = 0, hi = G;  // largest g with prefix[g] <= item
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (__ldg(prefix + mid) <= item) lo = mid;
        else hi = mid;
    }
    return lo;
}

// Copy graph g's descriptor to `dst` (shared memory), 4 bytes per lane of the calling warp:
// from the batch's array in global memory, or for one graph from the kernel parameter
// (every kernel takes its Ctx as a __grid_constant__ parameter, so it is read in place).
// A one-thread struct copy of the ~400-byte descriptor spilled registers in every kernel.
__device__ __forceinline__ void copy_desc(const Ctx &c, int g, GraphDesc *dst, int lane) {
    constexpr int kWords = (int)(sizeof(GraphDesc) / 4);
    static_assert(sizeof(GraphDesc) % 4 == 0, "descriptor words");
    uint32_t *d = reinterpret_cast<uint32_t *>(dst);
    if (c.G > 1) {
        const uint32_t *src = reinterpret_cast<const uint32_t *>(c.graphs + g);
        for (int i = lane; i < kWords; i += 32) d[i] = __ldg(src + i);
    } else {
        const uint32_t *src = reinterpret_cast<const uint32_t *>(&c.g0);
        for (int i = lane; i < kWords; i += 32) d[i] = src[i];
    }
}

// Copy graph g's descriptor to shared memory (warp 0 resolves the item) and return the
// item's index local to that graph.  Contains __syncthreads.
__device__ __forceinline__ int load_desc(const Ctx &c, int item, GraphDesc *sg, int *sl,
                                         const int32_t *prefix) {
    if (threadIdx.x < 32) {
        int g = 0, base = 0;
        if (c.G > 1) {
            g = find_graph(prefix, c.G, item);
            base = __ldg(prefix + g);
        }
        copy_desc(c, g, sg, threadIdx.x);
        if (threadIdx.x == 0) {
            sl[0] = item - base;
            sl[1] = g;
        }
    }
    __syncthreads();
    return sl[0];
}

__device__ __forceinline__ void load_desc_idx(const Ctx &c, int g, GraphDesc *sg) {
    if (threadIdx.x < 32) copy_desc(c, g, sg, threadIdx.x);
    __syncthreads();
}

// Exclusive scan over the 256 threads of a CTA; returns the thread's prefix and the total.
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t *s_warp, uint32_t &total) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t t = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += t;
    }
    if (lane == 31) s_warp[w] = x;
    __syncthreads();
    uint32_t before = 0, tot = 0;
#pragma unroll
    for (int i = 0; i < kWarps; ++i) {
        uint32_t s = s_warp[i];
        before += (i < w) ? s : 0u;
        tot += s;
    }
    __syncthreads();
    total = tot;
    return before + x - v;
}

// Error-free transformation: s + e == a + b exactly (Knuth's two-sum).
__device__ __forceinline__ float two_sum(float a, float b, float &e) {
    float s = a + b;
    float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
    return s;
}

// log2 of the lanes of a row of `len` entries: the smallest c with 8 * 2^c >= len, c <= 5
__device__ __forceinline__ uint32_t lanes_log2_for(int len) {
    if (len <= 8) return 0u;
    return (uint32_t)min(5, 32 - __clz(len - 1) - 3);
}

// Length bucket of a light row of a K > 8 graph that is taken one lane per row: 0 for at
// most 8 entries, b for (4 << b, 8 << b], capped at the last one-lane bucket.
__device__ __forceinline__ int bucket_of(int len) {
    if (len <= 8) return 0;
    return min(kWarpBucket - 1, 32 - __clz(len - 1) - 3);
}

__device__ __forceinline__ bool finite_f(float x) { return (__float_as_uint(x) & 0x7f800000u) != 0x7f800000u; }

// ------------------------------------------------------------------------------------
// TMA bulk copies (global -> shared memory, completion counted on an mbarrier)

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait for the phase `parity` of an mbarrier; false after ~1 s.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
    for (int i = 0; i < kSpinLimit; ++i) {
        if (mbar_try_wait(bar, parity)) return true;
        if (i > 16) __nanosleep(64);
    }
    return false;
}

__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// ------------------------------------------------------------------------------------
// k_prep: histograms of source-id digits (edge tiles), class sizes n_k (node tiles)

// ------------------------------------------------------------------------------------
// CSR build: stable LSD radix sort of the edges by source id (Section 3 CSR, rows in
// input order).  A graph's edges are cut into ranges of range_tiles x 4096 edges.
//
//   k_prep       per range: histogram of the first-pass digit of the source ids
//                (low lbits for 2-pass graphs, the whole id for graphs with <= 2^8
//                nodes); per node tile: class sizes n_k and label checks
//   k_offsets    per digit: exclusive prefix over (digit, range) -> the bucket offset
//                at which each range starts writing each digit
//   k_scatter    one CTA per range scatters its tiles in order from those offsets:
//                first pass -> packed ((src >> lbits) << nbits | dst) + weight,
//                final pass -> col / val of the CSR
//   k_count      (2-pass graphs) per range of the packed array: histogram of the
//                final-pass digit, and the exact row lengths rowcnt
// No CTA ever waits for another: the offsets are known before a range is scattered.

constexpr int kPrivDigits = 512;  // digit counts up to this get one private histogram per warp

__device__ __forceinline__ int64_t range_begin(const GraphDesc &g, int r) {
    return (int64_t)r * g.range_tiles * kSortTile;
}
__device__ __forceinline__ int range_len(const GraphDesc &g, int r) {
    const int64_t n = min64((int64_t)g.range_tiles * kSortTile, g.E - range_begin(g, r));
    return n > 0 ? (int)n : 0;
}

// With GEE_SYMMETRIZE the ranges cut the virtual list of 2 Ein entries in which input
// edge e gives entry 2e (i -> j) and entry 2e + 1 (j -> i): the CSR keeps a row's entries
// in that order.  vshift is 1 then: virtual entry v reads input edge v >> 1, so a range or
// tile reads its input slice once for both directions.
__device__ __forceinline__ int vshift(const GraphDesc &g) { return g.sym ? 1 : 0; }

// Stream the ids [0, n) of p through f(value), CTA-wide, through shared memory: stages of
// 2048 ids are filled by TMA bulk copies, kIdStages of them in flight, and each thread
// then takes 8 ids of a stage as two 16-byte reads.  The head up to the first 16-byte
// boundary and the last n mod 4 ids are read directly.  Every thread of the CTA calls it
// with the same arguments; `parity` (one bit per stage barrier) is kept by the caller.
constexpr int kIdStages = 4;
constexpr int kIdStage = 2048;
constexpr size_t kIdRingBytes = (size_t)kIdStages * kIdStage * 4;

struct IdRing {
    int32_t *buf;   // [kIdStages][kIdStage], dynamic shared memory
    uint64_t *bar;  // [kIdStages] mbarriers, initialised with count 1
};

__device__ __forceinline__ void id_ring_init(const IdRing &ring) {
    if (threadIdx.x == 0)
        for (int s = 0; s < kIdStages; ++s) mbar_init(&ring.bar[s], 1);
}

template <class F>
__device__ __forceinline__ void stream_ids_staged(const int32_t *p, int n, const IdRing &ring, uint32_t &parity,
                                                  uint32_t &err, F &&f) {
    const int tid = threadIdx.x;
    int head = (int)(((16u - (reinterpret_cast<uintptr_t>(p) & 15u)) & 15u) >> 2);
    if ((reinterpret_cast<uintptr_t>(p) & 3u) != 0) head = n;  // not even 4-byte aligned: all direct
    head = min(head, n);
    if (tid < head) f(ld_stream(p + tid));
    p += head;
    n -= head;
    const int nb = n & ~3;
    const int nst = (nb + kIdStage - 1) / kIdStage;
    auto issue = [&](int s) {
        const int slot = s % kIdStages;
        const uint32_t bytes = (uint32_t)min(kIdStage, nb - s * kIdStage) * 4u;
        mbar_expect_tx(&ring.bar[slot], bytes);
        bulk_g2s(ring.buf + slot * kIdStage, p + (size_t)s * kIdStage, bytes, &ring.bar[slot]);
    };
    __syncthreads();  // earlier reads of the ring are done
    if (tid == 0 && nst > 0) {
        fence_proxy_async();
        for (int s = 0; s < min(kIdStages, nst); ++s) issue(s);
    }
    for (int s = 0; s < nst; ++s) {
        const int slot = s % kIdStages;
        const int cnt4 = min(kIdStage, nb - s * kIdStage) >> 2;
        if (!mbar_wait(&ring.bar[slot], (parity >> slot) & 1u)) err |= kStTimeout;
        parity ^= 1u << slot;
        const int4 *v = reinterpret_cast<const int4 *>(ring.buf + slot * kIdStage);
        for (int i = tid; i < cnt4; i += kThreads) {
            const int4 x = v[i];
            f(x.x);
            f(x.y);
            f(x.z);
            f(x.w);
        }
        __syncthreads();  // the stage is consumed
        if (tid == 0 && s + kIdStages < nst) {
            fence_proxy_async();
            issue(s + kIdStages);
        }
    }
    if (tid < n - nb) f(ld_stream(p + nb + tid));
}

__global__ void __launch_bounds__(kThreads) k_prep(const __grid_constant__ Ctx c) {
    __shared__ GraphDesc sg;
    __shared__ int sl[2];
    __shared__ uint32_t h[kWarps * kPrivDigits];
    __shared__ uint32_t s_err;
    __shared__ __align__(8) uint64_t bars[kIdStages];
    extern __shared__ __align__(128) int32_t ringbuf[];
    const IdRing ring{ringbuf, bars};
    const int tid = threadIdx.x, warp = tid >> 5;
    id_ring_init(ring);
    const int t = load_desc(c, blockIdx.x, &sg, sl, c.prefix);
    if (tid == 0) s_err = 0;
    uint32_t err = 0;
    if (t < sg.ranges) {
        const int b1 = first_bits(sg);
        const int D = 1 << b1;
        const int str = (D <= kPrivDigits) ? D : 0;  // private per-warp histograms when they fit
        const int nh = str ? kWarps * D : D;
        for (int i = tid; i < nh; i += kThreads) h[i] = 0;
        __syncthreads();
        uint32_t *hw = h + warp * str;
        const uint32_t N = (uint32_t)sg.N, R0 = (uint32_t)sg.row0;
        const uint32_t m = (1u << b1) - 1u;
        uint32_t parity = 0;
        const int sh = vshift(sg);
        const int64_t e0 = range_begin(sg, t) >> sh;  // the range's slice of the input
        const int rn = range_len(sg, t) >> sh;
        auto count = [&](int v) {
            v = (int)((uint32_t)v - R0);
            if ((uint32_t)v >= N) {
                err |= kStIndex;
                v = 0;
            }
            atomicAdd(&hw[(uint32_t)v & m], 1u);
        };
        stream_ids_staged(sg.src + e0, rn, ring, parity, err, count);
        if (sh) {  // the reverse entries' rows are the targets
            __syncthreads();  // the ring is free again
            stream_ids_staged(sg.dst + e0, rn, ring, parity, err, count);
        }
        __syncthreads();
        uint32_t *out = sg.cnt1 + ((size_t)t << b1);
        for (int d = tid; d < D; d += kThreads) {
            uint32_t v = 0;
            if (str)
                for (int w = 0; w < kWarps; ++w) v += h[w * D + d];
            else
                v = h[d];
            out[d] = v;
            if (v) atomicAdd(&sg.hist1[((size_t)(t % kHistCopies) << b1) + d], v);
        }
    } else {
        const int64_t n0 = (int64_t)(t - sg.ranges) * kPrepTile;
        const int n = (int)min64(kPrepTile, (int64_t)sg.N - n0);
        const int K = sg.K;
        // class sizes in shared memory, or straight into n_k when the classes outnumber
        // the histogram (sparse Z with many classes)
        const bool local = K <= kWarps * kPrivDigits;
        if (local)
            for (int i = tid; i < K; i += kThreads) h[i] = 0;
        __syncthreads();
        for (int i = tid; i < n; i += kThreads) {
            int yv = __ldg(sg.y + n0 + i);
            if (yv < -1 || yv >= K) err |= kStLabel;
            else if (yv >= 0) atomicAdd(local ? &h[yv] : reinterpret_cast<unsigned *>(sg.nk) + yv, 1u);
        }
        __syncthreads();
        if (local)
            for (int i = tid; i < K; i += kThreads)
                if (h[i]) atomicAdd(reinterpret_cast<unsigned *>(sg.nk) + i, h[i]);
    }
    if (err) atomicOr(&s_err, err);
    __syncthreads();
    if (tid == 0 && s_err) atomicOr(sg.status, s_err);
}

// k_offsets: for a block of 32 digits, rewrite cnt[r][d] (counts) as the position where
// range r writes its first element of digit d: dbase[d] + sum_{r' < r} cnt[r'][d], with
// dbase the exclusive prefix over digits of the totals.  1024 threads: lane = digit of
// the block, each of the 32 warps owns a slice of the ranges (8 loads in flight).
constexpr int kOffThreads = 1024;
constexpr int kOffWarps = kOffThreads / 32;

template <bool SECOND>
__global__ void __launch_bounds__(kOffThreads) k_offsets(const __grid_constant__ Ctx c) {
    __shared__ GraphDesc sg;
    __shared__ int sl[2];
    __shared__ uint32_t s_red[kOffWarps];
    __shared__ uint32_t csum[kOffWarps][33];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int b = load_desc(c, blockIdx.x, &sg, sl, c.prefix);
    const int bits = SECOND ? sg.fbits : first_bits(sg);
    const int D = 1 << bits;
    uint32_t *cnt = SECOND ? sg.cnt2 : sg.cnt1;
    const uint32_t *tot = SECOND ? sg.hist2 : sg.hist1;
    const int d0 = 32 * b, d = d0 + lane;
    const int R = sg.ranges;
    const int chunk = (R + kOffWarps - 1) / kOffWarps;
    const int r0 = min(R, warp * chunk), r1 = min(R, r0 + chunk);
    // this warp's counts, kept in registers between the two passes when they fit
    constexpr int kHold = 24;
    const bool hold = chunk <= kHold;
    uint32_t held[kHold];
    uint32_t s = 0;
    if (hold && d < D) {
#pragma unroll
        for (int q = 0; q < kHold; ++q) held[q] = (r0 + q < r1) ? __ldcg(cnt + ((size_t)(r0 + q) << bits) + d) : 0u;
    }
    // sum of the totals below this digit block
    uint32_t part = 0;
    for (int i = tid; i < d0 * kHistCopies; i += kOffThreads) {
        const int cpy = i / d0, dd = i - cpy * d0;
        part += __ldcg(tot + ((size_t)cpy << bits) + dd);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    if (lane == 0) s_red[warp] = part;
    uint32_t td = 0;
    if (d < D)
#pragma unroll
        for (int cpy = 0; cpy < kHistCopies; ++cpy) td += __ldcg(tot + ((size_t)cpy << bits) + d);
    if (d < D) {
        if (hold) {
#pragma unroll
            for (int q = 0; q < kHold; ++q) s += held[q];
        } else {
            int r = r0;
            for (; r + 8 <= r1; r += 8) {
                uint32_t a[8];
#pragma unroll
                for (int q = 0; q < 8; ++q) a[q] = __ldcg(cnt + ((size_t)(r + q) << bits) + d);
#pragma unroll
                for (int q = 0; q < 8; ++q) s += a[q];
            }
            for (; r < r1; ++r) s += __ldcg(cnt + ((size_t)r << bits) + d);
        }
    }
    csum[warp][lane] = s;
    __syncthreads();
    uint32_t below = 0;
    for (int w = 0; w < kOffWarps; ++w) below += s_red[w];
    uint32_t x = td;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    uint32_t run = below + x - td;  // bucket base of digit d
    for (int w = 0; w < warp; ++w) run += csum[w][lane];
    if (d < D) {
        if (hold) {
#pragma unroll
            for (int q = 0; q < kHold; ++q)
                if (r0 + q < r1) {
                    cnt[((size_t)(r0 + q) << bits) + d] = run;
                    run += held[q];
                }
        } else {
            int r = r0;
            for (; r + 8 <= r1; r += 8) {
                uint32_t a[8];
#pragma unroll
                for (int q = 0; q < 8; ++q) a[q] = __ldcg(cnt + ((size_t)(r + q) << bits) + d);
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    cnt[((size_t)(r + q) << bits) + d] = run;
                    run += a[q];
                }
            }
            for (; r < r1; ++r) {
                uint32_t *p = cnt + ((size_t)r << bits) + d;
                const uint32_t v = __ldcg(p);
                *p = run;
                run += v;
            }
        }
        if (!SECOND && sg.npass == 1 && warp == 0 && d < sg.N) sg.rowcnt[d] = (int32_t)td;  // digit = row
    }
}

// ------------------------------------------------------------------------------------
// k_scatter: one CTA scatters one range, tile by tile, in order.
//
//   FINAL = false  first pass of a 2-pass graph: digit = low lbits of the source id,
//                  edge list -> packed + weight
//   FINAL = true   last pass: 1-pass graphs read the edge list (digit = source id) with
//                  the cnt1 offsets, 2-pass graphs read the packed array (digit = high
//                  bits) with the cnt2 offsets; writes col / val
//
// Tiles of 2048 edges, 8 per thread.  While a tile is ranked and scattered, the next tile
// of the range streams into shared memory by TMA bulk copies.  Warp w ranks tile
// elements [256 w, 256 w + 256), item i of lane l being element 256 w + 32 i + l.  The
// lanes of a warp holding the same digit are found through a per-warp table of peer
// masks: every lane ORs its bit into the entry of its digit, reads the entry back, and
// the lowest lane of the group clears it again (digits above 256 share entries, and one
// ballot per remaining digit bit separates them).  A per-warp counter per digit then
// gives each element its rank among the equal digits before it in input order, so the
// pass is stable.
//
// Shared memory (dynamic, sized by the digit count D), every part a multiple of 16 bytes:
//   stage  3 streams x 2048 words (src|packed, dst, weight): TMA destination
//   tile   the tile sorted by digit: global position, payload, weight (3 x 2048 words)
//   wcnt   [kWarps][D] u16 per-warp digit counters (apart from the tile for D <= 512,
//          else sharing its space)
//   tstart, dglob, run   [D] u32: tile-local start, tile -> global shift, range offset
//   bins   [kWarps][min(D, 256)] u32 peer masks (zero between items)

constexpr int kStreamWords = kSortTile;                       // one stream = 2048 words
constexpr size_t kStageBytes = (size_t)3 * kStreamWords * 4;  // src|tmpk, dst, w|tmpw
constexpr size_t kTileBytes = (size_t)3 * kSortTile * 4;      // sorted pos, payload, weight
constexpr int kSepDigits = 512;                               // wcnt apart from the tile up to here
constexpr int kBinDigits = 256;                               // peer-mask entries per warp
constexpr int kScatterCols = kMaxDigits / 2 / kThreads;       // digit pairs per thread, at most
static_assert(kScatterCols * kWarps <= 32, "column-warp totals are scanned by one warp");

__host__ __device__ constexpr size_t scatter_wcnt_bytes(int D) { return (size_t)D * kWarps * 2; }
__host__ __device__ constexpr size_t scatter_union_bytes(int D) {
    return D <= kSepDigits ? kTileBytes + ((scatter_wcnt_bytes(D) + 15) & ~(size_t)15)
                           : (scatter_wcnt_bytes(D) > kTileBytes ? scatter_wcnt_bytes(D) : kTileBytes);
}
__host__ __device__ constexpr size_t scatter_smem_bytes(int D) {
    return kStageBytes + scatter_union_bytes(D) + (size_t)3 * D * 4 +
           (size_t)kWarps * (D < kBinDigits ? D : kBinDigits) * 4;
}

template <bool FINAL>
// Stage n entries of the input from e0 (COO passes: src, dst and w; the final pass of a
// 2-pass graph: the packed keys and weights) into shared memory, a multiple of 4 of them.
__device__ __forceinline__ int scatter_issue_stage(const GraphDesc &g, int64_t e0, int n, uint32_t *stage,
                                                   uint64_t *bar) {
    const bool coo = !FINAL || g.npass == 1;
    const uint32_t bytes = (uint32_t)(n & ~3) * 4u;
    const void *p0 = coo ? (const void *)(g.src + e0) : (const void *)(g.tmpk + e0);
    const void *p1 = coo ? (const void *)(g.dst + e0) : nullptr;
    const void *p2 = g.w ? (coo ? (const void *)(g.w + e0) : (const void *)(g.tmpw + e0)) : nullptr;
    const bool ok = bytes > 0 && aligned16(p0) && (!p1 || aligned16(p1)) && (!p2 || aligned16(p2));
    if (ok) {
        fence_proxy_async();  // earlier generic reads of the stage precede these async writes
        const uint32_t nstreams = 1u + (p1 ? 1u : 0u) + (p2 ? 1u : 0u);
        mbar_expect_tx(bar, bytes * nstreams);
        bulk_g2s(stage, p0, bytes, bar);
        if (p1) bulk_g2s(stage + kStreamWords, p1, bytes, bar);
        if (p2) bulk_g2s(stage + 2 * kStreamWords, p2, bytes, bar);
    }
    return ok ? 1 : 0;
}

constexpr uint32_t kNoKey = 0xffffffffu;

// One element of a tile -> (digit, payload, weight).  Rows are source ids minus row0;
// rows outside [0, N) count as 0 (k_prep flags them and counts them as 0 too); targets
// outside [0, NC) are flagged and become 0.  Weights are checked by the pass that writes
// the CSR.
template <bool FINAL>
__device__ __forceinline__ void scatter_item(bool coo, bool rev, uint32_t a, uint32_t b, float x, uint32_t N,
                                             uint32_t R0, uint32_t NC, int lb, int nb, uint32_t nmask, uint32_t dmask,
                                             bool has_w, bool lap, uint32_t &key, uint32_t &pay, uint32_t &err) {
    if (coo) {
        const uint32_t s = a - R0 < N ? a - R0 : 0u;
        uint32_t d = b;
        if (d >= NC) {
            err |= kStIndex;
            d = 0;
        }
        if (FINAL) {
            key = s;
            pay = d;
        } else {
            key = s & ((1u << lb) - 1u);
            // the reverse copy of a self-loop is dropped: it keeps its place in the first
            // pass (k_prep counted it) but carries the sentinel, which the later passes skip
            pay = (rev && a == b) ? kSentinel : (((s >> lb) << nb) | d);
        }
    } else if (a == kSentinel) {
        key = kNoKey;  // a dropped element: not ranked, not written
        pay = 0;
    } else {
        key = (a >> nb) & dmask;  // < D for every packed value the first pass writes
        pay = a & nmask;
    }
    if (FINAL && has_w && (!finite_f(x) || (lap && x < 0.0f))) err |= kStWeight;
}

template <bool FINAL>
__global__ void __launch_bounds__(kThreads, 4) k_scatter(const __grid_constant__ Ctx c) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ GraphDesc sg;
    __shared__ int sl[2];
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t s_scan[kScatterCols * kWarps];
    __shared__ uint32_t s_err;
    __shared__ int s_staged;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int r = load_desc(c, blockIdx.x, &sg, sl, c.prefix);
    const bool coo = !FINAL || sg.npass == 1;
    const int bits = FINAL ? sg.fbits : sg.lbits;
    const int D = 1 << bits;
    const int BD = D < kBinDigits ? D : kBinDigits;
    const int bbits = bits < 8 ? bits : 8;
    const uint32_t bmask = (uint32_t)BD - 1u;
    const bool sep = D <= kSepDigits;
    const int nb = sg.pbits, lb = sg.lbits;
    const uint32_t nmask = (1u << nb) - 1u;  // nb <= 21
    const uint32_t R0 = (uint32_t)sg.row0, NC = (uint32_t)sg.ncols;
    const uint32_t dmask = (uint32_t)D - 1u;
    const bool has_w = sg.w != nullptr;
    const bool lap = (sg.flags & kOptLap) != 0;
    const uint32_t N = (uint32_t)sg.N;
    const uint32_t E32 = (uint32_t)sg.E;
    const uint32_t *offs = (FINAL && sg.npass == 2) ? sg.cnt2 : sg.cnt1;

    uint32_t *stage = reinterpret_cast<uint32_t *>(smem);
    unsigned char *uni = smem + kStageBytes;
    uint32_t *spos = reinterpret_cast<uint32_t *>(uni);  // sorted tile
    uint32_t *spay = spos + kSortTile;
    float *sw = reinterpret_cast<float *>(spay + kSortTile);
    uint16_t *wcnt = reinterpret_cast<uint16_t *>(sep ? uni + kTileBytes : uni);  // [kWarps][D]
    uint32_t *tstart = reinterpret_cast<uint32_t *>(uni + scatter_union_bytes(D));
    uint32_t *dglob = tstart + D;
    uint32_t *run = dglob + D;
    uint32_t *bins = run + D;  // [kWarps][BD]
    uint16_t *mycnt = wcnt + warp * D;
    uint32_t *mybins = bins + warp * BD;
    // per-digit work by digit pairs (D >= 2): thread t owns pairs p = t + kThreads j, j <
    // ppt, so a warp's accesses to the per-digit arrays are consecutive words
    const int P = D >> 1;
    const int ppt = (P + kThreads - 1) / kThreads;  // <= kScatterCols
    uint32_t *wc32 = reinterpret_cast<uint32_t *>(wcnt);  // [kWarps][P]: two u16 counters
    uint2 *tstart2 = reinterpret_cast<uint2 *>(tstart);
    uint2 *dglob2 = reinterpret_cast<uint2 *>(dglob);
    uint2 *run2 = reinterpret_cast<uint2 *>(run);
    // virtual entries of the range (a tile is kSortTile of them); with symmetrizing, the
    // COO pass reads input edge v >> 1 for entry v
    const int sh = coo ? vshift(sg) : 0;
    const int64_t r0 = range_begin(sg, r);
    const int rn = range_len(sg, r);
    const int ntiles = (rn + kSortTile - 1) / kSortTile;
    uint32_t err = 0;

    if (tid == 0) {
        s_err = 0;
        mbar_init(&bar, 1);
        s_staged = scatter_issue_stage<FINAL>(sg, r0 >> sh, min(rn, kSortTile) >> sh, stage, &bar);
    }
    for (int i = tid; i < kWarps * BD; i += kThreads) bins[i] = 0u;
    for (int d = tid; d < D; d += kThreads) run[d] = __ldcg(offs + ((size_t)r << bits) + d);
    __syncthreads();
    uint32_t parity = 0;
    const unsigned lt = lanemask_lt();

    for (int ti = 0; ti < ntiles; ++ti) {
        const int64_t e0 = r0 + (int64_t)ti * kSortTile;
        const int n = min(kSortTile, rn - ti * kSortTile);
        const int staged = s_staged;  // written before the last CTA barrier
        if (staged) {
            if (!mbar_wait(&bar, parity)) err |= kStTimeout;
            parity ^= 1u;
        }

        // ---- the 8 elements of this thread (stage, or global for the tail); entry idx of
        // the tile reads input entry idx >> sh, and with symmetrizing the odd entries are
        // the reverse copies (source and target swapped)
        uint32_t key[kSortItems], pay[kSortItems];
        float wv[kSortItems];
        const int wbase = warp * (32 * kSortItems);
        const int64_t ein = e0 >> sh;
        if (staged && n == kSortTile) {
#pragma unroll
            for (int i = 0; i < kSortItems; ++i) {
                const int idx = wbase + i * 32 + lane;
                const int j = idx >> sh;
                const bool rev = (idx & sh) != 0;
                const uint32_t a0 = stage[j];
                const uint32_t b0 = coo ? stage[kStreamWords + j] : 0u;
                wv[i] = has_w ? __uint_as_float(stage[2 * kStreamWords + j]) : 1.0f;
                scatter_item<FINAL>(coo, rev, rev ? b0 : a0, rev ? a0 : b0, wv[i], N, R0, NC, lb, nb, nmask, dmask,
                                    has_w, lap, key[i], pay[i], err);
            }
        } else {
            const int nst = staged ? ((n >> sh) & ~3) : 0;  // staged input entries
#pragma unroll
            for (int i = 0; i < kSortItems; ++i) {
                const int idx = wbase + i * 32 + lane;
                key[i] = kNoKey;
                pay[i] = 0;
                wv[i] = 1.0f;
                if (idx < n) {
                    const int j = idx >> sh;
                    const bool rev = (idx & sh) != 0;
                    uint32_t a, b = 0;
                    float x = 1.0f;
                    if (j < nst) {
                        a = stage[j];
                        if (coo) b = stage[kStreamWords + j];
                        if (has_w) x = __uint_as_float(stage[2 * kStreamWords + j]);
                    } else if (coo) {
                        a = (uint32_t)ld_stream(sg.src + ein + j);
                        b = (uint32_t)ld_stream(sg.dst + ein + j);
                        if (has_w) x = ld_stream(sg.w + ein + j);
                    } else {
                        a = ld_stream(sg.tmpk + ein + j);
                        if (has_w) x = ld_stream(sg.tmpw + ein + j);
                    }
                    wv[i] = x;
                    scatter_item<FINAL>(coo, rev, rev ? b : a, rev ? a : b, x, N, R0, NC, lb, nb, nmask, dmask, has_w,
                                        lap, key[i], pay[i], err);
                }
            }
        }
        __syncthreads();  // A: stage consumed; the previous tile's write-out is done

        // ---- start streaming the next tile of this range
        if (tid == 0 && ti + 1 < ntiles)
            s_staged = scatter_issue_stage<FINAL>(sg, (e0 + kSortTile) >> sh,
                                                  min(kSortTile, rn - (ti + 1) * kSortTile) >> sh, stage, &bar);

        // ---- stable rank within the warp: peer masks, then a per-warp counter per digit
        for (int i = lane; i < D / 2; i += 32) reinterpret_cast<uint32_t *>(mycnt)[i] = 0u;
        __syncwarp();
        uint32_t rank[kSortItems];
#pragma unroll
        for (int i = 0; i < kSortItems; ++i) {
            const uint32_t d = key[i];
            const bool valid = d != kNoKey;
            uint32_t *bin = mybins + (d & bmask);
            if (valid) atomicOr(bin, 1u << lane);
            __syncwarp();
            uint32_t peers = valid ? *bin : 0u;
            for (int b = bbits; b < bits; ++b) {  // digits that share a peer-mask entry
                const bool bit = (d >> b) & 1u;
                const unsigned bal = __ballot_sync(0xffffffffu, bit);
                peers &= bit ? bal : ~bal;
            }
            const uint32_t before = valid ? (uint32_t)mycnt[d] : 0u;
            __syncwarp();
            if (valid && (peers & lt) == 0u) {
                mycnt[d] = (uint16_t)(before + __popc(peers));
                *bin = 0u;
            }
            __syncwarp();
            rank[i] = before + __popc(peers & lt);
        }
        __syncthreads();  // B

        // ---- per digit: warp offsets, tile counts, tile-local starts, global positions.
        // The tile-local starts follow the digit order, which is the order (j, t) of the
        // owned pairs: a warp scan per column j, then a scan of the column-warp totals.
        uint32_t c0[kScatterCols], c1[kScatterCols], xs[kScatterCols];
#pragma unroll
        for (int j = 0; j < kScatterCols; ++j) {
            const int p = tid + j * kThreads;
            uint32_t s0 = 0, s1 = 0;
            if (j < ppt && p < P) {
#pragma unroll
                for (int w = 0; w < kWarps; ++w) {
                    const uint32_t v = wc32[w * P + p];
                    wc32[w * P + p] = s0 | (s1 << 16);  // counts of a tile fit 16 bits
                    s0 += v & 0xffffu;
                    s1 += v >> 16;
                }
            }
            c0[j] = s0;
            c1[j] = s1;
            uint32_t x = s0 + s1;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t t = __shfl_up_sync(0xffffffffu, x, o);
                if (lane >= o) x += t;
            }
            xs[j] = x - s0 - s1;  // exclusive within the warp
            if (lane == 31 && j < ppt) s_scan[j * kWarps + warp] = x;
        }
        __syncthreads();  // S
        uint32_t nranked;  // the tile's ranked elements (dropped ones are not)
        {
            const int ncol = ppt * kWarps;  // <= 32
            const uint32_t v = lane < ncol ? s_scan[lane] : 0u;
            uint32_t x = v;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t t = __shfl_up_sync(0xffffffffu, x, o);
                if (lane >= o) x += t;
            }
            nranked = __shfl_sync(0xffffffffu, x, 31);
            x -= v;
#pragma unroll
            for (int j = 0; j < kScatterCols; ++j) {
                const uint32_t base = __shfl_sync(0xffffffffu, x, (j * kWarps + warp) & 31);
                const int p = tid + j * kThreads;
                if (j < ppt && p < P) {
                    const uint32_t t0 = base + xs[j], t1 = t0 + c0[j];
                    uint2 rr = run2[p];
                    tstart2[p] = make_uint2(t0, t1);
                    dglob2[p] = make_uint2(rr.x - t0, rr.y - t1);
                    rr.x += c0[j];
                    rr.y += c1[j];
                    run2[p] = rr;
                }
            }
        }
        __syncthreads();  // C

        // ---- tile-local slot of each element, then the sorted tile with global positions
#pragma unroll
        for (int i = 0; i < kSortItems; ++i)
            if (key[i] != kNoKey) rank[i] += tstart[key[i]] + mycnt[key[i]];
        if (!sep) __syncthreads();  // the counters share the sorted tile's space
#pragma unroll
        for (int i = 0; i < kSortItems; ++i) {
            if (key[i] != kNoKey) {
                const uint32_t s = rank[i];
                spos[s] = dglob[key[i]] + s;
                spay[s] = pay[i];
                sw[s] = wv[i];
            }
        }
        __syncthreads();  // E

        // ---- write out: consecutive sorted slots of one digit go to consecutive addresses
        uint32_t *outk = FINAL ? reinterpret_cast<uint32_t *>(sg.col) : sg.tmpk;
        float *outw = FINAL ? sg.val : sg.tmpw;
#pragma unroll 4
        for (int s = tid; s < (int)nranked; s += kThreads) {
            const uint32_t pos = spos[s];
            if (pos >= E32) {
                err |= kStInternal;
                continue;
            }
            outk[pos] = spay[s];
            if (has_w) outw[pos] = sw[s];
        }
    }
    if (err) atomicOr(&s_err, err);
    __syncthreads();
    if (tid == 0 && s_err) atomicOr(sg.status, s_err);
}

// k_count (2-pass graphs): per range of the packed array, the histogram of the final-pass
// digit (-> cnt2, hist2) and the row lengths.  Positions of the packed array are grouped
// by first-pass digit lo (bucket bases = the offsets of range 0 in cnt1), so the range
// splits into segments of constant lo; within a segment the row of an element is
// (hi << lbits) | lo.
__global__ void __launch_bounds__(kThreads) k_count(const __grid_constant__ Ctx c) {
    __shared__ GraphDesc sg;
    __shared__ int sl[2];
    __shared__ uint32_t acc[kMaxDigits];
    __shared__ uint32_t seg[kMaxDigits];
    __shared__ int s_lo[2];
    __shared__ uint32_t s_err;
    __shared__ __align__(8) uint64_t bars[kIdStages];
    extern __shared__ __align__(128) int32_t ringbuf[];
    const IdRing ring{ringbuf, bars};
    const int tid = threadIdx.x;
    id_ring_init(ring);
    const int r = load_desc(c, blockIdx.x, &sg, sl, c.prefix);
    const int D2 = 1 << sg.fbits, D1 = 1 << sg.lbits;
    const int nb = sg.pbits, lb = sg.lbits;
    const int64_t e0 = range_begin(sg, r);
    const int n = range_len(sg, r);
    const uint32_t *lobase = sg.cnt1;  // row 0 of the first-pass offsets: the bucket bases
    uint32_t err = 0;
    if (tid == 0) s_err = 0;
    for (int d = tid; d < D2; d += kThreads) acc[d] = 0;
    if (tid < 2) {
        const uint32_t p = (uint32_t)(e0 + (tid == 0 ? 0 : n - 1));
        int a = 0, b = D1;  // largest bucket with base <= p
        while (b - a > 1) {
            const int m = (a + b) >> 1;
            if (__ldcg(lobase + m) <= p) a = m;
            else b = m;
        }
        s_lo[tid] = a;
    }
    __syncthreads();
    const int lof = s_lo[0], lol = s_lo[1];
    const bool per_segment = (int64_t)(lol - lof + 1) * D2 <= 4 * (int64_t)n;
    if (per_segment) {
        const int warp = tid >> 5;
        const int str = (D2 * kWarps <= kMaxDigits) ? D2 : 0;  // private per-warp histograms
        const int nseg = str ? kWarps * D2 : D2;
        uint32_t *hw = seg + warp * str;
        uint32_t parity = 0;
        for (int l = lof; l <= lol; ++l) {
            const int64_t ps = max((int64_t)__ldcg(lobase + l), e0);
            const int64_t pe = min(l + 1 < D1 ? (int64_t)__ldcg(lobase + l + 1) : sg.E, e0 + n);
            if (pe <= ps) continue;
            for (int d = tid; d < nseg; d += kThreads) seg[d] = 0;
            __syncthreads();
            stream_ids_staged(reinterpret_cast<const int32_t *>(sg.tmpk + ps), (int)(pe - ps), ring, parity, err,
                              [&](int v) {
                if ((uint32_t)v == kSentinel) return;  // a dropped element
                uint32_t hi = (uint32_t)v >> nb;
                if (hi >= (uint32_t)D2) {
                    err |= kStInternal;
                    hi = 0;
                }
                atomicAdd(&hw[hi], 1u);
            });
            __syncthreads();
            for (int d = tid; d < D2; d += kThreads) {
                uint32_t v = 0;
                if (str)
                    for (int w = 0; w < kWarps; ++w) v += seg[w * D2 + d];
                else
                    v = seg[d];
                if (v) {
                    acc[d] += v;
                    const uint32_t row = ((uint32_t)d << lb) | (uint32_t)l;
                    if (row < (uint32_t)sg.N) atomicAdd(sg.rowcnt + row, (int)v);
                }
            }
            __syncthreads();
        }
    } else {  // many tiny buckets: one atomic per edge
        for (int i = tid; i < n; i += kThreads) {
            const uint32_t p = (uint32_t)(e0 + i);
            const uint32_t pv = ld_stream(sg.tmpk + p);
            if (pv == kSentinel) continue;  // a dropped element
            uint32_t hi = pv >> nb;
            if (hi >= (uint32_t)D2) {
                err |= kStInternal;
                hi = 0;
            }
            int a = lof, b = lol + 1;
            while (b - a > 1) {
                const int m = (a + b) >> 1;
                if (__ldcg(lobase + m) <= p) a = m;
                else b = m;
            }
            atomicAdd(&acc[hi], 1u);
            const uint32_t row = (hi << lb) | (uint32_t)a;
            if (row < (uint32_t)sg.N) atomicAdd(sg.rowcnt + row, 1);
        }
        __syncthreads();
    }
    uint32_t *out = sg.cnt2 + ((size_t)r << sg.fbits);
    for (int d = tid; d < D2; d += kThreads) {
        const uint32_t v = acc[d];
        out[d] = v;
        if (v) atomicAdd(&sg.hist2[((size_t)(r % kHistCopies) << sg.fbits) + d], v);
    }
    if (err) atomicOr(&s_err, err);
    __syncthreads();
    if (tid == 0 && s_err) atomicOr(sg.status, s_err);
}

// ------------------------------------------------------------------------------------
// node-table helpers

// s_j = D_jj^-1/2 / n_{y_j} (Laplacian) or 1 / n_{y_j}; unlabelled nodes get {0, 0}.
// yv = y_j, ny = n_{y_j} (read by the caller when y_j is a class).
__device__ __forceinline__ void write_node_known(const GraphDesc &g, int64_t j, float deg, bool lap, int yv,
                                                 int ny) {
    const float dv = lap ? (deg > 0.0f ? 1.0f / sqrtf(deg) : 0.0f) : 1.0f;
    int2 tv = make_int2(0, 0);
    if (yv >= 0 && yv < g.K) {
        const float s = ny > 0 ? dv / (float)ny : 0.0f;
        tv = make_int2(yv, __float_as_int(s));
    }
    g.deg[j] = deg;
    g.dinv[j] = dv;
    g.tab[j] = tv;
}

__device__ __forceinline__ void write_node(const GraphDesc &g, int64_t j, float deg, bool lap) {
    const int yv = __ldg(g.y + j);
    // n_k is final before any kernel that reads it here: the read-only path lets L1 take
    // the repeated reads of the few class sizes that every node asks for
    const int ny = (yv >= 0 && yv < g.K) ? __ldg(g.nk + yv) : 0;
    write_node_known(g, j, deg, lap, yv, ny);
}

// ------------------------------------------------------------------------------------
// k_rowscan: index pointers from the bucket offsets of the last radix pass.  The rows
// of one final-pass digit hi are the 2^lbits consecutive ids (hi << lbits) | lo, in
// order, so a row starts at the bucket base of hi (range 0's offset of digit hi) plus
// the row lengths of the rows before it in that group.  1-pass graphs take the base
// directly (there the digit is the row).  Tiles of 256 to 2048 rows hold whole groups,
// so no tile depends on another.  Also: the hub list, and the node table when no weighted
// degree is needed.

// Chunk offsets of the hub rows (prefix over their chunk counts), by one CTA.
__device__ void hub_chunk_offsets(const CallBufs &cb, uint32_t *s_scan) {
    const uint32_t H = min(__ldcg(&cb.cs->hub_count), cb.hub_cap);
    uint32_t base_run = 0;
    for (uint32_t b = 0; b < H; b += kThreads) {
        const uint32_t h = b + threadIdx.x;
        const uint32_t v = h < H ? (uint32_t)__ldcg(&cb.hubs[h].nch) : 0u;
        uint32_t tot;
        const uint32_t x = block_excl_scan(v, s_scan, tot);
        if (h < H) {
            const uint32_t o = base_run + x;
            cb.chunk_off[h] = o;
            for (uint32_t k = 0; k < v && o + k < cb.chunk_cap; ++k) cb.chunk_hub[o + k] = h;
        }
        base_run += tot;
    }
    if (threadIdx.x == 0) {
        cb.chunk_off[H] = base_run;
        cb.cs->hub_chunks = min(base_run, cb.chunk_cap);
        cb.cs->hub_count = H;
    }
}

// Work items of the length buckets (k_spmm), by one CTA: bucket b of a K > 8 graph gives
// ceil(count / 32) items (one row per item for the whole-warp bucket); the prefix runs
// over (bucket, graph), longest bucket first, so long rows start early.
__device__ void bucket_item_prefix(const Ctx &c, uint32_t *s_scan) {
    const int G = c.G, nb = kBuckets * G;
    uint32_t run = 0;
    for (int b0 = 0; b0 < nb; b0 += kThreads) {
        const int idx = b0 + threadIdx.x;
        uint32_t v = 0;
        if (idx < nb) {
            const int bk = kWarpBucket - idx / G, g = idx % G;
            const int K = G > 1 ? __ldg(&c.graphs[g].K) : c.g0.K;
            if (K > kRegK) {
                const uint32_t *bc = G > 1 ? c.graphs[g].bcount : c.g0.bcount;
                const int lo = G > 1 ? __ldg(&c.graphs[g].bl_off[bk]) : c.g0.bl_off[bk];
                const int hi = G > 1 ? __ldg(&c.graphs[g].bl_off[bk + 1]) : c.g0.bl_off[bk + 1];
                const uint32_t cnt = min(__ldcg(bc + bk), (uint32_t)(hi - lo));
                v = bk == kWarpBucket ? cnt : (cnt + 31u) / 32u;
            }
        }
        uint32_t tot;
        const uint32_t x = block_excl_scan(v, s_scan, tot);
        if (idx < nb) c.cb.bitem[idx] = run + x;
        run += tot;
    }
    if (threadIdx.x == 0) {
        c.cb.bitem[nb] = run;
        c.cb.cs->light_items = run;
    }
}

__global__ void __launch_bounds__(kThreads) k_rowscan(const __grid_constant__ Ctx c) {
    __shared__ GraphDesc sg;
    __shared__ int sl[2];
    __shared__ uint32_t s_scan[kWarps];
    __shared__ int32_t buf[kScanTile + kScanTile / 32];
    __shared__ uint32_t s_err;
    __shared__ int s_last;
    __shared__ uint32_t s_bcnt[kBuckets], s_bbase[kBuckets];

    const int tid = threadIdx.x;
    if (tid == 0) s_err = 0;
    if (tid < kBuckets) s_bcnt[tid] = 0;
    const int t = load_desc(c, blockIdx.x, &sg, sl, c.prefix);
    const int tile = sg.scan_tile, ipt = tile / kThreads;  // 1, 2, 4 or 8 rows per thread
    const int64_t n0 = (int64_t)t * tile;
    const int n = (int)min64(tile, (int64_t)sg.N - n0);
    const int sb = sg.npass == 2 ? sg.lbits : 0;
    const uint32_t *bucket = sg.npass == 2 ? sg.cnt2 : sg.cnt1;
    // every global read of the thread's rows is issued first (the bucket bases and labels
    // do not depend on the scan, the class sizes only on the labels)
    uint32_t base[kScanItems];
    int yv[kScanItems], ny[kScanItems];
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        const int i = tid + k * kThreads;
        base[k] = (i < n && sg.E > 0) ? __ldcg(bucket + ((n0 + i) >> sb)) : 0u;
        yv[k] = (i < n && !sg.wdeg) ? __ldg(sg.y + n0 + i) : -1;
    }
    auto pad = [](int i) { return i + (i >> 5); };
    for (int i = tid; i < tile; i += kThreads) buf[pad(i)] = (i < n) ? __ldcg(sg.rowcnt + n0 + i) : 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) ny[k] = (yv[k] >= 0 && yv[k] < sg.K) ? __ldg(sg.nk + yv[k]) : 0;  // through L1
    __syncthreads();
    uint32_t loc = 0;
#pragma unroll
    for (int j = 0; j < kScanItems; ++j)
        if (j < ipt) loc += (uint32_t)buf[pad(tid * ipt + j)];
    uint32_t tot;
    uint32_t run = block_excl_scan(loc, s_scan, tot);
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
        if (j < ipt) {
            const int i = pad(tid * ipt + j);
            const uint32_t cnt = (uint32_t)buf[i];
            buf[i] = (int32_t)run;
            run += cnt;
        }
    }
    __syncthreads();
    uint32_t err = 0;
    const int gmask = (1 << sb) - 1;  // row offset within its group
    const bool lap = (sg.flags & kOptLap) != 0;
    const float aug = (sg.flags & kOptAug) ? 1.0f : 0.0f;
    const bool buckets = sg.K > kRegK;
    int bks[kScanItems];       // K > 8: length bucket of each light row of this thread (-1: none)
    uint32_t rk[kScanItems];   // its rank among this CTA's rows of that bucket
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        const int i = tid + k * kThreads;
        const int64_t j = n0 + i;
        bks[k] = -1;
        rk[k] = 0;
        if (i < n) {
            const uint32_t ex = (uint32_t)buf[pad(i)];
            const int32_t cnt = (int32_t)((i + 1 < tile ? (uint32_t)buf[pad(i + 1)] : tot) - ex);
            const int32_t start = (int32_t)(base[k] + ex - (uint32_t)buf[pad(i & ~gmask)]);
            sg.rowptr[j] = start;
            if (i == n - 1 && n0 + n == sg.N) sg.rowptr[sg.N] = start + cnt;
            if (cnt > sg.hub_C) {
                const uint32_t h = atomicAdd(&c.cb.cs->hub_count, 1u);
                if (h < c.cb.hub_cap) {
                    HubEntry he;
                    he.g = sl[1];
                    he.row = (int32_t)j;
                    he.len = cnt;
                    he.nch = (cnt + sg.hub_C - 1) / sg.hub_C;
                    c.cb.hubs[h] = he;
                } else {
                    err |= kStInternal;  // capacity is sized so this cannot happen
                }
            } else if (buckets) {
                bks[k] = cnt > sg.short_len ? kWarpBucket : bucket_of(cnt);
                rk[k] = atomicAdd(&s_bcnt[bks[k]], 1u);  // rank within the CTA (order is free)
            }
            if (!sg.wdeg) write_node_known(sg, j, (float)cnt + aug, lap, yv[k], ny[k]);
        }
    }
    // K > 8: one global atomic per bucket and CTA reserves the CTA's places in the lists
    if (buckets) {
        __syncthreads();
        if (tid < kBuckets) s_bbase[tid] = s_bcnt[tid] ? atomicAdd(sg.bcount + tid, s_bcnt[tid]) : 0u;
        __syncthreads();
#pragma unroll
        for (int k = 0; k < kScanItems; ++k) {
            const int b = bks[k];
            if (b < 0) continue;
            const uint32_t pos = s_bbase[b] + rk[k];
            if (pos < (uint32_t)(sg.bl_off[b + 1] - sg.bl_off[b])) sg.rowlist[sg.bl_off[b] + pos] = (int32_t)(n0 + tid + k * kThreads);
            else err |= kStInternal;  // capacity is sized so this cannot happen
        }
    }
    if (err) atomicOr(&s_err, err);
    __syncthreads();
    if (tid == 0 && s_err) atomicOr(sg.status, s_err);
    // the last CTA of the launch (over all graphs) turns the hub list into chunk offsets
    __threadfence();
    __syncthreads();
    if (tid == 0) s_last = atomicAdd(&c.cb.cs->ctr[2], 1u) == gridDim.x - 1u;
    __syncthreads();
    if (s_last) {
        __threadfence();
        hub_chunk_offsets(c.cb, s_scan);
        bucket_item_prefix(c, s_scan);
        // a single graph's workspace now holds a complete CSR, degrees, hub chunks and
        // length buckets for this plan: what gee_reembed may reuse
        if (threadIdx.x == 0 && c.G == 1) c.cb.cs->stamp = c.g0.stamp;
    }
}


// Work item claiming.  CTA-level (hub chunks, which need the whole CTA) and warp-level
// (light rows: every warp claims and finishes its own rows, with no CTA barrier, so a
// long row never holds up the other warps of its CTA).
__device__ __forceinline__ int cta_claim(uint32_t *ctr, int *s_it) {
    __syncthreads();
    if (threadIdx.x == 0) *s_it = (int)atomicAdd(ctr, 1u);
    __syncthreads();
    return *s_it;
}

__device__ __forceinline__ uint32_t warp_claim(uint32_t *ctr) {
    uint32_t it = 0;
    if ((threadIdx.x & 31) == 0) it = atomicAdd(ctr, 1u);
    return __shfl_sync(0xffffffffu, it, 0);
}

// Work items of persistent CTAs / warps: the first item of each is its own index (no
// atomic: thousands of warps starting at once would queue on one counter), later ones
// come from the counter, offset past those first items.
__device__ __forceinline__ uint32_t warp_first_item() { return blockIdx.x * kWarps + (threadIdx.x >> 5); }
__device__ __forceinline__ uint32_t warp_next_item(uint32_t *ctr) { return warp_claim(ctr) + gridDim.x * kWarps; }
__device__ __forceinline__ int cta_next_item(uint32_t *ctr, int *s_it) { return cta_claim(ctr, s_it) + (int)gridDim.x; }

// Copy graph g's descriptor into this warp's shared slot.
__device__ __forceinline__ void warp_load_desc(const Ctx &c, int g, GraphDesc *slot) {
    copy_desc(c, g, slot, threadIdx.x & 31);
    __syncwarp();
}

// Resolve a light-row item to (graph, local block) for the whole warp.
__device__ __forceinline__ int warp_item_graph(const Ctx &c, uint32_t it, int &local) {
    int g = 0, base = 0;
    if (c.G > 1) {
        if ((threadIdx.x & 31) == 0) {
            g = find_graph(c.prefix, c.G, (int)it);
            base = __ldg(c.prefix + g);
        }
        g = __shfl_sync(0xffffffffu, g, 0);
        base = __shfl_sync(0xffffffffu, base, 0);
    }
    local = (int)it - base;
    return g;
}

// clamp a CSR row range to [0, E] (only matters after a reported failure)
__device__ __forceinline__ void row_range(const GraphDesc &g, int64_t row, int64_t &s, int64_t &e) {
    row = min(max(row, (int64_t)0), (int64_t)g.N - 1);
    s = __ldcg(g.rowptr + row);
    e = __ldcg(g.rowptr + row + 1);
    s = min(max(s, (int64_t)0), g.E);
    e = min(max(e, s), g.E);
}

// ------------------------------------------------------------------------------------
// weighted degrees: D_ii = sum_j e_ij (+1), then D^-1/2 and the node table

__device__ __forceinline__ void neumaier_add(float &s, float &c, float v) {
    float t = s + v;
    if (fabsf(s) >= fabsf(v)) c += (s - t) + v;
    else c += (v - t) + s;
    s = t;
}

// ---- length-sorted row blocks --------------------------------------------------------
// A warp claims a block of up to 32 rows, sorts them by length class and runs the rows
// of one class together, each with its own number of lanes: 1 lane for rows of <= 8
// entries, 2 for <= 16, ..., 32 for rows longer than 128.  The lane count of a row
// depends only on its length, so its floating-point sum order (and its bits) do not
// depend on which rows share the block.  Rows longer than the split threshold belong
// to the hub kernels and are skipped here.  With K > 8, k_spmm takes rows of at most
// short_len entries one lane per row instead (short_rows_smem), and the others with at
// least 2 lanes.


// ascending bitonic sort of one 32-bit key per lane
__device__ __forceinline__ uint32_t warp_sort32(uint32_t key, int lane) {
#pragma unroll
    for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            const uint32_t other = __shfl_xor_sync(0xffffffffu, key, j);
            const bool up = (lane & k) == 0, lower = (lane & j) == 0;
            key = (lower == up) ? min(key, other) : max(key, other);
        }
    }
    return key;
}

constexpr uint32_t kNoRow = 0xffffffffu;

// What a pass needs of a row, read once per block: lane l holds row base + l.
struct BlockRow {
    int32_t rs, re;  // CSR entries [rs, re) (empty for no row)
    int2 tab;        // k_spmm: node table entry {y_i, s_i} of the row
    float dinv;      // k_spmm: D_ii^-1/2 (1 without the Laplacian)
    int y, ny;       // k_wdeg: label y_i and class size n_{y_i}
};

// Loads the block's rows (one round trip, two for k_wdeg's class sizes) and returns the
// sorted (class << 5 | offset) keys; kNoRow for rows to skip (none, hub rows, and rows of
// at most short_len entries, which are flagged in is_short; short_len < 0: none).
template <bool SPMM>
__device__ __forceinline__ uint32_t load_block_rows(const GraphDesc &g, int64_t base, int nrows, int lane,
                                                    BlockRow &br, int short_len, bool &is_short) {
    const int64_t row = base + lane;
    const bool has = lane < nrows && row < g.N;
    br.rs = br.re = 0;
    br.tab = make_int2(0, 0);
    br.dinv = 1.0f;
    br.y = -1;
    br.ny = 0;
    if (has) {
        const int32_t a = __ldcg(g.rowptr + row), b = __ldcg(g.rowptr + row + 1);
        if (SPMM) {
            br.tab = __ldg(g.tab + g.row0 + row);
            if (g.flags & kOptLap) br.dinv = __ldg(g.dinv + row);
        } else {
            br.y = __ldg(g.y + row);
        }
        const int32_t E32 = (int32_t)g.E;
        br.rs = min(max(a, 0), E32);
        br.re = min(max(b, br.rs), E32);
    }
    if (!SPMM && br.y >= 0 && br.y < g.K) br.ny = __ldg(g.nk + br.y);  // final n_k, through L1
    uint32_t key = kNoRow;
    const int len = br.re - br.rs;
    is_short = has && len <= short_len;
    const uint32_t cmin = short_len >= 0 ? 1u : 0u;
    if (has && !is_short && len <= g.hub_C) key = (max(cmin, lanes_log2_for(len)) << 5) | (uint32_t)lane;
    if (nrows <= 1) return key;  // one row: already in order
    return warp_sort32(key, lane);
}

// Run f(row, lane-in-group, lanes-per-row, lane of the row's BlockRow) over the block,
// one round per group of rows of a class; every lane of the warp takes part in every
// round (row = N when idle).
template <class F>
__device__ __forceinline__ void for_sorted_rows(const GraphDesc &g, int64_t base, uint32_t sk, int lane, F &&f) {
    const int nvalid = __popc(__ballot_sync(0xffffffffu, sk != kNoRow));
    int pos = 0;
    while (pos < nvalid) {
        const uint32_t c = __shfl_sync(0xffffffffu, sk, pos) >> 5;
        const int n_c = __popc(__ballot_sync(0xffffffffu, sk != kNoRow && (sk >> 5) == c));
        const int lpr = 1 << c, rpr = 32 >> c;
        const int grp = lane >> c, gl = lane & (lpr - 1);
        for (int j = 0; j < n_c; j += rpr) {
            const int idx = pos + j + grp;
            const uint32_t k = __shfl_sync(0xffffffffu, sk, min(idx, 31));
            const bool on = idx < pos + n_c;
            f(on ? base + (int64_t)(k & 31u) : (int64_t)g.N, gl, lpr, on ? (int)(k & 31u) : 0);
        }
        pos += n_c;
    }
}

// k_wdeg: weighted degrees D_ii = sum_j e_ij (+1) of the graphs that need them, then
// D^-1/2 and the node table.
//   hub rows   the CTA takes one chunk at a time: FP64 partial, and the last CTA of a
//              row sums the partials in chunk order
//   light rows then each warp claims row blocks: a group of lanes per row, 16-byte
//              loads, Neumaier-compensated FP32 per lane, deterministic two-sum tree
__global__ void __launch_bounds__(kThreads) k_wdeg(const __grid_constant__ Ctx c) {
    __shared__ GraphDesc sg;
    __shared__ int s_it;
    __shared__ double s_red[kThreads];
    __shared__ int s_last;
    __shared__ GraphDesc wd[kWarps];
    const int tid = threadIdx.x;
    const uint32_t hub_chunks = c.cb.hub_cap ? min(__ldcg(&c.cb.cs->hub_chunks), c.cb.chunk_cap) : 0u;
    for (int it = blockIdx.x; (uint32_t)it < hub_chunks; it = cta_next_item(&c.cb.cs->ctr[3], &s_it)) {
        const int hub = (int)min(__ldcg(c.cb.chunk_hub + it), c.cb.hub_cap - 1u);
        const int chunk = it - (int)__ldcg(c.cb.chunk_off + hub);
        const HubEntry he = c.cb.hubs[hub];
        load_desc_idx(c, he.g, &sg);
        if (!sg.wdeg) continue;  // degree and node table already written by k_rowscan
        int64_t rs, re;
        row_range(sg, he.row, rs, re);
        const int64_t cs = rs + (int64_t)chunk * sg.hub_C;
        const int64_t ce = min(re, cs + sg.hub_C);
        float s = 0.f, cc = 0.f;
        for (int64_t e = cs + tid; e < ce; e += kThreads) neumaier_add(s, cc, ld_stream(sg.val + e));
        s_red[tid] = (double)s + (double)cc;  // FP64 for the heavy-row reduction
        __syncthreads();
        for (int o = kThreads / 2; o > 0; o >>= 1) {
            if (tid < o) s_red[tid] += s_red[tid + o];
            __syncthreads();
        }
        if (tid == 0) {
            const uint32_t slot = __ldcg(c.cb.chunk_off + hub) + (uint32_t)chunk;
            if (slot < c.cb.chunk_cap) c.cb.part_deg[slot] = s_red[0];
            __threadfence();
            const uint32_t arrived = atomicAdd(c.cb.arrive_deg + hub, 1u);
            s_last = (arrived == (uint32_t)he.nch - 1u);
        }
        __syncthreads();
        if (s_last && tid == 0) {
            __threadfence();
            const uint32_t off = __ldcg(c.cb.chunk_off + hub);
            double tot = 0.0;
            for (int k = 0; k < he.nch; ++k)
                if (off + k < c.cb.chunk_cap) tot += __ldcg(c.cb.part_deg + off + k);
            const float aug = (sg.flags & kOptAug) ? 1.0f : 0.0f;
            write_node(sg, min(max(he.row, 0), sg.N - 1), (float)(tot + (double)aug), (sg.flags & kOptLap) != 0);
        }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int cur = -1;
    for (uint32_t it = warp_first_item(); it < (uint32_t)c.items; it = warp_next_item(&c.cb.cs->ctr[6])) {
        int blk;
        const int g = warp_item_graph(c, it, blk);
        if (g != cur) {
            __syncwarp();
            warp_load_desc(c, g, &wd[warp]);
            cur = g;
        }
        const GraphDesc &sg = wd[warp];
        if (!sg.wdeg) continue;
        const int64_t base = (int64_t)blk * sg.rows_per_item;
        BlockRow br;
        bool no_short;
        const uint32_t sk = load_block_rows<false>(sg, base, sg.rows_per_item, lane, br, -1, no_short);
        for_sorted_rows(sg, base, sk, lane, [&](int64_t row, int gl, int lpr, int bi) {
            const int64_t rs = __shfl_sync(0xffffffffu, br.rs, bi), re = __shfl_sync(0xffffffffu, br.re, bi);
            const int yv = __shfl_sync(0xffffffffu, br.y, bi), ny = __shfl_sync(0xffffffffu, br.ny, bi);
            float s = 0.f, cc = 0.f;
            bool active = false;
            if (row < sg.N) {
                active = true;
                const int64_t a0 = rs & ~(int64_t)3;
                const int64_t step = 4 * (int64_t)lpr;
                for (int64_t b = a0 + 4 * gl; b < re; b += 4 * step) {
                    float vv[16];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
                        if (b + u * step < re) v = ld_stream4(sg.val + b + u * step);
                        vv[4 * u] = v.x; vv[4 * u + 1] = v.y; vv[4 * u + 2] = v.z; vv[4 * u + 3] = v.w;
                    }
#pragma unroll
                    for (int q = 0; q < 16; ++q) {
                        const int64_t e = b + (q >> 2) * step + (q & 3);
                        if (e >= rs && e < re) neumaier_add(s, cc, vv[q]);
                    }
                }
            }
            // deterministic tree over the group; the result is taken from its lane 0
            for (int o = lpr >> 1; o > 0; o >>= 1) {
                const float s2 = __shfl_down_sync(0xffffffffu, s, o);
                const float c2 = __shfl_down_sync(0xffffffffu, cc, o);
                if (gl < o) {
                    float e;
                    s = two_sum(s, s2, e);
                    cc = cc + (c2 + e);
                }
            }
            if (active && gl == 0) {
                const float aug = (sg.flags & kOptAug) ? 1.0f : 0.0f;
                write_node_known(sg, row, (s + cc) + aug, (sg.flags & kOptLap) != 0, yv, ny);
            }
        });
    }
}

// ------------------------------------------------------------------------------------
// label-gather product + fused epilogue

// Accumulate val_ij * s_j into per-lane accumulators for the entries [lo, hi) of a row,
// this lane being lane `gl` of a group of `gsz` lanes.  Vector loads of 4 entries from
// 16-byte aligned addresses (col/val are padded by 4 entries at the end).
// kVecs = 16-byte col/val vectors each lane keeps in flight: 4 for rows that take the
// whole warp, 2 for short rows (fewer masked-off slots)
template <int KR, int kVecs>
__device__ __forceinline__ void acc_reg(const GraphDesc &g, int64_t lo, int64_t hi, int gl, int gsz,
                                        float (&acc)[KR], uint32_t &err) {
    const int64_t a0 = lo & ~(int64_t)3;
    const bool has_w = g.val != nullptr;  // the CSR values exist exactly for weighted graphs
    const uint32_t N = (uint32_t)g.ncols;
    const int64_t step = 4 * (int64_t)gsz;
    for (int64_t b = a0 + 4 * gl; b < hi; b += kVecs * step) {
        // kVecs 16-byte vectors of col (and val) in flight per lane, then their gathers
        int cc[4 * kVecs];
        float vv[4 * kVecs];
#pragma unroll
        for (int u = 0; u < kVecs; ++u) {
            const int64_t bu = b + u * step;
            int4 cv = make_int4(0, 0, 0, 0);
            float4 fv = make_float4(1.f, 1.f, 1.f, 1.f);
            if (bu < hi) {
                cv = ld_stream4(g.col + bu);
                if (has_w) fv = ld_stream4(g.val + bu);
            }
            cc[4 * u] = cv.x; cc[4 * u + 1] = cv.y; cc[4 * u + 2] = cv.z; cc[4 * u + 3] = cv.w;
            vv[4 * u] = fv.x; vv[4 * u + 1] = fv.y; vv[4 * u + 2] = fv.z; vv[4 * u + 3] = fv.w;
        }
#pragma unroll
        for (int q = 0; q < 4 * kVecs; ++q) {
            const int64_t e = b + (q >> 2) * step + (q & 3);
            if (e >= lo && e < hi) {
                uint32_t j = (uint32_t)cc[q];
                if (j >= N) { err |= kStInternal; continue; }
                const int2 t = __ldg(g.tab + j);
                const float p = vv[q] * __int_as_float(t.y);
#pragma unroll
                for (int k = 0; k < KR; ++k) acc[k] += (t.x == k) ? p : 0.0f;
            }
        }
    }
}

// Same, into a per-warp shared-memory accumulator sacc[k * 32 + lane] (K up to 64),
// recording the touched classes in a 64-bit mask (tlo: classes 0-31, thi: 32-63).
template <int kVecs>
__device__ __forceinline__ void acc_smem(const GraphDesc &g, int64_t lo, int64_t hi, int gl, int gsz,
                                         float *sacc, int lane, uint32_t &tlo, uint32_t &thi, uint32_t &err) {
    const int64_t a0 = lo & ~(int64_t)3;
    const bool has_w = g.val != nullptr;  // the CSR values exist exactly for weighted graphs
    const uint32_t N = (uint32_t)g.ncols;
    const int64_t step = 4 * (int64_t)gsz;
    for (int64_t b = a0 + 4 * gl; b < hi; b += kVecs * step) {
        // kVecs 16-byte vectors of col (and val) in flight per lane, then their gathers
        int cc[4 * kVecs];
        float vv[4 * kVecs];
#pragma unroll
        for (int u = 0; u < kVecs; ++u) {
            const int64_t bu = b + u * step;
            int4 cv = make_int4(0, 0, 0, 0);
            float4 fv = make_float4(1.f, 1.f, 1.f, 1.f);
            if (bu < hi) {
                cv = ld_stream4(g.col + bu);
                if (has_w) fv = ld_stream4(g.val + bu);
            }
            cc[4 * u] = cv.x; cc[4 * u + 1] = cv.y; cc[4 * u + 2] = cv.z; cc[4 * u + 3] = cv.w;
            vv[4 * u] = fv.x; vv[4 * u + 1] = fv.y; vv[4 * u + 2] = fv.z; vv[4 * u + 3] = fv.w;
        }
#pragma unroll
        for (int q = 0; q < 4 * kVecs; ++q) {
            const int64_t e = b + (q >> 2) * step + (q & 3);
            if (e >= lo && e < hi) {
                uint32_t j = (uint32_t)cc[q];
                if (j >= N) { err |= kStInternal; continue; }
                const int2 t = __ldg(g.tab + j);
                sacc[t.x * 32 + lane] += vv[q] * __int_as_float(t.y);
                if (t.x < 32) tlo |= 1u << t.x;
                else thi |= 1u << (t.x - 32);
            }
        }
    }
}

// ---- light-row entry stream --------------------------------------------------------
// stream_row adds e_ij s_j into slot y_j of the lane's shared-memory accumulator column
// (col[32 k] is class k of this lane: every lane owns one bank, so the adds are free of
// bank conflicts whatever the classes) for every entry of a row [rs, re), in order, taken
// by lane gl of a group of lpr lanes: the lane's 16-byte vectors of col (and val) start at
// (rs & ~3) + 4 gl and follow every 4 lpr entries.  They arrive through a private ring of
// S slots in shared memory filled by cp.async (16-byte asynchronous copies, one commit
// group per vector): S vectors of the lane are always in flight, without holding
// registers, and each lane waits only for its own copies.  A slot is refilled once its
// vector's gathers are issued (the gather addresses come from the slot, so the slot has
// been read by then).  Only a vector that crosses the row's ends tests its entries; the
// entries outside [rs, re) add +0 (exact no-ops).  Copies never read past the arrays
// (col/val are padded by 4 entries) and gathers use clamped indices.  Every copy has
// landed when the function returns.  32-bit indices: E < 2^30.
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(smem)), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// This warp's ring: slot s of lane l at rc[32 s + l] (col) and rv[32 s + l] (val).
struct Ring {
    int4 *rc;
    float4 *rv;
};

__device__ __forceinline__ int acc_slot(int k, int l) { return (k << 5) + l; }

// Accumulators of stream_row: the lane's shared-memory column (any K), or for K <= 4
// registers (no dependent shared-memory read-modify-write chain when consecutive entries
// share a class).
struct ColAcc {
    float *col;
    __device__ __forceinline__ void add(int c, float p) { col[(c & 63) << 5] += p; }
};
template <int KR>
struct RegAcc {
    float a[KR];
    __device__ __forceinline__ void add(int c, float p) {
#pragma unroll
        for (int k = 0; k < KR; ++k) a[k] += (c == k) ? p : 0.0f;
    }
};

template <int S, bool W, class A>
__device__ __forceinline__ void stream_row(const GraphDesc &g, int rs, int re, int gl, int lpr, A &acc,
                                           const Ring &ring, int lane) {
    const int step = 4 * lpr;
    const uint32_t nmax = (uint32_t)g.ncols - 1u;
    const int b0 = (rs & ~3) + 4 * gl;
    const int nv = b0 < re ? (re - b0 + step - 1) / step : 0;
#pragma unroll
    for (int s = 0; s < S; ++s) {
        if (s < nv) {
            cp_async16(ring.rc + 32 * s + lane, g.col + b0 + s * step);
            if (W) cp_async16(ring.rv + 32 * s + lane, g.val + b0 + s * step);
        }
        cp_async_commit();
    }
    for (int i = 0; i < nv; ++i) {
        cp_async_wait<S - 1>();
        const int slot = 32 * (i & (S - 1)) + lane;
        const int4 cv = ring.rc[slot];
        float4 wv = make_float4(1.f, 1.f, 1.f, 1.f);
        if (W) wv = ring.rv[slot];
        const int bi = b0 + i * step;
        int2 t[4];
        t[0] = __ldg(g.tab + min((uint32_t)cv.x, nmax));
        t[1] = __ldg(g.tab + min((uint32_t)cv.y, nmax));
        t[2] = __ldg(g.tab + min((uint32_t)cv.z, nmax));
        t[3] = __ldg(g.tab + min((uint32_t)cv.w, nmax));
        if (i + S < nv) {
            cp_async16(ring.rc + slot, g.col + bi + S * step);
            if (W) cp_async16(ring.rv + slot, g.val + bi + S * step);
        }
        cp_async_commit();
        const float ws[4] = {wv.x, wv.y, wv.z, wv.w};
        if (bi >= rs && bi + 4 <= re) {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float sj = __int_as_float(t[q].y);
                acc.add(t[q].x, W ? ws[q] * sj : sj);
            }
        } else {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float sj = __int_as_float(t[q].y);
                const bool in = bi + q >= rs && bi + q < re;
                acc.add(t[q].x, in ? (W ? ws[q] * sj : sj) : 0.0f);
            }
        }
    }
    cp_async_wait<0>();
}

// Epilogue of a row: augmentation term s_i on the row's own class, D_ii^-1/2 scaling
// (Laplacian), then the 2-norm of the row (correlation).
struct RowTail {
    float dv;     // D_ii^-1/2 (1 without the Laplacian)
    int yi;       // class of the row's node (0 if unlabelled; then si = 0)
    float si;     // s_i = D_ii^-1/2 / n_{y_i}
    bool aug, lap, cor;
};

__device__ __forceinline__ RowTail row_tail(const GraphDesc &g, int2 ti, float dinv) {
    RowTail rt;
    rt.yi = ti.x;
    rt.si = __int_as_float(ti.y);
    rt.aug = (g.flags & kOptAug) != 0;
    rt.lap = (g.flags & kOptLap) != 0;
    rt.cor = (g.flags & kOptCor) != 0;
    rt.dv = rt.lap ? dinv : 1.0f;
    return rt;
}

// Scale of a finished row: 1 / ||Z_i|| with the correlation option (rows with norm 0
// keep scale 1, so they stay 0), else 1.  One division per row; entries are multiplied.
__device__ __forceinline__ float row_scale(float ss, bool cor) {
    return (cor && ss > 0.0f) ? 1.0f / sqrtf(ss) : 1.0f;
}

__device__ __forceinline__ float finish_entry(float total, int k, const RowTail &rt) {
    float v = total;
    if (rt.aug && k == rt.yi) v += rt.si;
    if (rt.lap) v *= rt.dv;
    return v;
}

// Epilogue of one light row per lane group, K <= 8, from the lane's partial sums a[KR]:
// a butterfly over the group adds them up, and the group stores the finished row.
template <int KR>
__device__ __forceinline__ void light_row_reg(const GraphDesc &g, int row, const RowTail &rt, int gl, int lpr,
                                              float (&a)[KR]) {
#pragma unroll
    for (int k = 0; k < KR; ++k)
        for (int o = lpr >> 1; o > 0; o >>= 1) a[k] += __shfl_xor_sync(0xffffffffu, a[k], o);
    if (row >= g.N) return;
    const int K = g.K;
    float ss = 0.0f;
#pragma unroll
    for (int k = 0; k < KR; ++k) {
        a[k] = (k < K) ? finish_entry(a[k], k, rt) : 0.0f;
        ss += a[k] * a[k];
    }
    const float sc = row_scale(ss, rt.cor);
    float *z = g.Z + (int64_t)row * K;
    for (int k = gl; k < K; k += lpr) {
        float v = 0.0f;
#pragma unroll
        for (int kk = 0; kk < KR; ++kk) v = (kk == k) ? a[kk] : v;
        z[k] = v * sc;
    }
}

// one light row per lane group, K <= 8: K <= 4 accumulates in registers, 5 <= K <= 8 in
// the lane's shared-memory column (then taken into registers, clearing the slots)
template <int KR, int V, bool W>
__device__ __forceinline__ void light_row_small(const GraphDesc &g, int row, int rs, int re, const RowTail &rt,
                                                int gl, int lpr, float *sacc, const Ring &ring, int lane) {
    float a[KR];
    if (KR <= 4) {
        RegAcc<KR> acc;
#pragma unroll
        for (int k = 0; k < KR; ++k) acc.a[k] = 0.0f;
        if (row < g.N) stream_row<V, W>(g, rs, re, gl, lpr, acc, ring, lane);
#pragma unroll
        for (int k = 0; k < KR; ++k) a[k] = acc.a[k];
    } else {
        ColAcc acc{sacc + lane};
        if (row < g.N) stream_row<V, W>(g, rs, re, gl, lpr, acc, ring, lane);
#pragma unroll
        for (int k = 0; k < KR; ++k) {
            a[k] = acc.col[k << 5];
            acc.col[k << 5] = 0.0f;
        }
    }
    light_row_reg<KR>(g, row, rt, gl, lpr, a);
}

// one light row per group of lpr >= 2 lanes, 8 < K <= 64: every lane accumulates its
// share of the entries in its own shared-memory column; lane gl then owns the classes
// k = gl mod lpr and sums the group's lpr slots of each, starting at its own lane and
// going round (a fixed order per class, and at every step the lanes of the warp read
// distinct banks), zeroing them; it finishes the entry and keeps it in its own slot until
// the row's scale is known, then stores it.
template <int V, bool W>
__device__ __forceinline__ void long_row_smem(const GraphDesc &g, int row, int rs, int re, const RowTail &rt,
                                              int gl, int lpr, float *sacc, const Ring &ring, int lane) {
    const int K = g.K;
    const int g0 = lane - gl;
    const bool active = row < g.N;
    ColAcc acc{sacc + lane};
    if (active) stream_row<V, W>(g, rs, re, gl, lpr, acc, ring, lane);
    __syncwarp();
    float ss = 0.0f;
    if (active)
        for (int k = gl; k < K; k += lpr) {
            float tot = 0.0f;
            for (int j = 0; j < lpr; ++j) {
                float *p = sacc + acc_slot(k, g0 + ((j + gl) & (lpr - 1)));
                tot += *p;
                *p = 0.0f;
            }
            const float v = finish_entry(tot, k, rt);
            ss += v * v;
            sacc[acc_slot(k, lane)] = v;
        }
    for (int o = lpr >> 1; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
    if (active) {
        const float sc = row_scale(ss, rt.cor);
        float *z = g.Z + (int64_t)row * K;
        for (int k = gl; k < K; k += lpr) {
            float *p = sacc + acc_slot(k, lane);
            z[k] = *p * sc;
            *p = 0.0f;
        }
    }
    // every lane, active or not: the reduction above zeroed slots of other lanes' columns,
    // which the next pass accumulates into
    __syncwarp();
}

// Up to 32 rows of one length bucket, 8 < K <= 64: one lane per row (rows of similar
// length, so the lanes stay busy together), accumulating into its own column with no
// reduction.  The lane then adds the augmentation term and takes the row's scale
// D_ii^-1/2 / ||Z_i|| from its column.  Z is written 8 classes at a time: each lane moves
// its 8 values of the chunk into a transposed 32 x 8 tile laid over the chunk's own slots
// (entry (r, c) at 8 r + (c ^ (r / 4 mod 8)): conflict-free both when the 32 lanes write
// one class each and when they read 4 rows x 8 classes), then each store instruction
// writes 32 contiguous bytes of each of 4 rows.  `rows` holds the rows (cnt of them).
template <int V, bool W>
__device__ __forceinline__ void bucket_rows(const GraphDesc &g, const int32_t *rows, int cnt, float *sacc,
                                            const Ring &ring, int lane) {
    const int K = g.K;
    const bool has = lane < cnt;
    int row = 0;
    float mult = 0.0f;
    if (has) {
        row = min(max(__ldcg(rows + lane), 0), g.N - 1);
        int64_t rs, re;
        row_range(g, row, rs, re);
        ColAcc acc{sacc + lane};
        stream_row<V, W>(g, (int)rs, (int)re, 0, 1, acc, ring, lane);
        const RowTail rt = row_tail(g, __ldg(g.tab + g.row0 + row), (g.flags & kOptLap) ? __ldg(g.dinv + row) : 1.0f);
        if (rt.aug && rt.si != 0.0f) sacc[acc_slot(rt.yi & 63, lane)] += rt.si;
        float ss = 0.0f;
        if (rt.cor)
            for (int k = 0; k < K; ++k) {
                const float v = sacc[acc_slot(k, lane)] * rt.dv;
                ss += v * v;
            }
        mult = rt.dv * row_scale(ss, rt.cor);
    }
    for (int k0 = 0; k0 < K; k0 += 8) {
        float *tile = sacc + (k0 << 5);  // the 256 slots of classes k0 .. k0+7
        float v[8];
#pragma unroll
        for (int c = 0; c < 8; ++c) v[c] = tile[(c << 5) + lane];
        __syncwarp();
        const int sw = (lane >> 2) & 7;
#pragma unroll
        for (int c = 0; c < 8; ++c) tile[(lane << 3) + (c ^ sw)] = v[c];
        __syncwarp();
        const int c = lane & 7;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int r = 4 * q + (lane >> 3);
            const float m = __shfl_sync(0xffffffffu, mult, r);
            const int rr = __shfl_sync(0xffffffffu, row, r);
            if (r < cnt && k0 + c < K) g.Z[(int64_t)rr * K + k0 + c] = tile[(r << 3) + (c ^ (q & 7))] * m;
        }
        __syncwarp();
        float4 *t4 = reinterpret_cast<float4 *>(tile);
        t4[lane] = make_float4(0.f, 0.f, 0.f, 0.f);
        t4[lane + 32] = make_float4(0.f, 0.f, 0.f, 0.f);
        __syncwarp();
    }
}

// One chunk of a hub row, processed by the whole CTA; the last CTA of the row merges.
template <int KR>
__device__ void hub_chunk(const Ctx &c, const GraphDesc &g, const HubEntry &he, int hub, int chunk, float *wa,
                          float *wtot, int *s_last, uint32_t &err) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int K = g.K;
    int64_t rs, re;
    row_range(g, he.row, rs, re);
    const int64_t cs = rs + (int64_t)chunk * g.hub_C;
    const int64_t ce = min(re, cs + g.hub_C);
    // split the chunk into 8 contiguous warp ranges (multiples of 4 entries)
    const int64_t span = ((ce - cs + kWarps - 1) / kWarps + 3) & ~(int64_t)3;
    const int64_t ws = min(ce, cs + warp * span), we = min(ce, ws + span);
    if constexpr (KR > 0) {
        float acc[KR];
#pragma unroll
        for (int k = 0; k < KR; ++k) acc[k] = 0.0f;
        if (ws < we) acc_reg<KR, 4>(g, ws, we, lane, 32, acc, err);
#pragma unroll
        for (int k = 0; k < KR; ++k)
            for (int o = 16; o > 0; o >>= 1) acc[k] += __shfl_xor_sync(0xffffffffu, acc[k], o);
        if (lane == 0)
#pragma unroll
            for (int k = 0; k < KR; ++k)
                if (k < K) wtot[warp * kMaxK + k] = acc[k];
    } else {
        for (int k = 0; k < K; ++k) wa[k * 32 + lane] = 0.0f;
        __syncwarp();
        uint32_t tlo = 0, thi = 0;
        if (ws < we) acc_smem<4>(g, ws, we, lane, 32, wa, lane, tlo, thi, err);
        __syncwarp();
        for (int k = lane; k < K; k += 32) {
            float tot = 0.0f;
            for (int j = 0; j < 32; ++j) tot += wa[k * 32 + ((j + lane) & 31)];
            wtot[warp * kMaxK + k] = tot;
        }
    }
    __syncthreads();
    // combine the warps with two-sum, publish the chunk partial (sum, compensation)
    const uint32_t off = __ldcg(c.cb.chunk_off + hub);
    if (tid < K) {
        float s = wtot[tid], comp = 0.0f;
        for (int w = 1; w < kWarps; ++w) {
            float e;
            s = two_sum(s, wtot[w * kMaxK + tid], e);
            comp += e;
        }
        const uint32_t slot = off + (uint32_t)chunk;
        if (slot < c.cb.chunk_cap) c.cb.part_z[(size_t)slot * c.cb.kmax + tid] = make_float2(s, comp);
    }
    __threadfence();
    __syncthreads();
    if (tid == 0) {
        const uint32_t arrived = atomicAdd(c.cb.arrive_z + hub, 1u);
        *s_last = (arrived == (uint32_t)he.nch - 1u);
    }
    __syncthreads();
    if (!*s_last) return;
    __threadfence();
    // last chunk to finish: merge all chunks of the row in chunk order
    const int hrow = min(max(he.row, 0), g.N - 1);
    const RowTail rt = row_tail(g, __ldg(g.tab + g.row0 + hrow), (g.flags & kOptLap) ? __ldg(g.dinv + hrow) : 1.0f);
    if (tid < K) {
        float S = 0.0f, C = 0.0f;
        for (int ch = 0; ch < he.nch; ++ch) {
            const uint32_t slot = off + (uint32_t)ch;
            if (slot >= c.cb.chunk_cap) break;
            const float2 p = __ldcg(c.cb.part_z + (size_t)slot * c.cb.kmax + tid);
            float e;
            S = two_sum(S, p.x, e);
            C += e + p.y;
        }
        wtot[tid] = finish_entry(S + C, tid, rt);
    }
    __syncthreads();
    if (tid == 0) {
        float ss = 0.0f;
        for (int k = 0; k < K; ++k) ss += wtot[k] * wtot[k];
        wtot[kMaxK * kWarps - 1] = ss;
    }
    __syncthreads();
    if (tid < K) g.Z[(int64_t)hrow * K + tid] = wtot[tid] * row_scale(wtot[kMaxK * kWarps - 1], rt.cor);
}

// One block of rows_per_item consecutive light rows of a K <= 8 graph (k_spmm): the rows
// are loaded once (lane = row), then run in length-class passes.
template <int V, bool W>
__device__ __forceinline__ void spmm_block(const GraphDesc &sg, int64_t base, float *sacc, const Ring &ring,
                                           int lane) {
    const int K = sg.K;
    BlockRow br;
    bool no_short;
    const uint32_t sk = load_block_rows<true>(sg, base, sg.rows_per_item, lane, br, -1, no_short);
    for_sorted_rows(sg, base, sk, lane, [&](int64_t row, int gl, int lpr, int bi) {
        const int rs = __shfl_sync(0xffffffffu, br.rs, bi), re = __shfl_sync(0xffffffffu, br.re, bi);
        int2 t;
        t.x = __shfl_sync(0xffffffffu, br.tab.x, bi);
        t.y = __shfl_sync(0xffffffffu, br.tab.y, bi);
        const RowTail rt = row_tail(sg, t, __shfl_sync(0xffffffffu, br.dinv, bi));
        const int r = (int)row;
        if (K <= 1) light_row_small<1, V, W>(sg, r, rs, re, rt, gl, lpr, sacc, ring, lane);
        else if (K <= 2) light_row_small<2, V, W>(sg, r, rs, re, rt, gl, lpr, sacc, ring, lane);
        else if (K <= 4) light_row_small<4, V, W>(sg, r, rs, re, rt, gl, lpr, sacc, ring, lane);
        else light_row_small<8, V, W>(sg, r, rs, re, rt, gl, lpr, sacc, ring, lane);
    });
}

// One work item of the length buckets of a K > 8 graph: up to 32 rows of a lane-per-row
// bucket, or one row of the whole-warp bucket.
template <int V, bool W>
__device__ __forceinline__ void spmm_bucket_item(const GraphDesc &sg, int bk, uint32_t local, float *sacc,
                                                 const Ring &ring, int lane) {
    const int32_t *list = sg.rowlist + sg.bl_off[bk];
    const uint32_t cap = (uint32_t)(sg.bl_off[bk + 1] - sg.bl_off[bk]);
    const uint32_t count = min(__ldcg(sg.bcount + bk), cap);
    if (bk == kWarpBucket) {
        if (local >= count) return;
        const int row = min(max(__ldcg(list + local), 0), sg.N - 1);
        int64_t rs, re;
        row_range(sg, row, rs, re);
        const RowTail rt = row_tail(sg, __ldg(sg.tab + sg.row0 + row), (sg.flags & kOptLap) ? __ldg(sg.dinv + row) : 1.0f);
        long_row_smem<V, W>(sg, row, (int)rs, (int)re, rt, lane, 32, sacc, ring, lane);
    } else {
        const uint32_t first = local * 32u;
        if (first >= count) return;
        bucket_rows<V, W>(sg, list + first, (int)min(32u, count - first), sacc, ring, lane);
    }
}


// k_spmm: Z with the fused epilogue.
//   hub rows   the CTA takes one chunk at a time (two-sum partials; the last CTA of a
//              row merges them in chunk order and runs the epilogue)
//   light rows then persistent warps, each claiming blocks of rows_per_item rows
// Resident CTAs per SM the product kernel is compiled for: the 4-vector stream needs
// more registers per thread, so it runs 16 warps per SM instead of 24.
template <int V>
struct SpmmOcc {
    static constexpr int kMinBlocks = 3;
};

template <int V>
__global__ void __launch_bounds__(kThreads, SpmmOcc<V>::kMinBlocks) k_spmm(const __grid_constant__ Ctx c) {
    extern __shared__ __align__(16) unsigned char spmm_smem_all[];
    __shared__ GraphDesc sg;
    __shared__ int s_it;
    __shared__ int s_last;
    __shared__ float wtot[kWarps * kMaxK];
    __shared__ GraphDesc wd[kWarps];
    const uint32_t hub_chunks = c.cb.hub_cap ? min(__ldcg(&c.cb.cs->hub_chunks), c.cb.chunk_cap) : 0u;
    const int kpad = (c.cb.kmax + 7) & ~7;  // accumulator classes per lane: K rounded up to 8
    // per warp: the accumulator [kpad][32] floats, then the col ring [V][32] int4, then (if
    // any graph is weighted) the val ring [V][32] float4
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const size_t wstride = (size_t)kpad * 128 + (size_t)V * 512 * (c.cb.ringw ? 2 : 1);
    unsigned char *wbase = spmm_smem_all + warp * wstride;
    float *sacc = reinterpret_cast<float *>(wbase);
    const Ring ring{reinterpret_cast<int4 *>(wbase + (size_t)kpad * 128),
                    reinterpret_cast<float4 *>(wbase + (size_t)kpad * 128 + (size_t)V * 512)};
    uint32_t err = 0;
    for (int it = blockIdx.x; (uint32_t)it < hub_chunks; it = cta_next_item(&c.cb.cs->ctr[4], &s_it)) {
        const int hub = (int)min(__ldcg(c.cb.chunk_hub + it), c.cb.hub_cap - 1u);
        const int chunk = it - (int)__ldcg(c.cb.chunk_off + hub);
        const HubEntry he = c.cb.hubs[hub];
        load_desc_idx(c, he.g, &sg);
        const int K = sg.K;
        if (K <= 1) hub_chunk<1>(c, sg, he, hub, chunk, sacc, wtot, &s_last, err);
        else if (K <= 2) hub_chunk<2>(c, sg, he, hub, chunk, sacc, wtot, &s_last, err);
        else if (K <= 4) hub_chunk<4>(c, sg, he, hub, chunk, sacc, wtot, &s_last, err);
        else if (K <= 8) hub_chunk<8>(c, sg, he, hub, chunk, sacc, wtot, &s_last, err);
        else hub_chunk<0>(c, sg, he, hub, chunk, sacc, wtot, &s_last, err);
        if (err) {
            atomicOr(sg.status, err);
            err = 0;
        }
    }
    __syncthreads();  // the chunks are done with the accumulator space
    for (int i = lane; i < kpad * 32; i += 32) sacc[i] = 0.0f;
    __syncwarp();
    // length-bucket items of the K > 8 graphs (prefix built by k_rowscan's last CTA)
    const uint32_t nbucket = __ldcg(&c.cb.cs->light_items);
    const int nb = kBuckets * c.G;
    int cur = -1;
    for (uint32_t it = warp_first_item(); it < nbucket; it = warp_next_item(&c.cb.cs->ctr[7])) {
        int idx = 0;
        if (lane == 0) {  // largest idx with bitem[idx] <= it
            int lo = 0, hi = nb;
            while (hi - lo > 1) {
                const int mid = (lo + hi) >> 1;
                if (__ldcg(c.cb.bitem + mid) <= it) lo = mid;
                else hi = mid;
            }
            idx = lo;
        }
        idx = __shfl_sync(0xffffffffu, idx, 0);
        const int bk = kWarpBucket - idx / c.G, g = idx % c.G;
        const uint32_t local = it - __ldcg(c.cb.bitem + idx);
        if (g != cur) {
            __syncwarp();
            warp_load_desc(c, g, &wd[warp]);
            cur = g;
        }
        const GraphDesc &sg = wd[warp];
        if (sg.val) spmm_bucket_item<V, true>(sg, bk, local, sacc, ring, lane);
        else spmm_bucket_item<V, false>(sg, bk, local, sacc, ring, lane);
    }
    // blocks of consecutive light rows of the K <= 8 graphs
    cur = -1;
    for (uint32_t it = warp_first_item(); it < (uint32_t)c.items; it = warp_next_item(&c.cb.cs->ctr[5])) {
        int blk;
        const int g = warp_item_graph(c, it, blk);
        if (g != cur) {
            __syncwarp();
            warp_load_desc(c, g, &wd[warp]);
            cur = g;
        }
        const GraphDesc &sg = wd[warp];
        const int64_t base = (int64_t)blk * sg.rows_per_item;
        if (sg.val) spmm_block<V, true>(sg, base, sacc, ring, lane);
        else spmm_block<V, false>(sg, base, sacc, ring, lane);
    }
}

// ------------------------------------------------------------------------------------
// Re-embedding with new labels on the CSR a previous call built (Section 2: W from known or
// predicted labels; the CSR, the degrees D and the hub and bucket plans do not depend on
// the labels).  k_labels recounts n_k and checks the labels; its first thread also checks
// that the workspace was built for this plan, and if not reports GEE_STATUS_STALE and
// empties the hub and bucket work so that k_spmm only reads in-range memory.  k_nodetab
// then rebuilds the node table s_j = D_jj^-1/2 / n_{y_j} from the stored D^-1/2.

constexpr int kRelabelItems = 4;                          // nodes per thread
constexpr int kRelabelTile = kRelabelItems * kThreads;    // nodes per CTA

__global__ void __launch_bounds__(kThreads) k_labels(const __grid_constant__ Ctx c) {
    __shared__ uint32_t h[kMaxK];
    __shared__ uint32_t s_err;
    const GraphDesc &g = c.g0;
    const int tid = threadIdx.x;
    if (tid == 0) {
        s_err = 0;
        if (blockIdx.x == 0 && __ldcg(&c.cb.cs->stamp) != g.stamp) {
            atomicOr(g.status, kStStale);
            c.cb.cs->hub_chunks = 0u;
            c.cb.cs->light_items = 0u;
        }
    }
    for (int i = tid; i < g.K; i += kThreads) h[i] = 0;
    // tiles of kRelabelTile nodes; every label read of the thread is in flight at once
    const int64_t n0 = (int64_t)blockIdx.x * kRelabelTile;
    int yv[kRelabelItems];
#pragma unroll
    for (int q = 0; q < kRelabelItems; ++q) {
        const int64_t j = n0 + tid + q * kThreads;
        yv[q] = j < g.N ? __ldg(g.y + j) : -1;
    }
    __syncthreads();
    uint32_t err = 0;
#pragma unroll
    for (int q = 0; q < kRelabelItems; ++q) {
        if (yv[q] < -1 || yv[q] >= g.K) err |= kStLabel;
        else if (yv[q] >= 0) atomicAdd(&h[yv[q]], 1u);
    }
    if (err) atomicOr(&s_err, err);
    __syncthreads();
    for (int i = tid; i < g.K; i += kThreads)
        if (h[i]) atomicAdd(reinterpret_cast<unsigned *>(g.nk) + i, h[i]);
    if (tid == 0 && s_err) atomicOr(g.status, s_err);
}

// Node table with the new labels: kRelabelItems nodes per thread, their label and degree
// reads in flight at once, then their class sizes.
__global__ void __launch_bounds__(kThreads) k_nodetab(const __grid_constant__ Ctx c) {
    const GraphDesc &g = c.g0;
    const bool lap = (g.flags & kOptLap) != 0;
    const int64_t n0 = (int64_t)blockIdx.x * kRelabelTile + threadIdx.x;
    int yv[kRelabelItems], ny[kRelabelItems];
    float dv[kRelabelItems];
#pragma unroll
    for (int q = 0; q < kRelabelItems; ++q) {
        const int64_t j = n0 + q * kThreads;
        yv[q] = j < g.N ? __ldg(g.y + j) : -1;
        dv[q] = (lap && j < g.N) ? __ldcg(g.dinv + j) : 1.0f;
    }
#pragma unroll
    for (int q = 0; q < kRelabelItems; ++q) ny[q] = (yv[q] >= 0 && yv[q] < g.K) ? __ldg(g.nk + yv[q]) : 0;  // through L1
#pragma unroll
    for (int q = 0; q < kRelabelItems; ++q) {
        const int64_t j = n0 + q * kThreads;
        if (j >= g.N) continue;
        int2 tv = make_int2(0, 0);
        if (yv[q] >= 0 && yv[q] < g.K)
            tv = make_int2(yv[q], __float_as_int(ny[q] > 0 ? dv[q] / (float)ny[q] : 0.0f));
        g.tab[j] = tv;
    }
}

// A product on a workspace that must hold a build of this plan (a row shard): if its stamp
// does not match, report GEE_STATUS_STALE and empty the hub and bucket work.
__global__ void k_stamp(const __grid_constant__ Ctx c) {
    if (threadIdx.x == 0 && __ldcg(&c.cb.cs->stamp) != c.g0.stamp) {
        atomicOr(c.g0.status, kStStale);
        c.cb.cs->hub_chunks = 0u;
        c.cb.cs->light_items = 0u;
    }
}

cudaError_t launch_stamp_check(const Ctx &c, cudaStream_t st) {
    k_stamp<<<1, 32, 0, st>>>(c);
    return cudaGetLastError();
}

cudaError_t launch_nodetab(const Ctx &c, cudaStream_t st) {
    const int64_t N = c.g0.N;
    if (N <= 0) return cudaSuccess;
    k_nodetab<<<(int)min64((N + kThreads - 1) / kThreads, 152 * 8), kThreads, 0, st>>>(c);
    return cudaGetLastError();
}

cudaError_t launch_relabel(const Ctx &c, cudaStream_t st) {
    const int64_t N = c.g0.N;
    if (N <= 0) return cudaSuccess;
    const int tiles = (int)((N + kRelabelTile - 1) / kRelabelTile);
    k_labels<<<tiles, kThreads, 0, st>>>(c);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_nodetab<<<tiles, kThreads, 0, st>>>(c);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------
// k_class_counts: C[i][k] = #{entries of row i whose column has label k}; warp per row

constexpr int kCcWarps = 4;  // 4 warps x 64 classes x 32 lanes x 4 B = 32 KB of shared memory

__global__ void __launch_bounds__(kCcWarps * 32) k_class_counts(const int32_t *rowptr, const int32_t *col,
                                                                int32_t N, const int32_t *y, int32_t K,
                                                                int32_t *C) {
    __shared__ int32_t cnt[kCcWarps][kMaxK * 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int32_t *mine = cnt[warp];
    for (int64_t row = (int64_t)blockIdx.x * kCcWarps + warp; row < N; row += (int64_t)gridDim.x * kCcWarps) {
        for (int k = 0; k < K; ++k) mine[k * 32 + lane] = 0;
        const int64_t s = rowptr[row], e = rowptr[row + 1];
        for (int64_t p = s + lane; p < e; p += 32) {
            const int32_t j = col[p];
            if (j < 0 || j >= N) continue;
            const int32_t yk = y[j];
            if (yk >= 0 && yk < K) mine[yk * 32 + lane] += 1;
        }
        __syncwarp();
        for (int k = lane; k < K; k += 32) {
            int32_t tot = 0;
            for (int j = 0; j < 32; ++j) tot += mine[k * 32 + j];
            C[row * K + k] = tot;
        }
        __syncwarp();
    }
}

__global__ void k_fill(float *p, int64_t n, float v) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        p[i] = v;
}

// ------------------------------------------------------------------------------------
// host-side launchers (used by gee_api.cu)

cudaError_t launch_fill(float *p, int64_t n, float v, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    const int blocks = (int)min64((n + kThreads - 1) / kThreads, 4096);
    k_fill<<<blocks, kThreads, 0, st>>>(p, n, v);
    return cudaGetLastError();
}

cudaError_t launch_prep(const Ctx &c, int blocks, cudaStream_t st) {
    if (blocks <= 0) return cudaSuccess;
    k_prep<<<blocks, kThreads, kIdRingBytes, st>>>(c);
    return cudaGetLastError();
}

cudaError_t launch_offsets(const Ctx &c, int blocks, bool second, cudaStream_t st) {
    if (blocks <= 0) return cudaSuccess;
    if (second) k_offsets<true><<<blocks, kOffThreads, 0, st>>>(c);
    else k_offsets<false><<<blocks, kOffThreads, 0, st>>>(c);
    return cudaGetLastError();
}

// Shared memory for every digit count up to 2^max_digit_bits (the layout is not monotone
// in D: the counters stop having their own space above kSepDigits).
size_t scatter_smem(int max_digit_bits) {
    size_t m = 0;
    for (int b = 1; b <= max_digit_bits; ++b) m = std::max(m, scatter_smem_bytes(1 << b));
    return m;
}

cudaError_t launch_scatter(const Ctx &c, int blocks, bool final_pass, int max_digit_bits, cudaStream_t st) {
    if (blocks <= 0) return cudaSuccess;
    const size_t smem = scatter_smem(max_digit_bits);
    if (final_pass) k_scatter<true><<<blocks, kThreads, smem, st>>>(c);
    else k_scatter<false><<<blocks, kThreads, smem, st>>>(c);
    return cudaGetLastError();
}

cudaError_t launch_count(const Ctx &c, int blocks, cudaStream_t st) {
    if (blocks <= 0) return cudaSuccess;
    k_count<<<blocks, kThreads, kIdRingBytes, st>>>(c);
    return cudaGetLastError();
}

cudaError_t launch_rowscan(const Ctx &c, int blocks, cudaStream_t st) {
    if (blocks <= 0) return cudaSuccess;
    k_rowscan<<<blocks, kThreads, 0, st>>>(c);
    return cudaGetLastError();
}

cudaError_t launch_wdeg(const Ctx &c, int blocks, cudaStream_t st) {
    if (blocks <= 0) return cudaSuccess;
    k_wdeg<<<blocks, kThreads, 0, st>>>(c);
    return cudaGetLastError();
}

// shared memory of k_spmm: per warp a [kpad][32] float accumulator and rings of `ring`
// 16-byte slots per lane for col (and val when `ringw`)
size_t spmm_smem(int kpad, int ring, bool ringw) {
    return (size_t)kWarps * ((size_t)kpad * 128 + (size_t)ring * 512 * (ringw ? 2 : 1));
}

cudaError_t launch_spmm(const Ctx &c, int blocks, int kpad, int ring, cudaStream_t st) {
    if (blocks <= 0) return cudaSuccess;
    const size_t sm = spmm_smem(kpad, ring, c.cb.ringw != 0);
    if (ring >= 8) k_spmm<8><<<blocks, kThreads, sm, st>>>(c);
    else if (ring >= 4) k_spmm<4><<<blocks, kThreads, sm, st>>>(c);
    else k_spmm<2><<<blocks, kThreads, sm, st>>>(c);
    return cudaGetLastError();
}

cudaError_t launch_class_counts(const int32_t *rowptr, const int32_t *col, int32_t N, const int32_t *y, int32_t K,
                                int32_t *C, int blocks, cudaStream_t st) {
    if (N <= 0) return cudaSuccess;
    k_class_counts<<<blocks, kCcWarps * 32, 0, st>>>(rowptr, col, N, y, K, C);
    return cudaGetLastError();
}

cudaError_t configure_kernels() {
    const int big = (int)scatter_smem(kMaxDigitBits);
    cudaError_t e = cudaFuncSetAttribute(k_scatter<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_scatter<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_prep, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kIdRingBytes);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_count, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kIdRingBytes);
    if (e != cudaSuccess) return e;
    const int big_spmm = 200 * 1024;
    e = cudaFuncSetAttribute(k_spmm<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, big_spmm);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_spmm<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, big_spmm);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_spmm<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, big_spmm);
}

static int occ(const void *f, size_t smem) {
    int n = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, f, kThreads, smem);
    return n > 0 ? n : 1;
}

int occupancy_spmm(int kpad, int ring, bool ringw) {
    const void *f = ring >= 8 ? (const void *)k_spmm<8> : (ring >= 4 ? (const void *)k_spmm<4> : (const void *)k_spmm<2>);
    return occ(f, spmm_smem(kpad, ring, ringw));
}
int occupancy_wdeg() { return occ((const void *)k_wdeg, 0); }

}  // namespace gee
