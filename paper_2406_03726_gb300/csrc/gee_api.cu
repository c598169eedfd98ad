// Host runtime and C ABI of libgee (see include/gee.h).
//
// A call is planned on the host (digit widths, split threshold, lanes per row, the
// workspace layout) and then enqueued on the caller's stream as: one memset of the
// zero-initialised part of the workspace, then k_prep, k_offsets and k_scatter (1 or 2
// radix passes, with k_count between them), k_rowscan, k_wdeg (weighted Laplacian only)
// and k_spmm.  Nothing is
// allocated and nothing synchronises, so the sequence can be captured in a CUDA graph.
#include "gee_internal.cuh"
#include "gee_sparse.cuh"
#include "../../include/gee.h"

#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <string>
#include <functional>
#include <mutex>
#include <vector>

namespace gee {

cudaError_t launch_prep(const Ctx &c, int blocks, cudaStream_t st);
cudaError_t launch_offsets(const Ctx &c, int blocks, bool second, cudaStream_t st);
cudaError_t launch_scatter(const Ctx &c, int blocks, bool final_pass, int max_digit_bits, cudaStream_t st);
size_t scatter_smem(int max_digit_bits);
cudaError_t launch_count(const Ctx &c, int blocks, cudaStream_t st);
cudaError_t launch_rowscan(const Ctx &c, int blocks, cudaStream_t st);
cudaError_t launch_wdeg(const Ctx &c, int blocks, cudaStream_t st);
cudaError_t launch_spmm(const Ctx &c, int blocks, int kpad, int ring, cudaStream_t st);
cudaError_t launch_class_counts(const int32_t *rowptr, const int32_t *col, int32_t N, const int32_t *y, int32_t K,
                                int32_t *C, int blocks, cudaStream_t st);
cudaError_t launch_fill(float *p, int64_t n, float v, cudaStream_t st);
cudaError_t launch_relabel(const Ctx &c, cudaStream_t st);
cudaError_t launch_nodetab(const Ctx &c, cudaStream_t st);
cudaError_t launch_stamp_check(const Ctx &c, cudaStream_t st);
cudaError_t configure_kernels();
int occupancy_spmm(int kpad, int ring, bool ringw);
size_t spmm_smem(int kpad, int ring, bool ringw);
int occupancy_wdeg();

namespace {

constexpr size_t kAlign = 256;
constexpr int kSMs = 152;                   // GB300
constexpr size_t kSmemPerSM = 228 * 1024;   // shared memory per SM usable by CTAs
constexpr int kWarpsPerSM = 24;             // resident warps of the row kernels (3 CTAs)

struct DeviceInfo {
    bool ready = false;
    int sms = 0;
    int occ_spmm[3][8][2] = {};  // CTAs per SM of k_spmm by ring depth (2, 4, 8), classes / 8 - 1, val ring
    int occ_wdeg = 1;
};

std::mutex g_mu;
DeviceInfo g_dev[64];

int device_info(DeviceInfo &out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return GEE_ERR_CUDA;
    std::lock_guard<std::mutex> lk(g_mu);
    DeviceInfo &d = g_dev[dev];
    if (!d.ready) {
        if (cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return GEE_ERR_CUDA;
        if (configure_kernels() != cudaSuccess || configure_sparse_kernels() != cudaSuccess) return GEE_ERR_CUDA;
        for (int v = 0; v < 3; ++v)
            for (int i = 0; i < 8; ++i)
                for (int w = 0; w < 2; ++w) d.occ_spmm[v][i][w] = occupancy_spmm(8 * (i + 1), 2 << v, w != 0);
        d.occ_wdeg = occupancy_wdeg();
        d.ready = true;
    }
    out = d;
    return GEE_OK;
}

struct Bump {
    char *base;
    size_t off = 0;
    template <class T>
    T *take(size_t n) {
        off = (off + kAlign - 1) & ~(kAlign - 1);
        T *p = base ? reinterpret_cast<T *>(base + off) : nullptr;
        off += n * sizeof(T);
        return p;
    }
};

int bitlen(uint32_t x) {
    int b = 0;
    while (x) {
        ++b;
        x >>= 1;
    }
    return b;
}

int ilog2_pow2(int x) {
    int l = 0;
    while ((1 << l) < x) ++l;
    return l;
}

struct Shape {
    int64_t E;
    int32_t N, K;
    bool weighted;
};

// Ranges of range_tiles sort tiles, one scatter CTA each (over the 2 Ein virtual entries
// when symmetrizing).
void set_ranges(GraphDesc &d, int32_t range_tiles) {
    d.range_tiles = range_tiles;
    d.ranges = (d.tiles_e + d.range_tiles - 1) / d.range_tiles;
}

// Plan parameters of one graph.  Everything that decides the order of floating-point
// additions depends only on the graph and the options (never on the batch it is part of,
// so a graph gives the same bits alone and in a batch); the row-block size only groups
// rows into work items.
// rows_in_launch: rows of every graph the launch covers (N alone for a single graph);
// the automatic row-block size keeps the launch's warps busy, not each graph's.
void plan_params(const Shape &s, const gee_opts &o, bool want_deg, GraphDesc &d, int64_t rows_in_launch = -1) {
    if (rows_in_launch < 0) rows_in_launch = s.N;
    d.sym = (o.flags & GEE_SYMMETRIZE) ? 1 : 0;
    d.Ein = s.E;
    d.E = d.sym ? 2 * s.E : s.E;  // the CSR holds at most both copies of every input edge
    d.N = s.N;
    d.K = s.K;
    d.flags = o.flags & GEE_ALL_OPTIONS;
    d.nbits = std::max(d.sym ? 2 : 1, bitlen(s.N > 0 ? (uint32_t)(s.N - 1) : 0u));
    d.ncols = s.N;      // a row shard overrides these three (plan_shard)
    d.pbits = d.nbits;
    d.row0 = 0;
    if (d.nbits <= kOnePassBits && !d.sym) {  // symmetrizing always takes two passes (the
        d.npass = 1;                           // first one marks the dropped self-loop copies)
        d.lbits = 0;
        d.fbits = d.nbits;
    } else {
        d.npass = 2;
        d.lbits = (d.nbits + 1) / 2;
        d.fbits = d.nbits - d.lbits;
    }
    const double mean = s.N > 0 ? (double)d.E / (double)s.N : 0.0;
    int lpr = o.lanes_per_row;
    if (lpr <= 0) {
        lpr = 1;
        while (lpr < 32 && lpr * 8 < mean) lpr <<= 1;
    }
    lpr = std::min(32, std::max(1, lpr));
    d.lpr_log2 = ilog2_pow2(lpr);
    // rows longer than hub_C are split across CTAs: 64 vector loads per lane of the group
    d.hub_C = o.hub_threshold > 0 ? o.hub_threshold : std::max(1024, 256 * lpr);
    d.tiles_e = (int32_t)((d.E + kSortTile - 1) / kSortTile);
    // index-pointer tiles: whole final-digit groups of 2^lbits rows, at least 256 rows,
    // and no smaller than needed for about four tiles per SM over the launch's rows
    d.scan_tile = std::max(kThreads, d.npass == 2 ? (1 << d.lbits) : 1);
    while (d.scan_tile < kScanTile && rows_in_launch > (int64_t)4 * kSMs * d.scan_tile) d.scan_tile <<= 1;
    d.tiles_n = (int32_t)(((int64_t)s.N + d.scan_tile - 1) / d.scan_tile);
    // rows a warp claims at once: blocks of up to 32 rows sorted by length, small enough
    // that a launch of few rows still gives every resident warp two blocks (a row's lanes
    // come from its length, so short rows share a warp in any block)
    if (o.rows_per_item > 0) {
        d.rows_per_item = o.rows_per_item;
    } else {
        const int64_t warps = (int64_t)kSMs * kWarpsPerSM;
        int rpi = 32;
        while (rpi > 1 && rows_in_launch < 2 * warps * rpi) rpi >>= 1;
        d.rows_per_item = rpi;
    }
    d.wdeg = (s.weighted && ((d.flags & kOptLap) || want_deg)) ? 1 : 0;
    d.short_len = o.short_len > 0 ? o.short_len : 256;
    d.vec = o.vec_width;  // 0: chosen at launch from the shared memory it leaves
    // K > 8: capacities of the length buckets.  Bucket b >= 1 of the one-lane buckets
    // holds rows of more than lo_b entries (so at most E / (lo_b + 1) of them); the
    // whole-warp bucket rows of more than short_len entries.
    int64_t off = 0;
    for (int b = 0; b < kBuckets; ++b) {
        d.bl_off[b] = (int32_t)off;
        int64_t cap = 0;
        if (s.K > kRegK) {
            if (b == 0) {
                cap = s.N;
            } else if (b < kWarpBucket) {
                const int64_t lo = (int64_t)4 << b;  // 8, 16, 32, 64, 128
                cap = lo < d.short_len ? std::min<int64_t>(s.N, d.E / (lo + 1)) : 0;
            } else {
                cap = std::min<int64_t>(s.N, d.E / ((int64_t)d.short_len + 1));
            }
        }
        off += cap;
    }
    d.bl_off[kBuckets] = (int32_t)off;
    // one range per scatter CTA, as many ranges as CTAs fit at once on GB300's 152 SMs
    // (shared memory per CTA grows with the digit count; at most 4 CTAs by registers)
    const int maxbits = std::max(d.fbits, first_bits(d));
    const int per_sm = std::max<int>(1, std::min<int>(4, (int)(kSmemPerSM / (scatter_smem(maxbits) + 1024))));
    const int target = kSMs * per_sm;
    set_ranges(d, std::max<int32_t>(1, (d.tiles_e + target - 1) / target));
}

uint32_t hub_cap_of(const GraphDesc &d) { return (uint32_t)(d.E / ((int64_t)d.hub_C + 1)); }
uint32_t chunk_cap_of(const GraphDesc &d) { return (uint32_t)(d.E / d.hub_C) + hub_cap_of(d) + 1; }

// zero-initialised arrays of one graph (its status word is allocated by the caller)
void layout_zero(Bump &b, GraphDesc &d) {
    d.rowcnt = b.take<int32_t>((size_t)d.N);
    d.bcount = d.K > kRegK ? b.take<uint32_t>((size_t)kBuckets) : nullptr;
    d.nk = b.take<int32_t>((size_t)d.K);
    d.hist1 = b.take<uint32_t>((size_t)kHistCopies << first_bits(d));
    d.hist2 = d.npass == 2 ? b.take<uint32_t>((size_t)kHistCopies << d.fbits) : nullptr;
}

void layout_rest(Bump &b, GraphDesc &d, bool weighted) {
    d.rowptr = b.take<int32_t>((size_t)d.N + 1);
    d.col = b.take<int32_t>((size_t)d.E + 4);
    d.val = weighted ? b.take<float>((size_t)d.E + 4) : nullptr;
    d.tmpk = d.npass == 2 ? b.take<uint32_t>((size_t)d.E) : nullptr;
    d.tmpw = (d.npass == 2 && weighted) ? b.take<float>((size_t)d.E) : nullptr;
    d.cnt1 = b.take<uint32_t>((size_t)d.ranges << first_bits(d));
    d.cnt2 = d.npass == 2 ? b.take<uint32_t>((size_t)d.ranges << d.fbits) : nullptr;
    d.deg = b.take<float>((size_t)d.N);
    d.dinv = b.take<float>((size_t)d.N);
    d.tab = b.take<int2>((size_t)d.N);
    d.rowlist = d.K > kRegK ? b.take<int32_t>((size_t)d.bl_off[kBuckets]) : nullptr;
}

void layout_call_zero(Bump &b, CallBufs &cb) {
    cb.cs = b.take<CallState>(1);
    cb.arrive_deg = b.take<uint32_t>(cb.hub_cap);
    cb.arrive_z = b.take<uint32_t>(cb.hub_cap);
}

void layout_call_rest(Bump &b, CallBufs &cb, int32_t G) {
    cb.bitem = b.take<uint32_t>((size_t)kBuckets * G + 1);
    cb.hubs = b.take<HubEntry>(cb.hub_cap);
    cb.chunk_off = b.take<uint32_t>((size_t)cb.hub_cap + 1);
    cb.chunk_hub = b.take<uint32_t>(cb.chunk_cap);
    cb.part_deg = b.take<double>(cb.chunk_cap);
    cb.part_z = b.take<float2>((size_t)cb.chunk_cap * (size_t)cb.kmax);
}

int check_shape(int64_t E, int32_t N, int32_t K) {
    if (E < 0 || N < 0 || K < 1) return GEE_ERR_ARG;
    if (N > GEE_MAX_N || E >= GEE_MAX_E || K > GEE_MAX_K) return GEE_ERR_TOO_LARGE;
    return GEE_OK;
}

gee_opts opts_or_default(const gee_opts *o) {
    gee_opts r;
    std::memset(&r, 0, sizeof(r));
    if (o) r = *o;
    return r;
}

int check_opts(const gee_opts &o) {
    if (o.hub_threshold < 0 || o.lanes_per_row < 0 || o.lanes_per_row > 32 ||
        (o.lanes_per_row & (o.lanes_per_row - 1)) || o.rows_per_item < 0 || o.rows_per_item > 32 ||
        (o.rows_per_item & (o.rows_per_item - 1)) ||
        !(o.vec_width == 0 || o.vec_width == 2 || o.vec_width == 4 || o.vec_width == 8) ||
        !(o.short_len == 0 || (o.short_len >= 8 && o.short_len <= (4 << kWarpBucket) &&
                               !(o.short_len & (o.short_len - 1)))))
        return GEE_ERR_ARG;
    return GEE_OK;
}

int cuda_check(cudaError_t e) { return e == cudaSuccess ? GEE_OK : GEE_ERR_CUDA; }

#define GEE_TRY(x)                     \
    do {                               \
        int _rc = (x);                 \
        if (_rc != GEE_OK) return _rc; \
    } while (0)

// ---- launch plan: everything the launch sequence needs, for one graph or many -----------

struct LaunchPlan {
    Ctx base;                        // g0 (one graph) or graphs (G > 1), and the call buffers
    const int32_t *prefix[kNumPfx];  // device item prefixes per kernel (G > 1)
    int32_t items[kNumPfx];          // total items per kernel
    int b1max = 1, fmax = 1;         // widest digits (shared-memory size of k_scatter)
    bool any_two = false, any_wdeg = false, smem_acc = false;
    int vec = 0;                     // ring slots per lane of k_spmm (0: automatic)
    void *zero_base = nullptr;
    size_t zero_bytes = 0;
};

void plan_items(const GraphDesc &d, int32_t it[kNumPfx]) {
    const int node_tiles = (int)(((int64_t)d.N + kPrepTile - 1) / kPrepTile);
    const bool two = d.npass == 2, edges = d.ranges > 0;
    const int row_items = (int)(((int64_t)d.N + d.rows_per_item - 1) / d.rows_per_item);
    it[kPfxPrep] = d.ranges + node_tiles;
    it[kPfxOffs1] = edges ? ((1 << first_bits(d)) + 31) / 32 : 0;
    it[kPfxScat1] = (edges && two) ? d.ranges : 0;
    it[kPfxCount] = (edges && two) ? d.ranges : 0;
    it[kPfxOffs2] = (edges && two) ? ((1 << d.fbits) + 31) / 32 : 0;
    it[kPfxScatF] = d.ranges;
    it[kPfxScan] = d.tiles_n;
    it[kPfxRows] = d.K > kRegK ? 0 : row_items;  // K > 8: length-bucket items, counted on the device
    it[kPfxWRows] = d.wdeg ? row_items : 0;
}

void plan_accumulate(LaunchPlan &lp, const GraphDesc &d) {
    int32_t it[kNumPfx];
    plan_items(d, it);
    for (int k = 0; k < kNumPfx; ++k) lp.items[k] += it[k];
    lp.b1max = std::max(lp.b1max, d.npass == 2 ? d.lbits : 1);
    lp.fmax = std::max(lp.fmax, d.fbits);
    lp.any_two = lp.any_two || d.npass == 2;
    lp.any_wdeg = lp.any_wdeg || d.wdeg;
    lp.smem_acc = lp.smem_acc || d.K > kRegK;
    lp.vec = d.vec;  // every graph of a launch is planned with the same options
    lp.base.cb.ringw = lp.base.cb.ringw || d.val != nullptr || d.w != nullptr;
}

// Phases of one call, in launch order (the GEE_NUM_PHASES list in gee.h).
enum Phase {
    kPhMemset = 0,
    kPhPrep,
    kPhOffs1,
    kPhScat1,
    kPhCount,
    kPhOffs2,
    kPhScatF,
    kPhRowscan,
    kPhWdeg,
    kPhSpmm,
    kNumPhases
};

// Optional per-phase timing: events[i] is recorded before phase i, events[kNumPhases]
// after the last one; ran[i] tells whether phase i launched anything.
struct PhaseEvents {
    cudaEvent_t ev[kNumPhases + 1];
    bool ran[kNumPhases];
    bool external = false;  // being captured into a graph: record as event nodes
};

inline int mark(PhaseEvents *pe, int ph, cudaStream_t st) {
    if (!pe) return GEE_OK;
    return cuda_check(pe->external ? cudaEventRecordWithFlags(pe->ev[ph], st, cudaEventRecordExternal)
                                   : cudaEventRecord(pe->ev[ph], st));
}

int create_events(PhaseEvents &pe) {
    for (int i = 0; i <= kNumPhases; ++i)
        if (cudaEventCreate(&pe.ev[i]) != cudaSuccess) {
            for (int j = 0; j < i; ++j) cudaEventDestroy(pe.ev[j]);
            return GEE_ERR_CUDA;
        }
    return GEE_OK;
}

void destroy_events(PhaseEvents &pe) {
    for (int i = 0; i <= kNumPhases; ++i) cudaEventDestroy(pe.ev[i]);
}

// Receives the events of a timed call once its work is enqueued.
using PhaseSink = std::function<int(const PhaseEvents &)>;

#define GEE_PHASE(ph, cond, launch)                  \
    do {                                             \
        GEE_TRY(mark(pe, ph, st));                   \
        if (cond) {                                  \
            GEE_TRY(cuda_check(launch));             \
            if (pe) pe->ran[ph] = true;              \
        }                                            \
    } while (0)

// The product kernel (k_spmm) of a plan.  Every lane accumulates into a shared-memory
// column of K (rounded up to 8) classes; graphs with K > 8 count their work items on the
// device (length buckets), so they take a full grid.
cudaError_t launch_product(const LaunchPlan &lp, const DeviceInfo &dev, const Ctx &c, cudaStream_t st) {
    const CallBufs &cb = lp.base.cb;
    const int64_t hub_grid_max = cb.hub_cap > 0 ? cb.chunk_cap : 0;
    const int kpad = std::min(kMaxK, (std::max(1, cb.kmax) + 7) & ~7);
    const int wi = cb.ringw ? 1 : 0;
    // ring depth: the requested one, or automatically the depth that keeps at least two
    // CTAs per SM while their shared memory takes the least of the SM (the rest is L1,
    // which caches the node-table gathers: on a power-law graph, three CTAs with a small
    // L1 ran slower than two with a large one); ties go to the deeper ring
    auto occ_of = [&](int r) { return dev.occ_spmm[r >= 8 ? 2 : (r >= 4 ? 1 : 0)][kpad / 8 - 1][wi]; };
    int ring = lp.vec;
    if (ring <= 0) {
        ring = 2;
        size_t best = SIZE_MAX;
        for (int r = 2; r <= 8; r <<= 1) {
            const int o = occ_of(r);
            if (o < 2) continue;
            const size_t used = (size_t)o * spmm_smem(kpad, r, wi != 0);
            if (used <= best) {
                best = used;
                ring = r;
            }
        }
    }
    const int socc = std::max(1, occ_of(ring));
    const int64_t row_items = lp.items[kPfxRows];
    int64_t sneed = std::max<int64_t>(std::min<int64_t>(hub_grid_max, 2 * (int64_t)dev.sms),
                                      (row_items + kWarps - 1) / kWarps);
    if (lp.smem_acc) sneed = (int64_t)dev.sms * socc;
    const int sgrid = (int)std::min<int64_t>(sneed, (int64_t)dev.sms * socc);
    if (sgrid <= 0) return cudaSuccess;
    return launch_spmm(c, sgrid, kpad, ring, st);
}

// Enqueue the path: the CSR build, degrees and node table, and (embed) the product with
// its epilogue.  One kernel launch per phase covers every graph of the plan.
int run_plan(const LaunchPlan &lp, const DeviceInfo &dev, cudaStream_t st, PhaseEvents *pe, bool embed) {
    if (pe) std::memset(pe->ran, 0, sizeof(pe->ran));
    Ctx c = lp.base;
    auto ctx = [&](int kind) {
        c.prefix = lp.prefix[kind];
        c.items = lp.items[kind];
        return c;
    };
    const CallBufs &cb = lp.base.cb;
    GEE_PHASE(kPhMemset, lp.zero_bytes > 0, cudaMemsetAsync(lp.zero_base, 0, lp.zero_bytes, st));
    GEE_PHASE(kPhPrep, lp.items[kPfxPrep] > 0, launch_prep(ctx(kPfxPrep), lp.items[kPfxPrep], st));
    GEE_PHASE(kPhOffs1, lp.items[kPfxOffs1] > 0, launch_offsets(ctx(kPfxOffs1), lp.items[kPfxOffs1], false, st));
    GEE_PHASE(kPhScat1, lp.items[kPfxScat1] > 0,
              launch_scatter(ctx(kPfxScat1), lp.items[kPfxScat1], false, lp.b1max, st));
    GEE_PHASE(kPhCount, lp.items[kPfxCount] > 0, launch_count(ctx(kPfxCount), lp.items[kPfxCount], st));
    GEE_PHASE(kPhOffs2, lp.items[kPfxOffs2] > 0, launch_offsets(ctx(kPfxOffs2), lp.items[kPfxOffs2], true, st));
    GEE_PHASE(kPhScatF, lp.items[kPfxScatF] > 0, launch_scatter(ctx(kPfxScatF), lp.items[kPfxScatF], true, lp.fmax, st));
    GEE_PHASE(kPhRowscan, lp.items[kPfxScan] > 0, launch_rowscan(ctx(kPfxScan), lp.items[kPfxScan], st));
    // k_wdeg and k_spmm take the hub chunks first (CTA by CTA), then the light rows (warp
    // by warp): grids cover whichever part has more parallel work, within one wave
    const int64_t hub_grid_max = cb.hub_cap > 0 ? cb.chunk_cap : 0;
    const int64_t wrow_items = lp.items[kPfxWRows];
    const int64_t wneed = std::max<int64_t>(lp.any_wdeg ? std::min<int64_t>(hub_grid_max, dev.sms) : 0,
                                            (wrow_items + kWarps - 1) / kWarps);
    const int wgrid = (int)std::min<int64_t>(wneed, (int64_t)dev.sms * dev.occ_wdeg);
    GEE_PHASE(kPhWdeg, lp.any_wdeg && wgrid > 0, launch_wdeg(ctx(kPfxWRows), wgrid, st));
    GEE_PHASE(kPhSpmm, embed, launch_product(lp, dev, ctx(kPfxRows), st));
    GEE_TRY(mark(pe, kNumPhases, st));
    return GEE_OK;
}

// ---- one graph ------------------------------------------------------------------------

// FNV-1a hash of a single graph's plan (every scalar field) and of its workspace base: a
// workspace holds what gee_reembed needs only if its last CSR build had the same stamp.
uint32_t plan_stamp(const GraphDesc &d, const char *base) {
    uint32_t h = 2166136261u;
    auto mix = [&](uint64_t v) {
        for (int i = 0; i < 8; ++i) {
            h ^= (uint32_t)(v & 0xffu);
            h *= 16777619u;
            v >>= 8;
        }
    };
    mix((uint64_t)d.E);
    mix((uint64_t)(uint32_t)d.N | ((uint64_t)(uint32_t)d.K << 32));
    mix(d.flags | ((uint64_t)(d.val != nullptr) << 32) | ((uint64_t)d.wdeg << 33));
    const int32_t f[] = {d.nbits, d.ncols, d.pbits, d.row0, d.npass, d.lbits, d.fbits, d.hub_C, d.lpr_log2, d.tiles_e, d.tiles_n,
                         d.scan_tile, d.rows_per_item, d.short_len, d.vec, d.range_tiles, d.ranges};
    for (int32_t x : f) mix((uint64_t)(uint32_t)x);
    for (int i = 0; i <= kBuckets; ++i) mix((uint64_t)(uint32_t)d.bl_off[i]);
    mix((uint64_t)reinterpret_cast<uintptr_t>(base));
    return h == 0u ? 1u : h;  // 0 is the value of a zeroed workspace
}

struct SinglePlan {
    GraphDesc d;
    CallBufs cb;
    size_t zero_bytes = 0;
    size_t total_bytes = 0;
};

// cols / row0: column range and first row of a row shard (cols < 0: a whole graph)
// kmax < 0: the product kernel's classes are K (the sparse path, which does not run it,
// passes 1)
void plan_single(const Shape &s, const gee_opts &o, bool want_deg, char *base, SinglePlan &p, int32_t cols = -1,
                 int32_t row0 = 0, int32_t kmax = -1) {
    std::memset(&p.d, 0, sizeof(p.d));
    std::memset(&p.cb, 0, sizeof(p.cb));
    plan_params(s, o, want_deg, p.d);
    if (cols >= 0) {
        p.d.ncols = cols;
        p.d.pbits = std::max(1, bitlen(cols > 0 ? (uint32_t)(cols - 1) : 0u));
        p.d.row0 = row0;
    }
    p.cb.hub_cap = hub_cap_of(p.d);
    p.cb.chunk_cap = chunk_cap_of(p.d);
    p.cb.kmax = kmax >= 0 ? kmax : s.K;
    Bump b{base};
    layout_call_zero(b, p.cb);
    p.d.status = b.take<uint32_t>(1);
    layout_zero(b, p.d);
    p.zero_bytes = (b.off + kAlign - 1) & ~(kAlign - 1);
    layout_rest(b, p.d, s.weighted);
    layout_call_rest(b, p.cb, 1);
    p.total_bytes = (b.off + kAlign - 1) & ~(kAlign - 1);
    p.d.stamp = plan_stamp(p.d, base);
}

LaunchPlan launch_plan_single(const SinglePlan &p) {
    LaunchPlan lp;
    std::memset(&lp.base, 0, sizeof(lp.base));
    std::memset(lp.prefix, 0, sizeof(lp.prefix));
    std::memset(lp.items, 0, sizeof(lp.items));
    lp.base.g0 = p.d;
    lp.base.G = 1;
    lp.base.cb = p.cb;
    plan_accumulate(lp, p.d);
    lp.zero_base = p.cb.cs;
    lp.zero_bytes = p.zero_bytes;
    return lp;
}

int run_single(const SinglePlan &p, const DeviceInfo &dev, cudaStream_t st, PhaseEvents *pe, bool embed) {
    return run_plan(launch_plan_single(p), dev, st, pe, embed);
}

int check_ws(void *ws, size_t bytes, size_t need) {
    if (need == 0) return GEE_OK;
    if (!ws || (reinterpret_cast<uintptr_t>(ws) & (kAlign - 1)) || bytes < need) return GEE_ERR_WORKSPACE;
    return GEE_OK;
}

int check_inputs(const int32_t *src, const int32_t *dst, int64_t E, int32_t N, const int32_t *labels) {
    if (E > 0 && (!src || !dst)) return GEE_ERR_ARG;
    if (N > 0 && !labels) return GEE_ERR_ARG;
    return GEE_OK;
}

}  // namespace
}  // namespace gee

using namespace gee;

extern "C" {

int gee_version(void) { return 100; }

const char *gee_strerror(int code) {
    switch (code) {
        case GEE_OK: return "success";
        case GEE_ERR_ARG: return "invalid argument";
        case GEE_ERR_TOO_LARGE: return "size beyond the supported limits (N <= 2^21, E < 2^30, K <= 64)";
        case GEE_ERR_WORKSPACE: return "workspace missing, too small or not 256-byte aligned";
        case GEE_ERR_CUDA: return "CUDA runtime error";
        case GEE_ERR_DATA: return "the device reported invalid input data (see status bits)";
        case GEE_ERR_NOMEM: return "the memory budget cannot hold the request";
        case GEE_PENDING: return "the request has not completed yet";
        case GEE_ERR_STATE: return "unknown ticket or request state does not allow this";
        default: return "unknown error";
    }
}

size_t gee_workspace_size(int64_t E, int32_t N, int32_t K, int weighted, const gee_opts *opts) {
    if (check_shape(E, N, K) != GEE_OK) return 0;
    SinglePlan p;
    plan_single(Shape{E, N, K, weighted != 0}, opts_or_default(opts), false, nullptr, p);
    return p.total_bytes;
}

}  // extern "C"

namespace gee {
namespace {

// ---- launch-graph cache of gee_embed ------------------------------------------------
// An argument set seen once launches directly and is remembered; the second call with
// it captures the launch sequence (kernels, memset, status copy) on a private stream
// and instantiates it; later calls replay the executable graph with one launch.
struct EmbedKey {
    int device;
    const void *src, *dst, *w, *labels, *Z, *ws, *status;
    int64_t E;
    int32_t N, K;
    gee_opts o;
    size_t ws_bytes;
    bool timed;  // gee_embed_timed: the graph records the phase events
    int kind;    // 0 gee_embed, 1 gee_reembed
    bool operator==(const EmbedKey &b) const {
        return device == b.device && kind == b.kind && src == b.src && dst == b.dst && w == b.w && labels == b.labels && Z == b.Z &&
               ws == b.ws && status == b.status && E == b.E && N == b.N && K == b.K && o.flags == b.o.flags &&
               o.hub_threshold == b.o.hub_threshold && o.lanes_per_row == b.o.lanes_per_row &&
               o.rows_per_item == b.o.rows_per_item && o.vec_width == b.o.vec_width &&
               o.short_len == b.o.short_len && ws_bytes == b.ws_bytes && timed == b.timed;
    }
};

struct GraphCacheEntry {
    EmbedKey key;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;  // null: seen once, not captured yet
    uint64_t used = 0;
    PhaseEvents pe;        // timed entries: the events the graph records
    bool have_pe = false;
};

constexpr size_t kGraphCacheSize = 16;
std::mutex g_cache_mu;
std::vector<GraphCacheEntry> *g_cache = nullptr;  // never freed: no CUDA calls at exit
uint64_t g_cache_clock = 0;

void drop_entry(GraphCacheEntry &e) {
    if (e.exec) cudaGraphExecDestroy(e.exec);
    if (e.graph) cudaGraphDestroy(e.graph);
    if (e.have_pe) destroy_events(e.pe);
    e.exec = nullptr;
    e.graph = nullptr;
    e.have_pe = false;
}

// Enqueue fn(stream, events) for `key`: directly (with the caller's events pe), or
// through the cached graph (timed keys: with the entry's own events, captured as event
// nodes).  A timed call's sink then gets the events that were used, under the lock.
template <class F>
int launch_cached(const EmbedKey &key, cudaStream_t st, F &&fn, PhaseEvents *pe, const PhaseSink *sink) {
    auto direct = [&]() -> int {
        GEE_TRY(fn(st, pe));
        return (pe && sink) ? (*sink)(*pe) : GEE_OK;
    };
    std::lock_guard<std::mutex> lk(g_cache_mu);
    if (!g_cache) g_cache = new std::vector<GraphCacheEntry>();
    GraphCacheEntry *hit = nullptr;
    for (auto &e : *g_cache)
        if (e.key == key) hit = &e;
    if (!hit) {  // first sighting: remember it (evicting the least recently used)
        if (g_cache->size() >= kGraphCacheSize) {
            auto lru = g_cache->begin();
            for (auto it = g_cache->begin(); it != g_cache->end(); ++it)
                if (it->used < lru->used) lru = it;
            drop_entry(*lru);
            g_cache->erase(lru);
        }
        GraphCacheEntry e;
        e.key = key;
        e.used = ++g_cache_clock;
        g_cache->push_back(e);
        return direct();
    }
    hit->used = ++g_cache_clock;
    if (!hit->exec) {
        if (key.timed && !hit->have_pe) {
            GEE_TRY(create_events(hit->pe));
            hit->have_pe = true;
        }
        cudaStream_t cap = nullptr;
        GEE_TRY(cuda_check(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking)));
        int rc = cuda_check(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
        if (rc == GEE_OK) {
            hit->pe.external = true;
            const int run_rc = fn(cap, key.timed ? &hit->pe : nullptr);
            hit->pe.external = false;
            cudaGraph_t graph = nullptr;
            const int end_rc = cuda_check(cudaStreamEndCapture(cap, &graph));
            rc = run_rc != GEE_OK ? run_rc : end_rc;
            if (rc == GEE_OK) rc = cuda_check(cudaGraphInstantiate(&hit->exec, graph, 0));
            if (rc == GEE_OK) hit->graph = graph;
            else if (graph) cudaGraphDestroy(graph);
        }
        cudaStreamDestroy(cap);
        if (rc != GEE_OK) {  // capture is unavailable here: launch directly
            hit->exec = nullptr;
            cudaGetLastError();
            return direct();
        }
    }
    GEE_TRY(cuda_check(cudaGraphLaunch(hit->exec, st)));
    return (key.timed && sink) ? (*sink)(hit->pe) : GEE_OK;
}

int embed_impl(const int32_t *d_src, const int32_t *d_dst, const float *d_w, int64_t E, int32_t N,
               const int32_t *d_labels, int32_t K, const gee_opts *opts, float *d_Z, void *d_workspace,
               size_t workspace_bytes, void *stream, uint32_t *d_status, PhaseEvents *pe,
               const PhaseSink *sink) {
    GEE_TRY(check_shape(E, N, K));
    GEE_TRY(check_inputs(d_src, d_dst, E, N, d_labels));
    if (N > 0 && !d_Z) return GEE_ERR_ARG;
    const gee_opts o = opts_or_default(opts);
    GEE_TRY(check_opts(o));
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (N == 0) {
        if (d_status) GEE_TRY(cuda_check(cudaMemsetAsync(d_status, 0, sizeof(uint32_t), st)));
        if (pe) {
            std::memset(pe->ran, 0, sizeof(pe->ran));
            for (int i = 0; i <= kNumPhases; ++i) GEE_TRY(cuda_check(cudaEventRecord(pe->ev[i], st)));
            if (sink) GEE_TRY((*sink)(*pe));
        }
        return GEE_OK;
    }
    DeviceInfo dev;
    GEE_TRY(device_info(dev));
    SinglePlan p;
    const Shape s{E, N, K, d_w != nullptr};
    plan_single(s, o, false, nullptr, p);
    GEE_TRY(check_ws(d_workspace, workspace_bytes, p.total_bytes));
    plan_single(s, o, false, static_cast<char *>(d_workspace), p);
    p.d.src = d_src;
    p.d.dst = d_dst;
    p.d.w = d_w;
    p.d.y = d_labels;
    p.d.Z = d_Z;
    auto enqueue = [&](cudaStream_t s2, PhaseEvents *pe2) -> int {
        GEE_TRY(run_single(p, dev, s2, pe2, true));
        if (d_status)
            GEE_TRY(cuda_check(
                cudaMemcpyAsync(d_status, p.d.status, sizeof(uint32_t), cudaMemcpyDeviceToDevice, s2)));
        return GEE_OK;
    };
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    GEE_TRY(cuda_check(cudaStreamIsCapturing(st, &cs)));
    if ((o.flags & GEE_NO_GRAPH_CACHE) || cs != cudaStreamCaptureStatusNone) {
        GEE_TRY(enqueue(st, pe));
        return (pe && sink) ? (*sink)(*pe) : GEE_OK;
    }
    EmbedKey key;
    std::memset(&key, 0, sizeof(key));
    cudaGetDevice(&key.device);
    key.src = d_src;
    key.dst = d_dst;
    key.w = d_w;
    key.labels = d_labels;
    key.Z = d_Z;
    key.ws = d_workspace;
    key.status = d_status;
    key.E = E;
    key.N = N;
    key.K = K;
    key.o = o;
    key.ws_bytes = workspace_bytes;
    key.timed = pe != nullptr;
    return launch_cached(key, st, enqueue, pe, sink);
}
}  // namespace
}  // namespace gee

extern "C" {

int gee_embed(const int32_t *d_src, const int32_t *d_dst, const float *d_w, int64_t E, int32_t N,
              const int32_t *d_labels, int32_t K, const gee_opts *opts, float *d_Z, void *d_workspace,
              size_t workspace_bytes, void *stream, uint32_t *d_status) {
    return embed_impl(d_src, d_dst, d_w, E, N, d_labels, K, opts, d_Z, d_workspace, workspace_bytes, stream,
                      d_status, nullptr, nullptr);
}

}  // extern "C"

// ---- re-embedding with new labels ----------------------------------------------------
namespace gee {
namespace {

int reembed_impl(const int32_t *d_labels, int64_t E, int32_t N, int32_t K, int weighted, const gee_opts *opts,
                 float *d_Z, void *d_workspace, size_t workspace_bytes, void *stream, uint32_t *d_status) {
    GEE_TRY(check_shape(E, N, K));
    if (N > 0 && (!d_labels || !d_Z)) return GEE_ERR_ARG;
    const gee_opts o = opts_or_default(opts);
    GEE_TRY(check_opts(o));
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (N == 0) {
        if (d_status) GEE_TRY(cuda_check(cudaMemsetAsync(d_status, 0, sizeof(uint32_t), st)));
        return GEE_OK;
    }
    DeviceInfo dev;
    GEE_TRY(device_info(dev));
    SinglePlan p;
    const Shape s{E, N, K, weighted != 0};
    plan_single(s, o, false, nullptr, p);
    GEE_TRY(check_ws(d_workspace, workspace_bytes, p.total_bytes));
    plan_single(s, o, false, static_cast<char *>(d_workspace), p);
    p.d.y = d_labels;
    p.d.Z = d_Z;
    const LaunchPlan lp = launch_plan_single(p);
    auto enqueue = [&](cudaStream_t s2, PhaseEvents *) -> int {
        // counters of the product kernel, hub-merge arrivals, status and n_k start at zero;
        // the CSR, degrees, hub chunks and length buckets stay as the last build left them
        GEE_TRY(cuda_check(cudaMemsetAsync(p.cb.cs->ctr, 0, sizeof(p.cb.cs->ctr), s2)));
        if (p.cb.hub_cap) GEE_TRY(cuda_check(cudaMemsetAsync(p.cb.arrive_z, 0, sizeof(uint32_t) * p.cb.hub_cap, s2)));
        GEE_TRY(cuda_check(cudaMemsetAsync(p.d.status, 0, sizeof(uint32_t), s2)));
        GEE_TRY(cuda_check(cudaMemsetAsync(p.d.nk, 0, sizeof(int32_t) * (size_t)K, s2)));
        Ctx c = lp.base;
        c.prefix = lp.prefix[kPfxRows];
        c.items = lp.items[kPfxRows];
        GEE_TRY(cuda_check(launch_relabel(c, s2)));
        GEE_TRY(cuda_check(launch_product(lp, dev, c, s2)));
        if (d_status)
            GEE_TRY(cuda_check(cudaMemcpyAsync(d_status, p.d.status, sizeof(uint32_t), cudaMemcpyDeviceToDevice, s2)));
        return GEE_OK;
    };
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    GEE_TRY(cuda_check(cudaStreamIsCapturing(st, &cs)));
    if ((o.flags & GEE_NO_GRAPH_CACHE) || cs != cudaStreamCaptureStatusNone) return enqueue(st, nullptr);
    EmbedKey key;
    std::memset(&key, 0, sizeof(key));
    cudaGetDevice(&key.device);
    key.kind = 1;
    key.labels = d_labels;
    key.Z = d_Z;
    key.ws = d_workspace;
    key.status = d_status;
    key.w = weighted ? d_workspace : nullptr;
    key.E = E;
    key.N = N;
    key.K = K;
    key.o = o;
    key.ws_bytes = workspace_bytes;
    return launch_cached(key, st, enqueue, nullptr, nullptr);
}

}  // namespace
}  // namespace gee

extern "C" int gee_reembed(const int32_t *d_labels, int64_t E, int32_t N, int32_t K, int weighted,
                           const gee_opts *opts, float *d_Z, void *d_workspace, size_t workspace_bytes, void *stream,
                           uint32_t *d_status) {
    return gee::reembed_impl(d_labels, E, N, K, weighted, opts, d_Z, d_workspace, workspace_bytes, stream,
                             d_status);
}

// ---- row shards of one graph -------------------------------------------------------------
namespace gee {
namespace {

int check_shard(int64_t E, int32_t N, int32_t r0, int32_t r1, int32_t K) {
    GEE_TRY(check_shape(E, N, K));
    if (r0 < 0 || r1 < r0 || r1 > N) return GEE_ERR_ARG;
    return GEE_OK;
}

// The plan of rows [r0, r1) of a graph of N nodes (columns stay global ids).
int shard_plan(int64_t E, int32_t N, int32_t r0, int32_t r1, int32_t K, int weighted, const gee_opts &o, void *ws,
               size_t ws_bytes, SinglePlan &p) {
    GEE_TRY(check_shard(E, N, r0, r1, K));
    GEE_TRY(check_opts(o));
    // the reverse copies of a rank's edges belong to other ranks' rows: not supported
    if (o.flags & GEE_SYMMETRIZE) return GEE_ERR_ARG;
    const Shape s{E, r1 - r0, K, weighted != 0};
    plan_single(s, o, false, nullptr, p, N, r0);
    if (ws == nullptr && ws_bytes == 0) return GEE_OK;  // sizing only
    GEE_TRY(check_ws(ws, ws_bytes, p.total_bytes));
    plan_single(s, o, false, static_cast<char *>(ws), p, N, r0);
    return GEE_OK;
}

}  // namespace
}  // namespace gee

extern "C" {

size_t gee_shard_workspace_size(int64_t E, int32_t N, int32_t r0, int32_t r1, int32_t K, int weighted,
                                const gee_opts *opts) {
    gee::SinglePlan p;
    if (gee::shard_plan(E, N, r0, r1, K, weighted, gee::opts_or_default(opts), nullptr, 0, p) != GEE_OK) return 0;
    return p.total_bytes;
}

int gee_shard_build(const int32_t *d_src, const int32_t *d_dst, const float *d_w, int64_t E, int32_t N, int32_t r0,
                    int32_t r1, const int32_t *d_labels, int32_t K, const gee_opts *opts, int32_t *d_nk,
                    void *d_workspace, size_t workspace_bytes, void *stream, uint32_t *d_status) {
    using namespace gee;
    GEE_TRY(check_inputs(d_src, d_dst, E, r1 - r0, d_labels));
    if (!d_nk) return GEE_ERR_ARG;
    const gee_opts o = opts_or_default(opts);
    SinglePlan p;
    GEE_TRY(shard_plan(E, N, r0, r1, K, d_w != nullptr, o, d_workspace, workspace_bytes, p));
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (r1 == r0) {
        GEE_TRY(cuda_check(cudaMemsetAsync(d_nk, 0, sizeof(int32_t) * (size_t)K, st)));
        if (d_status) GEE_TRY(cuda_check(cudaMemsetAsync(d_status, 0, sizeof(uint32_t), st)));
        return GEE_OK;
    }
    DeviceInfo dev;
    GEE_TRY(device_info(dev));
    p.d.src = d_src;
    p.d.dst = d_dst;
    p.d.w = d_w;
    p.d.y = d_labels;
    GEE_TRY(run_single(p, dev, st, nullptr, false));
    GEE_TRY(cuda_check(cudaMemcpyAsync(d_nk, p.d.nk, sizeof(int32_t) * (size_t)K, cudaMemcpyDeviceToDevice, st)));
    if (d_status)
        GEE_TRY(cuda_check(cudaMemcpyAsync(d_status, p.d.status, sizeof(uint32_t), cudaMemcpyDeviceToDevice, st)));
    return GEE_OK;
}

int gee_shard_table(int64_t E, int32_t N, int32_t r0, int32_t r1, const int32_t *d_labels, int32_t K, int weighted,
                    const gee_opts *opts, const int32_t *d_nk, int32_t *d_tab, void *d_workspace,
                    size_t workspace_bytes, void *stream) {
    using namespace gee;
    if (r1 > r0 && (!d_labels || !d_nk || !d_tab)) return GEE_ERR_ARG;
    const gee_opts o = opts_or_default(opts);
    SinglePlan p;
    GEE_TRY(shard_plan(E, N, r0, r1, K, weighted, o, d_workspace, workspace_bytes, p));
    if (r1 == r0) return GEE_OK;
    p.d.y = d_labels;
    p.d.nk = const_cast<int32_t *>(d_nk);
    p.d.tab = reinterpret_cast<int2 *>(d_tab);
    Ctx c;
    std::memset(&c, 0, sizeof(c));
    c.g0 = p.d;
    c.G = 1;
    c.cb = p.cb;
    return cuda_check(launch_nodetab(c, reinterpret_cast<cudaStream_t>(stream)));
}

int gee_shard_embed(int64_t E, int32_t N, int32_t r0, int32_t r1, const int32_t *d_labels, int32_t K, int weighted,
                    const gee_opts *opts, const int32_t *d_tab, float *d_Z, void *d_workspace,
                    size_t workspace_bytes, void *stream, uint32_t *d_status) {
    using namespace gee;
    if (r1 > r0 && (!d_labels || !d_tab || !d_Z)) return GEE_ERR_ARG;
    const gee_opts o = opts_or_default(opts);
    SinglePlan p;
    GEE_TRY(shard_plan(E, N, r0, r1, K, weighted, o, d_workspace, workspace_bytes, p));
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (r1 == r0) {
        if (d_status) GEE_TRY(cuda_check(cudaMemsetAsync(d_status, 0, sizeof(uint32_t), st)));
        return GEE_OK;
    }
    DeviceInfo dev;
    GEE_TRY(device_info(dev));
    p.d.y = d_labels;
    p.d.Z = d_Z;
    p.d.tab = reinterpret_cast<int2 *>(const_cast<int32_t *>(d_tab));  // the gathered table of all N nodes
    const LaunchPlan lp = launch_plan_single(p);
    GEE_TRY(cuda_check(cudaMemsetAsync(p.cb.cs->ctr, 0, sizeof(p.cb.cs->ctr), st)));
    if (p.cb.hub_cap) GEE_TRY(cuda_check(cudaMemsetAsync(p.cb.arrive_z, 0, sizeof(uint32_t) * p.cb.hub_cap, st)));
    GEE_TRY(cuda_check(cudaMemsetAsync(p.d.status, 0, sizeof(uint32_t), st)));
    Ctx c = lp.base;
    c.prefix = lp.prefix[kPfxRows];
    c.items = lp.items[kPfxRows];
    GEE_TRY(cuda_check(launch_stamp_check(c, st)));
    GEE_TRY(cuda_check(launch_product(lp, dev, c, st)));
    if (d_status)
        GEE_TRY(cuda_check(cudaMemcpyAsync(d_status, p.d.status, sizeof(uint32_t), cudaMemcpyDeviceToDevice, st)));
    return GEE_OK;
}

}  // extern "C"

// ---- autotuner --------------------------------------------------------------------------
namespace gee {
namespace {

struct TuneEntry {
    int device;
    int64_t E;
    int32_t N, K;
    int weighted;
    gee_opts fixed;  // the caller's opts (flags and the fields it fixed)
    gee_opts best;
    float ms;
};

std::mutex g_tune_mu;
std::vector<TuneEntry> *g_tune = nullptr;  // never freed

bool same_opts(const gee_opts &a, const gee_opts &b) {
    return a.flags == b.flags && a.hub_threshold == b.hub_threshold && a.lanes_per_row == b.lanes_per_row &&
           a.rows_per_item == b.rows_per_item && a.vec_width == b.vec_width && a.short_len == b.short_len;
}

// The values the autotuner tries for each tuning field, around the automatic ones (a
// field the caller set to a non-zero value stays fixed).  The search is by coordinates:
// starting from the automatic options, each field in turn takes the value of its list
// that runs fastest with the others at their best so far.
struct TuneAxes {
    std::vector<int32_t> vec, shortl, hub, rpi;
};

TuneAxes tune_axes(const Shape &s, const gee_opts &o) {
    GraphDesc d;
    std::memset(&d, 0, sizeof(d));
    plan_params(s, o, false, d);
    TuneAxes ax;
    auto add = [](std::vector<int32_t> &v, int32_t x) {
        if (std::find(v.begin(), v.end(), x) == v.end()) v.push_back(x);
    };
    // an automatic ring depth is resolved: the tuner always returns an explicit one
    if (o.vec_width == 0)
        for (int32_t v : {8, 4, 2}) add(ax.vec, v);
    else
        add(ax.vec, d.vec);
    add(ax.shortl, d.short_len);
    if (o.short_len == 0 && s.K > kRegK)
        for (int32_t v : {32, 64, 128}) add(ax.shortl, v);
    add(ax.hub, d.hub_C);
    if (o.hub_threshold == 0) {
        add(ax.hub, std::max(1024, d.hub_C / 2));
        add(ax.hub, d.hub_C * 2);
    }
    add(ax.rpi, d.rows_per_item);
    if (o.rows_per_item == 0) {
        add(ax.rpi, std::max(1, d.rows_per_item / 4));
        add(ax.rpi, std::min(32, d.rows_per_item * 4));
    }
    return ax;
}

gee_opts with_fields(gee_opts o, int32_t vec, int32_t shortl, int32_t hub, int32_t rpi) {
    o.vec_width = vec;
    o.short_len = shortl;
    o.hub_threshold = hub;
    o.rows_per_item = rpi;
    return o;
}

}  // namespace
}  // namespace gee

extern "C" {

size_t gee_autotune_workspace_size(int64_t E, int32_t N, int32_t K, int weighted, const gee_opts *opts) {
    if (check_shape(E, N, K) != GEE_OK) return 0;
    const gee_opts o = opts_or_default(opts);
    const TuneAxes ax = tune_axes(Shape{E, N, K, weighted != 0}, o);
    size_t m = 0;
    for (int32_t h : ax.hub)
        for (int32_t r : ax.rpi) {
            const gee_opts c = with_fields(o, ax.vec[0], ax.shortl[0], h, r);
            m = std::max(m, gee_workspace_size(E, N, K, weighted, &c));
        }
    return m;
}

int gee_autotune(const int32_t *d_src, const int32_t *d_dst, const float *d_w, int64_t E, int32_t N,
                 const int32_t *d_labels, int32_t K, const gee_opts *opts, float *d_Z, void *d_workspace,
                 size_t workspace_bytes, void *stream, gee_opts *best, float *best_ms) {
    if (!best) return GEE_ERR_ARG;
    GEE_TRY(check_shape(E, N, K));
    const gee_opts o = opts_or_default(opts);
    GEE_TRY(check_opts(o));
    int dev = 0;
    GEE_TRY(cuda_check(cudaGetDevice(&dev)));
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        if (g_tune)
            for (const TuneEntry &t : *g_tune)
                if (t.device == dev && t.E == E && t.N == N && t.K == K && t.weighted == (d_w != nullptr) &&
                    same_opts(t.fixed, o)) {
                    *best = t.best;
                    if (best_ms) *best_ms = t.ms;
                    return GEE_OK;
                }
    }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    GEE_TRY(cuda_check(cudaEventCreate(&e0)));
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return GEE_ERR_CUDA;
    }
    constexpr int kReps = 3;
    int rc = GEE_OK;
    // mean time of kReps calls with candidate c (after one warm-up), or < 0 if it does not
    // fit the workspace
    auto time_of = [&](const gee_opts &c, float &ms) -> int {
        ms = -1.0f;
        if (gee_workspace_size(E, N, K, d_w != nullptr, &c) > workspace_bytes) return GEE_OK;
        gee_opts run = c;
        run.flags |= GEE_NO_GRAPH_CACHE;  // the candidates do not fill the launch cache
        GEE_TRY(gee_embed(d_src, d_dst, d_w, E, N, d_labels, K, &run, d_Z, d_workspace, workspace_bytes, stream,
                          nullptr));  // warm-up
        GEE_TRY(cuda_check(cudaEventRecord(e0, st)));
        for (int i = 0; i < kReps; ++i)
            GEE_TRY(gee_embed(d_src, d_dst, d_w, E, N, d_labels, K, &run, d_Z, d_workspace, workspace_bytes,
                              stream, nullptr));
        GEE_TRY(cuda_check(cudaEventRecord(e1, st)));
        GEE_TRY(cuda_check(cudaEventSynchronize(e1)));
        GEE_TRY(cuda_check(cudaEventElapsedTime(&ms, e0, e1)));
        ms /= kReps;
        return GEE_OK;
    };
    const TuneAxes ax = tune_axes(Shape{E, N, K, d_w != nullptr}, o);
    int32_t cur[4] = {ax.vec[0], ax.shortl[0], ax.hub[0], ax.rpi[0]};
    const std::vector<int32_t> *axes[4] = {&ax.vec, &ax.shortl, &ax.hub, &ax.rpi};
    float best_t = -1.0f;
    gee_opts pick = o;
    rc = time_of(with_fields(o, cur[0], cur[1], cur[2], cur[3]), best_t);
    if (rc == GEE_OK && best_t >= 0.0f) pick = with_fields(o, cur[0], cur[1], cur[2], cur[3]);
    for (int a = 0; a < 4 && rc == GEE_OK; ++a)
        for (int32_t v : *axes[a]) {
            if (v == cur[a]) continue;
            int32_t trial[4] = {cur[0], cur[1], cur[2], cur[3]};
            trial[a] = v;
            const gee_opts c = with_fields(o, trial[0], trial[1], trial[2], trial[3]);
            float ms = -1.0f;
            rc = time_of(c, ms);
            if (rc != GEE_OK) break;
            if (ms >= 0.0f && (best_t < 0.0f || ms < best_t)) {
                best_t = ms;
                pick = c;
                cur[a] = v;
            }
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != GEE_OK) return rc;
    if (best_t < 0.0f) return GEE_ERR_WORKSPACE;  // no candidate fits the workspace
    *best = pick;
    if (best_ms) *best_ms = best_t;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    if (!g_tune) g_tune = new std::vector<TuneEntry>();
    TuneEntry t;
    t.device = dev;
    t.E = E;
    t.N = N;
    t.K = K;
    t.weighted = d_w != nullptr;
    t.fixed = o;
    t.best = pick;
    t.ms = best_t;
    g_tune->push_back(t);
    return GEE_OK;
}

// ---- persistent autotuner cache: one JSON object per line, keyed by the GPU's name ----
namespace {

std::string device_name(int dev) {
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) {
        cudaGetLastError();
        return std::string();
    }
    std::string n(prop.name);
    for (char &ch : n)
        if (ch == '"' || ch == '\\' || (unsigned char)ch < 0x20) ch = '_';
    return n;
}

}  // namespace

int gee_tune_cache_save(const char *path) {
    if (!path) return GEE_ERR_ARG;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    FILE *f = std::fopen(path, "w");
    if (!f) return GEE_ERR_ARG;
    std::fprintf(f, "{\"format\": \"gee-tune-1\", \"entries\": [\n");
    size_t i = 0, n = g_tune ? g_tune->size() : 0;
    if (g_tune)
        for (const TuneEntry &t : *g_tune) {
            const gee_opts &a = t.fixed, &b = t.best;
            std::fprintf(f,
                         "{\"gpu\": \"%s\", \"E\": %lld, \"N\": %d, \"K\": %d, \"weighted\": %d, "
                         "\"fixed\": [%u, %d, %d, %d, %d, %d], \"best\": [%u, %d, %d, %d, %d, %d], \"ms\": %.9g}%s\n",
                         device_name(t.device).c_str(), (long long)t.E, t.N, t.K, t.weighted, a.flags, a.hub_threshold,
                         a.lanes_per_row, a.rows_per_item, a.vec_width, a.short_len, b.flags, b.hub_threshold,
                         b.lanes_per_row, b.rows_per_item, b.vec_width, b.short_len, (double)t.ms,
                         ++i < n ? "," : "");
        }
    std::fprintf(f, "]}\n");
    return std::fclose(f) == 0 ? GEE_OK : GEE_ERR_ARG;
}

int gee_tune_cache_load(const char *path, int *loaded) {
    if (loaded) *loaded = 0;
    if (!path) return GEE_ERR_ARG;
    int dev = 0;
    const std::string here = cudaGetDevice(&dev) == cudaSuccess ? device_name(dev) : std::string();
    FILE *f = std::fopen(path, "r");
    if (!f) return GEE_ERR_ARG;
    char line[1024];
    int count = 0, rc = GEE_OK;
    bool header = false;
    std::vector<TuneEntry> add;
    while (std::fgets(line, sizeof(line), f)) {
        if (std::strstr(line, "\"format\": \"gee-tune-1\"")) {
            header = true;
            continue;
        }
        if (!std::strstr(line, "\"gpu\"")) continue;
        char gpu[256] = {0};
        long long E = 0;
        TuneEntry t;
        std::memset(&t, 0, sizeof(t));
        double ms = 0.0;
        const int got = std::sscanf(
            line,
            " {\"gpu\": \"%255[^\"]\", \"E\": %lld, \"N\": %d, \"K\": %d, \"weighted\": %d, "
            "\"fixed\": [%u, %d, %d, %d, %d, %d], \"best\": [%u, %d, %d, %d, %d, %d], \"ms\": %lf",
            gpu, &E, &t.N, &t.K, &t.weighted, &t.fixed.flags, &t.fixed.hub_threshold, &t.fixed.lanes_per_row,
            &t.fixed.rows_per_item, &t.fixed.vec_width, &t.fixed.short_len, &t.best.flags, &t.best.hub_threshold,
            &t.best.lanes_per_row, &t.best.rows_per_item, &t.best.vec_width, &t.best.short_len, &ms);
        if (got != 18) {
            rc = GEE_ERR_ARG;  // a malformed entry: nothing of the file is taken
            break;
        }
        if (here.empty() || here != gpu) continue;  // entries of other GPUs stay in the file only
        if (check_shape(E, t.N, t.K) != GEE_OK || check_opts(t.best) != GEE_OK) {
            rc = GEE_ERR_ARG;
            break;
        }
        t.device = dev;
        t.E = E;
        t.ms = (float)ms;
        add.push_back(t);
    }
    std::fclose(f);
    if (rc == GEE_OK && !header) rc = GEE_ERR_ARG;
    if (rc != GEE_OK) return rc;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    if (!g_tune) g_tune = new std::vector<TuneEntry>();
    for (const TuneEntry &t : add) {
        bool dup = false;
        for (const TuneEntry &o : *g_tune)
            dup = dup || (o.device == t.device && o.E == t.E && o.N == t.N && o.K == t.K &&
                          o.weighted == t.weighted && same_opts(o.fixed, t.fixed));
        if (!dup) {
            g_tune->push_back(t);
            ++count;
        }
    }
    if (loaded) *loaded = count;
    return GEE_OK;
}

int gee_tune_cache_clear(void) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    if (g_tune) g_tune->clear();
    return GEE_OK;
}

int gee_graph_cache_clear(void) {
    std::lock_guard<std::mutex> lk(gee::g_cache_mu);
    if (!gee::g_cache) return GEE_OK;
    int cur = 0;
    const bool have_dev = cudaGetDevice(&cur) == cudaSuccess;
    for (auto &e : *gee::g_cache) {
        if (e.exec && have_dev) cudaSetDevice(e.key.device);
        gee::drop_entry(e);
    }
    if (have_dev) cudaSetDevice(cur);
    gee::g_cache->clear();
    return GEE_OK;
}

int gee_graph_cache_size(int *captured) {
    std::lock_guard<std::mutex> lk(gee::g_cache_mu);
    int n = 0, c = 0;
    if (gee::g_cache)
        for (const auto &e : *gee::g_cache) {
            ++n;
            if (e.exec) ++c;
        }
    if (captured) *captured = c;
    return n;
}

int gee_embed_timed(const int32_t *d_src, const int32_t *d_dst, const float *d_w, int64_t E, int32_t N,
                    const int32_t *d_labels, int32_t K, const gee_opts *opts, float *d_Z, void *d_workspace,
                    size_t workspace_bytes, void *stream, uint32_t *d_status, float *phase_ms) {
    if (!phase_ms) return GEE_ERR_ARG;
    for (int i = 0; i < kNumPhases; ++i) phase_ms[i] = -1.0f;
    PhaseEvents pe;
    GEE_TRY(create_events(pe));
    const PhaseSink sink = [&](const PhaseEvents &used) -> int {
        GEE_TRY(cuda_check(cudaEventSynchronize(used.ev[kNumPhases])));
        for (int i = 0; i < kNumPhases; ++i) {
            float ms = -1.0f;
            if (used.ran[i] && cudaEventElapsedTime(&ms, used.ev[i], used.ev[i + 1]) != cudaSuccess) ms = -1.0f;
            phase_ms[i] = ms;
        }
        return GEE_OK;
    };
    const int rc = embed_impl(d_src, d_dst, d_w, E, N, d_labels, K, opts, d_Z, d_workspace, workspace_bytes,
                              stream, d_status, &pe, &sink);
    destroy_events(pe);
    return rc;
}

int gee_build_csr(const int32_t *d_src, const int32_t *d_dst, const float *d_w, int64_t E, int32_t N,
                  const int32_t *d_labels, int32_t K, const gee_opts *opts, int32_t *d_rowptr, int32_t *d_col,
                  float *d_val, int32_t *d_nk, float *d_deg, void *d_workspace, size_t workspace_bytes, void *stream,
                  uint32_t *d_status) {
    GEE_TRY(check_shape(E, N, K));
    GEE_TRY(check_inputs(d_src, d_dst, E, N, d_labels));
    if (!d_rowptr || (E > 0 && !d_col)) return GEE_ERR_ARG;
    const gee_opts o = opts_or_default(opts);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (N == 0) {
        GEE_TRY(cuda_check(cudaMemsetAsync(d_rowptr, 0, sizeof(int32_t), st)));
        if (d_nk) GEE_TRY(cuda_check(cudaMemsetAsync(d_nk, 0, sizeof(int32_t) * K, st)));
        if (d_status) GEE_TRY(cuda_check(cudaMemsetAsync(d_status, 0, sizeof(uint32_t), st)));
        return GEE_OK;
    }
    DeviceInfo dev;
    GEE_TRY(device_info(dev));
    SinglePlan p;
    const Shape s{E, N, K, d_w != nullptr};
    plan_single(s, o, true, nullptr, p);
    GEE_TRY(check_ws(d_workspace, workspace_bytes, p.total_bytes));
    plan_single(s, o, true, static_cast<char *>(d_workspace), p);
    p.d.src = d_src;
    p.d.dst = d_dst;
    p.d.w = d_w;
    p.d.y = d_labels;
    p.d.Z = nullptr;
    const GraphDesc &d = p.d;
    GEE_TRY(run_single(p, dev, st, nullptr, false));
    GEE_TRY(cuda_check(cudaMemcpyAsync(d_rowptr, d.rowptr, sizeof(int32_t) * ((size_t)N + 1),
                                       cudaMemcpyDeviceToDevice, st)));
    const int64_t cap = d.E;  // E, or 2E with GEE_SYMMETRIZE (rowptr[N] entries are used)
    if (cap > 0) {
        GEE_TRY(cuda_check(
            cudaMemcpyAsync(d_col, d.col, sizeof(int32_t) * (size_t)cap, cudaMemcpyDeviceToDevice, st)));
        if (d_val) {
            if (d.val)
                GEE_TRY(cuda_check(
                    cudaMemcpyAsync(d_val, d.val, sizeof(float) * (size_t)cap, cudaMemcpyDeviceToDevice, st)));
            else
                GEE_TRY(cuda_check(launch_fill(d_val, cap, 1.0f, st)));
        }
    }
    if (d_nk)
        GEE_TRY(cuda_check(cudaMemcpyAsync(d_nk, d.nk, sizeof(int32_t) * (size_t)K, cudaMemcpyDeviceToDevice, st)));
    if (d_deg)
        GEE_TRY(cuda_check(cudaMemcpyAsync(d_deg, d.deg, sizeof(float) * (size_t)N, cudaMemcpyDeviceToDevice, st)));
    if (d_status)
        GEE_TRY(cuda_check(cudaMemcpyAsync(d_status, d.status, sizeof(uint32_t), cudaMemcpyDeviceToDevice, st)));
    return GEE_OK;
}

int gee_class_counts(const int32_t *d_rowptr, const int32_t *d_col, int32_t N, const int32_t *d_labels, int32_t K,
                     int32_t *d_C, void *stream) {
    if (N < 0 || K < 1) return GEE_ERR_ARG;
    if (K > GEE_MAX_K || N > GEE_MAX_N) return GEE_ERR_TOO_LARGE;
    if (N == 0) return GEE_OK;
    if (!d_rowptr || !d_col || !d_labels || !d_C) return GEE_ERR_ARG;
    DeviceInfo dev;
    GEE_TRY(device_info(dev));
    const int blocks = (int)std::min<int64_t>(((int64_t)N + 3) / 4, (int64_t)dev.sms * 8);
    return cuda_check(launch_class_counts(d_rowptr, d_col, N, d_labels, K, d_C, blocks,
                                          reinterpret_cast<cudaStream_t>(stream)));
}

size_t gee_host_workspace_size(int64_t E, int32_t N, int32_t K, int weighted, const gee_opts *opts) {
    if (check_shape(E, N, K) != GEE_OK) return 0;
    Bump b{nullptr};
    b.take<int32_t>((size_t)E);
    b.take<int32_t>((size_t)E);
    if (weighted) b.take<float>((size_t)E);
    b.take<int32_t>((size_t)N);
    b.take<float>((size_t)N * (size_t)K);
    b.take<uint32_t>(1);
    const size_t head = (b.off + kAlign - 1) & ~(kAlign - 1);
    return head + gee_workspace_size(E, N, K, weighted, opts);
}

int gee_embed_host(const int32_t *src, const int32_t *dst, const float *w, int64_t E, int32_t N,
                   const int32_t *labels, int32_t K, const gee_opts *opts, float *Z, void *d_workspace,
                   size_t workspace_bytes, void *stream, uint32_t *status) {
    GEE_TRY(check_shape(E, N, K));
    GEE_TRY(check_inputs(src, dst, E, N, labels));
    if (N > 0 && !Z) return GEE_ERR_ARG;
    const size_t need = gee_host_workspace_size(E, N, K, w != nullptr, opts);
    GEE_TRY(check_ws(d_workspace, workspace_bytes, need));
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    Bump b{static_cast<char *>(d_workspace)};
    int32_t *d_src = b.take<int32_t>((size_t)E);
    int32_t *d_dst = b.take<int32_t>((size_t)E);
    float *d_w = w ? b.take<float>((size_t)E) : nullptr;
    int32_t *d_y = b.take<int32_t>((size_t)N);
    float *d_Z = b.take<float>((size_t)N * (size_t)K);
    uint32_t *d_st = b.take<uint32_t>(1);
    const size_t head = (b.off + kAlign - 1) & ~(kAlign - 1);
    if (E > 0) {
        GEE_TRY(cuda_check(cudaMemcpyAsync(d_src, src, sizeof(int32_t) * (size_t)E, cudaMemcpyHostToDevice, st)));
        GEE_TRY(cuda_check(cudaMemcpyAsync(d_dst, dst, sizeof(int32_t) * (size_t)E, cudaMemcpyHostToDevice, st)));
        if (w) GEE_TRY(cuda_check(cudaMemcpyAsync(d_w, w, sizeof(float) * (size_t)E, cudaMemcpyHostToDevice, st)));
    }
    if (N > 0)
        GEE_TRY(cuda_check(cudaMemcpyAsync(d_y, labels, sizeof(int32_t) * (size_t)N, cudaMemcpyHostToDevice, st)));
    GEE_TRY(gee_embed(E > 0 ? d_src : nullptr, E > 0 ? d_dst : nullptr, d_w, E, N, d_y, K, opts, d_Z,
                      static_cast<char *>(d_workspace) + head, workspace_bytes - head, stream, d_st));
    uint32_t h_status = 0;
    if (N > 0)
        GEE_TRY(cuda_check(
            cudaMemcpyAsync(Z, d_Z, sizeof(float) * (size_t)N * (size_t)K, cudaMemcpyDeviceToHost, st)));
    GEE_TRY(cuda_check(cudaMemcpyAsync(&h_status, d_st, sizeof(uint32_t), cudaMemcpyDeviceToHost, st)));
    GEE_TRY(cuda_check(cudaStreamSynchronize(st)));
    if (status) *status = h_status;
    return h_status ? GEE_ERR_DATA : GEE_OK;
}

}  // extern "C"

// =====================================================================================
// Sparse Z (CSR over classes) for many classes

namespace gee {
namespace {

int check_sparse_shape(int64_t E, int32_t N, int32_t K) {
    if (E < 0 || N < 0 || K < 1) return GEE_ERR_ARG;
    if (N > GEE_MAX_N || E >= GEE_MAX_E || K > GEE_MAX_K_SPARSE) return GEE_ERR_TOO_LARGE;
    return GEE_OK;
}

// The CSR build's plan (no product-kernel buffers), then the sparse path's scratch.
void plan_sparse(const Shape &s, const gee_opts &o, char *base, SinglePlan &p, SparseArgs &a, size_t &total) {
    plan_single(s, o, false, base, p, -1, 0, 1);
    Bump b{base};
    b.off = p.total_bytes;
    const int64_t E = p.d.E, N = s.N;
    std::memset(&a, 0, sizeof(a));
    a.cnt = b.take<int32_t>((size_t)N);
    a.long_cap = (uint32_t)sparse_long_cap(E);
    a.long_list = b.take<int32_t>(a.long_cap);
    a.long_count = b.take<uint32_t>(2);
    a.chunk_cap = (uint32_t)sparse_chunk_cap(E);
    a.chunk_off = b.take<uint32_t>((size_t)a.long_cap + 1);
    a.chunk_cnt = b.take<int32_t>(a.chunk_cap);
    a.tile_sum = b.take<uint32_t>((size_t)sparse_scan_tiles(s.N) + 1);
    a.wstart = b.take<int32_t>((size_t)sparse_windows(E) + 1);
    a.runs_a = b.take<int4>((size_t)(E + N));
    a.runs_b = b.take<int4>((size_t)(E + N));
    total = (b.off + kAlign - 1) & ~(kAlign - 1);
}

}  // namespace
}  // namespace gee

extern "C" {

size_t gee_sparse_workspace_size(int64_t E, int32_t N, int32_t K, int weighted, const gee_opts *opts) {
    if (check_sparse_shape(E, N, K) != GEE_OK) return 0;
    const gee_opts o = opts_or_default(opts);
    if (check_opts(o) != GEE_OK) return 0;
    SinglePlan p;
    SparseArgs a;
    size_t total = 0;
    plan_sparse(Shape{E, N, K, weighted != 0}, o, nullptr, p, a, total);
    return total;
}

int gee_embed_sparse(const int32_t *d_src, const int32_t *d_dst, const float *d_w, int64_t E, int32_t N,
                     const int32_t *d_labels, int32_t K, const gee_opts *opts, int32_t *d_zrowptr, int32_t *d_zcol,
                     float *d_zval, int64_t zcap, void *d_workspace, size_t workspace_bytes, void *stream,
                     uint32_t *d_status) {
    GEE_TRY(check_sparse_shape(E, N, K));
    GEE_TRY(check_inputs(d_src, d_dst, E, N, d_labels));
    const gee_opts o = opts_or_default(opts);
    GEE_TRY(check_opts(o));
    const int64_t entries = (o.flags & GEE_SYMMETRIZE) ? 2 * E : E;
    if (!d_zrowptr || (N > 0 && (!d_zcol || !d_zval)) || zcap < entries + N) return GEE_ERR_ARG;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (N == 0) {
        GEE_TRY(cuda_check(cudaMemsetAsync(d_zrowptr, 0, sizeof(int32_t), st)));
        if (d_status) GEE_TRY(cuda_check(cudaMemsetAsync(d_status, 0, sizeof(uint32_t), st)));
        return GEE_OK;
    }
    DeviceInfo dev;
    GEE_TRY(device_info(dev));
    const Shape s{E, N, K, d_w != nullptr};
    SinglePlan p;
    SparseArgs a;
    size_t total = 0;
    plan_sparse(s, o, nullptr, p, a, total);
    GEE_TRY(check_ws(d_workspace, workspace_bytes, total));
    plan_sparse(s, o, static_cast<char *>(d_workspace), p, a, total);
    p.d.src = d_src;
    p.d.dst = d_dst;
    p.d.w = d_w;
    p.d.y = d_labels;
    p.d.Z = nullptr;
    GEE_TRY(run_single(p, dev, st, nullptr, false));  // CSR, degrees, node table
    const GraphDesc &d = p.d;
    a.rowptr = d.rowptr;
    a.col = d.col;
    a.val = d.val;
    a.y = d_labels;
    a.tab = d.tab;
    a.dinv = d.dinv;
    a.N = N;
    a.K = K;
    a.E = d.E;
    a.flags = o.flags & (GEE_DIAG_AUG | GEE_LAPLACIAN | GEE_CORRELATION);
    a.zrowptr = d_zrowptr;
    a.zcol = d_zcol;
    a.zval = d_zval;
    a.zcap = zcap;
    a.status = d.status;
    GEE_TRY(cuda_check(cudaMemsetAsync(a.long_count, 0, 2 * sizeof(uint32_t), st)));
    GEE_TRY(cuda_check(launch_sparse(a, dev.sms, st)));
    if (d_status)
        GEE_TRY(cuda_check(cudaMemcpyAsync(d_status, d.status, sizeof(uint32_t), cudaMemcpyDeviceToDevice, st)));
    return GEE_OK;
}

}  // extern "C"

// =====================================================================================
// Many graphs in one launch sequence

struct gee_batch_plan {
    int32_t G = 0;
    std::vector<unsigned char> staging;  // host copy of the descriptors and item prefixes
    void *d_meta = nullptr;              // their place in the workspace
    gee::LaunchPlan lp;
    uint32_t *d_statuses = nullptr;      // [G] status words, contiguous
    int device = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

namespace gee {
namespace {

constexpr int32_t kBatchRangeTiles = 8;  // 16K-edge ranges: many ranges, one CTA each

struct BatchLayout {
    std::vector<GraphDesc> descs;
    std::vector<int32_t> prefix;  // [kNumPfx][G + 1]
    LaunchPlan lp;
    uint32_t *statuses = nullptr;
    GraphDesc *d_descs = nullptr;
    int32_t *d_prefix = nullptr;
    size_t meta_bytes = 0;
    size_t total_bytes = 0;
};

int check_graph(const gee_graph &g) {
    GEE_TRY(check_shape(g.E, g.N, g.K));
    GEE_TRY(check_inputs(g.src, g.dst, g.E, g.N, g.labels));
    if (g.N > 0 && !g.Z) return GEE_ERR_ARG;
    return GEE_OK;
}

int plan_batch(const gee_graph *graphs, int32_t G, const gee_opts &o, char *base, BatchLayout &L) {
    if (G < 1 || !graphs) return GEE_ERR_ARG;
    GEE_TRY(check_opts(o));
    L.descs.assign((size_t)G, GraphDesc{});
    CallBufs cb;
    std::memset(&cb, 0, sizeof(cb));
    cb.kmax = 1;
    uint64_t hub_cap = 0, chunk_cap = 0;
    int64_t rows = 0;
    for (int32_t g = 0; g < G; ++g) {
        GEE_TRY(check_graph(graphs[g]));
        rows += graphs[g].N;
    }
    for (int32_t g = 0; g < G; ++g) {
        GraphDesc &d = L.descs[g];
        std::memset(&d, 0, sizeof(d));
        plan_params(Shape{graphs[g].E, graphs[g].N, graphs[g].K, graphs[g].w != nullptr}, o, false, d, rows);
        // ranges of at least 8 tiles (one CTA each, many graphs in flight); never more
        // ranges than the graph alone would use, so a batch needs no more workspace
        // than its graphs would separately.  Only how work is cut changes, never Z.
        set_ranges(d, std::max(kBatchRangeTiles, d.range_tiles));
        hub_cap += hub_cap_of(d);
        chunk_cap += chunk_cap_of(d);
        cb.kmax = std::max(cb.kmax, d.K);
    }
    if (hub_cap >= 0xffffffffull || chunk_cap >= 0xffffffffull) return GEE_ERR_TOO_LARGE;
    cb.hub_cap = (uint32_t)hub_cap;
    cb.chunk_cap = (uint32_t)chunk_cap;
    Bump b{base};
    layout_call_zero(b, cb);
    L.statuses = b.take<uint32_t>((size_t)G);
    for (int32_t g = 0; g < G; ++g) {
        layout_zero(b, L.descs[g]);
        L.descs[g].status = L.statuses ? L.statuses + g : nullptr;
    }
    const size_t zero_bytes = (b.off + kAlign - 1) & ~(kAlign - 1);
    L.d_descs = b.take<GraphDesc>((size_t)G);
    L.d_prefix = b.take<int32_t>((size_t)kNumPfx * (G + 1));
    L.meta_bytes = (reinterpret_cast<size_t>(L.d_prefix) + sizeof(int32_t) * (size_t)kNumPfx * (G + 1)) -
                   reinterpret_cast<size_t>(L.d_descs);
    for (int32_t g = 0; g < G; ++g) layout_rest(b, L.descs[g], graphs[g].w != nullptr);
    layout_call_rest(b, cb, G);
    L.total_bytes = (b.off + kAlign - 1) & ~(kAlign - 1);

    LaunchPlan &lp = L.lp;
    std::memset(&lp.base, 0, sizeof(lp.base));
    std::memset(lp.items, 0, sizeof(lp.items));
    lp.base.G = G;
    lp.base.graphs = L.d_descs;
    lp.base.cb = cb;
    L.prefix.assign((size_t)kNumPfx * (G + 1), 0);
    for (int32_t g = 0; g < G; ++g) {
        GraphDesc &d = L.descs[g];
        d.src = graphs[g].src;
        d.dst = graphs[g].dst;
        d.w = graphs[g].w;
        d.y = graphs[g].labels;
        d.Z = graphs[g].Z;
        int32_t it[kNumPfx];
        plan_items(d, it);
        for (int k = 0; k < kNumPfx; ++k) {
            const int64_t next = (int64_t)L.prefix[(size_t)k * (G + 1) + g] + it[k];
            if (next >= INT32_MAX) return GEE_ERR_TOO_LARGE;
            L.prefix[(size_t)k * (G + 1) + g + 1] = (int32_t)next;
        }
        plan_accumulate(lp, d);
    }
    for (int k = 0; k < kNumPfx; ++k) lp.prefix[k] = L.d_prefix ? L.d_prefix + (size_t)k * (G + 1) : nullptr;
    // the kernels read a lone graph's descriptor from the launch parameters (g0), not
    // from the device array
    if (G == 1) lp.base.g0 = L.descs[0];
    lp.zero_base = cb.cs;
    lp.zero_bytes = zero_bytes;
    return GEE_OK;
}

// host image of [d_descs, d_prefix end) to copy into the workspace
void batch_staging(const BatchLayout &L, std::vector<unsigned char> &out) {
    out.assign(L.meta_bytes, 0);
    std::memcpy(out.data(), L.descs.data(), sizeof(GraphDesc) * L.descs.size());
    const size_t poff = reinterpret_cast<size_t>(L.d_prefix) - reinterpret_cast<size_t>(L.d_descs);
    std::memcpy(out.data() + poff, L.prefix.data(), sizeof(int32_t) * L.prefix.size());
}

int batch_prepare(const gee_graph *graphs, int32_t G, const gee_opts *opts, void *d_ws, size_t ws_bytes,
                  BatchLayout &L) {
    const gee_opts o = opts_or_default(opts);
    GEE_TRY(plan_batch(graphs, G, o, nullptr, L));
    GEE_TRY(check_ws(d_ws, ws_bytes, L.total_bytes));
    return plan_batch(graphs, G, o, static_cast<char *>(d_ws), L);
}

}  // namespace
}  // namespace gee

extern "C" {

size_t gee_batch_workspace_size(const gee_graph *graphs, int32_t G, const gee_opts *opts) {
    gee::BatchLayout L;
    if (gee::plan_batch(graphs, G, gee::opts_or_default(opts), nullptr, L) != GEE_OK) return 0;
    return L.total_bytes;
}

int gee_embed_batch(const gee_graph *graphs, int32_t G, const gee_opts *opts, void *d_workspace,
                    size_t workspace_bytes, void *stream, uint32_t *d_status) {
    gee::BatchLayout L;
    GEE_TRY(gee::batch_prepare(graphs, G, opts, d_workspace, workspace_bytes, L));
    gee::DeviceInfo dev;
    GEE_TRY(gee::device_info(dev));
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    std::vector<unsigned char> staging;
    gee::batch_staging(L, staging);
    GEE_TRY(gee::cuda_check(cudaMemcpyAsync(L.d_descs, staging.data(), staging.size(), cudaMemcpyHostToDevice, st)));
    // the copy reads pageable host memory: it is staged before cudaMemcpyAsync returns
    GEE_TRY(gee::run_plan(L.lp, dev, st, nullptr, true));
    if (d_status)
        GEE_TRY(gee::cuda_check(
            cudaMemcpyAsync(d_status, L.statuses, sizeof(uint32_t) * (size_t)G, cudaMemcpyDeviceToDevice, st)));
    return GEE_OK;
}

int gee_batch_plan_create(const gee_graph *graphs, int32_t G, const gee_opts *opts, void *d_workspace,
                          size_t workspace_bytes, void *stream, gee_batch_plan **out) {
    if (!out) return GEE_ERR_ARG;
    *out = nullptr;
    gee::BatchLayout L;
    GEE_TRY(gee::batch_prepare(graphs, G, opts, d_workspace, workspace_bytes, L));
    gee::DeviceInfo dev;
    GEE_TRY(gee::device_info(dev));
    gee_batch_plan *p = new gee_batch_plan();
    p->G = G;
    p->lp = L.lp;
    p->d_statuses = L.statuses;
    p->d_meta = L.d_descs;
    cudaGetDevice(&p->device);
    gee::batch_staging(L, p->staging);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    int rc = gee::cuda_check(cudaMemcpyAsync(p->d_meta, p->staging.data(), p->staging.size(),
                                             cudaMemcpyHostToDevice, st));
    if (rc == GEE_OK) rc = gee::cuda_check(cudaStreamSynchronize(st));
    if (rc != GEE_OK) {
        delete p;
        return rc;
    }
    *out = p;
    return GEE_OK;
}

int gee_batch_plan_launch(gee_batch_plan *p, void *stream, uint32_t *d_status, int use_graph) {
    if (!p) return GEE_ERR_ARG;
    gee::DeviceInfo dev;
    GEE_TRY(gee::device_info(dev));
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (use_graph) {
        if (!p->exec) {
            cudaStream_t cap = nullptr;
            GEE_TRY(gee::cuda_check(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking)));
            int rc = gee::cuda_check(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
            if (rc == GEE_OK) {
                const int run_rc = gee::run_plan(p->lp, dev, cap, nullptr, true);
                cudaGraph_t graph = nullptr;
                const int end_rc = gee::cuda_check(cudaStreamEndCapture(cap, &graph));
                rc = run_rc != GEE_OK ? run_rc : end_rc;
                if (rc == GEE_OK) rc = gee::cuda_check(cudaGraphInstantiate(&p->exec, graph, 0));
                if (rc == GEE_OK) p->graph = graph;
                else if (graph) cudaGraphDestroy(graph);
            }
            cudaStreamDestroy(cap);
            GEE_TRY(rc);
        }
        GEE_TRY(gee::cuda_check(cudaGraphLaunch(p->exec, st)));
    } else {
        GEE_TRY(gee::run_plan(p->lp, dev, st, nullptr, true));
    }
    if (d_status)
        GEE_TRY(gee::cuda_check(cudaMemcpyAsync(d_status, p->d_statuses, sizeof(uint32_t) * (size_t)p->G,
                                                cudaMemcpyDeviceToDevice, st)));
    return GEE_OK;
}

int gee_batch_plan_launch_timed(gee_batch_plan *p, void *stream, float *phase_ms) {
    if (!p || !phase_ms) return GEE_ERR_ARG;
    gee::DeviceInfo dev;
    GEE_TRY(gee::device_info(dev));
    gee::PhaseEvents pe;
    for (int i = 0; i <= gee::kNumPhases; ++i)
        if (cudaEventCreate(&pe.ev[i]) != cudaSuccess) {
            for (int j = 0; j < i; ++j) cudaEventDestroy(pe.ev[j]);
            return GEE_ERR_CUDA;
        }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    int rc = gee::run_plan(p->lp, dev, st, &pe, true);
    if (rc == GEE_OK && cudaEventSynchronize(pe.ev[gee::kNumPhases]) != cudaSuccess) rc = GEE_ERR_CUDA;
    for (int i = 0; i < gee::kNumPhases; ++i) {
        float ms = -1.0f;
        if (rc == GEE_OK && pe.ran[i] && cudaEventElapsedTime(&ms, pe.ev[i], pe.ev[i + 1]) != cudaSuccess) ms = -1.0f;
        phase_ms[i] = ms;
    }
    for (int i = 0; i <= gee::kNumPhases; ++i) cudaEventDestroy(pe.ev[i]);
    return rc;
}

void gee_batch_plan_destroy(gee_batch_plan *p) {
    if (!p) return;
    if (p->exec) cudaGraphExecDestroy(p->exec);
    if (p->graph) cudaGraphDestroy(p->graph);
    delete p;
}

// The candidates of the batch tuner, around the automatic values (a field the caller set
// stays fixed).  In a batch the fields act by graph class: short_len on the graphs with
// K > 8 (their length buckets), rows_per_item on those with K <= 8 (their row blocks),
// vec_width on the whole product launch; split thresholds stay per graph (automatic).
static void batch_tune_axes(const gee_opts &o, std::vector<int32_t> (&ax)[3]) {
    if (o.vec_width == 0) ax[0] = {8, 4, 2};
    else ax[0] = {o.vec_width};
    if (o.short_len == 0) ax[1] = {256, 64, 128};
    else ax[1] = {o.short_len};
    if (o.rows_per_item == 0) ax[2] = {0, 4, 16, 32};
    else ax[2] = {o.rows_per_item};
}

size_t gee_batch_autotune_workspace_size(const gee_graph *graphs, int32_t G, const gee_opts *opts) {
    const gee_opts o = gee::opts_or_default(opts);
    std::vector<int32_t> ax[3];
    batch_tune_axes(o, ax);
    size_t m = 0;
    for (int32_t v : ax[0])
        for (int32_t sl : ax[1])
            for (int32_t r : ax[2]) {
                gee_opts c = o;
                c.vec_width = v;
                c.short_len = sl;
                c.rows_per_item = r;
                const size_t n = gee_batch_workspace_size(graphs, G, &c);
                if (n == 0) return 0;
                m = std::max(m, n);
            }
    return m;
}

int gee_batch_autotune(const gee_graph *graphs, int32_t G, const gee_opts *opts, void *d_workspace,
                       size_t workspace_bytes, void *stream, gee_opts *best, float *best_ms) {
    if (!best || G < 1) return GEE_ERR_ARG;
    const gee_opts o = gee::opts_or_default(opts);
    GEE_TRY(gee::check_opts(o));
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    GEE_TRY(gee::cuda_check(cudaEventCreate(&e0)));
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return GEE_ERR_CUDA;
    }
    // mean time of two replays (after one captured launch) of a plan with options c
    auto time_of = [&](const gee_opts &c, float &ms) -> int {
        ms = -1.0f;
        if (gee_batch_workspace_size(graphs, G, &c) > workspace_bytes) return GEE_OK;
        gee_batch_plan *plan = nullptr;
        GEE_TRY(gee_batch_plan_create(graphs, G, &c, d_workspace, workspace_bytes, stream, &plan));
        int rc = gee_batch_plan_launch(plan, stream, nullptr, 1);
        if (rc == GEE_OK) rc = gee::cuda_check(cudaEventRecord(e0, st));
        for (int i = 0; i < 2 && rc == GEE_OK; ++i) rc = gee_batch_plan_launch(plan, stream, nullptr, 1);
        if (rc == GEE_OK) rc = gee::cuda_check(cudaEventRecord(e1, st));
        if (rc == GEE_OK) rc = gee::cuda_check(cudaEventSynchronize(e1));
        if (rc == GEE_OK) rc = gee::cuda_check(cudaEventElapsedTime(&ms, e0, e1));
        gee_batch_plan_destroy(plan);
        ms = rc == GEE_OK ? ms / 2.0f : -1.0f;
        return rc;
    };
    std::vector<int32_t> ax[3];
    batch_tune_axes(o, ax);
    int32_t cur[3] = {ax[0][0], ax[1][0], ax[2][0]};
    auto with = [&](const int32_t (&f)[3]) {
        gee_opts c = o;
        c.vec_width = f[0];
        c.short_len = f[1];
        c.rows_per_item = f[2];
        return c;
    };
    float best_t = -1.0f;
    int rc = time_of(with(cur), best_t);
    for (int a = 0; a < 3 && rc == GEE_OK; ++a)
        for (int32_t v : ax[a]) {
            if (v == cur[a]) continue;
            int32_t trial[3] = {cur[0], cur[1], cur[2]};
            trial[a] = v;
            float ms = -1.0f;
            rc = time_of(with(trial), ms);
            if (rc != GEE_OK) break;
            if (ms >= 0.0f && (best_t < 0.0f || ms < best_t)) {
                best_t = ms;
                cur[a] = v;
            }
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != GEE_OK) return rc;
    if (best_t < 0.0f) return GEE_ERR_WORKSPACE;
    *best = with(cur);
    if (best_ms) *best_ms = best_t;
    return GEE_OK;
}

}  // extern "C"
