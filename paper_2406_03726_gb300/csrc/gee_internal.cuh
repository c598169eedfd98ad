// Internal definitions shared by the GEE kernels and the host runtime.
//
// One "graph descriptor" (GraphDesc) carries a graph's inputs, its plan (digit widths,
// split threshold, lanes per row) and the device pointers of its scratch arrays.  Every
// kernel processes a flat list of work items that spans one or many graphs: item i
// belongs to the graph g with prefix[g] <= i < prefix[g+1].  A single-graph call passes
// its descriptor by value in the launch parameters, so it needs no host-to-device copy.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace gee {

// ---- tile geometry --------------------------------------------------------------------
constexpr int kThreads = 256;                  // every kernel uses 256-thread CTAs
constexpr int kWarps = kThreads / 32;
constexpr int kSortItems = 8;                  // keys per thread in a sort pass
constexpr int kSortTile = kThreads * kSortItems;   // 2048 edges per sort tile
constexpr int kPrepTile = 8192;                // edges (or nodes) per histogram tile
constexpr int kScanItems = 8;
constexpr int kScanTile = kThreads * kScanItems;   // at most 2048 nodes per index-pointer tile
constexpr int kMaxDigitBits = 11;
constexpr int kOnePassBits = 8;                 // graphs with ids of at most this many bits take one pass
constexpr int kMaxDigits = 1 << kMaxDigitBits;     // 2048 buckets per radix pass
constexpr int kMaxK = 64;
constexpr int kRegK = 8;                       // K <= 8: per-lane register accumulators
constexpr int kHistCopies = 8;                 // digit totals are spread over 8 copies: fewer
                                               // atomics on one address at the end of k_prep
// K > 8: light rows are listed by length in kBuckets buckets (k_rowscan): buckets 0-5 hold
// rows of at most 8, 16, 32, 64, 128, 256 entries (up to short_len), taken one lane per
// row; the last bucket holds the longer light rows, taken by a whole warp each.
constexpr int kBuckets = 7;
constexpr int kWarpBucket = kBuckets - 1;

constexpr int kSpinLimit = 1 << 22;            // bounded copy waits: ~1 s, then GEE_STATUS_TIMEOUT

// status bits (must equal GEE_STATUS_* in gee.h)
constexpr uint32_t kStIndex = 1u, kStLabel = 2u, kStWeight = 4u, kStTimeout = 8u, kStInternal = 16u,
                   kStStale = 32u;
constexpr uint32_t kOptAug = 1u, kOptLap = 2u, kOptCor = 4u;
constexpr uint32_t kSentinel = 0xffffffffu;  // first-pass value of a dropped element (the reverse
                                             // copy of a self-loop); never a packed key: those
                                             // use at most 31 bits

struct GraphDesc {
    // inputs (device)
    const int32_t *src, *dst;
    const float *w;          // nullptr = unweighted
    const int32_t *y;
    float *Z;
    int64_t E;               // edges sorted into the CSR (2 x Ein with sym): capacity of the CSR
    int64_t Ein;             // edges of the input arrays
    int32_t sym;             // 1: every input edge (i, j, e), i != j, also gives (j, i, e)
    int32_t N, K;
    uint32_t flags;
    // plan
    int32_t nbits;           // bits of a row id (>= 1)
    int32_t ncols;           // column ids are in [0, ncols): N for a whole graph, the global node
                             // count for a row shard
    int32_t pbits;           // bits of a column id (payload of the packed first-pass keys)
    int32_t row0;            // global id of row 0 (0 for a whole graph, the first row of a shard)
    int32_t npass;           // radix passes: 1 (nbits <= kOnePassBits) or 2
    int32_t lbits;           // digit bits of the first pass (2-pass graphs)
    int32_t fbits;           // digit bits of the final pass
    int32_t hub_C;           // rows longer than this are split into chunks of hub_C
    int32_t lpr_log2;        // log2(lanes cooperating on one light row)
    int32_t tiles_e;         // ceil(E / kSortTile)
    int32_t tiles_n;         // ceil(N / scan_tile)
    int32_t scan_tile;       // rows per k_rowscan tile: 256..2048, whole final-digit groups
    int32_t rows_per_item;   // light rows per SpMM work item
    int32_t short_len;       // K > 8: light rows of at most this many entries take one lane each
    int32_t vec;             // 16-byte vectors per lane per round of the product loop (1, 2, 4)
    int32_t bl_off[kBuckets + 1];  // K > 8: start of each bucket's list in rowlist, end last
    uint32_t stamp;          // hash of the plan and workspace layout: what a re-embedding checks
    int32_t wdeg;            // 1: degrees and node table come from k_wdeg (weighted + Laplacian)
    int32_t range_tiles;     // sort tiles per range; one CTA scatters one range
    int32_t ranges;          // ceil(tiles_e / range_tiles)
    // scratch (device)
    int32_t *rowptr;         // [N+1]
    int32_t *rowcnt;         // [N]           zeroed
    int32_t *col;            // [E + 4]
    float *val;              // [E + 4]       weighted only
    uint32_t *tmpk;          // [E]           2-pass: (src >> lbits) << nbits | dst
    float *tmpw;             // [E]           2-pass weighted
    uint32_t *hist1;         // [kHistCopies][2^b1] zeroed: first-pass digit totals (b1 = lbits, or fbits for 1 pass)
    uint32_t *hist2;         // [kHistCopies][2^fbits] zeroed: final-pass digit totals (2-pass graphs)
    uint32_t *cnt1;          // [ranges << b1]    per-range first-pass digit counts, then bucket offsets
    uint32_t *cnt2;          // [ranges << fbits] per-range final-pass digit counts, then offsets (2-pass)
    int32_t *nk;             // [K]           zeroed
    float *deg;              // [N]  D_ii
    float *dinv;             // [N]  D_ii^-1/2 (1 without the Laplacian)
    int2 *tab;               // [N]  {class or 0, s_j as float bits (0 if unlabelled)}
    int32_t *rowlist;        // K > 8: [bl_off[kBuckets]] light rows by length bucket
    uint32_t *bcount;        // K > 8: [kBuckets] zeroed: rows listed per bucket
    uint32_t *status;        // [1]           zeroed
};

__host__ __device__ inline int first_bits(const GraphDesc &g) { return g.npass == 2 ? g.lbits : g.fbits; }

// Per-call state shared by all graphs of a launch sequence (zeroed at the start).
struct CallState {
    uint32_t ctr[8];         // work-stealing / tile-id counters, one per kernel
    uint32_t hub_count;      // rows longer than their graph's hub_C
    uint32_t hub_chunks;     // total chunks over those rows
    uint32_t light_items;    // k_spmm work items over the length buckets of all K > 8 graphs
    uint32_t stamp;          // single graph: the plan stamp of the last completed CSR build
    uint32_t pad[4];
};

struct HubEntry {
    int32_t g, row, len, nch;
};

struct CallBufs {
    CallState *cs;           // zeroed
    HubEntry *hubs;          // [hub_cap]
    uint32_t *chunk_off;     // [hub_cap + 1]
    uint32_t *chunk_hub;     // [chunk_cap]   hub of each chunk
    uint32_t *arrive_deg;    // [hub_cap] zeroed
    uint32_t *arrive_z;      // [hub_cap] zeroed
    double *part_deg;        // [chunk_cap]
    float2 *part_z;          // [chunk_cap * kmax]
    uint32_t *bitem;         // [kBuckets * G + 1]: prefix of the bucket work items, longest bucket
                             // first, graph by graph within a bucket
    uint32_t hub_cap, chunk_cap;
    int32_t kmax;            // largest K in the call
    int32_t ringw;           // k_spmm: 1 if any graph of the call is weighted (a val ring too)
};

// Launch context: which graphs, and how this kernel's items map onto them.
struct Ctx {
    GraphDesc g0;            // the graph when G == 1
    const GraphDesc *graphs; // device array [G] when G > 1
    const int32_t *prefix;   // device [G+1] item prefix for this kernel (G > 1)
    int32_t G;
    int32_t items;           // total items of this kernel (host-known part)
    CallBufs cb;
};

// item prefixes stored per kernel for batched calls
enum PrefixKind {
    kPfxPrep = 0,     // ranges + node tiles
    kPfxOffs1 = 1,    // 32-digit blocks of the first pass
    kPfxScat1 = 2,    // ranges of 2-pass graphs (first pass)
    kPfxCount = 3,    // ranges of 2-pass graphs (final-pass counts)
    kPfxOffs2 = 4,    // 32-digit blocks of the final pass (2-pass graphs)
    kPfxScatF = 5,    // ranges (final pass)
    kPfxScan = 6,     // node tiles of the row scan
    kPfxRows = 7,     // light-row items of the SpMM
    kPfxWRows = 8,    // light-row items of the weighted-degree kernel
    kNumPfx = 9
};

}  // namespace gee
