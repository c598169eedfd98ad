// Sparse Z (CSR over classes) for many classes: the arguments of the kernels in
// gee_sparse.cu and their host-side entry points.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace gee {

struct SparseArgs {
    // the graph, as the CSR build left it
    const int32_t *rowptr;   // [N+1]
    const int32_t *col;      // [E]
    const float *val;        // [E] or nullptr (unweighted)
    const int32_t *y;        // [N] labels (-1: unlabelled)
    const int2 *tab;         // [N] node table {class, bits of s_j}
    const float *dinv;       // [N] D_ii^-1/2 (read with the Laplacian)
    int32_t N, K;
    int64_t E;               // CSR capacity (rowptr[N] <= E)
    uint32_t flags;          // GEE_DIAG_AUG | GEE_LAPLACIAN | GEE_CORRELATION
    // scratch
    int32_t *cnt;            // [N] runs (distinct classes) per row
    int4 *runs_a, *runs_b;   // [E + N] {class, sum, compensation, 0}: row i at rowptr[i] + i
    int32_t *long_list;      // [long_cap] rows with more entries than one window holds
    uint32_t *long_count;    // [2] zeroed: rows listed, rows claimed by the merge
    uint32_t long_cap;
    uint32_t *chunk_off;     // [long_cap + 1] first chunk of each listed row, total last
    int32_t *chunk_cnt;      // [chunk_cap] runs of each chunk
    uint32_t chunk_cap;
    uint32_t *tile_sum;      // [scan tiles + 1]
    int32_t *wstart;         // [windows + 1] first row of each window of CSR positions
    // output
    int32_t *zrowptr;        // [N+1]
    int32_t *zcol;           // [zcap]
    float *zval;             // [zcap]
    int64_t zcap;
    uint32_t *status;
};

cudaError_t configure_sparse_kernels();
cudaError_t launch_sparse(const SparseArgs &a, int sms, cudaStream_t st);
int sparse_scan_tiles(int32_t N);
int64_t sparse_long_cap(int64_t E);
int64_t sparse_chunk_cap(int64_t E);
int64_t sparse_windows(int64_t E);

}  // namespace gee
