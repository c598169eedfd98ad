// gee_embed_static: gee_embed for callers that cannot allocate device memory.
//
// Some callers have no way to obtain scratch memory on the device: code that only
// receives device pointers from a host framework and has no handle to that framework's
// allocator, and latency-critical loops that must never call cudaMalloc because it can
// synchronise the whole device.  For them this file keeps a fixed scratch area in the
// library itself -- a file-scope __device__ array that every GPU loading the library
// holds until the process exits -- and runs the ordinary gee_embed path on it.
//
// Host code cannot pass the array's name to a kernel (on the host the name is only a
// stand-in, not a device address), so every call looks up the device address with
// cudaGetSymbolAddress for the current device.  The lookup allocates nothing and is not
// cached: a cached address could go stale after the context of a device is torn down and
// created again, and the kernels would then write through it.
#include "../../include/gee.h"

#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>

namespace {

static __device__ __align__(256) unsigned char g_static_scratch[GEE_STATIC_WORKSPACE_BYTES];

// Device address of g_static_scratch on the current device.
int static_scratch(void **out) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess || !p) return GEE_ERR_CUDA;
    *out = p;
    return GEE_OK;
}

}  // namespace

extern "C" int gee_embed_static(const int32_t *d_src, const int32_t *d_dst, const float *d_w, int64_t E,
                                int32_t N, const int32_t *d_labels, int32_t K, const gee_opts *opts, float *d_Z,
                                void *stream, uint32_t *d_status) {
    if (E < 0 || N < 0 || K < 1) return GEE_ERR_ARG;
    const size_t need = gee_workspace_size(E, N, K, d_w != nullptr, opts);
    if (need == 0 && N > 0) return GEE_ERR_TOO_LARGE;  // beyond the general limits
    if (need > (size_t)GEE_STATIC_WORKSPACE_BYTES) return GEE_ERR_TOO_LARGE;
    void *scratch = nullptr;
    if (N > 0) {
        const int rc = static_scratch(&scratch);
        if (rc != GEE_OK) return rc;
    }
    // The launch cache of gee_embed would capture and instantiate a CUDA graph on a repeated
    // call, which can allocate: it is always bypassed here.
    gee_opts o;
    std::memset(&o, 0, sizeof(o));
    if (opts) o = *opts;
    o.flags |= GEE_NO_GRAPH_CACHE;
    // gee_embed clears the part of the scratch that must start at zero, on `stream`,
    // before its first kernel; whatever an earlier call left there does not matter.
    return gee_embed(d_src, d_dst, d_w, E, N, d_labels, K, &o, d_Z, scratch, GEE_STATIC_WORKSPACE_BYTES, stream,
                     d_status);
}
