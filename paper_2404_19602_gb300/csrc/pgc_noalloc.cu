// pgc_noalloc.cu -- pgc_observe_static: the observation kernel (histogram of the current state
// at the quadrature nodes and the moment record) with its block-partial scratch in a file-scope
// device array instead of context or caller memory, so that the call allocates nothing.
//
// Who needs it: code that may not call cudaMalloc while it runs -- a host application whose
// device memory is owned by another allocator (a framework's caching pool that must see every
// allocation), a monitoring loop that samples the ensemble while other work is queued (cudaMalloc
// and cudaFree can synchronize the device and would stall it), or a process that has reserved
// all device memory up front.
//
// The scratch array is g_part, a fixed kNoAllocBytes (4 MiB) block of block-partial sums that
// every GPU which loads the library keeps until the process exits.  All calls share it and it
// keeps the last call's contents; every slot a call reads is written by the same call first.
// Two calls whose kernels overlap on the GPU (different streams, no ordering) race on it.
#include <mutex>
#include <string>

#include <cuda_runtime.h>

#include "pgc.h"
#include "pgc_ctx.h"
#include "pgc_kernels.cuh"

namespace {

constexpr size_t kNoAllocBytes = 4u << 20;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_part[kNoAllocBytes / sizeof(double)];

// Device address of g_part per device.  In host code the name g_part is only a host-side
// stand-in; a kernel must be given the address returned by cudaGetSymbolAddress, taken once per
// device with that device current.
std::mutex g_mu;
void *g_addr[kMaxDevices] = {};

cudaError_t part_address(int dev, void **out)
{
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_part);
        if (e != cudaSuccess) return e;
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" pgc_status pgc_observe_static(pgc_ctx *ctx, uint32_t *d_hist_out, double *d_record_out, void *stream)
{
    if (!ctx) return PGC_EINVAL;
    if (ctx->failed) { ctx->err = "context failed earlier: " + ctx->err; return PGC_ESTATE; }
    if (!d_hist_out || !d_record_out) { ctx->err = "pgc_observe_static: output pointers must be non-NULL"; return PGC_EINVAL; }
    const int Q = ctx->t.Q, g1 = ctx->run->grid1();
    const size_t need = (size_t)g1 * Q * 3 * sizeof(double);
    if (need > kNoAllocBytes) {
        ctx->err = "pgc_observe_static: " + std::to_string(g1) + " blocks x " + std::to_string(Q) +
                   " nodes need " + std::to_string(need) + " bytes of partial sums, more than the fixed " +
                   std::to_string(kNoAllocBytes) + "-byte device array";
        return PGC_EINVAL;
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess && (dev < 0 || dev >= kMaxDevices)) {
        ctx->err = "pgc_observe_static: device index out of range";
        return PGC_EINVAL;
    }
    void *part = nullptr;
    if (e == cudaSuccess) e = part_address(dev, &part);
    cudaStream_t s = (cudaStream_t)stream;
    const size_t hist_bytes = (size_t)Q * ctx->t.Nk * ctx->t.Nk * sizeof(uint32_t);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_hist_out, 0, hist_bytes, s);
    if (e == cudaSuccess) e = ctx->run->observe_into(d_hist_out, (double *)part, s);
    if (e == cudaSuccess) e = pgc::launch_finalize(ctx, (const double *)part, g1, ctx->step * ctx->t.dt, d_record_out, s);
    if (e != cudaSuccess) {
        // as every other entry point: a CUDA error leaves the context failed (PGC_ESTATE after)
        ctx->err = std::string("pgc_observe_static: ") + cudaGetErrorString(e);
        ctx->failed = true;
        return PGC_ECUDA;
    }
    return PGC_OK;
}
