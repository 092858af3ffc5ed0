// pic_noalloc.cu -- charge-density read-out that allocates no device memory.
//
// The regular read-out, pic_get_field(ctx, PIC_RHO, ...), deposits the particles' charge
// into a per-context FP64 work grid that pic_create allocated.  This variant deposits
// into a fixed array that the library itself owns instead (below), so it runs for
// callers that may not, or cannot, allocate device memory at the moment they read the
// density.  The deposit kernel is the same one (launch_rho); only its destination
// differs.
#include <cstdio>

#include "../../include/pic.h"
#include "pic_internal.h"

namespace pic {
pic_status ctx_fail(pic_ctx *c, pic_status s, const char *msg);
}

using namespace pic;

namespace {

// The work grid: PIC_NOALLOC_RHO_MAX_CELLS doubles (8 MiB) in every GPU on which a context
// was created, held until the process exits.  In host code this name is only a host-side
// stand-in; its device address comes from cudaGetSymbolAddress with the device current.
static __device__ __align__(256) double g_rho_scratch[PIC_NOALLOC_RHO_MAX_CELLS];

// Device address of the work grid on the current device, looked up on every call (cheap
// once the module is loaded, and never stale if another component resets the device's
// primary context).  Returns nullptr (and fills msg) when the lookup fails.
double *scratch_on_device(char *msg, size_t msglen)
{
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_rho_scratch);
    if (e != cudaSuccess || !p) {
        snprintf(msg, msglen, "cudaGetSymbolAddress of the no-allocation work grid failed: %s", cudaGetErrorString(e));
        return nullptr;
    }
    return static_cast<double *>(p);
}

}  // namespace

namespace pic {

// CUDA loads a module lazily, on the first use of one of its symbols, and loading this
// one allocates the work grid: pic_create (with its device current) does that first use,
// and loads the density kernels the read-out launches.
cudaError_t noalloc_load_grid(int order, int fp64)
{
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_rho_scratch);
    return e == cudaSuccess ? preload_rho(order, fp64) : e;
}

}  // namespace pic

extern "C" pic_status pic_get_rho_noalloc(pic_ctx *ctx, double *host_out, size_t count)
{
    CtxView v;
    if (!ctx_view(ctx, &v)) return PIC_ERR_ARG;
    char msg[256];
    if (v.is_batch) return ctx_fail(ctx, PIC_ERR_ARG, "pic_get_rho_noalloc takes a member, not a batch");
    if (v.ncell > PIC_NOALLOC_RHO_MAX_CELLS) {
        snprintf(msg, sizeof(msg), "grid of %lld cells exceeds the no-allocation work grid of %d cells", v.ncell,
                 (int)PIC_NOALLOC_RHO_MAX_CELLS);
        return ctx_fail(ctx, PIC_ERR_ARG, msg);
    }
    if (!host_out || count < (size_t)v.ncell) {
        snprintf(msg, sizeof(msg), "host_out needs room for %lld values", v.ncell);
        return ctx_fail(ctx, PIC_ERR_ARG, msg);
    }
    if (cudaSetDevice(v.device) != cudaSuccess) return ctx_fail(ctx, PIC_ERR_CUDA, "cudaSetDevice failed");
    pic_status st = pic_synchronize(ctx);  // also reports a sticky device error
    if (st != PIC_OK) return st;
    double *grid = scratch_on_device(msg, sizeof(msg));
    if (!grid) return ctx_fail(ctx, PIC_ERR_CUDA, msg);
    // the array keeps the previous call's contents: clear the part this grid uses
    const size_t bytes = sizeof(double) * (size_t)v.ncell;
    cudaError_t e = cudaMemsetAsync(grid, 0, bytes, v.stream);
    if (e == cudaSuccess && v.loaded) e = launch_rho(v.order, v.fp64, *v.launch, grid, v.stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(host_out, grid, bytes, cudaMemcpyDeviceToHost, v.stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(v.stream);
    if (e != cudaSuccess) {
        snprintf(msg, sizeof(msg), "no-allocation charge read-out failed: %s", cudaGetErrorString(e));
        return ctx_fail(ctx, PIC_ERR_CUDA, msg);
    }
    return pic_synchronize(ctx);
}
