// k_push.cuh -- host launchers of the fused particle kernel for one precision and
// injection setting; k_push_f32.cu, k_push_f64.cu and their _inj twins instantiate them
// (separate translation units compile in parallel).
#pragma once
#include "k_particles.cuh"

namespace pic {

// one: the instance of a one-instance launch (host copy, identical to the launch's device
// entry), passed by value; null for a batch
template <int ND, int ORD, typename R, int PUSHER, bool INJ>
static cudaError_t launch_particles_t(const Launch *L, const InstDev *one, size_t smem, cudaStream_t s)
{
    auto k = k_particles<ND, ORD, R, PUSHER, INJ>;
    auto k1 = k_particles_one<ND, ORD, R, PUSHER, INJ>;
    if (!L) {  // preparation: raise the dynamic shared-memory limit once, outside any capture
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        return e == cudaSuccess ? cudaFuncSetAttribute(k1, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) : e;
    }
    if (one && L->ninst == 1)
        k1<<<L->total_tiles, kNT, smem, s>>>(*one);
    else
        k<<<L->total_tiles, kNT, smem, s>>>(*L);
    return cudaGetLastError();
}

template <typename R, bool INJ>
static cudaError_t dispatch_particles_t(int ndim, int order, int pusher, const Launch *L, const InstDev *one, size_t smem,
                                        cudaStream_t s)
{
#define PIC_DISPATCH(ND, ORD, P) \
    if (ndim == ND && order == ORD && pusher == P) return launch_particles_t<ND, ORD, R, P, INJ>(L, one, smem, s);
    PIC_DISPATCH(2, 1, 0) PIC_DISPATCH(2, 1, 1) PIC_DISPATCH(2, 2, 0) PIC_DISPATCH(2, 2, 1)
    PIC_DISPATCH(3, 1, 0) PIC_DISPATCH(3, 1, 1) PIC_DISPATCH(3, 2, 0) PIC_DISPATCH(3, 2, 1)
#undef PIC_DISPATCH
    return cudaErrorInvalidValue;
}

}  // namespace pic
