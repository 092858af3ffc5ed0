// k_push.cuh -- host launchers of the fused particle kernel for one precision and
// injection setting; k_push_f32.cu, k_push_f64.cu and their _inj twins instantiate them
// (separate translation units compile in parallel).
#pragma once
#include "k_particles.cuh"

namespace pic {

template <int ND, int ORD, typename R, int PUSHER, bool INJ>
static cudaError_t launch_particles_t(const Launch *L, size_t smem, cudaStream_t s)
{
    auto k = k_particles<ND, ORD, R, PUSHER, INJ>;
    if (!L)  // preparation: raise the dynamic shared-memory limit once, outside any capture
        return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k<<<L->total_tiles, kNT, smem, s>>>(*L);
    return cudaGetLastError();
}

template <typename R, bool INJ>
static cudaError_t dispatch_particles_t(int ndim, int order, int pusher, const Launch *L, size_t smem, cudaStream_t s)
{
#define PIC_DISPATCH(ND, ORD, P) \
    if (ndim == ND && order == ORD && pusher == P) return launch_particles_t<ND, ORD, R, P, INJ>(L, smem, s);
    PIC_DISPATCH(2, 1, 0) PIC_DISPATCH(2, 1, 1) PIC_DISPATCH(2, 2, 0) PIC_DISPATCH(2, 2, 1)
    PIC_DISPATCH(3, 1, 0) PIC_DISPATCH(3, 1, 1) PIC_DISPATCH(3, 2, 0) PIC_DISPATCH(3, 2, 1)
#undef PIC_DISPATCH
    return cudaErrorInvalidValue;
}

}  // namespace pic
