// k_push_f64.cu -- double instantiations of the fused particle kernel (split from the
// FP32 ones so the two compile in parallel).
#include "k_particles.cuh"

namespace pic {

template <int ND, int ORD, typename R, int PUSHER>
static cudaError_t launch_particles_t(const Launch *L, size_t smem, cudaStream_t s)
{
    auto k = k_particles<ND, ORD, R, PUSHER>;
    if (!L)  // preparation: raise the dynamic shared-memory limit once, outside any capture
        return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k<<<L->total_tiles, kNT, smem, s>>>(*L);
    return cudaGetLastError();
}


cudaError_t dispatch_particles_f64(int ndim, int order, int pusher, const Launch *L, size_t smem, cudaStream_t s)
{
#define PIC_DISPATCH(ND, ORD, P) \
    if (ndim == ND && order == ORD && pusher == P) return launch_particles_t<ND, ORD, double, P>(L, smem, s);
    PIC_DISPATCH(2, 1, 0) PIC_DISPATCH(2, 1, 1) PIC_DISPATCH(2, 2, 0) PIC_DISPATCH(2, 2, 1)
    PIC_DISPATCH(3, 1, 0) PIC_DISPATCH(3, 1, 1) PIC_DISPATCH(3, 2, 0) PIC_DISPATCH(3, 2, 1)
#undef PIC_DISPATCH
    return cudaErrorInvalidValue;
}

}  // namespace pic
