// k_push_f32_inj.cu -- float instantiations of the fused particle kernel, with a beam injection plane.
#include "k_push.cuh"

namespace pic {

cudaError_t dispatch_particles_f32_inj(int ndim, int order, int pusher, const Launch *L, const InstDev *one, size_t smem,
                                     cudaStream_t s)
{
    return dispatch_particles_t<float, true>(ndim, order, pusher, L, one, smem, s);
}

}  // namespace pic
