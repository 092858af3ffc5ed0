// k_push_f32.cu -- float instantiations of the fused particle kernel, without an injection plane.
#include "k_push.cuh"

namespace pic {

cudaError_t dispatch_particles_f32(int ndim, int order, int pusher, const Launch *L, const InstDev *one, size_t smem,
                                     cudaStream_t s)
{
    return dispatch_particles_t<float, false>(ndim, order, pusher, L, one, smem, s);
}

}  // namespace pic
