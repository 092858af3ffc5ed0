// k_ions.cu -- the ion background of a lab-frame plasma load (Sec. 2 of Vay et al.: the
// plasma is at rest in the lab frame, so in the boosted frame its ions are the lab
// profile contracted by gamma_b, streaming rigidly at -beta_b).
//
// Only the electrons are macro-particles.  The ions enter each step as a current on the
// Jz faces -- the charge of the moving profile that crosses a face during the step,
// divided by dt -- and the rho read-out as the charge of each node's dual cell.  Both are
// integrals of one profile, so the ions satisfy the discrete continuity equation to
// rounding.  The per-face values (one per z plane) are formed in FP64 by a small kernel
// and broadcast over the planes in the working precision by a second, one thread per
// cell; FP64 work is thus n_z per instance and step, not one per cell.
#include "k_ions.cuh"

namespace pic {

// This step's ion current on the Jz faces of each instance (one CTA per instance).
template <typename R>
__global__ void __launch_bounds__(256) k_ion_faces(Launch L)
{
    ion_faces_of<R>(L.inst[blockIdx.x], threadIdx.x, blockDim.x);
}

// Jz <- the ion current of its plane, every interior cell (J was zeroed for the step).
template <typename R>
__global__ void __launch_bounds__(256) k_ion_current(Launch L)
{
    const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= L.total_cells) return;
    const int ii = find_instance_ll(L.cell_start, L.ninst, g);
    const InstDev &I = L.inst[ii];
    if (!I.ion) return;
    ion_current_cell<R>(I, (int)(g - L.cell_start[ii]));
}

// rho (dense FP64 grid of instance 0) += the ion charge of each node's dual cell
// [z_k - dz/2, z_k + dz/2] at the current time, divided by dz.
__global__ void __launch_bounds__(256) k_rho_ion(Launch L, double *rho)
{
    const InstDev &I = L.inst[0];
    if (!I.ion) return;
    const long long ncell = (long long)I.n[0] * I.n[1] * I.n[2];
    const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= ncell) return;
    const int k = (int)(g / ((long long)I.n[0] * I.n[1]));
    const double t = (double)(*I.phase) * I.dt, dz = I.dx[2];
    const double z = k * dz + I.ion_beta * t;
    rho[g] += ion_charge(I, z - 0.5 * dz, z + 0.5 * dz) / dz;
}

cudaError_t launch_ion_current(int fp64, const Launch &L, cudaStream_t s)
{
    const unsigned blocks = (unsigned)((L.total_cells + 255) / 256);
    if (fp64) {
        k_ion_faces<double><<<L.ninst, 256, 0, s>>>(L);
        k_ion_current<double><<<blocks, 256, 0, s>>>(L);
    } else {
        k_ion_faces<float><<<L.ninst, 256, 0, s>>>(L);
        k_ion_current<float><<<blocks, 256, 0, s>>>(L);
    }
    return cudaGetLastError();
}

cudaError_t preload_rho_ion()
{
    cudaFuncAttributes a;
    return cudaFuncGetAttributes(&a, k_rho_ion);
}

cudaError_t launch_rho_ion(const Launch &L, long long ncell, double *rho, cudaStream_t s)
{
    if (ncell <= 0) return cudaSuccess;
    k_rho_ion<<<(unsigned)((ncell + 255) / 256), 256, 0, s>>>(L, rho);
    return cudaGetLastError();
}

}  // namespace pic
