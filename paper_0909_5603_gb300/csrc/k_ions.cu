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

// J at the start of a step of one instance: Jx = Jy = 0 and Jz = the ion current of its
// plane (interior cells; 0 without ions and on the ghosts), one warp per padded (y, z) row
// with 16-byte stores -- one pass instead of a clear and a second pass over Jz.  The
// padding after the last row of each component is never written by any kernel and stays
// zero from the load.
template <typename R>
__global__ void __launch_bounds__(256) k_j_init_one(const __grid_constant__ InstDev I)
{
    constexpr int V = 16 / sizeof(R);  // values per 16-byte group
    const long long row = (long long)blockIdx.x * 8 + (threadIdx.x >> 5);
    if (row >= (long long)I.P[1] * I.P[2]) return;
    const int lane = threadIdx.x & 31;
    const int j = (int)(row % I.P[1]) - I.gh[1], k = (int)(row / I.P[1]) - I.gh[2];
    const bool ionrow = I.ion && j >= 0 && j < I.n[1] && k >= 0 && k < I.n[2];
    const R v = ionrow ? ((const R *)I.ion_face)[k] : R(0);
    const long long base = row * I.sy;  // rows are sy = P[0] elements, a multiple of V
    for (int g = lane; g * V < I.sy; g += 32) {
        const long long e = base + (long long)g * V;
        *reinterpret_cast<uint4 *>((R *)I.J[0] + e) = make_uint4(0, 0, 0, 0);
        *reinterpret_cast<uint4 *>((R *)I.J[1] + e) = make_uint4(0, 0, 0, 0);
        union {
            uint4 q;
            R r[V];
        } z;
#pragma unroll
        for (int t = 0; t < V; ++t) {
            const int x = g * V + t - I.gh[0];
            z.r[t] = (ionrow && x >= 0 && x < I.n[0]) ? v : R(0);
        }
        *reinterpret_cast<uint4 *>((R *)I.J[2] + e) = z.q;
    }
}

cudaError_t launch_j_init_one(int fp64, const Launch &L, const InstDev &h, cudaStream_t s)
{
    if (h.ion) {
        if (fp64) k_ion_faces<double><<<1, 256, 0, s>>>(L);
        else k_ion_faces<float><<<1, 256, 0, s>>>(L);
    }
    const unsigned blocks = (unsigned)(((long long)h.P[1] * h.P[2] + 7) / 8);
    if (fp64) k_j_init_one<double><<<blocks, 256, 0, s>>>(h);
    else k_j_init_one<float><<<blocks, 256, 0, s>>>(h);
    return cudaGetLastError();
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
