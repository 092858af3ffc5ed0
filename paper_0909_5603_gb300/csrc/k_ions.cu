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
#include "pic_internal.h"

namespace pic {

// Ion charge per unit transverse area between box coordinates lo < hi inside [0, Lz] at
// t = 0.  The lab profile is 0 below zs, rises linearly over `ramp`, then stays at n0;
// in box coordinates it is contracted by gamma_b.  Each linear piece is integrated
// exactly as its length times the profile at its midpoint.
__device__ double ion_charge_in_box(const InstDev &I, double lo, double hi)
{
    const double g = I.ion_gb;
    const double peak = -I.q * g * I.ion_n0;       // charge density of the plateau
    const double up = I.ion_zs / g;                 // ramp start
    const double top = (I.ion_zs + I.ion_ramp) / g; // ramp end
    double charge = 0.0;
    const double r0 = fmax(lo, up), r1 = fmin(hi, top);
    if (r1 > r0) charge += peak * (r1 - r0) * ((0.5 * g * (r0 + r1) - I.ion_zs) / I.ion_ramp);
    const double p0 = fmax(lo, top);
    if (hi > p0) charge += peak * (hi - p0);
    return charge;
}

// Ion charge between coordinates a < b of this grid at t = 0 (b - a below the box
// length), taken in the box the profile fills (this grid's, or the whole grid of which
// this one is a z slab): clipped to the box when its z is absorbing (only the loaded
// volume carries ions), wrapped into it when periodic.
__device__ double ion_charge(const InstDev &I, double a, double b)
{
    const double Lz = I.ion_lz;
    a += I.ion_z0;
    b += I.ion_z0;
    if (!I.ion_periodic) {
        a = fmax(a, 0.0);
        b = fmin(b, Lz);
        return b > a ? ion_charge_in_box(I, a, b) : 0.0;
    }
    const double m = floor(a / Lz);
    a -= m * Lz;
    b -= m * Lz;
    if (b <= Lz) return ion_charge_in_box(I, a, b);
    return ion_charge_in_box(I, a, Lz) + ion_charge_in_box(I, 0.0, fmin(b - Lz, Lz));
}

// This step's ion current on the Jz faces z = (k + 1/2) dz of each instance: the face
// at box coordinate z meets, at time t, the ions that started at z + beta t, so during
// [t^n, t^{n+1}] the charge of [z + beta t^n, z + beta t^{n+1}] crosses it downwards.
template <typename R>
__global__ void __launch_bounds__(256) k_ion_faces(Launch L)
{
    const InstDev &I = L.inst[blockIdx.x];
    if (!I.ion) return;
    const int n = *I.phase;
    const double t0 = (double)n * I.dt, t1 = (double)(n + 1) * I.dt;
    for (int k = threadIdx.x; k < I.n[2]; k += blockDim.x) {
        const double z = (k + 0.5) * I.dx[2];
        const double crossing = ion_charge(I, z + I.ion_beta * t0, z + I.ion_beta * t1);
        ((R *)I.ion_face)[k] = (k >= I.ion_k0 && k < I.ion_k1) ? R(-crossing / I.dt) : R(0);
    }
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
    const int r = (int)(g - L.cell_start[ii]);
    const int rq = fast_div(r, I.div_n0);
    const int i = r - rq * I.n[0];
    const int k = fast_div(rq, I.div_n1);
    const int j = rq - k * I.n[1];
    const long long p = (i + I.gh[0]) + I.sy * (j + I.gh[1]) + I.sz * (k + I.gh[2]);
    ((R *)I.J[2])[p] = ((const R *)I.ion_face)[k];
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
