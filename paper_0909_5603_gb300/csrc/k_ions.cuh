// k_ions.cuh -- device functions of the ion background of a lab-frame plasma load (Sec. 2
// of Vay et al.: the plasma is at rest in the lab frame, so in the boosted frame its ions
// are the lab profile contracted by gamma_b, streaming rigidly at -beta_b); used by
// k_ions.cu and the persistent batched step.
#pragma once
#include "pic_internal.h"

namespace pic {

// Ion charge per unit transverse area between box coordinates lo < hi inside [0, Lz] at
// t = 0.  The lab profile is 0 below zs, rises linearly over `ramp`, then stays at n0;
// in box coordinates it is contracted by gamma_b.  Each linear piece is integrated
// exactly as its length times the profile at its midpoint.
__device__ __forceinline__ double ion_charge_in_box(const InstDev &I, double lo, double hi)
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
__device__ __forceinline__ double ion_charge(const InstDev &I, double a, double b)
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

// This step's ion current on the Jz faces z = (k + 1/2) dz of instance I: the face at
// box coordinate z meets, at time t, the ions that started at z + beta t, so during
// [t^n, t^{n+1}] the charge of [z + beta t^n, z + beta t^{n+1}] crosses it downwards.
// Planes k = first, first + stride, ...
template <typename R>
__device__ __forceinline__ void ion_faces_of(const InstDev &I, int first, int stride)
{
    if (!I.ion) return;
    const int n = *I.phase;
    const double t0 = (double)n * I.dt, t1 = (double)(n + 1) * I.dt;
    for (int k = first; k < I.n[2]; k += stride) {
        const double z = (k + 0.5) * I.dx[2];
        const double crossing = ion_charge(I, z + I.ion_beta * t0, z + I.ion_beta * t1);
        ((R *)I.ion_face)[k] = (k >= I.ion_k0 && k < I.ion_k1) ? R(-crossing / I.dt) : R(0);
    }
}

// Jz of interior cell r (x fastest) of instance I <- the ion current of its plane.
template <typename R>
__device__ __forceinline__ void ion_current_cell(const InstDev &I, int r)
{
    const int rq = fast_div(r, I.div_n0);
    const int i = r - rq * I.n[0];
    const int k = fast_div(rq, I.div_n1);
    const int j = rq - k * I.n[1];
    const long long p = (i + I.gh[0]) + I.sy * (j + I.gh[1]) + I.sz * (k + I.gh[2]);
    ((R *)I.J[2])[p] = ((const R *)I.ion_face)[k];
}

}  // namespace pic
