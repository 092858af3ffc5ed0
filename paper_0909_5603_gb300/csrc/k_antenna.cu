// k_antenna.cu -- laser antenna on a plane fixed in the laboratory frame (Sec. 2 of Vay
// et al.: the laser enters through a plane fixed in the lab that drifts in the boosted
// frame).
//
// The lab pulse is emitted forward by the lab plane z = z_lab, which sits at
// z' = z_lab / gamma_b - beta_b t' in this frame.  The grid is split at the plane: values
// at z positions above it hold the total field, values at or below it the field minus
// the incident pulse (E_x = B_y = T(x, y) g, T = exp(-(x^2 + y^2) / w0^2)).  g is carried
// on a 1D lattice aligned with the grid's z lattice and advanced by the same leapfrog, so
// a plane wave crosses the boundary without reflection.  The plane's position is held for
// the Maxwell phase that starts at its time:
//  * every z difference joining the two regions takes its far value in the near value's
//    representation, which adds h T g_E / dz to B_y (each B half update) and
//    dt T g_B / dz to E_x (the E update), times the absorbing-layer factor where the
//    update is damped;
//  * after the phase, values the receding plane passed join the total field: the
//    incident value there is added.
// Under the low-dispersion solver every Faraday difference is averaged over its
// transverse neighbours (7/12 on itself, 1/12 on the edge and 1/48 on the corner ones),
// so the same rule -- each stencil reads its neighbours in its own node's representation
// -- spreads the B_y term over the neighbouring columns (the profile T replaced by its
// weighted average) and adds a B_z term: the averaged dE_x/dy at a B_z node next to the
// plane reads E_x on the z row across it.  The E update keeps the Yee differences.
// One thread per transverse cell; the plane touches one or two z planes.  FP64
// arithmetic, the result added in the working precision.
#include "pic_internal.h"

namespace pic {

namespace {

__device__ __forceinline__ double ant_plane(const AntDev &A, const InstDev &I, int n)
{
    return (A.zb - A.beta * (A.t0 + (double)n * I.dt)) / I.dx[2];
}

__device__ __forceinline__ double ant_ge(const AntDev &A, long long k)
{
    const long long a = k - A.lo;
    return a >= 0 && a < A.na ? A.ge[a] : 0.0;
}

__device__ __forceinline__ double ant_gb(const AntDev &A, long long k)
{
    const long long a = k - A.lo;
    return a >= 0 && a < A.na ? A.gb[a] : 0.0;
}

// profile at the transverse position shared by E_x and B_y: (i + 1/2, j)
__device__ __forceinline__ double ant_profile(const AntDev &A, const InstDev &I, int i, int j)
{
    const double x = (i + 0.5) * I.dx[0] - A.xc;
    const double y = I.ndim == 3 ? j * I.dx[1] - A.yc : 0.0;
    return exp(-(x * x + y * y) / (A.w0 * A.w0));
}

// the profile at E_x's (i + 1/2, j) as a neighbour in a difference stencil: outside the
// box an absorbing axis reads 0 (the ghost value), a periodic one wraps
__device__ __forceinline__ double ant_profile_nb(const AntDev &A, const InstDev &I, int i, int j)
{
    if (i < 0 || i >= I.n[0]) {
        if (I.bc[0] != 0) return 0.0;
        i = (i + I.n[0]) % I.n[0];
    }
    if (I.ndim == 3 && (j < 0 || j >= I.n[1])) {
        if (I.bc[1] != 0) return 0.0;
        j = (j + I.n[1]) % I.n[1];
    }
    return ant_profile(A, I, i, j);
}

// weight of a transverse neighbour of a low-dispersion difference (offsets db, dc)
__device__ __forceinline__ double ck_weight(int db, int dc)
{
    const int e = (db != 0) + (dc != 0);
    return e == 0 ? 7.0 / 12.0 : (e == 1 ? 1.0 / 12.0 : 1.0 / 48.0);
}

template <typename R>
__device__ __forceinline__ double damp_at(const InstDev &I, int i, int j, int k)
{
    const int idx[3] = {i, j, k};
    R f = R(1);
#pragma unroll
    for (int a = 0; a < 3; ++a)
        if (I.damp[a]) f *= ((const R *)I.damp[a])[idx[a]];
    return (double)f;
}

__device__ __forceinline__ long long padded(const InstDev &I, int i, int j, int k)
{
    return (i + I.gh[0]) + I.sy * (long long)(j + I.gh[1]) + I.sz * (long long)(k + I.gh[2]);
}

}  // namespace

// what 0: the incident field at E_x nodes and B_y half nodes above the plane (the set);
// what 1: at those in (plane now, plane one phase earlier] (after a phase)
template <typename R>
__global__ void __launch_bounds__(256) k_ant_add(const InstDev *Ip, AntDev A, int what)
{
    const InstDev &I = *Ip;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= I.n[0] * I.n[1]) return;
    const int i = t % I.n[0], j = t / I.n[0];
    const int n = *A.n;
    const double lo = ant_plane(A, I, n);
    const double hi = what == 0 ? INFINITY : ant_plane(A, I, n - 1);
    if (!(hi > lo)) return;
    const int k0 = lo < 0.0 ? 0 : (int)fmin(floor(lo), (double)I.n[2]);
    const int k1 = hi >= I.n[2] - 1 ? I.n[2] - 1 : (int)floor(hi);
    const double T = ant_profile(A, I, i, j);
    R *Ex = (R *)eb_field(I, 0), *By = (R *)eb_field(I, 4);
    for (int k = k0; k <= k1; ++k) {
        const long long p = padded(I, i, j, k);
        if (k > lo && k <= hi) Ex[p] += (R)(T * ant_ge(A, k));
        if (k + 0.5 > lo && k + 0.5 <= hi) By[p] += (R)(T * ant_gb(A, k));
    }
}

// B_y at the half node next to the plane, after a B half update (damp: the second one);
// CK: the low-dispersion solver's terms (B_y spread over the neighbouring columns, and
// in 3D B_z at the nodes on either side of the plane)
template <typename R, bool CK>
__global__ void __launch_bounds__(256) k_ant_bterm(const InstDev *Ip, AntDev A, int damp)
{
    const InstDev &I = *Ip;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= I.n[0] * I.n[1]) return;
    const int i = t % I.n[0], j = t / I.n[0];
    const double zp = ant_plane(A, I, *A.n);
    if (!(zp >= 0.0 && zp < I.n[2])) return;
    const int k = (int)floor(zp);
    const double h = 0.5 * I.dt;
    if (CK && I.ndim == 3) {
        // B_z at (i + 1/2, j + 1/2, kz): its averaged dE_x/dy reads E_x at kz - 1, kz,
        // kz + 1; the node below the plane (kz = k) reads the incident E_x of row k + 1
        // above it and subtracts it, the node above (kz = k + 1) adds that of row k
        R *Bz = (R *)eb_field(I, 5);
        for (int side = 0; side < 2; ++side) {
            const int kz = k + side;
            if (kz >= I.n[2]) continue;
            const int dk = side == 0 ? 1 : -1;
            const double g = ant_ge(A, kz + dk);
            double S = 0.0;
            for (int di = -1; di <= 1; ++di)
                S += ck_weight(dk, di) * (ant_profile_nb(A, I, i + di, j + 1) - ant_profile_nb(A, I, i + di, j));
            const double f = damp ? damp_at<R>(I, i, j, kz) : 1.0;
            const double term = (side == 0 ? -h : h) * S * g / I.dx[1];
            Bz[padded(I, i, j, kz)] += (R)(f * term);
        }
    }
    double g;
    if (zp < k + 0.5) {  // B_y at k + 1/2 total field, E_x at k scattered
        g = ant_ge(A, k);
    } else {             // B_y scattered, E_x at k + 1 total field
        if (k + 1 >= I.n[2]) return;
        g = ant_ge(A, k + 1);
    }
    double T;
    if (CK) {
        T = 0.0;
        for (int di = -1; di <= 1; ++di)
            for (int dj = -1; dj <= 1; ++dj) T += ck_weight(di, dj) * ant_profile_nb(A, I, i + di, j + dj);
    } else {
        T = ant_profile(A, I, i, j);
    }
    const double f = damp ? damp_at<R>(I, i, j, k) : 1.0;
    R *By = (R *)eb_field(I, 4);
    By[padded(I, i, j, k)] += (R)(f * h * (T * g / I.dx[2]));
}

// E_x at the node next to the plane, after the (damped) E update
template <typename R>
__global__ void __launch_bounds__(256) k_ant_eterm(const InstDev *Ip, AntDev A)
{
    const InstDev &I = *Ip;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= I.n[0] * I.n[1]) return;
    const int i = t % I.n[0], j = t / I.n[0];
    const double zp = ant_plane(A, I, *A.n);
    if (!(zp + 0.5 >= 0.0 && zp + 0.5 < I.n[2])) return;
    const int m = (int)floor(zp + 0.5);
    double g;
    if (zp < m) {  // E_x at m total field, B_y at m - 1/2 scattered
        if (m - 1 < 0) return;
        g = ant_gb(A, m - 1);
    } else {       // E_x scattered, B_y at m + 1/2 total field
        g = ant_gb(A, m);
    }
    const double f = damp_at<R>(I, i, j, m);
    R *Ex = (R *)eb_field(I, 0);
    Ex[padded(I, i, j, m)] += (R)(f * I.dt * (ant_profile(A, I, i, j) * g / I.dx[2]));
}

// The 1D lattice: what 0 / 2: B_y -= (dt / 2) dE_x/dz (2 also counts the phase);
// what 1: E_x -= dt dB_y/dz.  Zero beyond the lattice.
__global__ void __launch_bounds__(256) k_ant_lattice(AntDev A, double dt, double dz, int what)
{
    const long long a = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (what == 2 && a == 0) *A.n += 1;  // no other thread of this launch reads it
    if (a >= A.na) return;
    if (what == 1) {
        const double b0 = a > 0 ? A.gb[a - 1] : 0.0;
        A.ge[a] -= dt * (A.gb[a] - b0) / dz;
    } else {
        const double e1 = a + 1 < A.na ? A.ge[a + 1] : 0.0;
        A.gb[a] -= 0.5 * dt * (e1 - A.ge[a]) / dz;
    }
}

static inline unsigned blocks_of(long long n) { return (unsigned)((n + 255) / 256); }

cudaError_t launch_ant_add(int fp64, const InstDev *d_inst, const InstDev &I, const AntDev &A, int what, cudaStream_t s)
{
    const unsigned nb = blocks_of((long long)I.n[0] * I.n[1]);
    if (fp64)
        k_ant_add<double><<<nb, 256, 0, s>>>(d_inst, A, what);
    else
        k_ant_add<float><<<nb, 256, 0, s>>>(d_inst, A, what);
    return cudaGetLastError();
}

cudaError_t launch_ant_bterm(int fp64, int ck, const InstDev *d_inst, const InstDev &I, const AntDev &A, int damp,
                             cudaStream_t s)
{
    const unsigned nb = blocks_of((long long)I.n[0] * I.n[1]);
    if (fp64) {
        if (ck) k_ant_bterm<double, true><<<nb, 256, 0, s>>>(d_inst, A, damp);
        else k_ant_bterm<double, false><<<nb, 256, 0, s>>>(d_inst, A, damp);
    } else {
        if (ck) k_ant_bterm<float, true><<<nb, 256, 0, s>>>(d_inst, A, damp);
        else k_ant_bterm<float, false><<<nb, 256, 0, s>>>(d_inst, A, damp);
    }
    return cudaGetLastError();
}

cudaError_t launch_ant_eterm(int fp64, const InstDev *d_inst, const InstDev &I, const AntDev &A, cudaStream_t s)
{
    const unsigned nb = blocks_of((long long)I.n[0] * I.n[1]);
    if (fp64)
        k_ant_eterm<double><<<nb, 256, 0, s>>>(d_inst, A);
    else
        k_ant_eterm<float><<<nb, 256, 0, s>>>(d_inst, A);
    return cudaGetLastError();
}

cudaError_t launch_ant_lattice(const AntDev &A, double dt, double dz, int what, cudaStream_t s)
{
    k_ant_lattice<<<blocks_of(A.na), 256, 0, s>>>(A, dt, dz, what);
    return cudaGetLastError();
}

}  // namespace pic
