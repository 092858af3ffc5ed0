// k_stations.cu -- lab-frame stations (Sec. 2 of Vay et al.: results recorded at planes
// immobile in the laboratory frame, interpolated from the boosted grid and transformed
// back to the laboratory frame).
//
// Lab and boosted frames share their origin and the boost is along +z, so at boosted
// time t' the lab plane z = z_lab sits at z' = z_lab / g - b t', where the lab time is
// t = t' / g + b z_lab.  While z' lies in the box, each record samples every field
// component at its own transverse Yee position, linearly in z' between the two planes of
// that component's z stagger, and boosts the sample by -b:
//   E_x = g (E'_x + b B'_y),  E_y = g (E'_y - b B'_x),  E_z = E'_z,
//   B_x = g (B'_x - b E'_y),  B_y = g (B'_y + b E'_x),  B_z = B'_z.
// The arithmetic is FP64 (one thread per transverse cell and station); records are
// stored in the working precision.
#include "pic_internal.h"

namespace pic {

namespace {

__device__ __forceinline__ bool station_plane(const InstDev &I, double z_lab, double &zp, double &tp)
{
    tp = (double)(*I.phase) * I.dt;
    zp = z_lab / I.gb - I.beta_b * tp;
    return zp >= 0.0 && zp < I.n[2] * I.dx[2];
}

}  // namespace

template <typename R>
__global__ void __launch_bounds__(256) k_station_record(const InstDev *Ip, StationDev S)
{
    const InstDev &I = *Ip;
    const int st = blockIdx.y;
    const int plane = I.n[0] * I.n[1];
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= plane) return;
    const int rec = S.count[st];
    if (rec >= S.max_records) return;
    double zp, tp;
    if (!station_plane(I, S.z_lab[st], zp, tp)) return;
    const int i = e % I.n[0], j = e / I.n[0];
    const EBPtr cur = cur_eb(I);
    const void *F[6] = {cur.E[0], cur.E[1], cur.E[2], cur.B[0], cur.B[1], cur.B[2]};
    const double zst[6] = {0.0, 0.0, 0.5, 0.5, 0.5, 0.0};  // z stagger: Ex Ey Ez Bx By Bz
    double f[6];
#pragma unroll
    for (int c = 0; c < 6; ++c) {
        const double q = zp / I.dx[2] - zst[c];
        const double kf = floor(q);
        const double fr = q - kf;
        double v[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            int k = (int)kf + h;
            bool ok = true;
            if (k < 0 || k >= I.n[2]) {
                if (I.bc[2] == 0) k = ((k % I.n[2]) + I.n[2]) % I.n[2];
                else ok = false;
            }
            const long long p = (i + I.gh[0]) + I.sy * (j + I.gh[1]) + I.sz * (k + I.gh[2]);
            v[h] = ok ? (double)((const R *)F[c])[p] : 0.0;
        }
        f[c] = (1.0 - fr) * v[0] + fr * v[1];
    }
    const double g = I.gb, b = I.beta_b;
    const double lab[6] = {g * (f[0] + b * f[4]), g * (f[1] - b * f[3]), f[2],
                           g * (f[3] - b * f[1]), g * (f[4] + b * f[0]), f[5]};
    R *out = (R *)S.fields + ((long long)st * S.max_records + rec) * 6 * plane;
#pragma unroll
    for (int c = 0; c < 6; ++c) out[(long long)c * plane + e] = R(lab[c]);
    if (e == 0) S.t_lab[(long long)st * S.max_records + rec] = tp / g + b * S.z_lab[st];
}

// one thread per station: count the record just taken
__global__ void k_station_advance(const InstDev *Ip, StationDev S, int nst)
{
    const int st = blockIdx.x * blockDim.x + threadIdx.x;
    if (st >= nst) return;
    double zp, tp;
    if (S.count[st] < S.max_records && station_plane(*Ip, S.z_lab[st], zp, tp)) S.count[st] += 1;
}

cudaError_t launch_stations(int fp64, const InstDev *d_inst, const StationDev &S, int nst, int plane, cudaStream_t s)
{
    if (nst <= 0) return cudaSuccess;
    const dim3 grid((unsigned)((plane + 255) / 256), (unsigned)nst);
    if (fp64) k_station_record<double><<<grid, 256, 0, s>>>(d_inst, S);
    else k_station_record<float><<<grid, 256, 0, s>>>(d_inst, S);
    k_station_advance<<<(nst + 127) / 128, 128, 0, s>>>(d_inst, S, nst);
    return cudaGetLastError();
}

}  // namespace pic
