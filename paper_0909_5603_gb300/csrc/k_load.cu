// k_load.cu -- device side of the particle loads.
//
// k_place: particles arrive in FP64 (or, for an FP32 context, in FP32) in any order
// together with their slot in the canonical (tile-sorted) order, which the host computed
// with a stable counting sort; each thread converts one particle to the storage precision
// and writes it to its slot.
//
// k_plasma_count / k_plasma_write: the lab-frame plasma of pic_load_lab_frame generated
// on the device instead of on the host.  Every cell draws `ppc` candidates from the
// counter-based SplitMix64 streams (offsets 0..2, thermal momenta (3,4) (5,6) (7,8), the
// counter being cell * ppc + p), weights them by the lab density at the lab position of
// the t' = 0 sample (z_lab = gamma_b z'), drops those of zero weight, boosts the lab
// momentum and places the rest.  The arithmetic is the host transform's, operation by
// operation in IEEE FP64 without contraction, so cells, offsets, weights and cold
// momenta are bit-identical to it; thermal momenta go through the device's log and cos
// (within 2 ulp of the host's).  The count pass lets the host lay out the canonical
// order (slot and id of each cell's first particle) before the write pass.
#include "pic_internal.h"

namespace pic {

namespace {

template <typename R>
__device__ __forceinline__ R unit_offset(double o);

template <>
__device__ __forceinline__ float unit_offset<float>(double o)
{
    // an offset within half an FP32 ulp of 1 would round to 1: keep it in the cell
    const float v = __double2float_rn(o);
    return v >= 1.0f ? 0x1.fffffep-1f : v;
}

template <>
__device__ __forceinline__ double unit_offset<double>(double o)
{
    return o;
}

template <typename R>
__device__ __forceinline__ R narrow(double v);
template <>
__device__ __forceinline__ float narrow<float>(double v) { return __double2float_rn(v); }
template <>
__device__ __forceinline__ double narrow<double>(double v) { return v; }

template <typename R>
__device__ __forceinline__ void store_particle(const InstDev &I, int slot, int cell, const double off[3],
                                               const double u[3], double w, int id)
{
    I.cell[0][slot] = cell;
    if (I.id[0]) I.id[0][slot] = id;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (I.off[0][a]) ((R *)I.off[0][a])[slot] = unit_offset<R>(off[a]);
        ((R *)I.u[0][a])[slot] = narrow<R>(u[a]);
    }
    ((R *)I.w[0])[slot] = narrow<R>(w);
}

// SplitMix64 (Steele, Lea, Flood, OOPSLA 2014) as a counter-based generator
__device__ __forceinline__ uint64_t splitmix(uint64_t seed, uint64_t stream, uint64_t counter)
{
    uint64_t z = (seed ^ (stream << 40) ^ counter) + 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

__device__ __forceinline__ double uniform01(uint64_t seed, uint64_t stream, uint64_t counter)
{
    return (double)(splitmix(seed, stream, counter) >> 11) * 0x1.0p-53;
}

__device__ __forceinline__ double normal01(uint64_t seed, uint64_t stream, uint64_t counter)
{
    // Box-Muller, cosine branch
    const double r = sqrt(__dmul_rn(-2.0, log(__dsub_rn(1.0, uniform01(seed, stream, counter)))));
    return __dmul_rn(r, cos(__dmul_rn(6.283185307179586, uniform01(seed, stream + 1, counter))));
}

// Candidate p of cell `cidx`: kSkip when its weight is zero (no id), kOutside when it
// has a weight but falls outside the box (its id is used up, as on the host), kPlaced.
enum { kSkip = 0, kOutside = 1, kPlaced = 2 };

__device__ int plasma_candidate(const PlasmaGen &G, long long cidx, int p, int &cell, double off[3], double u[3],
                                 double &w)
{
    const int cc[3] = {(int)(cidx % G.n[0]), (int)((cidx / G.n[0]) % G.n[1]), (int)(cidx / ((long long)G.n[0] * G.n[1]))};
    const uint64_t ctr = (uint64_t)cidx * (uint64_t)G.ppc + (uint64_t)p;
    double pos[3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
        pos[a] = (a == 1 && G.ndim == 2) ? 0.0 : __dmul_rn(__dadd_rn((double)cc[a], uniform01(G.seed, a, ctr)), G.dx[a]);
    // density at the lab position of the t' = 0 sample
    const double zl = __dmul_rn(G.gb, pos[2]);
    double prof = 1.0;
    if (zl < G.zs) prof = 0.0;
    else if (G.ramp > 0.0 && zl < __dadd_rn(G.zs, G.ramp)) prof = __ddiv_rn(__dsub_rn(zl, G.zs), G.ramp);
    w = __ddiv_rn(__dmul_rn(__dmul_rn(__dmul_rn(G.gb, G.n0), prof), G.dV), (double)G.ppc);
    if (w == 0.0) return kSkip;
    double ul[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) ul[a] = __dmul_rn(G.uth[a], normal01(G.seed, 3 + 2 * (uint64_t)a, ctr));
    // boost of the lab momentum along z
    const double gl = __dsqrt_rn(__dadd_rn(__dadd_rn(__dadd_rn(1.0, __dmul_rn(ul[0], ul[0])), __dmul_rn(ul[1], ul[1])),
                                           __dmul_rn(ul[2], ul[2])));
    u[0] = ul[0];
    u[1] = ul[1];
    u[2] = __dmul_rn(G.gb, __dsub_rn(ul[2], __dmul_rn(G.beta, gl)));
    // cell and in-cell offset
    int c[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (a == 1 && G.ndim == 2) {
            c[a] = 0;
            off[a] = 0.0;
            continue;
        }
        const double x = __ddiv_rn(pos[a], G.dx[a]);
        const double k = floor(x);
        c[a] = (int)k;
        off[a] = __dsub_rn(x, k);
        if (off[a] >= 1.0) {
            off[a] = 0.0;
            c[a] += 1;
        }
        if (c[a] < 0 || c[a] >= G.n[a]) return kOutside;
    }
    cell = c[0] + G.n[0] * (c[1] + G.n[1] * c[2]);
    return kPlaced;
}

}  // namespace

// S: the source precision (an FP32 source widens exactly and narrows back to itself)
template <typename R, typename S>
__global__ void __launch_bounds__(256) k_place(InstDev I, PlaceSrc s)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= s.n) return;
    const S *so = (const S *)s.off, *su = (const S *)s.u, *sw = (const S *)s.w;
    const double off[3] = {(double)so[3 * i], (double)so[3 * i + 1], (double)so[3 * i + 2]};
    const double u[3] = {(double)su[3 * i], (double)su[3 * i + 1], (double)su[3 * i + 2]};
    store_particle<R>(I, s.slot[i], s.cell[i], off, u, (double)sw[i], s.id ? s.id[i] : (int)(s.id_base + i));
}

// Read-out staging (storage precision, canonical order) placed again: particle i goes to
// slot map[i] of buffer 0, or, for map[i] < 0, to position -1 - map[i] of buffer 1 (the
// particles taken out, packed).  No conversion: the values keep their bits.
template <typename R>
__global__ void __launch_bounds__(256) k_place_staged(InstDev I, StagedSrc s)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= s.n) return;
    const int m = s.map[i];
    const int b = m >= 0 ? 0 : 1;
    const int d = m >= 0 ? m : -1 - m;
    I.cell[b][d] = s.cell[i];
    if (I.id[b]) I.id[b][d] = s.id[i];
    const R *off = (const R *)s.off, *u = (const R *)s.u;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (I.off[b][a]) ((R *)I.off[b][a])[d] = off[3 * i + a];
        ((R *)I.u[b][a])[d] = u[3 * i + a];
    }
    ((R *)I.w[b])[d] = ((const R *)s.w)[i];
}

// per cell: particles placed (low 16 bits) and ids used (high bits); count[ncell] is set
// when a candidate lands in a cell other than the one that drew it (an offset rounding
// to the next cell), which the layout by drawing cell does not cover
__global__ void __launch_bounds__(256) k_plasma_count(PlasmaGen G, int *count)
{
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= G.ncell) return;
    int placed = 0, ids = 0;
    bool moved = false;
    for (int p = 0; p < G.ppc; ++p) {
        int cell;
        double off[3], u[3], w;
        const int r = plasma_candidate(G, c, p, cell, off, u, w);
        placed += r == kPlaced;
        ids += r != kSkip;
        moved = moved || (r == kPlaced && cell != c);
    }
    count[c] = placed | (ids << 16);
    if (moved) atomicOr(count + G.ncell, 1);
}

template <typename R>
__global__ void __launch_bounds__(256) k_plasma_write(InstDev I, PlasmaGen G, const int *slot0, const int *id0)
{
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= G.ncell) return;
    int slot = slot0[c], id = id0[c];
    for (int p = 0; p < G.ppc; ++p) {
        int cell;
        double off[3], u[3], w;
        const int r = plasma_candidate(G, c, p, cell, off, u, w);
        if (r == kPlaced) store_particle<R>(I, slot++, cell, off, u, w, id);
        id += r != kSkip;
    }
}

cudaError_t launch_place(int fp64, const InstDev &I, const PlaceSrc &s, cudaStream_t st)
{
    if (s.n <= 0) return cudaSuccess;
    const unsigned blocks = (unsigned)((s.n + 255) / 256);
    if (fp64) k_place<double, double><<<blocks, 256, 0, st>>>(I, s);
    else if (s.f32) k_place<float, float><<<blocks, 256, 0, st>>>(I, s);
    else k_place<float, double><<<blocks, 256, 0, st>>>(I, s);
    return cudaGetLastError();
}

cudaError_t launch_place_staged(int fp64, const InstDev &I, const StagedSrc &s, cudaStream_t st)
{
    if (s.n <= 0) return cudaSuccess;
    const unsigned blocks = (unsigned)((s.n + 255) / 256);
    if (fp64) k_place_staged<double><<<blocks, 256, 0, st>>>(I, s);
    else k_place_staged<float><<<blocks, 256, 0, st>>>(I, s);
    return cudaGetLastError();
}

cudaError_t launch_plasma_count(const PlasmaGen &G, int *count, cudaStream_t st)
{
    k_plasma_count<<<(unsigned)((G.ncell + 255) / 256), 256, 0, st>>>(G, count);
    return cudaGetLastError();
}

cudaError_t launch_plasma_write(int fp64, const InstDev &I, const PlasmaGen &G, const int *slot0, const int *id0,
                                cudaStream_t st)
{
    const unsigned blocks = (unsigned)((G.ncell + 255) / 256);
    if (fp64) k_plasma_write<double><<<blocks, 256, 0, st>>>(I, G, slot0, id0);
    else k_plasma_write<float><<<blocks, 256, 0, st>>>(I, G, slot0, id0);
    return cudaGetLastError();
}

}  // namespace pic
