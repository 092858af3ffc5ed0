// k_particles.cu -- particle-side helper kernels of the boosted-frame PIC step: the
// tile population scan that lays out each step's particle array, the canonical-order
// read-out, and the FP64 particle reductions and charge deposit used by the getters.
#include "k_particles.cuh"

namespace pic {

// Source records of every tile, one warp per tile (tile_sources_warp).
__global__ void __launch_bounds__(256) k_tile_sources(Launch L)
{
    __shared__ SrcScratch W[8];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = blockIdx.x * 8 + warp;
    if (g >= L.total_tiles) return;  // the whole warp
    tile_sources_warp(L, g, W[warp], lane);
}

// Tile population scan, one CTA per instance (scan_instance).
__global__ void __launch_bounds__(1024) k_scan(Launch L, int mode, int *const *dst)
{
    __shared__ int sh[66];
    scan_instance(L, blockIdx.x, mode, dst, sh);
}

// -------------------------------------------------------------------------------------
// Read-out of the particles in canonical order: per destination tile, the same source
// walk as the step, into FP64 / int32 staging arrays at the scanned tile offsets.
// -------------------------------------------------------------------------------------
// read-out staging, values in the storage precision R (widened to FP64 on the host)
template <typename R>
struct Stage {
    int *cell;
    R *off;  // 3 per particle
    R *u;    // 3 per particle
    R *w;
    int *id;
};

template <typename R>
__global__ void __launch_bounds__(256) k_readout(Launch L, const int *const *start, Stage<R> out)
{
    __shared__ SrcTable S;
    const int g = blockIdx.x;
    const int ii = find_instance(L.tile_start, L.ninst, g);
    const InstDev &I = L.inst[ii];
    const int t = g - L.tile_start[ii];
    const int cur = *I.cur;
    const int tx = t % I.nt[0], ty = (t / I.nt[0]) % I.nt[1], tz = t / (I.nt[0] * I.nt[1]);
    build_sources(I, cur, tx, ty, tz, S);
    const int dst0 = start[ii][t];
    for (int p = threadIdx.x; p < S.count; p += blockDim.x) {
        const int pos = slot_position(I, cur, S, p);
        if (pos < 0 || pos >= I.cap) { atomicOr(I.err, kErrInternal); continue; }
        const long long q = dst0 + p;
        out.cell[q] = I.cell[cur][pos];
        out.off[3 * q + 0] = ((const R *)I.off[cur][0])[pos];
        out.off[3 * q + 1] = I.ndim == 3 ? ((const R *)I.off[cur][1])[pos] : R(0);
        out.off[3 * q + 2] = ((const R *)I.off[cur][2])[pos];
        for (int a = 0; a < 3; ++a) out.u[3 * q + a] = ((const R *)I.u[cur][a])[pos];
        out.w[q] = ((const R *)I.w[cur])[pos];
        out.id[q] = I.id[cur] ? I.id[cur][pos] : (int)q;
    }
}

// -------------------------------------------------------------------------------------
// Particle reductions for the diagnostics and the charge density: walk every live
// particle of the current layout (per tile, the chunks' live prefix: buckets 0..26).
// -------------------------------------------------------------------------------------
template <typename R>
__device__ __forceinline__ void load_particle(const InstDev &I, int lay, int pos, int &cell, R o[3], R u[3], R &w)
{
    cell = I.cell[lay][pos];
    o[0] = ((const R *)I.off[lay][0])[pos];
    o[1] = I.ndim == 3 ? ((const R *)I.off[lay][1])[pos] : R(0);
    o[2] = ((const R *)I.off[lay][2])[pos];
    for (int a = 0; a < 3; ++a) u[a] = ((const R *)I.u[lay][a])[pos];
    w = ((const R *)I.w[lay])[pos];
}

// FP64 kinetic energy and charge sums per instance.  Each block takes kSumTiles
// consecutive tiles of the launch and adds, for every instance they belong to, its part
// with one pair of atomics (one pair per tile before: tens of thousands on two addresses).
constexpr int kSumTiles = 16;

template <typename R>
__global__ void __launch_bounds__(256) k_particle_sums(Launch L, double *sums /* 2 per instance */)
{
    __shared__ double s_ke[8], s_q[8];
    const int g0 = blockIdx.x * kSumTiles, g1 = min(g0 + kSumTiles, L.total_tiles);
    if (g0 >= g1) return;
    int ii = find_instance(L.tile_start, L.ninst, g0);
    for (int lo = g0; lo < g1; ++ii) {
        const int hi = min(g1, L.tile_start[ii + 1]);
        const InstDev &I = L.inst[ii];
        const int cur = *I.cur;
        // an instance with a device error may hold a step's layout half written: its
        // chunk records are not read (the read-out reports the error instead)
        const bool skip = *(volatile const int *)I.err != 0;
        double ke = 0.0, q = 0.0;
        for (int g = skip ? hi : lo; g < hi; ++g) {
            const int t = g - L.tile_start[ii];
            const int s0 = I.seg[cur][t];
            const int c0 = I.chunk_base[cur][t], c1 = I.chunk_base[cur][t + 1];
            for (int c = c0; c < c1; ++c) {
                const int live = I.chunk_pre[cur][(long long)c * kPre + kDead];
                const int start = s0 + (c - c0) * I.R;
                for (int p = threadIdx.x; p < live; p += blockDim.x) {
                    const int pos = start + p;  // momenta and weight only: half the particle's bytes
                    R u[3];
                    for (int a = 0; a < 3; ++a) u[a] = ((const R *)I.u[cur][a])[pos];
                    const R w = ((const R *)I.w[cur])[pos];
                    if (sizeof(R) == 8) {
                        const double g2 = 1.0 + (double)u[0] * u[0] + (double)u[1] * u[1] + (double)u[2] * u[2];
                        ke += (double)w * I.m * (sqrt(g2) - 1.0);
                    } else {
                        // FP32 storage: gamma - 1 = u^2 / (1 + gamma) in FP32 (no cancellation;
                        // the stored momenta carry FP32 precision anyway), summed in FP64
                        const float uu = (float)u[0] * (float)u[0] + (float)u[1] * (float)u[1] + (float)u[2] * (float)u[2];
                        ke += (double)((float)w * (uu / (1.f + sqrtf(1.f + uu)))) * I.m;
                    }
                    q += I.q * (double)w;
                }
            }
        }
        for (int o = 16; o > 0; o >>= 1) {
            ke += __shfl_down_sync(0xffffffffu, ke, o);
            q += __shfl_down_sync(0xffffffffu, q, o);
        }
        __syncthreads();  // the shared sums of the previous instance are read
        if ((threadIdx.x & 31) == 0) {
            s_ke[threadIdx.x >> 5] = ke;
            s_q[threadIdx.x >> 5] = q;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            double a = 0.0, b = 0.0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
                a += s_ke[w];
                b += s_q[w];
            }
            if (a != 0.0) atomicAdd(sums + 2 * ii + 0, a);
            if (b != 0.0) atomicAdd(sums + 2 * ii + 1, b);
        }
        lo = hi;
    }
}

template <int ORD, typename R>
__global__ void __launch_bounds__(256) k_rho(Launch L, double *rho /* dense n0*n1*n2 per instance 0 */)
{
    const int g = blockIdx.x;
    const int ii = find_instance(L.tile_start, L.ninst, g);
    const InstDev &I = L.inst[ii];
    const int t = g - L.tile_start[ii];
    const int cur = *I.cur;
    const int s0 = I.seg[cur][t];
    const int c0 = I.chunk_base[cur][t], c1 = I.chunk_base[cur][t + 1];
    const double dV = I.dx[0] * I.dx[1] * I.dx[2];
    for (int c = c0; c < c1; ++c) {
        const int live = I.chunk_pre[cur][(long long)c * kPre + kDead];
        const int start = s0 + (c - c0) * I.R;
        for (int p = threadIdx.x; p < live; p += blockDim.x) {
            int cell;
            R o[3], u[3], w;
            load_particle(I, cur, start + p, cell, o, u, w);
            const int cc[3] = {cell % I.n[0], (cell / I.n[0]) % I.n[1], cell / (I.n[0] * I.n[1])};
            double wt[3][ORD + 1];
            int b[3];
            for (int a = 0; a < 3; ++a) {
                if (I.ndim == 2 && a == 1) {
                    b[a] = 0;
                    for (int q = 0; q <= ORD; ++q) wt[a][q] = q == 0 ? 1.0 : 0.0;
                    continue;
                }
                b[a] = shape_nodal<ORD, double>(cc[a], (double)o[a], wt[a]);
            }
            const double qw = I.q * (double)w / dV;
            for (int k = 0; k <= ORD; ++k)
                for (int j = 0; j <= ORD; ++j)
                    for (int i = 0; i <= ORD; ++i) {
                        const double v = qw * wt[0][i] * wt[1][j] * wt[2][k];
                        if (v == 0.0) continue;
                        int x[3] = {b[0] + i, b[1] + j, b[2] + k};
                        bool keep = true;
                        for (int a = 0; a < 3; ++a) {
                            if (I.ndim == 2 && a == 1) { x[a] = 0; continue; }
                            if (x[a] < 0 || x[a] >= I.n[a]) {
                                if (I.bc[a] == 0) x[a] = (x[a] + I.n[a]) % I.n[a];
                                else keep = false;
                            }
                        }
                        if (keep) atomicAdd(rho + x[0] + (long long)I.n[0] * (x[1] + (long long)I.n[1] * x[2]), v);
                    }
        }
    }
}

// -------------------------------------------------------------------------------------
// Host-side launchers (called from pic_api.cu).
// -------------------------------------------------------------------------------------
cudaError_t dispatch_particles_f32(int ndim, int order, int pusher, const Launch *L, const InstDev *one, size_t smem,
                                   cudaStream_t s);
cudaError_t dispatch_particles_f64(int ndim, int order, int pusher, const Launch *L, const InstDev *one, size_t smem,
                                   cudaStream_t s);
cudaError_t dispatch_particles_f32_inj(int ndim, int order, int pusher, const Launch *L, const InstDev *one, size_t smem,
                                   cudaStream_t s);
cudaError_t dispatch_particles_f64_inj(int ndim, int order, int pusher, const Launch *L, const InstDev *one, size_t smem,
                                   cudaStream_t s);

static cudaError_t dispatch_particles(int ndim, int order, int fp64, int pusher, bool inj, const Launch *L,
                                      const InstDev *one, size_t smem, cudaStream_t s)
{
    if (fp64)
        return inj ? dispatch_particles_f64_inj(ndim, order, pusher, L, one, smem, s)
                   : dispatch_particles_f64(ndim, order, pusher, L, one, smem, s);
    return inj ? dispatch_particles_f32_inj(ndim, order, pusher, L, one, smem, s)
               : dispatch_particles_f32(ndim, order, pusher, L, one, smem, s);
}

cudaError_t launch_particles(int ndim, int order, int fp64, int pusher, bool inj, const Launch &L, const InstDev *one,
                             size_t smem, cudaStream_t s)
{
    return dispatch_particles(ndim, order, fp64, pusher, inj, &L, one, smem, s);
}

cudaError_t prepare_particles(int ndim, int order, int fp64, int pusher, size_t smem)
{
    cudaError_t e = dispatch_particles(ndim, order, fp64, pusher, false, nullptr, nullptr, smem, 0);
    return e == cudaSuccess ? dispatch_particles(ndim, order, fp64, pusher, true, nullptr, nullptr, smem, 0) : e;
}

int particle_chunk() { return kChunk; }
int particle_threads() { return kNT; }

cudaError_t launch_tile_sources(const Launch &L, cudaStream_t s)
{
    k_tile_sources<<<(L.total_tiles + 7) / 8, 256, 0, s>>>(L);
    return cudaGetLastError();
}

cudaError_t launch_scan(const Launch &L, int mode, int *const *dst, cudaStream_t s)
{
    k_scan<<<L.ninst, 1024, 0, s>>>(L, mode, dst);
    return cudaGetLastError();
}

cudaError_t launch_readout(int fp64, const Launch &L, const int *const *start, int *cell, void *off, void *u, void *w,
                           int *id, cudaStream_t s)
{
    if (fp64) {
        Stage<double> st{cell, (double *)off, (double *)u, (double *)w, id};
        k_readout<double><<<L.total_tiles, 256, 0, s>>>(L, start, st);
    } else {
        Stage<float> st{cell, (float *)off, (float *)u, (float *)w, id};
        k_readout<float><<<L.total_tiles, 256, 0, s>>>(L, start, st);
    }
    return cudaGetLastError();
}

cudaError_t launch_particle_sums(int fp64, const Launch &L, double *sums, cudaStream_t s)
{
    const unsigned nb = (unsigned)((L.total_tiles + kSumTiles - 1) / kSumTiles);
    if (fp64)
        k_particle_sums<double><<<nb, 256, 0, s>>>(L, sums);
    else
        k_particle_sums<float><<<nb, 256, 0, s>>>(L, sums);
    return cudaGetLastError();
}

// Loads the density kernels of one (order, precision) on the current device: CUDA loads
// kernels lazily, on their first launch or attribute query.
cudaError_t preload_rho(int order, int fp64)
{
    cudaFuncAttributes a;
    cudaError_t e = order == 1 ? (fp64 ? cudaFuncGetAttributes(&a, k_rho<1, double>) : cudaFuncGetAttributes(&a, k_rho<1, float>))
                               : (fp64 ? cudaFuncGetAttributes(&a, k_rho<2, double>) : cudaFuncGetAttributes(&a, k_rho<2, float>));
    return e == cudaSuccess ? preload_rho_ion() : e;
}

cudaError_t launch_rho(int order, int fp64, const Launch &L, double *rho, cudaStream_t s)
{
    if (order == 1) {
        if (fp64) k_rho<1, double><<<L.total_tiles, 256, 0, s>>>(L, rho);
        else k_rho<1, float><<<L.total_tiles, 256, 0, s>>>(L, rho);
    } else {
        if (fp64) k_rho<2, double><<<L.total_tiles, 256, 0, s>>>(L, rho);
        else k_rho<2, float><<<L.total_tiles, 256, 0, s>>>(L, rho);
    }
    cudaError_t e = cudaGetLastError();
    // plus the ion background of a lab-frame plasma (no-op without one)
    return e == cudaSuccess ? launch_rho_ion(L, L.total_cells, rho, s) : e;
}

}  // namespace pic
