// k_particles.cu -- particle-side helper kernels of the boosted-frame PIC step: the
// tile population scan that lays out each step's particle array, the canonical-order
// read-out, and the FP64 particle reductions and charge deposit used by the getters.
#include "k_particles.cuh"

namespace pic {

// -------------------------------------------------------------------------------------
// Tile population scan: one CTA per instance.  mode 0 (step): lays out the output
// layout (segment starts and chunk bases) from the populations, zeroes them, flips the
// parity and counts the particle phase.  mode 1 (read-out): writes the exclusive scan of the populations into
// `dst` (one int per tile + total) and the total into *live, changing nothing else.
// -------------------------------------------------------------------------------------
// The same table computed by one warp per tile ahead of the particle kernel (no block
// barriers, at full occupancy), stored as the tile's source record: the particle count,
// the number of non-empty sub-ranges (-1 when more than kSubCache) and their first slots
// and positions.  The particle kernel loads it in one coalesced read and builds the table
// itself only for a tile whose record overflowed.
struct SrcScratch {
    int n;
    int dir[kDirs], seg[kDirs], c0[kDirs];
    int chpre[kDirs + 1];
};

__global__ void __launch_bounds__(256) k_tile_sources(Launch L)
{
    __shared__ SrcScratch W[8];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = blockIdx.x * 8 + warp;
    if (g >= L.total_tiles) return;  // the whole warp
    const int ii = find_instance(L.tile_start, L.ninst, g);
    const InstDev &I = L.inst[ii];
    const int t = g - L.tile_start[ii];
    const int lay = 1 - *I.cur;  // the input layout of the coming phase (the scan flipped it)
    const int tx = t % I.nt[0], ty = (t / I.nt[0]) % I.nt[1], tz = t / (I.nt[0] * I.nt[1]);
    SrcScratch &S = W[warp];
    const int *pre = I.chunk_pre[lay];
    int dx[3], sx[3], dy[3], sy[3], dz[3], sz[3];
    const int mx = axis_sources(tx, I.nt[0], I.bc[0], dx, sx);
    const int my = I.ndim == 3 ? axis_sources(ty, I.nt[1], I.bc[1], dy, sy) : 1;
    if (I.ndim != 3) { dy[0] = 0; sy[0] = 0; }
    const int mz = axis_sources(tz, I.nt[2], I.bc[2], dz, sz);
    const int n = mx * my * mz;
    int nch = 0;
    if (lane < n) {
        const int c = lane % mx, b = (lane / mx) % my, a = lane / (mx * my);
        const int st = sx[c] + I.nt[0] * (sy[b] + I.nt[1] * sz[a]);
        const int d = (dz[a] + 1) * 9 + (dy[b] + 1) * 3 + (dx[c] + 1);
        const int c0 = I.chunk_base[lay][st];
        nch = I.chunk_base[lay][st + 1] - c0;
        S.dir[lane] = d;
        S.seg[lane] = I.seg[lay][st];
        S.c0[lane] = c0;
    }
    int pn = nch;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int yn = __shfl_up_sync(0xffffffffu, pn, o);
        if (lane >= o) pn += yn;
    }
    if (lane < n) S.chpre[lane] = pn - nch;
    if (lane == n - 1) S.chpre[n] = pn;
    __syncwarp();
    const int npairs = S.chpre[n];
    int *rec = I.srcrec + (size_t)t * kSrcRec;
    int written = 0, slot_run = 0;
    bool fits = true;
    for (int q0 = 0; q0 < npairs; q0 += 32) {
        const int q = q0 + lane;
        int cntq = 0, posq = 0;
        if (q < npairs) {
            int s = 0, top = n - 1;
            while (s < top) {
                const int mid = (s + top + 1) >> 1;
                if (S.chpre[mid] <= q) s = mid; else top = mid - 1;
            }
            const int k = q - S.chpre[s];
            const long long c = S.c0[s] + k;
            const int d = S.dir[s];
            const int p0 = pre[c * kPre + d];
            cntq = pre[c * kPre + d + 1] - p0;
            posq = S.seg[s] + k * I.R + p0;
        }
        const int ne = cntq > 0 ? 1 : 0;
        int ic = cntq, in_ = ne;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y1 = __shfl_up_sync(0xffffffffu, ic, o);
            const int y2 = __shfl_up_sync(0xffffffffu, in_, o);
            if (lane >= o) { ic += y1; in_ += y2; }
        }
        const int tot_cnt = __shfl_sync(0xffffffffu, ic, 31), tot_ne = __shfl_sync(0xffffffffu, in_, 31);
        if (written + tot_ne > kSubCache) fits = false;
        if (fits && ne) {
            rec[kRecSlot + written + in_ - 1] = slot_run + ic - cntq;
            rec[kRecPos + written + in_ - 1] = posq;
        }
        written += tot_ne;
        slot_run += tot_cnt;
    }
    if (lane == 0) {
        rec[0] = slot_run;
        rec[1] = fits ? written : -1;
        if (fits) rec[kRecSlot + written] = slot_run;
    }
}

__global__ void __launch_bounds__(1024) k_scan(Launch L, int mode, int *const *dst)
{
    const InstDev &I = L.inst[blockIdx.x];
    __shared__ int s_warp[32], s_warp2[32];
    __shared__ int s_carry, s_carry2;
    const int cur = *I.cur;
    const int out = 1 - cur;
    const int nt = I.ntiles;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) { s_carry = 0; s_carry2 = 0; }
    __syncthreads();
    for (int base = 0; base < nt; base += 1024) {
        const int t = base + tid;
        const int p = t < nt ? I.pop[t] : 0;
        const int ch = (p + I.R - 1) / I.R;
        int a = p, b = ch;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int x = __shfl_up_sync(0xffffffffu, a, o);
            const int y = __shfl_up_sync(0xffffffffu, b, o);
            if (lane >= o) { a += x; b += y; }
        }
        if (lane == 31) { s_warp[warp] = a; s_warp2[warp] = b; }
        __syncthreads();
        if (warp == 0) {
            int x = s_warp[lane], y = s_warp2[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int xx = __shfl_up_sync(0xffffffffu, x, o);
                const int yy = __shfl_up_sync(0xffffffffu, y, o);
                if (lane >= o) { x += xx; y += yy; }
            }
            s_warp[lane] = x;
            s_warp2[lane] = y;
        }
        __syncthreads();
        const int ex = s_carry + (warp ? s_warp[warp - 1] : 0) + a - p;
        const int ex2 = s_carry2 + (warp ? s_warp2[warp - 1] : 0) + b - ch;
        if (t < nt) {
            if (mode == 0) {
                I.seg[out][t] = ex;
                I.chunk_base[out][t] = ex2;
                I.pop[t] = 0;
            } else {
                dst[blockIdx.x][t] = ex;
            }
        }
        __syncthreads();
        if (tid == 0) { s_carry += s_warp[31]; s_carry2 += s_warp2[31]; }
        __syncthreads();
    }
    if (tid == 0) {
        if (mode == 0) {
            I.seg[out][nt] = s_carry;
            I.chunk_base[out][nt] = s_carry2;
            if (s_carry > I.cap || s_carry2 > I.chunk_cap) atomicOr(I.err, kErrCapacity);
            *I.cur = out;
            *I.phase += 1;  // one more particle phase (the ion current read the old count)
        } else {
            dst[blockIdx.x][nt] = s_carry;
        }
        *I.live = s_carry;
    }
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

template <typename R>
__global__ void __launch_bounds__(256) k_particle_sums(Launch L, double *sums /* 2 per instance */)
{
    const int g = blockIdx.x;
    const int ii = find_instance(L.tile_start, L.ninst, g);
    const InstDev &I = L.inst[ii];
    const int t = g - L.tile_start[ii];
    const int cur = *I.cur;
    const int s0 = I.seg[cur][t];
    const int c0 = I.chunk_base[cur][t], c1 = I.chunk_base[cur][t + 1];
    double ke = 0.0, q = 0.0;
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
                // FP32 storage: gamma - 1 = u^2 / (1 + gamma) in FP32 (no cancellation; the
                // stored momenta carry FP32 precision anyway), summed in FP64
                const float uu = (float)u[0] * (float)u[0] + (float)u[1] * (float)u[1] + (float)u[2] * (float)u[2];
                ke += (double)((float)w * (uu / (1.f + sqrtf(1.f + uu)))) * I.m;
            }
            q += I.q * (double)w;
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        ke += __shfl_down_sync(0xffffffffu, ke, o);
        q += __shfl_down_sync(0xffffffffu, q, o);
    }
    // one pair of atomics per block (the tile's instance), not per warp
    __shared__ double s_ke[8], s_q[8];
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
cudaError_t dispatch_particles_f32(int ndim, int order, int pusher, const Launch *L, size_t smem, cudaStream_t s);
cudaError_t dispatch_particles_f64(int ndim, int order, int pusher, const Launch *L, size_t smem, cudaStream_t s);
cudaError_t dispatch_particles_f32_inj(int ndim, int order, int pusher, const Launch *L, size_t smem, cudaStream_t s);
cudaError_t dispatch_particles_f64_inj(int ndim, int order, int pusher, const Launch *L, size_t smem, cudaStream_t s);

static cudaError_t dispatch_particles(int ndim, int order, int fp64, int pusher, bool inj, const Launch *L, size_t smem,
                                      cudaStream_t s)
{
    if (fp64)
        return inj ? dispatch_particles_f64_inj(ndim, order, pusher, L, smem, s)
                   : dispatch_particles_f64(ndim, order, pusher, L, smem, s);
    return inj ? dispatch_particles_f32_inj(ndim, order, pusher, L, smem, s)
               : dispatch_particles_f32(ndim, order, pusher, L, smem, s);
}

cudaError_t launch_particles(int ndim, int order, int fp64, int pusher, bool inj, const Launch &L, size_t smem,
                             cudaStream_t s)
{
    return dispatch_particles(ndim, order, fp64, pusher, inj, &L, smem, s);
}

cudaError_t prepare_particles(int ndim, int order, int fp64, int pusher, size_t smem)
{
    cudaError_t e = dispatch_particles(ndim, order, fp64, pusher, false, nullptr, smem, 0);
    return e == cudaSuccess ? dispatch_particles(ndim, order, fp64, pusher, true, nullptr, smem, 0) : e;
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
    if (fp64)
        k_particle_sums<double><<<L.total_tiles, 256, 0, s>>>(L, sums);
    else
        k_particle_sums<float><<<L.total_tiles, 256, 0, s>>>(L, sums);
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
