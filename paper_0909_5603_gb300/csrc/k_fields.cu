// k_fields.cu -- grid kernels of the boosted-frame PIC step on sm_103a: Yee FDTD
// half/whole updates with the absorbing layer, binomial current filter sweeps, periodic
// ghost exchange for the TMA gather boxes, and the FP64 field reductions / read-outs.
//
// All stencil kernels run one thread per interior cell of a flattened cell space over
// every instance of the launch (x fastest, so loads and stores coalesce along rows).
// Neighbours along periodic axes wrap by index; along absorbing axes they read the
// zero ghost layers.
#include "k_fields.cuh"

#include <algorithm>

namespace pic {

// Forward difference of F along axis a at padded index p, averaged over the two
// transverse axes with weights 7/12 (itself), 1/12 (edge neighbours), 1/48 (corners);
// up / dn are the +1 / -1 neighbour offsets of the cell (wrapping on periodic axes, 0 on
// an invariant one).
template <typename R>
__device__ __forceinline__ R ck_diff(const R *F, long long p, const long long up[3], const long long dn[3], int a)
{
    const int b = (a + 1) % 3, c = (a + 2) % 3;
    const long long ob[3] = {dn[b], 0, up[b]}, oc[3] = {dn[c], 0, up[c]};
    R sum = R(0);
#pragma unroll
    for (int ib = 0; ib < 3; ++ib)
#pragma unroll
        for (int ic = 0; ic < 3; ++ic) {
            const int edges = (ib != 1) + (ic != 1);
            const R w = edges == 0 ? R(7.0 / 12.0) : (edges == 1 ? R(1.0 / 12.0) : R(1.0 / 48.0));
            const long long q = p + ob[ib] + oc[ic];
            sum += w * (F[q + up[a]] - F[q]);
        }
    return sum;
}

// B <- B - (dt/2) curl E  [then x damping on the second half of the step].  CK: the
// low-dispersion differences (a template parameter, so that the Yee kernel keeps its
// small register footprint and full occupancy)
template <typename R, bool CK>
__global__ void __launch_bounds__(256) k_bhalf(Launch L, int damp)
{
    const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    CellPos c;
    const InstDev *Ip;
    if (!cell_of(L, g, c, Ip)) return;
    const InstDev &I = *Ip;
    long long up[3], dn[3];
    neighbour_offsets(I, c, up, dn);
    const EBPtr F = cur_eb(I);
    const R *Ex = (const R *)F.E[0], *Ey = (const R *)F.E[1], *Ez = (const R *)F.E[2];
    R *Bx = (R *)F.B[0], *By = (R *)F.B[1], *Bz = (R *)F.B[2];
    const StepCoef<R> &K = coef<R>(I);
    const R h = K.half_dt;
    const R ix = K.inv_dx[0], iy = K.inv_dx[1], iz = K.inv_dx[2];
    const long long p = c.p;
    R dEz_dy = R(0), dEy_dz, dEx_dz, dEz_dx, dEy_dx, dEx_dy = R(0);
    if (CK) {
        // low-dispersion solver: each forward difference averaged over its transverse
        // neighbours, 7/12 on itself, 1/12 on the edge and 1/48 on the corner ones (on
        // an invariant axis the neighbours are the cell itself)
        dEy_dz = ck_diff(Ey, p, up, dn, 2) * iz;
        dEx_dz = ck_diff(Ex, p, up, dn, 2) * iz;
        dEz_dx = ck_diff(Ez, p, up, dn, 0) * ix;
        dEy_dx = ck_diff(Ey, p, up, dn, 0) * ix;
        if (I.ndim == 3) {
            dEz_dy = ck_diff(Ez, p, up, dn, 1) * iy;
            dEx_dy = ck_diff(Ex, p, up, dn, 1) * iy;
        }
    } else {
        const R ex = Ex[p], ey = Ey[p], ez = Ez[p];
        dEy_dz = (Ey[p + up[2]] - ey) * iz;
        dEx_dz = (Ex[p + up[2]] - ex) * iz;
        dEz_dx = (Ez[p + up[0]] - ez) * ix;
        dEy_dx = (Ey[p + up[0]] - ey) * ix;
        if (I.ndim == 3) {
            dEz_dy = (Ez[p + up[1]] - ez) * iy;
            dEx_dy = (Ex[p + up[1]] - ex) * iy;
        }
    }
    R bx = Bx[p] - h * (dEz_dy - dEy_dz);
    R by = By[p] - h * (dEx_dz - dEz_dx);
    R bz = Bz[p] - h * (dEy_dx - dEx_dy);
    if (damp) {
        const R f = damp_factor<R>(I, c);
        bx *= f;
        by *= f;
        bz *= f;
    }
    Bx[p] = bx;
    By[p] = by;
    Bz[p] = bz;
}

// The fused Yee update, one CTA per tile and z chunk (maxwell_fused_block).
template <typename R, int ND>
__global__ void __launch_bounds__(256, sizeof(R) == 4 ? 3 : 2) k_maxwell_fused(Launch L, const long long *tile_start,
                                                                              int filtered)
{
    maxwell_fused_block<R, ND>(L, tile_start, filtered, blockIdx.x);
}

// After the fused update: every instance of the launch switches to the buffer pair it
// wrote.
__global__ void k_flip_fields(Launch L)
{
    for (int i = threadIdx.x; i < L.ninst; i += blockDim.x) {
        int *f = L.inst[i].fpar;
        *f ^= 1;
    }
}

// E <- damping x (E + dt (curl B - J)), J = the filtered current of this step.
template <typename R>
__global__ void __launch_bounds__(256) k_efull(Launch L, int filtered)
{
    const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    CellPos c;
    const InstDev *Ip;
    if (!cell_of(L, g, c, Ip)) return;
    const InstDev &I = *Ip;
    long long up[3], dn[3];
    neighbour_offsets(I, c, up, dn);
    const EBPtr F = cur_eb(I);
    const R *Bx = (const R *)F.B[0], *By = (const R *)F.B[1], *Bz = (const R *)F.B[2];
    R *Ex = (R *)F.E[0], *Ey = (R *)F.E[1], *Ez = (R *)F.E[2];
    // one filter sweep per active axis alternates J -> Jt -> J ...
    const int nsweeps = I.filter_passes > 0 ? (I.ndim == 3 ? 3 : 2) : 0;
    void *const *Jsrc = (filtered && (nsweeps & 1)) ? I.Jt : I.J;
    const R *Jx = (const R *)Jsrc[0], *Jy = (const R *)Jsrc[1], *Jz = (const R *)Jsrc[2];
    const StepCoef<R> &K = coef<R>(I);
    const R dt = K.dt;
    const R ix = K.inv_dx[0], iy = K.inv_dx[1], iz = K.inv_dx[2];
    const long long p = c.p;
    const R bx = Bx[p], by = By[p], bz = Bz[p];
    R dBz_dy = R(0), dBy_dz = (by - By[p + dn[2]]) * iz, dBx_dz = (bx - Bx[p + dn[2]]) * iz;
    R dBz_dx = (bz - Bz[p + dn[0]]) * ix, dBy_dx = (by - By[p + dn[0]]) * ix, dBx_dy = R(0);
    if (I.ndim == 3) {
        dBz_dy = (bz - Bz[p + dn[1]]) * iy;
        dBx_dy = (bx - Bx[p + dn[1]]) * iy;
    }
    const R f = damp_factor<R>(I, c);
    Ex[p] = f * (Ex[p] + dt * ((dBz_dy - dBy_dz) - Jx[p]));
    Ey[p] = f * (Ey[p] + dt * ((dBx_dz - dBz_dx) - Jy[p]));
    Ez[p] = f * (Ez[p] + dt * ((dBy_dx - dBx_dy) - Jz[p]));
}

// A pencil is 32 lines parallel to `axis` times kPencil cells along it.  Lines: for the
// x axis, 32 consecutive (y, z) rows; for y and z, 32 consecutive x columns at one z (y).
// Work assignment without divisions: for the x axis a warp walks one line (lanes along x,
// coalesced), the 8 warps take lines 8 at a time; for y and z the lanes take the 32
// columns (coalesced along x) and the warps step along the axis.
template <typename R>
__global__ void __launch_bounds__(256) k_filter_axis(Launch L, int axis, const long long *pencil_start, int src_is_jt)
{
    __shared__ R buf[2][kPencil + 2 * kMaxPasses][33];
    __shared__ long long s_line[32];
    const long long g = blockIdx.x;
    if (g >= pencil_start[L.ninst]) return;
    const int ii = find_instance_ll(pencil_start, L.ninst, g);
    const InstDev &I = L.inst[ii];
    if (!filter_active_axis(I, axis)) return;
    const int P = min(I.filter_passes, kMaxPasses);
    const int n = I.n[axis];
    const bool per = I.bc[axis] == 0;
    const int nseg = (n + kPencil - 1) / kPencil;
    long long r = g - pencil_start[ii];
    const int q0 = (int)(r % nseg) * kPencil;  // first cell of the segment along the axis
    r /= nseg;
    const long long st[3] = {1, I.sy, I.sz};
    const long long sa = st[axis];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    // line c -> padded offset of its cell 0 along the axis, or -1 when the line is absent
    if (tid < 32) {
        long long off = -1;
        const int c = tid;
        if (axis == 0) {
            const long long row = r * 32 + c;
            if (row < (long long)I.n[1] * I.n[2]) {
                const int y = (int)(row % I.n[1]), z = (int)(row / I.n[1]);
                off = I.gh[0] + st[1] * (y + I.gh[1]) + st[2] * (z + I.gh[2]);
            }
        } else {
            const int ncol = (I.n[0] + 31) / 32;
            const int x = (int)(r % ncol) * 32 + c;
            const int other = (int)(r / ncol);  // z for the y axis, y for the z axis
            if (x < I.n[0])
                off = axis == 1 ? (x + I.gh[0]) + st[1] * I.gh[1] + st[2] * (other + I.gh[2])
                                : (x + I.gh[0]) + st[1] * (other + I.gh[1]) + st[2] * I.gh[2];
        }
        s_line[c] = off;
    }
    __syncthreads();
    void *const *src = src_is_jt ? I.Jt : I.J;
    void *const *dst = src_is_jt ? I.J : I.Jt;
    const int len = kPencil + 2 * P;
    // (c, s) iteration: x axis: c = warp + 8 m, s = lane + 32 k; y, z: c = lane, s = warp + 8 k
    const int c_first = axis == 0 ? warp : lane, c_step = axis == 0 ? 8 : 32;
    const int s_first = axis == 0 ? lane : warp, s_step = axis == 0 ? 32 : 8;
    for (int comp = 0; comp < 3; ++comp) {
        const R *a = (const R *)src[comp];
        R *b = (R *)dst[comp];
        for (int c = c_first; c < 32; c += c_step) {
            const long long lo = s_line[c];
            for (int s_ = s_first; s_ < len; s_ += s_step) {
                int q = q0 + s_ - P;
                bool ok = lo >= 0;
                if (q < 0 || q >= n) {
                    // a ragged last pencil can reach more than one period past the end
                    if (per) q = ((q % n) + n) % n;
                    else ok = false;
                }
                buf[0][s_][c] = ok ? a[lo + (long long)q * sa] : R(0);
            }
        }
        __syncthreads();
        int cur = 0;
        for (int pass = 0; pass < P; ++pass) {
            for (int c = c_first; c < 32; c += c_step)
                for (int s_ = s_first; s_ < len; s_ += s_step) {
                    R v = R(0);
                    if (s_ >= 1 && s_ < len - 1) {
                        v = R(0.25) * buf[cur][s_ - 1][c] + R(0.5) * buf[cur][s_][c] + R(0.25) * buf[cur][s_ + 1][c];
                        const int q = q0 + s_ - P;
                        if (!per && (q < 0 || q >= n)) v = R(0);
                    }
                    buf[cur ^ 1][s_][c] = v;
                }
            __syncthreads();
            cur ^= 1;
        }
        for (int c = c_first; c < 32; c += c_step) {
            const long long lo = s_line[c];
            if (lo < 0) continue;
            for (int s_ = s_first; s_ < kPencil; s_ += s_step) {
                const int q = q0 + s_;
                if (q < n) b[lo + (long long)q * sa] = buf[cur][s_ + P][c];
            }
        }
        __syncthreads();
    }
}

template <typename R, int P>
__global__ void __launch_bounds__(256) k_filter_col(Launch L, int axis, const long long *pencil_start, int src_is_jt)
{
    filter_col_block<R, P>(L, axis, pencil_start, src_is_jt, blockIdx.x);
}

template <typename R, int P>
__global__ void __launch_bounds__(256) k_filter_row(Launch L, const long long *pencil_start, int src_is_jt)
{
    __shared__ R sw[8 * 3 * (kPencil + 2 * P)];
    filter_row_block<R, P>(L, pencil_start, src_is_jt, blockIdx.x, sw);
}

// Periodic ghost exchange of the six E/B components along one axis, per_inst_max
// elements per instance (ghost_elem).
template <typename R>
__global__ void __launch_bounds__(256) k_ghost(Launch L, int axis, long long per_inst_max)
{
    const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int ii = (int)(g / per_inst_max);
    if (ii >= L.ninst) return;
    const InstDev &I = L.inst[ii];
    const long long r = g - (long long)ii * per_inst_max;
    if (r < ghost_elems(I, axis)) ghost_elem<R>(I, axis, r);
}

// FP64 field energy sums (1/2) sum (E^2 + B^2) dV per instance.  Each block takes a
// contiguous range of kEnergyCells cells of the flattened cell space and, for every
// instance the range meets, sums its part (each cell's E^2 + B^2 in the storage
// precision, then FP64) and adds it with one atomic: a few thousand atomics per call
// instead of one per 256 cells, all on the same address.
constexpr long long kEnergyCells = 8192;

// sum of v over the block (every thread gets it)
__device__ __forceinline__ double block_sum(double v, double *red)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();  // red is free
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    return t;
}

template <typename R>
__global__ void __launch_bounds__(256) k_field_energy(Launch L, double *sums)
{
    __shared__ double red[8];
    const long long b0 = (long long)blockIdx.x * kEnergyCells;
    const long long b1 = min(b0 + kEnergyCells, L.total_cells);
    if (b0 >= b1) return;
    int ii = find_instance_ll(L.cell_start, L.ninst, b0);
    for (long long lo = b0; lo < b1; ++ii) {
        const long long hi = min(b1, L.cell_start[ii + 1]);
        const InstDev &I = L.inst[ii];
        const R *Ex = (const R *)eb_field(I, 0), *Ey = (const R *)eb_field(I, 1), *Ez = (const R *)eb_field(I, 2);
        const R *Bx = (const R *)eb_field(I, 3), *By = (const R *)eb_field(I, 4), *Bz = (const R *)eb_field(I, 5);
        double e = 0.0;
        for (long long g = lo + threadIdx.x; g < hi; g += blockDim.x) {
            const int r = (int)(g - L.cell_start[ii]);
            const int rq = fast_div(r, I.div_n0);
            const int i = r - rq * I.n[0];
            const int k = fast_div(rq, I.div_n1);
            const int j = rq - k * I.n[1];
            const long long p = (i + I.gh[0]) + I.sy * (j + I.gh[1]) + I.sz * (k + I.gh[2]);
            // the cell's E^2 + B^2 in the storage precision, then FP64
            R s2 = Ex[p] * Ex[p] + Bx[p] * Bx[p];
            s2 += Ey[p] * Ey[p] + By[p] * By[p];
            s2 += Ez[p] * Ez[p] + Bz[p] * Bz[p];
            e += (double)s2;
        }
        const double t = block_sum(e, red);
        if (threadIdx.x == 0 && t != 0.0) atomicAdd(sums + 2 * L.ninst + ii, t * (0.5 * I.dx[0] * I.dx[1] * I.dx[2]));
        lo = hi;
    }
}

// Interior values of one component as dense FP64 (x fastest), for the z planes k0 ..
// k0 + ncell / (n0 n1) - 1 (k0 = 0 and ncell = every cell for a whole field)
template <typename R>
__global__ void k_pack(InstDev I, int comp, int filtered, double *dense, long long ncell, int k0)
{
    const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= ncell) return;
    const int i = (int)(g % I.n[0]);
    const int j = (int)((g / I.n[0]) % I.n[1]);
    const int k = k0 + (int)(g / ((long long)I.n[0] * I.n[1]));
    const long long p = (i + I.gh[0]) + I.sy * (j + I.gh[1]) + I.sz * (k + I.gh[2]);
    const void *src;
    if (comp < 6) src = eb_field(I, comp);
    else {
        const int nsweeps = I.filter_passes > 0 ? (I.ndim == 3 ? 3 : 2) : 0;
        src = (filtered && (nsweeps & 1)) ? I.Jt[comp - 6] : I.J[comp - 6];
    }
    dense[g] = (double)((const R *)src)[p];
}

// The inverse of k_pack: writes (add = 0) or adds (add = 1) dense FP64 values
template <typename R>
__global__ void k_unpack(InstDev I, int comp, const double *dense, long long ncell, int k0, int add)
{
    const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= ncell) return;
    const int i = (int)(g % I.n[0]);
    const int j = (int)((g / I.n[0]) % I.n[1]);
    const int k = k0 + (int)(g / ((long long)I.n[0] * I.n[1]));
    const long long p = (i + I.gh[0]) + I.sy * (j + I.gh[1]) + I.sz * (k + I.gh[2]);
    R *dst = (R *)(comp < 6 ? eb_field(I, comp) : I.J[comp - 6]);
    dst[p] = add ? (R)((double)dst[p] + dense[g]) : (R)dense[g];
}

// div E on nodes: sum_a (E_a[i] - E_a[i - e_a]) / dx_a
template <typename R>
__global__ void k_dive(InstDev I, double *dense, long long ncell)
{
    const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= ncell) return;
    CellPos c;
    c.i = (int)(g % I.n[0]);
    c.j = (int)((g / I.n[0]) % I.n[1]);
    c.k = (int)(g / ((long long)I.n[0] * I.n[1]));
    c.p = (c.i + I.gh[0]) + I.sy * (c.j + I.gh[1]) + I.sz * (c.k + I.gh[2]);
    long long up[3], dn[3];
    neighbour_offsets(I, c, up, dn);
    double d = 0.0;
    for (int a = 0; a < 3; ++a) {
        if (I.ndim == 2 && a == 1) continue;
        const R *E = (const R *)eb_field(I, a);
        d += ((double)E[c.p] - (double)E[c.p + dn[a]]) / I.dx[a];
    }
    dense[g] = d;
}

// ------------------------------------------------------------------------------------
static inline unsigned blocks_for(long long n, int t) { return (unsigned)((n + t - 1) / t); }

template <typename R, int P>
static void filter_fixed(const Launch &L, int axis, unsigned nb, const long long *start, int src_is_jt, cudaStream_t s)
{
    if (axis == 0)
        k_filter_row<R, P><<<nb, 256, 0, s>>>(L, start, src_is_jt);
    else
        k_filter_col<R, P><<<nb, 256, 0, s>>>(L, axis, start, src_is_jt);
}

template <typename R>
static void filter_axis(const Launch &L, int axis, int passes, unsigned nb, const long long *start, int src_is_jt,
                        cudaStream_t s)
{
    switch (passes) {
    case 1: filter_fixed<R, 1>(L, axis, nb, start, src_is_jt, s); break;
    case 2: filter_fixed<R, 2>(L, axis, nb, start, src_is_jt, s); break;
    case 3: filter_fixed<R, 3>(L, axis, nb, start, src_is_jt, s); break;
    case 4: filter_fixed<R, 4>(L, axis, nb, start, src_is_jt, s); break;
    default: k_filter_axis<R><<<nb, 256, 0, s>>>(L, axis, start, src_is_jt); break;
    }
}

template <typename R, int ND>
static cudaError_t maxwell_fused_attr()
{
    return cudaFuncSetAttribute(k_maxwell_fused<R, ND>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)maxwell_fused_smem<R, ND>());
}

cudaError_t launch_maxwell_fused(int fp64, int ndim, const Launch &L, const long long *tile_start, long long ntiles,
                                 int filtered, cudaStream_t s)
{
    if (ntiles <= 0) return cudaSuccess;
    const unsigned nb = (unsigned)ntiles;
    if (fp64) {
        if (ndim == 3) k_maxwell_fused<double, 3><<<nb, 256, maxwell_fused_smem<double, 3>(), s>>>(L, tile_start, filtered);
        else k_maxwell_fused<double, 2><<<nb, 256, maxwell_fused_smem<double, 2>(), s>>>(L, tile_start, filtered);
    } else {
        if (ndim == 3) k_maxwell_fused<float, 3><<<nb, 256, maxwell_fused_smem<float, 3>(), s>>>(L, tile_start, filtered);
        else k_maxwell_fused<float, 2><<<nb, 256, maxwell_fused_smem<float, 2>(), s>>>(L, tile_start, filtered);
    }
    k_flip_fields<<<1, 128, 0, s>>>(L);
    return cudaGetLastError();
}

cudaError_t prepare_fields(int fp64)
{
    cudaError_t e = fp64 ? maxwell_fused_attr<double, 3>() : maxwell_fused_attr<float, 3>();
    if (e == cudaSuccess) e = fp64 ? maxwell_fused_attr<double, 2>() : maxwell_fused_attr<float, 2>();
    return e;
}

cudaError_t launch_filter(int fp64, const Launch &L, const long long *const pencil_start[3],
                          const long long pencil_total[3], int ndim, int passes, cudaStream_t s)
{
    // axes in order x, (y,) z; sweep k reads J when k is even, Jt when odd
    int k = 0;
    for (int axis = 0; axis < 3; ++axis) {
        if (ndim == 2 && axis == 1) continue;
        if (pencil_total[axis] > 0) {
            const unsigned nb = (unsigned)pencil_total[axis];
            if (fp64)
                filter_axis<double>(L, axis, passes, nb, pencil_start[axis], k & 1, s);
            else
                filter_axis<float>(L, axis, passes, nb, pencil_start[axis], k & 1, s);
        }
        ++k;
    }
    return cudaGetLastError();
}

template <typename R, bool CK>
static void maxwell_kernels(const Launch &L, int filtered, unsigned nb, cudaStream_t s)
{
    k_bhalf<R, CK><<<nb, 256, 0, s>>>(L, 0);
    k_efull<R><<<nb, 256, 0, s>>>(L, filtered);
    k_bhalf<R, CK><<<nb, 256, 0, s>>>(L, 1);
}

cudaError_t launch_maxwell(int fp64, int solver, const Launch &L, int filtered, cudaStream_t s)
{
    const unsigned nb = blocks_for(L.total_cells, 256);
    const bool ck = solver == PIC_SOLVER_CK;
    if (fp64)
        ck ? maxwell_kernels<double, true>(L, filtered, nb, s) : maxwell_kernels<double, false>(L, filtered, nb, s);
    else
        ck ? maxwell_kernels<float, true>(L, filtered, nb, s) : maxwell_kernels<float, false>(L, filtered, nb, s);
    return cudaGetLastError();
}

cudaError_t launch_bhalf(int fp64, int solver, const Launch &L, int damp, cudaStream_t s)
{
    const unsigned nb = blocks_for(L.total_cells, 256);
    const bool ck = solver == PIC_SOLVER_CK;
    if (fp64)
        ck ? k_bhalf<double, true><<<nb, 256, 0, s>>>(L, damp) : k_bhalf<double, false><<<nb, 256, 0, s>>>(L, damp);
    else
        ck ? k_bhalf<float, true><<<nb, 256, 0, s>>>(L, damp) : k_bhalf<float, false><<<nb, 256, 0, s>>>(L, damp);
    return cudaGetLastError();
}

cudaError_t launch_efull(int fp64, const Launch &L, int filtered, cudaStream_t s)
{
    const unsigned nb = blocks_for(L.total_cells, 256);
    if (fp64)
        k_efull<double><<<nb, 256, 0, s>>>(L, filtered);
    else
        k_efull<float><<<nb, 256, 0, s>>>(L, filtered);
    return cudaGetLastError();
}

cudaError_t launch_ghost(int fp64, const Launch &L, int axis, long long per_inst_max, cudaStream_t s)
{
    const long long n = per_inst_max * L.ninst;
    if (fp64)
        k_ghost<double><<<blocks_for(n, 256), 256, 0, s>>>(L, axis, per_inst_max);
    else
        k_ghost<float><<<blocks_for(n, 256), 256, 0, s>>>(L, axis, per_inst_max);
    return cudaGetLastError();
}

cudaError_t launch_field_energy(int fp64, const Launch &L, double *sums, cudaStream_t s)
{
    const unsigned nb = (unsigned)((L.total_cells + kEnergyCells - 1) / kEnergyCells);
    if (fp64)
        k_field_energy<double><<<nb, 256, 0, s>>>(L, sums);
    else
        k_field_energy<float><<<nb, 256, 0, s>>>(L, sums);
    return cudaGetLastError();
}

cudaError_t launch_pack(int fp64, const InstDev &I, int comp, int filtered, double *dense, long long ncell, cudaStream_t s)
{
    return launch_pack_planes(fp64, I, comp, filtered, dense, 0, (int)(ncell / ((long long)I.n[0] * I.n[1])), s);
}

cudaError_t launch_unpack(int fp64, const InstDev &I, int comp, const double *dense, long long ncell, cudaStream_t s)
{
    return launch_unpack_planes(fp64, I, comp, dense, 0, (int)(ncell / ((long long)I.n[0] * I.n[1])), 0, s);
}

cudaError_t launch_pack_planes(int fp64, const InstDev &I, int comp, int filtered, double *dense, int k0, int nk,
                               cudaStream_t s)
{
    const long long n = (long long)nk * I.n[0] * I.n[1];
    if (n <= 0) return cudaSuccess;
    if (fp64) k_pack<double><<<blocks_for(n, 256), 256, 0, s>>>(I, comp, filtered, dense, n, k0);
    else k_pack<float><<<blocks_for(n, 256), 256, 0, s>>>(I, comp, filtered, dense, n, k0);
    return cudaGetLastError();
}

cudaError_t launch_unpack_planes(int fp64, const InstDev &I, int comp, const double *dense, int k0, int nk, int add,
                                 cudaStream_t s)
{
    const long long n = (long long)nk * I.n[0] * I.n[1];
    if (n <= 0) return cudaSuccess;
    if (fp64) k_unpack<double><<<blocks_for(n, 256), 256, 0, s>>>(I, comp, dense, n, k0, add);
    else k_unpack<float><<<blocks_for(n, 256), 256, 0, s>>>(I, comp, dense, n, k0, add);
    return cudaGetLastError();
}

// max |a - b| and sum (a - b)^2 over n values (FP64); the maximum is kept as the bit
// pattern of a non-negative double, which orders like the value
__global__ void __launch_bounds__(256) k_residual(const double *a, const double *b, long long n,
                                                  unsigned long long *max_bits, double *sumsq)
{
    double m = 0.0, q = 0.0;
    for (long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x; g < n; g += (long long)gridDim.x * blockDim.x) {
        const double d = fabs(a[g] - b[g]);
        m = fmax(m, d);
        q += d * d;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
        q += __shfl_xor_sync(0xffffffffu, q, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMax(max_bits, (unsigned long long)__double_as_longlong(m));
        atomicAdd(sumsq, q);
    }
}

cudaError_t launch_residual(const double *a, const double *b, long long n, unsigned long long *max_bits, double *sumsq,
                            cudaStream_t s)
{
    const long long blocks = std::min<long long>(blocks_for(n, 256), 152LL * 8);
    k_residual<<<(unsigned)std::max<long long>(blocks, 1), 256, 0, s>>>(a, b, n, max_bits, sumsq);
    return cudaGetLastError();
}

cudaError_t launch_dive(int fp64, const InstDev &I, double *dense, long long ncell, cudaStream_t s)
{
    if (fp64) k_dive<double><<<blocks_for(ncell, 256), 256, 0, s>>>(I, dense, ncell);
    else k_dive<float><<<blocks_for(ncell, 256), 256, 0, s>>>(I, dense, ncell);
    return cudaGetLastError();
}

}  // namespace pic
