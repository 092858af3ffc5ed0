// k_fields.cu -- grid kernels of the boosted-frame PIC step on sm_103a: Yee FDTD
// half/whole updates with the absorbing layer, binomial current filter sweeps, periodic
// ghost exchange for the TMA gather boxes, and the FP64 field reductions / read-outs.
//
// All stencil kernels run one thread per interior cell of a flattened cell space over
// every instance of the launch (x fastest, so loads and stores coalesce along rows).
// Neighbours along periodic axes wrap by index; along absorbing axes they read the
// zero ghost layers.
#include "pic_internal.h"

#include <algorithm>

namespace pic {

struct CellPos {
    int ii;       // instance
    int i, j, k;  // interior cell
    long long p;  // padded linear index
};

__device__ __forceinline__ bool cell_of(const Launch &L, long long g, CellPos &c, const InstDev *&I)
{
    if (g >= L.total_cells) return false;
    c.ii = find_instance_ll(L.cell_start, L.ninst, g);
    I = L.inst + c.ii;
    const int r = (int)(g - L.cell_start[c.ii]);  // < 2^31 cells per instance
    const int rq = fast_div(r, I->div_n0);
    c.i = r - rq * I->n[0];
    c.k = fast_div(rq, I->div_n1);
    c.j = rq - c.k * I->n[1];
    c.p = (c.i + I->gh[0]) + I->sy * (c.j + I->gh[1]) + I->sz * (c.k + I->gh[2]);
    return true;
}

// Offsets to the +1 / -1 neighbour along each axis (0 on an inactive axis).
__device__ __forceinline__ void neighbour_offsets(const InstDev &I, const CellPos &c, long long up[3], long long dn[3])
{
    const long long st[3] = {1, I.sy, I.sz};
    const int idx[3] = {c.i, c.j, c.k};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (I.ndim == 2 && a == 1) {
            up[a] = dn[a] = 0;
            continue;
        }
        const bool per = I.bc[a] == 0;
        up[a] = (per && idx[a] == I.n[a] - 1) ? -(long long)(I.n[a] - 1) * st[a] : st[a];
        dn[a] = (per && idx[a] == 0) ? (long long)(I.n[a] - 1) * st[a] : -st[a];
    }
}

// Absorbing-layer factor prod_a (1 - s (d_a / L)^2), d_a = depth into the layer, read
// from the per-axis tables the host filled in FP64 (product taken x, y, z in order).
template <typename R>
__device__ __forceinline__ R damp_factor(const InstDev &I, const CellPos &c)
{
    R f = R(1);
    const int idx[3] = {c.i, c.j, c.k};
#pragma unroll
    for (int a = 0; a < 3; ++a)
        if (I.damp[a]) f *= ((const R *)I.damp[a])[idx[a]];
    return f;
}

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

// The whole Yee update of a step in one kernel (Yee solver, no antenna): B half step, E
// step, damped B half step.  It reads E^n, B^n and J once and writes E^{n+1}, B^{n+1}
// once (60 bytes per cell in FP32 instead of 120 for the three-kernel sequence).  The
// inputs are the current E / B buffer pair and the outputs go to the other one (*fpar
// flips after the kernel), so no CTA overwrites a value that a neighbouring CTA still
// reads.  A CTA takes an x-y tile of TX x TY columns (one thread each) and marches
// along z through a chunk of TZ planes, keeping in shared memory E^n of three planes on
// the tile widened by [-1, +2] in x and y, B^{n+1/2} of three planes on [-1, +1] and
// E^{n+1} of two planes on [0, +1].  For the output plane k, between two barriers:
//   B^{n+1/2}(k+2) = B^n - dt/2 curl E^n        (E^n of planes k+2, k+3)
//   E^{n+1}(k+1)  = f (E^n + dt (curl B^{n+1/2} - J))   (B^{n+1/2} of planes k, k+1)
// and after the second:
//   B^{n+1}(k)    = f (B^{n+1/2} - dt/2 curl E^{n+1})   (E^{n+1} of planes k, k+1)
// with the loads of the next plane issued one plane ahead.  Outside an absorbing box
// every field is zero; periodic axes wrap.  Each value is formed by the same expression
// as in k_bhalf / k_efull; the in-plane offsets of a thread's cells are computed once.
template <int ND>
struct MxTile;
template <>
struct MxTile<3> {
    static constexpr int X = 32, Y = 8, Z = 32;
};
template <>
struct MxTile<2> {
    static constexpr int X = 256, Y = 1, Z = 32;
};

template <typename R, int ND>
constexpr size_t maxwell_fused_smem()
{
    constexpr int HY = ND == 3 ? 1 : 0;
    constexpr int X = MxTile<ND>::X, Y = MxTile<ND>::Y;
    constexpr size_t NE = (size_t)(X + 3) * (Y + 3 * HY), NB = (size_t)(X + 2) * (Y + 2 * HY), NQ = (size_t)(X + 1) * (Y + HY);
    return sizeof(R) * 3 * (3 * NE + 3 * NB + 2 * NQ);
}

// index along one axis of the cell at q: false outside an absorbing box; wrapped on a
// periodic axis
__device__ __forceinline__ bool mx_axis(int q, int n, int bc, int &w)
{
    if (q >= 0 && q < n) {
        w = q;
        return true;
    }
    if (bc != 0) return false;
    w = ((q % n) + n) % n;
    return true;
}

template <typename R, int ND>
__global__ void __launch_bounds__(256, sizeof(R) == 4 ? 3 : 2) k_maxwell_fused(Launch L, const long long *tile_start,
                                                                              int filtered)
{
    constexpr int TX = MxTile<ND>::X, TY = MxTile<ND>::Y, TZ = MxTile<ND>::Z;
    constexpr int HY = ND == 3 ? 1 : 0;
    constexpr int EX = TX + 3, NE = EX * (TY + 3 * HY);  // E^n region: [-1, +2]
    constexpr int BX = TX + 2, NB = BX * (TY + 2 * HY);  // B^{n+1/2} region: [-1, +1]
    constexpr int QX = TX + 1, NQ = QX * (TY + HY);      // E^{n+1} region: [0, +1]
    static_assert(TX * TY == 256 && NE <= 512 && NB <= 512 && NQ <= 512, "two region cells per thread");
    extern __shared__ __align__(16) unsigned char msm[];
    R *sE = (R *)msm;     // [3 planes][3 comps][NE]
    R *sH = sE + 9 * NE;  // [3][3][NB]
    R *sQ = sH + 9 * NB;  // [2][3][NQ]
    const long long g = blockIdx.x;
    if (g >= tile_start[L.ninst]) return;
    const int ii = find_instance_ll(tile_start, L.ninst, g);
    const InstDev &I = L.inst[ii];
    const int n0 = I.n[0], n1 = I.n[1], n2 = I.n[2];
    const int ntx = (n0 + TX - 1) / TX, nty = (n1 + TY - 1) / TY;
    long long r = g - tile_start[ii];
    const int x0 = (int)(r % ntx) * TX;
    r /= ntx;
    const int y0 = (int)(r % nty) * TY;
    const int z0 = (int)(r / nty) * TZ;
    const int z1 = min(z0 + TZ, n2);
    const int par = *(volatile const int *)I.fpar;
    // the components of each field are cstride elements apart
    const long long cs = I.cstride;
    const int nsweeps = I.filter_passes > 0 ? (I.ndim == 3 ? 3 : 2) : 0;
    const R *Ein = (const R *)(par ? I.E2[0] : I.E[0]), *Bin = (const R *)(par ? I.B2[0] : I.B[0]);
    R *Eout = (R *)(par ? I.E[0] : I.E2[0]), *Bout = (R *)(par ? I.B[0] : I.B2[0]);
    const R *Jin = (const R *)((filtered && (nsweeps & 1)) ? I.Jt[0] : I.J[0]);
    const StepCoef<R> &K = coef<R>(I);
    const R h = K.half_dt, dt = K.dt;
    const R ix = K.inv_dx[0], iy = K.inv_dx[1], iz = K.inv_dx[2];
    const R *dampx = (const R *)I.damp[0], *dampy = (const R *)I.damp[1], *dampz = (const R *)I.damp[2];
    const int tid = threadIdx.x;
    // in-plane padded offset of the cell at (x0 + dx, y0 + dy), false outside the box;
    // fxy: its x and y damping factors multiplied in the order of damp_factor
    auto inplane = [&](int dx_, int dy_, int &off, R &fxy) -> bool {
        int x, y = 0;
        bool ok = mx_axis(x0 + dx_, n0, I.bc[0], x);
        if (ND == 3) ok = ok && mx_axis(y0 + dy_, n1, I.bc[1], y);
        off = (x + I.gh[0]) + I.sy * (y + I.gh[1]);  // < 2^31: one plane
        fxy = R(1);
        if (ok && dampx) fxy *= dampx[x];
        if (ok && ND == 3 && dampy) fxy *= dampy[y];
        return ok;
    };
    int eoff[2], boff[2], qoff[2], toff;
    bool eok[2], bok[2], qok[2], tok;
    R qf[2], tf, unused;
#pragma unroll
    for (int j = 0; j < 2; ++j) {
        const int e = tid + 256 * j, b = tid + 256 * j, q = tid + 256 * j;
        eok[j] = e < NE && inplane(e % EX - 1, e / EX - HY, eoff[j], unused);
        bok[j] = b < NB && inplane(b % BX - 1, b / BX - HY, boff[j], unused);
        qok[j] = q < NQ && inplane(q % QX, q / QX, qoff[j], qf[j]);
    }
    const int tx = tid % TX, ty = tid / TX;
    tok = x0 + tx < n0 && y0 + ty < n1 && inplane(tx, ty, toff, tf);
    // z: padded plane offset of plane k, false outside an absorbing box
    auto zplane = [&](int k, long long &zo, R &fz) -> bool {
        int z;
        const bool ok = mx_axis(k, n2, I.bc[2], z);
        zo = I.sz * (long long)(z + I.gh[2]);
        fz = (ok && dampz) ? dampz[z] : R(1);
        return ok;
    };
    auto slot3 = [](int k) { return ((k % 3) + 3) % 3; };
    // global loads of one plane for this thread's cells of a region
    auto load3 = [&](const R *F, const int *off, const bool *ok, int k, R (&v)[2][3]) {
        long long zo;
        R fz;
        const bool zk = zplane(k, zo, fz);
#pragma unroll
        for (int j = 0; j < 2; ++j)
#pragma unroll
            for (int c = 0; c < 3; ++c) v[j][c] = (zk && ok[j]) ? F[c * cs + off[j] + zo] : R(0);
    };
    auto storeE = [&](int k, const R (&v)[2][3]) {
        R *d = sE + slot3(k) * 3 * NE;
#pragma unroll
        for (int j = 0; j < 2; ++j)
            if (tid + 256 * j < NE)
#pragma unroll
                for (int c = 0; c < 3; ++c) d[c * NE + tid + 256 * j] = v[j][c];
    };
    // B^{n+1/2}(k) from E^n of planes k, k+1 and B^n(k) (bv)
    auto makeH = [&](int k, const R (&bv)[2][3]) {
        long long zo;
        R fz;
        const bool zk = zplane(k, zo, fz);
        const R *E0 = sE + slot3(k) * 3 * NE, *E1 = sE + slot3(k + 1) * 3 * NE;
        R *H = sH + slot3(k) * 3 * NB;
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const int b = tid + 256 * j;
            if (b >= NB) continue;
            R hb[3] = {R(0), R(0), R(0)};
            if (zk && bok[j]) {
                const int e = b % BX + EX * (b / BX);
                const R ex = E0[e], ey = E0[NE + e], ez = E0[2 * NE + e];
                R dEz_dy = R(0), dEx_dy = R(0);
                const R dEy_dz = (E1[NE + e] - ey) * iz;
                const R dEx_dz = (E1[e] - ex) * iz;
                const R dEz_dx = (E0[2 * NE + e + 1] - ez) * ix;
                const R dEy_dx = (E0[NE + e + 1] - ey) * ix;
                if (ND == 3) {
                    dEz_dy = (E0[2 * NE + e + EX] - ez) * iy;
                    dEx_dy = (E0[e + EX] - ex) * iy;
                }
                hb[0] = bv[j][0] - h * (dEz_dy - dEy_dz);
                hb[1] = bv[j][1] - h * (dEx_dz - dEz_dx);
                hb[2] = bv[j][2] - h * (dEy_dx - dEx_dy);
            }
#pragma unroll
            for (int c = 0; c < 3; ++c) H[c * NB + b] = hb[c];
        }
    };
    // E^{n+1}(k) from B^{n+1/2} of planes k-1, k, E^n(k) and J(k) (jv)
    auto makeQ = [&](int k, const R (&jv)[2][3]) {
        long long zo;
        R fz;
        const bool zk = zplane(k, zo, fz);
        const R *H1 = sH + slot3(k) * 3 * NB, *H0 = sH + slot3(k - 1) * 3 * NB;
        const R *E0 = sE + slot3(k) * 3 * NE;
        R *Q = sQ + (k & 1) * 3 * NQ;
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const int q = tid + 256 * j;
            if (q >= NQ) continue;
            R en[3] = {R(0), R(0), R(0)};
            if (zk && qok[j]) {
                const int qx = q % QX, qy = q / QX;
                const int b = (qx + 1) + BX * (qy + HY), e = (qx + 1) + EX * (qy + HY);
                const R bx = H1[b], by = H1[NB + b], bz = H1[2 * NB + b];
                R dBz_dy = R(0), dBx_dy = R(0);
                const R dBy_dz = (by - H0[NB + b]) * iz, dBx_dz = (bx - H0[b]) * iz;
                const R dBz_dx = (bz - H1[2 * NB + b - 1]) * ix, dBy_dx = (by - H1[NB + b - 1]) * ix;
                if (ND == 3) {
                    dBz_dy = (bz - H1[2 * NB + b - BX]) * iy;
                    dBx_dy = (bx - H1[b - BX]) * iy;
                }
                const R f = dampz ? qf[j] * fz : qf[j];
                en[0] = f * (E0[e] + dt * ((dBz_dy - dBy_dz) - jv[j][0]));
                en[1] = f * (E0[NE + e] + dt * ((dBx_dz - dBz_dx) - jv[j][1]));
                en[2] = f * (E0[2 * NE + e] + dt * ((dBy_dx - dBx_dy) - jv[j][2]));
            }
#pragma unroll
            for (int c = 0; c < 3; ++c) Q[c * NQ + q] = en[c];
        }
    };
    // B^{n+1}(k) on the tile from B^{n+1/2}(k), E^{n+1} of planes k, k+1; stores both
    auto emit = [&](int k) {
        if (!tok) return;
        long long zo;
        R fz;
        zplane(k, zo, fz);
        const R *Q0 = sQ + (k & 1) * 3 * NQ, *Q1 = sQ + ((k + 1) & 1) * 3 * NQ;
        const R *H = sH + slot3(k) * 3 * NB;
        const int q = tx + QX * ty, b = (tx + 1) + BX * (ty + HY);
        const R ex = Q0[q], ey = Q0[NQ + q], ez = Q0[2 * NQ + q];
        R dEz_dy = R(0), dEx_dy = R(0);
        const R dEy_dz = (Q1[NQ + q] - ey) * iz;
        const R dEx_dz = (Q1[q] - ex) * iz;
        const R dEz_dx = (Q0[2 * NQ + q + 1] - ez) * ix;
        const R dEy_dx = (Q0[NQ + q + 1] - ey) * ix;
        if (ND == 3) {
            dEz_dy = (Q0[2 * NQ + q + QX] - ez) * iy;
            dEx_dy = (Q0[q + QX] - ex) * iy;
        }
        R bx = H[b] - h * (dEz_dy - dEy_dz);
        R by = H[NB + b] - h * (dEx_dz - dEz_dx);
        R bz = H[2 * NB + b] - h * (dEy_dx - dEx_dy);
        const R f = dampz ? tf * fz : tf;
        bx *= f;
        by *= f;
        bz *= f;
        const long long p = toff + zo;
        Bout[p] = bx;
        Bout[cs + p] = by;
        Bout[2 * cs + p] = bz;
        Eout[p] = ex;
        Eout[cs + p] = ey;
        Eout[2 * cs + p] = ez;
    };

    R vE[2][3], cB[2][3], cJ[2][3], nB[2][3], nJ[2][3];
    // prologue: E^n of planes z0-1 .. z0+2, B^{n+1/2} of z0-1 .. z0+1, E^{n+1} of z0
    load3(Ein, eoff, eok, z0 - 1, vE);
    storeE(z0 - 1, vE);
    load3(Ein, eoff, eok, z0, vE);
    storeE(z0, vE);
    load3(Ein, eoff, eok, z0 + 1, vE);
    storeE(z0 + 1, vE);
    load3(Bin, boff, bok, z0 - 1, cB);
    load3(Bin, boff, bok, z0, nB);
    load3(Jin, qoff, qok, z0, cJ);
    __syncthreads();
    makeH(z0 - 1, cB);
    makeH(z0, nB);
    __syncthreads();
    makeQ(z0, cJ);
    __syncthreads();
    load3(Ein, eoff, eok, z0 + 2, vE);
    storeE(z0 + 2, vE);  // in the slot of plane z0 - 1
    load3(Bin, boff, bok, z0 + 1, cB);
    __syncthreads();
    makeH(z0 + 1, cB);   // the third slot
    // one plane ahead: E^n(z0+3), B^n(z0+2), J(z0+1)
    load3(Ein, eoff, eok, z0 + 3, vE);
    load3(Bin, boff, bok, z0 + 2, cB);
    load3(Jin, qoff, qok, z0 + 1, cJ);
#pragma unroll 1
    for (int k = z0; k < z1; ++k) {
        storeE(k + 3, vE);  // in the slot of plane k
        // the next plane's loads, in flight through this plane's arithmetic
        load3(Ein, eoff, eok, k + 4, vE);
        load3(Bin, boff, bok, k + 3, nB);
        load3(Jin, qoff, qok, k + 2, nJ);
        __syncthreads();
        makeH(k + 2, cB);  // in the slot of plane k - 1
        makeQ(k + 1, cJ);  // in the slot of plane k - 1
        __syncthreads();
        emit(k);
#pragma unroll
        for (int j = 0; j < 2; ++j)
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                cB[j][c] = nB[j][c];
                cJ[j][c] = nJ[j][c];
            }
    }
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

// Binomial filter along one axis, all passes at once.  The x, y and z operators (each
// with its boundary: periodic wrap, or zero outside an absorbing box after every pass)
// act on different axes and commute, so `passes` rounds of (x, y, z) equal x^passes,
// y^passes, z^passes.  One CTA takes a pencil of kPencil cells along the axis (times 32
// x-columns for the y and z axes), loads it with `passes` halo cells per side into shared
// memory, applies the passes there (J <- J(i-1)/4 + J(i)/2 + J(i+1)/4, re-zeroing cells
// outside an absorbing box after each pass) and writes the pencil back: one read and one
// write per cell and axis instead of one per pass.  Reads src, writes dst (J / Jt).
constexpr int kPencil = 64;
constexpr int kMaxPasses = 8;

__device__ __forceinline__ bool filter_active_axis(const InstDev &I, int axis)
{
    return I.filter_passes > 0 && !(I.ndim == 2 && axis == 1);
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

// The same filter with the number of passes P known at compile time (P <= 4, every
// instance of the launch alike), in registers, without shared memory or barriers, on the
// pencils of k_filter_axis.  Binomial weight C(2P, m) / 4^P of tap m (exact in FP32).
__host__ __device__ constexpr double binomial_weight(int P, int m)
{
    double c = 1.0;
    for (int t = 1; t <= m; ++t) c = c * (2 * P - t + 1) / t;
    return c / (double)(1 << (2 * P));
}

// y and z axes: lane = x column (coalesced), each warp takes kPencil / 8 consecutive
// cells along the axis and loads them with P halo cells per side into registers.  Away
// from the ends the output is the (2P+1)-tap convolution; a window that wraps (periodic)
// is loaded wrapped and convolved too; one that reaches past an absorbing face runs the
// P passes, re-zeroing the outside after each.
template <typename R, int P>
__global__ void __launch_bounds__(256) k_filter_col(Launch L, int axis, const long long *pencil_start, int src_is_jt)
{
    constexpr int S = kPencil / 8;
    constexpr int W = S + 2 * P;
    const long long g = blockIdx.x;
    if (g >= pencil_start[L.ninst]) return;
    const int ii = find_instance_ll(pencil_start, L.ninst, g);
    const InstDev &I = L.inst[ii];
    if (!filter_active_axis(I, axis)) return;
    const int n = I.n[axis];
    const bool per = I.bc[axis] == 0;
    const int nseg = (n + kPencil - 1) / kPencil;
    long long r = g - pencil_start[ii];
    const int qs = (int)(r % nseg) * kPencil + (threadIdx.x >> 5) * S;  // this thread's first cell
    r /= nseg;
    const int ncol = (I.n[0] + 31) / 32;
    const int x = (int)(r % ncol) * 32 + (threadIdx.x & 31);
    const int other = (int)(r / ncol);  // z for the y axis, y for the z axis
    if (x >= I.n[0] || qs >= n) return;
    const long long sa = axis == 1 ? I.sy : I.sz;
    const long long lo = axis == 1 ? (x + I.gh[0]) + I.sy * I.gh[1] + I.sz * (long long)(other + I.gh[2])
                                   : (x + I.gh[0]) + I.sy * (long long)(other + I.gh[1]) + I.sz * I.gh[2];
    const bool inside = qs - P >= 0 && qs + S + P <= n;
    void *const *src = src_is_jt ? I.Jt : I.J;
    void *const *dst = src_is_jt ? I.J : I.Jt;
    // all three windows first (the source and destination arrays differ)
    R win[3][W];
#pragma unroll
    for (int comp = 0; comp < 3; ++comp) {
        const R *__restrict__ a = (const R *)src[comp];
        if (inside) {
#pragma unroll
            for (int m = 0; m < W; ++m) win[comp][m] = a[lo + (long long)(qs - P + m) * sa];
        } else {
#pragma unroll
            for (int m = 0; m < W; ++m) {
                int q = qs - P + m;
                bool ok = true;
                if (q < 0 || q >= n) {
                    if (per) q = ((q % n) + n) % n;
                    else ok = false;
                }
                win[comp][m] = ok ? a[lo + (long long)q * sa] : R(0);
            }
        }
    }
#pragma unroll
    for (int comp = 0; comp < 3; ++comp) {
        R w[W];
#pragma unroll
        for (int m = 0; m < W; ++m) w[m] = win[comp][m];
        R out[S];
        if (inside || per) {
#pragma unroll
            for (int t = 0; t < S; ++t) {
                R v = R(0);
#pragma unroll
                for (int m = 0; m <= 2 * P; ++m) v += R(binomial_weight(P, m)) * w[t + m];
                out[t] = v;
            }
        } else {
#pragma unroll
            for (int pass = 1; pass <= P; ++pass) {
                R nw[W];
#pragma unroll
                for (int m = 0; m < W; ++m) nw[m] = w[m];
#pragma unroll
                for (int m = pass; m < W - pass; ++m) {
                    const int q = qs - P + m;
                    nw[m] = (q < 0 || q >= n) ? R(0) : R(0.25) * w[m - 1] + R(0.5) * w[m] + R(0.25) * w[m + 1];
                }
#pragma unroll
                for (int m = 0; m < W; ++m) w[m] = nw[m];
            }
#pragma unroll
            for (int t = 0; t < S; ++t) out[t] = w[t + P];
        }
        R *__restrict__ b = (R *)dst[comp];
#pragma unroll
        for (int t = 0; t < S; ++t)
            if (qs + t < n) b[lo + (long long)(qs + t) * sa] = out[t];
    }
}

// x axis: warp w takes rows w, w + 8, w + 16, w + 24 of the pencil; per row it loads the
// kPencil + 2P window of all three components with coalesced loads into its own slice of
// shared memory (warp-synchronous, no block barrier) and each lane forms two outputs
// from it.  Cells within P of an end convolve the wrapped window (periodic) or run the
// passes (absorbing).
template <typename R, int P>
__global__ void __launch_bounds__(256) k_filter_row(Launch L, const long long *pencil_start, int src_is_jt)
{
    constexpr int W = kPencil + 2 * P;
    __shared__ R sw[8][3][W];
    const long long g = blockIdx.x;
    if (g >= pencil_start[L.ninst]) return;
    const int ii = find_instance_ll(pencil_start, L.ninst, g);
    const InstDev &I = L.inst[ii];
    if (!filter_active_axis(I, 0)) return;
    const int n = I.n[0];
    const bool per = I.bc[0] == 0;
    const int nseg = (n + kPencil - 1) / kPencil;
    long long r = g - pencil_start[ii];
    const int q0 = (int)(r % nseg) * kPencil;
    r /= nseg;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const bool inside = q0 - P >= 0 && q0 + kPencil + P <= n;
    void *const *src = src_is_jt ? I.Jt : I.J;
    void *const *dst = src_is_jt ? I.J : I.Jt;
    R(*win)[W] = sw[warp];
#pragma unroll 1
    for (int rr = warp; rr < 32; rr += 8) {
        const long long row = r * 32 + rr;
        if (row >= (long long)I.n[1] * I.n[2]) break;
        const int y = (int)(row % I.n[1]), z = (int)(row / I.n[1]);
        const long long lo = I.gh[0] + I.sy * (long long)(y + I.gh[1]) + I.sz * (long long)(z + I.gh[2]);
#pragma unroll
        for (int i0 = 0; i0 < W; i0 += 32) {
            const int i = i0 + lane;
            if (i < W) {
                int q = q0 - P + i;
                bool ok = true;
                if (!inside && (q < 0 || q >= n)) {
                    if (per) q = ((q % n) + n) % n;
                    else ok = false;
                }
#pragma unroll
                for (int comp = 0; comp < 3; ++comp) win[comp][i] = ok ? ((const R *)src[comp])[lo + q] : R(0);
            }
        }
        __syncwarp();
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int t = lane + 32 * h;  // output q0 + t, window cells t .. t + 2P
            const int q = q0 + t;
            if (q >= n) continue;
            const bool conv = per || (q - P >= 0 && q + P < n);
#pragma unroll
            for (int comp = 0; comp < 3; ++comp) {
                R w[2 * P + 1];
#pragma unroll
                for (int m = 0; m <= 2 * P; ++m) w[m] = win[comp][t + m];
                R v = R(0);
                if (conv) {
#pragma unroll
                    for (int m = 0; m <= 2 * P; ++m) v += R(binomial_weight(P, m)) * w[m];
                } else {
#pragma unroll
                    for (int pass = 1; pass <= P; ++pass) {
                        R nw[2 * P + 1];
#pragma unroll
                        for (int m = 0; m <= 2 * P; ++m) nw[m] = w[m];
#pragma unroll
                        for (int m = pass; m <= 2 * P - pass; ++m) {
                            const int qq = q - P + m;
                            nw[m] = (qq < 0 || qq >= n) ? R(0) : R(0.25) * w[m - 1] + R(0.5) * w[m] + R(0.25) * w[m + 1];
                        }
#pragma unroll
                        for (int m = 0; m <= 2 * P; ++m) w[m] = nw[m];
                    }
                    v = w[P];
                }
                ((R *)dst[comp])[lo + q] = v;
            }
        }
        __syncwarp();  // the window is reloaded for the next row
    }
}

// Periodic ghost exchange of the six E/B components along one axis (after the whole
// step); ghosts of earlier axes are included so corners come out right.
template <typename R>
__global__ void __launch_bounds__(256) k_ghost(Launch L, int axis, long long per_inst_max)
{
    const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int ii = (int)(g / per_inst_max);
    if (ii >= L.ninst) return;
    const InstDev &I = L.inst[ii];
    if (I.bc[axis] != 0 || (I.ndim == 2 && axis == 1)) return;
    // ghost slab: 2*gh layers along `axis` x padded extents of the other two axes
    const int gh = I.gh[axis];
    long long r = g - (long long)ii * per_inst_max;
    const int o1 = axis == 0 ? 1 : 0, o2 = axis == 2 ? 1 : 2;
    const long long e1 = I.P[o1], e2 = I.P[o2];
    const long long slab = 2LL * gh * e1 * e2;
    if (r >= 6 * slab) return;
    const int comp = (int)(r / slab);
    r -= comp * slab;
    const int layer = (int)(r % (2 * gh));
    r /= 2 * gh;
    const long long a1 = r % e1, a2 = r / e1;
    const int n = I.n[axis];
    // destination padded coordinate along axis and its periodic source
    const int dpos = layer < gh ? layer : gh + n + (layer - gh);
    const int spos = layer < gh ? dpos + n : dpos - n;
    long long st[3] = {1, I.sy, I.sz};
    const long long base = a1 * st[o1] + a2 * st[o2];
    R *f = (R *)eb_field(I, comp);
    f[base + dpos * st[axis]] = f[base + spos * st[axis]];
}

// FP64 field energy sums (1/2) sum (E^2 + B^2) dV per instance.
template <typename R>
__global__ void __launch_bounds__(256) k_field_energy(Launch L, double *sums)
{
    __shared__ double s_e[8];
    __shared__ int s_ii[8];
    const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    CellPos c;
    const InstDev *Ip;
    double e = 0.0;
    int ii = -1;
    if (cell_of(L, g, c, Ip)) {
        const InstDev &I = *Ip;
        ii = c.ii;
        R s2 = R(0);  // the cell's E^2 + B^2 in the storage precision, then FP64
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const R x = ((const R *)eb_field(I, a))[c.p], y = ((const R *)eb_field(I, 3 + a))[c.p];
            s2 += x * x + y * y;
        }
        e = (double)s2 * (0.5 * I.dx[0] * I.dx[1] * I.dx[2]);
    }
    // instances are contiguous in g: reduce per warp when the whole warp shares one, then
    // per block (one atomic per instance present in the block)
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ii0 = __shfl_sync(0xffffffffu, ii, 0);
    const bool same = __all_sync(0xffffffffu, ii == ii0 || ii < 0);
    if (same) {
        for (int o = 16; o > 0; o >>= 1) e += __shfl_down_sync(0xffffffffu, e, o);
        if (lane == 0) {
            s_e[warp] = e;
            s_ii[warp] = ii0;
        }
    } else {
        if (ii >= 0) atomicAdd(sums + 2 * L.ninst + ii, e);
        if (lane == 0) s_ii[warp] = -1;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int cur = -1;
        double acc = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            if (s_ii[w] < 0) continue;
            if (s_ii[w] != cur) {
                if (cur >= 0) atomicAdd(sums + 2 * L.ninst + cur, acc);
                cur = s_ii[w];
                acc = 0.0;
            }
            acc += s_e[w];
        }
        if (cur >= 0) atomicAdd(sums + 2 * L.ninst + cur, acc);
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
    if (fp64)
        k_field_energy<double><<<blocks_for(L.total_cells, 256), 256, 0, s>>>(L, sums);
    else
        k_field_energy<float><<<blocks_for(L.total_cells, 256), 256, 0, s>>>(L, sums);
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
