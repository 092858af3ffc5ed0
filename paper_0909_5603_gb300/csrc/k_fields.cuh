// k_fields.cuh -- device functions of the grid phases (cell addressing, the absorbing
// layer, the fused Yee update, the fixed-pass filter sweeps, the periodic ghost copy),
// shared by the per-phase kernels of k_fields.cu and the persistent batched step.
#pragma once
#include "pic_internal.h"

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
__device__ __forceinline__ void maxwell_fused_block(const Launch &L, const long long *tile_start, int filtered,
                                                    const long long g)
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
__device__ __forceinline__ void filter_col_block(const Launch &L, int axis, const long long *pencil_start, int src_is_jt,
                                                 const long long g)
{
    constexpr int S = kPencil / 8;
    constexpr int W = S + 2 * P;
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

// x axis: warp w takes rows w, w + 8, w + 16, w + 24 of the pencil.  It first loads the
// kPencil + 2P window of all three components of all four rows into registers
// (coalesced, all in flight together), then per row stores the window into its own
// slice of shared memory (warp-synchronous, no block barrier) and each lane forms two
// outputs from it.  Cells within P of an end convolve the wrapped window (periodic) or
// run the passes (absorbing).
// sw: shared memory for the windows, 8 x 3 x (kPencil + 2P) values
template <typename R, int P>
__device__ __forceinline__ void filter_row_block(const Launch &L, const long long *pencil_start, int src_is_jt,
                                                 const long long g, R *sw)
{
    constexpr int W = kPencil + 2 * P;
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
    R(*win)[W] = reinterpret_cast<R(*)[W]>(sw + warp * 3 * W);
    constexpr int NR = 4, NC = (W + 31) / 32;  // rows per warp, window chunks of 32
    const long long nrows = (long long)I.n[1] * I.n[2];
    long long lo[NR];
    R pre[NR][3][NC];
    // this lane's window cells (the same in every row)
    int qi[NC];
    bool qok[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        const int i = 32 * c + lane;
        int q = q0 - P + i;
        bool ok = i < W;
        if (ok && !inside && (q < 0 || q >= n)) {
            if (per) q = ((q % n) + n) % n;
            else ok = false;
        }
        qi[c] = q;
        qok[c] = ok;
    }
#pragma unroll
    for (int j = 0; j < NR; ++j) {
        const long long row = r * 32 + warp + 8 * j;
        const bool rok = row < nrows;
        const int y = rok ? (int)(row % I.n[1]) : 0, z = rok ? (int)(row / I.n[1]) : 0;
        lo[j] = I.gh[0] + I.sy * (long long)(y + I.gh[1]) + I.sz * (long long)(z + I.gh[2]);
#pragma unroll
        for (int comp = 0; comp < 3; ++comp)
#pragma unroll
            for (int c = 0; c < NC; ++c)
                pre[j][comp][c] = (rok && qok[c]) ? ((const R *)src[comp])[lo[j] + qi[c]] : R(0);
    }
#pragma unroll
    for (int j = 0; j < NR; ++j) {
        if (r * 32 + warp + 8 * j >= nrows) break;
#pragma unroll
        for (int comp = 0; comp < 3; ++comp)
#pragma unroll
            for (int c = 0; c < NC; ++c)
                if (32 * c + lane < W) win[comp][32 * c + lane] = pre[j][comp][c];
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
                ((R *)dst[comp])[lo[j] + q] = v;
            }
        }
        __syncwarp();  // the window is rewritten for the next row
    }
}

// Periodic ghost exchange of the six E/B components along one axis (after the whole
// step); ghosts of earlier axes are included so corners come out right.
// Element r of the ghost copy of instance I along `axis` (0 <= r < ghost_elems(I, axis)).
template <typename R>
__device__ __forceinline__ void ghost_elem(const InstDev &I, int axis, long long r)
{
    // ghost slab: 2*gh layers along `axis` x padded extents of the other two axes
    const int gh = I.gh[axis];
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

// Elements of the ghost copy of instance I along `axis` (0 when the axis is not periodic).
__device__ __forceinline__ long long ghost_elems(const InstDev &I, int axis)
{
    if (I.bc[axis] != 0 || (I.ndim == 2 && axis == 1)) return 0;
    const int o1 = axis == 0 ? 1 : 0, o2 = axis == 2 ? 1 : 2;
    return 6LL * 2 * I.gh[axis] * I.P[o1] * I.P[o2];
}

}  // namespace pic
