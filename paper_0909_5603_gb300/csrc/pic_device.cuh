// pic_device.cuh -- per-particle device arithmetic of the boosted-frame PIC step:
// B-spline shape factors, Vay and Boris pushers, position update, and the TMA /
// mbarrier primitives of the field-staging stage (inline PTX, sm_103a).
#pragma once

#include "pic_internal.h"

namespace pic {

// ------------------------------------------------------------------------------------
// Shape factors of order 1 (linear) and 2 (quadratic B-spline) for a particle in cell l
// with in-cell offset o.  "Nodal" quantities sit at integer positions, "staggered" ones
// at i + 1/2 (Yee grid).  Each call returns the first node (relative to the tile) and
// the ORD + 1 weights.
// ------------------------------------------------------------------------------------
template <int ORD, typename R>
__device__ __forceinline__ int shape_nodal(int l, R o, R w[ORD + 1])
{
    if (ORD == 1) {
        w[0] = R(1) - o;
        w[1] = o;
        return l;
    } else {
        const bool up = o >= R(0.5);
        const R f = up ? o - R(1) : o;  // distance from the nearest node, in [-1/2, 1/2)
        const R a = R(0.5) - f, b = R(0.5) + f;
        w[0] = R(0.5) * a * a;
        w[1] = R(0.75) - f * f;
        w[2] = R(0.5) * b * b;
        return l + (up ? 1 : 0) - 1;
    }
}

template <int ORD, typename R>
__device__ __forceinline__ int shape_stag(int l, R o, R w[ORD + 1])
{
    if (ORD == 1) {
        const bool up = o >= R(0.5);
        const R f = up ? o - R(0.5) : o + R(0.5);
        w[0] = R(1) - f;
        w[1] = f;
        return up ? l : l - 1;
    } else {
        const R f = o - R(0.5);
        const R a = R(0.5) - f, b = R(0.5) + f;
        w[0] = R(0.5) * a * a;
        w[1] = R(0.75) - f * f;
        w[2] = R(0.5) * b * b;
        return l - 1;
    }
}

// Old shape S0 and its change DS = S1 - S0 on one common window starting at node `ws`
// (tile-relative), for the Esirkepov deposit; `nw` is the number of window nodes that can
// be non-zero: ORD + 1 when the particle keeps its nodes, ORD + 2 when it moves to the
// next set (moves stay below one cell per step).  In the first case DS is formed from
// d = f1 - f0, the exact difference of the two offsets from the first node, as products
// with d -- e.g. for order 2 the centre weight gives (3/4 - f1^2) - (3/4 - f0^2) =
// -d (f0 + f1) -- instead of subtracting two O(1) weights, which in FP32 would lose the
// small displacement to cancellation.  Entries at and beyond nw are zero.
//
// kDisp: take d as `disp`, the displacement the push computed, instead of f1 - f0.  The
// two differ by the rounding of the stored new offset (at most half an ulp of it): with
// FP32 offsets that rounding is ~3e-8 of a cell, i.e. a relative current error of
// 3e-8 / d, 6e-6 for a thermal particle moving 0.005 cells per step.  Taking the computed
// displacement keeps J at FP32 precision relative to the motion; the rounding then
// appears only as a charge-conservation residual of at most half an ulp times the shape
// slope per particle and step.  With kDisp a particle that changes its nodes gets DS from
// the slopes over the two parts of its move (below), not from a difference of weights.
template <int ORD, bool kDisp, typename R>
__device__ __forceinline__ int shape_window(int l0, R o0, int l1, R o1, R disp, R S0[ORD + 2], R DS[ORD + 2],
                                            int &nw)
{
    R w0[ORD + 1], w1[ORD + 1];
    const int b0 = shape_nodal<ORD>(l0, o0, w0);
    const int b1 = shape_nodal<ORD>(l1, o1, w1);
    if (b0 == b1) {
        const R f0 = o0 - R(b0 - l0 + (ORD == 2 ? 1 : 0));
        const R f1 = o1 - R(b1 - l1 + (ORD == 2 ? 1 : 0));
        const R d = kDisp ? disp : f1 - f0;
#pragma unroll
        for (int i = 0; i <= ORD; ++i) S0[i] = w0[i];
        S0[ORD + 1] = R(0);
        if (ORD == 1) {
            DS[0] = -d;
            DS[1] = d;
        } else {
            const R s = kDisp ? f0 + f0 + d : f0 + f1;
            DS[0] = R(-0.5) * d * (R(1) - s);
            DS[1] = -d * s;
            // = d (1 + s) / 2, taken as -(DS[0] + DS[1]) so the running sum over the
            // window ends at exactly zero
            DS[2] = -(DS[0] + DS[1]);
        }
        DS[ORD + 1] = R(0);
        nw = ORD + 1;
        return b0;
    }
    const int ws = b0 < b1 ? b0 : b1;
    const int s0 = b0 - ws, s1 = b1 - ws;  // 0 or 1
#pragma unroll
    for (int i = 0; i < ORD + 2; ++i) {
        const R a0 = (i < ORD + 1) ? w0[i < ORD + 1 ? i : 0] : R(0);
        const R a1 = (i >= 1) ? w0[i >= 1 ? i - 1 : 0] : R(0);
        const R c0 = (i < ORD + 1) ? w1[i < ORD + 1 ? i : 0] : R(0);
        const R c1 = (i >= 1) ? w1[i >= 1 ? i - 1 : 0] : R(0);
        S0[i] = s0 == 0 ? a0 : a1;
        if (!kDisp) DS[i] = (s1 == 0 ? c0 : c1) - S0[i];
    }
    if (kDisp) {
        // The move crosses one knot of the shape (order 2: the half-integer between the two
        // nearest nodes, 3/2 above the window start; order 1: the cell face, 1 above it).
        // Each weight is one polynomial piece on either side of the knot, so its change is
        // the integral of its slope over the two sub-moves, e0 up to the knot and e1 beyond
        // it: DS_i = e0 S'_i(mid0) + e1 S'_i(mid1), the slopes taken at the sub-moves'
        // midpoints (exact: the slope is linear, order 2, or constant, order 1, on a
        // piece).  e0 = knot - x0 is one rounding of a small constant minus the offset and
        // e1 = d - e0, so DS carries an error relative to the displacement rather than the
        // weights' rounding (~1e-7 absolute), which a small move would not resolve.
        const R xk = ORD == 2 ? R(1.5) : R(1);
        const R e0 = (xk - R(l0 - ws)) - o0;
        const R e1 = disp - e0;
        R sum = R(0);
#pragma unroll
        for (int i = 0; i < ORD + 2; ++i) {
            const R dk = xk - R(i);  // the knot relative to node i
            const R m0 = dk - R(0.5) * e0, m1 = dk + R(0.5) * e1;
            R g0, g1;
            if (ORD == 2) {
                const R a0 = fabs(m0), a1 = fabs(m1);
                // S = 3/4 - x^2 (|x| < 1/2), (3/2 - |x|)^2 / 2 (|x| < 3/2): S' = -2x, -sign(x)(3/2 - |x|)
                g0 = a0 < R(0.5) ? R(-2) * m0 : (a0 < R(1.5) ? copysign(R(1.5) - a0, -m0) : R(0));
                g1 = a1 < R(0.5) ? R(-2) * m1 : (a1 < R(1.5) ? copysign(R(1.5) - a1, -m1) : R(0));
            } else {
                // S = 1 - |x| (|x| < 1): S' = -sign(x)
                g0 = fabs(m0) < R(1) ? copysign(R(1), -m0) : R(0);
                g1 = fabs(m1) < R(1) ? copysign(R(1), -m1) : R(0);
            }
            if (i < ORD + 1) {
                DS[i] = e0 * g0 + e1 * g1;
                sum += DS[i];
            } else {
                DS[i] = -sum;  // the running sum over the window ends at exactly zero
            }
        }
    }
    nw = ORD + 2;
    return ws;
}

// ------------------------------------------------------------------------------------
// Shared-memory J accumulation policies for the deposit.
//
// ChunkAcc (FP32 mode): one 32-bit integer shared atomic per contribution, block floating
// point per chunk of 256 particles and per component.  The running sum of the Esirkepov
// weight changes along an axis is the charge flux through a cell face, at most |d| for a
// displacement d (its rate is the next lower-order spline, whose peak is 1), and the
// transverse factor is the time average of a product of the moving weights, at most
// S_max^2 (S_max in 2D3V; S_max, the shape's peak, is 1 for order 1 and 3/4 for order 2):
// any contribution to component a is at most S_max^2 |f_a d_a| (S_max |f_a d_a| in the
// 2D3V plane, S_max^2 |f_y| for its out-of-plane current, f_y carrying v_y; |d_a| is
// widened by 2^-18 for the rounding of the node-crossing weight changes).  Each chunk takes, per component, the
// scale that maps the chunk's largest such bound to 0.999 2^22: every contribution then
// stays within 2^22, the range in which the rounding below is exact, and 256
// contributions to one entry stay below 2^30, so the integer sums cannot overflow.  Each
// contribution is rounded to the nearest integer (one FMA against 1.5 * 2^23, whose float
// spacing is 1 up to 2^24, and an integer subtraction of that constant's bits) and added
// to the
// chunk accumulator A; after the chunk every thread folds the entries it owns into an
// FP32 tile, T += A / scale, A = 0.  The resolution is 2^-22 of the chunk's largest
// contribution bound per component, comparable with FP32 accumulation of a cell holding
// a few contributions, and the chunk sums do not depend on the order of the additions.
// DoubleAcc (FP64 mode): FP64 shared atomics, zero contributions skipped.
// ------------------------------------------------------------------------------------
struct ChunkAcc {
    static constexpr bool kSkipZero = false;  // 3D: zero adds cost less than the branch
    int *A;
    // adds round(a * b)
    __device__ __forceinline__ void add_prod(int idx, float a, float b) const
    {
        const float y = __fmaf_rn(a, b, 12582912.0f);  // 1.5 * 2^23 + a b, rounded to an integer
        atomicAdd(A + idx, __float_as_int(y) - 0x4B400000);
    }
    __device__ __forceinline__ void add(int idx, float x) const
    {
        const float y = __fadd_rn(x, 12582912.0f);
        atomicAdd(A + idx, __float_as_int(y) - 0x4B400000);
    }
};

struct DoubleAcc {
    static constexpr bool kSkipZero = true;
    double *J;
    __device__ __forceinline__ void add(int idx, double x) const { atomicAdd(J + idx, x); }
    __device__ __forceinline__ void add_prod(int idx, double a, double b) const { atomicAdd(J + idx, a * b); }
};

template <typename R, typename Acc>
__device__ __forceinline__ void acc_put(const Acc &acc, int idx, R a, R b)
{
    if (Acc::kSkipZero) {
        const R v = a * b;
        if (v != R(0)) acc.add(idx, v);
    } else {
        acc.add_prod(idx, a, b);
    }
}

// ------------------------------------------------------------------------------------
// Esirkepov charge-conserving deposit of one particle into the shared J tile (three
// components of jvol cells each).  With S0, DS the old shape and its change per axis on a
// common window, in 3D
//   Wx = DSx (S0y S0z + DSy S0z / 2 + S0y DSz / 2 + DSy DSz / 3)   (cyclic for y, z),
//   Jx(i+1/2) - Jx(i-1/2) = f_x Wx(i),  f_x = -(q w / dV) dx / dt,
// summed along x from zero at the window start.  The transverse factor is evaluated as
// S0a (S0b + DSb / 2) + DSa (S0b / 2 + DSb / 3) (two products per window row), and the
// running sums along the component's own axis, times f, are formed once per particle.
//
// WX, WY, WZ: window extents covered (each ORD + 1 or ORD + 2).  A particle that keeps
// its nodes along an axis has ORD + 1 non-zero entries there (the entry beyond is zero
// and so is the running sum at the window's last entry), so a particle that keeps its x
// and y nodes can be covered with ORD + 1 entries along x and y and lose nothing.
// ------------------------------------------------------------------------------------
template <int WX, int WY, int WZ, typename R, typename Acc>
__device__ __forceinline__ void esirkepov3d(const R *S0x, const R *DSx, const R *S0y, const R *DSy, const R *S0z,
                                            const R *DSz, R fx, R fy, R fz, int base, int jd0, int jd01, int jvol,
                                            const Acc &acc)
{
    const R half = R(0.5), third = R(1.0 / 3.0);
    R Ay[WY], Cy[WY], Az[WZ], Cz[WZ];
#pragma unroll
    for (int m = 0; m < WY; ++m) {
        Ay[m] = S0y[m] + half * DSy[m];
        Cy[m] = half * S0y[m] + third * DSy[m];
    }
#pragma unroll
    for (int m = 0; m < WZ; ++m) {
        Az[m] = S0z[m] + half * DSz[m];
        Cz[m] = half * S0z[m] + third * DSz[m];
    }
    R rx[WX - 1], ry[WY - 1], rz[WZ - 1];
    {
        R run = R(0);
#pragma unroll
        for (int i = 0; i < WX - 1; ++i) {
            run += DSx[i];
            rx[i] = fx * run;
        }
        run = R(0);
#pragma unroll
        for (int j = 0; j < WY - 1; ++j) {
            run += DSy[j];
            ry[j] = fy * run;
        }
        run = R(0);
#pragma unroll
        for (int k = 0; k < WZ - 1; ++k) {
            run += DSz[k];
            rz[k] = fz * run;
        }
    }
#pragma unroll
    for (int k = 0; k < WZ; ++k) {
#pragma unroll
        for (int j = 0; j < WY; ++j) {
            const R Y = S0y[j] * Az[k] + DSy[j] * Cz[k];
            const int row = base + jd0 * j + jd01 * k;
#pragma unroll
            for (int i = 0; i < WX - 1; ++i) acc_put<R>(acc, row + i, Y, rx[i]);
        }
    }
#pragma unroll
    for (int k = 0; k < WZ; ++k) {
#pragma unroll
        for (int i = 0; i < WX; ++i) {
            const R X = S0x[i] * Az[k] + DSx[i] * Cz[k];
            const int col = jvol + base + i + jd01 * k;
#pragma unroll
            for (int j = 0; j < WY - 1; ++j) acc_put<R>(acc, col + jd0 * j, X, ry[j]);
        }
    }
#pragma unroll
    for (int j = 0; j < WY; ++j) {
#pragma unroll
        for (int i = 0; i < WX; ++i) {
            const R X = S0x[i] * Ay[j] + DSx[i] * Cy[j];
            const int col = 2 * jvol + base + i + jd0 * j;
#pragma unroll
            for (int k = 0; k < WZ - 1; ++k) acc_put<R>(acc, col + jd01 * k, X, rz[k]);
        }
    }
}

// The entries of the N x N x W window outside the N x N x N one: what a particle that
// changes its z nodes adds beyond the window narrow along z as well (Jx and Jy at the
// last z entry, Jz at the last z face), with the values esirkepov3d<N, N, W> forms
// there.  Called only by the lanes that change their z nodes: for the others these
// entries are exactly zero (their z shape beyond entry N - 1 is zero and the running sum
// along z ends at exactly zero).
template <int N, int W, typename R, typename Acc>
__device__ __forceinline__ void esirkepov3d_zextra(const R *S0x, const R *DSx, const R *S0y, const R *DSy, const R *S0z,
                                                   const R *DSz, R fx, R fy, R fz, int base, int jd0, int jd01, int jvol,
                                                   const Acc &acc)
{
    const R half = R(0.5), third = R(1.0 / 3.0);
    constexpr int K = W - 1;  // the last z entry (Jx, Jy) and, less one, the last z face (Jz)
    const R Azk = S0z[K] + half * DSz[K];
    const R Czk = half * S0z[K] + third * DSz[K];
    R rx[N - 1], ry[N - 1];
    {
        R run = R(0);
#pragma unroll
        for (int i = 0; i < N - 1; ++i) {
            run += DSx[i];
            rx[i] = fx * run;
        }
        run = R(0);
#pragma unroll
        for (int j = 0; j < N - 1; ++j) {
            run += DSy[j];
            ry[j] = fy * run;
        }
    }
    R rzk;
    {
        R run = R(0);
#pragma unroll
        for (int k = 0; k < K; ++k) run += DSz[k];
        rzk = fz * run;
    }
#pragma unroll
    for (int j = 0; j < N; ++j) {
        const R Y = S0y[j] * Azk + DSy[j] * Czk;
        const int row = base + jd0 * j + jd01 * K;
#pragma unroll
        for (int i = 0; i < N - 1; ++i) acc_put<R>(acc, row + i, Y, rx[i]);
    }
#pragma unroll
    for (int i = 0; i < N; ++i) {
        const R X = S0x[i] * Azk + DSx[i] * Czk;
        const int col = jvol + base + i + jd01 * K;
#pragma unroll
        for (int j = 0; j < N - 1; ++j) acc_put<R>(acc, col + jd0 * j, X, ry[j]);
    }
#pragma unroll
    for (int j = 0; j < N; ++j) {
        const R Ay = S0y[j] + half * DSy[j], Cy = half * S0y[j] + third * DSy[j];
#pragma unroll
        for (int i = 0; i < N; ++i) {
            const R X = S0x[i] * Ay + DSx[i] * Cy;
            acc_put<R>(acc, 2 * jvol + base + i + jd0 * j + jd01 * (K - 1), X, rzk);
        }
    }
}

// The entries of the W x W x W window outside the N x N x W one (N = ORD + 1 along x and
// y): what a particle that changes its x or y nodes adds beyond the narrow window that
// esirkepov3d<N, N, W> covers.  The values are those esirkepov3d<W, W, W> forms at the
// same entries, so the narrow call plus this one is the wide deposit.  Called only by the
// lanes that change their x or y nodes: for the others these entries are exactly zero
// (their shape beyond entry N - 1 is zero and the running sums end at exactly zero), and
// leaving them out keeps the extra atomics of a warp to the lanes that need them instead
// of every lane.
template <int N, int W, typename R, typename Acc>
__device__ __forceinline__ void esirkepov3d_extra(const R *S0x, const R *DSx, const R *S0y, const R *DSy, const R *S0z,
                                                  const R *DSz, R fx, R fy, R fz, int base, int jd0, int jd01, int jvol,
                                                  const Acc &acc)
{
    const R half = R(0.5), third = R(1.0 / 3.0);
    R Ay[W], Cy[W], Az[W], Cz[W];
#pragma unroll
    for (int m = 0; m < W; ++m) {
        Ay[m] = S0y[m] + half * DSy[m];
        Cy[m] = half * S0y[m] + third * DSy[m];
        Az[m] = S0z[m] + half * DSz[m];
        Cz[m] = half * S0z[m] + third * DSz[m];
    }
    R rx[W - 1], ry[W - 1];
    {
        R run = R(0);
#pragma unroll
        for (int i = 0; i < W - 1; ++i) {
            run += DSx[i];
            rx[i] = fx * run;
        }
        run = R(0);
#pragma unroll
        for (int j = 0; j < W - 1; ++j) {
            run += DSy[j];
            ry[j] = fy * run;
        }
    }
    R rz[W - 1];
    {
        R run = R(0);
#pragma unroll
        for (int k = 0; k < W - 1; ++k) {
            run += DSz[k];
            rz[k] = fz * run;
        }
    }
#pragma unroll
    for (int k = 0; k < W; ++k) {
#pragma unroll
        for (int j = 0; j < W; ++j) {
            const R Y = S0y[j] * Az[k] + DSy[j] * Cz[k];
            const int row = base + jd0 * j + jd01 * k;
#pragma unroll
            for (int i = 0; i < W - 1; ++i)
                if (i >= N - 1 || j >= N) acc_put<R>(acc, row + i, Y, rx[i]);
        }
    }
#pragma unroll
    for (int k = 0; k < W; ++k) {
#pragma unroll
        for (int i = 0; i < W; ++i) {
            const R X = S0x[i] * Az[k] + DSx[i] * Cz[k];
            const int col = jvol + base + i + jd01 * k;
#pragma unroll
            for (int j = 0; j < W - 1; ++j)
                if (i >= N || j >= N - 1) acc_put<R>(acc, col + jd0 * j, X, ry[j]);
        }
    }
#pragma unroll
    for (int j = 0; j < W; ++j) {
#pragma unroll
        for (int i = 0; i < W; ++i) {
            if (i < N && j < N) continue;
            const R X = S0x[i] * Ay[j] + DSx[i] * Cy[j];
            const int col = 2 * jvol + base + i + jd0 * j;
#pragma unroll
            for (int k = 0; k < W - 1; ++k) acc_put<R>(acc, col + jd01 * k, X, rz[k]);
        }
    }
}

// The deposit of one particle; every lane of the warp calls it (a lane without a particle
// passes f = 0 and a position inside the tile).  In 2D3V (x-z plane) Wx = DSx (S0z +
// DSz/2), Wz = DSz (S0x + DSx/2) and the out-of-plane Jy = f_y' (S0x S0z + DSx S0z / 2 +
// S0x DSz / 2 + DSx DSz / 3) with f_y' = (q w / dV) v_y; the 2D3V loops skip zero
// contributions (up to 16 particles per cell contend there).  kNarrow (3D): the window
// adapts to the particles.  With kLane every lane covers ORD + 1 entries along each axis;
// a lane whose particle changes its z nodes adds the entries beyond them along z
// (esirkepov3d_zextra) and one that changes its x or y nodes those of the ORD + 2 window
// beyond them along x and y (esirkepov3d_extra), so the other lanes of its warp add none
// of those zeros.  Without kLane (fewer registers: the launches over many instances) the
// warp covers ORD + 1 entries along x and y when none of its particles changes its x or y
// nodes (one vote per warp), ORD + 2 otherwise, and ORD + 2 along z.
template <int ND, int ORD, bool kDisp, bool kNarrow, bool kLane, typename R, typename Acc>
__device__ __forceinline__ void deposit_esirkepov(const int l0[3], const R o0[3], const int l1[3], const R o1[3],
                                                  const R disp[3], R fx, R fy, R fz, int jlo, int jlo_y, int jd0,
                                                  int jd01, int jvol, const Acc &acc)
{
    constexpr int W = ORD + 2;
    R S0x[W], DSx[W], S0y[W], DSy[W], S0z[W], DSz[W];
    int nwx, nwy = 1, nwz;
    const int wsx = shape_window<ORD, kDisp>(l0[0], o0[0], l1[0], o1[0], disp[0], S0x, DSx, nwx) - jlo;
    const int wsz = shape_window<ORD, kDisp>(l0[2], o0[2], l1[2], o1[2], disp[2], S0z, DSz, nwz) - jlo;
    const R half = R(0.5), third = R(1.0 / 3.0);
    if (ND == 3) {
        const int wsy = shape_window<ORD, kDisp>(l0[1], o0[1], l1[1], o1[1], disp[1], S0y, DSy, nwy) - jlo_y;
        const int base = wsx + jd0 * wsy + jd01 * wsz;
        if (kNarrow && kLane) {
            esirkepov3d<ORD + 1, ORD + 1, ORD + 1, R>(S0x, DSx, S0y, DSy, S0z, DSz, fx, fy, fz, base, jd0, jd01, jvol, acc);
            if (nwz > ORD + 1)
                esirkepov3d_zextra<ORD + 1, W, R>(S0x, DSx, S0y, DSy, S0z, DSz, fx, fy, fz, base, jd0, jd01, jvol, acc);
            if (nwx > ORD + 1 || nwy > ORD + 1)
                esirkepov3d_extra<ORD + 1, W, R>(S0x, DSx, S0y, DSy, S0z, DSz, fx, fy, fz, base, jd0, jd01, jvol, acc);
        } else if (kNarrow && !__any_sync(0xffffffffu, nwx > ORD + 1 || nwy > ORD + 1)) {
            esirkepov3d<ORD + 1, ORD + 1, W, R>(S0x, DSx, S0y, DSy, S0z, DSz, fx, fy, fz, base, jd0, jd01, jvol, acc);
        } else {
            esirkepov3d<W, W, W, R>(S0x, DSx, S0y, DSy, S0z, DSz, fx, fy, fz, base, jd0, jd01, jvol, acc);
        }
    } else {
        // fy carries the out-of-plane factor (q w / dV) v_y here
        const int base = wsx + jd01 * wsz;
#pragma unroll
        for (int k = 0; k < W; ++k) {
            const R fY = fx * (S0z[k] + half * DSz[k]);
            R run = R(0);
#pragma unroll
            for (int i = 0; i < W - 1; ++i) {
                run += DSx[i];
                const R v = fY * run;
                if (v != R(0)) acc.add(base + i + jd01 * k, v);
            }
        }
#pragma unroll
        for (int i = 0; i < W; ++i) {
            const R fX = fz * (S0x[i] + half * DSx[i]);
            R run = R(0);
#pragma unroll
            for (int k = 0; k < W - 1; ++k) {
                run += DSz[k];
                const R v = fX * run;
                if (v != R(0)) acc.add(2 * jvol + base + i + jd01 * k, v);
            }
        }
#pragma unroll
        for (int k = 0; k < W; ++k) {
#pragma unroll
            for (int i = 0; i < W; ++i) {
                const R v = fy * (S0x[i] * S0z[k] + half * (DSx[i] * S0z[k] + S0x[i] * DSz[k]) + third * DSx[i] * DSz[k]);
                if (v != R(0)) acc.add(jvol + base + i + jd01 * k, v);
            }
        }
    }
}

// ------------------------------------------------------------------------------------
// Vay pusher (Sec. 2 of the paper; Vay, Phys. Plasmas 15, 056701 (2008)).  c = 1,
// h = q dt / (2 m):
//   u' = u + 2h E + h v x B,  tau = h B,  u* = u'.tau,  sigma = (1 + u'^2) - tau^2,
//   gamma^2 = (sigma + sqrt(sigma^2 + 4 (tau^2 + u*^2))) / 2   (sigma >= 0)
//           = 2 (tau^2 + u*^2) / (sqrt(...) - sigma)            (sigma < 0, same value),
//   t = tau / gamma,  s = 1 / (1 + t^2),  u_new = s (u' + (u'.t) t + u' x t).
// FP32 form: sigma is the one quantity that cancels at large gamma (gamma'^2 ~ tau^2), so
// where it can cancel gamma'^2, tau^2 and their difference are formed in FP64 from the
// FP32 operands; the roots are FP32, taken on the cancellation-free branch.  Where it
// cannot -- tau^2 < gamma'^2 / 4 for every particle of the warp (one vote), so that
// sigma > 3 gamma'^2 / 4 and its FP32 difference is within a few ulp of sigma -- the
// difference is taken in FP32: GB300's FP64 rate is a small fraction of its FP32 one.
// ------------------------------------------------------------------------------------
__device__ __forceinline__ void push_vay(float u[3], const float E[3], const float B[3], float h)
{
    const float g = sqrtf(1.f + u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    const float ig = 1.f / g;
    const float v0 = u[0] * ig, v1 = u[1] * ig, v2 = u[2] * ig;
    const float up0 = u[0] + 2.f * h * E[0] + h * (v1 * B[2] - v2 * B[1]);
    const float up1 = u[1] + 2.f * h * E[1] + h * (v2 * B[0] - v0 * B[2]);
    const float up2 = u[2] + 2.f * h * E[2] + h * (v0 * B[1] - v1 * B[0]);
    const float t0 = h * B[0], t1 = h * B[1], t2 = h * B[2];
    const float ustar = up0 * t0 + up1 * t1 + up2 * t2;
    const float gp2f = __fmaf_rn(up0, up0, __fmaf_rn(up1, up1, __fmaf_rn(up2, up2, 1.f)));
    const float tau2f = __fmaf_rn(t0, t0, __fmaf_rn(t1, t1, t2 * t2));
    float sigma, tau2;
    if (__all_sync(__activemask(), tau2f < 0.25f * gp2f)) {
        sigma = gp2f - tau2f;
        tau2 = tau2f;
    } else {
        const double gp2 = 1.0 + (double)up0 * up0 + (double)up1 * up1 + (double)up2 * up2;
        const double tau2d = (double)t0 * t0 + (double)t1 * t1 + (double)t2 * t2;
        sigma = (float)(gp2 - tau2d);
        tau2 = (float)tau2d;
    }
    const float q4 = tau2 + ustar * ustar;
    const float root = sqrtf(sigma * sigma + 4.f * q4);
    const float g2 = sigma >= 0.f ? 0.5f * (sigma + root) : 2.f * q4 / (root - sigma);
    const float ign = 1.f / sqrtf(g2);
    const float s0 = t0 * ign, s1 = t1 * ign, s2 = t2 * ign;
    const float s = 1.f / (1.f + s0 * s0 + s1 * s1 + s2 * s2);
    const float upt = up0 * s0 + up1 * s1 + up2 * s2;
    u[0] = s * (up0 + upt * s0 + (up1 * s2 - up2 * s1));
    u[1] = s * (up1 + upt * s1 + (up2 * s0 - up0 * s2));
    u[2] = s * (up2 + upt * s2 + (up0 * s1 - up1 * s0));
}

__device__ __forceinline__ void push_vay(double u[3], const double E[3], const double B[3], double h)
{
    const double g = sqrt(1.0 + u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    const double v0 = u[0] / g, v1 = u[1] / g, v2 = u[2] / g;
    const double up0 = u[0] + 2.0 * h * E[0] + h * (v1 * B[2] - v2 * B[1]);
    const double up1 = u[1] + 2.0 * h * E[1] + h * (v2 * B[0] - v0 * B[2]);
    const double up2 = u[2] + 2.0 * h * E[2] + h * (v0 * B[1] - v1 * B[0]);
    const double t0 = h * B[0], t1 = h * B[1], t2 = h * B[2];
    const double tau2 = t0 * t0 + t1 * t1 + t2 * t2;
    const double ustar = up0 * t0 + up1 * t1 + up2 * t2;
    const double sigma = (1.0 + up0 * up0 + up1 * up1 + up2 * up2) - tau2;
    const double q4 = tau2 + ustar * ustar;
    const double root = sqrt(sigma * sigma + 4.0 * q4);
    const double g2 = sigma >= 0.0 ? 0.5 * (sigma + root) : 2.0 * q4 / (root - sigma);
    const double gn = sqrt(g2);
    const double s0 = t0 / gn, s1 = t1 / gn, s2 = t2 / gn;
    const double s = 1.0 / (1.0 + s0 * s0 + s1 * s1 + s2 * s2);
    const double upt = up0 * s0 + up1 * s1 + up2 * s2;
    u[0] = s * (up0 + upt * s0 + (up1 * s2 - up2 * s1));
    u[1] = s * (up1 + upt * s1 + (up2 * s0 - up0 * s2));
    u[2] = s * (up2 + upt * s2 + (up0 * s1 - up1 * s0));
}

// Boris pusher (Sec. 2; BorisICNSP): half electric kick, rotation with t = h B / gamma^-,
// s = 2 t / (1 + t^2), half electric kick.
template <typename R>
__device__ __forceinline__ void push_boris(R u[3], const R E[3], const R B[3], R h)
{
    const R um0 = u[0] + h * E[0], um1 = u[1] + h * E[1], um2 = u[2] + h * E[2];
    const R gm = sqrt(R(1) + um0 * um0 + um1 * um1 + um2 * um2);
    const R t0 = h * B[0] / gm, t1 = h * B[1] / gm, t2 = h * B[2] / gm;
    const R f = R(2) / (R(1) + t0 * t0 + t1 * t1 + t2 * t2);
    const R s0 = f * t0, s1 = f * t1, s2 = f * t2;
    const R p0 = um0 + (um1 * t2 - um2 * t1);
    const R p1 = um1 + (um2 * t0 - um0 * t2);
    const R p2 = um2 + (um0 * t1 - um1 * t0);
    u[0] = um0 + (p1 * s2 - p2 * s1) + h * E[0];
    u[1] = um1 + (p2 * s0 - p0 * s2) + h * E[1];
    u[2] = um2 + (p0 * s1 - p1 * s0) + h * E[2];
}

// ------------------------------------------------------------------------------------
// Position update in cell units: o += dt v / dx; k = floor(o); o -= k; an offset that
// rounds to 1 after the subtraction becomes 0 in the next cell.  FP64 uses the same
// operation order as a plain evaluation of (o + (dt * (u / g)) / dx) with every product
// and quotient rounded (no contraction).  Returns the cell step k in {-1, 0, 1}; a move
// outside (-1, 2) (impossible below the Courant limit unless values are not finite)
// leaves the particle in place and sets *bad.
// ------------------------------------------------------------------------------------
__device__ __forceinline__ int move_axis(float &o, float u, float ig, float dt_dx, float &disp, bool &bad)
{
    disp = __fmul_rn(dt_dx, __fmul_rn(u, ig));
    float x = __fadd_rn(o, disp);
    if (!(x > -1.f && x < 2.f)) {
        bad = true;
        return 0;
    }
    const float k = floorf(x);
    x = __fsub_rn(x, k);
    int ki = (int)k;
    if (x >= 1.f) {
        x = 0.f;
        ki += 1;
    }
    o = x;
    return ki;
}

__device__ __forceinline__ int move_axis(double &o, double u, double g, double dt, double dx, bool &bad)
{
    double x = __dadd_rn(o, __ddiv_rn(__dmul_rn(dt, __ddiv_rn(u, g)), dx));
    if (!(x > -1.0 && x < 2.0)) {
        bad = true;
        return 0;
    }
    const double k = floor(x);
    x = __dsub_rn(x, k);
    int ki = (int)k;
    if (x >= 1.0) {
        x = 0.0;
        ki += 1;
    }
    o = x;
    return ki;
}

__device__ __forceinline__ double gamma_of(double u0, double u1, double u2)
{
    return __dsqrt_rn(__dadd_rn(__dadd_rn(__dadd_rn(1.0, __dmul_rn(u0, u0)), __dmul_rn(u1, u1)), __dmul_rn(u2, u2)));
}

// ------------------------------------------------------------------------------------
// TMA (cp.async.bulk.tensor) and mbarrier primitives.  Every wait is bounded in time.
// ------------------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return done != 0;
}

// Waits for phase `parity` of the barrier for at most ~`limit_cycles` SM clocks.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, long long limit_cycles)
{
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - t0 > limit_cycles) return false;
    }
    return true;
}

__device__ __forceinline__ void tmap_acquire(const CUtensorMap *map)
{
    asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(map) : "memory");
}

// Ampere-style asynchronous global -> shared copies of 4 or 8 bytes (cp.async), grouped
// per thread: commit closes a group, wait_all waits for this thread's groups.
template <int N>
__device__ __forceinline__ void cp_async(void *smem_dst, const void *gmem_src)
{
    static_assert(N == 4 || N == 8, "cp.async size");
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(smem_addr(smem_dst)), "l"(gmem_src), "n"(N)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, int x, int y, int z, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::
            "r"(smem_addr(dst)),
        "l"(map), "r"(x), "r"(y), "r"(z), "r"(smem_addr(bar))
        : "memory");
}

}  // namespace pic
