// pic_instance.h -- device view of one simulation instance (InstDev), its step
// constants and the launch-wide view of instances stepped together: everything the
// particle kernel reads.  Not part of the public ABI (include/pic.h).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <climits>

#include "../../include/pic.h"

namespace pic {

constexpr int kGhost = 4;       // ghost layers per side of every active axis (fields)
constexpr int kDirs = 27;       // tile-to-tile move directions (3 per axis)
constexpr int kDead = 27;       // bucket of particles removed at absorbing faces
constexpr int kBuckets = 28;    // 27 directions + dead
constexpr int kPre = 29;        // per chunk: exclusive prefix of the 28 buckets + size
constexpr int kCenterDir = 13;  // (0,0,0)
// Per-tile source record precomputed ahead of the particle kernel (k_tile_sources): the
// tile's particle count, its number of non-empty (source, chunk) sub-ranges (-1 when more
// than kSubCache) and their first destination slots and buffer positions.
constexpr int kSubCache = 64;
constexpr int kRecSlot = 4;                            // sub_slot[kSubCache + 1] from here
constexpr int kRecPos = kRecSlot + kSubCache + 1;      // sub_pos[kSubCache] from here
constexpr int kSrcRec = (kRecPos + kSubCache + 3) / 4 * 4;  // ints per tile

// Division of 0 <= x < 2^31 by a fixed divisor d >= 1 without a divide instruction
// (Granlund & Montgomery, "Division by invariant integers using multiplication", 1994,
// round-up variant): s = ceil(log2 d), m = floor(2^(32+s) / d) + 1 (33 bits), then
// floor(x / d) = (x * m) >> (32 + s).
struct FastDiv {
    unsigned long long m;
    int s;
    int d;
};

inline FastDiv make_fastdiv(int d)
{
    FastDiv f;
    f.d = d;
    f.s = 0;
    while ((1LL << f.s) < d) ++f.s;
    f.m = (1ULL << (32 + f.s)) / (unsigned long long)d + 1ULL;  // 32 + s <= 63 for d < 2^31
    return f;
}

__host__ __device__ __forceinline__ int fast_div(int x, const FastDiv &f)
{
    return (int)(((unsigned long long)(unsigned)x * f.m) >> (32 + f.s));
}

// device error word bits (sticky)
constexpr int kErrTimeout = 1;      // a bounded mbarrier wait gave up
constexpr int kErrSpeed = 2;        // |displacement| >= 1 cell or non-finite in a step
constexpr int kErrInternal = 4;     // layout/count consistency check failed
constexpr int kErrCapacity = 8;     // more particles than the buffers hold

// Device view of one instance.  Pointers are device addresses; field arrays are padded
// with kGhost layers per side on active axes, x rows padded to a 16-byte multiple.
// Per-instance step constants in the working precision, formed once on the host in FP64
// (and rounded to FP32 for FP32 instances) so that no kernel spends FP64 divisions on
// them: GB300's FP64 pipe is a small fraction of its FP32 rate.
template <typename R>
struct StepCoef {
    R h;          // q dt / (2 m)
    R qdv;        // q / dV
    R jf[3];      // dx_a / dt
    R dtdx[3];    // dt / dx_a
    R half_dt;    // dt / 2
    R dt;
    R inv_dx[3];  // 1 / dx_a
};

struct InstDev {
    int ndim;
    int n[3];       // interior cells
    int bc[3];      // 0 periodic, 1 absorbing
    int gh[3];      // ghost layers per axis (kGhost or 0 on the inactive y of 2D)
    int P[3];       // padded dims
    long long sy, sz;  // padded strides (elements)
    long long cstride; // elements per component array
    int ts[3];      // tile size
    int nt[3];      // tiles per axis
    int ntiles;
    int tile_base;  // first global tile index of this instance in a launch
    int R;          // particles per chunk (threads * particles per thread)
    int cap;        // particle capacity per buffer
    int chunk_cap;  // chunk records per layout
    int filter_passes;
    int solver;         // PIC_SOLVER_YEE or PIC_SOLVER_CK
    int absorb_cells;
    double absorb_strength;
    double dt, dx[3], q, m;
    StepCoef<float> cf;   // FP32 instances
    StepCoef<double> cd;  // FP64 instances
    // fields (element type set by the precision of the launch).  E and B have two
    // buffers: the fused Maxwell update reads one pair and writes the other, then flips
    // *fpar; every reader takes the current pair through cur_eb / eb_field.
    void *E[3], *B[3], *J[3], *Jt[3];  // Jt: scratch for filter sweeps
    void *E2[3], *B2[3];               // the second E / B buffer
    int *fpar;                         // 0: E, B current; 1: E2, B2
    // particles, two buffers
    int *cell[2];
    void *off[2][3];
    void *u[2][3];
    void *w[2];
    int *id[2];   // null when ids are not tracked
    // tile layouts, two sets (input / output of a step)
    int *seg[2];        // [ntiles + 1] segment starts in the particle buffer
    int *chunk_base[2]; // [ntiles + 1] first chunk record of each tile
    int *chunk_pre[2];  // [chunk_cap * kPre]
    int *chunk_cb[2];   // [chunk_cap * kBuckets] count of each bucket in earlier chunks of the tile
    int *tot[2];        // [ntiles * kBuckets] bucket totals of each tile
    int *pop;           // [ntiles] particles in each tile at the step boundary
    int *srcrec;        // [ntiles * kSrcRec] source records of the coming particle phase
    int *cur;           // device parity: which layout/buffer holds the current state
    int *jsel;          // which J array (0: J, 1: Jt) holds the filtered current
    int *err;           // sticky error word
    unsigned long long *lost; // particles removed so far
    int *live;          // live particles (written by the scan)
    const CUtensorMap *tmap;  // 12 maps: Ex Ey Ez Bx By Bz boxes for the gather stage, for
                              // buffer 0 then buffer 1
    const void *damp[3];      // absorbing-layer factor per cell index along each axis
                              // (working precision; null on periodic / inactive axes)
    FastDiv div_n0, div_n1;   // cell index -> (i, j, k)
    // ion background of a lab-frame plasma load: lab-stationary ions, i.e. in this frame
    // a rigid density gamma_b n0 p(gamma_b (z + beta_b t)) of charge -q on [0, Lz) at t = 0
    int ion;            // 0: none
    double ion_n0, ion_zs, ion_ramp, ion_gb, ion_beta;
    // the box the ion profile fills: this grid's own ([0, n2 dz), its own z boundary), or,
    // for a z slab of a larger grid, that grid's, with ion_z0 the coordinate there of this
    // grid's z = 0
    double ion_z0, ion_lz;
    int ion_periodic;
    int ion_k0, ion_k1; // z planes whose Jz faces carry the ion current (a slab: its own)
    void *ion_face;     // [n[2]] this step's ion current on the Jz faces (working precision)
    int *phase;         // particle phases run since the last load (device counter)
    double gb, beta_b;  // the frame's boost: Lorentz factor and velocity
    // beam injection plane: ids >= inj_id0 (INT_MAX: off) upstream of the lab plane, at
    // z' = inj_zb - beta_b t' in this frame, are frozen (no field acts on them)
    int inj_id0;
    double inj_zb;
    int box[3];         // TMA box extents (elements)
    int box_lo[3];      // box origin relative to the tile origin (cells, <= 0)
    int jlo;            // J tile origin relative to the tile origin (-1 or -2)
    int jdim[3];        // J tile extents
};

template <typename R>
__host__ __device__ __forceinline__ const StepCoef<R> &coef(const InstDev &I);
template <>
__host__ __device__ __forceinline__ const StepCoef<float> &coef<float>(const InstDev &I) { return I.cf; }
template <>
__host__ __device__ __forceinline__ const StepCoef<double> &coef<double>(const InstDev &I) { return I.cd; }

// The E / B buffer pair holding the current fields (read once per kernel).
struct EBPtr {
    void *E[3], *B[3];
};

__device__ __forceinline__ EBPtr cur_eb(const InstDev &I)
{
    const int par = *(volatile const int *)I.fpar;
    EBPtr f;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        f.E[a] = par ? I.E2[a] : I.E[a];
        f.B[a] = par ? I.B2[a] : I.B[a];
    }
    return f;
}

// Current buffer of field component comp (0..5: Ex Ey Ez Bx By Bz).
__device__ __forceinline__ void *eb_field(const InstDev &I, int comp)
{
    const int par = *(volatile const int *)I.fpar;
    return comp < 3 ? (par ? I.E2[comp] : I.E[comp]) : (par ? I.B2[comp - 3] : I.B[comp - 3]);
}

// launch-wide view of a set of instances stepped together
struct Launch {
    const InstDev *inst;  // device array
    const int *tile_start;// [ninst + 1] global tile offsets (device)
    const long long *cell_start; // [ninst + 1] global interior-cell offsets (device)
    int ninst;
    int total_tiles;
    long long total_cells;
};

__device__ __forceinline__ int find_instance(const int *tile_start, int ninst, int g)
{
    int lo = 0, hi = ninst - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (__ldg(tile_start + mid) <= g) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ int find_instance_ll(const long long *start, int ninst, long long g)
{
    int lo = 0, hi = ninst - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (__ldg(start + mid) <= g) lo = mid; else hi = mid - 1;
    }
    return lo;
}

}  // namespace pic
