// pic_internal.h -- device view of one simulation instance and shared definitions of
// the sm_103a boosted-frame PIC kernels.  Not part of the public ABI (include/pic.h).
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
    R qdv;        // q / dV, times the fixed-point current scale in FP32 mode
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
    // fields (element type set by the precision of the launch)
    void *E[3], *B[3], *J[3], *Jt[3];  // Jt: scratch for filter sweeps
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
    int *cur;           // device parity: which layout/buffer holds the current state
    int *jsel;          // which J array (0: J, 1: Jt) holds the filtered current
    int *err;           // sticky error word
    unsigned long long *lost; // particles removed so far
    int *live;          // live particles (written by the scan)
    const CUtensorMap *tmap;  // 6 maps: Ex Ey Ez Bx By Bz boxes for the gather stage
    const void *damp[3];      // absorbing-layer factor per cell index along each axis
                              // (working precision; null on periodic / inactive axes)
    FastDiv div_n0, div_n1;   // cell index -> (i, j, k)
    float jscale, jinv;       // FP32 fixed-point current: scale (a power of two) and 1/scale
    // ion background of a lab-frame plasma load: lab-stationary ions, i.e. in this frame
    // a rigid density gamma_b n0 p(gamma_b (z + beta_b t)) of charge -q on [0, Lz) at t = 0
    int ion;            // 0: none
    double ion_n0, ion_zs, ion_ramp, ion_gb, ion_beta;
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

// FP64 particles to place in the canonical order (device arrays, 3 values per particle
// for off and u); slot[i] is particle i's position in the sorted buffer.
struct PlaceSrc {
    const int *cell;
    const double *off, *u, *w;
    const int *id;  // null: ids id_base + i
    const int *slot;
    long long n;
    long long id_base;
};

// Lab-frame plasma drawn on the device (see k_load.cu)
struct PlasmaGen {
    int ndim;
    int n[3];
    long long ncell;
    double dx[3];
    double gb, beta, n0, zs, ramp, dV;
    double uth[3];
    int ppc;
    uint64_t seed;
};

// Lab-frame stations of one instance (k_stations.cu): device arrays
struct StationDev {
    const double *z_lab;  // [nst]
    int *count;           // [nst] records taken
    double *t_lab;        // [nst][max_records]
    void *fields;         // [nst][max_records][6][n1][n0], working precision
    int max_records;
};

// Laser antenna of one instance (k_antenna.cu): the incident pulse on a 1D lattice
// aligned with the grid's z lattice, and the lab plane it is emitted through
struct AntDev {
    double *ge, *gb;      // E_x on lattice nodes lo .. lo + na - 1, B_y half a node above
    long long lo, na;
    double zb, beta;      // the plane: z' = zb - beta t'
    double t0;            // t' when the antenna was set
    double w0, xc, yc;    // transverse profile exp(-((x - xc)^2 + (y - yc)^2) / w0^2)
    int *n;               // Maxwell phases since the antenna was set (device counter)
};

// host-side launchers
cudaError_t launch_stations(int fp64, const InstDev *d_inst, const StationDev &S, int nst, int plane, cudaStream_t s);
cudaError_t launch_place(int fp64, const InstDev &I, const PlaceSrc &s, cudaStream_t st);
cudaError_t launch_plasma_count(const PlasmaGen &G, int *count, cudaStream_t st);
cudaError_t launch_plasma_write(int fp64, const InstDev &I, const PlasmaGen &G, const int *slot0, const int *id0,
                                cudaStream_t st);
cudaError_t launch_ion_current(int fp64, const Launch &L, cudaStream_t s);
cudaError_t launch_rho_ion(const Launch &L, long long ncell, double *rho, cudaStream_t s);
// inj: some instance of the launch has a beam injection plane
cudaError_t launch_particles(int ndim, int order, int fp64, int pusher, bool inj, const Launch &L, size_t smem,
                             cudaStream_t s);
int particle_chunk();
int particle_threads();
cudaError_t launch_scan(const Launch &L, int mode, int *const *dst, cudaStream_t s);
cudaError_t launch_readout(int fp64, const Launch &L, const int *const *start, int *cell, double *off, double *u,
                           double *w, int *id, cudaStream_t s);
cudaError_t launch_particle_sums(int fp64, const Launch &L, double *sums, cudaStream_t s);
cudaError_t launch_rho(int order, int fp64, const Launch &L, double *rho, cudaStream_t s);
// passes: the filter passes of every instance of the launch (0 when they differ)
cudaError_t launch_filter(int fp64, const Launch &L, const long long *const pencil_start[3],
                          const long long pencil_total[3], int ndim, int passes, cudaStream_t s);
// pencils of the per-axis filter kernel for an instance: kPencil (64) cells along the
// axis times 32 lines (x: 32 consecutive (y, z) rows; y, z: 32 consecutive x columns)
inline long long filter_pencils(const int n[3], int ndim, int axis)
{
    const int kP = 64;
    if (ndim == 2 && axis == 1) return 0;
    if (axis == 0) return (long long)((n[0] + kP - 1) / kP) * (((long long)n[1] * n[2] + 31) / 32);
    const long long cols = (n[0] + 31) / 32;
    if (axis == 1) return cols * ((n[1] + kP - 1) / kP) * n[2];
    return cols * ((n[2] + kP - 1) / kP) * n[1];
}
cudaError_t launch_maxwell(int fp64, int solver, const Launch &L, int filtered, cudaStream_t s);
// the three sub-updates of launch_maxwell, for interleaving the antenna's kernels
cudaError_t launch_bhalf(int fp64, int solver, const Launch &L, int damp, cudaStream_t s);
cudaError_t launch_efull(int fp64, const Launch &L, int filtered, cudaStream_t s);
// antenna: what = 0 adds the incident field downstream of the plane (when set), 1 the
// values the plane passed in the last phase; B_y / E_x terms of the boundary; 1D lattice
cudaError_t launch_ant_add(int fp64, const InstDev *d_inst, const InstDev &I, const AntDev &A, int what, cudaStream_t s);
cudaError_t launch_ant_bterm(int fp64, const InstDev *d_inst, const InstDev &I, const AntDev &A, int damp, cudaStream_t s);
cudaError_t launch_ant_eterm(int fp64, const InstDev *d_inst, const InstDev &I, const AntDev &A, cudaStream_t s);
cudaError_t launch_ant_lattice(const AntDev &A, double dt, double dz, int what, cudaStream_t s);
cudaError_t launch_ghost(int fp64, const Launch &L, int axis, long long per_inst_max, cudaStream_t s);
cudaError_t prepare_particles(int ndim, int order, int fp64, int pusher, size_t smem);
cudaError_t launch_field_energy(int fp64, const Launch &L, double *sums, cudaStream_t s);
cudaError_t launch_pack(int fp64, const InstDev &I, int comp, int filtered, double *dense, long long ncell, cudaStream_t s);
cudaError_t launch_unpack(int fp64, const InstDev &I, int comp, const double *dense, long long ncell, cudaStream_t s);
cudaError_t launch_dive(int fp64, const InstDev &I, double *dense, long long ncell, cudaStream_t s);
// max |a - b| (as the bits of a non-negative double, atomicMax) and sum (a - b)^2
cudaError_t launch_residual(const double *a, const double *b, long long n, unsigned long long *max_bits, double *sumsq,
                            cudaStream_t s);

// Read-only view of a pic_ctx (defined in pic_api.cu) for entry points in other files.
struct CtxView {
    const Launch *launch;
    int order, fp64;
    long long ncell;
    cudaStream_t stream;
    int device;
    bool loaded, is_batch;
};

}  // namespace pic

struct pic_ctx;
namespace pic {
bool ctx_view(pic_ctx *c, CtxView *v);

}  // namespace pic
