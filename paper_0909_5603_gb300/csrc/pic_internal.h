// pic_internal.h -- shared definitions of the sm_103a boosted-frame PIC kernels and
// their host-side launchers.  Not part of the public ABI (include/pic.h).
#pragma once

#include "pic_instance.h"

#include <vector>

namespace pic {

// FP64 particles to place in the canonical order (device arrays, 3 values per particle
// for off and u); slot[i] is particle i's position in the sorted buffer.
struct PlaceSrc {
    const int *cell;
    const void *off, *u, *w;  // FP64, or FP32 when f32 is set
    const int *id;  // null: ids id_base + i
    const int *slot;
    long long n;
    long long id_base;
    int f32;
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
// Read-out staging in the storage precision (off and u 3 values per particle) with a map:
// map[i] >= 0 the slot in buffer 0, else -1 - map[i] the position in buffer 1
struct StagedSrc {
    const int *cell;
    const void *off, *u, *w;
    const int *id;
    const int *map;
    long long n;
};
cudaError_t launch_place_staged(int fp64, const InstDev &I, const StagedSrc &s, cudaStream_t st);
cudaError_t launch_plasma_count(const PlasmaGen &G, int *count, cudaStream_t st);
cudaError_t launch_plasma_write(int fp64, const InstDev &I, const PlasmaGen &G, const int *slot0, const int *id0,
                                cudaStream_t st);
// J of a step's start for a launch of one instance (h: its host copy): the ion faces
// (when it has ions), then Jx = Jy = 0, Jz = the ion current, in one pass
cudaError_t launch_j_init_one(int fp64, const Launch &L, const InstDev &h, cudaStream_t s);
cudaError_t launch_ion_current(int fp64, const Launch &L, cudaStream_t s);
cudaError_t launch_rho_ion(const Launch &L, long long ncell, double *rho, cudaStream_t s);
// inj: some instance of the launch has a beam injection plane
// one: for a launch of one instance, its host copy (passed to the kernel by value); null
// for a batch
cudaError_t launch_particles(int ndim, int order, int fp64, int pusher, bool inj, const Launch &L, const InstDev *one,
                             size_t smem, cudaStream_t s);
int particle_chunk();
int particle_threads();
cudaError_t launch_scan(const Launch &L, int mode, int *const *dst, cudaStream_t s);
// per-tile source records of the coming particle phase (after the scan of mode 0)
cudaError_t launch_tile_sources(const Launch &L, cudaStream_t s);
// off, u, w: staging in the storage precision (double or float)
cudaError_t launch_readout(int fp64, const Launch &L, const int *const *start, int *cell, void *off, void *u,
                           void *w, int *id, cudaStream_t s);
cudaError_t launch_particle_sums(int fp64, const Launch &L, double *sums, cudaStream_t s);
cudaError_t launch_rho(int order, int fp64, const Launch &L, double *rho, cudaStream_t s);
// ---- persistent batched step (k_persist.cu)
// sizes of one instance that set its work items per phase
struct PersistCounts {
    long long ncell;
    int ntiles;
    long long pencils[3];  // filter pencils per axis
    long long mx_tiles;    // fused Yee tiles
    long long ghost[3];    // periodic ghost-copy elements per axis (0: not periodic)
};
// The device work list of a batch (per-phase item offsets and the launch's counters).
class PersistPlan {
  public:
    struct Impl;
    PersistPlan();
    ~PersistPlan();
    PersistPlan(const PersistPlan &) = delete;
    PersistPlan &operator=(const PersistPlan &) = delete;
    // device memory from alloc(user, bytes), owned by the caller's context
    cudaError_t build(const std::vector<PersistCounts> &inst, void *(*alloc)(void *, size_t), void *user);
    long long items_per_step() const;
    // nsteps steps of the batch in one launch of grid CTAs (kNT threads, smem bytes of
    // dynamic shared memory); pencil_tables: the three per-axis pencil offset tables,
    // mx_start: the fused Yee tile offsets
    cudaError_t launch(const Launch &L, int ndim, int order, int nsteps, int passes, int filtered,
                       const long long *pencil_tables, const long long *mx_start, size_t smem, int grid,
                       long long spin_limit, int stall_inst, cudaStream_t s);

  private:
    Impl *impl;
};
// dynamic shared memory of the persistent kernel, and its resident CTAs per SM
size_t persist_smem(int ndim, size_t particle_smem);
cudaError_t persist_blocks_per_sm(int ndim, int order, size_t smem, int *bps);

// opt-in to the shared memory of the fused Yee update (once per device and precision)
cudaError_t prepare_fields(int fp64);
// the whole Yee update of the step (Yee solver, no antenna) in one launch over
// maxwell_tiles() tiles per instance, then the switch of every instance to the E / B
// buffer pair it wrote
cudaError_t launch_maxwell_fused(int fp64, int ndim, const Launch &L, const long long *tile_start, long long ntiles,
                                 int filtered, cudaStream_t s);
inline long long maxwell_tiles(const int n[3], int ndim)
{
    return ndim == 3 ? (long long)((n[0] + 31) / 32) * ((n[1] + 7) / 8) * ((n[2] + 31) / 32)
                     : (long long)((n[0] + 255) / 256) * ((n[2] + 31) / 32);
}
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
cudaError_t launch_ant_bterm(int fp64, int ck, const InstDev *d_inst, const InstDev &I, const AntDev &A, int damp,
                             cudaStream_t s);
cudaError_t launch_ant_eterm(int fp64, const InstDev *d_inst, const InstDev &I, const AntDev &A, cudaStream_t s);
cudaError_t launch_ant_lattice(const AntDev &A, double dt, double dz, int what, cudaStream_t s);
cudaError_t launch_ghost(int fp64, const Launch &L, int axis, long long per_inst_max, cudaStream_t s);
cudaError_t prepare_particles(int ndim, int order, int fp64, int pusher, size_t smem);
// Loads, on the current device, the no-allocation charge work grid (pic_get_rho_noalloc)
// and the density kernels that read-out launches: CUDA loads code and device arrays on
// first use, so pic_create calls this and the read-out itself never triggers a load.
cudaError_t noalloc_load_grid(int order, int fp64);
cudaError_t preload_rho(int order, int fp64);
cudaError_t preload_rho_ion();
cudaError_t launch_field_energy(int fp64, const Launch &L, double *sums, cudaStream_t s);
cudaError_t launch_pack(int fp64, const InstDev &I, int comp, int filtered, double *dense, long long ncell, cudaStream_t s);
cudaError_t launch_unpack(int fp64, const InstDev &I, int comp, const double *dense, long long ncell, cudaStream_t s);
// the same for the z planes k0 .. k0 + nk - 1 (unpack: add = 1 adds instead of writing)
cudaError_t launch_pack_planes(int fp64, const InstDev &I, int comp, int filtered, double *dense, int k0, int nk,
                               cudaStream_t s);
cudaError_t launch_unpack_planes(int fp64, const InstDev &I, int comp, const double *dense, int k0, int nk, int add,
                                 cudaStream_t s);
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
