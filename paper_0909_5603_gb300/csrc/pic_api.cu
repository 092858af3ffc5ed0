// pic_api.cu -- host side of the C ABI declared in include/pic.h: instance set-up
// (geometry, device memory through the caller's allocator, TMA descriptors), loaders,
// the step sequence (graph-captured), getters, profiling and batching.
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <thread>
#include <vector>

#include "../../include/pic.h"
#include "lab_frame.h"
#include "pic_internal.h"

using namespace pic;

namespace {

struct Block {
    void *p;
    size_t bytes;
};

constexpr int kPhases = 5;  // particles, scan, filter, maxwell, other
constexpr int kEventSteps = 1024;

}  // namespace

struct pic_ctx {
    bool is_batch = false;
    std::vector<pic_ctx *> members;
    std::vector<uint64_t> member_versions;
    // configuration
    int ndim = 3, n[3] = {1, 1, 1}, bc[3] = {0, 0, 0}, order = 1;
    double dx[3] = {1, 1, 1}, dt = 0, gamma_b = 1;
    pic_options opt{};
    int fp64 = 0;
    size_t es = 4;
    int device = 0;
    cudaStream_t stream = nullptr;
    // device views
    InstDev h{};
    InstDev *d_inst = nullptr;
    int *d_tile_start = nullptr;
    long long *d_cell_start = nullptr;
    Launch L{};
    size_t smem = 0;
    long long ncell = 0;
    FastDiv fd_ts[3] = {};  // host division by the tile extents (cell -> tile on loads)
    long long ghost_max = 0;
    bool any_periodic[3] = {false, false, false};
    int max_sweeps = 0;
    long long *d_pencil = nullptr;       // per axis: [ninst + 1] filter pencil offsets (device)
    long long pencil_total[4] = {0, 0, 0, 0};  // [3]: tiles of the fused Yee update
    std::vector<Block> blocks;
    uint64_t version = 1;  // bumps when device pointers of the instance change
    // state
    bool loaded = false;
    int64_t step = 0;
    int last_filtered = 0;
    // beam injection plane (pic_set_injection)
    bool inj_on = false;
    double inj_z = 0.0;
    int32_t inj_first = -1;          // < 0: the beam of the last lab-frame load
    int32_t beam_first_id = INT_MAX; // first beam id of the last lab-frame load (INT_MAX: none)
    // laser antenna (pic_set_laser_antenna)
    bool ant_on = false;
    AntDev ant{};
    int64_t mx_phases = 0;  // Maxwell phases since the last load
    // lab-frame stations
    int nst = 0, st_max = 0;
    double *d_st_z = nullptr, *d_st_t = nullptr;
    int *d_st_count = nullptr;
    void *d_st_fields = nullptr;
    // scratch
    double *d_dense = nullptr;   // ncell doubles (field exchange)
    double *d_sums = nullptr;    // diagnostics sums
    int *d_start = nullptr;      // ntiles + 1 read-out offsets
    int **d_start_ptr = nullptr; // device array holding d_start
    int stage_cap = 0;
    int *st_cell = nullptr, *st_id = nullptr;
    double *st_off = nullptr, *st_u = nullptr, *st_w = nullptr;
    // graph
    cudaGraphExec_t graph = nullptr;
    // persistent batched step (pic_batch_set_persistent)
    bool persistent = false;
    long long spin_limit = 0;
    int stall_inst = -1;
    PersistPlan *plan = nullptr;
    size_t persist_smem = 0;
    int persist_grid = 0;
    // profiling
    bool profiling = false;
    std::vector<cudaEvent_t> events;
    std::vector<unsigned char> recorded;  // per (slot, phase): both events recorded
    int ev_steps = 0;
    pic_timings acc{};
    std::string err;
};

static std::string g_create_error;

namespace pic {
// Read-only view of a context for entry points that live in other translation units.
bool ctx_view(pic_ctx *c, CtxView *v)
{
    if (!c || !v) return false;
    v->launch = &c->L;
    v->order = c->order;
    v->fp64 = c->fp64;
    v->ncell = c->ncell;
    v->stream = c->stream;
    v->device = c->device;
    v->loaded = c->loaded;
    v->is_batch = c->is_batch;
    return true;
}

pic_status ctx_fail(pic_ctx *c, pic_status s, const char *msg)
{
    if (c) c->err = msg;
    return s;
}
}  // namespace pic


static pic_status fail(pic_ctx *c, pic_status s, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    if (c)
        c->err = buf;
    else
        g_create_error = buf;
    return s;
}

#define CUDA_OR_FAIL(c, call)                                                                              \
    do {                                                                                                   \
        cudaError_t e_ = (call);                                                                           \
        if (e_ != cudaSuccess) return fail((c), PIC_ERR_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

static void *dalloc(pic_ctx *c, size_t bytes)
{
    bytes = (bytes + 255) & ~(size_t)255;
    if (bytes == 0) bytes = 256;
    void *p = nullptr;
    if (c->opt.alloc) {
        p = c->opt.alloc(bytes, c->opt.alloc_user);
    } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
    }
    if (p) c->blocks.push_back({p, bytes});
    return p;
}

static void dfree(pic_ctx *c, void *p)
{
    if (!p) return;
    for (size_t i = 0; i < c->blocks.size(); ++i)
        if (c->blocks[i].p == p) {
            if (c->opt.free) c->opt.free(p, c->opt.alloc_user);
            else cudaFree(p);
            c->blocks.erase(c->blocks.begin() + i);
            return;
        }
}

static void dfree_all(pic_ctx *c)
{
    for (auto &b : c->blocks) {
        if (c->opt.free) c->opt.free(b.p, c->opt.alloc_user);
        else cudaFree(b.p);
    }
    c->blocks.clear();
}

static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    }
    return fn;
}

static bool finite3(const double *v) { return std::isfinite(v[0]) && std::isfinite(v[1]) && std::isfinite(v[2]); }

// ------------------------------------------------------------------------------------
// options and creation
// ------------------------------------------------------------------------------------
extern "C" void pic_default_options(pic_options *o)
{
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->precision = PIC_PREC_FP32;
    o->pusher = PIC_PUSHER_VAY;
    o->filter_passes = 0;
    o->threads = 0;
    o->absorb_cells = 16;
    o->absorb_strength = 0.1;
    o->charge = -1.0;
    o->mass = 1.0;
    o->track_ids = 1;
    o->device = -1;
    o->absorb_faces = 0x3F;
}

extern "C" const char *pic_last_error(const pic_ctx *ctx)
{
    return ctx ? ctx->err.c_str() : g_create_error.c_str();
}

static int activeaxis(int ndim, int a) { return !(ndim == 2 && a == 1); }

// The instance's step constants in both precisions (see StepCoef), from dt, dx, q, m and
// the FP32 current scale.
static void fill_step_coef(InstDev &h)
{
    const double dV = h.dx[0] * h.dx[1] * h.dx[2];
    StepCoef<double> d;
    d.h = 0.5 * h.q / h.m * h.dt;
    d.qdv = h.q / dV;
    for (int a = 0; a < 3; ++a) {
        d.jf[a] = h.dx[a] / h.dt;
        d.dtdx[a] = h.dt / h.dx[a];
        d.inv_dx[a] = 1.0 / h.dx[a];
    }
    d.half_dt = 0.5 * h.dt;
    d.dt = h.dt;
    h.cd = d;
    StepCoef<float> f;
    f.h = (float)d.h;
    f.qdv = (float)d.qdv;
    for (int a = 0; a < 3; ++a) {
        f.jf[a] = (float)d.jf[a];
        f.dtdx[a] = (float)d.dtdx[a];
        f.inv_dx[a] = (float)d.inv_dx[a];
    }
    f.half_dt = (float)d.half_dt;
    f.dt = (float)d.dt;
    h.cf = f;
}

// The injection plane in the instance parameters: on only with a plane set; the first
// beam id is the caller's, or the last lab-frame load's beam (none: INT_MAX).
static void apply_injection(pic_ctx *c)
{
    const int32_t id0 = c->inj_first >= 0 ? c->inj_first : c->beam_first_id;
    c->h.inj_id0 = c->inj_on ? id0 : INT_MAX;
    c->h.inj_zb = c->inj_z / c->gamma_b;
}

// Removes the antenna (its lattice and counter).
static void antenna_off(pic_ctx *c)
{
    if (c->ant.ge) dfree(c, c->ant.ge);
    if (c->ant.gb) dfree(c, c->ant.gb);
    if (c->ant.n) dfree(c, c->ant.n);
    c->ant = AntDev{};
    c->ant_on = false;
}

static pic_status upload_inst(pic_ctx *c)
{
    CUDA_OR_FAIL(c, cudaMemcpyAsync(c->d_inst, &c->h, sizeof(InstDev), cudaMemcpyHostToDevice, c->stream));
    CUDA_OR_FAIL(c, cudaStreamSynchronize(c->stream));
    return PIC_OK;
}

static pic_status encode_tmaps(pic_ctx *c, CUtensorMap *maps)
{
    auto enc = tensor_map_encoder();
    if (!enc) return fail(c, PIC_ERR_CUDA, "cuTensorMapEncodeTiled is not available from the driver");
    const cuuint64_t dims[3] = {(cuuint64_t)c->h.P[0], (cuuint64_t)c->h.P[1], (cuuint64_t)c->h.P[2]};
    const cuuint64_t strides[2] = {(cuuint64_t)c->h.sy * c->es, (cuuint64_t)c->h.sz * c->es};
    const cuuint32_t box[3] = {(cuuint32_t)c->h.box[0], (cuuint32_t)c->h.box[1], (cuuint32_t)c->h.box[2]};
    const cuuint32_t estr[3] = {1, 1, 1};
    for (int comp = 0; comp < 12; ++comp) {
        const int f = comp % 6;
        void *base = comp < 6 ? (f < 3 ? c->h.E[f] : c->h.B[f - 3]) : (f < 3 ? c->h.E2[f] : c->h.B2[f - 3]);
        CUresult r = enc(&maps[comp], c->fp64 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, base,
                         dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return fail(c, PIC_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d) for component %d", (int)r, comp);
    }
    return PIC_OK;
}

extern "C" pic_status pic_create(const pic_grid *grid, const double dx[3], double dt, double gamma_boost, int shape_order,
                                 const pic_options *opt, pic_ctx **out)
{
    if (!out) return fail(nullptr, PIC_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!grid || !dx) return fail(nullptr, PIC_ERR_ARG, "grid or dx is NULL");
    if (grid->ndim != 2 && grid->ndim != 3) return fail(nullptr, PIC_ERR_ARG, "ndim must be 2 or 3");
    if (grid->ndim == 2 && grid->n[1] != 1) return fail(nullptr, PIC_ERR_ARG, "2D grids are x-z: n[1] must be 1");
    for (int a = 0; a < 3; ++a) {
        if (!activeaxis(grid->ndim, a)) continue;
        if (grid->n[a] < 8) return fail(nullptr, PIC_ERR_ARG, "n[%d] = %d: at least 8 cells per axis", a, grid->n[a]);
        if (grid->bc[a] != PIC_PERIODIC && grid->bc[a] != PIC_ABSORBING) return fail(nullptr, PIC_ERR_ARG, "bc[%d] invalid", a);
        if (!(dx[a] > 0.0) || !std::isfinite(dx[a])) return fail(nullptr, PIC_ERR_ARG, "dx[%d] must be finite and > 0", a);
    }
    if ((long long)grid->n[0] * grid->n[1] * grid->n[2] >= (1LL << 31))
        return fail(nullptr, PIC_ERR_ARG, "grid too large for int32 cell indices");
    if (shape_order != 1 && shape_order != 2) return fail(nullptr, PIC_ERR_ARG, "shape_order must be 1 or 2");
    if (!(gamma_boost >= 1.0) || !std::isfinite(gamma_boost)) return fail(nullptr, PIC_ERR_ARG, "gamma_boost must be >= 1");
    if (!(dt > 0.0) || !std::isfinite(dt)) return fail(nullptr, PIC_ERR_ARG, "dt must be finite and > 0");
    pic_options o;
    pic_default_options(&o);
    if (opt) o = *opt;
    if (o.solver != PIC_SOLVER_YEE && o.solver != PIC_SOLVER_CK) return fail(nullptr, PIC_ERR_ARG, "solver invalid");
    // Courant limit: Yee 1 / sqrt(sum_a 1/dx_a^2); the low-dispersion solver min_a dx_a
    double inv2 = 0.0, dmin = 1e300;
    for (int a = 0; a < 3; ++a)
        if (activeaxis(grid->ndim, a)) {
            inv2 += 1.0 / (dx[a] * dx[a]);
            dmin = std::min(dmin, dx[a]);
        }
    const double courant = o.solver == PIC_SOLVER_CK ? dmin : 1.0 / std::sqrt(inv2);
    if (dt > courant * (1.0 + 1e-12))
        return fail(nullptr, PIC_ERR_CFL, "dt = %g exceeds the Courant limit %g", dt, courant);
    if (o.precision != PIC_PREC_FP32 && o.precision != PIC_PREC_FP64) return fail(nullptr, PIC_ERR_ARG, "precision invalid");
    if (o.pusher != PIC_PUSHER_VAY && o.pusher != PIC_PUSHER_BORIS) return fail(nullptr, PIC_ERR_ARG, "pusher invalid");
    if (o.filter_passes < 0 || o.filter_passes > 8) return fail(nullptr, PIC_ERR_ARG, "filter_passes must be 0..8");
    if (o.threads != 0 && o.threads != particle_threads())
        return fail(nullptr, PIC_ERR_UNSUPPORTED, "threads = %d: this build runs %d threads per particle CTA", o.threads,
                    particle_threads());
    if (o.absorb_cells < 0 || !(o.absorb_strength >= 0.0 && o.absorb_strength < 1.0))
        return fail(nullptr, PIC_ERR_ARG, "absorbing layer parameters out of range");
    if (!(o.mass > 0.0) || !std::isfinite(o.charge)) return fail(nullptr, PIC_ERR_ARG, "species charge/mass invalid");
    if ((o.alloc == nullptr) != (o.free == nullptr)) return fail(nullptr, PIC_ERR_ARG, "alloc and free must be given together");

    pic_ctx *c = new pic_ctx();
    c->ndim = grid->ndim;
    c->order = shape_order;
    c->dt = dt;
    c->gamma_b = gamma_boost;
    c->opt = o;
    c->fp64 = o.precision == PIC_PREC_FP64;
    c->es = c->fp64 ? 8 : 4;
    c->stream = (cudaStream_t)o.stream;
    if (o.device >= 0) {
        if (cudaSetDevice(o.device) != cudaSuccess) {
            delete c;
            return fail(nullptr, PIC_ERR_CUDA, "cudaSetDevice(%d) failed", o.device);
        }
    }
    cudaGetDevice(&c->device);
    for (int a = 0; a < 3; ++a) {
        c->n[a] = grid->n[a];
        c->bc[a] = activeaxis(grid->ndim, a) ? grid->bc[a] : PIC_PERIODIC;
        c->dx[a] = dx[a];
    }
    InstDev &h = c->h;
    std::memset(&h, 0, sizeof(h));
    h.ndim = c->ndim;
    int ts[3] = {o.tile[0], o.tile[1], o.tile[2]};
    for (int a = 0; a < 3; ++a) {
        h.n[a] = c->n[a];
        h.bc[a] = c->bc[a];
        // x carries one extra ghost layer so the gather box can start one cell before the
        // tile on a 16-byte boundary (TMA)
        h.gh[a] = activeaxis(c->ndim, a) ? kGhost + (a == 0 ? 1 : 0) : 0;
        if (ts[a] <= 0) ts[a] = c->ndim == 3 ? 8 : 16;
        if (!activeaxis(c->ndim, a)) ts[a] = 1;
        h.ts[a] = ts[a];
        h.nt[a] = (c->n[a] + ts[a] - 1) / ts[a];
        h.dx[a] = dx[a];
        if (activeaxis(c->ndim, a) && c->bc[a] == PIC_PERIODIC) c->any_periodic[a] = true;
    }
    if (ts[0] % 4 != 0) {
        delete c;
        return fail(nullptr, PIC_ERR_ARG, "tile[0] = %d must be a multiple of 4", ts[0]);
    }
    for (int a = 0; a < 3; ++a)
        if (activeaxis(c->ndim, a) && ts[a] > 64) {
            delete c;
            return fail(nullptr, PIC_ERR_ARG, "tile[%d] = %d: at most 64", a, ts[a]);
        }
    h.P[0] = ((c->n[0] + 2 * h.gh[0]) + 3) / 4 * 4;
    h.P[1] = c->n[1] + 2 * h.gh[1];
    h.P[2] = c->n[2] + 2 * h.gh[2];
    h.sy = h.P[0];
    h.sz = (long long)h.P[0] * h.P[1];
    h.cstride = (h.sz * h.P[2] + 63) / 64 * 64;  // 256/512-byte aligned component arrays
    h.ntiles = h.nt[0] * h.nt[1] * h.nt[2];
    h.tile_base = 0;
    h.R = particle_chunk();
    h.filter_passes = o.filter_passes;
    h.solver = o.solver;
    h.absorb_cells = o.absorb_cells;
    h.absorb_strength = o.absorb_strength;
    h.dt = dt;
    h.gb = gamma_boost;
    h.beta_b = std::sqrt(1.0 - 1.0 / (gamma_boost * gamma_boost));
    h.inj_id0 = INT_MAX;
    h.q = o.charge;
    h.m = o.mass;
    fill_step_coef(h);
    // gather box (tile + guard) and J tile geometry; the box starts one cell before the
    // tile (padded x coordinate T0 + 4, 16-byte aligned) and its x extent is a multiple of
    // 16 bytes
    const int xal = c->fp64 ? 2 : 4;
    const int hi = shape_order == 2 ? 2 : 1;
    h.box_lo[0] = -1;
    h.box[0] = ((1 + ts[0] + hi) + xal - 1) / xal * xal;
    for (int a = 1; a < 3; ++a) {
        if (activeaxis(c->ndim, a)) {
            h.box_lo[a] = -1;
            h.box[a] = 1 + ts[a] + hi;
        } else {
            h.box_lo[a] = 0;
            h.box[a] = 1;
        }
    }
    h.div_n0 = make_fastdiv(c->n[0]);
    h.div_n1 = make_fastdiv(c->n[1]);
    for (int a = 0; a < 3; ++a) c->fd_ts[a] = make_fastdiv(h.ts[a]);
    h.jlo = -shape_order;
    for (int a = 0; a < 3; ++a) h.jdim[a] = activeaxis(c->ndim, a) ? ts[a] + (shape_order == 2 ? 5 : 3) : 1;
    const size_t boxb = ((size_t)h.box[0] * h.box[1] * h.box[2] * c->es + 127) / 128 * 128;
    // 6 field boxes + the J tile at 8 bytes per cell and component (FP64 values, or the
    // 32-bit chunk accumulator and the FP32 tile in FP32 mode; each component rounded up to
    // a multiple of 4 entries) + alignment slack
    c->smem = 128 + 6 * boxb + 3 * (((size_t)h.jdim[0] * h.jdim[1] * h.jdim[2] + 3) / 4 * 4) * 8;
    if (c->smem > 200 * 1024) {
        const size_t smem = c->smem;
        delete c;
        return fail(nullptr, PIC_ERR_ARG, "tile too large: %zu bytes of shared memory per CTA", smem);
    }
    c->ncell = (long long)c->n[0] * c->n[1] * c->n[2];
    {
        long long gm = 0;
        for (int a = 0; a < 3; ++a) {
            const int o1 = a == 0 ? 1 : 0, o2 = a == 2 ? 1 : 2;
            gm = std::max(gm, 6LL * 2 * h.gh[a] * h.P[o1] * h.P[o2]);
        }
        c->ghost_max = gm;
    }
    c->max_sweeps = o.filter_passes * (c->ndim == 3 ? 3 : 2);

    // device memory: 18 field components (E, B, J, J scratch, the second E and B),
    // bookkeeping, scratch
    const size_t fbytes = 18 * (size_t)h.cstride * c->es;
    unsigned char *F = (unsigned char *)dalloc(c, fbytes);
    int *small = (int *)dalloc(c, 4096);
    int nt1 = h.ntiles + 1;
    int *tiles = (int *)dalloc(c, sizeof(int) * (size_t)(4 * nt1 + 2 * h.ntiles * kBuckets + h.ntiles + 64));
    CUtensorMap *tm = (CUtensorMap *)dalloc(c, 12 * sizeof(CUtensorMap));
    c->d_inst = (InstDev *)dalloc(c, sizeof(InstDev));
    c->d_tile_start = (int *)dalloc(c, 2 * sizeof(int));
    c->d_cell_start = (long long *)dalloc(c, 2 * sizeof(long long));
    c->d_dense = (double *)dalloc(c, sizeof(double) * (size_t)c->ncell);
    c->d_sums = (double *)dalloc(c, 64 * sizeof(double));
    c->d_start = (int *)dalloc(c, sizeof(int) * (size_t)nt1);
    c->d_start_ptr = (int **)dalloc(c, sizeof(int *));
    c->d_pencil = (long long *)dalloc(c, 8 * sizeof(long long));
    h.ion_face = dalloc(c, sizeof(double) * (size_t)c->n[2]);
    h.srcrec = (int *)dalloc(c, sizeof(int) * (size_t)h.ntiles * kSrcRec);
    if (!F || !small || !tiles || !tm || !c->d_inst || !c->d_tile_start || !c->d_cell_start || !c->d_dense || !c->d_sums ||
        !c->d_start || !c->d_start_ptr || !c->d_pencil || !h.ion_face || !h.srcrec) {
        dfree_all(c);
        delete c;
        return fail(nullptr, PIC_ERR_OOM, "device allocation failed (%zu bytes of fields)", fbytes);
    }
    for (int a = 0; a < 3; ++a) {
        h.E[a] = F + (size_t)(0 + a) * h.cstride * c->es;
        h.B[a] = F + (size_t)(3 + a) * h.cstride * c->es;
        h.J[a] = F + (size_t)(6 + a) * h.cstride * c->es;
        h.Jt[a] = F + (size_t)(9 + a) * h.cstride * c->es;
        h.E2[a] = F + (size_t)(12 + a) * h.cstride * c->es;
        h.B2[a] = F + (size_t)(15 + a) * h.cstride * c->es;
    }
    h.cur = small;
    h.err = small + 1;
    h.live = small + 2;
    h.jsel = small + 3;
    h.lost = (unsigned long long *)(small + 4);
    h.phase = small + 6;
    h.fpar = small + 8;
    h.seg[0] = tiles;
    h.seg[1] = tiles + nt1;
    h.chunk_base[0] = tiles + 2 * nt1;
    h.chunk_base[1] = tiles + 3 * nt1;
    h.tot[0] = tiles + 4 * nt1;
    h.tot[1] = tiles + 4 * nt1 + h.ntiles * kBuckets;
    h.pop = tiles + 4 * nt1 + 2 * h.ntiles * kBuckets;
    h.tmap = tm;

    // absorbing-layer factors per axis: 1 - s (d/L)^2 at depth d = max(0, L - i, i - (n-1-L)),
    // evaluated in FP64 and stored in the working precision
    for (int a = 0; a < 3; ++a) {
        h.damp[a] = nullptr;
        if (!activeaxis(c->ndim, a) || c->bc[a] != PIC_ABSORBING || o.absorb_cells <= 0) continue;
        std::vector<double> f(c->n[a]);
        const int L = o.absorb_cells;
        const bool lo = (o.absorb_faces >> (2 * a)) & 1, hi = (o.absorb_faces >> (2 * a + 1)) & 1;
        for (int i = 0; i < c->n[a]; ++i) {
            int d = 0;
            if (lo && L - i > d) d = L - i;
            if (hi && i - (c->n[a] - 1 - L) > d) d = i - (c->n[a] - 1 - L);
            const double r = (double)d / (double)L;
            f[i] = 1.0 - o.absorb_strength * r * r;
        }
        void *tab = dalloc(c, c->es * (size_t)c->n[a]);
        if (!tab) {
            dfree_all(c);
            delete c;
            return fail(nullptr, PIC_ERR_OOM, "absorbing-layer table allocation failed");
        }
        std::vector<float> f32(f.begin(), f.end());
        const void *src = c->fp64 ? (const void *)f.data() : (const void *)f32.data();
        if (cudaMemcpyAsync(tab, src, c->es * (size_t)c->n[a], cudaMemcpyHostToDevice, c->stream) != cudaSuccess ||
            cudaStreamSynchronize(c->stream) != cudaSuccess) {
            dfree_all(c);
            delete c;
            return fail(nullptr, PIC_ERR_CUDA, "absorbing-layer table upload failed");
        }
        h.damp[a] = tab;
    }

    pic_status st = PIC_OK;
    CUtensorMap maps[12];
    if ((st = encode_tmaps(c, maps)) != PIC_OK) {
        std::string e = c->err;
        dfree_all(c);
        delete c;
        return fail(nullptr, st, "%s", e.c_str());
    }
    long long pencils[8];
    for (int a = 0; a < 4; ++a) {
        c->pencil_total[a] = a == 3 ? maxwell_tiles(c->n, c->ndim) : o.filter_passes > 0 ? filter_pencils(c->n, c->ndim, a) : 0;
        pencils[2 * a] = 0;
        pencils[2 * a + 1] = c->pencil_total[a];
    }
    const int tstart[2] = {0, h.ntiles};
    const long long cstart[2] = {0, c->ncell};
    int *dptr_start = c->d_start;
    bool okc = cudaMemsetAsync(F, 0, fbytes, c->stream) == cudaSuccess && cudaMemsetAsync(small, 0, 4096, c->stream) == cudaSuccess &&
               cudaMemsetAsync(tiles, 0, sizeof(int) * (size_t)(4 * nt1 + 2 * h.ntiles * kBuckets + h.ntiles), c->stream) == cudaSuccess &&
               cudaMemcpyAsync(tm, maps, sizeof(maps), cudaMemcpyHostToDevice, c->stream) == cudaSuccess &&
               cudaMemcpyAsync(c->d_tile_start, tstart, sizeof(tstart), cudaMemcpyHostToDevice, c->stream) == cudaSuccess &&
               cudaMemcpyAsync(c->d_cell_start, cstart, sizeof(cstart), cudaMemcpyHostToDevice, c->stream) == cudaSuccess &&
               cudaMemcpyAsync(c->d_start_ptr, &dptr_start, sizeof(int *), cudaMemcpyHostToDevice, c->stream) == cudaSuccess &&
               cudaMemcpyAsync(c->d_pencil, pencils, sizeof(pencils), cudaMemcpyHostToDevice, c->stream) == cudaSuccess &&
               prepare_particles(c->ndim, c->order, c->fp64, o.pusher, c->smem) == cudaSuccess &&
               prepare_fields(c->fp64) == cudaSuccess &&
               noalloc_load_grid(c->order, c->fp64) == cudaSuccess;
    if (!okc || upload_inst(c) != PIC_OK) {
        cudaError_t e = cudaGetLastError();
        dfree_all(c);
        delete c;
        return fail(nullptr, PIC_ERR_CUDA, "device set-up failed: %s", cudaGetErrorString(e));
    }
    c->L.inst = c->d_inst;
    c->L.tile_start = c->d_tile_start;
    c->L.cell_start = c->d_cell_start;
    c->L.ninst = 1;
    c->L.total_tiles = h.ntiles;
    c->L.total_cells = c->ncell;
    *out = c;
    return PIC_OK;
}

static void destroy_graph(pic_ctx *c)
{
    if (c->graph) {
        cudaGraphExecDestroy(c->graph);
        c->graph = nullptr;
    }
}

extern "C" void pic_destroy(pic_ctx *ctx)
{
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    destroy_graph(ctx);
    for (auto e : ctx->events) cudaEventDestroy(e);
    dfree_all(ctx);
    delete ctx->plan;
    delete ctx;
}

// ------------------------------------------------------------------------------------
// particle loading: host stable sort by tile, then the initial layout (every tile's
// particles in its own "stay" bucket, chunks of R particles)
// ------------------------------------------------------------------------------------
static pic_status ensure_particle_capacity(pic_ctx *c, int64_t n)
{
    InstDev &h = c->h;
    const int want = (int)std::max<int64_t>(n, 1);
    if (h.cell[0] && h.cap >= want) return PIC_OK;
    for (int b = 0; b < 2; ++b) {
        dfree(c, h.cell[b]);
        dfree(c, h.chunk_pre[b]);
        dfree(c, h.chunk_cb[b]);
        h.cell[b] = nullptr;
        h.chunk_pre[b] = h.chunk_cb[b] = nullptr;
        h.id[b] = nullptr;
    }
    const int cap = want;
    const int chunk_cap = h.ntiles + cap / h.R + 2;
    const int nreal = c->ndim == 3 ? 7 : 6;  // offsets (3 or 2), momenta 3, weight
    for (int b = 0; b < 2; ++b) {
        const size_t per = (size_t)cap;
        unsigned char *blk = (unsigned char *)dalloc(c, per * (sizeof(int) * 2) + per * nreal * c->es + 4096);
        int *cb = (int *)dalloc(c, sizeof(int) * (size_t)chunk_cap * kPre);
        int *cbb = (int *)dalloc(c, sizeof(int) * (size_t)chunk_cap * kBuckets);
        if (!blk || !cb || !cbb) return fail(c, PIC_ERR_OOM, "particle buffers (%d particles) do not fit", cap);
        size_t off = 0;
        auto take = [&](size_t bytes) {
            void *p = blk + off;
            off += (bytes + 255) & ~(size_t)255;
            return p;
        };
        h.cell[b] = (int *)blk;
        off = ((per * sizeof(int)) + 255) & ~(size_t)255;
        h.id[b] = c->opt.track_ids ? (int *)take(per * sizeof(int)) : nullptr;
        h.off[b][0] = take(per * c->es);
        h.off[b][1] = c->ndim == 3 ? take(per * c->es) : nullptr;
        h.off[b][2] = take(per * c->es);
        for (int a = 0; a < 3; ++a) h.u[b][a] = take(per * c->es);
        h.w[b] = take(per * c->es);
        h.chunk_pre[b] = cb;
        h.chunk_cb[b] = cbb;
    }
    h.cap = cap;
    h.chunk_cap = chunk_cap;
    c->stage_cap = 0;  // staging is re-sized lazily
    c->version++;
    return PIC_OK;
}

// Tile of a cell index (linear, x fastest).
// Host loops over many particles: fn(t, begin, end) on T threads over contiguous ranges
// of [0, n) in order (T = 1 below 2^18 items).
static int host_workers(int64_t n)
{
    if (n < (1 << 18)) return 1;
    const unsigned hw = std::thread::hardware_concurrency();
    return (int)std::max(1u, std::min(hw ? hw : 1u, 16u));
}

template <typename F>
static void parallel_ranges(int64_t n, int T, F fn)
{
    if (T <= 1) {
        fn(0, (int64_t)0, n);
        return;
    }
    std::vector<std::thread> th;
    th.reserve(T);
    for (int t = 0; t < T; ++t) th.emplace_back(fn, t, n * t / T, n * (t + 1) / T);
    for (auto &x : th) x.join();
}

// The first n floats of the n-double array d, widened to doubles in place.  The doubles
// [lo, hi) read floats [lo, hi) and write the bytes of floats [2 lo, 2 hi); with
// lo = ceil(hi / 2) those lie at or above hi, where every float has been read already,
// so each such range runs in parallel and the ranges go from the top down.
static void widen_in_place(double *d, size_t n)
{
    const float *f = reinterpret_cast<const float *>(d);
    size_t hi = n;
    while (hi > 1) {
        const size_t lo = (hi + 1) / 2;
        const int T = host_workers((int64_t)(hi - lo));
        parallel_ranges((int64_t)(hi - lo), T, [&](int, int64_t b, int64_t e) {
            for (int64_t j = (int64_t)lo + b; j < (int64_t)lo + e; ++j) d[j] = (double)f[j];
        });
        hi = lo;
    }
    if (hi == 1) {
        const float v = f[0];
        d[0] = (double)v;
    }
}

// Tile of a valid cell index (0 <= cell < ncell), by multiply-shift divisions: the loads
// and read-outs map tens of millions of particles with it.
static int tile_of_cell(const pic_ctx *c, int cell)
{
    const InstDev &h = c->h;
    const int cyz = fast_div(cell, h.div_n0);
    const int ci = cell - cyz * c->n[0];
    const int ck = fast_div(cyz, h.div_n1);
    const int cj = cyz - ck * c->n[1];
    return fast_div(ci, c->fd_ts[0]) + h.nt[0] * (fast_div(cj, c->fd_ts[1]) + h.nt[1] * fast_div(ck, c->fd_ts[2]));
}

// Device scratch for a load, released when it goes out of scope.
struct LoadScratch {
    pic_ctx *c;
    std::vector<void *> ps;
    void *get(size_t bytes)
    {
        void *p = dalloc(c, bytes);
        if (p) ps.push_back(p);
        return p;
    }
    ~LoadScratch()
    {
        for (void *p : ps) dfree(c, p);
    }
};

// Uploads n particles (host arrays, any order; values FP64, or FP32 when f32 is set) with
// their canonical slots and places them on the device in the storage precision (k_place).
static pic_status place_from_host(pic_ctx *c, int64_t n, const int32_t *cell, const void *off, const void *u,
                                  const void *w, const int32_t *id, long long id_base, const std::vector<int> &slot,
                                  bool f32 = false)
{
    if (n <= 0) return PIC_OK;
    const size_t vs = f32 ? sizeof(float) : sizeof(double);
    LoadScratch S{c, {}};
    int *d_cell = (int *)S.get(sizeof(int) * n), *d_slot = (int *)S.get(sizeof(int) * n);
    void *d_off = S.get(vs * 3 * n), *d_u = S.get(vs * 3 * n), *d_w = S.get(vs * n);
    int *d_id = id ? (int *)S.get(sizeof(int) * n) : nullptr;
    if (!d_cell || !d_slot || !d_off || !d_u || !d_w || (id && !d_id))
        return fail(c, PIC_ERR_OOM, "no device memory to stage %lld particles", (long long)n);
    CUDA_OR_FAIL(c, cudaMemcpyAsync(d_cell, cell, sizeof(int) * n, cudaMemcpyHostToDevice, c->stream));
    CUDA_OR_FAIL(c, cudaMemcpyAsync(d_slot, slot.data(), sizeof(int) * n, cudaMemcpyHostToDevice, c->stream));
    CUDA_OR_FAIL(c, cudaMemcpyAsync(d_off, off, vs * 3 * n, cudaMemcpyHostToDevice, c->stream));
    CUDA_OR_FAIL(c, cudaMemcpyAsync(d_u, u, vs * 3 * n, cudaMemcpyHostToDevice, c->stream));
    CUDA_OR_FAIL(c, cudaMemcpyAsync(d_w, w, vs * n, cudaMemcpyHostToDevice, c->stream));
    if (id) CUDA_OR_FAIL(c, cudaMemcpyAsync(d_id, id, sizeof(int) * n, cudaMemcpyHostToDevice, c->stream));
    PlaceSrc src{d_cell, d_off, d_u, d_w, d_id, d_slot, (long long)n, id_base, f32 ? 1 : 0};
    CUDA_OR_FAIL(c, launch_place(c->fp64, c->h, src, c->stream));
    CUDA_OR_FAIL(c, cudaStreamSynchronize(c->stream));  // before the scratch is released
    return PIC_OK;
}

// After the particles are in place: the initial tile layout (every tile's particles in
// its own segment, all in the "stays" bucket) in layout 0.
static pic_status upload_layout(pic_ctx *c, const std::vector<int> &seg)
{
    InstDev &h = c->h;
    const int R = h.R;
    std::vector<int> cbase(h.ntiles + 1, 0), tot((size_t)h.ntiles * kBuckets, 0), pop(h.ntiles, 0);
    for (int t = 0; t < h.ntiles; ++t) {
        const int m = seg[t + 1] - seg[t];
        cbase[t + 1] = cbase[t] + (m + R - 1) / R;
        tot[(size_t)t * kBuckets + kCenterDir] = m;
        pop[t] = m;
    }
    const int nchunks = cbase[h.ntiles];
    if (nchunks > h.chunk_cap) return fail(c, PIC_ERR_INTERNAL, "chunk capacity");
    std::vector<int> pre((size_t)std::max(nchunks, 1) * kPre, 0), cbv((size_t)std::max(nchunks, 1) * kBuckets, 0);
    for (int t = 0; t < h.ntiles; ++t) {
        const int m = seg[t + 1] - seg[t];
        for (int k = 0; k < cbase[t + 1] - cbase[t]; ++k) {
            const int cc = cbase[t] + k;
            const int sz = std::min(R, m - k * R);
            for (int d = 0; d <= kBuckets; ++d) pre[(size_t)cc * kPre + d] = d <= kCenterDir ? 0 : sz;
            cbv[(size_t)cc * kBuckets + kCenterDir] = k * R;
        }
    }
    // every copy and reset goes on the context's stream (which need not synchronise with
    // the legacy default stream) and completes before this function returns
    cudaStream_t s = c->stream;
    CUDA_OR_FAIL(c, cudaMemcpyAsync(h.seg[0], seg.data(), sizeof(int) * (h.ntiles + 1), cudaMemcpyHostToDevice, s));
    CUDA_OR_FAIL(c, cudaMemcpyAsync(h.chunk_base[0], cbase.data(), sizeof(int) * (h.ntiles + 1), cudaMemcpyHostToDevice, s));
    CUDA_OR_FAIL(c, cudaMemcpyAsync(h.tot[0], tot.data(), sizeof(int) * tot.size(), cudaMemcpyHostToDevice, s));
    CUDA_OR_FAIL(c, cudaMemcpyAsync(h.pop, pop.data(), sizeof(int) * pop.size(), cudaMemcpyHostToDevice, s));
    CUDA_OR_FAIL(c, cudaMemcpyAsync(h.chunk_pre[0], pre.data(), sizeof(int) * pre.size(), cudaMemcpyHostToDevice, s));
    CUDA_OR_FAIL(c, cudaMemcpyAsync(h.chunk_cb[0], cbv.data(), sizeof(int) * cbv.size(), cudaMemcpyHostToDevice, s));
    return PIC_OK;
}

// A load: the layout and a reset of the step state.
static pic_status finish_load(pic_ctx *c, const std::vector<int> &seg)
{
    InstDev &h = c->h;
    cudaStream_t s = c->stream;
    pic_status st0 = upload_layout(c, seg);
    if (st0 != PIC_OK) return st0;
    fill_step_coef(h);
    apply_injection(c);
    antenna_off(c);  // a load removes the antenna
    c->mx_phases = 0;
    // cur, err, live, jsel, lost and the particle-phase counter
    CUDA_OR_FAIL(c, cudaMemsetAsync(h.cur, 0, 16 + sizeof(unsigned long long) + sizeof(int), s));
    CUDA_OR_FAIL(c, cudaMemsetAsync(h.J[0], 0, 3 * (size_t)h.cstride * c->es, s));
    c->loaded = true;
    c->version++;  // a batch holding this instance re-reads its parameters
    c->step = 0;
    c->last_filtered = 0;
    destroy_graph(c);
    pic_status st = upload_inst(c);
    if (st != PIC_OK) return st;
    if (c->nst == 0) {
        CUDA_OR_FAIL(c, cudaStreamSynchronize(s));
        return PIC_OK;
    }
    // stations start a new history with the loaded state as its first record
    CUDA_OR_FAIL(c, cudaMemsetAsync(c->d_st_count, 0, sizeof(int) * c->nst, s));
    StationDev S{c->d_st_z, c->d_st_count, c->d_st_t, c->d_st_fields, c->st_max};
    CUDA_OR_FAIL(c, launch_stations(c->fp64, c->d_inst, S, c->nst, c->n[0] * c->n[1], c->stream));
    CUDA_OR_FAIL(c, cudaStreamSynchronize(c->stream));
    return PIC_OK;
}

// Host particles (FP64, any order): validated, laid out in the canonical order with a
// stable counting sort by tile on the host, then converted and placed on the device.
// A new particle set that continues the run (pic_extract_particles, pic_add_particles):
// the layout, the parity word pointing at it; the step count, phase counter, lost count,
// ion background, antenna, injection plane and stations are kept.
static pic_status finish_relayout(pic_ctx *c, const std::vector<int> &seg)
{
    pic_status st = upload_layout(c, seg);
    if (st != PIC_OK) return st;
    CUDA_OR_FAIL(c, cudaMemsetAsync(c->h.cur, 0, sizeof(int), c->stream));
    c->version++;  // a batch holding this instance re-reads its parameters
    destroy_graph(c);
    if ((st = upload_inst(c)) != PIC_OK) return st;
    CUDA_OR_FAIL(c, cudaStreamSynchronize(c->stream));
    return PIC_OK;
}

// The first invalid particle of [b, e) (kind 1: cell, 2: offset, 3: momentum or weight),
// or -1; values of type V.
template <typename V>
static int64_t first_invalid(const pic_ctx *c, const int32_t *cell, const V *off, const V *u, const V *w, int64_t b,
                             int64_t e, int &kind)
{
    for (int64_t p = b; p < e; ++p) {
        kind = 0;
        if (cell[p] < 0 || cell[p] >= c->ncell) kind = 1;
        for (int a = 0; a < 3 && !kind; ++a) {
            if (!activeaxis(c->ndim, a)) continue;
            const V o = off[3 * p + a];
            if (!(o >= V(0) && o < V(1))) kind = 2;
        }
        if (!kind && !(std::isfinite(u[3 * p]) && std::isfinite(u[3 * p + 1]) && std::isfinite(u[3 * p + 2]) &&
                       std::isfinite(w[p])))
            kind = 3;
        if (kind) return p;
    }
    return -1;
}

static pic_status load_internal(pic_ctx *c, int64_t n, const int32_t *cell, const void *offv, const void *uv,
                                const void *wv, const int32_t *id, bool keep_state = false, bool f32 = false)
{
    InstDev &h = c->h;
    if (n < 0 || n >= (1LL << 31) - 1) return fail(c, PIC_ERR_ARG, "particle count %lld out of range", (long long)n);
    if (n > 0 && (!cell || !offv || !uv || !wv)) return fail(c, PIC_ERR_ARG, "particle arrays must not be NULL");
    // validation and a stable counting sort by tile id, on T host threads over contiguous
    // ranges: each range finds its first invalid particle (the lowest over the ranges is
    // the one reported) and its tile histogram; slots are then assigned
    // range by range in order, which keeps the sort stable
    const int T = host_workers(n);
    std::vector<int64_t> bad(T, INT64_MAX);
    std::vector<int> bad_kind(T, 0);
    std::vector<std::vector<int>> hist(T);
    std::vector<int> seg(h.ntiles + 1, 0), slot(n > 0 ? n : 1);
    parallel_ranges(n, T, [&](int t, int64_t b, int64_t e) {
        std::vector<int> &hc = hist[t];
        hc.assign(h.ntiles, 0);
        // blocks of particles: checked, then their tiles counted while still in cache
        constexpr int64_t kBlock = 4096;
        for (int64_t b0 = b; b0 < e; b0 += kBlock) {
            const int64_t e0 = std::min(e, b0 + kBlock);
            int kind = 0;
            const int64_t p = f32 ? first_invalid(c, cell, (const float *)offv, (const float *)uv, (const float *)wv, b0, e0, kind)
                                  : first_invalid(c, cell, (const double *)offv, (const double *)uv, (const double *)wv, b0, e0, kind);
            if (p >= 0) {
                bad[t] = p;
                bad_kind[t] = kind;
                return;
            }
            for (int64_t q = b0; q < e0; ++q) {
                slot[q] = tile_of_cell(c, cell[q]);
                hc[slot[q]]++;
            }
        }
    });
    int first = 0;
    for (int t = 1; t < T; ++t)
        if (bad[t] < bad[first]) first = t;
    if (bad[first] != INT64_MAX) {
        const int64_t p = bad[first];
        if (bad_kind[first] == 1) return fail(c, PIC_ERR_ARG, "particle %lld: cell %d outside the grid", (long long)p, cell[p]);
        if (bad_kind[first] == 2) {
            for (int a = 0; a < 3; ++a) {
                const double o = f32 ? (double)((const float *)offv)[3 * p + a] : ((const double *)offv)[3 * p + a];
                if (activeaxis(c->ndim, a) && !(o >= 0.0 && o < 1.0))
                    return fail(c, PIC_ERR_ARG, "particle %lld: offset %g outside [0,1)", (long long)p, o);
            }
        }
        return fail(c, PIC_ERR_NAN, "particle %lld: non-finite momentum or weight", (long long)p);
    }
    // segment starts, then each range's first slot in each tile
    for (int t = 0; t < T; ++t)
        for (int k = 0; k < h.ntiles; ++k) seg[k + 1] += hist[t][k];
    for (int k = 0; k < h.ntiles; ++k) seg[k + 1] += seg[k];
    {
        std::vector<int> fill(seg.begin(), seg.end() - 1);
        for (int t = 0; t < T; ++t)
            for (int k = 0; k < h.ntiles; ++k) {
                const int m = hist[t][k];
                hist[t][k] = fill[k];
                fill[k] += m;
            }
    }
    parallel_ranges(n, T, [&](int t, int64_t b, int64_t e) {
        std::vector<int> &f = hist[t];
        for (int64_t p = b; p < e; ++p) slot[p] = f[slot[p]]++;
    });
    pic_status st = ensure_particle_capacity(c, n);
    if (st != PIC_OK) return st;
    if ((st = place_from_host(c, n, cell, offv, uv, wv, id, 0, slot, f32)) != PIC_OK) return st;
    return keep_state ? finish_relayout(c, seg) : finish_load(c, seg);
}

extern "C" pic_status pic_load_particles(pic_ctx *ctx, int64_t n, const int32_t *cell, const double *off3, const double *u3,
                                         const double *w, const int32_t *id)
{
    if (!ctx) return PIC_ERR_ARG;
    if (ctx->is_batch) return fail(ctx, PIC_ERR_ARG, "pic_load_particles on a batch");
    cudaSetDevice(ctx->device);
    CUDA_OR_FAIL(ctx, cudaStreamSynchronize(ctx->stream));
    ctx->h.ion = 0;  // particles loaded directly carry no ion background
    ctx->beam_first_id = INT_MAX;
    return load_internal(ctx, n, cell, off3, u3, w, id);
}

extern "C" pic_status pic_load_particles_stored(pic_ctx *ctx, int64_t n, const int32_t *cell, const void *off3,
                                                const void *u3, const void *w, const int32_t *id)
{
    if (!ctx) return PIC_ERR_ARG;
    if (ctx->is_batch) return fail(ctx, PIC_ERR_ARG, "pic_load_particles_stored on a batch");
    cudaSetDevice(ctx->device);
    CUDA_OR_FAIL(ctx, cudaStreamSynchronize(ctx->stream));
    ctx->h.ion = 0;
    ctx->beam_first_id = INT_MAX;
    return load_internal(ctx, n, cell, off3, u3, w, id, false, !ctx->fp64);
}

extern "C" pic_status pic_set_laser_antenna(pic_ctx *ctx, const pic_laser_lab *laser, double z_lab)
{
    if (!ctx) return PIC_ERR_ARG;
    if (ctx->is_batch) return fail(ctx, PIC_ERR_ARG, "pic_set_laser_antenna on a batch");
    if (laser && !(laser->lambda0 > 0 && laser->waist > 0 && laser->duration > 0 && std::isfinite(laser->a0) &&
                   std::isfinite(laser->z_center) && std::isfinite(z_lab)))
        return fail(ctx, PIC_ERR_ARG, "antenna laser parameters or plane invalid");
    if (laser && ctx->bc[2] != 1) return fail(ctx, PIC_ERR_ARG, "the laser antenna needs an absorbing z axis");
    if (!ctx->loaded) return fail(ctx, PIC_ERR_STATE, "pic_set_laser_antenna before any load");
    cudaSetDevice(ctx->device);
    CUDA_OR_FAIL(ctx, cudaStreamSynchronize(ctx->stream));
    antenna_off(ctx);
    destroy_graph(ctx);  // the Maxwell phase changes
    ctx->version++;      // a batch holding this instance re-reads its parameters
    if (!laser) return PIC_OK;
    // the boosted pulse, as for the loaded laser: lengths x gamma_b (1 + beta_b)
    const double gb = ctx->gamma_b, b = std::sqrt(1.0 - 1.0 / (gb * gb)), doppler = gb * (1.0 + b);
    const double kp = 6.283185307179586 / (laser->lambda0 * doppler), Lp = laser->duration * doppler;
    const double zc = laser->z_center * doppler, amp = laser->a0 * kp, dz = ctx->dx[2];
    AntDev A{};
    A.zb = z_lab / gb;
    A.beta = b;
    A.t0 = (double)ctx->mx_phases * ctx->dt;
    A.w0 = laser->waist;
    A.xc = 0.5 * ctx->n[0] * ctx->dx[0];
    A.yc = 0.5 * ctx->n[1] * ctx->dx[1];
    // lattice: from below the pulse's tail (5 L') and the grid to beyond the grid by the
    // distance light covers while the plane is still in the box (no echo of the lattice's
    // end reaches the box meanwhile)
    const double zp0 = (A.zb - A.beta * A.t0) / dz;
    double lo = std::floor((zc + A.t0 - 5.0 * Lp) / dz) - 2.0;
    if (lo > 0.0) lo = 0.0;
    const double top = std::max((double)ctx->n[2], std::ceil(zp0) + 2.0);
    const double stay = zp0 > -1.0 && b > 0.0 ? (zp0 + 1.0) / b : 0.0;
    const double hi = top + std::ceil(stay) + 8.0;
    if (!(hi - lo < 1e8)) return fail(ctx, PIC_ERR_ARG, "antenna lattice of %g nodes too long", hi - lo);
    A.lo = (long long)lo;
    A.na = (long long)(hi - lo) + 1;
    std::vector<double> ge((size_t)A.na), gbv((size_t)A.na);
    for (long long a = 0; a < A.na; ++a) {
        const double ue = (A.lo + a) * dz - A.t0 - zc, ub = (A.lo + a + 0.5) * dz - A.t0 - zc;
        ge[a] = amp * std::exp(-(ue / Lp) * (ue / Lp)) * std::cos(kp * ue);
        gbv[a] = amp * std::exp(-(ub / Lp) * (ub / Lp)) * std::cos(kp * ub);
    }
    A.ge = (double *)dalloc(ctx, sizeof(double) * (size_t)A.na);
    A.gb = (double *)dalloc(ctx, sizeof(double) * (size_t)A.na);
    A.n = (int *)dalloc(ctx, sizeof(int));
    ctx->ant = A;  // owned from here (antenna_off frees what was allocated)
    if (!A.ge || !A.gb || !A.n) {
        antenna_off(ctx);
        return fail(ctx, PIC_ERR_OOM, "no device memory for the antenna lattice");
    }
    cudaStream_t s = ctx->stream;
    CUDA_OR_FAIL(ctx, cudaMemcpyAsync(A.ge, ge.data(), sizeof(double) * ge.size(), cudaMemcpyHostToDevice, s));
    CUDA_OR_FAIL(ctx, cudaMemcpyAsync(A.gb, gbv.data(), sizeof(double) * gbv.size(), cudaMemcpyHostToDevice, s));
    CUDA_OR_FAIL(ctx, cudaMemsetAsync(A.n, 0, sizeof(int), s));
    // the pulse already emitted: the incident field above the plane
    CUDA_OR_FAIL(ctx, launch_ant_add(ctx->fp64, ctx->d_inst, ctx->h, A, 0, s));
    for (int a = 0; a < 3; ++a)  // periodic x / y: refresh the ghosts the gather reads
        if (ctx->any_periodic[a]) CUDA_OR_FAIL(ctx, launch_ghost(ctx->fp64, ctx->L, a, ctx->ghost_max, s));
    CUDA_OR_FAIL(ctx, cudaStreamSynchronize(s));
    ctx->ant_on = true;
    return PIC_OK;
}

extern "C" pic_status pic_set_injection(pic_ctx *ctx, int enable, double z_lab, int32_t first_id)
{
    if (!ctx) return PIC_ERR_ARG;
    if (ctx->is_batch) return fail(ctx, PIC_ERR_ARG, "pic_set_injection on a batch");
    if (enable && !std::isfinite(z_lab)) return fail(ctx, PIC_ERR_ARG, "injection plane z_lab must be finite");
    if (enable && !ctx->opt.track_ids) return fail(ctx, PIC_ERR_STATE, "beam injection needs particle ids (track_ids)");
    cudaSetDevice(ctx->device);
    CUDA_OR_FAIL(ctx, cudaStreamSynchronize(ctx->stream));
    ctx->inj_on = enable != 0;
    ctx->inj_z = enable ? z_lab : 0.0;
    ctx->inj_first = first_id < 0 ? -1 : first_id;
    apply_injection(ctx);
    destroy_graph(ctx);  // the particle kernel with or without the plane
    ctx->version++;      // a batch holding this instance re-reads its parameters
    pic_status st = upload_inst(ctx);
    if (st != PIC_OK) return st;
    CUDA_OR_FAIL(ctx, cudaStreamSynchronize(ctx->stream));
    return PIC_OK;
}

static pic_status ghost_fill_now(pic_ctx *c)
{
    for (int a = 0; a < 3; ++a)
        if (c->any_periodic[a]) CUDA_OR_FAIL(c, launch_ghost(c->fp64, c->L, a, c->ghost_max, c->stream));
    return PIC_OK;
}

static pic_status set_field_internal(pic_ctx *c, int comp, const double *host)
{
    CUDA_OR_FAIL(c, cudaMemcpyAsync(c->d_dense, host, sizeof(double) * (size_t)c->ncell, cudaMemcpyHostToDevice, c->stream));
    CUDA_OR_FAIL(c, launch_unpack(c->fp64, c->h, comp, c->d_dense, c->ncell, c->stream));
    pic_status st = ghost_fill_now(c);
    if (st != PIC_OK) return st;
    CUDA_OR_FAIL(c, cudaStreamSynchronize(c->stream));
    return PIC_OK;
}

extern "C" pic_status pic_set_field(pic_ctx *ctx, int comp, const double *host, size_t count)
{
    if (!ctx) return PIC_ERR_ARG;
    if (ctx->is_batch) return fail(ctx, PIC_ERR_ARG, "pic_set_field on a batch");
    if (comp < PIC_EX || comp > PIC_JZ) return fail(ctx, PIC_ERR_ARG, "component %d cannot be set", comp);
    if (!host || count < (size_t)ctx->ncell) return fail(ctx, PIC_ERR_ARG, "need %lld values", ctx->ncell);
    {
        const int T = host_workers(ctx->ncell);
        std::vector<long long> bad(T, -1);
        parallel_ranges(ctx->ncell, T, [&](int t, int64_t b, int64_t e) {
            for (int64_t i = b; i < e; ++i)
                if (!std::isfinite(host[i])) {
                    bad[t] = i;
                    return;
                }
        });
        for (int t = 0; t < T; ++t)  // the first one over the ranges
            if (bad[t] >= 0) return fail(ctx, PIC_ERR_NAN, "non-finite field value at %lld", bad[t]);
    }
    cudaSetDevice(ctx->device);
    return set_field_internal(ctx, comp, host);
}

extern "C" pic_status pic_load_lab_frame(pic_ctx *ctx, const pic_laser_lab *laser, const pic_plasma_lab *plasma,
                                         const pic_beam_lab *beam)
{
    if (!ctx) return PIC_ERR_ARG;
    if (ctx->is_batch) return fail(ctx, PIC_ERR_ARG, "pic_load_lab_frame on a batch");
    if (laser && !(laser->lambda0 > 0 && laser->waist > 0 && laser->duration > 0 && std::isfinite(laser->a0) &&
                   std::isfinite(laser->z_center)))
        return fail(ctx, PIC_ERR_ARG, "laser parameters invalid");
    if (plasma && !(plasma->ppc >= 1 && plasma->n0 >= 0 && std::isfinite(plasma->n0) && plasma->ramp_len >= 0 &&
                    std::isfinite(plasma->z_start) && finite3(plasma->u_th)))
        return fail(ctx, PIC_ERR_ARG, "plasma parameters invalid");
    if (beam && !(beam->n >= 1 && beam->gamma > 1.0 && beam->sigma_r >= 0 && beam->sigma_z >= 0 && beam->rel_spread >= 0 &&
                  std::isfinite(beam->z0) && std::isfinite(beam->total_weight)))
        return fail(ctx, PIC_ERR_ARG, "beam parameters invalid");
    cudaSetDevice(ctx->device);
    CUDA_OR_FAIL(ctx, cudaStreamSynchronize(ctx->stream));
    Geometry G{ctx->ndim, {ctx->n[0], ctx->n[1], ctx->n[2]}, {ctx->dx[0], ctx->dx[1], ctx->dx[2]}};
    for (int a = 0; a < 3; ++a) G.bc[a] = ctx->bc[a];
    G.order = ctx->order;
    G.charge = ctx->opt.charge;
    // the plasma's lab-stationary ions: a rigid background streaming at -beta_b
    InstDev &h = ctx->h;
    h.ion = plasma && plasma->n0 > 0.0;
    h.ion_n0 = plasma ? plasma->n0 : 0.0;
    h.ion_zs = plasma ? plasma->z_start : 0.0;
    h.ion_ramp = plasma ? plasma->ramp_len : 0.0;
    h.ion_gb = ctx->gamma_b;
    h.ion_beta = std::sqrt(1.0 - 1.0 / (ctx->gamma_b * ctx->gamma_b));
    h.ion_z0 = 0.0;
    h.ion_lz = ctx->n[2] * ctx->dx[2];
    h.ion_periodic = ctx->bc[2] == PIC_PERIODIC;
    h.ion_k0 = 0;
    h.ion_k1 = ctx->n[2];
    // the plasma is drawn on the device (k_load.cu); laser, beam and the beam's field on
    // the host.  Plasma ids come first, as in the host transform.
    std::vector<int> counts;
    long long plasma_ids = 0;
    bool on_device = plasma != nullptr;
    PlasmaGen PG{};
    if (plasma) {
        PG.ndim = ctx->ndim;
        for (int a = 0; a < 3; ++a) PG.n[a] = ctx->n[a], PG.dx[a] = ctx->dx[a], PG.uth[a] = plasma->u_th[a];
        PG.ncell = ctx->ncell;
        PG.gb = ctx->gamma_b;
        PG.beta = std::sqrt(1.0 - 1.0 / (ctx->gamma_b * ctx->gamma_b));
        PG.n0 = plasma->n0;
        PG.zs = plasma->z_start;
        PG.ramp = plasma->ramp_len;
        PG.dV = ctx->dx[0] * ctx->dx[1] * ctx->dx[2];
        PG.ppc = plasma->ppc;
        PG.seed = plasma->seed;
        if (plasma->ppc >= (1 << 15)) on_device = false;
        int *d_count = on_device ? (int *)dalloc(ctx, sizeof(int) * ((size_t)ctx->ncell + 1)) : nullptr;
        if (d_count) {
            counts.resize(ctx->ncell + 1);
            cudaError_t e = cudaMemsetAsync(d_count + ctx->ncell, 0, sizeof(int), ctx->stream);
            if (e == cudaSuccess) e = launch_plasma_count(PG, d_count, ctx->stream);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(counts.data(), d_count, sizeof(int) * counts.size(), cudaMemcpyDeviceToHost, ctx->stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
            dfree(ctx, d_count);
            if (e != cudaSuccess) return fail(ctx, PIC_ERR_CUDA, "plasma count: %s", cudaGetErrorString(e));
            if (counts[ctx->ncell] != 0) on_device = false;  // rare: take the host path
        } else {
            on_device = false;
        }
    }
    LabParticles P;
    LabFields F;
    transform_lab_inputs(G, ctx->gamma_b, laser, on_device ? nullptr : plasma, beam, P, F);
    // fields: zero except the laser and the beam's self-field
    CUDA_OR_FAIL(ctx, cudaMemsetAsync(ctx->h.E[0], 0, 18 * (size_t)ctx->h.cstride * ctx->es, ctx->stream));
    CUDA_OR_FAIL(ctx, cudaMemsetAsync(ctx->h.fpar, 0, sizeof(int), ctx->stream));
    pic_status st;
    for (int c = 0; c < 6; ++c)
        if (!F.comp[c].empty() && (st = set_field_internal(ctx, PIC_EX + c, F.comp[c].data())) != PIC_OK) return st;
    if (!on_device) {
        const int64_t np = (int64_t)P.cell.size();
        ctx->beam_first_id = beam ? P.beam_first : INT_MAX;
        return load_internal(ctx, np, P.cell.data(), P.off.data(), P.mom.data(), P.weight.data(), P.id.data());
    }
    // canonical layout: per tile the plasma particles (cells in linear order), then the
    // beam particles (in their order)
    const long long ncell = ctx->ncell;
    std::vector<int> seg(h.ntiles + 1, 0), plasma_in_tile(h.ntiles, 0);
    long long n_plasma = 0;
    for (long long cidx = 0; cidx < ncell; ++cidx) {
        const int placed = counts[cidx] & 0xffff;
        plasma_in_tile[tile_of_cell(ctx, (int)cidx)] += placed;
        n_plasma += placed;
    }
    const int64_t nb = (int64_t)P.cell.size();
    std::vector<int> beam_slot(nb > 0 ? nb : 1);
    for (int64_t p = 0; p < nb; ++p) seg[tile_of_cell(ctx, P.cell[p]) + 1]++;
    for (int t = 0; t < h.ntiles; ++t) seg[t + 1] += plasma_in_tile[t];
    for (int t = 0; t < h.ntiles; ++t) seg[t + 1] += seg[t];
    const long long n_total = seg[h.ntiles];
    if (n_total >= (1LL << 31) - 1) return fail(ctx, PIC_ERR_ARG, "particle count %lld out of range", n_total);
    std::vector<int> slot0(ncell), id0(ncell);
    {
        std::vector<int> fill(seg.begin(), seg.end() - 1);
        for (long long cidx = 0; cidx < ncell; ++cidx) {
            const int t = tile_of_cell(ctx, (int)cidx);
            slot0[cidx] = fill[t];
            fill[t] += counts[cidx] & 0xffff;
            id0[cidx] = (int)plasma_ids;
            plasma_ids += counts[cidx] >> 16;
        }
        for (int64_t p = 0; p < nb; ++p) beam_slot[p] = fill[tile_of_cell(ctx, P.cell[p])]++;
    }
    if ((st = ensure_particle_capacity(ctx, n_total)) != PIC_OK) return st;
    {
        LoadScratch S{ctx, {}};
        int *d_slot0 = (int *)S.get(sizeof(int) * (size_t)ncell), *d_id0 = (int *)S.get(sizeof(int) * (size_t)ncell);
        if (!d_slot0 || !d_id0) return fail(ctx, PIC_ERR_OOM, "no device memory for the plasma layout");
        CUDA_OR_FAIL(ctx, cudaMemcpyAsync(d_slot0, slot0.data(), sizeof(int) * ncell, cudaMemcpyHostToDevice, ctx->stream));
        CUDA_OR_FAIL(ctx, cudaMemcpyAsync(d_id0, id0.data(), sizeof(int) * ncell, cudaMemcpyHostToDevice, ctx->stream));
        CUDA_OR_FAIL(ctx, launch_plasma_write(ctx->fp64, h, PG, d_slot0, d_id0, ctx->stream));
        CUDA_OR_FAIL(ctx, cudaStreamSynchronize(ctx->stream));
    }
    for (auto &v : P.id) v += (int32_t)plasma_ids;  // beam ids follow the plasma's
    ctx->beam_first_id = beam ? (int32_t)plasma_ids + P.beam_first : INT_MAX;
    if ((st = place_from_host(ctx, nb, P.cell.data(), P.off.data(), P.mom.data(), P.weight.data(), P.id.data(), 0,
                              beam_slot)) != PIC_OK)
        return st;
    return finish_load(ctx, seg);
}

// ------------------------------------------------------------------------------------
// stepping
// ------------------------------------------------------------------------------------
static const Launch &launch_of(pic_ctx *c) { return c->L; }

struct PhaseTimer {
    pic_ctx *c;
    int slot;
    void begin(int phase)
    {
        if (c->profiling) cudaEventRecord(c->events[(size_t)(slot * kPhases + phase) * 2], c->stream);
    }
    void end(int phase)
    {
        if (!c->profiling) return;
        cudaEventRecord(c->events[(size_t)(slot * kPhases + phase) * 2 + 1], c->stream);
        c->recorded[(size_t)slot * kPhases + phase] = 1;
    }
};

static pic_status fold_timings(pic_ctx *c);

static pic_status enqueue_step(pic_ctx *c, int mask)
{
    const Launch &L = launch_of(c);
    const int fp64 = c->fp64;
    PhaseTimer tm{c, c->ev_steps};
    if (c->profiling && c->ev_steps >= kEventSteps) {
        pic_status st = fold_timings(c);
        if (st != PIC_OK) return st;
        tm.slot = 0;
    }
    int launches = 0;
    if (mask & PIC_PHASE_PARTICLES) {
        tm.begin(4);
        if (c->is_batch) {
            for (auto m : c->members)
                CUDA_OR_FAIL(c, cudaMemsetAsync(m->h.J[0], 0, 3 * (size_t)m->h.cstride * m->es, c->stream));
            bool ions = false;
            for (auto m : c->members) ions = ions || m->h.ion != 0;
            if (ions) {
                CUDA_OR_FAIL(c, launch_ion_current(fp64, L, c->stream));
                launches += 2;
            }
        } else {
            CUDA_OR_FAIL(c, launch_j_init_one(fp64, L, c->h, c->stream));
            launches += c->h.ion ? 2 : 1;
        }
        tm.end(4);
        tm.begin(1);
        CUDA_OR_FAIL(c, launch_scan(L, 0, nullptr, c->stream));
        CUDA_OR_FAIL(c, launch_tile_sources(L, c->stream));
        tm.end(1);
        tm.begin(0);
        bool inj = c->h.inj_id0 != INT_MAX;
        for (auto m : c->members) inj = inj || m->h.inj_id0 != INT_MAX;
        CUDA_OR_FAIL(c, launch_particles(c->ndim, c->order, fp64, c->opt.pusher, inj, L, c->is_batch ? nullptr : &c->h,
                                         c->smem, c->stream));
        tm.end(0);
        launches += 3;
    }
    // whether J holds the filtered current when the Yee update reads it: filtered in this
    // call, or by an earlier filter-only call since the last particle phase
    int filtered = (mask & PIC_PHASE_PARTICLES) ? 0 : c->last_filtered;
    if ((mask & PIC_PHASE_FILTER) && c->max_sweeps > 0) {
        const int nin = c->is_batch ? (int)c->members.size() : 1;
        const long long *starts[3] = {c->d_pencil, c->d_pencil + (nin + 1), c->d_pencil + 2 * (nin + 1)};
        tm.begin(2);
        int passes = c->opt.filter_passes;  // the compile-time kernels need one count for all
        for (auto m : c->members)
            if (m->opt.filter_passes != passes) passes = 0;
        CUDA_OR_FAIL(c, launch_filter(fp64, L, starts, c->pencil_total, c->ndim, passes, c->stream));
        tm.end(2);
        filtered = 1;
        for (int a = 0; a < 3; ++a) launches += c->pencil_total[a] > 0 ? 1 : 0;
    }
    if (mask & PIC_PHASE_MAXWELL) {
        tm.begin(3);
        std::vector<pic_ctx *> ants;  // instances with a laser antenna
        if (c->ant_on) ants.push_back(c);
        for (auto m : c->members)
            if (m->ant_on) ants.push_back(m);
        if (ants.empty() && c->opt.solver == PIC_SOLVER_YEE && c->pencil_total[3] > 0) {
            // the fused update: one launch, then the buffer switch
            const int nin = c->is_batch ? (int)c->members.size() : 1;
            CUDA_OR_FAIL(c, launch_maxwell_fused(fp64, c->ndim, L, c->d_pencil + 3 * (nin + 1), c->pencil_total[3], filtered,
                                                 c->stream));
            launches += 2;
        } else if (ants.empty()) {
            CUDA_OR_FAIL(c, launch_maxwell(fp64, c->opt.solver, L, filtered, c->stream));
            launches += 3;
        } else {
            // the antenna's boundary terms and lattice steps between the Yee sub-updates
            cudaStream_t s = c->stream;
            CUDA_OR_FAIL(c, launch_bhalf(fp64, c->opt.solver, L, 0, s));
            for (auto m : ants) {
                CUDA_OR_FAIL(c, launch_ant_bterm(fp64, c->opt.solver == PIC_SOLVER_CK, m->d_inst, m->h, m->ant, 0, s));
                CUDA_OR_FAIL(c, launch_ant_lattice(m->ant, m->dt, m->dx[2], 0, s));
            }
            CUDA_OR_FAIL(c, launch_efull(fp64, L, filtered, s));
            for (auto m : ants) {
                CUDA_OR_FAIL(c, launch_ant_eterm(fp64, m->d_inst, m->h, m->ant, s));
                CUDA_OR_FAIL(c, launch_ant_lattice(m->ant, m->dt, m->dx[2], 1, s));
            }
            CUDA_OR_FAIL(c, launch_bhalf(fp64, c->opt.solver, L, 1, s));
            for (auto m : ants) {
                CUDA_OR_FAIL(c, launch_ant_bterm(fp64, c->opt.solver == PIC_SOLVER_CK, m->d_inst, m->h, m->ant, 1, s));
                CUDA_OR_FAIL(c, launch_ant_lattice(m->ant, m->dt, m->dx[2], 2, s));
                CUDA_OR_FAIL(c, launch_ant_add(fp64, m->d_inst, m->h, m->ant, 1, s));
            }
            launches += 3 + 7 * (int)ants.size();
        }
        for (int a = 0; a < 3; ++a)
            if (c->any_periodic[a]) {
                CUDA_OR_FAIL(c, launch_ghost(fp64, L, a, c->ghost_max, c->stream));
                launches++;
            }
        tm.end(3);
    }
    if (mask == PIC_PHASE_ALL && c->nst > 0 && !c->is_batch) {
        tm.begin(4);
        StationDev S{c->d_st_z, c->d_st_count, c->d_st_t, c->d_st_fields, c->st_max};
        CUDA_OR_FAIL(c, launch_stations(fp64, c->d_inst, S, c->nst, c->n[0] * c->n[1], c->stream));
        tm.end(4);
        launches += 2;
    }
    if (mask & PIC_PHASE_PARTICLES) {
        // J now holds this phase's deposit; a filtered copy from an earlier step is stale
        c->last_filtered = 0;
        if (c->is_batch)
            for (auto m : c->members) m->last_filtered = 0;
    }
    if (mask & (PIC_PHASE_FILTER | PIC_PHASE_MAXWELL)) {
        c->last_filtered = filtered;
        if (c->is_batch)
            for (auto m : c->members) m->last_filtered = filtered;
    }
    if (c->profiling) {
        c->ev_steps = tm.slot + 1;
        c->acc.launches += launches;
        c->acc.steps += 1;
    }
    return PIC_OK;
}

static pic_status refresh_batch(pic_ctx *c);

extern "C" pic_status pic_step(pic_ctx *ctx, int n)
{
    if (!ctx) return PIC_ERR_ARG;
    if (n < 0) return fail(ctx, PIC_ERR_ARG, "n must be >= 0");
    cudaSetDevice(ctx->device);
    if (ctx->is_batch) {
        pic_status st = refresh_batch(ctx);
        if (st != PIC_OK) return st;
    } else if (!ctx->loaded) {
        return fail(ctx, PIC_ERR_STATE, "pic_step before any load");
    }
    if (ctx->is_batch && ctx->persistent && !ctx->profiling && n > 0) {
        // every step in one launch of the persistent kernel
        const int nin = (int)ctx->members.size();
        const pic_ctx *m0 = ctx->members[0];
        const int filtered = ctx->max_sweeps > 0 ? 1 : 0;
        CUDA_OR_FAIL(ctx, ctx->plan->launch(ctx->L, ctx->ndim, ctx->order, n, m0->opt.filter_passes, filtered, ctx->d_pencil,
                                            ctx->d_pencil + 3 * (nin + 1), ctx->persist_smem, ctx->persist_grid,
                                            ctx->spin_limit, ctx->stall_inst, ctx->stream));
        ctx->step += n;
        ctx->mx_phases += n;
        for (auto m : ctx->members) m->step += n, m->mx_phases += n, m->last_filtered = filtered;
        ctx->last_filtered = filtered;
        return PIC_OK;
    }
    for (int s = 0; s < n; ++s) {
        if (ctx->profiling || ctx->stream == nullptr) {
            pic_status st = enqueue_step(ctx, PIC_PHASE_ALL);
            if (st != PIC_OK) return st;
        } else {
            if (!ctx->graph) {
                cudaGraph_t g;
                CUDA_OR_FAIL(ctx, cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
                pic_status st = enqueue_step(ctx, PIC_PHASE_ALL);
                cudaError_t e = cudaStreamEndCapture(ctx->stream, &g);
                if (st != PIC_OK) return st;
                if (e != cudaSuccess) return fail(ctx, PIC_ERR_CUDA, "graph capture failed: %s", cudaGetErrorString(e));
                e = cudaGraphInstantiate(&ctx->graph, g, 0);
                cudaGraphDestroy(g);
                if (e != cudaSuccess) {
                    ctx->graph = nullptr;
                    return fail(ctx, PIC_ERR_CUDA, "graph instantiation failed: %s", cudaGetErrorString(e));
                }
            }
            CUDA_OR_FAIL(ctx, cudaGraphLaunch(ctx->graph, ctx->stream));
        }
        ctx->step++;
        ctx->mx_phases++;
        if (ctx->is_batch)
            for (auto m : ctx->members) m->step++, m->mx_phases++;
    }
    return PIC_OK;
}

extern "C" pic_status pic_run_phases(pic_ctx *ctx, int mask)
{
    if (!ctx) return PIC_ERR_ARG;
    if (mask <= 0 || mask > PIC_PHASE_ALL) return fail(ctx, PIC_ERR_ARG, "phase mask %d invalid", mask);
    cudaSetDevice(ctx->device);
    if (ctx->is_batch) {
        pic_status st = refresh_batch(ctx);
        if (st != PIC_OK) return st;
    } else if (!ctx->loaded) {
        return fail(ctx, PIC_ERR_STATE, "pic_run_phases before any load");
    }
    pic_status st = enqueue_step(ctx, mask);
    if (st != PIC_OK) return st;
    if (mask == PIC_PHASE_ALL) {
        ctx->step++;
        if (ctx->is_batch)
            for (auto m : ctx->members) m->step++;
    }
    if (mask & PIC_PHASE_MAXWELL) {
        ctx->mx_phases++;
        if (ctx->is_batch)
            for (auto m : ctx->members) m->mx_phases++;
    }
    return PIC_OK;
}

// Device -> host copy ordered after the context's work (its stream need not synchronise
// with the legacy default stream); returns when the data is on the host.
static cudaError_t d2h(pic_ctx *c, void *dst, const void *src, size_t bytes)
{
    cudaError_t e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, c->stream);
    return e == cudaSuccess ? cudaStreamSynchronize(c->stream) : e;
}

// The status of a sticky device error word (PIC_OK when it is 0).
static pic_status device_error_status(pic_ctx *c, int err)
{
    if (err & kErrTimeout) return fail(c, PIC_ERR_TIMEOUT, "a bounded device wait timed out (error word 0x%x)", err);
    if (err & kErrSpeed) return fail(c, PIC_ERR_PARTICLE_SPEED, "a particle moved a cell or more in one step, or is not finite (0x%x)", err);
    if (err & (kErrInternal | kErrCapacity)) return fail(c, PIC_ERR_INTERNAL, "device consistency check failed (0x%x)", err);
    return PIC_OK;
}

static pic_status check_device_error(pic_ctx *c)
{
    int err = 0;
    CUDA_OR_FAIL(c, d2h(c, &err, c->h.err, sizeof(int)));
    if (err & kErrTimeout) return fail(c, PIC_ERR_TIMEOUT, "a bounded device wait timed out (error word 0x%x)", err);
    if (err & kErrSpeed) return fail(c, PIC_ERR_PARTICLE_SPEED, "a particle moved a cell or more in one step, or is not finite (0x%x)", err);
    if (err & (kErrInternal | kErrCapacity)) return fail(c, PIC_ERR_INTERNAL, "device consistency check failed (0x%x)", err);
    return PIC_OK;
}

extern "C" pic_status pic_synchronize(pic_ctx *ctx)
{
    if (!ctx) return PIC_ERR_ARG;
    cudaSetDevice(ctx->device);
    CUDA_OR_FAIL(ctx, cudaStreamSynchronize(ctx->stream));
    CUDA_OR_FAIL(ctx, cudaGetLastError());
    if (ctx->is_batch) {
        for (auto m : ctx->members) {
            pic_status st = check_device_error(m);
            if (st != PIC_OK) return fail(ctx, st, "%s", m->err.c_str());
        }
        return PIC_OK;
    }
    return check_device_error(ctx);
}

// ------------------------------------------------------------------------------------
// getters
// ------------------------------------------------------------------------------------
extern "C" pic_status pic_get_field(pic_ctx *ctx, int comp, double *host_out, size_t count)
{
    if (!ctx) return PIC_ERR_ARG;
    if (ctx->is_batch) return fail(ctx, PIC_ERR_ARG, "getters take a member, not a batch");
    if (comp < PIC_EX || comp > PIC_DIVE) return fail(ctx, PIC_ERR_ARG, "component %d invalid", comp);
    if (!host_out || count < (size_t)ctx->ncell) return fail(ctx, PIC_ERR_ARG, "need room for %lld values", ctx->ncell);
    pic_status st = pic_synchronize(ctx);
    if (st != PIC_OK) return st;
    if (comp == PIC_RHO) {
        CUDA_OR_FAIL(ctx, cudaMemsetAsync(ctx->d_dense, 0, sizeof(double) * (size_t)ctx->ncell, ctx->stream));
        if (ctx->loaded) CUDA_OR_FAIL(ctx, launch_rho(ctx->order, ctx->fp64, ctx->L, ctx->d_dense, ctx->stream));
    } else if (comp == PIC_DIVE) {
        CUDA_OR_FAIL(ctx, launch_dive(ctx->fp64, ctx->h, ctx->d_dense, ctx->ncell, ctx->stream));
    } else {
        CUDA_OR_FAIL(ctx, launch_pack(ctx->fp64, ctx->h, comp, ctx->last_filtered, ctx->d_dense, ctx->ncell, ctx->stream));
    }
    CUDA_OR_FAIL(ctx, cudaMemcpyAsync(host_out, ctx->d_dense, sizeof(double) * (size_t)ctx->ncell, cudaMemcpyDeviceToHost, ctx->stream));
    CUDA_OR_FAIL(ctx, cudaStreamSynchronize(ctx->stream));
    return check_device_error(ctx);
}

extern "C" pic_status pic_get_fields(pic_ctx *ctx, const int *comps, int ncomp, double *host_out, size_t count)
{
    if (!ctx) return PIC_ERR_ARG;
    if (ncomp < 1 || !comps) return fail(ctx, PIC_ERR_ARG, "need at least one component");
    if (!host_out || count / (size_t)ncomp < (size_t)ctx->ncell)
        return fail(ctx, PIC_ERR_ARG, "need room for %d x %lld values", ncomp, ctx->ncell);
    for (int i = 0; i < ncomp; ++i) {
        const pic_status st = pic_get_field(ctx, comps[i], host_out + (size_t)i * ctx->ncell, (size_t)ctx->ncell);
        if (st != PIC_OK) return st;
    }
    return PIC_OK;
}

extern "C" pic_status pic_get_gauss_residual(pic_ctx *ctx, double *max_abs, double *rms)
{
    if (!ctx || !max_abs) return PIC_ERR_ARG;
    if (ctx->is_batch) return fail(ctx, PIC_ERR_ARG, "getters take a member, not a batch");
    pic_status st = pic_synchronize(ctx);
    if (st != PIC_OK) return st;
    double *rho = (double *)dalloc(ctx, sizeof(double) * (size_t)ctx->ncell);
    if (!rho) return fail(ctx, PIC_ERR_OOM, "no device memory for the charge density");
    cudaStream_t s = ctx->stream;
    cudaError_t e = cudaMemsetAsync(rho, 0, sizeof(double) * (size_t)ctx->ncell, s);
    if (e == cudaSuccess && ctx->loaded) e = launch_rho(ctx->order, ctx->fp64, ctx->L, rho, s);
    if (e == cudaSuccess) e = launch_dive(ctx->fp64, ctx->h, ctx->d_dense, ctx->ncell, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->d_sums, 0, 2 * sizeof(double), s);
    if (e == cudaSuccess)
        e = launch_residual(ctx->d_dense, rho, ctx->ncell, (unsigned long long *)ctx->d_sums, ctx->d_sums + 1, s);
    double host[2] = {0.0, 0.0};
    if (e == cudaSuccess) e = d2h(ctx, host, ctx->d_sums, sizeof(host));
    dfree(ctx, rho);
    if (e != cudaSuccess) return fail(ctx, PIC_ERR_CUDA, "Gauss residual: %s", cudaGetErrorString(e));
    unsigned long long bits;
    std::memcpy(&bits, &host[0], sizeof(bits));
    std::memcpy(max_abs, &bits, sizeof(double));
    if (rms) *rms = std::sqrt(host[1] / (double)ctx->ncell);
    return check_device_error(ctx);
}

static pic_status count_live(pic_ctx *c, int with_offsets, int *live)
{
    CUDA_OR_FAIL(c, launch_scan(c->L, 1, c->d_start_ptr, c->stream));
    CUDA_OR_FAIL(c, cudaMemcpyAsync(live, c->h.live, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CUDA_OR_FAIL(c, cudaStreamSynchronize(c->stream));
    (void)with_offsets;
    return PIC_OK;
}

extern "C" pic_status pic_num_particles(pic_ctx *ctx, int64_t *n_out)
{
    if (!ctx || !n_out) return PIC_ERR_ARG;
    if (ctx->is_batch) return fail(ctx, PIC_ERR_ARG, "getters take a member, not a batch");
    pic_status st = pic_synchronize(ctx);
    if (st != PIC_OK) return st;
    int live = 0;
    if (ctx->loaded && (st = count_live(ctx, 0, &live)) != PIC_OK) return st;
    *n_out = live;
    return PIC_OK;
}

// Device staging for the canonical read-out of every particle the buffers can hold.
static pic_status ensure_staging(pic_ctx *ctx)
{
    InstDev &h = ctx->h;
    if (ctx->stage_cap >= h.cap) return PIC_OK;
    dfree(ctx, ctx->st_cell);
    ctx->st_cell = nullptr;
    const size_t per = (size_t)h.cap;
    unsigned char *blk = (unsigned char *)dalloc(ctx, per * (2 * sizeof(int) + 7 * sizeof(double)) + 2048);
    if (!blk) return fail(ctx, PIC_ERR_OOM, "read-out staging does not fit");
    size_t o = 0;
    auto take = [&](size_t b) {
        void *p = blk + o;
        o += (b + 255) & ~(size_t)255;
        return p;
    };
    ctx->st_cell = (int *)take(per * sizeof(int));
    ctx->st_id = (int *)take(per * sizeof(int));
    ctx->st_off = (double *)take(per * 3 * sizeof(double));
    ctx->st_u = (double *)take(per * 3 * sizeof(double));
    ctx->st_w = (double *)take(per * sizeof(double));
    ctx->stage_cap = h.cap;
    return PIC_OK;
}

static pic_status get_particles_internal(pic_ctx *ctx, int32_t *cell, void *off3v, void *u3v, void *wv, int32_t *id,
                                         int64_t cap, int64_t *n_out, bool widen)
{
    if (!ctx || !n_out) return PIC_ERR_ARG;
    if (ctx->is_batch) return fail(ctx, PIC_ERR_ARG, "getters take a member, not a batch");
    pic_status st = pic_synchronize(ctx);
    if (st != PIC_OK) return st;
    *n_out = 0;
    if (!ctx->loaded) return PIC_OK;
    int live = 0;
    if ((st = count_live(ctx, 1, &live)) != PIC_OK) return st;
    *n_out = live;
    if (live > cap) return fail(ctx, PIC_ERR_ARG, "cap %lld < %d live particles", (long long)cap, live);
    if (live == 0) return PIC_OK;
    if ((st = ensure_staging(ctx)) != PIC_OK) return st;
    CUDA_OR_FAIL(ctx, launch_readout(ctx->fp64, ctx->L, ctx->d_start_ptr, ctx->st_cell, ctx->st_off, ctx->st_u, ctx->st_w,
                                     ctx->st_id, ctx->stream));
    // values copied in the storage precision (FP32: half the bytes) into the caller's
    // arrays, then widened there in place when FP64 values are asked for
    double *off3 = (double *)off3v, *u3 = (double *)u3v, *w = (double *)wv;
    const size_t n = (size_t)live, es = ctx->es;
    if (cell) CUDA_OR_FAIL(ctx, cudaMemcpyAsync(cell, ctx->st_cell, n * sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    if (id) CUDA_OR_FAIL(ctx, cudaMemcpyAsync(id, ctx->st_id, n * sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    if (off3) CUDA_OR_FAIL(ctx, cudaMemcpyAsync(off3, ctx->st_off, 3 * n * es, cudaMemcpyDeviceToHost, ctx->stream));
    if (u3) CUDA_OR_FAIL(ctx, cudaMemcpyAsync(u3, ctx->st_u, 3 * n * es, cudaMemcpyDeviceToHost, ctx->stream));
    if (w) CUDA_OR_FAIL(ctx, cudaMemcpyAsync(w, ctx->st_w, n * es, cudaMemcpyDeviceToHost, ctx->stream));
    CUDA_OR_FAIL(ctx, cudaStreamSynchronize(ctx->stream));
    if (widen && !ctx->fp64) {
        if (off3) widen_in_place(off3, 3 * n);
        if (u3) widen_in_place(u3, 3 * n);
        if (w) widen_in_place(w, n);
    }
    return check_device_error(ctx);
}

extern "C" pic_status pic_get_particles(pic_ctx *ctx, int32_t *cell, double *off3, double *u3, double *w, int32_t *id,
                                        int64_t cap, int64_t *n_out)
{
    return get_particles_internal(ctx, cell, off3, u3, w, id, cap, n_out, true);
}

extern "C" pic_status pic_get_particles_stored(pic_ctx *ctx, int32_t *cell, void *off3, void *u3, void *w, int32_t *id,
                                               int64_t cap, int64_t *n_out)
{
    return get_particles_internal(ctx, cell, off3, u3, w, id, cap, n_out, false);
}

// ---- z-slab exchange (domain decomposition along z) -----------------------------------
static pic_status check_planes(pic_ctx *c, int comp, int k0, int nk, size_t count)
{
    if (c->is_batch) return fail(c, PIC_ERR_ARG, "plane exchange takes a member, not a batch");
    if (comp < PIC_EX || comp > PIC_JZ) return fail(c, PIC_ERR_ARG, "component %d invalid for planes", comp);
    if (nk < 1 || k0 < 0 || k0 + nk > c->n[2]) return fail(c, PIC_ERR_ARG, "planes %d .. %d outside 0 .. %d", k0, k0 + nk - 1, c->n[2] - 1);
    if (count < (size_t)nk * c->n[0] * c->n[1]) return fail(c, PIC_ERR_ARG, "need room for %zu values", (size_t)nk * c->n[0] * c->n[1]);
    return PIC_OK;
}

extern "C" pic_status pic_get_planes(pic_ctx *ctx, int comp, int k0, int nk, double *host_out, size_t count)
{
    if (!ctx || !host_out) return PIC_ERR_ARG;
    pic_status st = check_planes(ctx, comp, k0, nk, count);
    if (st != PIC_OK) return st;
    if ((st = pic_synchronize(ctx)) != PIC_OK) return st;
    const size_t n = (size_t)nk * ctx->n[0] * ctx->n[1];
    CUDA_OR_FAIL(ctx, launch_pack_planes(ctx->fp64, ctx->h, comp, ctx->last_filtered, ctx->d_dense, k0, nk, ctx->stream));
    CUDA_OR_FAIL(ctx, cudaMemcpyAsync(host_out, ctx->d_dense, sizeof(double) * n, cudaMemcpyDeviceToHost, ctx->stream));
    CUDA_OR_FAIL(ctx, cudaStreamSynchronize(ctx->stream));
    return check_device_error(ctx);
}

extern "C" pic_status pic_put_planes(pic_ctx *ctx, int comp, int k0, int nk, const double *host_in, size_t count, int add)
{
    if (!ctx || !host_in) return PIC_ERR_ARG;
    pic_status st = check_planes(ctx, comp, k0, nk, count);
    if (st != PIC_OK) return st;
    if ((st = pic_synchronize(ctx)) != PIC_OK) return st;
    const size_t n = (size_t)nk * ctx->n[0] * ctx->n[1];
    CUDA_OR_FAIL(ctx, cudaMemcpyAsync(ctx->d_dense, host_in, sizeof(double) * n, cudaMemcpyHostToDevice, ctx->stream));
    CUDA_OR_FAIL(ctx, launch_unpack_planes(ctx->fp64, ctx->h, comp, ctx->d_dense, k0, nk, add ? 1 : 0, ctx->stream));
    // E and B carry copies of the periodic faces that the gather reads (the current does not)
    if (comp < PIC_JX && (st = ghost_fill_now(ctx)) != PIC_OK) return st;
    CUDA_OR_FAIL(ctx, cudaStreamSynchronize(ctx->stream));
    return check_device_error(ctx);
}

// Several components' planes in one call: packed one component after the other into the
// dense scratch (as many components at a time as it holds), one copy and one
// synchronisation per batch.
extern "C" pic_status pic_get_planes_n(pic_ctx *ctx, const int *comps, int ncomp, int k0, int nk, double *host_out,
                                       size_t count)
{
    if (!ctx || !comps || !host_out || ncomp < 1) return PIC_ERR_ARG;
    const size_t per = (size_t)nk * ctx->n[0] * ctx->n[1];
    for (int i = 0; i < ncomp; ++i) {
        pic_status st = check_planes(ctx, comps[i], k0, nk, per);
        if (st != PIC_OK) return st;
    }
    if (count < per * ncomp) return fail(ctx, PIC_ERR_ARG, "need room for %zu values", per * ncomp);
    pic_status st = pic_synchronize(ctx);
    if (st != PIC_OK) return st;
    const int fit = (int)std::max<size_t>(1, (size_t)ctx->ncell / std::max<size_t>(per, 1));
    for (int i0 = 0; i0 < ncomp; i0 += fit) {
        const int m = std::min(fit, ncomp - i0);
        for (int i = 0; i < m; ++i)
            CUDA_OR_FAIL(ctx, launch_pack_planes(ctx->fp64, ctx->h, comps[i0 + i], ctx->last_filtered, ctx->d_dense + per * i,
                                                 k0, nk, ctx->stream));
        CUDA_OR_FAIL(ctx, cudaMemcpyAsync(host_out + per * i0, ctx->d_dense, sizeof(double) * per * m, cudaMemcpyDeviceToHost,
                                          ctx->stream));
        CUDA_OR_FAIL(ctx, cudaStreamSynchronize(ctx->stream));
    }
    return check_device_error(ctx);
}

extern "C" pic_status pic_put_planes_n(pic_ctx *ctx, const int *comps, int ncomp, int k0, int nk, const double *host_in,
                                       size_t count, int add)
{
    if (!ctx || !comps || !host_in || ncomp < 1) return PIC_ERR_ARG;
    const size_t per = (size_t)nk * ctx->n[0] * ctx->n[1];
    bool eb = false;
    for (int i = 0; i < ncomp; ++i) {
        pic_status st = check_planes(ctx, comps[i], k0, nk, per);
        if (st != PIC_OK) return st;
        eb = eb || comps[i] < PIC_JX;
    }
    if (count < per * ncomp) return fail(ctx, PIC_ERR_ARG, "need room for %zu values", per * ncomp);
    pic_status st = pic_synchronize(ctx);
    if (st != PIC_OK) return st;
    const int fit = (int)std::max<size_t>(1, (size_t)ctx->ncell / std::max<size_t>(per, 1));
    for (int i0 = 0; i0 < ncomp; i0 += fit) {
        const int m = std::min(fit, ncomp - i0);
        CUDA_OR_FAIL(ctx, cudaMemcpyAsync(ctx->d_dense, host_in + per * i0, sizeof(double) * per * m, cudaMemcpyHostToDevice,
                                          ctx->stream));
        for (int i = 0; i < m; ++i)
            CUDA_OR_FAIL(ctx, launch_unpack_planes(ctx->fp64, ctx->h, comps[i0 + i], ctx->d_dense + per * i, k0, nk,
                                                   add ? 1 : 0, ctx->stream));
        CUDA_OR_FAIL(ctx, cudaStreamSynchronize(ctx->stream));  // before the scratch is reused
    }
    if (eb && (st = ghost_fill_now(ctx)) != PIC_OK) return st;
    CUDA_OR_FAIL(ctx, cudaStreamSynchronize(ctx->stream));
    return check_device_error(ctx);
}

// The live particles read out on the device into the staging arrays (storage precision,
// canonical order); their cells copied to the host.
static pic_status stage_particles(pic_ctx *c, std::vector<int32_t> &cells, int &live)
{
    pic_status st = pic_synchronize(c);
    if (st != PIC_OK) return st;
    live = 0;
    if ((st = count_live(c, 1, &live)) != PIC_OK) return st;
    cells.resize((size_t)std::max(live, 1));
    if (live == 0) return PIC_OK;
    if ((st = ensure_staging(c)) != PIC_OK) return st;
    CUDA_OR_FAIL(c, launch_readout(c->fp64, c->L, c->d_start_ptr, c->st_cell, c->st_off, c->st_u, c->st_w, c->st_id,
                                   c->stream));
    CUDA_OR_FAIL(c, cudaMemcpyAsync(cells.data(), c->st_cell, sizeof(int) * (size_t)live, cudaMemcpyDeviceToHost, c->stream));
    CUDA_OR_FAIL(c, cudaStreamSynchronize(c->stream));
    return PIC_OK;
}

// Stable counting sort by tile of n particles whose cells cell_at(q) gives: the slot of
// each in the canonical order and the tile segments (host threads over contiguous ranges,
// each range taking its slots in order, as the load does).
template <typename F>
static void canonical_slots(const pic_ctx *c, int64_t n, F cell_at, std::vector<int> &slot, std::vector<int> &seg)
{
    const int ntiles = c->h.ntiles;
    const int T = host_workers(n);
    std::vector<std::vector<int>> hist(T);
    slot.assign((size_t)std::max<int64_t>(n, 1), 0);
    seg.assign(ntiles + 1, 0);
    parallel_ranges(n, T, [&](int t, int64_t b, int64_t e) {
        std::vector<int> &hc = hist[t];
        hc.assign(ntiles, 0);
        for (int64_t q = b; q < e; ++q) {
            slot[q] = tile_of_cell(c, cell_at(q));
            hc[slot[q]]++;
        }
    });
    for (int t = 0; t < T; ++t)
        for (int k = 0; k < ntiles; ++k) seg[k + 1] += hist[t][k];
    for (int k = 0; k < ntiles; ++k) seg[k + 1] += seg[k];
    std::vector<int> fill(seg.begin(), seg.end() - 1);
    for (int t = 0; t < T; ++t)
        for (int k = 0; k < ntiles; ++k) {
            const int m = hist[t][k];
            hist[t][k] = fill[k];
            fill[k] += m;
        }
    parallel_ranges(n, T, [&](int t, int64_t b, int64_t e) {
        std::vector<int> &f = hist[t];
        for (int64_t q = b; q < e; ++q) slot[q] = f[slot[q]]++;
    });
}

// The first n values of an SoA device array in the storage precision, widened to FP64
// into host_strided[i * stride + lane].
static pic_status copy_out_widened(pic_ctx *c, const void *dev, size_t n, double *host_strided, int stride, int lane)
{
    std::vector<double> tmp(n);
    if (c->fp64) {
        CUDA_OR_FAIL(c, d2h(c, tmp.data(), dev, sizeof(double) * n));
    } else {
        std::vector<float> f(n);
        CUDA_OR_FAIL(c, d2h(c, f.data(), dev, sizeof(float) * n));
        for (size_t i = 0; i < n; ++i) tmp[i] = f[i];
    }
    for (size_t i = 0; i < n; ++i) host_strided[i * stride + lane] = tmp[i];
    return PIC_OK;
}

// The particles are read out and laid out again on the device; only their cells (and the
// particles taken out) cross to the host.
extern "C" pic_status pic_extract_particles(pic_ctx *ctx, int k_lo, int k_hi, int32_t *cell, double *off3, double *u3,
                                            double *w, int32_t *id, int64_t cap, int64_t *n_out)
{
    if (!ctx || !n_out) return PIC_ERR_ARG;
    if (ctx->is_batch) return fail(ctx, PIC_ERR_ARG, "pic_extract_particles takes a member, not a batch");
    if (!ctx->loaded) return fail(ctx, PIC_ERR_STATE, "pic_extract_particles before any load");
    if (k_lo > k_hi) return fail(ctx, PIC_ERR_ARG, "k_lo %d > k_hi %d", k_lo, k_hi);
    cudaSetDevice(ctx->device);
    *n_out = 0;
    std::vector<int32_t> cells;
    int live = 0;
    pic_status st = stage_particles(ctx, cells, live);
    if (st != PIC_OK) return st;
    const long long plane = (long long)ctx->n[0] * ctx->n[1];
    std::vector<int> map((size_t)std::max(live, 1));
    std::vector<int64_t> keep;
    keep.reserve((size_t)live);
    int ngo = 0;
    for (int i = 0; i < live; ++i) {
        const int k = (int)(cells[i] / plane);
        if (k < k_lo || k >= k_hi) map[i] = -1 - ngo++;
        else keep.push_back(i);
    }
    *n_out = ngo;
    if (ngo > cap) return fail(ctx, PIC_ERR_ARG, "cap %lld < %d particles to extract", (long long)cap, ngo);
    if (ngo == 0) return PIC_OK;
    std::vector<int> slot, seg;
    canonical_slots(ctx, (int64_t)keep.size(), [&](int64_t q) { return cells[keep[q]]; }, slot, seg);
    for (size_t q = 0; q < keep.size(); ++q) map[keep[q]] = slot[q];
    {
        LoadScratch S{ctx, {}};
        int *d_map = (int *)S.get(sizeof(int) * (size_t)live);
        if (!d_map) return fail(ctx, PIC_ERR_OOM, "no device memory for the particle map");
        CUDA_OR_FAIL(ctx, cudaMemcpyAsync(d_map, map.data(), sizeof(int) * (size_t)live, cudaMemcpyHostToDevice, ctx->stream));
        StagedSrc src{ctx->st_cell, ctx->st_off, ctx->st_u, ctx->st_w, ctx->st_id, d_map, (long long)live};
        CUDA_OR_FAIL(ctx, launch_place_staged(ctx->fp64, ctx->h, src, ctx->stream));
        CUDA_OR_FAIL(ctx, cudaStreamSynchronize(ctx->stream));
    }
    // the particles taken out, packed at the start of buffer 1
    const InstDev &h = ctx->h;
    const size_t ng = (size_t)ngo;
    if (cell) CUDA_OR_FAIL(ctx, d2h(ctx, cell, h.cell[1], sizeof(int) * ng));
    if (id) {
        if (h.id[1]) CUDA_OR_FAIL(ctx, d2h(ctx, id, h.id[1], sizeof(int) * ng));
        else std::memset(id, 0, sizeof(int) * ng);
    }
    for (int a = 0; a < 3; ++a) {
        if (off3) {
            if (h.off[1][a]) {
                if ((st = copy_out_widened(ctx, h.off[1][a], ng, off3, 3, a)) != PIC_OK) return st;
            } else {
                for (size_t i = 0; i < ng; ++i) off3[3 * i + a] = 0.0;
            }
        }
        if (u3 && (st = copy_out_widened(ctx, h.u[1][a], ng, u3, 3, a)) != PIC_OK) return st;
    }
    if (w && (st = copy_out_widened(ctx, h.w[1], ng, w, 1, 0)) != PIC_OK) return st;
    return finish_relayout(ctx, seg);
}

extern "C" pic_status pic_add_particles(pic_ctx *ctx, int64_t n, const int32_t *cell, const double *off3, const double *u3,
                                        const double *w, const int32_t *id)
{
    if (!ctx) return PIC_ERR_ARG;
    if (ctx->is_batch) return fail(ctx, PIC_ERR_ARG, "pic_add_particles takes a member, not a batch");
    if (!ctx->loaded) return fail(ctx, PIC_ERR_STATE, "pic_add_particles before any load");
    if (n < 0 || (n > 0 && (!cell || !off3 || !u3 || !w))) return fail(ctx, PIC_ERR_ARG, "particle arrays invalid");
    if (n == 0) return PIC_OK;
    cudaSetDevice(ctx->device);
    for (int64_t p = 0; p < n; ++p) {
        if (cell[p] < 0 || cell[p] >= ctx->ncell) return fail(ctx, PIC_ERR_ARG, "particle %lld: cell %d outside the grid", (long long)p, cell[p]);
        for (int a = 0; a < 3; ++a) {
            const double o = off3[3 * p + a];
            if (activeaxis(ctx->ndim, a) && !(o >= 0.0 && o < 1.0))
                return fail(ctx, PIC_ERR_ARG, "particle %lld: offset %g outside [0,1)", (long long)p, o);
        }
        if (!finite3(u3 + 3 * p) || !std::isfinite(w[p])) return fail(ctx, PIC_ERR_NAN, "particle %lld: non-finite momentum or weight", (long long)p);
    }
    std::vector<int32_t> cells;
    int live = 0;
    pic_status st = stage_particles(ctx, cells, live);
    if (st != PIC_OK) return st;
    const int64_t total = (int64_t)live + n;
    if (total >= (1LL << 31) - 1) return fail(ctx, PIC_ERR_ARG, "particle count %lld out of range", (long long)total);
    std::vector<int> slot, seg;
    canonical_slots(ctx, total, [&](int64_t q) { return q < live ? cells[q] : cell[q - live]; }, slot, seg);
    if ((st = ensure_particle_capacity(ctx, total)) != PIC_OK) return st;
    if (live > 0) {
        LoadScratch S{ctx, {}};
        int *d_map = (int *)S.get(sizeof(int) * (size_t)live);
        if (!d_map) return fail(ctx, PIC_ERR_OOM, "no device memory for the particle map");
        CUDA_OR_FAIL(ctx, cudaMemcpyAsync(d_map, slot.data(), sizeof(int) * (size_t)live, cudaMemcpyHostToDevice, ctx->stream));
        StagedSrc src{ctx->st_cell, ctx->st_off, ctx->st_u, ctx->st_w, ctx->st_id, d_map, (long long)live};
        CUDA_OR_FAIL(ctx, launch_place_staged(ctx->fp64, ctx->h, src, ctx->stream));
        CUDA_OR_FAIL(ctx, cudaStreamSynchronize(ctx->stream));
    }
    std::vector<int> slot_new(slot.begin() + live, slot.begin() + total);
    std::vector<int32_t> zero_ids;
    const int32_t *ids = id;
    if (!ids && ctx->opt.track_ids) {
        zero_ids.assign((size_t)n, 0);
        ids = zero_ids.data();
    }
    if ((st = place_from_host(ctx, n, cell, off3, u3, w, ids, 0, slot_new)) != PIC_OK) return st;
    return finish_relayout(ctx, seg);
}

extern "C" pic_status pic_adopt_slab(pic_ctx *slab, pic_ctx *whole, int k_origin, int k_lo, int k_hi)
{
    if (!slab || !whole) return PIC_ERR_ARG;
    if (k_lo < 0 || k_lo >= k_hi || k_hi > slab->n[2]) return fail(slab, PIC_ERR_ARG, "owned planes %d .. %d invalid", k_lo, k_hi);
    if (slab->is_batch || whole->is_batch) return fail(slab, PIC_ERR_ARG, "pic_adopt_slab takes members, not batches");
    if (slab == whole) return fail(slab, PIC_ERR_ARG, "a context cannot be its own slab");
    if (!slab->loaded || !whole->loaded) return fail(slab, PIC_ERR_STATE, "pic_adopt_slab needs both contexts loaded");
    bool same = slab->ndim == whole->ndim && slab->ndim == 3 && slab->order == whole->order && slab->dt == whole->dt &&
                slab->gamma_b == whole->gamma_b && slab->fp64 == whole->fp64;
    for (int a = 0; a < 3; ++a) same = same && slab->dx[a] == whole->dx[a];
    for (int a = 0; a < 2; ++a) same = same && slab->n[a] == whole->n[a] && slab->bc[a] == whole->bc[a];
    if (!same) return fail(slab, PIC_ERR_ARG, "slab and whole differ in dimension, x-y grid, steps, boost, shape or precision");
    if (whole->ant_on || whole->inj_on || whole->nst > 0 || slab->ant_on || slab->inj_on || slab->nst > 0)
        return fail(slab, PIC_ERR_STATE, "antenna, injection plane and stations are not carried over to a slab");
    pic_status st = pic_synchronize(whole);
    if (st != PIC_OK) return fail(slab, st, "whole: %s", whole->err.c_str());
    if ((st = pic_synchronize(slab)) != PIC_OK) return st;
    int phase = 0;
    cudaSetDevice(whole->device);
    CUDA_OR_FAIL(slab, cudaMemcpy(&phase, whole->h.phase, sizeof(int), cudaMemcpyDeviceToHost));
    cudaSetDevice(slab->device);
    InstDev &h = slab->h;
    const InstDev &w = whole->h;
    h.ion = w.ion;
    h.ion_n0 = w.ion_n0;
    h.ion_zs = w.ion_zs;
    h.ion_ramp = w.ion_ramp;
    h.ion_gb = w.ion_gb;
    h.ion_beta = w.ion_beta;
    h.ion_z0 = w.ion_z0 + k_origin * slab->dx[2];
    h.ion_lz = w.ion_lz;
    h.ion_periodic = w.ion_periodic;
    h.ion_k0 = k_lo;
    h.ion_k1 = k_hi;
    slab->step = whole->step;
    slab->mx_phases = whole->mx_phases;
    CUDA_OR_FAIL(slab, cudaMemcpyAsync(h.phase, &phase, sizeof(int), cudaMemcpyHostToDevice, slab->stream));
    slab->version++;
    destroy_graph(slab);
    return upload_inst(slab);
}

extern "C" pic_status pic_get_diagnostics(pic_ctx *ctx, pic_diag *out)
{
    if (!ctx || !out) return PIC_ERR_ARG;
    if (ctx->is_batch) return fail(ctx, PIC_ERR_ARG, "getters take a member, not a batch");
    cudaSetDevice(ctx->device);
    std::memset(out, 0, sizeof(*out));
    // the reductions, the live count and the read-back queued behind the work in flight,
    // with one synchronisation; the particle sums skip an instance whose error word is set
    // (its layout may be half written), and that error is what the call returns
    cudaStream_t s = ctx->stream;
    CUDA_OR_FAIL(ctx, cudaMemsetAsync(ctx->d_sums, 0, 3 * sizeof(double), s));
    if (ctx->loaded) CUDA_OR_FAIL(ctx, launch_particle_sums(ctx->fp64, ctx->L, ctx->d_sums, s));
    CUDA_OR_FAIL(ctx, launch_field_energy(ctx->fp64, ctx->L, ctx->d_sums, s));
    if (ctx->loaded) CUDA_OR_FAIL(ctx, launch_scan(ctx->L, 1, ctx->d_start_ptr, s));
    double sums[3];
    unsigned long long lost = 0;
    int live = 0, err = 0;
    CUDA_OR_FAIL(ctx, cudaMemcpyAsync(sums, ctx->d_sums, sizeof(sums), cudaMemcpyDeviceToHost, s));
    CUDA_OR_FAIL(ctx, cudaMemcpyAsync(&lost, ctx->h.lost, sizeof(lost), cudaMemcpyDeviceToHost, s));
    if (ctx->loaded) CUDA_OR_FAIL(ctx, cudaMemcpyAsync(&live, ctx->h.live, sizeof(int), cudaMemcpyDeviceToHost, s));
    CUDA_OR_FAIL(ctx, cudaMemcpyAsync(&err, ctx->h.err, sizeof(int), cudaMemcpyDeviceToHost, s));
    CUDA_OR_FAIL(ctx, cudaStreamSynchronize(s));
    CUDA_OR_FAIL(ctx, cudaGetLastError());
    out->error_flags = err;
    pic_status st = device_error_status(ctx, err);
    if (st != PIC_OK) return st;
    out->step = ctx->step;
    out->t = ctx->step * ctx->dt;
    out->kinetic_energy = sums[0];
    out->total_charge = sums[1];
    out->field_energy = sums[2];
    out->n_particles = live;
    out->n_lost = (int64_t)lost;
    return PIC_OK;
}

// ------------------------------------------------------------------------------------
// profiling
// ------------------------------------------------------------------------------------
static pic_status fold_timings(pic_ctx *c)
{
    CUDA_OR_FAIL(c, cudaStreamSynchronize(c->stream));
    for (int s = 0; s < c->ev_steps; ++s)
        for (int ph = 0; ph < kPhases; ++ph) {
            if (!c->recorded[(size_t)s * kPhases + ph]) continue;
            c->recorded[(size_t)s * kPhases + ph] = 0;
            cudaEvent_t a = c->events[(size_t)(s * kPhases + ph) * 2], b = c->events[(size_t)(s * kPhases + ph) * 2 + 1];
            float ms = 0.f;
            CUDA_OR_FAIL(c, cudaEventElapsedTime(&ms, a, b));
            double *dst = ph == 0 ? &c->acc.ms_particles : ph == 1 ? &c->acc.ms_scan : ph == 2 ? &c->acc.ms_filter
                          : ph == 3 ? &c->acc.ms_maxwell : &c->acc.ms_other;
            *dst += ms;
        }
    c->ev_steps = 0;
    return PIC_OK;
}

extern "C" pic_status pic_set_profiling(pic_ctx *ctx, int on, int reset)
{
    if (!ctx) return PIC_ERR_ARG;
    cudaSetDevice(ctx->device);
    if (on && ctx->events.empty()) {
        ctx->events.resize((size_t)kEventSteps * kPhases * 2);
        ctx->recorded.assign((size_t)kEventSteps * kPhases, 0);
        for (auto &e : ctx->events) CUDA_OR_FAIL(ctx, cudaEventCreate(&e));
    }
    if (ctx->profiling && !on) {
        pic_status st = fold_timings(ctx);
        if (st != PIC_OK) return st;
    }
    if (reset) {
        if (!ctx->events.empty()) {
            pic_status st = fold_timings(ctx);
            if (st != PIC_OK) return st;
        }
        std::memset(&ctx->acc, 0, sizeof(ctx->acc));
    }
    ctx->profiling = on != 0;
    return PIC_OK;
}

extern "C" pic_status pic_get_timings(pic_ctx *ctx, pic_timings *out)
{
    if (!ctx || !out) return PIC_ERR_ARG;
    cudaSetDevice(ctx->device);
    if (!ctx->events.empty()) {
        pic_status st = fold_timings(ctx);
        if (st != PIC_OK) return st;
    }
    *out = ctx->acc;
    return PIC_OK;
}

// ------------------------------------------------------------------------------------
// batching
// ------------------------------------------------------------------------------------
// ------------------------------------------------------------------------------------
// lab-frame stations
// ------------------------------------------------------------------------------------
extern "C" pic_status pic_set_stations(pic_ctx *ctx, int count, const double *z_lab, int max_records)
{
    if (!ctx) return PIC_ERR_ARG;
    if (ctx->is_batch) return fail(ctx, PIC_ERR_ARG, "pic_set_stations takes a member, not a batch");
    if (count < 0 || (count > 0 && (!z_lab || max_records < 1)))
        return fail(ctx, PIC_ERR_ARG, "need count >= 0, z_lab and max_records >= 1");
    for (int i = 0; i < count; ++i)
        if (!std::isfinite(z_lab[i])) return fail(ctx, PIC_ERR_NAN, "station %d position not finite", i);
    cudaSetDevice(ctx->device);
    CUDA_OR_FAIL(ctx, cudaStreamSynchronize(ctx->stream));
    dfree(ctx, ctx->d_st_z);
    dfree(ctx, ctx->d_st_t);
    dfree(ctx, ctx->d_st_count);
    dfree(ctx, ctx->d_st_fields);
    ctx->d_st_z = ctx->d_st_t = nullptr;
    ctx->d_st_count = nullptr;
    ctx->d_st_fields = nullptr;
    ctx->nst = 0;
    ctx->st_max = 0;
    destroy_graph(ctx);
    if (count == 0) return PIC_OK;
    const size_t plane = (size_t)ctx->n[0] * ctx->n[1];
    ctx->d_st_z = (double *)dalloc(ctx, sizeof(double) * count);
    ctx->d_st_t = (double *)dalloc(ctx, sizeof(double) * count * (size_t)max_records);
    ctx->d_st_count = (int *)dalloc(ctx, sizeof(int) * count);
    ctx->d_st_fields = dalloc(ctx, ctx->es * 6 * plane * count * (size_t)max_records);
    if (!ctx->d_st_z || !ctx->d_st_t || !ctx->d_st_count || !ctx->d_st_fields)
        return fail(ctx, PIC_ERR_OOM, "no device memory for %d stations x %d records", count, max_records);
    CUDA_OR_FAIL(ctx, cudaMemcpyAsync(ctx->d_st_z, z_lab, sizeof(double) * count, cudaMemcpyHostToDevice, ctx->stream));
    CUDA_OR_FAIL(ctx, cudaMemsetAsync(ctx->d_st_count, 0, sizeof(int) * count, ctx->stream));
    CUDA_OR_FAIL(ctx, cudaStreamSynchronize(ctx->stream));
    ctx->nst = count;
    ctx->st_max = max_records;
    if (ctx->loaded) {  // the current state is the first record
        StationDev S{ctx->d_st_z, ctx->d_st_count, ctx->d_st_t, ctx->d_st_fields, ctx->st_max};
        CUDA_OR_FAIL(ctx, launch_stations(ctx->fp64, ctx->d_inst, S, ctx->nst, (int)plane, ctx->stream));
        CUDA_OR_FAIL(ctx, cudaStreamSynchronize(ctx->stream));
    }
    return PIC_OK;
}

extern "C" pic_status pic_get_station(pic_ctx *ctx, int station, int *n_records, double *t_lab, size_t t_count,
                                      double *fields, size_t f_count)
{
    if (!ctx) return PIC_ERR_ARG;
    if (ctx->is_batch) return fail(ctx, PIC_ERR_ARG, "pic_get_station takes a member, not a batch");
    if (station < 0 || station >= ctx->nst) return fail(ctx, PIC_ERR_ARG, "no station %d", station);
    if (!n_records) return fail(ctx, PIC_ERR_ARG, "n_records is NULL");
    cudaSetDevice(ctx->device);
    pic_status st = pic_synchronize(ctx);
    if (st != PIC_OK) return st;
    int n = 0;
    CUDA_OR_FAIL(ctx, d2h(ctx, &n, ctx->d_st_count + station, sizeof(int)));
    *n_records = n;
    const size_t plane = (size_t)ctx->n[0] * ctx->n[1];
    if (t_lab) {
        if (t_count < (size_t)n) return fail(ctx, PIC_ERR_ARG, "t_lab needs room for %d values", n);
        CUDA_OR_FAIL(ctx, d2h(ctx, t_lab, ctx->d_st_t + (size_t)station * ctx->st_max, sizeof(double) * n));
    }
    if (fields) {
        const size_t need = (size_t)n * 6 * plane;
        if (f_count < need) return fail(ctx, PIC_ERR_ARG, "fields needs room for %zu values", need);
        const unsigned char *src = (const unsigned char *)ctx->d_st_fields + (size_t)station * ctx->st_max * 6 * plane * ctx->es;
        if (ctx->fp64) {
            CUDA_OR_FAIL(ctx, d2h(ctx, fields, src, sizeof(double) * need));
        } else {
            std::vector<float> tmp(need);
            CUDA_OR_FAIL(ctx, d2h(ctx, tmp.data(), src, sizeof(float) * need));
            for (size_t i = 0; i < need; ++i) fields[i] = tmp[i];
        }
    }
    return PIC_OK;
}

static pic_status refresh_batch(pic_ctx *c)
{
    bool stale = c->member_versions.size() != c->members.size();
    for (size_t i = 0; !stale && i < c->members.size(); ++i) stale = c->member_versions[i] != c->members[i]->version;
    for (auto m : c->members)
        if (!m->loaded) return fail(c, PIC_ERR_STATE, "a batch member has no particles loaded");
    if (!stale) return PIC_OK;
    const int n = (int)c->members.size();
    std::vector<InstDev> insts(n);
    std::vector<int> ts(n + 1, 0);
    std::vector<long long> cs(n + 1, 0);
    for (int i = 0; i < n; ++i) {
        insts[i] = c->members[i]->h;
        insts[i].tile_base = ts[i];
        ts[i + 1] = ts[i] + insts[i].ntiles;
        cs[i + 1] = cs[i] + c->members[i]->ncell;
    }
    CUDA_OR_FAIL(c, cudaMemcpyAsync(c->d_inst, insts.data(), sizeof(InstDev) * n, cudaMemcpyHostToDevice, c->stream));
    CUDA_OR_FAIL(c, cudaMemcpyAsync(c->d_tile_start, ts.data(), sizeof(int) * (n + 1), cudaMemcpyHostToDevice, c->stream));
    CUDA_OR_FAIL(c, cudaMemcpyAsync(c->d_cell_start, cs.data(), sizeof(long long) * (n + 1), cudaMemcpyHostToDevice, c->stream));
    std::vector<long long> ps((size_t)4 * (n + 1), 0);
    for (int a = 0; a < 4; ++a) {
        for (int i = 0; i < n; ++i) ps[(size_t)a * (n + 1) + i + 1] = ps[(size_t)a * (n + 1) + i] + c->members[i]->pencil_total[a];
        c->pencil_total[a] = ps[(size_t)a * (n + 1) + n];
    }
    CUDA_OR_FAIL(c, cudaMemcpyAsync(c->d_pencil, ps.data(), sizeof(long long) * ps.size(), cudaMemcpyHostToDevice, c->stream));
    CUDA_OR_FAIL(c, cudaStreamSynchronize(c->stream));
    c->L.total_tiles = ts[n];
    c->L.total_cells = cs[n];
    c->member_versions.clear();
    for (auto m : c->members) c->member_versions.push_back(m->version);
    destroy_graph(c);
    return PIC_OK;
}

static void *plan_alloc(void *user, size_t bytes) { return dalloc((pic_ctx *)user, bytes); }

extern "C" pic_status pic_batch_set_persistent(pic_ctx *batch, int on, long long spin_limit, int test_stall)
{
    if (!batch) return PIC_ERR_ARG;
    if (!batch->is_batch) return fail(batch, PIC_ERR_ARG, "pic_batch_set_persistent takes a batch");
    cudaSetDevice(batch->device);
    CUDA_OR_FAIL(batch, cudaStreamSynchronize(batch->stream));
    if (!on) {
        batch->persistent = false;
        return PIC_OK;
    }
    const int n = (int)batch->members.size();
    if (test_stall < -1 || test_stall >= n) return fail(batch, PIC_ERR_ARG, "test_stall %d outside -1 .. %d", test_stall, n - 1);
    const int passes = batch->members[0]->opt.filter_passes;
    for (auto m : batch->members) {
        if (m->fp64) return fail(batch, PIC_ERR_UNSUPPORTED, "the persistent step runs FP32 instances");
        if (m->opt.pusher != PIC_PUSHER_VAY) return fail(batch, PIC_ERR_UNSUPPORTED, "the persistent step runs the Vay pusher");
        if (m->opt.solver != PIC_SOLVER_YEE) return fail(batch, PIC_ERR_UNSUPPORTED, "the persistent step runs the Yee solver");
        if (m->ant_on || m->inj_on || m->nst > 0)
            return fail(batch, PIC_ERR_UNSUPPORTED, "the persistent step runs without antenna, injection plane and stations");
        if (m->opt.filter_passes != passes || passes > 4)
            return fail(batch, PIC_ERR_UNSUPPORTED, "the persistent step needs one filter pass count of at most 4");
    }
    if (!batch->plan) {
        std::vector<PersistCounts> counts(n);
        for (int i = 0; i < n; ++i) {
            const pic_ctx *m = batch->members[i];
            PersistCounts &k = counts[i];
            k.ncell = m->ncell;
            k.ntiles = m->h.ntiles;
            for (int a = 0; a < 3; ++a) {
                k.pencils[a] = m->pencil_total[a];
                const int o1 = a == 0 ? 1 : 0, o2 = a == 2 ? 1 : 2;
                k.ghost[a] = m->any_periodic[a] ? 6LL * 2 * m->h.gh[a] * m->h.P[o1] * m->h.P[o2] : 0;
            }
            k.mx_tiles = m->pencil_total[3];
        }
        PersistPlan *plan = new PersistPlan;
        cudaError_t e = plan->build(counts, plan_alloc, batch);
        if (e != cudaSuccess) {
            delete plan;
            return fail(batch, e == cudaErrorMemoryAllocation ? PIC_ERR_OOM : PIC_ERR_CUDA, "work list: %s", cudaGetErrorString(e));
        }
        batch->plan = plan;
        batch->persist_smem = persist_smem(batch->ndim, batch->smem);
        int bps = 0, sms = 0;
        CUDA_OR_FAIL(batch, persist_blocks_per_sm(batch->ndim, batch->order, batch->persist_smem, &bps));
        CUDA_OR_FAIL(batch, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, batch->device));
        if (bps < 1) return fail(batch, PIC_ERR_UNSUPPORTED, "the persistent kernel does not fit an SM");
        batch->persist_grid = bps * sms;
    }
    batch->spin_limit = spin_limit > 0 ? spin_limit : (1LL << 21);
    batch->stall_inst = test_stall;
    batch->persistent = true;
    return PIC_OK;
}

// Times `steps` steps of each launch form on the batch itself (real steps of the run,
// CUDA events on its stream) and keeps the faster one on.
extern "C" pic_status pic_batch_autotune(pic_ctx *batch, int steps, int *persistent, double *ms_graph,
                                         double *ms_persistent)
{
    if (!batch) return PIC_ERR_ARG;
    if (!batch->is_batch) return fail(batch, PIC_ERR_ARG, "pic_batch_autotune takes a batch");
    if (steps < 1) return fail(batch, PIC_ERR_ARG, "steps must be >= 1");
    if (batch->profiling) return fail(batch, PIC_ERR_STATE, "pic_batch_autotune with profiling on");
    cudaSetDevice(batch->device);
    const bool was = batch->persistent;
    const long long spin = batch->spin_limit;
    // the persistent form, when the batch admits it
    pic_status st = pic_batch_set_persistent(batch, 1, spin, -1);
    const bool can_persist = st == PIC_OK;
    if (!can_persist) batch->err.clear();
    double ms[2] = {-1.0, -1.0};
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CUDA_OR_FAIL(batch, cudaEventCreate(&e0));
    CUDA_OR_FAIL(batch, cudaEventCreate(&e1));
    for (int form = 0; form < 2 && st != PIC_ERR_CUDA; ++form) {
        if (form == 1 && !can_persist) break;
        batch->persistent = form == 1;
        // one untimed step builds the graph or warms the persistent kernel
        if ((st = pic_step(batch, 1)) != PIC_OK || (st = pic_synchronize(batch)) != PIC_OK) break;
        cudaEventRecord(e0, batch->stream);
        if ((st = pic_step(batch, steps)) != PIC_OK) break;
        cudaEventRecord(e1, batch->stream);
        if ((st = pic_synchronize(batch)) != PIC_OK) break;
        float t = 0.f;
        cudaEventElapsedTime(&t, e0, e1);
        ms[form] = t / steps;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != PIC_OK) {
        batch->persistent = was;
        return st;
    }
    batch->persistent = can_persist && ms[1] < ms[0];
    if (persistent) *persistent = batch->persistent ? 1 : 0;
    if (ms_graph) *ms_graph = ms[0];
    if (ms_persistent) *ms_persistent = ms[1];
    return PIC_OK;
}

extern "C" pic_status pic_batch_create(int n, pic_ctx *const *instances, pic_ctx **batch)
{
    if (!batch) return fail(nullptr, PIC_ERR_ARG, "batch is NULL");
    *batch = nullptr;
    if (n < 1 || !instances) return fail(nullptr, PIC_ERR_ARG, "need at least one instance");
    pic_ctx *f = instances[0];
    for (int i = 0; i < n; ++i) {
        pic_ctx *m = instances[i];
        if (!m || m->is_batch) return fail(nullptr, PIC_ERR_ARG, "instance %d is NULL or a batch", i);
        if (m->ndim != f->ndim || m->order != f->order || m->fp64 != f->fp64 || m->opt.pusher != f->opt.pusher ||
            m->opt.solver != f->opt.solver || m->device != f->device || m->smem != f->smem ||
            m->h.ts[0] != f->h.ts[0] || m->h.ts[1] != f->h.ts[1] || m->h.ts[2] != f->h.ts[2])
            return fail(nullptr, PIC_ERR_ARG,
                        "instance %d differs in dimension, shape, precision, pusher, field solver, tile or device", i);
        for (int j = 0; j < i; ++j)
            if (instances[j] == m) return fail(nullptr, PIC_ERR_ARG, "instance %d appears twice", i);
    }
    pic_ctx *c = new pic_ctx();
    c->is_batch = true;
    c->members.assign(instances, instances + n);
    c->ndim = f->ndim;
    c->order = f->order;
    c->fp64 = f->fp64;
    c->es = f->es;
    c->opt = f->opt;
    c->device = f->device;
    c->stream = f->stream;
    c->smem = f->smem;
    c->h = f->h;
    c->d_inst = (InstDev *)dalloc(c, sizeof(InstDev) * n);
    c->d_tile_start = (int *)dalloc(c, sizeof(int) * (n + 1));
    c->d_cell_start = (long long *)dalloc(c, sizeof(long long) * (n + 1));
    c->d_pencil = (long long *)dalloc(c, sizeof(long long) * 4 * (n + 1));
    if (!c->d_inst || !c->d_tile_start || !c->d_cell_start || !c->d_pencil) {
        dfree_all(c);
        delete c;
        return fail(nullptr, PIC_ERR_OOM, "batch tables do not fit");
    }
    for (auto m : c->members) {
        for (int a = 0; a < 3; ++a) c->any_periodic[a] = c->any_periodic[a] || m->any_periodic[a];
        c->ghost_max = std::max(c->ghost_max, m->ghost_max);
        c->max_sweeps = std::max(c->max_sweeps, m->max_sweeps);
    }
    c->L.inst = c->d_inst;
    c->L.tile_start = c->d_tile_start;
    c->L.cell_start = c->d_cell_start;
    c->L.ninst = n;
    *batch = c;
    return PIC_OK;
}
