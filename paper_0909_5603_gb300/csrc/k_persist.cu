// k_persist.cu -- the persistent batched step: every phase of a batch's steps (ion
// current, J set-up, scan, source records, particles, filter sweeps, fused Yee update,
// buffer switch, periodic ghost copies) run by one launch of CTAs that pull work items
// from a device list.
//
// The list orders the items by (step, phase, instance, item).  A CTA takes the next item
// with one atomic add, waits until the item's instance has completed every item of its
// previous phase (a per-(phase, instance) counter), runs the item with the phase's device
// function and counts it done.  An item waits only for items earlier in the list, which
// CTAs that are running already hold, so the launch makes progress at any grid size;
// instances do not wait for one another, so the small instances of an uneven batch flow
// through their phases while large ones are still in theirs.  Every wait is bounded: past
// the spin limit the item's instance gets PIC_ERR_TIMEOUT, the launch is marked aborted
// and every CTA leaves at its next item.
#include "k_fields.cuh"
#include "k_ions.cuh"
#include "k_particles.cuh"

#include <algorithm>

namespace pic {

enum PersistPhase : int {
    kPhIonFaces,
    kPhJInit,
    kPhScan,
    kPhSources,
    kPhParticles,
    kPhFilterX,
    kPhFilterY,
    kPhFilterZ,
    kPhMaxwell,
    kPhFlip,
    kPhGhostX,
    kPhGhostY,
    kPhGhostZ,
    kPhCount
};

// Items per instance and phase; a phase without work for an instance has one item that
// does nothing, so that every instance's phases chain through every phase.
struct PersistDesc {
    int ninst, nsteps, passes, filtered;
    long long per_step;                   // items per step
    long long phase_base[kPhCount + 1];   // first item of each phase within a step
    const long long *pre;                 // [kPhCount][ninst + 1] item offsets per instance
    const long long *pencil[3];           // filter pencil offsets per axis (ninst + 1 each)
    const long long *mx_start;            // fused Yee tile offsets (ninst + 1)
    unsigned long long *cursor;           // next item
    int *done;                            // [kPhCount][ninst] completed items
    int *abort_flag;
    long long spin_limit;                 // polls of a counter before a wait gives up
    int stall_inst;                       // test: this instance's J set-up waits for an item that never runs
};

constexpr int kJInitCells = 4096;  // cells per J set-up item (16 per thread)
constexpr int kGhostElems = 4096;  // elements per ghost-copy item

__device__ __forceinline__ int ld_acquire(const int *p)
{
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Polls *p until it reaches need (0), the limit runs out (1) or another CTA aborts the
// launch (2).
__device__ __forceinline__ int wait_count(const int *p, long long need, long long limit, const int *abort_flag)
{
    for (long long it = 0; it <= limit; ++it) {
        if (ld_acquire(p) >= need) return 0;
        if ((it & 63) == 63 && *(volatile const int *)abort_flag) return 2;
        __nanosleep(64);
    }
    return 1;
}

template <int P>
__device__ __forceinline__ void filter_item(const Launch &L, const long long *pen, int axis, int src_is_jt, long long g,
                                            float *win)
{
    if (axis == 0)
        filter_row_block<float, P>(L, pen, src_is_jt, g, win);
    else
        filter_col_block<float, P>(L, axis, pen, src_is_jt, g);
}

// Each phase body as a function of its own (not inlined), so that the registers of one
// phase do not crowd the others.
template <int ND, int ORD>
__device__ __noinline__ void particle_item(const Launch &L, int g)
{
    particle_tile_of_launch<ND, ORD, float, 0, false>(L, g);
}

template <int ND>
__device__ __noinline__ void maxwell_item(const Launch &L, const long long *mx_start, int filtered, long long g)
{
    maxwell_fused_block<float, ND>(L, mx_start, filtered, g);
}

__device__ __noinline__ void filter_any(const Launch &L, const long long *pen, int axis, int src_is_jt, long long g,
                                        float *win, int passes)
{
    switch (passes) {
    case 1: filter_item<1>(L, pen, axis, src_is_jt, g, win); break;
    case 2: filter_item<2>(L, pen, axis, src_is_jt, g, win); break;
    case 3: filter_item<3>(L, pen, axis, src_is_jt, g, win); break;
    default: filter_item<4>(L, pen, axis, src_is_jt, g, win); break;
    }
}

__device__ __noinline__ void sources_item(const Launch &L, int g, SrcScratch *S, int lane)
{
    tile_sources_warp(L, g, *S, lane);
}

template <int ND, int ORD>
__global__ void __launch_bounds__(kNT, 2) k_step_persistent(Launch L, PersistDesc D)
{
    extern __shared__ __align__(128) unsigned char dyn[];
    __shared__ long long s_item;
    __shared__ int s_ok;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const long long total = D.per_step * D.nsteps;
    for (;;) {
        __syncthreads();  // every thread is done with the previous item
        if (tid == 0) {
            long long q = -1;
            if (!*(volatile int *)D.abort_flag) q = (long long)atomicAdd(D.cursor, 1ULL);
            s_item = q < total ? q : -1;
        }
        __syncthreads();
        const long long q = s_item;
        if (q < 0) break;
        const int step = (int)(q / D.per_step);
        const long long w = q - (long long)step * D.per_step;
        int p = 0;  // (constant indices: the descriptor stays in the parameter space)
#pragma unroll
        for (int k = 1; k < kPhCount; ++k) p += w >= D.phase_base[k] ? 1 : 0;
        long long pbase = 0;
#pragma unroll
        for (int k = 0; k < kPhCount; ++k) pbase = k == p ? D.phase_base[k] : pbase;
        const long long *pre = D.pre + (size_t)p * (D.ninst + 1);
        const long long wp = w - pbase;
        const int ii = find_instance_ll(pre, D.ninst, wp);
        const long long local = wp - pre[ii];
        if (tid == 0) {
            // the instance's previous phase: this step's, or the last one of the step before
            const int pp = p > 0 ? p - 1 : kPhCount - 1;
            const long long *ppre = D.pre + (size_t)pp * (D.ninst + 1);
            const long long cnt = ppre[ii + 1] - ppre[ii];
            long long need = p > 0 ? (long long)(step + 1) * cnt : (long long)step * cnt;
            if (p == kPhJInit && ii == D.stall_inst) need += 1;
            const int w8 = wait_count(D.done + (size_t)pp * D.ninst + ii, need, D.spin_limit, D.abort_flag);
            const bool ok = w8 == 0;
            if (w8 == 1) {
                atomicOr(L.inst[ii].err, kErrTimeout);
                atomicExch(D.abort_flag, 1);
            }
            // the fields the item reads through TMA were written through the generic proxy
            asm volatile("fence.proxy.async;" ::: "memory");
            s_ok = ok ? 1 : 0;
        }
        __syncthreads();
        if (!s_ok) break;
        const InstDev &I = L.inst[ii];
        switch (p) {
        case kPhIonFaces:
            ion_faces_of<float>(I, tid, kNT);
            break;
        case kPhJInit: {
            const long long ncell = (long long)I.n[0] * I.n[1] * I.n[2];
            for (long long r = local * kJInitCells + tid; r < min(ncell, (local + 1) * kJInitCells); r += kNT) {
                const int rq = fast_div((int)r, I.div_n0);
                const int i = (int)r - rq * I.n[0];
                const int k = fast_div(rq, I.div_n1);
                const int j = rq - k * I.n[1];
                const long long pc = (i + I.gh[0]) + I.sy * (j + I.gh[1]) + I.sz * (k + I.gh[2]);
                ((float *)I.J[0])[pc] = 0.f;
                ((float *)I.J[1])[pc] = 0.f;
                ((float *)I.J[2])[pc] = I.ion ? ((const float *)I.ion_face)[k] : 0.f;
            }
            break;
        }
        case kPhScan:
            scan_instance(L, ii, 0, nullptr, (int *)dyn);  // small: inlined
            break;
        case kPhSources: {
            const long long t = local * 8 + warp;
            if (t < I.ntiles) sources_item(L, (int)(L.tile_start[ii] + t), (SrcScratch *)dyn + warp, lane);
            break;
        }
        case kPhParticles:
            particle_item<ND, ORD>(L, (int)(L.tile_start[ii] + local));
            break;
        case kPhFilterX:
        case kPhFilterY:
        case kPhFilterZ: {
            const int axis = p - kPhFilterX;
            const long long *pen = axis == 0 ? D.pencil[0] : (axis == 1 ? D.pencil[1] : D.pencil[2]);
            const long long npen = pen[ii + 1] - pen[ii];
            if (D.passes < 1 || local >= npen) break;
            // sweep k of the step reads J when k is even, Jt when odd (2D has no y sweep)
            const int sweep = (ND == 3 || axis == 0) ? axis : 1;
            const long long g = pen[ii] + local;
            filter_any(L, pen, axis, sweep & 1, g, (float *)dyn, D.passes);
            break;
        }
        case kPhMaxwell:
            maxwell_item<ND>(L, D.mx_start, D.filtered, D.mx_start[ii] + local);
            break;
        case kPhFlip:
            if (tid == 0) *I.fpar ^= 1;
            break;
        default: {  // ghost copies
            const int axis = p - kPhGhostX;
            const long long ne = min(ghost_elems(I, axis), (local + 1) * kGhostElems);
            for (long long r = local * kGhostElems + tid; r < ne; r += kNT) ghost_elem<float>(I, axis, r);
            break;
        }
        }
        __syncthreads();
        if (tid == 0) {
            __threadfence();
            atomicAdd(D.done + (size_t)p * D.ninst + ii, 1);
        }
    }
}

// ---- host side --------------------------------------------------------------------------
struct PersistPlan::Impl {
    int ninst = 0;
    long long per_step = 0;
    long long phase_base[kPhCount + 1] = {};
    long long *d_pre = nullptr;
    unsigned long long *d_counters = nullptr;  // cursor, abort flag, done[kPhCount][ninst]
    size_t counter_bytes = 0;
};

template <int ND, int ORD>
static cudaError_t persist_launch(const Launch &L, const PersistDesc &D, size_t smem, int grid, cudaStream_t s)
{
    k_step_persistent<ND, ORD><<<grid, kNT, smem, s>>>(L, D);
    return cudaGetLastError();
}

template <int ND, int ORD>
static cudaError_t persist_prepare(size_t smem, int *blocks_per_sm)
{
    cudaError_t e = cudaFuncSetAttribute(k_step_persistent<ND, ORD>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_step_persistent<ND, ORD>, kNT, smem);
}

static cudaError_t persist_dispatch(int ndim, int order, bool prepare, const Launch *L, const PersistDesc *D, size_t smem,
                                    int grid, int *bps, cudaStream_t s)
{
#define PIC_PERSIST(ND, ORD) \
    if (ndim == ND && order == ORD) return prepare ? persist_prepare<ND, ORD>(smem, bps) : persist_launch<ND, ORD>(*L, *D, smem, grid, s);
    PIC_PERSIST(2, 1) PIC_PERSIST(2, 2) PIC_PERSIST(3, 1) PIC_PERSIST(3, 2)
#undef PIC_PERSIST
    return cudaErrorInvalidValue;
}

size_t persist_smem(int ndim, size_t particle_smem)
{
    // the particle phase's dynamic shared memory, or the largest scratch of another phase
    size_t m = particle_smem;
    m = std::max(m, ndim == 3 ? maxwell_fused_smem<float, 3>() : maxwell_fused_smem<float, 2>());
    m = std::max(m, sizeof(float) * 8 * 3 * (size_t)(kPencil + 2 * 4) + 128);
    m = std::max(m, sizeof(SrcScratch) * 8 + 128);
    m = std::max(m, sizeof(int) * 66 + 128);
    return m;
}

cudaError_t persist_blocks_per_sm(int ndim, int order, size_t smem, int *bps)
{
    return persist_dispatch(ndim, order, true, nullptr, nullptr, smem, 0, bps, 0);
}

PersistPlan::PersistPlan() : impl(new Impl) {}
PersistPlan::~PersistPlan() { delete impl; }

cudaError_t PersistPlan::build(const std::vector<PersistCounts> &inst, void *(*alloc)(void *, size_t), void *user)
{
    const int n = (int)inst.size();
    impl->ninst = n;
    std::vector<long long> pre((size_t)kPhCount * (n + 1), 0);
    long long base = 0;
    for (int p = 0; p < kPhCount; ++p) {
        impl->phase_base[p] = base;
        for (int i = 0; i < n; ++i) {
            long long c = 1;
            const PersistCounts &k = inst[i];
            switch (p) {
            case kPhJInit: c = (k.ncell + kJInitCells - 1) / kJInitCells; break;
            case kPhSources: c = (k.ntiles + 7) / 8; break;
            case kPhParticles: c = k.ntiles; break;
            case kPhFilterX: case kPhFilterY: case kPhFilterZ: c = k.pencils[p - kPhFilterX]; break;
            case kPhMaxwell: c = k.mx_tiles; break;
            case kPhGhostX: case kPhGhostY: case kPhGhostZ: c = (k.ghost[p - kPhGhostX] + kGhostElems - 1) / kGhostElems; break;
            default: c = 1;
            }
            if (c < 1) c = 1;
            pre[(size_t)p * (n + 1) + i + 1] = pre[(size_t)p * (n + 1) + i] + c;
        }
        base += pre[(size_t)p * (n + 1) + n];
    }
    impl->phase_base[kPhCount] = base;
    impl->per_step = base;
    impl->d_pre = (long long *)alloc(user, sizeof(long long) * pre.size());
    impl->counter_bytes = sizeof(unsigned long long) * 2 + sizeof(int) * (size_t)kPhCount * n;
    impl->d_counters = (unsigned long long *)alloc(user, impl->counter_bytes);
    if (!impl->d_pre || !impl->d_counters) return cudaErrorMemoryAllocation;
    return cudaMemcpy(impl->d_pre, pre.data(), sizeof(long long) * pre.size(), cudaMemcpyHostToDevice);
}

long long PersistPlan::items_per_step() const { return impl->per_step; }

cudaError_t PersistPlan::launch(const Launch &L, int ndim, int order, int nsteps, int passes, int filtered,
                                const long long *pencil_tables, const long long *mx_start, size_t smem, int grid,
                                long long spin_limit, int stall_inst, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(impl->d_counters, 0, impl->counter_bytes, s);
    if (e != cudaSuccess) return e;
    PersistDesc D{};
    D.ninst = impl->ninst;
    D.nsteps = nsteps;
    D.passes = passes;
    D.filtered = filtered;
    D.per_step = impl->per_step;
    for (int p = 0; p <= kPhCount; ++p) D.phase_base[p] = impl->phase_base[p];
    D.pre = impl->d_pre;
    for (int a = 0; a < 3; ++a) D.pencil[a] = pencil_tables + (size_t)a * (impl->ninst + 1);
    D.mx_start = mx_start;
    D.cursor = impl->d_counters;
    D.abort_flag = (int *)(impl->d_counters + 1);
    D.done = (int *)(impl->d_counters + 2);
    D.spin_limit = spin_limit;
    D.stall_inst = stall_inst;
    return persist_dispatch(ndim, order, false, &L, &D, smem, grid, nullptr, s);
}

}  // namespace pic
