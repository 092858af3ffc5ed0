// k_particles.cuh -- the particle half of the boosted-frame PIC step on sm_103a.
//
// One CTA per particle tile.  It stages the tile's E and B plus guard cells into shared
// memory with TMA bulk-tensor copies, loads the tile's particles from the previous
// step's layout (the moved-in sub-ranges of the 27 neighbouring tiles), and for each
// particle: gathers E, B (shape order 1 or 2, each component at its Yee position), pushes
// u with the Vay (or Boris) pusher (Sec. 2 of the paper), moves it, and deposits the
// charge-conserving Esirkepov current into a shared-memory J tile.  Each chunk of
// particles is written out stably partitioned by the tile it moved to, so the next
// step finds every tile's particles in contiguous sub-ranges: the array stays sorted
// by tile at every step with no separate sort pass.  The J tile is flushed to global
// memory once, with wrap-around (periodic) or clipping (absorbing) of its guard cells.
#pragma once

#include "pic_device.cuh"

namespace pic {

constexpr int kNT = 256;          // threads per particle CTA
constexpr int kNW = kNT / 32;
constexpr int kChunk = kNT;       // particles per chunk: one per thread
constexpr long long kWaitCycles = 2000000000LL;  // ~1 s at GB300 clocks

// -------------------------------------------------------------------------------------
// Source table of one destination tile: the (tile, direction) pairs whose particles
// move into it, in ascending source-tile order (so the concatenation is the stable
// order of the previous array).
// -------------------------------------------------------------------------------------
constexpr int kMaxSub = 512;  // sub-ranges cached in shared memory per destination tile

struct SrcTable {
    int n;                      // sources (<= 27), ascending source tile
    int count;                  // particles moving into the tile
    int tile[kDirs];
    int dir[kDirs];
    int pre[kDirs + 1];         // prefix of the sources' particle counts
    int seg[kDirs];             // segment start of the source tile
    int c0[kDirs];              // first chunk record of the source tile
    int nch[kDirs];             // chunks of the source tile
    int chpre[kDirs + 1];       // prefix of nch: (source, chunk) pair index space
    int nsub;                   // non-empty (source, chunk) sub-ranges, -1 if > kMaxSub
    int sub_slot[kMaxSub + 1];  // first destination slot of each sub-range, then count
    int sub_pos[kMaxSub];       // buffer position of each sub-range's first particle
    int warp_tmp[2][32];        // two scans back to back need separate warp totals
};

// Block-wide exclusive scan of one int per thread (blockDim a multiple of 32, at most
// 1024); returns the exclusive prefix, *total the sum.  Contains two __syncthreads.
__device__ __forceinline__ int block_exclusive_scan(int v, int *tmp, int *total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) tmp[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int t = lane < nw ? tmp[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        tmp[lane] = t;  // inclusive over warps
    }
    __syncthreads();
    *total = tmp[nw - 1];
    return (warp ? tmp[warp - 1] : 0) + x - v;
}

// Valid (direction, source coordinate) pairs along one axis for destination coordinate
// T, sorted by source coordinate.  Returns how many.
__device__ __forceinline__ int axis_sources(int T, int nt, int bc, int dirs[3], int src[3])
{
    int m = 0;
    int cd[3], cs[3];
    if (bc == 0) {
        if (nt >= 3) {
            for (int d = -1; d <= 1; ++d) {
                cd[m] = d;
                cs[m] = ((T - d) % nt + nt) % nt;
                ++m;
            }
        } else if (nt == 2) {
            cd[0] = 0; cs[0] = T;
            cd[1] = 1; cs[1] = (T + 1) % 2;
            m = 2;
        } else {
            cd[0] = 0; cs[0] = T;
            m = 1;
        }
    } else {
        for (int d = -1; d <= 1; ++d) {
            const int s = T - d;
            if (s >= 0 && s < nt) {
                cd[m] = d;
                cs[m] = s;
                ++m;
            }
        }
    }
    // sort by source coordinate (m <= 3)
    for (int i = 0; i < m; ++i)
        for (int j = i + 1; j < m; ++j)
            if (cs[j] < cs[i]) {
                int a = cs[i]; cs[i] = cs[j]; cs[j] = a;
                a = cd[i]; cd[i] = cd[j]; cd[j] = a;
            }
    for (int i = 0; i < m; ++i) {
        dirs[i] = cd[i];
        src[i] = cs[i];
    }
    return m;
}

// Canonical direction along one axis from old tile coordinate to new one.
__device__ __forceinline__ int axis_dir(int told, int tnew, int nt, int bc)
{
    if (bc != 0) return tnew - told;
    int d = tnew - told;
    if (d < 0) d += nt;  // d in [0, nt)
    if (d == 0) return 0;
    if (d == 1) return 1;
    return -1;           // d == nt - 1 with nt >= 3
}

// Built by the whole CTA (every thread must call it).  `lay` = layout holding the source
// tiles.  Ends with the table complete and visible to all threads.
static __device__ void build_sources(const InstDev &I, int lay, int tx, int ty, int tz, SrcTable &S)
{
    const int tid = threadIdx.x, lane = tid & 31;
    const int *seg = I.seg[lay];
    const int *cbase = I.chunk_base[lay];
    const int *tot = I.tot[lay];
    const int *pre = I.chunk_pre[lay];
    if (tid < 32) {
        int dx[3], sx[3], dy[3], sy[3], dz[3], sz[3];
        const int mx = axis_sources(tx, I.nt[0], I.bc[0], dx, sx);
        const int my = I.ndim == 3 ? axis_sources(ty, I.nt[1], I.bc[1], dy, sy) : 1;
        if (I.ndim != 3) { dy[0] = 0; sy[0] = 0; }
        const int mz = axis_sources(tz, I.nt[2], I.bc[2], dz, sz);
        const int n = mx * my * mz;
        int cnt = 0, nch = 0;
        if (lane < n) {
            const int c = lane % mx, b = (lane / mx) % my, a = lane / (mx * my);
            const int st = sx[c] + I.nt[0] * (sy[b] + I.nt[1] * sz[a]);
            const int d = (dz[a] + 1) * 9 + (dy[b] + 1) * 3 + (dx[c] + 1);
            cnt = tot[st * kBuckets + d];
            const int c0 = cbase[st];
            nch = cbase[st + 1] - c0;
            S.tile[lane] = st;
            S.dir[lane] = d;
            S.seg[lane] = seg[st];
            S.c0[lane] = c0;
            S.nch[lane] = nch;
        }
        int pc = cnt, pn = nch;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int yc = __shfl_up_sync(0xffffffffu, pc, o);
            const int yn = __shfl_up_sync(0xffffffffu, pn, o);
            if (lane >= o) { pc += yc; pn += yn; }
        }
        if (lane < n) {
            S.pre[lane] = pc - cnt;
            S.chpre[lane] = pn - nch;
        }
        if (lane == n - 1) {
            S.pre[n] = pc;
            S.chpre[n] = pn;
            S.count = pc;
            S.n = n;
        }
    }
    __syncthreads();
    // (source, chunk) pairs -> non-empty sub-ranges, in source then chunk order
    const int npairs = S.chpre[S.n];
    int written = 0;  // sub-ranges so far (uniform)
    int slot_run = 0; // destination slots so far (uniform)
    bool fits = true;
    for (int q0 = 0; q0 < npairs; q0 += blockDim.x) {
        const int q = q0 + tid;
        int cntq = 0, posq = 0;
        if (q < npairs) {
            int s = 0, top = S.n - 1;
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
        int tot_cnt, tot_ne;
        const int ex_cnt = block_exclusive_scan(cntq, S.warp_tmp[0], &tot_cnt);
        const int ne = cntq > 0 ? 1 : 0;
        const int ex_ne = block_exclusive_scan(ne, S.warp_tmp[1], &tot_ne);
        if (written + tot_ne > kMaxSub) fits = false;
        if (fits && ne) {
            S.sub_slot[written + ex_ne] = slot_run + ex_cnt;
            S.sub_pos[written + ex_ne] = posq;
        }
        written += tot_ne;
        slot_run += tot_cnt;
        __syncthreads();
    }
    if (tid == 0) {
        S.nsub = fits ? written : -1;
        if (fits) S.sub_slot[written] = slot_run;
    }
    __syncthreads();
}

// Buffer position of slot p (0 <= p < S.count) of the destination tile.
__device__ __forceinline__ int slot_position(const InstDev &I, int lay, const SrcTable &S, int p)
{
    if (S.nsub >= 0) {
        // the last sub-range starting at or before p
        int e = 0, top = S.nsub - 1;
        while (e < top) {
            const int mid = (e + top + 1) >> 1;
            if (S.sub_slot[mid] <= p) e = mid; else top = mid - 1;
        }
        return S.sub_pos[e] + (p - S.sub_slot[e]);
    }
    // too many sub-ranges to cache: search the source, then its chunk records
    int s = 0, top = S.n - 1;
    while (s < top) {
        const int mid = (s + top + 1) >> 1;
        if (S.pre[mid] <= p) s = mid; else top = mid - 1;
    }
    const int j = p - S.pre[s];
    const int d = S.dir[s];
    const int *cb = I.chunk_cb[lay];
    int lo = 0, hi = S.nch[s] - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (cb[(long long)(S.c0[s] + mid) * kBuckets + d] <= j) lo = mid; else hi = mid - 1;
    }
    const long long c = S.c0[s] + lo;
    return S.seg[s] + lo * I.R + I.chunk_pre[lay][c * kPre + d] + (j - cb[c * kBuckets + d]);
}

// -------------------------------------------------------------------------------------
// Gather helpers: separable interpolation from a shared-memory box.
// -------------------------------------------------------------------------------------
template <int ND, int ORD, typename R>
__device__ __forceinline__ R interp(const R *f, int bx, int bxy, int i0, int j0, int k0, const R *wx, const R *wy,
                                    const R *wz)
{
    constexpr int NP = ORD + 1;
    R acc = R(0);
#pragma unroll
    for (int k = 0; k < NP; ++k) {
        R ay = R(0);
        if (ND == 3) {
#pragma unroll
            for (int j = 0; j < NP; ++j) {
                const R *row = f + i0 + bx * (j0 + j) + bxy * (k0 + k);
                R ax = R(0);
#pragma unroll
                for (int i = 0; i < NP; ++i) ax += wx[i] * row[i];
                ay += wy[j] * ax;
            }
        } else {
            const R *row = f + i0 + bxy * (k0 + k);
            R ax = R(0);
#pragma unroll
            for (int i = 0; i < NP; ++i) ax += wx[i] * row[i];
            ay = ax;
        }
        acc += wz[k] * ay;
    }
    return acc;
}

// Global index of J tile element e (component stride jst, local x, y, z) after wrapping
// (periodic) or clipping (absorbing, returns -1) its guard cells; -1 for the padding
// entries jvol .. jst - 1 of a component.
__device__ __forceinline__ long long j_global_index(const InstDev &I, const int T0[3], int ND, int e, int jvol, int jst,
                                                    int &comp)
{
    comp = e / jst;
    const int rem = e - comp * jst;
    if (rem >= jvol) return -1;
    const int lx = rem % I.jdim[0];
    const int ly = (rem / I.jdim[0]) % I.jdim[1];
    const int lz = rem / (I.jdim[0] * I.jdim[1]);
    int gidx[3] = {T0[0] + I.jlo + lx, ND == 3 ? T0[1] + I.jlo + ly : 0, T0[2] + I.jlo + lz};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (ND == 2 && a == 1) continue;
        if (gidx[a] < 0 || gidx[a] >= I.n[a]) {
            if (I.bc[a] != 0) return -1;
            gidx[a] += gidx[a] < 0 ? I.n[a] : -I.n[a];
        }
    }
    return (gidx[0] + I.gh[0]) + I.sy * (gidx[1] + I.gh[1]) + I.sz * (gidx[2] + I.gh[2]);
}

// FP32 tile, after a chunk: T += A * inv[component], A = 0 over the entries this thread
// owns, 4 at a time (components start on multiples of 4 entries, jst apart; the arrays
// start 16-byte aligned).
__device__ __forceinline__ void fold_chunk(int *A, float *T, int jst, const float inv[3], int tid, int nt)
{
    int4 *A4 = reinterpret_cast<int4 *>(A);
    float4 *T4 = reinterpret_cast<float4 *>(T);
    const int q1 = jst >> 2, q2 = jst >> 1, n4 = 3 * (jst >> 2);
    for (int e = tid; e < n4; e += nt) {
        const float s = e >= q2 ? inv[2] : e >= q1 ? inv[1] : inv[0];
        const int4 a = A4[e];
        float4 t = T4[e];
        t.x = __fmaf_rn((float)a.x, s, t.x);
        t.y = __fmaf_rn((float)a.y, s, t.y);
        t.z = __fmaf_rn((float)a.z, s, t.z);
        t.w = __fmaf_rn((float)a.w, s, t.w);
        T4[e] = t;
        A4[e] = make_int4(0, 0, 0, 0);
    }
}

__device__ __forceinline__ void red_add_v4(float *p, float a, float b, float c, float d)
{
    asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(a), "f"(b), "f"(c), "f"(d) : "memory");
}

// FP32 tile: value = T + A * inv[component] (the last chunk's accumulator and scale),
// added to global J.  Each J-tile row (component, y,
// z) is cut into groups of 4 entries aligned with the 16-byte groups of the global row;
// a group whose entries all lie inside the interior along x (entries before the row or
// after its end add 0 to the padded row) is added with one vector reduction, the others
// entry by entry with wrap-around (periodic) or clipping (absorbing) along x.  Rows
// outside the box along y or z wrap or are dropped as a whole.
__device__ __forceinline__ void flush_j_chunk(const InstDev &I, const int T0[3], int ND, const int *A, const float *T,
                                              int jst, const float inv[3], int warp, int lane)
{
    const int jd0 = I.jdim[0], jd1 = I.jdim[1], jd2 = I.jdim[2];
    const int rows = 3 * jd1 * jd2;
    const int gx0 = T0[0] + I.jlo;              // global x of tile entry 0 (unpadded)
    const int a0 = (4 - ((gx0 + I.gh[0]) & 3)) & 3;  // first entry on a 16-byte boundary
    const int lx0 = a0 > 0 ? a0 - 4 : 0;         // first group start (may be negative: pads)
    const int ng = (jd0 - lx0 + 3) >> 2;
    const int lpr = ng <= 4 ? 4 : ng <= 8 ? 8 : ng <= 16 ? 16 : 32;  // lanes per row
    const int rpw = 32 / lpr;
    for (int rb = warp * rpw; rb < rows; rb += kNW * rpw) {
        const int row = rb + lane / lpr;
        if (row >= rows) continue;
        const int comp = row / (jd1 * jd2);
        const int ryz = row - comp * jd1 * jd2;
        const int lz = ryz / jd1, ly = ryz - lz * jd1;
        int gy = ND == 3 ? T0[1] + I.jlo + ly : 0;
        int gz = T0[2] + I.jlo + lz;
        bool keep = true;
        if (ND == 3 && (gy < 0 || gy >= I.n[1])) {
            if (I.bc[1] != 0) keep = false;
            gy += gy < 0 ? I.n[1] : -I.n[1];
        }
        if (gz < 0 || gz >= I.n[2]) {
            if (I.bc[2] != 0) keep = false;
            gz += gz < 0 ? I.n[2] : -I.n[2];
        }
        const int e0 = comp * jst + ryz * jd0;
        const float sc = comp == 0 ? inv[0] : comp == 1 ? inv[1] : inv[2];
        float *grow = (float *)I.J[comp] + I.gh[0] + I.sy * (gy + I.gh[1]) + I.sz * (gz + I.gh[2]);
        for (int g = lane % lpr; g < ng; g += lpr) {
            const int lx = lx0 + 4 * g;
            float v[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int x = lx + q;
                v[q] = 0.f;
                if (x >= 0 && x < jd0) v[q] = __fmaf_rn((float)A[e0 + x], sc, T[e0 + x]);
            }
            if (!keep) continue;
            const int gx = gx0 + lx;  // global x of the group's first entry
            const int xr0 = lx < 0 ? gx0 : gx, xr1 = min(gx + 3, gx0 + jd0 - 1);  // real entries
            if (xr0 >= 0 && xr1 < I.n[0] && gx + I.gh[0] >= 0 && gx + 3 + I.gh[0] < I.P[0]) {
                if ((v[0] != 0.f) | (v[1] != 0.f) | (v[2] != 0.f) | (v[3] != 0.f))
                    red_add_v4(grow + gx, v[0], v[1], v[2], v[3]);
            } else {
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int x = lx + q;
                    if (x < 0 || x >= jd0 || v[q] == 0.f) continue;
                    int gxq = gx + q;
                    if (gxq < 0 || gxq >= I.n[0]) {
                        if (I.bc[0] != 0) continue;
                        gxq += gxq < 0 ? I.n[0] : -I.n[0];
                    }
                    atomicAdd(grow + gxq, v[q]);
                }
            }
        }
    }
}

__device__ __forceinline__ void flush_j_double(const InstDev &I, const int T0[3], int ND, const double *J, int jvol,
                                               int jst, int tid, int nt)
{
    for (int e = tid; e < 3 * jst; e += nt) {
        const double v = J[e];
        if (v == 0.0) continue;
        int comp;
        const long long gi = j_global_index(I, T0, ND, e, jvol, jst, comp);
        if (gi < 0) continue;
        atomicAdd((double *)I.J[comp] + gi, v);
    }
}

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

// The record of tile g of the launch by one warp (scratch S of its own).
__device__ __forceinline__ void tile_sources_warp(const Launch &L, int g, SrcScratch &S, int lane)
{
    const int ii = find_instance(L.tile_start, L.ninst, g);
    const InstDev &I = L.inst[ii];
    const int t = g - L.tile_start[ii];
    const int lay = 1 - *I.cur;  // the input layout of the coming phase (the scan flipped it)
    const int tx = t % I.nt[0], ty = (t / I.nt[0]) % I.nt[1], tz = t / (I.nt[0] * I.nt[1]);
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

// Tile population scan of instance ii by one CTA of any multiple of 32 threads (up to
// 1024).  mode 0 (step): lays out the output layout (segment starts and chunk bases) from
// the populations, zeroes them, flips the parity and counts the particle phase.  mode 1
// (read-out): writes the exclusive scan of the populations into dst[ii] (one int per
// tile + total) and the total into *live, changing nothing else.
// sh: 66 ints of shared memory.
__device__ __forceinline__ void scan_instance(const Launch &L, int ii, int mode, int *const *dst, int *sh)
{
    const InstDev &I = L.inst[ii];
    int *s_warp = sh, *s_warp2 = sh + 32;
    int &s_carry = sh[64], &s_carry2 = sh[65];
    const int cur = *I.cur;
    const int out = 1 - cur;
    const int nt = I.ntiles;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nthr = blockDim.x, nwarps = nthr >> 5;
    if (tid == 0) { s_carry = 0; s_carry2 = 0; }
    __syncthreads();
    for (int base = 0; base < nt; base += nthr) {
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
            int x = lane < nwarps ? s_warp[lane] : 0, y = lane < nwarps ? s_warp2[lane] : 0;
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
                dst[ii][t] = ex;
            }
        }
        __syncthreads();
        if (tid == 0) { s_carry += s_warp[nwarps - 1]; s_carry2 += s_warp2[nwarps - 1]; }
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
            dst[ii][nt] = s_carry;
        }
        *I.live = s_carry;
    }
}

// The particle phase of tile t of instance I, by one CTA of kNT threads.  INJ: instances
// with a beam injection plane (a separate instantiation, so that the kernel without a
// plane carries none of its code).  I is the instance's entry of the launch's device
// array, or, for a launch of one instance, a kernel parameter: its fields are then
// operands from the constant bank, which no store of the kernel can alias, so they are
// never reloaded after the particle write-out.  LANEWIN: the deposit window per lane
// (deposit_esirkepov's kLane), taken where the registers allow it (the one-instance
// kernel).
template <int ND, int ORD, typename R, int PUSHER, bool INJ, bool LANEWIN>
__device__ __forceinline__ void particle_tile(const InstDev &I, const int t)
{
    constexpr bool kFixed = sizeof(R) == 4;  // FP32: fixed-point chunk accumulator + FP32 tile
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ SrcTable S;
    __shared__ uint64_t bar;
    __shared__ int s_run[kBuckets];          // running bucket totals of the tile (warp 0)
    // each thread's particle of the next chunk, copied in (cp.async) while the current
    // chunk is processed; two buffers, chunk r in buffer r & 1
    __shared__ int s_pcell[2][kNT], s_pid[2][kNT];
    __shared__ R s_poff[2][3][kNT], s_pu[2][3][kNT], s_pw[2][kNT];
    __shared__ int s_cnt[2][kNW][kBuckets];  // per-warp bucket counts, double-buffered per chunk
    __shared__ __align__(16) unsigned s_bmax[3][kNW];  // FP32: per-warp contribution bounds of the chunk

    const int out = *I.cur;  // the scan of this step already flipped the parity
    const int in = 1 - out;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

    const int tx = t % I.nt[0];
    const int ty = (t / I.nt[0]) % I.nt[1];
    const int tz = t / (I.nt[0] * I.nt[1]);
    const int T0[3] = {tx * I.ts[0], ty * I.ts[1], tz * I.ts[2]};
    const int seg_out = I.seg[out][t];
    const int count = I.seg[out][t + 1] - seg_out;
    const int chunk_out = I.chunk_base[out][t];

    if (count == 0) {
        if (tid < kBuckets) I.tot[out][t * kBuckets + tid] = 0;
        return;
    }
    // the output layout must fit the buffers (it always does unless memory is corrupt)
    if (seg_out + count > I.cap || chunk_out + (count + kChunk - 1) / kChunk > I.chunk_cap) {
        if (tid == 0) atomicOr(I.err, kErrCapacity);
        return;
    }

    // shared-memory carve-up (base rounded up to 128 bytes for TMA): 6 field boxes, then
    // the J tile: 3 components of jvol cells, jst = jvol rounded up to a multiple of 4 apart,
    // as FP64 values (FP64 mode) or as the 32-bit integer chunk accumulator A and the FP32
    // tile T of 3 jst entries each (FP32 mode) -- 8 bytes per entry either way
    const int boxn = I.box[0] * I.box[1] * I.box[2];
    const int box_bytes = boxn * (int)sizeof(R);
    const int box_stride = (box_bytes + 127) & ~127;
    unsigned char *sbase = smem + ((128u - (smem_addr(smem) & 127u)) & 127u);
    R *sF = reinterpret_cast<R *>(sbase);
    unsigned char *sJraw = sbase + 6 * box_stride;
    const int jvol = I.jdim[0] * I.jdim[1] * I.jdim[2];
    const int jst = (jvol + 3) & ~3;
    const int jv4 = 3 * (jst >> 2);  // J-tile entries in groups of 4
    int *sJA = reinterpret_cast<int *>(sJraw);
    float *sJT = reinterpret_cast<float *>(sJA + 4 * jv4);
    double *sJD = reinterpret_cast<double *>(sJraw);

    if (tid == 0) {
        mbar_init(&bar, 1);
        const CUtensorMap *tm = I.tmap + 6 * *(volatile const int *)I.fpar;  // the current E / B buffer
        for (int c = 0; c < 6; ++c) tmap_acquire(tm + c);
        mbar_expect_tx(&bar, 6u * (uint32_t)box_bytes);
        const int x = T0[0] + I.box_lo[0] + I.gh[0];
        const int y = T0[1] + I.box_lo[1] + I.gh[1];
        const int z = T0[2] + I.box_lo[2] + I.gh[2];
        for (int c = 0; c < 6; ++c)
            tma_load_3d(sbase + c * box_stride, tm + c, x, y, z, &bar);
    }
    for (int e = tid; e < 2 * jv4; e += kNT)  // A and T (or the FP64 tile)
        reinterpret_cast<int4 *>(sJraw)[e] = make_int4(0, 0, 0, 0);
    for (int e = tid; e < 2 * kNW * kBuckets; e += kNT) (&s_cnt[0][0][0])[e] = 0;
    if (tid < kBuckets) s_run[tid] = 0;
    // the tile's source table: its precomputed record (one coalesced read), or built here
    // when the record overflowed
    {
        const int *rec = I.srcrec + (size_t)t * kSrcRec;
        if (tid < kSrcRec) {
            const int v = rec[tid];
            if (tid == 0) S.count = v;
            else if (tid == 1) S.nsub = v;
            else if (tid >= kRecSlot && tid < kRecPos) S.sub_slot[tid - kRecSlot] = v;
            else if (tid >= kRecPos && tid < kRecPos + kSubCache) S.sub_pos[tid - kRecPos] = v;
        }
        __syncthreads();
        if (S.nsub < 0) build_sources(I, in, tx, ty, tz, S);  // ends with __syncthreads
    }
    const bool ok = mbar_wait_bounded(&bar, 0, kWaitCycles);
    if (!__syncthreads_and(ok ? 1 : 0)) {
        if (tid == 0) {
            atomicOr(I.err, kErrTimeout);
            mbar_wait_bounded(&bar, 0, kWaitCycles);  // let copies in flight land
        }
        return;
    }
    if (tid == 0 && S.count != count) atomicOr(I.err, kErrInternal);

    // per-instance constants in the working precision (host-formed); in FP32 mode the
    // current factor qdv carries the fixed-point scale (see ChunkAcc)
    const StepCoef<R> &K = coef<R>(I);
    const R h = K.h;
    const R qdv = K.qdv;
    const R jfx = K.jf[0], jfy = K.jf[1], jfz = K.jf[2];
    const R dtdx[3] = {K.dtdx[0], K.dtdx[1], K.dtdx[2]};
    // beam injection plane in cells along z at this step's push time t^n = n dt (n: the
    // phases before this one), in FP64; beam particles upstream of it are frozen
    const bool inj = INJ && I.inj_id0 != INT_MAX;
    double zp_inj = 0.0;
    if (inj) zp_inj = (I.inj_zb - I.beta_b * ((double)(*I.phase - 1) * I.dt)) / I.dx[2];
    const int bx = I.box[0], bxy = I.box[0] * I.box[1];
    const int jd0 = I.jdim[0], jd01 = I.jdim[0] * I.jdim[1];
    const int jlo_y = ND == 3 ? I.jlo : 0;
    const int tsx = min(I.ts[0], I.n[0] - T0[0]);
    const int tsy = min(I.ts[1], I.n[1] - T0[1]);
    const int tsz = min(I.ts[2], I.n[2] - T0[2]);

    const int *cell_in = I.cell[in];
    const R *off_in[3] = {(const R *)I.off[in][0], (const R *)I.off[in][1], (const R *)I.off[in][2]};
    const R *u_in[3] = {(const R *)I.u[in][0], (const R *)I.u[in][1], (const R *)I.u[in][2]};
    const R *w_in = (const R *)I.w[in];
    const int *id_in = I.id[in];
    int *cell_out = I.cell[out];
    R *off_out[3] = {(R *)I.off[out][0], (R *)I.off[out][1], (R *)I.off[out][2]};
    R *u_out[3] = {(R *)I.u[out][0], (R *)I.u[out][1], (R *)I.u[out][2]};
    R *w_out = (R *)I.w[out];
    int *id_out = I.id[out];

    // stages this thread's particle of slot `sl` into buffer b of the s_p* arrays
    // (asynchronously); returns its position in the input buffer, or -1
    auto stage = [&](int sl, int b) -> int {
        const int p = sl < count ? slot_position(I, in, S, sl) : -1;
        if (p >= 0 && p < I.cap) {
            cp_async<4>(&s_pcell[b][tid], cell_in + p);
            cp_async<sizeof(R)>(&s_poff[b][0][tid], off_in[0] + p);
            if (ND == 3) cp_async<sizeof(R)>(&s_poff[b][1][tid], off_in[1] + p);
            cp_async<sizeof(R)>(&s_poff[b][2][tid], off_in[2] + p);
            cp_async<sizeof(R)>(&s_pu[b][0][tid], u_in[0] + p);
            cp_async<sizeof(R)>(&s_pu[b][1][tid], u_in[1] + p);
            cp_async<sizeof(R)>(&s_pu[b][2][tid], u_in[2] + p);
            cp_async<sizeof(R)>(&s_pw[b][tid], w_in + p);
            if (id_in) cp_async<4>(&s_pid[b][tid], id_in + p);
        }
        cp_async_commit();
        return p;
    };
    int pos_next = stage(tid, 0);
    float inv[3] = {1.f, 1.f, 1.f};  // FP32: the current chunk's per-component 1 / scale

    for (int base = 0, r = 0; base < count; base += kChunk, ++r) {
        int bucket = 28;  // 0..26 direction, 27 dead, 28 no particle
        int cell_new = 0, pid = 0;
        R o1[3] = {R(0), R(0), R(0)}, u[3] = {R(0), R(0), R(0)}, w = R(0);
        const int slot = base + tid;
        const int pos = pos_next;
        const int pb = r & 1;
        cp_async_wait_all();  // this thread's particle of this chunk has landed
        if (base + kChunk < count) pos_next = stage(base + kChunk + tid, pb ^ 1);
        if (slot < count && (pos < 0 || pos >= I.cap)) atomicOr(I.err, kErrInternal);
        int l[3] = {0, 0, 0}, cc[3] = {0, 0, 0};
        // deposit inputs; a lane without a particle deposits zero from inside the tile
        R o[3] = {R(0.5), R(0.5), R(0.5)};
        int l1[3] = {0, 0, 0};
        R disp[3] = {R(0), R(0), R(0)};
        R fx = R(0), fy = R(0), fz = R(0);
        o1[0] = o1[1] = o1[2] = R(0.5);
        bool have = false;
        if (pos >= 0 && pos < I.cap) {
            const int c = s_pcell[pb][tid];
            const int cyz = fast_div(c, I.div_n0);
            cc[0] = c - cyz * I.n[0];
            cc[2] = fast_div(cyz, I.div_n1);
            cc[1] = cyz - cc[2] * I.n[1];
            l[0] = cc[0] - T0[0];
            l[1] = cc[1] - T0[1];
            l[2] = cc[2] - T0[2];
            have = l[0] >= 0 && l[0] < tsx && l[1] >= 0 && l[1] < tsy && l[2] >= 0 && l[2] < tsz;
            if (!have) atomicOr(I.err, kErrInternal);
        }
        if (have) {
            o[0] = s_poff[pb][0][tid];
            o[1] = ND == 3 ? s_poff[pb][1][tid] : R(0);
            o[2] = s_poff[pb][2][tid];
            u[0] = s_pu[pb][0][tid];
            u[1] = s_pu[pb][1][tid];
            u[2] = s_pu[pb][2][tid];
            w = s_pw[pb][tid];
            pid = id_in ? s_pid[pb][tid] : 0;

            // ---- gather (Yee positions: E_a staggered along a, B_a along the other two)
            R E[3], B[3];
            {
                R wn[3][ORD + 1], wsg[3][ORD + 1];
                int bn[3], bsg[3];
                bn[0] = shape_nodal<ORD>(l[0], o[0], wn[0]) - I.box_lo[0];
                bsg[0] = shape_stag<ORD>(l[0], o[0], wsg[0]) - I.box_lo[0];
                if (ND == 3) {
                    bn[1] = shape_nodal<ORD>(l[1], o[1], wn[1]) - I.box_lo[1];
                    bsg[1] = shape_stag<ORD>(l[1], o[1], wsg[1]) - I.box_lo[1];
                } else {
                    bn[1] = bsg[1] = 0;
#pragma unroll
                    for (int q = 0; q <= ORD; ++q) wn[1][q] = wsg[1][q] = R(0);
                    wn[1][0] = wsg[1][0] = R(1);
                }
                bn[2] = shape_nodal<ORD>(l[2], o[2], wn[2]) - I.box_lo[2];
                bsg[2] = shape_stag<ORD>(l[2], o[2], wsg[2]) - I.box_lo[2];
                const int bs = box_stride / (int)sizeof(R);
                E[0] = interp<ND, ORD, R>(sF + 0 * bs, bx, bxy, bsg[0], bn[1], bn[2], wsg[0], wn[1], wn[2]);
                E[1] = interp<ND, ORD, R>(sF + 1 * bs, bx, bxy, bn[0], bsg[1], bn[2], wn[0], wsg[1], wn[2]);
                E[2] = interp<ND, ORD, R>(sF + 2 * bs, bx, bxy, bn[0], bn[1], bsg[2], wn[0], wn[1], wsg[2]);
                B[0] = interp<ND, ORD, R>(sF + 3 * bs, bx, bxy, bn[0], bsg[1], bsg[2], wn[0], wsg[1], wsg[2]);
                B[1] = interp<ND, ORD, R>(sF + 4 * bs, bx, bxy, bsg[0], bn[1], bsg[2], wsg[0], wn[1], wsg[2]);
                B[2] = interp<ND, ORD, R>(sF + 5 * bs, bx, bxy, bsg[0], bsg[1], bn[2], wsg[0], wsg[1], wn[2]);
            }

            // ---- push
            if (PUSHER == 0)
                push_vay(u, E, B, h);
            else
                push_boris(u, E, B, h);

            // a beam particle frozen upstream of the injection plane: the fields do not act
            // on it, it keeps its momentum (restored from the staged copy; pushing
            // unconditionally and restoring runs faster than branching around the push)
            if (INJ && inj && pid >= I.inj_id0 && (double)cc[2] + (double)o[2] < zp_inj) {
                u[0] = s_pu[pb][0][tid];
                u[1] = s_pu[pb][1][tid];
                u[2] = s_pu[pb][2][tid];
            }

            // ---- move
            bool bad = false;
            o1[0] = o[0]; o1[1] = o[1]; o1[2] = o[2];
            int kstep[3] = {0, 0, 0};
            R vy;
            if (sizeof(R) == 4) {
                const float gn = sqrtf(1.f + (float)u[0] * (float)u[0] + (float)u[1] * (float)u[1] + (float)u[2] * (float)u[2]);
                const float ig = 1.f / gn;
                float ox = (float)o1[0], oy = (float)o1[1], oz = (float)o1[2];
                float d[3] = {0.f, 0.f, 0.f};
                kstep[0] = move_axis(ox, (float)u[0], ig, (float)dtdx[0], d[0], bad);
                if (ND == 3) kstep[1] = move_axis(oy, (float)u[1], ig, (float)dtdx[1], d[1], bad);
                kstep[2] = move_axis(oz, (float)u[2], ig, (float)dtdx[2], d[2], bad);
                o1[0] = R(ox); o1[1] = R(oy); o1[2] = R(oz);
                disp[0] = R(d[0]); disp[1] = R(d[1]); disp[2] = R(d[2]);
                vy = R((float)u[1] * ig);
            } else {
                const double gn = gamma_of((double)u[0], (double)u[1], (double)u[2]);
                double ox = (double)o1[0], oy = (double)o1[1], oz = (double)o1[2];
                kstep[0] = move_axis(ox, (double)u[0], gn, I.dt, I.dx[0], bad);
                if (ND == 3) kstep[1] = move_axis(oy, (double)u[1], gn, I.dt, I.dx[1], bad);
                kstep[2] = move_axis(oz, (double)u[2], gn, I.dt, I.dx[2], bad);
                o1[0] = R(ox); o1[1] = R(oy); o1[2] = R(oz);
                vy = R((double)u[1] / gn);
            }
            if (bad) {
                atomicOr(I.err, kErrSpeed);
                o1[0] = o[0]; o1[1] = o[1]; o1[2] = o[2];
                kstep[0] = kstep[1] = kstep[2] = 0;
                disp[0] = disp[1] = disp[2] = R(0);
            }

            // ---- Esirkepov deposit inputs
            {
                l1[0] = l[0] + kstep[0];
                l1[1] = l[1] + kstep[1];
                l1[2] = l[2] + kstep[2];
                const R qw = qdv * w;
                fx = -qw * jfx;
                fy = ND == 3 ? -qw * jfy : qw * vy;
                fz = -qw * jfz;
            }

            // ---- new cell, destination tile, bucket
            int cn[3] = {cc[0] + kstep[0], cc[1] + kstep[1], cc[2] + kstep[2]};
            bool dead = false;
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                if (ND == 2 && a == 1) continue;
                if (cn[a] < 0 || cn[a] >= I.n[a]) {
                    if (I.bc[a] == 0)
                        cn[a] += cn[a] < 0 ? I.n[a] : -I.n[a];
                    else
                        dead = true;
                }
            }
            if (dead) {
                bucket = kDead;
            } else {
                // the new tile from the tile-local cell (a move stays below one cell, so it
                // is this tile or a neighbour; across a periodic face the coordinate wraps)
                const int l1v[3] = {l[0] + kstep[0], l[1] + kstep[1], l[2] + kstep[2]};
                const int tl[3] = {tsx, tsy, tsz}, to[3] = {tx, ty, tz};
                int dd[3] = {0, 0, 0};
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    if (ND == 2 && a == 1) continue;
                    int tn = to[a] + (l1v[a] < 0 ? -1 : (l1v[a] >= tl[a] ? 1 : 0));
                    tn += tn < 0 ? I.nt[a] : (tn >= I.nt[a] ? -I.nt[a] : 0);
                    dd[a] = axis_dir(to[a], tn, I.nt[a], I.bc[a]);
                }
                bucket = (dd[2] + 1) * 9 + (dd[1] + 1) * 3 + (dd[0] + 1);
            }
            cell_new = cn[0] + I.n[0] * (cn[1] + I.n[1] * cn[2]);
        }

        // ---- Esirkepov deposit into the shared J tile, by every lane of the warp.  FP32:
        // the chunk's per-component scale (see ChunkAcc) from the warps' bounds, after a
        // barrier that also completes the previous chunk's fold of A into T.
        if constexpr (kFixed) {
            // |f_a| (|d_a| + 2^-18): a particle that changes its nodes forms its weight changes
            // from differences of weights, whose rounding (< 2^-19 in the running sums) is
            // not relative to a small displacement
            const float eps = 0x1p-18f;
            const float bnd[3] = {fabsf(fx) * (fabsf(disp[0]) + eps),
                                  ND == 3 ? fabsf(fy) * (fabsf(disp[1]) + eps) : fabsf(fy),
                                  fabsf(fz) * (fabsf(disp[2]) + eps)};
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                const unsigned m = __reduce_max_sync(0xffffffffu, __float_as_uint(bnd[a]));
                if (lane == 0) s_bmax[a][warp] = m;
            }
            __syncthreads();
            float sc[3];
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                const uint4 m0 = reinterpret_cast<const uint4 *>(s_bmax[a])[0];
                const uint4 m1 = reinterpret_cast<const uint4 *>(s_bmax[a])[1];
                const unsigned m = max(max(max(m0.x, m0.y), max(m0.z, m0.w)), max(max(m1.x, m1.y), max(m1.z, m1.w)));
                // the largest contribution is at most K times the bound (see ChunkAcc): K =
                // S_max^2 in 3D and for the out-of-plane current of 2D3V, S_max for the
                // in-plane ones; S_max = 3/4 (order 2) or 1 (order 1)
                constexpr float Smax = ORD == 2 ? 0.75f : 1.0f;
                const float K = (ND == 3 || a == 1) ? Smax * Smax : Smax;
                // inv = K bound / (0.999 2^22), scale = 1 / inv (correctly rounded, so
                // scale x inv = 1 to FP32 precision)
                const float bk = K * __uint_as_float(m);
                inv[a] = bk > 1e-30f ? bk * (1.0f / (0.999f * 4194304.0f)) : 1.0f;
                sc[a] = __frcp_rn(inv[a]);
            }
            // the current follows the computed displacement (see shape_window)
            deposit_esirkepov<ND, ORD, true, true, LANEWIN, R>(l, o, l1, o1, disp, fx * sc[0], fy * sc[1], fz * sc[2], I.jlo,
                                                      jlo_y, jd0, jd01, jst, ChunkAcc{sJA});
        } else {
            deposit_esirkepov<ND, ORD, false, false, false, R>(l, o, l1, o1, disp, fx, fy, fz, I.jlo, jlo_y, jd0, jd01,
                                                        jst, DoubleAcc{sJD});
        }

        // ---- stable ranking of the chunk by bucket: order (warp, lane), one barrier per
        // chunk.  Each warp writes its bucket counts into its own row of s_cnt[cbuf]
        // (cleared by that warp first: the row was last read in chunk r - 2, before the
        // barrier of chunk r - 1), and after the barrier every warp forms the offsets it
        // needs itself: lane d sums bucket d over the warps (its own prefix and the total),
        // and a scan over the lanes gives the bucket bases.  Warp 0 keeps the running
        // bucket totals of the tile and writes the chunk's records.
        const int cbuf = r & 1;
        if (lane < kBuckets) s_cnt[cbuf][warp][lane] = 0;
        __syncwarp();
        const unsigned peers = __match_any_sync(0xffffffffu, bucket);
        const int rank = __popc(peers & ((1u << lane) - 1u));
        if (bucket < kBuckets && lane == __ffs(peers) - 1) s_cnt[cbuf][warp][bucket] = __popc(peers);
        __syncthreads();
        int totd = 0, below = 0;  // lane d: bucket d over all warps, and over the warps before this one
        if (lane < kBuckets) {
#pragma unroll
            for (int ww = 0; ww < kNW; ++ww) {
                const int v = s_cnt[cbuf][ww][lane];
                below += ww < warp ? v : 0;
                totd += v;
            }
        }
        int incl = totd;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        const int basev = incl - totd;  // lane d: first position of bucket d in the chunk
        const int myoff = __shfl_sync(0xffffffffu, basev + below, bucket < kBuckets ? bucket : 0);
        if (warp == 0) {
            const int c = chunk_out + r;
            if (lane < kBuckets) {
                I.chunk_pre[out][(long long)c * kPre + lane] = basev;
                I.chunk_cb[out][(long long)c * kBuckets + lane] = s_run[lane];
                s_run[lane] += totd;
                if (lane == kBuckets - 1) I.chunk_pre[out][(long long)c * kPre + kBuckets] = incl;
            }
        }

        // ---- write the particle out, partitioned by bucket
        if (bucket < kDead) {
            const int p = seg_out + base + myoff + rank;
            cell_out[p] = cell_new;
            off_out[0][p] = o1[0];
            if (ND == 3) off_out[1][p] = o1[1];
            off_out[2][p] = o1[2];
            u_out[0][p] = u[0];
            u_out[1][p] = u[1];
            u_out[2][p] = u[2];
            w_out[p] = w;
            if (id_out) id_out[p] = pid;
        }

        // ---- FP32: fold the chunk accumulator into the FP32 tile (the last chunk's is
        // added by the flush)
        if constexpr (kFixed) {
            if (base + kChunk < count) fold_chunk(sJA, sJT, jst, inv, tid, kNT);
        }
    }
    __syncthreads();  // all deposits and bucket totals complete

    // ---- tile bookkeeping for the next step
    if (tid < kBuckets) I.tot[out][t * kBuckets + tid] = s_run[tid];
    if (tid < kDirs && s_run[tid] > 0) {
        const int ddx = tid % 3 - 1, ddy = (tid / 3) % 3 - 1, ddz = tid / 9 - 1;
        int nx = tx + ddx, ny = ty + ddy, nz = tz + ddz;
        nx = (nx + I.nt[0]) % I.nt[0];
        ny = (ny + I.nt[1]) % I.nt[1];
        nz = (nz + I.nt[2]) % I.nt[2];
        atomicAdd(I.pop + nx + I.nt[0] * (ny + I.nt[1] * nz), s_run[tid]);
    }
    if (tid == 0 && s_run[kDead] > 0) atomicAdd(I.lost, (unsigned long long)s_run[kDead]);

    // ---- flush the J tile
    if constexpr (kFixed)
        flush_j_chunk(I, T0, ND, sJA, sJT, jst, inv, warp, lane);
    else
        flush_j_double(I, T0, ND, sJD, jvol, jst, tid, kNT);
}

// the particle phase of tile g of the launch (its global index over the instances)
template <int ND, int ORD, typename R, int PUSHER, bool INJ>
__device__ __forceinline__ void particle_tile_of_launch(const Launch &L, const int g)
{
    const int ii = find_instance(L.tile_start, L.ninst, g);
    particle_tile<ND, ORD, R, PUSHER, INJ, false>(L.inst[ii], g - L.tile_start[ii]);
}

template <int ND, int ORD, typename R, int PUSHER, bool INJ>
__global__ void __launch_bounds__(kNT, sizeof(R) == 4 ? 2 : 1) k_particles(Launch L)
{
    particle_tile_of_launch<ND, ORD, R, PUSHER, INJ>(L, blockIdx.x);
}

// a launch of one instance: the instance by value (tile = block)
template <int ND, int ORD, typename R, int PUSHER, bool INJ>
__global__ void __launch_bounds__(kNT, sizeof(R) == 4 ? 2 : 1) k_particles_one(const __grid_constant__ InstDev I)
{
    particle_tile<ND, ORD, R, PUSHER, INJ, true>(I, blockIdx.x);
}

}  // namespace pic
