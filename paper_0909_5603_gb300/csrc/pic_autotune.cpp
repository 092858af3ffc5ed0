// pic_autotune.cpp -- picks the particle tile shape for a workload by measurement.
//
// The particle kernel's cost per particle depends on the tile: a larger tile amortises
// the staged field boxes and the current-tile flush over more particles, a smaller one
// keeps shared memory, and with it the CTAs per SM, higher; the best shape depends on the
// grid, the shape order and the particle density.  pic_autotune builds the workload once
// per candidate tile, runs a few warm-up steps and times `steps` steps with the library's
// own per-phase CUDA-event timings, and returns the options of the fastest candidate.
// Candidates that pic_create rejects (shared memory, tile limits) are skipped.
#include <cstring>
#include <vector>

#include "../../include/pic.h"

namespace {

struct Tile {
    int t[3];
};

std::vector<Tile> candidates(int ndim)
{
    if (ndim == 3)
        return {{{8, 8, 8}},  {{16, 8, 8}}, {{8, 8, 16}}, {{8, 16, 8}}, {{16, 16, 4}},
                {{16, 8, 4}}, {{8, 8, 4}},  {{4, 8, 8}},  {{16, 16, 8}}, {{32, 8, 4}}};
    return {{{16, 1, 16}}, {{32, 1, 8}}, {{8, 1, 32}}, {{32, 1, 16}}, {{16, 1, 32}}, {{32, 1, 32}}, {{64, 1, 8}}};
}

}  // namespace

extern "C" pic_status pic_autotune(const pic_grid *grid, const double dx[3], double dt, double gamma_boost,
                                   int shape_order, const pic_options *base, const pic_laser_lab *laser,
                                   const pic_plasma_lab *plasma, const pic_beam_lab *beam, int steps,
                                   pic_options *best, double *ms_per_step)
{
    if (!grid || !dx || !best || steps < 1) return PIC_ERR_ARG;
    pic_options opt;
    if (base) opt = *base;
    else pic_default_options(&opt);
    double best_ms = -1.0;
    pic_status last = PIC_ERR_ARG;
    for (const Tile &c : candidates(grid->ndim)) {
        pic_options o = opt;
        std::memcpy(o.tile, c.t, sizeof(o.tile));
        pic_ctx *ctx = nullptr;
        pic_status st = pic_create(grid, dx, dt, gamma_boost, shape_order, &o, &ctx);
        if (st != PIC_OK) {
            last = st;
            continue;
        }
        pic_timings t{};
        if ((st = pic_load_lab_frame(ctx, laser, plasma, beam)) == PIC_OK && (st = pic_step(ctx, 2)) == PIC_OK &&
            (st = pic_set_profiling(ctx, 1, 1)) == PIC_OK && (st = pic_step(ctx, steps)) == PIC_OK &&
            (st = pic_get_timings(ctx, &t)) == PIC_OK && t.steps > 0) {
            const double ms = (t.ms_particles + t.ms_scan + t.ms_filter + t.ms_maxwell + t.ms_other) / (double)t.steps;
            if (best_ms < 0.0 || ms < best_ms) {
                best_ms = ms;
                *best = o;
            }
        }
        last = st;
        pic_destroy(ctx);
    }
    if (best_ms < 0.0) return last == PIC_OK ? PIC_ERR_INTERNAL : last;
    if (ms_per_step) *ms_per_step = best_ms;
    return PIC_OK;
}
