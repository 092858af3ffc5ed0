// lab_frame.h -- host-side lab -> boosted-frame input transform (internal).
#pragma once

#include <stdint.h>

#include <vector>

#include "../../include/pic.h"

namespace pic {

struct Geometry {
    int ndim;
    int n[3];
    double dx[3];
};

// Particles in FP64 as produced by the transform (cell index, offsets, momenta: 3 per
// particle), before the canonical tile sort.
struct LabParticles {
    std::vector<int32_t> cell, id;
    std::vector<double> off, mom, weight;
    void reserve(size_t n)
    {
        cell.reserve(n);
        id.reserve(n);
        off.reserve(3 * n);
        mom.reserve(3 * n);
        weight.reserve(n);
    }
    // appends a particle at box position pos (dropped when outside the box)
    void add(const Geometry &G, const double pos[3], const double u[3], double w, int32_t idv);
};

// Fills P with the plasma and beam macro-particles and Ex / By (n0*n1*n2, empty without
// a laser) with the boosted-frame laser at t' = 0.
void transform_lab_inputs(const Geometry &G, double gamma_b, const pic_laser_lab *laser, const pic_plasma_lab *plasma,
                          const pic_beam_lab *beam, LabParticles &P, std::vector<double> &Ex, std::vector<double> &By);

}  // namespace pic
