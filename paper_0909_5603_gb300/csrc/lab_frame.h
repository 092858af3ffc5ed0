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
    int bc[3] = {PIC_PERIODIC, PIC_PERIODIC, PIC_PERIODIC};
    int order = 1;        // particle shape order (charge deposit for the beam field)
    double charge = -1.0; // macro-particle charge per unit weight
};

// Boosted-frame fields at t' = 0 set by a load: Ex Ey Ez Bx By Bz, each n0*n1*n2 values
// (x fastest) or empty when zero.
struct LabFields {
    std::vector<double> comp[6];
};

// Particles in FP64 as produced by the transform (cell index, offsets, momenta: 3 per
// particle), before the canonical tile sort.
struct LabParticles {
    std::vector<int32_t> cell, id;
    std::vector<double> off, mom, weight;
    int32_t beam_first = 0;  // first id of the beam (its ids follow the plasma's)
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

// Fills P with the plasma and beam macro-particles and F with the boosted-frame laser
// (Ex, By) plus the beam's self-field at t' = 0.
void transform_lab_inputs(const Geometry &G, double gamma_b, const pic_laser_lab *laser, const pic_plasma_lab *plasma,
                          const pic_beam_lab *beam, LabParticles &P, LabFields &F);

// rho on the nodes (n0*n1*n2) of particles first .. end of P, with the order-G.order shape.
void deposit_node_charge(const Geometry &G, const LabParticles &P, size_t first, std::vector<double> &rho);

// Adds to F the self-field of node charge rho moving rigidly at beta along z (Lorentz
// factor gamma): E from the relativistic Poisson equation, B = beta z x E.
void add_beam_self_field(const Geometry &G, const std::vector<double> &rho, double gamma, double beta, LabFields &F);

}  // namespace pic
