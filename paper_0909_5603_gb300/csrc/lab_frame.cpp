// lab_frame.cpp -- host FP64 transformation of laboratory-frame inputs into the boosted
// frame (Sec. 2 of Vay et al., arXiv:0909.5603): the laser is Doppler-shifted, the
// plasma becomes denser and drifts, beam particles are boosted and then drifted
// ballistically to a common boosted time ("frozen" drifting macro-particles) and bring
// their self-field (beam_field.cpp).
//
// Random draws use SplitMix64 (Steele, Lea, Flood, OOPSLA 2014) as a counter-based
// generator: value(seed, stream, counter) = finaliser(seed ^ stream << 40 ^ counter +
// golden gamma); uniforms take the top 53 bits; normals use Box-Muller (cos branch).
// The streams and counters are part of the input definition, documented in pic.h's
// loader: offsets 0..2, thermal momenta (3,4) (5,6) (7,8), beam (10,11) .. (20,21).
#include "lab_frame.h"

#include <cmath>

namespace pic {
namespace {

struct Rng {
    uint64_t seed;
    uint64_t raw(uint64_t stream, uint64_t counter) const
    {
        uint64_t z = (seed ^ (stream << 40) ^ counter) + 0x9E3779B97F4A7C15ULL;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
        return z ^ (z >> 31);
    }
    double uni(uint64_t stream, uint64_t counter) const
    {
        return (double)(raw(stream, counter) >> 11) * 0x1.0p-53;
    }
    double gauss(uint64_t stream, uint64_t counter) const
    {
        const double r = std::sqrt(-2.0 * std::log(1.0 - uni(stream, counter)));
        return r * std::cos(6.283185307179586 * uni(stream + 1, counter));
    }
};

struct Boost {
    double g, b;
    explicit Boost(double gamma) : g(gamma), b(std::sqrt(1.0 - 1.0 / (gamma * gamma))) {}
    // event (t, x, y, z) and momentum u of the lab frame -> boosted frame
    void event(const double in[4], const double u[3], double out[4], double up[3]) const
    {
        const double gp = std::sqrt(1.0 + u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
        out[0] = g * (in[0] - b * in[3]);
        out[1] = in[1];
        out[2] = in[2];
        out[3] = g * (in[3] - b * in[0]);
        up[0] = u[0];
        up[1] = u[1];
        up[2] = g * (u[2] - b * gp);
    }
};

}  // namespace

void LabParticles::add(const Geometry &G, const double pos[3], const double u[3], double w, int32_t idv)
{
    int c[3];
    double o[3];
    for (int a = 0; a < 3; ++a) {
        if (G.ndim == 2 && a == 1) {
            c[a] = 0;
            o[a] = 0.0;
            continue;
        }
        const double x = pos[a] / G.dx[a];
        const double k = std::floor(x);
        c[a] = (int)k;
        o[a] = x - k;
        if (o[a] >= 1.0) {
            o[a] = 0.0;
            c[a] += 1;
        }
        if (c[a] < 0 || c[a] >= G.n[a]) return;
    }
    cell.push_back(c[0] + G.n[0] * (c[1] + G.n[1] * c[2]));
    for (int a = 0; a < 3; ++a) {
        off.push_back(o[a]);
        mom.push_back(u[a]);
    }
    weight.push_back(w);
    id.push_back(idv);
}

void transform_lab_inputs(const Geometry &G, double gamma_b, const pic_laser_lab *laser, const pic_plasma_lab *plasma,
                          const pic_beam_lab *beam, LabParticles &P, LabFields &F)
{
    const Boost bst(gamma_b);
    const double doppler = bst.g * (1.0 + bst.b);
    const bool has_y = G.ndim == 3;
    const double xc = 0.5 * (G.n[0] * G.dx[0]);
    const double yc = has_y ? 0.5 * (G.n[1] * G.dx[1]) : 0.0;
    const long long ncell = (long long)G.n[0] * G.n[1] * G.n[2];
    for (auto &c : F.comp) c.clear();
    std::vector<double> &Ex = F.comp[0], &By = F.comp[4];
    Ex.assign(laser ? ncell : 0, 0.0);
    By.assign(laser ? ncell : 0, 0.0);

    if (laser) {
        // boosted wavelength and length stretched by gamma (1 + beta), centroid at
        // gamma (1 + beta) z_center; a0 and waist unchanged; E'x = B'y
        const double lam = laser->lambda0 * doppler;
        const double len = laser->duration * doppler;
        const double zc = laser->z_center * doppler;
        const double k = 6.283185307179586 / lam;
        const double amp = laser->a0 * k;
        const double w2 = laser->waist * laser->waist;
        for (int kk = 0; kk < G.n[2]; ++kk) {
            const double ze = kk * G.dx[2] - zc;         // Ex row: z on nodes
            const double zb = (kk + 0.5) * G.dx[2] - zc; // By row: z staggered
            const double le = std::exp(-(ze / len) * (ze / len)) * std::cos(k * ze);
            const double lb = std::exp(-(zb / len) * (zb / len)) * std::cos(k * zb);
            for (int j = 0; j < G.n[1]; ++j) {
                const double y = has_y ? j * G.dx[1] - yc : 0.0;
                for (int i = 0; i < G.n[0]; ++i) {
                    const double x = (i + 0.5) * G.dx[0] - xc;
                    const double tr = std::exp(-(x * x + y * y) / w2);
                    const long long idx = i + (long long)G.n[0] * (j + (long long)G.n[1] * kk);
                    Ex[idx] = amp * tr * le;
                    By[idx] = amp * tr * lb;
                }
            }
        }
    }

    int32_t next_id = 0;
    if (plasma) {
        const Rng rng{plasma->seed};
        const int ppc = plasma->ppc;
        const double dV = G.dx[0] * G.dx[1] * G.dx[2];
        const double zs = plasma->z_start, ramp = plasma->ramp_len;
        P.reserve((size_t)ncell * ppc);
        for (long long cidx = 0; cidx < ncell; ++cidx) {
            const int cc[3] = {(int)(cidx % G.n[0]), (int)((cidx / G.n[0]) % G.n[1]), (int)(cidx / ((long long)G.n[0] * G.n[1]))};
            for (int p = 0; p < ppc; ++p) {
                const uint64_t ctr = (uint64_t)cidx * (uint64_t)ppc + (uint64_t)p;
                double pos[3];
                for (int a = 0; a < 3; ++a)
                    pos[a] = (a == 1 && !has_y) ? 0.0 : (cc[a] + rng.uni((uint64_t)a, ctr)) * G.dx[a];
                // lab position of the t' = 0 sample: z = gamma z'; density gamma n(z)
                const double zl = bst.g * pos[2];
                double prof = 1.0;
                if (zl < zs) prof = 0.0;
                else if (ramp > 0.0 && zl < zs + ramp) prof = (zl - zs) / ramp;
                const double w = bst.g * plasma->n0 * prof * dV / ppc;
                if (w == 0.0) continue;
                double ul[3];
                for (int a = 0; a < 3; ++a) ul[a] = plasma->u_th[a] * rng.gauss(3 + 2 * (uint64_t)a, ctr);
                const double ev[4] = {0.0, pos[0], pos[1], zl};
                double evp[4], up[3];
                bst.event(ev, ul, evp, up);
                P.add(G, pos, up, w, next_id++);
            }
        }
    }
    P.beam_first = next_id;
    if (beam) {
        const size_t first = P.cell.size();
        const Rng rng{beam->seed};
        const double g0 = std::sqrt(beam->gamma * beam->gamma - 1.0);
        const double wb = beam->total_weight / (double)beam->n;
        for (int64_t i = 0; i < beam->n; ++i) {
            const uint64_t ctr = (uint64_t)i;
            const double ev[4] = {0.0, xc + beam->sigma_r * rng.gauss(10, ctr),
                                  yc + (has_y ? beam->sigma_r * rng.gauss(12, ctr) : 0.0),
                                  beam->z0 + beam->sigma_z * rng.gauss(14, ctr)};
            const double s = beam->rel_spread * g0;
            const double u[3] = {s * rng.gauss(16, ctr), s * rng.gauss(18, ctr), g0 + s * rng.gauss(20, ctr)};
            double evp[4], up[3];
            bst.event(ev, u, evp, up);
            const double gp = std::sqrt(1.0 + up[0] * up[0] + up[1] * up[1] + up[2] * up[2]);
            const double back = -evp[0];  // drift from t'_event to t' = 0
            double pos[3] = {evp[1] + up[0] / gp * back, evp[2] + up[1] / gp * back, evp[3] + up[2] / gp * back};
            if (!has_y) pos[1] = 0.0;
            P.add(G, pos, up, wb, next_id++);
        }
        if (P.cell.size() > first) {
            // the beam's self-field for its centroid velocity in this frame:
            // rapidities subtract, gamma' = gb gamma (1 - beta b)
            const double bl = g0 / beam->gamma;
            const double gp = bst.g * beam->gamma * (1.0 - bl * bst.b);
            const double bp = (bl - bst.b) / (1.0 - bl * bst.b);
            std::vector<double> rho;
            deposit_node_charge(G, P, first, rho);
            add_beam_self_field(G, rho, gp, bp, F);
        }
    }
}

}  // namespace pic
