// beam_field.cpp -- host FP64 self-field of a beam at load time.
//
// Sec. 2 of Vay et al. (arXiv:0909.5603) discusses an isolated beam at relativistic
// velocity acting on itself through its own field: the radial E and the azimuthal B
// nearly cancel in the Lorentz force, which the Boris pusher resolves inexactly.  A beam
// loaded by pic_load_lab_frame therefore enters with that field.  For a charge density
// rho moving rigidly at beta along z (Lorentz factor gamma) the Lorenz-gauge potentials
// are phi and A = beta phi z, with
//     phi_xx + phi_yy + phi_zz / gamma^2 = -rho,
//     E = -(phi_x, phi_y, phi_z / gamma^2),   B = curl A = beta z x E.
// On the grid: rho on the nodes with the particles' own shape, second differences on
// the nodes (phi = 0 one node beyond an absorbing face, wrap on a periodic axis), E from
// the Yee differences of phi, and B_x = -beta E_y, B_y = beta E_x with E averaged over
// the two z nodes around B's half-integer z.  The separable system is inverted exactly
// by transforming each axis onto the eigenvectors of its second difference (sines on a
// Dirichlet axis, real Fourier modes on a periodic one), dividing by the summed
// eigenvalues and transforming back; O(n_a) work per node and axis, about a second at
// 64 x 64 x 256.  On an all-periodic grid the k = 0 mode is dropped (mean charge).
#include <cmath>
#include <vector>

#include "lab_frame.h"

namespace pic {
namespace {

constexpr double kPi = 3.141592653589793;

// Rows of V (n x n) are orthonormal eigenvectors of the 1D second difference with
// spacing h; ev holds the eigenvalues.
struct AxisModes {
    int n = 1;
    std::vector<double> V, ev;
};

AxisModes axis_modes(int n, bool periodic, double h)
{
    AxisModes M;
    M.n = n;
    M.V.assign((size_t)n * n, 0.0);
    M.ev.assign(n, 0.0);
    int row = 0;
    auto put = [&](double theta, auto basis) {
        for (int i = 0; i < n; ++i) M.V[(size_t)row * n + i] = basis(i);
        M.ev[row] = -4.0 * std::sin(0.5 * theta) * std::sin(0.5 * theta) / (h * h);
        ++row;
    };
    if (!periodic) {
        const double norm = std::sqrt(2.0 / (n + 1));
        for (int m = 1; m <= n; ++m) {
            const double th = kPi * m / (n + 1);
            put(th, [&](int i) { return norm * std::sin(th * (i + 1)); });
        }
        return M;
    }
    // cos modes k = 0 .. n/2, then sin modes k = 1 .. (n-1)/2
    for (int k = 0; 2 * k <= n; ++k) {
        const double th = 2.0 * kPi * k / n;
        const double norm = (k == 0 || 2 * k == n) ? std::sqrt(1.0 / n) : std::sqrt(2.0 / n);
        put(th, [&](int i) { return norm * std::cos(th * i); });
    }
    for (int k = 1; 2 * k < n; ++k) {
        const double th = 2.0 * kPi * k / n;
        const double norm = std::sqrt(2.0 / n);
        put(th, [&](int i) { return norm * std::sin(th * i); });
    }
    return M;
}

// a (x fastest, dims n) <- V a (to modes) or V^T a (back to nodes) along `axis`.
void transform_axis(std::vector<double> &a, const int n[3], int axis, const AxisModes &M, bool to_modes)
{
    const long long stride = axis == 0 ? 1 : (axis == 1 ? n[0] : (long long)n[0] * n[1]);
    const int len = n[axis];
    std::vector<double> in(len), out(len);
    const long long lines = (long long)n[0] * n[1] * n[2] / len;
    for (long long l = 0; l < lines; ++l) {
        // start of line l: the index with coordinate 0 along `axis`
        long long start;
        if (axis == 0) start = l * n[0];
        else if (axis == 1) start = (l % n[0]) + (l / n[0]) * (long long)n[0] * n[1];
        else start = l;
        for (int i = 0; i < len; ++i) in[i] = a[start + i * stride];
        for (int r = 0; r < len; ++r) out[r] = 0.0;
        if (to_modes) {
            for (int m = 0; m < len; ++m) {
                const double *v = &M.V[(size_t)m * len];
                double s = 0.0;
                for (int i = 0; i < len; ++i) s += v[i] * in[i];
                out[m] = s;
            }
        } else {
            for (int m = 0; m < len; ++m) {
                const double *v = &M.V[(size_t)m * len];
                const double c = in[m];
                for (int i = 0; i < len; ++i) out[i] += v[i] * c;
            }
        }
        for (int i = 0; i < len; ++i) a[start + i * stride] = out[i];
    }
}

}  // namespace

void deposit_node_charge(const Geometry &G, const LabParticles &P, size_t first, std::vector<double> &rho)
{
    const long long ncell = (long long)G.n[0] * G.n[1] * G.n[2];
    rho.assign(ncell, 0.0);
    const double inv_dv = 1.0 / (G.dx[0] * G.dx[1] * G.dx[2]);
    for (size_t p = first; p < P.cell.size(); ++p) {
        const int c = P.cell[p];
        const int cc[3] = {c % G.n[0], (c / G.n[0]) % G.n[1], c / (G.n[0] * G.n[1])};
        int lo[3];
        double wt[3][3];
        int cnt[3];
        for (int a = 0; a < 3; ++a) {
            const double o = P.off[3 * p + a];
            if (G.ndim == 2 && a == 1) {
                lo[a] = 0, cnt[a] = 1, wt[a][0] = 1.0;
            } else if (G.order == 1) {
                lo[a] = cc[a], cnt[a] = 2, wt[a][0] = 1.0 - o, wt[a][1] = o;
            } else {
                const int up = o >= 0.5 ? 1 : 0;
                const double f = o - up;  // offset from the nearest node, in [-1/2, 1/2)
                lo[a] = cc[a] + up - 1, cnt[a] = 3;
                wt[a][0] = 0.5 * (0.5 - f) * (0.5 - f);
                wt[a][1] = 0.75 - f * f;
                wt[a][2] = 0.5 * (0.5 + f) * (0.5 + f);
            }
        }
        const double qw = G.charge * P.weight[p] * inv_dv;
        for (int k = 0; k < cnt[2]; ++k)
            for (int j = 0; j < cnt[1]; ++j)
                for (int i = 0; i < cnt[0]; ++i) {
                    int node[3] = {lo[0] + i, lo[1] + j, lo[2] + k};
                    bool inside = true;
                    for (int a = 0; a < 3; ++a) {
                        if (node[a] >= 0 && node[a] < G.n[a]) continue;
                        if (G.bc[a] == PIC_PERIODIC) node[a] = (node[a] % G.n[a] + G.n[a]) % G.n[a];
                        else inside = false;
                    }
                    if (!inside) continue;
                    rho[node[0] + (long long)G.n[0] * (node[1] + (long long)G.n[1] * node[2])] +=
                        qw * wt[0][i] * wt[1][j] * wt[2][k];
                }
    }
}

void add_beam_self_field(const Geometry &G, const std::vector<double> &rho, double gamma, double beta, LabFields &F)
{
    const int *n = G.n;
    const long long ncell = (long long)n[0] * n[1] * n[2];
    const bool active[3] = {true, G.ndim == 3, true};
    bool all_periodic = true;
    AxisModes M[3];
    std::vector<double> phi(rho);
    for (int a = 0; a < 3; ++a) {
        if (!active[a]) continue;
        all_periodic = all_periodic && G.bc[a] == PIC_PERIODIC;
        M[a] = axis_modes(n[a], G.bc[a] == PIC_PERIODIC, G.dx[a]);
        transform_axis(phi, n, a, M[a], true);
    }
    const double zfac = 1.0 / (gamma * gamma);
    for (long long idx = 0; idx < ncell; ++idx) {
        const int m[3] = {(int)(idx % n[0]), (int)((idx / n[0]) % n[1]), (int)(idx / ((long long)n[0] * n[1]))};
        double lam = M[0].ev[m[0]] + (active[1] ? M[1].ev[m[1]] : 0.0) + zfac * M[2].ev[m[2]];
        // on an all-periodic grid the first mode of every axis is the constant (lam = 0)
        phi[idx] = (all_periodic && m[0] == 0 && m[1] == 0 && m[2] == 0) ? 0.0 : -phi[idx] / lam;
    }
    for (int a = 0; a < 3; ++a)
        if (active[a]) transform_axis(phi, n, a, M[a], false);

    // phi at node (i, j, k) + e_a: wrapped, or 0 beyond an absorbing face
    auto phi_next = [&](int i, int j, int k, int a) -> double {
        int c[3] = {i, j, k};
        c[a] += 1;
        if (c[a] == n[a]) {
            if (G.bc[a] != PIC_PERIODIC) return 0.0;
            c[a] = 0;
        }
        return phi[c[0] + (long long)n[0] * (c[1] + (long long)n[1] * c[2])];
    };
    for (int c = 0; c < 6; ++c)
        if (F.comp[c].empty()) F.comp[c].assign(ncell, 0.0);
    std::vector<double> ex(ncell), ey(ncell, 0.0);
    for (int k = 0; k < n[2]; ++k)
        for (int j = 0; j < n[1]; ++j)
            for (int i = 0; i < n[0]; ++i) {
                const long long id = i + (long long)n[0] * (j + (long long)n[1] * k);
                const double p0 = phi[id];
                ex[id] = -(phi_next(i, j, k, 0) - p0) / G.dx[0];
                if (active[1]) ey[id] = -(phi_next(i, j, k, 1) - p0) / G.dx[1];
                F.comp[0][id] += ex[id];
                F.comp[1][id] += ey[id];
                F.comp[2][id] += -(phi_next(i, j, k, 2) - p0) / G.dx[2] * zfac;
            }
    // B at z + 1/2 from E averaged over the nodes k and k + 1 (E beyond an absorbing
    // z face is zero)
    for (int k = 0; k < n[2]; ++k) {
        const bool top = k + 1 == n[2];
        const int k1 = top ? 0 : k + 1;
        const bool zero_above = top && G.bc[2] != PIC_PERIODIC;
        for (int j = 0; j < n[1]; ++j)
            for (int i = 0; i < n[0]; ++i) {
                const long long id = i + (long long)n[0] * (j + (long long)n[1] * k);
                const long long up = i + (long long)n[0] * (j + (long long)n[1] * k1);
                const double ex_up = zero_above ? 0.0 : ex[up], ey_up = zero_above ? 0.0 : ey[up];
                F.comp[3][id] += -beta * 0.5 * (ey[id] + ey_up);
                F.comp[4][id] += beta * 0.5 * (ex[id] + ex_up);
            }
    }
}

}  // namespace pic
