/*
 * pic_oracle.c -- plain FP64 CPU reference of the boosted-frame explicit EM-PIC step.
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the test suite, the smoke check and the
 * benchmark's CPU-baseline leg, never by the product path.  It shares no code with the
 * CUDA library.  Written for clarity: every sum runs over an explicit, generous node
 * window and evaluates the shape function from its definition; no blocking, fusion or
 * reordering beyond what each method states.
 *
 * Method passages followed (Vay et al., arXiv:0909.5603):
 *   Sec. 2  -- Boris pusher and its inexact E + v x B cancellation; the Vay pusher that
 *              solves the implicit Lorentz-force system analytically (details in the
 *              paper's reference VayPOP08: Vay, Phys. Plasmas 15, 056701 (2008)).
 *   Sec. 2  -- lab -> boosted-frame transformation of laser (Doppler shift) and plasma
 *              (denser, drifting) inputs; beam particles boosted then drifted to a common
 *              boosted time ("frozen" drifting macro-particles).
 *   Sec. 2  -- low-pass digital filtering of the current (binomial 1-2-1 passes).
 * Steps the paper names but does not write out, restated from their published sources:
 *   Yee FDTD (Yee 1966), charge-conserving current deposition (Esirkepov, Comput. Phys.
 *   Commun. 135, 144 (2001)), B-spline shape factors of order 1 and 2, SplitMix64
 *   (Steele, Lea, Flood, OOPSLA 2014).
 * Where the paper is silent (absorbing layer, crossing rule, seeds, 2D3V geometry) the
 * choice taken is stated where it is used and marked "reading" below.
 *
 * Parity pins: every public function here is pinned by a closed form, invariant or
 * brute-force check in tests/test_oracle_*.py.
 */
#include "pic_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

struct orc_sim {
    int ndim, n[3], bc[3], order, pusher, filter_passes, tile[3], absorb_cells;
    int active[3];
    double dx[3], dt, q, m, absorb_strength;
    int64_t ncell;
    double *f[ORC_NCOMP];
    int64_t np, cap;
    int32_t *cell, *id;
    double *off, *u, *w; /* off and u: 3 per particle, interleaved */
    int64_t n_lost, step;
    /* ion background of a lab-frame plasma load (see orc_ion_integral) */
    int ion;
    double ion_n0, ion_zs, ion_ramp, ion_gb, ion_beta;
    int64_t n_pp; /* particle phases run since the last load */
    int solver;   /* ORC_SOLVER_YEE or ORC_SOLVER_CK */
    /* beam injection through a lab-fixed plane (see orc_set_injection) */
    int inj;
    double inj_zb, inj_beta; /* the plane in this frame: z' = inj_zb - inj_beta t' */
    int32_t inj_first;       /* first beam id, or -1: the beam of the last lab-frame load */
    int32_t beam_id0;        /* first id of that beam (INT32_MAX: none) */
    /* laser antenna on a lab-fixed plane (see orc_set_antenna) */
    int64_t n_mx;            /* Maxwell phases run since the last load */
    int ant;
    double ant_zb, ant_beta, ant_t0; /* plane z' = ant_zb - ant_beta t'; t' at the set */
    int64_t ant_n;                   /* Maxwell phases since the set */
    double ant_w0, ant_xc, ant_yc;   /* transverse profile exp(-(x^2 + y^2) / w0^2) */
    int64_t ant_lo, ant_na;          /* 1D lattice: nodes ant_lo .. ant_lo + ant_na - 1 */
    double *ant_e, *ant_b;           /* its E_x on the nodes, B_y half a node above */
};

/* Yee staggering (in cells) of each component along each axis. */
static const double STAG[ORC_NCOMP][3] = {
    {0.5, 0.0, 0.0}, {0.0, 0.5, 0.0}, {0.0, 0.0, 0.5}, /* Ex Ey Ez */
    {0.0, 0.5, 0.5}, {0.5, 0.0, 0.5}, {0.5, 0.5, 0.0}, /* Bx By Bz */
    {0.5, 0.0, 0.0}, {0.0, 0.5, 0.0}, {0.0, 0.0, 0.5}, /* Jx Jy Jz */
};

/* ------------------------------------------------------------------------------------
 * Shape factors: centred B-splines.  Order 1: S(x) = 1 - |x| for |x| < 1.
 * Order 2: S(x) = 3/4 - x^2 for |x| <= 1/2, (3/2 - |x|)^2 / 2 for 1/2 < |x| < 3/2.
 * ---------------------------------------------------------------------------------- */
double orc_shape(int order, double x)
{
    double a = fabs(x);
    if (order == 1) return a < 1.0 ? 1.0 - a : 0.0;
    if (a <= 0.5) return 0.75 - a * a;
    if (a < 1.5) return 0.5 * (1.5 - a) * (1.5 - a);
    return 0.0;
}

/* ------------------------------------------------------------------------------------
 * Vay pusher (Sec. 2; VayPOP08).  With h = q dt / (2 m) and c = 1 the velocity average
 * in the magnetic term is (v^{n+1/2} + v^{n-1/2})/2, which gives
 *   u' = u^{n-1/2} + 2h E + h v^{n-1/2} x B,   tau = h B,   u* = u'.tau,
 *   sigma = gamma'^2 - tau^2,   gamma'^2 = 1 + u'^2,
 *   gamma^{n+1/2} = sqrt( (sigma + sqrt(sigma^2 + 4 (tau^2 + u*^2))) / 2 ),
 *   t = tau / gamma^{n+1/2},  s = 1 / (1 + t^2),
 *   u^{n+1/2} = s [u' + (u'.t) t + u' x t].
 * Where sigma < 0 the root is taken in its cancellation-free form
 *   gamma^2 = 2 (tau^2 + u*^2) / (sqrt(sigma^2 + 4 (tau^2 + u*^2)) - sigma)
 * (algebraically the same root; a reading: the paper gives no formula, and this form
 * avoids the cancellation of sigma + sqrt(...) when sigma < 0).
 * ---------------------------------------------------------------------------------- */
void orc_push_vay(double u[3], const double E[3], const double B[3], double q_over_m, double dt)
{
    double h = 0.5 * q_over_m * dt;
    double g = sqrt(1.0 + u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    double v[3] = {u[0] / g, u[1] / g, u[2] / g};
    double up[3] = {
        u[0] + 2.0 * h * E[0] + h * (v[1] * B[2] - v[2] * B[1]),
        u[1] + 2.0 * h * E[1] + h * (v[2] * B[0] - v[0] * B[2]),
        u[2] + 2.0 * h * E[2] + h * (v[0] * B[1] - v[1] * B[0]),
    };
    double tau[3] = {h * B[0], h * B[1], h * B[2]};
    double tau2 = tau[0] * tau[0] + tau[1] * tau[1] + tau[2] * tau[2];
    double ustar = up[0] * tau[0] + up[1] * tau[1] + up[2] * tau[2];
    double gp2 = 1.0 + up[0] * up[0] + up[1] * up[1] + up[2] * up[2];
    double sigma = gp2 - tau2;
    double root = sqrt(sigma * sigma + 4.0 * (tau2 + ustar * ustar));
    double gnew2 = sigma >= 0.0 ? 0.5 * (sigma + root) : 2.0 * (tau2 + ustar * ustar) / (root - sigma);
    double gnew = sqrt(gnew2);
    double t[3] = {tau[0] / gnew, tau[1] / gnew, tau[2] / gnew};
    double s = 1.0 / (1.0 + t[0] * t[0] + t[1] * t[1] + t[2] * t[2]);
    double upt = up[0] * t[0] + up[1] * t[1] + up[2] * t[2];
    double r0 = up[0] + upt * t[0] + (up[1] * t[2] - up[2] * t[1]);
    double r1 = up[1] + upt * t[1] + (up[2] * t[0] - up[0] * t[2]);
    double r2 = up[2] + upt * t[2] + (up[0] * t[1] - up[1] * t[0]);
    u[0] = s * r0;
    u[1] = s * r1;
    u[2] = s * r2;
}

/* ------------------------------------------------------------------------------------
 * Boris pusher (Sec. 2; BorisICNSP): half electric kick, magnetic rotation, half kick.
 *   u- = u + h E;  gamma- = sqrt(1 + u-^2);  t = h B / gamma-;  s = 2 t / (1 + t^2);
 *   u' = u- + u- x t;  u+ = u- + u' x s;  u^{n+1/2} = u+ + h E.
 * ---------------------------------------------------------------------------------- */
void orc_push_boris(double u[3], const double E[3], const double B[3], double q_over_m, double dt)
{
    double h = 0.5 * q_over_m * dt;
    double um[3] = {u[0] + h * E[0], u[1] + h * E[1], u[2] + h * E[2]};
    double gm = sqrt(1.0 + um[0] * um[0] + um[1] * um[1] + um[2] * um[2]);
    double t[3] = {h * B[0] / gm, h * B[1] / gm, h * B[2] / gm};
    double t2 = t[0] * t[0] + t[1] * t[1] + t[2] * t[2];
    double s[3] = {2.0 * t[0] / (1.0 + t2), 2.0 * t[1] / (1.0 + t2), 2.0 * t[2] / (1.0 + t2)};
    double uprime[3] = {
        um[0] + (um[1] * t[2] - um[2] * t[1]),
        um[1] + (um[2] * t[0] - um[0] * t[2]),
        um[2] + (um[0] * t[1] - um[1] * t[0]),
    };
    double upl[3] = {
        um[0] + (uprime[1] * s[2] - uprime[2] * s[1]),
        um[1] + (uprime[2] * s[0] - uprime[0] * s[2]),
        um[2] + (uprime[0] * s[1] - uprime[1] * s[0]),
    };
    u[0] = upl[0] + h * E[0];
    u[1] = upl[1] + h * E[1];
    u[2] = upl[2] + h * E[2];
}

/* ------------------------------------------------------------------------------------
 * Lorentz boost along +z with gamma_b (beta_b = sqrt(1 - 1/gamma_b^2)), Sec. 2 inputs.
 * Fields: E'x = g(Ex - b By), E'y = g(Ey + b Bx), E'z = Ez,
 *         B'x = g(Bx + b Ey), B'y = g(By - b Ex), B'z = Bz   (c = 1).
 * Events: t' = g(t - b z), z' = g(z - b t), x' = x, y' = y.
 * Momenta (u = gamma v): u'z = g(uz - b gamma_p), u'x = ux, u'y = uy.
 * ---------------------------------------------------------------------------------- */
static double boost_beta(double gb) { return sqrt(1.0 - 1.0 / (gb * gb)); }

void orc_boost_fields(double gb, const double E[3], const double B[3], double Ep[3], double Bp[3])
{
    double b = boost_beta(gb);
    Ep[0] = gb * (E[0] - b * B[1]);
    Ep[1] = gb * (E[1] + b * B[0]);
    Ep[2] = E[2];
    Bp[0] = gb * (B[0] + b * E[1]);
    Bp[1] = gb * (B[1] - b * E[0]);
    Bp[2] = B[2];
}

void orc_boost_event(double gb, const double tx[4], const double u[3], double txp[4], double up[3])
{
    double b = boost_beta(gb);
    double gp = sqrt(1.0 + u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    txp[0] = gb * (tx[0] - b * tx[3]);
    txp[1] = tx[1];
    txp[2] = tx[2];
    txp[3] = gb * (tx[3] - b * tx[0]);
    up[0] = u[0];
    up[1] = u[1];
    up[2] = gb * (u[2] - b * gp);
}

/* ------------------------------------------------------------------------------------
 * SplitMix64 (Steele, Lea, Flood 2014) used as a counter-based generator: the state is
 * seed ^ (stream << 40) ^ counter, advanced once by the golden gamma and finalised.
 * Uniform: top 53 bits * 2^-53 in [0, 1).  Normal: Box-Muller, cos branch, first
 * uniform taken as 1 - U so the logarithm never sees zero.
 * ---------------------------------------------------------------------------------- */
uint64_t orc_splitmix64(uint64_t seed, uint64_t stream, uint64_t counter)
{
    uint64_t z = (seed ^ (stream << 40) ^ counter) + 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

double orc_uniform(uint64_t seed, uint64_t stream, uint64_t counter)
{
    return (double)(orc_splitmix64(seed, stream, counter) >> 11) * (1.0 / 9007199254740992.0);
}

double orc_normal(uint64_t seed, uint64_t stream, uint64_t counter)
{
    /* two uniforms from the stream pair (stream, stream + 1) at the same counter */
    double u1 = 1.0 - orc_uniform(seed, stream, counter);
    double u2 = orc_uniform(seed, stream + 1, counter);
    return sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
}

/* ------------------------------------------------------------------------------------
 * Simulation state
 * ---------------------------------------------------------------------------------- */
orc_sim *orc_create(int ndim, const int n[3], const int bc[3], const double dx[3], double dt,
                    int order, int pusher, int filter_passes, const int tile[3], double q,
                    double m, int absorb_cells, double absorb_strength)
{
    orc_sim *s = (orc_sim *)calloc(1, sizeof(orc_sim));
    s->ndim = ndim;
    for (int a = 0; a < 3; ++a) {
        s->n[a] = n[a];
        s->bc[a] = bc[a];
        s->dx[a] = dx[a];
        s->tile[a] = tile[a];
        s->active[a] = 1;
    }
    if (ndim == 2) { /* 2D3V: the x-z plane, y invariant (reading) */
        s->n[1] = 1;
        s->tile[1] = 1;
        s->active[1] = 0;
    }
    s->dt = dt;
    s->order = order;
    s->pusher = pusher;
    s->filter_passes = filter_passes;
    s->q = q;
    s->m = m;
    s->absorb_cells = absorb_cells;
    s->absorb_strength = absorb_strength;
    s->ncell = (int64_t)s->n[0] * s->n[1] * s->n[2];
    s->beam_id0 = INT32_MAX;
    for (int c = 0; c < ORC_NCOMP; ++c) s->f[c] = (double *)calloc((size_t)s->ncell, sizeof(double));
    return s;
}

static void free_particles(orc_sim *s)
{
    free(s->cell);
    free(s->id);
    free(s->off);
    free(s->u);
    free(s->w);
    s->cell = s->id = NULL;
    s->off = s->u = s->w = NULL;
    s->np = s->cap = 0;
}

void orc_destroy(orc_sim *s)
{
    if (!s) return;
    for (int c = 0; c < ORC_NCOMP; ++c) free(s->f[c]);
    free_particles(s);
    free(s->ant_e);
    free(s->ant_b);
    free(s);
}

void orc_set_field(orc_sim *s, int comp, const double *data)
{
    memcpy(s->f[comp], data, (size_t)s->ncell * sizeof(double));
}

void orc_get_field(const orc_sim *s, int comp, double *out)
{
    memcpy(out, s->f[comp], (size_t)s->ncell * sizeof(double));
}

static void reserve(orc_sim *s, int64_t cap)
{
    if (cap <= s->cap) return;
    s->cell = (int32_t *)realloc(s->cell, (size_t)cap * sizeof(int32_t));
    s->id = (int32_t *)realloc(s->id, (size_t)cap * sizeof(int32_t));
    s->off = (double *)realloc(s->off, (size_t)cap * 3 * sizeof(double));
    s->u = (double *)realloc(s->u, (size_t)cap * 3 * sizeof(double));
    s->w = (double *)realloc(s->w, (size_t)cap * sizeof(double));
    s->cap = cap;
}

int orc_set_particles(orc_sim *s, int64_t np, const int32_t *cell, const double *off,
                      const double *u, const double *w, const int32_t *id)
{
    free_particles(s);
    reserve(s, np > 0 ? np : 1);
    for (int64_t p = 0; p < np; ++p) {
        if (cell[p] < 0 || cell[p] >= s->ncell) return -1;
        for (int a = 0; a < 3; ++a) {
            double o = off[3 * p + a];
            if (!(o >= 0.0 && o < 1.0)) return -2;
        }
    }
    s->beam_id0 = INT32_MAX; /* no lab-frame beam */
    s->n_mx = 0;
    orc_set_antenna(s, 0, 1.0, NULL, 0.0); /* a load removes the antenna */
    memcpy(s->cell, cell, (size_t)np * sizeof(int32_t));
    memcpy(s->off, off, (size_t)np * 3 * sizeof(double));
    memcpy(s->u, u, (size_t)np * 3 * sizeof(double));
    memcpy(s->w, w, (size_t)np * sizeof(double));
    for (int64_t p = 0; p < np; ++p) {
        s->id[p] = id ? id[p] : (int32_t)p;
        if (!s->active[1]) s->off[3 * p + 1] = 0.0;
    }
    s->np = np;
    s->n_lost = 0;
    s->ion = 0; /* particles loaded directly carry no ion background */
    s->n_pp = 0;
    orc_sort(s);
    return 0;
}

int64_t orc_num_particles(const orc_sim *s) { return s->np; }

void orc_get_particles(const orc_sim *s, int32_t *cell, double *off, double *u, double *w,
                       int32_t *id)
{
    if (cell) memcpy(cell, s->cell, (size_t)s->np * sizeof(int32_t));
    if (off) memcpy(off, s->off, (size_t)s->np * 3 * sizeof(double));
    if (u) memcpy(u, s->u, (size_t)s->np * 3 * sizeof(double));
    if (w) memcpy(w, s->w, (size_t)s->np * sizeof(double));
    if (id) memcpy(id, s->id, (size_t)s->np * sizeof(int32_t));
}

static void cell_coords(const orc_sim *s, int32_t cell, int c[3])
{
    c[0] = cell % s->n[0];
    c[1] = (cell / s->n[0]) % s->n[1];
    c[2] = cell / (s->n[0] * s->n[1]);
}

/* ------------------------------------------------------------------------------------
 * Canonical particle order (reading): a stable sort by tile id, tile id = tile
 * coordinates lexicographic with z slowest.  Applied after loading and after every
 * step, so the array order at a step boundary is always this sort applied to the
 * previous order.  Implemented as a counting sort.
 * ---------------------------------------------------------------------------------- */
static int64_t tile_of(const orc_sim *s, int32_t cell)
{
    int c[3];
    cell_coords(s, cell, c);
    int nt0 = (s->n[0] + s->tile[0] - 1) / s->tile[0];
    int nt1 = (s->n[1] + s->tile[1] - 1) / s->tile[1];
    return (int64_t)(c[0] / s->tile[0]) + (int64_t)nt0 * ((c[1] / s->tile[1]) + (int64_t)nt1 * (c[2] / s->tile[2]));
}

void orc_sort(orc_sim *s)
{
    int64_t ntiles = 1;
    for (int a = 0; a < 3; ++a) ntiles *= (s->n[a] + s->tile[a] - 1) / s->tile[a];
    int64_t *start = (int64_t *)calloc((size_t)ntiles + 1, sizeof(int64_t));
    for (int64_t p = 0; p < s->np; ++p) start[tile_of(s, s->cell[p]) + 1]++;
    for (int64_t t = 0; t < ntiles; ++t) start[t + 1] += start[t];
    int32_t *cell = (int32_t *)malloc((size_t)(s->np + 1) * sizeof(int32_t));
    int32_t *id = (int32_t *)malloc((size_t)(s->np + 1) * sizeof(int32_t));
    double *off = (double *)malloc((size_t)(s->np + 1) * 3 * sizeof(double));
    double *u = (double *)malloc((size_t)(s->np + 1) * 3 * sizeof(double));
    double *w = (double *)malloc((size_t)(s->np + 1) * sizeof(double));
    for (int64_t p = 0; p < s->np; ++p) {
        int64_t d = start[tile_of(s, s->cell[p])]++;
        cell[d] = s->cell[p];
        id[d] = s->id[p];
        w[d] = s->w[p];
        for (int a = 0; a < 3; ++a) {
            off[3 * d + a] = s->off[3 * p + a];
            u[3 * d + a] = s->u[3 * p + a];
        }
    }
    if (s->np > 0) { /* an empty set may have no arrays yet */
        memcpy(s->cell, cell, (size_t)s->np * sizeof(int32_t));
        memcpy(s->id, id, (size_t)s->np * sizeof(int32_t));
        memcpy(s->off, off, (size_t)s->np * 3 * sizeof(double));
        memcpy(s->u, u, (size_t)s->np * 3 * sizeof(double));
        memcpy(s->w, w, (size_t)s->np * sizeof(double));
    }
    free(cell);
    free(id);
    free(off);
    free(u);
    free(w);
    free(start);
}

/* ------------------------------------------------------------------------------------
 * Grid access with boundaries: periodic axes wrap, absorbing axes read zero outside and
 * drop deposits outside.  Returns -1 when the node lies outside an absorbing axis.
 * ---------------------------------------------------------------------------------- */
static int64_t node_index(const orc_sim *s, int i, int j, int k)
{
    int c[3] = {i, j, k};
    for (int a = 0; a < 3; ++a) {
        if (!s->active[a]) {
            c[a] = 0;
            continue;
        }
        if (c[a] < 0 || c[a] >= s->n[a]) {
            if (s->bc[a] == ORC_ABSORBING) return -1;
            c[a] = ((c[a] % s->n[a]) + s->n[a]) % s->n[a];
        }
    }
    return (int64_t)c[0] + (int64_t)s->n[0] * ((int64_t)c[1] + (int64_t)s->n[1] * c[2]);
}

static double fget(const orc_sim *s, int comp, int i, int j, int k)
{
    int64_t idx = node_index(s, i, j, k);
    return idx < 0 ? 0.0 : s->f[comp][idx];
}

static void fadd(orc_sim *s, int comp, int i, int j, int k, double v)
{
    int64_t idx = node_index(s, i, j, k);
    if (idx >= 0) s->f[comp][idx] += v;
}

/* Node window [c - 2, c + 3] per active axis covers every node with a non-zero order-1
 * or order-2 weight for a particle in cell c, before and after a move of under one
 * cell.  Inactive axes use the single node 0. */
#define WIN 6
static void window(const orc_sim *s, int a, int c, int *lo, int *cnt)
{
    if (!s->active[a]) {
        *lo = 0;
        *cnt = 1;
    } else {
        *lo = c - 2;
        *cnt = WIN;
    }
}

/* Weight of node index i (at position i + stag) for a particle at cell c + offset o
 * along axis a; 1 on inactive axes. */
static double node_weight(const orc_sim *s, int a, int c, double o, int i, double stag)
{
    if (!s->active[a]) return 1.0;
    return orc_shape(s->order, (double)(c - i) + o - stag);
}

/* ------------------------------------------------------------------------------------
 * Field gather (momentum-conserving direct interpolation, same shape order for every
 * component): F_p = sum_ijk F_ijk S(x_p - X_i) S(y_p - Y_j) S(z_p - Z_k), each component
 * at its own staggered Yee position.
 * ---------------------------------------------------------------------------------- */
void orc_gather(const orc_sim *s, int32_t cell, const double off[3], double E[3], double B[3])
{
    int c[3], lo[3], cnt[3];
    cell_coords(s, cell, c);
    for (int a = 0; a < 3; ++a) window(s, a, c[a], &lo[a], &cnt[a]);
    for (int comp = ORC_EX; comp <= ORC_BZ; ++comp) {
        double acc = 0.0;
        for (int kk = 0; kk < cnt[2]; ++kk) {
            int k = lo[2] + kk;
            double wz = node_weight(s, 2, c[2], off[2], k, STAG[comp][2]);
            if (wz == 0.0) continue;
            for (int jj = 0; jj < cnt[1]; ++jj) {
                int j = lo[1] + jj;
                double wy = node_weight(s, 1, c[1], off[1], j, STAG[comp][1]);
                if (wy == 0.0) continue;
                for (int ii = 0; ii < cnt[0]; ++ii) {
                    int i = lo[0] + ii;
                    double wx = node_weight(s, 0, c[0], off[0], i, STAG[comp][0]);
                    if (wx == 0.0) continue;
                    acc += wx * wy * wz * fget(s, comp, i, j, k);
                }
            }
        }
        if (comp < ORC_BX)
            E[comp] = acc;
        else
            B[comp - ORC_BX] = acc;
    }
}

/* ------------------------------------------------------------------------------------
 * Esirkepov charge-conserving deposit for one particle moving from (c0, o0) to
 * (c1, o1) during dt with weight w.  With S0, S1 the node shapes before and after and
 * DS = S1 - S0, in 3D
 *   Wx = DSx (S0y S0z + DSy S0z / 2 + S0y DSz / 2 + DSy DSz / 3)   (cyclic for y, z),
 *   Jx(i+1/2) - Jx(i-1/2) = -(q w / dV) (dx / dt) Wx(i),
 * summed along x from zero at the left of the window.  In 2D3V (x-z plane, y
 * invariant) Wx = DSx (S0z + DSz / 2), Wz = DSz (S0x + DSx / 2) and the out-of-plane
 * current is Jy = (q w / dV) vy (S0x S0z + DSx S0z / 2 + S0x DSz / 2 + DSx DSz / 3).
 * ---------------------------------------------------------------------------------- */
static void esirkepov(orc_sim *s, const int c0[3], const double o0[3], const int c1[3],
                      const double o1[3], double w, double vy_for_2d)
{
    int lo[3], cnt[3];
    double S0[3][WIN], DS[3][WIN];
    for (int a = 0; a < 3; ++a) {
        window(s, a, c0[a], &lo[a], &cnt[a]);
        for (int ii = 0; ii < cnt[a]; ++ii) {
            int i = lo[a] + ii;
            double s0 = node_weight(s, a, c0[a], o0[a], i, 0.0);
            double s1 = node_weight(s, a, c1[a], o1[a], i, 0.0);
            S0[a][ii] = s0;
            DS[a][ii] = s1 - s0;
        }
    }
    double dV = s->dx[0] * s->dx[1] * s->dx[2];
    double qw = s->q * w / dV;
    if (s->ndim == 3) {
        for (int a = 0; a < 3; ++a) {
            int b = (a + 1) % 3, cc = (a + 2) % 3; /* the two transverse axes */
            double fac = -qw * s->dx[a] / s->dt;
            for (int jb = 0; jb < cnt[b]; ++jb) {
                for (int jc = 0; jc < cnt[cc]; ++jc) {
                    double Y = S0[b][jb] * S0[cc][jc] + 0.5 * DS[b][jb] * S0[cc][jc] +
                               0.5 * S0[b][jb] * DS[cc][jc] + (1.0 / 3.0) * DS[b][jb] * DS[cc][jc];
                    double run = 0.0;
                    for (int ia = 0; ia < cnt[a]; ++ia) {
                        run += DS[a][ia] * Y; /* sum of W over nodes up to this one */
                        int idx[3];
                        idx[a] = lo[a] + ia;
                        idx[b] = lo[b] + jb;
                        idx[cc] = lo[cc] + jc;
                        fadd(s, ORC_JX + a, idx[0], idx[1], idx[2], fac * run);
                    }
                }
            }
        }
    } else {
        /* x (axis 0) and z (axis 2) in-plane */
        for (int pass = 0; pass < 2; ++pass) {
            int a = pass == 0 ? 0 : 2, b = pass == 0 ? 2 : 0;
            double fac = -qw * s->dx[a] / s->dt;
            for (int jb = 0; jb < cnt[b]; ++jb) {
                double Y = S0[b][jb] + 0.5 * DS[b][jb];
                double run = 0.0;
                for (int ia = 0; ia < cnt[a]; ++ia) {
                    run += DS[a][ia] * Y;
                    int idx[3] = {0, 0, 0};
                    idx[a] = lo[a] + ia;
                    idx[b] = lo[b] + jb;
                    fadd(s, ORC_JX + a, idx[0], idx[1], idx[2], fac * run);
                }
            }
        }
        double fy = qw * vy_for_2d;
        for (int kk = 0; kk < cnt[2]; ++kk) {
            for (int ii = 0; ii < cnt[0]; ++ii) {
                double v = S0[0][ii] * S0[2][kk] + 0.5 * DS[0][ii] * S0[2][kk] +
                           0.5 * S0[0][ii] * DS[2][kk] + (1.0 / 3.0) * DS[0][ii] * DS[2][kk];
                fadd(s, ORC_JY, lo[0] + ii, 0, lo[2] + kk, fy * v);
            }
        }
    }
}

/* ------------------------------------------------------------------------------------
 * Particle phase of one step: zero J; for each particle in array order gather E^n, B^n,
 * push u^{n-1/2} -> u^{n+1/2}, move x^n -> x^{n+1} = x^n + dt u/gamma, deposit J^{n+1/2};
 * particles whose new cell is outside an absorbing axis are removed after depositing.
 * Position update (reading): off += dt v / dx, k = floor(off), cell += k, off -= k; an
 * offset that rounds to exactly 1 after the subtraction becomes 0 in the next cell.
 * Then the canonical stable sort by tile.
 * ---------------------------------------------------------------------------------- */
/* ------------------------------------------------------------------------------------
 * Ion background of a lab-frame plasma (Sec. 2, reading).  The plasma's ions are at rest
 * in the lab frame, where they neutralise the electrons; only the electrons are
 * macro-particles here, so the ions are a rigid charge density.  In the boosted frame their density is the lab
 * profile contracted by gamma_b, rho_i0(s) = -q gamma_b n0 p(gamma_b s) at t' = 0 for s in
 * the box [0, Lz), zero outside it (the ions of the loaded volume only, like the
 * electrons), and it moves rigidly at -beta_b: rho_i(z, t') = rho_i0(z + beta_b t'),
 * wrapped into the box when z is periodic.
 *
 * orc_ion_integral(a, b) = integral of rho_i0 over [a, b] (box coordinates at t' = 0).
 * p is piecewise linear (zero, ramp, plateau), so each piece is integrated exactly by the
 * trapezoid rule.  From it, with t^n = n dt:
 *   current on the Jz face z_f = (k + 1/2) dz during step n (the ions crossing it):
 *     Jz_i = -orc_ion_integral(z_f + beta t^n, z_f + beta t^{n+1}) / dt,
 *   charge on node k (average over its dual cell [z_k - dz/2, z_k + dz/2]):
 *     rho_i = orc_ion_integral(z_k - dz/2 + beta t, z_k + dz/2 + beta t) / dz,
 * so the discrete continuity equation holds for the ions by construction.
 * ---------------------------------------------------------------------------------- */
static double ion_piece(const orc_sim *s, double lo, double hi)
{
    /* integral of rho_i0 over [lo, hi], both inside [0, Lz] */
    double g = s->ion_gb, rmax = -s->q * g * s->ion_n0;
    double za = s->ion_zs / g, zb = (s->ion_zs + s->ion_ramp) / g;
    double total = 0.0;
    /* ramp piece [za, zb): rho = rmax (g z - zs) / ramp, linear */
    double a = lo > za ? lo : za, b = hi < zb ? hi : zb;
    if (b > a) {
        double fa = rmax * (g * a - s->ion_zs) / s->ion_ramp;
        double fb = rmax * (g * b - s->ion_zs) / s->ion_ramp;
        total += 0.5 * (fa + fb) * (b - a);
    }
    /* plateau [zb, inf): rho = rmax */
    a = lo > zb ? lo : zb;
    b = hi;
    if (b > a) total += rmax * (b - a);
    return total;
}

double orc_ion_integral(const orc_sim *s, double a, double b)
{
    if (!s->ion || !(b > a)) return 0.0;
    double Lz = s->n[2] * s->dx[2];
    if (s->bc[2] == ORC_ABSORBING || !s->active[2]) {
        double lo = a > 0.0 ? a : 0.0, hi = b < Lz ? b : Lz;
        return hi > lo ? ion_piece(s, lo, hi) : 0.0;
    }
    /* periodic: sum over the periods [m Lz, (m+1) Lz) that [a, b] meets */
    double total = 0.0;
    for (double m = floor(a / Lz); m * Lz < b; m += 1.0) {
        double lo = a > m * Lz ? a : m * Lz, hi = b < (m + 1.0) * Lz ? b : (m + 1.0) * Lz;
        if (hi > lo) total += ion_piece(s, lo - m * Lz, hi - m * Lz);
    }
    return total;
}

static void add_ion_current(orc_sim *s)
{
    double t0 = (double)s->n_pp * s->dt, t1 = (double)(s->n_pp + 1) * s->dt;
    for (int k = 0; k < s->n[2]; ++k) {
        double zf = (k + 0.5) * s->dx[2];
        double jz = -orc_ion_integral(s, zf + s->ion_beta * t0, zf + s->ion_beta * t1) / s->dt;
        for (int j = 0; j < s->n[1]; ++j)
            for (int i = 0; i < s->n[0]; ++i) s->f[ORC_JZ][node_index(s, i, j, k)] += jz;
    }
}

/* ------------------------------------------------------------------------------------
 * Beam injection through a plane fixed in the laboratory (Sec. 2: the beam enters the
 * boosted frame through a transverse lab-fixed plane that drifts in this frame, and the
 * beam still upstream of it is represented by frozen macro-particles that drift).
 * Reading: the lab plane z = z_lab sits in this frame at z' = z_lab / gamma_b - beta_b t';
 * a beam particle (id >= first_id; first_id < 0: the beam of the last lab-frame load,
 * whose ids follow the plasma's) whose position z'^n at t^n = n dt lies strictly upstream
 * of the plane, z'^n / dz < (z_lab / gamma_b - beta_b t^n) / dz (compared in FP64 in cell
 * units), is frozen for that step: no field acts on it (its momentum is kept), it moves
 * at its own velocity and deposits its current like any particle, so the beam's charge
 * near the plane is present for the space-charge field.  Downstream of the plane it is
 * pushed as usual.  With a lab beam that drifts freely upstream of z_lab this reproduces
 * the lab-frame history: a frozen particle's straight worldline is the lab one.
 * ---------------------------------------------------------------------------------- */
void orc_set_injection(orc_sim *s, int enable, double gamma_b, double z_lab, int32_t first_id)
{
    s->inj = enable != 0;
    s->inj_zb = z_lab / gamma_b;
    s->inj_beta = boost_beta(gamma_b);
    s->inj_first = first_id;
}

static int frozen_at_plane(const orc_sim *s, int64_t p)
{
    if (!s->inj) return 0;
    int32_t id0 = s->inj_first >= 0 ? s->inj_first : s->beam_id0;
    if (s->id[p] < id0) return 0;
    double zp = (s->inj_zb - s->inj_beta * ((double)s->n_pp * s->dt)) / s->dx[2];
    int c[3];
    cell_coords(s, s->cell[p], c);
    return (double)c[2] + s->off[3 * p + 2] < zp;
}

int64_t orc_num_frozen(const orc_sim *s)
{
    int64_t n = 0;
    for (int64_t p = 0; p < s->np; ++p) n += frozen_at_plane(s, p);
    return n;
}

void orc_particle_phase(orc_sim *s)
{
    for (int c = ORC_JX; c <= ORC_JZ; ++c) memset(s->f[c], 0, (size_t)s->ncell * sizeof(double));
    if (s->ion && s->active[2]) add_ion_current(s);
    int64_t keep = 0;
    for (int64_t p = 0; p < s->np; ++p) {
        double E[3], B[3];
        double *o = &s->off[3 * p];
        double *u = &s->u[3 * p];
        if (!frozen_at_plane(s, p)) {
            orc_gather(s, s->cell[p], o, E, B);
            if (s->pusher == ORC_VAY)
                orc_push_vay(u, E, B, s->q / s->m, s->dt);
            else
                orc_push_boris(u, E, B, s->q / s->m, s->dt);
        }
        double g = sqrt(1.0 + u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
        int c0[3], c1[3];
        double o0[3] = {o[0], o[1], o[2]}, o1[3];
        cell_coords(s, s->cell[p], c0);
        int dead = 0;
        for (int a = 0; a < 3; ++a) {
            c1[a] = c0[a];
            o1[a] = o0[a];
            if (!s->active[a]) continue;
            double x = o0[a] + s->dt * (u[a] / g) / s->dx[a];
            double k = floor(x);
            x -= k;
            c1[a] = c0[a] + (int)k;
            if (x >= 1.0) {
                x = 0.0;
                c1[a] += 1;
            }
            o1[a] = x;
        }
        esirkepov(s, c0, o0, c1, o1, s->w[p], u[1] / g);
        for (int a = 0; a < 3; ++a) {
            if (!s->active[a]) continue;
            if (c1[a] < 0 || c1[a] >= s->n[a]) {
                if (s->bc[a] == ORC_ABSORBING)
                    dead = 1;
                else
                    c1[a] = ((c1[a] % s->n[a]) + s->n[a]) % s->n[a];
            }
        }
        if (dead) {
            s->n_lost++;
            continue;
        }
        s->cell[keep] = (int32_t)(c1[0] + s->n[0] * (c1[1] + s->n[1] * c1[2]));
        s->id[keep] = s->id[p];
        s->w[keep] = s->w[p];
        for (int a = 0; a < 3; ++a) {
            s->off[3 * keep + a] = o1[a];
            s->u[3 * keep + a] = u[a];
        }
        keep++;
    }
    s->np = keep;
    s->n_pp++;
    orc_sort(s);
}

/* ------------------------------------------------------------------------------------
 * Low-pass digital filtering of J (Sec. 2): `filter_passes` passes of the binomial
 * stencil J_i <- J_{i-1}/4 + J_i/2 + J_{i+1}/4, each pass along x, then y, then z
 * (active axes), on Jx, Jy, Jz; boundaries as for the fields.
 * ---------------------------------------------------------------------------------- */
void orc_filter(orc_sim *s)
{
    double *tmp = (double *)malloc((size_t)s->ncell * sizeof(double));
    for (int pass = 0; pass < s->filter_passes; ++pass) {
        for (int a = 0; a < 3; ++a) {
            if (!s->active[a]) continue;
            for (int comp = ORC_JX; comp <= ORC_JZ; ++comp) {
                memcpy(tmp, s->f[comp], (size_t)s->ncell * sizeof(double));
                orc_sim view = *s;
                view.f[comp] = tmp;
                for (int k = 0; k < s->n[2]; ++k)
                    for (int j = 0; j < s->n[1]; ++j)
                        for (int i = 0; i < s->n[0]; ++i) {
                            int lo[3] = {i, j, k}, hi[3] = {i, j, k};
                            lo[a] -= 1;
                            hi[a] += 1;
                            double v = 0.25 * fget(&view, comp, lo[0], lo[1], lo[2]) +
                                       0.5 * tmp[node_index(s, i, j, k)] +
                                       0.25 * fget(&view, comp, hi[0], hi[1], hi[2]);
                            s->f[comp][node_index(s, i, j, k)] = v;
                        }
            }
        }
    }
    free(tmp);
}

/* ------------------------------------------------------------------------------------
 * Absorbing layer (reading; the paper leaves the open boundary unspecified): on each
 * absorbing axis, cells within `absorb_cells` of either face are multiplied once per step
 * by 1 - strength * (d / L)^2, d = max(0, L - i, i - (n - 1 - L)), L = absorb_cells;
 * factors of several axes multiply.  Applied to E after its update and to B after the
 * second half update.
 * ---------------------------------------------------------------------------------- */
static double damp_factor(const orc_sim *s, const int c[3])
{
    double f = 1.0;
    int L = s->absorb_cells;
    if (L <= 0) return 1.0;
    for (int a = 0; a < 3; ++a) {
        if (!s->active[a] || s->bc[a] != ORC_ABSORBING) continue;
        int d = 0;
        if (L - c[a] > d) d = L - c[a];
        if (c[a] - (s->n[a] - 1 - L) > d) d = c[a] - (s->n[a] - 1 - L);
        double r = (double)d / (double)L;
        f *= 1.0 - s->absorb_strength * r * r;
    }
    return f;
}

/* Central differences on the Yee grid.  Forward difference of an E component (used for
 * curl E at B positions) and backward difference of a B component (curl B at E
 * positions); zero along inactive axes. */
static double dfwd(const orc_sim *s, int comp, int a, int i, int j, int k)
{
    if (!s->active[a]) return 0.0;
    int p[3] = {i, j, k};
    p[a] += 1;
    return (fget(s, comp, p[0], p[1], p[2]) - fget(s, comp, i, j, k)) / s->dx[a];
}

static double dbwd(const orc_sim *s, int comp, int a, int i, int j, int k)
{
    if (!s->active[a]) return 0.0;
    int p[3] = {i, j, k};
    p[a] -= 1;
    return (fget(s, comp, i, j, k) - fget(s, comp, p[0], p[1], p[2])) / s->dx[a];
}

/* ------------------------------------------------------------------------------------
 * Low-dispersion solver (Sec. 2 names low-dispersion electromagnetic solvers as one cure
 * of the boosted-frame instability, citing Karkkainen et al., ICAP 2006; reading): in the
 * Faraday update every forward difference along axis a is averaged over the two other
 * axes, weight 7/12 on the difference itself, 1/12 on each of its four edge neighbours
 * and 1/48 on each of its four corner neighbours (an invariant axis folds its neighbours
 * onto the centre: 3/4 and 1/8 in 2D3V).  In Fourier space the difference along a is
 * multiplied by
 *   S_a = 7/12 + (1/6) (cos th_b + cos th_c) + (1/12) cos th_b cos th_c,  th = k dx,
 * which lies in [1/3, 1] (no mode loses its Faraday coupling), so for fields with
 * discrete div E = 0 the dispersion relation is
 *   sin^2(w dt / 2) / dt^2 = sum_a S_a sin^2(k_a dx_a / 2) / dx_a^2:
 * a wave along the axis of the smallest cell travels without dispersion at dt equal to
 * that cell, and the scheme is stable up to dt = min_a dx_a (the Yee limit is
 * 1 / sqrt(sum_a 1 / dx_a^2)).  Ampere's law keeps the Yee differences.
 * ---------------------------------------------------------------------------------- */
static double dfwd_ck(const orc_sim *s, int comp, int a, int i, int j, int k)
{
    if (!s->active[a]) return 0.0;
    int b = (a + 1) % 3, c = (a + 2) % 3;
    double sum = 0.0;
    for (int db = -1; db <= 1; ++db)
        for (int dc = -1; dc <= 1; ++dc) {
            int p[3] = {i, j, k};
            p[b] += db; /* on an invariant axis this is the same cell */
            p[c] += dc;
            int edges = (db != 0) + (dc != 0);
            double w = edges == 0 ? 7.0 / 12.0 : (edges == 1 ? 1.0 / 12.0 : 1.0 / 48.0);
            sum += w * dfwd(s, comp, a, p[0], p[1], p[2]);
        }
    return sum;
}

void orc_set_solver(orc_sim *s, int solver) { s->solver = solver; }

/* ------------------------------------------------------------------------------------
 * Laser antenna on a plane fixed in the laboratory (Sec. 2: the laser enters through a
 * plane fixed in the lab frame that drifts in the boosted frame; reading).  The lab pulse
 * of the loader's parameters (a0, lambda0, waist, duration, z_center = where its
 * envelope centre would be at lab time 0 had it always propagated freely) is emitted
 * forward by the lab plane z = z_lab: downstream of the plane the field is the free
 * pulse, upstream there is none.  In this frame the plane sits at
 * z'_p(t') = z_lab / gamma_b - beta_b t', and the free pulse is
 *   E'_x = B'_y = T(x, y) g(z' - t'),  g(u) = a0 k' exp(-((u - z'_c) / L')^2) cos(k' (u - z'_c)),
 *   T = exp(-(x^2 + y^2) / w0^2)
 * (k', L', z'_c Doppler-scaled by gamma_b (1 + beta_b), as for the loaded laser).
 * Discretely the grid is split into a total-field region (z positions above
 * z'_p(t^n) / dz, t^n the time of the fields, held fixed through the Maxwell phase that
 * advances them) and a scattered-field region (at or below it), which holds the field
 * minus the incident pulse.  The incident field is T times g propagated on a 1D lattice aligned
 * with the grid's z lattice by the same leapfrog (so a plane wave crosses the boundary
 * without any reflection), started from samples of g.  Every difference stencil reads
 * its neighbours in its own node's representation: a node in the total-field region adds
 * the incident value of neighbours in the scattered-field region, and the other way
 * round it is subtracted -- the update's own curl evaluated on the incident pulse of the
 * other region.  Under the Yee scheme that is h T g_E / dz added to B_y in each B half
 * update and dt T g_B / dz to E_x in the E update; the low-dispersion solver's averaged
 * differences also reach across the plane from the B_z nodes (through dE_x/dy on the
 * neighbouring z rows) and spread the B_y term over the neighbouring columns.  At the end of each Maxwell phase the values the receding plane has passed
 * (between its positions at t^n and t^{n+1}) enter the total-field region: their incident
 * value at t^{n+1} is added.  Setting the antenna adds the incident field to the
 * total-field region.
 * ---------------------------------------------------------------------------------- */
static double ant_profile(const orc_sim *s, double x, double y)
{
    double dx = x - s->ant_xc, dy = s->active[1] ? y - s->ant_yc : 0.0;
    return exp(-(dx * dx + dy * dy) / (s->ant_w0 * s->ant_w0));
}

/* the plane's position in cells along z at the start of the antenna's Maxwell phase n */
static double ant_plane(const orc_sim *s, int64_t n)
{
    return (s->ant_zb - s->ant_beta * (s->ant_t0 + (double)n * s->dt)) / s->dx[2];
}

/* incident E_x at node k, B_y at half node k + 1/2 (0 outside the lattice) */
static double ant_ge(const orc_sim *s, int64_t k)
{
    int64_t a = k - s->ant_lo;
    return a >= 0 && a < s->ant_na ? s->ant_e[a] : 0.0;
}

static double ant_gb(const orc_sim *s, int64_t k)
{
    int64_t a = k - s->ant_lo;
    return a >= 0 && a < s->ant_na ? s->ant_b[a] : 0.0;
}

/* the 1D leapfrog of the incident pulse (E_x on nodes, B_y on half nodes, zero beyond
 * the lattice): B_y -= h dE_x/dz (h = dt / 2) or E_x -= dt dB_y/dz */
static void ant_aux_b(orc_sim *s, double h)
{
    for (int64_t a = 0; a < s->ant_na; ++a) {
        double e1 = a + 1 < s->ant_na ? s->ant_e[a + 1] : 0.0;
        s->ant_b[a] -= h * (e1 - s->ant_e[a]) / s->dx[2];
    }
}

static void ant_aux_e(orc_sim *s)
{
    for (int64_t a = s->ant_na - 1; a >= 0; --a) {
        double b0 = a > 0 ? s->ant_b[a - 1] : 0.0;
        s->ant_e[a] -= s->dt * (s->ant_b[a] - b0) / s->dx[2];
    }
}

/* adds the incident field at E_x nodes k and B_y half nodes k + 1/2 whose z position lies
 * in (lo, hi] (in cells) */
static void ant_add_incident(orc_sim *s, double lo, double hi)
{
    for (int k = 0; k < s->n[2]; ++k)
        for (int j = 0; j < s->n[1]; ++j)
            for (int i = 0; i < s->n[0]; ++i) {
                int64_t id = node_index(s, i, j, k);
                double T = ant_profile(s, (i + 0.5) * s->dx[0], j * s->dx[1]); /* E_x and B_y share x, y */
                if (k > lo && k <= hi) s->f[ORC_EX][id] += T * ant_ge(s, k);
                if (k + 0.5 > lo && k + 0.5 <= hi) s->f[ORC_BY][id] += T * ant_gb(s, k);
            }
}

void orc_set_antenna(orc_sim *s, int enable, double gb, const double *laser, double z_lab)
{
    free(s->ant_e);
    free(s->ant_b);
    s->ant_e = s->ant_b = NULL;
    s->ant = 0;
    if (!enable || !laser) return;
    double b = boost_beta(gb), doppler = gb * (1.0 + b);
    double kp = 6.283185307179586 / (laser[1] * doppler), Lp = laser[3] * doppler, zc = laser[4] * doppler;
    double amp = laser[0] * kp, dz = s->dx[2];
    s->ant = 1;
    s->ant_zb = z_lab / gb;
    s->ant_beta = b;
    s->ant_t0 = (double)s->n_mx * s->dt;
    s->ant_n = 0;
    s->ant_w0 = laser[2];
    s->ant_xc = 0.5 * s->n[0] * s->dx[0];
    s->ant_yc = 0.5 * s->n[1] * s->dx[1];
    /* lattice: from below the pulse's tail (5 L') and the grid, to beyond the grid by the
     * distance light covers while the plane is still in the box (no echo of the lattice's
     * end reaches the box meanwhile) */
    double zp0 = ant_plane(s, 0), t0 = s->ant_t0;
    double lo = floor((zc + t0 - 5.0 * Lp) / dz) - 2.0;
    if (lo > 0.0) lo = 0.0;
    double top = (double)s->n[2] > ceil(zp0) + 2.0 ? (double)s->n[2] : ceil(zp0) + 2.0;
    double stay = zp0 > -1.0 && b > 0.0 ? (zp0 + 1.0) / b : 0.0; /* in cells of time */
    double hi = top + ceil(stay) + 8.0;
    s->ant_lo = (int64_t)lo;
    s->ant_na = (int64_t)(hi - lo) + 1;
    s->ant_e = (double *)calloc((size_t)s->ant_na, sizeof(double));
    s->ant_b = (double *)calloc((size_t)s->ant_na, sizeof(double));
    for (int64_t a = 0; a < s->ant_na; ++a) {
        double ue = (s->ant_lo + a) * dz - t0 - zc, ub = (s->ant_lo + a + 0.5) * dz - t0 - zc;
        s->ant_e[a] = amp * exp(-(ue / Lp) * (ue / Lp)) * cos(kp * ue);
        s->ant_b[a] = amp * exp(-(ub / Lp) * (ub / Lp)) * cos(kp * ub);
    }
    ant_add_incident(s, zp0, INFINITY);
}

/* Two shallow copies of s whose fields are the incident pulse on one side of the plane
 * at zp (cells) and zero elsewhere: v[1] holds it where the node lies above the plane,
 * v[0] where it lies at or below it.  Only E_x (nodes k) and B_y (half nodes k + 1/2)
 * of the incident pulse are nonzero.  The solver's own difference functions read them
 * like the real fields.  Release with ant_views_free. */
static void ant_views(const orc_sim *s, double zp, orc_sim v[2])
{
    size_t nc = (size_t)s->ncell;
    double *zero = (double *)calloc(nc, sizeof(double));
    for (int side = 0; side < 2; ++side) {
        v[side] = *s;
        for (int c = 0; c < ORC_NCOMP; ++c) v[side].f[c] = zero;
        v[side].f[ORC_EX] = (double *)calloc(nc, sizeof(double));
        v[side].f[ORC_BY] = (double *)calloc(nc, sizeof(double));
    }
    for (int k = 0; k < s->n[2]; ++k)
        for (int j = 0; j < s->n[1]; ++j)
            for (int i = 0; i < s->n[0]; ++i) {
                int64_t id = node_index(s, i, j, k);
                double T = ant_profile(s, (i + 0.5) * s->dx[0], j * s->dx[1]); /* E_x and B_y share x, y */
                v[k + STAG[ORC_EX][2] > zp].f[ORC_EX][id] = T * ant_ge(s, k);
                v[k + STAG[ORC_BY][2] > zp].f[ORC_BY][id] = T * ant_gb(s, k);
            }
}

static void ant_views_free(orc_sim v[2])
{
    free(v[0].f[ORC_EY]); /* the shared zero array */
    for (int side = 0; side < 2; ++side) {
        free(v[side].f[ORC_EX]);
        free(v[side].f[ORC_BY]);
    }
}

/* The incident part of the curl a node of component comp (height k + its z staggering,
 * in cells) must add so that its difference stencil reads every neighbour in the node's
 * own representation: a node above the plane (total field) adds the incident pulse of
 * the neighbours at or below it, a node at or below (scattered field) subtracts that of
 * the neighbours above.  curl is the update's own curl component evaluated on a view
 * (which holds the incident pulse of one side only). */
static double ant_term(const orc_sim v[2], int comp, int k, double zp,
                       double (*curl)(const orc_sim *, int, int, int), int i, int j)
{
    int above = k + STAG[comp][2] > zp;
    double c = curl(&v[!above], i, j, k);
    return above ? c : -c;
}

/* The components of curl E at the B nodes (forward differences, averaged under the
 * low-dispersion solver) and of curl B at the E nodes (backward differences). */
typedef double (*diff_fn)(const orc_sim *, int, int, int, int, int);
static diff_fn faraday_diff(const orc_sim *s) { return s->solver == ORC_SOLVER_CK ? dfwd_ck : dfwd; }
static double curl_e_x(const orc_sim *s, int i, int j, int k)
{
    diff_fn d = faraday_diff(s);
    return d(s, ORC_EZ, 1, i, j, k) - d(s, ORC_EY, 2, i, j, k);
}
static double curl_e_y(const orc_sim *s, int i, int j, int k)
{
    diff_fn d = faraday_diff(s);
    return d(s, ORC_EX, 2, i, j, k) - d(s, ORC_EZ, 0, i, j, k);
}
static double curl_e_z(const orc_sim *s, int i, int j, int k)
{
    diff_fn d = faraday_diff(s);
    return d(s, ORC_EY, 0, i, j, k) - d(s, ORC_EX, 1, i, j, k);
}
static double curl_b_x(const orc_sim *s, int i, int j, int k)
{
    return dbwd(s, ORC_BZ, 1, i, j, k) - dbwd(s, ORC_BY, 2, i, j, k);
}
static double curl_b_y(const orc_sim *s, int i, int j, int k)
{
    return dbwd(s, ORC_BX, 2, i, j, k) - dbwd(s, ORC_BZ, 0, i, j, k);
}
static double curl_b_z(const orc_sim *s, int i, int j, int k)
{
    return dbwd(s, ORC_BY, 0, i, j, k) - dbwd(s, ORC_BX, 1, i, j, k);
}

/* nodes whose stencils can reach across the plane at zp (one cell each way, plus the
 * staggering) */
static int near_plane(int k, double zp) { return k >= zp - 3.0 && k <= zp + 3.0; }

/* B <- B - h curl E (h = dt / 2), optionally damped afterwards. */
static void half_b(orc_sim *s, int damp)
{
    int64_t nc = s->ncell;
    double *nb[3];
    for (int c = 0; c < 3; ++c) nb[c] = (double *)malloc((size_t)nc * sizeof(double));
    double h = 0.5 * s->dt;
    orc_sim av[2];
    double zp = 0.0;
    if (s->ant) {
        zp = ant_plane(s, s->ant_n);
        ant_views(s, zp, av);
    }
    for (int k = 0; k < s->n[2]; ++k)
        for (int j = 0; j < s->n[1]; ++j)
            for (int i = 0; i < s->n[0]; ++i) {
                int64_t id = node_index(s, i, j, k);
                double cx = curl_e_x(s, i, j, k);
                double cy = curl_e_y(s, i, j, k);
                double cz = curl_e_z(s, i, j, k);
                if (s->ant && near_plane(k, zp)) {
                    cx += ant_term(av, ORC_BX, k, zp, curl_e_x, i, j);
                    cy += ant_term(av, ORC_BY, k, zp, curl_e_y, i, j);
                    cz += ant_term(av, ORC_BZ, k, zp, curl_e_z, i, j);
                }
                int c[3] = {i, j, k};
                double f = damp ? damp_factor(s, c) : 1.0;
                nb[0][id] = f * (s->f[ORC_BX][id] - h * cx);
                nb[1][id] = f * (s->f[ORC_BY][id] - h * cy);
                nb[2][id] = f * (s->f[ORC_BZ][id] - h * cz);
            }
    if (s->ant) ant_views_free(av);
    for (int c = 0; c < 3; ++c) {
        memcpy(s->f[ORC_BX + c], nb[c], (size_t)nc * sizeof(double));
        free(nb[c]);
    }
}

/* E <- damp * (E + dt (curl B - J)). */
static void full_e(orc_sim *s)
{
    int64_t nc = s->ncell;
    double *ne[3];
    for (int c = 0; c < 3; ++c) ne[c] = (double *)malloc((size_t)nc * sizeof(double));
    double dt = s->dt;
    orc_sim av[2];
    double zp = 0.0;
    if (s->ant) {
        zp = ant_plane(s, s->ant_n);
        ant_views(s, zp, av);
    }
    for (int k = 0; k < s->n[2]; ++k)
        for (int j = 0; j < s->n[1]; ++j)
            for (int i = 0; i < s->n[0]; ++i) {
                int64_t id = node_index(s, i, j, k);
                double cx = curl_b_x(s, i, j, k);
                double cy = curl_b_y(s, i, j, k);
                double cz = curl_b_z(s, i, j, k);
                if (s->ant && near_plane(k, zp)) {
                    cx += ant_term(av, ORC_EX, k, zp, curl_b_x, i, j);
                    cy += ant_term(av, ORC_EY, k, zp, curl_b_y, i, j);
                    cz += ant_term(av, ORC_EZ, k, zp, curl_b_z, i, j);
                }
                int c[3] = {i, j, k};
                double f = damp_factor(s, c);
                ne[0][id] = f * (s->f[ORC_EX][id] + dt * (cx - s->f[ORC_JX][id]));
                ne[1][id] = f * (s->f[ORC_EY][id] + dt * (cy - s->f[ORC_JY][id]));
                ne[2][id] = f * (s->f[ORC_EZ][id] + dt * (cz - s->f[ORC_JZ][id]));
            }
    if (s->ant) ant_views_free(av);
    for (int c = 0; c < 3; ++c) {
        memcpy(s->f[ORC_EX + c], ne[c], (size_t)nc * sizeof(double));
        free(ne[c]);
    }
}

/* ------------------------------------------------------------------------------------
 * Yee FDTD leapfrog: B^{n+1/2} = B^n - (dt/2) curl E^n;
 * E^{n+1} = E^n + dt (curl B^{n+1/2} - J^{n+1/2});  B^{n+1} = B^{n+1/2} - (dt/2) curl E^{n+1}.
 * ---------------------------------------------------------------------------------- */
void orc_maxwell(orc_sim *s)
{
    half_b(s, 0);
    if (s->ant) ant_aux_b(s, 0.5 * s->dt);
    full_e(s);
    if (s->ant) ant_aux_e(s);
    half_b(s, 1);
    if (s->ant) {
        ant_aux_b(s, 0.5 * s->dt);
        s->ant_n++; /* the values the receding plane passed during the phase join the total field */
        ant_add_incident(s, ant_plane(s, s->ant_n), ant_plane(s, s->ant_n - 1));
    }
    s->n_mx++;
}

void orc_step(orc_sim *s, int nsteps)
{
    for (int n = 0; n < nsteps; ++n) {
        orc_particle_phase(s);
        orc_filter(s);
        orc_maxwell(s);
        s->step++;
    }
}

/* ------------------------------------------------------------------------------------
 * Charge density on nodes: rho_ijk = sum_p (q w_p / dV) S(x_p - i) S(y_p - j) S(z_p - k).
 * ---------------------------------------------------------------------------------- */
static void deposit_rho(const orc_sim *s, int64_t p0, int64_t p1, double *out)
{
    double dV = s->dx[0] * s->dx[1] * s->dx[2];
    for (int64_t p = p0; p < p1; ++p) {
        int c[3], lo[3], cnt[3];
        cell_coords(s, s->cell[p], c);
        const double *o = &s->off[3 * p];
        for (int a = 0; a < 3; ++a) window(s, a, c[a], &lo[a], &cnt[a]);
        for (int kk = 0; kk < cnt[2]; ++kk)
            for (int jj = 0; jj < cnt[1]; ++jj)
                for (int ii = 0; ii < cnt[0]; ++ii) {
                    int i = lo[0] + ii, j = lo[1] + jj, k = lo[2] + kk;
                    double wt = node_weight(s, 0, c[0], o[0], i, 0.0) * node_weight(s, 1, c[1], o[1], j, 0.0) *
                                node_weight(s, 2, c[2], o[2], k, 0.0);
                    if (wt == 0.0) continue;
                    int64_t idx = node_index(s, i, j, k);
                    if (idx >= 0) out[idx] += s->q * s->w[p] / dV * wt;
                }
    }
}

void orc_rho(const orc_sim *s, double *out)
{
    memset(out, 0, (size_t)s->ncell * sizeof(double));
    deposit_rho(s, 0, s->np, out);
    if (s->ion && s->active[2]) { /* plus the ion background on its dual cells */
        double t = (double)s->n_pp * s->dt, dz = s->dx[2];
        for (int k = 0; k < s->n[2]; ++k) {
            double r = orc_ion_integral(s, (k - 0.5) * dz + s->ion_beta * t, (k + 0.5) * dz + s->ion_beta * t) / dz;
            for (int j = 0; j < s->n[1]; ++j)
                for (int i = 0; i < s->n[0]; ++i) out[node_index(s, i, j, k)] += r;
        }
    }
}

/* Discrete divergence of E on nodes: sum_a (E_a[i] - E_a[i - e_a]) / dx_a. */
void orc_div_e(const orc_sim *s, double *out)
{
    for (int k = 0; k < s->n[2]; ++k)
        for (int j = 0; j < s->n[1]; ++j)
            for (int i = 0; i < s->n[0]; ++i)
                out[node_index(s, i, j, k)] = dbwd(s, ORC_EX, 0, i, j, k) + dbwd(s, ORC_EY, 1, i, j, k) +
                                              dbwd(s, ORC_EZ, 2, i, j, k);
}

/* ------------------------------------------------------------------------------------
 * Lab-frame station (Sec. 2, reading): a plane z = z_lab immobile in the laboratory
 * frame.  Lab and boosted frames share their origin (z = z' = 0 at t = t' = 0) and the
 * boost is along +z, so at boosted time t' the plane sits at z' = z_lab / g - b t' and the
 * lab time there is t = t' / g + b z_lab.  The station samples every field component at
 * its own transverse Yee position, interpolating linearly in z' between the two grid
 * planes of that component's z stagger around z' (zero beyond an absorbing face, wrapped
 * on a periodic axis), and transforms the sample back to the lab frame (a boost by -b):
 *   E_x = g (E'_x + b B'_y),  E_y = g (E'_y - b B'_x),  E_z = E'_z,
 *   B_x = g (B'_x - b E'_y),  B_y = g (B'_y + b E'_x),  B_z = B'_z.
 * t' is s->step dt: E and B after `step` full steps.  Returns 1 and fills out[6][n1][n0]
 * and *t_lab when z' lies in [0, n2 dz), else 0.
 * ---------------------------------------------------------------------------------- */
int orc_station_record(const orc_sim *s, double gb, double z_lab, double *out, double *t_lab)
{
    double b = boost_beta(gb);
    double tp = (double)s->step * s->dt;
    double zp = z_lab / gb - b * tp;
    double Lz = s->n[2] * s->dx[2];
    if (!(zp >= 0.0 && zp < Lz)) return 0;
    int64_t plane = (int64_t)s->n[0] * s->n[1];
    for (int j = 0; j < s->n[1]; ++j)
        for (int i = 0; i < s->n[0]; ++i) {
            double f[6];
            for (int c = ORC_EX; c <= ORC_BZ; ++c) {
                /* z' in units of the component's own grid planes */
                double q = zp / s->dx[2] - STAG[c][2];
                double k = floor(q);
                double fr = q - k;
                f[c] = (1.0 - fr) * fget(s, c, i, j, (int)k) + fr * fget(s, c, i, j, (int)k + 1);
            }
            double g = gb;
            double lab[6] = {g * (f[ORC_EX] + b * f[ORC_BY]), g * (f[ORC_EY] - b * f[ORC_BX]), f[ORC_EZ],
                             g * (f[ORC_BX] - b * f[ORC_EY]), g * (f[ORC_BY] + b * f[ORC_EX]), f[ORC_BZ]};
            for (int c = 0; c < 6; ++c) out[(int64_t)c * plane + (int64_t)j * s->n[0] + i] = lab[c];
        }
    *t_lab = tp / gb + b * z_lab;
    return 1;
}

/* Test helper: rounds the stored state (offsets, momenta, weights, E, B) to FP32, as an
 * FP32 implementation stores it between steps; offsets that round to 1 keep the largest
 * float below 1 (same cell).  Calling it after every step gives the error floor that FP32
 * storage alone imposes, with FP64 arithmetic everywhere else. */
void orc_round_state_fp32(orc_sim *s)
{
    const double below_one = (double)nextafterf(1.0f, 0.0f);
    for (int64_t p = 0; p < s->np; ++p) {
        for (int a = 0; a < 3; ++a) {
            double o = (double)(float)s->off[3 * p + a];
            s->off[3 * p + a] = o >= 1.0 ? below_one : o;
            s->u[3 * p + a] = (double)(float)s->u[3 * p + a];
        }
        s->w[p] = (double)(float)s->w[p];
    }
    for (int c = ORC_EX; c <= ORC_BZ; ++c)
        for (int64_t i = 0; i < s->ncell; ++i) s->f[c][i] = (double)(float)s->f[c][i];
}

/* out: field energy (1/2) sum (E^2 + B^2) dV, kinetic energy sum w m (gamma - 1),
 * total charge sum q w, particle count, lost count, step, 0, 0. */
void orc_diagnostics(const orc_sim *s, double out[8])
{
    double dV = s->dx[0] * s->dx[1] * s->dx[2];
    double fe = 0.0;
    for (int c = ORC_EX; c <= ORC_BZ; ++c)
        for (int64_t i = 0; i < s->ncell; ++i) fe += s->f[c][i] * s->f[c][i];
    double ke = 0.0, qt = 0.0;
    for (int64_t p = 0; p < s->np; ++p) {
        const double *u = &s->u[3 * p];
        double g = sqrt(1.0 + u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
        ke += s->w[p] * s->m * (g - 1.0);
        qt += s->q * s->w[p];
    }
    out[0] = 0.5 * fe * dV;
    out[1] = ke;
    out[2] = qt;
    out[3] = (double)s->np;
    out[4] = (double)s->n_lost;
    out[5] = (double)s->step;
    out[6] = 0.0;
    out[7] = 0.0;
}

/* ------------------------------------------------------------------------------------
 * Lab-frame inputs -> boosted frame (Sec. 2).  Box: x in [0, n0 dx), y in [0, n1 dy),
 * z' in [0, n2 dz) at boosted time t' = 0; lab z = 0 coincides with z' = 0 at t = t' = 0.
 *
 * laser[5]  = {a0, lambda0, waist, duration, z_center}: linearly polarised along x,
 *   propagating +z, Gaussian in r and in (z - z_center) (field 1/e lengths waist and
 *   duration), centred transversely in the box.  Boosted: lambda' = g(1+b) lambda0,
 *   length' = g(1+b) duration, centroid z'_c = g(1+b) z_center, a0 and waist invariant,
 *   E'x = B'y = a0 k' exp(-r^2/w0^2) exp(-((z'-z'_c)/L')^2) cos(k'(z'-z'_c)), k' = 2 pi / lambda'.
 * plasma[8] = {n0, z_start, ramp_len, ppc, uth_x, uth_y, uth_z, seed}: lab density n0 for
 *   z >= z_start + ramp_len, linear ramp from z_start, zero before.  For every cell
 *   (linear order) and every p < ppc: offsets from streams 0..2 at counter cell*ppc + p,
 *   lab momentum u = uth * N(0,1) from stream pairs (3,4), (5,6), (7,8), boosted;
 *   weight w = n(g z') g dV / ppc (density g n0 in the boosted frame); w = 0 -> skipped.
 * beam[8]   = {n, gamma, rel_spread, sigma_r, sigma_z, z0, total_weight, seed}: lab event at
 *   t = 0: x = xc + sigma_r N(10,11), y = yc + sigma_r N(12,13), z = z0 + sigma_z N(14,15),
 *   u = (0,0,gamma beta) + rel_spread * gamma beta * (N(16,17), N(18,19), N(20,21)),
 *   w = total_weight / n; boosted, then drifted ballistically to t' = 0; particles
 *   outside the box are dropped.  The beam's self-field (orc_beam_self_field) is added
 *   to the fields, for its centroid velocity in this frame.
 * Returns the number of particles loaded.
 * ---------------------------------------------------------------------------------- */
/* ------------------------------------------------------------------------------------
 * Self-field of a beam moving rigidly at beta along z (the field the beam carries when
 * it enters, so that the field it applies to itself is the one Sec. 2 discusses: a
 * radial E almost cancelled by the azimuthal B).  For a charge density rho moving
 * rigidly at v = beta z, the Lorenz-gauge potentials are phi and A = beta phi z, with
 *   d2phi/dx2 + d2phi/dy2 + (1/gamma^2) d2phi/dz2 = -rho,
 *   E = (-dphi/dx, -dphi/dy, -(1/gamma^2) dphi/dz),   B = curl A = beta z x E.
 * Discretely: rho on the nodes (the particles' shape, as orc_rho), the 3- / 5- / 7-point
 * second differences on the nodes (phi = 0 one node beyond an absorbing face, wrap on a
 * periodic axis), E as the Yee differences of phi, and B_x = -beta E_y, B_y = beta E_x
 * with E averaged over the two z nodes around B's half-integer z.  The linear system is
 * solved exactly by expanding in the eigenvectors of each axis's second difference
 * (sines for Dirichlet, real Fourier modes for periodic); on an all-periodic grid the
 * mean of rho is dropped (a neutralising background).
 * ---------------------------------------------------------------------------------- */
static void axis_modes(int n, int periodic, double dx, double *Q, double *lam)
{
    /* Q[m * n + i]: orthonormal eigenvector m of the second difference (1/dx^2) */
    const double pi = 3.141592653589793;
    for (int m = 0; m < n; ++m) {
        double theta;
        if (!periodic) {
            theta = pi * (m + 1) / (n + 1);
            for (int i = 0; i < n; ++i) Q[m * n + i] = sqrt(2.0 / (n + 1)) * sin(theta * (i + 1));
        } else {
            int k = (m + 1) / 2; /* m = 0: constant; then cos, sin pairs */
            theta = 2.0 * pi * k / n;
            for (int i = 0; i < n; ++i) {
                if (m == 0)
                    Q[m * n + i] = 1.0 / sqrt((double)n);
                else if (2 * k == n)
                    Q[m * n + i] = (i % 2 ? -1.0 : 1.0) / sqrt((double)n);
                else if (m % 2 == 1)
                    Q[m * n + i] = sqrt(2.0 / n) * cos(theta * i);
                else
                    Q[m * n + i] = sqrt(2.0 / n) * sin(theta * i);
            }
        }
        lam[m] = -(2.0 - 2.0 * cos(theta)) / (dx * dx);
    }
}

/* v <- Q v (forward, coefficients) or Q^T v (back) along axis a of an n0 x n1 x n2 array */
static void apply_modes(const orc_sim *s, int a, const double *Q, int forward, double *v)
{
    int n = s->n[a];
    double *line = (double *)malloc((size_t)n * sizeof(double));
    double *res = (double *)malloc((size_t)n * sizeof(double));
    int64_t stride = a == 0 ? 1 : (a == 1 ? s->n[0] : (int64_t)s->n[0] * s->n[1]);
    for (int64_t base = 0; base < s->ncell; ++base) {
        int c[3];
        cell_coords(s, (int32_t)base, c);
        if (c[a] != 0) continue; /* one line per start node */
        for (int i = 0; i < n; ++i) line[i] = v[base + i * stride];
        for (int m = 0; m < n; ++m) {
            double acc = 0.0;
            for (int i = 0; i < n; ++i) acc += (forward ? Q[m * n + i] * line[i] : Q[i * n + m] * line[i]);
            res[m] = acc;
        }
        for (int i = 0; i < n; ++i) v[base + i * stride] = res[i];
    }
    free(line);
    free(res);
}

int orc_beam_self_field(orc_sim *s, const double *rho, double gamma, double beta)
{
    double *phi = (double *)malloc((size_t)s->ncell * sizeof(double));
    double *Q[3] = {NULL, NULL, NULL}, *lam[3] = {NULL, NULL, NULL};
    int all_periodic = 1;
    memcpy(phi, rho, (size_t)s->ncell * sizeof(double));
    for (int a = 0; a < 3; ++a) {
        if (!s->active[a]) continue;
        if (s->bc[a] == ORC_ABSORBING) all_periodic = 0;
        Q[a] = (double *)malloc((size_t)s->n[a] * s->n[a] * sizeof(double));
        lam[a] = (double *)malloc((size_t)s->n[a] * sizeof(double));
        axis_modes(s->n[a], s->bc[a] == ORC_PERIODIC, s->dx[a], Q[a], lam[a]);
        apply_modes(s, a, Q[a], 1, phi);
    }
    for (int64_t idx = 0; idx < s->ncell; ++idx) {
        int c[3];
        cell_coords(s, (int32_t)idx, c);
        double L = 0.0;
        for (int a = 0; a < 3; ++a)
            if (s->active[a]) L += (a == 2 ? 1.0 / (gamma * gamma) : 1.0) * lam[a][c[a]];
        /* the (0,0,0) mode of an all-periodic grid has L = 0: dropped */
        phi[idx] = (all_periodic && c[0] == 0 && c[1] == 0 && c[2] == 0) ? 0.0 : -phi[idx] / L;
    }
    for (int a = 0; a < 3; ++a)
        if (s->active[a]) apply_modes(s, a, Q[a], 0, phi);
    /* fields from phi (added to what is there, e.g. a laser) */
    for (int k = 0; k < s->n[2]; ++k)
        for (int j = 0; j < s->n[1]; ++j)
            for (int i = 0; i < s->n[0]; ++i) {
                int64_t id = node_index(s, i, j, k);
                double p0 = phi[id];
                double px = node_index(s, i + 1, j, k) < 0 ? 0.0 : phi[node_index(s, i + 1, j, k)];
                double py = node_index(s, i, j + 1, k) < 0 ? 0.0 : phi[node_index(s, i, j + 1, k)];
                double pz = node_index(s, i, j, k + 1) < 0 ? 0.0 : phi[node_index(s, i, j, k + 1)];
                s->f[ORC_EX][id] += -(px - p0) / s->dx[0];
                if (s->active[1]) s->f[ORC_EY][id] += -(py - p0) / s->dx[1];
                s->f[ORC_EZ][id] += -(pz - p0) / (s->dx[2] * gamma * gamma);
            }
    /* B from the beam's E alone, averaged over the two z nodes around k + 1/2 */
    for (int k = 0; k < s->n[2]; ++k)
        for (int j = 0; j < s->n[1]; ++j)
            for (int i = 0; i < s->n[0]; ++i) {
                int64_t id = node_index(s, i, j, k);
                double ex[2], ey[2];
                for (int h = 0; h < 2; ++h) {
                    int64_t c0 = node_index(s, i, j, k + h);
                    int64_t cx = node_index(s, i + 1, j, k + h), cy = node_index(s, i, j + 1, k + h);
                    double p0 = c0 < 0 ? 0.0 : phi[c0];
                    ex[h] = c0 < 0 ? 0.0 : -((cx < 0 ? 0.0 : phi[cx]) - p0) / s->dx[0];
                    ey[h] = (c0 < 0 || !s->active[1]) ? 0.0 : -((cy < 0 ? 0.0 : phi[cy]) - p0) / s->dx[1];
                }
                s->f[ORC_BX][id] += -beta * 0.5 * (ey[0] + ey[1]);
                s->f[ORC_BY][id] += beta * 0.5 * (ex[0] + ex[1]);
            }
    for (int a = 0; a < 3; ++a) {
        free(Q[a]);
        free(lam[a]);
    }
    free(phi);
    return 0;
}

static void append_particle(orc_sim *s, const double pos[3], const double u[3], double w, int32_t id)
{
    int c[3];
    double o[3];
    for (int a = 0; a < 3; ++a) {
        if (!s->active[a]) {
            c[a] = 0;
            o[a] = 0.0;
            continue;
        }
        double x = pos[a] / s->dx[a];
        double k = floor(x);
        c[a] = (int)k;
        o[a] = x - k;
        if (o[a] >= 1.0) {
            o[a] = 0.0;
            c[a] += 1;
        }
        if (c[a] < 0 || c[a] >= s->n[a]) return;
    }
    if (s->np == s->cap) reserve(s, s->cap ? 2 * s->cap : 1024);
    int64_t p = s->np++;
    s->cell[p] = (int32_t)(c[0] + s->n[0] * (c[1] + s->n[1] * c[2]));
    s->id[p] = id;
    s->w[p] = w;
    for (int a = 0; a < 3; ++a) {
        s->off[3 * p + a] = o[a];
        s->u[3 * p + a] = u[a];
    }
}

int orc_load_lab_frame(orc_sim *s, double gb, const double *laser, const double *plasma,
                       const double *beam)
{
    double b = boost_beta(gb);
    double doppler = gb * (1.0 + b);
    double L[3] = {s->n[0] * s->dx[0], s->n[1] * s->dx[1], s->n[2] * s->dx[2]};
    double xc = 0.5 * L[0], yc = s->active[1] ? 0.5 * L[1] : 0.0;
    free_particles(s);
    reserve(s, 1024);
    s->n_lost = 0;
    s->step = 0;
    s->n_pp = 0;
    s->n_mx = 0;
    s->ion = 0;
    orc_set_antenna(s, 0, 1.0, NULL, 0.0); /* a load removes the antenna */
    for (int c = 0; c < ORC_NCOMP; ++c) memset(s->f[c], 0, (size_t)s->ncell * sizeof(double));

    if (laser) {
        double a0 = laser[0], lam = laser[1] * doppler, w0 = laser[2], len = laser[3] * doppler;
        double zc = laser[4] * doppler;
        double k = 6.283185307179586 / lam;
        double E0 = a0 * k;
        for (int kk = 0; kk < s->n[2]; ++kk)
            for (int j = 0; j < s->n[1]; ++j)
                for (int i = 0; i < s->n[0]; ++i) {
                    int64_t id = node_index(s, i, j, kk);
                    /* Ex at (i+1/2, j, k), By at (i+1/2, j, k+1/2) */
                    double x = (i + 0.5) * s->dx[0] - xc;
                    double y = s->active[1] ? j * s->dx[1] - yc : 0.0;
                    double tr = exp(-(x * x + y * y) / (w0 * w0));
                    double ze = kk * s->dx[2] - zc, zb = (kk + 0.5) * s->dx[2] - zc;
                    s->f[ORC_EX][id] = E0 * tr * exp(-(ze / len) * (ze / len)) * cos(k * ze);
                    s->f[ORC_BY][id] = E0 * tr * exp(-(zb / len) * (zb / len)) * cos(k * zb);
                }
    }
    int32_t next_id = 0;
    if (plasma) {
        double n0 = plasma[0], zs = plasma[1], ramp = plasma[2];
        int ppc = (int)plasma[3];
        double uth[3] = {plasma[4], plasma[5], plasma[6]};
        uint64_t seed = (uint64_t)plasma[7];
        double dV = s->dx[0] * s->dx[1] * s->dx[2];
        s->ion = n0 > 0.0;
        s->ion_n0 = n0;
        s->ion_zs = zs;
        s->ion_ramp = ramp;
        s->ion_gb = gb;
        s->ion_beta = b;
        for (int64_t cell = 0; cell < s->ncell; ++cell) {
            int c[3];
            cell_coords(s, (int32_t)cell, c);
            for (int p = 0; p < ppc; ++p) {
                uint64_t ctr = (uint64_t)cell * (uint64_t)ppc + (uint64_t)p;
                double pos[3];
                for (int a = 0; a < 3; ++a)
                    pos[a] = s->active[a] ? (c[a] + orc_uniform(seed, (uint64_t)a, ctr)) * s->dx[a] : 0.0;
                double zlab = gb * pos[2];
                double prof = zlab < zs ? 0.0 : (ramp > 0.0 && zlab < zs + ramp ? (zlab - zs) / ramp : 1.0);
                double w = gb * n0 * prof * dV / ppc;
                if (w == 0.0) continue;
                double ul[3], tx[4] = {0.0, pos[0], pos[1], zlab}, txp[4], up[3];
                for (int a = 0; a < 3; ++a) ul[a] = uth[a] * orc_normal(seed, 3 + 2 * (uint64_t)a, ctr);
                orc_boost_event(gb, tx, ul, txp, up);
                append_particle(s, pos, up, w, next_id++);
            }
        }
    }
    s->beam_id0 = beam ? next_id : INT32_MAX; /* beam ids follow the plasma's */
    if (beam) {
        int64_t first = s->np;
        int64_t nb = (int64_t)beam[0];
        double gam = beam[1], spread = beam[2], sr = beam[3], sz = beam[4], z0 = beam[5];
        double wb = beam[6] / (double)nb;
        uint64_t seed = (uint64_t)beam[7];
        double gb0 = sqrt(gam * gam - 1.0);
        for (int64_t i = 0; i < nb; ++i) {
            uint64_t ctr = (uint64_t)i;
            double tx[4] = {0.0, xc + sr * orc_normal(seed, 10, ctr), yc + (s->active[1] ? sr * orc_normal(seed, 12, ctr) : 0.0),
                            z0 + sz * orc_normal(seed, 14, ctr)};
            double u[3] = {spread * gb0 * orc_normal(seed, 16, ctr), spread * gb0 * orc_normal(seed, 18, ctr),
                           gb0 + spread * gb0 * orc_normal(seed, 20, ctr)};
            double txp[4], up[3];
            orc_boost_event(gb, tx, u, txp, up);
            double gp = sqrt(1.0 + up[0] * up[0] + up[1] * up[1] + up[2] * up[2]);
            double dtp = -txp[0]; /* drift to t' = 0 */
            double pos[3] = {txp[1] + up[0] / gp * dtp, txp[2] + up[1] / gp * dtp, txp[3] + up[2] / gp * dtp};
            if (!s->active[1]) pos[1] = 0.0;
            append_particle(s, pos, up, wb, next_id++);
        }
        if (s->np > first) {
            /* the beam enters with its self-field, moving at the centroid velocity of this
             * frame: beta' = (beta - b) / (1 - beta b), gamma' = gb gamma (1 - beta b) */
            double bl = gb0 / gam;
            double gp = gb * gam * (1.0 - bl * b), bp = (bl - b) / (1.0 - bl * b);
            double *rho = (double *)calloc((size_t)s->ncell, sizeof(double));
            deposit_rho(s, first, s->np, rho);
            orc_beam_self_field(s, rho, gp, bp);
            free(rho);
        }
    }
    orc_sort(s);
    return (int)s->np;
}
