/*
 * pic_oracle.h -- plain, slow FP64 CPU reference of the explicit electromagnetic
 * particle-in-cell step run in a Lorentz-boosted frame (Vay et al., "Speeding up
 * simulations of relativistic systems using an optimal boosted frame", Sec. 2).
 *
 * TEST INFRASTRUCTURE ONLY.  This library exists to check the CUDA path.  Only the
 * test suite, the smoke check and the benchmark's CPU-baseline leg may load it.  It
 * shares no code, header, table or helper with the CUDA library and includes nothing
 * from it.
 *
 * Units: c = eps0 = 1.  Grid index conventions (staggered Yee grid):
 *   Ex[i,j,k] sits at (i+1/2, j, k), Ey at (i, j+1/2, k), Ez at (i, j, k+1/2),
 *   Bx at (i, j+1/2, k+1/2), By at (i+1/2, j, k+1/2), Bz at (i+1/2, j+1/2, k);
 *   J like E; rho on nodes (i, j, k).  Arrays are n0*n1*n2, x fastest.
 *   In 2D3V (ndim = 2) n2 = 1 and d/dz = 0.
 * Particles: int32 linear cell index (x fastest) + FP64 in-cell offsets in [0,1)
 * per axis, momenta u = gamma*v (per unit mass), weight w (physical particles per
 * macro-particle), int32 id.
 */
#ifndef PIC_ORACLE_H
#define PIC_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_EX, ORC_EY, ORC_EZ, ORC_BX, ORC_BY, ORC_BZ, ORC_JX, ORC_JY, ORC_JZ, ORC_NCOMP };
enum { ORC_PERIODIC = 0, ORC_ABSORBING = 1 };
enum { ORC_VAY = 0, ORC_BORIS = 1 };
enum { ORC_SOLVER_YEE = 0, ORC_SOLVER_CK = 1 };

typedef struct orc_sim orc_sim;

/* --- single-particle and single-point building blocks (for pins) --- */
double orc_shape(int order, double x);
void orc_push_vay(double u[3], const double E[3], const double B[3], double q_over_m, double dt);
void orc_push_boris(double u[3], const double E[3], const double B[3], double q_over_m, double dt);
void orc_boost_fields(double gamma_b, const double E[3], const double B[3], double Ep[3], double Bp[3]);
void orc_boost_event(double gamma_b, const double tx[4], const double u[3], double txp[4], double up[3]);
uint64_t orc_splitmix64(uint64_t seed, uint64_t stream, uint64_t counter);
double orc_uniform(uint64_t seed, uint64_t stream, uint64_t counter);
double orc_normal(uint64_t seed, uint64_t stream, uint64_t counter);

/* --- simulation --- */
orc_sim *orc_create(int ndim, const int n[3], const int bc[3], const double dx[3], double dt,
                    int order, int pusher, int filter_passes, const int tile[3], double q,
                    double m, int absorb_cells, double absorb_strength);
void orc_destroy(orc_sim *s);
void orc_set_field(orc_sim *s, int comp, const double *data);
void orc_get_field(const orc_sim *s, int comp, double *out);
int orc_set_particles(orc_sim *s, int64_t np, const int32_t *cell, const double *off,
                      const double *u, const double *w, const int32_t *id);
int64_t orc_num_particles(const orc_sim *s);
void orc_get_particles(const orc_sim *s, int32_t *cell, double *off, double *u, double *w,
                       int32_t *id);
void orc_sort(orc_sim *s);
void orc_gather(const orc_sim *s, int32_t cell, const double off[3], double E[3], double B[3]);
void orc_particle_phase(orc_sim *s);
void orc_filter(orc_sim *s);
void orc_maxwell(orc_sim *s);
void orc_step(orc_sim *s, int nsteps);
void orc_rho(const orc_sim *s, double *out);
void orc_div_e(const orc_sim *s, double *out);
void orc_diagnostics(const orc_sim *s, double out[8]);
int orc_load_lab_frame(orc_sim *s, double gamma_b, const double *laser, const double *plasma,
                       const double *beam);
/* Charge of the lab-frame plasma's ion background between box coordinates a < b at
 * t' = 0 (per unit transverse area); 0 when the last load had no plasma. */
double orc_ion_integral(const orc_sim *s, double a, double b);
/* Adds the self-field of the node charge density rho[n0 n1 n2] moving rigidly at beta
 * (Lorentz factor gamma) along z: relativistic Poisson solve, E = -grad phi with the z
 * part over gamma^2, B = beta z x E.  Returns 0. */
int orc_beam_self_field(orc_sim *s, const double *rho, double gamma, double beta);
/* Lab-frame station z = z_lab at the current step: fills out[6][n1][n0] (lab-frame Ex Ey
 * Ez Bx By Bz at the plane, each at its transverse Yee position) and *t_lab; returns 1,
 * or 0 when the plane lies outside the box now. */
int orc_station_record(const orc_sim *s, double gamma_b, double z_lab, double *out, double *t_lab);
/* Field solver: ORC_SOLVER_YEE (default) or ORC_SOLVER_CK, the low-dispersion solver
 * (Faraday differences averaged over their transverse neighbours, 7/12, 1/12, 1/48). */
void orc_set_solver(orc_sim *s, int solver);
/* Beam injection through the lab plane z = z_lab (in this frame z' = z_lab / gamma_b -
 * beta_b t'): beam particles (id >= first_id; first_id < 0: the beam of the last
 * lab-frame load) upstream of the plane are frozen (no field acts on them; they drift and
 * deposit).  enable = 0 turns it off.  Kept across loads. */
void orc_set_injection(orc_sim *s, int enable, double gamma_b, double z_lab, int32_t first_id);
/* Particles frozen at the current step (upstream of the injection plane). */
int64_t orc_num_frozen(const orc_sim *s);
/* Laser antenna on the lab plane z = z_lab (in this frame z' = z_lab / gamma_b - beta_b t'):
 * laser[5] as for orc_load_lab_frame; the lab pulse is emitted forward by the plane
 * (total-field / scattered-field split at the plane, incident field propagated on a 1D
 * lattice by the same leapfrog).  Under either field solver: every difference that
 * straddles the plane reads the far value in the near node's representation.  Adds the
 * incident field downstream of the plane now; enable = 0 (or laser NULL) removes it.  A
 * load removes it. */
void orc_set_antenna(orc_sim *s, int enable, double gamma_b, const double *laser, double z_lab);
/* Test helper: rounds offsets (kept below 1), momenta, weights, E and B to FP32. */
void orc_round_state_fp32(orc_sim *s);

#ifdef __cplusplus
}
#endif
#endif
