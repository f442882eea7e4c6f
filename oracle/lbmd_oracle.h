/*
 * lbmd_oracle.h -- API of the FP64 CPU oracle for the coupled
 * lattice-Boltzmann / molecular-dynamics step of Fyta, Sircar, Kaxiras,
 * Melchionna, Bernaschi and Succi, "Parallel multiscale modeling of
 * biopolymer dynamics with hydrodynamic correlations" (Sec. II).
 *
 * TEST INFRASTRUCTURE ONLY.  The oracle exists to check and to time the CUDA
 * path.  Only the test-suite, the smoke check and the CPU-baseline leg of the
 * benchmark may load it; the product path never does.  It shares no code,
 * header, table or helper with the CUDA library.
 *
 * Units are lattice units (dx = dt = 1, bead mass m = 1, charge q = 1).
 * Arrays are flat, x fastest: site s = x + nx*(y + ny*z).  Populations are
 * laid out [19][nsites]; bead vectors [n_beads][3].
 */
#ifndef LBMD_ORACLE_H
#define LBMD_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int nx, ny, nz;
    double tau;               /* BGK relaxation time, omega = 1/tau */
    double body_force[3];     /* uniform force density on every fluid site */
    int wall_x;               /* pore-wall plane (field region, translocation); <0: none */
    int pore_h;               /* side of the square pore */
    int n_beads;
    double k_bond, r0;        /* harmonic bonds */
    double kappa_bend;        /* angular term kappa*phi^2/2 */
    double lj_sigma, lj_eps;  /* bead-bead WCA */
    double wall_sigma, wall_eps; /* bead-solid-node WCA */
    double E;                 /* driving force q*E along +x inside the pore channel */
    double gamma;             /* bead-fluid friction */
    double kT;                /* bead noise temperature (0: off) */
    int md_outer;             /* M: MD steps per LB step */
    int md_inner;             /* M^b: bonded sub-steps per MD step */
    uint64_t seed;            /* Philox key */
    uint32_t realization;     /* realization index, xor-ed into key word 1 */
    int interp;               /* bead-lattice weights: 0 trilinear, 1 nearest grid point (Sec. II) */
    int integrator;           /* 0: multiple-time-step velocity Verlet with explicit friction;
                                 1: stochastic position Verlet (Sec. II, Eq. SPValgo), nested */
    double lb_kT;             /* fluctuating-LB temperature (0: off) */
} orc_params;

typedef struct orc_sim orc_sim;

/* tables and single-site helpers */
void orc_tables(int *c /*19*3*/, double *w /*19*/, int *opp /*19*/);
void orc_feq(double rho, const double *u, double *feq /*19*/);
void orc_source(const double *G, double *S /*19*/);
void orc_philox4x32_10(const uint32_t *ctr, const uint32_t *key, uint32_t *out);
void orc_gauss3(uint64_t seed, uint32_t realization, uint32_t bead, int64_t step,
                uint32_t substep, double *z /*3*/);
void orc_gauss3_batch(uint64_t seed, uint32_t realization, uint32_t n_beads, int64_t step,
                      uint32_t substep, double *z /* [n_beads][3] */);

/* simulation */
orc_sim *orc_create(const orc_params *p, const uint8_t *solid /* nsites, may be NULL */);
void orc_destroy(orc_sim *s);
void orc_init_fluid(orc_sim *s, const double *rho /* nsites or NULL */,
                    const double *u /* [3][nsites] or NULL */);
void orc_set_populations(orc_sim *s, const double *f);
void orc_get_populations(const orc_sim *s, double *f);
void orc_set_beads(orc_sim *s, const double *r, const double *v /* may be NULL */);
void orc_get_beads(const orc_sim *s, double *r, double *v);
void orc_set_step(orc_sim *s, int64_t step);
int64_t orc_get_step(const orc_sim *s);
void orc_step(orc_sim *s, int n);

/* inspection */
void orc_moments(const orc_sim *s, double *rho /* nsites */, double *u /* [3][nsites] */);
int orc_interp_weights(const orc_sim *s, const double *r, int *nodes /*8*/, double *w /*8*/);
void orc_last_coupling(const orc_sim *s, double *up, double *J);
void orc_fast_forces(const orc_sim *s, const double *r, double *F);
void orc_fast_energies(const orc_sim *s, const double *r, double *e /* bond,bend,lj,wall */);
void orc_field_forces(const orc_sim *s, const double *r, double *F);
void orc_observables(const orc_sim *s, double *out /* ORC_NOBS */);

#define ORC_NOBS 16

/* events that make a loss non-differentiable (for finite-difference checks):
 * out[0] = half kicks taken inside the pore channel, out[1] = sum over steps
 * and beads of the index of the lattice cell holding the bead */
void orc_event_counts(const orc_sim *s, double *out /*2*/);

/* MD cycles alone, with the fluid velocity at the beads held at up [N][3]
 * (no lattice update, no spread): the MD part of n coupled steps, for pins of
 * the integrators.  The step counter advances as in orc_step. */
void orc_md_only(orc_sim *s, const double *up, int n);

/* fluctuating LB: mode k of the D3Q19 moment basis on velocity c, and the
 * sixteen standard normals of one site and step (Philox4x32-10, counters
 * (site, step_lo, 0xF0000000 + j, step_hi), j = 0..3; Box-Muller) */
double orc_mode(int k, const int *c /*3*/);
void orc_fluid_noise(uint64_t seed, uint32_t realization, uint32_t site, int64_t step, double *z /*16*/);

/* Pore-channel indicator trace, for finite differences of a loss with the
 * field events held: mode 1 records the indicator of every (step, half kick,
 * bead) into buf[len] in the order the kicks happen; mode 2 replays it
 * instead of testing the bead positions; mode 0 (or buf NULL) switches the
 * trace off.  The buffer stays owned by the caller and must outlive the
 * steps that use it. */
void orc_channel_trace(orc_sim *s, int mode, int *buf, int64_t len);

/* Discrete adjoint (reverse mode) of one coupled step.  s holds the state
 * (f^n, r^n, v^n, step n).  On entry lam_f [19][nsites], lam_r, lam_v [N][3]
 * are the adjoints of f^{n+1}, r^{n+1}, v^{n+1}; on return those of f^n, r^n,
 * v^n.  dpar[0] += dL/dgamma and dpar[1] += dL/dE of this step.  s is left at
 * the state after the step, as orc_step(s, 1) would leave it. */
void orc_step_adjoint(orc_sim *s, double *lam_f, double *lam_r, double *lam_v, double *dpar /*2*/);

/* Gradient of L = mean_p x_p(K) - mean_p x_p(0) (unwrapped bead x) over K
 * coupled steps from pre-collision populations f0 (NULL: fluid at rest),
 * bead positions r0 and velocities v0 (NULL: at rest) at step step0.
 * out = {L, dL/dgamma, dL/dE}; dr0, dv0 [N][3] and df0 [19][nsites] (each may
 * be NULL) receive dL/dr0, dL/dv0, dL/df0.  Keeps all K states in memory.
 * Returns 0, or < 0 for N < 1, K < 0 or an allocation failure. */
int orc_adjoint(const orc_params *p, const uint8_t *solid, const double *f0, const double *r0,
                const double *v0, int64_t step0, int K, double *out /*3*/, double *dr0,
                double *dv0, double *df0);

#ifdef __cplusplus
}
#endif
#endif
