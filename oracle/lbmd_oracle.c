/*
 * lbmd_oracle.c -- plain, slow FP64 oracle of the coupled lattice-Boltzmann /
 * molecular-dynamics step (Fyta et al., Sec. II; set-up of Sec. IV).
 *
 * TEST INFRASTRUCTURE ONLY: only the test-suite, the smoke check and the
 * CPU-baseline leg of the benchmark load this file's library.  It shares no
 * code with the CUDA path.  It is written for a reader checking it against
 * the paper, not for speed: every step is a loop over the definition, in the
 * order the method states it, with no blocking or fusion.
 *
 * One LB step, at step n, from the pre-collision populations f^n:
 *   1. moments rho, u of f^n                                (Sec. II, Eqs. 1-2)
 *   2. fluid velocity at every bead, frozen for the MD cycle (Sec. II, text
 *      after Eq. 21), by trilinear interpolation over fluid corners
 *   3. M multiple-time-step MD steps of dt = 1/M               (Sec. II, Eq. 22)
 *      slow forces: pore field, friction gamma(u_p - v), noise  (Eqs. 12, 13, 15)
 *      fast forces (M^b sub-steps): bonds, angular term, WCA    (Eqs. 11, 14, 19)
 *      the momentum J_p the fluid gave the bead is accumulated
 *   4. spread: G(x) = - sum_p W(x - r_p) J_p                   (Sec. II, Eq. 8)
 *   5. BGK collision + source: f* = f - omega (f - f_eq) + S    (Sec. II, Eqs. 4, 5, 9)
 *   6. streaming with halfway bounce-back at solid sites          (Sec. III, walls)
 *
 * Readings of passages that are garbled or silent (relaxation sign, f_eq,
 * lattice beta = 3, the D3Q19 ordering, pore region, bead-wall interaction,
 * fast/slow split of the forces, noise mapping) are listed in the design
 * notes of the repository.
 */
#include "lbmd_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* D3Q19 lattice (Sec. II: the standard 19-speed lattice).  Ordering:        */
/* 0 rest; 1..6 axis links; 7..18 face-diagonal links; opposites adjacent.   */
/* ------------------------------------------------------------------------ */
static const int CI[19][3] = {
    {0, 0, 0},
    {1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0}, {0, 0, 1}, {0, 0, -1},
    {1, 1, 0}, {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0},
    {1, 0, 1}, {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
    {0, 1, 1}, {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};

static double weight_of(int i)
{
    int n2 = CI[i][0] * CI[i][0] + CI[i][1] * CI[i][1] + CI[i][2] * CI[i][2];
    if (n2 == 0) return 1.0 / 3.0;
    if (n2 == 1) return 1.0 / 18.0;
    return 1.0 / 36.0;
}

/* opposite link found by search: c_opp = -c_i */
static int opposite_of(int i)
{
    for (int j = 0; j < 19; j++)
        if (CI[j][0] == -CI[i][0] && CI[j][1] == -CI[i][1] && CI[j][2] == -CI[i][2]) return j;
    return -1;
}

void orc_tables(int *c, double *w, int *opp)
{
    for (int i = 0; i < 19; i++) {
        for (int a = 0; a < 3; a++) c[3 * i + a] = CI[i][a];
        w[i] = weight_of(i);
        opp[i] = opposite_of(i);
    }
}

/* Sec. II, Eq. 5, read as the second-order expansion of a Maxwellian with the
 * lattice sound speed c_s^2 = 1/3 (beta = 3):
 *   f_eq_i = w_i rho [1 + 3 c.u + 9/2 (c.u)^2 - 3/2 u.u]                     */
void orc_feq(double rho, const double *u, double *feq)
{
    double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    for (int i = 0; i < 19; i++) {
        double cu = CI[i][0] * u[0] + CI[i][1] * u[1] + CI[i][2] * u[2];
        feq[i] = weight_of(i) * rho * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * uu);
    }
}

/* Sec. II, Eq. 9 with beta = 3: S_i = w_i beta G.c_i, where G is the momentum
 * handed to the fluid per unit time (G already carries the minus sign of
 * Eq. 9, G = -(F^f + F^r)).  Then sum_i S_i = 0 and sum_i S_i c_i = G (Eq. 8). */
void orc_source(const double *G, double *S)
{
    for (int i = 0; i < 19; i++) {
        double gc = CI[i][0] * G[0] + CI[i][1] * G[1] + CI[i][2] * G[2];
        S[i] = weight_of(i) * 3.0 * gc;
    }
}

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 counter-based generator (Salmon, Moraes, Dror, Shaw, SC'11): */
/* ten rounds of two 32x32->64 multiplies with a Weyl-sequence key schedule.  */
/* ------------------------------------------------------------------------ */
void orc_philox4x32_10(const uint32_t *ctr, const uint32_t *key, uint32_t *out)
{
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; round++) {
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)x0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)x2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t y0 = hi1 ^ x1 ^ k0;
        uint32_t y1 = lo1;
        uint32_t y2 = hi0 ^ x3 ^ k1;
        uint32_t y3 = lo0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* Three standard normals for one bead and one MD step (Sec. II, Eq. 15 asks
 * for Gaussian noise; the generator and the mapping are this build's choice):
 * key = (seed_lo, seed_hi ^ realization), counter = (bead, step_lo, substep,
 * step_hi); each 32-bit word -> u = (top 24 bits + 1/2) / 2^24 in (0,1);
 * Box-Muller on (u0,u1) gives two normals, on (u2,u3) the third.            */
void orc_gauss3(uint64_t seed, uint32_t realization, uint32_t bead, int64_t step,
                uint32_t substep, double *z)
{
    uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32) ^ realization};
    uint32_t ctr[4] = {bead, (uint32_t)((uint64_t)step & 0xffffffffu), substep,
                       (uint32_t)((uint64_t)step >> 32)};
    uint32_t x[4];
    orc_philox4x32_10(ctr, key, x);
    double u[4];
    for (int k = 0; k < 4; k++) u[k] = ((double)(x[k] >> 8) + 0.5) / 16777216.0;
    const double two_pi = 6.283185307179586476925286766559;
    double a = sqrt(-2.0 * log(u[0]));
    double b = sqrt(-2.0 * log(u[2]));
    z[0] = a * cos(two_pi * u[1]);
    z[1] = a * sin(two_pi * u[1]);
    z[2] = b * cos(two_pi * u[3]);
}

/* n_beads consecutive bead indices starting at 0, same step and substep */
void orc_gauss3_batch(uint64_t seed, uint32_t realization, uint32_t n_beads, int64_t step,
                      uint32_t substep, double *z)
{
    for (uint32_t i = 0; i < n_beads; i++) orc_gauss3(seed, realization, i, step, substep, z + 3 * (size_t)i);
}

/* ------------------------------------------------------------------------ */
/* simulation state                                                          */
/* ------------------------------------------------------------------------ */
struct orc_sim {
    orc_params p;
    int ns;
    uint8_t *solid;   /* [ns] */
    double *f;        /* [19][ns] pre-collision populations f^n */
    double *fstar;    /* [19][ns] post-collision scratch */
    double *rho;      /* [ns] */
    double *u;        /* [3][ns] */
    double *G;        /* [3][ns] momentum handed to the fluid this step */
    double *r, *v;    /* [N][3] unwrapped positions, velocities */
    double *up, *J;   /* [N][3] last step's interpolated fluid velocity and impulse */
    int64_t step;
    /* events that make the loss non-differentiable, for finite-difference
     * checks: half kicks taken inside the pore channel, and the sum over steps
     * and beads of the index of the lattice cell holding the bead */
    double field_kicks, cell_sum;
    /* channel trace: 0 off; 1 record the pore-channel indicator of every
     * (step, half kick, bead) into chan; 2 replay it from chan instead of
     * testing the position (finite differences with the field events held) */
    int chan_mode;
    int *chan;
    int64_t chan_len, chan_pos;
};

static int wrap_index(int i, int n)
{
    int m = i % n;
    return m < 0 ? m + n : m;
}

static int site_of(const orc_sim *s, int x, int y, int z)
{
    x = wrap_index(x, s->p.nx);
    y = wrap_index(y, s->p.ny);
    z = wrap_index(z, s->p.nz);
    return x + s->p.nx * (y + s->p.ny * z);
}

static double wrap_coord(double x, int n)
{
    double w = x - n * floor(x / n);
    if (w >= n) w -= n;
    if (w < 0) w = 0;
    return w;
}

/* minimum-image difference on a periodic axis of length n */
static double min_image(double d, int n)
{
    return d - n * floor(d / n + 0.5);
}

orc_sim *orc_create(const orc_params *p, const uint8_t *solid)
{
    orc_sim *s = (orc_sim *)calloc(1, sizeof(orc_sim));
    s->p = *p;
    s->ns = p->nx * p->ny * p->nz;
    int ns = s->ns, N = p->n_beads > 0 ? p->n_beads : 0;
    s->solid = (uint8_t *)calloc(ns, 1);
    if (solid) memcpy(s->solid, solid, ns);
    s->f = (double *)calloc((size_t)19 * ns, sizeof(double));
    s->fstar = (double *)calloc((size_t)19 * ns, sizeof(double));
    s->rho = (double *)calloc(ns, sizeof(double));
    s->u = (double *)calloc((size_t)3 * ns, sizeof(double));
    s->G = (double *)calloc((size_t)3 * ns, sizeof(double));
    s->r = (double *)calloc((size_t)3 * (N + 1), sizeof(double));
    s->v = (double *)calloc((size_t)3 * (N + 1), sizeof(double));
    s->up = (double *)calloc((size_t)3 * (N + 1), sizeof(double));
    s->J = (double *)calloc((size_t)3 * (N + 1), sizeof(double));
    orc_init_fluid(s, NULL, NULL);
    return s;
}

void orc_destroy(orc_sim *s)
{
    if (!s) return;
    free(s->solid); free(s->f); free(s->fstar); free(s->rho); free(s->u); free(s->G);
    free(s->r); free(s->v); free(s->up); free(s->J);
    free(s);
}

/* Sec. IV: the solvent starts from the equilibrium of a given density and
 * velocity (constant density, zero speed by default).  Solid sites hold 0. */
void orc_init_fluid(orc_sim *s, const double *rho, const double *u)
{
    int ns = s->ns;
    for (int site = 0; site < ns; site++) {
        double feq[19];
        double r = rho ? rho[site] : 1.0;
        double uu[3] = {0, 0, 0};
        if (u) { uu[0] = u[site]; uu[1] = u[ns + site]; uu[2] = u[2 * ns + site]; }
        orc_feq(r, uu, feq);
        for (int i = 0; i < 19; i++) s->f[(size_t)i * ns + site] = s->solid[site] ? 0.0 : feq[i];
    }
}

void orc_set_populations(orc_sim *s, const double *f) { memcpy(s->f, f, sizeof(double) * 19 * (size_t)s->ns); }
void orc_get_populations(const orc_sim *s, double *f) { memcpy(f, s->f, sizeof(double) * 19 * (size_t)s->ns); }

void orc_set_beads(orc_sim *s, const double *r, const double *v)
{
    int N = s->p.n_beads;
    memcpy(s->r, r, sizeof(double) * 3 * N);
    if (v) memcpy(s->v, v, sizeof(double) * 3 * N);
    else memset(s->v, 0, sizeof(double) * 3 * N);
}

void orc_get_beads(const orc_sim *s, double *r, double *v)
{
    int N = s->p.n_beads;
    if (r) memcpy(r, s->r, sizeof(double) * 3 * N);
    if (v) memcpy(v, s->v, sizeof(double) * 3 * N);
}

void orc_set_step(orc_sim *s, int64_t step) { s->step = step; }
int64_t orc_get_step(const orc_sim *s) { return s->step; }

/* Sec. II, Eqs. 1-2: rho = sum_i f_i, rho u = sum_i f_i c_i, at fluid sites. */
void orc_moments(const orc_sim *s, double *rho, double *u)
{
    int ns = s->ns;
    for (int site = 0; site < ns; site++) {
        double m = 0, j[3] = {0, 0, 0};
        if (!s->solid[site]) {
            for (int i = 0; i < 19; i++) {
                double fi = s->f[(size_t)i * ns + site];
                m += fi;
                for (int a = 0; a < 3; a++) j[a] += fi * CI[i][a];
            }
        }
        rho[site] = m;
        for (int a = 0; a < 3; a++) u[(size_t)a * ns + site] = (m > 0) ? j[a] / m : 0.0;
    }
}

/* Bead <-> lattice transfer weights.  The paper uses the nearest grid point
 * and reports that a (bi)linear scheme is as accurate (Sec. II, text before
 * Eq. 20); this build uses trilinear weights over the 8 corners of the cell
 * holding the bead, with solid corners given weight 0 and the remaining
 * weights renormalised to sum to 1.  Returns the number of fluid corners. */
int orc_interp_weights(const orc_sim *s, const double *r, int *nodes, double *w)
{
    const orc_params *p = &s->p;
    double xw = wrap_coord(r[0], p->nx), yw = wrap_coord(r[1], p->ny), zw = wrap_coord(r[2], p->nz);
    int x0 = (int)floor(xw), y0 = (int)floor(yw), z0 = (int)floor(zw);
    double fx = xw - x0, fy = yw - y0, fz = zw - z0;
    double sum = 0.0;
    int nfluid = 0;
    for (int k = 0; k < 8; k++) {
        int a = k & 1, b = (k >> 1) & 1, c = (k >> 2) & 1;
        nodes[k] = site_of(s, x0 + a, y0 + b, z0 + c);
        double wk = (a ? fx : 1.0 - fx) * (b ? fy : 1.0 - fy) * (c ? fz : 1.0 - fz);
        if (p->interp == 1) /* nearest grid point (Sec. II): the corner on the bead's side of each mid-plane */
            wk = (a == (fx >= 0.5) && b == (fy >= 0.5) && c == (fz >= 0.5)) ? 1.0 : 0.0;
        if (s->solid[nodes[k]]) wk = 0.0;
        else nfluid++;
        w[k] = wk;
        sum += wk;
    }
    for (int k = 0; k < 8; k++) w[k] = (sum > 0.0) ? w[k] / sum : 0.0;
    return nfluid;
}

static void gather_velocity(const orc_sim *s, const double *r, double *up)
{
    int nodes[8];
    double w[8];
    orc_interp_weights(s, r, nodes, w);
    up[0] = up[1] = up[2] = 0.0;
    for (int k = 0; k < 8; k++)
        for (int a = 0; a < 3; a++) up[a] += w[k] * s->u[(size_t)a * s->ns + nodes[k]];
}

/* ------------------------------------------------------------------------ */
/* bead forces                                                               */
/* ------------------------------------------------------------------------ */

/* WCA: the 12-6 Lennard-Jones potential of Sec. II, Eq. 14, cut at its
 * minimum 2^(1/6) sigma and shifted up by eps so that it is purely repulsive.
 * Returns the energy; adds -dV/dd to F (d = r_self - r_other). */
static double wca(double eps, double sigma, const double *d, double *F)
{
    double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    double rc2 = pow(2.0, 1.0 / 3.0) * sigma * sigma;
    if (r2 >= rc2) return 0.0;
    double sr2 = sigma * sigma / r2;
    double sr6 = sr2 * sr2 * sr2;
    double sr12 = sr6 * sr6;
    if (F) {
        double coef = 24.0 * eps * (2.0 * sr12 - sr6) / r2;
        for (int a = 0; a < 3; a++) F[a] += coef * d[a];
    }
    return 4.0 * eps * (sr12 - sr6) + eps;
}

/* Harmonic bonds, Sec. II, Eq. 19: V = k/2 (|r_{k+1} - r_k| - r0)^2. */
static double bonds(const orc_sim *s, const double *r, double *F)
{
    const orc_params *p = &s->p;
    double e = 0.0;
    for (int k = 0; k + 1 < p->n_beads; k++) {
        double b[3], len = 0.0;
        for (int a = 0; a < 3; a++) { b[a] = r[3 * (k + 1) + a] - r[3 * k + a]; len += b[a] * b[a]; }
        len = sqrt(len);
        double dl = len - p->r0;
        e += 0.5 * p->k_bond * dl * dl;
        if (F && len > 0.0) {
            for (int a = 0; a < 3; a++) {
                double fa = -p->k_bond * dl * b[a] / len; /* force on bead k+1 */
                F[3 * (k + 1) + a] += fa;
                F[3 * k + a] -= fa;
            }
        }
    }
    return e;
}

/* Angular term, Sec. II (text after Eq. 14): V = kappa phi^2 / 2, with phi
 * the angle between consecutive bond vectors b1 = r_k - r_{k-1} and
 * b2 = r_{k+1} - r_k (phi = 0 for a straight chain).  With c = cos phi,
 * -dV/dx = (kappa phi / sin phi) dc/dx. */
static double bending(const orc_sim *s, const double *r, double *F)
{
    const orc_params *p = &s->p;
    double e = 0.0;
    for (int k = 1; k + 1 < p->n_beads; k++) {
        double b1[3], b2[3], cr[3];
        for (int a = 0; a < 3; a++) {
            b1[a] = r[3 * k + a] - r[3 * (k - 1) + a];
            b2[a] = r[3 * (k + 1) + a] - r[3 * k + a];
        }
        cr[0] = b1[1] * b2[2] - b1[2] * b2[1];
        cr[1] = b1[2] * b2[0] - b1[0] * b2[2];
        cr[2] = b1[0] * b2[1] - b1[1] * b2[0];
        double l1 = sqrt(b1[0] * b1[0] + b1[1] * b1[1] + b1[2] * b1[2]);
        double l2 = sqrt(b2[0] * b2[0] + b2[1] * b2[1] + b2[2] * b2[2]);
        double dot = b1[0] * b2[0] + b1[1] * b2[1] + b1[2] * b2[2];
        double crn = sqrt(cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2]);
        double phi = atan2(crn, dot);
        e += 0.5 * p->kappa_bend * phi * phi;
        if (!F || l1 == 0.0 || l2 == 0.0) continue;
        double c = dot / (l1 * l2);
        double sn = crn / (l1 * l2);
        double A;
        if (sn > 1e-12) A = p->kappa_bend * phi / sn;
        else A = (c > 0.0) ? p->kappa_bend : 0.0; /* phi/sin(phi) -> 1 as phi -> 0 */
        for (int a = 0; a < 3; a++) {
            double dc_db1 = b2[a] / (l1 * l2) - c * b1[a] / (l1 * l1);
            double dc_db2 = b1[a] / (l1 * l2) - c * b2[a] / (l2 * l2);
            F[3 * (k - 1) + a] += -A * dc_db1;
            F[3 * k + a] += A * (dc_db1 - dc_db2);
            F[3 * (k + 1) + a] += A * dc_db2;
        }
    }
    return e;
}

/* Excluded volume between beads (Sec. II, Eqs. 11 and 14): WCA over every
 * non-bonded pair (|i - j| >= 2), minimum image in the periodic box. */
static double pair_wca(const orc_sim *s, const double *r, double *F)
{
    const orc_params *p = &s->p;
    double e = 0.0;
    for (int i = 0; i < p->n_beads; i++) {
        for (int j = i + 2; j < p->n_beads; j++) {
            double d[3] = {min_image(r[3 * i] - r[3 * j], p->nx),
                           min_image(r[3 * i + 1] - r[3 * j + 1], p->ny),
                           min_image(r[3 * i + 2] - r[3 * j + 2], p->nz)};
            double fi[3] = {0, 0, 0};
            e += wca(p->lj_eps, p->lj_sigma, d, fi);
            for (int a = 0; a < 3; a++) { F[3 * i + a] += fi[a]; F[3 * j + a] -= fi[a]; }
        }
    }
    return e;
}

/* Bead-wall interaction: WCA between a bead and the centre of every solid
 * site within the cutoff (the paper only names an interaction with the wall
 * molecules, Sec. I).  Candidate sites are all lattice points in the box
 * [r - rc, r + rc]. */
static double wall_wca(const orc_sim *s, const double *r, double *F)
{
    const orc_params *p = &s->p;
    double rc = pow(2.0, 1.0 / 6.0) * p->wall_sigma;
    double e = 0.0;
    for (int i = 0; i < p->n_beads; i++) {
        const double *ri = r + 3 * i;
        int lo[3], hi[3];
        for (int a = 0; a < 3; a++) { lo[a] = (int)floor(ri[a] - rc); hi[a] = (int)floor(ri[a] + rc) + 1; }
        for (int z = lo[2]; z <= hi[2]; z++)
            for (int y = lo[1]; y <= hi[1]; y++)
                for (int x = lo[0]; x <= hi[0]; x++) {
                    if (!s->solid[site_of(s, x, y, z)]) continue;
                    double d[3] = {ri[0] - x, ri[1] - y, ri[2] - z};
                    double fi[3] = {0, 0, 0};
                    e += wca(p->wall_eps, p->wall_sigma, d, fi);
                    for (int a = 0; a < 3; a++) F[3 * i + a] += fi[a];
                }
    }
    return e;
}

/* Fast (inner-cycle) forces: every conservative bead force. */
void orc_fast_forces(const orc_sim *s, const double *r, double *F)
{
    memset(F, 0, sizeof(double) * 3 * s->p.n_beads);
    bonds(s, r, F);
    bending(s, r, F);
    pair_wca(s, r, F);
    wall_wca(s, r, F);
}

void orc_fast_energies(const orc_sim *s, const double *r, double *e)
{
    e[0] = bonds(s, r, NULL);
    e[1] = bending(s, r, NULL);
    double *scratch = (double *)calloc((size_t)3 * s->p.n_beads + 3, sizeof(double));
    e[2] = pair_wca(s, r, scratch);
    e[3] = wall_wca(s, r, scratch);
    free(scratch);
}

/* Driving field (Sec. IV): a force q E x^ on beads inside the pore channel,
 * 3 sites long in x centred on the wall plane and as wide as the pore, with
 * half a site of padding: |x - wall_x| <= 3/2 and y, z within
 * [lo - 1/2, lo + h - 1/2] where lo = n/2 - floor(h/2) is the first pore
 * site along that axis. */
static int in_pore_channel(const orc_sim *s, const double *r)
{
    const orc_params *p = &s->p;
    if (p->wall_x < 0) return 0;
    double dx = min_image(r[0] - p->wall_x, p->nx);
    if (fabs(dx) > 1.5) return 0;
    double yw = wrap_coord(r[1], p->ny), zw = wrap_coord(r[2], p->nz);
    int ly = p->ny / 2 - p->pore_h / 2, lz = p->nz / 2 - p->pore_h / 2;
    if (yw < ly - 0.5 || yw > ly + p->pore_h - 0.5) return 0;
    if (zw < lz - 0.5 || zw > lz + p->pore_h - 0.5) return 0;
    return 1;
}

void orc_field_forces(const orc_sim *s, const double *r, double *F)
{
    for (int i = 0; i < s->p.n_beads; i++) {
        F[3 * i] = in_pore_channel(s, r + 3 * i) ? s->p.E : 0.0;
        F[3 * i + 1] = 0.0;
        F[3 * i + 2] = 0.0;
    }
}

/* ------------------------------------------------------------------------ */
/* one MD cycle (Sec. II, Eq. 22, as a multiple-time-step velocity Verlet)   */
/* ------------------------------------------------------------------------ */
/* pore-channel indicator of bead i at a half kick, through the trace */
static int kick_channel(orc_sim *s, int i)
{
    int ch;
    if (s->chan_mode == 2 && s->chan_pos < s->chan_len) ch = s->chan[s->chan_pos++];
    else {
        ch = in_pore_channel(s, s->r + 3 * i);
        if (s->chan_mode == 1 && s->chan_pos < s->chan_len) s->chan[s->chan_pos++] = ch;
    }
    return ch;
}

static void slow_half_kick(orc_sim *s, const double *xi, double h)
{
    const orc_params *p = &s->p;
    int N = p->n_beads;
    for (int i = 0; i < N; i++) {
        int ch = kick_channel(s, i);
        if (ch) s->field_kicks += 1.0;
        double Fe[3] = {ch ? p->E : 0.0, 0.0, 0.0}; /* q E x^ in the channel, q = 1 */
        for (int a = 0; a < 3; a++) {
            double drag = p->gamma * (s->up[3 * i + a] - s->v[3 * i + a]); /* Eq. 12 */
            double fluid = drag + xi[3 * i + a];                            /* Eqs. 12 + 13 */
            s->v[3 * i + a] += h * (Fe[a] + fluid);
            s->J[3 * i + a] += h * fluid;
        }
    }
}

/* What one MD cycle passed through, kept for the adjoint sweep. */
typedef struct {
    double *rt; /* [M*Mb + 1][3N] positions at the boundaries of the inner sub-steps */
    double *vk; /* [2M][3N] velocity just before each half kick */
    int *ch;    /* [2M][N] 1 where the bead sat in the pore channel at that kick */
    double *xi; /* [M][3N] noise of each MD step */
} md_record;

static void record_kick(const orc_sim *s, md_record *rec, int k)
{
    int N = s->p.n_beads;
    memcpy(rec->vk + (size_t)k * 3 * N, s->v, sizeof(double) * 3 * N);
    for (int i = 0; i < N; i++) {
        int ch = in_pore_channel(s, s->r + 3 * i);
        if (s->chan_mode == 2 && s->chan_pos + i < s->chan_len) ch = s->chan[s->chan_pos + i];
        rec->ch[(size_t)k * N + i] = ch;
    }
}

/* Stochastic position Verlet (Sec. II, Eq. SPValgo) nested as the
 * multiple-time-step scheme that follows it in the paper.  Per outer step
 * (dt = 1/M): a half kick with the slow force (the pore field); M^b inner
 * steps of length h = dt/M^b, each a half drift, the exact Ornstein-Uhlenbeck
 * velocity update over h with the fast (conservative) forces evaluated at the
 * half-drifted positions, and a half drift; a half kick.  With c = exp(-gamma h)
 * and m = 1:
 *   v' = c v + (1 - c) u_p + (1 - c)/gamma F + sqrt(kT (1 - c^2)) z,
 * a fresh normal vector z per bead and inner step (Philox counter word 2 =
 * the inner-step index).  The momentum the fluid gives the bead over the step
 * is what the velocity gains beyond the conservative impulse: v' - v - h F. */
/* half kick of the stochastic position Verlet cycle: the field only */
static void field_half_kick(orc_sim *s, double dt)
{
    for (int i = 0; i < s->p.n_beads; i++) {
        int ch = kick_channel(s, i);
        if (ch) s->field_kicks += 1.0;
        s->v[3 * i] += 0.5 * dt * (ch ? s->p.E : 0.0);
    }
}

static void md_cycle_spv(orc_sim *s)
{
    const orc_params *p = &s->p;
    int N = p->n_beads;
    double dt = 1.0 / p->md_outer, h = dt / p->md_inner;
    double c = exp(-p->gamma * h);
    double g1 = p->gamma > 0.0 ? (1.0 - c) / p->gamma : h;
    double sig = p->kT > 0.0 ? sqrt(p->kT * (1.0 - c * c)) : 0.0;
    double *F = (double *)malloc(sizeof(double) * (3 * N + 3));
    memset(s->J, 0, sizeof(double) * 3 * N);
    for (int sub = 0; sub < p->md_outer; sub++) {
        field_half_kick(s, dt);
        for (int b = 0; b < p->md_inner; b++) {
            int t = sub * p->md_inner + b;
            for (int k = 0; k < 3 * N; k++) s->r[k] += 0.5 * h * s->v[k];
            orc_fast_forces(s, s->r, F);
            for (int i = 0; i < N; i++) {
                double z[3] = {0, 0, 0};
                if (sig > 0.0) orc_gauss3(p->seed, p->realization, (uint32_t)i, s->step, (uint32_t)t, z);
                for (int a = 0; a < 3; a++) {
                    size_t q = 3 * (size_t)i + a;
                    double vn = c * s->v[q] + (1.0 - c) * s->up[q] + g1 * F[q] + sig * z[a];
                    s->J[q] += vn - s->v[q] - h * F[q];
                    s->v[q] = vn;
                }
            }
            for (int k = 0; k < 3 * N; k++) s->r[k] += 0.5 * h * s->v[k];
        }
        field_half_kick(s, dt);
    }
    free(F);
}

static void md_cycle(orc_sim *s, md_record *rec)
{
    const orc_params *p = &s->p;
    if (p->integrator == 1) {
        md_cycle_spv(s);
        return;
    }
    int N = p->n_beads;
    double dt = 1.0 / p->md_outer;
    double dtb = dt / p->md_inner;
    double *xi = (double *)malloc(sizeof(double) * 3 * N);
    double *F = (double *)malloc(sizeof(double) * 3 * N);
    /* Eq. 15: <xi xi> = 2 gamma kT / m delta(t - t'); held over one MD step of
     * length dt, each component has variance 2 gamma kT / dt. */
    double amp = (p->kT > 0.0) ? sqrt(2.0 * p->gamma * p->kT / dt) : 0.0;
    memset(s->J, 0, sizeof(double) * 3 * N);
    if (rec) memcpy(rec->rt, s->r, sizeof(double) * 3 * N);
    for (int sub = 0; sub < p->md_outer; sub++) {
        for (int i = 0; i < N; i++) {
            double z[3] = {0, 0, 0};
            if (amp > 0.0) orc_gauss3(p->seed, p->realization, (uint32_t)i, s->step, (uint32_t)sub, z);
            for (int a = 0; a < 3; a++) xi[3 * i + a] = amp * z[a];
        }
        if (rec) {
            memcpy(rec->xi + (size_t)sub * 3 * N, xi, sizeof(double) * 3 * N);
            record_kick(s, rec, 2 * sub);
        }
        slow_half_kick(s, xi, 0.5 * dt);
        for (int b = 0; b < p->md_inner; b++) {
            orc_fast_forces(s, s->r, F);
            for (int k = 0; k < 3 * N; k++) s->v[k] += 0.5 * dtb * F[k];
            for (int k = 0; k < 3 * N; k++) s->r[k] += dtb * s->v[k];
            if (rec) memcpy(rec->rt + ((size_t)sub * p->md_inner + b + 1) * 3 * N, s->r, sizeof(double) * 3 * N);
            orc_fast_forces(s, s->r, F);
            for (int k = 0; k < 3 * N; k++) s->v[k] += 0.5 * dtb * F[k];
        }
        if (rec) record_kick(s, rec, 2 * sub + 1);
        slow_half_kick(s, xi, 0.5 * dt);
    }
    free(xi);
    free(F);
}

/* ------------------------------------------------------------------------ */
/* fluctuating LB (Sec. II, the stochastic term F_i of Eq. 4, after the     */
/* moment-space scheme of the cited work of Adhikari et al.)                 */
/* ------------------------------------------------------------------------ */

/* Mode k of the D3Q19 moment basis evaluated on the velocity c: density,
 * momentum (k = 1..3), the six stress modes (4..9: bulk, two normal-stress
 * differences, three shear), and nine ghost modes (10..18).  The modes are
 * orthogonal under the lattice weights: sum_i w_i e_k(c_i) e_l(c_i) = b_k delta_kl. */
double orc_mode(int k, const int *c)
{
    double x = c[0], y = c[1], z = c[2], q = x * x + y * y + z * z;
    switch (k) {
    case 0: return 1.0;
    case 1: return x;
    case 2: return y;
    case 3: return z;
    case 4: return q - 1.0;
    case 5: return 3.0 * x * x - q;
    case 6: return y * y - z * z;
    case 7: return x * y;
    case 8: return y * z;
    case 9: return z * x;
    case 10: return (3.0 * q - 5.0) * x;
    case 11: return (3.0 * q - 5.0) * y;
    case 12: return (3.0 * q - 5.0) * z;
    case 13: return (y * y - z * z) * x;
    case 14: return (z * z - x * x) * y;
    case 15: return (x * x - y * y) * z;
    case 16: return 3.0 * q * q - 6.0 * q + 1.0;
    case 17: return (2.0 * q - 3.0) * (3.0 * x * x - q);
    case 18: return (2.0 * q - 3.0) * (y * y - z * z);
    }
    return 0.0;
}

/* Sixteen standard normals for the fluctuations of one site and step:
 * Philox4x32-10 with the bead key (seed_lo, seed_hi ^ realization) and the
 * counters (site, step_lo, 0xF0000000 + j, step_hi), j = 0..3; each word ->
 * u = (top 24 bits + 1/2) 2^-24; Box-Muller on (u0, u1) and (u2, u3). */
void orc_fluid_noise(uint64_t seed, uint32_t realization, uint32_t site, int64_t step, double *z)
{
    uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32) ^ realization};
    const double two_pi = 6.283185307179586476925286766559;
    for (uint32_t j = 0; j < 4; j++) {
        uint32_t ctr[4] = {site, (uint32_t)((uint64_t)step & 0xffffffffu), 0xF0000000u + j,
                           (uint32_t)((uint64_t)step >> 32)};
        uint32_t x[4];
        orc_philox4x32_10(ctr, key, x);
        double u[4];
        for (int k = 0; k < 4; k++) u[k] = ((double)(x[k] >> 8) + 0.5) / 16777216.0;
        double a = sqrt(-2.0 * log(u[0])), b = sqrt(-2.0 * log(u[2]));
        z[4 * j + 0] = a * cos(two_pi * u[1]);
        z[4 * j + 1] = a * sin(two_pi * u[1]);
        z[4 * j + 2] = b * cos(two_pi * u[3]);
        z[4 * j + 3] = b * sin(two_pi * u[3]);
    }
}

/* Fluctuation added to the post-collision populations of one site: every
 * non-conserved mode k (4..18) relaxes with gamma_k = 1 - omega (BGK) and
 * receives a kick of variance mu b_k (1 - gamma_k^2), mu = rho kT / c_s^2;
 * back in population space
 *   dF_i = w_i sum_k e_k(c_i) sqrt(mu (1 - gamma_k^2) / b_k) r_k.
 * The conserved modes get none, so mass and momentum are untouched. */
static void fluid_fluctuation(const orc_sim *s, int site, double rho, double *dF)
{
    const orc_params *p = &s->p;
    double gam = 1.0 - 1.0 / p->tau;
    double mu = 3.0 * rho * p->lb_kT;
    double z[16];
    orc_fluid_noise(p->seed, p->realization, (uint32_t)site, s->step, z);
    for (int i = 0; i < 19; i++) dF[i] = 0.0;
    for (int k = 4; k < 19; k++) {
        double b = 0.0;
        for (int i = 0; i < 19; i++) {
            double e = orc_mode(k, CI[i]);
            b += weight_of(i) * e * e;
        }
        double amp = sqrt(mu * (1.0 - gam * gam) / b) * z[k - 4];
        for (int i = 0; i < 19; i++) dF[i] += weight_of(i) * orc_mode(k, CI[i]) * amp;
    }
}

/* ------------------------------------------------------------------------ */
/* one coupled LB-MD step                                                    */
/* ------------------------------------------------------------------------ */
static void one_step(orc_sim *s)
{
    const orc_params *p = &s->p;
    int ns = s->ns, N = p->n_beads;
    double omega = 1.0 / p->tau;

    /* 1. moments of the pre-collision populations */
    orc_moments(s, s->rho, s->u);

    /* 2. fluid velocity at the beads, frozen for the MD cycle */
    double *r_start = (double *)malloc(sizeof(double) * 3 * (N + 1));
    memcpy(r_start, s->r, sizeof(double) * 3 * N);
    for (int i = 0; i < N; i++) {
        gather_velocity(s, s->r + 3 * i, s->up + 3 * i);
        int nodes[8];
        double w[8];
        orc_interp_weights(s, s->r + 3 * i, nodes, w);
        double id = nodes[0]; /* the cell (trilinear) or the chosen node (nearest grid point) */
        if (p->interp == 1) {
            id = -1.0;
            for (int k = 0; k < 8; k++)
                if (w[k] > 0.0) id = nodes[k];
        }
        s->cell_sum += id;
    }

    /* 3. MD cycle; J_i = momentum the fluid gave bead i */
    if (N > 0) md_cycle(s, NULL);

    /* 4. reaction: G(x) = - sum_i W(x - r_i) J_i, with the weights of step 2 */
    memset(s->G, 0, sizeof(double) * 3 * ns);
    for (int i = 0; i < N; i++) {
        int nodes[8];
        double w[8];
        orc_interp_weights(s, r_start + 3 * i, nodes, w);
        for (int k = 0; k < 8; k++)
            for (int a = 0; a < 3; a++) s->G[(size_t)a * ns + nodes[k]] -= w[k] * s->J[3 * i + a];
    }
    free(r_start);

    /* 5. collision (Eq. 4 with the relaxation sign that makes BGK dissipative)
     *    plus the source of Eq. 9 for the bead reaction and the body force */
    for (int site = 0; site < ns; site++) {
        if (s->solid[site]) continue;
        double uu[3] = {s->u[site], s->u[ns + site], s->u[2 * ns + site]};
        double feq[19], S[19];
        orc_feq(s->rho[site], uu, feq);
        double Gs[3] = {s->G[site] + p->body_force[0], s->G[ns + site] + p->body_force[1],
                        s->G[2 * ns + site] + p->body_force[2]};
        orc_source(Gs, S);
        double dF[19] = {0};
        if (p->lb_kT > 0.0) fluid_fluctuation(s, site, s->rho[site], dF);
        for (int i = 0; i < 19; i++) {
            double fi = s->f[(size_t)i * ns + site];
            s->fstar[(size_t)i * ns + site] = fi - omega * (fi - feq[i]) + S[i] + dF[i];
        }
    }

    /* 6. streaming along the links; a population headed into a solid site is
     *    reflected back into the opposite link of its own site */
    for (size_t k = 0; k < (size_t)19 * ns; k++) s->f[k] = 0.0;
    for (int z = 0; z < p->nz; z++)
        for (int y = 0; y < p->ny; y++)
            for (int x = 0; x < p->nx; x++) {
                int site = site_of(s, x, y, z);
                if (s->solid[site]) continue;
                for (int i = 0; i < 19; i++) {
                    int dest = site_of(s, x + CI[i][0], y + CI[i][1], z + CI[i][2]);
                    double val = s->fstar[(size_t)i * ns + site];
                    if (s->solid[dest]) s->f[(size_t)opposite_of(i) * ns + site] = val;
                    else s->f[(size_t)i * ns + dest] = val;
                }
            }
    s->step += 1;
}

void orc_step(orc_sim *s, int n)
{
    for (int k = 0; k < n; k++) one_step(s);
}

void orc_last_coupling(const orc_sim *s, double *up, double *J)
{
    int N = s->p.n_beads;
    if (up) memcpy(up, s->up, sizeof(double) * 3 * N);
    if (J) memcpy(J, s->J, sizeof(double) * 3 * N);
}

/* ------------------------------------------------------------------------ */
/* observables (Sec. III global momenta; Sec. IV.B radii; Sec. IV.C, Eqs.    */
/* 24-25 work rates, here for one realization and one instant)               */
/* ------------------------------------------------------------------------ */
static double radius_of_gyration(const double *r, const int *sel, int N)
{
    double cm[3] = {0, 0, 0};
    int n = 0;
    for (int i = 0; i < N; i++)
        if (sel[i]) { n++; for (int a = 0; a < 3; a++) cm[a] += r[3 * i + a]; }
    if (n == 0) return 0.0;
    for (int a = 0; a < 3; a++) cm[a] /= n;
    double acc = 0.0;
    for (int i = 0; i < N; i++)
        if (sel[i])
            for (int a = 0; a < 3; a++) { double d = r[3 * i + a] - cm[a]; acc += d * d; }
    return sqrt(acc / n);
}

void orc_observables(const orc_sim *s, double *out)
{
    const orc_params *p = &s->p;
    int ns = s->ns, N = p->n_beads;
    for (int k = 0; k < ORC_NOBS; k++) out[k] = 0.0;
    double *rho = (double *)malloc(sizeof(double) * ns);
    double *u = (double *)malloc(sizeof(double) * 3 * ns);
    orc_moments(s, rho, u);
    for (int site = 0; site < ns; site++) {
        out[0] += rho[site];
        for (int a = 0; a < 3; a++) out[1 + a] += rho[site] * u[(size_t)a * ns + site];
    }
    /* current fluid velocity at each bead, from the current populations */
    orc_sim tmp = *s;
    tmp.u = u;
    double *Fe = (double *)malloc(sizeof(double) * 3 * (N + 1));
    int *trans = (int *)calloc(N + 1, sizeof(int));
    int *untrans = (int *)calloc(N + 1, sizeof(int));
    orc_field_forces(s, s->r, Fe);
    for (int i = 0; i < N; i++) {
        double up[3];
        gather_velocity(&tmp, s->r + 3 * i, up);
        for (int a = 0; a < 3; a++) {
            out[4 + a] += s->v[3 * i + a];
            out[7 + a] += s->r[3 * i + a] / N;
            out[11] += p->gamma * s->v[3 * i + a] * up[a];
            out[12] += Fe[3 * i + a] * s->v[3 * i + a];
        }
        trans[i] = (p->wall_x >= 0) && (s->r[3 * i] > p->wall_x + 0.5);
        untrans[i] = !trans[i];
        out[10] += trans[i];
    }
    out[13] = radius_of_gyration(s->r, untrans, N);
    out[14] = radius_of_gyration(s->r, trans, N);
    out[15] = (double)s->step;
    free(rho); free(u); free(Fe); free(trans); free(untrans);
}

void orc_event_counts(const orc_sim *s, double *out)
{
    out[0] = s->field_kicks;
    out[1] = s->cell_sum;
}

/* ======================================================================== */
/* Discrete adjoint (reverse mode) of the coupled step, in FP64.             */
/*                                                                          */
/* The step above maps (f^n, r^n, v^n) to (f^{n+1}, r^{n+1}, v^{n+1}) with   */
/* the parameters gamma (friction, and the noise amplitude sqrt(2 gamma kT / */
/* dt)) and E (pore field).  Given the adjoints lam_f, lam_r, lam_v of the    */
/* outputs, the adjoint step returns those of the inputs and adds the       */
/* parameter sensitivities, walking the forward stages in reverse:          */
/*   6' streaming with bounce-back (a permutation: its transpose)           */
/*   5' collision + source, through f_eq(rho(f), u(f)) and S(G)             */
/*   4' spread G(x) = -sum_p W(x - r_p) J_p (through J_p and the weights)   */
/*   3' the MD cycle, kick by kick and sub-step by sub-step                  */
/*   2' the gather u_p = sum_k W_k u(x_k) (through u(f) and the weights)     */
/* The pore-field indicator is piecewise constant in r, so its derivative   */
/* is taken as 0 (the loss jumps where a bead crosses the channel boundary  */
/* at a kick; orc_event_counts lets a finite-difference check spot that).   */
/* ======================================================================== */

/* Renormalised trilinear weights of orc_interp_weights and their gradient
 * with respect to the bead position, dW[k][a] = dW_k / dr_a, from the
 * product form w_k = prod_a (fa or 1 - fa) and the quotient rule for
 * W_k = m_k w_k / sum_j m_j w_j (m = 1 on fluid corners, 0 on solid). */
static void weights_and_gradient(const orc_sim *s, const double *r, int *nodes, double *W, double dW[8][3])
{
    const orc_params *p = &s->p;
    double wr[3] = {wrap_coord(r[0], p->nx), wrap_coord(r[1], p->ny), wrap_coord(r[2], p->nz)};
    int c0[3];
    double fr[3];
    for (int a = 0; a < 3; a++) { c0[a] = (int)floor(wr[a]); fr[a] = wr[a] - c0[a]; }
    double raw[8], draw[8][3], sum = 0.0, dsum[3] = {0, 0, 0};
    for (int k = 0; k < 8; k++) {
        int bit[3] = {k & 1, (k >> 1) & 1, (k >> 2) & 1};
        nodes[k] = site_of(s, c0[0] + bit[0], c0[1] + bit[1], c0[2] + bit[2]);
        double m = s->solid[nodes[k]] ? 0.0 : 1.0;
        double fac[3];
        for (int a = 0; a < 3; a++) fac[a] = bit[a] ? fr[a] : 1.0 - fr[a];
        raw[k] = m * fac[0] * fac[1] * fac[2];
        for (int a = 0; a < 3; a++) {
            double d = bit[a] ? 1.0 : -1.0;
            for (int b = 0; b < 3; b++)
                if (b != a) d *= fac[b];
            draw[k][a] = m * d;
        }
        if (s->p.interp == 1) { /* nearest grid point: piecewise constant, gradient 0 */
            raw[k] = m * ((bit[0] == (fr[0] >= 0.5) && bit[1] == (fr[1] >= 0.5) && bit[2] == (fr[2] >= 0.5)) ? 1.0 : 0.0);
            for (int a = 0; a < 3; a++) draw[k][a] = 0.0;
        }
        sum += raw[k];
        for (int a = 0; a < 3; a++) dsum[a] += draw[k][a];
    }
    for (int k = 0; k < 8; k++) {
        W[k] = sum > 0.0 ? raw[k] / sum : 0.0;
        for (int a = 0; a < 3; a++) dW[k][a] = sum > 0.0 ? (draw[k][a] - W[k] * dsum[a]) / sum : 0.0;
    }
}

/* partial derivatives of f_eq_i = w_i rho (1 + 3 c.u + 9/2 (c.u)^2 - 3/2 u.u)
 * with respect to rho (u held) and to u_a (rho held) */
static void feq_partials(int i, double rho, const double *u, double *d_rho, double *d_u)
{
    double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    double cu = CI[i][0] * u[0] + CI[i][1] * u[1] + CI[i][2] * u[2];
    double w = weight_of(i);
    *d_rho = w * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * uu);
    for (int a = 0; a < 3; a++) d_u[a] = w * rho * (3.0 * CI[i][a] + 9.0 * cu * CI[i][a] - 3.0 * u[a]);
}

/* (dF/dr) w for the fast forces, by a central difference of orc_fast_forces
 * along w (step 1e-6 / max|w|; the forces are smooth between the rare
 * instants a pair crosses the cut-off). */
static void force_jacobian_times(const orc_sim *s, const double *r, const double *w, double *out)
{
    int n = 3 * s->p.n_beads;
    double wmax = 0.0;
    for (int k = 0; k < n; k++) wmax = fmax(wmax, fabs(w[k]));
    if (wmax == 0.0) {
        for (int k = 0; k < n; k++) out[k] = 0.0;
        return;
    }
    double eps = 1e-6 / wmax;
    double *rp = (double *)malloc(sizeof(double) * (n + 3));
    double *Fp = (double *)malloc(sizeof(double) * (n + 3));
    double *Fm = (double *)malloc(sizeof(double) * (n + 3));
    for (int k = 0; k < n; k++) rp[k] = r[k] + eps * w[k];
    orc_fast_forces(s, rp, Fp);
    for (int k = 0; k < n; k++) rp[k] = r[k] - eps * w[k];
    orc_fast_forces(s, rp, Fm);
    for (int k = 0; k < n; k++) out[k] = (Fp[k] - Fm[k]) / (2.0 * eps);
    free(rp); free(Fp); free(Fm);
}

/* Reverse of one half kick  v' = v + h (E chi x^ + gamma (u_p - v) + xi),
 * J' = J + h (gamma (u_p - v) + xi), with xi = sqrt(2 gamma kT / dt) z.
 * lam_v holds the adjoint of v' on entry and of v on return; lam_J is the
 * adjoint of J (constant through the cycle, J only accumulates). */
static void kick_adjoint(const orc_sim *s, const md_record *rec, int k, int sub, const double *up,
                         const double *lam_J, double *lam_v, double *lam_up, double *dpar)
{
    const orc_params *p = &s->p;
    int N = p->n_beads;
    double dt = 1.0 / p->md_outer, h = 0.5 * dt;
    int noisy = p->kT > 0.0 && p->gamma > 0.0;
    for (int i = 0; i < N; i++) {
        for (int a = 0; a < 3; a++) {
            size_t q = 3 * (size_t)i + a;
            double lv = lam_v[q], lj = lam_J[q];
            double vb = rec->vk[(size_t)k * 3 * N + q];
            double xi = rec->xi[(size_t)sub * 3 * N + q];
            double dxi_dgamma = noisy ? xi / (2.0 * p->gamma) : 0.0;
            dpar[0] += h * ((up[q] - vb) + dxi_dgamma) * (lv + lj);
            if (a == 0) dpar[1] += h * rec->ch[(size_t)k * N + i] * lv;
            lam_up[q] += h * p->gamma * (lv + lj);
            lam_v[q] = lv * (1.0 - h * p->gamma) - h * p->gamma * lj;
        }
    }
}

/* Reverse of md_cycle: lam_r, lam_v hold the adjoints of the end positions
 * and velocities on entry and of the start ones on return.  Velocity Verlet
 * sub-step t -> t+1:  v_h = v + hb F(r_t); r_{t+1} = r_t + dtb v_h;
 * v' = v_h + hb F(r_{t+1}). */
static void md_cycle_adjoint(const orc_sim *s, const md_record *rec, const double *up, const double *lam_J,
                             double *lam_r, double *lam_v, double *lam_up, double *dpar)
{
    const orc_params *p = &s->p;
    int N = p->n_beads, M = p->md_outer, Mb = p->md_inner;
    double dtb = 1.0 / M / Mb, hb = 0.5 * dtb;
    double *jw = (double *)malloc(sizeof(double) * (3 * N + 3));
    for (int sub = M - 1; sub >= 0; sub--) {
        kick_adjoint(s, rec, 2 * sub + 1, sub, up, lam_J, lam_v, lam_up, dpar);
        for (int b = Mb - 1; b >= 0; b--) {
            size_t t = (size_t)sub * Mb + b;
            force_jacobian_times(s, rec->rt + (t + 1) * 3 * N, lam_v, jw);
            for (int q = 0; q < 3 * N; q++) lam_r[q] += hb * jw[q];
            for (int q = 0; q < 3 * N; q++) lam_v[q] += dtb * lam_r[q];
            force_jacobian_times(s, rec->rt + t * 3 * N, lam_v, jw);
            for (int q = 0; q < 3 * N; q++) lam_r[q] += hb * jw[q];
        }
        kick_adjoint(s, rec, 2 * sub, sub, up, lam_J, lam_v, lam_up, dpar);
    }
    free(jw);
}

void orc_step_adjoint(orc_sim *s, double *lam_f, double *lam_r, double *lam_v, double *dpar)
{
    const orc_params *p = &s->p;
    int ns = s->ns, N = p->n_beads, M = p->md_outer, Mb = p->md_inner;
    double omega = 1.0 / p->tau;

    /* recompute the forward step's intermediates from (f^n, r^n, v^n) */
    orc_moments(s, s->rho, s->u);
    double *r_start = (double *)malloc(sizeof(double) * (3 * N + 3));
    memcpy(r_start, s->r, sizeof(double) * 3 * N);
    for (int i = 0; i < N; i++) gather_velocity(s, r_start + 3 * i, s->up + 3 * i);
    md_record rec;
    rec.rt = (double *)malloc(sizeof(double) * ((size_t)M * Mb + 1) * (3 * N + 3));
    rec.vk = (double *)malloc(sizeof(double) * 2 * M * (3 * N + 3));
    rec.ch = (int *)malloc(sizeof(int) * 2 * M * (N + 1));
    rec.xi = (double *)malloc(sizeof(double) * M * (3 * N + 3));
    if (N > 0) md_cycle(s, &rec);

    /* 6'. streaming: f^{n+1}_i(x + c_i) = f*_i(x), or f^{n+1}_opp(i)(x) = f*_i(x)
     *     when x + c_i is solid */
    double *lam_star = (double *)calloc((size_t)19 * ns, sizeof(double));
    for (int z = 0; z < p->nz; z++)
        for (int y = 0; y < p->ny; y++)
            for (int x = 0; x < p->nx; x++) {
                int site = site_of(s, x, y, z);
                if (s->solid[site]) continue;
                for (int i = 0; i < 19; i++) {
                    int dest = site_of(s, x + CI[i][0], y + CI[i][1], z + CI[i][2]);
                    lam_star[(size_t)i * ns + site] = s->solid[dest] ? lam_f[(size_t)opposite_of(i) * ns + site]
                                                                     : lam_f[(size_t)i * ns + dest];
                }
            }

    /* 5'. f*_i = f_i - omega (f_i - f_eq_i(f)) + S_i(G + g) at fluid sites */
    double *lam_new = (double *)calloc((size_t)19 * ns, sizeof(double));
    double *lam_G = (double *)calloc((size_t)3 * ns, sizeof(double));
    double dS[3][19];
    for (int a = 0; a < 3; a++) {
        double e[3] = {0, 0, 0};
        e[a] = 1.0;
        orc_source(e, dS[a]); /* S is linear in G: dS_i/dG_a */
    }
    for (int site = 0; site < ns; site++) {
        if (s->solid[site]) continue;
        double rho = s->rho[site];
        double uu[3] = {s->u[site], s->u[ns + site], s->u[2 * ns + site]};
        /* reverse through f_eq(rho, u): lam_rho = sum_i lam*_i d f_eq_i/d rho,
         * lam_u = sum_i lam*_i d f_eq_i/d u; then rho = sum f, u = sum f c / rho */
        double lam_rho = 0.0, lam_u[3] = {0, 0, 0};
        for (int i = 0; i < 19; i++) {
            double li = omega * lam_star[(size_t)i * ns + site];
            double d_rho, d_u[3];
            feq_partials(i, rho, uu, &d_rho, d_u);
            lam_rho += li * d_rho;
            for (int a = 0; a < 3; a++) lam_u[a] += li * d_u[a];
        }
        for (int k = 0; k < 19; k++) {
            double acc = (1.0 - omega) * lam_star[(size_t)k * ns + site] + lam_rho;
            for (int a = 0; a < 3; a++) acc += lam_u[a] * (CI[k][a] - uu[a]) / rho;
            lam_new[(size_t)k * ns + site] = acc;
        }
        for (int a = 0; a < 3; a++) {
            double acc = 0.0;
            for (int i = 0; i < 19; i++) acc += lam_star[(size_t)i * ns + site] * dS[a][i];
            lam_G[(size_t)a * ns + site] = acc;
        }
    }

    /* 4'. spread: G(x_k) -= W_k(r^n) J_p */
    double *lam_J = (double *)calloc((size_t)3 * N + 3, sizeof(double));
    double *lam_rw = (double *)calloc((size_t)3 * N + 3, sizeof(double));
    for (int i = 0; i < N; i++) {
        int nodes[8];
        double W[8], dW[8][3];
        weights_and_gradient(s, r_start + 3 * i, nodes, W, dW);
        for (int k = 0; k < 8; k++) {
            double jg = 0.0;
            for (int a = 0; a < 3; a++) {
                double lg = lam_G[(size_t)a * ns + nodes[k]];
                lam_J[3 * i + a] -= W[k] * lg;
                jg += s->J[3 * i + a] * lg;
            }
            for (int b = 0; b < 3; b++) lam_rw[3 * i + b] -= dW[k][b] * jg;
        }
    }

    /* 3'. the MD cycle */
    double *lam_up = (double *)calloc((size_t)3 * N + 3, sizeof(double));
    if (N > 0) md_cycle_adjoint(s, &rec, s->up, lam_J, lam_r, lam_v, lam_up, dpar);

    /* 2'. gather: u_p = sum_k W_k(r^n) u(x_k), u = sum_i f_i c_i / rho */
    for (int i = 0; i < N; i++) {
        int nodes[8];
        double W[8], dW[8][3];
        weights_and_gradient(s, r_start + 3 * i, nodes, W, dW);
        for (int k = 0; k < 8; k++) {
            int nd = nodes[k];
            double ug = 0.0;
            for (int a = 0; a < 3; a++) ug += s->u[(size_t)a * ns + nd] * lam_up[3 * i + a];
            for (int b = 0; b < 3; b++) lam_r[3 * i + b] += dW[k][b] * ug;
            if (W[k] == 0.0 || s->rho[nd] <= 0.0) continue;
            for (int q = 0; q < 19; q++) {
                double acc = 0.0;
                for (int a = 0; a < 3; a++)
                    acc += lam_up[3 * i + a] * (CI[q][a] - s->u[(size_t)a * ns + nd]) / s->rho[nd];
                lam_new[(size_t)q * ns + nd] += W[k] * acc;
            }
        }
    }
    for (int q = 0; q < 3 * N; q++) lam_r[q] += lam_rw[q];
    memcpy(lam_f, lam_new, sizeof(double) * 19 * (size_t)ns);

    /* leave s at the state after the step, like orc_step */
    memset(s->G, 0, sizeof(double) * 3 * ns);
    for (int i = 0; i < N; i++) {
        int nodes[8];
        double w[8];
        orc_interp_weights(s, r_start + 3 * i, nodes, w);
        for (int k = 0; k < 8; k++)
            for (int a = 0; a < 3; a++) s->G[(size_t)a * ns + nodes[k]] -= w[k] * s->J[3 * i + a];
    }
    for (int site = 0; site < ns; site++) {
        if (s->solid[site]) continue;
        double uu[3] = {s->u[site], s->u[ns + site], s->u[2 * ns + site]};
        double feq[19], S[19];
        orc_feq(s->rho[site], uu, feq);
        double Gs[3] = {s->G[site] + p->body_force[0], s->G[ns + site] + p->body_force[1],
                        s->G[2 * ns + site] + p->body_force[2]};
        orc_source(Gs, S);
        for (int i = 0; i < 19; i++) {
            double fi = s->f[(size_t)i * ns + site];
            s->fstar[(size_t)i * ns + site] = fi - omega * (fi - feq[i]) + S[i];
        }
    }
    for (size_t k = 0; k < (size_t)19 * ns; k++) s->f[k] = 0.0;
    for (int z = 0; z < p->nz; z++)
        for (int y = 0; y < p->ny; y++)
            for (int x = 0; x < p->nx; x++) {
                int site = site_of(s, x, y, z);
                if (s->solid[site]) continue;
                for (int i = 0; i < 19; i++) {
                    int dest = site_of(s, x + CI[i][0], y + CI[i][1], z + CI[i][2]);
                    double val = s->fstar[(size_t)i * ns + site];
                    if (s->solid[dest]) s->f[(size_t)opposite_of(i) * ns + site] = val;
                    else s->f[(size_t)i * ns + dest] = val;
                }
            }
    s->step += 1;

    free(r_start); free(rec.rt); free(rec.vk); free(rec.ch); free(rec.xi);
    free(lam_star); free(lam_new); free(lam_G); free(lam_J); free(lam_rw); free(lam_up);
}

int orc_adjoint(const orc_params *p, const uint8_t *solid, const double *f0, const double *r0, const double *v0,
                int64_t step0, int K, double *out, double *dr0, double *dv0, double *df0)
{
    int N = p->n_beads;
    if (N < 1 || K < 0) return -1;
    if (p->integrator != 0) return -3; /* the reverse sweep follows the velocity-Verlet cycle */
    if (p->lb_kT != 0.0) return -4;     /* and a deterministic fluid */
    orc_sim *s = orc_create(p, solid);
    size_t nf = (size_t)19 * s->ns, nb = (size_t)3 * N;
    if (f0) orc_set_populations(s, f0);
    orc_set_beads(s, r0, v0);
    orc_set_step(s, step0);
    double *fs = (double *)malloc(sizeof(double) * nf * (size_t)(K > 0 ? K : 1));
    double *rs = (double *)malloc(sizeof(double) * nb * (size_t)(K > 0 ? K : 1));
    double *vs = (double *)malloc(sizeof(double) * nb * (size_t)(K > 0 ? K : 1));
    if (!fs || !rs || !vs) { free(fs); free(rs); free(vs); orc_destroy(s); return -2; }
    double x0 = 0.0, xK = 0.0;
    for (int i = 0; i < N; i++) x0 += s->r[3 * i] / N;
    for (int n = 0; n < K; n++) {
        memcpy(fs + (size_t)n * nf, s->f, sizeof(double) * nf);
        memcpy(rs + (size_t)n * nb, s->r, sizeof(double) * nb);
        memcpy(vs + (size_t)n * nb, s->v, sizeof(double) * nb);
        one_step(s);
    }
    for (int i = 0; i < N; i++) xK += s->r[3 * i] / N;

    /* L = mean_p x_p(K) - mean_p x_p(0) */
    double *lam_f = (double *)calloc(nf, sizeof(double));
    double *lam_r = (double *)calloc(nb + 3, sizeof(double));
    double *lam_v = (double *)calloc(nb + 3, sizeof(double));
    double dpar[2] = {0.0, 0.0};
    for (int i = 0; i < N; i++) lam_r[3 * i] = 1.0 / N;
    for (int n = K - 1; n >= 0; n--) {
        memcpy(s->f, fs + (size_t)n * nf, sizeof(double) * nf);
        memcpy(s->r, rs + (size_t)n * nb, sizeof(double) * nb);
        memcpy(s->v, vs + (size_t)n * nb, sizeof(double) * nb);
        s->step = step0 + n;
        orc_step_adjoint(s, lam_f, lam_r, lam_v, dpar);
    }
    for (int i = 0; i < N; i++) lam_r[3 * i] -= 1.0 / N;
    out[0] = xK - x0;
    out[1] = dpar[0];
    out[2] = dpar[1];
    if (dr0) memcpy(dr0, lam_r, sizeof(double) * nb);
    if (dv0) memcpy(dv0, lam_v, sizeof(double) * nb);
    if (df0) memcpy(df0, lam_f, sizeof(double) * nf);
    free(fs); free(rs); free(vs); free(lam_f); free(lam_r); free(lam_v);
    orc_destroy(s);
    return 0;
}

void orc_channel_trace(orc_sim *s, int mode, int *buf, int64_t len)
{
    s->chan_mode = buf ? mode : 0;
    s->chan = buf;
    s->chan_len = buf ? len : 0;
    s->chan_pos = 0;
}

void orc_md_only(orc_sim *s, const double *up, int n)
{
    memcpy(s->up, up, sizeof(double) * 3 * s->p.n_beads);
    for (int k = 0; k < n; k++) {
        if (s->p.n_beads > 0) md_cycle(s, NULL);
        s->step += 1;
    }
}
