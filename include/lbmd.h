/*
 * lbmd.h -- C ABI of the GB300 (sm_103a) library for the coupled
 * lattice-Boltzmann / molecular-dynamics step of Fyta, Sircar, Kaxiras,
 * Melchionna, Bernaschi and Succi, "Parallel multiscale modeling of
 * biopolymer dynamics with hydrodynamic correlations".
 *
 * The problem the calls state follows Sec. IV of the paper: a periodic box
 * holding a D3Q19 BGK fluid (Sec. II, Eqs. 1-5), solid sites that reflect the
 * fluid by halfway bounce-back (the wall with a square pore), and one bead
 * chain per realization that exchanges momentum with the fluid (Sec. II,
 * Eqs. 8-13) and is driven through the pore by a local field.
 *
 * Conventions shared by every call:
 *  - Lattice units: dx = dt = 1, bead mass 1, charge 1.
 *  - Site index s = x + nx*(y + ny*z) (x fastest).  Host population arrays are
 *    [n_real][19][nz][ny][nx] float; host bead arrays are [total_beads][3]
 *    double, beads of realization r at rows bead_offsets[r] .. bead_offsets[r+1]-1.
 *  - D3Q19 link order: 0 rest; 1..6 = +x,-x,+y,-y,+z,-z; 7..18 =
 *    (1,1,0),(-1,-1,0),(1,-1,0),(-1,1,0),(1,0,1),(-1,0,-1),(1,0,-1),(-1,0,1),
 *    (0,1,1),(0,-1,-1),(0,1,-1),(0,-1,1).
 *  - Ownership: the caller allocates ONE device buffer of lbmd_required_bytes()
 *    bytes and passes it to lbmd_init; it must stay valid until lbmd_destroy.
 *    The library allocates no device memory itself.  It owns the handle, a
 *    small host state, one extra CUDA stream and a few events.
 *  - Streams: all device work is ordered on the stream given to lbmd_init.
 *    lbmd_step returns without waiting; calls that return data to the host
 *    (observables, diagnostics, get_*) synchronise that stream.
 *  - Errors: every call returns an lbmd_status and never aborts the process.
 *    lbmd_last_error() gives a one-line description of the last failure.
 *    Device-side problems (non-finite values, neighbour-list overflow) are
 *    latched in a status word that lbmd_observables / lbmd_check report.
 */
#ifndef LBMD_H
#define LBMD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LBMD_Q 19
/* Beads of one realization are integrated by one thread block. */
#define LBMD_MAX_BEADS_PER_REALIZATION 1024
/* Rows of the per-step diagnostics ring (per realization). */
#define LBMD_DIAG_RING 1024

typedef enum {
    LBMD_OK = 0,
    LBMD_ERR_INVALID_ARG = 1, /* bad configuration or argument; nothing was changed */
    LBMD_ERR_CUDA = 2,        /* a CUDA runtime call failed (message in lbmd_last_error) */
    LBMD_ERR_NONFINITE = 3,   /* a NaN/Inf appeared in the fluid or bead state */
    LBMD_ERR_TIMEOUT = 4,     /* a bounded device-side wait gave up: the tensor-copy lattice
                                 pass (tiles by = 0) waits at most 2^22 polls or 0.25 s for each
                                 stage's copies; a CTA that gives up latches this code and leaves
                                 its sites unwritten, so the state after it is not a valid step
                                 (lbmd_set_wait_probe makes such a wait run out, for tests) */
    LBMD_ERR_CAPACITY = 5,    /* a fixed-capacity list (neighbours, wall sites) overflowed */
    LBMD_ERR_BUFFER = 6       /* device buffer too small or misaligned */
} lbmd_status;

typedef enum {
    LBMD_FP32 = 0,    /* populations stored as FP32 deviations f_i - w_i */
    LBMD_FP16DEV = 1  /* populations stored as FP16 deviations (f_i - w_i) * 2^12, FP32 arithmetic */
} lbmd_precision;

/* Problem statement (Sec. IV set-up; Sec. II parameters). */
typedef struct lbmd_config {
    int32_t nx, ny, nz;      /* lattice of one realization (periodic in x, y and z) */
    int32_t n_real;          /* independent realizations (>= 1), each with its own lattice and chain */
    double tau;              /* BGK relaxation time, omega = 1/tau, nu = (tau - 1/2)/3; tau > 1/2 */
    double body_force[3];    /* uniform force density on every fluid site (0 for the paper's set-up) */
    int32_t wall_x;          /* x plane of the pore wall: defines the field channel and the
                                translocation count; -1 = none.  Solid sites come from the mask. */
    int32_t pore_h;          /* side of the square pore centred at (ny/2, nz/2) */
    double k_bond, r0;       /* harmonic bonds, Sec. II, Eq. 19 */
    double kappa_bend;       /* angular term kappa phi^2 / 2 (Sec. II) */
    double lj_sigma, lj_eps; /* bead-bead WCA (Eq. 14 cut at 2^(1/6) sigma, shifted) */
    double wall_sigma, wall_eps; /* bead-solid-site WCA */
    double E;                /* field force along +x inside the pore channel (Sec. IV) */
    double gamma;            /* bead-fluid friction (Sec. II, Eq. 12) */
    double kT;               /* bead noise temperature (Sec. II, Eq. 15); 0 = off */
    int32_t md_outer;        /* M, MD steps per LB step (paper: 5) */
    int32_t md_inner;        /* M^b, bonded sub-steps per MD step (paper: 20) */
    int32_t precision;       /* lbmd_precision */
    int32_t real_base;       /* global index of this handle's first realization (>= 0): realization r
                                draws its noise as realization real_base + r, so an ensemble split
                                over several handles (or GPUs) reproduces the unsplit one */
    uint64_t seed;           /* Philox key; global realization g uses key word 1 = seed_hi ^ g */
    int32_t interp;          /* bead-lattice transfer: 0 trilinear over the fluid corners of the
                                bead's cell; 1 nearest grid point, the paper's scheme (Sec. II) */
    int32_t integrator;      /* MD cycle: 0 multiple-time-step velocity Verlet with explicit
                                friction and noise at the half kicks; 1 stochastic position
                                Verlet (Sec. II, Eq. SPValgo) nested over the M^b sub-steps, with
                                the exact Ornstein-Uhlenbeck velocity update and fresh noise per
                                sub-step.  lbmd_adjoint needs 0 */
    double lb_kT;            /* fluctuating-LB temperature (Sec. II, the term F_i of Eq. 4): every
                                non-conserved mode of an orthogonal D3Q19 basis gets Philox noise of
                                variance 3 rho lb_kT b_k (1 - (1 - omega)^2) per site and step; 0 = off.
                                lbmd_adjoint needs 0 */
    int32_t slab_x0, slab_nx; /* slab mode (Sec. III domain decomposition, in x only): this handle
                                holds the planes [slab_x0, slab_x0 + slab_nx) of the nx x ny x nz
                                lattice, plus ghost planes; see lbmd_slab_gather.  slab_nx = 0: the
                                whole lattice (the default) */
} lbmd_config;

/* Observables of one realization at the current state (Sec. III global
 * momenta, Sec. IV.B radii of gyration, Sec. IV.C Eqs. 24-25 work rates). */
typedef struct lbmd_obs {
    double mass;              /* sum of rho over fluid sites (exact fixed-point sum of FP32 partials) */
    double p_fluid[3];        /* sum of rho u over fluid sites (likewise) */
    double p_beads[3];        /* sum of bead velocities */
    double com[3];            /* centre of mass of the chain (unwrapped) */
    double n_translocated;    /* beads with x > wall_x + 1/2 (unwrapped) */
    double dWH_dt;            /* gamma sum_i v_i . u(r_i) */
    double dWE_dt;            /* sum_i F_drive,i . v_i */
    double rg_untranslocated; /* radius of gyration of the beads not yet translocated */
    double rg_translocated;   /* radius of gyration of the translocated beads */
    int64_t step;             /* LB steps taken */
    int32_t status;           /* latched lbmd_status of the device state */
    int32_t pad;
} lbmd_obs;

/* One row of the per-step diagnostics that each step records on the device
 * at no extra pass over the lattice, for the state at the start of the step.
 * The fluid sums come from the stream-collide kernel; the bead sums from a
 * small kernel that runs beside it on the starting bead state the gather
 * kernel saves.  Every sum is a 64-bit fixed-point integer sum (exact, the
 * same in any order), converted to double at the end: mass and momentum at
 * 2^-40 per FP32 partial, bead velocities and work rates at 2^-40, positions
 * at 2^-36, squared distances at 2^-30. */
typedef struct lbmd_diag {
    int64_t step;
    double mass;
    double p_fluid[3];
    double p_beads[3];
    double com[3];
    double n_translocated;
    double dWH_dt;
    double dWE_dt;
    double rg_untranslocated; /* as in lbmd_obs, two-pass: centroid, then distances to it */
    double rg_translocated;
} lbmd_diag;

/* Translocation record of one realization (Sec. IV.A durations, Sec. IV.B
 * lambda_R = R_T(t_X) / R_U(0)).  A bead counts as translocated when its
 * unwrapped x exceeds wall_x + 1/2; "at step n" means the state step n starts
 * from (the state after n steps).  The particle kernel updates the record
 * every step, after the origin, at no extra launch. */
typedef struct lbmd_transloc {
    int64_t t_origin;        /* step at which the record was last reset */
    int64_t t_first;         /* first step >= t_origin with at least one bead translocated; -1 = none yet */
    int64_t t_x;             /* first step >= t_origin with every bead translocated; -1 = none yet */
    double rg_u_origin;      /* R_U at t_origin (-1 until that step has run) */
    double rg_t_x;           /* R_T at t_x (-1 until then) */
    double max_translocated; /* largest number of translocated beads seen at a step >= t_origin */
} lbmd_transloc;

typedef struct lbmd_kernel_time {
    char name[32];
    int64_t launches;
    double total_ms;
} lbmd_kernel_time;

typedef struct lbmd_handle lbmd_handle;

/* Bytes of device memory lbmd_init needs for this configuration.
 * bead_offsets: host array of n_real+1 CSR offsets (bead_offsets[0] = 0). */
lbmd_status lbmd_required_bytes(const lbmd_config *cfg, const int32_t *bead_offsets, size_t *bytes);

/* Set up one simulation.
 *  solid        host [nz][ny][nx] bytes, 1 = solid site (shared by all realizations)
 *  bead_offsets host [n_real+1] CSR offsets into the bead arrays
 *  r_init       host [total_beads][3] initial unwrapped bead positions; velocities start at 0
 *  device_buffer / device_bytes  caller-owned device memory (256-byte aligned)
 *  stream       cudaStream_t (as void*) that orders all work of this handle
 * The fluid starts at rest with rho = 1 (Sec. IV).  Synchronises the stream. */
lbmd_status lbmd_init(const lbmd_config *cfg, const uint8_t *solid, const int32_t *bead_offsets,
                      const double *r_init, void *device_buffer, size_t device_bytes,
                      void *stream, lbmd_handle **out);

/* Advance n_steps coupled LB-MD steps (Sec. II).  Asynchronous. */
lbmd_status lbmd_step(lbmd_handle *h, int64_t n_steps);

/* Observables of every realization at the current state: out has n_real
 * entries.  One pass over the populations; synchronises the stream. */
lbmd_status lbmd_observables(lbmd_handle *h, lbmd_obs *out);

/* Latched device status (LBMD_OK if clean); synchronises the stream. */
lbmd_status lbmd_check(lbmd_handle *h);

/* Copy the newest per-step diagnostics rows to the host: out holds
 * n_real * max_rows rows, [realization][row], oldest first; *rows receives
 * the number of rows written per realization.  Synchronises the stream. */
lbmd_status lbmd_diagnostics(lbmd_handle *h, lbmd_diag *out, int32_t max_rows, int32_t *rows);

/* Translocation records of every realization (out: n_real entries; the
 * duration of a completed event is t_x - t_origin).  Synchronises the stream. */
lbmd_status lbmd_translocation(lbmd_handle *h, lbmd_transloc *out);

/* Restart every realization's translocation record at the current step
 * (t_origin = that step, everything else "none yet").  lbmd_init does this
 * at step 0; setting beads or the step does not.  Asynchronous. */
lbmd_status lbmd_reset_translocation(lbmd_handle *h);

/* Fluid initial condition: f = f_eq(rho, u) at every fluid site.
 * rho: host [n_real][ns] or NULL (rho = 1); u: host [n_real][3][ns] or NULL (u = 0). */
lbmd_status lbmd_init_fluid(lbmd_handle *h, const double *rho, const double *u);

/* Pre-collision populations f^n (the state the next step starts from).
 * f: host [n_real][19][ns]; solid sites read as 0.  The library stores the
 * deviations h = f - w_i (Sec. II, w_i the D3Q19 weights); the conversions
 * round exactly as the FP64 expressions f = (float)((double)h + w_i) and
 * h = (float)((double)f - w_i) with w_i the double nearest the weight (then,
 * with FP16 deviation storage, h 2^12 rounded to FP16).  Synchronous: both
 * calls return once the copy is complete. */
lbmd_status lbmd_get_populations(lbmd_handle *h, float *f);
lbmd_status lbmd_set_populations(lbmd_handle *h, const float *f);
/* The same state as deviations from rest, h = f - w_i (what the library
 * stores), in FP32: accurate where the flow is weak.  Host [n_real][19][ns].
 * lbmd_set_deviations loads such a state (solid sites are ignored); with
 * FP32 storage it is stored exactly, with FP16 deviations rounded once. */
lbmd_status lbmd_get_deviations(lbmd_handle *h, float *dev);
lbmd_status lbmd_set_deviations(lbmd_handle *h, const float *dev);

/* Bead state: r unwrapped positions, v velocities; host [total_beads][3]. */
lbmd_status lbmd_get_beads(lbmd_handle *h, double *r, double *v);
lbmd_status lbmd_set_beads(lbmd_handle *h, const double *r, const double *v /* NULL: zero */);

/* Coupling of the last step: fluid velocity at each bead (frozen for the MD
 * cycle) and the momentum the fluid gave each bead; host [total_beads][3]. */
lbmd_status lbmd_get_coupling(lbmd_handle *h, float *up, float *J);

/* LB step counter; it is also the Philox counter of the bead noise, so a
 * state restored together with its step continues bit for bit. */
lbmd_status lbmd_get_step(lbmd_handle *h, int64_t *step);
lbmd_status lbmd_set_step(lbmd_handle *h, int64_t step);

/* Replay steps from a captured CUDA graph of steps_per_graph steps
 * (0 = launch kernels one by one).  Results are identical either way. */
lbmd_status lbmd_set_graph(lbmd_handle *h, int32_t steps_per_graph);

/* Advance n steps with one launch of a CUDA graph whose conditional WHILE
 * node repeats a body of two coupled steps on the device, counting the
 * bodies down in device memory: the host issues two operations for any n.
 * The graph is captured on first use and dropped with the other graphs
 * (parameter, tile, shape or overlap changes).  An odd n ends with one
 * ordinary step.  Results are identical to lbmd_step(h, n).  Needs a
 * non-default stream (LBMD_ERR_INVALID_ARG otherwise); while profiling is on
 * it runs as lbmd_step. */
lbmd_status lbmd_step_loop(lbmd_handle *h, int64_t n);

/* Launch shapes of the stream-collide kernel: block (32, by) threads, each
 * thread walking zc consecutive z planes.  by in {1,2,4,8,16}, zc in 1..64.
 * by = 0 selects the kernel fed by tensor copies (rows of x staged in shared
 * memory by cp.async.bulk.tensor), with zc in 1..256 row groups per thread
 * block; it needs nx <= 256, rows of a multiple of 16 bytes and no
 * fluctuating fluid.  by in {-1,-2,-4,-8} selects the kernel with two x
 * sites per thread (block (32, -by), 64 sites of a row per warp, pair loads
 * and stores, shuffles for the x-shifted links), zc in 1..64; it needs an
 * even nx and no fluctuating fluid.  LBMD_ERR_INVALID_ARG otherwise.  The state
 * (populations, beads) is bit-identical for every shape; the diagnostics
 * sums group their FP32 per-thread partials by shape and so agree to
 * rounding only. */
lbmd_status lbmd_set_tiles(lbmd_handle *h, int32_t by, int32_t zc);
lbmd_status lbmd_get_tiles(lbmd_handle *h, int32_t *by, int32_t *zc);

/* Shape of the particle kernel: threads_per_bead in {1,2,4,8} split each
 * bead's force terms; blocks_per_chain in 1..16 is the size C of the
 * thread-block clusters, over which the longest chain is spread (positions
 * replicated through distributed shared memory), Nc = ceil(longest / C) beads
 * per block.  A shorter chain takes ceil(N / Nc) blocks, and chains share
 * clusters.  0 = automatic.  A block may hold at most 512 threads
 * (Nc * threads_per_bead); LBMD_ERR_INVALID_ARG otherwise.  Clusters above 8
 * blocks are a non-portable size: where the device cannot schedule one, the
 * next step returns LBMD_ERR_CUDA.  The placement does not change the
 * arithmetic; other lane counts agree to rounding (the force terms are summed
 * in a different order). */
lbmd_status lbmd_set_md_shape(lbmd_handle *h, int32_t threads_per_bead, int32_t blocks_per_chain);
lbmd_status lbmd_get_md_shape(lbmd_handle *h, int32_t *threads_per_bead, int32_t *blocks_per_chain);

/* How the blocks of a chain exchange positions each MD sub-step (Sec. II,
 * Eq. 22: every sub-step's forces need the positions of the one before):
 * mode 1 push (each bead's new position is written to every block's replica
 * of the chain before the cluster barrier), 2 pull (written to its own
 * block's replica; after the barrier each block copies the other blocks' beads
 * that its force terms read, and the whole chain when the lists are rebuilt),
 * 0 leave the choice to lbmd_autotune (push until it runs).  Only chains over
 * more than one block exchange anything.  The mode does not change the
 * arithmetic: the state is bit-identical.  LBMD_ERR_INVALID_ARG for another
 * mode.  lbmd_get_md_exchange reports the mode in effect (1 or 2). */
lbmd_status lbmd_set_md_exchange(lbmd_handle *h, int32_t mode);

/* Who evaluates the bonded terms (bonds, Eq. 19, and the angular term) in
 * the particle kernel: mode 1 every bead's lanes (an angle is evaluated by
 * each of its three beads, a bond by both of its beads); 2 ceil((Nc + 2)/32)
 * extra warps per block of Nc beads, which evaluate each bond and angle once
 * while the other warps sum the pair terms; 0 automatic (2 for blocks of at
 * most 30 beads, else 1, until lbmd_autotune times both).
 * The modes add the terms in different orders, so their results agree to
 * rounding; within one mode the state does not depend on the shape's number of
 * blocks.  LBMD_ERR_INVALID_ARG for another mode, or if the extra warp would
 * take the block past 512 threads.  lbmd_get_md_bonded reports the mode in
 * effect (1 or 2). */
lbmd_status lbmd_set_md_bonded(lbmd_handle *h, int32_t mode);
lbmd_status lbmd_get_md_bonded(lbmd_handle *h, int32_t *mode);

/* 1 if the particle kernel's blocks are launched with their SMs' whole
 * shared memory (226 KB), so that no block of the lattice pass or the gather
 * shares their SMs; 0 if they take only what they use.  lbmd_set_md_reserve:
 * mode 1 do not reserve, 2 reserve, 0 leave it to lbmd_autotune (which
 * times both; until it runs, no reserving).  The state does not depend on
 * it.  LBMD_ERR_INVALID_ARG for another mode. */
lbmd_status lbmd_set_md_reserve(lbmd_handle *h, int32_t mode);

/* Test of the device-side bounded waits (failure detection without a fault):
 * with on = 1, every launch of the tensor-copy lattice pass (tiles by = 0)
 * first waits on an mbarrier phase that nothing completes, before it issues
 * any copy; the wait gives up after 1 ms, the kernel latches the timeout and
 * returns without writing its sites, and lbmd_check then returns
 * LBMD_ERR_TIMEOUT.  The step's state after such a launch is not valid.  No
 * other kernel is affected.  on = 0 (the default) turns it off;
 * LBMD_ERR_INVALID_ARG for another value. */
lbmd_status lbmd_set_wait_probe(lbmd_handle *h, int32_t on);
lbmd_status lbmd_get_md_reserve(lbmd_handle *h, int32_t *reserve);
lbmd_status lbmd_get_md_exchange(lbmd_handle *h, int32_t *mode);

/* overlap = 1 (default): the particle kernel runs concurrently with the
 * stream-collide kernel of the same step (both only read the populations the
 * step starts from); 0: one after the other.  Concurrency shares SMs between
 * a latency-bound and a bandwidth-bound kernel, which can slow both; results
 * are bit-identical either way. */
lbmd_status lbmd_set_overlap(lbmd_handle *h, int32_t overlap);
lbmd_status lbmd_get_overlap(lbmd_handle *h, int32_t *overlap);

/* Time every candidate tile shape of the stream-collide kernel on the
 * current state and keep the fastest; then, unless the caller fixed the
 * particle-kernel shape with lbmd_set_md_shape, time pseudo-steps (gather,
 * particle kernel concurrent with the lattice pass and the bead
 * diagnostics, as in a step) for every admissible
 * shape and keep the fastest: lanes per bead in {1,2,4,8}; blocks per chain in
 * {1,2,4,8,16} (16 where the device can place such a cluster); push or pull
 * exchange for more than one block, unless the caller fixed it with
 * lbmd_set_md_exchange; both bonded modes, unless fixed with
 * lbmd_set_md_bonded; with and without reserving the SMs
 * (lbmd_get_md_reserve).  The state (populations, beads, G, step, the
 * translocation records and every diagnostics row lbmd_diagnostics can
 * return) is restored afterwards.  The choice is made on the state the call
 * finds: a chain's cost changes along its path (a chain threading the pore
 * carries long wall lists), and a later call may choose differently.
 * Synchronises the stream. */
lbmd_status lbmd_autotune(lbmd_handle *h, int32_t steps_per_candidate, int32_t *by, int32_t *zc);

/* Per-kernel timing with CUDA events on the launching streams (eager launches
 * only while enabled) and the count of kernels this handle launched.  While
 * enabled, the particle kernel of realization 0 also records the SM-clock
 * cycles of its phases (load, lists, md, spread, and the list rebuilds inside
 * md, whose entry counts rebuilds as launches), reported as extra entries
 * "particles.<phase>" converted to ms at the device's nominal SM clock. */
lbmd_status lbmd_profile(lbmd_handle *h, int32_t enable);
lbmd_status lbmd_kernel_times(lbmd_handle *h, lbmd_kernel_time *out, int32_t max_entries,
                              int32_t *n_entries);
lbmd_status lbmd_launch_count(lbmd_handle *h, int64_t *launches);

/* Friction gamma (Sec. II, Eq. 12; it also sets the noise amplitude
 * sqrt(2 gamma kT / dt) of Eq. 15) and pore field E (Sec. IV) of every
 * realization, replacing the values the handle was created with.  A captured
 * step graph is dropped (it is captured again at the next lbmd_step).
 * gamma >= 0, finite E; LBMD_ERR_INVALID_ARG otherwise. */
lbmd_status lbmd_set_drive(lbmd_handle *h, double gamma, double E);

/* ---- reverse mode -------------------------------------------------------
 * Gradient of the centre-of-mass displacement of each chain along the field,
 *   L_r = mean_p x_p(K) - mean_p x_p(0)   (unwrapped x, realization r),
 * over the next K coupled steps (Sec. II, Eqs. 1-22; Sec. IV), with respect
 * to the friction gamma, the pore field E and the initial bead positions.
 * This is the exact derivative of the discrete FP32 step (discrete adjoint):
 * the pore-field indicator is piecewise constant in r and is differentiated
 * as 0; the trilinear weights have kinks on cell faces.
 *
 * Scheme: the K forward steps run from the handle's state, storing the
 * populations and bead state every checkpoint_every steps in `scratch`; then,
 * segment by segment from the last, the steps are replayed from their
 * checkpoint while the particle kernel records its trajectory, and the
 * adjoint kernels run backwards through the segment: the lattice adjoint
 * (BGK Jacobian-transpose and transposed pull with bounce-back), the bead
 * adjoint (spread, MD cycle with force Jacobian-vector products, gather; one
 * block per chain) and a fix-up of the lattice adjoint at the beads' corner
 * sites.  dL/dgamma and dL/dE are summed in FP64.
 *
 * scratch: caller-owned device memory, 256-byte aligned, at least the size
 * lbmd_adjoint_required_bytes reports (for K = 200, checkpoint_every = 20 on
 * 96x48x48: about 0.6 GB).  Outputs (host): loss, dgamma, dE [n_real];
 * dr0 [total_beads][3] (dL_r/dr0 of realization r's beads); any may be NULL.
 * On return the handle holds the state after the K steps, as lbmd_step(h, K)
 * would leave it.  Synchronises.
 *
 * Requirements (LBMD_ERR_INVALID_ARG otherwise): FP32 populations; K >= 1;
 * 1 <= checkpoint_every; every realization holds at least one bead; the
 * bead-wall cut-off 2^(1/6) wall_sigma below 2; gamma > 0 when kT > 0 (the
 * noise amplitude has no derivative at gamma = 0). */
lbmd_status lbmd_adjoint_required_bytes(const lbmd_handle *h, int32_t K, int32_t checkpoint_every,
                                        size_t *bytes);
lbmd_status lbmd_adjoint(lbmd_handle *h, int32_t K, int32_t checkpoint_every, void *scratch,
                         size_t scratch_bytes, double *loss, double *dgamma, double *dE, double *dr0);

/* ---- the random numbers of the noise ------------------------------------
 * The bead noise of Sec. II, Eq. 15 (and the fluctuating fluid of Eq. 4's
 * F_i term) draws from the counter-based generator Philox4x32-10 of Salmon,
 * Moraes, Dror and Shaw (SC'11).  These two calls expose the device
 * generator and the bead-noise mapping that the step kernels use, so that
 * both can be checked against an independent implementation.  Neither is
 * needed to run a simulation.
 *
 * lbmd_philox4x32_10: n independent draws.  ctr_key: device array [n][6] of
 * uint32 (ctr0, ctr1, ctr2, ctr3, key0, key1); out: device array [n][4] of
 * uint32, the four output words.  Asynchronous on `stream`.  n >= 0 and
 * non-null pointers when n > 0, else LBMD_ERR_INVALID_ARG.
 *
 * lbmd_noise_gauss3: the three standard normals the particle kernel draws for
 * beads bead0 .. bead0 + n - 1 of realization `realization` at LB step
 * `step` and counter word 2 = `substep` (the outer MD step, or the inner step
 * of the stochastic position Verlet cycle): key = (seed_lo, seed_hi ^
 * realization), counter = (bead, step_lo, substep, step_hi), u = (top 24 bits
 * + 1/2) 2^-24, Box-Muller in FP32.  out: device array [n][3] float.
 * Asynchronous on `stream`. */
lbmd_status lbmd_philox4x32_10(const uint32_t *ctr_key, uint32_t *out, int64_t n, void *stream);
lbmd_status lbmd_noise_gauss3(uint64_t seed, uint32_t realization, uint32_t bead0, int64_t n, int64_t step,
                              uint32_t substep, float *out, void *stream);

/* ---- one lattice over several handles: x-slabs --------------------------
 * Sec. III splits the lattice over tasks and exchanges halos for streaming.
 * Here a handle created with slab_nx > 0 holds the x-slab [slab_x0,
 * slab_x0 + slab_nx) of the nx x ny x nz lattice (periodic), every slab at
 * least 2 planes wide, n_real = 1, lb_kT = 0.  Its populations cover
 * slab_nx + 3 local planes: local plane 0 is global plane slab_x0 - 1 (a ghost
 * copy of the left neighbour's last plane), local planes 1 .. slab_nx the
 * slab, and the last two the ghost copies of the right neighbour's first two
 * planes.  lbmd_init takes the WHOLE lattice's solid mask; lbmd_get/set_
 * populations/deviations and lbmd_init_fluid address the local planes.  The
 * chain is replicated: every slab integrates all beads identically.
 *
 * One coupled step, per slab, in this order:
 *   1. lbmd_slab_gather(h): the fluid velocity u_p of every bead whose lattice
 *      cell starts in this slab (0 for the others) into io.up;
 *   2. the caller sums io.up over all slabs (each bead gets exactly one
 *      non-zero term, so the sum is exact) and writes the sum back into every
 *      slab's io.up, ordered before step 3 on the handle's stream;
 *   3. lbmd_slab_advance(h): the MD cycle, the spread onto the corners this
 *      slab owns, the lattice pass and the source, then io.send_lo (local
 *      planes 1, 2) and io.send_hi (local plane slab_nx) are filled;
 *   4. the caller copies every slab's send_lo into its left neighbour's
 *      recv_hi and its send_hi into its right neighbour's recv_lo (a single
 *      slab: into its own), ordered before step 5;
 *   5. lbmd_slab_import(h): the received planes into the ghost planes.
 * The result equals the unsplit lattice's step bit for bit.  All three calls
 * are asynchronous on the handle's stream.  The diagnostics rows hold this
 * slab's fluid sums (sum them over slabs) and the whole chain's bead sums.
 * In slab mode lbmd_step, lbmd_step_loop, lbmd_set_graph (> 0),
 * lbmd_observables and lbmd_adjoint return LBMD_ERR_INVALID_ARG; the slab
 * calls return it for a handle without slabs.
 *
 * io (from lbmd_slab_buffers): device pointers into the handle's buffer.
 * up: [total_beads][4] float (x, y, z, 0).  send_lo, recv_hi: 2 planes;
 * send_hi, recv_lo: 1 plane; a plane is [19][nz][ny] populations in the
 * storage format (FP32 deviations, or FP16 deviations x 2^12), plane_bytes
 * bytes. */
typedef struct lbmd_slab_io {
    float *up;
    void *send_lo, *send_hi, *recv_lo, *recv_hi;
    size_t plane_bytes;
} lbmd_slab_io;
lbmd_status lbmd_slab_buffers(lbmd_handle *h, lbmd_slab_io *io);
lbmd_status lbmd_slab_gather(lbmd_handle *h);
lbmd_status lbmd_slab_advance(lbmd_handle *h);
lbmd_status lbmd_slab_import(lbmd_handle *h);

/* Allocation-free fluid sums.  The paper has no counterpart: this is a
 * utility for callers that cannot allocate device memory where they call it,
 * such as a monitoring loop beside a running simulation on a GPU whose memory
 * another framework's pool already holds, or time-critical code that cannot
 * afford the device-wide synchronisation of cudaMalloc.
 *
 * Computes, for one lattice of FP32 population deviations dev = f_i - w_i
 * (device array [19][nz][ny][nx], the per-realization layout and storage
 * format of lbmd_get_deviations), out[0] = sum of rho over fluid sites and
 * out[1..3] = sum of rho u over fluid sites (device array of 4 doubles,
 * written when the kernel finishes).
 * solid: device [nz][ny][nx] bytes (1 = solid, skipped) or NULL (all fluid).
 * Asynchronous on `stream` (cudaStream_t as void*).
 *
 * It allocates nothing after its first call on a device: its per-block
 * partial sums live in one file-scope device array of about 160 KB.  CUDA
 * loads the array's module lazily (the default module loading), so the FIRST
 * call on each device loads it, which allocates the array and may
 * synchronise; the array then stays allocated until the process exits or the
 * context is reset.  A caller that cannot allocate later makes one call
 * early, before it hands the GPU's memory to a pool or starts a stream
 * capture.  Every call looks the array's device address up again with the
 * device current, so a call after cudaDeviceReset finds the new context's
 * array (reloading the module, which allocates again).  Lattices above
 * LBMD_STATIC_SUMS_MAX_SITES sites return LBMD_ERR_CAPACITY.  Every call
 * shares the array, and it keeps the last call's contents: calls whose
 * kernels overlap on the GPU race and give wrong sums; order them on one
 * stream. */
#define LBMD_STATIC_SUMS_MAX_SITES 8388608
lbmd_status lbmd_population_sums_static(const float *dev, const uint8_t *solid, int32_t nx, int32_t ny,
                                        int32_t nz, double *out, void *stream);

const char *lbmd_status_string(lbmd_status s);
const char *lbmd_last_error(const lbmd_handle *h);

/* Release the handle (not the caller's device buffer).  Synchronises. */
void lbmd_destroy(lbmd_handle *h);

#ifdef __cplusplus
}
#endif
#endif
