/*
 * dss.h -- C ABI of the GB300 dense-suspension time-step library (libdss.so).
 *
 * The library advances N rigid spheres in a sheared periodic box following
 * Monti, Rathee, Shen & Rosti, "A fast and efficient tool to study the
 * rheology of dense suspensions" (arXiv:2108.01013):
 *   - fixed-radius near-neighbour search by counting sort into cells with the
 *     symmetric half-stencil (Sec. II A, Fig. 4 and 5) and the per-particle
 *     list capacity estimated from the shell around the largest particle
 *     (Sec. II A, last paragraphs);
 *   - pair forces: lubrication (Eq. 3, App. A Eq. A2-A7) and stick-and-slide
 *     frictional contact with tangential-spring history (Eq. 4, 5);
 *   - Stokes drag (Eq. A1) and the modified velocity-Verlet update (Eq. 15)
 *     in the Lees-Edwards box (Eq. 16);
 *   - bulk stress from stresslets (Eq. 8, 9);
 *   - optionally: electro-chemical forces (Eq. 6, 7), the wavy shear flow of
 *     Eq. 17 with the Faxen term of the Stokes drag (Eq. A1), and rolling
 *     resistance between contacting particles (App. B, Eq. B1).
 *
 * Conventions: flow along x, gradient along y, vorticity along z;
 * U_inf = (gdot y, 0, 0), Omega_inf = (0, 0, -gdot/2); with the wave of
 * Eq. 17, U_inf,x = gdot y + U sin(2 pi n y / L_y) and Omega_inf, E_inf follow
 * the local rate dU_inf,x/dy.  Vector arrays are
 * SoA with three planes: v[0*n + k], v[1*n + k], v[2*n + k].
 *
 * Pointers: every array argument may be host memory (pageable or pinned) or
 * device memory of the handle's device; the library copies with
 * cudaMemcpyDefault on the handle's stream.  The caller owns every buffer it
 * passes; the library owns its internal state, cell, list, history and pair
 * buffers, allocated in dss_create (and re-allocated when a pair-capacity
 * overflow is recovered, see dss_step).
 *
 * Particle order: ids passed to dss_set_state must be a permutation of
 * 0..n-1 (NULL means k -> k).  Every per-particle output is written in id
 * order (entry id), whatever order the library keeps internally.
 *
 * Errors: every int-returning call returns DSS_OK (0) or a negative code;
 * dss_strerror gives a message.  No call aborts, traps or waits without a
 * bound on the device.  After DSS_ERR_CUDA the handle should be destroyed.
 */
#ifndef DSS_H_
#define DSS_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum dss_status {
  DSS_OK = 0,
  DSS_ERR_ARG = -1,        /* bad argument (NULL, size, range, ids not a permutation) */
  DSS_ERR_BOX = -2,        /* box too small: < 3 cells per axis (4 along x) */
  DSS_ERR_CAPACITY = -3,   /* a particle exceeded the list capacity M; step not committed */
  DSS_ERR_NONFINITE = -4,  /* non-finite force or state; step not committed */
  DSS_ERR_UNSTABLE = -5,   /* dt above the explicit stability estimate (dss_create, strict only) */
  DSS_ERR_CUDA = -6,       /* CUDA runtime error */
  DSS_ERR_TIMEOUT = -7,    /* a bounded device-side wait gave up */
  DSS_ERR_STATE = -8,      /* call order (e.g. dss_step before dss_set_state) */
  DSS_ERR_INTERNAL = -9,   /* internal consistency check failed on the device */
  DSS_ERR_SCRATCH_LIMIT = -10, /* dss_pairs_noalloc: problem larger than its fixed scratch array */
  DSS_ERR_NOMEM = -11          /* a host-side allocation inside the call failed */
};

enum dss_precision {
  DSS_FP64 = 0,   /* everything in FP64 */
  DSS_MIXED = 1   /* pair forces in FP32; positions, gaps, Lees-Edwards offset
                     and stress accumulation in FP64 or double-float (two FP32
                     words, ~48 bits); tangential stretch as double-float */
};

typedef struct dss_params {
  double kn, kt, gamma_n, mu;   /* Eq. 4-5: normal and tangential spring, dashpot, Coulomb */
  double eta0, rho;             /* fluid viscosity; particle density (m = 4/3 pi rho a^3) */
  double delta_lub, lub_eps;    /* lubrication range, regulariser eps of Eq. A6 */
  double a0;                    /* reference radius (cutoff mode 1) */
  int32_t lub_cutoff_mode;      /* 0: pair listed iff d* = 2d/(a_i+a_j) < delta_lub;
                                   1: iff d < delta_lub*a0 (d = surface gap) */
  int32_t precision;            /* enum dss_precision */
  double shear_rate, dt;        /* gdot, time step */
  double cell_size;             /* 0: smallest size >= largest interaction range */
  int32_t capacity_M;           /* half-list capacity per particle; 0: Sec. II A estimate */
  int32_t pair_capacity;        /* mean half-list pairs per particle to allocate for; 0: 16 */
  double lub_taper;             /* w in [0, 1): lubrication scaled by s = t^2 (3 - 2t),
                                   t = clamp((delta_ij - d) / (w delta_ij), 0, 1), so it
                                   vanishes continuously at the cutoff (an extension for
                                   differentiation, not in the paper); 0: hard cutoff */
  int32_t cell_mode;            /* 0: cells >= 2 a_max + delta_max, one list (Sec. II A);
                                   1: smaller cells, particles binned by size class, larger
                                   classes search larger stencils (Sec. II A, for highly
                                   polydisperse suspensions); cell_size 0: auto */
  int32_t reserved_;
  double f_er;                  /* Eq. 6: double-layer repulsion -F_ER (abar/a0) exp(-d/lambda_D) n,
                                   acting below d = 20 lambda_D (Fig. 3); 0: off */
  double lambda_d;              /* Debye length lambda_D (> 0 when f_er > 0) */
  double hamaker;               /* Eq. 7: van der Waals attraction A abar / (12 (d^2 + eps^2)) n,
                                   acting below d = 4 a0 (Fig. 3); 0: off */
  double vdw_eps;               /* eps / abar of Eq. 7 (> 0 when hamaker > 0).  Pairs are
                                   listed out to the larger of the lubrication and
                                   electro-chemical ranges; lubrication acts within its own
                                   range only.  abar = 2 a_i a_j / (a_i + a_j) */
  double wave_amp;              /* Eq. 17: amplitude U of the wave added to U_inf,x,
                                   U sin(2 pi wave_n y / L_y) (L_y of each instance).  The
                                   Stokes drag then takes the Faxen velocity
                                   (1 + a^2/6 Laplacian) U_inf and the local Omega_inf at the
                                   centre (Eq. A1); lubrication takes the velocities relative
                                   to the flow at each centre and the strain of the mean of
                                   the two centres' local rates; a particle's stresslet takes
                                   the strain at its centre.  0: simple shear */
  double k_r;                   /* App. B: rolling spring stiffness (k_r << k_n).  A contact
                                   then also carries a rolling stretch xi_r integrating
                                   u_r = abar (n x w_i - n x w_j) under the Coulomb limit
                                   |k_r xi_r| <= mu |F_nor| (Eq. 5 with k_r for k_t); it adds
                                   the torques abar n x (k_r xi_r) on i and its opposite on j,
                                   no force and no stresslet.  0: off */
  int32_t wave_n;               /* Eq. 17: whole number n >= 0 of wave periods along L_y
                                   (the wave stays periodic under Lees-Edwards); 0: no wave */
  int32_t reserved2_;           /* 0 */
} dss_params;

typedef struct dss_handle dss_handle;

/* Counters of the last force evaluation (dss_get_counters). */
typedef struct dss_counters {
  int64_t steps_done;       /* committed time steps since dss_set_state */
  int64_t nstep;            /* time = nstep * dt */
  int64_t npairs;           /* listed half pairs */
  int64_t ncontacts;        /* pairs with d < 0 */
  int64_t max_row;          /* largest half-list row */
  int64_t band_checks;      /* candidates decided by the exact FP64 predicate */
  int32_t M, pad_;
  int64_t ncell[3];
} dss_counters;

/* Half-list capacity M from the shell estimate of Sec. II A: the number of
 * smallest spheres (radius a_min) whose volume fits in the shell of
 * thickness 2*a0 around the largest sphere (radius a_max),
 * ceil(((a_max + 2 a0)^3 - a_max^3) / a_min^3).  Host-only, needs no GPU.
 * Returns -1 for non-positive radii. */
int32_t dss_capacity_estimate(double a_min, double a_max, double a0);

/* Creates a handle for n particles in the box (edges box[0..2]) on the
 * current CUDA device.  Work is issued on cuda_stream (a cudaStream_t); when
 * it is NULL (the legacy default stream, on which CUDA graphs cannot be
 * captured) the library issues its work on a stream of its own, ordered after
 * the legacy stream at every call.  Validates the parameters and the cell
 * grid (needs >= 4 cells along x and >= 3 along y and z; the cutoff must be
 * below half of every edge).  The radius range used for the cell size and
 * M is fixed by dss_set_state; dss_create only stores the parameters.
 * On success *h receives the handle. */
int dss_create(dss_handle **h, const dss_params *p, int64_t n, const double box[3],
               void *cuda_stream);

/* Batch of K independent suspensions in one handle (the flow-curve sweep of
 * Sec. IV runs one suspension per shear rate; here they share every launch).
 * Instance k has n[k] particles (n[k] >= DSS_BATCH_MIN_N when K > 1), box
 * edges box[3k..3k+2], shear rate shear_rate[k] and normal dashpot
 * gamma_n[k] (gamma_n NULL: p->gamma_n for all); p->shear_rate and
 * p->gamma_n are otherwise ignored, every other parameter (contact,
 * lubrication, dt, precision) is shared.  Particles are numbered
 * instance-major: instance k holds indices and ids
 * [n[0]+...+n[k-1], n[0]+...+n[k]).  Every other entry point applies to the
 * concatenated system: dss_set_state takes the concatenated arrays (ids of
 * instance k a permutation of its own range), dss_step advances all
 * instances together, one CUDA graph per step for the whole batch.  The
 * instances do not interact; each has its own cell grid and Lees-Edwards
 * offset.  All pointers are host memory.  dss_create is the case K = 1. */
#define DSS_BATCH_MIN_N 256
int dss_batch_create(dss_handle **h, const dss_params *p, int32_t K, const int64_t *n,
                     const double *box, const double *shear_rate, const double *gamma_n,
                     void *cuda_stream);

/* Number of instances of the handle (0 for NULL). */
int32_t dss_batch_size(const dss_handle *h);

/* Stress of every instance (Eq. 8, row-major 3x3 each): sigma[9K] at the
 * last force evaluation, and sigma_mean[9K] = the mean over the steps
 * committed by dss_step since dss_set_state or the last reset (*steps
 * receives their number; the mean is 0 when none).  Any of sigma,
 * sigma_mean, steps may be NULL; reset != 0 restarts the mean after
 * reading it.  Host or device pointers; synchronises the stream. */
int dss_batch_stress(dss_handle *h, double *sigma, double *sigma_mean, int64_t *steps, int reset);

/* Loads the state: x (3n, inside [0, L) on every axis), radii a (n, > 0),
 * ids (n, permutation of 0..n-1, or NULL), velocity u (3n, NULL: U_inf(x)),
 * angular velocity w (3n, NULL: Omega_inf), accelerations alpha_lin,
 * alpha_ang (3n each; when both are NULL they are computed by one force
 * evaluation at the loaded state, with an empty contact history), and the
 * step count nstep (time nstep*dt).  Clears the contact history.  Sizes the
 * cell grid and the list capacity for the radii on the first call
 * (DSS_ERR_BOX / DSS_ERR_CAPACITY when they do not fit). */
int dss_set_state(dss_handle *h, const double *x, const double *a, const int32_t *ids,
                  const double *u, const double *w, const double *alpha_lin,
                  const double *alpha_ang, int64_t nstep);

/* Replaces the dynamic state of the particles loaded by dss_set_state,
 * keeping their radii, the contact history and the time: x, u, w, alpha_lin,
 * alpha_ang (3n each, id order, all required).  No validation and no force
 * evaluation: this is the per-step upload of a caller that keeps the state
 * in its own (host or device) memory.  Stream-ordered, does not synchronise. */
int dss_load_state(dss_handle *h, const double *x, const double *u, const double *w,
                   const double *alpha_lin, const double *alpha_ang);

/* One step loop of a caller that keeps the state in its own memory: loads
 * x, u, w, alpha_lin, alpha_ang (in[0..4], 3n each, id order, all required,
 * as dss_load_state), advances nsteps steps (Eq. 15-16, as dss_step), writes
 * the state after them to out[0..4] (id order; any entry may be NULL, as
 * dss_get_state) and the last stress to sigma (9 values, or NULL; instance
 * 0).  Host (pinned or pageable) or device pointers; in and out may be the
 * same buffers.  The upload, the step graphs, the download and the stress
 * read are issued back to back and the stream is synchronised once; a step
 * that fails on the pair capacity is recovered as by dss_step.  Errors as
 * dss_step. */
int dss_step_io(dss_handle *h, const double *const in[5], int64_t nsteps, double *const out[5],
                double sigma[9]);

/* Copies the current state out in id order; any pointer may be NULL. */
int dss_get_state(dss_handle *h, double *x, double *u, double *w, double *alpha_lin,
                  double *alpha_ang);

/* Replaces the contact history: k entries with keys (lo_id << 32 | hi_id)
 * and tangential stretch xi (3 per entry, row-major [k][3], orientation
 * lo -> hi).  Used to resume from a checkpoint.  The rolling stretch of
 * every entry (App. B) is set to zero. */
int dss_set_history(dss_handle *h, int64_t k, const int64_t *keys, const double *xi);

/* Copies the committed contact history out, sorted by key.  Writes up to
 * cap entries; *count receives the number of entries. */
int dss_get_history(dss_handle *h, int64_t *keys, double *xi, int64_t cap, int64_t *count);

/* The same with the rolling stretch of App. B: xr (row-major [k][3]; it does
 * not depend on the orientation of the pair) may be NULL (zero), and is kept
 * only when k_r > 0; dss_get_history_rolling writes zeros when k_r = 0. */
int dss_set_history_rolling(dss_handle *h, int64_t k, const int64_t *keys, const double *xi,
                            const double *xr);
int dss_get_history_rolling(dss_handle *h, int64_t *keys, double *xi, double *xr, int64_t cap,
                            int64_t *count);

/* Counting sort and half-stencil enumeration at the current state (no time
 * advance).  The pairs can then be read with dss_get_pairs. */
int dss_neighbour_build(dss_handle *h);

/* Pairs of the last neighbour build / force evaluation as (lo id, hi id),
 * row-major [count][2], sorted lexicographically.  Writes up to cap pairs;
 * *count receives the total.  Synchronises the stream. */
int dss_get_pairs(dss_handle *h, int64_t *lohi, int64_t cap, int64_t *count);

/* One force evaluation at the current state with the committed history,
 * without advancing or committing: total force F and torque T on every
 * particle (pairs + Stokes drag), in id order; either may be NULL.  Also
 * sets the stress read by dss_stress. */
int dss_force_eval(dss_handle *h, double *F, double *T);

/* Advances nsteps time steps (Eq. 15, 16): predictor and wrap, counting
 * sort, half-stencil enumeration, history carry, pair forces, symmetric
 * deterministic accumulation, drag, corrector, stress.  Steps run as CUDA
 * graph replays; the host synchronises once at the end.  When a step fails
 * (capacity, non-finite, timeout) it is not committed, later steps do
 * nothing, and the state stays at the last committed step; a pair-capacity
 * overflow is recovered by growing the pair buffers and resuming. */
int dss_step(dss_handle *h, int64_t nsteps);

/* Bulk stress of the last force evaluation (Eq. 8), row-major 3x3, host
 * memory (instance 0 of a batch).  Synchronises the stream. */
int dss_stress(dss_handle *h, double sigma[9]);

/* Counters of the last force evaluation (synchronises). */
int dss_get_counters(dss_handle *h, dss_counters *c);

/* Per-kernel timing of dss_step.  When on, the captured step records a CUDA
 * event before each of its DSS_PROF_KERNELS kernels (and after the last) on
 * the work stream; dss_step then synchronises after every step and adds each
 * kernel's event-to-event time to a running sum.  Turning it on or off
 * resets the sums and re-captures the step. */
#define DSS_PROF_KERNELS 7
int dss_set_profiling(dss_handle *h, int on);

/* Running per-kernel sums in milliseconds (ms[DSS_PROF_KERNELS]) and the
 * number of profiled steps. */
int dss_get_profile(dss_handle *h, double *ms, int64_t *steps);

/* Name of profiled kernel k (0 <= k < DSS_PROF_KERNELS), "" otherwise. */
const char *dss_profile_name(int k);

/* GPU time in milliseconds of the step graphs of the last dss_step call
 * (CUDA events recorded on the work stream just before the first and just
 * after the last graph launch; no per-kernel events). */
int dss_last_step_ms(dss_handle *h, double *ms);

/* Checkpoint of the whole dynamic state: positions, velocities, angular
 * velocities and both accelerations (id order), radii, the contact history
 * (keys, tangential stretch and, when k_r > 0, rolling stretch), the step count, the last stress and the
 * running stress sums of every instance.  With buf == NULL, *len receives the
 * size needed; otherwise buf (host memory, *len bytes) receives the
 * checkpoint and *len its size (DSS_ERR_ARG, with *len set, when too small).
 * Synchronises the stream. */
int dss_save(dss_handle *h, void *buf, size_t *len);

/* Restores a checkpoint written by dss_save into a handle created with the
 * same instances, boxes, shear rates, dashpots and model constants
 * (DSS_ERR_ARG otherwise, or for a damaged buffer).  Because the library's
 * sorted order depends only on positions and ids, the resumed run repeats the
 * uninterrupted one bit for bit.  Synchronises the stream. */
int dss_load(dss_handle *h, const void *buf, size_t len);

/* Chooses the cell edge from timed trials.  Candidate k uses a cell edge of
 * factors[k] (>= 1) times the smallest admissible one, 2 a_max + delta_max
 * (Sec. II A); factors == NULL with ncand == 0 tries 1.0, 1.1, 1.25, 1.5.
 * Each candidate rebuilds the grid, runs 2 untimed and trial_steps timed
 * steps (GPU time of the step graphs) from the state at the call, and
 * writes its ms per step to ms_per_step[k] (may be NULL; INFINITY for a
 * grid the box does not admit).  The fastest edge is kept (*cell_size, may
 * be NULL) and the state at the call is restored exactly (dss_save /
 * dss_load), so the trials leave no trace in the trajectory.  ncand <= 16. */
int dss_autotune(dss_handle *h, int32_t trial_steps, int32_t ncand, const double *factors,
                 double *ms_per_step, double *cell_size);

/* Kernel shapes (the tile parameters of the step; north star: "tile shape
 * picked by an autotuner"), timed at the current cell grid: the register
 * budget of the pair kernel (cut for 3 or 4 resident 256-thread blocks per
 * SM: 80 or 64 registers; more warps in flight against more spills) and the
 * enumeration's candidate loop (one candidate at a time, or screened: four
 * loaded ahead and rejected by one test into a bit mask, the rest decided
 * afterwards in order).  Each of the 4 combinations runs 2 + trial_steps
 * steps from a checkpoint of the current state; the fastest is kept and the
 * state restored.  ms_per_step (host, 4 doubles, may be NULL): ms per step of
 * (3 blocks, 1), (3, 4), (4, 1), (4, 4); choice (host, 2 ints, may be NULL):
 * the kept (blocks per SM, candidate loop: 1 plain, 4 screened).  Errors: DSS_ERR_ARG
 * (trial_steps < 1), DSS_ERR_STATE, and any error of a trial step (the
 * built-in rule is kept then). */
int dss_autotune_kernels(dss_handle *h, int32_t trial_steps, double *ms_per_step, int32_t *choice);

/* Gradient of a stress functional of a rollout (reverse mode).  Runs nsteps
 * steps from the current state (as dss_step would), with
 *     J = sum_{n=1..nsteps} sum_q weights[(n-1)*9 + q] * sigma^n_q
 * (sigma^n: the bulk stress of Eq. 8 after step n, row major; weights are
 * host or device memory, [nsteps][9]; e.g. e_xy / (nsteps eta0 gdot) gives
 * the time-averaged relative viscosity), and returns J and its derivatives
 * with respect to the model constants, dJ_dparams[5] = (k_n, k_t, gamma_n,
 * mu, delta_lub) (partials: a caller tying k_t = k_n/2 adds them up), and to
 * the initial state in id order: positions, velocities, angular velocities
 * (3n each) and, unless initial_forces, the initial accelerations.  With
 * initial_forces != 0 the initial accelerations are taken to be those of a
 * force evaluation at the initial state with an empty contact history (what
 * dss_set_state computes when given none), and their dependence is folded
 * into the other derivatives (dJ_dalpha0/beta0 then return zero).
 * The forward keeps a device copy of the committed state (state, history
 * list and stretch records, status words, stresses) every ckpt_every steps
 * and sums J on the device; the reverse sweep restores one segment's copy at
 * a time, replays it taping each step, and walks it backwards: device memory
 * is one segment of tapes plus the copies (~ (160 + 4 M) B per particle and
 * 32 B per pair, 64 with rolling, each; DSS_ERR_CUDA when they do not fit).
 * A step of the forward that fails on the pair capacity is recovered as by
 * dss_step.
 * Derivatives are pathwise: the pair set, contacts, Coulomb slips (of the
 * sliding and, with k_r > 0, the rolling spring) and the taper ends of each
 * step are those of the forward run and held fixed; with the hard cutoff
 * (lub_taper = 0) J has no pathwise dependence on delta_lub.  The wavy shear
 * flow of Eq. 17 (its y dependence in the ambient flow, the pair strain, the
 * Faxen drag and the local stresslets) and rolling resistance (App. B; the
 * rolling stretch carried like the sliding one; k_r itself is not among the
 * parameters) are differentiated.  Single-instance handles only
 * (DSS_ERR_ARG otherwise).  The handle is left
 * in the state after the rollout.  Output pointers are host or device
 * memory and may be NULL.  Synchronises the stream. */
int dss_adjoint(dss_handle *h, int64_t nsteps, int32_t ckpt_every, const double *weights,
                int32_t initial_forces, double *J, double *dJ_dparams, double *dJ_dx0,
                double *dJ_du0, double *dJ_dw0, double *dJ_dalpha0, double *dJ_dbeta0);

/* Self-test of the bounded device waits (failure detection without a GPU
 * fault): runs one warp of the decoupled look-back used by the scans on a
 * predecessor that never publishes.  The wait gives up after its time limit
 * (0.5 s) and records DSS_ERR_TIMEOUT, which this call returns (DSS_OK would
 * mean the wait did not notice).  The context stays usable.  cuda_stream:
 * stream to run on (NULL: legacy default stream); synchronises it. */
int dss_selftest_bounded_wait(void *cuda_stream);

/* Self-test of the conversions the sort kernels take by integer operations
 * on the IEEE-754 bit patterns instead of GB300's narrow FP64 pipe; each must
 * equal the hardware conversion bit for bit.  For k < n: hi[k] =
 * RN_f32(v[k]); (split_hi[k], split_lo[k]) = (RN_f32(v[k]),
 * RN_f32(v[k] - split_hi[k])) (the double-float split); back[k] =
 * (double)hi[k]; floor_out[k] = floor(RN_f64(v[k] * inv)) (the cell
 * coordinate, int, for |v[k] inv| < 2^31); ints_out[k] = (double)ints[k]
 * (ints[k] >= 0).  All arrays device memory of n elements.  DSS_ERR_ARG for
 * n < 0 or a NULL array; DSS_ERR_CUDA on a launch failure.  cuda_stream:
 * stream to run on (NULL: legacy default stream); synchronises it. */
int dss_selftest_conversions(const double *v, int64_t n, double inv, float *hi, float *split_hi,
                             float *split_lo, double *back, int32_t *floor_out, const int32_t *ints,
                             double *ints_out, void *cuda_stream);

/* ---- Analysis pass (not part of the time step; each call synchronises) ---- */

/* Rheology of every instance from its bulk stress (Sec. II, after Eq. 9):
 * out[6k .. 6k+5] = {sigma = S_xy, N1 = S_xx - S_yy, N2 = S_yy - S_zz,
 * Pi = -tr(S)/3, eta_r = sigma / (eta0 gdot_k), eta_n = Pi / (eta0 gdot_k)},
 * from the running mean of the committed steps (mean != 0, as dss_batch_stress
 * returns it) or from the last force evaluation (mean == 0).  out: 6K doubles,
 * host or device.  DSS_ERR_ARG for a zero shear rate or eta0. */
int dss_rheology(dss_handle *h, int mean, double *out);

/* Lees-Edwards image count along y of every particle, by id: how many times
 * it left through y = L_y minus how many times through y = 0 since the state
 * was set (dss_set_state, dss_load_state and dss_load restart it at 0); the
 * unwrapped shear-wise coordinate is y + count L_y.  iy: n int32, host or
 * device. */
int dss_get_images(dss_handle *h, int32_t *iy);

/* Shear-wise dispersion (Sec. III B, Eq. 18-19).  dss_dispersion_mark records
 * the current time t0, and the unwrapped y and the shear-wise velocity
 * fluctuation v' = u_y of every particle.  dss_dispersion then returns, per
 * instance k, out[3k .. 3k+2] = {D_y = <(y(t) - y(t0))^2> / (2 (t - t0)) /
 * (a0^2 gdot_k), C_v = <v'(t) v'(t0)> / <v'(t)^2>, t - t0}, the averages over
 * the instance's particles (D_y = 0 at t = t0).  out: 3K doubles, host or
 * device.  DSS_ERR_STATE before a mark, or after the state was set again. */
int dss_dispersion_mark(dss_handle *h);
int dss_dispersion(dss_handle *h, double *out);

/* Clusters of contacting particles (Sec. III A, Fig. 10-11): the connected
 * components of the graph whose edges are the pairs in contact (d < 0) at
 * the last committed step (or the history set by dss_set_history).  label:
 * n int32 by id (host or device, may be NULL), the smallest id in the
 * particle's cluster; *nclusters: the number of clusters (a particle without
 * contact is a cluster of one).  The result is unique (no dependence on
 * thread order). */
int dss_contact_clusters(dss_handle *h, int32_t *label, int64_t *nclusters);

/* Local volume fraction along the shear-wise direction y by size class
 * (Sec. III B, Fig. 12: the distribution of the large and of the small
 * particles across the gradient direction, whose peaks show the large
 * particles migrating to the zero-shear planes of the wavy flow).  The box
 * of each instance is cut into nbins slabs of equal width along y; for each
 * slab and class, out holds the volume of the class's spheres inside the
 * slab (each sphere's exact integral of its cross-sections over the slab,
 * its periodic images across y = 0 and y = L_y included) divided by the
 * slab's volume.  Class 0: radius <= a_split, class 1: radius > a_split.
 * The mean over the slabs of a class is that class's volume fraction.  At
 * the committed state; averaging over snapshots is the caller's.  out: K x 2
 * x nbins doubles (instance-major, then class, then slab), host or device.
 * Deterministic (integer sums in a unit of 2^-62 of the instance's solid
 * volume).  Errors: DSS_ERR_ARG (nbins < 1 or > 2^20, a_split not finite),
 * DSS_ERR_STATE, DSS_ERR_CUDA. */
int dss_phi_profile(dss_handle *h, int32_t nbins, double a_split, double *out);

/* Bytes of device memory the handle holds. */
int64_t dss_device_bytes(const dss_handle *h);

void dss_destroy(dss_handle *h);
const char *dss_strerror(int code);

/* ---- Neighbour pairs without any device allocation ----------------------
 * The paper has no counterpart of this entry point.  It exists for callers
 * that may not allocate GPU memory themselves or through us: code embedded in
 * a host application that owns every device allocation (a plugin inside
 * another framework's memory pool), or a process whose device memory is
 * fully reserved in advance.  Every other entry point allocates its buffers
 * in dss_create / dss_set_state; this one calls no cudaMalloc, cudaFree or
 * allocating library routine.
 *
 * It computes the same pair set as dss_neighbour_build + dss_get_pairs for
 * the state (x, a, ids) at time nstep*dt, with the parameters p: every pair
 * with r^2 < (a_i + a_j + delta_ij)^2 under Lees-Edwards minimum images, where
 * delta_ij is the larger of the lubrication range (delta_lub, a0,
 * lub_cutoff_mode) and the electro-chemical range (f_er, lambda_d, hamaker,
 * a0: 20 lambda_d and 4 a0 while the respective force is on); shear_rate and
 * dt set the Lees-Edwards offset; the other fields are not read.  Pairs are
 * written as (lo id, hi id) into pairs[2*k], pairs[2*k+1] in no particular
 * order.
 *
 * Arguments: x (3n, SoA, inside [0, L)), a (n), ids (n, or NULL for k -> k)
 * and pairs (2*cap int64) are DEVICE memory of the current device; box,
 * p and count are host memory.  a_max must bound every radius from above
 * (it sets the cell size; a larger radius returns DSS_ERR_ARG).  *count
 * receives the number of pairs; at most cap are written.  The call is
 * ordered on cuda_stream (NULL: legacy stream) and synchronises it.
 *
 * Errors: DSS_ERR_ARG (NULL pointer, n < 2, a non-positive box edge or
 * a_max, nstep < 0, an unknown cutoff mode, a radius above a_max),
 * DSS_ERR_BOX (fewer than 4 x 3 x 3 cells of that edge fit in the box),
 * DSS_ERR_SCRATCH_LIMIT (below), DSS_ERR_CUDA.
 *
 * Working memory: one file-scope __device__ array of DSS_NOALLOC_SCRATCH_INTS
 * 32-bit words (8 MiB), which every GPU that loads the library holds until
 * the process exits.  A problem needs n + 3*cells + 17 words (cells: the
 * cell grid of edge >= 2 a_max + max delta_ij); larger problems are rejected
 * with DSS_ERR_SCRATCH_LIMIT.  All calls share the array and each call clears
 * what it needs at its start, so calls whose GPU work overlaps (on different
 * streams, or from several host threads) race and must be serialised by the
 * caller.  The first call on each device looks up the array's device
 * address (cudaGetSymbolAddress, with that device current); make that first
 * call outside any stream capture. */
#define DSS_NOALLOC_SCRATCH_INTS (1 << 21)
int dss_pairs_noalloc(const double *x, const double *a, const int32_t *ids, int64_t n,
                      const double box[3], const dss_params *p, double a_max, int64_t nstep,
                      int64_t *pairs, int64_t cap, int64_t *count, void *cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* DSS_H_ */
