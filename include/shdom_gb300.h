/*
 * shdom_gb300.h -- C ABI of the GB300 (sm_103a) library for one source
 * iteration per time step of the time-dependent, multi-group, mixed-frame
 * SHDOM method (Tominaga, Shibata & Blinnikov, arXiv:1507.05141).
 *
 * One step (Sec. 2, Sec. 2.2 frame order) runs, on the GPU:
 *   a1  project   laboratory intensity -> comoving ordinates/groups (Lorentz,
 *                 eq:lorentzfreq, eq:lorentzray, I/nu^3 invariant) -> real
 *                 spherical harmonics I_lm (Sec. 2.3); laboratory moments J,
 *                 H_i, K_ij (the Eddington tensor f_ij = K_ij / J);
 *   a2  source    S_lm = n_e/chi0 sum_g' K_l[g][g'] I_lm(g') + T_lm
 *                 (Sec. 2.3: Thomson / Klein-Nishina, eq:comptoncross);
 *   a3  sh2lab    S_lm -> comoving ordinates -> laboratory eta, chi
 *                 (eta/nu^2, chi nu invariant; Sec. 2.2);
 *   a4  sweep     short-characteristic transfer along every laboratory
 *                 ordinate and group with the time term chi~ = chi + 1/(c dt),
 *                 eta~ = eta + I^n/(c dt)  (Sec. 2 eq:shdom, Sec. 2.1 eq:time);
 *   a5  sums      FP64 energy, photon number and relative source change.
 *
 * Conventions (every entry point):
 *   - Return SHD_OK (0) on success, a negative SHD_ERR_* code otherwise; the
 *     message of the last failure on the calling thread is shd_last_error().
 *   - Host pointers are caller-owned; the library copies what it needs before
 *     returning.  Device state is library-owned and freed by shd_destroy().
 *   - Node index c = (iz*ny + iy)*nx + ix; node spacing h_a = l_a/(n_a - 1)
 *     (nodes on the faces).
 *   - Ordinate index k = a*n_phi + b: mu_a ascending Gauss-Legendre, phi_b =
 *     2 pi b / n_phi from +x towards +y; weights sum to 4 pi.
 *   - Spherical-harmonic index p = l*l + l + m, real orthonormal, no
 *     Condon-Shortley phase, all l <= L.
 *   - Host intensity arrays are [c][g][k] (double); SH arrays [c][g][p].
 *   - Energies are in units of m_e c^2; group g spans [edges[g], edges[g+1]],
 *     its specific intensity is taken at the centre sqrt(e_g e_{g+1}).
 *   - A context is not thread-safe; distinct contexts are independent.
 *   - Setters validate their arguments before touching the GPU.  A setter
 *     that changes sizes (grid, angles, groups) discards the fields, state
 *     and scattering table that depended on them.
 */
#ifndef SHDOM_GB300_H
#define SHDOM_GB300_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct shd_ctx shd_ctx;

enum shd_status {
    SHD_OK = 0,
    SHD_ERR_ARG = -1,     /* invalid argument or call order            */
    SHD_ERR_OOM = -2,     /* device or host allocation failed          */
    SHD_ERR_CUDA = -3,    /* a CUDA runtime call or kernel failed      */
    SHD_ERR_STATE = -4,   /* context not fully configured              */
    SHD_ERR_NAN = -5,     /* non-finite or out-of-range input rejected */
    SHD_ERR_TIMEOUT = -6  /* iteration limit reached without converging */
};

enum shd_precision {
    SHD_FP64 = 0,  /* every stage in FP64 (parity path)                       */
    SHD_FP32 = 1,  /* every stage in FP32 ("plain FP32")                      */
    SHD_MIXED = 2  /* FP32 transfer; FP64 where stability needs it             */
};

enum shd_scattering {
    SHD_SCAT_ISO = 1,      /* isotropic: K_0 = 1, sigma_out = 1                 */
    SHD_SCAT_THOMSON = 2,  /* Thomson: K_0 = 1, K_2 = 1/10, sigma_out = 1       */
    SHD_SCAT_KN = 3,       /* cold-electron Klein-Nishina multigroup kernel,
                              built on the GPU from the group edges            */
    SHD_SCAT_TABLE = 4,    /* caller-supplied K[l][g][g'] and sigma_out[g']     */
    SHD_SCAT_KN_THERMAL = 5 /* Compton scattering off thermal electrons at each
                              node's temperature theta_e (shd_set_fields):
                              shd_set_scattering tabulates the kernel on the
                              grid theta_i = 10^(-3 + i/4), i = 0..12, and each
                              node blends its two bracketing tables linearly
                              in log10(theta) (clamped into the grid)        */
};

enum shd_time_scheme {
    SHD_TIME_EULER = 0,  /* one backward-Euler source iteration per step (Sec. 2.1) */
    SHD_TIME_RK4 = 1     /* four sub-solves combined as in App. A, eq:rk4th        */
};

enum shd_integrator {
    SHD_SC_LINEAR = 0,  /* source linear in optical depth along the segment    */
    SHD_SC_BEZIER = 1   /* cubic Bezier source (Sec. 2, the paper's scheme)     */
};

enum shd_boundary {
    SHD_BC_VACUUM = 0,  /* inflow intensity 0                                  */
    SHD_BC_ISO = 1,     /* inflow intensity data[g], same for every ordinate   */
    SHD_BC_FULL = 2     /* inflow intensity data[c][g][k] (only inflow-face
                           nodes are read)                                     */
};

/* Create a context on CUDA device `device` computing in `precision`
 * (enum shd_precision).  *out receives an opaque handle. */
int shd_create(shd_ctx **out, int device, int precision);

/* Free every device and host resource of ctx (NULL is ignored). */
void shd_destroy(shd_ctx *ctx);

/* Message of the last failure on this thread ("" if none).  The pointer
 * stays valid until the next call on this thread. */
const char *shd_last_error(void);

/* Grid of nx*ny*nz nodes spanning [0,lx]x[0,ly]x[0,lz] (Sec. 2: 3-D
 * Cartesian mesh; every n >= 2, every l > 0). */
int shd_set_grid(shd_ctx *ctx, int nx, int ny, int nz, double lx, double ly, double lz);

/* Angular order L (NLM = (L+1)^2 harmonics, Sec. 2.3) and the ordinate mesh
 * n_mu x n_phi (Sec. 2.2 (theta, phi) mesh).  Requires n_mu >= L+1 and
 * n_phi >= 2L+1 (discrete orthogonality of the harmonics), L <= 9,
 * n_mu*n_phi <= 4096. */
int shd_set_angles(shd_ctx *ctx, int L, int n_mu, int n_phi);

/* G groups with G+1 strictly ascending positive edges (units m_e c^2;
 * Sec. 2.3 multi-group treatment).  1 <= G <= 256. */
int shd_set_groups(shd_ctx *ctx, int G, const double *edges);

/* Comoving-frame fields (Sec. 2, Sec. 2.2):
 *   alpha0 [Nc][G]  absorption coefficient (>= 0)
 *   ne     [Nc]     scattering coefficient scale n_e sigma_T (>= 0)
 *   u      [Nc][3]  spatial 4-velocity Gamma v/c (finite)
 *   emis0  [Nc][G]  isotropic emissivity eta0 (>= 0)
 *   theta_e [Nc]    electron temperature kT_e / m_e c^2 (>= 0), or NULL; read
 *                   by the thermal Compton kernel (SHD_SCAT_KN_THERMAL),
 *                   which needs it (its absence is reported at the next step
 *                   with SHD_ERR_STATE); other kernels ignore it.  It is
 *                   checked on the host (SHD_ERR_NAN, "theta_e"), after the
 *                   other four fields.
 * Requires grid, angles and groups.  The host arrays are copied (the call
 * returns once the copies are done and checked); the check runs on the
 * device over a staging copy, before any field array changes, so a refused
 * call leaves the previous fields in place.  Non-finite or negative values
 * -> SHD_ERR_NAN, naming the first offending field in the order alpha0, ne,
 * u, emis0.  A new flow on the same moving nodes keeps the captured step. */
int shd_set_fields(shd_ctx *ctx, const double *alpha0, const double *ne, const double *u,
                   const double *emis0, const double *theta_e);

/* Scattering kernel (Sec. 2.3): kind from enum shd_scattering.  For
 * SHD_SCAT_TABLE, K is [L+1][G][G] (row = final group) and sigma_out [G];
 * both are ignored (may be NULL) for the built-in kinds.  The extinction is
 * chi0(c,g) = alpha0 + n_e sigma_out(g).  Requires angles and groups. */
int shd_set_scattering(shd_ctx *ctx, int kind, const double *K, const double *sigma_out);

/* Copy the active scattering table out: K [L+1][G][G], sigma_out [G] (for
 * SHD_SCAT_KN_THERMAL: the coldest table of the grid). */
int shd_get_scattering(shd_ctx *ctx, double *K, double *sigma_out);

/* The thermal Compton kernel's tables (after shd_set_scattering with
 * SHD_SCAT_KN_THERMAL): K_th [13][L+1][G][G] and sigma_out_th [13][G] on the
 * temperature grid 10^(-3 + i/4) (either may be NULL).  Each is the average
 * of the single-electron Klein-Nishina scattering over isotropic
 * Maxwell-Juttner electrons (laboratory kinematics; no counterpart formula
 * in the paper, whose electrons are cold), by a fixed product quadrature in
 * FP64: 16 energies per incident group, 48 scattering cosines, 24 x 16 x 16
 * electron speeds, direction cosines and azimuths. */
int shd_get_thermal_tables(shd_ctx *ctx, double *K_th, double *sigma_out_th);

/* Inflow boundary intensity (enum shd_boundary); data as described there,
 * NULL for SHD_BC_VACUUM. */
int shd_set_boundary(shd_ctx *ctx, int mode, const double *data);

/* kappa = 1/(c dt) of the backward-Euler time term (Sec. 2.1); 0 gives the
 * static equation.  kappa >= 0. */
int shd_set_time(shd_ctx *ctx, double kappa);

/* Source interpolation of the short-characteristic sweep (enum
 * shd_integrator).  SHD_SC_LINEAR (the default): S~ linear in optical depth
 * between the upwind point U and the node P.  SHD_SC_BEZIER: the cubic
 * Bezier interpolant of Sec. 2 (de la Cruz Rodriguez & Piskunov 2013): S~
 * on the segment is the cubic Bezier curve through S_U and S_P whose control
 * points lie a third of the segment's optical depth along the end
 * derivatives dS~/dtau, each clamped into [S_U, S_P] (no overshoot); the
 * derivative at P is Fritsch and Butland's weighted harmonic mean of the
 * upwind slope and the slope to the downwind point D = P + s n (the upwind
 * slope where D leaves the grid), the derivative at U is bilinear in those
 * of the upwind face nodes that have one (weights renormalised; the
 * segment's slope if none has), and inflow nodes take the downwind slope
 * (none without a downwind point).  Exact
 * for a source linear in optical depth, third order for a smooth one.  The
 * Bezier sweep takes planes of at most 4096 nodes (2365 in SHD_FP64);
 * larger grids are refused at the next step with SHD_ERR_ARG. */
int shd_set_integrator(shd_ctx *ctx, int integrator);

/* Time scheme of shd_step (enum shd_time_scheme).  SHD_TIME_EULER (the
 * default): one source iteration with the time term of Sec. 2.1, eq:time.
 * SHD_TIME_RK4: App. A, eq:rk4th -- the step from t to t + dt is divided
 * into four sub-solves of eq:time from I(t) with time steps dt/6, dt/3,
 * dt/3, dt/6, each one source iteration; with dI_i = (result - input) of
 * sub-solve i, the inputs are I(t), I(t) + 3 dI_1, I(t) + 3/2 dI_2,
 * I(t) + 3 dI_3 and the new state is I(t) + dI_1 + dI_2 + dI_3 + dI_4.
 * RK4 holds three more intensity-sized device arrays (allocated here when
 * the sizes are known, else on the next step) and costs four source
 * iterations per step; shd_get_sums then reports the energy and photon
 * number of I(t) and the source change of the last sub-solve.  Per-stage
 * timing records each sub-solve as one step.  shd_solve_static always
 * iterates the static equation (the scheme does not apply). */
int shd_set_time_scheme(shd_ctx *ctx, int scheme);

/* Ng acceleration of shd_solve_static (Sec. 2: the Lambda iteration is
 * accelerated by Ng's method).  period = 0 turns it off (the default);
 * period >= 4 extrapolates the source at iterations n >= 4 with
 * n - (last extrapolation) >= period:  S* = (1 - a - b) S^n + a S^(n-1) +
 * b S^(n-2), where (a, b) minimise |Q3 - a Q1 - b Q2|^2 over all (c, g, p)
 * with Q1 = S^n - 2 S^(n-1) + S^(n-2), Q2 = S^n - S^(n-1) - S^(n-2) + S^(n-3),
 * Q3 = S^n - S^(n-1) (inner products in FP64; no extrapolation when that
 * 2 x 2 system is singular), and S* replaces S^n before its transform to
 * the ordinates.  Holds three more SH-sized device arrays during the solve. */
int shd_set_ng(shd_ctx *ctx, int period);

/* Set / read the laboratory intensity state I [c][g][k] (host, double).
 * shd_get_state synchronises with the library's stream. */
int shd_set_state(shd_ctx *ctx, const double *I);
int shd_get_state(shd_ctx *ctx, double *I);

/* Run `nsteps` time steps, one source iteration each (stages a1..a5), on
 * `cuda_stream` (a cudaStream_t; NULL = the context's own stream, which is a
 * non-blocking stream: pass cudaStreamLegacy to run on the legacy default
 * stream).  The steps are ordered after all earlier work of the context and
 * before its later calls.  Returns once the work is enqueued.  The state must
 * have been set (or zeroed by shd_zero_state). */
int shd_step(shd_ctx *ctx, int nsteps, void *cuda_stream);

/* Zero the intensity state on the device. */
int shd_zero_state(shd_ctx *ctx);

/* Lambda iteration of the static problem (kappa treated as 0) from the
 * current state until the relative L2 change of S_lm is <= rel_tol
 * (Sec. 2: iterate source and transfer).  Writes the iteration count and
 * final residual; returns SHD_ERR_TIMEOUT if max_iter is reached first. */
int shd_solve_static(shd_ctx *ctx, double rel_tol, int max_iter, int *iters_out, double *resid_out);

/* Laboratory moments of the current state (stage a1 is run on it):
 *   J [c][g], H [c][g][3], K [c][g][6] (xx, yy, zz, xy, xz, yz) -- all
 * divided by 4 pi so that J is the mean intensity -- and the comoving SH
 * projection Ish [c][g][p].  Any output may be NULL.  Synchronous. */
int shd_get_moments(shd_ctx *ctx, double *J, double *H, double *K, double *Ish);

/* The same moments of the current state (Sec. 2: the projection of stage a1)
 * into caller-owned device memory: dev_mom [c][g][10] doubles on ctx's
 * device, J, H_x, H_y, H_z, K_xx, K_yy, K_zz, K_xy, K_xz, K_yz per node and
 * group, divided by 4 pi, the values shd_get_moments returns (single-precision
 * results widened exactly).  Asynchronous on cuda_stream (NULL = the
 * context's stream), ordered after the context's earlier work and before its
 * later work; nothing is copied to the host.  A bounded-wait flag raised by
 * the projection is reported by the next synchronous call.  Errors:
 * SHD_ERR_ARG (dev_mom NULL), SHD_ERR_STATE (not configured, no state). */
int shd_get_moments_dev(shd_ctx *ctx, double *dev_mom, void *cuda_stream);

/* FP64 diagnostics of the last step (stage a5) of the state it started
 * from: energy = sum 4 pi J de_g, photons = sum 4 pi J de_g / ebar_g, resid =
 * ||S_new - S_old|| / ||S_new|| over all (c, g, p).  Synchronous. */
int shd_get_sums(shd_ctx *ctx, double *energy, double *photons, double *resid);

/* ---- single stages on caller-supplied host data (tests, composition) ----
 * Each runs one stage of the step on the fields and tables already set and
 * is synchronous.  Layouts as above: DO arrays [c][g][k], SH [c][g][p]. */
int shd_stage_project(shd_ctx *ctx, const double *I, double *Ish, double *J, double *H, double *K);
int shd_stage_source(shd_ctx *ctx, const double *Ish, double *Ssh);
int shd_stage_sh2lab(shd_ctx *ctx, const double *Ssh, double *eta_lab, double *chi_lab);
int shd_stage_sweep(shd_ctx *ctx, const double *I_old, const double *eta_lab, const double *chi_lab,
                    double *I_new);

/* Device-pointer forms for callers that own device memory (e.g. PyTorch).
 * dev_I points to Nc*G*N doubles in the [c][g][k] layout on ctx's device;
 * the copy runs on cuda_stream (the stream that produced / will consume
 * dev_I; NULL = the context's stream, cudaStreamLegacy = the legacy default
 * stream) and is ordered before the context's later calls. */
int shd_set_state_dev(shd_ctx *ctx, const double *dev_I, void *cuda_stream);
int shd_get_state_dev(shd_ctx *ctx, double *dev_I, void *cuda_stream);

/* Schedule of the single-precision sweep (SHD_FP32 and SHD_MIXED, the
 * linear integrator): every plane of an (ordinate, group) pair is swept by
 * one CTA of NT threads (C = 1; NT = 1024, or 512 / 256 for planes of at
 * most 4 NT nodes, several CTAs an SM; any grid) or split over a
 * thread-block cluster of C CTAs (C = 2, 4, 8 or 16; NT = 256, 384, 512, 768 or
 * 1024; grids whose planes and node count are multiples of 4), each CTA
 * owning a block of rows; rows next to another CTA's block read it through
 * distributed shared memory.  The result does not depend on the schedule
 * (the same arithmetic per node).  By default the library times every
 * schedule that fits on the first sweep run outside a stream capture (over
 * a sample of pairs, on a scratch intensity it allocates and frees there)
 * and keeps the fastest until the grid, angles or groups change.  The choice
 * is also kept for the process: a later context of the same shape (device,
 * grid, groups, ordinates per sweep class, chi0-table use) takes it, with its
 * timing record, instead of timing again.
 * shd_set_sweep_schedule forces (C, NT) (SHD_ERR_ARG if it does not fit the
 * problem), or with C = 0 returns to the automatic choice.
 * shd_get_sweep_schedule reports the schedule in use (0, 0 before the first
 * choice) and, when cand is not NULL, the timing of the last choice:
 * *ncand rows of {C, NT, milliseconds} (at most 16; cand holds 48 floats). */
int shd_set_sweep_schedule(shd_ctx *ctx, int C, int NT);
int shd_get_sweep_schedule(shd_ctx *ctx, int *C, int *NT, int *ncand, float *cand);

/* Source pass (stage a2) of a kernel that mixes groups (Klein-Nishina or a
 * non-diagonal table) in SHD_MIXED: the contraction over g' runs either on
 * the CUDA cores in FP32 or on the tcgen05 tensor cores (per l, the (node,
 * m) rows of eight nodes times K_l, FP32 operands split into three BF16
 * pieces, six products accumulated in FP32: FP32-level rounding).  By
 * default (path 0) the first step outside a stream capture times both and
 * keeps the faster; shd_set_source_path forces 1 (CUDA cores) or 2 (tensor
 * cores; SHD_ERR_ARG where it does not apply).  shd_get_source_path reports
 * the path in use (0 before the timing, 1 where only the CUDA cores apply)
 * and the two timings in milliseconds (0 before). */
int shd_set_source_path(shd_ctx *ctx, int path);
int shd_get_source_path(shd_ctx *ctx, int *path, float *ms_cuda_cores, float *ms_tensor_cores);

/* Which kernels carry the transforms of the configured problem, Eq. 12-14
 * (stage a1, DO -> SH) and Eq. 3 with the Lorentz remap of Eq. 8-9 (stage a3,
 * SH -> DO): 0 the CUDA-core kernels (FP64 and FP32 precisions, or a mixed
 * problem no tensor-core form fits), 1 the tensor-core tile kernels, 2 the
 * tensor-core segment kernels fed and drained by TMA, 3 the same segment
 * kernels with 4-byte cp.async loads and direct stores (planes whose rows
 * are not multiples of 4 nodes, which no tensor map can stride).  Read
 * only; SHD_ERR_STATE before the grid, angles and groups are set. */
int shd_get_transform_path(shd_ctx *ctx, int *path);

/* Self-check of the failure path of the tensor-core kernels' bounded waits
 * (no counterpart in the paper).  Every mbarrier wait in those kernels polls
 * a bounded number of times; when the limit runs out the kernel raises the
 * context's device flag, finishes its outstanding copies and returns, and the
 * next synchronous call (shd_get_moments, shd_get_sums, ...) returns
 * SHD_ERR_TIMEOUT and clears the flag.  This call runs that path on purpose:
 * one thread waits on an mbarrier that nothing arrives on, `polls` times
 * (1 <= polls <= 2^22, about a second at the top), with no copy or MMA in
 * flight, then the call synchronises and reports.  Expected result:
 * SHD_ERR_TIMEOUT with the flag cleared.  A flag left by an earlier kernel is
 * reported first (also SHD_ERR_TIMEOUT) without running the check. */
int shd_check_bounded_wait(shd_ctx *ctx, long long polls);

/* Sizes of the configured problem (any output may be NULL). */
int shd_get_sizes(shd_ctx *ctx, long long *n_nodes, int *n_ord, int *n_groups, int *n_lm);

/* Device bytes held by the context. */
long long shd_device_bytes(shd_ctx *ctx);

/* Per-stage timing of shd_step: with on != 0, every later step records CUDA
 * events around its stages on the stream it runs on (no host
 * synchronisation; at most 2048 steps per enable).  shd_get_timing waits for
 * the last recorded step and returns the summed milliseconds of the stages
 * {project, source, sums, sh2lab, sweep} in stage_ms[5] and the number of
 * steps recorded. */
int shd_set_timing(shd_ctx *ctx, int on);
int shd_get_timing(shd_ctx *ctx, double *stage_ms, long long *steps);

/* Number of CUDA kernels this library has launched in the process so far,
 * over all contexts and threads (counted on the host as each launch is
 * issued).  The difference across a region is how many of the library's
 * kernels that region ran.  Never fails. */
unsigned long long shd_launch_count(void);

/* ---- many independent problems -------------------------------------------
 * Independent problems of uneven size (grid, groups, angular order, flow,
 * precision) stepped together: every step of a batch is one CUDA graph launch
 * holding one captured time step per problem as independent branches, so the
 * problems' kernels run side by side on the GPU.  Each problem is one step of
 * the paper's method (Sec. 2, Sec. 2.1) as shd_step defines it.
 *
 * shd_batch_create: a batch over nprob (>= 1) configured contexts on one
 *   device.  The batch does not own them: they must outlive it, and results
 *   are read from each context (shd_get_moments, shd_get_sums, ...).  A context
 *   may belong to several batches; setters on a context are allowed between
 *   batch steps.  Errors: SHD_ERR_ARG (NULL or mixed devices), SHD_ERR_OOM.
 * shd_batch_step: nsteps time steps of every problem on cuda_stream (NULL =
 *   the first problem's stream), ordered after earlier work of every
 *   problem's own stream and before its later work.  A problem's first step
 *   after its state was set, and every step while its per-stage timing is on,
 *   runs as direct launches.  Errors: those of shd_step, per problem (the
 *   message names it).
 *   In sweep mode 1 the replayed steps of FP32 backward-Euler
 *   problems with the linear short-characteristics integrator, planes the
 *   one-CTA sweep holds, and no cluster schedule forced or timed more than
 *   3 % faster (shd_get_sweep_schedule) run stages a1-a3 per problem and
 *   then stage a4 of all of them in one persistent launch per kernel
 *   variant, over a work list of every such problem's (ordinate, group)
 *   pairs; the other problems sweep in their own launches.  Results are
 *   those of shd_step, bit for bit.
 * shd_batch_set_sweep_mode: 0 (default) every problem sweeps in its own
 *   launches, concurrent with the other problems' stages; 1 as above (one
 *   launch, after every member's stages a1-a3).  Synchronises the device
 *   when the mode changes.
 *   Errors: SHD_ERR_ARG (NULL batch, mode not 0 or 1).
 * shd_batch_destroy: frees the batch (not the contexts). */
typedef struct shd_batch shd_batch;
int shd_batch_create(shd_batch **out, int nprob, shd_ctx *const *problems);
int shd_batch_step(shd_batch *batch, int nsteps, void *cuda_stream);
int shd_batch_set_sweep_mode(shd_batch *batch, int mode);
void shd_batch_destroy(shd_batch *batch);

/* ---- projection without allocation --------------------------------------
 * No counterpart in the paper.  For callers that cannot call cudaMalloc when
 * they need the moments: programs whose device memory belongs to another
 * allocator (a framework's pool), loops that must not meet the allocator's
 * implicit device synchronisation, processes at their memory limit.
 *
 * shd_project_noalloc runs stage a1 on the context's current state and writes
 *   dev_Ish [c][g][p]  comoving SH projection I_lm
 *   dev_mom [c][g][10] laboratory moments J, H_x, H_y, H_z, K_xx, K_yy, K_zz,
 *                      K_xy, K_xz, K_yz (divided by 4 pi)
 * to caller-owned device memory, in the context's working precision (double
 * for SHD_FP64, float otherwise).  It allocates nothing: the comoving
 * intensities of moving nodes live in one static device array of
 * SHD_NOALLOC_SCRATCH_BYTES (64 MiB), present on every device that loads the
 * library until the process exits.  Problems whose moving nodes need more
 * than that -- 2 * (moving nodes) * G * N * (bytes per real) -- are
 * rejected with SHD_ERR_ARG (message: shd_noalloc_last_error()); nodes at
 * rest need no scratch.
 *   - The first call on a device looks up the array's device address (with
 *     that device current); make that first call before any stream capture.
 *     The address is kept for the life of the process: it does not survive a
 *     cudaDeviceReset of that device (the primary context, and with it the
 *     array, is then a new one), so do not call this entry point after one.
 *   - The call makes ctx's device current while it works and restores the
 *     caller's current device before it returns.
 *   - Work runs on cuda_stream (NULL: the context's stream, ordered after the
 *     context's earlier work); with another stream the caller orders it after
 *     the steps that produced the state.
 *   - Every call shares the one array and leaves its contents behind; nothing
 *     in it needs to start at zero (each call writes every entry it reads).
 *     Calls that overlap on the GPU race on it.
 *   - In SHD_MIXED the tensor-core kernels give up on a wait that runs out
 *     of its iteration limit and raise the context's device flag; this call
 *     does not read it back (that would synchronise).  The next
 *     shd_get_moments or shd_get_sums on ctx reports it as SHD_ERR_TIMEOUT:
 *     call one of them before trusting outputs whose timing matters.
 * Returns SHD_OK, SHD_ERR_ARG (null pointer, too large, a stage's shared
 * memory over the limit), SHD_ERR_STATE (not configured) or SHD_ERR_CUDA. */
#define SHD_NOALLOC_SCRATCH_BYTES (64ull << 20)
int shd_project_noalloc(shd_ctx *ctx, void *dev_Ish, void *dev_mom, void *cuda_stream);
const char *shd_noalloc_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* SHDOM_GB300_H */
