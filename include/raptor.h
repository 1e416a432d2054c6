/* raptor.h -- C ABI of the B300 ray-tracing / radiative-transfer library.
 *
 * The library integrates, for every camera pixel (and frame), one null geodesic backward
 * from a distant camera through Kerr spacetime and, along it, unpolarised thermal
 * synchrotron radiative transfer for a set of observing frequencies (Bronzwaer et al.
 * 2018, "RAPTOR I").  The operations and the passages that define them:
 *   - camera initial conditions: sec. 2.3, Eqs. 24-28 (Bardeen camera) and Eq. 4;
 *   - geodesic equation as 8 first-order ODEs, Eqs. 5-6, with the connection of Eq. 2;
 *   - classical RK4 step, Eqs. 7-15, with the adaptive step of Eqs. 20-23;
 *   - backward transfer, Eqs. 35-36, per-step formal solution of Eq. 34,
 *     fluid-frame frequency nu = -k.u (Eq. 30), observed intensity (Eq. 31);
 *   - thermal synchrotron emissivity and Kirchhoff absorption, Eqs. 41-44;
 *   - GRMHD unit scaling and R-beta electron temperature, Eqs. 45-46;
 *   - MKS coordinates and Newton-Raphson theta -> x2, App. A.2; BL -> KS, App. A.1;
 *   - fast- and slow-light sampling of GRMHD snapshots, sec. 5;
 *   - flux density in Jy as the sum of pixel intensities times the pixel solid angle
 *     (sec. 4.2.2, Table 3).
 *
 * Conventions for every call:
 *   - Units: G = c = M = 1 inside; the camera's impact parameters alpha, beta, radii and
 *     coordinate times are in M.  Frequencies in Hz.  Images in Jy per pixel.
 *   - Pointers named *_dev are CUDA device pointers; *_host are host pointers.  The caller
 *     owns every buffer it passes; the library never frees caller memory.  Descriptors are
 *     copied at call time.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  Work is enqueued on it.
 *     Calls that return host data (flux_jy_host, stats) synchronise that stream first.
 *   - Errors: every call returns a raptor_status.  Arguments are validated on the host
 *     before any launch (RAPTOR_EINVAL, nothing enqueued).  A failing CUDA call returns
 *     RAPTOR_ECUDA.  raptor_last_error() returns a message for the last failure on that
 *     context.  No exception or abort crosses this ABI.
 *   - Threads: a context is used by one host thread at a time.
 */
#ifndef RAPTOR_H
#define RAPTOR_H

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    RAPTOR_OK = 0,
    RAPTOR_EINVAL = 1,       /* invalid argument or descriptor; nothing was enqueued      */
    RAPTOR_ENOMEM = 2,       /* device or host allocation failed                          */
    RAPTOR_ECUDA = 3,        /* a CUDA runtime call or kernel launch failed               */
    RAPTOR_ETIMEOUT = 4,     /* a bounded device-side wait of the tensor-core kernels
                                expired; the context stays usable                         */
    RAPTOR_ENOPLASMA = 5,    /* render before raptor_load_plasma                          */
    RAPTOR_EUNSUPPORTED = 6  /* option recognised but not available in this library       */
} raptor_status;

/* Returned by the learned-surrogate calls (RAPTOR_MIXED_MLP) before a surrogate exists. */
#define RAPTOR_ENOSURROGATE RAPTOR_EUNSUPPORTED

/* Arithmetic of the integration.
 *   RAPTOR_FP64:  every step in FP64.
 *   RAPTOR_MIXED: geodesic steps and transfer in FP32 where r >= r_fp64 and away from radial
 *                 turning points; FP64 inside r < r_fp64 and where |k^r| < turn_kr |k^t|;
 *                 the optical depth beyond tau = 10 with a 48-bit significand (compensated
 *                 float pair).  Rays are moved between FP32 and FP64 work queues so each
 *                 warp runs one precision.
 *   RAPTOR_MIXED_MLP: RAPTOR_MIXED, with every ray outside the critical curve and a band
 *                 around it started from the learned surrogate's prediction of the state
 *                 after 60 steps (see raptor_surrogate_*), and rays leaving r > r_exit on
 *                 the way out stopped (transfer beyond r_exit neglected).  Needs a trained
 *                 or loaded surrogate (else RAPTOR_EUNSUPPORTED). */
typedef enum { RAPTOR_FP64 = 0, RAPTOR_MIXED = 1, RAPTOR_MIXED_MLP = 2 } raptor_precision;

typedef enum {
    RAPTOR_PLASMA_ANALYTIC = 0,  /* n_e = n0 r^n_pow, Theta_e = the0 r^the_pow, B = B0 r^B_pow;
                                    prograde Keplerian flow for r >= r_isco, free fall from rest
                                    at infinity inside; toroidal field                     */
    RAPTOR_PLASMA_GRID_MKS2D = 1 /* axisymmetric GRMHD-shaped snapshots on an MKS grid       */
} raptor_plasma_kind;

#define RAPTOR_FLAG_K2_EXACT 0x1u      /* exact K2(1/Theta_e) instead of 2 Theta_e^2 (sec. 4.2.2) */
#define RAPTOR_FLAG_STEP_LINEAR_R 0x2u /* literal d lambda = eps r (no polar limiter)            */
#define RAPTOR_FLAG_INNER_DF64 0x4u    /* MIXED/MIXED_MLP: inner-region geodesic steps in double-
                                          float arithmetic on the FP32 pipe (48-bit significand,
                                          ~1e-14 relative) instead of native FP64              */
#define RAPTOR_FLAG_VERLET 0x8u        /* RAPTOR_FP64: velocity Verlet (sec. 2.2.2, Eqs. 16-19,
                                          one connection evaluation per step) instead of RK4  */
#define RAPTOR_FLAG_VERLET_REEVAL 0x10u /* RAPTOR_FP64: velocity Verlet with the re-evaluation
                                          of Eqs. 18-19 (two evaluations per step); the
                                          derivative carried on is the last one evaluated    */
#define RAPTOR_FLAG_FORWARD_RT 0x20u   /* RAPTOR_FP64: forward formal-solution transfer (sec. 3,
                                          Eq. 34 from the far end) instead of the backward
                                          accumulation: each ray records its steps' optical
                                          depth and contribution (at most 2048 emitting steps:
                                          beyond, status RAPTOR_RAY_ERROR) in a context buffer
                                          of (launched threads x 2048 x n_freq) pairs; at most
                                          4 frequencies per call (EINVAL); the same results to
                                          rounding; not with raptor_render_noalloc
                                          (EUNSUPPORTED)                                     */

/* Ray termination codes written to status_dev (render_ex) and trace calls. */
#define RAPTOR_RAY_ESCAPED 0   /* r > r_escape                       */
#define RAPTOR_RAY_CAPTURED 1  /* r < r_stop_factor * r_horizon      */
#define RAPTOR_RAY_THICK 2     /* min over frequencies of tau > tau_cut */
#define RAPTOR_RAY_TRUNCATED 3 /* max_steps reached                  */
#define RAPTOR_RAY_ERROR 4     /* non-finite state or nu_fluid <= 0  */

typedef struct raptor_ctx raptor_ctx; /* opaque, library-owned */

/* Camera, spacetime and integration settings (sec. 2.2-2.3, Table 2).  Fill with
 * raptor_camera_desc_default() and override. */
typedef struct {
    double spin;          /* a/M, |a| < 1                                         [0.9]   */
    double mass_msun;     /* black-hole mass M in solar masses                    [4e6]   */
    double distance_pc;   /* distance D in parsec                                 [7880]  */
    double r_cam;         /* camera radius (BL), M                                [1000]  */
    double incl_deg;      /* inclination i, degrees, in (0, 180)                  [60]    */
    int nx, ny;           /* pixels; pixel (row i, col j) has centre
                             alpha = alpha_min + (j+1/2) dalpha, beta = beta_min + (i+1/2) dbeta */
    double alpha_min, alpha_max, beta_min, beta_max; /* image plane, M           [+-20]  */
    double eps;           /* step scale of Eqs. 20-23 (read in log r)             [0.05]  */
    double r_stop_factor; /* capture when r < r_stop_factor r_horizon             [1.01]  */
    double r_escape;      /* escape when r > r_escape                             [1000]  */
    double tau_cut;       /* stop when every frequency has tau > tau_cut          [inf]   */
    int max_steps;        /* per-ray step cap; capped rays are counted            [1e5]   */
    int precision;        /* raptor_precision                                     [FP64]  */
    unsigned flags;       /* RAPTOR_FLAG_*                                        [0]     */
    int reserved0;
    double r_fp64;        /* MIXED: FP64 for r < r_fp64                           [6]     */
    double turn_kr;       /* MIXED: FP64 where |k^r| < turn_kr |k^t|              [0.05]  */
    double t_delay;       /* slow light: added to each frame's camera time, M     [r_cam] */
} raptor_camera_desc;

/* Plasma (sec. 4.2.2, sec. 5).  For GRID_MKS2D, `fields` holds n_snap snapshots, each
 * 8 FP32 planes [field][x2][x1] in the order rho, u, U1, U2, U3, B1, B2, B3 (HARM
 * primitives in MKS components; U^i is the velocity relative to the normal observer),
 * cell-centred on x1 in [x1_min, x1_max] (x1 = ln r) and x2 in [0, 1], with
 * theta = pi x2 + (1-h)/2 sin(2 pi x2).  Snapshot s is at KS time t0 + s dt_snap. */
typedef struct {
    int kind;             /* raptor_plasma_kind                                          */
    int slow_light;       /* GRID: 1 = interpolate snapshots linearly in ray time (sec. 5) */
    double n0, n_pow, the0, the_pow, B0_gauss, B_pow; /* ANALYTIC profiles [1e6,-1.5,10,-1,20,-1] */
    const float* fields;  /* GRID: host pointer (copied) or device pointer, see below     */
    int n1, n2, n_snap;   /* GRID: sizes; n1, n2 >= 2, n_snap >= 1                        */
    int fields_on_device; /* GRID: 1 = `fields` is a device pointer (copied device-to-device) */
    double x1_min, x1_max, h_mks; /* GRID: radial range (ln r) and MKS h in (0, 1]        */
    double t0, dt_snap;   /* GRID: time of snapshot 0 and spacing, M                      */
    double mass_unit_g;   /* GRID: mass unit (Eq. 45), grams                             */
    double r_high, r_low; /* GRID: R-beta parameters (Eq. 46)                             */
    double gamma_ad;      /* GRID: adiabatic index                                 [4/3]  */
    double theta_e_min;   /* emission (and absorption) only where Theta_e >= theta_e_min: the
                             validity mask of the emissivity fit (the paper quotes < 1 %
                             error for Theta_e > 0.5, sec. 4.2.2); 0 = no mask          [0]    */
} raptor_plasma_desc;

/* Fill descriptors with the defaults shown in brackets above. */
void raptor_camera_desc_default(raptor_camera_desc* desc);
void raptor_plasma_desc_default(raptor_plasma_desc* desc);

/* Create a context for one camera (sec. 2.3).  Validates desc (EINVAL), selects the
 * current CUDA device, allocates the context's device work buffers (ENOMEM/ECUDA).
 * *out receives the context; release it with raptor_destroy. */
raptor_status raptor_camera_init(const raptor_camera_desc* desc, raptor_ctx** out);

/* Replace the camera settings of an existing context (same rules as camera_init). */
raptor_status raptor_camera_set(raptor_ctx* ctx, const raptor_camera_desc* desc);

/* Load the plasma model the transfer samples (sec. 4.2.2; sec. 5).  ANALYTIC copies the
 * profile constants (power laws in r of n_e, Theta_e and B, Keplerian / free-fall velocity;
 * not a model of the paper).  GRID copies the snapshot array into a context-owned device
 * buffer (host->device or device->device on `stream`; the caller's buffer may be freed once
 * the call returns): HARM primitives on a modified Kerr-Schild grid (sec. 4.2.2 and App. A.2,
 * the theta map inverted by Newton's iteration), scaled to CGS by the mass unit of Eq. 45
 * (rho_0 = M_unit / L^3, n_e = rho rho_0 / (m_e + m_p), B from b.b and rho_0), electron
 * temperature from the R-beta prescription of Eq. 46 with R_high and R_low, and with
 * slow_light a time series of snapshots dt_snap apart interpolated linearly in the ray's
 * coordinate time (sec. 5.1).  RAPTOR_EINVAL for an unknown kind, non-positive sizes or
 * spacings, a NULL field pointer or non-finite constants; RAPTOR_ENOMEM / RAPTOR_ECUDA when
 * the copy fails (the previous plasma is then kept). */
raptor_status raptor_load_plasma(raptor_ctx* ctx, const raptor_plasma_desc* desc, void* stream);

/* Render one image at camera time t_obs (fast light): every pixel's ray is integrated
 * backwards from the camera (sec. 2.3, Eqs. 24-28) with the adaptive step of Eqs. 20-23 and
 * the integrator of sec. 2.2.2, and the invariant intensity is accumulated by the backward
 * transfer scheme of Eqs. 35-36 with the per-step formal solution of Eq. 34 and the
 * thermal-synchrotron coefficients of Eqs. 41-44.  The image holds each pixel's flux density
 * in Jy, I_nu dalpha dbeta L^2 / D^2 / 1e-23 with L = GM/c^2 (the pixel sum is the total flux
 * density of sec. 4.2.2 and Table 3).  freqs_hz[n_freq] is a host array (1 <= n_freq <= 64).
 * image_dev: device double [n_freq][ny][nx] (row 0 = beta_min), caller-owned, written
 * completely.  flux_jy_host: optional host double [n_freq] (NULL to skip; otherwise the
 * stream is synchronised).  Grid plasma uses snapshot 0 unless slow_light is set.
 * RAPTOR_EINVAL for a NULL image, n_freq outside 1..64 or a non-positive frequency;
 * RAPTOR_ENOPLASMA before raptor_load_plasma; RAPTOR_ETIMEOUT when a bounded wait of the
 * learned path's tensor-core kernels expires; RAPTOR_ECUDA on a CUDA error (message in
 * raptor_last_error). */
raptor_status raptor_render(raptor_ctx* ctx, const double* freqs_hz, int n_freq, double t_obs,
                            double* image_dev, double* flux_jy_host, void* stream);

/* As raptor_render, for rows [row0, row0 + n_rows) only (image_dev is [n_freq][n_rows][nx]),
 * fast-light snapshot `snap` for grid plasma, and optional per-pixel diagnostics:
 * steps_dev (int32 [n_rows][nx], accepted RK4 steps) and status_dev (int32, RAPTOR_RAY_*). */
raptor_status raptor_render_ex(raptor_ctx* ctx, const double* freqs_hz, int n_freq, double t_obs,
                               int row0, int n_rows, int snap, double* image_dev, double* flux_jy_host,
                               int* steps_dev, int* status_dev, void* stream);

/* Thin-disk line emitter (sec. 4.2.1): an opaque disk in the equatorial plane between r_in
 * and r_out on circular Keplerian orbits (Omega = 1/(r^{3/2} + a): prograde for a > 0,
 * retrograde relative to the hole for a < 0), emitting one line with emission ~ r^-q and no
 * absorption. */
typedef struct {
    double r_in;        /* inner radius in M; <= 0: the ISCO of the camera's spin [0] */
    double r_out;       /* outer radius in M [15] */
    double q;           /* emission ~ r^-q [2] */
    int max_cross;      /* crossings of the equatorial plane after which a ray gives up [10] */
    int profile_order;  /* crossing number of the hits that form the spectrum; 0: all [1] */
    int n_bins;         /* spectrum bins of E_obs/E_em over [x_min, x_max) [64] */
    double x_min, x_max; /* [0.2, 1.6] */
} raptor_disk_desc;

raptor_status raptor_disk_desc_default(raptor_disk_desc* d);

/* Render the thin disk with the context's camera (spin, inclination, field of view, step
 * rule, r_stop, r_escape, max_steps), always in FP64 (no plasma needed).  Each pixel's ray
 * is integrated until it crosses theta = pi/2 inside the disk (a hit: crossing point refined
 * by Newton's iteration on the length of the last RK4 step), is captured or escapes, or has
 * crossed the plane max_cross times.  Outputs (caller-owned device arrays [ny][nx], row-major
 * as the images): ratio_dev = E_obs/E_em = 1 / (k.u) at the hit, intensity_dev = the line's
 * frequency-integrated intensity (E_obs/E_em)^4 r^-q, order_dev = crossing number of the hit
 * (0 and zeros elsewhere for rays without a hit); optional status_dev (0 escaped, 1 captured,
 * 3 truncated, 4 error, 5 hit, 6 max_cross crossings without a hit) and steps_dev (may be
 * NULL).  profile_host (host, [n_bins], may be NULL): the line spectrum, the sum of
 * intensity x pixel area (d alpha d beta in M^2) over the hits of crossing number
 * profile_order in bins floor((ratio - x_min) / dx), dx = (x_max - x_min) / n_bins, summed
 * in 64-bit fixed point (order-independent); with a spectrum the call synchronises the
 * stream.  RAPTOR_EINVAL for NULL required buffers, r_in >= r_out, max_cross < 1 or a bad
 * bin range. */
raptor_status raptor_disk_render(raptor_ctx* ctx, const raptor_disk_desc* d, double* ratio_dev, double* intensity_dev,
                                 int* order_dev, int* status_dev, int* steps_dev, double* profile_host, void* stream);

/* Render an image from host buffers: copies nothing in but the frequencies, renders, copies
 * the image to image_host (double [n_freq][ny][nx], may be NULL) and the flux to
 * flux_jy_host (may be NULL), and synchronises `stream`.  Device scratch is context-owned. */
raptor_status raptor_render_host(raptor_ctx* ctx, const double* freqs_hz, int n_freq, double t_obs,
                                 double* image_host, double* flux_jy_host, void* stream);

/* Light curve (sec. 5): frames f = 0..n_frames-1 at camera times t_obs_host[f]; every
 * (frame, pixel) ray of every frame goes through one persistent launch.  Slow light when the
 * grid plasma has slow_light = 1; otherwise frame f uses snapshot first_frame + f (fast
 * light).  flux_jy_host: host double [n_frames][n_freq] (required; stream synchronised).
 * images_dev: optional device double [n_frames][n_freq][ny][nx]. */
raptor_status raptor_lightcurve(raptor_ctx* ctx, const double* freqs_hz, int n_freq,
                                const double* t_obs_host, int n_frames, int first_frame,
                                double* flux_jy_host, double* images_dev, void* stream);

/* Trace one ray on the device and record every step: rec_host[n][12] = x^mu (4), k^mu (4),
 * d lambda, nu_fluid/nu_obs (0 on the terminating step), I_obs and tau of the first
 * frequency.  Returns up to max_rec records; *n_steps = total steps; *ray_status = RAPTOR_RAY_*.
 * Synchronises `stream`.  Same arithmetic as raptor_render's FP64 path. */
raptor_status raptor_trace_ray(raptor_ctx* ctx, double alpha, double beta, double t_obs,
                               const double* freqs_hz, int n_freq, int max_rec, double* rec_host,
                               int* n_steps, int* ray_status, double* intensity_host, void* stream);

/* Counters accumulated over all launches since the context was created (synchronises the
 * last stream used): rays traced (one ray = one pixel x frame; a ray carries all
 * frequencies of the call), accepted integration steps (one step of the integrator of
 * sec. 2.2.2: an RK4 step, Eqs. 7-15, with its four right-hand sides, or a velocity-Verlet
 * step, Eqs. 16-19, with the step length of Eqs. 20-23; the steps a learned start state
 * replaces are counted as taken), of which FP64 steps, rays truncated at max_steps, rays
 * with an error status, learned-surrogate fallbacks.  The host pointers are caller-owned;
 * NULL skips a value.  RAPTOR_EINVAL for a NULL context, RAPTOR_ECUDA on a CUDA error. */
raptor_status raptor_stats(raptor_ctx* ctx, unsigned long long* rays, unsigned long long* steps,
                           unsigned long long* fp64_steps, unsigned long long* truncated,
                           unsigned long long* errors, unsigned long long* fallback);

/* Reset the counters of raptor_stats. */
raptor_status raptor_stats_reset(raptor_ctx* ctx);

/* All counters behind raptor_stats (synchronises the context's last stream): values[count]
 * (caller's host array, 1 <= count <= 16) receives, in order, rays, accepted steps (as in
 * raptor_stats), FP64 steps, truncated rays, rays with an error status, surrogate
 * fallbacks, re-entries of the FP64 region during the outbound FP32 phase (counted, not
 * moved), clamped slow-light samples, the FP64 steps taken on the mixed path's second
 * stream (near-critical rays), and the FP32 steps executed by the mixed path's inbound
 * phase (A) and outbound phase (C) launches (steps a learned start state replaces are not
 * executed and not counted there); later slots are zero.  RAPTOR_EINVAL for a count outside
 * 1..16. */
raptor_status raptor_stats_ex(raptor_ctx* ctx, unsigned long long* values, int count);

/* Launch shape of the persistent kernels (used by the autotuner): threads per block in
 * {32, 64, 96, 128}, resident blocks per SM of the FP64 and FP32 ray kernels, and of the
 * mixed path's FP64 passes (0 = the occupancy maximum). */
raptor_status raptor_set_launch(raptor_ctx* ctx, int threads_per_block, int blocks_per_sm, int blocks_per_sm_fp64);

/* Mixed path scheduling: rays whose pixel centre lies within crit_band M of the critical
 * curve (Bardeen's closed form) form phase A1 and run their FP64 phase, then their outbound
 * FP32 phase, on a second stream, concurrently with the other rays' phases A2, B and C
 * [0.5].  The other rays' FP64 phase
 * runs in n_passes passes (1..8): pass k continues each ray for at most budgets[k] steps
 * and re-queues the unfinished ones for pass k + 1; the last pass has no limit (budgets may
 * be NULL: the default schedule).  With tail_split = K in 1 .. n_passes - 1, the rays still
 * in the FP64 region after K passes finish their FP64 phase on the second stream (after the
 * near-critical rays, and with them their outbound phase), while the first stream goes on
 * with phase C [0: no split].  Only the
 * schedule changes: every ray's arithmetic, and so every result, is the same for any
 * setting.  RAPTOR_EINVAL for a negative or non-finite band, n_passes outside 1..8, a
 * budget < 1 or a negative tail_split. */
raptor_status raptor_mixed_config(raptor_ctx* ctx, double crit_band, int n_passes, const int* budgets, int tail_split);

/* Schedule of the near-critical rays' FP64 phase on the mixed path's second stream:
 * threads_per_block in {32, 64, 96, 128} (0: the block size of the other launches) and
 * n_passes (1..8) passes, pass k continuing each ray for at most budgets[k] steps and
 * re-queueing the unfinished ones, packed into full warps, for pass k + 1; the last pass has
 * no limit (budgets may be NULL for n_passes = 1) [0, 1].  The grid keeps the thread count of
 * the other FP64 passes.  Only the schedule changes, never a result.  RAPTOR_EINVAL for a
 * block size or pass count out of range, or a budget < 1. */
raptor_status raptor_long_config(raptor_ctx* ctx, int threads_per_block, int n_passes, const int* budgets);

/* CUDA graphs (enable != 0, the default): the second raptor_render / raptor_render_ex /
 * raptor_lightcurve call with the same arguments, context settings and device buffers
 * captures its whole launch sequence (both streams of the mixed path) into a graph, and
 * later identical calls replay it with one launch; light curves keep their frame times in a
 * context buffer, so a batch of frames with new times replays the same graph.  Calls of more
 * than 2^19 rays (pixels x frames) and calls made while profiling is on run directly (at that
 * size the launch latencies are negligible and direct launches overlap the two streams
 * better).  raptor_graph_stats returns the number of captures and
 * replays so far (outputs may be NULL). */
raptor_status raptor_graph_config(raptor_ctx* ctx, int enable);
raptor_status raptor_graph_stats(raptor_ctx* ctx, long long* captures, long long* replays);

/* Autotuner: renders the context's camera once per candidate launch shape (threads per
 * block {64, 128}; blocks per SM of the ray kernels {max, 2, 3, 4}; for RAPTOR_MIXED also
 * blocks per SM of the FP64 passes {1, 2, 3, 4}), times each with CUDA events on `stream`
 * (best of two), keeps the fastest on the context and returns it (outputs may be NULL).
 * Uses a context-owned image buffer; synchronises `stream`. */
raptor_status raptor_autotune(raptor_ctx* ctx, const double* freqs_hz, int n_freq, double t_obs, int* best_block,
                              int* best_bps, int* best_bps64, double* best_ms, void* stream);

/* ---- Learned surrogate (a learned map of the integration; the paper has none) ------------
 * A 4-layer, 256-wide MLP maps (alpha, beta, a, i) to the FP64 integrator's state after 60
 * adaptive RK4 steps from the camera (t - t_cam, ln r, theta, phi and the signs of k^theta,
 * k^r; the wave vector is rebuilt from E, L, Q).  Training data come from the integrator
 * itself; forward and backward run in the library's kernels (hidden layers on BF16 tensor
 * cores with FP32 accumulation), optimiser Adam.  The surrogate lives in the context. */

/* Number of FP32 parameters (weights, biases and the input/output normalisation). */
int raptor_surrogate_param_count(void);

/* Training set: n samples with alpha, beta uniform over the context's image plane, spin
 * uniform in [spin_min, spin_max], inclination uniform in [incl_min, incl_max] degrees
 * (counter-based generator seeded by `seed`).  inputs_dev: device float [n][4] = (alpha,
 * beta, a, i_deg).  states_dev (optional, device double [n][6]) receives the integrator's
 * state after 60 steps (FP64, same arithmetic as the FP64 path) as (t - t_cam, ln r, theta,
 * phi, k^theta, k^r); targets_dev (device double [n][6]) the same state minus a fixed
 * flat-space baseline (straight line advanced by the same step rule), which the network
 * learns. */
raptor_status raptor_surrogate_generate(raptor_ctx* ctx, long long n, unsigned long long seed, double spin_min,
                                        double spin_max, double incl_min_deg, double incl_max_deg, float* inputs_dev,
                                        double* targets_dev, double* states_dev, void* stream);

/* Initialise the network (seeded uniform weights) and its output normalisation from the
 * first min(n, 65536) targets; resets the optimiser.  Synchronises `stream`. */
raptor_status raptor_surrogate_init(raptor_ctx* ctx, const double* targets_dev, long long n, unsigned long long seed,
                                    void* stream);

/* `steps` Adam steps on batches of 4096 samples drawn (with replacement, counter-based,
 * `seed`) from the n samples; learning rate cosine-decayed from lr to lr_final.
 * loss_host (optional, [steps]) receives each batch's mean squared error (normalised
 * outputs); when given, every step synchronises `stream`. */
raptor_status raptor_surrogate_train(raptor_ctx* ctx, const float* inputs_dev, const double* targets_dev, long long n,
                                     int steps, double lr, double lr_final, unsigned long long seed, double* loss_host,
                                     void* stream);

/* Loss and parameter gradient of one batch of n samples (n a multiple of 128, <= 4096) at
 * the current parameters, without an update: grad_host receives the gradient of every
 * weight and bias (raptor_surrogate_param_count() - 24 floats), loss_host the loss. */
raptor_status raptor_surrogate_grad(raptor_ctx* ctx, const float* inputs_dev, const double* targets_dev, long long n,
                                    float* grad_host, double* loss_host, void* stream);

/* Predictions for n inputs (device float [n][4]) into pred_dev (device double [n][6], same
 * units as the targets).  Synchronises `stream`. */
raptor_status raptor_surrogate_eval(raptor_ctx* ctx, const float* inputs_dev, long long n, double* pred_dev, void* stream);

/* Copy the parameters out / in (host float [raptor_surrogate_param_count()]); `set` makes the
 * context's surrogate ready without training. */
raptor_status raptor_surrogate_get(raptor_ctx* ctx, float* params_host, int n);
raptor_status raptor_surrogate_set(raptor_ctx* ctx, const float* params_host, int n);

/* Save the trained surrogate to a file / load one into this context (checkpoint and reuse
 * of a trained network; the paper has no counterpart).  Format: the 8 bytes "RAPTMLP1",
 * u32 format version (1), u32 parameter count, the FP32 parameters in raptor_surrogate_get
 * order (little-endian), u64 FNV-1a hash of the parameter bytes.  `load` validates magic,
 * version, count, length and hash before touching the context (RAPTOR_EINVAL otherwise) and
 * then acts as raptor_surrogate_set.  `save` returns RAPTOR_EUNSUPPORTED without a network. */
raptor_status raptor_surrogate_save(raptor_ctx* ctx, const char* path);
raptor_status raptor_surrogate_load(raptor_ctx* ctx, const char* path);

/* Kernel of the surrogate's inference (raptor_surrogate_eval and RAPTOR_MIXED_MLP renders):
 *   RAPTOR_MLP_TCGEN05 (default): hidden layers on the 5th-generation tensor cores
 *     (tcgen05.mma, accumulators in tensor memory, weights resident in shared memory);
 *   RAPTOR_MLP_MMA_SYNC: one fused kernel on warp-level mma.sync BF16 instructions.
 * Both compute the training forward pass's arithmetic (BF16 operands, FP32 accumulation)
 * and differ only in FP32 summation order.  A tensor-core wait that exceeds 2 s makes the
 * next synchronising call (raptor_surrogate_eval, a render that returns fluxes) fail with
 * RAPTOR_ETIMEOUT.  RAPTOR_EINVAL for another value. */
#define RAPTOR_MLP_TCGEN05 0
#define RAPTOR_MLP_MMA_SYNC 1
raptor_status raptor_surrogate_kernel(raptor_ctx* ctx, int kind);

/* Fallback: rays whose pixel centre lies inside the critical curve (Bardeen's closed form)
 * or within fallback_band M of it start at the camera (exact integration) [0.5], and so do
 * the pixel centres within 0.01 M of alpha = 0 (rays of nearly zero angular momentum pass
 * the polar axis, where the transfer's samples follow tiny changes of L; fixed); r_exit:
 * outbound rays stop at r > r_exit in RAPTOR_MIXED_MLP (0 = off) [50]. */
raptor_status raptor_surrogate_config(raptor_ctx* ctx, double fallback_band, double r_exit);

/* Hand-off step count of the learned start states (no counterpart in the paper): the state
 * network predicts the integrator's state after n_steps adaptive steps from the camera
 * [60].  This call sets the count for the data raptor_surrogate_generate writes next;
 * raptor_surrogate_init stores it with the network's parameters (an unused output-mean
 * slot), and a render uses the count of the network in use (raptor_surrogate_set / _load
 * read it back; 0 there reads as 60).  The network's angular error at the hand-off carries
 * over to the ray's path in the emitting region, and the deflection it learns relative to
 * the flat-space baseline falls like r^-2 with the hand-off radius (r ~ r_cam e^{-eps n}):
 * fewer steps give more accurate paths and skip less integration.  RAPTOR_EINVAL outside
 * [1, 1000]; raptor_surrogate_set: RAPTOR_EINVAL when the stored count is not 0 or an
 * integer in [1, 1000]. */
raptor_status raptor_surrogate_handoff(raptor_ctx* ctx, int n_steps);

/* Host-side fault injection for failure-handling tests (no counterpart in the paper; no
 * device fault is raised).  RAPTOR_FAULT_TC_WAIT: set, from the host and after the context's
 * last stream has drained, the device flag that a bounded mbarrier wait of the tensor-core
 * network kernels sets when it runs out, so that the next learned render (or crossing
 * network evaluation) that synchronises returns RAPTOR_ETIMEOUT with the reason in
 * raptor_last_error, clears the flag and leaves the context usable.  RAPTOR_EINVAL for an
 * unknown kind; RAPTOR_EUNSUPPORTED when the context has no network yet. */
enum { RAPTOR_FAULT_TC_WAIT = 1 };
raptor_status raptor_inject_fault(raptor_ctx* ctx, int kind);

/* Learned equatorial crossings (the learned surrogate's thin-disk outputs; the geometry is
 * sec. 4.2.1's disk plane theta = pi/2, the network has no counterpart in the paper).  A
 * second network of the same shape (4 -> 256 -> 256 -> 256 -> 16, SiLU; BF16 hidden layers
 * with FP32 accumulation, FP32 input and output layers) maps (alpha, beta, a, i in degrees)
 * to the first four crossings n = 0..3 of the plane by the backward ray, four outputs each:
 *   presence logit; ln r_n (for n = 0 relative to the straight camera ray's crossing radius,
 *   flat space, FP32, as ln sqrt(r_flat^2 + 9)); lambda_n - lambda_{n-1}, lambda the affine
 *   length from the camera (E = 1), lambda_{-1} the straight ray's length to the plane;
 *   E_obs/E_em of a prograde Keplerian emitter at r_n (Eq. 30), trained for r_n >= r_isco.
 *
 * raptor_crossings_generate: n counter-based samples over the camera's field of view and the
 * given spin (-1 < a < 1; a < 0: the emitter's orbit retrograde relative to the hole) and
 * inclination ranges (0 < i < 90), inputs_dev (device float [n][4], rounded
 * to FP32 before tracing) and targets_dev (device double [n][16]: presence 1/0; NaN for the
 * regression entries of absent crossings and for ratios inside the ISCO), raw_dev (optional,
 * device double [n][16]: per crossing presence, r_n, lambda_n, E_obs/E_em, NaN if absent).
 * The targets come from the FP64 RK4 integrator with the camera's step rule, r_stop, r_escape
 * and max_steps; every step that ends across the plane is refined by Newton's iteration on
 * its length (as raptor_disk_render).  Asynchronous on `stream`.
 * raptor_crossings_init / _train / _grad / _get / _set: as the raptor_surrogate_* calls, for
 * this network (targets [n][16]; param count raptor_crossings_param_count()).  The loss is the
 * mean over rows x 16 outputs of the logistic loss log(1 + e^z) - y z on the presence logits
 * and the squared normalised error on the others, with NaN targets carrying no weight.
 * raptor_crossings_eval: decoded predictions pred_dev (device double [n][16]) per crossing:
 * presence probability, r_n, lambda_n, E_obs/E_em.  Asynchronous on `stream`.  Inference runs
 * on the kernel raptor_surrogate_kernel selects (tcgen05 by default, the 16 output sums
 * reduced in two rounds of 8; or mma.sync); a tensor-core wait that runs out is reported by
 * the next learned disk render that returns a spectrum (RAPTOR_ETIMEOUT).
 * RAPTOR_EUNSUPPORTED before init or set; RAPTOR_EINVAL for bad sizes or ranges. */
int raptor_crossings_param_count(void);
raptor_status raptor_crossings_generate(raptor_ctx* ctx, long long n, unsigned long long seed, double spin_min,
                                        double spin_max, double incl_min_deg, double incl_max_deg, float* inputs_dev,
                                        double* targets_dev, double* raw_dev, void* stream);
/* raptor_crossings_init: inputs_dev (device float [n][4], may be NULL) sets the spin and
 * inclination normalisation to the range of all n inputs, found on the device (else a in
 * [0, 1] and i in [5, 85] deg map to [-1, 1]); alpha and beta are normalised over the
 * camera's field of view.  RAPTOR_EINVAL for a non-finite spin or inclination input. */
raptor_status raptor_crossings_init(raptor_ctx* ctx, const float* inputs_dev, const double* targets_dev, long long n,
                                    unsigned long long seed, void* stream);
raptor_status raptor_crossings_train(raptor_ctx* ctx, const float* inputs_dev, const double* targets_dev, long long n,
                                     int steps, double lr, double lr_final, unsigned long long seed, double* loss_host,
                                     void* stream);
raptor_status raptor_crossings_grad(raptor_ctx* ctx, const float* inputs_dev, const double* targets_dev, long long n,
                                    float* grad_host, double* loss_host, void* stream);
raptor_status raptor_crossings_eval(raptor_ctx* ctx, const float* inputs_dev, long long n, double* pred_dev, void* stream);
raptor_status raptor_crossings_get(raptor_ctx* ctx, float* params_host, int n);
/* Fallback of raptor_disk_render_learned: pixel centres inside the critical curve or within
 * fallback_band M of it are integrated by the disk ray of raptor_disk_render [1.0].  The
 * learned disk's radius changes steeply across the image just outside the curve (rays
 * deflected behind the hole), so its band is wider than the volumetric render's
 * (raptor_surrogate_config).  fallback_df64 = 1 [default]: those rays' state, RK4 steps and
 * crossing refinement in double-float arithmetic (float pairs, ~48-bit significands, on the
 * FP32 pipe; the step length from the FP32 view of the state) and E_obs/E_em at the hit in
 * FP64; 0: in FP64, equal to raptor_disk_render bit for bit.  RAPTOR_EINVAL for a negative
 * or non-finite band or another flag value. */
raptor_status raptor_crossings_config(raptor_ctx* ctx, double fallback_band, int fallback_df64);

/* Confidence fallback of the learned thin disk (sec. 4.2.1 geometry; no counterpart in the
 * paper): a pixel whose decoding reads a presence logit within presence_margin of 0 [2.0],
 * or a predicted crossing radius within radius_margin of r_in or r_out in ln r [0.01], is
 * integrated by the fallback disk ray as well, because there a wrong decision of the network
 * (a false hit or a false miss) would be an O(1) intensity error.  0, 0: the band alone.
 * RAPTOR_EINVAL for a negative or non-finite margin. */
raptor_status raptor_crossings_confidence(raptor_ctx* ctx, double presence_margin, double radius_margin);
raptor_status raptor_crossings_set(raptor_ctx* ctx, const float* params_host, int n);

/* The thin disk of raptor_disk_render from the learned crossings (sec. 4.2.1): pixels whose
 * centre lies outside the critical curve and its fallback band (raptor_crossings_config)
 * take the first predicted crossing (presence probability > 1/2, in order) with r_in <= r_n
 * <= r_out: E_obs/E_em of the Keplerian emitter at the predicted r_n (closed form, exact given
 * the radius: 1 / (u^t (1 - Omega L)), L = -alpha sin i), intensity (E_obs/E_em)^4 r_n^-q,
 * order n + 1,
 * status 5 (6 without a hit), steps 0; the other pixels are integrated by the disk ray of
 * raptor_disk_render (in double-float arithmetic by default: raptor_crossings_config).  The network is valid inside the spin, inclination and field-of-view
 * range of its training data; the caller keeps the camera there.  Same arguments and
 * outputs; r_in must not lie inside the ISCO
 * (RAPTOR_EUNSUPPORTED), nor may the crossing network be missing (RAPTOR_EUNSUPPORTED), nor
 * may the camera's spin or inclination lie outside the network's training range (more than
 * 1 % of the range beyond it after the network's normalisation: RAPTOR_EUNSUPPORTED). */
raptor_status raptor_disk_render_learned(raptor_ctx* ctx, const raptor_disk_desc* d, double* ratio_dev,
                                         double* intensity_dev, int* order_dev, int* status_dev, int* steps_dev,
                                         double* profile_host, void* stream);

/* Per-kernel device time, measured with CUDA events recorded around every kernel launch on
 * the launch's own stream.  raptor_profile(ctx, 1) clears the accumulators and starts
 * recording; raptor_profile(ctx, 0) stops.  raptor_profile_read waits for the recorded
 * events and returns, per kernel slot RAPTOR_KERNEL_* (13 slots), the summed milliseconds
 * (ms[13], may be NULL) and the number of launches since the last clear (launches[13],
 * may be NULL; counted whether or not recording is on).  A scope times its kernels as one
 * interval (e.g. the network's two tensor-core kernels in RAPTOR_KERNEL_SURROGATE_MLP). */
#define RAPTOR_KERNEL_RENDER_FP64 0  /* persistent FP64 ray kernel                         */
#define RAPTOR_KERNEL_MIXED_A 1      /* mixed: FP32 phase on camera rays                   */
#define RAPTOR_KERNEL_MIXED_B 2      /* mixed: FP64 phase (inner region, turning points) of
                                        the first stream                                    */
#define RAPTOR_KERNEL_MIXED_C 3      /* mixed: FP32 phase on outbound rays                 */
#define RAPTOR_KERNEL_REDUCE 4       /* flux reduction (two launches per render)          */
#define RAPTOR_KERNEL_TRACE 5        /* single-ray trace                                   */
#define RAPTOR_KERNEL_LOAD 6         /* grid interleave at load time                       */
#define RAPTOR_KERNEL_PEAK 7         /* unused by the renders                              */
#define RAPTOR_KERNEL_SURROGATE 8    /* surrogate stage of a render without the network:   */
                                     /* inputs and fallback flags, start states (two scopes) */
#define RAPTOR_KERNEL_TRAIN 9        /* surrogate data generation and training             */
#define RAPTOR_KERNEL_SURROGATE_MLP 10 /* the network of the surrogate stage               */
#define RAPTOR_KERNEL_DISK 11        /* thin-disk rays and their spectrum                  */
#define RAPTOR_KERNEL_MIXED_B_LONG 12 /* mixed: FP64 phase of the near-critical rays (second
                                        stream); RAPTOR_KERNEL_MIXED_B has the other rays'  */
raptor_status raptor_profile(raptor_ctx* ctx, int enable);
raptor_status raptor_profile_read(raptor_ctx* ctx, double* ms, long long* launches);

/* Per-launch timeline of the recorded scopes since the last raptor_profile(ctx, 1), in
 * launch order: kernel slot (RAPTOR_KERNEL_*), lane (0: the call's stream, 1: the mixed
 * path's second stream), start relative to the first recorded scope and duration, both in
 * ms from CUDA events on the launch's stream.  Waits for the recorded events (as
 * raptor_profile_read, whose sums include the same scopes).  Writes min(cap, count) records
 * into the caller's host arrays slot[cap], lane[cap], start_ms[cap], dur_ms[cap] (may be
 * NULL when cap = 0) and the number of records held in *count (at most 65,536 are kept).
 * RAPTOR_EINVAL for a NULL count, a negative cap or NULL arrays with cap > 0. */
raptor_status raptor_profile_timeline(raptor_ctx* ctx, int cap, int* slot, int* lane, double* start_ms,
                                      double* dur_ms, int* count);

/* Self-check of the FP32 code paths' own arithmetic primitives over n inputs each:
 * max_ulp[5] (caller's host array) receives the largest distance in ulps from the reference
 * rounded to float of (0) the reciprocal (approximate reciprocal + one Newton-Raphson step)
 * against 1/v over +-2^-100 .. 2^101, (1) the square root against sqrtf and (2) the cube root
 * against the FP64 cube root over 2^-100 .. 2^101, (3) x / (e^x - 1) and (4) (1 - e^-x) / x
 * (series below 1, quotients above) against FP64 over 2^-40 .. 36.  Synchronises the
 * device.  RAPTOR_EINVAL for n < 1 or a NULL max_ulp.  The paper has no counterpart. */
raptor_status raptor_check_fp32_math(long long n, unsigned int* max_ulp);

/* FMA-chain microbenchmark on the current device: dependent FP64 (fp64 = 1) or FP32
 * (fp64 = 0) fused multiply-adds on every SM; *tflops = achieved rate (2 flops per FMA).
 * Measures the arithmetic ceiling used for the rooflines of the ray kernels. */
raptor_status raptor_measure_fma_peak(int fp64, double* tflops);

/* Allocation-free rendering (the paper has no counterpart).  Some callers cannot allocate
 * device memory: a host program whose own memory pool already holds the GPU's memory, or a
 * code path that must not call cudaMalloc/cudaFree after start-up because those calls can
 * synchronise the device.  raptor_render_noalloc renders like raptor_render (FP64 path,
 * analytic plasma) without any allocation: no context, no cudaMalloc/cudaFree, no
 * allocating library call.  The caller passes the descriptors, the host frequency array,
 * image_dev (device double [n_freq][ny][nx], Jy per pixel) and flux_dev (device double
 * [n_freq], may be NULL); work is enqueued on `stream` and the call returns without waiting.
 * The kernels' scratch (ray counters and partial flux sums) lives in one static device
 * array of RAPTOR_NOALLOC_SCRATCH_BYTES on every device that loads the library, held until
 * the process exits and shared by every call; each call clears what must start at zero.
 * Calls whose GPU work overlaps in time (other streams or host threads) race on that array:
 * the caller must serialise them.  The first call on a device looks up the array's device
 * address with that device current and loads every kernel this entry point can launch (with
 * lazy module loading, a kernel's first launch would otherwise load its code then, which can
 * allocate in the driver); make that first call before any stream capture.
 * Limits: cam->precision must be RAPTOR_FP64 (else RAPTOR_EINVAL); plasma->kind must be
 * RAPTOR_PLASMA_ANALYTIC (else RAPTOR_EUNSUPPORTED); 1 <= n_freq <= RAPTOR_NOALLOC_MAX_FREQ
 * (else RAPTOR_EINVAL).  Invalid descriptors return RAPTOR_EINVAL before any launch. */
#define RAPTOR_NOALLOC_MAX_FREQ 64
#define RAPTOR_NOALLOC_SCRATCH_BYTES 131584
raptor_status raptor_render_noalloc(const raptor_camera_desc* cam, const raptor_plasma_desc* plasma,
                                    const double* freqs_hz, int n_freq, double t_obs, double* image_dev,
                                    double* flux_dev, void* stream);

/* Message for the last failure on ctx ("" if none).  Valid until the next call on ctx. */
const char* raptor_last_error(const raptor_ctx* ctx);

/* Release the context and its device buffers (synchronises its device first). */
void raptor_destroy(raptor_ctx* ctx);

/* Library version: major * 10000 + minor * 100 + patch. */
int raptor_version(void);

#ifdef __cplusplus
}
#endif

#endif /* RAPTOR_H */
