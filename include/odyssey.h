/*
 * odyssey.h -- C ABI of the GB300 (sm_103a) library for backward ray tracing and
 * general-relativistic radiative transfer in Kerr spacetime, after Pu, Yun, Younsi &
 * Yoon 2016 ("Odyssey: a public GPU-based code for GRRT in Kerr spacetime").
 *
 * Units: G = c = M = 1 (Section 2).  Every traced photon has E = 1.
 *
 * Conventions shared by all calls
 *   - Pointers named *_dev are device pointers on the context's device; *_host are host
 *     pointers.  All output buffers are owned by the caller; the library owns only its
 *     context scratch (ray queue counters, statistics, scene table, error flag).
 *   - Calls that take a `stream` (a cudaStream_t, NULL = legacy default stream) are
 *     asynchronous on that stream; the caller must not reuse outputs before the stream
 *     reaches them.  Calls on one context must not overlap on different streams: the
 *     context's scratch is shared.
 *   - Every call returns an odx status code (0 = ODX_OK).  Invalid arguments are rejected
 *     before any launch with ODX_ERR_INVALID_ARG and leave outputs untouched; CUDA
 *     failures return ODX_ERR_CUDA.  odx_last_error() gives the message of the last failure
 *     on a context.  No C++ exception crosses this interface.
 *   - Per-ray outcomes are statuses in the ray record, not errors.
 */
#ifndef ODYSSEY_H
#define ODYSSEY_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ODX_MAX_FREQ 8

/* return codes */
#define ODX_OK 0
#define ODX_ERR_INVALID_ARG 1
#define ODX_ERR_CUDA 2
#define ODX_ERR_TIMEOUT 3
#define ODX_ERR_DEVICE_FLAG 4 /* a kernel raised its device error flag (see odx_stats) */
#define ODX_ERR_NO_DEVICE 5
#define ODX_ERR_UNSUPPORTED 6
#define ODX_ERR_TOO_LARGE 7 /* request exceeds a fixed capacity (odx_render_static) */

/* ray status written to odx_ray_record.status */
#define ODX_RUNNING 0
#define ODX_ESCAPED 1  /* moving outward beyond its starting radius              */
#define ODX_CAPTURED 2 /* r < horizon_factor * r_+                               */
#define ODX_DISK_HIT 3 /* crossed the equator with r_in <= r <= r_out (thin disk) */
#define ODX_MAXSTEPS 4 /* max_steps Runge-Kutta attempts without terminating     */
#define ODX_NUMERR 5   /* step size underflow (|h| < 1e-12) or non-finite state  */

/* emission models */
#define ODX_EMIT_NONE 0      /* geodesics only: grid projection, shadows (Sections 4.1-4.2) */
#define ODX_EMIT_THIN_DISK 1 /* opaque Keplerian equatorial disk, I = g^4 r^-q (Section 4.3) */
#define ODX_EMIT_TORUS 2     /* analytic thermal flow, radiative transfer Eqs. 30-31         */
#define ODX_EMIT_NT_DISK 3   /* Novikov-Thorne disk (Section 4.3): opaque like THIN_DISK; each
                                hit emits a blackbody at T(r) = T0 (8 pi F(r) / 3)^(1/4), F the
                                Page-Thorne flux for unit accretion rate, seen as B_nu(g T) at
                                the n_freq observed frequencies (n_freq image planes) */
#define ODX_EMIT_SYNCH 4     /* Keplerian shell of thermal synchrotron plasma (Section 4.5,
                                Eqs. 37-39) with Kirchhoff absorption, transfer Eqs. 30-31 in
                                CGS: freqs in Hz, n_freq image planes of I_nu in
                                erg s^-1 cm^-2 Hz^-1 sr^-1; n_e = n_e0 r^-ne_index
                                exp(-cos^2 theta / (2 theta_width^2)) cm^-3, Theta_e = k T_e /
                                m_e c^2 = T0 r^-T_index, B^2 / 8 pi = n_e m_p c^2 /
                                (6 beta_B r), emission for r <= r_out, lengths in
                                r_g = G mass / c^2; the flow is the torus's.  The printed
                                emissivity integrates over directions: the transfer uses
                                j_nu / 4 pi per steradian */
#define ODX_EMIT_SPOT 5      /* optically thick Keplerian hot spot (Section 4.4); the mixed
                                path takes FP64 steps within r_spot / 2 of it.  The centre
                                orbits the equatorial circle r = spot_r
                                (<= 0: r_ISCO) at Omega = 1/(r^1.5 + a), azimuth spot_phase +
                                Omega t; a photon seen at t_obs left its point at t_obs - dt
                                (dt: coordinate time along the ray); the spot is d < 4
                                spot_size, z > 0 in the pseudo-Cartesian coordinates x, y =
                                sqrt(r^2 + a^2) (cos, sin) phi, z = r cos theta; a ray ends
                                at its first entry (status ODX_DISK_HIT) and sees
                                C_norm exp(-d^2 / (2 spot_size^2)) B_nu(g T0) at the n_freq
                                frequencies (n_freq image planes; record intensity: the
                                bolometric value), g for gas co-rotating at Omega */

/* arithmetic of the integrator */
#define ODX_FP64 0  /* every stage in FP64                                             */
#define ODX_MIXED 1 /* FP32 stages in bulk, FP64 within r_switch, compensated sums     */

/* step control of the transfer equation (Section 2.3, Eqs. 30-31, integrated along with the
 * geodesic; the paper names no error norm for them).  In both modes the medium ends at the
 * stopping radius horizon_factor * r_+: no emission or absorption inside it, so a captured
 * ray's intensity does not depend on where its last step lands. */
#define ODX_RT_CONTROLLED 0 /* each invariant intensity I_k enters the Cash-Karp error norm
                               with the scale |I_k| + |h dI_k/ds| + 3e-5 B_nu(T0)/nu^3 (the
                               medium's source function at its temperature scale T0, seen
                               at nu_k); tau stays out (its error reaches I through
                               exp(-tau)).  Default.                                       */
#define ODX_RT_RIDE 1       /* only the geodesic components set the steps; tau and I ride
                               on them (intensities good to ~1e-3 - 1e-2 per pixel where
                               the emission varies faster than the geodesic)               */

/* direction reading of the traced photon */
#define ODX_CONV_PHYSICAL 0 /* the real outgoing photon traced back in affine time (default) */
#define ODX_CONV_LITERAL 1  /* Eqs. 24-26 taken as the velocity of the traced photon        */

/*
 * One image (Sections 2.2, 3 and 4).  Pixel (i, j), i along alpha, j along beta, sits at
 * alpha_i = alpha_min + (i + 1/2)(alpha_max - alpha_min)/n_alpha (same for beta); flat
 * pixel index p = j * n_alpha + i.  The observer is at (r_obs, theta_obs, phi_obs)
 * (Eqs. 18-19); the ray through a pixel leaves the image plane perpendicular to it.
 */
typedef struct odx_scene {
    double a;                       /* spin, |a| < 1                                    */
    double r_obs, theta_obs, phi_obs; /* observer distance (> 10 r_+), inclination in
                                       [0, pi], azimuth (radians)                      */
    double alpha_min, alpha_max, beta_min, beta_max; /* image window (M), min < max       */
    int32_t n_alpha, n_beta;        /* resolution, >= 1 each                             */
    int32_t emitter;                /* ODX_EMIT_*                                        */
    int32_t n_freq;                 /* torus: 1..ODX_MAX_FREQ observed frequencies      */
    double freqs[ODX_MAX_FREQ];     /* observed frequencies nu_obs (dimensionless)      */
    double r_in, r_out, q_emis;     /* thin disk edges (r_in <= 0: r_ISCO(a)), index q   */
    double ne_index, theta_width;   /* torus n_e = r^-ne_index exp(-cos^2 / (2 w^2))    */
    double T0, T_index;             /* torus T_e = T0 r^-T_index; NT disk: T0 scale     */
    double C_norm;                  /* torus emissivity normalisation (odx_torus_norm)  */
    double rtol;                    /* Cash-Karp relative tolerance (FP64 stages)       */
    double h0;                      /* first step in affine parameter                  */
    double hmax_frac;               /* |h| <= hmax_frac * r                             */
    double horizon_factor;          /* stop when r < horizon_factor * r_+ (> 1)         */
    int32_t max_steps;              /* cap on Runge-Kutta attempts per ray (>= 1)       */
    int32_t convention;             /* ODX_CONV_*                                        */
    int32_t precision;              /* ODX_FP64 or ODX_MIXED                             */
    int32_t rt_control;             /* ODX_RT_*: step control of the transfer equation   */
    double rtol_fp32;               /* ODX_MIXED: relative tolerance of the FP32 stages  */
    double r_switch;                /* ODX_MIXED: FP64 stages where r < r_switch         */
    double n_e0;                    /* synchrotron shell: n_e at r = 1 (cm^-3), > 0      */
    double beta_B;                  /* synchrotron shell: field parameter, > 0           */
    double mass;                    /* synchrotron shell: black-hole mass (M_sun), > 0   */
    double spot_r;                  /* hot spot: orbit radius (<= 0: r_ISCO)             */
    double spot_size;               /* hot spot: Gaussian width r_spot (> 0)             */
    double spot_phase;              /* hot spot: azimuth of the centre at t = 0          */
    double t_obs;                   /* hot spot: observer time of the image              */
} odx_scene;

/*
 * Per-ray result, 80 bytes, written once per ray with 16-byte vector stores
 * (the record array must be 16-byte aligned).
 *   r_cross, phi_cross: first equatorial crossing (NaN if none), Section 4.1.
 *   r_hit, phi_hit, g, intensity: thin-disk hit, g from Eq. 2 and I = g^4 r^-q (Section 4.3);
 *     NaN / 0 if the ray did not hit the disk.
 *   H_end: relative violation of the null condition at the end,
 *     (2 Sigma H) / (sum of the magnitudes of its terms);
 *   Q_drift: (Q_end - Q_0) / max(|Q_0|, 1), Carter constant Eq. 13.
 *   n_acc, n_rej: accepted and rejected Runge-Kutta steps (n_acc + n_rej = attempts).
 */
typedef struct odx_ray_record {
    int32_t status, n_acc, n_rej, n_cross;
    double r_cross, phi_cross;
    double r_hit, phi_hit, g, intensity;
    double H_end, Q_drift;
} odx_ray_record;

/* Launch shape of the tracing kernels (the default is {128, 3, 0, 2, 16}). */
typedef struct odx_launch {
    int32_t block;         /* threads per block, multiple of 32, 32..1024          */
    int32_t blocks_per_sm; /* resident blocks per SM the grid is sized for and the
                              register cap of the mixed tracer (2, 3 or 4) (>= 1)   */
    int32_t chunk;         /* rays a warp takes from the global queue at a time;
                              0: the default (32; mixed tracer with persistent 1: 8) */
    int32_t persistent;    /* 1: persistent warps refilling each finished lane from
                              the queue; 3: persistent warps that take 32 consecutive
                              rays once all their lanes are done (warp-coherent
                              queue); 0: one ray per thread, no queue; 2 (auto): 3,
                              with 4 blocks per SM for mixed launches of 2^18 rays or
                              more with up to 3 transfer slots and 3 otherwise      */
    int32_t fp64_batch;    /* ODX_MIXED: a warp runs an FP64 step once this many of
                              its lanes wait for one (or no FP32 lane is left), 1..32 */
} odx_launch;

/* Counters accumulated on the device by every tracing launch since the last reset. */
typedef struct odx_stats {
    int64_t rays;           /* rays finished                                        */
    int64_t steps_accepted; /* accepted Runge-Kutta steps                           */
    int64_t steps_rejected; /* rejected Runge-Kutta steps                           */
    int64_t steps_fp64;     /* attempts taken with FP64 stages (ODX_MIXED)           */
    int64_t lane_slots;     /* warp iterations x 32                                  */
    int64_t lane_active;    /* lanes holding a live ray summed over warp iterations */
    int32_t error_flag;     /* nonzero: a kernel met an invalid internal state     */
    int32_t reserved;
    int64_t trace_launches; /* tracing-kernel launches timed (odx_set_kernel_timing)    */
    double trace_ms;        /* their summed duration, CUDA events on the launch stream */
} odx_stats;

typedef struct odx_ctx odx_ctx;

/* Library version string. */
const char *odx_version(void);

/* Human-readable text of a return code. */
const char *odx_error_string(int32_t code);

/* Message of the last failure on ctx (empty string if none); valid until the next call. */
const char *odx_last_error(const odx_ctx *ctx);

/* Create a context on CUDA device `device` (ordinal) and allocate its scratch.
 * Returns ODX_ERR_NO_DEVICE if the device does not exist or is not sm_103. */
int32_t odx_create(odx_ctx **out, int32_t device);

/* Release the context and its scratch; NULL is accepted. */
int32_t odx_destroy(odx_ctx *ctx);

/* Set / read the launch shape (validated: see odx_launch). */
int32_t odx_set_launch(odx_ctx *ctx, const odx_launch *launch);
int32_t odx_get_launch(const odx_ctx *ctx, odx_launch *launch);

/*
 * Render n_scenes images in ONE launch (Section 3: one ray per pixel; the rays of all scenes
 * form one index range, handed to warps by a queue or one ray per thread as the launch
 * shape says, see odx_launch).  Per ray: initial state from the image plane (Section 2.2,
 * Eqs. 18-26, 7, 8, 4, 5, 13), adaptive Cash-Karp integration of the geodesic equations
 * (Section 2.1, Eqs. 4, 5, 9, 12, 14, 15), termination and disk crossing, redshift (Eq. 2)
 * and radiative transfer (Section 2.3, Eqs. 30-31).
 *   scenes_host:  n_scenes >= 1 scene descriptions (host memory, copied during the call).
 *                 All scenes of one call must share emitter, precision and, for the torus,
 *                 n_freq.
 *   records_dev:  sum_k n_alpha_k n_beta_k records, scene k's pixels after scene k-1's.
 *   image_dev:    sum_k nf_k n_alpha_k n_beta_k doubles (nf = n_freq for the torus, else 1),
 *                 scene by scene, each [nf][n_beta][n_alpha]: I_nu,obs = nu^3 * invariant I
 *                 for the torus, g^4 r^-q for the thin disk, 0 without emitter.  May be NULL.
 */
int32_t odx_render(odx_ctx *ctx, const odx_scene *scenes_host, int32_t n_scenes,
                   odx_ray_record *records_dev, double *image_dev, void *stream);

/*
 * Trace an explicit ray list (training data for the learned transfer function, fallback
 * pixels).  rays_dev[n][4] = (alpha, beta, a, cos i) in device memory; every other scene
 * parameter from proto_host (its window and resolution are ignored).  records_dev[n];
 * image_dev [nf][n] or NULL.  n == 0 is a no-op.
 */
int32_t odx_trace_rays(odx_ctx *ctx, const odx_scene *proto_host, const double *rays_dev,
                       int64_t n, odx_ray_record *records_dev, double *image_dev,
                       void *stream);

/*
 * odx_render with HOST output buffers: copies the scene table in, renders into context
 * buffers and copies records and image back to records_host / image_host (image_host may be
 * NULL).  Synchronous.  Pinned host memory makes the copies faster.  A single scene of 2^23
 * rays or more is rendered in two slabs of consecutive rays (one launch each over the same
 * scene table, so every ray is computed as in one launch): the last 7/8 of the rays first,
 * whose records and image rows are copied back on a second stream while the first 1/8
 * renders.
 */
int32_t odx_render_host(odx_ctx *ctx, const odx_scene *scenes_host, int32_t n_scenes,
                        odx_ray_record *records_host, double *image_host);

/* Read (stream-ordered, then synchronised) and optionally reset the device counters. */
int32_t odx_get_stats(odx_ctx *ctx, void *stream, odx_stats *out, int32_t reset);

/* Time every tracing-kernel launch of this context (CUDA events around the kernel on its
 * stream, reported by odx_get_stats) when on != 0; off by default.  Not during capture. */
int32_t odx_set_kernel_timing(odx_ctx *ctx, int32_t on);

/*
 * Spectra and light curves (Section 4.4: the light curve integrates the intensity over the
 * frequency bins of each image).  For the scene table of an odx_render call and the image
 * it wrote (image_dev, same layout: per scene [planes][n_beta][n_alpha], planes = n_freq
 * for the torus, else 1):
 *   flux_dev[k * planes + j] = sum over the pixels of scene k of I_j * dalpha * dbeta / r_obs^2,
 *     the flux density at the observer (intensity times steradian; dalpha = (alpha_max -
 *     alpha_min) / n_alpha, likewise dbeta), one entry per scene and plane;
 *   lum_dev[k] (if non-NULL) = trapezoid rule of F over the scene's frequencies (torus with
 *     n_freq >= 2), else the single plane's F.
 * Fixed-order reduction: results do not depend on the launch schedule.  Device pointers,
 * caller-owned, 8-byte aligned; asynchronous on `stream`; the context keeps a small scratch
 * buffer (plane table and chunk sums).  Scenes as for odx_render (same emitter and n_freq).
 */
int32_t odx_image_flux(odx_ctx *ctx, const odx_scene *scenes_host, int32_t n_scenes,
                       const double *image_dev, double *flux_dev, double *lum_dev,
                       void *stream);

/* Wait for `stream` with a deadline; ODX_ERR_TIMEOUT if it has not finished in timeout_s
 * seconds (the work keeps running), ODX_ERR_DEVICE_FLAG if a kernel raised its flag. */
int32_t odx_sync(odx_ctx *ctx, void *stream, double timeout_s);

/*
 * Emissivity normalisation of the analytic torus (host computation, no device work): the C
 * for which a static path along the equator from r_+ to r_outer has optical depth 1 at
 * frequency nu, i.e. C = 1 / int alpha_nu(r, pi/2)|_{C=1} dr (reading of "tau about 1 at the
 * middle frequency").  Returns NaN for invalid arguments.
 */
double odx_torus_norm(double a, double nu, double ne_index, double T0, double T_index,
                      double r_outer);

/*
 * FMA-chain microbenchmark of the FP32 (precision = ODX_MIXED) or FP64 (ODX_FP64) vector
 * pipe: writes the measured FLOP/s (FMA = 2 flops) of a full-device launch to *flops.
 * Used as the denominator of the integrator's roofline.  Synchronous.
 */
int32_t odx_fma_peak(odx_ctx *ctx, int32_t precision, double *flops);

/*
 * A render captured once as a CUDA graph (queue reset + tracing kernel) and replayed: the
 * batched many-image launch of the parameter sweep, repeated without per-call host work.
 * The scene table is uploaded at creation into memory the graph owns; every replay renders
 * the same scenes into the same records_dev / image_dev (layout as odx_render) with the
 * context's launch shape at creation.  Replays use the context's queue and statistics:
 * they must not overlap other work on the same context.  Destroy graphs before their
 * context.
 */
typedef struct odx_graph odx_graph;
int32_t odx_graph_create(odx_ctx *ctx, const odx_scene *scenes_host, int32_t n_scenes,
                         odx_ray_record *records_dev, double *image_dev, odx_graph **out);
int32_t odx_graph_launch(odx_graph *graph, void *stream);
int32_t odx_graph_destroy(odx_graph *graph);

/*
 * Launch-shape autotuner: renders the given scenes (keep them small: about 10^5 - 10^6 rays)
 * once per candidate shape (threads per block, resident blocks per SM, queue chunk, FP64
 * batch, persistent or not), times each with CUDA events on `stream`, sets the fastest on
 * the context and returns it in *best.  Allocates temporary outputs on the device.
 * Synchronous.
 */
int32_t odx_autotune(odx_ctx *ctx, const odx_scene *scenes_host, int32_t n_scenes,
                     void *stream, odx_launch *best);

/*
 * Learned thin-disk transfer function (the surrogate): an MLP
 * (alpha/20, beta/20, a, cos i) -> (capture logit, ln r, phi / pi, g) with 4 hidden layers
 * of 256 SiLU units, BF16 weights and activations, FP32 accumulation, trained on rays the
 * integrator traces.  (r, phi) is the disk hit for rays that stop on the thin disk, else
 * the first equatorial crossing; g the disk redshift (Eq. 2) at the hit.
 * Parameters (FP32 master copy, flat, ODX_MLP_PARAMS floats): W1[4][256], b1[256], then for
 * each of the three 256 x 256 layers W[256][256] (row = input unit), b[256], then
 * W5[256][4], b5[4].  Weights enter the kernels rounded to BF16; biases are added in FP32.
 * Loss over a batch of n rows with targets t[n][8] = (captured, ln r, phi / pi, g,
 * mask_cross, mask_g, 0, 0):  mean over rows of
 *   BCE(logit, captured) + mask_cross ((y1 - t1)^2 + (y2 - t2)^2) + mask_g (y3 - t3)^2.
 * Training uses Adam (beta1 0.9, beta2 0.999, eps 1e-8).  The paper has no learned
 * component; this is the surrogate of the thin-disk images of Section 4.3.
 */
#define ODX_MLP_IN 4
#define ODX_MLP_HIDDEN 256
#define ODX_MLP_DEPTH 4
#define ODX_MLP_OUT 4
#define ODX_MLP_PARAMS 199684
typedef struct odx_mlp odx_mlp;
/* max_batch: rows per training step / inference chunk (rounded up to 128, <= 2^22). */
int32_t odx_mlp_create(odx_ctx *ctx, int64_t max_batch, uint64_t seed, odx_mlp **out);
int32_t odx_mlp_destroy(odx_mlp *mlp);
int32_t odx_mlp_get_params(odx_mlp *mlp, float *params_host);
int32_t odx_mlp_set_params(odx_mlp *mlp, const float *params_host); /* resets Adam state */
/* y_dev[n][4] = MLP(x_dev[n][4]), any n, on the tensor cores (tcgen05: 128-row tiles, the
 * FP32 accumulators and the BF16 activations in tensor memory); x_dev and y_dev 16-byte
 * aligned (else INVALID_ARG).
 * Asynchronous on `stream`.  A tensor-core wait that times out leaves its tile's outputs
 * unwritten and raises a device flag, reported (and cleared) as ODX_ERR_DEVICE_FLAG by the
 * next odx_mlp_get_params, odx_mlp_gradients or odx_surrogate_render call. */
int32_t odx_mlp_forward(odx_mlp *mlp, const float *x_dev, int64_t n, float *y_dev, void *stream);
/* Test hook for the tensor-core kernels' failure path: the number of polls after which a
 * wait inside the tile loop of the forward and backward chains (odx_mlp_forward,
 * odx_mlp_train_step, odx_mlp_gradients) gives up; 0 restores the default, 2^20 polls (the
 * inference kernel sleeps up to 1 us in each poll of 4,096 or more, and not below).  A
 * kernel that gives up raises the device flag and returns after waiting, with the default
 * limit, for its own copies and MMAs in flight and freeing its tensor memory; the flag is
 * reported as above.  No counterpart in the paper. */
int32_t odx_mlp_set_wait_limit(odx_mlp *mlp, uint32_t tries);
/* Training rows: x_dev[n][4] = (alpha / 20, beta / 20, a, cos i), 16-byte aligned;
 * t_dev[n][8] as written by odx_mlp_targets (captured flag, log r_cross, phi_cross / pi, g,
 * crossing mask, g mask, 0, 0), 16-byte aligned.  Both device pointers, caller-owned.
 * Loss and gradients (dL/dparams, layout as the parameters) of one batch, n a multiple of
 * 128 and <= max_batch; synchronous, results copied to host (either may be NULL); returns
 * ODX_ERR_DEVICE_FLAG if a tensor-core wait timed out in this or an earlier call. */
int32_t odx_mlp_gradients(odx_mlp *mlp, const float *x_dev, const float *t_dev, int64_t n,
                          float *grad_host, float *loss_host);
/* One Adam step on a batch (n a multiple of 128, <= max_batch; x_dev, t_dev as above);
 * loss_dev: 1 float or NULL.  Asynchronous on `stream`; a tensor-core time-out is reported
 * by the next odx_mlp_get_params or odx_mlp_gradients call. */
int32_t odx_mlp_train_step(odx_mlp *mlp, const float *x_dev, const float *t_dev, int64_t n,
                           float lr, float *loss_dev, void *stream);
/* Inputs and targets from traced rays (odx_trace_rays with a thin-disk prototype):
 * x_dev[n_pad][4], t_dev[n_pad][8] with n_pad = n rounded up to 128 (padding rows zero);
 * crossings beyond r_max are masked. */
int32_t odx_mlp_targets(odx_ctx *ctx, const odx_ray_record *records_dev, const double *rays_dev,
                        int64_t n, double r_max, float *x_dev, float *t_dev, void *stream);
/*
 * Surrogate render of a thin-disk scene into image_dev[n_beta][n_alpha]: the MLP classifies
 * every pixel; pixels within `band` (M) of the Bardeen critical curve along their polar
 * angle, or with capture probability in [p_lo, p_hi], fall back to the ray tracer (the
 * scene's precision), whose records go to fallback_records_dev (capacity n_alpha*n_beta),
 * their flat pixel indices to fallback_pixels_dev (same capacity; may be NULL), and whose
 * intensities replace the surrogate's.  *n_fallback = number of fallback rays.
 * Synchronous (the fallback count is read back to size the tracer launch).
 */
int32_t odx_surrogate_render(odx_mlp *mlp, const odx_scene *scene_host, double band, double p_lo,
                             double p_hi, odx_ray_record *fallback_records_dev,
                             int64_t *fallback_pixels_dev, double *image_dev,
                             int64_t *n_fallback, void *stream);

/*
 * odx_render without any device allocation, for callers that must not call cudaMalloc:
 * code whose device memory is owned entirely by another allocator (a framework's caching
 * pool, or a fixed budget reserved at start-up) and which must not allocate behind that
 * allocator's back, such as a renderer embedded as a plug-in in a host application or a
 * serving loop that forbids allocation after warm-up.  The paper has no counterpart; this
 * is a deployment variant of odx_render.
 *
 * The ray queue counter, the device statistics and the scene table live in one file-scope
 * device array of 45,056 bytes that every GPU loading this library holds until the process
 * exits; at most ODX_STATIC_MAX_SCENES scenes per call (more: ODX_ERR_TOO_LARGE, nothing
 * launched).  The caller still provides the outputs (records_dev, image_dev, same layout
 * as odx_render) and the scene descriptions in host memory.  The call works on the calling
 * thread's current device.  Its first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) and sets the FP64 tracer's shared-memory limit, with that device
 * current; make that first call before any stream capture.  The call allocates no device
 * memory and frees none, and copies the scene table into the array with a stream-ordered
 * copy from a buffer on its own stack; while `stream` is capturing a graph it returns
 * ODX_ERR_UNSUPPORTED and does nothing (a replay would copy from that stack frame after the
 * call has returned).
 *
 * Every call shares the one array, which keeps the previous call's contents (the counter is
 * cleared on each call): calls whose work overlaps on the GPU (on different streams, or
 * from different threads without ordering) race and give wrong results; order them on one
 * stream.  Same argument checks and return codes as odx_render, without odx_last_error text.
 */
#define ODX_STATIC_MAX_SCENES 64
int32_t odx_render_static(const odx_scene *scenes_host, int32_t n_scenes,
                          odx_ray_record *records_dev, double *image_dev, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* ODYSSEY_H */
