/*
 * mcao.h -- C ABI of the GB300 MCAO closed-loop step library (libmcao.so).
 *
 * The library advances an end-to-end multi-conjugate adaptive optics Monte-Carlo loop one
 * time step at a time, as described in arXiv:1608.00386 ("The numerical simulation tool for
 * the MAORY multiconjugate adaptive optics system"):
 *   - frozen-flow turbulence layers, static screens translated by the wind
 *     ("The atmospheric layers generation");
 *   - open-loop wavefront along each guide star by geometric projection, laser guide stars at
 *     finite distance ("The open loop wave-front measurements");
 *   - DMs as linear combinations of analytic (Gaussian) influence functions
 *     ("Influence function and modal base");
 *   - Shack-Hartmann X/Y slopes of the residual phase (open-loop wavefront minus DMs), the
 *     slope vector times the control matrix giving differential commands added to the mirror
 *     shape, pure integrator ("The closed loop");
 *   - science PSF at a user wavelength and Strehl ratio ("The Point Spread Functions (PSFs)").
 * Every stage runs in the library's own CUDA kernels for sm_103a.
 *
 * Conventions
 *   - Every call returns mcao_status; no C++ exception crosses the boundary.  On failure the
 *     handle keeps a message readable with mcao_last_error() until the next failing call.
 *   - A handle is not thread-safe: use it from one host thread at a time.
 *   - Arrays are row-major, [y][x] with x fastest.  Phases are in radians at the reference
 *     wavelength cfg.lambda_ref (500 nm in the shipped configurations); DM surfaces and commands
 *     use the same unit (wavefront-equivalent radians).
 *   - Pupil sample i of a grid of n samples across the diameter D sits at (i - (n-1)/2) D/n;
 *     the pupil amplitude is 1 for obstruction*D/2 <= r <= D/2 and 0 elsewhere.
 *   - Host pointers are read during the call and not kept, unless a struct says on_device = 1,
 *     in which case the pointer is a device address that the caller keeps valid until
 *     mcao_sim_destroy (the library adopts it without copying).
 *   - Output buffers are host memory of the stated capacity n (in elements); a smaller n gives
 *     MCAO_E_SHAPE.  mcao_query() returns the element count each getter needs.
 *   - Work is queued on library-owned CUDA streams.  mcao_set_stream() names a caller stream
 *     (for example PyTorch's current stream) that every call orders itself after and that
 *     waits for the call's device work.  Getters synchronise before returning.
 */
#ifndef MCAO_H
#define MCAO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    MCAO_OK = 0,
    MCAO_E_INVALID_ARG = 1,   /* null pointer, non-finite or out-of-range value              */
    MCAO_E_SHAPE = 2,         /* size or count does not match the configuration             */
    MCAO_E_STATE = 3,         /* call out of order (e.g. step before every load_*)          */
    MCAO_E_CUDA = 4,          /* a CUDA runtime call failed; message holds its error string */
    MCAO_E_OOM = 5,           /* device allocation failed                                   */
    MCAO_E_TIMEOUT = 6,       /* a bounded device-side wait gave up                         */
    MCAO_E_UNSUPPORTED = 7    /* valid request that this build has no kernel for            */
} mcao_status;

enum { MCAO_WFS_NGS = 0, MCAO_WFS_LGS = 1 };
/* Element format of the stored control matrix (mcao_load_reconstructor, mcao_quantize_rows):
 * float32; bfloat16 (round to nearest even); FP8 E4M3 in the OCP 8-bit format (round to nearest
 * even, saturating to +-448) with one float32 scale per row, scale = max|row| / 448 (1 for an
 * all-zero row, and for a row whose max|row| / 448 is below the smallest normal float 2^-126: its
 * entries are then stored as zero).  The product always accumulates in float32 against float32
 * slopes. */
enum { MCAO_DTYPE_F32 = 0, MCAO_DTYPE_BF16 = 1, MCAO_DTYPE_FP8_E4M3 = 2 };

/* One Shack-Hartmann wavefront sensor.  Its pupil grid has n_sub * n_px samples across D.
 * Each valid subaperture (illuminated fraction >= valid_thr) forms an n_fft x n_fft spot
 * (zero-padded field, requires n_fft >= 2 n_px), binned n_bin x n_bin into
 * (n_fft/n_bin)^2 detector pixels.  Sodium elongation (laser stars, na_fwhm > 0): Gaussian of
 * FWHM b * na_fwhm / height^2 rad along the launch-to-subaperture direction, b that
 * distance.  Flux: n_photons times the illuminated fraction per frame.  Supported shapes
 * (n_px, n_fft, n_bin), each with or without elongation: (8, 16, 2), (8, 32, 2), (8, 16, 1) on
 * the warp-per-subaperture autocorrelation route; (16, 32, 2) (a laser star with twice the field
 * of view of 8 samples) and (32, 64, 4) on the block-per-subaperture FFT route. */
typedef struct {
    int type;                 /* MCAO_WFS_NGS (source at infinity) or MCAO_WFS_LGS           */
    int n_sub, n_px, n_fft, n_bin;
    double theta_x, theta_y;  /* direction, rad                                              */
    double height;            /* laser star height above the telescope, m                    */
    double lambda;            /* sensing wavelength, m                                        */
    double n_photons;         /* photons per fully illuminated subaperture per frame         */
    double read_noise;        /* e- rms per detector pixel                                    */
    double valid_thr;         /* minimum illuminated fraction                                 */
    double na_fwhm;           /* sodium layer FWHM thickness, m (0: no elongation)            */
    double launch_x, launch_y;/* launch position in the pupil, m                             */
} mcao_wfs;

/* One science direction: n_px pupil samples across D, PSF FFT of pad * n_px points (pixel
 * lambda / (pad D)), on-axis Strehl |sum A e^{i phi}|^2 / (sum A)^2 every step. */
typedef struct {
    int n_px, pad;
    double theta_x, theta_y;  /* rad                                                          */
    double lambda;            /* m                                                            */
} mcao_science;

typedef struct {
    size_t struct_size;       /* sizeof(mcao_config), checked                                 */
    double D;                 /* telescope diameter, m                                        */
    double obstruction;       /* central obstruction, fraction of D                           */
    double lambda_ref;        /* wavelength of the phase unit, m                              */
    double dt;                /* loop period, s                                               */
    double gain;              /* integrator gain g in c <- c + g R s                          */
    uint64_t seed;            /* Philox key of the detector noise                             */
    int noise;                /* 1: photon + read noise on the detector frames                */
    int psf_every;            /* accumulate the PSF every psf_every steps (0: never)          */
    int keep_frames;          /* 1: keep the last step's intensities and frames (tests)       */
    int n_wfs;
    const mcao_wfs* wfs;
    int n_sci;
    const mcao_science* sci;
    int n_real;               /* independent realizations advanced together (>= 1): each has
                                 its own screens, commands, noise key seed + r, slopes and
                                 Strehl / PSF accumulators; geometry and the reconstructor are
                                 shared.  With n_real > 1 one step forms the product for all
                                 realizations at once as a matrix product R S: a bfloat16 R on
                                 the tensor cores (64 realizations per pass over R), an FP8
                                 E4M3 R there too (its code values, exact in bfloat16, with the
                                 row scales applied after the sum), a float32 R on the CUDA
                                 cores (16 per pass) */
} mcao_config;

/* A periodic n x n phase screen with square samples of pixel_m metres, at altitude alt_m,
 * moving so that step k samples it shifted by (k dt)(vx, vy) metres. */
typedef struct {
    int n;
    double pixel_m, alt_m, vx, vy;
    const float* phase;       /* [n][n] rad at lambda_ref                                     */
    int on_device;
} mcao_layer;

/* A DM conjugated at alt_m: nx * ny actuators at pitch_m (actuator a at
 * (a - (nx-1)/2) pitch), Gaussian influence functions with g(pitch) = coupling; the surface is
 * held on a surf_n x surf_n grid of pitch surf_dx centred on the axis and sampled bilinearly
 * (indices clamped to the grid).  Commands of the valid actuators, in row-major order, form
 * this DM's block of the command vector; blocks follow the DM order. */
typedef struct {
    double alt_m, pitch_m, coupling;
    int nx, ny;
    const uint8_t* valid;     /* [ny][nx] host array, nonzero = valid actuator                */
    int surf_n;
    double surf_dx;
} mcao_dm;

typedef struct mcao_sim mcao_sim;

/* What mcao_query() sizes. */
typedef enum {
    MCAO_Q_SLOPES = 0,        /* length of the slope vector                                   */
    MCAO_Q_COMMANDS = 1,      /* length of the command vector (after mcao_load_dms)           */
    MCAO_Q_VALID = 2,         /* valid subapertures of WFS `index`                            */
    MCAO_Q_FRAME = 3,         /* detector pixels of WFS `index` (valid subaps x n_det^2)      */
    MCAO_Q_WFS_PHASE = 4,     /* pupil samples of WFS `index`                                 */
    MCAO_Q_DM_SURFACE = 5,    /* surface samples of DM `index`                                */
    MCAO_Q_PSF = 6,           /* PSF pixels of science direction `index`                      */
    MCAO_Q_STATE = 7,         /* bytes of a checkpoint                                        */
    MCAO_Q_REALIZATIONS = 8   /* realizations advanced together (cfg.n_real)                  */
} mcao_query_kind;

/* Create a simulation for a configuration ("Numerical Simulation Tool": the high-level system
 * configuration).  Validates it, derives pupils and valid subapertures, allocates device
 * state.  *out receives the handle (NULL on failure).  Errors: MCAO_E_INVALID_ARG,
 * MCAO_E_UNSUPPORTED (no kernel for a WFS shape), MCAO_E_CUDA, MCAO_E_OOM. */
mcao_status mcao_sim_create(const mcao_config* cfg, mcao_sim** out);

/* Free every device and host resource of the handle (NULL is accepted). */
mcao_status mcao_sim_destroy(mcao_sim* sim);

/* Message of the last failing call on this handle ("" if none); valid until the next call. */
const char* mcao_last_error(const mcao_sim* sim);

/* Message of the last mcao_sim_create failure in this thread. */
const char* mcao_create_error(void);

/* Order every later call after work queued on `stream` (a cudaStream_t, NULL = legacy
 * default stream) and make that stream wait for each call's device work. */
mcao_status mcao_set_stream(mcao_sim* sim, void* stream);

/* Load the turbulence layers ("The atmospheric layers generation"): copies each screen to the
 * device (or adopts it when on_device = 1).  Replaces previously loaded layers.  Errors:
 * MCAO_E_INVALID_ARG (n < 2, pixel <= 0, null phase), MCAO_E_OOM, MCAO_E_CUDA. */
mcao_status mcao_load_atmosphere(mcao_sim* sim, int n_layers, const mcao_layer* layers);

/* Load the DMs ("Influence function and modal base"): actuator maps, influence-function
 * tables and surface buffers; resets the commands to zero.  Errors: MCAO_E_INVALID_ARG,
 * MCAO_E_OOM, MCAO_E_CUDA. */
mcao_status mcao_load_dms(mcao_sim* sim, int n_dms, const mcao_dm* dms);

/* Load the control matrix R [n_cmd][n_slopes] (row-major float32) and the reference slopes
 * s_ref [n_slopes] (NULL = zeros) ("Control Matrix"; "The calibration of the interaction
 * matrices": reference slope vector).  The library keeps its own copy in a padded layout.
 * on_device = 1: R and s_ref are device addresses; the call first waits for all work queued
 * on the device, so the kernel producing R may still be running when it is made.  Errors:
 * R is always given in float32; dtype selects the format the library stores and streams
 * (MCAO_DTYPE_F32, MCAO_DTYPE_BF16 or MCAO_DTYPE_FP8_E4M3, converted once here).
 * Errors: MCAO_E_STATE (DMs not loaded), MCAO_E_SHAPE (n_cmd or n_slopes differ from the
 * configuration), MCAO_E_UNSUPPORTED (unknown dtype), MCAO_E_OOM, MCAO_E_CUDA. */
mcao_status mcao_load_reconstructor(mcao_sim* sim, int n_cmd, int n_slopes, const float* R,
                                    const float* s_ref, int dtype, int on_device);

/* Advance the closed loop n_steps steps ("The closed loop"): for step k, DM surfaces from
 * c_k, residual phase along every guide star, Shack-Hartmann frames (photon and read noise if
 * enabled), centre-of-gravity slopes s_k minus s_ref, science Strehl (and PSF every psf_every
 * steps), then c_{k+1} = c_k + gain R s_k.  Asynchronous: returns once the work is queued.
 * Errors: MCAO_E_STATE (a load_* missing), MCAO_E_INVALID_ARG (n_steps < 0), MCAO_E_CUDA. */
mcao_status mcao_step(mcao_sim* sim, int n_steps);

/* Wait for all queued work of the handle. */
mcao_status mcao_sync(mcao_sim* sim);

/* Element count (bytes for MCAO_Q_STATE) a getter needs; index selects the WFS, DM or
 * science direction.  Errors: MCAO_E_INVALID_ARG (bad kind or index), MCAO_E_STATE. */
mcao_status mcao_query(const mcao_sim* sim, int kind, int index, size_t* n);

/* Number of completed steps. */
mcao_status mcao_get_step_index(mcao_sim* sim, int64_t* k);

/* Last slopes s_k (pixels, reference subtracted): for each WFS in order, the x slopes of its
 * valid subapertures in row-major subaperture order, then their y slopes. */
mcao_status mcao_get_slopes(mcao_sim* sim, float* out, size_t n);

/* Current commands c (after the last step's update). */
mcao_status mcao_get_commands(mcao_sim* sim, float* out, size_t n);

/* Overwrite the commands (calibration pokes, tests). */
mcao_status mcao_set_commands(mcao_sim* sim, const float* in, size_t n);

/* Row-major subaperture index sy*n_sub+sx of every valid subaperture of WFS `wfs`. */
mcao_status mcao_get_valid(mcao_sim* sim, int wfs, int32_t* out, size_t n);

/* Residual phase of WFS `wfs` on its full pupil grid at the current step index and commands
 * (layers minus DMs, radians at lambda_ref), evaluated by the propagation kernel. */
mcao_status mcao_get_wfs_phase(mcao_sim* sim, int wfs, float* out, size_t n);

/* Surface of DM `dm` for the current commands (radians at lambda_ref). */
mcao_status mcao_get_dm_surface(mcao_sim* sim, int dm, float* out, size_t n);

/* Last step's detector data of WFS `wfs`, [valid subap][n_det][n_det]: noise-free expected
 * photo-electrons lambda (float) and, with noise on, the integer frames.  Needs
 * keep_frames = 1 (else MCAO_E_STATE).  Either pointer may be NULL. */
mcao_status mcao_get_frames(mcao_sim* sim, int wfs, float* lambda, int32_t* frames, size_t n);

/* Long-exposure PSF of science direction `sci` ([pad n_px]^2, centred, divided by the
 * diffraction-limited peak and by the number of accumulated frames, so a perfect wavefront
 * peaks at 1), the long-exposure Strehl (mean of the per-step on-axis Strehl) and the last
 * step's Strehl.  out may be NULL to read only the Strehl values. */
mcao_status mcao_get_psf(mcao_sim* sim, int sci, double* out, size_t n, double* sr_long,
                         double* sr_last);

/* Strehl ratio by the Marechal approximation ("The Point Spread Functions (PSFs)": Strehl on
 * the closed-loop wavefront history) of science direction `sci` (current realization): each
 * step's residual phase at the science wavelength, piston removed and weighted by the pupil
 * amplitude, has variance s2_k; *sr_long = exp(-mean_k s2_k), *sr_last = exp(-s2_last).
 * Either pointer may be NULL.  Errors: MCAO_E_INVALID_ARG. */
mcao_status mcao_get_marechal(mcao_sim* sim, int sci, double* sr_long, double* sr_last);

/* Reset the PSF and Strehl accumulators (for example after a convergence period). */
mcao_status mcao_reset_psf(mcao_sim* sim);

/* Checkpoint: step index, commands, last slopes, PSF and Strehl accumulators.  Noise is
 * counter-based on (seed, step, WFS, pixel), so resuming from a checkpoint reproduces the
 * same frames.  buf needs mcao_query(MCAO_Q_STATE) bytes. */
mcao_status mcao_get_state(mcao_sim* sim, void* buf, size_t n);
mcao_status mcao_set_state(mcao_sim* sim, const void* buf, size_t n);

/* Reconstructor update without device allocation: c <- c + gain * R s on the current device,
 * queued on `stream` (a cudaStream_t; NULL = legacy default stream).  The paper has no
 * counterpart: it is a service for callers that cannot allocate device memory -- for example a
 * real-time controller that reserves all of its memory at start-up and must never block on the
 * allocator inside its loop, or code that runs under another framework's memory pool where a
 * stray cudaMalloc would fragment or oversubscribe that pool.  It needs no mcao_sim handle and
 * calls no cudaMalloc, cudaFree or allocating library routine.
 *   R      device pointer, row-major [n_cmd][ld] float32, 16-byte aligned; ld >= n_slopes and
 *          ld a multiple of 4; columns n_slopes..ld-1 are never read (they may hold anything).
 *   s      device pointer, [n_slopes] float32.     c  device pointer, [n_cmd] float32, updated.
 *   err    optional host buffer of err_len bytes that receives a message on failure.
 * Split-K partial sums live in one fixed device array of 524288 floats (2 MiB) inside the
 * library, created on every device that loads the library and kept until the process exits;
 * n_cmd times ceil(n_slopes / 4096) must not exceed that size, and ceil(n_slopes / 4096) must
 * not exceed 65535 (else MCAO_E_SHAPE, nothing is launched).  A CUDA error already pending
 * when the call is made (left by the caller's earlier work) is returned as MCAO_E_CUDA with
 * that error's text, before anything is launched.  Each partial sum is written before it is read, so nothing needs clearing between
 * calls.  The first call on a device looks up the array's device address (cudaGetSymbolAddress,
 * under a lock); make that first call before any stream capture.  All calls share the array:
 * calls whose kernels overlap on the GPU (different streams, or concurrent host threads on
 * different streams) race on it -- order them on one stream.  Asynchronous: returns once the two
 * kernels are queued.  Errors: MCAO_E_INVALID_ARG, MCAO_E_SHAPE, MCAO_E_UNSUPPORTED (device
 * index >= 64), MCAO_E_CUDA. */
mcao_status mcao_reconstruct_noalloc(const float* R, int n_cmd, int n_slopes, int ld, const float* s,
                                     float* c, float gain, void* stream, char* err, size_t err_len);

/* Convert a float32 matrix to the stored reduced formats, as mcao_load_reconstructor does (no
 * counterpart in the paper; exposed so that callers and tests can inspect the codes).
 *   R      device pointer, row-major [rows][ld] float32, ld >= cols.
 *   dtype  MCAO_DTYPE_BF16 (codes: uint16 per element) or MCAO_DTYPE_FP8_E4M3 (uint8 per element).
 *   codes  device pointer, row-major [rows][cols] codes, 16-byte aligned; cols must be a multiple
 *          of 8 (BF16) or 16 (FP8 E4M3).
 *   scales device pointer [rows] float32: written for FP8 E4M3 (max|row| / 448; 1 for a zero row or a
 *          row whose max|row| / 448 is below 2^-126, whose codes are then zero);
 *          may be NULL for BF16.
 *   stream CUDA stream (cudaStream_t) or NULL for the legacy stream; the call only queues work.
 * err receives a message on failure (err_len bytes, may be NULL).  Errors: MCAO_E_INVALID_ARG
 * (null pointers, rows < 0, ld < cols), MCAO_E_SHAPE (cols not a multiple of the vector width,
 * codes not 16-byte aligned), MCAO_E_UNSUPPORTED (dtype), MCAO_E_CUDA. */
mcao_status mcao_quantize_rows(const float* R, int rows, int cols, int ld, int dtype, void* codes,
                               float* scales, void* stream, char* err, size_t err_len);

/* Sodium layer evolution ("The closed loop": the sodium layer temporal evolution): from the
 * next step on, laser sensor `wfs` sees the layer at `height` m (its cone projection) with
 * thickness `na_fwhm` m (its elongation).  Call between steps to follow a profile in time.
 * Errors: MCAO_E_INVALID_ARG (not a laser sensor, height not above every layer, negative
 * thickness), MCAO_E_UNSUPPORTED (elongation on a sensor without an elongated-spot kernel). */
mcao_status mcao_set_sodium(mcao_sim* sim, int wfs, double height, double na_fwhm);

/* Controller ("The closed loop": a pure integrator or a second-order low-pass filter), read as
 * the recursion per command c_{k+1} = a1 c_k + a2 c_{k-1} + b0 dc_k + b1 dc_{k-1}, dc_k = R s_k,
 * for every realization.  The default is the pure integrator c_{k+1} = c_k + gain dc_k
 * (equivalent to (1, 0, gain, 0)).  A low-pass-filtered integrator with filter constant beta is
 * (2 - beta, -(1 - beta), gain beta, 0).  The filter's memory restarts from the current
 * commands and a zero update (also after mcao_set_commands for that realization); the
 * checkpoint keeps it.  Errors: MCAO_E_INVALID_ARG (non-finite), MCAO_E_STATE (DMs not loaded). */
mcao_status mcao_set_controller(mcao_sim* sim, double a1, double a2, double b0, double b1);

/* Select the realization (0 <= r < n_real, default 0) that later calls address: the screens
 * given to mcao_load_atmosphere, and the slopes, commands (get and set), WFS phase, DM
 * surfaces, frames and PSF / Strehl read back.  mcao_step, mcao_reset_psf and the checkpoint
 * cover every realization.  No counterpart in the paper: its tool runs one realization per
 * process.  Errors: MCAO_E_INVALID_ARG (r out of range). */
mcao_status mcao_set_realization(mcao_sim* sim, int r);

/* Phase screen of a turbulent layer on the device ("The atmospheric layers generation"): the
 * FFT method on the periodic n x n grid of pitch pixel_m with the von Karman spectrum
 * PSD(kappa) = 0.023 r0^(-5/3) (kappa^2 + L0^-2)^(-11/6) (kappa in cycles/m, no DC term), the
 * complex Gaussian coefficients drawn from Philox4x32-10 (counter (index, 0, 0, 1), key seed,
 * Box-Muller pair of the detector-noise sampler); the screen is the real part of the
 * unnormalized inverse DFT, in rad at the wavelength r0 refers to.
 *   out    device pointer, row-major [n][n] float32.
 *   stream CUDA stream (cudaStream_t) or NULL; temporaries (8 n^2 + 8 n bytes) are allocated
 *          and freed in stream order.  Call outside stream capture (sets a kernel attribute).
 * Errors: MCAO_E_INVALID_ARG (null out, non-positive or non-finite pixel / r0 / L0),
 * MCAO_E_SHAPE (n outside [2, 4096] or not a product of 2, 3 and 5), MCAO_E_UNSUPPORTED,
 * MCAO_E_CUDA.  err receives a message on failure (err_len bytes, may be NULL). */
mcao_status mcao_generate_screen(int n, double pixel_m, double r0_m, double L0_m, uint64_t seed, float* out,
                                 void* stream, char* err, size_t err_len);

/* Misregistration of DM `dm` ("Conclusions": rotation of the DM and its modal basis with respect
 * to the sensors; also translation and magnification): the DM moves as a rigid body, its
 * surface at beam coordinates p being the aligned surface at q = R(-rotation)(p - shift) / mag
 * (shift in m at the DM's conjugate altitude, rotation in rad counter-clockwise, magnification
 * of actuator pitch and influence width).  Applies to every later step, measurement and
 * interaction matrix; (0, 0, 0, 1) restores the nominal DM.  Without rotation the transform is
 * folded into the separable Gaussian tables; with rotation the DM kernel evaluates every surface
 * sample against the actuators around q (slower).  Errors: MCAO_E_INVALID_ARG (bad index,
 * non-finite values, |rotation| > pi, magnification outside (0.5, 2)), MCAO_E_STATE (DMs not
 * loaded), MCAO_E_UNSUPPORTED (too many actuators per surface tile), MCAO_E_CUDA. */
mcao_status mcao_set_misregistration(mcao_sim* sim, int dm, double shift_x, double shift_y, double rotation,
                                     double magnification);

/* Self-check of the device-side timeouts: launches one bounded mbarrier wait that nothing
 * satisfies (the wait the reconstructor product uses, about one second of clock).  The wait
 * must expire, record its error flag and let the kernel exit; the call then returns
 * MCAO_E_TIMEOUT exactly as after a product wait that gave up, the flag is cleared and the
 * simulation stays usable.  Any other status means the timeout path is broken. */
mcao_status mcao_check_bounded_wait(mcao_sim* sim);

/* Queue, after the work queued so far, a copy of the current realization's commands
 * (commands: host [n_commands] float32, or NULL) and of every science direction's
 * (long-exposure, instantaneous) Strehl ratio (strehl: host [n_sci][2] double, or NULL), and
 * return at once: a closed loop can read each step's result without waiting for it.  The values
 * are in place after mcao_sync, or once the stream set by mcao_set_stream passes this point.
 * Host buffers should be pinned (cudaHostAlloc / page-locked) for the copies to overlap the
 * next steps; the caller keeps them alive until then.  The values are first snapshotted on the
 * device (one small kernel after the queued steps, into one of 64 ring slots) and copied to the
 * host from there on a stream of their own, so the next steps do not wait for the copies; a
 * slot is reused once its earlier copy is done.  Errors: MCAO_E_INVALID_ARG (both NULL),
 * MCAO_E_STATE (commands before the DMs are loaded), MCAO_E_CUDA. */
mcao_status mcao_read_async(mcao_sim* sim, float* commands, double* strehl);

/* Advance several simulations of any configurations (sizes, sensors, layers, reconstructor
 * formats) by n_steps together: each step is one launch of a graph that holds every
 * simulation's step graph as an independent child, so that small configurations run side by
 * side on the GPU ("The closed loop" of each, unchanged; results are identical to stepping each
 * simulation alone).  Ordered after each simulation's earlier work and before its later work
 * (and after / before the streams set by mcao_set_stream).  Errors: MCAO_E_INVALID_ARG (null or
 * repeated handles, n_steps < 0, several devices), MCAO_E_STATE (a simulation not fully
 * loaded), MCAO_E_UNSUPPORTED (the stage profiler is on), MCAO_E_CUDA. */
mcao_status mcao_step_group(mcao_sim* const* sims, int n_sims, int n_steps);

/* Noise-free (with_noise = 0) or configured-noise (1) slopes of every realization at the current
 * step and commands, without reconstruction and without advancing time ("The calibration of
 * the interaction matrices": measurements at a fixed state); read them with mcao_get_slopes.
 * Errors: MCAO_E_STATE (atmosphere or DMs not loaded), MCAO_E_CUDA. */
mcao_status mcao_measure(mcao_sim* sim, int with_noise);

/* Interaction matrix as the exact Jacobian D = d s / d c of the noise-free slopes with respect to
 * the DM commands at the current step, commands and realization ("The calibration of the
 * interaction matrices"), by the adjoint of the sensing (centre of gravity, binning, elongation,
 * |FFT|^2, field) and of the DM projection (clamped bilinear sampling of S = Gy C Gx^T).
 *   D   device pointer, row-major [n_slopes][ld] float32, ld >= n_commands; overwritten (zero
 *       where no actuator reaches a subaperture: influence weights below 1e-10 are left out).
 * Synchronous: waits for the device before and after.  Errors: MCAO_E_INVALID_ARG, MCAO_E_SHAPE,
 * MCAO_E_STATE, MCAO_E_UNSUPPORTED (a subaperture footprint meets more than 128 actuators per
 * axis), MCAO_E_OOM, MCAO_E_CUDA. */
mcao_status mcao_interaction_matrix(mcao_sim* sim, float* D, size_t ld);

/* Gauss-Newton normal equations of a DM misregistration fit ("Conclusions": the rotation of the DM
 * and its modal basis with respect to the sensors; also translation and magnification).  With DM
 * `dm` at its current misregistration p = (shift_x m, shift_y m, rotation rad, magnification)
 * (mcao_set_misregistration), D(p) the exact interaction matrix restricted to that DM's columns
 * and D_meas a measured one, for J(p) = ||D(p) - D_meas||_F^2:
 *   cost = J(p);  Jte[i] = sum dD/dp_i (D - D_meas);  JtJ[4][4] = sum dD/dp_i dD/dp_j (row-major,
 *   symmetric);  meas_sq = ||D_meas||_F^2 over the same entries,
 * so that (JtJ) dp = -Jte is the Gauss-Newton step and 2 Jte the gradient of J.  The derivatives are
 * analytic: every influence function is evaluated at the four bilinear corners of each pupil
 * sample in the DM's own frame and differentiated with respect to p; no model matrix is formed.
 *   D_meas  device pointer, row-major [n_slopes][ld] float32, column j = the DM's command j (its
 *           block of the command vector, in order; pass a full matrix's pointer offset to the
 *           DM's first command), ld >= the DM's command count.
 * Any output pointer may be NULL.  Sums in double in a fixed order.  Synchronous.  Errors:
 * MCAO_E_INVALID_ARG, MCAO_E_SHAPE, MCAO_E_STATE (atmosphere or DMs not loaded), MCAO_E_OOM,
 * MCAO_E_CUDA. */
mcao_status mcao_misreg_normal_equations(mcao_sim* sim, int dm, const float* D_meas, size_t ld, double* JtJ,
                                         double* Jte, double* cost, double* meas_sq);

/* Vector-Jacobian products of the noise-free slopes at the current state: for each of n_vec
 * vectors g (device, row-major [n_vec][n_slopes]):
 *   g_commands  device [n_vec][n_commands] = D^T g (or NULL);
 *   g_phase     device [n_vec][sum over sensors of N_w^2] = (d s / d phi)^T g on each sensor's
 *               pupil grid (rad at the reference wavelength), sensors concatenated in order, zero
 *               outside valid subapertures (or NULL);
 *   g_layers    device [n_vec][sum over layers of n_l^2] = (d s / d screen)^T g on every turbulent
 *               layer's screen (the adjoint of the cone-beam projection at this step's frozen-flow
 *               position), layers concatenated in order (or NULL).
 * Outputs are overwritten.  Command and layer gradients are accumulated with atomic adds
 * (summation order not fixed).  Synchronous.  Errors: MCAO_E_INVALID_ARG (null g, n_vec < 1,
 * every output NULL), MCAO_E_STATE, MCAO_E_UNSUPPORTED, MCAO_E_OOM, MCAO_E_CUDA. */
mcao_status mcao_slopes_vjp(mcao_sim* sim, const float* g_slopes, int n_vec, float* g_commands, float* g_phase,
                            float* g_layers);

/* Reconstructor product of a batch of slope vectors with the loaded control matrix ("The closed
 * loop": slopes times the control matrix), by the kernels of the batched step: out[r] = R s_r for
 * r < n_rhs, with no integrator and no change to the simulation's commands.  A bfloat16 matrix is
 * multiplied on the tensor cores with float32 slopes (each split exactly into three bfloat16
 * terms) and float32 accumulation; a float32 matrix on the CUDA cores.
 *   slopes device pointer, row-major [n_rhs][n_slopes] float32 (the layout of mcao_get_slopes).
 *   out    device pointer, row-major [n_rhs][n_commands] float32, overwritten.
 * Needs a simulation created with n_real > 1 (else MCAO_E_UNSUPPORTED) and 1 <= n_rhs <= n_real.
 * Synchronous: waits for the device before and after; reuses the step's padded-slope scratch,
 * which the next step rewrites.  Errors: MCAO_E_INVALID_ARG, MCAO_E_STATE (no reconstructor),
 * MCAO_E_SHAPE, MCAO_E_UNSUPPORTED, MCAO_E_TIMEOUT, MCAO_E_CUDA. */
mcao_status mcao_reconstruct_batch(mcao_sim* sim, const float* slopes, int n_rhs, float* out);

/* Control matrix by Tikhonov-regularised least squares, computed in FP64 on the GPU ("Control
 * Matrix": the reconstructor is a pseudo-inverse of the interaction matrix; MCAO least squares is
 * ill-posed, hence the regularisation coefficient):
 *   R = -(D^T D + lambda I)^(-1) D^T,   lambda = alpha tr(D^T D) / n_cmd.
 * The minus sign follows the library's conventions: D = d s / d c is measured with the DM
 * subtracted from the wavefront (mcao_interaction_matrix) and the loop applies c <- c + g R s, so
 * R = -D^+ in the limit alpha -> 0 for a full-rank D.  No mcao_sim handle is needed.
 *   D       device pointer, row-major [n_slopes][ld_d] float32, ld_d >= n_cmd (read only).
 *   R       device pointer, row-major [n_cmd][ld_r], ld_r >= n_slopes: float32 (r_fp64 = 0, the
 *           format mcao_load_reconstructor takes) or float64 (r_fp64 = 1); overwritten.
 *   stream  CUDA stream (cudaStream_t) or NULL for the legacy stream.
 *   lambda  optional host pointer: receives lambda.
 * Every step runs in double precision in the library's kernels on 64 x 64 tiles: the Gram matrix
 * (tiles of D that hold only zeros are skipped: a subaperture sees only nearby actuators), its
 * regularisation, a blocked Cholesky factorisation L L^T, L^(-1), M^(-1) = L^-T L^-1 and
 * -M^(-1) D^T (zero tiles skipped again); float32 output is rounded once, at the store.
 * Temporaries of 2 (64 ceil(n_cmd / 64))^2 doubles are allocated and freed by the call (1.04 GB
 * for n_cmd = 8051).  Synchronous.  Errors: MCAO_E_INVALID_ARG (null pointers, alpha < 0 or not
 * finite, r_fp64 not 0 or 1), MCAO_E_SHAPE, MCAO_E_OOM, MCAO_E_UNSUPPORTED (a Cholesky pivot <= 0:
 * the regularised matrix is not positive definite in double precision; raise alpha), MCAO_E_CUDA.
 * err receives a message on failure (err_len bytes, may be NULL). */
mcao_status mcao_tikhonov_reconstructor(const float* D, int n_slopes, int n_cmd, size_t ld_d, double alpha, void* R,
                                        size_t ld_r, int r_fp64, void* stream, double* lambda, char* err,
                                        size_t err_len);

/* Launch shapes ("tuning") of a simulation, in this order (values per MCAO_TUNE_*):
 *   MCAO_TUNE_SENSE_BLOCKS_PER_SM  warp-per-subaperture sensing launches: blocks per SM, [1, 8] (4)
 *   MCAO_TUNE_RECON_CTAS_PCT       reconstructor slices: blocks per SM x 100, [25, 400] (85); the
 *                                  step's last slice, which runs after the last sensor, takes at
 *                                  least one block per SM
 *   MCAO_TUNE_SCIENCE_AFTER_AUX    science waits for the block-per-subaperture sensors, 0 or 1 (1)
 *   MCAO_TUNE_TC_CHUNK             tensor-core batched product: k-blocks per TMEM accumulator,
 *                                  [1, 64] (8)
 *   MCAO_TUNE_MULTI_BLOCKS_PER_SM  batched float32 product: blocks per SM, [1, 2] (2)
 *   MCAO_TUNE_STEPS_PER_GRAPH      steps captured in one CUDA graph, [1, 16] (1): mcao_step(n)
 *                                  launches it n / k times, then the one-step graph n % k times
 *                                  (always the one-step graph while the stage profiler is on)
 * No counterpart in the paper.  Results do not depend on them, except MCAO_TUNE_TC_CHUNK, which
 * regroups the tensor-core product's float32 sums (float32 rounding only). */
enum {
    MCAO_TUNE_SENSE_BLOCKS_PER_SM = 0,
    MCAO_TUNE_RECON_CTAS_PCT = 1,
    MCAO_TUNE_SCIENCE_AFTER_AUX = 2,
    MCAO_TUNE_TC_CHUNK = 3,
    MCAO_TUNE_MULTI_BLOCKS_PER_SM = 4,
    MCAO_TUNE_STEPS_PER_GRAPH = 5,
    MCAO_N_TUNE = 6
};

/* Current launch shapes into values[MCAO_N_TUNE] (n >= MCAO_N_TUNE, else MCAO_E_INVALID_ARG). */
mcao_status mcao_get_tuning(const mcao_sim* sim, int* values, int n);

/* Set the launch shapes (n == MCAO_N_TUNE, each within its range, else MCAO_E_SHAPE /
 * MCAO_E_INVALID_ARG); applies from the next step. */
mcao_status mcao_set_tuning(mcao_sim* sim, const int* values, int n);

/* Autotuner: for each launch shape that applies to this configuration (the sensing grid when it
 * has warp-per-subaperture sensors, the slices' grid without batching, the science ordering when
 * it has block-per-subaperture sensors, the batched products' shapes with batching, the steps per
 * graph among 1, 2, 4 and 8), in that order,
 * time steps_per_trial steps (after 2 warm-up steps) for every candidate value with the others
 * held at their best so far, and keep the fastest (coordinate descent, CUDA events on the device).
 * The trials advance the simulation; its state is saved first and restored at the end (as
 * mcao_get_state / mcao_set_state), so the caller's run continues as if no trial had run.  The
 * chosen shapes stay set; values (n >= MCAO_N_TUNE, may be NULL) receives them and report (may be
 * NULL) the measured ms/step of every trial ("knob: value=ms ... -> chosen").  Errors:
 * MCAO_E_INVALID_ARG (steps_per_trial outside [1, 100000]), MCAO_E_SHAPE, MCAO_E_STATE (not fully
 * loaded), MCAO_E_UNSUPPORTED (stage profiler on), MCAO_E_CUDA. */
mcao_status mcao_autotune(mcao_sim* sim, int steps_per_trial, int* values, int n, char* report, size_t report_len);

/* Stages timed by the profiler. */
enum {
    MCAO_STAGE_DM = 0,          /* DM surfaces                                                  */
    MCAO_STAGE_WFS_MAIN = 1,    /* wavefront-sensor kernel of the largest group (laser stars)   */
    MCAO_STAGE_WFS_AUX = 2,     /* other wavefront-sensor kernels (concurrent stream)           */
    MCAO_STAGE_RECON = 3,       /* reconstructor product R s                                    */
    MCAO_STAGE_RECON_REDUCE = 4,/* partial-sum reduction and integrator                         */
    MCAO_STAGE_SCIENCE = 5,     /* science field, Strehl and PSF (concurrent stream)            */
    MCAO_N_STAGES = 6
};

/* Profiling on: every later mcao_step records a CUDA event pair around each stage of each
 * step, on the stream that stage runs on.  Off (default): no events are kept.  Each pair is a
 * pair of event-record nodes in the step's graph, between the launches it brackets, so a
 * profiled step is slower than an unprofiled one (by about 8 % on the 39 m workload with every
 * stage timed); the step graph is captured again when the profiled stages change. */
mcao_status mcao_set_profiling(mcao_sim* sim, int on);

/* As mcao_set_profiling, timing only the stages of mask (bit 1 << MCAO_STAGE_*; 0 = off), e.g.
 * the reconstructor product alone while the step is timed as a whole.  Errors:
 * MCAO_E_INVALID_ARG (bits at or above MCAO_N_STAGES). */
mcao_status mcao_set_profiling_stages(mcao_sim* sim, unsigned int mask);

/* Synchronise and return, per stage, the summed device milliseconds and the number of timed
 * steps since profiling was switched on or last read; launches_per_step receives the number
 * of kernel launches of one step.  Any pointer may be NULL.  Resets the records. */
mcao_status mcao_get_profile(mcao_sim* sim, double* ms, int64_t* counts, int n_stages,
                             int64_t* launches_per_step);

/* Synchronise and return the launch timeline of the profiled steps (call before
 * mcao_get_profile, which clears the records): for each profiled launch, in issue order, its
 * stage, its start and end in device milliseconds relative to the start of the first launch
 * of the same step, and the index of that step among the profiled ones.  Fills at most n
 * entries of each non-NULL array; *n_total (if not NULL) receives the number of records. */
mcao_status mcao_get_timeline(mcao_sim* sim, int32_t* stage, double* start_ms, double* end_ms,
                              int32_t* step, size_t n, size_t* n_total);

#ifdef __cplusplus
}
#endif
#endif /* MCAO_H */
