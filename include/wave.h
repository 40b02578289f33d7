/*
 * wave.h -- C ABI of libwave: batched 2D/3D isotropic acoustic modelling, its
 * adjoint and the FWI/RTM gradient on one NVIDIA GB300 (sm_103a).
 *
 * The operations follow arxiv 2304.05592 (Louboutin, Yin et al., "Learned
 * multiphysics inversion with differentiable programming and machine
 * learning"), section "Wave-equation-based inversion":
 *   F(m) = P_r A(m)^{-1} P_s^T           (Eq. eq-fwi), m = squared slowness,
 *   Phi(m) = 1/2 || F(m) q - d ||_2^2     (Eq. eq-fwi, the loss of the AD example),
 *   grad Phi = J'(F(m) q - d)             (judiJacobian; the paper's gradient is taken
 *                                          with respect to the squared slowness),
 *   F' dy                                 (pullback of the rrule for F*q).
 * The paper leaves the discretisation open.  This library uses
 *   (M+E) u^{n+1} = (2M + dt^2 L) u^n - (M-E) u^{n-1} + dt^2 S q^n,  u^{-1} = u^0 = 0,
 *   d^n = R u^n  (n = 0 .. nt-1; d^0 is always zero),
 * with M = diag(1/v^2) on a grid padded by nb sponge cells on every side (the
 * model is copied outward from the nearest physical cell), E = diag(eta dt/2),
 * eta = gamma0 (d/nb)^2 / vref^2 with d the depth into the sponge in cells and
 * gamma0 = 3 vref ln(1000) / (2 nb h), L the 8th-order centred Laplacian with
 * zero values beyond the padded grid, S bilinear (2D) or trilinear (3D)
 * injection with weights w / h^ndim, R the same interpolation as sampling.
 *
 * Conventions shared by every entry point
 *  - Arrays are C order with x fastest: 2D velocity [nz][nx], 3D [nz][ny][nx].
 *  - Coordinates are metres from the first physical grid point, ordered (x, z)
 *    in 2D and (x, y, z) in 3D, and must lie inside the physical grid
 *    (0 <= x <= (nx-1) h, ...); otherwise WAVE_ERR_GEOMETRY.
 *  - "dev" pointers are CUDA device memory, "host" pointers are host memory.
 *    The caller owns every buffer.  The library allocates nothing: all scratch
 *    comes from the caller's workspace (size from wave_workspace_size).
 *  - `stream` is a cudaStream_t (NULL = legacy default stream).  wave_forward,
 *    wave_adjoint, wave_gradient, wave_jacobian_adjoint and wave_born are
 *    stream-ordered and asynchronous: they queue their work on the stream and
 *    return without waiting for it (the set-up tables go through a pinned
 *    host staging buffer of the library, so no copy waits either).  Results
 *    are complete once the stream has reached the end of the call.
 *  - Errors found before any launch (arguments, geometry, workspace size)
 *    are returned by the call itself, without touching the outputs.
 *    Errors found on the device -- a velocity that is not finite and
 *    positive or a non-finite result (WAVE_ERR_NONFINITE), a time step above
 *    the stability limit (WAVE_ERR_CFL), a bounded wait that gave up
 *    (WAVE_ERR_TIMEOUT) -- set bits of an error word kept at the start of the
 *    workspace; wave_status_wait(work, stream, ...) waits for the stream and
 *    returns them.  Each call clears that word when it starts on the device,
 *    so wave_status_wait reports the last call queued on the workspace.  When
 *    it reports an error, the outputs of that call hold unspecified values.
 *  - Shot s uses sources src_xyz[s][0..nsrc) and receivers rec_xyz[s][0..nrec);
 *    every shot shares the grid and the velocity model.
 */
#ifndef WAVE_H
#define WAVE_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    WAVE_OK = 0,
    WAVE_ERR_ARG = 1,       /* null pointer, negative count, bad grid, unknown mode */
    WAVE_ERR_CFL = 2,       /* dt * vmax / h above 2 / sqrt(ndim * 2048/315)          */
    WAVE_ERR_GEOMETRY = 3,  /* a source or receiver outside the physical grid         */
    WAVE_ERR_WORKSPACE = 4, /* workspace null or smaller than wave_workspace_size     */
    WAVE_ERR_CUDA = 5,      /* a CUDA runtime call or kernel launch failed            */
    WAVE_ERR_TIMEOUT = 6,   /* a bounded device-side wait ran out (persistent launch) */
    WAVE_ERR_NONFINITE = 7  /* velocity not finite and positive, or NaN in a result   */
} wave_status_t;

typedef struct {
    int ndim;   /* 2 or 3                                                  */
    int nx;     /* physical grid points along x (>= 2)                      */
    int ny;     /* physical grid points along y (3D only, >= 2)             */
    int nz;     /* physical grid points along z (>= 2)                      */
    int nb;     /* sponge cells added outside the physical grid, each side  */
    int nt;     /* time samples (>= 1); time step n is at t = n dt          */
    float h;    /* grid spacing in metres, all axes                         */
    float dt;   /* time step in seconds                                     */
    float vref; /* sponge reference velocity in m/s (frozen, independent of
                   the model); 0 disables damping                           */
} wave_grid_t;

/* How wave_gradient keeps the forward wavefield for the imaging condition. */
typedef enum {
    WAVE_STORE_CHECKPOINT = 0, /* binomial time checkpointing of FP32 states      */
    WAVE_STORE_BF16 = 1,       /* every u^n stored in BF16 (round to nearest even) */
    WAVE_STORE_FP32 = 2        /* every u^n stored in FP32 (exact, most memory)    */
} wave_store_t;

/* Bytes of device workspace that wave_forward (op 0), wave_adjoint (op 1),
 * wave_gradient / wave_jacobian_adjoint (op 2) or wave_born (op 3) needs for
 * this problem.  The coordinates (host, same
 * layout as in the calls) are needed because interpolation taps of zero
 * weight are dropped.  `store` and `nsnap` matter for op 2 only (nsnap =
 * number of checkpoint slots, each holding two FP32 wavefields per shot; the
 * library uses at most nt/2 of them: one per pair of time steps).  The workspace must be
 * 256-byte aligned.  Host function, no device work. */
wave_status_t wave_workspace_size(const wave_grid_t* grid, int op, int nshot, int nsrc, const float* src_xyz,
                                  int nrec, const float* rec_xyz, int store, int nsnap,
                                  size_t* bytes /* host out */);

/* Waits for `stream` and returns the device-side status of the last call
 * queued on the workspace `work` (dev, as passed to that call): WAVE_OK,
 * WAVE_ERR_CFL, WAVE_ERR_NONFINITE or WAVE_ERR_TIMEOUT from the error word,
 * WAVE_ERR_CUDA if the stream reports a CUDA error (a failed kernel).
 * misfit (host out, may be NULL) receives that call's misfit (wave_gradient;
 * 0 for the other calls).  WAVE_ERR_ARG for a NULL workspace.  Not part of the
 * paper: the status channel of the asynchronous calls. */
wave_status_t wave_status_wait(const void* work, void* stream, double* misfit);

/* Forward modelling d = F(m) q (Eq. eq-fwi, P_r A(m)^{-1} P_s^T).
 *   vel      dev  [nz][(ny)][nx] velocity (m/s)
 *   src_xyz  host [nshot][nsrc][ndim] source coordinates
 *   wavelet  dev  [nshot][nt][nsrc] source time functions q
 *   rec_xyz  host [nshot][nrec][ndim] receiver coordinates
 *   data     dev  out [nshot][nt][nrec] shot records (row n = 0 is zero) */
wave_status_t wave_forward(const wave_grid_t* grid, const float* vel, int nshot, int nsrc,
                           const float* src_xyz, const float* wavelet, int nrec, const float* rec_xyz,
                           float* data, void* work, size_t work_bytes, void* stream);

/* Adjoint in the source, F(m)' r (the pullback of the rrule for F*q):
 *   (F' r)^n = dt^2 S' mu^{n+1} for n = 0..nt-2 and 0 at n = nt-1, where
 *   (M+E) mu^k = (2M + dt^2 L) mu^{k+1} - (M-E) mu^{k+2} + R' r^k, k = nt-1..1.
 *   resid    dev  [nshot][nt][nrec] data-space input r
 *   src_out  dev  out [nshot][nt][nsrc] */
wave_status_t wave_adjoint(const wave_grid_t* grid, const float* vel, int nshot, int nsrc,
                           const float* src_xyz, int nrec, const float* rec_xyz, const float* resid,
                           float* src_out, void* work, size_t work_bytes, void* stream);

/* Parameter the gradients are taken with respect to. */
typedef enum {
    WAVE_WRT_SLOWNESS2 = 0, /* dPhi/dm, m = 1/v^2 (the paper's parameter) */
    WAVE_WRT_VELOCITY = 1   /* dPhi/dv = -2 / v^3 dPhi/dm                  */
} wave_wrt_t;

/* FWI gradient (judiJacobian(F, q)' * (F q - d), i.e. J' applied to the data
 * residual) of Phi(m) = 1/2 sum_s ||F_s(m) q_s - d_s||^2 with respect to the
 * physical squared slowness m = 1/v^2, summed over shots:
 *   grad_pad = - sum_n mu^{n+1} .* (u^{n+1} - 2 u^n + u^{n-1})  (zero-lag
 *   cross-correlation of the adjoint field with the second time difference of
 *   the forward field), then summed back onto the physical cells the padded
 *   model was copied from.
 *   d_obs    dev  [nshot][nt][nrec] observed data
 *   grad     dev  out [nz][(ny)][nx] dPhi/dm
 *   d_syn    dev  out [nshot][nt][nrec] synthetic data, or NULL
 *   misfit   host out Phi (double), or NULL: written by a stream-ordered copy,
 *            valid once the stream has reached the end of the call (pinned
 *            memory keeps the call asynchronous; a pageable address makes the
 *            call wait for its own work).  wave_status_wait also returns it.
 *   store    a wave_store_t; nsnap = checkpoint slots (CHECKPOINT only, >= 1)
 *   wrt      a wave_wrt_t: gradient w.r.t. m (default) or w.r.t. v */
wave_status_t wave_gradient(const wave_grid_t* grid, const float* vel, int nshot, int nsrc,
                            const float* src_xyz, const float* wavelet, int nrec, const float* rec_xyz,
                            const float* d_obs, float* grad, float* d_syn, double* misfit, int store,
                            int nsnap, int wrt, void* work, size_t work_bytes, void* stream);

/* Adjoint of the Jacobian applied to an arbitrary data-space vector r,
 * summed over shots: J(m)' r with J the Jacobian of d = F(m) q (the first
 * output of the pullback of the rrule for F*q, judiJacobian(F, q)' * dy).
 * Same arguments as wave_gradient, with the residual r (dev [nshot][nt][nrec])
 * in place of d_obs and no synthetic data or misfit.  Workspace: op 2. */
wave_status_t wave_jacobian_adjoint(const wave_grid_t* grid, const float* vel, int nshot, int nsrc,
                                    const float* src_xyz, const float* wavelet, int nrec, const float* rec_xyz,
                                    const float* resid, float* grad, int store, int nsnap, int wrt, void* work,
                                    size_t work_bytes, void* stream);

/* Born modelling, the Jacobian applied to a model perturbation:
 * d = J(m) dm (judiJacobian(F, q) * dm), linearised about m = 1/vel^2:
 *   (M+E) du^{n+1} = (2M + dt^2 L) du^n - (M-E) du^{n-1}
 *                    - Extend(dm) .* (u^{n+1} - 2 u^n + u^{n-1}),  d^n = R du^n,
 * u the background field of wave_forward.
 *   dm    dev [nz][(ny)][nx] perturbation of the squared slowness
 *   data  dev out [nshot][nt][nrec]
 * Workspace: op 3 of wave_workspace_size. */
wave_status_t wave_born(const wave_grid_t* grid, const float* vel, int nshot, int nsrc, const float* src_xyz,
                        const float* wavelet, int nrec, const float* rec_xyz, const float* dm, float* data,
                        void* work, size_t work_bytes, void* stream);

/* Forward modelling without a caller workspace, for callers that cannot
 * allocate device memory when they model: e.g. a plugin whose host
 * application has reserved all device memory up front, or a latency-critical
 * loop that must not pay for an allocation and the synchronisation it can
 * bring.  The paper has no counterpart; this is a deployment convenience.
 * Same arguments and results as wave_forward, minus work/work_bytes; unlike
 * wave_forward it waits for its work and returns the device-side errors
 * itself (the caller has no workspace to hand to wave_status_wait).
 * Scratch is a file-scope device array of WAVE_STATIC_WORKSPACE_BYTES inside
 * the library, held by every GPU that loads the library until the process
 * exits.  Problems whose workspace (wave_workspace_size, op 0) exceeds it
 * return WAVE_ERR_WORKSPACE before any device work.  The call allocates
 * nothing on the device.  Every call looks up the array's device address on
 * the current device (cudaGetSymbolAddress), so a device reset between calls
 * does no harm; the first call on a device may load the library's device code
 * there, so make that first call before any stream capture.  Every call on a
 * device shares the one array and
 * the array keeps the last call's contents (each call clears what must start
 * at zero): calls that overlap on the GPU, from two streams or two host
 * threads, race and must be serialised by the caller. */
#define WAVE_STATIC_WORKSPACE_BYTES (32u << 20)
wave_status_t wave_forward_static(const wave_grid_t* grid, const float* vel, int nshot, int nsrc,
                                  const float* src_xyz, const float* wavelet, int nrec, const float* rec_xyz,
                                  float* data, void* stream);

/* One problem of an uneven batch: its own 2D grid, model, time axis, one
 * shot's sources and receivers, observed data, and outputs. */
typedef struct {
    wave_grid_t grid;      /* 2D grid of this problem                      */
    const float* vel;      /* dev [nz][nx] velocity                         */
    int nsrc;
    const float* src_xyz;  /* host [nsrc][2]                                */
    const float* wavelet;  /* dev [nt][nsrc]                                */
    int nrec;
    const float* rec_xyz;  /* host [nrec][2]                                */
    const float* d_obs;    /* dev [nt][nrec]                                */
    float* grad;           /* dev out [nz][nx] gradient of this problem     */
    double misfit;         /* out: 1/2 ||F q - d_obs||^2 of this problem    */
} wave_problem_t;

/* Low-cut wavelet for the paper's FWI experiment (a Ricker wavelet stripped of
 * its content under 4 Hz, section "Deep priors and normalizing flows"): the real
 * DFT of q (nt samples, spacing dt) is multiplied by H(f) = 0 below f_cut, the
 * raised-cosine ramp 0.5 (1 - cos(pi (f - f_cut) / (f_pass - f_cut))) up to
 * f_pass and 1 above (f_k = k / (nt dt), k = 0..nt/2), and transformed back.
 * The DFT and its inverse are direct sums in double.  q and out are device
 * arrays of nt floats (out may not alias q); work holds
 * wave_lowcut_work_bytes(nt) device bytes.  Stream-ordered, no
 * synchronisation; WAVE_ERR_ARG for null pointers, nt < 1, dt <= 0 or
 * f_pass <= f_cut. */
size_t wave_lowcut_work_bytes(int nt);
wave_status_t wave_lowcut(const float* q, int nt, float dt, float f_cut, float f_pass, float* out, void* work,
                          void* stream);

/* Additive coloured Gaussian noise with the bandwidth of the data (the same
 * experiment): noise[s][t][r] = sum_k filt[k] white[s][t - k + center][r]
 * (zero outside the trace), scaled so that 20 log10(||data|| / ||noise||) =
 * snr_db, and out = data + noise.  data, white and out are device arrays
 * [nshot][nt][nrec] (white holds the caller's standard normal draws; out may
 * alias data); filt is a device array of nf taps, normally the source
 * wavelet, so that the noise has the data's band.  work holds
 * wave_add_noise_work_bytes(nshot, nt, nrec) device bytes.  Stream-ordered. */
size_t wave_add_noise_work_bytes(int nshot, int nt, int nrec);
wave_status_t wave_add_noise(const float* data, const float* white, int nshot, int nt, int nrec, const float* filt,
                             int nf, int center, double snr_db, float* out, void* work, void* stream);

/* Model updates of an FWI iteration: y += alpha x, and y = min(max(y, lo), hi)
 * (n device floats each).  Stream-ordered. */
wave_status_t wave_axpy(long long n, float alpha, const float* x, float* y, void* stream);
wave_status_t wave_clamp(long long n, float lo, float hi, float* y, void* stream);

/* Vector steps of the least-squares RTM iteration (conjugate gradients on
 * the normal equations J'J dm = J' dd of judiJacobian, section
 * "Wave-equation-based inversion"): y = alpha x + beta y, and the dot product
 * sum_i x_i y_i accumulated in double in a fixed order (the same bits on every
 * run) into out[0]; out is a device array of 1 + WAVE_DOT_PARTIALS doubles
 * (the rest is scratch).  n device floats; stream-ordered, no
 * synchronisation; WAVE_ERR_ARG for n < 0 or a null pointer (x and y may be
 * null when n = 0, which gives out[0] = 0). */
#define WAVE_DOT_PARTIALS 256
wave_status_t wave_axpby(long long n, float alpha, const float* x, float beta, float* y, void* stream);
/* y = x .* y elementwise (n device floats), e.g. a diagonal preconditioner
 * applied to a gradient; stream-ordered. */
wave_status_t wave_mul(long long n, const float* x, float* y, void* stream);
wave_status_t wave_dot(long long n, const float* x, const float* y, double* out, void* stream);

/* The bounded wait that the persistent batch sweep uses between tiles, run by
 * one thread on a caller-given device flag: it polls *flag >= want through L2
 * and gives up after a fixed number of polls (a few seconds) or as soon as
 * *abort_word is non-zero.  flag, abort_word and err are device ints owned by
 * the caller (err is overwritten).  Synchronises the stream; returns WAVE_OK
 * if the flag was released, WAVE_ERR_TIMEOUT if the wait gave up (the context
 * stays usable), WAVE_ERR_ARG for a null pointer, WAVE_ERR_CUDA on a launch
 * error.  For tests of the failure path (a flag that nothing sets); the paper
 * has no counterpart. */
wave_status_t wave_wait_probe(int* flag, int want, int* abort_word, int* err, void* stream);

/* Workspace for wave_gradient_batch (store: WAVE_STORE_BF16 or _FP32). */
wave_status_t wave_workspace_size_batch(const wave_problem_t* probs, int nprob, int store, size_t* bytes);

/* FWI gradients of nprob independent 2D problems of different sizes, time
 * axes and models (each problem is the gradient of wave_gradient for its own
 * single shot), computed together: one persistent forward sweep that stores
 * every level (store = WAVE_STORE_BF16 or WAVE_STORE_FP32) and one persistent
 * adjoint sweep, in which each 128 x TZ tile advances as soon as its
 * neighbours have finished the previous step (bounded waits; a wait that
 * runs out returns WAVE_ERR_TIMEOUT).  The time loop has no per-step launch
 * and no global barrier, so short problems leave the sweep early.  The sweep
 * kernel (tile height TZ, warps, pipeline depth, CTAs per SM) is the one
 * wave_autotune_batch picked for batches of the same shapes, else a default.
 * With use_graph != 0 the device work after the set-up is captured once into
 * a CUDA graph and replayed by later calls with the same problems, buffers
 * and kernel choice.  Each problem's misfit field is written on return (the
 * call synchronises the stream).  The batch is the paper's per-shot
 * parallelism of the gradient (section "Putting it all together": gradients
 * of randomly drawn shots per iteration). */
wave_status_t wave_gradient_batch(wave_problem_t* probs, int nprob, int store, int wrt, int use_graph, void* work,
                                  size_t work_bytes, void* stream);

/* Autotuner of the uneven batch (no counterpart in the paper): runs the first
 * `steps` steps of both sweeps of every sweep-kernel variant on this batch
 * (same arguments and workspace as wave_gradient_batch; grads are not
 * written), times them with CUDA events on `stream`, and records the fastest
 * forward/adjoint pair with a common tile height for the batch's shapes
 * (grid sizes, nb, nt, source and receiver counts, store); later
 * wave_gradient_batch calls on batches of those shapes use it.  best_fwd /
 * best_adj (host out, may be NULL) receive the chosen variants, numbered
 * 0 .. wave_batch_variant_count() - 1.  Synchronises the stream. */
wave_status_t wave_autotune_batch(wave_problem_t* probs, int nprob, int store, int steps, void* work,
                                  size_t work_bytes, void* stream, int* best_fwd, int* best_adj);
int wave_batch_variant_count(void);

/* Forces the sweep kernels of later wave_gradient_batch calls (for tests and
 * measurements; no counterpart in the paper): fwd and adj in
 * [0, wave_batch_variant_count()) with the same tile height (variant 0: direct
 * loads, 128 x 32 tiles; 1 and up: TMA producer/consumer sweeps), or both -1
 * to return to the autotuned or default choice.  Process-wide; WAVE_ERR_ARG
 * for an invalid pair. */
wave_status_t wave_set_batch_variant(int fwd, int adj);

/* Ricker wavelet q(t_n) = (1 - 2 a) exp(-a), a = (pi f0 (n dt - 1/f0))^2,
 * n = 0..nt-1 (the wavelet of the paper's FWI example, peak delayed by 1/f0).
 *   out dev out [nt] */
wave_status_t wave_ricker(float f0, float dt, int nt, float* out, void* stream);

/* The binomial checkpoint schedule that wave_gradient runs in
 * WAVE_STORE_CHECKPOINT mode (Griewank and Walther's optimal reversal with a
 * fixed number of snapshots; the paper itself only needs J' and leaves the
 * memory strategy open).  Host function, no device work.
 *   fwd_steps host out: forward time steps executed, first sweep included
 *   actions   host out [capacity][3]: (kind, arg, state) per action with kind
 *             0 advance (arg = start state, state = end state), 1 save
 *             (arg = slot), 2 restore (arg = slot, -1 = zero state), 3 adjoint
 *             steps state and state-1 (arg = state), 4 data complete;
 *             state j stands for (u^j, u^{j-1})
 *   nactions  host out: total number of actions (may exceed capacity) */
wave_status_t wave_checkpoint_schedule(int nt, int nsnap, long long* fwd_steps, int* actions, int capacity,
                                       int* nactions);

/* Measurement support (no counterpart in the paper).
 * wave_launch_count: number of kernels this library has launched so far in
 * the process.  wave_profile_start(every): from now on, bracket every
 * `every`-th stencil time-step launch with two CUDA events on its stream
 * (at most 8192 samples); every = 0 instead brackets each run of consecutive
 * step launches of one kind (forward or adjoint) on one stream, which keeps
 * the overlap between consecutive launches inside a run (at most 16384 runs;
 * a run ends at a change of kind or stream or at another library kernel).
 * wave_profile_stop: stops sampling, waits for the sampled events and returns
 * the summed milliseconds and the number of forward and adjoint step
 * launches they cover (any pointer may be NULL). */
long long wave_launch_count(void);
wave_status_t wave_profile_start(int every);
wave_status_t wave_profile_stop(double* fwd_ms, long long* fwd_n, double* adj_ms, long long* adj_n);

/* Kernel variant selection for the time step (no counterpart in the paper;
 * used by the autotuner and by measurements).  which = 0 selects the 2D
 * forward step, 1 the 2D adjoint step, 2 the 3D step (forward and adjoint);
 * variant in [0, wave_variant_count(which)) or -1 for the library default.
 * 2D variants: direct loads, TMA pipeline, shot groups (cp.async or TMA fed),
 * z-march, persistent items, with different tile shapes; 3D variants: a
 * z-march with a shared-memory halo plane (0) and TMA plane rings with
 * different tile heights and z chunks.  All variants of a step compute the
 * same shot records bit for bit (one arithmetic order); gradients agree to
 * rounding of the per-group sums.  The choice is process-wide and applies to
 * calls that start after it (not thread-safe against calls in flight). */
wave_status_t wave_set_variant(int which, int variant);
int wave_variant_count(int which);

/* Autotuner for the 2D step kernels (no counterpart in the paper): times
 * `steps` forward steps (sources, receivers gathered) and `steps` adjoint
 * steps (imaging on) of every variant on this exact problem, with CUDA events
 * on `stream`, and records the fastest pair for (padded grid, nshot); later
 * calls on the same grid and shot count use it unless wave_set_variant forces
 * a variant.  Arguments as in wave_gradient (the workspace must be sized for
 * op 2, WAVE_STORE_CHECKPOINT, nsnap = 1 or more); the field buffers of the
 * workspace are overwritten.  best_fwd / best_adj (host out, may be NULL)
 * receive the chosen variants (-1 for 3D grids, which have one kernel). */
wave_status_t wave_autotune(const wave_grid_t* grid, const float* vel, int nshot, int nsrc, const float* src_xyz,
                            const float* wavelet, int nrec, const float* rec_xyz, int steps, void* work,
                            size_t work_bytes, void* stream, int* best_fwd, int* best_adj);

/* Name of the last failing CUDA runtime call in this thread (for
 * WAVE_ERR_CUDA diagnostics; "cudaSuccess" if none). */
const char* wave_cuda_error_name(void);

/* Largest stable dt * vmax / h for ndim = 2 or 3 (0 for other ndim). */
double wave_courant_limit(int ndim);

/* Static text for a status code. */
const char* wave_status_str(wave_status_t status);

#ifdef __cplusplus
}
#endif

#endif /* WAVE_H */
