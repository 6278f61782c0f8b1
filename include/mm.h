/*
 * mm.h -- C ABI of the GB300 (sm_103a) demag + LLG hot path.
 *
 * The library implements the per-step loop of a finite-difference
 * micromagnetic solver (Zhu, "Speedup of Micromagnetic Simulations with C++
 * AMP on Graphics Processing Units"):
 *   - the demagnetising field as the zero-padded FFT convolution of M with
 *     the demag tensor (Sec. 2, Eqs. (7)-(13); Sec. 3, Eqs. (14)-(16)),
 *   - the effective field H_eff = H_exch + H_anis + H_demag + H_ext
 *     (Eqs. (2)-(5)), the LLG right-hand side (Eq. (6)) and a forward-Euler
 *     step (Table 1 caption) followed by renormalisation to |M| = Ms,
 *   - the energy of Eq. (1).
 *
 * Conventions shared by every call
 *   Grid      nx x ny x nz cells, zero-indexed i, j, k (Sec. 2).
 *   Layout    M and H are three SoA planes of float32 (x, y, z components),
 *             each nx*ny*nz long, x fastest: element (c, i, j, k) sits at
 *             c*N + i + nx*(j + ny*k), N = nx*ny*nz.
 *   Units     SI: M, H in A/m; cell sizes in m; A in J/m; Ku in J/m^3;
 *             gamma = gamma_0 in m/(A s) (mu0 absorbed, e.g. 2.211e5);
 *             dt in s; energies in J.  mu0 = 4 pi 1e-7.
 *   Pointers  The caller owns every pointer it passes.  Arguments named
 *             *_dev must be device memory of the context's GPU.  Arguments
 *             documented as "host or device" may be either (the copy uses
 *             unified addressing).  The library owns its own device buffers
 *             (tensor spectrum, FFT workspace, M ping-pong) and frees them in
 *             mm_destroy.
 *   Streams   All GPU work of a context is issued on the stream given to
 *             mm_create (NULL = the CUDA legacy default stream) and is
 *             asynchronous unless a call says it synchronises.
 *   Errors    Every call returns MM_OK (0) or a negative MM_E* code; no C++
 *             exception crosses the ABI.  mm_last_error() gives a message for
 *             the last failing call on the calling thread.  A failing call
 *             leaves the context's state unchanged, except MM_ENONFINITE,
 *             which leaves the offending state in place for inspection.
 *   Threads   A context may be used from one thread at a time.
 */
#ifndef MM_H
#define MM_H

#ifdef __cplusplus
extern "C" {
#endif

enum {
    MM_OK = 0,
    MM_EINVAL = -1,       /* bad grid, cell, material value or null pointer */
    MM_ENOMEM = -2,       /* device allocation failed                         */
    MM_ECUDA = -3,        /* a CUDA runtime call or kernel launch failed      */
    MM_ENONFINITE = -4,   /* a step produced a non-finite magnetisation       */
    MM_ETIMEOUT = -5,     /* a bounded device-side wait gave up               */
    MM_EUNSUPPORTED = -6, /* a size outside the supported plan limits         */
    MM_ELIMIT = -7        /* an adaptive run used up its step budget          */
};

typedef struct mm_ctx mm_ctx;

/* Integrators for mm_step (mm_set_integrator). */
enum {
    MM_INTEGRATOR_EULER = 0,   /* forward Euler, the paper's scheme (default)   */
    MM_INTEGRATOR_HEUN = 1,    /* explicit trapezoid, second order              */
    MM_INTEGRATOR_RK4 = 2      /* classic Runge-Kutta, fourth order             */
};

/* How mm_step runs Euler steps (mm_set_step_path). */
enum {
    MM_STEP_AUTO = 0,          /* the faster of the two on this device: graphs       */
    MM_STEP_GRAPH = 1,         /* one launch per kernel per step, replayed from graphs */
    MM_STEP_PERSISTENT = 2     /* one cooperative launch for many steps            */
};

/* How the x-step kernel of the graph step moves its spectrum tiles
 * (mm_set_tiled_copies): bits that make the gather from the plane kernel's
 * output, and the scatter of the next spectrum, tiled tensor copies. */
enum {
    MM_TILED_GATHER = 1,
    MM_TILED_SCATTER = 2
};

/*
 * mm_create -- build a solver context; the tensor set-up happens here, once
 * (Sec. 3: the tensor FFT "carried out at the beginning of simulation").
 *
 *   out     receives the new context (set to NULL on failure).
 *   grid    {nx, ny, nz}, each >= 1.
 *   cell    {dx, dy, dz} in m, each > 0.
 *   Ms      saturation magnetisation, A/m, > 0 (Sec. 2).
 *   A       exchange constant, J/m, >= 0 (Eq. (1), (3)).
 *   Ku      uniaxial anisotropy constant, J/m^3, easy axis x (Eq. (1), (5)).
 *   alpha   damping, >= 0 (Eq. (6)).
 *   gamma   gamma_0 in m/(A s), > 0 (Eq. (6)).
 *   cuda_stream  cudaStream_t to issue work on, or NULL.
 *
 * Set-up computes the cell-averaged (Newell) demag tensor in FP64 on the GPU
 * (closed form near the source, Gauss-Legendre cell average far away), its
 * transform on the zero-padded box (padded length per axis: 2n when n is a
 * power of two, else the smallest 2^a 3^b 5^c >= 2n - 1; 1 when n = 1), and
 * stores the real, octant-symmetric spectrum in FP32.  The initial M is
 * uniform +x and H_ext = 0.  Synchronises the stream.
 * Returns MM_EINVAL, MM_EUNSUPPORTED (padded length > 4096 on an axis or
 * a working set beyond shared-memory plan limits), MM_ENOMEM or MM_ECUDA.
 */
int mm_create(mm_ctx **out, const int grid[3], const double cell[3],
              double Ms, double A, double Ku, double alpha, double gamma,
              void *cuda_stream);

/* mm_destroy -- free every resource of ctx.  NULL-safe.  Synchronises. */
int mm_destroy(mm_ctx *ctx);

/*
 * mm_set_integrator -- choose the time stepper of mm_step.  Forward Euler
 * (Table 1 caption) is the default and runs as the two-kernel step on
 * power-of-two grids.  Heun and classic RK4 go beyond the paper: each stage
 * evaluates H_eff of the stage state with the same three demag/field passes,
 * stage states are not renormalised, the new state is renormalised to
 * |M| = Ms.  They allocate two extra 3*N float32 buffers on first use.
 * Returns MM_EINVAL for an unknown method, MM_ENOMEM on allocation failure.
 */
int mm_set_integrator(mm_ctx *ctx, int method);

/*
 * mm_run_adaptive -- integrate Eq. (6) over t_span seconds from the current
 * M with the embedded Dormand-Prince RK5(4) pair and step-size control
 * (beyond the paper, whose scheme is forward Euler, Table 1 caption).
 * Every stage evaluates H_eff of its (plain, not renormalised) stage state
 * with the three demag/field passes; the fifth-order state is renormalised
 * to |M| = Ms; the seventh stage is the right-hand side at that state and
 * is reused as the first stage of the next step.  The error of a trial step
 * is err = max over cells |dt sum_i e_i k_i| / Ms (e: fifth- minus fourth-
 * order weights).  A step is accepted when err <= tol; the next trial step
 * is h * clamp(0.9 (tol / err)^(1/5), 0.2, 5), without growth right after a
 * rejection; the last step is shortened to end on t_span.
 *
 *   t_span     seconds to cover, finite, >= 0 (0: nothing happens).
 *   dt         in: the first trial step (s, > 0); out: the step the
 *              controller proposes next (host memory).
 *   tol        error bound per step, > 0 (dimensionless, relative to Ms).
 *   max_steps  limit on accepted + rejected trial steps, >= 1.
 *   stats      NULL or 4 doubles (host): accepted steps, rejected steps,
 *              field evaluations, seconds covered.
 *
 * Synchronises once per trial step (the error estimate is read back to the
 * host, which runs the controller).  Allocates 8 extra 3*N float32 buffers on
 * first use.  Returns MM_OK once t_span is covered, MM_ELIMIT when
 * max_steps ran out first (M is the last accepted state), MM_EINVAL, MM_ENOMEM
 * or MM_ECUDA.  A non-finite trial state gives an infinite error and is
 * rejected like any other.
 */
int mm_run_adaptive(mm_ctx *ctx, double t_span, double *dt, double tol, int max_steps, double stats[4]);

/* mm_set_field -- uniform external (Zeeman) field H_ext in A/m (Eq. (1),
 * (2)); applies to later steps.  H_ext: 3 doubles, host memory. */
int mm_set_field(mm_ctx *ctx, const double H_ext[3]);

/* mm_set_m -- copy a magnetisation state into the context (Sec. 3: the
 * initial conditions are the only host-to-device input).  M: 3*N float32,
 * host or device.  Used as given, not renormalised: the caller supplies
 * |M| = Ms (a departure from a set-and-renormalise contract, so that a state
 * read with mm_get_m and set again is bit for bit the same state; every
 * step renormalises its result to Ms). */
int mm_set_m(mm_ctx *ctx, const float *M);

/* mm_get_m -- copy the current magnetisation out.  M: 3*N float32, host or
 * device.  Synchronises when M is host memory. */
int mm_get_m(mm_ctx *ctx, float *M);

/*
 * mm_demag_field -- H_demag of M by the padded FFT convolution:
 * forward x R2C (pruned), forward y/z FFT (pruned), 3x3 real-tensor product
 * (Eq. (13)/(15)), inverse z/y (pruned), inverse x C2R keeping i < nx
 * (Eq. (10)/(16)); on power-of-two films the z part is the exact direct sum
 * over the layers with the (x, y) spectrum of each z offset.  M_dev, H_dev:
 * 3*N float32 device arrays, must not overlap.  Does not touch the
 * context's own M (it does overwrite the context's spectrum workspace, so
 * the next mm_step re-forms it).  Asynchronous.
 */
int mm_demag_field(mm_ctx *ctx, const float *M_dev, float *H_dev);

/*
 * mm_effective_field -- H_eff = H_exch + H_anis + H_demag + H_ext of M
 * (Eqs. (2)-(5)); exchange with free (Neumann) boundaries.  M_dev, H_dev:
 * 3*N float32 device arrays, must not overlap.  Asynchronous.
 */
int mm_effective_field(mm_ctx *ctx, const float *M_dev, float *H_dev);

/*
 * mm_step -- n steps of Eq. (6) of size dt on the resident M with the
 * chosen integrator (default forward Euler:
 * M <- Ms * (M + dt f(M)) / |M + dt f(M)|, every field term at M^n).  An
 * Euler step is three kernels (x R2C; per-kx-plane y/z FFT + tensor product
 * + inverse y/z; inverse x C2R fused with exchange, anisotropy, Zeeman, LLG,
 * Euler and renormalisation); the update kernel also forms the next step's
 * x R2C, so a film step is two kernels (on power-of-two films the exchange
 * stencil rides in the tensor spectrum) and a thick sample's four; steps are
 * replayed from CUDA graphs of 16 steps (the remainder one step each).
 * On the square power-of-two films the persistent step is built for
 * (64, 128, 256 wide with nz = 4; 256 x 256 with nz = 1 or 2) the two
 * kernels' work can instead run as one cooperative launch for up to 1024
 * steps (plane phase, grid barrier, x-step phase per step; same
 * arithmetic, same result bits), see mm_set_step_path.  n >= 0, dt > 0.
 * Asynchronous: a non-finite result is reported by mm_sync / mm_energy, a
 * grid-barrier wait that gave up (MM_ETIMEOUT, state incomplete) by mm_sync.
 */
int mm_step(mm_ctx *ctx, int n, double dt);

/*
 * mm_step_host -- n steps (n >= 0, dt > 0) from a state held in host
 * memory, with the result written back to host memory: the same result as
 * mm_set_m(M_in), mm_step(n, dt), mm_get_m(M_out), bit for bit, with one
 * synchronisation.  M_in, M_out: 3*N float32 in host memory (they may be
 * the same buffer).  On the power-of-two films' Euler step (graph path),
 * the kernels themselves read M_in and write M_out over the host link
 * (no staging copies) when the buffers are page-locked, or pageable on a
 * device with coherent access to pageable host memory; otherwise the data
 * is staged with copies.  The context's state becomes the result.  A
 * non-finite result is reported by the next mm_sync.  Synchronises.
 */
int mm_step_host(mm_ctx *ctx, const float *M_in, int n, double dt, float *M_out);

/*
 * mm_set_step_path -- choose how mm_step runs Euler steps: MM_STEP_AUTO
 * (default; the graph step, measured faster on GB300), MM_STEP_GRAPH or
 * MM_STEP_PERSISTENT.  The persistent step keeps
 * each block's tensor-spectrum slice, twiddles and M rows in shared memory
 * across the steps of a launch and replaces the per-step kernel boundaries
 * by grid barriers (the launch and I/O overhead the paper names in Sec. 4).
 * Returns MM_EINVAL for an unknown path, MM_EUNSUPPORTED when the
 * persistent step is asked for but not available for this grid or device.
 */
int mm_set_step_path(mm_ctx *ctx, int path);

/* mm_get_step_path -- MM_STEP_PERSISTENT or MM_STEP_GRAPH: how the next
 * mm_step will run, or a negative error code. */
int mm_get_step_path(const mm_ctx *ctx);

/*
 * mm_set_tiled_copies -- how the x-step kernel of the two-kernel step
 * (power-of-two films up to nx = 256) moves the transposed spectrum of the
 * per-axis transforms (Sec. 3, Eqs. (14)-(16)): 0 (default) with 16-byte
 * asynchronous copies issued by every thread and plain stores; a mask of
 * MM_TILED_GATHER / MM_TILED_SCATTER makes the gather of the tile's
 * 3 (nx + 1) runs of 32 bytes, or the scatter of the next spectrum, one
 * tiled tensor copy of a 4-D box per block.  Same arithmetic, same result
 * bits; the default measured faster on GB300.  Mask bits outside the two:
 * MM_EINVAL; a nonzero mask for a grid without the tiled form:
 * MM_EUNSUPPORTED.  Takes effect from the next step or field evaluation.
 */
int mm_set_tiled_copies(mm_ctx *ctx, int mask);

/* mm_get_tiled_copies -- the mask in effect, or a negative error code. */
int mm_get_tiled_copies(const mm_ctx *ctx);

/*
 * mm_set_wait_limit -- a diagnostic: the number of polls a grid-barrier
 * wait of the persistent step makes before it gives up (default 2^20, of
 * the order of a second).  0 makes every wait that would block give up at
 * once, which exercises the timeout path: the blocks leave, mm_sync returns
 * MM_ETIMEOUT and the state is incomplete until the next mm_set_m.
 * polls >= 0, else MM_EINVAL.
 */
int mm_set_wait_limit(mm_ctx *ctx, long long polls);

/*
 * mm_energy -- the energy of Eq. (1) for the current M, summed in FP64:
 * E[0] total, E[1] exchange (link sum A V sum |m_i - m_j|^2 / delta^2),
 * E[2] anisotropy, E[3] demag (-1/2 mu0 V sum H_d . M), E[4] Zeeman, in J.
 * E: 5 doubles, host memory.  Synchronises; returns MM_ENONFINITE if any
 * earlier step produced a non-finite value.
 */
int mm_energy(mm_ctx *ctx, double E[5]);

/* mm_sync -- wait for the context's stream; MM_ENONFINITE if any step since
 * mm_create / mm_set_m produced a non-finite magnetisation. */
int mm_sync(mm_ctx *ctx);

/* mm_last_error -- message for the last nonzero status returned on the
 * calling thread ("" if none).  ctx may be NULL.  The string stays valid
 * until the next call on this thread. */
const char *mm_last_error(const mm_ctx *ctx);

/*
 * mm_plan_info -- the padded lengths and the decomposition chosen by
 * mm_create.  L: {Lx, Ly, Lz} (may be NULL).  Returns the number of kernel
 * launches per Euler step (2 on films, 4 on thick samples whose pass 2 is
 * split into y / z / y kernels; 3 or 5 when only the x passes are
 * compile-time) or a negative error code.
 */
int mm_plan_info(const mm_ctx *ctx, int L[3]);

/*
 * mm_tensor_octant -- recompute the FP64 real-space demag tensor N (K = -N)
 * on the non-negative offset octant, as used by set-up: out holds
 * 6*nx*ny*nz doubles, component-major (xx, xy, xz, yy, yz, zz), then
 * offset (i, j, k) at i + nx*(j + ny*k).  Host or device.  Synchronises.
 * Diagnostic; not on the per-step path.
 */
int mm_tensor_octant(mm_ctx *ctx, double *out);

/*
 * mm_kernel_spectrum -- copy the stored FP32 spectrum of K = -N, already
 * divided by Lx*Ly*Lz (the inverse-FFT normalisation is folded in), on the
 * octant 0..L/2 of each axis: out holds (Lx/2+1)*(Lz/2+1)*(Ly/2+1)*6 floats
 * laid out [kx][kz][ky][component].  Host or device.  Synchronises.
 * Diagnostic; not on the per-step path.
 */
int mm_kernel_spectrum(mm_ctx *ctx, float *out);

/*
 * mm_time_passes -- diagnostic timing of the three step kernels.  Runs
 * `reps` Euler steps of size dt on the resident M (advancing it exactly as
 * mm_step does), launching the passes directly and bracketing each with CUDA
 * events on the context's stream.  When flush is non-NULL, flush_bytes of
 * that device buffer are overwritten before every step so that each step
 * starts with a cold L2 (the memset is outside the bracketed passes).
 * ms[3] (host) receives the mean duration in milliseconds of pass 1 (x R2C),
 * pass 2 (y/z FFT + tensor product + inverse y/z) and pass 3 (x C2R + field +
 * LLG + Euler).  Synchronises.  Returns MM_EINVAL for reps < 1 or null ms.
 */
int mm_time_passes(mm_ctx *ctx, int reps, double dt, void *flush, unsigned long long flush_bytes,
                   float ms[3]);

/* ------------------------------------------------------------------------
 * Batches: many independent samples of uneven size stepped together (not in
 * the paper, whose runs are one sample at a time; its Sec. 4 blames small-
 * size slowness on launch overhead, which batching removes).  Sample s has
 * its own grid (nz <= 4), cell, material, field and tensor spectrum; every
 * call of mm_batch_step advances all samples by forward-Euler steps of the
 * same dt, with two batched kernels per step (the plane pass; the update,
 * which also forms the next step's x spectra) replayed from a CUDA graph
 * after one x transform of a new state, or (mm_batch_set_path
 * MM_STEP_PERSISTENT) as one cooperative launch for up to 1024 steps whose
 * blocks take (sample, tile) items from a work queue per pass, the passes
 * separated by bounded grid barriers (same arithmetic); that launch is
 * captured in a CUDA graph and replayed while its arguments stay the same.
 * M arrays of a batch are the samples' SoA blocks back to back (sample s
 * starts at float offset sum_{t<s} 3 N_t).
 * ------------------------------------------------------------------------ */
typedef struct mm_batch mm_batch;

/* grids: 3n ints; cells: 3n doubles (m); Ms, A, Ku, alpha, gamma: n doubles
 * each, same meaning as in mm_create.  Initial M uniform +x, H_ext = 0.
 * Synchronises.  MM_EINVAL / MM_EUNSUPPORTED / MM_ENOMEM / MM_ECUDA. */
int mm_batch_create(mm_batch **out, int n, const int *grids, const double *cells, const double *Ms,
                    const double *A, const double *Ku, const double *alpha, const double *gamma,
                    void *cuda_stream);
int mm_batch_destroy(mm_batch *b);                       /* NULL-safe */
int mm_batch_set_field(mm_batch *b, const double *H_ext); /* 3n doubles, A/m */
int mm_batch_set_m(mm_batch *b, const float *M);          /* host or device; synchronises */
int mm_batch_get_m(mm_batch *b, float *M);                /* host or device; synchronises */
int mm_batch_step(mm_batch *b, int n, double dt);         /* asynchronous */
/* MM_ENONFINITE if any step failed, MM_ETIMEOUT if a grid-barrier wait of the
 * persistent step gave up (the state is then incomplete until mm_batch_set_m) */
int mm_batch_sync(mm_batch *b);
/* MM_STEP_AUTO (default: the graph step), MM_STEP_GRAPH or MM_STEP_PERSISTENT;
 * MM_EUNSUPPORTED if the persistent step's blocks cannot all be resident. */
int mm_batch_set_path(mm_batch *b, int path);
/* Polls a grid-barrier wait of the persistent batch step makes before it gives
 * up (default 2^20; 0: at once, to exercise the timeout path).  polls >= 0. */
int mm_batch_set_wait_limit(mm_batch *b, long long polls);
long long mm_batch_cells(const mm_batch *b);              /* total cells, or -1 */
/* How the last mm_batch_step ran: 0 the graph step, 1 the persistent launch
 * replayed from a CUDA graph (captured once per set of launch arguments), 2
 * the persistent launch issued directly (the runtime refused its capture);
 * -1 for NULL or before any step. */
int mm_batch_launch_form(const mm_batch *b);
/*
 * mm_batch_autotune -- time the candidate tile shapes on this batch with
 * steps of size dt, keep the fastest, and restore the state (tuning does not
 * advance the samples): first the rows per CTA of the x passes and the
 * threads per CTA (12 candidates), then, with those, the kx planes per CTA
 * of the plane pass (1, 2, 4, 8).  choice (may be NULL): {rows pass 1, rows
 * pass 3, threads, planes per CTA}; ms_out (may be NULL): 16 floats, mean ms
 * per step of each candidate in that order.  Synchronises.
 */
int mm_batch_autotune(mm_batch *b, double dt, int choice[4], float *ms_out);

/* ------------------------------------------------------------------------
 * Learned surrogate of the demag field (not in the paper): a Fourier neural
 * operator that maps a magnetisation increment dM/Ms on an H x W film
 * (nz = 1) to H_demag(dM)/Ms.  Width C channels, `modes` retained modes per
 * axis direction (kx < modes, ky < modes or ky >= H - modes), `layers`
 * Fourier layers with GELU between them; BF16 weights and activations with
 * FP32 accumulation (tcgen05 tensor-core MMAs, accumulator in tensor memory,
 * for the dense contractions), an FP32 master copy of the parameters and
 * Adam.  The tensor-core waits are bounded: if one expires, the next call
 * that synchronises (mm_fno_grad, mm_fno_train_step with a loss) returns
 * MM_ETIMEOUT.  Parameter vector layout:
 * [P (C*5: three inputs, row/H, column/W), p (C), R_re (L*C*C*2m*m), R_im (same), W (L*C*C), b (L*C),
 *  Q (3*C), q (3)].  x, y, t are (batch, 3, H, W) FP32 device arrays.
 * ------------------------------------------------------------------------ */
typedef struct mm_fno mm_fno;
int mm_fno_create(mm_fno **out, int H, int W, int width, int modes, int layers, int max_batch,
                  unsigned long long seed, void *cuda_stream);
int mm_fno_destroy(mm_fno *f);                                   /* NULL-safe */
long long mm_fno_param_count(const mm_fno *f);
int mm_fno_set_params(mm_fno *f, const float *p);                /* host or device; resets Adam */
int mm_fno_get_params(mm_fno *f, float *p);                      /* host or device */
int mm_fno_forward(mm_fno *f, int batch, const float *x, float *y);
/* loss = mean (y - t)^2 and its gradient (grad: host or device, may be NULL); synchronises */
int mm_fno_grad(mm_fno *f, int batch, const float *x, const float *t, double *loss, float *grad);
/* one Adam step (beta 0.9, 0.999) with learning rate lr; loss may be NULL */
int mm_fno_train_step(mm_fno *f, int batch, const float *x, const float *t, float lr, double *loss);
/*
 * mm_step_surrogate -- n forward-Euler steps where the demag field is the
 * exact FFT convolution every `refresh` steps and, in between,
 * H_ref + Ms r FNO((M - M_ref) / (Ms r)) with (M_ref, H_ref) from the last
 * exact refresh and r the root mean square of (M - M_ref) / Ms: H_demag is
 * linear in M, so the network is trained on (and sees) unit-scale
 * increments x = dM / (Ms r) with targets H_demag(dM) / (Ms r).  At each refresh the surrogate's prediction is compared with the
 * exact field; once the relative L2 residual exceeds tol the stepper falls
 * back to the exact field for the remaining steps.  stats (may be NULL):
 * {surrogate steps, exact steps, largest residual, fell back (0/1)}.
 * Synchronises at each refresh.
 */
int mm_step_surrogate(mm_ctx *ctx, mm_fno *f, int n, double dt, int refresh, double tol, double stats[4]);

/*
 * mm_gemm_bf16 -- the surrogate's tensor-core GEMM on caller buffers (a
 * diagnostic entry point; not in the paper):
 *   C[z] = alpha A[z] B[z] + beta C[z]   (atomic == 0), or
 *   C[z] += alpha A[z] B[z]              (atomic != 0, atomicAdd per element)
 * for z < batch.  A (M x K) and B (K x N) are BF16 bit patterns (16-bit
 * words), C (M x N) FP32; element (i, k) of A[z] is A[z zA + i sam + k sak],
 * likewise B with (sbk, sbn, zB) and C with (scm, scn, zC).  All device
 * pointers owned by the caller; runs on cuda_stream (NULL: the default
 * stream) with tcgen05 MMAs (BF16 inputs, FP32 accumulation in tensor
 * memory) and synchronises it.  M, N >= 1, K >= 0 (K = 0 gives beta C),
 * batch in 1..65535, M and N <= 65535 * 128.  Returns MM_EINVAL for a null
 * pointer or a size out of range, MM_ETIMEOUT if a tensor-core wait expired
 * (C incomplete), MM_ECUDA for a launch failure.
 */
int mm_gemm_bf16(const void *A, const void *B, float *C, int M, int N, int K, long long sam, long long sak,
                 long long sbk, long long sbn, long long scm, long long scn, int batch, long long zA, long long zB,
                 long long zC, float alpha, float beta, int atomic, void *cuda_stream);

/*
 * mm_demag_field_noalloc -- H_demag of M, like mm_demag_field, for callers
 * that cannot allocate device memory: for example a host program that
 * reserves its whole device-memory budget up front and forbids later
 * allocation, or code on a latency-critical path where cudaMalloc (which may
 * synchronise the device) is not allowed.  No context is needed and nothing
 * is allocated (no cudaMalloc, cudaFree or allocating library routine): the
 * only workspace is one file-scope device array of 8 MiB inside the
 * library, which every GPU that loads the library keeps until the process
 * exits.  The paper has no counterpart; it is an interface addition.
 *
 *   grid      {nx, ny, nz}, the same limits as mm_create; the twiddle tables
 *             plus the x half-spectrum workspace, (Lx+Ly+Lz) + 3*(Lx/2+1)*ny*nz
 *             complex floats (each padded length chosen as in mm_create), must
 *             fit in the 8 MiB array (e.g. 256 x 256 x 4 fits, 512 x 512 x 8
 *             does not); larger grids return MM_EUNSUPPORTED with the sizes
 *             in mm_last_error().
 *   Kt_dev    the scaled tensor spectrum exactly as mm_kernel_spectrum
 *             copies it out of a context built for the same grid and cell
 *             (device memory).
 *   kt_elems  the number of floats in Kt_dev; it must equal
 *             6*(Lx/2+1)*(Ly/2+1)*(Lz/2+1) for this grid's padded lengths
 *             (the size mm_kernel_spectrum writes), else MM_EINVAL.
 *   M_dev, H_dev  3*N float32 device arrays, must not overlap.
 *   cuda_stream   stream to run on (NULL = legacy default stream).
 *
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture.  Every call shares the array and its last
 * contents: calls whose GPU work overlaps in time (other streams, other host
 * threads) race and give wrong results, so serialise them.  Each call writes
 * every workspace element it reads before reading it, so no clearing is
 * needed.  Asynchronous.  Returns MM_EINVAL, MM_EUNSUPPORTED or MM_ECUDA.
 */
int mm_demag_field_noalloc(const int grid[3], const float *Kt_dev, long long kt_elems, const float *M_dev,
                           float *H_dev, void *cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* MM_H */
