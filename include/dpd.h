/*
 * libdpd — augmented-parallel-Hammerstein (APH) digital predistortion on one
 * NVIDIA GB300 (sm_103a).
 *
 * The filter is the joint PA / I/Q-modulator predistorter of Li et al.,
 * "Parallel Digital Predistortion Design on Mobile GPU and Embedded Multicore
 * CPU for Mobile Transmitters" (Eq. 1, Algorithm 1):
 *
 *   y_n = sum_{p in I_P} sum_{k=0}^{M} h_{p,k}    |x_{n-k}|^{p-1} x_{n-k}
 *       + sum_{q in I_Q} sum_{k=0}^{M} hbar_{q,k} |x_{n-k}|^{q-1} conj(x_{n-k})
 *       + c,
 *
 * I_P = {1, 3, ..., P}, I_Q = {1, 3, ..., Q}, every branch an FIR of L = M + 1
 * taps, samples before x_0 taken as zero.  (The paper writes the input x and the
 * output z; this library calls the output y.)  The paper's orthogonalising
 * polynomial coefficients u_{m,p} (Sec. 2.1) are the identity here; a caller who
 * wants them folds them into h, since the filter is linear in h.
 *
 * Data layout.  Samples are complex64: interleaved (re, im) float32 pairs, the
 * layout of C99 `float complex`, `std::complex<float>` and torch.complex64.
 * Coefficient vectors use the stacking order of Sec. 2.2:
 *   h = [h_1[0..M], h_3[0..M], ..., h_P[0..M], hbar_1[0..M], ..., hbar_Q[0..M], c]
 * so K = ((P+1)/2 + (Q+1)/2) * (M+1) + 1 complex values.
 *
 * Streams.  Every `stream` argument is a cudaStream_t passed as void* (NULL is
 * the legacy default stream).  Device work is enqueued on it and the call
 * returns without synchronising unless stated otherwise.  Call every function
 * with the CUDA device that was current at dpd_create current.
 *
 * Errors.  Every call returns a dpd_status; nothing exits, aborts or traps.
 * Argument errors are found on the host before any work is enqueued.  Errors
 * raised by kernels (a bounded wait that ran out) are recorded in a per-handle
 * device word that dpd_sync_status reads.
 *
 * Thread safety.  A handle may be used from one host thread at a time.
 */
#ifndef DPD_H
#define DPD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum dpd_status {
    DPD_OK = 0,
    DPD_ERR_INVALID_ARGUMENT = 1, /* bad pointer, size, order, overlap or alignment */
    DPD_ERR_UNSUPPORTED = 2,      /* valid in principle but outside the built range */
    DPD_ERR_NO_COEFFS = 3,        /* dpd_apply/dpd_grad before dpd_set_coeffs */
    DPD_ERR_CUDA = 4,             /* a CUDA runtime call or launch failed */
    DPD_ERR_ALLOC = 5,            /* device or host allocation failed */
    DPD_ERR_NOT_SPD = 6,          /* least-squares Gram matrix not positive definite */
    DPD_ERR_TIMEOUT = 7           /* a kernel's bounded wait ran out (device flag) */
} dpd_status;

/* Where a coefficient buffer lives. */
enum { DPD_HOST = 0, DPD_DEVICE = 1 };

typedef struct dpd_filter *dpd_handle;

/*
 * Create a filter for main-branch order P, conjugate-branch order Q and memory
 * depth M (L = M + 1 taps per branch), on the current CUDA device.
 *   P, Q : odd, 1..11, or 0 for "no such branch".  The paper uses odd orders
 *          only (Sec. 2.1): an even order, or one above 11, gives
 *          DPD_ERR_UNSUPPORTED; a negative order, or P = Q = 0, gives
 *          DPD_ERR_INVALID_ARGUMENT.
 *   M    : 0..7 (1 to 8 taps); M > 7 gives DPD_ERR_UNSUPPORTED, M < 0
 *          DPD_ERR_INVALID_ARGUMENT.
 * dpd_plan_batched and dpd_grad_coeffs_noalloc check their models the same way.
 * The handle owns its device memory (coefficients, their transformed form, an
 * error word and the gradient workspace).  *out is set only on success.
 */
dpd_status dpd_create(int P, int Q, int M, dpd_handle *out);

/* Release a handle and its device memory.  NULL is accepted.  The caller must
 * make sure no work that uses the handle is still running. */
dpd_status dpd_destroy(dpd_handle h);

/* Number of complex coefficients K of the handle's model (Sec. 2.2). */
dpd_status dpd_num_coeffs(dpd_handle h, int *K);

/*
 * Install the coefficient vector h (K complex64 values, stacking order of
 * Sec. 2.2).  `where` is DPD_HOST or DPD_DEVICE.  Host buffers are copied and
 * the call synchronises `stream` (it keeps a host copy of the prepared table,
 * so it must not be captured in a CUDA graph); device buffers are read by a
 * kernel on `stream` without synchronising (capturable), so they must stay
 * valid until that kernel has run.  The caller keeps ownership.
 * The kernels take the prepared tables as launch arguments when a host copy
 * exists, else read them from device memory (same results, bit for bit).  After
 * a device-side set outside graph capture the tables are copied back to pinned
 * host memory behind the set, without waiting; calls made once that copy has
 * landed (checked without blocking) take them as arguments.  A CUDA graph
 * captured after a host-side set keeps those coefficients; one captured after
 * a device-side set reads the tables on the device at every replay.
 * K must equal dpd_num_coeffs.  Work is ordered on `stream`: later calls on
 * the same stream see the new coefficients.
 */
dpd_status dpd_set_coeffs(dpd_handle h, const void *coeffs, int K, int where, void *stream);

/*
 * Predistort n samples: y = DPD(x) (Eq. 1), zero history before x[0].
 *   x, y : device pointers to n complex64 each, 8-byte aligned, owned by the
 *          caller; the ranges must not overlap (DPD_ERR_INVALID_ARGUMENT).
 *          16-byte alignment of both selects the bulk-copy (TMA) pipeline.
 *   n    : >= 0; n == 0 returns DPD_OK and launches nothing.
 * Allocates nothing and does not synchronise; safe to capture in a CUDA graph.
 */
dpd_status dpd_apply(dpd_handle h, const void *x, void *y, int64_t n, void *stream);

/* Modes of dpd_apply_host. */
enum { DPD_HOST_PIPELINED = 0, DPD_HOST_ZERO_COPY = 1 };

/*
 * dpd_apply on buffers in host memory (x, y: n complex64 each, 8-byte aligned,
 * not overlapping; pinned / registered, managed, or -- where the GPU can access
 * it, as on Grace-Blackwell -- ordinary pageable memory; device memory is
 * rejected, use dpd_apply).
 *   DPD_HOST_PIPELINED : the input is cut into chunks of 2^21 samples; each
 *       chunk (with 8 samples of history in front) is copied to the device,
 *       filtered and copied back on one of three internal streams in turn, so
 *       copies in both directions overlap the kernels (the multi-stream
 *       alternative of Sec. 3.4).  The first call allocates the staging buffers
 *       (3 x 2 x 16 MB) and streams; pinned buffers make the copies
 *       asynchronous.
 *   DPD_HOST_ZERO_COPY : the kernel reads and writes the host buffers in place
 *       over the CPU-GPU link, without staging copies (Sec. 3.3.1).  With both
 *       buffers 16-byte aligned, each CTA moves a 2048-sample tile (plus 8
 *       history samples) with coalesced 16-byte accesses through shared
 *       memory, so every byte crosses the link once; otherwise every thread
 *       loads its own window with 8-byte loads (slower).
 * Ordered after earlier work on `stream`; returns without synchronising, and
 * `stream` is ordered after the last chunk: synchronise it before reading y.
 * Not capturable in a CUDA graph.
 */
dpd_status dpd_apply_host(dpd_handle h, const void *x, void *y, int64_t n, int mode, void *stream);

/*
 * Coefficient gradient without any device allocation.  (Not in the paper; a
 * library convenience.)  Some callers may not allocate device memory at all:
 * a transmit chain that forbids cudaMalloc once it is streaming (an allocation
 * can synchronise the device and take unbounded time), or a host framework
 * that owns every byte of device memory.  Such a caller cannot create a
 * handle, because dpd_create allocates the handle's workspace.  This entry
 * point needs no handle and allocates nothing: its scratch is a fixed array of
 * 512 x 97 complex64 values (397,312 bytes) compiled into the library, which
 * every device that loads the library keeps until the process exits.
 *
 * Computes the same gh as dpd_grad (K values for the model P, Q, M; no
 * coefficients are needed).  x, gy: device, n complex64, 8-byte aligned; gh:
 * device, K complex64, overwritten, must not overlap x or gy.  n == 0 zeroes
 * gh.  Models beyond the scratch (K > 97) give DPD_ERR_UNSUPPORTED, as does a
 * device ordinal >= 64.  The first call on a device looks up the scratch's
 * device address (cudaGetSymbolAddress); with CUDA's lazy module loading that
 * lookup also loads the library's device code, which reserves the scratch and
 * the code on the device and may synchronise it.  So a caller that must not
 * allocate later makes one call with n == 0 at start-up (it does this one-time
 * set-up and zeroes gh), before any stream capture; each kernel is then
 * loaded at its own first launch, so such a caller also runs each model once
 * before streaming.  After that a call allocates nothing.  All calls on a
 * device share the scratch and each call rewrites the rows it reads, so
 * nothing carries over between calls, but calls whose kernels overlap on the
 * GPU (different streams, or different host threads) race on it and must be
 * serialised by the caller.  This entry point has no device error word: it
 * runs the plain-load coefficient-gradient kernel (no bulk-copy ring and no
 * bounded waits, so there is no timeout to report), which is slower than
 * dpd_grad's staged kernel on 16-byte aligned buffers.
 */
dpd_status dpd_grad_coeffs_noalloc(int P, int Q, int M, const void *x, const void *gy, int64_t n,
                                   void *gh, void *stream);

/*
 * Adjoint of dpd_apply for a real loss L (not in the paper: used for
 * gradient-based direct learning).  Given gy = dL/dy for y = DPD(x), writes
 *   gh[j] = sum_n conj(Psi_{n,j}) gy_n            (K values, Psi of Eq. 2)
 *   gx[i] = sum_k conj(dy_{i+k}/dx_i) gy_{i+k} + (dy_{i+k}/dconj(x_i)) conj(gy_{i+k})
 * with every gradient in the convention dL/dRe + j dL/dIm (PyTorch's).
 *   x, gy : device, n complex64 each, 8-byte aligned.
 *   gh    : device, K complex64, or NULL; overwritten (not accumulated).
 *   gx    : device, n complex64, or NULL; overwritten; must not overlap x, gy, gh.
 * At least one of gh, gx non-NULL.  gx needs coefficients (DPD_ERR_NO_COEFFS),
 * gh does not.  The basis is recomputed from x; nothing from dpd_apply is kept.
 * gh is reduced through the handle's workspace (one partial row per CTA, summed
 * in FP64 in a fixed order): results are deterministic, and calls on one handle
 * must not run concurrently on different streams.  n == 0 zeroes gh.
 * Allocates nothing; does not synchronise.
 */
dpd_status dpd_grad(dpd_handle h, const void *x, const void *gy, int64_t n, void *gh, void *gx,
                    void *stream);

/*
 * Launch shape of dpd_grad's coefficient-gradient kernel (used by the
 * autotuner): gh_blocks CTAs per tap group (1 .. 4 * SM count), tap_group taps
 * per group (1 .. 5).  Returns DPD_ERR_INVALID_ARGUMENT outside those ranges.
 */
dpd_status dpd_set_adj_launch(dpd_handle h, int gh_blocks, int tap_group);

/*
 * Streaming predistortion: consecutive calls filter consecutive blocks of one
 * continuous sample stream (the predistortion stage filters a continuous
 * stream of transmit samples, Sec. 2 and Sec. 4).  The history before x[0] is the last M input
 * samples of the previous dpd_apply_stream call on this handle (zero after
 * dpd_create or dpd_reset_stream), so the outputs equal one dpd_apply over the
 * concatenated input.  Two launches on `stream`: the forward filter (zero
 * history), then one warp that recomputes y[0 .. min(M, n)) with the saved
 * history and saves the last 8 input samples into the handle.  Calls on one
 * handle must therefore be ordered on one stream (or synchronised), and x must
 * stay valid until the second launch has run.  Same buffer rules and errors as
 * dpd_apply; n == 0 changes nothing.  Allocation-free and capturable.
 */
dpd_status dpd_apply_stream(dpd_handle h, const void *x, void *y, int64_t n, void *stream);

/* Zero the streaming history (asynchronously on `stream`). */
dpd_status dpd_reset_stream(dpd_handle h, void *stream);

/*
 * Direct-learning loss and its gradient in one pass (not in the paper, whose
 * coefficients are found by indirect learning, Sec. 2.2):
 *   loss[0] = scale * sum_n |y_n - g x_n|^2            (FP64 sum, fixed order, stored as float)
 *   gy[n]   = 2 scale (y_n - g x_n)  (dL/dRe + j dL/dIm), when gy is non-null
 * with g = gain_re + j gain_im.  y, x, gy: device complex64 (n each, 8-byte
 * aligned; gy must not overlap x or y); loss: one device float.  Uses the
 * handle's scratch, so calls on one handle must be ordered on one stream.
 * Allocation-free and capturable.
 */
dpd_status dpd_sq_error(dpd_handle h, const void *y, const void *x, int64_t n, float gain_re, float gain_im,
                        double scale, float *loss, void *gy, void *stream);

/*
 * Launch shape of dpd_apply for this handle (used by the autotuner):
 *   mode        bit 0: coefficients passed by value as kernel parameters (used
 *               only after dpd_set_coeffs from host memory; otherwise ignored);
 *               bit 1: packed two-wide FP32 fused multiply-adds
 *   V           samples per thread, 2, 4, 6 or 8 (with 6 the 16-byte window
 *               loads of a warp are free of shared-memory bank conflicts)
 *   warps       consumer warps per CTA, 1..16 (tile = warps*32*V samples)
 *   stages      depth of each group's shared-memory bulk-copy ring, 2..8
 *   ctas_per_sm CTAs per SM of the persistent grid, 0 = as many as fit
 *   use_tma     1 = bulk-copy pipeline, 0 = plain global loads
 *   group       warps per group, dividing `warps`, or 0 for one group of all
 *               warps: every group has its own ring and barriers and runs on
 *               its own sub-tile (group*32*V samples), independently of the
 *               CTA's other groups
 * Default: mode 3, V 8, 16 warps in groups of 4, 4 stages, as many CTAs as
 * fit, TMA.  Every (P, Q, M) has modes 2 and 3 at V 4, 6 and 8 and mode 0 at
 * V 4; other combinations exist only for the benchmarked orders.  Rings that do
 * not fit one CTA's shared memory give DPD_ERR_UNSUPPORTED; a shape that does
 * not fit the device otherwise, or one not built for the handle's (P, Q, M),
 * makes dpd_apply return DPD_ERR_CUDA.
 */
dpd_status dpd_set_fwd_launch(dpd_handle h, int mode, int V, int warps, int stages, int ctas_per_sm,
                              int use_tma, int group);

/* ------------------------------------------------------------ least squares */

/* Precision of the Gram contraction Psi^H Psi (accumulation is FP32, the
 * K x K solve FP64 in every mode):
 *   DPD_PREC_FP32    plain FP32 fused multiply-adds on the CUDA cores
 *   DPD_PREC_TF32X3  tensor cores, operands split a = hi + lo in TF32,
 *                    hi*hi + hi*lo + lo*hi (about FP32 accuracy)
 *   DPD_PREC_BF16X3  tensor cores, the same split in BF16 (about 16 bits) */
enum { DPD_PREC_FP32 = 0, DPD_PREC_TF32X3 = 1, DPD_PREC_BF16X3 = 2 };

/*
 * Normal equations of the least-squares estimate of Sec. 2.2 for the
 * handle's model: G = Psi^H Psi (K x K) and g = Psi^H t, Psi the basis matrix
 * of Eq. 2 built from u (zero history, n rows).
 *   u  : device, n complex64, 8-byte aligned (n >= 1)
 *   t  : device, n complex64, or NULL (then g and tt are not formed)
 *   G  : device, K*K complex128 (row-major, full Hermitian), written
 *   g  : device, K complex128, or NULL;  tt : host double (t^H t) or NULL
 * Uses and may grow the handle's estimation workspace (growing allocates and
 * synchronises the device); tt != NULL synchronises `stream`.
 */
dpd_status dpd_gram(dpd_handle h, const void *u, const void *t, int64_t n, int precision, void *G, void *g,
                    double *tt, void *stream);

/* Bases of the least-squares estimate. */
enum { DPD_BASIS_MONOMIAL = 0, DPD_BASIS_ORTHOGONAL = 1 };

/*
 * Basis in which dpd_estimate and dpd_estimate_batched solve the least-squares
 * problem (the handle's state; default DPD_BASIS_MONOMIAL).
 *   DPD_BASIS_ORTHOGONAL : the statistically orthogonal polynomials of Sec. 2.1,
 *       psi_p(x) = sum_{m <= p} u_{m,p} |x|^{m-1} x, with u_{m,p} computed from
 *       the estimation input itself: the power sums of |u|^2 give the Gram
 *       matrix of the monomials, whose Cholesky factor L yields U = L^{-T}
 *       (FP64 on the host), so the basis functions are orthonormal over u.
 *       Both branches and every tap use the same U.  The Gram matrix is
 *       formed and solved in that basis (much better conditioned), and the
 *       coefficients are converted back, h = W h_orth, so the output is always
 *       in the monomial stacking order of Sec. 2.2 that dpd_set_coeffs takes.
 *       One extra synchronisation per call (the power sums are read back).
 * dpd_gram always uses the monomials.
 */
dpd_status dpd_set_estimate_basis(dpd_handle h, int basis);

/*
 * Least-squares coefficients (Sec. 2.2): h = argmin ||Psi(u) h - t||_2, i.e.
 * (Psi^H Psi) h = Psi^H t.  The Gram matrix is formed in `precision`, the
 * system is equilibrated (D = diag(G)^{-1/2}) and solved by an FP64 Cholesky
 * factorisation, then refined `refine_iters` times (0..100) with
 * h += G^{-1} Psi^H (t - Psi h), the residual computed by the FP32 filter
 * and adjoint kernels.  In the indirect learning architecture u is the PA
 * output divided by its gain and t the predistorter output.
 *   h_out : device, K complex64, written (the handle's own coefficients are
 *           left unchanged; install the result with dpd_set_coeffs)
 *   stats : host double[2] or NULL: [0] 2-norm condition number of D G D
 *           (Lanczos on the FP64 Cholesky factor, host; about 1e-11 relative),
 *           [1] ||t - Psi h||^2 / ||t||^2 of the returned h (FP32 residual,
 *           FP32 squares summed in runs of 32, runs summed in FP64)
 * Synchronises `stream` once, at the end: the condition estimate runs on the
 * host while the refinement runs on the device.  DPD_ERR_NOT_SPD if G is not
 * positive definite (e.g. u all zero); h_out and stats are then unspecified.
 * Uses and may grow the handle's workspace (device buffers and a few pinned
 * host buffers).
 */
dpd_status dpd_estimate(dpd_handle h, const void *u, const void *t, int64_t n, int precision, int refine_iters,
                        void *h_out, double *stats, void *stream);

/*
 * `count` independent estimates for the handle's model (e.g. one per antenna):
 * u[i], t[i] device pointers to n[i] complex64.  One Gram launch covers every
 * problem; h_out receives count*K complex64 (problem-major).  info_out (host,
 * count ints, nullable) gets 0 or the failing Cholesky pivot + 1 per problem;
 * any failure returns DPD_ERR_NOT_SPD after the others are solved.
 */
dpd_status dpd_estimate_batched(dpd_handle h, const void *const *u, const void *const *t, const int64_t *n,
                                int count, int precision, int refine_iters, void *h_out, int *info_out,
                                void *stream);

/* ------------------------------------------------------------------ batched */

/*
 * One antenna stream of a batched plan (not in the paper; the batched form
 * filters many independent transmit chains in one launch).  Each stream is an
 * independent instance of Eq. 1 with its own model, coefficients and zero
 * history.
 *   x : device, n complex64, 16-byte aligned (bulk copies)
 *   y : device, n complex64, 8-byte aligned; must not overlap any stream's x
 *       or another stream's y
 *   n : >= 0;  P, Q, M : as for dpd_create
 *   h : K complex64 coefficients, stacking order of Sec. 2.2, in host or
 *       device memory as given by the `where` argument of dpd_plan_batched
 */
typedef struct dpd_stream_desc {
    const void *x;
    void *y;
    int64_t n;
    int P, Q, M;
    const void *h;
} dpd_stream_desc;

typedef struct dpd_plan_s *dpd_plan;

/*
 * Build a plan for `count` streams: copies the coefficients and prepares their
 * tables, cuts the streams into tiles and uploads the work list (ordered by
 * per-sample cost).  The x / y pointers are recorded in the plan; a plan is
 * executed on those buffers.  Allocates the plan's device memory and
 * synchronises the device; the caller keeps ownership of descs and h.
 */
dpd_status dpd_plan_batched(const dpd_stream_desc *descs, int count, int where, dpd_plan *out);

/*
 * Filter every stream of the plan with ONE persistent kernel launch on
 * `stream`.  Allocates nothing and does not synchronise: capture it in a CUDA
 * graph and replay.  Concurrent executions of one plan must not overlap.
 */
dpd_status dpd_exec_batched(dpd_plan plan, void *stream);

/*
 * Launch shape of dpd_exec_batched (autotuner): V in {4, 6, 8} samples per thread,
 * warps 1..16 consumer warps (tile = warps*32*V samples; changing the tile
 * rebuilds the work list, synchronously, in a new device buffer), stages 2..8,
 * ctas_per_sm >= 0 (0 = as many as fit), group = warps per group dividing
 * `warps` (every group has its own ring of slots and barriers and filters its
 * own part of each work item) or 0 for one group.  Default 8, 8, 4, 0, 0.
 * Rings larger than one CTA's shared memory give DPD_ERR_UNSUPPORTED.  On any
 * error the plan keeps its previous shape and work list.  A CUDA graph
 * captured from dpd_exec_batched holds the shape and work list of its
 * capture: capture again after changing the shape.
 */
dpd_status dpd_plan_set_launch(dpd_plan plan, int V, int warps, int stages, int ctas_per_sm, int group);

/* Synchronise `stream`, read and clear the plan's device error word (as dpd_sync_status). */
dpd_status dpd_plan_sync_status(dpd_plan plan, void *stream);

/* Free a plan (NULL accepted).  No execution of it may still be running. */
dpd_status dpd_plan_destroy(dpd_plan plan);

/*
 * Synchronise `stream`, then read and clear the handle's device error word.
 * Returns DPD_ERR_TIMEOUT if a kernel recorded that a bounded wait ran out,
 * DPD_ERR_CUDA if the stream reported an error, else DPD_OK.
 */
dpd_status dpd_sync_status(dpd_handle h, void *stream);

/* Human-readable name of a status code (static storage). */
const char *dpd_status_string(dpd_status s);

/* Number of kernels this library has launched in this process (all handles). */
uint64_t dpd_kernel_launches(void);

/*
 * Measurement aid (not in the paper): the FP32 fused-multiply-add ceiling that
 * bounds the filter and adjoint kernels, measured rather than taken from
 * nominal lane counts.  Launches `blocks` CTAs of 256 threads on `stream`;
 * every thread runs `iters` iterations of 16 independent FMAs (as 8 packed
 * f32x2 FMAs when `packed` is non-zero, else 16 scalar ones) and writes one
 * float to sink[block * 256 + thread].
 *   sink : device, blocks * 256 floats, 4-byte aligned, owned by the caller.
 * FMAs executed = blocks * 256 * iters * 16; time the launch with events on
 * `stream`.  Allocates nothing, does not synchronise.
 */
dpd_status dpd_probe_fma(int blocks, int iters, int packed, void *sink, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* DPD_H */
