/*
 * leg.h -- C ABI of the GB300 (sm_103a) Legendre-coefficient library.
 *
 * Method: De Micheli & Viano, "A new and efficient method for the computation
 * of Legendre coefficients" (arXiv:1106.0463).  For f(x) = sum_n c_n P_n(x)
 * (Eq. 2.1) with c_n = (n + 1/2) int_{-1}^{1} f P_n dx (Eq. 2.3), Theorem 1
 * (Eq. 2.4, Eq. 2.5) gives a_n = c_n / (2n+1) as the nonnegative-index Fourier
 * coefficients of the Abel-type transform
 *     fhat(y) = eps(y) e^{iy/2} / (2 pi i) * int_{cos y}^{1} f(x) / sqrt(2(x - cos y)) dx.
 * The library evaluates fhat on the periodic grid y_j = 2 pi j / M by
 * quadrature (substitution x = cos y + s^2, Gauss-Legendre in s; Sec. 2, the
 * paragraph after Eq. 2.14) and takes one length-M FFT (the paragraph that
 * follows it).  For f given by samples at the K Chebyshev-Lobatto nodes the
 * Abel step is a dense (M/2+1) x K operator applied to a batch of functions
 * (the rows j and M-j coincide by the symmetry Eq. 2.12).
 *
 * Conventions used by every entry point:
 *  - Input samples: f[b*K + k] = f_b(x_k), x_k = cos(pi k / (K-1)),
 *    k = 0..K-1 (x_0 = +1 first, x_{K-1} = -1 last), row-major B x K.
 *  - Output: c[b*N + n] = c_n of function b, n = 0..N-1, row-major B x N.
 *  - All array pointers are DEVICE pointers unless stated otherwise; the
 *    caller owns them.  Nothing is copied to or from the host, and no call
 *    synchronises the host with the stream (except leg_plan_create and the
 *    first call that grows a plan's workspace, see leg_plan_reserve).
 *  - Calls are asynchronous on the given stream (0 = legacy default stream).
 *  - Return value: LEG_OK (0) or one of the LEG_ERR_* codes below; a
 *    human-readable message for the last error of the calling thread is
 *    returned by leg_last_error().  Argument errors are reported before any
 *    work is enqueued.
 *  - Fault injection (tests of the error paths): with the environment
 *    variable LEG_FAULT_ALLOC = k (k >= 1), the k-th device allocation the
 *    library attempts after the variable took that value fails on the host,
 *    without allocating, and the call returns LEG_ERR_OOM having released
 *    what it had allocated for that call (a plan's grown workspace stays with
 *    the plan until it is destroyed).
 */
#ifndef LEG_H
#define LEG_H

#include <stddef.h>
#include <cuda_runtime_api.h>

#if defined(__GNUC__)
#define LEG_API __attribute__((visibility("default")))
#else
#define LEG_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define LEG_OK               0
#define LEG_ERR_INVALID_ARG  1  /* bad size, null pointer, bad enum, N > M/2 ... */
#define LEG_ERR_OOM          2  /* device or host allocation failed            */
#define LEG_ERR_CUDA         3  /* a CUDA runtime/driver call failed           */
#define LEG_ERR_UNSUPPORTED  4  /* valid request this build does not implement */
#define LEG_ERR_TIMEOUT      5  /* a bounded device-side wait expired          */

/* ---- arithmetic of a plan ---------------------------------------------- */
/*
 * The operator itself is always built in FP64 (Gauss nodes and weights, the
 * node mapping 1 - x = 2 sin^2(y/2)(1 - tau^2), barycentric interpolation).
 * The dtype selects how it is applied:
 *   LEG_F64        f, c in FP64; FP64 GEMM on the CUDA cores, FP64 FFT.
 *                  The plain FP64 GPU path.
 *   LEG_F32        f, c in FP32; FP32 GEMM on the CUDA cores (FFMA), FP32 FFT.
 *   LEG_BF16       f, c in FP32; one BF16 x BF16 tensor-core product with
 *                  FP32 accumulation (tcgen05), FP32 FFT.
 *   LEG_SPLIT_FP16 f, c in FP32; operator split into three FP16 slices (a
 *                  fixed-point leading slice, two residual slices), input
 *                  into seven pre-scaled FP16 planes (slice widths chosen by
 *                  K: 15 + 8 bits for K <= 1025, 16 + 7 above); eight tcgen05 products
 *                  into three FP32 TMEM accumulators of which the leading one
 *                  is exact, combined into a double-float result;
 *                  double-float FFT.  The path aimed at a 1e-6 relative error.
 */
typedef enum {
    LEG_F64 = 0,
    LEG_F32 = 1,
    LEG_BF16 = 2,
    LEG_SPLIT_FP16 = 3
} leg_dtype;

/* plan flags (leg_plan_create_ex) */
#define LEG_FLAG_TAU_LITERAL 1u  /* Q-point Gauss rule mapped onto tau in [0,1]
                                    instead of the nonnegative half of a
                                    2Q-point rule (the default)               */
/*
 * LEG_FLAG_COLLAPSED: the plan multiplies out, at plan time and in FP64, the
 * whole linear map of Theorem 1 (Eq. 2.4, Eq. 2.5) on sampled inputs,
 *     L = R A   (N x K),  c = L f,
 * A the (M/2+1) x K Abel-interpolation operator and R the N x (M/2+1)
 * matrix of the twisted transform with the (2n+1) factor (computed by
 * applying the plan's FP64 transform to the columns of A).  leg_forward is
 * then one GEMM with no transform stage and leg_backward one transposed
 * GEMM (df = L^T dc), in the plan's dtype.  The paper evaluates the map as
 * the Abel step followed by an FFT; the collapsed form is the same linear
 * map (up to rounding) with a different factorisation, cheaper when N < M/2
 * and the batch is large.  Ragged batches and leg_forward_noalloc take plans
 * without this flag.
 */
#define LEG_FLAG_COLLAPSED   2u
/*
 * LEG_FLAG_SINE_FORM: the plan's forward transform evaluates the half-range
 * sine form of the coefficients (Eq. 2.13, with phi of Eq. 2.14; the paper
 * derives it from the symmetry Eq. 2.12),
 *     c_n = (2/pi)(n + 1/2) int_0^pi phi(y) sin((n + 1/2) y) dy,
 *     phi(y) = int_{cos y}^1 f(x) / sqrt(2(x - cos y)) dx = 2 sin(y/2) g(y),
 * by the trapezoid rule on y_j = 2 pi j / M, j = 0..M/2: a DST-III of length
 * M/2 of phi, computed through one complex FFT of length M/4 (the factor
 * 2 sin(y/2) merged into its pre-twiddle), instead of the real-even transform
 * of the full period followed by a first difference (Eq. 2.4, Eq. 2.5).  Both
 * are the same discrete linear map; results differ by rounding only.  Needs
 * M >= 256 (LEG_ERR_UNSUPPORTED otherwise); not with LEG_FLAG_COLLAPSED.  The
 * same choice is available on any plan through leg_plan_set_transform.
 */
#define LEG_FLAG_SINE_FORM   4u

/* Forward transform kernels (leg_plan_set_transform); the same map, rounding differs. */
#define LEG_TRANSFORM_REG      0  /* register-tiled real-even transform (M >= 256; FP32 plans: Stockham) */
#define LEG_TRANSFORM_STOCKHAM 1  /* shared-memory Stockham real-even transform                     */
#define LEG_TRANSFORM_SINE     2  /* register-tiled half-range sine form, Eq. 2.13 (M >= 256)        */

typedef struct leg_plan *leg_plan_t;

/*
 * leg_plan_create -- build the Abel-interpolation operator for one problem size.
 *   N  number of coefficients returned, 1 <= N <= M/2.
 *   M  trapezoid points on [0, 2 pi), a power of two, 8 <= M <= 32768.
 *   K  Chebyshev-Lobatto samples per function, 2 <= K <= 16385.
 *   Q  distinct Gauss nodes per y-point in the Abel integral; Q = 0 selects
 *      ceil(K/2), which integrates the degree-(K-1) interpolant exactly.
 *   dtype  one of leg_dtype.
 * Builds the operator on the current device (FP64 kernels), derives the
 * operand planes for dtype, and stores them in device memory owned by the
 * plan.  Synchronises the host with the device once.  *out receives the
 * plan; on error *out is set to NULL.
 * Errors: LEG_ERR_INVALID_ARG (sizes, dtype, out == NULL), LEG_ERR_OOM,
 * LEG_ERR_CUDA, LEG_ERR_UNSUPPORTED (dtype not available for this size).
 */
LEG_API int leg_plan_create(leg_plan_t *out, int N, int M, int K, int Q, int dtype);
LEG_API int leg_plan_create_ex(leg_plan_t *out, int N, int M, int K, int Q, int dtype, unsigned flags);

/*
 * leg_plan_create_like -- a plan of another dtype for the same (N, M, K, Q,
 * flags) as src, reusing src's FP64 operator (a device copy) instead of
 * building it again; only the operand planes of the new dtype are derived.
 * Synchronises the host with the device.  Errors as leg_plan_create.
 */
LEG_API int leg_plan_create_like(leg_plan_t *out, leg_plan_t src, int dtype);

/* Releases every device buffer of the plan.  NULL is accepted. */
LEG_API int leg_plan_destroy(leg_plan_t plan);

/*
 * leg_plan_reserve -- make the plan's workspace large enough for batches of
 * up to B functions.  Allocation synchronises; call it before capturing
 * leg_forward / leg_backward into a CUDA graph.  leg_forward grows the
 * workspace by itself when B exceeds the reservation.
 */
LEG_API int leg_plan_reserve(leg_plan_t plan, int B);

/* Sizes of a plan: N, M, K, Q (resolved), dtype, padded K, rows M/2+1. */
LEG_API int leg_plan_info(leg_plan_t plan, int *N, int *M, int *K, int *Q, int *dtype,
                  int *K_padded, int *rows);

/*
 * leg_forward -- c = L f for a batch of B functions (Theorem 1, Eq. 2.4-2.5).
 *   f  device, B x K row-major (FP64 for LEG_F64, FP32 otherwise).
 *   c  device, B x N row-major (FP64 for LEG_F64, FP32 otherwise).
 *   B  >= 0; B = 0 is a no-op.
 * Enqueued on stream; f and c must not overlap.  Concurrent calls on one
 * plan from different streams race on its workspace: use one plan per stream.
 * The kernels are chained by programmatic dependent launch.  The first call
 * with given (f, c, B) and launch settings runs its launches directly, the
 * second captures them into a CUDA graph (on a stream of the plan's own) and
 * later ones replay that graph on `stream` (the graphs of the two most
 * recently used (f, c, B, settings) keys are kept); a change of f, c, B, the
 * workspace, the tile width, the transform kernel or the wait limit starts
 * over.  A call made while `stream` is being captured by the caller launches
 * directly, so its kernels become part of the caller's graph.
 */
LEG_API int leg_forward(leg_plan_t plan, const void *f, void *c, int B, cudaStream_t stream);

/*
 * leg_forward_batches -- leg_forward on nbatch batches of B functions, one
 * after another (Theorem 1, Eq. 2.4-2.5, for each function).  (A scheduling
 * convenience for a stream of batches; the paper has no counterpart.)
 *   f  device, nbatch x B x K row-major (batch b starts at row b*B), the
 *      type of leg_forward's f;
 *   c  device, nbatch x B x N, leg_forward's c type; overwritten.
 *   B, nbatch  >= 0; either 0 is a no-op.
 * The results are those of nbatch calls of leg_forward, bit for bit.  For
 * LEG_SPLIT_FP16 plans of the Abel GEMM + transform, the batches run as a
 * two-stage pipeline on two internal streams of the plan: the input split
 * and the GEMM of batch b on a high-priority stream, the transform of batch
 * b-1 on a low-priority one after batch b's split, so that the transform
 * runs on the SMs the GEMM's CTA pairs leave free.  The GEMM results
 * alternate between the plan's two G-sized workspaces (the forward's and the
 * backward's).  Ordered after the work already on `stream`; later work on
 * `stream` sees every batch complete.  Other plans, nbatch = 1 and calls on
 * a stream being captured run the batches through leg_forward in order.
 * Errors: those of leg_forward; LEG_ERR_INVALID_ARG for B < 0 or nbatch < 0.
 */
LEG_API int leg_forward_batches(leg_plan_t plan, const void *f, void *c, int B, int nbatch, cudaStream_t stream);

/*
 * leg_forward_batches_profiled -- leg_forward_batches that also returns the
 * mean time per batch (milliseconds) of each stage: ms[0] the input
 * preparation, ms[1] the GEMM, ms[2] the transform, taken with CUDA events on
 * the stage's own stream inside the pipeline (for pipelined plans; other
 * plans and nbatch = 1 average leg_forward_profiled over the batches).  The
 * events between the stages change the launch chaining slightly, so the
 * stage times are for the roofline figures, not for the throughput.
 * Synchronises `stream`; LEG_ERR_INVALID_ARG on a stream being captured or
 * for a NULL ms.  Otherwise as leg_forward_batches.
 */
LEG_API int leg_forward_batches_profiled(leg_plan_t plan, const void *f, void *c, int B, int nbatch,
                                         cudaStream_t stream, float *ms);

/*
 * leg_forward_profiled -- leg_forward with CUDA events recorded on `stream`
 * between its stages.  Blocks the host until the pass completes, then writes
 * the stage durations in milliseconds: ms[0] input preparation (split or
 * conversion; 0 for LEG_F64/LEG_F32), ms[1] Abel GEMM, ms[2] FFT stage.
 * ms: host array of 3 floats.
 */
LEG_API int leg_forward_profiled(leg_plan_t plan, const void *f, void *c, int B, cudaStream_t stream,
                                 float *ms);

/*
 * leg_backward -- df = L^T dc, the exact adjoint (transpose) of the linear
 * map of leg_forward for the same plan: the transposed twist + Fourier sum
 * followed by the transposed Abel operator.  The transposed transform follows
 * the plan's transform kernel: the transpose of the sine-form pipeline
 * (Eq. 2.13) on plans that use it, of the real-even one (Eq. 2.4, 2.5)
 * otherwise; both are the transpose of the same map.
 *   dc device, B x N (FP64 for LEG_F64, FP32 otherwise).
 *   df device, B x K (same type); overwritten.
 */
LEG_API int leg_backward(leg_plan_t plan, const void *dc, void *df, int B, cudaStream_t stream);

/*
 * leg_plain_forward -- the plain method: the Abel integral of a closed-form
 * function evaluated at the quadrature points themselves (no interpolation),
 * then the same FFT.  FP64 throughout; uses N, M, Q of the plan (any dtype).
 *   family  LEG_FAMILY_GENFN: f(x) = (1 - 2 x t + t^2)^(-1/2)  (Eq. 2.2),
 *                            params[b] = t, |t| < 1;
 *           LEG_FAMILY_EXP:   f(x) = exp(a x), params[b] = a;
 *           LEG_FAMILY_ABSPOW: f(x) = |x|^alpha, params[b] = alpha > 0.
 *   params  device, B doubles.   c  device, B x N doubles.
 */
#define LEG_FAMILY_GENFN 0
#define LEG_FAMILY_EXP   1
#define LEG_FAMILY_CHEB  2   /* leg_sample_cl, leg_plain_forward_cheb: sum_m coef_m T_m(x) */
#define LEG_FAMILY_ABSPOW 3  /* leg_plain_forward: f(x) = |x|^alpha, params[b] = alpha > 0
                                (Table 1's test function for alpha = 3/2, Eq. 2.15)       */
LEG_API int leg_plain_forward(leg_plan_t plan, int family, const double *params, int B,
                      double *c, cudaStream_t stream);

/*
 * leg_plain_forward_cheb -- the plain method for Chebyshev series
 * f(x) = sum_{m < Kc} coef[b, m] T_m(x) (the third ragged family): f is
 * evaluated at the quadrature points by Clenshaw's recurrence, then the
 * quadrature and the FFT as in leg_plain_forward.  FP64; N, M, Q of the plan.
 *   coef  device, B x Kc doubles, row-major; 1 <= Kc <= 16385.
 *   c     device, B x N doubles.
 * Invalid sizes or null pointers: LEG_ERR_INVALID_ARG.
 */
LEG_API int leg_plain_forward_cheb(leg_plan_t plan, const double *coef, int Kc, int B, double *c,
                                   cudaStream_t stream);

/*
 * Ragged batches (functions of different sizes, grouped in size buckets).
 *
 * leg_forward_ragged -- Theorem 1 (Eq. 2.4, Eq. 2.5) for every function of a
 * ragged batch in one call:
 *   plans[0..nplans-1]  bucket plans (LEG_SPLIT_FP16, current device, without
 *                       LEG_FLAG_COLLAPSED); 1 <= nplans <= 64;
 *   count               functions in the batch (0 is a no-op);
 *   plan_idx[i]         bucket of function i (0..nplans-1);
 *   n_out[i]            coefficients kept for function i, 1..N of its plan;
 *   in_off[i]           offset (in floats) of its K samples in f_packed;
 *   out_off[i]          offset (in floats) of its n_out[i] coefficients in
 *                       c_packed;
 *   f_packed, c_packed  device, FP32.
 * The four per-function arrays are device arrays (host pointers also work on
 * unified-addressing systems).  They are read back once per call, ordered
 * after the work already on `stream` (count x 24 bytes, one host
 * synchronisation with the stream); the batch built from them (workspaces,
 * the grouped-GEMM tile list, a CUDA graph) is kept in a cache of the four
 * most recently used batches, keyed by the device, the plans and the arrays'
 * contents, and replayed by later calls with the same key.  Destroying a plan
 * drops the cached batches that use it.  Calls from several host threads
 * share the cache: their launches are enqueued one at a time, and calls whose
 * work overlaps on the GPU through the same cached batch race on its
 * workspace.  Not while `stream` is being captured (LEG_ERR_UNSUPPORTED): the
 * handle-based form below has no host synchronisation and joins a caller's
 * capture.  Errors: as leg_ragged_create, and LEG_ERR_INVALID_ARG for null
 * arrays.
 */
LEG_API int leg_forward_ragged(const leg_plan_t *plans, int nplans, int count, const int *plan_idx,
                               const int *n_out, const long long *in_off, const long long *out_off,
                               const float *f_packed, float *c_packed, cudaStream_t stream);

/*
 * The same computation with an explicit batch handle.
 *
 * leg_ragged_create -- prepare the computation of `count` functions over the
 * bucket plans plans[0..nplans-1] (all LEG_SPLIT_FP16, current device).
 * Host arrays, copied (meanings as for leg_forward_ragged).  Allocates the
 * per-bucket workspaces, a private stream and three streams for the
 * concurrent transforms; synchronises.  The tile width of the grouped GEMM is
 * the one stored in the tuning cache (LEG_TUNE_CACHE) for this batch's
 * buckets by leg_ragged_autotune, else the library's cost model.  The plans
 * must outlive the batch.
 *
 * leg_ragged_forward -- one input-split launch over all functions, ONE
 * persistent tcgen05 launch over the Abel-GEMM tiles of all buckets, one
 * transform launch per bucket writing the packed output (the transforms of
 * the buckets run concurrently on the batch's internal streams; each uses its
 * plan's transform kernel, see leg_plan_set_transform, as set when the
 * batch's launches are captured on its second call: later changes to the
 * plans reach the batch through a new batch, or the new graph that
 * leg_ragged_set_tile causes).  The first call runs
 * the sequence directly; later calls replay it as a CUDA graph (captured
 * again when f_packed, c_packed or the tile width change).  When `stream` is
 * itself being captured, the launches join the caller's graph instead.
 * Ordered after prior work on `stream`, and later work on `stream` waits for
 * it.  Device pointers; no host synchronisation.
 *
 * leg_ragged_forward_profiled -- the same launches run directly with CUDA
 * events between the stages; blocks the host until they complete and writes
 * ms[0] input split, ms[1] grouped Abel GEMM, ms[2] transforms (all buckets,
 * concurrent).  ms: host array of 3 floats.
 *
 * leg_ragged_set_tile -- width of the grouped GEMM's tiles: a multiple of 16
 * in 16..128, or 0 for the cost model's choice; synchronises the batch's
 * stream.  Results do not depend on it.  leg_ragged_tile_info -- the current
 * width and the number of pair tiles of the grouped launch (either may be NULL).
 *
 * leg_ragged_autotune -- time the grouped GEMM at the model's tile width and
 * at 128, 112, ..., 64 on the caller's data (each candidate once untimed and
 * three times timed, leg_ragged_forward_profiled), keep the fastest, and,
 * with LEG_TUNE_CACHE naming a file, store it there keyed by the device and
 * every bucket's (N, M, K, Q, functions); a stored choice is taken without
 * timing.  c_packed is overwritten.  *tn (may be NULL): the chosen width.
 *
 * leg_ragged_status -- as leg_plan_status, for the batch's kernels.
 */
typedef struct leg_ragged *leg_ragged_t;
LEG_API int leg_ragged_create(leg_ragged_t *out, const leg_plan_t *plans, int nplans, int count,
                              const int *plan_idx, const int *n_out, const long long *in_off,
                              const long long *out_off);
LEG_API int leg_ragged_forward(leg_ragged_t batch, const float *f_packed, float *c_packed, cudaStream_t stream);
LEG_API int leg_ragged_forward_profiled(leg_ragged_t batch, const float *f_packed, float *c_packed,
                                        cudaStream_t stream, float *ms);
LEG_API int leg_ragged_set_tile(leg_ragged_t batch, int tn);
LEG_API int leg_ragged_tile_info(leg_ragged_t batch, int *tn, int *tiles);
LEG_API int leg_ragged_autotune(leg_ragged_t batch, const float *f_packed, float *c_packed, cudaStream_t stream,
                                int *tn);
LEG_API int leg_ragged_status(leg_ragged_t batch, int reset);
LEG_API int leg_ragged_destroy(leg_ragged_t batch);

/*
 * leg_sample_cl -- input generation (no counterpart in the method): samples of
 * closed-form functions at their Chebyshev-Lobatto nodes, evaluated in FP64 on
 * the device and stored in FP32.  For function i with K[i] nodes,
 *   f_packed[in_off[i] + k] = f_i(cos(pi k / (K[i]-1))),  k = 0..K[i]-1,
 * family[i] = LEG_FAMILY_GENFN (param[i] = t), LEG_FAMILY_EXP (param[i] = a),
 * or LEG_FAMILY_CHEB (sum_{m<K[i]} coef[coef_off[i] + m] T_m(x), by Clenshaw's
 * recurrence; coef/coef_off may be NULL if no function uses this family).
 * All arrays on the device.
 */
LEG_API int leg_sample_cl(int count, const int *family, const double *param, const int *K,
                          const long long *coef_off, const double *coef, const long long *in_off,
                          float *f_packed, cudaStream_t stream);

/*
 * leg_plan_status -- synchronise with the device and report whether any
 * bounded device-side wait of this plan's tensor-core kernels expired since
 * the last reset (LEG_ERR_TIMEOUT; the outputs of that call are invalid).
 * reset != 0 clears the status word.  Blocks the host.
 */
LEG_API int leg_plan_status(leg_plan_t plan, int reset);

/*
 * leg_plan_set_wait_limit -- cycle budget of each bounded wait (mbarrier
 * waits between the TMA, MMA and epilogue roles) in the tensor-core kernels;
 * default 2e9 (about one second), or the environment variable
 * LEG_WAIT_LIMIT_CYCLES at plan creation.  Teardown waits use a fixed budget.
 */
LEG_API int leg_plan_set_wait_limit(leg_plan_t plan, long long cycles);

/*
 * leg_plan_set_tile -- width of the output tile of the tensor-core Abel GEMM
 * (LEG_SPLIT_FP16 forward and adjoint, LEG_BF16): tn functions per CTA-pair
 * tile of 256 operator rows, a multiple of 16 in 16..128 (LEG_BF16: 16..256);
 * 0 (the default) lets the library pick tn per call from the batch size,
 * the rows and the number of resident CTA pairs (fewest MMA cycles on the
 * busiest pair).
 * A tuning knob only: results do not depend on it.
 */
LEG_API int leg_plan_set_tile(leg_plan_t plan, int tn);

/*
 * leg_plan_set_transform -- the kernel of the plan's forward transform stage:
 * variant LEG_TRANSFORM_REG (the default), LEG_TRANSFORM_STOCKHAM or
 * LEG_TRANSFORM_SINE (the sine form of Eq. 2.13, see LEG_FLAG_SINE_FORM;
 * M >= 256, else LEG_ERR_UNSUPPORTED), and the radix of the register-tiled
 * kernels' FFT passes: 8 or 16 complex values per thread (0 = the default, 8;
 * 16 takes effect for M >= 2048).  All choices compute the same linear map;
 * results differ by rounding.  The plain method (leg_plain_forward*) and
 * ragged batches use the plan's choice too; leg_backward always applies the
 * real-even adjoint (the transpose of that same map).
 * leg_plan_get_transform -- the current variant and radix (either may be NULL).
 */
LEG_API int leg_plan_set_transform(leg_plan_t plan, int variant, int radix);
LEG_API int leg_plan_get_transform(leg_plan_t plan, int *variant, int *radix);

/*
 * leg_plan_tile_info -- the tile of the forward GEMM for a batch of B
 * functions: *tn functions per pair tile, *pairs CTA pairs resident at once
 * on the current device, *tiles pair tiles of the launch.  LEG_SPLIT_FP16
 * plans only (LEG_ERR_UNSUPPORTED otherwise).  Any output may be NULL.
 */
LEG_API int leg_plan_tile_info(leg_plan_t plan, int B, int *tn, int *pairs, int *tiles);

/*
 * leg_plan_autotune -- choose, by timing on the caller's batch, the launch
 * parameters of the plan and store them in it: the tile width of the
 * tensor-core GEMM (LEG_SPLIT_FP16, LEG_BF16: the library's model choice and
 * the multiples of 16 from the plan's maximum down to 64; results do not
 * depend on it) and the forward transform (variant and radix, as
 * leg_plan_set_transform; the candidates compute the same map and differ by
 * rounding; plans created with LEG_FLAG_SINE_FORM keep the sine form and tune
 * its radix).  Not a step of the paper's method: a tuning aid.
 *   f  device, B x K input (as leg_forward);  c  device, B x N output buffer
 *      (overwritten).  Synchronises the stream; runs each candidate four times.
 *   *tn, *fft (either may be NULL): the chosen tile width (0 = the model's
 *      choice per call) and transform variant (LEG_TRANSFORM_*; its radix:
 *      leg_plan_get_transform).
 * With the environment variable LEG_TUNE_CACHE naming a file, choices are
 * appended there keyed by (device name, dtype, N, M, K, Q, flags, B) and
 * reused without timing by later calls with the same key.
 */
LEG_API int leg_plan_autotune(leg_plan_t plan, const void *f, void *c, int B, cudaStream_t stream, int *tn,
                              int *fft);

/*
 * leg_forward_noalloc -- leg_forward for a LEG_SPLIT_FP16 plan that allocates
 * no device memory.  (The paper has no counterpart: this is a library
 * convenience.)  It is meant for callers that must not allocate at call time,
 * such as a host framework that owns the whole device-memory budget through
 * its own fixed pool, or a latency-critical caller that cannot afford the
 * host blocking and device synchronisation that cudaMalloc/cudaFree may
 * cause.  The plan is created (and allocates) beforehand, as usual.
 *   f  device, B x K FP32;  c  device, B x N FP32 (as leg_forward).
 * The intermediate buffers (input slices, per-function scales, the Abel
 * GEMM result) come from one static device array of 64 MiB in the library,
 * which every GPU that loads the library keeps reserved until process exit.
 * A batch needing more scratch than that (about B*(14*Kp + 8*Mr) bytes, Kp = K
 * rounded up to 32, Mr = M/2+1 rounded up to 32) is rejected with
 * LEG_ERR_INVALID_ARG and a message stating the sizes.  The first call on each
 * device looks up the array's device address (cudaGetSymbolAddress) with that
 * device current, and so does the first call after the device's context
 * changed (cudaDeviceReset); make those calls before any stream capture.  All calls
 * share the array and it keeps the last call's contents: calls whose work
 * overlaps on the GPU race on it, so serialise them.
 */
LEG_API int leg_forward_noalloc(leg_plan_t plan, const float *f, float *c, int B, cudaStream_t stream);

/*
 * leg_forward_host -- leg_forward on HOST buffers: the batch is copied to the
 * device, transformed and copied back, with the copies overlapped with the
 * computation.  (A library convenience with no counterpart in the paper.)
 *   f_host  host, B x K (FP64 for LEG_F64, FP32 otherwise), row-major;
 *   c_host  host, B x N (same type); overwritten.
 * For LEG_SPLIT_FP16 and LEG_BF16 plans, page-locked host buffers that are
 * mapped into the device's address space (cudaHostAlloc, cudaHostRegister
 * with cudaHostRegisterMapped, pinned tensors on unified-addressing systems)
 * are read and written in place by the kernels: the input split reads each
 * row of f once over the host link and the last kernel writes each
 * coefficient once, with no staging copy.
 * Otherwise, for LEG_SPLIT_FP16 plans the input goes over in four pieces on
 * an internal stream and the split of each piece starts when it has landed;
 * the coefficients come back per piece while the next piece is transformed.
 * Results equal leg_forward's bit for bit.  Ordered after the work already on
 * `stream`; c_host is complete once `stream` has reached the end of the call
 * (synchronise `stream` before reading it); both host buffers must stay valid
 * until then.  Page-locked host memory (cudaHostAlloc, or a pinned tensor)
 * lets the copies run at full speed and overlap; pageable memory works but
 * the copies then run through a staging buffer.  The plan keeps device
 * copies of the largest batch it has seen (B x (K + N) values) and two
 * internal streams; growing them synchronises the device.  For a stream of
 * batches, leg_plan_set_host_overlap lets each call's input copy run during
 * the previous call's kernels.
 */
LEG_API int leg_forward_host(leg_plan_t plan, const void *f_host, void *c_host, int B, cudaStream_t stream);

/*
 * leg_plan_set_host_overlap -- how leg_forward_host orders its input copy for
 * a stream of batches.  (A library convenience with no counterpart in the
 * paper.)
 *   on = 0 (default): every step of leg_forward_host is ordered after the
 *      work already queued on `stream`.
 *   on = 1: for LEG_SPLIT_FP16 and LEG_BF16 plans with page-locked, mapped
 *      host buffers, leg_forward_host copies f_host with a copy engine into
 *      one of two device staging buffers of the plan (the calls alternate
 *      between them) on an internal stream, and that copy waits only for the
 *      previous call that used the same staging buffer to finish, not for the
 *      rest of the work on `stream`: the input of one call crosses the host
 *      link while the kernels of the call before it run.  f_host must
 *      therefore hold the batch when the call is made (written by the host,
 *      or by device work the caller has already synchronised).  The kernels
 *      read the staging buffer; c_host is written in place by the last kernel
 *      as with on = 0 and is complete once `stream` has reached the end of
 *      the call.  Calls made while `stream` is being captured, and other
 *      plans and buffers, run as with on = 0.
 * Results equal leg_forward's bit for bit either way.  The staging buffers
 * (2 x B x K FP32 values of the largest batch seen) are allocated by the
 * first call that needs them; growing them synchronises the device.
 * Errors: LEG_ERR_INVALID_ARG for a NULL plan or on outside {0, 1}.
 */
LEG_API int leg_plan_set_host_overlap(leg_plan_t plan, int on);

/*
 * leg_forward_host_batches -- leg_forward_host on nbatch batches of B
 * functions, one after another.  (A library convenience with no counterpart
 * in the paper.)
 *   f_host  host, nbatch x B x K (FP64 for LEG_F64, FP32 otherwise);
 *   c_host  host, nbatch x B x N (same type); overwritten.
 *   B, nbatch  >= 0; either 0 is a no-op.
 * For LEG_SPLIT_FP16 plans of the Abel GEMM + transform with page-locked,
 * mapped host buffers, the batches run through the pipeline of
 * leg_forward_batches, and each batch's input is copied by a copy engine into
 * one of the plan's two staging buffers (2 x B x K FP32 values, allocated by
 * the first call that needs them, which synchronises the device): the first
 * copy after the work already on `stream`, each later one while the kernels
 * of the batches before it run; each batch's transform writes its
 * coefficients into c_host in place.  Other plans and buffers, nbatch = 1 and
 * calls on a stream being captured run leg_forward_host on each batch in
 * turn.  Results equal leg_forward's bit for bit.  c_host is complete once
 * `stream` has reached the end of the call; both buffers must stay valid
 * until then.
 * Errors: those of leg_forward_host; LEG_ERR_INVALID_ARG for B < 0 or
 * nbatch < 0.
 */
LEG_API int leg_forward_host_batches(leg_plan_t plan, const void *f_host, void *c_host, int B, int nbatch,
                                     cudaStream_t stream);

/*
 * leg_memory_info -- device memory the library holds at this moment for the
 * objects it created (plans and their workspaces, ragged batches, the
 * host-buffer path's copies, cached one-call batches): the number of live
 * allocations and their total bytes, over all devices.  The static scratch of
 * leg_forward_noalloc is not counted.  Either output may be NULL.  A library
 * diagnostic with no counterpart in the paper; the error-path tests use it to
 * show that failed calls release what they took.
 */
LEG_API int leg_memory_info(long long *allocations, long long *bytes);

/* Message for the most recent failing call on this host thread ("" if none). */
LEG_API const char *leg_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* LEG_H */
