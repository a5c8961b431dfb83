// Internal declarations shared by the CUDA translation units of libleg.
// Target: sm_103a (GB300).  Method: De Micheli & Viano, arXiv:1106.0463.
#pragma once

#include <cuda.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>
#include <string>

#include "leg.h"

// ---------------------------------------------------------------------------
// Error plumbing: every host entry point returns an int status and records a
// message retrievable through leg_last_error().
// ---------------------------------------------------------------------------
int leg_set_error(int code, const std::string &msg);

#define LEG_CUDA_TRY(expr)                                                        \
    do {                                                                          \
        cudaError_t _e = (expr);                                                  \
        if (_e != cudaSuccess)                                                    \
            return leg_set_error(_e == cudaErrorMemoryAllocation ? LEG_ERR_OOM    \
                                                                 : LEG_ERR_CUDA,  \
                                 std::string(#expr) + ": " + cudaGetErrorString(_e)); \
    } while (0)

#define LEG_LAUNCH_CHECK(what)                                                    \
    do {                                                                          \
        cudaError_t _e = cudaGetLastError();                                      \
        if (_e != cudaSuccess)                                                    \
            return leg_set_error(LEG_ERR_CUDA, std::string(what) + ": " +         \
                                                   cudaGetErrorString(_e));       \
    } while (0)

// ---------------------------------------------------------------------------
// Sizes.
// ---------------------------------------------------------------------------
static inline int leg_round_up(int x, int m) { return (x + m - 1) / m * m; }

// Programmatic dependent launch.  A kernel launched with
// cudaLaunchAttributeProgrammaticStreamSerialization may start before the
// previous kernel on its stream has finished; leg_griddep_wait() returns once
// that kernel has completed and its memory is visible, so every thread calls
// it before touching the previous kernel's output.  leg_griddep_trigger()
// lets the next such kernel start early.  Both are no-ops for kernels launched
// without the attribute.
__device__ __forceinline__ void leg_griddep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void leg_griddep_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

constexpr int LEG_KPAD = 32;      // K is padded to a multiple of this (one 32-wide K block of the tensor-core GEMMs)
constexpr int LEG_MAX_M = 32768;
constexpr int LEG_MAX_K = 16385;

// Split-FP16 scheme (fixed-point leading slice): granularity exponents of the
// leading slices of the operator (A0 on a 2^-abits grid) and of the input (F0
// on a 2^-s grid, s = fbits).  Their sum is LEG_SPLIT_GRID = 23, so products
// A0*F0 lie on a 2^-23 grid and every partial sum (below 2 in magnitude for
// L1-normalised operator rows) is exact in FP32.  The residual slices carry
// weights 2^-s and 2^-2s.  The split is chosen per plan by K: operator
// entries are ~1/K, so long rows need a fine A0 grid (abits 16: with (15, 8)
// the K = 8193 workload measured 1.0e-6 against 2.8e-7, with (14, 9) 1.3e-6),
// while for K <= 1025 a finer F0 grid wins (8 bits: a peaked input such as
// (1 - 2xt + t^2)^-1/2, t = 0.95, keeps more of itself in F0, and the error
// of the N = 8192 ragged bucket fell from 7.5e-7 to 4.1e-7).
constexpr int LEG_SPLIT_GRID = 23;
__host__ __device__ inline int leg_split_fbits(int K) { return K <= 1025 ? 8 : 7; }
// Planes of the split-FP16 GEMM: the operator side keeps its three slices
// A0, A1, A2s; the input side carries F0, F1, the residual r - F1 at weight
// 2^-s, and the pre-scaled copies 2^-s F1, 2^-s F0, 2^-2s F1, 2^-s (r - F1),
// so that every product after A0 F0 lands in an accumulator of weight 2^-s
// (leg_gemm_tc.cu).
constexpr int LEG_SPLIT_NA = 3;
constexpr int LEG_SPLIT_NF = 7;

// ---------------------------------------------------------------------------
// Plan.
// ---------------------------------------------------------------------------
struct LegHostState;                  // leg_forward_host's device copies, streams, events (leg_host.cu)
struct LegPipeState;                  // leg_forward_batches' streams and events (leg_api.cu)
constexpr int LEG_HOST_CHUNKS = 4;     // pieces of a leg_forward_host batch (split-FP16 plans)

struct leg_plan {
    int N, M, K, Q, dtype;
    int fbits;  // split-FP16 slice width s (leg_split_fbits(K)); the operator's is LEG_SPLIT_GRID - s
    unsigned flags;
    int L;      // M/2: length of the complex FFT (real transform of length M)
    int rows;   // M/2 + 1 distinct rows of the Abel operator (Eq. 2.12)
    int Kp;     // K padded to LEG_KPAD
    int device;

    // tau rule of the Abel integral: 1 - tau_q^2 and w_q (Q each, FP64)
    double *omt2 = nullptr;
    double *wq = nullptr;
    // operator, FP64, rows x K (ld = K); kept for every dtype (adjoint, checks)
    double *A64 = nullptr;
    // LEG_FLAG_COLLAPSED: L = R A, FP64, N x K (ld = K); the per-dtype planes
    // below (A32, Ah, Abf, AhT) then hold L instead of A
    double *L64 = nullptr;
    int grows = 0;   // rows of the operator the planes hold: rows (Abel) or N (collapsed)
    // FP32 copy (LEG_F32), rows x K
    float *A32 = nullptr;
    // tensor-core planes, rows x Kp, K-major
    __half *Ah[3] = {nullptr, nullptr, nullptr};   // LEG_SPLIT_FP16: A0, A1, A2s, one allocation
                                                  // (Ah[s] = Ah[0] + s rows Kp)
    __nv_bfloat16 *Abf = nullptr;                 // LEG_BF16
    int *rowexp = nullptr;                        // per-row power-of-two scale (split)
    double a00 = 0.0;         // A[0,0] = sum_q w_q: row 0 (y = 0, x = 1) is a00 times f at x = 1
    int tn = 0;               // functions per tensor-core pair tile (0: chosen per launch)
    int fft_variant = 0;      // LEG_TRANSFORM_*: the forward transform kernel (same map, rounding differs)
    int fft_log2e = 3;        // register-tiled forward transforms: 2^fft_log2e values per thread (radix 8 or 16)
    bool collapsed() const { return (flags & LEG_FLAG_COLLAPSED) != 0; }
    // transposed split planes for the adjoint GEMM: K x Kpr (Kpr = rows padded),
    // each column k of the operator scaled by its own power of two
    __half *AhT[3] = {nullptr, nullptr, nullptr};   // one allocation (AhT[s] = AhT[0] + s K Kpr)
    int *colexp = nullptr;

    // twiddles e^{2 pi i n / M}, n = 0..M-1 (computed in FP64 on the device),
    // followed by the compact copy e^{2 pi i q / (M/4)}, q < M/4 (entries M..)
    double2 *tw64 = nullptr;
    float2 *tw32 = nullptr;
    float4 *twdf = nullptr;   // (re.hi, re.lo, im.hi, im.lo)

    // device status word (bit 0: a bounded wait in a tensor-core kernel expired)
    int *status = nullptr;
    long long wait_limit = 2000000000LL;   // cycles per bounded wait

    // workspace for batches of up to ws_B functions
    int ws_B = 0;
    int ldg = 0;              // row stride (elements) of G
    void *G = nullptr;        // B x ldg, type by dtype (double / float / float2)
    __half *Fh = nullptr;     // LEG_SPLIT_NF split input planes, each ws_B x ldf
    int ldf = 0;              // row stride of the split input planes
    __nv_bfloat16 *Fbf = nullptr;                 // bf16 input plane B x Kp
    int *fexp = nullptr;                          // per-function power-of-two scale
    void *Gbar = nullptr;     // backward: B x ldg (FP64 for LEG_F64, FP32 otherwise)
    LegHostState *host = nullptr;   // created by the first leg_forward_host
    LegPipeState *pipe = nullptr;   // created by the first pipelined leg_forward_batches

    // leg_forward replays a CUDA graph of its launches when called again with
    // the same buffers and launch parameters (the key); captured on `cap`.
    // Two keys are kept (the least recently used one is replaced), so calls
    // alternating between two buffers (leg_forward_host's staging buffers)
    // replay too.
    struct GraphKey {
        const void *f = nullptr;
        void *c = nullptr;
        int B = 0, wsB = 0;   // wsB: the workspace's capacity (plane strides depend on it)
        void *G = nullptr, *Fh = nullptr;
        int tn = 0, fft = 0, fft_log2e = 0;
        long long wait = 0;
        bool operator==(const GraphKey &o) const
        {
            return f == o.f && c == o.c && B == o.B && wsB == o.wsB && G == o.G && Fh == o.Fh && tn == o.tn &&
                   fft == o.fft && fft_log2e == o.fft_log2e && wait == o.wait;
        }
    };
    struct GraphEntry {
        GraphKey key;
        bool seen = false;                 // the key's launches ran once directly
        cudaGraphExec_t exec = nullptr;
        unsigned long long used = 0;       // last use (0: never)
    };
    GraphEntry fwd[2];
    unsigned long long fwd_clock = 0;
    int host_overlap = 0;                  // leg_plan_set_host_overlap
    cudaStream_t cap = nullptr;
};

void leg_host_free(leg_plan *p);

// Sources and sinks of the split-FP16 batch pipeline (leg_api.cu): batch b
// reads f + b fstride (device-readable, or host memory copied into
// stage[b % 2] on `copy` when stage[0] is set) and writes c + b cstride.
struct LegPipeIO {
    const void *f = nullptr;
    void *c = nullptr;
    size_t fstride = 0, cstride = 0;   // bytes per batch
    void *stage[2] = {};
    cudaStream_t copy = nullptr;
    cudaEvent_t stage_ready[2] = {}, stage_free[2] = {};
    // stage timing (or nullptr): five events per batch, recorded before and
    // after its split and after its GEMM (GEMM stream), and before and after
    // its transform (transform stream)
    cudaEvent_t *prof = nullptr;
};
int leg_pipeline_split(leg_plan *p, int B, int nbatch, const LegPipeIO &io, cudaStream_t st);
bool leg_pipeline_applies(const leg_plan *p);
// drops the one-call ragged batches built over plan p (leg_ragged.cu)
void leg_ragged_forget_plan(const leg_plan *p);

// ---------------------------------------------------------------------------
// Device allocations of the library go through leg_dev_malloc (and
// leg_dev_free).  With the
// environment variable LEG_FAULT_ALLOC = k (k >= 1), the k-th call after the
// variable took its current value fails with cudaErrorMemoryAllocation
// without allocating anything: a host-side fault injection for the tests of
// the LEG_ERR_OOM paths (no kernel ever sees a bad pointer).
// ---------------------------------------------------------------------------
cudaError_t leg_dev_malloc_bytes(void **ptr, size_t bytes);
cudaError_t leg_dev_malloc_async_bytes(void **ptr, size_t bytes, cudaStream_t st);
template <class T>
inline cudaError_t leg_dev_malloc(T **ptr, size_t bytes)
{
    return leg_dev_malloc_bytes(reinterpret_cast<void **>(ptr), bytes);
}
// The matching releases (NULL accepted).  Together they keep the count and
// bytes of the library's live device allocations (leg_memory_info).
cudaError_t leg_dev_free(void *ptr);
cudaError_t leg_dev_free_async(void *ptr, cudaStream_t st);

// Tuning cache file (LEG_TUNE_CACHE): one "key a b" line per choice, the
// last matching line wins (leg_tune.cu).  b may be NULL on lookup.
std::mutex &leg_tune_mutex();
bool leg_tune_cache_lookup(const char *path, const std::string &key, int *a, int *b);
void leg_tune_cache_store(const char *path, const std::string &key, int a, int b);

// Split input planes of a batch: LEG_SPLIT_NF FP16 planes of B rows with row
// stride ld; plane s starts at base + s * pstride.
struct LegSplitIn {
    __half *base;
    size_t pstride;   // elements between consecutive planes
    int ld;           // row stride (elements), a multiple of LEG_KPAD
    int *fexp;        // per-row power-of-two scales
    int fbits;        // slice width s of the split (the plan's)
};

// One GEMM problem of the tcgen05 kernel (leg_gemm_tc.cu):
//   out[b * ldo + j] = 2^(aexp[j] + fexp[b]) sum_k A[j, k] F[b, k],  j < rows, b < B,
// operator rows on the MMA's M side (256 per CTA pair), functions on its N
// side (tn per pair tile), both given as FP16/BF16 planes through TMA maps.
struct TcProblem {
    CUtensorMap a;           // operator planes (planes x rows x Kp), one 3-D map
    CUtensorMap f;           // input planes    (planes x B x Kp), one 3-D map
    const int *aexp;         // per-row power-of-two scales of A (or null)
    const int *fexp;         // per-function scales of F (or null)
    void *out;               // float2 (double-float) or float, row stride ldo
    int ldo, rows, B;
    int nkb;                 // Kp / 32
    int tn;                  // functions per pair tile (multiple of 16, <= 256)
    int ntm, ntn;            // tiles along rows (256 each) and along functions (tn each)
    int tile0;               // first global tile index of this problem (grouped launches)
    int fn_fast;             // 1: function tiles vary fastest in the tile order (operator-heavy problems)
    float w1;                // 2^-s: weight of acc1 and acc2 (split path)
};

// Device descriptor of one bucket of a ragged batch (input-split targets).
struct LegRaggedBucket {
    LegSplitIn in;       // B_b x Kp split planes
    float2 *G;           // B_b x ldg double-float G (row 0 written by the split)
    int ldg;
    float2 a00;          // the plan's a00 as a double-float pair (hi, lo)
    int K, Kp;
};

// ---------------------------------------------------------------------------
// Launchers (each returns a LEG_* status).
// ---------------------------------------------------------------------------
// operator build (leg_operator.cu)
int leg_build_operator(leg_plan *p);   // FP64 operator, then leg_build_planes
int leg_build_planes(leg_plan *p);
int leg_build_collapsed(leg_plan *p);   // L = R A for LEG_FLAG_COLLAPSED
int leg_build_twiddles(leg_plan *p);

// SIMT GEMMs (leg_gemm_simt.cu)
//   forward: G[b, j] = sum_k F[b, k] A[j, k]     (F: B x K ld ldf, A: rows x K ld lda)
//   adjoint: D[b, k] = sum_j Gb[b, j] A[j, k]    (Gb: B x rows ld ldg, D: B x K)
int leg_gemm_f64_fwd(const double *F, int ldf, const double *A, int lda, double *G, int ldg,
                     int B, int rows, int K, cudaStream_t st);
int leg_gemm_f32_fwd(const float *F, int ldf, const float *A, int lda, float *G, int ldg,
                     int B, int rows, int K, cudaStream_t st);
int leg_gemm_f64_adj(const double *Gb, int ldg, const double *A, int lda, double *D, int ldd,
                     int B, int rows, int K, cudaStream_t st);
int leg_gemm_f32_adj(const float *Gb, int ldg, const float *A, int lda, float *D, int ldd,
                     int B, int rows, int K, cudaStream_t st);

// FFT stage (leg_fft.cu)
//   forward: c[b, n] = (2n+1) (Ghat_n - Ghat_{n+1}),  Ghat_n = (1/M) sum_{j<M} g_j cos(2 pi n j/M)
//   adjoint: gbar[b, j] = (w_j / M) sum_{n<=N} d_n cos(2 pi n j / M), d_n = (2n+1)v_n - (2n-1)v_{n-1}
// gkind: 0 = double G, 1 = float G, 2 = double-float G (float2)
int leg_fft_forward(const leg_plan *p, const void *G, int ldg, void *c, int B, cudaStream_t st);
int leg_fft_adjoint(const leg_plan *p, const void *v, void *gbar, int ldg, int B, cudaStream_t st);
// split-FP16 plans on the sine-form transform: the adjoint transform writes the
// transposed GEMM's input planes directly (no gbar, no separate split)
bool leg_fft_adjoint_writes_planes(const leg_plan *p);
int leg_fft_adjoint_planes(const leg_plan *p, const void *v, int B, cudaStream_t st);
int leg_fft_forward_f64(const leg_plan *p, const double *G, int ldg, double *c, int B, cudaStream_t st);

// Forward transform kernels of a plan (leg_plan::fft_variant).  All compute the
// same linear map; their rounding differs.
//   LEG_TRANSFORM_REG       register-tiled real-even transform (M >= 256; the
//                           shared-memory one below that), FP32 plans: Stockham
//   LEG_TRANSFORM_STOCKHAM  shared-memory Stockham transforms (leg_fft.cu)
//   LEG_TRANSFORM_SINE      register-tiled half-range sine form, Eq. 2.13
//                           (leg_dst16.cu; M >= 256)
// The adjoint of every variant is the real-even adjoint (register-tiled unless
// LEG_TRANSFORM_STOCKHAM is chosen).
// (LEG_TRANSFORM_REG, LEG_TRANSFORM_STOCKHAM, LEG_TRANSFORM_SINE: leg.h)
constexpr int LEG_TRANSFORM_MIN_M_REG = 256;   // smallest M of the register-tiled kernels (H = 64)

// register-tiled transforms (leg_dct16.cu), H = 2^log2h with 6 <= log2h <= 13;
// dtype LEG_F64 (FP64 G, c) or LEG_SPLIT_FP16 (double-float G, FP32 c)
// log2e: at most 2^log2e values per thread (3 or 4: radix-8 or radix-16 passes)
int leg_dct16_forward(int dtype, int log2h, int log2e, const void *G, int ldg, void *c, int N, int B,
                      const void *tw, cudaStream_t st, const int *rowfn, const long long *out_off, const int *n_out);
int leg_dct16_adjoint(int dtype, int log2h, const void *v, void *gbar, int ldg, int N, int B, const void *tw,
                      cudaStream_t st);
// register-tiled sine form (leg_dst16.cu), same H range; dtype LEG_F64,
// LEG_SPLIT_FP16 (double-float G, FP32 c) or LEG_F32 / LEG_BF16 (FP32)
int leg_dst16_forward(int dtype, int log2h, int log2e, const void *G, int ldg, void *c, int N, int B,
                      const void *tw, cudaStream_t st, const int *rowfn, const long long *out_off, const int *n_out);
int leg_dst16_adjoint(int dtype, int log2h, const void *v, void *gbar, int ldg, int N, int B, const void *tw,
                      cudaStream_t st);
int leg_dst16_adjoint_planes(int log2h, const float *v, const LegSplitIn &sp, int npr, int N, int B,
                             const void *twdf, cudaStream_t st);

// plain method (leg_plain.cu): g_j from a closed form at the quadrature points
int leg_plain_g(const leg_plan *p, int family, const double *params, int B, double *G, int ldg,
                cudaStream_t st);
int leg_plain_g_cheb(const leg_plan *p, const double *coef, int Kc, int B, double *G, int ldg, cudaStream_t st);

// split-FP16 tensor-core path (leg_gemm_tc.cu)
LegSplitIn leg_split_workspace(const leg_plan *p);
int leg_split_prepare_input(const leg_plan *p, const float *f, int B, cudaStream_t st);
int leg_gemm_split_fwd(leg_plan *p, int B, cudaStream_t st);
int leg_gemm_bf16_fwd(leg_plan *p, int B, void *out, int ldo, cudaStream_t st);   // rows p->grows
int leg_bf16_prepare_input(const leg_plan *p, const float *f, int B, cudaStream_t st);
int leg_gemm_split_adj(leg_plan *p, void *df, int B, cudaStream_t st);
// the transposed GEMM from planes already in the plan's split workspace
int leg_gemm_split_adj_planes(leg_plan *p, void *df, int B, cudaStream_t st);
int leg_build_split_transposed(leg_plan *p);
// collapsed plans (LEG_FLAG_COLLAPSED): c = L f and df = L^T dc, FP32
int leg_gemm_split_collapsed_fwd(leg_plan *p, int B, float *c, cudaStream_t st);
int leg_gemm_split_collapsed_adj(leg_plan *p, const float *dc, void *df, int B, cudaStream_t st);
// operator rows of the forward split GEMM: M/2 (row 0 goes through the split) or N (collapsed)
int leg_split_fwd_rows(const leg_plan *p);
// K-depth of the adjoint split GEMM: the operator's rows padded to LEG_KPAD
inline int leg_adj_depth(const leg_plan *p) { return leg_round_up(leg_round_up(p->grows, 8), LEG_KPAD); }
int leg_make_split_problem(TcProblem *pr, const leg_plan *p, const LegSplitIn &in, int B, float2 *G, int ldg,
                           int tn);
int leg_split_problem_tiles(const TcProblem &pr);
int leg_gemm_split_grouped(const TcProblem *d_probs, int nprob, int ntiles, int tn, int *status, long long limit,
                           cudaStream_t st);
int leg_split_ragged(const float *f_packed, const long long *in_off, const int *bucket, const int *row,
                     const LegRaggedBucket *bk, int count, int max_k, cudaStream_t st);   // max_k: longest row
int leg_fft_forward_ragged(const leg_plan *p, const void *G, int ldg, float *c_packed, int B, const int *rowfn,
                           const long long *out_off, const int *n_out, cudaStream_t st);
int leg_split_prepare_input_into(const leg_plan *p, const float *f, int B, const LegSplitIn &in, float2 *G,
                                 int ldg, cudaStream_t st);
int leg_gemm_split_fwd_into(leg_plan *p, int B, const LegSplitIn &in, float2 *G, int ldg, cudaStream_t st);
// functions per pair tile for a forward of B functions (plan override, else the wave-count rule)
int leg_split_choose_tn(const leg_plan *p, int B);
// resident CTA pairs of the tensor-core GEMM on the current device; estimated
// cycles of the busiest pair for ntm row tiles x B functions of K-depth nkb
int leg_split_max_pairs(int *pairs);
long long leg_split_tile_cost(int tn, int ntm, int B, int nkb, int pairs);
