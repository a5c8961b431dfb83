// Internal declarations shared by the CUDA translation units of libleg.
// Target: sm_103a (GB300).  Method: De Micheli & Viano, arXiv:1106.0463.
#pragma once

#include <cuda.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

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

constexpr int LEG_KPAD = 64;      // K is padded to a multiple of this for tensor-core planes
constexpr int LEG_MAX_M = 32768;
constexpr int LEG_MAX_K = 16385;

// Split-FP16 scheme (fixed-point leading slice): granularity exponents of the
// leading slices of the operator (A0 on a 2^-16 grid) and of the input
// (F0 on a 2^-7 grid); products A0*F0 lie on a 2^-23 grid and every partial
// sum stays below 2 in magnitude, so their FP32 accumulation is exact.  The
// residual slices carry weights 2^-7 and 2^-14 (LEG_SPLIT_FBITS per level).
constexpr int LEG_SPLIT_ABITS = 16;
constexpr int LEG_SPLIT_FBITS = 7;

// ---------------------------------------------------------------------------
// Plan.
// ---------------------------------------------------------------------------
struct leg_plan {
    int N, M, K, Q, dtype;
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
    // FP32 copy (LEG_F32), rows x K
    float *A32 = nullptr;
    // tensor-core planes, rows x Kp, K-major
    __half *Ah[3] = {nullptr, nullptr, nullptr};   // LEG_SPLIT_FP16: A0, A1, A2s
    __nv_bfloat16 *Abf = nullptr;                 // LEG_BF16
    int *rowexp = nullptr;                        // per-row power-of-two scale (split)
    // transposed split planes for the adjoint GEMM: K x Kpr (Kpr = rows padded),
    // each column k of the operator scaled by its own power of two
    __half *AhT[3] = {nullptr, nullptr, nullptr};
    int *colexp = nullptr;

    // twiddles e^{2 pi i n / M}, n = 0..M-1 (computed in FP64 on the device)
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
    __half *Fh[3] = {nullptr, nullptr, nullptr};  // split input planes B x Kp
    __nv_bfloat16 *Fbf = nullptr;                 // bf16 input plane B x Kp
    int *fexp = nullptr;                          // per-function power-of-two scale
    void *Gbar = nullptr;     // backward: B x ldg (FP64 for LEG_F64, FP32 otherwise)
};

// ---------------------------------------------------------------------------
// Launchers (each returns a LEG_* status).
// ---------------------------------------------------------------------------
// operator build (leg_operator.cu)
int leg_build_operator(leg_plan *p);   // FP64 operator, then leg_build_planes
int leg_build_planes(leg_plan *p);
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
int leg_fft_forward_f64(const leg_plan *p, const double *G, int ldg, double *c, int B, cudaStream_t st);

// plain method (leg_plain.cu): g_j from a closed form at the quadrature points
int leg_plain_g(const leg_plan *p, int family, const double *params, int B, double *G, int ldg,
                cudaStream_t st);

// split-FP16 tensor-core path (leg_gemm_tc.cu)
int leg_split_prepare_input(const leg_plan *p, const float *f, int B, cudaStream_t st);
int leg_gemm_split_fwd(leg_plan *p, int B, cudaStream_t st);
int leg_gemm_bf16_fwd(leg_plan *p, int B, cudaStream_t st);
int leg_bf16_prepare_input(const leg_plan *p, const float *f, int B, cudaStream_t st);
int leg_gemm_split_adj(leg_plan *p, void *df, int B, cudaStream_t st);
int leg_build_split_transposed(leg_plan *p);
int leg_split_prepare_input_into(const leg_plan *p, const float *f, int B, __half *const planes[3], int *fexp,
                                 cudaStream_t st);
int leg_gemm_split_fwd_into(leg_plan *p, int B, __half *const planes[3], const int *fexp, float2 *G, int ldg,
                            cudaStream_t st);
