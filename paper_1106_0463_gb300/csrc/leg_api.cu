// C ABI of libleg: plans, argument validation, workspace, dispatch.
// The operations and their citations are documented in include/leg.h.
#include <stdlib.h>

#include <mutex>
#include <new>
#include <string>
#include <unordered_map>
#include <vector>

#include "leg_internal.cuh"

namespace {
thread_local std::string g_last_error;

bool is_pow2(int x) { return x > 0 && (x & (x - 1)) == 0; }

void free_workspace(leg_plan *p)
{
    leg_dev_free(p->G);
    leg_dev_free(p->Gbar);
    leg_dev_free(p->Fh);
    p->Fh = nullptr;
    leg_dev_free(p->Fbf);
    leg_dev_free(p->fexp);
    p->G = p->Gbar = nullptr;
    p->Fbf = nullptr;
    p->fexp = nullptr;
    p->ws_B = 0;
}

}  // namespace

// leg_forward_batches: a high-priority stream for the input splits and GEMMs,
// a low-priority one for the transforms, and the events between them.
struct LegPipeState {
    cudaStream_t hi = nullptr, lo = nullptr;
    cudaEvent_t start = nullptr, gemm_done = nullptr, done = nullptr;
    cudaEvent_t split[2] = {}, tf[2] = {};
};

namespace {

void pipe_free(leg_plan *p)
{
    LegPipeState *q = p->pipe;
    if (!q) return;
    for (cudaEvent_t e : {q->start, q->gemm_done, q->done, q->split[0], q->split[1], q->tf[0], q->tf[1]})
        if (e) cudaEventDestroy(e);
    if (q->hi) cudaStreamDestroy(q->hi);
    if (q->lo) cudaStreamDestroy(q->lo);
    delete q;
    p->pipe = nullptr;
}

void free_plan(leg_plan *p)
{
    if (!p) return;
    leg_ragged_forget_plan(p);
    pipe_free(p);
    for (auto &e : p->fwd)
        if (e.exec) cudaGraphExecDestroy(e.exec);
    if (p->cap) cudaStreamDestroy(p->cap);
    leg_host_free(p);
    free_workspace(p);
    leg_dev_free(p->omt2);
    leg_dev_free(p->wq);
    leg_dev_free(p->A64);
    leg_dev_free(p->L64);
    leg_dev_free(p->A32);
    leg_dev_free(p->Ah[0]);    // the three planes share one allocation
    leg_dev_free(p->AhT[0]);
    leg_dev_free(p->Abf);
    leg_dev_free(p->rowexp);
    leg_dev_free(p->colexp);
    leg_dev_free(p->status);
    leg_dev_free(p->tw64);
    leg_dev_free(p->tw32);
    leg_dev_free(p->twdf);
    delete p;
}

size_t g_elem_bytes(int dtype)
{
    switch (dtype) {
    case LEG_F64: return sizeof(double);
    case LEG_SPLIT_FP16: return sizeof(float2);
    default: return sizeof(float);
    }
}

int alloc_workspace(leg_plan *p, int B);

// Grow the workspace to B functions; on failure nothing of it stays allocated.
int ensure_workspace(leg_plan *p, int B)
{
    if (B <= p->ws_B) return LEG_OK;
    free_workspace(p);
    const int rc = alloc_workspace(p, B);
    if (rc) free_workspace(p);
    return rc;
}

int alloc_workspace(leg_plan *p, int B)
{
    const size_t eb = g_elem_bytes(p->dtype);
    const size_t Bz = (size_t)B;
    const int rowsKp = leg_round_up(p->rows, 8);
    const int bwdKp = (p->dtype == LEG_SPLIT_FP16) ? leg_adj_depth(p) : 0;
    if (p->collapsed()) {
        p->ldg = 0;   // one GEMM straight into c / df: no G
    } else {
        p->ldg = (p->dtype == LEG_SPLIT_FP16) ? bwdKp : rowsKp;
        LEG_CUDA_TRY(leg_dev_malloc(&p->G, eb * Bz * p->ldg));
        LEG_CUDA_TRY(leg_dev_malloc(&p->Gbar, eb * Bz * p->ldg));
    }
    if (p->dtype == LEG_SPLIT_FP16) {
        // input planes serve both directions: B x Kp (forward) or B x bwdKp (adjoint)
        p->ldf = (p->Kp > bwdKp) ? p->Kp : bwdKp;
        LEG_CUDA_TRY(leg_dev_malloc(&p->Fh, sizeof(__half) * LEG_SPLIT_NF * Bz * p->ldf));
        LEG_CUDA_TRY(leg_dev_malloc(&p->fexp, sizeof(int) * Bz));
    } else if (p->dtype == LEG_BF16) {
        LEG_CUDA_TRY(leg_dev_malloc(&p->Fbf, sizeof(__nv_bfloat16) * Bz * p->Kp));
    }
    p->ws_B = B;
    return LEG_OK;
}

int check_plan(leg_plan *p)
{
    if (!p) return leg_set_error(LEG_ERR_INVALID_ARG, "plan is NULL");
    int dev = -1;
    LEG_CUDA_TRY(cudaGetDevice(&dev));
    if (dev != p->device)
        return leg_set_error(LEG_ERR_INVALID_ARG, "current device differs from the plan's device");
    return LEG_OK;
}
}  // namespace

namespace {
std::mutex g_alloc_mutex;
std::unordered_map<void *, size_t> g_live;   // live device allocations of the library and their sizes
long long g_live_bytes = 0;
std::string g_fault_setting;   // value of LEG_FAULT_ALLOC the count below refers to
long long g_fault_count = 0;   // allocations since LEG_FAULT_ALLOC took that value

// true when this allocation is the one LEG_FAULT_ALLOC asks to fail
bool fault_injected()
{
    const char *env = getenv("LEG_FAULT_ALLOC");
    std::lock_guard<std::mutex> lock(g_alloc_mutex);
    const std::string v = env ? env : "";
    if (v != g_fault_setting) {
        g_fault_setting = v;
        g_fault_count = 0;
    }
    const long long k = env ? atoll(env) : 0;
    if (k < 1) return false;
    return ++g_fault_count == k;
}
}  // namespace

namespace {
void track(void *ptr, size_t bytes)
{
    std::lock_guard<std::mutex> lock(g_alloc_mutex);
    g_live[ptr] = bytes;
    g_live_bytes += (long long)bytes;
}

void untrack(void *ptr)
{
    std::lock_guard<std::mutex> lock(g_alloc_mutex);
    auto it = g_live.find(ptr);
    if (it == g_live.end()) return;
    g_live_bytes -= (long long)it->second;
    g_live.erase(it);
}
}  // namespace

cudaError_t leg_dev_malloc_bytes(void **ptr, size_t bytes)
{
    if (fault_injected()) {
        *ptr = nullptr;
        return cudaErrorMemoryAllocation;
    }
    const cudaError_t e = cudaMalloc(ptr, bytes);
    if (e == cudaSuccess) track(*ptr, bytes);
    return e;
}

cudaError_t leg_dev_malloc_async_bytes(void **ptr, size_t bytes, cudaStream_t st)
{
    if (fault_injected()) {
        *ptr = nullptr;
        return cudaErrorMemoryAllocation;
    }
    const cudaError_t e = cudaMallocAsync(ptr, bytes, st);
    if (e == cudaSuccess) track(*ptr, bytes);
    return e;
}

cudaError_t leg_dev_free(void *ptr)
{
    if (!ptr) return cudaSuccess;
    untrack(ptr);
    return cudaFree(ptr);
}

cudaError_t leg_dev_free_async(void *ptr, cudaStream_t st)
{
    if (!ptr) return cudaSuccess;
    untrack(ptr);
    return cudaFreeAsync(ptr, st);
}

extern "C" int leg_memory_info(long long *allocations, long long *bytes)
{
    std::lock_guard<std::mutex> lock(g_alloc_mutex);
    if (allocations) *allocations = (long long)g_live.size();
    if (bytes) *bytes = g_live_bytes;
    return LEG_OK;
}

int leg_set_error(int code, const std::string &msg)
{
    g_last_error = msg;
    return code;
}

extern "C" const char *leg_last_error(void) { return g_last_error.c_str(); }

extern "C" int leg_plan_create_ex(leg_plan_t *out, int N, int M, int K, int Q, int dtype, unsigned flags)
{
    if (!out) return leg_set_error(LEG_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!is_pow2(M) || M < 8 || M > LEG_MAX_M)
        return leg_set_error(LEG_ERR_INVALID_ARG, "M must be a power of two in [8, 32768]");
    if (N < 1 || N > M / 2)
        return leg_set_error(LEG_ERR_INVALID_ARG, "N must satisfy 1 <= N <= M/2");
    if (K < 2 || K > LEG_MAX_K)
        return leg_set_error(LEG_ERR_INVALID_ARG, "K must be in [2, 16385]");
    if (Q < 0 || Q > 16384)
        return leg_set_error(LEG_ERR_INVALID_ARG, "Q must be in [0, 16384]");
    if (dtype < LEG_F64 || dtype > LEG_SPLIT_FP16)
        return leg_set_error(LEG_ERR_INVALID_ARG, "unknown dtype");
    if (flags & ~(LEG_FLAG_TAU_LITERAL | LEG_FLAG_COLLAPSED | LEG_FLAG_SINE_FORM))
        return leg_set_error(LEG_ERR_INVALID_ARG, "unknown flag");
    if ((flags & LEG_FLAG_SINE_FORM) && (flags & LEG_FLAG_COLLAPSED))
        return leg_set_error(LEG_ERR_INVALID_ARG, "LEG_FLAG_SINE_FORM selects a transform; collapsed plans have none");
    if ((flags & LEG_FLAG_SINE_FORM) && M < LEG_TRANSFORM_MIN_M_REG)
        return leg_set_error(LEG_ERR_UNSUPPORTED, "LEG_FLAG_SINE_FORM needs M >= 256");

    leg_plan *p = new (std::nothrow) leg_plan();
    if (!p) return leg_set_error(LEG_ERR_OOM, "host allocation of the plan failed");
    p->N = N;
    p->M = M;
    p->K = K;
    p->fbits = leg_split_fbits(K);
    p->Q = (Q == 0) ? (K + 1) / 2 : Q;
    p->dtype = dtype;
    p->flags = flags;
    p->L = M / 2;
    p->rows = M / 2 + 1;
    p->Kp = leg_round_up(K, LEG_KPAD);
    if (flags & LEG_FLAG_SINE_FORM) p->fft_variant = LEG_TRANSFORM_SINE;
    int rc = LEG_OK;
    if (cudaGetDevice(&p->device) != cudaSuccess) {
        delete p;
        return leg_set_error(LEG_ERR_CUDA, "cudaGetDevice failed");
    }
    if (const char *env = getenv("LEG_WAIT_LIMIT_CYCLES")) {
        long long v = atoll(env);
        if (v > 0) p->wait_limit = v;
    }
    if (leg_dev_malloc(&p->status, sizeof(int)) != cudaSuccess || cudaMemset(p->status, 0, sizeof(int)) != cudaSuccess) {
        free_plan(p);
        return leg_set_error(LEG_ERR_OOM, "status word allocation failed");
    }
    if ((rc = leg_build_twiddles(p)) != LEG_OK || (rc = leg_build_operator(p)) != LEG_OK) {
        free_plan(p);
        return rc;
    }
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        free_plan(p);
        return leg_set_error(LEG_ERR_CUDA, std::string("plan build: ") + cudaGetErrorString(e));
    }
    *out = p;
    return LEG_OK;
}

extern "C" int leg_plan_create_like(leg_plan_t *out, leg_plan_t src, int dtype)
{
    if (!out) return leg_set_error(LEG_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    int rc = check_plan(src);
    if (rc) return rc;
    if (dtype < LEG_F64 || dtype > LEG_SPLIT_FP16) return leg_set_error(LEG_ERR_INVALID_ARG, "unknown dtype");
    leg_plan *p = new (std::nothrow) leg_plan();
    if (!p) return leg_set_error(LEG_ERR_OOM, "host allocation of the plan failed");
    p->N = src->N;
    p->M = src->M;
    p->K = src->K;
    p->fbits = src->fbits;
    p->Q = src->Q;
    p->dtype = dtype;
    p->flags = src->flags;
    p->L = src->L;
    p->rows = src->rows;
    p->Kp = src->Kp;
    p->device = src->device;
    p->wait_limit = src->wait_limit;
    if (p->flags & LEG_FLAG_SINE_FORM) p->fft_variant = LEG_TRANSFORM_SINE;
    auto fail = [&](int code, const char *what) {
        free_plan(p);
        return leg_set_error(code, what);
    };
    if (leg_dev_malloc(&p->status, sizeof(int)) != cudaSuccess || cudaMemset(p->status, 0, sizeof(int)) != cudaSuccess)
        return fail(LEG_ERR_OOM, "status word allocation failed");
    if (leg_dev_malloc(&p->omt2, sizeof(double) * p->Q) != cudaSuccess ||
        leg_dev_malloc(&p->wq, sizeof(double) * p->Q) != cudaSuccess ||
        leg_dev_malloc(&p->A64, sizeof(double) * (size_t)p->rows * p->K) != cudaSuccess)
        return fail(LEG_ERR_OOM, "operator allocation failed");
    if (cudaMemcpy(p->omt2, src->omt2, sizeof(double) * p->Q, cudaMemcpyDeviceToDevice) != cudaSuccess ||
        cudaMemcpy(p->wq, src->wq, sizeof(double) * p->Q, cudaMemcpyDeviceToDevice) != cudaSuccess ||
        cudaMemcpy(p->A64, src->A64, sizeof(double) * (size_t)p->rows * p->K, cudaMemcpyDeviceToDevice) != cudaSuccess)
        return fail(LEG_ERR_CUDA, "operator copy failed");
    if ((rc = leg_build_twiddles(p)) != LEG_OK || (rc = leg_build_planes(p)) != LEG_OK) {
        free_plan(p);
        return rc;
    }
    *out = p;
    return LEG_OK;
}

extern "C" int leg_plan_create(leg_plan_t *out, int N, int M, int K, int Q, int dtype)
{
    return leg_plan_create_ex(out, N, M, K, Q, dtype, 0u);
}

extern "C" int leg_plan_destroy(leg_plan_t plan)
{
    free_plan(plan);
    return LEG_OK;
}

extern "C" int leg_plan_reserve(leg_plan_t p, int B)
{
    int rc = check_plan(p);
    if (rc) return rc;
    if (B < 0) return leg_set_error(LEG_ERR_INVALID_ARG, "B < 0");
    return ensure_workspace(p, B);
}

extern "C" int leg_plan_info(leg_plan_t p, int *N, int *M, int *K, int *Q, int *dtype, int *Kp, int *rows)
{
    if (!p) return leg_set_error(LEG_ERR_INVALID_ARG, "plan is NULL");
    if (N) *N = p->N;
    if (M) *M = p->M;
    if (K) *K = p->K;
    if (Q) *Q = p->Q;
    if (dtype) *dtype = p->dtype;
    if (Kp) *Kp = p->Kp;
    if (rows) *rows = p->rows;
    return LEG_OK;
}

namespace {
// The forward pass; when ev != nullptr, events ev[0..3] are recorded on the
// stream before the input preparation, the GEMM, the FFT, and after the FFT.
int forward_impl(leg_plan_t p, const void *f, void *c, int B, cudaStream_t st, cudaEvent_t *ev)
{
    int rc = check_plan(p);
    if (rc) return rc;
    if (B < 0) return leg_set_error(LEG_ERR_INVALID_ARG, "B < 0");
    if (B == 0) return LEG_OK;
    if (!f || !c) return leg_set_error(LEG_ERR_INVALID_ARG, "null f or c");
    if ((rc = ensure_workspace(p, B))) return rc;
    if (ev) LEG_CUDA_TRY(cudaEventRecord(ev[0], st));
    if (p->collapsed()) {
        // c = L f: one GEMM into c, no transform stage
        switch (p->dtype) {
        case LEG_F64:
            if (ev) LEG_CUDA_TRY(cudaEventRecord(ev[1], st));
            rc = leg_gemm_f64_fwd(static_cast<const double *>(f), p->K, p->L64, p->K, static_cast<double *>(c),
                                  p->N, B, p->N, p->K, st);
            break;
        case LEG_F32:
            if (ev) LEG_CUDA_TRY(cudaEventRecord(ev[1], st));
            rc = leg_gemm_f32_fwd(static_cast<const float *>(f), p->K, p->A32, p->K, static_cast<float *>(c), p->N,
                                  B, p->N, p->K, st);
            break;
        case LEG_SPLIT_FP16:
            rc = leg_split_prepare_input(p, static_cast<const float *>(f), B, st);
            if (!rc && ev) LEG_CUDA_TRY(cudaEventRecord(ev[1], st));
            if (!rc) rc = leg_gemm_split_collapsed_fwd(p, B, static_cast<float *>(c), st);
            break;
        case LEG_BF16:
            rc = leg_bf16_prepare_input(p, static_cast<const float *>(f), B, st);
            if (!rc && ev) LEG_CUDA_TRY(cudaEventRecord(ev[1], st));
            if (!rc) rc = leg_gemm_bf16_fwd(p, B, c, p->N, st);
            break;
        }
        if (rc) return rc;
        if (ev) {
            LEG_CUDA_TRY(cudaEventRecord(ev[2], st));
            LEG_CUDA_TRY(cudaEventRecord(ev[3], st));
        }
        return LEG_OK;
    }
    switch (p->dtype) {
    case LEG_F64:
        if (ev) LEG_CUDA_TRY(cudaEventRecord(ev[1], st));
        rc = leg_gemm_f64_fwd(static_cast<const double *>(f), p->K, p->A64, p->K,
                              static_cast<double *>(p->G), p->ldg, B, p->rows, p->K, st);
        break;
    case LEG_F32:
        if (ev) LEG_CUDA_TRY(cudaEventRecord(ev[1], st));
        rc = leg_gemm_f32_fwd(static_cast<const float *>(f), p->K, p->A32, p->K,
                              static_cast<float *>(p->G), p->ldg, B, p->rows, p->K, st);
        break;
    case LEG_SPLIT_FP16:
        rc = leg_split_prepare_input(p, static_cast<const float *>(f), B, st);
        if (!rc && ev) LEG_CUDA_TRY(cudaEventRecord(ev[1], st));
        if (!rc) rc = leg_gemm_split_fwd(p, B, st);
        break;
    case LEG_BF16:
        rc = leg_bf16_prepare_input(p, static_cast<const float *>(f), B, st);
        if (!rc && ev) LEG_CUDA_TRY(cudaEventRecord(ev[1], st));
        if (!rc) rc = leg_gemm_bf16_fwd(p, B, p->G, p->ldg, st);
        break;
    }
    if (rc) return rc;
    if (ev) LEG_CUDA_TRY(cudaEventRecord(ev[2], st));
    rc = leg_fft_forward(p, p->G, p->ldg, c, B, st);
    if (rc) return rc;
    if (ev) LEG_CUDA_TRY(cudaEventRecord(ev[3], st));
    return LEG_OK;
}
}  // namespace

// Launches of the same call replayed from a CUDA graph: the first call with a
// key runs directly, the second captures and instantiates, later ones replay
// (two keys cached).  A call made while the caller's stream is itself being
// captured runs directly (its launches join the caller's graph).
extern "C" int leg_forward(leg_plan_t p, const void *f, void *c, int B, cudaStream_t st)
{
    int rc = check_plan(p);
    if (rc) return rc;
    if (B <= 0 || !f || !c) return forward_impl(p, f, c, B, st, nullptr);   // no-op or argument error
    if ((rc = ensure_workspace(p, B))) return rc;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    LEG_CUDA_TRY(cudaStreamIsCapturing(st, &cs));
    if (cs != cudaStreamCaptureStatusNone) return forward_impl(p, f, c, B, st, nullptr);
    leg_plan::GraphKey key;
    key.f = f;
    key.c = c;
    key.B = B;
    key.wsB = p->ws_B;
    key.G = p->G;
    key.Fh = p->Fh;
    key.tn = p->tn;
    key.fft = p->fft_variant;
    key.fft_log2e = p->fft_log2e;
    key.wait = p->wait_limit;
    leg_plan::GraphEntry *e = nullptr;
    for (auto &x : p->fwd)
        if (x.seen && x.key == key) e = &x;
    if (e && e->exec) {
        e->used = ++p->fwd_clock;
        LEG_CUDA_TRY(cudaGraphLaunch(e->exec, st));
        return LEG_OK;
    }
    if (!e) {   // a new key replaces the least recently used entry
        e = &p->fwd[0];
        for (auto &x : p->fwd)
            if (x.used < e->used) e = &x;
        if (e->exec) cudaGraphExecDestroy(e->exec);
        e->exec = nullptr;
        e->key = key;
        e->seen = true;
        e->used = ++p->fwd_clock;
        return forward_impl(p, f, c, B, st, nullptr);
    }
    // second call with this key: capture the launches on the plan's own stream
    e->used = ++p->fwd_clock;
    if (!p->cap) LEG_CUDA_TRY(cudaStreamCreateWithFlags(&p->cap, cudaStreamNonBlocking));
    LEG_CUDA_TRY(cudaStreamBeginCapture(p->cap, cudaStreamCaptureModeThreadLocal));
    rc = forward_impl(p, f, c, B, p->cap, nullptr);
    cudaGraph_t g = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(p->cap, &g);
    if (rc || ec != cudaSuccess || !g) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        e->seen = false;
        if (rc) return rc;
        return forward_impl(p, f, c, B, st, nullptr);   // capture unavailable: run directly
    }
    const cudaError_t ei = cudaGraphInstantiateWithFlags(&e->exec, g, 0);
    cudaGraphDestroy(g);
    if (ei != cudaSuccess) {
        cudaGetLastError();
        e->exec = nullptr;
        e->seen = false;
        return forward_impl(p, f, c, B, st, nullptr);
    }
    LEG_CUDA_TRY(cudaGraphLaunch(e->exec, st));
    return LEG_OK;
}

namespace {
int pipe_state(leg_plan *p, LegPipeState **out)
{
    if (!p->pipe) {
        LegPipeState *q = new (std::nothrow) LegPipeState();
        if (!q) return leg_set_error(LEG_ERR_OOM, "host allocation of the pipeline state failed");
        p->pipe = q;
        int least = 0, greatest = 0;
        LEG_CUDA_TRY(cudaDeviceGetStreamPriorityRange(&least, &greatest));
        LEG_CUDA_TRY(cudaStreamCreateWithPriority(&q->hi, cudaStreamNonBlocking, greatest));
        LEG_CUDA_TRY(cudaStreamCreateWithPriority(&q->lo, cudaStreamNonBlocking, least));
        for (cudaEvent_t *e : {&q->start, &q->gemm_done, &q->done, &q->split[0], &q->split[1], &q->tf[0], &q->tf[1]})
            LEG_CUDA_TRY(cudaEventCreateWithFlags(e, cudaEventDisableTiming));
    }
    *out = p->pipe;
    return LEG_OK;
}
}  // namespace

// The split-FP16 pipeline over nbatch batches: batch b's input split and
// GEMM go to a high-priority stream and write G or, for odd b, the backward's
// G-sized workspace; batch b-1's transform goes to a low-priority stream once
// batch b's split is done, so the GEMM's CTA pairs take their SMs first and
// the transform runs on the SMs the GEMM's tiles leave free.  Batch b's split
// waits for batch b-2's transform (the last reader of its G buffer).  Each
// kernel is the one leg_forward launches for a batch of B.  With io.stage,
// batch b's input is first copied from io.f (host) into staging buffer b % 2
// on io.copy, after the split that last read that buffer.
namespace {
// Queues the pipeline's launches on q's streams (and the copies on io.copy).
int pipeline_body(leg_plan *p, LegPipeState *q, int B, int nbatch, const LegPipeIO &io)
{
    int rc = LEG_OK;
    const LegSplitIn in = leg_split_workspace(p);
    float2 *Gs[2] = {static_cast<float2 *>(p->G), static_cast<float2 *>(p->Gbar)};
    const char *fb = static_cast<const char *>(io.f);
    char *cb = static_cast<char *>(io.c);
    for (int b = 0; b < nbatch; ++b) {
        const int s = b & 1;
        const float *fin = reinterpret_cast<const float *>(fb + io.fstride * b);
        if (io.stage[0]) {
            // a never-recorded event counts as completed: the first uses wait for nothing
            LEG_CUDA_TRY(cudaStreamWaitEvent(io.copy, io.stage_free[s], 0));
            LEG_CUDA_TRY(cudaMemcpyAsync(io.stage[s], fin, io.fstride, cudaMemcpyHostToDevice, io.copy));
            LEG_CUDA_TRY(cudaEventRecord(io.stage_ready[s], io.copy));
            LEG_CUDA_TRY(cudaStreamWaitEvent(q->hi, io.stage_ready[s], 0));
            fin = static_cast<const float *>(io.stage[s]);
        }
        if (b >= 2) LEG_CUDA_TRY(cudaStreamWaitEvent(q->hi, q->tf[s], 0));   // batch b-2's transform read Gs[s]
        if (io.prof) LEG_CUDA_TRY(cudaEventRecord(io.prof[5 * b], q->hi));
        if ((rc = leg_split_prepare_input_into(p, fin, B, in, Gs[s], p->ldg, q->hi))) return rc;
        LEG_CUDA_TRY(cudaEventRecord(q->split[s], q->hi));
        if (io.prof) LEG_CUDA_TRY(cudaEventRecord(io.prof[5 * b + 1], q->hi));
        if (io.stage[0]) LEG_CUDA_TRY(cudaEventRecord(io.stage_free[s], q->hi));
        if (b >= 1) {   // batch b-1's GEMM is done (it precedes this split on hi)
            LEG_CUDA_TRY(cudaStreamWaitEvent(q->lo, q->split[s], 0));
            if (io.prof) LEG_CUDA_TRY(cudaEventRecord(io.prof[5 * (b - 1) + 3], q->lo));
            if ((rc = leg_fft_forward(p, Gs[s ^ 1], p->ldg, cb + io.cstride * (b - 1), B, q->lo))) return rc;
            LEG_CUDA_TRY(cudaEventRecord(q->tf[s ^ 1], q->lo));
            if (io.prof) LEG_CUDA_TRY(cudaEventRecord(io.prof[5 * (b - 1) + 4], q->lo));
        }
        if ((rc = leg_gemm_split_fwd_into(p, B, in, Gs[s], p->ldg, q->hi))) return rc;
        if (io.prof) LEG_CUDA_TRY(cudaEventRecord(io.prof[5 * b + 2], q->hi));
    }
    LEG_CUDA_TRY(cudaEventRecord(q->gemm_done, q->hi));
    LEG_CUDA_TRY(cudaStreamWaitEvent(q->lo, q->gemm_done, 0));
    const int l = (nbatch - 1) & 1;
    if (io.prof) LEG_CUDA_TRY(cudaEventRecord(io.prof[5 * (nbatch - 1) + 3], q->lo));
    if ((rc = leg_fft_forward(p, Gs[l], p->ldg, cb + io.cstride * (nbatch - 1), B, q->lo))) return rc;
    if (io.prof) LEG_CUDA_TRY(cudaEventRecord(io.prof[5 * (nbatch - 1) + 4], q->lo));
    return LEG_OK;
}
}  // namespace

int leg_pipeline_split(leg_plan *p, int B, int nbatch, const LegPipeIO &io, cudaStream_t st)
{
    int rc = ensure_workspace(p, B);
    if (rc) return rc;
    LegPipeState *q = nullptr;
    if ((rc = pipe_state(p, &q))) return rc;
    LEG_CUDA_TRY(cudaEventRecord(q->start, st));   // after the work already on `stream`
    LEG_CUDA_TRY(cudaStreamWaitEvent(q->hi, q->start, 0));
    LEG_CUDA_TRY(cudaStreamWaitEvent(q->lo, q->start, 0));
    if (io.stage[0]) LEG_CUDA_TRY(cudaStreamWaitEvent(io.copy, q->start, 0));
    rc = pipeline_body(p, q, B, nbatch, io);
    // later work on `stream` follows everything queued, also after an error
    // part of the way through
    cudaError_t e = cudaEventRecord(q->gemm_done, q->hi);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st, q->gemm_done, 0);
    if (e == cudaSuccess) e = cudaEventRecord(q->done, q->lo);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st, q->done, 0);
    if (rc) return rc;
    if (e != cudaSuccess) return leg_set_error(LEG_ERR_CUDA, cudaGetErrorString(e));
    return LEG_OK;
}

// Batches one after another: the pipeline above for split-FP16 plans of the
// Abel GEMM + transform, results those of leg_forward bit for bit; other
// plans, a single batch and calls on a stream being captured loop leg_forward.
extern "C" int leg_forward_batches(leg_plan_t p, const void *f, void *c, int B, int nbatch, cudaStream_t st)
{
    int rc = check_plan(p);
    if (rc) return rc;
    if (B < 0 || nbatch < 0) return leg_set_error(LEG_ERR_INVALID_ARG, "B < 0 or nbatch < 0");
    if (B == 0 || nbatch == 0) return LEG_OK;
    if (!f || !c) return leg_set_error(LEG_ERR_INVALID_ARG, "null f or c");
    const size_t eb = (p->dtype == LEG_F64) ? sizeof(double) : sizeof(float);
    LegPipeIO io;
    io.f = f;
    io.c = c;
    io.fstride = eb * (size_t)B * p->K;
    io.cstride = eb * (size_t)B * p->N;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    LEG_CUDA_TRY(cudaStreamIsCapturing(st, &cs));
    if (!leg_pipeline_applies(p) || nbatch == 1 || cs != cudaStreamCaptureStatusNone) {
        for (int b = 0; b < nbatch; ++b)
            if ((rc = leg_forward(p, static_cast<const char *>(f) + io.fstride * b,
                                  static_cast<char *>(c) + io.cstride * b, B, st)))
                return rc;
        return LEG_OK;
    }
    return leg_pipeline_split(p, B, nbatch, io, st);
}

bool leg_pipeline_applies(const leg_plan *p) { return p->dtype == LEG_SPLIT_FP16 && !p->collapsed(); }

// leg_forward_batches with the mean time of each stage per batch, taken with
// events on the stage's own stream inside the pipeline (or averaged over
// leg_forward_profiled calls where there is no pipeline); synchronises.
extern "C" int leg_forward_batches_profiled(leg_plan_t p, const void *f, void *c, int B, int nbatch,
                                            cudaStream_t st, float *ms)
{
    if (!ms) return leg_set_error(LEG_ERR_INVALID_ARG, "ms is NULL");
    int rc = check_plan(p);
    if (rc) return rc;
    if (B < 0 || nbatch < 0) return leg_set_error(LEG_ERR_INVALID_ARG, "B < 0 or nbatch < 0");
    ms[0] = ms[1] = ms[2] = 0.0f;
    if (B == 0 || nbatch == 0) return LEG_OK;
    if (!f || !c) return leg_set_error(LEG_ERR_INVALID_ARG, "null f or c");
    const size_t eb = (p->dtype == LEG_F64) ? sizeof(double) : sizeof(float);
    LegPipeIO io;
    io.f = f;
    io.c = c;
    io.fstride = eb * (size_t)B * p->K;
    io.cstride = eb * (size_t)B * p->N;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    LEG_CUDA_TRY(cudaStreamIsCapturing(st, &cs));
    if (cs != cudaStreamCaptureStatusNone)
        return leg_set_error(LEG_ERR_INVALID_ARG, "leg_forward_batches_profiled synchronises: not on a capturing stream");
    if (!leg_pipeline_applies(p) || nbatch == 1) {
        for (int b = 0; b < nbatch; ++b) {
            float t[3];
            rc = leg_forward_profiled(p, static_cast<const char *>(f) + io.fstride * b,
                                      static_cast<char *>(c) + io.cstride * b, B, st, t);
            if (rc) return rc;
            for (int i = 0; i < 3; ++i) ms[i] += t[i] / nbatch;
        }
        return LEG_OK;
    }
    std::vector<cudaEvent_t> ev(5 * (size_t)nbatch, nullptr);
    cudaError_t e = cudaSuccess;
    for (auto &x : ev)
        if (e == cudaSuccess) e = cudaEventCreate(&x);
    if (e == cudaSuccess) {
        io.prof = ev.data();
        rc = leg_pipeline_split(p, B, nbatch, io, st);
        if (!rc) e = cudaStreamSynchronize(st);
        double sum[3] = {0.0, 0.0, 0.0};
        for (int b = 0; !rc && e == cudaSuccess && b < nbatch; ++b) {
            const int from[3] = {0, 1, 3}, to[3] = {1, 2, 4};
            for (int i = 0; i < 3 && e == cudaSuccess; ++i) {
                float t = 0.0f;
                e = cudaEventElapsedTime(&t, ev[5 * b + from[i]], ev[5 * b + to[i]]);
                sum[i] += t;
            }
        }
        for (int i = 0; i < 3; ++i) ms[i] = (float)(sum[i] / nbatch);
    }
    for (auto &x : ev)
        if (x) cudaEventDestroy(x);
    if (rc) return rc;
    if (e != cudaSuccess) return leg_set_error(LEG_ERR_CUDA, cudaGetErrorString(e));
    return LEG_OK;
}

extern "C" int leg_forward_profiled(leg_plan_t p, const void *f, void *c, int B, cudaStream_t st, float *ms)
{
    if (!ms) return leg_set_error(LEG_ERR_INVALID_ARG, "ms is NULL");
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    for (int i = 0; i < 4; ++i) LEG_CUDA_TRY(cudaEventCreate(&ev[i]));
    int rc = forward_impl(p, f, c, B, st, ev);
    if (!rc && B > 0) {
        cudaError_t e = cudaEventSynchronize(ev[3]);
        for (int i = 0; i < 3 && e == cudaSuccess; ++i) e = cudaEventElapsedTime(&ms[i], ev[i], ev[i + 1]);
        if (e != cudaSuccess) rc = leg_set_error(LEG_ERR_CUDA, cudaGetErrorString(e));
    } else if (!rc) {
        ms[0] = ms[1] = ms[2] = 0.0f;
    }
    for (int i = 0; i < 4; ++i) cudaEventDestroy(ev[i]);
    return rc;
}

extern "C" int leg_backward(leg_plan_t p, const void *dc, void *df, int B, cudaStream_t st)
{
    int rc = check_plan(p);
    if (rc) return rc;
    if (B < 0) return leg_set_error(LEG_ERR_INVALID_ARG, "B < 0");
    if (B == 0) return LEG_OK;
    if (!dc || !df) return leg_set_error(LEG_ERR_INVALID_ARG, "null dc or df");
    if ((rc = ensure_workspace(p, B))) return rc;
    if (p->collapsed()) {
        // df = L^T dc: one transposed GEMM
        switch (p->dtype) {
        case LEG_F64:
            return leg_gemm_f64_adj(static_cast<const double *>(dc), p->N, p->L64, p->K, static_cast<double *>(df),
                                    p->K, B, p->N, p->K, st);
        case LEG_F32:
            return leg_gemm_f32_adj(static_cast<const float *>(dc), p->N, p->A32, p->K, static_cast<float *>(df),
                                    p->K, B, p->N, p->K, st);
        case LEG_SPLIT_FP16:
            return leg_gemm_split_collapsed_adj(p, static_cast<const float *>(dc), df, B, st);
        default:
            return leg_set_error(LEG_ERR_UNSUPPORTED, "leg_backward is not available for LEG_BF16");
        }
    }
    if (leg_fft_adjoint_writes_planes(p)) {
        if ((rc = leg_fft_adjoint_planes(p, dc, B, st))) return rc;
        return leg_gemm_split_adj_planes(p, df, B, st);
    }
    if ((rc = leg_fft_adjoint(p, dc, p->Gbar, p->ldg, B, st))) return rc;
    switch (p->dtype) {
    case LEG_F64:
        return leg_gemm_f64_adj(static_cast<const double *>(p->Gbar), p->ldg, p->A64, p->K,
                                static_cast<double *>(df), p->K, B, p->rows, p->K, st);
    case LEG_F32:
        return leg_gemm_f32_adj(static_cast<const float *>(p->Gbar), p->ldg, p->A32, p->K,
                                static_cast<float *>(df), p->K, B, p->rows, p->K, st);
    case LEG_SPLIT_FP16:
        return leg_gemm_split_adj(p, df, B, st);
    default:
        return leg_set_error(LEG_ERR_UNSUPPORTED, "leg_backward is not available for LEG_BF16");
    }
}

// The plain method's FP64 G (B rows) filled by `fill`, then the FP64 transform.
template <class Fill>
int plain_run(leg_plan *p, int B, double *c, cudaStream_t st, Fill fill)
{
    int rc = ensure_workspace(p, B);
    if (rc) return rc;
    // the FP64 plain path needs 8-byte G elements: the plan's G when it has
    // them, else a stream-ordered allocation
    double *G = nullptr;
    int ldg = leg_round_up(p->rows, 8);
    if (g_elem_bytes(p->dtype) >= sizeof(double) && p->G) {
        G = static_cast<double *>(p->G);
        ldg = p->ldg;
    } else {
        LEG_CUDA_TRY(leg_dev_malloc_async_bytes(reinterpret_cast<void **>(&G), sizeof(double) * (size_t)B * ldg, st));
    }
    rc = fill(G, ldg);
    if (!rc) rc = leg_fft_forward_f64(p, G, ldg, c, B, st);
    if (G != p->G) leg_dev_free_async(G, st);
    return rc;
}

extern "C" int leg_plain_forward(leg_plan_t p, int family, const double *params, int B, double *c,
                                 cudaStream_t st)
{
    int rc = check_plan(p);
    if (rc) return rc;
    if (family != LEG_FAMILY_GENFN && family != LEG_FAMILY_EXP && family != LEG_FAMILY_ABSPOW)
        return leg_set_error(LEG_ERR_INVALID_ARG, "unknown family");
    if (B < 0 || B > 65535) return leg_set_error(LEG_ERR_INVALID_ARG, "B must be in [0, 65535]");
    if (B == 0) return LEG_OK;
    if (!params || !c) return leg_set_error(LEG_ERR_INVALID_ARG, "null params or c");
    return plain_run(p, B, c, st, [&](double *G, int ldg) { return leg_plain_g(p, family, params, B, G, ldg, st); });
}

extern "C" int leg_plain_forward_cheb(leg_plan_t p, const double *coef, int Kc, int B, double *c, cudaStream_t st)
{
    int rc = check_plan(p);
    if (rc) return rc;
    if (Kc < 1 || Kc > LEG_MAX_K)
        return leg_set_error(LEG_ERR_INVALID_ARG, "Kc must be in [1, " + std::to_string(LEG_MAX_K) + "]");
    if (B < 0 || B > 65535) return leg_set_error(LEG_ERR_INVALID_ARG, "B must be in [0, 65535]");
    if (B == 0) return LEG_OK;
    if (!coef || !c) return leg_set_error(LEG_ERR_INVALID_ARG, "null coef or c");
    return plain_run(p, B, c, st, [&](double *G, int ldg) { return leg_plain_g_cheb(p, coef, Kc, B, G, ldg, st); });
}

extern "C" int leg_plan_status(leg_plan_t p, int reset)
{
    int rc = check_plan(p);
    if (rc) return rc;
    int h = 0;
    LEG_CUDA_TRY(cudaMemcpy(&h, p->status, sizeof(int), cudaMemcpyDeviceToHost));
    if (reset && h) LEG_CUDA_TRY(cudaMemset(p->status, 0, sizeof(int)));
    if (h & 1) return leg_set_error(LEG_ERR_TIMEOUT, "a bounded device-side wait expired");
    return LEG_OK;
}

extern "C" int leg_plan_set_wait_limit(leg_plan_t p, long long cycles)
{
    if (!p) return leg_set_error(LEG_ERR_INVALID_ARG, "plan is NULL");
    if (cycles < 0) return leg_set_error(LEG_ERR_INVALID_ARG, "cycles < 0");
    p->wait_limit = cycles;
    return LEG_OK;
}

extern "C" int leg_plan_set_tile(leg_plan_t p, int tn)
{
    if (!p) return leg_set_error(LEG_ERR_INVALID_ARG, "plan is NULL");
    const int maxtn = (p->dtype == LEG_BF16) ? 256 : 128;
    if (tn != 0 && (tn < 16 || tn > maxtn || tn % 16 != 0))
        return leg_set_error(LEG_ERR_INVALID_ARG, "tile width must be 0 or a multiple of 16 in 16.." +
                                                      std::to_string(maxtn) + " for this plan");
    p->tn = tn;
    return LEG_OK;
}

extern "C" int leg_plan_set_host_overlap(leg_plan_t p, int on)
{
    if (!p) return leg_set_error(LEG_ERR_INVALID_ARG, "plan is NULL");
    if (on != 0 && on != 1) return leg_set_error(LEG_ERR_INVALID_ARG, "on must be 0 or 1");
    p->host_overlap = on;
    return LEG_OK;
}

extern "C" int leg_plan_set_transform(leg_plan_t p, int variant, int radix)
{
    if (!p) return leg_set_error(LEG_ERR_INVALID_ARG, "plan is NULL");
    if (variant < LEG_TRANSFORM_REG || variant > LEG_TRANSFORM_SINE)
        return leg_set_error(LEG_ERR_INVALID_ARG, "unknown transform variant");
    if (radix != 0 && radix != 8 && radix != 16)
        return leg_set_error(LEG_ERR_INVALID_ARG, "radix must be 0 (default), 8 or 16");
    if (variant == LEG_TRANSFORM_SINE && p->M < LEG_TRANSFORM_MIN_M_REG)
        return leg_set_error(LEG_ERR_UNSUPPORTED, "the sine-form transform needs M >= 256");
    p->fft_variant = variant;
    p->fft_log2e = (radix == 16) ? 4 : 3;
    return LEG_OK;
}

extern "C" int leg_plan_get_transform(leg_plan_t p, int *variant, int *radix)
{
    if (!p) return leg_set_error(LEG_ERR_INVALID_ARG, "plan is NULL");
    if (variant) *variant = p->fft_variant;
    if (radix) *radix = 1 << p->fft_log2e;
    return LEG_OK;
}

extern "C" int leg_plan_tile_info(leg_plan_t p, int B, int *tn, int *pairs, int *tiles)
{
    int rc = check_plan(p);
    if (rc) return rc;
    if (p->dtype != LEG_SPLIT_FP16)
        return leg_set_error(LEG_ERR_UNSUPPORTED, "tile information is for LEG_SPLIT_FP16 plans");
    if (B < 1) return leg_set_error(LEG_ERR_INVALID_ARG, "B < 1");
    int np = 0;
    if ((rc = leg_split_max_pairs(&np))) return rc;
    const int t = leg_split_choose_tn(p, B);
    if (tn) *tn = t;
    if (pairs) *pairs = np;
    if (tiles) *tiles = ((leg_split_fwd_rows(p) + 255) / 256) * ((B + t - 1) / t);
    return LEG_OK;
}
