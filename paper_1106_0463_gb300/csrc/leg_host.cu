// leg_forward_host: leg_forward on host buffers.  Page-locked host buffers
// mapped into the device's address space are used in place by the split-FP16
// and BF16 paths (their first kernel reads each input value once, their last
// writes each coefficient once).  With the plan's host overlap on, the input
// of such a call is instead copied by a copy engine into one of two staging
// buffers, ordered only after the last use of that buffer, so that it crosses
// the host link while the previous call's kernels run.  Otherwise the batch
// is copied to the device, transformed and copied back with the copies
// overlapped with the computation: for the split-FP16 path the host-to-device
// copy runs in LEG_HOST_CHUNKS pieces on an internal stream and the input
// split of each piece starts as soon as it has landed; the transform runs per
// piece and each piece's coefficients are copied back while the next piece is
// transformed.  The Abel GEMM (or the collapsed GEMM) runs once on the whole
// batch in between.  Results are the same as leg_forward's bit for bit: every
// kernel computes each function independently of the others.
#include <new>

#include "leg_internal.cuh"

struct LegHostState {
    void *f = nullptr, *c = nullptr;   // device copies of the batch (input, output)
    int cap = 0;                       // functions they hold
    cudaStream_t h2d = nullptr, d2h = nullptr;
    cudaEvent_t start = nullptr, done = nullptr;
    cudaEvent_t in[LEG_HOST_CHUNKS] = {}, out[LEG_HOST_CHUNKS] = {};
    // host overlap: two staging buffers of the input, the event after the
    // last call that read each (recorded on that call's stream) and the
    // event after each one's copy
    void *stage[2] = {};
    int stage_cap = 0;   // functions each holds
    int slot = 0;        // the buffer the next call uses
    cudaEvent_t stage_free[2] = {}, stage_ready[2] = {};
};

void leg_host_free(leg_plan *p)
{
    LegHostState *h = p->host;
    if (!h) return;
    leg_dev_free(h->f);
    leg_dev_free(h->c);
    for (int i = 0; i < LEG_HOST_CHUNKS; ++i) {
        if (h->in[i]) cudaEventDestroy(h->in[i]);
        if (h->out[i]) cudaEventDestroy(h->out[i]);
    }
    for (int i = 0; i < 2; ++i) {
        leg_dev_free(h->stage[i]);
        if (h->stage_free[i]) cudaEventDestroy(h->stage_free[i]);
        if (h->stage_ready[i]) cudaEventDestroy(h->stage_ready[i]);
    }
    if (h->start) cudaEventDestroy(h->start);
    if (h->done) cudaEventDestroy(h->done);
    if (h->h2d) cudaStreamDestroy(h->h2d);
    if (h->d2h) cudaStreamDestroy(h->d2h);
    delete h;
    p->host = nullptr;
}

namespace {

// The plan's copy state: streams and events, created by the first call.
int host_base(leg_plan *p, LegHostState **out)
{
    if (!p->host) {
        LegHostState *h = new (std::nothrow) LegHostState();
        if (!h) return leg_set_error(LEG_ERR_OOM, "host allocation of the copy state failed");
        p->host = h;
        LEG_CUDA_TRY(cudaStreamCreateWithFlags(&h->h2d, cudaStreamNonBlocking));
        LEG_CUDA_TRY(cudaStreamCreateWithFlags(&h->d2h, cudaStreamNonBlocking));
        LEG_CUDA_TRY(cudaEventCreateWithFlags(&h->start, cudaEventDisableTiming));
        LEG_CUDA_TRY(cudaEventCreateWithFlags(&h->done, cudaEventDisableTiming));
        for (int i = 0; i < LEG_HOST_CHUNKS; ++i) {
            LEG_CUDA_TRY(cudaEventCreateWithFlags(&h->in[i], cudaEventDisableTiming));
            LEG_CUDA_TRY(cudaEventCreateWithFlags(&h->out[i], cudaEventDisableTiming));
        }
        for (int i = 0; i < 2; ++i) {
            LEG_CUDA_TRY(cudaEventCreateWithFlags(&h->stage_free[i], cudaEventDisableTiming));
            LEG_CUDA_TRY(cudaEventCreateWithFlags(&h->stage_ready[i], cudaEventDisableTiming));
        }
    }
    *out = p->host;
    return LEG_OK;
}

// The copy state with device copies of a batch of B functions (input and output).
int host_state(leg_plan *p, int B, size_t eb, LegHostState **out)
{
    LegHostState *h = nullptr;
    int rc = host_base(p, &h);
    if (rc) return rc;
    if (B > h->cap) {
        LEG_CUDA_TRY(cudaDeviceSynchronize());   // earlier calls may still use the old buffers
        leg_dev_free(h->f);
        leg_dev_free(h->c);
        h->f = h->c = nullptr;
        h->cap = 0;
        cudaError_t e = leg_dev_malloc(&h->f, eb * (size_t)B * p->K);
        if (e == cudaSuccess) e = leg_dev_malloc(&h->c, eb * (size_t)B * p->N);
        if (e != cudaSuccess) {   // release what was taken: nothing stays half-grown
            leg_dev_free(h->f);
            leg_dev_free(h->c);
            h->f = h->c = nullptr;
            return leg_set_error(e == cudaErrorMemoryAllocation ? LEG_ERR_OOM : LEG_ERR_CUDA,
                                 std::string("leg_forward_host device copies: ") + cudaGetErrorString(e));
        }
        h->cap = B;
    }
    *out = h;
    return LEG_OK;
}

// The device address of host memory the GPU can access in place (page-locked
// memory, mapped into the device's address space), or nullptr.
const void *device_view(const void *host)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, host) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (a.type != cudaMemoryTypeHost || !a.devicePointer) return nullptr;
    return a.devicePointer;
}

// Two staging buffers of B input rows each (grown on demand; growing
// synchronises the device).
int ensure_stage(LegHostState *h, const leg_plan *p, int B)
{
    if (B <= h->stage_cap) return LEG_OK;
    LEG_CUDA_TRY(cudaDeviceSynchronize());   // earlier calls may still use the old buffers
    for (int i = 0; i < 2; ++i) {
        leg_dev_free(h->stage[i]);
        h->stage[i] = nullptr;
    }
    h->stage_cap = 0;
    const size_t bytes = sizeof(float) * (size_t)B * p->K;
    for (int i = 0; i < 2; ++i) {
        const cudaError_t e = leg_dev_malloc(&h->stage[i], bytes);
        if (e != cudaSuccess) {   // release what was taken: nothing stays half-grown
            for (int j = 0; j < 2; ++j) {
                leg_dev_free(h->stage[j]);
                h->stage[j] = nullptr;
            }
            return leg_set_error(e == cudaErrorMemoryAllocation ? LEG_ERR_OOM : LEG_ERR_CUDA,
                                 std::string("leg_forward_host staging buffers: ") + cudaGetErrorString(e));
        }
    }
    h->stage_cap = B;
    return LEG_OK;
}

// Host overlap: the input goes to staging buffer `slot` by a copy on the
// internal stream that waits only for the previous call that used the same
// buffer to finish; the kernels read it there and write c in place (cv).
int forward_staged(leg_plan *p, const void *f_host, void *cv, int B, cudaStream_t st)
{
    LegHostState *h = nullptr;
    int rc = host_base(p, &h);
    if (rc) return rc;
    if ((rc = ensure_stage(h, p, B))) return rc;
    const size_t bytes = sizeof(float) * (size_t)B * p->K;
    const int s = h->slot;
    // a never-recorded event counts as completed: the first use waits for nothing
    LEG_CUDA_TRY(cudaStreamWaitEvent(h->h2d, h->stage_free[s], 0));
    LEG_CUDA_TRY(cudaMemcpyAsync(h->stage[s], f_host, bytes, cudaMemcpyHostToDevice, h->h2d));
    LEG_CUDA_TRY(cudaEventRecord(h->stage_ready[s], h->h2d));
    LEG_CUDA_TRY(cudaStreamWaitEvent(st, h->stage_ready[s], 0));
    if ((rc = leg_forward(p, h->stage[s], cv, B, st))) return rc;
    LEG_CUDA_TRY(cudaEventRecord(h->stage_free[s], st));
    h->slot = s ^ 1;
    return LEG_OK;
}

}  // namespace

extern "C" int leg_forward_host(leg_plan_t p, const void *f_host, void *c_host, int B, cudaStream_t st)
{
    if (!p) return leg_set_error(LEG_ERR_INVALID_ARG, "plan is NULL");
    if (B < 0) return leg_set_error(LEG_ERR_INVALID_ARG, "B < 0");
    if (B == 0) return LEG_OK;
    if (!f_host || !c_host) return leg_set_error(LEG_ERR_INVALID_ARG, "null f_host or c_host");
    int dev = -1;
    LEG_CUDA_TRY(cudaGetDevice(&dev));
    if (dev != p->device) return leg_set_error(LEG_ERR_INVALID_ARG, "current device differs from the plan's device");
    const size_t eb = (p->dtype == LEG_F64) ? sizeof(double) : sizeof(float);
    int rc = leg_plan_reserve(p, B);
    if (rc) return rc;
    // page-locked, mapped host buffers: the kernels read f and write c in
    // place over the host link (the split reads each row once, the transform
    // writes each coefficient once), so the transfers overlap the computation
    // with no staging copy
    if (p->dtype == LEG_SPLIT_FP16 || p->dtype == LEG_BF16) {   // the SIMT GEMMs re-read f per tile
        const void *fv = device_view(f_host);
        void *cv = const_cast<void *>(device_view(c_host));
        if (fv && cv) {
            cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
            LEG_CUDA_TRY(cudaStreamIsCapturing(st, &cs));
            if (p->host_overlap && cs == cudaStreamCaptureStatusNone) return forward_staged(p, f_host, cv, B, st);
            return leg_forward(p, fv, cv, B, st);
        }
    }
    LegHostState *h = nullptr;
    if ((rc = host_state(p, B, eb, &h))) return rc;

    const bool split = (p->dtype == LEG_SPLIT_FP16);
    const int nch = split ? (B < LEG_HOST_CHUNKS ? B : LEG_HOST_CHUNKS) : 1;
    auto off = [&](int i) { return (int)((long long)B * i / nch); };
    const size_t frow = eb * p->K, crow = eb * p->N;
    const char *fh = static_cast<const char *>(f_host);
    char *ch = static_cast<char *>(c_host);
    char *fd = static_cast<char *>(h->f), *cd = static_cast<char *>(h->c);

    // the copies start after the work already queued on `stream` (which may
    // still read the device buffers of an earlier call)
    LEG_CUDA_TRY(cudaEventRecord(h->start, st));
    LEG_CUDA_TRY(cudaStreamWaitEvent(h->h2d, h->start, 0));
    LEG_CUDA_TRY(cudaStreamWaitEvent(h->d2h, h->start, 0));
    for (int i = 0; i < nch; ++i) {
        const int b0 = off(i), nb = off(i + 1) - b0;
        LEG_CUDA_TRY(cudaMemcpyAsync(fd + frow * b0, fh + frow * b0, frow * nb, cudaMemcpyHostToDevice, h->h2d));
        LEG_CUDA_TRY(cudaEventRecord(h->in[i], h->h2d));
    }
    if (split) {
        const LegSplitIn in = leg_split_workspace(p);
        float2 *G = p->collapsed() ? nullptr : static_cast<float2 *>(p->G);
        for (int i = 0; i < nch; ++i) {
            const int b0 = off(i), nb = off(i + 1) - b0;
            LegSplitIn ini = in;
            ini.base = in.base + (size_t)b0 * in.ld;
            ini.fexp = in.fexp + b0;
            LEG_CUDA_TRY(cudaStreamWaitEvent(st, h->in[i], 0));
            rc = leg_split_prepare_input_into(p, reinterpret_cast<const float *>(fd + frow * b0), nb, ini,
                                              G ? G + (size_t)b0 * p->ldg : nullptr, p->ldg, st);
            if (rc) return rc;
        }
        if (p->collapsed()) {
            if ((rc = leg_gemm_split_collapsed_fwd(p, B, reinterpret_cast<float *>(cd), st))) return rc;
            LEG_CUDA_TRY(cudaEventRecord(h->out[0], st));
            LEG_CUDA_TRY(cudaStreamWaitEvent(h->d2h, h->out[0], 0));
            LEG_CUDA_TRY(cudaMemcpyAsync(ch, cd, crow * B, cudaMemcpyDeviceToHost, h->d2h));
        } else {
            if ((rc = leg_gemm_split_fwd(p, B, st))) return rc;
            for (int i = 0; i < nch; ++i) {
                const int b0 = off(i), nb = off(i + 1) - b0;
                rc = leg_fft_forward(p, G + (size_t)b0 * p->ldg, p->ldg, cd + crow * b0, nb, st);
                if (rc) return rc;
                LEG_CUDA_TRY(cudaEventRecord(h->out[i], st));
                LEG_CUDA_TRY(cudaStreamWaitEvent(h->d2h, h->out[i], 0));
                LEG_CUDA_TRY(cudaMemcpyAsync(ch + crow * b0, cd + crow * b0, crow * nb, cudaMemcpyDeviceToHost,
                                             h->d2h));
            }
        }
    } else {
        LEG_CUDA_TRY(cudaStreamWaitEvent(st, h->in[0], 0));
        if ((rc = leg_forward(p, fd, cd, B, st))) return rc;
        LEG_CUDA_TRY(cudaEventRecord(h->out[0], st));
        LEG_CUDA_TRY(cudaStreamWaitEvent(h->d2h, h->out[0], 0));
        LEG_CUDA_TRY(cudaMemcpyAsync(ch, cd, crow * B, cudaMemcpyDeviceToHost, h->d2h));
    }
    // later work on `stream` (and a synchronisation of it) sees c_host complete
    LEG_CUDA_TRY(cudaEventRecord(h->done, h->d2h));
    LEG_CUDA_TRY(cudaStreamWaitEvent(st, h->done, 0));
    return LEG_OK;
}

// Batches on host buffers.  Split-FP16 plans with pinned, mapped buffers run
// the batch pipeline of leg_forward_batches with each batch's input copied
// by a copy engine into one of the two staging buffers (the first copy after
// the work already on `stream`, each later one during the kernels of the
// batches before it) and each batch's coefficients written into c_host in
// place by its transform.  Otherwise the batches go through
// leg_forward_host in turn.
extern "C" int leg_forward_host_batches(leg_plan_t p, const void *f_host, void *c_host, int B, int nbatch,
                                        cudaStream_t st)
{
    if (!p) return leg_set_error(LEG_ERR_INVALID_ARG, "plan is NULL");
    if (B < 0 || nbatch < 0) return leg_set_error(LEG_ERR_INVALID_ARG, "B < 0 or nbatch < 0");
    if (B == 0 || nbatch == 0) return LEG_OK;
    if (!f_host || !c_host) return leg_set_error(LEG_ERR_INVALID_ARG, "null f_host or c_host");
    int dev = -1;
    LEG_CUDA_TRY(cudaGetDevice(&dev));
    if (dev != p->device) return leg_set_error(LEG_ERR_INVALID_ARG, "current device differs from the plan's device");
    int rc = leg_plan_reserve(p, B);
    if (rc) return rc;
    const size_t eb = (p->dtype == LEG_F64) ? sizeof(double) : sizeof(float);
    LegPipeIO io;
    io.f = f_host;
    io.fstride = eb * (size_t)B * p->K;
    io.cstride = eb * (size_t)B * p->N;
    if (leg_pipeline_applies(p) && nbatch > 1) {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        LEG_CUDA_TRY(cudaStreamIsCapturing(st, &cs));
        void *cv = const_cast<void *>(device_view(c_host));
        if (cs == cudaStreamCaptureStatusNone && device_view(f_host) && cv) {
            LegHostState *h = nullptr;
            if ((rc = host_base(p, &h))) return rc;
            if ((rc = ensure_stage(h, p, B))) return rc;
            io.c = cv;
            io.copy = h->h2d;
            for (int i = 0; i < 2; ++i) {
                io.stage[i] = h->stage[i];
                io.stage_ready[i] = h->stage_ready[i];
                io.stage_free[i] = h->stage_free[i];
            }
            return leg_pipeline_split(p, B, nbatch, io, st);
        }
    }
    for (int b = 0; b < nbatch; ++b) {
        rc = leg_forward_host(p, static_cast<const char *>(f_host) + io.fstride * b,
                              static_cast<char *>(c_host) + io.cstride * b, B, st);
        if (rc) return rc;
    }
    return LEG_OK;
}
