// leg_forward_noalloc: the split-FP16 forward pass with its intermediate
// buffers taken from a fixed, statically sized device array instead of the
// plan's cudaMalloc'd workspace.
//
// Who needs it: callers that must not allocate device memory at call time --
// a host framework that owns the whole device-memory budget through its own
// fixed pool and forbids other allocations, or a latency-critical caller that
// cannot afford cudaMalloc/cudaFree (which may block the host and synchronise
// the device).  Such a caller creates its plan once, up front, and then runs
// batches through this entry point without any further allocation.
//
// The scratch is a file-scope __device__ array of LEG_NOALLOC_SCRATCH_BYTES
// (64 MiB).  Every GPU that loads this library keeps that much device memory
// reserved for the array until the process exits.  Host code cannot use the
// array's name as a device address (on the host it names a host-side
// stand-in), so on the first call on each device, with that device current,
// the entry point looks the address up with cudaGetSymbolAddress and caches
// it with the device's context (a new context after cudaDeviceReset triggers
// the lookup again); make that first call before any stream capture.  All calls on a
// device share the one array, and it keeps the contents of the last call:
// calls whose work overlaps on the GPU (for example on two streams) race on
// it and must be serialised by the caller.  Nothing in the array needs to
// start at zero: each call rewrites every scratch element it later reads
// (the input planes including their zero padding, the per-function scales,
// and every G element the FFT reads).
#include <mutex>
#include <string>

#include "leg_internal.cuh"

namespace {

constexpr size_t LEG_NOALLOC_SCRATCH_BYTES = size_t(64) << 20;
constexpr int LEG_NOALLOC_MAX_DEVICES = 64;

static __device__ __align__(256) unsigned char g_leg_scratch[LEG_NOALLOC_SCRATCH_BYTES];

std::mutex g_scratch_mutex;
void *g_scratch_ptr[LEG_NOALLOC_MAX_DEVICES] = {};
CUcontext g_scratch_ctx[LEG_NOALLOC_MAX_DEVICES] = {};   // the context the address belongs to

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

// The current driver context (cuCtxGetCurrent through the runtime's entry
// point lookup, so that the library needs no link against the driver library).
int current_context(CUcontext *ctx)
{
    using GetCurrent = CUresult (*)(CUcontext *);
    static GetCurrent fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q);
        if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !p)
            return leg_set_error(LEG_ERR_CUDA, "leg_forward_noalloc: cuCtxGetCurrent entry point not found");
        fn = reinterpret_cast<GetCurrent>(p);
    }
    if (fn(ctx) != CUDA_SUCCESS) return leg_set_error(LEG_ERR_CUDA, "leg_forward_noalloc: cuCtxGetCurrent failed");
    return LEG_OK;
}

// Device address of the scratch array on the current device: looked up on the
// first use, and again when the device's context has changed since (after a
// cudaDeviceReset the array lives at a new address in the new context).
int scratch_address(int dev, unsigned char **out)
{
    if (dev < 0 || dev >= LEG_NOALLOC_MAX_DEVICES)
        return leg_set_error(LEG_ERR_UNSUPPORTED, "leg_forward_noalloc: device ordinal out of range");
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    CUcontext ctx = nullptr;
    int rc = current_context(&ctx);
    if (rc) return rc;
    if (!g_scratch_ptr[dev] || g_scratch_ctx[dev] != ctx) {
        void *ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_leg_scratch);
        if (e != cudaSuccess || !ptr)
            return leg_set_error(LEG_ERR_CUDA, std::string("leg_forward_noalloc: cudaGetSymbolAddress: ") +
                                                   cudaGetErrorString(e));
        g_scratch_ptr[dev] = ptr;
        g_scratch_ctx[dev] = ctx;
    }
    *out = static_cast<unsigned char *>(g_scratch_ptr[dev]);
    return LEG_OK;
}

}  // namespace

extern "C" int leg_forward_noalloc(leg_plan_t p, const float *f, float *c, int B, cudaStream_t st)
{
    if (!p) return leg_set_error(LEG_ERR_INVALID_ARG, "plan is NULL");
    if (p->dtype != LEG_SPLIT_FP16)
        return leg_set_error(LEG_ERR_INVALID_ARG, "leg_forward_noalloc needs a LEG_SPLIT_FP16 plan");
    if (p->collapsed())
        return leg_set_error(LEG_ERR_UNSUPPORTED, "leg_forward_noalloc takes plans without LEG_FLAG_COLLAPSED");
    if (B < 0) return leg_set_error(LEG_ERR_INVALID_ARG, "B < 0");
    if (B == 0) return LEG_OK;
    if (!f || !c) return leg_set_error(LEG_ERR_INVALID_ARG, "null f or c");
    int dev = -1;
    LEG_CUDA_TRY(cudaGetDevice(&dev));
    if (dev != p->device)
        return leg_set_error(LEG_ERR_INVALID_ARG, "current device differs from the plan's device");

    // scratch layout: the split input planes (LEG_SPLIT_NF x B x Kp FP16),
    // per-function scales, G (B x ldg double-float)
    const int ldg = leg_round_up(leg_round_up(p->rows, 8), LEG_KPAD);
    const size_t plane = align256(sizeof(__half) * (size_t)B * p->Kp);
    const size_t exps = align256(sizeof(int) * (size_t)B);
    const size_t gbytes = align256(sizeof(float2) * (size_t)B * ldg);
    const size_t need = LEG_SPLIT_NF * plane + exps + gbytes;
    if (need > LEG_NOALLOC_SCRATCH_BYTES)
        return leg_set_error(LEG_ERR_INVALID_ARG,
                             "leg_forward_noalloc: this batch needs " + std::to_string(need) +
                                 " bytes of scratch; the static scratch holds " +
                                 std::to_string(LEG_NOALLOC_SCRATCH_BYTES) + " bytes (use a smaller B)");
    unsigned char *base = nullptr;
    int rc = scratch_address(dev, &base);
    if (rc) return rc;
    LegSplitIn in;
    in.base = reinterpret_cast<__half *>(base);
    in.pstride = plane / sizeof(__half);
    in.ld = p->Kp;
    in.fexp = reinterpret_cast<int *>(base + LEG_SPLIT_NF * plane);
    in.fbits = p->fbits;
    float2 *G = reinterpret_cast<float2 *>(base + LEG_SPLIT_NF * plane + exps);

    if ((rc = leg_split_prepare_input_into(p, f, B, in, G, ldg, st))) return rc;
    if ((rc = leg_gemm_split_fwd_into(p, B, in, G, ldg, st))) return rc;
    return leg_fft_forward(p, G, ldg, c, B, st);
}
