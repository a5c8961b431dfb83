// Ragged batches: functions of different sizes, grouped in size buckets (one
// LEG_SPLIT_FP16 plan per bucket), computed by
//   1. one input-split launch over every function (each writes its bucket's planes),
//   2. ONE persistent tcgen05 launch over the tiles of every bucket's Abel GEMM
//      (the problems are ordered by K-depth; CTA c takes tiles c, c + #SMs, ...),
//   3. one transform launch per bucket, scattering each function's first n_out
//      coefficients into the packed output; the buckets read disjoint G
//      buffers and write disjoint output ranges, so their launches run
//      concurrently on LEG_RAGGED_LANES streams (the largest bucket first),
// the whole sequence captured once in a CUDA graph on a private stream (the
// lanes become parallel branches) and replayed on later calls.  Method: arXiv:1106.0463, Theorem 1 (Eq. 2.4,
// Eq. 2.5), per bucket exactly as leg_forward.
//
// Also: leg_sample_cl, the on-device closed-form sampler used to generate
// ragged workloads (input generation; not part of the method).
#include <math.h>

#include <algorithm>
#include <new>
#include <numeric>
#include <string>
#include <vector>

#include "leg_internal.cuh"

// streams the per-bucket transforms are spread over (the private stream and
// LEG_RAGGED_LANES - 1 more)
constexpr int LEG_RAGGED_LANES = 4;

struct leg_ragged {
    int device = 0, nplans = 0, count = 0;
    std::vector<leg_plan *> plans;
    std::vector<int> Bp, ldg;
    int *d_bucket = nullptr, *d_row = nullptr, *d_n_out = nullptr;
    long long *d_in_off = nullptr, *d_out_off = nullptr;
    std::vector<int *> d_rowfn;
    std::vector<__half *> planes;   // LEG_SPLIT_NF planes per bucket, one allocation
    std::vector<int *> fexp;
    std::vector<float2 *> G;
    LegRaggedBucket *d_bk = nullptr;
    TcProblem *d_probs = nullptr;
    int nprob = 0, ntiles = 0, tn = 128;
    int max_k = 0;   // longest row (samples) over the buckets
    int *status = nullptr;
    long long wait_limit = 2000000000LL;
    cudaStream_t rs = nullptr;
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    cudaStream_t lane[LEG_RAGGED_LANES - 1] = {};
    cudaEvent_t ev_gemm = nullptr, ev_lane[LEG_RAGGED_LANES - 1] = {};
    std::vector<int> fft_order;   // buckets by transform work, largest first
    cudaGraphExec_t gexec = nullptr;
    const void *g_f = nullptr;
    void *g_c = nullptr;
    bool ran_eager = false;
};

namespace {

void free_ragged(leg_ragged *r)
{
    if (!r) return;
    if (r->gexec) cudaGraphExecDestroy(r->gexec);
    if (r->ev_in) cudaEventDestroy(r->ev_in);
    if (r->ev_out) cudaEventDestroy(r->ev_out);
    if (r->ev_gemm) cudaEventDestroy(r->ev_gemm);
    for (int i = 0; i < LEG_RAGGED_LANES - 1; ++i) {
        if (r->ev_lane[i]) cudaEventDestroy(r->ev_lane[i]);
        if (r->lane[i]) cudaStreamDestroy(r->lane[i]);
    }
    if (r->rs) cudaStreamDestroy(r->rs);
    cudaFree(r->d_bucket);
    cudaFree(r->d_row);
    cudaFree(r->d_n_out);
    cudaFree(r->d_in_off);
    cudaFree(r->d_out_off);
    for (auto p : r->d_rowfn) cudaFree(p);
    for (auto p : r->planes) cudaFree(p);
    for (auto p : r->fexp) cudaFree(p);
    for (auto p : r->G) cudaFree(p);
    cudaFree(r->d_bk);
    cudaFree(r->d_probs);
    cudaFree(r->status);
    delete r;
}

template <class T>
int upload(T **dst, const T *src, size_t n)
{
    LEG_CUDA_TRY(cudaMalloc(dst, sizeof(T) * (n ? n : 1)));
    if (n) LEG_CUDA_TRY(cudaMemcpy(*dst, src, sizeof(T) * n, cudaMemcpyHostToDevice));
    return LEG_OK;
}

int enqueue(leg_ragged *r, const float *f, float *c, cudaStream_t st)
{
    int rc = leg_split_ragged(f, r->d_in_off, r->d_bucket, r->d_row, r->d_bk, r->count, r->max_k, st);
    if (rc) return rc;
    if ((rc = leg_gemm_split_grouped(r->d_probs, r->nprob, r->ntiles, r->tn, r->status, r->wait_limit, st))) return rc;
    // bucket i of fft_order goes to lane i mod LEG_RAGGED_LANES (lane 0 = st):
    // the largest transforms start first, one per lane, and the small ones
    // fill the GPU beside them
    const int nb = (int)r->fft_order.size();
    const int nl = nb < LEG_RAGGED_LANES ? nb : LEG_RAGGED_LANES;
    if (nl > 1) {
        LEG_CUDA_TRY(cudaEventRecord(r->ev_gemm, st));
        for (int l = 1; l < nl; ++l) LEG_CUDA_TRY(cudaStreamWaitEvent(r->lane[l - 1], r->ev_gemm, 0));
    }
    for (int i = 0; i < nb; ++i) {
        const int p = r->fft_order[i], l = i % LEG_RAGGED_LANES;
        rc = leg_fft_forward_ragged(r->plans[p], r->G[p], r->ldg[p], c, r->Bp[p], r->d_rowfn[p], r->d_out_off,
                                    r->d_n_out, l ? r->lane[l - 1] : st);
        if (rc) return rc;
    }
    for (int l = 1; l < nl; ++l) {
        LEG_CUDA_TRY(cudaEventRecord(r->ev_lane[l - 1], r->lane[l - 1]));
        LEG_CUDA_TRY(cudaStreamWaitEvent(st, r->ev_lane[l - 1], 0));
    }
    return LEG_OK;
}

// ---------------------------------------------------------------- sampler
__global__ void sample_cl_kernel(const int *__restrict__ family, const double *__restrict__ param,
                                 const int *__restrict__ Kf, const long long *__restrict__ coef_off,
                                 const double *__restrict__ coef, const long long *__restrict__ in_off,
                                 float *__restrict__ f_packed)
{
    const int i = blockIdx.x;
    const int K = Kf[i], fam = family[i];
    const double par = param[i];
    float *out = f_packed + in_off[i];
    for (int k = threadIdx.x; k < K; k += blockDim.x) {
        const double s = sinpi(k / (2.0 * (K - 1)));
        const double omx = 2.0 * s * s;                 // 1 - x_k
        const double x = cospi((double)k / (K - 1));    // x_k
        double v;
        if (fam == LEG_FAMILY_GENFN) {
            const double om = 1.0 - par;
            v = rsqrt(om * om + 2.0 * par * omx);
        } else if (fam == LEG_FAMILY_EXP) {
            v = exp(par * x);
        } else {
            // Clenshaw for sum_m c_m T_m(x)
            const double *cm = coef + coef_off[i];
            double b1 = 0.0, b2 = 0.0;
            for (int m = K - 1; m >= 1; --m) {
                const double b0 = cm[m] + 2.0 * x * b1 - b2;
                b2 = b1;
                b1 = b0;
            }
            v = cm[0] + x * b1 - b2;
        }
        out[k] = (float)v;
    }
}

}  // namespace

extern "C" int leg_ragged_create(leg_ragged_t *out, const leg_plan_t *plans, int nplans, int count,
                                 const int *plan_idx, const int *n_out, const long long *in_off,
                                 const long long *out_off)
{
    if (!out) return leg_set_error(LEG_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!plans || nplans < 1 || nplans > 64) return leg_set_error(LEG_ERR_INVALID_ARG, "need 1..64 plans");
    if (count < 0) return leg_set_error(LEG_ERR_INVALID_ARG, "count < 0");
    if (count > 0 && (!plan_idx || !n_out || !in_off || !out_off))
        return leg_set_error(LEG_ERR_INVALID_ARG, "null per-function array");
    int dev = -1;
    LEG_CUDA_TRY(cudaGetDevice(&dev));
    for (int p = 0; p < nplans; ++p) {
        if (!plans[p]) return leg_set_error(LEG_ERR_INVALID_ARG, "null plan");
        if (plans[p]->dtype != LEG_SPLIT_FP16)
            return leg_set_error(LEG_ERR_UNSUPPORTED, "ragged batches need LEG_SPLIT_FP16 plans");
        if (plans[p]->collapsed())
            return leg_set_error(LEG_ERR_UNSUPPORTED, "ragged batches take plans without LEG_FLAG_COLLAPSED");
        if (plans[p]->device != dev) return leg_set_error(LEG_ERR_INVALID_ARG, "plan on another device");
    }
    for (int i = 0; i < count; ++i) {
        if (plan_idx[i] < 0 || plan_idx[i] >= nplans)
            return leg_set_error(LEG_ERR_INVALID_ARG, "plan_idx out of range at " + std::to_string(i));
        if (n_out[i] < 1 || n_out[i] > plans[plan_idx[i]]->N)
            return leg_set_error(LEG_ERR_INVALID_ARG, "n_out outside 1..N of its plan at " + std::to_string(i));
        if (in_off[i] < 0 || out_off[i] < 0)
            return leg_set_error(LEG_ERR_INVALID_ARG, "negative offset at " + std::to_string(i));
    }
    leg_ragged *r = new (std::nothrow) leg_ragged();
    if (!r) return leg_set_error(LEG_ERR_OOM, "host allocation failed");
    r->device = dev;
    r->nplans = nplans;
    r->count = count;
    r->plans.assign(plans, plans + nplans);
    r->wait_limit = plans[0]->wait_limit;
    int rc = LEG_OK;
    auto fail = [&](int code) {
        free_ragged(r);
        return code;
    };
    // bucket rows in function order
    r->Bp.assign(nplans, 0);
    std::vector<int> row(count), bucket(count);
    std::vector<std::vector<int>> rowfn(nplans);
    for (int i = 0; i < count; ++i) {
        const int p = plan_idx[i];
        bucket[i] = p;
        row[i] = r->Bp[p]++;
        rowfn[p].push_back(i);
    }
    if ((rc = upload(&r->d_bucket, bucket.data(), count)) || (rc = upload(&r->d_row, row.data(), count)) ||
        (rc = upload(&r->d_n_out, n_out, count)) || (rc = upload(&r->d_in_off, in_off, count)) ||
        (rc = upload(&r->d_out_off, out_off, count)))
        return fail(rc);
    std::vector<LegRaggedBucket> bk(nplans);
    std::vector<TcProblem> probs;
    r->ldg.assign(nplans, 0);
    r->d_rowfn.assign(nplans, nullptr);
    r->fexp.assign(nplans, nullptr);
    r->G.assign(nplans, nullptr);
    r->planes.assign(nplans, nullptr);
    // one tile width for the whole grouped launch: the widest tile whose
    // estimated cycles on the busiest pair are within 1/16 of the best
    int tn = 128;
    {
        int pairs = 0;
        if ((rc = leg_split_max_pairs(&pairs))) return fail(rc);
        std::vector<int> cands;
        std::vector<double> cost;
        double best = -1.0;
        for (int w = 128; w >= 16; w -= 16) {
            double cycles = 0.0, longest = 0.0;
            for (int p = 0; p < nplans; ++p) {
                if (!r->Bp[p]) continue;
                const int ntm = (plans[p]->rows - 1 + 255) / 256;
                const double tile = (double)leg_split_tile_cost(w, 1, 1, plans[p]->Kp / 32, 1 << 30);
                cycles += (double)ntm * (double)((r->Bp[p] + w - 1) / w) * tile;
                longest = std::max(longest, tile);
            }
            cands.push_back(w);
            cost.push_back(std::max(cycles / pairs, longest));
            if (best < 0 || cost.back() < best) best = cost.back();
        }
        for (size_t c = 0; c < cands.size(); ++c)
            if (cost[c] <= best * (1.0 + 1.0 / 16)) {
                tn = cands[c];
                break;
            }
    }
    r->tn = tn;
    for (int p = 0; p < nplans; ++p) {
        leg_plan *pl = plans[p];
        const int B = r->Bp[p];
        const size_t Bz = B ? B : 1;
        r->ldg[p] = leg_round_up(leg_round_up(pl->rows, 8), LEG_KPAD);
        if (cudaMalloc(&r->fexp[p], sizeof(int) * Bz) != cudaSuccess ||
            cudaMalloc(&r->G[p], sizeof(float2) * Bz * r->ldg[p]) != cudaSuccess ||
            cudaMalloc(&r->planes[p], sizeof(__half) * LEG_SPLIT_NF * Bz * pl->Kp) != cudaSuccess)
            return fail(leg_set_error(LEG_ERR_OOM, "ragged workspace allocation failed"));
        if ((rc = upload(&r->d_rowfn[p], rowfn[p].data(), rowfn[p].size()))) return fail(rc);
        bk[p].in.base = r->planes[p];
        bk[p].in.pstride = Bz * pl->Kp;
        bk[p].in.ld = pl->Kp;
        bk[p].in.fexp = r->fexp[p];
        bk[p].in.fbits = pl->fbits;
        bk[p].G = r->G[p];
        bk[p].ldg = r->ldg[p];
        const float ah = (float)pl->a00;
        bk[p].a00 = make_float2(ah, (float)(pl->a00 - (double)ah));
        bk[p].K = pl->K;
        bk[p].Kp = pl->Kp;
        if (pl->K > r->max_k) r->max_k = pl->K;
        if (B > 0) {
            TcProblem pr;
            if ((rc = leg_make_split_problem(&pr, pl, bk[p].in, B, r->G[p], r->ldg[p], tn))) return fail(rc);
            probs.push_back(pr);
        }
    }
    // deepest K first, then most rows: the long tiles start first
    std::stable_sort(probs.begin(), probs.end(), [](const TcProblem &a, const TcProblem &b) {
        return a.nkb != b.nkb ? a.nkb > b.nkb : a.rows > b.rows;
    });
    int t0 = 0;
    for (auto &pr : probs) {
        pr.tile0 = t0;
        t0 += leg_split_problem_tiles(pr);
    }
    r->nprob = (int)probs.size();
    r->ntiles = t0;
    if ((rc = upload(&r->d_bk, bk.data(), bk.size())) || (rc = upload(&r->d_probs, probs.data(), probs.size())))
        return fail(rc);
    if (cudaMalloc(&r->status, sizeof(int)) != cudaSuccess || cudaMemset(r->status, 0, sizeof(int)) != cudaSuccess)
        return fail(leg_set_error(LEG_ERR_OOM, "status allocation failed"));
    if (cudaStreamCreateWithFlags(&r->rs, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&r->ev_in, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&r->ev_out, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&r->ev_gemm, cudaEventDisableTiming) != cudaSuccess)
        return fail(leg_set_error(LEG_ERR_CUDA, "stream/event creation failed"));
    for (int i = 0; i < LEG_RAGGED_LANES - 1; ++i)
        if (cudaStreamCreateWithFlags(&r->lane[i], cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&r->ev_lane[i], cudaEventDisableTiming) != cudaSuccess)
            return fail(leg_set_error(LEG_ERR_CUDA, "stream/event creation failed"));
    // transform work of a bucket ~ functions x M log M
    for (int p = 0; p < nplans; ++p)
        if (r->Bp[p] > 0) r->fft_order.push_back(p);
    auto work = [&](int p) { return (double)r->Bp[p] * r->plans[p]->M * std::log2((double)r->plans[p]->M); };
    std::stable_sort(r->fft_order.begin(), r->fft_order.end(), [&](int a, int b) { return work(a) > work(b); });
    if (cudaDeviceSynchronize() != cudaSuccess) return fail(leg_set_error(LEG_ERR_CUDA, "synchronise failed"));
    *out = r;
    return LEG_OK;
}

extern "C" int leg_forward_ragged(leg_ragged_t r, const float *f_packed, float *c_packed, cudaStream_t st)
{
    if (!r) return leg_set_error(LEG_ERR_INVALID_ARG, "ragged batch is NULL");
    if (r->count == 0) return LEG_OK;
    if (!f_packed || !c_packed) return leg_set_error(LEG_ERR_INVALID_ARG, "null f_packed or c_packed");
    int dev = -1;
    LEG_CUDA_TRY(cudaGetDevice(&dev));
    if (dev != r->device) return leg_set_error(LEG_ERR_INVALID_ARG, "current device differs from the batch's");
    // the caller is capturing its own graph: the launches join it directly
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    LEG_CUDA_TRY(cudaStreamIsCapturing(st, &cs));
    if (cs != cudaStreamCaptureStatusNone) return enqueue(r, f_packed, c_packed, st);
    LEG_CUDA_TRY(cudaEventRecord(r->ev_in, st));
    LEG_CUDA_TRY(cudaStreamWaitEvent(r->rs, r->ev_in, 0));
    int rc = LEG_OK;
    if (!r->ran_eager) {
        // first call: run eagerly (also sets kernel attributes), then capture
        if ((rc = enqueue(r, f_packed, c_packed, r->rs))) return rc;
        r->ran_eager = true;
    } else {
        if (!r->gexec || r->g_f != f_packed || r->g_c != c_packed) {
            if (r->gexec) {
                cudaGraphExecDestroy(r->gexec);
                r->gexec = nullptr;
            }
            cudaGraph_t g = nullptr;
            LEG_CUDA_TRY(cudaStreamBeginCapture(r->rs, cudaStreamCaptureModeRelaxed));
            rc = enqueue(r, f_packed, c_packed, r->rs);
            cudaError_t e = cudaStreamEndCapture(r->rs, &g);
            if (rc) {
                if (g) cudaGraphDestroy(g);
                return rc;
            }
            if (e != cudaSuccess) return leg_set_error(LEG_ERR_CUDA, std::string("capture: ") + cudaGetErrorString(e));
            e = cudaGraphInstantiate(&r->gexec, g, 0);
            cudaGraphDestroy(g);
            if (e != cudaSuccess) return leg_set_error(LEG_ERR_CUDA, std::string("instantiate: ") + cudaGetErrorString(e));
            r->g_f = f_packed;
            r->g_c = c_packed;
        }
        LEG_CUDA_TRY(cudaGraphLaunch(r->gexec, r->rs));
    }
    LEG_CUDA_TRY(cudaEventRecord(r->ev_out, r->rs));
    LEG_CUDA_TRY(cudaStreamWaitEvent(st, r->ev_out, 0));
    return LEG_OK;
}

extern "C" int leg_ragged_status(leg_ragged_t r, int reset)
{
    if (!r) return leg_set_error(LEG_ERR_INVALID_ARG, "ragged batch is NULL");
    int h = 0;
    LEG_CUDA_TRY(cudaMemcpy(&h, r->status, sizeof(int), cudaMemcpyDeviceToHost));
    if (reset && h) LEG_CUDA_TRY(cudaMemset(r->status, 0, sizeof(int)));
    if (h & 1) return leg_set_error(LEG_ERR_TIMEOUT, "a bounded device-side wait expired");
    return LEG_OK;
}

extern "C" int leg_ragged_destroy(leg_ragged_t r)
{
    if (r) cudaStreamSynchronize(r->rs);
    free_ragged(r);
    return LEG_OK;
}

extern "C" int leg_sample_cl(int count, const int *family, const double *param, const int *K,
                             const long long *coef_off, const double *coef, const long long *in_off,
                             float *f_packed, cudaStream_t st)
{
    if (count < 0) return leg_set_error(LEG_ERR_INVALID_ARG, "count < 0");
    if (count == 0) return LEG_OK;
    if (!family || !param || !K || !in_off || !f_packed)
        return leg_set_error(LEG_ERR_INVALID_ARG, "null array");
    sample_cl_kernel<<<count, 128, 0, st>>>(family, param, K, coef_off, coef, in_off, f_packed);
    LEG_LAUNCH_CHECK("sample_cl_kernel");
    return LEG_OK;
}
