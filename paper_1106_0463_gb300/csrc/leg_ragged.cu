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

#include <stdlib.h>

#include <algorithm>
#include <mutex>
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
    std::vector<LegRaggedBucket> bk;   // host copy of the bucket descriptors (problems are rebuilt per tile width)
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
    leg_dev_free(r->d_bucket);
    leg_dev_free(r->d_row);
    leg_dev_free(r->d_n_out);
    leg_dev_free(r->d_in_off);
    leg_dev_free(r->d_out_off);
    for (auto p : r->d_rowfn) leg_dev_free(p);
    for (auto p : r->planes) leg_dev_free(p);
    for (auto p : r->fexp) leg_dev_free(p);
    for (auto p : r->G) leg_dev_free(p);
    leg_dev_free(r->d_bk);
    leg_dev_free(r->d_probs);
    leg_dev_free(r->status);
    delete r;
}

template <class T>
int upload(T **dst, const T *src, size_t n)
{
    LEG_CUDA_TRY(leg_dev_malloc(dst, sizeof(T) * (n ? n : 1)));
    if (n) LEG_CUDA_TRY(cudaMemcpy(*dst, src, sizeof(T) * n, cudaMemcpyHostToDevice));
    return LEG_OK;
}

// The batch's launches on st; with ev != nullptr, events ev[0..3] are recorded
// before the split, before the grouped GEMM, before the transforms and after
// the last transform (the lanes joined back into st).
int enqueue(leg_ragged *r, const float *f, float *c, cudaStream_t st, cudaEvent_t *ev = nullptr)
{
    if (ev) LEG_CUDA_TRY(cudaEventRecord(ev[0], st));
    int rc = leg_split_ragged(f, r->d_in_off, r->d_bucket, r->d_row, r->d_bk, r->count, r->max_k, st);
    if (rc) return rc;
    if (ev) LEG_CUDA_TRY(cudaEventRecord(ev[1], st));
    if ((rc = leg_gemm_split_grouped(r->d_probs, r->nprob, r->ntiles, r->tn, r->status, r->wait_limit, st))) return rc;
    if (ev) LEG_CUDA_TRY(cudaEventRecord(ev[2], st));
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
    if (ev) LEG_CUDA_TRY(cudaEventRecord(ev[3], st));
    return LEG_OK;
}

// Grouped-GEMM problems of every non-empty bucket at tile width tn, deepest K
// first (the long tiles start first), uploaded to d_probs; drops the graph.
int set_tile(leg_ragged *r, int tn)
{
    std::vector<TcProblem> probs;
    int rc;
    for (int p = 0; p < r->nplans; ++p) {
        if (r->Bp[p] == 0) continue;
        TcProblem pr;
        if ((rc = leg_make_split_problem(&pr, r->plans[p], r->bk[p].in, r->Bp[p], r->G[p], r->ldg[p], tn))) return rc;
        probs.push_back(pr);
    }
    std::stable_sort(probs.begin(), probs.end(), [](const TcProblem &a, const TcProblem &b) {
        return a.nkb != b.nkb ? a.nkb > b.nkb : a.rows > b.rows;
    });
    int t0 = 0;
    for (auto &pr : probs) {
        pr.tile0 = t0;
        t0 += leg_split_problem_tiles(pr);
    }
    if (r->d_probs && (int)probs.size() > r->nprob) {
        leg_dev_free(r->d_probs);
        r->d_probs = nullptr;
    }
    if (!r->d_probs) LEG_CUDA_TRY(leg_dev_malloc(&r->d_probs, sizeof(TcProblem) * (probs.empty() ? 1 : probs.size())));
    if (!probs.empty())
        LEG_CUDA_TRY(cudaMemcpy(r->d_probs, probs.data(), sizeof(TcProblem) * probs.size(), cudaMemcpyHostToDevice));
    r->nprob = (int)probs.size();
    r->ntiles = t0;
    r->tn = tn;
    if (r->gexec) {
        cudaGraphExecDestroy(r->gexec);
        r->gexec = nullptr;
    }
    return LEG_OK;
}

// Model choice of the grouped launch's tile width: the widest tile whose
// estimated cycles on the busiest pair are within 1/16 of the best.
int model_tile(const leg_ragged *r, int *tn_out)
{
    int pairs = 0;
    int rc = leg_split_max_pairs(&pairs);
    if (rc) return rc;
    std::vector<int> cands;
    std::vector<double> cost;
    double best = -1.0;
    for (int w = 128; w >= 16; w -= 16) {
        double cycles = 0.0, longest = 0.0;
        for (int p = 0; p < r->nplans; ++p) {
            if (!r->Bp[p]) continue;
            const int ntm = (r->plans[p]->rows - 1 + 255) / 256;
            const double tile = (double)leg_split_tile_cost(w, 1, 1, r->plans[p]->Kp / 32, 1 << 30);
            cycles += (double)ntm * (double)((r->Bp[p] + w - 1) / w) * tile;
            longest = std::max(longest, tile);
        }
        cands.push_back(w);
        cost.push_back(std::max(cycles / pairs, longest));
        if (best < 0 || cost.back() < best) best = cost.back();
    }
    *tn_out = 128;
    for (size_t c = 0; c < cands.size(); ++c)
        if (cost[c] <= best * (1.0 + 1.0 / 16)) {
            *tn_out = cands[c];
            break;
        }
    return LEG_OK;
}

// Key of a batch in the tuning cache: device, then (N, M, K, Q, functions)
// of every bucket.
std::string ragged_key(const leg_ragged *r)
{
    cudaDeviceProp prop;
    std::string dev = "gpu";
    if (cudaGetDeviceProperties(&prop, r->device) == cudaSuccess) dev = prop.name;
    for (auto &ch : dev)
        if (ch == ' ' || ch == '|') ch = '_';
    std::string k = "ragged|" + dev;
    for (int p = 0; p < r->nplans; ++p) {
        const leg_plan *pl = r->plans[p];
        k += "|" + std::to_string(pl->N) + "," + std::to_string(pl->M) + "," + std::to_string(pl->K) + "," +
             std::to_string(pl->Q) + "," + std::to_string(r->Bp[p]);
    }
    return k;
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
    std::vector<LegRaggedBucket> &bk = r->bk;
    bk.assign(nplans, LegRaggedBucket{});
    r->ldg.assign(nplans, 0);
    r->d_rowfn.assign(nplans, nullptr);
    r->fexp.assign(nplans, nullptr);
    r->G.assign(nplans, nullptr);
    r->planes.assign(nplans, nullptr);
    for (int p = 0; p < nplans; ++p) {
        leg_plan *pl = plans[p];
        const int B = r->Bp[p];
        const size_t Bz = B ? B : 1;
        r->ldg[p] = leg_round_up(leg_round_up(pl->rows, 8), LEG_KPAD);
        if (leg_dev_malloc(reinterpret_cast<void **>(&r->fexp[p]), sizeof(int) * Bz) != cudaSuccess ||
            leg_dev_malloc(reinterpret_cast<void **>(&r->G[p]), sizeof(float2) * Bz * r->ldg[p]) != cudaSuccess ||
            leg_dev_malloc(reinterpret_cast<void **>(&r->planes[p]), sizeof(__half) * LEG_SPLIT_NF * Bz * pl->Kp) !=
                cudaSuccess)
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
    }
    // tile width of the grouped launch: a tuned choice from LEG_TUNE_CACHE,
    // else the cost model (leg_ragged_autotune times the candidates)
    int tn = 0;
    {
        const char *path = getenv("LEG_TUNE_CACHE");
        int cached = 0;
        if (path && *path && leg_tune_cache_lookup(path, ragged_key(r), &cached, nullptr) && cached >= 16 &&
            cached <= 128 && cached % 16 == 0)
            tn = cached;
        else if ((rc = model_tile(r, &tn)))
            return fail(rc);
    }
    if ((rc = set_tile(r, tn))) return fail(rc);
    if ((rc = upload(&r->d_bk, bk.data(), bk.size()))) return fail(rc);
    if (leg_dev_malloc(&r->status, sizeof(int)) != cudaSuccess || cudaMemset(r->status, 0, sizeof(int)) != cudaSuccess)
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

extern "C" int leg_ragged_forward(leg_ragged_t r, const float *f_packed, float *c_packed, cudaStream_t st)
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

extern "C" int leg_ragged_forward_profiled(leg_ragged_t r, const float *f_packed, float *c_packed, cudaStream_t st,
                                           float *ms)
{
    if (!r) return leg_set_error(LEG_ERR_INVALID_ARG, "ragged batch is NULL");
    if (!ms) return leg_set_error(LEG_ERR_INVALID_ARG, "ms is NULL");
    ms[0] = ms[1] = ms[2] = 0.0f;
    if (r->count == 0) return LEG_OK;
    if (!f_packed || !c_packed) return leg_set_error(LEG_ERR_INVALID_ARG, "null f_packed or c_packed");
    int dev = -1;
    LEG_CUDA_TRY(cudaGetDevice(&dev));
    if (dev != r->device) return leg_set_error(LEG_ERR_INVALID_ARG, "current device differs from the batch's");
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    int rc = LEG_OK;
    for (int i = 0; i < 4 && !rc; ++i)
        if (cudaEventCreate(&ev[i]) != cudaSuccess) rc = leg_set_error(LEG_ERR_CUDA, "event creation failed");
    if (!rc) rc = enqueue(r, f_packed, c_packed, st, ev);
    if (!rc) {
        cudaError_t e = cudaEventSynchronize(ev[3]);
        for (int i = 0; i < 3 && e == cudaSuccess; ++i) e = cudaEventElapsedTime(&ms[i], ev[i], ev[i + 1]);
        if (e != cudaSuccess) rc = leg_set_error(LEG_ERR_CUDA, cudaGetErrorString(e));
    }
    for (int i = 0; i < 4; ++i)
        if (ev[i]) cudaEventDestroy(ev[i]);
    return rc;
}

extern "C" int leg_ragged_set_tile(leg_ragged_t r, int tn)
{
    if (!r) return leg_set_error(LEG_ERR_INVALID_ARG, "ragged batch is NULL");
    if (tn != 0 && (tn < 16 || tn > 128 || tn % 16 != 0))
        return leg_set_error(LEG_ERR_INVALID_ARG, "tile width must be 0 or a multiple of 16 in 16..128");
    int dev = -1;
    LEG_CUDA_TRY(cudaGetDevice(&dev));
    if (dev != r->device) return leg_set_error(LEG_ERR_INVALID_ARG, "current device differs from the batch's");
    int rc;
    if (tn == 0 && (rc = model_tile(r, &tn))) return rc;
    LEG_CUDA_TRY(cudaStreamSynchronize(r->rs));   // d_probs is rewritten below
    return set_tile(r, tn);
}

extern "C" int leg_ragged_tile_info(leg_ragged_t r, int *tn, int *tiles)
{
    if (!r) return leg_set_error(LEG_ERR_INVALID_ARG, "ragged batch is NULL");
    if (tn) *tn = r->tn;
    if (tiles) *tiles = r->ntiles;
    return LEG_OK;
}

extern "C" int leg_ragged_autotune(leg_ragged_t r, const float *f_packed, float *c_packed, cudaStream_t st,
                                   int *tn_out)
{
    if (!r) return leg_set_error(LEG_ERR_INVALID_ARG, "ragged batch is NULL");
    if (r->count > 0 && (!f_packed || !c_packed))
        return leg_set_error(LEG_ERR_INVALID_ARG, "null f_packed or c_packed");
    int dev = -1;
    LEG_CUDA_TRY(cudaGetDevice(&dev));
    if (dev != r->device) return leg_set_error(LEG_ERR_INVALID_ARG, "current device differs from the batch's");
    std::lock_guard<std::mutex> lock(leg_tune_mutex());
    const char *path = getenv("LEG_TUNE_CACHE");
    const std::string key = ragged_key(r);
    int rc;
    int tn = 0;
    LEG_CUDA_TRY(cudaStreamSynchronize(r->rs));
    if (path && *path && leg_tune_cache_lookup(path, key, &tn, nullptr) && tn >= 16 && tn <= 128 && tn % 16 == 0) {
        if ((rc = set_tile(r, tn))) return rc;
    } else if (r->count > 0) {
        int model = 128;
        if ((rc = model_tile(r, &model))) return rc;
        std::vector<int> cand = {model};
        for (int w = 128; w >= 64; w -= 16)
            if (w != model) cand.push_back(w);
        float best = -1.0f;
        int best_tn = model;
        for (int w : cand) {
            if ((rc = set_tile(r, w))) return rc;
            float ms[3];
            std::vector<float> v;
            for (int rep = 0; rep < 4; ++rep) {   // one untimed, three timed
                if ((rc = leg_ragged_forward_profiled(r, f_packed, c_packed, st, ms))) return rc;
                if (rep) v.push_back(ms[1]);
            }
            std::sort(v.begin(), v.end());
            if (best < 0 || v[1] < best * 0.99f) {   // ties stay with the earlier (model) choice
                best = v[1];
                best_tn = w;
            }
        }
        if ((rc = set_tile(r, best_tn))) return rc;
        if (path && *path) leg_tune_cache_store(path, key, best_tn, 0);
    }
    if (tn_out) *tn_out = r->tn;
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

// ---------------------------------------------------------------- one-call form
// leg_forward_ragged takes the per-function arrays on the device, reads them
// back (one small copy and a host synchronisation per call), and keeps the
// batches built from them in a small cache keyed by the device, the plans and
// the arrays' contents, so that repeated calls replay the same graph.
namespace {

struct RaggedCacheEntry {
    int device = -1;
    std::vector<leg_plan *> plans;
    std::vector<int> plan_idx, n_out;
    std::vector<long long> in_off, out_off;
    leg_ragged *batch = nullptr;
    unsigned long long last_use = 0;
};

constexpr size_t LEG_RAGGED_CACHE = 4;   // batches kept by the one-call form
std::mutex g_rc_mutex;
std::vector<RaggedCacheEntry> g_rc;
unsigned long long g_rc_clock = 0;

}  // namespace

// Drops the cached one-call batches that use plan p (called when p is destroyed).
void leg_ragged_forget_plan(const leg_plan *p)
{
    std::lock_guard<std::mutex> lock(g_rc_mutex);
    for (size_t i = 0; i < g_rc.size();) {
        const auto &pl = g_rc[i].plans;
        if (std::find(pl.begin(), pl.end(), p) != pl.end()) {
            leg_ragged_destroy(g_rc[i].batch);
            g_rc.erase(g_rc.begin() + i);
        } else {
            ++i;
        }
    }
}

extern "C" int leg_forward_ragged(const leg_plan_t *plans, int nplans, int count, const int *plan_idx,
                                  const int *n_out, const long long *in_off, const long long *out_off,
                                  const float *f_packed, float *c_packed, cudaStream_t st)
{
    if (!plans || nplans < 1 || nplans > 64) return leg_set_error(LEG_ERR_INVALID_ARG, "need 1..64 plans");
    if (count < 0) return leg_set_error(LEG_ERR_INVALID_ARG, "count < 0");
    if (count == 0) return LEG_OK;
    if (!plan_idx || !n_out || !in_off || !out_off)
        return leg_set_error(LEG_ERR_INVALID_ARG, "null per-function array");
    if (!f_packed || !c_packed) return leg_set_error(LEG_ERR_INVALID_ARG, "null f_packed or c_packed");
    int dev = -1;
    LEG_CUDA_TRY(cudaGetDevice(&dev));
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    LEG_CUDA_TRY(cudaStreamIsCapturing(st, &cs));
    if (cs != cudaStreamCaptureStatusNone)
        return leg_set_error(LEG_ERR_UNSUPPORTED,
                             "leg_forward_ragged reads its arrays on the host; under stream capture use "
                             "leg_ragged_create + leg_ragged_forward");
    RaggedCacheEntry key;
    key.device = dev;
    key.plans.assign(plans, plans + nplans);
    key.plan_idx.resize(count);
    key.n_out.resize(count);
    key.in_off.resize(count);
    key.out_off.resize(count);
    // the arrays as written by the work already on st
    LEG_CUDA_TRY(cudaMemcpyAsync(key.plan_idx.data(), plan_idx, sizeof(int) * count, cudaMemcpyDefault, st));
    LEG_CUDA_TRY(cudaMemcpyAsync(key.n_out.data(), n_out, sizeof(int) * count, cudaMemcpyDefault, st));
    LEG_CUDA_TRY(cudaMemcpyAsync(key.in_off.data(), in_off, sizeof(long long) * count, cudaMemcpyDefault, st));
    LEG_CUDA_TRY(cudaMemcpyAsync(key.out_off.data(), out_off, sizeof(long long) * count, cudaMemcpyDefault, st));
    LEG_CUDA_TRY(cudaStreamSynchronize(st));
    leg_ragged *batch = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_rc_mutex);   // one-call batches are shared by all threads
        for (auto &e : g_rc)
            if (e.device == key.device && e.plans == key.plans && e.plan_idx == key.plan_idx &&
                e.n_out == key.n_out && e.in_off == key.in_off && e.out_off == key.out_off) {
                e.last_use = ++g_rc_clock;
                batch = e.batch;
                break;
            }
        if (!batch) {
            int rc = leg_ragged_create(&batch, plans, nplans, count, key.plan_idx.data(), key.n_out.data(),
                                       key.in_off.data(), key.out_off.data());
            if (rc) return rc;
            if (g_rc.size() >= LEG_RAGGED_CACHE) {
                auto lru = std::min_element(g_rc.begin(), g_rc.end(), [](const RaggedCacheEntry &a,
                                                                         const RaggedCacheEntry &b) {
                    return a.last_use < b.last_use;
                });
                leg_ragged_destroy(lru->batch);
                g_rc.erase(lru);
            }
            key.batch = batch;
            key.last_use = ++g_rc_clock;
            g_rc.push_back(std::move(key));
        }
        // enqueued under the lock: no other thread evicts the batch meanwhile
        return leg_ragged_forward(batch, f_packed, c_packed, st);
    }
}
