// leg_plan_autotune: per-plan choice of the launch parameters that do not
// change results, by timing them on the caller's batch.
//
//   * tile width of the split-FP16 / BF16 tensor-core GEMM (functions per CTA
//     pair tile): the cost model's choice and the multiples of 16 from the
//     plan's maximum down to 64;
//   * transform kernel of the FP64 / double-float FFT stage: the
//     register-tiled real-even transform or the shared-memory Stockham one.
//
// Each candidate runs once untimed and three times timed (CUDA events around
// the stage, on the caller's stream); the fastest median wins and is stored
// in the plan.  With the environment variable LEG_TUNE_CACHE naming a file,
// choices are kept there, one line per (device, dtype, N, M, K, B), and a
// later call with the same key takes the stored choice without timing.
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <string>
#include <vector>

#include "leg_internal.cuh"

namespace {

std::mutex g_tune_mutex;

std::string tune_key(const leg_plan *p, int B)
{
    cudaDeviceProp prop;
    std::string dev = "gpu";
    if (cudaGetDeviceProperties(&prop, p->device) == cudaSuccess) dev = prop.name;
    for (auto &ch : dev)
        if (ch == ' ' || ch == '|') ch = '_';
    char buf[256];
    snprintf(buf, sizeof(buf), "%s|%d|%d|%d|%d|%d|%d", dev.c_str(), p->dtype, p->N, p->M, p->K, p->Q, B);
    return buf;
}

bool cache_lookup(const char *path, const std::string &key, int *tn, int *fft)
{
    FILE *fp = fopen(path, "r");
    if (!fp) return false;
    char line[512];
    bool found = false;
    while (fgets(line, sizeof(line), fp)) {
        char k[400];
        int a = 0, b = 0;
        if (sscanf(line, "%399s %d %d", k, &a, &b) == 3 && key == k) {
            *tn = a;
            *fft = b;
            found = true;   // the last matching line wins
        }
    }
    fclose(fp);
    return found;
}

void cache_store(const char *path, const std::string &key, int tn, int fft)
{
    FILE *fp = fopen(path, "a");
    if (!fp) return;
    fprintf(fp, "%s %d %d\n", key.c_str(), tn, fft);
    fclose(fp);
}

// Median of `reps` timings of stage `stage` (0 split, 1 GEMM, 2 FFT) of the forward pass.
int time_stage(leg_plan *p, const void *f, void *c, int B, cudaStream_t st, int stage, int reps, float *out)
{
    float ms[3];
    int rc = leg_forward_profiled(p, f, c, B, st, ms);   // untimed warm-up
    if (rc) return rc;
    std::vector<float> v;
    for (int r = 0; r < reps; ++r) {
        if ((rc = leg_forward_profiled(p, f, c, B, st, ms))) return rc;
        v.push_back(ms[stage]);
    }
    std::sort(v.begin(), v.end());
    *out = v[v.size() / 2];
    return LEG_OK;
}

}  // namespace

extern "C" int leg_plan_autotune(leg_plan_t p, const void *f, void *c, int B, cudaStream_t st, int *tn_out,
                                 int *fft_out)
{
    if (!p) return leg_set_error(LEG_ERR_INVALID_ARG, "plan is NULL");
    if (B < 1) return leg_set_error(LEG_ERR_INVALID_ARG, "B < 1");
    if (!f || !c) return leg_set_error(LEG_ERR_INVALID_ARG, "null f or c");
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    const char *path = getenv("LEG_TUNE_CACHE");
    const std::string key = tune_key(p, B);
    int tn = p->tn, fft = p->fft_variant;
    if (path && *path && cache_lookup(path, key, &tn, &fft)) {
        p->tn = tn;
        p->fft_variant = fft;
    } else {
        int rc;
        const bool tc = (p->dtype == LEG_SPLIT_FP16 || p->dtype == LEG_BF16);
        if (tc) {
            const int maxtn = (p->dtype == LEG_BF16) ? 256 : 128;
            std::vector<int> cand = {0};
            for (int w = maxtn; w >= 64; w -= 16) cand.push_back(w);
            float best = -1.0f;
            int best_tn = 0;
            for (int w : cand) {
                p->tn = w;
                float t;
                if ((rc = time_stage(p, f, c, B, st, 1, 3, &t))) {
                    p->tn = 0;
                    return rc;
                }
                if (best < 0 || t < best * 0.99f) {   // ties stay with the earlier (model, wider) choice
                    best = t;
                    best_tn = w;
                }
            }
            p->tn = best_tn;
        }
        if ((p->dtype == LEG_SPLIT_FP16 || p->dtype == LEG_F64) && !p->collapsed()) {   // collapsed: no transform
            float t0 = 0.0f, t1 = 0.0f;
            p->fft_variant = 0;
            if ((rc = time_stage(p, f, c, B, st, 2, 3, &t0))) return rc;
            p->fft_variant = 1;
            if ((rc = time_stage(p, f, c, B, st, 2, 3, &t1))) {
                p->fft_variant = 0;
                return rc;
            }
            p->fft_variant = (t1 < t0 * 0.99f) ? 1 : 0;
        }
        if (path && *path) cache_store(path, key, p->tn, p->fft_variant);
    }
    if (tn_out) *tn_out = p->tn;
    if (fft_out) *fft_out = p->fft_variant;
    return LEG_OK;
}
