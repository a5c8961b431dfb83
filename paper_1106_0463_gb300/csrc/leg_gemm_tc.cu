// Tensor-core (tcgen05) Abel GEMMs for sm_103a.
//
// The Abel step of the method (arXiv:1106.0463, Eq. 2.5 evaluated by the
// quadrature of Sec. 2 after Eq. 2.14) is, for a batch of sampled functions,
// the dense product  G[b, j] = sum_k A[j, k] F[b, k]  (rows j = 0..M/2 of the
// grid y_j = 2 pi j/M, K Chebyshev-Lobatto samples).  Its result is
// differenced and scaled by (2n+1) in the FFT stage, which turns white
// rounding noise in G into errors ~ (2N/sqrt(M)) times larger in c_n; FP32
// accumulation of the whole product therefore cannot meet 1e-6.
//
// LEG_SPLIT_FP16 (three-slice split, eight products, three accumulators):
//   each operand row is scaled by a power of two (the operator by its L1
//   norm, the input by its max-norm) and split into FP16 slices, with the
//   plan's slice width s (8 for K <= 1025, else 7; leg_split_fbits) and
//   abits = 23 - s:
//     a = A0 + 2^-s A1 + 2^-2s A2s,     A0 on a 2^-abits grid,
//     f = F0 + 2^-s r,  r = F1 + (r - F1),   F0 on a 2^-s grid.
//   acc0 takes A0 F0 over the whole tile: the products lie on a 2^-23 grid
//   and every partial sum stays below 2, so it is EXACT in FP32 whatever the
//   order or truncation of the tensor core's additions.
//   acc1 (weight 2^-s) takes the two largest correction terms A1 F0 + A0 F1
//   in K chunks of 128: after each chunk the epilogue warps add it into
//   registers and release its TMEM buffer (two buffers), which bounds the
//   tensor core's truncating FP32 accumulation (its error grows with the
//   chunk's length and magnitude).
//   acc2 (weight 2^-s as well, whole tile) takes the small terms through input
//   planes pre-scaled by 2^-s or 2^-2s: A0 (r - F1), A1 2^-s F1, A2s 2^-s F0
//   (weight 2^-2s) and A2s 2^-2s F1, A1 2^-s (r - F1) (weight 2^-3s); below
//   the FP16 normal range the pre-scaled planes keep an absolute 2^-25, which
//   the L1-normalised rows bound by 2^-32 in G.  Only A2s (r - F1) (weight
//   2^-4s) is dropped.
//   The epilogue forms G = 2^(e_j + e_b) (acc0 + 2^-s (acc1 + acc2)) as a
//   double-float pair.
// LEG_BF16: one BF16 product, one accumulator (FP32 G).
//
// Kernel: persistent, CTA pairs (cluster of 2, tcgen05 cta_group::2).  A pair
// tile is 256 operator rows (MMA M; 128 per CTA = its TMEM lanes) by tn
// functions (MMA N, a multiple of 16 up to 128 for the split path and 256 for
// BF16; each CTA stages tn/2 of them), and K advances in blocks of 32 (one
// 64-byte swizzle row of FP16).
//   warp 0         TMA producer (each CTA): its operator tiles (128 rows) and
//                  input tiles (tn/2 rows) of a K block into one of the stages;
//                  the copies of both CTAs complete on the even CTA's full
//                  barrier (cta_group::2 TMA);
//   warp 1         even CTA: issues the pair MMAs (M=256, N=tn, K=16) once a
//                  stage is full, commits each stage back to both producers
//                  and each finished chunk / tile to both epilogues (multicast
//                  commits); odd CTA: idle after the TMEM allocation;
//                  (the producer and MMA loops run on the whole warp, so that
//                  descriptors and coordinates stay warp-uniform; one elected
//                  lane issues the TMA, MMA and commit instructions)
//   warps 2..17    epilogue (each CTA, own TMEM lanes): chunk promotion into
//                  registers, then scaling and double-float stores.
// TMEM (split path): acc0 in columns [0, tn), acc2 in [tn, 2tn), acc1 chunk
// buffer b in [(2 + b) tn, (3 + b) tn); the MMAs of one chunk overlap the
// promotion of the previous one.  BF16: one accumulator in [0, tn).  The
// epilogue copies acc0 and acc2 to registers and releases the tile's TMEM
// before its global stores, so the next tile's MMAs overlap them.  Every wait
// is bounded by a cycle limit; on expiry the kernel records LEG_ERR_TIMEOUT in
// the status word, tells the other CTA of the pair, drains its own TMA copies
// and MMAs (again bounded), releases TMEM and returns.
#include <stdio.h>
#include <string.h>

#include <mutex>

#include "leg_fft.cuh"
#include "leg_internal.cuh"
#include "leg_sm100.cuh"
#include "leg_split.cuh"

namespace {

constexpr int CTA_M = 128;                          // operator rows per CTA (TMEM lanes)
constexpr int PAIR_M = 2 * CTA_M;                   // MMA M of a CTA pair
constexpr int TILE_K = 32;                          // K per stage: 64-byte FP16 rows
constexpr int ATILE_BYTES = CTA_M * TILE_K * 2;     // 8 KB per operator plane
constexpr int CHUNK_KB = 4;                         // K blocks per accumulation chunk of acc1
constexpr int MAX_STAGES = 8;
constexpr int EPI_WARPS = 16;                       // four per TMEM lane quadrant
constexpr int THREADS = 64 + 32 * EPI_WARPS;
constexpr uint32_t TMEM_COLS = 512;
constexpr size_t SMEM_LIMIT = 232448;               // opt-in shared memory per block
constexpr size_t SMEM_STATIC_RESERVE = 1024 + 512;  // 1 KB alignment slack + static barriers
constexpr long long DRAIN_LIMIT = 4000000000LL;     // cycles, teardown waits

template <int NPROD> struct TcCfg;
template <> struct TcCfg<8> {
    static constexpr int NA = LEG_SPLIT_NA, NF = LEG_SPLIT_NF, BF16 = 0;
};
template <> struct TcCfg<1> {
    static constexpr int NA = 1, NF = 1, BF16 = 1;
};

// Stage layout of a launch with tiles tn functions wide: NA operator tiles
// (128 rows x 32 K each), then NF input tiles (tn/2 rows x 32 K each), 64-byte
// swizzled rows; a stage spans a multiple of 1 KB.
__host__ __device__ constexpr int ftile_bytes(int tn) { return (tn / 2) * TILE_K * 2; }

template <int NPROD>
__host__ __device__ constexpr int stage_bytes(int tn)
{
    return (TcCfg<NPROD>::NA * ATILE_BYTES + TcCfg<NPROD>::NF * ftile_bytes(tn) + 1023) / 1024 * 1024;
}

template <int NPROD>
constexpr int stages_for(int tn)
{
    const int s = (int)((SMEM_LIMIT - SMEM_STATIC_RESERVE) / (size_t)stage_bytes<NPROD>(tn));
    return s > MAX_STAGES ? MAX_STAGES : s;
}

// Maximum tile width of a launch: the split path keeps four tn-wide TMEM
// regions (acc0, acc2, two acc1 chunk buffers), the BF16 path one.
template <int NPROD> __host__ __device__ constexpr int max_tn() { return NPROD > 1 ? 128 : 256; }

// TMEM columns of the split path: acc0 [0, tn), acc2 [tn, 2tn) for the whole
// tile; acc1 chunk buffer b in [(2 + b) tn, (3 + b) tn).
__device__ __forceinline__ uint32_t acc1_col(int tn, int b) { return (uint32_t)(tn * (2 + b)); }

// Pair tile t of a launch: its problem, first operator row j0, first function b0.
// The tiles of a problem are ordered so that the pairs running at the same time
// share the larger operand's tiles in L2: row tiles vary fastest when the input
// planes outweigh the operator planes (each input tile is then read from DRAM
// once), function tiles when the operator does (each operator tile is read
// once while the input planes stay in L2).
__device__ __forceinline__ const TcProblem &tile_problem(const TcProblem &single, const TcProblem *multi,
                                                         int nprob, int t, int tn, int &j0, int &b0)
{
    const TcProblem *pr = &single;
    int lt = t;
    if (multi) {
        int p = 0;
        while (p + 1 < nprob && t >= multi[p + 1].tile0) ++p;
        pr = &multi[p];
        lt = t - pr->tile0;
    }
    if (pr->fn_fast) {
        b0 = (lt % pr->ntn) * tn;
        j0 = (lt / pr->ntn) * PAIR_M;
    } else {
        j0 = (lt % pr->ntm) * PAIR_M;
        b0 = (lt / pr->ntm) * tn;
    }
    return *pr;
}

// x 2^e: one exact multiply for normal powers of two, ldexpf beyond.
__device__ __forceinline__ float scale2(float x, int e)
{
    return (e >= -126 && e <= 127) ? x * __int_as_float((e + 127) << 23) : ldexpf(x, e);
}

// Warp-uniform bounded wait: lane 0 polls, the outcome is broadcast.
__device__ __forceinline__ bool warp_wait(uint64_t *bar, uint32_t parity, long long limit,
                                          const volatile int *abort_flag)
{
    int ok = 0;
    if ((threadIdx.x & 31) == 0) ok = sm100::mbar_wait_ab(bar, parity, limit, abort_flag) ? 1 : 0;
    return __shfl_sync(0xffffffffu, ok, 0) != 0;
}

// tn: functions per pair tile (multiple of 16, <= max_tn; every problem of the
// launch uses it); stages: pipeline depth (<= MAX_STAGES, fits stage_bytes(tn)).
template <int NPROD, bool OUT_DF>
__global__ void __launch_bounds__(THREADS, 1) tc_gemm_kernel(const __grid_constant__ TcProblem single,
                                                         const TcProblem *__restrict__ multi, int nprob,
                                                         int ntiles, int tn, int stages, int *status,
                                                         long long wait_limit)
{
    using Cfg = TcCfg<NPROD>;
    constexpr int NA = Cfg::NA, NF = Cfg::NF;
    const int FT = ftile_bytes(tn);
    const int SB = stage_bytes<NPROD>(tn);

    extern __shared__ unsigned char smem_raw[];
    unsigned char *smem = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));   // swizzle atoms need 512 B
    __shared__ __align__(8) uint64_t full_bar[MAX_STAGES];    // (even CTA) both CTAs' copies of a stage landed
    __shared__ __align__(8) uint64_t empty_bar[MAX_STAGES];   // the pair MMAs reading a stage completed
    __shared__ __align__(8) uint64_t chunk_full[2];           // an acc1 chunk is final
    __shared__ __align__(8) uint64_t chunk_empty[2];          // (even CTA) both epilogues have read it
    __shared__ __align__(8) uint64_t acc_full;                // acc0 (and acc2) of a tile are final
    __shared__ __align__(8) uint64_t acc_empty;               // (even CTA) both epilogues have read them
    __shared__ __align__(8) uint64_t drain_bar;
    __shared__ uint32_t tmem_slot;
    __shared__ volatile int s_abort;
    __shared__ volatile uint32_t s_peer_issued;               // (even CTA) copies issued by the odd CTA

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t rank = sm100::cluster_ctarank();   // 0: MMA issuer of the pair
    const int cid = blockIdx.x >> 1, ncl = gridDim.x >> 1;

    if (threadIdx.x == 0) {
        for (int s = 0; s < MAX_STAGES; ++s) {
            sm100::mbar_init(&full_bar[s], 1);
            sm100::mbar_init(&empty_bar[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            sm100::mbar_init(&chunk_full[b], 1);
            sm100::mbar_init(&chunk_empty[b], 2 * EPI_WARPS);
        }
        sm100::mbar_init(&acc_full, 1);
        sm100::mbar_init(&acc_empty, 2 * EPI_WARPS);
        sm100::mbar_init(&drain_bar, 1);
        s_abort = 0;
        s_peer_issued = 0;
        sm100::fence_mbar_init();
        if (!multi) {
            sm100::prefetch_tmap(&single.a);
            sm100::prefetch_tmap(&single.f);
        }
    }
    if (warp == 1) {
        sm100::tmem_alloc_pair(&tmem_slot, TMEM_COLS);
        sm100::tc_fence_before();
    }
    sm100::cluster_sync();
    sm100::tc_fence_after();
    const uint32_t tmem = tmem_slot;
    // launched as a dependent of the input split: the setup above overlaps its
    // tail; the inputs (planes, scales) and the output are touched only below
    leg_griddep_wait();
    leg_griddep_trigger();

    const uint32_t peer_abort = sm100::mapa_shared(sm100::smem_u32(const_cast<int *>(&s_abort)), rank ^ 1u);
    auto fail = [&]() {
        atomicOr(status, 1);
        s_abort = 1;
        sm100::st_cluster_u32(peer_abort, 1u);
    };
    const uint32_t bytes = NA * ATILE_BYTES + NF * FT;   // one CTA's copies per stage
    uint32_t issued = 0;                                  // producer: stages issued (lane 0 of warp 0)

    if (warp == 0) {
        // ------------------------------------------------ TMA producer warp (both CTAs)
        // Both CTAs' copies of a stage complete on the even CTA's full barrier,
        // which the even producer arms with both CTAs' byte counts.
        const bool leader = sm100::elect_one();
        const uint32_t full0 = sm100::mapa_shared(sm100::smem_u32(&full_bar[0]), 0u);
        uint32_t s = 0, ph = 0;
        bool ok = true;
        const int half = tn >> 1;
        for (int t = cid; ok && t < ntiles; t += ncl) {
            int j0, b0;
            const TcProblem &pr = tile_problem(single, multi, nprob, t, tn, j0, b0);
            const int arow = j0 + (int)rank * CTA_M, frow = b0 + (int)rank * half;
            for (int kb = 0; kb < pr.nkb; ++kb) {
                if (!warp_wait(&empty_bar[s], ph ^ 1, wait_limit, &s_abort)) {
                    ok = false;
                    break;
                }
                if (leader) {
                    unsigned char *st = smem + s * SB;
                    const uint32_t fb = full0 + 8u * s;
                    if (rank == 0) sm100::mbar_arrive_expect_tx(&full_bar[s], 2 * bytes);
#pragma unroll
                    for (int p = 0; p < NA; ++p)
                        sm100::tma_load_3d_pair(st + p * ATILE_BYTES, &pr.a, fb, kb * TILE_K, arow, p);
#pragma unroll
                    for (int p = 0; p < NF; ++p)
                        sm100::tma_load_3d_pair(st + NA * ATILE_BYTES + p * FT, &pr.f, fb, kb * TILE_K, frow, p);
                }
                __syncwarp();
                ++issued;
                if (++s == (uint32_t)stages) {
                    s = 0;
                    ph ^= 1;
                }
            }
        }
        if (!ok && lane == 0) fail();
        if (lane == 0 && rank == 1)   // the even CTA reconciles and drains both CTAs' copies
            sm100::st_cluster_u32(sm100::mapa_shared(sm100::smem_u32(const_cast<uint32_t *>(&s_peer_issued)), 0u),
                                  issued);
    } else if (warp == 1 && rank == 0) {
        // ------------------------------------------------ MMA warp (even CTA)
        const bool leader = sm100::elect_one();
        const int nbuf = 2;
        uint32_t s = 0, ph = 0, cc = 0;   // stage ring position, acc1 chunk counter
        bool ok = true;
        const uint32_t idesc = sm100::idesc_f16(PAIR_M, tn, Cfg::BF16);
        int ti = 0;
        for (int t = cid; ok && t < ntiles; t += ncl, ++ti) {
            int j0, b0;
            const TcProblem &pr = tile_problem(single, multi, nprob, t, tn, j0, b0);
            // acc0 / acc2 of the previous tile have been read by both epilogues
            if (!warp_wait(&acc_empty, (ti & 1) ^ 1, wait_limit, &s_abort)) {
                ok = false;
                break;
            }
            sm100::tc_fence_after();
            const uint32_t acc2 = tmem + (uint32_t)tn;
            uint32_t acc1 = tmem + acc1_col(tn, 0);
            for (int kb = 0; kb < pr.nkb; ++kb) {
                if (!warp_wait(&full_bar[s], ph, wait_limit, &s_abort)) {
                    ok = false;
                    break;
                }
                sm100::tc_fence_after();
                // descriptors: the stage base once, planes and K-steps as offsets
                // of the 16-byte address field (addresses stay below 2^18)
                const uint64_t d0 = sm100::desc_k_sw64(sm100::smem_u32(smem + s * SB));
                auto A = [&](int p, int kk) { return d0 + (uint64_t)((p * ATILE_BYTES + kk * 32) >> 4); };
                auto F = [&](int p, int kk) { return d0 + (uint64_t)((NA * ATILE_BYTES + p * FT + kk * 32) >> 4); };
                const uint32_t first = (kb == 0) ? 0u : 1u;   // first K block of the tile
                if (leader) {
#pragma unroll
                    for (int kk = 0; kk < TILE_K / 16; ++kk) {
                        // acc0 (weight 1): A0 F0, whole tile, exact
                        sm100::mma_f16_pair(tmem, A(0, kk), F(0, kk), idesc, (first | kk) ? 1u : 0u);
                        if constexpr (NPROD > 1) {
                            // acc2 (weight 2^-s): the terms of weight 2^-2s and 2^-3s through
                            // the pre-scaled input planes, whole tile
                            sm100::mma_f16_pair(acc2, A(0, kk), F(2, kk), idesc, (first | kk) ? 1u : 0u);   // A0 (r - F1)
                            sm100::mma_f16_pair(acc2, A(1, kk), F(3, kk), idesc, 1u);   // A1 2^-s F1
                            sm100::mma_f16_pair(acc2, A(2, kk), F(4, kk), idesc, 1u);   // A2s 2^-s F0
                            sm100::mma_f16_pair(acc2, A(2, kk), F(5, kk), idesc, 1u);   // A2s 2^-2s F1
                            sm100::mma_f16_pair(acc2, A(1, kk), F(6, kk), idesc, 1u);   // A1 2^-s (r - F1)
                        }
                    }
                }
                if constexpr (NPROD > 1) {
                    const int kc = kb % CHUNK_KB;
                    if (kc == 0) {   // a new acc1 chunk: its buffer must have been read
                        const uint32_t b = cc % nbuf, u = cc / nbuf;
                        if (!warp_wait(&chunk_empty[b], (u & 1) ^ 1, wait_limit, &s_abort)) {
                            ok = false;
                            break;
                        }
                        sm100::tc_fence_after();
                        acc1 = tmem + acc1_col(tn, (int)b);
                    }
                    if (leader) {
#pragma unroll
                        for (int kk = 0; kk < TILE_K / 16; ++kk) {
                            // acc1 (weight 2^-s): the two largest products, in K chunks
                            sm100::mma_f16_pair(acc1, A(1, kk), F(0, kk), idesc, (kc == 0 && kk == 0) ? 0u : 1u);  // A1 F0
                            sm100::mma_f16_pair(acc1, A(0, kk), F(1, kk), idesc, 1u);   // A0 F1
                        }
                        sm100::mma_commit_pair_mc(&empty_bar[s], 0x3);
                        if (kc == CHUNK_KB - 1 || kb == pr.nkb - 1) sm100::mma_commit_pair_mc(&chunk_full[cc % nbuf], 0x3);
                    }
                    if (kc == CHUNK_KB - 1 || kb == pr.nkb - 1) ++cc;
                } else {
                    if (leader) sm100::mma_commit_pair_mc(&empty_bar[s], 0x3);
                }
                __syncwarp();
                if (++s == (uint32_t)stages) {
                    s = 0;
                    ph ^= 1;
                }
            }
            if (!ok) break;
            if (leader) sm100::mma_commit_pair_mc(&acc_full, 0x3);
            __syncwarp();
        }
        if (leader) {
            if (!ok) fail();
            // every MMA issued by this lane has completed before TMEM is released
            sm100::mma_commit_pair_mc(&drain_bar, 0x1);
            sm100::mbar_wait(&drain_bar, 0, DRAIN_LIMIT);
        }
    } else if (warp >= 2) {
        // ------------------------------------------------ epilogue (both CTAs)
        // Warp (quadrant q, group cg) owns TMEM lanes 32q.. (operator rows) and the
        // 16-column units cg, cg + 4, cg + 8, cg + 12 below tn (functions).
        const int q = warp & 3;
        const int cg = (warp - 2) >> 2;
        const uint32_t lane_base = tmem + ((uint32_t)(q * 32) << 16);
        const uint32_t chunk_empty0 = sm100::mapa_shared(sm100::smem_u32(&chunk_empty[0]), 0u);
        const uint32_t acc_empty0 = sm100::mapa_shared(sm100::smem_u32(&acc_empty), 0u);
        const int nunits = tn >> 4;
        constexpr int MU = max_tn<NPROD>() / 64;        // units per warp, at most
        uint32_t cc = 0;
        int ti = 0;
        bool ok = true;
        for (int t = cid; ok && t < ntiles; t += ncl, ++ti) {
            int j0, b0;
            const TcProblem &pr = tile_problem(single, multi, nprob, t, tn, j0, b0);
            // per-function scales of this warp's columns: lane l holds unit m's
            // column (l & 15); fetched before the accumulators are ready
            int fe[MU];
#pragma unroll
            for (int m = 0; m < MU; ++m) {
                fe[m] = 0;
                const int bi = b0 + (cg + 4 * m) * 16 + (lane & 15);
                if (NPROD > 1 && pr.fexp && cg + 4 * m < nunits && bi < pr.B) fe[m] = pr.fexp[bi];
            }
            float r1[16 * MU];
#pragma unroll
            for (int i = 0; i < 16 * MU; ++i) r1[i] = 0.0f;
            if constexpr (NPROD > 1) {
                const int nch = (pr.nkb + CHUNK_KB - 1) / CHUNK_KB;
                for (int ch = 0; ch < nch; ++ch, ++cc) {
                    const uint32_t b = cc % 2, u = cc / 2;
                    if (!warp_wait(&chunk_full[b], u & 1, wait_limit, &s_abort)) {
                        ok = false;
                        break;
                    }
                    __syncwarp();
                    sm100::tc_fence_after();
                    const uint32_t base = lane_base + acc1_col(tn, (int)b);
#pragma unroll
                    for (int m = 0; m < MU; ++m) {
                        if (cg + 4 * m < nunits) {
                            float tv[16];
                            sm100::tmem_ld_32x32b_x16(base + (uint32_t)((cg + 4 * m) * 16), tv);
                            sm100::tmem_ld_wait();
#pragma unroll
                            for (int i = 0; i < 16; ++i) r1[16 * m + i] += tv[i];
                        }
                    }
                    sm100::tc_fence_before();
                    __syncwarp();
                    if (lane == 0) sm100::mbar_arrive_cluster(chunk_empty0 + 8u * b);
                }
                if (!ok) break;
            }
            if (!warp_wait(&acc_full, ti & 1, wait_limit, &s_abort)) {
                ok = false;
                break;
            }
            __syncwarp();
            sm100::tc_fence_after();
            // acc0 (and acc2, folded into r1) into registers, then release TMEM
            // before the stores: the MMA warp starts the next tile meanwhile
            float a0[16 * MU];
#pragma unroll
            for (int m = 0; m < MU; ++m) {
                if (cg + 4 * m >= nunits) continue;
                const uint32_t col = (uint32_t)((cg + 4 * m) * 16);
                float tv[16];
                sm100::tmem_ld_32x32b_x16(lane_base + col, tv);
                if constexpr (NPROD > 1) {
                    float t2[16];
                    sm100::tmem_ld_32x32b_x16(lane_base + (uint32_t)tn + col, t2);
                    sm100::tmem_ld_wait();
#pragma unroll
                    for (int i = 0; i < 16; ++i) r1[16 * m + i] += t2[i];
                } else {
                    sm100::tmem_ld_wait();
                }
#pragma unroll
                for (int i = 0; i < 16; ++i) a0[16 * m + i] = tv[i];
            }
            sm100::tc_fence_before();
            __syncwarp();
            if (lane == 0) sm100::mbar_arrive_cluster(acc_empty0);

            const int j = j0 + (int)rank * CTA_M + q * 32 + lane;
            const bool row_ok = j < pr.rows;
            const int ej = (row_ok && pr.aexp) ? pr.aexp[j] : 0;
#pragma unroll
            for (int m = 0; m < MU; ++m) {
                if (cg + 4 * m >= nunits) continue;
                const int bb = b0 + (cg + 4 * m) * 16;
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    const int e = ej + __shfl_sync(0xffffffffu, fe[m], i);
                    const int bi = bb + i;
                    if (!row_ok || bi >= pr.B) continue;
                    const size_t o = (size_t)bi * pr.ldo + j;
                    if constexpr (NPROD == 1) {
                        static_cast<float *>(pr.out)[o] = a0[16 * m + i];
                    } else if constexpr (OUT_DF) {
                        const dfl sm = df_two_sum(a0[16 * m + i], r1[16 * m + i] * pr.w1);
                        static_cast<float2 *>(pr.out)[o] = make_float2(scale2(sm.hi, e), scale2(sm.lo, e));
                    } else {
                        static_cast<float *>(pr.out)[o] = scale2(fmaf(r1[16 * m + i], pr.w1, a0[16 * m + i]), e);
                    }
                }
            }
        }
        if (!ok && lane == 0) fail();
    }
    __syncwarp();
    sm100::tc_fence_before();
    sm100::cluster_sync();   // every role of both CTAs has stopped issuing
    if (rank == 0 && warp == 0 && lane == 0) {
        // Drain both CTAs' copies.  After an abort the two producers may have
        // issued different numbers of stages (at most `stages` apart): stages
        // the even CTA armed but the odd one never loaded have their missing
        // bytes cancelled, stages only the odd CTA loaded are armed for its bytes.
        const uint32_t mine = issued, peer = s_peer_issued;
        const uint32_t lo = mine < peer ? mine : peer, hi = mine < peer ? peer : mine;
        for (uint32_t i = lo; i < hi; ++i) {
            uint64_t *fb = &full_bar[i % stages];
            if (i < mine) sm100::mbar_complete_tx(fb, bytes);
            else sm100::mbar_arrive_expect_tx(fb, bytes);
        }
        const uint32_t first = hi > (uint32_t)stages ? hi - stages : 0;
        for (uint32_t i = first; i < hi; ++i)
            sm100::mbar_wait(&full_bar[i % stages], (i / stages) & 1, DRAIN_LIMIT);
    }
    sm100::cluster_sync();   // the odd CTA's shared memory outlives its copies
    if (warp == 1) {
        sm100::tc_fence_after();
        sm100::tmem_dealloc_pair(tmem, TMEM_COLS);
    }
}

// ---------------------------------------------------------------- input split
// One CTA per row (the scale and planes of leg_split.cuh, s = in.fbits).
// Input FP32 (forward) or a double-float pair (adjoint).  g0 (forward only):
// row 0 of G, a00 * x[0] as a double-float pair (the operator's row 0 is
// a00 e_0).
constexpr int SPLIT_THREADS = 128;   // one CTA per row
constexpr int SPLIT_U = 16;          // loads in flight per thread in the max reduction

// The CTA splits one row: n values, zero-padded to np (a multiple of 8).
// Pass 1 reduces max |x| with coalesced loads (SPLIT_U in flight per thread)
// and, with STAGE, keeps the row in shared memory (n values of T); pass 2
// handles 8 consecutive elements per thread, read back from shared memory
// (or again from global memory without STAGE), and writes each plane's 8 FP16
// values as one 16-byte store.
template <class T, bool STAGE, int NT = SPLIT_THREADS>
__device__ __forceinline__ void split_row(const T *__restrict__ row, int n, int np, __half *__restrict__ P,
                                          size_t pstride, int *__restrict__ xexp, float2 *g0, float2 a00, int fbits)
{
    const float SC = __int_as_float((127 + fbits) << 23), ISC = __int_as_float((127 - fbits) << 23);
    __shared__ float red[NT / 32];
    __shared__ int s_e;
    extern __shared__ __align__(16) unsigned char split_smem[];
    T *xs = reinterpret_cast<T *>(split_smem);   // STAGE: np values, zero beyond n
    float m = 0.0f;
    for (int base = 0; base < np; base += NT * SPLIT_U) {
        T t[SPLIT_U];
#pragma unroll
        for (int u = 0; u < SPLIT_U; ++u) {
            const int k = base + u * NT + threadIdx.x;
            t[u] = (k < n) ? row[k] : zero_of<T>();
        }
#pragma unroll
        for (int u = 0; u < SPLIT_U; ++u) {
            m = fmaxf(m, fabsf(hi_of(t[u])));
            const int k = base + u * NT + threadIdx.x;
            if (STAGE && k < np) xs[k] = t[u];
        }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, off));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        float mm = 0.0f;
        for (int w = 0; w < NT / 32; ++w) mm = fmaxf(mm, red[w]);
        const int e = split_scale_exp(mm);
        s_e = e;
        *xexp = e;
    }
    __syncthreads();
    const int e = s_e;
    if (g0 && threadIdx.x == 32) *g0 = split_g0(hi_of(STAGE ? xs[0] : row[0]), a00);
    for (int c = threadIdx.x; c < np / 8; c += NT) {
        T v[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int k = 8 * c + i;
            v[i] = zero_of<T>();
            if (STAGE) v[i] = xs[k];                 // zero-padded: no bound check
            else if (k < n) v[i] = row[k];
        }
        split_planes8<T>(v, e, SC, ISC, P + 8 * c, pstride);
    }
}

template <class T, bool STAGE, int NT>
__global__ void __launch_bounds__(NT) split_rows_kernel(const T *__restrict__ x, int ldx, int n, int np,
                                                        LegSplitIn in, float2 *G, int ldg, float2 a00)
{
    const int b = blockIdx.x;
    split_row<T, STAGE, NT>(x + (size_t)b * ldx, n, np, in.base + (size_t)b * in.ld, in.pstride, in.fexp + b,
                        G ? G + (size_t)b * ldg : nullptr, a00, in.fbits);
    leg_griddep_trigger();   // after this CTA's stores: the GEMM's setup may start
}

// Ragged batch: function i (one CTA) goes to row row[i] of bucket bucket[i];
// with STAGE the dynamic shared memory holds the longest row.
template <bool STAGE>
__global__ void __launch_bounds__(SPLIT_THREADS) split_ragged_kernel(const float *__restrict__ f_packed,
                                                                     const long long *__restrict__ in_off,
                                                                     const int *__restrict__ bucket,
                                                                     const int *__restrict__ row,
                                                                     const LegRaggedBucket *__restrict__ bk)
{
    const int i = blockIdx.x;
    const LegRaggedBucket &b = bk[bucket[i]];
    const int r = row[i];
    split_row<float, STAGE>(f_packed + in_off[i], b.K, b.Kp, b.in.base + (size_t)r * b.in.ld, b.in.pstride,
                           b.in.fexp + r, b.G + (size_t)r * b.ldg, b.a00, b.in.fbits);
    leg_griddep_trigger();
}

// Rows of at most this many bytes are staged in shared memory by the split
// (below the 48 KB a CTA gets without opting in).
constexpr size_t SPLIT_STAGE_MAX = 40960;
// Rows of at least this many (padded) elements are split by CTAs of
// SPLIT_THREADS_LONG threads: with one CTA per row, a batch of a few hundred
// long rows leaves the SMs too few loads in flight at 128 threads.
constexpr int SPLIT_LONG_NP = 4096;
constexpr int SPLIT_THREADS_LONG = 512;

template <class T, int NT>
void split_rows_launch(const T *x, int ldx, int n, int np, const LegSplitIn &in, float2 *G, int ldg, float2 a00p,
                       int B, cudaStream_t st)
{
    const size_t bytes = ((size_t)np * sizeof(T) + 15) / 16 * 16;
    if (bytes <= SPLIT_STAGE_MAX)
        split_rows_kernel<T, true, NT><<<B, NT, bytes, st>>>(x, ldx, n, np, in, G, ldg, a00p);
    else
        split_rows_kernel<T, false, NT><<<B, NT, 0, st>>>(x, ldx, n, np, in, G, ldg, a00p);
}

// FP32 rows of at least SPLIT_LONG_NP elements whose padded length splits into
// SPLIT_CL segments of whole 8-element groups go to clusters of SPLIT_CL CTAs.
template <class T>
int split_rows(const T *x, int ldx, int n, int np, const LegSplitIn &in, float2 *G, int ldg, double a00, int B,
               cudaStream_t st)
{
    if (B == 0) return LEG_OK;
    const float ah = (float)a00;
    const float2 a00p = make_float2(ah, (float)(a00 - (double)ah));
    if (np >= SPLIT_LONG_NP)
        split_rows_launch<T, SPLIT_THREADS_LONG>(x, ldx, n, np, in, G, ldg, a00p, B, st);
    else
        split_rows_launch<T, SPLIT_THREADS>(x, ldx, n, np, in, G, ldg, a00p, B, st);
    LEG_LAUNCH_CHECK("split_rows_kernel");
    return LEG_OK;
}

__global__ void __launch_bounds__(256) bf16_rows_kernel(const float *__restrict__ x, int n, int np,
                                                        __nv_bfloat16 *__restrict__ X)
{
    const int b = blockIdx.x;
    for (int k = threadIdx.x; k < np; k += blockDim.x)
        X[(size_t)b * np + k] = __float2bfloat16_rn(k < n ? x[(size_t)b * n + k] : 0.0f);
}

// Transposed split planes of the operator for the adjoint GEMM: row k of the
// result is column k of A (j = 0..rows-1, zero-padded to npr), scaled by
// 2^e_k >= sum_j |A[j,k]|, split as the operator's own planes.
__global__ void __launch_bounds__(256) split_cols_kernel(const double *__restrict__ A, int rows, int K, int npr,
                                                         __half *__restrict__ T0, __half *__restrict__ T1,
                                                         __half *__restrict__ T2, int *__restrict__ colexp,
                                                         int fbits)
{
    const int abits = LEG_SPLIT_GRID - fbits;
    const int k = blockIdx.x;
    __shared__ double red[8];
    __shared__ double s_inv;
    double s = 0.0;
    for (int j = threadIdx.x; j < rows; j += blockDim.x) s += fabs(A[(size_t)j * K + k]);
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        int e = 0;
        if (t > 0.0) {
            double m = frexp(t, &e);
            if (m == 0.5) e -= 1;
        }
        colexp[k] = e;
        s_inv = ldexp(1.0, -e);
    }
    __syncthreads();
    const double inv = s_inv;
    for (int j = threadIdx.x; j < npr; j += blockDim.x) {
        double a = (j < rows) ? A[(size_t)j * K + k] * inv : 0.0;
        double a0;
        if (fabs(a) >= ldexp(1.0, 10 - abits)) a0 = (double)__double2half(a);
        else a0 = rint(ldexp(a, abits)) * ldexp(1.0, -abits);
        double r1 = ldexp(a - a0, fbits);
        __half h1 = __double2half(r1);
        size_t o = (size_t)k * npr + j;
        T0[o] = __double2half(a0);
        T1[o] = h1;
        T2[o] = __double2half(ldexp(r1 - (double)h1, fbits));
    }
}

// ---------------------------------------------------------------- tensor maps
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *,
                                  CUtensorMapInterleave, CUtensorMapSwizzle, CUtensorMapL2promotion,
                                  CUtensorMapFloatOOBfill);

int get_encoder(EncodeTiledFn *fn)
{
    static EncodeTiledFn cached = nullptr;
    if (!cached) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q);
        if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !p)
            return leg_set_error(LEG_ERR_CUDA, "cuTensorMapEncodeTiled entry point not found");
        cached = reinterpret_cast<EncodeTiledFn>(p);
    }
    *fn = cached;
    return LEG_OK;
}

// 3-D map over `planes` [outer x inner] 16-bit arrays with row stride ld and
// plane stride pstride (elements); box = 32 (inner) x box_outer x 1 plane,
// 64-byte swizzle, zero fill out of bounds: one copy per plane and K block
// (several smaller copies in flight load a stage faster than one large box).
int make_map(CUtensorMap *m, const void *base, int inner, int outer, int ld, int planes, size_t pstride, bool bf16,
             int box_outer)
{
    EncodeTiledFn enc = nullptr;
    int rc = get_encoder(&enc);
    if (rc) return rc;
    cuuint64_t dims[3] = {(cuuint64_t)inner, (cuuint64_t)outer, (cuuint64_t)planes};
    cuuint64_t strides[2] = {(cuuint64_t)ld * 2, (cuuint64_t)pstride * 2};
    cuuint32_t box[3] = {TILE_K, (cuuint32_t)box_outer, 1};   // 32 x 16 bit = 64 B rows
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = enc(m, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 3,
                     const_cast<void *>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                     CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return leg_set_error(LEG_ERR_CUDA, "cuTensorMapEncodeTiled failed");
    return LEG_OK;
}

// Number of CTA pairs of the split kernel that can be resident at once on
// the current device (queried once per device, at the largest shared-memory
// footprint, which allows one CTA per SM).
int max_pairs(int *out)
{
    static std::mutex mu;
    static int cache[64] = {};
    int dev = 0;
    LEG_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return leg_set_error(LEG_ERR_INVALID_ARG, "device index out of range");
    std::lock_guard<std::mutex> lock(mu);
    if (!cache[dev]) {
        auto kern = tc_gemm_kernel<8, true>;
        const size_t smem = SMEM_LIMIT - SMEM_STATIC_RESERVE + 1024;
        LEG_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = 2;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.gridDim = dim3(2, 1, 1);
        cfg.blockDim = dim3(THREADS, 1, 1);
        cfg.dynamicSmemBytes = smem;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        int n = 0;
        LEG_CUDA_TRY(cudaOccupancyMaxActiveClusters(&n, (const void *)kern, &cfg));
        if (n < 1) return leg_set_error(LEG_ERR_CUDA, "no CTA pair of the tensor-core GEMM fits on this device");
        cache[dev] = n;
    }
    *out = cache[dev];
    return LEG_OK;
}

template <int NPROD, bool OUT_DF>
int launch_tc(const TcProblem &single, const TcProblem *multi, int nprob, int ntiles, int tn, int *status,
              long long limit, cudaStream_t st)
{
    if (ntiles <= 0) return LEG_OK;
    if (tn < 16 || tn > max_tn<NPROD>() || tn % 16)
        return leg_set_error(LEG_ERR_INVALID_ARG, "tile width out of range");
    auto kern = tc_gemm_kernel<NPROD, OUT_DF>;
    const int stages = stages_for<NPROD>(tn);
    const size_t smem = (size_t)stages * stage_bytes<NPROD>(tn) + 1024;
    LEG_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int pairs = 0;
    int rc = max_pairs(&pairs);
    if (rc) return rc;
    const int npairs = ntiles < pairs ? ntiles : pairs;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[2];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 2;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    at[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;   // overlaps the split's tail
    at[1].val.programmaticStreamSerializationAllowed = 1;
    cfg.gridDim = dim3(2 * npairs, 1, 1);
    cfg.blockDim = dim3(THREADS, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cfg.attrs = at;
    cfg.numAttrs = 2;
    LEG_CUDA_TRY(cudaLaunchKernelEx(&cfg, kern, single, multi, nprob, ntiles, tn, stages, status, limit));
    return LEG_OK;
}

// Cycles of one pair MMA (M = 256, N = tn, K = 16) on each SM of the pair:
// the slowest of the tensor rate (128 x tn x 16 MACs at 4096 per cycle), the
// operand reads from shared memory (4 KB of A plus tn/2 rows of B at 128
// bytes per cycle) and the issue cost of one pair instruction from the MMA
// warp (about 48 cycles, measured on GB300 with clock64 around the issue loop
// of this kernel for tn = 128..224).
int mma_cycles(int tn)
{
    int c = tn / 2;
    if (32 + tn / 8 > c) c = 32 + tn / 8;
    if (48 > c) c = 48;
    return c;
}

int ceil_div(int a, int b) { return (a + b - 1) / b; }

// Estimated cycles of the busiest pair for ntm row tiles x B functions with
// K-depth nkb: waves x (per-tile fixed cost + nkb x 16 MMAs).
long long tile_cost(int tn, int ntm, int B, int nkb, int pairs)
{
    const long long tiles = (long long)ntm * ceil_div(B, tn);
    const long long waves = (tiles + pairs - 1) / pairs;
    return waves * (2000 + (long long)nkb * 16 * mma_cycles(tn));
}

// Functions per pair tile (<= maxtn): the lowest tile_cost, ties to the wider tile.
int choose_tn(int ntm, int B, int nkb, int pairs, int maxtn = 128)
{
    int best = maxtn;
    long long best_cost = -1;
    for (int tn = maxtn; tn >= 16; tn -= 16) {
        const long long cost = tile_cost(tn, ntm, B, nkb, pairs);
        if (best_cost < 0 || cost < best_cost) {
            best_cost = cost;
            best = tn;
        }
    }
    return best;
}

// na, nf: operator and input planes of the problem (their bytes set the tile order).
void finish_problem(TcProblem *pr, const int *aexp, const int *fexp, void *out, int ldo, int rows, int B, int Kc,
                    int tn, int na, int nf)
{
    pr->aexp = aexp;
    pr->fexp = fexp;
    pr->out = out;
    pr->ldo = ldo;
    pr->rows = rows;
    pr->B = B;
    pr->nkb = Kc / TILE_K;
    pr->tn = tn;
    pr->ntm = ceil_div(rows, PAIR_M);
    pr->ntn = ceil_div(B, tn);
    pr->tile0 = 0;
    pr->fn_fast = (long long)na * rows > (long long)nf * B ? 1 : 0;
    pr->w1 = 1.0f;
}

// Split problem: operator planes a0 + s apstride (rows x Kc, row stride lda),
// input planes of `in`.
int make_split(TcProblem *pr, const __half *a0, size_t apstride, int rows, int lda, const int *aexp,
               const LegSplitIn &in, int B, int Kc, void *out, int ldo, int tn)
{
    int rc;
    if ((rc = make_map(&pr->a, a0, Kc, rows, lda, LEG_SPLIT_NA, apstride, false, CTA_M))) return rc;
    if ((rc = make_map(&pr->f, in.base, Kc, B, in.ld, LEG_SPLIT_NF, in.pstride, false, tn / 2))) return rc;
    finish_problem(pr, aexp, in.fexp, out, ldo, rows, B, Kc, tn, LEG_SPLIT_NA, LEG_SPLIT_NF);
    pr->w1 = ldexpf(1.0f, -in.fbits);
    return LEG_OK;
}

int tiles_of(const TcProblem &pr) { return pr.ntm * pr.ntn; }

}  // namespace

LegSplitIn leg_split_workspace(const leg_plan *p)
{
    LegSplitIn in;
    in.base = p->Fh;
    in.pstride = (size_t)p->ws_B * p->ldf;
    in.ld = p->ldf;
    in.fexp = p->fexp;
    in.fbits = p->fbits;
    return in;
}

int leg_split_max_pairs(int *pairs) { return max_pairs(pairs); }

long long leg_split_tile_cost(int tn, int ntm, int B, int nkb, int pairs) { return tile_cost(tn, ntm, B, nkb, pairs); }

int leg_split_choose_tn(const leg_plan *p, int B)
{
    if (p->tn) return p->tn;
    int pairs = 0;
    if (max_pairs(&pairs)) return max_tn<8>();
    return choose_tn(ceil_div(leg_split_fwd_rows(p), PAIR_M), B, p->Kp / TILE_K, pairs);
}

int leg_split_fwd_rows(const leg_plan *p) { return p->collapsed() ? p->N : p->rows - 1; }

int leg_build_split_transposed(leg_plan *p)
{
    const int npr = leg_adj_depth(p);
    const size_t plane = (size_t)p->K * npr;
    LEG_CUDA_TRY(leg_dev_malloc(&p->AhT[0], sizeof(__half) * 3 * plane));
    p->AhT[1] = p->AhT[0] + plane;
    p->AhT[2] = p->AhT[0] + 2 * plane;
    LEG_CUDA_TRY(leg_dev_malloc(&p->colexp, sizeof(int) * p->K));
    split_cols_kernel<<<p->K, 256>>>(p->collapsed() ? p->L64 : p->A64, p->grows, p->K, npr, p->AhT[0], p->AhT[1],
                                     p->AhT[2], p->colexp, p->fbits);
    LEG_LAUNCH_CHECK("split_cols_kernel");
    return LEG_OK;
}

int leg_split_prepare_input_into(const leg_plan *p, const float *f, int B, const LegSplitIn &in, float2 *G,
                                 int ldg, cudaStream_t st)
{
    return split_rows<float>(f, p->K, p->K, p->Kp, in, G, ldg, p->a00, B, st);
}

int leg_split_prepare_input(const leg_plan *p, const float *f, int B, cudaStream_t st)
{
    // collapsed plans have no G (row 0 of G is written by the split otherwise)
    return leg_split_prepare_input_into(p, f, B, leg_split_workspace(p),
                                        p->collapsed() ? nullptr : static_cast<float2 *>(p->G), p->ldg, st);
}

// Forward split problem: operator rows 1..rows-1 (row 0 is a00 e_0 and is
// written by the input split), output columns 1..rows-1 of G.
int leg_make_split_problem(TcProblem *pr, const leg_plan *p, const LegSplitIn &in, int B, float2 *G, int ldg,
                           int tn)
{
    return make_split(pr, p->Ah[0] + p->Kp, (size_t)p->rows * p->Kp, p->rows - 1, p->Kp, p->rowexp + 1, in, B,
                      p->Kp, G + 1, ldg, tn);
}

int leg_gemm_split_fwd_into(leg_plan *p, int B, const LegSplitIn &in, float2 *G, int ldg, cudaStream_t st)
{
    TcProblem pr;
    int rc = leg_make_split_problem(&pr, p, in, B, G, ldg, leg_split_choose_tn(p, B));
    if (rc) return rc;
    return launch_tc<8, true>(pr, nullptr, 1, tiles_of(pr), pr.tn, p->status, p->wait_limit, st);
}

int leg_gemm_split_fwd(leg_plan *p, int B, cudaStream_t st)
{
    return leg_gemm_split_fwd_into(p, B, leg_split_workspace(p), static_cast<float2 *>(p->G), p->ldg, st);
}

// df[b, k] = sum_j in[b, j] S[j, k] from the split planes `in` (B x npr) of
// the cotangent and the transposed planes of the plan's operator S.
int split_adj_gemm(leg_plan *p, const LegSplitIn &in, void *df, int B, cudaStream_t st)
{
    const int npr = leg_adj_depth(p);
    int pairs = 0;
    int rc = max_pairs(&pairs);
    if (rc) return rc;
    TcProblem pr;
    rc = make_split(&pr, p->AhT[0], (size_t)p->K * npr, p->K, npr, p->colexp, in, B, npr, df, p->K,
                    p->tn ? p->tn : choose_tn(ceil_div(p->K, PAIR_M), B, npr / TILE_K, pairs));
    if (rc) return rc;
    return launch_tc<8, false>(pr, nullptr, 1, tiles_of(pr), pr.tn, p->status, p->wait_limit, st);
}

int leg_gemm_split_adj_planes(leg_plan *p, void *df, int B, cudaStream_t st)
{
    return split_adj_gemm(p, leg_split_workspace(p), df, B, st);
}

int leg_gemm_split_adj(leg_plan *p, void *df, int B, cudaStream_t st)
{
    // Gbar (double-float, B x ldg, rows valid) -> split planes B x npr
    const LegSplitIn in = leg_split_workspace(p);
    int rc = split_rows<float2>(static_cast<const float2 *>(p->Gbar), p->ldg, p->rows, leg_adj_depth(p), in, nullptr,
                                0, 0.0, B, st);
    if (rc) return rc;
    return split_adj_gemm(p, in, df, B, st);
}

// Collapsed plans: c = L f in one split GEMM (L's rows on the MMA's M side),
// FP32 output; no transform stage.
int leg_gemm_split_collapsed_fwd(leg_plan *p, int B, float *c, cudaStream_t st)
{
    TcProblem pr;
    int rc = make_split(&pr, p->Ah[0], (size_t)p->N * p->Kp, p->N, p->Kp, p->rowexp, leg_split_workspace(p), B,
                        p->Kp, c, p->N, leg_split_choose_tn(p, B));
    if (rc) return rc;
    return launch_tc<8, false>(pr, nullptr, 1, tiles_of(pr), pr.tn, p->status, p->wait_limit, st);
}

// Collapsed plans: df = L^T dc (dc FP32, B x N).
int leg_gemm_split_collapsed_adj(leg_plan *p, const float *dc, void *df, int B, cudaStream_t st)
{
    const LegSplitIn in = leg_split_workspace(p);
    int rc = split_rows<float>(dc, p->N, p->N, leg_adj_depth(p), in, nullptr, 0, 0.0, B, st);
    if (rc) return rc;
    return split_adj_gemm(p, in, df, B, st);
}

int leg_bf16_prepare_input(const leg_plan *p, const float *f, int B, cudaStream_t st)
{
    bf16_rows_kernel<<<B, 256, 0, st>>>(f, p->K, p->Kp, p->Fbf);
    LEG_LAUNCH_CHECK("bf16_rows_kernel");
    return LEG_OK;
}

int leg_gemm_bf16_fwd(leg_plan *p, int B, void *out, int ldo, cudaStream_t st)
{
    int pairs = 0;
    int rc = max_pairs(&pairs);
    if (rc) return rc;
    const int rows = p->grows;
    const int tn = p->tn ? p->tn : choose_tn(ceil_div(rows, PAIR_M), B, p->Kp / TILE_K, pairs, max_tn<1>());
    TcProblem pr;
    memset(&pr, 0, sizeof(pr));
    if ((rc = make_map(&pr.a, p->Abf, p->Kp, rows, p->Kp, 1, (size_t)rows * p->Kp, true, CTA_M))) return rc;
    if ((rc = make_map(&pr.f, p->Fbf, p->Kp, B, p->Kp, 1, (size_t)B * p->Kp, true, tn / 2))) return rc;
    finish_problem(&pr, nullptr, nullptr, out, ldo, rows, B, p->Kp, tn, 1, 1);
    return launch_tc<1, false>(pr, nullptr, 1, tiles_of(pr), tn, p->status, p->wait_limit, st);
}

// ---------------------------------------------------------------- grouped (ragged) launches
int leg_split_problem_tiles(const TcProblem &pr) { return tiles_of(pr); }

int leg_gemm_split_grouped(const TcProblem *d_probs, int nprob, int ntiles, int tn, int *status, long long limit,
                           cudaStream_t st)
{
    TcProblem dummy;
    memset(&dummy, 0, sizeof(dummy));
    return launch_tc<8, true>(dummy, d_probs, nprob, ntiles, tn, status, limit, st);
}

int leg_split_ragged(const float *f_packed, const long long *in_off, const int *bucket, const int *row,
                     const LegRaggedBucket *bk, int count, int max_k, cudaStream_t st)
{
    if (count == 0) return LEG_OK;
    const size_t bytes = ((size_t)leg_round_up(max_k, LEG_KPAD) * sizeof(float) + 15) / 16 * 16;
    if (bytes <= SPLIT_STAGE_MAX)
        split_ragged_kernel<true><<<count, SPLIT_THREADS, bytes, st>>>(f_packed, in_off, bucket, row, bk);
    else
        split_ragged_kernel<false><<<count, SPLIT_THREADS, 0, st>>>(f_packed, in_off, bucket, row, bk);
    LEG_LAUNCH_CHECK("split_ragged_kernel");
    return LEG_OK;
}
