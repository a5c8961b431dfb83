// The input split of the split-FP16 path: per-row power-of-two scale and the
// seven FP16 planes of a row (device helpers shared by the split kernels of
// leg_gemm_tc.cu and the transform kernels that write planes directly).
//
// One row: power-of-two scale 2^e >= max|x|, then with s = the plan's slice
// width
//   xs = x 2^-e,  F0 = round(xs 2^s) 2^-s,  r = (xs - F0) 2^s,  F1 = fp16(r),
// and the seven planes  F0, F1, fp16(r - F1), fp16(2^-s F1), 2^-s F0,
// fp16(2^-2s F1), fp16(2^-s (r - F1))  (plane p at P + p * pstride), so that
// xs = F0 + 2^-s (F1 + (r - F1)).  Values are FP32 (forward) or double-float
// pairs (adjoint, float2 = (hi, lo)).
#pragma once

#include <cuda_fp16.h>

#include "leg_internal.cuh"

namespace {

template <class T> __device__ __forceinline__ float hi_of(T v);
template <> __device__ __forceinline__ float hi_of<float>(float v) { return v; }
template <> __device__ __forceinline__ float hi_of<float2>(float2 v) { return v.x; }
template <class T> __device__ __forceinline__ float lo_of(T v);
template <> __device__ __forceinline__ float lo_of<float>(float) { return 0.0f; }
template <> __device__ __forceinline__ float lo_of<float2>(float2 v) { return v.y; }

template <class T> __device__ __forceinline__ T zero_of();
template <> __device__ __forceinline__ float zero_of<float>() { return 0.0f; }
template <> __device__ __forceinline__ float2 zero_of<float2>() { return make_float2(0.0f, 0.0f); }

// Planes of two scaled values (h, l: leading and trailing parts of x 2^-e)
// as FP16 pairs: the seven planes' values for elements i and i + 1
// (SC = 2^s, ISC = 2^-s).
__device__ __forceinline__ void split_pair(float ha, float la, float hb, float lb, float SC, float ISC,
                                           __half2 (&o)[LEG_SPLIT_NF])
{
    const float x0a = rintf(ha * SC) * ISC, x0b = rintf(hb * SC) * ISC;
    const float ra = (ha - x0a) * SC + la * SC, rb = (hb - x0b) * SC + lb * SC;
    const __half2 f1 = __floats2half2_rn(ra, rb);
    const float2 f1f = __half22float2(f1);
    const float da = ra - f1f.x, db = rb - f1f.y;
    o[0] = __floats2half2_rn(x0a, x0b);
    o[1] = f1;
    o[2] = __floats2half2_rn(da, db);
    o[3] = __floats2half2_rn(f1f.x * ISC, f1f.y * ISC);
    o[4] = __floats2half2_rn(x0a * ISC, x0b * ISC);
    o[5] = __floats2half2_rn(f1f.x * (ISC * ISC), f1f.y * (ISC * ISC));
    o[6] = __floats2half2_rn(da * ISC, db * ISC);
}

// Power of two e of a row's scale: max |x| 2^-e <= 1 (0 for a zero row).
__device__ __forceinline__ int split_scale_exp(float mm)
{
    int e = 0;
    if (mm > 0.0f) {
        const float fr = frexpf(mm, &e);   // mm = fr 2^e, fr in [0.5, 1)
        if (fr == 0.5f) e -= 1;            // scaled |hi| <= 1, hence |F0| <= 1
    }
    return e;
}

// a00 x[0] as a double-float pair (a00 = hi + lo; x[0] is FP32): exact
// product of the leading parts by FMA, the rest in FP32
__device__ __forceinline__ float2 split_g0(float x, float2 a00)
{
    const float p = x * a00.x;
    const float q = fmaf(x, a00.x, -p) + x * a00.y;
    const float h = p + q;
    return make_float2(h, q - (h - p));
}

// The seven planes of the 8 values v[0..7] of a row scaled by 2^-e, one
// 16-byte store per plane at P + p pstride.
template <class T>
__device__ __forceinline__ void split_planes8(const T (&v)[8], int e, float SC, float ISC, __half *__restrict__ P,
                                              size_t pstride)
{
    // x 2^-e: one exact multiply while 2^-e is a normal float (ldexpf beyond)
    const bool mul_ok = (-e >= -126 && -e <= 127);
    const float sc = mul_ok ? __int_as_float((127 - e) << 23) : 0.0f;
    float h[8], l[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        h[i] = mul_ok ? hi_of(v[i]) * sc : ldexpf(hi_of(v[i]), -e);
        l[i] = mul_ok ? lo_of(v[i]) * sc : ldexpf(lo_of(v[i]), -e);
    }
    __align__(16) __half2 o[LEG_SPLIT_NF][4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        __half2 q[LEG_SPLIT_NF];
        split_pair(h[2 * i], l[2 * i], h[2 * i + 1], l[2 * i + 1], SC, ISC, q);
#pragma unroll
        for (int p = 0; p < LEG_SPLIT_NF; ++p) o[p][i] = q[p];
    }
#pragma unroll
    for (int p = 0; p < LEG_SPLIT_NF; ++p)
        *reinterpret_cast<uint4 *>(P + p * pstride) = *reinterpret_cast<const uint4 *>(o[p]);
}

}  // namespace
