// Real-number arithmetics used by the FFT stage: FP64, FP32 and double-float
// (an unevaluated sum hi + lo of two FP32 numbers, about 48 significant bits).
//
// Double-float operations are built from the classical error-free
// transformations: Knuth's TwoSum, Dekker's Fast2Sum, and the FMA-based exact
// product.  They rely on IEEE FP32 round-to-nearest and on the compiler not
// re-associating additions (no fast-math flags are used).
#pragma once

#include <cuda_runtime.h>

struct dfl {
    float hi, lo;
};

__device__ __forceinline__ dfl df_two_sum(float a, float b)
{
    float s = a + b;
    float bb = s - a;
    float e = (a - (s - bb)) + (b - bb);
    return {s, e};
}

__device__ __forceinline__ dfl df_fast_two_sum(float a, float b)   // |a| >= |b|
{
    float s = a + b;
    float e = b - (s - a);
    return {s, e};
}

__device__ __forceinline__ dfl df_add(dfl a, dfl b)
{
    dfl s = df_two_sum(a.hi, b.hi);
    float lo = s.lo + (a.lo + b.lo);
    return df_fast_two_sum(s.hi, lo);
}

__device__ __forceinline__ dfl df_neg(dfl a) { return {-a.hi, -a.lo}; }

__device__ __forceinline__ dfl df_sub(dfl a, dfl b) { return df_add(a, df_neg(b)); }

__device__ __forceinline__ dfl df_mul(dfl a, dfl b)
{
    float p = a.hi * b.hi;
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    return df_fast_two_sum(p, e);
}

// multiply by an exact power of two
__device__ __forceinline__ dfl df_ldexp(dfl a, int e) { return {ldexpf(a.hi, e), ldexpf(a.lo, e)}; }

// ---------------------------------------------------------------------------
// Arithmetic traits.  R is the real type; GT the type of a G element on input;
// TW the twiddle-table element; OUT the output element.
// ---------------------------------------------------------------------------
template <class R> struct Ar;

template <> struct Ar<double> {
    using T = double;
    using GT = double;
    using TW = double2;
    using OUT = double;
    static __device__ __forceinline__ T zero() { return 0.0; }
    static __device__ __forceinline__ T add(T a, T b) { return a + b; }
    static __device__ __forceinline__ T sub(T a, T b) { return a - b; }
    static __device__ __forceinline__ T mul(T a, T b) { return a * b; }
    static __device__ __forceinline__ T neg(T a) { return -a; }
    static __device__ __forceinline__ T pow2(T a, int e) { return ldexp(a, e); }
    static __device__ __forceinline__ T from_g(GT g) { return g; }
    static __device__ __forceinline__ T from_int(int n) { return (double)n; }
    static __device__ __forceinline__ T from_in(double v) { return v; }
    static __device__ __forceinline__ void tw(const TW *t, int i, T &c, T &s) { TW v = t[i]; c = v.x; s = v.y; }
    static __device__ __forceinline__ OUT out(T a) { return a; }
    static __device__ __forceinline__ GT to_g(T a) { return a; }
};

template <> struct Ar<float> {
    using T = float;
    using GT = float;
    using TW = float2;
    using OUT = float;
    static __device__ __forceinline__ T zero() { return 0.0f; }
    static __device__ __forceinline__ T add(T a, T b) { return a + b; }
    static __device__ __forceinline__ T sub(T a, T b) { return a - b; }
    static __device__ __forceinline__ T mul(T a, T b) { return a * b; }
    static __device__ __forceinline__ T neg(T a) { return -a; }
    static __device__ __forceinline__ T pow2(T a, int e) { return ldexpf(a, e); }
    static __device__ __forceinline__ T from_g(GT g) { return g; }
    static __device__ __forceinline__ T from_int(int n) { return (float)n; }
    static __device__ __forceinline__ T from_in(float v) { return v; }
    static __device__ __forceinline__ void tw(const TW *t, int i, T &c, T &s) { TW v = t[i]; c = v.x; s = v.y; }
    static __device__ __forceinline__ OUT out(T a) { return a; }
    static __device__ __forceinline__ GT to_g(T a) { return a; }
};

template <> struct Ar<dfl> {
    using T = dfl;
    using GT = float2;
    using TW = float4;
    using OUT = float;
    static __device__ __forceinline__ T zero() { return {0.0f, 0.0f}; }
    static __device__ __forceinline__ T add(T a, T b) { return df_add(a, b); }
    static __device__ __forceinline__ T sub(T a, T b) { return df_sub(a, b); }
    static __device__ __forceinline__ T mul(T a, T b) { return df_mul(a, b); }
    static __device__ __forceinline__ T neg(T a) { return df_neg(a); }
    static __device__ __forceinline__ T pow2(T a, int e) { return df_ldexp(a, e); }
    static __device__ __forceinline__ T from_g(GT g) { return {g.x, g.y}; }
    static __device__ __forceinline__ T from_int(int n) { return {(float)n, 0.0f}; }
    static __device__ __forceinline__ T from_in(float v) { return {v, 0.0f}; }
    static __device__ __forceinline__ void tw(const TW *t, int i, T &c, T &s)
    {
        TW v = t[i];
        c = {v.x, v.y};
        s = {v.z, v.w};
    }
    static __device__ __forceinline__ OUT out(T a) { return a.hi + a.lo; }
    static __device__ __forceinline__ GT to_g(T a) { return make_float2(a.hi, a.lo); }
};

template <class T> struct Cx {
    T re, im;
};
