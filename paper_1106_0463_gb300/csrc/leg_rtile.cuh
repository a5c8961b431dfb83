// Register-tiled transforms of the FFT stage: shared machinery.
//
// A function's length-H complex sequence (H = M/4) lives in registers:
// E = min(2^LEG_DCT16_LOG2E, H/32) values per thread (min(8, H/32) with the
// default LEG_DCT16_LOG2E = 3), T = H/E threads per function (two warps for
// H = 512).  The FFT is a Stockham autosort of radix-E
// passes (the last pass takes the remaining power of two): each thread holds
// x[t + b T], b < E, forms E/R radix-R butterflies from them, applies the
// inter-pass twiddles (H-th roots of unity from the compact FP64-built table),
// transforms in registers (a radix-2 network with constant twiddles) and
// writes the outputs to their autosorted positions in shared memory, padded by
// one slot per E values to avoid bank conflicts.  Double-float sums and
// products skip the final renormalisation, between passes as well as inside
// them: the error terms stay exact (TwoSum of the leading parts, FMA
// products), the trailing part grows by about one rounding unit of the
// leading part per operation, and over the few dozen operations a value goes
// through its own FP32 rounding stays near 2^-42 of the value; results are
// rounded once, at the output.  (Renormalising every stored value cost 3-9 %
// of the transform time and changed results by 1e-12 to 6e-11 of max |c|.)
// Functions of T = 32 synchronise with __syncwarp only.
//
// Users: leg_dct16.cu (the real-even transform of Theorem 1 with the twist as
// a first difference) and leg_dst16.cu (the half-range sine form, Eq. 2.13).
#pragma once

#include "leg_fft.cuh"
#include "leg_internal.cuh"

#include <type_traits>

namespace {

// ---------------------------------------------------------------- arithmetic
template <class T> struct Fa;

template <> struct Fa<double> {
    using T = double;
    static __device__ __forceinline__ T add(T a, T b) { return a + b; }
    static __device__ __forceinline__ T sub(T a, T b) { return a - b; }
    static __device__ __forceinline__ T mul(T a, T b) { return a * b; }
    static __device__ __forceinline__ T neg(T a) { return -a; }
    static __device__ __forceinline__ T half(T a) { return 0.5 * a; }
    static __device__ __forceinline__ T norm(T a) { return a; }
    static __device__ __forceinline__ T cst(double v) { return v; }
    static __device__ __forceinline__ T of_int(int v) { return (double)v; }
    static __device__ __forceinline__ T of_float(float v) { return (double)v; }
    static __device__ __forceinline__ T zero() { return 0.0; }
    static __device__ __forceinline__ T pow2(T a, int e) { return ldexp(a, e); }
};

template <> struct Fa<dfl> {
    using T = dfl;
    // TwoSum of the leading parts, trailing parts added without renormalising
    static __device__ __forceinline__ T add(T a, T b)
    {
        const float s = a.hi + b.hi;
        const float bb = s - a.hi;
        const float e = (a.hi - (s - bb)) + (b.hi - bb);
        return {s, e + (a.lo + b.lo)};
    }
    static __device__ __forceinline__ T neg(T a) { return {-a.hi, -a.lo}; }
    static __device__ __forceinline__ T sub(T a, T b) { return add(a, neg(b)); }
    // exact product of the leading parts (FMA), cross terms added, no renormalisation
    static __device__ __forceinline__ T mul(T a, T b)
    {
        const float p = a.hi * b.hi;
        float e = fmaf(a.hi, b.hi, -p);
        e = fmaf(a.hi, b.lo, e);
        e = fmaf(a.lo, b.hi, e);
        return {p, e};
    }
    static __device__ __forceinline__ T half(T a) { return {0.5f * a.hi, 0.5f * a.lo}; }
    static __device__ __forceinline__ T norm(T a)
    {
        const float s = a.hi + a.lo;
        return {s, a.lo - (s - a.hi)};
    }
    // compile-time constants only (the FP64 arithmetic folds away)
    static __device__ __forceinline__ T cst(double v)
    {
        const float h = (float)v;
        return {h, (float)(v - (double)h)};
    }
    // exact for |v| < 2^24 and for FP32 values: no FP64 instruction at run time
    static __device__ __forceinline__ T of_int(int v) { return {__int2float_rn(v), 0.0f}; }
    static __device__ __forceinline__ T of_float(float v) { return {v, 0.0f}; }
    static __device__ __forceinline__ T zero() { return {0.0f, 0.0f}; }
    // a 2^e: one exact multiply per part while 2^e is a normal float
    static __device__ __forceinline__ T pow2(T a, int e)
    {
        if (e >= -126 && e <= 127) {
            const float m = __int_as_float((e + 127) << 23);
            return {a.hi * m, a.lo * m};
        }
        return {ldexpf(a.hi, e), ldexpf(a.lo, e)};
    }
};

template <> struct Fa<float> {
    using T = float;
    static __device__ __forceinline__ T add(T a, T b) { return a + b; }
    static __device__ __forceinline__ T sub(T a, T b) { return a - b; }
    static __device__ __forceinline__ T mul(T a, T b) { return a * b; }
    static __device__ __forceinline__ T neg(T a) { return -a; }
    static __device__ __forceinline__ T half(T a) { return 0.5f * a; }
    static __device__ __forceinline__ T norm(T a) { return a; }
    static __device__ __forceinline__ T cst(double v) { return (float)v; }
    static __device__ __forceinline__ T of_int(int v) { return __int2float_rn(v); }
    static __device__ __forceinline__ T of_float(float v) { return v; }
    static __device__ __forceinline__ T zero() { return 0.0f; }
    static __device__ __forceinline__ T pow2(T a, int e)
    {
        if (e >= -126 && e <= 127) return a * __int_as_float((e + 127) << 23);
        return ldexpf(a, e);
    }
};

template <class R> using CxT = Cx<typename Fa<R>::T>;

template <class R>
__device__ __forceinline__ CxT<R> cadd(CxT<R> a, CxT<R> b)
{
    using F = Fa<R>;
    return {F::add(a.re, b.re), F::add(a.im, b.im)};
}

template <class R>
__device__ __forceinline__ CxT<R> csub(CxT<R> a, CxT<R> b)
{
    using F = Fa<R>;
    return {F::sub(a.re, b.re), F::sub(a.im, b.im)};
}

template <class R>
__device__ __forceinline__ CxT<R> cmul(CxT<R> a, typename Fa<R>::T c, typename Fa<R>::T s)
{
    using F = Fa<R>;
    return {F::sub(F::mul(a.re, c), F::mul(a.im, s)), F::add(F::mul(a.re, s), F::mul(a.im, c))};
}

// a * e^{2 pi i m / 16}, m = 0..7 (constant)
template <class R, int m>
__device__ __forceinline__ CxT<R> wmul16(CxT<R> a)
{
    using F = Fa<R>;
    constexpr double C1 = 0.92387953251128675613, S1 = 0.38268343236508977173, H2 = 0.70710678118654752440;
    if constexpr (m == 0) {
        return a;
    } else if constexpr (m == 4) {
        return {F::neg(a.im), a.re};
    } else if constexpr (m == 2) {
        const auto h = F::cst(H2);
        return {F::mul(h, F::sub(a.re, a.im)), F::mul(h, F::add(a.re, a.im))};
    } else if constexpr (m == 6) {
        const auto h = F::cst(H2);
        return {F::neg(F::mul(h, F::add(a.re, a.im))), F::mul(h, F::sub(a.re, a.im))};
    } else {
        constexpr double c = (m == 1) ? C1 : (m == 3) ? S1 : (m == 5) ? -S1 : -C1;
        constexpr double s = (m == 1) ? S1 : (m == 3) ? C1 : (m == 5) ? C1 : S1;
        return cmul<R>(a, F::cst(c), F::cst(s));
    }
}

__host__ __device__ constexpr int bitrev(int n, int bits)
{
    int r = 0;
    for (int i = 0; i < bits; ++i) r |= ((n >> i) & 1) << (bits - 1 - i);
    return r;
}

// Butterflies m..S-1 of a radix-2 stage (half-size S) on the block at blk:
// twiddle e^{2 pi i m / (2S)} = W16^{m * 16 / (2S)}.
template <class R, int P, int S, int m>
struct Bfly {
    static __device__ __forceinline__ void run(CxT<R> (&x)[P], int blk)
    {
        if constexpr (m < S) {
            const CxT<R> b = wmul16<R, m * (16 / (2 * S))>(x[blk + m + S]);
            const CxT<R> a = x[blk + m];
            x[blk + m] = cadd<R>(a, b);
            x[blk + m + S] = csub<R>(a, b);
            Bfly<R, P, S, m + 1>::run(x, blk);
        }
    }
};

template <class R, int P, int S>
__device__ __forceinline__ void dft_stage(CxT<R> (&x)[P])
{
    if constexpr (S < P) {
#pragma unroll
        for (int blk = 0; blk < P; blk += 2 * S) Bfly<R, P, S, 0>::run(x, blk);
        dft_stage<R, P, 2 * S>(x);
    }
}

// In-register DFT of size P (2, 4, 8 or 16), positive exponent, natural order
// in and out: radix-2 decimation in time on the bit-reversed inputs.
template <class R, int P, int LOGP>
__device__ __forceinline__ void dft(CxT<R> (&x)[P])
{
    CxT<R> y[P];
#pragma unroll
    for (int i = 0; i < P; ++i) y[i] = x[bitrev(i, LOGP)];
#pragma unroll
    for (int i = 0; i < P; ++i) x[i] = y[i];
    dft_stage<R, P, 1>(x);
}

#ifndef LEG_DCT16_LOG2E
#define LEG_DCT16_LOG2E 3   // at most 2^LEG_DCT16_LOG2E complex values per thread
#endif


// Shape of a register-tiled transform of length H = 2^LOG2H with at most 2^XE
// complex values per thread (XE = 3: radix-8 passes, 4: radix-16).
template <int LOG2H, int XE = LEG_DCT16_LOG2E> struct D16 {
    static constexpr int H = 1 << LOG2H;
    static constexpr int L = 2 * H;
    static constexpr int M = 2 * L;
    static constexpr int LOG2E = (LOG2H - 5 < XE) ? LOG2H - 5 : XE;
    static constexpr int E = 1 << LOG2E;
    static constexpr int T = H / E;                                 // threads per function, >= 32
    static constexpr int FPB = (T >= 128) ? 1 : 128 / T;            // functions per CTA
    static constexpr int THREADS = T * FPB;
    // resident CTAs per SM the register allocation aims at: six for CTAs of
    // 128 threads (H <= 1024; 80 registers, measured 51 us against 53 us at
    // H = 512 for B = 4096), none imposed for larger CTAs
    // resident CTAs per SM asked of the register allocator: about 24-32 warps
    // per SM (80 registers at 128 and 256 threads, 64 at 512; 158 and 128
    // registers without the target left one CTA per SM)
    // radix-16 threads hold twice the values: a 128-register budget
    static constexpr int MINB = XE >= 4 ? (THREADS >= 512 ? 1 : 512 / THREADS)
                                        : THREADS <= 128 ? 6 : THREADS == 256 ? 3 : THREADS == 512 ? 2 : 1;
    static constexpr int SLOTS = H + H / E + 1;                     // padded complex slots per function
    static constexpr int WARPS = T / 32;
    // FFT buffer: one padding slot per E complex values; real view (X): one
    // padding word per 2E words.  Both keep a warp's accesses conflict-free
    // for consecutive and for E-strided indices.
    static __device__ __forceinline__ int pc(int i) { return i + (i >> LOG2E); }
    static __device__ __forceinline__ int px(int i) { return i + (i >> (LOG2E + 1)); }
};

// Complex slots between consecutive functions' exchange buffers for the
// arithmetic type R: D16::SLOTS, rounded up so that every buffer starts on a
// 16-byte boundary (the row staging copies 16 bytes at a time).  SLOTS is odd,
// so 8-byte complex values (FP32) take one more slot; 16-byte ones keep SLOTS.
template <class R, int LOG2H, int XE = LEG_DCT16_LOG2E>
__host__ __device__ constexpr int gslots()
{
    constexpr int S = D16<LOG2H, XE>::SLOTS;
    return (S * (int)sizeof(CxT<R>)) % 16 == 0 ? S : S + (16 / (int)sizeof(CxT<R>)) - 1;
}

template <int T>
__device__ __forceinline__ void fsync()
{
    if constexpr (T == 32) __syncwarp();
    else __syncthreads();
}

// Twiddle (cos, sin) of 2 pi i / M from the table (double2, float2 or float4 double-float).
__device__ __forceinline__ void twid(const double2 *tw, int i, double &c, double &s)
{
    const double2 v = tw[i];
    c = v.x;
    s = v.y;
}
__device__ __forceinline__ void twid(const float2 *tw, int i, float &c, float &s)
{
    const float2 v = tw[i];
    c = v.x;
    s = v.y;
}
__device__ __forceinline__ void twid(const float4 *tw, int i, dfl &c, dfl &s)
{
    const float4 v = tw[i];
    c = {v.x, v.y};
    s = {v.z, v.w};
}

// One Stockham pass of radix P over v = x[t + b T] (b < E): butterflies
// j = t + bb T (bb < E/P) of stride Ns, twiddles e^{2 pi i r k / (P Ns)},
// outputs to buf[D::pc((j - k) P + k + r Ns)].
template <class R, int LOG2H, int P, int LOGP, int XE = LEG_DCT16_LOG2E>
__device__ __forceinline__ void fft_pass(CxT<R> (&v)[D16<LOG2H, XE>::E], CxT<R> *buf, int t, int Ns,
                                         const typename Ar<R>::TW *tw)
{
    using D = D16<LOG2H, XE>;
    using F = Fa<R>;
    constexpr int E = D::E, T = D::T, NB = E / P;
    // e^{2 pi i r k / (P Ns)} = entry r k H / (P Ns) of the compact table of
    // H = M/4 entries that follows the full one (a quarter of the cache footprint)
    const int tstep = D::H / (P * Ns);
    const typename Ar<R>::TW *twc = tw + D::M;
#pragma unroll
    for (int bb = 0; bb < NB; ++bb) {
        const int j = t + bb * T;
        const int k = j & (Ns - 1);
        CxT<R> x[P];
#pragma unroll
        for (int r = 0; r < P; ++r) x[r] = v[bb + r * NB];
        if (k != 0) {
#pragma unroll
            for (int r = 1; r < P; ++r) {
                typename F::T c, s;
                twid(twc, r * k * tstep, c, s);
                x[r] = cmul<R>(x[r], c, s);
            }
        }
        dft<R, P, LOGP>(x);
        const int o = (j - k) * P + k;
#pragma unroll
        for (int r = 0; r < P; ++r) {
            buf[D::pc(o + r * Ns)] = x[r];
        }
    }
}

template <class R, int LOG2H, int XE = LEG_DCT16_LOG2E>
__device__ __forceinline__ void fft_pass_any(int P, CxT<R> (&v)[D16<LOG2H, XE>::E], CxT<R> *buf, int t, int Ns,
                                             const typename Ar<R>::TW *tw)
{
    if constexpr (D16<LOG2H, XE>::E >= 16) {
        if (P == 16) return fft_pass<R, LOG2H, 16, 4, XE>(v, buf, t, Ns, tw);
    }
    if constexpr (D16<LOG2H, XE>::E >= 8) {
        if (P == 8) return fft_pass<R, LOG2H, 8, 3, XE>(v, buf, t, Ns, tw);
    }
    if constexpr (D16<LOG2H, XE>::E >= 4) {
        if (P == 4) return fft_pass<R, LOG2H, 4, 2, XE>(v, buf, t, Ns, tw);
    }
    fft_pass<R, LOG2H, 2, 1, XE>(v, buf, t, Ns, tw);
}

__device__ __forceinline__ double shfl_up(double v, int off) { return __shfl_up_sync(0xffffffffu, v, off); }
__device__ __forceinline__ dfl shfl_up(dfl v, int off)
{
    return {__shfl_up_sync(0xffffffffu, v.hi, off), __shfl_up_sync(0xffffffffu, v.lo, off)};
}
__device__ __forceinline__ float shfl_up(float v, int off) { return __shfl_up_sync(0xffffffffu, v, off); }
__device__ __forceinline__ double shfl_xor(double v, int off) { return __shfl_xor_sync(0xffffffffu, v, off); }
__device__ __forceinline__ float shfl_xor(float v, int off) { return __shfl_xor_sync(0xffffffffu, v, off); }
__device__ __forceinline__ dfl shfl_xor(dfl v, int off)
{
    return {__shfl_xor_sync(0xffffffffu, v.hi, off), __shfl_xor_sync(0xffffffffu, v.lo, off)};
}

// Inclusive scan of v over the T threads of a function (warp shuffles, then
// the warp totals through shared memory).  wsum: D::WARPS slots per function.
template <class R, int LOG2H, int XE = LEG_DCT16_LOG2E>
__device__ __forceinline__ typename Fa<R>::T fn_scan(typename Fa<R>::T v, int t, typename Fa<R>::T *wsum)
{
    using D = D16<LOG2H, XE>;
    using F = Fa<R>;
    using T_ = typename F::T;
    const int lane = t & 31;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const T_ u = shfl_up(v, off);
        if (lane >= off) v = F::add(v, u);
    }
    if constexpr (D::WARPS > 1) {
        const int w = t >> 5;
        if (lane == 31) wsum[w] = v;
        __syncthreads();
        T_ before = F::zero();
        for (int i = 0; i < w; ++i) before = F::add(before, wsum[i]);
        v = F::add(before, v);
        __syncthreads();
    }
    return v;
}

// Sum of v over the T threads of a function, returned to every thread.
template <class R, int LOG2H, int XE = LEG_DCT16_LOG2E>
__device__ __forceinline__ typename Fa<R>::T fn_sum(typename Fa<R>::T v, int t, typename Fa<R>::T *wsum)
{
    using D = D16<LOG2H, XE>;
    using F = Fa<R>;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v = F::add(v, shfl_xor(v, off));
    if constexpr (D::WARPS > 1) {
        if ((t & 31) == 0) wsum[t >> 5] = v;
        __syncthreads();
        v = wsum[0];
        for (int i = 1; i < D::WARPS; ++i) v = F::add(v, wsum[i]);
        __syncthreads();
    }
    return v;
}

// The length-H FFT (positive exponent) of v = x[t + b T], b < E, in place:
// on return buf[D::pc(k)] holds X_k, k < H, in natural order.  Stockham
// passes of radix E (the last one smaller).  The caller synchronises the
// function's threads before the first pass if load-time reads of buf must
// precede its writes, and after the return before reading buf.
template <class R, int LOG2H, int XE = LEG_DCT16_LOG2E>
__device__ __forceinline__ void fft16(CxT<R> (&v)[D16<LOG2H, XE>::E], CxT<R> *buf, int t, const typename Ar<R>::TW *tw)
{
    using D = D16<LOG2H, XE>;
    constexpr int E = D::E, T = D::T, H = D::H;
    int Ns = 1;
    {
        constexpr int P0 = (E < H) ? E : H;
        fft_pass_any<R, LOG2H, XE>(P0, v, buf, t, 1, tw);
        Ns = P0;
    }
    // one copy of the pass body (runtime Ns and radix): fully unrolled passes
    // of double-float butterflies outgrow the instruction cache
#pragma unroll 1
    while (Ns < H) {
        fsync<T>();
#pragma unroll
        for (int b = 0; b < E; ++b) v[b] = buf[D::pc(t + b * T)];
        fsync<T>();
        // below H = 8192 the remaining bits go to passes of near-equal radix
        // (H = 1024: 8 8 4 4 instead of 8 8 8 2, 16 8 8 instead of 16 16 4;
        // measured 2-17 % faster there); at H = 8192 full-radix passes and a
        // radix-2 tail measured 2 % faster than 8 8 8 4 4
        int P;
        if constexpr (LOG2H < 13) {
            const int rem = LOG2H - (31 - __clz(Ns));
            const int np = (rem + D::LOG2E - 1) / D::LOG2E;
            P = 1 << ((rem + np - 1) / np);
        } else {
            P = (H / Ns < E) ? H / Ns : E;
        }
        fft_pass_any<R, LOG2H, XE>(P, v, buf, t, Ns, tw);
        Ns *= P;
    }
}

// Stage row f of G (L + 1 values, rounded up to 16 bytes; rows are 16-byte
// aligned with at least one padding element) in buf, which the transform's
// first step reads before the first FFT pass overwrites it: every 16-byte
// copy of the row is in flight at once.  Synchronises the function's threads.
template <class R, int LOG2H, int XE = LEG_DCT16_LOG2E>
__device__ __forceinline__ void stage_row(CxT<R> *buf, const typename Ar<R>::GT *G, int ldg, int f, int t)
{
    using D = D16<LOG2H, XE>;
    using GT = typename Ar<R>::GT;
    constexpr int BYTES = ((D::L + 1) * (int)sizeof(GT) + 15) / 16 * 16;
    static_assert(BYTES <= D::SLOTS * (int)sizeof(CxT<R>), "row of G exceeds the exchange buffer");
    static_assert((gslots<R, LOG2H, XE>() * (int)sizeof(CxT<R>)) % 16 == 0, "exchange buffers must be 16-byte aligned");
    const char *src = reinterpret_cast<const char *>(G + (size_t)f * ldg);
    const uint32_t dst = (uint32_t)__cvta_generic_to_shared(buf);
    for (int o = 16 * t; o < BYTES; o += 16 * D::T)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst + o), "l"(src + o) : "memory");
    asm volatile("cp.async.wait_all;" ::: "memory");
    fsync<D::T>();
}

template <class R> struct GIn;
template <> struct GIn<double> {
    static __device__ __forceinline__ double get(const double *g, int j) { return g[j]; }
};
template <> struct GIn<float> {
    static __device__ __forceinline__ float get(const float *g, int j) { return g[j]; }
};
template <> struct GIn<dfl> {
    static __device__ __forceinline__ dfl get(const float2 *g, int j)
    {
        const float2 v = g[j];
        return {v.x, v.y};
    }
};

// a cotangent value (FP64, or FP32 for the double-float path) in the arithmetic type
template <class R> __device__ __forceinline__ typename Fa<R>::T in_of(double v) { return Fa<R>::cst(v); }
template <class R> __device__ __forceinline__ typename Fa<R>::T in_of(float v) { return Fa<R>::of_float(v); }

__device__ __forceinline__ double out_of(double a) { return a; }
__device__ __forceinline__ float out_of(float a) { return a; }
__device__ __forceinline__ float out_of(dfl a) { return a.hi + a.lo; }

// The double-float forward transform up to H = 512 runs at 7 resident CTAs
// per SM (72 registers, a 4-byte spill): 2 us faster per step than 6 at
// M = 2048, B = 4096; the other variants spill 48-64 bytes there and keep 6.
template <class R, int LOG2H, int XE = LEG_DCT16_LOG2E>
constexpr int fwd_minb()
{
    return (std::is_same<R, dfl>::value && LOG2H <= 9 && XE == 3) ? 7 : D16<LOG2H, XE>::MINB;
}

template <class R, int LOG2H, int XE = LEG_DCT16_LOG2E>
size_t d16_smem()
{
    using D = D16<LOG2H, XE>;
    return sizeof(CxT<R>) * D::FPB * gslots<R, LOG2H, XE>() + sizeof(typename Fa<R>::T) * D::FPB * D::WARPS;
}

}  // namespace
