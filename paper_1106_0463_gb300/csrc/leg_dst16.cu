// Register-tiled sine-form transform for the FFT stage (FP64, double-float, FP32).
//
// The half-range sine form of the coefficients (arXiv:1106.0463, Eq. 2.13
// with phi of Eq. 2.14; the paper obtains it from the symmetry Eq. 2.12):
//   c_n = (2/pi)(n + 1/2) int_0^pi phi(y) sin((n + 1/2) y) dy,
//   phi(y) = int_{cos y}^1 f(x) / sqrt(2(x - cos y)) dx = 2 sin(y/2) g(y),
// with g the row of G that the Abel GEMM (or the plain method) delivers on
// y_j = pi j / L, j = 0..L (L = M/2).  The trapezoid rule on [0, pi] gives
//   c_n = ((2n+1) / L) sum''_{j=0..L} phi_j sin((n + 1/2) pi j / L)
// (end points at half weight; phi_0 = 0), a DST-III of length L.
//
// Fast evaluation.  With m = L - j, sin((n + 1/2) pi (L - m)/L) =
// (-1)^n cos(pi m (2n+1) / (2L)), so the sum is (-1)^n times a DCT-III of
// v_m = phi_{L-m} (v_0 = phi_L enters at half weight, v_L = phi_0 = 0).  A
// DCT-III of length L is the real output z of the length-L inverse DFT of
// the Hermitian sequence W_k = e^{i pi k / M} (v_k - i v_{L-k}), read as
//   DCT-III_{2p} = z_p / 2,   DCT-III_{2p+1} = z_{L-1-p} / 2.
// The factor 2 sin(y/2) of phi merges into the pre-twiddle: with
// theta = pi k / M, v_k = 2 cos(theta) g_{L-k} and v_{L-k} = 2 sin(theta) g_k,
//   W_k = (g_k + g_{L-k}) + e^{2 pi i k / M} (g_{L-k} - g_k),   W_0 = 2 g_L,
// so only the M-th roots of unity of the plan's twiddle table appear.  The
// real-output DFT of length L is one complex FFT of length H = L/2:
//   Y_k = (W_k + conj W_{H-k}) + i e^{2 pi i k / L} (W_k - conj W_{H-k}),
//   zeta = FFT_H(Y) (positive exponent),  zeta_m = z_{2m} + i z_{2m+1},
// and finally c_n = (-1)^n (2n+1) z_{i(n)} / M, i(2p) = p, i(2p+1) = L-1-p.
//
// Against the real-even route of leg_dct16.cu (the same discrete map, Theorem 1
// with the twist as a first difference): the pre-twiddle replaces the fold,
// and there is no recombination after the FFT and no prefix scan, so the
// outputs need no first difference of two large sums.
#include "leg_rtile.cuh"
#include "leg_split.cuh"

namespace {

// zeta = FFT_H(Y) of the row delivered by load(j), j = 0..L (the caller's
// element type converted to the arithmetic type), left in buf[D::pc(m)].
template <class R, int LOG2H, int XE, class Load>
__device__ __forceinline__ void dst16(CxT<R> *buf, int t, const typename Ar<R>::TW *tw, Load load)
{
    using D = D16<LOG2H, XE>;
    using F = Fa<R>;
    using T_ = typename F::T;
    constexpr int E = D::E, T = D::T, H = D::H, L = D::L;
    CxT<R> v[E];
    // W_k and W_{H-k} of the merged pre-twiddle (k < H) from one table entry:
    // e^{2 pi i (H - k) / M} = i e^{-2 pi i k / M} = (s, c) for (c, s) = e^{2 pi i k / M}
    auto wpair = [&](int k, CxT<R> &w, CxT<R> &u) {
        T_ c, s;
        twid(tw, k, c, s);
        if (k == 0) {
            w = {F::pow2(load(L), 1), F::zero()};
        } else {
            const T_ a = load(k), b = load(L - k), d = F::sub(b, a);
            w = {F::add(F::add(a, b), F::mul(c, d)), F::mul(s, d)};
        }
        const T_ a = load(H - k), b = load(H + k), d = F::sub(b, a);
        u = {F::add(F::add(a, b), F::mul(s, d)), F::mul(c, d)};
    };
    // 1. Y_k for k = t + b T
#pragma unroll
    for (int b = 0; b < E; ++b) {
        const int k = t + b * T;
        CxT<R> w, u;
        wpair(k, w, u);
        // W_k + conj W_{H-k} and W_k - conj W_{H-k}
        const T_ pre = F::add(w.re, u.re), pim = F::sub(w.im, u.im);
        const T_ dre = F::sub(w.re, u.re), dim = F::add(w.im, u.im);
        T_ c, s;
        twid(tw, 2 * k, c, s);   // e^{2 pi i k / L}
        // i e^{2 pi i k/L} (dre + i dim) = -(s dre + c dim) + i (c dre - s dim)
        v[b] = {F::sub(pre, F::add(F::mul(s, dre), F::mul(c, dim))),
                F::add(pim, F::sub(F::mul(c, dre), F::mul(s, dim)))};
    }
    fsync<T>();   // load() reads buf (the staged row): all reads precede the first pass's writes
    // 2. FFT of length H
    fft16<R, LOG2H, XE>(v, buf, t, tw);
    fsync<T>();
}

// c[f, n] = (-1)^n (2n+1) z_{i(n)} / M, n < N (or, with rowfn, the first
// n_out coefficients of function rowfn[f] at c + out_off[.]).
template <class R, int LOG2H, int XE>
__global__ void __launch_bounds__(D16<LOG2H, XE>::THREADS, fwd_minb<R, LOG2H, XE>()) dst16_forward_kernel(
    const typename Ar<R>::GT *__restrict__ G, int ldg, typename Ar<R>::OUT *__restrict__ c, int N, int B,
    const typename Ar<R>::TW *__restrict__ tw, const int *__restrict__ rowfn, const long long *__restrict__ out_off,
    const int *__restrict__ n_out)
{
    using D = D16<LOG2H, XE>;
    using F = Fa<R>;
    using T_ = typename F::T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int grp = threadIdx.x / D::T, t = threadIdx.x % D::T;
    CxT<R> *buf = reinterpret_cast<CxT<R> *>(smem_raw) + grp * gslots<R, LOG2H, XE>();
    const int f = min(blockIdx.x * D::FPB + grp, B - 1);   // tail groups recompute the last function
    const bool live = blockIdx.x * D::FPB + grp < B;
    leg_griddep_wait();   // launched as a dependent of the GEMM that writes G
    using GT = typename Ar<R>::GT;
    stage_row<R, LOG2H, XE>(buf, G, ldg, f, t);
    const GT *g = reinterpret_cast<const GT *>(buf);
    dst16<R, LOG2H, XE>(buf, t, tw, [&](int j) -> T_ { return GIn<R>::get(g, j); });
    if (!live) return;
    typename Ar<R>::OUT *cf = c + (size_t)f * N;
    int nn = N;
    if (rowfn) {
        const int fg = rowfn[f];
        cf = c + out_off[fg];
        nn = min(N, n_out[fg]);
    }
    constexpr int L = D::L;
    constexpr int SHIFT = -(LOG2H + 2);   // 1 / M
    for (int n = t; n < nn; n += D::T) {
        const int i = (n & 1) ? L - 1 - (n >> 1) : (n >> 1);
        const CxT<R> zz = buf[D::pc(i >> 1)];
        T_ z = (i & 1) ? zz.im : zz.re;
        if (n & 1) z = F::neg(z);
        cf[n] = out_of(F::norm(F::mul(F::of_int(2 * n + 1), F::pow2(z, SHIFT))));
    }
}

// The exact adjoint of the sine-form map above (v -> gbar = S^T v, S the map
// from a row of G to c), step by step in reverse order (each step's transpose
// for the real inner product, complex values as pairs):
//   zbar_i(n) = (-1)^n (2n+1) v_n / M (zero for the i no n < N reaches);
//   conj(zetabar_m) = zbar_2m - i zbar_2m+1;
//   Ybar = conj(FFT_H(conj(zetabar))) (positive exponent: the transpose of the
//   forward FFT is the negative-exponent DFT);
//   Wbar_k = conj(1 + i e_k) Ybar_k + (1 - i e_{H-k}) conj(Ybar_{H-k}),
//   e_k = e^{2 pi i k / L}, e_{H-k} = -conj(e_k) (0 < k < H);
//   Wbar_0 = (1 - i) Ybar_0, Wbar_H = (1 - i) conj(Ybar_0);
//   gbar_k = (1 - c_k) Re Wbar_k - s_k Im Wbar_k, gbar_{L-k} = (1 + c_k) Re Wbar_k
//   + s_k Im Wbar_k with (c_k, s_k) = e^{2 pi i k / M} (0 < k < H);
//   gbar_L = 2 Re Wbar_0, gbar_H = 2 Re Wbar_H, gbar_0 = 0 (g_0 does not
//   enter the sine form: phi vanishes at y = 0).
// Every gbar index receives exactly one of these terms, so each thread writes
// its own outputs.
// With PLANES (double-float only) the kernel writes, instead of gbar, the
// seven FP16 planes of gbar and its per-function scale (the input of the
// split-FP16 transposed GEMM: sp, rows of npr columns, zero beyond L): the row
// is staged in shared memory after the transform, its maximum reduced over the
// function's threads, and the planes written 8 columns per 16-byte store, the
// same values the separate split of gbar would write.
template <class R, class VIN, int LOG2H, bool PLANES>
__global__ void __launch_bounds__(D16<LOG2H>::THREADS, D16<LOG2H>::MINB) dst16_adjoint_kernel(
    const VIN *__restrict__ v, typename Ar<R>::GT *__restrict__ gbar, int ldg, int N, int B,
    const typename Ar<R>::TW *__restrict__ tw, LegSplitIn sp, int npr)
{
    using D = D16<LOG2H>;
    using F = Fa<R>;
    using T_ = typename F::T;
    constexpr int E = D::E, T = D::T, H = D::H, L = D::L;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int grp = threadIdx.x / T, t = threadIdx.x % T;
    CxT<R> *buf = reinterpret_cast<CxT<R> *>(smem_raw) + grp * gslots<R, LOG2H>();
    const int f = min(blockIdx.x * D::FPB + grp, B - 1);
    const bool live = blockIdx.x * D::FPB + grp < B;
    const VIN *vf = v + (size_t)f * N;
    // (-1)^n (2n+1) v_n / M staged in the exchange buffer (N <= L values of the
    // arithmetic type fit in its 2L words)
    T_ *ws = reinterpret_cast<T_ *>(buf);
    for (int n = t; n < N; n += T) {
        const T_ x = F::mul(F::of_int(2 * n + 1), F::pow2(in_of<R>(vf[n]), -(LOG2H + 2)));
        ws[n] = (n & 1) ? F::neg(x) : x;
    }
    fsync<T>();
    // zbar_i: i < H holds n = 2i, i >= H holds n = 2(L - 1 - i) + 1
    auto zbar = [&](int i) -> T_ {
        const int n = (i < H) ? 2 * i : 2 * (L - 1 - i) + 1;
        return n < N ? ws[n] : F::zero();
    };
    CxT<R> x[E];
#pragma unroll
    for (int b = 0; b < E; ++b) {
        const int m = t + b * T;
        x[b] = {zbar(2 * m), F::neg(zbar(2 * m + 1))};
    }
    fsync<T>();   // the staged values are read before the first pass writes buf
    fft16<R, LOG2H>(x, buf, t, tw);
    fsync<T>();
    if (!PLANES && !live) return;
    // gbar_{ia[b]} = ga[b], gbar_{ib[b]} = gb[b] (k = t + b T: ia = k, ib = L - k;
    // k = 0: ia = L, ib = H; gbar_0 = 0 besides)
    T_ ga[E], gb[E];
#pragma unroll
    for (int b = 0; b < E; ++b) {
        const int k = t + b * T;
        const CxT<R> pk = buf[D::pc(k)], pm = buf[D::pc((H - k) & (H - 1))];
        // Ybar_k = conj(pk), Ybar_{H-k} = conj(pm)
        const T_ yr = pk.re, yi = F::neg(pk.im), mr = pm.re, mi = F::neg(pm.im);
        if (k == 0) {
            ga[b] = F::norm(F::pow2(F::add(yr, yi), 1));
            gb[b] = F::norm(F::pow2(F::sub(yr, yi), 1));
            continue;
        }
        T_ ec, es;
        twid(tw, 2 * k, ec, es);   // e_k = e^{2 pi i k / L}
        const T_ one = F::of_int(1);
        const T_ am = F::sub(one, es), ap = F::add(one, es);
        // Wbar_k = ((1 - es) - i ec) Ybar_k + ((1 + es) + i ec) conj(Ybar_{H-k})
        const T_ wr = F::add(F::add(F::mul(am, yr), F::mul(ec, yi)), F::add(F::mul(ap, mr), F::mul(ec, mi)));
        const T_ wi = F::add(F::sub(F::mul(am, yi), F::mul(ec, yr)), F::sub(F::mul(ec, mr), F::mul(ap, mi)));
        T_ c, sn;
        twid(tw, k, c, sn);        // e^{2 pi i k / M}
        ga[b] = F::norm(F::sub(F::mul(F::sub(one, c), wr), F::mul(sn, wi)));
        gb[b] = F::norm(F::add(F::mul(F::add(one, c), wr), F::mul(sn, wi)));
    }
    if constexpr (!PLANES) {
        typename Ar<R>::GT *gf = gbar + (size_t)f * ldg;
#pragma unroll
        for (int b = 0; b < E; ++b) {
            const int k = t + b * T;
            gf[k == 0 ? L : k] = Ar<R>::to_g(ga[b]);
            gf[k == 0 ? H : L - k] = Ar<R>::to_g(gb[b]);
        }
        if (t == 0) gf[0] = Ar<R>::to_g(F::zero());
    } else {
        static_assert(std::is_same<R, dfl>::value, "planes are written from double-float values");
        fsync<T>();   // every value of buf has been read
        float2 *gs = reinterpret_cast<float2 *>(buf);   // npr <= L + 32 values fit in the buffer
        float m = 0.0f;
#pragma unroll
        for (int b = 0; b < E; ++b) {
            const int k = t + b * T;
            gs[k == 0 ? L : k] = make_float2(ga[b].hi, ga[b].lo);
            gs[k == 0 ? H : L - k] = make_float2(gb[b].hi, gb[b].lo);
            m = fmaxf(m, fmaxf(fabsf(ga[b].hi), fabsf(gb[b].hi)));
        }
        if (t == 0) gs[0] = make_float2(0.0f, 0.0f);
        for (int j = L + 1 + t; j < npr; j += T) gs[j] = make_float2(0.0f, 0.0f);
        // the row maximum over the function's threads
        float *red = reinterpret_cast<float *>(reinterpret_cast<T_ *>(reinterpret_cast<CxT<R> *>(smem_raw) +
                                                                      D::FPB * gslots<R, LOG2H>()) +
                                               grp * D::WARPS);
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, off));
        if ((t & 31) == 0) red[t >> 5] = m;
        fsync<T>();
        float mm = 0.0f;
        for (int w = 0; w < D::WARPS; ++w) mm = fmaxf(mm, red[w]);
        const int e = split_scale_exp(mm);
        if (!live) return;
        if (t == 0) sp.fexp[f] = e;
        const float SC = __int_as_float((127 + sp.fbits) << 23), ISC = __int_as_float((127 - sp.fbits) << 23);
        __half *P = sp.base + (size_t)f * sp.ld;
        for (int c8 = t; c8 < npr / 8; c8 += T) {
            float2 v8[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) v8[i] = gs[8 * c8 + i];
            split_planes8<float2>(v8, e, SC, ISC, P + 8 * c8, sp.pstride);
        }
    }
}

template <class R, class VIN, int LOG2H, bool PLANES>
int launch_adj(const void *v, void *gbar, int ldg, int N, int B, const void *tw, cudaStream_t st,
               const LegSplitIn &sp, int npr)
{
    using D = D16<LOG2H>;
    if (PLANES && (size_t)npr * sizeof(float2) > (size_t)gslots<R, LOG2H>() * sizeof(CxT<R>))
        return leg_set_error(LEG_ERR_UNSUPPORTED, "adjoint planes exceed the exchange buffer");
    auto kern = dst16_adjoint_kernel<R, VIN, LOG2H, PLANES>;
    const size_t smem = d16_smem<R, LOG2H>();
    LEG_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int grid = (B + D::FPB - 1) / D::FPB;
    kern<<<grid, D::THREADS, smem, st>>>(static_cast<const VIN *>(v), static_cast<typename Ar<R>::GT *>(gbar), ldg,
                                         N, B, static_cast<const typename Ar<R>::TW *>(tw), sp, npr);
    LEG_LAUNCH_CHECK("dst16_adjoint_kernel");
    return LEG_OK;
}

template <class R, class VIN, bool PLANES, int LO, int HI>
int dispatch_adj(int lg, const void *v, void *gbar, int ldg, int N, int B, const void *tw, cudaStream_t st,
                 const LegSplitIn &sp, int npr)
{
    if constexpr (LO > HI) {
        return leg_set_error(LEG_ERR_UNSUPPORTED, "transform length out of range");
    } else {
        if (lg == LO) return launch_adj<R, VIN, LO, PLANES>(v, gbar, ldg, N, B, tw, st, sp, npr);
        return dispatch_adj<R, VIN, PLANES, LO + 1, HI>(lg, v, gbar, ldg, N, B, tw, st, sp, npr);
    }
}

template <class R, int LOG2H, int XE>
int launch_fwd(const void *G, int ldg, void *c, int N, int B, const void *tw, cudaStream_t st, const int *rowfn,
               const long long *out_off, const int *n_out)
{
    using D = D16<LOG2H, XE>;
    auto kern = dst16_forward_kernel<R, LOG2H, XE>;
    const size_t smem = d16_smem<R, LOG2H, XE>();
    LEG_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int grid = (B + D::FPB - 1) / D::FPB;
    // programmatic dependent launch, as the real-even transform
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.gridDim = dim3(grid, 1, 1);
    cfg.blockDim = dim3(D::THREADS, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    LEG_CUDA_TRY(cudaLaunchKernelEx(&cfg, kern, static_cast<const typename Ar<R>::GT *>(G), ldg,
                                    static_cast<typename Ar<R>::OUT *>(c), N, B,
                                    static_cast<const typename Ar<R>::TW *>(tw), rowfn, out_off, n_out));
    return LEG_OK;
}

template <class R, int LO, int HI>
int dispatch_fwd(int lg, int xe, const void *G, int ldg, void *c, int N, int B, const void *tw, cudaStream_t st,
                 const int *rowfn, const long long *out_off, const int *n_out)
{
    if constexpr (LO > HI) {
        return leg_set_error(LEG_ERR_UNSUPPORTED, "transform length out of range");
    } else {
        if (lg == LO) {
            // radix 16 differs from radix 8 only from H = 512 on (at least 32 threads of 16 values)
            if constexpr (LO >= 9) {
                if (xe == 4) return launch_fwd<R, LO, 4>(G, ldg, c, N, B, tw, st, rowfn, out_off, n_out);
            }
            return launch_fwd<R, LO, 3>(G, ldg, c, N, B, tw, st, rowfn, out_off, n_out);
        }
        return dispatch_fwd<R, LO + 1, HI>(lg, xe, G, ldg, c, N, B, tw, st, rowfn, out_off, n_out);
    }
}

}  // namespace

// H = 2^log2h with 6 <= log2h <= 13 (M = 4H from 256 to 32768); at most
// 2^log2e values per thread (3: radix-8 passes, 4: radix-16).  dtype
// LEG_F64: FP64 G and c, table of double2; LEG_SPLIT_FP16: double-float G
// (float2), FP32 c, table of float4; LEG_F32 / LEG_BF16: FP32 G and c,
// table of float2.
int leg_dst16_forward(int dtype, int log2h, int log2e, const void *G, int ldg, void *c, int N, int B,
                      const void *tw, cudaStream_t st, const int *rowfn, const long long *out_off, const int *n_out)
{
    switch (dtype) {
    case LEG_F64:
        return dispatch_fwd<double, 6, 13>(log2h, log2e, G, ldg, c, N, B, tw, st, rowfn, out_off, n_out);
    case LEG_SPLIT_FP16:
        return dispatch_fwd<dfl, 6, 13>(log2h, log2e, G, ldg, c, N, B, tw, st, rowfn, out_off, n_out);
    default:
        return dispatch_fwd<float, 6, 13>(log2h, log2e, G, ldg, c, N, B, tw, st, rowfn, out_off, n_out);
    }
}

// The adjoint of leg_dst16_forward (radix-8 passes): v (B x N: FP32 for
// LEG_SPLIT_FP16, FP64 for LEG_F64) to gbar (B x ldg, rows 0..L written).
int leg_dst16_adjoint(int dtype, int log2h, const void *v, void *gbar, int ldg, int N, int B, const void *tw,
                      cudaStream_t st)
{
    const LegSplitIn none = {};
    if (dtype == LEG_F64)
        return dispatch_adj<double, double, false, 6, 13>(log2h, v, gbar, ldg, N, B, tw, st, none, 0);
    return dispatch_adj<dfl, float, false, 6, 13>(log2h, v, gbar, ldg, N, B, tw, st, none, 0);
}

// The split-FP16 adjoint straight into the transposed GEMM's input: the
// planes and scales of sp (B rows of npr columns) instead of gbar.
int leg_dst16_adjoint_planes(int log2h, const float *v, const LegSplitIn &sp, int npr, int N, int B,
                             const void *twdf, cudaStream_t st)
{
    return dispatch_adj<dfl, float, true, 6, 13>(log2h, v, nullptr, 0, N, B, twdf, st, sp, npr);
}
