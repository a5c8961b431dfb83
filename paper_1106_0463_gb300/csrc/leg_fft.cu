// The FFT stage of the method (arXiv:1106.0463, Theorem 1: Eq. 2.4 with the
// twist of Eq. 2.5; the paragraph after Eq. 2.14 takes it by one FFT).
//
// On the grid y_j = 2 pi j / M the Abel step delivers g_j (even: g_j = g_{M-j},
// Eq. 2.12), and Eq. 2.5 reads fhat(y) = (1 - e^{iy}) g(y) / (2 pi).  The
// trapezoid form of Eq. 2.4 is then
//     a_n = (1/M) sum_j (1 - e^{i y_j}) g_j e^{i n y_j} = Ghat_n - Ghat_{n+1},
//     Ghat_n = (1/M) sum_{j<M} g_j e^{i n y_j}  (real, since g is even),
// i.e. the twist is applied exactly as a first difference of the transform
// (shift theorem), and c_n = (2n+1) a_n.  The length-M real transform is
// taken as one length-L = M/2 complex FFT of w_m = g_{2m} + i g_{2m+1}
// followed by the usual even/odd recombination:
//     Re S_n = 1/2 [ (Re W_n + Re W_{L-n}) + cos(2 pi n/M)(Im W_n + Im W_{L-n})
//                    + sin(2 pi n/M)(Re W_n - Re W_{L-n}) ],   Ghat_n = Re S_n / M.
//
// The complex FFT is an in-place shared-memory Stockham transform (radix-4
// stages, one radix-2 stage when log2 L is odd): each thread loads its
// butterflies' operands into registers, the CTA synchronises, and the results
// are written to their autosorted positions.  Positive exponent, no scaling.
// Twiddles e^{2 pi i n/M} come from a table computed in FP64.
//
// The adjoint (leg_backward) is the transposed map: with
// d_n = (2n+1) v_n - (2n-1) v_{n-1}, n = 0..N (v_{-1} = v_N = 0),
//     gbar_j = (w_j / M) sum_n d_n cos(2 pi n j / M),   j = 0..M/2,
// w_0 = w_{M/2} = 1, w_j = 2 otherwise (the mirrored rows folded in), which is
// the same real transform applied to d.
#include "leg_fft.cuh"
#include "leg_internal.cuh"

namespace {

template <int LOG2L> struct FftShape {
    static constexpr int L = 1 << LOG2L;
    static constexpr int TPF = (L / 4 < 1) ? 1 : ((L / 4 > 512) ? 512 : L / 4);
    static constexpr int FPB = (256 / TPF > 1) ? 256 / TPF : 1;
    static constexpr int BPT = (L / 4 >= TPF) ? L / (4 * TPF) : 1;   // radix-4 butterflies / thread
    static constexpr int THREADS = TPF * FPB;
};

template <class R>
__device__ __forceinline__ Cx<typename Ar<R>::T> cmul(Cx<typename Ar<R>::T> a, typename Ar<R>::T c,
                                                      typename Ar<R>::T s)
{
    using A = Ar<R>;
    return {A::sub(A::mul(a.re, c), A::mul(a.im, s)), A::add(A::mul(a.re, s), A::mul(a.im, c))};
}

template <class R>
__device__ __forceinline__ Cx<typename Ar<R>::T> cadd(Cx<typename Ar<R>::T> a, Cx<typename Ar<R>::T> b)
{
    using A = Ar<R>;
    return {A::add(a.re, b.re), A::add(a.im, b.im)};
}

template <class R>
__device__ __forceinline__ Cx<typename Ar<R>::T> csub(Cx<typename Ar<R>::T> a, Cx<typename Ar<R>::T> b)
{
    using A = Ar<R>;
    return {A::sub(a.re, b.re), A::sub(a.im, b.im)};
}

// In-place Stockham FFT of one length-L sequence held in shared memory by the
// TPF threads t = 0..TPF-1 of a function group.  Every thread of the CTA calls
// it (barriers inside).
template <class R, int LOG2L>
__device__ void stockham_fft(Cx<typename Ar<R>::T> *buf, int t, const typename Ar<R>::TW *tw)
{
    using A = Ar<R>;
    using T = typename A::T;
    using C = Cx<T>;
    using S = FftShape<LOG2L>;
    constexpr int L = S::L;
    int Ns = 1;
    if (LOG2L & 1) {   // one radix-2 stage, Ns = 1 (no twiddles)
        constexpr int NB = (L / 2 + S::TPF - 1) / S::TPF;
        C v[NB][2];
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            int j = t + b * S::TPF;
            if (j < L / 2) {
                v[b][0] = buf[j];
                v[b][1] = buf[j + L / 2];
            }
        }
        __syncthreads();
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            int j = t + b * S::TPF;
            if (j < L / 2) {
                buf[2 * j] = cadd<R>(v[b][0], v[b][1]);
                buf[2 * j + 1] = csub<R>(v[b][0], v[b][1]);
            }
        }
        __syncthreads();
        Ns = 2;
    }
#pragma unroll 1
    for (; Ns < L; Ns *= 4) {
        constexpr int NB = S::BPT;
        C v[NB][4];
        const int tstride = L / (2 * Ns);   // twiddle index step in units of 2 pi / M
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            int j = t + b * S::TPF;
            if (j < L / 4) {
                int k = j & (Ns - 1);
#pragma unroll
                for (int r = 0; r < 4; ++r) v[b][r] = buf[j + r * (L / 4)];
                if (k != 0) {
#pragma unroll
                    for (int r = 1; r < 4; ++r) {
                        T c, s;
                        A::tw(tw, r * k * tstride, c, s);
                        v[b][r] = cmul<R>(v[b][r], c, s);
                    }
                }
            }
        }
        __syncthreads();
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            int j = t + b * S::TPF;
            if (j < L / 4) {
                int k = j & (Ns - 1);
                C a = cadd<R>(v[b][0], v[b][2]);
                C bb = csub<R>(v[b][0], v[b][2]);
                C c = cadd<R>(v[b][1], v[b][3]);
                C d = csub<R>(v[b][1], v[b][3]);
                C id = {A::neg(d.im), d.re};                  // i * d
                int base = (j - k) * 4 + k;                   // (j / Ns) * 4 Ns + k
                buf[base] = cadd<R>(a, c);
                buf[base + Ns] = cadd<R>(bb, id);
                buf[base + 2 * Ns] = csub<R>(a, c);
                buf[base + 3 * Ns] = csub<R>(bb, id);
            }
        }
        __syncthreads();
    }
}

// 2 M Ghat_n, the even/odd recombination of the half-length transform W.
template <class R, int LOG2L>
__device__ __forceinline__ typename Ar<R>::T recombine(const Cx<typename Ar<R>::T> *W, int n,
                                                       const typename Ar<R>::TW *tw)
{
    using A = Ar<R>;
    using T = typename A::T;
    constexpr int L = 1 << LOG2L;
    Cx<T> wn = W[n & (L - 1)];
    Cx<T> wm = W[(L - n) & (L - 1)];
    T c, s;
    A::tw(tw, n, c, s);
    T t0 = A::add(wn.re, wm.re);
    T t1 = A::mul(c, A::add(wn.im, wm.im));
    T t2 = A::mul(s, A::sub(wn.re, wm.re));
    return A::add(t0, A::add(t1, t2));
}

template <class R, int LOG2L>
__global__ void __launch_bounds__(FftShape<LOG2L>::THREADS) fft_forward_kernel(
    const typename Ar<R>::GT *__restrict__ G, int ldg, typename Ar<R>::OUT *__restrict__ c,
    int N, int B, const typename Ar<R>::TW *__restrict__ tw)
{
    using A = Ar<R>;
    using T = typename A::T;
    using C = Cx<T>;
    using S = FftShape<LOG2L>;
    constexpr int L = S::L, M = 2 * L;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *buf = reinterpret_cast<C *>(smem_raw) + (threadIdx.x / S::TPF) * L;
    const int t = threadIdx.x % S::TPF;
    const int f = blockIdx.x * S::FPB + threadIdx.x / S::TPF;
    const bool live = f < B;
    const typename A::GT *g = G + (size_t)(live ? f : 0) * ldg;

    // w_m = g_{2m} + i g_{2m+1}; g_j for j > L is g_{M-j}
    for (int m = t; m < L; m += S::TPF) {
        int j0 = 2 * m, j1 = 2 * m + 1;
        j0 = (j0 <= L) ? j0 : M - j0;
        j1 = (j1 <= L) ? j1 : M - j1;
        C w;
        if (live) {
            w.re = A::from_g(g[j0]);
            w.im = A::from_g(g[j1]);
        } else {
            w.re = A::zero();
            w.im = A::zero();
        }
        buf[m] = w;
    }
    __syncthreads();
    stockham_fft<R, LOG2L>(buf, t, tw);
    if (!live) return;
    // c_n = (2n+1) (Ghat_n - Ghat_{n+1});  Ghat = recombine / (2M)
    constexpr int SHIFT = -(LOG2L + 2);   // 1 / (2M) = 2^-(log2 L + 2)
    for (int n = t; n < N; n += S::TPF) {
        T g0 = recombine<R, LOG2L>(buf, n, tw);
        T g1 = recombine<R, LOG2L>(buf, n + 1, tw);
        T a = A::pow2(A::sub(g0, g1), SHIFT);
        c[(size_t)f * N + n] = A::out(A::mul(A::from_int(2 * n + 1), a));
    }
}

template <class R, class VIN, int LOG2L>
__global__ void __launch_bounds__(FftShape<LOG2L>::THREADS) fft_adjoint_kernel(
    const VIN *__restrict__ v, typename Ar<R>::GT *__restrict__ gbar, int ldg, int N, int B,
    const typename Ar<R>::TW *__restrict__ tw)
{
    using A = Ar<R>;
    using T = typename A::T;
    using C = Cx<T>;
    using S = FftShape<LOG2L>;
    constexpr int L = S::L, M = 2 * L;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *buf = reinterpret_cast<C *>(smem_raw) + (threadIdx.x / S::TPF) * L;
    const int t = threadIdx.x % S::TPF;
    const int f = blockIdx.x * S::FPB + threadIdx.x / S::TPF;
    const bool live = f < B;
    const VIN *vf = v + (size_t)(live ? f : 0) * N;

    // z_m = d_{2m} + i d_{2m+1},  d_n = (2n+1) v_n - (2n-1) v_{n-1}, zero beyond n = N
    auto dval = [&](int n) -> T {
        if (!live || n > N) return A::zero();
        T x = A::zero();
        if (n < N) x = A::mul(A::from_int(2 * n + 1), A::from_in(vf[n]));
        if (n >= 1) x = A::sub(x, A::mul(A::from_int(2 * n - 1), A::from_in(vf[n - 1])));
        return x;
    };
    for (int m = t; m < L; m += S::TPF) {
        C z;
        z.re = dval(2 * m);
        z.im = dval(2 * m + 1);
        buf[m] = z;
    }
    __syncthreads();
    stockham_fft<R, LOG2L>(buf, t, tw);
    if (!live) return;
    (void)M;
    for (int j = t; j <= L; j += S::TPF) {
        T s = recombine<R, LOG2L>(buf, j, tw);     // 2 sum_n d_n cos(2 pi n j/M)
        int e = (j == 0 || j == L) ? -(LOG2L + 2) : -(LOG2L + 1);   // w_j / (2M)
        gbar[(size_t)f * ldg + j] = A::to_g(A::pow2(s, e));
    }
}

template <class R, int LOG2L>
int launch_forward(const void *G, int ldg, void *c, int N, int B, const void *tw, cudaStream_t st)
{
    using A = Ar<R>;
    using S = FftShape<LOG2L>;
    size_t smem = sizeof(Cx<typename A::T>) * S::L * S::FPB;
    auto kern = fft_forward_kernel<R, LOG2L>;
    LEG_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int grid = (B + S::FPB - 1) / S::FPB;
    kern<<<grid, S::THREADS, smem, st>>>(static_cast<const typename A::GT *>(G), ldg,
                                         static_cast<typename A::OUT *>(c), N, B,
                                         static_cast<const typename A::TW *>(tw));
    LEG_LAUNCH_CHECK("fft_forward_kernel");
    return LEG_OK;
}

template <class R, class VIN, int LOG2L>
int launch_adjoint(const void *v, void *gbar, int ldg, int N, int B, const void *tw, cudaStream_t st)
{
    using A = Ar<R>;
    using S = FftShape<LOG2L>;
    size_t smem = sizeof(Cx<typename A::T>) * S::L * S::FPB;
    auto kern = fft_adjoint_kernel<R, VIN, LOG2L>;
    LEG_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int grid = (B + S::FPB - 1) / S::FPB;
    kern<<<grid, S::THREADS, smem, st>>>(static_cast<const VIN *>(v),
                                         static_cast<typename A::GT *>(gbar), ldg, N, B,
                                         static_cast<const typename A::TW *>(tw));
    LEG_LAUNCH_CHECK("fft_adjoint_kernel");
    return LEG_OK;
}

// runtime log2 L -> template
template <class R, int LO, int HI>
int dispatch_forward(int lg, const void *G, int ldg, void *c, int N, int B, const void *tw, cudaStream_t st)
{
    if constexpr (LO > HI) {
        return leg_set_error(LEG_ERR_UNSUPPORTED, "FFT length not supported for this precision");
    } else {
        if (lg == LO) return launch_forward<R, LO>(G, ldg, c, N, B, tw, st);
        return dispatch_forward<R, LO + 1, HI>(lg, G, ldg, c, N, B, tw, st);
    }
}

template <class R, class VIN, int LO, int HI>
int dispatch_adjoint(int lg, const void *v, void *gbar, int ldg, int N, int B, const void *tw, cudaStream_t st)
{
    if constexpr (LO > HI) {
        return leg_set_error(LEG_ERR_UNSUPPORTED, "FFT length not supported for this precision");
    } else {
        if (lg == LO) return launch_adjoint<R, VIN, LO>(v, gbar, ldg, N, B, tw, st);
        return dispatch_adjoint<R, VIN, LO + 1, HI>(lg, v, gbar, ldg, N, B, tw, st);
    }
}

int ilog2(int x)
{
    int l = 0;
    while ((1 << l) < x) ++l;
    return l;
}

}  // namespace

int leg_fft_forward(const leg_plan *p, const void *G, int ldg, void *c, int B, cudaStream_t st)
{
    if (B == 0) return LEG_OK;
    const int lg = ilog2(p->L);
    switch (p->dtype) {
    case LEG_F64:
        return dispatch_forward<double, 2, 13>(lg, G, ldg, c, p->N, B, p->tw64, st);
    case LEG_F32:
    case LEG_BF16:
        return dispatch_forward<float, 2, 14>(lg, G, ldg, c, p->N, B, p->tw32, st);
    case LEG_SPLIT_FP16:
        return dispatch_forward<dfl, 2, 13>(lg, G, ldg, c, p->N, B, p->twdf, st);
    }
    return leg_set_error(LEG_ERR_INVALID_ARG, "bad dtype");
}

int leg_fft_adjoint(const leg_plan *p, const void *v, void *gbar, int ldg, int B, cudaStream_t st)
{
    if (B == 0) return LEG_OK;
    const int lg = ilog2(p->L);
    switch (p->dtype) {
    case LEG_F64:
        return dispatch_adjoint<double, double, 2, 13>(lg, v, gbar, ldg, p->N, B, p->tw64, st);
    case LEG_F32:
    case LEG_BF16:
        return dispatch_adjoint<float, float, 2, 14>(lg, v, gbar, ldg, p->N, B, p->tw32, st);
    case LEG_SPLIT_FP16:
        return dispatch_adjoint<dfl, float, 2, 13>(lg, v, gbar, ldg, p->N, B, p->twdf, st);
    }
    return leg_set_error(LEG_ERR_INVALID_ARG, "bad dtype");
}

// Plain-method entry used by leg_plain_forward: FP64 transform of an FP64 G.
int leg_fft_forward_f64(const leg_plan *p, const double *G, int ldg, double *c, int B, cudaStream_t st)
{
    if (B == 0) return LEG_OK;
    return dispatch_forward<double, 2, 13>(ilog2(p->L), G, ldg, c, p->N, B, p->tw64, st);
}
