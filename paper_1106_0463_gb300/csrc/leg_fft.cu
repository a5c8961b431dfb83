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
// TWS = log2(M / L): the twiddle table holds the M-th roots of unity.
template <class R, int LOG2L, int TWS = 1>
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
        const int tstride = (L << TWS) / (4 * Ns);   // twiddle index step in units of 2 pi / M
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

// ---------------------------------------------------------------------------
// Real-even transform at half length (FP64 and double-float paths).
//
// X_n = sum_{j<M} g_j cos(2 pi n j / M) = x_0 + (-1)^n x_L + 2 sum_{j=1}^{L-1} x_j cos(pi n j / L)
// (a type-I cosine transform of the L+1 distinct values, L = M/2) is taken with
// ONE complex FFT of length H = L/2:
//   y_j = (x_j + x_{L-j})/2 - sin(pi j/L) (x_j - x_{L-j}),  j = 0..L-1,
//   Y_k = sum_j y_j e^{2 pi i k j / L}  (real data of length L: a complex FFT of
//         z_m = y_{2m} + i y_{2m+1} and the even/odd recombination),
//   X_{2k} = 2 Re Y_k,   X_{2k+1} = X_1 + 2 sum_{k'=1..k} Im Y_{k'},
//   X_1 = x_0 - x_L + 2 sum_{j=1}^{L-1} x_j cos(pi j / L).
// (The symmetric part of y carries the even outputs; the antisymmetric part,
// through 2 sin(a) sin(b) = cos(a-b) - cos(a+b), the differences of the odd
// outputs, which a prefix scan accumulates.)  Half the arithmetic and half the
// shared memory of the length-L transform, so M = 32768 fits one CTA.
template <int LOG2H> struct DctShape {
    using S = FftShape<LOG2H>;
    static constexpr int H = S::L;
    static constexpr int L = 2 * H;
    static constexpr int TPF = S::TPF;
    static constexpr int FPB = S::FPB;
    static constexpr int THREADS = S::THREADS;
    static constexpr int CH = (H + TPF - 1) / TPF;   // Y values per thread in the scan
    static constexpr size_t smem(size_t tsize) { return (2 * tsize) * (H + 1) * FPB + tsize * THREADS + tsize * FPB; }
};

// The transform X_0..X_L of the values x_0..x_L delivered by `load(j)`;
// on return Xs[0..L] holds X (Xs aliases the group's FFT buffer).
template <class R, int LOG2H, class Load>
__device__ void dct1_half(Cx<typename Ar<R>::T> *buf, typename Ar<R>::T *red, typename Ar<R>::T *x1s,
                          int t, int grp, const typename Ar<R>::TW *tw, Load load)
{
    using A = Ar<R>;
    using T = typename A::T;
    using C = Cx<T>;
    using D = DctShape<LOG2H>;
    constexpr int H = D::H, L = D::L, TPF = D::TPF;
    T *Ts = reinterpret_cast<T *>(buf);   // Ts[j] = y_j: z_m = (y_{2m}, y_{2m+1})
    const int tid = threadIdx.x;

    // 1. fold: y_j and y_{L-j}; partial sums of (x_j - x_{L-j}) cos(pi j/L)
    T part = A::zero();
    for (int j = t; j <= L / 2; j += TPF) {
        T xj = load(j), xl = load(L - j);
        T a = A::pow2(A::add(xj, xl), -1);
        T d = A::sub(xj, xl);
        if (j == 0) {
            Ts[0] = a;
        } else if (j == L / 2) {
            Ts[j] = xj;
        } else {
            T c, s;
            A::tw(tw, j, c, s);            // cos, sin of pi j / L = 2 pi j / M
            T sd = A::mul(s, d);
            Ts[j] = A::sub(a, sd);
            Ts[L - j] = A::add(a, sd);
            part = A::add(part, A::mul(c, d));
        }
    }
    red[tid] = part;
    __syncthreads();
    for (int sft = TPF / 2; sft > 0; sft >>= 1) {
        if (t < sft) red[tid] = A::add(red[tid], red[tid + sft]);
        __syncthreads();
    }
    if (t == 0) x1s[grp] = A::add(A::sub(load(0), load(L)), A::pow2(red[tid], 1));
    __syncthreads();

    // 2. complex FFT of length H (twiddles: M-th roots, M = 4H)
    stockham_fft<R, LOG2H, 2>(buf, t, tw);

    // 3. Y_k for this thread's chunk of k, kept in registers
    T ry[D::CH], iy[D::CH];
    T xL = A::zero();
    const int k0 = t * D::CH;
#pragma unroll
    for (int i = 0; i < D::CH; ++i) {
        const int k = k0 + i;
        ry[i] = A::zero();
        iy[i] = A::zero();
        if (k < H) {
            C za = buf[k & (H - 1)], zb = buf[(H - k) & (H - 1)];
            T c, s;
            A::tw(tw, 2 * k, c, s);        // e^{2 pi i k / L}
            T sre = A::add(za.re, zb.re), dre = A::sub(za.re, zb.re);
            T sim = A::add(za.im, zb.im), dim = A::sub(za.im, zb.im);
            // Re Y = (sre + c sim + s dre)/2, Im Y = (dim + s sim - c dre)/2 ; keep 2 Re Y and 2 Im Y
            ry[i] = A::add(sre, A::add(A::mul(c, sim), A::mul(s, dre)));
            iy[i] = (k == 0) ? A::zero() : A::add(dim, A::sub(A::mul(s, sim), A::mul(c, dre)));
        }
    }
    if (t == TPF - 1) {
        C z0 = buf[0];
        xL = A::pow2(A::sub(z0.re, z0.im), 1);   // X_L = 2 Re Y_H
    }
    // local inclusive prefix of 2 Im Y
    T run = A::zero();
#pragma unroll
    for (int i = 0; i < D::CH; ++i) {
        run = A::add(run, iy[i]);
        iy[i] = run;
    }
    red[tid] = run;
    __syncthreads();
    // 4. inclusive scan of the thread totals within the group (Hillis-Steele)
    for (int off = 1; off < TPF; off <<= 1) {
        T v = (t >= off) ? red[tid - off] : A::zero();
        __syncthreads();
        if (t >= off) red[tid] = A::add(red[tid], v);
        __syncthreads();
    }
    const T offs = A::sub(red[tid], run);   // exclusive prefix
    const T x1 = x1s[grp];
    // 5. X into the (now free) buffer
#pragma unroll
    for (int i = 0; i < D::CH; ++i) {
        const int k = k0 + i;
        if (k < H) {
            Ts[2 * k] = ry[i];
            Ts[2 * k + 1] = A::add(x1, A::add(offs, iy[i]));
        }
    }
    if (t == TPF - 1) Ts[L] = xL;
    __syncthreads();
}

// rowfn == nullptr: c is B x N row-major.  Otherwise (ragged batches) row f of
// G belongs to function rowfn[f], whose first n_out[.] coefficients go to
// c + out_off[.].
template <class R, int LOG2H>
__global__ void __launch_bounds__(DctShape<LOG2H>::THREADS) dct_forward_kernel(
    const typename Ar<R>::GT *__restrict__ G, int ldg, typename Ar<R>::OUT *__restrict__ c,
    int N, int B, const typename Ar<R>::TW *__restrict__ tw, const int *__restrict__ rowfn,
    const long long *__restrict__ out_off, const int *__restrict__ n_out)
{
    using A = Ar<R>;
    using T = typename A::T;
    using C = Cx<T>;
    using D = DctShape<LOG2H>;
    constexpr int H = D::H;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int grp = threadIdx.x / D::TPF, t = threadIdx.x % D::TPF;
    C *buf = reinterpret_cast<C *>(smem_raw) + grp * (H + 1);
    T *red = reinterpret_cast<T *>(reinterpret_cast<C *>(smem_raw) + D::FPB * (H + 1));
    T *x1s = red + D::THREADS;
    const int f = blockIdx.x * D::FPB + grp;
    const bool live = f < B;
    const typename A::GT *g = G + (size_t)(live ? f : 0) * ldg;
    auto load = [&](int j) -> T { return live ? A::from_g(g[j]) : A::zero(); };
    dct1_half<R, LOG2H>(buf, red, x1s, t, grp, tw, load);
    if (!live) return;
    const T *Xs = reinterpret_cast<const T *>(buf);
    constexpr int SHIFT = -(LOG2H + 2);   // 1 / M
    typename A::OUT *cf = c + (size_t)f * N;
    int nn = N;
    if (rowfn) {
        const int fg = rowfn[f];
        cf = c + out_off[fg];
        nn = min(N, n_out[fg]);
    }
    for (int n = t; n < nn; n += D::TPF) {
        T a = A::pow2(A::sub(Xs[n], Xs[n + 1]), SHIFT);
        cf[n] = A::out(A::mul(A::from_int(2 * n + 1), a));
    }
}

template <class R, class VIN, int LOG2H>
__global__ void __launch_bounds__(DctShape<LOG2H>::THREADS) dct_adjoint_kernel(
    const VIN *__restrict__ v, typename Ar<R>::GT *__restrict__ gbar, int ldg, int N, int B,
    const typename Ar<R>::TW *__restrict__ tw)
{
    using A = Ar<R>;
    using T = typename A::T;
    using C = Cx<T>;
    using D = DctShape<LOG2H>;
    constexpr int H = D::H, L = D::L;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int grp = threadIdx.x / D::TPF, t = threadIdx.x % D::TPF;
    C *buf = reinterpret_cast<C *>(smem_raw) + grp * (H + 1);
    T *red = reinterpret_cast<T *>(reinterpret_cast<C *>(smem_raw) + D::FPB * (H + 1));
    T *x1s = red + D::THREADS;
    const int f = blockIdx.x * D::FPB + grp;
    const bool live = f < B;
    const VIN *vf = v + (size_t)(live ? f : 0) * N;
    // x_n = d_n = (2n+1) v_n - (2n-1) v_{n-1} for n <= N, zero beyond
    auto load = [&](int n) -> T {
        if (!live || n > N) return A::zero();
        T x = A::zero();
        if (n < N) x = A::mul(A::from_int(2 * n + 1), A::from_in(vf[n]));
        if (n >= 1) x = A::sub(x, A::mul(A::from_int(2 * n - 1), A::from_in(vf[n - 1])));
        return x;
    };
    dct1_half<R, LOG2H>(buf, red, x1s, t, grp, tw, load);
    if (!live) return;
    const T *Xs = reinterpret_cast<const T *>(buf);
    const T x0 = load(0), xL = load(L);
    // gbar_j = (w_j / M) sum_{n<=L} x_n cos(pi n j / L) = (w_j / 2M) (X_j + x_0 + (-1)^j x_L)
    for (int j = t; j <= L; j += D::TPF) {
        T s = A::add(Xs[j], A::add(x0, (j & 1) ? A::neg(xL) : xL));
        int e = (j == 0 || j == L) ? -(LOG2H + 3) : -(LOG2H + 2);
        gbar[(size_t)f * ldg + j] = A::to_g(A::pow2(s, e));
    }
}

template <class R, int LOG2H>
int launch_dct_forward(const void *G, int ldg, void *c, int N, int B, const void *tw, cudaStream_t st,
                       const int *rowfn = nullptr, const long long *out_off = nullptr, const int *n_out = nullptr)
{
    using A = Ar<R>;
    using D = DctShape<LOG2H>;
    const size_t smem = D::smem(sizeof(typename A::T));
    auto kern = dct_forward_kernel<R, LOG2H>;
    LEG_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int grid = (B + D::FPB - 1) / D::FPB;
    kern<<<grid, D::THREADS, smem, st>>>(static_cast<const typename A::GT *>(G), ldg,
                                         static_cast<typename A::OUT *>(c), N, B,
                                         static_cast<const typename A::TW *>(tw), rowfn, out_off, n_out);
    LEG_LAUNCH_CHECK("dct_forward_kernel");
    return LEG_OK;
}

template <class R, class VIN, int LOG2H>
int launch_dct_adjoint(const void *v, void *gbar, int ldg, int N, int B, const void *tw, cudaStream_t st)
{
    using A = Ar<R>;
    using D = DctShape<LOG2H>;
    const size_t smem = D::smem(sizeof(typename A::T));
    auto kern = dct_adjoint_kernel<R, VIN, LOG2H>;
    LEG_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int grid = (B + D::FPB - 1) / D::FPB;
    kern<<<grid, D::THREADS, smem, st>>>(static_cast<const VIN *>(v),
                                         static_cast<typename A::GT *>(gbar), ldg, N, B,
                                         static_cast<const typename A::TW *>(tw));
    LEG_LAUNCH_CHECK("dct_adjoint_kernel");
    return LEG_OK;
}

template <class R, int LO, int HI>
int dispatch_dct_forward(int lg, const void *G, int ldg, void *c, int N, int B, const void *tw, cudaStream_t st,
                         const int *rowfn = nullptr, const long long *out_off = nullptr,
                         const int *n_out = nullptr)
{
    if constexpr (LO > HI) {
        return leg_set_error(LEG_ERR_UNSUPPORTED, "transform length not supported");
    } else {
        if (lg == LO) return launch_dct_forward<R, LO>(G, ldg, c, N, B, tw, st, rowfn, out_off, n_out);
        return dispatch_dct_forward<R, LO + 1, HI>(lg, G, ldg, c, N, B, tw, st, rowfn, out_off, n_out);
    }
}

template <class R, class VIN, int LO, int HI>
int dispatch_dct_adjoint(int lg, const void *v, void *gbar, int ldg, int N, int B, const void *tw, cudaStream_t st)
{
    if constexpr (LO > HI) {
        return leg_set_error(LEG_ERR_UNSUPPORTED, "transform length not supported");
    } else {
        if (lg == LO) return launch_dct_adjoint<R, VIN, LO>(v, gbar, ldg, N, B, tw, st);
        return dispatch_dct_adjoint<R, VIN, LO + 1, HI>(lg, v, gbar, ldg, N, B, tw, st);
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

// The FP64 and double-float transforms take the register-tiled kernels of
// leg_dct16.cu from H = L/2 = 64 up (M >= 256), the shared-memory Stockham
// kernels above below that.
constexpr int DCT16_MIN_LOG2H = 6;

int leg_fft_forward(const leg_plan *p, const void *G, int ldg, void *c, int B, cudaStream_t st)
{
    if (B == 0) return LEG_OK;
    const int lg = ilog2(p->L);
    if (p->fft_variant == LEG_TRANSFORM_SINE && lg - 1 >= DCT16_MIN_LOG2H) {
        const void *tw = p->dtype == LEG_F64 ? (const void *)p->tw64
                         : p->dtype == LEG_SPLIT_FP16 ? (const void *)p->twdf : (const void *)p->tw32;
        return leg_dst16_forward(p->dtype, lg - 1, p->fft_log2e, G, ldg, c, p->N, B, tw, st, nullptr, nullptr,
                                 nullptr);
    }
    switch (p->dtype) {
    case LEG_F64:
        if (p->fft_variant == LEG_TRANSFORM_REG && lg - 1 >= DCT16_MIN_LOG2H)
            return leg_dct16_forward(LEG_F64, lg - 1, p->fft_log2e, G, ldg, c, p->N, B, p->tw64, st, nullptr,
                                     nullptr, nullptr);
        return dispatch_dct_forward<double, 1, 13>(lg - 1, G, ldg, c, p->N, B, p->tw64, st);
    case LEG_F32:
    case LEG_BF16:
        return dispatch_forward<float, 2, 14>(lg, G, ldg, c, p->N, B, p->tw32, st);
    case LEG_SPLIT_FP16:
        if (p->fft_variant == LEG_TRANSFORM_REG && lg - 1 >= DCT16_MIN_LOG2H)
            return leg_dct16_forward(LEG_SPLIT_FP16, lg - 1, p->fft_log2e, G, ldg, c, p->N, B, p->twdf, st,
                                     nullptr, nullptr, nullptr);
        return dispatch_dct_forward<dfl, 1, 13>(lg - 1, G, ldg, c, p->N, B, p->twdf, st);
    }
    return leg_set_error(LEG_ERR_INVALID_ARG, "bad dtype");
}

bool leg_fft_adjoint_writes_planes(const leg_plan *p)
{
    return p->dtype == LEG_SPLIT_FP16 && p->fft_variant == LEG_TRANSFORM_SINE && ilog2(p->L) - 1 >= DCT16_MIN_LOG2H;
}

int leg_fft_adjoint_planes(const leg_plan *p, const void *v, int B, cudaStream_t st)
{
    if (B == 0) return LEG_OK;
    return leg_dst16_adjoint_planes(ilog2(p->L) - 1, static_cast<const float *>(v), leg_split_workspace(p),
                                    leg_adj_depth(p), p->N, B, p->twdf, st);
}

int leg_fft_adjoint(const leg_plan *p, const void *v, void *gbar, int ldg, int B, cudaStream_t st)
{
    if (B == 0) return LEG_OK;
    const int lg = ilog2(p->L);
    switch (p->dtype) {
    case LEG_F64:
        if (p->fft_variant == LEG_TRANSFORM_SINE && lg - 1 >= DCT16_MIN_LOG2H)
            return leg_dst16_adjoint(LEG_F64, lg - 1, v, gbar, ldg, p->N, B, p->tw64, st);
        if (p->fft_variant != LEG_TRANSFORM_STOCKHAM && lg - 1 >= DCT16_MIN_LOG2H)
            return leg_dct16_adjoint(LEG_F64, lg - 1, v, gbar, ldg, p->N, B, p->tw64, st);
        return dispatch_dct_adjoint<double, double, 1, 13>(lg - 1, v, gbar, ldg, p->N, B, p->tw64, st);
    case LEG_F32:
    case LEG_BF16:
        return dispatch_adjoint<float, float, 2, 14>(lg, v, gbar, ldg, p->N, B, p->tw32, st);
    case LEG_SPLIT_FP16:
        if (p->fft_variant == LEG_TRANSFORM_SINE && lg - 1 >= DCT16_MIN_LOG2H)
            return leg_dst16_adjoint(LEG_SPLIT_FP16, lg - 1, v, gbar, ldg, p->N, B, p->twdf, st);
        if (p->fft_variant != LEG_TRANSFORM_STOCKHAM && lg - 1 >= DCT16_MIN_LOG2H)
            return leg_dct16_adjoint(LEG_SPLIT_FP16, lg - 1, v, gbar, ldg, p->N, B, p->twdf, st);
        return dispatch_dct_adjoint<dfl, float, 1, 13>(lg - 1, v, gbar, ldg, p->N, B, p->twdf, st);
    }
    return leg_set_error(LEG_ERR_INVALID_ARG, "bad dtype");
}

// Plain-method entry used by leg_plain_forward: FP64 transform of an FP64 G.
int leg_fft_forward_f64(const leg_plan *p, const double *G, int ldg, double *c, int B, cudaStream_t st)
{
    if (B == 0) return LEG_OK;
    const int lg = ilog2(p->L);
    if (p->fft_variant == LEG_TRANSFORM_SINE && lg - 1 >= DCT16_MIN_LOG2H)
        return leg_dst16_forward(LEG_F64, lg - 1, p->fft_log2e, G, ldg, c, p->N, B, p->tw64, st, nullptr, nullptr,
                                 nullptr);
    if (p->fft_variant == LEG_TRANSFORM_REG && lg - 1 >= DCT16_MIN_LOG2H)
        return leg_dct16_forward(LEG_F64, lg - 1, p->fft_log2e, G, ldg, c, p->N, B, p->tw64, st, nullptr, nullptr,
                                 nullptr);
    return dispatch_dct_forward<double, 1, 13>(lg - 1, G, ldg, c, p->N, B, p->tw64, st);
}

// Ragged batches: the rows of G (double-float) scatter their first n_out
// coefficients into the packed output.
int leg_fft_forward_ragged(const leg_plan *p, const void *G, int ldg, float *c_packed, int B, const int *rowfn,
                           const long long *out_off, const int *n_out, cudaStream_t st)
{
    if (B == 0) return LEG_OK;
    if (p->dtype != LEG_SPLIT_FP16) return leg_set_error(LEG_ERR_UNSUPPORTED, "ragged batches need split plans");
    const int lg = ilog2(p->L);
    if (p->fft_variant == LEG_TRANSFORM_SINE && lg - 1 >= DCT16_MIN_LOG2H)
        return leg_dst16_forward(LEG_SPLIT_FP16, lg - 1, p->fft_log2e, G, ldg, c_packed, p->N, B, p->twdf, st, rowfn,
                                 out_off, n_out);
    if (p->fft_variant == LEG_TRANSFORM_REG && lg - 1 >= DCT16_MIN_LOG2H)
        return leg_dct16_forward(LEG_SPLIT_FP16, lg - 1, p->fft_log2e, G, ldg, c_packed, p->N, B, p->twdf, st, rowfn,
                                 out_off, n_out);
    return dispatch_dct_forward<dfl, 1, 13>(lg - 1, G, ldg, c_packed, p->N, B, p->twdf, st, rowfn, out_off, n_out);
}
