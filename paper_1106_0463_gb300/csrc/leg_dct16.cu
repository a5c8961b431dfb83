// Register-tiled real-even transform for the FFT stage (FP64 and double-float).
//
// Same mathematics as the half-length transform in leg_fft.cu (arXiv:1106.0463,
// Theorem 1: Eq. 2.4 with the twist of Eq. 2.5 as a first difference, the
// symmetry Eq. 2.12 folding the M-point real-even sequence to L + 1 = M/2 + 1
// values, and c_n = (2n+1) a_n):
//   y_j = (x_j + x_{L-j})/2 - sin(pi j/L)(x_j - x_{L-j}),  0 <= j < L,
//   z_m = y_{2m} + i y_{2m+1},  Z = FFT_H(z)  (H = L/2, positive exponent),
//   2 Y_k = (Z_k + conj Z_{H-k}) + e^{2 pi i k/L}(...)  (real-data recombination),
//   X_{2k} = 2 Re Y_k,  X_{2k+1} = X_1 + sum_{k'=1..k} 2 Im Y_{k'},
//   X_1 = x_0 - x_L + 2 sum_{j=1}^{L/2-1} (x_j - x_{L-j}) cos(pi j/L),
// so that X_n = sum_{j<M} g_j cos(2 pi n j/M) for n = 0..L.
//
// The FFT of length H runs register-tiled (leg_rtile.cuh); the fold is
// computed while the first pass reads G, the prefix of Im Y by warp shuffles.
#include "leg_rtile.cuh"

namespace {

// X_0..X_L of the L+1 values delivered by load(j) (the caller's element type
// converted to the arithmetic type), left in Xs[D::px(n)], n = 0..L (a real
// view of buf).  Only X_0..X_{2 kmax + 1} and X_L are exact: the
// recombination skips k > kmax (kmax = H - 1 for all of them).
template <class R, int LOG2H, int XE, class Load>
__device__ __forceinline__ void dct16(CxT<R> *buf, typename Fa<R>::T *wsum, int t, const typename Ar<R>::TW *tw,
                                      int kmax, Load load)
{
    using D = D16<LOG2H, XE>;
    using F = Fa<R>;
    using T_ = typename F::T;
    constexpr int E = D::E, T = D::T, H = D::H, L = D::L;
    CxT<R> v[E];

    // 1. fold into z_m = y_{2m} + i y_{2m+1} for m = t + b T; partial X_1 sum
    T_ part = F::zero();
#pragma unroll
    for (int b = 0; b < E; ++b) {
        const int m = t + b * T;
        T_ yy[2];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int j = 2 * m + u;
            const T_ xj = load(j), xl = load(L - j);
            T_ c, s;
            twid(tw, j, c, s);                 // cos, sin of pi j / L
            const T_ d = F::sub(xj, xl);
            yy[u] = F::sub(F::half(F::add(xj, xl)), F::mul(s, d));
            if (j >= 1 && j < L / 2) part = F::add(part, F::mul(c, d));
        }
        v[b] = {yy[0], yy[1]};
    }
    const T_ x1 = F::norm(F::add(F::sub(load(0), load(L)), F::pow2(fn_sum<R, LOG2H, XE>(part, t, wsum), 1)));
    fsync<T>();   // load() may read buf (the staged row): all reads precede the first pass's writes

    // 2. FFT of length H
    fft16<R, LOG2H, XE>(v, buf, t, tw);
    fsync<T>();

    // 3. recombination for k = t + i T: 2 Re Y_k (= X_2k) and 2 Im Y_k
    T_ ry[E], iy[E];
#pragma unroll
    for (int i = 0; i < E; ++i) {
        const int k = t + i * T;
        ry[i] = F::zero();
        iy[i] = F::zero();
        if (k <= kmax) {                       // outputs above X_{2 kmax + 1} are not wanted
            const CxT<R> za = buf[D::pc(k)], zb = buf[D::pc((H - k) & (H - 1))];
            T_ c, s;
            twid(tw, 2 * k, c, s);             // e^{2 pi i k / L}
            const T_ sre = F::add(za.re, zb.re), dre = F::sub(za.re, zb.re);
            const T_ sim = F::add(za.im, zb.im), dim = F::sub(za.im, zb.im);
            ry[i] = F::norm(F::add(sre, F::add(F::mul(c, sim), F::mul(s, dre))));
            if (k != 0) iy[i] = F::norm(F::add(dim, F::sub(F::mul(s, sim), F::mul(c, dre))));
        }
    }
    T_ xL = F::zero();
    if (t == T - 1) {
        const CxT<R> z0 = buf[D::pc(0)];
        xL = F::norm(F::pow2(F::sub(z0.re, z0.im), 1));   // X_L = 2 Re Y_H
    }
    fsync<T>();
    // 4. X_2k in place; 2 Im Y_k parked in the odd slots
    T_ *Xs = reinterpret_cast<T_ *>(buf);
#pragma unroll
    for (int i = 0; i < E; ++i) {
        const int k = t + i * T;
        Xs[D::px(2 * k)] = ry[i];
        Xs[D::px(2 * k + 1)] = iy[i];
    }
    if (t == T - 1) Xs[D::px(L)] = xL;
    fsync<T>();
    // 5. X_{2k+1} = X_1 + sum_{k' <= k} 2 Im Y_k': each thread scans k = t E .. t E + E - 1
    T_ run = F::zero();
#pragma unroll
    for (int i = 0; i < E; ++i) {
        run = F::add(run, Xs[D::px(2 * (t * E + i) + 1)]);
        iy[i] = run;
    }
    const T_ incl = fn_scan<R, LOG2H, XE>(run, t, wsum);
    const T_ offs = F::add(x1, F::sub(incl, run));   // X_1 + exclusive prefix
#pragma unroll
    for (int i = 0; i < E; ++i) Xs[D::px(2 * (t * E + i) + 1)] = F::norm(F::add(offs, iy[i]));
    fsync<T>();
}


template <class R, int LOG2H, int XE>
__global__ void __launch_bounds__(D16<LOG2H, XE>::THREADS, fwd_minb<R, LOG2H, XE>()) dct16_forward_kernel(
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
    T_ *wsum = reinterpret_cast<T_ *>(reinterpret_cast<CxT<R> *>(smem_raw) + D::FPB * gslots<R, LOG2H, XE>()) + grp * D::WARPS;
    const int f = min(blockIdx.x * D::FPB + grp, B - 1);   // tail groups recompute the last function
    const bool live = blockIdx.x * D::FPB + grp < B;
    leg_griddep_wait();   // launched as a dependent of the GEMM that writes G
    using GT = typename Ar<R>::GT;
    stage_row<R, LOG2H, XE>(buf, G, ldg, f, t);
    const GT *g = reinterpret_cast<const GT *>(buf);
    // c_n for n < N reads X_0..X_N: X_2k for k <= N/2 and X_2k+1 for k <= (N-1)/2
    const int kmax = min(D::H - 1, N / 2);
    dct16<R, LOG2H, XE>(buf, wsum, t, tw, kmax, [&](int j) -> T_ { return GIn<R>::get(g, j); });
    if (!live) return;
    const T_ *Xs = reinterpret_cast<const T_ *>(buf);
    typename Ar<R>::OUT *cf = c + (size_t)f * N;
    int nn = N;
    if (rowfn) {
        const int fg = rowfn[f];
        cf = c + out_off[fg];
        nn = min(N, n_out[fg]);
    }
    constexpr int SHIFT = -(LOG2H + 2);   // 1 / M
    for (int n = t; n < nn; n += D::T) {
        const T_ a = F::pow2(F::sub(Xs[D::px(n)], Xs[D::px(n + 1)]), SHIFT);
        cf[n] = out_of(F::norm(F::mul(F::of_int(2 * n + 1), a)));
    }
}

// gbar[f, j] = (w_j / 2M)(X_j + x_0 + (-1)^j x_L), j = 0..L, for
// x_n = (2n+1) v_n - (2n-1) v_{n-1} (n <= N, zero beyond).
template <class R, class VIN, int LOG2H>
__global__ void __launch_bounds__(D16<LOG2H>::THREADS, D16<LOG2H>::MINB) dct16_adjoint_kernel(
    const VIN *__restrict__ v, typename Ar<R>::GT *__restrict__ gbar, int ldg, int N, int B,
    const typename Ar<R>::TW *__restrict__ tw)
{
    using D = D16<LOG2H>;
    using F = Fa<R>;
    using T_ = typename F::T;
    constexpr int L = D::L;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int grp = threadIdx.x / D::T, t = threadIdx.x % D::T;
    CxT<R> *buf = reinterpret_cast<CxT<R> *>(smem_raw) + grp * gslots<R, LOG2H>();
    T_ *wsum = reinterpret_cast<T_ *>(reinterpret_cast<CxT<R> *>(smem_raw) + D::FPB * gslots<R, LOG2H>()) + grp * D::WARPS;
    const int f = min(blockIdx.x * D::FPB + grp, B - 1);
    const bool live = blockIdx.x * D::FPB + grp < B;
    const VIN *vf = v + (size_t)f * N;
    // w_n = (2n+1) v_n staged in the exchange buffer (N <= L values of the
    // arithmetic type fit in its 2L words), read by the fold below: coalesced
    // loads of the row once, then x_n = w_n - w_{n-1} from shared memory
    T_ *ws = reinterpret_cast<T_ *>(buf);
    for (int n = t; n < N; n += D::T) ws[n] = F::mul(F::of_int(2 * n + 1), in_of<R>(vf[n]));
    fsync<D::T>();
    auto load = [&](int n) -> T_ {
        if (n > N) return F::zero();
        T_ x = F::zero();
        if (n < N) x = ws[n];
        if (n >= 1) x = F::sub(x, ws[n - 1]);
        return x;
    };
    // x_0 and x_L before the transform overwrites the staged values
    const T_ x0 = load(0), xL = load(L);
    dct16<R, LOG2H, LEG_DCT16_LOG2E>(buf, wsum, t, tw, D::H - 1, load);
    if (!live) return;
    const T_ *Xs = reinterpret_cast<const T_ *>(buf);
    for (int j = t; j <= L; j += D::T) {
        const T_ s = F::add(Xs[D::px(j)], F::add(x0, (j & 1) ? F::neg(xL) : xL));
        const int e = (j == 0 || j == L) ? -(LOG2H + 3) : -(LOG2H + 2);
        gbar[(size_t)f * ldg + j] = Ar<R>::to_g(F::norm(F::pow2(s, e)));
    }
}

template <class R, int LOG2H, int XE>
int launch_fwd(const void *G, int ldg, void *c, int N, int B, const void *tw, cudaStream_t st, const int *rowfn,
               const long long *out_off, const int *n_out)
{
    using D = D16<LOG2H, XE>;
    auto kern = dct16_forward_kernel<R, LOG2H, XE>;
    const size_t smem = d16_smem<R, LOG2H, XE>();
    LEG_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int grid = (B + D::FPB - 1) / D::FPB;
    // programmatic dependent launch: CTAs start on SMs the GEMM has left
    // while its last tiles finish, and wait there for G
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

template <class R, class VIN, int LOG2H>
int launch_adj(const void *v, void *gbar, int ldg, int N, int B, const void *tw, cudaStream_t st)
{
    using D = D16<LOG2H>;
    auto kern = dct16_adjoint_kernel<R, VIN, LOG2H>;
    const size_t smem = d16_smem<R, LOG2H>();
    LEG_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int grid = (B + D::FPB - 1) / D::FPB;
    kern<<<grid, D::THREADS, smem, st>>>(static_cast<const VIN *>(v), static_cast<typename Ar<R>::GT *>(gbar), ldg,
                                         N, B, static_cast<const typename Ar<R>::TW *>(tw));
    LEG_LAUNCH_CHECK("dct16_adjoint_kernel");
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

template <class R, class VIN, int LO, int HI>
int dispatch_adj(int lg, const void *v, void *gbar, int ldg, int N, int B, const void *tw, cudaStream_t st)
{
    if constexpr (LO > HI) {
        return leg_set_error(LEG_ERR_UNSUPPORTED, "transform length out of range");
    } else {
        if (lg == LO) return launch_adj<R, VIN, LO>(v, gbar, ldg, N, B, tw, st);
        return dispatch_adj<R, VIN, LO + 1, HI>(lg, v, gbar, ldg, N, B, tw, st);
    }
}

}  // namespace

// H = 2^log2h with 6 <= log2h <= 13 (M = 4H from 256 to 32768); at most
// 2^log2e values per thread (3: radix-8 passes, 4: radix-16).
int leg_dct16_forward(int dtype, int log2h, int log2e, const void *G, int ldg, void *c, int N, int B,
                      const void *tw, cudaStream_t st, const int *rowfn, const long long *out_off, const int *n_out)
{
    if (dtype == LEG_F64)
        return dispatch_fwd<double, 6, 13>(log2h, log2e, G, ldg, c, N, B, tw, st, rowfn, out_off, n_out);
    return dispatch_fwd<dfl, 6, 13>(log2h, log2e, G, ldg, c, N, B, tw, st, rowfn, out_off, n_out);
}

int leg_dct16_adjoint(int dtype, int log2h, const void *v, void *gbar, int ldg, int N, int B, const void *tw,
                      cudaStream_t st)
{
    if (dtype == LEG_F64) return dispatch_adj<double, double, 6, 13>(log2h, v, gbar, ldg, N, B, tw, st);
    return dispatch_adj<dfl, float, 6, 13>(log2h, v, gbar, ldg, N, B, tw, st);
}
