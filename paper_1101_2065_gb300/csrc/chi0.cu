// a3 + a4: spectral weights of chi0 and their Cauchy transform by FFT.
//
// For every matrix element (m, n) of the compressed response, the weights
//   A_j = sum_p 2 w_j(Delta_p) u_pm u_pn      (Eq. chi_by_spectra, spin 2)
// live only on the band of bins j_lo..j_hi.  The Cauchy integral of
// Eq. chi_by_spectra on the grid,
//   chi0_k = sum_j A_j [kap(k-j) - kap(k+j)],  kap(d) = 1/(d dw + i eta),
// is a Toeplitz part plus a Hankel part.  With L = 2 n_omega both are exact
// circular products of length L:
//   chi0 = IFFT( FFT(A) C1 - conj(FFT(A)) C2 )[0..n_omega)
// where C1 = FFT of kap(d) on d in (-(N-1), N-1) (index d mod L) and
// C2 = FFT of kap(d) on d in [0, 2N-2] (the Hankel sum is a correlation).
// Two real elements share one forward complex FFT.  The deposit of A_j is
// fused into the same CTA (the pair segments of each bin are read from U),
// so A is never written to HBM.
#include <cmath>

#include "internal.h"

namespace {

// Radix-2 Stockham FFT in shared memory (natural order in and out).
// Returns the buffer holding the result (a or b).  All threads of the CTA
// must call it.
template <typename C>
__device__ C* fft_smem(C* a, C* b, int L, int logL, const C* __restrict__ tw, bool inverse) {
    const int half = L >> 1;
    int Ns = 1;
    for (int t = 0; t < logL; ++t, Ns <<= 1) {
        const int stride = half / Ns;   // twiddle index step: L/(2 Ns)
        for (int j = threadIdx.x; j < half; j += blockDim.x) {
            int k = j & (Ns - 1);
            C w = tw[k * stride];
            if (inverse) w.y = -w.y;
            C u0 = a[j];
            C u1 = cmul(a[j + half], w);
            int idx = ((j - k) << 1) + k;
            b[idx] = cadd(u0, u1);
            b[idx + Ns] = csub(u0, u1);
        }
        __syncthreads();
        C* tmp = a; a = b; b = tmp;
    }
    return a;
}

__device__ __forceinline__ void tri_index(long long e, int& m, int& n) {
    // packed lower triangle: e = m(m+1)/2 + n, 0 <= n <= m
    long long mm = (long long)((sqrt(8.0 * (double)e + 1.0) - 1.0) * 0.5);
    while (mm * (mm + 1) / 2 > e) --mm;
    while ((mm + 1) * (mm + 2) / 2 <= e) ++mm;
    m = (int)mm;
    n = (int)(e - mm * (mm + 1) / 2);
}

__global__ void k_twiddles(double2* __restrict__ tw, int L) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= L / 2) return;
    double s, c;
    sincospi(2.0 * (double)k / (double)L, &s, &c);
    tw[k] = make_double2(c, -s);   // exp(-2 pi i k / L)
}

__device__ __forceinline__ double2 kappa(long long d, double dw, double eta) {
    double x = (double)d * dw;
    double den = x * x + eta * eta;
    return make_double2(x / den, -eta / den);
}

// C1 and C2 (one CTA each): build the kernel sequence, forward FFT.
__global__ void k_kernel_spectra(const double2* __restrict__ tw, int N, int logL, double dw, double eta,
                                 double2* __restrict__ C1, double2* __restrict__ C2) {
    extern __shared__ double2 sbuf[];
    const int L = 2 * N;
    double2* a = sbuf;
    double2* b = sbuf + L;
    for (int d = threadIdx.x; d < L; d += blockDim.x) {
        double2 v = make_double2(0.0, 0.0);
        if (blockIdx.x == 0) {
            if (d <= N - 1) v = kappa(d, dw, eta);
            else if (d >= N + 1) v = kappa((long long)d - L, dw, eta);
        } else {
            if (d <= 2 * N - 2) v = kappa(d, dw, eta);
        }
        a[d] = v;
    }
    __syncthreads();
    double2* r = fft_smem(a, b, L, logL, tw, false);
    double2* out = blockIdx.x == 0 ? C1 : C2;
    for (int d = threadIdx.x; d < L; d += blockDim.x) out[d] = r[d];
}

// Tent-deposited weight of bin j = j_lo + b for the element pair (m1,n1),(m2,n2).
template <typename R>
__device__ __forceinline__ void deposit2(int b, int nb_bins, const int* __restrict__ seg,
                                         const double* __restrict__ frac, const R* __restrict__ Ut, int n_pair,
                                         int m1, int n1, int m2, int n2, R& a1, R& a2) {
    a1 = R(0);
    a2 = R(0);
    const R* u1 = Ut + (long long)m1 * n_pair;
    const R* v1 = Ut + (long long)n1 * n_pair;
    const R* u2 = Ut + (long long)m2 * n_pair;
    const R* v2 = Ut + (long long)n2 * n_pair;
    if (b < nb_bins)
        for (int p = seg[b]; p < seg[b + 1]; ++p) {
            R w = R(2.0 * (1.0 - frac[p]));
            a1 = fma(w * u1[p], v1[p], a1);
            a2 = fma(w * u2[p], v2[p], a2);
        }
    if (b >= 1)
        for (int p = seg[b - 1]; p < seg[b]; ++p) {
            R w = R(2.0 * frac[p]);
            a1 = fma(w * u1[p], v1[p], a1);
            a2 = fma(w * u2[p], v2[p], a2);
        }
}

template <typename C> struct Real;
template <> struct Real<double2> { typedef double T; static __device__ double2 make(double a, double b) { return make_double2(a, b); } };
template <> struct Real<float2> { typedef float T; static __device__ float2 make(float a, float b) { return make_float2(a, b); } };

template <typename C>
__global__ void __launch_bounds__(256) k_chi0_fft(const typename Real<C>::T* __restrict__ Ut, int n_pair, int n_sub,
                                                  const int* __restrict__ seg, const double* __restrict__ frac,
                                                  int j_lo, int nb_bins, int N, int logL,
                                                  const C* __restrict__ tw, const C* __restrict__ C1,
                                                  const C* __restrict__ C2, C* __restrict__ chi0) {
    typedef typename Real<C>::T R;
    extern __shared__ __align__(16) unsigned char sraw[];
    C* sbuf = reinterpret_cast<C*>(sraw);
    const int L = 2 * N;
    const int band = nb_bins + 1;
    const long long n_el = (long long)n_sub * (n_sub + 1) / 2;
    const long long n_grp = (n_el + 1) / 2;
    const long long nn = (long long)n_sub * n_sub;
    const R scale = R(1.0 / (double)L);
    C* B0 = sbuf;
    C* B1 = sbuf + L;
    C* B2 = sbuf + 2 * L;
    for (long long g = blockIdx.x; g < n_grp; g += gridDim.x) {
        int m1, n1, m2, n2;
        tri_index(2 * g, m1, n1);
        bool two = 2 * g + 1 < n_el;
        if (two) tri_index(2 * g + 1, m2, n2); else { m2 = m1; n2 = n1; }
        for (int d = threadIdx.x; d < L; d += blockDim.x) B0[d] = Real<C>::make(R(0), R(0));
        __syncthreads();
        for (int b = threadIdx.x; b < band; b += blockDim.x) {
            R a1, a2;
            deposit2<R>(b, nb_bins, seg, frac, Ut, n_pair, m1, n1, m2, n2, a1, a2);
            B0[j_lo + b] = Real<C>::make(a1, two ? a2 : R(0));
        }
        __syncthreads();
        C* Zb = fft_smem(B0, B1, L, logL, tw, false);
        C* Y1 = (Zb == B0) ? B1 : B0;
        // split the two real transforms and apply the kernel spectra
        for (int m = threadIdx.x; m <= N; m += blockDim.x) {
            int mr = (L - m) & (L - 1);
            C zm = Zb[m], zr = Zb[mr];
            // X1 = (Z[m] + conj Z[L-m])/2, X2 = (Z[m] - conj Z[L-m])/(2i)
            const R h = R(0.5);
            C x1 = Real<C>::make(h * (zm.x + zr.x), h * (zm.y - zr.y));
            C x2 = Real<C>::make(h * (zm.y + zr.y), -h * (zm.x - zr.x));
            C c1m = C1[m], c2m = C2[m], c1r = C1[mr], c2r = C2[mr];
            C y1m = csub(cmul(x1, c1m), cmul(cconj(x1), c2m));
            C y2m = csub(cmul(x2, c1m), cmul(cconj(x2), c2m));
            C y1r = csub(cmul(cconj(x1), c1r), cmul(x1, c2r));
            C y2r = csub(cmul(cconj(x2), c1r), cmul(x2, c2r));
            Y1[m] = y1m;
            Zb[m] = y2m;
            if (mr != m) { Y1[mr] = y1r; Zb[mr] = y2r; }
        }
        __syncthreads();
        C* r1 = fft_smem(Y1, B2, L, logL, tw, true);
        C* free1 = (r1 == Y1) ? B2 : Y1;
        C* r2 = fft_smem(Zb, free1, L, logL, tw, true);
        const long long o1 = (long long)m1 * n_sub + n1;
        const long long o2 = (long long)m2 * n_sub + n2;
        for (int k = threadIdx.x; k < N; k += blockDim.x) {
            C v1 = r1[k];
            chi0[(long long)k * nn + o1] = Real<C>::make(v1.x * scale, v1.y * scale);
            if (two) {
                C v2 = r2[k];
                chi0[(long long)k * nn + o2] = Real<C>::make(v2.x * scale, v2.y * scale);
            }
        }
        __syncthreads();
    }
}

__global__ void k_spectral_readback(const double* __restrict__ Ut, int n_pair, int n_sub, const int* __restrict__ seg,
                                    const double* __restrict__ frac, int j_lo, int nb_bins, int j0, int nj,
                                    double* __restrict__ A) {
    long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    long long nn = (long long)n_sub * n_sub;
    if (t >= nn * nj) return;
    int jj = (int)(t / nn);
    int e = (int)(t % nn);
    int m = e / n_sub, n = e % n_sub;
    int b = j0 + jj - j_lo;
    double a = 0.0, dummy = 0.0;
    if (b >= 0 && b <= nb_bins) deposit2<double>(b, nb_bins, seg, frac, Ut, n_pair, m, n, m, n, a, dummy);
    A[t] = a;
}

__global__ void k_to_f32(const double* __restrict__ a, float* __restrict__ b, long long n) {
    long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t < n) b[t] = (float)a[t];
}

}  // namespace

void launch_to_f32(gw_ctx* ctx, const double* a, float* b, long long n) {
    if (n > 0) klaunch(ctx, "k_to_f32", k_to_f32, div_up(n, 256), 256, 0, a, b, n);
}

void launch_fft_tables(gw_ctx* ctx, gw_chi0* c) {
    const int L = c->L, N = c->grid.n_omega;
    c->tw = dalloc<double2>(ctx, L / 2);
    c->C1 = dalloc<double2>(ctx, L);
    c->C2 = dalloc<double2>(ctx, L);
    klaunch(ctx, "k_twiddles", k_twiddles, div_up(L / 2, 256), 256, 0, c->tw, L);
    size_t smem = 2 * (size_t)L * sizeof(double2);
    allow_max_smem(k_kernel_spectra);
    klaunch(ctx, "k_kernel_spectra", k_kernel_spectra, 2, 256, smem, c->tw, N, c->logL, c->grid.d_omega, c->grid.eta, c->C1, c->C2);
}

void launch_chi0_fft(gw_ctx* ctx, gw_chi0* c) {
    const int L = c->L, N = c->grid.n_omega, n = c->n_sub;
    const bool f32 = c->prec == GW_MIXED;
    const size_t csz = f32 ? sizeof(float2) : sizeof(double2);
    size_t smem = 3 * (size_t)L * csz;
    if (smem > 227 * 1024) gw_throw(GW_ERR_INVALID_ARG, "n_omega too large for the FFT kernel");
    int per_sm = std::max(1, (int)((228 * 1024) / (smem + 1024)));
    long long n_grp = ((long long)n * (n + 1) / 2 + 1) / 2;
    int grid = (int)std::min<long long>(n_grp, (long long)ctx->num_sms * per_sm);
    if (f32) {
        c->Ut32 = dalloc<float>(ctx, (size_t)n * c->n_pair);
        c->tw32 = dalloc<float2>(ctx, L / 2);
        c->C1_32 = dalloc<float2>(ctx, L);
        c->C2_32 = dalloc<float2>(ctx, L);
        launch_to_f32(ctx, c->Ut, c->Ut32, (long long)n * c->n_pair);
        launch_to_f32(ctx, (const double*)c->tw, (float*)c->tw32, L);
        launch_to_f32(ctx, (const double*)c->C1, (float*)c->C1_32, 2LL * L);
        launch_to_f32(ctx, (const double*)c->C2, (float*)c->C2_32, 2LL * L);
        c->chi0_32 = dalloc<float2>(ctx, (size_t)N * n * n);
        allow_max_smem(k_chi0_fft<float2>);
        klaunch(ctx, "k_chi0_fft32", k_chi0_fft<float2>, grid, 256, smem, (const float*)c->Ut32, c->n_pair, n,
                (const int*)c->seg, (const double*)c->pFrac, c->j_lo, c->nb_bins, N, c->logL,
                (const float2*)c->tw32, (const float2*)c->C1_32, (const float2*)c->C2_32, c->chi0_32);
    } else {
        c->chi0 = dalloc<double2>(ctx, (size_t)N * n * n);
        allow_max_smem(k_chi0_fft<double2>);
        klaunch(ctx, "k_chi0_fft", k_chi0_fft<double2>, grid, 256, smem, (const double*)c->Ut, c->n_pair, n,
                (const int*)c->seg, (const double*)c->pFrac, c->j_lo, c->nb_bins, N, c->logL,
                (const double2*)c->tw, (const double2*)c->C1, (const double2*)c->C2, c->chi0);
    }
}

void launch_spectral_readback(gw_ctx* ctx, const gw_chi0* c, int j0, int nj, double* A) {
    long long tot = (long long)c->n_sub * c->n_sub * nj;
    if (tot == 0) return;
    klaunch(ctx, "k_spectral_readback", k_spectral_readback, div_up(tot, 256), 256, 0, c->Ut, c->n_pair, c->n_sub, c->seg, c->pFrac,
                                                                   c->j_lo, c->nb_bins, j0, nj, A);
}
