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
__device__ __forceinline__ void deposit2(int b, int nb_bins, const int* __restrict__ seg,
                                         const double* __restrict__ frac, const double* __restrict__ Ut, int n_pair,
                                         int m1, int n1, int m2, int n2, double& a1, double& a2) {
    a1 = 0.0;
    a2 = 0.0;
    const double* u1 = Ut + (long long)m1 * n_pair;
    const double* v1 = Ut + (long long)n1 * n_pair;
    const double* u2 = Ut + (long long)m2 * n_pair;
    const double* v2 = Ut + (long long)n2 * n_pair;
    if (b < nb_bins)
        for (int p = seg[b]; p < seg[b + 1]; ++p) {
            double w = 2.0 * (1.0 - frac[p]);
            a1 = fma(w * u1[p], v1[p], a1);
            a2 = fma(w * u2[p], v2[p], a2);
        }
    if (b >= 1)
        for (int p = seg[b - 1]; p < seg[b]; ++p) {
            double w = 2.0 * frac[p];
            a1 = fma(w * u1[p], v1[p], a1);
            a2 = fma(w * u2[p], v2[p], a2);
        }
}

__global__ void __launch_bounds__(256) k_chi0_fft(const double* __restrict__ Ut, int n_pair, int n_sub,
                                                  const int* __restrict__ seg, const double* __restrict__ frac,
                                                  int j_lo, int nb_bins, int N, int logL,
                                                  const double2* __restrict__ tw, const double2* __restrict__ C1,
                                                  const double2* __restrict__ C2, double2* __restrict__ chi0) {
    extern __shared__ double2 sbuf[];
    const int L = 2 * N;
    const int band = nb_bins + 1;
    const long long n_el = (long long)n_sub * (n_sub + 1) / 2;
    const long long n_grp = (n_el + 1) / 2;
    const long long nn = (long long)n_sub * n_sub;
    const double scale = 1.0 / (double)L;
    double2* B0 = sbuf;
    double2* B1 = sbuf + L;
    double2* B2 = sbuf + 2 * L;
    for (long long g = blockIdx.x; g < n_grp; g += gridDim.x) {
        int m1, n1, m2, n2;
        tri_index(2 * g, m1, n1);
        bool two = 2 * g + 1 < n_el;
        if (two) tri_index(2 * g + 1, m2, n2); else { m2 = m1; n2 = n1; }
        for (int d = threadIdx.x; d < L; d += blockDim.x) B0[d] = make_double2(0.0, 0.0);
        __syncthreads();
        for (int b = threadIdx.x; b < band; b += blockDim.x) {
            double a1, a2;
            deposit2(b, nb_bins, seg, frac, Ut, n_pair, m1, n1, m2, n2, a1, a2);
            B0[j_lo + b] = make_double2(a1, two ? a2 : 0.0);
        }
        __syncthreads();
        double2* Zb = fft_smem(B0, B1, L, logL, tw, false);
        double2* Y1 = (Zb == B0) ? B1 : B0;
        // split the two real transforms and apply the kernel spectra
        for (int m = threadIdx.x; m <= N; m += blockDim.x) {
            int mr = (L - m) & (L - 1);
            double2 zm = Zb[m], zr = Zb[mr];
            // X1 = (Z[m] + conj Z[L-m])/2, X2 = (Z[m] - conj Z[L-m])/(2i)
            double2 x1 = make_double2(0.5 * (zm.x + zr.x), 0.5 * (zm.y - zr.y));
            double2 x2 = make_double2(0.5 * (zm.y + zr.y), -0.5 * (zm.x - zr.x));
            double2 c1m = C1[m], c2m = C2[m], c1r = C1[mr], c2r = C2[mr];
            double2 y1m = csub(cmul(x1, c1m), cmul(cconj(x1), c2m));
            double2 y2m = csub(cmul(x2, c1m), cmul(cconj(x2), c2m));
            double2 y1r = csub(cmul(cconj(x1), c1r), cmul(x1, c2r));
            double2 y2r = csub(cmul(cconj(x2), c1r), cmul(x2, c2r));
            Y1[m] = y1m;
            Zb[m] = y2m;
            if (mr != m) { Y1[mr] = y1r; Zb[mr] = y2r; }
        }
        __syncthreads();
        double2* r1 = fft_smem(Y1, B2, L, logL, tw, true);
        double2* free1 = (r1 == Y1) ? B2 : Y1;
        double2* r2 = fft_smem(Zb, free1, L, logL, tw, true);
        const long long o1 = (long long)m1 * n_sub + n1;
        const long long o2 = (long long)m2 * n_sub + n2;
        for (int k = threadIdx.x; k < N; k += blockDim.x) {
            double2 v1 = r1[k];
            chi0[(long long)k * nn + o1] = make_double2(v1.x * scale, v1.y * scale);
            if (two) {
                double2 v2 = r2[k];
                chi0[(long long)k * nn + o2] = make_double2(v2.x * scale, v2.y * scale);
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
    if (b >= 0 && b <= nb_bins) deposit2(b, nb_bins, seg, frac, Ut, n_pair, m, n, m, n, a, dummy);
    A[t] = a;
}

}  // namespace

void launch_fft_tables(gw_ctx* ctx, gw_chi0* c) {
    const int L = c->L, N = c->grid.n_omega;
    c->tw = dalloc<double2>(ctx, L / 2);
    c->C1 = dalloc<double2>(ctx, L);
    c->C2 = dalloc<double2>(ctx, L);
    klaunch(ctx, "k_twiddles", k_twiddles, div_up(L / 2, 256), 256, 0, c->tw, L);
    size_t smem = 2 * (size_t)L * sizeof(double2);
    CUDA_CHECK(cudaFuncSetAttribute(k_kernel_spectra, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    klaunch(ctx, "k_kernel_spectra", k_kernel_spectra, 2, 256, smem, c->tw, N, c->logL, c->grid.d_omega, c->grid.eta, c->C1, c->C2);
}

void launch_chi0_fft(gw_ctx* ctx, gw_chi0* c) {
    const int L = c->L, N = c->grid.n_omega, n = c->n_sub;
    size_t smem = 3 * (size_t)L * sizeof(double2);
    if (smem > 227 * 1024) gw_throw(GW_ERR_INVALID_ARG, "n_omega too large for the binary64 FFT kernel (max 4096)");
    c->chi0 = dalloc<double2>(ctx, (size_t)N * n * n);
    CUDA_CHECK(cudaFuncSetAttribute(k_chi0_fft, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = std::max(1, (int)((228 * 1024) / (smem + 1024)));
    long long n_grp = ((long long)n * (n + 1) / 2 + 1) / 2;
    int grid = (int)std::min<long long>(n_grp, (long long)ctx->num_sms * per_sm);
    klaunch(ctx, "k_chi0_fft", k_chi0_fft, grid, 256, smem, c->Ut, c->n_pair, n, c->seg, c->pFrac, c->j_lo, c->nb_bins, N,
                                                 c->logL, c->tw, c->C1, c->C2, c->chi0);
}

void launch_spectral_readback(gw_ctx* ctx, const gw_chi0* c, int j0, int nj, double* A) {
    long long tot = (long long)c->n_sub * c->n_sub * nj;
    if (tot == 0) return;
    klaunch(ctx, "k_spectral_readback", k_spectral_readback, div_up(tot, 256), 256, 0, c->Ut, c->n_pair, c->n_sub, c->seg, c->pFrac,
                                                                   c->j_lo, c->nb_bins, j0, nj, A);
}
