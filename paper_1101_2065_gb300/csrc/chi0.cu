// a3 + a4: spectral weights of chi0 and their Cauchy transform.
//
// For every matrix element (m, n) of the compressed response, the weights
//   A_j = sum_p 2 w_j(Delta_p) u_pm u_pn      (Eq. chi_by_spectra, spin 2)
// live only on the band of bins j_lo..j_hi.  The deposit (a3) is a
// segmented SYRK over the frequency bins, A_j = U_j^T W_j U_j with U_j the
// pairs of bins j-1 and j and W_j their tent weights, computed by 64 x 64
// element tiles (U staged through shared memory, each U value reused by 64
// outputs) and written once per (bin, element): as A[bin][element] (packed
// lower triangle) on the binary64 path, as TF32 hi/lo operand images for the
// tensor-core product of kk_tc.cu on the binary32 path.
//
// The binary64 path takes the Cauchy integral of Eq. chi_by_spectra on the
// grid,
//   chi0_k = sum_j A_j [kap(k-j) - kap(k+j)],  kap(d) = 1/(d dw + i eta),
// by FFT: a Toeplitz part plus a Hankel part, both exact circular products
// of length L = 2 n_omega:
//   chi0 = IFFT( FFT(A) C1 - conj(FFT(A)) C2 )[0..n_omega)
// where C1 = FFT of kap(d) on d in (-(N-1), N-1) (index d mod L) and
// C2 = FFT of kap(d) on d in [0, 2N-2] (the Hankel sum is a correlation).
// Two real elements share one forward complex FFT; the FFT kernel reads its
// two elements' band from A.
#include <cmath>
#include <cstdint>

#include "internal.h"
#include "kk_layout.cuh"
#include "tc.cuh"

namespace {

// Mixed-radix Stockham FFT in shared memory (natural order in and out):
// one radix-2 or radix-4 pass first (no twiddles), then radix-8 passes.
// The radix-8 passes read their twiddles from per-pass tables
// [w^k | w^2k | w^4k], k < Ns, w = exp(-2 pi i c / L), c = L / (8 Ns),
// built once per CTA (build_pass_twiddles), so consecutive butterflies read
// consecutive entries.  The inverse uses conjugate twiddles and rotations
// (unnormalised).  Returns the buffer holding the result (a or b).  All
// threads of the CTA must call it.
template <typename C>
__device__ __forceinline__ C tw_at(const C* __restrict__ tw, int t, int L) {   // exp(-2 pi i t / L), 0 <= t < L
    const int h = L >> 1;
    if (t < h) return tw[t];
    C w = tw[t - h];
    w.x = -w.x;
    w.y = -w.y;
    return w;
}
// FFT buffers in shared memory are padded by one entry per 16 (index fp(i)):
// the strided writes of the first two passes then fall in distinct banks.
__host__ __device__ __forceinline__ int fp(int i) { return i + (i >> 4); }
__host__ __device__ __forceinline__ int fft_buf_len(int L) { return L + (L >> 4); }
__device__ __forceinline__ int first_radix(int logL) { return logL % 3 == 1 ? 2 : logL % 3 == 2 ? 4 : 1; }
__host__ __device__ __forceinline__ int pass_twiddle_count(int logL) {   // entries of all per-pass tables
    int Ns = logL % 3 == 1 ? 2 : logL % 3 == 2 ? 4 : 1, tot = 0;
    for (int s = 0; s < logL / 3; ++s, Ns *= 8) tot += 3 * Ns;
    return tot;
}
// tw = exp(-2 pi i t / L), t < L/2 (global); ptw = per-pass tables (shared)
template <typename C>
__device__ void build_pass_twiddles(C* ptw, const C* __restrict__ tw, int L, int logL) {
    int Ns = first_radix(logL), off = 0;
    for (int s = 0; s < logL / 3; ++s, Ns *= 8) {
        const int c = L / (8 * Ns);
        for (int t = threadIdx.x; t < 3 * Ns; t += blockDim.x) {
            const int r = t / Ns, k = t % Ns;            // r = 0, 1, 2 -> power 1, 2, 4
            ptw[off + t] = tw_at(tw, (1 << r) * k * c, L);
        }
        off += 3 * Ns;
    }
}
template <typename C, bool INV>
__device__ __forceinline__ C rot_mi(C z) {        // z * (-i) forward, z * (+i) inverse
    C r;
    if (INV) { r.x = -z.y; r.y = z.x; }
    else { r.x = z.y; r.y = -z.x; }
    return r;
}
template <typename C, bool INV>
__device__ __forceinline__ void dft4(C& z0, C& z1, C& z2, C& z3) {
    const C c0 = cadd(z0, z2), c1 = csub(z0, z2), c2 = cadd(z1, z3), c3 = rot_mi<C, INV>(csub(z1, z3));
    z0 = cadd(c0, c2);
    z2 = csub(c0, c2);
    z1 = cadd(c1, c3);
    z3 = csub(c1, c3);
}
template <typename C, bool INV>
__device__ __forceinline__ void dft8(C (&x)[8]) {
    typedef decltype(x[0].x) R;
    const R s = R(0.70710678118654752440);
    C a[4], b[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        a[r] = cadd(x[r], x[r + 4]);
        b[r] = csub(x[r], x[r + 4]);
    }
    // b_r *= w8^r (forward w8 = exp(-i pi/4))
    {
        C t = b[1];
        if (INV) { b[1].x = s * (t.x - t.y); b[1].y = s * (t.x + t.y); }
        else { b[1].x = s * (t.x + t.y); b[1].y = s * (t.y - t.x); }
        b[2] = rot_mi<C, INV>(b[2]);
        t = b[3];
        if (INV) { b[3].x = -s * (t.x + t.y); b[3].y = s * (t.x - t.y); }
        else { b[3].x = s * (t.y - t.x); b[3].y = -s * (t.x + t.y); }
    }
    dft4<C, INV>(a[0], a[1], a[2], a[3]);
    dft4<C, INV>(b[0], b[1], b[2], b[3]);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        x[2 * q] = a[q];
        x[2 * q + 1] = b[q];
    }
}

// One Stockham pass of radix RAD on L points, Ns = product of the radices
// before it; ptw = this pass's table (radix 8 only).
template <typename C, int RAD, bool INV>
__device__ __forceinline__ void stockham_pass(const C* __restrict__ a, C* __restrict__ b, int L, int Ns,
                                              const C* __restrict__ ptw) {
    const int nb = L / RAD;
    for (int j = threadIdx.x; j < nb; j += blockDim.x) {
        const int k = j & (Ns - 1);
        C x[RAD];
#pragma unroll
        for (int r = 0; r < RAD; ++r) x[r] = a[fp(j + r * nb)];
        if constexpr (RAD == 8) {
            C w1 = ptw[k], w2 = ptw[Ns + k], w4 = ptw[2 * Ns + k];
            if (INV) { w1.y = -w1.y; w2.y = -w2.y; w4.y = -w4.y; }
            const C w3 = cmul(w1, w2), w5 = cmul(w1, w4), w6 = cmul(w2, w4), w7 = cmul(w3, w4);
            x[1] = cmul(x[1], w1); x[2] = cmul(x[2], w2); x[3] = cmul(x[3], w3);
            x[4] = cmul(x[4], w4); x[5] = cmul(x[5], w5); x[6] = cmul(x[6], w6); x[7] = cmul(x[7], w7);
            dft8<C, INV>(x);
        } else if constexpr (RAD == 4) {
            dft4<C, INV>(x[0], x[1], x[2], x[3]);       // first pass: Ns = 1, no twiddles
        } else {
            const C u0 = x[0];
            x[0] = cadd(u0, x[1]);
            x[1] = csub(u0, x[1]);
        }
        const int base = (j - k) * RAD + k;
#pragma unroll
        for (int q = 0; q < RAD; ++q) b[fp(base + q * Ns)] = x[q];
    }
}

template <typename C>
__device__ C* fft_smem(C* a, C* b, int L, int logL, const C* ptw, bool inverse) {
    int Ns = 1;
    const int rem = logL % 3;
    if (rem == 1) {
        if (inverse) stockham_pass<C, 2, true>(a, b, L, Ns, ptw); else stockham_pass<C, 2, false>(a, b, L, Ns, ptw);
        Ns *= 2;
    } else if (rem == 2) {
        if (inverse) stockham_pass<C, 4, true>(a, b, L, Ns, ptw); else stockham_pass<C, 4, false>(a, b, L, Ns, ptw);
        Ns *= 4;
    }
    if (rem) {
        __syncthreads();
        C* t = a; a = b; b = t;
    }
    for (int s = 0; s < logL / 3; ++s) {
        if (inverse) stockham_pass<C, 8, true>(a, b, L, Ns, ptw); else stockham_pass<C, 8, false>(a, b, L, Ns, ptw);
        ptw += 3 * Ns;
        Ns *= 8;
        __syncthreads();
        C* t = a; a = b; b = t;
    }
    return a;
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

// per-pass twiddle tables of the FFT in global memory (one CTA)
template <typename C>
__global__ void k_pass_twiddles(const C* __restrict__ tw, int L, int logL, C* __restrict__ ptw) {
    build_pass_twiddles(ptw, tw, L, logL);
}

// C1 and C2 (one CTA each): build the kernel sequence, forward FFT.
__global__ void k_kernel_spectra(const double2* __restrict__ tw, int N, int logL, double dw, double eta,
                                 double2* __restrict__ C1, double2* __restrict__ C2) {
    extern __shared__ double2 sbuf[];
    const int L = 2 * N, LB = fft_buf_len(L);
    double2* a = sbuf;
    double2* b = sbuf + LB;
    double2* tws = sbuf + 2 * LB;
    build_pass_twiddles(tws, tw, L, logL);
    for (int d = threadIdx.x; d < L; d += blockDim.x) {
        double2 v = make_double2(0.0, 0.0);
        if (blockIdx.x == 0) {
            if (d <= N - 1) v = kappa(d, dw, eta);
            else if (d >= N + 1) v = kappa((long long)d - L, dw, eta);
        } else {
            if (d <= 2 * N - 2) v = kappa(d, dw, eta);
        }
        a[fp(d)] = v;
    }
    __syncthreads();
    double2* r = fft_smem(a, b, L, logL, (const double2*)tws, false);
    double2* out = blockIdx.x == 0 ? C1 : C2;
    for (int d = threadIdx.x; d < L; d += blockDim.x) out[d] = r[fp(d)];
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

// lower-triangular tile index tt -> (I, J), J <= I
__device__ __forceinline__ void tile_ij(int tt, int& I, int& J) {
    I = (int)((sqrtf(8.0f * tt + 1.0f) - 1.0f) * 0.5f);
    while (I * (I + 1) / 2 > tt) --I;
    while ((I + 1) * (I + 2) / 2 <= tt) ++I;
    J = tt - I * (I + 1) / 2;
}

// a3: A[b][e] = sum_p w_bp u_pm u_pn for output bin b (band index; bin
// j_lo + b), e = m(m+1)/2 + n, n <= m.  Bin b takes the pairs of segment b
// with weight 2(1 - f_p) and of segment b-1 with weight 2 f_p (tent, spin 2);
// those pairs are contiguous in the sorted table: [seg[b-1], seg[b+1]).
// Tile (I, J) of 64 x 64 elements = blockIdx.x, bins [blockIdx.y BC, + BC).
// With Asplit given (binary32 path), the weights are written instead as
// TF32 hi/lo operand images for the tensor-core Kramers-Kronig product
// (kk_layout.cuh).
// four consecutive entries of a 16-byte aligned shared-memory row
__device__ __forceinline__ void load4(const float* p, float (&v)[4]) {
    const float4 q = *reinterpret_cast<const float4*>(p);
    v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
}
__device__ __forceinline__ void load4(const double* p, double (&v)[4]) {
    const double2 q0 = *reinterpret_cast<const double2*>(p), q1 = *reinterpret_cast<const double2*>(p + 2);
    v[0] = q0.x; v[1] = q0.y; v[2] = q1.x; v[3] = q1.y;
}

// asynchronous copy of one R from global (bytes = 0: zero fill) into shared memory
__device__ __forceinline__ void cp_async_r(float* dst, const float* src, bool in) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(d), "l"(src), "r"(in ? 4 : 0) : "memory");
}
__device__ __forceinline__ void cp_async_r(double* dst, const double* src, bool in) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(d), "l"(src), "r"(in ? 8 : 0) : "memory");
}

constexpr int DEP_T = 64, DEP_KC = 32, DEP_TP = DEP_T + 4;   // row pitch: 16-byte aligned rows
template <typename R> constexpr size_t dep_smem() { return sizeof(R) * 2 * (2 * DEP_KC * DEP_TP + DEP_KC); }

// Segmented SYRK of the spectral weights: bin b of a CTA's range takes the
// pairs of bins b - 1 and b (contiguous in the sorted pair order, [lo, hi))
// with their tent weights.  Chunks of 32 pairs are copied asynchronously
// (cp.async) into two buffers, the next chunk (possibly of the next bin) in
// flight while the current one is summed; the weight multiplies the staged
// row value in the inner loop (the same product as weighting it before
// staging).
template <typename R>
__global__ void __launch_bounds__(256) k_deposit_syrk(const R* __restrict__ Ut, int n_pair, int n_sub,
                                                      const int* __restrict__ seg, const double* __restrict__ frac,
                                                      int nb_bins, int BC, long long n_el, R* __restrict__ A,
                                                      uint32_t* __restrict__ Asplit, long long n_et) {
    constexpr int T = DEP_T, KC = DEP_KC, TP = DEP_TP;
    extern __shared__ __align__(16) unsigned char sraw_dep[];
    R (*Um)[KC][TP] = reinterpret_cast<R (*)[KC][TP]>(sraw_dep);                 // [2][pair][row m]: u_pm
    R (*Un)[KC][TP] = Um + 2;                                                   // [2][pair][column n]: u_pn
    R (*sW)[KC] = reinterpret_cast<R (*)[KC]>(Un + 2);                          // [2][pair]: tent weight
    int I, J;
    tile_ij(blockIdx.x, I, J);
    const int m0 = I * T, n0 = J * T;
    const int band = nb_bins + 1;
    const int b0 = blockIdx.y * BC, b1 = min(b0 + BC, band);
    // each thread: rows m0 + 4 ty .. + 3, columns n0 + 4 tx .. + 3 (four consecutive entries of
    // a staged row per vector load)
    const int tid = threadIdx.x, ty = tid / 16, tx = tid % 16;
    auto bin_lo = [&](int b) { return seg[b > 0 ? b - 1 : 0]; };
    auto bin_hi = [&](int b) { return seg[b < nb_bins ? b + 1 : nb_bins]; };
    // the chunk after (b, p0) in the CTA's sequence, skipping bins without pairs; b = b1: none
    auto next_chunk = [&](int& b, int& p0) {
        if (p0 + KC < bin_hi(b)) { p0 += KC; return; }
        for (++b; b < b1; ++b)
            if (bin_lo(b) < bin_hi(b)) { p0 = bin_lo(b); return; }
    };
    auto stage = [&](int b, int p0, int buf) {
        const int mid = seg[b], hi = bin_hi(b);
        for (int t = tid; t < KC * T; t += blockDim.x) {
            const int r = t / KC, k = t % KC, p = p0 + k;
            const bool inp = p < hi;
            cp_async_r(&Um[buf][k][r], Ut + (inp && m0 + r < n_sub ? (long long)(m0 + r) * n_pair + p : 0),
                       inp && m0 + r < n_sub);
            cp_async_r(&Un[buf][k][r], Ut + (inp && n0 + r < n_sub ? (long long)(n0 + r) * n_pair + p : 0),
                       inp && n0 + r < n_sub);
        }
        if (tid < KC) {
            const int p = p0 + tid;
            sW[buf][tid] = p < hi ? R(p < mid ? 2.0 * frac[p] : 2.0 * (1.0 - frac[p])) : R(0);
        }
        asm volatile("cp.async.commit_group;\n" ::: "memory");
    };
    // first chunk of the range
    int sb = b0, sp = 0;
    while (sb < b1 && bin_lo(sb) >= bin_hi(sb)) ++sb;
    if (sb < b1) {
        sp = bin_lo(sb);
        stage(sb, sp, 0);
    }
    int buf = 0;
    for (int b = b0; b < b1; ++b) {
        const int lo = bin_lo(b), hi = bin_hi(b);
        R acc[4][4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] = R(0);
        for (int p0 = lo; p0 < hi; p0 += KC) {
            // this chunk (b, p0) is in buffer buf; stage the one after it
            next_chunk(sb, sp);
            if (sb < b1) {
                stage(sb, sp, buf ^ 1);
                asm volatile("cp.async.wait_group 1;\n" ::: "memory");
            } else {
                asm volatile("cp.async.wait_group 0;\n" ::: "memory");
            }
            __syncthreads();
            const int kc = min(KC, hi - p0);
            for (int k = 0; k < kc; ++k) {
                R a[4], c[4];
                load4(&Um[buf][k][4 * ty], a);
                load4(&Un[buf][k][4 * tx], c);
                const R w = sW[buf][k];
#pragma unroll
                for (int i = 0; i < 4; ++i) a[i] = w * a[i];
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], c[j], acc[i][j]);
            }
            __syncthreads();                          // buffer buf is refilled two chunks later
            buf ^= 1;
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int m = m0 + 4 * ty + i;
            if (m >= n_sub) continue;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int n = n0 + 4 * tx + j;
                if (n > m) continue;
                const long long e = (long long)m * (m + 1) / 2 + n;
                if (Asplit) {
                    uint32_t hi_, lo_;
                    tc::split_tf32((float)acc[i][j], hi_, lo_);
                    const long long w = kk::weight_word(b, e, n_et);
                    Asplit[w] = hi_;
                    Asplit[w + kk::TILE_WORDS] = lo_;
                } else {
                    A[(long long)b * n_el + e] = acc[i][j];
                }
            }
        }
    }
}

template <typename C> struct Real;
template <> struct Real<double2> { typedef double T; static __device__ double2 make(double a, double b) { return make_double2(a, b); } };

template <typename C>
__global__ void __launch_bounds__(256) k_chi0_fft(const typename Real<C>::T* __restrict__ A, int n_sub,
                                                  int j_lo, int nb_bins, int N, int logL,
                                                  const C* __restrict__ ptw, const C* __restrict__ C1,
                                                  const C* __restrict__ C2, C* __restrict__ chi0) {
    typedef typename Real<C>::T R;
    extern __shared__ __align__(16) unsigned char sraw[];
    C* sbuf = reinterpret_cast<C*>(sraw);
    const int L = 2 * N, LB = fft_buf_len(L);
    const int band = nb_bins + 1;
    const long long n_el = (long long)n_sub * (n_sub + 1) / 2;
    const long long n_grp = (n_el + 1) / 2;
    const R scale = R(1.0 / (double)L);
    C* B0 = sbuf;
    C* B1 = sbuf + LB;
    C* B2 = sbuf + 2 * LB;
    const C* tws = ptw;                    // per-pass twiddle tables (global, cached)
    for (long long g = blockIdx.x; g < n_grp; g += gridDim.x) {
        const bool two = 2 * g + 1 < n_el;
        for (int d = threadIdx.x; d < LB; d += blockDim.x) B0[d] = Real<C>::make(R(0), R(0));
        __syncthreads();
        for (int b = threadIdx.x; b < band; b += blockDim.x) {
            const R* Ab = A + (long long)b * n_el + 2 * g;
            B0[fp(j_lo + b)] = Real<C>::make(Ab[0], two ? Ab[1] : R(0));
        }
        __syncthreads();
        C* Zb = fft_smem(B0, B1, L, logL, (const C*)tws, false);
        C* Y1 = (Zb == B0) ? B1 : B0;
        // split the two real transforms and apply the kernel spectra
        for (int m = threadIdx.x; m <= N; m += blockDim.x) {
            int mr = (L - m) & (L - 1);
            C zm = Zb[fp(m)], zr = Zb[fp(mr)];
            // X1 = (Z[m] + conj Z[L-m])/2, X2 = (Z[m] - conj Z[L-m])/(2i)
            const R h = R(0.5);
            C x1 = Real<C>::make(h * (zm.x + zr.x), h * (zm.y - zr.y));
            C x2 = Real<C>::make(h * (zm.y + zr.y), -h * (zm.x - zr.x));
            C c1m = C1[m], c2m = C2[m], c1r = C1[mr], c2r = C2[mr];
            C y1m = csub(cmul(x1, c1m), cmul(cconj(x1), c2m));
            C y2m = csub(cmul(x2, c1m), cmul(cconj(x2), c2m));
            C y1r = csub(cmul(cconj(x1), c1r), cmul(x1, c2r));
            C y2r = csub(cmul(cconj(x2), c1r), cmul(x2, c2r));
            Y1[fp(m)] = y1m;
            Zb[fp(m)] = y2m;
            if (mr != m) { Y1[fp(mr)] = y1r; Zb[fp(mr)] = y2r; }
        }
        __syncthreads();
        C* r1 = fft_smem(Y1, B2, L, logL, (const C*)tws, true);
        C* free1 = (r1 == Y1) ? B2 : Y1;
        C* r2 = fft_smem(Zb, free1, L, logL, (const C*)tws, true);
        // packed lower triangle: the group's elements are 2g and 2g + 1
        for (int k = threadIdx.x; k < N; k += blockDim.x) {
            C v1 = r1[fp(k)];
            C* row = chi0 + (long long)k * n_el + 2 * g;
            row[0] = Real<C>::make(v1.x * scale, v1.y * scale);
            if (two) {
                C v2 = r2[fp(k)];
                row[1] = Real<C>::make(v2.x * scale, v2.y * scale);
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

__global__ void k_to_f64(const float* __restrict__ a, double* __restrict__ b, long long n) {
    long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t < n) b[t] = (double)a[t];
}

}  // namespace

void launch_to_f32(gw_ctx* ctx, const double* a, float* b, long long n) {
    if (n > 0) klaunch(ctx, "k_to_f32", k_to_f32, div_up(n, 256), 256, 0, a, b, n);
}

void launch_to_f64(gw_ctx* ctx, const float* a, double* b, long long n) {
    if (n > 0) klaunch(ctx, "k_to_f64", k_to_f64, div_up(n, 256), 256, 0, a, b, n);
}

void launch_fft_tables(gw_ctx* ctx, gw_chi0* c) {
    const int L = c->L, N = c->grid.n_omega;
    c->tw = dalloc<double2>(ctx, L / 2);
    c->C1 = dalloc<double2>(ctx, L);
    c->C2 = dalloc<double2>(ctx, L);
    klaunch(ctx, "k_twiddles", k_twiddles, div_up(L / 2, 256), 256, 0, c->tw, L);
    size_t smem = (2 * (size_t)fft_buf_len(L) + pass_twiddle_count(c->logL)) * sizeof(double2);
    allow_max_smem(k_kernel_spectra);
    klaunch(ctx, "k_kernel_spectra", k_kernel_spectra, 2, 256, smem, c->tw, N, c->logL, c->grid.d_omega, c->grid.eta, c->C1, c->C2);
}

template <typename R>
static void deposit(gw_ctx* ctx, const gw_chi0* c, const R* Ut, R* A, long long n_el, uint32_t* Asplit = nullptr) {
    const int n = c->n_sub, band = c->nb_bins + 1;
    const int nt = div_up(n, 64), tiles = nt * (nt + 1) / 2;
    // bins per CTA: about eight CTAs per SM in all
    const int BC = std::max(1, (int)std::min<long long>(band, (long long)tiles * band / (8LL * ctx->num_sms)));
    const int nbc = div_up(band, BC);
    if (nbc > 65535) gw_throw(GW_ERR_INVALID_ARG, "spectral band too wide for the deposit kernel");
    allow_max_smem(k_deposit_syrk<R>);
    klaunch(ctx, sizeof(R) == 4 ? "k_deposit_syrk32" : "k_deposit_syrk", k_deposit_syrk<R>, dim3(tiles, nbc), 256,
            dep_smem<R>(), Ut, c->n_pair, n, (const int*)c->seg, (const double*)c->pFrac, c->nb_bins, BC, n_el, A, Asplit,
            kk::elem_tiles(n_el));
}

void launch_chi0_fft(gw_ctx* ctx, gw_chi0* c) {
    const int L = c->L, N = c->grid.n_omega, n = c->n_sub;
    size_t smem = 3 * (size_t)fft_buf_len(L) * sizeof(double2);
    if (smem > 227 * 1024) gw_throw(GW_ERR_INVALID_ARG, "n_omega too large for the FFT kernel");
    const int ntw = pass_twiddle_count(c->logL);
    int per_sm = std::max(1, (int)((228 * 1024) / (smem + 1024)));
    const long long n_el = (long long)n * (n + 1) / 2;
    long long n_grp = (n_el + 1) / 2;
    int grid = (int)std::min<long long>(n_grp, (long long)ctx->num_sms * per_sm);
    const size_t band = (size_t)c->nb_bins + 1;
    double* A = dalloc<double>(ctx, band * n_el);
    double2* ptw = nullptr;
    try {
        ptw = dalloc<double2>(ctx, std::max(ntw, 1));
        klaunch(ctx, "k_pass_twiddles", k_pass_twiddles<double2>, 1, 256, 0, (const double2*)c->tw, L, c->logL, ptw);
        deposit<double>(ctx, c, c->Ut, A, n_el);
        c->chi0 = dalloc<double2>(ctx, (size_t)N * n_el);
        allow_max_smem(k_chi0_fft<double2>);
        klaunch(ctx, "k_chi0_fft", k_chi0_fft<double2>, grid, 256, smem, (const double*)A, n, c->j_lo, c->nb_bins,
                N, c->logL, (const double2*)ptw, (const double2*)c->C1, (const double2*)c->C2, c->chi0);
    } catch (...) {
        ctx_free(ctx, A);
        ctx_free(ctx, ptw);
        throw;
    }
    ctx_free(ctx, ptw);
    ctx_free(ctx, A);
}

// Weights of a contiguous range of sorted pairs on any grid (second window
// technique): seg [nb_bins + 1] holds absolute pair indices, frac the tent
// fractions of the pairs on that grid; A [nb_bins + 1][n_el] in the working
// precision of the chi0 handle.
void launch_deposit_range(gw_ctx* ctx, const gw_chi0* c, const int* seg, const double* frac, int nb_bins, void* A) {
    const int n = c->n_sub, band = nb_bins + 1;
    const long long n_el = (long long)n * (n + 1) / 2;
    const int nt = div_up(n, 64), tiles = nt * (nt + 1) / 2;
    const int BC = std::max(1, (int)std::min<long long>(band, (long long)tiles * band / (8LL * ctx->num_sms)));
    const int nbc = div_up(band, BC);
    if (nbc > 65535) gw_throw(GW_ERR_INVALID_ARG, "spectral band too wide for the deposit kernel");
    if (c->prec == GW_MIXED) {
        allow_max_smem(k_deposit_syrk<float>);
        klaunch(ctx, "k_deposit_syrk32", k_deposit_syrk<float>, dim3(tiles, nbc), 256, dep_smem<float>(),
                (const float*)c->Ut32, c->n_pair, n, seg, frac, nb_bins, BC, n_el, (float*)A, (uint32_t*)nullptr,
                0LL);
    } else {
        allow_max_smem(k_deposit_syrk<double>);
        klaunch(ctx, "k_deposit_syrk", k_deposit_syrk<double>, dim3(tiles, nbc), 256, dep_smem<double>(),
                (const double*)c->Ut, c->n_pair, n, seg, frac, nb_bins, BC, n_el, (double*)A, (uint32_t*)nullptr,
                0LL);
    }
}

// Binary64 spectral weights A64 [band][n_el] of the binary32 path (near-pole
// policy), deposited from the binary64 U^T.
void launch_spectral64(gw_ctx* ctx, gw_chi0* c) {
    const long long n_el = tri(c->n_sub);
    c->A64 = dalloc<double>(ctx, (size_t)(c->nb_bins + 1) * n_el);
    deposit<double>(ctx, c, c->Ut, c->A64, n_el);
}

void launch_chi0_kk32(gw_ctx* ctx, gw_chi0* c) {
    const int n = c->n_sub, band = c->nb_bins + 1;
    const long long n_el = (long long)n * (n + 1) / 2;
    if (!c->Ut32) {            // U^T in binary32 (normally produced directly by the a2 product)
        c->Ut32 = dalloc<float>(ctx, (size_t)n * c->n_pair);
        launch_to_f32(ctx, c->Ut, c->Ut32, (long long)n * c->n_pair);
    }
    if (ctx->kk_tensor) {
        const size_t words = kk::weight_words(band, n_el);
        uint32_t* Asplit = dalloc<uint32_t>(ctx, words);
        try {
            // padding bins of the last chunk and padding elements of the last tile stay zero
            CUDA_CHECK(cudaMemsetAsync(Asplit, 0, words * sizeof(uint32_t), ctx->stream));
            deposit<float>(ctx, c, c->Ut32, nullptr, n_el, Asplit);
            launch_chi0_kk_tc(ctx, c, Asplit);
        } catch (...) {
            ctx_free(ctx, Asplit);
            throw;
        }
        ctx_free(ctx, Asplit);
    } else {
        float* A = dalloc<float>(ctx, (size_t)band * n_el);
        try {
            deposit<float>(ctx, c, c->Ut32, A, n_el);
            launch_chi0_kk_fma(ctx, c, A);
        } catch (...) {
            ctx_free(ctx, A);
            throw;
        }
        ctx_free(ctx, A);
    }
}

void launch_spectral_readback(gw_ctx* ctx, const gw_chi0* c, int j0, int nj, double* A) {
    long long tot = (long long)c->n_sub * c->n_sub * nj;
    if (tot == 0) return;
    const double* Ut = c->Ut;
    double* tmp = nullptr;
    if (!Ut) {                 // mixed path: U^T exists in binary32 only
        const long long nu = (long long)c->n_sub * c->n_pair;
        tmp = dalloc<double>(ctx, nu);
        launch_to_f64(ctx, c->Ut32, tmp, nu);
        Ut = tmp;
    }
    try {
        klaunch(ctx, "k_spectral_readback", k_spectral_readback, div_up(tot, 256), 256, 0, Ut, c->n_pair, c->n_sub,
                c->seg, c->pFrac, c->j_lo, c->nb_bins, j0, nj, A);
    } catch (...) {
        ctx_free(ctx, tmp);
        throw;
    }
    ctx_free(ctx, tmp);
}
