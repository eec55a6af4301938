// a5 + a6: screening and self-energy forms, one frequency per CTA.
//
// a5  M_k = 1 - chi0_k is complex symmetric (chi0 is symmetric in the real
//     product basis, Sec. 4).  It is factorised in place as M_k = L D L^T
//     (unit lower L, diagonal D, no pivoting) by a right-looking blocked
//     algorithm: 16-column panels, diagonal block in shared memory, rows
//     below solved against it, trailing lower triangle updated by 32x32
//     tiles.  chi^RPA_k = M_k^-1 chi0_k = M_k^-1 - 1 (Eq. chi_RPA) is never
//     formed on the hot path: the forms only need M_k^-1.
// a6  c_r(s_k) = q_r^T gamma_k q_r with gamma_k = -(1/pi) Im chi^RPA_k, and
//     q^T chi^RPA q = q^T M^-1 q - q^T q with q real, so
//     c_r = -(1/pi) Im sum_i y_i^2 / d_i,  y = L^-1 q  (one forward
//     substitution per right-hand side; D^-1 in the middle of the
//     symmetric form).  c_r(s_0) = 0 (odd spectral function).
#include <cmath>

#include "internal.h"

namespace {

constexpr int NB = 16;     // panel width
constexpr int TS = 64;     // row tile of the forms update
// Trailing-update tile of the factorisation and right-hand-side columns per
// thread of the forms update: binary64 is issue-bound (small tiles waste
// less on the triangle), binary32 needs register blocking.
template <typename C> struct Tile;
template <> struct Tile<double2> { static constexpr int T = 32, A = 2, CB = 2; };
template <> struct Tile<float2> { static constexpr int T = 64, A = 4, CB = 5; };

template <typename C> struct CT;
template <> struct CT<double2> {
    typedef double R;
    static __device__ __forceinline__ double2 mk(double a, double b) { return make_double2(a, b); }
};
template <> struct CT<float2> {
    typedef float R;
    static __device__ __forceinline__ float2 mk(float a, float b) { return make_float2(a, b); }
};

template <typename C>
__device__ __forceinline__ C cdiv(C a, C b) {
    typedef typename CT<C>::R R;
    R r = R(1) / (b.x * b.x + b.y * b.y);
    return CT<C>::mk((a.x * b.x + a.y * b.y) * r, (a.y * b.x - a.x * b.y) * r);
}

template <typename C>
__device__ __forceinline__ C cfma(C a, C b, C c) {   // c + a*b
    return CT<C>::mk(fma(a.x, b.x, fma(-a.y, b.y, c.x)), fma(a.x, b.y, fma(a.y, b.x, c.y)));
}

template <typename C>
__device__ __forceinline__ C cfms(C a, C b, C c) {   // c - a*b
    return CT<C>::mk(fma(-a.x, b.x, fma(a.y, b.y, c.x)), fma(-a.x, b.y, fma(-a.y, b.x, c.y)));
}

__device__ double block_max(double v, double* red) {
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
        double w = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) w = fmax(w, __shfl_xor_sync(0xffffffffu, w, o));
        if (threadIdx.x == 0) red[32] = w;
    }
    __syncthreads();
    double r = red[32];
    __syncthreads();
    return r;
}

template <typename C>
__global__ void __launch_bounds__(256) k_ldlt(const C* __restrict__ chi0, C* __restrict__ fac, int n,
                                              int N, double* __restrict__ piv, int* status) {
    typedef typename CT<C>::R R;
    __shared__ C S[NB][NB + 1];
    constexpr int TT = Tile<C>::T, TA = Tile<C>::A;
    __shared__ C sL[TT][NB + 1];
    __shared__ C sW[TT][NB + 1];
    __shared__ double red[33];
    const int tid = threadIdx.x;
    const long long nn = (long long)n * n;
    for (int k = blockIdx.x; k < N; k += gridDim.x) {
        const C* X = chi0 + k * nn;
        C* M = fac + k * nn;
        double mx = 0.0;
        for (long long t = tid; t < nn; t += blockDim.x) {
            int i = (int)(t / n), j = (int)(t % n);
            if (j > i) continue;
            C x = X[t];
            C m = CT<C>::mk((i == j ? R(1) : R(0)) - x.x, -x.y);
            M[t] = m;
            mx = fmax(mx, hypot((double)m.x, (double)m.y));
        }
        mx = block_max(mx, red);
        double dmin = INFINITY;
        for (int k0 = 0; k0 < n; k0 += NB) {
            const int kb = min(NB, n - k0), k1 = k0 + kb;
            // (a) diagonal block, unblocked L D L^T in shared memory
            for (int t = tid; t < kb * kb; t += blockDim.x) {
                int i = t / kb, j = t % kb;
                if (j <= i) S[i][j] = M[(long long)(k0 + i) * n + k0 + j];
            }
            __syncthreads();
            for (int j = 0; j < kb; ++j) {
                C d = S[j][j];
                for (int i = j + 1 + tid; i < kb; i += blockDim.x) S[i][j] = cdiv(S[i][j], d);
                __syncthreads();
                for (int t = tid; t < kb * kb; t += blockDim.x) {
                    int i = t / kb, l = t % kb;
                    if (l > j && l <= i) S[i][l] = cfms(cmul(S[i][j], d), S[l][j], S[i][l]);
                }
                __syncthreads();
            }
            for (int t = tid; t < kb * kb; t += blockDim.x) {
                int i = t / kb, j = t % kb;
                if (j <= i) M[(long long)(k0 + i) * n + k0 + j] = S[i][j];
            }
            for (int j = 0; j < kb; ++j) dmin = fmin(dmin, hypot((double)S[j][j].x, (double)S[j][j].y));
            // (b) panel rows below: x D L11^T = a
            for (int r = k1 + tid; r < n; r += blockDim.x) {
                C x[NB];
                C* row = M + (long long)r * n + k0;
#pragma unroll
                for (int j = 0; j < NB; ++j) {
                    if (j < kb) {
                        C a = row[j];
#pragma unroll
                        for (int p = 0; p < NB; ++p)
                            if (p < j) a = cfms(cmul(x[p], S[p][p]), S[j][p], a);
                        x[j] = cdiv(a, S[j][j]);
                    }
                }
#pragma unroll
                for (int j = 0; j < NB; ++j)
                    if (j < kb) row[j] = x[j];
            }
            __syncthreads();
            // (c) trailing update of the lower triangle: M22 -= L21 D L21^T,
            //     TT x TT tiles, TA x TA complex outputs per thread
            const int nt = (n - k1 + TT - 1) / TT;
            const int ntile = nt * (nt + 1) / 2;
            for (int tt = 0; tt < ntile; ++tt) {
                int I = (int)((sqrtf(8.0f * tt + 1.0f) - 1.0f) * 0.5f);
                while (I * (I + 1) / 2 > tt) --I;
                while ((I + 1) * (I + 2) / 2 <= tt) ++I;
                int J = tt - I * (I + 1) / 2;
                const int r0 = k1 + I * TT, c0 = k1 + J * TT;
                for (int t = tid; t < TT * NB; t += blockDim.x) {
                    int rr = t / NB, p = t % NB;
                    C lv = CT<C>::mk(R(0), R(0)), wv = CT<C>::mk(R(0), R(0));
                    if (p < kb) {
                        if (r0 + rr < n) lv = M[(long long)(r0 + rr) * n + k0 + p];
                        if (c0 + rr < n) wv = cmul(M[(long long)(c0 + rr) * n + k0 + p], S[p][p]);
                    }
                    sL[rr][p] = lv;
                    sW[rr][p] = wv;
                }
                __syncthreads();
                const int ty = tid / 16, tx = tid % 16;
                C acc[TA][TA];
#pragma unroll
                for (int a = 0; a < TA; ++a)
#pragma unroll
                    for (int b = 0; b < TA; ++b) acc[a][b] = CT<C>::mk(R(0), R(0));
#pragma unroll
                for (int p = 0; p < NB; ++p) {
                    C l[TA], w[TA];
#pragma unroll
                    for (int a = 0; a < TA; ++a) l[a] = sL[ty + 16 * a][p];
#pragma unroll
                    for (int b = 0; b < TA; ++b) w[b] = sW[tx + 16 * b][p];
#pragma unroll
                    for (int a = 0; a < TA; ++a)
#pragma unroll
                        for (int b = 0; b < TA; ++b) acc[a][b] = cfma(l[a], w[b], acc[a][b]);
                }
#pragma unroll
                for (int a = 0; a < TA; ++a)
#pragma unroll
                    for (int b = 0; b < TA; ++b) {
                        int i = r0 + ty + 16 * a, j = c0 + tx + 16 * b;
                        if (i < n && j <= i) {
                            C* m = M + (long long)i * n + j;
                            *m = csub(*m, acc[a][b]);
                        }
                    }
                __syncthreads();
            }
        }
        if (tid == 0) {
            double ratio = dmin / (mx > 0.0 ? mx : 1.0);
            piv[k] = ratio;
            if (!(dmin > 0.0) || !isfinite(dmin)) atomicOr(status, ST_SINGULAR);
        }
        __syncthreads();
    }
}

// c[r*N + k] = -(1/pi) Im sum_i y_i^2/d_i, y = L_k^-1 q_r, for k >= 1.
template <typename C>
__global__ void __launch_bounds__(256) k_forms(const C* __restrict__ fac, int n, int N,
                                               const double* __restrict__ Q, int R, int RC,
                                               double* __restrict__ c) {
    typedef typename CT<C>::R T;
    constexpr int CB = Tile<C>::CB;
    extern __shared__ __align__(16) unsigned char sraw[];
    C* sY = reinterpret_cast<C*>(sraw);      // [n][RC]
    __shared__ C S[NB][NB + 1];
    __shared__ C sL[TS][NB + 1];
    __shared__ C acc[256];
    const int tid = threadIdx.x;
    const long long nn = (long long)n * n;
    if (blockIdx.x == 0)
        for (int r = tid; r < R; r += blockDim.x) c[(long long)r * N] = 0.0;
    for (int k = 1 + blockIdx.x; k < N; k += gridDim.x) {
        const C* F = fac + k * nn;
        for (int rc0 = 0; rc0 < R; rc0 += RC) {
            const int rc = min(RC, R - rc0);
            for (long long t = tid; t < (long long)n * RC; t += blockDim.x) {
                int i = (int)(t / RC), r = (int)(t % RC);
                sY[t] = CT<C>::mk(r < rc ? T(Q[(long long)i * R + rc0 + r]) : T(0), T(0));
            }
            if (tid < RC) acc[tid] = CT<C>::mk(T(0), T(0));
            __syncthreads();
            for (int k0 = 0; k0 < n; k0 += NB) {
                const int kb = min(NB, n - k0), k1 = k0 + kb;
                for (int t = tid; t < kb * kb; t += blockDim.x) {
                    int i = t / kb, j = t % kb;
                    if (j <= i) S[i][j] = F[(long long)(k0 + i) * n + k0 + j];
                }
                __syncthreads();
                if (tid < rc) {
                    const int r = tid;
                    C a = acc[r];
                    for (int i = 0; i < kb; ++i) {
                        C y = sY[(k0 + i) * RC + r];
                        for (int p = 0; p < i; ++p) y = cfms(S[i][p], sY[(k0 + p) * RC + r], y);
                        sY[(k0 + i) * RC + r] = y;
                        a = cadd(a, cdiv(cmul(y, y), S[i][i]));
                    }
                    acc[r] = a;
                }
                __syncthreads();
                for (int r0 = k1; r0 < n; r0 += TS) {
                    for (int t = tid; t < TS * NB; t += blockDim.x) {
                        int rr = t / NB, p = t % NB;
                        sL[rr][p] = (p < kb && r0 + rr < n) ? F[(long long)(r0 + rr) * n + k0 + p] : CT<C>::mk(T(0), T(0));
                    }
                    __syncthreads();
                    // thread (ty, tx): rows ty + 16a (a < 4), columns tx + 16b (b < CB)
                    const int ty = tid / 16, tx = tid % 16;
                    C acc2[4][CB];
#pragma unroll
                    for (int a = 0; a < 4; ++a)
#pragma unroll
                        for (int b = 0; b < CB; ++b) acc2[a][b] = CT<C>::mk(T(0), T(0));
#pragma unroll
                    for (int p = 0; p < NB; ++p) {
                        C l[4], y[CB];
#pragma unroll
                        for (int a = 0; a < 4; ++a) l[a] = sL[ty + 16 * a][p];
#pragma unroll
                        for (int b = 0; b < CB; ++b) {
                            int r = tx + 16 * b;
                            y[b] = r < RC ? sY[(k0 + p) * RC + r] : CT<C>::mk(T(0), T(0));
                        }
#pragma unroll
                        for (int a = 0; a < 4; ++a)
#pragma unroll
                            for (int b = 0; b < CB; ++b) acc2[a][b] = cfma(l[a], y[b], acc2[a][b]);
                    }
#pragma unroll
                    for (int a = 0; a < 4; ++a) {
                        const int i = r0 + ty + 16 * a;
                        if (i >= n) continue;
#pragma unroll
                        for (int b = 0; b < CB; ++b) {
                            const int r = tx + 16 * b;
                            if (r < rc) sY[i * RC + r] = csub(sY[i * RC + r], acc2[a][b]);
                        }
                    }
                    __syncthreads();
                }
            }
            if (tid < rc) c[(long long)(rc0 + tid) * N + k] = -(double)acc[tid].y / M_PI;
            __syncthreads();
        }
    }
}

// out = M_k^-1 - 1 = chi^RPA_k from the factors (one CTA; test read-back).
__global__ void __launch_bounds__(256) k_ldlt_inverse(const double2* __restrict__ F, int n, double2* __restrict__ X) {
    // column c of X solves L D L^T x = e_c
    for (int col = threadIdx.x; col < n; col += blockDim.x) {
        double2* x = X + (long long)col;      // strided column (row-major X)
        for (int i = 0; i < n; ++i) x[(long long)i * n] = make_double2(i == col ? 1.0 : 0.0, 0.0);
        for (int i = 0; i < n; ++i) {
            double2 y = x[(long long)i * n];
            for (int p = 0; p < i; ++p) y = cfms(F[(long long)i * n + p], x[(long long)p * n], y);
            x[(long long)i * n] = y;
        }
        for (int i = 0; i < n; ++i) x[(long long)i * n] = cdiv(x[(long long)i * n], F[(long long)i * n + i]);
        for (int i = n - 1; i >= 0; --i) {
            double2 y = x[(long long)i * n];
            for (int p = i + 1; p < n; ++p) y = cfms(F[(long long)p * n + i], x[(long long)p * n], y);
            x[(long long)i * n] = y;
        }
        x[(long long)col * n].x -= 1.0;
    }
}

__global__ void k_c64_to_c128(const float2* __restrict__ a, double2* __restrict__ b, long long n) {
    long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t < n) b[t] = make_double2(a[t].x, a[t].y);
}

}  // namespace

void launch_ldlt(gw_ctx* ctx, gw_W* W) {
    const gw_chi0* c = W->chi0;
    const int n = c->n_sub, N = c->grid.n_omega;
    // binary64: 254 registers, one CTA per SM; binary32: 128 registers, two
    int grid = std::min(N, ctx->num_sms * (c->prec == GW_MIXED ? 2 : 1));
    if (c->prec == GW_MIXED)
        klaunch(ctx, "k_ldlt32", k_ldlt<float2>, grid, 256, 0, (const float2*)c->chi0_32, W->fac32, n, N, W->piv,
                ctx->d_status);
    else
        klaunch(ctx, "k_ldlt", k_ldlt<double2>, grid, 256, 0, (const double2*)c->chi0, W->fac, n, N, W->piv,
                ctx->d_status);
}

void launch_forms(gw_ctx* ctx, const gw_W* W, const double* Q, int R, double* cout) {
    const gw_chi0* c = W->chi0;
    const int n = c->n_sub, N = c->grid.n_omega;
    const bool f32 = c->prec == GW_MIXED;
    const size_t csz = f32 ? sizeof(float2) : sizeof(double2);
    const size_t budget = 190 * 1024;
    int rc_max = (int)std::min<size_t>(16 * (f32 ? Tile<float2>::CB : Tile<double2>::CB), budget / (csz * (size_t)n));
    if (rc_max < 1) gw_throw(GW_ERR_INVALID_ARG, "n_sub too large for the forms kernel");
    int chunks = div_up(R, rc_max);
    int RC = f32 ? div_up(R, chunks) : rc_max;     // binary64: full 16-wide column groups
    size_t smem = csz * (size_t)n * RC;
    int grid = std::max(1, std::min(N - 1, ctx->num_sms));
    if (f32) {
        allow_max_smem(k_forms<float2>);
        klaunch(ctx, "k_forms32", k_forms<float2>, grid, 256, smem, (const float2*)W->fac32, n, N, Q, R, RC, cout);
    } else {
        allow_max_smem(k_forms<double2>);
        klaunch(ctx, "k_forms", k_forms<double2>, grid, 256, smem, (const double2*)W->fac, n, N, Q, R, RC, cout);
    }
}

void launch_ldlt_inverse(gw_ctx* ctx, const gw_W* W, int k, double2* out, double2* work) {
    const gw_chi0* c = W->chi0;
    const long long nn = (long long)c->n_sub * c->n_sub;
    const double2* F = W->fac ? W->fac + k * nn : work;
    if (!W->fac) klaunch(ctx, "k_c64_to_c128", k_c64_to_c128, div_up(nn, 256), 256, 0,
                         (const float2*)(W->fac32 + k * nn), work, nn);
    klaunch(ctx, "k_ldlt_inverse", k_ldlt_inverse, 1, 256, 0, F, c->n_sub, out);
}
