// a5 + a6: screening and self-energy forms, batched over all frequencies.
//
// a5  M_k = 1 - chi0_k is complex symmetric (chi0 is symmetric in the real
//     product basis, Sec. 4).  It is factorised in place as M_k = L D L^T
//     (unit lower L, diagonal D, no pivoting) by a right-looking blocked
//     algorithm with NB-column panels.  Each panel step is two launches over
//     all N frequencies at once: k_ldlt_panel (one CTA per frequency: the
//     NB x NB diagonal block factorised by one warp in shared memory, the
//     rows below solved against it one row per thread) and k_ldlt_syrk (the
//     trailing lower triangle M22 -= L21 D L21^T, one CTA per frequency and
//     tile).  The steps are small one by one, but N of them side by side
//     fill the GPU.  chi^RPA_k = M_k^-1 chi0_k = M_k^-1 - 1 (Eq. chi_RPA) is
//     never formed on the hot path: the forms only need M_k^-1.
// a6  c_r(s_k) = q_r^T gamma_k q_r with gamma_k = -(1/pi) Im chi^RPA_k, and
//     q^T chi^RPA q = q^T M^-1 q - q^T q with q real, so
//     c_r = -(1/pi) Im sum_i y_i^2 / d_i,  y = L^-1 q.  All right-hand sides
//     of all frequencies go through the same blocked forward substitution:
//     k_forms_diag solves the NB rows of the diagonal block (one thread per
//     right-hand side) and accumulates y_i^2/d_i in binary64, k_forms_update
//     applies Y_rest -= L_rest,b Y_b.  c_r(s_0) = 0 (odd spectral function).
#include <cmath>

#include "internal.h"

namespace {

// Panel width NB; trailing-update tile T x T with A x A complex outputs per
// thread; forms update tile FT rows x FC right-hand sides, FA x FA per
// thread.  binary64 is issue-bound (1/64 of the binary32 rate): small tiles
// waste less on the triangle and keep the panel row in registers.
template <typename C> struct Tile;
template <> struct Tile<double2> { static constexpr int NB = 16, T = 32, A = 2, FT = 32, FC = 32, FA = 2; };
template <> struct Tile<float2> { static constexpr int NB = 32, T = 64, A = 4, FT = 64, FC = 64, FA = 4; };

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

// lower-triangular tile index tt -> (I, J), J <= I
__device__ __forceinline__ void tri_ij(int tt, int& I, int& J) {
    I = (int)((sqrtf(8.0f * tt + 1.0f) - 1.0f) * 0.5f);
    while (I * (I + 1) / 2 > tt) --I;
    while ((I + 1) * (I + 2) / 2 <= tt) ++I;
    J = tt - I * (I + 1) / 2;
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

// M_k = 1 - chi0_k on the lower triangle; piv[k] = max |M_k|.
template <typename C>
__global__ void __launch_bounds__(256) k_ldlt_init(const C* __restrict__ chi0, C* __restrict__ fac, int n,
                                                   double* __restrict__ piv) {
    typedef typename CT<C>::R R;
    __shared__ double red[33];
    const int k = blockIdx.x;
    const long long nn = (long long)n * n;
    const C* X = chi0 + k * nn;
    C* M = fac + k * nn;
    R mx2 = R(0);     // max |M|^2 in the working precision (binary64 arithmetic is 1/64 rate)
    for (int i = 0; i < n; ++i)
        for (int j = threadIdx.x; j <= i; j += blockDim.x) {
            C x = X[(long long)i * n + j];
            C m = CT<C>::mk((i == j ? R(1) : R(0)) - x.x, -x.y);
            M[(long long)i * n + j] = m;
            mx2 = fmax(mx2, m.x * m.x + m.y * m.y);
        }
    const double mx = block_max((double)mx2, red);
    if (threadIdx.x == 0) piv[k] = sqrt(mx);
}

// Panel k0 of every frequency: factor the diagonal block, then solve the
// rows below, x D L11^T = a.  piv[N + k] carries min |d| between steps; the
// last panel writes piv[k] = min |d| / max |M| and flags a zero pivot.
template <typename C>
__global__ void __launch_bounds__(256, 2) k_ldlt_panel(C* __restrict__ fac, int n, int N, int k0,
                                                    double* __restrict__ piv, int* status) {
    constexpr int NB = Tile<C>::NB;
    __shared__ C S[NB][NB + 1];     // L11 strictly below the diagonal, D on it
    __shared__ C SD[NB][NB + 1];    // SD[j][p] = L_jp d_p
    __shared__ C Dinv[NB];
    const int k = blockIdx.x, tid = threadIdx.x;
    C* A = fac + (long long)k * n * n;
    const int kb = min(NB, n - k0), k1 = k0 + kb;
    for (int t = tid; t < kb * kb; t += blockDim.x) {
        int i = t / kb, j = t % kb;
        if (j <= i) S[i][j] = A[(long long)(k0 + i) * n + k0 + j];
    }
    __syncthreads();
    // unblocked L D L^T of the diagonal block, one column per step: every
    // thread updates pairs (i, l), j < l <= i, with the unscaled column j,
    // then column j is scaled by 1/d_j
    for (int j = 0; j < kb; ++j) {
        const C dinv = cdiv(CT<C>::mk(1, 0), S[j][j]);
        const int m = kb - 1 - j;
        for (int t = tid; t < m * (m + 1) / 2; t += blockDim.x) {
            int ii, ll;
            tri_ij(t, ii, ll);
            const int i = j + 1 + ii, l = j + 1 + ll;
            S[i][l] = cfms(cmul(S[i][j], dinv), S[l][j], S[i][l]);
        }
        __syncthreads();
        if (tid > j && tid < kb) S[tid][j] = cmul(S[tid][j], dinv);
    }
    __syncthreads();
    for (int t = tid; t < kb * kb; t += blockDim.x) {
        int i = t / kb, p = t % kb;
        if (p < i) SD[i][p] = cmul(S[i][p], S[p][p]);
        if (p <= i) A[(long long)(k0 + i) * n + k0 + p] = S[i][p];
    }
    if (tid < kb) Dinv[tid] = cdiv(CT<C>::mk(1, 0), S[tid][tid]);
    __syncthreads();
    C x[NB];
    for (int r = k1 + tid; r < n; r += blockDim.x) {
        C* row = A + (long long)r * n + k0;
#pragma unroll
        for (int j = 0; j < NB; ++j)
            if (j < kb) x[j] = row[j];
#pragma unroll
        for (int j = 0; j < NB; ++j) {
            if (j < kb) {
                C a = x[j];
#pragma unroll
                for (int p = 0; p < NB; ++p)
                    if (p < j) a = cfms(x[p], SD[j][p], a);
                x[j] = cmul(a, Dinv[j]);
            }
            asm volatile("" ::: "memory");   // keep the SD loads of later rows from being hoisted (registers)
        }
#pragma unroll
        for (int j = 0; j < NB; ++j)
            if (j < kb) row[j] = x[j];
    }
    if (tid == 0) {
        typename CT<C>::R d2 = S[0][0].x * S[0][0].x + S[0][0].y * S[0][0].y;
        for (int j = 1; j < kb; ++j) d2 = fmin(d2, S[j][j].x * S[j][j].x + S[j][j].y * S[j][j].y);
        double dm = sqrt((double)d2);
        if (k0 > 0) dm = fmin(dm, piv[N + k]);
        if (k1 < n) piv[N + k] = dm;
        else {
            const double mx = piv[k];
            piv[k] = dm / (mx > 0.0 ? mx : 1.0);
            if (!(dm > 0.0) || !isfinite(dm)) atomicOr(status, ST_SINGULAR);
        }
    }
}

// Trailing update after panel k0: M22 -= L21 D L21^T on the lower triangle,
// tile blockIdx.x of frequency blockIdx.y.
template <typename C>
__global__ void __launch_bounds__(256) k_ldlt_syrk(C* __restrict__ fac, int n, int k0) {
    typedef typename CT<C>::R R;
    constexpr int NB = Tile<C>::NB, TT = Tile<C>::T, TA = Tile<C>::A;
    __shared__ C sL[TT][NB + 1];
    __shared__ C sW[TT][NB + 1];
    __shared__ C dd[NB];
    const int tid = threadIdx.x;
    C* A = fac + (long long)blockIdx.y * n * n;
    const int kb = min(NB, n - k0), k1 = k0 + kb;
    int I, J;
    tri_ij(blockIdx.x, I, J);
    const int r0 = k1 + I * TT, c0 = k1 + J * TT;
    if (tid < NB) dd[tid] = tid < kb ? A[(long long)(k0 + tid) * n + k0 + tid] : CT<C>::mk(R(0), R(0));
    __syncthreads();
    for (int t = tid; t < TT * NB; t += blockDim.x) {
        int rr = t / NB, p = t % NB;
        C lv = CT<C>::mk(R(0), R(0)), wv = CT<C>::mk(R(0), R(0));
        if (p < kb) {
            if (r0 + rr < n) lv = A[(long long)(r0 + rr) * n + k0 + p];
            if (c0 + rr < n) wv = cmul(A[(long long)(c0 + rr) * n + k0 + p], dd[p]);
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
#pragma unroll 8
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
                C* m = A + (long long)i * n + j;
                *m = csub(*m, acc[a][b]);
            }
        }
}

// Forward substitution, diagonal block k0 of frequency k = 1 + blockIdx.x:
// L_bb y_b = y_b for every right-hand side (one thread each), then
// acc_r += y_i^2 / d_i in binary64.  Before the first update the
// right-hand sides are the real q (Q [n][R]); afterwards Y [N-1][n][R].
// The last block writes c[r*N + k] = -(1/pi) Im acc_r.
template <typename C>
__global__ void __launch_bounds__(256, 2) k_forms_diag(const C* __restrict__ fac, int n, int N,
                                                    const double* __restrict__ Q, int R, C* __restrict__ Y,
                                                    double2* __restrict__ accum, double* __restrict__ c, int k0) {
    typedef typename CT<C>::R T;
    constexpr int NB = Tile<C>::NB;
    __shared__ C S[NB][NB + 1];
    __shared__ C dinv[NB];
    const int k = 1 + blockIdx.x, tid = threadIdx.x;
    const C* F = fac + (long long)k * n * n;
    C* Yk = Y + (long long)(k - 1) * n * R;
    const int kb = min(NB, n - k0), k1 = k0 + kb;
    const bool last = k1 == n;
    for (int t = tid; t < kb * kb; t += blockDim.x) {
        int i = t / kb, j = t % kb;
        if (j <= i) S[i][j] = F[(long long)(k0 + i) * n + k0 + j];
    }
    __syncthreads();
    if (tid < kb) dinv[tid] = cdiv(CT<C>::mk(T(1), T(0)), S[tid][tid]);
    __syncthreads();
    for (int r = tid; r < R; r += blockDim.x) {
        C y[NB];
#pragma unroll
        for (int i = 0; i < NB; ++i)
            if (i < kb) {
                const long long o = (long long)(k0 + i) * R + r;
                y[i] = k0 == 0 ? CT<C>::mk(T(Q[o]), T(0)) : Yk[o];
            }
        // this block's y_i^2/d_i summed in the working precision, added to the
        // binary64 running sum once per block
        C part = CT<C>::mk(T(0), T(0));
#pragma unroll
        for (int i = 0; i < NB; ++i)
            if (i < kb) {
                C v = y[i];
#pragma unroll
                for (int p = 0; p < NB; ++p)
                    if (p < i) v = cfms(S[i][p], y[p], v);
                y[i] = v;
                part = cfma(cmul(v, v), dinv[i], part);
                asm volatile("" ::: "memory");
            }
        double2 a = k0 == 0 ? make_double2(0.0, 0.0) : accum[(long long)(k - 1) * R + r];
        a.x += (double)part.x;
        a.y += (double)part.y;
        if (last) {
            c[(long long)r * N + k] = -a.y / M_PI;
            if (k == 1) c[(long long)r * N] = 0.0;
        } else {
            accum[(long long)(k - 1) * R + r] = a;
#pragma unroll
            for (int i = 0; i < NB; ++i)
                if (i < kb) Yk[(long long)(k0 + i) * R + r] = y[i];
        }
    }
}

// Forward substitution update after block k0: Y_rest -= L_rest,b Y_b, rows
// tile blockIdx.x, right-hand-side tile blockIdx.y, frequency 1 + blockIdx.z.
template <typename C>
__global__ void __launch_bounds__(256) k_forms_update(const C* __restrict__ fac, int n, const double* __restrict__ Q,
                                                      int R, C* __restrict__ Y, int k0) {
    typedef typename CT<C>::R T;
    constexpr int NB = Tile<C>::NB, FT = Tile<C>::FT, FC = Tile<C>::FC, FA = Tile<C>::FA;
    __shared__ C sL[FT][NB + 1];
    __shared__ C sY[NB][FC];
    const int tid = threadIdx.x, k = 1 + blockIdx.z;
    const C* F = fac + (long long)k * n * n;
    C* Yk = Y + (long long)(k - 1) * n * R;
    const int kb = min(NB, n - k0), k1 = k0 + kb;
    const int r0 = k1 + blockIdx.x * FT, c0 = blockIdx.y * FC;
    for (int t = tid; t < FT * NB; t += blockDim.x) {
        int rr = t / NB, p = t % NB;
        sL[rr][p] = (p < kb && r0 + rr < n) ? F[(long long)(r0 + rr) * n + k0 + p] : CT<C>::mk(T(0), T(0));
    }
    for (int t = tid; t < NB * FC; t += blockDim.x) {
        int p = t / FC, cc = t % FC;
        sY[p][cc] = (p < kb && c0 + cc < R) ? Yk[(long long)(k0 + p) * R + c0 + cc] : CT<C>::mk(T(0), T(0));
    }
    __syncthreads();
    const int ty = tid / 16, tx = tid % 16;
    C acc[FA][FA];
#pragma unroll
    for (int a = 0; a < FA; ++a)
#pragma unroll
        for (int b = 0; b < FA; ++b) acc[a][b] = CT<C>::mk(T(0), T(0));
#pragma unroll 8
    for (int p = 0; p < NB; ++p) {
        C l[FA], y[FA];
#pragma unroll
        for (int a = 0; a < FA; ++a) l[a] = sL[ty + 16 * a][p];
#pragma unroll
        for (int b = 0; b < FA; ++b) y[b] = sY[p][tx + 16 * b];
#pragma unroll
        for (int a = 0; a < FA; ++a)
#pragma unroll
            for (int b = 0; b < FA; ++b) acc[a][b] = cfma(l[a], y[b], acc[a][b]);
    }
#pragma unroll
    for (int a = 0; a < FA; ++a) {
        const int i = r0 + ty + 16 * a;
        if (i >= n) continue;
#pragma unroll
        for (int b = 0; b < FA; ++b) {
            const int cc = c0 + tx + 16 * b;
            if (cc >= R) continue;
            const long long o = (long long)i * R + cc;
            const C src = k0 == 0 ? CT<C>::mk(T(Q[o]), T(0)) : Yk[o];
            Yk[o] = csub(src, acc[a][b]);
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

template <typename C>
static void ldlt_steps(gw_ctx* ctx, const C* chi0, C* fac, int n, int N, double* piv, const char* const names[3]) {
    constexpr int NB = Tile<C>::NB, TT = Tile<C>::T;
    klaunch(ctx, names[0], k_ldlt_init<C>, N, 256, 0, chi0, fac, n, piv);
    for (int k0 = 0; k0 < n; k0 += NB) {
        klaunch(ctx, names[1], k_ldlt_panel<C>, N, 256, 0, fac, n, N, k0, piv, ctx->d_status);
        const int m = n - std::min(n, k0 + NB);
        if (m == 0) break;
        const int nt = div_up(m, TT);
        klaunch(ctx, names[2], k_ldlt_syrk<C>, dim3(nt * (nt + 1) / 2, N), 256, 0, fac, n, k0);
    }
}

void launch_ldlt(gw_ctx* ctx, gw_W* W) {
    const gw_chi0* c = W->chi0;
    const int n = c->n_sub, N = c->grid.n_omega;
    if (c->prec == GW_MIXED) {
        static const char* const nm[3] = {"k_ldlt32_init", "k_ldlt32_panel", "k_ldlt32_syrk"};
        ldlt_steps<float2>(ctx, (const float2*)c->chi0_32, W->fac32, n, N, W->piv, nm);
    } else {
        static const char* const nm[3] = {"k_ldlt_init", "k_ldlt_panel", "k_ldlt_syrk"};
        ldlt_steps<double2>(ctx, (const double2*)c->chi0, W->fac, n, N, W->piv, nm);
    }
}

template <typename C>
static void forms_steps(gw_ctx* ctx, const C* fac, int n, int N, const double* Q, int R, double* cout,
                        const char* const names[2]) {
    constexpr int NB = Tile<C>::NB, FT = Tile<C>::FT, FC = Tile<C>::FC;
    C* Y = dalloc<C>(ctx, (size_t)(N - 1) * n * R);
    double2* acc = nullptr;
    try {
        acc = dalloc<double2>(ctx, (size_t)(N - 1) * R);
        for (int k0 = 0; k0 < n; k0 += NB) {
            klaunch(ctx, names[0], k_forms_diag<C>, N - 1, 256, 0, fac, n, N, Q, R, Y, acc, cout, k0);
            const int m = n - std::min(n, k0 + NB);
            if (m == 0) break;
            klaunch(ctx, names[1], k_forms_update<C>, dim3(div_up(m, FT), div_up(R, FC), N - 1), 256, 0, fac, n, Q,
                    R, Y, k0);
        }
    } catch (...) {
        ctx_free(ctx, Y);
        ctx_free(ctx, acc);
        throw;
    }
    ctx_free(ctx, Y);
    ctx_free(ctx, acc);
}

void launch_forms(gw_ctx* ctx, const gw_W* W, const double* Q, int R, double* cout) {
    const gw_chi0* c = W->chi0;
    const int n = c->n_sub, N = c->grid.n_omega;
    if (N < 2) gw_throw(GW_ERR_GRID, "the forms need at least two frequencies");
    if (c->prec == GW_MIXED) {
        static const char* const nm[2] = {"k_forms32_diag", "k_forms32_update"};
        forms_steps<float2>(ctx, W->fac32, n, N, Q, R, cout, nm);
    } else {
        static const char* const nm[2] = {"k_forms_diag", "k_forms_update"};
        forms_steps<double2>(ctx, W->fac, n, N, Q, R, cout, nm);
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
