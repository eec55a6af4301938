// Dense row-major GEMM C = alpha op(A) op(B) + beta C in binary64 (and a
// binary32 instance for the mixed path's basis and U products), used for
// the plain matrix products of the path: g = X_r^T v X_r and Z = X_r xi
// lambda^-1/2 (Eqs. projector0, subspace), U = V^EF Zup (Eq. subspace_chi0),
// q = Zup^T V^{nk}, v V^{nk} (Eq. instantaneous), W = v + Zup chi Zup^T.
// 64x64, 32x32 or 16x16 output tile per CTA (chosen per call to balance the
// SMs), K staged by 16 through shared memory, (BM/16)^2 outputs per thread;
// binary64 issue rate bounds it on this GPU.
#include "internal.h"

namespace {

constexpr int BK = 16;

// BM x BM output tile per CTA, (BM/16)^2 outputs per thread.
template <typename T, bool TA, bool TB, int BM>
__global__ void __launch_bounds__(256) k_dgemm(int M, int N, int K, T alpha, const T* __restrict__ A,
                                               long long lda, const T* __restrict__ B, long long ldb,
                                               T beta, T* __restrict__ C, long long ldc, long long sA,
                                               long long sB, long long sC) {
    constexpr int BN = BM, RM = BM / 16;
    __shared__ T As[BK][BM + 1];
    __shared__ T Bs[BK][BN + 1];
    A += blockIdx.z * sA;
    B += blockIdx.z * sB;
    C += blockIdx.z * sC;
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    T acc[RM][RM];
#pragma unroll
    for (int i = 0; i < RM; ++i)
#pragma unroll
        for (int j = 0; j < RM; ++j) acc[i][j] = T(0);
    for (int k0 = 0; k0 < K; k0 += BK) {
        for (int i = threadIdx.x; i < BK * BM; i += 256) {
            int kk, mm;
            if (TA) { kk = i / BM; mm = i % BM; } else { mm = i / BK; kk = i % BK; }
            int gm = m0 + mm, gk = k0 + kk;
            T val = T(0);
            if (gm < M && gk < K) val = TA ? A[(long long)gk * lda + gm] : A[(long long)gm * lda + gk];
            As[kk][mm] = val;
        }
        for (int i = threadIdx.x; i < BK * BN; i += 256) {
            int kk, nn;
            if (!TB) { kk = i / BN; nn = i % BN; } else { nn = i / BK; kk = i % BK; }
            int gn = n0 + nn, gk = k0 + kk;
            T val = T(0);
            if (gn < N && gk < K) val = TB ? B[(long long)gn * ldb + gk] : B[(long long)gk * ldb + gn];
            Bs[kk][nn] = val;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            T a[RM], b[RM];
#pragma unroll
            for (int i = 0; i < RM; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < RM; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < RM; ++i)
#pragma unroll
                for (int j = 0; j < RM; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < RM; ++i) {
        int gm = m0 + ty + 16 * i;
        if (gm >= M) continue;
#pragma unroll
        for (int j = 0; j < RM; ++j) {
            int gn = n0 + tx + 16 * j;
            if (gn >= N) continue;
            T* c = C + (long long)gm * ldc + gn;
            *c = beta == T(0) ? alpha * acc[i][j] : fma(alpha, acc[i][j], beta * *c);
        }
    }
}

// C = alpha A^T B (+ beta C) in binary32 on the FMA units for A [K][M] and
// B [K][N] row-major (the layout of U^T = Zup^T V^EF and q = Zup^T V^nk):
// both operands stream K-major rows, so their tiles are copied to shared
// memory without transposition.  128 x 128 output tile per CTA, K in steps
// of 16 staged through two shared-memory buffers (the next step's values
// are loaded into registers while the current one is multiplied), 8 x 8
// outputs per thread in four 4 x 4 quadrants so that every shared-memory
// read is a conflict-free 16-byte vector.  Every addition rounds to nearest.
constexpr int SG_T = 128, SG_K = 16;

__global__ void __launch_bounds__(256) k_sgemm_tn(int M, int N, int K, float alpha, const float* __restrict__ A,
                                                  long long lda, const float* __restrict__ B, long long ldb,
                                                  float beta, float* __restrict__ C, long long ldc) {
    __shared__ __align__(16) float As[2][SG_K][SG_T];
    __shared__ __align__(16) float Bs[2][SG_K][SG_T];
    const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
    const int m0 = blockIdx.y * SG_T, n0 = blockIdx.x * SG_T;
    // loader: thread covers column lc of rows lr, lr + 2, ..., lr + 14 of the K step
    const int lc = tid % SG_T, lr = tid / SG_T;
    const bool am = m0 + lc < M, bn = n0 + lc < N;
    float ra[8], rb[8];
    auto fetch = [&](int k0) {
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int k = k0 + lr + 2 * u;
            ra[u] = (am && k < K) ? A[(long long)k * lda + m0 + lc] : 0.f;
            rb[u] = (bn && k < K) ? B[(long long)k * ldb + n0 + lc] : 0.f;
        }
    };
    auto stash = [&](int buf) {
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            As[buf][lr + 2 * u][lc] = ra[u];
            Bs[buf][lr + 2 * u][lc] = rb[u];
        }
    };
    float acc[8][8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;
    fetch(0);
    stash(0);
    __syncthreads();
    const int nk = (K + SG_K - 1) / SG_K;
    for (int t = 0; t < nk; ++t) {
        const int buf = t & 1;
        if (t + 1 < nk) fetch((t + 1) * SG_K);
#pragma unroll
        for (int kk = 0; kk < SG_K; ++kk) {
            const float4 a0 = *reinterpret_cast<const float4*>(&As[buf][kk][4 * ty]);
            const float4 a1 = *reinterpret_cast<const float4*>(&As[buf][kk][64 + 4 * ty]);
            const float4 b0 = *reinterpret_cast<const float4*>(&Bs[buf][kk][4 * tx]);
            const float4 b1 = *reinterpret_cast<const float4*>(&Bs[buf][kk][64 + 4 * tx]);
            const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            const float b[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
        }
        if (t + 1 < nk) stash(buf ^ 1);      // the other buffer was last read before the previous barrier
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int gm = m0 + (i < 4 ? 4 * ty + i : 64 + 4 * ty + i - 4);
        if (gm >= M) continue;
        float* cr = C + (long long)gm * ldc;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int gn = n0 + (j < 4 ? 4 * tx + j : 64 + 4 * tx + j - 4);
            if (gn >= N) continue;
            cr[gn] = beta == 0.f ? alpha * acc[i][j] : fmaf(alpha, acc[i][j], beta * cr[gn]);
        }
    }
}

template <typename T>
static void gemm_t(gw_ctx* ctx, const char* name, bool ta, bool tb, int M, int N, int K, T alpha, const T* A,
                   long long lda, const T* B, long long ldb, T beta, T* C, long long ldc, int batch, long long sA,
                   long long sB, long long sC) {
    if (M <= 0 || N <= 0) return;
    // Tile edge: the FMA throughput bounds every SM, so the time is the work
    // of the busiest SM, ceil(tiles / SMs) * bm^2 (per unit of K); take the
    // smallest, preferring larger tiles on ties (fewer loads).
    int bm = 64;
    long long best = -1;
    for (int t : {64, 32, 16}) {
        const long long tiles = (long long)div_up(N, t) * div_up(M, t) * batch;
        const long long span = (tiles + ctx->num_sms - 1) / ctx->num_sms * t * t;
        if (best < 0 || span < best) { best = span; bm = t; }
    }
    dim3 grid(div_up(N, bm), div_up(M, bm), batch);
    auto pick = [&](auto k64, auto k32, auto k16) { return bm == 64 ? k64 : bm == 32 ? k32 : k16; };
    auto kern = (!ta && !tb) ? pick(k_dgemm<T, false, false, 64>, k_dgemm<T, false, false, 32>, k_dgemm<T, false, false, 16>)
              : (ta && !tb)  ? pick(k_dgemm<T, true, false, 64>, k_dgemm<T, true, false, 32>, k_dgemm<T, true, false, 16>)
              : (!ta && tb)  ? pick(k_dgemm<T, false, true, 64>, k_dgemm<T, false, true, 32>, k_dgemm<T, false, true, 16>)
                             : pick(k_dgemm<T, true, true, 64>, k_dgemm<T, true, true, 32>, k_dgemm<T, true, true, 16>);
    klaunch(ctx, name, kern, grid, 256, 0, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, sA, sB, sC);
}

__global__ void k_f64_to_f32_2d(const double* __restrict__ a, long long lda, int rows, int cols, float* __restrict__ b) {
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= (long long)rows * cols) return;
    const int r = (int)(t / cols), c = (int)(t % cols);
    b[t] = (float)a[(long long)r * lda + c];
}

}  // namespace

void gemm_f64(gw_ctx* ctx, bool ta, bool tb, int M, int N, int K, double alpha, const double* A, long long lda,
              const double* B, long long ldb, double beta, double* C, long long ldc, int batch, long long sA,
              long long sB, long long sC) {
    gemm_t<double>(ctx, "k_dgemm", ta, tb, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, batch, sA, sB, sC);
}

void gemm_f32(gw_ctx* ctx, bool ta, bool tb, int M, int N, int K, float alpha, const float* A, long long lda,
              const float* B, long long ldb, float beta, float* C, long long ldc) {
    if (!ctx->gemm_simt && sgemm_tc(ctx, ta, tb, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc)) return;
    gemm_t<float>(ctx, "k_sgemm", ta, tb, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, 1, 0, 0, 0);
}

void gemm_f32_rn(gw_ctx* ctx, bool ta, bool tb, int M, int N, int K, float alpha, const float* A, long long lda,
                 const float* B, long long ldb, float beta, float* C, long long ldc) {
    if (ta && !tb && M > 0 && N > 0) {
        const long long gx = (N + SG_T - 1) / SG_T, gy = (M + SG_T - 1) / SG_T;
        if (gx <= 0x7fffffffLL && gy <= 65535) {
            klaunch(ctx, "k_sgemm_tn", k_sgemm_tn, dim3((unsigned)gx, (unsigned)gy), 256, 0, M, N, K, alpha, A, lda,
                    B, ldb, beta, C, ldc);
            return;
        }
    }
    gemm_t<float>(ctx, "k_sgemm", ta, tb, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, 1, 0, 0, 0);
}

void launch_f64_to_f32_2d(gw_ctx* ctx, const double* a, long long lda, int rows, int cols, float* b) {
    const long long tot = (long long)rows * cols;
    if (tot > 0) klaunch(ctx, "k_to_f32", k_f64_to_f32_2d, div_up(tot, 256), 256, 0, a, lda, rows, cols, b);
}
