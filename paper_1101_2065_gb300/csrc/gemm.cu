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
    gemm_t<float>(ctx, "k_sgemm", ta, tb, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, 1, 0, 0, 0);
}

void launch_f64_to_f32_2d(gw_ctx* ctx, const double* a, long long lda, int rows, int cols, float* b) {
    const long long tot = (long long)rows * cols;
    if (tot > 0) klaunch(ctx, "k_to_f32", k_f64_to_f32_2d, div_up(tot, 256), 256, 0, a, lda, rows, cols, b);
}
