// a0 dense linear algebra in binary64: blocked right-looking Cholesky
// v = L L^T for the uncompressed basis Zup = L (Z = L^-T satisfies
// Z^T v Z = I, Eq. global-basis-orthogonality).
#include <cmath>

#include "internal.h"

namespace {

// ------------------------------------------------------------------ Cholesky
constexpr int CNB = 32;

// Factor the kb x kb diagonal block at (k0,k0) in shared memory, then solve
// the rows below it: x L11^T = a.  Every CTA factors the (small) block
// redundantly; CTA 0 writes it back.
__global__ void __launch_bounds__(256) k_chol_panel(double* __restrict__ A, int n, int k0, int kb, int* status) {
    __shared__ double S[CNB][CNB + 1];
    const int tid = threadIdx.x;
    for (int t = tid; t < kb * kb; t += blockDim.x) {
        int i = t / kb, j = t % kb;
        S[i][j] = (j <= i) ? A[(long long)(k0 + i) * n + k0 + j] : 0.0;
    }
    __syncthreads();
    for (int j = 0; j < kb; ++j) {
        if (tid == 0) {
            double d = S[j][j];
            if (!(d > 0.0) || !isfinite(d)) {
                atomicOr(status, ST_NOT_SPD);
                d = 1.0;
            }
            S[j][j] = sqrt(d);
        }
        __syncthreads();
        for (int i = j + 1 + tid; i < kb; i += blockDim.x) S[i][j] /= S[j][j];
        __syncthreads();
        for (int t = tid; t < kb * kb; t += blockDim.x) {
            int i = t / kb, l = t % kb;
            if (l > j && l <= i) S[i][l] -= S[i][j] * S[l][j];
        }
        __syncthreads();
    }
    if (blockIdx.x == 0)
        for (int t = tid; t < kb * kb; t += blockDim.x) {
            int i = t / kb, j = t % kb;
            if (j <= i) A[(long long)(k0 + i) * n + k0 + j] = S[i][j];
        }
    int r = k0 + kb + blockIdx.x * blockDim.x + tid;
    if (r < n) {
        double x[CNB];
#pragma unroll
        for (int j = 0; j < CNB; ++j) {
            if (j < kb) {
                double a = A[(long long)r * n + k0 + j];
                for (int p = 0; p < j; ++p) a -= x[p] * S[j][p];
                x[j] = a / S[j][j];
            }
        }
#pragma unroll
        for (int j = 0; j < CNB; ++j)
            if (j < kb) A[(long long)r * n + k0 + j] = x[j];
    }
}

__global__ void k_zero_upper(double* A, int n) {
    long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= (long long)n * n) return;
    int i = (int)(t / n), j = (int)(t % n);
    if (j > i) A[t] = 0.0;
}

__global__ void k_split_complex(const double2* __restrict__ z, double* __restrict__ re, double* __restrict__ im,
                                long long n) {
    long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t < n) { re[t] = z[t].x; im[t] = z[t].y; }
}

}  // namespace

void cholesky_lower(gw_ctx* ctx, double* A, int n) {
    for (int k0 = 0; k0 < n; k0 += CNB) {
        int kb = std::min(CNB, n - k0), k1 = k0 + kb;
        int rows = n - k1;
        klaunch(ctx, "k_chol_panel", k_chol_panel, std::max(1, div_up(rows, 256)), 256, 0, A, n, k0, kb, ctx->d_status);
        if (rows > 0)
            gemm_f64(ctx, false, true, rows, rows, kb, -1.0, A + (long long)k1 * n + k0, n, A + (long long)k1 * n + k0,
                     n, 1.0, A + (long long)k1 * n + k1, n);
    }
    klaunch(ctx, "k_zero_upper", k_zero_upper, div_up((long long)n * n, 256), 256, 0, A, n);
}

void launch_split_complex(gw_ctx* ctx, const double2* z, double* re, double* im, size_t n) {
    klaunch(ctx, "k_split_complex", k_split_complex, div_up((long long)n, 256), 256, 0, z, re, im, (long long)n);
}
