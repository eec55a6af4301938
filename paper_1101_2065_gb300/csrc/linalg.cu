// a0 dense linear algebra in binary64:
//  * blocked right-looking Cholesky v = L L^T (uncompressed basis Zup = L);
//  * cyclic parallel Jacobi eigensolver for the symmetric g = X_r^T v X_r of
//    Eq. projector0 (Eq. subspace diagonalises g);
//  * selection of the n_sub dominant eigenpairs and the scaling
//    xi / sqrt(lambda) of Eq. subspace.
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

// ------------------------------------------------------------------ Jacobi
// Round-robin ("circle") schedule over np (even) indices: in round r the
// pairs are (r mod m, m) and ((r+i) mod m, (r-i) mod m), i = 1..np/2-1,
// m = np-1.  Every unordered pair occurs once in the m rounds of a sweep.
__device__ __forceinline__ void jac_pair(int i, int r, int m, int& p, int& q) {
    if (i == 0) { p = r % m; q = m; }
    else { p = (r + i) % m; q = (r - i + m) % m; }
}

__device__ __forceinline__ void jac_slot(int x, int r, int m, int& pair, int& role) {
    if (x == m) { pair = 0; role = 1; return; }
    int d = ((x - r) % m + m) % m;
    if (d == 0) { pair = 0; role = 0; }
    else if (d <= (m - 1) / 2) { pair = d; role = 0; }
    else { pair = m - d; role = 1; }
}

// Rotation (c, s) zeroing A[p][q] of the 2x2 symmetric block (the classical
// symmetric Schur step of the Jacobi method).
__global__ void k_jacobi_rot(const double* __restrict__ A, int np, int r, double2* __restrict__ rot) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= np / 2) return;
    int m = np - 1, p, q;
    jac_pair(i, r, m, p, q);
    double app = A[(long long)p * np + p], aqq = A[(long long)q * np + q], apq = A[(long long)p * np + q];
    double c = 1.0, s = 0.0;
    if (apq != 0.0 && fabs(apq) > 1e-300) {
        double tau = (aqq - app) / (2.0 * apq);
        double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + hypot(1.0, tau));
        c = 1.0 / sqrt(1.0 + t * t);
        s = t * c;
    }
    rot[i] = make_double2(c, s);
}

// A' = J^T A J and V' = V J for all np/2 disjoint rotations of round r.
__global__ void __launch_bounds__(256) k_jacobi_apply(const double* __restrict__ A, double* __restrict__ A2,
                                                      const double* __restrict__ V, double* __restrict__ V2,
                                                      const double2* __restrict__ rot, int np, int r) {
    long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    long long nn = (long long)np * np;
    if (t >= 2 * nn) return;
    const int m = np - 1;
    bool isV = t >= nn;
    if (isV) t -= nn;
    int x = (int)(t / np), y = (int)(t % np);
    int l, ry;
    jac_slot(y, r, m, l, ry);
    int pl, ql;
    jac_pair(l, r, m, pl, ql);
    double2 cl = rot[l];
    double u0 = ry == 0 ? cl.x : cl.y;      // J[p_l][y]
    double u1 = ry == 0 ? -cl.y : cl.x;     // J[q_l][y]
    if (isV) {
        V2[t] = V[(long long)x * np + pl] * u0 + V[(long long)x * np + ql] * u1;
        return;
    }
    int i, rx;
    jac_slot(x, r, m, i, rx);
    if (i == l && x != y) { A2[t] = 0.0; return; }
    int pi, qi;
    jac_pair(i, r, m, pi, qi);
    double2 ci = rot[i];
    double w0 = rx == 0 ? ci.x : ci.y;
    double w1 = rx == 0 ? -ci.y : ci.x;
    double a00 = A[(long long)pi * np + pl], a01 = A[(long long)pi * np + ql];
    double a10 = A[(long long)qi * np + pl], a11 = A[(long long)qi * np + ql];
    A2[t] = w0 * (u0 * a00 + u1 * a01) + w1 * (u0 * a10 + u1 * a11);
}

__global__ void k_jacobi_init(const double* __restrict__ g, int n, int np, double* __restrict__ A,
                              double* __restrict__ V) {
    long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= (long long)np * np) return;
    int x = (int)(t / np), y = (int)(t % np);
    double a;
    if (x < n && y < n) a = 0.5 * (g[(long long)x * n + y] + g[(long long)y * n + x]);
    else a = (x == y) ? -1.0 : 0.0;     // padding index: decoupled, never selected
    A[t] = a;
    V[t] = x == y ? 1.0 : 0.0;
}

// Deterministic single-CTA sums of the squared off-diagonal and diagonal.
__global__ void __launch_bounds__(1024) k_jacobi_off(const double* __restrict__ A, int n, int np, double* out) {
    __shared__ double so[1024], sd[1024];
    double off = 0.0, dg = 0.0;
    for (long long t = threadIdx.x; t < (long long)n * n; t += blockDim.x) {
        int x = (int)(t / n), y = (int)(t % n);
        double a = A[(long long)x * np + y];
        if (x == y) dg += a * a; else off += a * a;
    }
    so[threadIdx.x] = off;
    sd[threadIdx.x] = dg;
    __syncthreads();
    for (int s = 512; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            so[threadIdx.x] += so[threadIdx.x + s];
            sd[threadIdx.x] += sd[threadIdx.x + s];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) { out[0] = so[0]; out[1] = sd[0]; }
}

__global__ void k_jacobi_diag(const double* __restrict__ A, int np, double* __restrict__ ev) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < np) ev[i] = A[(long long)i * np + i];
}

// sel[rank] = index of the rank-th largest eigenvalue (ties by index).
__global__ void k_rank_desc(const double* __restrict__ ev, int np, int n_sub, int* __restrict__ sel) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= np) return;
    double e = ev[i];
    int r = 0;
    for (int j = 0; j < np; ++j) {
        double f = ev[j];
        r += (f > e) || (f == e && j < i);
    }
    if (r < n_sub) sel[r] = i;
}

// B[row][k] = V[row][sel[k]] / sqrt(lambda_sel[k]); rank check on thread 0.
__global__ void k_scale_sel(const double* __restrict__ ev, const double* __restrict__ V, int n, int np,
                            int n_sub, const int* __restrict__ sel, double* __restrict__ B, int* status) {
    long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t == 0) {
        double lmax = ev[sel[0]], lmin = ev[sel[n_sub - 1]];
        if (!(lmin >= 1e-12 * lmax) || !(lmax > 0.0)) atomicOr(status, ST_RANK);
    }
    if (t >= (long long)n * n_sub) return;
    int row = (int)(t / n_sub), k = (int)(t % n_sub);
    int c = sel[k];
    double lam = ev[c];
    B[t] = lam > 0.0 ? V[(long long)row * np + c] / sqrt(lam) : 0.0;
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

int jacobi_eigh(gw_ctx* ctx, double* g, int n, double* evals, double* evecs) {
    const int np = n + (n & 1);
    const long long nn = (long long)np * np;
    double* A0 = dalloc<double>(ctx, nn);
    double* A1 = dalloc<double>(ctx, nn);
    double* V1 = dalloc<double>(ctx, nn);
    double2* rot = dalloc<double2>(ctx, np / 2);
    double* off = dalloc<double>(ctx, 2);
    double* hoff = nullptr;
    CUDA_CHECK(cudaMallocHost(&hoff, 2 * sizeof(double)));
    double* V0 = evecs;
    int sweeps = 0;
    try {
        klaunch(ctx, "k_jacobi_init", k_jacobi_init, div_up(nn, 256), 256, 0, g, n, np, A0, V0);
        double *Ac = A0, *An = A1, *Vc = V0, *Vn = V1;
        bool ok = false;
        double prev = INFINITY;
        for (sweeps = 0; sweeps < 40; ++sweeps) {
            klaunch(ctx, "k_jacobi_off", k_jacobi_off, 1, 1024, 0, Ac, n, np, off);
            CUDA_CHECK(cudaMemcpyAsync(hoff, off, 2 * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
            CUDA_CHECK(cudaStreamSynchronize(ctx->stream));
            double o = hoff[0], d = hoff[1];
            if (!std::isfinite(o) || !std::isfinite(d)) break;
            if (o <= 1e-30 * d || o == 0.0) { ok = true; break; }
            // converged to roundoff: no further decrease
            if (sweeps >= 3 && o >= 0.25 * prev && o <= 1e-24 * d) { ok = true; break; }
            prev = o;
            for (int r = 0; r < np - 1; ++r) {
                klaunch(ctx, "k_jacobi_rot", k_jacobi_rot, div_up(np / 2, 128), 128, 0, Ac, np, r, rot);
                klaunch(ctx, "k_jacobi_apply", k_jacobi_apply, div_up(2 * nn, 256), 256, 0, Ac, An, Vc, Vn, rot, np, r);
                std::swap(Ac, An);
                std::swap(Vc, Vn);
            }
        }
        if (!ok) gw_throw(GW_ERR_NO_CONVERGENCE, "Jacobi eigensolver did not converge in 40 sweeps");
        klaunch(ctx, "k_jacobi_diag", k_jacobi_diag, div_up(np, 256), 256, 0, Ac, np, evals);
        if (Vc != evecs)
            CUDA_CHECK(cudaMemcpyAsync(evecs, Vc, nn * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
        CUDA_CHECK(cudaStreamSynchronize(ctx->stream));
    } catch (...) {
        ctx_free(ctx, A0); ctx_free(ctx, A1); ctx_free(ctx, V1); ctx_free(ctx, rot); ctx_free(ctx, off);
        cudaFreeHost(hoff);
        throw;
    }
    ctx_free(ctx, A0); ctx_free(ctx, A1); ctx_free(ctx, V1); ctx_free(ctx, rot); ctx_free(ctx, off);
    cudaFreeHost(hoff);
    return sweeps;
}

void select_top_scaled(gw_ctx* ctx, const double* evals, const double* evecs, int n, int n_sub, double* B) {
    const int np = n + (n & 1);
    int* sel = dalloc<int>(ctx, n_sub);
    klaunch(ctx, "k_rank_desc", k_rank_desc, div_up(np, 256), 256, 0, evals, np, n_sub, sel);
    klaunch(ctx, "k_scale_sel", k_scale_sel, div_up((long long)n * n_sub, 256), 256, 0, evals, evecs, n, np, n_sub, sel, B,
                                                                            ctx->d_status);
    ctx_free(ctx, sel);
}

void launch_split_complex(gw_ctx* ctx, const double2* z, double* re, double* im, size_t n) {
    klaunch(ctx, "k_split_complex", k_split_complex, div_up((long long)n, 256), 256, 0, z, re, im, (long long)n);
}
