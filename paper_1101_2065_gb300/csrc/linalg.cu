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
__device__ __forceinline__ double2 jac_rotation(double app, double aqq, double apq) {
    double c = 1.0, s = 0.0;
    if (apq != 0.0 && fabs(apq) > 1e-300) {
        double tau = (aqq - app) / (2.0 * apq);
        double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + hypot(1.0, tau));
        c = 1.0 / sqrt(1.0 + t * t);
        s = t * c;
    }
    return make_double2(c, s);
}

__global__ void k_jacobi_rot(const double* __restrict__ A, int np, int r, double2* __restrict__ rot) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= np / 2) return;
    int m = np - 1, p, q;
    jac_pair(i, r, m, p, q);
    rot[i] = jac_rotation(A[(long long)p * np + p], A[(long long)q * np + q], A[(long long)p * np + q]);
}

// Column x of the round's rotation matrix J restricted to its pair (p, q):
// (J[p][x], J[q][x]) = (c, -s) for x = p, (s, c) for x = q.
__device__ __forceinline__ void jac_col(int role, double2 cs, double& a, double& b) {
    if (role == 0) { a = cs.x; b = -cs.y; } else { a = cs.y; b = cs.x; }
}

// (J^T A J)[x][y] for round r.
__device__ __forceinline__ double jac_elem(const double* __restrict__ A, int np, int r, int m,
                                           const double2* __restrict__ rot, int x, int y) {
    int i, rx, l, ry, pi, qi, pl, ql;
    jac_slot(x, r, m, i, rx);
    jac_slot(y, r, m, l, ry);
    if (i == l && x != y) return 0.0;
    jac_pair(i, r, m, pi, qi);
    jac_pair(l, r, m, pl, ql);
    double w0, w1, u0, u1;
    jac_col(rx, rot[i], w0, w1);
    jac_col(ry, rot[l], u0, u1);
    const double* Ap = A + (long long)pi * np;
    const double* Aq = A + (long long)qi * np;
    return w0 * (u0 * Ap[pl] + u1 * Ap[ql]) + w1 * (u0 * Aq[pl] + u1 * Aq[ql]);
}

// Grid-wide barrier for a cooperative launch.  bar[0] counts arrivals,
// bar[1] is the generation.  The wait gives up after a bounded number of
// polls, sets ST_TIMEOUT and returns false.
__device__ bool grid_barrier(unsigned int* bar, int* status, int* s_flag) {
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned int* vgen = bar + 1;
        unsigned int gen = *vgen;
        int ok = 1;
        __threadfence();
        unsigned int arrived = atomicAdd(bar, 1u);
        if (arrived == gridDim.x - 1) {
            atomicExch(bar, 0u);
            __threadfence();
            atomicAdd(bar + 1, 1u);
        } else {
            unsigned long long polls = 0;
            while (*vgen == gen) {
                if (++polls > (1ull << 25)) { atomicOr(status, ST_TIMEOUT); ok = 0; break; }
                __nanosleep(32);
            }
        }
        __threadfence();
        *s_flag = ok;
    }
    __syncthreads();
    return *s_flag != 0;
}

// One Jacobi sweep (m = np-1 rounds) in one cooperative launch.  Each round
// writes A' = J^T A J (upper triangle computed, mirrored), V' = V J and the
// rotations of the next round: the thread that produces A'[p'][q'] for a
// pair of the next round also recomputes A'[p'][p'] and A'[q'][q'].
__global__ void __launch_bounds__(512) k_jacobi_sweep(double* A0, double* A1, double* V0, double* V1,
                                                      double2* rot0, double2* rot1, int np,
                                                      unsigned int* bar, int* status) {
    __shared__ int s_flag;
    const int m = np - 1;
    const long long nsym = (long long)np * (np + 1) / 2;
    const long long total = nsym + (long long)np * np;
    double *Ac = A0, *An = A1, *Vc = V0, *Vn = V1;
    double2 *rc = rot0, *rn = rot1;
    for (int r = 0; r < m; ++r) {
        const int r2 = (r + 1) % m;
        for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
             t += (long long)gridDim.x * blockDim.x) {
            if (t < nsym) {
                // packed upper triangle: t = y(y+1)/2 + x, x <= y
                long long yy = (long long)((sqrtf(8.0f * (float)t + 1.0f) - 1.0f) * 0.5f);
                while (yy * (yy + 1) / 2 > t) --yy;
                while ((yy + 1) * (yy + 2) / 2 <= t) ++yy;
                const int y = (int)yy, x = (int)(t - yy * (yy + 1) / 2);
                const double val = jac_elem(Ac, np, r, m, rc, x, y);
                An[(long long)x * np + y] = val;
                An[(long long)y * np + x] = val;
                if (x != y) {
                    int i2, rx2, p2, q2;
                    jac_slot(x, r2, m, i2, rx2);
                    jac_pair(i2, r2, m, p2, q2);
                    if ((rx2 == 0 ? q2 : p2) == y) {
                        double app = jac_elem(Ac, np, r, m, rc, p2, p2);
                        double aqq = jac_elem(Ac, np, r, m, rc, q2, q2);
                        rn[i2] = jac_rotation(app, aqq, val);
                    }
                }
            } else {
                const long long t2 = t - nsym;
                const int row = (int)(t2 / np), y = (int)(t2 % np);
                int l, ry, pl, ql;
                jac_slot(y, r, m, l, ry);
                jac_pair(l, r, m, pl, ql);
                double u0, u1;
                jac_col(ry, rc[l], u0, u1);
                const double* Vr = Vc + (long long)row * np;
                Vn[t2] = Vr[pl] * u0 + Vr[ql] * u1;
            }
        }
        if (!grid_barrier(bar, status, &s_flag)) return;
        double* ta = Ac; Ac = An; An = ta;
        double* tv = Vc; Vc = Vn; Vn = tv;
        double2* tr = rc; rc = rn; rn = tr;
    }
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
    double2* rot0 = dalloc<double2>(ctx, np / 2);
    double2* rot1 = dalloc<double2>(ctx, np / 2);
    unsigned int* bar = dalloc<unsigned int>(ctx, 2);
    double* off = dalloc<double>(ctx, 2);
    double* hoff = nullptr;
    CUDA_CHECK(cudaMallocHost(&hoff, 2 * sizeof(double)));
    double* V0 = evecs;
    int sweeps = 0;
    try {
        CUDA_CHECK(cudaMemsetAsync(bar, 0, 2 * sizeof(unsigned int), ctx->stream));
        klaunch(ctx, "k_jacobi_init", k_jacobi_init, div_up(nn, 256), 256, 0, (const double*)g, n, np, A0, V0);
        klaunch(ctx, "k_jacobi_rot", k_jacobi_rot, div_up(np / 2, 128), 128, 0, (const double*)A0, np, 0, rot0);
        static int blocks_per_sm = -1;
        if (blocks_per_sm < 0) {
            CUDA_CHECK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm, k_jacobi_sweep, 512, 0));
            if (blocks_per_sm < 1) gw_throw(GW_ERR_CUDA, "Jacobi sweep kernel cannot be resident");
        }
        const int grid = ctx->num_sms;     // one CTA per SM: co-resident by cooperative launch
        double *Ac = A0, *An = A1, *Vc = V0, *Vn = V1;
        double2 *rc = rot0, *rn = rot1;
        bool ok = false;
        double prev = INFINITY;
        for (sweeps = 0; sweeps < 40; ++sweeps) {
            klaunch(ctx, "k_jacobi_off", k_jacobi_off, 1, 1024, 0, (const double*)Ac, n, np, off);
            CUDA_CHECK(cudaMemcpyAsync(hoff, off, 2 * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
            CUDA_CHECK(cudaStreamSynchronize(ctx->stream));
            double o = hoff[0], d = hoff[1];
            if (!std::isfinite(o) || !std::isfinite(d)) break;
            if (o <= 1e-30 * d || o == 0.0) { ok = true; break; }
            if (sweeps >= 3 && o >= 0.25 * prev && o <= 1e-24 * d) { ok = true; break; }
            prev = o;
            void* args[] = {&Ac, &An, &Vc, &Vn, &rc, &rn, (void*)&np, &bar, &ctx->d_status};
            prof_begin(ctx, "k_jacobi_sweep");
            CUDA_CHECK(cudaLaunchCooperativeKernel((const void*)k_jacobi_sweep, dim3(grid), dim3(512), args, 0,
                                                   ctx->stream));
            after_launch(ctx, "k_jacobi_sweep");
            // m = np - 1 rounds (odd): the result sits in the other buffers
            std::swap(Ac, An);
            std::swap(Vc, Vn);
            std::swap(rc, rn);
        }
        if (!ok) gw_throw(GW_ERR_NO_CONVERGENCE, "Jacobi eigensolver did not converge in 40 sweeps");
        klaunch(ctx, "k_jacobi_diag", k_jacobi_diag, div_up(np, 256), 256, 0, (const double*)Ac, np, evals);
        if (Vc != evecs)
            CUDA_CHECK(cudaMemcpyAsync(evecs, Vc, nn * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
        CUDA_CHECK(cudaStreamSynchronize(ctx->stream));
    } catch (...) {
        ctx_free(ctx, A0); ctx_free(ctx, A1); ctx_free(ctx, V1); ctx_free(ctx, rot0); ctx_free(ctx, rot1);
        ctx_free(ctx, bar); ctx_free(ctx, off);
        cudaFreeHost(hoff);
        throw;
    }
    ctx_free(ctx, A0); ctx_free(ctx, A1); ctx_free(ctx, V1); ctx_free(ctx, rot0); ctx_free(ctx, rot1);
    ctx_free(ctx, bar); ctx_free(ctx, off);
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
