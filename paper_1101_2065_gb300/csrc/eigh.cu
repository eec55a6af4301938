// a0: dominant eigenpairs of g = X_r^T v X_r (Eqs. projector0, subspace).
//
// Mixed-precision symmetric eigensolver:
//  1. binary32 Householder tridiagonalisation T = Q^T g Q on a cluster of 8
//     CTAs holding the matrix row-cyclically in distributed shared memory,
//     or, when it does not fit, on the whole GPU (cooperative launch, matrix
//     in L2); reflector k is kept in row k of the global copy;
//  2. all eigenvalues of T by bisection on Sturm counts (one thread each);
//  3. eigenvectors of T by binary64 inverse iteration with a pivoted
//     tridiagonal LU (one thread per eigenvalue, hashed random start), then
//     Gram-Schmidt inside clusters of near-degenerate eigenvalues (such as
//     the null space of g when N_rank exceeds N_prod);
//  4. back-transformation X = Q Y (one warp per vector);
//  5. binary64 refinement of the full eigenbasis by the iteration of Ogita
//     and Aishima (2018): R = I - X^T X, S = X^T g X,
//     lambda_i = S_ii / (1 - R_ii), E_ij = (S_ij + lambda_j R_ij)/(lambda_j -
//     lambda_i) for well separated pairs, R_ij / 2 otherwise, X <- X + X E;
//     each step squares the error (binary64 GEMMs only); repeated until
//     |S - diag| / |g| falls below a tolerance, at most oa_iters times;
//  6. the n_sub largest eigenpairs are selected, their block re-orthonormalised
//     by one Newton-Schulz step X <- X (3 I - X^T X) / 2, and scaled by
//     lambda^-1/2 (Eq. subspace).
#include <cooperative_groups.h>

#include <cfloat>
#include <cmath>

#include "internal.h"

namespace cg = cooperative_groups;

namespace {

__device__ __forceinline__ float warp_sum(float v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// block-wide sum for a 1024-thread CTA; red has 33 floats
__device__ float block_sum1024(float v, float* red) {
    v = warp_sum(v);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
        float w = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.f;
        w = warp_sum(w);
        if (threadIdx.x == 0) red[32] = w;
    }
    __syncthreads();
    float r = red[32];
    __syncthreads();
    return r;
}

// block-wide binary64 sum (blockDim <= 1024, a multiple of 32); red has 33 doubles
__device__ double block_sum1024d(double v, double* red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
        double w = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
        if (threadIdx.x == 0) red[32] = w;
    }
    __syncthreads();
    double r = red[32];
    __syncthreads();
    return r;
}

// ------------------------------------------------------------------ 1
// Same reduction on a cluster of CL CTAs: CTA r holds the rows i = r (mod CL)
// of the matrix in its shared memory; the reflector, the partial dot
// products and w travel through distributed shared memory.
constexpr int CL = 8;

__global__ void __cluster_dims__(CL, 1, 1) __launch_bounds__(1024)
    k_sytrd32_cl(float* __restrict__ A, int n, float* __restrict__ d, float* __restrict__ e, float* __restrict__ tau) {
    extern __shared__ float sm[];
    cg::cluster_group cluster = cg::this_cluster();
    const int rank = (int)cluster.block_rank();
    const int rows = (n + CL - 1) / CL;
    float* Ar = sm;                        // [rows][n] own rows
    float* svb = Ar + (long long)rows * n; // [2][n] reflector, pushed by its owner (by step parity)
    float* pb = svb + 2 * n;               // [2][n] p_i, i > k, pushed by the CTA owning row i
    float* sw = pb + 2 * n;                // [n] w
    __shared__ float s_part[2][CL][32];    // partial v^T p of every warp of every CTA, pushed
    __shared__ float s_tau[2];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    for (int li = 0; li < rows; ++li) {
        const int i = li * CL + rank;
        for (int j = tid; j < n; j += blockDim.x) Ar[(long long)li * n + j] = i < n ? A[(long long)i * n + j] : 0.f;
    }
    // Two cluster barriers per step.  Everything another CTA needs is
    // stored into that CTA's shared memory before a barrier (distributed
    // shared memory stores), so after each barrier all reads are local:
    //   (1) the owner of row k pushes the reflector v and tau;
    //   (2) every CTA pushes p_i of its rows and its partial v^T p.
    // Buffers alternate by step parity: a CTA that runs ahead writes the
    // other half.
    for (int k = 0; k + 2 < n; ++k) {
        const int m = n - k - 1;
        const int owner = k % CL, par = k & 1;
        float* sv = svb + par * n;
        float* p = pb + par * n;
        __syncthreads();
        if (rank == owner) {
            const float* rk = Ar + (long long)(k / CL) * n + k + 1;
            for (int j = tid; j < m; j += blockDim.x) sv[j] = rk[j];
            if (warp == 0) {
                // |x|^2 by one warp (no block-wide barrier)
                float part = 0.f;
                for (int j = lane; j < m; j += 32) part += rk[j] * rk[j];
                const float sig = warp_sum(part);
                if (lane == 0) {
                    const float x0 = rk[0];
                    const float alpha = sig > 0.f ? -copysignf(sqrtf(sig), x0) : 0.f;
                    const float v0 = x0 - alpha;
                    const float vtv = sig - x0 * x0 + v0 * v0;
                    const float t = vtv > 0.f ? 2.f / vtv : 0.f;
                    sv[0] = v0;
                    d[k] = Ar[(long long)(k / CL) * n + k];
                    e[k] = sig > 0.f ? alpha : x0;
                    tau[k] = t;
                    for (int r = 0; r < CL; ++r) cluster.map_shared_rank(s_tau, r)[par] = t;
                }
            }
            __syncthreads();
            for (int j = tid; j < m; j += blockDim.x) {
                const float x = sv[j];
                A[(long long)k * n + k + 1 + j] = x;   // reflector
#pragma unroll
                for (int r = 0; r < CL; ++r)
                    if (r != owner) cluster.map_shared_rank(sv, r)[j] = x;
            }
        }
        cluster.sync();
        const float t = s_tau[par];
        // own rows i > k: p_i = t sum_j A[i][j] v_j, pushed to every CTA
        const int li0 = (k + 1 - rank + CL - 1) / CL;      // first own row index with i >= k+1
        float pv = 0.f;
        for (int li = li0 + warp; li < rows; li += nw) {
            const int i = li * CL + rank;
            if (i >= n) break;
            const float* ri = Ar + (long long)li * n + k + 1;
            float acc = 0.f;
            for (int j = lane; j < m; j += 32) acc += ri[j] * sv[j];
            acc = warp_sum(acc) * t;
            if (lane < CL) cluster.map_shared_rank(p, lane)[i - k - 1] = acc;
            if (lane == 0) pv += acc * sv[i - k - 1];
        }
        // lane 0 holds this warp's partial v^T p: push it to every CTA
        pv = __shfl_sync(0xffffffffu, pv, 0);
        if (lane < CL) cluster.map_shared_rank(&s_part[0][0][0], lane)[(par * CL + rank) * 32 + warp] = pv;
        cluster.sync();
        float tot = 0.f;
#pragma unroll
        for (int r = 0; r < CL; ++r) tot += (lane < nw) ? s_part[par][r][lane] : 0.f;
        tot = warp_sum(tot);
        const float K = 0.5f * t * tot;
        for (int j = tid; j < m; j += blockDim.x) sw[j] = p[j] - K * sv[j];
        __syncthreads();
        for (int li = li0 + warp; li < rows; li += nw) {
            const int i = li * CL + rank;
            if (i >= n) break;
            float* ri = Ar + (long long)li * n + k + 1;
            const float vi = sv[i - k - 1], wi = sw[i - k - 1];
            for (int j = lane; j < m; j += 32) ri[j] -= vi * sw[j] + wi * sv[j];
        }
    }
    cluster.sync();
    if (tid == 0 && n >= 2) {
        const int a = n - 2, b = n - 1;
        if (a % CL == rank) {
            d[a] = Ar[(long long)(a / CL) * n + a];
            tau[a] = 0.f;
        }
        if (b % CL == rank) {
            d[b] = Ar[(long long)(b / CL) * n + b];
            e[a] = Ar[(long long)(b / CL) * n + a];
            tau[b] = 0.f;
        }
    }
    cluster.sync();
}

// Same reduction on the whole GPU for ranks too large for the cluster:
// cooperative launch, matrix in global memory (L2), one grid barrier per
// Householder step (k_sytrd32_grid below).
__device__ bool grid_barrier(unsigned int* bar, int* status, int* s_flag, unsigned long long poll_limit) {
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
                if (++polls > poll_limit) { atomicOr(status, ST_TIMEOUT); ok = 0; break; }
                __nanosleep(32);
            }
        }
        __threadfence();
        *s_flag = ok;
    }
    __syncthreads();
    return *s_flag != 0;
}

// Householder vector of the row r[0 .. mm) held in shared memory (all
// threads of the CTA): v = r - alpha e_0, tau = 2 / v^T v, alpha = -sign(r_0)
// |r|; returns alpha (or r_0 when |r| = 0) in *e_out and tau in *tau_out.
__device__ void house_row(float* r, int mm, float* red, float* e_out, float* tau_out) {
    float pp = 0.f;
    for (int j = threadIdx.x; j < mm; j += blockDim.x) pp += r[j] * r[j];
    const float sig = block_sum1024(pp, red);
    if (threadIdx.x == 0) {
        const float x0 = r[0];
        const float alpha = sig > 0.f ? -copysignf(sqrtf(sig), x0) : 0.f;
        const float v0 = x0 - alpha;
        const float vtv = sig - x0 * x0 + v0 * v0;
        r[0] = v0;
        *e_out = sig > 0.f ? alpha : x0;
        *tau_out = vtv > 0.f ? 2.f / vtv : 0.f;
    }
    __syncthreads();
}

// Step k: trailing block rows/columns k+1 .. n-1 (m = n - k - 1), v_k and
// w_k in shared memory (sv, sw), identical in every CTA.  Every CTA forms
// the updated row k+1 of A - v w^T - w v^T and its Householder vector
// v_{k+1} redundantly (no barrier needed for it); then each warp updates its
// rows i >= k+2 in one pass and, in the same pass, takes the dot products of
// the updated rows with v_{k+1} (p_{k+1} = tau A_{k+1} v_{k+1}); one grid
// barrier publishes p_{k+1} and the partial sums of v^T p, after which every
// CTA forms w_{k+1} = p - (tau v^T p / 2) v.  The trailing matrix is read
// and written once per step, with one grid barrier.  CTA 0 writes the
// reflector v_k into row k of A (every CTA read that row in the step
// before), and d, e, tau.
__global__ void __launch_bounds__(512) k_sytrd32_grid(float* __restrict__ A, int n, float* __restrict__ d,
                                                      float* __restrict__ e, float* __restrict__ tau,
                                                      float* __restrict__ vbuf, float* __restrict__ pbuf,
                                                      float* __restrict__ part, unsigned int* bar, int* status,
                                                      unsigned long long poll_limit) {
    extern __shared__ float sm[];
    float* sv = sm;              // v_k   (entries k+1 .. n-1)
    float* sw = sm + n;          // w_k
    float* sr = sm + 2 * n;      // updated row k+1, then v_{k+1}
    __shared__ float red[33];
    __shared__ int s_flag;
    __shared__ float s_e, s_tau;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    const int gwarp = blockIdx.x * nw + warp, nwarps = gridDim.x * nw;
    (void)vbuf;
    if (n < 3) {
        if (blockIdx.x == 0 && tid == 0) {
            for (int i = 0; i < n; ++i) { d[i] = A[(long long)i * n + i]; tau[i] = 0.f; }
            if (n == 2) e[0] = A[(long long)n + 0];
        }
        return;
    }
    // step 0: v_0 from row 0, p_0 = tau A v_0 over rows 1 .. n-1
    {
        const int m = n - 1;
        for (int j = tid; j < m; j += blockDim.x) sr[j] = A[1 + j];
        __syncthreads();
        house_row(sr, m, red, &s_e, &s_tau);
        if (blockIdx.x == 0 && tid == 0) { d[0] = A[0]; e[0] = s_e; tau[0] = s_tau; }
        for (int j = tid; j < m; j += blockDim.x) sv[j] = sr[j];
        __syncthreads();
        const float t = s_tau;
        float pv = 0.f;
        for (int i = gwarp; i < m; i += nwarps) {
            const float* ri = A + (long long)(1 + i) * n + 1;
            float acc = 0.f;
            for (int j = lane; j < m; j += 32) acc += ri[j] * sv[j];
            acc = warp_sum(acc) * t;
            if (lane == 0) { pbuf[i] = acc; pv += acc * sv[i]; }          // parity 0
        }
        pv = block_sum1024(pv, red);
        if (tid == 0) part[blockIdx.x] = pv;
        if (!grid_barrier(bar, status, &s_flag, poll_limit)) return;
        float tot = 0.f;
        for (int q = 0; q < (int)gridDim.x; ++q) tot += part[q];
        const float K = 0.5f * t * tot;
        for (int j = tid; j < m; j += blockDim.x) sw[j] = pbuf[j] - K * sv[j];
        __syncthreads();
    }
    for (int k = 0; k + 2 < n; ++k) {
        const int m = n - k - 1;                 // v_k, w_k cover rows k+1 .. n-1
        // reflector v_k into row k (all CTAs read row k during the previous step)
        if (blockIdx.x == 0)
            for (int j = tid; j < m; j += blockDim.x) A[(long long)k * n + k + 1 + j] = sv[j];
        // updated row k+1 (local row 0 of the trailing block), redundantly in every CTA
        const float* r1 = A + (long long)(k + 1) * n + k + 1;
        const float v0 = sv[0], w0 = sw[0];
        {
            // up to eight loads of the row in flight per thread
            const int stride = blockDim.x;
            int j = tid;
            for (; j + 7 * stride < m; j += 8 * stride) {
                float a[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) a[u] = r1[j + u * stride];
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int jj = j + u * stride;
                    sr[jj] = a[u] - v0 * sw[jj] - w0 * sv[jj];
                }
            }
            for (; j < m; j += stride) sr[j] = r1[j] - v0 * sw[j] - w0 * sv[j];
        }
        __syncthreads();
        const bool last = k + 3 >= n;            // row k+1 = n-2: no further reflector
        if (blockIdx.x == 0 && tid == 0) d[k + 1] = sr[0];
        float t1 = 0.f;
        if (!last) {
            house_row(sr + 1, m - 1, red, &s_e, &s_tau);           // v_{k+1} in sr[1 .. m)
            if (blockIdx.x == 0 && tid == 0) { e[k + 1] = s_e; tau[k + 1] = s_tau; }
            t1 = s_tau;
        } else if (blockIdx.x == 0 && tid == 0) {
            e[k + 1] = sr[1];
            tau[k + 1] = 0.f;
        }
        // fused pass over rows i = k+2 .. n-1 (local 1 .. m-1): A -= v w^T + w v^T on columns
        // k+2 .. n-1, and the dot product of the updated row with v_{k+1}
        const float* vn = sr + 1;                // v_{k+1}, local column j - 1
        float* pb = pbuf + (long long)((k + 1) & 1) * n;                  // p_{k+1}: parity k+1
        float* pt = part + (long long)((k + 1) & 1) * gridDim.x;
        float pv = 0.f;
        for (int i = 1 + gwarp; i < m; i += nwarps) {
            float* ri = A + (long long)(k + 1 + i) * n + k + 2;
            const float vi = sv[i], wi = sw[i];
            float acc = 0.f;
            int j = lane;
            // eight loads of the row in flight per lane (the pass is bound by their latency);
            // each lane still accumulates its columns in ascending order
            for (; j + 32 * 7 < m - 1; j += 32 * 8) {
                float a[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) a[u] = ri[j + 32 * u];
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int jj = j + 32 * u;
                    a[u] = a[u] - vi * sw[1 + jj] - wi * sv[1 + jj];
                    ri[jj] = a[u];
                    acc += a[u] * vn[jj];
                }
            }
            for (; j < m - 1; j += 32) {
                const float a = ri[j] - vi * sw[1 + j] - wi * sv[1 + j];
                ri[j] = a;
                acc += a * vn[j];
            }
            acc = warp_sum(acc) * t1;
            if (lane == 0) { pb[i - 1] = acc; pv += acc * vn[i - 1]; }
        }
        if (last) break;
        pv = block_sum1024(pv, red);
        if (tid == 0) pt[blockIdx.x] = pv;
        if (!grid_barrier(bar, status, &s_flag, poll_limit)) return;
        float tot = 0.f;
        for (int q = 0; q < (int)gridDim.x; ++q) tot += pt[q];
        const float K = 0.5f * t1 * tot;
        {
            const int stride = blockDim.x;
            int j = tid;
            for (; j + 7 * stride < m - 1; j += 8 * stride) {
                float a[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) a[u] = pb[j + u * stride];
#pragma unroll
                for (int u = 0; u < 8; ++u) sw[j + u * stride] = a[u] - K * vn[j + u * stride];
            }
            for (; j < m - 1; j += stride) sw[j] = pb[j] - K * vn[j];
        }
        __syncthreads();
        for (int j = tid; j < m - 1; j += blockDim.x) sv[j] = vn[j];
        __syncthreads();
    }
    // the last diagonal entry: row n-1 was updated by the last pass (its owner warp)
    if (!grid_barrier(bar, status, &s_flag, poll_limit)) return;
    if (blockIdx.x == 0 && tid == 0) {
        d[n - 1] = A[(long long)(n - 1) * n + n - 1];
        tau[n - 1] = 0.f;
    }
}

// ------------------------------------------------------------------ 2
// Eigenvalue i (ascending) of T by multisection: one warp per eigenvalue,
// each lane counts the eigenvalues below one of 32 interior points of the
// current bracket, so each step shrinks it 33-fold (8 steps ~ 40 bisection
// steps).  d and e^2 are staged in shared memory.
__global__ void __launch_bounds__(256) k_bisect(const float* __restrict__ d, const float* __restrict__ e, int n,
                                                float bnd, float* __restrict__ lam) {
    extern __shared__ float sde[];
    float* sd = sde;
    float* se2 = sde + n;
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        sd[j] = d[j];
        se2[j] = j + 1 < n ? e[j] * e[j] : 0.f;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (i >= n) return;
    const float tiny = 1e-30f;
    float lo = -bnd, hi = bnd;
    for (int it = 0; it < 12; ++it) {
        const float w = (hi - lo) * (1.0f / 33.0f);
        const float x = lo + w * (float)(lane + 1);
        int c = 0;
        float q = sd[0] - x;
        if (q < 0.f) ++c;
        for (int j = 1; j < n; ++j) {
            if (fabsf(q) < tiny) q = -tiny;
            q = (sd[j] - x) - se2[j - 1] / q;
            if (q < 0.f) ++c;
        }
        const unsigned below = __ballot_sync(0xffffffffu, c <= i);   // a prefix of the lanes
        const int l = __popc(below) - 1;                              // last point with count <= i
        const float nlo = l >= 0 ? __shfl_sync(0xffffffffu, x, max(l, 0)) : lo;
        const float nhi = l + 1 < 32 ? __shfl_sync(0xffffffffu, x, min(l + 1, 31)) : hi;
        if (nlo == lo && nhi == hi) break;
        lo = nlo;
        hi = nhi;
        if (hi - lo <= 4.f * FLT_EPSILON * fmaxf(fabsf(lo), fabsf(hi))) break;
    }
    if (lane == 0) lam[i] = 0.5f * (lo + hi);
}

// ------------------------------------------------------------------ 3
// Pivoted LU of T - lam (partial pivoting, LAPACK-style tridiagonal LU): U
// has three diagonals (rdu = reciprocal of its diagonal, du1, du2), L the
// multipliers mul and row swaps piv.  One reciprocal per row; the solves
// below only multiply.
template <typename R>
__device__ void tri_factor(const float* __restrict__ d, const float* __restrict__ e, int n, R lam, R tiny,
                           R* rdu, R* du1, R* du2, R* mul, unsigned char* piv) {
    R ca = R(d[0]) - lam, cb = n > 1 ? R(e[0]) : R(0);
    for (int i = 0; i + 1 < n; ++i) {
        const R c = e[i];
        const R a1 = R(d[i + 1]) - lam;
        const R b1 = (i + 2 < n) ? R(e[i + 1]) : R(0);
        if (fabs(c) > fabs(ca)) {
            const R r = R(1) / c;
            const R m = ca * r;
            rdu[i] = r; du1[i] = a1; du2[i] = b1; mul[i] = m; piv[i] = 1;
            ca = cb - m * a1;
            cb = -m * b1;
        } else {
            if (fabs(ca) < tiny) ca = copysign(tiny, ca);
            const R r = R(1) / ca;
            const R m = c * r;
            rdu[i] = r; du1[i] = cb; du2[i] = R(0); mul[i] = m; piv[i] = 0;
            ca = a1 - m * cb;
            cb = b1;
        }
    }
    if (fabs(ca) < tiny) ca = copysign(tiny, ca);
    rdu[n - 1] = R(1) / ca;
}

template <typename R>
__device__ void tri_solve(int n, const R* rdu, const R* du1, const R* du2, const R* mul,
                          const unsigned char* piv, R* x) {
    for (int i = 0; i + 1 < n; ++i) {
        if (piv[i]) { R t = x[i]; x[i] = x[i + 1]; x[i + 1] = t; }
        x[i + 1] -= mul[i] * x[i];
    }
    x[n - 1] *= rdu[n - 1];
    if (n >= 2) x[n - 2] = (x[n - 2] - du1[n - 2] * x[n - 1]) * rdu[n - 2];
    for (int i = n - 3; i >= 0; --i) x[i] = (x[i] - du1[i] * x[i + 1] - du2[i] * x[i + 2]) * rdu[i];
}

// Inverse iteration, one thread per eigenvalue, in binary64 (R = double)
// or binary32 (R = float); the pivoted LU of T - lam lives in shared memory
// (IT threads per CTA) or in a per-eigenvalue slice of gws.  The vectors of
// distinct eigenvalues come out orthogonal to ~u |T| / gap; vectors inside
// clusters of close eigenvalues are orthonormalised by k_cluster_mgs.
constexpr int IT = 8;

template <typename R>
__global__ void __launch_bounds__(IT) k_invit(const float* __restrict__ d, const float* __restrict__ e,
                                              const float* __restrict__ lam, int n, int i0, double tiny,
                                              float* __restrict__ Y, R* __restrict__ gws) {
    extern __shared__ __align__(16) unsigned char swraw[];
    R* swd = reinterpret_cast<R*>(swraw);
    const int li = blockIdx.x * blockDim.x + threadIdx.x, i = i0 + li;      // eigenvalues i0 .. n-1
    if (i >= n) return;
    const long long per = 5LL * n + (n + sizeof(R) - 1) / sizeof(R);   // R words per eigenvalue in gws
    R* base = gws ? gws + (long long)li * per : swd + (long long)threadIdx.x * 5 * n;
    R* du = base;
    R* du1 = du + n;
    R* du2 = du1 + n;
    R* mul = du2 + n;
    R* x = mul + n;
    unsigned char* piv = gws ? reinterpret_cast<unsigned char*>(base + 5 * n)
                             : reinterpret_cast<unsigned char*>(swd + (long long)blockDim.x * 5 * n) + (long long)threadIdx.x * n;
    tri_factor<R>(d, e, n, (R)lam[i], (R)tiny, du, du1, du2, mul, piv);
    // start from a hashed pseudo-random vector so that the vectors of a
    // degenerate eigenvalue start in different directions
    for (int j = 0; j < n; ++j) {
        unsigned int h = (unsigned int)i * 2654435761u ^ ((unsigned int)j * 2246822519u + 0x9e3779b9u);
        h ^= h >> 15; h *= 2246822519u; h ^= h >> 13; h *= 3266489917u; h ^= h >> 16;
        x[j] = R(0.5) + (R)(h & 0xffffff) * R(1.0 / 16777216.0);
    }
    for (int it = 0; it < 3; ++it) {
        tri_solve<R>(n, du, du1, du2, mul, piv, x);
        R nr = R(0);
        for (int j = 0; j < n; ++j) nr += x[j] * x[j];
        nr = R(1) / sqrt(fmax(nr, sizeof(R) == 8 ? R(1e-300) : R(1e-38)));
        for (int j = 0; j < n; ++j) x[j] *= nr;
    }
    float* yo = Y + (long long)i * n;
    for (int j = 0; j < n; ++j) yo[j] = (float)x[j];
}

// Modified Gram-Schmidt (twice) inside each cluster of near-degenerate
// eigenvalues (consecutive gaps < tol), one CTA per cluster.  Inverse
// iteration cannot separate the vectors of an (almost) multiple eigenvalue;
// Gram-Schmidt turns the differently started vectors into an orthonormal
// basis of the eigenspace.
__global__ void __launch_bounds__(256) k_cluster_mgs(const float* __restrict__ lam, int n, float tol, int n_keep,
                                                     float* __restrict__ Y) {
    __shared__ float red[33];
    const int i0 = blockIdx.x;
    if (i0 > 0 && lam[i0] - lam[i0 - 1] < tol) return;
    int i1 = i0 + 1;
    while (i1 < n && lam[i1] - lam[i1 - 1] < tol) ++i1;
    if (i1 - i0 < 2) return;
    if (i1 <= n - n_keep) return;        // cluster entirely among the discarded (smallest) eigenvalues
    for (int i = i0; i < i1; ++i) {
        float* x = Y + (long long)i * n;
        for (int pass = 0; pass < 2; ++pass)
            for (int q = i0; q < i; ++q) {
                const float* y = Y + (long long)q * n;
                float s = 0.f;
                for (int j = threadIdx.x; j < n; j += blockDim.x) s += y[j] * x[j];
                s = block_sum1024(s, red);
                for (int j = threadIdx.x; j < n; j += blockDim.x) x[j] -= s * y[j];
                __syncthreads();
            }
        float nr = 0.f;
        for (int j = threadIdx.x; j < n; j += blockDim.x) nr += x[j] * x[j];
        nr = rsqrtf(fmaxf(block_sum1024(nr, red), 1e-38f));
        for (int j = threadIdx.x; j < n; j += blockDim.x) x[j] *= nr;
        __syncthreads();
    }
}

// ------------------------------------------------------------------ 4
// X[:, i] = Q Y[i], Q = H_0 ... H_{n-3}; one warp per eigenvector.  With
// MT > 0 each lane keeps its MT entries of the current reflector in
// registers and the next reflector is loaded while the current one is
// applied (n <= 32 MT); MT = 0 is the plain loop for any n.
template <int MT>
__global__ void __launch_bounds__(256) k_backtransform(const float* __restrict__ A, const float* __restrict__ tau,
                                                       int n, const float* __restrict__ Y, double* __restrict__ X) {
    extern __shared__ float sy[];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int i = blockIdx.x * (blockDim.x >> 5) + w;
    if (i >= n) return;
    float* y = sy + (long long)w * n;   // one vector per warp
    for (int j = lane; j < n; j += 32) y[j] = Y[(long long)i * n + j];
    __syncwarp();
    if constexpr (MT == 0) {
        for (int k = n - 3; k >= 0; --k) {
            const float t = tau[k];
            if (t == 0.f) continue;
            const float* v = A + (long long)k * n + k + 1;
            float s = 0.f;
            for (int j = lane; j < n - k - 1; j += 32) s += v[j] * y[k + 1 + j];
            s = warp_sum(s) * t;
            for (int j = lane; j < n - k - 1; j += 32) y[k + 1 + j] -= s * v[j];
            __syncwarp();
        }
    } else {
        float vn[MT], vc[MT];
        auto load = [&](float (&v)[MT], int k) {
            const float* src = A + (long long)k * n + k + 1;
            const int m = n - k - 1;
#pragma unroll
            for (int q = 0; q < MT; ++q) {
                const int j = lane + 32 * q;
                v[q] = j < m ? src[j] : 0.f;
            }
        };
        if (n >= 3) load(vn, n - 3);
        float tn = n >= 3 ? tau[n - 3] : 0.f;
        for (int k = n - 3; k >= 0; --k) {
            const float t = tn;
#pragma unroll
            for (int q = 0; q < MT; ++q) vc[q] = vn[q];
            if (k > 0) {
                load(vn, k - 1);
                tn = tau[k - 1];
            }
            if (t == 0.f) continue;
            const int m = n - k - 1;
            float s = 0.f;
#pragma unroll
            for (int q = 0; q < MT; ++q) {
                const int j = lane + 32 * q;
                if (j < m) s += vc[q] * y[k + 1 + j];
            }
            s = warp_sum(s) * t;
#pragma unroll
            for (int q = 0; q < MT; ++q) {
                const int j = lane + 32 * q;
                if (j < m) y[k + 1 + j] -= s * vc[q];
            }
            __syncwarp();
        }
    }
    for (int j = lane; j < n; j += 32) X[(long long)j * n + i] = (double)y[j];
}

// Blocked back-transformation for large n (compact WY form): the reflectors
// k0 .. k0 + nb - 1 give Q_b = H_k0 ... H_k0+nb-1 = I - V T V^T, V the
// reflectors as columns (v_k stored in row k of A from column k + 1), T upper
// triangular (T_ii = tau_i, T_{0:i,i} = -tau_i T_{0:i,0:i} V_{:,0:i}^T v_i).
// Y <- Q_b Y for the blocks from last to first, each as binary32 products
// W = V^T Y, W = T W, Y -= V W: the same arithmetic as one reflector at a
// time, with every reflector read once per block instead of once per vector.
// Vt [nb][m]: Vt[r][j] = v_{k0+r}[k0 + 1 + j] (zero where j < r), m = n - k0 - 1
__global__ void k_wy_vt(const float* __restrict__ A, int n, int k0, int nb, float* __restrict__ Vt) {
    const int m = n - k0 - 1;
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= (long long)nb * m) return;
    const int r = (int)(t / m), j = (int)(t % m);
    Vt[t] = j >= r ? A[(long long)(k0 + r) * n + k0 + 1 + j] : 0.f;
}

// T from G = V^T V (nb x nb) and tau (one CTA, column by column)
__global__ void k_wy_t(const float* __restrict__ G, const float* __restrict__ tau, int k0, int nb,
                       float* __restrict__ T) {
    const int r = threadIdx.x;
    for (int t = r; t < nb * nb; t += blockDim.x) T[t] = 0.f;
    __syncthreads();
    for (int i = 0; i < nb; ++i) {
        const float ti = tau[k0 + i];
        float acc = 0.f;
        if (r < i) {
            for (int q = r; q < i; ++q) acc += T[r * nb + q] * G[q * nb + i];
        }
        __syncthreads();
        if (r < i) T[r * nb + i] = -ti * acc;
        if (r == i) T[i * nb + i] = ti;
        __syncthreads();
    }
}

// X[j][i0 + q] = Y[q][j] (binary64), q < nv
__global__ void k_wy_out(const float* __restrict__ Y, int n, int i0, int nv, double* __restrict__ X) {
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= (long long)nv * n) return;
    const int j = (int)(t / nv), q = (int)(t % nv);
    X[(long long)j * n + i0 + q] = (double)Y[(long long)q * n + j];
}

// ------------------------------------------------------------------ 5
__global__ void k_identity_minus(double* __restrict__ R, int n) {     // R <- I - R
    long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= (long long)n * n) return;
    int i = (int)(t / n), j = (int)(t % n);
    R[t] = (i == j ? 1.0 : 0.0) - R[t];
}

// lam_i = S_ii/(1 - R_ii); sums for delta (single CTA, deterministic)
// Refinement statistics, stage 1: lam_i = S_ii / (1 - R_ii) and per-CTA
// partial sums of |S - diag(lam)|^2, |R|^2, |g|^2 over rows blockIdx.x,
// blockIdx.x + gridDim.x, ... (binary64 is 1/64 rate: spread over all SMs).
__global__ void __launch_bounds__(256) k_oa_stats(const double* __restrict__ S, const double* __restrict__ R,
                                                  const double* __restrict__ g, int n, double* __restrict__ lam,
                                                  double* __restrict__ part) {
    __shared__ double red[33];
    double a = 0.0, b = 0.0, c = 0.0;
    for (int i = blockIdx.x; i < n; i += gridDim.x) {
        const double li = S[(long long)i * n + i] / (1.0 - R[(long long)i * n + i]);
        if (threadIdx.x == 0) lam[i] = li;
        for (int j = threadIdx.x; j < n; j += blockDim.x) {
            const long long t = (long long)i * n + j;
            const double s = S[t] - (i == j ? li : 0.0);
            a = fma(s, s, a);
            b = fma(R[t], R[t], b);
            c = fma(g[t], g[t], c);
        }
    }
    a = block_sum1024d(a, red);
    b = block_sum1024d(b, red);
    c = block_sum1024d(c, red);
    if (threadIdx.x == 0) {
        part[blockIdx.x] = a;
        part[gridDim.x + blockIdx.x] = b;
        part[2 * gridDim.x + blockIdx.x] = c;
    }
}

// Stage 2 (one warp, fixed order): out[0] = delta for the clustering test,
// out[1] = |S - diag| / |g|, out[2] = |I - X^T X|.
__global__ void k_oa_stats_fin(const double* __restrict__ part, int np, double* __restrict__ out) {
    if (threadIdx.x != 0) return;
    double a = 0.0, b = 0.0, c = 0.0;
    for (int q = 0; q < np; ++q) {
        a += part[q];
        b += part[np + q];
        c += part[2 * np + q];
    }
    out[0] = 2.0 * (sqrt(a) + sqrt(c) * sqrt(b));
    out[1] = sqrt(a) / fmax(sqrt(c), 1e-300);
    out[2] = sqrt(b);
}

__global__ void k_oa_E(const double* __restrict__ S, const double* __restrict__ R, const double* __restrict__ lam,
                       const double* __restrict__ delta, int n, double* __restrict__ E) {
    long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= (long long)n * n) return;
    int i = (int)(t / n), j = (int)(t % n);
    double r = R[t];
    if (i == j) { E[t] = 0.5 * r; return; }
    double dl = lam[j] - lam[i];
    E[t] = fabs(dl) > *delta ? (S[t] + lam[j] * r) / dl : 0.5 * r;
}

// ------------------------------------------------------------------ 6
__global__ void k_rank_desc_ld(const double* __restrict__ ev, int n, int n_sub, int* __restrict__ sel) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double e = ev[i];
    int r = 0;
    for (int j = 0; j < n; ++j) {
        double f = ev[j];
        r += (f > e) || (f == e && j < i);
    }
    if (r < n_sub) sel[r] = i;
}

__global__ void k_gather_cols(const double* __restrict__ X, int n, int n_sub, const int* __restrict__ sel,
                              double* __restrict__ B) {
    long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= (long long)n * n_sub) return;
    int row = (int)(t / n_sub), k = (int)(t % n_sub);
    B[t] = X[(long long)row * n + sel[k]];
}

__global__ void k_ns_coeff(double* __restrict__ G, int m) {          // G <- (3 I - G)/2
    long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= (long long)m * m) return;
    int i = (int)(t / m), j = (int)(t % m);
    G[t] = 0.5 * ((i == j ? 3.0 : 0.0) - G[t]);
}

__global__ void k_ns_coeff32(float* __restrict__ G, int m) {          // G <- (3 I - G)/2
    long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= (long long)m * m) return;
    int i = (int)(t / m), j = (int)(t % m);
    G[t] = 0.5f * ((i == j ? 3.f : 0.f) - G[t]);
}

// lam[k] = B[:, k]^T T[:, k] (B, T row-major n x n_sub), one CTA per column;
// lam[n_sub + k] = lam[k]^-1/2 (0 for lam[k] <= 0), the column's scale factor
__global__ void __launch_bounds__(256) k_rayleigh_cols(const double* __restrict__ B, const double* __restrict__ T,
                                                       int n, int n_sub, double* __restrict__ lam) {
    __shared__ double red[33];
    const int k = blockIdx.x;
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) s = fma(B[(long long)i * n_sub + k], T[(long long)i * n_sub + k], s);
    s = block_sum1024d(s, red);
    if (threadIdx.x == 0) {
        lam[k] = s;
        lam[n_sub + k] = s > 0.0 ? 1.0 / sqrt(s) : 0.0;
    }
}
// B[:, k] *= lam[n_sub + k] (= lam[k]^-1/2); flags a rank-deficient selection
__global__ void __launch_bounds__(256) k_scale_cols_by(double* __restrict__ B, int n, int n_sub,
                                                       const double* __restrict__ lam, int* status) {
    long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (blockIdx.x == 0) {
        // the rank check: min and max of the quotients by the whole first block
        __shared__ double smin[8], smax[8];
        double lmax = -INFINITY, lmin = INFINITY;
        for (int k = threadIdx.x; k < n_sub; k += blockDim.x) {
            lmax = fmax(lmax, lam[k]);
            lmin = fmin(lmin, lam[k]);
        }
        for (int o = 16; o > 0; o >>= 1) {
            lmax = fmax(lmax, __shfl_xor_sync(0xffffffffu, lmax, o));
            lmin = fmin(lmin, __shfl_xor_sync(0xffffffffu, lmin, o));
        }
        if ((threadIdx.x & 31) == 0) {
            smax[threadIdx.x >> 5] = lmax;
            smin[threadIdx.x >> 5] = lmin;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
                lmax = fmax(lmax, smax[w]);
                lmin = fmin(lmin, smin[w]);
            }
            lmax = fmax(lmax, smax[0]);
            lmin = fmin(lmin, smin[0]);
            if (!(lmin >= 1e-12 * lmax) || !(lmax > 0.0)) atomicOr(status, ST_RANK);
        }
    }
    if (t >= (long long)n * n_sub) return;
    B[t] *= lam[n_sub + (int)(t % n_sub)];
}
__global__ void k_top_indices(int n, int n_sub, int* __restrict__ sel) {   // ascending order -> top n_sub, descending
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n_sub) sel[k] = n - 1 - k;
}
__global__ void k_scale_cols(double* __restrict__ B, int n, int n_sub, const double* __restrict__ lam,
                             const int* __restrict__ sel, int* status) {
    long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t == 0) {
        double lmax = lam[sel[0]], lmin = lam[sel[n_sub - 1]];
        if (!(lmin >= 1e-12 * lmax) || !(lmax > 0.0)) atomicOr(status, ST_RANK);
    }
    if (t >= (long long)n * n_sub) return;
    double l = lam[sel[(int)(t % n_sub)]];
    B[t] = l > 0.0 ? B[t] / sqrt(l) : 0.0;
}

}  // namespace

void launch_to_f32(gw_ctx* ctx, const double* a, float* b, long long n);

// g (n x n, binary64, symmetric) -> B (n x n_sub) = xi_top lambda_top^-1/2
// Z[:, j] and Zup[:, j] (rows x n_sub, row-major) scaled by lambda_j^-1/2,
// lambda_j = Z[:, j]^T Zup[:, j] (= Z_j^T v Z_j when Zup = v Z), so that
// Z^T v Z has a unit diagonal in binary64; flags a rank-deficient basis.
void basis_rayleigh_scale(gw_ctx* ctx, double* Z, double* Zup, int rows, int n_sub) {
    double* lam = dalloc<double>(ctx, 2 * (size_t)n_sub);      // quotients, then their scale factors
    try {
        klaunch(ctx, "k_rayleigh_cols", k_rayleigh_cols, n_sub, 256, 0, (const double*)Z, (const double*)Zup, rows,
                n_sub, lam);
        klaunch(ctx, "k_scale_cols_by", k_scale_cols_by, div_up((long long)rows * n_sub, 256), 256, 0, Z, rows, n_sub,
                (const double*)lam, ctx->d_status);
        klaunch(ctx, "k_scale_cols_by", k_scale_cols_by, div_up((long long)rows * n_sub, 256), 256, 0, Zup, rows,
                n_sub, (const double*)lam, ctx->d_status);
    } catch (...) {
        ctx_free(ctx, lam);
        throw;
    }
    ctx_free(ctx, lam);
}

// All eigenvalues of g (ascending) in binary32: the tridiagonalisation and
// multisection of eigh_top_scaled without the vectors (threshold-driven
// choice of the subspace dimension).
std::vector<float> eigvals32(gw_ctx* ctx, const double* g, const float* g32, int n) {
    const long long nn = (long long)n * n;
    float *A32 = nullptr, *d = nullptr, *e = nullptr, *tau = nullptr, *lam32 = nullptr, *vb = nullptr, *pb = nullptr,
          *pt = nullptr;
    unsigned int* bar = nullptr;
    std::vector<float> out(n);
    auto release = [&]() {
        for (void* p : {(void*)A32, (void*)d, (void*)e, (void*)tau, (void*)lam32, (void*)vb, (void*)pb, (void*)pt,
                        (void*)bar})
            ctx_free(ctx, p);
    };
    try {
        A32 = dalloc<float>(ctx, nn);
        d = dalloc<float>(ctx, n); e = dalloc<float>(ctx, n); tau = dalloc<float>(ctx, n);
        lam32 = dalloc<float>(ctx, n);
        if (g32) CUDA_CHECK(cudaMemcpyAsync(A32, g32, sizeof(float) * nn, cudaMemcpyDeviceToDevice, ctx->stream));
        else launch_to_f32(ctx, g, A32, nn);
        const int rows = (n + CL - 1) / CL;
        const size_t smem_cl = sizeof(float) * ((size_t)rows * n + 5 * (size_t)n);
        if (smem_cl <= 220 * 1024) {
            allow_max_smem(k_sytrd32_cl);
            klaunch(ctx, "k_sytrd32_cl", k_sytrd32_cl, CL, 1024, smem_cl, A32, n, d, e, tau);
        } else {
            const size_t smem = 3 * (size_t)n * sizeof(float);
            if (smem > 200 * 1024) gw_throw(GW_ERR_INVALID_ARG, "compression rank too large for the eigensolver");
            allow_max_smem(k_sytrd32_grid);
            const int grid = ctx->num_sms;
            vb = dalloc<float>(ctx, n); pb = dalloc<float>(ctx, 2 * (size_t)n); pt = dalloc<float>(ctx, 2 * (size_t)grid);
            bar = dalloc<unsigned int>(ctx, 2);
            CUDA_CHECK(cudaMemsetAsync(bar, 0, 2 * sizeof(unsigned int), ctx->stream));
            // bounded grid barriers: a CTA gives up after poll_limit polls (about a second by default)
            unsigned long long poll_limit = ctx->barrier_polls ? (unsigned long long)ctx->barrier_polls : (1ull << 25);
            void* args[] = {&A32, (void*)&n, &d, &e, &tau, &vb, &pb, &pt, &bar, &ctx->d_status, &poll_limit};
            prof_begin(ctx, "k_sytrd32_grid");
            CUDA_CHECK(cudaLaunchCooperativeKernel((const void*)k_sytrd32_grid, dim3(grid), dim3(512), args, smem,
                                                   ctx->stream));
            after_launch(ctx, "k_sytrd32_grid");
            ctx_finish(ctx, "tridiagonalisation");     // a timed-out barrier stops here, before T is used
        }
        std::vector<float> hd(n), he(n);
        CUDA_CHECK(cudaMemcpyAsync(hd.data(), d, n * sizeof(float), cudaMemcpyDeviceToHost, ctx->stream));
        CUDA_CHECK(cudaMemcpyAsync(he.data(), e, n * sizeof(float), cudaMemcpyDeviceToHost, ctx->stream));
        CUDA_CHECK(cudaStreamSynchronize(ctx->stream));
        float bnd = 0.f;
        for (int i = 0; i < n; ++i) {
            float r = std::fabs(hd[i]) + (i > 0 ? std::fabs(he[i - 1]) : 0.f) + (i + 1 < n ? std::fabs(he[i]) : 0.f);
            bnd = std::max(bnd, r);
        }
        bnd = bnd * 1.01f + 1e-30f;
        allow_max_smem(k_bisect);
        if (2 * (size_t)n * sizeof(float) > 200 * 1024) gw_throw(GW_ERR_INVALID_ARG, "rank too large for the bisection");
        klaunch(ctx, "k_bisect", k_bisect, div_up(n, 8), 256, 2 * (size_t)n * sizeof(float), (const float*)d,
                (const float*)e, n, bnd, lam32);
        CUDA_CHECK(cudaMemcpyAsync(out.data(), lam32, n * sizeof(float), cudaMemcpyDeviceToHost, ctx->stream));
        ctx_finish(ctx, "eigenvalues of g");
    } catch (...) {
        release();
        throw;
    }
    release();
    return out;
}

void eigh_top_scaled(gw_ctx* ctx, const double* g, const float* g32, int n, int n_sub, int oa_iters, double oa_tol,
                     bool vectors_f64, double* B) {
    if (!g && oa_iters > 0) gw_throw(GW_ERR_INVALID_ARG, "eigensolver refinement needs the binary64 matrix");
    const long long nn = (long long)n * n;
    float* A32 = nullptr; float *d = nullptr, *e = nullptr, *tau = nullptr, *lam32 = nullptr, *Y = nullptr;
    double *X = nullptr, *X2 = nullptr, *R = nullptr, *S = nullptr, *T = nullptr, *E = nullptr, *lam = nullptr;
    double *stat = nullptr, *G = nullptr, *Bt = nullptr;
    void* gws = nullptr;
    float *vb = nullptr, *pb = nullptr, *pt = nullptr, *Bt32 = nullptr, *G32 = nullptr, *B32 = nullptr;
    unsigned int* bar = nullptr;
    int* sel = nullptr;
    auto release = [&]() {
        for (void* p : {(void*)A32, (void*)d, (void*)e, (void*)tau, (void*)lam32, (void*)Y,
                        (void*)X, (void*)X2, (void*)R, (void*)S, (void*)T, (void*)E, (void*)lam, (void*)stat,
                        (void*)G, (void*)Bt, (void*)sel, (void*)gws, (void*)vb, (void*)pb, (void*)pt,
                        (void*)bar, (void*)Bt32, (void*)G32, (void*)B32})
            ctx_free(ctx, p);
    };
    try {
        A32 = dalloc<float>(ctx, nn);
        d = dalloc<float>(ctx, n); e = dalloc<float>(ctx, n); tau = dalloc<float>(ctx, n);
        lam32 = dalloc<float>(ctx, n);
        Y = dalloc<float>(ctx, nn);
        X = dalloc<double>(ctx, nn);
        if (g32) CUDA_CHECK(cudaMemcpyAsync(A32, g32, sizeof(float) * nn, cudaMemcpyDeviceToDevice, ctx->stream));
        else launch_to_f32(ctx, g, A32, nn);
        const int rows = (n + CL - 1) / CL;
        const size_t smem_cl = sizeof(float) * ((size_t)rows * n + 5 * (size_t)n);
        if (smem_cl <= 220 * 1024) {
            allow_max_smem(k_sytrd32_cl);
            klaunch(ctx, "k_sytrd32_cl", k_sytrd32_cl, CL, 1024, smem_cl, A32, n, d, e, tau);
        } else {
            const size_t smem = 3 * (size_t)n * sizeof(float);
            if (smem > 200 * 1024) gw_throw(GW_ERR_INVALID_ARG, "compression rank too large for the eigensolver");
            allow_max_smem(k_sytrd32_grid);
            int per_sm = 0;
            CUDA_CHECK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sytrd32_grid, 512, smem));
            if (per_sm < 1) gw_throw(GW_ERR_CUDA, "tridiagonalisation kernel cannot be resident");
            const int grid = ctx->num_sms;          // one CTA per SM, co-resident (cooperative launch)
            vb = dalloc<float>(ctx, n);
            pb = dalloc<float>(ctx, 2 * (size_t)n);          // two parities
            pt = dalloc<float>(ctx, 2 * (size_t)grid);
            bar = dalloc<unsigned int>(ctx, 2);
            CUDA_CHECK(cudaMemsetAsync(bar, 0, 2 * sizeof(unsigned int), ctx->stream));
            // bounded grid barriers: a CTA gives up after poll_limit polls (about a second by default)
            unsigned long long poll_limit = ctx->barrier_polls ? (unsigned long long)ctx->barrier_polls : (1ull << 25);
            void* args[] = {&A32, (void*)&n, &d, &e, &tau, &vb, &pb, &pt, &bar, &ctx->d_status, &poll_limit};
            prof_begin(ctx, "k_sytrd32_grid");
            CUDA_CHECK(cudaLaunchCooperativeKernel((const void*)k_sytrd32_grid, dim3(grid), dim3(512), args, smem,
                                                   ctx->stream));
            after_launch(ctx, "k_sytrd32_grid");
            ctx_finish(ctx, "tridiagonalisation");     // a timed-out barrier stops here, before T is used
        }
        // Gershgorin bound of T (host needs d, e: small copy)
        std::vector<float> hd(n), he(n);
        CUDA_CHECK(cudaMemcpyAsync(hd.data(), d, n * sizeof(float), cudaMemcpyDeviceToHost, ctx->stream));
        CUDA_CHECK(cudaMemcpyAsync(he.data(), e, n * sizeof(float), cudaMemcpyDeviceToHost, ctx->stream));
        CUDA_CHECK(cudaStreamSynchronize(ctx->stream));
        float bnd = 0.f;
        for (int i = 0; i < n; ++i) {
            float r = std::fabs(hd[i]) + (i > 0 ? std::fabs(he[i - 1]) : 0.f) + (i + 1 < n ? std::fabs(he[i]) : 0.f);
            bnd = std::max(bnd, r);
        }
        bnd = bnd * 1.01f + 1e-30f;
        allow_max_smem(k_bisect);       // d and e^2 staged in shared memory: 8 n bytes
        if (2 * (size_t)n * sizeof(float) > 200 * 1024) gw_throw(GW_ERR_INVALID_ARG, "rank too large for the bisection");
        klaunch(ctx, "k_bisect", k_bisect, div_up(n, 8), 256, 2 * (size_t)n * sizeof(float), (const float*)d,
                (const float*)e, n, bnd, lam32);
        // cluster tolerance: eigenvalue gaps below which inverse iteration cannot keep
        // the vectors orthogonal in its working precision
        const float cl_tol = (vectors_f64 ? 1e-6f : 1e-4f) * bnd;
        // the vectors needed: every one for the binary64 refinement, else the top
        // n_sub and the rest of a cluster that the cut runs through (the kept
        // vectors of that cluster are orthogonalised against its discarded ones);
        // the others stay zero
        int i0 = 0;
        if (oa_iters == 0) {
            std::vector<float> hl(n);
            CUDA_CHECK(cudaMemcpyAsync(hl.data(), lam32, n * sizeof(float), cudaMemcpyDeviceToHost, ctx->stream));
            CUDA_CHECK(cudaStreamSynchronize(ctx->stream));
            i0 = n - n_sub;
            while (i0 > 0 && hl[i0] - hl[i0 - 1] < cl_tol) --i0;
        }
        // binary64 vectors when they are refined to binary64 accuracy afterwards
        auto invit = [&](auto zero) {
            typedef decltype(zero) R;
            const double tiny = (sizeof(R) == 8 ? 1e-13 : 1e-6) * (double)bnd;
            const size_t per_thread = (size_t)n * (5 * sizeof(R) + 1);
            if (per_thread <= 200 * 1024) {
                // few threads per CTA so that the eigenvalues spread over all SMs
                const int it_threads = (int)std::max<size_t>(
                    1, std::min(std::min((size_t)IT, (200 * 1024) / per_thread), (size_t)div_up(n, ctx->num_sms)));
                const size_t smem_it = per_thread * it_threads + 16;
                allow_max_smem(k_invit<R>);
                klaunch(ctx, "k_invit", k_invit<R>, div_up(n - i0, it_threads), it_threads, smem_it, (const float*)d,
                        (const float*)e, (const float*)lam32, n, i0, tiny, Y, (R*)nullptr);
            } else {
                const size_t per = 5 * (size_t)n + (n + sizeof(R) - 1) / sizeof(R);
                gws = ctx_alloc(ctx, (size_t)(n - i0) * per * sizeof(R));
                klaunch(ctx, "k_invit", k_invit<R>, div_up(n - i0, IT), IT, 0, (const float*)d, (const float*)e,
                        (const float*)lam32, n, i0, tiny, Y, (R*)gws);
            }
        };
        if (i0 > 0) CUDA_CHECK(cudaMemsetAsync(Y, 0, sizeof(float) * (size_t)i0 * n, ctx->stream));
        if (vectors_f64) invit(0.0);
        else invit(0.0f);
        // clusters (the refinement of the binary64 path works on every vector;
        // without it only the clusters that hold kept vectors matter)
        klaunch(ctx, "k_cluster_mgs", k_cluster_mgs, n, 256, 0, (const float*)lam32, n, cl_tol,
                oa_iters > 0 ? n : n_sub, Y);
        // two warps per CTA: the vectors spread over all SMs
        const int bt_warps = (int)std::max<size_t>(1, std::min<size_t>(2, (200 * 1024) / ((size_t)n * sizeof(float))));
        const size_t smem_bt = (size_t)bt_warps * n * sizeof(float);
        auto backtransform = [&](auto kern) {
            allow_max_smem(kern);
            klaunch(ctx, "k_backtransform", kern, div_up(n, bt_warps), 32 * bt_warps, smem_bt, (const float*)A32,
                    (const float*)tau, n, (const float*)Y, X);
        };
        if (n <= 32 * 8) backtransform(k_backtransform<8>);
        else if (n <= 32 * 16) backtransform(k_backtransform<16>);
        else if (n <= 32 * 24) backtransform(k_backtransform<24>);
        else {
            // compact WY blocks of WYB reflectors, binary32 products (Y rows i0 .. n-1 in place)
            constexpr int WYB = 64;
            const int nv = n - i0;
            float* Yv = Y + (size_t)i0 * n;
            float* Vt = dalloc<float>(ctx, (size_t)WYB * n);
            float* Gm = nullptr; float* Tm = nullptr; float* Wm = nullptr; float* W2 = nullptr;
            try {
                Gm = dalloc<float>(ctx, WYB * WYB);
                Tm = dalloc<float>(ctx, WYB * WYB);
                Wm = dalloc<float>(ctx, (size_t)WYB * nv);
                W2 = dalloc<float>(ctx, (size_t)WYB * nv);
                const int nref = n - 2;                         // reflectors 0 .. n-3
                for (int k0 = ((nref - 1) / WYB) * WYB; k0 >= 0; k0 -= WYB) {
                    const int nb = std::min(WYB, nref - k0), m = n - k0 - 1;
                    klaunch(ctx, "k_backtransform", k_wy_vt, div_up((long long)nb * m, 256), 256, 0,
                            (const float*)A32, n, k0, nb, Vt);
                    gemm_f32(ctx, false, true, nb, nb, m, 1.f, Vt, m, Vt, m, 0.f, Gm, nb);        // G = V^T V
                    klaunch(ctx, "k_backtransform", k_wy_t, 1, 64, 0, (const float*)Gm, (const float*)tau, k0, nb,
                            Tm);
                    gemm_f32(ctx, false, true, nb, nv, m, 1.f, Vt, m, Yv + k0 + 1, n, 0.f, Wm, nv);  // W = V^T Y
                    gemm_f32(ctx, false, false, nb, nv, nb, 1.f, Tm, nb, Wm, nv, 0.f, W2, nv);      // W = T W
                    gemm_f32(ctx, true, false, nv, m, nb, -1.f, W2, nv, Vt, m, 1.f, Yv + k0 + 1, n); // Y -= V W
                }
                klaunch(ctx, "k_backtransform", k_wy_out, div_up((long long)nv * n, 256), 256, 0, (const float*)Yv,
                        n, i0, nv, X);
            } catch (...) {
                ctx_free(ctx, Vt); ctx_free(ctx, Gm); ctx_free(ctx, Tm); ctx_free(ctx, Wm); ctx_free(ctx, W2);
                throw;
            }
            ctx_free(ctx, Vt); ctx_free(ctx, Gm); ctx_free(ctx, Tm); ctx_free(ctx, Wm); ctx_free(ctx, W2);
        }
        // binary64 refinement
        if (oa_iters > 0) {
            X2 = dalloc<double>(ctx, nn); R = dalloc<double>(ctx, nn); S = dalloc<double>(ctx, nn);
            E = dalloc<double>(ctx, nn);
        }
        T = dalloc<double>(ctx, nn); lam = dalloc<double>(ctx, std::max(n, 2 * n_sub));
        const int n_part = ctx->num_sms;
        stat = dalloc<double>(ctx, 3 + 3 * (size_t)n_part);      // [3) results, then the partial sums
        auto oa_stats = [&]() {
            klaunch(ctx, "k_oa_stats", k_oa_stats, n_part, 256, 0, (const double*)S, (const double*)R, g, n, lam,
                    stat + 3);
            klaunch(ctx, "k_oa_stats_fin", k_oa_stats_fin, 1, 32, 0, (const double*)(stat + 3), n_part, stat);
        };
        double hstat[3] = {0, 0, 0};
        for (int it = 0; it < oa_iters; ++it) {
            gemm_f64(ctx, true, false, n, n, n, 1.0, X, n, X, n, 0.0, R, n);           // X^T X
            klaunch(ctx, "k_identity_minus", k_identity_minus, div_up(nn, 256), 256, 0, R, n);
            gemm_f64(ctx, false, false, n, n, n, 1.0, g, n, X, n, 0.0, T, n);          // g X
            gemm_f64(ctx, true, false, n, n, n, 1.0, X, n, T, n, 0.0, S, n);           // X^T g X
            oa_stats();
            klaunch(ctx, "k_oa_E", k_oa_E, div_up(nn, 256), 256, 0, (const double*)S, (const double*)R,
                    (const double*)lam, (const double*)stat, n, E);
            // stop once the basis is an eigenbasis to working accuracy (residual of
            // the previous iterate; the correction below squares it once more)
            CUDA_CHECK(cudaMemcpyAsync(hstat, stat, 3 * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
            CUDA_CHECK(cudaStreamSynchronize(ctx->stream));
            const bool done = it > 0 && hstat[1] < oa_tol && hstat[2] < 1e3 * oa_tol;
            CUDA_CHECK(cudaMemcpyAsync(X2, X, nn * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
            gemm_f64(ctx, false, false, n, n, n, 1.0, X, n, E, n, 1.0, X2, n);         // X + X E
            std::swap(X, X2);
            if (done) break;
        }
        sel = dalloc<int>(ctx, n_sub);
        Bt = dalloc<double>(ctx, (size_t)n * n_sub);
        G = dalloc<double>(ctx, (size_t)n_sub * n_sub);
        if (oa_iters == 0) {
            // no refinement: the top n_sub of the binary32 eigenvalues (ascending
            // from the bisection), re-orthonormalised, scaled by the binary64
            // Rayleigh quotients of the re-orthonormalised vectors
            klaunch(ctx, "k_top_indices", k_top_indices, div_up(n_sub, 256), 256, 0, n, n_sub, sel);
        } else {
            klaunch(ctx, "k_rank_desc_ld", k_rank_desc_ld, div_up(n, 256), 256, 0, (const double*)lam, n, n_sub, sel);
        }
        klaunch(ctx, "k_gather_cols", k_gather_cols, div_up((long long)n * n_sub, 256), 256, 0, (const double*)X, n,
                n_sub, (const int*)sel, Bt);
        if (oa_iters == 0 && !g) {
            // binary32 basis (the caller forms Z = X_r B in binary32): the
            // Newton-Schulz step B = Bt (3 I - Bt^T Bt) / 2 in binary32 as well
            Bt32 = dalloc<float>(ctx, (size_t)n * n_sub);
            G32 = dalloc<float>(ctx, (size_t)n_sub * n_sub);
            B32 = dalloc<float>(ctx, (size_t)n * n_sub);
            launch_to_f32(ctx, Bt, Bt32, (long long)n * n_sub);
            gemm_f32(ctx, true, false, n_sub, n_sub, n, 1.f, Bt32, n_sub, Bt32, n_sub, 0.f, G32, n_sub);
            klaunch(ctx, "k_ns_coeff32", k_ns_coeff32, div_up((long long)n_sub * n_sub, 256), 256, 0, G32, n_sub);
            gemm_f32(ctx, false, false, n, n_sub, n_sub, 1.f, Bt32, n_sub, G32, n_sub, 0.f, B32, n_sub);
            launch_to_f64(ctx, B32, B, (long long)n * n_sub);
        } else {
            gemm_f64(ctx, true, false, n_sub, n_sub, n, 1.0, Bt, n_sub, Bt, n_sub, 0.0, G, n_sub);
            klaunch(ctx, "k_ns_coeff", k_ns_coeff, div_up((long long)n_sub * n_sub, 256), 256, 0, G, n_sub);
            gemm_f64(ctx, false, false, n, n_sub, n_sub, 1.0, Bt, n_sub, G, n_sub, 0.0, B, n_sub);
        }
        if (oa_iters == 0 && !g) {
            // no binary64 g: B is returned orthonormal and unscaled (the caller
            // scales the basis it builds from it)
        } else if (oa_iters == 0) {
            gemm_f64(ctx, false, false, n, n_sub, n, 1.0, g, n, B, n_sub, 0.0, T, n_sub);     // g B
            klaunch(ctx, "k_rayleigh_cols", k_rayleigh_cols, n_sub, 256, 0, (const double*)B, (const double*)T, n,
                    n_sub, lam);
            klaunch(ctx, "k_scale_cols_by", k_scale_cols_by, div_up((long long)n * n_sub, 256), 256, 0, B, n, n_sub,
                    (const double*)lam, ctx->d_status);
        } else {
            klaunch(ctx, "k_scale_cols", k_scale_cols, div_up((long long)n * n_sub, 256), 256, 0, B, n, n_sub,
                    (const double*)lam, (const int*)sel, ctx->d_status);
        }
    } catch (...) {
        release();
        throw;
    }
    release();
}
