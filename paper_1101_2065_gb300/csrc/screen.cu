// a5 + a6: screening and self-energy forms, batched over all frequencies.
//
// a5  M_k = 1 - chi0_k is complex symmetric (chi0 is symmetric in the real
//     product basis, Sec. 4).  It is factorised in place as M_k = L D L^T
//     (unit lower L, diagonal D, no pivoting) by a right-looking blocked
//     algorithm with NB-column panels.  Each panel step is two launches over
//     all N frequencies at once: k_ldlt_panel (one CTA per frequency: the
//     NB x NB diagonal block factorised by one warp in shared memory, the
//     rows below solved against it one row per thread) and the trailing
//     update M22 -= L21 D L21^T: k_ldlt_syrk (one CTA per frequency and
//     64 x 64 tile, FMA units) or, on the binary32 path for 128 rows and
//     more, k_ldlt_syrk_tc (one CTA per frequency and 128-row block, 3xTF32
//     on the tensor cores).  While 128 rows remain after the next panel, the
//     binary32 path takes two panels per pass over the trailing matrix: the
//     first panel's update of the next panel's columns, that panel, then
//     k_ldlt_syrk_tc2 for both updates of the rest, with the rounding of two
//     separate passes.  The steps are small one by one, but N of them
//     side by side fill the GPU.  chi^RPA_k = M_k^-1 chi0_k = M_k^-1 - 1
//     (Eq. chi_RPA) is never formed on the hot path: the forms only need
//     M_k^-1.
// a6  c_r(s_k) = q_r^T gamma_k q_r with gamma_k = -(1/pi) Im chi^RPA_k, and
//     q^T chi^RPA q = q^T M^-1 q - q^T q with q real, so
//     c_r = -(1/pi) Im sum_i y_i^2 / d_i,  y = L^-1 q.  One CTA per
//     frequency and chunk of right-hand sides keeps its chunk of Y in shared
//     memory for the whole blocked forward substitution: per panel it applies
//     the inverse of the unit lower diagonal block (precomputed by the panel
//     step of a5, so no serial chain remains), adds y_i^2/d_i to binary64
//     sums, and updates the rows below from L tiles streamed through a
//     cp.async double buffer (k_forms).  The binary32 path with N_sub <= 384
//     keeps the updates in tensor memory instead and runs them as 3xTF32
//     products (k_forms_tm).  c_r(s_0) = 0 (odd spectral function).
#include <algorithm>
#include <cmath>

#include "internal.h"
#include "tc.cuh"

namespace {

// Panel width NB; trailing-update tile T x T with A x A complex outputs per
// thread; the forms stream L in tiles of FT rows.  binary64 is issue-bound
// (1/64 of the binary32 rate): small tiles waste less on the triangle and
// keep the panel row in registers.
template <typename C> struct Tile;
template <> struct Tile<double2> { static constexpr int NB = 16, T = 32, A = 2, FT = 32; };
template <> struct Tile<float2> { static constexpr int NB = 32, T = 64, A = 4, FT = 64; };

// shared-memory row pitch of an NB-wide tile (a multiple of 16 bytes, for cp.async)
template <typename C> __host__ __device__ constexpr int tile_pitch() {
    return sizeof(C) == 8 ? Tile<C>::NB + 2 : Tile<C>::NB + 1;
}

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

// row of packed lower-triangular index t (tri(i) <= t < tri(i + 1))
__device__ __forceinline__ int tri_row(long long t) {
    int i = (int)((sqrtf(8.0f * (float)t + 1.0f) - 1.0f) * 0.5f);
    while (tri(i) > t) --i;
    while (tri(i + 1) <= t) ++i;
    return i;
}

// M = delta - X for packed entry t (delta = 1 on the diagonal); returns |M|^2
template <typename C>
__device__ __forceinline__ typename CT<C>::R init_elem(const C* __restrict__ X, C* __restrict__ M, long long t) {
    typedef typename CT<C>::R R;
    const int i = tri_row(t);
    const C x = X[t];
    const C m = CT<C>::mk((t == tri(i) + i ? R(1) : R(0)) - x.x, -x.y);
    M[t] = m;
    return m.x * m.x + m.y * m.y;
}

// M_k = 1 - chi0_k on the lower triangle; piv[k] = max |M_k|.  A flat pass
// over the packed triangle (pairs of binary32 entries as one 16-byte access);
// the row of an entry, needed only to spot the diagonal, comes from a float
// square root corrected in integers.
template <typename C>
__global__ void __launch_bounds__(256) k_ldlt_init(const C* __restrict__ chi0, C* __restrict__ fac, int n,
                                                   double* __restrict__ piv) {
    typedef typename CT<C>::R R;
    __shared__ double red[33];
    const int k = blockIdx.x, tid = threadIdx.x;
    const long long pk = tri(n), base = k * pk;
    const C* X = chi0 + base;
    C* M = fac + base;
    R mx2 = R(0);     // max |M|^2 in the working precision (binary64 arithmetic is 1/64 rate)
    if (sizeof(C) == 8) {
        // binary32: entry pairs (t, t + 1) with base + t even are 16-byte aligned
        const long long t0 = base & 1;
        if (t0 && tid == 0 && pk > 0) mx2 = fmax(mx2, init_elem<C>(X, M, 0));
        const long long np = (pk - t0) / 2;
#pragma unroll 4
        for (long long q = tid; q < np; q += blockDim.x) {
            const long long t = t0 + 2 * q;
            const int i = tri_row(t);
            const long long d = tri(i) + i;       // t + 1 can only be diagonal of row i
            const float4 x = *reinterpret_cast<const float4*>(X + t);
            const float4 m = make_float4((t == d ? 1.f : 0.f) - x.x, -x.y, (t + 1 == d ? 1.f : 0.f) - x.z, -x.w);
            *reinterpret_cast<float4*>(M + t) = m;
            mx2 = fmax(mx2, R(fmaxf(m.x * m.x + m.y * m.y, m.z * m.z + m.w * m.w)));
        }
        if (((pk - t0) & 1) && tid == 0) mx2 = fmax(mx2, init_elem<C>(X, M, pk - 1));
    } else {
#pragma unroll 4
        for (long long t = tid; t < pk; t += blockDim.x) mx2 = fmax(mx2, init_elem<C>(X, M, t));
    }
    const double mx = block_max((double)mx2, red);
    if (threadIdx.x == 0) piv[k] = sqrt(mx);
}

// x D L11^T = a for one panel row held in registers: x_j = (a_j - sum_{p<j}
// x_p SD[j][p]) / d_j.
template <typename C, bool FULL>
__device__ __forceinline__ void panel_row_solve(C* __restrict__ row, const C (*SD)[Tile<C>::NB + 1],
                                                const C* Dinv, int kb) {
    constexpr int NB = Tile<C>::NB;
    C x[NB];
#pragma unroll
    for (int j = 0; j < NB; ++j)
        if (FULL || j < kb) x[j] = row[j];
#pragma unroll
    for (int j = 0; j < NB; ++j) {
        if (FULL || j < kb) {
            C a = x[j];
#pragma unroll
            for (int p = 0; p < j; ++p) a = cfms(x[p], SD[j][p], a);
            x[j] = cmul(a, Dinv[j]);
        }
        asm volatile("" ::: "memory");   // keep the SD loads of later rows from being hoisted (registers)
    }
#pragma unroll
    for (int j = 0; j < NB; ++j)
        if (FULL || j < kb) row[j] = x[j];
}

// Panel k0 of every frequency: factor the diagonal block, solve the rows
// below (x D L11^T = a), and store L11^-1 for the forward substitution of
// a6.  piv[N + k] carries min |d| between steps; the last panel writes
// piv[k] = min |d| / max |M| and flags a zero pivot.
template <typename C>
__global__ void __launch_bounds__(256, 2) k_ldlt_panel(C* __restrict__ fac, int n, int N, int k0,
                                                    C* __restrict__ linv, double* __restrict__ piv, int* status) {
    constexpr int NB = Tile<C>::NB, H = NB / 2, NPAIR = NB * (NB - 1) / 2, PPT = (NPAIR + 255) / 256;
    __shared__ C S[NB][NB + 1];     // L11 strictly below the diagonal, D on it
    __shared__ C SD[NB][NB + 1];    // SD[j][p] = L_jp d_p
    __shared__ C X[NB][NB + 1];     // L11^-1
    __shared__ C Dinv[NB];
    const int k = blockIdx.x, tid = threadIdx.x;
    C* A = fac + (long long)k * tri(n);
    const int kb = min(NB, n - k0), k1 = k0 + kb;
    for (int t = tid; t < NB * NB; t += blockDim.x) {
        const int i = t / NB, j = t % NB;
        // outside kb: identity, so the block inverse below needs no special case
        S[i][j] = (i < kb && j < kb) ? (j <= i ? A[tri(k0 + i) + k0 + j] : CT<C>::mk(0, 0))
                                     : CT<C>::mk(i == j ? 1 : 0, 0);
    }
    // pairs (i, l), 1 <= l <= i < NB, owned by this thread for the whole factorisation
    int pi[PPT], pl[PPT];
#pragma unroll
    for (int q = 0; q < PPT; ++q) {
        const int t = tid + 256 * q;
        int I = 0, J = 0;
        if (t < NPAIR) tri_ij(t, I, J);
        pi[q] = t < NPAIR ? I + 1 : -1;
        pl[q] = J + 1;
    }
    __syncthreads();
    // unblocked L D L^T of the diagonal block, one column per step: the pairs
    // with l > j take the update with the unscaled column j, then column j is
    // scaled by 1/d_j
    for (int j = 0; j < kb; ++j) {
        const C dinv = cdiv(CT<C>::mk(1, 0), S[j][j]);
#pragma unroll
        for (int q = 0; q < PPT; ++q) {
            const int i = pi[q], l = pl[q];
            if (i >= 0 && l > j && i < kb) S[i][l] = cfms(cmul(S[i][j], dinv), S[l][j], S[i][l]);
        }
        __syncthreads();
        if (tid > j && tid < kb) S[tid][j] = cmul(S[tid][j], dinv);
    }
    __syncthreads();
    for (int t = tid; t < kb * kb; t += blockDim.x) {
        const int i = t / kb, p = t % kb;
        if (p < i) SD[i][p] = cmul(S[i][p], S[p][p]);
        if (p <= i) A[tri(k0 + i) + k0 + p] = S[i][p];
    }
    if (tid < kb) Dinv[tid] = cdiv(CT<C>::mk(1, 0), S[tid][tid]);
    __syncthreads();
    if (tid < 32) {
        // warp 0: L11^-1 = [[A^-1, 0], [-C^-1 B A^-1, C^-1]] with H x H blocks
        // (the unit diagonal is implied: S holds D there, replaced by 1 here)
        const int lane = tid;
        if (lane < NB) {
            const int off = lane < H ? 0 : H, c = lane % H;
            C x[H];
#pragma unroll
            for (int i = 0; i < H; ++i) {
                C v = CT<C>::mk(i == c ? 1 : 0, 0);
#pragma unroll
                for (int p = 0; p < i; ++p)
                    if (p >= c) v = cfms(S[off + i][off + p], x[p], v);
                x[i] = v;
                asm volatile("" ::: "memory");
            }
#pragma unroll
            for (int i = 0; i < H; ++i) X[off + i][off + c] = x[i];
        }
        __syncwarp();
        // W = B A^-1 into the (zero) upper right block of X
        for (int t = lane; t < H * H; t += 32) {
            const int i = t / H, j = t % H;
            C w = CT<C>::mk(0, 0);
            for (int p = j; p < H; ++p) w = cfma(S[H + i][p], X[p][j], w);
            X[i][H + j] = w;
        }
        __syncwarp();
        for (int t = lane; t < H * H; t += 32) {
            const int i = t / H, j = t % H;
            C w = CT<C>::mk(0, 0);
            for (int p = 0; p <= i; ++p) w = cfma(X[H + i][H + p], X[p][H + j], w);
            X[H + i][j] = CT<C>::mk(-w.x, -w.y);
        }
        __syncwarp();
        C* Li = linv + ((long long)k * ((n + NB - 1) / NB) + k0 / NB) * NB * NB;
        for (int t = lane; t < NB * NB; t += 32) {
            const int i = t / NB, j = t % NB;
            Li[t] = (i < kb && j < kb && j <= i) ? X[i][j] : CT<C>::mk(0, 0);
        }
        if (lane == 0) {
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
    } else {
        const int nthr = blockDim.x - 32;
        for (int r = k1 + tid - 32; r < n; r += nthr) {
            if (kb == NB) panel_row_solve<C, true>(A + tri(r) + k0, SD, Dinv, kb);
            else panel_row_solve<C, false>(A + tri(r) + k0, SD, Dinv, kb);
        }
    }
}

// M -= sL sW^T on one tile of the lower triangle.  Thread (ty, tx) owns rows
// ty + 16a and columns tx + 16b; on a diagonal tile the sub-blocks b > a lie
// above the diagonal and are skipped at compile time.  The thread's entries
// of M are loaded into the accumulators before the panel tiles are staged, so
// that both global-load latencies overlap.
template <typename C, bool DIAG>
__device__ __forceinline__ void syrk_tile(C* __restrict__ A, int n, int k0, int kb, int r0, int c0,
                                          C (*sL)[Tile<C>::NB + 1], C (*sW)[Tile<C>::NB + 1], C* dd) {
    typedef typename CT<C>::R R;
    constexpr int NB = Tile<C>::NB, TT = Tile<C>::T, TA = Tile<C>::A;
    const int tid = threadIdx.x, ty = tid / 16, tx = tid % 16;
    C acc[TA][TA];
#pragma unroll
    for (int a = 0; a < TA; ++a)
#pragma unroll
        for (int b = 0; b < TA; ++b) {
            const int i = r0 + ty + 16 * a, j = c0 + tx + 16 * b;
            acc[a][b] = ((!DIAG || b <= a) && i < n && j <= i) ? A[tri(i) + j] : CT<C>::mk(R(0), R(0));
        }
    if (tid < NB) dd[tid] = tid < kb ? A[tri(k0 + tid) + k0 + tid] : CT<C>::mk(R(0), R(0));
    __syncthreads();
    for (int t = tid; t < TT * NB; t += blockDim.x) {
        const int rr = t / NB, p = t % NB;
        C lv = CT<C>::mk(R(0), R(0)), wv = CT<C>::mk(R(0), R(0));
        if (p < kb) {
            if (r0 + rr < n) lv = A[tri(r0 + rr) + k0 + p];
            if (c0 + rr < n) wv = cmul(A[tri(c0 + rr) + k0 + p], dd[p]);
        }
        sL[rr][p] = lv;
        sW[rr][p] = wv;
    }
    __syncthreads();
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
            for (int b = 0; b < TA; ++b)
                if (!DIAG || b <= a) acc[a][b] = cfms(l[a], w[b], acc[a][b]);
    }
#pragma unroll
    for (int a = 0; a < TA; ++a)
#pragma unroll
        for (int b = 0; b < TA; ++b) {
            if (DIAG && b > a) continue;
            const int i = r0 + ty + 16 * a, j = c0 + tx + 16 * b;
            if (i < n && j <= i) A[tri(i) + j] = acc[a][b];
        }
}

// Trailing update after panel k0: M22 -= L21 D L21^T on the lower triangle,
// tile blockIdx.x of frequency blockIdx.y.
template <typename C>
__global__ void __launch_bounds__(256) k_ldlt_syrk(C* __restrict__ fac, int n, int k0) {
    constexpr int NB = Tile<C>::NB, TT = Tile<C>::T;
    __shared__ C sL[TT][NB + 1];
    __shared__ C sW[TT][NB + 1];
    __shared__ C dd[NB];
    C* A = fac + (long long)blockIdx.y * tri(n);
    const int kb = min(NB, n - k0), k1 = k0 + kb;
    int I, J;
    tri_ij(blockIdx.x, I, J);
    const int r0 = k1 + I * TT, c0 = k1 + J * TT;
    if (I == J) syrk_tile<C, true>(A, n, k0, kb, r0, c0, sL, sW, dd);
    else syrk_tile<C, false>(A, n, k0, kb, r0, c0, sL, sW, dd);
}

// Trailing update of the binary32 factorisation on the tensor cores: the tile
// (128 rows) x (32 complex columns) of M22 -= L21 D L21^T is one real TF32
// product with the complex entries interleaved along K (3xTF32, hi products
// and cross terms in two tensor-memory accumulators):
//   A[r][2p] = Re L[r][p], A[r][2p+1] = Im L[r][p]             (rows r of the tile)
//   B[q][2p] = Re w, B[q][2p+1] = -Im w;  B[32+q][2p] = Im w, B[32+q][2p+1] = Re w
// with w = L[c_q][p] d_p for the tile's columns c_q, so that accumulator
// columns q and 32 + q hold Re and Im of (L21 D L21^T)[r][c_q].  One CTA per
// frequency and 128-row block I of the trailing matrix stages the block's
// panel rows (A) once and walks its min(ceil(m / 32), 4 I + 4) column tiles
// with two accumulator sets and two B buffers: the MMAs of tile J run while
// tile J - 1 is read back, subtracted and stored.  The read-back goes through
// a per-warp shared-memory transpose so that the read-modify-write of M is
// row-contiguous; entries above the diagonal are skipped.
constexpr int ST_NC = 32, ST_N = 2 * ST_NC, ST_XP = 17;
constexpr int ST_A_BYTES = 128 * 64 * 4;            // 128 x 64 binary32 (hi or lo)
constexpr int ST_B_BYTES = ST_N * 64 * 4;           // 64 x 64 binary32 (hi or lo)
constexpr uint32_t ST_SBO = (64 / 4) * 128;
constexpr uint32_t ST_IDESC = tc::idesc_tf32(128, ST_N);
constexpr uint32_t ST_IDESC2 = tc::idesc_tf32(128, 2 * ST_N);     // A_hi x [B_hi; B_lo]
constexpr size_t ST_SMEM = 2 * (size_t)ST_A_BYTES + 4 * (size_t)ST_B_BYTES + 8 * 32 * ST_XP * sizeof(float2);
// per-block dynamic shared memory ceiling (227 KB), 1 KB kept for the static arrays
constexpr size_t SMEM_DYN_MAX = 227 * 1024 - 1024, SMEM_PER_SM = 228 * 1024;
static_assert(ST_SMEM <= SMEM_DYN_MAX, "trailing update: shared memory");

__host__ __device__ inline int st_row_tiles(int nj, int I) { return nj < 4 * I + 4 ? nj : 4 * I + 4; }

__device__ __forceinline__ void st_shared_quad(unsigned char* hi, unsigned char* lo, uint32_t o, float a, float b,
                                               float c, float d) {
    uint32_t h0, l0, h1, l1, h2, l2, h3, l3;
    tc::split_tf32(a, h0, l0);
    tc::split_tf32(b, h1, l1);
    tc::split_tf32(c, h2, l2);
    tc::split_tf32(d, h3, l3);
    asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(tc::smem_u32(hi + o)), "r"(h0), "r"(h1), "r"(h2),
                 "r"(h3) : "memory");
    asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(tc::smem_u32(lo + o)), "r"(l0), "r"(l1), "r"(l2),
                 "r"(l3) : "memory");
}

// raw panel entries of the B operand of column tile c0: two K-quads per thread
__device__ __forceinline__ void st_load_b(float2 (&wr)[2][2], const float2* __restrict__ A, int n, int k0, int c0) {
#pragma unroll
    for (int j = 0; j < 2; ++j) {
        const int idx = threadIdx.x + 256 * j, kq = (idx >> 3) & 15, q = 8 * (idx >> 7) + (idx & 7), cc = c0 + q;
        wr[j][0] = wr[j][1] = make_float2(0.f, 0.f);
        if (cc < n) {
            const float2* src = A + tri(cc) + k0 + 2 * kq;
            wr[j][0] = src[0];
            wr[j][1] = src[1];
        }
    }
}

// this lane's entries of M in the row-contiguous read-back layout: rows
// rb + (lane >> 2) + 8 i, complex columns cb + 4 (lane & 3) + t
__device__ __forceinline__ void st_load_c(float2 (&cv)[4][4], const float2* __restrict__ A, int n, int rb, int cb) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int r = rb + (lane >> 2) + 8 * i;
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const int cc = cb + 4 * (lane & 3) + t;
            cv[i][t] = (r < n && cc <= r) ? A[tri(r) + cc] : make_float2(0.f, 0.f);
        }
    }
}

__global__ void __launch_bounds__(256, 1) k_ldlt_syrk_tc(float2* __restrict__ fac, int n, int k0, int nj_max,
                                                         int* status) {
    extern __shared__ __align__(128) unsigned char sraw_st[];
    unsigned char* sAh = sraw_st;
    unsigned char* sAl = sAh + ST_A_BYTES;
    unsigned char* sB = sAl + ST_A_BYTES;                            // [2][hi, lo][ST_B_BYTES]
    float2* sX = reinterpret_cast<float2*>(sB + 4 * ST_B_BYTES);     // [8 warps][32][ST_XP]
    __shared__ float2 dd[32];
    __shared__ __align__(8) uint64_t mbar[2];
    __shared__ uint32_t tbase;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    float2* A = fac + (long long)blockIdx.y * tri(n);
    const int k1 = k0 + 32, m = n - k1, nj = (m + ST_NC - 1) / ST_NC, I = blockIdx.x;
    const int r0 = k1 + 128 * I, ntile = min(st_row_tiles(nj, I), nj_max);
    // this warp's read-back block: rows rw .. rw + 31, complex columns 16 h .. + 15 of a tile
    const int rw = r0 + 32 * (warp & 3), h = warp >> 2;
    if (warp == 0) tc::tmem_alloc(&tbase, 4 * ST_N);
    if (tid == 0) {
        tc::mbar_init(&mbar[0]);
        tc::mbar_init(&mbar[1]);
    }
    if (tid < 32) dd[tid] = A[tri(k0 + tid) + k0 + tid];
    // entries of M: tile t lands in register set t % 3, two tiles ahead of its
    // read-back (sets used in turn, no copies between them that would wait
    // for the loads in flight)
    float2 wr[2][2], cs0[4][4], cs1[4][4], cs2[4][4];
    st_load_b(wr, A, n, k0, k1);
    st_load_c(cs0, A, n, rw, k1 + 16 * h);
    if (ntile > 1) st_load_c(cs1, A, n, rw, k1 + ST_NC + 16 * h);
    // A operand: rows r0 .. r0 + 127 of the panel, staged once
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const int idx = tid + 256 * j, rr = idx & 7, kq = (idx >> 3) & 15, rg = idx >> 7;
        const int ra = r0 + 8 * rg + rr;
        float2 a = make_float2(0.f, 0.f), b = a;
        if (ra < n) {
            const float2* src = A + tri(ra) + k0 + 2 * kq;
            a = src[0];
            b = src[1];
        }
        st_shared_quad(sAh, sAl, tc::core_off(8 * rg + rr, 4 * kq, 16), a.x, a.y, b.x, b.y);
    }
    __syncthreads();
    tc::fence_after();
    const uint32_t taddr = tbase;
    bool ok = true;
    float2* X = sX + warp * 32 * ST_XP;
    int J = 0;
    // step J: stage and multiply tile J, read back tile J - 1 from register
    // set `cp`, load tile J + 1 into set `cnx`; false once a wait timed out
    auto step = [&](float2 (&cp)[4][4], float2 (&cnx)[4][4]) -> bool {
        if (J < ntile) {
            // B operand of tile J (its buffer was last read by the MMAs of tile J - 2, complete)
            unsigned char* bh = sB + 2 * (J & 1) * ST_B_BYTES;
            unsigned char* bl = bh + ST_B_BYTES;
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                const int idx = tid + 256 * j, rr = idx & 7, kq = (idx >> 3) & 15, rg = idx >> 7, q = 8 * rg + rr;
                const float2 w0 = cmul(wr[j][0], dd[2 * kq]), w1 = cmul(wr[j][1], dd[2 * kq + 1]);
                st_shared_quad(bh, bl, tc::core_off(q, 4 * kq, 16), w0.x, -w0.y, w1.x, -w1.y);
                st_shared_quad(bh, bl, tc::core_off(ST_NC + q, 4 * kq, 16), w0.y, w0.x, w1.y, w1.x);
            }
            if (J + 1 < ntile) st_load_b(wr, A, n, k0, k1 + ST_NC * (J + 1));
            tc::fence_async_smem();
            __syncthreads();
            if (tid == 0) {
                tc::fence_after();
                const uint32_t ah = tc::smem_u32(sAh), al = tc::smem_u32(sAl);
                const uint32_t b0 = tc::smem_u32(bh);
                const uint32_t d = taddr + (uint32_t)(2 * ST_N * (J & 1));
#pragma unroll
                // B lo follows B hi (rows ST_N .. 2 ST_N - 1 of one operand), the cross-term
                // accumulator follows the hi x hi one: A_hi x [B_hi; B_lo] is one N = 2 ST_N product
                for (int ks = 0; ks < 8; ++ks) {
                    const uint32_t o = ks * 256, acc = ks > 0 ? 1u : 0u;
                    tc::mma_tf32(d, tc::smem_desc(ah + o, ST_SBO), tc::smem_desc(b0 + o, ST_SBO), ST_IDESC2, acc);
                    tc::mma_tf32(d + ST_N, tc::smem_desc(al + o, ST_SBO), tc::smem_desc(b0 + o, ST_SBO), ST_IDESC, 1u);
                }
                tc::commit(tc::smem_u32(&mbar[J & 1]));
            }
        }
        if (J >= 1) {
            // tile J - 1: read back, transpose through shared memory, M -= product
            const int Jp = J - 1, cb = k1 + ST_NC * Jp + 16 * h;
            if (J + 1 < ntile) st_load_c(cnx, A, n, rw, k1 + ST_NC * (J + 1) + 16 * h);
            ok = tc::mbar_wait(tc::smem_u32(&mbar[Jp & 1]), (Jp >> 1) & 1) && ok;
            ok = __syncthreads_and(ok);
            if (!ok) return false;
            tc::fence_after();
            const uint32_t base = taddr + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(2 * ST_N * (Jp & 1) + 16 * h);
            uint32_t re[16], im[16], re2[16], im2[16];
            tc::tmem_ld16(base, re);
            tc::tmem_ld16(base + ST_NC, im);
            tc::tmem_ld16(base + ST_N, re2);
            tc::tmem_ld16(base + ST_N + ST_NC, im2);
            tc::tmem_wait_ld();
            tc::fence_before();
#pragma unroll
            for (int j = 0; j < 16; ++j)
                X[lane * ST_XP + j] = make_float2(__uint_as_float(re[j]) + __uint_as_float(re2[j]),
                                                  __uint_as_float(im[j]) + __uint_as_float(im2[j]));
            __syncwarp();
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int rl = (lane >> 2) + 8 * i, r = rw + rl;
                if (r < n) {
                    float2* row = A + tri(r);
#pragma unroll
                    for (int t = 0; t < 4; ++t) {
                        const int cl = 4 * (lane & 3) + t, cc = cb + cl;
                        if (cc <= r) {
                            const float2 x = X[rl * ST_XP + cl];
                            row[cc] = make_float2(cp[i][t].x - x.x, cp[i][t].y - x.y);
                        }
                    }
                }
            }
            __syncwarp();
        }
        return true;
    };
    // tile J - 1 sits in set (J - 1) % 3, tile J + 1 goes to set (J + 1) % 3
    while (J <= ntile) {
        if (!step(cs2, cs1) || ++J > ntile) break;
        if (!step(cs0, cs2) || ++J > ntile) break;
        if (!step(cs1, cs0)) break;
        ++J;
    }
    if (!ok) {
        // the loop ended early at tile J: the MMAs issued so far finish before the columns are freed
        if (tid == 0) atomicOr(status, ST_TIMEOUT);
        const int issued = min(J + 1, ntile);
        for (int s2 = 0; s2 < 2; ++s2) {
            const int cnt = (issued - s2 + 1) / 2;
            if (cnt > 0) tc::mbar_wait(tc::smem_u32(&mbar[s2]), (cnt - 1) & 1);
        }
    }
    tc::fence_before();
    __syncthreads();
    if (warp == 0) {
        tc::fence_after();
        tc::tmem_dealloc(taddr, 4 * ST_N);
    }
}

// The trailing update of two consecutive panels in one pass (binary32): with
// panel p0 = [g0, g0 + 32) factored, its update restricted to the columns of
// panel p1 = [g0 + 32, g0 + 64) (k_ldlt_syrk_tc with one column tile) and
// p1 factored, the rest of the trailing matrix takes
//   M[r][c] <- (M[r][c] - u0[r][c]) - u1[r][c],  g0 + 64 <= c <= r,
// u_j the 3xTF32 product of panel j, each in its own tensor-memory
// accumulators and subtracted in that order: the same operations, in the same
// order, as two k_ldlt_syrk_tc launches, with the packed triangle read and
// written once instead of twice.  One CTA per frequency and 128-row block:
// both panels' rows staged once (128 KB), one B buffer holding both panels'
// w for a column tile of 32 (64 KB), two accumulator sets of 256 columns, and
// the per-warp read-back turn-around of k_ldlt_syrk_tc.
constexpr size_t ST2_SMEM = 4 * (size_t)ST_A_BYTES + 4 * (size_t)ST_B_BYTES + 8 * 32 * ST_XP * sizeof(float2);
static_assert(ST2_SMEM <= SMEM_DYN_MAX, "paired trailing update: shared memory");
// all 512 tensor-memory columns: a second CTA of the kernel never fits beside the first
static_assert(8 * ST_N == 512 && 2 * ST2_SMEM > SMEM_PER_SM, "paired trailing update: one CTA per SM");

__global__ void __launch_bounds__(256, 1) k_ldlt_syrk_tc2(float2* __restrict__ fac, int n, int g0, int* status) {
    extern __shared__ __align__(128) unsigned char sraw_s2[];
    unsigned char* sA = sraw_s2;                                       // [panel][hi, lo][ST_A_BYTES]
    unsigned char* sB = sA + 4 * ST_A_BYTES;                           // [panel][hi, lo][ST_B_BYTES]
    float2* sX = reinterpret_cast<float2*>(sB + 4 * ST_B_BYTES);       // [8 warps][32][ST_XP]
    __shared__ float2 dd[64];
    __shared__ __align__(8) uint64_t mbar[2];
    __shared__ uint32_t tbase;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    float2* A = fac + (long long)blockIdx.y * tri(n);
    const int k2 = g0 + 64, m = n - k2, nj = (m + ST_NC - 1) / ST_NC, I = blockIdx.x;
    const int r0 = k2 + 128 * I, ntile = st_row_tiles(nj, I);
    const int rw = r0 + 32 * (warp & 3), h = warp >> 2;
    if (warp == 0) tc::tmem_alloc(&tbase, 8 * ST_N);
    if (tid == 0) {
        tc::mbar_init(&mbar[0]);
        tc::mbar_init(&mbar[1]);
    }
    if (tid < 64) dd[tid] = A[tri(g0 + tid) + g0 + tid];
    float2 wr0[2][2], wr1[2][2], cs0[4][4], cs1[4][4], cs2[4][4];
    st_load_b(wr0, A, n, g0, k2);
    st_load_b(wr1, A, n, g0 + 32, k2);
    st_load_c(cs0, A, n, rw, k2 + 16 * h);
    if (ntile > 1) st_load_c(cs1, A, n, rw, k2 + ST_NC + 16 * h);
    // A operands: rows r0 .. r0 + 127 of both panels, staged once
#pragma unroll 4
    for (int j = 0; j < 16; ++j) {
        const int pj = j >> 3, idx = tid + 256 * (j & 7), rr = idx & 7, kq = (idx >> 3) & 15, rg = idx >> 7;
        const int ra = r0 + 8 * rg + rr;
        float2 a = make_float2(0.f, 0.f), b = a;
        if (ra < n) {
            const float2* src = A + tri(ra) + g0 + 32 * pj + 2 * kq;
            a = src[0];
            b = src[1];
        }
        unsigned char* ah = sA + 2 * pj * ST_A_BYTES;
        st_shared_quad(ah, ah + ST_A_BYTES, tc::core_off(8 * rg + rr, 4 * kq, 16), a.x, a.y, b.x, b.y);
    }
    __syncthreads();
    tc::fence_after();
    const uint32_t taddr = tbase;
    bool ok = true;
    float2* X = sX + warp * 32 * ST_XP;
    int J = 0;
    auto stage_b = [&](const float2 (&wr)[2][2], int pj) {
        unsigned char* bh = sB + 2 * pj * ST_B_BYTES;
        unsigned char* bl = bh + ST_B_BYTES;
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const int idx = tid + 256 * j, rr = idx & 7, kq = (idx >> 3) & 15, rg = idx >> 7, q = 8 * rg + rr;
            const float2 w0 = cmul(wr[j][0], dd[32 * pj + 2 * kq]), w1 = cmul(wr[j][1], dd[32 * pj + 2 * kq + 1]);
            st_shared_quad(bh, bl, tc::core_off(q, 4 * kq, 16), w0.x, -w0.y, w1.x, -w1.y);
            st_shared_quad(bh, bl, tc::core_off(ST_NC + q, 4 * kq, 16), w0.y, w0.x, w1.y, w1.x);
        }
    };
    // this warp's 16 columns of one panel's product: per 8 columns, hi x hi + cross terms
    auto to_x = [&](uint32_t base) {
#pragma unroll
        for (int hh = 0; hh < 2; ++hh) {
            uint32_t re[8], im[8], re2[8], im2[8];
            tc::tmem_ld8(base + 8 * hh, re);
            tc::tmem_ld8(base + ST_NC + 8 * hh, im);
            tc::tmem_ld8(base + ST_N + 8 * hh, re2);
            tc::tmem_ld8(base + ST_N + ST_NC + 8 * hh, im2);
            tc::tmem_wait_ld();
#pragma unroll
            for (int j = 0; j < 8; ++j)
                X[lane * ST_XP + 8 * hh + j] = make_float2(__uint_as_float(re[j]) + __uint_as_float(re2[j]),
                                                           __uint_as_float(im[j]) + __uint_as_float(im2[j]));
        }
    };
    // step J: wait for tile J - 1's MMAs (the B buffer is free, its accumulators ready), stage
    // and multiply tile J, read back tile J - 1 from register set `cp`, load tile J + 1 into `cnx`
    auto step = [&](float2 (&cp)[4][4], float2 (&cnx)[4][4]) -> bool {
        if (J >= 1) {
            if (J + 1 < ntile) st_load_c(cnx, A, n, rw, k2 + ST_NC * (J + 1) + 16 * h);
            ok = tc::mbar_wait(tc::smem_u32(&mbar[(J - 1) & 1]), ((J - 1) >> 1) & 1) && ok;
            ok = __syncthreads_and(ok);
            if (!ok) return false;
        }
        if (J < ntile) {
            stage_b(wr0, 0);
            stage_b(wr1, 1);
            if (J + 1 < ntile) {
                st_load_b(wr0, A, n, g0, k2 + ST_NC * (J + 1));
                st_load_b(wr1, A, n, g0 + 32, k2 + ST_NC * (J + 1));
            }
            tc::fence_async_smem();
            __syncthreads();
            if (tid == 0) {
                tc::fence_after();
#pragma unroll
                for (int pj = 0; pj < 2; ++pj) {
                    const uint32_t ah = tc::smem_u32(sA + 2 * pj * ST_A_BYTES), al = ah + ST_A_BYTES;
                    const uint32_t b0 = tc::smem_u32(sB + 2 * pj * ST_B_BYTES);
                    const uint32_t d = taddr + (uint32_t)(4 * ST_N * (J & 1) + 2 * ST_N * pj);
#pragma unroll
                    for (int ks = 0; ks < 8; ++ks) {
                        const uint32_t o = ks * 256, acc = ks > 0 ? 1u : 0u;
                        tc::mma_tf32(d, tc::smem_desc(ah + o, ST_SBO), tc::smem_desc(b0 + o, ST_SBO), ST_IDESC2, acc);
                        tc::mma_tf32(d + ST_N, tc::smem_desc(al + o, ST_SBO), tc::smem_desc(b0 + o, ST_SBO), ST_IDESC,
                                     1u);
                    }
                }
                tc::commit(tc::smem_u32(&mbar[J & 1]));
            }
        }
        if (J >= 1) {
            // tile J - 1: M - u0, then - u1, through the turn-around
            const int Jp = J - 1, cb = k2 + ST_NC * Jp + 16 * h;
            tc::fence_after();
            const uint32_t base = taddr + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(4 * ST_N * (Jp & 1) + 16 * h);
            to_x(base);
            __syncwarp();
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int rl = (lane >> 2) + 8 * i;
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    const float2 x = X[rl * ST_XP + 4 * (lane & 3) + t];
                    cp[i][t] = make_float2(cp[i][t].x - x.x, cp[i][t].y - x.y);
                }
            }
            __syncwarp();
            to_x(base + 2 * ST_N);
            tc::fence_before();
            __syncwarp();
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int rl = (lane >> 2) + 8 * i, r = rw + rl;
                if (r < n) {
                    float2* row = A + tri(r);
#pragma unroll
                    for (int t = 0; t < 4; ++t) {
                        const int cl = 4 * (lane & 3) + t, cc = cb + cl;
                        if (cc <= r) {
                            const float2 x = X[rl * ST_XP + cl];
                            row[cc] = make_float2(cp[i][t].x - x.x, cp[i][t].y - x.y);
                        }
                    }
                }
            }
            __syncwarp();
        }
        return true;
    };
    while (J <= ntile) {
        if (!step(cs2, cs1) || ++J > ntile) break;
        if (!step(cs0, cs2) || ++J > ntile) break;
        if (!step(cs1, cs0)) break;
        ++J;
    }
    if (!ok) {
        // the loop ended at tile J: tiles 0 .. J - 1 were issued; their MMAs finish before the columns are freed
        if (tid == 0) atomicOr(status, ST_TIMEOUT);
        const int issued = min(J, ntile);
        for (int s2 = 0; s2 < 2; ++s2) {
            const int cnt = (issued - s2 + 1) / 2;
            if (cnt > 0) tc::mbar_wait(tc::smem_u32(&mbar[s2]), (cnt - 1) & 1);
        }
    }
    tc::fence_before();
    __syncthreads();
    if (warp == 0) {
        tc::fence_after();
        tc::tmem_dealloc(taddr, 8 * ST_N);
    }
}

__device__ __forceinline__ void cp_async8(void* dst, const void* src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
}
template <typename C> __device__ __forceinline__ void cp_async_c(C* dst, const C* src) {
    if (sizeof(C) == 8) cp_async8(dst, src);
    else cp_async16(dst, src);
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int K> __device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(K) : "memory");
}

// rows [r0, r0 + FT) x columns [k0, k0 + NB) of F into a pitched tile (zero
// outside the matrix or the panel); no commit
template <typename C, int FT = Tile<C>::FT>
__device__ __forceinline__ void load_l_tile(C* dst, const C* __restrict__ F, int n, int r0, int k0, int kb) {
    constexpr int NB = Tile<C>::NB, LP = tile_pitch<C>();
    for (int t = threadIdx.x; t < FT * NB; t += blockDim.x) {
        const int rr = t / NB, p = t % NB;
        C* d = dst + rr * LP + p;
        if (p < kb && r0 + rr < n) cp_async_c(d, F + tri(r0 + rr) + k0 + p);
        else *d = CT<C>::mk(0, 0);
    }
}

// L11^-1 of panel k0 into rows of pitch LIP (a multiple of 16 bytes) and its
// pivots d_i (binary32 only); no commit
template <int LIP>
__device__ __forceinline__ void load_diag_pitched(float2* sLi, float2* sD, const float2* __restrict__ Li,
                                                  const float2* __restrict__ F, int n, int k0, int kb) {
    for (int t = threadIdx.x; t < 32 * 16; t += blockDim.x) {
        const int r = t >> 4, q = t & 15;
        cp_async16(sLi + r * LIP + 2 * q, Li + r * 32 + 2 * q);
    }
    for (int i = threadIdx.x; i < 32; i += blockDim.x) {
        if (i < kb) cp_async8(sD + i, F + tri(k0 + i) + k0 + i);
        else sD[i] = make_float2(0.f, 0.f);
    }
}

// L11^-1 of panel k0 (NB x NB, zero outside kb) and its pivots d_i; no commit
template <typename C>
__device__ __forceinline__ void load_diag_data(C* sLi, C* sD, const C* __restrict__ Li, const C* __restrict__ F,
                                               int n, int k0, int kb) {
    constexpr int NB = Tile<C>::NB, V = 16 / sizeof(C);
    for (int t = threadIdx.x; t < NB * NB / V; t += blockDim.x) cp_async16(sLi + t * V, Li + t * V);
    for (int i = threadIdx.x; i < NB; i += blockDim.x) {
        if (i < kb) cp_async_c(sD + i, F + tri(k0 + i) + k0 + i);
        else sD[i] = CT<C>::mk(0, 0);
    }
}

__device__ __forceinline__ void load_pair(const float2* p, float2& a, float2& b) {
    const float4 v = *reinterpret_cast<const float4*>(p);
    a = make_float2(v.x, v.y);
    b = make_float2(v.z, v.w);
}
__device__ __forceinline__ void load_pair(const double2* p, double2& a, double2& b) {
    a = p[0];
    b = p[1];
}

// c[r*N + k] = -(1/pi) Im sum_i y_i^2/d_i, y = L_k^-1 q_r: right-hand sides
// [chunk*RC, chunk*RC + RC) of frequency k = 1 + blockIdx.y, chunk = blockIdx.x.
// Thread (g, c), g < FG, c < RC (blockDim = FG*RC) owns column c: per panel
// it keeps y_b[:, c] (NB values) in registers and walks the rows g, g + FG,
// ... with the L rows read from shared memory (the same row for all threads
// of a group).  Shared memory: two L tiles [FT][LP], two L11^-1 [NB][NB]
// and pivots [NB] (next panel prefetched), Y [n][RC].
constexpr int FG = 4;          // row groups per CTA (default variant)
constexpr int FR = 4;          // rows per thread in flight

template <typename C>
__device__ __forceinline__ void load_yb(C (&y)[Tile<C>::NB], const C* __restrict__ sY, int RC, int k0, int kb, int c) {
    constexpr int NB = Tile<C>::NB;
#pragma unroll
    for (int p = 0; p < NB; ++p) y[p] = p < kb ? sY[(long long)(k0 + p) * RC + c] : CT<C>::mk(0, 0);
}

// acc[q] = sum_p A[rows[q]*lda + p] y[p] for FR rows (p over the full panel;
// A is zero beyond kb)
template <typename C>
__device__ __forceinline__ void rows_dot(C (&acc)[FR], const C* __restrict__ A, int lda, const int (&rows)[FR],
                                         const C (&y)[Tile<C>::NB]) {
    typedef typename CT<C>::R T;
    constexpr int NB = Tile<C>::NB;
#pragma unroll
    for (int q = 0; q < FR; ++q) acc[q] = CT<C>::mk(T(0), T(0));
#pragma unroll
    for (int p = 0; p < NB; p += 2) {
        C l0[FR], l1[FR];
#pragma unroll
        for (int q = 0; q < FR; ++q) load_pair(A + rows[q] * lda + p, l0[q], l1[q]);
#pragma unroll
        for (int q = 0; q < FR; ++q) acc[q] = cfma(l1[q], y[p + 1], cfma(l0[q], y[p], acc[q]));
    }
}

// G row groups and FT-row L tiles; the launch uses <C, FG, Tile<C>::FT>: up to
// 80 right-hand sides per CTA, one CTA per SM.  (Halving the chunk to fit two
// CTAs per SM with eight row groups measured slower on the ring, 3.75 vs
// 3.34 ms: the doubled L re-reads cost more than the extra warps recover.)
template <typename C, int G, int FT>
__global__ void __launch_bounds__(320, 1)
    k_forms(const C* __restrict__ fac, const C* __restrict__ linv, int n, int N, const double* __restrict__ Q, int R,
            int RC, double* __restrict__ c, const int* __restrict__ kmap) {
    typedef typename CT<C>::R T;
    constexpr int NB = Tile<C>::NB, LP = tile_pitch<C>(), FG = G;
    extern __shared__ __align__(16) unsigned char sraw[];
    C* sL = reinterpret_cast<C*>(sraw);                 // [2][FT][LP]
    C* sLi = sL + 2 * FT * LP;                          // [2][NB][NB]
    C* sD = sLi + 2 * NB * NB;                          // [2][NB]
    C* sY = sD + 2 * NB;                                // [n][RC]
    const int tid = threadIdx.x, col = tid % RC, g = tid / RC;
    // factors of frequency k = 1 + blockIdx.y, or (kmap given) of the compact set's entry
    // blockIdx.y, whose frequency is kmap[blockIdx.y]
    const int kd = kmap ? (int)blockIdx.y : 1 + (int)blockIdx.y;
    const int k = kmap ? kmap[blockIdx.y] : kd, rc0 = blockIdx.x * RC, rc = min(RC, R - rc0);
    const C* F = fac + (long long)kd * tri(n);
    const int nblk = (n + NB - 1) / NB;
    const C* Lk = linv + (long long)kd * nblk * NB * NB;
    load_diag_data<C>(sLi, sD, Lk, F, n, 0, min(NB, n));
    if (n > NB) load_l_tile<C, FT>(sL, F, n, NB, 0, NB);
    cp_async_commit();
    {
        // thread (g, col) fills rows g, g + FG, ... of its column (no integer division)
        const double* q = Q + rc0 + col;
        const bool live = col < rc;
#pragma unroll 8
        for (int i = g; i < n; i += FG) sY[i * RC + col] = CT<C>::mk(live ? T(q[(long long)i * R]) : T(0), T(0));
    }
    double2 part = make_double2(0.0, 0.0);
    C y[NB];
    int buf = 0;
    for (int blk = 0; blk < nblk; ++blk) {
        const int k0 = blk * NB, kb = min(NB, n - k0), k1 = k0 + kb, db = blk & 1;
        const int ntile = (n - k1 + FT - 1) / FT;
        cp_async_wait<0>();
        __syncthreads();
        if (blk + 1 < nblk)
            load_diag_data<C>(sLi + (db ^ 1) * NB * NB, sD + (db ^ 1) * NB, Lk + (long long)(blk + 1) * NB * NB, F, n,
                              k1, min(NB, n - k1));
        cp_async_commit();
        // y_b = L11^-1 y_b: this thread's rows g, g + FG, ... of the block
        load_yb<C>(y, sY, RC, k0, kb, col);
        __syncthreads();
        {
            const C* Li = sLi + db * NB * NB;
            for (int i0 = g; i0 < kb; i0 += FG * FR) {
                int rows[FR];
#pragma unroll
                for (int q = 0; q < FR; ++q) rows[q] = min(i0 + FG * q, NB - 1);
                C acc[FR];
                rows_dot<C>(acc, Li, NB, rows, y);
#pragma unroll
                for (int q = 0; q < FR; ++q) {
                    const int i = i0 + FG * q;
                    if (i < kb) {
                        sY[(long long)(k0 + i) * RC + col] = acc[q];
                        const C v = cdiv(cmul(acc[q], acc[q]), sD[db * NB + i]);
                        part.x += (double)v.x;
                        part.y += (double)v.y;
                    }
                }
            }
        }
        __syncthreads();
        load_yb<C>(y, sY, RC, k0, kb, col);
        // Y[k1:n] -= L[k1:n, k0:k1] y_b, FT rows per tile; the next tile (of
        // this panel or the first of the next) streams in meanwhile
        for (int t = 0; t < ntile; ++t) {
            const int r0 = k1 + t * FT;
            int nr0 = n, nk0 = k0, nkb = kb;
            if (t + 1 < ntile) nr0 = r0 + FT;
            else if (blk + 1 < nblk) {
                nk0 = k1;
                nkb = min(NB, n - k1);
                nr0 = nk0 + nkb;
            }
            if (nr0 < n) load_l_tile<C, FT>(sL + (buf ^ 1) * FT * LP, F, n, nr0, nk0, nkb);
            cp_async_commit();
            cp_async_wait<1>();
            __syncthreads();
            const C* Lt = sL + buf * FT * LP;
            const int nrow = min(FT, n - r0);
            for (int i0 = g; i0 < nrow; i0 += FG * FR) {
                int rows[FR];
#pragma unroll
                for (int q = 0; q < FR; ++q) rows[q] = min(i0 + FG * q, FT - 1);
                C acc[FR];
                rows_dot<C>(acc, Lt, LP, rows, y);
#pragma unroll
                for (int q = 0; q < FR; ++q) {
                    const int i = i0 + FG * q;
                    if (i < nrow) {
                        C* yy = sY + (long long)(r0 + i) * RC + col;
                        *yy = csub(*yy, acc[q]);
                    }
                }
            }
            __syncthreads();      // the buffer just read is refilled next
            buf ^= 1;
        }
    }
    cp_async_wait<0>();
    // sum the FG row groups of each column (reusing the start of sY)
    double* red = reinterpret_cast<double*>(sY);
    __syncthreads();
    red[g * RC + col] = part.y;
    __syncthreads();
    if (tid < rc) {
        double im = 0.0;
        for (int q = 0; q < FG; ++q) im += red[q * RC + tid];
        c[(long long)(rc0 + tid) * N + k] = -im / M_PI;
        if (!kmap && k == 1) c[(long long)(rc0 + tid) * N] = 0.0;
    }
}

__device__ __forceinline__ void st_shared_v4(unsigned char* p, uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
    asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(tc::smem_u32(p)), "r"(a), "r"(b), "r"(c), "r"(d)
                 : "memory");
}

// Forms of the binary32 path with the updates of Y kept in tensor memory.
// One CTA per frequency k = 1 + blockIdx.y and chunk of TM_RC right-hand
// sides, two CTAs per SM.  The update of every row below panel b,
//   dY[r] -= L[r, panel b] y_b,
// is one real TF32 product per 128-row tile and quarter panel (3xTF32 into
// one binary32 accumulator per tile), with the complex entries interleaved
// along K so that a raw row segment of L is the A operand as it lies in
// memory:
//   A[r][2p] = Re L[r][p],  A[r][2p+1] = Im L[r][p]
//   B[c][2p] = -Re y_p[c], B[c][2p+1] = Im y_p[c]      (output Re Y[., c])
//   B[TM_RC+c][2p] = -Im y_p[c], B[TM_RC+c][2p+1] = -Re y_p[c]   (output Im)
// The accumulators of all tiles (rows 0 .. n-1 as tensor-memory lanes) hold
// dY for the whole forward substitution and are never written back: panel b
// reads its own 32 rows once (two warps, tcgen05.ld), adds q, applies the
// stored L11^-1 and the forms sum, and builds its B operand; its MMAs then
// run while the next panel is prepared (and while the other CTA of the SM
// runs its own serial steps).  The MMAs of the tile that holds the next
// panel's rows are committed to their own mbarrier, so the next panel waits
// for that tile only; the B operand is rebuilt once the whole panel's MMAs
// are done.  L rows stream through TM_NS operand stages (register prefetch
// two stages ahead); every mbarrier wait is bounded.
constexpr int TM_RC = 40, TM_N = 2 * TM_RC, TM_KS = 16, TM_NS = 3, TM_MAXT = 3, TM_RCP = TM_RC + 1;
constexpr int TM_A_BYTES = 128 * TM_KS * 4;         // one 128 x 16 binary32 operand (hi or lo)
constexpr int TM_B_BYTES = TM_N * 64 * 4;           // one 80 x 64 binary32 operand (hi or lo)
constexpr uint32_t TM_SBO_A = (TM_KS / 4) * 128, TM_SBO_B = (64 / 4) * 128;
constexpr uint32_t TM_IDESC = tc::idesc_tf32(128, TM_N);
constexpr int TM_GROUPS = 6;                        // row groups of the y_b step (6 x 40 = 240 threads)
constexpr int TM_TMEM_COLS = 256;                   // TM_MAXT x TM_N = 240, rounded to a power of two
constexpr int TM_LIP = 34;                          // L11^-1 row pitch: rows 16 bytes apart in the banks

__device__ __forceinline__ void tmem_ld8(uint32_t addr, uint32_t (&v)[8]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
                 : "r"(addr));
}

// stage = (panel b, tile T, quarter qk of the panel's 32 complex columns);
// the panels with rows below them are b = 0 .. nblk - 2, the tiles of panel
// b are T = (32 (b + 1)) / 128 .. nt - 1
struct TmStage {
    int b, T, qk;
};
__device__ __forceinline__ bool tm_next(TmStage& s, int nblk, int nt) {
    if (++s.qk < 4) return true;
    s.qk = 0;
    if (++s.T < nt) return true;
    if (++s.b >= nblk - 1) return false;
    s.T = (32 * (s.b + 1)) >> 7;
    return true;
}

// this thread's two K-quads of stage s: rows 8 rg + rr of the tile, quad kq
// (idx = tid + 256 j); zero outside rows [k1, n)
__device__ __forceinline__ void tm_load(float (&v)[2][4], const float2* __restrict__ F, int n, const TmStage& s) {
    const int k0 = 32 * s.b, k1 = k0 + 32;
#pragma unroll
    for (int j = 0; j < 2; ++j) {
        const int idx = threadIdx.x + 256 * j, rr = idx & 7, kq = (idx >> 3) & 3, rg = idx >> 5;
        const int r = 128 * s.T + 8 * rg + rr;
        if (r >= k1 && r < n) {
            const float2* src = F + tri(r) + k0 + 8 * s.qk + 2 * kq;
            const float2 a = src[0], b = src[1];
            v[j][0] = a.x; v[j][1] = a.y; v[j][2] = b.x; v[j][3] = b.y;
        } else {
            v[j][0] = v[j][1] = v[j][2] = v[j][3] = 0.f;
        }
    }
}

// rows outside [rlo, rhi) of the tile are not staged: they meet only
// accumulator lanes whose rows are already final (above the panel) or do not
// exist (n and beyond), which are never read again
__device__ __forceinline__ void tm_store(unsigned char* hi, unsigned char* lo, const float (&v)[2][4], int rlo,
                                         int rhi) {
#pragma unroll
    for (int j = 0; j < 2; ++j) {
        const int idx = threadIdx.x + 256 * j, rr = idx & 7, kq = (idx >> 3) & 3, rg = idx >> 5;
        if (8 * rg + rr < rlo || 8 * rg + rr >= rhi) continue;
        uint32_t h[4], l[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) tc::split_tf32(v[j][q], h[q], l[q]);
        const uint32_t o = tc::core_off(8 * rg + rr, 4 * kq, TM_KS / 4);
        st_shared_v4(hi + o, h[0], h[1], h[2], h[3]);
        st_shared_v4(lo + o, l[0], l[1], l[2], l[3]);
    }
}

__global__ void __launch_bounds__(256, 2) k_forms_tm(const float2* __restrict__ fac, const float2* __restrict__ linv,
                                                     int n, int N, const double* __restrict__ Q, int R,
                                                     double* __restrict__ c, int* status) {
    constexpr int NB = 32, RC = TM_RC, RCP = TM_RCP;
    extern __shared__ __align__(128) unsigned char sraw_tm[];
    unsigned char* sA = sraw_tm;                                     // [TM_NS][hi, lo][TM_A_BYTES]
    unsigned char* sB = sA + 2 * TM_NS * TM_A_BYTES;                 // [hi, lo][TM_B_BYTES]
    float2* sYb = reinterpret_cast<float2*>(sB + 2 * TM_B_BYTES);    // [NB][RCP]
    float2* sLi = sYb + NB * RCP;                                    // [NB][TM_LIP]
    float2* sD = sLi + NB * TM_LIP;                                  // [NB]
    double* red = reinterpret_cast<double*>(sYb);                    // [TM_GROUPS][RC], after the last panel
    __shared__ __align__(8) uint64_t mbar_buf[TM_NS];
    __shared__ __align__(8) uint64_t mbar_next, mbar_all;
    __shared__ uint32_t tbase;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int col = tid % RC, grp = tid / RC;                        // grp < TM_GROUPS: a y_b thread
    const int k = 1 + blockIdx.y, rc0 = blockIdx.x * RC, rc = min(RC, R - rc0);
    const float2* F = fac + (long long)k * tri(n);
    const int nblk = (n + NB - 1) / NB, nt = (n + 127) >> 7;
    const float2* Lk = linv + (long long)k * nblk * NB * NB;
    if (warp == 0) tc::tmem_alloc(&tbase, TM_TMEM_COLS);
    if (tid == 0) {
        for (int i = 0; i < TM_NS; ++i) tc::mbar_init(&mbar_buf[i]);
        tc::mbar_init(&mbar_next);
        tc::mbar_init(&mbar_all);
    }
    load_diag_pitched<TM_LIP>(sLi, sD, Lk, F, n, 0, min(NB, n));
    cp_async_commit();
    // q of this thread's rows of panel 0
    const bool ythread = grp < TM_GROUPS, live = ythread && col < rc;
    float qr[6];
#pragma unroll
    for (int m = 0; m < 6; ++m) {
        const int i = grp + TM_GROUPS * m;
        qr[m] = (live && i < NB && i < n) ? (float)Q[(long long)i * R + rc0 + col] : 0.f;
    }
    // operand rows of the first two stages; stages alternate the parity of
    // qk, and the set of a parity is refilled with the stage two ahead as soon
    // as it is stored
    TmStage ld{0, (32 >> 7), 0};
    bool have = nblk > 1;
    float av0[2][4], av1[2][4];
    if (have) {
        tm_load(av0, F, n, ld);
        tm_next(ld, nblk, nt);
        tm_load(av1, F, n, ld);
        have = tm_next(ld, nblk, nt);
    }
    tc::fence_async_smem();
    __syncthreads();
    tc::fence_after();
    const uint32_t taddr = tbase;
    int stage = 0;          // operand stages issued; stage s uses buffer s % TM_NS for the (s / TM_NS)-th time
    bool ok = true;
    double part = 0.0;
    for (int b = 0; b < nblk; ++b) {
        const int k0 = b * NB, kb = min(NB, n - k0), k1 = k0 + kb;
        // Y_b = q_b + dY_b
        if (b > 0) {
            ok = tc::mbar_wait(tc::smem_u32(&mbar_next), (b - 1) & 1) && ok;
            ok = __syncthreads_and(ok);
            if (!ok) break;
            tc::fence_after();
            const int T = k0 >> 7, qd = (k0 >> 5) & 3;
            if ((warp & 3) == qd) {
                const int part_im = warp >> 2;          // warp qd: Re columns, warp qd + 4: Im columns
                const uint32_t base = taddr + ((uint32_t)(32 * qd) << 16) + (uint32_t)(T * TM_N + RC * part_im);
                uint32_t v[RC / 8][8];
#pragma unroll
                for (int j = 0; j < RC / 8; ++j) tmem_ld8(base + 8 * j, v[j]);
                tc::tmem_wait_ld();
                // lanes past n hold whatever the unstaged operand rows produced: zero
                const bool row_live = k0 + lane < n;
#pragma unroll
                for (int j = 0; j < RC / 8; ++j)
#pragma unroll
                    for (int e = 0; e < 8; ++e)
                        reinterpret_cast<float*>(sYb + lane * RCP + 8 * j + e)[part_im] =
                            row_live ? __uint_as_float(v[j][e]) : 0.f;
            }
            tc::fence_before();
        }
        __syncthreads();
        if (ythread) {
#pragma unroll
            for (int m = 0; m < 6; ++m) {
                const int i = grp + TM_GROUPS * m;
                if (i < NB) {
                    float2* y = sYb + i * RCP + col;
                    if (b > 0) y->x += qr[m];
                    else *y = make_float2(qr[m], 0.f);
                }
            }
            // q of the next panel's rows, in flight while this panel runs
#pragma unroll
            for (int m = 0; m < 6; ++m) {
                const int i = k1 + grp + TM_GROUPS * m;
                qr[m] = (live && grp + TM_GROUPS * m < NB && i < n) ? (float)Q[(long long)i * R + rc0 + col] : 0.f;
            }
        }
        cp_async_wait<0>();
        __syncthreads();
        // y_b = L11^-1 Y_b for rows grp + 6 m of column col, and the forms sum
        float2 yb[6];
#pragma unroll
        for (int m = 0; m < 6; ++m) yb[m] = make_float2(0.f, 0.f);
        if (ythread) {
            // L11^-1 is lower triangular: row grp + 6 m needs p <= 6 m + 5 at most
            const float2* lrow = sLi + grp * TM_LIP;
#pragma unroll
            for (int p = 0; p < NB; ++p) {
                const float2 yv = sYb[p * RCP + col];
#pragma unroll
                for (int m = 0; m < 6; ++m)
                    if (TM_GROUPS * m + TM_GROUPS - 1 >= p && (m < 5 || TM_GROUPS * m < NB))
                        yb[m] = cfma(lrow[min(TM_GROUPS * m, NB - 1 - grp) * TM_LIP + p], yv, yb[m]);
            }
#pragma unroll
            for (int m = 0; m < 6; ++m) {
                const int i = grp + TM_GROUPS * m;
                if (i < kb) {
                    const float2 w = cdiv(cmul(yb[m], yb[m]), sD[i]);
                    part += (double)w.y;
                } else {
                    yb[m] = make_float2(0.f, 0.f);
                }
            }
        }
        // the previous panel's MMAs read the B operand: all done before it is rebuilt
        if (b > 0 && k0 < n) ok = tc::mbar_wait(tc::smem_u32(&mbar_all), (b - 1) & 1) && ok;
        if (k1 < n) {
            // y_b replaces Y_b in sYb, then the B operand is written in 16-byte
            // quads (rows 2q, 2q + 1 of y_b for one output column), lanes
            // spread over the eight rows of a core matrix
            __syncthreads();
            if (ythread) {
#pragma unroll
                for (int m = 0; m < 6; ++m) {
                    const int i = grp + TM_GROUPS * m;
                    if (i < NB) sYb[i * RCP + col] = yb[m];
                }
            }
            __syncthreads();
            for (int t = tid; t < TM_N * 16; t += blockDim.x) {
                const int rr = t & 7, q = (t >> 3) & 15, rg = t >> 7;    // B row 8 rg + rr, K quad q
                const int nr = 8 * rg + rr, c = nr < RC ? nr : nr - RC;
                const float2 y0 = sYb[(2 * q) * RCP + c], y1 = sYb[(2 * q + 1) * RCP + c];
                float v[4];
                if (nr < RC) { v[0] = -y0.x; v[1] = y0.y; v[2] = -y1.x; v[3] = y1.y; }
                else { v[0] = -y0.y; v[1] = -y0.x; v[2] = -y1.y; v[3] = -y1.x; }
                uint32_t h[4], l[4];
#pragma unroll
                for (int e = 0; e < 4; ++e) tc::split_tf32(v[e], h[e], l[e]);
                const uint32_t o = tc::core_off(nr, 4 * q, 16);
                st_shared_v4(sB + o, h[0], h[1], h[2], h[3]);
                st_shared_v4(sB + TM_B_BYTES + o, l[0], l[1], l[2], l[3]);
            }
        }
        tc::fence_async_smem();
        ok = __syncthreads_and(ok);
        if (!ok) break;
        if (b + 1 < nblk)      // next panel's L11^-1 and pivots: this panel's are no longer read
            load_diag_pitched<TM_LIP>(sLi, sD, Lk + (long long)(b + 1) * NB * NB, F, n, k1, min(NB, n - k1));
        cp_async_commit();
        if (k1 >= n) break;
        // MMAs of this panel: tiles T_first .. nt - 1, four K quarters each
        const int T_first = k1 >> 7;
        for (int T = T_first; T < nt; ++T) {
#pragma unroll
            for (int qk = 0; qk < 4; ++qk, ++stage) {
                const int buf = stage % TM_NS;
                if (stage >= TM_NS) ok = tc::mbar_wait(tc::smem_u32(&mbar_buf[buf]), ((stage / TM_NS) - 1) & 1) && ok;
                unsigned char* ah = sA + 2 * buf * TM_A_BYTES;
                if ((qk & 1) == 0) {
                    tm_store(ah, ah + TM_A_BYTES, av0, k1 - 128 * T, n - 128 * T);
                    if (have) tm_load(av0, F, n, ld);
                } else {
                    tm_store(ah, ah + TM_A_BYTES, av1, k1 - 128 * T, n - 128 * T);
                    if (have) tm_load(av1, F, n, ld);
                }
                if (have) have = tm_next(ld, nblk, nt);
                tc::fence_async_smem();
                __syncthreads();
                if (tid == 0) {
                    tc::fence_after();
                    const uint32_t a0 = tc::smem_u32(ah), a1 = a0 + TM_A_BYTES;
                    const uint32_t b0 = tc::smem_u32(sB), b1 = b0 + TM_B_BYTES;
                    const uint32_t d = taddr + (uint32_t)(T * TM_N);
#pragma unroll
                    for (int ks = 0; ks < TM_KS / 8; ++ks) {
                        const uint32_t oa = ks * 256, ob = (4 * qk + 2 * ks) * 128;
                        const uint32_t acc = (b > 0 || qk > 0 || ks > 0) ? 1u : 0u;
                        tc::mma_tf32(d, tc::smem_desc(a0 + oa, TM_SBO_A), tc::smem_desc(b0 + ob, TM_SBO_B), TM_IDESC, acc);
                        tc::mma_tf32(d, tc::smem_desc(a0 + oa, TM_SBO_A), tc::smem_desc(b1 + ob, TM_SBO_B), TM_IDESC, 1u);
                        tc::mma_tf32(d, tc::smem_desc(a1 + oa, TM_SBO_A), tc::smem_desc(b0 + ob, TM_SBO_B), TM_IDESC, 1u);
                    }
                    tc::commit(tc::smem_u32(&mbar_buf[buf]));
                    if (T == T_first && qk == 3) tc::commit(tc::smem_u32(&mbar_next));
                    if (T == nt - 1 && qk == 3) tc::commit(tc::smem_u32(&mbar_all));
                }
            }
        }
    }
    // every MMA done before the accumulators are released
    for (int i = 0; i < TM_NS; ++i) {
        const int cnt = (stage - i + TM_NS - 1) / TM_NS;     // stages that used buffer i
        if (cnt > 0) ok = tc::mbar_wait(tc::smem_u32(&mbar_buf[i]), (cnt - 1) & 1) && ok;
    }
    cp_async_wait<0>();
    ok = __syncthreads_and(ok);
    if (!ok && tid == 0) atomicOr(status, ST_TIMEOUT);
    if (ythread) red[grp * RC + col] = part;
    __syncthreads();
    if (ok && tid < rc) {
        double im = 0.0;
        for (int q = 0; q < TM_GROUPS; ++q) im += red[q * RC + tid];
        c[(long long)(rc0 + tid) * N + k] = -im / M_PI;
        if (k == 1) c[(long long)(rc0 + tid) * N] = 0.0;
    }
    tc::fence_before();
    __syncthreads();
    if (warp == 0) {
        tc::fence_after();
        tc::tmem_dealloc(taddr, TM_TMEM_COLS);
    }
}

// Batched forward substitution for large n (the right-hand-side chunk no
// longer fits on chip): Y [nb][n][R] lives in HBM for a batch of nb
// frequencies k = kbase + z, and every panel takes two launches over the
// whole batch.  k_formsb_diag: y_b = L11^-1 y_b for 64 right-hand sides per
// CTA (one column per thread group, the column's NB values in registers),
// y_i^2/d_i added to the binary64 sums acc [nb][R]; the last panel writes
// c.  k_formsb_update: Y -= L y_b by T x T tiles.  On the binary32 path
// panels go in pairs: the first panel's update reaches only the second
// panel's rows, and the rows below the pair take both panels' updates in one
// read-modify-write of Y (K = 2 NB), which halves the HBM traffic of Y.  Before the first update
// the right-hand sides are the real q (Q [n][R]).
template <typename C>
__global__ void __launch_bounds__(256) k_formsb_diag(const C* __restrict__ fac, const C* __restrict__ linv, int n,
                                                     int N, const double* __restrict__ Q, int R, C* __restrict__ Y,
                                                     double* __restrict__ acc, double* __restrict__ c, int k0,
                                                     int kbase, const int* __restrict__ kmap) {
    typedef typename CT<C>::R T;
    constexpr int NB = Tile<C>::NB, G = 4, RPT = NB / G;     // row groups, rows per thread
    __shared__ C sLi[NB][NB];
    __shared__ C sD[NB];
    __shared__ double red[G][64];
    const int tid = threadIdx.x, cl = tid % 64, g = tid / 64;
    const int z = blockIdx.y, k = kbase + z, col = blockIdx.x * 64 + cl;
    const C* F = fac + (long long)k * tri(n);
    C* Yk = Y + (long long)z * n * R;
    const int kb = min(NB, n - k0), nblk = (n + NB - 1) / NB;
    const bool last = k0 + kb == n;
    const C* Li = linv + ((long long)k * nblk + k0 / NB) * NB * NB;
    for (int t = tid; t < NB * NB; t += blockDim.x) sLi[t / NB][t % NB] = Li[t];
    if (tid < NB) sD[tid] = tid < kb ? F[tri(k0 + tid) + k0 + tid] : CT<C>::mk(T(1), T(0));
    C y[NB];
    const bool live = col < R;
#pragma unroll
    for (int p = 0; p < NB; ++p) {
        const long long o = (long long)(k0 + p) * R + col;
        y[p] = (live && p < kb) ? (k0 == 0 ? CT<C>::mk(T(Q[o]), T(0)) : Yk[o]) : CT<C>::mk(T(0), T(0));
    }
    __syncthreads();                    // every column read before any row is rewritten
    C part = CT<C>::mk(T(0), T(0));
#pragma unroll
    for (int q = 0; q < RPT; ++q) {
        const int i = g + G * q;
        C v = CT<C>::mk(T(0), T(0));
#pragma unroll
        for (int p = 0; p < NB; ++p) v = cfma(sLi[i][p], y[p], v);
        if (live && i < kb) {
            if (!last) Yk[(long long)(k0 + i) * R + col] = v;
            part = cadd(part, cdiv(cmul(v, v), sD[i]));
        }
    }
    red[g][cl] = (double)part.y;
    __syncthreads();
    if (g == 0 && live) {
        double s = red[0][cl] + red[1][cl] + red[2][cl] + red[3][cl];
        double* a = acc + (long long)z * R + col;
        s += k0 == 0 ? 0.0 : *a;
        if (last) {
            // factors k of the compact set (kmap given) belong to frequency kmap[k]
            c[(long long)col * N + (kmap ? kmap[k] : k)] = -s / M_PI;
            if (!kmap && k == 1) c[(long long)col * N] = 0.0;
        } else {
            *a = s;
        }
    }
}

// The four panels of one 128-row block of the left-looking substitution in
// one launch (binary32): the block's rows of Y for 64 right-hand sides stay
// in shared memory while each panel takes its diagonal solve y_b = L11^-1 y_b
// (with its y^2/d sums) and updates the block's later rows,
// Y[r] -= L[r][panel] y_b.  The arithmetic of every entry is that of
// k_formsb_diag and k_formsb_update (same operations in the same order); Y
// is read and written once per block instead of once per panel step, and
// one launch replaces seven.  Rows before the first block come from q; the
// last block of the matrix writes c and no Y.
constexpr size_t BK_SMEM = sizeof(float2) * (128 * 64 + 96 * 33);

__global__ void __launch_bounds__(256) k_formsb_block(const float2* __restrict__ fac, const float2* __restrict__ linv,
                                                      int n, int N, const double* __restrict__ Q, int R,
                                                      float2* __restrict__ Y, double* __restrict__ acc,
                                                      double* __restrict__ c, int i0, int kbase,
                                                      const int* __restrict__ kmap) {
    constexpr int NB = 32, G = 4, RPT = NB / G, RC = 64, LP = NB + 1;
    extern __shared__ __align__(16) unsigned char sraw_bk[];
    float2* Ys = reinterpret_cast<float2*>(sraw_bk);                 // [128][RC]
    float2* sL = Ys + 128 * RC;                                       // [96][LP]: later rows x panel columns
    __shared__ float2 sLi[NB][NB];
    __shared__ float2 sD[NB];
    __shared__ double red[G][RC];
    __shared__ double sacc[RC];
    const int tid = threadIdx.x, cl = tid % RC, g = tid / RC;
    const int z = blockIdx.y, k = kbase + z, col = blockIdx.x * RC + cl;
    const bool live = col < R;
    const float2* F = fac + (long long)k * tri(n);
    float2* Yk = Y + (long long)z * n * R;
    const int i1 = min(n, i0 + 128), nblk = (n + NB - 1) / NB;
    // the block's rows of Y (q before any update)
    for (int t = tid; t < 128 * RC; t += blockDim.x) {
        const int rr = t / RC, cc = t % RC, r = i0 + rr, cg = blockIdx.x * RC + cc;
        float2 v = make_float2(0.f, 0.f);
        if (r < i1 && cg < R) {
            const long long o = (long long)r * R + cg;
            v = i0 == 0 ? make_float2((float)Q[o], 0.f) : Yk[o];
        }
        Ys[t] = v;
    }
    if (g == 0) sacc[cl] = (i0 == 0 || !live) ? 0.0 : acc[(long long)z * R + col];
    for (int k0 = i0; k0 < i1; k0 += NB) {
        const int kb = min(NB, n - k0), k1 = k0 + kb, nl = i1 - k1;
        const bool last = k1 == n;
        const float2* Li = linv + ((long long)k * nblk + k0 / NB) * NB * NB;
        __syncthreads();                          // previous panel's update done
        for (int t = tid; t < NB * NB; t += blockDim.x) sLi[t / NB][t % NB] = Li[t];
        if (tid < NB) sD[tid] = tid < kb ? F[tri(k0 + tid) + k0 + tid] : make_float2(1.f, 0.f);
        for (int t = tid; t < nl * NB; t += blockDim.x) {
            const int rr = t / NB, p = t % NB;
            sL[rr * LP + p] = p < kb ? F[tri(k1 + rr) + k0 + p] : make_float2(0.f, 0.f);
        }
        float2 y[NB];
#pragma unroll
        for (int p = 0; p < NB; ++p)
            y[p] = (live && p < kb) ? Ys[(k0 - i0 + p) * RC + cl] : make_float2(0.f, 0.f);
        __syncthreads();                          // every panel row read before any is rewritten
        // diagonal block: rows g + G q of the panel
        float2 part = make_float2(0.f, 0.f);
        float2 vq[RPT];
#pragma unroll
        for (int q = 0; q < RPT; ++q) {
            const int i = g + G * q;
            float2 v = make_float2(0.f, 0.f);
#pragma unroll
            for (int p = 0; p < NB; ++p) v = cfma(sLi[i][p], y[p], v);
            vq[q] = v;
            if (live && i < kb) part = cadd(part, cdiv(cmul(v, v), sD[i]));
        }
#pragma unroll
        for (int q = 0; q < RPT; ++q) {
            const int i = g + G * q;
            if (i < kb) Ys[(k0 - i0 + i) * RC + cl] = vq[q];
        }
        red[g][cl] = (double)part.y;
        __syncthreads();
        if (g == 0 && live) {
            double sum = red[0][cl] + red[1][cl] + red[2][cl] + red[3][cl];
            sum += k0 == 0 ? 0.0 : sacc[cl];
            if (last) {
                c[(long long)col * N + (kmap ? kmap[k] : k)] = -sum / M_PI;
                if (!kmap && k == 1) c[(long long)col * N] = 0.0;
            }
            sacc[cl] = sum;
        }
        // the block's later rows: Y[r] -= sum_p L[r][k0 + p] y_b[p], rows g + G q' of them
        // (the solved panel column in registers)
        if (nl > 0) {
#pragma unroll
            for (int p = 0; p < NB; ++p) y[p] = p < kb ? Ys[(k0 - i0 + p) * RC + cl] : make_float2(0.f, 0.f);
        }
        for (int rr = g; rr < nl; rr += G) {
            float2 a = make_float2(0.f, 0.f);
#pragma unroll
            for (int p = 0; p < NB; ++p) a = cfma(sL[rr * LP + p], y[p], a);
            float2* dst = &Ys[(k1 - i0 + rr) * RC + cl];
            *dst = csub(*dst, a);
        }
    }
    __syncthreads();
    if (i1 < n) {
        // Y of the block for the later block products, and the running sums
        for (int t = tid; t < (i1 - i0) * RC; t += blockDim.x) {
            const int rr = t / RC, cc = t % RC, cg = blockIdx.x * RC + cc;
            if (cg < R) Yk[(long long)(i0 + rr) * R + cg] = Ys[t];
        }
        if (g == 0 && live) acc[(long long)z * R + col] = sacc[cl];
    }
}

// Y[r_lo, r_hi) -= L[r_lo.., kk0 .. kk0 + kw) y[kk0 .. kk0 + kw) for one
// T x T tile (rows, right-hand sides) of frequency kbase + blockIdx.z; KW >=
// kw is the compile-time panel width (one panel, or two panels at once so
// that the rows below a panel pair are read and written once).  The first
// update of an element starts from the real q (kk0 == 0).
template <typename C, int KW>
__global__ void __launch_bounds__(256) k_formsb_update(const C* __restrict__ fac, int n, const double* __restrict__ Q,
                                                       int R, C* __restrict__ Y, int kk0, int kw, int r_lo, int r_hi,
                                                       int kbase) {
    typedef typename CT<C>::R T;
    constexpr int TT = Tile<C>::T, TA = Tile<C>::A;
    extern __shared__ __align__(16) unsigned char sraw_fb[];
    C (*sL)[KW + 1] = reinterpret_cast<C (*)[KW + 1]>(sraw_fb);
    C (*sY)[TT] = reinterpret_cast<C (*)[TT]>(sraw_fb + sizeof(C) * TT * (KW + 1));
    const int tid = threadIdx.x, z = blockIdx.z, k = kbase + z;
    const C* F = fac + (long long)k * tri(n);
    C* Yk = Y + (long long)z * n * R;
    const int r0 = r_lo + blockIdx.x * TT, c0 = blockIdx.y * TT;
    for (int t = tid; t < TT * KW; t += blockDim.x) {
        const int rr = t / KW, p = t % KW;
        sL[rr][p] = (p < kw && r0 + rr < r_hi) ? F[tri(r0 + rr) + kk0 + p] : CT<C>::mk(T(0), T(0));
    }
    for (int t = tid; t < KW * TT; t += blockDim.x) {
        const int p = t / TT, cc = t % TT;
        sY[p][cc] = (p < kw && c0 + cc < R) ? Yk[(long long)(kk0 + p) * R + c0 + cc] : CT<C>::mk(T(0), T(0));
    }
    __syncthreads();
    const int ty = tid / 16, tx = tid % 16;
    C acc[TA][TA];
#pragma unroll
    for (int a = 0; a < TA; ++a)
#pragma unroll
        for (int b = 0; b < TA; ++b) acc[a][b] = CT<C>::mk(T(0), T(0));
#pragma unroll 8
    for (int p = 0; p < KW; ++p) {
        C l[TA], yv[TA];
#pragma unroll
        for (int a = 0; a < TA; ++a) l[a] = sL[ty + 16 * a][p];
#pragma unroll
        for (int b = 0; b < TA; ++b) yv[b] = sY[p][tx + 16 * b];
#pragma unroll
        for (int a = 0; a < TA; ++a)
#pragma unroll
            for (int b = 0; b < TA; ++b) acc[a][b] = cfma(l[a], yv[b], acc[a][b]);
    }
#pragma unroll
    for (int a = 0; a < TA; ++a) {
        const int i = r0 + ty + 16 * a;
        if (i >= r_hi) continue;
#pragma unroll
        for (int b = 0; b < TA; ++b) {
            const int cc = c0 + tx + 16 * b;
            if (cc >= R) continue;
            const long long o = (long long)i * R + cc;
            const C src = kk0 == 0 ? CT<C>::mk(T(Q[o]), T(0)) : Yk[o];
            Yk[o] = csub(src, acc[a][b]);
        }
    }
}

// Left-looking form of the batched forward substitution (binary32 path):
// block I of 128 rows (rows i0 .. i1) first takes the product of every row
// above it at once,
//   Y[i0:i1, :] = q[i0:i1, :] - L[i0:i1, 0:i0] Y[0:i0, :],
// as one real TF32 product per 128-row block and tile of 128 right-hand
// sides, with the complex entries interleaved along K (3xTF32: A_hi B_hi
// into one tensor-memory accumulator, A_hi B_lo + A_lo B_hi into a second;
// M = 128, N = 256 = Re and Im of 128 right-hand sides, K = 8 per MMA).  The
// K loop runs over chunks of 16 columns of L in two shared-memory buffers
// (hi and lo of the block's L rows and of the chunk's rows of Y, 96 KB
// each): eight producer warps load a chunk two chunks ahead, split it and
// store it in the canonical K-major layout, then arrive on the buffer's
// `full` barrier; a ninth warp issues the chunk's 12 MMAs once it is full
// and commits their completion to the buffer's `empty` barrier.  The
// accumulators stay in tensor memory (all 512 columns) for the whole K loop
// and each block of Y is written once.  The four 32-row panels of the block
// then take the diagonal-block solves and the small updates inside the
// block (k_formsb_diag, k_formsb_update).  Y is read once per block below
// it instead of read and written once per panel pair.  One CTA per (tile of
// right-hand sides, frequency); the tiles of one frequency are neighbours
// in the grid and share L through L2.
constexpr int FG_KC = 16, FG_KR = 2 * FG_KC, FG_NC = 128, FG_N = 2 * FG_NC;
constexpr int FG_A_BYTES = 128 * FG_KR * 4;             // 128 x 32 binary32 (hi or lo): 16 KB
constexpr int FG_B_BYTES = FG_N * FG_KR * 4;            // 256 x 32 binary32 (hi or lo): 32 KB
constexpr int FG_STAGE = 2 * FG_A_BYTES + 2 * FG_B_BYTES;
constexpr uint32_t FG_SBO = (FG_KR / 4) * 128;
constexpr uint32_t FG_IDESC = tc::idesc_tf32(128, FG_N);
constexpr size_t FG_SMEM = 2 * (size_t)FG_STAGE;
constexpr uint32_t FG_TMEM = 2 * FG_N;                  // hi x hi and cross terms: all 512 columns
static_assert(FG_SMEM <= SMEM_DYN_MAX, "forms product: shared memory");
static_assert(FG_TMEM == 512 && 2 * FG_SMEM > SMEM_PER_SM, "forms product: one CTA per SM");

// this thread's raw entries of chunk kk (columns kk .. kk + 15 of L rows i0 ..,
// rows kk .. kk + 15 of Y): 4 quads of A, 4 quads of B (two complex each)
__device__ __forceinline__ void fg_load(float2 (&av)[4][2], float2 (&bv)[4][2], const float2* __restrict__ F,
                                        const float2* __restrict__ Yk, int R, int i0, int i1, int kk, int c0) {
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int idx = threadIdx.x + 256 * j, rr = idx & 7, kq = (idx >> 3) & 7, rg = idx >> 6;
        const int ra = i0 + 8 * rg + rr;
        if (ra < i1) {
            const float2* src = F + tri(ra) + kk + 2 * kq;
            av[j][0] = src[0];
            av[j][1] = src[1];
        } else {
            av[j][0] = av[j][1] = make_float2(0.f, 0.f);
        }
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int idx = threadIdx.x + 256 * j, q = idx & 127, kq = idx >> 7, col = c0 + q;
        if (col < R) {
            bv[j][0] = Yk[(long long)(kk + 2 * kq) * R + col];
            bv[j][1] = Yk[(long long)(kk + 2 * kq + 1) * R + col];
        } else {
            bv[j][0] = bv[j][1] = make_float2(0.f, 0.f);
        }
    }
}

__device__ __forceinline__ void fg_store(const float2 (&av)[4][2], const float2 (&bv)[4][2], unsigned char* st) {
    unsigned char* ah = st;
    unsigned char* al = ah + FG_A_BYTES;
    unsigned char* bh = al + FG_A_BYTES;
    unsigned char* bl = bh + FG_B_BYTES;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int idx = threadIdx.x + 256 * j, rr = idx & 7, kq = (idx >> 3) & 7, rg = idx >> 6;
        st_shared_quad(ah, al, tc::core_off(8 * rg + rr, 4 * kq, FG_KR / 4), av[j][0].x, av[j][0].y, av[j][1].x,
                       av[j][1].y);
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int idx = threadIdx.x + 256 * j, q = idx & 127, kq = idx >> 7;
        const float2 y0 = bv[j][0], y1 = bv[j][1];
        st_shared_quad(bh, bl, tc::core_off(q, 4 * kq, FG_KR / 4), y0.x, -y0.y, y1.x, -y1.y);
        st_shared_quad(bh, bl, tc::core_off(FG_NC + q, 4 * kq, FG_KR / 4), y0.y, y0.x, y1.y, y1.x);
    }
}

__global__ void __launch_bounds__(288, 1) k_formsb_gemm_tc(const float2* __restrict__ fac, int n,
                                                           const double* __restrict__ Q, int R,
                                                           float2* __restrict__ Y, int i0, int i1, int kbase,
                                                           int* status) {
    extern __shared__ __align__(128) unsigned char sraw_fg[];
    __shared__ __align__(8) uint64_t full[2], empty[2], done;
    __shared__ uint32_t tbase;
    __shared__ int s_abort;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int z = blockIdx.y, k = kbase + z, c0 = FG_NC * blockIdx.x;
    const float2* F = fac + (long long)k * tri(n);
    float2* Yk = Y + (long long)z * n * R;
    const int nk = i0 / FG_KC;                            // i0 is a multiple of 128
    if (warp == 0) tc::tmem_alloc(&tbase, FG_TMEM);
    if (tid == 0) {
        tc::mbar_init_n(&full[0], 256);
        tc::mbar_init_n(&full[1], 256);
        tc::mbar_init(&empty[0]);
        tc::mbar_init(&empty[1]);
        tc::mbar_init(&done);
        s_abort = 0;
    }
    __syncthreads();
    tc::fence_after();
    const uint32_t taddr = tbase;
    volatile int* abort = &s_abort;
    int issued = 0;                                       // chunks whose MMAs the issuing lane committed
    if (warp < 8) {
        // producers: chunk kc into buffer kc % 2 once the MMAs of chunk kc - 2 have released
        // it (chunk c's raw entries in register set c % 2, loaded two chunks ahead)
        float2 av0[4][2], bv0[4][2], av1[4][2], bv1[4][2];
        fg_load(av0, bv0, F, Yk, R, i0, i1, 0, c0);
        if (nk > 1) fg_load(av1, bv1, F, Yk, R, i0, i1, FG_KC, c0);
        int kc = 0;
        auto step = [&](float2 (&av)[4][2], float2 (&bv)[4][2]) -> bool {
            const int s = kc & 1;
            if (kc >= 2 && !tc::mbar_wait_abort(tc::smem_u32(&empty[s]), ((kc - 2) >> 1) & 1, abort)) return false;
            fg_store(av, bv, sraw_fg + s * FG_STAGE);
            if (kc + 2 < nk) fg_load(av, bv, F, Yk, R, i0, i1, FG_KC * (kc + 2), c0);
            tc::fence_async_smem();
            tc::mbar_arrive(tc::smem_u32(&full[s]));
            return true;
        };
        while (kc < nk) {
            if (!step(av0, bv0) || ++kc >= nk) break;
            if (!step(av1, bv1)) break;
            ++kc;
        }
    } else if (lane == 0) {
        // the MMA lane: chunk kc once its buffer is full, completion to empty[kc % 2]
        for (int kc = 0; kc < nk; ++kc) {
            const int s = kc & 1;
            if (!tc::mbar_wait_abort(tc::smem_u32(&full[s]), (kc >> 1) & 1, abort)) break;
            tc::fence_after();
            const uint32_t st = tc::smem_u32(sraw_fg + s * FG_STAGE);
            const uint32_t ah = st, al = st + FG_A_BYTES, bh = st + 2 * FG_A_BYTES, bl = bh + FG_B_BYTES;
#pragma unroll
            for (int ks = 0; ks < FG_KR / 8; ++ks) {
                const uint32_t o = ks * 256, acc = (kc > 0 || ks > 0) ? 1u : 0u;
                tc::mma_tf32(taddr, tc::smem_desc(ah + o, FG_SBO), tc::smem_desc(bh + o, FG_SBO), FG_IDESC, acc);
                tc::mma_tf32(taddr + FG_N, tc::smem_desc(ah + o, FG_SBO), tc::smem_desc(bl + o, FG_SBO), FG_IDESC,
                             acc);
                tc::mma_tf32(taddr + FG_N, tc::smem_desc(al + o, FG_SBO), tc::smem_desc(bh + o, FG_SBO), FG_IDESC,
                             1u);
            }
            tc::commit(tc::smem_u32(&empty[s]));
            issued = kc + 1;
        }
        if (issued == nk) tc::commit(tc::smem_u32(&done));
    }
    // epilogue (producer warps): Y rows i0 .. i1 = q - product; warp w reads lanes
    // 32 (w % 4) .. (rows) and right-hand sides 64 (w / 4) .. + 63 of the tile, 16 at a time
    if (warp < 8) {
        bool ok = tc::mbar_wait_abort(tc::smem_u32(&done), 0, abort);
        ok = __all_sync(0xffffffffu, ok);                // tcgen05.ld below is warp-collective
        if (ok) {
            tc::fence_after();
            const int r = i0 + 32 * (warp & 3) + lane, h = warp >> 2;
            const uint32_t base = taddr + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(64 * h);
#pragma unroll 1
            for (int j = 0; j < 4; ++j) {
                uint32_t re[16], im[16], re2[16], im2[16];
                tc::tmem_ld16(base + 16 * j, re);
                tc::tmem_ld16(base + FG_NC + 16 * j, im);
                tc::tmem_ld16(base + FG_N + 16 * j, re2);
                tc::tmem_ld16(base + FG_N + FG_NC + 16 * j, im2);
                tc::tmem_wait_ld();
                if (r < i1) {
                    const int cb = c0 + 64 * h + 16 * j;
                    const long long o = (long long)r * R + cb;
#pragma unroll
                    for (int q = 0; q < 16; ++q)
                        if (cb + q < R)
                            Yk[o + q] = make_float2(
                                (float)Q[o + q] - (__uint_as_float(re[q]) + __uint_as_float(re2[q])),
                                -(__uint_as_float(im[q]) + __uint_as_float(im2[q])));
                }
            }
        }
    }
    __syncthreads();
    if (*abort) {
        // a wait ran out: the MMAs committed so far finish before the columns are freed
        if (tid == 0) atomicOr(status, ST_TIMEOUT);
        if (warp == 8 && lane == 0 && issued > 0)
            tc::mbar_wait(tc::smem_u32(&empty[(issued - 1) & 1]), ((issued - 1) >> 1) & 1);
    }
    tc::fence_before();
    __syncthreads();
    if (warp == 0) {
        tc::fence_after();
        tc::tmem_dealloc(taddr, FG_TMEM);
    }
}

// out = M_k^-1 - 1 = chi^RPA_k from the factors (test read-back): column
// col = blockIdx.x * blockDim.x + threadIdx.x of X solves L D L^T x = e_col.
__global__ void __launch_bounds__(256) k_ldlt_inverse(const double2* __restrict__ F, int n, double2* __restrict__ X) {
    {
        const int col = blockIdx.x * blockDim.x + threadIdx.x;
        if (col >= n) return;
        double2* x = X + (long long)col;      // strided column (row-major X)
        for (int i = 0; i < n; ++i) x[(long long)i * n] = make_double2(i == col ? 1.0 : 0.0, 0.0);
        for (int i = 0; i < n; ++i) {
            double2 y = x[(long long)i * n];
            for (int p = 0; p < i; ++p) y = cfms(F[tri(i) + p], x[(long long)p * n], y);
            x[(long long)i * n] = y;
        }
        for (int i = 0; i < n; ++i) x[(long long)i * n] = cdiv(x[(long long)i * n], F[tri(i) + i]);
        for (int i = n - 1; i >= 0; --i) {
            double2 y = x[(long long)i * n];
            for (int p = i + 1; p < n; ++p) y = cfms(F[tri(p) + i], x[(long long)p * n], y);
            x[(long long)i * n] = y;
        }
        x[(long long)col * n].x -= 1.0;
    }
}

// out[i] = chi0_32 of frequency kd[i] (or k1 when kd is null), packed, in binary64
__global__ void k_gather_c128(const float2* __restrict__ chi0, const int* __restrict__ kd, int k1, int np, long long pk,
                              double2* __restrict__ out) {
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= (long long)np * pk) return;
    const int i = (int)(t / pk);
    const long long e = t % pk;
    const float2 v = chi0[(long long)(kd ? kd[i] : k1) * pk + e];
    out[t] = make_double2(v.x, v.y);
}

// out[i][e] = chi0 of frequency kd[i] (or k1 when kd is null), packed element
// e, in binary64 by the direct Cauchy sum over the band of the binary64
// weights A64 [band][n_el] (Eq. chi_by_spectra):
//   chi0_k[e] = sum_b A64[b][e] [kap(k - j_lo - b) - kap(k + j_lo + b)].
// One CTA per (element tile of 256, frequency); the CTA's kernel row is
// tabulated in shared memory first.
__global__ void __launch_bounds__(256) k_kk_band64(const double* __restrict__ A64, int band, long long n_el, int j_lo,
                                                   double dw, double eta, const int* __restrict__ kd, int k1,
                                                   double2* __restrict__ out) {
    extern __shared__ double2 sk[];
    const int i = blockIdx.y, k = kd ? kd[i] : k1;
    for (int b = threadIdx.x; b < band; b += blockDim.x) {
        const long long j = j_lo + b;
        const double x1 = (double)(k - j) * dw, x2 = (double)(k + j) * dw, e2 = eta * eta;
        const double d1 = x1 * x1 + e2, d2 = x2 * x2 + e2;
        sk[b] = make_double2(x1 / d1 - x2 / d2, -eta / d1 + eta / d2);
    }
    __syncthreads();
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n_el) return;
    double re = 0.0, im = 0.0;
    for (int b = 0; b < band; ++b) {
        const double a = A64[(long long)b * n_el + e];
        re = fma(a, sk[b].x, re);
        im = fma(a, sk[b].y, im);
    }
    out[(long long)i * n_el + e] = make_double2(re, im);
}

__global__ void k_c64_to_c128(const float2* __restrict__ a, double2* __restrict__ b, long long n) {
    long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t < n) b[t] = make_double2(a[t].x, a[t].y);
}

}  // namespace

template <typename C>
static void ldlt_steps(gw_ctx* ctx, const C* chi0, C* fac, int n, int N, C* linv, double* piv,
                       const char* const names[4]) {
    constexpr int NB = Tile<C>::NB, TT = Tile<C>::T;
    klaunch(ctx, names[0], k_ldlt_init<C>, N, 256, 0, chi0, fac, n, piv);
    for (int k0 = 0; k0 < n; k0 += NB) {
        klaunch(ctx, names[1], k_ldlt_panel<C>, N, 256, 0, fac, n, N, k0, linv, piv, ctx->d_status);
        const int m = n - std::min(n, k0 + NB);
        if (m == 0) break;
        if constexpr (sizeof(C) == 8) {
            // binary32: trailing updates with at least one full 128-row block on the tensor cores
            if (!ctx->syrk_simt && m >= 128 && N <= 65535) {
                allow_max_smem(k_ldlt_syrk_tc);
                if (m - NB >= 128) {
                    // two panels per pass over the trailing matrix: the next panel's columns
                    // first, that panel factored, then both updates of the rest in one launch
                    klaunch(ctx, names[3], k_ldlt_syrk_tc, dim3(div_up(m, 128), N), 256, ST_SMEM, (float2*)fac, n,
                            k0, 1, ctx->d_status);
                    klaunch(ctx, names[1], k_ldlt_panel<C>, N, 256, 0, fac, n, N, k0 + NB, linv, piv,
                            ctx->d_status);
                    allow_max_smem(k_ldlt_syrk_tc2);
                    klaunch(ctx, "k_ldlt32_syrk_tc2", k_ldlt_syrk_tc2, dim3(div_up(m - NB, 128), N), 256, ST2_SMEM,
                            (float2*)fac, n, k0, ctx->d_status);
                    k0 += NB;
                    continue;
                }
                klaunch(ctx, names[3], k_ldlt_syrk_tc, dim3(div_up(m, 128), N), 256, ST_SMEM, (float2*)fac, n, k0,
                        1 << 30, ctx->d_status);
                continue;
            }
        }
        const int nt = div_up(m, TT);
        klaunch(ctx, names[2], k_ldlt_syrk<C>, dim3(nt * (nt + 1) / 2, N), 256, 0, fac, n, k0);
    }
}

size_t ldlt_linv_bytes(int n, int N, gw_precision prec) {
    if (prec == GW_MIXED) return (size_t)N * div_up(n, Tile<float2>::NB) * Tile<float2>::NB * Tile<float2>::NB * sizeof(float2);
    return (size_t)N * div_up(n, Tile<double2>::NB) * Tile<double2>::NB * Tile<double2>::NB * sizeof(double2);
}

void launch_ldlt(gw_ctx* ctx, gw_W* W) {
    const gw_chi0* c = W->chi0;
    const int n = c->n_sub, N = c->grid.n_omega;
    if (c->prec == GW_MIXED) {
        static const char* const nm[4] = {"k_ldlt32_init", "k_ldlt32_panel", "k_ldlt32_syrk", "k_ldlt32_syrk_tc"};
        ldlt_steps<float2>(ctx, (const float2*)c->chi0_32, W->fac32, n, N, (float2*)W->linv, W->piv, nm);
    } else {
        static const char* const nm[4] = {"k_ldlt_init", "k_ldlt_panel", "k_ldlt_syrk", "k_ldlt_syrk_tc"};
        ldlt_steps<double2>(ctx, (const double2*)c->chi0, W->fac, n, N, (double2*)W->linv, W->piv, nm);
    }
}

// kmap == nullptr: the factors of frequencies 1 .. N-1 (frequency 0 has c = 0);
// else the nd factors of a compact set, entry i belonging to frequency kmap[i].
template <typename C>
static void forms_batched(gw_ctx* ctx, const C* fac, const C* linv, int n, int N, const double* Q, int R,
                          double* cout, const char* const names[3], const int* kmap = nullptr, int nd = 0) {
    constexpr int NB = Tile<C>::NB, TT = Tile<C>::T;
    const int kfirst = kmap ? 0 : 1, kend = kmap ? nd : N;
    // frequencies per batch: Y [nb][n][R] within about 2 GB
    const size_t per = sizeof(C) * (size_t)n * R;
    const int nb = (int)std::max<size_t>(1, std::min<size_t>((size_t)(kend - kfirst), ((size_t)2 << 30) / per));
    if (nb > 65535 || div_up(R, 64) > 65535) gw_throw(GW_ERR_INVALID_ARG, "forms batch too large");
    C* Y = dalloc<C>(ctx, (size_t)nb * n * R);
    double* acc = nullptr;
    try {
        acc = dalloc<double>(ctx, (size_t)nb * R);
        const size_t sm1 = sizeof(C) * ((size_t)TT * (NB + 1) + (size_t)NB * TT);
        const size_t sm2 = sizeof(C) * ((size_t)TT * (2 * NB + 1) + (size_t)2 * NB * TT);
        allow_max_smem(k_formsb_update<C, NB>);
        allow_max_smem(k_formsb_update<C, 2 * NB>);
        for (int kbase = kfirst; kbase < kend; kbase += nb) {
            const int nbb = std::min(nb, kend - kbase);
            if constexpr (sizeof(C) == 16) {
                // binary64: bound by the binary64 arithmetic, not by the traffic of Y, so one
                // panel per update (fewer launches)
                for (int k0 = 0; k0 < n; k0 += NB) {
                    const int k1 = std::min(n, k0 + NB);
                    klaunch(ctx, names[0], k_formsb_diag<C>, dim3(div_up(R, 64), nbb), 256, 0, fac, linv, n, N, Q, R,
                            Y, acc, cout, k0, kbase, kmap);
                    if (k1 == n) break;
                    klaunch(ctx, names[1], k_formsb_update<C, NB>, dim3(div_up(n - k1, TT), div_up(R, TT), nbb), 256,
                            sm1, fac, n, Q, R, Y, k0, k1 - k0, k1, n, kbase);
                }
            } else if (!ctx->forms_simt) {
                // left-looking in blocks of 128 rows: the product of all rows above the block on
                // the tensor cores, then the block's four panels
                allow_max_smem(k_formsb_gemm_tc);
                allow_max_smem(k_formsb_block);
                for (int i0 = 0; i0 < n; i0 += 128) {
                    const int i1 = std::min(n, i0 + 128);
                    if (i0 > 0)
                        klaunch(ctx, names[2], k_formsb_gemm_tc, dim3(div_up(R, FG_NC), nbb), 288, FG_SMEM,
                                (const float2*)fac, n, Q, R, (float2*)Y, i0, i1, kbase, ctx->d_status);
                    klaunch(ctx, "k_forms32_block", k_formsb_block, dim3(div_up(R, 64), nbb), 256, BK_SMEM,
                            (const float2*)fac, (const float2*)linv, n, N, Q, R, (float2*)Y, acc, cout, i0, kbase,
                            kmap);
                }
            } else {
                for (int k0 = 0; k0 < n; k0 += 2 * NB) {
                    // panel pair k0 .. k2: diagonal block, second panel's rows, diagonal block, rows below
                    const int k1 = std::min(n, k0 + NB), k2 = std::min(n, k1 + NB);
                    klaunch(ctx, names[0], k_formsb_diag<C>, dim3(div_up(R, 64), nbb), 256, 0, fac, linv, n, N, Q, R, Y, acc,
                            cout, k0, kbase, kmap);
                    if (k1 == n) break;
                    klaunch(ctx, names[1], k_formsb_update<C, NB>, dim3(div_up(k2 - k1, TT), div_up(R, TT), nbb), 256, sm1,
                            fac, n, Q, R, Y, k0, k1 - k0, k1, k2, kbase);
                    klaunch(ctx, names[0], k_formsb_diag<C>, dim3(div_up(R, 64), nbb), 256, 0, fac, linv, n, N, Q, R, Y, acc,
                            cout, k1, kbase, kmap);
                    if (k2 == n) break;
                    klaunch(ctx, names[1], k_formsb_update<C, 2 * NB>, dim3(div_up(n - k2, TT), div_up(R, TT), nbb), 256,
                            sm2, fac, n, Q, R, Y, k0, k2 - k0, k2, n, kbase);
                }
            }
        }
    } catch (...) {
        ctx_free(ctx, Y);
        ctx_free(ctx, acc);
        throw;
    }
    ctx_free(ctx, Y);
    ctx_free(ctx, acc);
}

template <typename C>
static void forms_run(gw_ctx* ctx, const C* fac, const C* linv, int n, int N, const double* Q, int R, double* cout,
                      const char* name, const char* const bnames[3], const int* kmap = nullptr, int nd = 0) {
    constexpr int NB = Tile<C>::NB, FT = Tile<C>::FT, LP = tile_pitch<C>();
    const int ny = kmap ? nd : N - 1;
    if (ny > 65535) gw_throw(GW_ERR_INVALID_ARG, "too many frequencies for the forms kernel");
    const size_t fixed = sizeof(C) * ((size_t)2 * FT * LP + 2 * NB * NB + 2 * NB);
    const size_t budget = 224 * 1024;
    // columns per CTA: at most 320 / FG threads, and Y [n][RC] must fit
    int rc_max = (int)std::min<size_t>(320 / FG, budget > fixed ? (budget - fixed) / (sizeof(C) * (size_t)n) : 0);
    // too few resident right-hand sides per CTA: Y in HBM instead
    if (rc_max < std::min(R, 48)) {
        forms_batched<C>(ctx, fac, linv, n, N, Q, R, cout, bnames, kmap, nd);
        return;
    }
    const int chunks = div_up(R, rc_max);
    const int RC = div_up(R, chunks);
    const size_t smem = fixed + std::max(sizeof(C) * (size_t)n * RC, sizeof(double) * FG * (size_t)RC);
    if (chunks > 65535) gw_throw(GW_ERR_INVALID_ARG, "too many right-hand sides for the forms kernel");
    allow_max_smem(k_forms<C, FG, FT>);
    klaunch(ctx, name, k_forms<C, FG, FT>, dim3(chunks, ny), FG * RC, smem, fac, linv, n, N, Q, R, RC, cout, kmap);
}

// Forms with dY in tensor memory: n <= 384 (three 128-lane tiles of an
// 80-column accumulator, 256 columns per CTA, two CTAs per SM).
static size_t forms_tm_smem() {
    return 2 * (size_t)TM_NS * TM_A_BYTES + 2 * (size_t)TM_B_BYTES +
           sizeof(float2) * ((size_t)32 * TM_RCP + 32 * TM_LIP + 32);
}

static bool forms_tm(gw_ctx* ctx, const gw_W* W, const double* Q, int R, double* cout) {
    const gw_chi0* c = W->chi0;
    const int n = c->n_sub, N = c->grid.n_omega;
    if (n <= 32 || n > 128 * TM_MAXT) return false;
    const int chunks = div_up(R, TM_RC);
    if (chunks > 65535 || N - 1 > 65535) return false;
    allow_max_smem(k_forms_tm);
    klaunch(ctx, "k_forms32_tm", k_forms_tm, dim3(chunks, N - 1), 256, forms_tm_smem(), (const float2*)W->fac32,
            (const float2*)W->linv, n, N, Q, R, cout, ctx->d_status);
    return true;
}

void launch_forms(gw_ctx* ctx, const gw_W* W, const double* Q, int R, double* cout) {
    const gw_chi0* c = W->chi0;
    const int n = c->n_sub, N = c->grid.n_omega;
    if (c->prec == GW_MIXED && !ctx->forms_simt && forms_tm(ctx, W, Q, R, cout)) return;
    static const char* const b32[3] = {"k_forms32_diag", "k_forms32_update", "k_forms32_gemm_tc"};
    static const char* const b64[3] = {"k_forms_diag", "k_forms_update", "k_forms_gemm_tc"};
    if (c->prec == GW_MIXED)
        forms_run<float2>(ctx, W->fac32, (const float2*)W->linv, n, N, Q, R, cout, "k_forms32", b32);
    else
        forms_run<double2>(ctx, W->fac, (const double2*)W->linv, n, N, Q, R, cout, "k_forms", b64);
}

// Binary64 factors of np frequencies of the binary32 path's chi0 (kd: device
// list, or the single frequency k1 when kd is null) into fac [np][tri(n)].
static void pole_factor(gw_ctx* ctx, const gw_W* W, const int* kd, int k1, int np, double2* fac, void* linv,
                        double* piv) {
    static const char* const nm[4] = {"k_ldlt_init", "k_ldlt_panel", "k_ldlt_syrk", "k_ldlt_syrk_tc"};
    const gw_chi0* c = W->chi0;
    const int n = c->n_sub;
    const long long pk = tri(n);
    double2* chi = dalloc<double2>(ctx, (size_t)np * pk);
    try {
        if (c->A64) {          // binary64 weights kept by the build: chi0_k in binary64
            const int band = c->nb_bins + 1;
            if (div_up(pk, 256) > 0x7fffffff || np > 65535)
                gw_throw(GW_ERR_INVALID_ARG, "near-pole batch too large");
            klaunch(ctx, "k_kk_band64", k_kk_band64, dim3(div_up(pk, 256), np), 256, sizeof(double2) * band,
                    (const double*)c->A64, band, pk, c->j_lo, c->grid.d_omega, c->grid.eta, kd, k1, chi);
        } else {
            klaunch(ctx, "k_gather_c128", k_gather_c128, div_up((long long)np * pk, 256), 256, 0,
                    (const float2*)c->chi0_32, kd, k1, np, pk, chi);
        }
        ldlt_steps<double2>(ctx, chi, fac, n, np, (double2*)linv, piv, nm);
    } catch (...) {
        ctx_free(ctx, chi);
        throw;
    }
    ctx_free(ctx, chi);
}

void launch_pole_forms(gw_ctx* ctx, const gw_W* W, const double* Q, int R, double* cout) {
    static const char* const b64[3] = {"k_forms_diag", "k_forms_update", "k_forms_gemm_tc"};
    const gw_chi0* c = W->chi0;
    const int n = c->n_sub, N = c->grid.n_omega, np = (int)W->pole_k.size();
    if (np == 0) return;
    const long long pk = tri(n);
    const size_t per = (size_t)pk * 2 * sizeof(double2) + ldlt_linv_bytes(n, 1, GW_FP64) + 2 * sizeof(double);
    const int nb = (int)std::max<size_t>(1, std::min<size_t>({(size_t)np, ((size_t)4 << 30) / per, (size_t)65535}));
    double2* fac = dalloc<double2>(ctx, (size_t)nb * pk);
    void* linv = nullptr;
    double* piv = nullptr;
    try {
        linv = ctx_alloc(ctx, ldlt_linv_bytes(n, nb, GW_FP64));
        piv = dalloc<double>(ctx, 2 * (size_t)nb);
        for (int b0 = 0; b0 < np; b0 += nb) {
            const int m = std::min(nb, np - b0);
            pole_factor(ctx, W, W->d_pole + b0, 0, m, fac, linv, piv);
            forms_run<double2>(ctx, fac, (const double2*)linv, n, N, Q, R, cout, "k_forms", b64, W->d_pole + b0, m);
        }
    } catch (...) {
        ctx_free(ctx, fac); ctx_free(ctx, linv); ctx_free(ctx, piv);
        throw;
    }
    ctx_free(ctx, fac); ctx_free(ctx, linv); ctx_free(ctx, piv);
}

void launch_ldlt_inverse(gw_ctx* ctx, const gw_W* W, int k, double2* out, double2* work) {
    const gw_chi0* c = W->chi0;
    const long long pk = tri(c->n_sub);
    const double2* F = W->fac ? W->fac + k * pk : work;
    if (!W->fac) {
        if (std::binary_search(W->pole_k.begin(), W->pole_k.end(), k)) {
            // a frequency the binary32 path refines: its binary64 factors
            void* linv = ctx_alloc(ctx, ldlt_linv_bytes(c->n_sub, 1, GW_FP64));
            double* piv = nullptr;
            try {
                piv = dalloc<double>(ctx, 2);
                pole_factor(ctx, W, nullptr, k, 1, work, linv, piv);
            } catch (...) {
                ctx_free(ctx, linv); ctx_free(ctx, piv);
                throw;
            }
            ctx_free(ctx, linv); ctx_free(ctx, piv);
        } else {
            klaunch(ctx, "k_c64_to_c128", k_c64_to_c128, div_up(pk, 256), 256, 0,
                    (const float2*)(W->fac32 + k * pk), work, pk);
        }
    }
    klaunch(ctx, "k_ldlt_inverse", k_ldlt_inverse, div_up(c->n_sub, 64), 64, 0, F, c->n_sub, out);
}
