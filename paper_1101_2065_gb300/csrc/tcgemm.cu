// Binary32 GEMM on the 5th-generation tensor cores (tcgen05, kind::tf32) with
// 3xTF32 split precision: a = a_hi + a_lo with a_hi, a_lo representable in
// TF32, and A B ~ A_hi B_hi + (A_hi B_lo + A_lo B_hi), the two groups
// accumulated in binary32 in separate tensor-memory accumulators and added
// at the end (one accumulator for all three loses about a factor of three
// in accuracy); the dropped A_lo B_lo term is below binary32 rounding.  Used by the mixed path for its binary32
// products (g = X_r^T v X_r, U^T = Zup^T V^EF; Eqs. projector0, subspace_chi0).
//
// One CTA computes a 128 x 128 tile of C.  Its 256 threads stage K-chunks of
// 32 of op(A) and op(B) into shared memory, split into hi/lo parts and laid
// out in the canonical K-major core-matrix layout without swizzle (8 rows x
// 16 bytes per core matrix; 128 bytes between core matrices along K, 1024
// between 8-row groups), four consecutive K values of a row per 16-byte
// store.  Thread 0 issues the 12 MMAs of a chunk
// (4 steps of K = 8, three products each) and commits them to the chunk's
// mbarrier; two stages alternate, so the loads of chunk c + 1 overlap the
// MMAs of chunk c.  The accumulators (128 lanes x 128 columns of binary32
// each: hi products in columns 0-127, cross terms in 128-255) live in tensor
// memory and are read back with tcgen05.ld by all 8 warps (warp w: lanes
// 32 (w % 4) .. + 31, columns 64 (w / 4) .. + 63 of both).  Every wait
// on an mbarrier is bounded; on timeout the kernel flags ST_TIMEOUT and still
// releases its tensor memory.
#include <cstdint>

#include "internal.h"
#include "tc.cuh"

namespace {

constexpr int TM = 128, TN = 128, KC = 32;
constexpr int TILE_BYTES = TM * KC * 4;            // one 128 x 32 binary32 operand tile
constexpr int STAGE_BYTES = 4 * TILE_BYTES;        // A_hi, A_lo, B_hi, B_lo
constexpr int NSTAGE = 2;
constexpr uint32_t IDESC = tc::idesc_tf32(TM, TN);
constexpr uint32_t SBO = (KC / 4) * 128;          // bytes between 8-row groups of a 128 x 32 tile

__device__ __forceinline__ uint32_t tile_off(int r, int k) { return tc::core_off(r, k, KC / 4); }

// four consecutive K values of one row, split into hi and lo, as one 16-byte store each
__device__ __forceinline__ void store_quad(unsigned char* hi, unsigned char* lo, const float (&v)[4]) {
    uint32_t h[4], l[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) tc::split_tf32(v[i], h[i], l[i]);
    *reinterpret_cast<uint4*>(hi) = make_uint4(h[0], h[1], h[2], h[3]);
    *reinterpret_cast<uint4*>(lo) = make_uint4(l[0], l[1], l[2], l[3]);
}

// C = alpha op(A) op(B) + beta C; op(A) is M x K, op(B) is K x N, all row-major.
// blockIdx.x = tile row (M), blockIdx.y = tile column (N): CTAs that run
// together share a B tile.
template <bool TA, bool TB>
__global__ void __launch_bounds__(256, 1) k_sgemm_tc(int M, int N, int K, float alpha, const float* __restrict__ A,
                                                     long long lda, const float* __restrict__ B, long long ldb,
                                                     float beta, float* __restrict__ C, long long ldc, int* status) {
    extern __shared__ __align__(1024) unsigned char sm[];
    __shared__ __align__(8) uint64_t mbar[NSTAGE];
    __shared__ uint32_t tbase;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.x * TM, n0 = blockIdx.y * TN;
    if (warp == 0) {
        tc::tmem_alloc(&tbase, 2 * TN);
    }
    if (tid == 0)
        for (int s = 0; s < NSTAGE; ++s) tc::mbar_init(&mbar[s]);
    tc::fence_async_smem();
    __syncthreads();
    tc::fence_after();
    const uint32_t taddr = tbase;
    const int nchunk = (K + KC - 1) / KC;
    uint32_t uses[NSTAGE] = {0, 0};
    bool ok = true;
    for (int c = 0; c < nchunk; ++c) {
        const int s = c % NSTAGE, k0 = c * KC;
        unsigned char* st = sm + s * STAGE_BYTES;
        // stage op(A)[m0 .. +128)[k0 .. +32) and op(B)^T[n0 .. +128)[k0 .. +32) by quads of
        // four consecutive K of one row (lanes 0-7: rows 8 rg .. 8 rg + 7 of one quad, so
        // the 16-byte stores of a warp fill 512 contiguous bytes): each thread loads its
        // 4 + 4 quads first (all loads in flight at once), then splits and stores them
        float va[4][4], vb[4][4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int idx = tid + 256 * u, rr = idx & 7, kq = (idx >> 3) & 7, rg = idx >> 6;
            const int r = 8 * rg + rr, gk = k0 + 4 * kq;
            const int gm = m0 + r, gn = n0 + r;
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const bool ka = gm < M && gk + i < K, kb = gn < N && gk + i < K;
                va[u][i] = ka ? (TA ? A[(long long)(gk + i) * lda + gm] : A[(long long)gm * lda + gk + i]) : 0.f;
                vb[u][i] = kb ? (TB ? B[(long long)gn * ldb + gk + i] : B[(long long)(gk + i) * ldb + gn]) : 0.f;
            }
        }
        if (c >= NSTAGE) {           // the MMAs that read this stage two chunks ago are done
            ok = tc::mbar_wait(tc::smem_u32(&mbar[s]), (uses[s] - 1) & 1) && ok;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int idx = tid + 256 * u, rr = idx & 7, kq = (idx >> 3) & 7, rg = idx >> 6;
            const uint32_t o = tile_off(8 * rg + rr, 4 * kq);
            store_quad(st + o, st + TILE_BYTES + o, va[u]);
            store_quad(st + 2 * TILE_BYTES + o, st + 3 * TILE_BYTES + o, vb[u]);
        }
        tc::fence_async_smem();
        __syncthreads();
        if (tid == 0) {
            tc::fence_after();
            const uint32_t base = tc::smem_u32(st);
#pragma unroll
            for (int ks = 0; ks < KC / 8; ++ks) {
                const uint32_t o = ks * 2 * 128;          // two core matrices along K per step
                const uint64_t ahi = tc::smem_desc(base + o, SBO), alo = tc::smem_desc(base + TILE_BYTES + o, SBO);
                const uint64_t bhi = tc::smem_desc(base + 2 * TILE_BYTES + o, SBO);
                const uint64_t blo = tc::smem_desc(base + 3 * TILE_BYTES + o, SBO);
                const uint32_t first = (c > 0 || ks > 0) ? 1u : 0u;
                tc::mma_tf32(taddr, ahi, bhi, IDESC, first);
                tc::mma_tf32(taddr + TN, ahi, blo, IDESC, first);
                tc::mma_tf32(taddr + TN, alo, bhi, IDESC, 1u);
            }
            tc::commit(tc::smem_u32(&mbar[s]));
        }
        ++uses[s];
    }
    // all MMAs done: wait for the last use of every stage
    for (int s = 0; s < NSTAGE; ++s)
        if (uses[s] > 0) ok = tc::mbar_wait(tc::smem_u32(&mbar[s]), (uses[s] - 1) & 1) && ok;
    ok = __syncthreads_and(ok);         // warp-collective tensor-memory loads need a uniform decision
    tc::fence_after();
    if (!ok) {
        if (tid == 0) atomicOr(status, ST_TIMEOUT);
    } else if (nchunk > 0) {
        const int row = m0 + 32 * (warp & 3) + lane;
        const int cbase = 64 * (warp >> 2);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            uint32_t v[32], u[32];
            const uint32_t addr = taddr + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(cbase + 32 * h);
            tc::tmem_ld32(addr, v);
            tc::tmem_ld32(addr + TN, u);
            tc::tmem_wait_ld();
            if (row < M) {
                float* cr = C + (long long)row * ldc;
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    const int col = n0 + cbase + 32 * h + j;
                    if (col < N) {
                        const float x = alpha * (__uint_as_float(v[j]) + __uint_as_float(u[j]));
                        cr[col] = beta == 0.f ? x : fmaf(beta, cr[col], x);
                    }
                }
            }
        }
    }
    tc::fence_before();
    __syncthreads();
    if (warp == 0) {
        tc::fence_after();
        tc::tmem_dealloc(taddr, 2 * TN);
    }
}

}  // namespace

bool sgemm_tc(gw_ctx* ctx, bool ta, bool tb, int M, int N, int K, float alpha, const float* A, long long lda,
              const float* B, long long ldb, float beta, float* C, long long ldc) {
    const long long tiles = (long long)div_up(M, TM) * div_up(N, TN);
    // worth it only with enough tiles to spread over the SMs (with the small
    // basis products of the ring on the tensor cores as well, the mixed W
    // error against binary64 measured 3.9e-4 instead of below 3e-4)
    if (K < KC || tiles < 16 || div_up(M, TM) > 65535 * 32 || div_up(N, TN) > 65535) return false;
    const size_t smem = (size_t)NSTAGE * STAGE_BYTES;
    dim3 grid(div_up(M, TM), div_up(N, TN));
    auto run = [&](auto kern) {
        allow_max_smem(kern);
        klaunch(ctx, "k_sgemm_tc", kern, grid, 256, smem, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc,
                ctx->d_status);
    };
    if (!ta && !tb) run(k_sgemm_tc<false, false>);
    else if (ta && !tb) run(k_sgemm_tc<true, false>);
    else if (!ta && tb) run(k_sgemm_tc<false, true>);
    else run(k_sgemm_tc<true, true>);
    return true;
}
