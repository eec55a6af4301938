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
// between 8-row groups).  Thread 0 issues the 12 MMAs of a chunk
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

namespace {

constexpr int TM = 128, TN = 128, KC = 32;
constexpr int TILE_BYTES = TM * KC * 4;            // one 128 x 32 binary32 operand tile
constexpr int STAGE_BYTES = 4 * TILE_BYTES;        // A_hi, A_lo, B_hi, B_lo
constexpr int NSTAGE = 2;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared memory matrix descriptor: start address, leading (K) and stride
// (8-row group) byte offsets, descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
    constexpr uint32_t LBO = 128, SBO = 1024;
    uint64_t d = (uint64_t)((addr & 0x3FFFF) >> 4);
    d |= (uint64_t)((LBO >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((SBO >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// instruction descriptor: D binary32, A and B TF32, both K-major, N = 128, M = 128
constexpr uint32_t IDESC = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(TN >> 3) << 17) | ((uint32_t)(TM >> 4) << 24);

// byte offset of element (r, k) of a 128 x 32 tile
__device__ __forceinline__ uint32_t tile_off(int r, int k) {
    return (uint32_t)((((r >> 3) * (KC / 4) + (k >> 2)) * 128) + (r & 7) * 16 + (k & 3) * 4);
}

__device__ __forceinline__ void split_tf32(float a, uint32_t& hi, uint32_t& lo) {
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(hi) : "f"(a));
    const float r = a - __uint_as_float(hi);
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(lo) : "f"(r));
}

__device__ __forceinline__ void mma_tf32(uint32_t taddr, uint64_t da, uint64_t db, uint32_t acc) {
    asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                 " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}"
                 ::"r"(taddr), "l"(da), "l"(db), "r"(IDESC), "r"(acc));
}

// 32 consecutive tensor-memory columns of this warp's 32 lanes into v
__device__ __forceinline__ void tmem_ld32(uint32_t addr, uint32_t (&v)[32]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,"
                 "%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                 : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                   "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
                   "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]),
                   "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]),
                   "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
                 : "r"(addr));
}

// bounded wait for the given parity of an mbarrier; false on timeout
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity) {
    for (long it = 0; it < (1L << 24); ++it) {
        uint32_t done;
        asm volatile("{\n .reg .pred P;\n mbarrier.try_wait.parity.shared::cta.b64 P, [%1], %2;\n"
                     " selp.u32 %0, 1, 0, P;\n}" : "=r"(done) : "r"(mbar), "r"(parity) : "memory");
        if (done) return true;
    }
    return false;
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
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tbase)),
                     "r"((uint32_t)(2 * TN)));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0)
        for (int s = 0; s < NSTAGE; ++s) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[s])));
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t taddr = tbase;
    const int nchunk = (K + KC - 1) / KC;
    uint32_t uses[NSTAGE] = {0, 0};
    bool ok = true;
    for (int c = 0; c < nchunk; ++c) {
        const int s = c % NSTAGE, k0 = c * KC;
        unsigned char* st = sm + s * STAGE_BYTES;
        if (c >= NSTAGE) {           // the MMAs that read this stage two chunks ago are done
            ok = mbar_wait(smem_u32(&mbar[s]), (uses[s] - 1) & 1) && ok;
        }
        // stage op(A)[m0 .. +128)[k0 .. +32) and op(B)^T[n0 .. +128)[k0 .. +32)
        for (int t = tid; t < TM * KC; t += blockDim.x) {
            int r, k;
            if (TA) { k = t / TM; r = t % TM; } else { r = t / KC; k = t % KC; }
            const int gm = m0 + r, gk = k0 + k;
            const float a = (gm < M && gk < K) ? (TA ? A[(long long)gk * lda + gm] : A[(long long)gm * lda + gk]) : 0.f;
            uint32_t hi, lo;
            split_tf32(a, hi, lo);
            *reinterpret_cast<uint32_t*>(st + tile_off(r, k)) = hi;
            *reinterpret_cast<uint32_t*>(st + TILE_BYTES + tile_off(r, k)) = lo;
        }
        for (int t = tid; t < TN * KC; t += blockDim.x) {
            int r, k;
            if (TB) { r = t / KC; k = t % KC; } else { k = t / TN; r = t % TN; }
            const int gn = n0 + r, gk = k0 + k;
            const float b = (gn < N && gk < K) ? (TB ? B[(long long)gn * ldb + gk] : B[(long long)gk * ldb + gn]) : 0.f;
            uint32_t hi, lo;
            split_tf32(b, hi, lo);
            *reinterpret_cast<uint32_t*>(st + 2 * TILE_BYTES + tile_off(r, k)) = hi;
            *reinterpret_cast<uint32_t*>(st + 3 * TILE_BYTES + tile_off(r, k)) = lo;
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t base = smem_u32(st);
#pragma unroll
            for (int ks = 0; ks < KC / 8; ++ks) {
                const uint32_t o = ks * 2 * 128;          // two core matrices along K per step
                const uint64_t ahi = smem_desc(base + o), alo = smem_desc(base + TILE_BYTES + o);
                const uint64_t bhi = smem_desc(base + 2 * TILE_BYTES + o), blo = smem_desc(base + 3 * TILE_BYTES + o);
                const uint32_t first = (c > 0 || ks > 0) ? 1u : 0u;
                mma_tf32(taddr, ahi, bhi, first);
                mma_tf32(taddr + TN, ahi, blo, first);
                mma_tf32(taddr + TN, alo, bhi, 1u);
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                         ::"r"(smem_u32(&mbar[s])) : "memory");
        }
        ++uses[s];
    }
    // all MMAs done: wait for the last use of every stage
    for (int s = 0; s < NSTAGE; ++s)
        if (uses[s] > 0) ok = mbar_wait(smem_u32(&mbar[s]), (uses[s] - 1) & 1) && ok;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (!ok) {
        if (tid == 0) atomicOr(status, ST_TIMEOUT);
    } else if (nchunk > 0) {
        const int row = m0 + 32 * (warp & 3) + lane;
        const int cbase = 64 * (warp >> 2);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            uint32_t v[32], u[32];
            const uint32_t addr = taddr + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(cbase + 32 * h);
            tmem_ld32(addr, v);
            tmem_ld32(addr + TN, u);
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
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
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"((uint32_t)(2 * TN)));
    }
}

}  // namespace

bool sgemm_tc(gw_ctx* ctx, bool ta, bool tb, int M, int N, int K, float alpha, const float* A, long long lda,
              const float* B, long long ldb, float beta, float* C, long long ldc) {
    const long long tiles = (long long)div_up(M, TM) * div_up(N, TN);
    // worth it only with enough tiles to spread over the SMs
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
