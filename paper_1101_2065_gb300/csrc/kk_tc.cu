// a4 on the binary32 path: the Cauchy (Kramers-Kronig) transform of the
// spectral weights as a product on the 5th-generation tensor cores.
//
// Eq. chi_by_spectra on the grid (readings R1-R3):
//   chi0_k[e] = sum_{j in band} A_j[e] K(k, j),
//   K(k, j)   = kap(k - j) - kap(k + j),  kap(d) = 1/(d dw + i eta),
// for every packed element e of the compressed response.  The weights A_j
// are nonzero only on the band of bins j_lo .. j_lo + nb_bins (the pair
// transitions), so the sum is a product of a [2 N_omega x band] kernel
// matrix (row 2k = Re K(k, .), row 2k+1 = Im K(k, .)) with the [band x n_el]
// weights: a dense contraction with a short K dimension (the band, ~200
// bins), written once as chi0 [N_omega][n_el] complex binary32.
//
// Precision.  A binary32 FFT spreads its rounding evenly over all
// frequencies (relative to the whole sequence), and 1 - chi0 amplifies it by
// its condition number near the RPA poles; the direct band sum keeps each
// chi0_k accurate relative to its own terms.  Both operands are split into
// TF32 hi + lo parts (3xTF32: hi.hi into one accumulator, hi.lo + lo.hi into
// a second); the band is taken in chunks of 32 bins whose partial sums are
// read back from tensor memory and added in registers, so no binary32
// accumulator runs over more than one chunk.
//
// Operands.  The kernel matrix is tabulated once per call in binary64,
// split and stored in the exact shared-memory image of each (frequency
// tile, bin chunk) operand tile (canonical K-major core-matrix layout, no
// swizzle); the deposit writes the weights pre-split in the same per-tile
// image.  Each stage of the pipeline is therefore two 32 KB bulk copies
// (cp.async.bulk on the TMA unit, completion counted on an mbarrier):
// no thread touches an operand value.
//
// Tile.  One CTA computes 64 frequencies (128 rows: Re and Im interleaved)
// x 128 packed elements.  Thread 0 issues the 12 MMAs of a chunk
// (M = 128, N = 128, K = 8; 4 steps x 3 products) into one of two tensor-
// memory accumulator sets and commits them to the chunk's mbarrier; while
// they run, all 8 warps read back the previous chunk's set (tcgen05.ld) and
// add it to their register sums, and thread 0 starts the bulk copies of the
// next chunk.  The result tile is transposed through shared memory (Re/Im
// pairs exchanged between neighbouring lanes) and written as 1 KB rows.
// Every mbarrier wait is bounded; on a timeout the CTA flags ST_TIMEOUT,
// waits for what it issued and still releases its tensor memory.
#include <algorithm>
#include <cstdint>

#include "internal.h"
#include "kk_layout.cuh"
#include "tc.cuh"

namespace {

using namespace kk;
constexpr int STAGE_BYTES = 2 * OPER_WORDS * 4;   // kernel matrix + weights (64 KB)
constexpr int NSTAGE = 2;
// all 512 tensor-memory columns: a second CTA of the kernel never fits beside the first (228 KB per SM)
static_assert(NSTAGE * STAGE_BYTES <= 227 * 1024 - 1024 && 2 * NSTAGE * STAGE_BYTES > 228 * 1024,
              "tensor-core Cauchy sum: one CTA per SM");
constexpr uint32_t IDESC = tc::idesc_tf32(TM, TN);
constexpr uint32_t SBO = (KC / 4) * 128;      // bytes between 8-row groups
constexpr int OUT_LD = 266;                   // words per staged output row (128 complex + padding)

__device__ __forceinline__ void split_store(uint32_t* img, int r, int k, double x) {
    uint32_t hi, lo;
    tc::split_tf32(__double2float_rn(x), hi, lo);
    const float rem = (float)(x - (double)__uint_as_float(hi));
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(lo) : "f"(rem));
    img[img_word(r, k)] = hi;
    img[TILE_WORDS + img_word(r, k)] = lo;
}

// Kernel matrix image: table[(mt * nch + c) * OPER_WORDS + ...], row r of
// frequency tile mt is frequency 64 mt + r/2 (Re for even r, Im for odd),
// column k of chunk c is bin j_lo + 32 c + k.  Rows beyond the grid and
// bins beyond the band are zero.
__global__ void k_kk_table(int N, int j_lo, int band, int nch, double dw, double eta, long long total,
                           uint32_t* __restrict__ table) {
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= total) return;
    const int k = (int)(t % KC);
    const int r = (int)((t / KC) % TM);
    const long long tc_ = t / (KC * TM);              // mt * nch + c
    const int c = (int)(tc_ % nch);
    const int mt = (int)(tc_ / nch);
    const int row = mt * TM + r, freq = row >> 1, b = c * KC + k;
    double v = 0.0;
    if (freq < N && b < band) {
        const long long j = j_lo + b;
        const double x1 = (double)(freq - j) * dw, x2 = (double)(freq + j) * dw, e2 = eta * eta;
        const double d1 = x1 * x1 + e2, d2 = x2 * x2 + e2;
        v = (row & 1) ? (-eta / d1 + eta / d2) : (x1 / d1 - x2 / d2);
    }
    split_store(table + tc_ * OPER_WORDS, r, k, v);
}

__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t mbar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(dst), "l"(src), "r"(bytes), "r"(mbar) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t mbar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"(bytes) : "memory");
}

// chi0[k][e] for frequency tiles x packed-element tiles; see the file header.
__global__ void __launch_bounds__(256, 1) k_chi0_kk_tc(const uint32_t* __restrict__ table,
                                                        const uint32_t* __restrict__ Asplit, int N, long long n_el,
                                                        int n_mt, long long n_et, int nch, float2* __restrict__ chi0,
                                                        int* status) {
    extern __shared__ __align__(1024) unsigned char sm[];
    __shared__ __align__(8) uint64_t full[NSTAGE], done[NSTAGE];
    __shared__ uint32_t tbase;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (warp == 0) tc::tmem_alloc(&tbase, 512);
    if (tid == 0)
        for (int s = 0; s < NSTAGE; ++s) {
            tc::mbar_init(&full[s]);
            tc::mbar_init(&done[s]);
        }
    tc::fence_async_smem();
    __syncthreads();
    tc::fence_after();
    const uint32_t taddr = tbase;
    const uint32_t sbase = tc::smem_u32(sm);
    uint32_t n_full[NSTAGE] = {0, 0}, n_done[NSTAGE] = {0, 0};   // phases waited for (all threads)
    // thread 0's record of what it issued and saw complete, for the clean-up after a timeout
    uint32_t issued[NSTAGE] = {0, 0}, full_ok[NSTAGE] = {0, 0}, committed[NSTAGE] = {0, 0}, done_ok[NSTAGE] = {0, 0};
    bool ok = true;
    const int q = warp & 3, h = warp >> 2;          // tensor-memory lane quarter, column half
    const long long n_tiles = (long long)n_mt * n_et;
    for (long long tile = blockIdx.x; tile < n_tiles && ok; tile += gridDim.x) {
        const int mt = (int)(tile % n_mt);
        const long long et = tile / n_mt;
        const uint32_t* tab = table + (long long)mt * nch * OPER_WORDS;
        auto issue = [&](int c) {           // thread 0: both operand images of chunk c into stage c & 1
            const int s = c & 1;
            const uint32_t st = sbase + s * STAGE_BYTES, mb = tc::smem_u32(&full[s]);
            mbar_expect_tx(mb, STAGE_BYTES);
            bulk_g2s(st, tab + (long long)c * OPER_WORDS, OPER_WORDS * 4, mb);
            bulk_g2s(st + OPER_WORDS * 4, Asplit + ((long long)c * n_et + et) * OPER_WORDS, OPER_WORDS * 4, mb);
            ++issued[s];
        };
        float sum[64];
#pragma unroll
        for (int j = 0; j < 64; ++j) sum[j] = 0.f;
        auto readback = [&](int c) {        // all threads: add chunk c's accumulators (set c & 1)
            const uint32_t set = (uint32_t)(c & 1) * 256;
            const uint32_t row = (uint32_t)(32 * q) << 16;
#pragma unroll
            for (int part = 0; part < 2; ++part) {
                uint32_t v[32], u[32];
                const uint32_t col = set + 64 * h + 32 * part;
                tc::tmem_ld32(taddr + row + col, v);
                tc::tmem_ld32(taddr + row + col + TN, u);
                tc::tmem_wait_ld();
#pragma unroll
                for (int j = 0; j < 32; ++j) sum[32 * part + j] += __uint_as_float(v[j]) + __uint_as_float(u[j]);
            }
        };
        if (tid == 0) {
            issue(0);
            if (nch > 1) issue(1);
        }
        for (int c = 0; c < nch; ++c) {
            const int s = c & 1;
            if (tid == 0) {
                bool got = tc::mbar_wait(tc::smem_u32(&full[s]), n_full[s] & 1);
                if (got) {
                    ++full_ok[s];
                    tc::fence_after();
                    const uint32_t st = sbase + s * STAGE_BYTES, acc = taddr + (uint32_t)s * 256;
#pragma unroll
                    for (int ks = 0; ks < KC / 8; ++ks) {
                        const uint32_t o = ks * 2 * 128;
                        const uint64_t ahi = tc::smem_desc(st + o, SBO);
                        const uint64_t alo = tc::smem_desc(st + TILE_WORDS * 4 + o, SBO);
                        const uint64_t bhi = tc::smem_desc(st + OPER_WORDS * 4 + o, SBO);
                        const uint64_t blo = tc::smem_desc(st + OPER_WORDS * 4 + TILE_WORDS * 4 + o, SBO);
                        const uint32_t accum = ks > 0 ? 1u : 0u;
                        tc::mma_tf32(acc, ahi, bhi, IDESC, accum);
                        tc::mma_tf32(acc + TN, ahi, blo, IDESC, accum);
                        tc::mma_tf32(acc + TN, alo, bhi, IDESC, 1u);
                    }
                }
                // commit even without MMAs so that the done barrier always completes its phase
                tc::commit(tc::smem_u32(&done[s]));
                ++committed[s];
                ok = got && ok;
            }
            ++n_full[s];
            if (c >= 1) {
                const int sp = (c - 1) & 1;
                const bool d = tc::mbar_wait(tc::smem_u32(&done[sp]), n_done[sp] & 1);
                ++n_done[sp];
                if (d) ++done_ok[sp];
                ok = __syncthreads_and(d && ok);
                tc::fence_after();
                if (!ok) break;
                readback(c - 1);
                tc::fence_before();
                __syncthreads();           // set (c-1) & 1 and stage (c-1) & 1 are free again
                if (tid == 0 && c + 1 < nch) issue(c + 1);
            }
        }
        ok = __syncthreads_and(ok);          // thread 0 may have seen the last chunk's copies time out
        if (ok) {
            const int sl = (nch - 1) & 1;
            const bool d = tc::mbar_wait(tc::smem_u32(&done[sl]), n_done[sl] & 1);
            ++n_done[sl];
            if (d) ++done_ok[sl];
            ok = __syncthreads_and(d && ok);
            tc::fence_after();
            if (ok) readback(nch - 1);
        }
        if (!ok) break;
        // epilogue: lane pairs (Re, Im) of one frequency exchange halves; row f of the
        // staged tile holds 128 complex values (padding: one complex every 32)
        float* out = reinterpret_cast<float*>(sm);
        const int f = 16 * q + (lane >> 1);
        const bool re = (lane & 1) == 0;
#pragma unroll
        for (int j = 0; j < 32; ++j) {
            const float send = re ? sum[32 + j] : sum[j];
            const float got = __shfl_xor_sync(0xffffffffu, send, 1);
            const int col = 64 * h + (re ? j : 32 + j);
            const int w = f * OUT_LD + 2 * (col + (col >> 5));
            if (re) { out[w] = sum[j]; out[w + 1] = got; }
            else { out[w] = got; out[w + 1] = sum[32 + j]; }
        }
        __syncthreads();
        const long long e0 = et * TN;
        const int ne = (int)((n_el - e0) < TN ? (n_el - e0) : TN);
        for (int rr = warp; rr < 64; rr += 8) {
            const int k = mt * 64 + rr;
            if (k >= N) break;
            float2* dst = chi0 + (long long)k * n_el + e0;
            for (int col = lane; col < ne; col += 32) {
                const int w = rr * OUT_LD + 2 * (col + (col >> 5));
                dst[col] = make_float2(out[w], out[w + 1]);
            }
        }
        tc::fence_async_smem();             // generic accesses before the next tile's bulk copies
        __syncthreads();                    // the staging area is the next tile's stage 0
    }
    if (!ok) {
        if (tid == 0) {
            atomicOr(status, ST_TIMEOUT);
            // let the copies and MMAs this CTA issued finish (phases in order, bounded)
            for (int s = 0; s < NSTAGE; ++s) {
                for (uint32_t p = full_ok[s]; p < issued[s]; ++p)
                    if (!tc::mbar_wait(tc::smem_u32(&full[s]), p & 1)) break;
                for (uint32_t p = done_ok[s]; p < committed[s]; ++p)
                    if (!tc::mbar_wait(tc::smem_u32(&done[s]), p & 1)) break;
            }
        }
        __syncthreads();
    }
    tc::fence_before();
    __syncthreads();
    if (warp == 0) {
        tc::fence_after();
        tc::tmem_dealloc(taddr, 512);
    }
}

}  // namespace

void launch_chi0_kk_tc(gw_ctx* ctx, gw_chi0* c, const uint32_t* Asplit) {
    const int N = c->grid.n_omega, band = c->nb_bins + 1, nch = kk::chunks(band);
    const long long n_el = tri(c->n_sub);
    const int n_mt = div_up(2LL * N, TM);
    const long long n_et = kk::elem_tiles(n_el);
    uint32_t* table = dalloc<uint32_t>(ctx, (size_t)n_mt * nch * OPER_WORDS);
    try {
        const long long tot = (long long)n_mt * nch * TM * KC;
        klaunch(ctx, "k_kk_table", k_kk_table, div_up(tot, 256), 256, 0, N, c->j_lo, band, nch, c->grid.d_omega,
                c->grid.eta, tot, table);
        if (!c->chi0_32) c->chi0_32 = dalloc<float2>(ctx, (size_t)N * n_el);
        const long long n_tiles = (long long)n_mt * n_et;
        const int grid = (int)std::min<long long>(n_tiles, 64LL * ctx->num_sms);
        allow_max_smem(k_chi0_kk_tc);
        klaunch(ctx, "k_chi0_kk_tc", k_chi0_kk_tc, grid, 256, (size_t)NSTAGE * STAGE_BYTES, (const uint32_t*)table,
                Asplit, N, n_el, n_mt, n_et, nch, c->chi0_32, ctx->d_status);
    } catch (...) {
        ctx_free(ctx, table);
        throw;
    }
    ctx_free(ctx, table);
}

// ----------------------------------------------------------------------
// The same band sum on the binary32 FMA units (the binary32 path's
// default).  Its additions round to nearest, so the rounding errors of
// chi0 carry no common sign; the tensor cores' binary32 accumulation
// leaves a systematic shrink of a few 1e-8 in every element, which
// 1 - chi0 amplifies near the RPA poles into W errors above 1e-5.
//
// One CTA computes 64 frequencies x 128 packed elements from plain
// A[band][n_el] weights and a binary32 kernel table Kc[b][k] (complex).
// Thread (ty, tx) of 8 x 32 owns frequencies 8 ty .. + 7 and elements
// 4 tx .. + 3: per bin 8 complex kernel values (broadcast reads) and one
// 16-byte weight read feed 64 FMAs.  The bins are taken in chunks of 32
// staged in shared memory; each chunk is summed into its own registers
// and then added to the running totals.
namespace {

constexpr int FK = 64, FE = 128, FB = 32;

__global__ void k_kk_ctable(int N, int j_lo, int band, double dw, double eta, float2* __restrict__ Kc) {
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= (long long)N * band) return;
    const int b = (int)(t / N), k = (int)(t % N);             // Kc[b][k], bin-major
    const long long j = j_lo + b;
    const double x1 = (double)(k - j) * dw, x2 = (double)(k + j) * dw, e2 = eta * eta;
    const double d1 = x1 * x1 + e2, d2 = x2 * x2 + e2;
    Kc[t] = make_float2((float)(x1 / d1 - x2 / d2), (float)(-eta / d1 + eta / d2));
}

// asynchronous copies into shared memory: `bytes` of src (0 = zero fill) into a dst slot of `size`
__device__ __forceinline__ void cp_async_z8(void* dst, const void* src, int bytes) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(d), "l"(src), "r"(bytes) : "memory");
}
__device__ __forceinline__ void cp_async_z16(void* dst, const void* src, int bytes) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(src), "r"(bytes) : "memory");
}
__device__ __forceinline__ void cp_async_z4(void* dst, const void* src, int bytes) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(d), "l"(src), "r"(bytes) : "memory");
}

constexpr size_t KKF_SMEM = 2 * (sizeof(float2) * FB * FK + sizeof(float) * FB * FE);

// The chunks of FB bins go through two shared-memory buffers: chunk c + 1 is
// copied asynchronously while chunk c is summed.
__global__ void __launch_bounds__(256) k_chi0_kk_fma(const float2* __restrict__ Kc, const float* __restrict__ A,
                                                     int N, int band, long long n_el, float2* __restrict__ chi0) {
    extern __shared__ __align__(16) unsigned char sraw_kf[];
    float2 (*sK)[FB][FK] = reinterpret_cast<float2 (*)[FB][FK]>(sraw_kf);                       // [2][bin][frequency]
    float (*sA)[FB][FE] = reinterpret_cast<float (*)[FB][FE]>(sraw_kf + 2 * sizeof(float2) * FB * FK);  // [2][bin][element]
    const int tid = threadIdx.x, ty = tid >> 5, tx = tid & 31;
    const int k0 = blockIdx.y * FK;
    const long long e0 = (long long)blockIdx.x * FE;
    float tr[8][4], ti[8][4];
#pragma unroll
    for (int f = 0; f < 8; ++f)
#pragma unroll
        for (int i = 0; i < 4; ++i) tr[f][i] = ti[f][i] = 0.f;
    const bool vec = (n_el % 4 == 0);
    const int nch = (band + FB - 1) / FB;
    auto stage = [&](int ch, int buf) {
        const int b0 = ch * FB;
        for (int t = tid; t < FB * FK; t += 256) {
            const int f = t % FK, bb = t / FK, k = k0 + f, b = b0 + bb;
            const bool in = k < N && b < band;
            cp_async_z8(&sK[buf][bb][f], in ? (const void*)(Kc + (long long)b * N + k) : (const void*)Kc, in ? 8 : 0);
        }
        for (int t = tid; t < FB * FE / 4; t += 256) {
            const int bb = t / (FE / 4), q = t % (FE / 4), b = b0 + bb;
            const long long e = e0 + 4 * q;
            const float* row = A + (long long)(b < band ? b : 0) * n_el;
            if (vec) {
                const int nb = (b < band && e < n_el) ? 16 : 0;       // n_el % 4 == 0: whole quads
                cp_async_z16(&sA[buf][bb][4 * q], nb ? (const void*)(row + e) : (const void*)A, nb);
            } else {
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const bool in = b < band && e + u < n_el;
                    cp_async_z4(&sA[buf][bb][4 * q + u], in ? (const void*)(row + e + u) : (const void*)A, in ? 4 : 0);
                }
            }
        }
        asm volatile("cp.async.commit_group;\n" ::: "memory");
    };
    stage(0, 0);
    for (int ch = 0; ch < nch; ++ch) {
        const int buf = ch & 1;
        if (ch + 1 < nch) {
            stage(ch + 1, buf ^ 1);
            asm volatile("cp.async.wait_group 1;\n" ::: "memory");
        } else {
            asm volatile("cp.async.wait_group 0;\n" ::: "memory");
        }
        __syncthreads();
        float pr[8][4], pi[8][4];
#pragma unroll
        for (int f = 0; f < 8; ++f)
#pragma unroll
            for (int i = 0; i < 4; ++i) pr[f][i] = pi[f][i] = 0.f;
#pragma unroll 4
        for (int bb = 0; bb < FB; ++bb) {
            const float4 a = *reinterpret_cast<const float4*>(&sA[buf][bb][4 * tx]);
            const float av[4] = {a.x, a.y, a.z, a.w};
            const float4* kp = reinterpret_cast<const float4*>(&sK[buf][bb][8 * ty]);
#pragma unroll
            for (int f2 = 0; f2 < 4; ++f2) {
                const float4 kk2 = kp[f2];                            // frequencies 2 f2, 2 f2 + 1
                const float2 kvs[2] = {make_float2(kk2.x, kk2.y), make_float2(kk2.z, kk2.w)};
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int f = 2 * f2 + h;
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        pr[f][i] = fmaf(kvs[h].x, av[i], pr[f][i]);
                        pi[f][i] = fmaf(kvs[h].y, av[i], pi[f][i]);
                    }
                }
            }
        }
#pragma unroll
        for (int f = 0; f < 8; ++f)
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                tr[f][i] += pr[f][i];
                ti[f][i] += pi[f][i];
            }
        __syncthreads();                              // buffer buf is refilled by the next iteration's copies
    }
#pragma unroll
    for (int f = 0; f < 8; ++f) {
        const int k = k0 + 8 * ty + f;
        if (k >= N) break;
        float2* row = chi0 + (long long)k * n_el;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const long long e = e0 + 4 * tx + i;
            if (e < n_el) row[e] = make_float2(tr[f][i], ti[f][i]);
        }
    }
}

}  // namespace

// ----------------------------------------------------------------------
// Second window technique (Sec. 4.2, Eq. win2-for-response): chi0 on the
// small window's grid w_k = k dws takes the small window's bins (s = j dws,
// broadening eta_s) and the large window's truncated bins (s = j dwl,
// broadening eta_l) in one band sum: the kernel table holds both blocks of
// rows, the weights both blocks of bins.
namespace {

template <typename C>
__global__ void k_kk_ctable_2w(int N, double dws, int js, int band_s, double eta_s, double dwl, int jl, int band_l,
                               double eta_l, C* __restrict__ Kc) {
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const int band = band_s + band_l;
    if (t >= (long long)N * band) return;
    const int b = (int)(t / N), k = (int)(t % N);
    const double w = (double)k * dws;
    const double sb = b < band_s ? (double)(js + b) * dws : (double)(jl + b - band_s) * dwl;
    const double eta = b < band_s ? eta_s : eta_l;
    const double x1 = w - sb, x2 = w + sb, e2 = eta * eta;
    const double d1 = x1 * x1 + e2, d2 = x2 * x2 + e2;
    const double re = x1 / d1 - x2 / d2, im = -eta / d1 + eta / d2;
    if constexpr (sizeof(C) == 8) Kc[t] = make_float2((float)re, (float)im);
    else Kc[t] = make_double2(re, im);
}

// binary64 band sum chi0[k][e] = sum_b A[b][e] Kc[b][k]: one thread per
// element, the CTA's frequency row of the table in shared memory.
__global__ void __launch_bounds__(256) k_chi0_kk64(const double2* __restrict__ Kc, const double* __restrict__ A,
                                                   int N, int band, long long n_el, double2* __restrict__ chi0) {
    extern __shared__ double2 krow[];
    const int k = blockIdx.y;
    for (int b = threadIdx.x; b < band; b += blockDim.x) krow[b] = Kc[(long long)b * N + k];
    __syncthreads();
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n_el) return;
    double re = 0.0, im = 0.0;
    for (int b = 0; b < band; ++b) {
        const double a = A[(long long)b * n_el + e];
        re = fma(a, krow[b].x, re);
        im = fma(a, krow[b].y, im);
    }
    chi0[(long long)k * n_el + e] = make_double2(re, im);
}

}  // namespace

void launch_chi0_kk_2w(gw_ctx* ctx, gw_chi0* c, const void* A, int js, int band_s, int jl, int band_l,
                       const gw_grid& gl) {
    const int N = c->grid.n_omega, band = band_s + band_l;
    const long long n_el = tri(c->n_sub);
    const bool f32 = c->prec == GW_MIXED;
    void* Kc = ctx_alloc(ctx, (size_t)N * band * (f32 ? sizeof(float2) : sizeof(double2)));
    try {
        const int nb = div_up((long long)N * band, 256);
        if (f32) {
            klaunch(ctx, "k_kk_ctable", k_kk_ctable_2w<float2>, nb, 256, 0, N, c->grid.d_omega, js, band_s,
                    c->grid.eta, gl.d_omega, jl, band_l, gl.eta, (float2*)Kc);
            if (!c->chi0_32) c->chi0_32 = dalloc<float2>(ctx, (size_t)N * n_el);
            const long long net = (n_el + FE - 1) / FE;
            allow_max_smem(k_chi0_kk_fma);
            klaunch(ctx, "k_chi0_kk_fma", k_chi0_kk_fma, dim3((unsigned)net, (unsigned)div_up(N, FK)), 256, KKF_SMEM,
                    (const float2*)Kc, (const float*)A, N, band, n_el, c->chi0_32);
        } else {
            klaunch(ctx, "k_kk_ctable", k_kk_ctable_2w<double2>, nb, 256, 0, N, c->grid.d_omega, js, band_s,
                    c->grid.eta, gl.d_omega, jl, band_l, gl.eta, (double2*)Kc);
            if (!c->chi0) c->chi0 = dalloc<double2>(ctx, (size_t)N * n_el);
            if ((size_t)band * sizeof(double2) > 48 * 1024) gw_throw(GW_ERR_INVALID_ARG, "spectral band too wide");
            klaunch(ctx, "k_chi0_kk64", k_chi0_kk64, dim3((unsigned)div_up(n_el, 256), (unsigned)N), 256,
                    sizeof(double2) * band, (const double2*)Kc, (const double*)A, N, band, n_el, c->chi0);
        }
    } catch (...) {
        ctx_free(ctx, Kc);
        throw;
    }
    ctx_free(ctx, Kc);
}

void launch_chi0_kk_fma(gw_ctx* ctx, gw_chi0* c, const float* A) {
    const int N = c->grid.n_omega, band = c->nb_bins + 1;
    const long long n_el = tri(c->n_sub);
    float2* Kc = dalloc<float2>(ctx, (size_t)N * band);
    try {
        klaunch(ctx, "k_kk_ctable", k_kk_ctable, div_up((long long)N * band, 256), 256, 0, N, c->j_lo, band,
                c->grid.d_omega, c->grid.eta, Kc);
        if (!c->chi0_32) c->chi0_32 = dalloc<float2>(ctx, (size_t)N * n_el);
        const long long net = (n_el + FE - 1) / FE;
        if (net > 0x7fffffffLL) gw_throw(GW_ERR_INVALID_ARG, "too many matrix elements for the Kramers-Kronig kernel");
        dim3 grid((unsigned)net, (unsigned)div_up(N, FK));
        allow_max_smem(k_chi0_kk_fma);
        klaunch(ctx, "k_chi0_kk_fma", k_chi0_kk_fma, grid, 256, KKF_SMEM, (const float2*)Kc, A, N, band, n_el, c->chi0_32);
    } catch (...) {
        ctx_free(ctx, Kc);
        throw;
    }
    ctx_free(ctx, Kc);
}
