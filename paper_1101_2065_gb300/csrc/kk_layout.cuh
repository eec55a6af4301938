// Operand images of the tensor-core Kramers-Kronig product (kk_tc.cu),
// shared with the deposit that writes the spectral weights in that form.
//
// An image is one 128 x 32 operand tile (rows = frequencies or packed
// elements, columns = 32 bins) in the canonical K-major core-matrix layout
// without swizzle, stored as TF32 hi parts (4096 words) followed by the lo
// parts (4096 words): exactly what the MMA reads from shared memory, so a
// stage is filled by one bulk copy per operand.  Weights are stored
// [bin chunk][element tile][image].
#pragma once
#include <cstdint>

#include "tc.cuh"

namespace kk {

constexpr int TM = 128;                       // rows: 64 frequencies x (Re, Im)
constexpr int TN = 128;                       // packed elements per tile
constexpr int KC = 32;                        // bins per chunk
constexpr int TILE_WORDS = TM * KC;           // one 128 x 32 tile (4096 words, 16 KB)
constexpr int OPER_WORDS = 2 * TILE_WORDS;    // hi + lo image (32 KB)

__device__ __forceinline__ uint32_t img_word(int r, int k) { return tc::core_off(r, k, KC / 4) >> 2; }

// word of (bin b of the band, packed element e) in the weight images
__device__ __forceinline__ long long weight_word(int b, long long e, long long n_et) {
    const int c = b / KC, k = b % KC;
    const long long et = e / TN;
    const int r = (int)(e % TN);
    return ((long long)c * n_et + et) * OPER_WORDS + img_word(r, k);
}

inline int chunks(int band) { return (band + KC - 1) / KC; }
inline long long elem_tiles(long long n_el) { return (n_el + TN - 1) / TN; }
inline size_t weight_words(int band, long long n_el) {
    return (size_t)chunks(band) * (size_t)elem_tiles(n_el) * OPER_WORDS;
}

}  // namespace kk
