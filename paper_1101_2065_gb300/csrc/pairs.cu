// a0: electron-hole pair table sorted by (Delta, E, F) with tent bins.
//
// Pairs (E occupied, F virtual) are ordered by Delta = eps_F - eps_E as in
// Eq. subsetof_vef (the compression takes the pairs of smallest |E - F|);
// ties break by (E, F).  Delta >= 0, so the IEEE bit pattern of Delta orders
// like the value and the key is an integer comparison: the rank of a pair is
// the number of pairs with a smaller (bits(Delta), natural index) key.  Each
// pair then carries the tent bin j = floor(Delta/d_omega) and the fraction
// f = Delta/d_omega - j of the deposit.
#include "internal.h"

namespace {

__global__ void k_pair_keys(const double* __restrict__ eps, int n_occ, int n_virt,
                            unsigned long long* __restrict__ key, double* __restrict__ delta) {
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n_occ * n_virt) return;
    int E = p / n_virt, F = n_occ + p % n_virt;
    double d = eps[F] - eps[E];
    delta[p] = d;
    key[p] = (unsigned long long)__double_as_longlong(d);
}

// rank[p] = #{q : (key[q], q) < (key[p], p)}; keys staged through shared memory.
__global__ void k_pair_rank(const unsigned long long* __restrict__ key, int n, int* __restrict__ rank) {
    __shared__ unsigned long long sk[1024];
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long kp = p < n ? key[p] : 0ull;
    int r = 0;
    for (int base = 0; base < n; base += 1024) {
        int m = min(1024, n - base);
        __syncthreads();
        for (int i = threadIdx.x; i < m; i += blockDim.x) sk[i] = key[base + i];
        __syncthreads();
        if (p < n) {
            for (int i = 0; i < m; ++i) {
                unsigned long long kq = sk[i];
                int q = base + i;
                r += (kq < kp) || (kq == kp && q < p);
            }
        }
    }
    if (p < n) rank[p] = r;
}

__global__ void k_pair_scatter(const int* __restrict__ rank, const double* __restrict__ delta, int n_occ,
                               int n_virt, double d_omega, int* __restrict__ sE, int* __restrict__ sF,
                               double* __restrict__ sDelta, int* __restrict__ sBin, double* __restrict__ sFrac) {
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n_occ * n_virt) return;
    int s = rank[p];
    double d = delta[p];
    double x = d / d_omega;
    double j = floor(x);
    sE[s] = p / n_virt;
    sF[s] = n_occ + p % n_virt;
    sDelta[s] = d;
    sBin[s] = (int)j;
    sFrac[s] = x - j;
}

// seg[b] = first sorted pair with bin >= j_lo + b, b = 0..nb_bins; seg[nb_bins] = n.
__global__ void k_pair_segments(const int* __restrict__ sBin, int n, int j_lo, int nb_bins, int* __restrict__ seg,
                                int* __restrict__ status) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s > n) return;
    int b = s < n ? sBin[s] - j_lo : nb_bins;
    int prev = s > 0 ? sBin[s - 1] - j_lo : -1;
    if (b < 0 || b > nb_bins || prev < -1 || prev > b) {
        atomicOr(status, ST_BOUNDS);
        return;
    }
    for (int q = prev + 1; q <= b; ++q) seg[q] = s;
}

__global__ void k_invert_perm(const int* __restrict__ sE, const int* __restrict__ sF, int n, int n_occ,
                              int n_virt, int* __restrict__ rank_of) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    rank_of[sE[s] * n_virt + (sF[s] - n_occ)] = s;
}

}  // namespace

void launch_pair_table(gw_ctx* ctx, const gw_mol* mol, gw_chi0* c) {
    const int n_occ = mol->n_occ, n_virt = mol->n_orb - mol->n_occ, n = c->n_pair;
    unsigned long long* key = dalloc<unsigned long long>(ctx, n);
    double* delta = dalloc<double>(ctx, n);
    int* rank = dalloc<int>(ctx, n);
    c->pE = dalloc<int>(ctx, n); c->pF = dalloc<int>(ctx, n); c->pBin = dalloc<int>(ctx, n);
    c->pDelta = dalloc<double>(ctx, n); c->pFrac = dalloc<double>(ctx, n);
    c->seg = dalloc<int>(ctx, c->nb_bins + 1);
    const int T = 256;
    klaunch(ctx, "k_pair_keys", k_pair_keys, div_up(n, T), T, 0, mol->eps, n_occ, n_virt, key, delta);
    klaunch(ctx, "k_pair_rank", k_pair_rank, div_up(n, T), T, 0, key, n, rank);
    klaunch(ctx, "k_pair_scatter", k_pair_scatter, div_up(n, T), T, 0, rank, delta, n_occ, n_virt, c->grid.d_omega, c->pE, c->pF,
                                                         c->pDelta, c->pBin, c->pFrac);
    klaunch(ctx, "k_pair_segments", k_pair_segments, div_up(n + 1, T), T, 0, c->pBin, n, c->j_lo, c->nb_bins, c->seg, ctx->d_status);
    ctx_free(ctx, key); ctx_free(ctx, delta); ctx_free(ctx, rank);
}

void launch_invert_perm(gw_ctx* ctx, const gw_chi0* c, int* rank_of) {
    const int n = c->n_pair;
    const gw_mol* mol = c->mol;
    klaunch(ctx, "k_invert_perm", k_invert_perm, div_up(n, 256), 256, 0, c->pE, c->pF, n, mol->n_occ, mol->n_orb - mol->n_occ, rank_of);
}
