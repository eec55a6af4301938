// a6-a8: spectral function of the diagonal self-energy, its Cauchy
// transform, the exchange part and the quasiparticle root.
//
// sigma_n(s) is the convolution of Eq. spectral_3 with the discrete
// spectral density of G0 (one delta per state): every form c_nk(s2) is
// shifted by E_k (virtual k: s = E_k + s2; occupied k: s = E_k - s2 with
// gamma_-(s2) = -gamma_+(-s2)) and deposited with tent weights on
// E_k/d_omega.  Each output bin gathers its contributions in state order
// (deterministic, no atomics).  Sigma_c(w) = d_omega sum_j sigma_j /
// (w - s_j + i eta sgn(s_j)) (Eq. Cauchy1, time ordering, sgn(0) = +1).
#include <cmath>

#include "internal.h"

namespace {

__global__ void __launch_bounds__(256) k_sigma_grid(const double* __restrict__ c, const double* __restrict__ eps,
                                                    int n_orb, int n_occ, int N, double dw, int j0, int n_sig,
                                                    int n_states, double* __restrict__ sig) {
    extern __shared__ double sm[];
    int* si = reinterpret_cast<int*>(sm + n_orb);
    double* sf = sm;
    for (int k = threadIdx.x; k < n_orb; k += blockDim.x) {
        double x = eps[k] / dw;
        double i = floor(x);
        si[k] = (int)i;
        sf[k] = x - i;
    }
    __syncthreads();
    long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= (long long)n_states * n_sig) return;
    int s = (int)(t / n_sig);
    int j = j0 + (int)(t % n_sig);
    const double* cs = c + (long long)s * n_orb * N;
    double acc = 0.0;
    for (int k = 0; k < n_orb; ++k) {
        const double* ck = cs + (long long)k * N;
        int ik = si[k];
        double f = sf[k];
        int t1, t2;
        if (k >= n_occ) { t1 = j - ik; t2 = j - ik - 1; }
        else { t1 = ik - j; t2 = ik + 1 - j; }
        if (t1 >= 0 && t1 < N) acc = fma(1.0 - f, ck[t1], acc);
        if (t2 >= 0 && t2 < N) acc = fma(f, ck[t2], acc);
    }
    sig[t] = acc;
}

// kernel table K[d - dmin] = 1/(d dw + i eta), d = k - j
__global__ void k_cauchy_table(double2* __restrict__ K, long long dmin, long long nd, double dw, double eta) {
    long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= nd) return;
    double x = (double)(dmin + t) * dw;
    double den = x * x + eta * eta;
    K[t] = make_double2(x / den, -eta / den);
}

// One warp per output point (binary64 runs at 1/64 rate: the sum over the
// sigma grid is spread over the lanes and all SMs, then reduced in a fixed
// order).
__global__ void __launch_bounds__(256) k_sigma_c(const double* __restrict__ sig, int n_sig, int j0, int N, double dw,
                                                 const double2* __restrict__ K, long long dmin, int n_states,
                                                 double2* __restrict__ out) {
    const long long t = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    const int nk = 2 * N - 1;
    if (t >= (long long)n_states * nk) return;
    const int s = (int)(t / nk);
    const int k = (int)(t % nk) - (N - 1);
    const double* sg = sig + (long long)s * n_sig;
    double re = 0.0, im = 0.0;
    for (int q = lane; q < n_sig; q += 32) {
        const int j = j0 + q;
        const double2 kv = K[(long long)(k - j) - dmin];
        const double v = sg[q];
        re = fma(v, kv.x, re);
        im = fma(v, j >= 0 ? kv.y : -kv.y, im);
    }
    for (int o = 16; o > 0; o >>= 1) {
        re += __shfl_xor_sync(0xffffffffu, re, o);
        im += __shfl_xor_sync(0xffffffffu, im, o);
    }
    if (lane == 0) out[t] = make_double2(dw * re, dw * im);
}

__device__ double block_sum(double v, double* red) {
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

// Sigma_x_n = -sum_{k occ} sum_mu V^{nk}_mu (v V^{nk})_mu, one CTA per state.
__global__ void __launch_bounds__(256) k_sigma_x(const double* __restrict__ Vnk, const double* __restrict__ T, int ld,
                                                 int n_prod, int n_orb, int n_occ, double* __restrict__ sx) {
    __shared__ double red[33];
    const int s = blockIdx.x;
    double acc = 0.0;
    for (long long t = threadIdx.x; t < (long long)n_prod * n_occ; t += blockDim.x) {
        int mu = (int)(t / n_occ), k = (int)(t % n_occ);
        long long o = (long long)mu * ld + (long long)s * n_orb + k;
        acc = fma(Vnk[o], T[o], acc);
    }
    acc = block_sum(acc, red);
    if (threadIdx.x == 0) sx[s] = -acc;
}

// Re Sigma_c(E) and d/dE (block-wide, deterministic).
__device__ void re_sigma(const double* __restrict__ sg, int n_sig, int j0, double dw, double eta, double E,
                         double* red, double& re, double& der) {
    double a = 0.0, b = 0.0;
    const double e2 = eta * eta;
    for (int q = threadIdx.x; q < n_sig; q += blockDim.x) {
        double x = E - (double)(j0 + q) * dw;
        double den = x * x + e2;
        double v = sg[q];
        a += v * x / den;
        b += v * (e2 - x * x) / (den * den);
    }
    re = dw * block_sum(a, red);
    der = dw * block_sum(b, red);
}

// The second window's sigma (large grid), when there is one.
struct Window2 {
    const double* sig;               // [n_states * n_sig] or null
    int n_sig, j0;
    double dw, eta;
};

// One CTA per state: linearised start, Newton, bracket scan + bisection.
// With a second window, Re Sigma_c and its derivative add the large
// window's Cauchy sum (the scan keeps the small window's step).
__global__ void __launch_bounds__(256) k_qp(const double* __restrict__ sig_, int n_sig, int j0, double dw, double eta,
                                            const double* __restrict__ eks, const double* __restrict__ sx,
                                            const double* __restrict__ vxc, double* __restrict__ e_out,
                                            double* __restrict__ z_out, int* __restrict__ st_out, Window2 w2) {
    __shared__ double red[33];
    const int s = blockIdx.x;
    const double* sg1 = sig_ + (long long)s * n_sig;
    const double* sg2 = w2.sig ? w2.sig + (long long)s * w2.n_sig : nullptr;
    auto re_sig = [&](double E, double& re, double& der) {
        re_sigma(sg1, n_sig, j0, dw, eta, E, red, re, der);
        if (sg2) {
            double re2, der2;
            re_sigma(sg2, w2.n_sig, w2.j0, w2.dw, w2.eta, E, red, re2, der2);
            re += re2;
            der += der2;
        }
    };
    const double e_ks = eks[s], sig_x = sx[s];
    const double v_xc = vxc ? vxc[s] : sig_x;
    double re, der;
    re_sig(e_ks, re, der);
    const double E1 = e_ks + (sig_x - v_xc + re) / (1.0 - der);
    double E = E1;
    bool ok = false;
    for (int it = 0; it < 100; ++it) {
        re_sig(E, re, der);
        double f = E - e_ks - sig_x + v_xc - re, df = 1.0 - der;
        if (!isfinite(f) || !isfinite(df) || df == 0.0) break;
        double step = f / df;
        E = E - step;
        if (fabs(E - E1) > 0.5) break;
        if (fabs(step) < 1e-11) { ok = true; break; }
    }
    int status = 0;
    if (!ok) {
        const int n = (int)floor(1.0 / dw);
        int best = -1;
        double bestd = 0.0, fprev = 0.0, xprev = 0.0, fbest = 0.0;
        for (int i = 0; i <= n; ++i) {
            double x = E1 - 0.5 + (double)i * dw;
            re_sig(x, re, der);
            double f = x - e_ks - sig_x + v_xc - re;
            if (i > 0 && (fprev == 0.0 || fprev * f < 0.0)) {
                double mid = 0.5 * (xprev + x);
                if (best < 0 || fabs(mid - E1) < bestd) { best = i - 1; bestd = fabs(mid - E1); fbest = fprev; }
            }
            fprev = f;
            xprev = x;
        }
        if (best < 0) { E = E1; status = 2; }
        else {
            double a = E1 - 0.5 + (double)best * dw, b = E1 - 0.5 + (double)(best + 1) * dw;
            double fa = fbest;
            if (fa == 0.0) b = a;
            for (int it = 0; it < 200; ++it) {
                if (b - a < 1e-11) break;
                double m = 0.5 * (a + b);
                re_sig(m, re, der);
                double fm = m - e_ks - sig_x + v_xc - re;
                if (((fm < 0.0) == (fa < 0.0)) && fm != 0.0) { a = m; fa = fm; }
                else b = m;
            }
            E = 0.5 * (a + b);
            status = 1;
        }
    }
    re_sig(E, re, der);
    if (threadIdx.x == 0) {
        e_out[s] = E;
        z_out[s] = 1.0 / (1.0 - der);
        st_out[s] = status;
    }
}

}  // namespace

void launch_sigma_grid(gw_ctx* ctx, gw_sigma* s) {
    const gw_chi0* c = s->W->chi0;
    const gw_mol* mol = c->mol;
    long long tot = (long long)s->n_states * s->n_sig;
    size_t smem = mol->n_orb * (sizeof(double) + sizeof(int));
    klaunch(ctx, "k_sigma_grid", k_sigma_grid, div_up(tot, 256), 256, smem, s->c, mol->eps, mol->n_orb, mol->n_occ,
                                                               c->grid.n_omega, c->grid.d_omega, s->j0, s->n_sig,
                                                               s->n_states, s->sig);
}

void launch_sigma_c(gw_ctx* ctx, gw_sigma* s) {
    const gw_chi0* c = s->W->chi0;
    const int N = c->grid.n_omega;
    // d = k - j, k in [-(N-1), N-1], j in [j0, j0 + n_sig - 1]
    long long dmin = -(long long)(N - 1) - (s->j0 + s->n_sig - 1);
    long long dmax = (long long)(N - 1) - s->j0;
    long long nd = dmax - dmin + 1;
    double2* K = dalloc<double2>(ctx, nd);
    klaunch(ctx, "k_cauchy_table", k_cauchy_table, div_up(nd, 256), 256, 0, K, dmin, nd, c->grid.d_omega, c->grid.eta);
    long long tot = (long long)s->n_states * (2 * N - 1) * 32;      // one warp per output
    klaunch(ctx, "k_sigma_c", k_sigma_c, div_up(tot, 256), 256, 0, s->sig, s->n_sig, s->j0, N, c->grid.d_omega, K, dmin,
                                                         s->n_states, s->sigc);
    ctx_free(ctx, K);
}

void launch_sigma_x(gw_ctx* ctx, gw_sigma* s, const double* Vnk, const double* T, int ld) {
    const gw_mol* mol = s->W->chi0->mol;
    klaunch(ctx, "k_sigma_x", k_sigma_x, s->n_states, 256, 0, Vnk, T, ld, mol->n_prod, mol->n_orb, mol->n_occ, s->sx);
}

void launch_qp(gw_ctx* ctx, const gw_sigma* s, const double* vxc, double* e, double* z, int* st) {
    const gw_chi0* c = s->W->chi0;
    Window2 w2{nullptr, 0, 0, 0.0, 0.0};
    if (s->W2) w2 = {s->sig2, s->n_sig2, s->j0_2, s->W2->chi0->grid.d_omega, s->W2->chi0->grid.eta};
    klaunch(ctx, "k_qp", k_qp, s->n_states, 256, 0, s->sig, s->n_sig, s->j0, c->grid.d_omega, c->grid.eta, s->eks, s->sx,
                                               vxc, e, z, st, w2);
}

// Second window: sigma of the large window's forms on the large grid.
void launch_sigma_grid2(gw_ctx* ctx, gw_sigma* s) {
    const gw_chi0* c = s->W2->chi0;
    const gw_mol* mol = c->mol;
    long long tot = (long long)s->n_states * s->n_sig2;
    size_t smem = mol->n_orb * (sizeof(double) + sizeof(int));
    klaunch(ctx, "k_sigma_grid", k_sigma_grid, div_up(tot, 256), 256, smem, s->c2, mol->eps, mol->n_orb, mol->n_occ,
            c->grid.n_omega, c->grid.d_omega, s->j0_2, s->n_sig2, s->n_states, s->sig2);
}

namespace {
// sigc[s][k] += dwl sum_j sig2_j / (w_k - s_j + i eta_l sgn(s_j)), w_k = k dws,
// s_j = (j0_2 + j) dwl: the large window's Cauchy sum at the small grid's
// points, one warp per output, direct divisions (Eq. Cauchy1, R7).
__global__ void __launch_bounds__(256) k_sigma_c2(const double* __restrict__ sig2, int n_sig2, int j0_2, double dwl,
                                                  double eta_l, int N, double dws, int n_states,
                                                  double2* __restrict__ out) {
    const long long t = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    const int nk = 2 * N - 1;
    if (t >= (long long)n_states * nk) return;
    const int st = (int)(t / nk);
    const double w = (double)((int)(t % nk) - (N - 1)) * dws;
    const double* sg = sig2 + (long long)st * n_sig2;
    double re = 0.0, im = 0.0;
    for (int q = lane; q < n_sig2; q += 32) {
        const int j = j0_2 + q;
        const double x = w - (double)j * dwl, e = j >= 0 ? eta_l : -eta_l;
        const double den = x * x + e * e, v = sg[q];
        re = fma(v, x / den, re);
        im = fma(v, -e / den, im);
    }
    for (int o = 16; o > 0; o >>= 1) {
        re += __shfl_xor_sync(0xffffffffu, re, o);
        im += __shfl_xor_sync(0xffffffffu, im, o);
    }
    if (lane == 0) {
        double2 v = out[t];
        out[t] = make_double2(v.x + dwl * re, v.y + dwl * im);
    }
}
}  // namespace

void launch_sigma_c2(gw_ctx* ctx, gw_sigma* s) {
    const gw_chi0* cs = s->W->chi0;
    const gw_chi0* cl = s->W2->chi0;
    const int N = cs->grid.n_omega;
    long long tot = (long long)s->n_states * (2 * N - 1) * 32;
    klaunch(ctx, "k_sigma_c2", k_sigma_c2, div_up(tot, 256), 256, 0, s->sig2, s->n_sig2, s->j0_2, cl->grid.d_omega,
            cl->grid.eta, N, cs->grid.d_omega, s->n_states, s->sigc);
}
