// Self-energy as a matrix over a set of states and Dyson's equation with the
// density of states (Sec. 3, Eqs. tensorform-self-energy, tensorform-dyson,
// instantaneous; the Kohn-Sham basis is orthonormal, so the overlap is 1).
//
// Off-diagonal forms.  For the pair of states (n, m) and every state k,
// q_nk^T M^-1 q_mk with M = 1 - chi0 complex symmetric follows from three
// quadratic forms (polarisation):
//   q_n^T M^-1 q_m = ( (q_n+q_m)^T M^-1 (q_n+q_m) - q_n^T M^-1 q_n - q_m^T M^-1 q_m ) / 2,
// so the forms kernels of the diagonal self-energy run unchanged on the
// right-hand sides q_nk (n = m) and q_nk + q_mk (n < m), and a flat pass
// turns the latter into c_nm,k.  Pairs are stored n <= m, row-major upper
// triangle: p(n, m) = n S - n(n-1)/2 + m - n.
//
// Dyson's equation on the grid w_k = k d_omega, |k| < N: one thread per
// frequency builds A = (w + i eta - E_n) delta_nm - Sigma_c,nm(w) - (Sigma_x -
// vxc)_nm (S <= 16 states), inverts it by Gauss-Jordan elimination with
// partial pivoting in binary64, and sums -(1/pi) Im G_nn; the states outside
// the set add their non-interacting Lorentzians.
#include <cmath>

#include "internal.h"

namespace {

__host__ __device__ inline int pair_index(int n, int m, int S) { return n * S - n * (n - 1) / 2 + (m - n); }

// Qp[:, p n_orb + k] = q_nk (+ q_mk if n != m); Q [n_sub][S n_orb], Qp [n_sub][P n_orb]
__global__ void k_pair_rhs(const double* __restrict__ Q, int S, int n_orb, int n_sub, double* __restrict__ Qp) {
    const int P = S * (S + 1) / 2;
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const long long Rp = (long long)P * n_orb;
    if (t >= (long long)n_sub * Rp) return;
    const int row = (int)(t / Rp);
    const int col = (int)(t % Rp), p = col / n_orb, k = col % n_orb;
    int n = 0;
    while (pair_index(n, S - 1, S) < p) ++n;       // pair p lies in row n of the triangle
    const int m = n + (p - pair_index(n, n, S));
    const double* q = Q + (long long)row * S * n_orb;
    Qp[t] = q[n * n_orb + k] + (m != n ? q[m * n_orb + k] : 0.0);
}

// c[p(n,m)] = (c[p(n,m)] - c[p(n,n)] - c[p(m,m)]) / 2 for n < m; c [P n_orb][N]
__global__ void k_offdiag(double* __restrict__ c, int S, int n_orb, int N) {
    const int P = S * (S + 1) / 2;
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const long long per = (long long)n_orb * N;
    if (t >= (long long)P * per) return;
    const int p = (int)(t / per);
    const long long r = t % per;
    int n = 0;
    while (pair_index(n, S - 1, S) < p) ++n;
    const int m = n + (p - pair_index(n, n, S));
    if (m == n) return;
    const double a = c[(long long)pair_index(n, n, S) * per + r], b = c[(long long)pair_index(m, m, S) * per + r];
    c[t] = 0.5 * (c[t] - a - b);
}

// Sigma_x,nm = -sum_{k occ} sum_mu V^{nk}_mu (v V^{mk})_mu, one CTA per pair
__global__ void __launch_bounds__(256) k_sigma_x_pairs(const double* __restrict__ Vnk, const double* __restrict__ T,
                                                       int ld, int n_prod, int n_orb, int n_occ, int S,
                                                       double* __restrict__ sx) {
    __shared__ double red[256];
    const int p = blockIdx.x;
    int n = 0;
    while (pair_index(n, S - 1, S) < p) ++n;
    const int m = n + (p - pair_index(n, n, S));
    double acc = 0.0;
    for (long long t = threadIdx.x; t < (long long)n_prod * n_occ; t += blockDim.x) {
        const int mu = (int)(t / n_occ), k = (int)(t % n_occ);
        acc = fma(Vnk[(long long)mu * ld + n * n_orb + k], T[(long long)mu * ld + m * n_orb + k], acc);
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) sx[p] = -red[0];
}

constexpr int SMAX = 16;

// dos[k] = -(1/pi) Im Tr G(w_k + i eta); g[i][k] = G_ii for the states of the set
__global__ void __launch_bounds__(64) k_dyson(const double2* __restrict__ sigc, const double* __restrict__ sx_minus_vxc,
                                              const double* __restrict__ eps, const int* __restrict__ states, int S,
                                              int n_orb, int N, double dw, double eta, double* __restrict__ dos,
                                              double2* __restrict__ g) {
    const int nk = 2 * N - 1;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nk) return;
    const double w = (double)(k - (N - 1)) * dw;
    double2 A[SMAX][SMAX], B[SMAX][SMAX];
    for (int i = 0; i < S; ++i)
        for (int j = 0; j < S; ++j) {
            const int a = i < j ? i : j, b = i < j ? j : i;
            const int p = pair_index(a, b, S);
            const double2 sc = sigc[(long long)p * nk + k];
            A[i][j] = make_double2(-sc.x - sx_minus_vxc[p], -sc.y);
            B[i][j] = make_double2(i == j ? 1.0 : 0.0, 0.0);
        }
    for (int i = 0; i < S; ++i) {
        A[i][i].x += w - eps[states[i]];
        A[i][i].y += eta;
    }
    // Gauss-Jordan with partial pivoting: A^-1 into B
    for (int col = 0; col < S; ++col) {
        int piv = col;
        double best = A[col][col].x * A[col][col].x + A[col][col].y * A[col][col].y;
        for (int r = col + 1; r < S; ++r) {
            const double v = A[r][col].x * A[r][col].x + A[r][col].y * A[r][col].y;
            if (v > best) { best = v; piv = r; }
        }
        if (piv != col)
            for (int j = 0; j < S; ++j) {
                double2 t = A[col][j]; A[col][j] = A[piv][j]; A[piv][j] = t;
                t = B[col][j]; B[col][j] = B[piv][j]; B[piv][j] = t;
            }
        const double2 d = A[col][col];
        const double inv = 1.0 / (d.x * d.x + d.y * d.y);
        const double2 r = make_double2(d.x * inv, -d.y * inv);       // 1 / d
        for (int j = 0; j < S; ++j) {
            A[col][j] = cmul(A[col][j], r);
            B[col][j] = cmul(B[col][j], r);
        }
        for (int i = 0; i < S; ++i) {
            if (i == col) continue;
            const double2 f = A[i][col];
            for (int j = 0; j < S; ++j) {
                A[i][j] = csub(A[i][j], cmul(f, A[col][j]));
                B[i][j] = csub(B[i][j], cmul(f, B[col][j]));
            }
        }
    }
    double im = 0.0;
    for (int i = 0; i < S; ++i) {
        im += B[i][i].y;
        if (g) g[(long long)i * nk + k] = B[i][i];
    }
    // states outside the set: non-interacting, Im 1/(w + i eta - E) = -eta / ((w - E)^2 + eta^2)
    for (int q = 0; q < n_orb; ++q) {
        bool active = false;
        for (int i = 0; i < S; ++i) active = active || states[i] == q;
        if (active) continue;
        const double x = w - eps[q];
        im += -eta / (x * x + eta * eta);
    }
    dos[k] = -im / M_PI;
}

}  // namespace

int dyson_max_states() { return SMAX; }

void launch_pair_rhs(gw_ctx* ctx, const double* Q, int S, int n_orb, int n_sub, double* Qp) {
    const long long tot = (long long)n_sub * (S * (S + 1) / 2) * n_orb;
    klaunch(ctx, "k_pair_rhs", k_pair_rhs, div_up(tot, 256), 256, 0, Q, S, n_orb, n_sub, Qp);
}

void launch_offdiag(gw_ctx* ctx, double* c, int S, int n_orb, int N) {
    const long long tot = (long long)(S * (S + 1) / 2) * n_orb * N;
    klaunch(ctx, "k_offdiag", k_offdiag, div_up(tot, 256), 256, 0, c, S, n_orb, N);
}

void launch_sigma_x_pairs(gw_ctx* ctx, const gw_sigma* s, const double* Vnk, const double* T, int ld) {
    const gw_mol* mol = s->W->chi0->mol;
    const int S = s->matrix_S;
    klaunch(ctx, "k_sigma_x", k_sigma_x_pairs, S * (S + 1) / 2, 256, 0, Vnk, T, ld, mol->n_prod, mol->n_orb,
            mol->n_occ, S, s->sx);
}

void launch_dyson(gw_ctx* ctx, const gw_sigma* s, const double* sx_minus_vxc, const int* states, double* dos,
                  double2* g) {
    const gw_chi0* c = s->W->chi0;
    const int N = c->grid.n_omega;
    klaunch(ctx, "k_dyson", k_dyson, div_up(2 * N - 1, 64), 64, 0, (const double2*)s->sigc, sx_minus_vxc,
            (const double*)c->mol->eps, states, s->matrix_S, c->mol->n_orb, N, c->grid.d_omega, c->grid.eta, dos,
            g);
}
