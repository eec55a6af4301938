// a1: vertex products V^{EF}_mu = sum_{a,b in L(A)} X_aE V^mu_ab X_bF
// (Sec. 6.1; locality of Eq. VertexDefinition: V^mu vanishes outside the
// local orbitals L(A) of the atom pair set around the atom A that carries mu).
//
// One CTA per (product mu, chunk of FC states F).  The dense local block V^mu
// and the rows X[L(A), F-chunk] are staged in shared memory; the CTA forms
// T = V^mu X[L, F] once and contracts it with X[L, E] for every E chunk, so
// each product costs n_loc^2 nF + n_loc nE nF multiply-adds instead of
// n_loc^2 per (E, F) pair.  T is the arithmetic type: binary64, or binary32
// for the mixed path's pair vertices (inputs rounded once in shared memory).
#include "internal.h"

namespace {

constexpr int FC = 32;   // F states per CTA
constexpr int EC = 32;   // E states per inner chunk

template <typename T>
__global__ void __launch_bounds__(256) k_vertex_contract(
    const double* __restrict__ X, int n_orb, const double* __restrict__ vertex,
    const long long* __restrict__ voff, const int* __restrict__ prod_atom, const int* __restrict__ loc_ptr,
    const int* __restrict__ loc_idx, const int* __restrict__ Es, int nE, const int* __restrict__ Fs, int nF,
    const int* __restrict__ map, T* __restrict__ out, long long ld) {
    extern __shared__ __align__(16) unsigned char smraw[];
    T* sm = reinterpret_cast<T*>(smraw);
    const int mu = blockIdx.x;
    const int f0 = blockIdx.y * FC;
    const int A = prod_atom[mu];
    const int lb = loc_ptr[A];
    const int nl = loc_ptr[A + 1] - lb;
    const int fc = min(FC, nF - f0);
    T* sV = sm;                        // nl*nl
    T* sXf = sV + nl * nl;             // nl*FC
    T* sT = sXf + nl * FC;             // nl*FC
    T* sXe = sT + nl * FC;             // nl*EC
    const double* V = vertex + voff[mu];
    for (int i = threadIdx.x; i < nl * nl; i += blockDim.x) sV[i] = (T)V[i];
    for (int i = threadIdx.x; i < nl * FC; i += blockDim.x) {
        int a = i / FC, f = i % FC;
        sXf[i] = f < fc ? (T)X[(long long)loc_idx[lb + a] * n_orb + Fs[f0 + f]] : T(0);
    }
    __syncthreads();
    // T[a][f] = sum_b V[a][b] Xf[b][f]
    for (int i = threadIdx.x; i < nl * FC; i += blockDim.x) {
        int a = i / FC, f = i % FC;
        T s = T(0);
        for (int b = 0; b < nl; ++b) s = fma(sV[a * nl + b], sXf[b * FC + f], s);
        sT[i] = s;
    }
    for (int e0 = 0; e0 < nE; e0 += EC) {
        const int ec = min(EC, nE - e0);
        __syncthreads();
        for (int i = threadIdx.x; i < nl * EC; i += blockDim.x) {
            int a = i / EC, e = i % EC;
            sXe[i] = e < ec ? (T)X[(long long)loc_idx[lb + a] * n_orb + Es[e0 + e]] : T(0);
        }
        __syncthreads();
        for (int i = threadIdx.x; i < EC * FC; i += blockDim.x) {
            int e = i / FC, f = i % FC;
            if (e >= ec || f >= fc) continue;
            T s = T(0);
            for (int a = 0; a < nl; ++a) s = fma(sXe[a * EC + e], sT[a * FC + f], s);
            long long col = (long long)(e0 + e) * nF + (f0 + f);
            if (map) col = map[col];
            out[(long long)mu * ld + col] = s;
        }
    }
}

}  // namespace

template <typename T>
static void vertex_contract(gw_ctx* ctx, const char* name, const gw_mol* mol, const int* Es, int nE, const int* Fs,
                            int nF, const int* map, T* out, long long ld) {
    const int nl = mol->max_nloc;
    size_t smem = sizeof(T) * ((size_t)nl * nl + (size_t)nl * (2 * FC + EC));
    allow_max_smem(k_vertex_contract<T>);
    dim3 grid(mol->n_prod, div_up(nF, FC));
    klaunch(ctx, name, k_vertex_contract<T>, grid, 256, smem, mol->X, mol->n_orb, mol->vertex, mol->voff,
            mol->prod_atom, mol->loc_ptr, mol->loc_idx, Es, nE, Fs, nF, map, out, ld);
}

void launch_vertex_contract(gw_ctx* ctx, const gw_mol* mol, const int* Es, int nE, const int* Fs, int nF,
                            const int* map, double* out, long long ld) {
    vertex_contract<double>(ctx, "k_vertex_contract", mol, Es, nE, Fs, nF, map, out, ld);
}

void launch_vertex_contract32(gw_ctx* ctx, const gw_mol* mol, const int* Es, int nE, const int* Fs, int nF,
                              const int* map, float* out, long long ld) {
    vertex_contract<float>(ctx, "k_vertex_contract32", mol, Es, nE, Fs, nF, map, out, ld);
}
