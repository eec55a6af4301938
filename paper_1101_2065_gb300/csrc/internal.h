// Internal declarations of the GW library: context, handles, launchers.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <string>
#include <unordered_map>
#include <vector>

#include "gw.h"

// ------------------------------------------------------------------ status
// Bits of the per-context device status word.  Kernels set them with
// atomicOr; the host reads the word at the end of every API call.
enum : int {
    ST_NOT_SPD = 1,
    ST_SINGULAR = 2,
    ST_RANK = 4,
    ST_NONFINITE = 8,
    ST_BOUNDS = 16,
    ST_TIMEOUT = 32,
};

struct GwError {
    gw_status code;
    std::string msg;
};

struct ProfRec {
    const char* name;
    cudaEvent_t start, stop;
};

struct gw_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    size_t budget = 0;
    size_t in_use = 0;
    size_t peak = 0;
    long long launches = 0;
    std::string err;
    std::unordered_map<void*, size_t> blocks;
    int* d_status = nullptr;
    int* h_status = nullptr;
    int num_sms = 0;
    bool forms_simt = false;         // GW_OPT_FORMS_SIMT
    bool syrk_simt = false;          // GW_OPT_SYRK_SIMT
    bool gemm_simt = false;          // GW_OPT_GEMM_SIMT
    bool kk_tensor = false;          // GW_OPT_KK_TENSOR
    int poles_permille = 0;          // GW_OPT_POLES_FP64 (0 = off)
    int barrier_polls = 0;           // GW_OPT_BARRIER_POLLS (0 = default limit)
    // optional CUDA-event timing of kernel launches whose name matches prof_filter
    bool prof_on = false;
    std::string prof_filter;
    cudaEvent_t prof_pending = nullptr;     // start event recorded by prof_begin
    std::vector<ProfRec> prof_recs;
    std::vector<cudaEvent_t> prof_pool;
    std::unordered_map<std::string, std::pair<double, long long>> prof_acc;
};

// Throws GwError; every extern "C" entry point catches and converts.
void gw_throw(gw_status code, const std::string& msg);
void cuda_check(cudaError_t e, const char* what);
#define CUDA_CHECK(x) cuda_check((x), #x)

void* ctx_alloc(gw_ctx* ctx, size_t bytes);
void ctx_free(gw_ctx* ctx, void* p);
template <class T>
T* dalloc(gw_ctx* ctx, size_t n) { return static_cast<T*>(ctx_alloc(ctx, n * sizeof(T))); }

// Counts a launch, checks the launch error and, when profiling is on,
// closes the timing interval opened by prof_begin.
void after_launch(gw_ctx* ctx, const char* name);
void prof_begin(gw_ctx* ctx, const char* name);
#define LAUNCH_CHECK(ctx, name) after_launch((ctx), (name))

// Allow a kernel the device's full dynamic shared memory, once per process.
// (The attribute is process-wide: setting per-call sizes from concurrent
// host threads would race.)
void allow_max_smem_impl(const void* func);
template <typename... KArgs>
inline void allow_max_smem(void (*kernel)(KArgs...)) { allow_max_smem_impl((const void*)kernel); }

// Launch a kernel on the context stream with launch accounting.
template <typename... KArgs, typename... Args>
inline void klaunch(gw_ctx* ctx, const char* name, void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                    Args... args) {
    prof_begin(ctx, name);
    kernel<<<grid, block, smem, ctx->stream>>>(args...);
    after_launch(ctx, name);
}

// Synchronise the context stream and convert status bits into an error.
void ctx_finish(gw_ctx* ctx, const char* where);

// ------------------------------------------------------------------ handles
struct gw_mol {
    gw_ctx* ctx = nullptr;
    int n_atoms = 0, n_orb = 0, n_occ = 0, n_prod = 0, n_sub = 0;
    int max_nloc = 0;
    std::vector<double> h_eps;       // host copy (validation of the grid)
    double* eps = nullptr;           // [n_orb]
    double* X = nullptr;             // [n_orb*n_orb] X[a*n_orb+E]
    double* vertex = nullptr;
    long long* voff = nullptr;       // [n_prod+1]
    double* v = nullptr;             // [n_prod*n_prod]
    double* Z = nullptr;             // optional [n_prod*n_sub]
    int* prod_atom = nullptr;        // [n_prod]
    int* loc_ptr = nullptr;          // [n_atoms+1]
    int* loc_idx = nullptr;          // local orbital lists
    size_t vertex_len = 0;
};

struct gw_chi0 {
    gw_ctx* ctx = nullptr;
    const gw_mol* mol = nullptr;
    gw_grid grid{};
    gw_precision prec = GW_FP64;
    int n_pair = 0, n_rank = 0, n_sub = 0;
    int j_lo = 0, j_hi = 0;          // band of nonzero spectral bins (inclusive)
    int nb_bins = 0;                 // number of pair bins j_lo..j_lo+nb_bins-1
    int L = 0, logL = 0;             // FFT length 2*n_omega
    // pair table (sorted)
    int* pE = nullptr; int* pF = nullptr; int* pBin = nullptr;
    double* pDelta = nullptr; double* pFrac = nullptr;
    int* seg = nullptr;              // [nb_bins+1]
    double* Z = nullptr;             // [n_prod*n_sub] (nullptr for Cholesky basis; formed on first read-back)
    double* Xr = nullptr;            // [n_prod*n_rank] and [n_rank*n_sub]: Z = Xr Bsel, kept for the read-back
    double* Bsel = nullptr;
    double* Zup = nullptr;           // [n_prod*n_sub]
    double* Ut = nullptr;            // [n_sub*n_pair] U transposed
    double2* tw = nullptr;           // [L/2] exp(-2 pi i k/L) (binary64 FFT)
    double2* C1 = nullptr;           // [L] FFT of the Toeplitz kernel
    double2* C2 = nullptr;           // [L] FFT of the Hankel kernel
    double2* chi0 = nullptr;         // [n_omega*n_sub*n_sub], lower triangle valid
    // mixed precision copies
    float* Ut32 = nullptr;
    float2* chi0_32 = nullptr;       // [n_omega][tri(n_sub)] binary32 path
    double* A64 = nullptr;           // [band][tri(n_sub)] binary64 weights (binary32 path, near-pole policy)
    // second window technique: the small window's handle refers to the large one's
    const gw_chi0* large = nullptr;  // set on the small window's handle
    double lam_cut = 0.0;            // spectral arguments below it belong to the small window
};

struct gw_W {
    gw_ctx* ctx = nullptr;
    const gw_chi0* chi0 = nullptr;
    double2* fac = nullptr;          // [n_omega*n*n] strict lower L, diagonal D
    float2* fac32 = nullptr;
    void* linv = nullptr;            // [n_omega][panels][NB][NB] inverses of the unit lower diagonal blocks
    double* piv = nullptr;           // [n_omega] min|d| / max|M|
    double min_pivot_ratio = 0.0;
    // binary32 path, near-pole policy: frequencies (ascending) whose factorisation
    // and forms are redone in binary64 where they are consumed
    std::vector<int> pole_k;
    int* d_pole = nullptr;
};

struct gw_sigma {
    gw_ctx* ctx = nullptr;
    const gw_W* W = nullptr;
    int n_states = 0, R = 0;
    std::vector<int> states;
    int j0 = 0, n_sig = 0;
    double* c = nullptr;             // [R*n_omega]
    double* sig = nullptr;           // [n_states*n_sig]
    double2* sigc = nullptr;         // [n_states*(2N-1)]
    double* sx = nullptr;            // [n_states]
    double* eks = nullptr;           // [n_states]
    // second window technique: the large window's forms and sigma (W2 = its factors)
    const gw_W* W2 = nullptr;
    int j0_2 = 0, n_sig2 = 0;
    double* c2 = nullptr;            // [R*n_omega_large]
    double* sig2 = nullptr;          // [n_states*n_sig2]
    // self-energy matrix over matrix_S states (Dyson's equation): the rows of
    // c, sig, sigc and sx are the pairs n <= m, n_states = S(S+1)/2 of them
    int matrix_S = 0;
    int* d_states = nullptr;         // [matrix_S]
};

// ------------------------------------------------------------------ launchers
// pairs.cu
void launch_pair_table(gw_ctx* ctx, const gw_mol* mol, gw_chi0* c);
void launch_invert_perm(gw_ctx* ctx, const gw_chi0* c, int* rank_of);
// vertex.cu: out[mu*ld + col(e,f)] = sum_ab X[L_a,Es[e]] V^mu_ab X[L_b,Fs[f]],
// col(e,f) = map ? map[e*nF+f] : e*nF+f
void launch_vertex_contract(gw_ctx* ctx, const gw_mol* mol, const int* Es, int nE,
                            const int* Fs, int nF, const int* map, double* out, long long ld);
void launch_vertex_contract32(gw_ctx* ctx, const gw_mol* mol, const int* Es, int nE, const int* Fs, int nF,
                              const int* map, float* out, long long ld);
// gemm.cu: C = alpha*op(A) op(B) + beta*C, row-major, batched by stride.
void gemm_f64(gw_ctx* ctx, bool ta, bool tb, int M, int N, int K, double alpha,
              const double* A, long long lda, const double* B, long long ldb, double beta,
              double* C, long long ldc, int batch = 1, long long sA = 0, long long sB = 0,
              long long sC = 0);
// linalg.cu
void cholesky_lower(gw_ctx* ctx, double* A, int n);          // in place, zeroes upper
// eigh.cu: B = xi lambda^-1/2 for the n_sub largest eigenpairs of g
void eigh_top_scaled(gw_ctx* ctx, const double* g, const float* g32, int n, int n_sub, int oa_iters, double oa_tol,
                     bool vectors_f64, double* B);
void basis_rayleigh_scale(gw_ctx* ctx, double* Z, double* Zup, int rows, int n_sub);
std::vector<float> eigvals32(gw_ctx* ctx, const double* g, const float* g32, int n);   // ascending
// chi0.cu
void launch_fft_tables(gw_ctx* ctx, gw_chi0* c);
void launch_chi0_fft(gw_ctx* ctx, gw_chi0* c);           // binary64: deposit + FFT
void launch_chi0_kk32(gw_ctx* ctx, gw_chi0* c);          // binary32: deposit + Cauchy sum
void launch_spectral64(gw_ctx* ctx, gw_chi0* c);         // binary64 weights A64 from c->Ut
void launch_deposit_range(gw_ctx* ctx, const gw_chi0* c, const int* seg, const double* frac, int nb_bins, void* A);
// second window: chi0 of c (small window grid) from [small bins; large bins] weights A
void launch_chi0_kk_2w(gw_ctx* ctx, gw_chi0* c, const void* A, int js, int band_s, int jl, int band_l,
                       const gw_grid& gl);
// kk_tc.cu: chi0_32 from the TF32 hi/lo weight images (kk_layout.cuh)
void launch_chi0_kk_tc(gw_ctx* ctx, gw_chi0* c, const uint32_t* Asplit);
void launch_chi0_kk_fma(gw_ctx* ctx, gw_chi0* c, const float* A);   // A[band][n_el]
void launch_spectral_readback(gw_ctx* ctx, const gw_chi0* c, int j0, int nj, double* A);
void launch_to_f32(gw_ctx* ctx, const double* a, float* b, long long n);
void launch_to_f64(gw_ctx* ctx, const float* a, double* b, long long n);
void launch_f64_to_f32_2d(gw_ctx* ctx, const double* a, long long lda, int rows, int cols, float* b);
void gemm_f32(gw_ctx* ctx, bool ta, bool tb, int M, int N, int K, float alpha, const float* A, long long lda,
              const float* B, long long ldb, float beta, float* C, long long ldc);
// binary32 FMA units only (every addition rounded to nearest): the products whose
// rounding must carry no common sign (U and q, which chi0 and the forms square)
void gemm_f32_rn(gw_ctx* ctx, bool ta, bool tb, int M, int N, int K, float alpha, const float* A, long long lda,
                 const float* B, long long ldb, float beta, float* C, long long ldc);
// tcgen05 3xTF32 tile GEMM; false when the shape is not worth it (caller falls back)
bool sgemm_tc(gw_ctx* ctx, bool ta, bool tb, int M, int N, int K, float alpha, const float* A, long long lda,
              const float* B, long long ldb, float beta, float* C, long long ldc);
// screen.cu
size_t ldlt_linv_bytes(int n, int n_omega, gw_precision prec);
void launch_ldlt(gw_ctx* ctx, gw_W* W);
void launch_forms(gw_ctx* ctx, const gw_W* W, const double* Q, int R, double* c);
void launch_ldlt_inverse(gw_ctx* ctx, const gw_W* W, int k, double2* out, double2* work);
// binary32 path: binary64 factorisation and forms at W->pole_k, overwriting those columns of c
void launch_pole_forms(gw_ctx* ctx, const gw_W* W, const double* Q, int R, double* cout);
// dyson.cu: self-energy matrix (pairs n <= m) and Dyson's equation
int dyson_max_states();
void launch_pair_rhs(gw_ctx* ctx, const double* Q, int S, int n_orb, int n_sub, double* Qp);
void launch_offdiag(gw_ctx* ctx, double* c, int S, int n_orb, int N);
void launch_sigma_x_pairs(gw_ctx* ctx, const gw_sigma* s, const double* Vnk, const double* T, int ld);
void launch_dyson(gw_ctx* ctx, const gw_sigma* s, const double* sx_minus_vxc, const int* states, double* dos,
                  double2* g);
// sigma.cu
void launch_sigma_grid(gw_ctx* ctx, gw_sigma* s);
void launch_sigma_c(gw_ctx* ctx, gw_sigma* s);
// second window: the large window's sigma (from s->c2) and its Cauchy sum added to s->sigc
void launch_sigma_grid2(gw_ctx* ctx, gw_sigma* s);
void launch_sigma_c2(gw_ctx* ctx, gw_sigma* s);
void launch_sigma_x(gw_ctx* ctx, gw_sigma* s, const double* Vnk, const double* T, int ld);
void launch_qp(gw_ctx* ctx, const gw_sigma* s, const double* vxc, double* e, double* z, int* st);
// utilities (misc kernels in linalg.cu)
void launch_split_complex(gw_ctx* ctx, const double2* z, double* re, double* im, size_t n);

// ------------------------------------------------------------------ complex
// Packed lower triangle (row-major): element (i, j), j <= i, of an n x n
// symmetric matrix sits at tri(i) + j; a matrix takes tri(n) elements.
__host__ __device__ inline long long tri(long long i) { return i * (i + 1) / 2; }

__host__ __device__ inline double2 cmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ inline double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__host__ __device__ inline double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__host__ __device__ inline double2 cconj(double2 a) { return make_double2(a.x, -a.y); }
__host__ __device__ inline float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ inline float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__host__ __device__ inline float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__host__ __device__ inline float2 cconj(float2 a) { return make_float2(a.x, -a.y); }

inline int div_up(long long a, long long b) { return (int)((a + b - 1) / b); }
