/*
 * gw.h -- C ABI of the GB300 GW screening library (libgw.so).
 *
 * The library computes, on one GPU, the frequency-resolved screening
 * pipeline of Foerster, Koval and Sanchez-Portal, "An O(N^3) implementation
 * of Hedin's GW approximation for molecules" (arXiv:1101.2065):
 *
 *   gw_build_chi0  spectral function of chi0 in the dominant-product basis
 *                  (Eq. chi_by_spectra, closed form of Sec. 6.1), compressed
 *                  (Eqs. subsetof_vef, projector0, subspace, subspace_chi0),
 *                  and its Cauchy (Kramers-Kronig) transform (binary64: by
 *                  FFT; binary32: direct sum over the transition band).
 *   gw_screen_W    chi^RPA = (1 - chi0)^-1 chi0 per frequency (Eq. chi_RPA),
 *                  W = v + Zup chi^RPA Zup^T.
 *   gw_sigma_diag  diagonal GW self-energy from the spectral convolution of
 *                  Eq. spectral_3 and the Cauchy integral of Eq. Cauchy1;
 *                  exchange part by Eq. instantaneous.
 *   gw_qp_solve    diagonal quasiparticle equation E = E_KS + Sigma(E) - vxc.
 *
 * Conventions (all readings are stated here so that a caller needs nothing
 * else):
 *  - Units: Hartree, bohr.  All floating point arguments are IEEE binary64.
 *  - Grid: s_j = j*d_omega, j = 0..n_omega-1 (non-negative half; spectral
 *    functions are odd, a(-s) = -a(s)); eta = broadening (1.5*d_omega in the
 *    paper, Sec. 4.2).  Transitions are deposited with tent weights:
 *    x = Delta/d_omega, j = floor(x), f = x - j, weight 1-f on bin j and f on
 *    bin j+1.
 *  - chi0_k = sum_j A_j [1/(w_k - s_j + i eta) - 1/(w_k + s_j + i eta)],
 *    w_k = k*d_omega, A_j = sum_p 2 w_j(Delta_p) u_p u_p^T (spin factor 2).
 *  - Pairs (E occupied, F virtual) are ordered by (Delta = eps_F - eps_E,
 *    E, F).  Compression keeps the top n_sub eigenvectors of
 *    g = X_r^T v X_r over the first N_rank = min(N_pair, max(5 n_orb, n_sub))
 *    pairs; n_sub == n_prod selects the uncompressed basis Zup = L (v = L L^T).
 *  - gamma_k = -(1/pi) Im chi^RPA_k for k >= 1, gamma_0 = 0.
 *  - Matrices are row-major.  Complex numbers are interleaved (re, im)
 *    binary64 pairs.
 *
 * Ownership: host arrays passed in belong to the caller and are copied (or
 * fully consumed) before the call returns.  Opaque handles own device memory
 * until their gw_*_free or gw_ctx_destroy.  Every call is synchronous with
 * respect to the calling host thread: it enqueues its kernels on the
 * context stream and returns after they finished and their status word was
 * checked.  Functions are thread-compatible per context (one host thread at
 * a time per context), not thread-safe.
 *
 * Errors: every function returns a gw_status (0 = GW_OK, negative = error)
 * and records a message readable with gw_last_error().  No C++ exception
 * crosses this interface.  On error the output handle is set to NULL and
 * nothing is leaked.
 */
#ifndef GW_GB300_GW_H
#define GW_GB300_GW_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int gw_status;
#define GW_OK                  0
#define GW_ERR_INVALID_ARG    -1   /* bad size, NULL pointer, inconsistent layout */
#define GW_ERR_NOT_SPD        -2   /* Coulomb metric v not positive definite */
#define GW_ERR_GRID           -3   /* a transition falls outside the frequency window */
#define GW_ERR_RANK           -4   /* compression subspace rank below n_sub */
#define GW_ERR_SINGULAR       -5   /* zero or non-finite pivot of 1 - chi0 */
#define GW_ERR_NO_CONVERGENCE -6   /* eigensolver did not converge */
#define GW_ERR_OOM            -7   /* device allocation failed */
#define GW_ERR_ADMISSION      -8   /* request exceeds the context's HBM budget */
#define GW_ERR_TIMEOUT        -9   /* a bounded device wait gave up */
#define GW_ERR_CUDA          -10   /* CUDA runtime error (message has details) */
#define GW_ERR_CANCELLED     -11   /* serving: the server was destroyed before the job started */

typedef enum {
    GW_FP64 = 0,      /* every step in binary64 */
    GW_MIXED = 1      /* binary32 contractions, Cauchy sum, factorisation and forms
                         (3xTF32 tensor-core products where the tensor cores'
                         accumulation bias stays below the tolerance, binary32 FMA
                         elsewhere), binary64 setup, Sigma and quasiparticle root;
                         error stated against GW_FP64 */
} gw_precision;

typedef struct gw_ctx gw_ctx;       /* device, stream, HBM accounting */
typedef struct gw_mol gw_mol;       /* device-resident molecule */
typedef struct gw_chi0 gw_chi0;     /* pair table, basis, chi0(w_k) for all k */
typedef struct gw_W gw_W;           /* factorised 1 - chi0(w_k) for all k */
typedef struct gw_sigma gw_sigma;   /* Sigma forms, sigma(s), Sigma_c grid, Sigma_x */

/* Molecule description, host pointers, read during gw_mol_upload only.
 * Orbitals and products are atom-major: atom A owns orbitals
 * [sum_{B<A} atom_norb[B], ... + atom_norb[A]) and likewise products.
 * L(A) = orbitals of the atoms {A} u N(A) in ascending atom order; the
 * vertex block of product mu (on atom A) is a dense symmetric row-major
 * |L(A)| x |L(A)| matrix at vertex + vertex_off[mu] (Eq. VertexDefinition;
 * entries outside L(A) x L(A) are zero by locality). */
typedef struct {
    int n_atoms, n_orb, n_occ, n_prod, n_sub;
    const int* atom_norb;          /* [n_atoms] */
    const int* atom_nprod;         /* [n_atoms] */
    const int* nbr_ptr;            /* [n_atoms+1] CSR neighbour lists, no self loops */
    const int* nbr_idx;            /* [nbr_ptr[n_atoms]] */
    const double* eps;             /* [n_orb] ascending; first n_occ occupied */
    const double* X;               /* [n_orb*n_orb] X[a*n_orb + E], column E = state E */
    const double* vertex;          /* concatenated blocks */
    const long long* vertex_off;   /* [n_prod+1] */
    const double* v;               /* [n_prod*n_prod] symmetric positive definite */
    const double* Z;               /* optional [n_prod*n_sub] basis Z[mu*n_sub + m] with
                                      Z^T v Z = I; NULL => built by the library */
} gw_molecule_desc;

typedef struct { int n_omega; double d_omega; double eta; } gw_grid;

typedef struct {
    int n_orb, n_occ, n_prod, n_sub, n_pair, n_rank;  /* n_rank = 0: uncompressed */
    int n_omega, j_lo, j_hi;       /* bins j_lo..j_hi carry all spectral weight */
    int precision;
    double min_pivot_ratio;        /* min_k min_i |d_i(k)| / max|1 - chi0_k| (after screen_W) */
    int n_pole;                    /* frequencies refactorised in binary64 (GW_OPT_POLES_FP64) */
} gw_info;

/* ---------------------------------------------------------------- context */
const char* gw_version(void);
/* device: CUDA ordinal; hbm_budget_bytes: 0 = unlimited, else allocations
 * beyond it fail with GW_ERR_ADMISSION; cuda_stream: a cudaStream_t to
 * enqueue on (e.g. a PyTorch stream), or NULL for a stream owned by the
 * context. */
gw_status gw_ctx_create(gw_ctx** out, int device, size_t hbm_budget_bytes, void* cuda_stream);
void      gw_ctx_destroy(gw_ctx* ctx);
const char* gw_last_error(const gw_ctx* ctx);
size_t    gw_ctx_bytes_in_use(const gw_ctx* ctx);
/* Number of this library's kernel launches issued on the context so far. */
long long gw_ctx_launch_count(const gw_ctx* ctx);
/* Per-kernel timing with CUDA events recorded on the context stream around
 * each launch of the named kernel (kernel_name NULL or "" = every kernel).
 * Enabling (or disabling) clears the accumulated totals.  The events add
 * one record before and one after every matched launch. */
gw_status gw_ctx_profile(gw_ctx* ctx, int enable, const char* kernel_name);
/* Accumulated device time (ms) and launch count of one kernel since the last
 * gw_ctx_profile call; synchronises the context stream. */
gw_status gw_ctx_profile_get(gw_ctx* ctx, const char* kernel_name, double* total_ms, long long* launches);
/* Kernel selection switches of a context (implementation choices with the
 * same results within the precision's tolerance; the paper has no
 * counterpart).
 * GW_OPT_FORMS_SIMT (value 0 or 1, default 0): for 32 < N_sub <= 384 the
 * binary32 path by default keeps the forward substitution's updates in
 * tensor memory (3xTF32 products), and for larger N_sub it runs the
 * forward substitution left-looking by blocks of 128 rows, the product of
 * all rows above a block on the tensor cores (3xTF32); 1 runs both on the
 * FMA units instead (right-looking, by pairs of 32-column panels).
 * GW_OPT_SYRK_SIMT (value 0 or 1, default 0): the binary32 factorisation
 * runs its trailing updates of 128 or more rows as 3xTF32 tensor-core
 * products by default, two 32-column panels per pass over the trailing
 * matrix while 128 rows remain after the second (the same factors as one
 * pass per panel); 1 keeps them on the FMA units.
 * GW_OPT_GEMM_SIMT (value 0 or 1, default 0): the binary32 path's dense
 * products (g, U, Z, Zup, q) run as 3xTF32 tensor-core products by default;
 * 1 runs them on the binary32 FMA units (round to nearest throughout).
 * GW_OPT_KK_TENSOR (value 0 or 1, default 0): the binary32 path's
 * Cauchy (Kramers-Kronig) sum of Eq. chi_by_spectra runs on the binary32
 * FMA units by default (round to nearest); 1 runs it as a 3xTF32
 * tensor-core product, faster, but the tensor cores' accumulation shrinks
 * every chi0 element by a few 1e-8 relative, which 1 - chi0 amplifies to
 * about 3e-5 in W near the RPA poles.
 * GW_OPT_POLES_FP64 (value t in 0..1000, default 0 = off; a precision
 * policy, Eq. chi_RPA): on the binary32 path, gw_screen_W measures the
 * spectral weight of chi^RPA_k along 8 fixed pseudo-random directions b,
 * s(k) = sum_b |Im b^T (1 - chi0_k)^-1 b| from the binary32 factors, and
 * the frequencies k >= 1 with s(k) >= (t/1000) max_k s(k), those near the
 * poles of W, are factorised again in binary64 (from the binary32 chi0_k)
 * where they are consumed: their quadratic forms in gw_sigma_diag and the
 * read-back of chi^RPA and W.  gw_W_info reports how many (n_pole).
 * GW_OPT_BARRIER_POLLS (value >= 0, default 0 = about a second): how many
 * times a CTA of the whole-GPU tridiagonalisation (compression ranks above
 * about 645) polls a grid barrier before it gives up, flags GW_ERR_TIMEOUT
 * and returns; the call then fails with GW_ERR_TIMEOUT and the context stays
 * usable.  A small value exercises that path (tests).
 * GW_ERR_INVALID_ARG for an unknown option or value. */
enum { GW_OPT_FORMS_SIMT = 2, GW_OPT_SYRK_SIMT = 3, GW_OPT_GEMM_SIMT = 4,
       GW_OPT_KK_TENSOR = 5, GW_OPT_POLES_FP64 = 6, GW_OPT_BARRIER_POLLS = 7 };
gw_status gw_ctx_set_option(gw_ctx* ctx, int option, int value);

/* ---------------------------------------------------------------- molecule */
/* Validates the description (sizes, CSR, offsets) and copies it to the
 * device.  GW_ERR_INVALID_ARG on inconsistent input. */
gw_status gw_mol_upload(gw_ctx* ctx, const gw_molecule_desc* desc, gw_mol** out);
void      gw_mol_free(gw_mol* mol);

/* ---------------------------------------------------------------- pipeline */
/* a0-a4: pair table, vertex products V^{EF}_mu = X_aE V^mu_ab X_bF
 * (Sec. 6.1), compression basis (Eqs. projector0, subspace,
 * global-basis-orthogonality) unless desc->Z was given, u_p = Zup^T V^p
 * (Eq. subspace_chi0), tent deposit of A_j and chi0_k by the Cauchy integral
 * (Eq. chi_by_spectra; binary64: exact FFT form, binary32: direct sum over
 * the bins that carry weight).  Errors: GW_ERR_GRID if
 * max Delta/d_omega + 1 > n_omega - 1; GW_ERR_NOT_SPD; GW_ERR_RANK if
 * lambda_{n_sub} < 1e-12 lambda_max; GW_ERR_NO_CONVERGENCE. */
gw_status gw_build_chi0(gw_ctx* ctx, const gw_mol* mol, const gw_grid* grid,
                        gw_precision prec, gw_chi0** out);
/* As gw_build_chi0 with the compression chosen by thresholds (Sec. 7.2)
 * instead of desc->n_sub: the first N_rank pairs are those with
 * |E - F| < e_threshold (Ha; Eq. subsetof_vef), and N_sub is the number of
 * eigenvalues of g = X_r^T v X_r at least lambda_rel times the largest one
 * (Eq. subspace; lambda_rel in [1e-6, 1): the deciding eigenvalues are
 * binary32).  gw_chi0_info reports the n_rank and n_sub chosen; every later
 * step works in that subspace.  GW_ERR_RANK if no pair or no eigenvalue
 * passes; GW_ERR_INVALID_ARG if the molecule carries its own basis Z. */
gw_status gw_build_chi0_thr(gw_ctx* ctx, const gw_mol* mol, const gw_grid* grid, gw_precision prec,
                            double e_threshold, double lambda_rel, gw_chi0** out);
/* Second window technique (Sec. 4.2, Eq. win2-for-response): chi0 on a
 * small, fine window and on a large, coarse one.  large: the one-window grid
 * (n_omega a power of two, every transition inside it); small: any n_omega in
 * [4, 32768] with d_omega below the large grid's (eta of each grid is its
 * broadening, 1.5 d_omega in the paper).  With lam = (small.n_omega - 1)
 * small.d_omega, spectral arguments below lam belong to the small window and
 * the others to the large one: *large_out is gw_build_chi0 on the large
 * grid; *small_out is chi0 at the small grid's frequencies from the pairs
 * with Delta < lam deposited on the small grid (small broadening) plus the
 * other pairs deposited on the large grid (large broadening).  Keep the
 * large handle alive while the small one is in use; each is screened by
 * gw_screen_W and freed by gw_chi0_free.  The small handle keeps no pair
 * table, U or spectral weights (their read-backs return GW_ERR_INVALID_ARG). */
gw_status gw_build_chi0_2w(gw_ctx* ctx, const gw_mol* mol, const gw_grid* small, const gw_grid* large,
                           gw_precision prec, gw_chi0** small_out, gw_chi0** large_out);
/* a5: factorises 1 - chi0_k = L_k D_k L_k^T (complex symmetric) for every
 * k (Eq. chi_RPA).  chi0 stays valid.  GW_ERR_SINGULAR on a zero or
 * non-finite pivot. */
gw_status gw_screen_W(gw_ctx* ctx, const gw_chi0* chi0, gw_W** out);
/* a6-a7 for the host list of states (each in [0, n_orb)):
 * q_nk = Zup^T V^{nk}, c_nk(s_j) = q_nk^T gamma_j q_nk, sigma_n(s) by the
 * tent shift of Eq. spectral_3 (virtual k: s = E_k + s2; occupied k:
 * s = E_k - s2), Sigma_c on w_k = k d_omega, |k| < n_omega, by Eq. Cauchy1
 * with time ordering sgn(s_j) (sgn 0 = +1), and
 * Sigma_x_n = -sum_{k occ} V^{nk} v V^{nk} (Eq. instantaneous). */
gw_status gw_sigma_diag(gw_ctx* ctx, const gw_W* W, const int* states, int n_states,
                        gw_sigma** out);
/* Self-energy with the second window technique (Sec. 4.2): the forms of
 * both windows, c_nk on the small grid kept for s2 < lam (its last point
 * zeroed) and on the large grid kept for s2 >= lam (its first points
 * zeroed); sigma_n on each grid from its forms; Sigma_c on the small grid's
 * points is the sum of both Cauchy sums, each with its window's broadening.
 * gw_qp_solve then adds both windows' Re Sigma_c.  W_small, W_large: the
 * screened handles of a gw_build_chi0_2w pair.  gw_sigma_copy returns the
 * small window's arrays (c as used, sigma, the combined Sigma_c);
 * gw_sigma_copy_large the large window's c and sigma. */
gw_status gw_sigma_diag_2w(gw_ctx* ctx, const gw_W* W_small, const gw_W* W_large, const int* states,
                           int n_states, gw_sigma** out);
/* Self-energy as a matrix over a set of states (Sec. 3, Eqs.
 * tensorform-self-energy and instantaneous; at most 16 states): Sigma_c,nm
 * on w_k = k d_omega, |k| < n_omega, from the forms c_nm,k = q_nk^T gamma
 * q_mk (obtained by polarisation from the quadratic forms of q_nk and
 * q_nk + q_mk), shifted by E_k and Cauchy-summed as the diagonal;
 * Sigma_x,nm = -sum_{k occ} V^{nk} v V^{mk}.  The handle is consumed by
 * gw_dyson_dos and gw_sigma_matrix_copy (not by gw_qp_solve). */
gw_status gw_sigma_matrix(gw_ctx* ctx, const gw_W* W, const int* states, int n_states, gw_sigma** out);
/* sigma_c: host complex [S][S][2 n_omega - 1]; sigma_x: host [S][S]; either may be NULL */
gw_status gw_sigma_matrix_copy(gw_ctx* ctx, const gw_sigma* s, double* sigma_c, double* sigma_x);
/* Dyson's equation (Eq. tensorform-dyson) on w_k = k d_omega, |k| < n_omega:
 * G(w)^-1 = (w + i eta - E_n) delta_nm - Sigma_c,nm(w) - Sigma_x,nm + vxc_nm over
 * the matrix's states (binary64 Gauss-Jordan per frequency), the states
 * outside the set non-interacting; dos [2 n_omega - 1] = -(1/pi) Im Tr G.
 * vxc: host [S][S] or NULL (vxc = Sigma_x).  g_diag: host complex
 * [S][2 n_omega - 1] = G_nn, or NULL. */
gw_status gw_dyson_dos(gw_ctx* ctx, const gw_sigma* s, const double* vxc, double* dos, double* g_diag);
/* a8 (Sec. 2: the quasiparticle equation with the exchange-correlation
 * potential of the mean field removed, the diagonal approximation of
 * Dyson's equation Eq. tensorform-dyson):
 * E solves E - E_KS - Sigma_x + vxc - Re Sigma_c(E) = 0 per state:
 * linearised start, Newton to |step| < 1e-11 Ha (100 steps, confined to
 * +-0.5 Ha of the start), else bracket scan at step d_omega over +-0.5 Ha
 * and bisection.  vxc: host [n_states] or NULL for vxc = Sigma_x (the
 * mean field is taken to contain exchange).  Outputs are host arrays
 * [n_states]; root_status 0 = Newton, 1 = bisection, 2 = no root found
 * (the linearised value is returned). */
gw_status gw_qp_solve(gw_ctx* ctx, const gw_sigma* sigma, const double* vxc,
                      double* e_qp, double* z_factor, int* root_status);

/* a0-a8 on a device-resident molecule (which may have been uploaded through
 * another context of the same device; it is only read): the steps of
 * gw_build_chi0, gw_screen_W, gw_sigma_diag and gw_qp_solve (Eqs.
 * chi_by_spectra, chi_RPA, spectral_3, Cauchy1, instantaneous and the QP
 * rule of gw_qp_solve), QP results to host arrays [n_states], intermediate
 * device state released.  sigma_x: host [n_states] or NULL. */
gw_status gw_solve(gw_ctx* ctx, const gw_mol* mol, const gw_grid* grid, gw_precision prec,
                   const int* states, int n_states, const double* vxc, double* e_qp, double* z_factor,
                   int* root_status, double* sigma_x);

/* End to end through host memory: upload, a0-a8, QP results to host,
 * device state released.  sigma_x: host [n_states] or NULL. */
gw_status gw_solve_host(gw_ctx* ctx, const gw_molecule_desc* desc, const gw_grid* grid,
                        gw_precision prec, const int* states, int n_states,
                        const double* vxc, double* e_qp, double* z_factor,
                        int* root_status, double* sigma_x);

/* ---------------------------------------------------------------- serving
 * Continuous batching of GW jobs on one device.  n_workers host threads,
 * each with its own context and CUDA stream, take jobs from a FIFO queue;
 * the head job is admitted as soon as its estimated device footprint fits
 * the remaining hbm_budget_bytes (0 = unlimited), so jobs arriving while
 * others run start as memory frees up and overlap on the GPU.  A job is
 * one molecule through a0-a8 (as gw_solve_host); the description is copied
 * at submission.  Results do not depend on the other jobs in flight
 * (fixed-order reductions, no cross-job state). */
typedef struct gw_server gw_server;
gw_status gw_server_create(gw_server** out, int device, int n_workers, size_t hbm_budget_bytes);
/* Stops the workers after their running jobs; jobs still queued end with
 * GW_ERR_CANCELLED.  Must not run concurrently with gw_server_wait or
 * gw_server_submit on the same server (collect the results first). */
void      gw_server_destroy(gw_server* s);
/* GW_ERR_ADMISSION if the job alone exceeds the budget. */
gw_status gw_server_submit(gw_server* s, const gw_molecule_desc* desc, const gw_grid* grid,
                           gw_precision prec, const int* states, int n_states, const double* vxc,
                           long long* job_id);
/* As gw_server_submit for a device-resident molecule (gw_mol_upload on any
 * context of the server's device): no host copy, no upload in the job.  The
 * caller keeps the molecule alive until the job's gw_server_wait returns. */
gw_status gw_server_submit_resident(gw_server* s, const gw_mol* mol, const gw_grid* grid, gw_precision prec,
                                    const int* states, int n_states, const double* vxc, long long* job_id);
/* This library's kernel launches over all worker contexts so far. */
long long gw_server_launch_count(const gw_server* s);
/* gw_ctx_profile / gw_ctx_profile_get over all worker contexts (times and
 * launches summed; each kernel timed on its worker's stream, so concurrent
 * jobs stretch one another's intervals).  Call while no job is queued or
 * running. */
gw_status gw_server_profile(gw_server* s, int enable, const char* kernel_name);
gw_status gw_server_profile_get(gw_server* s, const char* kernel_name, double* total_ms, long long* launches);
/* 0 queued, 1 running, 2 done; a negative gw_status if the job failed. */
int       gw_server_poll(gw_server* s, long long job_id);
/* Waits up to timeout_ms (< 0: no limit; GW_ERR_TIMEOUT when it runs out),
 * copies the results (host arrays [n_states], each may be NULL) and
 * releases the job.  times_ms [3] (nullable): queue wait, run time, total.
 * err (nullable, err_len bytes) receives the failure message.  Returns the
 * job's status. */
gw_status gw_server_wait(gw_server* s, long long job_id, int timeout_ms, double* e_qp,
                         double* z_factor, int* root_status, double* sigma_x, double* times_ms,
                         char* err, size_t err_len);
/* Estimated device footprint of a job (bytes), the figure gw_server_submit
 * compares with the budget: the molecule plus the largest phase (basis
 * construction, chi0 with the spectral weights of the band spanned by
 * desc->eps, or the factors and forms of the screening), plus one eighth and
 * 64 MiB of slack.  Host-only; 0 for a NULL or incomplete desc or grid. */
size_t    gw_server_job_bytes(const gw_molecule_desc* desc, const gw_grid* grid, gw_precision prec,
                              int n_states);

/* Allocation-free Sigma_c grid (no counterpart in the paper: an interface
 * for callers that cannot allocate device memory, such as an application
 * whose device memory belongs to another allocator or a latency-critical
 * loop).  Computes the same Sigma_c(w_k), k = -(n_omega-1)..n_omega-1, as
 * gw_sigma_diag from sigma_n(s_j), s_j = (j0 + i) d_omega.
 *   sigma  device [n_states*n_sig] binary64, read
 *   sigc   device [n_states*(2 n_omega - 1)] complex binary64, written
 *   stream cudaStream_t to enqueue on (NULL: legacy default stream); the
 *          call is asynchronous and does not synchronise
 *   err    optional host buffer of err_len bytes for a message
 * Scratch: a fixed table of n_sig + 2 n_omega - 1 complex entries inside
 * the library, at most 65536 entries (1 MiB, held on every GPU that loads
 * the library until the process exits); larger requests return
 * GW_ERR_INVALID_ARG.  Allocates no device or host memory.  All calls on
 * a device share the table: calls that overlap on the GPU race.  The first
 * call in a CUDA context (normally the device's primary context) resolves
 * the table's address with that context current and caches it per context
 * (after a device reset the next call resolves it again); make that first
 * call before any stream capture.  Launch errors return GW_ERR_CUDA. */
gw_status gw_sigma_c_static(const double* sigma, int n_states, int n_sig, int j0, int n_omega,
                            double d_omega, double eta, double* sigc, void* stream, char* err,
                            size_t err_len);

void gw_chi0_free(gw_chi0* chi0);
void gw_W_free(gw_W* W);
void gw_sigma_free(gw_sigma* sigma);

/* ---------------------------------------------------------------- read-back
 * Blocking copies into caller-owned host buffers (used by tests). */
gw_status gw_chi0_info(const gw_chi0* chi0, gw_info* out);
gw_status gw_W_info(const gw_W* W, gw_info* out);
/* pair table in sorted order: E, F [n_pair] int, delta, frac [n_pair] double,
 * bin [n_pair] int; any pointer may be NULL */
gw_status gw_chi0_copy_pairs(gw_ctx* ctx, const gw_chi0* chi0, int* E, int* F,
                             double* delta, int* bin, double* frac);
/* Z and Zup: [n_prod*n_sub] row-major; either may be NULL */
gw_status gw_chi0_copy_basis(gw_ctx* ctx, const gw_chi0* chi0, double* Z, double* Zup);
/* U: [n_pair*n_sub] row-major, u_p = Zup^T V^p for sorted pair p */
gw_status gw_chi0_copy_U(gw_ctx* ctx, const gw_chi0* chi0, double* U);
/* A_j for j in [j0, j0+nj): [nj*n_sub*n_sub] real, recomputed on the device */
gw_status gw_chi0_copy_spectral(gw_ctx* ctx, const gw_chi0* chi0, int j0, int nj, double* A);
/* chi0_k for k in [k0, k0+nk): [nk*n_sub*n_sub] complex (full symmetric) */
gw_status gw_chi0_copy(gw_ctx* ctx, const gw_chi0* chi0, int k0, int nk, double* out);
/* the frequencies refactorised in binary64 by GW_OPT_POLES_FP64, ascending, [n_pole] */
gw_status gw_W_pole_freqs(const gw_W* W, int* freqs);
/* min_i |d_i(k)| / max |1 - chi0_k| of the factorisation, [n_omega] */
gw_status gw_W_copy_pivots(gw_ctx* ctx, const gw_W* W, double* ratio);
/* chi0_k[m_i, n_i] for every k and the ne host index pairs (m_i, n_i):
 * complex [n_omega][ne] */
gw_status gw_chi0_copy_elements(gw_ctx* ctx, const gw_chi0* chi0, const int* m, const int* n, int ne,
                                double* out);
/* chi^RPA_k (compressed, complex [nf*n_sub*n_sub]) for the host list freqs */
gw_status gw_W_copy_chi_rpa(gw_ctx* ctx, const gw_W* W, const int* freqs, int nf, double* out);
/* W_k = v + Zup chi^RPA_k Zup^T (complex [nf*n_prod*n_prod]) for the host list freqs */
gw_status gw_W_copy_full(gw_ctx* ctx, const gw_W* W, const int* freqs, int nf, double* out);
/* sigma read-back; every pointer may be NULL.
 *   c      [n_states*n_orb*n_omega] real   c_nk(s_j)
 *   sigma  [n_states*n_sig] real           sigma_n(s_j), s_j = (j0 + i) d_omega
 *   sigc   [n_states*(2 n_omega - 1)] complex  Sigma_c(w_k), k = -(n_omega-1)..n_omega-1
 *   sigma_x [n_states] */
gw_status gw_sigma_copy(gw_ctx* ctx, const gw_sigma* s, double* c, double* sigma,
                        double* sigc, double* sigma_x);
gw_status gw_sigma_grid(const gw_sigma* s, int* j0, int* n_sig);
/* second window (gw_sigma_diag_2w): the large window's c [n_states*n_orb*n_omega_large]
 * (zero for s2 < lam) and sigma [n_states*n_sig2] on bins j0 .. j0 + n_sig2 - 1 */
gw_status gw_sigma_copy_large(gw_ctx* ctx, const gw_sigma* s, double* c, double* sigma);
gw_status gw_sigma_grid_large(const gw_sigma* s, int* j0, int* n_sig);

#ifdef __cplusplus
}
#endif
#endif
