// C ABI of the GW library: argument validation, device memory accounting,
// orchestration of the kernels of steps a0-a8, read-back for tests.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <new>

#include "internal.h"

// ======================================================================
// runtime helpers
// ======================================================================
void gw_throw(gw_status code, const std::string& msg) { throw GwError{code, msg}; }

void cuda_check(cudaError_t e, const char* what) {
    if (e != cudaSuccess) {
        cudaGetLastError();
        gw_throw(e == cudaErrorMemoryAllocation ? GW_ERR_OOM : GW_ERR_CUDA,
                 std::string(what) + ": " + cudaGetErrorString(e));
    }
}

void* ctx_alloc(gw_ctx* ctx, size_t bytes) {
    if (bytes == 0) bytes = 16;
    bytes = (bytes + 255) & ~size_t(255);
    if (ctx->budget && ctx->in_use + bytes > ctx->budget)
        gw_throw(GW_ERR_ADMISSION, "allocation of " + std::to_string(bytes) +
                                       " bytes exceeds the HBM budget of the context");
    void* p = nullptr;
    cudaError_t e = cudaMallocAsync(&p, bytes, ctx->stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        gw_throw(GW_ERR_OOM, "device allocation of " + std::to_string(bytes) + " bytes failed: " +
                                 cudaGetErrorString(e));
    }
    ctx->blocks[p] = bytes;
    ctx->in_use += bytes;
    ctx->peak = std::max(ctx->peak, ctx->in_use);
    return p;
}

void ctx_free(gw_ctx* ctx, void* p) {
    if (!p || !ctx) return;
    auto it = ctx->blocks.find(p);
    if (it == ctx->blocks.end()) return;
    ctx->in_use -= it->second;
    ctx->blocks.erase(it);
    cudaFreeAsync(p, ctx->stream);
}

void allow_max_smem_impl(const void* func) {
    static std::mutex mu;
    static std::unordered_map<const void*, bool> done;
    std::lock_guard<std::mutex> lk(mu);
    if (done[func]) return;
    int dev = 0, optin = 0;
    CUDA_CHECK(cudaGetDevice(&dev));
    CUDA_CHECK(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    cudaFuncAttributes fa{};
    CUDA_CHECK(cudaFuncGetAttributes(&fa, func));
    CUDA_CHECK(cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    optin - (int)fa.sharedSizeBytes));
    done[func] = true;
}

static bool prof_match(const gw_ctx* ctx, const char* name) {
    return ctx->prof_on && (ctx->prof_filter.empty() || ctx->prof_filter == name);
}

static cudaEvent_t prof_event(gw_ctx* ctx) {
    if (!ctx->prof_pool.empty()) {
        cudaEvent_t e = ctx->prof_pool.back();
        ctx->prof_pool.pop_back();
        return e;
    }
    cudaEvent_t e;
    CUDA_CHECK(cudaEventCreate(&e));
    return e;
}

void prof_begin(gw_ctx* ctx, const char* name) {
    if (!prof_match(ctx, name)) return;
    cudaEvent_t e = prof_event(ctx);
    CUDA_CHECK(cudaEventRecord(e, ctx->stream));
    ctx->prof_pending = e;
}

static void prof_collect(gw_ctx* ctx) {
    if (ctx->prof_recs.empty()) return;
    CUDA_CHECK(cudaStreamSynchronize(ctx->stream));
    for (auto& r : ctx->prof_recs) {
        float ms = 0.f;
        CUDA_CHECK(cudaEventElapsedTime(&ms, r.start, r.stop));
        auto& acc = ctx->prof_acc[r.name];
        acc.first += ms;
        acc.second += 1;
        ctx->prof_pool.push_back(r.start);
        ctx->prof_pool.push_back(r.stop);
    }
    ctx->prof_recs.clear();
}

void after_launch(gw_ctx* ctx, const char* name) {
    ctx->launches++;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) gw_throw(GW_ERR_CUDA, std::string("launch of ") + name + ": " + cudaGetErrorString(e));
    if (ctx->prof_pending && prof_match(ctx, name)) {
        cudaEvent_t stop = prof_event(ctx);
        CUDA_CHECK(cudaEventRecord(stop, ctx->stream));
        ctx->prof_recs.push_back({name, ctx->prof_pending, stop});
        ctx->prof_pending = nullptr;
        if (ctx->prof_recs.size() > 4096) prof_collect(ctx);
    }
}

void ctx_finish(gw_ctx* ctx, const char* where) {
    CUDA_CHECK(cudaMemcpyAsync(ctx->h_status, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    CUDA_CHECK(cudaStreamSynchronize(ctx->stream));
    int st = *ctx->h_status;
    if (st) {
        CUDA_CHECK(cudaMemsetAsync(ctx->d_status, 0, sizeof(int), ctx->stream));
        CUDA_CHECK(cudaStreamSynchronize(ctx->stream));
        std::string w(where);
        if (st & ST_TIMEOUT) gw_throw(GW_ERR_TIMEOUT, w + ": a bounded device wait gave up");
        if (st & ST_NOT_SPD) gw_throw(GW_ERR_NOT_SPD, w + ": Coulomb metric is not positive definite");
        if (st & ST_RANK) gw_throw(GW_ERR_RANK, w + ": compression rank below n_sub (lambda_nsub < 1e-12 lambda_max)");
        if (st & ST_SINGULAR) gw_throw(GW_ERR_SINGULAR, w + ": zero or non-finite pivot of 1 - chi0");
        if (st & ST_NONFINITE) gw_throw(GW_ERR_SINGULAR, w + ": non-finite value");
        if (st & ST_BOUNDS) gw_throw(GW_ERR_INVALID_ARG, w + ": index out of bounds detected on the device");
        gw_throw(GW_ERR_CUDA, w + ": unknown device status");
    }
}

#define API_BEGIN(ctxp) gw_ctx* _api_ctx = (ctxp); try {
#define API_END                                                                  \
    }                                                                            \
    catch (const GwError& e) {                                                   \
        if (_api_ctx) _api_ctx->err = e.msg;                                     \
        return e.code;                                                           \
    }                                                                            \
    catch (const std::bad_alloc&) {                                              \
        if (_api_ctx) _api_ctx->err = "host allocation failed";                  \
        return GW_ERR_OOM;                                                       \
    }                                                                            \
    catch (...) {                                                                \
        if (_api_ctx) _api_ctx->err = "unexpected internal error";               \
        return GW_ERR_CUDA;                                                      \
    }                                                                            \
    return GW_OK;

#define REQUIRE(cond, msg) do { if (!(cond)) gw_throw(GW_ERR_INVALID_ARG, msg); } while (0)

template <class T>
static T* upload(gw_ctx* ctx, const T* h, size_t n) {
    T* d = dalloc<T>(ctx, n);
    CUDA_CHECK(cudaMemcpyAsync(d, h, n * sizeof(T), cudaMemcpyHostToDevice, ctx->stream));
    return d;
}

template <class T>
static void download(gw_ctx* ctx, T* h, const T* d, size_t n) {
    CUDA_CHECK(cudaMemcpyAsync(h, d, n * sizeof(T), cudaMemcpyDeviceToHost, ctx->stream));
}

// ======================================================================
// context
// ======================================================================
extern "C" const char* gw_version(void) { return "gw-gb300 0.1 (sm_103a)"; }

extern "C" gw_status gw_ctx_create(gw_ctx** out, int device, size_t hbm_budget_bytes, void* cuda_stream) {
    if (!out) return GW_ERR_INVALID_ARG;
    *out = nullptr;
    gw_ctx* ctx = new (std::nothrow) gw_ctx();
    if (!ctx) return GW_ERR_OOM;
    try {
        int ndev = 0;
        CUDA_CHECK(cudaGetDeviceCount(&ndev));
        REQUIRE(device >= 0 && device < ndev, "device ordinal out of range");
        CUDA_CHECK(cudaSetDevice(device));
        ctx->device = device;
        ctx->budget = hbm_budget_bytes;
        if (cuda_stream) {
            ctx->stream = (cudaStream_t)cuda_stream;
        } else {
            CUDA_CHECK(cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking));
            ctx->own_stream = true;
        }
        CUDA_CHECK(cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device));
        cudaMemPool_t pool;
        CUDA_CHECK(cudaDeviceGetDefaultMemPool(&pool, device));
        uint64_t thr = UINT64_MAX;
        CUDA_CHECK(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr));
        CUDA_CHECK(cudaMalloc(&ctx->d_status, sizeof(int)));
        CUDA_CHECK(cudaMemset(ctx->d_status, 0, sizeof(int)));
        CUDA_CHECK(cudaMallocHost(&ctx->h_status, sizeof(int)));
    } catch (const GwError& e) {
        gw_status code = e.code;
        if (ctx->d_status) cudaFree(ctx->d_status);
        if (ctx->h_status) cudaFreeHost(ctx->h_status);
        if (ctx->own_stream && ctx->stream) cudaStreamDestroy(ctx->stream);
        delete ctx;
        return code;
    }
    *out = ctx;
    return GW_OK;
}

extern "C" void gw_ctx_destroy(gw_ctx* ctx) {
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    for (auto& r : ctx->prof_recs) { cudaEventDestroy(r.start); cudaEventDestroy(r.stop); }
    for (auto e : ctx->prof_pool) cudaEventDestroy(e);
    if (ctx->prof_pending) cudaEventDestroy(ctx->prof_pending);
    for (auto& kv : ctx->blocks) cudaFreeAsync(kv.first, ctx->stream);
    ctx->blocks.clear();
    cudaStreamSynchronize(ctx->stream);
    cudaFree(ctx->d_status);
    cudaFreeHost(ctx->h_status);
    if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
    delete ctx;
}

extern "C" const char* gw_last_error(const gw_ctx* ctx) { return ctx ? ctx->err.c_str() : "no context"; }
extern "C" size_t gw_ctx_bytes_in_use(const gw_ctx* ctx) { return ctx ? ctx->in_use : 0; }
extern "C" long long gw_ctx_launch_count(const gw_ctx* ctx) { return ctx ? ctx->launches : 0; }

extern "C" gw_status gw_ctx_profile(gw_ctx* ctx, int enable, const char* kernel_name) {
    if (!ctx) return GW_ERR_INVALID_ARG;
    API_BEGIN(ctx)
    CUDA_CHECK(cudaSetDevice(ctx->device));
    prof_collect(ctx);
    ctx->prof_on = enable != 0;
    ctx->prof_filter = kernel_name ? kernel_name : "";
    ctx->prof_acc.clear();
    API_END
}

extern "C" gw_status gw_ctx_profile_get(gw_ctx* ctx, const char* kernel_name, double* total_ms, long long* launches) {
    if (!ctx || !kernel_name || !total_ms || !launches) return GW_ERR_INVALID_ARG;
    API_BEGIN(ctx)
    CUDA_CHECK(cudaSetDevice(ctx->device));
    prof_collect(ctx);
    auto it = ctx->prof_acc.find(kernel_name);
    *total_ms = it == ctx->prof_acc.end() ? 0.0 : it->second.first;
    *launches = it == ctx->prof_acc.end() ? 0 : it->second.second;
    API_END
}

extern "C" gw_status gw_ctx_set_option(gw_ctx* ctx, int option, int value) {
    if (!ctx) return GW_ERR_INVALID_ARG;
    if (option == GW_OPT_FORMS_SIMT && (value == 0 || value == 1)) {
        ctx->forms_simt = value != 0;
        return GW_OK;
    }
    if (option == GW_OPT_SYRK_SIMT && (value == 0 || value == 1)) {
        ctx->syrk_simt = value != 0;
        return GW_OK;
    }
    if (option == GW_OPT_GEMM_SIMT && (value == 0 || value == 1)) {
        ctx->gemm_simt = value != 0;
        return GW_OK;
    }
    if (option == GW_OPT_KK_TENSOR && (value == 0 || value == 1)) {
        ctx->kk_tensor = value != 0;
        return GW_OK;
    }
    if (option == GW_OPT_POLES_FP64 && value >= 0 && value <= 1000) {
        ctx->poles_permille = value;
        return GW_OK;
    }
    if (option == GW_OPT_BARRIER_POLLS && value >= 0) {
        ctx->barrier_polls = value;
        return GW_OK;
    }
    ctx->err = "gw_ctx_set_option: unknown option or value";
    return GW_ERR_INVALID_ARG;
}

// ======================================================================
// molecule
// ======================================================================
static void mol_release(gw_mol* m) {
    if (!m) return;
    gw_ctx* c = m->ctx;
    ctx_free(c, m->eps); ctx_free(c, m->X); ctx_free(c, m->vertex); ctx_free(c, m->voff);
    ctx_free(c, m->v); ctx_free(c, m->Z); ctx_free(c, m->prod_atom); ctx_free(c, m->loc_ptr);
    ctx_free(c, m->loc_idx);
    delete m;
}

static gw_mol* mol_upload(gw_ctx* ctx, const gw_molecule_desc* d) {
    REQUIRE(d, "NULL molecule description");
    REQUIRE(d->n_atoms > 0 && d->n_orb > 1 && d->n_prod > 0, "empty molecule");
    REQUIRE(d->n_occ > 0 && d->n_occ < d->n_orb, "need at least one occupied and one virtual state");
    REQUIRE(d->n_sub > 0 && d->n_sub <= d->n_prod, "n_sub must be in [1, n_prod]");
    REQUIRE(d->atom_norb && d->atom_nprod && d->nbr_ptr && d->eps && d->X && d->vertex &&
                d->vertex_off && d->v,
            "NULL array in molecule description");
    const int na = d->n_atoms;
    std::vector<int> optr(na + 1, 0), pptr(na + 1, 0);
    for (int a = 0; a < na; ++a) {
        REQUIRE(d->atom_norb[a] >= 0 && d->atom_nprod[a] >= 0, "negative per-atom count");
        optr[a + 1] = optr[a] + d->atom_norb[a];
        pptr[a + 1] = pptr[a] + d->atom_nprod[a];
    }
    REQUIRE(optr[na] == d->n_orb, "sum of atom_norb differs from n_orb");
    REQUIRE(pptr[na] == d->n_prod, "sum of atom_nprod differs from n_prod");
    REQUIRE(d->nbr_ptr[0] == 0, "nbr_ptr[0] must be 0");
    for (int a = 0; a < na; ++a) REQUIRE(d->nbr_ptr[a + 1] >= d->nbr_ptr[a], "nbr_ptr not monotone");
    const int nnz = d->nbr_ptr[na];
    REQUIRE(nnz == 0 || d->nbr_idx, "NULL nbr_idx");
    for (int a = 0; a < na; ++a)
        for (int q = d->nbr_ptr[a]; q < d->nbr_ptr[a + 1]; ++q)
            REQUIRE(d->nbr_idx[q] >= 0 && d->nbr_idx[q] < na && d->nbr_idx[q] != a,
                    "neighbour index out of range or self loop");
    for (int i = 1; i < d->n_orb; ++i) REQUIRE(d->eps[i] >= d->eps[i - 1], "eps must be ascending");
    for (int i = 0; i < d->n_orb; ++i) REQUIRE(std::isfinite(d->eps[i]), "non-finite eps");

    // local orbital lists L(A)
    std::vector<int> loc_ptr(na + 1, 0), loc_idx;
    int max_nloc = 0;
    for (int a = 0; a < na; ++a) {
        std::vector<int> atoms{a};
        for (int q = d->nbr_ptr[a]; q < d->nbr_ptr[a + 1]; ++q) atoms.push_back(d->nbr_idx[q]);
        std::sort(atoms.begin(), atoms.end());
        atoms.erase(std::unique(atoms.begin(), atoms.end()), atoms.end());
        for (int b : atoms)
            for (int o = optr[b]; o < optr[b + 1]; ++o) loc_idx.push_back(o);
        loc_ptr[a + 1] = (int)loc_idx.size();
        max_nloc = std::max(max_nloc, loc_ptr[a + 1] - loc_ptr[a]);
    }
    REQUIRE(max_nloc <= 112, "a local orbital set L(A) larger than 112 orbitals is not supported");
    std::vector<int> prod_atom(d->n_prod);
    REQUIRE(d->vertex_off[0] == 0, "vertex_off[0] must be 0");
    for (int a = 0; a < na; ++a)
        for (int mu = pptr[a]; mu < pptr[a + 1]; ++mu) {
            prod_atom[mu] = a;
            long long nl = loc_ptr[a + 1] - loc_ptr[a];
            REQUIRE(d->vertex_off[mu + 1] - d->vertex_off[mu] == nl * nl,
                    "vertex block size differs from |L(A)|^2");
        }
    gw_mol* m = new gw_mol();
    m->ctx = ctx;
    m->n_atoms = na; m->n_orb = d->n_orb; m->n_occ = d->n_occ; m->n_prod = d->n_prod; m->n_sub = d->n_sub;
    m->max_nloc = max_nloc;
    m->h_eps.assign(d->eps, d->eps + d->n_orb);
    m->vertex_len = (size_t)d->vertex_off[d->n_prod];
    try {
        m->eps = upload(ctx, d->eps, d->n_orb);
        m->X = upload(ctx, d->X, (size_t)d->n_orb * d->n_orb);
        m->vertex = upload(ctx, d->vertex, m->vertex_len);
        m->voff = upload(ctx, d->vertex_off, d->n_prod + 1);
        m->v = upload(ctx, d->v, (size_t)d->n_prod * d->n_prod);
        if (d->Z) m->Z = upload(ctx, d->Z, (size_t)d->n_prod * d->n_sub);
        m->prod_atom = upload(ctx, prod_atom.data(), prod_atom.size());
        m->loc_ptr = upload(ctx, loc_ptr.data(), loc_ptr.size());
        m->loc_idx = upload(ctx, loc_idx.data(), std::max<size_t>(loc_idx.size(), 1));
        CUDA_CHECK(cudaStreamSynchronize(ctx->stream));
    } catch (...) {
        mol_release(m);
        throw;
    }
    return m;
}

extern "C" gw_status gw_mol_upload(gw_ctx* ctx, const gw_molecule_desc* desc, gw_mol** out) {
    if (!ctx || !out) return GW_ERR_INVALID_ARG;
    *out = nullptr;
    API_BEGIN(ctx)
    CUDA_CHECK(cudaSetDevice(ctx->device));
    *out = mol_upload(ctx, desc);
    API_END
}

extern "C" void gw_mol_free(gw_mol* mol) { mol_release(mol); }

// ======================================================================
// a0-a4: chi0
// ======================================================================
static void chi0_release(gw_chi0* c) {
    if (!c) return;
    gw_ctx* x = c->ctx;
    ctx_free(x, c->pE); ctx_free(x, c->pF); ctx_free(x, c->pBin); ctx_free(x, c->pDelta);
    ctx_free(x, c->pFrac); ctx_free(x, c->seg); ctx_free(x, c->Z); ctx_free(x, c->Zup);
    ctx_free(x, c->Xr); ctx_free(x, c->Bsel);
    ctx_free(x, c->Ut); ctx_free(x, c->tw); ctx_free(x, c->C1); ctx_free(x, c->C2);
    ctx_free(x, c->chi0); ctx_free(x, c->Ut32); ctx_free(x, c->chi0_32); ctx_free(x, c->A64);
    delete c;
}

static void check_grid(const gw_grid* g) {
    REQUIRE(g, "NULL grid");
    REQUIRE(g->n_omega >= 4 && (g->n_omega & (g->n_omega - 1)) == 0 && g->n_omega <= (1 << 15),
            "n_omega must be a power of two in [4, 32768]");
    REQUIRE(g->d_omega > 0 && std::isfinite(g->d_omega), "d_omega must be positive");
    REQUIRE(g->eta > 0 && std::isfinite(g->eta), "eta must be positive");
}

// Threshold-driven compression (Sec. 7.2): N_rank = the pairs with
// |E - F| < e_threshold (Eq. subsetof_vef), N_sub = the eigenvalues of g at
// least lambda_rel times the largest (Eq. subspace).
struct Compression {
    double e_threshold, lambda_rel;
};

static gw_chi0* build_chi0(gw_ctx* ctx, const gw_mol* mol, const gw_grid* grid, gw_precision prec,
                           const Compression* cmp = nullptr) {
    // a molecule uploaded through another context of the same device may be shared
    // (read only; its upload was synchronised): serving keeps molecules resident
    REQUIRE(mol && mol->ctx && mol->ctx->device == ctx->device, "molecule belongs to another device");
    check_grid(grid);
    REQUIRE(prec == GW_FP64 || prec == GW_MIXED, "unknown precision");
    const int n_occ = mol->n_occ, n_orb = mol->n_orb, n_virt = n_orb - n_occ;
    const int N = grid->n_omega;
    // band of the tent bins, from the same binary64 operations as the device
    const std::vector<double>& e = mol->h_eps;
    double dmin = e[n_occ] - e[n_occ - 1], dmax = e[n_orb - 1] - e[0];
    double xlo = std::floor(dmin / grid->d_omega), xhi = std::floor(dmax / grid->d_omega);
    if (!(xlo >= 0) || !(xhi + 1 <= N - 1))
        gw_throw(GW_ERR_GRID, "a transition lies outside the frequency window (need floor(Delta/d_omega)+1 <= n_omega-1)");
    gw_chi0* c = new gw_chi0();
    c->ctx = ctx; c->mol = mol; c->grid = *grid; c->prec = prec;
    c->n_pair = n_occ * n_virt;
    c->n_sub = mol->n_sub;
    c->j_lo = (int)xlo;
    c->nb_bins = (int)xhi - (int)xlo + 1;
    c->j_hi = (int)xhi + 1;
    c->L = 2 * N;
    c->logL = 0;
    while ((1 << c->logL) < c->L) c->logL++;
    const int n_prod = mol->n_prod, n_pair = c->n_pair;
    int n_sub = mol->n_sub;
    int nr_thr = 0;
    if (cmp) {
        REQUIRE(cmp->e_threshold > 0 && std::isfinite(cmp->e_threshold), "e_threshold must be positive");
        // the eigenvalues that decide are binary32: a ratio below 1e-6 would not separate g's null space
        REQUIRE(cmp->lambda_rel >= 1e-6 && cmp->lambda_rel < 1, "lambda_rel must be in [1e-6, 1)");
        REQUIRE(!mol->Z, "a given basis Z and compression thresholds exclude each other");
        for (int E = 0; E < n_occ; ++E)
            for (int F = n_occ; F < n_orb; ++F) nr_thr += (e[F] - e[E] < cmp->e_threshold) ? 1 : 0;
        if (nr_thr < 1) gw_throw(GW_ERR_RANK, "no pair below e_threshold");
    }
    double* VEFt = nullptr;
    float* V32 = nullptr;
    double *T1 = nullptr, *g = nullptr, *Bsel = nullptr;
    int* occ = nullptr; int* virt = nullptr; int* rank_of = nullptr;
    try {
        // a0: pair table
        launch_pair_table(ctx, mol, c);
        // a1: vertex products for every pair, product-major [n_prod][n_pair] in sorted order
        std::vector<int> ho(n_occ), hv(n_virt);
        for (int i = 0; i < n_occ; ++i) ho[i] = i;
        for (int i = 0; i < n_virt; ++i) hv[i] = n_occ + i;
        occ = upload(ctx, ho.data(), ho.size());
        virt = upload(ctx, hv.data(), hv.size());
        rank_of = dalloc<int>(ctx, n_pair);
        // inverse permutation: natural pair index -> sorted position
        launch_invert_perm(ctx, c, rank_of);
        // near-pole policy on the binary32 path: binary64 V^EF, U and weights as well,
        // for the binary64 chi0 of the frequencies flagged by gw_screen_W
        const bool poles64 = prec == GW_MIXED && ctx->poles_permille > 0;
        if (prec == GW_MIXED) {
            // the mixed path uses V^EF only in binary32 (g, U, and X_r for Z)
            V32 = dalloc<float>(ctx, (size_t)n_prod * n_pair);
            launch_vertex_contract32(ctx, mol, occ, n_occ, virt, n_virt, rank_of, V32, n_pair);
            if (poles64) {
                VEFt = dalloc<double>(ctx, (size_t)n_prod * n_pair);
                launch_vertex_contract(ctx, mol, occ, n_occ, virt, n_virt, rank_of, VEFt, n_pair);
            }
        } else {
            VEFt = dalloc<double>(ctx, (size_t)n_prod * n_pair);
            launch_vertex_contract(ctx, mol, occ, n_occ, virt, n_virt, rank_of, VEFt, n_pair);
        }
        // a0: basis (threshold-driven: N_sub is known once the eigenvalues of g are)
        if (!cmp) c->Zup = dalloc<double>(ctx, (size_t)n_prod * n_sub);
        auto choose_n_sub = [&](const double* g64, const float* g32_, int nr) {
            std::vector<float> lam = eigvals32(ctx, g64, g32_, nr);
            const double top = lam.back();
            int k = 0;
            for (float x : lam) k += ((double)x >= cmp->lambda_rel * top) ? 1 : 0;
            if (!(top > 0) || k < 1) gw_throw(GW_ERR_RANK, "no eigenvalue of g above lambda_rel");
            n_sub = k;
            c->n_sub = n_sub;
            c->Zup = dalloc<double>(ctx, (size_t)n_prod * n_sub);
        };
        if (mol->Z) {
            c->Z = dalloc<double>(ctx, (size_t)n_prod * n_sub);
            CUDA_CHECK(cudaMemcpyAsync(c->Z, mol->Z, sizeof(double) * n_prod * n_sub, cudaMemcpyDeviceToDevice, ctx->stream));
            gemm_f64(ctx, false, false, n_prod, n_sub, n_prod, 1.0, mol->v, n_prod, c->Z, n_sub, 0.0, c->Zup, n_sub);
        } else if (!cmp && n_sub == n_prod) {
            CUDA_CHECK(cudaMemcpyAsync(c->Zup, mol->v, sizeof(double) * n_prod * n_prod, cudaMemcpyDeviceToDevice, ctx->stream));
            cholesky_lower(ctx, c->Zup, n_prod);
        } else {
            const int nr = cmp ? nr_thr : std::min(n_pair, std::max(5 * n_orb, n_sub));
            c->n_rank = nr;
            if (prec == GW_FP64) {
                T1 = dalloc<double>(ctx, (size_t)n_prod * nr);
                g = dalloc<double>(ctx, (size_t)nr * nr);
                // T1 = v X_r, g = X_r^T v X_r  (X_r = first nr columns of VEFt)
                gemm_f64(ctx, false, false, n_prod, nr, n_prod, 1.0, mol->v, n_prod, VEFt, n_pair, 0.0, T1, nr);
                gemm_f64(ctx, true, false, nr, nr, n_prod, 1.0, VEFt, n_pair, T1, nr, 0.0, g, nr);
                if (cmp) choose_n_sub(g, nullptr, nr);
                Bsel = dalloc<double>(ctx, (size_t)nr * n_sub);
                // binary32 start refined to binary64 accuracy
                eigh_top_scaled(ctx, g, nullptr, nr, n_sub, 6, 1e-13, true, Bsel);
                gemm_f64(ctx, false, false, n_prod, n_sub, nr, 1.0, T1, nr, Bsel, n_sub, 0.0, c->Zup, n_sub);
                // Z = X_r Bsel is only read back: keep its factors, form it on request
                c->Xr = dalloc<double>(ctx, (size_t)n_prod * nr);
                CUDA_CHECK(cudaMemcpy2DAsync(c->Xr, sizeof(double) * nr, VEFt, sizeof(double) * n_pair,
                                             sizeof(double) * nr, n_prod, cudaMemcpyDeviceToDevice, ctx->stream));
                c->Bsel = Bsel;
                Bsel = nullptr;
            } else {
                // mixed: g only feeds the binary32 eigensolver, so it is formed in
                // binary32; the basis Z = X_r B and Zup = v Z are binary32 products
                // of the kept (re-orthonormalised) vectors, scaled by the binary64
                // quotients Z_j^T Zup_j, so that Z^T Zup has a unit diagonal (Z^T v Z
                // with the binary64 v one to binary32 accuracy; no binary64 refinement)
                float* v32 = dalloc<float>(ctx, (size_t)n_prod * n_prod);
                float* X32 = dalloc<float>(ctx, (size_t)n_prod * nr);
                float* T32 = dalloc<float>(ctx, (size_t)n_prod * nr);
                float* g32 = dalloc<float>(ctx, (size_t)nr * nr);
                float* B32 = nullptr;
                float* Z32 = nullptr;
                try {
                    launch_to_f32(ctx, mol->v, v32, (long long)n_prod * n_prod);
                    CUDA_CHECK(cudaMemcpy2DAsync(X32, sizeof(float) * nr, V32, sizeof(float) * n_pair, sizeof(float) * nr,
                                                 n_prod, cudaMemcpyDeviceToDevice, ctx->stream));
                    gemm_f32(ctx, false, false, n_prod, nr, n_prod, 1.f, v32, n_prod, X32, nr, 0.f, T32, nr);
                    gemm_f32(ctx, true, false, nr, nr, n_prod, 1.f, X32, nr, T32, nr, 0.f, g32, nr);
                    ctx_free(ctx, v32); v32 = nullptr;
                    ctx_free(ctx, T32); T32 = nullptr;
                    if (cmp) choose_n_sub(nullptr, g32, nr);
                    Bsel = dalloc<double>(ctx, (size_t)nr * n_sub);
                    eigh_top_scaled(ctx, nullptr, g32, nr, n_sub, 0, 0.0, false, Bsel);
                    ctx_free(ctx, g32); g32 = nullptr;
                    // Z = X_r B (binary32 product; the scaling below is exact for whatever
                    // Z results), then Zup = v Z and the Rayleigh scaling in binary64
                    B32 = dalloc<float>(ctx, (size_t)nr * n_sub);
                    Z32 = dalloc<float>(ctx, (size_t)n_prod * n_sub);
                    launch_to_f32(ctx, Bsel, B32, (long long)nr * n_sub);
                    gemm_f32(ctx, false, false, n_prod, n_sub, nr, 1.f, X32, nr, B32, n_sub, 0.f, Z32, n_sub);
                    c->Z = dalloc<double>(ctx, (size_t)n_prod * n_sub);
                    launch_to_f64(ctx, Z32, c->Z, (long long)n_prod * n_sub);
                    // Zup = v Z in binary32 too (B32 is reused for it)
                    ctx_free(ctx, B32); B32 = nullptr;
                    v32 = dalloc<float>(ctx, (size_t)n_prod * n_prod);
                    B32 = dalloc<float>(ctx, (size_t)n_prod * n_sub);
                    launch_to_f32(ctx, mol->v, v32, (long long)n_prod * n_prod);
                    gemm_f32(ctx, false, false, n_prod, n_sub, n_prod, 1.f, v32, n_prod, Z32, n_sub, 0.f, B32, n_sub);
                    launch_to_f64(ctx, B32, c->Zup, (long long)n_prod * n_sub);
                } catch (...) {
                    ctx_free(ctx, v32); ctx_free(ctx, X32); ctx_free(ctx, T32); ctx_free(ctx, g32);
                    ctx_free(ctx, B32); ctx_free(ctx, Z32);
                    throw;
                }
                ctx_free(ctx, v32); ctx_free(ctx, X32); ctx_free(ctx, B32); ctx_free(ctx, Z32);
                // binary64 Rayleigh quotients Z_j^T Zup_j of the stored pair; the
                // scaling makes them exactly one
                basis_rayleigh_scale(ctx, c->Z, c->Zup, n_prod, n_sub);
            }
        }
        // a2: U^T = Zup^T V^EF  -> [n_sub][n_pair]; the mixed path only ever
        // uses it in binary32, so it is formed in binary32 there
        if (prec == GW_MIXED) {
            float* Zup32 = dalloc<float>(ctx, (size_t)n_prod * n_sub);
            try {
                launch_to_f32(ctx, c->Zup, Zup32, (long long)n_prod * n_sub);
                c->Ut32 = dalloc<float>(ctx, (size_t)n_sub * n_pair);
                // on the FMA units: the tensor cores' binary32 accumulation rounds toward zero,
                // a common shrink of every u_p that chi0 squares and 1 - chi0 amplifies near its poles
                gemm_f32_rn(ctx, true, false, n_sub, n_pair, n_prod, 1.f, Zup32, n_sub, V32, n_pair, 0.f, c->Ut32,
                            n_pair);
            } catch (...) {
                ctx_free(ctx, Zup32);
                throw;
            }
            ctx_free(ctx, Zup32);
            ctx_free(ctx, V32); V32 = nullptr;
            if (poles64) {
                c->Ut = dalloc<double>(ctx, (size_t)n_sub * n_pair);
                gemm_f64(ctx, true, false, n_sub, n_pair, n_prod, 1.0, c->Zup, n_sub, VEFt, n_pair, 0.0, c->Ut, n_pair);
            }
        } else {
            c->Ut = dalloc<double>(ctx, (size_t)n_sub * n_pair);
            gemm_f64(ctx, true, false, n_sub, n_pair, n_prod, 1.0, c->Zup, n_sub, VEFt, n_pair, 0.0, c->Ut, n_pair);
        }
        ctx_free(ctx, VEFt); VEFt = nullptr;
        ctx_free(ctx, T1); T1 = nullptr; ctx_free(ctx, g); g = nullptr;
        ctx_free(ctx, Bsel); Bsel = nullptr;
        ctx_free(ctx, occ); occ = nullptr; ctx_free(ctx, virt); virt = nullptr;
        ctx_free(ctx, rank_of); rank_of = nullptr;
        // a3 + a4: deposit and Cauchy transform by FFT
        if (prec == GW_MIXED) {
            launch_chi0_kk32(ctx, c);
            if (poles64) {
                launch_spectral64(ctx, c);
                ctx_free(ctx, c->Ut); c->Ut = nullptr;
            }
        } else {
            launch_fft_tables(ctx, c);
            launch_chi0_fft(ctx, c);
        }
        ctx_finish(ctx, "gw_build_chi0");
    } catch (...) {
        ctx_free(ctx, VEFt); ctx_free(ctx, V32); ctx_free(ctx, T1); ctx_free(ctx, g); ctx_free(ctx, Bsel);
        ctx_free(ctx, occ); ctx_free(ctx, virt); ctx_free(ctx, rank_of);
        chi0_release(c);
        throw;
    }
    return c;
}

extern "C" gw_status gw_build_chi0(gw_ctx* ctx, const gw_mol* mol, const gw_grid* grid,
                                   gw_precision prec, gw_chi0** out) {
    if (!ctx || !out) return GW_ERR_INVALID_ARG;
    *out = nullptr;
    API_BEGIN(ctx)
    CUDA_CHECK(cudaSetDevice(ctx->device));
    *out = build_chi0(ctx, mol, grid, prec);
    API_END
}

extern "C" gw_status gw_build_chi0_thr(gw_ctx* ctx, const gw_mol* mol, const gw_grid* grid, gw_precision prec,
                                       double e_threshold, double lambda_rel, gw_chi0** out) {
    if (!ctx || !out) return GW_ERR_INVALID_ARG;
    *out = nullptr;
    API_BEGIN(ctx)
    CUDA_CHECK(cudaSetDevice(ctx->device));
    const Compression cmp{e_threshold, lambda_rel};
    *out = build_chi0(ctx, mol, grid, prec, &cmp);
    API_END
}

extern "C" void gw_chi0_free(gw_chi0* c) { chi0_release(c); }

// Second window technique (Sec. 4.2, Eq. win2-for-response, reading R10):
// chi0 on the small window's grid from the large window's build (its pairs,
// basis and U).  Pairs with Delta < lam = (N_s - 1) dws are deposited on the
// small grid and enter with the small broadening; the others are deposited
// on the large grid (the large window's spectral function truncated below
// lam) and enter with the large broadening; one band sum over both blocks of
// bins gives chi0 at the small grid's frequencies.
static gw_chi0* build_small_window(gw_ctx* ctx, const gw_chi0* cl, const gw_grid* gs) {
    REQUIRE(cl && cl->ctx == ctx, "chi0 belongs to another context");
    REQUIRE(!cl->large, "the large window's handle must be a one-window build");
    REQUIRE(gs && gs->n_omega >= 4 && gs->n_omega <= (1 << 15) && gs->d_omega > 0 && std::isfinite(gs->d_omega) &&
                gs->eta > 0 && std::isfinite(gs->eta),
            "small window: n_omega in [4, 32768], positive d_omega and eta");
    REQUIRE(gs->d_omega < cl->grid.d_omega, "the small window's grid must be finer than the large window's");
    const double lam = (double)(gs->n_omega - 1) * gs->d_omega;
    REQUIRE(lam < (double)cl->grid.n_omega * cl->grid.d_omega, "the small window must lie inside the large one");
    const int n_pair = cl->n_pair;
    std::vector<double> delta(n_pair);
    download(ctx, delta.data(), cl->pDelta, n_pair);
    CUDA_CHECK(cudaStreamSynchronize(ctx->stream));
    int P = 0;
    while (P < n_pair && delta[P] < lam) ++P;        // sorted ascending: the small window's pairs lead
    std::vector<double> fs(n_pair, 0.0), fl(n_pair, 0.0);
    std::vector<int> bs(n_pair, 0), bl(n_pair, 0);
    for (int p = 0; p < n_pair; ++p) {
        const double x = delta[p] / (p < P ? gs->d_omega : cl->grid.d_omega);
        const double j = std::floor(x);
        (p < P ? fs : fl)[p] = x - j;
        (p < P ? bs : bl)[p] = (int)j;
    }
    auto segments = [](const std::vector<int>& bins, int p0, int p1, int& jlo, int& nb) {
        jlo = bins[p0];
        nb = bins[p1 - 1] - jlo + 1;
        std::vector<int> seg(nb + 1);
        int p = p0;
        for (int b = 0; b < nb; ++b) {
            while (p < p1 && bins[p] < jlo + b) ++p;
            seg[b] = p;
        }
        seg[nb] = p1;
        return seg;
    };
    int js = 0, nbs = 0, jl = 0, nbl = 0;
    std::vector<int> seg_s, seg_l;
    if (P > 0) seg_s = segments(bs, 0, P, js, nbs);
    if (P < n_pair) seg_l = segments(bl, P, n_pair, jl, nbl);
    const int band_s = P > 0 ? nbs + 1 : 0, band_l = P < n_pair ? nbl + 1 : 0;
    gw_chi0* c = new gw_chi0();
    c->ctx = ctx; c->mol = cl->mol; c->grid = *gs; c->prec = cl->prec;
    c->n_pair = n_pair; c->n_rank = cl->n_rank; c->n_sub = cl->n_sub;
    c->j_lo = js; c->nb_bins = nbs; c->j_hi = js + nbs;
    c->large = cl; c->lam_cut = lam;
    const long long n_el = tri(c->n_sub);
    const size_t rz = c->prec == GW_MIXED ? sizeof(float) : sizeof(double);
    int *dseg_s = nullptr, *dseg_l = nullptr;
    double *dfs = nullptr, *dfl = nullptr;
    void* A = nullptr;
    try {
        const size_t nz = (size_t)c->mol->n_prod * c->n_sub;
        c->Zup = dalloc<double>(ctx, nz);
        CUDA_CHECK(cudaMemcpyAsync(c->Zup, cl->Zup, nz * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
        A = ctx_alloc(ctx, (size_t)(band_s + band_l) * n_el * rz);
        if (band_s) {
            dseg_s = upload(ctx, seg_s.data(), seg_s.size());
            dfs = upload(ctx, fs.data(), fs.size());
            launch_deposit_range(ctx, cl, dseg_s, dfs, nbs, A);
        }
        if (band_l) {
            dseg_l = upload(ctx, seg_l.data(), seg_l.size());
            dfl = upload(ctx, fl.data(), fl.size());
            launch_deposit_range(ctx, cl, dseg_l, dfl, nbl, (char*)A + (size_t)band_s * n_el * rz);
        }
        launch_chi0_kk_2w(ctx, c, A, js, band_s, jl, band_l, cl->grid);
        ctx_finish(ctx, "gw_build_chi0_2w");
    } catch (...) {
        ctx_free(ctx, dseg_s); ctx_free(ctx, dseg_l); ctx_free(ctx, dfs); ctx_free(ctx, dfl); ctx_free(ctx, A);
        chi0_release(c);
        throw;
    }
    ctx_free(ctx, dseg_s); ctx_free(ctx, dseg_l); ctx_free(ctx, dfs); ctx_free(ctx, dfl); ctx_free(ctx, A);
    return c;
}

extern "C" gw_status gw_build_chi0_2w(gw_ctx* ctx, const gw_mol* mol, const gw_grid* small, const gw_grid* large,
                                      gw_precision prec, gw_chi0** small_out, gw_chi0** large_out) {
    if (!ctx || !small_out || !large_out) return GW_ERR_INVALID_ARG;
    *small_out = nullptr;
    *large_out = nullptr;
    API_BEGIN(ctx)
    CUDA_CHECK(cudaSetDevice(ctx->device));
    gw_chi0* cl = build_chi0(ctx, mol, large, prec);
    try {
        *small_out = build_small_window(ctx, cl, small);
    } catch (...) {
        chi0_release(cl);
        throw;
    }
    *large_out = cl;
    API_END
}

// ======================================================================
// a5: screening
// ======================================================================
static void W_release(gw_W* w) {
    if (!w) return;
    ctx_free(w->ctx, w->fac); ctx_free(w->ctx, w->fac32); ctx_free(w->ctx, w->linv); ctx_free(w->ctx, w->piv);
    ctx_free(w->ctx, w->d_pole);
    delete w;
}

// Near-pole policy of the binary32 path (Eq. chi_RPA near the poles of W):
// the spectral weight of chi^RPA_k along 8 fixed pseudo-random directions b,
// s(k) = sum_b |Im b^T (1 - chi0_k)^-1 b|, from the binary32 factors (the
// forms kernel with the b as right-hand sides); frequencies k >= 1 with
// s(k) >= tau max_k s(k) are refactorised in binary64 where consumed.
static void flag_poles(gw_ctx* ctx, gw_W* w, double tau) {
    const gw_chi0* c = w->chi0;
    const int n = c->n_sub, N = c->grid.n_omega, NP = 8;
    std::vector<double> hb((size_t)n * NP);
    uint64_t st = 0x9E3779B97F4A7C15ull;
    for (auto& x : hb) {                    // splitmix64 -> uniform (-1, 1)
        uint64_t z = (st += 0x9E3779B97F4A7C15ull);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        x = 2.0 * ((double)(z >> 11) * 0x1.0p-53) - 1.0;
    }
    double* b = nullptr;
    double* cp = nullptr;
    std::vector<double> hc((size_t)NP * N);
    try {
        b = upload(ctx, hb.data(), hb.size());
        cp = dalloc<double>(ctx, (size_t)NP * N);
        launch_forms(ctx, w, b, NP, cp);
        download(ctx, hc.data(), cp, hc.size());
        CUDA_CHECK(cudaStreamSynchronize(ctx->stream));
    } catch (...) {
        ctx_free(ctx, b); ctx_free(ctx, cp);
        throw;
    }
    ctx_free(ctx, b); ctx_free(ctx, cp);
    std::vector<double> sk(N, 0.0);
    double mx = 0.0;
    for (int k = 1; k < N; ++k) {
        for (int p = 0; p < NP; ++p) sk[k] += std::fabs(hc[(size_t)p * N + k]);
        mx = std::max(mx, sk[k]);
    }
    w->pole_k.clear();
    for (int k = 1; k < N; ++k)
        if (mx > 0.0 && sk[k] >= tau * mx) w->pole_k.push_back(k);
    if (!w->pole_k.empty()) w->d_pole = upload(ctx, w->pole_k.data(), w->pole_k.size());
}

static gw_W* screen_W(gw_ctx* ctx, const gw_chi0* c) {
    REQUIRE(c && c->ctx == ctx, "chi0 belongs to another context");
    gw_W* w = new gw_W();
    w->ctx = ctx; w->chi0 = c;
    const size_t n = c->n_sub, N = c->grid.n_omega;
    try {
        if (c->prec == GW_MIXED) w->fac32 = dalloc<float2>(ctx, N * (size_t)tri(n));     // packed lower triangles
        else w->fac = dalloc<double2>(ctx, N * (size_t)tri(n));
        w->linv = ctx_alloc(ctx, ldlt_linv_bytes((int)n, (int)N, c->prec));
        w->piv = dalloc<double>(ctx, 2 * N);      // [N) ratios, [N, 2N) running min |d|
        launch_ldlt(ctx, w);
        std::vector<double> piv(N);
        download(ctx, piv.data(), w->piv, N);
        ctx_finish(ctx, "gw_screen_W");
        w->min_pivot_ratio = *std::min_element(piv.begin(), piv.end());
        if (c->prec == GW_MIXED && ctx->poles_permille > 0) {
            flag_poles(ctx, w, ctx->poles_permille * 1e-3);
            ctx_finish(ctx, "gw_screen_W");
        }
    } catch (...) {
        W_release(w);
        throw;
    }
    return w;
}

extern "C" gw_status gw_screen_W(gw_ctx* ctx, const gw_chi0* chi0, gw_W** out) {
    if (!ctx || !out) return GW_ERR_INVALID_ARG;
    *out = nullptr;
    API_BEGIN(ctx)
    CUDA_CHECK(cudaSetDevice(ctx->device));
    *out = screen_W(ctx, chi0);
    API_END
}

extern "C" void gw_W_free(gw_W* W) { W_release(W); }

// ======================================================================
// a6-a7: self-energy
// ======================================================================
static void sigma_release(gw_sigma* s) {
    if (!s) return;
    gw_ctx* x = s->ctx;
    ctx_free(x, s->c); ctx_free(x, s->sig); ctx_free(x, s->sigc); ctx_free(x, s->sx); ctx_free(x, s->eks);
    ctx_free(x, s->c2); ctx_free(x, s->sig2); ctx_free(x, s->d_states);
    delete s;
}

static gw_sigma* sigma_diag(gw_ctx* ctx, const gw_W* W, const int* states, int n_states, const gw_W* W2 = nullptr,
                            bool matrix = false) {
    REQUIRE(W && W->ctx == ctx, "W belongs to another context");
    REQUIRE(!matrix || (!W2 && n_states <= dyson_max_states()), "self-energy matrix: one window, at most 16 states");
    REQUIRE(!W2 || (W2->ctx == ctx && W->chi0->large == W2->chi0),
            "the second window's W must be the large window of the first's chi0");
    REQUIRE(W2 || !W->chi0->large, "a small window's W needs its large window (gw_sigma_diag_2w)");
    REQUIRE(states && n_states > 0, "empty state list");
    const gw_chi0* c = W->chi0;
    const gw_mol* mol = c->mol;
    for (int i = 0; i < n_states; ++i) REQUIRE(states[i] >= 0 && states[i] < mol->n_orb, "state index out of range");
    gw_sigma* s = new gw_sigma();
    s->ctx = ctx; s->W = W; s->W2 = W2; s->n_states = n_states; s->states.assign(states, states + n_states);
    const int n_orb = mol->n_orb, n_prod = mol->n_prod, n_sub = c->n_sub, N = c->grid.n_omega;
    const int R = n_states * n_orb;
    s->R = R;
    // sigma grid range: floor(E/d_omega) - (N-1) .. floor(E/d_omega) + N over all states
    const double dw = c->grid.d_omega;
    double imin = std::floor(mol->h_eps.front() / dw), imax = std::floor(mol->h_eps.back() / dw);
    s->j0 = (int)imin - (N - 1);
    s->n_sig = ((int)imax + N) - s->j0 + 1;
    int *Es = nullptr, *Fs = nullptr;
    double *Vnk = nullptr, *Q = nullptr, *T = nullptr;
    try {
        std::vector<int> all(n_orb);
        for (int i = 0; i < n_orb; ++i) all[i] = i;
        Es = upload(ctx, states, n_states);
        Fs = upload(ctx, all.data(), n_orb);
        std::vector<double> eks(n_states);
        for (int i = 0; i < n_states; ++i) eks[i] = mol->h_eps[states[i]];
        s->eks = upload(ctx, eks.data(), n_states);
        // V^{nk}_mu, columns r = i*n_orb + k; q_nk = Zup^T V^{nk}: Q [n_sub][R];
        // T = v V^{nk} for Sigma_x.  The mixed path forms all three in
        // binary32 (its forms read q in binary32) and keeps binary64 copies
        // of V^{nk} and T for the Sigma_x sums.
        Vnk = dalloc<double>(ctx, (size_t)n_prod * R);
        Q = dalloc<double>(ctx, (size_t)n_sub * R);
        T = dalloc<double>(ctx, (size_t)n_prod * R);
        if (c->prec == GW_MIXED) {
            float *Zup32 = nullptr, *V32 = nullptr, *Q32 = nullptr, *v32 = nullptr, *T32 = nullptr;
            try {
                V32 = dalloc<float>(ctx, (size_t)n_prod * R);
                launch_vertex_contract32(ctx, mol, Es, n_states, Fs, n_orb, nullptr, V32, R);
                Zup32 = dalloc<float>(ctx, (size_t)n_prod * n_sub);
                Q32 = dalloc<float>(ctx, (size_t)n_sub * R);
                launch_to_f32(ctx, c->Zup, Zup32, (long long)n_prod * n_sub);
                gemm_f32_rn(ctx, true, false, n_sub, R, n_prod, 1.f, Zup32, n_sub, V32, R, 0.f, Q32, R);   // as U
                launch_to_f64(ctx, Q32, Q, (long long)n_sub * R);
                v32 = dalloc<float>(ctx, (size_t)n_prod * n_prod);
                T32 = dalloc<float>(ctx, (size_t)n_prod * R);
                launch_to_f32(ctx, mol->v, v32, (long long)n_prod * n_prod);
                gemm_f32(ctx, false, false, n_prod, R, n_prod, 1.f, v32, n_prod, V32, R, 0.f, T32, R);
                launch_to_f64(ctx, V32, Vnk, (long long)n_prod * R);
                launch_to_f64(ctx, T32, T, (long long)n_prod * R);
            } catch (...) {
                ctx_free(ctx, Zup32); ctx_free(ctx, V32); ctx_free(ctx, Q32); ctx_free(ctx, v32); ctx_free(ctx, T32);
                throw;
            }
            ctx_free(ctx, Zup32); ctx_free(ctx, V32); ctx_free(ctx, Q32); ctx_free(ctx, v32); ctx_free(ctx, T32);
        } else {
            launch_vertex_contract(ctx, mol, Es, n_states, Fs, n_orb, nullptr, Vnk, R);
            gemm_f64(ctx, true, false, n_sub, R, n_prod, 1.0, c->Zup, n_sub, Vnk, R, 0.0, Q, R);
            gemm_f64(ctx, false, false, n_prod, R, n_prod, 1.0, mol->v, n_prod, Vnk, R, 0.0, T, R);
        }
        // c_nk(s_j); for the matrix, the pairs' right-hand sides q_nk (+ q_mk), then
        // the off-diagonal forms by polarisation
        double* Qf = Q;
        int Rf = R;
        if (matrix) {
            const int S = n_states, P = S * (S + 1) / 2;
            Rf = P * n_orb;
            Qf = dalloc<double>(ctx, (size_t)n_sub * Rf);
            launch_pair_rhs(ctx, Q, S, n_orb, n_sub, Qf);
            s->matrix_S = S;
            s->n_states = P;
            s->R = Rf;
            s->d_states = upload(ctx, states, n_states);
        }
        s->c = dalloc<double>(ctx, (size_t)Rf * N);
        try {
            launch_forms(ctx, W, Qf, Rf, s->c);
            launch_pole_forms(ctx, W, Qf, Rf, s->c);      // near-pole frequencies in binary64 (policy on)
        } catch (...) {
            if (Qf != Q) ctx_free(ctx, Qf);
            throw;
        }
        if (Qf != Q) ctx_free(ctx, Qf);
        if (matrix) launch_offdiag(ctx, s->c, s->matrix_S, n_orb, N);
        if (W2) {
            // second window (R10): the small window's forms for s2 < lam, the large
            // window's for s2 >= lam
            const gw_grid& gl = W2->chi0->grid;
            const int NL = gl.n_omega;
            s->c2 = dalloc<double>(ctx, (size_t)R * NL);
            launch_forms(ctx, W2, Q, R, s->c2);
            launch_pole_forms(ctx, W2, Q, R, s->c2);
            const double lam = c->lam_cut;
            int jcut = 0;
            while (jcut < NL && (double)jcut * gl.d_omega < lam) ++jcut;
            CUDA_CHECK(cudaMemset2DAsync(s->c + (N - 1), sizeof(double) * N, 0, sizeof(double), R, ctx->stream));
            if (jcut > 0)
                CUDA_CHECK(cudaMemset2DAsync(s->c2, sizeof(double) * NL, 0, sizeof(double) * jcut, R, ctx->stream));
            const double dwl = gl.d_omega;
            double jmin = std::floor(mol->h_eps.front() / dwl), jmax = std::floor(mol->h_eps.back() / dwl);
            s->j0_2 = (int)jmin - (NL - 1);
            s->n_sig2 = ((int)jmax + NL) - s->j0_2 + 1;
        }
        // sigma_n(s), Sigma_c grid
        s->sig = dalloc<double>(ctx, (size_t)s->n_states * s->n_sig);
        launch_sigma_grid(ctx, s);
        s->sigc = dalloc<double2>(ctx, (size_t)s->n_states * (2 * N - 1));
        launch_sigma_c(ctx, s);
        if (W2) {
            s->sig2 = dalloc<double>(ctx, (size_t)n_states * s->n_sig2);
            launch_sigma_grid2(ctx, s);
            launch_sigma_c2(ctx, s);
        }
        // Sigma_x = -sum_{k occ} V^{nk} v V^{nk} (matrix: V^{nk} v V^{mk})
        s->sx = dalloc<double>(ctx, s->n_states);
        if (matrix) launch_sigma_x_pairs(ctx, s, Vnk, T, R);
        else launch_sigma_x(ctx, s, Vnk, T, R);
        ctx_finish(ctx, "gw_sigma_diag");
        ctx_free(ctx, Es); ctx_free(ctx, Fs); ctx_free(ctx, Vnk); ctx_free(ctx, Q); ctx_free(ctx, T);
    } catch (...) {
        ctx_free(ctx, Es); ctx_free(ctx, Fs); ctx_free(ctx, Vnk); ctx_free(ctx, Q); ctx_free(ctx, T);
        sigma_release(s);
        throw;
    }
    return s;
}

extern "C" gw_status gw_sigma_diag(gw_ctx* ctx, const gw_W* W, const int* states, int n_states,
                                   gw_sigma** out) {
    if (!ctx || !out) return GW_ERR_INVALID_ARG;
    *out = nullptr;
    API_BEGIN(ctx)
    CUDA_CHECK(cudaSetDevice(ctx->device));
    *out = sigma_diag(ctx, W, states, n_states);
    API_END
}

extern "C" gw_status gw_sigma_diag_2w(gw_ctx* ctx, const gw_W* W_small, const gw_W* W_large, const int* states,
                                      int n_states, gw_sigma** out) {
    if (!ctx || !out || !W_large) return GW_ERR_INVALID_ARG;
    *out = nullptr;
    API_BEGIN(ctx)
    CUDA_CHECK(cudaSetDevice(ctx->device));
    *out = sigma_diag(ctx, W_small, states, n_states, W_large);
    API_END
}

extern "C" gw_status gw_sigma_matrix(gw_ctx* ctx, const gw_W* W, const int* states, int n_states, gw_sigma** out) {
    if (!ctx || !out) return GW_ERR_INVALID_ARG;
    *out = nullptr;
    API_BEGIN(ctx)
    CUDA_CHECK(cudaSetDevice(ctx->device));
    *out = sigma_diag(ctx, W, states, n_states, nullptr, true);
    API_END
}

extern "C" gw_status gw_sigma_matrix_copy(gw_ctx* ctx, const gw_sigma* s, double* sigma_c, double* sigma_x) {
    if (!ctx || !s || !s->matrix_S) return GW_ERR_INVALID_ARG;
    API_BEGIN(ctx)
    CUDA_CHECK(cudaSetDevice(ctx->device));
    const int S = s->matrix_S, P = s->n_states, nk = 2 * s->W->chi0->grid.n_omega - 1;
    std::vector<double2> sc((size_t)P * nk);
    std::vector<double> sx(P);
    download(ctx, sc.data(), s->sigc, sc.size());
    download(ctx, sx.data(), s->sx, P);
    CUDA_CHECK(cudaStreamSynchronize(ctx->stream));
    for (int n = 0; n < S; ++n)
        for (int m = 0; m < S; ++m) {
            const int a = std::min(n, m), b = std::max(n, m);
            const int p = a * S - a * (a - 1) / 2 + (b - a);
            if (sigma_c)
                std::memcpy(reinterpret_cast<double2*>(sigma_c) + ((size_t)n * S + m) * nk, sc.data() + (size_t)p * nk,
                            sizeof(double2) * nk);
            if (sigma_x) sigma_x[n * S + m] = sx[p];
        }
    API_END
}

extern "C" gw_status gw_dyson_dos(gw_ctx* ctx, const gw_sigma* s, const double* vxc, double* dos, double* g_diag) {
    if (!ctx || !s || !s->matrix_S || !dos) return GW_ERR_INVALID_ARG;
    API_BEGIN(ctx)
    CUDA_CHECK(cudaSetDevice(ctx->device));
    const int S = s->matrix_S, P = s->n_states, nk = 2 * s->W->chi0->grid.n_omega - 1;
    // Sigma_x - vxc per pair (vxc NULL: vxc = Sigma_x, the mean field contains exchange)
    std::vector<double> d(P, 0.0);
    if (vxc) {
        std::vector<double> sx(P);
        download(ctx, sx.data(), s->sx, P);
        CUDA_CHECK(cudaStreamSynchronize(ctx->stream));
        for (int n = 0; n < S; ++n)
            for (int m = n; m < S; ++m) {
                const int p = n * S - n * (n - 1) / 2 + (m - n);
                d[p] = sx[p] - vxc[n * S + m];
            }
    }
    double *dd = nullptr, *ddos = nullptr;
    double2* dg = nullptr;
    try {
        dd = upload(ctx, d.data(), d.size());
        ddos = dalloc<double>(ctx, nk);
        if (g_diag) dg = dalloc<double2>(ctx, (size_t)S * nk);
        launch_dyson(ctx, s, dd, s->d_states, ddos, dg);
        download(ctx, dos, ddos, nk);
        if (g_diag) download(ctx, reinterpret_cast<double2*>(g_diag), dg, (size_t)S * nk);
        ctx_finish(ctx, "gw_dyson_dos");
    } catch (...) {
        ctx_free(ctx, dd); ctx_free(ctx, ddos); ctx_free(ctx, dg);
        throw;
    }
    ctx_free(ctx, dd); ctx_free(ctx, ddos); ctx_free(ctx, dg);
    API_END
}

extern "C" void gw_sigma_free(gw_sigma* s) { sigma_release(s); }

// ======================================================================
// a8: quasiparticle equation
// ======================================================================
static void qp_solve(gw_ctx* ctx, const gw_sigma* s, const double* vxc, double* e, double* z, int* st) {
    REQUIRE(s && s->ctx == ctx, "sigma belongs to another context");
    REQUIRE(!s->matrix_S, "a self-energy matrix is solved by gw_dyson_dos");
    REQUIRE(e && z && st, "NULL output array");
    const int ns = s->n_states;
    double* dv = nullptr; double* de = nullptr; double* dz = nullptr; int* ds = nullptr;
    try {
        if (vxc) dv = upload(ctx, vxc, ns);
        de = dalloc<double>(ctx, ns); dz = dalloc<double>(ctx, ns); ds = dalloc<int>(ctx, ns);
        launch_qp(ctx, s, dv, de, dz, ds);
        download(ctx, e, de, ns); download(ctx, z, dz, ns); download(ctx, st, ds, ns);
        ctx_finish(ctx, "gw_qp_solve");
    } catch (...) {
        ctx_free(ctx, dv); ctx_free(ctx, de); ctx_free(ctx, dz); ctx_free(ctx, ds);
        throw;
    }
    ctx_free(ctx, dv); ctx_free(ctx, de); ctx_free(ctx, dz); ctx_free(ctx, ds);
}

extern "C" gw_status gw_qp_solve(gw_ctx* ctx, const gw_sigma* sigma, const double* vxc,
                                 double* e_qp, double* z_factor, int* root_status) {
    if (!ctx) return GW_ERR_INVALID_ARG;
    API_BEGIN(ctx)
    CUDA_CHECK(cudaSetDevice(ctx->device));
    qp_solve(ctx, sigma, vxc, e_qp, z_factor, root_status);
    API_END
}

extern "C" gw_status gw_solve(gw_ctx* ctx, const gw_mol* mol, const gw_grid* grid, gw_precision prec,
                              const int* states, int n_states, const double* vxc, double* e_qp, double* z_factor,
                              int* root_status, double* sigma_x) {
    if (!ctx) return GW_ERR_INVALID_ARG;
    API_BEGIN(ctx)
    CUDA_CHECK(cudaSetDevice(ctx->device));
    gw_chi0* c = nullptr; gw_W* w = nullptr; gw_sigma* s = nullptr;
    try {
        c = build_chi0(ctx, mol, grid, prec);
        w = screen_W(ctx, c);
        s = sigma_diag(ctx, w, states, n_states);
        qp_solve(ctx, s, vxc, e_qp, z_factor, root_status);
        if (sigma_x) {
            download(ctx, sigma_x, s->sx, n_states);
            CUDA_CHECK(cudaStreamSynchronize(ctx->stream));
        }
    } catch (...) {
        sigma_release(s); W_release(w); chi0_release(c);
        throw;
    }
    sigma_release(s); W_release(w); chi0_release(c);
    API_END
}

extern "C" gw_status gw_solve_host(gw_ctx* ctx, const gw_molecule_desc* desc, const gw_grid* grid,
                                   gw_precision prec, const int* states, int n_states,
                                   const double* vxc, double* e_qp, double* z_factor,
                                   int* root_status, double* sigma_x) {
    if (!ctx) return GW_ERR_INVALID_ARG;
    API_BEGIN(ctx)
    CUDA_CHECK(cudaSetDevice(ctx->device));
    gw_mol* m = nullptr; gw_chi0* c = nullptr; gw_W* w = nullptr; gw_sigma* s = nullptr;
    try {
        m = mol_upload(ctx, desc);
        c = build_chi0(ctx, m, grid, prec);
        w = screen_W(ctx, c);
        s = sigma_diag(ctx, w, states, n_states);
        qp_solve(ctx, s, vxc, e_qp, z_factor, root_status);
        if (sigma_x) {
            download(ctx, sigma_x, s->sx, n_states);
            CUDA_CHECK(cudaStreamSynchronize(ctx->stream));
        }
    } catch (...) {
        sigma_release(s); W_release(w); chi0_release(c); mol_release(m);
        throw;
    }
    sigma_release(s); W_release(w); chi0_release(c); mol_release(m);
    API_END
}

// ======================================================================
// read-back
// ======================================================================
extern "C" gw_status gw_chi0_info(const gw_chi0* c, gw_info* out) {
    if (!c || !out) return GW_ERR_INVALID_ARG;
    std::memset(out, 0, sizeof(*out));
    out->n_orb = c->mol->n_orb; out->n_occ = c->mol->n_occ; out->n_prod = c->mol->n_prod;
    out->n_sub = c->n_sub; out->n_pair = c->n_pair; out->n_rank = c->n_rank;
    out->n_omega = c->grid.n_omega; out->j_lo = c->j_lo; out->j_hi = c->j_hi;
    out->precision = (int)c->prec;
    return GW_OK;
}

extern "C" gw_status gw_W_info(const gw_W* W, gw_info* out) {
    if (!W || !out) return GW_ERR_INVALID_ARG;
    gw_status s = gw_chi0_info(W->chi0, out);
    out->min_pivot_ratio = W->min_pivot_ratio;
    out->n_pole = (int)W->pole_k.size();
    return s;
}

extern "C" gw_status gw_W_pole_freqs(const gw_W* W, int* freqs) {
    if (!W || !freqs) return GW_ERR_INVALID_ARG;
    std::copy(W->pole_k.begin(), W->pole_k.end(), freqs);
    return GW_OK;
}

extern "C" gw_status gw_chi0_copy_pairs(gw_ctx* ctx, const gw_chi0* c, int* E, int* F,
                                        double* delta, int* bin, double* frac) {
    if (!ctx || !c) return GW_ERR_INVALID_ARG;
    API_BEGIN(ctx)
    REQUIRE(!c->large, "a small window keeps no pair table; read the large window's");
    CUDA_CHECK(cudaSetDevice(ctx->device));
    if (E) download(ctx, E, c->pE, c->n_pair);
    if (F) download(ctx, F, c->pF, c->n_pair);
    if (delta) download(ctx, delta, c->pDelta, c->n_pair);
    if (bin) download(ctx, bin, c->pBin, c->n_pair);
    if (frac) download(ctx, frac, c->pFrac, c->n_pair);
    CUDA_CHECK(cudaStreamSynchronize(ctx->stream));
    API_END
}

extern "C" gw_status gw_chi0_copy_basis(gw_ctx* ctx, const gw_chi0* c, double* Z, double* Zup) {
    if (!ctx || !c) return GW_ERR_INVALID_ARG;
    API_BEGIN(ctx)
    CUDA_CHECK(cudaSetDevice(ctx->device));
    size_t n = (size_t)c->mol->n_prod * c->n_sub;
    if (Z) {
        REQUIRE(c->Z || c->Bsel, "Z is not formed for the Cholesky (uncompressed) basis; read Zup");
        if (!c->Z) {
            gw_chi0* cm = const_cast<gw_chi0*>(c);      // cached product, same value on every read
            cm->Z = dalloc<double>(ctx, n);
            gemm_f64(ctx, false, false, c->mol->n_prod, c->n_sub, c->n_rank, 1.0, c->Xr, c->n_rank, c->Bsel, c->n_sub,
                     0.0, cm->Z, c->n_sub);
        }
        download(ctx, Z, c->Z, n);
    }
    if (Zup) download(ctx, Zup, c->Zup, n);
    CUDA_CHECK(cudaStreamSynchronize(ctx->stream));
    API_END
}

extern "C" gw_status gw_chi0_copy_U(gw_ctx* ctx, const gw_chi0* c, double* U) {
    if (!ctx || !c || !U) return GW_ERR_INVALID_ARG;
    API_BEGIN(ctx)
    REQUIRE(!c->large, "a small window keeps no U; read the large window's");
    CUDA_CHECK(cudaSetDevice(ctx->device));
    std::vector<double> t((size_t)c->n_sub * c->n_pair);
    if (c->Ut) {
        download(ctx, t.data(), c->Ut, t.size());
    } else {                   // mixed path: binary32 only
        std::vector<float> t32(t.size());
        download(ctx, t32.data(), c->Ut32, t32.size());
        CUDA_CHECK(cudaStreamSynchronize(ctx->stream));
        for (size_t i = 0; i < t.size(); ++i) t[i] = t32[i];
    }
    CUDA_CHECK(cudaStreamSynchronize(ctx->stream));
    for (int m = 0; m < c->n_sub; ++m)
        for (int p = 0; p < c->n_pair; ++p) U[(size_t)p * c->n_sub + m] = t[(size_t)m * c->n_pair + p];
    API_END
}

extern "C" gw_status gw_chi0_copy_spectral(gw_ctx* ctx, const gw_chi0* c, int j0, int nj, double* A) {
    if (!ctx || !c || !A) return GW_ERR_INVALID_ARG;
    API_BEGIN(ctx)
    CUDA_CHECK(cudaSetDevice(ctx->device));
    REQUIRE(!c->large, "spectral weights of a small window are not kept; read the large window's");
    REQUIRE(nj >= 0 && j0 >= 0 && j0 + nj <= c->grid.n_omega, "bin range outside the grid");
    size_t n = (size_t)nj * c->n_sub * c->n_sub;
    double* d = dalloc<double>(ctx, std::max<size_t>(n, 1));
    try {
        launch_spectral_readback(ctx, c, j0, nj, d);
        download(ctx, A, d, n);
        ctx_finish(ctx, "gw_chi0_copy_spectral");
    } catch (...) { ctx_free(ctx, d); throw; }
    ctx_free(ctx, d);
    API_END
}

extern "C" gw_status gw_chi0_copy(gw_ctx* ctx, const gw_chi0* c, int k0, int nk, double* out) {
    if (!ctx || !c || !out) return GW_ERR_INVALID_ARG;
    API_BEGIN(ctx)
    CUDA_CHECK(cudaSetDevice(ctx->device));
    REQUIRE(nk >= 0 && k0 >= 0 && k0 + nk <= c->grid.n_omega, "frequency range outside the grid");
    const size_t n = c->n_sub, pk = (size_t)tri(n);
    std::vector<double2> t(nk * pk);
    if (c->prec == GW_MIXED && c->chi0_32) {
        std::vector<float2> t32(t.size());
        download(ctx, t32.data(), c->chi0_32 + (size_t)k0 * pk, t32.size());
        CUDA_CHECK(cudaStreamSynchronize(ctx->stream));
        for (size_t i = 0; i < t.size(); ++i) t[i] = make_double2(t32[i].x, t32[i].y);
    } else {
        download(ctx, t.data(), c->chi0 + (size_t)k0 * pk, t.size());
        CUDA_CHECK(cudaStreamSynchronize(ctx->stream));
    }
    // packed lower triangle -> full symmetric matrices
    double2* o = reinterpret_cast<double2*>(out);
    for (int k = 0; k < nk; ++k)
        for (size_t i = 0; i < n; ++i)
            for (size_t j = 0; j < n; ++j) {
                size_t a = std::max(i, j), b = std::min(i, j);
                o[(k * n + i) * n + j] = t[k * pk + (size_t)tri(a) + b];
            }
    API_END
}

namespace {
// out[k * ne + i] = chi0_k at packed element e[i], binary64 or binary32 storage
__global__ void k_chi0_elements(const double2* __restrict__ c64, const float2* __restrict__ c32, long long pk, int N,
                                const long long* __restrict__ e, int ne, double2* __restrict__ out) {
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= (long long)N * ne) return;
    const int k = (int)(t / ne), i = (int)(t % ne);
    const long long o = (long long)k * pk + e[i];
    out[t] = c64 ? c64[o] : make_double2(c32[o].x, c32[o].y);
}
}  // namespace

extern "C" gw_status gw_chi0_copy_elements(gw_ctx* ctx, const gw_chi0* c, const int* m, const int* n, int ne,
                                           double* out) {
    if (!ctx || !c || !out || ne <= 0 || !m || !n) return GW_ERR_INVALID_ARG;
    API_BEGIN(ctx)
    CUDA_CHECK(cudaSetDevice(ctx->device));
    std::vector<long long> he(ne);
    for (int i = 0; i < ne; ++i) {
        REQUIRE(m[i] >= 0 && m[i] < c->n_sub && n[i] >= 0 && n[i] < c->n_sub, "element index out of range");
        const long long a = std::max(m[i], n[i]), b = std::min(m[i], n[i]);
        he[i] = tri(a) + b;
    }
    const int N = c->grid.n_omega;
    long long* de = nullptr;
    double2* d = nullptr;
    try {
        de = upload(ctx, he.data(), he.size());
        d = dalloc<double2>(ctx, (size_t)N * ne);
        klaunch(ctx, "k_chi0_elements", k_chi0_elements, div_up((long long)N * ne, 256), 256, 0,
                (const double2*)c->chi0, (const float2*)c->chi0_32, tri(c->n_sub), N, (const long long*)de, ne, d);
        download(ctx, reinterpret_cast<double2*>(out), d, (size_t)N * ne);
        ctx_finish(ctx, "gw_chi0_copy_elements");
    } catch (...) {
        ctx_free(ctx, de); ctx_free(ctx, d);
        throw;
    }
    ctx_free(ctx, de); ctx_free(ctx, d);
    API_END
}

extern "C" gw_status gw_W_copy_pivots(gw_ctx* ctx, const gw_W* W, double* ratio) {
    if (!ctx || !W || !ratio) return GW_ERR_INVALID_ARG;
    API_BEGIN(ctx)
    CUDA_CHECK(cudaSetDevice(ctx->device));
    download(ctx, ratio, W->piv, W->chi0->grid.n_omega);
    CUDA_CHECK(cudaStreamSynchronize(ctx->stream));
    API_END
}

extern "C" gw_status gw_W_copy_chi_rpa(gw_ctx* ctx, const gw_W* W, const int* freqs, int nf, double* out) {
    if (!ctx || !W || !out || (nf > 0 && !freqs)) return GW_ERR_INVALID_ARG;
    API_BEGIN(ctx)
    CUDA_CHECK(cudaSetDevice(ctx->device));
    const gw_chi0* c = W->chi0;
    const size_t n = c->n_sub;
    for (int i = 0; i < nf; ++i) REQUIRE(freqs[i] >= 0 && freqs[i] < c->grid.n_omega, "frequency out of range");
    double2* d = dalloc<double2>(ctx, n * n);
    double2* work = dalloc<double2>(ctx, n * n);
    try {
        for (int i = 0; i < nf; ++i) {
            launch_ldlt_inverse(ctx, W, freqs[i], d, work);   // chi^RPA = M^-1 - I
            download(ctx, reinterpret_cast<double2*>(out) + i * n * n, d, n * n);
        }
        ctx_finish(ctx, "gw_W_copy_chi_rpa");
    } catch (...) { ctx_free(ctx, d); ctx_free(ctx, work); throw; }
    ctx_free(ctx, d); ctx_free(ctx, work);
    API_END
}

extern "C" gw_status gw_W_copy_full(gw_ctx* ctx, const gw_W* W, const int* freqs, int nf, double* out) {
    if (!ctx || !W || !out || (nf > 0 && !freqs)) return GW_ERR_INVALID_ARG;
    API_BEGIN(ctx)
    CUDA_CHECK(cudaSetDevice(ctx->device));
    const gw_chi0* c = W->chi0;
    const int n = c->n_sub, np = c->mol->n_prod;
    for (int i = 0; i < nf; ++i) REQUIRE(freqs[i] >= 0 && freqs[i] < c->grid.n_omega, "frequency out of range");
    double2* d = dalloc<double2>(ctx, (size_t)n * n);
    double2* work = dalloc<double2>(ctx, (size_t)n * n);
    double* re = dalloc<double>(ctx, (size_t)n * n);
    double* im = dalloc<double>(ctx, (size_t)n * n);
    double* T = dalloc<double>(ctx, (size_t)np * n);
    double* Wre = dalloc<double>(ctx, (size_t)np * np);
    double* Wim = dalloc<double>(ctx, (size_t)np * np);
    try {
        std::vector<double> hre((size_t)np * np), him((size_t)np * np);
        for (int i = 0; i < nf; ++i) {
            launch_ldlt_inverse(ctx, W, freqs[i], d, work);
            launch_split_complex(ctx, d, re, im, (size_t)n * n);
            CUDA_CHECK(cudaMemcpyAsync(Wre, c->mol->v, sizeof(double) * np * np, cudaMemcpyDeviceToDevice, ctx->stream));
            gemm_f64(ctx, false, false, np, n, n, 1.0, c->Zup, n, re, n, 0.0, T, n);
            gemm_f64(ctx, false, true, np, np, n, 1.0, T, n, c->Zup, n, 1.0, Wre, np);
            gemm_f64(ctx, false, false, np, n, n, 1.0, c->Zup, n, im, n, 0.0, T, n);
            gemm_f64(ctx, false, true, np, np, n, 1.0, T, n, c->Zup, n, 0.0, Wim, np);
            download(ctx, hre.data(), Wre, hre.size());
            download(ctx, him.data(), Wim, him.size());
            CUDA_CHECK(cudaStreamSynchronize(ctx->stream));
            double2* o = reinterpret_cast<double2*>(out) + (size_t)i * np * np;
            for (size_t q = 0; q < hre.size(); ++q) o[q] = make_double2(hre[q], him[q]);
        }
        ctx_finish(ctx, "gw_W_copy_full");
    } catch (...) {
        ctx_free(ctx, d); ctx_free(ctx, work); ctx_free(ctx, re); ctx_free(ctx, im);
        ctx_free(ctx, T); ctx_free(ctx, Wre); ctx_free(ctx, Wim);
        throw;
    }
    ctx_free(ctx, d); ctx_free(ctx, work); ctx_free(ctx, re); ctx_free(ctx, im);
    ctx_free(ctx, T); ctx_free(ctx, Wre); ctx_free(ctx, Wim);
    API_END
}

extern "C" gw_status gw_sigma_copy(gw_ctx* ctx, const gw_sigma* s, double* c, double* sigma,
                                   double* sigc, double* sigma_x) {
    if (!ctx || !s) return GW_ERR_INVALID_ARG;
    API_BEGIN(ctx)
    CUDA_CHECK(cudaSetDevice(ctx->device));
    const int N = s->W->chi0->grid.n_omega;
    if (c) download(ctx, c, s->c, (size_t)s->R * N);
    if (sigma) download(ctx, sigma, s->sig, (size_t)s->n_states * s->n_sig);
    if (sigc) download(ctx, reinterpret_cast<double2*>(sigc), s->sigc, (size_t)s->n_states * (2 * N - 1));
    if (sigma_x) download(ctx, sigma_x, s->sx, s->n_states);
    CUDA_CHECK(cudaStreamSynchronize(ctx->stream));
    API_END
}

extern "C" gw_status gw_sigma_copy_large(gw_ctx* ctx, const gw_sigma* s, double* c, double* sigma) {
    if (!ctx || !s || !s->W2) return GW_ERR_INVALID_ARG;
    API_BEGIN(ctx)
    CUDA_CHECK(cudaSetDevice(ctx->device));
    const int NL = s->W2->chi0->grid.n_omega;
    if (c) download(ctx, c, s->c2, (size_t)s->R * NL);
    if (sigma) download(ctx, sigma, s->sig2, (size_t)s->n_states * s->n_sig2);
    CUDA_CHECK(cudaStreamSynchronize(ctx->stream));
    API_END
}

extern "C" gw_status gw_sigma_grid_large(const gw_sigma* s, int* j0, int* n_sig) {
    if (!s || !s->W2 || !j0 || !n_sig) return GW_ERR_INVALID_ARG;
    *j0 = s->j0_2;
    *n_sig = s->n_sig2;
    return GW_OK;
}

extern "C" gw_status gw_sigma_grid(const gw_sigma* s, int* j0, int* n_sig) {
    if (!s || !j0 || !n_sig) return GW_ERR_INVALID_ARG;
    *j0 = s->j0;
    *n_sig = s->n_sig;
    return GW_OK;
}
