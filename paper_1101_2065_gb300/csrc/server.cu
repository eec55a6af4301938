// Continuous-batching GW service: jobs (one molecule each, steps a0-a8) are
// queued on the host, admitted in arrival order as soon as their estimated
// device footprint fits the remaining HBM budget, and run by worker threads
// that each own a context (and so a CUDA stream): admitted jobs overlap on
// the GPU.  Kernels reduce in a fixed order and use atomics only for status
// flags, so a job's result does not depend on what runs beside it.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>

#include "internal.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Job {
    long long id = 0;
    // owned copies of the description
    int n_atoms = 0, n_orb = 0, n_occ = 0, n_prod = 0, n_sub = 0;
    std::vector<int> atom_norb, atom_nprod, nbr_ptr, nbr_idx, states;
    std::vector<double> eps, X, vertex, v, vxc;
    std::vector<long long> vertex_off;
    size_t vertex_len = 0;
    const gw_mol* dmol = nullptr;   // device-resident molecule (borrowed), or null: the copies above
    bool has_vxc = false;
    gw_grid grid{};
    gw_precision prec = GW_FP64;
    size_t bytes = 0;
    // state
    int state = 0;            // 0 queued, 1 running, 2 done
    gw_status status = GW_OK;
    std::string err;
    std::vector<double> e_qp, z, sx;
    std::vector<int> root;
    Clock::time_point t_submit, t_start, t_end;
};

}  // namespace

struct gw_server {
    int device = 0;
    size_t budget = 0, in_flight = 0;
    bool stop = false;
    long long next_id = 0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<std::shared_ptr<Job>> queue;
    std::unordered_map<long long, std::shared_ptr<Job>> jobs;
    std::vector<std::thread> workers;
    std::vector<gw_ctx*> ctxs;
};

// Device bytes a job holds at its peak.  The phases of a solve do not hold
// their buffers at the same time: basis and U (V^EF and its binary32 copy,
// eigensolver work), chi0 (U, spectral weights A, chi0), then W and Sigma
// (chi0, U, factors, block inverses, forms right-hand sides); the molecule
// stays resident throughout.
static size_t job_bytes(const Job& j) {
    const size_t N = j.grid.n_omega, n = j.n_sub, np = j.n_prod, no = j.n_orb;
    if (j.n_occ <= 0 || j.n_occ >= j.n_orb) return ~size_t(0) / 4;
    const size_t n_pair = (size_t)j.n_occ * (j.n_orb - j.n_occ);
    const size_t cz = j.prec == GW_MIXED ? sizeof(float2) : sizeof(double2);
    const size_t rz = cz / 2;                                        // real element of the working precision
    const size_t n_rank = std::min(n_pair, std::max<size_t>(5 * no, n));
    const size_t R = (size_t)j.states.size() * no;
    const size_t pk = n * (n + 1) / 2;                               // packed triangle
    const double span = j.eps.empty() ? 0.0 : j.eps.back() - j.eps.front();
    const size_t band = (size_t)(span / j.grid.d_omega) + 3;         // spectral bins (upper bound)
    const size_t mol = np * np * 8 + j.vertex_len * 8 + no * no * 8;
    const size_t U = n * n_pair * rz;
    const size_t basis = np * n_pair * (j.prec == GW_MIXED ? 4 : 8) + U + 12 * n_rank * n_rank * 8 + 3 * np * n * 8;
    const size_t chi0 = U + band * pk * rz + N * pk * cz;
    const size_t screen = U + 2 * N * pk * cz + N * (n + 32) * 32 * cz +
                          std::min<size_t>((size_t)2 << 30, (N ? N - 1 : 0) * n * R * cz) + 3 * np * R * 8;
    const size_t b = mol + std::max(basis, std::max(chi0, screen));
    return b + b / 8 + (64u << 20);
}

static void run_job(gw_ctx* ctx, Job& j) {
    const int nst = (int)j.states.size();
    if (j.dmol) {
        j.e_qp.assign(nst, 0.0); j.z.assign(nst, 0.0); j.sx.assign(nst, 0.0); j.root.assign(nst, 0);
        j.status = gw_solve(ctx, j.dmol, &j.grid, j.prec, j.states.data(), nst, j.has_vxc ? j.vxc.data() : nullptr,
                            j.e_qp.data(), j.z.data(), j.root.data(), j.sx.data());
        if (j.status != GW_OK) j.err = gw_last_error(ctx);
        return;
    }
    gw_molecule_desc d{};
    d.n_atoms = j.n_atoms; d.n_orb = j.n_orb; d.n_occ = j.n_occ; d.n_prod = j.n_prod; d.n_sub = j.n_sub;
    d.atom_norb = j.atom_norb.data(); d.atom_nprod = j.atom_nprod.data();
    d.nbr_ptr = j.nbr_ptr.data(); d.nbr_idx = j.nbr_idx.empty() ? nullptr : j.nbr_idx.data();
    d.eps = j.eps.data(); d.X = j.X.data(); d.vertex = j.vertex.data(); d.vertex_off = j.vertex_off.data();
    d.v = j.v.data(); d.Z = nullptr;
    const int ns = (int)j.states.size();
    j.e_qp.assign(ns, 0.0); j.z.assign(ns, 0.0); j.sx.assign(ns, 0.0); j.root.assign(ns, 0);
    j.status = gw_solve_host(ctx, &d, &j.grid, j.prec, j.states.data(), ns, j.has_vxc ? j.vxc.data() : nullptr,
                             j.e_qp.data(), j.z.data(), j.root.data(), j.sx.data());
    if (j.status != GW_OK) j.err = gw_last_error(ctx);
}

static void worker_loop(gw_server* s, int w) {
    gw_ctx* ctx = s->ctxs[w];
    for (;;) {
        std::shared_ptr<Job> job;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            // admit the head of the queue once its footprint fits (arrival order, no overtaking)
            s->cv_work.wait(lk, [&] {
                return s->stop || (!s->queue.empty() && s->in_flight + s->queue.front()->bytes <= s->budget);
            });
            if (s->stop) return;
            job = s->queue.front();
            s->queue.pop_front();
            s->in_flight += job->bytes;
            job->state = 1;
            job->t_start = Clock::now();
        }
        cudaSetDevice(s->device);
        run_job(ctx, *job);
        {
            std::lock_guard<std::mutex> lk(s->mu);
            s->in_flight -= job->bytes;
            job->t_end = Clock::now();
            job->state = 2;
        }
        s->cv_work.notify_all();
        s->cv_done.notify_all();
    }
}

extern "C" gw_status gw_server_create(gw_server** out, int device, int n_workers, size_t hbm_budget_bytes) {
    if (!out || n_workers < 1 || n_workers > 64) return GW_ERR_INVALID_ARG;
    *out = nullptr;
    gw_server* s = new gw_server();
    s->device = device;
    s->budget = hbm_budget_bytes ? hbm_budget_bytes : ~size_t(0) / 2;
    for (int w = 0; w < n_workers; ++w) {
        gw_ctx* c = nullptr;
        gw_status st = gw_ctx_create(&c, device, 0, nullptr);
        if (st != GW_OK) {
            for (auto x : s->ctxs) gw_ctx_destroy(x);
            delete s;
            return st;
        }
        s->ctxs.push_back(c);
    }
    for (int w = 0; w < n_workers; ++w) s->workers.emplace_back(worker_loop, s, w);
    *out = s;
    return GW_OK;
}

extern "C" void gw_server_destroy(gw_server* s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        // jobs that never started end as cancelled (a wait on them returns at once)
        for (auto& j : s->queue) {
            j->state = 2;
            j->status = GW_ERR_CANCELLED;
            j->err = "server destroyed before the job started";
            j->t_start = j->t_end = Clock::now();
        }
        s->queue.clear();
    }
    s->cv_work.notify_all();
    s->cv_done.notify_all();
    for (auto& t : s->workers) t.join();
    for (auto c : s->ctxs) gw_ctx_destroy(c);
    delete s;
}

extern "C" gw_status gw_server_submit(gw_server* s, const gw_molecule_desc* d, const gw_grid* grid,
                                      gw_precision prec, const int* states, int n_states, const double* vxc,
                                      long long* job_id) {
    if (!s || !d || !grid || !states || n_states <= 0 || !job_id) return GW_ERR_INVALID_ARG;
    if (d->n_atoms <= 0 || d->n_orb <= 1 || d->n_prod <= 0 || !d->atom_norb || !d->atom_nprod || !d->nbr_ptr ||
        !d->eps || !d->X || !d->vertex || !d->vertex_off || !d->v)
        return GW_ERR_INVALID_ARG;
    auto j = std::make_shared<Job>();
    j->n_atoms = d->n_atoms; j->n_orb = d->n_orb; j->n_occ = d->n_occ; j->n_prod = d->n_prod; j->n_sub = d->n_sub;
    j->atom_norb.assign(d->atom_norb, d->atom_norb + d->n_atoms);
    j->atom_nprod.assign(d->atom_nprod, d->atom_nprod + d->n_atoms);
    j->nbr_ptr.assign(d->nbr_ptr, d->nbr_ptr + d->n_atoms + 1);
    const int nnz = d->nbr_ptr[d->n_atoms];
    if (nnz < 0 || (nnz > 0 && !d->nbr_idx)) return GW_ERR_INVALID_ARG;
    j->nbr_idx.assign(d->nbr_idx, d->nbr_idx + nnz);
    j->eps.assign(d->eps, d->eps + d->n_orb);
    j->X.assign(d->X, d->X + (size_t)d->n_orb * d->n_orb);
    j->vertex_off.assign(d->vertex_off, d->vertex_off + d->n_prod + 1);
    if (j->vertex_off.back() < 0) return GW_ERR_INVALID_ARG;
    j->vertex.assign(d->vertex, d->vertex + j->vertex_off.back());
    j->vertex_len = j->vertex.size();
    j->v.assign(d->v, d->v + (size_t)d->n_prod * d->n_prod);
    j->states.assign(states, states + n_states);
    if (vxc) { j->vxc.assign(vxc, vxc + n_states); j->has_vxc = true; }
    j->grid = *grid;
    j->prec = prec;
    j->bytes = job_bytes(*j);
    if (j->bytes > s->budget) return GW_ERR_ADMISSION;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        j->id = s->next_id++;
        j->t_submit = Clock::now();
        s->jobs[j->id] = j;
        s->queue.push_back(j);
        *job_id = j->id;
    }
    s->cv_work.notify_all();
    return GW_OK;
}

extern "C" gw_status gw_server_submit_resident(gw_server* s, const gw_mol* mol, const gw_grid* grid,
                                               gw_precision prec, const int* states, int n_states,
                                               const double* vxc, long long* job_id) {
    if (!s || !mol || !grid || !states || n_states <= 0 || !job_id) return GW_ERR_INVALID_ARG;
    auto j = std::make_shared<Job>();
    j->dmol = mol;
    j->n_atoms = mol->n_atoms; j->n_orb = mol->n_orb; j->n_occ = mol->n_occ; j->n_prod = mol->n_prod;
    j->n_sub = mol->n_sub;
    j->eps = mol->h_eps;                     // the energy span sizes the admission estimate
    j->vertex_len = mol->vertex_len;
    j->states.assign(states, states + n_states);
    if (vxc) { j->vxc.assign(vxc, vxc + n_states); j->has_vxc = true; }
    j->grid = *grid;
    j->prec = prec;
    j->bytes = job_bytes(*j);
    if (j->bytes > s->budget) return GW_ERR_ADMISSION;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        j->id = s->next_id++;
        j->t_submit = Clock::now();
        s->jobs[j->id] = j;
        s->queue.push_back(j);
        *job_id = j->id;
    }
    s->cv_work.notify_all();
    return GW_OK;
}

extern "C" gw_status gw_server_profile(gw_server* s, int enable, const char* kernel_name) {
    if (!s) return GW_ERR_INVALID_ARG;
    for (auto c : s->ctxs) {
        gw_status st = gw_ctx_profile(c, enable, kernel_name);
        if (st != GW_OK) return st;
    }
    return GW_OK;
}

extern "C" gw_status gw_server_profile_get(gw_server* s, const char* kernel_name, double* total_ms,
                                           long long* launches) {
    if (!s || !kernel_name || !total_ms || !launches) return GW_ERR_INVALID_ARG;
    *total_ms = 0.0;
    *launches = 0;
    for (auto c : s->ctxs) {
        double ms = 0.0;
        long long n = 0;
        gw_status st = gw_ctx_profile_get(c, kernel_name, &ms, &n);
        if (st != GW_OK) return st;
        *total_ms += ms;
        *launches += n;
    }
    return GW_OK;
}

extern "C" long long gw_server_launch_count(const gw_server* s) {
    if (!s) return 0;
    long long n = 0;
    for (auto c : s->ctxs) n += gw_ctx_launch_count(c);
    return n;
}

extern "C" int gw_server_poll(gw_server* s, long long job_id) {
    if (!s) return GW_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->jobs.find(job_id);
    if (it == s->jobs.end()) return GW_ERR_INVALID_ARG;
    const Job& j = *it->second;
    if (j.state == 2 && j.status != GW_OK) return j.status;
    return j.state;
}

extern "C" gw_status gw_server_wait(gw_server* s, long long job_id, int timeout_ms, double* e_qp, double* z_factor,
                                    int* root_status, double* sigma_x, double* times_ms, char* err,
                                    size_t err_len) {
    if (!s) return GW_ERR_INVALID_ARG;
    std::shared_ptr<Job> j;
    {
        std::unique_lock<std::mutex> lk(s->mu);
        auto it = s->jobs.find(job_id);
        if (it == s->jobs.end()) return GW_ERR_INVALID_ARG;
        j = it->second;
        auto done = [&] { return j->state == 2; };
        if (timeout_ms < 0) s->cv_done.wait(lk, done);
        else if (!s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), done)) return GW_ERR_TIMEOUT;
        s->jobs.erase(job_id);
    }
    const size_t ns = j->states.size();
    if (j->status == GW_OK) {
        if (e_qp) std::memcpy(e_qp, j->e_qp.data(), ns * sizeof(double));
        if (z_factor) std::memcpy(z_factor, j->z.data(), ns * sizeof(double));
        if (root_status) std::memcpy(root_status, j->root.data(), ns * sizeof(int));
        if (sigma_x) std::memcpy(sigma_x, j->sx.data(), ns * sizeof(double));
    }
    if (times_ms) {
        using ms = std::chrono::duration<double, std::milli>;
        times_ms[0] = ms(j->t_start - j->t_submit).count();
        times_ms[1] = ms(j->t_end - j->t_start).count();
        times_ms[2] = ms(j->t_end - j->t_submit).count();
    }
    if (err && err_len) {
        std::strncpy(err, j->err.c_str(), err_len - 1);
        err[err_len - 1] = '\0';
    }
    return j->status;
}

extern "C" size_t gw_server_job_bytes(const gw_molecule_desc* d, const gw_grid* grid, gw_precision prec,
                                      int n_states) {
    if (!d || !grid || !d->vertex_off || !d->eps || d->n_orb <= 0 || n_states < 0) return 0;
    Job j;
    j.n_orb = d->n_orb; j.n_occ = d->n_occ; j.n_prod = d->n_prod; j.n_sub = d->n_sub;
    j.eps.assign(d->eps, d->eps + d->n_orb);     // the energy span sizes the spectral band, as at submission
    j.grid = *grid; j.prec = prec;
    j.vertex_len = (size_t)d->vertex_off[d->n_prod];
    j.states.resize(n_states);
    return job_bytes(j);
}
