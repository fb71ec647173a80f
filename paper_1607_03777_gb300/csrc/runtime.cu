// Batched and served Stokes solves: many independent problems of different
// mesh sizes, degrees and viscosity fields on one GPU.
//
// Each in-flight solve owns a CUDA stream, its device-resident multigrid and
// Krylov state and a captured V-cycle graph; solves in flight at the same
// time overlap on the device.  The server admits queued requests in arrival
// order whenever a slot is free and the request's device footprint fits in
// the remaining budget, so requests that arrive while others run join as
// capacity frees up (continuous batching).  A head request that does not fit
// yet does not hold up smaller ones behind it: the first queued request that
// fits runs ahead of it (backfilling), at most 4 x slots times per head
// request, after which the head is reserved and runs as soon as memory frees.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdlib>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>

#include "admission.h"
#include "sip_solver.h"

using sip::Error;

namespace {

double wall_ms() {
    using namespace std::chrono;
    return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

}  // namespace

namespace sip {

// Device bytes of a problem after its first solve (multigrid, FGMRES basis
// of `restart` vectors, work vectors), from the sizes alone.
int64_t estimate_problem_bytes(const sip_problem_desc& d, int restart) {
    const int64_t ne = int64_t(d.nx) * d.ny;
    const int64_t n = d.k + 1, nb = 2 * n * n, mp = int64_t(d.k) * d.k;
    const int64_t n_u = ne * nb, n_p = ne * mp, nk = n_u + n_p;
    const bool mixed = d.precision != SIP_PREC_FP64;
    const int64_t w = mixed ? 4 : 8;
    int64_t b = ne * (8 + 4 + 8 + 4);                      // eta, eta_f, 1/eta (FP64, FP32)
    // multigrid: block inverses (class + unique worst case is bounded by the
    // elements with a stiffer neighbour; count them all), work vectors
    b += 16 * nb * nb * w + ne * nb * nb * w / 4;
    b += 11 * n_u * w + 16 * ne * w + ne * 8;
    int64_t nv = int64_t(d.nx + 1) * (d.ny + 1);
    for (int l = 0; l <= d.n_hlevels; ++l) {
        b += nv * (36 + 8) * w + nv * 36 * 8;             // stencils (+ FP64 set-up copy)
        nv = nv / 4 + 1;
    }
    b += int64_t(d.eig_iters + 1) * n_u * 8;               // Arnoldi basis of the set-up
    b += int64_t(2 * restart + 1) * nk * 8 + 8 * nk * 8;  // FGMRES V, Z and work vectors
    b += 4 * n_u * 8;                                      // FP64 inner Krylov vectors
    return b;
}

int64_t estimate_problem_bytes(const sip_problem_desc& d, const sip_solve_opts& o) {
    int64_t b = estimate_problem_bytes(d, std::max(1, std::min(o.restart, o.max_outer)));
    const int64_t ne = int64_t(d.nx) * d.ny;
    const int64_t n = d.k + 1, n_u = ne * 2 * n * n, nk = n_u + ne * int64_t(d.k) * d.k;
    if (o.inner_krylov == 3) b += 2 * int64_t(o.inner_restart) * n_u * 8;   // GCR directions
    if (o.refine > 0) b += ne * 16 + 3 * nk * 16 + n_u * 16 + 2 * nk * 8;  // refinement
    return b;
}

}  // namespace sip

// ------------------------------------------------------------------ batch
namespace {

struct Job {
    sip_problem* prob;
    const double* f;
    double* u;
    double* p;
    sip_solve_report* rep;
    sip_status st = SIP_OK;
    std::string err;
};

// Worker streams of batched solves, per device and worker slot, created once
// and never destroyed: buffers a batched solve allocates belong to the
// caller's problem and are ordered on these streams for the problem's life.
cudaStream_t batch_stream(int device, int slot) {
    static std::mutex mu;
    static std::map<std::pair<int, int>, cudaStream_t> streams;
    std::lock_guard<std::mutex> lk(mu);
    auto it = streams.find({device, slot});
    if (it != streams.end()) return it->second;
    cudaStream_t s = nullptr;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        throw Error(SIP_ERR_CUDA, "batch worker stream creation failed");
    }
    streams[{device, slot}] = s;
    return s;
}

void run_jobs(int device, std::vector<Job>& jobs, const sip_solve_opts& o, int n_streams) {
    std::atomic<size_t> next{0};
    const double deadline = o.time_limit_ms > 0.0 ? sip::steady_ms() + o.time_limit_ms : 0.0;
    auto worker = [&](int slot) {
        cudaSetDevice(device);
        cudaStream_t s = nullptr;
        try {
            s = batch_stream(device, slot);
        } catch (const Error& e) {
            for (size_t i = next++; i < jobs.size(); i = next++) {
                jobs[i].st = e.status;
                jobs[i].err = e.what();
                if (jobs[i].rep) jobs[i].rep->status = e.status;
            }
            return;
        }
        sip::AllocStreamScope scope(s);
        const sip::StopScope stop(deadline, nullptr);
        for (size_t i = next++; i < jobs.size(); i = next++) {
            Job& j = jobs[i];
            try {
                sip_solve_report local{};
                j.st = sip::solve_dispatch(j.prob, j.f, nullptr, j.u, j.p, o, j.rep ? j.rep : &local, s);
            } catch (const Error& e) {
                j.st = e.status;
                j.err = e.what();
                if (j.rep) j.rep->status = e.status;
            } catch (const std::exception& e) {
                j.st = SIP_ERR_CUDA;
                j.err = e.what();
                if (j.rep) j.rep->status = SIP_ERR_CUDA;
            }
        }
        cudaStreamSynchronize(s);
    };
    std::vector<std::thread> pool;
    const int nt = std::max(1, std::min<int>(n_streams, int(jobs.size())));
    for (int t = 0; t < nt; ++t) pool.emplace_back(worker, t);
    for (auto& t : pool) t.join();
}

// Whether the jobs can share batched inner solves: one V-cycle precision
// (FP64, or FP32 with the FP64 inner iterate), the default inner method and
// stopping test on the device loop, the Q^2_1 coarse space with at least one
// h-coarsening, degree <= 5 and one smoothing schedule.
bool groupable(const std::vector<Job>& jobs, const sip_solve_opts& o) {
    if (jobs.empty() || o.inner_loop != 0 || o.inner_norm != 0 || o.inner_krylov == 3) return false;
    const sip_problem_desc& d0 = jobs[0].prob->desc;
    const bool mixed = d0.precision == SIP_PREC_MIXED;
    if (d0.precision != SIP_PREC_FP64 && !mixed) return false;
    if (o.inner_krylov == 1 && mixed) return false;      // PCG on the FP32 V-cycle
    if (o.inner_krylov == 2 && !mixed) return false;     // FCG on the FP64 V-cycle
    for (const Job& j : jobs) {
        const sip_problem_desc& d = j.prob->desc;
        if (d.precision != d0.precision || d.coarse != SIP_COARSE_Q1 || d.n_hlevels < 1 ||
            d.n_hlevels > 11 || d.k > 5 || d.cheb_steps_p != d0.cheb_steps_p ||
            d.cheb_steps_h != d0.cheb_steps_h || d.cheb_steps_p < 1 || d.cheb_steps_p > 8 ||
            d.cheb_steps_h < 2 || d.cheb_steps_h > 8)
            return false;
    }
    return true;
}

// Groups of up to `width` jobs solved in lockstep: one host thread per job
// runs its outer Krylov method; the inner solves of a group are batched
// (batch.cu).  Groups run one after the other.
void run_jobs_grouped(int device, std::vector<Job>& jobs, const sip_solve_opts& o, int width) {
    const double deadline = o.time_limit_ms > 0.0 ? sip::steady_ms() + o.time_limit_ms : 0.0;
    const bool mixed = jobs[0].prob->desc.precision == SIP_PREC_MIXED;
    for (size_t g0 = 0; g0 < jobs.size(); g0 += size_t(width)) {
        const size_t g1 = std::min(jobs.size(), g0 + size_t(width));
        std::vector<sip_problem*> probs;
        for (size_t i = g0; i < g1; ++i) probs.push_back(jobs[i].prob);
        std::unique_ptr<sip::BatchCollector, void (*)(sip::BatchCollector*)> col(
            sip::make_collector(probs, mixed, o.inner_rtol, o.max_inner), sip::free_collector);
        auto worker = [&](size_t i) {
            Job& j = jobs[i];
            cudaSetDevice(device);
            sip::batch_collector() = col.get();
            struct Leave {
                sip::BatchCollector* c;
                sip_problem* p;
                ~Leave() {
                    sip::batch_collector() = nullptr;
                    sip::collector_leave(c, p);
                }
            } leave{col.get(), j.prob};
            try {
                const cudaStream_t s = batch_stream(device, int(i - g0));
                sip::AllocStreamScope scope(s);
                const sip::StopScope stop(deadline, nullptr);
                sip_solve_report local{};
                j.st = sip::solve_dispatch(j.prob, j.f, nullptr, j.u, j.p, o, j.rep ? j.rep : &local, s);
                cudaStreamSynchronize(s);
            } catch (const Error& e) {
                j.st = e.status;
                j.err = e.what();
                if (j.rep) j.rep->status = e.status;
            } catch (const std::exception& e) {
                j.st = SIP_ERR_CUDA;
                j.err = e.what();
                if (j.rep) j.rep->status = SIP_ERR_CUDA;
            }
        };
        std::vector<std::thread> pool;
        for (size_t i = g0; i < g1; ++i) pool.emplace_back(worker, i);
        for (auto& t : pool) t.join();
    }
}

}  // namespace

// ------------------------------------------------------------------ server
struct ServerRequest {
    uint64_t id = 0;
    sip_problem_desc desc{};
    std::vector<double> eta, rho;
    double g = 0.0;
    double* u_host = nullptr;
    double* p_host = nullptr;
    sip_solve_opts opts{};
    int64_t bytes = 0;
    double t_submit = 0.0;
    int bypassed = 0;   // requests admitted ahead of this one while it was the head
    std::shared_ptr<volatile bool> cancel = std::make_shared<volatile bool>(false);
};

struct ServerDone {
    uint64_t id;
    sip_solve_report rep;
};

struct sip_server {
    sip_ctx* ctx = nullptr;
    int64_t budget = 0;
    int64_t in_use = 0;
    int slots = 0;
    int busy = 0;
    bool stop = false;
    std::mutex mu;
    std::condition_variable cv_work, cv_idle;
    std::deque<ServerRequest> queue;
    std::vector<ServerDone> done;
    std::vector<std::thread> workers;
    std::vector<double> latencies_ms;
    std::map<uint64_t, std::shared_ptr<volatile bool>> running;   // cancel flags by id

    void worker_loop();
    sip_status solve_one(ServerRequest& r, cudaStream_t s, sip_solve_report& rep);
    // index of the queued request to admit now, or -1 (called with mu held)
    int pick() const { return sip::admission_pick(queue, in_use, budget, 4 * slots); }
};

sip_status sip_server::solve_one(ServerRequest& r, cudaStream_t s, sip_solve_report& rep) {
    sip_problem* prob = nullptr;
    sip_problem_desc d = r.desc;
    d.eta_host = r.eta.data();
    sip_status st = sip_problem_create(ctx, &d, &prob);
    if (st != SIP_OK) return st;
    double *f = nullptr, *u = nullptr, *p = nullptr, *rho = nullptr;
    try {
        const size_t n_u = size_t(prob->n_u), n_p = size_t(prob->n_p), ne = size_t(prob->ne);
        SIP_CUDA(cudaMallocAsync(&f, n_u * sizeof(double), s));
        SIP_CUDA(cudaMallocAsync(&u, n_u * sizeof(double), s));
        SIP_CUDA(cudaMallocAsync(&p, n_p * sizeof(double), s));
        SIP_CUDA(cudaMallocAsync(&rho, ne * sizeof(double), s));
        SIP_CUDA(cudaMemcpyAsync(rho, r.rho.data(), ne * sizeof(double), cudaMemcpyHostToDevice, s));
        sip::launch_rhs_body_force(prob->k, prob->geom, rho, r.g, f, s);
        st = sip::solve_dispatch(prob, f, nullptr, u, p, r.opts, &rep, s);
        SIP_CUDA(cudaMemcpyAsync(r.u_host, u, n_u * sizeof(double), cudaMemcpyDeviceToHost, s));
        SIP_CUDA(cudaMemcpyAsync(r.p_host, p, n_p * sizeof(double), cudaMemcpyDeviceToHost, s));
        SIP_CUDA(cudaStreamSynchronize(s));
    } catch (const Error& e) {
        st = e.status;
    } catch (const std::exception&) {
        st = SIP_ERR_CUDA;
    }
    for (double* q : {f, u, p, rho})
        if (q) cudaFreeAsync(q, s);
    // all of this request's work ran on s: wait for s only (no device-wide
    // synchronisation), then return the buffers to the stream-ordered pool
    cudaStreamSynchronize(s);
    delete prob;
    return st;
}

void sip_server::worker_loop() {
    cudaSetDevice(ctx->device);
    cudaStream_t s = nullptr;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        s = nullptr;
    }
    sip::AllocStreamScope scope(s);
    for (;;) {
        ServerRequest r;
        {
            std::unique_lock<std::mutex> lk(mu);
            // admission in arrival order with bounded backfilling (pick)
            int i = -1;
            cv_work.wait(lk, [&] {
                i = pick();
                return stop || i >= 0;
            });
            if (stop && queue.empty()) break;
            if (queue.empty()) continue;
            if (i < 0) i = 0;   // stopping: drain in order
            if (i > 0) ++queue.front().bypassed;
            r = std::move(queue[size_t(i)]);
            queue.erase(queue.begin() + i);
            in_use += r.bytes;
            ++busy;
            running[r.id] = r.cancel;
        }
        sip_solve_report rep{};
        sip_status st = SIP_OK;
        const double deadline = r.opts.time_limit_ms > 0.0 ? r.t_submit + r.opts.time_limit_ms : 0.0;
        if (deadline > 0.0 && wall_ms() > deadline) {
            st = SIP_ERR_TIMEOUT;   // expired while queued: not solved
        } else if (*r.cancel) {
            st = SIP_ERR_CANCELLED;
        } else {
            const sip::StopScope stop(deadline, r.cancel.get());
            st = solve_one(r, s, rep);
        }
        rep.status = st;
        const double lat = wall_ms() - r.t_submit;
        {
            std::lock_guard<std::mutex> lk(mu);
            running.erase(r.id);
            in_use -= r.bytes;
            --busy;
            rep.solve_ms = lat;   // for served requests: submit-to-result latency
            done.push_back({r.id, rep});
            latencies_ms.push_back(lat);
        }
        cv_work.notify_all();
        cv_idle.notify_all();
    }
    if (s) cudaStreamDestroy(s);
}

extern "C" {

namespace {

sip_status solve_batch_impl(sip_ctx* ctx, int n, sip_problem* const* probs,
                            const double* const* f_u, double* const* u, double* const* p,
                            const sip_solve_opts* opts, sip_solve_report* reports, int n_streams,
                            bool grouped) {
    if (!ctx) return SIP_ERR_INVALID_ARG;
    if (n < 0 || (n > 0 && (!probs || !f_u || !u || !p))) {
        ctx->err = "bad batch arguments";
        return SIP_ERR_INVALID_ARG;
    }
    sip_solve_opts o;
    sip_solve_opts_default(&o);
    if (opts) o = *opts;
    std::vector<Job> jobs(n);
    for (int i = 0; i < n; ++i) {
        if (!probs[i] || !f_u[i] || !u[i] || !p[i] || probs[i]->ctx != ctx) {
            ctx->err = "bad batch entry " + std::to_string(i);
            return SIP_ERR_INVALID_ARG;
        }
        try {
            sip::require_valid_opts(o, probs[i]->desc.precision);
        } catch (const sip::Error& e) {
            ctx->err = e.what();
            return SIP_ERR_INVALID_ARG;
        }
        jobs[i] = Job{probs[i], f_u[i], u[i], p[i], reports ? &reports[i] : nullptr};
    }
    if (grouped) {
        if (n > 0 && !groupable(jobs, o)) {
            ctx->err = "grouped batch: one precision (FP64 or mixed), the default inner method "
                       "and stopping test on the device loop, the Q^2_1 coarse space with 1..11 "
                       "h-coarsenings, k <= 5 and one smoothing schedule (2..8 h-level steps)";
            return SIP_ERR_INVALID_ARG;
        }
        if (n > 0) run_jobs_grouped(ctx->device, jobs, o, n_streams < 1 ? 32 : n_streams);
    } else {
        run_jobs(ctx->device, jobs, o, n_streams < 1 ? 8 : n_streams);
    }
    sip_status worst = SIP_OK;
    for (auto& j : jobs)
        if (j.st != SIP_OK) {
            worst = j.st;
            ctx->err = j.err.empty() ? sip::status_message(j.st) : j.err;
        }
    if (worst == SIP_OK) ctx->err.clear();
    return worst;
}

}  // namespace

sip_status sip_solve_batch(sip_ctx* ctx, int n, sip_problem* const* probs, const double* const* f_u,
                           double* const* u, double* const* p, const sip_solve_opts* opts,
                           sip_solve_report* reports, int n_streams) {
    return solve_batch_impl(ctx, n, probs, f_u, u, p, opts, reports, n_streams, false);
}

sip_status sip_solve_batch_grouped(sip_ctx* ctx, int n, sip_problem* const* probs,
                                   const double* const* f_u, double* const* u, double* const* p,
                                   const sip_solve_opts* opts, sip_solve_report* reports,
                                   int group) {
    return solve_batch_impl(ctx, n, probs, f_u, u, p, opts, reports, group, true);
}

sip_status sip_server_create(sip_ctx* ctx, int64_t budget_bytes, int max_slots, sip_server** out) {
    if (!ctx || !out || budget_bytes <= 0 || max_slots < 1 || max_slots > 256)
        return SIP_ERR_INVALID_ARG;
    auto* sv = new (std::nothrow) sip_server();
    if (!sv) return SIP_ERR_OOM;
    sv->ctx = ctx;
    sv->budget = budget_bytes;
    sv->slots = max_slots;
    try {
        for (int i = 0; i < max_slots; ++i) sv->workers.emplace_back([sv] { sv->worker_loop(); });
    } catch (...) {
        {
            std::lock_guard<std::mutex> lk(sv->mu);
            sv->stop = true;
        }
        sv->cv_work.notify_all();
        for (auto& t : sv->workers) t.join();
        delete sv;
        return SIP_ERR_OOM;
    }
    *out = sv;
    return SIP_OK;
}

int64_t sip_problem_footprint(const sip_problem_desc* desc, int restart) {
    if (!desc) return -1;
    return sip::estimate_problem_bytes(*desc, restart < 1 ? 100 : restart);
}

sip_status sip_server_submit(sip_server* sv, const sip_problem_desc* desc, const double* rho_host,
                             double g, double* u_host, double* p_host, const sip_solve_opts* opts,
                             uint64_t request_id) {
    if (!sv || !desc || !desc->eta_host || !rho_host || !u_host || !p_host)
        return SIP_ERR_INVALID_ARG;
    ServerRequest r;
    r.id = request_id;
    r.desc = *desc;
    r.desc.eta_host = nullptr;
    const size_t ne = size_t(desc->nx) * size_t(desc->ny);
    if (desc->nx < 1 || desc->ny < 1 || desc->k < 1 || desc->k > 6) return SIP_ERR_INVALID_ARG;
    r.eta.assign(desc->eta_host, desc->eta_host + ne);
    r.rho.assign(rho_host, rho_host + ne);
    for (size_t e = 0; e < ne; ++e)
        if (!std::isfinite(r.eta[e]) || !(r.eta[e] > 0.0) || !std::isfinite(r.rho[e]))
            return SIP_ERR_INVALID_ARG;
    if (!std::isfinite(g)) return SIP_ERR_INVALID_ARG;
    r.g = g;
    r.u_host = u_host;
    r.p_host = p_host;
    sip_solve_opts_default(&r.opts);
    if (opts) r.opts = *opts;
    try {
        sip::require_valid_opts(r.opts, r.desc.precision);
    } catch (const sip::Error&) {
        return SIP_ERR_INVALID_ARG;
    }
    r.bytes = sip::estimate_problem_bytes(r.desc, r.opts);
    r.t_submit = wall_ms();
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        if (r.bytes > sv->budget) {
            sip_solve_report rep{};
            rep.status = SIP_ERR_REJECTED;
            sv->done.push_back({r.id, rep});
            return SIP_ERR_REJECTED;
        }
        sv->queue.push_back(std::move(r));
    }
    sv->cv_work.notify_all();
    return SIP_OK;
}

sip_status sip_server_poll(sip_server* sv, uint64_t* ids, sip_solve_report* reps, int cap,
                           int* n_done) {
    if (!sv || !n_done || cap < 0 || (cap > 0 && (!ids || !reps))) return SIP_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(sv->mu);
    const int n = std::min<int>(cap, int(sv->done.size()));
    for (int i = 0; i < n; ++i) {
        ids[i] = sv->done[i].id;
        reps[i] = sv->done[i].rep;
    }
    sv->done.erase(sv->done.begin(), sv->done.begin() + n);
    *n_done = n;
    return SIP_OK;
}

sip_status sip_server_cancel(sip_server* sv, uint64_t id) {
    if (!sv) return SIP_ERR_INVALID_ARG;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        auto run = sv->running.find(id);
        if (run != sv->running.end()) {
            *run->second = true;   // the solve stops at its next outer iteration
            return SIP_OK;
        }
        auto it = std::find_if(sv->queue.begin(), sv->queue.end(),
                               [&](const ServerRequest& q) { return q.id == id; });
        if (it == sv->queue.end()) return SIP_ERR_INVALID_ARG;
        sip_solve_report rep{};
        rep.status = SIP_ERR_CANCELLED;
        sv->done.push_back({id, rep});
        sv->queue.erase(it);
    }
    sv->cv_work.notify_all();
    sv->cv_idle.notify_all();
    return SIP_OK;
}

sip_status sip_server_drain(sip_server* sv) {
    if (!sv) return SIP_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> lk(sv->mu);
    sv->cv_idle.wait(lk, [&] { return sv->queue.empty() && sv->busy == 0; });
    return SIP_OK;
}

sip_status sip_server_stats(sip_server* sv, int* queued, int* running, int64_t* bytes_in_use) {
    if (!sv) return SIP_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(sv->mu);
    if (queued) *queued = int(sv->queue.size());
    if (running) *running = sv->busy;
    if (bytes_in_use) *bytes_in_use = sv->in_use;
    return SIP_OK;
}

void sip_server_destroy(sip_server* sv) {
    if (!sv) return;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->stop = true;
        sv->queue.clear();
    }
    sv->cv_work.notify_all();
    for (auto& t : sv->workers) t.join();
    delete sv;
}

}  // extern "C"
