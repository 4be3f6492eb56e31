// Serving loop: continuous batching of solve requests over many operators.
//
// A request is (operator, right-hand side, tolerance); an operator is a
// pm_surface with its coefficient set (geometry, near field and coefficient
// stay resident on the device).  Worker threads, each with its own CUDA stream,
// repeatedly take the operator whose oldest waiting request arrived first and
// that no other worker is serving, admit as many of its waiting requests as
// the batch limit and the device-memory budget allow, and solve them together
// (batched multi-RHS applies + lockstep GMRES, pm_solve_batch).  Requests that
// arrive while others run wait in the queue and join the next batch of their
// operator as soon as a worker and memory are free, so work on different
// operators overlaps on the device and the queue never blocks on one batch.
//
// Memory admission: each admitted request reserves its Krylov and vector
// footprint, (m + 1 + 10) N doubles, against the budget given at creation; a
// request whose footprint alone exceeds the budget is rejected at submit.
#include "pm_internal.cuh"

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
    unsigned long long ticket = 0;
    pm_surface* op = nullptr;
    std::vector<double> f, u;
    double tol = 1e-8;
    pm_precision prec = PM_PREC_FP32;
    size_t bytes = 0;
    Clock::time_point t_submit, t_start, t_end;
    pm_solve_info info{};
    pm_status status = PM_OK;
    bool done = false;
    bool taken = false;
};

}  // namespace

struct pm_server {
    pm_ctx* ctx = nullptr;
    size_t budget = 0, in_use = 0;
    int max_batch = 64;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request*> queue;                       // waiting, in arrival order
    std::unordered_map<unsigned long long, Request*> all;
    std::map<pm_surface*, bool> busy;
    unsigned long long next_ticket = 1;
    bool stopping = false;
    std::vector<std::thread> workers;
    long long batches = 0, solved = 0, max_batch_seen = 0;
};

namespace {

size_t request_bytes(const pm_surface* op) {
    const int m = std::max(2, std::min(op->opts.gmres_restart, 400));
    return (size_t)(m + 1 + 10) * (size_t)op->N * sizeof(double);
}

void worker_main(pm_server* sv, int index) {
    cudaSetDevice(sv->ctx->device);
    cudaStream_t st = nullptr;
    cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    std::vector<Request*> batch;
    std::vector<double> F, U;
    std::vector<pm_solve_info> infos;
    for (;;) {
        batch.clear();
        {
            std::unique_lock<std::mutex> lk(sv->mu);
            for (;;) {
                if (sv->stopping) {
                    if (st) cudaStreamDestroy(st);
                    return;
                }
                // oldest waiting request whose operator is free
                pm_surface* op = nullptr;
                for (Request* r : sv->queue)
                    if (!sv->busy[r->op]) {
                        op = r->op;
                        break;
                    }
                if (op) {
                    // admit its waiting requests of the oldest one's precision in arrival
                    // order while memory allows (a batch is solved in one precision)
                    pm_precision prec = PM_PREC_FP32;
                    for (Request* r : sv->queue)
                        if (r->op == op) {
                            prec = r->prec;
                            break;
                        }
                    for (auto it = sv->queue.begin(); it != sv->queue.end() &&
                                                      (int)batch.size() < sv->max_batch;) {
                        Request* r = *it;
                        if (r->op == op && r->prec == prec && sv->in_use + r->bytes <= sv->budget) {
                            sv->in_use += r->bytes;
                            r->taken = true;
                            batch.push_back(r);
                            it = sv->queue.erase(it);
                        } else {
                            ++it;
                        }
                    }
                    if (!batch.empty()) {
                        sv->busy[op] = true;
                        break;
                    }
                }
                sv->cv_work.wait(lk);
            }
        }
        // solve the batch on this worker's stream (the operator is ours alone)
        pm_surface* op = batch[0]->op;
        const int nb = (int)batch.size();
        const size_t N = op->N;
        const auto t_start = Clock::now();
        F.resize(nb * N);
        U.resize(nb * N);
        infos.assign(nb, pm_solve_info{});
        double tol = batch[0]->tol;
        for (int r = 0; r < nb; ++r) {
            std::copy(batch[r]->f.begin(), batch[r]->f.end(), F.begin() + r * N);
            tol = std::min(tol, batch[r]->tol);
        }
        cudaSetDevice(sv->ctx->device);
        pm_status st_solve;
        if (nb == 1)
            st_solve = pm_solve_impl(op, F.data(), U.data(), tol, 4000, batch[0]->prec, 0u,
                                     nullptr, infos.data(), st);
        else
            st_solve = pm_solve_batch(op, F.data(), U.data(), nb, tol, 4000, batch[0]->prec, 0u,
                                      nullptr, infos.data(), st);
        const auto t_end = Clock::now();
        {
            std::lock_guard<std::mutex> lk(sv->mu);
            for (int r = 0; r < nb; ++r) {
                Request* q = batch[r];
                q->u.assign(U.begin() + r * N, U.begin() + (r + 1) * N);
                q->info = infos[r];
                q->status = st_solve;
                q->t_start = t_start;
                q->t_end = t_end;
                q->done = true;
                sv->in_use -= q->bytes;
            }
            sv->busy[op] = false;
            sv->batches += 1;
            sv->solved += nb;
            sv->max_batch_seen = std::max<long long>(sv->max_batch_seen, nb);
        }
        sv->cv_done.notify_all();
        sv->cv_work.notify_all();
        (void)index;
    }
}

}  // namespace

extern "C" pm_status pm_server_create(pm_ctx* ctx, size_t hbm_budget_bytes, int max_batch,
                                      int n_workers, pm_server** out) {
    if (!out || !ctx || hbm_budget_bytes == 0 || max_batch < 1 || n_workers < 1 || n_workers > 64) {
        pm_set_error("pm_server_create: bad argument");
        return PM_ERR_INVALID_ARG;
    }
    pm_server* sv = new pm_server();
    sv->ctx = ctx;
    sv->budget = hbm_budget_bytes;
    sv->max_batch = max_batch;
    for (int k = 0; k < n_workers; ++k) sv->workers.emplace_back(worker_main, sv, k);
    *out = sv;
    return PM_OK;
}

extern "C" void pm_server_destroy(pm_server* sv) {
    if (!sv) return;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->stopping = true;
    }
    sv->cv_work.notify_all();
    for (auto& t : sv->workers) t.join();
    for (auto& kv : sv->all) delete kv.second;
    delete sv;
}

extern "C" pm_status pm_server_submit(pm_server* sv, pm_surface* op, const double* f, double tol,
                                      pm_precision prec, unsigned long long* ticket) {
    if (!sv || !op || !f || !ticket || !(tol > 0) ||
        !(prec == PM_PREC_FP64 || prec == PM_PREC_FP32 || prec == PM_PREC_FF ||
          prec == PM_PREC_FMM)) {
        pm_set_error("pm_server_submit: bad argument (NULL, tol <= 0 or unknown precision)");
        return PM_ERR_INVALID_ARG;
    }
    if (!op->has_coeff) {
        pm_set_error("pm_server_submit: operator has no coefficient");
        return PM_ERR_NO_COEFF;
    }
    Request* r = new Request();
    r->op = op;
    r->f.assign(f, f + op->N);
    r->tol = tol;
    r->prec = prec;
    r->bytes = request_bytes(op);
    r->t_submit = Clock::now();
    if (r->bytes > sv->budget) {
        delete r;
        pm_set_error("pm_server_submit: request needs %zu bytes, budget is %zu", request_bytes(op),
                     sv->budget);
        return PM_ERR_OOM;
    }
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        r->ticket = sv->next_ticket++;
        sv->all[r->ticket] = r;
        sv->queue.push_back(r);
        *ticket = r->ticket;
    }
    sv->cv_work.notify_one();
    return PM_OK;
}

extern "C" pm_status pm_server_poll(pm_server* sv, unsigned long long ticket, int* done) {
    if (!sv || !done) { pm_set_error("pm_server_poll: NULL argument"); return PM_ERR_INVALID_ARG; }
    std::lock_guard<std::mutex> lk(sv->mu);
    auto it = sv->all.find(ticket);
    if (it == sv->all.end()) { pm_set_error("pm_server_poll: unknown ticket"); return PM_ERR_INVALID_ARG; }
    *done = it->second->done ? 1 : 0;
    return PM_OK;
}

extern "C" pm_status pm_server_wait(pm_server* sv, unsigned long long ticket, double* u,
                                    pm_solve_info* info, double* latency_s, int timeout_ms) {
    if (!sv || !u) { pm_set_error("pm_server_wait: NULL argument"); return PM_ERR_INVALID_ARG; }
    std::unique_lock<std::mutex> lk(sv->mu);
    auto it = sv->all.find(ticket);
    if (it == sv->all.end()) { pm_set_error("pm_server_wait: unknown ticket"); return PM_ERR_INVALID_ARG; }
    Request* r = it->second;
    const auto pred = [&] { return r->done; };
    if (timeout_ms < 0) {
        sv->cv_done.wait(lk, pred);
    } else if (!sv->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), pred)) {
        pm_set_error("pm_server_wait: ticket %llu not finished within %d ms", ticket, timeout_ms);
        return PM_ERR_TIMEOUT;
    }
    std::copy(r->u.begin(), r->u.end(), u);
    if (info) *info = r->info;
    if (latency_s) *latency_s = std::chrono::duration<double>(r->t_end - r->t_submit).count();
    const pm_status st = r->status;
    sv->all.erase(it);
    delete r;
    return st;
}

extern "C" pm_status pm_server_stats(pm_server* sv, long long* batches, long long* solved,
                                     long long* max_batch, size_t* bytes_in_use) {
    if (!sv) { pm_set_error("pm_server_stats: NULL server"); return PM_ERR_INVALID_ARG; }
    std::lock_guard<std::mutex> lk(sv->mu);
    if (batches) *batches = sv->batches;
    if (solved) *solved = sv->solved;
    if (max_batch) *max_batch = sv->max_batch_seen;
    if (bytes_in_use) *bytes_in_use = sv->in_use;
    return PM_OK;
}
