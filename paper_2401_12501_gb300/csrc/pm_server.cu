// Serving loop: continuous batching of solve requests over many operators.
//
// A request is (operator, right-hand side, tolerance, precision).  Its operator
// is either a caller's pm_surface with its coefficient set, or a description
// (geometry arrays, coefficient, caller ids of the geometry and of the
// coefficient) from which the server builds the operator itself: the first
// request on a geometry triggers its near-field build, a new coefficient on a
// known geometry a clone (shared near-field weights) with its own coefficient,
// and later requests reuse the resident operator.  Geometry, near field,
// coefficient and Krylov workspaces stay on the device.
//
// Worker threads, each with its own CUDA stream, repeatedly take the operator
// whose oldest waiting request arrived first and that no other worker is
// serving.  If it is not built yet the worker builds it; otherwise it admits as
// many of its waiting requests (of one precision) as the batch limit and device
// memory allow and solves them together (batched multi-RHS applies + lockstep
// GMRES, pm_solve_batch; pm_solve_impl for one).  Requests that arrive while
// others run wait in the queue and join their operator's next batch as soon as a
// worker and memory are free, so work on different operators overlaps on the
// device and the queue never blocks on one batch.
//
// Memory admission: a build or a batch reserves the device bytes it will
// allocate, from an a-priori model of the library's allocations
// (pm_operator_need_bytes, pm_solve_need_bytes: workspaces an operator already
// holds cost nothing), and is admitted only while the server's reservations
// plus this one stay within the creation budget and within the device's free
// memory (cudaMemGetInfo at admission time) less a safety margin.  A
// reservation ends when its work returns (its allocations are then part of the
// free-memory reading).  When nothing is in flight the oldest item is admitted
// regardless of the free-memory reading (its own allocation then fails with
// PM_ERR_OOM if the device is full, which ends that request, not the server).
#include "pm_internal.cuh"

#include <algorithm>
#include <cstdlib>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

namespace {

using Clock = std::chrono::steady_clock;

struct OpDesc {
    int npatch = 0, p = 0;
    std::vector<double> nodes, normals, tangents, curvature, weights, a, grad_a;
    pm_opts opts{};
};

struct Operator {
    pm_surface* s = nullptr;
    bool owned = false;                  // built by the server (destroyed with it)
    unsigned long long gid = 0, cid = 0;
    std::unique_ptr<OpDesc> desc;        // until built
    enum State { READY, PENDING, BUILDING, FAILED } state = READY;
    pm_status build_status = PM_OK;
    std::string build_err;
    bool busy = false;
    int N = 0;
};

struct Request {
    unsigned long long ticket = 0;
    Operator* op = nullptr;
    std::vector<double> f, u;
    double tol = 1e-8;
    pm_precision prec = PM_PREC_FP32;
    Clock::time_point t_submit, t_start, t_end;
    double build_s = 0.0;                // time its operator's build took while it waited
    pm_solve_info info{};
    pm_status status = PM_OK;
    std::string err;
    bool done = false;
    bool waiting = false;                // a thread is in pm_server_wait on it
};

}  // namespace

struct pm_server {
    pm_ctx* ctx = nullptr;
    size_t budget = 0, reserved = 0, margin = 0;
    int max_batch = 64;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request*> queue;                       // waiting, in arrival order
    std::unordered_map<unsigned long long, Request*> all;
    std::map<pm_surface*, Operator*> borrowed;
    std::map<std::pair<unsigned long long, unsigned long long>, Operator*> described;
    std::map<unsigned long long, Operator*> geometry;  // first built operator of each geometry
    unsigned long long next_ticket = 1;
    int in_flight = 0;
    int active_workers = 0;            // workers with an index below this take work
    bool stopping = false;
    std::vector<std::thread> workers;
    long long batches = 0, solved = 0, max_batch_seen = 0, builds = 0;
};

namespace {

// free device memory now (the worker thread's device is the context's); the
// environment variable PM_FAKE_HBM_BYTES, when set, replaces the reading
size_t free_bytes() { return pm_free_hbm_bytes(); }

bool can_reserve(pm_server* sv, size_t need) {
    if (sv->reserved + need > sv->budget) return sv->in_flight == 0 && need <= sv->budget;
    if (sv->in_flight == 0) return true;
    const size_t fr = free_bytes();
    return sv->reserved + need + sv->margin <= fr;
}

void finish_request(Request* r, pm_status st, const std::string& err) {
    r->status = st;
    r->err = err;
    r->done = true;
    r->t_end = Clock::now();
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
        Operator* build_op = nullptr;
        size_t reservation = 0;
        {
            std::unique_lock<std::mutex> lk(sv->mu);
            for (;;) {
                if (sv->stopping) {
                    if (st) cudaStreamDestroy(st);
                    return;
                }
                if (index >= sv->active_workers) {
                    sv->cv_work.wait(lk);
                    continue;
                }
                // requests of operators whose build failed end with the build's status
                for (auto it = sv->queue.begin(); it != sv->queue.end();) {
                    if ((*it)->op->state == Operator::FAILED) {
                        finish_request(*it, (*it)->op->build_status, (*it)->op->build_err);
                        it = sv->queue.erase(it);
                        sv->cv_done.notify_all();
                    } else {
                        ++it;
                    }
                }
                // oldest waiting request whose operator is free (an unbuilt operator whose
                // geometry is being built by another worker waits for that build and is
                // then cloned from it)
                Operator* op = nullptr;
                for (Request* r : sv->queue) {
                    if (r->op->busy) continue;
                    if (r->op->state == Operator::PENDING) {
                        bool geom_building = false;
                        for (auto& kv : sv->described)
                            if (kv.first.first == r->op->gid && kv.second->state == Operator::BUILDING &&
                                sv->geometry.find(r->op->gid) == sv->geometry.end())
                                geom_building = true;
                        if (geom_building) continue;
                    }
                    op = r->op;
                    break;
                }
                if (op && op->state == Operator::PENDING) {
                    auto g = sv->geometry.find(op->gid);
                    const bool clone = g != sv->geometry.end() && g->second->state == Operator::READY;
                    const size_t need = pm_operator_need_bytes(op->desc->npatch, op->desc->p, clone);
                    if (can_reserve(sv, need)) {
                        reservation = need;
                        sv->reserved += need;
                        sv->in_flight++;
                        op->busy = true;
                        op->state = Operator::BUILDING;
                        build_op = op;
                        break;
                    }
                } else if (op) {
                    // admit its waiting requests of the oldest one's precision in arrival
                    // order while the batch's workspace fits (a batch is one precision)
                    pm_precision prec = PM_PREC_FP32;
                    for (Request* r : sv->queue)
                        if (r->op == op) {
                            prec = r->prec;
                            break;
                        }
                    for (auto it = sv->queue.begin(); it != sv->queue.end() &&
                                                      (int)batch.size() < sv->max_batch;) {
                        Request* r = *it;
                        if (r->op == op && r->prec == prec) {
                            const size_t need =
                                pm_solve_need_bytes(op->s, (int)batch.size() + 1, prec);
                            const size_t extra = need > reservation ? need - reservation : 0;
                            if (!(batch.empty() ? can_reserve(sv, need)
                                                : sv->reserved + extra + sv->margin <=
                                                      std::min(sv->budget + sv->margin,
                                                               free_bytes())))
                                break;
                            sv->reserved += extra;
                            reservation += extra;
                            batch.push_back(r);
                            it = sv->queue.erase(it);
                        } else {
                            ++it;
                        }
                    }
                    if (!batch.empty()) {
                        op->busy = true;
                        sv->in_flight++;
                        break;
                    }
                }
                sv->cv_work.wait(lk);
            }
        }
        if (build_op) {
            // build the operator from its description (outside the lock)
            Operator* op = build_op;
            Operator* base = nullptr;
            {
                std::lock_guard<std::mutex> lk(sv->mu);
                auto g = sv->geometry.find(op->gid);
                if (g != sv->geometry.end() && g->second->state == Operator::READY) base = g->second;
            }
            const OpDesc& d = *op->desc;
            const auto t0 = Clock::now();
            cudaSetDevice(sv->ctx->device);
            pm_surface* s = nullptr;
            pm_status bst = base ? pm_surface_clone(base->s, &s)
                                 : pm_surface_create(sv->ctx, d.npatch, d.p, d.nodes.data(),
                                                     d.normals.data(), d.tangents.data(),
                                                     d.curvature.data(), d.weights.data(),
                                                     &d.opts, &s);
            if (bst == PM_OK)
                bst = pm_surface_set_coeff(s, d.a.data(), d.grad_a.empty() ? nullptr : d.grad_a.data());
            const std::string err = bst == PM_OK ? std::string() : std::string(pm_last_error());
            if (bst != PM_OK && s) {
                pm_surface_destroy(s);
                s = nullptr;
            }
            const double dt = std::chrono::duration<double>(Clock::now() - t0).count();
            {
                std::lock_guard<std::mutex> lk(sv->mu);
                op->s = s;
                op->owned = s != nullptr;
                op->state = bst == PM_OK ? Operator::READY : Operator::FAILED;
                op->build_status = bst;
                op->build_err = err;
                op->desc.reset();
                op->busy = false;
                if (bst == PM_OK && sv->geometry.find(op->gid) == sv->geometry.end())
                    sv->geometry[op->gid] = op;
                for (Request* r : sv->queue)
                    if (r->op == op) r->build_s += dt;
                sv->reserved -= reservation;
                sv->in_flight--;
                sv->builds += 1;
            }
            sv->cv_work.notify_all();
            continue;
        }
        // solve the batch on this worker's stream (the operator is ours alone)
        Operator* op = batch[0]->op;
        pm_surface* s = op->s;
        const int nb = (int)batch.size();
        const size_t N = s->N;
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
            st_solve = pm_solve_impl(s, F.data(), U.data(), tol, 4000, batch[0]->prec, 0u,
                                     nullptr, infos.data(), st);
        else
            st_solve = pm_solve_batch(s, F.data(), U.data(), nb, tol, 4000, batch[0]->prec, 0u,
                                      nullptr, infos.data(), st);
        if (st_solve == PM_OK && batch[0]->prec == PM_PREC_FMM) st_solve = pm_fmm_check(s);
        const std::string err = st_solve == PM_OK ? std::string() : std::string(pm_last_error());
        {
            std::lock_guard<std::mutex> lk(sv->mu);
            for (int r = 0; r < nb; ++r) {
                Request* q = batch[r];
                q->u.assign(U.begin() + r * N, U.begin() + (r + 1) * N);
                q->info = infos[r];
                q->t_start = t_start;
                finish_request(q, st_solve, err);
            }
            op->busy = false;
            sv->reserved -= reservation;
            sv->in_flight--;
            sv->batches += 1;
            sv->solved += nb;
            sv->max_batch_seen = std::max<long long>(sv->max_batch_seen, nb);
        }
        sv->cv_done.notify_all();
        sv->cv_work.notify_all();
    }
}

// copy of a host array of n doubles (NULL -> empty)
std::vector<double> copy_of(const double* p, size_t n) {
    return p ? std::vector<double>(p, p + n) : std::vector<double>();
}

pm_status enqueue(pm_server* sv, Operator* op, const double* f, double tol, pm_precision prec,
                  size_t need, unsigned long long* ticket) {
    Request* r = new Request();
    r->op = op;
    r->f.assign(f, f + op->N);
    r->tol = tol;
    r->prec = prec;
    r->t_submit = Clock::now();
    r->ticket = sv->next_ticket++;
    sv->all[r->ticket] = r;
    sv->queue.push_back(r);
    *ticket = r->ticket;
    (void)need;
    return PM_OK;
}

bool prec_ok(pm_precision prec) {
    return prec == PM_PREC_FP64 || prec == PM_PREC_FP32 || prec == PM_PREC_FF ||
           prec == PM_PREC_FMM;
}

}  // namespace

extern "C" pm_status pm_server_create(pm_ctx* ctx, size_t hbm_budget_bytes, int max_batch,
                                      int n_workers, pm_server** out) {
    if (!out || !ctx || hbm_budget_bytes == 0 || max_batch < 1 || n_workers < 1 || n_workers > 64) {
        pm_set_error("pm_server_create: bad argument");
        return PM_ERR_INVALID_ARG;
    }
    PM_CUDA_TRY(cudaSetDevice(ctx->device));
    size_t fr = 0, tot = 0;
    PM_CUDA_TRY(cudaMemGetInfo(&fr, &tot));
    pm_server* sv = new pm_server();
    sv->ctx = ctx;
    sv->budget = hbm_budget_bytes;
    sv->margin = std::max<size_t>((size_t)256 << 20, tot / 50);
    sv->max_batch = max_batch;
    sv->active_workers = n_workers;
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
    for (auto& kv : sv->borrowed) delete kv.second;
    // clones first, then the geometry's first operator (the near field is shared and
    // reference-counted, so the order only keeps the bookkeeping simple)
    for (auto& kv : sv->described)
        if (kv.second->owned && kv.second->s) pm_surface_destroy(kv.second->s);
    for (auto& kv : sv->described) delete kv.second;
    delete sv;
}

extern "C" pm_status pm_server_submit(pm_server* sv, pm_surface* op, const double* f, double tol,
                                      pm_precision prec, unsigned long long* ticket) {
    if (!sv || !op || !f || !ticket || !(tol > 0) || !prec_ok(prec)) {
        pm_set_error("pm_server_submit: bad argument (NULL, tol <= 0 or unknown precision)");
        return PM_ERR_INVALID_ARG;
    }
    if (!op->has_coeff) {
        pm_set_error("pm_server_submit: operator has no coefficient");
        return PM_ERR_NO_COEFF;
    }
    if (op->has_c) {
        pm_set_error("pm_server_submit: operator has c != 0 (pm_solve_c solves it)");
        return PM_ERR_INVALID_ARG;
    }
    std::lock_guard<std::mutex> lk(sv->mu);
    Operator*& o = sv->borrowed[op];
    if (!o) {
        o = new Operator();
        o->s = op;
        o->N = op->N;
        o->state = Operator::READY;
    }
    const size_t need = pm_solve_need_bytes(op, 1, prec);
    if (need > sv->budget) {
        pm_set_error("pm_server_submit: request needs %zu bytes, budget is %zu", need, sv->budget);
        return PM_ERR_OOM;
    }
    PM_TRY(enqueue(sv, o, f, tol, prec, need, ticket));
    sv->cv_work.notify_one();
    return PM_OK;
}

extern "C" pm_status pm_server_submit_desc(pm_server* sv, const pm_operator_desc* d,
                                           const double* f, double tol, pm_precision prec,
                                           unsigned long long* ticket) {
    if (!sv || !d || !f || !ticket || !(tol > 0) || !prec_ok(prec)) {
        pm_set_error("pm_server_submit_desc: bad argument (NULL, tol <= 0 or unknown precision)");
        return PM_ERR_INVALID_ARG;
    }
    if (d->npatch < 1 || d->p < 2 || d->p > PM_MAX_P_API) {
        pm_set_error("pm_server_submit_desc: npatch = %d, p = %d out of range", d->npatch, d->p);
        return PM_ERR_INVALID_ARG;
    }
    const size_t N = (size_t)d->npatch * d->p * d->p;
    const size_t need = pm_operator_need_bytes(d->npatch, d->p, 0);
    if (need > sv->budget) {
        pm_set_error("pm_server_submit_desc: the operator needs about %zu bytes, budget is %zu",
                     need, sv->budget);
        return PM_ERR_OOM;
    }
    std::lock_guard<std::mutex> lk(sv->mu);
    Operator*& o = sv->described[{d->geometry_id, d->coeff_id}];
    if (!o) {
        // a geometry id names one geometry: its size must agree with the first one
        for (auto& kv : sv->described)
            if (kv.first.first == d->geometry_id && kv.second && kv.second->N != (int)N) {
                const int n0 = kv.second->N;
                sv->described.erase({d->geometry_id, d->coeff_id});
                pm_set_error("pm_server_submit_desc: geometry %llu was described with %d nodes",
                             d->geometry_id, n0);
                return PM_ERR_INVALID_ARG;
            }
        if (!d->a || !d->nodes || !d->normals || !d->tangents || !d->curvature || !d->weights) {
            sv->described.erase({d->geometry_id, d->coeff_id});
            pm_set_error("pm_server_submit_desc: a new operator needs a and every geometry array");
            return PM_ERR_INVALID_ARG;
        }
        o = new Operator();
        o->gid = d->geometry_id;
        o->cid = d->coeff_id;
        o->N = (int)N;
        o->state = Operator::PENDING;
        o->desc.reset(new OpDesc());
        OpDesc& c = *o->desc;
        c.npatch = d->npatch;
        c.p = d->p;
        c.nodes = copy_of(d->nodes, 3 * N);
        c.normals = copy_of(d->normals, 3 * N);
        c.tangents = copy_of(d->tangents, 6 * N);
        c.curvature = copy_of(d->curvature, N);
        c.weights = copy_of(d->weights, N);
        c.a = copy_of(d->a, N);
        c.grad_a = copy_of(d->grad_a, 3 * N);
        if (d->opts) c.opts = *d->opts;
        else pm_default_opts(&c.opts);
    }
    PM_TRY(enqueue(sv, o, f, tol, prec, need, ticket));
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

extern "C" pm_status pm_server_wait_ex(pm_server* sv, unsigned long long ticket, double* u,
                                       pm_solve_info* info, pm_request_times* times,
                                       int timeout_ms) {
    if (!sv || !u) { pm_set_error("pm_server_wait: NULL argument"); return PM_ERR_INVALID_ARG; }
    std::unique_lock<std::mutex> lk(sv->mu);
    auto it = sv->all.find(ticket);
    if (it == sv->all.end()) { pm_set_error("pm_server_wait: unknown ticket"); return PM_ERR_INVALID_ARG; }
    Request* r = it->second;
    if (r->waiting) {
        pm_set_error("pm_server_wait: another thread is already waiting on ticket %llu", ticket);
        return PM_ERR_INVALID_ARG;
    }
    r->waiting = true;
    const auto pred = [&] { return r->done; };
    if (timeout_ms < 0) {
        sv->cv_done.wait(lk, pred);
    } else if (!sv->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), pred)) {
        r->waiting = false;
        pm_set_error("pm_server_wait: ticket %llu not finished within %d ms", ticket, timeout_ms);
        return PM_ERR_TIMEOUT;
    }
    if (!r->u.empty()) std::copy(r->u.begin(), r->u.end(), u);
    if (info) *info = r->info;
    if (times) {
        times->latency_s = std::chrono::duration<double>(r->t_end - r->t_submit).count();
        times->build_s = r->build_s;
        times->solve_s = r->status == PM_OK || r->t_start > r->t_submit
                             ? std::chrono::duration<double>(r->t_end - r->t_start).count()
                             : 0.0;
        times->queue_s = std::max(0.0, times->latency_s - times->solve_s - times->build_s);
    }
    const pm_status st = r->status;
    if (st != PM_OK) pm_set_error("%s", r->err.empty() ? "solve failed" : r->err.c_str());
    sv->all.erase(it);
    delete r;
    return st;
}

extern "C" pm_status pm_server_wait(pm_server* sv, unsigned long long ticket, double* u,
                                    pm_solve_info* info, double* latency_s, int timeout_ms) {
    pm_request_times t{};
    const pm_status st = pm_server_wait_ex(sv, ticket, u, info, latency_s ? &t : nullptr,
                                           timeout_ms);
    if (latency_s && (st == PM_OK || st != PM_ERR_INVALID_ARG)) *latency_s = t.latency_s;
    return st;
}

extern "C" pm_status pm_server_stats(pm_server* sv, long long* batches, long long* solved,
                                     long long* max_batch, size_t* bytes_in_use) {
    if (!sv) { pm_set_error("pm_server_stats: NULL server"); return PM_ERR_INVALID_ARG; }
    std::lock_guard<std::mutex> lk(sv->mu);
    if (batches) *batches = sv->batches;
    if (solved) *solved = sv->solved;
    if (max_batch) *max_batch = sv->max_batch_seen;
    if (bytes_in_use) *bytes_in_use = sv->reserved;
    return PM_OK;
}

extern "C" pm_status pm_server_configure(pm_server* sv, int max_batch, int active_workers) {
    if (!sv || max_batch < 1 || active_workers < 1 ||
        active_workers > (int)sv->workers.size()) {
        pm_set_error("pm_server_configure: max_batch >= 1 and 1 <= active_workers <= %d required",
                     sv ? (int)sv->workers.size() : 0);
        return PM_ERR_INVALID_ARG;
    }
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->max_batch = max_batch;
        sv->active_workers = active_workers;
    }
    sv->cv_work.notify_all();
    return PM_OK;
}

extern "C" pm_status pm_server_stats_ex(pm_server* sv, long long* builds, size_t* reserved_bytes,
                                        size_t* margin_bytes, int* operators) {
    if (!sv) { pm_set_error("pm_server_stats_ex: NULL server"); return PM_ERR_INVALID_ARG; }
    std::lock_guard<std::mutex> lk(sv->mu);
    if (builds) *builds = sv->builds;
    if (reserved_bytes) *reserved_bytes = sv->reserved;
    if (margin_bytes) *margin_bytes = sv->margin;
    if (operators) *operators = (int)(sv->borrowed.size() + sv->described.size());
    return PM_OK;
}
