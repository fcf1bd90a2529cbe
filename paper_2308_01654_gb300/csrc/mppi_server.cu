// mppi_server.cu - continuous-batching planning server over the batched planner.
//
// Requests from many vehicle sessions arrive at any time (mppi_server_enqueue, thread
// safe; the inputs are copied).  A scheduler thread forms a micro-batch whenever a
// pipeline of the batch engine is free: it takes queued requests in arrival order while
// their device footprint (noise, costs, weights, scene) fits the free HBM budget and the
// batch's capacities, and never puts one session in two batches in flight (a session's
// warm start lives in its device slot, so its requests run in order).  Up to `pipelines`
// micro-batches are on the GPU at once; requests that arrive meanwhile join the next one.
// A completion thread waits for the batches in submission order, stamps each request's
// latency (completion - arrival) and frees its footprint and session; mppi_server_poll
// hands the results out.
#include <stdio.h>
#include <string.h>

#include <atomic>
#include <cmath>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <memory>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "mppi.h"
#include "mppi_internal.h"
#include "mppi_trace.h"

// the batch engine's completion query (mppi_batch.cu)
int batch_ticket_done(mppi_batch* B, int32_t ticket);

namespace {

using Clock = std::chrono::steady_clock;

struct Req {
    uint64_t id = 0;
    int32_t session = 0;
    mppi_params params{};
    std::vector<double> x0, ref, circ, centres;
    int32_t n_ref = 0, n_circ = 0;
    std::vector<double> u, x;
    mppi_info info{};
    int32_t status = 0;
    size_t footprint = 0;
    Clock::time_point t_arrive, t_submit, t_done;
};

struct InFlight {
    int32_t ticket = -1;
    std::vector<std::unique_ptr<Req>> reqs;
    std::vector<mppi_request> creq;
    size_t footprint = 0;
    Clock::time_point t_submit;
    nvtxRangeId_t range = 0;       // NVTX range of the micro-batch, submission to completion
};

}  // namespace

struct mppi_server {
    mppi_server_config cfg{};
    mppi_batch* batch = nullptr;
    std::mutex mu;
    std::condition_variable cv_sched, cv_done, cv_poll;
    std::deque<std::unique_ptr<Req>> queue;
    std::deque<std::unique_ptr<InFlight>> inflight;   // in submission order
    std::deque<std::unique_ptr<Req>> done;
    std::vector<char> session_busy;
    size_t budget = 0, used = 0;
    int free_pipes = 0;
    uint64_t epoch = 0;   // advanced by every arrival and every completion
    uint64_t next_id = 1;
    bool stop = false;
    std::thread sched, compl_;
    double watchdog_ms = 0.0;      // a micro-batch still running this long after its submission is abandoned
    // statistics
    uint64_t n_batches = 0, n_plans = 0, n_timeouts = 0;
    std::string err;
};

static thread_local std::string g_srv_err;

static int sfail(mppi_server* s, int st, const std::string& m) {
    if (s) s->err = m;
    g_srv_err = m;
    return st;
}

// Device bytes a request occupies while in flight: its noise, costs, weights and scene.
static size_t footprint_of(const mppi_params& p, int n_ref, int n_circ) {
    const size_t K = (size_t)p.K, T = (size_t)p.T;
    const mppi::SceneLayout L = mppi::make_layout(p.T, n_ref, n_circ);
    return K * T * (p.noise_bf16 ? 4 : 8) + K * (8 + 4) + (size_t)L.total + T * (size_t)(n_circ > 0 ? n_circ : 1) * 8;
}

static void scheduler_loop(mppi_server* S) {
    std::unique_lock<std::mutex> lk(S->mu);
    for (;;) {
        S->cv_sched.wait(lk, [&] { return S->stop || (S->free_pipes > 0 && !S->queue.empty()); });
        if (S->stop) return;
        // optional hold to let a batch grow while the GPU is busy anyway
        if (S->cfg.max_wait_us > 0.0 && (int)S->inflight.size() > 0) {
            S->cv_sched.wait_for(lk, std::chrono::microseconds((long long)S->cfg.max_wait_us),
                                 [&] { return S->stop || (int)S->queue.size() >= S->cfg.max_batch; });
            if (S->stop) return;
        }
        auto job = std::make_unique<InFlight>();
        long long sum_k = 0, sum_kt = 0;
        std::vector<char> in_batch(S->session_busy.size(), 0);
        for (auto it = S->queue.begin(); it != S->queue.end() && (int)job->reqs.size() < S->cfg.max_batch;) {
            Req& r = **it;
            const long long k = r.params.K, kt = (long long)r.params.K * r.params.T;
            const bool session_free = !S->session_busy[(size_t)r.session] && !in_batch[(size_t)r.session];
            const bool fits = sum_k + k <= S->cfg.max_samples && sum_kt + kt <= S->cfg.max_rollout_steps &&
                              S->used + job->footprint + r.footprint <= S->budget;
            if (session_free && fits) {
                in_batch[(size_t)r.session] = 1;
                sum_k += k;
                sum_kt += kt;
                job->footprint += r.footprint;
                job->reqs.push_back(std::move(*it));
                it = S->queue.erase(it);
            } else {
                // a request left in the queue (its session busy, or too large for what is free
                // now) keeps its place and holds back every later request of its session, so
                // that a session's requests run in arrival order; other sessions may go ahead
                in_batch[(size_t)r.session] = 1;
                ++it;
            }
        }
        if (job->reqs.empty()) {
            // nothing admissible now (its sessions are in flight or the budget is used up):
            // sleep until a request arrives or a batch completes
            const uint64_t e0 = S->epoch;
            S->cv_sched.wait(lk, [&] { return S->stop || S->epoch != e0; });
            continue;
        }
        for (auto& r : job->reqs) S->session_busy[(size_t)r->session] = 1;
        S->used += job->footprint;
        S->free_pipes -= 1;
        job->creq.resize(job->reqs.size());
        const auto now = Clock::now();
        for (size_t i = 0; i < job->reqs.size(); ++i) {
            Req& r = *job->reqs[i];
            r.t_submit = now;
            mppi_request& q = job->creq[i];
            memset(&q, 0, sizeof(q));
            q.params = &r.params;
            q.slot = r.session;
            q.x0 = r.x0.data();
            q.ref_xy = r.ref.data();
            q.n_ref = r.n_ref;
            q.circ = r.n_circ ? reinterpret_cast<const mppi_circle*>(r.circ.data()) : nullptr;
            q.n_circ = r.n_circ;
            q.centres = r.centres.empty() ? nullptr : r.centres.data();
            q.u_out = r.u.data();
            q.x_out = r.x.data();
            q.info = &r.info;
        }
        InFlight* jp = job.get();
        jp->t_submit = now;
        jp->range = mppi::trace_start("serve micro-batch");
        S->inflight.push_back(std::move(job));
        lk.unlock();
        int32_t ticket = -1;
        const int rc = mppi_batch_submit(S->batch, jp->creq.data(), (int32_t)jp->creq.size(), &ticket);
        lk.lock();
        jp->ticket = rc == MPPI_OK ? ticket : -1;
        if (rc != MPPI_OK)
            for (auto& r : jp->reqs) r->status = rc;
        S->n_batches += 1;
        S->cv_done.notify_all();
    }
}

static void completion_loop(mppi_server* S) {
    std::unique_lock<std::mutex> lk(S->mu);
    for (;;) {
        S->cv_done.wait(lk, [&] { return S->stop || (!S->inflight.empty() && S->inflight.front()->ticket >= 0) ||
                                         (!S->inflight.empty() && S->inflight.front()->reqs.front()->status != 0); });
        if (S->stop && S->inflight.empty()) return;
        if (S->inflight.empty()) continue;
        InFlight* jp = S->inflight.front().get();
        bool abandoned = false;
        if (jp->ticket >= 0) {
            const double wd = S->watchdog_ms;
            lk.unlock();
            if (wd > 0.0) {
                // watchdog: a micro-batch still running wd ms after its submission is abandoned
                const auto deadline =
                    jp->t_submit + std::chrono::duration_cast<Clock::duration>(std::chrono::duration<double, std::milli>(wd));
                int d = batch_ticket_done(S->batch, jp->ticket);
                while (d == 0 && Clock::now() < deadline) {
                    std::this_thread::sleep_for(std::chrono::microseconds(20));
                    d = batch_ticket_done(S->batch, jp->ticket);
                }
                abandoned = d == 0;
            }
            if (abandoned) {
                // its requests complete now with MPPI_ERR_TIMEOUT (copies: the batch still writes
                // into the originals); the sessions, the budget and the pipeline stay taken until
                // the device work has ended, and its results are then dropped
                lk.lock();
                const auto now = Clock::now();
                for (auto& r : jp->reqs) {
                    auto t = std::make_unique<Req>();
                    t->id = r->id;
                    t->session = r->session;
                    t->params = r->params;
                    t->u.assign(r->u.size(), 0.0);
                    t->x.assign(r->x.size(), 0.0);
                    t->status = MPPI_ERR_TIMEOUT;
                    t->t_arrive = r->t_arrive;
                    t->t_submit = r->t_submit;
                    t->t_done = now;
                    S->done.push_back(std::move(t));
                    S->n_plans += 1;
                    S->n_timeouts += 1;
                }
                S->cv_poll.notify_all();
                lk.unlock();
            }
            mppi_batch_wait(S->batch, jp->ticket);   // per-plan status is in creq[i].status
            lk.lock();
            for (size_t i = 0; i < jp->reqs.size(); ++i) jp->reqs[i]->status = jp->creq[i].status;
        }
        const auto now = Clock::now();
        auto job = std::move(S->inflight.front());
        S->inflight.pop_front();
        mppi::trace_end(job->range);
        for (auto& r : job->reqs) {
            S->session_busy[(size_t)r->session] = 0;
            if (abandoned) continue;
            r->t_done = now;
            S->done.push_back(std::move(r));
            S->n_plans += 1;
        }
        S->used -= job->footprint;
        S->free_pipes += 1;
        S->epoch += 1;
        S->cv_sched.notify_all();
        S->cv_poll.notify_all();
        if (S->stop && S->inflight.empty()) return;
    }
}

extern "C" {

int mppi_server_create(const mppi_server_config* cfg, mppi_server** out) {
    if (!cfg || !out) return sfail(nullptr, MPPI_ERR_ARG, "NULL argument");
    *out = nullptr;
    if (cfg->max_sessions < 1 || cfg->max_batch < 1 || cfg->pipelines < 1 || cfg->hbm_budget_bytes < 1)
        return sfail(nullptr, MPPI_ERR_ARG, "server capacities out of range");
    mppi_server* S = new (std::nothrow) mppi_server();
    if (!S) return sfail(nullptr, MPPI_ERR_OOM, "host allocation failed");
    S->cfg = *cfg;
    int rc = mppi_batch_create(cfg->max_sessions, cfg->max_batch, cfg->max_samples, cfg->max_rollout_steps, cfg->max_T,
                               cfg->max_ref, cfg->max_circ, cfg->noise_bf16, cfg->pipelines, cfg->device, &S->batch);
    if (rc != MPPI_OK) {
        std::string m = mppi_batch_last_error(nullptr);
        delete S;
        return sfail(nullptr, rc, "batch engine: " + m);
    }
    S->session_busy.assign((size_t)cfg->max_sessions, 0);
    S->budget = (size_t)cfg->hbm_budget_bytes;
    S->watchdog_ms = cfg->watchdog_ms > 0.0 ? cfg->watchdog_ms : 0.0;
    S->free_pipes = cfg->pipelines;
    S->sched = std::thread(scheduler_loop, S);
    S->compl_ = std::thread(completion_loop, S);
    *out = S;
    return MPPI_OK;
}

int mppi_server_autotune(mppi_server* S, const mppi_params* params, const double* x0, const double* ref_xy,
                         int32_t n_ref, const mppi_circle* circ, int32_t n_circ, int32_t n_plans, int32_t* group,
                         int32_t* block) {
    if (!S || !params || n_plans < 1) return sfail(S, MPPI_ERR_ARG, "bad argument");
    std::vector<mppi_request> rq((size_t)n_plans);
    std::vector<std::vector<double>> u((size_t)n_plans), x((size_t)n_plans);
    for (int i = 0; i < n_plans; ++i) {
        u[(size_t)i].assign(2 * (size_t)params->T, 0.0);
        x[(size_t)i].assign(4 * (size_t)(params->T + 1), 0.0);
        mppi_request& q = rq[(size_t)i];
        memset(&q, 0, sizeof(q));
        q.params = params;
        q.slot = i % S->cfg.max_sessions;
        q.x0 = x0;
        q.ref_xy = ref_xy;
        q.n_ref = n_ref;
        q.circ = circ;
        q.n_circ = n_circ;
        q.u_out = u[(size_t)i].data();
        q.x_out = x[(size_t)i].data();
    }
    std::lock_guard<std::mutex> lk(S->mu);
    if (!S->inflight.empty() || !S->queue.empty()) return sfail(S, MPPI_ERR_CAPACITY, "tune an idle server");
    int rc = mppi_batch_autotune(S->batch, rq.data(), n_plans, group, block);
    if (rc != MPPI_OK) return sfail(S, rc, mppi_batch_last_error(S->batch));
    return MPPI_OK;
}

int mppi_server_enqueue(mppi_server* S, const mppi_params* params, int32_t session, const double* x0,
                        const double* ref_xy, int32_t n_ref, const mppi_circle* circ, int32_t n_circ,
                        const double* centres, uint64_t* request_id) {
    if (!S || !params || !x0 || !ref_xy || (n_circ > 0 && !circ)) return sfail(S, MPPI_ERR_ARG, "NULL argument");
    if (session < 0 || session >= S->cfg.max_sessions) return sfail(S, MPPI_ERR_ARG, "session out of range");
    if (params->model != 0 || params->cost_to_go != 0)
        return sfail(S, MPPI_ERR_ARG, "the server runs model 0 with whole-cost weights");
    if (params->T > S->cfg.max_T || n_ref > S->cfg.max_ref || n_circ > S->cfg.max_circ || n_ref < 2 || n_circ < 0 ||
        (long long)params->K > S->cfg.max_samples || (long long)params->K * params->T > S->cfg.max_rollout_steps)
        return sfail(S, MPPI_ERR_CAPACITY, "request above the server's capacities");
    auto r = std::make_unique<Req>();
    r->session = session;
    r->params = *params;
    r->x0.assign(x0, x0 + 4);
    r->ref.assign(ref_xy, ref_xy + 2 * (size_t)n_ref);
    if (n_circ > 0) r->circ.assign(reinterpret_cast<const double*>(circ), reinterpret_cast<const double*>(circ) + 5 * (size_t)n_circ);
    if (centres) r->centres.assign(centres, centres + 2 * (size_t)params->T * n_circ);
    r->n_ref = n_ref;
    r->n_circ = n_circ;
    r->u.assign(2 * (size_t)params->T, 0.0);
    r->x.assign(4 * (size_t)(params->T + 1), 0.0);
    r->footprint = footprint_of(*params, n_ref, n_circ);
    if (r->footprint > S->budget) return sfail(S, MPPI_ERR_CAPACITY, "request larger than the HBM budget");
    r->t_arrive = Clock::now();
    std::lock_guard<std::mutex> lk(S->mu);
    r->id = S->next_id++;
    if (request_id) *request_id = r->id;
    S->queue.push_back(std::move(r));
    S->epoch += 1;
    S->cv_sched.notify_all();
    return MPPI_OK;
}

int mppi_server_poll(mppi_server* S, mppi_result* out, int32_t max, double* u_out, double* x_out, int32_t max_T,
                     int32_t wait_ms, int32_t* n_out) {
    if (!S || !out || !n_out || max < 1) return sfail(S, MPPI_ERR_ARG, "bad argument");
    std::unique_lock<std::mutex> lk(S->mu);
    if (S->done.empty() && wait_ms > 0)
        S->cv_poll.wait_for(lk, std::chrono::milliseconds(wait_ms), [&] { return !S->done.empty() || S->stop; });
    int n = 0;
    while (n < max && !S->done.empty()) {
        std::unique_ptr<Req> r = std::move(S->done.front());
        S->done.pop_front();
        mppi_result& o = out[n];
        o.request_id = r->id;
        o.session = r->session;
        o.status = r->status;
        o.T = r->params.T;
        o.latency_us = std::chrono::duration<double, std::micro>(r->t_done - r->t_arrive).count();
        o.queue_us = std::chrono::duration<double, std::micro>(r->t_submit - r->t_arrive).count();
        o.info = r->info;
        if ((u_out || x_out) && r->params.T > max_T) {
            // the caller's rows are too short for this result's u* and x*: not copied, and said so
            o.status = MPPI_ERR_CAPACITY;
        } else {
            if (u_out) memcpy(u_out + (size_t)n * max_T * 2, r->u.data(), r->u.size() * sizeof(double));
            if (x_out) memcpy(x_out + (size_t)n * (max_T + 1) * 4, r->x.data(), r->x.size() * sizeof(double));
        }
        ++n;
    }
    *n_out = n;
    return MPPI_OK;
}

int mppi_server_pending(mppi_server* S, int32_t* queued, int32_t* in_flight, uint64_t* batches, uint64_t* plans) {
    if (!S) return sfail(nullptr, MPPI_ERR_ARG, "NULL server");
    std::lock_guard<std::mutex> lk(S->mu);
    if (queued) *queued = (int32_t)S->queue.size();
    if (in_flight) {
        int n = 0;
        for (auto& j : S->inflight) n += (int)j->reqs.size();
        *in_flight = n;
    }
    if (batches) *batches = S->n_batches;
    if (plans) *plans = S->n_plans;
    return MPPI_OK;
}

int mppi_server_set_controls(mppi_server* S, int32_t session, const double* U, int32_t T, uint64_t iter) {
    if (!S) return sfail(nullptr, MPPI_ERR_ARG, "NULL server");
    std::lock_guard<std::mutex> lk(S->mu);
    if (session < 0 || session >= S->cfg.max_sessions || S->session_busy[(size_t)session])
        return sfail(S, MPPI_ERR_ARG, "session out of range or in flight");
    return mppi_batch_set_controls(S->batch, session, U, T, iter);
}

int mppi_server_destroy(mppi_server* S) {
    if (!S) return MPPI_OK;
    {
        std::unique_lock<std::mutex> lk(S->mu);
        // let the batches in flight finish
        S->cv_poll.wait_for(lk, std::chrono::seconds(30), [&] { return S->inflight.empty(); });
        S->stop = true;
    }
    S->cv_sched.notify_all();
    S->cv_done.notify_all();
    S->cv_poll.notify_all();
    if (S->sched.joinable()) S->sched.join();
    if (S->compl_.joinable()) S->compl_.join();
    mppi_batch_destroy(S->batch);
    delete S;
    return MPPI_OK;
}

int mppi_server_set_watchdog(mppi_server* S, double watchdog_ms) {
    if (!S) return sfail(nullptr, MPPI_ERR_ARG, "NULL server");
    if (std::isnan(watchdog_ms)) return sfail(S, MPPI_ERR_ARG, "watchdog_ms is NaN");
    std::lock_guard<std::mutex> lk(S->mu);
    S->watchdog_ms = watchdog_ms > 0.0 ? watchdog_ms : 0.0;
    return MPPI_OK;
}

int mppi_server_timeouts(mppi_server* S, uint64_t* n) {
    if (!S || !n) return sfail(S, MPPI_ERR_ARG, "NULL argument");
    std::lock_guard<std::mutex> lk(S->mu);
    *n = S->n_timeouts;
    return MPPI_OK;
}

// Session table file: "MPPISNAP", version 1, max_sessions, max_T, then per session its
// iteration counter and its warm start U[max_T][2] (little-endian as written by this host).
static const char kSnapMagic[8] = {'M', 'P', 'P', 'I', 'S', 'N', 'A', 'P'};

int mppi_server_snapshot(mppi_server* S, const char* path) {
    if (!S || !path) return sfail(S, MPPI_ERR_ARG, "NULL argument");
    std::lock_guard<std::mutex> lk(S->mu);
    if (!S->inflight.empty() || !S->queue.empty()) return sfail(S, MPPI_ERR_CAPACITY, "snapshot an idle server");
    FILE* f = fopen(path, "wb");
    if (!f) return sfail(S, MPPI_ERR_ARG, std::string("cannot write ") + path);
    const int32_t hdr[3] = {1, S->cfg.max_sessions, S->cfg.max_T};
    bool ok = fwrite(kSnapMagic, 1, 8, f) == 8 && fwrite(hdr, sizeof(int32_t), 3, f) == 3;
    std::vector<double> U(2 * (size_t)S->cfg.max_T);
    for (int s = 0; ok && s < S->cfg.max_sessions; ++s) {
        uint64_t iter = 0;
        if (mppi_batch_get_controls(S->batch, s, U.data(), S->cfg.max_T, &iter) != MPPI_OK) {
            fclose(f);
            return sfail(S, MPPI_ERR_CUDA, std::string("session read: ") + mppi_batch_last_error(S->batch));
        }
        ok = fwrite(&iter, sizeof(iter), 1, f) == 1 && fwrite(U.data(), sizeof(double), U.size(), f) == U.size();
    }
    ok = (fclose(f) == 0) && ok;
    return ok ? MPPI_OK : sfail(S, MPPI_ERR_ARG, std::string("write failed: ") + path);
}

int mppi_server_restore(mppi_server* S, const char* path) {
    if (!S || !path) return sfail(S, MPPI_ERR_ARG, "NULL argument");
    std::lock_guard<std::mutex> lk(S->mu);
    if (!S->inflight.empty() || !S->queue.empty()) return sfail(S, MPPI_ERR_CAPACITY, "restore into an idle server");
    FILE* f = fopen(path, "rb");
    if (!f) return sfail(S, MPPI_ERR_ARG, std::string("cannot read ") + path);
    char magic[8];
    int32_t hdr[3];
    if (fread(magic, 1, 8, f) != 8 || memcmp(magic, kSnapMagic, 8) != 0 || fread(hdr, sizeof(int32_t), 3, f) != 3 ||
        hdr[0] != 1 || hdr[1] != S->cfg.max_sessions || hdr[2] != S->cfg.max_T) {
        fclose(f);
        return sfail(S, MPPI_ERR_ARG, "not a session table of this server's size");
    }
    std::vector<double> U(2 * (size_t)S->cfg.max_T);
    for (int s = 0; s < S->cfg.max_sessions; ++s) {
        uint64_t iter = 0;
        if (fread(&iter, sizeof(iter), 1, f) != 1 || fread(U.data(), sizeof(double), U.size(), f) != U.size()) {
            fclose(f);
            return sfail(S, MPPI_ERR_ARG, "session table truncated");
        }
        const int rc = mppi_batch_set_controls(S->batch, s, U.data(), S->cfg.max_T, iter);
        if (rc != MPPI_OK) {
            fclose(f);
            return sfail(S, rc, std::string("session write: ") + mppi_batch_last_error(S->batch));
        }
    }
    fclose(f);
    return MPPI_OK;
}

const char* mppi_server_last_error(mppi_server* S) { return S ? S->err.c_str() : g_srv_err.c_str(); }

}  // extern "C"
