// server.cu -- request loop that runs discharges to periodic steady state.
//
// Clients submit discharge parameters from any thread; one worker thread owns
// the device work.  It admits queued requests in arrival order while their
// state fits the device-memory budget, keeps every admitted discharge
// resident, steps all of them together (one pic_batch, or a plain loop of
// pic_step calls when batching is off) in chunks of a fraction of an RF
// period, and at the end of each window of whole RF periods compares a
// discharge's window-averaged electron and ion densities with those of the
// window before.
// A discharge whose relative change (of the inventories, the spatial integrals
// of the densities, or of the profiles in L2 over the nodes; the larger of the
// two species) falls below the tolerance has reached periodic steady state: its
// last period-averaged n_e, n_i and phi are kept on the host, its device state
// is released and its request completes.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/pic_gb300.h"
#include "launch.h"

using pg::set_last_error;

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
    int64_t id = 0;
    pic_params p;
    pic_request_info info;
    long long steps = 0;                 // steps run since admission
    long long period = 0;                // steps per RF period of this discharge
    int slot = -1;                       // batch slot (batched mode)
    pic_ctx* ctx = nullptr;              // the discharge while it runs
    std::vector<double> prev[2];         // previous window's n_e, n_i
    std::vector<double> res[3];          // last window's n_e, n_i, phi
    std::string err;
};

// particles per unit electrode area: sum of node densities times node volumes
double inventory(const std::vector<double>& n, double dx)
{
    double s = 0.0;
    for (size_t m = 0; m < n.size(); ++m) s += n[m] * ((m == 0 || m + 1 == n.size()) ? 0.5 * dx : dx);
    return s;
}

double rel_change(const std::vector<double>& a, const std::vector<double>& b)
{
    double num = 0.0, den = 0.0;
    for (size_t m = 0; m < a.size(); ++m) {
        const double d = a[m] - b[m];
        num += d * d;
        den += a[m] * a[m];
    }
    return den > 0.0 ? std::sqrt(num / den) : (num > 0.0 ? INFINITY : 0.0);
}

long long steps_per_period(const pic_params& p)
{
    const double r = 1.0 / (p.rf_freq_hz * p.dt);
    const long long P = std::llrint(r);
    return (P >= 1 && P <= (1ll << 24) && std::fabs((double)P * p.rf_freq_hz * p.dt - 1.0) < 1e-9) ? P : 0;
}

}  // namespace

struct pic_server {
    pic_server_opts o;
    int device = 0;
    cudaStream_t stream = nullptr;
    pic_batch* batch = nullptr;
    Clock::time_point t0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<int64_t> queue;
    std::unordered_map<int64_t, std::unique_ptr<Request>> req;
    std::vector<Request*> running;       // touched by the worker only
    int64_t next_id = 1;
    int64_t bytes_used = 0;
    long long period = 0, chunk = 0;     // steps per RF period of the first request admitted since the
                                         // server was last idle, and per worker chunk (a divisor of
                                         // every running period and a multiple of every running
                                         // diag_every); both reset when nothing runs
    bool stop = false;
    std::string fatal;
    pic_server_stats st;
    std::thread worker;

    double now() const { return std::chrono::duration<double>(Clock::now() - t0).count(); }
};

namespace {

// Complete r (admitted: its state was counted in the memory in use).
void finish(pic_server* S, Request* r, int state, const std::string& err, bool was_running)
{
    std::lock_guard<std::mutex> lk(S->mu);
    r->info.state = state;
    r->info.t_done = S->now();
    r->err = err;
    S->bytes_used -= r->info.bytes;
    if (was_running) S->st.running -= 1;
    else S->st.queued -= 1;
    S->st.done += 1;
    S->cv_done.notify_all();
}

void release(pic_server* S, Request* r)
{
    if (S->batch && r->slot >= 0) pic_batch_remove(S->batch, r->slot);
    else if (r->ctx) pic_destroy(r->ctx);
    r->ctx = nullptr;
    r->slot = -1;
}

// The worker's chunk for a first request of period P and sampling stride de:
// the largest chunk P / m, m <= chunks_per_period, that divides P and is a
// multiple of de (P itself when none is).
long long chunk_for(const pic_server* S, long long P, int de)
{
    const int want = std::max(1, S->o.chunks_per_period);
    for (int m = want; m >= 1; --m)
        if (P % m == 0 && (P / m) % de == 0) return P / m;
    return P;
}

// Whether r can join the running discharges: its period a multiple of the
// chunk and the chunk a multiple of its sampling stride.  A request that cannot
// waits in the queue until the running ones have finished.
bool fits(const pic_server* S, const Request* r)
{
    const long long P = steps_per_period(r->p);
    if (P == 0 || S->period == 0) return true;        // (P == 0 fails at admission)
    const int de = r->p.diag_every > 0 ? r->p.diag_every : 1;
    return P % S->chunk == 0 && S->chunk % de == 0;
}

// Admit r: create its discharge.  Returns false (and completes r as failed)
// if its RF period is not a whole number of steps or creation fails.
bool admit(pic_server* S, Request* r)
{
    const long long P = steps_per_period(r->p);
    std::string why;
    if (P == 0) why = "the RF period is not a whole number of steps";
    int rc = PIC_OK;
    if (why.empty()) {
        if (S->batch) {
            rc = pic_batch_add(S->batch, &r->p, &r->slot);
            if (!rc) rc = pic_batch_ctx(S->batch, r->slot, &r->ctx);
        } else {
            rc = pic_create(&r->p, S->stream, &r->ctx);
        }
        if (rc) why = std::string(pic_strerror(rc)) + ": " + pic_last_error();
    }
    if (!why.empty()) {
        release(S, r);
        finish(S, r, PIC_REQ_FAILED, why, false);
        return false;
    }
    r->period = P;
    std::lock_guard<std::mutex> lk(S->mu);
    r->info.state = PIC_REQ_RUNNING;
    r->info.t_admit = S->now();
    S->st.queued -= 1;
    S->st.running += 1;
    return true;
}

// At r's period boundary; at the end of each window of window_periods
// periods: the window's averages, the steady-state test and a new window.
// Returns the state r ends in, or PIC_REQ_RUNNING.
int period_check(pic_server* S, Request* r, std::string* err)
{
    int periods;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        periods = ++r->info.periods;
    }
    const bool capped = S->o.max_periods > 0 && periods >= S->o.max_periods;
    if (periods % S->o.window_periods != 0) return capped ? PIC_REQ_MAX_PERIODS : PIC_REQ_RUNNING;
    std::vector<double> v[3];
    const int kinds[3] = {PIC_DIAG_NE, PIC_DIAG_NI, PIC_DIAG_PHI};
    for (int k = 0; k < 3; ++k) {
        int64_t n = 0;
        v[k].resize((size_t)r->p.n_cells + 1);
        int rc = pic_diag(r->ctx, kinds[k], v[k].data(), (int64_t)v[k].size(), &n);
        if (!rc) rc = pic_sync(r->ctx);
        if (rc) {
            *err = std::string(pic_strerror(rc)) + ": " + pic_last_error();
            return PIC_REQ_FAILED;
        }
    }
    int rc = pic_reset_averages(r->ctx);
    if (rc) {
        *err = std::string(pic_strerror(rc)) + ": " + pic_last_error();
        return PIC_REQ_FAILED;
    }
    double change = INFINITY;
    if (!r->prev[0].empty()) {
        if (S->o.criterion == PIC_STEADY_PROFILE) {
            change = std::max(rel_change(v[0], r->prev[0]), rel_change(v[1], r->prev[1]));
        } else {
            const double dx = r->p.gap_m / r->p.n_cells;
            for (int k = 0; k < 2; ++k) {
                const double a = inventory(v[k], dx), b = inventory(r->prev[k], dx);
                const double c = a > 0.0 ? std::fabs(a - b) / a : (b > 0.0 ? INFINITY : 0.0);
                change = k == 0 ? c : std::max(change, c);
            }
        }
    }
    r->prev[0] = v[0];
    r->prev[1] = v[1];
    std::lock_guard<std::mutex> lk(S->mu);
    r->info.change = std::isfinite(change) ? change : -1.0;
    for (int k = 0; k < 3; ++k) r->res[k] = v[k];
    if (periods >= S->o.min_periods && change < S->o.tol) return PIC_REQ_CONVERGED;
    return capped ? PIC_REQ_MAX_PERIODS : PIC_REQ_RUNNING;
}

void fail_all(pic_server* S, const std::string& why)
{
    for (Request* r : S->running) {
        release(S, r);
        finish(S, r, PIC_REQ_FAILED, why, true);
    }
    S->running.clear();
    std::lock_guard<std::mutex> lk(S->mu);
    S->fatal = why;
}

void work(pic_server* S)
{
    cudaSetDevice(S->device);
    for (;;) {
        std::vector<Request*> adm;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            S->cv_work.wait(lk, [&] { return S->stop || !S->queue.empty() || !S->running.empty(); });
            if (S->stop) break;
            if (S->running.empty()) S->period = S->chunk = 0;   // idle: the next request sets the schedule
            while (!S->queue.empty()) {                     // arrival order, within the budget
                Request* r = S->req[S->queue.front()].get();
                if (S->bytes_used + r->info.bytes > S->o.hbm_budget_bytes) break;
                if (!fits(S, r)) break;                     // waits until the running ones finish
                const long long P = steps_per_period(r->p);
                if (S->period == 0 && P > 0) {
                    S->period = P;
                    S->chunk = chunk_for(S, P, r->p.diag_every > 0 ? r->p.diag_every : 1);
                }
                S->queue.pop_front();
                S->bytes_used += r->info.bytes;
                adm.push_back(r);
            }
        }
        for (Request* r : adm)
            if (admit(S, r)) S->running.push_back(r);
        if (S->running.empty()) continue;
        const auto t1 = Clock::now();
        int rc = PIC_OK;
        if (S->batch) rc = pic_batch_step(S->batch, S->chunk);
        else
            for (Request* r : S->running)
                if (!rc) rc = pic_step(r->ctx, S->chunk);
        if (!rc && cudaStreamSynchronize(S->stream) != cudaSuccess) rc = PIC_ERR_CUDA;
        if (rc) {
            fail_all(S, std::string(pic_strerror(rc)) + ": " + pic_last_error());
            continue;
        }
        long long parts = 0;
        for (Request* r : S->running) parts += r->info.particles;
        {
            std::lock_guard<std::mutex> lk(S->mu);
            S->st.chunks += 1;
            S->st.steps += S->chunk;
            S->st.particle_steps += (double)parts * (double)S->chunk;
            S->st.busy_s += std::chrono::duration<double>(Clock::now() - t1).count();
        }
        std::vector<Request*> keep;
        for (Request* r : S->running) {
            r->steps += S->chunk;
            int state = PIC_REQ_RUNNING;
            std::string err;
            if (r->steps % r->period == 0) state = period_check(S, r, &err);
            if (state == PIC_REQ_RUNNING) {
                keep.push_back(r);
                continue;
            }
            release(S, r);
            finish(S, r, state, err, true);
        }
        S->running.swap(keep);
    }
    for (Request* r : S->running) release(S, r);
    S->running.clear();
}

int lookup(pic_server* S, int64_t id, Request** out)
{
    auto it = S->req.find(id);
    if (it == S->req.end()) {
        set_last_error("unknown request id");
        return PIC_ERR_INVALID_ARG;
    }
    *out = it->second.get();
    return PIC_OK;
}

bool finished(int state) { return state >= PIC_REQ_CONVERGED; }

}  // namespace

extern "C" {

int pic_server_opts_default(pic_server_opts* o)
{
    if (!o) {
        set_last_error("opts is NULL");
        return PIC_ERR_INVALID_ARG;
    }
    std::memset(o, 0, sizeof *o);
    o->hbm_budget_bytes = 0;
    o->min_periods = 2;
    o->max_periods = 0;
    o->tol = 0.01;
    o->batched = 1;
    o->graphs = 1;
    o->chunks_per_period = 10;
    o->criterion = PIC_STEADY_INVENTORY;
    o->window_periods = 1;
    return PIC_OK;
}

int pic_server_create(const pic_server_opts* opts, pic_server** out)
{
    if (!out) {
        set_last_error("out is NULL");
        return PIC_ERR_INVALID_ARG;
    }
    *out = nullptr;
    pic_server_opts o;
    if (opts) o = *opts;
    else pic_server_opts_default(&o);
    if (o.min_periods < 2 || o.max_periods < 0 || !(o.tol > 0) || o.hbm_budget_bytes < 0 ||
        o.chunks_per_period < 0 || (o.criterion != PIC_STEADY_INVENTORY && o.criterion != PIC_STEADY_PROFILE) ||
        o.window_periods < 1) {
        set_last_error("min_periods >= 2, max_periods >= 0, tol > 0, budget >= 0, criterion 0 or 1, "
                       "window_periods >= 1");
        return PIC_ERR_INVALID_ARG;
    }
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        set_last_error("no CUDA device visible");
        return PIC_ERR_NO_DEVICE;
    }
    auto S = std::make_unique<pic_server>();
    cudaGetDevice(&S->device);
    if (o.hbm_budget_bytes == 0) {                       // 80 % of what is free now
        size_t fr = 0, tot = 0;
        if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
            set_last_error("cudaMemGetInfo failed");
            return PIC_ERR_CUDA;
        }
        o.hbm_budget_bytes = (int64_t)(0.8 * (double)fr);
    }
    S->o = o;
    std::memset(&S->st, 0, sizeof S->st);
    S->st.budget = o.hbm_budget_bytes;
    if (cudaStreamCreateWithFlags(&S->stream, cudaStreamNonBlocking) != cudaSuccess) {
        set_last_error("cudaStreamCreate failed");
        return PIC_ERR_CUDA;
    }
    if (o.batched) {
        int rc = pic_batch_create(S->stream, &S->batch);
        if (!rc) rc = pic_batch_graphs(S->batch, o.graphs);
        if (rc) {
            cudaStreamDestroy(S->stream);
            return rc;
        }
    }
    S->t0 = Clock::now();
    pic_server* s = S.release();
    s->worker = std::thread(work, s);
    *out = s;
    return PIC_OK;
}

int pic_server_clock(pic_server* s, double* t)
{
    if (!s || !t) {
        set_last_error("NULL argument");
        return PIC_ERR_INVALID_ARG;
    }
    *t = s->now();
    return PIC_OK;
}

int pic_server_submit(pic_server* s, const pic_params* p, double t_arrival, int64_t* id)
{
    if (!s || !p || !id) {
        set_last_error("NULL argument");
        return PIC_ERR_INVALID_ARG;
    }
    int64_t bytes = 0;
    int rc = pic_state_bytes(p, &bytes);
    if (rc) return rc;
    auto r = std::make_unique<Request>();
    r->p = *p;
    std::memset(&r->info, 0, sizeof r->info);
    r->info.state = PIC_REQ_QUEUED;
    r->info.bytes = bytes;
    r->info.particles = p->n_e0 + p->n_i0;
    r->info.change = -1.0;
    r->info.t_admit = r->info.t_done = -1.0;
    std::lock_guard<std::mutex> lk(s->mu);
    const double t = s->now();
    r->info.t_arrival = (t_arrival >= 0.0 && t_arrival <= t) ? t_arrival : t;
    r->id = r->info.id = s->next_id++;
    *id = r->id;
    if (bytes > s->o.hbm_budget_bytes) {                 // could never be admitted
        r->info.state = PIC_REQ_REJECTED;
        r->info.t_done = t;
        r->err = "state larger than the device-memory budget";
        s->st.done += 1;
    } else {
        s->queue.push_back(r->id);
        s->st.queued += 1;
    }
    s->req.emplace(r->id, std::move(r));
    s->cv_work.notify_one();
    return PIC_OK;
}

int pic_server_info(pic_server* s, int64_t id, pic_request_info* info)
{
    if (!s || !info) {
        set_last_error("NULL argument");
        return PIC_ERR_INVALID_ARG;
    }
    std::lock_guard<std::mutex> lk(s->mu);
    Request* r = nullptr;
    int rc = lookup(s, id, &r);
    if (rc) return rc;
    *info = r->info;
    return PIC_OK;
}

int pic_server_wait(pic_server* s, int64_t id, double timeout_s, pic_request_info* info)
{
    if (!s) {
        set_last_error("server is NULL");
        return PIC_ERR_INVALID_ARG;
    }
    std::unique_lock<std::mutex> lk(s->mu);
    Request* r = nullptr;
    int rc = lookup(s, id, &r);
    if (rc) return rc;
    auto done = [&] { return finished(r->info.state); };
    if (timeout_s < 0) s->cv_done.wait(lk, done);
    else if (!s->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), done)) {
        set_last_error("request still running");
        return PIC_ERR_TIMEOUT;
    }
    if (info) *info = r->info;
    return PIC_OK;
}

int pic_server_error(pic_server* s, int64_t id, char* out, int64_t cap)
{
    if (!s || (!out && cap > 0)) {
        set_last_error("bad arguments");
        return PIC_ERR_INVALID_ARG;
    }
    std::lock_guard<std::mutex> lk(s->mu);
    Request* r = nullptr;
    int rc = lookup(s, id, &r);
    if (rc) return rc;
    if (cap > 0) {
        const size_t n = std::min((size_t)cap - 1, r->err.size());
        std::memcpy(out, r->err.data(), n);
        out[n] = 0;
    }
    return PIC_OK;
}

int pic_server_result(pic_server* s, int64_t id, int what, double* out, int64_t cap, int64_t* n)
{
    if (!s || what < 0 || what > 2 || (!out && cap > 0)) {
        set_last_error("bad arguments");
        return PIC_ERR_INVALID_ARG;
    }
    std::lock_guard<std::mutex> lk(s->mu);
    Request* r = nullptr;
    int rc = lookup(s, id, &r);
    if (rc) return rc;
    const std::vector<double>& v = r->res[what];
    if (n) *n = (int64_t)v.size();
    if (out) std::memcpy(out, v.data(), sizeof(double) * std::min((size_t)cap, v.size()));
    return PIC_OK;
}

int pic_server_forget(pic_server* s, int64_t id)
{
    if (!s) {
        set_last_error("server is NULL");
        return PIC_ERR_INVALID_ARG;
    }
    std::lock_guard<std::mutex> lk(s->mu);
    Request* r = nullptr;
    int rc = lookup(s, id, &r);
    if (rc) return rc;
    if (!finished(r->info.state)) {
        set_last_error("request has not finished");
        return PIC_ERR_INVALID_ARG;
    }
    s->req.erase(id);
    return PIC_OK;
}

int pic_server_status(pic_server* s, pic_server_stats* out)
{
    if (!s || !out) {
        set_last_error("NULL argument");
        return PIC_ERR_INVALID_ARG;
    }
    std::lock_guard<std::mutex> lk(s->mu);
    *out = s->st;
    out->bytes_used = s->bytes_used;
    if (!s->fatal.empty()) {
        set_last_error(s->fatal.c_str());
        return PIC_ERR_CUDA;
    }
    return PIC_OK;
}

void pic_server_destroy(pic_server* s)
{
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    if (s->worker.joinable()) s->worker.join();
    if (s->batch) pic_batch_destroy(s->batch);
    cudaStreamDestroy(s->stream);
    delete s;
}

}  // extern "C"
