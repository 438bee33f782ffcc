// Serving loop: continuous batching of cavity solves over an lbm_batch whose
// arena is the device-memory budget (declared in include/lbm.h).
#include <cuda_runtime.h>

#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <deque>
#include <new>
#include <string>
#include <vector>

#include "../../include/lbm.h"

namespace {

thread_local std::string g_err;

struct Pending {
    lbm_instance inst;
    double tol, nush_tol;
    int64_t max_steps;
    int64_t id;
    double t_submit;
};

struct Running {
    bool used = false;
    Pending req{};
    double t_admit = 0;
    int checks = 0;
    double prev[4] = {0, 0, 0, 0};
};

}  // namespace

struct lbm_server {
    lbm_batch* batch = nullptr;
    int max_slots = 0, check_every = 100;
    std::deque<Pending> queue;
    std::vector<Running> run;
    std::vector<lbm_result> done;
    std::vector<double> r, nush;
    std::vector<int> div;
    std::chrono::steady_clock::time_point t0;
    std::string err;

    double now() const {
        return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
    lbm_status fail(lbm_status s, const char* fmt, ...) {
        char b[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(b, sizeof b, fmt, ap);
        va_end(ap);
        err = b;
        g_err = b;
        return s;
    }
    int active() const {
        int n = 0;
        for (const Running& x : run) n += x.used;
        return n;
    }
};

extern "C" {

lbm_status lbm_server_create(size_t budget_bytes, int max_slots, int check_every,
                             const lbm_options* opt, lbm_server** out) {
    if (!out || max_slots < 1 || check_every < 2 || budget_bytes == 0) {
        g_err = "lbm_server_create: need out, max_slots >= 1, check_every >= 2, budget > 0";
        return LBM_ERR_INVALID;
    }
    *out = nullptr;
    lbm_server* s = new (std::nothrow) lbm_server();
    if (!s) {
        g_err = "lbm_server_create: out of host memory";
        return LBM_ERR_NOMEM;
    }
    s->max_slots = max_slots;
    s->check_every = check_every + (check_every & 1);
    s->run.assign(max_slots, Running{});
    s->r.assign(max_slots, 0.0);
    s->div.assign(max_slots, 0);
    s->nush.assign((size_t)max_slots * 4, 0.0);
    s->t0 = std::chrono::steady_clock::now();
    lbm_status st = lbm_batch_create(nullptr, 0, max_slots, budget_bytes, opt, &s->batch);
    if (st != LBM_OK) {
        g_err = std::string("lbm_server_create: ") + lbm_batch_last_error(nullptr);
        delete s;
        return st;
    }
    *out = s;
    return LBM_OK;
}

lbm_status lbm_server_submit(lbm_server* s, const lbm_instance* inst, double tol, double nush_tol,
                             int64_t max_steps, int64_t id) {
    if (!s || !inst || !(tol >= 0.0) || !(nush_tol >= 0.0) || max_steps < 1) {
        g_err = "lbm_server_submit: need a server, an instance, tol, nush_tol >= 0 and max_steps >= 1";
        if (s) s->err = g_err;
        return LBM_ERR_INVALID;
    }
    if (lbm_batch_instance_bytes(lbm_grid{inst->params.nx, inst->params.ny}, nullptr) == 0)
        return s->fail(LBM_ERR_INVALID, "lbm_server_submit: request %lld: grid too small", (long long)id);
    Pending p;
    p.inst = *inst;
    p.tol = tol;
    p.nush_tol = nush_tol;
    p.max_steps = max_steps;
    p.id = id;
    p.t_submit = s->now();
    s->queue.push_back(p);
    return LBM_OK;
}

lbm_status lbm_server_tick(lbm_server* s, int* active) {
    if (!s) {
        g_err = "lbm_server_tick: NULL server";
        return LBM_ERR_INVALID;
    }
    // 1. admission, first come first served with backfill
    for (auto it = s->queue.begin(); it != s->queue.end();) {
        if (s->active() >= s->max_slots) break;
        int slot = -1;
        lbm_status st = lbm_batch_add(s->batch, &it->inst, &slot);
        if (st == LBM_ERR_NOMEM) {   // does not fit now: try the next one
            ++it;
            continue;
        }
        if (st != LBM_OK) {          // invalid request: fail it, keep serving
            lbm_result res;
            std::memset(&res, 0, sizeof res);
            res.id = it->id;
            res.status = st;
            res.t_submit = it->t_submit;
            res.t_admit = res.t_done = s->now();
            s->done.push_back(res);
            it = s->queue.erase(it);
            continue;
        }
        Running& r = s->run[slot];
        r.used = true;
        r.req = *it;
        r.t_admit = s->now();
        r.checks = 0;
        it = s->queue.erase(it);
    }
    if (s->active() == 0) {
        if (active) *active = 0;
        return LBM_OK;
    }
    // 2. one fused launch per step for every cavity in flight
    lbm_status st = lbm_batch_step(s->batch, s->check_every);
    if (st == LBM_OK) st = lbm_batch_residual(s->batch, s->r.data(), s->div.data());
    if (st == LBM_OK) st = lbm_batch_nusselt_sherwood(s->batch, s->nush.data());
    if (st != LBM_OK) return s->fail(st, "lbm_server_tick: %s", lbm_batch_last_error(s->batch));
    // 3. retire
    bool any = false;
    std::vector<int> finish(s->max_slots, -1);
    for (int k = 0; k < s->max_slots; ++k) {
        Running& r = s->run[k];
        if (!r.used) continue;
        r.checks += 1;
        const int64_t steps = lbm_batch_time(s->batch, k);
        const double* ns = &s->nush[(size_t)k * 4];
        double dn = 0.0;
        bool finite = true;
        for (int q = 0; q < 4; ++q) {
            finite = finite && std::isfinite(ns[q]);
            const double d = std::fabs(ns[q] - r.prev[q]) / std::fmax(std::fabs(ns[q]), 1e-300);
            dn = d > dn ? d : dn;
            r.prev[q] = ns[q];
        }
        if (s->div[k] || !finite || (!std::isfinite(s->r[k]) && r.checks > 1))
            finish[k] = LBM_ERR_DIVERGED;
        else if ((r.req.tol > 0.0 && s->r[k] < r.req.tol) ||
                 (r.req.nush_tol > 0.0 && r.checks > 1 && dn < r.req.nush_tol))
            finish[k] = LBM_OK;
        else if (steps >= r.req.max_steps)
            finish[k] = LBM_ERR_UNCONVERGED;
        any = any || finish[k] >= 0;
    }
    if (any) {
        const double t = s->now();
        for (int k = 0; k < s->max_slots; ++k) {
            if (finish[k] < 0) continue;
            Running& r = s->run[k];
            lbm_result res;
            std::memset(&res, 0, sizeof res);
            res.id = r.req.id;
            res.status = finish[k];
            res.steps = lbm_batch_time(s->batch, k);
            res.residual = s->r[k];
            for (int q = 0; q < 4; ++q) res.nush[q] = s->nush[(size_t)k * 4 + q];
            res.t_submit = r.req.t_submit;
            res.t_admit = r.t_admit;
            res.t_done = t;
            s->done.push_back(res);
            st = lbm_batch_remove(s->batch, k);
            if (st != LBM_OK) return s->fail(st, "lbm_server_tick: %s", lbm_batch_last_error(s->batch));
            r = Running{};
        }
    }
    if (active) *active = s->active();
    return LBM_OK;
}

lbm_status lbm_server_poll(lbm_server* s, lbm_result* out, int cap, int* n) {
    if (!s || !n || (cap > 0 && !out)) {
        g_err = "lbm_server_poll: NULL argument";
        return LBM_ERR_INVALID;
    }
    const int m = (int)std::min<size_t>((size_t)std::max(cap, 0), s->done.size());
    for (int k = 0; k < m; ++k) out[k] = s->done[k];
    s->done.erase(s->done.begin(), s->done.begin() + m);
    *n = m;
    return LBM_OK;
}

double lbm_server_clock(const lbm_server* s) { return s ? s->now() : 0.0; }

lbm_status lbm_server_info(const lbm_server* s, int* queued, int* active, int* done, size_t* arena_used) {
    if (!s) {
        g_err = "lbm_server_info: NULL server";
        return LBM_ERR_INVALID;
    }
    if (queued) *queued = (int)s->queue.size();
    if (active) *active = s->active();
    if (done) *done = (int)s->done.size();
    if (arena_used) lbm_batch_info(s->batch, nullptr, nullptr, nullptr, arena_used);
    return LBM_OK;
}

void lbm_server_destroy(lbm_server* s) {
    if (!s) return;
    lbm_batch_destroy(s->batch);
    delete s;
}

const char* lbm_server_last_error(const lbm_server* s) { return s ? s->err.c_str() : g_err.c_str(); }

}  // extern "C"
