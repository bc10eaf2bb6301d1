// Continuous-batching request server over the batched step.
//
// Requests (independent SPH runs of different sizes) arrive on a clock.  Each
// tick the server admits queued requests whose arrival time has passed, as
// long as a slot is free and the caller-provided device pool has room for the
// request's footprint (its particle arrays, its own context workspace and its
// share of the batch workspace); admitted problems get their first density and
// force evaluation and then join the resident set.  Every resident problem
// advances by one step per tick inside one batched launch set, so work of
// requests that arrived at different times overlaps on the device.  A problem
// that has taken its requested number of steps is copied back to host memory
// and its memory is released.  Latency = completion - arrival.
#include <algorithm>
#include <chrono>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <thread>
#include <vector>

#include "sph_internal.cuh"

namespace {

constexpr size_t kAlign = 256;

// First-fit allocator over the caller's pool (host bookkeeping only).
struct PoolAlloc {
    char *base = nullptr;
    size_t size = 0;
    std::map<size_t, size_t> free_;  // offset -> length
    void init(void *b, size_t s)
    {
        base = (char *)b;
        size_t a = ((uintptr_t)base + kAlign - 1) & ~(uintptr_t)(kAlign - 1);
        size_t skip = a - (uintptr_t)base;
        size = s > skip ? s - skip : 0;
        base += skip;
        free_.clear();
        if (size) free_[0] = size;
    }
    void *alloc(size_t n)
    {
        n = (n + kAlign - 1) & ~(kAlign - 1);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= n) {
                size_t off = it->first, len = it->second;
                free_.erase(it);
                if (len > n) free_[off + n] = len - n;
                return base + off;
            }
        }
        return nullptr;
    }
    void release(void *p, size_t n)
    {
        if (!p) return;
        n = (n + kAlign - 1) & ~(kAlign - 1);
        size_t off = (char *)p - base;
        auto it = free_.emplace(off, n).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
};

enum ReqState { QUEUED, RUNNING, DONE };

struct Req {
    uint64_t ticket;
    long long n;
    sph_params prm;
    int nsteps;
    double arrival, admitted = 0, completed = 0, t_sim = 0;
    std::vector<double> host[9];  // x y z vx vy vz u m h (inputs, then final state)
    std::vector<double> rho;
    ReqState state = QUEUED;
    int status = SPH_OK;
    int steps_done = 0;
    // resident data
    void *mem = nullptr;
    size_t mem_bytes = 0;
    sph_ctx *ctx = nullptr;
    sph_state st{};
};

size_t state_bytes(long long n) { return 18 * sizeof(double) * (size_t)(n > 0 ? n : 1) + 18 * kAlign; }

}  // namespace

struct sph_server {
    sph_server_cfg cfg;
    PoolAlloc pool;
    std::deque<Req *> queue;
    std::map<uint64_t, std::unique_ptr<Req>> all;
    std::vector<Req *> active;
    uint64_t next_ticket = 1;
    double clock = 0.0;
    std::chrono::steady_clock::time_point t0;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    void *staging = nullptr;      // pinned host memory for retiring requests' states
    size_t staging_bytes = 0;
};

static size_t footprint(const sph_params &p, long long n)
{
    size_t ws = sph_workspace_bytes(n, &p);
    // own workspace + its share of the batch workspace + the particle arrays
    return state_bytes(n) + 2 * ws + 4 * kAlign;
}

static double wall_now(const sph_server *s)
{
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - s->t0).count();
}

static int admit(sph_server *s, Req *r)
{
    cudaStream_t st = (cudaStream_t)s->cfg.stream;
    size_t sb = state_bytes(r->n), wb = sph_workspace_bytes(r->n, &r->prm);
    r->mem_bytes = sb + wb + kAlign;
    r->mem = s->pool.alloc(r->mem_bytes);
    if (!r->mem) return SPH_EAGAIN;
    char *p = (char *)r->mem;
    double **fields[18] = {&r->st.x, &r->st.y, &r->st.z, &r->st.vx, &r->st.vy, &r->st.vz, &r->st.u, &r->st.m,
                           &r->st.h, &r->st.rho, &r->st.omega, &r->st.P, &r->st.c, &r->st.ax, &r->st.ay,
                           &r->st.az, &r->st.du, &r->st.vsig};
    size_t arr = ((sizeof(double) * (size_t)(r->n > 0 ? r->n : 1)) + kAlign - 1) & ~(kAlign - 1);
    for (int k = 0; k < 18; ++k) {
        *fields[k] = (double *)p;
        p += arr;
    }
    void *ws = (void *)(((uintptr_t)p + kAlign - 1) & ~(uintptr_t)(kAlign - 1));
    for (int k = 0; k < 9; ++k)
        if (r->n > 0)
            cudaMemcpyAsync(*fields[k], r->host[k].data(), sizeof(double) * r->n, cudaMemcpyHostToDevice, st);
    sph_params prm = r->prm;
    prm.precision = s->cfg.precision;
    prm.flags = SPH_FLAG_ASYNC;
    int rc = sph_setup(&r->ctx, &prm, r->n, &r->st, ws, wb, s->cfg.stream);
    if (rc == SPH_OK) rc = sph_density_h(r->ctx);
    if (rc == SPH_OK) rc = sph_forces(r->ctx);
    if (rc != SPH_OK) {
        if (r->ctx) sph_destroy(r->ctx);
        r->ctx = nullptr;
        s->pool.release(r->mem, r->mem_bytes);
        r->mem = nullptr;
        r->status = rc;
        r->state = DONE;
        r->completed = s->clock;
        return rc;
    }
    r->state = RUNNING;
    r->admitted = s->clock;
    s->active.push_back(r);
    return SPH_OK;
}

// Copy the final states of the finished requests back: every array goes
// through the server's pinned staging buffer with cudaMemcpyAsync (one copy
// per array), then one synchronisation for all of them.
static void retire_all(sph_server *s, const std::vector<Req *> &done)
{
    if (done.empty()) return;
    cudaStream_t st = (cudaStream_t)s->cfg.stream;
    size_t need = 0;
    for (Req *r : done) need += 10 * sizeof(double) * (size_t)(r->n > 0 ? r->n : 0);
    if (need > s->staging_bytes) {
        if (s->staging) cudaFreeHost(s->staging);
        s->staging = nullptr;
        s->staging_bytes = 0;
        if (cudaHostAlloc(&s->staging, need, cudaHostAllocDefault) == cudaSuccess) s->staging_bytes = need;
        else s->staging = nullptr;
    }
    double *stage = (double *)s->staging;
    size_t off = 0;
    for (Req *r : done) {
        double *src[10] = {r->st.x, r->st.y, r->st.z, r->st.vx, r->st.vy, r->st.vz, r->st.u, r->st.m, r->st.h, r->st.rho};
        r->rho.resize(r->n);
        for (int k = 0; k < 10; ++k) {
            if (r->n <= 0) continue;
            double *dst = k < 9 ? r->host[k].data() : r->rho.data();
            if (stage) {
                cudaMemcpyAsync(stage + off, src[k], sizeof(double) * r->n, cudaMemcpyDeviceToHost, st);
                off += (size_t)r->n;
            } else {
                cudaMemcpyAsync(dst, src[k], sizeof(double) * r->n, cudaMemcpyDeviceToHost, st);
            }
        }
    }
    cudaStreamSynchronize(st);
    off = 0;
    for (Req *r : done) {
        for (int k = 0; k < 10 && stage; ++k) {
            if (r->n <= 0) continue;
            double *dst = k < 9 ? r->host[k].data() : r->rho.data();
            memcpy(dst, stage + off, sizeof(double) * r->n);
            off += (size_t)r->n;
        }
        sph_diag d;
        if (sph_diagnostics(r->ctx, &d) == SPH_OK) {
            r->t_sim = d.time;
            if (d.status != SPH_OK && r->status == SPH_OK) r->status = d.status;
        }
        sph_destroy(r->ctx);
        r->ctx = nullptr;
        s->pool.release(r->mem, r->mem_bytes);
        r->mem = nullptr;
        r->state = DONE;
        r->completed = s->clock;
    }
}

extern "C" {

int sph_server_create(sph_server **out, const sph_server_cfg *cfg)
{
    if (!out || !cfg) return SPH_EINVAL;
    *out = nullptr;
    if (!cfg->pool || cfg->pool_bytes < 4096 || cfg->max_slots < 1 || cfg->max_slots > 4096 || cfg->max_queue < 1)
        return SPH_EINVAL;
    if (cfg->precision != SPH_PREC_FP64 && cfg->precision != SPH_PREC_MIXED) return SPH_EINVAL;
    sph_server *s = new sph_server();
    s->cfg = *cfg;
    s->pool.init(cfg->pool, cfg->pool_bytes);
    s->t0 = std::chrono::steady_clock::now();
    cudaEventCreate(&s->ev0);
    cudaEventCreate(&s->ev1);
    *out = s;
    return SPH_OK;
}

int sph_server_submit(sph_server *s, const sph_request *req, uint64_t *ticket)
{
    if (!s || !req || !ticket) return SPH_EINVAL;
    if (req->n < 0 || req->nsteps < 1) return SPH_EINVAL;  // (a request asks for at least one step)
    const double *in[9] = {req->x, req->y, req->z, req->vx, req->vy, req->vz, req->u, req->m, req->h};
    if (req->n > 0)
        for (const double *p : in)
            if (!p) return SPH_EINVAL;
    sph_params prm = req->params;
    prm.precision = s->cfg.precision;
    if (prm.av_switch != SPH_AV_CONSTANT) return SPH_EINVAL;  // (per-particle alpha is not kept by the server)
    if (sph_workspace_bytes(req->n, &prm) == 0) return SPH_EINVAL;
    if (footprint(prm, req->n) > s->pool.size) return SPH_ETOOBIG;
    if ((int)s->queue.size() >= s->cfg.max_queue) return SPH_EBUSY;
    auto r = std::make_unique<Req>();
    r->ticket = s->next_ticket++;
    r->n = req->n;
    r->prm = prm;
    r->nsteps = req->nsteps;
    r->arrival = req->arrival;
    for (int k = 0; k < 9; ++k) r->host[k].assign(in[k], in[k] + (req->n > 0 ? req->n : 0));
    *ticket = r->ticket;
    // keep the queue ordered by arrival time (stable for equal times)
    auto pos = std::upper_bound(s->queue.begin(), s->queue.end(), r->arrival,
                                [](double a, const Req *q) { return a < q->arrival; });
    s->queue.insert(pos, r.get());
    s->all.emplace(r->ticket, std::move(r));
    return SPH_OK;
}

double sph_server_clock(const sph_server *s) { return s ? s->clock : 0.0; }

int sph_server_run(sph_server *s, double until, int virtual_clock)
{
    if (!s) return SPH_EINVAL;
    cudaStream_t st = (cudaStream_t)s->cfg.stream;
    for (;;) {
        if (!virtual_clock) s->clock = std::max(s->clock, wall_now(s));
        if (s->clock >= until) return SPH_OK;
        cudaEventRecord(s->ev0, st);
        // admission: arrival order, slots and pool memory permitting
        size_t resident = 0;
        for (Req *r : s->active) resident += footprint(r->prm, r->n);
        while (!s->queue.empty() && s->queue.front()->arrival <= s->clock &&
               (int)s->active.size() < s->cfg.max_slots) {
            Req *r = s->queue.front();
            if (resident + footprint(r->prm, r->n) > s->pool.size) break;
            s->queue.pop_front();
            int rc = admit(s, r);
            if (rc == SPH_EAGAIN) {  // fragmented pool: retry after a retirement
                s->queue.push_front(r);
                break;
            }
            if (rc == SPH_OK) resident += footprint(r->prm, r->n);
        }
        if (s->active.empty()) {
            if (s->queue.empty()) return SPH_OK;
            double next = s->queue.front()->arrival;
            if (next > s->clock) {
                if (virtual_clock) s->clock = std::min(next, until);
                else std::this_thread::sleep_for(std::chrono::microseconds(50));
                continue;
            }
            continue;
        }
        // one batched step over every resident problem; each request takes
        // its own problem's status (one failing problem fails no other)
        std::vector<sph_ctx *> ctxs;
        ctxs.reserve(s->active.size());
        for (Req *r : s->active) ctxs.push_back(r->ctx);
        std::vector<int> status(ctxs.size(), SPH_OK);
        size_t bw = sph_batch_workspace_bytes(ctxs.data(), (int)ctxs.size());
        void *bmem = bw ? s->pool.alloc(bw) : nullptr;
        if (bmem) {
            sph_batch *bt = nullptr;
            int rc = sph_batch_create(&bt, ctxs.data(), (int)ctxs.size(), bmem, bw, 0);
            if (rc == SPH_OK) rc = sph_batch_run(bt, 1);
            if (bt) {
                sph_batch_sync(bt, status.data());
                sph_batch_destroy(bt);
            }
            if (rc != SPH_OK)
                for (int &v : status)
                    if (v == SPH_OK) v = rc;
            s->pool.release(bmem, bw);
        } else {
            // no contiguous room: step the problems one by one
            for (size_t k = 0; k < ctxs.size(); ++k) {
                const int r2 = sph_step(ctxs[k], -1.0, nullptr);
                status[k] = r2 != SPH_OK ? r2 : sph_sync(ctxs[k]);
            }
        }
        cudaEventRecord(s->ev1, st);
        cudaEventSynchronize(s->ev1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, s->ev0, s->ev1);
        if (virtual_clock) s->clock += 1e-3 * ms;
        else s->clock = std::max(s->clock, wall_now(s));
        std::vector<Req *> keep, done;
        for (size_t k = 0; k < s->active.size(); ++k) {
            Req *r = s->active[k];
            r->steps_done += 1;
            if (status[k] != SPH_OK && r->status == SPH_OK) r->status = status[k];
            // a failed request stops here; the others go on
            if (r->steps_done >= r->nsteps || r->status != SPH_OK) done.push_back(r);
            else keep.push_back(r);
        }
        retire_all(s, done);
        s->active.swap(keep);
    }
}

int sph_server_poll(sph_server *s, uint64_t ticket, sph_result *out)
{
    if (!s || !out) return SPH_EINVAL;
    auto it = s->all.find(ticket);
    if (it == s->all.end()) return SPH_EINVAL;
    Req *r = it->second.get();
    if (r->state != DONE) return SPH_EAGAIN;
    out->status = r->status;
    out->n = r->n;
    out->steps_done = r->steps_done;
    out->arrival = r->arrival;
    out->admitted = r->admitted;
    out->completed = r->completed;
    out->t_sim = r->t_sim;
    double *dst[9] = {out->x, out->y, out->z, out->vx, out->vy, out->vz, out->u, out->h, out->rho};
    const std::vector<double> *srcs[9] = {&r->host[0], &r->host[1], &r->host[2], &r->host[3], &r->host[4],
                                          &r->host[5], &r->host[6], &r->host[8], &r->rho};
    for (int k = 0; k < 9; ++k)
        if (dst[k] && (long long)srcs[k]->size() == r->n && r->n > 0)
            memcpy(dst[k], srcs[k]->data(), sizeof(double) * r->n);
    return SPH_OK;
}

int sph_server_destroy(sph_server *s)
{
    if (!s) return SPH_OK;
    for (Req *r : s->active) {
        if (r->ctx) sph_destroy(r->ctx);
    }
    if (s->ev0) cudaEventDestroy(s->ev0);
    if (s->ev1) cudaEventDestroy(s->ev1);
    if (s->staging) cudaFreeHost(s->staging);
    delete s;
    return SPH_OK;
}

}  // extern "C"
