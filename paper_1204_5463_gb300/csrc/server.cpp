// Continuous-batching solve server: requests of different lattices, masses,
// gauge fields and right-hand-side counts are admitted while their estimated
// device memory fits the budget and a slot is free; every admitted request
// gets its own CUDA stream and context (gauge field, Krylov bases and
// deflation vectors stay resident for the whole solve), so the SAP sweeps and
// Gram-Schmidt kernels of concurrent requests interleave on the device.
// Allocations are stream-ordered, so a finishing request never synchronises
// the others.
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <list>
#include <map>
#include <mutex>
#include <thread>

#include "internal.h"

namespace {

using clk = std::chrono::steady_clock;

struct Req {
    dw_request r;
    size_t bytes = 0;
    dw_ctx* ctx = nullptr;  // cached context handed to this request, if any
    cudaStream_t st = nullptr;
    int state = 0;  // 0 queued, 1 running, 2 done
    int status = DW_OK;
    bool cancelled = false;
    std::atomic<int> stop{0};  // set by dw_server_cancel while running: the solve stops before its next step
    dw_stats stats{};
    clk::time_point t_submit, t_start, t_done;
};

}  // namespace

// An idle context kept after its request finished: the converted gauge field
// and the Krylov workspace stay on the device for the next request that names
// the same host gauge buffer and lattice.
struct CachedCtx {
    const double* U;
    int dims[4], block[4];
    dw_ctx* ctx;
    cudaStream_t st;
    size_t bytes;
};

struct dw_server {
    size_t budget = 0;
    std::list<CachedCtx> cache;  // most recently used first; counted in in_use
    int max_slots = 1;
    int device = 0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<uint64_t> queue;
    std::map<uint64_t, Req> reqs;
    size_t in_use = 0, peak = 0;
    int running = 0, peak_running = 0;
    long long completed = 0, reused = 0;
    uint64_t next_id = 1;
    bool stop = false;
    std::vector<std::thread> workers;
};

namespace {

// SIZE_MAX for a lattice no context accepts (extents < 2 or too many sites),
// so that such a request exceeds every budget.
size_t request_bytes(const dw_request* q) {
    long long V = 0;
    if (!dwk::lattice_volume(q->lattice.dims, dwk::kMaxSites, &V)) return SIZE_MAX;
    for (int j = 0; j < 4; ++j)
        if (q->lattice.block[j] < 1 || q->lattice.dims[j] % q->lattice.block[j] != 0) return SIZE_MAX;
    const dw_solver_params& P = q->params;
    const int sp = (int)P.sap_prec;
    const bool half = (sp == dwk::P16 || sp == dwk::PB16);
    const long long sb = dwk::spinor_bytes(sp, V);
    const long long zb = (half && P.k > 0) ? dwk::spinor_bytes(dwk::P32, V) : sb;  // Z basis vector
    const long long fb = 192 * V;                                                  // x, b, r
    const long long fv = (P.outer_prec == DW_F32) ? 96 * V : fb;                   // Arnoldi basis vector
    long long gauge = dwk::link_bytes(dwk::P64, V) + 576 * V;  // FP64 links + upload staging
    gauge += dwk::link_bytes(dwk::P32, V);                       // Arnoldi product
    if (half) gauge += dwk::link_bytes(sp, V);
    if (P.outer_prec != DW_F64) gauge += 576 * V;  // double-float links of the residual stencil
    {  // SAP links packed per domain for the sweep's CTA size
        long long B = 1, ndom = 1;
        for (int j = 0; j < 4; ++j) {
            B *= q->lattice.block[j];
            ndom *= q->lattice.block[j] > 0 ? q->lattice.dims[j] / q->lattice.block[j] : 0;
        }
        gauge += dwk::link_bytes(sp, 1) * ((B + 31) / 32 * 32) * ndom;
    }
    long long per_rhs = (long long)(P.m + 1) * fv + (long long)P.m * zb + 3 * fb + sb + 24 * 8 * V;
    if (zb != sb) per_rhs += sb;  // SAP output before widening
    if (fv != fb) per_rhs += fv;  // FP32 copy of the residual
    return (size_t)(gauge + (long long)P.nrhs * per_rhs + (long long)(P.k > 0 ? P.k : 1) * zb + (8LL << 20));
}

bool same_field(const CachedCtx& c, const dw_request& r) {
    if (c.U != r.U) return false;
    for (int j = 0; j < 4; ++j)
        if (c.dims[j] != r.lattice.dims[j] || c.block[j] != r.lattice.block[j]) return false;
    return true;
}

void destroy_cached(CachedCtx& c) {
    dw_destroy(c.ctx);
    cudaStreamDestroy(c.st);
}

void run_request(dw_server* s, uint64_t id) {
    Req* rq;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        rq = &s->reqs[id];
    }
    int rc = DW_OK;
    cudaStream_t st = rq->st;
    dw_ctx* ctx = rq->ctx;
    dw_stats S{};
    if (!ctx) {
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            st = nullptr;
            rc = DW_ECUDA;
        }
        if (rc == DW_OK) rc = dw_create(&rq->r.lattice, st, &ctx);
        if (rc == DW_OK) rc = dw_set_gauge(ctx, rq->r.U, 0);
    } else {
        rc = dw_set_mass(ctx, rq->r.lattice.m0);
    }
    if (rc == DW_OK) {
        dw_solver_params P = rq->r.params;
        P.host_buffers = 1;
        rc = dwk::solve_checked(ctx, rq->r.b, rq->r.x, &P, &S, &rq->stop);
    }
    // a cancelled solve stopped between two steps: its context is consistent
    const bool keep = ctx && (rc == DW_OK || rc == DW_ENOTCONV || rc == DW_ECANCELLED);
    if (!keep) {
        if (ctx) dw_destroy(ctx);
        if (st) cudaStreamDestroy(st);
    }
    std::lock_guard<std::mutex> lock(s->mu);
    rq->status = rc;
    rq->stats = S;
    rq->state = 2;
    rq->t_done = clk::now();
    if (keep) {
        CachedCtx c;
        c.U = rq->r.U;
        for (int j = 0; j < 4; ++j) c.dims[j] = rq->r.lattice.dims[j], c.block[j] = rq->r.lattice.block[j];
        c.ctx = ctx;
        c.st = st;
        c.bytes = rq->bytes;  // stays counted in in_use while cached
        s->cache.push_front(c);
    } else {
        s->in_use -= rq->bytes;
    }
    s->running--;
    s->completed++;
    s->cv_done.notify_all();
    s->cv_work.notify_all();
}

// First queued request that fits (FIFO order, later requests may backfill).
// A request on a cached gauge field takes over that context (its bytes are
// already counted); otherwise idle cached contexts are evicted, least
// recently used first, while that makes room.
bool pick(dw_server* s, uint64_t* id) {
    for (auto it = s->queue.begin(); it != s->queue.end(); ++it) {
        Req& r = s->reqs[*it];
        for (auto c = s->cache.begin(); c != s->cache.end(); ++c)
            if (same_field(*c, r.r)) {
                const size_t need = r.bytes > c->bytes ? r.bytes - c->bytes : 0;
                size_t idle = 0;
                for (auto& o : s->cache)
                    if (&o != &*c) idle += o.bytes;
                if (s->in_use + need > s->budget + idle) break;
                r.ctx = c->ctx;
                r.st = c->st;
                s->reused++;
                s->in_use -= c->bytes;
                s->cache.erase(c);
                while (s->in_use + r.bytes > s->budget && !s->cache.empty()) {
                    s->in_use -= s->cache.back().bytes;
                    destroy_cached(s->cache.back());
                    s->cache.pop_back();
                }
                *id = *it;
                s->queue.erase(it);
                return true;
            }
        size_t idle = 0;
        for (auto& o : s->cache) idle += o.bytes;
        if (s->in_use + r.bytes <= s->budget + idle) {
            while (s->in_use + r.bytes > s->budget && !s->cache.empty()) {
                s->in_use -= s->cache.back().bytes;
                destroy_cached(s->cache.back());
                s->cache.pop_back();
            }
            *id = *it;
            s->queue.erase(it);
            return true;
        }
    }
    return false;
}

void worker(dw_server* s) {
    cudaSetDevice(s->device);
    for (;;) {
        uint64_t id = 0;
        {
            std::unique_lock<std::mutex> lock(s->mu);
            s->cv_work.wait(lock, [&] { return s->stop || (!s->queue.empty() && pick(s, &id)); });
            if (s->stop && id == 0) return;
            Req& r = s->reqs[id];
            r.state = 1;
            r.t_start = clk::now();
            s->in_use += r.bytes;
            if (s->in_use > s->peak) s->peak = s->in_use;
            s->running++;
            if (s->running > s->peak_running) s->peak_running = s->running;
        }
        run_request(s, id);
    }
}

}  // namespace

using namespace dwk;

extern "C" {

size_t dw_request_bytes(const dw_request* r) { return r ? request_bytes(r) : 0; }

int dw_server_create(size_t hbm_budget_bytes, int max_slots, dw_server** out) {
    if (!out || max_slots < 1 || max_slots > 64 || hbm_budget_bytes == 0) return fail(DW_EINVAL, "bad server arguments");
    dw_server* s = new (std::nothrow) dw_server();
    if (!s) return fail(DW_ENOMEM, "host allocation failed");
    s->budget = hbm_budget_bytes;
    s->max_slots = max_slots;
    if (cudaGetDevice(&s->device) != cudaSuccess) {
        cudaGetLastError();
        delete s;
        return fail(DW_ECUDA, "no CUDA device");
    }
    for (int i = 0; i < max_slots; ++i) s->workers.emplace_back(worker, s);
    *out = s;
    return DW_OK;
}

int dw_server_submit(dw_server* s, const dw_request* r, uint64_t* id) {
    if (!s || !r || !id || !r->U || !r->b || !r->x) return fail(DW_EINVAL, "null argument");
    const dw_solver_params& P = r->params;
    if (P.nrhs < 1 || P.nrhs > DW_MAX_RHS || P.m < 1 || P.m > 63 || P.k < 0 || P.k >= P.m || P.k > 16)
        return fail(DW_EINVAL, "bad solver parameters");
    long long V = 0;
    if (!lattice_volume(r->lattice.dims, kMaxSites, &V)) return fail(DW_EINVAL, "bad lattice extents");
    const size_t bytes = request_bytes(r);
    if (bytes == SIZE_MAX) return fail(DW_EINVAL, "bad lattice or domain block");
    if (bytes > s->budget) return fail(DW_ENOMEM, "request larger than the whole memory budget");
    std::lock_guard<std::mutex> lock(s->mu);
    const uint64_t k = s->next_id++;
    Req& q = s->reqs[k];
    q.r = *r;
    q.bytes = bytes;
    q.t_submit = clk::now();
    s->queue.push_back(k);
    *id = k;
    s->cv_work.notify_one();
    return DW_OK;
}

static void fill(const Req& q, int* status, dw_stats* S, double* latency_s) {
    if (status) *status = q.cancelled ? DW_ECANCELLED : q.status;
    if (S) *S = q.stats;
    if (latency_s) *latency_s = std::chrono::duration<double>(q.t_done - q.t_submit).count();
}

int dw_server_poll(dw_server* s, uint64_t id, int* done, int* status, dw_stats* S, double* latency_s) {
    if (!s || !done) return fail(DW_EINVAL, "null argument");
    std::lock_guard<std::mutex> lock(s->mu);
    auto it = s->reqs.find(id);
    if (it == s->reqs.end()) return fail(DW_EINVAL, "unknown request");
    *done = it->second.state == 2;
    if (*done) fill(it->second, status, S, latency_s);
    return DW_OK;
}

int dw_server_wait(dw_server* s, uint64_t id, double timeout_s, int* status, dw_stats* S, double* latency_s) {
    if (!s) return fail(DW_EINVAL, "null server");
    std::unique_lock<std::mutex> lock(s->mu);
    auto it = s->reqs.find(id);
    if (it == s->reqs.end()) return fail(DW_EINVAL, "unknown request");
    const bool ok = s->cv_done.wait_for(lock, std::chrono::duration<double>(timeout_s),
                                        [&] { return s->reqs[id].state == 2; });
    if (!ok) return fail(DW_ETIMEOUT, "request not finished before the timeout");
    fill(s->reqs[id], status, S, latency_s);
    return DW_OK;
}

int dw_server_cancel(dw_server* s, uint64_t id) {
    if (!s) return fail(DW_EINVAL, "null server");
    std::lock_guard<std::mutex> lock(s->mu);
    for (auto it = s->queue.begin(); it != s->queue.end(); ++it)
        if (*it == id) {
            s->queue.erase(it);
            Req& q = s->reqs[id];
            q.cancelled = true;
            q.state = 2;
            q.status = DW_ECANCELLED;
            q.t_done = clk::now();
            s->cv_done.notify_all();
            return DW_OK;
        }
    auto it = s->reqs.find(id);
    if (it != s->reqs.end() && it->second.state == 1) {
        // running: its solve returns DW_ECANCELLED before its next Arnoldi step
        it->second.stop.store(1);
        return DW_OK;
    }
    return fail(DW_EINVAL, "request is finished or unknown");
}

int dw_server_info(dw_server* s, dw_server_status* out) {
    if (!s || !out) return fail(DW_EINVAL, "null argument");
    std::lock_guard<std::mutex> lock(s->mu);
    out->budget_bytes = s->budget;
    out->in_use_bytes = s->in_use;
    out->peak_bytes = s->peak;
    out->running = s->running;
    out->queued = (int)s->queue.size();
    out->completed = s->completed;
    out->reused = s->reused;
    out->peak_running = s->peak_running;
    return DW_OK;
}

void dw_server_destroy(dw_server* s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        for (uint64_t id : s->queue) {
            Req& q = s->reqs[id];
            q.cancelled = true;
            q.state = 2;
            q.status = DW_ECANCELLED;
        }
        s->queue.clear();
        s->stop = true;
    }
    s->cv_work.notify_all();
    for (auto& t : s->workers) t.join();
    for (auto& c : s->cache) destroy_cached(c);
    delete s;
}

}  // extern "C"
