// serve.cu -- a request loop for Fiedler solves (host code around the C-ABI).
//
// Graphs are registered once; requests name a graph.  Worker threads, each
// with its own CUDA stream, take jobs from the pending queue, so the device
// work of different jobs overlaps.  A job is admitted only when its device
// memory fits in the budget (idle resident hierarchies are evicted, least
// recently used first, to make room).  Three kinds of job:
//   warm     the graph's hierarchy is resident: cmg_fiedler only;
//   single   a large graph (n > batch_max_n) without a hierarchy: cmg_setup,
//            cmg_fiedler, and the hierarchy stays resident (keep_resident);
//   batch    small graphs without a hierarchy, when at least min_batch of
//            them are pending: every such request (up to max_batch) joins one
//            cmg_setup_batch / cmg_fiedler_batch, so requests that arrive
//            while others run are admitted together as soon as a worker and
//            memory free up (continuous batching).  With fewer pending, a
//            small graph runs alone like a large one: a batched job gives a
//            graph one group of threads, the single form the whole GPU.
// A request's result does not depend on the job it ran in beyond rounding:
// the batched form computes each graph's hierarchy bit for bit as the single
// form does.
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <list>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "internal.h"

namespace {

uint64_t now_ns() {
    return (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(
               std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

struct Graph {
    int64_t n = 0, nnz = 0;
    bool heavy_tail = false;      // max degree > 8 x mean: coarse levels stay dense
    const int64_t *rp = nullptr;
    const int32_t *col = nullptr;
    const double *w = nullptr;
    cmg_hierarchy_t h = nullptr;  // resident hierarchy (single form)
    size_t h_bytes = 0;           // its device bytes (counted in the budget)
    bool busy = false;            // a job is using or building the hierarchy
    uint64_t last_use = 0;
};

struct Request {
    int64_t ticket = 0;
    int64_t gid = 0;
    double *u_out = nullptr;
    bool custom = false;           // solved with its own options (never batched)
    cmg_solve_options_t so;
    cmg_request_t res;
    bool done = false;
};

struct Job {
    int kind = 0;                  // 0 warm, 1 single, 2 batch
    std::vector<Request *> reqs;
    size_t reserve = 0;            // bytes reserved for the job's duration
};

}  // namespace

struct cmg_server_s {
    cmg_server_config_t cfg;
    cmg_options_t opts;
    int device = 0;
    size_t budget = 0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Graph> graphs;      // deque: references stay valid while graphs are added
    std::deque<Request *> pending;
    std::unordered_map<int64_t, Request *> reqs;
    int64_t next_ticket = 1;
    size_t used = 0;               // reserved for running jobs + resident hierarchies
    size_t peak = 0;
    int running = 0;
    bool stop = false;
    cmg_server_stats_t stats;
    // one stream per worker, owned by the server: resident hierarchies are
    // freed on the stream that built them, also after the workers stopped
    std::vector<cudaStream_t> streams;
    std::vector<std::thread> workers;
};

namespace {

size_t estimate(const cmg_server_s *S, const Graph &g) {
    size_t b = 0;
    cmg_estimate_device_bytes(g.n, g.nnz, S->opts.precision, &b);
    if (g.heavy_tail) {
        // the coarse levels of a heavy-tailed graph keep most of level 0's
        // entries (a 4.19M-vertex Chung-Lu graph: 4x level 0 over all levels),
        // where the general estimate budgets one more copy of level 0: add
        // three more copies of level 0's stored levels
        const double wb = (S->opts.precision == CMG_PRECISION_FP32_SWEEP) ? 16.0 : 12.0;
        b += (size_t)(3.0 * (wb * (double)g.nnz + 16.0 * (double)g.n));
    }
    return b;
}

// Evicts idle resident hierarchies (least recently used first) until `need`
// more bytes fit.  Called with the lock held.
bool make_room(cmg_server_s *S, size_t need) {
    while (S->used + need > S->budget) {
        Graph *victim = nullptr;
        for (auto &g : S->graphs)
            if (g.h && !g.busy && (!victim || g.last_use < victim->last_use)) victim = &g;
        if (!victim) return false;
        cmg_free(victim->h);
        victim->h = nullptr;
        S->used -= victim->h_bytes;
        victim->h_bytes = 0;
        S->stats.evictions++;
    }
    return true;
}

// Picks the next admissible job (lock held); empty job if none.
Job pick_job(cmg_server_s *S) {
    Job job;
    for (auto it = S->pending.begin(); it != S->pending.end(); ++it) {
        Request *r = *it;
        Graph &g = S->graphs[r->gid];
        if (g.busy) continue;
        if (g.h) {
            job.kind = 0;
            job.reqs.push_back(r);
            S->pending.erase(it);
            g.busy = true;
            return job;
        }
        const size_t est = estimate(S, g);
        bool small = g.n <= S->cfg.batch_max_n && S->cfg.max_batch > 1 && !r->custom;
        if (small) {
            // batch only when enough small cold requests wait for it
            int waiting = 0;
            for (auto jt = it; jt != S->pending.end() && waiting < S->cfg.min_batch; ++jt) {
                const Graph &gj = S->graphs[(*jt)->gid];
                if (!gj.busy && !gj.h && gj.n <= S->cfg.batch_max_n && !(*jt)->custom) waiting++;
            }
            small = waiting >= S->cfg.min_batch;
        }
        if (!small) {
            if (!make_room(S, est)) {
                if (S->running == 0 && S->used == 0) {
                    // can never fit: fail the request
                    r->res.status = CMG_ERR_TOO_LARGE;
                    r->res.done_ns = now_ns();
                    r->done = true;
                    S->pending.erase(it);
                    S->cv_done.notify_all();
                    return pick_job(S);
                }
                continue;
            }
            job.kind = 1;
            job.reqs.push_back(r);
            job.reserve = est;
            S->used += est;
            g.busy = true;
            S->pending.erase(it);
            return job;
        }
        // batch: this request and every later small cold request that fits
        std::vector<std::deque<Request *>::iterator> take;
        size_t total = 0;
        for (auto jt = it; jt != S->pending.end() && (int)take.size() < S->cfg.max_batch; ++jt) {
            Graph &gj = S->graphs[(*jt)->gid];
            if (gj.busy || gj.h || gj.n > S->cfg.batch_max_n || (*jt)->custom) continue;
            const size_t e = estimate(S, gj);
            if (!make_room(S, total + e)) break;
            total += e;
            take.push_back(jt);
            gj.busy = true;   // one copy of a graph per job
        }
        if (take.empty()) {
            if (S->running == 0 && S->used == 0) {
                r->res.status = CMG_ERR_TOO_LARGE;
                r->res.done_ns = now_ns();
                r->done = true;
                S->pending.erase(it);
                S->cv_done.notify_all();
                return pick_job(S);
            }
            continue;
        }
        job.kind = 2;
        job.reserve = total;
        S->used += total;
        for (auto jt : take) job.reqs.push_back(*jt);
        // an erase inside a deque invalidates every iterator: rebuild the
        // queue without the taken requests instead
        std::deque<Request *> rest;
        size_t t = 0;
        for (Request *x : S->pending) {
            if (t < job.reqs.size() && x == job.reqs[t]) t++;
            else rest.push_back(x);
        }
        S->pending.swap(rest);
        return job;
    }
    return job;
}

void run_job(cmg_server_s *S, Job &job, cudaStream_t s) {
    const uint64_t t_admit = now_ns();
    for (Request *r : job.reqs) r->res.admit_ns = t_admit;
    if (job.kind == 0 || job.kind == 1) {
        Request *r = job.reqs[0];
        Graph &g = S->graphs[r->gid];
        cmg_status_t st = CMG_OK;
        cmg_hierarchy_t h = g.h;
        if (job.kind == 1) st = cmg_setup(g.n, g.rp, g.col, g.w, CMG_MEM_HOST, &S->opts, s, &h);
        cmg_stats_t stt;
        double lam = 0.0;
        if (st == CMG_OK)
            st = r->custom ? cmg_fiedler_ex(h, &r->so, r->u_out, CMG_MEM_HOST, &lam, &stt, s)
                           : cmg_fiedler(h, r->u_out, CMG_MEM_HOST, &lam, &stt, s);
        r->res.status = st;
        r->res.lambda2 = lam;
        r->res.residual = (st == CMG_OK || st == CMG_WARN_MAXITER) ? stt.residual : 0.0;
        r->res.batch_size = 1;
        r->res.warm = job.kind == 0;
        std::lock_guard<std::mutex> lk(S->mu);
        if (job.kind == 1) {
            S->used -= job.reserve;
            if (h && st >= 0 && S->cfg.keep_resident) {
                size_t hb = 0;
                cmg_hierarchy_device_bytes(h, &hb);
                g.h = h;
                g.h_bytes = hb;
                S->used += hb;
            } else if (h) {
                cmg_free(h);
            }
            S->stats.single_jobs++;
        } else {
            S->stats.warm_jobs++;
        }
        g.busy = false;
        g.last_use = now_ns();
        return;
    }
    // batched job: union CSR on the host
    const int G = (int)job.reqs.size();
    std::vector<int64_t> offs(G + 1, 0), eoffs(G + 1, 0);
    for (int q = 0; q < G; q++) {
        const Graph &g = S->graphs[job.reqs[q]->gid];
        offs[q + 1] = offs[q] + g.n;
        eoffs[q + 1] = eoffs[q] + g.nnz;
    }
    std::vector<int64_t> rp(offs[G] + 1);
    std::vector<int32_t> col(eoffs[G]);
    std::vector<double> w(eoffs[G]);
    for (int q = 0; q < G; q++) {
        const Graph &g = S->graphs[job.reqs[q]->gid];
        for (int64_t i = 0; i < g.n; i++) rp[offs[q] + i] = g.rp[i] + eoffs[q];
        for (int64_t e = 0; e < g.nnz; e++) col[eoffs[q] + e] = g.col[e] + (int32_t)offs[q];
        memcpy(w.data() + eoffs[q], g.w, sizeof(double) * g.nnz);
    }
    rp[offs[G]] = eoffs[G];
    std::vector<double> u(offs[G]), lam(G), res(G);
    std::vector<int32_t> sts(G, 0);
    cmg_batch_t b = nullptr;
    cmg_status_t st = cmg_setup_batch(G, offs.data(), rp.data(), col.data(), w.data(), CMG_MEM_HOST,
                                      &S->opts, s, &b);
    if (st == CMG_OK)
        st = cmg_fiedler_batch(b, u.data(), CMG_MEM_HOST, lam.data(), res.data(), sts.data(), s);
    if (b) cmg_batch_free(b);
    for (int q = 0; q < G; q++) {
        Request *r = job.reqs[q];
        const bool ok = st == CMG_OK || st == CMG_WARN_MAXITER;
        r->res.status = ok ? sts[q] : st;
        r->res.lambda2 = ok ? lam[q] : 0.0;
        r->res.residual = ok ? res[q] : 0.0;
        r->res.batch_size = G;
        r->res.warm = 0;
        if (ok && r->u_out) memcpy(r->u_out, u.data() + offs[q], sizeof(double) * (offs[q + 1] - offs[q]));
    }
    std::lock_guard<std::mutex> lk(S->mu);
    S->used -= job.reserve;
    for (Request *r : job.reqs) {
        Graph &g = S->graphs[r->gid];
        g.busy = false;
        g.last_use = now_ns();
    }
    S->stats.batch_jobs++;
}

// With CMG_DEBUG_SERVE set in the environment, job events go to stderr.
void trace(const char *what, const Job &job, int worker, int status) {
    static const bool on = getenv("CMG_DEBUG_SERVE") != nullptr;
    if (!on) return;
    fprintf(stderr, "cmg-serve %llu w%d %s kind=%d n=%zu first_gid=%lld status=%d\n",
            (unsigned long long)(now_ns() / 1000), worker, what, job.kind, job.reqs.size(),
            job.reqs.empty() ? -1ll : (long long)job.reqs[0]->gid, status);
}

void worker_main(cmg_server_s *S, cudaStream_t s, int worker) {
    cudaSetDevice(S->device);
    for (;;) {
        Job job;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            for (;;) {
                if (S->stop && S->pending.empty()) break;
                job = pick_job(S);
                if (!job.reqs.empty()) break;
                S->cv_work.wait(lk);
            }
            if (job.reqs.empty()) break;
            S->running++;
            S->peak = std::max(S->peak, S->used);
        }
        trace("start", job, worker, 0);
        run_job(S, job, s);
        trace("end", job, worker, job.reqs[0]->res.status);
        {
            std::lock_guard<std::mutex> lk(S->mu);
            S->running--;
            const uint64_t t = now_ns();
            for (Request *r : job.reqs) {
                r->res.done_ns = t;
                r->done = true;
                S->stats.completed++;
            }
        }
        S->cv_done.notify_all();
        S->cv_work.notify_all();
    }
}

}  // namespace

extern "C" cmg_status_t cmg_server_config_default(cmg_server_config_t *cfg) {
    if (!cfg) return CMG_ERR_INVALID_ARG;
    memset(cfg, 0, sizeof(*cfg));
    cfg->workers = 4;
    cfg->max_batch = 256;
    cfg->batch_max_n = 8192;
    cfg->mem_budget = 0;
    cfg->keep_resident = 1;
    cfg->min_batch = 32;
    return CMG_OK;
}

extern "C" cmg_status_t cmg_server_create(const cmg_server_config_t *cfg, const cmg_options_t *opts,
                                          cmg_server_t *out) {
    if (!out) return CMG_ERR_INVALID_ARG;
    *out = nullptr;
    cmg_server_config_t c;
    cmg_server_config_default(&c);
    if (cfg) c = *cfg;
    if (c.workers < 1 || c.workers > 64 || c.max_batch < 1 || c.batch_max_n < 0 || c.min_batch < 0)
        return CMG_ERR_INVALID_ARG;
    if (c.min_batch == 0) c.min_batch = 32;
    cmg_options_t o;
    cmg_options_default(&o);
    if (opts) o = *opts;
    CMG_TRY(cmg::check_options(o));
    if (o.timing) return CMG_ERR_INVALID_ARG;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return CMG_ERR_CUDA;
    size_t budget = c.mem_budget;
    if (budget == 0) {
        size_t fr = 0, tot = 0;
        if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) return CMG_ERR_CUDA;
        budget = (size_t)(0.8 * (double)fr);
    }
    cmg_server_s *S = new cmg_server_s();
    S->cfg = c;
    S->opts = o;
    S->device = dev;
    S->budget = budget;
    memset(&S->stats, 0, sizeof(S->stats));
    for (int k = 0; k < c.workers; k++) {
        cudaStream_t st = nullptr;
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
            for (cudaStream_t t : S->streams) cudaStreamDestroy(t);
            delete S;
            return CMG_ERR_CUDA;
        }
        S->streams.push_back(st);
    }
    // the measured high-water mark starts here (the pool is the library's,
    // shared by every user of the library in this process on this device)
    cmg::pool_used_high(nullptr, 1);
    for (int k = 0; k < c.workers; k++) S->workers.emplace_back(worker_main, S, S->streams[k], k);
    *out = S;
    return CMG_OK;
}

extern "C" cmg_status_t cmg_server_add_graph(cmg_server_t S, int64_t n, const int64_t *row_ptr,
                                             const int32_t *col, const double *w, int64_t *graph_id) {
    if (!S || !row_ptr || !graph_id) return CMG_ERR_INVALID_ARG;
    if (n < 2) return CMG_ERR_TOO_SMALL;
    const int64_t nnz = row_ptr[n];
    if (nnz < 0 || (nnz > 0 && (!col || !w))) return CMG_ERR_INVALID_ARG;
    int64_t maxdeg = 0;
    for (int64_t i = 0; i < n; i++) maxdeg = std::max<int64_t>(maxdeg, row_ptr[i + 1] - row_ptr[i]);
    std::lock_guard<std::mutex> lk(S->mu);
    Graph g;
    g.n = n;
    g.nnz = nnz;
    g.heavy_tail = (double)maxdeg > 8.0 * (double)nnz / (double)n;
    g.rp = row_ptr;
    g.col = col;
    g.w = w;
    S->graphs.push_back(g);
    *graph_id = (int64_t)S->graphs.size() - 1;
    return CMG_OK;
}

static cmg_status_t submit_impl(cmg_server_t S, int64_t graph_id, const cmg_solve_options_t *so,
                                double *u_out, int64_t *ticket) {
    if (!S || !ticket) return CMG_ERR_INVALID_ARG;
    if (so) {
        for (int k = 0; k < 4; k++)
            if (so->reserved[k] != 0) return CMG_ERR_INVALID_ARG;
        if (so->x0 && (so->x0_mem != CMG_MEM_HOST || so->x0_level < 0)) return CMG_ERR_INVALID_ARG;
    }
    Request *r = new Request();
    {
        std::lock_guard<std::mutex> lk(S->mu);
        if (graph_id < 0 || graph_id >= (int64_t)S->graphs.size() || S->stop) {
            delete r;
            return CMG_ERR_INVALID_ARG;
        }
        r->ticket = S->next_ticket++;
        r->gid = graph_id;
        r->u_out = u_out;
        if (so) {
            r->custom = true;
            r->so = *so;
        }
        memset(&r->res, 0, sizeof(r->res));
        r->res.submit_ns = now_ns();
        S->reqs[r->ticket] = r;
        S->pending.push_back(r);
        *ticket = r->ticket;
    }
    S->cv_work.notify_one();
    return CMG_OK;
}

extern "C" cmg_status_t cmg_server_submit(cmg_server_t S, int64_t graph_id, double *u_out,
                                          int64_t *ticket) {
    return submit_impl(S, graph_id, nullptr, u_out, ticket);
}

extern "C" cmg_status_t cmg_server_submit_ex(cmg_server_t S, int64_t graph_id,
                                             const cmg_solve_options_t *so, double *u_out,
                                             int64_t *ticket) {
    if (!so) return CMG_ERR_INVALID_ARG;
    return submit_impl(S, graph_id, so, u_out, ticket);
}

static cmg_status_t wait_impl(cmg_server_t S, int64_t ticket, int64_t timeout_ms, cmg_request_t *out) {
    if (!S) return CMG_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end()) return CMG_ERR_INVALID_ARG;
    Request *r = it->second;
    if (timeout_ms < 0) {
        S->cv_done.wait(lk, [&] { return r->done; });
    } else if (!S->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), [&] { return r->done; })) {
        return CMG_ERR_TIMEOUT;
    }
    if (out) *out = r->res;
    S->reqs.erase(it);
    const cmg_status_t st = (cmg_status_t)r->res.status;
    delete r;
    return st;
}

extern "C" cmg_status_t cmg_server_wait(cmg_server_t S, int64_t ticket, cmg_request_t *out) {
    return wait_impl(S, ticket, -1, out);
}

extern "C" cmg_status_t cmg_server_wait_for(cmg_server_t S, int64_t ticket, int64_t timeout_ms,
                                            cmg_request_t *out) {
    if (timeout_ms < 0) return CMG_ERR_INVALID_ARG;
    return wait_impl(S, ticket, timeout_ms, out);
}

extern "C" cmg_status_t cmg_server_get_stats(cmg_server_t S, cmg_server_stats_t *out) {
    if (!S || !out) return CMG_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    *out = S->stats;
    out->peak_bytes = S->peak;
    out->used_bytes = S->used;
    {
        int prev = 0;
        cudaGetDevice(&prev);
        if (prev != S->device) cudaSetDevice(S->device);
        size_t hi = 0;
        if (cmg::pool_used_high(&hi, 0) == CMG_OK) out->measured_peak_bytes = hi;
        if (prev != S->device) cudaSetDevice(prev);
    }
    out->budget_bytes = S->budget;
    int64_t res = 0;
    for (auto &g : S->graphs) res += g.h ? 1 : 0;
    out->resident = res;
    return CMG_OK;
}

extern "C" cmg_status_t cmg_server_destroy(cmg_server_t S) {
    if (!S) return CMG_ERR_INVALID_ARG;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
    }
    S->cv_work.notify_all();
    for (auto &t : S->workers) t.join();
    for (auto &g : S->graphs)
        if (g.h) cmg_free(g.h);
    for (cudaStream_t t : S->streams) cudaStreamDestroy(t);
    for (auto &kv : S->reqs) delete kv.second;
    delete S;
    return CMG_OK;
}
