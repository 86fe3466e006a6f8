// Request server for the serving pattern: coarsen + partition + project +
// cut/gain requests arrive over time; each worker (a host thread with two
// non-blocking CUDA streams: a high-priority one for groups of small requests,
// a low-priority one for large requests) takes the oldest waiting request once its
// estimated device footprint fits the HBM budget, merges further small
// waiting requests into the same batched call, and runs the whole path on
// its stream, so the work of several groups overlaps on the device.  Results
// stay resident on the device until the client releases them; released
// memory lets waiting requests in.  A request's result does not depend on the
// group it ran in: batched coarsening coarsens every graph exactly as alone.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "kp_internal.cuh"

namespace kp {

kp_status project_impl(const kp_hierarchy *h, const int32_t *coarse_part, int32_t *fine_part, cudaStream_t s);
kp_status project_batch_impl(const kp_hierarchy *h, const int32_t *coarse_part, const int32_t *coarse_offsets,
                             int32_t *fine_part, cudaStream_t s);
kp_status batch_coarsest_impl(const kp_hierarchy *h, int32_t *sizes, cudaStream_t s);
kp_status cut_gain_impl(const kp_graph *g, const int32_t *part, int32_t k, double eps, kp_cut_gain_out *out,
                        cudaStream_t s);
kp_status cut_gain_slice(const kp_graph *view, int32_t id_base, const int32_t *part, int32_t k, double eps,
                         kp_cut_gain_out *out, cudaStream_t s);

namespace {

uint64_t mix64(uint64_t x) {
    uint64_t z = x + 0x9e3779b97f4a7c15ull;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

}  // namespace

// The initial partition the server applies to a coarsest graph (the stand-in
// for initial partitioning): a seeded permutation (Fisher-Yates driven by
// splitmix64) dealt round-robin to blocks 0..k-1.
void server_initial_partition(int32_t n, int32_t k, uint64_t seed, int32_t *part) {
    std::vector<int32_t> perm((size_t)n);
    for (int32_t i = 0; i < n; i++) perm[(size_t)i] = i;
    uint64_t state = seed;
    for (int32_t i = n - 1; i > 0; i--) {
        state += 0x9e3779b97f4a7c15ull;
        const int32_t j = (int32_t)(mix64(state) % (uint64_t)(i + 1));
        std::swap(perm[(size_t)i], perm[(size_t)j]);
    }
    for (int32_t i = 0; i < n; i++) part[perm[(size_t)i]] = i % k;
}

}  // namespace kp

using namespace kp;

struct ServerGroup;

struct ServerRequest {
    uint64_t id = 0;
    std::vector<eoff> own_x;    // the server's copy (empty when borrowed): offsets
    std::vector<int32_t> own;   // and the other arrays
    const eoff *xadj = nullptr;
    const int32_t *adjncy = nullptr, *ewgt = nullptr, *vwgt = nullptr;
    int32_t n = 0;
    eoff nnz = 0;
    kp_request_params params{};
    int64_t footprint = 0;  // while running
    int64_t resident = 0;   // after the run, until release
    kp_request_result res{};
    std::string error;
    std::vector<int32_t> coarse_part;
    ServerGroup *grp = nullptr;
    int32_t node_base = 0;   // first node in the group's graph
    int32_t block_base = 0;  // first block weight slot in the group's buffer
    bool done = false;
    bool released = false;
    // calls inside wait or fetch that hold this request without the lock;
    // a request whose id is already forgotten (cancelled, released) is
    // deleted by the last of them
    int32_t users = 0;
    bool forgotten = false;
};

struct ServerGroup {
    std::vector<ServerRequest *> reqs;
    kp_hierarchy *h = nullptr;
    cudaStream_t s = nullptr;
    std::vector<void *> dev;
    int32_t *d_fine = nullptr, *d_target = nullptr;
    int64_t *d_gain = nullptr, *d_bw = nullptr;
    int64_t footprint = 0;  // charged against the budget now
    int64_t resident = 0;
    int64_t grown = 0;      // arena chunks taken beyond the estimate
    uint64_t min_id = 0;    // its oldest request
    bool finished = false;  // run_group has returned (only its resident part is charged)
    int32_t live = 0;
    int64_t id = 0;
    int32_t launches = 0;
};

struct kp_server {
    kp_server_config cfg{};
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<ServerRequest *> queue;
    std::map<uint64_t, ServerRequest *> reqs;
    std::vector<ServerGroup *> finished;   // groups whose results wait for release
    uint64_t next_id = 1;
    int64_t next_group = 1;
    int64_t used = 0;
    bool stopping = false;
    int device = 0;
    std::vector<std::thread> workers;
    std::vector<cudaStream_t> streams;
    std::chrono::steady_clock::time_point t0;
    double now_us() const {
        return std::chrono::duration<double, std::micro>(std::chrono::steady_clock::now() - t0).count();
    }
};

namespace {

// Device bytes of one request: what stays resident until release (the input
// graph, the arena holding the coarse levels and maps, fine partition, gains,
// targets) and the engine's level-0 scratch, freed when coarsening returns.
int64_t resident_bytes(int64_t n, int64_t nnz) {
    return 8 * n + 8 * nnz + 64 * n + 32 * nnz + 16 * n + 2 * ((int64_t)sizeof(eoff) - 4) * n + (1 << 20);
}
int64_t scratch_bytes(int64_t n, int64_t nnz) { return 60 * n + 17 * nnz + (1 << 20); }

// Stream-ordered frees on the group's stream; the caller does not wait.
void free_group(ServerGroup *g) {
    if (g->h) {
        for (void *p : g->h->allocations) dev_free(p, g->s);
        delete g->h;
        g->h = nullptr;
    }
    for (void *p : g->dev) dev_free(p, g->s);
    g->dev.clear();
}

template <class T>
kp_status galloc(ServerGroup *g, T **p, int64_t count) {
    KP_TRY(dev_alloc_n(p, count, g->s));
    g->dev.push_back(*p);
    return KP_OK;
}

kp_status run_group(kp_server *S, ServerGroup *g) {
    TraceRange trace(g->reqs.size() > 1 ? "server batch group" : "server request");
    cudaStream_t s = g->s;
    const size_t G = g->reqs.size();
    kp_options o = S->cfg.options;
    o.stop_size = g->reqs[0]->params.stop_size;   // a batch takes every graph's own
    // the group's graph: one request, or the disjoint union of several
    int64_t n = 0, nnz = 0, kt = 0;
    std::vector<int32_t> off(G + 1, 0);
    std::vector<eoff> eo(G + 1, 0);
    for (size_t i = 0; i < G; i++) {
        ServerRequest *r = g->reqs[i];
        r->node_base = (int32_t)n;
        r->block_base = (int32_t)kt;
        n += r->n;
        nnz += r->nnz;
        kt += r->params.k;
        off[i + 1] = (int32_t)n;
        eo[i + 1] = (eoff)nnz;
    }
    if (n >= (1ll << 31) || nnz >= NNZ_LIMIT) return set_error(KP_ERR_OVERFLOW, "group too large");
    // host arrays of the group's graph: a single request's own, or the union
    std::vector<eoff> hx;
    std::vector<int32_t> ha, hw, hc;
    const eoff *px = g->reqs[0]->xadj;
    const int32_t *pa = g->reqs[0]->adjncy, *pw = g->reqs[0]->ewgt, *pc = g->reqs[0]->vwgt;
    if (G > 1) {
        hx.resize((size_t)n + 1);
        ha.resize((size_t)nnz);
        hw.resize((size_t)nnz);
        hc.resize((size_t)n);
        for (size_t i = 0; i < G; i++) {
            ServerRequest *r = g->reqs[i];
            for (int32_t v = 0; v <= r->n; v++) hx[(size_t)off[i] + v] = r->xadj[(size_t)v] + eo[i];
            for (eoff e = 0; e < r->nnz; e++) ha[(size_t)eo[i] + (size_t)e] = r->adjncy[(size_t)e] + off[i];
            std::memcpy(hw.data() + eo[i], r->ewgt, sizeof(int32_t) * (size_t)r->nnz);
            std::memcpy(hc.data() + off[i], r->vwgt, sizeof(int32_t) * (size_t)r->n);
        }
        px = hx.data();
        pa = ha.data();
        pw = hw.data();
        pc = hc.data();
    }
    eoff *dx;
    int32_t *da, *dw, *dc, *doff, *dstops;
    uint64_t *dseeds;
    KP_TRY(galloc(g, &dx, n + 1));
    KP_TRY(galloc(g, &da, nnz));
    KP_TRY(galloc(g, &dw, nnz));
    KP_TRY(galloc(g, &dc, n));
    KP_TRY(galloc(g, &doff, (int64_t)G + 1));
    KP_TRY(galloc(g, &dseeds, (int64_t)G));
    KP_TRY(galloc(g, &dstops, (int64_t)G));
    KP_TRY(galloc(g, &g->d_fine, n));
    KP_TRY(galloc(g, &g->d_target, n));
    KP_TRY(galloc(g, &g->d_gain, n));
    KP_TRY(galloc(g, &g->d_bw, kt));
    std::vector<uint64_t> seeds(G);
    std::vector<int32_t> stops(G);
    for (size_t i = 0; i < G; i++) {
        seeds[i] = g->reqs[i]->params.seed;
        stops[i] = g->reqs[i]->params.stop_size;
    }
    KP_CUDA(cudaMemcpyAsync(dx, px, sizeof(eoff) * (size_t)(n + 1), cudaMemcpyHostToDevice, s));
    if (nnz > 0) {
        KP_CUDA(cudaMemcpyAsync(da, pa, sizeof(int32_t) * (size_t)nnz, cudaMemcpyHostToDevice, s));
        KP_CUDA(cudaMemcpyAsync(dw, pw, sizeof(int32_t) * (size_t)nnz, cudaMemcpyHostToDevice, s));
    }
    if (n > 0) KP_CUDA(cudaMemcpyAsync(dc, pc, sizeof(int32_t) * (size_t)n, cudaMemcpyHostToDevice, s));
    KP_CUDA(cudaMemcpyAsync(doff, off.data(), sizeof(int32_t) * off.size(), cudaMemcpyHostToDevice, s));
    KP_CUDA(cudaMemcpyAsync(dseeds, seeds.data(), sizeof(uint64_t) * G, cudaMemcpyHostToDevice, s));
    KP_CUDA(cudaMemcpyAsync(dstops, stops.data(), sizeof(int32_t) * G, cudaMemcpyHostToDevice, s));
    kp_graph ug = {(int32_t)n, (eoff)nnz, dx, da, dw, dc};

    // coarsen, partition the coarsest graphs, project
    std::vector<int32_t> csz(G), cpart, coff(G + 1, 0);
    if (G == 1) {
        o.seed = seeds[0];
        KP_TRY(coarsen_impl(&ug, &o, s, &g->h));
        csz[0] = g->h->levels.back().n;
    } else {
        BatchSpec b{(int32_t)G, doff, dseeds, dstops};
        KP_TRY(coarsen_impl(&ug, &o, s, &g->h, &b));
        KP_TRY(batch_coarsest_impl(g->h, csz.data(), s));
    }
    // coarsening, coarsest sizes (batch), projection
    g->launches = g->h->total.launches + (G > 1 ? 1 : 0) + 1;
    for (size_t i = 0; i < G; i++) coff[i + 1] = coff[i] + csz[i];
    cpart.resize((size_t)std::max(coff[G], 1));
    for (size_t i = 0; i < G; i++) {
        ServerRequest *r = g->reqs[i];
        server_initial_partition(csz[i], r->params.k, r->params.seed, cpart.data() + coff[i]);
        r->coarse_part.assign(cpart.begin() + coff[i], cpart.begin() + coff[i + 1]);
        r->res.coarsest_n = csz[i];
        r->res.num_levels = G == 1 ? (int32_t)g->h->levels.size() : g->h->glevels[i];
    }
    int32_t *dcp, *dco;
    KP_TRY(galloc(g, &dcp, std::max(coff[G], 1)));
    KP_TRY(galloc(g, &dco, (int64_t)G + 1));
    if (coff[G] > 0)
        KP_CUDA(cudaMemcpyAsync(dcp, cpart.data(), sizeof(int32_t) * (size_t)coff[G], cudaMemcpyHostToDevice, s));
    KP_CUDA(cudaMemcpyAsync(dco, coff.data(), sizeof(int32_t) * coff.size(), cudaMemcpyHostToDevice, s));
    if (G == 1) KP_TRY(project_impl(g->h, dcp, g->d_fine, s));
    else KP_TRY(project_batch_impl(g->h, dcp, dco, g->d_fine, s));

    // evaluate every request on its own graph
    for (size_t i = 0; i < G; i++) {
        ServerRequest *r = g->reqs[i];
        kp_graph view = {r->n, r->nnz, dx + off[i], da, dw, dc + off[i]};
        kp_cut_gain_out out;
        std::memset(&out, 0, sizeof out);
        out.block_w = g->d_bw + r->block_base;
        out.gain = g->d_gain + off[i];
        out.target = g->d_target + off[i];
        KP_TRY(cut_gain_slice(&view, off[i], g->d_fine + off[i], r->params.k, r->params.eps, &out, s));
        r->res.cut = out.cut;
        r->res.total_c = out.total_c;
        r->res.l_max = out.l_max;
        r->res.imbalance = out.imbalance;
        r->res.group_size = (int32_t)G;
        g->launches += 2;   // evaluation: gains + block maximum
    }
    KP_CUDA(cudaStreamSynchronize(s));
    return KP_OK;
}

struct GrowthCharge {
    kp_server *S;
    ServerGroup *g;
};

void charge_growth(void *ctx, int64_t bytes) {
    GrowthCharge *c = static_cast<GrowthCharge *>(ctx);
    std::lock_guard<std::mutex> lk(c->S->mu);
    c->S->used += bytes;
    c->g->footprint += bytes;
    c->g->resident += bytes;
    c->g->grown += bytes;
}

// Whether r may start: what is charged, less the resident results of
// requests younger than r (a worker for small requests may have run them
// past r; a client that releases in submission order would release them
// only after r, so counting them could keep r waiting for ever), leaves room
// for r's footprint, or nothing older is charged at all.
bool fits(const kp_server *S, const ServerRequest *r) {
    int64_t used = S->used;
    for (const ServerGroup *g : S->finished)
        if (g->min_id > r->id) used -= g->footprint;
    return used == 0 || used + r->footprint <= S->cfg.hbm_budget_bytes;
}

// The request a worker takes next: the oldest one, or for a worker kept for
// small requests the oldest small one; end() when it does not fit yet.
std::deque<ServerRequest *>::iterator next_request(kp_server *S, bool small_only) {
    auto it = S->queue.begin();
    if (small_only)
        while (it != S->queue.end() && (*it)->n > S->cfg.batch_max_nodes) ++it;
    if (it != S->queue.end() && !fits(S, *it)) it = S->queue.end();
    return it;
}

void worker_main(kp_server *S, int wi) {
    cudaSetDevice(S->device);
    const bool small_only = wi < S->cfg.small_workers;
    for (;;) {
        ServerGroup *g = new ServerGroup();
        {
            std::unique_lock<std::mutex> lk(S->mu);
            S->cv_work.wait(lk, [&] { return S->stopping || next_request(S, small_only) != S->queue.end(); });
            if (S->stopping) {
                delete g;
                return;
            }
            auto hit = next_request(S, small_only);
            ServerRequest *head = *hit;
            S->queue.erase(hit);
            g->reqs.push_back(head);
            g->footprint = head->footprint;
            g->resident = head->resident;
            // merge further small waiting requests that fit
            if (head->n <= S->cfg.batch_max_nodes) {
                for (auto it = S->queue.begin(); it != S->queue.end() && (int)g->reqs.size() < S->cfg.max_batch;) {
                    ServerRequest *r = *it;
                    if (r->n <= S->cfg.batch_max_nodes &&
                        S->used + g->footprint + r->footprint <= S->cfg.hbm_budget_bytes) {
                        g->reqs.push_back(r);
                        g->footprint += r->footprint;
                        g->resident += r->resident;
                        it = S->queue.erase(it);
                    } else {
                        ++it;
                    }
                }
            }
            S->used += g->footprint;
            // small groups on the worker's high-priority stream, so their
            // blocks are scheduled ahead of a large request's on the device
            g->s = S->streams[2 * (size_t)wi + (head->n <= S->cfg.batch_max_nodes ? 0 : 1)];
            const double t = S->now_us();
            for (ServerRequest *r : g->reqs) {
                r->res.t_admit_us = t;
                r->grp = g;
            }
            g->live = (int32_t)g->reqs.size();
            g->id = S->next_group++;
            g->min_id = head->id;
            for (ServerRequest *r : g->reqs) g->min_id = std::min(g->min_id, r->id);
        }
        kp_status st;
        // arena chunks the coarsening adds beyond the estimate stay with the
        // group's hierarchy until release: they are charged to the budget
        // as they are taken, so later admissions wait for them
        GrowthCharge charge{S, g};
        arena_observer() = ArenaObserver{&charge_growth, &charge};
        try {
            st = run_group(S, g);
        } catch (const std::bad_alloc &) {
            st = set_error(KP_ERR_OOM, "host allocation failed");
        }
        arena_observer() = ArenaObserver{};
        std::string msg = st == KP_OK ? "" : kp_last_error();
        {
            std::lock_guard<std::mutex> lk(S->mu);
            // the scratch is back in the pool: charge only what stays
            S->used -= g->footprint - g->resident;
            g->footprint = g->resident;
            g->finished = true;
            S->finished.push_back(g);
            const double t = S->now_us();
            for (ServerRequest *r : g->reqs) {
                r->res.arena_grown_bytes = g->grown;
                r->res.group_id = g->id;
                r->res.launches = g->launches;
                r->res.status = st;
                r->error = msg;
                r->res.t_done_us = t;
                r->done = true;
            }
        }
        S->cv_done.notify_all();
        S->cv_work.notify_all();
    }
}

ServerRequest *find(kp_server *S, uint64_t id) {
    auto it = S->reqs.find(id);
    return it == S->reqs.end() ? nullptr : it->second;
}

// Ends a use of r begun under the lock (the lock is held again here).
void drop_user(kp_server *S, ServerRequest *r) {
    if (--r->users == 0 && r->forgotten) {
        delete r;
        return;
    }
    S->cv_done.notify_all();   // a release may be waiting for the readers
}

}  // namespace

extern "C" {

kp_status kp_server_create(const kp_server_config *cfg, kp_server **out) {
    if (!cfg || !out) return set_error(KP_ERR_INVALID, "null argument");
    if (cfg->workers < 1 || cfg->workers > 64 || cfg->max_batch < 1 || cfg->hbm_budget_bytes <= 0 ||
        cfg->small_workers < 0 || cfg->small_workers >= cfg->workers)
        return set_error(KP_ERR_INVALID, "bad server configuration");
    // host allocations fail with KP_ERR_OOM: no exception leaves the C ABI
    kp_server *S = nullptr;
    try {
        S = new kp_server();
        S->streams.reserve(2 * (size_t)cfg->workers);
        S->workers.reserve((size_t)cfg->workers);
    } catch (const std::bad_alloc &) {
        delete S;
        return set_error(KP_ERR_OOM, "host allocation failed");
    }
    S->cfg = *cfg;
    S->t0 = std::chrono::steady_clock::now();
    if (cudaGetDevice(&S->device) != cudaSuccess) {
        delete S;
        return cuda_error(cudaGetLastError(), "cudaGetDevice");
    }
    int prio_low = 0, prio_high = 0;
    if (cudaDeviceGetStreamPriorityRange(&prio_low, &prio_high) != cudaSuccess) {
        cudaGetLastError();
        prio_low = prio_high = 0;
    }
    for (int i = 0; i < 2 * cfg->workers; i++) {   // per worker: high priority (small), low priority (large)
        cudaStream_t s;
        if (cudaStreamCreateWithPriority(&s, cudaStreamNonBlocking, (i & 1) ? prio_low : prio_high) != cudaSuccess) {
            for (cudaStream_t q : S->streams) cudaStreamDestroy(q);
            delete S;
            return cuda_error(cudaGetLastError(), "cudaStreamCreate");
        }
        S->streams.push_back(s);
    }
    try {
        for (int i = 0; i < cfg->workers; i++) S->workers.emplace_back(worker_main, S, i);
    } catch (...) {
        kp_server_destroy(S);
        return set_error(KP_ERR_INVALID, "cannot start worker threads");
    }
    *out = S;
    return KP_OK;
}

kp_status kp_server_submit(kp_server *S, const kp_graph *g, const kp_request_params *p, uint64_t *id) {
    if (!S || !g || !p || !id) return set_error(KP_ERR_INVALID, "null argument");
    if (g->n < 0 || g->nnz < 0 || (g->n > 0 && (!g->xadj || !g->vwgt)) || (g->nnz > 0 && (!g->adjncy || !g->ewgt)))
        return set_error(KP_ERR_INVALID, "bad graph");
    if ((int64_t)g->nnz >= NNZ_LIMIT) return set_error(KP_ERR_OVERFLOW, "nnz >= 2^32: the edge weights sum to 2^31 or more");
    if (p->k < 1 || !(p->eps >= 0.0) || p->eps > 1000.0 || (p->flags & ~KP_REQUEST_BORROW))
        return set_error(KP_ERR_INVALID, "bad request parameters");
    const double t_in = S->now_us();   // latency includes the host copy
    ServerRequest *r = new (std::nothrow) ServerRequest();
    if (!r) return set_error(KP_ERR_OOM, "host allocation failed");
    r->n = g->n;
    r->nnz = g->nnz;
    if (p->flags & KP_REQUEST_BORROW) {
        r->xadj = g->xadj;
        r->adjncy = g->adjncy;
        r->ewgt = g->ewgt;
        r->vwgt = g->vwgt;
    } else {
        const size_t n1 = (size_t)g->n + 1, m = (size_t)g->nnz, n = (size_t)g->n;
        try {
            r->own_x.resize(n1);
            r->own.resize(2 * m + n);
        } catch (...) {
            delete r;
            return set_error(KP_ERR_OOM, "host copy of the request");
        }
        std::memcpy(r->own_x.data(), g->xadj, sizeof(eoff) * n1);
        int32_t *b = r->own.data();
        if (m) std::memcpy(b, g->adjncy, 4 * m);
        if (m) std::memcpy(b + m, g->ewgt, 4 * m);
        if (n) std::memcpy(b + 2 * m, g->vwgt, 4 * n);
        r->xadj = r->own_x.data();
        r->adjncy = b;
        r->ewgt = b + m;
        r->vwgt = b + 2 * m;
    }
    r->params = *p;
    r->resident = resident_bytes(g->n, g->nnz);
    r->footprint = r->resident + scratch_bytes(g->n, g->nnz);
    {
        std::lock_guard<std::mutex> lk(S->mu);
        if (S->stopping) {
            delete r;
            return set_error(KP_ERR_INVALID, "server is stopping");
        }
        r->id = S->next_id++;
        r->res.t_submit_us = t_in;
        try {
            S->reqs[r->id] = r;
        } catch (const std::bad_alloc &) {
            delete r;
            return set_error(KP_ERR_OOM, "host allocation failed");
        }
        try {
            S->queue.push_back(r);
        } catch (const std::bad_alloc &) {
            S->reqs.erase(r->id);
            delete r;
            return set_error(KP_ERR_OOM, "host allocation failed");
        }
        *id = r->id;
    }
    S->cv_work.notify_all();
    return KP_OK;
}

kp_status kp_server_poll(kp_server *S, uint64_t id, int32_t *done, kp_request_result *res) {
    if (!S || !done) return set_error(KP_ERR_INVALID, "null argument");
    std::lock_guard<std::mutex> lk(S->mu);
    ServerRequest *r = find(S, id);
    if (!r) return set_error(KP_ERR_INVALID, "unknown request");
    *done = r->done ? 1 : 0;
    if (res) *res = r->res;
    return KP_OK;
}

kp_status kp_server_wait(kp_server *S, uint64_t id, kp_request_result *res) {
    if (!S) return set_error(KP_ERR_INVALID, "null argument");
    std::unique_lock<std::mutex> lk(S->mu);
    ServerRequest *r = find(S, id);
    if (!r) return set_error(KP_ERR_INVALID, "unknown request");
    r->users++;   // a cancel meanwhile finishes r instead of deleting it
    S->cv_done.wait(lk, [&] { return r->done; });
    if (res) *res = r->res;
    const kp_status st = r->res.status;
    const std::string msg = r->error;
    drop_user(S, r);
    if (st != KP_OK) return set_error(st, msg);
    return KP_OK;
}

kp_status kp_server_fetch(kp_server *S, uint64_t id, int32_t *fine_part, int64_t *gain, int32_t *target,
                          int32_t *coarse_part) {
    if (!S) return set_error(KP_ERR_INVALID, "null argument");
    ServerRequest *r;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        r = find(S, id);
        if (!r) return set_error(KP_ERR_INVALID, "unknown request");
        if (!r->done || r->released) return set_error(KP_ERR_INVALID, "request not finished or released");
        if (r->res.status != KP_OK) return set_error(r->res.status, r->error);
        r->users++;   // a release meanwhile waits until the copies are done
    }
    ServerGroup *g = r->grp;
    const size_t n = (size_t)r->n;
    cudaError_t e = cudaSuccess;
    if (fine_part && n) e = cudaMemcpy(fine_part, g->d_fine + r->node_base, 4 * n, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && gain && n) e = cudaMemcpy(gain, g->d_gain + r->node_base, 8 * n, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && target && n)
        e = cudaMemcpy(target, g->d_target + r->node_base, 4 * n, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && coarse_part) std::memcpy(coarse_part, r->coarse_part.data(), 4 * r->coarse_part.size());
    {
        std::lock_guard<std::mutex> lk(S->mu);
        drop_user(S, r);
    }
    if (e != cudaSuccess) return cuda_error(e, "kp_server_fetch copy");
    return KP_OK;
}

kp_status kp_server_cancel(kp_server *S, uint64_t id) {
    if (!S) return set_error(KP_ERR_INVALID, "null argument");
    {
        std::lock_guard<std::mutex> lk(S->mu);
        auto q = std::find_if(S->queue.begin(), S->queue.end(), [&](ServerRequest *r) { return r->id == id; });
        if (q == S->queue.end()) return set_error(KP_ERR_INVALID, "unknown or already started request");
        ServerRequest *r = *q;
        S->queue.erase(q);
        S->reqs.erase(id);
        // finished as cancelled: threads waiting on it return an error and
        // the last of them deletes it
        r->done = true;
        r->res.status = KP_ERR_INVALID;
        r->error = "request cancelled";
        r->forgotten = true;
        if (r->users == 0) delete r;
    }
    S->cv_done.notify_all();
    S->cv_work.notify_all();   // the next request may fit now that this one is gone
    return KP_OK;
}

kp_status kp_server_release(kp_server *S, uint64_t id) {
    if (!S) return set_error(KP_ERR_INVALID, "null argument");
    ServerGroup *to_free = nullptr;
    {
        std::unique_lock<std::mutex> lk(S->mu);
        ServerRequest *r = find(S, id);
        if (!r) return set_error(KP_ERR_INVALID, "unknown request");
        if (!r->done) return set_error(KP_ERR_INVALID, "request not finished");
        if (r->released) return set_error(KP_ERR_INVALID, "request already being released");
        // claimed: no fetch starts from here on; the fetches still copying
        // from the group's buffers finish first (other users of r are
        // waiters that have seen it done and leave at once)
        r->released = true;
        r->users++;
        S->cv_done.wait(lk, [&] { return r->users == 1; });
        ServerGroup *g = r->grp;
        if (g && --g->live == 0) {
            S->used -= g->footprint;
            S->finished.erase(std::remove(S->finished.begin(), S->finished.end(), g), S->finished.end());
            to_free = g;
        }
        S->reqs.erase(id);
        r->forgotten = true;
        drop_user(S, r);   // deletes r
    }
    if (to_free) {
        free_group(to_free);
        delete to_free;
    }
    S->cv_work.notify_all();
    return KP_OK;
}

void kp_server_destroy(kp_server *S) {
    if (!S) return;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stopping = true;
    }
    S->cv_work.notify_all();
    for (auto &t : S->workers) t.join();
    std::vector<ServerGroup *> groups;
    for (auto &kv : S->reqs) {
        ServerRequest *r = kv.second;
        if (r->grp && std::find(groups.begin(), groups.end(), r->grp) == groups.end()) groups.push_back(r->grp);
        delete r;
    }
    for (ServerGroup *g : groups) {
        free_group(g);
        delete g;
    }
    for (cudaStream_t s : S->streams) cudaStreamDestroy(s);
    delete S;
}

}  // extern "C"
