// Autotuner of the coarsening's tuning knobs (lanes per proposing node, the
// tail launch's threshold and block size, the shared-memory sort limit, the
// radix width and the cluster tail's threshold).  None of them changes a result, only the time, so the
// tuner may pick them by measurement: coordinate descent from the caller's
// options, every candidate timed on the caller's own graph (or batch) with
// CUDA events on the caller's stream, the minimum over `reps` runs after one
// untimed run.
#include <cstring>
#include <new>
#include <limits>
#include <vector>

#include "kp_internal.cuh"

using namespace kp;

namespace {

struct Knob {
    int32_t kp_options::*field;
    std::vector<int32_t> values;
};

kp_status time_once(const kp_graph *g, const kp_options *o, const BatchSpec *b, cudaStream_t s, cudaEvent_t e0,
                    cudaEvent_t e1, float *ms) {
    kp_hierarchy *h = nullptr;
    KP_CUDA(cudaEventRecord(e0, s));
    KP_TRY(coarsen_impl(g, o, s, &h, b));
    cudaEventRecord(e1, s);
    const cudaError_t e = cudaEventSynchronize(e1);
    kp_hierarchy_free(h);
    if (e != cudaSuccess) return cuda_error(e, "event");
    KP_CUDA(cudaEventElapsedTime(ms, e0, e1));
    return KP_OK;
}

}  // namespace

static kp_status autotune_impl(const kp_graph *g, int32_t num_graphs, const int32_t *node_offsets,
                               const uint64_t *seeds, const int32_t *stop_sizes, const kp_options *o, int32_t reps,
                               kp_options *best, kp_tune_trial *trials, int32_t max_trials, int32_t *num_trials,
                               kp_stream stream) {
    if (!g || !o || !best) return set_error(KP_ERR_INVALID, "null argument");
    if (reps < 1 || reps > 100 || max_trials < 0 || (max_trials > 0 && !trials))
        return set_error(KP_ERR_INVALID, "bad tuner arguments");
    cudaStream_t s = (cudaStream_t)stream;
    TraceRange trace("kp_autotune");
    BatchSpec b;
    b.num_graphs = num_graphs;
    b.node_offsets = node_offsets;
    b.seeds = seeds;
    b.stop_sizes = stop_sizes;
    const BatchSpec *bp = num_graphs > 0 ? &b : nullptr;
    if (num_graphs < 0) return set_error(KP_ERR_INVALID, "negative num_graphs");
    kp_options cur = *o;
    cur.profile = 0;
    int32_t nt = 0;
    cudaEvent_t e0, e1;
    KP_CUDA(cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return cuda_error(cudaGetLastError(), "event");
    }
    auto measure = [&](const kp_options &c, double *out_ms) -> kp_status {
        float ms = 0.f, bestms = std::numeric_limits<float>::max();
        KP_TRY(time_once(g, &c, bp, s, e0, e1, &ms));   // untimed: allocator, caches
        for (int r = 0; r < reps; r++) {
            KP_TRY(time_once(g, &c, bp, s, e0, e1, &ms));
            if (ms < bestms) bestms = ms;
        }
        *out_ms = bestms;
        if (nt < max_trials) {
            trials[nt].options = c;
            trials[nt].ms = bestms;
        }
        nt++;
        return KP_OK;
    };
    // the input is checked once, not on every candidate
    kp_status st = KP_OK;
    double cur_ms = 0.0;
    if (cur.validate) {
        double dummy;
        st = measure(cur, &dummy);
        cur.validate = 0;
    }
    if (st == KP_OK) st = measure(cur, &cur_ms);
    std::vector<Knob> knobs;
    knobs.push_back({&kp_options::tail_nodes, {-1, 1 << 14, 1 << 16, 1 << 18, 1 << 20, 0x7fffffff}});
    if (cur.matcher == KP_MATCHER_SUITOR) {
        knobs.push_back({&kp_options::suitor_lanes, {1, 2, 4, 8, 32}});
        knobs.push_back({&kp_options::suitor_blocks, {3, 4}});
    }
    knobs.push_back({&kp_options::tail_block_nodes, {512, 1024, 2048, 4096, 8192}});
    knobs.push_back({&kp_options::sort_shared_max, {128, 256, 512, 1024, 2048}});
    knobs.push_back({&kp_options::radix_bits, {6, 7, 8}});
    knobs.push_back({&kp_options::cluster_nodes, {-1, 8192, 32768, 131072}});
    for (const Knob &k : knobs) {
        if (st != KP_OK) break;
        const int32_t start = cur.*(k.field);
        int32_t pick = start;
        for (int32_t v : k.values) {
            if (v == start) continue;
            kp_options c = cur;
            c.*(k.field) = v;
            double ms = 0.0;
            st = measure(c, &ms);
            if (st != KP_OK) break;
            if (ms < cur_ms) {
                cur_ms = ms;
                pick = v;
            }
        }
        cur.*(k.field) = pick;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (num_trials) *num_trials = nt;
    if (st != KP_OK) return st;
    cur.profile = o->profile;
    cur.validate = o->validate;
    *best = cur;
    return KP_OK;
}

extern "C" kp_status kp_autotune(const kp_graph *g, int32_t num_graphs, const int32_t *node_offsets,
                                 const uint64_t *seeds, const int32_t *stop_sizes, const kp_options *o,
                                 int32_t reps, kp_options *best, kp_tune_trial *trials, int32_t max_trials,
                                 int32_t *num_trials, kp_stream stream) {
    try {
        return autotune_impl(g, num_graphs, node_offsets, seeds, stop_sizes, o, reps, best, trials, max_trials,
                             num_trials, stream);
    } catch (const std::bad_alloc &) {
        return set_error(KP_ERR_OOM, "host allocation failed");
    }
}
