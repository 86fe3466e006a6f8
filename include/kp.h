/*
 * kp.h - C ABI of the GB300 coarsening / projection / cut-gain library.
 *
 * The library implements the data-parallel path of the multilevel graph
 * partitioner of "Engineering a Scalable High Quality Graph Partitioner"
 * (Holtgrewe, Sanders, Schulz): edge rating (Section 3.1), matching of
 * locally heaviest edges by handshake rounds (Section 3.3, which under a
 * strict edge order yields the Greedy matching of Section 3.2), contraction
 * level after level (Section 2), projection of a coarse partition back to the
 * input (uncontraction, Section 2) and the cut, block weights, balance bound
 * and per-node FM gains of a partition (Sections 2 and 5.2).
 *
 * Conventions
 *  - All arithmetic is integer: int32 node ids, node weights c and edge
 *    weights omega; int64 sums.  Ratings are exact fractions.
 *  - A graph is a symmetric CSR: row v lists the neighbours of v in strictly
 *    increasing order, each undirected edge {u,v} appears as (u,v) and (v,u)
 *    with the same weight, there are no self loops, omega > 0 and c >= 0.
 *    nnz = 2|E| directed entries.  Section 2 requires omega > 0, c >= 0.
 *  - Integer ranges: sum of c < 2^31, sum of omega over undirected edges
 *    < 2^31.  Then every coarse weight fits in int32.  Entry offsets and
 *    counts (xadj, nnz) have the type kp_eoff below: int32 in the default
 *    build (nnz < 2^31), int64 in the wide build, where nnz is bounded only
 *    by the weight range (omega >= 1, so nnz = 2|E| < 2^32) and by device
 *    memory (Section 5.2's static adjacency array with 64-bit offsets).
 *  - Pointers are DEVICE pointers unless a parameter says "host".
 *    Every call is ordered on the stream passed in (NULL = legacy default
 *    stream); calls that return host scalars synchronise that stream.
 *  - Every call returns a kp_status.  On failure no output is valid and a
 *    message is available from kp_last_error() (thread local).
 *  - Ties between equal ratings are broken by a seeded splitmix64 hash of the
 *    edge's endpoints (higher first), then by the smaller (min id, max id);
 *    the paper leaves tie breaking open.  All results are bit-exact and do not
 *    depend on launch shapes or scheduling.
 */
#ifndef KP_H
#define KP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Entry offsets and entry counts.  The library is built twice from the same
 * sources: libkp (kp_eoff = int32_t) and libkp64 (KP_WIDE_OFFSETS defined,
 * kp_eoff = int64_t).  A caller compiles against this header with the macro
 * of the library it links (the struct layouts that hold a kp_eoff differ);
 * kp_offset_bits() returns the linked library's width. */
#ifdef KP_WIDE_OFFSETS
typedef int64_t kp_eoff;
#define KP_OFFSET_BITS 64
#else
typedef int32_t kp_eoff;
#define KP_OFFSET_BITS 32
#endif

/* A CUDA stream (cudaStream_t / CUstream); NULL is the legacy default stream. */
typedef struct CUstream_st *kp_stream;

typedef enum {
    KP_OK = 0,
    KP_ERR_INVALID = 1,     /* malformed input (see each call) */
    KP_ERR_OVERFLOW = 2,    /* input outside the integer ranges above */
    KP_ERR_OOM = 3,         /* a device or host allocation failed */
    KP_ERR_CUDA = 4,        /* a CUDA runtime call failed */
    KP_ERR_TIMEOUT = 5,     /* a bounded device-side wait gave up */
    KP_ERR_UNSUPPORTED = 6  /* a parameter value this library does not handle */
} kp_status;

/* Edge ratings of Section 3.1, each kept as an exact fraction num/den:
 *   EXPANSION_STAR2  omega^2 / (c(u) c(v))          (the paper's default)
 *   INNER_OUTER      omega / (Out(u) + Out(v) - 2 omega),
 *                    Out(v) = sum of omega over v's edges
 *   WEIGHT           omega
 *   EXPANSION        omega / (c(u) + c(v))
 *   EXPANSION_STAR   omega / (c(u) c(v))
 * A zero denominator means +infinity; two infinities are equal. */
typedef enum {
    KP_RATING_EXPANSION_STAR2 = 0,
    KP_RATING_INNER_OUTER = 1,
    KP_RATING_WEIGHT = 2,
    KP_RATING_EXPANSION = 3,
    KP_RATING_EXPANSION_STAR = 4
} kp_rating;

/* A graph G = (V, E, c, omega) (Section 2) as a symmetric CSR (the static
 * adjacency array of Section 5.2).  Arrays are caller-owned:
 *   xadj[n+1] row offsets, adjncy[nnz] neighbours, ewgt[nnz] omega,
 *   vwgt[n] c. */
typedef struct {
    int32_t n;
    kp_eoff nnz;
    const kp_eoff *xadj;
    const int32_t *adjncy;
    const int32_t *ewgt;
    const int32_t *vwgt;
} kp_graph;

/* How the matching of each level is found.  SUITOR and HANDSHAKE reach the
 * matching of locally heaviest edges (Section 3.3); under the strict edge
 * order both end in the same unique matching, the Greedy matching of
 * Section 3.2:
 *   SUITOR     every node proposes to its best neighbour whose standing offer
 *              it beats (one 128-bit compare-and-swap per proposal); a
 *              displaced proposer proposes again (Manne & Halappanavar's
 *              Suitor scheme).  No rounds, no grid barriers.
 *   HANDSHAKE  rounds: every free node names its best free neighbour, mutual
 *              names are matched, repeated until no edge has two free ends;
 *              one cooperative launch per level, rounds separated by bounded
 *              grid barriers.
 * GPA computes the Global Path Algorithm's matching (Section 3.2, the
 * paper's default matcher): the edges are taken in the strict order into a
 * collection of paths and even cycles (an edge joins when both ends have
 * fewer than two collected edges and it does not close an odd cycle), then
 * every path and cycle gets a maximum weight matching by dynamic programming
 * over the ratings in IEEE double, walked from the path end with the smaller
 * id, a cycle from the smaller end of its closing (lightest) edge, an edge
 * taken only when strictly better.  The result equals the sequential
 * algorithm's; one cooperative launch per level decides the edges that are
 * the best undecided edge at both ends in rounds.  With GPA every level is
 * launched on its own (tail_nodes and cluster_nodes are not used). */
typedef enum {
    KP_MATCHER_SUITOR = 0,
    KP_MATCHER_HANDSHAKE = 1,
    KP_MATCHER_GPA = 2
} kp_matcher;

/* Coarsening options.
 *   rating               a kp_rating
 *   seed                 tie-break hash seed
 *   stop_size            stop before contracting a graph with <= stop_size
 *                        nodes (Section 4: "small enough"; 20*k in the
 *                        measured workloads)
 *   max_levels           at most this many contractions (default 64)
 *   min_shrink_permille  stop after a contraction that kept more than
 *                        (1000 - this)/1000 of the nodes (default 50); a
 *                        contraction that matches nothing is not kept
 *   spin_limit           iteration bound of every device-side wait; a wait
 *                        that runs out sets KP_ERR_TIMEOUT (default 1<<22)
 *   validate             1: check the input graph on the device first
 *   profile              1: time every phase with CUDA events on the stream
 *                        (read with kp_hierarchy_profile)
 *   matcher              a kp_matcher: how the matching of each level is
 *                        found (SUITOR and HANDSHAKE give the same unique
 *                        matching, GPA the Global Path Algorithm's)
 *   arena_bytes          initial size of the device arena that holds the
 *                        coarse levels (0: sized from the input); further
 *                        chunks are added ahead of need when the levels
 *                        shrink slowly, and the arena grows (the level is
 *                        redone) when a level still does not fit
 *   tail_nodes           levels with at most this many nodes and at most 8
 *                        times as many directed edges are contracted
 *                        together in one persistent launch (0: 262144;
 *                        -1: never; 2^31-1: the whole hierarchy)
 * Tuning knobs (0: the built-in choice; results never depend on them, only
 * the time does -- kp_autotune picks them by measurement):
 *   suitor_lanes         lanes per proposing node in the first Suitor pass:
 *                        1, 2, 4, 8 or 32 (0: from the level's mean degree);
 *                        longer rows go to a warp (up to 1024 entries) or
 *                        a block each
 *   tail_block_nodes     nodes per block of the persistent tail launch,
 *                        256..16384 (0: 2048)
 *   sort_shared_max      coarse rows of up to this many gathered entries are
 *                        sorted by one block in shared memory (rows of 129
 *                        to 512 by one warp in registers when the level is
 *                        launched phase by phase), longer ones by the radix
 *                        path (rows above 32768 entries by a thread-block
 *                        cluster each), 128..2048 (0: 256)
 *   radix_bits           bits per pass of the radix path, 4..8 (0: 8)
 *   cluster_nodes        tail levels with at most this many nodes run in one
 *                        thread-block cluster (16 CTAs, or 8) whose phases
 *                        are separated by the hardware cluster barrier
 *                        (0: 8192; -1: never)
 *   suitor_blocks        resident 256-thread blocks per SM the first Suitor
 *                        pass is compiled for: 3 (up to 80 registers per
 *                        thread) or 4 (up to 64, more proposal chains in
 *                        flight) (0: 3) */
typedef struct {
    int32_t rating;
    uint64_t seed;
    int32_t stop_size;
    int32_t max_levels;
    int32_t min_shrink_permille;
    int64_t spin_limit;
    int32_t validate;
    int32_t profile;
    int32_t matcher;
    int64_t arena_bytes;
    int32_t tail_nodes;
    int32_t suitor_lanes;
    int32_t tail_block_nodes;
    int32_t sort_shared_max;
    int32_t radix_bits;
    int32_t cluster_nodes;
    int32_t suitor_blocks;
} kp_options;

/* Fills *o with the defaults: EXPANSION_STAR2, seed 1, stop_size 40,
 * max_levels 64, min_shrink_permille 50, spin_limit 1<<22, validate 1,
 * profile 0, matcher SUITOR, arena_bytes 0, tail_nodes 0, and 0 for every
 * tuning knob. */
void kp_options_default(kp_options *o);

/* A hierarchy of graphs G_0 (the input) .. G_L (the coarsest) with the maps
 * map_l : V(G_l) -> V(G_{l+1}).  Opaque and library-owned. */
typedef struct kp_hierarchy kp_hierarchy;

/* Contraction phase (Sections 2, 3, 4).  Level after level: rate every edge,
 * find the matching of locally heaviest edges by handshake rounds (every free
 * node names its best free neighbour, mutual names are matched, repeated
 * until no edge has two free ends; Section 3.3), and contract it (matched
 * pairs become one node with c = c(u)+c(v); parallel edges are merged with
 * summed omega; Section 2).  Coarse node ids are the ranks of each pair's
 * smaller fine id; coarse rows are sorted.  Stops by the options' rules.
 *   g    input graph (device arrays); BORROWED: it must stay alive and
 *        unchanged until kp_hierarchy_free
 *   o    options (host; NULL = defaults)
 *   out  receives the hierarchy (host pointer to a handle)
 * Blocks until the hierarchy is complete (level sizes are data-dependent).
 * Errors: KP_ERR_INVALID (malformed graph, with o->validate), KP_ERR_OVERFLOW
 * (a weight sum out of range, with o->validate; nnz >= 2^32 in the wide
 * build, always, before any device work), KP_ERR_UNSUPPORTED (unknown rating
 * or matcher), KP_ERR_OOM, KP_ERR_CUDA,
 * KP_ERR_TIMEOUT (a grid-barrier wait, or a proposal chain longer than
 * spin_limit steps, gave up). */
kp_status kp_coarsen(const kp_graph *g, const kp_options *o, kp_stream s, kp_hierarchy **out);

/* Number of levels L+1 including the input (host output). */
kp_status kp_hierarchy_num_levels(const kp_hierarchy *h, int32_t *num_levels);

/* Read-only device view of level l (0 = input).  *map (may be NULL) receives
 * map_l (n_l entries, values < n_{l+1}), or NULL for the coarsest level.
 * The arrays stay valid until kp_hierarchy_free. */
kp_status kp_hierarchy_level(const kp_hierarchy *h, int32_t l, kp_graph *view, const int32_t **map);

/* Statistics of the kp_coarsen that built h (host outputs, any may be NULL):
 * handshake rounds summed over all levels (one per level with SUITOR), and
 * matched pairs summed over all levels. */
kp_status kp_hierarchy_stats(const kp_hierarchy *h, int32_t *total_rounds, int64_t *total_matched);

/* Phases timed when kp_options.profile is set. */
typedef enum {
    KP_PHASE_VALIDATE = 0,   /* input check */
    KP_PHASE_OUT = 1,        /* Out(v) of the input (innerOuter) */
    KP_PHASE_MATCH = 2,      /* rating + handshake rounds, all levels */
    KP_PHASE_RELABEL = 3,    /* coarse ids, map, c', row bounds */
    KP_PHASE_CONTRACT = 4,   /* gather, sort, merge of coarse rows */
    KP_PHASE_CSR = 5,        /* coarse xadj scan and row compaction */
    KP_PHASE_TAIL = 6,       /* all remaining small levels in one launch */
    KP_NUM_PHASES = 7
} kp_phase;

/* Per-level record of a kp_coarsen run.  Times are device milliseconds
 * measured with CUDA events (zeros unless built with profile = 1); the
 * counters are always kept.
 *   n, nnz         size of the level that was contracted
 *   launches       kernels launched for this level
 *   rounds         handshake rounds (1 with SUITOR)
 *   searches       neighbourhood scans (rating passes over a row)
 *   failed_cas     proposals whose compare-and-swap lost a race (SUITOR) */
typedef struct {
    double phase_ms[KP_NUM_PHASES];
    int64_t n;
    int64_t nnz;
    int64_t searches;
    int64_t failed_cas;
    int32_t launches;
    int32_t rounds;
} kp_level_profile;

/* Profile of level l (0 .. num_levels-2: the contraction of level l), or
 * with l = -1 the sums over all levels plus the input check.  Host output. */
kp_status kp_hierarchy_profile(const kp_hierarchy *h, int32_t l, kp_level_profile *out);

/* Releases the hierarchy (synchronises the stream it was built on). */
void kp_hierarchy_free(kp_hierarchy *h);

/* Batches of independent graphs.  The graphs are stored as one disjoint
 * union (a symmetric CSR with no edge between two graphs); graph i owns the
 * nodes [node_offsets[i], node_offsets[i+1]).  Every graph is coarsened
 * exactly as kp_coarsen would coarsen it alone with seed seeds[i] (all of
 * them with o->seed when seeds is NULL): tie-break hashes use graph-local
 * ids, and the stop rule is applied to each graph on its own, so a graph's
 * result does not depend on the rest of the batch.  A graph that stops
 * leaves the union; the union's levels keep the graphs still being
 * contracted, in order.  One call coarsens the whole batch (the levels of
 * all graphs together, small levels in one persistent launch).
 *   node_offsets  device int32[num_graphs+1], from 0 to g->n, non-decreasing;
 *                 BORROWED like the graph
 *   seeds         device uint64[num_graphs] or NULL
 *   stop_sizes    device int32[num_graphs] or NULL: graph i stops at
 *                 stop_sizes[i] nodes instead of o->stop_size
 * The view of graph i at level l (l < its level count) is nodes
 * [off_l[i], off_l[i+1]) of union level l (kp_hierarchy_level_offsets),
 * with neighbour ids off_l[i] higher than its local ids; map_l sends them to
 * union level l+1.
 * Errors: as kp_coarsen, plus KP_ERR_INVALID for bad offsets or (with
 * o->validate) an edge between two graphs. */
kp_status kp_coarsen_batch(const kp_graph *g, int32_t num_graphs, const int32_t *node_offsets,
                           const uint64_t *seeds, const int32_t *stop_sizes, const kp_options *o, kp_stream s,
                           kp_hierarchy **out);

/* Batch sizes (host outputs, either may be NULL): the number of graphs (0
 * for a single-graph hierarchy) and, per graph, its number of levels
 * including the input (host array of num_graphs). */
kp_status kp_hierarchy_batch(const kp_hierarchy *h, int32_t *num_graphs, int32_t *levels);

/* Coarsest size of every graph of a batch (host int32[num_graphs]).
 * Synchronises the stream. */
kp_status kp_hierarchy_batch_coarsest(const kp_hierarchy *h, int32_t *sizes, kp_stream s);

/* Device int32[num_graphs+1]: first node of every graph on union level l. */
kp_status kp_hierarchy_level_offsets(const kp_hierarchy *h, int32_t l, const int32_t **node_offsets);

/* Writes the whole hierarchy (every level's CSR and node weights, every map,
 * a batch's per-level offsets, per-graph level counts and graph ids) to a
 * file, little-endian: u64 magic "KPHIER01", i32 version, i32 levels,
 * i32 num_graphs, i32 0; per level its sizes and row offsets -- version 1
 * (libkp, 32-bit offsets): i32 n, i32 nnz, int32 xadj[n+1]; version 2
 * (libkp64): i32 n, i32 0, i64 nnz, int64 xadj[n+1] -- then adjncy[nnz],
 * ewgt[nnz], vwgt[n], map[n] (not on the coarsest), goff[G+1] (batches);
 * then glevels[G] and gid0[n_0] (batches); everything else int32.
 * Synchronises the hierarchy's stream.  Errors: KP_ERR_INVALID (null
 * arguments, the file cannot be written), KP_ERR_CUDA. */
kp_status kp_hierarchy_save(const kp_hierarchy *h, const char *path);

/* Reads a file written by kp_hierarchy_save (either version: offsets are
 * converted to this library's width, and a level of 2^31 entries or more is
 * refused by the 32-bit library with KP_ERR_OVERFLOW) into device memory on the
 * current device: every level, including the input level, is owned by the
 * returned hierarchy (release with kp_hierarchy_free); projection works as
 * on the original.  The whole file is read and checked on the host first
 * (CSR offsets and neighbour ids in range, maps into the next level, batch
 * offsets and graph ids consistent) so that no kernel indexes with a bad
 * value.  Synchronises s.  Errors: KP_ERR_INVALID (cannot open, not a
 * hierarchy file, truncated, inconsistent contents, trailing bytes),
 * KP_ERR_UNSUPPORTED (another version), KP_ERR_OOM, KP_ERR_CUDA. */
kp_status kp_hierarchy_load(const char *path, kp_stream s, kp_hierarchy **out);

/* Uncontraction of a batch: every graph from its own coarsest level.  The
 * coarse partition of graph i sits at coarse_part[coarse_offsets[i] + j] for
 * its coarsest node j (device arrays; coarse_offsets has num_graphs+1
 * entries).  fine_part: device int32[n_0].  Does not synchronise. */
kp_status kp_project_batch(const kp_hierarchy *h, const int32_t *coarse_part, const int32_t *coarse_offsets,
                           int32_t *fine_part, kp_stream s);

/* Uncontraction (Section 2): the block of every input node is the block of
 * the coarsest node it was contracted into, p_l(v) = p_{l+1}(map_l(v)) from
 * the coarsest level down to level 0.
 *   coarse_part  device int32[n_L] (values are copied through unchecked)
 *   fine_part    device int32[n_0], caller-owned output
 * Does not synchronise. */
kp_status kp_project(const kp_hierarchy *h, const int32_t *coarse_part, int32_t *fine_part, kp_stream s);

/* Results of kp_cut_gain.  The three pointers are caller-owned DEVICE
 * buffers the call fills: block_w[k], gain[n], target[n]. */
typedef struct {
    int64_t cut;        /* sum over blocks i<j of omega(E_ij) (Section 2) */
    int64_t total_c;    /* c(V) */
    int64_t max_c;      /* max_v c(v) */
    int64_t l_max;      /* floor((1+eps) c(V)/k + max_v c(v)), eps read in ppm */
    int64_t imbalance;  /* max(0, max_i c(V_i) - L_max) (Section 5.2) */
    int64_t *block_w;   /* c(V_i) */
    int64_t *gain;      /* decrease of the cut when v moves to target[v] */
    int32_t *target;    /* adjacent block with the largest connection, the
                           smallest id on ties; -1 when v has no neighbour in
                           another block (then gain = -sum of v's omega) */
} kp_cut_gain_out;

/* Cut, block weights, balance bound L_max = (1+eps) c(V)/k + max c(v)
 * (Section 2, rounded down with eps taken in parts per million), imbalance,
 * and per-node FM gains (Section 5.2; with k > 2 a node's gain is for the
 * adjacent block it is best connected to).
 *   part  device int32[n], values in [0,k)
 *   out   host struct; its device buffers are filled, its scalars set
 * Synchronises the stream (the scalars are returned on the host).
 * Errors: KP_ERR_INVALID (k < 1, eps < 0, eps > 1000, a negative size, a
 * null array, or a block id outside [0,k)), KP_ERR_OVERFLOW (nnz >= 2^32 in
 * the 64-bit library), KP_ERR_OOM, KP_ERR_CUDA. */
kp_status kp_cut_gain(const kp_graph *g, const int32_t *part, int32_t k, double eps,
                      kp_cut_gain_out *out, kp_stream s);

/* Largest k accepted by kp_cut_gain_noalloc. */
#define KP_CUT_GAIN_NOALLOC_MAX_K 16384

/* kp_cut_gain without any allocation.  The paper has no counterpart: this
 * entry point serves callers that cannot allocate device memory (or pinned
 * host memory) while they evaluate a partition -- serving loops that must
 * not enter an allocator on their hot path, applications that embed the
 * library under a fixed device-memory budget or behind their own allocator,
 * and code paths where an allocation may block or fail.  It computes exactly
 * what kp_cut_gain computes, with the same arguments, outputs, errors and
 * synchronisation, and calls no cudaMalloc, cudaFree or other allocating
 * routine.
 * Its scratch (the accumulators and one int64 partial weight per block) is a
 * fixed static device array of 64 + 8 * KP_CUT_GAIN_NOALLOC_MAX_K bytes
 * (about 128 KB) that every GPU which loads the library holds until the
 * process exits.  k above KP_CUT_GAIN_NOALLOC_MAX_K returns
 * KP_ERR_UNSUPPORTED without touching the GPU.
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress, with that device current); make that first call
 * before any stream capture.  All calls share the array and each call clears
 * the part that must start at zero, so calls whose GPU work overlaps (other
 * streams or threads) race on it: serialise them.  The scalars are read back
 * through pageable host memory. */
kp_status kp_cut_gain_noalloc(const kp_graph *g, const int32_t *part, int32_t k, double eps,
                              kp_cut_gain_out *out, kp_stream s);

/* Quotient graph (Section 5): one node per block, an edge {a,b} whenever an
 * edge of G joins blocks a and b, weighted by the total edge weight between
 * them (the a-b cut).  Written as a symmetric CSR over the k blocks with
 * ascending neighbour blocks:
 *   q_xadj    device int32[k+1] (always written)
 *   q_adjncy  device int32[capacity], q_ewgt device int64[capacity]
 *   *q_nnz    host: the number of directed quotient entries
 * Synchronises the stream.  Errors: KP_ERR_INVALID (k < 1, null arrays, a
 * block id outside [0,k)), KP_ERR_OVERFLOW (*q_nnz > capacity: the entries are
 * not written; retry with larger buffers; or g->nnz >= 2^32 in the 64-bit
 * library), KP_ERR_UNSUPPORTED (k > 4096: the
 * accumulator is a dense k x k matrix), KP_ERR_OOM, KP_ERR_CUDA. */
kp_status kp_quotient_graph(const kp_graph *g, const int32_t *part, int32_t k, int32_t *q_xadj, int32_t *q_adjncy,
                            int64_t *q_ewgt, int64_t capacity, int64_t *q_nnz, kp_stream s);

/* Bounded breadth-first search from the block boundaries (Section 5: local
 * search is limited to the band it finds; the strategies use depths 1, 5
 * and 20).  dist[v] (device int32[n]) = the length of a shortest path from v
 * to a boundary node of its own block through nodes of that block, when at
 * most `depth`, else -1.  A boundary node has a neighbour in another block.
 * With pair_a, pair_b >= 0 (two different blocks) only those two blocks take
 * part: the boundary is the a-b boundary and nodes of other blocks get -2;
 * (-1, -1) means every block.  Synchronises the stream.  Errors:
 * KP_ERR_INVALID (k < 1, depth < 0, a bad pair, null arrays, a block id
 * outside [0,k)), KP_ERR_OVERFLOW (g->nnz >= 2^32 in the 64-bit library),
 * KP_ERR_OOM, KP_ERR_CUDA. */
kp_status kp_boundary_band(const kp_graph *g, const int32_t *part, int32_t k, int32_t depth, int32_t pair_a,
                           int32_t pair_b, int32_t *dist, kp_stream s);

/* Initial partitioning callback for kp_pipeline_host (Section 4 partitions
 * the coarsest graph on one PE).  Receives the coarsest graph's size and its
 * node weights (host) and writes a block id in [0,k) for every coarsest node
 * into part (host).  Returns 0 on success. */
typedef int (*kp_initial_partition_fn)(int32_t n_coarse, const int32_t *coarse_vwgt, int32_t k,
                                       int32_t *part, void *user);

/* End to end on HOST buffers: copies the input CSR to the device, coarsens,
 * asks `ip` for a partition of the coarsest graph, projects it to the input,
 * evaluates cut/gain and copies part/gain/target/block_w back.
 *   g        host arrays of the input graph (pinned memory copies fastest)
 *   fine_part, gain, target: host outputs of n entries; block_w host [k]
 *   out      host scalars (its pointer fields are ignored)
 *   num_levels (may be NULL) receives the hierarchy's level count
 * Synchronises the stream.  Errors as kp_coarsen and kp_cut_gain, plus
 * KP_ERR_INVALID if ip fails. */
kp_status kp_pipeline_host(const kp_graph *g, const kp_options *o, int32_t k, double eps,
                           kp_initial_partition_fn ip, void *user, int32_t *fine_part,
                           int64_t *gain, int32_t *target, int64_t *block_w,
                           kp_cut_gain_out *out, int32_t *num_levels, kp_stream s);

/* ------------------------------------------------------------------------
 * Request server (serving pattern; the paper has no counterpart).  Clients
 * submit graphs on HOST memory over time; each request runs the whole path
 * (coarsening as kp_coarsen, a seeded initial partition of the coarsest graph,
 * projection as kp_project, evaluation as kp_cut_gain) and its results stay
 * on the device until the client releases the request.
 * Workers: `workers` host threads, each with two non-blocking CUDA streams on
 * the device current at kp_server_create (high priority for groups of small
 * requests, low priority for large ones), so groups run concurrently and the
 * small ones are scheduled first.
 * Admission: first in, first out; the oldest waiting request starts once its
 * estimated device footprint fits into hbm_budget_bytes minus the footprint
 * of running requests and of resident results of older requests (a request
 * runs alone if nothing older is charged, whatever its size; results of
 * younger requests that a small-request worker ran past it do not hold it
 * back, so a client releasing in submission order cannot stall the queue).
 * Workers kept for small requests take the
 * oldest waiting request of at most batch_max_nodes nodes instead, so small
 * requests do not queue behind large ones.  Footprint while running:
 * 148 n + 57 nnz + 2 MB
 * bytes; while resident: 88 n + 40 nnz + 1 MB.  A coarsening that needs more
 * arena than that (graphs that shrink slowly take spare chunks) is charged
 * for every chunk as it is taken, until release, so requests admitted later
 * wait for that memory too.
 * Continuous batching: when a worker takes a request with at most
 * batch_max_nodes nodes, it also takes further waiting requests with at most
 * batch_max_nodes nodes that fit the budget, up to
 * max_batch in all, and runs them as one kp_coarsen_batch call and one batched
 * projection.  A request's results do not depend on the group it ran in.
 * The initial partition of a coarsest graph with c nodes: a permutation of
 * 0..c-1 by Fisher-Yates driven by splitmix64 from the request's seed, dealt
 * round-robin to blocks 0..k-1.
 * ------------------------------------------------------------------------ */
typedef struct kp_server kp_server;

typedef struct kp_server_config {
    int32_t workers;           /* worker threads/streams, 1..64 */
    int32_t max_batch;         /* most requests merged into one group, >= 1 */
    int32_t batch_max_nodes;   /* requests above this size always run alone */
    int32_t small_workers;     /* of the workers, how many take only requests of
                                  at most batch_max_nodes nodes (0..workers-1) */
    int64_t hbm_budget_bytes;  /* device bytes for running + resident requests */
    kp_options options;        /* engine options; seed and stop_size are per request */
} kp_server_config;

/* kp_request_params.flags: the server reads the caller's arrays when the
 * request runs instead of copying them at submit; they must stay valid and
 * unchanged until the request has finished. */
#define KP_REQUEST_BORROW 1

typedef struct kp_request_params {
    int32_t k;          /* blocks, >= 1 */
    int32_t stop_size;  /* coarsening stops at this many nodes (kp_options.stop_size) */
    double eps;         /* imbalance parameter of L_max */
    uint64_t seed;      /* tie-break hash seed and initial-partition seed */
    int32_t flags;      /* 0 or KP_REQUEST_BORROW */
    int32_t pad;
} kp_request_params;

typedef struct kp_request_result {
    kp_status status;
    int32_t num_levels;   /* levels of the request's hierarchy (input included) */
    int32_t coarsest_n;
    int32_t group_size;   /* requests in the group it ran in */
    int32_t launches;     /* kernel launches of that group (all its requests) */
    int32_t pad;
    int64_t group_id;     /* groups are numbered from 1 in start order */
    int64_t cut;          /* as kp_cut_gain_out */
    int64_t total_c;
    int64_t l_max;
    int64_t imbalance;
    double t_submit_us;   /* microseconds since kp_server_create: entry of submit */
    double t_admit_us;    /* taken by a worker */
    double t_done_us;     /* results on the device, scalars on the host */
    int64_t arena_grown_bytes;   /* device bytes the group's coarsening took beyond the
                                    footprint estimate (spare arena chunks); charged to the
                                    budget from the moment they were taken until release */
} kp_request_result;

/* Starts the workers.  Errors: KP_ERR_INVALID (workers outside 1..64,
 * max_batch < 1, budget <= 0, small_workers outside 0..workers-1),
 * KP_ERR_CUDA. */
kp_status kp_server_create(const kp_server_config *cfg, kp_server **out);

/* Copies the host graph into the server (unless p->flags has
 * KP_REQUEST_BORROW) and queues it; *id receives the request id.  Without
 * KP_REQUEST_BORROW the caller's arrays may be reused once this returns.
 * Errors: KP_ERR_INVALID (null pointers, negative sizes, k < 1, eps outside
 * [0,1000], server stopping), KP_ERR_OOM (host copy). */
kp_status kp_server_submit(kp_server *sv, const kp_graph *g, const kp_request_params *p, uint64_t *id);

/* *done = 1 once the request has finished (successfully or not); res (may
 * be NULL) receives its result so far.  Errors: KP_ERR_INVALID (unknown id). */
kp_status kp_server_poll(kp_server *sv, uint64_t id, int32_t *done, kp_request_result *res);

/* Blocks until the request has finished; res (may be NULL) receives its
 * result; returns the request's own status (with its message). */
kp_status kp_server_wait(kp_server *sv, uint64_t id, kp_request_result *res);

/* Copies a finished request's results to HOST buffers (each may be NULL):
 * fine_part int32[n], gain int64[n], target int32[n], coarse_part
 * int32[coarsest_n] (the initial partition).  Errors: KP_ERR_INVALID
 * (unknown, unfinished or released request), the request's own error. */
kp_status kp_server_fetch(kp_server *sv, uint64_t id, int32_t *fine_part, int64_t *gain, int32_t *target,
                          int32_t *coarse_part);

/* Withdraws a request that is still waiting (not yet taken by a worker): it
 * leaves the queue and its id is forgotten.  Errors: KP_ERR_INVALID (unknown
 * id, or the request has started: wait for it and release it instead). */
kp_status kp_server_cancel(kp_server *sv, uint64_t id);

/* Drops a finished request; its device memory returns to the budget when
 * every request of its group has been released.  Does not wait for the GPU.
 * Errors: KP_ERR_INVALID (unknown or unfinished request). */
kp_status kp_server_release(kp_server *sv, uint64_t id);

/* Stops the workers after their running groups, frees every request. */
void kp_server_destroy(kp_server *sv);

/* ------------------------------------------------------------------------
 * Captured plans (the paper has no counterpart).  kp_plan_create records the
 * coarsening of one graph (num_graphs = 0) or of a batch (num_graphs > 0,
 * arguments as kp_coarsen_batch) into a CUDA graph: the state upload, the
 * batch's graph ids, Out (innerOuter), the per-phase launches of the levels
 * that a first, checking coarsening found above the tail threshold
 * (o->tail_nodes; their grids sized by that run) and one persistent
 * cooperative launch for every later level.  With tail_nodes = 2^31-1 the
 * whole hierarchy is that one persistent launch.  kp_plan_run replays the
 * graph on any stream and returns the hierarchy.
 * The input arrays, offsets, seeds and stop sizes are BORROWED for the
 * plan's life and read at every run: their contents may change between runs
 * (the sizes n, nnz and num_graphs may not).  Results equal kp_coarsen[_batch]
 * with the same options.
 * kp_plan_create first coarsens once (this checks the options, offsets and,
 * with o->validate, the input), then allocates the plan's scratch and arena
 * and records the graph; it synchronises s.
 * Errors: those of kp_coarsen[_batch]; KP_ERR_INVALID for n = 0;
 * KP_ERR_CUDA when the device cannot record the launch sequence.
 * ------------------------------------------------------------------------ */
typedef struct kp_plan kp_plan;

kp_status kp_plan_create(const kp_graph *g, int32_t num_graphs, const int32_t *node_offsets, const uint64_t *seeds,
                         const int32_t *stop_sizes, const kp_options *o, kp_stream s, kp_plan **out);

/* Replays the plan on stream s and synchronises it.  *out is a hierarchy
 * whose coarse levels live in the plan's arena: it is valid until the next
 * kp_plan_run or kp_plan_destroy of this plan; release it with
 * kp_hierarchy_free (which then frees only the handle).  If the arena turns
 * out too small, a larger one is taken and the run repeated.  Errors:
 * KP_ERR_TIMEOUT (a bounded wait gave up), KP_ERR_OOM, KP_ERR_CUDA. */
kp_status kp_plan_run(kp_plan *p, kp_stream s, kp_hierarchy **out);

/* Waits for the plan's work and frees it (hierarchies from it become
 * invalid). */
void kp_plan_destroy(kp_plan *p);

/* ------------------------------------------------------------------------
 * Autotuning (the paper has no counterpart).  The tuning knobs of
 * kp_options never change a result, only the time; kp_autotune measures.
 * Coordinate descent from *o over tail_nodes, suitor_lanes and suitor_blocks
 * (Suitor only), tail_block_nodes, sort_shared_max, radix_bits and
 * cluster_nodes, in that order: every
 * candidate coarsens the caller's graph (num_graphs = 0) or batch
 * (num_graphs > 0, arguments as kp_coarsen_batch) once untimed and `reps`
 * times timed by CUDA events on the stream; a knob keeps the value with the
 * least minimum time.  *best receives *o with the chosen knobs.  trials
 * (may be NULL when max_trials is 0) receives up to max_trials candidates
 * with their times in measuring order, *num_trials (may be NULL) how many
 * were measured.  Synchronises the stream many times; allocates like
 * kp_coarsen.  Errors: KP_ERR_INVALID (null pointers, reps outside 1..100,
 * negative num_graphs or max_trials), and those of kp_coarsen[_batch].
 * ------------------------------------------------------------------------ */
typedef struct kp_tune_trial {
    kp_options options;
    double ms;
} kp_tune_trial;

kp_status kp_autotune(const kp_graph *g, int32_t num_graphs, const int32_t *node_offsets, const uint64_t *seeds,
                      const int32_t *stop_sizes, const kp_options *o, int32_t reps, kp_options *best,
                      kp_tune_trial *trials, int32_t max_trials, int32_t *num_trials, kp_stream s);

/* Test hooks (failure injection on the host; no GPU fault is ever made).
 * kp_test_fail_allocation(after): the library's device allocation that
 * follows `after` more successful ones fails with KP_ERR_OOM as if the device
 * were full, then the hook switches itself off (after < 0: off).  Every entry
 * point must then return KP_ERR_OOM with nothing leaked.
 * kp_test_device_bytes_in_use(): bytes currently allocated from the current
 * device's default memory pool (the library's allocations), -1 on error. */
void kp_test_fail_allocation(int64_t after);
int64_t kp_test_device_bytes_in_use(void);

/* Message of the last failed call on this thread ("" if none). */
const char *kp_last_error(void);

/* Library version string. */
const char *kp_version(void);

/* Width in bits of kp_eoff in the linked library: 32 (libkp) or 64
 * (libkp64).  A caller whose KP_OFFSET_BITS differs must not pass it a
 * kp_graph. */
int32_t kp_offset_bits(void);

#ifdef __cplusplus
}
#endif

#endif /* KP_H */
