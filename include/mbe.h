/*
 * mbe.h -- C ABI of the GB300 maximal-biclique-enumeration library.
 *
 * Problem (Hsieh et al., "Accelerating Maximal Biclique Enumeration on GPUs",
 * arXiv 2401.05039, Section II-A): G = (U u V, E) is bipartite. A biclique
 * is a pair (R, L), R a subset of U and L a subset of V, with every u in R
 * adjacent to every v in L; it is maximal when no vertex can be added to
 * either side. The library enumerates every maximal biclique with both sides
 * nonempty, by the depth-first search of Section II-B, Algorithm 1 (MBEA:
 * candidate selection, L' construction, maximality check against Q, maximal
 * expansion of R', recursion on P'), run on the GPU as described in
 * Section III (coarse-grained subtree tasks per 1st-level candidate,
 * fine-grained set operations inside them, work stealing between workers).
 *
 * Conventions for every entry point:
 *  - Return value: an mbe_status (0 = MBE_OK). Nothing is thrown; a failing
 *    call leaves caller-owned buffers in an unspecified but valid state.
 *  - Vertex ids are 0-based int32. U is the candidate side (P, Q, R are
 *    subsets of U; L is a subset of V).
 *  - "stream" is a cudaStream_t passed as void* (NULL = the legacy default
 *    stream). Calls enqueue on it and synchronise it before returning,
 *    because their results are read on the host.
 *  - Device memory that the library allocates is owned by the object that
 *    allocated it (a graph or model handle) and released by its destroy
 *    call, except the search workspace: one per device, shared by every
 *    call on that device, grown on demand and released by
 *    mbe_release_workspace() or at process exit. Caller buffers stay owned
 *    by the caller.
 *  - Because of that shared workspace, calls on one device must not overlap
 *    in time: use one host thread per device, one call at a time.
 */
#ifndef MBE_H
#define MBE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    MBE_OK = 0,
    MBE_ERR_INVALID_ARG = 1,   /* NULL where a pointer is required, negative size, bad option */
    MBE_ERR_INVALID_GRAPH = 2, /* unsorted or duplicate adjacency, id out of range, CSR/CSC not transposes */
    MBE_ERR_OOM = 3,           /* device allocation failed */
    MBE_ERR_ARENA_FULL = 4,    /* a search stack outgrew its arena even after the automatic retries */
    MBE_ERR_OUTPUT_FULL = 5,   /* biclique buffer too small: the search still ran to the end, count,
                                  hash, nodes and bytes_alg are exact and the sizes the output needs
                                  are reported in the buffer's n_*_written fields */
    MBE_ERR_TIMEOUT = 6,       /* a device wait exceeded options.watchdog_ms; the kernel stopped cleanly */
    MBE_ERR_CUDA = 7,          /* a CUDA runtime call failed (no device, launch failure, ...) */
    MBE_ERR_UNSUPPORTED = 8,   /* input outside the limits stated at the entry point */
    MBE_ERR_INTERNAL = 9       /* an internal consistency check of the search failed; the launch stopped
                                  before the access it guards */
} mbe_status;

/* Human-readable name of a status code (static storage, never NULL). */
const char *mbe_status_string(int status);

/* ------------------------------------------------------------------ graph */

typedef struct mbe_graph mbe_graph; /* opaque, immutable after create */

/*
 * Build a graph from its two adjacency forms (Section II-A: N(v) for every
 * vertex). u_off[nU+1] / u_adj[nE] is the CSR of U -> V and v_off[nV+1] /
 * v_adj[nE] the CSR of V -> U; every list strictly increasing, the two forms
 * transposes of each other, u_off[0] = v_off[0] = 0, u_off[nU] = v_off[nV]
 * = nE. ptr_kind = 0: the arrays are host memory; 1: device memory of the
 * current device. The arrays are copied; the caller keeps them. Host input
 * is checked on the host before anything is copied (offsets, id ranges,
 * order); then both forms are checked on the device (order, transposes),
 * by kernels that never index with an unchecked value. Violations return
 * MBE_ERR_INVALID_GRAPH.
 * Limits: 0 <= nU, nV; 0 <= nE < 2^31.
 */
int mbe_graph_create(int32_t nU, int32_t nV, int64_t nE, const int32_t *u_off, const int32_t *u_adj,
                     const int32_t *v_off, const int32_t *v_adj, int32_t ptr_kind, void *stream,
                     mbe_graph **out);

/* Release a graph and every device buffer it owns. NULL is accepted. */
int mbe_graph_destroy(mbe_graph *g);

/* Sizes of a graph: any output pointer may be NULL. */
int mbe_graph_info(const mbe_graph *g, int32_t *nU, int32_t *nV, int64_t *nE, int32_t *max_deg_u,
                   int32_t *max_deg_v);

/*
 * Diagnostics (no counterpart in the paper): in a library built with
 * MBE_TRACE=1 (the default build leaves the timers out: they slow the
 * search by 5-13%) and with the environment variable MBE_DEBUG_TRACE set,
 * every search launch keeps a progress record per worker: [0] phase, [1] argument, [2] nodes, [3] depth, [4] donations,
 * [5] steals, [6] elapsed ns, [8..13] ns in root setup, node scans, child
 * builds, frame copies, sorting, tasks; [14] root tasks, [15] stolen tasks;
 * column layout only: [16..21] child builds: sum of |Q'|, sum of |P'|,
 * builds, sum of |L'|, sum of parent row words, sum of parent candidates;
 * [22] ns in the check against Q, [23] ns building child columns, of which
 * [24] forming Q', [25] copying or compressing the parent's columns, [26]
 * transposing P'; [27] child builds that copied the columns uncompressed;
 * both layouts: [28] ns from the launch to the end of the worker's last
 * task, [29] ns the worker spent idle between tasks (before that end), [30]
 * (pruned variants) ns finding the twin classes of new frames.
 * This copies up to max_workers of them (MBE_TRACE_WORDS uint64 each) to
 * `host` and returns how many were copied (0 when none are kept). MBE_DEADLINE_MS bounds any single launch
 * (default 30 minutes); a launch past it stops with MBE_ERR_TIMEOUT.
 */
#define MBE_TRACE_WORDS 32
int mbe_debug_trace(uint64_t *host, int32_t max_workers);

/* Free the current device's search workspace (the next call re-allocates it). */
int mbe_release_workspace(void);

/*
 * Device copy bandwidth (bench support, no counterpart in the paper): copies
 * `bytes` (>= 1 MiB, multiple of 16) between two device buffers `iters`
 * times with 16-byte loads/stores on all SMs and returns the best
 * (read + write bytes) / time in GB/s. With bytes well below the L2 size
 * this measures L2 bandwidth; well above it, HBM bandwidth.
 */
int mbe_copy_bandwidth(int64_t bytes, int32_t iters, void *stream, double *gbps);

/* ------------------------------------------------------------ cost model */
/*
 * The learned schedule (no counterpart in the paper; it feeds Section III-C's
 * task distribution). A small network predicts log(1 + nodes of a root's
 * subtree) from eight per-root features; mbe_enumerate with schedule = 1
 * runs the roots heaviest-predicted first and, without work stealing, splits
 * the heaviest into several tasks. Counts, hashes and nodes never depend on
 * it.
 */
typedef struct mbe_model mbe_model;

/* Parameters: W1[64][8], b1[64], W2[64][64], b2[64], W3[64], b3 (float32 master copy). */
#define MBE_MODEL_PARAMS 4801
#define MBE_N_FEATURES 8

/* Network with Uniform(+-1/sqrt(fan_in)) weights (SplitMix64 stream of seed) and zero biases. */
int mbe_model_create(uint64_t seed, mbe_model **out);
int mbe_model_destroy(mbe_model *m);
/* Copy MBE_MODEL_PARAMS floats in / out (HOST memory); set also clears the optimiser state. */
int mbe_model_set_params(mbe_model *m, const float *host_params);
int mbe_model_get_params(const mbe_model *m, float *host_params);

/*
 * Per-root features of every U vertex (DEVICE outputs, [nU][8]): log1p of
 * degree, |N2(r)|, |P0| (later in (degree, id) order), |Q0| (earlier), core
 * number of G as a general graph, sum and max of the neighbours' degrees,
 * and the fraction of U vertices of larger degree; all zero for isolated
 * vertices. d_raw (may be NULL) receives the integer values before log1p.
 */
int mbe_root_features(const mbe_graph *g, float *d_feat, int32_t *d_raw, void *stream);

/* Forward pass: d_out[i] = prediction for d_feat[i][0..7] (FP16 operands, FP32 accumulation). */
int mbe_model_predict(const mbe_model *m, const float *d_feat, int32_t n, float *d_out, void *stream);

/*
 * Mean squared error of the predictions for n rows against d_target (DEVICE)
 * and its gradient with respect to the parameters (HOST output, 4801 floats).
 */
int mbe_model_loss_grad(mbe_model *m, const float *d_feat, const float *d_target, int32_t n, float *host_grad,
                        float *host_loss, void *stream);

/*
 * Adam training on the GPU: `epochs` passes over n rows (DEVICE features and
 * targets) in shuffled minibatches of `batch`; *final_loss is the mean
 * minibatch loss of the last epoch.
 */
int mbe_model_train(mbe_model *m, const float *d_feat, const float *d_target, int32_t n, int32_t epochs,
                    int32_t batch, float lr, uint64_t seed, void *stream, float *final_loss);

/* ---------------------------------------------------------------- options */

typedef struct {
    int32_t block_threads;    /* threads per block, multiple of 32, 32..1024; 0 = auto */
    int32_t blocks_per_sm;    /* resident blocks per SM for the persistent launch; 0 = auto */
    int32_t bitset_max_words; /* bitset limit, in 64-bit words (1..32; 0 = 32): a level set of at most
                                 64 * bitset_max_words vertices is packed into bitset rows; a wider one
                                 (a root of higher degree, or a node below it) is kept as sorted id
                                 lists, and its counts come from a reverse scan over L' (Sec. III-D) */
    int32_t steal;            /* 1 = busy workers split their shallowest frame for idle ones (Sec. III-C) */
    int32_t schedule;         /* 0 = static execution order (descending degree); 1 = learned: roots by
                                 descending predicted cost, predicted-heavy roots split into up to 32
                                 tasks when steal = 0 (with steal = 1 idle workers split frames
                                 instead, and nothing is pre-split); 2 = learned order without
                                 splitting (needs `model`) */
    int32_t emit;             /* 0 = count + hash only, 1 = also write the bicliques */
    int32_t watchdog_ms;      /* bound on any device wait; 0 = 60000 */
    int32_t root_begin;       /* shard of the execution order: positions [root_begin, root_end) */
    int32_t root_end;         /* -1 = to the end */
    int64_t arena_bytes;      /* per-worker search-stack bytes (exact limit); 0 = sized from the graph,
                                 grown automatically on overflow */
    const void *model;        /* mbe_model* used when schedule = 1 */
    uint64_t *per_root;       /* optional DEVICE array [nU][4]: receives (count, hash, nodes, bytes)
                                 of each top-level candidate's subtree (overwritten by the call) */
    int32_t *exec_order;      /* optional DEVICE array [nU]: explicit execution order of the roots
                                 (any permutation of a subset of U); overrides schedule */
    int32_t n_exec;           /* length of exec_order */
    const void *class_params; /* mbe_enumerate_batch: const mbe_class_params[MBE_N_CLASSES] from
                                 mbe_autotune_batch, or NULL for the defaults */
    int32_t layout;           /* search frame layout (no counterpart in the paper; the result does not
                                 depend on it): 1 = rows (every candidate's row over L; checks stop at
                                 the first superset row), 2 = columns (Q and P as one bitset per vertex
                                 of L: checks are ANDs of the |L'| columns), 0 = auto: columns when some
                                 V vertex has at least 256 neighbours, else rows */
    int32_t min_r;            /* size filter (0 or 1 = none): only the maximal bicliques with |R| >= min_r */
    int32_t min_l;            /* and |L| >= min_l are counted, hashed and written. The search skips what
                                 cannot pass: a call recurses only when |L'| - 1 >= min_l and
                                 |R'| + |P'| >= min_r, a candidate reaching fewer than min_l vertices of
                                 L' does not enter P', and a root of degree below min_l is never popped
                                 (nodes and bytes_alg count what was searched) */
    int32_t prune;            /* 1 = embedded pruning by L - L' removal (iMBE, Sec. II-C): a candidate
                                 whose neighbourhood in L equals that of a candidate popped before it
                                 leaves P at that pop (whether or not that node is maximal) and joins
                                 neither P' nor Q'. Same bicliques, fewer nodes; nodes and bytes_alg
                                 count the pruned search. Both layouts and mbe_enumerate_batch; bitset
                                 level sets only (MBE_ERR_UNSUPPORTED for a graph with a root above the
                                 bitset limit); 0 = off. The first pruned call on a graph computes its
                                 top-level twin classes (kept with the graph) */
} mbe_options;

/* Fill *opt with the defaults (all "auto"). */
int mbe_default_options(mbe_options *opt);

/* ---------------------------------------------------------------- results */

typedef struct {
    uint64_t count;     /* number of maximal bicliques */
    uint64_t hash;      /* sum mod 2^64 over bicliques of SM(sum_{u in R} SM(2u) + sum_{v in L} SM(2v+1)),
                           SM = one SplitMix64 output step (golden-gamma add, then the mix) */
    uint64_t nodes;     /* iterations of Algorithm 1's while loop, candidate order (|N(v) n L|, id) */
    uint64_t bytes_alg; /* algorithmic bytes of the search (roofline numerator) */
    double device_ms;   /* time of the search kernel(s) on the stream, CUDA events */
    double prep_ms;     /* time of ordering / features / model inference before the search */
    int32_t status;     /* same as the return value */
    int32_t n_workers;  /* warps of the persistent launch */
    uint64_t n_donations; /* frames split off for idle workers */
} mbe_result;

/*
 * Caller-owned buffers for the bicliques themselves (emit = 1; the emit
 * step of Algorithm 1), in device memory or in pinned host memory that the
 * device can address (cudaHostAlloc / cudaHostRegister): the kernels write
 * the records directly, so an output larger than device memory can go
 * straight to the host. Biclique b is the record at ids[offsets[b]]:
 * |R|, |L|, then R's ids in ascending order, then L's ids in ascending
 * order (ids of the caller's U and V). Records appear in any order.
 *
 * On return n_ids_written and n_bicliques_written hold the sizes the whole
 * output needs (sum over bicliques of 2 + |R| + |L|, and the number of
 * bicliques), also when they exceed the capacities. If the output does not
 * fit, mbe_enumerate returns MBE_ERR_OUTPUT_FULL after a complete search:
 * count, hash, nodes and bytes_alg are exact, the buffers hold an
 * unspecified subset of the records (do not read them), and a second call
 * with capacities of at least the reported sizes returns every record.
 */
typedef struct {
    int32_t *ids;
    int64_t capacity_ids;
    int64_t *offsets;
    int64_t capacity_bicliques;
    int64_t n_ids_written;       /* out: ids the whole output needs (written when <= capacity_ids) */
    int64_t n_bicliques_written; /* out: bicliques found (records written when they all fit) */
} mbe_biclique_buffer;

/*
 * Enumerate every maximal biclique of g (Algorithm 1 over all of U, run as
 * one persistent launch of warp workers). opts may be NULL (defaults).
 * out receives count, hash, nodes and timings; bicliques may be NULL
 * (count + hash only). The result is independent of every option except
 * root_begin/root_end (which select a shard of roots; shards add up). Any
 * degree is accepted: level sets wider than the bitset limit run on sorted
 * lists (a second variant of the search kernel, launched only for graphs
 * with such roots).
 */
int mbe_enumerate(const mbe_graph *g, const mbe_options *opts, void *stream, mbe_result *out,
                  mbe_biclique_buffer *bicliques);

/*
 * Batch size classes: graph (nU, nV, nE) falls in class
 * 4*(nU >= 128) + 2*(nV >= 512) + (nE >= 0.1*nU*nV). Each class runs as one
 * persistent launch with its own launch parameters.
 */
#define MBE_N_CLASSES 8

typedef struct {
    int32_t block_threads; /* 0 = default */
    int32_t blocks_per_sm; /* 0 = default */
    int32_t steal;         /* frame donation on/off for this class */
    int32_t valid;         /* 0: the class uses the defaults */
    int32_t layout;        /* frame layout as mbe_options.layout (0 = auto) */
    int32_t reserved;
    double tuned_ms;       /* time the autotuner measured for this choice on its sample */
    double default_ms;     /* time of the default launch parameters on the same sample */
} mbe_class_params;

/* Size class of one graph (see MBE_N_CLASSES). */
int mbe_batch_class(int32_t nU, int32_t nV, int64_t nE);

/*
 * Autotuner (no counterpart in the paper): for every size class present in
 * the batch, times a set of launch shapes -- 8, 12 or 16 resident warps per
 * SM in blocks of 64 to 512 threads, work stealing on or off, the row or
 * the column frame layout -- on a sample of the class's (graph, root) tasks
 * (every k-th task of its heavy-first order, about sample_per_class tasks
 * per default worker, or the whole class; halved while one run takes more
 * than 250 ms, down to one task per worker), every shape once and the two
 * fastest again, and writes the fastest into table[class] (valid = 1,
 * tuned_ms = its time on the sample, default_ms = the defaults' time there).
 * Arguments as in mbe_enumerate_batch; table has MBE_N_CLASSES entries.
 */
int mbe_autotune_batch(int32_t n_graphs, const int64_t *edge_off, const int32_t *nU, const int32_t *nV,
                       const int64_t *u_off_start, const int64_t *v_off_start, const int32_t *u_off_cat,
                       const int32_t *u_adj_cat, const int32_t *v_off_cat, const int32_t *v_adj_cat,
                       int32_t sample_per_class, void *stream, mbe_class_params *table);

/*
 * Enumerate many independent graphs in one call. Graph i has nU[i] x nV[i]
 * vertices, its edges are positions [edge_off[i], edge_off[i+1]) of the
 * concatenated u_adj_cat / v_adj_cat (ids local to the graph), and its
 * offset arrays start at u_off_cat[u_off_start[i]] (nU[i]+1 entries,
 * local, starting at 0) and v_off_cat[v_off_start[i]] (nV[i]+1 entries).
 * All arrays are HOST memory. per_graph[i] receives graph i's result;
 * total the sums and the device time of the whole batch. Graphs are binned
 * into size classes; each class is one persistent launch over its (graph,
 * root) tasks with the parameters of opts->class_params (autotuned) or the
 * defaults; the launches of all classes are captured in one CUDA graph and
 * replayed. per_graph[i].device_ms is the device time of the launch that
 * ran graph i (its size class); total->device_ms that of the whole batch.
 * Limits: per graph nU <= 65536 and every degree <= 2048.
 */
int mbe_enumerate_batch(int32_t n_graphs, const int64_t *edge_off, const int32_t *nU, const int32_t *nV,
                        const int64_t *u_off_start, const int64_t *v_off_start, const int32_t *u_off_cat,
                        const int32_t *u_adj_cat, const int32_t *v_off_cat, const int32_t *v_adj_cat,
                        const mbe_options *opts, void *stream, mbe_result *per_graph, mbe_result *total);

/*
 * Enumeration that allocates nothing (the paper has no counterpart; this is
 * a deployment variant of mbe_enumerate). Some callers cannot call
 * cudaMalloc: code inside a framework that owns all device memory through
 * its own pool, where a raw allocation can fail or fragment that pool, and
 * latency-critical loops that must not meet cudaMalloc/cudaFree (cudaFree
 * synchronises the device). Such a caller passes its graph in its own
 * DEVICE arrays (same layout and rules as mbe_graph_create) and receives
 * count, hash, nodes and bytes_alg in the host struct *out (device_ms is -1:
 * the call creates no timing events). The search runs in the column layout.
 *
 * Scratch: every call uses one fixed 64 MiB array compiled into the
 * library (it exists on every GPU that loads the library until the process
 * exits). A graph whose search workspace does not fit in it with at least
 * one block of workers returns MBE_ERR_UNSUPPORTED; a search stack that
 * outgrows its share returns MBE_ERR_ARENA_FULL (there is no retry). The
 * first call on a device looks up the array's device address; make that
 * first call before any stream capture. All calls on a device share the
 * array: calls that overlap on the GPU race, so issue them one at a time.
 * The graph is validated first (MBE_ERR_INVALID_GRAPH), and nothing else
 * reads the arrays before that verdict is back on the host. The call
 * synchronises `stream` before it returns. Its device waits are bounded by
 * fixed limits (60 s for an idle worker, 30 minutes for the search), as the
 * defaults of mbe_enumerate. Returns an mbe_status like every entry point.
 */
int mbe_enumerate_noalloc(int32_t nU, int32_t nV, int64_t nE, const int32_t *u_off, const int32_t *u_adj,
                          const int32_t *v_off, const int32_t *v_adj, void *stream, mbe_result *out);

#ifdef __cplusplus
}
#endif

#endif /* MBE_H */
