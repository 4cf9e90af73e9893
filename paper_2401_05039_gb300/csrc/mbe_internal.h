// Internal declarations shared by the library's translation units (not part of the C ABI).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/mbe.h"

namespace mbe {

// One graph of a launch. For a single graph there is one descriptor with
// zero bases; for a batch, graph g's arrays start at these bases of the
// concatenated arrays.
struct GraphDesc {
    int64_t u_off_base;  // index of the graph's u_off[0] in the concatenated u_off
    int64_t v_off_base;  // index of its v_off[0]
    int64_t edge_base;   // index of its first edge in u_adj / v_adj
    int32_t nU, nV;
};

// Everything the persistent search kernel reads. All pointers are device pointers.
struct SearchArgs {
    const int32_t *u_off, *u_adj, *v_off, *v_adj; // concatenated for a batch
    const GraphDesc *graphs;
    int32_t n_graphs;
    int32_t key_shift;      // bits for a vertex id in the (count, id) sort key
    const int32_t *task_root;  // [n_tasks] root (graph-local id) in execution order
    const int32_t *task_graph; // [n_tasks] graph of the task, NULL when n_graphs == 1
    const int32_t *task_split; // [n_tasks] (parts << 16 | part) of a pre-split root, 0 = whole; or NULL
    int64_t n_tasks;

    // per-worker workspace
    char *arena;          // n_warps * arena_bytes
    int64_t arena_bytes;  // per warp: [stack ... | scratch]
    int64_t scratch_bytes;
    int64_t stack_bytes;  // usable stack (<= arena_bytes - scratch_bytes)
    char *slots;          // n_warps * slot_bytes, donation slots
    int64_t slot_bytes;
    int32_t *slot_state;  // [n_warps]
    int32_t *mark;        // n_warps * mark_stride, all -1 between uses
    int64_t mark_stride;
    int64_t n_cand_cap;   // largest candidate count of any root (bounds every frame)
    int64_t urow_bytes;   // largest root-universe row storage

    // control
    unsigned long long *cursor;   // next task
    int32_t *n_idle;              // workers looking for work
    long long *outstanding;       // tasks claimed or published and not finished
    int32_t *error;               // first error status, 0 = none
    long long watchdog_ns;        // longest idle wait of a worker
    long long deadline_ns;        // longest run of the whole launch, measured by every worker
    int32_t *n_published;         // donation slots currently FULL
    unsigned long long *debug;    // optional [n_warps][8] progress records
    int32_t steal;
    int32_t n_warps;
    int32_t max_words;    // bitset limit: level sets of more than 64 * max_words vertices use sorted lists
    int32_t lbuf_cap;     // entries of the scratch list for a wide node's L' (the largest U degree)
    int32_t lists;        // 1: launch the extended variant (some root exceeds the bitset limit, or a size
                          // filter is set)
    int32_t min_r, min_l; // size filter: only bicliques with |R| >= min_r and |L| >= min_l (1, 1 = all)
    int32_t prune;        // 1: launch the pruned variant (iMBE's L - L' removal, Section II-C)
    const int32_t *trep;  // pruned variant: per graph, at its u_off base, [nU] smallest local U id with the
                          // same neighbourhood (itself if none)

    // outputs
    unsigned long long *totals;   // [8]: count, hash, nodes, bytes, donations, steals, -, -
    unsigned long long *per_task_owner; // [n_owner][4] per root (single) or per graph (batch), or NULL
    int32_t per_root_mode;        // 1: index per_task_owner by root id, 2: by graph id

    // biclique output (emit)
    int32_t emit;
    int32_t *out_ids;
    int64_t cap_ids;
    int64_t *out_offsets;
    int64_t cap_bic;
    unsigned long long *used_ids; // ids needed so far (keeps counting past cap_ids)
    unsigned long long *used_bic; // records needed so far (keeps counting past cap_bic)
    int32_t *out_full;            // set to 1 when a record did not fit (the search goes on)
};

// Status codes the kernel writes into *error.
enum : int32_t {
    kErrArena = MBE_ERR_ARENA_FULL,
    kErrTimeout = MBE_ERR_TIMEOUT,
    kErrUnsupported = MBE_ERR_UNSUPPORTED,
    kErrInternal = MBE_ERR_INTERNAL,
};

// Bytes of a worker's scratch region (top of its arena) for lists of
// `ncap` candidates, root-universe rows of `urow_bytes` and a list of `dmax`
// ids (L' of a node wider than the bitset limit); the kernels lay the region
// out in the same order: five int32 lists, two uint64 key lists, then
// (column layout only) the L' position list (2048 entries), the Q' mask, its
// word offsets and its compress masks (one entry per 64 candidates), then
// the universe rows, and after them the wide L' list.
inline int64_t scratch_layout_bytes(int64_t ncap, int64_t urow_bytes, int64_t dmax)
{
    auto p16 = [](int64_t b) { return (b + 15) / 16 * 16; };
    const int64_t qw = (ncap + 63) / 64 + 1;
    const int64_t b = 5 * p16(4 * ncap) + 2 * p16(8 * ncap) + p16(4 * 2048) + p16(8 * qw) + p16(4 * qw) +
                      p16(56 * qw) + urow_bytes + p16(4 * dmax) + 256;
    return (b + 255) / 256 * 256;
}

// Bytes of a search frame's header.
constexpr int64_t kFrameHdrBytes = 80;

// Widest level set held as bitsets (64-bit words per row); wider level
// sets are held as sorted id lists.
constexpr int kMaxBitsetWords = 32;

// Upper bound of the largest frame below a root of degree d with at most nc
// candidates. A bitset frame (level set of w <= 64 * kMaxBitsetWords
// vertices): header, L ids, X columns (w x ceil(nc/64) words), P ids, P
// rows (32-row tiles of ceil(w/64) words), the pruned variant's twin
// sections (two int32 per P entry), R ids. A list frame (a wider level
// set): header, L ids, Q ids, P ids, R ids.
#if defined(__CUDACC__)
__host__ __device__
#endif
inline int64_t level1_frame_bound(int64_t d, int64_t nc)
{
    auto p16 = [](int64_t b) { return (b + 15) / 16 * 16; };
    const int64_t w = d < 64 * kMaxBitsetWords ? d : 64 * kMaxBitsetWords;
    const int64_t W = (w + 63) / 64;
    const int64_t bits = kFrameHdrBytes + p16(4 * w) + p16(8 * w * ((nc + 63) / 64)) + p16(4 * nc) +
                         256 * W * ((nc + 31) / 32) + 2 * p16(4 * nc) + p16(4 * (nc + 1));
    const int64_t list = kFrameHdrBytes + p16(4 * d) + 2 * p16(4 * nc) + p16(4 * (nc + 1));
    return d > w && list > bits ? list : bits;
}

// Upper bound of the root-universe rows of a root of degree d with at most
// nc candidates (bitset rows of at most kMaxBitsetWords words).
#if defined(__CUDACC__)
__host__ __device__
#endif
inline int64_t universe_rows_bound(int64_t d, int64_t nc)
{
    const int64_t W = (d + 63) / 64;
    return 256 * (W < kMaxBitsetWords ? W : kMaxBitsetWords) * ((nc + 31) / 32);
}

// Launch the persistent search kernel on stream (grid = blocks, block = threads).
cudaError_t launch_search(const SearchArgs &a, int blocks, int threads, cudaStream_t stream);

// Bytes of per-warp shared memory the search kernel uses.
int search_smem_per_warp();

// 1 when the search kernels were built with their progress records and
// phase timers (MBE_TRACE = 1), else 0.
int search_trace_compiled();

// The column-layout kernel's variant with the sorted-list path
// (mbe_search_lists.cu); launch_search dispatches to it when args.lists.
cudaError_t launch_search_lists(const SearchArgs &a, int blocks, int threads, cudaStream_t stream);
int search_lists_fit_shape(int threads, int blocks_per_sm_req);

// The column-layout kernel's pruned variant (mbe_search_prune.cu), bitset
// level sets only; launch_search dispatches to it when args.prune.
cudaError_t launch_search_prune(const SearchArgs &a, int blocks, int threads, cudaStream_t stream);
int search_prune_fit_shape(int threads, int blocks_per_sm_req);

// Resident blocks per SM for a block of `threads` threads, at most
// blocks_per_sm_req; a negative value -t means `threads` exceeds the
// kernel's limit and t is the largest allowed block size.
int search_fit_shape(int threads, int blocks_per_sm_req);

// The same three for the row-layout search kernel (mbe_search_rows.cu),
// its list-path variant (mbe_search_rows_lists.cu) and its pruned variant
// (mbe_search_rows_prune.cu).
cudaError_t launch_search_rows(const SearchArgs &a, int blocks, int threads, cudaStream_t stream);
int search_rows_smem_per_warp();
int search_rows_fit_shape(int threads, int blocks_per_sm_req);
cudaError_t launch_search_rows_lists(const SearchArgs &a, int blocks, int threads, cudaStream_t stream);
int search_rows_lists_fit_shape(int threads, int blocks_per_sm_req);
cudaError_t launch_search_rows_prune(const SearchArgs &a, int blocks, int threads, cudaStream_t stream);
int search_rows_prune_fit_shape(int threads, int blocks_per_sm_req);

// Frame layouts of the two search kernels.
enum : int32_t { kLayoutAuto = 0, kLayoutRows = 1, kLayoutColumns = 2 };

// Automatic choice: the column layout when some V vertex has at least this
// many neighbours (Q sets stay long at depth), else the row layout.
constexpr int32_t kColumnsMinDegV = 256;

} // namespace mbe
