// Host runtime internals shared by the library's translation units (not part of the C ABI).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/mbe.h"
#include "mbe_internal.h"

namespace mbe {

// Device-side control block of one search launch (zeroed before each launch).
struct Ctl {
    unsigned long long cursor;
    long long outstanding;
    int32_t n_idle;
    int32_t error;
    int32_t n_published;
    int32_t out_full; // a biclique record did not fit in the caller's buffer
    unsigned long long totals[8];
    unsigned long long used_ids;
    unsigned long long used_bic;
};

struct Workspace {
    char *arena = nullptr;
    int64_t arena_bytes = 0, scratch_bytes = 0;
    char *slots = nullptr;
    int64_t slot_bytes = 0;
    int32_t *slot_state = nullptr;
    int32_t *mark = nullptr;
    int64_t mark_stride = 0;
    int n_warps = 0;
    int threads = 0, blocks = 0;
    Ctl *ctl = nullptr;
    int64_t n_cand_cap = 0, urow_bytes = 0;
    int32_t lbuf_cap = 0; // entries of the wide-node L' list in the scratch split
    bool marks_dirty = false;
    bool budget_limited = false; // fewer warps than requested because of device memory

    void release()
    {
        cudaFree(arena);
        cudaFree(slots);
        cudaFree(slot_state);
        cudaFree(mark);
        cudaFree(ctl);
        *this = Workspace();
    }
};


struct LaunchShape {
    int threads, blocks, warps;
    int layout; // kLayoutRows or kLayoutColumns: which search kernel
};

struct RunInput {
    const int32_t *u_off, *u_adj, *v_off, *v_adj;
    const GraphDesc *d_desc;
    int32_t n_graphs;
    int32_t max_nU;
    const int32_t *task_root, *task_graph;
    const int32_t *task_split = nullptr;
    int64_t n_tasks;
    int64_t nc_max, urow_max, frame_max;
    unsigned long long *per_owner; // [n_owner][4], zeroed here before every launch
    int64_t n_owner;
    int32_t per_mode;
    int32_t layout = kLayoutColumns; // resolved frame layout (kLayoutRows / kLayoutColumns)
    int32_t max_deg = 0;             // largest U degree of the graphs searched
    int32_t prune = 0;               // the pruned variant (single graphs, bitset level sets)
    const int32_t *trep = nullptr;   // its top-level twin classes ([nU])
};


// The current device's shared search workspace.
Workspace &device_workspace();
int set_status(mbe_result *out, int st);
int cuda_status(cudaError_t e);
int64_t round_up(int64_t x, int64_t a);
int key_bits_for(int64_t n);
long long deadline_ms();
unsigned long long *debug_buffer(int n_warps);
// kLayoutRows / kLayoutColumns for a requested layout (0 = auto by the
// largest V degree of the graphs searched).
int resolve_layout(int32_t requested, int32_t max_deg_v);
LaunchShape shape_for(int block_threads, int blocks_per_sm, int layout);
LaunchShape choose_shape(const mbe_options &o, int layout);
cudaError_t launch_layout(const SearchArgs &a, int blocks, const LaunchShape &shape, cudaStream_t s);
int ensure_workspace(Workspace &ws, int64_t nc_max, int64_t urow_max, int64_t frame_max, int32_t max_nU,
                     const LaunchShape &shape, int64_t stack_bytes_req, int stack_factor, int32_t max_deg);
int run_search(Workspace &ws, const RunInput &in, const mbe_options &o, cudaStream_t s, mbe_result *out,
               mbe_biclique_buffer *bic);

// Host-side check of one adjacency form held in HOST memory: off[0] = 0,
// off[n] = nE, offsets non-decreasing, every list strictly increasing with
// ids in [0, n_other). Run before such arrays are copied to the device, so
// that no device kernel ever indexes with an unchecked value.
bool host_csr_ok(const int32_t *off, const int32_t *adj, int32_t n, int32_t n_other, int64_t nE);

} // namespace mbe
