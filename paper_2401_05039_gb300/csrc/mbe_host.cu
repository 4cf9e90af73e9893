// Host runtime behind the C ABI (include/mbe.h): graph handles, workspace
// sizing, the persistent search launch, result read-back.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "../../include/mbe.h"
#include "mbe_internal.h"
#include "mbe_learn.h"
#include "mbe_prep.h"
#include "mbe_runtime.h"

#include <cmath>

struct mbe_graph {
    int device = 0;
    int32_t nU = 0, nV = 0;
    int64_t nE = 0;
    int32_t *u_off = nullptr, *u_adj = nullptr, *v_off = nullptr, *v_adj = nullptr;
    mbe::GraphDesc *d_desc = nullptr;
    int32_t max_deg_u = 0, max_deg_v = 0, n_live = 0;
    int64_t nc_max = 0, urow_max = 0, frame_max = 0;
    int32_t *order_static = nullptr; // non-isolated U by descending degree
    int32_t *hist = nullptr;         // max(max_deg_u, key range) + 1 entries
    int32_t hist_len = 0;
    // learned schedule (allocated on first use)
    float *feat = nullptr;           // [nU][8] root features
    float *pred = nullptr;           // [nU] predicted log cost
    int32_t *key = nullptr;          // [nU] order keys
    int32_t *order_l = nullptr;      // [nU] learned order
    int32_t *task_root = nullptr;    // [nU + 32 * kSplitHead] tasks of the learned schedule
    int32_t *task_split = nullptr;
    int32_t *bad = nullptr;
    int32_t *trep = nullptr;         // [nU + 1] top-level twin classes of the pruned search (first use)
};

namespace mbe {
constexpr int kSplitHead = 1024;  // predicted-heaviest roots considered for splitting
constexpr int kMaxParts = 32;     // most tasks one root is split into
constexpr int kMaxKey = 16383;    // order keys: predicted log cost in steps of 1/256
} // namespace mbe

namespace mbe {

// Search workspace shared by every call on a device (grown on demand, kept
// until mbe_release_workspace or process exit).
namespace {
constexpr int kMaxDevices = 64;
Workspace g_ws[kMaxDevices];
} // namespace

Workspace &device_workspace()
{
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= kMaxDevices) dev = 0;
    return g_ws[dev];
}

int set_status(mbe_result *out, int st)
{
    if (out) out->status = st;
    return st;
}

int cuda_status(cudaError_t e)
{
    if (e == cudaSuccess) return MBE_OK;
    if (e == cudaErrorMemoryAllocation) return MBE_ERR_OOM;
    return MBE_ERR_CUDA;
}

#define MBE_TRY(expr)                                                                                                 \
    do {                                                                                                              \
        cudaError_t _e = (expr);                                                                                      \
        if (_e != cudaSuccess) {                                                                                      \
            cudaGetLastError();                                                                                       \
            return cuda_status(_e);                                                                                   \
        }                                                                                                             \
    } while (0)

int64_t round_up(int64_t x, int64_t a) { return (x + a - 1) / a * a; }

// Upper bound on one search launch (MBE_DEADLINE_MS, default 30 minutes):
// every worker compares its own elapsed time with it and stops the launch
// with MBE_ERR_TIMEOUT, so no launch can run unbounded.
long long deadline_ms()
{
    const char *e = getenv("MBE_DEADLINE_MS");
    long long v = e ? atoll(e) : 0;
    return v > 0 ? v : 30LL * 60 * 1000;
}

// Per-worker progress records when MBE_DEBUG_TRACE is set (dumped with mbe_debug_trace).
namespace {
unsigned long long *g_debug = nullptr;
int g_debug_warps = 0;
} // namespace
unsigned long long *debug_buffer(int n_warps)
{
    if (!getenv("MBE_DEBUG_TRACE") || !search_trace_compiled()) return nullptr;
    if (g_debug_warps < n_warps) {
        cudaFree(g_debug);
        g_debug = nullptr;
        g_debug_warps = 0;
        if (cudaMalloc(&g_debug, sizeof(unsigned long long) * MBE_TRACE_WORDS * (size_t)n_warps) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        g_debug_warps = n_warps;
    }
    cudaMemset(g_debug, 0, sizeof(unsigned long long) * MBE_TRACE_WORDS * (size_t)n_warps);
    return g_debug;
}

int key_bits_for(int64_t n)
{
    int b = 1;
    while (b < 31 && ((int64_t)1 << b) < n) ++b;
    return b;
}

int resolve_layout(int32_t requested, int32_t max_deg_v)
{
    if (requested == kLayoutRows || requested == kLayoutColumns) return requested;
    return max_deg_v >= kColumnsMinDegV ? kLayoutColumns : kLayoutRows;
}

LaunchShape shape_for(int block_threads, int blocks_per_sm, int layout)
{
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    auto fit_shape = layout == kLayoutRows ? search_rows_fit_shape : search_fit_shape;
    int threads = block_threads > 0 ? block_threads : 256;
    threads = std::max(32, std::min(1024, threads / 32 * 32));
    int per_sm = blocks_per_sm > 0 ? blocks_per_sm : std::max(1, 512 / threads); // 16 warps per SM by default
    int fit = fit_shape(threads, per_sm);
    if (fit < 0) { // block too large for the kernel's register use
        threads = -fit;
        per_sm = blocks_per_sm > 0 ? blocks_per_sm : std::max(1, 512 / threads);
        fit = fit_shape(threads, per_sm);
    }
    if (fit > 0) per_sm = fit;
    LaunchShape s;
    s.threads = threads;
    s.blocks = sms * per_sm;
    s.warps = s.blocks * (threads / 32);
    s.layout = layout == kLayoutRows ? kLayoutRows : kLayoutColumns;
    return s;
}

LaunchShape choose_shape(const mbe_options &o, int layout)
{
    return shape_for(o.block_threads, o.blocks_per_sm, layout);
}

cudaError_t launch_layout(const SearchArgs &a, int blocks, const LaunchShape &shape, cudaStream_t s)
{
    return shape.layout == kLayoutRows ? launch_search_rows(a, blocks, shape.threads, s)
                                       : launch_search(a, blocks, shape.threads, s);
}

// Sizes (and allocates when needed) the per-warp workspace for a launch.
int ensure_workspace(Workspace &ws, int64_t nc_max, int64_t urow_max, int64_t frame_max, int32_t max_nU,
                     const LaunchShape &shape, int64_t stack_bytes_req, int stack_factor, int32_t max_deg)
{
    // one entry more than the largest candidate set: a new R' list holds the
    // candidates that join R' and the popped vertex itself
    const int64_t ncap = std::max<int64_t>(nc_max + 1, 32);
    const int64_t urow = round_up(std::max<int64_t>(urow_max, 256), 256);
    const int32_t dmax = std::max<int32_t>(max_deg, 32);
    const int64_t scratch = scratch_layout_bytes(ncap, urow, dmax);
    int64_t stack = stack_bytes_req > 0 ? stack_bytes_req : (int64_t)stack_factor * frame_max + (256 << 10);
    stack = round_up(stack, 256);
    const int64_t arena = stack + scratch;
    const int64_t slot = round_up(std::max<int64_t>(frame_max, 4096), 256);
    const int64_t mark_stride = round_up(std::max<int32_t>(max_nU, 1), 64);
    int n_warps = shape.warps;

    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) return MBE_ERR_CUDA;
    const int64_t per_warp = arena + slot + 4 * mark_stride + 4;
    // an existing workspace is reused when every region is large enough; the
    // scratch split is recomputed for this graph inside the same arena
    const bool fits_current = ws.arena && ws.arena_bytes >= arena && ws.slot_bytes >= slot &&
                              ws.mark_stride >= mark_stride && (ws.n_warps >= n_warps || ws.budget_limited);
    if (fits_current) {
        ws.scratch_bytes = scratch;
        ws.n_cand_cap = ncap;
        ws.urow_bytes = urow;
        ws.lbuf_cap = dmax;
        return MBE_OK;
    }
    if (ws.arena) {
        free_b += (size_t)(ws.arena_bytes + ws.slot_bytes + 4 * ws.mark_stride + 4) * ws.n_warps;
        ws.release();
    }
    const int64_t budget = (int64_t)(0.75 * (double)free_b);
    bool limited = false;
    if (per_warp * (int64_t)n_warps > budget) {
        limited = true;
        // fewer resident workers rather than failing: whole blocks only
        int warps_per_block = shape.threads / 32;
        int blocks = (int)(budget / per_warp) / warps_per_block;
        if (blocks < 1) return MBE_ERR_OOM;
        n_warps = blocks * warps_per_block;
    }
    if (cudaMalloc(&ws.arena, (size_t)arena * n_warps) != cudaSuccess ||
        cudaMalloc(&ws.slots, (size_t)slot * n_warps) != cudaSuccess ||
        cudaMalloc(&ws.slot_state, sizeof(int32_t) * (size_t)n_warps) != cudaSuccess ||
        cudaMalloc(&ws.mark, sizeof(int32_t) * (size_t)mark_stride * n_warps) != cudaSuccess ||
        cudaMalloc(&ws.ctl, sizeof(Ctl)) != cudaSuccess) {
        cudaGetLastError();
        ws.release();
        return MBE_ERR_OOM;
    }
    if (cudaMemset(ws.mark, 0xff, sizeof(int32_t) * (size_t)mark_stride * n_warps) != cudaSuccess) {
        ws.release();
        return MBE_ERR_CUDA;
    }
    ws.arena_bytes = arena;
    ws.scratch_bytes = scratch;
    ws.slot_bytes = slot;
    ws.mark_stride = mark_stride;
    ws.n_warps = n_warps;
    ws.threads = shape.threads;
    ws.blocks = n_warps / (shape.threads / 32);
    ws.n_cand_cap = ncap;
    ws.urow_bytes = urow;
    ws.lbuf_cap = dmax;
    ws.budget_limited = limited;
    return MBE_OK;
}


// One persistent search launch (with automatic arena growth on overflow).
int run_search(Workspace &ws, const RunInput &in, const mbe_options &o, cudaStream_t s, mbe_result *out,
               mbe_biclique_buffer *bic)
{
    LaunchShape shape = choose_shape(o, in.layout);
    int stack_factor = 2;
    for (int attempt = 0; attempt < 4; ++attempt) {
        int st = ensure_workspace(ws, in.nc_max, in.urow_max, in.frame_max, in.max_nU, shape, o.arena_bytes,
                                  stack_factor, in.max_deg);
        if (st != MBE_OK) return st;
        if (ws.marks_dirty) {
            MBE_TRY(cudaMemsetAsync(ws.mark, 0xff, sizeof(int32_t) * (size_t)ws.mark_stride * ws.n_warps, s));
            ws.marks_dirty = false;
        }
        MBE_TRY(cudaMemsetAsync(ws.ctl, 0, sizeof(Ctl), s));
        if (in.per_owner)
            MBE_TRY(cudaMemsetAsync(in.per_owner, 0, sizeof(unsigned long long) * 4 * (size_t)in.n_owner, s));
        MBE_TRY(cudaMemsetAsync(ws.slot_state, 0, sizeof(int32_t) * (size_t)ws.n_warps, s));
        SearchArgs a;
        memset(&a, 0, sizeof(a));
        a.u_off = in.u_off;
        a.u_adj = in.u_adj;
        a.v_off = in.v_off;
        a.v_adj = in.v_adj;
        a.graphs = in.d_desc;
        a.n_graphs = in.n_graphs;
        a.key_shift = key_bits_for(std::max<int32_t>(in.max_nU, 2));
        a.task_root = in.task_root;
        a.task_graph = in.task_graph;
        a.task_split = in.task_split;
        a.n_tasks = in.n_tasks;
        a.arena = ws.arena;
        a.arena_bytes = ws.arena_bytes;
        a.scratch_bytes = ws.scratch_bytes;
        a.stack_bytes = ws.arena_bytes - ws.scratch_bytes;
        if (o.arena_bytes > 0) a.stack_bytes = std::min<int64_t>(a.stack_bytes, round_up(o.arena_bytes, 256));
        a.slots = ws.slots;
        a.slot_bytes = ws.slot_bytes;
        a.slot_state = ws.slot_state;
        a.mark = ws.mark;
        a.mark_stride = ws.mark_stride;
        a.n_cand_cap = ws.n_cand_cap;
        a.urow_bytes = ws.urow_bytes;
        a.lbuf_cap = ws.lbuf_cap;
        a.cursor = &ws.ctl->cursor;
        a.n_idle = &ws.ctl->n_idle;
        a.outstanding = &ws.ctl->outstanding;
        a.error = &ws.ctl->error;
        a.watchdog_ns = (long long)(o.watchdog_ms > 0 ? o.watchdog_ms : 60000) * 1000000LL;
        a.deadline_ns = deadline_ms() * 1000000LL;
        a.n_published = &ws.ctl->n_published;
        a.debug = debug_buffer(ws.n_warps);
        a.steal = o.steal ? 1 : 0;
        const int wpb = shape.threads / 32;
        const int blocks = std::min(shape.blocks, ws.n_warps / wpb);
        a.n_warps = blocks * wpb;
        a.max_words = o.bitset_max_words > 0 ? std::min(o.bitset_max_words, kMaxBitsetWords) : kMaxBitsetWords;
        a.min_r = std::max(1, o.min_r);
        a.min_l = std::max(1, o.min_l);
        // the extended kernel variant: some root needs the sorted-list path, a size filter is set, or the
        // bicliques are written
        a.lists = (in.max_deg > 64 * a.max_words || a.min_r > 1 || a.min_l > 1 || (o.emit && bic)) ? 1 : 0;
        // the pruned variant carries the size filter too (and no list path)
        a.prune = in.prune;
        a.trep = in.trep;
        if (a.prune) a.lists = 0;
        a.totals = ws.ctl->totals;
        a.per_task_owner = in.per_owner;
        a.per_root_mode = in.per_mode;
        a.emit = (o.emit && bic) ? 1 : 0;
        if (a.emit) {
            a.out_ids = bic->ids;
            a.cap_ids = bic->capacity_ids;
            a.out_offsets = bic->offsets;
            a.cap_bic = bic->capacity_bicliques;
            a.used_ids = &ws.ctl->used_ids;
            a.used_bic = &ws.ctl->used_bic;
            a.out_full = &ws.ctl->out_full;
        }
        cudaEvent_t e0, e1;
        MBE_TRY(cudaEventCreate(&e0));
        MBE_TRY(cudaEventCreate(&e1));
        cudaEventRecord(e0, s);
        cudaError_t le = launch_layout(a, blocks, shape, s);
        cudaEventRecord(e1, s);
        Ctl h;
        cudaError_t ce = cudaMemcpyAsync(&h, ws.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s);
        cudaError_t se = cudaStreamSynchronize(s);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        if (le != cudaSuccess) return cuda_status(le);
        if (ce != cudaSuccess) return cuda_status(ce);
        if (se != cudaSuccess) return cuda_status(se);
        if (h.error != 0) ws.marks_dirty = true;
        if (h.error == MBE_ERR_ARENA_FULL && o.arena_bytes == 0) {
            stack_factor *= 4; // grow the stacks and run again from scratch
            continue;
        }
        if (out) {
            out->count = h.totals[0];
            out->hash = h.totals[1];
            out->nodes = h.totals[2];
            out->bytes_alg = h.totals[3];
            out->n_donations = h.totals[4];
            out->device_ms = ms;
            out->n_workers = a.n_warps;
        }
        if (a.emit) {
            // sizes the whole output needs (the counters run past the capacities)
            bic->n_ids_written = (int64_t)h.used_ids;
            bic->n_bicliques_written = (int64_t)h.used_bic;
        }
        if (h.error == 0 && h.out_full) return MBE_ERR_OUTPUT_FULL;
        return h.error;
    }
    return MBE_ERR_ARENA_FULL;
}

bool host_csr_ok(const int32_t *off, const int32_t *adj, int32_t n, int32_t n_other, int64_t nE)
{
    if (n < 0 || nE < 0 || !off || off[0] != 0 || (int64_t)off[n] != nE) return false;
    if (nE > 0 && !adj) return false;
    for (int32_t i = 0; i < n; ++i) {
        const int64_t a = off[i], b = off[i + 1];
        if (b < a || b > nE) return false;
        int32_t prev = -1;
        for (int64_t k = a; k < b; ++k) {
            const int32_t x = adj[k];
            if (x <= prev || x >= n_other) return false;
            prev = x;
        }
    }
    return true;
}

// Root features of g into d_feat (and d_raw), using the shared workspace's
// stamp arrays; core numbers are computed on the way.
int root_features(mbe_graph *g, float *d_feat, int32_t *d_raw, cudaStream_t s)
{
    if (g->nU == 0) return MBE_OK;
    Workspace &ws = device_workspace();
    mbe_options o;
    mbe_default_options(&o);
    int st = ensure_workspace(ws, g->nc_max, g->urow_max, g->frame_max, g->nU,
                              choose_shape(o, resolve_layout(o.layout, g->max_deg_v)), 0, 2, g->max_deg_u);
    if (st != MBE_OK) return st;
    const int n = g->nU + g->nV;
    int32_t *tmp = nullptr, *raw = nullptr;
    if (cudaMalloc(&tmp, sizeof(int32_t) * (3 * (size_t)n + 1 + (size_t)g->max_deg_u + 1)) != cudaSuccess ||
        (!d_raw && cudaMalloc(&raw, sizeof(int32_t) * 8 * (size_t)g->nU) != cudaSuccess)) {
        cudaFree(tmp);
        cudaGetLastError();
        return MBE_ERR_OOM;
    }
    int32_t *deg = tmp, *alive = tmp + n, *core = tmp + 2 * n, *removed = tmp + 3 * n, *larger = removed + 1;
    cudaError_t e = compute_core_numbers(g->u_off, g->u_adj, g->v_off, g->v_adj, g->nU, g->nV, deg, alive, core,
                                         removed, s);
    if (e == cudaSuccess) e = degree_larger(g->u_off, g->nU, g->max_deg_u, larger, s);
    const int nw = ws.n_warps / 8 * 8;
    if (e == cudaSuccess)
        e = compute_root_features(g->u_off, g->u_adj, g->v_off, g->v_adj, g->nU, larger, core, ws.mark, ws.mark_stride,
                                  nw, d_raw ? d_raw : raw, d_feat, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(tmp);
    cudaFree(raw);
    return cuda_status(e);
}

// The learned execution order: predicted log cost per root, roots by
// descending prediction (counting sort on quantised keys), and the
// predicted-heaviest roots split into contiguous shares of their level-1
// frames. Without work stealing the split is the only balance: a root
// predicted above half a worker's fair share of the total becomes up to
// kMaxParts tasks. With stealing, idle workers split heavy frames anyway
// and every extra part rebuilds its root (measured: splitting even the few
// heaviest roots into 4 parts cost 10% on the 20k Chung-Lu graph), so
// nothing is pre-split. Falls back to the static order when a prediction is
// not finite.
int learned_schedule(mbe_graph *g, const mbe_model *md, bool presplit, bool stealing, cudaStream_t s,
                     int64_t *n_tasks, bool *fallback, double *prep_ms)
{
    const int nU = g->nU;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, s);
    if (!g->feat) {
        const size_t cap = (size_t)nU + (size_t)kMaxParts * kSplitHead;
        if (cudaMalloc(&g->feat, sizeof(float) * 8 * (size_t)nU) != cudaSuccess ||
            cudaMalloc(&g->pred, sizeof(float) * (size_t)nU) != cudaSuccess ||
            cudaMalloc(&g->key, sizeof(int32_t) * (size_t)nU) != cudaSuccess ||
            cudaMalloc(&g->order_l, sizeof(int32_t) * (size_t)nU) != cudaSuccess ||
            cudaMalloc(&g->task_root, sizeof(int32_t) * cap) != cudaSuccess ||
            cudaMalloc(&g->task_split, sizeof(int32_t) * cap) != cudaSuccess ||
            cudaMalloc(&g->bad, sizeof(int32_t)) != cudaSuccess) {
            cudaGetLastError();
            cudaFree(g->feat);
            g->feat = nullptr;
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            return MBE_ERR_OOM;
        }
        int st = root_features(g, g->feat, nullptr, s);
        if (st != MBE_OK) {
            cudaFree(g->feat);
            g->feat = nullptr;
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            return st;
        }
    }
    cudaError_t e = model_predict(md, g->feat, nU, g->pred, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(g->bad, 0, sizeof(int32_t), s);
    if (e == cudaSuccess) e = learned_order_keys(g->pred, g->u_off, nU, kMaxKey, g->key, g->bad, s);
    if (e == cudaSuccess) e = order_by_key_desc(g->key, nU, kMaxKey, g->hist, g->order_l, s);
    const int64_t n_live = g->n_live;
    const int head = (int)std::min<int64_t>(n_live, kSplitHead);
    std::vector<float> pred((size_t)nU);
    std::vector<int32_t> top((size_t)head);
    int32_t bad = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&bad, g->bad, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(pred.data(), g->pred, sizeof(float) * (size_t)nU, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && head > 0)
        e = cudaMemcpyAsync(top.data(), g->order_l, sizeof(int32_t) * (size_t)head, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        return cuda_status(e);
    }
    *fallback = bad != 0;
    int64_t nt = 0;
    if (!*fallback) {
        std::vector<int32_t> hr, hs;
        if (presplit) {
            double total = 0.0; // predicted nodes over the live roots
            for (int u = 0; u < nU; ++u)
                if (std::isfinite(pred[u]) && pred[u] > 0.f) total += std::expm1((double)pred[u]);
            mbe_options o;
            mbe_default_options(&o);
            const double share =
                total / std::max(1, choose_shape(o, resolve_layout(o.layout, g->max_deg_v)).warps);
            for (int k = 0; k < head; ++k) {
                const int r = top[k];
                const double pn = std::expm1((double)pred[r]);
                int parts = 1;
                if (!stealing && share > 0 && pn > 0.5 * share)
                    parts = (int)std::min<double>(kMaxParts, std::ceil(pn / (0.5 * share)));
                for (int p = 0; p < parts; ++p) {
                    hr.push_back(r);
                    hs.push_back(parts > 1 ? (parts << 16) | p : 0);
                }
            }
        } else {
            hr.assign(top.begin(), top.end());
            hs.assign(top.size(), 0);
        }
        nt = (int64_t)hr.size() + (n_live - head);
        e = cudaMemcpyAsync(g->task_root, hr.data(), sizeof(int32_t) * hr.size(), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(g->task_split, hs.data(), sizeof(int32_t) * hs.size(), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess && n_live > head)
            e = cudaMemcpyAsync(g->task_root + hr.size(), g->order_l + head, sizeof(int32_t) * (size_t)(n_live - head),
                                cudaMemcpyDeviceToDevice, s);
        if (e == cudaSuccess && n_live > head)
            e = cudaMemsetAsync(g->task_split + hr.size(), 0, sizeof(int32_t) * (size_t)(n_live - head), s);
    }
    cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *prep_ms = ms;
    *n_tasks = nt;
    return cuda_status(e);
}

} // namespace mbe

using namespace mbe;

extern "C" {

const char *mbe_status_string(int status)
{
    switch (status) {
    case MBE_OK: return "MBE_OK";
    case MBE_ERR_INVALID_ARG: return "MBE_ERR_INVALID_ARG";
    case MBE_ERR_INVALID_GRAPH: return "MBE_ERR_INVALID_GRAPH";
    case MBE_ERR_OOM: return "MBE_ERR_OOM";
    case MBE_ERR_ARENA_FULL: return "MBE_ERR_ARENA_FULL";
    case MBE_ERR_OUTPUT_FULL: return "MBE_ERR_OUTPUT_FULL";
    case MBE_ERR_TIMEOUT: return "MBE_ERR_TIMEOUT";
    case MBE_ERR_CUDA: return "MBE_ERR_CUDA";
    case MBE_ERR_UNSUPPORTED: return "MBE_ERR_UNSUPPORTED";
    case MBE_ERR_INTERNAL: return "MBE_ERR_INTERNAL";
    default: return "MBE_ERR_UNKNOWN";
    }
}

int mbe_default_options(mbe_options *opt)
{
    if (!opt) return MBE_ERR_INVALID_ARG;
    memset(opt, 0, sizeof(*opt));
    opt->steal = 1;
    opt->root_end = -1;
    return MBE_OK;
}

int mbe_graph_destroy(mbe_graph *g)
{
    if (!g) return MBE_OK;
    cudaFree(g->u_off);
    cudaFree(g->u_adj);
    cudaFree(g->v_off);
    cudaFree(g->v_adj);
    cudaFree(g->d_desc);
    cudaFree(g->order_static);
    cudaFree(g->hist);
    cudaFree(g->feat);
    cudaFree(g->pred);
    cudaFree(g->key);
    cudaFree(g->order_l);
    cudaFree(g->task_root);
    cudaFree(g->task_split);
    cudaFree(g->trep);
    cudaFree(g->bad);
    delete g;
    return MBE_OK;
}

int mbe_graph_create(int32_t nU, int32_t nV, int64_t nE, const int32_t *u_off, const int32_t *u_adj,
                     const int32_t *v_off, const int32_t *v_adj, int32_t ptr_kind, void *stream, mbe_graph **out)
{
    if (!out) return MBE_ERR_INVALID_ARG;
    *out = nullptr;
    if (nU < 0 || nV < 0 || nE < 0 || nE >= ((int64_t)1 << 31) || (ptr_kind != 0 && ptr_kind != 1))
        return MBE_ERR_INVALID_ARG;
    if (!u_off || !v_off || (nE > 0 && (!u_adj || !v_adj))) return MBE_ERR_INVALID_ARG;
    // host input is range-checked before anything reaches the device
    if (ptr_kind == 0 && (!host_csr_ok(u_off, u_adj, nU, nV, nE) || !host_csr_ok(v_off, v_adj, nV, nU, nE)))
        return MBE_ERR_INVALID_GRAPH;
    cudaStream_t s = (cudaStream_t)stream;
    mbe_graph *g = new mbe_graph();
    g->nU = nU;
    g->nV = nV;
    g->nE = nE;
    cudaGetDevice(&g->device);
    auto fail = [&](int st) {
        mbe_graph_destroy(g);
        return st;
    };
    const size_t eb = sizeof(int32_t) * (size_t)std::max<int64_t>(nE, 1);
    if (cudaMalloc(&g->u_off, sizeof(int32_t) * (size_t)(nU + 1)) != cudaSuccess ||
        cudaMalloc(&g->v_off, sizeof(int32_t) * (size_t)(nV + 1)) != cudaSuccess ||
        cudaMalloc(&g->u_adj, eb) != cudaSuccess || cudaMalloc(&g->v_adj, eb) != cudaSuccess ||
        cudaMalloc(&g->d_desc, sizeof(GraphDesc)) != cudaSuccess) {
        cudaGetLastError();
        return fail(MBE_ERR_OOM);
    }
    cudaMemcpyKind kind = ptr_kind == 0 ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    if (cudaMemcpyAsync(g->u_off, u_off, sizeof(int32_t) * (size_t)(nU + 1), kind, s) != cudaSuccess ||
        cudaMemcpyAsync(g->v_off, v_off, sizeof(int32_t) * (size_t)(nV + 1), kind, s) != cudaSuccess ||
        (nE > 0 && cudaMemcpyAsync(g->u_adj, u_adj, sizeof(int32_t) * (size_t)nE, kind, s) != cudaSuccess) ||
        (nE > 0 && cudaMemcpyAsync(g->v_adj, v_adj, sizeof(int32_t) * (size_t)nE, kind, s) != cudaSuccess)) {
        cudaGetLastError();
        return fail(MBE_ERR_CUDA);
    }
    GraphDesc desc{0, 0, 0, nU, nV};
    unsigned long long *d_bounds = nullptr;
    int32_t *d_bad = nullptr;
    if (cudaMalloc(&d_bounds, sizeof(unsigned long long) * 8) != cudaSuccess ||
        cudaMalloc(&d_bad, sizeof(int32_t)) != cudaSuccess) {
        cudaFree(d_bounds);
        cudaGetLastError();
        return fail(MBE_ERR_OOM);
    }
    unsigned long long hb[8] = {0};
    int32_t hbad = 0;
    cudaError_t e = cudaMemcpyAsync(g->d_desc, &desc, sizeof(desc), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_bounds, 0, sizeof(unsigned long long) * 8, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_bad, 0, sizeof(int32_t), s);
    if (e == cudaSuccess) e = validate_graph(g->u_off, g->u_adj, g->v_off, g->v_adj, nU, nV, nE, d_bad, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hbad, d_bad, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess && hbad == 0 && nU > 0)
        e = root_bounds(g->d_desc, 1, nU, g->u_off, g->u_adj, g->v_off, d_bounds, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hb, d_bounds, sizeof(hb), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(d_bounds);
    cudaFree(d_bad);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(cuda_status(e));
    }
    if (hbad != 0) return fail(MBE_ERR_INVALID_GRAPH);
    g->nc_max = (int64_t)hb[0];
    g->urow_max = (int64_t)hb[1];
    g->frame_max = (int64_t)hb[2];
    g->max_deg_u = (int32_t)hb[3];
    g->n_live = (int32_t)hb[4];
    {
        int32_t *d_m = nullptr, hm = 0;
        e = cudaMalloc(&d_m, sizeof(int32_t));
        if (e == cudaSuccess) e = cudaMemsetAsync(d_m, 0, sizeof(int32_t), s);
        if (e == cudaSuccess && nV > 0) e = max_degree(g->v_off, nV, d_m, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&hm, d_m, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        cudaFree(d_m);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(cuda_status(e));
        }
        g->max_deg_v = hm;
    }
    g->hist_len = std::max<int32_t>(g->max_deg_u, kMaxKey) + 1;
    if (cudaMalloc(&g->order_static, sizeof(int32_t) * (size_t)std::max(nU, 1)) != cudaSuccess ||
        cudaMalloc(&g->hist, sizeof(int32_t) * (size_t)g->hist_len) != cudaSuccess) {
        cudaGetLastError();
        return fail(MBE_ERR_OOM);
    }
    if (nU > 0) {
        e = order_by_degree_desc(g->u_off, nU, g->max_deg_u, g->hist, g->order_static, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(cuda_status(e));
        }
    }
    *out = g;
    return MBE_OK;
}

// Copies the progress records of the last launch (8 u64 per worker) to host
// memory; returns the number of workers recorded (0 unless MBE_DEBUG_TRACE).
int mbe_debug_trace(uint64_t *host, int32_t max_workers)
{
    if (!g_debug || !host) return 0;
    int n = std::min(max_workers, g_debug_warps);
    if (cudaMemcpy(host, g_debug, sizeof(uint64_t) * MBE_TRACE_WORDS * (size_t)n, cudaMemcpyDeviceToHost) != cudaSuccess) return 0;
    return n;
}

int mbe_root_features(const mbe_graph *gc, float *d_feat, int32_t *d_raw, void *stream)
{
    if (!gc || (gc->nU > 0 && !d_feat)) return MBE_ERR_INVALID_ARG;
    return root_features(const_cast<mbe_graph *>(gc), d_feat, d_raw, (cudaStream_t)stream);
}

int mbe_release_workspace(void)
{
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev >= 0 && dev < kMaxDevices) g_ws[dev].release();
    return MBE_OK;
}

int mbe_graph_info(const mbe_graph *g, int32_t *nU, int32_t *nV, int64_t *nE, int32_t *max_deg_u,
                   int32_t *max_deg_v)
{
    if (!g) return MBE_ERR_INVALID_ARG;
    if (nU) *nU = g->nU;
    if (nV) *nV = g->nV;
    if (nE) *nE = g->nE;
    if (max_deg_u) *max_deg_u = g->max_deg_u;
    if (max_deg_v) *max_deg_v = g->max_deg_v;
    return MBE_OK;
}

int mbe_enumerate(const mbe_graph *gc, const mbe_options *opts, void *stream, mbe_result *out,
                  mbe_biclique_buffer *bicliques)
{
    if (out) memset(out, 0, sizeof(*out));
    if (!gc) return set_status(out, MBE_ERR_INVALID_ARG);
    mbe_graph *g = const_cast<mbe_graph *>(gc);
    mbe_options o;
    mbe_default_options(&o);
    if (opts) o = *opts;
    if (o.emit && !bicliques) return set_status(out, MBE_ERR_INVALID_ARG);
    if (o.emit && (!bicliques->ids || !bicliques->offsets || bicliques->capacity_ids < 0 ||
                   bicliques->capacity_bicliques < 0))
        return set_status(out, MBE_ERR_INVALID_ARG);
    if (o.block_threads < 0 || o.blocks_per_sm < 0 || o.watchdog_ms < 0 || o.arena_bytes < 0 || o.layout < 0 ||
        o.layout > kLayoutColumns || o.bitset_max_words < 0 || o.min_r < 0 || o.min_l < 0 || o.prune < 0 ||
        o.prune > 1)
        return set_status(out, MBE_ERR_INVALID_ARG);
    cudaStream_t s = (cudaStream_t)stream;
    if (g->nU == 0 || g->n_live == 0) return set_status(out, MBE_OK);

    const int32_t *order = g->order_static;
    const int32_t *split = nullptr;
    int64_t n_order = g->n_live;
    double prep_ms = 0.0;
    if (o.exec_order) {
        if (o.n_exec < 0 || o.n_exec > g->nU) return set_status(out, MBE_ERR_INVALID_ARG);
        order = o.exec_order;
        n_order = o.n_exec;
    } else if (o.schedule == 1 || o.schedule == 2) {
        if (!o.model) return set_status(out, MBE_ERR_INVALID_ARG);
        int64_t n_tasks = 0;
        bool fallback = false;
        int st = learned_schedule(g, static_cast<const mbe_model *>(o.model), o.schedule == 1, o.steal != 0, s, &n_tasks,
                                  &fallback, &prep_ms);
        if (st != MBE_OK) return set_status(out, st);
        if (!fallback) {
            order = g->task_root;
            split = g->task_split;
            n_order = n_tasks;
        }
    } else if (o.schedule != 0) {
        return set_status(out, MBE_ERR_INVALID_ARG);
    }
    if (split && (o.root_begin > 0 || o.root_end >= 0)) return set_status(out, MBE_ERR_INVALID_ARG);
    int64_t b = std::max<int64_t>(0, o.root_begin);
    int64_t e = o.root_end < 0 ? n_order : std::min<int64_t>(o.root_end, n_order);
    if (b > e) return set_status(out, MBE_ERR_INVALID_ARG);

    RunInput in;
    in.u_off = g->u_off;
    in.u_adj = g->u_adj;
    in.v_off = g->v_off;
    in.v_adj = g->v_adj;
    in.d_desc = g->d_desc;
    in.n_graphs = 1;
    in.max_nU = g->nU;
    in.task_root = order + b;
    in.task_graph = nullptr;
    in.task_split = split;
    in.n_tasks = e - b;
    in.nc_max = g->nc_max;
    in.urow_max = g->urow_max;
    in.frame_max = g->frame_max;
    in.per_owner = reinterpret_cast<unsigned long long *>(o.per_root);
    in.n_owner = g->nU;
    in.per_mode = 1;
    in.layout = resolve_layout(o.layout, g->max_deg_v);
    in.max_deg = g->max_deg_u;
    if (o.prune) {
        const int32_t mw = o.bitset_max_words > 0 ? std::min(o.bitset_max_words, kMaxBitsetWords) : kMaxBitsetWords;
        if (g->max_deg_u > 64 * mw) return set_status(out, MBE_ERR_UNSUPPORTED);
        if (!g->trep) {
            if (cudaMalloc(&g->trep, sizeof(int32_t) * (size_t)(g->nU + 1)) != cudaSuccess) {
                cudaGetLastError();
                g->trep = nullptr;
                return set_status(out, MBE_ERR_OOM);
            }
            cudaError_t te = twin_classes(g->d_desc, 1, g->nU, (int64_t)g->nU + 1, g->u_off, g->u_adj, g->trep, s);
            if (te != cudaSuccess) {
                cudaFree(g->trep);
                g->trep = nullptr;
                return set_status(out, cuda_status(te));
            }
        }
        in.prune = 1;
        in.trep = g->trep;
    }
    int st = run_search(device_workspace(), in, o, s, out, bicliques);
    if (out) out->prep_ms = prep_ms;
    return set_status(out, st);
}

} // extern "C"
