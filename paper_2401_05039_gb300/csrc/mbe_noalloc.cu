// mbe_enumerate_noalloc: the whole-graph enumeration of mbe_enumerate with
// every byte of scratch taken from one fixed array compiled into this file,
// for callers that must not allocate device memory.
//
// Some callers cannot call cudaMalloc: code that runs inside a framework
// which owns all device memory through its own pool (a raw cudaMalloc there
// can fail, or fragment the pool), and latency-critical loops that must not
// hit cudaMalloc/cudaFree (cudaFree synchronises the whole device). Such a
// caller keeps its graph in its own device buffers and gets the result in a
// host struct; this entry point allocates nothing on the device or the host
// and calls no allocating library routine.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>

#include "../../include/mbe.h"
#include "mbe_internal.h"
#include "mbe_prep.h"

namespace mbe {
namespace {

// The scratch of every mbe_enumerate_noalloc call on a device. It exists on
// every GPU that loads the library, for the life of the process.
constexpr size_t kNoAllocBytes = (size_t)64 << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

// Its device address, looked up once per device (host code cannot use the
// symbol itself: on the host it names a stand-in, not device memory).
constexpr int kMaxDev = 64;
unsigned char *g_noalloc_ptr[kMaxDev] = {nullptr};

// Control block at the start of the array (cleared by every call).
struct NoAllocCtl {
    unsigned long long cursor;
    long long outstanding;
    int32_t n_idle;
    int32_t error;
    int32_t n_published;
    int32_t bad;
    unsigned long long totals[8];
    unsigned long long bounds[8];
    GraphDesc desc;
};

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

int status_of(cudaError_t e)
{
    if (e == cudaSuccess) return MBE_OK;
    cudaGetLastError();
    return MBE_ERR_CUDA;
}

} // namespace
} // namespace mbe

using namespace mbe;

extern "C" int mbe_enumerate_noalloc(int32_t nU, int32_t nV, int64_t nE, const int32_t *u_off, const int32_t *u_adj,
                                     const int32_t *v_off, const int32_t *v_adj, void *stream, mbe_result *out)
{
    if (out) memset(out, 0, sizeof(*out));
    if (!out || nU < 0 || nV < 0 || nE < 0 || nE >= ((int64_t)1 << 31) || !u_off || !v_off ||
        (nE > 0 && (!u_adj || !v_adj)))
        return out ? (out->status = MBE_ERR_INVALID_ARG) : MBE_ERR_INVALID_ARG;
    auto fail = [&](int st) {
        out->status = st;
        return st;
    };
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev) return fail(status_of(cudaErrorInvalidDevice));

    // Set-up, once per device, with that device current. Two host threads
    // that race here both store the same address, so the race is benign.
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) return fail(status_of(e == cudaSuccess ? cudaErrorInvalidSymbol : e));
        g_noalloc_ptr[dev] = static_cast<unsigned char *>(p);
    }
    unsigned char *base = g_noalloc_ptr[dev];
    NoAllocCtl *ctl = reinterpret_cast<NoAllocCtl *>(base);
    size_t used = align256(sizeof(NoAllocCtl));

    // Validation (clears what must start at zero first). Its verdict is read
    // back before anything else touches the caller's arrays: the bounds
    // kernel below indexes with the graph's offsets and ids.
    GraphDesc desc{0, 0, 0, nU, nV};
    cudaError_t e = cudaMemsetAsync(ctl, 0, sizeof(NoAllocCtl), s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&ctl->desc, &desc, sizeof(desc), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = validate_graph(u_off, u_adj, v_off, v_adj, nU, nV, nE, &ctl->bad, s);
    int32_t bad = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&bad, &ctl->bad, sizeof(bad), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail(status_of(e));
    if (bad) return fail(MBE_ERR_INVALID_GRAPH);
    // Per-root workspace bounds of the validated graph.
    unsigned long long hb[8] = {0};
    if (nU > 0) e = root_bounds(&ctl->desc, 1, nU, u_off, u_adj, v_off, ctl->bounds, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hb, ctl->bounds, sizeof(hb), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail(status_of(e));
    const int64_t nc_max = (int64_t)hb[0], urow_max = (int64_t)hb[1], frame_max = (int64_t)hb[2];
    const int32_t max_deg = (int32_t)hb[3], n_live = (int32_t)hb[4];
    if (nU == 0 || n_live == 0) return fail(MBE_OK);

    // Layout: execution order and its histogram, then the per-worker regions.
    int32_t *order = reinterpret_cast<int32_t *>(base + used);
    used += align256(sizeof(int32_t) * (size_t)nU);
    int32_t *hist = reinterpret_cast<int32_t *>(base + used);
    used += align256(sizeof(int32_t) * (size_t)(max_deg + 1));
    const int64_t ncap = std::max<int64_t>(nc_max + 1, 32);
    const int64_t urow = (int64_t)align256((size_t)std::max<int64_t>(urow_max, 256));
    const int32_t dmax = std::max<int32_t>(max_deg, 32);
    const int64_t scratch = scratch_layout_bytes(ncap, urow, dmax);
    const int64_t slot = (int64_t)align256((size_t)std::max<int64_t>(frame_max, 4096));
    const int64_t mark_stride = (nU + 63) / 64 * 64;
    const int64_t min_stack = (int64_t)align256((size_t)(2 * frame_max + (256 << 10)));
    const int64_t fixed_per_warp = scratch + slot + 4 * mark_stride + 4;
    if (used >= kNoAllocBytes) return fail(MBE_ERR_UNSUPPORTED);
    const int64_t room = (int64_t)(kNoAllocBytes - used) - 256 * 4;
    const int threads = 256, wpb = threads / 32;
    int per_sm = search_fit_shape(threads, 2);
    int sms = 152;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int n_warps = std::max(per_sm, 1) * sms * wpb;
    int64_t fit = room / (fixed_per_warp + min_stack);
    if (fit < n_warps) n_warps = (int)(fit / wpb) * wpb;
    if (n_warps < wpb) return fail(MBE_ERR_UNSUPPORTED); // the graph needs more scratch than the array holds
    // every worker gets the same stack: the room left after the fixed parts
    const int64_t stack = std::max<int64_t>(
        min_stack, (room - fixed_per_warp * n_warps) / n_warps / 256 * 256);
    const int64_t arena = stack + scratch;
    int32_t *slot_state = reinterpret_cast<int32_t *>(base + used);
    used += align256(sizeof(int32_t) * (size_t)n_warps);
    int32_t *mark = reinterpret_cast<int32_t *>(base + used);
    used += align256(sizeof(int32_t) * (size_t)mark_stride * n_warps);
    char *slots = reinterpret_cast<char *>(base + used);
    used += (size_t)slot * n_warps;
    char *arenas = reinterpret_cast<char *>(base + used);
    used += (size_t)arena * n_warps;
    if (used > kNoAllocBytes) return fail(MBE_ERR_UNSUPPORTED);

    // The array keeps the previous call's contents: reset what the search
    // expects in a known state.
    e = order_by_degree_desc(u_off, nU, max_deg, hist, order, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(slot_state, 0, sizeof(int32_t) * (size_t)n_warps, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(mark, 0xff, sizeof(int32_t) * (size_t)mark_stride * n_warps, s);
    if (e != cudaSuccess) return fail(status_of(e));

    SearchArgs a;
    memset(&a, 0, sizeof(a));
    a.u_off = u_off;
    a.u_adj = u_adj;
    a.v_off = v_off;
    a.v_adj = v_adj;
    a.graphs = &ctl->desc;
    a.n_graphs = 1;
    int kb = 1;
    while (kb < 31 && ((int64_t)1 << kb) < std::max<int32_t>(nU, 2)) ++kb;
    a.key_shift = kb;
    a.task_root = order;
    a.task_graph = nullptr;
    a.n_tasks = n_live;
    a.arena = arenas;
    a.arena_bytes = arena;
    a.scratch_bytes = scratch;
    a.stack_bytes = stack;
    a.slots = slots;
    a.slot_bytes = slot;
    a.slot_state = slot_state;
    a.mark = mark;
    a.mark_stride = mark_stride;
    a.n_cand_cap = ncap;
    a.urow_bytes = urow;
    a.lbuf_cap = dmax;
    a.cursor = &ctl->cursor;
    a.n_idle = &ctl->n_idle;
    a.outstanding = &ctl->outstanding;
    a.error = &ctl->error;
    a.watchdog_ns = 60000LL * 1000000LL;
    a.deadline_ns = 30LL * 60 * 1000 * 1000000LL;
    a.n_published = &ctl->n_published;
    a.debug = nullptr;
    a.steal = 1;
    a.n_warps = n_warps;
    a.max_words = kMaxBitsetWords;
    a.lists = max_deg > 64 * kMaxBitsetWords ? 1 : 0;
    a.min_r = 1;
    a.min_l = 1;
    a.totals = ctl->totals;
    a.per_task_owner = nullptr;
    a.per_root_mode = 1;
    a.emit = 0;
    e = launch_search(a, n_warps / wpb, threads, s);
    if (e != cudaSuccess) return fail(status_of(e));
    NoAllocCtl h;
    e = cudaMemcpyAsync(&h, ctl, sizeof(h), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail(status_of(e));
    out->count = h.totals[0];
    out->hash = h.totals[1];
    out->nodes = h.totals[2];
    out->bytes_alg = h.totals[3];
    out->n_donations = h.totals[4];
    out->device_ms = -1.0; // not timed: timing events would be allocations
    out->n_workers = n_warps;
    return fail(h.error);
}
