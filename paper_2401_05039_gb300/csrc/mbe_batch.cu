// Many-graph enumeration: size classes, one persistent launch per class,
// all class launches captured in one CUDA graph, and the per-class
// autotuner. The search kernel is the single-graph one; graphs are told
// apart by a descriptor per (graph, root) task.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "../../include/mbe.h"
#include "mbe_internal.h"
#include "mbe_prep.h"
#include "mbe_runtime.h"

namespace mbe {
namespace {

struct HostBatch {
    int32_t n_graphs;
    const int64_t *edge_off;
    const int32_t *nU, *nV;
    const int64_t *u_off_start, *v_off_start;
    const int32_t *u_off_cat, *u_adj_cat, *v_off_cat, *v_adj_cat;
};

int class_of(int32_t nU, int32_t nV, int64_t nE)
{
    return (nU >= 128 ? 4 : 0) + (nV >= 512 ? 2 : 0) + ((double)nE >= 0.1 * (double)nU * (double)nV ? 1 : 0);
}

// Device copy of a batch plus its per-graph bounds.
struct DeviceBatch {
    int32_t *uo = nullptr, *vo = nullptr, *ua = nullptr, *va = nullptr, *bad = nullptr;
    GraphDesc *desc = nullptr;
    unsigned long long *gbounds = nullptr; // [G][4]
    unsigned long long *owner = nullptr;   // [G][4]
    Ctl *ctls = nullptr;                   // [MBE_N_CLASSES]
    int32_t *tasks = nullptr;              // task_root then task_graph, 2 * n_tasks
    int64_t n_tasks_cap = 0;
    std::vector<unsigned long long> hb;    // host copy of gbounds
    int32_t max_nU = 1;
    int64_t n_uoff = 0;                    // entries of the concatenated u_off
    int32_t *trep = nullptr;               // [n_uoff] twin classes of the pruned search (on request)

    void release()
    {
        cudaFree(uo);
        cudaFree(vo);
        cudaFree(ua);
        cudaFree(va);
        cudaFree(bad);
        cudaFree(desc);
        cudaFree(gbounds);
        cudaFree(owner);
        cudaFree(ctls);
        cudaFree(tasks);
        cudaFree(trep);
        *this = DeviceBatch();
    }
};

int upload(const HostBatch &b, DeviceBatch &d, cudaStream_t s)
{
    const int32_t G = b.n_graphs;
    std::vector<GraphDesc> desc((size_t)G);
    int64_t n_uoff = 0, n_voff = 0, n_tasks = 0;
    const int64_t nE = b.edge_off[G];
    for (int32_t i = 0; i < G; ++i) {
        if (b.nU[i] < 0 || b.nV[i] < 0 || b.nU[i] > 65536 || b.edge_off[i + 1] < b.edge_off[i] ||
            b.u_off_start[i] < 0 || b.v_off_start[i] < 0)
            return MBE_ERR_INVALID_ARG;
        desc[i] = GraphDesc{b.u_off_start[i], b.v_off_start[i], b.edge_off[i], b.nU[i], b.nV[i]};
        n_uoff = std::max<int64_t>(n_uoff, b.u_off_start[i] + b.nU[i] + 1);
        n_voff = std::max<int64_t>(n_voff, b.v_off_start[i] + b.nV[i] + 1);
        d.max_nU = std::max(d.max_nU, b.nU[i]);
        n_tasks += b.nU[i];
    }
    if (nE > 0 && (!b.u_adj_cat || !b.v_adj_cat)) return MBE_ERR_INVALID_ARG;
    if (nE >= ((int64_t)1 << 31)) return MBE_ERR_UNSUPPORTED;
    if (b.edge_off[0] < 0) return MBE_ERR_INVALID_ARG;
    // the arrays are host memory: check every graph's offsets and ids here,
    // so that the device checks below (sortedness, transposes) and every
    // later kernel index only with values that stay inside the graph
    for (int32_t i = 0; i < G; ++i) {
        const int64_t ne = b.edge_off[i + 1] - b.edge_off[i];
        if (!host_csr_ok(b.u_off_cat + b.u_off_start[i], b.u_adj_cat ? b.u_adj_cat + b.edge_off[i] : nullptr,
                         b.nU[i], b.nV[i], ne) ||
            !host_csr_ok(b.v_off_cat + b.v_off_start[i], b.v_adj_cat ? b.v_adj_cat + b.edge_off[i] : nullptr,
                         b.nV[i], b.nU[i], ne))
            return MBE_ERR_INVALID_GRAPH;
    }
    const size_t eb = sizeof(int32_t) * (size_t)std::max<int64_t>(nE, 1);
    d.n_tasks_cap = std::max<int64_t>(n_tasks, 1);
    d.n_uoff = n_uoff;
    if (cudaMalloc(&d.uo, sizeof(int32_t) * (size_t)n_uoff) != cudaSuccess ||
        cudaMalloc(&d.vo, sizeof(int32_t) * (size_t)n_voff) != cudaSuccess || cudaMalloc(&d.ua, eb) != cudaSuccess ||
        cudaMalloc(&d.va, eb) != cudaSuccess || cudaMalloc(&d.bad, sizeof(int32_t)) != cudaSuccess ||
        cudaMalloc(&d.desc, sizeof(GraphDesc) * (size_t)G) != cudaSuccess ||
        cudaMalloc(&d.gbounds, sizeof(unsigned long long) * 4 * (size_t)G) != cudaSuccess ||
        cudaMalloc(&d.owner, sizeof(unsigned long long) * 4 * (size_t)G) != cudaSuccess ||
        cudaMalloc(&d.ctls, sizeof(Ctl) * MBE_N_CLASSES) != cudaSuccess ||
        cudaMalloc(&d.tasks, sizeof(int32_t) * 2 * (size_t)d.n_tasks_cap) != cudaSuccess) {
        cudaGetLastError();
        return MBE_ERR_OOM;
    }
    cudaError_t e = cudaMemcpyAsync(d.uo, b.u_off_cat, sizeof(int32_t) * (size_t)n_uoff, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d.vo, b.v_off_cat, sizeof(int32_t) * (size_t)n_voff, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && nE > 0) e = cudaMemcpyAsync(d.ua, b.u_adj_cat, eb, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && nE > 0) e = cudaMemcpyAsync(d.va, b.v_adj_cat, eb, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d.desc, desc.data(), sizeof(GraphDesc) * (size_t)G, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(d.bad, 0, sizeof(int32_t), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(d.gbounds, 0, sizeof(unsigned long long) * 4 * (size_t)G, s);
    if (e == cudaSuccess) e = validate_batch(d.desc, G, d.uo, d.ua, d.vo, d.va, d.bad, s);
    if (e == cudaSuccess) e = graph_bounds(d.desc, G, d.uo, d.ua, d.vo, d.gbounds, s);
    int32_t hbad = 0;
    d.hb.assign((size_t)G * 4, 0);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hbad, d.bad, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d.hb.data(), d.gbounds, sizeof(unsigned long long) * 4 * (size_t)G,
                            cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_status(e);
    if (hbad) return MBE_ERR_INVALID_GRAPH;
    for (int32_t i = 0; i < G; ++i)
        if (d.hb[4 * (size_t)i + 3] > 2048) return MBE_ERR_UNSUPPORTED;
    return MBE_OK;
}

// The (graph, root) tasks of one class, heaviest graphs first (edges x
// density^2), roots of a graph by falling degree.
struct ClassPlan {
    int cls = 0;
    std::vector<int32_t> troot, tgraph;
    int64_t nc_max = 0, urow_max = 0, frame_max = 0;
    int32_t max_nU = 1;
    int32_t max_deg_v = 0; // largest V degree of the class's graphs (automatic layout choice)
};

void plan_class(const HostBatch &b, const DeviceBatch &d, const std::vector<int32_t> &graphs, ClassPlan &p)
{
    std::vector<int32_t> order(graphs);
    auto key = [&](int32_t i) {
        double ne = (double)(b.edge_off[i + 1] - b.edge_off[i]);
        double dens = (b.nU[i] && b.nV[i]) ? ne / ((double)b.nU[i] * b.nV[i]) : 0.0;
        return ne * dens * dens;
    };
    std::stable_sort(order.begin(), order.end(), [&](int32_t x, int32_t y) { return key(x) > key(y); });
    std::vector<std::pair<int32_t, int32_t>> tmp;
    for (int32_t gi : order) {
        const int32_t *uo = b.u_off_cat + b.u_off_start[gi];
        tmp.clear();
        for (int32_t u = 0; u < b.nU[gi]; ++u) {
            int32_t deg = uo[u + 1] - uo[u];
            if (deg > 0) tmp.push_back({-deg, u});
        }
        std::sort(tmp.begin(), tmp.end());
        for (auto &t : tmp) {
            p.troot.push_back(t.second);
            p.tgraph.push_back(gi);
        }
        p.nc_max = std::max<int64_t>(p.nc_max, (int64_t)d.hb[4 * (size_t)gi + 0]);
        p.urow_max = std::max<int64_t>(p.urow_max, (int64_t)d.hb[4 * (size_t)gi + 1]);
        p.frame_max = std::max<int64_t>(p.frame_max, (int64_t)d.hb[4 * (size_t)gi + 2]);
        p.max_nU = std::max(p.max_nU, b.nU[gi]);
        const int32_t *vo = b.v_off_cat + b.v_off_start[gi];
        for (int32_t v = 0; v < b.nV[gi]; ++v) p.max_deg_v = std::max(p.max_deg_v, vo[v + 1] - vo[v]);
    }
}

struct ClassLaunch {
    LaunchShape shape;
    int steal;
};

ClassLaunch launch_for(const mbe_class_params *prm, const mbe_options &o, const ClassPlan &p)
{
    ClassLaunch c;
    if (prm && prm->valid) {
        c.shape = shape_for(prm->block_threads, prm->blocks_per_sm, resolve_layout(prm->layout, p.max_deg_v));
        c.steal = prm->steal ? 1 : 0;
    } else {
        c.shape = shape_for(o.block_threads, o.blocks_per_sm, resolve_layout(o.layout, p.max_deg_v));
        c.steal = o.steal ? 1 : 0;
    }
    return c;
}

// Library-owned stream to capture into (the legacy default stream cannot
// be captured); the captured graph is then launched on the caller's stream.
cudaStream_t capture_stream()
{
    static cudaStream_t cs[64] = {nullptr};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) return nullptr;
    if (!cs[dev] && cudaStreamCreateWithFlags(&cs[dev], cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return cs[dev];
}

// Runs the given classes back to back on the stream, one persistent launch
// each; with `capture` the whole sequence is captured into a CUDA graph and
// launched as one. *ms = device time of the sequence.
int run_classes(DeviceBatch &d, std::vector<ClassPlan> &plans, const std::vector<ClassLaunch> &cl,
                const mbe_options &o, cudaStream_t s, bool capture, double *ms, uint64_t *donations,
                std::vector<double> *class_ms = nullptr)
{
    Workspace &ws = device_workspace();
    int64_t nc = 0, urow = 0, frame = 0, n_tasks = 0;
    int32_t max_nU = 1;
    LaunchShape big = cl.empty() ? shape_for(0, 0, kLayoutColumns) : cl[0].shape;
    for (size_t k = 0; k < plans.size(); ++k) {
        nc = std::max(nc, plans[k].nc_max);
        urow = std::max(urow, plans[k].urow_max);
        frame = std::max(frame, plans[k].frame_max);
        max_nU = std::max(max_nU, plans[k].max_nU);
        n_tasks += (int64_t)plans[k].troot.size();
        if (cl[k].shape.warps > big.warps) big = cl[k].shape;
    }
    if (n_tasks > d.n_tasks_cap) return MBE_ERR_INVALID_ARG;
    // task arrays: class k's tasks are contiguous
    std::vector<int32_t> host_tasks((size_t)2 * n_tasks);
    std::vector<int64_t> off(plans.size() + 1, 0);
    for (size_t k = 0; k < plans.size(); ++k) {
        std::copy(plans[k].troot.begin(), plans[k].troot.end(), host_tasks.begin() + off[k]);
        std::copy(plans[k].tgraph.begin(), plans[k].tgraph.end(), host_tasks.begin() + n_tasks + off[k]);
        off[k + 1] = off[k] + (int64_t)plans[k].troot.size();
    }
    cudaError_t e = cudaMemcpyAsync(d.tasks, host_tasks.data(), sizeof(int32_t) * host_tasks.size(),
                                    cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_status(e);

    int stack_factor = 2;
    for (int attempt = 0; attempt < 4; ++attempt) {
        int st = ensure_workspace(ws, nc, urow, frame, max_nU, big, o.arena_bytes, stack_factor, kMaxBitsetWords * 64);
        if (st != MBE_OK) return st;
        if (ws.marks_dirty) {
            e = cudaMemsetAsync(ws.mark, 0xff, sizeof(int32_t) * (size_t)ws.mark_stride * ws.n_warps, s);
            if (e != cudaSuccess) return cuda_status(e);
            ws.marks_dirty = false;
        }
        e = cudaMemsetAsync(d.owner, 0, sizeof(unsigned long long) * 4 * (size_t)(d.hb.size() / 4), s);
        if (e != cudaSuccess) return cuda_status(e);
        // one SearchArgs per class
        std::vector<SearchArgs> args(plans.size());
        std::vector<int> blocks(plans.size());
        for (size_t k = 0; k < plans.size(); ++k) {
            SearchArgs &a = args[k];
            memset(&a, 0, sizeof(a));
            a.u_off = d.uo;
            a.u_adj = d.ua;
            a.v_off = d.vo;
            a.v_adj = d.va;
            a.graphs = d.desc;
            a.n_graphs = (int32_t)(d.hb.size() / 4);
            a.key_shift = key_bits_for(std::max<int32_t>(max_nU, 2));
            a.task_root = d.tasks + off[k];
            a.task_graph = d.tasks + n_tasks + off[k];
            a.n_tasks = off[k + 1] - off[k];
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
            Ctl *c = d.ctls + k;
            a.cursor = &c->cursor;
            a.n_idle = &c->n_idle;
            a.outstanding = &c->outstanding;
            a.error = &c->error;
            a.n_published = &c->n_published;
            a.totals = c->totals;
            a.watchdog_ns = (long long)(o.watchdog_ms > 0 ? o.watchdog_ms : 60000) * 1000000LL;
            a.deadline_ns = deadline_ms() * 1000000LL;
            a.debug = nullptr;
            a.steal = cl[k].steal;
            const int wpb = cl[k].shape.threads / 32;
            blocks[k] = std::min(cl[k].shape.blocks, ws.n_warps / wpb);
            a.n_warps = blocks[k] * wpb;
            a.max_words = kMaxBitsetWords;
            a.min_r = std::max(1, o.min_r);
            a.min_l = std::max(1, o.min_l);
            a.lists = (a.min_r > 1 || a.min_l > 1) ? 1 : 0; // the size filter runs in the extended variant
            a.prune = d.trep ? 1 : 0;                      // the pruned variant carries the filter too
            a.trep = d.trep;
            if (a.prune) a.lists = 0;
            a.per_task_owner = d.owner;
            a.per_root_mode = 2;
            a.emit = 0;
        }
        cudaGraph_t graph = nullptr;
        cudaGraphExec_t exec = nullptr;
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        // one event after every class launch (inside a capture: external
        // event nodes, recorded when the graph runs) for per-class times
        std::vector<cudaEvent_t> ce(plans.size(), nullptr);
        for (auto &x : ce) cudaEventCreate(&x);
        auto enqueue = [&](cudaStream_t q) -> cudaError_t {
            cudaError_t r = cudaMemsetAsync(d.ctls, 0, sizeof(Ctl) * MBE_N_CLASSES, q);
            for (size_t k = 0; k < plans.size() && r == cudaSuccess; ++k) {
                if (args[k].n_tasks > 0) {
                    r = cudaMemsetAsync(ws.slot_state, 0, sizeof(int32_t) * (size_t)ws.n_warps, q);
                    if (r == cudaSuccess) r = launch_layout(args[k], blocks[k], cl[k].shape, q);
                }
                if (r == cudaSuccess)
                    r = capture ? cudaEventRecordWithFlags(ce[k], q, cudaEventRecordExternal) : cudaEventRecord(ce[k], q);
            }
            return r;
        };
        if (capture) {
            cudaStream_t cs = capture_stream();
            e = cs ? cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) : cudaErrorInvalidResourceHandle;
            if (e == cudaSuccess) {
                cudaError_t q = enqueue(cs);
                e = cudaStreamEndCapture(cs, &graph);
                if (e == cudaSuccess) e = q;
            }
            if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
            if (e == cudaSuccess) e = cudaEventRecord(e0, s);
            if (e == cudaSuccess) e = cudaGraphLaunch(exec, s);
            if (e == cudaSuccess) e = cudaEventRecord(e1, s);
        } else {
            e = cudaEventRecord(e0, s);
            if (e == cudaSuccess) e = enqueue(s);
            if (e == cudaSuccess) e = cudaEventRecord(e1, s);
        }
        std::vector<Ctl> hc(MBE_N_CLASSES);
        if (e == cudaSuccess) e = cudaMemcpyAsync(hc.data(), d.ctls, sizeof(Ctl) * MBE_N_CLASSES, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        float t = 0.f;
        if (e == cudaSuccess) cudaEventElapsedTime(&t, e0, e1);
        if (class_ms) {
            class_ms->assign(plans.size(), -1.0);
            for (size_t k = 0; k < plans.size() && e == cudaSuccess; ++k) {
                float tk = 0.f;
                if (cudaEventElapsedTime(&tk, k == 0 ? e0 : ce[k - 1], ce[k]) == cudaSuccess) (*class_ms)[k] = tk;
                else cudaGetLastError();
            }
        }
        for (auto &x : ce) cudaEventDestroy(x);
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        if (e != cudaSuccess) return cuda_status(e);
        int err = 0;
        uint64_t don = 0;
        for (size_t k = 0; k < plans.size(); ++k) {
            if (hc[k].error && !err) err = hc[k].error;
            don += hc[k].totals[4];
        }
        if (err) ws.marks_dirty = true;
        if (err == MBE_ERR_ARENA_FULL && o.arena_bytes == 0) {
            stack_factor *= 4;
            continue;
        }
        if (ms) *ms = t;
        if (donations) *donations = don;
        return err;
    }
    return MBE_ERR_ARENA_FULL;
}

// Longest single timing the autotuner spends on one class sample.
constexpr double kTuneTargetMs = 250.0;

int check_args(const HostBatch &b)
{
    if (b.n_graphs < 0) return MBE_ERR_INVALID_ARG;
    if (b.n_graphs > 0 && (!b.edge_off || !b.nU || !b.nV || !b.u_off_start || !b.v_off_start || !b.u_off_cat ||
                           !b.v_off_cat))
        return MBE_ERR_INVALID_ARG;
    for (int32_t i = 0; i < b.n_graphs; ++i) {
        if (b.nU[i] < 0 || b.nV[i] < 0 || b.u_off_start[i] < 0 || b.v_off_start[i] < 0) return MBE_ERR_INVALID_ARG;
        const int32_t *uo = b.u_off_cat + b.u_off_start[i];
        const int32_t *vo = b.v_off_cat + b.v_off_start[i];
        const int64_t ne = b.edge_off[i + 1] - b.edge_off[i];
        if (ne < 0) return MBE_ERR_INVALID_ARG;
        if (uo[0] != 0 || vo[0] != 0 || (int64_t)uo[b.nU[i]] != ne || (int64_t)vo[b.nV[i]] != ne)
            return MBE_ERR_INVALID_GRAPH;
    }
    return MBE_OK;
}

} // namespace
} // namespace mbe

using namespace mbe;

extern "C" {

int mbe_batch_class(int32_t nU, int32_t nV, int64_t nE) { return class_of(nU, nV, nE); }

int mbe_enumerate_batch(int32_t n_graphs, const int64_t *edge_off, const int32_t *nU, const int32_t *nV,
                        const int64_t *u_off_start, const int64_t *v_off_start, const int32_t *u_off_cat,
                        const int32_t *u_adj_cat, const int32_t *v_off_cat, const int32_t *v_adj_cat,
                        const mbe_options *opts, void *stream, mbe_result *per_graph, mbe_result *total)
{
    if (total) memset(total, 0, sizeof(*total));
    HostBatch b{n_graphs, edge_off, nU, nV, u_off_start, v_off_start, u_off_cat, u_adj_cat, v_off_cat, v_adj_cat};
    int st = check_args(b);
    if (st != MBE_OK) return set_status(total, st);
    if (n_graphs > 0 && !per_graph) return set_status(total, MBE_ERR_INVALID_ARG);
    if (n_graphs == 0) return set_status(total, MBE_OK);
    mbe_options o;
    mbe_default_options(&o);
    if (opts) o = *opts;
    if (o.layout < 0 || o.layout > kLayoutColumns) return set_status(total, MBE_ERR_INVALID_ARG);
    if (o.prune < 0 || o.prune > 1) return set_status(total, MBE_ERR_INVALID_ARG);
    const mbe_class_params *tab = static_cast<const mbe_class_params *>(o.class_params);
    for (int k = 0; tab && k < MBE_N_CLASSES; ++k)
        if (tab[k].valid && (tab[k].layout < 0 || tab[k].layout > kLayoutColumns)) return set_status(total, MBE_ERR_INVALID_ARG);
    cudaStream_t s = (cudaStream_t)stream;
    DeviceBatch d;
    st = upload(b, d, s);
    if (st == MBE_OK && o.prune) {
        // the pruned search: twin classes of every graph (the batch keeps
        // every degree within the bitset limit, so no list path is needed)
        if (cudaMalloc(&d.trep, sizeof(int32_t) * (size_t)std::max<int64_t>(d.n_uoff, 1)) != cudaSuccess) {
            cudaGetLastError();
            d.trep = nullptr;
            st = MBE_ERR_OOM;
        } else {
            cudaError_t e = twin_classes(d.desc, n_graphs, d.max_nU, d.n_uoff, d.uo, d.ua, d.trep, s);
            if (e != cudaSuccess) st = cuda_status(e);
        }
    }
    if (st != MBE_OK) {
        d.release();
        return set_status(total, st);
    }
    std::vector<std::vector<int32_t>> members(MBE_N_CLASSES);
    for (int32_t i = 0; i < n_graphs; ++i)
        members[class_of(nU[i], nV[i], edge_off[i + 1] - edge_off[i])].push_back(i);
    const mbe_class_params *table = static_cast<const mbe_class_params *>(o.class_params);
    std::vector<ClassPlan> plans;
    std::vector<ClassLaunch> cl;
    for (int k = 0; k < MBE_N_CLASSES; ++k) {
        if (members[k].empty()) continue;
        ClassPlan p;
        p.cls = k;
        plan_class(b, d, members[k], p);
        if (p.troot.empty()) continue;
        cl.push_back(launch_for(table ? table + k : nullptr, o, p));
        plans.push_back(std::move(p));
    }
    double ms = 0.0;
    uint64_t don = 0;
    std::vector<double> cms;
    st = plans.empty() ? MBE_OK : run_classes(d, plans, cl, o, s, true, &ms, &don, &cms);
    std::vector<double> ms_of_class(MBE_N_CLASSES, 0.0);
    for (size_t k = 0; k < plans.size() && k < cms.size(); ++k) ms_of_class[plans[k].cls] = cms[k];
    std::vector<unsigned long long> res((size_t)n_graphs * 4, 0);
    if (st == MBE_OK || st == MBE_ERR_TIMEOUT) {
        cudaError_t e = cudaMemcpy(res.data(), d.owner, sizeof(unsigned long long) * 4 * (size_t)n_graphs,
                                   cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) st = cuda_status(e);
    }
    uint64_t c = 0, h = 0, n = 0, by = 0;
    for (int32_t i = 0; i < n_graphs; ++i) {
        mbe_result &r = per_graph[i];
        memset(&r, 0, sizeof(r));
        r.count = res[4 * (size_t)i + 0];
        r.hash = res[4 * (size_t)i + 1];
        r.nodes = res[4 * (size_t)i + 2];
        r.bytes_alg = res[4 * (size_t)i + 3];
        r.device_ms = ms_of_class[class_of(nU[i], nV[i], edge_off[i + 1] - edge_off[i])];
        r.status = st;
        c += r.count;
        h += r.hash;
        n += r.nodes;
        by += r.bytes_alg;
    }
    if (total) {
        total->count = c;
        total->hash = h;
        total->nodes = n;
        total->bytes_alg = by;
        total->device_ms = ms;
        total->n_donations = don;
        total->n_workers = (int32_t)plans.size();
    }
    d.release();
    return set_status(total, st);
}

int mbe_autotune_batch(int32_t n_graphs, const int64_t *edge_off, const int32_t *nU, const int32_t *nV,
                       const int64_t *u_off_start, const int64_t *v_off_start, const int32_t *u_off_cat,
                       const int32_t *u_adj_cat, const int32_t *v_off_cat, const int32_t *v_adj_cat,
                       int32_t sample_per_class, void *stream, mbe_class_params *table)
{
    if (!table || sample_per_class < 1) return MBE_ERR_INVALID_ARG;
    memset(table, 0, sizeof(mbe_class_params) * MBE_N_CLASSES);
    HostBatch b{n_graphs, edge_off, nU, nV, u_off_start, v_off_start, u_off_cat, u_adj_cat, v_off_cat, v_adj_cat};
    int st = check_args(b);
    if (st != MBE_OK || n_graphs == 0) return st;
    cudaStream_t s = (cudaStream_t)stream;
    DeviceBatch d;
    st = upload(b, d, s);
    if (st != MBE_OK) {
        d.release();
        return st;
    }
    mbe_options o;
    mbe_default_options(&o);
    // candidates: (threads, blocks per SM, steal, frame layout) -- 8, 12 and
    // 16 resident warps per SM (the register budget of the search kernels
    // allows 16 at most), work stealing on and off, both frame layouts
    const int cand[][4] = {{256, 1, 1, kLayoutRows},    {128, 3, 1, kLayoutRows},    {256, 2, 1, kLayoutRows},
                           {256, 2, 0, kLayoutRows},    {128, 3, 0, kLayoutRows},    {256, 1, 1, kLayoutColumns},
                           {128, 3, 1, kLayoutColumns}, {256, 2, 1, kLayoutColumns}, {256, 2, 0, kLayoutColumns},
                           {64, 8, 1, kLayoutRows},     {512, 1, 1, kLayoutRows}};
    const int n_cand = (int)(sizeof(cand) / sizeof(cand[0]));
    std::vector<std::vector<int32_t>> members(MBE_N_CLASSES);
    for (int32_t i = 0; i < n_graphs; ++i)
        members[class_of(nU[i], nV[i], edge_off[i + 1] - edge_off[i])].push_back(i);
    for (int k = 0; k < MBE_N_CLASSES && st == MBE_OK; ++k) {
        if (members[k].empty()) continue;
        ClassPlan full;
        full.cls = k;
        plan_class(b, d, members[k], full);
        if (full.troot.empty()) continue;
        // the sample: every step-th (graph, root) task of the class in its
        // heavy-first order, about sample_per_class tasks per default worker
        // (or the whole class), thinned by halves while one run of the default
        // shape takes more than kTuneTargetMs, so that a class of heavy roots
        // is tuned in seconds and not in minutes
        const LaunchShape def = shape_for(0, 0, kLayoutColumns);
        const int64_t want = (int64_t)sample_per_class * def.warps;
        const int64_t nt = (int64_t)full.troot.size();
        int64_t step = std::max<int64_t>(1, nt / std::max<int64_t>(want, 1));
        std::vector<ClassPlan> plans(1);
        ClassPlan &p = plans[0];
        auto take = [&](int64_t stp) {
            p = full;
            p.troot.clear();
            p.tgraph.clear();
            for (int64_t t = 0; t < nt; t += stp) {
                p.troot.push_back(full.troot[t]);
                p.tgraph.push_back(full.tgraph[t]);
            }
        };
        take(step);
        auto time_of = [&](const mbe_class_params &prm, double *out) {
            std::vector<ClassLaunch> cl(1, launch_for(&prm, o, p));
            return run_classes(d, plans, cl, o, s, false, out, nullptr);
        };
        const mbe_class_params dflt{0, 0, 1, 1, 0, 0, 0.0};
        double t_def = 0.0;
        st = time_of(dflt, &t_def); // also sizes the workspace
        if (st == MBE_OK) st = time_of(dflt, &t_def);
        while (st == MBE_OK && t_def > kTuneTargetMs && (int64_t)p.troot.size() >= 2LL * def.warps) {
            step *= 2;
            take(step);
            st = time_of(dflt, &t_def);
        }
        // every candidate once on the sample, then the two fastest again
        std::vector<std::pair<double, int>> res;
        for (int c = 0; c < n_cand && st == MBE_OK; ++c) {
            mbe_class_params prm{cand[c][0], cand[c][1], cand[c][2], 1, cand[c][3], 0, 0.0};
            if (launch_for(&prm, o, p).shape.threads != prm.block_threads) continue; // not on this device
            double ms = 0.0;
            st = time_of(prm, &ms);
            if (st == MBE_OK) res.push_back({ms, c});
        }
        std::sort(res.begin(), res.end());
        double best = 1e300;
        for (size_t r = 0; r < res.size() && r < 2 && st == MBE_OK; ++r) {
            const int c = res[r].second;
            mbe_class_params prm{cand[c][0], cand[c][1], cand[c][2], 1, cand[c][3], 0, 0.0};
            double ms = 0.0;
            st = time_of(prm, &ms);
            ms = std::min(ms, res[r].first);
            if (st == MBE_OK && ms < best) {
                best = ms;
                table[k] = prm;
                table[k].tuned_ms = ms;
            }
        }
        table[k].default_ms = t_def;
    }
    d.release();
    return st;
}

} // extern "C"
