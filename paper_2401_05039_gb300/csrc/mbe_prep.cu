// Preprocessing kernels: input validation, per-root workspace bounds and the
// static execution order of the roots.
#include "mbe_bits.h"
#include "mbe_internal.h"
#include "mbe_prep.h"

#include <algorithm>

namespace mbe {
namespace {

// CSR well-formedness: offsets start at 0, end at nE and never decrease;
// every list strictly increasing (sorted, no duplicates) with ids in
// [0, n_other). One thread per vertex.
__global__ void validate_csr_kernel(const int32_t *off, const int32_t *adj, int32_t n, int32_t n_other, int64_t nE,
                                    int32_t *bad)
{
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i <= n; i += stride) {
        if (i == 0 && off[0] != 0) atomicOr(bad, 1);
        if (i == n) {
            if ((int64_t)off[n] != nE) atomicOr(bad, 2);
            continue;
        }
        int a = off[i], b = off[i + 1];
        if (b < a || a < 0 || (int64_t)b > nE) {
            atomicOr(bad, 4);
            continue;
        }
        int prev = -1;
        for (int k = a; k < b; ++k) {
            int x = adj[k];
            if (x <= prev || x >= n_other) {
                atomicOr(bad, 8);
                break;
            }
            prev = x;
        }
    }
}

// Every (u, v) of the U-side CSR appears in N(v) of the V-side CSR. With
// both forms duplicate-free and of equal size, this makes them transposes.
// It runs on the same stream right after the CSR checks, before anyone has
// read their verdict, so it trusts nothing: an offset outside [0, nE] or
// out of order, or an id outside its side, is reported and never used as an
// index.
__global__ void validate_transpose_kernel(const int32_t *u_off, const int32_t *u_adj, const int32_t *v_off,
                                          const int32_t *v_adj, int32_t nU, int32_t nV, int64_t nE, int32_t *bad)
{
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < nU; u += stride) {
        const int a = u_off[u], b = u_off[u + 1];
        if (a < 0 || b < a || (int64_t)b > nE) {
            atomicOr(bad, 4);
            continue;
        }
        for (int k = a; k < b; ++k) {
            const int v = u_adj[k];
            if (v < 0 || v >= nV) {
                atomicOr(bad, 8);
                break;
            }
            const int vlo = v_off[v], vhi = v_off[v + 1];
            if (vlo < 0 || vhi < vlo || (int64_t)vhi > nE) {
                atomicOr(bad, 4);
                break;
            }
            int lo = vlo, hi = vhi;
            while (lo < hi) {
                int mid = lo + ((hi - lo) >> 1);
                if (v_adj[mid] < u) lo = mid + 1;
                else hi = mid;
            }
            if (lo >= vhi || v_adj[lo] != (int32_t)u) {
                atomicOr(bad, 16);
                break;
            }
        }
    }
}

// Per-root bounds of the search workspace. For root r with d = |N(r)|, its
// local universe has at most nc = min(sum_{w in N(r)} (|N(w)| - 1), nU - 1)
// candidates, rows of W = ceil(d/64) words, and the level-1 frame holds at
// most nc rows. out: [0] max nc, [1] max universe row bytes, [2] max level-1
// frame bytes, [3] max degree, [4] number of non-isolated roots.
__global__ void root_bounds_kernel(const GraphDesc *graphs, int32_t n_graphs, const int32_t *u_off_cat,
                                   const int32_t *u_adj_cat, const int32_t *v_off_cat, unsigned long long *out)
{
    int g = blockIdx.y;
    if (g >= n_graphs) return;
    GraphDesc G = graphs[g];
    const int32_t *u_off = u_off_cat + G.u_off_base;
    const int32_t *v_off = v_off_cat + G.v_off_base;
    const int32_t *u_adj = u_adj_cat + G.edge_base;
    unsigned long long m_nc = 0, m_urow = 0, m_frame = 0, m_deg = 0, live = 0;
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < G.nU; r += gridDim.x * blockDim.x) {
        int a = u_off[r], d = u_off[r + 1] - a;
        if (d == 0) continue;
        long long s = 0;
        for (int k = 0; k < d; ++k) {
            int w = u_adj[a + k];
            s += v_off[w + 1] - v_off[w] - 1;
        }
        long long nc = s < (long long)G.nU - 1 ? s : (long long)G.nU - 1;
        unsigned long long urow = (unsigned long long)universe_rows_bound(d, nc);
        unsigned long long frame = (unsigned long long)level1_frame_bound(d, nc);
        m_nc = max(m_nc, (unsigned long long)nc);
        m_urow = max(m_urow, urow);
        m_frame = max(m_frame, frame);
        m_deg = max(m_deg, (unsigned long long)d);
        live += 1;
    }
    atomicMax(out + 0, m_nc);
    atomicMax(out + 1, m_urow);
    atomicMax(out + 2, m_frame);
    atomicMax(out + 3, m_deg);
    atomicAdd(out + 4, live);
}

__global__ void degree_hist_kernel(const int32_t *u_off, int32_t nU, int32_t *hist)
{
    for (int u = blockIdx.x * blockDim.x + threadIdx.x; u < nU; u += gridDim.x * blockDim.x) {
        int d = u_off[u + 1] - u_off[u];
        if (d > 0) atomicAdd(hist + d, 1);
    }
}

// Exclusive scan of hist[0..n) from the top bin down (descending keys first),
// one block, in place: hist[b] = number of items with key > b.
__global__ void scan_desc_kernel(int32_t *hist, int32_t n)
{
    __shared__ int32_t carry;
    __shared__ int32_t part[1024];
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int base = n - 1; base >= 0; base -= blockDim.x) {
        int b = base - (int)threadIdx.x;
        int v = b >= 0 ? hist[b] : 0;
        part[threadIdx.x] = v;
        __syncthreads();
        for (int o = 1; o < (int)blockDim.x; o <<= 1) {
            int y = threadIdx.x >= (unsigned)o ? part[threadIdx.x - o] : 0;
            __syncthreads();
            part[threadIdx.x] += y;
            __syncthreads();
        }
        int excl = part[threadIdx.x] - v + carry;
        if (b >= 0) hist[b] = excl;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry += part[threadIdx.x];
        __syncthreads();
    }
}

__global__ void scatter_by_degree_kernel(const int32_t *u_off, int32_t nU, int32_t *pos, int32_t *order)
{
    for (int u = blockIdx.x * blockDim.x + threadIdx.x; u < nU; u += gridDim.x * blockDim.x) {
        int d = u_off[u + 1] - u_off[u];
        if (d > 0) order[atomicAdd(pos + d, 1)] = u;
    }
}

// Roots ordered by a non-negative integer key, descending (ties in any order).
__global__ void key_hist_kernel(const int32_t *key, int32_t n, int32_t *hist)
{
    for (int u = blockIdx.x * blockDim.x + threadIdx.x; u < n; u += gridDim.x * blockDim.x)
        if (key[u] >= 0) atomicAdd(hist + key[u], 1);
}

__global__ void key_scatter_kernel(const int32_t *key, int32_t n, int32_t *pos, int32_t *order)
{
    for (int u = blockIdx.x * blockDim.x + threadIdx.x; u < n; u += gridDim.x * blockDim.x)
        if (key[u] >= 0) order[atomicAdd(pos + key[u], 1)] = u;
}

// Batched validation: grid.y = graph. Same checks as validate_csr_kernel and
// validate_transpose_kernel for every graph of a concatenated batch.
__global__ void validate_batch_kernel(const GraphDesc *graphs, const int32_t *u_off_cat, const int32_t *u_adj_cat,
                                      const int32_t *v_off_cat, const int32_t *v_adj_cat, int32_t *bad)
{
    const GraphDesc G = graphs[blockIdx.y];
    const int32_t *uo = u_off_cat + G.u_off_base, *vo = v_off_cat + G.v_off_base;
    const int32_t *ua = u_adj_cat + G.edge_base, *va = v_adj_cat + G.edge_base;
    const int t = blockIdx.x * blockDim.x + threadIdx.x, stride = gridDim.x * blockDim.x;
    if (t == 0 && (uo[0] != 0 || vo[0] != 0 || uo[G.nU] != vo[G.nV])) atomicOr(bad, 1);
    const int nE = uo[G.nU];
    for (int u = t; u < G.nU; u += stride) {
        int a = uo[u], b = uo[u + 1], prev = -1;
        if (b < a || a < 0 || b > nE) {
            atomicOr(bad, 4);
            continue;
        }
        for (int k = a; k < b; ++k) {
            int v = ua[k];
            if (v <= prev || v >= G.nV) {
                atomicOr(bad, 8);
                break;
            }
            prev = v;
            int lo = vo[v], hi = vo[v + 1];
            while (lo < hi) {
                int mid = lo + ((hi - lo) >> 1);
                if (va[mid] < u) lo = mid + 1;
                else hi = mid;
            }
            if (lo >= vo[v + 1] || va[lo] != u) {
                atomicOr(bad, 16);
                break;
            }
        }
    }
    for (int v = t; v < G.nV; v += stride) {
        int a = vo[v], b = vo[v + 1], prev = -1;
        if (b < a || a < 0 || b > nE) {
            atomicOr(bad, 4);
            continue;
        }
        for (int k = a; k < b; ++k) {
            if (va[k] <= prev || va[k] >= G.nU) {
                atomicOr(bad, 8);
                break;
            }
            prev = va[k];
        }
    }
}

// Per-graph workspace bounds: out[4g..4g+3] = max over the roots of graph g
// of (candidates, universe row bytes, level-1 frame bytes, degree); same
// per-root bounds as root_bounds_kernel.
__global__ void graph_bounds_kernel(const GraphDesc *graphs, const int32_t *u_off_cat, const int32_t *u_adj_cat,
                                    const int32_t *v_off_cat, unsigned long long *out)
{
    const int g = blockIdx.y;
    const GraphDesc G = graphs[g];
    const int32_t *u_off = u_off_cat + G.u_off_base, *v_off = v_off_cat + G.v_off_base;
    const int32_t *u_adj = u_adj_cat + G.edge_base;
    unsigned long long m_nc = 0, m_urow = 0, m_frame = 0, m_deg = 0;
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < G.nU; r += gridDim.x * blockDim.x) {
        int a = u_off[r], d = u_off[r + 1] - a;
        if (d == 0) continue;
        long long s = 0;
        for (int k = 0; k < d; ++k) {
            int w = u_adj[a + k];
            s += v_off[w + 1] - v_off[w] - 1;
        }
        long long nc = s < (long long)G.nU - 1 ? s : (long long)G.nU - 1;
        unsigned long long urow = (unsigned long long)universe_rows_bound(d, nc);
        unsigned long long frame = (unsigned long long)level1_frame_bound(d, nc);
        m_nc = max(m_nc, (unsigned long long)nc);
        m_urow = max(m_urow, urow);
        m_frame = max(m_frame, frame);
        m_deg = max(m_deg, (unsigned long long)d);
    }
    atomicMax(out + 4LL * g + 0, m_nc);
    atomicMax(out + 4LL * g + 1, m_urow);
    atomicMax(out + 4LL * g + 2, m_frame);
    atomicMax(out + 4LL * g + 3, m_deg);
}

__global__ void max_degree_kernel(const int32_t *off, int32_t n, int32_t *out)
{
    int m = 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        m = max(m, off[i + 1] - off[i]);
    atomicMax(out, m);
}

// Top-level twin classes for the pruned search: U vertices of one graph
// with the same neighbourhood. A digest of (graph, degree, sorted list)
// keys an open-addressing table (2^k >= 2 entries per vertex, linear
// probing) that keeps the smallest index of each key; every vertex then
// compares its list with that vertex's list, so a digest collision only
// costs pruning (the vertex keeps itself as representative), never a
// wrong removal. Indices are those of the concatenated u_off (graph base +
// local id), one grid row per graph.
__device__ __forceinline__ unsigned long long twin_digest(int g, const int32_t *adj, int d)
{
    unsigned long long h = splitmix(((unsigned long long)(uint32_t)g << 32) | (unsigned long long)(uint32_t)d);
    for (int k = 0; k < d; ++k) h = splitmix(h ^ (unsigned long long)(uint32_t)adj[k]);
    return h | 1ULL; // 0 marks an empty slot
}

__global__ void twin_fill_kernel(int32_t *minid, int64_t T)
{
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < T; t += (int64_t)gridDim.x * blockDim.x)
        minid[t] = 0x7fffffff;
}

__global__ void twin_insert_kernel(const GraphDesc *graphs, int32_t n_graphs, const int32_t *u_off_cat,
                                   const int32_t *u_adj_cat, unsigned long long *keys, int32_t *minid, int64_t T,
                                   int32_t *slot_of)
{
    const int g = blockIdx.y;
    if (g >= n_graphs) return;
    const GraphDesc G = graphs[g];
    const int32_t *u_off = u_off_cat + G.u_off_base;
    const int32_t *u_adj = u_adj_cat + G.edge_base;
    for (int u = blockIdx.x * blockDim.x + threadIdx.x; u < G.nU; u += gridDim.x * blockDim.x) {
        const int64_t p = G.u_off_base + u;
        const int o = u_off[u], d = u_off[u + 1] - o;
        slot_of[p] = -1;
        if (d == 0) continue;
        const unsigned long long h = twin_digest(g, u_adj + o, d);
        int64_t slot = (int64_t)(h & (unsigned long long)(T - 1));
        for (int64_t t = 0; t < T; ++t) { // fewer keys than T / 2: a free slot is always found
            const unsigned long long prev = atomicCAS(keys + slot, 0ULL, h);
            if (prev == 0ULL || prev == h) {
                atomicMin(minid + slot, (int32_t)p);
                slot_of[p] = (int32_t)slot;
                break;
            }
            slot = (slot + 1) & (T - 1);
        }
    }
}

__global__ void twin_rep_kernel(const GraphDesc *graphs, int32_t n_graphs, const int32_t *u_off_cat,
                                const int32_t *u_adj_cat, const int32_t *minid, const int32_t *slot_of,
                                int32_t *trep)
{
    const int g = blockIdx.y;
    if (g >= n_graphs) return;
    const GraphDesc G = graphs[g];
    const int32_t *u_off = u_off_cat + G.u_off_base;
    const int32_t *u_adj = u_adj_cat + G.edge_base;
    for (int u = blockIdx.x * blockDim.x + threadIdx.x; u < G.nU; u += gridDim.x * blockDim.x) {
        const int64_t p = G.u_off_base + u;
        int r = u;
        if (slot_of[p] >= 0) {
            const int64_t cp = minid[slot_of[p]];
            const int64_t c = cp - G.u_off_base; // a local id when the vertex is of this graph
            if (c >= 0 && c < u) {
                const int o = u_off[u], d = u_off[u + 1] - o;
                const int oc = u_off[c], dc = u_off[c + 1] - oc;
                bool same = dc == d;
                for (int k = 0; same && k < d; ++k) same = u_adj[o + k] == u_adj[oc + k];
                if (same) r = (int)c;
            }
        }
        trep[p] = r;
    }
}

} // namespace

cudaError_t validate_batch(const GraphDesc *d_graphs, int32_t n_graphs, const int32_t *u_off, const int32_t *u_adj,
                           const int32_t *v_off, const int32_t *v_adj, int32_t *d_bad, cudaStream_t s)
{
    for (int32_t g0 = 0; g0 < n_graphs; g0 += 65535) {
        dim3 grid(2, std::min<int32_t>(65535, n_graphs - g0));
        validate_batch_kernel<<<grid, 256, 0, s>>>(d_graphs + g0, u_off, u_adj, v_off, v_adj, d_bad);
    }
    return cudaGetLastError();
}

cudaError_t graph_bounds(const GraphDesc *d_graphs, int32_t n_graphs, const int32_t *u_off, const int32_t *u_adj,
                         const int32_t *v_off, unsigned long long *d_out, cudaStream_t s)
{
    for (int32_t g0 = 0; g0 < n_graphs; g0 += 65535) {
        dim3 grid(2, std::min<int32_t>(65535, n_graphs - g0));
        graph_bounds_kernel<<<grid, 256, 0, s>>>(d_graphs + g0, u_off, u_adj, v_off, d_out + 4LL * g0);
    }
    return cudaGetLastError();
}

cudaError_t max_degree(const int32_t *off, int32_t n, int32_t *d_out, cudaStream_t s)
{
    int blocks = (n + 255) / 256;
    if (blocks > 4 * 152) blocks = 4 * 152;
    if (blocks < 1) blocks = 1;
    max_degree_kernel<<<blocks, 256, 0, s>>>(off, n, d_out);
    return cudaGetLastError();
}

cudaError_t validate_graph(const int32_t *u_off, const int32_t *u_adj, const int32_t *v_off, const int32_t *v_adj,
                           int32_t nU, int32_t nV, int64_t nE, int32_t *d_bad, cudaStream_t s)
{
    int blocks = 2 * 152, threads = 256;
    validate_csr_kernel<<<blocks, threads, 0, s>>>(u_off, u_adj, nU, nV, nE, d_bad);
    validate_csr_kernel<<<blocks, threads, 0, s>>>(v_off, v_adj, nV, nU, nE, d_bad);
    validate_transpose_kernel<<<blocks, threads, 0, s>>>(u_off, u_adj, v_off, v_adj, nU, nV, nE, d_bad);
    return cudaGetLastError();
}

cudaError_t root_bounds(const GraphDesc *d_graphs, int32_t n_graphs, int32_t max_nU, const int32_t *u_off,
                        const int32_t *u_adj, const int32_t *v_off, unsigned long long *d_out, cudaStream_t s)
{
    int gx = (max_nU + 255) / 256;
    if (gx > 64) gx = 64;
    if (gx < 1) gx = 1;
    dim3 grid(gx, n_graphs);
    root_bounds_kernel<<<grid, 256, 0, s>>>(d_graphs, n_graphs, u_off, u_adj, v_off, d_out);
    return cudaGetLastError();
}

cudaError_t order_by_degree_desc(const int32_t *u_off, int32_t nU, int32_t max_deg, int32_t *d_hist,
                                 int32_t *d_order, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(d_hist, 0, sizeof(int32_t) * (size_t)(max_deg + 1), s);
    if (e != cudaSuccess) return e;
    int blocks = (nU + 255) / 256;
    if (blocks > 4 * 152) blocks = 4 * 152;
    if (blocks < 1) blocks = 1;
    degree_hist_kernel<<<blocks, 256, 0, s>>>(u_off, nU, d_hist);
    scan_desc_kernel<<<1, 1024, 0, s>>>(d_hist, max_deg + 1);
    scatter_by_degree_kernel<<<blocks, 256, 0, s>>>(u_off, nU, d_hist, d_order);
    return cudaGetLastError();
}

cudaError_t degree_larger(const int32_t *u_off, int32_t nU, int32_t max_deg, int32_t *d_hist, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(d_hist, 0, sizeof(int32_t) * (size_t)(max_deg + 1), s);
    if (e != cudaSuccess) return e;
    int blocks = (nU + 255) / 256;
    if (blocks > 4 * 152) blocks = 4 * 152;
    if (blocks < 1) blocks = 1;
    degree_hist_kernel<<<blocks, 256, 0, s>>>(u_off, nU, d_hist);
    scan_desc_kernel<<<1, 1024, 0, s>>>(d_hist, max_deg + 1);
    return cudaGetLastError();
}

cudaError_t order_by_key_desc(const int32_t *d_key, int32_t n, int32_t max_key, int32_t *d_hist, int32_t *d_order,
                              cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(d_hist, 0, sizeof(int32_t) * (size_t)(max_key + 1), s);
    if (e != cudaSuccess) return e;
    int blocks = (n + 255) / 256;
    if (blocks > 4 * 152) blocks = 4 * 152;
    if (blocks < 1) blocks = 1;
    key_hist_kernel<<<blocks, 256, 0, s>>>(d_key, n, d_hist);
    scan_desc_kernel<<<1, 1024, 0, s>>>(d_hist, max_key + 1);
    key_scatter_kernel<<<blocks, 256, 0, s>>>(d_key, n, d_hist, d_order);
    return cudaGetLastError();
}

cudaError_t twin_classes(const GraphDesc *d_graphs, int32_t n_graphs, int32_t max_nU, int64_t n_uoff,
                         const int32_t *u_off, const int32_t *u_adj, int32_t *d_trep, cudaStream_t s)
{
    if (n_uoff >= 0x7fffffffLL) return cudaErrorInvalidValue; // indices are int32
    int64_t T = 2;
    while (T < 2 * n_uoff) T <<= 1;
    unsigned long long *keys = nullptr;
    int32_t *minid = nullptr, *slot_of = nullptr;
    cudaError_t e = cudaMalloc(&keys, sizeof(unsigned long long) * (size_t)T);
    if (e == cudaSuccess) e = cudaMalloc(&minid, sizeof(int32_t) * (size_t)T);
    if (e == cudaSuccess) e = cudaMalloc(&slot_of, sizeof(int32_t) * (size_t)std::max<int64_t>(n_uoff, 1));
    if (e == cudaSuccess) e = cudaMemsetAsync(keys, 0, sizeof(unsigned long long) * (size_t)T, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(slot_of, 0xff, sizeof(int32_t) * (size_t)std::max<int64_t>(n_uoff, 1), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_trep, 0, sizeof(int32_t) * (size_t)std::max<int64_t>(n_uoff, 1), s);
    if (e == cudaSuccess) {
        const int fill = (int)std::min<int64_t>((T + 255) / 256, 4 * 152);
        int gx = (max_nU + 255) / 256;
        gx = std::max(1, std::min(gx, 64));
        const dim3 grid(gx, n_graphs);
        twin_fill_kernel<<<fill, 256, 0, s>>>(minid, T);
        twin_insert_kernel<<<grid, 256, 0, s>>>(d_graphs, n_graphs, u_off, u_adj, keys, minid, T, slot_of);
        twin_rep_kernel<<<grid, 256, 0, s>>>(d_graphs, n_graphs, u_off, u_adj, minid, slot_of, d_trep);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(keys);
    cudaFree(minid);
    cudaFree(slot_of);
    return e;
}

} // namespace mbe
