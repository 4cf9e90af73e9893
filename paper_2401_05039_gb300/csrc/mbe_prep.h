// Host launchers of the preprocessing kernels (internal).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "mbe_internal.h"

namespace mbe {

// ORs a nonzero code into *d_bad when the CSR/CSC pair is malformed.
cudaError_t validate_graph(const int32_t *u_off, const int32_t *u_adj, const int32_t *v_off, const int32_t *v_adj,
                           int32_t nU, int32_t nV, int64_t nE, int32_t *d_bad, cudaStream_t s);

// Every graph of a concatenated batch checked in one launch (ORs into *d_bad).
cudaError_t validate_batch(const GraphDesc *d_graphs, int32_t n_graphs, const int32_t *u_off, const int32_t *u_adj,
                           const int32_t *v_off, const int32_t *v_adj, int32_t *d_bad, cudaStream_t s);

// d_out[4g..4g+3] (zeroed by the caller): max candidates, universe bytes,
// level-1 frame bytes and degree over the roots of graph g.
cudaError_t graph_bounds(const GraphDesc *d_graphs, int32_t n_graphs, const int32_t *u_off, const int32_t *u_adj,
                         const int32_t *v_off, unsigned long long *d_out, cudaStream_t s);

// *d_out = max(*d_out, largest list length of the CSR off[0..n]).
cudaError_t max_degree(const int32_t *off, int32_t n, int32_t *d_out, cudaStream_t s);

// Workspace bounds over all roots of all graphs; d_out[5] must be zeroed.
cudaError_t root_bounds(const GraphDesc *d_graphs, int32_t n_graphs, int32_t max_nU, const int32_t *u_off,
                        const int32_t *u_adj, const int32_t *v_off, unsigned long long *d_out, cudaStream_t s);

// d_order receives the non-isolated U vertices by descending degree.
// d_hist needs max_deg + 1 entries.
cudaError_t order_by_degree_desc(const int32_t *u_off, int32_t nU, int32_t max_deg, int32_t *d_hist,
                                 int32_t *d_order, cudaStream_t s);

// d_hist[d] = number of non-isolated U vertices with degree > d (max_deg + 1 entries).
cudaError_t degree_larger(const int32_t *u_off, int32_t nU, int32_t max_deg, int32_t *d_hist, cudaStream_t s);

// d_order receives every u with d_key[u] >= 0, by descending key (keys <= max_key).
cudaError_t order_by_key_desc(const int32_t *d_key, int32_t n, int32_t max_key, int32_t *d_hist, int32_t *d_order,
                              cudaStream_t s);

// Top-level twin classes of the pruned search, for every graph of a
// (possibly one-graph) batch: d_trep[u_off_base + u] = the smallest local U
// id of the graph whose neighbourhood equals N(u) (u itself when there is
// none, and for an isolated u). n_uoff = entries of the concatenated u_off
// (d_trep has as many). Allocates and frees its own table; synchronises s.
cudaError_t twin_classes(const GraphDesc *d_graphs, int32_t n_graphs, int32_t max_nU, int64_t n_uoff,
                         const int32_t *u_off, const int32_t *u_adj, int32_t *d_trep, cudaStream_t s);

} // namespace mbe
