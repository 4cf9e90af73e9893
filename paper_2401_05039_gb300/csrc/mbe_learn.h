// Internal launchers of the learned-schedule kernels.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/mbe.h"

namespace mbe {

// Core numbers of G as a general graph (U vertices 0..nU-1, then V); d_deg,
// d_alive, d_core hold nU + nV entries, d_removed one.
cudaError_t compute_core_numbers(const int32_t *u_off, const int32_t *u_adj, const int32_t *v_off,
                                 const int32_t *v_adj, int32_t nU, int32_t nV, int32_t *d_deg, int32_t *d_alive,
                                 int32_t *d_core, int32_t *d_removed, cudaStream_t s);

// Raw ([nU][8] int32) and float ([nU][8]) root features. d_larger[d] = number
// of U vertices with degree > d; d_mark: n_warps stamp arrays of mark_stride.
cudaError_t compute_root_features(const int32_t *u_off, const int32_t *u_adj, const int32_t *v_off,
                                  const int32_t *v_adj, int32_t nU, const int32_t *d_larger, const int32_t *d_core,
                                  int32_t *d_mark, int64_t mark_stride, int32_t n_warps, int32_t *d_raw,
                                  float *d_feat, cudaStream_t s);

// Order keys from predicted log costs (-1 for isolated roots).
cudaError_t learned_order_keys(const float *d_pred, const int32_t *u_off, int32_t nU, int32_t max_key,
                               int32_t *d_key, int32_t *d_bad, cudaStream_t s);

cudaError_t model_predict(const mbe_model *md, const float *d_feat, int32_t n, float *d_out, cudaStream_t s);

} // namespace mbe
