// Internal interface of the fuzzy-graph builder.
#pragma once
#include "common.cuh"

namespace drgb {

size_t fuzzy_scratch_bytes(int64_t n, int k);
// Directed memberships w_{j|i} of n query rows whose k neighbours are indices
// into a separate set of db_n points; out_col/out_w are the rows sorted by column.
int launch_directed_weights(Ctx* c, const int32_t* idx, const float* dist, int64_t n, int k, int64_t db_n,
                            float* w_dir, int32_t* out_col, float* out_w, cudaStream_t st);
int build_fuzzy_graph(Ctx* c, const int32_t* idx, const float* dist, int64_t n, int k, int T,
                      int32_t* row_ptr, int32_t* col, float* w, uint32_t* q, float* rho,
                      float* sigma, void* scratch, cudaStream_t st);

}  // namespace drgb
