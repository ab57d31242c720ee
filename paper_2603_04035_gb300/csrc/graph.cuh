// Internal interface of the fuzzy-graph builder.
#pragma once
#include "common.cuh"

namespace drgb {

size_t fuzzy_scratch_bytes(int64_t n, int k);
int build_fuzzy_graph(Ctx* c, const int32_t* idx, const float* dist, int64_t n, int k, int T,
                      int32_t* row_ptr, int32_t* col, float* w, uint32_t* q, float* rho,
                      float* sigma, void* scratch, cudaStream_t st);

}  // namespace drgb
