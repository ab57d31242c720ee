// Internal interface of the spectral initial layout (spectral.cu).
#pragma once
#include "common.cuh"

namespace drgb {

// Bytes of scratch spectral_layout needs for n rows and nnz_cap CSR entries.
size_t spectral_scratch_bytes(int64_t n, int64_t nnz_cap, int num_sms);

// Y = the spectral layout of the CSR graph (row_ptr, col, w), scaled to
// init_range with the initialisation stream's jitter (key seed); the three
// leading eigenvalues of the normalised adjacency go to eig_out (host, may be
// null).  Synchronises `st` once per subspace step.
int spectral_layout(Ctx* c, const int32_t* rp, const int32_t* col, const float* w, int64_t n, int64_t nnz_cap,
                    float init_range, uint64_t seed, float2* Y, double* eig_out, void* scratch, cudaStream_t st);

}  // namespace drgb
