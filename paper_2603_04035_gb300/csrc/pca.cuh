// PCA preprocessing (pca.cu), for the fit's optional pca_dim step.
#pragma once
#include "common.cuh"

namespace drgb {

static constexpr int PCA_MAX_DIM = 56;   // components at most (the subspace block is 64)
static constexpr int PCA_MAX_FEATURES = 1024;

// Scratch bytes of pca_run for n rows of D features.
size_t pca_scratch_bytes(int64_t n, int D);

// Z (n x dim) = the projection of X (n x D) on its dim leading principal
// components; comps (dim x D), mu (D) and eig (host, dim) are optional.
// Arguments as checked by drgb_pca; synchronises the stream.
int pca_run(Ctx* c, const float* X, int64_t n, int D, int dim, float* Z, float* comps, float* mu_out,
            double* eig_out, void* scratch, cudaStream_t st);

}  // namespace drgb
