// NNDescent approximate k-NN graph (nndescent.cu), for drgb_knn_nndescent and
// the fit's knn_mode 4.
#pragma once
#include "common.cuh"

namespace drgb {

static constexpr int NND_MAX_ITER = 1000;
static constexpr int NND_MAX_D = 1024;
static constexpr double NND_DELTA = 0.015;  // the early-termination update rate
static constexpr int NND_ITER_DEFAULT = 30;

size_t nnd_scratch_bytes(int64_t n, int k, bool reverse);

// The graph (idx n x k, Euclidean dist n x k, rows in (distance, index)
// order), the reverse form (k <= 16) when `reverse`; iters_out (host,
// nullable) receives the iterations run and
// rates_out (host, nullable, max_iter entries) each iteration's update rate.
// Arguments as checked by drgb_knn_nndescent; synchronises the stream once
// per iteration.
int nnd_run(Ctx* c, const float* X, int64_t n, int d, int k, uint64_t seed, double delta, int max_iter, bool reverse,
            int32_t* idx_out, float* dist_out, int32_t* iters_out, double* rates_out, void* scratch,
            cudaStream_t st);

}  // namespace drgb
