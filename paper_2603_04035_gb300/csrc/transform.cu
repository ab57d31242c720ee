// Plain-optimisation embedding of new points against a fixed embedding of
// training points (the fallback of the learned embedder, and the judge of its
// recall): each new point gets its exact k nearest training points, their
// directed memberships w_{j|i} (the per-row rho / sigma construction of the
// fuzzy graph), a start at the w-weighted mean of those neighbours' training
// coordinates, and ceil(T / 3) synchronous epochs in which only the new points
// move: attraction along their k entries, negatives drawn from the training
// embedding, lr_t = lr0 (1 - t / T').  The training embedding never changes.
#include "common.cuh"
#include "epoch.cuh"
#include "graph.cuh"
#include "knn.cuh"

namespace drgb {

// Schedule words of the new rows (w_max = 1: every row's nearest neighbour has
// membership 1) and the start positions.
__global__ void transform_setup_kernel(const int32_t* __restrict__ out_col, const float* __restrict__ out_w,
                                       int64_t n_new, int k, const float2* __restrict__ Y_train,
                                       uint32_t* __restrict__ q, float2* __restrict__ Y_new_a,
                                       float2* __restrict__ Y_new_b) {
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n_new;
         i += int64_t(gridDim.x) * blockDim.x) {
        float sx = 0.f, sy = 0.f, sw = 0.f;
        for (int s = 0; s < k; ++s) {
            const float w = out_w[i * k + s];
            const float2 y = Y_train[out_col[i * k + s]];
            sx = fmaf(w, y.x, sx);
            sy = fmaf(w, y.y, sy);
            sw += w;
            q[i * k + s] = __float2uint_rn(16777216.0f * w);
        }
        const float2 y0 = make_float2(sx / sw, sy / sw);
        Y_new_a[i] = y0;
        Y_new_b[i] = y0;
    }
}

__global__ void arange_kernel(int32_t* __restrict__ rp, int64_t n, int k) {
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i <= n; i += int64_t(gridDim.x) * blockDim.x)
        rp[i] = int32_t(i * k);
}

}  // namespace drgb

using namespace drgb;

extern "C" int drgb_transform(drgb_ctx* c, const float* X_train, const float* Y_train, int64_t n_train,
                              const float* X_new, int64_t n_new, int32_t d, const drgb_params* p, float* Y_new,
                              void* stream) {
    if (!c) return DRGB_ERR_INVALID;
    if (!X_train || !Y_train || !X_new || !p || !Y_new || n_new < 1 || d < 1 || !aligned(X_train, 4) ||
        !aligned(X_new, 4) || !aligned(Y_train, 8) || !aligned(Y_new, 8))
        return set_error(c, DRGB_ERR_INVALID, "transform: bad pointers or sizes");
    const int k = p->k;
    if (k < 1 || k > DRGB_MAX_K || n_train < k + 1 || n_train + n_new > INT32_MAX / 2 || p->n_epochs < 1 ||
        p->neg < 0 || p->neg > 64)
        return set_error(c, DRGB_ERR_INVALID, "transform: bad parameters");
    if (p->pca_dim != 0)
        return set_error(c, DRGB_ERR_INVALID, "transform: pca_dim is not supported (project X_new first)");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int64_t N = n_train + n_new;
    const size_t nk = size_t(n_new) * k;
    const size_t bytes = 4 * Carve::round(nk * 4) + Carve::round(nk * 4) + Carve::round((n_new + 1) * 4) +
                         2 * Carve::round(size_t(N) * 8) + Carve::round(epoch_scratch_bytes(N, int64_t(nk), 0)) + 4096;
    int rc = ensure_scratch(c, bytes, st);
    if (rc) return rc;
    Carve cv(c->scratch);
    int32_t* idx = cv.take<int32_t>(nk);
    float* dist = cv.take<float>(nk);
    float* w_dir = cv.take<float>(nk);
    int32_t* out_col = cv.take<int32_t>(nk);
    float* out_w = cv.take<float>(nk);
    uint32_t* q = reinterpret_cast<uint32_t*>(w_dir);  // the directed weights are no longer needed
    int32_t* rp = cv.take<int32_t>(n_new + 1);
    float2* Ya = cv.take<float2>(N);
    float2* Yb = cv.take<float2>(N);
    void* ep = cv.take<char>(epoch_scratch_bytes(N, int64_t(nk), 0));

    float a = 0.f, b = 0.f;
    if ((rc = drgb_find_ab(p->spread, p->min_dist, &a, &b))) return set_error(c, rc, "bad spread/min_dist");
    if ((rc = launch_knn_query(c, X_new, n_new, X_train, n_train, d, k, idx, dist, st))) return rc;
    if ((rc = launch_directed_weights(c, idx, dist, n_new, k, n_train, w_dir, out_col, out_w, st))) return rc;
    DRGB_CUDA(c, cudaMemcpyAsync(Ya, Y_train, size_t(n_train) * 8, cudaMemcpyDeviceToDevice, st));
    DRGB_CUDA(c, cudaMemcpyAsync(Yb, Y_train, size_t(n_train) * 8, cudaMemcpyDeviceToDevice, st));
    transform_setup_kernel<<<grid_for(n_new, 256, c->num_sms * 8), 256, 0, st>>>(
        out_col, out_w, n_new, k, reinterpret_cast<const float2*>(Y_train), q, Ya + n_train, Yb + n_train);
    DRGB_CHECK_LAUNCH(c);
    arange_kernel<<<grid_for(n_new + 1, 256, c->num_sms * 8), 256, 0, st>>>(rp, n_new, k);
    DRGB_CHECK_LAUNCH(c);
    const int T3 = (p->n_epochs + 2) / 3;
    rc = run_epochs(c, Ya, Yb, rp, out_col, q, N, a, b, p->lr0, p->neg, 0, T3, T3, p->seed_neg, st, int64_t(nk), ep,
                    0, nullptr, nullptr, n_train, uint32_t(n_train));
    if (rc) return rc;
    DRGB_CUDA(c, cudaMemcpyAsync(Y_new, Ya + n_train, size_t(n_new) * 8, cudaMemcpyDeviceToDevice, st));
    return drgb_sync(c, stream);
}
