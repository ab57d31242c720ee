// Embedding-quality metrics on the device: k-NN preservation and
// trustworthiness (Section 3.2: exact neighbour ranks from pairwise Euclidean
// distances).  Query rows are all rows, or the evenly strided rows
// i_r = floor(r n / m) for a sample of m rows.
#include <vector>

#include "common.cuh"
#include "knn.cuh"

namespace drgb {

__global__ void strided_rows_kernel(int64_t* rows, int64_t m, int64_t n) {
    for (int64_t r = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; r < m;
         r += int64_t(gridDim.x) * blockDim.x)
        rows[r] = (r * n) / m;
}

// Per row: |A_r & B_r| for two k-sets of indices.
__global__ void intersect_kernel(const int32_t* __restrict__ A, const int32_t* __restrict__ B,
                                 int64_t m, int k, int32_t* __restrict__ hits) {
    for (int64_t r = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; r < m;
         r += int64_t(gridDim.x) * blockDim.x) {
        int h = 0;
        for (int s = 0; s < k; ++s) {
            const int32_t a = A[r * k + s];
            for (int t = 0; t < k; ++t) h += (a == B[r * k + t]);
        }
        hits[r] = h;
    }
}

static int eval_common(Ctx* c, const float* X, const float* Y, int64_t n, int d, int k,
                       int64_t n_query, bool want_recall, double* out, cudaStream_t st) {
    if (!c) return DRGB_ERR_INVALID;
    if (!X || !Y || !out) return set_error(c, DRGB_ERR_INVALID, "eval: NULL pointer");
    if (!aligned(X, 4) || !aligned(Y, 8)) return set_error(c, DRGB_ERR_INVALID, "eval: misaligned");
    if (k < 1 || k > DRGB_MAX_K || n < int64_t(k) + 1 || n > INT32_MAX || d < 1)
        return set_error(c, DRGB_ERR_INVALID, "eval: bad sizes");
    if (!want_recall && 2.0 * n - 3.0 * k - 1.0 <= 0)
        return set_error(c, DRGB_ERR_INVALID, "eval: trustworthiness needs 2n - 3k - 1 > 0");
    const int64_t m = (n_query <= 0 || n_query >= n) ? n : n_query;
    const size_t bytes = Carve::round(m * 8) + 2 * Carve::round(m * k * 4) * 2 +
                         Carve::round(m * 8) + Carve::round(m * 4) + 4096;
    int rc = ensure_scratch(c, bytes, st);
    if (rc) return rc;
    Carve cv(c->scratch);
    int64_t* rows = cv.take<int64_t>(m);
    int32_t* ny = cv.take<int32_t>(m * k);
    float* dy = cv.take<float>(m * k);
    int32_t* nx = cv.take<int32_t>(m * k);
    float* dx = cv.take<float>(m * k);
    int64_t* excess = cv.take<int64_t>(m);
    int32_t* hits = cv.take<int32_t>(m);
    strided_rows_kernel<<<grid_for(m, 256, c->num_sms * 8), 256, 0, st>>>(rows, m, n);
    DRGB_CHECK_LAUNCH(c);
    rc = launch_knn_exact(c, Y, n, 2, k, rows, m, ny, dy, false, st);
    if (rc) return rc;
    if (want_recall) {
        rc = launch_knn_exact(c, X, n, d, k, rows, m, nx, dx, false, st);
        if (rc) return rc;
        intersect_kernel<<<grid_for(m, 256, c->num_sms * 8), 256, 0, st>>>(nx, ny, m, k, hits);
        DRGB_CHECK_LAUNCH(c);
        std::vector<int32_t> h(m);
        DRGB_CUDA(c, cudaMemcpyAsync(h.data(), hits, m * 4, cudaMemcpyDeviceToHost, st));
        DRGB_CUDA(c, cudaStreamSynchronize(st));
        double s = 0;
        for (int64_t r = 0; r < m; ++r) s += h[r];
        *out = s / (double(k) * double(m));
    } else {
        rc = launch_rank(c, X, n, d, k, rows, m, ny, excess, st);
        if (rc) return rc;
        std::vector<int64_t> e(m);
        DRGB_CUDA(c, cudaMemcpyAsync(e.data(), excess, m * 8, cudaMemcpyDeviceToHost, st));
        DRGB_CUDA(c, cudaStreamSynchronize(st));
        double s = 0;
        for (int64_t r = 0; r < m; ++r) s += double(e[r]);
        *out = 1.0 - 2.0 / (double(m) * k * (2.0 * n - 3.0 * k - 1.0)) * s;
    }
    return DRGB_OK;
}

// dst[r] = src[rows[r]] for rows of d floats.
__global__ void gather_rows_kernel(const float* __restrict__ src, int d, const int64_t* __restrict__ rows,
                                   int64_t m, float* __restrict__ dst) {
    for (int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < m * d;
         t += int64_t(gridDim.x) * blockDim.x) {
        const int64_t r = t / d;
        dst[t] = src[rows[r] * d + (t - r * d)];
    }
}

// Held-out k-NN preservation: for the strided sample of new points, the k
// nearest training points in the input space against the k nearest training
// points in the 2-D embedding (the new point's position against the training
// embedding).  Both neighbour sets are exact FP32 scans, ties by index.
static int eval_heldout(Ctx* c, const float* Xt, const float* Yt, int64_t n, const float* Xn, const float* Yn,
                        int64_t n_new, int d, int k, int64_t n_query, double* out, cudaStream_t st) {
    if (!c) return DRGB_ERR_INVALID;
    if (!Xt || !Yt || !Xn || !Yn || !out) return set_error(c, DRGB_ERR_INVALID, "eval_recall_heldout: NULL pointer");
    if (!aligned(Xt, 4) || !aligned(Xn, 4) || !aligned(Yt, 8) || !aligned(Yn, 8))
        return set_error(c, DRGB_ERR_INVALID, "eval_recall_heldout: misaligned");
    if (k < 1 || k > DRGB_MAX_K || n < int64_t(k) || n > INT32_MAX || n_new < 1 || d < 1)
        return set_error(c, DRGB_ERR_INVALID, "eval_recall_heldout: bad sizes");
    const int64_t m = (n_query <= 0 || n_query >= n_new) ? n_new : n_query;
    const size_t bytes = Carve::round(m * 8) + Carve::round(m * d * 4) + Carve::round(m * 8) +
                         4 * Carve::round(m * k * 4) + Carve::round(m * 4) + 4096;
    int rc = ensure_scratch(c, bytes, st);
    if (rc) return rc;
    Carve cv(c->scratch);
    int64_t* rows = cv.take<int64_t>(m);
    float* xq = cv.take<float>(m * d);
    float* yq = cv.take<float>(m * 2);
    int32_t* nx = cv.take<int32_t>(m * k);
    float* dx = cv.take<float>(m * k);
    int32_t* ny = cv.take<int32_t>(m * k);
    float* dy = cv.take<float>(m * k);
    int32_t* hits = cv.take<int32_t>(m);
    strided_rows_kernel<<<grid_for(m, 256, c->num_sms * 8), 256, 0, st>>>(rows, m, n_new);
    DRGB_CHECK_LAUNCH(c);
    gather_rows_kernel<<<grid_for(m * d, 256, c->num_sms * 8), 256, 0, st>>>(Xn, d, rows, m, xq);
    DRGB_CHECK_LAUNCH(c);
    gather_rows_kernel<<<grid_for(m * 2, 256, c->num_sms * 8), 256, 0, st>>>(Yn, 2, rows, m, yq);
    DRGB_CHECK_LAUNCH(c);
    if ((rc = launch_knn_query(c, xq, m, Xt, n, d, k, nx, dx, st))) return rc;
    if ((rc = launch_knn_query(c, yq, m, Yt, n, 2, k, ny, dy, st))) return rc;
    intersect_kernel<<<grid_for(m, 256, c->num_sms * 8), 256, 0, st>>>(nx, ny, m, k, hits);
    DRGB_CHECK_LAUNCH(c);
    std::vector<int32_t> h(m);
    DRGB_CUDA(c, cudaMemcpyAsync(h.data(), hits, m * 4, cudaMemcpyDeviceToHost, st));
    DRGB_CUDA(c, cudaStreamSynchronize(st));
    double s = 0;
    for (int64_t r = 0; r < m; ++r) s += h[r];
    *out = s / (double(k) * double(m));
    return DRGB_OK;
}

}  // namespace drgb

using namespace drgb;

extern "C" {

int drgb_eval_recall(drgb_ctx* c, const float* X, const float* Y, int64_t n, int32_t d, int32_t k,
                     int64_t n_query, double* out, void* stream) {
    return eval_common(c, X, Y, n, d, k, n_query, true, out, static_cast<cudaStream_t>(stream));
}

int drgb_eval_trust(drgb_ctx* c, const float* X, const float* Y, int64_t n, int32_t d, int32_t k,
                    int64_t n_query, double* out, void* stream) {
    return eval_common(c, X, Y, n, d, k, n_query, false, out, static_cast<cudaStream_t>(stream));
}

int drgb_eval_recall_heldout(drgb_ctx* c, const float* X_train, const float* Y_train, int64_t n,
                             const float* X_new, const float* Y_new, int64_t n_new, int32_t d, int32_t k,
                             int64_t n_query, double* out, void* stream) {
    return eval_heldout(c, X_train, Y_train, n, X_new, Y_new, n_new, d, k, n_query, out,
                        static_cast<cudaStream_t>(stream));
}

}  // extern "C"
