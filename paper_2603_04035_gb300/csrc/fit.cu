// fit_transform(X) -> Y: the whole hot path on one stream (Section 2.1, the
// public API; Section 3, the timed fit_transform).  [PCA to pca_dim ->] k-NN
// graph -> fuzzy graph -> a, b -> initialisation -> T epochs (one captured
// graph), all enqueued before the single synchronisation at the end (the
// optional PCA synchronises on its own first).
#include "common.cuh"
#include "epoch.cuh"
#include "graph.cuh"
#include "knn.cuh"
#include "nndescent.cuh"
#include "pca.cuh"
#include "spectral.cuh"

namespace drgb {

struct FitBuffers {
    int32_t* idx;
    float* dist;
    int32_t* row_ptr;
    int32_t* col;
    float* w;
    uint32_t* q;
    float2* Y_tmp;
    float2* Y_tune;
    void* fuzzy_scratch;
    void* epoch_scratch;
};

static size_t fit_bytes(int64_t n, int k) {
    const size_t nk = size_t(n) * k;
    return Carve::round(nk * 4) * 2 + Carve::round((n + 1) * 4) + Carve::round(2 * nk * 4) * 3 +
           Carve::round(n * 8) * 2 + Carve::round(fuzzy_scratch_bytes(n, k)) +
           Carve::round(epoch_scratch_bytes(n, int64_t(2 * nk), 0)) + 4096;
}

// Fit buffers first, then the k-NN scratch region (disjoint from them).
static FitBuffers carve_fit(void* base, int64_t n, int k) {
    const size_t nk = size_t(n) * k;
    Carve cv(base);
    FitBuffers b;
    b.idx = cv.take<int32_t>(nk);
    b.dist = cv.take<float>(nk);
    b.row_ptr = cv.take<int32_t>(n + 1);
    b.col = cv.take<int32_t>(2 * nk);
    b.w = cv.take<float>(2 * nk);
    b.q = cv.take<uint32_t>(2 * nk);
    b.Y_tmp = cv.take<float2>(n);
    b.Y_tune = cv.take<float2>(n);
    b.fuzzy_scratch = cv.take<char>(fuzzy_scratch_bytes(n, k));
    b.epoch_scratch = cv.take<char>(epoch_scratch_bytes(n, int64_t(2 * nk), 0));
    return b;
}

}  // namespace drgb

using namespace drgb;

extern "C" int drgb_fit_transform(drgb_ctx* c, const float* X, int64_t n, int32_t d,
                                  const drgb_params* p, float* Y_out, drgb_epoch_cb cb, void* user,
                                  void* stream) {
    if (!c) return DRGB_ERR_INVALID;
    if (!p || !Y_out) return set_error(c, DRGB_ERR_INVALID, "fit_transform: NULL pointer");
    int rc = check_knn_args(c, X, n, d, p->k, Y_out, Y_out);
    if (rc) return rc;
    if (!aligned(Y_out, 8)) return set_error(c, DRGB_ERR_INVALID, "fit_transform: Y_out misaligned");
    if (p->n_epochs < 1 || p->neg < 0 || p->neg > 64 || !(p->init_range > 0.f) || n > (INT32_MAX / 2) / p->k)
        return set_error(c, DRGB_ERR_INVALID, "fit_transform: bad parameters");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int k = p->k;
    if (p->knn_mode < 0 || p->knn_mode > 4) return set_error(c, DRGB_ERR_INVALID, "fit_transform: bad knn_mode");
    if (p->pca_dim < 0 || p->pca_dim > PCA_MAX_DIM)
        return set_error(c, DRGB_ERR_INVALID, "fit_transform: pca_dim must be 0..%d", PCA_MAX_DIM);
    const bool do_pca = p->pca_dim > 0 && p->pca_dim < d;
    if (do_pca && d > PCA_MAX_FEATURES)
        return set_error(c, DRGB_ERR_INVALID, "fit_transform: PCA takes at most %d features", PCA_MAX_FEATURES);
    const int dk = do_pca ? p->pca_dim : d;  // the k-NN graph's dimension
    const bool nnd = p->knn_mode == 4;
    if (nnd && dk > NND_MAX_D)
        return set_error(c, DRGB_ERR_INVALID, "fit_transform: NNDescent takes at most %d dimensions", NND_MAX_D);
    const size_t fb = Carve::round(fit_bytes(n, k));
    const size_t zb = do_pca ? Carve::round(size_t(n) * dk * 4) : 0;
    const bool spectral = (p->flags & DRGB_FLAG_INIT_SPECTRAL) != 0;
    const bool nnd_rev = k <= 16;  // the reverse form (general neighbours) where a warp holds them
    const size_t kb = nnd ? nnd_scratch_bytes(n, k, nnd_rev) : knn_scratch_bytes(n, dk, k, p->knn_mode);
    // the PCA's, then the k-NN's, then the spectral layout's scratch share one
    // region (each is free by the time the next starts)
    const size_t sb = spectral ? spectral_scratch_bytes(n, int64_t(2) * n * k, c->num_sms) : 0;
    const size_t pb = do_pca ? pca_scratch_bytes(n, d) : 0;
    size_t rb = kb > sb ? kb : sb;
    rb = rb > pb ? rb : pb;
    rc = ensure_scratch(c, fb + zb + rb, st);
    if (rc) return rc;
    FitBuffers b = carve_fit(c->scratch, n, k);
    float* Z = do_pca ? reinterpret_cast<float*>(static_cast<char*>(c->scratch) + fb) : nullptr;
    void* knn_scratch = static_cast<char*>(c->scratch) + fb + zb;

    float a = 0.f, bb = 0.f;
    rc = drgb_find_ab(p->spread, p->min_dist, &a, &bb);
    if (rc) return set_error(c, rc, "fit_transform: bad spread/min_dist");

    c->stage_marks = 0;
    c->knn_marks = 0;
    rc = launch_nonfinite_scan(c, X, n * d, st);
    if (rc) return rc;
    const float* Xk = X;
    if (do_pca) {  // synchronises the stream (its Rayleigh-Ritz steps read back a few values)
        rc = pca_run(c, X, n, d, dk, Z, nullptr, nullptr, nullptr, knn_scratch, st);
        if (rc) return rc;
        Xk = Z;
    }
    if ((rc = stage_mark(c, 0, st))) return rc;
    if (nnd)  // synchronises the stream once per iteration
        rc = nnd_run(c, Xk, n, dk, k, p->seed_init, NND_DELTA, NND_ITER_DEFAULT, nnd_rev, b.idx, b.dist, nullptr, nullptr,
                     knn_scratch, st);
    else
        rc = knn_run(c, Xk, n, dk, k, p->knn_mode, b.idx, b.dist, st, knn_scratch);
    if (rc) return rc;
    if ((rc = stage_mark(c, 1, st))) return rc;
    rc = build_fuzzy_graph(c, b.idx, b.dist, n, k, p->n_epochs, b.row_ptr, b.col, b.w, b.q, nullptr,
                           nullptr, b.fuzzy_scratch, st);
    if (rc) return rc;
    if ((rc = stage_mark(c, 2, st))) return rc;
    float2* Y = reinterpret_cast<float2*>(Y_out);
    if (spectral)
        rc = spectral_layout(c, b.row_ptr, b.col, b.w, n, int64_t(2) * n * k, p->init_range, p->seed_init, Y,
                             nullptr, knn_scratch, st);
    else
        rc = launch_init(c, Y, n, p->init_range, p->seed_init, st);
    if (rc) return rc;
    const int64_t nnz_cap = int64_t(2) * n * k;
    if (p->flags & DRGB_FLAG_AUTOTUNE) {
        float us = 0.f;
        EpochScratch es;
        if ((rc = epoch_prepare(c, b.row_ptr, n, 0, nnz_cap, 0, nullptr, b.epoch_scratch, &es, st))) return rc;
        rc = autotune_epoch(c, Y, b.Y_tune, b.Y_tmp, b.row_ptr, b.col, b.q, n, a, bb, p->neg, p->n_epochs,
                            p->seed_neg, 3, st, es, 0, nullptr, nullptr, &us);
        if (rc) return rc;
    }
    if ((rc = stage_mark(c, 3, st))) return rc;
    if (!cb) {
        rc = run_epochs(c, Y, b.Y_tmp, b.row_ptr, b.col, b.q, n, a, bb, p->lr0, p->neg, 0, p->n_epochs,
                        p->n_epochs, p->seed_neg, st, nnz_cap, b.epoch_scratch);
        if (rc) return rc;
    } else {
        for (int t = 0; t < p->n_epochs; ++t) {
            rc = run_epochs(c, Y, b.Y_tmp, b.row_ptr, b.col, b.q, n, a, bb, p->lr0, p->neg, t, t + 1,
                            p->n_epochs, p->seed_neg, st, nnz_cap, b.epoch_scratch);
            if (rc) return rc;
            rc = drgb_sync(c, stream);
            if (rc) return rc;
            if (cb(t, Y_out, n, user)) break;
        }
    }
    if ((rc = stage_mark(c, 4, st))) return rc;
    // the embedding itself is scanned too: a non-finite output (which the
    // clipped updates should never produce) is reported, not returned silently
    if ((rc = launch_nonfinite_scan(c, Y_out, 2 * n, st))) return rc;
    return drgb_sync(c, stream);
}
