// Batched form: many independent instances of uneven size embedded together.
// The concatenated instances form one block-diagonal problem: each instance's
// k-NN graph is computed separately (rows of one instance only see that
// instance; the k-NN runs of all instances are enqueued back to back with no
// host synchronisation between them: the uncertified rows of each run are
// collected on the device and re-scanned after the last run, with one read of
// their counts), its indices are made global, the fuzzy graph of the whole
// concatenation is built at once (its rows never cross instances), and every
// epoch runs as one launch over all rows with instance-local entry numbers,
// negative ranges and Philox keys.  Every arithmetic step of a row is the one a
// single-instance fit performs, so each instance's embedding is bit-identical
// to fitting it alone with the same seeds.  The epoch loop of all instances is
// one captured CUDA graph.
//
// Also here: the epoch autotuner's entry point, which times every supported
// force-kernel setting (width 4 or 8 warps per CTA, pipelined or flat form)
// on the actual graph; all of them give bit-identical results, so it changes
// speed only.
#include <vector>

#include "common.cuh"
#include "epoch.cuh"
#include "graph.cuh"
#include "knn.cuh"

namespace drgb {

// Streams the batched k-NN runs spread over.
static constexpr int BATCH_STREAMS = 8;

__global__ void globalize_idx_kernel(int32_t* __restrict__ idx, int64_t n_total, int k, int count,
                                     const int64_t* __restrict__ inst_off) {
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n_total;
         i += int64_t(gridDim.x) * blockDim.x) {
        int lo = 0, hi = count - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (inst_off[mid] <= i) lo = mid; else hi = mid - 1;
        }
        const int32_t off = int32_t(inst_off[lo]);
        for (int s = 0; s < k; ++s) idx[i * k + s] += off;
    }
}

}  // namespace drgb

using namespace drgb;

extern "C" {

int drgb_fit_transform_batched(drgb_ctx* c, const float* X_cat, const int64_t* offsets, int32_t count,
                               int32_t d, const drgb_params* p, const uint64_t* seeds_init,
                               const uint64_t* seeds_neg, float* Y_cat, void* stream) {
    if (!c) return DRGB_ERR_INVALID;
    if (!X_cat || !offsets || !p || !Y_cat || count < 1)
        return set_error(c, DRGB_ERR_INVALID, "fit_transform_batched: NULL pointer or count < 1");
    const int k = p->k;
    if (k < 1 || k > DRGB_MAX_K || d < 1 || p->n_epochs < 1 || p->neg < 0 || p->neg > 64 ||
        !(p->init_range > 0.f) || p->knn_mode < 0 || p->knn_mode > 3 || !aligned(Y_cat, 8) ||
        !aligned(X_cat, 4))
        return set_error(c, DRGB_ERR_INVALID, "fit_transform_batched: bad parameters");
    if (offsets[0] != 0) return set_error(c, DRGB_ERR_INVALID, "fit_transform_batched: offsets[0] != 0");
    if (p->pca_dim != 0) return set_error(c, DRGB_ERR_INVALID, "fit_transform_batched: pca_dim is not supported");
    int64_t max_n = 0;
    for (int b = 0; b < count; ++b) {
        const int64_t nb = offsets[b + 1] - offsets[b];
        if (nb < int64_t(k) + 1)
            return set_error(c, DRGB_ERR_INVALID, "fit_transform_batched: instance %d has %lld < k + 1 rows", b,
                             (long long)nb);
        max_n = nb > max_n ? nb : max_n;
    }
    const int64_t N = offsets[count];
    if (N > (INT32_MAX / 2) / k) return set_error(c, DRGB_ERR_INVALID, "fit_transform_batched: too many rows");
    cudaStream_t st = static_cast<cudaStream_t>(stream);

    // scratch: per-row buffers of the concatenation, then the k-NN region for
    // the largest instance
    size_t knn_bytes = 0;
    for (int b = 0; b < count; ++b) {
        const size_t kb = knn_scratch_bytes(offsets[b + 1] - offsets[b], d, k, p->knn_mode);
        knn_bytes = kb > knn_bytes ? kb : knn_bytes;
    }
    const size_t Nk = size_t(N) * k;
    const size_t main_bytes = Carve::round(Nk * 4) * 2 + Carve::round((N + 1) * 4) + Carve::round(2 * Nk * 4) * 3 +
                              Carve::round(N * 4) + Carve::round(count * 4) +
                              Carve::round(N * 8) * 2 + Carve::round((count + 1) * 8) + 2 * Carve::round(count * 8) +
                              Carve::round(fuzzy_scratch_bytes(N, k)) +
                              Carve::round(epoch_scratch_bytes(N, int64_t(2 * Nk), count)) + 8192;
    // instances are small: their k-NN runs go round-robin to BATCH_STREAMS
    // streams, each with its own k-NN scratch region, so that several run at once
    const int n_str = count < BATCH_STREAMS ? count : BATCH_STREAMS;
    const size_t knn_region = Carve::round(knn_bytes);
    int rc = ensure_scratch(c, Carve::round(main_bytes) + size_t(n_str) * knn_region, st);
    if (rc) return rc;
    Carve cv(c->scratch);
    int32_t* idx = cv.take<int32_t>(Nk);
    float* dist = cv.take<float>(Nk);
    int32_t* row_ptr = cv.take<int32_t>(N + 1);
    int32_t* col = cv.take<int32_t>(2 * Nk);
    float* w = cv.take<float>(2 * Nk);
    uint32_t* q = cv.take<uint32_t>(2 * Nk);
    float2* Y_tmp = cv.take<float2>(N);
    float2* Y_tune = cv.take<float2>(N);
    int64_t* d_off = cv.take<int64_t>(count + 1);
    uint64_t* d_seed_init = cv.take<uint64_t>(count);
    uint64_t* d_seed_neg = cv.take<uint64_t>(count);
    void* fz = cv.take<char>(fuzzy_scratch_bytes(N, k));
    void* ep = cv.take<char>(epoch_scratch_bytes(N, int64_t(2 * Nk), count));
    int32_t* fail_rows = cv.take<int32_t>(N);      // uncertified rows of instance b at [offsets[b], ...)
    int32_t* fail_count = cv.take<int32_t>(count);
    void* knn_scratch = static_cast<char*>(c->scratch) + Carve::round(main_bytes);

    std::vector<uint64_t> si(count), sn(count);
    for (int b = 0; b < count; ++b) {
        si[b] = seeds_init ? seeds_init[b] : p->seed_init;
        sn[b] = seeds_neg ? seeds_neg[b] : p->seed_neg;
    }
    DRGB_CUDA(c, cudaMemcpyAsync(d_off, offsets, (count + 1) * 8, cudaMemcpyHostToDevice, st));
    DRGB_CUDA(c, cudaMemcpyAsync(d_seed_init, si.data(), count * 8, cudaMemcpyHostToDevice, st));
    DRGB_CUDA(c, cudaMemcpyAsync(d_seed_neg, sn.data(), count * 8, cudaMemcpyHostToDevice, st));

    float a = 0.f, bb = 0.f;
    if ((rc = drgb_find_ab(p->spread, p->min_dist, &a, &bb))) return set_error(c, rc, "bad spread/min_dist");
    c->stage_marks = 0;
    c->knn_marks = 0;
    if ((rc = launch_nonfinite_scan(c, X_cat, N * d, st))) return rc;
    if ((rc = stage_mark(c, 0, st))) return rc;
    DRGB_CUDA(c, cudaMemsetAsync(fail_count, 0, size_t(count) * 4, st));
    {
        // side streams start after the work already on `st` and `st` waits
        // for all of them; they are created and destroyed per call
        cudaStream_t ss[BATCH_STREAMS] = {};
        cudaEvent_t ev[BATCH_STREAMS + 1] = {};
        auto release = [&]() {
            for (int i = 0; i < n_str; ++i)
                if (ss[i]) cudaStreamDestroy(ss[i]);
            for (int i = 0; i <= n_str; ++i)
                if (ev[i]) cudaEventDestroy(ev[i]);
        };
        cudaError_t e = cudaEventCreateWithFlags(&ev[n_str], cudaEventDisableTiming);
        for (int i = 0; i < n_str && e == cudaSuccess; ++i) {
            e = cudaStreamCreateWithFlags(&ss[i], cudaStreamNonBlocking);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev[i], cudaEventDisableTiming);
        }
        if (e == cudaSuccess) e = cudaEventRecord(ev[n_str], st);
        for (int i = 0; i < n_str && e == cudaSuccess; ++i) e = cudaStreamWaitEvent(ss[i], ev[n_str], 0);
        if (e != cudaSuccess) {
            release();
            return set_error(c, DRGB_ERR_CUDA, "fit_transform_batched: side streams: %s", cudaGetErrorString(e));
        }
        for (int b = 0; b < count && rc == DRGB_OK; ++b) {
            const int64_t off = offsets[b], nb = offsets[b + 1] - off;
            const int si_ = b % n_str;
            rc = knn_run(c, X_cat + off * d, nb, d, k, p->knn_mode, idx + off * k, dist + off * k, ss[si_],
                         static_cast<char*>(knn_scratch) + size_t(si_) * knn_region, fail_rows + off, fail_count + b);
        }
        for (int i = 0; i < n_str; ++i) {
            if (cudaEventRecord(ev[i], ss[i]) != cudaSuccess || cudaStreamWaitEvent(st, ev[i], 0) != cudaSuccess) {
                if (rc == DRGB_OK) rc = set_error(c, DRGB_ERR_CUDA, "fit_transform_batched: joining side streams");
            }
        }
        release();
        if (rc) return rc;
    }
    // exact re-scan of every instance's uncertified rows (the k-NN scratch is
    // free again: its partial lists go there)
    {
        std::vector<int32_t> h(count);
        DRGB_CUDA(c, cudaMemcpyAsync(h.data(), fail_count, size_t(count) * 4, cudaMemcpyDeviceToHost, st));
        DRGB_CUDA(c, cudaStreamSynchronize(st));
        const size_t part = knn_bytes < knn_rescan_part_bytes() ? knn_bytes : knn_rescan_part_bytes();
        for (int b = 0; b < count; ++b) {
            const int64_t off = offsets[b], nb = offsets[b + 1] - off;
            const int64_t cnt = h[b] < nb ? h[b] : nb;
            if (cnt <= 0) continue;
            rc = launch_knn_exact_rows_n(c, X_cat + off * d, nb, d, k, fail_rows + off, fail_count + b, cnt,
                                         idx + off * k, dist + off * k, st, knn_scratch, part);
            if (rc) return rc;
        }
    }
    globalize_idx_kernel<<<grid_for(N, 256, c->num_sms * 8), 256, 0, st>>>(idx, N, k, count, d_off);
    DRGB_CHECK_LAUNCH(c);
    if ((rc = stage_mark(c, 1, st))) return rc;
    rc = build_fuzzy_graph(c, idx, dist, N, k, p->n_epochs, row_ptr, col, w, q, nullptr, nullptr, fz, st);
    if (rc) return rc;
    if ((rc = stage_mark(c, 2, st))) return rc;
    float2* Y = reinterpret_cast<float2*>(Y_cat);
    if ((rc = launch_init_batched(c, Y, N, p->init_range, count, d_off, d_seed_init, st))) return rc;
    if (p->flags & DRGB_FLAG_AUTOTUNE) {
        // a setting tuned earlier for this device and problem size, if the
        // context has a tuning cache that holds one; else time the choices
        // (and record the winner there)
        const std::string key = tuning_key(c, N, count, k);
        int32_t cached_w = 0, cached_p = 1;
        if (!c->tuning_cache.empty() &&
            drgb_tuning_cache_lookup(c->tuning_cache.c_str(), key.c_str(), &cached_w, &cached_p) == DRGB_OK) {
            c->epoch_warps = cached_w;
            c->epoch_pipe = cached_p;
        } else {
            float us = 0.f;
            EpochScratch es;
            if ((rc = epoch_prepare(c, row_ptr, N, 0, int64_t(2 * Nk), count, d_off, ep, &es, st))) return rc;
            rc = autotune_epoch(c, Y, Y_tune, Y_tmp, row_ptr, col, q, N, a, bb, p->neg, p->n_epochs, 0, 3, st, es,
                                count, d_off, d_seed_neg, &us);
            if (rc) return rc;
            if (!c->tuning_cache.empty() &&
                drgb_tuning_cache_store(c->tuning_cache.c_str(), key.c_str(), c->epoch_warps, c->epoch_pipe) !=
                    DRGB_OK)
                return set_error(c, DRGB_ERR_INVALID, "tuning cache %s could not be written", c->tuning_cache.c_str());
        }
    }
    if ((rc = stage_mark(c, 3, st))) return rc;
    rc = run_epochs(c, Y, Y_tmp, row_ptr, col, q, N, a, bb, p->lr0, p->neg, 0, p->n_epochs, p->n_epochs, 0, st,
                    int64_t(2 * Nk), ep, count, d_off, d_seed_neg);
    if (rc) return rc;
    if ((rc = stage_mark(c, 4, st))) return rc;
    return drgb_sync(c, stream);
}

int drgb_autotune_epoch(drgb_ctx* c, const float* Y, const int32_t* row_ptr, const int32_t* col,
                        const uint32_t* q, int64_t n, float a, float b, int32_t neg, int32_t n_epochs,
                        uint64_t seed, int32_t trials, int32_t* choice, float* us_per_epoch, void* stream) {
    if (!c) return DRGB_ERR_INVALID;
    if (!Y || !row_ptr || !col || !q || n < 1 || n > INT32_MAX || neg < 0 || neg > 64 || n_epochs < 1 ||
        trials < 1 || !aligned(Y, 8) || !aligned(row_ptr, 4) || !aligned(col, 4) || !aligned(q, 4))
        return set_error(c, DRGB_ERR_INVALID, "autotune_epoch: bad arguments");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int32_t nnz = 0;
    DRGB_CUDA(c, cudaMemcpyAsync(&nnz, row_ptr + n, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    DRGB_CUDA(c, cudaStreamSynchronize(st));
    if (nnz < 0) return set_error(c, DRGB_ERR_INVALID, "autotune_epoch: row_ptr[n] < 0");
    const size_t yb = Carve::round(size_t(n) * 8);
    int rc = ensure_scratch(c, 2 * yb + epoch_scratch_bytes(n, nnz, 0), st);
    if (rc) return rc;
    Carve cv(c->scratch);
    float2* Ya = cv.take<float2>(n);
    float2* Yb = cv.take<float2>(n);
    void* ep = cv.take<char>(epoch_scratch_bytes(n, nnz, 0));
    EpochScratch es;
    if ((rc = epoch_prepare(c, row_ptr, n, 0, nnz, 0, nullptr, ep, &es, st))) return rc;
    rc = autotune_epoch(c, reinterpret_cast<const float2*>(Y), Ya, Yb, row_ptr, col, q, n, a, b, neg, n_epochs, seed,
                        trials, st, es, 0, nullptr, nullptr, us_per_epoch);
    if (rc) return rc;
    if (choice) {
        choice[0] = c->epoch_warps;
        choice[1] = c->epoch_pipe;
        choice[2] = 0;
    }
    return drgb_sync(c, stream);
}

}  // extern "C"
