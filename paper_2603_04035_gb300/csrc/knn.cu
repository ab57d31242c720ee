// Exact k-NN by an FP32 scan (SIMT), and the FP32 rank counts used by the
// trustworthiness metric.
//
// One thread owns one query row and keeps its best K (distance, index) pairs
// sorted in registers.  The database is streamed through shared memory in
// tiles of 32 points x 32 dimensions; every thread reads the same tile element
// (a broadcast), so the tile costs no bank conflicts.  Squared distances are
// evaluated directly as sum_c (x_qc - x_pc)^2 in dimension order, so the
// result is the exact FP32 ranking (ties resolved by lower index because the
// scan visits points in increasing index order and only strictly smaller
// distances displace a kept entry).
#include "common.cuh"
#include "knn.cuh"

namespace drgb {

static constexpr int KNN_THREADS = 128;
static constexpr int TP = 32;  // points per tile
static constexpr int DC = 32;  // dimensions per tile

// Accumulate squared distances between this thread's query and TP database
// points starting at p0, over all d dimensions.
__device__ __forceinline__ void tile_distances(const float* __restrict__ X, int64_t n, int d,
                                               int64_t qi, bool qvalid, int64_t p0, float* s_db,
                                               float (&acc)[TP], const float* __restrict__ Q) {
#pragma unroll
    for (int p = 0; p < TP; ++p) acc[p] = 0.f;
    for (int c0 = 0; c0 < d; c0 += DC) {
        __syncthreads();
        for (int t = threadIdx.x; t < TP * DC; t += blockDim.x) {
            const int p = t / DC, cc = t % DC;
            const int64_t gp = p0 + p;
            const int gc = c0 + cc;
            s_db[t] = (gp < n && gc < d) ? X[gp * d + gc] : 0.f;
        }
        __syncthreads();
        float qv[DC];
#pragma unroll
        for (int cc = 0; cc < DC; ++cc) qv[cc] = (qvalid && c0 + cc < d) ? Q[qi * d + c0 + cc] : 0.f;
        // fully unrolled so that acc stays in registers; dimensions are added
        // in order (beyond d both sides are 0 and the fma leaves a unchanged)
#pragma unroll
        for (int p = 0; p < TP; ++p) {
            float a = acc[p];
#pragma unroll
            for (int cc = 0; cc < DC; cc += 4) {
                const float4 v = *reinterpret_cast<const float4*>(&s_db[p * DC + cc]);
                float df = qv[cc] - v.x;
                a = fmaf(df, df, a);
                df = qv[cc + 1] - v.y;
                a = fmaf(df, df, a);
                df = qv[cc + 2] - v.z;
                a = fmaf(df, df, a);
                df = qv[cc + 3] - v.w;
                a = fmaf(df, df, a);
            }
            acc[p] = a;
        }
    }
}

// Query rows: rows[r] (int64), or rows32[r] (int32), or r.  With n_rows_dev
// the number of rows is read on the device (blocks past it exit at once) and
// results go to row rows32[r] of the outputs instead of row r.
//
// With p_end > 0 the scan covers only database points [p_begin, p_end) and the
// k best of that range are written as partial list blockIdx.y of row r
// (idx_out/dist_out + (blockIdx.y * n_rows + r) * k, squared distances).
//
// With ub, ub[qi * k + k - 1] is the distance (FP32, square-rooted) of the
// k-th of k distinct points other than qi, or INFINITY; only points at most
// that far are kept (the k nearest all are), so lists may end early with
// index -1.
template <int K>
__global__ void __launch_bounds__(KNN_THREADS)
knn_exact_kernel(const float* __restrict__ X, int64_t n, int d, int k,
                 const int64_t* __restrict__ rows, int64_t n_rows, int32_t* __restrict__ idx_out,
                 float* __restrict__ dist_out, int write_sqrt, const int32_t* __restrict__ rows32,
                 const int32_t* __restrict__ n_rows_dev, int64_t chunk = 0, const float* __restrict__ Qx = nullptr,
                 const float* __restrict__ ub = nullptr) {
    // queries come from Qx (a separate matrix, no self to exclude) or from X
    const float* Q = Qx ? Qx : X;
    const int64_t self_off = Qx ? -1 : 0;
    __shared__ __align__(16) float s_db[TP * DC];
    if (n_rows_dev) {
        n_rows = *n_rows_dev;
        if (int64_t(blockIdx.x) * KNN_THREADS >= n_rows) return;  // whole block idle
    }
    const int64_t r = int64_t(blockIdx.x) * KNN_THREADS + threadIdx.x;
    const bool valid = r < n_rows;
    const int64_t qi = valid ? (rows ? rows[r] : (rows32 ? int64_t(rows32[r]) : r)) : 0;
    int64_t orow = (n_rows_dev && !chunk) ? qi : r;
    int64_t p_begin = 0, p_end = n;
    if (chunk) {
        p_begin = int64_t(blockIdx.y) * chunk;
        p_end = p_begin + chunk < n ? p_begin + chunk : n;
        orow = int64_t(blockIdx.y) * n_rows + r;
    }
    // admission bound: the square of the k-th listed distance, rounded up past
    // the rounding of the square root and of this square, plus the smallest
    // normal number so that a k-th distance of 0 (k or more exact copies of
    // the query) still admits the points at distance 0 (the test is strict)
    float T = INFINITY;
    if (ub && valid) {
        const float u = ub[qi * k + k - 1];
        T = fmaf(u * u, 1.0f + 1e-6f, 1.17549435e-38f);
        if (!(T < INFINITY)) T = INFINITY;
    }
    float D[K];
    int32_t I[K];
#pragma unroll
    for (int s = 0; s < K; ++s) {
        D[s] = T;
        I[s] = -1;
    }
    float acc[TP];
    for (int64_t p0 = p_begin; p0 < p_end; p0 += TP) {
        tile_distances(X, p_end, d, qi, valid, p0, s_db, acc, Q);
        const int64_t self = self_off ? int64_t(-1) : qi;
#pragma unroll
        for (int p = 0; p < TP; ++p) {
            const int64_t gp = p0 + p;
            if (acc[p] < D[K - 1] && gp < p_end && gp != self) topk_insert<K>(D, I, acc[p], int32_t(gp));
        }
    }
    if (valid) {
#pragma unroll
        for (int s = 0; s < K; ++s) {
            if (s < k) {
                idx_out[orow * k + s] = I[s];
                dist_out[orow * k + s] = write_sqrt ? sqrtf(D[s]) : D[s];
            }
        }
    }
}

// Merge the C partial k-lists (squared distances, ascending) of each listed
// row into its final k nearest, ordered by (distance, index).  One warp per
// row: lane l keeps the best K of the lists l, l + 32, ...; then k rounds each
// take the warp-wide smallest head by (distance, index).  The chunks cover
// disjoint index ranges, so no index appears twice.
template <int K>
__device__ __forceinline__ bool lex_less(float a, int32_t i, float b, int32_t j) {
    return a < b || (a == b && i < j);
}

template <int K>
__global__ void merge_partials_kernel(const int32_t* __restrict__ pidx, const float* __restrict__ pd2,
                                      int64_t cnt, int C, int k, const int32_t* __restrict__ rows32,
                                      int32_t* __restrict__ idx_out, float* __restrict__ dist_out) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = int64_t(gridDim.x) * (blockDim.x >> 5);
    for (int64_t r = int64_t(blockIdx.x) * (blockDim.x >> 5) + (threadIdx.x >> 5); r < cnt; r += warps) {
        float D[K];
        int32_t I[K];
#pragma unroll
        for (int s = 0; s < K; ++s) {
            D[s] = INFINITY;
            I[s] = INT32_MAX;
        }
        for (int c0 = lane; c0 < C; c0 += 4 * 32) {
          // the heads of four lists are loaded together; a list whose head
          // is empty (-1) or not better than the current K-th is skipped
          int32_t hj[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
              const int c = c0 + u * 32;
              hj[u] = c < C ? pidx[(int64_t(c) * cnt + r) * k] : -1;
          }
#pragma unroll 1
          for (int u = 0; u < 4; ++u) {
            if (hj[u] < 0) continue;
            const int64_t base = (int64_t(c0 + u * 32) * cnt + r) * k;
            for (int s = 0; s < k; ++s) {
                const float a = pd2[base + s];
                const int32_t j = s ? pidx[base + s] : hj[u];
                if (j < 0 || !lex_less<K>(a, j, D[K - 1], I[K - 1])) break;  // each list is ascending
#pragma unroll
                for (int t = K - 1; t > 0; --t) {
                    const bool shift = lex_less<K>(a, j, D[t - 1], I[t - 1]);
                    const bool place = !shift && lex_less<K>(a, j, D[t], I[t]);
                    D[t] = shift ? D[t - 1] : (place ? a : D[t]);
                    I[t] = shift ? I[t - 1] : (place ? j : I[t]);
                }
                if (lex_less<K>(a, j, D[0], I[0])) {
                    D[0] = a;
                    I[0] = j;
                }
            }
          }
        }
        const int64_t row = rows32[r];
        for (int s = 0; s < k; ++s) {
            float bd = D[0];
            int32_t bi = I[0];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const float od = __shfl_xor_sync(0xffffffffu, bd, o);
                const int32_t oi = __shfl_xor_sync(0xffffffffu, bi, o);
                if (lex_less<K>(od, oi, bd, bi)) {
                    bd = od;
                    bi = oi;
                }
            }
            if (lane == 0) {
                idx_out[row * k + s] = bi;
                dist_out[row * k + s] = sqrtf(bd);
            }
            if (I[0] == bi && D[0] == bd) {  // the owner pops its head
#pragma unroll
                for (int t = 0; t < K - 1; ++t) {
                    D[t] = D[t + 1];
                    I[t] = I[t + 1];
                }
                D[K - 1] = INFINITY;
                I[K - 1] = INT32_MAX;
            }
        }
    }
}

int launch_knn_exact_rows_n(Ctx* c, const float* X, int64_t n, int d, int k, const int32_t* rows32,
                            const int32_t* n_rows_dev, int64_t cnt, int32_t* idx_out, float* dist_out,
                            cudaStream_t st, void* part_scratch, size_t part_bytes) {
    if (cnt <= 0) return DRGB_OK;
    const int row_blocks = int((cnt + KNN_THREADS - 1) / KNN_THREADS);
    int64_t C = (8 * int64_t(c->num_sms) + row_blocks - 1) / row_blocks;
    const int64_t max_c = (n + 127) / 128;               // at least 128 points per chunk
    if (C > max_c) C = max_c;
    if (C > 1024) C = 1024;
    const int64_t fit_c = part_scratch ? int64_t(part_bytes / 2 / (size_t(cnt) * k * 4 + 256)) : 0;
    if (C > fit_c) C = fit_c;                            // partial lists must fit the scratch
    if (C <= 1) {
        const int blocks = row_blocks;
        if (k <= 16)
            knn_exact_kernel<16><<<blocks, KNN_THREADS, 0, st>>>(X, n, d, k, nullptr, cnt, idx_out, dist_out, 1,
                                                                rows32, n_rows_dev, 0, nullptr, dist_out);
        else
            knn_exact_kernel<32><<<blocks, KNN_THREADS, 0, st>>>(X, n, d, k, nullptr, cnt, idx_out, dist_out, 1,
                                                                rows32, n_rows_dev, 0, nullptr, dist_out);
        DRGB_CHECK_LAUNCH(c);
        return DRGB_OK;
    }
    Carve cv(part_scratch);
    int32_t* pidx = cv.take<int32_t>(size_t(cnt) * C * k);
    float* pd2 = cv.take<float>(size_t(cnt) * C * k);
    const int64_t chunk = (n + C - 1) / C;
    dim3 grid(row_blocks, unsigned(C));
    if (k <= 16)
        knn_exact_kernel<16><<<grid, KNN_THREADS, 0, st>>>(X, n, d, k, nullptr, cnt, pidx, pd2, 0, rows32,
                                                          nullptr, chunk, nullptr, dist_out);
    else
        knn_exact_kernel<32><<<grid, KNN_THREADS, 0, st>>>(X, n, d, k, nullptr, cnt, pidx, pd2, 0, rows32,
                                                          nullptr, chunk, nullptr, dist_out);
    DRGB_CHECK_LAUNCH(c);
    return launch_merge_partials(c, pidx, pd2, cnt, int(C), k, rows32, idx_out, dist_out, st);
}

int launch_merge_partials(Ctx* c, const int32_t* pidx, const float* pd2, int64_t cnt, int C, int k,
                          const int32_t* rows32, int32_t* idx_out, float* dist_out, cudaStream_t st) {
    if (cnt <= 0) return DRGB_OK;
    const int mb = grid_for(cnt, 4, c->num_sms * 8);   // one warp per row, 4 warps per CTA
    if (k <= 16)
        merge_partials_kernel<16><<<mb, 128, 0, st>>>(pidx, pd2, cnt, C, k, rows32, idx_out, dist_out);
    else
        merge_partials_kernel<32><<<mb, 128, 0, st>>>(pidx, pd2, cnt, C, k, rows32, idx_out, dist_out);
    DRGB_CHECK_LAUNCH(c);
    return DRGB_OK;
}

int launch_knn_query(Ctx* c, const float* Q, int64_t nq, const float* X, int64_t n, int d, int k,
                     int32_t* idx_out, float* dist_out, cudaStream_t st) {
    const int blocks = int((nq + KNN_THREADS - 1) / KNN_THREADS);
    if (blocks < 1) return DRGB_OK;
    if (k <= 16)
        knn_exact_kernel<16><<<blocks, KNN_THREADS, 0, st>>>(X, n, d, k, nullptr, nq, idx_out, dist_out, 1, nullptr,
                                                            nullptr, 0, Q);
    else
        knn_exact_kernel<32><<<blocks, KNN_THREADS, 0, st>>>(X, n, d, k, nullptr, nq, idx_out, dist_out, 1, nullptr,
                                                            nullptr, 0, Q);
    DRGB_CHECK_LAUNCH(c);
    return DRGB_OK;
}

int launch_knn_exact(Ctx* c, const float* X, int64_t n, int d, int k, const int64_t* rows,
                     int64_t n_rows, int32_t* idx_out, float* dist_out, bool write_sqrt,
                     cudaStream_t st) {
    const int blocks = int((n_rows + KNN_THREADS - 1) / KNN_THREADS);
    if (blocks < 1) return DRGB_OK;
    if (k <= 16)
        knn_exact_kernel<16><<<blocks, KNN_THREADS, 0, st>>>(X, n, d, k, rows, n_rows, idx_out, dist_out,
                                                            write_sqrt, nullptr, nullptr);
    else
        knn_exact_kernel<32><<<blocks, KNN_THREADS, 0, st>>>(X, n, d, k, rows, n_rows, idx_out, dist_out,
                                                            write_sqrt, nullptr, nullptr);
    DRGB_CHECK_LAUNCH(c);
    return DRGB_OK;
}

// For query row r (point qi) and its k targets tgt[r][s], count the points l != qi
// that precede the target in the FP32 (distance, index) order: rank - 1.
template <int K>
__global__ void __launch_bounds__(KNN_THREADS)
rank_kernel(const float* __restrict__ X, int64_t n, int d, int k, const int64_t* __restrict__ rows,
            int64_t n_rows, const int32_t* __restrict__ tgt, int64_t* __restrict__ excess_out) {
    __shared__ __align__(16) float s_db[TP * DC];
    const int64_t r = int64_t(blockIdx.x) * KNN_THREADS + threadIdx.x;
    const bool valid = r < n_rows;
    const int64_t qi = valid ? (rows ? rows[r] : r) : 0;
    float td[K];
    int32_t tj[K];
    int32_t cnt[K];
#pragma unroll
    for (int s = 0; s < K; ++s) {
        tj[s] = (valid && s < k) ? tgt[r * k + s] : -1;
        cnt[s] = 0;
        td[s] = -1.f;  // filled during the scan when the target itself is met
    }
    // pass 1: distances to the targets (same formula and order as the scan)
    for (int s = 0; s < K; ++s) {
        if (s >= k || tj[s] < 0) continue;
        float a = 0.f;
        for (int cc = 0; cc < d; ++cc) {
            const float df = X[qi * d + cc] - X[int64_t(tj[s]) * d + cc];
            a = fmaf(df, df, a);
        }
        td[s] = a;
    }
    float acc[TP];
    for (int64_t p0 = 0; p0 < n; p0 += TP) {
        tile_distances(X, n, d, qi, valid, p0, s_db, acc, X);
#pragma unroll
        for (int p = 0; p < TP; ++p) {
            const int64_t gp = p0 + p;
            if (gp >= n || gp == qi) continue;
#pragma unroll
            for (int s = 0; s < K; ++s)
                cnt[s] += (acc[p] < td[s]) || (acc[p] == td[s] && gp < tj[s]);
        }
    }
    if (valid) {
        int64_t ex = 0;
#pragma unroll
        for (int s = 0; s < K; ++s)
            if (s < k && tj[s] >= 0 && cnt[s] + 1 > k) ex += cnt[s] + 1 - k;
        excess_out[r] = ex;
    }
}

int launch_rank(Ctx* c, const float* X, int64_t n, int d, int k, const int64_t* rows,
                int64_t n_rows, const int32_t* tgt, int64_t* excess_out, cudaStream_t st) {
    const int blocks = int((n_rows + KNN_THREADS - 1) / KNN_THREADS);
    if (blocks < 1) return DRGB_OK;
    if (k <= 16)
        rank_kernel<16><<<blocks, KNN_THREADS, 0, st>>>(X, n, d, k, rows, n_rows, tgt, excess_out);
    else
        rank_kernel<32><<<blocks, KNN_THREADS, 0, st>>>(X, n, d, k, rows, n_rows, tgt, excess_out);
    DRGB_CHECK_LAUNCH(c);
    return DRGB_OK;
}

__global__ void nonfinite_scan_kernel(const float* __restrict__ X, int64_t count, int* status) {
    bool bad = false;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < count;
         i += int64_t(gridDim.x) * blockDim.x)
        bad |= !isfinite(X[i]);
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) report_status(status, DRGB_ERR_NONFINITE);
}

int launch_nonfinite_scan(Ctx* c, const float* X, int64_t count, cudaStream_t st) {
    nonfinite_scan_kernel<<<grid_for(count, 256, c->num_sms * 8), 256, 0, st>>>(X, count, c->d_status);
    DRGB_CHECK_LAUNCH(c);
    return DRGB_OK;
}

int check_knn_args(Ctx* c, const float* X, int64_t n, int d, int k, const void* idx_out,
                   const void* dist_out) {
    if (!c) return DRGB_ERR_INVALID;
    if (!X || !idx_out || !dist_out) return set_error(c, DRGB_ERR_INVALID, "knn_graph: NULL pointer");
    if (!aligned(X, 4)) return set_error(c, DRGB_ERR_INVALID, "knn_graph: X must be 4-byte aligned");
    if (k < 1 || k > DRGB_MAX_K || d < 1 || n < int64_t(k) + 1 || n > INT32_MAX)
        return set_error(c, DRGB_ERR_INVALID, "knn_graph: bad sizes n=%lld d=%d k=%d", (long long)n, d, k);
    return DRGB_OK;
}

}  // namespace drgb

using namespace drgb;

namespace drgb {

int knn_resolve_mode(int64_t n, int d, int k, int mode) {
    if (mode == 0) return knn_tc_preferred(n, d, k) ? 3 : 1;
    return mode;
}

size_t knn_scratch_bytes(int64_t n, int d, int k, int mode) {
    (void)k;
    const int m = knn_resolve_mode(n, d, k, mode);
    return (m == 2 || m == 3) ? knn_tc_scratch_bytes(n, d) : 0;
}

int knn_run(Ctx* c, const float* X, int64_t n, int d, int k, int mode, int32_t* idx_out, float* dist_out,
            cudaStream_t st, void* scratch, int32_t* defer_rows, int32_t* defer_count) {
    const int m = knn_resolve_mode(n, d, k, mode);
    if (m == 2 || m == 3)
        return knn_tc(c, X, n, d, k, m == 3, idx_out, dist_out, st, scratch, defer_rows, defer_count);
    if (m != 1) return set_error(c, DRGB_ERR_INVALID, "knn_graph: bad mode %d", mode);
    return launch_knn_exact(c, X, n, d, k, nullptr, n, idx_out, dist_out, true, st);
}

}  // namespace drgb

extern "C" int drgb_knn_graph(drgb_ctx* c, const float* X, int64_t n, int32_t d, int32_t k,
                              int32_t mode, int32_t* idx_out, float* dist_out, void* stream) {
    int rc = check_knn_args(c, X, n, d, k, idx_out, dist_out);
    if (rc) return rc;
    if (mode < 0 || mode > 3) return set_error(c, DRGB_ERR_INVALID, "knn_graph: bad mode %d", mode);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const size_t bytes = knn_scratch_bytes(n, d, k, mode);
    if (bytes && (rc = ensure_scratch(c, bytes, st))) return rc;
    return knn_run(c, X, n, d, k, mode, idx_out, dist_out, st, c->scratch);
}
