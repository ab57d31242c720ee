// Fuzzy simplicial-set graph: per-row rho/sigma and directed weights, then the
// fuzzy union of both directions as a head-sorted CSR with integer schedule
// words.  Everything is deterministic: the in-lists built with atomics are
// re-sorted by source before use, so the output does not depend on the order
// in which atomics resolved.
//
// Passes (n rows, k neighbours, m_j = in-degree of j):
//   1 rows      rho, sigma (64 bisection steps), w_{j|i}; out-list sorted by column
//   2 indegree  histogram of tails
//   3 scan      in_ptr
//   4 scatter   in_src[in_ptr[j] + slot] = p   (p = i*k + s with idx[p] = j)
//   5 sort      each in-list by p (rank sort, warp per row)
//   6 merge     union of out-list and in-list by column -> tmp (cap k + m_i per row), w_max
//   7 count     entries kept (T q >= 2^24)
//   8 scan      row_ptr
//   9 fill      col, w, q
// Passes 6, 7 and 9 take a warp per row.
#include <mutex>

#include "common.cuh"
#include "graph.cuh"

namespace drgb {

static constexpr uint32_t Q_ONE = 1u << 24;

// ---------------------------------------------------------------- pass 1
// Rows are the n query points; neighbour indices lie in [0, db_n) and, when
// self_check is set (a graph of X on itself), must differ from the row.
__global__ void fuzzy_rows_kernel(const int32_t* __restrict__ idx, const float* __restrict__ dist,
                                  int64_t n, int k, float target, float* __restrict__ w_dir,
                                  int32_t* __restrict__ out_col, float* __restrict__ out_w,
                                  float* __restrict__ rho_out, float* __restrict__ sigma_out,
                                  int* __restrict__ status, int64_t db_n, int self_check) {
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
         i += int64_t(gridDim.x) * blockDim.x) {
        float dr[DRGB_MAX_K];
        int32_t jr[DRGB_MAX_K];
        float mean = 0.f;
        bool bad = false;
        for (int s = 0; s < k; ++s) {
            dr[s] = dist[i * k + s];
            jr[s] = idx[i * k + s];
            mean += dr[s];
            bad |= !(dr[s] >= 0.f && dr[s] < INFINITY) || jr[s] < 0 || jr[s] >= db_n || (self_check && jr[s] == i);
        }
        if (bad) report_status(status, DRGB_ERR_INVALID);
        mean /= float(k);
        const float rho = dr[0];
        float lo = 0.f, hi = INFINITY, mid = 1.f;
        for (int it = 0; it < 64; ++it) {
            float psum = 0.f;
            for (int s = 0; s < k; ++s) psum += expf(-fmaxf(0.f, dr[s] - rho) / mid);
            if (psum > target) {
                hi = mid;
            } else {
                lo = mid;
            }
            const float nxt = (hi == INFINITY) ? mid * 2.f : 0.5f * (lo + hi);
            // a step that leaves mid unchanged repeats itself (same test, same
            // bound): every later step would too, so the 64-step result is mid
            if (nxt == mid) break;
            mid = nxt;
        }
        const float sigma = fmaxf(mid, 1e-3f * mean);
        if (rho_out) rho_out[i] = rho;
        if (sigma_out) sigma_out[i] = sigma;
        float wr[DRGB_MAX_K];
        for (int s = 0; s < k; ++s) {
            const float ex = dr[s] - rho;
            wr[s] = ex > 0.f ? expf(-ex / sigma) : 1.f;
            w_dir[i * k + s] = wr[s];
        }
        // out-list sorted by column (insertion sort; k <= DRGB_MAX_K)
        for (int s = 1; s < k; ++s) {
            int32_t jj = jr[s];
            float ww = wr[s];
            int t = s - 1;
            while (t >= 0 && jr[t] > jj) {
                jr[t + 1] = jr[t];
                wr[t + 1] = wr[t];
                --t;
            }
            jr[t + 1] = jj;
            wr[t + 1] = ww;
        }
        bool dup = false;
        for (int s = 0; s < k; ++s) {
            out_col[i * k + s] = jr[s];
            out_w[i * k + s] = wr[s];
            dup |= s > 0 && jr[s] == jr[s - 1];
        }
        if (dup) report_status(status, DRGB_ERR_INVALID);  // a neighbour listed twice
    }
}

// ---------------------------------------------------------------- passes 2, 4
__global__ void indegree_kernel(const int32_t* __restrict__ idx, int64_t n, int k,
                                int32_t* __restrict__ in_cnt) {
    const int64_t nk = n * k;
    for (int64_t p = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; p < nk;
         p += int64_t(gridDim.x) * blockDim.x) {
        const int32_t j = idx[p];
        if (j >= 0 && j < n && j != p / k) atomicAdd(&in_cnt[j], 1);
    }
}

__global__ void in_scatter_kernel(const int32_t* __restrict__ idx, int64_t n, int k,
                                  const int32_t* __restrict__ in_ptr, int32_t* __restrict__ in_fill,
                                  int32_t* __restrict__ in_src) {
    const int64_t nk = n * k;
    for (int64_t p = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; p < nk;
         p += int64_t(gridDim.x) * blockDim.x) {
        const int32_t j = idx[p];
        if (j >= 0 && j < n && j != p / k) {
            const int32_t slot = atomicAdd(&in_fill[j], 1);
            in_src[in_ptr[j] + slot] = int32_t(p);
        }
    }
}

// ---------------------------------------------------------------- pass 5
// Warp per row, ascending order of the row's (distinct) p values whatever
// order the scatter produced.  A row of at most 32 elements (the common case:
// the mean in-degree is k) is held one element per lane and every element
// goes to its rank, counted through shuffles; rows of up to IS_WARP_MAX
// elements are ranked by reading the row back for every element.  Longer
// rows (hubs: at 70K the in-degree reaches 620) of up to IS_BIG_MAX elements
// are listed in big_rows for in_sort_big_kernel; beyond that the warp ranks
// them itself.
static constexpr int IS_WARP_MAX = 128;
static constexpr int IS_BIG_MAX = 8192;
static constexpr int IS_BIG_THREADS = 256;

__global__ void in_sort_kernel(const int32_t* __restrict__ in_ptr, const int32_t* __restrict__ src,
                               int32_t* __restrict__ dst, int64_t n, int32_t* __restrict__ big_rows,
                               unsigned int* __restrict__ big_cnt) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = int64_t(gridDim.x) * (blockDim.x >> 5);
    for (int64_t j = int64_t(blockIdx.x) * (blockDim.x >> 5) + (threadIdx.x >> 5); j < n; j += warps) {
        const int32_t b = in_ptr[j], m = in_ptr[j + 1] - b;
        if (m <= 32) {
            const int32_t x = lane < m ? src[b + lane] : INT32_MAX;
            int32_t rank = 0;
#pragma unroll
            for (int t = 0; t < 32; ++t) {
                const int32_t y = __shfl_sync(0xffffffffu, x, t);
                rank += (t < m && y < x) ? 1 : 0;
            }
            if (lane < m) dst[b + rank] = x;
            continue;
        }
        if (m > IS_WARP_MAX && m <= IS_BIG_MAX) {
            if (lane == 0) big_rows[atomicAdd(big_cnt, 1u)] = int32_t(j);
            continue;
        }
        for (int32_t a = lane; a < m; a += 32) {
            const int32_t x = src[b + a];
            int32_t rank = 0;
            for (int32_t t = 0; t < m; ++t) rank += src[b + t] < x;
            dst[b + rank] = x;
        }
    }
}

// CTA per listed row: the row, padded with INT32_MAX to a power of two, is
// sorted ascending by a bitonic network in shared memory.
__global__ void __launch_bounds__(IS_BIG_THREADS)
in_sort_big_kernel(const int32_t* __restrict__ in_ptr, const int32_t* __restrict__ src,
                   int32_t* __restrict__ dst, const int32_t* __restrict__ big_rows,
                   const unsigned int* __restrict__ big_cnt) {
    extern __shared__ int32_t s_row[];  // [IS_BIG_MAX]
    const unsigned cnt = *big_cnt;
    for (unsigned r = blockIdx.x; r < cnt; r += gridDim.x) {
        const int64_t j = big_rows[r];
        const int32_t b = in_ptr[j], m = in_ptr[j + 1] - b;
        int P = 2 * IS_WARP_MAX;
        while (P < m) P <<= 1;
        __syncthreads();  // the previous row's read-back is done
        for (int a = threadIdx.x; a < P; a += IS_BIG_THREADS) s_row[a] = a < m ? src[b + a] : INT32_MAX;
        __syncthreads();
        for (int kk = 2; kk <= P; kk <<= 1) {
            for (int jj = kk >> 1; jj > 0; jj >>= 1) {
                for (int a = threadIdx.x; a < P; a += IS_BIG_THREADS) {
                    const int l = a ^ jj;
                    if (l > a) {
                        const int32_t x = s_row[a], y = s_row[l];
                        if ((x > y) == ((a & kk) == 0)) {
                            s_row[a] = y;
                            s_row[l] = x;
                        }
                    }
                }
                __syncthreads();
            }
        }
        for (int a = threadIdx.x; a < m; a += IS_BIG_THREADS) dst[b + a] = s_row[a];
    }
}

// ---------------------------------------------------------------- pass 6
__device__ __forceinline__ float fuzzy_union(float a, float b) {
    // a + b - ab, written symmetrically in (a, b) so that w_ij == w_ji exactly
    // and exactly 1 whenever either side is 1.
    const float hi = fmaxf(a, b), lo = fminf(a, b);
    return fmaf(lo, 1.0f - hi, hi);
}

// Warp per row.  Out-list entry a (lane a < k; sorted by column, entries
// reported invalid by pass 1 skipped) and in-list entry b (sorted by source,
// hence by column) go straight to their place in the union sorted by column:
// for a column x that place is #(valid out columns < x) + #(in columns < x)
// - #(columns < x present in both), and a column present in both is written
// once, by its out entry, with the fuzzy union of the two weights.  Columns
// are distinct within each list.
__global__ void merge_kernel(const int32_t* __restrict__ out_col, const float* __restrict__ out_w,
                             const int32_t* __restrict__ in_ptr, const int32_t* __restrict__ in_sorted,
                             const float* __restrict__ w_dir, int64_t n, int k,
                             int32_t* __restrict__ tcol, float* __restrict__ tw,
                             int32_t* __restrict__ tcnt, unsigned int* __restrict__ wmax_bits) {
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    const int64_t warps = int64_t(gridDim.x) * (blockDim.x >> 5);
    float local_max = 0.f;
    for (int64_t i = int64_t(blockIdx.x) * (blockDim.x >> 5) + (threadIdx.x >> 5); i < n; i += warps) {
        const int32_t ib = in_ptr[i], m = in_ptr[i + 1] - ib;
        const int64_t base = i * k + ib;
        int32_t ca = INT32_MAX;  // this lane's out column (INT32_MAX: none or invalid)
        float wa = 0.f;
        if (lane < k) {
            const int32_t c0 = out_col[i * k + lane];
            if (c0 >= 0 && c0 < n && c0 != i) {
                ca = c0;
                wa = out_w[i * k + lane];
            }
        }
        // out entries: in columns below ca, and ca's in weight if present
        int32_t in_less = 0;
        bool matched = false;
        float w_in = 0.f;
        for (int32_t t0 = 0; t0 < m; t0 += 32) {
            int32_t cb = INT32_MAX;
            float wb = 0.f;
            if (t0 + lane < m) {
                const int32_t p = in_sorted[ib + t0 + lane];
                cb = p / k;
                wb = w_dir[p];
            }
            const int cnt = m - t0 < 32 ? m - t0 : 32;
            for (int u = 0; u < cnt; ++u) {
                const int32_t cu = __shfl_sync(0xffffffffu, cb, u);
                const float wu = __shfl_sync(0xffffffffu, wb, u);
                in_less += cu < ca;
                if (cu == ca) {
                    matched = true;
                    w_in = wu;
                }
            }
        }
        const bool va = ca != INT32_MAX;
        const unsigned vmask = __ballot_sync(0xffffffffu, va);
        const unsigned mmask = __ballot_sync(0xffffffffu, va && matched);
        if (va) {
            const int32_t pos = __popc(vmask & lt) + in_less - __popc(mmask & lt);
            const float wv = matched ? fuzzy_union(wa, w_in) : wa;
            tcol[base + pos] = ca;
            tw[base + pos] = wv;
            local_max = fmaxf(local_max, wv);
        }
        // in entries without an out partner
        for (int32_t t0 = 0; t0 < m; t0 += 32) {
            const int32_t t = t0 + lane;
            int32_t cb = INT32_MAX;
            float wb = 0.f;
            if (t < m) {
                const int32_t p = in_sorted[ib + t];
                cb = p / k;
                wb = w_dir[p];
            }
            int32_t out_less = 0, both_less = 0;
            bool partner = false;
            for (int a = 0; a < k; ++a) {
                const int32_t c_a = __shfl_sync(0xffffffffu, ca, a);
                const bool lt_a = c_a < cb;
                out_less += lt_a;
                both_less += lt_a && ((mmask >> a) & 1u);
                partner |= c_a == cb && c_a != INT32_MAX;
            }
            if (t < m && !partner) {
                const int32_t pos = t + out_less - both_less;
                tcol[base + pos] = cb;
                tw[base + pos] = wb;
                local_max = fmaxf(local_max, wb);
            }
        }
        if (lane == 0) tcnt[i] = __popc(vmask) + m - __popc(mmask);
    }
    // non-negative floats order like their bit patterns
    for (int o = 16; o > 0; o >>= 1) local_max = fmaxf(local_max, __shfl_xor_sync(0xffffffffu, local_max, o));
    if (lane == 0) atomicMax(wmax_bits, __float_as_uint(local_max));
}

__device__ __forceinline__ uint32_t schedule_word(float w, float w_max) {
    return __float2uint_rn(float(Q_ONE) * (w / w_max));
}

// ---------------------------------------------------------------- passes 7, 9
// Warp per row; the kept entries keep their order.
__global__ void prune_count_kernel(const int32_t* __restrict__ in_ptr, const float* __restrict__ tw,
                                   const int32_t* __restrict__ tcnt, int64_t n, int k, int T,
                                   const unsigned int* __restrict__ wmax_bits,
                                   int32_t* __restrict__ keep_cnt) {
    const float w_max = __uint_as_float(*wmax_bits);
    const int lane = threadIdx.x & 31;
    const int64_t warps = int64_t(gridDim.x) * (blockDim.x >> 5);
    for (int64_t i = int64_t(blockIdx.x) * (blockDim.x >> 5) + (threadIdx.x >> 5); i < n; i += warps) {
        const int64_t base = i * k + in_ptr[i];
        const int32_t cnt = tcnt[i];
        int32_t c = 0;
        for (int32_t t0 = 0; t0 < cnt; t0 += 32) {
            const int32_t t = t0 + lane;
            const bool keep = t < cnt && uint64_t(T) * schedule_word(tw[base + t], w_max) >= Q_ONE;
            c += __popc(__ballot_sync(0xffffffffu, keep));
        }
        if (lane == 0) keep_cnt[i] = c;
    }
}

__global__ void fill_kernel(const int32_t* __restrict__ in_ptr, const int32_t* __restrict__ tcol,
                            const float* __restrict__ tw, const int32_t* __restrict__ tcnt,
                            int64_t n, int k, int T, const unsigned int* __restrict__ wmax_bits,
                            const int32_t* __restrict__ row_ptr, int32_t* __restrict__ col,
                            float* __restrict__ w, uint32_t* __restrict__ q) {
    const float w_max = __uint_as_float(*wmax_bits);
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    const int64_t warps = int64_t(gridDim.x) * (blockDim.x >> 5);
    for (int64_t i = int64_t(blockIdx.x) * (blockDim.x >> 5) + (threadIdx.x >> 5); i < n; i += warps) {
        const int64_t base = i * k + in_ptr[i];
        const int32_t cnt = tcnt[i];
        int64_t o = row_ptr[i];
        for (int32_t t0 = 0; t0 < cnt; t0 += 32) {
            const int32_t t = t0 + lane;
            float wt = 0.f;
            uint32_t qt = 0;
            bool keep = false;
            if (t < cnt) {
                wt = tw[base + t];
                qt = schedule_word(wt, w_max);
                keep = uint64_t(T) * qt >= Q_ONE;
            }
            const unsigned km = __ballot_sync(0xffffffffu, keep);
            if (keep) {
                const int64_t d = o + __popc(km & lt);
                col[d] = tcol[base + t];
                w[d] = wt;
                q[d] = qt;
            }
            o += __popc(km);
        }
    }
}

int launch_directed_weights(Ctx* c, const int32_t* idx, const float* dist, int64_t n, int k, int64_t db_n,
                            float* w_dir, int32_t* out_col, float* out_w, cudaStream_t st) {
    const float target = float(std::log2(double(k)));
    fuzzy_rows_kernel<<<grid_for(n, 128, c->num_sms * 16), 128, 0, st>>>(idx, dist, n, k, target, w_dir, out_col,
                                                                        out_w, nullptr, nullptr, c->d_status, db_n, 0);
    DRGB_CHECK_LAUNCH(c);
    return DRGB_OK;
}

size_t fuzzy_scratch_bytes(int64_t n, int k) {
    const size_t nk = size_t(n) * k;
    size_t b = 0;
    b += Carve::round(nk * 4) * 3;          // w_dir, out_col, out_w
    b += Carve::round((n + 1) * 4) * 4;     // in_cnt, in_ptr, in_fill, keep_cnt
    b += Carve::round(nk * 4) * 2;          // in_src, in_sorted
    b += Carve::round(2 * nk * 4) * 2;      // tcol, tw
    b += Carve::round(n * 4);               // tcnt
    b += Carve::round(256);                 // w_max
    b += Carve::round(scan_scratch_elems(n) * 4);
    return b + 4096;
}

int build_fuzzy_graph(Ctx* c, const int32_t* idx, const float* dist, int64_t n, int k, int T,
                      int32_t* row_ptr, int32_t* col, float* w, uint32_t* q, float* rho,
                      float* sigma, void* scratch, cudaStream_t st) {
    const size_t nk = size_t(n) * k;
    Carve cv(scratch);
    float* w_dir = cv.take<float>(nk);
    int32_t* out_col = cv.take<int32_t>(nk);
    float* out_w = cv.take<float>(nk);
    int32_t* in_cnt = cv.take<int32_t>(n + 1);
    int32_t* in_ptr = cv.take<int32_t>(n + 1);
    int32_t* in_fill = cv.take<int32_t>(n + 1);
    int32_t* keep_cnt = cv.take<int32_t>(n + 1);
    int32_t* in_src = cv.take<int32_t>(nk);
    int32_t* in_sorted = cv.take<int32_t>(nk);
    int32_t* tcol = cv.take<int32_t>(2 * nk);
    float* tw = cv.take<float>(2 * nk);
    int32_t* tcnt = cv.take<int32_t>(n);
    unsigned int* wmax = cv.take<unsigned int>(64);
    int32_t* scan_tmp = cv.take<int32_t>(scan_scratch_elems(n));

    const int TB = 256;
    const int gmax = c->num_sms * 16;
    const float target = float(std::log2(double(k)));
    fuzzy_rows_kernel<<<grid_for(n, 128, gmax), 128, 0, st>>>(idx, dist, n, k, target, w_dir, out_col,
                                                             out_w, rho, sigma, c->d_status, n, 1);
    DRGB_CHECK_LAUNCH(c);
    DRGB_CUDA(c, cudaMemsetAsync(in_cnt, 0, (n + 1) * 4, st));
    DRGB_CUDA(c, cudaMemsetAsync(in_fill, 0, (n + 1) * 4, st));
    DRGB_CUDA(c, cudaMemsetAsync(wmax, 0, 4, st));
    indegree_kernel<<<grid_for(int64_t(nk), TB, gmax), TB, 0, st>>>(idx, n, k, in_cnt);
    DRGB_CHECK_LAUNCH(c);
    int rc = exclusive_scan(c, in_cnt, in_ptr, n, scan_tmp, st);
    if (rc) return rc;
    in_scatter_kernel<<<grid_for(int64_t(nk), TB, gmax), TB, 0, st>>>(idx, n, k, in_ptr, in_fill, in_src);
    DRGB_CHECK_LAUNCH(c);
    {
        // rows longer than a warp ranks well go to a CTA each; keep_cnt is
        // free until the prune pass and holds their list
        int32_t* big_rows = keep_cnt;
        unsigned int* big_cnt = wmax + 32;
        DRGB_CUDA(c, cudaMemsetAsync(big_cnt, 0, 4, st));
        in_sort_kernel<<<grid_for(n, TB / 32, gmax), TB, 0, st>>>(in_ptr, in_src, in_sorted, n, big_rows, big_cnt);
        DRGB_CHECK_LAUNCH(c);
        const size_t big_smem = size_t(IS_BIG_MAX) * 4;
        in_sort_big_kernel<<<c->num_sms * 2, IS_BIG_THREADS, big_smem, st>>>(in_ptr, in_src, in_sorted, big_rows,
                                                                              big_cnt);
    }
    DRGB_CHECK_LAUNCH(c);
    merge_kernel<<<grid_for(n, TB / 32, gmax), TB, 0, st>>>(out_col, out_w, in_ptr, in_sorted, w_dir, n, k,
                                                           tcol, tw, tcnt, wmax);
    DRGB_CHECK_LAUNCH(c);
    prune_count_kernel<<<grid_for(n, TB / 32, gmax), TB, 0, st>>>(in_ptr, tw, tcnt, n, k, T, wmax, keep_cnt);
    DRGB_CHECK_LAUNCH(c);
    rc = exclusive_scan(c, keep_cnt, row_ptr, n, scan_tmp, st);
    if (rc) return rc;
    fill_kernel<<<grid_for(n, TB / 32, gmax), TB, 0, st>>>(in_ptr, tcol, tw, tcnt, n, k, T, wmax, row_ptr,
                                                          col, w, q);
    DRGB_CHECK_LAUNCH(c);
    return DRGB_OK;
}

}  // namespace drgb

using namespace drgb;

extern "C" int drgb_fuzzy_weights(drgb_ctx* c, const int32_t* idx, const float* dist, int64_t n,
                                  int32_t k, int32_t n_epochs, int32_t* row_ptr, int32_t* col,
                                  float* w, uint32_t* q, int64_t cap, float* rho, float* sigma,
                                  void* stream) {
    if (!c) return DRGB_ERR_INVALID;
    if (!idx || !dist || !row_ptr || !col || !w || !q)
        return set_error(c, DRGB_ERR_INVALID, "fuzzy_weights: NULL pointer");
    if (k < 1 || k > DRGB_MAX_K || n < k + 1 || n > (INT32_MAX / 2) / k || n_epochs < 1)
        return set_error(c, DRGB_ERR_INVALID, "fuzzy_weights: bad n=%lld k=%d n_epochs=%d",
                         (long long)n, k, n_epochs);
    if (cap < 2 * n * k)
        return set_error(c, DRGB_ERR_WORKSPACE, "fuzzy_weights: cap %lld < 2nk = %lld",
                         (long long)cap, (long long)(2 * n * k));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int rc = ensure_scratch(c, fuzzy_scratch_bytes(n, k), st);
    if (rc) return rc;
    return build_fuzzy_graph(c, idx, dist, n, k, n_epochs, row_ptr, col, w, q, rho, sigma,
                             c->scratch, st);
}

// ---------------------------------------------------------------------------
// Allocation-free variant.  Its scratch is this file-scope device array: every
// device that loads the library reserves it for the life of the process.  The
// first 256 bytes hold the device status word, the rest is carved exactly as
// the context scratch of drgb_fuzzy_weights.
static __device__ __align__(256) unsigned char g_fuzzy_static_scratch[DRGB_STATIC_SCRATCH_BYTES];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_static_mutex;
void* g_static_ptr[kMaxDevices] = {};
int g_static_sms[kMaxDevices] = {};
}  // namespace

extern "C" int drgb_fuzzy_weights_static(const int32_t* idx, const float* dist, int64_t n, int32_t k,
                                         int32_t n_epochs, int32_t* row_ptr, int32_t* col, float* w,
                                         uint32_t* q, int64_t cap, float* rho, float* sigma,
                                         void* stream) {
    if (!idx || !dist || !row_ptr || !col || !w || !q) return DRGB_ERR_INVALID;
    if (k < 1 || k > DRGB_MAX_K || n < k + 1 || n > (INT32_MAX / 2) / k || n_epochs < 1) return DRGB_ERR_INVALID;
    if (cap < 2 * n * k) return DRGB_ERR_WORKSPACE;
    if (256 + fuzzy_scratch_bytes(n, k) > size_t(DRGB_STATIC_SCRATCH_BYTES)) return DRGB_ERR_WORKSPACE;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return DRGB_ERR_DEVICE;
    void* base = nullptr;
    int sms = 0;
    {
        // one-time set-up per device, with that device current: look up the
        // device address of the array (the host-side symbol is only a handle)
        std::lock_guard<std::mutex> lock(g_static_mutex);
        if (!g_static_ptr[dev]) {
            void* p = nullptr;
            if (cudaGetSymbolAddress(&p, g_fuzzy_static_scratch) != cudaSuccess || !p) {
                cudaGetLastError();
                return DRGB_ERR_CUDA;
            }
            int count = 0;
            if (cudaDeviceGetAttribute(&count, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
                cudaGetLastError();
                return DRGB_ERR_CUDA;
            }
            g_static_ptr[dev] = p;
            g_static_sms[dev] = count;
        }
        base = g_static_ptr[dev];
        sms = g_static_sms[dev];
    }
    // a stack context: no device memory of its own, status word in the array
    Ctx c;
    c.device = dev;
    c.num_sms = sms;
    c.d_status = static_cast<int*>(base);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (cudaMemsetAsync(c.d_status, 0, sizeof(int), st) != cudaSuccess) return DRGB_ERR_CUDA;
    int rc = build_fuzzy_graph(&c, idx, dist, n, k, n_epochs, row_ptr, col, w, q, rho, sigma,
                               static_cast<unsigned char*>(base) + 256, st);
    if (rc) return rc;
    if (cudaStreamSynchronize(st) != cudaSuccess) return DRGB_ERR_CUDA;
    int status = 0;
    if (cudaMemcpy(&status, c.d_status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return DRGB_ERR_CUDA;
    return status ? status : DRGB_OK;
}
