// NNDescent approximate k-NN graph (Section 2.2: every point starts with k
// random neighbours, the graph is refined by exploring neighbours of
// neighbours with a top-k selection, and the loop ends once the update rate
// falls below delta = 0.015).
//
// The iteration is synchronous (every list read is the previous
// iteration's), so the graph is a pure function of X, k, the seed and the
// stopping rule:
//   start      point i takes the words of Philox4x32-10 (key = seed, counters
//              (i, r, 0, 5), r = 0..15, words in order); a word u proposes
//              floor(u n / 2^32), accepted when it is not i and not yet in
//              the list, until k are accepted (then the smallest unused
//              indices, if 64 words were not enough);
//   iteration  C(i) = G(i) united with G(j), j in G(i), without i; the new
//              G(i) is the k candidates of smallest (squared distance, index);
//   reverse    (optional: the basic algorithm of Dong et al., which Section
//              2.2 cites) R(i) = up to k of the points whose lists hold i,
//              the k of smallest (squared distance, index); the join runs
//              over general neighbours B(i) = G(i) united with R(i): C(i) =
//              B(i) united with B(u), u in B(i), without i;
//   updates    the number of new neighbours entering the lists; the loop
//              stops after the first iteration whose rate (updates / n k) is
//              below delta, or after max_iter iterations.
//
// One warp per point: the candidates' indices are deduplicated in a per-warp
// open-addressing table in shared memory, each lane computes the FP32 direct
// squared distance sum_j (x_cj - x_ij)^2 (j in order) of its candidates, and
// the k smallest (distance, index) keys are selected exactly by k rounds of a
// warp minimum.  Distances are gathered row by row rather than through a
// GEMM: the candidates of a point are irregular, so the work is the gathers.
#include <vector>

#include "common.cuh"
#include "knn.cuh"
#include "nndescent.cuh"

namespace drgb {

static constexpr uint32_t TAG_NND = 5u;
static constexpr int NND_WORDS = 64;
static constexpr int NND_WARPS = 8;  // warps per block when shared memory allows
static constexpr size_t NND_SMEM_CAP = 200u << 10;  // dynamic shared memory per block at most

// Shared memory of one warp: keys (8 B each), the unique list, the hash
// table, the query row, the count.
struct NndLayout {
    int cmax, H, logH, d_pad;
    size_t bytes;
};

static NndLayout nnd_layout(int k, int d, bool rev) {
    NndLayout L;
    const int b = rev ? 2 * k : k;  // general neighbours of a point
    L.cmax = b + b * b;
    L.H = 1;
    L.logH = 0;
    while (L.H < 2 * L.cmax) {
        L.H <<= 1;
        ++L.logH;
    }
    L.d_pad = (d + 1) & ~1;
    L.bytes = size_t(L.cmax) * 8 + size_t(L.cmax) * 4 + size_t(L.H) * 4 + size_t(L.d_pad) * 4 + 8;
    L.bytes = (L.bytes + 15) & ~size_t(15);
    return L;
}

__global__ void nnd_init_kernel(int64_t n, int k, uint32_t k0, uint32_t k1, int32_t* __restrict__ G) {
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
        int taken[DRGB_MAX_K];
        int cnt = 0;
        for (int r = 0; r < NND_WORDS / 4 && cnt < k; ++r) {
            const U4 w = philox4x32_10(U4{uint32_t(i), uint32_t(r), 0u, TAG_NND}, k0, k1);
            const uint32_t ws[4] = {w.x, w.y, w.z, w.w};
            for (int q = 0; q < 4 && cnt < k; ++q) {
                const int m = int((uint64_t(ws[q]) * uint64_t(n)) >> 32);
                if (m == int(i)) continue;
                bool dup = false;
                for (int t = 0; t < cnt; ++t) dup |= taken[t] == m;
                if (!dup) taken[cnt++] = m;
            }
        }
        for (int64_t cidx = 0; cnt < k && cidx < n; ++cidx) {  // completion: smallest unused indices
            if (cidx == i) continue;
            bool dup = false;
            for (int t = 0; t < cnt; ++t) dup |= taken[t] == int(cidx);
            if (!dup) taken[cnt++] = int(cidx);
        }
        for (int t = 0; t < k; ++t) G[i * k + t] = taken[t];
    }
}

__device__ __forceinline__ void nnd_insert(int id, int* __restrict__ table, int H, int logH, int* __restrict__ list,
                                           int* __restrict__ cnt) {
    uint32_t h = (uint32_t(id) * 2654435761u) >> (32 - logH);  // multiplicative hashing (Knuth)
    for (int p = 0; p < H; ++p) {  // the table holds at most half its size: a free slot is always found
        const int old = atomicCAS(&table[h], -1, id);
        if (old == -1) {
            list[atomicAdd(cnt, 1)] = id;
            return;
        }
        if (old == id) return;
        h = (h + 1) & uint32_t(H - 1);
    }
}

template <bool PAIRS>
__device__ __forceinline__ float nnd_dist2(const float* __restrict__ xc, const float* __restrict__ xq, int d) {
    float s = 0.f;
    if (PAIRS) {  // d even, rows 8-byte aligned: the same order of terms, two per load
        const float2* a = reinterpret_cast<const float2*>(xc);
#pragma unroll 4
        for (int j = 0; j < d / 2; ++j) {
            const float2 v = a[j];
            const float dx = v.x - xq[2 * j], dy = v.y - xq[2 * j + 1];
            s = fmaf(dx, dx, s);
            s = fmaf(dy, dy, s);
        }
    } else {
#pragma unroll 4
        for (int j = 0; j < d; ++j) {
            const float df = xc[j] - xq[j];
            s = fmaf(df, df, s);
        }
    }
    return s;
}

template <bool PAIRS, bool REV>
__global__ void __launch_bounds__(NND_WARPS * 32) nnd_iter_kernel(const float* __restrict__ X, int64_t n, int d,
                                                                  int k, NndLayout L, const int32_t* __restrict__ G,
                                                                  const int32_t* __restrict__ R,
                                                                  int32_t* __restrict__ Gn, float* __restrict__ Dn,
                                                                  unsigned long long* __restrict__ updates) {
    extern __shared__ __align__(16) unsigned char nsm[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
    unsigned char* base = nsm + size_t(warp) * L.bytes;
    uint64_t* keys = reinterpret_cast<uint64_t*>(base);
    int* list = reinterpret_cast<int*>(keys + L.cmax);
    int* table = list + L.cmax;
    float* xq = reinterpret_cast<float*>(table + L.H);
    int* cnt = reinterpret_cast<int*>(xq + L.d_pad);
    for (int64_t i = int64_t(blockIdx.x) * wpb + warp; i < n; i += int64_t(gridDim.x) * wpb) {
        for (int t = lane; t < L.H; t += 32) table[t] = -1;
        if (lane == 0) *cnt = 0;
        for (int t = lane; t < d; t += 32) xq[t] = X[i * d + t];
        // lanes < k hold G(i); with REV lanes k..2k-1 hold R(i) (-1 pads)
        const int g = lane < k ? G[i * k + lane] : ((REV && lane < 2 * k) ? R[i * k + lane - k] : -1);
        const int nbk = REV ? 2 * k : k;
        int nb[DRGB_MAX_K];  // lane l: entry l of the general neighbours of the point in lane r
#pragma unroll
        for (int r = 0; r < DRGB_MAX_K; ++r) {
            const int jr = __shfl_sync(0xffffffffu, g, r);
            int v = -1;
            if (r < nbk && jr >= 0) {
                if (lane < k) v = G[int64_t(jr) * k + lane];
                else if (REV && lane < 2 * k) v = R[int64_t(jr) * k + lane - k];
            }
            nb[r] = v;
        }
        __syncwarp();
        if (g >= 0) nnd_insert(g, table, L.H, L.logH, list, cnt);
#pragma unroll
        for (int r = 0; r < DRGB_MAX_K; ++r)
            if (nb[r] >= 0 && nb[r] != int(i)) nnd_insert(nb[r], table, L.H, L.logH, list, cnt);
        __syncwarp();
        const int U = *cnt;
        for (int u = lane; u < U; u += 32) {
            const int cidx = list[u];
            const float s = nnd_dist2<PAIRS>(X + int64_t(cidx) * d, xq, d);
            keys[u] = (uint64_t(__float_as_uint(s)) << 32) | uint32_t(cidx);
        }
        __syncwarp();
        // the k smallest keys: distances are >= 0, so the bit patterns order
        // like the values, and (distance, index) keys are distinct
        uint64_t lo = 0, mine = ~0ull;
        for (int r = 0; r < k; ++r) {
            uint64_t best = ~0ull;
            for (int u = lane; u < U; u += 32) {
                const uint64_t key = keys[u];
                if (key >= lo && key < best) best = key;
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const uint64_t ob = __shfl_xor_sync(0xffffffffu, best, o);
                best = ob < best ? ob : best;
            }
            if (lane == r) mine = best;
            lo = best + 1;
        }
        const int nid = lane < k ? int(uint32_t(mine)) : -1;
        bool found = false;
        for (int l = 0; l < k; ++l) found |= __shfl_sync(0xffffffffu, g, l) == nid;
        const unsigned fresh = __popc(__ballot_sync(0xffffffffu, lane < k && !found));
        if (lane == 0 && fresh) atomicAdd(updates, (unsigned long long)fresh);
        if (lane < k) {
            Gn[i * k + lane] = nid;
            Dn[i * k + lane] = __uint_as_float(uint32_t(mine >> 32));
        }
        __syncwarp();  // the next point reuses this warp's shared memory
    }
}

// Squared FP32 distances of a graph's entries (the start's, for the reverse
// lists of the first iteration).
template <bool PAIRS>
__global__ void nnd_graph_dist_kernel(const float* __restrict__ X, int d, int k, const int32_t* __restrict__ G,
                                      int64_t nk, float* __restrict__ D2) {
    for (int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < nk; t += int64_t(gridDim.x) * blockDim.x)
        D2[t] = nnd_dist2<PAIRS>(X + int64_t(G[t]) * d, X + (t / k) * d, d);
}

// Reverse lists: count the entries pointing at each point, scan, fill
// (owner, distance) pairs in any order, then keep per point the k of
// smallest (distance, owner), exactly, by k rounds of a warp minimum.
__global__ void nnd_rcount_kernel(const int32_t* __restrict__ G, int64_t nk, int32_t* __restrict__ cnt) {
    for (int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < nk; t += int64_t(gridDim.x) * blockDim.x)
        atomicAdd(&cnt[G[t]], 1);
}

__global__ void nnd_rfill_kernel(const int32_t* __restrict__ G, const float* __restrict__ D2, int64_t nk, int k,
                                 const int32_t* __restrict__ start, int32_t* __restrict__ cur,
                                 uint64_t* __restrict__ rkey) {
    for (int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < nk; t += int64_t(gridDim.x) * blockDim.x) {
        const int32_t tgt = G[t];
        const int pos = atomicAdd(&cur[tgt], 1);
        rkey[start[tgt] + pos] = (uint64_t(__float_as_uint(D2[t])) << 32) | uint32_t(t / k);
    }
}

__global__ void nnd_rselect_kernel(const int32_t* __restrict__ start, const uint64_t* __restrict__ rkey, int64_t n,
                                   int k, int32_t* __restrict__ R) {
    const int lane = threadIdx.x & 31;
    for (int64_t i = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; i < n;
         i += (int64_t(gridDim.x) * blockDim.x) >> 5) {
        const int32_t e0 = start[i], e1 = start[i + 1];
        uint64_t lo = 0, mine = ~0ull;
        for (int r = 0; r < k; ++r) {
            uint64_t best = ~0ull;
            for (int32_t e = e0 + lane; e < e1; e += 32) {
                const uint64_t key = rkey[e];
                if (key >= lo && key < best) best = key;
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const uint64_t ob = __shfl_xor_sync(0xffffffffu, best, o);
                best = ob < best ? ob : best;
            }
            if (lane == r) mine = best;
            lo = best + 1;
        }
        if (lane < k) R[i * k + lane] = mine == ~0ull ? -1 : int32_t(uint32_t(mine));
    }
}

__global__ void nnd_final_kernel(const int32_t* __restrict__ G, const float* __restrict__ D2, int64_t nk,
                                 int32_t* __restrict__ idx, float* __restrict__ dist) {
    for (int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < nk; t += int64_t(gridDim.x) * blockDim.x) {
        idx[t] = G[t];
        dist[t] = sqrtf(D2[t]);
    }
}

size_t nnd_scratch_bytes(int64_t n, int k, bool reverse) {
    const size_t nk = size_t(n) * k;
    size_t b = 2 * Carve::round(nk * 4) + Carve::round(nk * 4) + 256 + 4096;
    if (reverse)
        b += 3 * Carve::round(size_t(n + 1) * 4) + Carve::round(scan_scratch_elems(n) * 4) + Carve::round(nk * 8) +
             Carve::round(nk * 4);
    return b;
}

int nnd_run(Ctx* c, const float* X, int64_t n, int d, int k, uint64_t seed, double delta, int max_iter, bool rev,
            int32_t* idx_out, float* dist_out, int32_t* iters_out, double* rates_out, void* scratch,
            cudaStream_t st) {
    const size_t nk = size_t(n) * k;
    if (rev && 2 * k > 32) return set_error(c, DRGB_ERR_INVALID, "knn_nndescent: the reverse form takes k <= 16");
    Carve cv(scratch);
    int32_t* Ga = cv.take<int32_t>(nk);
    int32_t* Gb = cv.take<int32_t>(nk);
    float* D2 = cv.take<float>(nk);
    unsigned long long* upd = cv.take<unsigned long long>(4);
    int32_t *rcnt = nullptr, *rstart = nullptr, *rcur = nullptr, *stmp = nullptr, *R = nullptr;
    uint64_t* rkey = nullptr;
    if (rev) {
        rcnt = cv.take<int32_t>(n + 1);
        rstart = cv.take<int32_t>(n + 1);
        rcur = cv.take<int32_t>(n + 1);
        stmp = cv.take<int32_t>(scan_scratch_elems(n));
        rkey = cv.take<uint64_t>(nk);
        R = cv.take<int32_t>(nk);
    }
    const NndLayout L = nnd_layout(k, d, rev);
    int wpb = NND_WARPS;
    while (wpb > 1 && size_t(wpb) * L.bytes > NND_SMEM_CAP) wpb >>= 1;
    if (size_t(wpb) * L.bytes > NND_SMEM_CAP)
        return set_error(c, DRGB_ERR_INVALID, "knn_nndescent: k = %d, d = %d need too much shared memory", k, d);
    const bool pairs = (d % 2 == 0) && aligned(X, 8);
    const size_t smem = size_t(wpb) * L.bytes;
    auto kern = pairs ? (rev ? nnd_iter_kernel<true, true> : nnd_iter_kernel<true, false>)
                      : (rev ? nnd_iter_kernel<false, true> : nnd_iter_kernel<false, false>);
    DRGB_CUDA(c, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
    int per_sm = 0;
    DRGB_CUDA(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, wpb * 32, smem));
    const int64_t need = (n + wpb - 1) / wpb;
    const int64_t cap = int64_t(c->num_sms) * (per_sm > 0 ? per_sm : 1) * 8;
    const unsigned grid = unsigned(need < cap ? need : cap);

    nnd_init_kernel<<<grid_for(n, 128, c->num_sms * 16), 128, 0, st>>>(n, k, uint32_t(seed), uint32_t(seed >> 32), Ga);
    DRGB_CHECK_LAUNCH(c);
    const int eg = grid_for(int64_t(nk), 256, c->num_sms * 8);
    if (rev) {  // the start's distances, for the first reverse lists
        if (pairs) nnd_graph_dist_kernel<true><<<eg, 256, 0, st>>>(X, d, k, Ga, int64_t(nk), D2);
        else nnd_graph_dist_kernel<false><<<eg, 256, 0, st>>>(X, d, k, Ga, int64_t(nk), D2);
        DRGB_CHECK_LAUNCH(c);
    }
    int it = 0;
    for (; it < max_iter;) {
        if (rev) {
            DRGB_CUDA(c, cudaMemsetAsync(rcnt, 0, size_t(n) * 4, st));
            DRGB_CUDA(c, cudaMemsetAsync(rcur, 0, size_t(n) * 4, st));
            nnd_rcount_kernel<<<eg, 256, 0, st>>>(Ga, int64_t(nk), rcnt);
            DRGB_CHECK_LAUNCH(c);
            int rc = exclusive_scan(c, rcnt, rstart, n, stmp, st);
            if (rc) return rc;
            nnd_rfill_kernel<<<eg, 256, 0, st>>>(Ga, D2, int64_t(nk), k, rstart, rcur, rkey);
            DRGB_CHECK_LAUNCH(c);
            nnd_rselect_kernel<<<grid_for(n * 32, 256, c->num_sms * 8), 256, 0, st>>>(rstart, rkey, n, k, R);
            DRGB_CHECK_LAUNCH(c);
        }
        DRGB_CUDA(c, cudaMemsetAsync(upd, 0, sizeof(unsigned long long), st));
        kern<<<grid, wpb * 32, smem, st>>>(X, n, d, k, L, Ga, R, Gb, D2, upd);
        DRGB_CHECK_LAUNCH(c);
        unsigned long long h = 0;
        DRGB_CUDA(c, cudaMemcpyAsync(&h, upd, sizeof(h), cudaMemcpyDeviceToHost, st));
        DRGB_CUDA(c, cudaStreamSynchronize(st));
        std::swap(Ga, Gb);
        const double rate = double(h) / (double(n) * double(k));
        if (rates_out) rates_out[it] = rate;
        ++it;
        if (rate < delta) break;
    }
    nnd_final_kernel<<<grid_for(int64_t(nk), 256, c->num_sms * 8), 256, 0, st>>>(Ga, D2, int64_t(nk), idx_out, dist_out);
    DRGB_CHECK_LAUNCH(c);
    if (iters_out) *iters_out = it;
    return DRGB_OK;
}

}  // namespace drgb

using namespace drgb;

extern "C" int drgb_knn_nndescent(drgb_ctx* c, const float* X, int64_t n, int32_t d, int32_t k, uint64_t seed,
                                  double delta, int32_t max_iter, int32_t reverse, int32_t* idx_out,
                                  float* dist_out, int32_t* iterations, double* rates, void* stream) {
    int rc = check_knn_args(c, X, n, d, k, idx_out, dist_out);
    if (rc) return rc;
    if (!(delta >= 0.0 && delta <= 1.0) || max_iter < 1 || max_iter > NND_MAX_ITER || d > NND_MAX_D)
        return set_error(c, DRGB_ERR_INVALID, "knn_nndescent: need 0 <= delta <= 1, 1 <= max_iter <= %d, d <= %d",
                         NND_MAX_ITER, NND_MAX_D);
    if (reverse && k > 16) return set_error(c, DRGB_ERR_INVALID, "knn_nndescent: the reverse form takes k <= 16");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if ((rc = ensure_scratch(c, nnd_scratch_bytes(n, k, reverse != 0), st))) return rc;
    if ((rc = launch_nonfinite_scan(c, X, n * d, st))) return rc;
    rc = nnd_run(c, X, n, d, k, seed, delta, max_iter, reverse != 0, idx_out, dist_out, iterations, rates,
                 c->scratch, st);
    if (rc) return rc;
    return drgb_sync(c, stream);
}
