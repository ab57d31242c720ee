// Spatial ordering of the points for the tensor-core k-NN: K pivots chosen by
// farthest-point sampling on a hashed subsample (one CTA), every point assigned to its
// nearest pivot (exact FP32 scan), a stable counting sort by pivot ("cell"),
// and a bounding sphere per cell (the pivot and the largest distance of the
// cell's points to it).  The order only decides which database
// tiles a query block visits first and which it may skip; the k-NN result
// does not depend on it (skipped cells enter the certificate as a distance
// bound, and rows the bound cannot certify are scanned exactly).
#include <cuda_fp16.h>

#include "common.cuh"
#include "knn.cuh"

namespace drgb {

static constexpr int ORD_SUB = 1536;      // subsample size for the pivot choice (one CTA)
static constexpr int ORD_THREADS = 256;
static constexpr int ORD_CHUNK = 4096;    // points per counting-sort chunk (one warp each)

// Subsample point i of m: splitmix64(i) mod n, a fixed pseudo-random sample
// (a strided sample aliases with periodic point orders such as labels i mod c).
__device__ __forceinline__ int64_t sub_point(int i, int64_t n) {
    uint64_t z = uint64_t(i) + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    return int64_t(z % uint64_t(n));
}

// Farthest-point sampling in one CTA: the subsample is held in shared memory
// as FP16 (the pivot choice is a heuristic; any deterministic choice is
// valid).  Pivot 0 is the first subsample point;
// pivot it + 1 is the subsample point farthest from pivots 0..it (ties: the
// lowest subsample index).
__global__ void __launch_bounds__(ORD_THREADS) fps_cta_kernel(const float* __restrict__ X, int64_t n, int d, int m,
                                                           int K, int32_t* __restrict__ pivots) {
    extern __shared__ __align__(16) uint8_t s_raw[];
    float* s_min = reinterpret_cast<float*>(s_raw);                 // [m]
    unsigned long long* s_best = reinterpret_cast<unsigned long long*>(s_min + ORD_SUB);  // [32]
    __half* s_x = reinterpret_cast<__half*>(s_best + 32);          // [m][d]
    for (int t = threadIdx.x; t < m * d; t += blockDim.x) {
        const int i = t / d, c = t % d;
        s_x[t] = __float2half_rn(X[sub_point(i, n) * d + c]);
    }
    for (int i = threadIdx.x; i < m; i += blockDim.x) s_min[i] = INFINITY;
    __syncthreads();
    int p = 0;
    for (int it = 0; it < K; ++it) {
        if (threadIdx.x == 0) pivots[it] = int32_t(sub_point(p, n));
        if (it == K - 1) break;
        unsigned long long best = 0;
        for (int i = threadIdx.x; i < m; i += blockDim.x) {
            float sq = 0.f;
            for (int c = 0; c < d; ++c) {
                const float df = __half2float(s_x[i * d + c]) - __half2float(s_x[p * d + c]);
                sq = fmaf(df, df, sq);
            }
            const float v = fminf(s_min[i], sq);
            s_min[i] = v;
            const unsigned long long key = (uint64_t(__float_as_uint(v)) << 32) | uint64_t(~uint32_t(i));
            best = key > best ? key : best;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long other = __shfl_xor_sync(0xffffffffu, best, o);
            best = other > best ? other : best;
        }
        if ((threadIdx.x & 31) == 0) s_best[threadIdx.x >> 5] = best;
        __syncthreads();
        if (threadIdx.x < 32) {
            unsigned long long b = threadIdx.x < (blockDim.x >> 5) ? s_best[threadIdx.x] : 0ull;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const unsigned long long other = __shfl_xor_sync(0xffffffffu, b, o);
                b = other > b ? other : b;
            }
            if (threadIdx.x == 0) s_best[0] = b;
        }
        __syncthreads();
        p = int(~uint32_t(s_best[0] & 0xffffffffull));
        __syncthreads();
    }
}

__global__ void gather_rows_kernel(const float* __restrict__ X, int d, const int32_t* __restrict__ rows, int count,
                                   float* __restrict__ out) {
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < count * d; t += gridDim.x * blockDim.x)
        out[t] = X[int64_t(rows[t / d]) * d + t % d];
}

// Per chunk of ORD_CHUNK points: how many fall in each cell, and (radius
// bits, atomicMax) the largest distance of a point to its cell's pivot.
__global__ void cell_count_kernel(const int32_t* __restrict__ cell, const float* __restrict__ cdist, int64_t n,
                                  int K, int nchunk, int32_t* __restrict__ counts, unsigned int* __restrict__ rbits) {
    extern __shared__ int32_t s_cnt[];  // [K] counts, [K] radius bits
    unsigned int* s_r = reinterpret_cast<unsigned int*>(s_cnt + K);
    for (int c = threadIdx.x; c < K; c += blockDim.x) {
        s_cnt[c] = 0;
        s_r[c] = 0u;
    }
    __syncthreads();
    const int64_t b0 = int64_t(blockIdx.x) * ORD_CHUNK;
    for (int64_t i = b0 + threadIdx.x; i < b0 + ORD_CHUNK && i < n; i += blockDim.x) {
        atomicAdd(&s_cnt[cell[i]], 1);
        atomicMax(&s_r[cell[i]], __float_as_uint(cdist[i]));
    }
    __syncthreads();
    for (int c = threadIdx.x; c < K; c += blockDim.x) {
        counts[int64_t(c) * nchunk + blockIdx.x] = s_cnt[c];
        if (s_r[c]) atomicMax(&rbits[c], s_r[c]);
    }
}

// Stable scatter: one warp walks its chunk in index order, 32 points a round;
// a point's position is its cell's offset for this chunk plus the number of
// earlier points of the chunk in the same cell.
__global__ void cell_scatter_kernel(const int32_t* __restrict__ cell, int64_t n, int K, int nchunk,
                                    const int32_t* __restrict__ offs, int32_t* __restrict__ perm) {
    extern __shared__ int32_t s_run[];  // [warps][K]
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    int32_t* run = s_run + w * K;
    const int chunk = blockIdx.x * nw + w;
    if (chunk >= nchunk) return;
    for (int c = lane; c < K; c += 32) run[c] = offs[int64_t(c) * nchunk + chunk];
    __syncwarp();
    const unsigned lt = (1u << lane) - 1u;
    const int64_t b0 = int64_t(chunk) * ORD_CHUNK;
    for (int64_t r = b0; r < b0 + ORD_CHUNK && r < n; r += 32) {
        const int64_t i = r + lane;
        const bool v = i < n && i < b0 + ORD_CHUNK;
        const int32_t c = v ? cell[i] : -1 - lane;
        const unsigned peers = __match_any_sync(0xffffffffu, c);
        int32_t base = 0;
        if (v) base = run[c];
        __syncwarp();
        if (v) {
            perm[base + __popc(peers & lt)] = int32_t(i);
            if (lane == __ffs(peers) - 1) run[c] = base + __popc(peers);
        }
        __syncwarp();
    }
}

__global__ void cell_begin_kernel(const int32_t* __restrict__ offs, int K, int nchunk, int64_t n,
                                  int32_t* __restrict__ cell_beg) {
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c <= K; c += gridDim.x * blockDim.x)
        cell_beg[c] = c < K ? offs[int64_t(c) * nchunk] : int32_t(n);
}

int knn_order_cells(int64_t n) {
    int64_t K = n / 2048;
    if (K < 16) K = 16;
    if (K > 128) K = 128;
    return int(K);
}

size_t knn_order_scratch_bytes(int64_t n, int d, int K) {
    const int64_t nchunk = (n + ORD_CHUNK - 1) / ORD_CHUNK;
    const size_t kc = size_t(K) * nchunk;
    return Carve::round(size_t(K) * 4) + Carve::round(size_t(n) * 4) * 2 + 2 * Carve::round(kc * 4) +
           Carve::round(scan_scratch_elems(int64_t(kc)) * 4) + 4096;
}

int knn_order(Ctx* c, const float* X, int64_t n, int d, int K, int32_t* perm, int32_t* cell_beg, float* centre,
              float* radius, void* scratch, cudaStream_t st) {
    if (d > 64) return set_error(c, DRGB_ERR_INVALID, "knn order: d > 64");
    const int m = int(n < ORD_SUB ? n : ORD_SUB);
    const int nchunk = int((n + ORD_CHUNK - 1) / ORD_CHUNK);
    const size_t kc = size_t(K) * nchunk;
    Carve cv(scratch);
    int32_t* pivots = cv.take<int32_t>(K);
    int32_t* cell = cv.take<int32_t>(n);
    float* cdist = cv.take<float>(n);
    int32_t* counts = cv.take<int32_t>(kc);
    int32_t* offs = cv.take<int32_t>(kc);
    int32_t* tmp = cv.take<int32_t>(scan_scratch_elems(int64_t(kc)));

    const size_t fsm = size_t(ORD_SUB) * 4 + 32 * 8 + size_t(m) * d * 2;
    DRGB_CUDA(c, cudaFuncSetAttribute(fps_cta_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(fsm)));
    fps_cta_kernel<<<1, ORD_THREADS, fsm, st>>>(X, n, d, m, K, pivots);
    DRGB_CHECK_LAUNCH(c);
    // the pivots are the cells' centres; a cell's radius is the largest
    // distance from its points to its pivot (the assignment's own distances)
    gather_rows_kernel<<<grid_for(int64_t(K) * d, 256, c->num_sms), 256, 0, st>>>(X, d, pivots, K, centre);
    DRGB_CHECK_LAUNCH(c);
    int rc = launch_knn_query(c, X, n, centre, K, d, 1, cell, cdist, st);
    if (rc) return rc;
    DRGB_CUDA(c, cudaMemsetAsync(radius, 0, size_t(K) * 4, st));
    cell_count_kernel<<<nchunk, 256, size_t(K) * 8, st>>>(cell, cdist, n, K, nchunk, counts,
                                                         reinterpret_cast<unsigned int*>(radius));
    DRGB_CHECK_LAUNCH(c);
    if ((rc = exclusive_scan(c, counts, offs, int64_t(kc), tmp, st))) return rc;
    const int sw = 4;  // warps (chunks) per CTA of the scatter
    cell_scatter_kernel<<<(nchunk + sw - 1) / sw, 32 * sw, size_t(sw) * K * 4, st>>>(cell, n, K, nchunk, offs,
                                                                                    perm);
    DRGB_CHECK_LAUNCH(c);
    cell_begin_kernel<<<1, 256, 0, st>>>(offs, K, nchunk, n, cell_beg);
    DRGB_CHECK_LAUNCH(c);
    return DRGB_OK;
}

}  // namespace drgb
