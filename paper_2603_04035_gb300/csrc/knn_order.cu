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

static constexpr int ORD_SUB = 1536;      // largest subsample for the pivot choice (distance matrix 9.4 MB)
static constexpr int ORD_PER_PIVOT = 16;  // subsample points per pivot
static constexpr int ORD_THREADS = 1024;
static constexpr int ORD_PPT = (ORD_SUB + ORD_THREADS - 1) / ORD_THREADS;  // subsample points per thread
static constexpr int ORD_CHUNK = 512;     // points per counting-sort chunk (one warp each)
static constexpr int ORD_DMAX = 64;       // widest row the order supports

// Subsample point i of m: splitmix64(i) mod n, a fixed pseudo-random sample
// (a strided sample aliases with periodic point orders such as labels i mod c).
__device__ __forceinline__ int64_t sub_point(int i, int64_t n) {
    uint64_t z = uint64_t(i) + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    return int64_t(z % uint64_t(n));
}

// Row pitch of the FP16 subsample in half2 words: odd, so that the rows the
// lanes of a warp read at one offset fall in distinct shared-memory banks.
static inline int sub_pitch(int d) { return ((d + 1) / 2) | 1; }

// S[i][c] = dimensions (2c, 2c + 1) of subsample point i as FP16 (zero past d).
__global__ void sub_gather_kernel(const float* __restrict__ X, int64_t n, int d, int m, int pitch,
                                  __half2* __restrict__ S) {
    const int64_t total = int64_t(m) * pitch;
    for (int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < total; t += int64_t(gridDim.x) * blockDim.x) {
        const int i = int(t / pitch), c = int(t % pitch) * 2;
        const int64_t r = sub_point(i, n) * d;
        S[t] = __floats2half2_rn(c < d ? X[r + c] : 0.f, c + 1 < d ? X[r + c + 1] : 0.f);
    }
}

// Squared distances between the points of the FP16 subsample S, as FP32 sums
// over the dimension pairs in order: Dm[p m + i] = |s_i - s_p|^2 (block p
// holds row p; symmetric, since fl(a - b) = -fl(b - a)).
__global__ void sub_dist_kernel(const __half2* __restrict__ S, int m, int pitch, float* __restrict__ Dm) {
    extern __shared__ __align__(16) __half2 s_p[];  // [pitch]: point p
    const int p = blockIdx.x;
    for (int c = threadIdx.x; c < pitch; c += blockDim.x) s_p[c] = S[int64_t(p) * pitch + c];
    __syncthreads();
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
        const __half2* xv = S + int64_t(i) * pitch;
        float sq = 0.f;
#pragma unroll 4
        for (int c = 0; c < pitch; ++c) {
            const float2 a = __half22float2(xv[c]), b = __half22float2(s_p[c]);
            float df = a.x - b.x;
            sq = fmaf(df, df, sq);
            df = a.y - b.y;
            sq = fmaf(df, df, sq);
        }
        Dm[int64_t(p) * m + i] = sq;
    }
}

// Farthest-point sampling in one CTA over the subsample's distance matrix Dm
// (the pivot choice is a heuristic; any deterministic choice is valid).
// Pivot 0 is the first subsample point; pivot it + 1 is the subsample point
// farthest from pivots 0..it (ties: the lowest subsample index).  Each thread
// keeps the running minimum distances of its ORD_PPT points in registers and
// reads row p of Dm for the new pivot p; one barrier per step (the per-warp
// maxima are double-buffered by step parity).
__global__ void __launch_bounds__(ORD_THREADS) fps_cta_kernel(const float* __restrict__ Dm, int64_t n, int m, int K,
                                                           int32_t* __restrict__ pivots) {
    __shared__ unsigned long long s_best[2][32];
    float mn[ORD_PPT];
#pragma unroll
    for (int j = 0; j < ORD_PPT; ++j) mn[j] = INFINITY;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int p = 0;
    for (int it = 0; it < K; ++it) {
        if (threadIdx.x == 0) pivots[it] = int32_t(sub_point(p, n));
        if (it == K - 1) break;
        const float* row = Dm + int64_t(p) * m;
        unsigned long long best = 0;
#pragma unroll
        for (int j = 0; j < ORD_PPT; ++j) {
            const int i = threadIdx.x + j * ORD_THREADS;
            if (i < m) {
                mn[j] = fminf(mn[j], row[i]);
                const unsigned long long key = (uint64_t(__float_as_uint(mn[j])) << 32) | uint64_t(~uint32_t(i));
                best = key > best ? key : best;
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long other = __shfl_xor_sync(0xffffffffu, best, o);
            best = other > best ? other : best;
        }
        unsigned long long* sb = s_best[it & 1];
        if (lane == 0) sb[warp] = best;
        __syncthreads();
        unsigned long long bb = sb[lane];  // ORD_THREADS / 32 = 32 warps
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long other = __shfl_xor_sync(0xffffffffu, bb, o);
            bb = other > bb ? other : bb;
        }
        p = int(~uint32_t(bb & 0xffffffffull));
    }
}

// Nearest centre of every point (exact FP32, dimensions summed in order; ties:
// the lower centre) and its distance.  Centres are zero-padded to ORD_DMAX
// dimensions in shared memory and the point's row to ORD_DMAX registers, so
// the padded terms add exactly 0.
__global__ void __launch_bounds__(256) cell_assign_kernel(const float* __restrict__ X, int64_t n, int d,
                                                         const float* __restrict__ centre, int K,
                                                         int32_t* __restrict__ cell, float* __restrict__ cdist) {
    extern __shared__ __align__(16) float s_c[];  // [K][ORD_DMAX]
    for (int t = threadIdx.x; t < K * ORD_DMAX; t += blockDim.x) {
        const int k = t / ORD_DMAX, c = t % ORD_DMAX;
        s_c[t] = c < d ? centre[k * d + c] : 0.f;
    }
    __syncthreads();
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float x[ORD_DMAX];
#pragma unroll
    for (int c = 0; c < ORD_DMAX; ++c) x[c] = c < d ? X[i * d + c] : 0.f;
    float bd = INFINITY;
    int32_t bk = 0;
    for (int k = 0; k < K; ++k) {
        const float4* cv = reinterpret_cast<const float4*>(s_c + k * ORD_DMAX);
        float sq = 0.f;
#pragma unroll
        for (int c4 = 0; c4 < ORD_DMAX / 4; ++c4) {
            const float4 v = cv[c4];
            float df = x[4 * c4] - v.x;
            sq = fmaf(df, df, sq);
            df = x[4 * c4 + 1] - v.y;
            sq = fmaf(df, df, sq);
            df = x[4 * c4 + 2] - v.z;
            sq = fmaf(df, df, sq);
            df = x[4 * c4 + 3] - v.w;
            sq = fmaf(df, df, sq);
        }
        if (sq < bd) {
            bd = sq;
            bk = k;
        }
    }
    cell[i] = bk;
    cdist[i] = sqrtf(bd);
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
    const int64_t m = n < ORD_SUB ? n : ORD_SUB;
    return Carve::round(size_t(K) * 4) + Carve::round(size_t(m) * sub_pitch(d) * 4) + Carve::round(size_t(m) * m * 4) +
           Carve::round(size_t(n) * 4) * 2 + 2 * Carve::round(kc * 4) + Carve::round(scan_scratch_elems(int64_t(kc)) * 4) +
           4096;
}

int knn_order(Ctx* c, const float* X, int64_t n, int d, int K, int32_t* perm, int32_t* cell_beg, float* centre,
              float* radius, void* scratch, cudaStream_t st) {
    if (d > ORD_DMAX) return set_error(c, DRGB_ERR_INVALID, "knn order: d > 64");
    if (K > 128) return set_error(c, DRGB_ERR_INVALID, "knn order: more than 128 cells");
    int64_t m64 = int64_t(K) * ORD_PER_PIVOT;
    if (m64 > ORD_SUB) m64 = ORD_SUB;
    if (m64 > n) m64 = n;
    const int m = int(m64), pitch = sub_pitch(d);
    const int nchunk = int((n + ORD_CHUNK - 1) / ORD_CHUNK);
    const size_t kc = size_t(K) * nchunk;
    Carve cv(scratch);
    int32_t* pivots = cv.take<int32_t>(K);
    __half2* S = cv.take<__half2>(size_t(m) * pitch);
    float* Dm = cv.take<float>(size_t(m) * m);
    int32_t* cell = cv.take<int32_t>(n);
    float* cdist = cv.take<float>(n);
    int32_t* counts = cv.take<int32_t>(kc);
    int32_t* offs = cv.take<int32_t>(kc);
    int32_t* tmp = cv.take<int32_t>(scan_scratch_elems(int64_t(kc)));

    sub_gather_kernel<<<grid_for(int64_t(m) * pitch, 256, c->num_sms), 256, 0, st>>>(X, n, d, m, pitch, S);
    DRGB_CHECK_LAUNCH(c);
    sub_dist_kernel<<<m, 256, size_t(pitch) * 4, st>>>(S, m, pitch, Dm);
    DRGB_CHECK_LAUNCH(c);
    fps_cta_kernel<<<1, ORD_THREADS, 0, st>>>(Dm, n, m, K, pivots);
    DRGB_CHECK_LAUNCH(c);
    // the pivots are the cells' centres; a cell's radius is the largest
    // distance from its points to its pivot (the assignment's own distances)
    gather_rows_kernel<<<grid_for(int64_t(K) * d, 256, c->num_sms), 256, 0, st>>>(X, d, pivots, K, centre);
    DRGB_CHECK_LAUNCH(c);
    const size_t asm_bytes = size_t(K) * ORD_DMAX * 4;
    DRGB_CUDA(c, cudaFuncSetAttribute(cell_assign_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(asm_bytes)));
    cell_assign_kernel<<<unsigned((n + 255) / 256), 256, asm_bytes, st>>>(X, n, d, centre, K, cell, cdist);
    DRGB_CHECK_LAUNCH(c);
    int rc = DRGB_OK;
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
