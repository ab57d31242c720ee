// Exact k-NN through a BF16 tensor-core distance GEMM (tcgen05, TMEM, TMA),
// a fused per-row top-k' selection, an FP32 re-rank of the candidates and a
// certificate that proves the candidate set holds the exact FP32 k nearest.
//
// Stage (A1): the columns are centred (distances are translation invariant,
// centring shrinks the rounding error), scaled by a power of two S, rounded to
// the 16-bit operand type and written as two K = 64 operand matrices
//     XA_i = [ x~_i, C, C, C, 0 ... ]       XB_j = [ -2 x~_j, h_j, m_j, l_j, 0 ... ]
// where C (h + m + l) is a three-way 16-bit split of n_j = |x~_j|^2 (FP32).
// The tensor-core product XA_i . XB_j is then s_ij = n_j - 2 x~_i . x~_j, and
// the squared distance between the rounded points is n_i + s_ij.  For a fixed
// query row i, ordering by s is ordering by distance, so the epilogue needs
// no norms at all.  Two operand types share the code: BF16 (S = C = 1) and
// FP16 (S scales max |x - mean| to 2^10, C = 2^15), whose 11-bit significand
// leaves an 8x smaller rounding residual at the same tensor-core rate.
//
// GEMM + select (A2): one CTA owns 128 query rows (TMEM lanes) and streams the
// database tiles of 256 rows that its cell schedule admits (points are staged
// in the spatial cell order of knn_order.cu; see knn_tc_kernel for the cell
// bounds).  Warp 0 issues TMA loads into a 4-stage ring,
// warp 1 issues 4 MMAs (M128 N256 K16) per tile into one of two TMEM
// accumulators, and 8 epilogue warps (two per TMEM lane quarter, one per
// column half) read the accumulator with tcgen05.ld, reject a 32-column chunk
// with one min-reduction unless it can enter the row's list, and keep the
// best 32 (s, j) pairs per row sorted in registers.
//
// Re-rank + certify (A3): exact FP32 squared distances sum_c (x_ic - x_jc)^2
// of the 32 candidates (the same arithmetic as the FP32 scan), top-k by
// (distance, index).  With delta_i = |x_i - x~_i| (BF16 rounding residual)
// and eps_i bounding the FP32 accumulation error, every point outside the
// list is at distance >= sqrt(n_i + s_thr - eps_i) - delta_i - delta_max if
// its tile was multiplied or its cell skipped (a skipped cell lies beyond the
// row's upper bound, which is at least that), and beyond lbstop, the bound at
// which the schedule stopped, otherwise.  If the smaller of the two exceeds
// the k-th exact distance the row is certified; other rows are recomputed by
// the exact FP32 scan.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "common.cuh"
#include "knn.cuh"
#include "tc_ptx.cuh"

namespace drgb {

static constexpr int TC_BM = 128;
static constexpr int TC_BN = 256;
static constexpr int TC_K = 64;
static constexpr int TC_STAGES = 3;
static constexpr int TC_KP = 32;                 // candidates kept per row
static constexpr int TC_EPI_WARPS = 8;
static constexpr int TC_THREADS = 64 + TC_EPI_WARPS * 32;
static constexpr int TC_A_BYTES = TC_BM * TC_K * 2;   // 16 KiB
static constexpr int TC_B_BYTES = TC_BN * TC_K * 2;   // 32 KiB
static constexpr int TC_TMEM_COLS = 512;               // two 256-column accumulators
static constexpr int TC_QCAP = 32;                     // per-thread candidate queue slots (one chunk)
static constexpr size_t TC_QUEUE_BYTES = size_t(TC_EPI_WARPS) * 32 * TC_QCAP * 8;
static constexpr int TC_NQ = 4;                       // list quantiles a column half publishes
static constexpr size_t TC_THR_BYTES = size_t(2) * TC_BM * TC_NQ * 4;   // per (column half, row) quantiles
static constexpr int TC_CELLS = 128;                   // most cells a schedule may hold
static constexpr int TC_GROUPS = 4;                    // row groups (runs of one cell) bounded separately
static constexpr int TC_RING = 16;                     // tile-index ring (slots in flight < 16)
static constexpr int TC_MAX_TILES = 98304;             // database tiles the visited-tile bitmap covers
static constexpr size_t TC_SCHED_BYTES =
    size_t(TC_CELLS) * 8 + size_t(TC_GROUPS) * TC_CELLS * 4 + 32 + TC_BM * 4 + TC_RING * 8 + 64 + TC_MAX_TILES / 8 +
    size_t(2) * TC_BM * 4;
static constexpr size_t TC_SMEM =
    1024 + TC_A_BYTES + TC_STAGES * TC_B_BYTES + 256 + TC_QUEUE_BYTES + TC_THR_BYTES + TC_SCHED_BYTES;

// Compare-exchange of (value, index) pairs i < l: afterwards the pair at i is
// the smaller (asc) or the larger (!asc) of the two values.
__device__ __forceinline__ void cas(float& vi, int32_t& ii, float& vl, int32_t& il, bool asc) {
    const bool sw = asc ? (vl < vi) : (vi < vl);
    const float a = vi, b = vl;
    const int32_t x = ii, y = il;
    vi = sw ? b : a;
    vl = sw ? a : b;
    ii = sw ? y : x;
    il = sw ? x : y;
}

// Bitonic merge of a bitonic sequence of N (power of two) into ascending order.
template <int N>
__device__ __forceinline__ void bitonic_merge_asc(float (&v)[N], int32_t (&ix)[N]) {
#pragma unroll
    for (int j = N / 2; j > 0; j >>= 1) {
#pragma unroll
        for (int i = 0; i < N; ++i)
            if ((i & j) == 0) cas(v[i], ix[i], v[i + j], ix[i + j], true);
    }
}

// Bitonic sort of N (power of two) into ascending order.
template <int N>
__device__ __forceinline__ void bitonic_sort_asc(float (&v)[N], int32_t (&ix)[N]) {
#pragma unroll
    for (int k = 2; k <= N; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
#pragma unroll
            for (int i = 0; i < N; ++i) {
                const int l = i ^ j;
                if (l > i) cas(v[i], ix[i], v[l], ix[l], (i & k) == 0);
            }
        }
    }
}

// Three-input minimum (sm_100 and later).
__device__ __forceinline__ float min3f(float a, float b, float c) {
    float r;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}

// ------------------------------------------------------------------ A1: staging
typedef uint16_t op16;  // raw 16-bit operand (BF16 or FP16 bits)

template <bool F16>
__device__ __forceinline__ op16 to_op(float v) {
    if constexpr (F16) return __half_as_ushort(__float2half_rn(v));
    else return __bfloat16_as_ushort(__float2bfloat16_rn(v));
}
template <bool F16>
__device__ __forceinline__ float from_op(op16 b) {
    if constexpr (F16) return __half2float(__ushort_as_half(b));
    else return __bfloat162float(__ushort_as_bfloat16(b));
}

// Power-of-two operand scale: FP16 maps max |x - mean| to at most 2^10.
template <bool F16>
__device__ __forceinline__ float operand_scale(const unsigned int* maxbits) {
    if constexpr (!F16) return 1.0f;
    const float amax = __uint_as_float(maxbits[2]);
    if (!(amax > 0.f)) return 1.0f;
    int e;
    frexpf(amax, &e);                      // amax < 2^e
    return ldexpf(1.0f, e - 10);
}

// Column statistics of X (d <= 64) for the operand staging.  Block b sums,
// and takes the minimum and maximum of, every column over its range of rows
// (a warp per row, lanes on dimensions (lane, lane + 32)) into partial[b]; the
// last block to finish (ticket maxbits[3]) reduces the partials to the column
// means (summed in double) and the largest |x - mean| (maxbits[2]).  Rounding
// is monotone, so over a column the largest fl(x - m) is fl(max - m) and the
// largest fl(m - x) is fl(m - min): this equals max |fl(x - m)| elementwise.
static constexpr int TC_STAT_WARPS = 8;

__global__ void __launch_bounds__(TC_STAT_WARPS * 32)
tc_colstats_kernel(const float* __restrict__ X, int64_t n, int d, float* __restrict__ partial,
                   float* __restrict__ mean, unsigned int* __restrict__ maxbits) {
    __shared__ float s_sum[TC_STAT_WARPS][64], s_lo[TC_STAT_WARPS][64], s_hi[TC_STAT_WARPS][64];
    __shared__ bool s_last;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t per = (n + gridDim.x - 1) / gridDim.x;
    const int64_t r0 = int64_t(blockIdx.x) * per;
    const int64_t r1 = r0 + per < n ? r0 + per : n;
    const bool in0 = lane < d, in1 = lane + 32 < d;
    float s0 = 0.f, s1 = 0.f, lo0 = INFINITY, lo1 = INFINITY, hi0 = -INFINITY, hi1 = -INFINITY;
#pragma unroll 4
    for (int64_t r = r0 + w; r < r1; r += TC_STAT_WARPS) {
        const float* xr = X + r * d;
        if (in0) {
            const float v = xr[lane];
            s0 += v;
            lo0 = fminf(lo0, v);
            hi0 = fmaxf(hi0, v);
        }
        if (in1) {
            const float v = xr[lane + 32];
            s1 += v;
            lo1 = fminf(lo1, v);
            hi1 = fmaxf(hi1, v);
        }
    }
    s_sum[w][lane] = s0;
    s_sum[w][lane + 32] = s1;
    s_lo[w][lane] = lo0;
    s_lo[w][lane + 32] = lo1;
    s_hi[w][lane] = hi0;
    s_hi[w][lane + 32] = hi1;
    __syncthreads();
    if (threadIdx.x < 64) {
        const int c = threadIdx.x;
        float s = 0.f, lo = INFINITY, hi = -INFINITY;
        for (int u = 0; u < TC_STAT_WARPS; ++u) {
            s += s_sum[u][c];
            lo = fminf(lo, s_lo[u][c]);
            hi = fmaxf(hi, s_hi[u][c]);
        }
        float* pb = partial + int64_t(blockIdx.x) * 3 * 64;
        pb[c] = s;
        pb[64 + c] = lo;
        pb[128 + c] = hi;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(&maxbits[3], 1u) == gridDim.x - 1;
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    // the partials of blocks g, g + G, ... (G = TC_STAT_WARPS * 32 / 64
    // groups per column) are summed by one thread each, eight blocks' loads
    // in flight at a time, and the groups are then added in order
    constexpr int G = TC_STAT_WARPS * 32 / 64;
    __shared__ double s_gs[G][64];
    __shared__ float s_glo[G][64], s_ghi[G][64];
    {
        const int c = threadIdx.x & 63, g = threadIdx.x >> 6;
        double sg = 0.0;
        float lo = INFINITY, hi = -INFINITY;
        const int nb = int(gridDim.x);
        for (int b0 = g; b0 < nb; b0 += 8 * G) {
            float vs[8], vl[8], vh[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int b = b0 + u * G;
                const float* pb = partial + int64_t(b < nb ? b : 0) * 3 * 64;
                vs[u] = b < nb ? __ldcg(pb + c) : 0.f;
                vl[u] = b < nb ? __ldcg(pb + 64 + c) : INFINITY;
                vh[u] = b < nb ? __ldcg(pb + 128 + c) : -INFINITY;
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                sg += double(vs[u]);
                lo = fminf(lo, vl[u]);
                hi = fmaxf(hi, vh[u]);
            }
        }
        s_gs[g][c] = sg;
        s_glo[g][c] = lo;
        s_ghi[g][c] = hi;
    }
    __syncthreads();
    if (threadIdx.x < d) {
        const int c = threadIdx.x;
        double sum = 0.0;
        float lo = INFINITY, hi = -INFINITY;
        for (int g = 0; g < G; ++g) {
            sum += s_gs[g][c];
            lo = fminf(lo, s_glo[g][c]);
            hi = fmaxf(hi, s_ghi[g][c]);
        }
        const float m = float(sum / double(n));
        mean[c] = m;
        const float amax = fmaxf(0.f, fmaxf(hi - m, m - lo));
        atomicMax(&maxbits[2], __float_as_uint(amax));
    }
}

// Warp per row: lanes own dimensions (lane, lane + 32).  Norms and residuals
// are stored in the original units (the scale S is a power of two).
// Position i of the operands holds point perm[i] (positions >= n: padding);
// norms and residuals are stored at the point's own index, and Xp (FP32, n x d)
// receives the rows in position order.  A warp takes STAGE_ROWS consecutive
// positions at a time and issues all their loads before using any.
static constexpr int STAGE_ROWS = 4;

template <bool F16>
__global__ void tc_stage_kernel(const float* __restrict__ X, int64_t n, int64_t n_pad, int d,
                                const float* __restrict__ mean, const int32_t* __restrict__ perm,
                                op16* __restrict__ XA, op16* __restrict__ XB, float* __restrict__ norm,
                                float* __restrict__ resid, unsigned int* __restrict__ maxbits,
                                float* __restrict__ Xp) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = int64_t(gridDim.x) * (blockDim.x >> 5);
    const float S = operand_scale<F16>(maxbits), inv_S = 1.0f / S;
    const float C = F16 ? 32768.0f : 1.0f, inv_C = 1.0f / C;
    const float m0 = lane < d ? mean[lane] : 0.f, m1 = lane + 32 < d ? mean[lane + 32] : 0.f;
    float nmax = 0.f, rmax = 0.f;
    for (int64_t i0 = (int64_t(blockIdx.x) * (blockDim.x >> 5) + (threadIdx.x >> 5)) * STAGE_ROWS; i0 < n_pad;
         i0 += warps * STAGE_ROWS) {
        int64_t src[STAGE_ROWS];
        float xr[STAGE_ROWS][2];
#pragma unroll
        for (int u = 0; u < STAGE_ROWS; ++u) src[u] = i0 + u < n ? int64_t(perm[i0 + u]) : -1;
#pragma unroll
        for (int u = 0; u < STAGE_ROWS; ++u)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int c = lane + 32 * h;
                xr[u][h] = (src[u] >= 0 && c < d) ? X[src[u] * d + c] : 0.f;
            }
#pragma unroll
        for (int u = 0; u < STAGE_ROWS; ++u) {
            const int64_t i = i0 + u;
            if (i >= n_pad) break;
            float xc[2], xb[2];
            float sq = 0.f, rs = 0.f, cs = 0.f;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int c = lane + 32 * h;
                float v = 0.f;
                if (i < n && c < d) {
                    const float x = xr[u][h];
                    Xp[i * d + c] = x;
                    v = (x - (h ? m1 : m0)) * inv_S;
                }
                xc[h] = v;
                xb[h] = from_op<F16>(to_op<F16>(v));
                sq = fmaf(xb[h], xb[h], sq);
                const float r = v - xb[h];
                rs = fmaf(r, r, rs);
                cs = fmaf(v, v, cs);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                sq += __shfl_xor_sync(0xffffffffu, sq, o);
                rs += __shfl_xor_sync(0xffffffffu, rs, o);
                cs += __shfl_xor_sync(0xffffffffu, cs, o);
            }
            // three-way split of n / C (huge for padding rows: never selected)
            const float nv = i < n ? sq * inv_C : (F16 ? 65504.0f : 3.0e38f);
            const op16 nh = to_op<F16>(nv);
            const float r1 = nv - from_op<F16>(nh);
            const op16 nm = to_op<F16>(r1);
            const op16 nl = to_op<F16>(r1 - from_op<F16>(nm));
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int c = lane + 32 * h;
                op16 a = to_op<F16>(xb[h]);
                op16 b = to_op<F16>(-2.0f * xb[h]);
                if (c == d || c == d + 1 || c == d + 2) {
                    a = to_op<F16>(C);
                    b = c == d ? nh : (c == d + 1 ? nm : nl);
                }
                XA[i * TC_K + c] = a;
                XB[i * TC_K + c] = b;
            }
            if (lane == 0) {
                // residual norm, widened by the FP32 rounding of the centring and
                // scaling and (FP16) by a possible flush of subnormal operands
                const float flush = F16 ? 6.2e-5f * sqrtf(float(d)) : 0.f;
                const float delta = (sqrtf(rs) * (1.0f + 1e-6f) + 2.4e-7f * sqrtf(cs) + flush) * S;
                if (i < n) {
                    norm[src[u]] = sq * S * S;
                    resid[src[u]] = delta;
                    nmax = fmaxf(nmax, sq * S * S);
                    rmax = fmaxf(rmax, delta);
                }
            }
            (void)xc;
        }
    }
    if (lane == 0) {
        atomicMax(&maxbits[0], __float_as_uint(nmax));
        atomicMax(&maxbits[1], __float_as_uint(rmax));
    }
}

// ------------------------------------------------------------------ A2: GEMM + top-k'
struct TcParams {
    int64_t n;
    int n_tiles;
    int32_t* cand_idx;   // n x TC_KP candidate positions, by query position
    float* cand_s;       // n x TC_KP
    int* status;
    // spatial schedule: positions p (rows of the staged operands) hold point
    // perm[p]; cell c holds positions [cell_beg[c], cell_beg[c+1]) and lies
    // in the sphere (cell_c[c], cell_r[c]) (original units)
    const float* X;
    int d;
    const int32_t* perm;
    int K;
    const int32_t* cell_beg;
    const float* cell_c;
    const float* cell_r;
    const float* norm;          // per point, original units (see the staging)
    const float* resid;
    const unsigned int* maxbits;
    float* lbstop;       // per position: no point of a skipped cell is nearer (original units)
    unsigned long long* tiles_done;  // += tiles this CTA multiplied
};

// Bitonic sort (ascending by (value, index)) of TC_CELLS pairs in shared
// memory by the whole CTA.
__device__ __forceinline__ void cta_sort_pairs(float* v, int32_t* ix) {
    for (int k = 2; k <= TC_CELLS; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            __syncthreads();
            for (int i = threadIdx.x; i < TC_CELLS; i += blockDim.x) {
                const int l = i ^ j;
                if (l > i) {
                    const bool asc = (i & k) == 0;
                    const float a = v[i], b = v[l];
                    const int32_t x = ix[i], y = ix[l];
                    const bool gt = a > b || (a == b && x > y);
                    if (gt == asc) {
                        v[i] = b;
                        v[l] = a;
                        ix[i] = y;
                        ix[l] = x;
                    }
                }
            }
        }
    }
    __syncthreads();
}

// Cell of position p: the c with cell_beg[c] <= p < cell_beg[c + 1].
__device__ __forceinline__ int cell_of(const int32_t* __restrict__ cell_beg, int K, int64_t p) {
    int lo = 0, hi = K - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (cell_beg[mid] <= p) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// One CTA per 128 query positions.  Before the pipeline starts, the CTA splits
// its rows into groups (rows are in cell order: each run of one cell is a
// group; rows past the fourth run join the last group), bounds every group by
// a sphere, computes for every (group, cell) a lower bound on the distance
// between any row of the group and any point of the cell, and sorts the cells
// by their smallest bound.  Warp 0 then streams the database tiles of the
// cells in that order (each tile once).  A cell is skipped when, for every
// group, its bound exceeds the largest current upper bound on a row's
// 32nd-nearest distance in that group (its points cannot enter any row's
// list), and the stream stops at the first cell whose smallest bound exceeds
// every group's: the same then holds for it and every later cell.  The bound
// at which it stopped is returned per row for the certificate.  Tile indices travel to
// the MMA and epilogue warps through a small ring; a slot holding -1 ends the
// stream.
template <bool F16>
__global__ void __launch_bounds__(TC_THREADS, 1)
knn_tc_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, TcParams P) {
    extern __shared__ uint8_t smem_raw[];
    // 1024-byte aligned (swizzled operand tiles); an offset from the shared
    // array, so that every pointer below stays a known shared-memory address
    uint8_t* base = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    uint8_t* sA = base;
    uint8_t* sB = base + TC_A_BYTES;
    uint64_t* bars = reinterpret_cast<uint64_t*>(sB + TC_STAGES * TC_B_BYTES);
    uint64_t* full = bars;                       // [TC_STAGES]
    uint64_t* empty = bars + TC_STAGES;          // [TC_STAGES]
    uint64_t* a_full = bars + 2 * TC_STAGES;     // [1]
    uint64_t* acc_full = a_full + 1;             // [2]
    uint64_t* acc_empty = acc_full + 2;          // [2]
    uint64_t* mma_done = acc_empty + 2;          // [1]
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(mma_done + 1);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
    // per epilogue thread: a queue of candidates (value bits, column) that
    // passed the threshold
    int2* q = reinterpret_cast<int2*>(reinterpret_cast<uint8_t*>(bars) + 256);
    // per (column half, row): the 8th, 16th, 24th and 32nd best values that
    // half's list holds so far
    float* s_thr = reinterpret_cast<float*>(q + TC_EPI_WARPS * 32 * TC_QCAP);
    // schedule: sorted cell bounds and cells, per-row distance bounds, the
    // tile ring (slot number and tile), misc words, visited-tile bitmap
    float* s_lb = s_thr + 2 * TC_BM * TC_NQ;
    int32_t* s_cl = reinterpret_cast<int32_t*>(s_lb + TC_CELLS);
    float* s_glb = reinterpret_cast<float*>(s_cl + TC_CELLS);                // [TC_GROUPS][TC_CELLS]
    int32_t* s_gb = reinterpret_cast<int32_t*>(s_glb + TC_GROUPS * TC_CELLS);  // [TC_GROUPS + 1] (+pad)
    volatile float* s_U = reinterpret_cast<volatile float*>(s_gb + 8);
    volatile int32_t* ring_t = reinterpret_cast<volatile int32_t*>(s_U + TC_BM);
    volatile int32_t* ring_tile = ring_t + TC_RING;
    float* s_misc = const_cast<float*>(reinterpret_cast<volatile float*>(ring_tile + TC_RING));  // [16]
    uint32_t* s_done = reinterpret_cast<uint32_t*>(s_misc + 16);
    // per row: the constant parts of its distance bound (see the epilogue)
    float* s_ua = reinterpret_cast<float*>(s_done + TC_MAX_TILES / 32);
    float* s_uc = s_ua + TC_BM;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t q0 = int64_t(blockIdx.x) * TC_BM;
    const int nrow = int(P.n - q0 < TC_BM ? P.n - q0 : TC_BM);

    if (threadIdx.x == 0) {
        for (int s = 0; s < TC_STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(a_full, 1);
        for (int b = 0; b < 2; ++b) {
            mbar_init(&acc_full[b], 1);
            mbar_init(&acc_empty[b], TC_EPI_WARPS);
        }
        mbar_init(mma_done, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(smem_u32(tmem_slot)), "r"(TC_TMEM_COLS) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    // ---------------- schedule (all warps; the B ring is still idle and holds
    // the block's rows meanwhile)
    {
        float* s_rows = reinterpret_cast<float*>(sB);    // [TC_BM][64]
        float* s_gcen = s_rows + TC_BM * 64;             // [TC_GROUPS][64] group centres
        unsigned int* s_grad = reinterpret_cast<unsigned int*>(s_gcen + TC_GROUPS * 64);  // radius bits
        float* s_gcn = reinterpret_cast<float*>(s_grad + TC_GROUPS);                     // |centre|
        for (int t = threadIdx.x; t < TC_BM * 64; t += blockDim.x) {
            const int r = t >> 6, c = t & 63;
            s_rows[t] = (r < nrow && c < P.d) ? P.X[int64_t(P.perm[q0 + r]) * P.d + c] : 0.f;
        }
        for (int t = threadIdx.x; t < TC_MAX_TILES / 32; t += blockDim.x) s_done[t] = 0u;
        if (threadIdx.x < TC_BM) s_U[threadIdx.x] = INFINITY;
        if (threadIdx.x < TC_RING) {
            ring_t[threadIdx.x] = -1;
            ring_tile[threadIdx.x] = -1;
        }
        if (threadIdx.x <= TC_GROUPS) s_gb[threadIdx.x] = nrow;
        if (threadIdx.x < TC_GROUPS) s_grad[threadIdx.x] = 0u;
        if (threadIdx.x == 0) {
            s_misc[1] = INFINITY;   // stopping bound
            const float S = operand_scale<F16>(P.maxbits);
            s_misc[2] = S * S;      // threshold units -> squared distance units
        }
        __syncthreads();
        int grp = -1;
        if (threadIdx.x < nrow) {
            const int c0 = cell_of(P.cell_beg, P.K, q0);
            const int cr = cell_of(P.cell_beg, P.K, q0 + threadIdx.x);
            grp = cr - c0 < TC_GROUPS - 1 ? cr - c0 : TC_GROUPS - 1;
            atomicMin(&s_gb[grp], int32_t(threadIdx.x));
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            // group g holds rows [s_gb[g], s_gb[g + 1]) (empty groups: equal ends)
            for (int g = TC_GROUPS - 1; g >= 0; --g) s_gb[g] = s_gb[g] < s_gb[g + 1] ? s_gb[g] : s_gb[g + 1];
        }
        __syncthreads();
        if (threadIdx.x < 64) {
            for (int g = 0; g < TC_GROUPS; ++g) {
                const int r0 = s_gb[g], r1 = s_gb[g + 1];
                float sum = 0.f;
                for (int r = r0; r < r1; ++r) sum += s_rows[r * 64 + threadIdx.x];
                s_gcen[g * 64 + threadIdx.x] = r1 > r0 ? sum / float(r1 - r0) : 0.f;
            }
        }
        __syncthreads();
        if (grp >= 0) {
            float sq = 0.f;
            for (int c = 0; c < P.d; ++c) {
                const float df = s_rows[threadIdx.x * 64 + c] - s_gcen[grp * 64 + c];
                sq = fmaf(df, df, sq);
            }
            atomicMax(&s_grad[grp], __float_as_uint(sqrtf(sq)));
        }
        if (threadIdx.x < TC_GROUPS) {
            float cb2 = 0.f;
            for (int c = 0; c < P.d; ++c) cb2 = fmaf(s_gcen[threadIdx.x * 64 + c], s_gcen[threadIdx.x * 64 + c], cb2);
            s_gcn[threadIdx.x] = sqrtf(cb2);
        }
        __syncthreads();
        for (int ci = threadIdx.x; ci < TC_CELLS; ci += blockDim.x) {
            float lbmin = INFINITY;
            float lbg[TC_GROUPS];
#pragma unroll
            for (int g = 0; g < TC_GROUPS; ++g) lbg[g] = INFINITY;
            if (ci < P.K && P.cell_beg[ci + 1] > P.cell_beg[ci]) {
                float dd[TC_GROUPS], cc = 0.f;
#pragma unroll
                for (int g = 0; g < TC_GROUPS; ++g) dd[g] = 0.f;
                for (int c = 0; c < P.d; ++c) {
                    const float v = P.cell_c[int64_t(ci) * P.d + c];
                    cc = fmaf(v, v, cc);
#pragma unroll
                    for (int g = 0; g < TC_GROUPS; ++g) {
                        const float df = s_gcen[g * 64 + c] - v;
                        dd[g] = fmaf(df, df, dd[g]);
                    }
                }
                const float rc = P.cell_r[ci], cn = sqrtf(cc);
#pragma unroll
                for (int g = 0; g < TC_GROUPS; ++g) {
                    if (s_gb[g + 1] > s_gb[g]) {
                        const float dist = sqrtf(dd[g]), rb = __uint_as_float(s_grad[g]);
                        // FP32 rounding of the centres, radii and this distance
                        // is covered by a relative margin on everything involved
                        lbg[g] = fmaxf(0.f, dist - rb - rc - 1e-5f * (dist + rb + rc + s_gcn[g] + cn));
                        lbmin = fminf(lbmin, lbg[g]);
                    }
                }
            }
#pragma unroll
            for (int g = 0; g < TC_GROUPS; ++g) s_glb[g * TC_CELLS + ci] = lbg[g];
            s_lb[ci] = lbmin;
            s_cl[ci] = ci;
        }
        cta_sort_pairs(s_lb, s_cl);   // ends with __syncthreads
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        // ---------------- schedule + TMA producer (lane 0 issues)
        bool stop_ok = true;
        if (lane == 0) {
            mbar_expect_tx(a_full, TC_A_BYTES);
            tma_load_2d(sA, &tmA, 0, int(q0), a_full);
        }
        int t = 0;
        float lbstop = INFINITY;
        for (int ci = 0; ci < P.K && stop_ok; ++ci) {
            const float lb = s_lb[ci];
            if (!(lb < INFINITY)) break;  // empty cells sort last
            const int cell = s_cl[ci];
            // per group: the largest current bound of its rows; the cell is
            // needed when its bound for some group does not exceed that
            float umax = -INFINITY;
            bool need = false;
#pragma unroll
            for (int g = 0; g < TC_GROUPS; ++g) {
                const int r0 = s_gb[g], r1 = s_gb[g + 1];
                float u = -INFINITY;
                for (int r = r0 + lane; r < r1; r += 32) u = fmaxf(u, s_U[r]);
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) u = fmaxf(u, __shfl_xor_sync(0xffffffffu, u, o));
                umax = fmaxf(umax, u);
                need = need || s_glb[g * TC_CELLS + cell] <= u;
            }
            if (lb > umax) {
                lbstop = lb;
                break;
            }
            if (!need) continue;
            const int tb = P.cell_beg[cell] / TC_BN, te = (P.cell_beg[cell + 1] - 1) / TC_BN;
            for (int tile = tb; tile <= te && stop_ok; ++tile) {
                if (P.K > 1) {  // one cell covers every tile once: no bitmap needed
                    int seen = 0;
                    if (lane == 0) {
                        const uint32_t bit = 1u << (tile & 31);
                        seen = (s_done[tile >> 5] & bit) != 0;
                        s_done[tile >> 5] |= bit;
                    }
                    if (__shfl_sync(0xffffffffu, seen, 0)) continue;
                }
                if (lane == 0) {
                    const int s = t % TC_STAGES;
                    if (t >= TC_STAGES && !mbar_wait(&empty[s], ((t / TC_STAGES) & 1) ^ 1, abort_flag, P.status)) {
                        stop_ok = false;
                    } else {
                        ring_tile[t % TC_RING] = tile;
                        __threadfence_block();
                        ring_t[t % TC_RING] = t;
                        mbar_expect_tx(&full[s], TC_B_BYTES);
                        tma_load_2d(sB + s * TC_B_BYTES, &tmB, 0, tile * TC_BN, &full[s]);
                    }
                }
                stop_ok = __shfl_sync(0xffffffffu, stop_ok, 0);
                ++t;
            }
        }
        if (lane == 0) {
            s_misc[1] = lbstop;
            atomicAdd(P.tiles_done, static_cast<unsigned long long>(t));
            // loads issued: slots 0 .. issued - 1 (an aborted slot issued none)
            int issued = stop_ok ? t : t - 1;
            if (stop_ok) {
                // end of the stream: slot t carries tile -1 (no data)
                const int s = t % TC_STAGES;
                if (t < TC_STAGES || mbar_wait(&empty[s], ((t / TC_STAGES) & 1) ^ 1, abort_flag, P.status)) {
                    ring_tile[t % TC_RING] = -1;
                    __threadfence_block();
                    ring_t[t % TC_RING] = t;
                    mbar_arrive(&full[s]);
                } else {
                    stop_ok = false;
                }
            }
            if (!stop_ok) {
                // aborted: let every load already issued land before the CTA
                // exits (each wait bounded by 100 ms).  Slots before
                // issued - TC_STAGES were consumed by the MMA warp, whose
                // wait on them completed; their buffers were reused only
                // after that.  The A tile's load was issued first of all.
                for (int u = (issued > TC_STAGES ? issued - TC_STAGES : 0); u < issued; ++u) {
                    const unsigned long long t0 = global_timer();
                    while (!mbar_try(&full[u % TC_STAGES], (u / TC_STAGES) & 1) &&
                           global_timer() - t0 < 100000000ull) {
                    }
                }
                const unsigned long long t0 = global_timer();
                while (!mbar_try(a_full, 0) && global_timer() - t0 < 100000000ull) {
                }
            }
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer
        if (lane == 0) {
            const uint32_t idesc = idesc_f16kind(TC_BM, TC_BN, F16);
            const uint64_t adesc = sdesc_sw128(smem_u32(sA));
            bool ok = mbar_wait(a_full, 0, abort_flag, P.status);
            for (int t = 0; ok; ++t) {
                const int s = t % TC_STAGES, buf = t & 1, use = t >> 1;
                if (t >= 2 && !mbar_wait(&acc_empty[buf], (use & 1) ^ 1, abort_flag, P.status)) break;
                tc_fence_after();
                if (!mbar_wait(&full[s], (t / TC_STAGES) & 1, abort_flag, P.status)) break;
                tc_fence_after();
                if (ring_t[t % TC_RING] != t || ring_tile[t % TC_RING] < 0) {
                    mbar_arrive(&acc_full[buf]);  // end of the stream: pass it on
                    break;
                }
                const uint64_t bdesc = sdesc_sw128(smem_u32(sB + s * TC_B_BYTES));
#pragma unroll
                for (int k = 0; k < TC_K / 16; ++k)  // K step of 16 BF16 = 32 bytes = 2 descriptor units
                    mma_f16kind(tmem + uint32_t(buf * TC_BN), adesc + 2 * k, bdesc + 2 * k, idesc, k > 0);
                mma_commit(&empty[s]);
                mma_commit(&acc_full[buf]);
            }
            // every MMA issued above has completed once this barrier fires
            mma_commit(mma_done);
            const unsigned long long t0 = global_timer();
            while (!mbar_try(mma_done, 0) && global_timer() - t0 < 100000000ull) {
            }
        }
    } else {
        // ---------------- epilogue: warps 2..9
        const int e = warp - 2;
        const int quarter = warp & 3;             // TMEM lanes [32 quarter, 32 quarter + 32)
        const int half = e >> 2;                  // columns [128 half, 128 half + 128) of a tile
        const int row = quarter * 32 + lane;
        float L[TC_KP];
        int32_t I[TC_KP];
#pragma unroll
        for (int s = 0; s < TC_KP; ++s) {
            L[s] = INFINITY;
            I[s] = -1;
        }
        // this row's point (its norm and residual convert a threshold on s
        // into an upper bound on the distance of its 32nd candidate)
        const int64_t g_row = row < nrow ? int64_t(P.perm[q0 + row]) : -1;
        // the row's bound on its 32nd candidate's distance for threshold thr
        // is (sqrt(max(ua + thr S^2, 0)) + uc)(1 + 1e-5), ua = n_i + eps_i and
        // uc = resid_i + r_max (the relative margin covers FP32 rounding)
        if (half == 0) {
            float ua = INFINITY, uc = 0.f;
            if (g_row >= 0) {
                const float r_max = __uint_as_float(P.maxbits[1]), n_max = __uint_as_float(P.maxbits[0]);
                const float ni = P.norm[g_row];
                ua = ni + 6.103515625e-05f * (ni + n_max);
                uc = P.resid[g_row] + r_max;
            }
            s_ua[row] = ua;
            s_uc[row] = uc;
        }
        // Candidates below the row's threshold are appended to this thread's
        // queue (slot s at q[s * 256 + tid], conflict-free).  The threshold
        // is a bound on the row's 32nd-best value over both column halves:
        // each half publishes the 8th, 16th, 24th and 32nd values of its
        // sorted list, and for b in {0, 8, 16, 24, 32} the 32 - b smallest of
        // this half's list together with the b smallest of the other's are 32
        // distinct columns, so max(own[31 - b], other's b-th) bounds the
        // row's 32nd-best; the threshold is the smallest of the five.  A value
        // at or above it cannot be among the row's 32 best.  A stale (larger)
        // published value still bounds correctly, since a list only improves.
        // When a chunk would overflow any lane's queue, all lanes merge their
        // queues into their lists in lockstep: the queue (padded with +inf)
        // is sorted by a bitonic network, the 32 smallest of list and queue
        // are selected by pairing the list's upper half with the reversed
        // queue, and a bitonic merge restores the order.
        const int qb = e * 32 + lane;
        volatile float* q_mine = s_thr + (half * TC_BM + row) * TC_NQ;
        volatile float* q_other = s_thr + ((1 - half) * TC_BM + row) * TC_NQ;
#pragma unroll
        for (int j = 0; j < TC_NQ; ++j) q_mine[j] = INFINITY;
        asm volatile("bar.sync 1, %0;" ::"r"(TC_EPI_WARPS * 32) : "memory");
        // the row's threshold from this half's list and the other's quantiles
        auto row_bound = [&]() {
            const float o8 = q_other[0], o16 = q_other[1], o24 = q_other[2], o32 = q_other[3];
            float t = fminf(L[TC_KP - 1], o32);
            t = fminf(t, fmaxf(L[23], o8));
            t = fminf(t, fmaxf(L[15], o16));
            t = fminf(t, fmaxf(L[7], o24));
            return t;
        };
        int qn = 0;
        auto flush = [&]() {
            float qv[TC_QCAP];
            int32_t qi[TC_QCAP];
#pragma unroll
            for (int s = 0; s < TC_QCAP; ++s) {
                const int2 c = s < qn ? q[s * (TC_EPI_WARPS * 32) + qb] : make_int2(__float_as_int(INFINITY), -1);
                qv[s] = __int_as_float(c.x);
                qi[s] = c.y;
            }
            bitonic_sort_asc<TC_QCAP>(qv, qi);
            // the 32 smallest of L and Q: min(L[s], Q[31 - s]) is bitonic
#pragma unroll
            for (int s = 0; s < TC_KP; ++s) {
                const bool take = qv[TC_KP - 1 - s] < L[s];
                L[s] = take ? qv[TC_KP - 1 - s] : L[s];
                I[s] = take ? qi[TC_KP - 1 - s] : I[s];
            }
            bitonic_merge_asc<TC_KP>(L, I);
            qn = 0;
            q_mine[0] = L[7];
            q_mine[1] = L[15];
            q_mine[2] = L[23];
            q_mine[3] = L[TC_KP - 1];
            const float thr = row_bound();
            if (g_row >= 0 && thr < INFINITY)
                s_U[row] = (sqrtf(fmaxf(s_ua[row] + thr * s_misc[2], 0.f)) + s_uc[row]) * (1.0f + 1e-5f);
        };
        for (int t = 0;; ++t) {
            const int buf = t & 1, use = t >> 1;
            if (!mbar_wait(&acc_full[buf], use & 1, abort_flag, P.status)) break;
            tc_fence_after();
            // the slot's tile (written before its data was requested)
            int tile = -1;
            {
                const unsigned long long w0 = global_timer();
                while (ring_t[t % TC_RING] != t) {
                    if (*abort_flag || global_timer() - w0 > TC_TIMEOUT_NS) break;
                }
                __threadfence_block();
                if (ring_t[t % TC_RING] == t) tile = ring_tile[t % TC_RING];
            }
            if (tile < 0) break;
            const uint32_t tbase = tmem + (uint32_t(quarter * 32) << 16) + uint32_t(buf * TC_BN + half * 128);
            const int32_t j0 = tile * TC_BN + half * 128;
            // the row's threshold, with the other half's quantiles read once
            // per tile (stale, larger, values still bound correctly)
            float thr_t = row_bound();
#pragma unroll 1
            for (int c = 0; c < 4; ++c) {
                float v[32];
                __syncwarp();
                tmem_ld32(tbase + c * 32, v);
                float thr = thr_t;
                float gm[4];
#pragma unroll
                for (int g = 0; g < 4; ++g)
                    gm[g] = min3f(min3f(v[8 * g], v[8 * g + 1], v[8 * g + 2]),
                                  min3f(v[8 * g + 3], v[8 * g + 4], v[8 * g + 5]), fminf(v[8 * g + 6], v[8 * g + 7]));
                const float m = fminf(min3f(gm[0], gm[1], gm[2]), gm[3]);
                if (__any_sync(0xffffffffu, m < thr)) {
                    // room for this chunk's candidates: a bound from the groups
                    // first, the exact count only when the bound overflows
                    const int ub = 8 * ((gm[0] < thr) + (gm[1] < thr) + (gm[2] < thr) + (gm[3] < thr));
                    if (__any_sync(0xffffffffu, qn + ub > TC_QCAP)) {
                        int cnt = 0;
#pragma unroll
                        for (int u = 0; u < 32; ++u) cnt += v[u] < thr ? 1 : 0;
                        if (__any_sync(0xffffffffu, qn + cnt > TC_QCAP)) {
                            // the chunk is read again after the merge, which
                            // keeps its 32 values out of registers meanwhile
                            flush();
                            __syncwarp();
                            tmem_ld32(tbase + c * 32, v);
                            thr = thr_t = row_bound();
                        }
                    }
#pragma unroll
                    for (int g = 0; g < 4; ++g) {
                        if (__any_sync(0xffffffffu, gm[g] < thr)) {
#pragma unroll
                            for (int u = 0; u < 8; ++u) {
                                if (v[8 * g + u] < thr) {
                                    q[qn * (TC_EPI_WARPS * 32) + qb] =
                                        make_int2(__float_as_int(v[8 * g + u]), j0 + c * 32 + 8 * g + u);
                                    ++qn;
                                }
                            }
                        }
                    }
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&acc_empty[buf]);
        }
        flush();
        // merge the two column halves of each row through shared memory (the
        // B ring is idle once the last accumulator has been read)
        float* ms = reinterpret_cast<float*>(sB);                 // [2][128][TC_KP]
        int32_t* mi = reinterpret_cast<int32_t*>(sB + 2 * TC_BM * TC_KP * 4);
        asm volatile("bar.sync 1, %0;" ::"r"(TC_EPI_WARPS * 32) : "memory");
#pragma unroll
        for (int s = 0; s < TC_KP; ++s) {
            ms[(half * TC_BM + row) * TC_KP + s] = L[s];
            mi[(half * TC_BM + row) * TC_KP + s] = I[s];
        }
        asm volatile("bar.sync 1, %0;" ::"r"(TC_EPI_WARPS * 32) : "memory");
        if (half == 0 && row < nrow && !*abort_flag) {
            const int64_t g = q0 + row;
            const float* As = ms + row * TC_KP;
            const int32_t* Ai = mi + row * TC_KP;
            const float* Bs = ms + (TC_BM + row) * TC_KP;
            const int32_t* Bi = mi + (TC_BM + row) * TC_KP;
            int a = 0, b = 0;
            for (int o = 0; o < TC_KP; ++o) {
                const bool take_a = (As[a] < Bs[b]) || (As[a] == Bs[b] && uint32_t(Ai[a]) <= uint32_t(Bi[b]));
                const int32_t pos = take_a ? Ai[a] : Bi[b];
                P.cand_s[g * TC_KP + o] = take_a ? As[a] : Bs[b];
                P.cand_idx[g * TC_KP + o] = pos;
                if (take_a) ++a; else ++b;
            }
            P.lbstop[g] = s_misc[1];
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_TMEM_COLS)
                     : "memory");
    }
}

// ------------------------------------------------------------------ A3: re-rank + certify
// One warp per row: lane l takes candidate l.  The 32 candidate rows are
// staged in shared memory (coalesced), each lane sums its candidate's squared
// distance over the dimensions in order (the FP32 scan's arithmetic, so every
// mode returns the same bits), and a bitonic network over the lanes orders the
// candidates by (distance, index).
// Asynchronous 4-byte copy global -> shared (completes at cp.async.wait_group).
__device__ __forceinline__ void cp_async4(float* dst, const float* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}

static constexpr int RR_WARPS = 4;

// Floats per staged row.  Odd d: d rounded up to an odd count, so that the
// lanes of a warp reading one column of 32 rows hit 32 distinct banks.  Even
// d (rows read as float pairs): twice an odd number of pairs, which keeps the
// 64-bit reads of a half-warp on distinct bank pairs.
static inline int rr_pitch(int d) { return (d & 1) ? d : 2 * ((d >> 1) | 1); }
static inline size_t rr_smem(int d) { return size_t(RR_WARPS) * (32 * rr_pitch(d) + 64) * 4; }

__device__ __forceinline__ void cp_async8(float* dst, const float* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}

// PAIRS (even d): rows are copied and read as float pairs, lane l taking
// dimensions (2l, 2l + 1); the dimensions are still added in order, so both
// forms give the same bits.
template <bool F16, bool PAIRS>
__global__ void __launch_bounds__(RR_WARPS * 32)
tc_rerank_kernel(const float* __restrict__ Xp, const int32_t* __restrict__ perm, int64_t n, int d, int k,
                 const int32_t* __restrict__ cand_pos, const float* __restrict__ cand_s,
                 const float* __restrict__ norm, const float* __restrict__ resid,
                 const unsigned int* __restrict__ maxbits, const float* __restrict__ lbstop,
                 int32_t* __restrict__ idx_out, float* __restrict__ dist_out, int32_t* __restrict__ fail_rows,
                 int32_t* __restrict__ fail_count) {
    extern __shared__ __align__(16) float s_rr[];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int pitch = PAIRS ? 2 * ((d >> 1) | 1) : d;
    float* s_rows = s_rr + w * (32 * pitch + 64);   // [32][pitch] candidate rows
    float* s_q = s_rows + 32 * pitch;               // [64] the query row
    const float n_max = __uint_as_float(maxbits[0]);
    const float r_max = __uint_as_float(maxbits[1]);
    const float S = operand_scale<F16>(maxbits);
    const int64_t warps = int64_t(gridDim.x) * RR_WARPS;
    // rows in position order: neighbouring warps share candidates in L2
    for (int64_t p = int64_t(blockIdx.x) * RR_WARPS + w; p < n; p += warps) {
        const int64_t i = perm[p];
        const int32_t q = cand_pos[p * TC_KP + lane];
        const bool valid = q >= 0 && q < n && q != p;
        // stage the query row and the 32 candidate rows with asynchronous
        // copies: all of a lane's copies are in flight together and hold no
        // registers
        const int qv = valid ? q : -1;
        if constexpr (PAIRS) {
            const int h = d >> 1;
            if (lane < h) cp_async8(s_q + 2 * lane, Xp + p * d + 2 * lane);
#pragma unroll 8
            for (int t = 0; t < 32; ++t) {
                const int32_t qt = __shfl_sync(0xffffffffu, qv, t);
                if (qt >= 0 && lane < h) cp_async8(s_rows + t * pitch + 2 * lane, Xp + int64_t(qt) * d + 2 * lane);
            }
        } else {
            for (int c = lane; c < d; c += 32) cp_async4(s_q + c, Xp + p * d + c);
#pragma unroll 8
            for (int t = 0; t < 32; ++t) {
                const int32_t qt = __shfl_sync(0xffffffffu, qv, t);
                if (qt >= 0) {
                    const float* src = Xp + int64_t(qt) * d;
                    if (lane < d) cp_async4(s_rows + t * pitch + lane, src + lane);
                    if (lane + 32 < d) cp_async4(s_rows + t * pitch + lane + 32, src + lane + 32);
                }
            }
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
        asm volatile("cp.async.wait_group 0;" ::: "memory");
        __syncwarp();
        float a = INFINITY;
        int32_t jj = INT32_MAX;
        if (valid) {
            a = 0.f;
            if constexpr (PAIRS) {
                const float2* row2 = reinterpret_cast<const float2*>(s_rows + lane * pitch);
                const float2* q2 = reinterpret_cast<const float2*>(s_q);
#pragma unroll 5
                for (int c2 = 0; c2 < (d >> 1); ++c2) {
                    const float2 x = q2[c2], y = row2[c2];
                    float df = x.x - y.x;
                    a = fmaf(df, df, a);
                    df = x.y - y.y;
                    a = fmaf(df, df, a);
                }
            } else {
                for (int c = 0; c < d; ++c) {
                    const float df = s_q[c] - s_rows[lane * pitch + c];
                    a = fmaf(df, df, a);
                }
            }
            jj = perm[q];
        }
        // bitonic sort across the lanes, ascending by (a, point index)
#pragma unroll
        for (int kk = 2; kk <= 32; kk <<= 1) {
#pragma unroll
            for (int st = kk >> 1; st > 0; st >>= 1) {
                const float oa = __shfl_xor_sync(0xffffffffu, a, st);
                const int32_t oj = __shfl_xor_sync(0xffffffffu, jj, st);
                const bool up = (lane & kk) == 0, lower = (lane & st) == 0;
                const bool self_less = a < oa || (a == oa && jj < oj);
                if (self_less != (lower == up)) {
                    a = oa;
                    jj = oj;
                }
            }
        }
        const int n_valid = __popc(__ballot_sync(0xffffffffu, valid));
        const float dk2 = __shfl_sync(0xffffffffu, a, k - 1);
        if (lane < k) {
            idx_out[i * k + lane] = jj;
            dist_out[i * k + lane] = sqrtf(a);
        }
        if (lane == 0) {
            // certificate: every point outside the list is beyond lb (points
            // never compared lie in skipped cells, beyond lbstop)
            const float s_thr = cand_s[p * TC_KP + TC_KP - 1] * (S * S);
            const float ni = norm[i];
            const float eps = 6.103515625e-05f * (ni + n_max);  // 2^-14 (n_i + n_max)
            const float lb2 = ni + s_thr - eps;
            const float lb = fminf(sqrtf(fmaxf(lb2, 0.f)) - resid[i] - r_max, lbstop[p]);
            const bool ok = n_valid >= k && lb > sqrtf(dk2) * (1.0f + 3.8e-6f);
            if (!ok) fail_rows[atomicAdd(fail_count, 1)] = int32_t(i);
        }
        __syncwarp();
    }
}

// Exact re-scan of the uncertified rows over the cells they can reach.  The
// cells are cut into chunks of at most CH positions (chunk_beg[C] = the first
// chunk of cell C; chunks of one cell are consecutive), so that a large cell
// does not become one long scan.  CTA (chunk y, listed row r) scans chunk y
// of its cell C for row q = rows[r], unless the cell's sphere lies beyond the
// row's re-ranked k-th distance u.
// For a point p of C, |x_q - p| >= |x_q - c_C| - |p - c_C|; the FP32 values
// D~ of |x_q - c_C| and r~_C >= max |p - c_C| carry a relative error below
// 1e-5 each (sums of at most 61 squares), and a point that can enter the
// row's k nearest has FP32 distance <= u, exact distance <= u (1 + 1.1e-5).
// So C is skipped when D~ - r~_C - 1e-5 (D~ + r~_C) > u (1 + 2e-5).
// The scan itself is the FP32 scan's arithmetic: squared distance
// sum_c (x_qc - p_c)^2 over the dimensions in order, kept when below the
// admission bound of the k-th distance, per thread sorted by distance, then
// merged by (distance, index) within each warp and over the CTA's warps into
// partial list (y, r), which launch_merge_partials combines over the chunks.
// Within a cell, positions follow the point index (the cell sort is stable),
// so every per-thread list is ordered by (distance, index).  The cell's
// points are staged 128 at a time with asynchronous copies into two
// alternating buffers, the next tile in flight while the current one is used.
static constexpr int RS_THREADS = 128;
static constexpr int RS_PITCH = 65;  // floats per staged point (d <= 61), odd: conflict-free
static constexpr size_t RS_SMEM = size_t(2) * RS_THREADS * RS_PITCH * 4;
static constexpr int64_t RS_CHUNK_MIN = 2048;  // positions per chunk of a cell (at least)

// chunk_beg[C] = sum over cells c < C of ceil(|c| / CH) (one CTA, K <= 128).
__global__ void tc_chunks_kernel(const int32_t* __restrict__ cell_beg, int K, int32_t CH,
                                 int32_t* __restrict__ chunk_beg) {
    if (threadIdx.x != 0) return;
    int32_t acc = 0;
    for (int c = 0; c < K; ++c) {
        chunk_beg[c] = acc;
        acc += (cell_beg[c + 1] - cell_beg[c] + CH - 1) / CH;
    }
    chunk_beg[K] = acc;
}

template <int KL>
__global__ void __launch_bounds__(RS_THREADS)
tc_rescan_kernel(const float* __restrict__ X, const float* __restrict__ Xp, const int32_t* __restrict__ perm,
                 int d, int k, const int32_t* __restrict__ rows, int cnt, int K, int32_t CH,
                 const int32_t* __restrict__ cell_beg, const int32_t* __restrict__ chunk_beg,
                 const float* __restrict__ cell_c, const float* __restrict__ cell_r,
                 const float* __restrict__ dist_in, int32_t* __restrict__ pidx, float* __restrict__ pd2) {
    extern __shared__ __align__(16) float s_pts[];   // [2][RS_THREADS][RS_PITCH]
    __shared__ float s_x[64];
    __shared__ float s_part[RS_THREADS / 32];
    __shared__ float s_wd[RS_THREADS / 32][32];
    __shared__ int32_t s_wi[RS_THREADS / 32][32];
    const int y = blockIdx.x, r = blockIdx.y, t = threadIdx.x, lane = t & 31, w = t >> 5;
    const int32_t q = rows[r];
    const int64_t out = (int64_t(y) * cnt + r) * k;
    if (y >= chunk_beg[K]) {  // past the last chunk
        if (t == 0) pidx[out] = -1;
        return;
    }
    int C = 0;  // the cell holding chunk y: the last C with chunk_beg[C] <= y
    for (int lo = 0, hi = K - 1; lo <= hi;) {
        const int mid = (lo + hi) >> 1;
        if (chunk_beg[mid] <= y) {
            C = mid;
            lo = mid + 1;
        } else {
            hi = mid - 1;
        }
    }
    for (int c = t; c < 64; c += RS_THREADS) s_x[c] = c < d ? X[int64_t(q) * d + c] : 0.f;
    __syncthreads();
    float part = 0.f;
    for (int c = t; c < d; c += RS_THREADS) {
        const float df = s_x[c] - cell_c[int64_t(C) * d + c];
        part = fmaf(df, df, part);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    if (lane == 0) s_part[w] = part;
    __syncthreads();
    const float Dc = sqrtf(s_part[0] + s_part[1] + s_part[2] + s_part[3]);
    const float rc = cell_r[C];
    const float u = dist_in[int64_t(q) * k + k - 1];
    if (Dc - rc - 1e-5f * (Dc + rc) > u * (1.0f + 2e-5f)) {  // false for u = INFINITY
        if (t == 0) pidx[out] = -1;
        return;
    }
    // admission bound: as in the FP32 scan's re-scan (the smallest normal
    // number keeps a k-th distance of 0 admitting distance 0)
    float T = fmaf(u * u, 1.0f + 1e-6f, 1.17549435e-38f);
    if (!(T < INFINITY)) T = INFINITY;
    float D[KL];
    int32_t I[KL];
#pragma unroll
    for (int s2 = 0; s2 < KL; ++s2) {
        D[s2] = T;
        I[s2] = -1;
    }
    const int32_t b = cell_beg[C] + (y - chunk_beg[C]) * CH;
    const int32_t e = cell_beg[C + 1] - b < CH ? cell_beg[C + 1] : b + CH;
    // warp w copies points w, w + 4, ... of a tile, lanes on dimensions
    // (lane, lane + 32)
    auto stage = [&](int32_t p0, float* buf) {
        const int m = e - p0 < RS_THREADS ? e - p0 : RS_THREADS;
        for (int row = w; row < m; row += RS_THREADS / 32) {
            const float* src = Xp + int64_t(p0 + row) * d;
            if (lane < d) cp_async4(buf + row * RS_PITCH + lane, src + lane);
            if (lane + 32 < d) cp_async4(buf + row * RS_PITCH + lane + 32, src + lane + 32);
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
    if (b < e) stage(b, s_pts);
    int buf = 0;
    for (int32_t p0 = b; p0 < e; p0 += RS_THREADS, buf ^= 1) {
        const bool more = p0 + RS_THREADS < e;
        if (more) {
            stage(p0 + RS_THREADS, s_pts + (buf ^ 1) * RS_THREADS * RS_PITCH);
            asm volatile("cp.async.wait_group 1;" ::: "memory");
        } else {
            asm volatile("cp.async.wait_group 0;" ::: "memory");
        }
        __syncthreads();
        const float* tile = s_pts + buf * RS_THREADS * RS_PITCH;
        if (p0 + t < e) {
            float a = 0.f;
            for (int c = 0; c < d; ++c) {
                const float df = s_x[c] - tile[t * RS_PITCH + c];
                a = fmaf(df, df, a);
            }
            if (a < D[KL - 1]) {
                const int32_t j = perm[p0 + t];
                if (j != q) topk_insert<KL>(D, I, a, j);
            }
        }
        __syncthreads();  // the buffer is refilled two tiles later
    }
    // the warp's k best by (distance, index): k rounds of a warp-wide minimum
    // over the lanes' list heads, the owner popping its head
    for (int s2 = 0; s2 < k; ++s2) {
        float bd = I[0] >= 0 ? D[0] : INFINITY;
        int32_t bi = I[0] >= 0 ? I[0] : INT32_MAX;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float od = __shfl_xor_sync(0xffffffffu, bd, o);
            const int32_t oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (od < bd || (od == bd && oi < bi)) {
                bd = od;
                bi = oi;
            }
        }
        if (lane == 0) {
            s_wd[w][s2] = bd;
            s_wi[w][s2] = bi == INT32_MAX ? -1 : bi;
        }
        if (I[0] >= 0 && I[0] == bi && D[0] == bd) {
#pragma unroll
            for (int s3 = 0; s3 < KL - 1; ++s3) {
                D[s3] = D[s3 + 1];
                I[s3] = I[s3 + 1];
            }
            D[KL - 1] = T;
            I[KL - 1] = -1;
        }
    }
    __syncthreads();
    // the CTA's k best from the four sorted warp lists (lanes 0..3 hold heads)
    if (w == 0) {
        int ptr = 0;
        for (int s2 = 0; s2 < k; ++s2) {
            float hd = INFINITY;
            int32_t hi = INT32_MAX;
            if (lane < RS_THREADS / 32 && ptr < k && s_wi[lane][ptr] >= 0) {
                hd = s_wd[lane][ptr];
                hi = s_wi[lane][ptr];
            }
            float bd = hd;
            int32_t bi = hi;
#pragma unroll
            for (int o = 2; o > 0; o >>= 1) {
                const float od = __shfl_xor_sync(0xffffffffu, bd, o);
                const int32_t oi = __shfl_xor_sync(0xffffffffu, bi, o);
                if (od < bd || (od == bd && oi < bi)) {
                    bd = od;
                    bi = oi;
                }
            }
            if (lane == 0) {
                pidx[out + s2] = bi == INT32_MAX ? -1 : bi;
                pd2[out + s2] = bd;
            }
            if (lane < RS_THREADS / 32 && hi == bi && hd == bd && bi != INT32_MAX) ++ptr;
        }
    }
}

// Positions past n hold themselves (padding); with a single cell the whole
// order is the identity and the cell covers every position.
__global__ void tc_identity_kernel(int32_t* __restrict__ perm, int64_t n, int64_t n_pad, bool all,
                                   int32_t* __restrict__ cell_beg, float* __restrict__ cell_r) {
    for (int64_t p = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; p < n_pad; p += int64_t(gridDim.x) * blockDim.x)
        if (all || p >= n) perm[p] = int32_t(p);
    if (all && blockIdx.x == 0 && threadIdx.x == 0) {
        cell_beg[0] = 0;
        cell_beg[1] = int32_t(n);
        cell_r[0] = INFINITY;
    }
}

// ------------------------------------------------------------------ host
bool knn_tc_preferred(int64_t n, int d, int k) { return n >= 4096 && d + 3 <= TC_K && k < TC_KP; }

// partial lists of the exact re-scan of uncertified rows (up to this many bytes)
static constexpr size_t TC_PART_BYTES = size_t(64) << 20;

static int tc_cells(int64_t n_pad, int64_t n) { return n_pad / TC_BN > TC_MAX_TILES ? 1 : knn_order_cells(n); }

static size_t tc_scratch_bytes(int64_t n, int d, int64_t n_pad, int nblk) {
    const int K = tc_cells(n_pad, n);
    return Carve::round(size_t(nblk) * 3 * 64 * 4) + Carve::round(d * 4) + 2 * Carve::round(n_pad * TC_K * 2) +
           2 * Carve::round(n_pad * 4) + Carve::round(64) + 2 * Carve::round(n_pad * TC_KP * 4) +
           Carve::round(n * 4) + Carve::round(64) + TC_PART_BYTES + Carve::round(n_pad * 4) +
           Carve::round((TC_CELLS + 1) * 4) + Carve::round(size_t(TC_CELLS) * d * 4) + Carve::round(TC_CELLS * 4) +
           Carve::round(n * 4) + Carve::round(size_t(n) * d * 4) + (K > 1 ? knn_order_scratch_bytes(n, d, K) : 0) +
           16384;
}

static constexpr int TC_COLSUM_BLOCKS = 256;

size_t knn_tc_scratch_bytes(int64_t n, int d) {
    const int64_t n_pad = (n + TC_BN - 1) / TC_BN * TC_BN;
    return tc_scratch_bytes(n, d, n_pad, TC_COLSUM_BLOCKS);
}

size_t knn_rescan_part_bytes() { return TC_PART_BYTES; }

template <bool F16>
static int knn_tc_impl(Ctx* c, const float* X, int64_t n, int d, int k, int32_t* idx_out, float* dist_out,
                       cudaStream_t st, void* scratch, int32_t* defer_rows, int32_t* defer_count) {
    if (d + 3 > TC_K || k >= TC_KP)
        return set_error(c, DRGB_ERR_INVALID, "knn_graph: tensor-core mode needs d <= %d and k < %d", TC_K - 3,
                         TC_KP);
    const int64_t n_pad = (n + TC_BN - 1) / TC_BN * TC_BN;
    const int nblk = TC_COLSUM_BLOCKS;
    int rc = DRGB_OK;
    Carve cv(scratch);
    float* partial = cv.take<float>(size_t(nblk) * 3 * 64);
    float* mean = cv.take<float>(d);
    op16* XA = cv.take<op16>(n_pad * TC_K);
    op16* XB = cv.take<op16>(n_pad * TC_K);
    float* norm = cv.take<float>(n_pad);
    float* resid = cv.take<float>(n_pad);
    unsigned int* maxbits = cv.take<unsigned int>(16);
    int32_t* cand_idx = cv.take<int32_t>(n_pad * TC_KP);
    float* cand_s = cv.take<float>(n_pad * TC_KP);
    int32_t* fail_rows = cv.take<int32_t>(n);
    int32_t* fail_count = cv.take<int32_t>(16);
    void* part = cv.take<char>(TC_PART_BYTES);
    int32_t* perm = cv.take<int32_t>(n_pad);
    int32_t* cell_beg = cv.take<int32_t>(TC_CELLS + 1);
    float* cell_c = cv.take<float>(size_t(TC_CELLS) * d);
    float* cell_r = cv.take<float>(TC_CELLS);
    float* lbstop = cv.take<float>(n);
    float* Xp = cv.take<float>(size_t(n) * d);
    const int K = tc_cells(n_pad, n);
    void* order_scratch = K > 1 ? cv.take<char>(knn_order_scratch_bytes(n, d, K)) : nullptr;

    if ((rc = stage_mark(c, 8, st))) return rc;
    DRGB_CUDA(c, cudaMemsetAsync(maxbits, 0, 64, st));
    DRGB_CUDA(c, cudaMemsetAsync(fail_count, 0, 64, st));
    tc_colstats_kernel<<<nblk, TC_STAT_WARPS * 32, 0, st>>>(X, n, d, partial, mean, maxbits);
    DRGB_CHECK_LAUNCH(c);
    // spatial order (K > 1) or the identity with one cell holding everything
    if (K == 1) DRGB_CUDA(c, cudaMemsetAsync(cell_c, 0, size_t(d) * 4, st));
    tc_identity_kernel<<<grid_for(n_pad, 256, c->num_sms * 8), 256, 0, st>>>(perm, n, n_pad, K == 1, cell_beg,
                                                                           cell_r);
    DRGB_CHECK_LAUNCH(c);
    if (K > 1 && (rc = knn_order(c, X, n, d, K, perm, cell_beg, cell_c, cell_r, order_scratch, st))) return rc;
    tc_stage_kernel<F16><<<grid_for(n_pad, 8 * STAGE_ROWS, c->num_sms * 8), 256, 0, st>>>(X, n, n_pad, d, mean, perm, XA,
                                                                              XB, norm, resid, maxbits, Xp);
    DRGB_CHECK_LAUNCH(c);

    CUtensorMap mA, mB;
    if ((rc = make_map_k64(c, &mA, XA, n_pad, TC_K, TC_BM, F16))) return rc;
    if ((rc = make_map_k64(c, &mB, XB, n_pad, TC_K, TC_BN, F16))) return rc;
    static bool attr_set = false;
    if (!attr_set) {
        DRGB_CUDA(c, cudaFuncSetAttribute(knn_tc_kernel<F16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          int(TC_SMEM)));
        attr_set = true;
    }
    TcParams P;
    P.n = n;
    P.n_tiles = int(n_pad / TC_BN);
    P.cand_idx = cand_idx;
    P.cand_s = cand_s;
    P.status = c->d_status;
    P.X = X;
    P.d = d;
    P.perm = perm;
    P.K = K;
    P.cell_beg = cell_beg;
    P.cell_c = cell_c;
    P.cell_r = cell_r;
    P.norm = norm;
    P.resid = resid;
    P.maxbits = maxbits;
    P.lbstop = lbstop;
    P.tiles_done = c->d_counter + 4;
    c->knn_tiles_total = int64_t((n + TC_BM - 1) / TC_BM) * (n_pad / TC_BN);
    DRGB_CUDA(c, cudaMemsetAsync(c->d_counter + 4, 0, 8, st));
    const int grid = int((n + TC_BM - 1) / TC_BM);
    if ((rc = stage_mark(c, 6, st))) return rc;
    knn_tc_kernel<F16><<<grid, TC_THREADS, TC_SMEM, st>>>(mA, mB, P);
    DRGB_CHECK_LAUNCH(c);
    if ((rc = stage_mark(c, 7, st))) return rc;

    {
        auto rr = (d & 1) ? tc_rerank_kernel<F16, false> : tc_rerank_kernel<F16, true>;
        DRGB_CUDA(c, cudaFuncSetAttribute(rr, cudaFuncAttributeMaxDynamicSharedMemorySize, int(rr_smem(d))));
        rr<<<grid_for(n, RR_WARPS, c->num_sms * 8), RR_WARPS * 32, rr_smem(d), st>>>(
            Xp, perm, n, d, k, cand_idx, cand_s, norm, resid, maxbits, lbstop, idx_out, dist_out,
            defer_rows ? defer_rows : fail_rows, defer_count ? defer_count : fail_count);
        DRGB_CHECK_LAUNCH(c);
    }
    if ((rc = stage_mark(c, 9, st))) return rc;
    if (defer_rows) return DRGB_OK;  // the caller re-scans the uncertified rows
    // exact FP32 scan of the uncertified rows (row list on the device, the
    // count read back once): over the cells each row can reach when their
    // partial lists fit, else over all points in chunks
    DRGB_CUDA(c, cudaMemcpyAsync(c->d_counter, fail_count, sizeof(int32_t), cudaMemcpyDeviceToDevice, st));
    int32_t cnt32 = 0;
    DRGB_CUDA(c, cudaMemcpyAsync(&cnt32, fail_count, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    DRGB_CUDA(c, cudaStreamSynchronize(st));
    const int64_t cnt = cnt32 < n ? cnt32 : n;
    // chunks: at least RS_CHUNK_MIN positions, at most as many as the
    // partial lists' scratch holds (at most n / CH + K chunks in all)
    int64_t CH = RS_CHUNK_MIN;
    const size_t per_list = size_t(cnt > 0 ? cnt : 1) * k * 8;
    const int64_t max_lists = int64_t((TC_PART_BYTES - 4096) / per_list) - K;
    if (max_lists > 0 && CH * max_lists < n) CH = (n + max_lists - 1) / max_lists;
    const int64_t nchunk = (n + CH - 1) / CH + K;
    if (cnt > 0 && K > 1 && max_lists > 0 && nchunk <= int64_t(INT32_MAX) && cnt <= 65535) {
        Carve pc(part);
        int32_t* pidx = pc.take<int32_t>(size_t(cnt) * nchunk * k);
        float* pd2 = pc.take<float>(size_t(cnt) * nchunk * k);
        int32_t* chunk_beg = pc.take<int32_t>(TC_CELLS + 1);
        tc_chunks_kernel<<<1, 32, 0, st>>>(cell_beg, K, int32_t(CH), chunk_beg);
        DRGB_CHECK_LAUNCH(c);
        const dim3 grid(static_cast<unsigned>(nchunk), static_cast<unsigned>(cnt));
        auto rs = k <= 16 ? tc_rescan_kernel<16> : tc_rescan_kernel<32>;
        DRGB_CUDA(c, cudaFuncSetAttribute(rs, cudaFuncAttributeMaxDynamicSharedMemorySize, int(RS_SMEM)));
        rs<<<grid, RS_THREADS, RS_SMEM, st>>>(X, Xp, perm, d, k, fail_rows, int(cnt), K, int32_t(CH), cell_beg,
                                              chunk_beg, cell_c, cell_r, dist_out, pidx, pd2);
        DRGB_CHECK_LAUNCH(c);
        rc = launch_merge_partials(c, pidx, pd2, cnt, int(nchunk), k, fail_rows, idx_out, dist_out, st);
    } else {
        rc = launch_knn_exact_rows_n(c, X, n, d, k, fail_rows, fail_count, cnt, idx_out, dist_out, st, part,
                                     TC_PART_BYTES);
    }
    if (rc) return rc;
    return stage_mark(c, 10, st);
}

int knn_tc(Ctx* c, const float* X, int64_t n, int d, int k, bool f16, int32_t* idx_out, float* dist_out,
           cudaStream_t st, void* scratch, int32_t* defer_rows, int32_t* defer_count) {
    if ((defer_rows == nullptr) != (defer_count == nullptr))
        return set_error(c, DRGB_ERR_INVALID, "knn: deferred re-scan needs both the row list and its count");
    return f16 ? knn_tc_impl<true>(c, X, n, d, k, idx_out, dist_out, st, scratch, defer_rows, defer_count)
               : knn_tc_impl<false>(c, X, n, d, k, idx_out, dist_out, st, scratch, defer_rows, defer_count);
}

}  // namespace drgb

extern "C" int drgb_knn_tiles(drgb_ctx* c, int64_t* done, int64_t* total, void* stream) {
    if (!c || !done || !total) return DRGB_ERR_INVALID;
    unsigned long long v = 0;
    DRGB_CUDA(c, cudaStreamSynchronize(static_cast<cudaStream_t>(stream)));
    DRGB_CUDA(c, cudaMemcpy(&v, c->d_counter + 4, sizeof(v), cudaMemcpyDeviceToHost));
    *done = int64_t(v);
    *total = c->knn_tiles_total;
    return DRGB_OK;
}

extern "C" int drgb_knn_uncertified(drgb_ctx* c, int64_t* count, void* stream) {
    if (!c || !count) return DRGB_ERR_INVALID;
    int32_t v = 0;
    DRGB_CUDA(c, cudaStreamSynchronize(static_cast<cudaStream_t>(stream)));
    DRGB_CUDA(c, cudaMemcpy(&v, c->d_counter, sizeof(int32_t), cudaMemcpyDeviceToHost));
    *count = v;
    return DRGB_OK;
}
