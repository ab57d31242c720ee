// Learned parametric embedder (a project addition; the paper embeds each data
// set by plain optimisation): an MLP d -> 256 -> 256 -> 2 with exact-erf GELU,
// BF16 weights and activations, FP32 accumulation and FP32 master weights,
// trained with Adam on the UMAP cross-entropy over edges of the method's own
// fuzzy graph, then used to embed new points.
//
// Every dense product runs on the tcgen05 tensor cores through one kernel,
// mlp_gemm_kernel: C[M x N] = A[M x K] * B[N x K]^T with both operands K-major
// BF16 (TMA, 128-byte swizzle), FP32 accumulation in TMEM, and a fused
// epilogue: bias + GELU (forward), GELU derivative (backward) or plain FP32
// (weight gradients, split over K).  Activations are also written transposed,
// so the weight-gradient products are K-major as well.  The 256 -> 2 layer,
// the loss, the reductions and Adam are small SIMT kernels.
//
// One training step (batch of B edges, each with `neg` negatives, R = 2 + neg
// rows per edge, M = B R rows):
//   sample     edges proportional to w (integer rejection on q) + negatives
//   gather     X rows -> Xb (M x 64) and Xb^T (64 x M), BF16
//   F1, F2     pre_l = H_{l-1} W_l^T + b_l ; H_l = GELU(pre_l)  (BF16, + transposed)
//   head       z = H2 W3^T + b3 ; loss and dL/dz per edge
//   L3 back    dpre2 = (dz W3) . GELU'(pre2) ; dW3, db3, db2 partial sums
//   dW2        dpre2^T H1     (split-K, FP32 partials)
//   dH1        dpre1 = (dpre2 W2) . GELU'(pre1)
//   dW1        dpre1^T Xb     (split-K)
//   reduce     gradient vector (fixed summation order) ; Adam ; BF16 copies
#include <cuda_bf16.h>

#include <cmath>
#include <cstring>
#include <vector>

#include "common.cuh"
#include "gemm.cuh"
#include "tc_ptx.cuh"

namespace drgb {

// ------------------------------------------------------------------ layout
static constexpr int MLP_IN = 64;   // padded input width (d <= 64)
static constexpr int MLP_H = 256;
static constexpr int MLP_OUT = 2;
static constexpr int64_t OFF_W1 = 0;
static constexpr int64_t OFF_B1 = OFF_W1 + MLP_H * MLP_IN;
static constexpr int64_t OFF_W2 = OFF_B1 + MLP_H;
static constexpr int64_t OFF_B2 = OFF_W2 + MLP_H * MLP_H;
static constexpr int64_t OFF_W3 = OFF_B2 + MLP_H;
static constexpr int64_t OFF_B3 = OFF_W3 + MLP_OUT * MLP_H;
static constexpr int64_t MLP_P = OFF_B3 + MLP_OUT;

typedef __nv_bfloat16 bf16;

// ------------------------------------------------------------------ GELU
__device__ __forceinline__ float gelu(float x) { return 0.5f * x * (1.0f + erff(x * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float x) {
    return 0.5f * (1.0f + erff(x * 0.70710678118654752f)) + x * 0.39894228040143268f * expf(-0.5f * x * x);
}

// ------------------------------------------------------------------ tensor-core GEMM
static constexpr int G_BM = 128;
static constexpr int G_STAGES = 4;
static constexpr int G_THREADS = 192;  // warp 0 TMA, warp 1 MMA, warps 2..5 epilogue
enum { EPI_GELU = 0, EPI_GELU_GRAD = 1, EPI_F32 = 2 };

struct GemmArgs {
    int M, N, K;          // M, N multiples of 128 / BN; K multiple of 64
    int kb_per_split;     // 64-wide K blocks per split (grid z)
    const float* bias;    // EPI_GELU: [N]
    float* pre;           // EPI_GELU: out [M][N] (nullable); EPI_GELU_GRAD: in [M][N]
    bf16* out;            // [M][N] (nullable)
    bf16* out_t;          // [N][M] transposed (nullable)
    float* out_f32;       // EPI_F32: [splits][M][N]; EPI_GELU_GRAD: FP32 copy [M][N] (nullable)
    int* status;
};

template <int BN>
struct GemmSmem {
    static constexpr int A_BYTES = G_BM * 64 * 2;
    static constexpr int B_BYTES = BN * 64 * 2;
    static constexpr size_t TOTAL = 1024 + size_t(G_STAGES) * (A_BYTES + B_BYTES) + 256;
};

template <int BN, int EPI>
__global__ void __launch_bounds__(G_THREADS, 1)
mlp_gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, GemmArgs G) {
    using SM = GemmSmem<BN>;
    extern __shared__ uint8_t smem_raw[];
    // 1024-byte aligned (swizzled operand tiles); an offset from the shared
    // array, so that every pointer below stays a known shared-memory address
    uint8_t* base = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    uint8_t* sA = base;
    uint8_t* sB = base + G_STAGES * SM::A_BYTES;
    uint64_t* bars = reinterpret_cast<uint64_t*>(sB + G_STAGES * SM::B_BYTES);
    uint64_t* full = bars;
    uint64_t* empty = bars + G_STAGES;
    uint64_t* acc_full = bars + 2 * G_STAGES;
    uint64_t* mma_done = acc_full + 1;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(mma_done + 1);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.x * G_BM, n0 = blockIdx.y * BN;
    const int kb0 = blockIdx.z * G.kb_per_split;
    int nkb = G.K / 64 - kb0;
    if (nkb > G.kb_per_split) nkb = G.kb_per_split;

    if (threadIdx.x == 0) {
        for (int s = 0; s < G_STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(acc_full, 1);
        mbar_init(mma_done, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(smem_u32(tmem_slot)), "r"(BN) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            int kb = 0;
            for (; kb < nkb; ++kb) {
                const int s = kb % G_STAGES;
                if (kb >= G_STAGES && !mbar_wait(&empty[s], ((kb / G_STAGES) & 1) ^ 1, abort_flag, G.status)) break;
                mbar_expect_tx(&full[s], SM::A_BYTES + SM::B_BYTES);
                tma_load_2d(sA + s * SM::A_BYTES, &tmA, (kb0 + kb) * 64, m0, &full[s]);
                tma_load_2d(sB + s * SM::B_BYTES, &tmB, (kb0 + kb) * 64, n0, &full[s]);
            }
            if (kb < nkb) {  // aborted: let issued loads land before exit
                for (int u = (kb > G_STAGES ? kb - G_STAGES : 0); u < kb; ++u) {
                    const unsigned long long t0 = global_timer();
                    while (!mbar_try(&full[u % G_STAGES], (u / G_STAGES) & 1) && global_timer() - t0 < 100000000ull) {
                    }
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            const uint32_t idesc = idesc_f16kind(G_BM, BN, false);
            for (int kb = 0; kb < nkb; ++kb) {
                const int s = kb % G_STAGES;
                if (!mbar_wait(&full[s], (kb / G_STAGES) & 1, abort_flag, G.status)) break;
                tc_fence_after();
                const uint64_t ad = sdesc_sw128(smem_u32(sA + s * SM::A_BYTES));
                const uint64_t bd = sdesc_sw128(smem_u32(sB + s * SM::B_BYTES));
#pragma unroll
                for (int k = 0; k < 4; ++k) mma_f16kind(tmem, ad + 2 * k, bd + 2 * k, idesc, (kb > 0 || k > 0) ? 1u : 0u);
                mma_commit(&empty[s]);
            }
            mma_commit(acc_full);
            mma_commit(mma_done);
            const unsigned long long t0 = global_timer();
            while (!mbar_try(mma_done, 0) && global_timer() - t0 < 100000000ull) {
            }
        }
    } else {
        const int quarter = warp & 3;
        const int row = quarter * 32 + lane;
        const int64_t gr = m0 + row;
        const bool ok = mbar_wait(acc_full, 0, abort_flag, G.status) && nkb > 0;
        tc_fence_after();
        if (ok) {
#pragma unroll 1
            for (int c = 0; c < BN / 32; ++c) {
                float v[32];
                __syncwarp();
                tmem_ld32(tmem + (uint32_t(quarter * 32) << 16) + uint32_t(c * 32), v);
                const int gc0 = n0 + c * 32;
                if (EPI == EPI_F32) {
                    float* o = G.out_f32 + (int64_t(blockIdx.z) * G.M + gr) * G.N + gc0;
#pragma unroll
                    for (int i = 0; i < 32; i += 4) *reinterpret_cast<float4*>(o + i) = make_float4(v[i], v[i + 1], v[i + 2], v[i + 3]);
                } else {
                    if (EPI == EPI_GELU) {
#pragma unroll
                        for (int i = 0; i < 32; ++i) v[i] += G.bias[gc0 + i];
                        if (G.pre) {
                            float* o = G.pre + gr * G.N + gc0;
#pragma unroll
                            for (int i = 0; i < 32; i += 4)
                                *reinterpret_cast<float4*>(o + i) = make_float4(v[i], v[i + 1], v[i + 2], v[i + 3]);
                        }
#pragma unroll
                        for (int i = 0; i < 32; ++i) v[i] = gelu(v[i]);
                    } else {  // EPI_GELU_GRAD
                        const float* p = G.pre + gr * G.N + gc0;
#pragma unroll
                        for (int i = 0; i < 32; i += 4) {
                            const float4 x = *reinterpret_cast<const float4*>(p + i);
                            v[i] *= gelu_grad(x.x);
                            v[i + 1] *= gelu_grad(x.y);
                            v[i + 2] *= gelu_grad(x.z);
                            v[i + 3] *= gelu_grad(x.w);
                        }
                        if (G.out_f32) {
                            float* o = G.out_f32 + gr * G.N + gc0;
#pragma unroll
                            for (int i = 0; i < 32; i += 4)
                                *reinterpret_cast<float4*>(o + i) = make_float4(v[i], v[i + 1], v[i + 2], v[i + 3]);
                        }
                    }
                    if (G.out) {
                        uint32_t packed[16];
#pragma unroll
                        for (int i = 0; i < 16; ++i) {
                            const __nv_bfloat162 h2 = __floats2bfloat162_rn(v[2 * i], v[2 * i + 1]);
                            packed[i] = *reinterpret_cast<const uint32_t*>(&h2);
                        }
                        uint4* o = reinterpret_cast<uint4*>(G.out + gr * G.N + gc0);
#pragma unroll
                        for (int i = 0; i < 4; ++i)
                            o[i] = make_uint4(packed[4 * i], packed[4 * i + 1], packed[4 * i + 2], packed[4 * i + 3]);
                    }
                    if (G.out_t) {
#pragma unroll
                        for (int i = 0; i < 32; ++i) G.out_t[int64_t(gc0 + i) * G.M + gr] = __float2bfloat16_rn(v[i]);
                    }
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(BN) : "memory");
    }
}

struct Gemm {
    CUtensorMap a, b;
    GemmArgs g;
    dim3 grid;
    int bn;
    int epi;
};

// C[M x N] = A[M x K] B[N x K]^T with A, B row-major BF16 (K contiguous).
static int gemm_setup(Ctx* c, Gemm& G, const bf16* A, const bf16* B, int M, int N, int K, int bn, int epi,
                      int splits) {
    if (M % G_BM || N % bn || K % 64 || splits < 1)
        return set_error(c, DRGB_ERR_INVALID, "mlp gemm: bad shape %d x %d x %d", M, N, K);
    int rc = make_map_k64(c, &G.a, A, M, K, G_BM, false);
    if (rc) return rc;
    if ((rc = make_map_k64(c, &G.b, B, N, K, bn, false))) return rc;
    std::memset(&G.g, 0, sizeof(G.g));
    G.g.M = M;
    G.g.N = N;
    G.g.K = K;
    const int kbs = K / 64;
    G.g.kb_per_split = (kbs + splits - 1) / splits;
    G.g.status = c->d_status;
    G.grid = dim3(M / G_BM, N / bn, (kbs + G.g.kb_per_split - 1) / G.g.kb_per_split);
    G.bn = bn;
    G.epi = epi;
    return DRGB_OK;
}

template <int BN, int EPI>
static int gemm_attr(Ctx* c) {
    DRGB_CUDA(c, cudaFuncSetAttribute(mlp_gemm_kernel<BN, EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      int(GemmSmem<BN>::TOTAL)));
    return DRGB_OK;
}

// Opt the GEMM instantiations into their shared-memory size (before any capture).
static int gemm_prepare(Ctx* c) {
    int rc;
    if ((rc = gemm_attr<256, EPI_GELU>(c)) || (rc = gemm_attr<256, EPI_GELU_GRAD>(c)) ||
        (rc = gemm_attr<256, EPI_F32>(c)) || (rc = gemm_attr<64, EPI_F32>(c)))
        return rc;
    return DRGB_OK;
}

template <int BN, int EPI>
static int gemm_launch_t(Ctx* c, const Gemm& G, cudaStream_t st) {
    mlp_gemm_kernel<BN, EPI><<<G.grid, G_THREADS, GemmSmem<BN>::TOTAL, st>>>(G.a, G.b, G.g);
    DRGB_CHECK_LAUNCH(c);
    return DRGB_OK;
}

static int gemm_launch(Ctx* c, const Gemm& G, cudaStream_t st) {
    if (G.bn == 256 && G.epi == EPI_GELU) return gemm_launch_t<256, EPI_GELU>(c, G, st);
    if (G.bn == 256 && G.epi == EPI_GELU_GRAD) return gemm_launch_t<256, EPI_GELU_GRAD>(c, G, st);
    if (G.bn == 256 && G.epi == EPI_F32) return gemm_launch_t<256, EPI_F32>(c, G, st);
    if (G.bn == 64 && G.epi == EPI_F32) return gemm_launch_t<64, EPI_F32>(c, G, st);
    return set_error(c, DRGB_ERR_INVALID, "mlp gemm: unsupported tile");
}

// The plain product for other users of the library (the PCA covariance):
// partials[z][M][N] = A[M x K] B[N x K]^T over the z-th share of K.
int tc_gemm_nt_f32(Ctx* c, const void* A, const void* B, int M, int N, int K, int splits, float* partials,
                   int* splits_used, cudaStream_t st) {
    Gemm G;
    const int bn = (N % 256 == 0) ? 256 : 64;
    int rc = gemm_setup(c, G, static_cast<const bf16*>(A), static_cast<const bf16*>(B), M, N, K, bn, EPI_F32, splits);
    if (rc) return rc;
    G.g.out_f32 = partials;
    if ((rc = bn == 256 ? gemm_attr<256, EPI_F32>(c) : gemm_attr<64, EPI_F32>(c))) return rc;
    if (splits_used) *splits_used = int(G.grid.z);
    return gemm_launch(c, G, st);
}

// ------------------------------------------------------------------ SIMT kernels
struct MlpWeights {          // BF16 working copies of the master weights
    bf16* W1b;               // [256][64]
    bf16* W2b;               // [256][256]  (out, in)
    bf16* W2tb;              // [256][256]  (in, out)
    float* W3f;              // [2][256]    BF16-rounded values in FP32
};

__global__ void mlp_cast_kernel(const float* __restrict__ P, MlpWeights W) {
    for (int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < MLP_H * MLP_H;
         t += int64_t(gridDim.x) * blockDim.x) {
        const int o = int(t / MLP_H), i = int(t % MLP_H);
        const bf16 v = __float2bfloat16_rn(P[OFF_W2 + t]);
        W.W2b[t] = v;
        W.W2tb[int64_t(i) * MLP_H + o] = v;
        if (t < MLP_H * MLP_IN) W.W1b[t] = __float2bfloat16_rn(P[OFF_W1 + t]);
        if (t < MLP_OUT * MLP_H) W.W3f[t] = __bfloat162float(__float2bfloat16_rn(P[OFF_W3 + t]));
    }
}

// Edge sampling proportional to w: try uniform entries e, accept when the
// next 24 random bits fall below q_e = round(2^24 w_e); 64 tries at most.
__global__ void mlp_sample_kernel(const int32_t* __restrict__ rp, const int32_t* __restrict__ col,
                                  const uint32_t* __restrict__ q, int64_t n, int64_t nnz, int B, int neg,
                                  const uint32_t* __restrict__ step_dev, uint32_t k0, uint32_t k1,
                                  int32_t* __restrict__ rows) {
    const int R = 2 + neg;
    const uint32_t step = *step_dev;
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < B; s += gridDim.x * blockDim.x) {
        uint32_t e = 0;
        for (uint32_t r = 0; r < 64; ++r) {
            const U4 u = philox4x32_10(U4{step, uint32_t(s), r, TAG_MLP}, k0, k1);
            e = __umulhi(u.x, uint32_t(nnz));
            if ((u.y >> 8) < q[e]) break;
        }
        int64_t lo = 0, hi = n - 1;  // head row: last i with rp[i] <= e
        while (lo < hi) {
            const int64_t mid = (lo + hi + 1) >> 1;
            if (rp[mid] <= int32_t(e)) lo = mid; else hi = mid - 1;
        }
        rows[int64_t(s) * R] = int32_t(lo);
        rows[int64_t(s) * R + 1] = col[e];
        for (int t = 0; t < neg; ++t) {
            const U4 u = philox4x32_10(U4{step, uint32_t(s), 64u + uint32_t(t / 4), TAG_MLP}, k0, k1);
            const uint32_t w4[4] = {u.x, u.y, u.z, u.w};
            rows[int64_t(s) * R + 2 + t] = int32_t(__umulhi(w4[t & 3], uint32_t(n)));
        }
    }
}

// Gather BF16 rows (zero-padded to 64 columns) and their transpose.
__global__ void mlp_gather_kernel(const float* __restrict__ X, int d, const int32_t* __restrict__ rows, int M,
                                  int M_valid, bf16* __restrict__ Xb, bf16* __restrict__ Xbt) {
    __shared__ bf16 tile[32][33];
    const int r0 = blockIdx.x * 32, c0 = blockIdx.y * 32;
    for (int ty = threadIdx.y; ty < 32; ty += blockDim.y) {
        const int r = r0 + ty, cc = c0 + threadIdx.x;
        float v = 0.f;
        if (r < M_valid && cc < d) v = X[int64_t(rows ? rows[r] : r) * d + cc];
        const bf16 b = __float2bfloat16_rn(v);
        if (r < M) Xb[int64_t(r) * MLP_IN + cc] = b;
        tile[ty][threadIdx.x] = b;
    }
    __syncthreads();
    if (Xbt)
        for (int ty = threadIdx.y; ty < 32; ty += blockDim.y) {
            const int cc = c0 + ty, r = r0 + threadIdx.x;
            if (r < M) Xbt[int64_t(cc) * M + r] = tile[threadIdx.x][ty];
        }
}

// z = H2 W3^T + b3: one warp per row.
__global__ void mlp_head_kernel(const bf16* __restrict__ H2, const float* __restrict__ W3f,
                                const float* __restrict__ P, int M, float* __restrict__ z) {
    const int lane = threadIdx.x & 31;
    for (int64_t r = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; r < M;
         r += (int64_t(gridDim.x) * blockDim.x) >> 5) {
        float s0 = 0.f, s1 = 0.f;
        for (int cc = lane; cc < MLP_H; cc += 32) {
            const float h = __bfloat162float(H2[r * MLP_H + cc]);
            s0 = fmaf(h, W3f[cc], s0);
            s1 = fmaf(h, W3f[MLP_H + cc], s1);
        }
        for (int o = 16; o > 0; o >>= 1) {
            s0 += __shfl_xor_sync(0xffffffffu, s0, o);
            s1 += __shfl_xor_sync(0xffffffffu, s1, o);
        }
        if (lane == 0) {
            z[2 * r] = s0 + P[OFF_B3];
            z[2 * r + 1] = s1 + P[OFF_B3 + 1];
        }
    }
}

// UMAP cross-entropy of each edge (head, tail, negatives) on the embedded
// rows, with Phi = 1 / (1 + a d^b) clamped to [1e-4, 1 - 1e-4] (zero
// gradient where clamped); loss and dL/dz are divided by the batch size.
__global__ void mlp_loss_kernel(const float* __restrict__ z, const int32_t* __restrict__ rows, int B, int neg,
                                float a, float b, float* __restrict__ dz, float* __restrict__ loss_part) {
    const int R = 2 + neg;
    const float lo = 1e-4f, hi = 1.0f - 1e-4f, invB = 1.0f / float(B);
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < B; s += gridDim.x * blockDim.x) {
        const int64_t r0 = int64_t(s) * R;
        const float zi0 = z[2 * r0], zi1 = z[2 * r0 + 1];
        float gi0 = 0.f, gi1 = 0.f, L = 0.f;
        for (int t = 1; t < R; ++t) {
            const int64_t r = r0 + t;
            float g0 = 0.f, g1 = 0.f;
            if (t >= 2 && rows[r] == rows[r0]) {  // a negative that is the head itself
                dz[2 * r] = 0.f;
                dz[2 * r + 1] = 0.f;
                continue;
            }
            const float d0 = zi0 - z[2 * r], d1 = zi1 - z[2 * r + 1];
            const float d = d0 * d0 + d1 * d1;
            const float adb = d > 0.f ? a * powf(d, b) : 0.f;
            const float phi = 1.0f / (1.0f + adb);
            const bool inside = phi > lo && phi < hi;
            const float pc = fminf(fmaxf(phi, lo), hi);
            float dLdd = 0.f;
            if (t == 1) {
                L += -logf(pc);
                if (inside) dLdd = b * adb / (d * (1.0f + adb));  // a b d^(b-1) / (1 + a d^b)
            } else {
                L += -logf(1.0f - pc);
                if (inside) dLdd = -b / (d * (1.0f + adb));
            }
            g0 = dLdd * 2.0f * d0 * invB;
            g1 = dLdd * 2.0f * d1 * invB;
            gi0 += g0;
            gi1 += g1;
            dz[2 * r] = -g0;
            dz[2 * r + 1] = -g1;
        }
        dz[2 * r0] = gi0;
        dz[2 * r0 + 1] = gi1;
        loss_part[s] = L * invB;
    }
}

// dpre2 = (dz W3) . GELU'(pre2): BF16 row-major and transposed (32 x 32 tiles).
__global__ void mlp_l3back_kernel(const float* __restrict__ dz, const float* __restrict__ W3f,
                                  const float* __restrict__ pre2, int M, bf16* __restrict__ D, bf16* __restrict__ Dt,
                                  float* __restrict__ Df) {
    __shared__ bf16 tile[32][33];
    const int r0 = blockIdx.x * 32, c0 = blockIdx.y * 32;
    for (int ty = threadIdx.y; ty < 32; ty += blockDim.y) {
        const int64_t r = r0 + ty;
        const int cc = c0 + threadIdx.x;
        const float g = dz[2 * r] * W3f[cc] + dz[2 * r + 1] * W3f[MLP_H + cc];
        const float v = g * gelu_grad(pre2[r * MLP_H + cc]);
        Df[r * MLP_H + cc] = v;
        const bf16 bv = __float2bfloat16_rn(v);
        D[r * MLP_H + cc] = bv;
        tile[ty][threadIdx.x] = bv;
    }
    __syncthreads();
    for (int ty = threadIdx.y; ty < 32; ty += blockDim.y) {
        const int cc = c0 + ty;
        Dt[int64_t(cc) * M + r0 + threadIdx.x] = tile[threadIdx.x][ty];
    }
}

// Column sums of an FP32 [M x C] matrix over row chunks: part[blk][c].
__global__ void mlp_colsum_kernel(const float* __restrict__ A, int M, int C, int chunk, float* __restrict__ part) {
    for (int cc = threadIdx.x; cc < C; cc += blockDim.x) {
        float s = 0.f;
        const int r_end = (blockIdx.x + 1) * chunk < M ? (blockIdx.x + 1) * chunk : M;
        for (int r = blockIdx.x * chunk; r < r_end; ++r) s += A[int64_t(r) * C + cc];
        part[int64_t(blockIdx.x) * C + cc] = s;
    }
}

// dW3[o][c] = sum_r dz[r][o] H2[r][c] and db3[o] = sum_r dz[r][o] over row chunks.
__global__ void mlp_w3grad_kernel(const float* __restrict__ dz, const bf16* __restrict__ H2, int M, int chunk,
                                  float* __restrict__ part) {
    const int r_end = (blockIdx.x + 1) * chunk < M ? (blockIdx.x + 1) * chunk : M;
    for (int t = threadIdx.x; t < 2 * MLP_H + 2; t += blockDim.x) {
        float s = 0.f;
        if (t < 2 * MLP_H) {
            const int o = t / MLP_H, cc = t % MLP_H;
            for (int r = blockIdx.x * chunk; r < r_end; ++r)
                s += dz[2 * int64_t(r) + o] * __bfloat162float(H2[int64_t(r) * MLP_H + cc]);
        } else {
            const int o = t - 2 * MLP_H;
            for (int r = blockIdx.x * chunk; r < r_end; ++r) s += dz[2 * int64_t(r) + o];
        }
        part[int64_t(blockIdx.x) * (2 * MLP_H + 2) + t] = s;
    }
}

struct GradParts {
    const float* dW1;   // [s1][256][64]
    int s1;
    const float* dW2;   // [s2][256][256]
    int s2;
    const float* db1;   // [n1][256]
    int n1;
    const float* db2;   // [n2][256]
    int n2;
    const float* w3;    // [n3][514]
    int n3;
    const float* loss;  // [B]
    int B;
};

// Gradient vector from the partial sums (each summed in a fixed order) and
// the batch loss.
__global__ void mlp_reduce_kernel(GradParts g, float* __restrict__ grad, float* __restrict__ loss_out,
                                  const uint32_t* __restrict__ step_dev) {
    for (int64_t p = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; p < MLP_P; p += int64_t(gridDim.x) * blockDim.x) {
        float s = 0.f;
        if (p < OFF_B1) {
            for (int z = 0; z < g.s1; ++z) s += g.dW1[int64_t(z) * MLP_H * MLP_IN + p];
        } else if (p < OFF_W2) {
            for (int z = 0; z < g.n1; ++z) s += g.db1[int64_t(z) * MLP_H + (p - OFF_B1)];
        } else if (p < OFF_B2) {
            for (int z = 0; z < g.s2; ++z) s += g.dW2[int64_t(z) * MLP_H * MLP_H + (p - OFF_W2)];
        } else if (p < OFF_W3) {
            for (int z = 0; z < g.n2; ++z) s += g.db2[int64_t(z) * MLP_H + (p - OFF_B2)];
        } else {
            for (int z = 0; z < g.n3; ++z) s += g.w3[int64_t(z) * (2 * MLP_H + 2) + (p - OFF_W3)];
        }
        grad[p] = s;
    }
    if (blockIdx.x == 0 && loss_out) {
        __shared__ float red[256];
        float s = 0.f;
        for (int t = threadIdx.x; t < g.B; t += blockDim.x) s += g.loss[t];
        red[threadIdx.x] = s;
        __syncthreads();
        for (int o = blockDim.x / 2; o > 0; o >>= 1) {
            if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
            __syncthreads();
        }
        if (threadIdx.x == 0) loss_out[step_dev ? *step_dev : 0] = red[0];
    }
}

// Adam on the FP32 master weights (bias-corrected step t = *step + 1), then
// the step counter advances.
__global__ void mlp_adam_kernel(float* __restrict__ P, float* __restrict__ m, float* __restrict__ v,
                                const float* __restrict__ grad, float lr, float b1, float b2, float eps,
                                uint32_t* __restrict__ step_dev) {
    const float t = float(*step_dev + 1);
    const float c1 = 1.0f - powf(b1, t), c2 = 1.0f - powf(b2, t);
    for (int64_t p = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; p < MLP_P; p += int64_t(gridDim.x) * blockDim.x) {
        const float g = grad[p];
        const float mm = b1 * m[p] + (1.0f - b1) * g;
        const float vv = b2 * v[p] + (1.0f - b2) * g * g;
        m[p] = mm;
        v[p] = vv;
        P[p] -= lr * (mm / c1) / (sqrtf(vv / c2) + eps);
    }
}

__global__ void mlp_step_advance_kernel(uint32_t* step_dev) { *step_dev += 1; }

// Initial weights: U(-1/sqrt(fan_in), 1/sqrt(fan_in)) from Philox, biases 0,
// columns of W1 beyond d exactly 0.
__global__ void mlp_init_kernel(float* __restrict__ P, int d, uint32_t k0, uint32_t k1) {
    for (int64_t p = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; p < MLP_P; p += int64_t(gridDim.x) * blockDim.x) {
        const U4 u = philox4x32_10(U4{uint32_t(p), 0u, 0u, TAG_MLP | 0x100u}, k0, k1);
        const float r = float(u.x >> 8) * 5.9604644775390625e-08f * 2.0f - 1.0f;  // [-1, 1)
        float val = 0.f;
        if (p < OFF_B1) val = (int(p % MLP_IN) < d) ? r / sqrtf(float(d)) : 0.f;
        else if (p >= OFF_W2 && p < OFF_B2) val = r / 16.0f;     // fan_in 256
        else if (p >= OFF_W3 && p < OFF_B3) val = r / 16.0f;
        P[p] = val;
    }
}

// ------------------------------------------------------------------ host: one forward/backward
struct MlpBuffers {
    int M;                       // rows of the batch (padded to 128)
    int32_t* rows;
    bf16 *Xb, *Xbt, *H1b, *H1bt, *H2b, *H2bt, *D2b, *D2bt, *D1b, *D1bt;
    float *pre1, *pre2, *z, *dz, *D2f, *D1f, *loss_part;
    float *pW2, *pW1, *pb1, *pb2, *pw3;
    float* grad;
    MlpWeights W;
    uint32_t* step;
    int s_split, n_chunks;
};

static constexpr int MLP_SPLITS = 32;
static constexpr int MLP_CHUNK = 512;

static size_t mlp_batch_bytes(int M) {
    const size_t m = size_t(M);
    const int nch = int((m + MLP_CHUNK - 1) / MLP_CHUNK);
    size_t b = Carve::round(m * 4);                                   // rows
    b += 2 * Carve::round(m * MLP_IN * 2);                            // Xb, Xbt
    b += 8 * Carve::round(m * MLP_H * 2);                             // H1b, H1bt, H2b, H2bt, D2b, D2bt, D1b, D1bt
    b += 4 * Carve::round(m * MLP_H * 4);                             // pre1, pre2, D2f, D1f
    b += 2 * Carve::round(m * 2 * 4) + Carve::round(m * 4);           // z, dz, loss_part
    b += Carve::round(size_t(MLP_SPLITS) * MLP_H * MLP_H * 4);        // pW2
    b += Carve::round(size_t(MLP_SPLITS) * MLP_H * MLP_IN * 4);       // pW1
    b += 2 * Carve::round(size_t(nch) * MLP_H * 4);                   // pb1, pb2
    b += Carve::round(size_t(nch) * (2 * MLP_H + 2) * 4);             // pw3
    b += Carve::round(MLP_P * 4);                                     // grad
    b += 2 * Carve::round(MLP_H * MLP_H * 2) + Carve::round(MLP_H * MLP_IN * 2) + Carve::round(2 * MLP_H * 4);
    b += Carve::round(64);
    return b + 8192;
}

static MlpBuffers mlp_carve(void* base, int M) {
    Carve cv(base);
    MlpBuffers b;
    const size_t m = size_t(M);
    b.M = M;
    b.n_chunks = int((m + MLP_CHUNK - 1) / MLP_CHUNK);
    b.s_split = MLP_SPLITS;
    b.rows = cv.take<int32_t>(m);
    b.Xb = cv.take<bf16>(m * MLP_IN);
    b.Xbt = cv.take<bf16>(m * MLP_IN);
    b.H1b = cv.take<bf16>(m * MLP_H);
    b.H1bt = cv.take<bf16>(m * MLP_H);
    b.H2b = cv.take<bf16>(m * MLP_H);
    b.H2bt = cv.take<bf16>(m * MLP_H);
    b.D2b = cv.take<bf16>(m * MLP_H);
    b.D2bt = cv.take<bf16>(m * MLP_H);
    b.D1b = cv.take<bf16>(m * MLP_H);
    b.D1bt = cv.take<bf16>(m * MLP_H);
    b.pre1 = cv.take<float>(m * MLP_H);
    b.pre2 = cv.take<float>(m * MLP_H);
    b.D2f = cv.take<float>(m * MLP_H);
    b.D1f = cv.take<float>(m * MLP_H);
    b.z = cv.take<float>(m * 2);
    b.dz = cv.take<float>(m * 2);
    b.loss_part = cv.take<float>(m);
    b.pW2 = cv.take<float>(size_t(MLP_SPLITS) * MLP_H * MLP_H);
    b.pW1 = cv.take<float>(size_t(MLP_SPLITS) * MLP_H * MLP_IN);
    b.pb1 = cv.take<float>(size_t(b.n_chunks) * MLP_H);
    b.pb2 = cv.take<float>(size_t(b.n_chunks) * MLP_H);
    b.pw3 = cv.take<float>(size_t(b.n_chunks) * (2 * MLP_H + 2));
    b.grad = cv.take<float>(MLP_P);
    b.W.W2b = cv.take<bf16>(MLP_H * MLP_H);
    b.W.W2tb = cv.take<bf16>(MLP_H * MLP_H);
    b.W.W1b = cv.take<bf16>(MLP_H * MLP_IN);
    b.W.W3f = cv.take<float>(2 * MLP_H);
    b.step = cv.take<uint32_t>(16);
    return b;
}

// Forward + backward of the batch whose rows are already gathered (Xb, Xbt)
// with B edges of R rows; leaves the gradient in b.grad and the loss in
// loss_out[*step] (if given).
static int mlp_fwd_bwd(Ctx* c, MlpBuffers& b, const float* P, int B, int neg, float a, float bb,
                       float* loss_out, cudaStream_t st) {
    const int M = b.M;
    int rc;
    Gemm F1, F2, DW2, DH1, DW1;
    if ((rc = gemm_setup(c, F1, b.Xb, b.W.W1b, M, MLP_H, MLP_IN, 256, EPI_GELU, 1))) return rc;
    F1.g.bias = P + OFF_B1;
    F1.g.pre = b.pre1;
    F1.g.out = b.H1b;
    F1.g.out_t = b.H1bt;
    if ((rc = gemm_setup(c, F2, b.H1b, b.W.W2b, M, MLP_H, MLP_H, 256, EPI_GELU, 1))) return rc;
    F2.g.bias = P + OFF_B2;
    F2.g.pre = b.pre2;
    F2.g.out = b.H2b;
    F2.g.out_t = b.H2bt;
    if ((rc = gemm_launch(c, F1, st))) return rc;
    if ((rc = gemm_launch(c, F2, st))) return rc;
    mlp_head_kernel<<<grid_for(int64_t(M) * 32, 256, c->num_sms * 16), 256, 0, st>>>(b.H2b, b.W.W3f, P, M, b.z);
    DRGB_CHECK_LAUNCH(c);
    if (M > B * (2 + neg))  // padding rows carry no gradient
        DRGB_CUDA(c, cudaMemsetAsync(b.dz + 2 * int64_t(B) * (2 + neg), 0,
                                     (size_t(M) - size_t(B) * (2 + neg)) * 2 * 4, st));
    mlp_loss_kernel<<<grid_for(B, 128, c->num_sms * 8), 128, 0, st>>>(b.z, b.rows, B, neg, a, bb, b.dz, b.loss_part);
    DRGB_CHECK_LAUNCH(c);
    mlp_l3back_kernel<<<dim3(M / 32, MLP_H / 32), dim3(32, 8), 0, st>>>(b.dz, b.W.W3f, b.pre2, M, b.D2b, b.D2bt,
                                                                      b.D2f);
    DRGB_CHECK_LAUNCH(c);
    mlp_w3grad_kernel<<<b.n_chunks, 256, 0, st>>>(b.dz, b.H2b, M, MLP_CHUNK, b.pw3);
    DRGB_CHECK_LAUNCH(c);
    mlp_colsum_kernel<<<b.n_chunks, 256, 0, st>>>(b.D2f, M, MLP_H, MLP_CHUNK, b.pb2);
    DRGB_CHECK_LAUNCH(c);
    // dW2 = dpre2^T H1 (K = M, split)
    if ((rc = gemm_setup(c, DW2, b.D2bt, b.H1bt, MLP_H, MLP_H, M, 256, EPI_F32, MLP_SPLITS))) return rc;
    DW2.g.out_f32 = b.pW2;
    if ((rc = gemm_launch(c, DW2, st))) return rc;
    // dpre1 = (dpre2 W2) . GELU'(pre1): A = dpre2 [M x 256(out)], B = W2^T [256(in) x 256(out)]
    if ((rc = gemm_setup(c, DH1, b.D2b, b.W.W2tb, M, MLP_H, MLP_H, 256, EPI_GELU_GRAD, 1))) return rc;
    DH1.g.pre = b.pre1;
    DH1.g.out = b.D1b;
    DH1.g.out_t = b.D1bt;
    DH1.g.out_f32 = b.D1f;
    if ((rc = gemm_launch(c, DH1, st))) return rc;
    mlp_colsum_kernel<<<b.n_chunks, 256, 0, st>>>(b.D1f, M, MLP_H, MLP_CHUNK, b.pb1);
    DRGB_CHECK_LAUNCH(c);
    // dW1 = dpre1^T Xb: A = dpre1^T [256 x M], B = Xb^T [64 x M]
    if ((rc = gemm_setup(c, DW1, b.D1bt, b.Xbt, MLP_H, MLP_IN, M, 64, EPI_F32, MLP_SPLITS))) return rc;
    DW1.g.out_f32 = b.pW1;
    if ((rc = gemm_launch(c, DW1, st))) return rc;
    GradParts gp;
    gp.dW1 = b.pW1;
    gp.s1 = int(DW1.grid.z);
    gp.dW2 = b.pW2;
    gp.s2 = int(DW2.grid.z);
    gp.db1 = b.pb1;
    gp.n1 = b.n_chunks;
    gp.db2 = b.pb2;
    gp.n2 = b.n_chunks;
    gp.w3 = b.pw3;
    gp.n3 = b.n_chunks;
    gp.loss = b.loss_part;
    gp.B = B;
    mlp_reduce_kernel<<<grid_for(MLP_P, 256, c->num_sms * 4), 256, 0, st>>>(gp, b.grad, loss_out, b.step);
    DRGB_CHECK_LAUNCH(c);
    return DRGB_OK;
}

static int mlp_check(Ctx* c, int d) {
    if (!c) return DRGB_ERR_INVALID;
    if (d < 1 || d > MLP_IN) return set_error(c, DRGB_ERR_INVALID, "mlp: d must be in 1..%d", MLP_IN);
    return DRGB_OK;
}

static int round_up(int64_t x, int64_t m) { return int((x + m - 1) / m * m); }

}  // namespace drgb

using namespace drgb;

extern "C" {

int64_t drgb_mlp_param_count(void) { return MLP_P; }

int drgb_mlp_init(drgb_ctx* c, float* params, int32_t d, uint64_t seed, void* stream) {
    int rc = mlp_check(c, d);
    if (rc) return rc;
    if (!params) return set_error(c, DRGB_ERR_INVALID, "mlp_init: NULL params");
    mlp_init_kernel<<<grid_for(MLP_P, 256, c->num_sms * 4), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        params, d, uint32_t(seed), uint32_t(seed >> 32));
    DRGB_CHECK_LAUNCH(c);
    return DRGB_OK;
}

int drgb_mlp_grad(drgb_ctx* c, const float* params, const float* X, int64_t n, int32_t d, const int32_t* rows,
                  int32_t n_edges, int32_t neg, float a, float b, float* grad_out, float* loss_out, void* stream) {
    int rc = mlp_check(c, d);
    if (rc) return rc;
    if (!params || !X || !rows || !grad_out || n_edges < 1 || neg < 0 || neg > 8 || n < 2)
        return set_error(c, DRGB_ERR_INVALID, "mlp_grad: bad arguments");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if ((rc = gemm_prepare(c))) return rc;
    const int Mv = n_edges * (2 + neg);
    const int M = round_up(Mv, 128);
    if ((rc = ensure_scratch(c, mlp_batch_bytes(M), st))) return rc;
    MlpBuffers bu = mlp_carve(c->scratch, M);
    DRGB_CUDA(c, cudaMemsetAsync(bu.rows, 0, size_t(M) * 4, st));
    DRGB_CUDA(c, cudaMemcpyAsync(bu.rows, rows, size_t(Mv) * 4, cudaMemcpyDeviceToDevice, st));
    DRGB_CUDA(c, cudaMemsetAsync(bu.step, 0, 64, st));
    mlp_cast_kernel<<<grid_for(MLP_H * MLP_H, 256, c->num_sms * 4), 256, 0, st>>>(params, bu.W);
    DRGB_CHECK_LAUNCH(c);
    mlp_gather_kernel<<<dim3(M / 32, MLP_IN / 32), dim3(32, 8), 0, st>>>(X, d, bu.rows, M, Mv, bu.Xb, bu.Xbt);
    DRGB_CHECK_LAUNCH(c);
    if ((rc = mlp_fwd_bwd(c, bu, params, n_edges, neg, a, b, loss_out, st))) return rc;
    DRGB_CUDA(c, cudaMemcpyAsync(grad_out, bu.grad, MLP_P * 4, cudaMemcpyDeviceToDevice, st));
    return drgb_sync(c, stream);
}

int drgb_mlp_train(drgb_ctx* c, const float* X, int64_t n, int32_t d, const int32_t* row_ptr, const int32_t* col,
                   const uint32_t* q, int64_t nnz, float a, float b, const drgb_mlp_params* mp, float* params,
                   float* adam_m, float* adam_v, float* losses, void* stream) {
    int rc = mlp_check(c, d);
    if (rc) return rc;
    if (!X || !row_ptr || !col || !q || !mp || !params || !adam_m || !adam_v || nnz < 1 || n < 2 ||
        mp->batch_edges < 1 || mp->neg < 0 || mp->neg > 8 || mp->steps < 0)
        return set_error(c, DRGB_ERR_INVALID, "mlp_train: bad arguments");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if ((rc = gemm_prepare(c))) return rc;
    const int B = mp->batch_edges, neg = mp->neg, R = 2 + neg;
    const int Mv = B * R;
    const int M = round_up(Mv, 128);
    if ((rc = ensure_scratch(c, mlp_batch_bytes(M), st))) return rc;
    MlpBuffers bu = mlp_carve(c->scratch, M);
    DRGB_CUDA(c, cudaMemsetAsync(bu.rows, 0, size_t(M) * 4, st));
    DRGB_CUDA(c, cudaMemsetAsync(bu.step, 0, 64, st));
    const uint32_t k0 = uint32_t(mp->seed), k1 = uint32_t(mp->seed >> 32);

    // capture one step, replay it mp->steps times (the step counter lives on
    // the device, so every replay draws a fresh batch)
    cudaStream_t cap;
    DRGB_CUDA(c, cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
        cudaStreamDestroy(cap);
        return set_error(c, DRGB_ERR_CUDA, "mlp_train: begin capture: %s", cudaGetErrorString(e));
    }
    do {
        mlp_cast_kernel<<<grid_for(MLP_H * MLP_H, 256, c->num_sms * 4), 256, 0, cap>>>(params, bu.W);
        if ((rc = [&]() { DRGB_CHECK_LAUNCH(c); return DRGB_OK; }())) break;
        mlp_sample_kernel<<<grid_for(B, 128, c->num_sms * 8), 128, 0, cap>>>(row_ptr, col, q, n, nnz, B, neg, bu.step,
                                                                            k0, k1, bu.rows);
        if ((rc = [&]() { DRGB_CHECK_LAUNCH(c); return DRGB_OK; }())) break;
        mlp_gather_kernel<<<dim3(M / 32, MLP_IN / 32), dim3(32, 8), 0, cap>>>(X, d, bu.rows, M, Mv, bu.Xb, bu.Xbt);
        if ((rc = [&]() { DRGB_CHECK_LAUNCH(c); return DRGB_OK; }())) break;
        if ((rc = mlp_fwd_bwd(c, bu, params, B, neg, a, b, losses, cap))) break;
        mlp_adam_kernel<<<grid_for(MLP_P, 256, c->num_sms * 4), 256, 0, cap>>>(
            params, adam_m, adam_v, bu.grad, mp->lr, mp->beta1, mp->beta2, mp->eps, bu.step);
        if ((rc = [&]() { DRGB_CHECK_LAUNCH(c); return DRGB_OK; }())) break;
        mlp_step_advance_kernel<<<1, 1, 0, cap>>>(bu.step);
        if ((rc = [&]() { DRGB_CHECK_LAUNCH(c); return DRGB_OK; }())) break;
    } while (0);
    e = cudaStreamEndCapture(cap, &graph);
    if (rc == DRGB_OK && e != cudaSuccess) rc = set_error(c, DRGB_ERR_CUDA, "mlp_train: end capture: %s", cudaGetErrorString(e));
    if (rc == DRGB_OK && (e = cudaGraphInstantiate(&exec, graph, 0)) != cudaSuccess)
        rc = set_error(c, DRGB_ERR_CUDA, "mlp_train: instantiate: %s", cudaGetErrorString(e));
    for (int s = 0; rc == DRGB_OK && s < mp->steps; ++s) {
        e = cudaGraphLaunch(exec, st);
        if (e != cudaSuccess) rc = set_error(c, DRGB_ERR_CUDA, "mlp_train: launch: %s", cudaGetErrorString(e));
    }
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    cudaStreamDestroy(cap);
    if (rc) return rc;
    return drgb_sync(c, stream);
}

int drgb_mlp_sample(drgb_ctx* c, const int32_t* row_ptr, const int32_t* col, const uint32_t* q, int64_t n,
                    int64_t nnz, int32_t n_edges, int32_t neg, uint32_t step, uint64_t seed, int32_t* rows,
                    void* stream) {
    if (!c) return DRGB_ERR_INVALID;
    if (!row_ptr || !col || !q || !rows || n < 2 || nnz < 1 || n_edges < 1 || neg < 0 || neg > 8)
        return set_error(c, DRGB_ERR_INVALID, "mlp_sample: bad arguments");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int rc = ensure_scratch(c, 256, st);
    if (rc) return rc;
    uint32_t* step_dev = static_cast<uint32_t*>(c->scratch);
    DRGB_CUDA(c, cudaMemcpyAsync(step_dev, &step, 4, cudaMemcpyHostToDevice, st));
    mlp_sample_kernel<<<grid_for(n_edges, 128, c->num_sms * 8), 128, 0, st>>>(row_ptr, col, q, n, nnz, n_edges, neg,
                                                                             step_dev, uint32_t(seed),
                                                                             uint32_t(seed >> 32), rows);
    DRGB_CHECK_LAUNCH(c);
    return drgb_sync(c, stream);
}

int drgb_mlp_embed(drgb_ctx* c, const float* params, const float* X, int64_t n, int32_t d, float* Y, void* stream) {
    int rc = mlp_check(c, d);
    if (rc) return rc;
    if (!params || !X || !Y || n < 1) return set_error(c, DRGB_ERR_INVALID, "mlp_embed: bad arguments");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if ((rc = gemm_prepare(c))) return rc;
    const int CH = 1 << 16;  // rows per chunk
    const size_t bytes = Carve::round(size_t(CH) * MLP_IN * 2) + 2 * Carve::round(size_t(CH) * MLP_H * 2) +
                         Carve::round(size_t(CH) * 2 * 4) + 2 * Carve::round(MLP_H * MLP_H * 2) +
                         Carve::round(MLP_H * MLP_IN * 2) + Carve::round(2 * MLP_H * 4) + 8192;
    if ((rc = ensure_scratch(c, bytes, st))) return rc;
    Carve cv(c->scratch);
    bf16* Xb = cv.take<bf16>(size_t(CH) * MLP_IN);
    bf16* H1 = cv.take<bf16>(size_t(CH) * MLP_H);
    bf16* H2 = cv.take<bf16>(size_t(CH) * MLP_H);
    float* z = cv.take<float>(size_t(CH) * 2);
    MlpWeights W;
    W.W2b = cv.take<bf16>(MLP_H * MLP_H);
    W.W2tb = cv.take<bf16>(MLP_H * MLP_H);
    W.W1b = cv.take<bf16>(MLP_H * MLP_IN);
    W.W3f = cv.take<float>(2 * MLP_H);
    mlp_cast_kernel<<<grid_for(MLP_H * MLP_H, 256, c->num_sms * 4), 256, 0, st>>>(params, W);
    DRGB_CHECK_LAUNCH(c);
    for (int64_t r0 = 0; r0 < n; r0 += CH) {
        const int mv = int(n - r0 < CH ? n - r0 : CH);
        const int M = round_up(mv, 128);
        mlp_gather_kernel<<<dim3(M / 32, MLP_IN / 32), dim3(32, 8), 0, st>>>(X + r0 * d, d, nullptr, M, mv, Xb,
                                                                            nullptr);
        DRGB_CHECK_LAUNCH(c);
        Gemm F1, F2;
        if ((rc = gemm_setup(c, F1, Xb, W.W1b, M, MLP_H, MLP_IN, 256, EPI_GELU, 1))) return rc;
        F1.g.bias = params + OFF_B1;
        F1.g.out = H1;
        if ((rc = gemm_setup(c, F2, H1, W.W2b, M, MLP_H, MLP_H, 256, EPI_GELU, 1))) return rc;
        F2.g.bias = params + OFF_B2;
        F2.g.out = H2;
        if ((rc = gemm_launch(c, F1, st)) || (rc = gemm_launch(c, F2, st))) return rc;
        mlp_head_kernel<<<grid_for(int64_t(M) * 32, 256, c->num_sms * 16), 256, 0, st>>>(H2, W.W3f, params, M, z);
        DRGB_CHECK_LAUNCH(c);
        DRGB_CUDA(c, cudaMemcpyAsync(Y + 2 * r0, z, size_t(mv) * 8, cudaMemcpyDeviceToDevice, st));
    }
    return DRGB_OK;
}

}  // extern "C"
