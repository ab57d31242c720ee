// PCA preprocessing to pca_dim (Section 3: the paper's timed pipeline starts
// from the raw features and reduces them by PCA): column means, the sample
// covariance C = Xc^T Xc / (n - 1), its `dim` leading eigenvectors V (each
// signed so that its largest-magnitude entry, lowest index among equals, is
// positive) and the projection Z = Xc V.
//
// Covariance on the tensor cores: Xc is staged transposed (D_pad x n_pad, the
// n points contiguous) as two BF16 parts, hi = bf16(xc) and lo = bf16(xc -
// hi), so that hi + lo carries 16 significant bits.  C = sym(hi hi^T) + hi
// lo^T + lo hi^T (the dropped lo lo^T is below 2^-16 of the diagonal), from
// two products of the tcgen05 GEMM (gemm.cuh) whose FP32 accumulation runs
// over at most 2048 points per split, the splits summed in FP64.
//
// Eigenvectors: Chebyshev-filtered subspace iteration (Zhou & Saad 2007) on a
// block of 64 vectors, all on the device: products C X (SIMT), FP64 Gram
// matrices, Cholesky QR in one CTA (FP64), and a Rayleigh-Ritz step whose
// small eigenproblem is a parallel cyclic Jacobi in one CTA (FP32).  Leading
// pairs whose residual |C v - theta v| is below 1e-5 theta_1 are locked and
// deflated from C (Hotelling), so the filter then works on the rest of the
// spectrum.  The host reads the Ritz values and residuals once per
// Rayleigh-Ritz step to steer the filter.  Stops when the dim leading pairs
// are locked, after 300 filter steps, or when the worst residual has not
// halved in 40.  Projection: a tiled FP32 SIMT product.
#include <cuda_bf16.h>

#include <cmath>
#include <vector>

#include "common.cuh"
#include "gemm.cuh"
#include "pca.cuh"

namespace drgb {

static constexpr int PCA_P = 64;        // subspace block
static constexpr int PCA_MAX_D = PCA_MAX_FEATURES;
static constexpr int PCA_DEG = 10;      // Chebyshev degree per step
static constexpr int PCA_MAXIT = 300;
static constexpr int PCA_STALL = 40;
static constexpr double PCA_TOL = 1e-5;
static constexpr int PCA_MEAN_CHUNKS = 2048;
static constexpr int PCA_GCHUNK = 64;   // rows per partial Gram
static constexpr int PCA_KCHUNK = 128;  // rows of X per split of the product C X
static constexpr int PCA_CROWS = 16;    // rows of C per block of the product
static constexpr int PCA_RR_EVERY = 3;  // filter steps per Rayleigh-Ritz step
static constexpr double PCA_GROWTH = 1e4;  // largest filter gain over the damped interval
static constexpr int PCA_CHAIN_KB = 32;  // 64-point K blocks per accumulation chain of the covariance

static int64_t round_up(int64_t v, int64_t m) { return (v + m - 1) / m * m; }

// Float-float accumulation (Knuth's TwoSum): (hi, lo) += v, exactly up to
// the rounding of lo; keeps sums on the FP32 pipes, which run about 64 times
// the FP64 rate on this part.
__device__ __forceinline__ void ff_add(float& hi, float& lo, float v) {
    const float s = __fadd_rn(hi, v);
    const float bb = __fsub_rn(s, hi);
    lo = __fadd_rn(lo, __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(v, bb)));
    hi = s;
}

// Column sums of row chunk blockIdx.x (FP64), one thread per column.
__global__ void pca_colsum_kernel(const float* __restrict__ X, int64_t n, int D, int64_t rows_per,
                                  double* __restrict__ part) {
    const int64_t r0 = int64_t(blockIdx.x) * rows_per;
    const int64_t r1 = r0 + rows_per < n ? r0 + rows_per : n;
    const int j = blockIdx.y * blockDim.x + threadIdx.x;
    if (j >= D) return;
    float h0 = 0.f, l0 = 0.f, h1 = 0.f, l1 = 0.f;
    int64_t i = r0;
    for (; i + 2 <= r1; i += 2) {
        ff_add(h0, l0, X[i * D + j]);
        ff_add(h1, l1, X[(i + 1) * D + j]);
    }
    if (i < r1) ff_add(h0, l0, X[i * D + j]);
    part[int64_t(blockIdx.x) * D + j] = (double(h0) + double(l0)) + (double(h1) + double(l1));
}

// mu_j = sum over the chunks / n: one block per column, a fixed-order tree.
__global__ void pca_mean_kernel(const double* __restrict__ part, int chunks, int64_t n, int D, float* __restrict__ mu) {
    __shared__ double red[256];
    const int j = blockIdx.x;
    double s = 0.0;
    for (int c = threadIdx.x; c < chunks; c += blockDim.x) s += part[int64_t(c) * D + j];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (int(threadIdx.x) < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) mu[j] = float(red[0] / double(n));
}

// hi[j][i], lo[j][i] = the split of X[i][j] - mu[j] (zero outside n x D),
// through 32 x 32 tiles in shared memory.
__global__ void pca_stage_kernel(const float* __restrict__ X, const float* __restrict__ mu, int64_t n, int D,
                                 int64_t n_pad, int D_pad, __nv_bfloat16* __restrict__ hi,
                                 __nv_bfloat16* __restrict__ lo) {
    __shared__ float tile[32][33];
    const int64_t i0 = int64_t(blockIdx.x) * 32;
    const int j0 = blockIdx.y * 32;
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int64_t i = i0 + r;
        const int j = j0 + threadIdx.x;
        tile[r][threadIdx.x] = (i < n && j < D) ? X[i * D + j] - mu[j] : 0.f;
    }
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int j = j0 + r;
        const int64_t i = i0 + threadIdx.x;
        if (j < D_pad && i < n_pad) {
            const float v = tile[threadIdx.x][r];
            const __nv_bfloat16 h = __float2bfloat16_rn(v);
            hi[int64_t(j) * n_pad + i] = h;
            lo[int64_t(j) * n_pad + i] = __float2bfloat16_rn(v - __bfloat162float(h));
        }
    }
}

// T = sum_z (hh_z + hl_z) and Hs = sum_z hh_z over the split partials
// (each D_pad x D_pad), float-float in split order, stored as FP64; a, b < D.
__global__ void pca_covsum_kernel(const float* __restrict__ hh, const float* __restrict__ hl, int S, int D_pad,
                                  int D, double* __restrict__ T, double* __restrict__ Hs) {
    const int64_t total = int64_t(D) * D, stride = int64_t(D_pad) * D_pad;
    for (int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < total; t += int64_t(gridDim.x) * blockDim.x) {
        const int a = int(t / D), b = int(t - int64_t(a) * D);
        const int64_t off = int64_t(a) * D_pad + b;
        float th = 0.f, tl = 0.f, hh_ = 0.f, hl_ = 0.f;
#pragma unroll 4
        for (int z = 0; z < S; ++z) {
            const float h = hh[z * stride + off], l = hl[z * stride + off];
            ff_add(hh_, hl_, h);
            ff_add(th, tl, h);
            ff_add(th, tl, l);
        }
        T[t] = double(th) + double(tl);
        Hs[t] = double(hh_) + double(hl_);
    }
}

// C = (T + T^T - (Hs + Hs^T) / 2) / (n - 1) = (sym(hi hi^T) + hi lo^T +
// lo hi^T) / (n - 1): FP32, and FP64 when C64 is given.
__global__ void pca_cov_kernel(const double* __restrict__ T, const double* __restrict__ Hs, int D, int64_t n,
                               float* __restrict__ C, double* __restrict__ C64) {
    const int64_t total = int64_t(D) * D;
    for (int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < total; t += int64_t(gridDim.x) * blockDim.x) {
        const int a = int(t / D), b = int(t - int64_t(a) * D);
        const int64_t u = int64_t(b) * D + a;
        const double v = (T[t] + T[u] - 0.5 * (Hs[t] + Hs[u])) / double(n - 1);
        C[t] = float(v);
        if (C64) C64[t] = v;
    }
}

// Blocks are D x P row-major; columns < L are the locked vectors, columns
// L..P-1 the active ones (m = P - L of them).

// part[s][a][p] = sum over b in split s (PCA_KCHUNK rows) of C[a][b] X[b][p]:
// a block takes PCA_CROWS rows of C and one split, both staged in shared
// memory; a thread computes 4 adjacent columns of one row.
__global__ void __launch_bounds__(256) pca_cmul_part_kernel(const float* __restrict__ C, int D,
                                                            const float* __restrict__ X, float* __restrict__ part) {
    __shared__ __align__(16) float Xs[PCA_KCHUNK][PCA_P];
    __shared__ float Cs[PCA_CROWS][PCA_KCHUNK + 1];
    const int a0 = blockIdx.x * PCA_CROWS, b0 = blockIdx.y * PCA_KCHUNK;
    const int kb = D - b0 < PCA_KCHUNK ? D - b0 : PCA_KCHUNK;
    // all of a thread's loads are issued before any is stored, so the block
    // waits for one round trip instead of one per element
    constexpr int NX = PCA_KCHUNK * (PCA_P / 4) / 256, NC = PCA_CROWS * PCA_KCHUNK / 256;
    float4 xv[NX];
    float cv_[NC];
#pragma unroll
    for (int u = 0; u < NX; ++u) {
        const int t = threadIdx.x + u * 256, k = t / (PCA_P / 4), c4 = t % (PCA_P / 4);
        xv[u] = k < kb ? *reinterpret_cast<const float4*>(X + int64_t(b0 + k) * PCA_P + 4 * c4)
                       : make_float4(0.f, 0.f, 0.f, 0.f);
    }
#pragma unroll
    for (int u = 0; u < NC; ++u) {
        const int t = threadIdx.x + u * 256, r = t / PCA_KCHUNK, k = t % PCA_KCHUNK;
        cv_[u] = (k < kb && a0 + r < D) ? C[int64_t(a0 + r) * D + b0 + k] : 0.f;
    }
#pragma unroll
    for (int u = 0; u < NX; ++u) {
        const int t = threadIdx.x + u * 256;
        *reinterpret_cast<float4*>(&Xs[t / (PCA_P / 4)][4 * (t % (PCA_P / 4))]) = xv[u];
    }
#pragma unroll
    for (int u = 0; u < NC; ++u) {
        const int t = threadIdx.x + u * 256;
        Cs[t / PCA_KCHUNK][t % PCA_KCHUNK] = cv_[u];
    }
    __syncthreads();
    const int r = threadIdx.x / (PCA_P / 4), c4 = threadIdx.x % (PCA_P / 4);
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int k = 0; k < kb; ++k) {
        const float cv = Cs[r][k];
        const float4 x = *reinterpret_cast<const float4*>(&Xs[k][4 * c4]);
        acc.x = fmaf(cv, x.x, acc.x);
        acc.y = fmaf(cv, x.y, acc.y);
        acc.z = fmaf(cv, x.z, acc.z);
        acc.w = fmaf(cv, x.w, acc.w);
    }
    if (a0 + r < D)
        *reinterpret_cast<float4*>(part + (int64_t(blockIdx.y) * D + a0 + r) * PCA_P + 4 * c4) = acc;
}

// Active columns: Y = alpha C X + beta X + gamma Z, C X the sum of the splits
// in order; locked columns: Y = X.
__global__ void pca_cmul_kernel(const float* __restrict__ part, int nsplit, int D, const float* __restrict__ X,
                                const float* __restrict__ Z, float alpha, float beta, float gamma, int L,
                                float* __restrict__ Y) {
    const int64_t total = int64_t(D) * PCA_P;
    for (int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < total; t += int64_t(gridDim.x) * blockDim.x) {
        const int p = int(t % PCA_P);
        if (p < L) {
            Y[t] = X[t];
            continue;
        }
        float s = 0.f;
        for (int z = 0; z < nsplit; ++z) s += part[z * total + t];
        float y = alpha * s + beta * X[t];
        if (Z) y = fmaf(gamma, Z[t], y);
        Y[t] = y;
    }
}

// Gp[z][p][q] = sum over rows a of chunk z of A[a][p] B[a][L + q], p < P,
// q < m (chunks of PCA_GCHUNK rows, staged in shared memory).  The sum runs
// in float-float arithmetic (Ogita, Rump & Oishi 2005, Dot2: the exact
// product split by an FMA, the running sum by Knuth's TwoSum), about as
// accurate as FP64 and all on the FP32 pipes, and is stored as FP64.
__global__ void __launch_bounds__(256) pca_gram_kernel(const float* __restrict__ A, const float* __restrict__ B,
                                                       int D, int L, double* __restrict__ Gp) {
    __shared__ float As[PCA_GCHUNK][PCA_P + 1];
    __shared__ float Bs[PCA_GCHUNK][PCA_P + 1];
    const int m = PCA_P - L;
    const int a0 = blockIdx.y * PCA_GCHUNK;
    const int rows = D - a0 < PCA_GCHUNK ? D - a0 : PCA_GCHUNK;
    {  // all loads issued before any store
        constexpr int NU = PCA_GCHUNK * PCA_P / 4 / 256;
        float4 av[NU], bv[NU];
#pragma unroll
        for (int u = 0; u < NU; ++u) {
            const int t = threadIdx.x + u * 256, a = t / (PCA_P / 4), c4 = t % (PCA_P / 4);
            const bool ok = a < rows;
            av[u] = ok ? *reinterpret_cast<const float4*>(A + int64_t(a0 + a) * PCA_P + 4 * c4)
                       : make_float4(0.f, 0.f, 0.f, 0.f);
            bv[u] = ok ? *reinterpret_cast<const float4*>(B + int64_t(a0 + a) * PCA_P + 4 * c4)
                       : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int u = 0; u < NU; ++u) {
            const int t = threadIdx.x + u * 256, a = t / (PCA_P / 4), c = 4 * (t % (PCA_P / 4));
            As[a][c] = av[u].x;
            As[a][c + 1] = av[u].y;
            As[a][c + 2] = av[u].z;
            As[a][c + 3] = av[u].w;
            Bs[a][c] = bv[u].x;
            Bs[a][c + 1] = bv[u].y;
            Bs[a][c + 2] = bv[u].z;
            Bs[a][c + 3] = bv[u].w;
        }
    }
    __syncthreads();
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= PCA_P * m) return;
    const int p = t / m, q = L + (t - p * m);
    float hi = 0.f, lo = 0.f;
    for (int a = 0; a < rows; ++a) {
        const float x = As[a][p], y = Bs[a][q];
        const float pr = __fmul_rn(x, y);
        const float pe = fmaf(x, y, -pr);
        const float s = __fadd_rn(hi, pr);
        const float bb = __fsub_rn(s, hi);
        const float se = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(pr, bb));
        hi = s;
        lo = __fadd_rn(lo, __fadd_rn(se, pe));
    }
    Gp[int64_t(blockIdx.y) * PCA_P * m + t] = double(hi) + double(lo);
}

// G[t] = sum_z Gp[z][t] (chunk order), t < P m.
__global__ void pca_gsum_kernel(const double* __restrict__ Gp, int nch, int pm, double* __restrict__ G) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= pm) return;
    double v = 0.0;
    for (int z = 0; z < nch; ++z) v += Gp[int64_t(z) * pm + t];
    G[t] = v;
}

// rn[j] = sum_a (W[a][L + j] - theta_j Y[a][L + j])^2 (FP64), one warp per
// active column.
__global__ void pca_resid_kernel(const float* __restrict__ Y, const float* __restrict__ W,
                                 const float* __restrict__ theta, int D, int L, double* __restrict__ rn) {
    const int j = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (j >= PCA_P - L) return;
    const int k = L + j;
    const float th = theta[j];
    double s = 0.0;
    for (int a = lane; a < D; a += 32) {
        const double r = double(W[int64_t(a) * PCA_P + k]) - double(th) * double(Y[int64_t(a) * PCA_P + k]);
        s = fma(r, r, s);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) rn[j] = s;
}

// Locked columns: Y = X; active columns: Y[a][L + q] = sum_p X[a][p] M[p][q]
// (M: P x m, device).
__global__ void pca_apply_kernel(const float* __restrict__ X, int D, const float* __restrict__ M, int L,
                                 float* __restrict__ Y) {
    const int m = PCA_P - L;
    const int64_t total = int64_t(D) * PCA_P;
    for (int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < total; t += int64_t(gridDim.x) * blockDim.x) {
        const int a = int(t / PCA_P), q = int(t - int64_t(a) * PCA_P);
        if (q < L) {
            Y[t] = X[t];
            continue;
        }
        const float* Xa = X + int64_t(a) * PCA_P;
        float s = 0.f;
        for (int p = 0; p < PCA_P; ++p) s = fmaf(Xa[p], M[p * m + (q - L)], s);
        Y[t] = s;
    }
}

// Mode 0 of the orthonormalisation step (the mode word is the factor
// kernel's): Y = X T^-1 for the upper-triangular T = [I, W; 0, R]
// (Y[:, :L] = X[:, :L], Y[:, L:] = (X[:, L:] - X[:, :L] W) R^-1), each thread
// solving y T = x for one row by forward substitution.  Rows pass through
// shared memory to keep global accesses coalesced.
__global__ void __launch_bounds__(64) pca_tsolve_kernel(const float* __restrict__ X, int D,
                                                        const float* __restrict__ T, const int* __restrict__ mode,
                                                        float* __restrict__ Y) {
    __shared__ float Ts[PCA_P][PCA_P];
    __shared__ float rdiag[PCA_P];
    __shared__ float Xs[64][PCA_P + 1];
    const int a0 = blockIdx.x * 64;
    const int rows = D - a0 < 64 ? D - a0 : 64;
    if (*mode != 0) return;
    for (int u = threadIdx.x; u < PCA_P * PCA_P; u += blockDim.x) Ts[u / PCA_P][u % PCA_P] = T[u];
    for (int u = threadIdx.x; u < rows * PCA_P; u += blockDim.x) Xs[u / PCA_P][u % PCA_P] = X[int64_t(a0) * PCA_P + u];
    __syncthreads();
    if (threadIdx.x < PCA_P) rdiag[threadIdx.x] = 1.f / Ts[threadIdx.x][threadIdx.x];
    __syncthreads();
    if (int(threadIdx.x) < rows) {
        float y[PCA_P];
#pragma unroll
        for (int j = 0; j < PCA_P; ++j) {
            float v = Xs[threadIdx.x][j];
#pragma unroll
            for (int i = 0; i < j; ++i) v = fmaf(-y[i], Ts[i][j], v);
            y[j] = v * rdiag[j];
        }
#pragma unroll
        for (int j = 0; j < PCA_P; ++j) Xs[threadIdx.x][j] = y[j];
    }
    __syncthreads();
    for (int u = threadIdx.x; u < rows * PCA_P; u += blockDim.x) Y[int64_t(a0) * PCA_P + u] = Xs[u / PCA_P][u % PCA_P];
}

// Mode 1 of the orthonormalisation step: Y = X M, M general P x P, one
// thread per output.
__global__ void pca_mprod_kernel(const float* __restrict__ X, int D, const float* __restrict__ M,
                                 const int* __restrict__ mode, float* __restrict__ Y) {
    if (*mode != 1) return;
    const int64_t total = int64_t(D) * PCA_P;
    for (int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < total; t += int64_t(gridDim.x) * blockDim.x) {
        const int a = int(t / PCA_P), q = int(t % PCA_P);
        const float* Xa = X + int64_t(a) * PCA_P;
        float s = 0.f;
#pragma unroll 16
        for (int p = 0; p < PCA_P; ++p) s = fmaf(Xa[p], M[p * PCA_P + q], s);
        Y[t] = s;
    }
}

// Hotelling deflation by newly locked pairs: C[a][b] -= sum_{k0 <= k < k1}
// theta_k X[a][k] X[b][k] (the same expression for (a, b) and (b, a), so C
// stays exactly symmetric), by 32 x 32 tiles with the rows' X staged in
// shared memory.
__global__ void __launch_bounds__(256) pca_deflate_kernel(float* __restrict__ C, int D, const float* __restrict__ X,
                                                          const float* __restrict__ theta, int k0, int k1) {
    __shared__ float Xa[32][PCA_P + 1], Xb[32][PCA_P + 1];
    const int a0 = blockIdx.y * 32, b0 = blockIdx.x * 32, nk = k1 - k0;
    for (int u = threadIdx.x; u < 32 * nk; u += blockDim.x) {
        const int r = u / nk, k = u - r * nk;
        Xa[r][k] = (a0 + r < D) ? X[int64_t(a0 + r) * PCA_P + k0 + k] : 0.f;
        Xb[r][k] = (b0 + r < D) ? X[int64_t(b0 + r) * PCA_P + k0 + k] : 0.f;
    }
    __syncthreads();
    const int bl = threadIdx.x & 31;
    for (int al = threadIdx.x >> 5; al < 32; al += blockDim.x >> 5) {
        const int a = a0 + al, b = b0 + bl;
        if (a >= D || b >= D) continue;
        float s = 0.f;
        for (int k = 0; k < nk; ++k) s = fmaf(theta[k], Xa[al][k] * Xb[bl][k], s);
        C[int64_t(a) * D + b] -= s;
    }
}

// Starting block: uniform values in [-1, 1) from Philox at counter (a, g, 0, 4).
__global__ void pca_start_kernel(int D, float* __restrict__ X) {
    for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < D; a += gridDim.x * blockDim.x) {
        for (int g = 0; g < PCA_P / 4; ++g) {
            const U4 r = philox4x32_10(U4{uint32_t(a), uint32_t(g), 0u, 4u}, 0x5ca1ab1eu, 0u);
            const uint32_t u[4] = {r.x, r.y, r.z, r.w};
            for (int k = 0; k < 4; ++k)
                X[int64_t(a) * PCA_P + 4 * g + k] = fmaf(float(u[k] >> 8), 2.0f * 5.9604644775390625e-08f, -1.0f);
        }
    }
}

// Z[i][k] = sum_j (X[i][j] - mu[j]) V[j][k] for k < dim: 64 x 64 output
// tiles, 16 x 16 threads with 4 x 4 outputs each, D in steps of 32.
__global__ void __launch_bounds__(256) pca_project_kernel(const float* __restrict__ X, const float* __restrict__ mu,
                                                          const float* __restrict__ V, int64_t n, int D, int dim,
                                                          float* __restrict__ Z) {
    __shared__ float As[64][33];
    __shared__ float Bs[32][65];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int64_t i0 = int64_t(blockIdx.x) * 64;
    float acc[4][4] = {};
    for (int j0 = 0; j0 < D; j0 += 32) {
        for (int t = threadIdx.x; t < 64 * 32; t += 256) {
            const int r = t / 32, cc = t % 32;
            const int64_t i = i0 + r;
            const int j = j0 + cc;
            As[r][cc] = (i < n && j < D) ? X[i * D + j] - mu[j] : 0.f;
        }
        for (int t = threadIdx.x; t < 32 * 64; t += 256) {
            const int r = t / 64, cc = t % 64;
            const int j = j0 + r;
            Bs[r][cc] = (j < D && cc < dim) ? V[int64_t(j) * PCA_P + cc] : 0.f;
        }
        __syncthreads();
#pragma unroll 8
        for (int kk = 0; kk < 32; ++kk) {
            float a[4], b[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                a[u] = As[ty * 4 + u][kk];
                b[u] = Bs[kk][tx * 4 + u];
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) acc[u][v] = fmaf(a[u], b[v], acc[u][v]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const int64_t i = i0 + ty * 4 + u;
        if (i >= n) continue;
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const int k = tx * 4 + v;
            if (k < dim) Z[i * dim + k] = acc[u][v];
        }
    }
}

// V_out[k][j] = V[j][k] (components as rows).
__global__ void pca_components_kernel(const float* __restrict__ V, int D, int dim, float* __restrict__ out) {
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < D * dim; t += gridDim.x * blockDim.x) {
        const int k = t / D, j = t - k * D;
        out[t] = V[int64_t(j) * PCA_P + k];
    }
}

// ------------------------------------------------------------ small dense steps (one CTA)
static constexpr int PCA_CHOL_THREADS = 512;
static constexpr int PCA_JAC_THREADS = 1024;
static constexpr int PCA_JAC_SWEEPS = 6;

// The factor of one orthonormalisation pass, from G = X^T X[:, L:] (P x m)
// with W = G[:L] (the active columns' overlap with the locked ones).
// Pass 0, and any pass after a shifted one: S = sym(G[L:]) - W^T W (the Gram
// of the active columns after projection off the locked ones; W is tiny, so
// W^T W is taken in FP32), S (+ shift) = R^T R in FP64, and T = [I, W; 0, R]
// (P x P, FP32) with mode 0 for pca_tsolve_kernel, which forms X T^-1 =
// [X_L, (X_a - X_L W) R^-1] (Cholesky QR).  Pass 0 also requires min R_jj >
// 1e-5 max R_jj; where the plain factor fails that or breaks down, it is
// retaken of S + 1e-10 tr(S) I (shifted Cholesky QR, Fukaya et al. 2020),
// flags[0] is set and the later passes are Cholesky QR too; a shifted factor
// that still breaks down sets flags[1] and writes T = I.  Passes 1 and 2
// otherwise find the block orthonormal to about cond 2^-24 and take one
// Newton-Schulz step: M = [I, -W; 0, I - (S - I) / 2] with mode 1, i.e. X_a
// <- X_a (3 I - S) / 2 - X_L W, which squares the distance from
// orthonormality.
static constexpr int PCA_MODE = 2;  // index of the mode word in the flags
static constexpr size_t PCA_CHOL_SMEM = size_t(2) * PCA_P * PCA_P * sizeof(double) + size_t(PCA_P) * PCA_P * 4;
__global__ void __launch_bounds__(PCA_CHOL_THREADS) pca_chol_kernel(const double* __restrict__ G, int L, int pass,
                                                                   int* __restrict__ flags, float* __restrict__ T) {
    extern __shared__ double csm[];
    const int m = PCA_P - L;
    const int tid = threadIdx.x, nt = blockDim.x;
    if (pass > 0 && flags[0] == 0) {  // Newton-Schulz step
        for (int t = tid; t < PCA_P * PCA_P; t += nt) {
            const int row = t / PCA_P, col = t - row * PCA_P;
            float v;
            if (col < L) v = (row == col) ? 1.f : 0.f;
            else if (row < L) v = -float(G[row * m + (col - L)]);
            else {
                const int i = row - L, j = col - L;
                const double sij = 0.5 * (G[(L + i) * m + j] + G[(L + j) * m + i]);
                v = float((i == j ? 1.5 : 0.0) - 0.5 * sij);
            }
            T[t] = v;
        }
        if (tid == 0) flags[PCA_MODE] = 1;
        return;
    }
    if (tid == 0) flags[PCA_MODE] = 0;
    double* Gs = csm;                                         // P x m
    double* R = Gs + PCA_P * PCA_P;                           // m x m
    float* Wf = reinterpret_cast<float*>(R + PCA_P * PCA_P);  // L x m
    __shared__ int s_fail, s_ok;
    __shared__ double s_shift, s_rinv;
    for (int t = tid; t < PCA_P * m; t += nt) {
        const double v = G[t];
        Gs[t] = v;
        if (t < L * m) Wf[t] = float(v);
    }
    __syncthreads();
    bool identity = false;
    double shift = 0.0;
    for (int attempt = 0; attempt < 2; ++attempt) {
        for (int t = tid; t < m * m; t += nt) {
            const int i = t / m, j = t - i * m;
            float ww = 0.f;
            for (int k = 0; k < L; ++k) ww = fmaf(Wf[k * m + i], Wf[k * m + j], ww);
            R[t] = 0.5 * (Gs[(L + i) * m + j] + Gs[(L + j) * m + i]) - double(ww) + (i == j ? shift : 0.0);
        }
        if (tid == 0) s_fail = 0;
        __syncthreads();
        for (int j = 0; j < m; ++j) {
            if (tid == 0) {  // one FP64 square root and reciprocal per column
                double d = R[j * m + j];
                if (!(d > 0.0)) {
                    s_fail = 1;
                    d = 1.0;
                }
                const double rjj = sqrt(d);
                R[j * m + j] = rjj;
                s_rinv = 1.0 / rjj;
            }
            __syncthreads();
            const double rinv = s_rinv;
            for (int i = j + 1 + tid; i < m; i += nt) R[j * m + i] *= rinv;
            __syncthreads();
            {
                const int k = j + 1 + (tid & (PCA_P - 1));  // a column per lane group, rows by stride
                if (k < m) {
                    const double rjk = R[j * m + k];
                    for (int i = j + 1 + (tid >> 6); i <= k; i += nt >> 6) R[i * m + k] -= R[j * m + i] * rjk;
                }
            }
            __syncthreads();
        }
        if (tid == 0) {
            int ok = !s_fail;
            if (ok && pass == 0 && attempt == 0) {
                double rmax = 0.0, rmin = 1e300;
                for (int k = 0; k < m; ++k) {
                    rmax = fmax(rmax, R[k * m + k]);
                    rmin = fmin(rmin, R[k * m + k]);
                }
                ok = rmin > 1e-5 * rmax;
            }
            s_ok = ok;
            if (!ok && attempt == 0) {
                double tr = 0.0;
                for (int i = 0; i < m; ++i) tr += Gs[(L + i) * m + i];
                s_shift = 1e-10 * fabs(tr);
                flags[0] = 1;
            }
            if (!ok && attempt == 1) flags[1] = 1;
            if (ok && attempt == 0 && pass == 0) flags[0] = 0;
        }
        __syncthreads();
        if (s_ok) break;
        if (attempt == 1) identity = true;
        shift = s_shift;
    }
    for (int t = tid; t < PCA_P * PCA_P; t += nt) {
        const int row = t / PCA_P, col = t - row * PCA_P;
        float v;
        if (identity) v = (row == col) ? 1.f : 0.f;
        else if (row < L) v = (col < L) ? (row == col ? 1.f : 0.f) : Wf[row * m + (col - L)];
        else v = (col < row) ? 0.f : float(R[(row - L) * m + (col - L)]);
        T[t] = v;
    }
}

// Eigen-decomposition of the symmetric m x m matrix H (m <= 64), H[i][j] =
// sym(sum_z Gp[z][(row0 + i) ld + j]), by parallel cyclic Jacobi in FP32.
// Each round applies m/2 disjoint rotations (round-robin pairing); warp w
// owns pair w, computes its rotation in every lane (the stable
// form t = sign(z) / (|z| + sqrt(z^2 + 1)), z = (h_qq - h_pp) / (2 h_pq)),
// rotates rows p and q, then (after a barrier) columns p and q and the
// eigenvector matrix, writing the rotated 2 x 2 block in closed form (zero
// off the diagonal).  A pair is rotated only while |h_pq| > 2.5e-7 max_i
// |h_ii| (near the FP32 rounding of the rotations themselves, far below the
// 1e-5 residual the iteration asks for); the sweeps stop after one that
// rotates nothing, at most 6 (a Rayleigh-Ritz step that stops short only
// leaves its vectors' residuals larger, which the locking test sees).  Output, by decreasing eigenvalue: th_f, th_d,
// and eigenvector k as column k of Vout rows row_out..row_out+m-1 (leading
// dimension ldv); rows < row_out are zeroed when zero_lead.
__global__ void __launch_bounds__(PCA_JAC_THREADS) pca_jacobi_kernel(const double* __restrict__ Gp, int nparts,
                                                                    int64_t part_stride, int ld, int row0, int m,
                                                                    float* __restrict__ Vout, int ldv, int row_out,
                                                                    int zero_lead, float* __restrict__ th_f,
                                                                    double* __restrict__ th_d) {
    __shared__ float H[PCA_P][PCA_P + 1];
    __shared__ float V[PCA_P][PCA_P + 1];
    __shared__ float s_thr;
    __shared__ int s_rot;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int t = tid; t < m * m; t += blockDim.x) {
        const int i = t / m, j = t - i * m;
        double a = 0.0, b = 0.0;
        for (int z = 0; z < nparts; ++z) {
            a += Gp[z * part_stride + int64_t(row0 + i) * ld + j];
            b += Gp[z * part_stride + int64_t(row0 + j) * ld + i];
        }
        H[i][j] = float(0.5 * (a + b));
        V[i][j] = (i == j) ? 1.f : 0.f;
    }
    __syncthreads();
    if (tid == 0) {
        float mx = 0.f;
        for (int i = 0; i < m; ++i) mx = fmaxf(mx, fabsf(H[i][i]));
        s_thr = 2.5e-7f * mx;
    }
    const int Mv = (m + 1) & ~1;  // with a dummy index m when m is odd
    const int half = Mv / 2, n1 = Mv - 1;
    for (int sweep = 0; sweep < PCA_JAC_SWEEPS && Mv > 1; ++sweep) {
        if (tid == 0) s_rot = 0;
        __syncthreads();
        static_assert(PCA_JAC_THREADS == 32 * (PCA_P / 2), "one rotation pair per warp");
        for (int r = 0; r < n1; ++r) {
            // warp w's pair of this round (round-robin: position 0 fixed, the
            // others rotating), its rotation computed in every lane
            int p = -1, q = -1;
            float cs = 1.f, sn = 0.f, dp = 0.f, dq = 0.f;
            if (warp < half) {
                int a = 0;
                if (warp > 0) {
                    a = warp - 1 + r;
                    a = 1 + (a >= n1 ? a - n1 : a);
                }
                int b = n1 - 1 - warp + r;
                b = 1 + (b >= n1 ? b - n1 : b);
                const int pa = min(a, b), qa = max(a, b);
                if (qa < m) {
                    const float apq = H[pa][qa], app = H[pa][pa], aqq = H[qa][qa];
                    if (fabsf(apq) > s_thr) {
                        // fast divide and reciprocal square root, then one
                        // Newton step on c = 1 / sqrt(1 + t^2) so that
                        // c^2 + s^2 = 1 to rounding (t itself need not be exact)
                        const float z = __fdividef(aqq - app, 2.f * apq);
                        const float t = __fdividef(copysignf(1.f, z), fabsf(z) + __fsqrt_rn(fmaf(z, z, 1.f)));
                        const float u = fmaf(t, t, 1.f);
                        float c = rsqrtf(u);
                        c = fmaf(-0.5f * fmaf(c * c, u, -1.f), c, c);
                        p = pa;
                        q = qa;
                        cs = c;
                        sn = t * c;
                        dp = fmaf(-t, apq, app);
                        dq = fmaf(t, apq, aqq);
                    }
                }
            }
            if (lane == 0 && p >= 0) s_rot = 1;
            if (p >= 0) {  // rows p, q
#pragma unroll
                for (int hh = 0; hh < PCA_P / 32; ++hh) {
                    const int k = lane + 32 * hh;
                    if (k < m) {
                        const float x = H[p][k], y = H[q][k];
                        H[p][k] = cs * x - sn * y;
                        H[q][k] = sn * x + cs * y;
                    }
                }
            }
            __syncthreads();
            if (p >= 0) {  // columns p, q (the 2 x 2 block in closed form) and the eigenvectors
#pragma unroll
                for (int hh = 0; hh < PCA_P / 32; ++hh) {
                    const int k = lane + 32 * hh;
                    if (k < m) {
                        const float x = H[k][p], y = H[k][q];
                        float nx = cs * x - sn * y, ny = sn * x + cs * y;
                        nx = k == p ? dp : (k == q ? 0.f : nx);
                        ny = k == q ? dq : (k == p ? 0.f : ny);
                        H[k][p] = nx;
                        H[k][q] = ny;
                        const float u = V[k][p], w = V[k][q];
                        V[k][p] = cs * u - sn * w;
                        V[k][q] = sn * u + cs * w;
                    }
                }
            }
            __syncthreads();
        }
        if (s_rot == 0) break;
        __syncthreads();  // s_rot is reset only after every thread has read it
    }
    if (zero_lead)
        for (int t = tid; t < row_out * ldv; t += blockDim.x) Vout[t] = 0.f;
    for (int k = tid; k < m; k += blockDim.x) {
        const float d = H[k][k];
        int rank = 0;
        for (int j = 0; j < m; ++j) rank += (H[j][j] > d) || (H[j][j] == d && j < k);
        th_f[rank] = d;
        th_d[rank] = double(d);
        for (int i = 0; i < m; ++i) Vout[int64_t(row_out + i) * ldv + rank] = V[i][k];
    }
}

// Column k < dim of V (D rows, leading dimension ld) negated unless its
// largest-magnitude entry (lowest index among equals) is positive; one warp
// per column.
__global__ void pca_sign_kernel(float* __restrict__ V, int D, int ld, int dim) {
    const int k = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (k >= dim) return;
    float best = -1.f;
    int idx = D;
    for (int a = lane; a < D; a += 32) {
        const float v = fabsf(V[int64_t(a) * ld + k]);
        if (v > best) {
            best = v;
            idx = a;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, idx, o);
        if (ob > best || (ob == best && oi < idx)) {
            best = ob;
            idx = oi;
        }
    }
    if (V[int64_t(idx) * ld + k] < 0.f)
        for (int a = lane; a < D; a += 32) V[int64_t(a) * ld + k] = -V[int64_t(a) * ld + k];
}

// ------------------------------------------------------------------ host
// T_m(x) for x >= 1.
static double cheb_t(int m, double x) {
    double t0 = 1.0, t1 = x;
    for (int k = 2; k <= m; ++k) {
        const double t2 = 2.0 * x * t1 - t0;
        t0 = t1;
        t1 = t2;
    }
    return m == 0 ? 1.0 : t1;
}

static int pca_splits(int64_t n_pad) {
    const int kbs = int(n_pad / 64);
    return (kbs + PCA_CHAIN_KB - 1) / PCA_CHAIN_KB;
}

size_t pca_scratch_bytes(int64_t n, int D) {
    const int64_t n_pad = round_up(n, 64), D_pad = round_up(D, 128);
    const size_t blk = Carve::round(size_t(D) * PCA_P * 4);
    const int nch = (D + PCA_GCHUNK - 1) / PCA_GCHUNK;
    const size_t dd = size_t(D) * D;
    return Carve::round(size_t(PCA_MEAN_CHUNKS) * D * 8) + Carve::round(size_t(D) * 4) +
           2 * Carve::round(size_t(D_pad) * n_pad * 2) +
           Carve::round(size_t(2) * pca_splits(n_pad) * D_pad * D_pad * 4) + 3 * Carve::round(dd * 8) +
           Carve::round(dd * 4) + 4 * blk + Carve::round(size_t(nch + 1) * PCA_P * PCA_P * 8) +
           Carve::round(size_t((D + PCA_KCHUNK - 1) / PCA_KCHUNK) * D * PCA_P * 4) +
           Carve::round(size_t(PCA_P) * PCA_P * 4) + Carve::round(size_t(PCA_P) * 4) +
           Carve::round(size_t(2) * PCA_P * 8) + Carve::round(64) + 4096;
}

int pca_run(Ctx* c, const float* X, int64_t n, int D, int dim, float* Z, float* comps, float* mu_out,
            double* eig_out, void* scratch, cudaStream_t st) {
    const int64_t n_pad = round_up(n, 64);
    const int D_pad = int(round_up(D, 128));
    const int P = PCA_P;
    const int S = pca_splits(n_pad);
    const int64_t dpp = int64_t(D_pad) * D_pad;
    Carve cv(scratch);
    double* part = cv.take<double>(size_t(PCA_MEAN_CHUNKS) * D);
    float* mu = cv.take<float>(D);
    __nv_bfloat16* hi = cv.take<__nv_bfloat16>(size_t(D_pad) * n_pad);
    __nv_bfloat16* lo = cv.take<__nv_bfloat16>(size_t(D_pad) * n_pad);
    float* gp = cv.take<float>(size_t(2) * S * dpp);
    double* Tacc = cv.take<double>(size_t(D) * D);
    double* Hacc = cv.take<double>(size_t(D) * D);
    double* C64 = cv.take<double>(size_t(D) * D);
    float* C = cv.take<float>(size_t(D) * D);
    float* Xb = cv.take<float>(size_t(D) * P);
    float* Yb = cv.take<float>(size_t(D) * P);
    float* Zb = cv.take<float>(size_t(D) * P);
    float* Wb = cv.take<float>(size_t(D) * P);
    const int nch = (D + PCA_GCHUNK - 1) / PCA_GCHUNK;
    double* Gd = cv.take<double>(size_t(nch) * P * P);
    double* Gsum = cv.take<double>(size_t(P) * P);
    float* cpart = cv.take<float>(size_t((D + PCA_KCHUNK - 1) / PCA_KCHUNK) * D * P);  // splits of C X
    float* Md = cv.take<float>(size_t(P) * P);
    float* thf = cv.take<float>(P);             // Ritz values of the last Rayleigh-Ritz step
    double* rr_out = cv.take<double>(2 * P);    // the same in FP64, then the residual norms^2
    int* dflags = cv.take<int>(16);

    // means and the transposed, split operands
    const int64_t rows_per = (n + PCA_MEAN_CHUNKS - 1) / PCA_MEAN_CHUNKS;
    const int chunks = int((n + rows_per - 1) / rows_per);
    pca_colsum_kernel<<<dim3(chunks, (D + 255) / 256), 256, 0, st>>>(X, n, D, rows_per, part);
    DRGB_CHECK_LAUNCH(c);
    pca_mean_kernel<<<D, 256, 0, st>>>(part, chunks, n, D, mu);
    DRGB_CHECK_LAUNCH(c);
    pca_stage_kernel<<<dim3(unsigned(n_pad / 32), unsigned(D_pad / 32)), dim3(32, 8), 0, st>>>(X, mu, n, D, n_pad,
                                                                                           D_pad, hi, lo);
    DRGB_CHECK_LAUNCH(c);
    // covariance: hi hi^T and hi lo^T, accumulation chains of at most
    // PCA_CHAIN_KB blocks, summed in FP64
    int used_hh = 0, used_hl = 0;
    int rc = tc_gemm_nt_f32(c, hi, hi, D_pad, D_pad, int(n_pad), S, gp, &used_hh, st);
    if (rc) return rc;
    rc = tc_gemm_nt_f32(c, hi, lo, D_pad, D_pad, int(n_pad), S, gp + size_t(S) * dpp, &used_hl, st);
    if (rc) return rc;
    if (used_hh != used_hl) return set_error(c, DRGB_ERR_CUDA, "pca: split mismatch");
    pca_covsum_kernel<<<grid_for(int64_t(D) * D, 256, c->num_sms * 8), 256, 0, st>>>(gp, gp + size_t(S) * dpp,
                                                                                      used_hh, D_pad, D, Tacc, Hacc);
    DRGB_CHECK_LAUNCH(c);
    pca_cov_kernel<<<grid_for(int64_t(D) * D, 256, c->num_sms * 8), 256, 0, st>>>(Tacc, Hacc, D, n, C,
                                                                                  D <= P ? C64 : nullptr);
    DRGB_CHECK_LAUNCH(c);
    DRGB_CUDA(c, cudaMemsetAsync(dflags, 0, 16 * sizeof(int), st));

    std::vector<double> theta(P, 0.0), resid(P, 0.0);
    float* V = Xb;  // the components, D x P (columns >= dim unused)
    if (D <= P) {
        // small D: the whole covariance in one Jacobi CTA
        DRGB_CUDA(c, cudaMemsetAsync(Wb, 0, size_t(D) * P * 4, st));
        pca_jacobi_kernel<<<1, PCA_JAC_THREADS, 0, st>>>(C64, 1, 0, D, 0, D, Wb, P, 0, 0, thf, rr_out);
        DRGB_CHECK_LAUNCH(c);
        std::vector<double> h(D);
        DRGB_CUDA(c, cudaMemcpyAsync(h.data(), rr_out, size_t(D) * 8, cudaMemcpyDeviceToHost, st));
        DRGB_CUDA(c, cudaStreamSynchronize(st));
        for (int k = 0; k < D; ++k) theta[k] = h[k];
        V = Wb;
    } else {
        DRGB_CUDA(c, cudaFuncSetAttribute(pca_chol_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          int(PCA_CHOL_SMEM)));
        const int gblk = grid_for(int64_t(D) * P, 256, c->num_sms * 4);
        int L = 0;  // locked (converged and deflated) leading pairs
        const int nks = (D + PCA_KCHUNK - 1) / PCA_KCHUNK;
        auto cmul = [&](const float* A, const float* Zz, double al, double be, double ga, float* B) -> int {
            pca_cmul_part_kernel<<<dim3((D + PCA_CROWS - 1) / PCA_CROWS, nks), 256, 0, st>>>(C, D, A, cpart);
            DRGB_CHECK_LAUNCH(c);
            pca_cmul_kernel<<<gblk, 256, 0, st>>>(cpart, nks, D, A, Zz, float(al), float(be), float(ga), L, B);
            DRGB_CHECK_LAUNCH(c);
            return DRGB_OK;
        };
        auto gram = [&](const float* A, const float* B) -> int {
            const int m = P - L;
            pca_gram_kernel<<<dim3((P * m + 255) / 256, nch), 256, 0, st>>>(A, B, D, L, Gd);
            DRGB_CHECK_LAUNCH(c);
            pca_gsum_kernel<<<(P * m + 255) / 256, 256, 0, st>>>(Gd, nch, P * m, Gsum);
            DRGB_CHECK_LAUNCH(c);
            return DRGB_OK;
        };
        auto apply = [&](const float* A, float* B) -> int {
            pca_apply_kernel<<<gblk, 256, 0, st>>>(A, D, Md, L, B);
            DRGB_CHECK_LAUNCH(c);
            return DRGB_OK;
        };
        // orthonormalise the active columns against the locked ones and among
        // themselves: Cholesky QR twice, three times after a shifted factor
        auto orth = [&](float*& A, float*& tmp) -> int {
            for (int pass = 0; pass < 3; ++pass) {
                int r = gram(A, A);
                if (r) return r;
                pca_chol_kernel<<<1, PCA_CHOL_THREADS, PCA_CHOL_SMEM, st>>>(Gsum, L, pass, dflags, Md);
                DRGB_CHECK_LAUNCH(c);
                pca_tsolve_kernel<<<(D + 63) / 64, 64, 0, st>>>(A, D, Md, dflags + PCA_MODE, tmp);
                DRGB_CHECK_LAUNCH(c);
                pca_mprod_kernel<<<gblk, 256, 0, st>>>(A, D, Md, dflags + PCA_MODE, tmp);
                DRGB_CHECK_LAUNCH(c);
                std::swap(A, tmp);
            }
            return DRGB_OK;
        };
        // Rayleigh-Ritz on the active columns: X_a <- X_a V, their theta and
        // residual norms |C x - theta x|; the one synchronisation per step
        std::vector<double> hr(2 * P);
        int hflags[2] = {0, 0};
        auto rayleigh_ritz = [&]() -> int {
            const int m = P - L;
            int r = cmul(Xb, nullptr, 1.0, 0.0, 0.0, Zb);
            if (r || (r = gram(Xb, Zb))) return r;
            pca_jacobi_kernel<<<1, PCA_JAC_THREADS, 0, st>>>(Gsum, 1, 0, m, L, m, Md, m, L, 1, thf, rr_out);
            DRGB_CHECK_LAUNCH(c);
            if ((r = apply(Xb, Yb)) || (r = apply(Zb, Wb))) return r;
            pca_resid_kernel<<<(m * 32 + 255) / 256, 256, 0, st>>>(Yb, Wb, thf, D, L, rr_out + P);
            DRGB_CHECK_LAUNCH(c);
            DRGB_CUDA(c, cudaMemcpyAsync(hr.data(), rr_out, size_t(2) * P * 8, cudaMemcpyDeviceToHost, st));
            DRGB_CUDA(c, cudaMemcpyAsync(hflags, dflags, sizeof(hflags), cudaMemcpyDeviceToHost, st));
            DRGB_CUDA(c, cudaStreamSynchronize(st));
            if (hflags[1]) return set_error(c, DRGB_ERR_CUDA, "pca: block lost rank");
            for (int j = 0; j < m; ++j) {
                theta[L + j] = hr[j];
                resid[L + j] = std::sqrt(hr[P + j]);
            }
            std::swap(Xb, Yb);
            return DRGB_OK;
        };
        auto worst = [&]() {
            double w = 0.0;
            for (int k = 0; k < dim; ++k) w = std::fmax(w, resid[k]);
            return w / std::fmax(theta[0], 1e-300);
        };
        pca_start_kernel<<<(D + 127) / 128, 128, 0, st>>>(D, Xb);
        DRGB_CHECK_LAUNCH(c);
        if ((rc = orth(Xb, Yb)) || (rc = rayleigh_ritz())) return rc;
        double best = worst();
        int best_it = 0;
        for (int it = 0; it < PCA_MAXIT && theta[0] > 0.0 && it - best_it < PCA_STALL;) {
            // lock the leading converged pairs and deflate them from C, so
            // that the filter below neither amplifies what is left of them in
            // the active block nor has to span their eigenvalues
            int L1 = L;
            while (L1 < dim && resid[L1] <= PCA_TOL * theta[0]) ++L1;
            if (L1 > L) {
                pca_deflate_kernel<<<dim3((D + 31) / 32, (D + 31) / 32), 256, 0, st>>>(C, D, Xb, thf, L, L1);
                DRGB_CHECK_LAUNCH(c);
                L = L1;
            }
            if (L >= dim) break;
            // Chebyshev filter on the active columns, damping [0, cut] (C is
            // positive semi-definite and the deflated pairs sit near 0) with
            // cut the smallest Ritz value, at least 1e-3 of the largest active
            // one (so that a null space of C, where the filter is +-1, is not
            // squeezed out of the block), scaled to 1 just above the largest
            // active Ritz value; its degree keeps the gain over the damped
            // interval below PCA_GROWTH so that FP32 blocks stay well
            // conditioned.
            const double cut = std::fmax(theta[P - 1], 1e-3 * theta[L]), lo_ = 0.0;
            const double a0 = theta[L] * 1.001;
            const double e = 0.5 * (cut - lo_), cc = 0.5 * (cut + lo_);
            int deg = 1;
            if (e > 0.0)
                while (deg < PCA_DEG && cheb_t(deg + 1, (a0 - cc) / e) <= PCA_GROWTH) ++deg;
            for (int r = 0; r < PCA_RR_EVERY; ++r, ++it) {
                if (e > 0.0) {
                    const double s1 = e / (a0 - cc), tau = 2.0 / s1;
                    double sig = s1;
                    float* prev = Xb;
                    float* cur = Yb;
                    float* nxt = Zb;
                    if ((rc = cmul(Xb, nullptr, s1 / e, -cc * s1 / e, 0.0, cur))) return rc;
                    for (int k = 2; k <= deg; ++k) {
                        const double sn = 1.0 / (tau - sig);
                        if ((rc = cmul(cur, prev, 2.0 * sn / e, -2.0 * cc * sn / e, -sig * sn, nxt))) return rc;
                        sig = sn;
                        float* t = prev;
                        prev = cur;
                        cur = nxt;
                        nxt = t;
                    }
                    Xb = cur;
                    Yb = prev;
                    Zb = nxt;
                } else {  // nothing left above 0: shifted products keep the block's rank
                    if ((rc = cmul(Xb, nullptr, 1.0, 1e-3 * theta[0], 0.0, Yb))) return rc;
                    std::swap(Xb, Yb);
                }
                if ((rc = orth(Xb, Yb))) return rc;
            }
            if ((rc = rayleigh_ritz())) return rc;
            if (worst() < 0.5 * best) {
                best = worst();
                best_it = it;
            }
        }
        V = Xb;
    }
    pca_sign_kernel<<<(dim * 32 + 255) / 256, 256, 0, st>>>(V, D, P, dim);
    DRGB_CHECK_LAUNCH(c);
    pca_project_kernel<<<unsigned((n + 63) / 64), 256, 0, st>>>(X, mu, V, n, D, dim, Z);
    DRGB_CHECK_LAUNCH(c);
    if (comps) {
        pca_components_kernel<<<grid_for(int64_t(D) * dim, 256, c->num_sms * 4), 256, 0, st>>>(V, D, dim, comps);
        DRGB_CHECK_LAUNCH(c);
    }
    if (mu_out) DRGB_CUDA(c, cudaMemcpyAsync(mu_out, mu, size_t(D) * 4, cudaMemcpyDeviceToDevice, st));
    if (eig_out)
        for (int k = 0; k < dim; ++k) eig_out[k] = theta[k];
    return DRGB_OK;
}

}  // namespace drgb

using namespace drgb;

extern "C" int drgb_pca(drgb_ctx* c, const float* X, int64_t n, int32_t D, int32_t dim, float* Z, float* components,
                        float* mean, double* eigvals, void* stream) {
    if (!c) return DRGB_ERR_INVALID;
    if (!X || !Z) return set_error(c, DRGB_ERR_INVALID, "pca: NULL pointer");
    if (!aligned(X, 4) || !aligned(Z, 4) || (components && !aligned(components, 4)) || (mean && !aligned(mean, 4)))
        return set_error(c, DRGB_ERR_INVALID, "pca: misaligned");
    if (D < 1 || D > PCA_MAX_D || dim < 1 || dim > PCA_MAX_DIM || dim > D || n < 2 || round_up(n, 64) > INT32_MAX)
        return set_error(c, DRGB_ERR_INVALID, "pca: need 1 <= dim <= min(D, %d), D <= %d, 2 <= n < 2^31",
                         PCA_MAX_DIM, PCA_MAX_D);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int rc = ensure_scratch(c, pca_scratch_bytes(n, D), st);
    if (rc) return rc;
    rc = pca_run(c, X, n, D, dim, Z, components, mean, eigvals, c->scratch, st);
    if (rc) return rc;
    return drgb_sync(c, stream);
}
