// Spectral initial layout: the two leading non-trivial eigenvectors of the
// normalised fuzzy-graph adjacency M = D^-1/2 W D^-1/2 (the smallest of the
// normalised graph Laplacian I - M), scaled to the initialisation range.  The
// UMAP optimisation the paper times (Section 3) starts from this layout.
//
// Eigen-solver: Chebyshev-filtered subspace iteration (Zhou & Saad 2007) on a
// block of P = 8 vectors, in FP32 on the device, with the small dense steps
// (Cholesky factors, the P x P Rayleigh-Ritz eigenproblem) in FP64 on the
// host.  One iteration:
//   Y  = p_m(M) X        degree-m Chebyshev polynomial that damps [-1, cut]
//                        and keeps the eigenvalues above cut, scaled so that
//                        the top one stays O(1)
//   X  = Y R^-1          Cholesky QR, twice (Y^T Y = R^T R)
//   H  = X^T M X         Rayleigh-Ritz: H = V diag(theta) V^T, X <- X V
// until the residuals |M x_k - theta_k x_k| of the three leading Ritz pairs
// fall below SPEC_TOL, for at most SPEC_MAXIT steps, or until the worst of
// them has not halved in SPEC_STALL steps; cut is the smallest Ritz value of
// the block.  A vector's angle to its eigenvector is then about
// SPEC_TOL / (gap to the neighbouring eigenvalues).
// The layout takes Ritz vectors 1 and 2 (vector 0 is D^1/2 1, eigenvalue 1),
// each with the sign that makes its largest-magnitude entry positive.
//
// Layout of the block vectors: n x P row-major FP32 (one 32-byte row per
// point, so one gather of a neighbour's row is one sector).
#include <cmath>
#include <vector>

#include "common.cuh"
#include "spectral.cuh"

namespace drgb {

static constexpr int SP = 8;          // block size
static constexpr int SPEC_DEG = 12;   // Chebyshev degree per iteration
static constexpr int SPEC_MAXIT = 400;
static constexpr int SPEC_STALL = 40;
static constexpr double SPEC_TOL = 1e-5;
static constexpr float SPEC_JITTER = 1e-5f;
static constexpr int GRAM_BLOCKS_PER_SM = 2;

struct Mat8 {
    float v[SP * SP];  // row-major P x P
};

// d_i = sum of row i's weights (in entry order), s_i = 1 / sqrt(d_i) (0 for
// an empty row).
__global__ void spec_degree_kernel(const int32_t* __restrict__ rp, const float* __restrict__ w, int64_t n,
                                   float* __restrict__ s) {
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
        float d = 0.f;
        for (int32_t e = rp[i]; e < rp[i + 1]; ++e) d += w[e];
        s[i] = d > 0.f ? 1.0f / sqrtf(d) : 0.f;
    }
}

// m_e = s_i w_e s_j: the entries of M in the CSR's order.
__global__ void spec_entries_kernel(const int32_t* __restrict__ rp, const int32_t* __restrict__ col,
                                    const float* __restrict__ w, const float* __restrict__ s, int64_t n,
                                    float* __restrict__ m) {
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
        const float si = s[i];
        for (int32_t e = rp[i]; e < rp[i + 1]; ++e) m[e] = si * w[e] * s[col[e]];
    }
}

// Y = alpha (M X) + beta X + gamma Z (Z may be null when gamma = 0); eight
// threads per row, one per block column.
__global__ void spec_spmm_kernel(const int32_t* __restrict__ rp, const int32_t* __restrict__ col,
                                 const float* __restrict__ m, int64_t n, const float* __restrict__ X,
                                 const float* __restrict__ Z, float alpha, float beta, float gamma,
                                 float* __restrict__ Y) {
    const int64_t total = n * SP;
    for (int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < total; t += int64_t(gridDim.x) * blockDim.x) {
        const int64_t i = t / SP;
        const int c = int(t - i * SP);
        float acc = 0.f;
        for (int32_t e = rp[i]; e < rp[i + 1]; ++e) acc = fmaf(m[e], X[int64_t(col[e]) * SP + c], acc);
        float y = alpha * acc + beta * X[t];
        if (Z) y = fmaf(gamma, Z[t], y);
        Y[t] = y;
    }
}

// Per-block partial sums of A^T B (P x P), FP32 within the block.
__global__ void spec_gram_kernel(const float* __restrict__ A, const float* __restrict__ B, int64_t n,
                                 float* __restrict__ partial) {
    float acc[SP * SP];
#pragma unroll
    for (int q = 0; q < SP * SP; ++q) acc[q] = 0.f;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
        float a[SP], b[SP];
#pragma unroll
        for (int c = 0; c < SP; ++c) {
            a[c] = A[i * SP + c];
            b[c] = B[i * SP + c];
        }
#pragma unroll
        for (int r = 0; r < SP; ++r)
#pragma unroll
            for (int c = 0; c < SP; ++c) acc[r * SP + c] = fmaf(a[r], b[c], acc[r * SP + c]);
    }
    __shared__ float s_red[32][SP * SP + 1];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < SP * SP; ++q) {
        float v = acc[q];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) s_red[warp][q] = v;
    }
    __syncthreads();
    if (threadIdx.x < SP * SP) {
        float v = 0.f;
        for (int u = 0; u < int(blockDim.x >> 5); ++u) v += s_red[u][threadIdx.x];
        partial[int64_t(blockIdx.x) * SP * SP + threadIdx.x] = v;
    }
}

// Y = X C (C: P x P in the parameters).
__global__ void spec_apply_kernel(const float* __restrict__ X, int64_t n, const Mat8 C, float* __restrict__ Y) {
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
        float x[SP];
#pragma unroll
        for (int c = 0; c < SP; ++c) x[c] = X[i * SP + c];
#pragma unroll
        for (int c = 0; c < SP; ++c) {
            float y = 0.f;
#pragma unroll
            for (int r = 0; r < SP; ++r) y = fmaf(x[r], C.v[r * SP + c], y);
            Y[i * SP + c] = y;
        }
    }
}

// Starting block: uniform values in [-1, 1) from Philox words at counter
// (i, c / 4, 0, 3) under the given key.
__global__ void spec_start_kernel(int64_t n, uint32_t k0, uint32_t k1, float* __restrict__ X) {
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
#pragma unroll
        for (int g = 0; g < SP / 4; ++g) {
            const U4 r = philox4x32_10(U4{uint32_t(i), uint32_t(g), 0u, TAG_SPECTRAL}, k0, k1);
            const uint32_t u[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
            for (int q = 0; q < 4; ++q)
                X[i * SP + 4 * g + q] = fmaf(float(u[q] >> 8), 2.0f * 5.9604644775390625e-08f, -1.0f);
        }
    }
}

// Per block: the largest |X[i][c]| of columns 1 and 2, with the lowest index
// among equal magnitudes (value bits << 32 | ~index, taken as a maximum).
__global__ void spec_argmax_kernel(const float* __restrict__ X, int64_t n, unsigned long long* __restrict__ best) {
    unsigned long long b1 = 0ull, b2 = 0ull;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
        const unsigned long long k1 = (uint64_t(__float_as_uint(fabsf(X[i * SP + 1]))) << 32) | (~uint32_t(i));
        const unsigned long long k2 = (uint64_t(__float_as_uint(fabsf(X[i * SP + 2]))) << 32) | (~uint32_t(i));
        b1 = k1 > b1 ? k1 : b1;
        b2 = k2 > b2 ? k2 : b2;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long o1 = __shfl_xor_sync(0xffffffffu, b1, o), o2 = __shfl_xor_sync(0xffffffffu, b2, o);
        b1 = o1 > b1 ? o1 : b1;
        b2 = o2 > b2 ? o2 : b2;
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMax(&best[0], b1);
        atomicMax(&best[1], b2);
    }
}

// Y0[i] = R (g1 X[i][1], g2 X[i][2]) + R * jitter * (2u - 1), u from words 2
// and 3 of the initialisation stream (counter (i, 0, 0, 1), key seed).
__global__ void spec_layout_kernel(const float* __restrict__ X, int64_t n, float g1, float g2, float range,
                                   uint32_t k0, uint32_t k1, float2* __restrict__ Y) {
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
        const U4 r = philox4x32_10(U4{uint32_t(i), 0u, 0u, TAG_INIT}, k0, k1);
        const float s = 5.9604644775390625e-08f;  // 2^-24
        const float jx = fmaf(float(r.z >> 8), 2.0f * s, -1.0f), jy = fmaf(float(r.w >> 8), 2.0f * s, -1.0f);
        const float rj = range * SPEC_JITTER;
        Y[i] = make_float2(fmaf(rj, jx, range * (g1 * X[i * SP + 1])), fmaf(rj, jy, range * (g2 * X[i * SP + 2])));
    }
}

// ------------------------------------------------------------------ host linear algebra (P x P, FP64)
// Upper Cholesky factor R of a symmetric positive definite G (G = R^T R);
// false if G is not numerically positive definite.
static bool cholesky_upper(const double* G, double* R) {
    for (int q = 0; q < SP * SP; ++q) R[q] = 0.0;
    for (int j = 0; j < SP; ++j) {
        double d = G[j * SP + j];
        for (int k = 0; k < j; ++k) d -= R[k * SP + j] * R[k * SP + j];
        if (!(d > 1e-300)) return false;
        R[j * SP + j] = std::sqrt(d);
        for (int i = j + 1; i < SP; ++i) {
            double v = G[j * SP + i];
            for (int k = 0; k < j; ++k) v -= R[k * SP + j] * R[k * SP + i];
            R[j * SP + i] = v / R[j * SP + j];
        }
    }
    return true;
}

// Inverse of an upper-triangular R.
static void invert_upper(const double* R, double* Ri) {
    for (int q = 0; q < SP * SP; ++q) Ri[q] = 0.0;
    for (int j = 0; j < SP; ++j) {
        Ri[j * SP + j] = 1.0 / R[j * SP + j];
        for (int i = j - 1; i >= 0; --i) {
            double v = 0.0;
            for (int k = i + 1; k <= j; ++k) v += R[i * SP + k] * Ri[k * SP + j];
            Ri[i * SP + j] = -v / R[i * SP + i];
        }
    }
}

// Cyclic Jacobi eigen-decomposition of a symmetric H: H = V diag(e) V^T,
// eigenvalues in decreasing order, columns of V the eigenvectors.
static void jacobi_eigen(const double* H, double* e, double* V) {
    double A[SP * SP];
    for (int q = 0; q < SP * SP; ++q) {
        A[q] = H[q];
        V[q] = (q / SP == q % SP) ? 1.0 : 0.0;
    }
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0;
        for (int p = 0; p < SP; ++p)
            for (int q = p + 1; q < SP; ++q) off += A[p * SP + q] * A[p * SP + q];
        if (off < 1e-30) break;
        for (int p = 0; p < SP; ++p) {
            for (int q = p + 1; q < SP; ++q) {
                const double apq = A[p * SP + q];
                if (std::fabs(apq) < 1e-300) continue;
                const double theta = (A[q * SP + q] - A[p * SP + p]) / (2.0 * apq);
                const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
                const double cs = 1.0 / std::sqrt(t * t + 1.0), sn = t * cs;
                for (int k = 0; k < SP; ++k) {  // A <- J^T A J
                    const double akp = A[k * SP + p], akq = A[k * SP + q];
                    A[k * SP + p] = cs * akp - sn * akq;
                    A[k * SP + q] = sn * akp + cs * akq;
                }
                for (int k = 0; k < SP; ++k) {
                    const double apk = A[p * SP + k], aqk = A[q * SP + k];
                    A[p * SP + k] = cs * apk - sn * aqk;
                    A[q * SP + k] = sn * apk + cs * aqk;
                }
                for (int k = 0; k < SP; ++k) {
                    const double vkp = V[k * SP + p], vkq = V[k * SP + q];
                    V[k * SP + p] = cs * vkp - sn * vkq;
                    V[k * SP + q] = sn * vkp + cs * vkq;
                }
            }
        }
    }
    int order[SP];
    for (int i = 0; i < SP; ++i) order[i] = i;
    for (int i = 0; i < SP; ++i)  // decreasing eigenvalues (stable)
        for (int j = i + 1; j < SP; ++j)
            if (A[order[j] * SP + order[j]] > A[order[i] * SP + order[i]]) {
                const int tmp = order[i];
                order[i] = order[j];
                order[j] = tmp;
            }
    double W[SP * SP];
    for (int c = 0; c < SP; ++c) {
        e[c] = A[order[c] * SP + order[c]];
        for (int r = 0; r < SP; ++r) W[r * SP + c] = V[r * SP + order[c]];
    }
    for (int q = 0; q < SP * SP; ++q) V[q] = W[q];
}

static Mat8 to_mat(const double* D) {
    Mat8 m;
    for (int q = 0; q < SP * SP; ++q) m.v[q] = float(D[q]);
    return m;
}

size_t spectral_scratch_bytes(int64_t n, int64_t nnz_cap, int num_sms) {
    const size_t blk = Carve::round(size_t(n) * SP * 4);
    return Carve::round(size_t(nnz_cap > 0 ? nnz_cap : 1) * 4) + Carve::round(size_t(n) * 4) + 3 * blk +
           Carve::round(size_t(num_sms) * GRAM_BLOCKS_PER_SM * SP * SP * 4) + Carve::round(16) + 1024;
}

int spectral_layout(Ctx* c, const int32_t* rp, const int32_t* col, const float* w, int64_t n, int64_t nnz_cap,
                    float init_range, uint64_t seed, float2* Y, double* eig_out, void* scratch, cudaStream_t st) {
    Carve cv(scratch);
    float* m = cv.take<float>(size_t(nnz_cap > 0 ? nnz_cap : 1));
    float* s = cv.take<float>(n);
    float* X = cv.take<float>(size_t(n) * SP);
    float* Yb = cv.take<float>(size_t(n) * SP);
    float* Zb = cv.take<float>(size_t(n) * SP);
    const int gb = c->num_sms * GRAM_BLOCKS_PER_SM;
    float* partial = cv.take<float>(size_t(gb) * SP * SP);
    unsigned long long* best = cv.take<unsigned long long>(2);
    const int g1 = grid_for(n, 256, c->num_sms * 8);
    const int gspmm = grid_for(n * SP, 256, c->num_sms * 16);

    spec_degree_kernel<<<g1, 256, 0, st>>>(rp, w, n, s);
    DRGB_CHECK_LAUNCH(c);
    spec_entries_kernel<<<g1, 256, 0, st>>>(rp, col, w, s, n, m);
    DRGB_CHECK_LAUNCH(c);
    spec_start_kernel<<<g1, 256, 0, st>>>(n, uint32_t(seed), uint32_t(seed >> 32), X);
    DRGB_CHECK_LAUNCH(c);

    std::vector<float> hp(size_t(gb) * SP * SP);
    // G = A^T B summed in FP64 (synchronous)
    auto gram = [&](const float* A, const float* B, double* G) -> int {
        spec_gram_kernel<<<gb, 256, 0, st>>>(A, B, n, partial);
        DRGB_CHECK_LAUNCH(c);
        DRGB_CUDA(c, cudaMemcpyAsync(hp.data(), partial, hp.size() * 4, cudaMemcpyDeviceToHost, st));
        DRGB_CUDA(c, cudaStreamSynchronize(st));
        for (int q = 0; q < SP * SP; ++q) {
            double v = 0.0;
            for (int b = 0; b < gb; ++b) v += double(hp[size_t(b) * SP * SP + q]);
            G[q] = v;
        }
        return DRGB_OK;
    };
    auto apply = [&](const float* A, const double* C, float* B) -> int {
        spec_apply_kernel<<<g1, 256, 0, st>>>(A, n, to_mat(C), B);
        DRGB_CHECK_LAUNCH(c);
        return DRGB_OK;
    };
    auto spmm = [&](const float* A, const float* Z, float alpha, float beta, float gamma, float* B) -> int {
        spec_spmm_kernel<<<gspmm, 256, 0, st>>>(rp, col, m, n, A, Z, alpha, beta, gamma, B);
        DRGB_CHECK_LAUNCH(c);
        return DRGB_OK;
    };
    // X <- X R^-1 twice (Cholesky QR); `tmp` is scratch
    auto orthonormalise = [&](float*& A, float*& tmp) -> int {
        for (int pass = 0; pass < 2; ++pass) {
            double G[SP * SP], R[SP * SP], Ri[SP * SP];
            int rc = gram(A, A, G);
            if (rc) return rc;
            for (int r = 0; r < SP; ++r)  // symmetrise
                for (int q = r + 1; q < SP; ++q) G[r * SP + q] = G[q * SP + r] = 0.5 * (G[r * SP + q] + G[q * SP + r]);
            if (!cholesky_upper(G, R)) return set_error(c, DRGB_ERR_CUDA, "spectral_init: block lost rank");
            invert_upper(R, Ri);
            if ((rc = apply(A, Ri, tmp))) return rc;
            float* t = A;
            A = tmp;
            tmp = t;
        }
        return DRGB_OK;
    };
    int rc = orthonormalise(X, Yb);
    if (rc) return rc;
    double theta[SP] = {0}, resid[3] = {1, 1, 1};
    // Rayleigh-Ritz: X <- X V, theta = Ritz values (decreasing), and the
    // residuals of the three leading pairs
    auto rayleigh_ritz = [&]() -> int {
        double H[SP * SP], V[SP * SP];
        int rc2 = spmm(X, nullptr, 1.f, 0.f, 0.f, Zb);
        if (rc2) return rc2;
        if ((rc2 = gram(X, Zb, H))) return rc2;
        for (int r = 0; r < SP; ++r)
            for (int q = r + 1; q < SP; ++q) H[r * SP + q] = H[q * SP + r] = 0.5 * (H[r * SP + q] + H[q * SP + r]);
        jacobi_eigen(H, theta, V);
        if ((rc2 = apply(X, V, Yb))) return rc2;
        std::swap(X, Yb);
        // residuals of the three leading pairs: |M x_k - theta_k x_k|
        double Dm[SP * SP];
        for (int q = 0; q < SP * SP; ++q) Dm[q] = (q / SP == q % SP) ? -theta[q % SP] : 0.0;
        if ((rc2 = apply(X, Dm, Zb))) return rc2;                            // -X diag(theta)
        if ((rc2 = spmm(X, Zb, 1.f, 0.f, 1.f, Yb))) return rc2;             // M X - X diag(theta)
        double R2[SP * SP];
        if ((rc2 = gram(Yb, Yb, R2))) return rc2;
        for (int k = 0; k < 3; ++k) resid[k] = std::sqrt(std::fmax(R2[k * SP + k], 0.0));
        return DRGB_OK;
    };
    if ((rc = rayleigh_ritz())) return rc;
    int it = 0;
    double best_res = std::fmax(resid[0], std::fmax(resid[1], resid[2]));
    int best_it = 0;
    for (; it < SPEC_MAXIT && std::fmax(resid[0], std::fmax(resid[1], resid[2])) > SPEC_TOL; ++it) {
        // stagnation: the worst residual has not halved in SPEC_STALL steps,
        // so the leading eigenvalues are too close to separate in FP32 (a
        // nearly disconnected graph); any combination of their eigenvectors
        // serves as the layout
        if (it - best_it >= SPEC_STALL) break;
        // Chebyshev filter damping [a, b] = [-1, cut], scaled at a0 = 1 (the
        // top eigenvalue of M)
        double cut = theta[SP - 1];
        if (!(cut < theta[2] - 1e-7)) cut = theta[2] - 1e-7;
        const double a = -1.0, b = cut, a0 = 1.0;
        const double e = 0.5 * (b - a), cc = 0.5 * (b + a);
        const double s1 = e / (a0 - cc), tau = 2.0 / s1;
        double sig = s1;
        // Y1 = (s1/e)(M X - cc X); then Y_{k+1} = (2 s'/e)(M Y_k - cc Y_k) - s s' Y_{k-1}
        float* prev = X;
        float* cur = Yb;
        float* nxt = Zb;
        if ((rc = spmm(X, nullptr, float(s1 / e), float(-cc * s1 / e), 0.f, cur))) return rc;
        for (int k = 2; k <= SPEC_DEG; ++k) {
            const double sn = 1.0 / (tau - sig);
            if ((rc = spmm(cur, prev, float(2.0 * sn / e), float(-2.0 * cc * sn / e), float(-sig * sn), nxt)))
                return rc;
            sig = sn;
            float* t = prev;
            prev = cur;
            cur = nxt;
            nxt = t;
        }
        // cur holds the filtered block: it becomes X (prev, cur and nxt are
        // the three buffers X, Yb, Zb in some order)
        X = cur;
        Yb = prev;
        Zb = nxt;
        if ((rc = orthonormalise(X, Yb))) return rc;
        if ((rc = rayleigh_ritz())) return rc;
        const double worst = std::fmax(resid[0], std::fmax(resid[1], resid[2]));
        if (worst < 0.5 * best_res) {
            best_res = worst;
            best_it = it + 1;
        }
    }
    // (after SPEC_MAXIT steps the current Ritz vectors are taken as they are:
    // a slow finish means nearly equal eigenvalues, whose eigenvectors any
    // combination approximates)
    // sign of each layout column: its largest-magnitude entry positive
    DRGB_CUDA(c, cudaMemsetAsync(best, 0, 16, st));
    spec_argmax_kernel<<<g1, 256, 0, st>>>(X, n, best);
    DRGB_CHECK_LAUNCH(c);
    unsigned long long hb[2];
    float hv[2];
    DRGB_CUDA(c, cudaMemcpyAsync(hb, best, 16, cudaMemcpyDeviceToHost, st));
    DRGB_CUDA(c, cudaStreamSynchronize(st));
    for (int k = 0; k < 2; ++k) {
        const int64_t i = int64_t(~uint32_t(hb[k] & 0xffffffffu));
        DRGB_CUDA(c, cudaMemcpy(&hv[k], X + i * SP + 1 + k, 4, cudaMemcpyDeviceToHost));
    }
    const float vmax = fmaxf(fabsf(hv[0]), fabsf(hv[1]));
    if (!(vmax > 0.f)) return set_error(c, DRGB_ERR_CUDA, "spectral_init: zero layout");
    const float g1s = (hv[0] < 0.f ? -1.0f : 1.0f) / vmax, g2s = (hv[1] < 0.f ? -1.0f : 1.0f) / vmax;
    spec_layout_kernel<<<g1, 256, 0, st>>>(X, n, g1s, g2s, init_range, uint32_t(seed), uint32_t(seed >> 32), Y);
    DRGB_CHECK_LAUNCH(c);
    if (eig_out)
        for (int k = 0; k < 3; ++k) eig_out[k] = theta[k];
    return DRGB_OK;
}

}  // namespace drgb

using namespace drgb;

extern "C" int drgb_spectral_init(drgb_ctx* c, const int32_t* row_ptr, const int32_t* col, const float* w,
                                  int64_t n, float init_range, uint64_t seed, float* Y_out, double* eigvals,
                                  void* stream) {
    if (!c) return DRGB_ERR_INVALID;
    if (!row_ptr || !col || !w || !Y_out) return set_error(c, DRGB_ERR_INVALID, "spectral_init: NULL pointer");
    if (n < SP + 1 || n > INT32_MAX || !(init_range > 0.f) || !aligned(Y_out, 8) || !aligned(row_ptr, 4) ||
        !aligned(col, 4) || !aligned(w, 4))
        return set_error(c, DRGB_ERR_INVALID, "spectral_init: bad arguments (n must exceed %d)", SP);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int32_t nnz = 0;
    DRGB_CUDA(c, cudaMemcpyAsync(&nnz, row_ptr + n, 4, cudaMemcpyDeviceToHost, st));
    DRGB_CUDA(c, cudaStreamSynchronize(st));
    if (nnz < 0) return set_error(c, DRGB_ERR_INVALID, "spectral_init: row_ptr[n] < 0");
    int rc = ensure_scratch(c, spectral_scratch_bytes(n, nnz, c->num_sms), st);
    if (rc) return rc;
    rc = spectral_layout(c, row_ptr, col, w, n, nnz, init_range, seed, reinterpret_cast<float2*>(Y_out), eigvals,
                         c->scratch, st);
    if (rc) return rc;
    return drgb_sync(c, stream);
}
