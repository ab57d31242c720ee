// Shared internals of libdrgb: the context, error plumbing, Philox and small
// device helpers.  Not part of the public ABI (see include/drgb.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdarg>
#include <cstdio>
#include <string>

#include "drgb.h"

namespace drgb {

// ------------------------------------------------------------------ context
struct Ctx {
    int device = 0;
    int num_sms = 0;
    size_t l2_bytes = 0;
    size_t smem_per_sm = 0;       // shared memory an SM can give CTAs (bytes)
    void* scratch = nullptr;      // grown on demand, 256-byte aligned carve-outs
    size_t scratch_bytes = 0;
    size_t scratch_limit = 0;     // largest scratch the context may allocate (0 = no limit)
    int* d_status = nullptr;      // device status word (0 = ok, else DRGB_ERR_*)
    unsigned long long* d_counter = nullptr;  // [0] uncertified rows, [4] k-NN tile products computed
    int64_t knn_tiles_total = 0;              // tile products of a full scan (last tensor-core k-NN)
    int64_t launches = 0;         // kernels launched (host-side count)
    int epoch_warps = 8;          // warps per CTA of the epoch force kernel (tuning)
    int epoch_pipe = 1;           // epoch force kernel form: 1 pipelined, 0 flat (tuning)
    std::string device_name;      // for tuning-cache keys
    std::string tuning_cache;     // JSON file of tuned settings ("" = none)
    bool profiling = false;       // record stage events in fit_transform
    cudaEvent_t stage_ev[11] = {};
    int stage_marks = 0;
    // events 6..10 of the tensor-core k-NN recorded in this fit (bit idx - 6):
    // 8 its start, 6 and 7 around the GEMM kernel, 9 after the re-rank, 10
    // after the re-scan of uncertified rows
    unsigned knn_marks = 0;
    // The executable graph of the last epoch loop, refreshed in place
    // (cudaGraphExecUpdate) when the next loop has the same shape.
    cudaGraphExec_t epoch_exec = nullptr;
    std::string err;
};

// Record stage boundary `idx` on `st` when profiling is enabled.
int stage_mark(Ctx* c, int idx, cudaStream_t st);

// Force-kernel widths (warps per CTA) the epoch kernel supports.
bool epoch_warps_supported(int warps);

// Tuning-cache key of a problem on this context's device: device name, SM
// count, and the powers of two below the row and instance counts, and k.
std::string tuning_key(const Ctx* c, int64_t rows, int64_t instances, int k);

// Record a formatted error message in the context; returns `code`.
int set_error(Ctx* c, int code, const char* fmt, ...);

// Check a CUDA runtime call; on failure record it and return DRGB_ERR_CUDA.
#define DRGB_CUDA(ctx, call)                                                          \
    do {                                                                              \
        cudaError_t e_ = (call);                                                      \
        if (e_ != cudaSuccess)                                                        \
            return ::drgb::set_error((ctx), DRGB_ERR_CUDA, "%s failed: %s (%s:%d)",   \
                                     #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
    } while (0)

#define DRGB_CHECK_LAUNCH(ctx)              \
    do {                                     \
        ++(ctx)->launches;                   \
        DRGB_CUDA(ctx, cudaGetLastError());  \
    } while (0)

// Ensure the context holds at least `bytes` of scratch.  Growing synchronises
// `stream` first, so that work still using the old buffer has finished.
int ensure_scratch(Ctx* c, size_t bytes, cudaStream_t stream);

// Bump allocator over the scratch buffer (256-byte aligned slices).
struct Carve {
    char* base;
    size_t off = 0;
    explicit Carve(void* b) : base(static_cast<char*>(b)) {}
    template <class T>
    T* take(size_t count) {
        off = (off + 255) & ~size_t(255);
        T* p = reinterpret_cast<T*>(base + off);
        off += count * sizeof(T);
        return p;
    }
    static size_t round(size_t bytes) { return (bytes + 255) & ~size_t(255); }
};

inline bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

// ------------------------------------------------------------------ device status
__device__ __forceinline__ void report_status(int* status, int code) {
    atomicCAS(status, 0, code);
}

// ------------------------------------------------------------------ Philox4x32-10
// Salmon et al., SC'11: four 32-bit counter words pass through 10 rounds of two
// multiply-high/low S-boxes and a word permutation; the two key words are
// bumped by the Weyl constants between rounds.
struct U4 {
    uint32_t x, y, z, w;
};

__host__ __device__ __forceinline__ U4 philox4x32_10(U4 c, uint32_t k0, uint32_t k1) {
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) {
            k0 += W0;
            k1 += W1;
        }
#ifdef __CUDA_ARCH__
        const uint32_t hi0 = __umulhi(M0, c.x), lo0 = M0 * c.x;
        const uint32_t hi1 = __umulhi(M1, c.z), lo1 = M1 * c.z;
#else
        const uint64_t p0 = uint64_t(M0) * c.x, p1 = uint64_t(M1) * c.z;
        const uint32_t hi0 = uint32_t(p0 >> 32), lo0 = uint32_t(p0);
        const uint32_t hi1 = uint32_t(p1 >> 32), lo1 = uint32_t(p1);
#endif
        c = U4{hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0};
    }
    return c;
}

// The same generator with its ten round keys given: rk[2r], rk[2r + 1] are the
// key words of round r (k0 + r W0, k1 + r W1).  A kernel whose key is the same
// for every thread takes them from its parameters, which saves the key bumps.
__device__ __forceinline__ U4 philox4x32_10_rk(U4 c, const uint32_t* rk) {
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint64_t p0 = uint64_t(M0) * c.x, p1 = uint64_t(M1) * c.z;
        c = U4{uint32_t(p1 >> 32) ^ c.y ^ rk[2 * r], uint32_t(p1), uint32_t(p0 >> 32) ^ c.w ^ rk[2 * r + 1],
               uint32_t(p0)};
    }
    return c;
}

inline void philox_round_keys(uint32_t k0, uint32_t k1, uint32_t* rk) {
    for (int r = 0; r < 10; ++r) {
        rk[2 * r] = k0 + uint32_t(r) * 0x9E3779B9u;
        rk[2 * r + 1] = k1 + uint32_t(r) * 0xBB67AE85u;
    }
}

enum : uint32_t { TAG_NEGATIVE = 0u, TAG_INIT = 1u, TAG_MLP = 2u, TAG_SPECTRAL = 3u };

// floor(u * n / 2^32): maps a uniform 32-bit word onto [0, n).
__device__ __forceinline__ int64_t mulshift_index(uint32_t u, int64_t n) {
    return int64_t((uint64_t(u) * uint64_t(n)) >> 32);
}

// ------------------------------------------------------------------ launch helpers
inline int grid_for(int64_t work, int per_block, int max_blocks) {
    int64_t g = (work + per_block - 1) / per_block;
    if (g < 1) g = 1;
    if (g > max_blocks) g = max_blocks;
    return int(g);
}

// Exclusive prefix sum of `n` int32 counts into `out` (n + 1 entries, out[n] =
// total), on `stream`, using `tmp` scratch of scan_scratch_elems(n) ints.
size_t scan_scratch_elems(int64_t n);
int exclusive_scan(Ctx* c, const int32_t* in, int32_t* out, int64_t n, int32_t* tmp,
                   cudaStream_t stream);

}  // namespace drgb

struct drgb_ctx : public drgb::Ctx {};
