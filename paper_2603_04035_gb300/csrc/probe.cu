// Random-gather probe (no counterpart in the paper; a roofline denominator):
// the rate at which this GPU serves independent random 8-byte loads from an
// array of n float2 values, the access the SGD epoch makes for every tail and
// every negative sample.  Every resident thread (the largest L1 carveout, the
// most warps an SM holds) draws indices from a multiplicative congruential
// stream, maps them onto [0, n) by multiply-shift, and sums the values it
// loads (the sums are stored so that no load is dropped).  For an array that
// fits in L2 the rate is bounded by the SMs' L1/L2 sector throughput and
// latency, not by HBM bandwidth.
#include "common.cuh"

namespace drgb {

static constexpr int PROBE_THREADS = 256;
static constexpr int PROBE_STREAMS = 8;  // independent index streams per thread

__global__ void __launch_bounds__(PROBE_THREADS) gather_probe_kernel(const float2* __restrict__ Y, uint32_t n,
                                                                     int rounds, uint32_t seed,
                                                                     float2* __restrict__ sink) {
    const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t x[PROBE_STREAMS];
#pragma unroll
    for (int s = 0; s < PROBE_STREAMS; ++s) x[s] = (tid * PROBE_STREAMS + s) * 2654435761u + seed * 40503u + 1u;
    float ax = 0.f, ay = 0.f;
    for (int r = 0; r < rounds; ++r) {
#pragma unroll
        for (int s = 0; s < PROBE_STREAMS; ++s) {
            x[s] = x[s] * 1664525u + 1013904223u;
            const float2 v = Y[(uint64_t(x[s]) * n) >> 32];
            ax += v.x;
            ay += v.y;
        }
    }
    sink[tid] = make_float2(ax, ay);
}

}  // namespace drgb

using namespace drgb;

extern "C" int drgb_gather_probe(drgb_ctx* c, const float* Y, int64_t n, int32_t rounds, uint32_t seed,
                                 double* gathers_per_s, void* stream) {
    if (!c) return DRGB_ERR_INVALID;
    if (!Y || !gathers_per_s || !aligned(Y, 8) || n < 1 || n > int64_t(UINT32_MAX) || rounds < 1 ||
        rounds > 4096)
        return set_error(c, DRGB_ERR_INVALID, "gather_probe: bad arguments");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    DRGB_CUDA(c, cudaFuncSetAttribute(gather_probe_kernel, cudaFuncAttributePreferredSharedMemoryCarveout, 0));
    int per_sm = 0;
    DRGB_CUDA(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, gather_probe_kernel, PROBE_THREADS, 0));
    const int blocks = c->num_sms * (per_sm > 0 ? per_sm : 1);
    const int64_t threads = int64_t(blocks) * PROBE_THREADS;
    int rc = ensure_scratch(c, Carve::round(size_t(threads) * 8), st);
    if (rc) return rc;
    float2* sink = static_cast<float2*>(c->scratch);
    const float2* Y2 = reinterpret_cast<const float2*>(Y);
    gather_probe_kernel<<<blocks, PROBE_THREADS, 0, st>>>(Y2, uint32_t(n), rounds, seed, sink);  // warm-up
    DRGB_CHECK_LAUNCH(c);
    cudaEvent_t e0, e1;
    DRGB_CUDA(c, cudaEventCreate(&e0));
    DRGB_CUDA(c, cudaEventCreate(&e1));
    DRGB_CUDA(c, cudaEventRecord(e0, st));
    gather_probe_kernel<<<blocks, PROBE_THREADS, 0, st>>>(Y2, uint32_t(n), rounds, seed + 1, sink);
    DRGB_CHECK_LAUNCH(c);
    DRGB_CUDA(c, cudaEventRecord(e1, st));
    DRGB_CUDA(c, cudaEventSynchronize(e1));
    float ms = 0.f;
    DRGB_CUDA(c, cudaEventElapsedTime(&ms, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *gathers_per_s = double(threads) * rounds * PROBE_STREAMS / (double(ms) * 1e-3);
    return drgb_sync(c, stream);
}
