// Circle-splatting renderer of an embedding (Section 2.4, the GPU rendering
// pipeline): every point is splatted as a disc of radius R with the linear
// falloff w = max(0, 1 - r / R) at each pixel centre, its premultiplied
// colour added into an RGBA accumulator by atomic scatter-add, and a resolve
// pass divides colour by alpha and composites over the background into an
// 8-bit RGB frame.  Headless: the frame is a device buffer.
//
// Pixel space: px = (x - x0) s, py = (y - y0) s; pixel (u, v) (column u, row
// v, row v growing with y) has its centre at (u + 1/2, v + 1/2).  The view
// (x0, y0, s) is the caller's, or fitted to the points' bounding box with a
// 5% margin on each side, the larger extent filling the frame, centred.
//
// Layout: accumulator H x W float4 (C_r, C_g, C_b, A) in the context's
// scratch; frame H x W x 3 uint8 (row-major, row 0 first) in the caller's
// memory.  The scatter-add order is not fixed, so a pixel's sums may differ
// between runs by FP32 rounding.
#include "common.cuh"

namespace drgb {

static constexpr float RENDER_MARGIN = 0.05f;

// Order-preserving map of a float to an unsigned int (for atomic min/max).
__device__ __forceinline__ unsigned int float_key(float f) {
    const unsigned int b = __float_as_uint(f);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float key_float(unsigned int k) {
    return __uint_as_float((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k);
}

// keys[0..3] = min x, min y, max x, max y (order-preserving keys).
__global__ void render_bbox_kernel(const float2* __restrict__ Y, int64_t n, unsigned int* __restrict__ keys) {
    float mnx = INFINITY, mny = INFINITY, mxx = -INFINITY, mxy = -INFINITY;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
        const float2 y = Y[i];
        mnx = fminf(mnx, y.x);
        mny = fminf(mny, y.y);
        mxx = fmaxf(mxx, y.x);
        mxy = fmaxf(mxy, y.y);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        mnx = fminf(mnx, __shfl_xor_sync(0xffffffffu, mnx, o));
        mny = fminf(mny, __shfl_xor_sync(0xffffffffu, mny, o));
        mxx = fmaxf(mxx, __shfl_xor_sync(0xffffffffu, mxx, o));
        mxy = fmaxf(mxy, __shfl_xor_sync(0xffffffffu, mxy, o));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMin(&keys[0], float_key(mnx));
        atomicMin(&keys[1], float_key(mny));
        atomicMax(&keys[2], float_key(mxx));
        atomicMax(&keys[3], float_key(mxy));
    }
}

// view[0..2] = (x0, y0, s) from the bounding box (one thread).
__global__ void render_view_kernel(const unsigned int* __restrict__ keys, int width, int height,
                                   float* __restrict__ view) {
    const float lox = key_float(keys[0]), loy = key_float(keys[1]), hix = key_float(keys[2]),
                hiy = key_float(keys[3]);
    const float ex = fmaxf(hix - lox, 1e-12f) * (1.0f + 2.0f * RENDER_MARGIN);
    const float ey = fmaxf(hiy - loy, 1e-12f) * (1.0f + 2.0f * RENDER_MARGIN);
    const float s = fminf(float(width) / ex, float(height) / ey);
    const float cx = 0.5f * (lox + hix), cy = 0.5f * (loy + hiy);
    view[0] = cx - 0.5f * float(width) / s;
    view[1] = cy - 0.5f * float(height) / s;
    view[2] = s;
}

__global__ void render_clear_kernel(float4* __restrict__ acc, int64_t pixels) {
    for (int64_t p = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; p < pixels; p += int64_t(gridDim.x) * blockDim.x)
        acc[p] = make_float4(0.f, 0.f, 0.f, 0.f);
}

// One thread per point: the pixels of the square around its disc.
__global__ void render_splat_kernel(const float2* __restrict__ Y, const float* __restrict__ rgb, int64_t n,
                                    const float* __restrict__ view, int width, int height, float radius,
                                    float alpha, float4* __restrict__ acc) {
    const float x0 = view[0], y0 = view[1], s = view[2];
    const float inv_r = 1.0f / radius;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
        const float2 y = Y[i];
        const float px = (y.x - x0) * s, py = (y.y - y0) * s;
        if (!(px > -radius - 1.f && px < float(width) + radius + 1.f && py > -radius - 1.f &&
              py < float(height) + radius + 1.f))
            continue;  // off the frame (or not finite)
        const float cr = rgb[3 * i], cg = rgb[3 * i + 1], cb = rgb[3 * i + 2];
        const int u0 = max(int(floorf(px - radius)), 0), u1 = min(int(ceilf(px + radius)), width - 1);
        const int v0 = max(int(floorf(py - radius)), 0), v1 = min(int(ceilf(py + radius)), height - 1);
        for (int v = v0; v <= v1; ++v) {
            const float dy = float(v) + 0.5f - py;
            for (int u = u0; u <= u1; ++u) {
                const float dx = float(u) + 0.5f - px;
                const float w = 1.0f - sqrtf(fmaf(dx, dx, dy * dy)) * inv_r;
                if (w > 0.f) {
                    const float aw = alpha * w;
                    float* p = reinterpret_cast<float*>(acc + int64_t(v) * width + u);
                    atomicAdd(p, aw * cr);
                    atomicAdd(p + 1, aw * cg);
                    atomicAdd(p + 2, aw * cb);
                    atomicAdd(p + 3, aw);
                }
            }
        }
    }
}

__device__ __forceinline__ unsigned char store_u8(float v) {
    return static_cast<unsigned char>(floorf(255.0f * fminf(1.0f, fmaxf(0.0f, v)) + 0.5f));
}

// colour = C / A, coverage = min(1, A), composited over the background.
__global__ void render_resolve_kernel(const float4* __restrict__ acc, int64_t pixels, float br, float bg, float bb,
                                      unsigned char* __restrict__ out) {
    for (int64_t p = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; p < pixels; p += int64_t(gridDim.x) * blockDim.x) {
        const float4 a = acc[p];
        float r = br, g = bg, b = bb;
        if (a.w > 0.f) {
            const float cov = fminf(1.0f, a.w), inv = 1.0f / a.w;
            r = fmaf(cov, a.x * inv - br, br);
            g = fmaf(cov, a.y * inv - bg, bg);
            b = fmaf(cov, a.z * inv - bb, bb);
        }
        out[3 * p] = store_u8(r);
        out[3 * p + 1] = store_u8(g);
        out[3 * p + 2] = store_u8(b);
    }
}

}  // namespace drgb

using namespace drgb;

extern "C" int drgb_render(drgb_ctx* c, const float* Y, const float* rgb, int64_t n, int32_t width, int32_t height,
                           float radius, float alpha, const float* background, const float* view_in,
                           float* view_out, uint8_t* frame, void* stream) {
    if (!c) return DRGB_ERR_INVALID;
    if (!Y || !rgb || !frame || !background) return set_error(c, DRGB_ERR_INVALID, "render: NULL pointer");
    if (n < 1 || width < 1 || height < 1 || int64_t(width) * height > (int64_t(1) << 28) || !(radius > 0.f) ||
        !(radius <= 64.f) || !(alpha >= 0.f) || !aligned(Y, 8) || !aligned(rgb, 4))
        return set_error(c, DRGB_ERR_INVALID, "render: bad sizes, radius (0, 64], alpha or alignment");
    if (view_in && !(view_in[2] > 0.f)) return set_error(c, DRGB_ERR_INVALID, "render: view scale must be > 0");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int64_t pixels = int64_t(width) * height;
    int rc = ensure_scratch(c, Carve::round(size_t(pixels) * 16) + 256 + 256, st);
    if (rc) return rc;
    Carve cv(c->scratch);
    float4* acc = cv.take<float4>(size_t(pixels));
    float* view = cv.take<float>(4);
    unsigned int* keys = cv.take<unsigned int>(4);
    const float2* Y2 = reinterpret_cast<const float2*>(Y);
    if (view_in) {
        DRGB_CUDA(c, cudaMemcpyAsync(view, view_in, 3 * sizeof(float), cudaMemcpyHostToDevice, st));
    } else {
        const unsigned int init[4] = {0xffffffffu, 0xffffffffu, 0u, 0u};
        DRGB_CUDA(c, cudaMemcpyAsync(keys, init, sizeof(init), cudaMemcpyHostToDevice, st));
        render_bbox_kernel<<<grid_for(n, 256, c->num_sms * 4), 256, 0, st>>>(Y2, n, keys);
        DRGB_CHECK_LAUNCH(c);
        render_view_kernel<<<1, 1, 0, st>>>(keys, width, height, view);
        DRGB_CHECK_LAUNCH(c);
    }
    render_clear_kernel<<<grid_for(pixels, 256, c->num_sms * 8), 256, 0, st>>>(acc, pixels);
    DRGB_CHECK_LAUNCH(c);
    render_splat_kernel<<<grid_for(n, 128, c->num_sms * 16), 128, 0, st>>>(Y2, rgb, n, view, width, height, radius,
                                                                           alpha, acc);
    DRGB_CHECK_LAUNCH(c);
    render_resolve_kernel<<<grid_for(pixels, 256, c->num_sms * 8), 256, 0, st>>>(acc, pixels, background[0],
                                                                                 background[1], background[2], frame);
    DRGB_CHECK_LAUNCH(c);
    if (view_out) {
        DRGB_CUDA(c, cudaMemcpyAsync(view_out, view, 3 * sizeof(float), cudaMemcpyDeviceToHost, st));
        DRGB_CUDA(c, cudaStreamSynchronize(st));
    }
    return DRGB_OK;
}
