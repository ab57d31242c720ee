// Initialisation and the synchronous SGD epoch (the method's per-epoch step:
// attraction along active CSR entries, repulsion from Philox negatives, clip
// to +-4, Y' = Y + lr g), plus the epoch loop replayed as a CUDA graph.
//
// Layout: Y is n x 2 FP32 read as float2 (one 8-byte gather per point); the
// CSR is head-sorted (row_ptr int32, col int32, q uint32 schedule words).
// No atomics: every row is written by exactly one lane, and all reads come
// from Y^(t).
#include "common.cuh"
#include "epoch.cuh"

namespace drgb {

__global__ void init_embedding_kernel(float2* __restrict__ Y, int64_t n, float range, uint32_t k0,
                                      uint32_t k1) {
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
         i += int64_t(gridDim.x) * blockDim.x) {
        U4 r = philox4x32_10(U4{uint32_t(i), 0u, 0u, TAG_INIT}, k0, k1);
        const float s = 5.9604644775390625e-08f;  // 2^-24
        float ux = float(r.x >> 8) * s, uy = float(r.y >> 8) * s;
        Y[i] = make_float2(fmaf(ux, 2.0f * range, -range), fmaf(uy, 2.0f * range, -range));
    }
}

__global__ void init_batched_kernel(float2* __restrict__ Y, int64_t n, float range, int count,
                                    const int64_t* __restrict__ inst_off, const uint64_t* __restrict__ inst_seed) {
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
         i += int64_t(gridDim.x) * blockDim.x) {
        int lo = 0, hi = count - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (inst_off[mid] <= i) lo = mid; else hi = mid - 1;
        }
        const uint64_t seed = inst_seed[lo];
        U4 r = philox4x32_10(U4{uint32_t(i - inst_off[lo]), 0u, 0u, TAG_INIT}, uint32_t(seed), uint32_t(seed >> 32));
        const float s = 5.9604644775390625e-08f;  // 2^-24
        float ux = float(r.x >> 8) * s, uy = float(r.y >> 8) * s;
        Y[i] = make_float2(fmaf(ux, 2.0f * range, -range), fmaf(uy, 2.0f * range, -range));
    }
}

__device__ __forceinline__ float clip4(float v) { return fminf(4.0f, fmaxf(-4.0f, v)); }

__device__ __forceinline__ float hw_ex2(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float hw_lg2(float x) {
    float y;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// d^b for d > 0 via the hardware base-2 logarithm and exponential.
__device__ __forceinline__ float pow_pos(float d, float b) { return hw_ex2(b * hw_lg2(d)); }

// Warps per CTA of the epoch kernel; rows per warp block is a template
// parameter (a tuning knob: fewer rows give more warps, more rows fill the
// per-warp queue of active entries better).
static constexpr int EPOCH_WARPS = 8;
static constexpr int QPF_MAX = 16;                 // most 32-entry chunks whose q words load together
static constexpr int QCAP = 32 + 32 * QPF_MAX;     // queue slots per warp
static constexpr unsigned FULL = 0xffffffffu;

// Force on head i from one active entry e = (i, j) and its negatives, summed in
// the fixed order: attraction, then negatives j' = 0 .. neg-1.  The first
// eight negatives are drawn before any gather, so their loads, the col[e]
// load and the Y_j load overlap; further negatives (neg > 8) follow in groups
// of four.
// Instance-local view of a row: rows [off, off + n) with entries from eoff on,
// negatives drawn under Philox key (k0, k1).  A single instance has off = 0,
// n = A.n, eoff = 0 and the call's key.
struct RowInst {
    int64_t off;
    uint32_t n;
    int32_t eoff;
    uint32_t k0, k1;
};

__device__ __forceinline__ float2 entry_force(const EpochArgs& A, int32_t e, int64_t i, float2 yi,
                                              float two_ab, float two_b, const RowInst& R) {
    const int32_t j = A.col[e];
    const uint32_t n32 = R.n, i32 = uint32_t(i - R.off), e32 = uint32_t(e - R.eoff);
    const float2* Yb = A.Y_in + R.off;
    const U4 r0 = philox4x32_10(U4{e32, A.t, 0u, TAG_NEGATIVE}, R.k0, R.k1);
    const U4 r1 = A.neg > 4 ? philox4x32_10(U4{e32, A.t, 1u, TAG_NEGATIVE}, R.k0, R.k1) : r0;
    const uint32_t u[8] = {r0.x, r0.y, r0.z, r0.w, r1.x, r1.y, r1.z, r1.w};
    bool ok[8];
    float2 ym[8];
#pragma unroll
    for (int w = 0; w < 8; ++w) {
        const uint32_t m = __umulhi(u[w], n32);  // floor(u n / 2^32)
        ok[w] = (w < A.neg) && (m != i32);
        ym[w] = ok[w] ? Yb[m] : yi;
    }
    const bool j_ok = uint64_t(uint32_t(j)) < uint64_t(A.n);
    if (!j_ok) {  // malformed CSR: report and skip the entry
        report_status(A.status, DRGB_ERR_INVALID);
        return make_float2(0.f, 0.f);
    }
    const float2 yj = A.Y_in[j];
    float gx = 0.f, gy = 0.f;
    {
        const float dx = yi.x - yj.x, dy = yi.y - yj.y;
        const float d = fmaf(dx, dx, dy * dy);
        if (d > 0.f) {
            const float pb = pow_pos(d, A.b);
            const float c = __fdividef(-two_ab * pb, d * fmaf(A.a, pb, 1.0f));
            gx += clip4(c * dx);
            gy += clip4(c * dy);
        }
    }
    auto repel = [&](float2 y) {
        const float rx = yi.x - y.x, ry = yi.y - y.y;
        const float dm = fmaf(rx, rx, ry * ry);
        const float pb = dm > 0.f ? pow_pos(dm, A.b) : 0.f;
        const float c = __fdividef(two_b, (0.001f + dm) * fmaf(A.a, pb, 1.0f));
        gx += clip4(c * rx);
        gy += clip4(c * ry);
    };
#pragma unroll
    for (int w = 0; w < 8; ++w)
        if (ok[w]) repel(ym[w]);
    for (int g = 2; g * 4 < A.neg; ++g) {
        const U4 r = philox4x32_10(U4{e32, A.t, uint32_t(g), TAG_NEGATIVE}, R.k0, R.k1);
        const uint32_t v[4] = {r.x, r.y, r.z, r.w};
        bool okg[4];
        float2 yg[4];
#pragma unroll
        for (int w = 0; w < 4; ++w) {
            const uint32_t m = __umulhi(v[w], n32);
            okg[w] = (g * 4 + w < A.neg) && (m != i32);
            yg[w] = okg[w] ? Yb[m] : yi;
        }
#pragma unroll
        for (int w = 0; w < 4; ++w)
            if (okg[w]) repel(yg[w]);
    }
    return make_float2(gx, gy);
}

// Row blocks are handed out dynamically (one atomic per block from a counter
// that the last CTA to finish resets), so no SM idles while others still hold
// several blocks; which warp takes a block does not change any result.
//
// One warp owns a block of EPOCH_ROWS consecutive head rows.  Its lanes scan
// the block's CSR entries 32 at a time (coalesced q loads), test the schedule,
// and append the active entries to a per-warp queue in shared memory; each
// time 32 are queued, every lane computes the force of one queued entry, so
// all lanes work although only about a quarter of the entries fire in an
// epoch.  The lane that owns a row then adds that row's forces in entry order,
// which makes each row's sum independent of how entries fell into batches.
template <int EPOCH_ROWS, int Q_PREFETCH, bool DYNAMIC>
__global__ void __launch_bounds__(EPOCH_WARPS * 32, 4)
embed_epoch_kernel(EpochArgs A) {
    __shared__ int32_t s_rp[EPOCH_WARPS][EPOCH_ROWS + 1];
    __shared__ float2 s_y[EPOCH_WARPS][EPOCH_ROWS];
    __shared__ int32_t s_qe[EPOCH_WARPS][QCAP];
    __shared__ int32_t s_qh[EPOCH_WARPS][QCAP];
    __shared__ float2 s_term[EPOCH_WARPS][32];
    __shared__ int32_t s_seg[EPOCH_WARPS][32];   // per owner row: first queue slot | count << 8
    __shared__ RowInst s_inst[EPOCH_WARPS][EPOCH_ROWS];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const unsigned lt_mask = (1u << lane) - 1u;
    const float two_ab = 2.0f * A.a * A.b, two_b = 2.0f * A.b;
    const uint64_t t0 = A.t, t1 = uint64_t(A.t) + 1;
    const int64_t n_blocks = (A.n - A.row_begin + EPOCH_ROWS - 1) / EPOCH_ROWS;
    int64_t rb_static = int64_t(blockIdx.x) * EPOCH_WARPS + w;
    for (;;) {
        int64_t rb = 0;
        if (DYNAMIC) {
            if (lane == 0) rb = atomicAdd(A.work, 1u);
            rb = __shfl_sync(FULL, rb, 0);
        } else {
            rb = rb_static;
            rb_static += int64_t(gridDim.x) * EPOCH_WARPS;
        }
        if (rb >= n_blocks) break;
        const int64_t r0 = A.row_begin + rb * EPOCH_ROWS;
        const int nr = int(A.n - r0 < EPOCH_ROWS ? A.n - r0 : EPOCH_ROWS);
        if (lane <= nr) s_rp[w][lane] = A.row_ptr[r0 - A.row_begin + lane];
        if (lane < nr) {
            s_y[w][lane] = A.Y_in[r0 + lane];
            RowInst R{0, A.neg_n ? A.neg_n : uint32_t(A.n), 0, A.k0, A.k1};
            if (A.count > 0) {
                const int64_t i = r0 + lane;
                int lo = 0, hi = A.count - 1;  // instance b with inst_off[b] <= i
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (A.inst_off[mid] <= i) lo = mid; else hi = mid - 1;
                }
                R.off = A.inst_off[lo];
                R.n = uint32_t(A.inst_off[lo + 1] - R.off);
                R.eoff = A.row_ptr[R.off];
                R.k0 = uint32_t(A.inst_seed[lo]);
                R.k1 = uint32_t(A.inst_seed[lo] >> 32);
            }
            s_inst[w][lane] = R;
        }
        __syncwarp();
        const int32_t e_begin = s_rp[w][0], e_end = s_rp[w][nr];
        float ax = 0.f, ay = 0.f;
        int qn = 0;

        auto process = [&](int cnt) {
            float2 f = make_float2(0.f, 0.f);
            const int h = lane < cnt ? s_qh[w][lane] : -1 - lane;
            if (lane < cnt) f = entry_force(A, s_qe[w][lane], r0 + h, s_y[w][h], two_ab, two_b, s_inst[w][h]);
            s_term[w][lane] = f;
            s_seg[w][lane] = 0;
            __syncwarp();
            // queue slots are sorted by head: each head's slots are contiguous
            const unsigned same = __match_any_sync(FULL, h);
            if (lane < cnt && lane == __ffs(same) - 1) s_seg[w][h] = lane | (__popc(same) << 8);
            __syncwarp();
            const int seg = s_seg[w][lane];
            for (int t = seg & 0xff, t_end = (seg & 0xff) + (seg >> 8); t < t_end; ++t) {
                ax += s_term[w][t].x;
                ay += s_term[w][t].y;
            }
            __syncwarp();
        };

        // fill the queue (scanning Q_PREFETCH chunks per step) until 32
        // entries wait or the block is scanned, then process 32 (or the rest)
        int32_t e_cur = e_begin;
        for (;;) {
            while (qn < 32 && e_cur < e_end) {
                uint32_t qv[Q_PREFETCH];
#pragma unroll
                for (int c = 0; c < Q_PREFETCH; ++c) {
                    const int32_t e = e_cur + 32 * c + lane;
                    qv[c] = e < e_end ? A.q[e] : 0u;  // q = 0 never fires
                }
#pragma unroll
                for (int c = 0; c < Q_PREFETCH; ++c) {
                    const int32_t e = e_cur + 32 * c + lane;
                    const uint32_t qe = qv[c];
                    const bool act = ((t1 * qe) >> 24) != ((t0 * qe) >> 24);
                    const unsigned mask = __ballot_sync(FULL, act);
                    if (act) {
                        int lo = 0, hi = nr - 1;  // last row h with s_rp[h] <= e
                        while (lo < hi) {
                            const int mid = (lo + hi + 1) >> 1;
                            if (s_rp[w][mid] <= e) lo = mid; else hi = mid - 1;
                        }
                        const int pos = qn + __popc(mask & lt_mask);
                        s_qe[w][pos] = e;
                        s_qh[w][pos] = lo;
                    }
                    qn += __popc(mask);
                }
                e_cur += 32 * Q_PREFETCH;
                __syncwarp();
            }
            if (qn == 0) break;
            const int cnt = qn < 32 ? qn : 32;
            process(cnt);
            for (int t = lane; t < qn - cnt; t += 32) {
                const int32_t qe = s_qe[w][t + cnt], qh = s_qh[w][t + cnt];
                __syncwarp(__activemask());
                s_qe[w][t] = qe;
                s_qh[w][t] = qh;
            }
            qn -= cnt;
            __syncwarp();
        }
        if (lane < nr) {
            const float2 yi = s_y[w][lane];
            A.Y_out[r0 + lane] = make_float2(fmaf(A.lr, ax, yi.x), fmaf(A.lr, ay, yi.y));
        }
        __syncwarp();
    }
    // the last CTA to finish resets the work counter for the next launch
    if (!DYNAMIC) return;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(A.work + 1, 1u) == gridDim.x - 1) {
            A.work[0] = 0;
            A.work[1] = 0;
            __threadfence();
        }
    }
}

int launch_epoch(Ctx* c, const EpochArgs& A, int rows, cudaStream_t st) {
    const int threads = EPOCH_WARPS * 32;
    if (rows <= 0) rows = c->epoch_rows;
    const int64_t row_blocks = (A.n - A.row_begin + rows - 1) / rows;
    const int blocks = grid_for(row_blocks, EPOCH_WARPS, c->num_sms * 4);
    if (!A.work) return set_error(c, DRGB_ERR_INVALID, "epoch: no work counter");
    const int pf = c->epoch_prefetch;
    const bool dyn = c->epoch_dynamic != 0;
#define DRGB_EPOCH_CASE(R, P)                                                           \
    if (rows == R && pf == P) {                                                        \
        if (dyn) embed_epoch_kernel<R, P, true><<<blocks, threads, 0, st>>>(A);        \
        else embed_epoch_kernel<R, P, false><<<blocks, threads, 0, st>>>(A);           \
        DRGB_CHECK_LAUNCH(c);                                                          \
        return DRGB_OK;                                                                \
    }
    DRGB_EPOCH_CASE(4, 4)
    DRGB_EPOCH_CASE(4, 8)
    DRGB_EPOCH_CASE(8, 4)
    DRGB_EPOCH_CASE(8, 8)
    DRGB_EPOCH_CASE(8, 16)
    DRGB_EPOCH_CASE(16, 4)
    DRGB_EPOCH_CASE(16, 8)
    DRGB_EPOCH_CASE(16, 16)
    DRGB_EPOCH_CASE(31, 16)
#undef DRGB_EPOCH_CASE
    return set_error(c, DRGB_ERR_INVALID, "epoch: unsupported rows/prefetch combination %d/%d", rows, pf);
}

int launch_init_batched(Ctx* c, float2* Y, int64_t n_total, float range, int count,
                        const int64_t* inst_off, const uint64_t* inst_seed, cudaStream_t st) {
    int blocks = grid_for(n_total, 256, c->num_sms * 16);
    init_batched_kernel<<<blocks, 256, 0, st>>>(Y, n_total, range, count, inst_off, inst_seed);
    DRGB_CHECK_LAUNCH(c);
    return DRGB_OK;
}

int launch_init(Ctx* c, float2* Y, int64_t n, float range, uint64_t seed, cudaStream_t st) {
    int blocks = grid_for(n, 256, c->num_sms * 16);
    init_embedding_kernel<<<blocks, 256, 0, st>>>(Y, n, range, uint32_t(seed), uint32_t(seed >> 32));
    DRGB_CHECK_LAUNCH(c);
    return DRGB_OK;
}

// Epochs [t_begin, t_end) of a T-epoch schedule, ping-ponging between Y and
// Y_tmp; the result is left in Y.  The launches are captured once into a CUDA
// graph (on a private stream) and the graph is launched on `st`.
int run_epochs(Ctx* c, float2* Y, float2* Y_tmp, const int32_t* rp, const int32_t* col,
               const uint32_t* q, int64_t n, float a, float b, float lr0, int neg, int t_begin,
               int t_end, int T, uint64_t seed, int rows_per_warp, cudaStream_t st, int count,
               const int64_t* inst_off, const uint64_t* inst_seed, int64_t row_begin, uint32_t neg_n) {
    if (t_end <= t_begin) return DRGB_OK;
    cudaStream_t cap;
    DRGB_CUDA(c, cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int rc = DRGB_OK;
    cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
        cudaStreamDestroy(cap);
        return set_error(c, DRGB_ERR_CUDA, "begin capture: %s", cudaGetErrorString(e));
    }
    float2* src = Y;
    float2* dst = Y_tmp;
    for (int t = t_begin; t < t_end && rc == DRGB_OK; ++t) {
        EpochArgs A;
        A.Y_in = src;
        A.Y_out = dst;
        A.row_ptr = rp;
        A.col = col;
        A.q = q;
        A.n = n;
        A.a = a;
        A.b = b;
        A.lr = float(double(lr0) * (1.0 - double(t) / double(T)));
        A.neg = neg;
        A.t = uint32_t(t);
        A.k0 = uint32_t(seed);
        A.k1 = uint32_t(seed >> 32);
        A.status = c->d_status;
        A.work = c->d_work;
        A.count = count;
        A.inst_off = inst_off;
        A.inst_seed = inst_seed;
        A.row_begin = row_begin;
        A.neg_n = neg_n;
        rc = launch_epoch(c, A, rows_per_warp, cap);
        float2* tmp = src;
        src = dst;
        dst = tmp;
    }
    if (rc == DRGB_OK && src != Y)
        cudaMemcpyAsync(Y, src, size_t(n) * sizeof(float2), cudaMemcpyDeviceToDevice, cap);
    e = cudaStreamEndCapture(cap, &graph);
    if (rc == DRGB_OK && e != cudaSuccess)
        rc = set_error(c, DRGB_ERR_CUDA, "end capture: %s", cudaGetErrorString(e));
    if (rc == DRGB_OK) {
        e = cudaGraphInstantiate(&exec, graph, 0);
        if (e != cudaSuccess) rc = set_error(c, DRGB_ERR_CUDA, "instantiate: %s", cudaGetErrorString(e));
    }
    if (rc == DRGB_OK) {
        e = cudaGraphLaunch(exec, st);
        if (e != cudaSuccess) rc = set_error(c, DRGB_ERR_CUDA, "graph launch: %s", cudaGetErrorString(e));
    }
    // The executable graph may be destroyed right after the launch is
    // enqueued; the launch keeps what it needs.
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    cudaStreamDestroy(cap);
    return rc;
}

}  // namespace drgb

using namespace drgb;

extern "C" {

int drgb_init_embedding(drgb_ctx* c, int64_t n, float init_range, uint64_t seed, float* Y,
                        void* stream) {
    if (!c || !Y || n < 1 || !aligned(Y, 8) || !(init_range > 0.f))
        return set_error(c, DRGB_ERR_INVALID, "init_embedding: invalid argument");
    return launch_init(c, reinterpret_cast<float2*>(Y), n, init_range, seed,
                       static_cast<cudaStream_t>(stream));
}

static int check_epoch_args(drgb_ctx* c, const float* Y_in, const float* Y_out, const int32_t* rp,
                            const int32_t* col, const uint32_t* q, int64_t n, int32_t neg) {
    if (!c) return DRGB_ERR_INVALID;
    if (!Y_in || !Y_out || !rp || !col || !q)
        return set_error(c, DRGB_ERR_INVALID, "embed_epoch: NULL pointer");
    if (Y_in == Y_out) return set_error(c, DRGB_ERR_INVALID, "embed_epoch: Y_out aliases Y_in");
    if (!aligned(Y_in, 8) || !aligned(Y_out, 8))
        return set_error(c, DRGB_ERR_INVALID, "embed_epoch: Y must be 8-byte aligned");
    if (n < 1 || n > INT32_MAX) return set_error(c, DRGB_ERR_INVALID, "embed_epoch: bad n");
    if (neg < 0 || neg > 64) return set_error(c, DRGB_ERR_INVALID, "embed_epoch: neg out of range");
    return DRGB_OK;
}

int drgb_embed_epoch(drgb_ctx* c, const float* Y_in, float* Y_out, const int32_t* row_ptr,
                     const int32_t* col, const uint32_t* q, int64_t n, float a, float b, float lr,
                     int32_t neg, int32_t epoch, uint64_t seed, void* stream) {
    int rc = check_epoch_args(c, Y_in, Y_out, row_ptr, col, q, n, neg);
    if (rc) return rc;
    if (epoch < 0) return set_error(c, DRGB_ERR_INVALID, "embed_epoch: epoch < 0");
    EpochArgs A;
    A.Y_in = reinterpret_cast<const float2*>(Y_in);
    A.Y_out = reinterpret_cast<float2*>(Y_out);
    A.row_ptr = row_ptr;
    A.col = col;
    A.q = q;
    A.n = n;
    A.a = a;
    A.b = b;
    A.lr = lr;
    A.neg = neg;
    A.t = uint32_t(epoch);
    A.k0 = uint32_t(seed);
    A.k1 = uint32_t(seed >> 32);
    A.status = c->d_status;
    A.work = c->d_work;
    return launch_epoch(c, A, 0, static_cast<cudaStream_t>(stream));
}

int drgb_embed_epochs(drgb_ctx* c, float* Y, float* Y_tmp, const int32_t* row_ptr,
                      const int32_t* col, const uint32_t* q, int64_t n, float a, float b,
                      float lr0, int32_t neg, int32_t t_begin, int32_t t_end, int32_t n_epochs,
                      uint64_t seed, void* stream) {
    int rc = check_epoch_args(c, Y, Y_tmp, row_ptr, col, q, n, neg);
    if (rc) return rc;
    if (!(0 <= t_begin && t_begin <= t_end && t_end <= n_epochs) || n_epochs < 1)
        return set_error(c, DRGB_ERR_INVALID, "embed_epochs: bad epoch range");
    return run_epochs(c, reinterpret_cast<float2*>(Y), reinterpret_cast<float2*>(Y_tmp), row_ptr,
                      col, q, n, a, b, lr0, neg, t_begin, t_end, n_epochs, seed, 0,
                      static_cast<cudaStream_t>(stream));
}

}  // extern "C"
