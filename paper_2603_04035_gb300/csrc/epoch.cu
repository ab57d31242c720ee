// Initialisation and the synchronous SGD epoch (the method's per-epoch step:
// attraction along active CSR entries, repulsion from Philox negatives, clip
// to +-4, Y' = Y + lr g), plus the epoch loop replayed as a CUDA graph.
//
// Layout: Y is n x 2 FP32 read as float2 (one 8-byte gather per point); the
// CSR is head-sorted (row_ptr int32, col int32, q uint32 schedule words).
// All reads come from Y^(t); there are no atomics.
//
// An epoch is one kernel.  The rows of an instance are cut into windows by
// their first entry: window w holds the rows whose first entry lies in
// [w EPOCH_WIN, (w + 1) EPOCH_WIN) (counted from the instance's first entry).
// One warp takes a window: it compacts the active entries of the window's
// rows into shared memory, computes their forces 32 at a time (one entry per
// lane), adds each head's terms and writes Y' = Y + lr * sum for every row of
// the window.  No row crosses a window, so no row needs a second writer.
//
// Summation order of a row's force (a fixed function of the row's instance
// CSR, so results do not depend on the launch shape, the tuning or on other
// instances of a batch):
//   term(e)    = (((0 + attraction) + repulsion_0) + ...) + repulsion_{neg-1}
//   group sum  = the window's active entries, in entry order, form groups of
//                32; the terms of one head in one group are added by the
//                5-step segmented inclusive scan over the group's lanes (step d
//                adds the partial d lanes to the left)
//   force      = 0 + (((group sum_0) + group sum_1) + ...) over the groups that
//                hold the head, in order
#include <type_traits>

#include "common.cuh"
#include "epoch.cuh"
#include "knn.cuh"  // launch_nonfinite_scan

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

static constexpr unsigned FULL = 0xffffffffu;

// Read of one point of Y^(t).  (Read-only-path and L1 evict-last loads were
// measured and made no difference.)
__device__ __forceinline__ float2 load_y(const float2* p) { return *p; }

// Instance-local view of a row: rows [off, off + n) with entries from eoff on,
// negatives drawn under Philox key (k0, k1).  A single instance has off = 0,
// n = A.n (or the anchored negative range), eoff = 0 and the call's key.
struct RowInst {
    int64_t off;
    uint32_t n;
    int32_t eoff;
    uint32_t k0, k1;
};

// What changes from one epoch to the next: the positions read and written,
// the learning rate and the epoch number.
struct EpochStep {
    const float2* __restrict__ Y_in;
    float2* __restrict__ Y_out;
    float lr;
    uint32_t t;
};

// Negative words of entry e32 at epoch t, group g (negatives 4g .. 4g+3):
// Philox4x32-10 at counter (e, t, g, 0) under the row's key.  A single
// instance takes the precomputed round keys from the kernel parameters.
template <bool BATCHED>
__device__ __forceinline__ U4 negative_words(const EpochArgs& A, const EpochStep& S, const RowInst& R, uint32_t e32,
                                             uint32_t g) {
    if (BATCHED) return philox4x32_10(U4{e32, S.t, g, TAG_NEGATIVE}, R.k0, R.k1);
    return philox4x32_10_rk(U4{e32, S.t, g, TAG_NEGATIVE}, A.rk);
}

// Force on head i from one active entry e = (i, j) and its negatives, summed in
// the fixed order: attraction, then negatives j' = 0 .. neg-1.  NEG is the
// negative count when fixed at compile time (5, the method's default), or -1
// for any count up to 64 (A.neg).
//
// It is split in two so that a warp can gather one group's points while it
// computes the previous group's forces: fetch_entry draws the first (up to
// eight) negatives and issues the loads of Y_i, Y_j and Y_m; entry_math does
// the arithmetic (and, for more than eight negatives, draws and gathers the
// rest itself).
//
// A skipped negative (m = i) is evaluated with Y_m = Y_i: its difference vector
// is zero, so it adds exactly +0 and needs no branch (a sum that starts at +0
// never becomes -0).  A zero distance takes d^b = 0, so coincident points
// repel with zero force as well.
template <int NEG>
struct EntryInputs {
    static constexpr int NP = NEG >= 0 ? (NEG < 8 ? NEG : 8) : 8;  // negatives drawn with the fetch
    float2 yi, yj;
    float2 ym[NP > 0 ? NP : 1];
    int32_t e;
    int32_t i;   // head row; -1 - lane for a lane without a valid entry
    bool ok;
};

template <int NEG, bool BATCHED>
__device__ __forceinline__ void fetch_entry(const EpochArgs& A, const EpochStep& S, const RowInst& R, bool valid,
                                            int32_t e, int32_t j,
                                            int32_t i, int64_t h_lo, int64_t h_hi, int lane,
                                            EntryInputs<NEG>& in) {
    constexpr int NP = EntryInputs<NEG>::NP;
    const int neg = NEG >= 0 ? NEG : A.neg;
    bool ok = valid && i >= h_lo && i < h_hi && uint64_t(uint32_t(j)) < uint64_t(A.n);
    if (valid && !ok) report_status(A.status, DRGB_ERR_INVALID);  // malformed CSR: skip the entry
    in.ok = ok;
    in.e = e;
    in.i = ok ? i : -1 - lane;
    const int32_t ii = ok ? i : int32_t(h_lo);
    in.yi = load_y(S.Y_in + ii);
    in.yj = load_y(S.Y_in + (ok ? j : ii));
    const uint32_t n32 = R.n, i32 = uint32_t(ii - R.off), e32 = uint32_t(e - R.eoff);
    const float2* Yb = S.Y_in + R.off;
    U4 r0{0u, 0u, 0u, 0u}, r1{0u, 0u, 0u, 0u};
    if (NP > 0 && neg > 0) r0 = negative_words<BATCHED>(A, S, R, e32, 0u);
    if (NP > 4 && neg > 4) r1 = negative_words<BATCHED>(A, S, R, e32, 1u);
    const uint32_t u[8] = {r0.x, r0.y, r0.z, r0.w, r1.x, r1.y, r1.z, r1.w};
#pragma unroll
    for (int w = 0; w < NP; ++w) {
        const uint32_t m = __umulhi(u[w], n32);  // floor(u n / 2^32)
        const bool take = ok && (NEG >= 0 || w < neg) && (m != i32);
        in.ym[w] = load_y(Yb + (take ? m : i32));  // a skipped negative reads Y_i
    }
}

template <int NEG, bool BATCHED>
__device__ __forceinline__ float2 entry_math(const EpochArgs& A, const EpochStep& S, const RowInst& R,
                                             const EntryInputs<NEG>& in, float two_ab, float two_b) {
    constexpr int NP = EntryInputs<NEG>::NP;
    const float2 yi = in.yi;
    float gx = 0.f, gy = 0.f;
    {
        const float dx = yi.x - in.yj.x, dy = yi.y - in.yj.y;
        const float d = fmaf(dx, dx, dy * dy);
        const float pb = d > 0.f ? pow_pos(d, A.b) : 0.f;
        const float c = d > 0.f ? __fdividef(-two_ab * pb, d * fmaf(A.a, pb, 1.0f)) : 0.f;
        gx += clip4(c * dx);
        gy += clip4(c * dy);
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
    for (int w = 0; w < NP; ++w) repel(in.ym[w]);
    if (NEG < 0 || NEG > 8) {
        const int neg = NEG >= 0 ? NEG : A.neg;
        const uint32_t n32 = R.n, i32 = uint32_t(in.i - R.off), e32 = uint32_t(in.e - R.eoff);
        const float2* Yb = S.Y_in + R.off;
        for (int g = 2; g * 4 < neg; ++g) {
            const U4 r = negative_words<BATCHED>(A, S, R, e32, uint32_t(g));
            const uint32_t v[4] = {r.x, r.y, r.z, r.w};
            float2 yg[4];
#pragma unroll
            for (int w = 0; w < 4; ++w) {
                const uint32_t m = __umulhi(v[w], n32);
                const bool ok = (g * 4 + w < neg) && (m != i32);
                yg[w] = ok ? load_y(Yb + m) : yi;
            }
#pragma unroll
            for (int w = 0; w < 4; ++w) repel(yg[w]);
        }
    }
    return make_float2(gx, gy);
}

// ------------------------------------------------------------------ per-call preparation
// Head row of every CSR entry of rows [row_begin, n).  Entries not covered by
// any row keep -1; a row whose bounds leave [0, nnz_cap] is reported.
__global__ void epoch_heads_kernel(const int32_t* __restrict__ rp, int64_t n_rows, int64_t row_begin,
                                   int64_t nnz_cap, int32_t* __restrict__ row_of, int* status) {
    for (int64_t lr = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; lr < n_rows;
         lr += int64_t(gridDim.x) * blockDim.x) {
        const int32_t beg = rp[lr], end = rp[lr + 1];
        if (beg < 0 || end < beg || end > nnz_cap) {
            report_status(status, DRGB_ERR_INVALID);
            continue;
        }
        const int32_t r = int32_t(row_begin + lr);
        for (int32_t e = beg; e < end; ++e) row_of[e] = r;
    }
}

// Entry offsets of the instances and their window counts.
__global__ void epoch_instances_kernel(const int32_t* __restrict__ rp, const int64_t* __restrict__ inst_off,
                                       int count, int32_t* __restrict__ inst_eoff, int32_t* __restrict__ win_cnt) {
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b <= count; b += gridDim.x * blockDim.x) {
        inst_eoff[b] = rp[inst_off[b]];
        if (b < count) {
            // an instance without entries still takes one (empty) window, so
            // that its rows are written (Y + lr * 0) and no other instance's
            // window reaches into them
            const int32_t ne = rp[inst_off[b + 1]] - rp[inst_off[b]];
            win_cnt[b] = ne > 0 ? (ne + EPOCH_WIN - 1) / EPOCH_WIN : 1;
        }
    }
}

// First row of every window: window w of an instance holds the rows whose
// first entry lies in [eoff + w EPOCH_WIN, eoff + (w + 1) EPOCH_WIN) (relative
// to the instance's first entry), plus, in the instance's last window, its
// trailing empty rows.  win_row[w + 1] ends window w.
__global__ void epoch_windows_kernel(const int32_t* __restrict__ rp, int64_t n, int64_t row_begin, int count,
                                     const int64_t* __restrict__ inst_off, const int32_t* __restrict__ inst_eoff,
                                     const int32_t* __restrict__ win_base, int64_t win_cap,
                                     int32_t* __restrict__ win_row) {
    const int64_t n_rows = n - row_begin;
    const int32_t n_win = count > 0 ? win_base[count] : (rp[n_rows] + EPOCH_WIN - 1) / EPOCH_WIN;
    for (int64_t w = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; w <= win_cap;
         w += int64_t(gridDim.x) * blockDim.x) {
        if (w >= n_win) {
            win_row[w] = int32_t(n);
            continue;
        }
        int64_t lo, hi;     // rows searched (relative to row_begin), the target entry
        int32_t target;
        if (count > 0) {
            int a = 0, z = count - 1;  // instance whose windows hold w
            while (a < z) {
                const int mid = (a + z + 1) >> 1;
                if (win_base[mid] <= w) a = mid; else z = mid - 1;
            }
            lo = inst_off[a];
            hi = inst_off[a + 1];
            target = inst_eoff[a] + int32_t(w - win_base[a]) * EPOCH_WIN;
        } else {
            lo = 0;
            hi = n_rows;
            target = int32_t(w) * EPOCH_WIN;
        }
        while (lo < hi) {  // first row whose first entry is >= target
            const int64_t mid = (lo + hi) >> 1;
            if (rp[mid] < target) lo = mid + 1; else hi = mid;
        }
        win_row[w] = int32_t(row_begin + lo);
    }
}

size_t epoch_scratch_bytes(int64_t n, int64_t nnz_cap, int count) {
    const int64_t win_cap = (nnz_cap + EPOCH_WIN - 1) / EPOCH_WIN + count;
    size_t b = Carve::round(size_t(nnz_cap > 0 ? nnz_cap : 1) * 4) + Carve::round(size_t(win_cap + 2) * 4);
    if (count > 0)
        b += 3 * Carve::round(size_t(count + 1) * 4) + Carve::round(scan_scratch_elems(count) * 4);
    (void)n;
    return b + 1024;
}

int epoch_prepare(Ctx* c, const int32_t* rp, int64_t n, int64_t row_begin, int64_t nnz_cap, int count,
                  const int64_t* inst_off, void* scratch, EpochScratch* es, cudaStream_t st) {
    Carve cv(scratch);
    es->nnz_cap = nnz_cap;
    es->win_cap = (nnz_cap + EPOCH_WIN - 1) / EPOCH_WIN + count;
    es->row_of = cv.take<int32_t>(size_t(nnz_cap > 0 ? nnz_cap : 1));
    es->win_row = cv.take<int32_t>(size_t(es->win_cap + 2));
    DRGB_CUDA(c, cudaMemsetAsync(es->row_of, 0xFF, size_t(nnz_cap > 0 ? nnz_cap : 1) * 4, st));
    const int64_t n_rows = n - row_begin;
    if (n_rows > 0) {
        epoch_heads_kernel<<<grid_for(n_rows, 256, c->num_sms * 8), 256, 0, st>>>(rp, n_rows, row_begin, nnz_cap,
                                                                                 es->row_of, c->d_status);
        DRGB_CHECK_LAUNCH(c);
    }
    if (count > 0) {
        es->inst_eoff = cv.take<int32_t>(count + 1);
        int32_t* win_cnt = cv.take<int32_t>(count + 1);
        es->win_base = cv.take<int32_t>(count + 1);
        int32_t* tmp = cv.take<int32_t>(scan_scratch_elems(count));
        epoch_instances_kernel<<<grid_for(count + 1, 256, c->num_sms), 256, 0, st>>>(rp, inst_off, count,
                                                                                    es->inst_eoff, win_cnt);
        DRGB_CHECK_LAUNCH(c);
        int rc = exclusive_scan(c, win_cnt, es->win_base, count, tmp, st);
        if (rc) return rc;
    }
    epoch_windows_kernel<<<grid_for(es->win_cap + 1, 256, c->num_sms * 4), 256, 0, st>>>(
        rp, n, row_begin, count, inst_off, es->inst_eoff, es->win_base, es->win_cap, es->win_row);
    DRGB_CHECK_LAUNCH(c);
    return DRGB_OK;
}

// ------------------------------------------------------------------ epoch kernel
// Programmatic dependent launch: an epoch launched right after another one
// may start while that one finishes.  Everything before grid_dep_wait() reads
// only the CSR and the prepared tables (which no epoch writes); Y is read and
// written only after it, when the previous epoch's grid has completed and its
// writes are visible.  Without a programmatic dependency both are no-ops.
__device__ __forceinline__ void grid_dep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void grid_dep_launch() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// CSR chunks (of 32 entries) a warp loads at once before testing them.  The
// window's CSR words are streamed in bursts so that several loads are in
// flight per lane; the active entries of a burst wait in a per-warp queue of
// at most 31 + 32 * burst entries.  The queue is kept this small on
// purpose: shared memory left unused goes to the L1 cache, and the random
// 8-byte gathers of Y run at about 2.5x the rate with the largest L1 (the
// misses in flight per SM are bounded by L1 capacity).
static constexpr int EPOCH_BURST = 4;
constexpr int epoch_qcap(int burst) { return 32 * burst + 32; }
// Warps per SM each form's register budget is sized for: the pipelined form
// holds two groups' gathered points (about 80 registers a thread), the flat
// form one (about 48).
static constexpr int epoch_warps_per_sm(bool pipe) { return pipe ? 24 : 40; }

// Where a window's CSR words come from: global memory, streamed with
// evict-first loads (they are read once per epoch, so L2 keeps the gathered
// positions Y instead).
struct CsrGlobal {
    const uint32_t* __restrict__ q;
    const int32_t* __restrict__ col;
    const int32_t* __restrict__ row_of;
    __device__ __forceinline__ void load(int32_t e, bool in, uint32_t& qv, int32_t& jv, int32_t& hv) const {
        qv = in ? __ldcs(q + e) : 0u;  // q = 0 never fires
        jv = in ? __ldcs(col + e) : 0;
        hv = in ? __ldcs(row_of + e) : -1;
    }
};
// One window W of epoch S, by one warp.  No row crosses a window, so the warp
// writes the final Y' of every row of the window.
//
// The warp streams the window's CSR in bursts of BURST chunks of 32 entries
// (one entry per lane and chunk, coalesced) and appends each burst's active
// entries to its queue, in entry order.  Every 32 waiting entries form a
// group: one entry per lane, its negatives drawn and its points gathered
// (fetch), then its force computed and the group's terms added by head
// (segmented scan, carry between groups).  The window's last group may be
// partial.
//
// PIPE: the gathers of a group are issued before the previous group's forces
// are computed, so one warp keeps two groups' loads in flight (for grids with
// few windows per SM); the next burst's CSR loads are issued before the held
// group is finished.  Without PIPE each group is finished before the next is
// fetched, and latency is hidden by more warps per SM (for grids with many
// windows).  Both forms form the same groups and add in the same order, so
// they give the same bits.
template <bool BATCHED, int NEG, bool PIPE, int BURST, class Csr>
__device__ __forceinline__ void epoch_window(const EpochArgs& A, const EpochStep& S, const Csr& csr, int32_t W,
                                             int lane, int2* act_w, int32_t* head_w, float4* carry_w,
                                             int32_t* chead_w, float two_ab, float two_b) {
    const unsigned lt_mask = (1u << lane) - 1u;
    const int32_t rA = A.win_row[W], rB = A.win_row[W + 1];
    if (rA >= rB) return;  // a long row started in an earlier window covers this one
    RowInst R{0, A.neg_n ? A.neg_n : uint32_t(A.n), 0, A.k0, A.k1};
    int64_t h_lo = A.row_begin, h_hi = A.n;  // rows a head may take (the instance's rows)
    if (BATCHED) {
        int lo = 0, hi = A.count - 1;  // the instance whose windows hold W
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (A.win_base[mid] <= W) lo = mid; else hi = mid - 1;
        }
        R.off = A.inst_off[lo];
        R.n = uint32_t(A.inst_off[lo + 1] - R.off);
        R.eoff = A.inst_eoff[lo];
        R.k0 = uint32_t(A.inst_seed[lo]);
        R.k1 = uint32_t(A.inst_seed[lo] >> 32);
        h_lo = R.off;
        h_hi = R.off + R.n;
    }
    if (rA < h_lo || rB > h_hi) {
        if (lane == 0) report_status(A.status, DRGB_ERR_INVALID);
        return;
    }
    const int32_t es = A.row_ptr[rA - A.row_begin], ee = A.row_ptr[rB - A.row_begin];
    // Negatives and gathers of `cnt` waiting entries from queue position p.
    auto fetch_group = [&](int p, int cnt, EntryInputs<NEG>& in) {
        const bool v = lane < cnt;
        const int2 ej = v ? act_w[p + lane] : make_int2(es, 0);
        fetch_entry<NEG, BATCHED>(A, S, R, v, ej.x, ej.y, v ? head_w[p + lane] : -1, h_lo, h_hi, lane, in);
    };
    // Forces of a fetched group of `cnt` entries, added by head.
    auto finish_group = [&](const EntryInputs<NEG>& cur, int cnt) {
        float fx = 0.f, fy = 0.f;
        if (cur.ok) {
            const float2 f = entry_math<NEG, BATCHED>(A, S, R, cur, two_ab, two_b);
            fx = f.x;
            fy = f.y;
        }
        const int32_t i = cur.i;
        const int32_t chead = *chead_w;
        // the carried head ends unless this group starts with it
        if (chead >= 0 && lane == 0 && i != chead) {
            const float4 cv = *carry_w;
            S.Y_out[chead] = make_float2(fmaf(S.lr, 0.f + cv.x, cv.z), fmaf(S.lr, 0.f + cv.y, cv.w));
        }
        // segmented inclusive scan over runs of equal heads
        const int32_t i_prev = __shfl_up_sync(FULL, i, 1);
        const unsigned starts = __ballot_sync(FULL, lane == 0 || i_prev != i);
        const int seg0 = 31 - __clz(starts & (FULL >> (31 - lane)));
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const float ox = __shfl_up_sync(FULL, fx, d), oy = __shfl_up_sync(FULL, fy, d);
            if (lane - d >= seg0) {
                fx = ox + fx;
                fy = oy + fy;
            }
        }
        if (seg0 == 0 && i == chead) {
            const float4 cv = *carry_w;
            fx = cv.x + fx;
            fy = cv.y + fy;
        }
        // a run that ends inside the group is the row's last: write it; the
        // group's last run is carried
        const int32_t i_next = __shfl_down_sync(FULL, i, 1);
        if (cur.ok && lane < cnt - 1 && i_next != i)
            S.Y_out[i] = make_float2(fmaf(S.lr, 0.f + fx, cur.yi.x), fmaf(S.lr, 0.f + fy, cur.yi.y));
        __syncwarp();
        if (lane == cnt - 1) {
            *carry_w = make_float4(fx, fy, cur.yi.x, cur.yi.y);
            *chead_w = cur.ok ? i : -1;
        }
        __syncwarp();
    };
    EntryInputs<NEG> held;  // PIPE: the fetched group waiting for its forces
    int held_cnt = 0;
    int qn = 0;             // active entries waiting at the front of the queue
    // (a window whose rows are all empty still takes one, empty, burst)
    for (int32_t c0 = es; c0 == es || c0 < ee; c0 += 32 * BURST) {
        // the burst's CSR words, all loads in flight before any test
        uint32_t qv[BURST];
        int32_t jv[BURST], hv[BURST];
#pragma unroll
        for (int b = 0; b < BURST; ++b) {
            const int32_t e = c0 + 32 * b + lane;
            csr.load(e, e < ee, qv[b], jv[b], hv[b]);
        }
        if (PIPE && held_cnt) {  // the previous burst's last group, while the loads fly
            finish_group(held, held_cnt);
            held_cnt = 0;
        }
#pragma unroll
        for (int b = 0; b < BURST; ++b) {
            // floor((t+1) q / 2^24) > floor(t q / 2^24)  <=>  (t q mod 2^24) + q >= 2^24
            const bool act = qv[b] >= 0x1000000u - ((S.t * qv[b]) & 0xFFFFFFu);
            const unsigned m = __ballot_sync(FULL, act);
            if (act) {
                const int pos = qn + __popc(m & lt_mask);
                act_w[pos] = make_int2(c0 + 32 * b + lane, jv[b]);
                head_w[pos] = hv[b];
            }
            qn += __popc(m);
        }
        __syncwarp();
        if (c0 == es) {
            // every row of the window first gets Y + lr * 0; rows with active
            // entries are rewritten with their force below.  The wait for the
            // previous epoch comes here, after the first burst has been loaded
            // and tested.
            grid_dep_wait();
            for (int64_t r = rA + lane; r < rB; r += 32) {
                const float2 y = load_y(S.Y_in + r);
                S.Y_out[r] = make_float2(fmaf(S.lr, 0.f, y.x), fmaf(S.lr, 0.f, y.y));
            }
            if (lane == 0) *chead_w = -1;
            __syncwarp();
        }
        const bool last = c0 + 32 * BURST >= ee;
        const int ng = last ? (qn + 31) / 32 : qn / 32;
        for (int g = 0; g < ng; ++g) {
            const int cnt = qn - 32 * g < 32 ? qn - 32 * g : 32;
            EntryInputs<NEG> in;
            fetch_group(32 * g, cnt, in);
            if (PIPE) {
                if (held_cnt) finish_group(held, held_cnt);
                held = in;
                held_cnt = cnt;
            } else {
                finish_group(in, cnt);
            }
        }
        // move the waiting partial group to the front
        const int left = qn - 32 * ng > 0 ? qn - 32 * ng : 0;
        int2 lv = make_int2(0, 0);
        int32_t lh = -1;
        if (lane < left) {
            lv = act_w[32 * ng + lane];
            lh = head_w[32 * ng + lane];
        }
        __syncwarp();
        if (lane < left) {
            act_w[lane] = lv;
            head_w[lane] = lh;
        }
        qn = left;
        __syncwarp();
    }
    if (PIPE && held_cnt) finish_group(held, held_cnt);
    if (lane == 0 && *chead_w >= 0) {
        const float4 cv = *carry_w;
        S.Y_out[*chead_w] = make_float2(fmaf(S.lr, 0.f + cv.x, cv.z), fmaf(S.lr, 0.f + cv.y, cv.w));
    }
    __syncwarp();
}

// Entries and windows of the call, checked against the prepared tables.
__device__ __forceinline__ bool epoch_extent(const EpochArgs& A, int32_t& nnz, int32_t& n_win) {
    if (A.count > 0) {
        nnz = A.inst_eoff[A.count];
        n_win = A.win_base[A.count];
    } else {
        nnz = A.row_ptr[A.n - A.row_begin];
        n_win = (nnz + EPOCH_WIN - 1) / EPOCH_WIN;
    }
    return nnz >= 0 && nnz <= A.nnz_cap && n_win <= A.win_cap;
}

// One epoch: one warp per window (grid-stride over windows).
template <bool BATCHED, int NEG, int NW, bool PIPE>
__global__ void __launch_bounds__(NW * 32, epoch_warps_per_sm(PIPE) / NW)
    epoch_force_kernel(const __grid_constant__ EpochArgs A) {
    constexpr int QCAP = epoch_qcap(EPOCH_BURST);
    __shared__ int2 s_ej[NW][QCAP];     // (entry, tail) of the waiting active entries
    __shared__ int32_t s_hd[NW][QCAP];  // their heads
    // carry of each warp: running sum of the previous group's last head and
    // that head's position; the head itself (-1 when none)
    __shared__ float4 s_carry[NW];
    __shared__ int32_t s_chead[NW];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const float two_ab = 2.0f * A.a * A.b, two_b = 2.0f * A.b;
    const EpochStep S{A.Y_in, A.Y_out, A.lr, A.t};
    grid_dep_launch();
    int32_t nnz = 0, n_win = 0;
    if (!epoch_extent(A, nnz, n_win)) {
        if (threadIdx.x == 0 && blockIdx.x == 0) report_status(A.status, DRGB_ERR_INVALID);
        return;
    }
    if (n_win == 0) {  // no entries at all: every row keeps its position
        grid_dep_wait();
        for (int64_t r = A.row_begin + int64_t(blockIdx.x) * blockDim.x + threadIdx.x; r < A.n;
             r += int64_t(gridDim.x) * blockDim.x) {
            const float2 y = A.Y_in[r];
            A.Y_out[r] = make_float2(fmaf(A.lr, 0.f, y.x), fmaf(A.lr, 0.f, y.y));
        }
        return;
    }
    const CsrGlobal csr{A.q, A.col, A.row_of};
    for (int32_t W = int32_t(blockIdx.x) * NW + w; W < n_win; W += int32_t(gridDim.x) * NW)
        epoch_window<BATCHED, NEG, PIPE, EPOCH_BURST>(A, S, csr, W, lane, s_ej[w], s_hd[w], &s_carry[w], &s_chead[w],
                                                      two_ab, two_b);
}

bool epoch_warps_supported(int warps) { return warps == 4 || warps == 8; }

int launch_epoch(Ctx* c, const EpochArgs& A_in, int warps, cudaStream_t st, bool after_epoch) {
    if (warps <= 0) warps = c->epoch_warps;
    if (!epoch_warps_supported(warps))
        return set_error(c, DRGB_ERR_INVALID, "epoch: unsupported force-kernel width %d", warps);
    if (!A_in.row_of || !A_in.win_row) return set_error(c, DRGB_ERR_INVALID, "epoch: state not prepared");
    EpochArgs A = A_in;
    philox_round_keys(A.k0, A.k1, A.rk);
    const bool bat = A.count > 0, n5 = A.neg == 5;
    const bool pipe = c->epoch_pipe != 0;
    const int per_sm = epoch_warps_per_sm(pipe) / warps;
    const int fgrid = grid_for(A.win_cap, warps, c->num_sms * per_sm);
    auto go = [&](auto kernel) -> int {
        // Ask for no more shared memory than the resident CTAs hold (their
        // queues plus the 1 KB the hardware reserves per CTA); the rest of the
        // SM's 256 KB stays L1 cache for the gathers of Y.
        cudaFuncAttributes fa;
        DRGB_CUDA(c, cudaFuncGetAttributes(&fa, kernel));
        const size_t need = size_t(per_sm) * (fa.sharedSizeBytes + 1024);
        int pct = int((need * 100 + c->smem_per_sm - 1) / (c->smem_per_sm ? c->smem_per_sm : 1));
        pct = pct < 1 ? 1 : (pct > 100 ? 100 : pct);
        DRGB_CUDA(c, cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout, pct));
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(fgrid);
        cfg.blockDim = dim3(warps * 32);
        cfg.dynamicSmemBytes = 0;
        cfg.stream = st;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[0].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = attr;
        cfg.numAttrs = after_epoch ? 1 : 0;  // only an epoch may precede with overlap
        DRGB_CUDA(c, cudaLaunchKernelEx(&cfg, kernel, A));
        return DRGB_OK;
    };
    auto pick = [&](auto nw, auto pp) -> int {
        constexpr int NW = decltype(nw)::value;
        constexpr bool P = decltype(pp)::value;
        return bat ? (n5 ? go(epoch_force_kernel<true, 5, NW, P>) : go(epoch_force_kernel<true, -1, NW, P>))
                   : (n5 ? go(epoch_force_kernel<false, 5, NW, P>) : go(epoch_force_kernel<false, -1, NW, P>));
    };
    using I4 = std::integral_constant<int, 4>;
    using I8 = std::integral_constant<int, 8>;
    using PT = std::true_type;
    using PF = std::false_type;
    int rc = warps == 4 ? (pipe ? pick(I4{}, PT{}) : pick(I4{}, PF{})) : (pipe ? pick(I8{}, PT{}) : pick(I8{}, PF{}));
    if (rc) return rc;
    DRGB_CHECK_LAUNCH(c);
    return DRGB_OK;
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

static void fill_args(EpochArgs& A, const int32_t* rp, const int32_t* col, const uint32_t* q, int64_t n, float a,
                      float b, int neg, uint64_t seed, int* status, const EpochScratch& es, int count,
                      const int64_t* inst_off, const uint64_t* inst_seed, int64_t row_begin, uint32_t neg_n) {
    A.row_ptr = rp;
    A.col = col;
    A.q = q;
    A.n = n;
    A.a = a;
    A.b = b;
    A.neg = neg;
    A.k0 = uint32_t(seed);
    A.k1 = uint32_t(seed >> 32);
    A.status = status;
    A.row_of = es.row_of;
    A.win_row = es.win_row;
    A.nnz_cap = es.nnz_cap;
    A.win_cap = es.win_cap;
    A.count = count;
    A.inst_off = inst_off;
    A.inst_seed = inst_seed;
    A.inst_eoff = es.inst_eoff;
    A.win_base = es.win_base;
    A.row_begin = row_begin;
    A.neg_n = neg_n;
}

// Epochs [t_begin, t_end) of a T-epoch schedule, ping-ponging between Y and
// Y_tmp; the result is left in Y.  The launches are captured into a CUDA
// graph (on a private stream) and the graph is launched on `st`.  Building an
// executable graph of hundreds of nodes costs milliseconds of host time, so
// the context keeps the last one and refreshes it in place
// (cudaGraphExecUpdate: same nodes, new parameters) whenever the new loop has
// the same shape; a launch already enqueued keeps the parameters it had.
int run_epochs(Ctx* c, float2* Y, float2* Y_tmp, const int32_t* rp, const int32_t* col, const uint32_t* q,
               int64_t n, float a, float b, float lr0, int neg, int t_begin, int t_end, int T, uint64_t seed,
               cudaStream_t st, int64_t nnz_cap, void* scratch, int count, const int64_t* inst_off,
               const uint64_t* inst_seed, int64_t row_begin, uint32_t neg_n) {
    if (t_end <= t_begin) return DRGB_OK;
    EpochScratch es;
    int rc = epoch_prepare(c, rp, n, row_begin, nnz_cap, count, inst_off, scratch, &es, st);
    if (rc) return rc;
    cudaStream_t cap;
    DRGB_CUDA(c, cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
        cudaStreamDestroy(cap);
        return set_error(c, DRGB_ERR_CUDA, "begin capture: %s", cudaGetErrorString(e));
    }
    float2* src = Y;
    float2* dst = Y_tmp;
    for (int t = t_begin; t < t_end && rc == DRGB_OK; ++t) {
        EpochArgs A;
        fill_args(A, rp, col, q, n, a, b, neg, seed, c->d_status, es, count, inst_off, inst_seed, row_begin, neg_n);
        A.Y_in = src;
        A.Y_out = dst;
        A.lr = float(double(lr0) * (1.0 - double(t) / double(T)));
        A.t = uint32_t(t);
        rc = launch_epoch(c, A, 0, cap, t > t_begin);
        float2* tmp = src;
        src = dst;
        dst = tmp;
    }
    if (rc == DRGB_OK && src != Y)
        cudaMemcpyAsync(Y, src, size_t(n) * sizeof(float2), cudaMemcpyDeviceToDevice, cap);
    e = cudaStreamEndCapture(cap, &graph);
    if (rc == DRGB_OK && e != cudaSuccess)
        rc = set_error(c, DRGB_ERR_CUDA, "end capture: %s", cudaGetErrorString(e));
    if (rc == DRGB_OK && c->epoch_exec) {
        cudaGraphExecUpdateResultInfo info;
        if (cudaGraphExecUpdate(c->epoch_exec, graph, &info) != cudaSuccess) {
            cudaGetLastError();  // a different shape: build a new executable graph
            cudaGraphExecDestroy(c->epoch_exec);
            c->epoch_exec = nullptr;
        }
    }
    if (rc == DRGB_OK && !c->epoch_exec) {
        e = cudaGraphInstantiate(&c->epoch_exec, graph, 0);
        if (e != cudaSuccess) {
            c->epoch_exec = nullptr;
            rc = set_error(c, DRGB_ERR_CUDA, "instantiate: %s", cudaGetErrorString(e));
        }
    }
    if (rc == DRGB_OK) {
        e = cudaGraphLaunch(c->epoch_exec, st);
        if (e != cudaSuccess) rc = set_error(c, DRGB_ERR_CUDA, "graph launch: %s", cudaGetErrorString(e));
    }
    if (graph) cudaGraphDestroy(graph);
    cudaStreamDestroy(cap);
    return rc;
}

// Force-kernel widths and forms tried by the tuner.
static const int kWarpChoices[] = {4, 8};
static const int kPipeChoices[] = {1, 0};

int autotune_epoch(Ctx* c, const float2* Y, float2* Ya, float2* Yb, const int32_t* rp, const int32_t* col,
                   const uint32_t* q, int64_t n, float a, float b, int neg, int T, uint64_t seed, int trials,
                   cudaStream_t st, const EpochScratch& es, int count, const int64_t* inst_off,
                   const uint64_t* inst_seed, float* best_us) {
    cudaEvent_t e0, e1;
    DRGB_CUDA(c, cudaEventCreate(&e0));
    DRGB_CUDA(c, cudaEventCreate(&e1));
    const int saved_pipe = c->epoch_pipe;
    int best_w = c->epoch_warps, best_p = c->epoch_pipe, rc = DRGB_OK;
    float best = 1e30f;
    const int t0 = T / 4 < T - trials ? T / 4 : (T - trials > 0 ? T - trials : 0);
    for (int pipe : kPipeChoices) {
        c->epoch_pipe = pipe;
        for (int warps : kWarpChoices) {
            EpochArgs A;
            fill_args(A, rp, col, q, n, a, b, neg, seed, c->d_status, es, count, inst_off, inst_seed, 0, 0);
            if (cudaMemcpyAsync(Ya, Y, size_t(n) * 8, cudaMemcpyDeviceToDevice, st) != cudaSuccess) {
                rc = set_error(c, DRGB_ERR_CUDA, "autotune: copy failed");
                break;
            }
            float ms = 0.f;
            for (int pass = 0; pass < 2 && rc == DRGB_OK; ++pass) {  // pass 0 warms up
                cudaEventRecord(e0, st);
                for (int k = 0; k < trials && rc == DRGB_OK; ++k) {
                    A.Y_in = (k & 1) ? Yb : Ya;
                    A.Y_out = (k & 1) ? Ya : Yb;
                    A.t = uint32_t(t0 + k);
                    A.lr = 1.0f - float(t0 + k) / float(T);
                    rc = launch_epoch(c, A, warps, st, k > 0);
                }
                cudaEventRecord(e1, st);
                if (cudaEventSynchronize(e1) != cudaSuccess) rc = set_error(c, DRGB_ERR_CUDA, "autotune: sync failed");
                cudaEventElapsedTime(&ms, e0, e1);
            }
            if (rc) break;
            const float us = ms * 1000.f / trials;
            if (us < best) {
                best = us;
                best_w = warps;
                best_p = pipe;
            }
        }
        if (rc) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    c->epoch_pipe = saved_pipe;
    if (rc) return rc;
    c->epoch_warps = best_w;
    c->epoch_pipe = best_p;
    if (best_us) *best_us = best;
    return DRGB_OK;
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
    if (!aligned(rp, 4) || !aligned(col, 4) || !aligned(q, 4))
        return set_error(c, DRGB_ERR_INVALID, "embed_epoch: CSR arrays must be 4-byte aligned");
    if (n < 1 || n > INT32_MAX) return set_error(c, DRGB_ERR_INVALID, "embed_epoch: bad n");
    if (neg < 0 || neg > 64) return set_error(c, DRGB_ERR_INVALID, "embed_epoch: neg out of range");
    return DRGB_OK;
}

// Entry count row_ptr[n] (read back to size the per-call state) and that state.
static int epoch_state_for(drgb_ctx* c, const int32_t* rp, int64_t n, cudaStream_t st, EpochScratch* es) {
    int32_t nnz = 0;
    DRGB_CUDA(c, cudaMemcpyAsync(&nnz, rp + n, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    DRGB_CUDA(c, cudaStreamSynchronize(st));
    if (nnz < 0) return set_error(c, DRGB_ERR_INVALID, "embed_epoch: row_ptr[n] < 0");
    int rc = ensure_scratch(c, epoch_scratch_bytes(n, nnz, 0), st);
    if (rc) return rc;
    return epoch_prepare(c, rp, n, 0, nnz, 0, nullptr, c->scratch, es, st);
}

int drgb_embed_epoch(drgb_ctx* c, const float* Y_in, float* Y_out, const int32_t* row_ptr,
                     const int32_t* col, const uint32_t* q, int64_t n, float a, float b, float lr,
                     int32_t neg, int32_t epoch, uint64_t seed, void* stream) {
    int rc = check_epoch_args(c, Y_in, Y_out, row_ptr, col, q, n, neg);
    if (rc) return rc;
    if (epoch < 0) return set_error(c, DRGB_ERR_INVALID, "embed_epoch: epoch < 0");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    EpochScratch es;
    if ((rc = epoch_state_for(c, row_ptr, n, st, &es))) return rc;
    if ((rc = launch_nonfinite_scan(c, Y_in, 2 * n, st))) return rc;  // reported by the next synchronising call
    EpochArgs A;
    fill_args(A, row_ptr, col, q, n, a, b, neg, seed, c->d_status, es, 0, nullptr, nullptr, 0, 0);
    A.Y_in = reinterpret_cast<const float2*>(Y_in);
    A.Y_out = reinterpret_cast<float2*>(Y_out);
    A.lr = lr;
    A.t = uint32_t(epoch);
    return launch_epoch(c, A, 0, st);
}

int drgb_embed_epochs(drgb_ctx* c, float* Y, float* Y_tmp, const int32_t* row_ptr,
                      const int32_t* col, const uint32_t* q, int64_t n, float a, float b,
                      float lr0, int32_t neg, int32_t t_begin, int32_t t_end, int32_t n_epochs,
                      uint64_t seed, void* stream) {
    int rc = check_epoch_args(c, Y, Y_tmp, row_ptr, col, q, n, neg);
    if (rc) return rc;
    if (!(0 <= t_begin && t_begin <= t_end && t_end <= n_epochs) || n_epochs < 1)
        return set_error(c, DRGB_ERR_INVALID, "embed_epochs: bad epoch range");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int32_t nnz = 0;
    DRGB_CUDA(c, cudaMemcpyAsync(&nnz, row_ptr + n, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    DRGB_CUDA(c, cudaStreamSynchronize(st));
    if (nnz < 0) return set_error(c, DRGB_ERR_INVALID, "embed_epochs: row_ptr[n] < 0");
    if ((rc = ensure_scratch(c, epoch_scratch_bytes(n, nnz, 0), st))) return rc;
    if ((rc = launch_nonfinite_scan(c, Y, 2 * n, st))) return rc;  // reported by the next synchronising call
    return run_epochs(c, reinterpret_cast<float2*>(Y), reinterpret_cast<float2*>(Y_tmp), row_ptr, col, q, n, a,
                      b, lr0, neg, t_begin, t_end, n_epochs, seed, st, nnz, c->scratch);
}

}  // extern "C"
