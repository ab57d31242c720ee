// Internal interface of the epoch kernels.
#pragma once
#include "common.cuh"

namespace drgb {

// CSR entries per window of the epoch kernel.  Part of the summation order
// (see epoch.cu), so it is a constant, not a tuning knob.
static constexpr int EPOCH_WIN = 512;

struct EpochArgs {
    const float2* __restrict__ Y_in;
    float2* __restrict__ Y_out;
    const int32_t* __restrict__ row_ptr;
    const int32_t* __restrict__ col;
    const uint32_t* __restrict__ q;
    int64_t n;
    float a, b, lr;
    int neg;
    uint32_t t;
    uint32_t k0, k1;
    uint32_t rk[20];      // Philox round keys of (k0, k1); filled by launch_epoch
    int* status;          // device status word (malformed CSR is reported here)
    // Prepared per call (epoch_prepare): head row of every CSR entry, and the
    // first row of every window (win_row[w] .. win_row[w + 1] - 1 are its rows).
    const int32_t* __restrict__ row_of;
    const int32_t* __restrict__ win_row;
    int64_t nnz_cap;      // entries row_of covers (the CSR may not hold more)
    int64_t win_cap;      // windows win_row covers
    // Batched form (count > 0): rows [inst_off[b], inst_off[b+1]) form instance b,
    // whose entries, negatives and Philox key (inst_seed[b]) are instance-local.
    // Its entries are [inst_eoff[b], inst_eoff[b+1]) and its windows start at
    // win_base[b] (win_base[count] windows in all).
    int count = 0;
    const int64_t* inst_off = nullptr;
    const uint64_t* inst_seed = nullptr;
    const int32_t* inst_eoff = nullptr;
    const int32_t* win_base = nullptr;
    // Anchored form: only rows [row_begin, n) are updated (row_ptr is indexed
    // by row - row_begin) and negatives are drawn from [0, neg_n) (0: [0, n)).
    int64_t row_begin = 0;
    uint32_t neg_n = 0;
};

// Device buffers an epoch needs besides the CSR and Y (carved from `scratch`).
struct EpochScratch {
    int32_t* row_of = nullptr;
    int32_t* win_row = nullptr;
    int32_t* inst_eoff = nullptr;
    int32_t* win_base = nullptr;
    int64_t nnz_cap = 0;
    int64_t win_cap = 0;
};

// Bytes of scratch for n rows (all instances), at most nnz_cap CSR entries
// and `count` instances (0: one instance).
size_t epoch_scratch_bytes(int64_t n, int64_t nnz_cap, int count);

// Build the per-call epoch state on `st`: heads of the CSR entries of rows
// [row_begin, n), the windows' first rows and, for count > 0, the instances'
// entry offsets and window bases.
int epoch_prepare(Ctx* c, const int32_t* rp, int64_t n, int64_t row_begin, int64_t nnz_cap, int count,
                  const int64_t* inst_off, void* scratch, EpochScratch* es, cudaStream_t st);

// One epoch (one kernel launch).  `warps` = warps per CTA (0: the context's
// setting).  `after_epoch`: the previous launch on `st` is an epoch of the same
// prepared state, so this one may start early (programmatic dependent launch).
int launch_epoch(Ctx* c, const EpochArgs& A, int warps, cudaStream_t st, bool after_epoch = false);
int launch_init(Ctx* c, float2* Y, int64_t n, float range, uint64_t seed, cudaStream_t st);

// Epochs [t_begin, t_end) of a T-epoch schedule, ping-ponging between Y and
// Y_tmp (the result is left in Y), captured as one CUDA graph.  `scratch`
// holds epoch_scratch_bytes(n, nnz_cap, count) bytes.
int run_epochs(Ctx* c, float2* Y, float2* Y_tmp, const int32_t* rp, const int32_t* col, const uint32_t* q,
               int64_t n, float a, float b, float lr0, int neg, int t_begin, int t_end, int T, uint64_t seed,
               cudaStream_t st, int64_t nnz_cap, void* scratch, int count = 0, const int64_t* inst_off = nullptr,
               const uint64_t* inst_seed = nullptr, int64_t row_begin = 0, uint32_t neg_n = 0);

// Time every supported force-kernel width and form on this graph for `trials`
// epochs (Ya, Yb: n-float2 scratch; Y is not modified) and keep the fastest in
// the context; results do not depend on the choice.  `es` comes from
// epoch_prepare.
int autotune_epoch(Ctx* c, const float2* Y, float2* Ya, float2* Yb, const int32_t* rp, const int32_t* col,
                   const uint32_t* q, int64_t n, float a, float b, int neg, int T, uint64_t seed, int trials,
                   cudaStream_t st, const EpochScratch& es, int count, const int64_t* inst_off,
                   const uint64_t* inst_seed, float* best_us);

// Batched initialisation: row i of instance b gets Philox counter (i - inst_off[b], 0, 0, 1)
// under key inst_seed[b].
int launch_init_batched(Ctx* c, float2* Y, int64_t n_total, float range, int count,
                        const int64_t* inst_off, const uint64_t* inst_seed, cudaStream_t st);

}  // namespace drgb
