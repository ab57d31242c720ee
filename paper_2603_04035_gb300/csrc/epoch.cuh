// Internal interface of the epoch kernels.
#pragma once
#include "common.cuh"

namespace drgb {

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
    int* status;          // device status word (malformed CSR is reported here)
    unsigned int* work;   // [0] next row block, [1] finished CTAs; zero between launches
    // Batched form (count > 0): rows [inst_off[b], inst_off[b+1]) form instance b,
    // whose entries, negatives and Philox key (inst_seed[b]) are instance-local.
    int count = 0;
    const int64_t* inst_off = nullptr;
    const uint64_t* inst_seed = nullptr;
    // Anchored form: only rows [row_begin, n) are updated (row_ptr is indexed
    // by row - row_begin) and negatives are drawn from [0, neg_n) (0: [0, n)).
    int64_t row_begin = 0;
    uint32_t neg_n = 0;
};

int launch_epoch(Ctx* c, const EpochArgs& A, int rows_per_warp, cudaStream_t st);
int launch_init(Ctx* c, float2* Y, int64_t n, float range, uint64_t seed, cudaStream_t st);
int run_epochs(Ctx* c, float2* Y, float2* Y_tmp, const int32_t* rp, const int32_t* col,
               const uint32_t* q, int64_t n, float a, float b, float lr0, int neg, int t_begin,
               int t_end, int T, uint64_t seed, int rows_per_warp, cudaStream_t st,
               int count = 0, const int64_t* inst_off = nullptr, const uint64_t* inst_seed = nullptr,
               int64_t row_begin = 0, uint32_t neg_n = 0);
// Time every supported epoch schedule on this graph (Ya, Yb: n-float2 scratch)
// and keep the fastest in the context; results do not depend on the choice.
int autotune_epoch(Ctx* c, const float2* Y, float2* Ya, float2* Yb, const int32_t* rp, const int32_t* col,
                   const uint32_t* q, int64_t n, float a, float b, int neg, int T, uint64_t seed, int trials,
                   cudaStream_t st, int count, const int64_t* inst_off, const uint64_t* inst_seed,
                   float* best_us);
// Batched initialisation: row i of instance b gets Philox counter (i - inst_off[b], 0, 0, 1)
// under key inst_seed[b].
int launch_init_batched(Ctx* c, float2* Y, int64_t n_total, float range, int count,
                        const int64_t* inst_off, const uint64_t* inst_seed, cudaStream_t st);

}  // namespace drgb
