// Internal interface of the k-NN kernels.
#pragma once
#include "common.cuh"

namespace drgb {

// Insert (d, j) into a list D[0..K) sorted ascending by d, dropping the last
// entry; precondition d < D[K-1].  Equal values keep their arrival order.
template <int K>
__device__ __forceinline__ void topk_insert(float (&D)[K], int32_t (&I)[K], float d, int32_t j) {
#pragma unroll
    for (int s = K - 1; s > 0; --s) {
        const bool shift = d < D[s - 1];
        const bool place = !shift && d < D[s];
        D[s] = shift ? D[s - 1] : (place ? d : D[s]);
        I[s] = shift ? I[s - 1] : (place ? j : I[s]);
    }
    if (d < D[0]) {
        D[0] = d;
        I[0] = j;
    }
}

int check_knn_args(Ctx* c, const float* X, int64_t n, int d, int k, const void* idx_out,
                   const void* dist_out);
// Exact FP32 scan for the given query rows (rows == nullptr: rows 0..n_rows-1).
int launch_knn_exact(Ctx* c, const float* X, int64_t n, int d, int k, const int64_t* rows,
                     int64_t n_rows, int32_t* idx_out, float* dist_out, bool write_sqrt,
                     cudaStream_t st);
// Exact FP32 scan of the rows listed in rows32[0 .. cnt) (cnt known on the
// host; n_rows_dev, the same count on the device, is read by the single-pass
// form).  On entry each listed row of idx_out/dist_out must already hold k
// distinct points other than the row in ascending order of their FP32
// distances (the direct sum over dimensions), INFINITY where it has fewer:
// the scan keeps only points within the listed k-th distance.  The scan is
// split over database chunks (partial lists in part_scratch, merged by a
// second kernel); results are written to the listed rows.
int launch_knn_exact_rows_n(Ctx* c, const float* X, int64_t n, int d, int k, const int32_t* rows32,
                            const int32_t* n_rows_dev, int64_t cnt, int32_t* idx_out, float* dist_out,
                            cudaStream_t st, void* part_scratch, size_t part_bytes);
// Merge C partial k-lists per listed row: list l of row r at
// (l * cnt + r) * k in pidx/pd2 (squared distances, ascending by (distance,
// index), ended early by index -1); the k best by (distance, index) go to
// row rows32[r] of idx_out/dist_out (Euclidean distances).
int launch_merge_partials(Ctx* c, const int32_t* pidx, const float* pd2, int64_t cnt, int C, int k,
                          const int32_t* rows32, int32_t* idx_out, float* dist_out, cudaStream_t st);
// Exact FP32 k-NN of the nq rows of Q among the n rows of X (no self exclusion).
int launch_knn_query(Ctx* c, const float* Q, int64_t nq, const float* X, int64_t n, int d, int k,
                     int32_t* idx_out, float* dist_out, cudaStream_t st);
// Per query row: sum over its k targets of max(0, rank_X - k).
int launch_rank(Ctx* c, const float* X, int64_t n, int d, int k, const int64_t* rows,
                int64_t n_rows, const int32_t* tgt, int64_t* excess_out, cudaStream_t st);
int launch_nonfinite_scan(Ctx* c, const float* X, int64_t count, cudaStream_t st);

// BF16 tensor-core candidate generation + FP32 re-rank (knn_tc.cu).
bool knn_tc_preferred(int64_t n, int d, int k);
size_t knn_tc_scratch_bytes(int64_t n, int d);
// `scratch` must hold knn_tc_scratch_bytes(n, d) bytes (256-byte aligned).
// With defer_rows/defer_count (device; *defer_count zeroed by the caller) the
// uncertified rows are appended there (row indices of X) and not re-scanned:
// the caller re-scans them later (launch_knn_exact_rows_n), which lets many
// k-NN runs be enqueued without a host synchronisation.
int knn_tc(Ctx* c, const float* X, int64_t n, int d, int k, bool f16, int32_t* idx_out, float* dist_out,
           cudaStream_t st, void* scratch, int32_t* defer_rows = nullptr, int32_t* defer_count = nullptr);
// Bytes of scratch a deferred re-scan may use for its partial lists.
size_t knn_rescan_part_bytes();

// Spatial order for the tensor-core k-NN (knn_order.cu): K cells from
// farthest-point pivots; perm[p] = point at position p (p < n), cell c holds
// positions [cell_beg[c], cell_beg[c+1]) inside the sphere (centre[c], radius[c]).
int knn_order_cells(int64_t n);
size_t knn_order_scratch_bytes(int64_t n, int d, int K);
int knn_order(Ctx* c, const float* X, int64_t n, int d, int K, int32_t* perm, int32_t* cell_beg, float* centre,
              float* radius, void* scratch, cudaStream_t st);

// k-NN graph with the mode resolved (0 = auto); `scratch` holds
// knn_scratch_bytes(n, d, k, mode) bytes (may be null when that is 0).
int knn_resolve_mode(int64_t n, int d, int k, int mode);
size_t knn_scratch_bytes(int64_t n, int d, int k, int mode);
// defer_rows/defer_count: as for knn_tc (the exact-scan modes leave no
// uncertified rows).
int knn_run(Ctx* c, const float* X, int64_t n, int d, int k, int mode, int32_t* idx_out, float* dist_out,
            cudaStream_t st, void* scratch, int32_t* defer_rows = nullptr, int32_t* defer_count = nullptr);

}  // namespace drgb
