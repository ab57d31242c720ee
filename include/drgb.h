/*
 * drgb.h - C ABI of the GB300 neighbour-embedding library (libdrgb.so).
 *
 * The library computes the data-parallel hot path of the UMAP method as used
 * by mlx-vis (arXiv 2603.04035): the exact k-NN graph (Section 2.2), the
 * fuzzy simplicial-set graph and the a, b kernel fit (Section 2.3), and the
 * synchronous negative-sampling SGD epoch (Section 2.5, the UMAP optimiser step;
 * Section 4.1, scatter-add updates on sampled edges), composed into
 * fit_transform(X) -> n x 2 (Section 2.1, public API).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Pointers named X, Y, idx, dist, row_ptr, col, w, q, ... are DEVICE
 *   pointers owned by the caller; the library never frees them and never keeps
 *   them past the call.  Matrices are dense row-major: X is n x d FP32 (row
 *   stride d), Y is n x 2 FP32 (x, y interleaved; 8-byte aligned).
 * - `stream` is a cudaStream_t passed as void*; NULL means the legacy default
 *   stream.  All device work is enqueued on it; calls return before it runs
 *   unless documented as synchronous.
 * - A drgb_ctx owns the library's scratch memory (grown on demand with
 *   cudaMalloc, released by drgb_ctx_destroy), a device status word that the
 *   kernels set on device-side errors, and the last error message.  A context
 *   is bound to one device and must not be used from two host threads at once.
 * - Every function returns an int status: DRGB_OK or a negative DRGB_ERR_*.
 *   Argument errors are detected on the host before anything is enqueued.
 *   Device-side errors (non-finite input, a timed-out wait) are recorded in
 *   the context and reported by the next synchronising call (drgb_sync or a
 *   call documented as synchronous).
 */
#ifndef DRGB_H
#define DRGB_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define DRGB_OK 0
#define DRGB_ERR_INVALID (-1)    /* bad argument: null/misaligned pointer, n < k+1, k out of range */
#define DRGB_ERR_WORKSPACE (-2)  /* caller-provided capacity too small */
#define DRGB_ERR_CUDA (-3)       /* a CUDA runtime call failed (message in drgb_last_error) */
#define DRGB_ERR_TIMEOUT (-4)    /* a bounded device-side wait gave up */
#define DRGB_ERR_NONFINITE (-5)  /* NaN or Inf found in an input */
#define DRGB_ERR_DEVICE (-6)     /* device is not sm_103 (GB300) */

#define DRGB_MAX_K 32            /* largest supported number of neighbours */

typedef struct drgb_ctx drgb_ctx;

/* Hyper-parameters of fit_transform (Section 2.1: a method object is created
 * with its hyper-parameters; defaults follow UMAP as used in Section 3). */
typedef struct drgb_params {
    int32_t k;            /* neighbours per point (default 15), 1..DRGB_MAX_K */
    int32_t n_epochs;     /* T, number of SGD epochs (Section 3: 500 for UMAP) */
    int32_t neg;          /* negative samples per active edge (default 5) */
    float lr0;            /* initial learning rate, decayed as lr0 (1 - t/T) */
    float min_dist;       /* output-kernel min_dist (default 0.1) */
    float spread;         /* output-kernel spread (default 1.0) */
    float init_range;     /* Y0 ~ U[-init_range, init_range]^2 (default 10) */
    uint64_t seed_init;   /* Philox key of the initialisation */
    uint64_t seed_neg;    /* Philox key of the negative samples */
    int32_t knn_mode;     /* 0 auto, 1 exact FP32 scan, 2 BF16 / 3 FP16 tensor-core + FP32 re-rank,
                             4 approximate NNDescent (drgb_knn_nndescent with seed_init, delta 0.015,
                             at most 30 iterations, the reverse form when k <= 16; fit_transform
                             only) */
    int32_t flags;        /* DRGB_FLAG_* bits */
    int32_t pca_dim;      /* 0 (default): none; 1..56: fit_transform first projects X on its pca_dim
                             leading principal components (drgb_pca) when d > pca_dim (Section 3:
                             the timed pipeline includes PCA preprocessing; Section 3.3 names
                             the pca_dim knob) */
} drgb_params;

/* drgb_params.flags: time the epoch schedules on the actual graph before the
 * loop and keep the fastest (results are identical for every schedule). */
#define DRGB_FLAG_AUTOTUNE 1
/* drgb_params.flags: start from the spectral layout of the fuzzy graph
 * (drgb_spectral_init, with init_range and seed_init) instead of the uniform
 * one; the fit then synchronises its stream during the initialisation. */
#define DRGB_FLAG_INIT_SPECTRAL 2

/* Called after each epoch by fit_transform (Section 2.1, epoch_callback).
 * Y_dev is the current device embedding (n x 2, valid during the call only);
 * the stream is synchronised before the call.  Return non-zero to stop early. */
typedef int (*drgb_epoch_cb)(int32_t epoch, const float* Y_dev, int64_t n, void* user);

/* ------------------------------------------------------------------ context */

/* Library version as 10000*major + 100*minor + patch. */
int drgb_version(void);

/* Create a context on `device` (must be compute capability 10.3).
 * Errors: DRGB_ERR_INVALID (out == NULL), DRGB_ERR_DEVICE, DRGB_ERR_CUDA. */
int drgb_ctx_create(int device, drgb_ctx** out);

/* Free the context's scratch memory and the context.  NULL is a no-op. */
int drgb_ctx_destroy(drgb_ctx* ctx);

/* Last error message of `ctx` ("" if none); valid until the next call. */
const char* drgb_last_error(const drgb_ctx* ctx);

/* Synchronise `stream`, read and clear the device status word.
 * Returns DRGB_OK or the first device-side error since the last sync. */
int drgb_sync(drgb_ctx* ctx, void* stream);

/* Self-test of the bounded device-side waits (no counterpart in the paper):
 * every tensor-core kernel of the library waits on its mbarriers for at most
 * 2 s, then reports DRGB_ERR_TIMEOUT through the context's status word,
 * drains what it has issued and returns instead of hanging the GPU.  This
 * call runs that same wait in a one-thread kernel on a barrier nothing
 * arrives at (arrive = 0; with arrive != 0 the thread arrives first and the
 * wait succeeds), with a limit of limit_us microseconds (1 .. 10,000,000).
 * Synchronous: returns DRGB_ERR_TIMEOUT (arrive = 0) or DRGB_OK (arrive != 0)
 * as read back by drgb_sync, which clears the status word, so later calls on
 * the context start clean.  DRGB_ERR_INVALID for a NULL context or a limit
 * out of range. */
int drgb_wait_selftest(drgb_ctx* ctx, int64_t limit_us, int32_t arrive, void* stream);

/* Random-gather probe (no counterpart in the paper; the roofline denominator
 * of the SGD epoch, whose work is one random 8-byte load of Y per tail and per
 * negative sample): every thread the GPU holds resident (largest L1 carveout)
 * makes rounds x 8 loads of float2 values of Y at indices drawn from
 * multiplicative congruential streams (seed) and mapped onto [0, n) by
 * multiply-shift.  *gathers_per_s receives the loads per second of the timed
 * launch (one warm-up launch first).  Y: n x 2 FP32 (device, 8-byte aligned,
 * caller-owned), 1 <= n < 2^32; 1 <= rounds <= 4096.  Synchronous.  Errors:
 * DRGB_ERR_INVALID (NULL, misaligned, sizes). */
int drgb_gather_probe(drgb_ctx* ctx, const float* Y, int64_t n, int32_t rounds, uint32_t seed,
                      double* gathers_per_s, void* stream);

/* Bytes of scratch the context currently holds (for memory accounting). */
int64_t drgb_ctx_scratch_bytes(const drgb_ctx* ctx);

/* Cap on the context's scratch memory (no counterpart in the paper, whose
 * runs fail with out-of-memory when a problem does not fit, Section 3.3):
 * bytes > 0 makes every later call that would need more scratch than `bytes`
 * fail with DRGB_ERR_WORKSPACE before anything is enqueued (the message
 * gives both sizes), and frees the current scratch now if it is larger
 * (waiting for the device); 0 (the default) removes the cap.  A refused call
 * leaves the context usable.  Errors: DRGB_ERR_INVALID (NULL, bytes < 0). */
int drgb_set_scratch_limit(drgb_ctx* ctx, int64_t bytes);

/* Number of kernels this context has launched (graph replays count every
 * kernel node they contain).  Host-side counter, for launch accounting. */
int64_t drgb_launch_count(const drgb_ctx* ctx);

/* Tuning knobs (performance only; results do not depend on them):
 *   DRGB_TUNE_EPOCH_WARPS     warps per CTA of the epoch's force kernel: 4 or 8
 *   DRGB_TUNE_EPOCH_PIPE      form of the epoch's force kernel: 1 (default)
 *                             pipelined (a warp keeps two groups of gathers in
 *                             flight, 24 warps per SM), 0 flat (one group, 40
 *                             warps per SM)
 * Returns DRGB_ERR_INVALID for an unknown parameter or value. */
#define DRGB_TUNE_EPOCH_WARPS 1
#define DRGB_TUNE_EPOCH_PIPE 2
int drgb_set_tuning(drgb_ctx* ctx, int32_t param, int32_t value);
/* Current value of a tuning knob in *value.  DRGB_ERR_INVALID for an unknown
 * parameter or a NULL pointer. */
int drgb_get_tuning(const drgb_ctx* ctx, int32_t param, int32_t* value);

/* Tuning cache (host only; no counterpart in the paper, for repeated batched runs):
 * a JSON file mapping "device name|SM count|rows 2^a|instances 2^b|k c" keys
 * to tuned settings, one entry per line:
 * {"<key>": {"epoch_warps": 8, "epoch_pipe": 1}, ...}.
 * drgb_set_tuning_cache makes drgb_fit_transform_batched with
 * DRGB_FLAG_AUTOTUNE use the file's setting for its key when there is one,
 * and otherwise time the choices and add the winner to the file (path NULL
 * or "": no cache).  drgb_tuning_cache_lookup writes the stored force-kernel
 * width and form of `key` to *epoch_warps and *epoch_pipe (an entry without
 * "epoch_pipe" reads as the default form 1; DRGB_ERR_INVALID if the file or
 * key is missing or a stored value unsupported); drgb_tuning_cache_store adds or
 * replaces the entry, rewriting the file through a temporary file and a
 * rename (DRGB_ERR_INVALID for a bad key or value, or an I/O failure).  Keys
 * are printable ASCII without quotes or backslashes, shorter than 256 bytes.
 * Calls that update one file concurrently may lose each other's entries. */
int drgb_set_tuning_cache(drgb_ctx* ctx, const char* path);
int drgb_tuning_cache_lookup(const char* path, const char* key, int32_t* epoch_warps, int32_t* epoch_pipe);
int drgb_tuning_cache_store(const char* path, const char* key, int32_t epoch_warps, int32_t epoch_pipe);

/* Stage timing of drgb_fit_transform.  When enabled (on != 0), each fit
 * records CUDA events on its stream between its stages; drgb_stage_times
 * (synchronous: waits for the events) writes up to `max` elapsed times in
 * milliseconds: [0] k-NN graph, [1] fuzzy graph, [2] initialisation,
 * [3] epoch loop, and within [0], for the tensor-core k-NN (each 0 if the
 * exact scan ran): [4] the GEMM + selection kernel alone, [5] its ordering
 * and operand staging, [6] the FP32 re-rank and certificate, [7] the exact
 * re-scan of uncertified rows; returns the number written (or a negative
 * error). */
int drgb_set_profiling(drgb_ctx* ctx, int on);
int drgb_stage_times(drgb_ctx* ctx, float* ms, int max);

/* ------------------------------------------------------------- k-NN graph */

/* Exact k-nearest-neighbour graph (Section 2.2: every method starts from a
 * k-NN search, approximate NNDescent in the paper; this library returns the
 * exact graph).
 *   X        n x d FP32, row-major (4-byte aligned).
 *   idx_out  n x k int32: the k nearest OTHER points of each row (self
 *            excluded), ordered by FP32 squared distance sum_c (x_ic - x_jc)^2
 *            evaluated directly (not by the expansion), ties by lower index.
 *   dist_out n x k FP32 Euclidean distances (square roots), same order.
 * mode: 0 auto (3 when n >= 4096, d <= 61, k < 32; else 1), 1 exact FP32
 * SIMT scan, 2 BF16 tcgen05 distance GEMM with a fused top-32 selection and
 * an FP32 re-rank, 3 the same GEMM with FP16 operands (power-of-two scaled;
 * 8x smaller rounding residual at the same tensor-core rate).  In modes 2
 * and 3, rows whose candidate set cannot be certified to contain the exact
 * FP32 k nearest are recomputed by the exact scan (over the spatial cells
 * each such row can reach), so every mode returns the same exact result;
 * these modes synchronise `stream` once, to read the number of such rows
 * (drgb_knn_uncertified reports it).
 * Errors: DRGB_ERR_INVALID if n < k + 1, k < 1, k > DRGB_MAX_K, d < 1,
 * a pointer is NULL or X is not 4-byte aligned. */
int drgb_knn_graph(drgb_ctx* ctx, const float* X, int64_t n, int32_t d, int32_t k,
                   int32_t mode, int32_t* idx_out, float* dist_out, void* stream);

/* Number of rows whose 16-bit candidate set was not certified during the last
 * tensor-core (mode 2 or 3) drgb_knn_graph call on `ctx` (synchronous: waits
 * for that call). */
int drgb_knn_uncertified(drgb_ctx* ctx, int64_t* count, void* stream);

/* Work of the last tensor-core drgb_knn_graph call on `ctx`: the number of
 * (128-row block, 256-column tile) products the distance GEMM computed, and
 * the number a full scan would compute; blocks skip the tiles of cells that
 * their distance bound rules out (synchronous). */
int drgb_knn_tiles(drgb_ctx* ctx, int64_t* done, int64_t* total, void* stream);

/* Approximate k-NN graph by NNDescent (Section 2.2: k random neighbours per
 * point, refined by exploring neighbours of neighbours with a top-k
 * selection, stopped once the update rate falls below delta = 0.015).  The
 * iteration is synchronous, so the graph is a pure function of X, k, seed,
 * delta and max_iter:
 *   start      point i takes the words of Philox4x32-10 (key = seed, counter
 *              (i, r, 0, 5), r = 0..15, words in order); a word u proposes
 *              floor(u n / 2^32), accepted when it is not i and not yet in the
 *              list, until k are accepted (then the smallest unused indices);
 *   iteration  the candidates of i are its list and the lists of its
 *              members, without i; its new list is the k candidates of
 *              smallest (squared FP32 distance sum_j (x_cj - x_ij)^2, index);
 *   reverse    0: that candidate set (the paper's wording); 1 (k <= 16): the
 *              basic algorithm of Dong et al., which Section 2.2 cites: R(i)
 *              = up to k of the points whose lists hold i, the k of smallest
 *              (squared distance, index), and the candidates of i are its
 *              general neighbours B(i) = list + R(i) and B(u) for each u in
 *              B(i), without i;
 *   stop       after the first iteration in which (new neighbours entering
 *              the lists) / (n k) < delta, or after max_iter iterations.
 *   X          n x d FP32 row-major (device), 1 <= d <= 1024
 *   idx_out    n x k int32, dist_out n x k FP32 Euclidean (device,
 *              caller-owned), each row in (distance, index) order
 *   iterations NULL, or host int: the iterations run
 *   rates      NULL, or host array of max_iter doubles: each iteration's
 *              update rate
 * Scratch: 12 n k bytes in the context's (about 24 n k more with reverse).
 * Synchronous (one synchronisation per iteration to read its update count).
 * Errors: as drgb_knn_graph, plus DRGB_ERR_INVALID for delta outside [0, 1],
 * max_iter outside 1..1000, d > 1024 or reverse with k > 16;
 * DRGB_ERR_NONFINITE if X holds NaN/Inf. */
int drgb_knn_nndescent(drgb_ctx* ctx, const float* X, int64_t n, int32_t d, int32_t k, uint64_t seed,
                       double delta, int32_t max_iter, int32_t reverse, int32_t* idx_out, float* dist_out,
                       int32_t* iterations, double* rates, void* stream);

/* -------------------------------------------------------- fuzzy weights */

/* Fuzzy simplicial-set graph of a k-NN graph (Section 3, the graph UMAP
 * builds; the construction is UMAP's, cited in Section 1):
 *   rho_i   = dist[i][0];
 *   sigma_i : sum_j exp(-max(0, dist[i][j] - rho_i) / sigma_i) = log2 k, by 64
 *             bisection steps (start 1, double until bracketed, then halve),
 *             floored at 1e-3 * mean_j dist[i][j];
 *   w_{j|i} = exp(-max(0, dist[i][j] - rho_i) / sigma_i);
 *   w_ij    = w_{j|i} + w_{i|j} - w_{j|i} w_{i|j} (fuzzy union).
 * Output is a CSR holding both (i,j) and (j,i), rows sorted by column, with
 * schedule words q = round(2^24 w / w_max); entries with n_epochs * q < 2^24
 * (never active in n_epochs epochs) are dropped.
 *   idx, dist  n x k (as produced by drgb_knn_graph; dist ascending per row;
 *              the k neighbours of a row distinct and other than the row).
 *   row_ptr    n + 1 int32 (row_ptr[n] = number of entries, written on device).
 *   col, w, q  capacity `cap` entries each (int32, FP32, uint32); cap >= 2 n k
 *              always suffices.
 *   rho, sigma optional n-float outputs (may be NULL).
 * Errors: DRGB_ERR_INVALID (bad sizes/pointers; malformed neighbour lists
 * are reported through the context's status word), DRGB_ERR_WORKSPACE if
 * cap < 2 n k. */
int drgb_fuzzy_weights(drgb_ctx* ctx, const int32_t* idx, const float* dist, int64_t n,
                       int32_t k, int32_t n_epochs, int32_t* row_ptr, int32_t* col, float* w,
                       uint32_t* q, int64_t cap, float* rho, float* sigma, void* stream);

/* Allocation-free variant of drgb_fuzzy_weights (the paper has no
 * counterpart).  For callers that cannot allocate device memory at all, for
 * example code that runs under an external memory manager which owns every
 * byte of the device, or in a setting where cudaMalloc is forbidden: it takes
 * no context and calls no cudaMalloc, cudaFree or allocating library routine.
 * Its scratch is a file-scope device array of DRGB_STATIC_SCRATCH_BYTES that
 * every GPU which loads the library holds until the process exits; inputs and
 * outputs are the caller's, exactly as for drgb_fuzzy_weights, and the result
 * is identical to it.
 *   - Sizes whose scratch would not fit the array (about 36 n k + 20 n bytes;
 *     n k up to roughly 440 000, e.g. n = 29 000 at k = 15) are rejected
 *     with DRGB_ERR_WORKSPACE before anything is enqueued.
 *   - The first call on each device, with that device current, looks up the
 *     array's device address (cudaGetSymbolAddress).
 *   - Every call shares the one array, which keeps the previous call's
 *     contents (each call clears what must start at zero): calls that overlap
 *     on the GPU, from two streams or two host threads, race.
 *   - Synchronous: returns after `stream` has finished the work, with
 *     DRGB_ERR_INVALID if the neighbour lists were malformed. */
#define DRGB_STATIC_SCRATCH_BYTES (16u << 20)
int drgb_fuzzy_weights_static(const int32_t* idx, const float* dist, int64_t n, int32_t k,
                              int32_t n_epochs, int32_t* row_ptr, int32_t* col, float* w,
                              uint32_t* q, int64_t cap, float* rho, float* sigma, void* stream);

/* ------------------------------------------------------------- a, b fit */

/* Host, synchronous.  Least-squares fit of Phi(x) = 1 / (1 + a x^(2b)) to
 * psi(x) = 1 (x < min_dist), exp(-(x - min_dist) / spread) otherwise, on 300
 * points in [0, 3 spread], by Gauss-Newton (Section 2.3 fits UMAP's output
 * kernel parameters this way).  FP64 internally.
 * Errors: DRGB_ERR_INVALID (NULL outputs, spread <= 0, min_dist < 0). */
int drgb_find_ab(float spread, float min_dist, float* a, float* b);

/* ----------------------------------------------------- initialisation */

/* Y0[i] = (u_x, u_y) * 2R - R with u = (Philox4x32-10 word >> 8) / 2^24 at
 * counter (i, 0, 0, 1), key = seed (low word, high word); one FP32 rounding.
 * Y is n x 2 FP32 (8-byte aligned).  Errors: DRGB_ERR_INVALID. */
int drgb_init_embedding(drgb_ctx* ctx, int64_t n, float init_range, uint64_t seed, float* Y,
                        void* stream);

/* Spectral initial layout (the UMAP optimisation the paper times in Section 3
 * starts from it): the two eigenvectors of the normalised adjacency
 * M = D^-1/2 W D^-1/2 of the fuzzy graph (W = the CSR's weights w, d_i their
 * row sums) with the largest eigenvalues after the trivial D^1/2 1
 * (eigenvalue 1), i.e. the smallest non-trivial ones of the normalised graph
 * Laplacian.  Each is signed so that its entry of largest magnitude (lowest
 * index among equal magnitudes) is positive, both are scaled by one factor
 * so that the largest |Y| is init_range, and each coordinate gets a jitter of
 * init_range * 1e-5 * (2u - 1), u from words 2, 3 of the initialisation
 * stream (Philox4x32-10, counter (i, 0, 0, 1), key = seed).
 *   row_ptr, col, w  the symmetric CSR graph (device, n + 1 / nnz entries)
 *   Y_out            n x 2 FP32 (device, 8-byte aligned)
 *   eigvals          optional host array of 3: the leading eigenvalues of M
 * Computed in FP32 by Chebyshev-filtered subspace iteration on 8 vectors
 * until the residual |M v - lambda v| of the three leading pairs is below
 * 1e-5, for at most 400 subspace steps, or until the worst residual has not
 * halved in 40 steps (then the current vectors are used: the leading
 * eigenvalues are too close to separate); on a disconnected graph eigenvalue
 * 1 repeats and the layout is some pair of vectors of its eigenspace.  Synchronous.  Errors: DRGB_ERR_INVALID
 * (NULL, misaligned, n < 9, init_range <= 0), DRGB_ERR_CUDA. */
int drgb_spectral_init(drgb_ctx* ctx, const int32_t* row_ptr, const int32_t* col, const float* w, int64_t n,
                       float init_range, uint64_t seed, float* Y_out, double* eigvals, void* stream);

/* PCA preprocessing to dim components (the paper's pipeline reduces the raw
 * features by PCA before the k-NN graph, Section 3; Section 3.3 names pca_dim):
 * mu = the column means of X, C = (X - mu)^T (X - mu) / (n - 1), V = the
 * eigenvectors of C for its dim largest eigenvalues in decreasing order, each
 * signed so that its entry of largest magnitude (lowest index among equal
 * magnitudes) is positive, and Z = (X - mu) V.
 *   X           n x D FP32 row-major (device), 1 <= D <= 1024, n >= 2
 *   dim         1 <= dim <= min(D, 56)
 *   Z           n x dim FP32 (device, caller-owned)
 *   components  NULL, or dim x D FP32 (device): V^T, one component per row
 *   mean        NULL, or D FP32 (device): mu
 *   eigvals     NULL, or host array of dim: the eigenvalues of C
 * C is formed on the tensor cores from a two-term BF16 split of X - mu (hi +
 * lo, about 16 significant bits): sym(hi hi^T) + hi lo^T + lo hi^T with FP32
 * accumulation over at most 2048 points per split, the splits summed in
 * float-float.  The eigenvectors come from Chebyshev-filtered subspace
 * iteration on 64 vectors, all on the device (FP32 products, float-float
 * Gram matrices, Cholesky QR with an FP64 factor, Rayleigh-Ritz by FP32
 * Jacobi); leading pairs whose residual |C v - theta v| is below
 * 1e-5 theta_1 are locked and deflated, until the dim leading pairs are
 * (at most 300 steps, or until the worst residual has not halved in 40: then
 * the current vectors, which span the leading eigenspace to that accuracy,
 * are used); Z is an FP32 product.  Scratch, in the context's: about
 * 4 n D' + n D'^2 / 256 bytes, D' = D rounded up to 128.  Synchronous.
 * Errors: DRGB_ERR_INVALID (NULL, misaligned, sizes), DRGB_ERR_CUDA. */
int drgb_pca(drgb_ctx* ctx, const float* X, int64_t n, int32_t D, int32_t dim, float* Z, float* components,
             float* mean, double* eigvals, void* stream);

/* ---------------------------------------------------------- SGD epoch */

/* One synchronous SGD epoch t over a head-sorted CSR (Section 2.5, the UMAP
 * optimiser step; Section 4.1, scatter-add on randomly sampled edges).  For every
 * row i and entry e = (i, j) active at t, i.e.
 *   floor((t+1) q_e / 2^24) > floor(t q_e / 2^24):
 *   d = |Y_i - Y_j|^2;  g_i += clip4(-2ab d^(b-1) / (1 + a d^b) (Y_i - Y_j)),
 *   (0 when d = 0); then for j' < neg: u = word (j' mod 4) of
 *   Philox4x32-10(key = seed, counter = (e, t, j' div 4, 0)), m = (u n) >> 32,
 *   skipped if m = i, d = |Y_i - Y_m|^2,
 *   g_i += clip4(2b / ((0.001 + d)(1 + a d^b)) (Y_i - Y_m)).
 * Y_out[i] = Y_in[i] + lr g_i.  All reads are from Y_in (Y^(t)); Y_out must
 * not alias Y_in.  No atomics.  The terms of a row are added in an order
 * fixed by the CSR alone (entry order within groups of 32 active entries of
 * 512-entry windows; see the epoch source), so the result does not depend on
 * the launch configuration.
 *   Y_in, Y_out  n x 2 FP32 (8-byte aligned);  row_ptr n+1, col, q as from
 *   drgb_fuzzy_weights (4-byte aligned).
 * Reads row_ptr[n] back to the host (one small synchronising copy on
 * `stream`) to size the context scratch; the epoch itself is asynchronous.
 * Errors: DRGB_ERR_INVALID (NULL/aliasing/misaligned pointers, n < 1,
 * neg < 0; a malformed CSR is reported by the next synchronising call);
 * DRGB_ERR_NONFINITE, reported by the next synchronising call, if Y_in holds
 * NaN or Inf (the epoch still runs; non-finite values spread through it). */
int drgb_embed_epoch(drgb_ctx* ctx, const float* Y_in, float* Y_out, const int32_t* row_ptr,
                     const int32_t* col, const uint32_t* q, int64_t n, float a, float b, float lr,
                     int32_t neg, int32_t epoch, uint64_t seed, void* stream);

/* Epochs t_begin .. t_end-1 of a T = n_epochs schedule, lr_t = lr0 (1 - t/T),
 * as one captured CUDA graph replayed on `stream`.  Y (n x 2) holds Y^(t_begin)
 * on entry and Y^(t_end) on return; Y_tmp (n x 2) is ping-pong scratch.
 * Because the schedule and the negatives are pure functions of (t, seed),
 * running [0, t1) then [t1, T) gives bit-identical results to [0, T).
 * Like drgb_embed_epoch it reads row_ptr[n] back first.
 * Errors: as drgb_embed_epoch (Y is scanned on entry), plus DRGB_ERR_INVALID
 * if 0 <= t_begin <= t_end <= n_epochs does not hold. */
int drgb_embed_epochs(drgb_ctx* ctx, float* Y, float* Y_tmp, const int32_t* row_ptr,
                      const int32_t* col, const uint32_t* q, int64_t n, float a, float b,
                      float lr0, int32_t neg, int32_t t_begin, int32_t t_end, int32_t n_epochs,
                      uint64_t seed, void* stream);

/* ----------------------------------------------------------- full fit */

/* fit_transform(X) -> Y (Section 2.1): with p->pca_dim > 0 and d > pca_dim,
 * PCA of X to pca_dim (as drgb_pca; d <= 1024) first; then k-NN graph, fuzzy
 * graph, a, b fit, initialisation and p->n_epochs epochs.  X is n x d FP32 on
 * the device, Y_out n x 2 FP32 on the device.  Synchronous (returns after
 * Y_out is written and the device status has been checked).  `cb` may be
 * NULL; when set it is called after every epoch (this costs one host sync per
 * epoch).  Errors: as the steps above; DRGB_ERR_NONFINITE if X, or the
 * returned embedding, holds NaN/Inf;
 * DRGB_ERR_INVALID for pca_dim outside 0..56.  drgb_fit_transform_batched and
 * drgb_transform take pca_dim = 0 only. */
int drgb_fit_transform(drgb_ctx* ctx, const float* X, int64_t n, int32_t d,
                       const drgb_params* p, float* Y_out, drgb_epoch_cb cb, void* user,
                       void* stream);

/* Batched form (a project addition; the paper embeds one data set at a
 * time): `count` independent instances embedded together.  Instance b is rows
 * offsets[b] .. offsets[b+1]-1 of X_cat ((sum n_b) x d FP32, device, 4-byte
 * aligned) and of Y_cat ((sum n_b) x 2 FP32, device).  `offsets` is a HOST
 * array of count + 1 int64 with offsets[0] = 0; seeds_init / seeds_neg are
 * optional HOST arrays of per-instance Philox keys (NULL: every instance uses
 * p->seed_init / p->seed_neg).  Each instance's k-NN graph is computed on its
 * own rows, the fuzzy graph of all instances is built in one pass, and each
 * of the p->n_epochs epochs is one force and one update launch over all rows
 * (the loop is one captured CUDA graph).  Instance b's result is bit-identical to
 * drgb_fit_transform of its rows alone with the same parameters and seeds.
 * Synchronous.  Errors: DRGB_ERR_INVALID (an instance with fewer than k + 1
 * rows, bad offsets or parameters), plus those of drgb_fit_transform. */
int drgb_fit_transform_batched(drgb_ctx* ctx, const float* X_cat, const int64_t* offsets,
                               int32_t count, int32_t d, const drgb_params* p,
                               const uint64_t* seeds_init, const uint64_t* seeds_neg, float* Y_cat,
                               void* stream);

/* Epoch autotuner: times every supported force-kernel setting (width 4 or 8
 * warps per CTA x form pipelined or flat, see drgb_set_tuning) for `trials`
 * epochs of the given graph on a scratch copy of Y (n x 2, device; not
 * modified), keeps the fastest in the context and returns it in choice[0]
 * (width) and choice[1] (form; choice[2] is set to 0) with its time per
 * epoch.  Every choice gives bit-identical results.  Synchronous. */
int drgb_autotune_epoch(drgb_ctx* ctx, const float* Y, const int32_t* row_ptr, const int32_t* col,
                        const uint32_t* q, int64_t n, float a, float b, int32_t neg, int32_t n_epochs,
                        uint64_t seed, int32_t trials, int32_t* choice, float* us_per_epoch,
                        void* stream);

/* ---------------------------------------------------- learned embedder */

/* Learned parametric form (a project addition; the paper has no learned
 * embedder): an MLP d -> 256 -> 256 -> 2 with exact-erf GELU, BF16 weights
 * and activations, FP32 accumulation (tcgen05 tensor cores) and FP32 master
 * weights, trained by Adam on the UMAP cross-entropy of the fuzzy graph's
 * edges (Section 2.5's loss, with Phi clamped to [1e-4, 1 - 1e-4]).
 * Parameters are one FP32 device vector of drgb_mlp_param_count() floats:
 * W1 [256][64] (input columns >= d stay 0), b1 [256], W2 [256][256], b2 [256],
 * W3 [2][256], b3 [2]; weights are (out, in) row-major. */
typedef struct drgb_mlp_params {
    int32_t steps;        /* optimiser steps */
    int32_t batch_edges;  /* edges per step (4096) */
    int32_t neg;          /* negatives per edge (5), 0..8 */
    float lr;             /* Adam learning rate (1e-3) */
    float beta1, beta2;   /* Adam moments (0.9, 0.999) */
    float eps;            /* Adam epsilon (1e-8) */
    uint64_t seed;        /* Philox key of edge and negative sampling */
} drgb_mlp_params;

int64_t drgb_mlp_param_count(void);

/* Initialise params (device, drgb_mlp_param_count floats): weights uniform in
 * +-1/sqrt(fan_in) from Philox under `seed`, biases 0.  Errors: d outside 1..64. */
int drgb_mlp_init(drgb_ctx* ctx, float* params, int32_t d, uint64_t seed, void* stream);

/* Sample one batch (test aid): for edge slot s, draw CSR entries e uniformly
 * (Philox4x32-10 at counter (step, s, try, 2), word 0 -> e = (u n_nz) >> 32)
 * and accept the first whose word 1 >> 8 is below q_e (so edges are drawn
 * proportional to q = 2^24 w; at most 64 tries); then rows[s R] = head(e),
 * rows[s R + 1] = col[e], rows[s R + 2 + t] = (u n) >> 32 with u = word
 * (t mod 4) at counter (step, s, 64 + t div 4, 2); R = 2 + neg.
 * rows: device int32 [n_edges R].  Synchronous. */
int drgb_mlp_sample(drgb_ctx* ctx, const int32_t* row_ptr, const int32_t* col, const uint32_t* q,
                    int64_t n, int64_t nnz, int32_t n_edges, int32_t neg, uint32_t step, uint64_t seed,
                    int32_t* rows, void* stream);

/* Gradient of the mean batch loss for explicit rows (device int32 [n_edges
 * (2 + neg)], layout as drgb_mlp_sample) of X (n x d FP32 device): writes
 * grad_out (device FP32, drgb_mlp_param_count) and, if loss_out (device
 * float) is given, the loss.  Synchronous. */
int drgb_mlp_grad(drgb_ctx* ctx, const float* params, const float* X, int64_t n, int32_t d,
                  const int32_t* rows, int32_t n_edges, int32_t neg, float a, float b, float* grad_out,
                  float* loss_out, void* stream);

/* mp->steps Adam steps on batches sampled as in drgb_mlp_sample (step s of
 * this call uses counter s) from the CSR (row_ptr, col, q; nnz entries) over
 * X (n x d).  params, adam_m, adam_v: device FP32 vectors updated in place
 * (zero the moments before the first call).  losses: device float[steps]
 * receiving each step's mean batch loss (nullable).  One step is captured as
 * a CUDA graph and replayed.  Synchronous. */
int drgb_mlp_train(drgb_ctx* ctx, const float* X, int64_t n, int32_t d, const int32_t* row_ptr,
                   const int32_t* col, const uint32_t* q, int64_t nnz, float a, float b,
                   const drgb_mlp_params* mp, float* params, float* adam_m, float* adam_v,
                   float* losses, void* stream);

/* Embed n new points: Y (n x 2 FP32, device) = MLP(X) for X (n x d FP32,
 * device), in chunks of 65536 rows on the tensor cores.  Asynchronous. */
int drgb_mlp_embed(drgb_ctx* ctx, const float* params, const float* X, int64_t n, int32_t d, float* Y,
                   void* stream);

/* Plain-optimisation embedding of new points against a fixed training
 * embedding (the fallback of the learned embedder and the judge of its
 * recall; the paper embeds only whole data sets).  X_train (n_train x d),
 * Y_train (n_train x 2), X_new (n_new x d): device FP32.  Each new point gets
 * its exact k nearest training points and their directed memberships (the
 * rho / sigma construction of drgb_fuzzy_weights), starts at the
 * membership-weighted mean of their training coordinates, then moves for
 * ceil(T/3) synchronous epochs (T = p->n_epochs, lr0 (1 - t/T'), negatives
 * from the training embedding, Philox key p->seed_neg) while Y_train stays
 * fixed.  Writes Y_new (n_new x 2).  Synchronous. */
int drgb_transform(drgb_ctx* ctx, const float* X_train, const float* Y_train, int64_t n_train,
                   const float* X_new, int64_t n_new, int32_t d, const drgb_params* p, float* Y_new,
                   void* stream);

/* Fill *p with the defaults (k 15, 200 epochs, neg 5, lr0 1, min_dist 0.1,
 * spread 1, init_range 10, seeds 1 and 2, knn_mode auto). */
int drgb_default_params(drgb_params* p);

/* -------------------------------------------------------- rendering */

/* Circle-splatting renderer (Section 2.4, the GPU rendering pipeline): every
 * point i adds, at each pixel whose centre lies at distance r < radius (in
 * pixels) from it, alpha * w and alpha * w * rgb_i with w = 1 - r / radius to
 * the pixel's alpha and colour accumulators (atomic scatter-add); the
 * resolve pass writes, where the accumulated alpha A > 0, the colour C / A
 * composited over the background with coverage min(1, A), and the background
 * elsewhere, each channel stored as round(255 * clamp(v, 0, 1)).
 *   Y          n x 2 FP32 embedding (device, 8-byte aligned)
 *   rgb        n x 3 FP32 colours in [0, 1] (device)
 *   width, height  frame size (at most 2^28 pixels); radius in (0, 64]
 *   alpha      opacity of one splat's centre (>= 0)
 *   background 3 floats (host)
 *   view_in    host (x0, y0, s): pixel px = (x - x0) s, py = (y - y0) s,
 *              pixel (u, v) centred at (u + 1/2, v + 1/2), row v growing with
 *              y; or NULL: fitted to the points' bounding box with a 5%
 *              margin on each side, the larger extent filling the frame,
 *              centred
 *   view_out   NULL, or host 3 floats receiving the view used (synchronises
 *              the stream)
 *   frame      height x width x 3 uint8, row-major (device, caller-owned)
 * The accumulator (16 bytes per pixel) lives in the context's scratch; the
 * order of the scatter-add is not fixed, so sums may differ between runs by
 * FP32 rounding.  Asynchronous unless view_out is given.  Errors:
 * DRGB_ERR_INVALID (NULL, sizes, radius, alpha, alignment, view scale <= 0). */
int drgb_render(drgb_ctx* ctx, const float* Y, const float* rgb, int64_t n, int32_t width, int32_t height,
                float radius, float alpha, const float* background, const float* view_in, float* view_out,
                uint8_t* frame, void* stream);

/* -------------------------------------------------------- evaluation */

/* k-NN preservation (kNN-P, Section 3.2): mean over the query rows of
 * |N_X(i) & N_Y(i)| / k, with exact neighbour sets in X (n x d, FP32 direct
 * distances) and in Y (n x 2).  Query rows: all rows if n_query <= 0 or
 * n_query >= n, else the evenly strided rows i_r = floor(r n / n_query),
 * r < n_query.  Synchronous; *out receives the value. */
int drgb_eval_recall(drgb_ctx* ctx, const float* X, const float* Y, int64_t n, int32_t d,
                     int32_t k, int64_t n_query, double* out, void* stream);

/* Trustworthiness (Section 3.2, Venna & Kaski 2006):
 * 1 - 2 / (m k (2n - 3k - 1)) sum_i sum_{j in N_Y(i) \ N_X(i)} (r_X(i,j) - k)
 * over the same query rows as drgb_eval_recall (m = number of rows), with
 * exact FP32 ranks.  Synchronous. */
int drgb_eval_trust(drgb_ctx* ctx, const float* X, const float* Y, int64_t n, int32_t d,
                    int32_t k, int64_t n_query, double* out, void* stream);

/* Held-out k-NN preservation, for embeddings of new points (the paper
 * evaluates training points only; this carries its kNN-P measure of Section
 * 3.2 over to points outside the training set): mean over the query new
 * points p of |N_X(p) & N_Y(p)| / k, where N_X(p) are the k nearest of the n
 * training points X_train (n x d) to X_new[p], and N_Y(p) the k nearest of
 * the training embedding Y_train (n x 2) to Y_new[p] (n_new x 2): for the
 * plain transform Y_train is the fitted embedding, for the learned embedder
 * its own image of the training set.  Exact FP32 scans, ties by index.
 * Query points: all if n_query <= 0 or n_query >= n_new, else the evenly
 * strided p_r = floor(r n_new / n_query).  Device pointers, caller-owned;
 * X rows 4-byte and Y rows 8-byte aligned.  Errors: DRGB_ERR_INVALID (NULL,
 * misaligned, k outside [1, DRGB_MAX_K], n < k, n_new < 1, d < 1).
 * Synchronous; *out receives the value. */
int drgb_eval_recall_heldout(drgb_ctx* ctx, const float* X_train, const float* Y_train, int64_t n,
                             const float* X_new, const float* Y_new, int64_t n_new, int32_t d,
                             int32_t k, int64_t n_query, double* out, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* DRGB_H */
