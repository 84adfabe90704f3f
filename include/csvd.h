/*
 * csvd -- incremental truncated SVD of horizontally concatenated matrices,
 * its tail-error estimate and bounds, and error-constrained clustering, on
 * one NVIDIA GB300 GPU (sm_103a).  C ABI: plain pointers and sizes only.
 *
 * Method: arXiv 2601.11626, "Concatenated Matrix SVD: Compression Bounds,
 * Incremental Approximation, and Error-Constrained Clustering".
 *
 * Conventions (all entry points):
 *   - A block A_j is row-major m x k: element (i, c) at ptr[i * ld + c],
 *     ld >= k, in DEVICE memory, dtype CSVD_F32 or CSVD_BF16.  Block memory is
 *     borrowed: it must stay valid until the work enqueued on the stream has
 *     finished.  A 16-byte-aligned ptr with ld a multiple of 8 (f32) or 16
 *     (bf16) lets the batched scorer stage tiles with bulk (TMA) copies;
 *     other layouts take a register-load path.
 *   - Work is enqueued on the caller's CUDA stream (cudaStream_t passed as
 *     void*, NULL = legacy default stream).  Calls documented as "syncs" wait
 *     for that stream before returning host values.
 *   - Errors are returned as csvd_status; no exception crosses the ABI.
 *     csvd_last_error() gives a thread-local message for the last failure.
 *     Device-side conditions (an iteration cap reached) set a status word that
 *     the next synchronising call returns.
 *   - State objects own their device memory.  Temporary workspace comes from
 *     the allocator installed with csvd_set_allocator (default: the CUDA
 *     stream-ordered pool, cudaMallocAsync / cudaFreeAsync).
 *
 * Notation (paper -> here): Q_t -> U (m x r_t, orthonormal), S_t = diag(s^2)
 * -> sigma (r_t values), Y = Q_t^T A -> P, residual R = A - Q_t Y, thin QR
 * R = Q_res B, core K = [[diag(sigma), P], [0, B]] (K K^T = S_{t+1}).
 */
#ifndef CSVD_H_
#define CSVD_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  CSVD_OK = 0,
  CSVD_ERR_ARG = 1,            /* invalid argument (NULL, negative size, bad enum) */
  CSVD_ERR_SHAPE = 2,          /* block row count differs from the state's m, or a size limit */
  CSVD_ERR_CUDA = 3,           /* a CUDA runtime call failed */
  CSVD_ERR_OOM = 4,            /* device allocation failed */
  CSVD_ERR_NOT_CONVERGED = 5,  /* an iterative core solver hit its sweep cap */
  CSVD_ERR_TIMEOUT = 6,        /* a bounded device-side wait gave up */
  CSVD_ERR_UNIMPLEMENTED = 7
} csvd_status;

typedef enum { CSVD_F32 = 0, CSVD_BF16 = 1 } csvd_dtype;

/* Arithmetic of the merge evaluation:
 *   CSVD_PLAIN_FP32 -- the step as the Lemma states it, all in FP32 SIMT:
 *     P = U^T A, R = A - U P with one re-orthogonalisation pass, Householder
 *     QR of R, one-sided Jacobi SVD of the core K.
 *   CSVD_MIXED -- the same quantities from one pass over A on the tensor
 *     cores: P = U^T A and A^T A (tf32 split operands hi + lo, three MMAs per
 *     product, FP32 accumulation; the diagonal of A^T A replaced by exact
 *     column energies), the core's eigenvalues from the Gram K^T K =
 *     [[S, diag(s) P],[P^T diag(s), A^T A]] by Householder tridiagonalisation
 *     and bisection; tails in FP64.  Cores whose estimated tail is too small
 *     for FP32 eigenvalues to resolve it (E~^2 below 2e-3 of the merged
 *     energy) are solved again in FP64 from the same Gram.
 *   CSVD_GRAM_FP32 -- the CSVD_MIXED route with the two products taken by
 *     FP32 SIMT GEMMs instead of the tensor cores (the plain-FP32 form of the
 *     same algorithm).  Blocks with k = 1 take the arrowhead core in both.
 * Basis commits (csvd_incr_append) always take the CSVD_PLAIN_FP32 step. */
typedef enum { CSVD_PLAIN_FP32 = 0, CSVD_MIXED = 1, CSVD_GRAM_FP32 = 2 } csvd_precision;

typedef enum { CSVD_ALG_WEYL = 1, CSVD_ALG_RESIDUAL = 2, CSVD_ALG_APPROX = 3 } csvd_algo;
typedef enum { CSVD_SORT_FROBENIUS = 0, CSVD_SORT_RESIDUAL = 1 } csvd_sort;

typedef struct {
  const void* ptr;  /* device pointer to element (0, 0) */
  int64_t k;        /* columns (block width n_i), 1 <= k */
  int64_t ld;       /* row pitch in elements, ld >= k */
  int32_t dtype;    /* csvd_dtype */
  int32_t reserved; /* must be 0 */
} csvd_block;

typedef struct csvd_state_s* csvd_state;

typedef void* (*csvd_alloc_fn)(size_t bytes, void* stream, void* ctx);
typedef void (*csvd_free_fn)(void* ptr, void* stream, void* ctx);

/* Install a device allocator for temporary workspace (e.g. a framework's
 * caching allocator); NULL, NULL restores the default stream-ordered pool.
 * Process-wide; not thread-safe against concurrent csvd calls. */
csvd_status csvd_set_allocator(csvd_alloc_fn alloc, csvd_free_fn free_, void* ctx);

/* Create an empty rank-r state for blocks with m rows (M_0 := 0, Thm. 2's
 * convention; Lemma 1 applied from the empty state gives the rank-r SVD of
 * the first block, Alg. 3 step 1).  1 <= r <= m <= 65536, r <= 1024.
 * The state owns U (m x r), sigma (r) and FP64 scalars on the device. */
csvd_status csvd_incr_init(csvd_state* out, int64_t m, int32_t r, int32_t precision,
                           void* cuda_stream);

/* Append one block (Lemma 1 + Cor. 3, Appendix B): projection, residual,
 * thin QR, core SVD, truncation back to rank min(r, r_t + k', m) with
 * k' = min(k, m - r_t), and the energy update sum_i ||A_i||_F^2.
 * Stream-ordered, asynchronous.  A->ptr must hold m rows. */
csvd_status csvd_incr_append(csvd_state s, const csvd_block* A);

/* Replace the state's contents (checkpoint / resume): basis U (m x rt,
 * row-major, device, leading dimension ldu, orthonormal columns), retained
 * singular values sigma_host (rt values, non-increasing, host), the energy
 * sum_i ||A_i||_F^2 and the accumulated discarded energy.  0 <= rt <= r.
 * A state saved with csvd_incr_basis, csvd_incr_sigma and csvd_tail_error
 * resumes exactly.  Syncs. */
csvd_status csvd_incr_load(csvd_state s, const float* U_dev, int64_t ldu, int32_t rt,
                           const float* sigma_host, double energy, double discarded);

/* Copy the retained singular values sigma~_1..r_eff (Cor. 3, item 2) to
 * host memory (at least r floats) and the current rank.  Syncs. */
csvd_status csvd_incr_sigma(csvd_state s, float* sigma_host, int32_t* r_eff);

/* Copy the current basis U (m x r_eff, row-major, leading dimension ldu)
 * into a caller-owned device buffer.  Stream-ordered. */
csvd_status csvd_incr_basis(csvd_state s, float* U_dev, int64_t ldu);

/* Plug-in estimate of Cor. 2, E~_r^2 = sum_i ||A_i||_F^2 - sum_{j<=r}
 * sigma~_j^2, and E~_r / ||M||_F.  tail_sq is the accumulated discarded
 * energy (equal in exact arithmetic, free of the subtraction's
 * cancellation); tail_sq_paper, if non-NULL, is the subtraction evaluated
 * in FP64; energy, if non-NULL, is ||M||_F^2.  Syncs. */
csvd_status csvd_tail_error(csvd_state s, double* tail_sq, double* tail_rel,
                            double* tail_sq_paper, double* energy);

/* Release the state.  Syncs its stream first. */
csvd_status csvd_incr_free(csvd_state s);

/* Batched merge evaluation (Alg. 3 step 3(a)-(e)): for every candidate i,
 * a tentative append of cands[i] to states[cand_state[i]] producing
 * sigma~ (first r_i = rank after the append values, row i of sigma_out with
 * leading dimension ld_sigma), E~^2 (tail_sq_out[i]) and the accept flag
 * accept_out[i] = (E~^2 <= eps^2 * (||M_C||^2 + ||A_i||^2)).  No state is
 * modified.  Outputs are DEVICE pointers (tail_paper_out may be NULL).
 * All states must share m and the stream of states[0] is used.
 * precision selects CSVD_PLAIN_FP32 or CSVD_MIXED. */
csvd_status csvd_score(const csvd_state* states, int32_t n_states, const int32_t* cand_state,
                       const csvd_block* cands, int32_t n, double eps, int32_t precision,
                       float* sigma_out, int64_t ld_sigma, double* tail_sq_out,
                       double* tail_paper_out, uint8_t* accept_out);

/* Prepared batched merge evaluation: the same evaluation as csvd_score
 * (same arguments and outputs, Alg. 3 step 3(a)-(e)), split into a set-up
 * that does all host work once -- argument checks, descriptors, tile lists,
 * TMA tensor maps, the workspace (from the installed allocator) and its
 * upload; it syncs the stream of states[0] before returning -- and
 * csvd_plan_launch, which only enqueues memsets and kernel launches.  The
 * plan keeps the device addresses of the states' bases, singular values
 * and energies, of the candidate blocks and of the outputs: while it lives
 * no state may be appended to, loaded or freed and every buffer must stay
 * allocated (their contents may change between launches: a launch reads
 * whatever the blocks hold when it runs).  The paper has no counterpart; it
 * serves repeated evaluation of fixed candidate sets and CUDA graphs.
 * Errors: as csvd_score (nothing is allocated on failure). */
typedef struct csvd_plan_s* csvd_plan;
csvd_status csvd_score_plan(const csvd_state* states, int32_t n_states, const int32_t* cand_state,
                            const csvd_block* cands, int32_t n, double eps, int32_t precision,
                            float* sigma_out, int64_t ld_sigma, double* tail_sq_out,
                            double* tail_paper_out, uint8_t* accept_out, csvd_plan* out);

/* Enqueue one evaluation of the plan on cuda_stream (NULL: the stream of
 * states[0] at set-up): memsets and kernel launches only, no allocation,
 * host copy or synchronisation, so the call can be captured into a CUDA
 * graph (after one launch outside the capture, which sets the kernels'
 * shared-memory limits).  Launches of one plan share its workspace: order
 * them on one stream.  Device-side failures (caps, bounded waits) are
 * recorded in the plan's status word, read by csvd_plan_status. */
csvd_status csvd_plan_launch(csvd_plan p, void* cuda_stream);

/* Synchronise cuda_stream (NULL: the set-up stream), then read and clear
 * the plan's status word: CSVD_ERR_NOT_CONVERGED, CSVD_ERR_TIMEOUT or
 * CSVD_ERR_SHAPE for failures recorded since the last read. */
csvd_status csvd_plan_status(csvd_plan p, void* cuda_stream);

/* Release the plan and its workspace (synchronises the device first). */
csvd_status csvd_plan_free(csvd_plan p);

/* Batched merge evaluation of one-column candidates (blocks of width 1,
 * the k = 1 regime of the evaluation section's dataset table) given as the
 * rows of one matrix: candidate j is the column a_j = Xt[j * ldx + i],
 * i < m (Xt: n x m row-major f32, DEVICE, ldx >= m), tentatively appended
 * to states[cand_state[j]] (cand_state: n entries on the HOST; NULL means
 * state 0).  Outputs as in csvd_score, indexed by j (DEVICE; tail_paper_out
 * and accept_out may be NULL).  Mixed form only: with k = 1 the Gram of the
 * core (Lemma 1) is the arrowhead [[diag(sigma^2), sigma * p], [., ||a||^2]]
 * with p = U^T a, whose top eigenvalues are found by bisection on its exact
 * inertia count.  Rows whose state has r_t > 128 take the general mixed
 * path.  Adjacent rows of one state share each read of its basis (up to
 * four at a time), so order the rows by state where possible.  The host
 * arrays may be reused on return; stream-ordered on the stream of
 * states[0]; no state is modified. */
csvd_status csvd_score_columns(const csvd_state* states, int32_t n_states,
                               const int32_t* cand_state, const float* Xt, int64_t ldx, int32_t n,
                               double eps, float* sigma_out, int64_t ld_sigma, double* tail_sq_out,
                               double* tail_paper_out, uint8_t* accept_out);

/* Streaming cluster assignment: the incremental setting named as future
 * work in the paper's discussion section, where matrices arrive one at a
 * time and each joins an existing cluster or starts a new one by its
 * predicted compression error.  The rule (the paper gives none): a pushed
 * block is scored against every open cluster in one batched evaluation
 * (csvd_score semantics: a tentative rank-r append, Lemma 1 and Cor. 3, and
 * the plug-in estimate of Cor. 2); a cluster accepts when
 * E~^2 <= eps^2 ||M_{C u block}||_F^2; among the accepting clusters the one
 * with the smallest E~^2 / ||M||_F^2 receives the block (ties to the lowest
 * index) and commits it; when none accepts, the block starts a new cluster.
 * Clusters are numbered in order of creation.  The stream owns its cluster
 * states; precision as in csvd_incr_init; stream-ordered work on
 * cuda_stream.  Errors: CSVD_ERR_ARG for bad sizes, eps < 0 or a bad
 * precision. */
typedef struct csvd_stream_s* csvd_stream;
csvd_status csvd_stream_init(csvd_stream* out, int64_t m, int32_t r, double eps,
                             int32_t precision, void* cuda_stream);

/* Assign one block (m x k, borrowed for the call).  Host outputs, any may be
 * NULL: the cluster index, and E~^2 (accumulated discarded energy) and
 * ||M_C||_F^2 of that cluster after the block joined.  Syncs. */
csvd_status csvd_stream_push(csvd_stream s, const csvd_block* block, int32_t* label_out,
                             double* tail_sq_out, double* energy_out);

/* Number of clusters so far. */
csvd_status csvd_stream_count(csvd_stream s, int32_t* n_clusters);

/* Cluster c's state (borrowed: valid until csvd_stream_free; read it with
 * csvd_incr_sigma / csvd_incr_basis / csvd_tail_error to export the
 * cluster's basis) and its number of blocks (either output may be NULL). */
csvd_status csvd_stream_cluster(csvd_stream s, int32_t c, csvd_state* state_out,
                                int32_t* n_blocks_out);

/* Release the stream and every cluster state it owns. */
csvd_status csvd_stream_free(csvd_stream s);

/* Host-side consistency checks of the library's launch planning, no GPU
 * needed: the tile placement of the eigen core for every launch class and
 * core size (tiles partitioned among global memory, shared memory and
 * TMEM within their capacities), its tile-list walk, the launch classes'
 * shared memory, the row grouping of csvd_score_columns and the grouping
 * of one-column candidates of csvd_score into CTAs.  Writes "ok"
 * or the first failure into msg (cap bytes, may be NULL); returns CSVD_OK
 * or CSVD_ERR_SHAPE. */
csvd_status csvd_selftest(char* msg, int64_t cap);

/* Bounds for blocks taken in the given order (Section 3):
 *   weyl_sq     Thm. 1: sum ||A_j||^2 - max_j sum_{i<=r} sigma_i^2(A_j)
 *   residual_sq Cor. 1: sum ||A_j||^2 - sum_{j<=r} mu_j^2, mu the singular
 *               values of the residuals against a full-span basis
 *   plugin_sq   Cor. 2 with a rank-r incremental state
 *   energy      sum ||A_j||^2
 * Host outputs (any may be NULL).  Syncs. */
csvd_status csvd_bounds(const csvd_block* blocks, int32_t n, int64_t m, int32_t r,
                        void* cuda_stream, double* weyl_sq, double* residual_sq,
                        double* plugin_sq, double* energy);

/* Error-constrained clustering, Algorithms 1-3 of Appendix E.  labels_out[j]
 * receives the cluster index of block j (clusters numbered in creation
 * order); cluster_est_sq_out (length n, may be NULL) receives each cluster's
 * certificate value (bound^2 or E~^2) at its index; energy_out likewise
 * ||M_C||^2; compression_ratio_out (may be NULL) the ratio of stored numbers
 * (Section 4).  Host outputs.  Syncs. */
csvd_status csvd_cluster(const csvd_block* blocks, int32_t n, int64_t m, int32_t r, double eps,
                         int32_t algo, int32_t sort_mode, int32_t precision, void* cuda_stream,
                         int32_t* labels_out, double* cluster_est_sq_out, double* energy_out,
                         double* compression_ratio_out);

/* Backward of E = sum_j ||(I - U U^T) A_j||_F^2 for a fixed basis U (m x r,
 * row-major, device, leading dimension ldu): dA_j = 2 g (I - U U^T) A_j
 * written to grads[j] (f32 blocks with their own ld).  With U the top-r left
 * singular vectors of the concatenation this is the gradient of the
 * Eckart-Young tail (Thm. 4), valid when sigma_r > sigma_{r+1}.
 * Stream-ordered. */
csvd_status csvd_tail_grad(const float* U, int64_t ldu, int64_t m, int32_t r,
                           const csvd_block* blocks, const csvd_block* grads, int32_t n,
                           double g, void* cuda_stream);

/* Eckart-Young tail energy of a basis (Thm. 4; the differentiable
 * objective of the spec extension): resid_sq[j] = ||(I - U U^T) A_j||_F^2
 * for every block (host array of n doubles), U m x r orthonormal (row-major,
 * device, ldu).  P_j = U^T A_j is formed by a GEMM; the residual is not
 * stored: its squares are summed tile by tile (exact squares, compensated
 * FP32 sums, FP64 totals).  f32 blocks.  Syncs. */
csvd_status csvd_tail_energy(const float* U, int64_t ldu, int64_t m, int32_t r,
                             const csvd_block* blocks, int32_t n, void* cuda_stream,
                             double* resid_sq);

/* Randomized range-finder tail estimate (the discussion section's sketching
 * variant of the estimator): Y = sum_i A_i Omega_i with the caller's test
 * matrices Omega_i (k_i x l, row-major, device, ld l; l = r + oversampling,
 * r <= l <= m), power_iters iterations Y <- M M^T Q (Q the left singular
 * basis of Y), U_r = the top-r left singular vectors of Y, and
 * *tail_sq = sum_i ||(I - U_r U_r^T) A_i||_F^2 -- the explicit residual of
 * a rank-r projection, hence never below the optimal E_r^2 (Thm. 4) for any
 * draw: a certified estimate.  U_out (m x r, device, ldu; may be NULL)
 * receives U_r.  f32 blocks.  Syncs. */
csvd_status csvd_randomized_tail(const csvd_block* blocks, const float* const* omegas, int32_t n,
                                 int64_t m, int32_t r, int32_t l, int32_t power_iters,
                                 void* cuda_stream, double* tail_sq, float* U_out, int64_t ldu);

/* Top-r left singular basis of the concatenation of n blocks: the
 * incremental estimator (Lemma 1, Cor. 3) at rank working_rank (>= r), then
 * `refine` sweeps of subspace iteration Y = M M^T U, each followed by taking
 * the left singular vectors of Y (a rank-r append) -- each sweep shrinks the
 * angle to the exact top-r subspace by (sigma_{r+1} / sigma_r)^2.  Writes
 * U_out (m x r_eff, row-major, device, ldu >= r), r_eff = min(r, rank).
 * Allocates its temporary states with cudaMalloc.  Syncs. */
csvd_status csvd_top_basis(const csvd_block* blocks, int32_t n, int64_t m, int32_t r,
                           int32_t working_rank, int32_t refine, void* cuda_stream, float* U_out,
                           int64_t ldu, int32_t* r_eff);

/* Y = sum_j A_j (A_j^T U) = M M^T U for the concatenation M of the blocks:
 * one sweep of subspace iteration, used to refine a basis U (m x r,
 * row-major, device, ldu) towards the top-r left singular subspace of M
 * before the tail gradient (the gradient formula needs the exact top-r
 * basis; each sweep shrinks the angle by sigma_{r+1}^2 / sigma_r^2).
 * Y is m x r row-major (device, ldy).  Stream-ordered. */
csvd_status csvd_gram_apply(const float* U, int64_t ldu, int64_t m, int32_t r,
                            const csvd_block* blocks, int32_t n, float* Y, int64_t ldy,
                            void* cuda_stream);

/* Final decomposition of one cluster (Section 2, problem formulation): with
 * the cluster's rank-r left basis U (m x r, orthonormal columns, row-major,
 * device, ldu) and singular values s (r floats, device) the cluster keeps
 * U~ = U diag(s) and, per block A_i (m x k_i), the coefficient block
 * V_i = A_i^T U diag(s)^-1 (k_i x r; columns with s_j = 0 are zero), so that
 * A^_i = U~ V_i^T = U U^T A_i.  With U, s the exact top-r SVD of the
 * concatenation, the stacked V has orthonormal columns.  Writes U~ to Ut_out
 * (m x r, row-major, device, ldut >= r; may be NULL), V_i to V_out[i]
 * (device pointers, row-major with leading dimension ldv >= r; V_out may be
 * NULL) and, on the host, resid_sq[i] = ||A_i - A^_i||_F^2 from the
 * explicit residual and energy[i] = ||A_i||_F^2 (FP64); the cluster's
 * relative reconstruction error (Section 4) is
 * sqrt(sum resid_sq / sum energy) and its storage r (m + sum k_i) numbers.
 * Blocks are f32.  Syncs. */
csvd_status csvd_reconstruct(const float* U, int64_t ldu, const float* s, int64_t m, int32_t r,
                             const csvd_block* blocks, int32_t n, float* Ut_out, int64_t ldut,
                             float* const* V_out, int64_t ldv, void* cuda_stream,
                             double* resid_sq, double* energy);

/* ||A_j||_F^2 of each block (Kahan-compensated FP32 partial sums, FP64
 * totals) into energy_host[0..n).  Syncs. */
csvd_status csvd_block_energy(const csvd_block* blocks, int32_t n, int64_t m, void* cuda_stream,
                              double* energy_host);

/* Allocation-free merge evaluation.  The paper has no counterpart: this is
 * a deployment variant of csvd_score (CSVD_MIXED) for one candidate A
 * against state s, for callers that cannot allocate device memory at the
 * call -- e.g. a process whose GPU memory is wholly owned by another
 * allocator, or a latency-bound loop that cannot afford cudaMalloc /
 * cudaFree and the device synchronisation they may imply.  Every
 * intermediate lives in one file-scope device array of 4 MiB that each GPU
 * loading the library holds until the process exits; no call allocates.
 * Limits: f32 block with 16-byte aligned rows (ptr % 16 == 0, ld % 4 == 0),
 * k <= 512, state rank r_t <= 128 and rank cap r divisible by 4, state
 * basis 16-byte aligned; larger sizes (or a basis or block that no TMA
 * tensor map can describe) return CSVD_ERR_SHAPE, a misaligned block
 * CSVD_ERR_ARG, before any launch.  The products always run on the tensor
 * cores (the CSVD_GRAM environment switch does not apply), and there is no
 * FP64 re-solve: a tail below 2e-3 of the merged energy keeps the FP32
 * core's absolute accuracy of a few u ||M||^2.  Outputs are device pointers as in
 * csvd_score (sigma_out: at least min(r, r_t + k) floats; tail_paper_out
 * and accept_out may be NULL).  The first call on a device looks up the
 * array's device address (cudaGetSymbolAddress) with that device current,
 * so make the first call before any stream capture.  All calls share the
 * array: calls that may run concurrently on the GPU (different streams
 * without ordering) race and must be serialised by the caller.
 * Stream-ordered on the state's stream. */
csvd_status csvd_score_one_noalloc(csvd_state s, const csvd_block* A, double eps, float* sigma_out,
                                   double* tail_sq_out, double* tail_paper_out,
                                   uint8_t* accept_out);

/* Tunable launch configuration of the mixed form's eigen core (set by the
 * autotuner, paper_2601_11626_gb300/tune.py; the paper has no
 * counterpart).  Cores of size n = r_t + k <= edge_small run in the small
 * launch class (4 warps, 4 CTAs per SM), n <= edge_medium in the medium one
 * (8 warps, 2 CTAs per SM), larger ones one CTA of 16 warps per SM.
 * Ranges: 64 <= edge_small <= 288, edge_small < edge_medium <= 480;
 * (-1, -1) restores the defaults (192, 320); out-of-range values return
 * CSVD_ERR_ARG and change nothing.  Process-wide; results change only at
 * the level of FP32 rounding (the order of the core's sums). */
csvd_status csvd_tune_set(int32_t edge_small, int32_t edge_medium);
csvd_status csvd_tune_get(int32_t* edge_small, int32_t* edge_medium);

/* Failure-path test hook (the paper has no counterpart).  Sets, for the
 * current device, the sweep cap of the one-sided Jacobi core
 * (jacobi_sweeps, default 40), the iteration cap of every bisection and
 * secular-root iteration (solver_iters, default 64; 128 for the FP64
 * re-solve) and the limit of the tensor-core Gram kernel's pipeline waits
 * in ns of device time (wait_ns, default 2e9; the drains after an abort
 * keep the default).  A negative value restores the default.  With
 * stall_gram = 1 the Gram kernel's MMA role first waits on a barrier that
 * nothing arrives at, so that its bounded wait runs out after wait_ns and
 * the kernel aborts cleanly (copies drained, TMEM freed); 0 restores normal
 * operation.  A cap that is hit surfaces as CSVD_ERR_NOT_CONVERGED, a wait
 * that gives up as CSVD_ERR_TIMEOUT, both at the next synchronising call on
 * the state whose status word the launch used; results of that call are not
 * meaningful.  Not thread-safe against concurrent launches. */
csvd_status csvd_debug_limits(int32_t jacobi_sweeps, int32_t solver_iters, int64_t wait_ns,
                              int32_t stall_gram);

/* Launch tracing.  csvd_launch_count: kernels launched by this library so
 * far in the process.  csvd_profile(1) clears and starts recording a pair of
 * CUDA events on the launch stream around every kernel launch, csvd_profile(0)
 * clears and stops; csvd_profile_report writes one line per kernel name,
 * "name launches total_ms", into buf (NUL-terminated, truncated to len) and
 * waits for the recorded events. */
int64_t csvd_launch_count(void);
csvd_status csvd_profile(int32_t enable);
csvd_status csvd_profile_report(char* buf, int64_t len);

/* Thread-local message describing the last non-OK status (never NULL). */
const char* csvd_last_error(void);

/* Library version string. */
const char* csvd_version(void);

#ifdef __cplusplus
}
#endif
#endif /* CSVD_H_ */
