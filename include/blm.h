/*
 * blm.h -- C ABI of the GB300 library for one step of the blocked linear method (BLM) of
 * Zhao & Neuscamman, "A Blocked Linear Method for Optimizing Large Parameter Sets in
 * Variational Monte Carlo" (arXiv:1702.01481).
 *
 * One step, in call order (Sec. II.B):
 *   blm_accumulate      per sample chunk: Monte Carlo sums of Eq. 3 for every block's
 *                       self-plus-tangent space (Eq. 5; with history directions, Eq. 9-10)
 *   blm_block_solve     per block: generalized eigenproblem, keep the N_K lowest directions
 *                       as the rows of B^(b)
 *   blm_project         per sample chunk, the SAME samples again ("re-run the same sample"):
 *                       project onto the retained directions and accumulate Eq. 7's sums
 *   blm_combined_solve  lowest eigenpair of Eq. 7, update of Eq. 8, predicted energy
 *
 * Inputs per sample s (row s of each array, parameters contiguous, row stride `ld` elements):
 *   O[s, x]   = <n_s|Psi^x>/<n_s|Psi>          log-derivative ratio of parameter x
 *   dEL[s, x] = d E_L(n_s) / d mu_x            derivative of the local energy
 *   EL[s]     = <n_s|H|Psi>/<n_s|Psi>          local energy
 *   w[s]      = |<n_s|Psi>|^2 / P(n_s)         weight (NULL means 1, i.e. P = |Psi|^2)
 * The Hamiltonian ratio of Eq. 3 is <n|H|Psi^x>/<n|Psi> = EL * O_x + dEL_x.
 *
 * Conventions
 *   - Sample arrays may be device memory or host memory (pinned or pageable); host arrays are
 *     copied in pieces of up to 32768 samples through the handle's two staging buffers
 *     (allocated on the handle's first host-memory call), the copies on a stream of their own
 *     overlapping the computation on the previous piece (see also blm_set_host_cache).
 *     Element type per blm_problem.input_type.
 *   - All calls are asynchronous on the handle's stream; results are valid once it syncs.
 *   - The handle owns every accumulator and workspace it needs (allocated in blm_create; the
 *     host staging buffers on its first host-memory call).
 *   - Call order is enforced: accumulate+ -> block_solve -> project+ -> combined_solve;
 *     a call out of order returns BLM_ERR_STATE and changes nothing.
 *   - Numeric failures (non-finite sums, overlap not positive definite, no real lowest
 *     eigenvalue, alpha ~ 0) return BLM_ERR_NUMERIC from the solve that meets them;
 *     blm_last_error() gives a one-line reason.
 *   - Device waits inside the library are bounded: a wait that runs out returns
 *     BLM_ERR_TIMEOUT instead of hanging.
 */
#ifndef BLM_H
#define BLM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  BLM_OK = 0,
  BLM_ERR_ARG = 1,          /* invalid argument (sizes, pointers, offsets)               */
  BLM_ERR_STATE = 2,        /* call out of order                                          */
  BLM_ERR_NUMERIC = 3,      /* see blm_last_error()                                       */
  BLM_ERR_NOMEM = 4,        /* device allocation failed                                   */
  BLM_ERR_CUDA = 5,         /* a CUDA call failed (message in blm_last_error())           */
  BLM_ERR_TIMEOUT = 6,      /* a bounded device wait ran out                              */
  BLM_ERR_UNSUPPORTED = 7   /* valid but not implemented combination                      */
} blm_status;

typedef enum {
  BLM_PREC_F64 = 0,    /* sample contractions in FP64 on CUDA cores                         */
  BLM_PREC_BF16X4 = 1, /* sample contractions on tcgen05 tensor cores: each operand split into
                          bf16 hi + lo (2^-16 relative), the four products hi*hi + hi*lo +
                          lo*hi + lo*lo accumulated in FP32 (TMEM), promoted to FP64;
                          centring and eigen-solves stay FP64                                */
  BLM_PREC_TF32X4 = 2  /* the same four products on kind::tf32 with a finer lo: hi = the value
                          rounded to 8 significant bits, lo = tf32(v - hi) (11 bits), so hi + lo
                          represents v to 2^-21 (8x the BF16 split's resolution) at twice the
                          tensor-core cost                                                      */
} blm_precision;

/* Element type of the sample arrays.  The tensor-core precisions take FP32 samples; the FP64
 * path takes either (FP32 values are widened to FP64 on load). */
typedef enum { BLM_IN_F64 = 0, BLM_IN_F32 = 1 } blm_input_type;

typedef struct {
  int64_t n_params;               /* N_V                                                     */
  int32_t n_blocks;               /* N_B                                                     */
  const int64_t* block_offsets;   /* host, n_blocks+1 increasing, [0] = 0, [N_B] = N_V;
                                     block b is parameters [off[b], off[b+1]) (contiguous)   */
  int32_t n_keep;                 /* N_K: directions kept per block (min(N_K, M_b) used)     */
  int32_t n_old;                  /* N_O: previous-update directions (Eq. 9), 0 = none; 0..16
                                     (every precision: on the split paths their projections
                                     and sums are tensor-core tiles of the first sweep)      */
  const double* old_dirs;         /* host or device, n_old x n_params row-major: row j is the
                                     overall update of iteration n-j (Sec. II.B); block k's
                                     slice of row j is D_jk.  Copied at blm_create.          */
  int32_t precision;              /* blm_precision                                           */
  int32_t input_type;             /* blm_input_type                                          */
  double shift;                   /* diagonal shift of Sec. II.A on the tangent space (>= 0) */
  int64_t pass_samples;           /* samples per internal pass of a sweep (0 = 65536): the
                                     operand and projection scratch are sized for it (split
                                     precisions: 12 (BF16X4) or 24 (TF32X4) bytes per parameter
                                     and sample); a multiple of 1024 in 1024 .. 2^20          */
} blm_problem;

typedef struct blm_handle blm_handle;

/* Sec. II.B.  Validates the problem, allocates the handle's device memory on the current
 * device and binds the handle to `stream` (a cudaStream_t; NULL = legacy default stream).
 * Returns BLM_ERR_ARG for invalid sizes/offsets, BLM_ERR_NOMEM if allocation fails.
 * On failure *out is NULL. */
blm_status blm_create(const blm_problem* problem, void* stream, blm_handle** out);

/* Sec. II.A Eq. 3 and Sec. II.B Eq. 5/10, first sweep.  Adds one chunk of n_samples samples
 * to every block's sums.  O and dEL are n_samples x ld (ld >= n_params), EL and w length
 * n_samples, all of the problem's input type; w may be NULL.  The first call also fixes the
 * per-parameter reference shift used for centring (the chunk's mean of O).  n_samples == 0 is
 * a no-op.  Chunks may have any sizes. */
blm_status blm_accumulate(blm_handle* h, const void* O, const void* dEL, const void* EL,
                          const void* w, int64_t n_samples, int64_t ld);

/* Sec. II.B Eq. 5 / Eq. 10.  Builds every block's overlap and Hamiltonian from the sums (mean
 * centring in FP64), solves each generalized eigenproblem and keeps the min(N_K, M_b) lowest
 * directions (smallest real part; a complex pair gives its real and imaginary parts) as the
 * rows of B^(b), each of unit 2-norm with its largest-magnitude entry positive.
 * BLM_ERR_STATE before any accumulate; BLM_ERR_NUMERIC if a block's overlap is not positive
 * definite or its sums are not finite. */
blm_status blm_block_solve(blm_handle* h);

/* Sec. II.B, second sweep over the same samples (Eq. 6-7 matrices).  Same argument rules as
 * blm_accumulate.  The chunks must be the ones given to blm_accumulate (any order). */
blm_status blm_project(blm_handle* h, const void* O, const void* dEL, const void* EL,
                       const void* w, int64_t n_samples, int64_t ld);

/* Sec. II.B Eq. 7-8.  Solves the combined problem of dimension 1 + sum_b min(N_K, M_b), takes
 * its lowest eigenpair (c_0, A) and writes Delta mu_{i,b} = sum_j A_bj B^(b)_ji / alpha into
 * dmu (device or host, n_params doubles) and the eigenvalue (the predicted energy) into
 * *e_pred (host).  alpha is the coefficient of the raw Psi, c_0 - sum_bj A_bj (B^(b)_j . <O_b>).
 * Synchronises the handle's stream.  BLM_ERR_NUMERIC if the lowest eigenvalue is complex or
 * alpha ~ 0. */
blm_status blm_combined_solve(blm_handle* h, double* dmu, double* e_pred);

/* One whole step as a CUDA graph (Sec. II.B's step: both sweeps and both solves; the graph is
 * an execution device with no counterpart in the paper).  blm_graph_capture records, on a
 * stream of the handle's own, the step over the device sample arrays O, dEL (n_samples x ld),
 * EL and w (NULL = unit weights) taken in chunks of `chunk` samples -- reset, blm_accumulate per
 * chunk, blm_block_solve, blm_project per chunk, blm_combined_solve with Delta mu written to
 * the device array dmu (n_params doubles) -- with no host synchronisation inside (statuses
 * stay on the device; Davidson's dense fallback is decided on the device).  Nothing runs at
 * capture.  blm_graph_launch enqueues the captured step on the handle's stream; it reads
 * whatever the arrays hold at that time, so a sampler can refill the same buffers between
 * launches.  blm_graph_result synchronises the stream and reports the launched step as the
 * eager calls would (BLM_ERR_TIMEOUT, BLM_ERR_NUMERIC with blm_last_error) and its predicted
 * energy; blm_get_block / blm_get_combined then read its matrices.  The graph and the eager
 * calls share the handle's buffers: do not interleave them within a step.  All pointers must be
 * device memory (BLM_ERR_ARG otherwise); a new capture replaces the previous graph. */
blm_status blm_graph_capture(blm_handle* h, const void* O, const void* dEL, const void* EL,
                             const void* w, int64_t n_samples, int64_t chunk, int64_t ld,
                             double* dmu);
blm_status blm_graph_launch(blm_handle* h);
blm_status blm_graph_result(blm_handle* h, double* e_pred);

/* Many independent optimisations in one graph (Sec. II.B: the block problems of a step are
 * independent of one another, and so are separate optimisations; the batch is an execution
 * device with no counterpart in the paper).  blm_batch_create makes one handle per problem
 * (each as blm_create would; NULL on failure) bound to `stream`.  blm_batch_capture records one
 * step of every problem, from the device arrays O[i], dEL[i], EL[i], w[i] (w or its entries may
 * be NULL) of n_samples[i] rows with stride ld[i], taken in chunks of `chunk` samples, with
 * Delta mu written to the device array dmu[i]: the problems' sweeps run on parallel branches of
 * the graph, the block eigen-solves of all problems in one launch (the largest block problems
 * on teams of CTAs, the rest taken one CTA at a time from a shared queue), the dense combined
 * solves of all problems in one launch, larger
 * combined problems by Davidson one after another.  blm_batch_launch enqueues the graph on
 * `stream`; blm_batch_result synchronises it and writes every problem's predicted energy
 * (NaN where it failed) and, if status is not NULL, its blm_status; it returns BLM_OK if every
 * problem succeeded, else the first failure (message in blm_batch_last_error).
 * blm_batch_handle(b, i) is problem i's handle, for blm_get_block / blm_get_combined (do not
 * destroy it); blm_batch_destroy frees everything. */
typedef struct blm_batch blm_batch;
blm_status blm_batch_create(const blm_problem* problems, int32_t count, void* stream,
                            blm_batch** out);
blm_status blm_batch_capture(blm_batch* b, const void* const* O, const void* const* dEL,
                             const void* const* EL, const void* const* w,
                             const int64_t* n_samples, const int64_t* ld, int64_t chunk,
                             double* const* dmu);
blm_status blm_batch_launch(blm_batch* b);
blm_status blm_batch_result(blm_batch* b, double* e_pred, int32_t* status);
blm_handle* blm_batch_handle(blm_batch* b, int32_t i);
const char* blm_batch_last_error(const blm_batch* b);
blm_status blm_batch_destroy(blm_batch* b);

/* Tile autotuner for the split-precision sweeps (no counterpart in the paper).  Times the first
 * sweep's preparation and tensor-core contraction on the given device FP32 samples (at most one
 * pass, see blm_problem.pass_samples) for each candidate -- tile layout (one set of 128 x 256
 * tiles per block, or 128-row band tiles across the parameter range that keep only products
 * within a block, better for blocks much smaller than a tile) x the longest work unit (16384 or
 * 4096 samples) -- keeps the fastest for the handle and clears the sums (the step starts
 * afresh).  *choice (may be NULL) = 2 layout + unit index.  Synchronises the stream; no-op
 * (choice 0) on the FP64 path.  Results do not depend on the choice beyond the rounding of the
 * sums' accumulation order. */
blm_status blm_autotune(blm_handle* h, const void* O, const void* dEL, const void* EL,
                        const void* w, int64_t n_samples, int64_t ld, int32_t* choice);
/* Sets a candidate of blm_autotune directly (0 .. 3, e.g. one recorded from an earlier tuning);
 * takes effect from the next sweep.  Synchronises the stream; no-op on the FP64 path. */
blm_status blm_set_tiles(blm_handle* h, int32_t choice);

/* Read back block b's matrices (host, row-major (1+d_b)^2 with d_b = M_b + N_O (N_B - 1)),
 * its kept eigenvalues (host, min(N_K,M_b)) and B^(b) (host, min(N_K,M_b) x M_b).  Any output
 * pointer may be NULL.  Valid after blm_block_solve; synchronises the stream. */
blm_status blm_get_block(blm_handle* h, int32_t b, double* S, double* H, double* lambda,
                         double* B);

/* Combined matrices (host, row-major (1+N_K_total)^2), valid after blm_combined_solve. */
blm_status blm_get_combined(blm_handle* h, double* S, double* H);

/* Dimensions: block b's tangent dimension d_b, and the combined tangent dimension. */
int64_t blm_block_dim(const blm_handle* h, int32_t b);
int64_t blm_combined_dim(const blm_handle* h);

/* Clears all sums and solutions so that a new step can start with the same problem. */
blm_status blm_reset(blm_handle* h);

/* Frees the handle (NULL is a no-op). */
blm_status blm_destroy(blm_handle* h);

/* Last error message of the handle ("" if none); valid until the next call on it. */
const char* blm_last_error(const blm_handle* h);

/* Second sweep without a second host-to-device copy (Sec. II.B: the second sweep re-runs the
 * same samples).  Reserves `bytes` of device memory (0 releases it) in which blm_accumulate
 * keeps its device copies of host sample arrays, piece by piece while room remains; blm_project
 * given the same host arrays (same addresses, same chunking) then reads the kept copies instead
 * of copying the samples again.  Pieces that do not fit are copied in both sweeps as before.
 * blm_reset forgets the kept copies.  Synchronises the handle's stream; BLM_ERR_NOMEM if the
 * reservation fails.  Device sample arrays are never copied, with or without a cache. */
blm_status blm_set_host_cache(blm_handle* h, size_t bytes);

/* Failure detection (no counterpart in the paper).  Every wait of a tensor-core kernel on its
 * pipeline (operand stages, accumulator drains) polls an mbarrier at most `polls` times; then
 * the kernel records a timeout, waits for the copies and tensor-core operations it already
 * issued (those always complete), frees its tensor memory and returns, and the next solve on
 * the handle returns BLM_ERR_TIMEOUT (blm_reset clears it).  A handle starts with
 * BLM_WAIT_LIMIT_DEFAULT, far beyond any healthy wait.  polls = 0 makes every pipeline wait give
 * up at once: a deterministic way to run the timeout path, to test that the handle and the CUDA
 * context stay usable after it. */
#define BLM_WAIT_LIMIT_DEFAULT (1u << 24)
blm_status blm_set_wait_limit(blm_handle* h, uint32_t polls);

/* Profiling (no counterpart in the paper: measurement support).  While enabled, the handle
 * records a pair of CUDA events on its stream around each kernel it launches and counts the
 * launches, per kernel class.  blm_profile_read synchronises the stream and fills, for classes
 * 0 .. n-1 (n <= BLM_PROF_CLASSES), the summed device milliseconds and launch counts since the
 * last reset (enable != 0 also resets).  blm_profile_class_name(i) names class i. */
#define BLM_PROF_CLASSES 14
blm_status blm_profile(blm_handle* h, int enable);
blm_status blm_profile_read(blm_handle* h, int n, double* ms, int64_t* launches);
const char* blm_profile_class_name(int i);

/* Allocation-free solve of one block problem.  The paper has no counterpart: this is an
 * interface for callers that cannot allocate device memory when they need a block solved (a
 * VMC program that reserves the whole device at start-up and then forbids cudaMalloc, code that
 * must avoid the device-wide synchronisation cudaMalloc/cudaFree may imply, or a runtime that
 * only lends the library pointers it already owns).
 *
 * Same computation as blm_block_solve for a block without history directions: solves
 * H v = lambda S v (S, H: device, row-major dim x dim, the block's overlap and Hamiltonian
 * including row/column 0) and writes the n_keep lowest eigenvalues (real parts) into lambda
 * (device, n_keep) and the corresponding directions into B (device, n_keep x (dim - 1),
 * unit 2-norm, largest-magnitude entry positive), exactly as blm_get_block reports them.
 *
 * Workspace: a static device array inside the library (about 20.3 MB, held by every GPU that
 * loads the library until the process exits); nothing is allocated or freed.  Limits: 2 <= dim
 * <= blm_noalloc_max_dim() (257), 1 <= n_keep <= min(64, dim - 1); larger sizes return
 * BLM_ERR_ARG with a message on stderr.  The first call on each device looks up the array's
 * device address (cudaGetSymbolAddress) with that device current; make that first call before
 * any stream capture.  Every call shares the one array: calls that overlap on the GPU (other
 * streams, other threads) race and must be serialised by the caller.  Runs on `stream`, then
 * copies its status word to the host and synchronises `stream` before it returns;
 * BLM_ERR_NUMERIC if the overlap is not positive definite, the solve fails, or a kept direction
 * has a zero or non-finite norm. */
int32_t blm_noalloc_max_dim(void);
blm_status blm_block_solve_noalloc(const double* S, const double* H, int32_t dim, int32_t n_keep,
                                   double* lambda, double* B, void* stream);

/* Device bytes blm_create allocates for this problem (0 if the problem is invalid).  Host
 * function: needs no GPU. */
size_t blm_memory_estimate(const blm_problem* problem);

/* Storage of Sec. II.B's memory discussion, in bytes of 8-byte words: the traditional LM's
 * H and S, 2 (1 + N_V)^2, and the BLM's dominant terms (N_V^2/N_B + 2 N_V N_O (N_B - 1)
 * for H, N_V^2/N_B + N_V N_O (N_B - 1) for the symmetric S).  Host functions. */
double blm_lm_matrix_bytes(int64_t n_params);
double blm_matrix_bytes_dominant(int64_t n_params, int32_t n_blocks, int32_t n_old);

#ifdef __cplusplus
}
#endif
#endif /* BLM_H */
