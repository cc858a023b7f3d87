/*
 * tucker.h -- C ABI of libtucker: the HOOI hot path for sparse Tucker
 * decomposition (Chakaravarthy et al., "On Optimizing Distributed Tucker
 * Decomposition for Sparse Tensors", arXiv:1804.09494) on one NVIDIA GB300.
 *
 * Conventions shared by every call
 * --------------------------------
 *  - A tensor has N modes (2 <= N <= 6) of lengths L[0..N-1] and a core of
 *    size K[0..N-1], 1 <= K[n] <= min(L[n], 32) (Section 2.2: K_n <= L_n).
 *    Indices are 0-based (the paper is 1-based).
 *  - Khat_n = prod_{m != n} K[m] is the row length of the penultimate matrix
 *    Z_(n) (Section 2.2); it must be <= 4096.
 *  - Precision: a context is FP32 ("mixed": FP32 TTM-chain, Gram in split
 *    TF32 -- or split BF16 with TUCKER_BF16X3 -- on the tensor cores with FP64
 *    reductions, FP64 eigen-polish, Cholesky and reductions) or FP64 (plain
 *    FP64 everywhere).  Every "real" buffer below is float for FP32 and BF16X3
 *    contexts and double for FP64 contexts, except where double is stated.
 *  - Pointers prefixed d_ are device pointers, h_ are host pointers.  The
 *    caller owns every buffer it passes; the library owns its workspace.
 *  - Factor matrices F_m are L[m] x K[m], row-major, leading dimension K[m].
 *  - Z_(n) is returned *compact*: only the R_n non-empty slices (Section 3,
 *    "truncated local copy"), as an R_n x Khat_n row-major matrix whose row r
 *    belongs to slice d_row_id[r]; rows are in increasing slice id.  Columns
 *    follow Section 2.1 / Appendix A: the first remaining mode varies fastest.
 *  - The core G is prod K entries, first mode fastest.
 *  - Every call is asynchronous on `stream` (a cudaStream_t, NULL = legacy
 *    default stream) unless it says it synchronises.
 *  - Errors: a call returns TUCKER_OK or an error code; tucker_last_error()
 *    gives the message.  Arguments are checked on the host before anything is
 *    launched.  A device-side failure (e.g. a Cholesky breakdown) is latched
 *    in the context and returned by the next call that synchronises.
 */
#ifndef TUCKER_H
#define TUCKER_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct tucker_ctx* tucker_t;

typedef enum {
  TUCKER_OK = 0,
  TUCKER_ERR_ARG = 1,      /* invalid argument (host-side validation)              */
  TUCKER_ERR_OOM = 2,      /* device allocation failed                             */
  TUCKER_ERR_CUDA = 3,     /* a CUDA runtime call failed                           */
  TUCKER_ERR_NUMERIC = 4,  /* numeric breakdown (Cholesky pivot <= 0, non-finite)  */
  TUCKER_ERR_TIMEOUT = 5,  /* a bounded device wait ran out (see tucker_opts.wait_cap) */
  TUCKER_ERR_STATE = 6,    /* call not valid for this context                      */
  TUCKER_ERR_INDEX = 7     /* an input coordinate lies outside [0, L[m])           */
} tucker_status;

/*
 * Precision of a context.  TUCKER_FP32 (= TUCKER_TF32X3): FP32 TTM-chain and
 * values, Gram W = Z^T Z on the tensor cores from z = hi + lo with hi the
 * TF32-truncated value (W = hi^T hi + hi^T lo + lo^T hi, FP32 accumulation,
 * FP64 reductions), FP64 eigen-polish and CholeskyQR2.  TUCKER_BF16X3: the same
 * with every value of Z as three BF16 terms z = b0 + b1 + b2 (round to nearest
 * each; the rest is O(2^-27 z)) and W from the six products down to order
 * 2^-18, at the BF16 MMA rate (twice TF32's, so the same time as the three TF32
 * products; the same accuracy class).  TUCKER_FP64: plain FP64 everywhere
 * (CUDA cores).
 */
typedef enum { TUCKER_FP32 = 0, TUCKER_FP64 = 1, TUCKER_BF16X3 = 2, TUCKER_TF32X3 = TUCKER_FP32 } tucker_prec;

/*
 * Device-memory callbacks.  alloc returns `bytes` bytes of device memory
 * (256-byte aligned) that stay valid until free is called on them, or NULL
 * when it cannot; it is called on the host thread of tucker_init (context
 * memory and init temporaries), of tucker_partition (a scan temporary) and of
 * ttm_chain_backward (the adjoint's workspace, on its first call).  `stream` is the stream of that call: the
 * library orders its own use of the memory on that stream and on internal
 * streams, and synchronises the device before calling free, so an allocator
 * that reuses freed memory on `stream` (a caching allocator) is safe.
 */
typedef void* (*tucker_alloc_fn)(size_t bytes, void* stream, void* user);
typedef void (*tucker_free_fn)(void* ptr, size_t bytes, void* stream, void* user);

typedef struct {
  int32_t prec;          /* tucker_prec                                                  */
  int32_t P_bins;        /* Lite bins per mode (one TTM-chain thread each); 0 = one per   *
                          * resident thread of the TTM-chain kernel on all SMs (from the  *
                          * device's SM count and occupancy), less one CTA, so that a     *
                          * one-CTA kernel of a concurrent factor update finds room       */
  int32_t gauss_seidel;  /* 0 = Fig. 1 as printed (every mode from the input factors),     *
                          * 1 = textbook HOOI (each mode sees the factors refined so far) */
  int32_t timing;        /* 1 = record CUDA events around every phase (tucker_timings)    */
  int32_t wait_cap;      /* polls allowed per device wait (the mbarrier waits of the       *
                          * tensor-core Gram and of the bulk-copy back-projection) before *
                          * the wait is abandoned with TUCKER_ERR_TIMEOUT; 0 = no poll    *
                          * limit (each wait is still bounded by ~4e9 clock cycles);      *
                          * -1 = abandon every such wait at once (fault injection: runs   *
                          * the timeout path -- copies and MMAs in flight are still       *
                          * awaited -- with no stuck wait)                                */
  int32_t ttm_path;      /* 0 = the tensor-core TTM-chain where it applies (4-mode FP32   *
                          * contexts with 32 <= K_a K_b <= 128, K_c <= 48, Khat >= 256,    *
                          * a < b < c the other modes; it keeps a second, block-padded     *
                          * copy of those modes' elements), 1 = CUDA cores only,          *
                          * 2 = CUDA cores, fiber-factored where the fiber mode is the     *
                          * second remaining mode (3-mode FP32 contexts, exact tiles:      *
                          * K_a x K_b of 10 x 10, 8 x 8, 16 x 16): each element adds       *
                          * val F_a into a fiber sum, F_b is gathered once per fiber      */
  tucker_alloc_fn alloc; /* NULL: the library calls cudaMalloc / cudaFree itself          */
  tucker_free_fn free;   /* must be non-NULL exactly when alloc is                        */
  void* alloc_user;      /* passed to alloc and free                                      */
  int32_t svd;           /* factor update: 0 = the exact leading subspace of Z (Gram       *
                          * W = Z^T Z, eigensolve, back-projection); 1 = the paper's      *
                          * route (Section 3 "SVD component", Section 7): a Lanczos        *
                          * bidiagonalisation of Z with m = min(2 K_n, Khat_n, R_n) steps  *
                          * from the all-ones start vector, full re-orthogonalisation,     *
                          * then the same back-projection (an approximation of the         *
                          * subspace; it keeps R_n x m FP64 Lanczos vectors per mode)      */
  int32_t reserved[3];   /* must be zero                                                  */
} tucker_opts;

/* Fills *opts with the defaults (FP32, automatic P, Jacobi reading, no timing,
 * cudaMalloc). */
void tucker_default_opts(tucker_opts* opts);

/*
 * tucker_init -- builds a context for one COO tensor (Section 3: the element
 * set E with coordinates (l_1..l_N) and values val(e)).
 *
 * For every mode n it runs the Lite distribution (Section 6.1, Fig. 7) with P
 * bins, one bin per TTM-chain thread: slice histogram, sort of the non-empty
 * slices by (cardinality, slice id), stage 1 round robin under the limit
 * ceil(nnz/P), stage 2 contiguous fill; and it stores a permuted copy of the
 * tensor grouped bin by bin ("multi-policy scheme", Section 3), so the
 * caller may free its COO arrays once this call returns.
 *   N, L, K  : host arrays as above.
 *   nnz      : number of elements, 1 <= nnz < 2^31; coordinates must be distinct.
 *   d_idx    : host array of N device pointers; d_idx[m] holds nnz int32 coordinates.
 *   d_val    : nnz values (float or double per opts->prec).
 *   opts     : NULL = defaults.
 * Every byte of device memory the context owns, and every temporary of this
 * call, comes from opts->alloc when it is set (cudaMalloc otherwise).
 * Synchronises `stream`.  Returns TUCKER_ERR_INDEX if a coordinate is out of
 * range, TUCKER_ERR_ARG for bad sizes or non-finite values, TUCKER_ERR_OOM if
 * the workspace does not fit.  On error *out is NULL.
 */
tucker_status tucker_init(tucker_t* out, int N, const int64_t* L, const int32_t* K, int64_t nnz,
                          const int32_t* const* d_idx, const void* d_val, const tucker_opts* opts,
                          void* stream);

/* Releases the context and all library-owned device memory (synchronises the
 * device, then returns the memory through opts->free or cudaFree). */
void tucker_destroy(tucker_t t);

/* Message of the last error on this context (or of the last failed init when t is NULL). */
const char* tucker_last_error(tucker_t t);

/*
 * tucker_scheme_metrics -- the Section 4.1 metrics along `mode` of one of the
 * prior distribution schemes the paper compares Lite with (Section 5),
 * computed on the device from the context's tensor, for P processors:
 *   scheme 1 = CoarseG: every slice whole; the slices in the random order
 *     d_pos[mode] (d_pos[mode][l] = position of slice l) are cut into
 *     contiguous blocks balanced by elements: the slice at position t, with
 *     H_t elements in the slices before it, goes to processor
 *     floor(P * H_t / nnz);
 *   scheme 2 = MediumG: a processor grid q_1 x ... x q_N = P (the prime
 *     factors of P, largest first, each to the mode with the largest L_m / q_m
 *     so far, the lowest mode on a tie) over the permuted indices d_pos[m][l];
 *     mode m's positions fall in range floor(x * q_m / L_m); cell
 *     (b_1, ..., b_N) is processor b_1 + q_1 (b_2 + q_2 (...)).
 * d_pos: N device pointers to int32 permutations of [0, L_m) (read: d_pos[mode]
 * for CoarseG, all for MediumG; an out-of-range entry, or for CoarseG a
 * position given twice, returns TUCKER_ERR_INDEX).  Outputs: E_max = max_p |E^p|, R_sum = sum_p R^p, R_max =
 * max_p R^p (R^p = distinct mode-`mode` slices among processor p's elements),
 * on the host (any may be NULL); d_E, d_R: optional device arrays of P int64
 * receiving E^p and R^p.  MediumG needs L_mode * P / q_mode <= 2^35 (a
 * presence bit map).  Temporary device memory comes from the context's
 * callbacks; synchronises `stream`.  The Lite metrics of the context's own
 * partition are tucker_stats.
 */
tucker_status tucker_scheme_metrics(tucker_t t, int mode, int scheme, int P, const int32_t* const* d_pos,
                                    int64_t* E_max, int64_t* R_sum, int64_t* R_max, int64_t* d_E, int64_t* d_R,
                                    void* stream);

/*
 * tucker_ttm_form -- which TTM-chain form mode `mode` uses (Section 3, eq. (1)):
 * *tensor_cores = 1 for the tensor-core form (tcgen05 MMAs over 8-element
 * blocks of a slice; see tucker_opts.ttm_path), 0 for the CUDA-core form;
 * *blocks = the 8-element blocks of that mode's padded copy (elements plus
 * padding, / 8), 0 for the CUDA-core form.  Either output may be NULL.
 * Host-only.
 */
tucker_status tucker_ttm_form(tucker_t t, int mode, int32_t* tensor_cores, int64_t* blocks);

/*
 * tucker_stats -- Section 4.1 metrics of the mode-n Lite partition and the
 * compact row count.  E_max = max_p |E_n^p|, R_sum = sum_p R_n^p,
 * R_max = max_p R_n^p, R_n = number of non-empty slices, P = bins.
 * Any output pointer may be NULL.  Host-only, does not touch the device.
 */
tucker_status tucker_stats(tucker_t t, int mode, int64_t* E_max, int64_t* R_sum, int64_t* R_max,
                           int64_t* R_n, int64_t* P);

/*
 * tucker_partition -- exports the mode-n partition for checking: bin p owns
 * the original element ids d_perm[d_bin_ptr[p] .. d_bin_ptr[p+1]), in the
 * order the Lite pseudocode assigns them (stage-1 slices in sorted order,
 * then stage-2 pieces; original COO order inside a slice).
 *   d_bin_ptr : P+1 int64 (device), d_perm : nnz int32 (device).
 */
tucker_status tucker_partition(tucker_t t, int mode, int64_t* d_bin_ptr, int32_t* d_perm, void* stream);

/*
 * tucker_partition_noalloc -- the same export as tucker_partition, for callers
 * that cannot allocate device memory while they run (their device memory is
 * all handed out by their own pool or caching allocator, or a device-wide
 * synchronising cudaMalloc/cudaFree is not acceptable where they call from).
 * The paper has no counterpart; it is a deployment convenience.
 *   - Allocates nothing: the only scratch (the prefix-scan block sums over the
 *     bin lengths) is a static 256 KiB device array that every GPU loading the
 *     library holds until exit.  It holds one FP64 block sum per 2048 bins
 *     (plus the sums of those sums), which limits a mode to 67,008,511 bins;
 *     larger partitions return TUCKER_ERR_ARG.
 *   - Host threads may make their first call on a device concurrently (the
 *     address lookup is serialised inside the library).
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current; make that first call
 *     before any stream capture.
 *   - Every call shares the array: calls that overlap on the GPU (other
 *     streams, other threads) race and must be serialised by the caller.
 *   - Asynchronous on `stream` (tucker_partition synchronises).
 */
tucker_status tucker_partition_noalloc(tucker_t t, int mode, int64_t* d_bin_ptr, int32_t* d_perm, void* stream);

/*
 * ttm_chain -- penultimate matrix Z_(n) = T x_{m != n} F_m^T (Fig. 1
 * "TTM-Chain") through the Kronecker reformulation of Section 3, eq. (1):
 * Z_(n)[l,:] = sum_{e in Slice_n^l} val(e) Kron_n(e), Kron_n as in Appendix A.
 *   d_F      : host array of N device pointers to the factors (entry `mode` unused, may be NULL).
 *   d_vals   : NULL = the tensor's own values; else nnz replacement values in
 *              original element order (used for differentiation w.r.t. values).
 *   d_Z      : output, R_n x Khat_n (compact, see above).
 *   d_row_id : output, R_n int32 slice ids (may be NULL).
 * Owned slices are summed by one thread each; slices Lite splits over bins
 * are summed by a fixed-order fix-up, so the result is deterministic.
 */
tucker_status ttm_chain(tucker_t t, int mode, const void* const* d_F, const void* d_vals, void* d_Z,
                        int32_t* d_row_id, void* stream);

/*
 * factor_update -- new factor F~_n = leading K_n left singular vectors of
 * Z_(n) (Fig. 1 "SVD"), computed as: Gram W = Z^T Z (FP64 result), top-K_n
 * eigenpairs of W, back-projection U = Z V Sigma^-1, CholeskyQR2 of U, column
 * signs fixed so that each column's entry of largest magnitude (lowest slice
 * id on a tie) is positive, rows of empty slices zero.
 *   d_Z     : R_n x Khat_n compact matrix as produced by ttm_chain for this mode.
 *   d_F_out : output, L[mode] x K[mode].
 *   d_sigma : output, K[mode] doubles (singular values, descending); may be NULL.
 * Latches TUCKER_ERR_NUMERIC if U is rank deficient (e.g. R_n < K_n).
 */
tucker_status factor_update(tucker_t t, int mode, const void* d_Z, void* d_F_out, double* d_sigma,
                            void* stream);

/*
 * core -- G = T x_1 F_1^T x_2 ... x_N F_N^T (Fig. 1 "New core"), computed as
 * F_n*^T Z_(n*) for the cheapest mode n*.  d_G: prod K values, first mode fastest.
 */
tucker_status core(tucker_t t, const void* const* d_F, void* d_G, void* stream);

/*
 * hooi_iter -- one invocation of the HOOI procedure (Fig. 1): for every mode
 * n, ttm_chain + factor_update, then the new core and the fit
 *   fit = 1 - sqrt(max(0, ||T||^2 - ||G||^2)) / ||T||   (orthonormal factors).
 * With opts.gauss_seidel = 0 every TTM-chain uses the input factors (Fig. 1 as
 * printed); otherwise mode n uses the factors already refined in this call.
 * In the first reading the factor update of each mode runs on a stream of the
 * context, ordered after that mode's TTM-chain on `stream` by an event, and
 * `stream` waits for all of them before the core is formed: to the caller the
 * call is ordered on `stream` like a single kernel.
 *   d_F   : host array of N device pointers, factors in (initial) and out (new).
 *   d_G   : output core, prod K values.
 *   h_fit : output fit (host double); may be NULL.  Synchronises when non-NULL.
 */
tucker_status hooi_iter(tucker_t t, void* const* d_F, void* d_G, double* h_fit, void* stream);

/*
 * ttm_chain_backward -- adjoint of ttm_chain.  For a cotangent dZ (R_n x
 * Khat_n, compact rows as produced by ttm_chain):
 *   dval(e)        = < dZ[row(l_n(e))], Kron_n(e) >
 *   dF_m[l_m(e),:] += w(e) * dZ[row(l_n(e))] contracted with every other Kronecker row
 * where w(e) is the tensor's value or d_vals[e].  The Kronecker rows are
 * recomputed, never stored.
 *   d_dF   : host array of N device pointers; entries are ACCUMULATED into
 *            (caller zeroes them); a NULL entry (and entry `mode`) is skipped.
 *   d_dval : output, nnz values in original element order; may be NULL.
 */
tucker_status ttm_chain_backward(tucker_t t, int mode, const void* const* d_F, const void* d_dZ,
                                 const void* d_vals, void* const* d_dF, void* d_dval, void* stream);

/*
 * tucker_timings -- with opts.timing = 1, accumulated device milliseconds and
 * launch counts per phase since the last reset, from CUDA events recorded on
 * the launching stream.  Phases: 0 TTM-chain kernel, 1 split-slice fix-up,
 * 2 Gram, 3 eigensolve, 4 back-projection + CholeskyQR2, 5 core + fit,
 * 6 adjoint, 7 other.  ms[8] and launches[8] (either may be NULL); reset != 0
 * clears the counters after reading.  Synchronises `stream`.
 */
tucker_status tucker_timings(tucker_t t, double* ms, int64_t* launches, int reset, void* stream);

/* Bytes of device memory owned by the context (for reporting). */
tucker_status tucker_memory(tucker_t t, int64_t* bytes);

#ifdef __cplusplus
}
#endif
#endif /* TUCKER_H */
