/*
 * pasta.h -- C ABI of libpasta: COO MTTKRP, the sparse CP least-squares
 * loss and its gradient, CP-ALS, TTV/TTM and TEW-eq/TS on one NVIDIA GB300
 * (sm_103a).
 *
 * The operations follow arXiv:1902.03317 (PASTA, a sparse tensor benchmark
 * suite):
 *   - COO storage, Sec. 5.1: per stored entry one index per mode ("inds") and
 *     one value ("val"); 32-bit indices and FP32 values (Table 2 caption);
 *     indices are 0-based (the Sec. 5.1 example names entries (1,0,0) and
 *     (1,0,2)).
 *   - MTTKRP, Eq. (mttkrp-init) in Sec. 3.6 and Algorithm 6 in Sec. 5.2.6.
 *   - Sorting in mode order, Sec. 5.2.2 (Algorithm 2's preprocessing) and the
 *     mode-orientation discussion of Sec. 2.3.
 *   - Factor matrices U_k are I_k x R, stored row-major (element (i, r) at
 *     i*R + r): the footnote to Eq. (ttm) in Sec. 3.4 transposes Kolda's
 *     convention for row-major C storage, and Algorithm 6 indexes A(i*R + r).
 *   - The CP model (a sum of R rank-one terms, Sec. 2.2) fitted by gradient
 *     descent (Sec. 2.2 lists gradient-descent CPD); the loss is the
 *     least-squares objective over the stored entries.
 *   - CP-ALS, the ALS-based CPD of Sec. 2.2 (steps of the survey it cites).
 *   - TEW-eq and TS, Sec. 3.1/3.2 and Algorithms 1 and 3; TTV and TTM,
 *     Sec. 3.3/3.4 and Algorithms 4 and 5.
 *
 * General rules
 *   - Every call returns a pasta_status.  Nothing aborts, throws or traps; a
 *     CUDA runtime failure becomes PASTA_ERR_CUDA and its text is available
 *     from pasta_last_error() on the same host thread.
 *   - "d_" pointers are device pointers (cudaMalloc'ed or equivalent) on the
 *     current CUDA device; "h_"/unprefixed pointers are host pointers.
 *   - stream is a cudaStream_t passed as void* (NULL = legacy default stream).
 *     Compute calls enqueue work on it and return without synchronising;
 *     results are ready when the stream reaches that point.
 *   - Modes are 0-based: mode 0 is the paper's mode 1.
 *   - Limits: 2 <= order <= PASTA_MAX_ORDER, 1 <= R <= PASTA_MAX_RANK,
 *     nnz < 2^32 - 2^16, every dims[k] in [1, 2^32).
 *   - Factor element type is one pasta_dtype for all modes of a call.  FP32,
 *     BF16 and FP16 factors accumulate in FP32 and produce FP32 outputs; FP64
 *     factors accumulate in FP64 and produce FP64 outputs.
 *   - Fast path: R * sizeof(element) a multiple of 16 bytes and every factor
 *     and output pointer 16-byte aligned (row loads and vector atomics are
 *     16 bytes wide).  Otherwise a scalar path with the same results runs.
 */
#ifndef PASTA_H
#define PASTA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PASTA_MAX_ORDER 8
#define PASTA_MAX_RANK 256
#define PASTA_ALS_MAX_RANK 128
#define PASTA_VERSION 3

typedef struct pasta_coo_s *pasta_coo; /* opaque, owned by the library */

typedef enum {
    PASTA_OK = 0,
    PASTA_ERR_INVALID_ARG = 1,  /* a NULL/out-of-range argument or size */
    PASTA_ERR_ALIGNMENT = 2,    /* reserved; misaligned data takes the scalar path */
    PASTA_ERR_INDEX_OOB = 3,    /* an index >= dims[k] found at create time */
    PASTA_ERR_NONFINITE = 4,    /* a NaN/Inf value found at create time */
    PASTA_ERR_NOT_SORTED = 5,   /* the mode-sorted copy a call needs is missing */
    PASTA_ERR_NOMEM = 6,        /* device allocation failed */
    PASTA_ERR_CUDA = 7,         /* a CUDA runtime call failed (see pasta_last_error) */
    PASTA_ERR_UNSUPPORTED = 8,  /* a combination this build does not implement */
    PASTA_ERR_SINGULAR = 9      /* CP-ALS: a normal-equation matrix has no inverse */
} pasta_status;

typedef enum {
    PASTA_F32 = 0,
    PASTA_BF16 = 1,
    PASTA_F16 = 2,
    PASTA_F64 = 3
} pasta_dtype;

/* Flags for pasta_coo_create. */
#define PASTA_CREATE_DEFAULT 0u
/* Skip the bounds / finiteness scan (and its one host synchronisation). The
 * caller vouches that every index is < dims[k]; an out-of-range index is then
 * undefined behaviour of the compute calls. */
#define PASTA_CREATE_NO_VALIDATE 1u

/* Short constant text for a status code. */
const char *pasta_status_str(pasta_status s);

/* Detail of the last failing call on this host thread ("" if none). */
const char *pasta_last_error(void);

/* PASTA_VERSION of the loaded library. */
int pasta_version(void);

/*
 * pasta_coo_create -- copy a COO tensor (Sec. 5.1) into library-owned device
 * memory.
 *   out    receives the handle (set to NULL on failure)
 *   order  number of modes N
 *   dims   host array of N mode sizes
 *   nnz    number of stored entries (0 allowed)
 *   d_idx  host array of N pointers; d_idx[k][m] is entry m's index in mode k
 *          (uint32, nnz elements each; any alignment)
 *   d_val  pointer to nnz FP32 values
 *   flags  PASTA_CREATE_DEFAULT or PASTA_CREATE_NO_VALIDATE
 * Each input array may be device memory or host memory: it is copied with
 * cudaMemcpyAsync(..., cudaMemcpyDefault) on `stream`, so pinned host memory
 * goes straight into the handle's copy (no device staging buffer; read by a
 * kernel as pasta_memcpy does).  The input arrays are only read, and may be
 * freed once the stream has passed this call (pageable host memory: once the
 * call returns).  Storage order is kept ("creation order").  Unless
 * PASTA_CREATE_NO_VALIDATE is given, a device scan counts out-of-range indices
 * and non-finite values and this call waits for it: PASTA_ERR_INDEX_OOB /
 * PASTA_ERR_NONFINITE are returned and no handle is made.  Duplicated
 * coordinates are legal and stay separate entries.
 */
pasta_status pasta_coo_create(pasta_coo *out, int order, const uint64_t *dims, uint64_t nnz,
                              const uint32_t *const *d_idx, const float *d_val,
                              unsigned flags, void *stream);

/*
 * pasta_coo_create_sorted -- pasta_coo_create followed by
 * pasta_coo_sort_by_mode(mode), with the same arguments, result and errors,
 * but overlapped: for at least 2^22 entries in pinned host memory (every
 * array 16-byte aligned) whose sort key holds every index, the entries are
 * cut into parts (4 from 2^24 entries on, else 2); each part is sorted once
 * it has been copied in while the later parts are still being copied (on a
 * high-priority stream of the library's own, joined back to `stream`), and
 * the sorted parts are merged (stable, ties to the earlier part: the order
 * one sort gives).  Otherwise it runs the two calls.  The sort's scratch
 * grows to about 24 (2 parts) or 36 (4 parts) bytes per entry.
 * PASTA_ERR_INVALID_ARG also for mode outside [0, order).
 */
pasta_status pasta_coo_create_sorted(pasta_coo *out, int order, const uint64_t *dims, uint64_t nnz,
                                     const uint32_t *const *d_idx, const float *d_val, unsigned flags,
                                     int mode, void *stream);

/* Free the handle and every copy it owns (synchronises the device). NULL is a no-op. */
pasta_status pasta_coo_destroy(pasta_coo X);

/* Order, dims (host array of >= order entries, may be NULL) and nnz of X. */
pasta_status pasta_coo_info(pasta_coo X, int *order, uint64_t *dims, uint64_t *nnz);

/*
 * pasta_coo_sort_by_mode -- build (once) the copy of X sorted for mode
 * `mode` (Sec. 5.2.2 sorts lexicographically in mode order; Sec. 2.3 notes
 * that each iteration order wants its own copy).  The key is the coordinate
 * in cyclic mode order (mode, mode+1, ..., N-1, 0, ..., mode-1), each mode
 * taking ceil(log2(dims[k])) bits, truncated to its leading 64 bits; the sort
 * is stable, so entries with equal keys keep creation order.  The copy holds
 * sorted indices, values and the permutation perm (sorted position p holds
 * creation-order entry perm[p]).  When the key holds every index (the modes'
 * bits fit 64), the sort carries the values and leaves perm to be built on
 * first request (pasta_coo_view with d_perm, pasta_coo_copy_out with
 * d_perm_out), which sorts again.  In that case the copy of mode+1, when it
 * exists, is only re-sorted on the mode-`mode` field (it is ordered by the
 * other fields already), else the copy of mode-1 on every field but mode-1's;
 * so sorting the modes in the order 0, N-1, N-2, ..., 1 (pasta's Python
 * sort_all) costs the least.  The result is the same whichever copies exist.
 * A second call for the same mode is a no-op.
 * Temporary device memory (about 21 bytes per entry) is the handle's scratch
 * buffer: allocated on first use (cudaMalloc, which waits for the device),
 * reused by later sorts and CP-ALS sweeps on the handle, grown when a call
 * needs more, freed by pasta_coo_destroy.  Calls on one handle that use it
 * must be ordered (one stream, or synchronised between streams).
 */
pasta_status pasta_coo_sort_by_mode(pasta_coo X, int mode, void *stream);

/*
 * Read-only device views of one stored copy: mode in [0, N) is the
 * mode-sorted copy (PASTA_ERR_NOT_SORTED if absent), mode == -1 the creation
 * order copy (perm is then NULL).  d_idx receives N pointers.  The pointers
 * stay valid until pasta_coo_destroy.  Any output pointer may be NULL.  Asking
 * for d_perm of a copy whose permutation was left out builds it on the
 * legacy default stream and waits for it.
 */
pasta_status pasta_coo_view(pasta_coo X, int mode, const uint32_t **d_idx,
                            const float **d_val, const uint32_t **d_perm);

/*
 * Copy one stored copy (mode as for pasta_coo_view) into caller-owned device
 * buffers of nnz elements each: d_idx_out (host array of N device pointers,
 * uint32), d_val_out (FP32) and d_perm_out (uint32; must be NULL for mode -1).
 * Any output may be NULL to skip it.  Asynchronous on `stream`.
 */
pasta_status pasta_coo_copy_out(pasta_coo X, int mode, uint32_t *const *d_idx_out,
                                float *d_val_out, uint32_t *d_perm_out, void *stream);

/*
 * pasta_mttkrp -- mode-n MTTKRP, Eq. (mttkrp-init) / Algorithm 6:
 *     M(i, r) = sum_{m : i_n(m) = i} val(m) * prod_{k != n} U_k(i_k(m), r).
 *   d_U     host array of N device pointers to row-major dims[k] x R factors
 *           of element type u_dtype; d_U[mode] is not read (may be NULL)
 *   mode    output mode n; the mode-n sorted copy must exist
 *           (pasta_coo_sort_by_mode), else PASTA_ERR_NOT_SORTED
 *   d_M     device output, dims[mode] x R row-major, FP32 (FP64 when u_dtype
 *           is PASTA_F64); overwritten (zero-filled, then accumulated, as the
 *           paper's Algorithm 6 expects an initialised output)
 * Rows of M that no entry reaches are 0.  Summation order differs from the
 * sequential loop, so FP32 results match it to rounding, not bitwise.
 */
pasta_status pasta_mttkrp(pasta_coo X, const void *const *d_U, pasta_dtype u_dtype, int mode,
                          int R, void *d_M, void *stream);

/*
 * pasta_gather_probe -- diagnostic companion of pasta_mttkrp (not a paper
 * operation).  Streams the mode-`mode` sorted copy with the same kernel,
 * geometry and launch as pasta_mttkrp and gathers, for every stored entry,
 * the same N-1 factor rows, but neither multiplies them by the value nor
 * reduces them into output rows: each thread sums what it gathered and
 * writes that one float to d_sink.  Its time is the row-gather ceiling of
 * pasta_mttkrp on that tensor (the cost of the gathers alone, at the
 * kernel's own parallelism).
 *   d_U, u_dtype, mode, R  as for pasta_mttkrp
 *   d_sink     device buffer of sink_len floats (>= 256); the launch uses at
 *              most sink_len / 256 thread blocks; contents are meaningless
 * PASTA_ERR_UNSUPPORTED outside the streaming MTTKRP's cases (FP32/BF16/FP16
 * factors, order 2..5, R * sizeof(element) = 16 L with L a power of two,
 * 16-byte aligned factors and sink).  Asynchronous on `stream`.
 */
pasta_status pasta_gather_probe(pasta_coo X, const void *const *d_U, pasta_dtype u_dtype, int mode,
                                int R, float *d_sink, uint64_t sink_len, void *stream);

/*
 * pasta_cp_loss_fwd -- sparse CP least-squares loss over the stored entries:
 *     model(m) = sum_r prod_k U_k(i_k(m), r),   e(m) = val(m) - model(m),
 *     loss = 1/2 * sum_m e(m)^2.
 *   mode     which stored copy to stream: -1 = creation order, or a sorted
 *            mode (PASTA_ERR_NOT_SORTED if absent)
 *   d_loss   device FP64 scalar, overwritten; the sum is taken in FP64 in a
 *            fixed order (the same inputs and launch give the same bits)
 *   d_resid  optional device output of nnz residuals e(m) (FP32; FP64 when
 *            u_dtype is PASTA_F64), in the order of the streamed copy
 * Per-entry arithmetic is FP32 (FP64 for PASTA_F64 factors).
 */
pasta_status pasta_cp_loss_fwd(pasta_coo X, const void *const *d_U, pasta_dtype u_dtype, int R,
                               int mode, double *d_loss, void *d_resid, void *stream);

/*
 * pasta_cp_loss_bwd -- gradient of g * loss with respect to every factor, in
 * one pass over the stored entries:
 *     G_k(i, r) = -g * sum_{m : i_k(m) = i} e(m) * prod_{j != k} U_j(i_j(m), r)
 * (-g times the mode-k MTTKRP of the residual tensor).  e(m) is recomputed
 * from the factors.
 *   mode     -1: one pass over the creation-order copy, every gradient
 *            added with vector atomics;
 *            n in [0, N): one pass over the mode-n sorted copy, G_n reduced
 *            in registers along runs of equal index, the other modes with
 *            vector atomics;
 *            PASTA_BWD_PER_MODE (-2): N passes, pass k over the mode-k sorted
 *            copy computing only G_k by run reduction (no atomics on hot
 *            rows; every sorted copy must exist)
 *   d_gscale device FP64 scalar g (NULL means g = 1)
 *   d_G      host array of N device pointers to dims[k] x R row-major outputs,
 *            FP32 (FP64 for PASTA_F64 factors); all overwritten
 */
#define PASTA_BWD_PER_MODE (-2)

pasta_status pasta_cp_loss_bwd(pasta_coo X, const void *const *d_U, pasta_dtype u_dtype, int R,
                               int mode, const double *d_gscale, void *const *d_G, void *stream);

/*
 * pasta_cp_loss_fwd_noalloc -- the loss of pasta_cp_loss_fwd for callers that
 * cannot allocate device memory.  The paper has no counterpart: this is a
 * deployment variant of the same forward kernel.
 *
 * Who needs it: code that may not call cudaMalloc (or any allocating library
 * routine) where it computes the loss -- real-time or callback contexts,
 * processes whose device memory belongs to a different allocator.  pasta_coo_create copies
 * the tensor and keeps per-handle scratch, so it is not usable there; this
 * call reads the caller's own arrays and keeps its scratch (the FP64 partial
 * sums of the loss, one per thread block) in a fixed device array inside the
 * library, so it allocates nothing and needs no handle.
 *
 *   order, dims, nnz  as for pasta_coo_create (limits as there)
 *   d_idx             host array of order device pointers, uint32 indices in
 *                     creation order; each array 16-byte aligned and readable
 *                     up to nnz rounded up to a multiple of 4 entries (entries
 *                     past nnz are read but ignored)
 *   d_val             FP32 values, same alignment and readability rule
 *   d_U, u_dtype, R, d_loss, d_resid   as for pasta_cp_loss_fwd with mode -1
 * Indices are not validated: each must be < dims[k].
 * Errors: PASTA_ERR_INVALID_ARG for sizes outside the library limits (order,
 * dims, nnz, R) or NULL pointers, PASTA_ERR_ALIGNMENT for an input array that
 * is not 16-byte aligned.
 *
 * The scratch array holds PASTA_NOALLOC_MAX_PARTIALS doubles (32 KB); every
 * GPU that loads the library keeps it until the process exits.  Launches never
 * use more thread blocks than it holds (the kernel strides over any nnz with
 * that many blocks), and nothing in it has to start at zero.  All calls share
 * it: calls whose work overlaps on the GPU (for example on two streams at
 * once) race and give wrong losses; calls in sequence on one stream are safe.
 * Every call looks up the array's device address on the current device
 * (cudaGetSymbolAddress).  The first call on a device may load the library's
 * device code, which allocates, and so may the first call after
 * cudaDeviceReset (the array may then sit at a new address, which the lookup
 * finds); later calls allocate nothing.  So make the first call on each
 * device (and the first after a reset) before any stream capture begins.
 */
#define PASTA_NOALLOC_MAX_PARTIALS 4096

pasta_status pasta_cp_loss_fwd_noalloc(int order, const uint64_t *dims, uint64_t nnz,
                                       const uint32_t *const *d_idx, const float *d_val,
                                       const void *const *d_U, pasta_dtype u_dtype, int R,
                                       double *d_loss, void *d_resid, void *stream);

/*
 * pasta_cp_loss_fwd_bwd -- the loss of pasta_cp_loss_fwd and the gradients of
 * g * loss (pasta_cp_loss_bwd with PASTA_BWD_PER_MODE) in N passes instead of
 * N + 1: pass k streams the mode-k sorted copy and reduces G_k along runs,
 * and the first pass also sums the squared residuals.  Every sorted copy must
 * exist (else PASTA_ERR_NOT_SORTED).  For training steps that always need
 * both; the loss is summed in a fixed order (reproducible bits for the same
 * inputs and launch) but not necessarily in the same order as
 * pasta_cp_loss_fwd, so the two may differ in the last bits.
 *   d_loss    device FP64 scalar, overwritten
 *   d_gscale  device FP64 scalar g (NULL means g = 1)
 *   d_G       as for pasta_cp_loss_bwd
 */
pasta_status pasta_cp_loss_fwd_bwd(pasta_coo X, const void *const *d_U, pasta_dtype u_dtype,
                                   int R, double *d_loss, const double *d_gscale,
                                   void *const *d_G, void *stream);

/*
 * pasta_convert -- element-wise conversion of n values between pasta_dtypes
 * (round to nearest even on narrowing), e.g. FP32 gradient accumulators to
 * BF16 parameters.  Not a paper operation; it keeps the mixed-precision
 * backward on the device.
 */
pasta_status pasta_convert(const void *d_src, pasta_dtype src_dtype, void *d_dst,
                           pasta_dtype dst_dtype, uint64_t n, void *stream);

/*
 * pasta_convert_scaled -- as pasta_convert, with dst = scale * src, where
 * scale is the device FP64 scalar at d_scale (NULL means 1); e.g. applying
 * the incoming gradient of a loss to gradients computed for g = 1.  The
 * product is formed in FP32 for FP32/BF16/FP16 sources, in FP64 for FP64.
 * In place (d_dst == d_src) only when both types are equal; otherwise the two
 * buffers must not overlap.
 */
pasta_status pasta_convert_scaled(const void *d_src, pasta_dtype src_dtype, void *d_dst,
                                  pasta_dtype dst_dtype, uint64_t n, const double *d_scale,
                                  void *stream);

/*
 * pasta_cp_als_sweep -- one sweep of CP alternating least squares, the CPD
 * method whose bottleneck is MTTKRP (Sec. 2.2, the CPD paragraph; the steps
 * follow the Kolda-Bader survey the paper cites).  For n = 0, ..., N-1:
 *     M     = MTTKRP_n(X, U)                     (pasta_mttkrp, FP32)
 *     V     = Hadamard product over k != n of U_k^T U_k   (R x R, FP64)
 *     U_n   = M V^{-1}                           (V inverted in FP64)
 *     lam_r = || U_n(:, r) ||_2,  U_n(:, r) /= lam_r (a zero column stays 0)
 * and then, if d_fit is not NULL, the fit 1 - ||X - model|| / ||X|| of the
 * model sum_r lam_r U_0(:, r) o ... o U_{N-1}(:, r), from
 * ||X - model||^2 = ||X||^2 + ||model||^2 - 2 <X, model>, where ||X||^2 is
 * the sum of the squared stored values (stored entries are taken as distinct
 * coordinates; duplicates should be merged before calling for a
 * meaningful fit; the factors do not depend on this).
 *   d_U       host array of N device pointers to row-major dims[k] x R FP32
 *             factors, read and updated in place
 *   R         1..PASTA_ALS_MAX_RANK, else PASTA_ERR_UNSUPPORTED
 *   d_lambda  device output, R doubles: lam of the last mode
 *   d_fit     device output (one double) or NULL
 * Every mode-sorted copy must exist (PASTA_ERR_NOT_SORTED).  Scratch
 * (dims_max x R floats plus small R x R buffers) is the handle's scratch
 * buffer (see pasta_coo_sort_by_mode).
 * The call synchronises `stream` once, at its end, to read the solve status:
 * PASTA_ERR_SINGULAR when some V has a non-positive pivot (for example a
 * factor column that became zero); the factors then hold unspecified values.
 */
pasta_status pasta_cp_als_sweep(pasta_coo X, float *const *d_U, int R, double *d_lambda,
                                double *d_fit, void *stream);

/*
 * pasta_cp_als -- CP-ALS: up to max_sweeps sweeps as in pasta_cp_als_sweep,
 * stopping early once the fits of two consecutive sweeps differ by less than
 * tol (tol < 0: always max_sweeps).  Each factor's Gram matrix is formed once
 * from the factors as given and afterwards kept from the pass that
 * normalises it, so a sweep after the first skips N Gram passes.
 *   d_U, R, d_lambda  as for pasta_cp_als_sweep (d_lambda: the last sweep's)
 *   max_sweeps        >= 1
 *   h_fits            host array of max_sweeps doubles: the fit after each
 *                     sweep run (entries past *h_sweeps are left unwritten)
 *   h_sweeps          host output: sweeps completed
 * The call synchronises `stream` once per sweep (solve status and fit).  On
 * PASTA_ERR_SINGULAR, *h_sweeps sweeps completed before the failing one.
 * PASTA_ERR_INVALID_ARG for max_sweeps < 1, NULL h_fits / h_sweeps or a NaN
 * tol; otherwise the errors of pasta_cp_als_sweep.
 */
pasta_status pasta_cp_als(pasta_coo X, float *const *d_U, int R, int max_sweeps, double tol,
                          double *d_lambda, double *h_fits, int *h_sweeps, void *stream);

/* Element-wise operators of TEW-eq and TS (Sec. 3.1, 3.2). */
typedef enum {
    PASTA_OP_ADD = 0,
    PASTA_OP_SUB = 1,
    PASTA_OP_MUL = 2,
    PASTA_OP_DIV = 3
} pasta_op;

/*
 * pasta_tew_eq -- Z = X op Y for two tensors with exactly the same stored
 * coordinates in the same order (TEW-eq, Sec. 3.1 and Algorithm 1): every
 * stored value z_m = x_m op y_m, computed in FP32 with IEEE rounding (a
 * division by a stored zero gives Inf or NaN; Z is not validated).
 *   X, Y   same order, dims and nnz, else PASTA_ERR_INVALID_ARG; the
 *          creation-order coordinates are compared on the device (one pass,
 *          then one synchronisation of `stream`) and PASTA_ERR_INVALID_ARG is
 *          returned if any differs
 *   op     PASTA_OP_ADD / SUB / MUL / DIV
 *   Z      in/out: *Z == NULL makes a new handle (caller destroys it);
 *          otherwise *Z must be a handle of the same order, dims and nnz,
 *          neither X nor Y, and its creation-order copy is overwritten (its
 *          sorted copies and fiber tables are dropped)
 * Z holds only a creation-order copy: X's coordinates and the new values.
 */
pasta_status pasta_tew_eq(pasta_coo X, pasta_coo Y, pasta_op op, pasta_coo *Z, void *stream);

/*
 * pasta_ts -- Z = X op s for every stored value (TS, Sec. 3.2 and
 * Algorithm 3), in FP32 with s rounded to FP32 once.  Z as for
 * pasta_tew_eq (new, or a same-shaped handle that is neither X).  The paper
 * reduces subtraction and division to addition and multiplication by -s and
 * 1/s; here all four are computed directly (x / s is correctly rounded).
 */
pasta_status pasta_ts(pasta_coo X, pasta_op op, double s, pasta_coo *Z, void *stream);

/*
 * pasta_coo_fibers -- build (once) the mode-n fiber table, the preprocessing
 * of Algorithms 4 and 5 (Sec. 5.2: the number of mode-n fibers and where
 * each begins).  A mode-n fiber is the set of stored entries sharing every
 * index but i_n; each is a contiguous run of the mode-(n+1 mod N) sorted
 * copy, which must exist (else PASTA_ERR_NOT_SORTED), and the other modes'
 * index bits must fit its 64-bit key (else PASTA_ERR_UNSUPPORTED).  Fibers
 * are numbered in that copy's order: lexicographic in the modes n+1, ...,
 * N-1, 0, ..., n-1.  *nfibs (host, may be NULL) receives their number.
 * Synchronises `stream` once (to size the table).  Device memory: 4 bytes
 * per stored entry plus 4 (N-1) per fiber, freed by pasta_coo_destroy.
 */
pasta_status pasta_coo_fibers(pasta_coo X, int mode, uint64_t *nfibs, void *stream);

/* The fibers' coordinates: d_coords is a host array of N-1 device pointers
 * (nfibs uint32 each; NULL entries are skipped) for modes n+1, ..., n-1
 * (cyclic).  PASTA_ERR_NOT_SORTED without the fiber table.  Asynchronous. */
pasta_status pasta_coo_fiber_coords(pasta_coo X, int mode, uint32_t *const *d_coords, void *stream);

/*
 * pasta_ttm -- mode-n Tensor-Times-Matrix, Eq. (ttm) / Algorithm 5 with the
 * paper's transposed convention (U is dims[mode] x R, row-major):
 *     Y(f, r) = sum over the entries m of fiber f of val(m) * U(i_n(m), r).
 * d_Y: device, nfibs x R row-major, FP32 (FP64 when u_dtype is PASTA_F64),
 * overwritten (may be NULL when there are no fibers); row f is fiber f of
 * pasta_coo_fibers.  The fiber table must
 * exist (PASTA_ERR_NOT_SORTED).  Runs as an MTTKRP of the order-2 tensor
 * (fiber, i_n), so its accuracy and speed follow pasta_mttkrp's.
 */
pasta_status pasta_ttm(pasta_coo X, int mode, const void *d_U, pasta_dtype u_dtype, int R, void *d_Y,
                       void *stream);

/* pasta_ttv -- mode-n Tensor-Times-Vector, Algorithm 4: y(f) = sum over
 * fiber f of val(m) * v(i_n(m)); pasta_ttm with R = 1 (d_v has dims[mode]
 * elements, d_y nfibs). */
pasta_status pasta_ttv(pasta_coo X, int mode, const void *d_v, pasta_dtype v_dtype, void *d_y,
                       void *stream);

/*
 * Range forms, for splitting one tensor over several processes or devices
 * (each computing a contiguous range of the stored entries, the partial
 * results then summed, e.g. by an all-reduce: Sec. 5.3's privatization, the
 * partial outputs being the ranks' instead of the threads').  Not paper
 * operations.
 *
 * pasta_mttkrp_range -- pasta_mttkrp restricted to the entries at positions
 * [lo, hi) of the mode-`mode` sorted copy: d_M (dims[mode] x R) is
 * overwritten with their MTTKRP (rows they do not reach are 0).  Summing the
 * outputs of ranges that partition [0, nnz) gives pasta_mttkrp's result (to
 * FP32 rounding).  lo must be a multiple of 4 (PASTA_ERR_ALIGNMENT) and
 * lo <= hi <= nnz (PASTA_ERR_INVALID_ARG).
 */
pasta_status pasta_mttkrp_range(pasta_coo X, const void *const *d_U, pasta_dtype u_dtype, int mode, int R,
                                uint64_t lo, uint64_t hi, void *d_M, void *stream);

/*
 * pasta_cp_loss_fwd_bwd_range -- pasta_cp_loss_fwd_bwd over the entries at
 * positions [lo, hi) of every sorted copy: pass k covers [lo, hi) of the
 * mode-k copy, and the loss is summed over [lo, hi) of the mode-0 copy.
 * Ranges that partition [0, nnz) therefore cover every entry once in each
 * pass, and the sums of their losses and gradients are the whole tensor's.
 * Same arguments as pasta_cp_loss_fwd_bwd plus lo, hi (limits as for
 * pasta_mttkrp_range).
 */
pasta_status pasta_cp_loss_fwd_bwd_range(pasta_coo X, const void *const *d_U, pasta_dtype u_dtype, int R,
                                         uint64_t lo, uint64_t hi, double *d_loss, const double *d_gscale,
                                         void *const *d_G, void *stream);

/*
 * pasta_coo_hicoo -- build (once per block size) the HiCOO copy of X: the
 * hierarchical COO format (Li, Choi and Vuduc, SC'18) that Sec. 8 names with
 * CSF as the compressed formats to add.  The index space is cut into blocks
 * of 2^block_bits cells per mode; entry coordinate i_k splits into the block
 * coordinate i_k >> block_bits and the offset i_k & (2^block_bits - 1).  The
 * copy holds the nonempty blocks (bptr: nb + 1 entry positions, the last one
 * nnz; binds[k]: nb block coordinates per mode, uint32) and, per entry in
 * block order, one offset byte per mode (einds[k]) and the FP32 value.
 * Blocks are in lexicographic order of their coordinates (mode 0 first);
 * entries of a block in lexicographic order of their offsets.  Both come
 * from one stable sort of the key (block coordinates, each mode taking
 * ceil(log2(ceil(dims[k] / 2^block_bits))) bits, then the offsets,
 * block_bits each), cut to its leading 64 bits; where offset bits are cut,
 * entries with equal leading bits keep creation order.  One copy serves
 * every mode.
 *   block_bits  1..8 (PASTA_ERR_INVALID_ARG otherwise); a later call with
 *               another value rebuilds the copy
 *   nblocks     host output (may be NULL): nb
 * PASTA_ERR_UNSUPPORTED when the block coordinates need more than 64 key
 * bits.  Synchronises `stream` (block count, then the end of the build).
 * Device memory: N + 4 bytes per entry (padded like the stored copies) plus
 * 4 N + 4 per block, freed by pasta_coo_destroy; the sort uses the handle's
 * scratch.
 */
pasta_status pasta_coo_hicoo(pasta_coo X, int block_bits, uint64_t *nblocks, void *stream);

/* Copy the HiCOO arrays into caller-owned device buffers (any may be NULL;
 * d_binds / d_einds are host arrays of N device pointers, entries may be
 * NULL): d_bptr nb + 1 uint32, d_binds[k] nb uint32, d_einds[k] nnz bytes,
 * d_val nnz FP32.  PASTA_ERR_NOT_SORTED without a HiCOO copy.  Asynchronous. */
pasta_status pasta_hicoo_copy_out(pasta_coo X, uint32_t *d_bptr, uint32_t *const *d_binds,
                                  uint8_t *const *d_einds, float *d_val, void *stream);

/*
 * pasta_hicoo_mttkrp -- the mode-n MTTKRP of pasta_mttkrp (Eq.
 * (mttkrp-init)), computed from the HiCOO copy (PASTA_ERR_NOT_SORTED if
 * absent) instead of a mode-sorted copy.  Same arguments and output.  The
 * copy is not ordered by the output mode, so rows are summed in two FP32
 * register slots per lane group (at most one 512-entry tile each) and, when
 * evicted, added with FP64 atomics into FP64 images of M in the handle's
 * scratch (block b into image b mod K, K images within 256 MB, at most 64),
 * which are then summed and rounded into d_M; the summation order differs
 * from pasta_mttkrp.  Calls on one handle that use the scratch must be
 * ordered.
 * Covers FP32/BF16/FP16 factors, order 2..5, R * sizeof(element) = 16 L with
 * L a power of two, 16-byte aligned factors and output; otherwise
 * PASTA_ERR_UNSUPPORTED.
 */
pasta_status pasta_hicoo_mttkrp(pasta_coo X, const void *const *d_U, pasta_dtype u_dtype, int mode, int R,
                                void *d_M, void *stream);

/*
 * pasta_memcpy -- copy `bytes` from src to dst on `stream` (asynchronous).
 * Either pointer may be device memory, pinned host memory or pageable host
 * memory.  Where one side is pinned host memory, both are 16-byte aligned and
 * bytes is a multiple of 4, a kernel moves the data (the SMs read or write
 * the host memory over the host link) instead of the copy engine; otherwise
 * cudaMemcpyAsync does (pageable memory: it returns once the source is read).
 * Host memory must stay allocated, and unchanged or unread, until the stream
 * has passed the copy.  pasta_coo_create copies its inputs the same way.
 * Not a paper operation: measured on GB300, copy-engine transfers between
 * pinned host memory and the GPU stalled for 20-90 ms about every 0.4 s in
 * some runs while SM-driven ones did not, at the same ~210 GB/s.
 * PASTA_ERR_INVALID_ARG for a NULL pointer with bytes > 0.
 */
pasta_status pasta_memcpy(void *dst, const void *src, uint64_t bytes, void *stream);

/*
 * pasta_set_grid_cap -- upper bound on the thread blocks of every MTTKRP and
 * CP-loss launch (streaming and general kernels; TTM, which runs as an
 * MTTKRP, included); 0 (the default) removes it.  Not a paper operation: a
 * diagnostic.  The kernels stride over the stored entries with whatever grid
 * they get, so results do not depend on it beyond FP32 rounding; a small cap
 * makes each block walk many block tiles in turn, which lets small inputs
 * exercise the same multi-round path that large ones take with the full grid.
 * Process-wide (all host threads and devices); it applies to launches made
 * after the call.  PASTA_ERR_INVALID_ARG for max_blocks < 0.
 * pasta_get_grid_cap returns the current cap.
 */
pasta_status pasta_set_grid_cap(int max_blocks);
int pasta_get_grid_cap(void);

/*
 * Device memory of the library's own buffers (stored copies, scratch, fiber
 * tables, partial sums).  By default cudaMalloc/cudaFree; a caller with its
 * own caching allocator (a framework's) can route them through it, so that
 * handles created and destroyed in a loop reuse memory instead of mapping it
 * anew.  alloc returns NULL on failure (the call then fails with
 * PASTA_ERR_NOMEM); blocks must be at least 256-byte aligned.  The library
 * synchronises the device before it frees a block that kernels may still
 * use.  Both NULL restores the default.  Refused (PASTA_ERR_INVALID_ARG)
 * while any block from the current allocator is still held.  The paper has
 * no counterpart.
 */
typedef void *(*pasta_alloc_fn)(size_t bytes, int device, void *stream, void *ctx);
typedef void (*pasta_free_fn)(void *ptr, void *ctx);
pasta_status pasta_set_allocator(pasta_alloc_fn alloc, pasta_free_fn free_fn, void *ctx);

#ifdef __cplusplus
}
#endif

#endif /* PASTA_H */
