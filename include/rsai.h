/*
 * rsai.h -- C ABI of the GB300 RSAI(tol) library (librsai.so).
 *
 * RSAI(tol) (Jia & Kang, residual based sparse approximate inverse) builds a
 * sparse M ~ A^{-1} by minimising ||AM - I||_F (Section 2, Eq. 2.1) one column
 * at a time (Eq. 2.2): for each k it solves the small least-squares problem
 * min ||A(I_k,J_k) m - e_k(I_k)|| (Eq. 2.3) by Householder QR, forms the
 * residual r_k = A m_k - e_k (Eq. 2.4), picks the c largest |r_k(i)| not used
 * before (Algorithm 1, Eq. 3.2), adds the columns of those rows of A to J_k
 * (Algorithm 1), drops entries |m_jk| <= tol_k (Eq. 4.3) and loops until
 * ||r_k|| <= eps or l_max loops (Algorithm 1).
 *
 * Conventions for every entry point:
 *   - Indices are 0-based, int32 for row/column indices, int64 for pointers
 *     and counts.  CSR rows and CSC columns are strictly ascending; explicit
 *     zeros count as structural nonzeros.
 *   - Unless a comment says otherwise, pointers may be host or device memory
 *     (the library asks the CUDA driver which one it is).  Host inputs are
 *     copied to the device inside the call; host outputs are written back
 *     before the call returns.
 *   - `stream` is a cudaStream_t passed as void*; NULL is the legacy default
 *     stream.  Work is stream-ordered: device inputs must stay valid until
 *     the stream reaches the call, device outputs are valid once it has.
 *   - Inputs are borrowed for the duration of the call.  A handle owns its
 *     device memory until rsai_handle_free.
 *   - Every function returns an rsai_status; no exception, device trap or
 *     device assert ever crosses this boundary.  On error nothing is written
 *     to outputs and *out handles are set to NULL.
 *   - One GPU: the device current on the calling thread is used.
 */
#ifndef RSAI_H
#define RSAI_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define RSAI_ABI_VERSION 2

typedef enum {
    RSAI_OK = 0,
    RSAI_ERR_INVALID_ARG = 1,   /* NULL pointer, bad parameter value */
    RSAI_ERR_SHAPE = 2,         /* n/nnz inconsistent between CSR and CSC */
    RSAI_ERR_UNSORTED = 3,      /* indices not strictly ascending in a row/column */
    RSAI_ERR_INDEX_RANGE = 4,   /* an index outside [0, n) or a bad pointer array */
    RSAI_ERR_EMPTY_COLUMN = 5,  /* a column of A without nonzeros: A is singular */
    RSAI_ERR_OOM = 6,           /* device allocation failed */
    RSAI_ERR_CUDA = 7,          /* a CUDA runtime call failed */
    RSAI_ERR_TIMEOUT = 8,       /* a bounded device wait ran out */
    RSAI_ERR_WORKSPACE = 9,     /* a column outgrew every size bin (see rsai_stats) */
    RSAI_ERR_BREAKDOWN = 10,    /* BiCGStab breakdown (rho = 0, rhat^T v = 0, t^T t = 0 or omega = 0) */
    RSAI_ERR_NOT_CONVERGED = 11,/* BiCGStab reached maxit */
    RSAI_ERR_NO_DEVICE = 12,    /* no CUDA device is visible */
    RSAI_ERR_TOO_LARGE = 13     /* problem larger than a fixed-size workspace */
} rsai_status;

/* Sparse A in CSR (row_ptr[n+1], col_idx[nnz], val[nnz]). */
typedef struct {
    int64_t n, nnz;
    const int64_t *row_ptr;
    const int32_t *col_idx;
    const double *val;
} rsai_csr;

/* The same A in CSC (col_ptr[n+1], row_idx[nnz], val[nnz]); used to gather
 * the columns A(:,J_k) and their nonzero rows I_k (Section 2). */
typedef struct {
    int64_t n, nnz;
    const int64_t *col_ptr;
    const int32_t *row_idx;
    const double *val;
} rsai_csc;

/* Dropping rule applied after every LS solve (Eq. 4.3 and its readings). */
enum {
    RSAI_DROP_NONE = 0,     /* basic RSAI, Algorithm 1 */
    RSAI_DROP_ADAPTIVE = 1, /* tol_k = eps / (nnz(m_k) ||A||_1), Eq. 4.3 */
    RSAI_DROP_FIXED = 2     /* tol_k = tol / ||A||_1 (absolute tol on A/||A||_1) */
};

/* Arithmetic of the LS solves.  The residual r_k, its norm, the dominant-row
 * choice and the stopping test are FP64 in both. */
enum {
    RSAI_FP64 = 0,        /* Householder QR and solve in FP64 */
    RSAI_FP32_REFINE = 1  /* QR in FP32, FP64 residual, one FP64 refinement step */
};

/* Flags */
enum {
    /* bit 0 is reserved: the input checks (ranges, sortedness, the CSR/CSC
       pairing) always run and report status codes, so there is no flag for them */
    RSAI_FLAG_INIT_PATTERN_A = 2u, /* initial pattern J_k^(0) = rows of column k of A instead of {k}
                                      (Algorithm 1 leaves it to the user; Section 3 suggests
                                      that of I, the default, when A has a nonzero diagonal) */
    RSAI_FLAG_SELECT_SPAI = 4u     /* SPAI's choice of new indices (Section 2, Eqs. 2.5-2.7) instead of
                                      the dominant rows of Algorithm 1: the candidates are the nonzero
                                      columns of the rows where r_k != 0, less J_k, and the c with the
                                      smallest rho_j^2 = ||r_k||^2 - (r_k^T A e_j)^2 / ||A e_j||^2 are
                                      added (ties by lowest index within tie_band * ||r_k||^2); a loop
                                      with no candidate ends the column.  Solve, drop and residual
                                      are RSAI(tol)'s.  The method the paper compares with (Section 5.2). */
};

/* Parameters of RSAI(tol) (Algorithm 1; Section 3 defaults c ~ 3,
 * eps = 0.1..0.4, l_max ~ 10; Eq. 4.3). */
typedef struct {
    int32_t c;          /* dominant rows per loop (|Rhat_k|), 1..32 */
    int32_t l_max;      /* maximum number of loops, >= 0 */
    double eps;         /* stop when ||r_k|| <= eps, > 0 */
    int32_t drop_mode;  /* RSAI_DROP_* */
    double tol;         /* threshold of RSAI_DROP_FIXED, >= 0 */
    int32_t precision;  /* RSAI_FP64 or RSAI_FP32_REFINE */
    double tie_band;    /* relative tie band for the dominant-row order, >= 0 (default 1e-12) */
    uint32_t flags;     /* RSAI_FLAG_* */
} rsai_params;

/* Per-build statistics (Section 5 reporting: spar = nnz(M)/nnz(A), n_c). */
typedef struct {
    int64_t n;            /* columns of M */
    int64_t nnz_A;
    int64_t nnz_M;        /* nonzeros of M */
    int64_t n_c;          /* columns with ||r_k|| > eps (Section 5, n_c) */
    double frob;          /* ||AM - I||_F = sqrt(sum_k ||r_k||^2) */
    double norm1_A;       /* ||A||_1 (Eq. 4.3) */
    double qr_flops;      /* algorithmic QR + solve flops (paper's QR update), in the QR precision */
    double res_flops;     /* algorithmic FP64 residual flops (Eq. 2.4) */
    double refine_flops;  /* FP32_REFINE only: FP32 flops of the refinement solves */
    double refine_flops_f64; /* FP32_REFINE only: FP64 flops of the refinement residuals */
    double bytes;         /* algorithmic bytes */
    int64_t loops;        /* sum over columns of the loops used */
    int64_t solves;       /* LS solves */
    int64_t drops;        /* solves that dropped entries (each costs a re-solve) */
    int32_t p_max, q_max; /* largest LS problem met */
    int64_t cols_bin[3];  /* columns finished by the warp bins (W, W2), the CTA bin and the global bin */
    int64_t n_rank;       /* columns flagged rank deficient */
    int64_t n_nonfinite;  /* columns with a non-finite value */
    int64_t n_failed;     /* columns no bin could hold (then status WORKSPACE) */
    int64_t cols_bin_half; /* of cols_bin[0]: columns finished by the half-warp bin (|I| <= 48, |J| <= 16) */
    double select_flops;  /* RSAI_FLAG_SELECT_SPAI only: FP64 flops of the candidates' rho_j (Eq. 2.7) */
} rsai_stats;

/* Per-column outcome bits (rsai_get_columns). */
enum { RSAI_COL_CONVERGED = 1, RSAI_COL_RANK = 2, RSAI_COL_NONFINITE = 4, RSAI_COL_FAILED = 8 };

typedef struct rsai_handle rsai_handle;

/* Library version (RSAI_ABI_VERSION).  No counterpart in the paper. */
int32_t rsai_abi_version(void);

/* Text of a status code (static storage, never NULL).  No counterpart in the
 * paper. */
const char *rsai_status_string(rsai_status s);

/* Defaults of Section 3 / Section 5: c = 3, l_max = 10, eps = 0.3,
 * RSAI_DROP_FIXED with tol = 1e-3, RSAI_FP64, tie_band = 1e-12. */
rsai_status rsai_params_default(rsai_params *p);

/* Host-only validation of a parameter block (no device work): the ranges of
 * Algorithm 1's c, l_max and eps (Section 3), the drop mode and tol of Eq. 4.3,
 * and the flags.  Errors: INVALID_ARG. */
rsai_status rsai_params_check(const rsai_params *p);

/*
 * rsai_build -- build M column by column (Algorithm 1 + Eq. 4.3; the columns
 * are independent, Eq. 2.2).
 *   A, Acsc : the same n x n matrix in CSR and CSC (host or device arrays).
 *   params   : see rsai_params.
 *   out      : receives a handle owning M (CSR and CSC on the device), the
 *              frozen pattern, ||r_k|| and the per-column flags.
 * Validates A (shape, sorted, index range, no empty column) on the device
 * before building.  The call returns when M and its statistics are ready.
 * Errors: INVALID_ARG, SHAPE, UNSORTED, INDEX_RANGE, EMPTY_COLUMN, OOM, CUDA,
 * WORKSPACE (a column outgrew every bin: the handle is still returned with
 * those columns flagged RSAI_COL_FAILED).
 */
rsai_status rsai_build(const rsai_csr *A, const rsai_csc *Acsc, const rsai_params *params,
                       void *stream, rsai_handle **out);

/*
 * rsai_build_batch -- build M for `count` independent matrices in one
 * sequence of launches (Eq. 2.2 over all their columns at once).  The members
 * are placed side by side as one block-diagonal matrix: a column's pattern
 * never leaves its block (I_k, the dominant rows and the new columns all stay
 * in it), and ||A||_1 of the drop rule (Eq. 4.3) is taken per member, so every
 * block of the result equals the member's own build.
 *   As[b], Acscs[b] : member b in CSR and CSC (host or device arrays), b < count.
 * The handle's M is block diagonal (n = sum of the members' n); read it with
 * rsai_get_M and split it by the members' sizes; per-member statistics come
 * from rsai_get_block_stats.  rsai_rebuild, rsai_refit, rsai_backward and
 * rsai_apply work on the whole batch.  Errors as rsai_build.
 */
rsai_status rsai_build_batch(const rsai_csr *As, const rsai_csc *Acscs, int32_t count, const rsai_params *params,
                             void *stream, rsai_handle **out);

/* Per-member ||A_b M_b - I||_F (Eq. 2.1), n_c and nnz(M_b) (the Section 5
 * metrics) of a batch handle (one entry for a single-matrix handle); host
 * arrays of `count` entries, any may be NULL.  Synchronises the stream. */
rsai_status rsai_get_block_stats(rsai_handle *h, void *stream, double *frob, int64_t *n_c, int64_t *nnz_M);

/*
 * rsai_rebuild -- Algorithm 1 with Eq. 4.3 over every column (Eq. 2.2) again,
 * on the handle's own copy of A after
 * new values were written with rsai_set_values (same structure), reusing every
 * buffer: no allocation, no host synchronisation; the launch sequence is
 * recorded in a CUDA graph on first use and replayed afterwards.
 * Statistics are refreshed by rsai_get_stats.  Errors: INVALID_ARG, CUDA.
 */
rsai_status rsai_rebuild(rsai_handle *h, void *stream);

/* Overwrite the handle's copy of A's values (CSR order; host or device): the
 * matrix whose LS problems (Eq. 2.3) the next rsai_rebuild solves, on the same
 * structure.  The CSC copy follows on the device. */
rsai_status rsai_set_values(rsai_handle *h, const double *A_val, void *stream);

/* Statistics of the last build (synchronises the stream): ||AM - I||_F
 * (Eq. 2.1), spar and n_c (Section 5) and the algorithmic work counters. */
rsai_status rsai_get_stats(rsai_handle *h, void *stream, rsai_stats *out);

/*
 * rsai_get_M -- copy M (the columns m_k of Eq. 2.2) out in CSR: row_ptr[n+1]
 * (int64), col_idx[nnz_M] (int32), val[nnz_M]; any pointer may be NULL to
 * skip it.  Sized by rsai_stats.nnz_M.  Host or device destinations.
 */
rsai_status rsai_get_M(rsai_handle *h, int64_t *row_ptr, int32_t *col_idx, double *val, void *stream);

/* Per-column results: rho[k] = ||r_k|| (Eq. 2.4), loops[k] (l of Algorithm
 * 1), flags[k] (RSAI_COL_*); NULL pointers are skipped.  Host or device
 * destinations. */
rsai_status rsai_get_columns(rsai_handle *h, double *rho, int32_t *loops, int32_t *flags, void *stream);

/*
 * rsai_refit -- re-solve every column on the frozen pattern of M with new
 * values of A (same structure, CSR order): m_k = argmin ||A(:,J_k) x - e_k||
 * (Eq. 2.3), rho2[k] = ||r_k||^2 (Eq. 2.4).  No dropping, no pattern change.
 * M_val receives the values in M's CSR order; either output may be NULL.
 * Uses the handle's precision.  Device pointers only.
 */
rsai_status rsai_refit(rsai_handle *h, const double *A_val, double *M_val, double *rho2, void *stream);

/*
 * rsai_apply -- y = M x (the right preconditioner, Eq. 1.2: x = M y).
 * x, y: device arrays of length n.
 */
rsai_status rsai_apply(rsai_handle *h, const double *x, double *y, void *stream);

/*
 * rsai_backward -- adjoint of the frozen-pattern solves.  For a scalar loss
 * L(M, rho^2) with G_M = dL/dM (values in M's CSR order) and g = dL/d(rho_k^2)
 * (may be NULL), writes dL/d(values of A) (CSR order of A) through every
 * column's LS solve (Eq. 2.3) at the values A_val:
 *   dL/dB_k = -r_k z_k^T - (B_k z_k) x_k^T + 2 g_k r_k x_k^T,
 *   z_k = (B_k^T B_k)^{-1} G_M(J_k, k),  B_k = A(I_k, J_k),  x_k = m_k(J_k),
 * each QR recomputed (not stored).  The pattern is not differentiated.
 * Device pointers only.  The sum over columns has a fixed order and uses no
 * atomics, so the result is bit-identical from run to run (there is no
 * separate deterministic mode).
 */
rsai_status rsai_backward(rsai_handle *h, const double *A_val, const double *grad_M, const double *grad_rho2,
                          double *grad_A, void *stream);

/*
 * rsai_bicgstab -- right-preconditioned BiCGStab on A M y = b, x = M y
 * (Eq. 1.2; Section 5 protocol: x0 = 0, stop when the recursive residual
 * satisfies ||r||/||b|| < rtol at a half or full step, at most maxit
 * iterations).  M may be NULL (no preconditioner).  A: device CSR (the
 * handle's copy is not used, so A may differ from the matrix M was built for).
 * b, x: device arrays.  On return *iters holds the iterations (a half-step exit
 * counts as its full iteration) and *relres the true ||b - A x|| / ||b||.
 * Errors: BREAKDOWN, NOT_CONVERGED (x still holds the last iterate).
 */
rsai_status rsai_bicgstab(const rsai_csr *A, rsai_handle *M, const double *b, double *x, double rtol,
                          int32_t maxit, int32_t *iters, double *relres, void *stream);

/* Phases of the build sequence timed by rsai_build_phase_times. */
enum {
    RSAI_PHASE_SETUP = 0,   /* counters reset, ||A||_1 */
    RSAI_PHASE_BIN_WARP,    /* columns on one warp each */
    RSAI_PHASE_BIN_CTA,     /* columns on one CTA each, shared-memory workspace */
    RSAI_PHASE_BIN_GLOBAL,  /* columns on one CTA each, global-memory workspace */
    RSAI_PHASE_ASSEMBLE,    /* statistics, M to CSC and CSR */
    RSAI_PHASE_COUNT
};

/*
 * rsai_build_phase_times -- no counterpart in the paper (timing of the build's
 * phases for the roofline).  Runs the build sequence of rsai_rebuild once more,
 * launched phase by phase (not as a graph) with a CUDA event between phases on
 * `stream`, and write each phase's duration in milliseconds to
 * ms[RSAI_PHASE_COUNT].  Synchronises the stream.  The result of the build is
 * the same as rsai_rebuild's.
 */
rsai_status rsai_build_phase_times(rsai_handle *h, void *stream, double *ms);

/*
 * rsai_bicgstab_noalloc -- the solve of rsai_bicgstab for callers that must not
 * allocate device memory (for example code running inside another
 * framework's memory pool or plugin interface, or a real-time loop where an
 * allocation and its implicit synchronisation are not allowed).  The paper has
 * no counterpart: this is a deployment variant of rsai_bicgstab.
 *   A : device CSR of A;  M : device CSR of the preconditioner (e.g. copied out
 *       with rsai_get_M) or NULL;  b, x : device arrays of length n.
 * It allocates nothing: its work vectors live in one fixed device array inside
 * the library (about 4.7 MB, held by every GPU that loads the library until the
 * process exits) and n must not exceed 65536 (else RSAI_ERR_TOO_LARGE).  Like
 * rsai_bicgstab it waits for the stream at every iteration to read the scalars
 * of its stopping test, so it cannot be captured into a CUDA graph.  The first
 * call on each device looks up the array's device address (and keeps it); make
 * that first call while no stream of the process is being captured.  After a
 * cudaDeviceReset of a device the kept address is stale, so do not call it on
 * that device again.  Every call shares the array: calls that overlap on the
 * GPU race and must be ordered on one stream.
 * It runs rsai_bicgstab's solver code: same results, statuses and outputs.
 */
rsai_status rsai_bicgstab_noalloc(const rsai_csr *A, const rsai_csr *M, const double *b, double *x, double rtol,
                                  int32_t maxit, int32_t *iters, double *relres, void *stream);

/*
 * Launch shapes of the size bins.  The CTA shapes and grid sizes change speed
 * only: every column is computed by the same arithmetic whatever the shape, so
 * M is identical bit for bit.  small_qr_max_p chooses between the
 * register-resident and the shared-memory Householder QR of the warp bin, which
 * agree to rounding (same patterns in practice, values within ~1e-14 relative
 * in FP64).  Picked per GPU and problem by the autotuner of the Python package
 * (paper_1503_04500_gb300/autotune.py).
 */
typedef struct {
    int32_t warp_bin_warps;       /* warps per CTA of the warp bin: 1, 2, 4 or 8 (default 8); the second
                                     warp bin (|I| <= 128) uses it halved until its workspace fits */
    int32_t warp_bin_ctas_per_sm; /* resident CTAs per SM of the warp bin, 0 = as many as fit */
    int32_t small_qr_max_p;       /* largest |J| solved by the register-resident warp QR, 0..16
                                     (default 16; 8 for RSAI_FP64) */
    int32_t global_bin_ctas;      /* CTAs of the global bin, 0 = one per column that reaches it, <= SMs;
                                     the bin's global-memory workspace (one slab per CTA) is resized to
                                     match */
    int32_t half_bin;             /* 1: columns start in the half-warp bin (two columns per warp, |I| <= 48,
                                     |J| <= 16) and move on to the warp bin when they outgrow it; 0: they start
                                     in the warp bin.  Default 1 for RSAI_FP64, 0 for RSAI_FP32_REFINE. */
} rsai_tuning;

/* Read / replace a handle's launch shapes (no counterpart in the paper); the
 * next rsai_rebuild records a new graph.  Synchronises the handle's stream.  Errors: INVALID_ARG (a value out
 * of range or a shape that cannot be resident), OOM. */
rsai_status rsai_get_tuning(const rsai_handle *h, rsai_tuning *t);
rsai_status rsai_set_tuning(rsai_handle *h, const rsai_tuning *t);

/* Release a handle and its device memory (NULL is a no-op).  No counterpart in
 * the paper. */
void rsai_handle_free(rsai_handle *h);

/*
 * rsai_get_M_csc -- M's pattern in CSC (the patterns J_k of the columns m_k,
 * Eq. 2.2), as the build assembled it:
 * col_ptr[n+1] (int64), row_idx[nnz_M] (int32, ascending within a column)
 * and csc_to_csr[nnz_M] (int64): the position in rsai_get_M's CSR value array
 * of each CSC entry, so that the CSC values of M (or of any array in M's CSR
 * order, such as rsai_refit's output) are val_csr[csc_to_csr[e]].  Any
 * pointer may be NULL.  Host or device destinations; synchronises the stream.
 * With it, products with M^T are CSR products over (col_ptr, row_idx).
 */
rsai_status rsai_get_M_csc(rsai_handle *h, int64_t *col_ptr, int32_t *row_idx, int64_t *csc_to_csr, void *stream);

/*
 * rsai_spmv -- y = A x for a CSR matrix on the device (Eq. 1.2 applies A and
 * M by such products; BiCGStab, Section 5).  A->row_ptr/col_idx/val, x and y
 * are device pointers; y is overwritten, x and y must not overlap.  A product
 * with A^T is the same call on A's CSC arrays (col_ptr, row_idx, CSC values)
 * read as the CSR of A^T.  8 lanes per row, a fixed reduction order (repeated
 * calls give identical y).  Errors: INVALID_ARG, SHAPE, NO_DEVICE, CUDA.
 */
rsai_status rsai_spmv(const rsai_csr *A, const double *x, double *y, void *stream);

/*
 * rsai_spmv_grad_values -- gval[e] = gy[i] * x[col_idx[e]] for every stored
 * entry e of row i: the gradient of <gy, A x> with respect to the stored values
 * of A, in A's CSR order (the adjoint of rsai_spmv in its values; the adjoint
 * in x is rsai_spmv on A^T).  No counterpart in the paper, which does not
 * differentiate; it lets a caller differentiate a Krylov solve preconditioned
 * by M.  A->val is not read.  Device pointers; gval is overwritten.  Errors:
 * INVALID_ARG, SHAPE, NO_DEVICE, CUDA.
 */
rsai_status rsai_spmv_grad_values(const rsai_csr *A, const double *gy, const double *x, double *gval, void *stream);

/*
 * rsai_set_allocator -- where the library takes its device memory from.
 *
 * No counterpart in the paper: the plumbing that lets a host framework (for
 * example PyTorch's caching allocator) own every device buffer of the library.
 *
 * alloc(bytes, stream, ctx) returns a device pointer (aligned to at least 256
 * bytes) usable in stream order on `stream`, or NULL when out of memory (the
 * call then fails with RSAI_ERR_OOM).  release(ptr, bytes, stream, ctx) gives
 * a buffer back; `stream` is the stream its last use was ordered on, or NULL
 * after a device-wide synchronisation (rsai_handle_free).  Both are called on
 * the calling host thread, never during a CUDA graph replay.
 *
 * The setting is process-wide and applies to handles created afterwards (a
 * handle frees with the allocator it was created with), to the temporaries of
 * rsai_refit and to the workspace of rsai_bicgstab.  alloc = release = NULL
 * restores the default: a stream-ordered pool of the library's own on each
 * device (cudaMallocFromPoolAsync / cudaFreeAsync), which keeps up to 2 GiB of
 * freed handle memory mapped for the next handle.  Not thread-safe against builds
 * running on other threads.  Errors: INVALID_ARG when exactly one of the two
 * is NULL.
 */
typedef void *(*rsai_alloc_fn)(size_t bytes, void *stream, void *ctx);
typedef void (*rsai_free_fn)(void *ptr, size_t bytes, void *stream, void *ctx);
rsai_status rsai_set_allocator(rsai_alloc_fn alloc, rsai_free_fn release, void *ctx);

/*
 * rsai_peak_fma -- no counterpart in the paper.  Measures the CUDA-core FMA
 * pipe rate: launches a grid of
 * independent FMA chains (FP32 if fp64 == 0, FP64 otherwise) and returns the
 * achieved flop/s in *flops_per_s (2 flops per FMA).  Used for the roofline
 * of the build kernels.
 */
rsai_status rsai_peak_fma(int32_t fp64, void *stream, double *flops_per_s);

#ifdef __cplusplus
}
#endif

#endif /* RSAI_H */
