/*
 * dbcsr_gb.h -- C ABI of the GB300 block-sparse sign-matrix library.
 *
 * The library implements, for one GPU, the block-sparse matrix operations and
 * the density-matrix sign iteration of the CP2K/Quickstep review
 * (Kuehne et al. 2020):
 *   - DBCSR block-CSR matrices of atom blocks (section "DBCSR library": blocks
 *     whose sizes follow the basis of each atom, stored in a blocked CSR format);
 *   - the local block-sparse product C = beta*C + alpha*A*B as batches of small
 *     dense block products (section "Local multiplication") followed by the
 *     eps_filter truncation (section "Sign-Method");
 *   - trace and the trace of a product (DBCSR's single-matrix operations);
 *   - the sign iteration X <- X (3 - X^2) / 2 and the density matrix
 *     P = (1 - sign(H - mu 1)) / 2 (section "Sign-Method", Eq. signdef and the
 *     density-matrix relation with S = 1).
 *
 * Conventions shared by every entry point:
 *   - Every function returns a dbcsr_status; no C++ exception crosses the ABI.
 *     On failure dbcsr_last_error() returns a message (per host thread), and
 *     the output arguments are left unchanged unless stated otherwise.
 *   - Handles are created and destroyed by the caller.  The library owns all
 *     device memory of a matrix (stream-ordered allocations on the matrix's
 *     stream); input buffers are copied, never retained.
 *   - Matrices are square block grids: block row and block column I both have
 *     edge blk_size[I].  Blocks are dense, row-major, FP64 unless a function
 *     says otherwise.  Both triangles of symmetric matrices are stored.
 *   - Work is queued on the matrix's CUDA stream.  Functions that return host
 *     values (traces, reports, statistics, get_block, export) synchronise that
 *     stream before returning.
 *   - "on_device" arguments: 0 = the pointer is host memory, 1 = it is device
 *     memory of the current device.  Index arrays are always host memory.
 */
#ifndef DBCSR_GB_H
#define DBCSR_GB_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dbcsr_matrix_* dbcsr_matrix;

typedef enum {
    DBCSR_OK = 0,
    DBCSR_EINVAL = 1,     /* bad argument: null handle, index out of range, size mismatch, duplicate block */
    DBCSR_ENOMEM = 2,     /* a device or host allocation failed */
    DBCSR_ECAPACITY = 3,  /* a size exceeds a fixed limit of the library */
    DBCSR_ECUDA = 4,      /* a CUDA runtime call failed (message holds cudaGetErrorString) */
    DBCSR_ENAN = 5,       /* a NaN or Inf appeared in a result */
    DBCSR_ENOTCONV = 6,   /* the sign iteration stopped without reaching the tolerance */
    DBCSR_ETIMEOUT = 7,   /* a bounded device-side wait ran out */
    DBCSR_ESTATE = 8      /* the call is not allowed in the matrix's current state (e.g. not finalized) */
} dbcsr_status;

typedef enum {
    DBCSR_FP64 = 0,       /* FP64 operands, FP64 accumulation */
    DBCSR_BF16 = 2,       /* BF16 operands (round to nearest even), FP32 accumulation, FP64 result */
    DBCSR_MIXED = 3,      /* sign iteration only: low-precision tier while the residual >= switch, then FP64 */
    DBCSR_BF16X3 = 4,     /* split BF16 operands a = hi + lo (both BF16), A B ~ Ah Bh + Ah Bl + Al Bh on the
                             BF16 tensor cores with FP32 accumulation (about 16 significant bits), FP64 result */
    DBCSR_TF32 = 5,       /* dense products only: FP32 data, TF32 operands (10 stored bits), FP32 accumulation */
    DBCSR_TF32X3 = 6      /* dense products only: FP32 data, split TF32 operands (three products, about 21 bits) */
} dbcsr_prec;

/* Work counters of one product.  Counts refer to the blocks the product
 * actually formed, after the exact norm-bound prescreen (a candidate C block
 * whose bound |alpha| sum_K ||A_IK||_F ||B_KJ||_F + |beta| ||C_IJ||_F is below
 * eps_filter can only be filtered, so it is not formed). */
typedef struct {
    int64_t n_candidates;      /* blocks of the full pattern of A*B (union C when beta != 0) */
    int64_t n_formed;          /* candidate blocks that passed the prescreen and were computed */
    int64_t n_kept;            /* blocks left after the eps_filter truncation */
    int64_t n_products;        /* block products A_IK * B_KJ executed */
    double flops;              /* sum of 2*m*k*n over the executed products (unpadded) */
    double dev2_filtered;      /* ||C_filtered - 1||_F^2 (meaningful for X*X in the sign iteration) */
    double ms_symbolic;        /* device time of the stack builder, ms */
    double ms_numeric;         /* device time of the block-product kernel, ms */
    double ms_filter;          /* device time of norm-filter-compaction, ms */
    double bytes_min;          /* compulsory bytes of the block-product launches: A and B read once,
                                  computed C blocks written once (a C input other than A, B read once) */
    int32_t n_launches;        /* block-product kernel launches (one per block shape) */
    int32_t reserved;
    /* BF16 products (the tensor-core tier on groups of atom blocks): */
    double flops_tensor;       /* executed MMA flops, 2 M N K per MMA, padding and every split product counted */
    double bytes_tensor;       /* bytes its bulk copies move from global into shared memory */
    int64_t n_tiles;           /* group tiles of C formed */
} dbcsr_mult_stats;

/* Options of the sign iteration. */
typedef struct {
    double eps_filter;         /* block Frobenius-norm threshold applied after every product */
    double tol;                /* stop when ||X^2 - 1||_F / N < tol */
    int32_t max_iter;          /* at most this many steps (default 100 when <= 0) */
    int32_t prec;              /* dbcsr_prec: DBCSR_FP64 or DBCSR_MIXED */
    double switch_tol;         /* DBCSR_MIXED: residual below which FP64 takes over (e.g. 1e-4) */
    double stall_ratio;        /* stall test: r_k > ratio*r_{k-1} after r_{k-1} < ratio*r_{k-2} (default 0.5 when <= 0) */
    int32_t verbose;           /* 1: print one line per step to stderr */
    int32_t flags;             /* DBCSR_SIGN_* bits, 0 = defaults */
    int32_t order;             /* order of the iteration, 2 to 7 (0 = 2, Newton-Schulz); see dbcsr_sign_iterate */
    int32_t reserved;          /* 0 */
} dbcsr_sign_opts;

/* dbcsr_sign_opts.flags.  Every product of the iteration has a symmetric exact
 * result.  By default every product forms only the blocks I <= J, copies the
 * blocks I > J as transposes (blocks without a formed twin are dropped) and
 * replaces each diagonal block by its symmetric part, so X stays exactly symmetric
 * and the products cost half.  (Left as computed, the antisymmetric part of the
 * diagonal blocks grows from product to product under mirroring.)  The low tier of
 * a DBCSR_MIXED iteration uses split-BF16 products (DBCSR_BF16X3), which commute
 * with X to about 1e-5.
 * DBCSR_SIGN_FULL_PRODUCTS: form both triangles of every product and keep them as
 * computed (no final symmetrisation).
 * DBCSR_SIGN_PLAIN_BF16: DBCSR_MIXED's low tier uses plain BF16 products.  A BF16
 * X2 commutes with X only to about 1e-3, so this ladder forms both triangles of
 * every product and symmetrises the final X. */
#define DBCSR_SIGN_FULL_PRODUCTS 1
#define DBCSR_SIGN_PLAIN_BF16 2
/* DBCSR_MIXED, after the switch: the update X <- 1.5 X - 0.5 X X2 is taken as
 * X - 0.5 X (X2 - 1), with the product X (X2 - 1) in split BF16.  Near convergence
 * X2 - 1 is small, so the error of that product (about 2^-16 of |X| |X2 - 1|) stays far
 * below the eps_filter truncation; X*X, the residual, the convergence test, the filter
 * and the traces stay FP64.  Off by default: the default FP64 tier computes both
 * products in FP64.  Order 2 only (EINVAL with a higher order). */
#define DBCSR_SIGN_LOW_CORRECTION 4
/* The iteration's state instead of the density matrix: P_out receives X as it stands when the
 * iteration stops (for a checkpoint: dbcsr_save it, and continue later with
 * dbcsr_sign_iterate_resume); rep->trace_p and rep->e_band are NaN. */
#define DBCSR_SIGN_RETURN_X 8

#define DBCSR_MAX_HISTORY 128

/* Outcome of dbcsr_sign_iterate. */
typedef struct {
    int32_t iterations;        /* steps taken (products X*X formed) */
    int32_t converged;         /* 1 if r < tol was reached */
    int32_t stalled;           /* 1 if the stall test stopped the iteration */
    int32_t fp64_from;         /* first step whose X*X was formed in FP64 (1 for DBCSR_FP64) */
    double alpha;              /* Gershgorin scale: X_0 = (H - mu 1) / alpha */
    double residual;           /* last r = ||X^2 - 1||_F / N */
    double trace_p;            /* Tr(P) */
    double e_band;             /* Tr(P H) */
    double flops;              /* sum over every product of the executed 2*m*k*n */
    int64_t n_products;        /* executed block products */
    double ms_total;           /* wall time of the call (device-synchronised), ms */
    double ms_multiply;        /* device time spent in block-product kernels, ms */
    int64_t nnzb_x;            /* blocks of the converged X */
    double residual_history[DBCSR_MAX_HISTORY];
    int64_t nnzb_history[DBCSR_MAX_HISTORY];
    double ms_symbolic;        /* device time of the stack builders, ms */
    double ms_filter;          /* device time of norm-filter-compaction (and mirroring), ms */
    double ms_low;             /* device time of the low tier's block-product kernels, ms */
    double flops_low;          /* executed 2*m*k*n of the low tier's products */
    double bytes_min_fp64;     /* sum of dbcsr_mult_stats.bytes_min over the FP64 products */
    int64_t launches_fp64;     /* sum of dbcsr_mult_stats.n_launches over the FP64 products */
    double flops_tensor;       /* sum of dbcsr_mult_stats.flops_tensor over the low tier's products */
    double bytes_tensor;       /* sum of dbcsr_mult_stats.bytes_tensor over the low tier's products */
} dbcsr_sign_report;

/* Last error message of the calling host thread ("" if none). */
const char* dbcsr_last_error(void);

/* Library version string. */
const char* dbcsr_version(void);

/*
 * Device memory.  Every buffer of the library (matrices, product stacks, scratch)
 * comes from one stream-ordered memory pool per device, owned by the library, that
 * keeps freed memory cached for reuse (the per-product stacks are allocated and freed
 * every product).  dbcsr_pool_trim waits for the current device, then returns the
 * cached memory above keep_bytes to the driver; memory held by live matrices stays.
 * Not from the paper (an allocator detail of this library).
 */
dbcsr_status dbcsr_pool_trim(uint64_t keep_bytes);

/*
 * Creates an empty matrix with nblk block rows/columns of edges blk_size[0..nblk-1]
 * (host array, each in [1, 32]).  stream: a cudaStream_t (NULL = the legacy
 * default stream); all work on the matrix is queued there.  The matrix starts
 * in the "building" state: blocks are added with put_block(s), then finalize().
 */
dbcsr_status dbcsr_create(dbcsr_matrix* out, int32_t nblk, const int32_t* blk_size, void* stream);

/* Frees the matrix and its device memory (stream-ordered).  NULL is accepted. */
dbcsr_status dbcsr_destroy(dbcsr_matrix m);

/*
 * Stages block (row, col): blk_size[row] x blk_size[col] doubles, row-major, at
 * data (host or device per on_device).  The data is copied before return.
 * Allowed in the building state only; a duplicate (row, col) makes finalize fail.
 */
dbcsr_status dbcsr_put_block(dbcsr_matrix m, int32_t row, int32_t col, const double* data, int on_device);

/*
 * Stages n blocks at once: rows[i], cols[i] (host arrays); their data packed one
 * after the other, each row-major, in the order given (host or device).
 */
dbcsr_status dbcsr_put_blocks(dbcsr_matrix m, int64_t n, const int32_t* rows, const int32_t* cols,
                              const double* packed, int on_device);

/* Sorts the staged blocks into block-CSR order and moves them to the device.
 * Fails with DBCSR_EINVAL on a duplicate block (the matrix stays building). */
dbcsr_status dbcsr_finalize(dbcsr_matrix m);

/* Block count and stored element count of a finalized matrix. */
dbcsr_status dbcsr_get_info(dbcsr_matrix m, int32_t* nblk, int64_t* nnzb, int64_t* nelem);

/* Copies block (row, col) to out_host (row-major) and sets *present; absent
 * blocks set *present = 0 and leave out_host untouched. */
dbcsr_status dbcsr_get_block(dbcsr_matrix m, int32_t row, int32_t col, double* out_host, int* present);

/*
 * Copies the whole matrix to host arrays: row_ptr[nblk+1], col[nnzb] and the
 * packed FP64 data[nelem] in block-CSR order (each may be NULL to skip it).
 */
dbcsr_status dbcsr_export(dbcsr_matrix m, int64_t* row_ptr, int32_t* col, double* data);

/*
 * Matrix files.  dbcsr_save writes the finalized m to path; dbcsr_load creates *out (on
 * the given CUDA stream, NULL = default) from such a file and finalizes it.  The file:
 * 8 bytes "DBCSRGB1", int32 nblk, int32 0, int64 nnzb, int64 nel, int32 blk_size[nblk],
 * int64 row_ptr[nblk + 1], int32 col[nnzb] (ascending per row), double data[nel] (blocks
 * row-major in CSR order), in the host's byte order, then the uint32 CRC-32 (IEEE 802.3 /
 * zlib) of all the bytes before it.  dbcsr_file_info reads and checks a
 * whole file on the host, without device work, and returns its sizes (each pointer may be
 * NULL).  Errors: EINVAL (null argument, unreadable or unwritable path, a file that is
 * not a valid matrix file: wrong magic, length, checksum, row pointers, columns or sizes),
 * ESTATE (save of an unfinalized matrix), ENOMEM, ECUDA.
 */
dbcsr_status dbcsr_save(dbcsr_matrix m, const char* path);
dbcsr_status dbcsr_load(dbcsr_matrix* out, const char* path, void* stream);
dbcsr_status dbcsr_file_info(const char* path, int32_t* nblk, int64_t* nnzb, int64_t* nel);

/* dst = src (pattern and values); dst must have the same block sizes. */
dbcsr_status dbcsr_copy(dbcsr_matrix dst, dbcsr_matrix src);

/* m = scale * m + shift * 1.  Every diagonal block must be present. */
dbcsr_status dbcsr_scale_shift(dbcsr_matrix m, double scale, double shift);

/*
 * A = alpha * A + beta * B on the union of the two patterns (DBCSR's add; the
 * higher-order sign iterations of section "Sign-Method" sum polynomial terms with
 * it).  A block present in one operand only is that operand's term alone.  Each
 * element is alpha*a + beta*b with both products rounded before the sum (no fused
 * multiply-add), so results do not depend on the launch.  No filtering.  B may be
 * the same handle as A.  A's arrays are replaced; B is unchanged.
 * Errors: EINVAL (null handle, different block sizes), ESTATE (A or B not
 * finalized, A used by a multiply plan), ENOMEM, ECUDA.
 */
dbcsr_status dbcsr_add(double alpha, dbcsr_matrix A, double beta, dbcsr_matrix B);

/*
 * C = beta * C + alpha * A * B, then every block of C with Frobenius norm
 * strictly below eps_filter is removed (diagonal blocks are always kept).
 * The sum over K of each C_IJ is taken in ascending K.  C may be the same
 * handle as A and/or B.  The result is formed on the pattern of A*B (union C's
 * pattern when beta != 0) less the candidates that the exact norm-bound
 * prescreen proves would be filtered.  prec: DBCSR_FP64, DBCSR_BF16 or DBCSR_BF16X3
 * (BF16 kinds: the operands are rounded to BF16 once per call; the sums run in FP32 on
 * the tensor cores; alpha, beta, C_in and the result stay FP64).  The stack of block
 * products is built on the device (section "Local multiplication": traversal and
 * generation) and each block shape runs as one batched launch (section "Batched
 * execution"), with the tuned launch configuration when the tune table has one.
 * stats may be NULL; when given, the call synchronises and fills it.
 * Errors: EINVAL (null handle, A, B, C with different block sizes, unknown prec,
 * eps_filter < 0 or NaN), ESTATE (A, B, or C when beta != 0, not finalized), ECAPACITY
 * (more than 262,144 block rows), ENOMEM (device memory), ECUDA.  On error C is
 * unchanged unless the failure happened after the new blocks were installed (ECUDA).
 */
dbcsr_status dbcsr_multiply(double alpha, dbcsr_matrix A, dbcsr_matrix B, double beta, dbcsr_matrix C,
                            double eps_filter, int32_t prec, dbcsr_mult_stats* stats);

/*
 * Planned products on fixed patterns (DBCSR's multiply with a retained sparsity, for
 * repeated products whose patterns do not change, as in an SCF loop).
 *
 * dbcsr_multiply_plan computes C = alpha * A * B once, like dbcsr_multiply with beta = 0,
 * and keeps what its numeric phase needs: the product stacks (built with the norm-bound
 * prescreen on the current values), the per-shape block lists and, for BF16 kinds, the
 * packed operands.  C receives the formed pattern; blocks whose norm is below eps_filter
 * are set to zero instead of removed, so the pattern stays fixed.  The numeric phase
 * (packing, block products, zeroing) is captured as one CUDA graph.
 * dbcsr_multiply_execute replays it on C's stream: C = alpha * A * B on C's planned
 * pattern, with the current values of A and B (change them with dbcsr_put_values), and
 * no host synchronisation.  A block product whose prescreen bound was below eps at plan
 * time stays excluded.
 *   - A, B, C: finalized (C may be empty), C distinct from A and B, equal block sizes.
 *     While the plan lives, their arrays are pinned: put_block, finalize, filter, copy into
 *     them, multiply into C and destroy fail with DBCSR_ESTATE.  Values may change.
 *   - prec: DBCSR_FP64, DBCSR_BF16 or DBCSR_BF16X3.  stats (may be NULL): of the plan's
 *     first product.
 *   - *out: the plan, owned by the caller; dbcsr_plan_destroy waits for its executions
 *     and frees it (NULL accepted).
 * Errors: as dbcsr_multiply, and EINVAL for C aliasing A or B; ECUDA if the graph cannot
 * be captured.  Not from the paper's text beyond DBCSR's operations.
 */
/*
 * How the FP64 block products of a product are launched (section "Local multiplication":
 * block products are batched into stacks and the stacks executed by the small-matrix kernels).
 *   DBCSR_SCHEDULE_PER_SHAPE (default): one launch per (m, n) block shape, each with the
 *     configuration of the tune table (dbcsr_autotune) or the default;
 *   DBCSR_SCHEDULE_QUEUE: one launch for every shape: the warps take C blocks from one work
 *     queue (an atomic counter over the shape lists) and run the single-warp kernel of each
 *     block's shape (K-split where m n = 32 EF + 1).  Products with a shape of more than 17
 *     element slots per lane (m n > 544) keep the per-shape launches.
 * Every C element is summed in the same order either way; the block norms differ only in
 * rounding where the per-shape schedule uses warp pairs.  Library-wide; not from the paper.
 * Errors: EINVAL (unknown mode).
 */
#define DBCSR_SCHEDULE_PER_SHAPE 0
#define DBCSR_SCHEDULE_QUEUE 1
dbcsr_status dbcsr_set_fp64_schedule(int32_t mode);
int32_t dbcsr_get_fp64_schedule(void);

typedef struct dbcsr_plan_* dbcsr_plan;
dbcsr_status dbcsr_multiply_plan(double alpha, dbcsr_matrix A, dbcsr_matrix B, dbcsr_matrix C, double eps_filter,
                                 int32_t prec, dbcsr_plan* out, dbcsr_mult_stats* stats);
dbcsr_status dbcsr_multiply_execute(dbcsr_plan plan);
dbcsr_status dbcsr_plan_destroy(dbcsr_plan plan);

/*
 * Replaces every value of the finalized matrix m, keeping its pattern: data holds nelem
 * doubles, the blocks row-major in block-CSR order (the layout of dbcsr_export);
 * on_device as for dbcsr_put_blocks.  Allowed while a plan uses m.  Host sources are
 * copied before the call returns.
 */
dbcsr_status dbcsr_put_values(dbcsr_matrix m, const double* data, int on_device);

/* Removes the blocks of m with Frobenius norm strictly below eps (diagonal blocks kept). */
dbcsr_status dbcsr_filter(dbcsr_matrix m, double eps);

/* *out = Tr(A) (synchronises). */
dbcsr_status dbcsr_trace(dbcsr_matrix A, double* out);

/* *out = Tr(A * B) = sum_IJ <A_IJ, B_JI^T>, without forming the product (synchronises). */
dbcsr_status dbcsr_trace_product(dbcsr_matrix A, dbcsr_matrix B, double* out);

/*
 * *out_dev = Tr(A * B), like dbcsr_trace_product, but allocating nothing.  The
 * paper has no counterpart: this entry point exists for callers that may not
 * allocate device memory during the call -- an application whose own arena owns
 * the GPU memory, code recording a CUDA graph that must not contain allocations,
 * or a loop that cannot pay for the allocator.
 *   - out_dev: device pointer to one double, owned by the caller; written in
 *     stream order on A's stream.  The call does not synchronise; read the value
 *     after the stream has reached it.  A and B must share that stream.
 *   - Scratch is a fixed device array inside the library (8 MB + 8 KB on every
 *     GPU that loads it, kept until the process exits), so A may hold at most
 *     1,048,576 blocks; larger A fails with DBCSR_ECAPACITY before any work.
 *   - The first call on each device looks up the array's device address with
 *     that device current; make that first call before any stream capture.
 *   - All calls share the one array: calls whose work overlaps on the GPU (on
 *     different streams, or from several threads) race and give wrong values.
 *     Each call writes every scratch word before reading it.
 *   - Same kernels and summation order as dbcsr_trace_product.
 */
dbcsr_status dbcsr_trace_product_noalloc(dbcsr_matrix A, dbcsr_matrix B, double* out_dev);

/* *out = max_i sum_j |(A - mu 1)_ij| (Gershgorin bound of the spectral radius; synchronises). */
dbcsr_status dbcsr_gershgorin(dbcsr_matrix A, double mu, double* out);

/*
 * Density matrix by the sign iteration (section "Sign-Method"; S = 1):
 *   X_0 = (H - mu 1) / alpha, alpha = dbcsr_gershgorin(H, mu);
 *   repeat: X2 = filter(X X); r = ||X2 - 1||_F / N; stop if r < tol;
 *           X <- filter(X p(X2));
 *   P_out = (1 - X) / 2.
 * opts->order picks p.  Order 2 (default) is the Newton-Schulz step, taken as
 * X <- filter(1.5 X - 0.5 X X2) (= X (3 - X^2) / 2).  Orders 3 to 7 are the polynomial
 * Pade steps p(y) = sum_{j <= order-1} binom(2j, j) / 4^j (1 - y)^j; order 5 is the
 * printed X (35 X^8 - 180 X^6 + 378 X^4 - 420 X^2 + 315) / 128.  They evaluate p in
 * powers of Y2 = filter(X2 X2) with a filter after every product: 3, 4, 4, 5 and 5
 * products per iteration for orders 3, 4, 5, 6 and 7 (order 5: X2, Y2, Y2 U, X U).
 * H must be symmetric with every diagonal block present.  P_out receives the
 * result (its previous content is replaced).  rep may be NULL.  Returns
 * DBCSR_ENOTCONV (P_out and rep still filled) when max_iter or the stall test
 * ended the iteration before r < tol.
 */
dbcsr_status dbcsr_sign_iterate(dbcsr_matrix H, double mu, const dbcsr_sign_opts* opts, dbcsr_matrix P_out,
                                dbcsr_sign_report* rep);

/*
 * Checkpoint / resume of the sign iteration (no counterpart in the paper).  The state of
 * the iteration after k steps is (X_k, k, the tier of the next product): X from a run with
 * DBCSR_SIGN_RETURN_X that max_iter = k stopped (possibly written with dbcsr_save and read
 * back with dbcsr_load), k and the switch step from that run's report `prev`.  The call
 * continues the iteration from there with opts (the same options as the first run, max_iter
 * counting all steps), the stall test looking back into prev's residual history, and fills
 * P_out and rep as dbcsr_sign_iterate would (rep continues prev's histories and totals).
 * An FP64 iteration, and a mixed one resumed after its switch to FP64, take exactly the
 * products of the uninterrupted run: the resumed P equals its P bit for bit.  Resumed inside
 * a split-BF16 tier, the tensor-core tier regroups the blocks of X, so the products agree to
 * rounding.  X is not modified.  Errors: EINVAL (null arguments, block sizes of X or P_out
 * not those of H, a report with a negative or too long history); as dbcsr_sign_iterate.
 */
dbcsr_status dbcsr_sign_iterate_resume(dbcsr_matrix H, dbcsr_matrix X, const dbcsr_sign_report* prev,
                                       const dbcsr_sign_opts* opts, dbcsr_matrix P_out, dbcsr_sign_report* rep);

/*
 * S^(-1/2) and S^(1/2) of a symmetric positive definite S (section "Sign-Method": the
 * sign of the block matrix [[0, A], [1, 0]] is [[0, A^(1/2)], [A^(-1/2), 0]]).  The sign
 * iteration of order opts->order runs on that block matrix in its coupled form, on
 * A = S / g with g = dbcsr_gershgorin(S, 0):
 *   Y_0 = A, Z_0 = 1;  repeat: W = filter(Z Y); r = ||W - 1||_F / N; stop if r < tol;
 *                               U = p(W); Y <- filter(Y U); Z <- filter(U Z);
 *   S_invsqrt = Z / sqrt(g), S_sqrt = sqrt(g) Y.
 * With the precision ladder (prec DBCSR_MIXED), Y = A Z is restored in FP64 at the
 * switch (the iteration does not undo the low tier's perturbations of A by itself).
 * p is the step polynomial of dbcsr_sign_iterate (order 2: U = (3 - W) / 2).  opts as
 * for dbcsr_sign_iterate (eps_filter, tol, max_iter, prec FP64 or MIXED with switch_tol,
 * stall_ratio, order, DBCSR_SIGN_FULL_PRODUCTS / DBCSR_SIGN_PLAIN_BF16); the
 * low-precision correction is refused.  S_sqrt may be NULL.  The outputs are replaced
 * and must differ from S and from each other.  rep (may be NULL): iterations,
 * residuals, alpha = g, nnzb_x = blocks of Z, work and times; trace_p and e_band are 0.
 * Returns DBCSR_ENOTCONV (outputs and rep still filled) when max_iter or the stall test
 * ended the iteration.  Errors: EINVAL, ESTATE, ENOMEM, ENAN, ECUDA.
 */
dbcsr_status dbcsr_inverse_sqrt(dbcsr_matrix S, const dbcsr_sign_opts* opts, dbcsr_matrix S_invsqrt,
                                dbcsr_matrix S_sqrt, dbcsr_sign_report* rep);

/*
 * A^-1 of a symmetric positive definite A by Hotelling's iteration (section
 * "Preconditioners": X <- X (2 1 - A X), the iterates filtered):
 *   X_0 = 1 / g, g = dbcsr_gershgorin(A, 0);
 *   repeat: T = filter(A X); r = ||T - 1||_F / N; stop if r < tol; X <- filter(2 X - X T).
 * The unfiltered residual squares at every step, (1 - A X') = (1 - A X)^2.  Products are
 * mirrored (X is a polynomial in A) unless DBCSR_SIGN_FULL_PRODUCTS.  opts: eps_filter,
 * tol, max_iter, stall_ratio, verbose, flags; prec must be DBCSR_FP64.  A_inv is replaced
 * and must differ from A.  rep (may be NULL): iterations, residuals, alpha = g, work.
 * Returns DBCSR_ENOTCONV when max_iter or the stall test ended the iteration.
 */
dbcsr_status dbcsr_inverse_hotelling(dbcsr_matrix A, const dbcsr_sign_opts* opts, dbcsr_matrix A_inv,
                                     dbcsr_sign_report* rep);

/*
 * Density matrix in a non-orthogonal basis (section "Sign-Method"):
 *   P = (1 - sign(S^-1 K - mu 1)) S^-1 / 2,
 * evaluated through the similarity sign(S^-1 K - mu 1) = S^(-1/2) sign(K' - mu 1) S^(1/2)
 * with K' = S^(-1/2) K S^(-1/2):
 *   S^(-1/2) by dbcsr_inverse_sqrt (same opts), K' = filter(filter(S^(-1/2) K) S^(-1/2)),
 *   P' = dbcsr_sign_iterate(K', mu, opts), P = filter(filter(S^(-1/2) P') S^(-1/2)).
 * The four congruence products run in FP64.  K and S symmetric with the same block sizes,
 * every diagonal block present; P_out is replaced and must differ from K and S.
 * rep (may be NULL): the sign iteration's report, with trace_p = Tr(P S) (the occupied
 * count), e_band = Tr(P K), and the congruences' work and the square root's time included
 * in flops / ms_multiply / ms_total.  rep_sqrt (may be NULL): the square root's report.
 * Returns DBCSR_ENOTCONV (P_out and the reports still filled) when either iteration
 * ended before its tolerance.  Errors: as dbcsr_sign_iterate.
 */
dbcsr_status dbcsr_sign_iterate_nonorth(dbcsr_matrix K, dbcsr_matrix S, double mu, const dbcsr_sign_opts* opts,
                                        dbcsr_matrix P_out, dbcsr_sign_report* rep, dbcsr_sign_report* rep_sqrt);

/*
 * Canonical density matrix without a chemical potential (section "Purification
 * methods": CP2K's trace-conserving TC2 and trace-resetting TRS4; the steps follow the
 * published algorithms of Niklasson (2002) and Niklasson, Tymczak and Challacombe (2003)):
 *   X_0 = (g 1 - H) / (2 g), g = dbcsr_gershgorin(H, 0);
 *   repeat: e = (Tr X - Tr X^2) / N; stop when |e| < tol;
 *     DBCSR_PURIFY_TC2:  X <- X^2 if Tr X > n_occ, else 2 X - X^2;
 *     DBCSR_PURIFY_TRS4: X2 = X^2, gamma = (n_occ - Tr F) / Tr G with F = X2 (4 X - 3 X2),
 *       G = X2 (1 - X)^2; gamma in [0, 6]: X <- F + gamma G; gamma > 6: 2 X - X2;
 *       gamma < 0: X2.
 *   P_out = X, the projector on the n_occ lowest states of H (H symmetric, a gap after
 *   state n_occ, every diagonal block present).
 * Every product is filtered with eps_filter (and mirrored unless DBCSR_SIGN_FULL_PRODUCTS).
 * opts: eps_filter, tol, max_iter (default 100), verbose, flags; prec must be DBCSR_FP64.
 * rep (may be NULL): iterations = steps, residual_history = e before each step, alpha = g,
 * trace_p = Tr P, e_band = Tr(P H), work and times.  Returns DBCSR_ENOTCONV (P_out and
 * rep still filled) after max_iter steps.  Errors: EINVAL (unknown method, n_occ outside
 * [0, N], ...), ESTATE, ENOMEM, ENAN, ECUDA.
 */
/*
 * Density matrix by the submatrix method (section "Submatrix Method"): one dense
 * principal submatrix per block column j, over I_j = the pattern of column j of H (the
 * atom and the atoms overlapping it), purified densely; block (i, j) of P_out, i in I_j,
 * is taken from submatrix j.  P_out receives H's pattern (H symmetric in pattern).
 *   X_0 = (H[I_j, I_j] - mu 1) / alpha, alpha = dbcsr_gershgorin(H, mu), padded to a
 *   multiple of 16 with an identity block; all submatrices of one padded size run as one
 *   batch of dense Newton-Schulz steps X <- 1.5 X - 0.5 X X^2 until every
 *   ||X^2 - 1||_F / n_pad < tol; P = (1 - X) / 2 on the taken blocks.
 * The dense products are strided-batched cuBLAS GEMMs.  opts: tol, max_iter, verbose;
 * prec DBCSR_FP64 (DGEMM) or DBCSR_MIXED (FP32: TF32 tensor-core GEMMs while the largest
 * residual is >= switch_tol, default 1e-3, then plain FP32 GEMMs; tol must then stay
 * above the FP32 rounding floor, about 1e-6).  eps_filter is not used.  rep: iterations
 * (the most of any batch), residual (the largest), fp64_from = the first step after the
 * TF32 phase, n_products = submatrices, flops = dense GEMM flops, trace_p, e_band.
 * Returns DBCSR_ENOTCONV when a batch ended at max_iter.  Errors: EINVAL (a missing
 * diagonal block, ...), ESTATE, ENOMEM, ENAN, ECUDA.
 */
dbcsr_status dbcsr_submatrix_sign(dbcsr_matrix H, double mu, const dbcsr_sign_opts* opts, dbcsr_matrix P_out,
                                  dbcsr_sign_report* rep);

#define DBCSR_PURIFY_TC2 1
#define DBCSR_PURIFY_TRS4 2
dbcsr_status dbcsr_purify(dbcsr_matrix H, double n_occ, int32_t method, const dbcsr_sign_opts* opts,
                          dbcsr_matrix P_out, dbcsr_sign_report* rep);

/*
 * The sign method with its chemical potential placed for a canonical occupation
 * (section "Purification methods": extra iterations that find mu): mu bisects
 * [mu_lo, mu_hi] (NaN: the Gershgorin interval [-g, g] of H), one dbcsr_sign_iterate per
 * trial, until |Tr P(mu) - n_occ| < 1/2.  *mu_out and *evaluations (may be NULL) receive
 * the final mu and the number of trials (at most 60); rep (may be NULL) the last trial's
 * report with the work and time of all trials.  Returns DBCSR_ENOTCONV when no trial
 * reached the occupation, or the last sign iteration did not converge.
 */
dbcsr_status dbcsr_sign_mu_search(dbcsr_matrix H, double n_occ, double mu_lo, double mu_hi, const dbcsr_sign_opts* opts,
                                  dbcsr_matrix P_out, double* mu_out, int32_t* evaluations, dbcsr_sign_report* rep);

/* Configuration of the FP64 block-product kernel of one (m, n, k) stack: its work split
 * and its launch.  The launch fields leave the arithmetic unchanged (every C element is
 * summed in the same order); split changes the rounding order only (the block norm's for a
 * warp pair, one remainder element's for the K-split). */
#define DBCSR_SPLIT_DEFAULT (-1) /* K-split when m n = 32 EF + 1, else a warp pair from 6 slots per lane */
#define DBCSR_SPLIT_WARP 0       /* one warp per C block, lane l owns elements l, l + 32, ... */
#define DBCSR_SPLIT_PAIR 1       /* two warps per C block, half of the element slots each (m n > 32, tpb % 64 == 0) */
#define DBCSR_SPLIT_K 2          /* 32 EF elements over the lanes, the last one summed along K by all lanes
                                    (m n = 32 EF + 1 only) */
typedef struct {
    int32_t tpb;          /* threads per CTA: 32 to 256, a multiple of 32 */
    int32_t ctas_per_sm;  /* grid = min(C blocks / warps per CTA, (SM count) * ctas_per_sm) */
    int32_t colmajor;     /* lane-to-element order, 0 row-major, 1 column-major */
    int32_t prefetch2;    /* 1 = fetch the next 32 products' metadata ahead */
    int32_t split;        /* DBCSR_SPLIT_* */
} dbcsr_kernel_cfg;

/* One timing of the autotuner. */
typedef struct {
    int32_t m, n, k, prec;
    dbcsr_kernel_cfg cfg;
    double ms;            /* median time of one launch over the synthetic stack */
    double gflops;        /* 2 m n k * stack_len / time */
} dbcsr_tune_record;

/* The configurations the autotuner times (prec DBCSR_FP64; the BF16 products run on the
 * tensor-core tier, one tile shape for every block shape, with nothing to tune per (m, n, k):
 * EINVAL): work splits x threads per CTA x CTAs per SM x lane order x metadata prefetch.
 * Not every configuration applies to every shape (a warp pair needs m n > 32, the K-split
 * m n = 32 EF + 1); the tuner, the model's choice and the table skip or reject those.
 * *n receives their number; up to cap of them are written to out (may be NULL). */
dbcsr_status dbcsr_tune_space(int32_t prec, dbcsr_kernel_cfg* out, int32_t cap, int32_t* n);

/*
 * Autotuner (section "Batched execution": kernels are tuned per (m, n, k) over
 * their parameters and the best parameter set kept).  For each triple
 * mnk[3t..3t+2] (each in [1, 32]) a synthetic stack of stack_len products is
 * built on the device, imitating one shape launch of a real product: C blocks of
 * 32 products, A/B blocks drawn at random from pools of about 512 MB together
 * (several times the L2).  Real launches hold 1e4 to 1e6 C blocks, so stack_len
 * of 5e5 or more gives timings that carry over.  Every configuration of
 * dbcsr_tune_space is launched reps times
 * (median taken) and the fastest becomes the tuned entry (prec, m, n, k) that
 * dbcsr_multiply uses for its m x n blocks when the largest block edge of the
 * matrix is k.  Up to cap timings go to recs (may be NULL); *nrec = their total.
 */
dbcsr_status dbcsr_autotune(const int32_t* mnk, int32_t ntriples, int32_t prec, int64_t stack_len, int32_t reps,
                            dbcsr_tune_record* recs, int64_t cap, int64_t* nrec);

/* Times ncfg given configurations on the synthetic (m, n, k) stack: ms_out[i] (EINVAL when one
 * does not apply to the shape). */
dbcsr_status dbcsr_time_config(int32_t prec, int32_t m, int32_t n, int32_t k, int64_t stack_len, int32_t reps,
                               const dbcsr_kernel_cfg* cfgs, int32_t ncfg, double* ms_out);

/* Tune table: set (cfg NULL removes), get (*found = 0 and the default when absent),
 * clear, and save/load as text lines "prec m n k tpb ctas_per_sm colmajor prefetch2 split". */
dbcsr_status dbcsr_tune_set(int32_t prec, int32_t m, int32_t n, int32_t k, const dbcsr_kernel_cfg* cfg);
dbcsr_status dbcsr_tune_get(int32_t prec, int32_t m, int32_t n, int32_t k, dbcsr_kernel_cfg* cfg, int* found);
dbcsr_status dbcsr_tune_clear(void);
dbcsr_status dbcsr_tune_save(const char* path);
dbcsr_status dbcsr_tune_load(const char* path);

/*
 * Performance-prediction MLP (section "Batched execution": the autotuning data
 * train a model that predicts near-optimal parameters of the untuned kernels).
 * Model: DBCSR_MLP_FEATURES inputs -> 64 ReLU -> 64 ReLU -> 1, FP32, trained on
 * the GPU (full-batch mean squared error, Adam); parameters are a flat host
 * array of dbcsr_mlp_param_count(nfeat) floats:
 *   W1[64][nfeat], b1[64], W2[64][64], b2[64], W3[64], b3.
 * Targets are whatever the caller regresses (the tests use standardised log times).
 */
#define DBCSR_MLP_FEATURES 12

typedef struct {
    int32_t epochs;       /* full-batch Adam steps */
    int32_t reserved;
    double lr, beta1, beta2, eps;
} dbcsr_mlp_opts;

typedef struct {
    float loss_first;     /* mean squared error before the first step */
    float loss_last;      /* after the last step */
    double ms;            /* device time of the training */
    int32_t epochs;
    int32_t reserved;
} dbcsr_mlp_report;

int64_t dbcsr_mlp_param_count(int32_t nfeat);

/* Glorot-uniform weights (SplitMix64 stream of seed), zero biases, into params. */
dbcsr_status dbcsr_mlp_init(int32_t nfeat, uint64_t seed, float* params);

/* Features of samples (m, n, k, cfg): mnk[3i..3i+2], cfgs[i] -> out[i * DBCSR_MLP_FEATURES ...]:
 * m/32, n/32, k/32, log2(m n k)/15, useful fraction of the lane slots, K-split flag, tpb/256,
 * log2(ctas_per_sm)/6, colmajor, prefetch2, warp-pair flag, element slots per lane / 32 (the
 * work split resolved for the shape).  EINVAL when a configuration does not apply. */
dbcsr_status dbcsr_mlp_features(int32_t prec, const int32_t* mnk, const dbcsr_kernel_cfg* cfgs, int64_t n, float* out);

/* y_out[b] = model(X[b * nfeat ...]) for B samples (host arrays; runs on the GPU). */
dbcsr_status dbcsr_mlp_forward(int32_t nfeat, const float* params, const float* X, int64_t B, float* y_out);

/* Mean squared error over B samples and its gradient with respect to every parameter. */
dbcsr_status dbcsr_mlp_loss_grad(int32_t nfeat, const float* params, const float* X, const float* T, int64_t B,
                                 float* loss, float* grad);

/* Trains params in place: opts->epochs full-batch Adam steps on the GPU. */
dbcsr_status dbcsr_mlp_train(int32_t nfeat, float* params, const float* X, const float* T, int64_t B,
                             const dbcsr_mlp_opts* opts, dbcsr_mlp_report* rep);

/* For each triple, the configuration of dbcsr_tune_space(prec) with the lowest
 * predicted value (and that value in best_pred, may be NULL).  params == NULL takes the
 * model dbcsr_predictor_train keeps for prec (ESTATE if there is none). */
dbcsr_status dbcsr_mlp_predict_best(int32_t prec, const float* params, const int32_t* mnk, int32_t ntriples,
                                    dbcsr_kernel_cfg* best, float* best_pred);

/*
 * The autotuner's timings as a records file (text, one record per line:
 * "prec m n k tpb ctas_per_sm colmajor prefetch2 split ms", a '#' line first), the input of
 * dbcsr_predictor_train.  append = 0 truncates the file and writes the header line;
 * append = 1 adds the records after those already there.  Errors: EINVAL (bad argument,
 * file not writable).  Not from the paper (a file format of this library).
 */
dbcsr_status dbcsr_tune_records_save(const char* path, const dbcsr_tune_record* recs, int64_t n, int32_t append);

/*
 * Trains the performance-prediction model on the autotuner's timings (section "Batched
 * execution": the tuning data train a model that predicts parameters for the kernels
 * nobody tuned).  From the records of precision prec in the records file tune_records:
 *   - features of each (m, n, k, configuration) as dbcsr_mlp_features;
 *   - target = log(ms) minus the mean log(ms) of the record's (m, n, k) triple, divided
 *     by the standard deviation of these centred values over all the records (population
 *     form, at least 1e-12): the model learns how the configuration changes a triple's time;
 *   - Glorot-uniform initial weights from seed (dbcsr_mlp_init), then opts->epochs
 *     full-batch Adam steps on the GPU (dbcsr_mlp_train; rep receives its losses and time).
 * The trained parameters are kept by the library, one model per precision (a later call
 * replaces it): dbcsr_mlp_predict_best and dbcsr_tune_predicted use it when given
 * params == NULL, and dbcsr_predictor_params copies it out.
 * Errors: EINVAL (null opts, unreadable or malformed file, no record of prec, a record out
 * of range), those of dbcsr_mlp_train.
 */
dbcsr_status dbcsr_predictor_train(const char* tune_records, int32_t prec, uint64_t seed, const dbcsr_mlp_opts* opts,
                                   dbcsr_mlp_report* rep);

/* The features (X[n * DBCSR_MLP_FEATURES]) and targets (T[n]) dbcsr_predictor_train builds
 * from a records file, on the host: *n receives the number of records of prec; up to cap of
 * them are written (X and T may be NULL).  Errors as dbcsr_predictor_train's file checks. */
dbcsr_status dbcsr_predictor_data(const char* tune_records, int32_t prec, float* X, float* T, int64_t cap,
                                  int64_t* n);

/* Copies the model kept for prec (dbcsr_mlp_param_count(DBCSR_MLP_FEATURES) floats) into
 * params.  Errors: EINVAL (null params), ESTATE (no model trained for prec). */
dbcsr_status dbcsr_predictor_params(int32_t prec, float* params);

/*
 * The prediction with the exhaustive autotune as its fallback and measured time deciding
 * (section "Batched execution": the model fills in the untuned kernels; the tuner
 * stays the reference).  For each triple mnk[3t..3t+2]:
 *   - the MLP (params, as for dbcsr_mlp_predict_best) picks a configuration;
 *   - the prediction and the default configuration are timed on the synthetic stack
 *     (stack_len products, median of reps launches);
 *   - if the prediction's time is at most (1 + tolerance) times the default's, it enters
 *     the tune table; otherwise every configuration of dbcsr_tune_space is timed on that
 *     stack and the fastest enters the table.
 * fell_back[t] (may be NULL) receives 1 where the exhaustive search ran.  params == NULL
 * takes the model dbcsr_predictor_train keeps for prec.
 * Errors: EINVAL (bad argument or triple), and those of dbcsr_mlp_predict_best.
 */
dbcsr_status dbcsr_tune_predicted(int32_t prec, const float* params, const int32_t* mnk, int32_t ntriples,
                                  int64_t stack_len, int32_t reps, double tolerance, int32_t* fell_back);

/*
 * Batched dense product C[b] = alpha A[b] B[b] + beta C[b], b < nb, for row-major n x n
 * matrices at A + b n^2, B + b n^2, C + b n^2 in device memory (the caller's; the library
 * allocates only its packing scratch), on the stream given (cudaStream_t, may be NULL).
 * The submatrix method's dense step (section "Submatrix Method") runs on it.
 *   prec DBCSR_FP64: double data, FP64 pipe;
 *   DBCSR_TF32 / DBCSR_TF32X3: float data on the TF32 tensor cores, plain or split (three
 *   products of TF32 halves, close to FP32 arithmetic).
 * C must not overlap A or B.  Returns after the product completes.  Errors: EINVAL (bad
 * argument, other prec), ECAPACITY (nb > 65535), ENOMEM, ETIMEOUT (a bounded wait of the
 * tensor-core kernel ran out), ECUDA.
 */
dbcsr_status dbcsr_dense_multiply(int32_t prec, int64_t nb, int32_t n, double alpha, const void* A, const void* B,
                                  double beta, void* C, void* stream);

/*
 * Sharding over several GPUs (section "DBCSR library": block rows and columns distributed over
 * the processes, products by Cannon's algorithm with asynchronous point-to-point messages).
 * Here a matrix is split into domains of block rows, one per rank; C = A B then needs on each
 * rank the rows of B indexed by the block columns of its rows of A -- its own rows and a halo
 * of neighbouring rows -- so one exchange of halo rows per product suffices and scalars
 * (residual, traces) take one sum over the ranks.  Both calls are host-only (no GPU, no
 * matrix handle): they take a block pattern as host arrays (row_ptr[nblk + 1], col[nnzb],
 * columns in [0, nblk)).
 *
 * dbcsr_partition_rows: owner[nblk] receives the rank (0 .. nparts-1) of every block row.
 * The domains come from recursive bisection of the block graph (I ~ J when block (I, J) is
 * present): each part is ordered by breadth-first distance from a far block and cut at the
 * median of the row weights (blocks per row + 1), so domains are compact regions of the
 * coupling graph, found without coordinates.  Deterministic.  A rank may receive no row when
 * nparts is close to nblk.  Errors: EINVAL (bad pattern, nparts outside [1, nblk]).
 *
 * dbcsr_halo_rows: the block rows that rank's rows reference through their block columns but
 * that other ranks own, ascending: *n receives their number, up to cap are written to halo.
 * Errors: EINVAL.
 */
dbcsr_status dbcsr_partition_rows(int32_t nblk, const int64_t* row_ptr, const int32_t* col, int32_t nparts,
                                  int32_t* owner);
dbcsr_status dbcsr_halo_rows(int32_t nblk, const int64_t* row_ptr, const int32_t* col, const int32_t* owner,
                             int32_t rank, int32_t* halo, int32_t cap, int32_t* n);

/*
 * Solves nsys independent systems H[s] (each symmetric, all diagonal blocks
 * present, any block sizes) as one batch: the matrices are stacked into one
 * block-diagonal matrix, so every product forms all systems' blocks in the same
 * kernel launches (one per block-shape class) -- the paper's batching of block
 * products into stacks (section "Local multiplication") applied across systems.
 * Per system: X_0 = (H[s] - mu[s] 1) / alpha_s with its own Gershgorin bound,
 * its own residual ||X2_s - 1||_F / N_s, convergence and stall tests as in
 * dbcsr_sign_iterate, and the step of opts->order (2 to 7).  A system that
 * converges or stalls writes its P_out and leaves the batch (the matrices are
 * compacted to the running systems).  With DBCSR_MIXED the batch leaves the BF16
 * tier once any system's residual is below switch_tol.
 *   H[nsys], mu[nsys] (host arrays); P_out[nsys]: created by the caller with the
 *   block sizes of H[s], receive (1 - X_s) / 2; reps[nsys] (may be NULL):
 *   per-system iterations, residuals, alpha, Tr(P), E_band; flops, products and
 *   times are the batch totals.  Work runs on H[0]'s stream.  Returns
 *   DBCSR_ENOTCONV if any system stopped without reaching tol.
 */
dbcsr_status dbcsr_sign_iterate_batched(int32_t nsys, const dbcsr_matrix* H, const double* mu,
                                        const dbcsr_sign_opts* opts, dbcsr_matrix* P_out,
                                        dbcsr_sign_report* reps);

#ifdef __cplusplus
}
#endif

#endif /* DBCSR_GB_H */
