/*
 * dbcsr_gb_bench.h -- measurement helpers of the GB300 block-sparse library.
 *
 * These calls have no counterpart in the paper: they measure the machine (the
 * FP64 rates that bound the FP64 block products) and count kernel launches, so
 * that reported throughput can be set against a roofline.
 */
#ifndef DBCSR_GB_BENCH_H
#define DBCSR_GB_BENCH_H

#include <stdint.h>

#include "dbcsr_gb.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Kinds of dbcsr_bench_peak. */
#define DBCSR_PEAK_DFMA 0   /* FP64 fused multiply-add on the CUDA cores */
#define DBCSR_PEAK_DMMA 1   /* FP64 tensor-core mma.sync m8n8k4 */

/*
 * Runs a compute-only loop of the given kind on the current device: `blocks`
 * CTAs of `threads` threads, each issuing `iters` rounds of independent
 * operations, timed with CUDA events.  Returns the achieved rate in GFLOP/s
 * (2 flops per FMA), or a negative value on error (dbcsr_last_error() says why).
 * threads must be a multiple of 32 in [32, 1024]; blocks in [1, 65535]; iters >= 1.
 */
double dbcsr_bench_peak(int32_t kind, int32_t iters, int32_t blocks, int32_t threads);

/* Number of kernels this library has launched in this process so far. */
int64_t dbcsr_launch_count(void);

/*
 * Device memory of the library's stream-ordered pool on the current device: bytes in use
 * now (*used_now) and the most in use at once since the last reset (*used_high); either
 * pointer may be NULL.  reset_high != 0 then restarts the high-water mark at the current
 * use.  Lets a caller check that a call allocated nothing (allocation-free entry points).
 * Returns 0, or a dbcsr_status code on a CUDA error.
 */
int32_t dbcsr_pool_usage(int64_t* used_now, int64_t* used_high, int32_t reset_high);

/*
 * Self-test of the bounded device-side waits every persistent kernel of the library uses:
 * one CTA waits on an mbarrier for at most limit_cycles SM clock cycles (limit_cycles >= 0).
 * arrive != 0: a thread of the CTA arrives first, so the wait completes (DBCSR_OK);
 * arrive == 0: nothing ever arrives, the wait runs out and the call returns DBCSR_ETIMEOUT,
 * the context staying usable.  *waited (nullable) receives the cycles the wait took.
 */
int32_t dbcsr_wait_selftest(int64_t limit_cycles, int32_t arrive, int64_t* waited);

/*
 * The block groups of the tensor-core tier, built now from m's block norms (a BF16 product with
 * m as A builds the same groups when m carries none): the block rows are merged along their
 * strongest couplings -- every row's 12 largest off-diagonal block norms, ties to the lower
 * column, taken in decreasing norm (then lower row, then lower column) -- as long as a group
 * keeps at most 112 rows and 16 blocks.  Host outputs, each nullable: g_of[nblk] the group of
 * every block row (groups numbered in the order of their first block), norms[nnzb] the FP64
 * block Frobenius norms the couplings were ranked by (m's block order), *ngrp the number of
 * groups.  m is not changed.  Errors: DBCSR_ESTATE if m is not finalized; DBCSR_ECUDA.
 */
int32_t dbcsr_matrix_groups(dbcsr_matrix m, int32_t* g_of, double* norms, int32_t* ngrp);

#ifdef __cplusplus
}
#endif

#endif /* DBCSR_GB_BENCH_H */
