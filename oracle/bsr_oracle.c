/*
 * Plain FP64 block-CSR oracle.  TEST INFRASTRUCTURE ONLY: tests, the smoke check
 * and the benchmark's CPU-baseline leg call it; the product path never does.
 *
 * What it computes follows the paper's DBCSR section ("Local multiplication"):
 * a block-sparse product is a sum of small dense block products
 * C_IJ += A_IK * B_KJ over the block-CSR pattern, traversing A's block rows and,
 * for each, B's block columns.  Written as plainly as possible: one block row of
 * C per loop iteration, a row-local accumulator, the sum over K taken in
 * ascending K and, inside a block product, in ascending k; no blocking, no
 * reordering, no BLAS.  Compiled with -ffp-contract=off so that a*b + c is
 * never fused (rounding is the same on every host).  OpenMP only splits the
 * block rows between threads; every C element is summed by one thread in the
 * fixed order above, so the result does not depend on the thread count.
 *
 * Matrix layout (shared with the input generator, not with the CUDA library):
 *   bs[nblk]      block edge of block row/column I
 *   rp[nblk+1]    int64 row pointers into the block list
 *   col[nnzb]     int32 block columns, ascending within a row
 *   boff[nnzb]    int64 offset of each block in data (blocks row-major)
 *   roff[nblk+1]  int64 first matrix row of block row I
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

static int cmp_i32(const void* a, const void* b) {
    int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
    return (x > y) - (x < y);
}

/* Collects the distinct block columns of row I of A*B (and of C_in when given). */
static int64_t row_pattern(int32_t I, const int64_t* a_rp, const int32_t* a_col,
                           const int64_t* b_rp, const int32_t* b_col,
                           const int64_t* c_rp, const int32_t* c_col,
                           unsigned char* mark, int32_t* list) {
    int64_t n = 0;
    for (int64_t p = a_rp[I]; p < a_rp[I + 1]; ++p) {
        int32_t K = a_col[p];
        for (int64_t q = b_rp[K]; q < b_rp[K + 1]; ++q) {
            int32_t J = b_col[q];
            if (!mark[J]) { mark[J] = 1; list[n++] = J; }
        }
    }
    if (c_col) {
        for (int64_t q = c_rp[I]; q < c_rp[I + 1]; ++q) {
            int32_t J = c_col[q];
            if (!mark[J]) { mark[J] = 1; list[n++] = J; }
        }
    }
    for (int64_t t = 0; t < n; ++t) mark[list[t]] = 0;
    return n;
}

/* Number of blocks in each row of the pattern of A*B (union C_in's pattern if c_col != NULL). */
int oracle_mm_count(int32_t nblk, const int64_t* a_rp, const int32_t* a_col,
                    const int64_t* b_rp, const int32_t* b_col,
                    const int64_t* c_rp, const int32_t* c_col, int64_t* out_cnt) {
    int err = 0;
#pragma omp parallel
    {
        unsigned char* mark = (unsigned char*)calloc((size_t)nblk + 1, 1);
        int32_t* list = (int32_t*)malloc(sizeof(int32_t) * ((size_t)nblk + 1));
        if (!mark || !list) {
#pragma omp atomic write
            err = 1;
        } else {
#pragma omp for schedule(dynamic, 16)
            for (int32_t I = 0; I < nblk; ++I)
                out_cnt[I] = row_pattern(I, a_rp, a_col, b_rp, b_col, c_rp, c_col, mark, list);
        }
        free(mark);
        free(list);
    }
    return err;
}

/* Sorted block columns of every row of the pattern; out_rp from oracle_mm_count's prefix sum. */
int oracle_mm_pattern(int32_t nblk, const int64_t* a_rp, const int32_t* a_col,
                      const int64_t* b_rp, const int32_t* b_col,
                      const int64_t* c_rp, const int32_t* c_col,
                      const int64_t* out_rp, int32_t* out_col) {
    int err = 0;
#pragma omp parallel
    {
        unsigned char* mark = (unsigned char*)calloc((size_t)nblk + 1, 1);
        int32_t* list = (int32_t*)malloc(sizeof(int32_t) * ((size_t)nblk + 1));
        if (!mark || !list) {
#pragma omp atomic write
            err = 1;
        } else {
#pragma omp for schedule(dynamic, 16)
            for (int32_t I = 0; I < nblk; ++I) {
                int64_t n = row_pattern(I, a_rp, a_col, b_rp, b_col, c_rp, c_col, mark, list);
                qsort(list, (size_t)n, sizeof(int32_t), cmp_i32);
                memcpy(out_col + out_rp[I], list, sizeof(int32_t) * (size_t)n);
            }
        }
        free(mark);
        free(list);
    }
    return err;
}

/*
 * C = alpha * A*B + beta * C_in on C's (precomputed) pattern, no filtering.
 * out_stats[0] = number of block products A_IK*B_KJ, out_stats[1] = sum of 2*m*k*n.
 */
int oracle_mm_numeric(int32_t nblk, const int32_t* bs,
                      double alpha,
                      const int64_t* a_rp, const int32_t* a_col, const int64_t* a_boff, const double* a_data,
                      const int64_t* b_rp, const int32_t* b_col, const int64_t* b_boff, const double* b_data,
                      double beta,
                      const int64_t* ci_rp, const int32_t* ci_col, const int64_t* ci_boff, const double* ci_data,
                      const int64_t* c_rp, const int32_t* c_col, const int64_t* c_boff, double* c_data,
                      int64_t* out_stats) {
    int err = 0;
    int64_t nprod = 0, nflop = 0;
    int32_t maxbs = 0;
    for (int32_t I = 0; I < nblk; ++I) if (bs[I] > maxbs) maxbs = bs[I];
#pragma omp parallel reduction(+ : nprod, nflop)
    {
        int64_t* pos = (int64_t*)malloc(sizeof(int64_t) * ((size_t)nblk + 1));
        size_t cap = 0;
        double* acc = NULL;
        if (!pos) {
#pragma omp atomic write
            err = 1;
        } else {
            for (int32_t J = 0; J <= nblk; ++J) pos[J] = -1;    /* not in C's pattern */
#pragma omp for schedule(dynamic, 8)
            for (int32_t I = 0; I < nblk; ++I) {
                const int64_t m = bs[I];
                /* accumulator: the blocks of C row I, one after the other, row-major */
                int64_t width = 0;
                for (int64_t q = c_rp[I]; q < c_rp[I + 1]; ++q) {
                    pos[c_col[q]] = m * width;
                    width += bs[c_col[q]];
                }
                size_t need = (size_t)(m * width) + 1;
                if (need > cap) {
                    free(acc);
                    cap = need * 2;
                    acc = (double*)malloc(sizeof(double) * cap);
                    if (!acc) {
#pragma omp atomic write
                        err = 1;
                        cap = 0;
                        continue;
                    }
                }
                for (int64_t e = 0; e < m * width; ++e) acc[e] = 0.0;
                for (int64_t p = a_rp[I]; p < a_rp[I + 1]; ++p) {
                    const int32_t K = a_col[p];
                    const int64_t k = bs[K];
                    const double* a = a_data + a_boff[p];
                    for (int64_t q = b_rp[K]; q < b_rp[K + 1]; ++q) {
                        const int32_t J = b_col[q];
                        if (pos[J] < 0) continue;   /* a candidate the caller left out (prescreen) */
                        const int64_t n = bs[J];
                        const double* b = b_data + b_boff[q];
                        double* c = acc + pos[J];
                        for (int64_t i = 0; i < m; ++i)
                            for (int64_t j = 0; j < n; ++j) {
                                double s = c[i * n + j];
                                for (int64_t kk = 0; kk < k; ++kk) s = s + a[i * k + kk] * b[kk * n + j];
                                c[i * n + j] = s;
                            }
                        nprod += 1;
                        nflop += 2 * m * n * k;
                    }
                }
                /* epilogue: alpha * sum + beta * C_in (C_in row merged by column) */
                int64_t r = ci_rp ? ci_rp[I] : 0;
                const int64_t rend = ci_rp ? ci_rp[I + 1] : 0;
                for (int64_t q = c_rp[I]; q < c_rp[I + 1]; ++q) {
                    const int32_t J = c_col[q];
                    const int64_t area = m * bs[J];
                    const double* s = acc + pos[J];
                    double* out = c_data + c_boff[q];
                    while (r < rend && ci_col[r] < J) ++r;
                    if (r < rend && ci_col[r] == J) {
                        const double* ci = ci_data + ci_boff[r];
                        for (int64_t e = 0; e < area; ++e) out[e] = alpha * s[e] + beta * ci[e];
                    } else {
                        for (int64_t e = 0; e < area; ++e) out[e] = alpha * s[e];
                    }
                }
                for (int64_t q = c_rp[I]; q < c_rp[I + 1]; ++q) pos[c_col[q]] = -1;
            }
        }
        free(pos);
        free(acc);
    }
    out_stats[0] = nprod;
    out_stats[1] = nflop;
    return err;
}

/*
 * The norm-bound prescreen of a product, for every candidate block (I, J) of a pattern of
 * alpha*A*B + beta*C_in (c_rp, c_col): bound = |alpha| sum_K ||A_IK|| ||B_KJ|| in ascending K,
 * plus |beta| ||C_in,IJ|| where C_in has the block; keep[q] = 1 if I == J or bound >= eps_lo.
 * By the triangle inequality and ||XY||_F <= ||X||_F ||Y||_F the block's norm is at most its
 * bound, so a block left out has norm below eps_lo and the filter would drop it.
 */
int oracle_prescreen(int32_t nblk, double abs_alpha,
                     const int64_t* a_rp, const int32_t* a_col, const double* a_norm,
                     const int64_t* b_rp, const int32_t* b_col, const double* b_norm,
                     double abs_beta, const int64_t* ci_rp, const int32_t* ci_col, const double* ci_norm,
                     const int64_t* c_rp, const int32_t* c_col, double eps_lo, int32_t* keep) {
    int err = 0;
#pragma omp parallel
    {
        int64_t* pos = (int64_t*)malloc(sizeof(int64_t) * ((size_t)nblk + 1));
        double* bound = (double*)malloc(sizeof(double) * ((size_t)nblk + 1));
        if (!pos || !bound) {
#pragma omp atomic write
            err = 1;
        } else {
            for (int32_t J = 0; J <= nblk; ++J) pos[J] = -1;
#pragma omp for schedule(dynamic, 8)
            for (int32_t I = 0; I < nblk; ++I) {
                for (int64_t q = c_rp[I]; q < c_rp[I + 1]; ++q) {
                    pos[c_col[q]] = q - c_rp[I];
                    bound[q - c_rp[I]] = 0.0;
                }
                for (int64_t p = a_rp[I]; p < a_rp[I + 1]; ++p) {
                    const int32_t K = a_col[p];
                    const double na = abs_alpha * a_norm[p];
                    for (int64_t q = b_rp[K]; q < b_rp[K + 1]; ++q) {
                        const int64_t t = pos[b_col[q]];
                        if (t >= 0) bound[t] = bound[t] + na * b_norm[q];
                    }
                }
                if (ci_rp)
                    for (int64_t r = ci_rp[I]; r < ci_rp[I + 1]; ++r) {
                        const int64_t t = pos[ci_col[r]];
                        if (t >= 0) bound[t] = bound[t] + abs_beta * ci_norm[r];
                    }
                for (int64_t q = c_rp[I]; q < c_rp[I + 1]; ++q) {
                    keep[q] = (c_col[q] == I || bound[q - c_rp[I]] >= eps_lo) ? 1 : 0;
                    pos[c_col[q]] = -1;
                }
            }
        }
        free(pos);
        free(bound);
    }
    return err;
}

/*
 * Per-block Frobenius norm ||M_IJ||_F = sqrt(sum of squares, row-major order) and
 * per-block squared distance to the identity ||M_IJ - delta_IJ 1||_F^2.
 */
void oracle_block_norms(int64_t nnzb, const int32_t* rows, const int32_t* col, const int32_t* bs,
                        const int64_t* boff, const double* data, double* norm, double* dev2) {
#pragma omp parallel for schedule(static)
    for (int64_t b = 0; b < nnzb; ++b) {
        const int64_t m = bs[rows[b]], n = bs[col[b]];
        const double* x = data + boff[b];
        double s = 0.0, d = 0.0;
        for (int64_t i = 0; i < m; ++i)
            for (int64_t j = 0; j < n; ++j) {
                double v = x[i * n + j];
                s = s + v * v;
                double w = (rows[b] == col[b] && i == j) ? v - 1.0 : v;
                d = d + w * w;
            }
        norm[b] = sqrt(s);
        dev2[b] = d;
    }
}

/* ||M - 1||_F^2: sum of dev2 in block order, plus m for each block row whose diagonal block is absent. */
double oracle_sum_dev2(int32_t nblk, const int32_t* bs, const int64_t* rp, const int32_t* col, const double* dev2) {
    double s = 0.0;
    for (int32_t I = 0; I < nblk; ++I) {
        int has_diag = 0;
        for (int64_t q = rp[I]; q < rp[I + 1]; ++q) {
            s = s + dev2[q];
            if (col[q] == I) has_diag = 1;
        }
        if (!has_diag) s = s + (double)bs[I];
    }
    return s;
}

/* Tr(M): sum of the diagonal entries of the diagonal blocks, block rows ascending. */
double oracle_trace(int32_t nblk, const int32_t* bs, const int64_t* rp, const int32_t* col,
                    const int64_t* boff, const double* data) {
    double s = 0.0;
    for (int32_t I = 0; I < nblk; ++I)
        for (int64_t q = rp[I]; q < rp[I + 1]; ++q)
            if (col[q] == I) {
                const int64_t m = bs[I];
                for (int64_t i = 0; i < m; ++i) s = s + data[boff[q] + i * m + i];
            }
    return s;
}

static int64_t find_block(const int64_t* rp, const int32_t* col, int32_t row, int32_t c) {
    int64_t lo = rp[row], hi = rp[row + 1];
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (col[mid] < c) lo = mid + 1; else hi = mid;
    }
    return (lo < rp[row + 1] && col[lo] == c) ? lo : -1;
}

/*
 * Tr(A*B) = sum_{I,J} sum_{i,j} A_IJ[i][j] * B_JI[j][i].  Per block row I a
 * partial sum is formed (blocks of A's row in order, entries row-major); the
 * partials are then added in ascending I.
 */
double oracle_trace_product(int32_t nblk, const int32_t* bs,
                            const int64_t* a_rp, const int32_t* a_col, const int64_t* a_boff, const double* a_data,
                            const int64_t* b_rp, const int32_t* b_col, const int64_t* b_boff, const double* b_data) {
    double* part = (double*)calloc((size_t)nblk + 1, sizeof(double));
    if (!part) return NAN;
#pragma omp parallel for schedule(dynamic, 16)
    for (int32_t I = 0; I < nblk; ++I) {
        double s = 0.0;
        const int64_t m = bs[I];
        for (int64_t p = a_rp[I]; p < a_rp[I + 1]; ++p) {
            const int32_t J = a_col[p];
            const int64_t q = find_block(b_rp, b_col, J, I);
            if (q < 0) continue;
            const int64_t n = bs[J];
            const double* a = a_data + a_boff[p];
            const double* b = b_data + b_boff[q];
            for (int64_t i = 0; i < m; ++i)
                for (int64_t j = 0; j < n; ++j) s = s + a[i * n + j] * b[j * m + i];
        }
        part[I] = s;
    }
    double t = 0.0;
    for (int32_t I = 0; I < nblk; ++I) t = t + part[I];
    free(part);
    return t;
}

/* Absolute row sums of (M - mu 1), one per matrix row (Gershgorin discs). */
void oracle_abs_row_sums(int32_t nblk, const int32_t* bs, const int64_t* roff, const int64_t* rp,
                         const int32_t* col, const int64_t* boff, const double* data, double mu, double* out) {
#pragma omp parallel for schedule(dynamic, 16)
    for (int32_t I = 0; I < nblk; ++I) {
        const int64_t m = bs[I];
        for (int64_t i = 0; i < m; ++i) out[roff[I] + i] = 0.0;
        int has_diag = 0;
        for (int64_t q = rp[I]; q < rp[I + 1]; ++q) {
            const int32_t J = col[q];
            const int64_t n = bs[J];
            const double* x = data + boff[q];
            if (J == I) has_diag = 1;
            for (int64_t i = 0; i < m; ++i)
                for (int64_t j = 0; j < n; ++j) {
                    double v = x[i * n + j];
                    if (J == I && i == j) v = v - mu;
                    out[roff[I] + i] = out[roff[I] + i] + fabs(v);
                }
        }
        if (!has_diag)
            for (int64_t i = 0; i < m; ++i) out[roff[I] + i] = out[roff[I] + i] + fabs(mu);
    }
}

int oracle_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Threads of the parallel loops that follow (n >= 1); for timing the oracle on one core. */
void oracle_set_num_threads(int n) {
#ifdef _OPENMP
    if (n >= 1) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/*
 * One block of the product: out = alpha * sum_K A_IK * B_KJ (ascending K, then k)
 * + beta * ci (ci may be NULL).  Used to check single outputs of large products.
 */
void oracle_mm_block(int32_t I, int32_t J, const int32_t* bs, double alpha,
                     const int64_t* a_rp, const int32_t* a_col, const int64_t* a_boff, const double* a_data,
                     const int64_t* b_rp, const int32_t* b_col, const int64_t* b_boff, const double* b_data,
                     double beta, const double* ci, double* out) {
    const int64_t m = bs[I], n = bs[J];
    for (int64_t e = 0; e < m * n; ++e) out[e] = 0.0;
    for (int64_t p = a_rp[I]; p < a_rp[I + 1]; ++p) {
        const int32_t K = a_col[p];
        const int64_t k = bs[K];
        /* find B_KJ */
        int64_t lo = b_rp[K], hi = b_rp[K + 1];
        while (lo < hi) {
            int64_t mid = lo + (hi - lo) / 2;
            if (b_col[mid] < J) lo = mid + 1; else hi = mid;
        }
        if (!(lo < b_rp[K + 1] && b_col[lo] == J)) continue;
        const double* a = a_data + a_boff[p];
        const double* b = b_data + b_boff[lo];
        for (int64_t i = 0; i < m; ++i)
            for (int64_t j = 0; j < n; ++j) {
                double s = out[i * n + j];
                for (int64_t kk = 0; kk < k; ++kk) s = s + a[i * k + kk] * b[kk * n + j];
                out[i * n + j] = s;
            }
    }
    for (int64_t e = 0; e < m * n; ++e) out[e] = ci ? alpha * out[e] + beta * ci[e] : alpha * out[e];
}
