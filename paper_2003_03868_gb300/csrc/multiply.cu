// The block-sparse product C = beta*C + alpha*A*B followed by the eps_filter
// truncation (DBCSR sections "Local multiplication" and "Batched execution";
// the filter is from section "Sign-Method").
//
// The paper separates *what* to multiply (CPU traversal + batch generation) from
// *performing* the batches (SMM kernels).  Here both halves run on the GPU:
//
//  1. k_cand_count   per block row I: bitmap (shared memory) of the block columns
//                    J reached through A_IK B_KJ (and C_IJ when beta != 0).
//  2. k_cand_bound   per row: the candidates in ascending J, and for each the
//                    exact norm bound |alpha| sum_K ||A_IK|| ||B_KJ|| (+ |beta|
//                    ||C_IJ||), the product count and sum of k.  A candidate
//                    whose bound is below eps can only be filtered away, so it
//                    is not formed (diagonal blocks always are).
//  3. k_form_meta    compacted list of formed blocks with their product-list
//                    offsets (prefix sums) and data offsets.
//  4. k_fill_stack   per row: the product stack (a_blk, b_blk), grouped by C
//                    block and in ascending K inside each group.
//  5. k_smm_f64      output-stationary batched small GEMM: one warp (or a pair of
//                    warps for large blocks) owns one C block and sums its
//                    products in stack order (no atomics); the epilogue applies
//                    alpha/beta and writes the block norm.  BF16 products run on
//                    the tensor-core tier instead (lowtier.cu).
//     With a symmetric result only the blocks I <= J are computed; k_mirror_copy
//     copies the others as transposes and k_sym_diag takes the symmetric part of
//     the diagonal blocks.
//  6. filter         blocks with norm < eps dropped (diagonal kept), compaction.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <utility>
#include <vector>

#include "common.cuh"
#include "smm.cuh"

namespace dbg {

// Largest number of block rows: the per-row bitmap and its rank table live in
// shared memory (2 * 4 bytes per 32 block columns).
constexpr int32_t kMaxBlockRows = 262144;

namespace {

constexpr int kSymThreads = 256;
// Shared memory kept for per-row candidate accumulators (the rest goes to global).
constexpr int kSymSmemBudget = 96 * 1024;

__device__ __forceinline__ int block_excl_scan_int(int v, int* sh, int& total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sh[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int t = lane < nw ? sh[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        sh[lane] = t;
    }
    __syncthreads();
    const int excl = (warp ? sh[warp - 1] : 0) + x - v;
    total = sh[nw - 1];
    __syncthreads();
    return excl;
}

struct RowPattern {
    const int64_t* a_rp; const int32_t* a_col;
    const int64_t* b_rp; const int32_t* b_col;
    const int64_t* c_rp; const int32_t* c_col;   // C_in pattern (beta != 0) or null
};

// Bitmap of the candidate block columns of row I; returns the candidate count
// and fills wpre with the exclusive prefix popcount of the words.
__device__ int build_row(const RowPattern& P, int32_t I, uint32_t* bm, int* wpre, int nwords, int* sh_scan) {
    for (int w = threadIdx.x; w < nwords; w += blockDim.x) bm[w] = 0u;
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int64_t p = P.a_rp[I] + warp; p < P.a_rp[I + 1]; p += nw) {
        const int32_t K = P.a_col[p];
        for (int64_t q = P.b_rp[K] + lane; q < P.b_rp[K + 1]; q += 32) {
            const int32_t J = P.b_col[q];
            atomicOr(&bm[J >> 5], 1u << (J & 31));
        }
    }
    if (P.c_col)
        for (int64_t q = P.c_rp[I] + threadIdx.x; q < P.c_rp[I + 1]; q += blockDim.x) {
            const int32_t J = P.c_col[q];
            atomicOr(&bm[J >> 5], 1u << (J & 31));
        }
    __syncthreads();
    const int per = (nwords + blockDim.x - 1) / blockDim.x;
    const int lo = min(nwords, (int)threadIdx.x * per), hi = min(nwords, lo + per);
    int s = 0;
    for (int w = lo; w < hi; ++w) s += __popc(bm[w]);
    int total;
    int run = block_excl_scan_int(s, sh_scan, total);
    for (int w = lo; w < hi; ++w) {
        wpre[w] = run;
        run += __popc(bm[w]);
    }
    __syncthreads();
    return total;
}

__device__ __forceinline__ int rank_of(const uint32_t* bm, const int* wpre, int32_t J) {
    return wpre[J >> 5] + __popc(bm[J >> 5] & ((1u << (J & 31)) - 1u));
}

__global__ void k_cand_count(int32_t nblk, RowPattern P, int nwords, int64_t* __restrict__ ccnt,
                             unsigned long long* __restrict__ max_row) {
    extern __shared__ uint32_t smem[];
    __shared__ int sh_scan[32];
    uint32_t* bm = smem;
    int* wpre = (int*)(smem + nwords);
    for (int32_t I = blockIdx.x; I < nblk; I += gridDim.x) {
        const int n = build_row(P, I, bm, wpre, nwords, sh_scan);
        if (threadIdx.x == 0) {
            ccnt[I] = n;
            atomicMax(max_row, (unsigned long long)n);
            atomicMax(max_row + 1, (unsigned long long)(P.a_rp[I + 1] - P.a_rp[I]));
        }
        __syncthreads();
    }
}

struct BoundArgs {
    double abs_alpha, abs_beta, eps_lo;
    const double* a_norm; const double* b_norm; const double* c_norm;
    const int32_t* bs;
    const int64_t* coff;
    int32_t* cand_row; int32_t* cand_col;
    double* bound; int32_t* pcnt; int32_t* ksum; int64_t* cin;
    int32_t* keep;
    int use_smem;
    int use_fast;            // FP32 upper bound with atomics (needs use_smem and < 4096 terms per candidate)
    const float* b_norm_ru;  // use_fast: B's norms rounded up to FP32, once per block
};

// B's block norms rounded up to FP32 for the fast bound: one conversion per block instead of one
// per (K, J) term (the FP64 pipe that converts runs at a few operations per clock per SM).
__global__ void k_norms_f32_ru(int64_t n, const double* __restrict__ in, float* __restrict__ out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = __double2float_ru(in[i]);
}

// The norm bound is accumulated in FP32 with shared-memory atomics, in any order, so the
// K loop needs no barrier.  Each term is scaled up by (1 + 2^-10) before it is added; with
// fewer than 2^12 terms per candidate (checked by the caller, or the exact FP64 path runs)
// the FP32 rounding of the sum stays below that margin, so the result is an upper bound of
// the exact bound and a candidate is skipped only when its exact bound is below eps_lo.
// Which near-threshold blocks are formed may then vary from run to run; the filtered
// result cannot (a block whose norm reaches eps always has its bound above eps_lo).
__global__ void k_cand_bound(int32_t nblk, RowPattern P, int nwords, BoundArgs B) {
    extern __shared__ uint32_t smem[];
    __shared__ int sh_scan[32];
    uint32_t* bm = smem;
    int* wpre = (int*)(smem + nwords);
    double* sh_bound = (double*)(smem + 2 * ((nwords + 1) & ~1));
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int32_t I = blockIdx.x; I < nblk; I += gridDim.x) {
        const int nc = build_row(P, I, bm, wpre, nwords, sh_scan);
        const int64_t cb = B.coff[I];
        double* bnd = B.use_smem ? sh_bound : B.bound + cb;
        int32_t* pc = B.use_smem ? (int32_t*)(sh_bound + nc) : B.pcnt + cb;
        int32_t* ks = B.use_smem ? pc + nc : B.ksum + cb;
        float* fb = (float*)(pc + 2 * nc);      // use_fast: FP32 bounds after the counters
        // candidates in ascending J
        for (int w = threadIdx.x; w < nwords; w += blockDim.x) {
            uint32_t bits = bm[w];
            int r = wpre[w];
            while (bits) {
                const int b = __ffs(bits) - 1;
                bits &= bits - 1u;
                B.cand_col[cb + r] = 32 * w + b;
                B.cand_row[cb + r] = I;
                bnd[r] = 0.0;
                pc[r] = 0;
                ks[r] = 0;
                if (B.use_fast) fb[r] = 0.f;
                if (B.cin) B.cin[cb + r] = -1;
                ++r;
            }
        }
        __syncthreads();
        if (P.c_col)
            for (int64_t q = P.c_rp[I] + threadIdx.x; q < P.c_rp[I + 1]; q += blockDim.x)
                B.cin[cb + rank_of(bm, wpre, P.c_col[q])] = q;
        if (B.use_fast) {
            // warps over K, lanes over the blocks of B's row K, no barrier
            for (int64_t p = P.a_rp[I] + warp; p < P.a_rp[I + 1]; p += nw) {
                const int32_t K = P.a_col[p];
                const float na = (float)(B.abs_alpha * B.a_norm[p]) * 1.0009765625f;
                const int kk = B.bs[K];
                for (int64_t q = P.b_rp[K] + lane; q < P.b_rp[K + 1]; q += 32) {
                    const int r = rank_of(bm, wpre, P.b_col[q]);
                    atomicAdd(&fb[r], __fmul_ru(na, B.b_norm_ru[q]));
                    atomicAdd(&pc[r], 1);
                    atomicAdd(&ks[r], kk);
                }
            }
            __syncthreads();
            for (int r = threadIdx.x; r < nc; r += blockDim.x) bnd[r] = (double)fb[r] * 1.0009765625;
        } else {
            __syncthreads();
            // ascending K, one K at a time: every accumulator is updated in a fixed order
            for (int64_t p = P.a_rp[I]; p < P.a_rp[I + 1]; ++p) {
                const int32_t K = P.a_col[p];
                const double na = B.abs_alpha * B.a_norm[p];
                const int kk = B.bs[K];
                for (int64_t q = P.b_rp[K] + threadIdx.x; q < P.b_rp[K + 1]; q += blockDim.x) {
                    const int r = rank_of(bm, wpre, P.b_col[q]);
                    bnd[r] = bnd[r] + na * B.b_norm[q];
                    pc[r] += 1;
                    ks[r] += kk;
                }
                __syncthreads();
            }
        }
        __syncthreads();
        for (int r = threadIdx.x; r < nc; r += blockDim.x) {
            double b = bnd[r];
            const int64_t ci = B.cin ? B.cin[cb + r] : -1;
            if (ci >= 0) b += B.abs_beta * B.c_norm[ci];
            const int32_t J = B.cand_col[cb + r];
            B.keep[cb + r] = (J == I || b >= B.eps_lo) ? 1 : 0;
            if (B.use_smem) {
                B.pcnt[cb + r] = pc[r];
                B.ksum[cb + r] = ks[r];
            }
        }
        __syncthreads();
    }
}

// FP64 launch classes: 1..32 padded (E = ceil(m n / 32)); 33 + EF for m n = 32 EF + 1
// (EF = 1..31, K-split remainder of one element).  A K-split of more elements
// (13x13: EF = 5, R = 9) measured slower than the padded class, because the
// lanes' own products differ in k and the remainder loop diverges.
constexpr int kF64ClassKs1 = 33, kF64Classes = 65;


__global__ void k_form_meta(int64_t ncand, const int32_t* __restrict__ keep, const int64_t* __restrict__ kidx,
                            const int32_t* __restrict__ cand_row, const int32_t* __restrict__ cand_col,
                            const int32_t* __restrict__ pcnt, const int32_t* __restrict__ ksum,
                            const int64_t* __restrict__ cin, const int32_t* __restrict__ bs,
                            int32_t* __restrict__ f_row, int32_t* __restrict__ f_col, int64_t* __restrict__ f_area,
                            int64_t* __restrict__ f_np, int64_t* __restrict__ f_cin, int32_t* __restrict__ f_ksum) {
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < ncand; c += (int64_t)gridDim.x * blockDim.x) {
        if (!keep[c]) continue;
        const int64_t k = kidx[c];
        const int32_t I = cand_row[c], J = cand_col[c];
        f_row[k] = I;
        f_col[k] = J;
        f_area[k] = (int64_t)bs[I] * bs[J];
        f_np[k] = pcnt[c];
        f_cin[k] = cin ? cin[c] : -1;
        f_ksum[k] = ksum[c];
    }
}

// With a symmetric result (sym != 0), each formed block's twin (J, I) is looked up:
// mirror[k] = its index, or -1 if the twin was not formed.  Blocks then take one of
// three roles: computed (diagonal, or I < J with a formed twin), copied as the
// twin's transpose (I > J with a formed twin), or dropped (no formed twin: the
// exact product is symmetric, so the twin's bound below eps -- or its absence from
// the pattern -- bounds this block too; what is left is asymmetric rounding noise).
// Without sym every block is computed.
__global__ void k_find_mirror(int64_t nform, const int32_t* __restrict__ f_row, const int32_t* __restrict__ f_col,
                              const int64_t* __restrict__ f_rp, int64_t* __restrict__ mirror) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nform; k += (int64_t)gridDim.x * blockDim.x) {
        const int32_t I = f_row[k], J = f_col[k];
        int64_t src = -1;
        if (I != J) {
            int64_t lo = f_rp[J], hi = f_rp[J + 1];
            while (lo < hi) {
                const int64_t mid = (lo + hi) >> 1;
                if (f_col[mid] < I) lo = mid + 1; else hi = mid;
            }
            if (lo < f_rp[J + 1] && f_col[lo] == I) src = lo;
        } else {
            src = k;
        }
        mirror[k] = src;
    }
}

// role of formed block k: 0 computed, 1 copied from its twin, 2 dropped.
// sym = 1 (mirror): I < J computed, I > J copied; sym = 2 (average): both twins
// computed and then replaced by their symmetric mean; blocks without a formed twin
// are dropped in both modes.
// grp (BF16 products, nullable): blocks are ordered by their group first, so that all the
// computed blocks between two groups lie in one group tile of the tensor-core tier.
__device__ __forceinline__ int block_role(int sym, int32_t I, int32_t J, int64_t mirror, const int32_t* grp) {
    if (!sym || I == J) return 0;
    if (mirror < 0) return 2;
    if (sym == 2) return 0;
    const bool first = grp ? (grp[I] < grp[J] || (grp[I] == grp[J] && I < J)) : I < J;
    return first ? 0 : 1;
}

// One warp: the m x m block P becomes (P + P^T) / 2 in place; *sq and *d receive the
// lane's share of its squared norm and squared distance to 1.
__device__ __forceinline__ void sym_diag_block(double* P, int m, int lane, double* sq, double* d) {
    for (int e = lane; e < m * m; e += 32) {
        const int i = e / m, j = e - i * m;
        if (i < j) {
            const double v = 0.5 * (P[i * m + j] + P[j * m + i]);
            P[i * m + j] = v;
            P[j * m + i] = v;
        }
    }
    __syncwarp();
    double s = 0.0, t = 0.0;
    for (int e = lane; e < m * m; e += 32) {
        const int i = e / m, j = e - i * m;
        const double v = P[e];
        s = fma(v, v, s);
        const double w = (i == j) ? v - 1.0 : v;
        t = fma(w, w, t);
    }
    *sq = s;
    *d = t;
}

// sym = 1 (mirror): the diagonal blocks, computed in full, become their symmetric parts, so
// that the result is exactly symmetric.  A diagonal block of A B is symmetric only as far
// as A and B commute (and, in split BF16, only to the order of its FP32 sums); with
// mirrored off-diagonal blocks an antisymmetric part left there grows from product to
// product instead of dying out.  One warp per block row.
__global__ void k_sym_diag(int32_t nblk, const int64_t* __restrict__ f_rp, const int32_t* __restrict__ f_col,
                           const int64_t* __restrict__ f_off, const int32_t* __restrict__ bs,
                           double* __restrict__ c_data, double* __restrict__ c_norm, double* __restrict__ c_dev2) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t I = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); I < nblk; I += warps) {
        int64_t lo = f_rp[I], hi = f_rp[I + 1];
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if (f_col[mid] < I) lo = mid + 1; else hi = mid;
        }
        if (!(lo < f_rp[I + 1] && f_col[lo] == I)) continue;
        double sq, d;
        sym_diag_block(c_data + f_off[lo], bs[I], lane, &sq, &d);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            sq += __shfl_xor_sync(0xffffffffu, sq, o);
            d += __shfl_xor_sync(0xffffffffu, d, o);
        }
        if (lane == 0) {
            c_norm[lo] = sqrt(sq);
            c_dev2[lo] = d;
        }
    }
}

// sym = 2: C_IJ and C_JI become (C_IJ + C_JI^T) / 2 and its transpose, with their
// norms and distances to 1 (the pair is handled by the warp of its I < J block;
// diagonal blocks by their own warp).
__global__ void k_sym_average(int64_t nform, const int64_t* __restrict__ mirror, const int32_t* __restrict__ f_row,
                              const int32_t* __restrict__ f_col, const int64_t* __restrict__ f_off,
                              const int32_t* __restrict__ bs, double* __restrict__ c_data,
                              double* __restrict__ c_norm, double* __restrict__ c_dev2) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t k = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); k < nform; k += warps) {
        const int32_t I = f_row[k], J = f_col[k];
        const int64_t t = mirror[k];
        if (t < 0 || I > J) continue;
        const int m = bs[I], n = bs[J];
        double* P = c_data + f_off[k];
        double* Q = c_data + f_off[t];
        double sq = 0.0, d = 0.0;
        if (I == J) {
            sym_diag_block(P, m, lane, &sq, &d);
        } else {
            for (int e = lane; e < m * n; e += 32) {
                const int i = e / n, j = e - i * n;
                const double v = 0.5 * (P[e] + Q[j * m + i]);
                P[e] = v;
                Q[j * m + i] = v;
                sq = fma(v, v, sq);
            }
            d = sq;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            sq += __shfl_xor_sync(0xffffffffu, sq, o);
            d += __shfl_xor_sync(0xffffffffu, d, o);
        }
        if (lane == 0) {
            c_norm[k] = sqrt(sq);
            c_dev2[k] = d;
            if (I != J) {
                c_norm[t] = sqrt(sq);
                c_dev2[t] = sq;
            }
        }
    }
}

// Work of the blocks that are computed (not mirrored): flops, products, and a
// histogram by block shape (m, n).  Blocks that are copied or dropped get no product
// stack (f_np = 0, comp = 0).
__global__ void k_form_stats(int64_t nform, const int32_t* __restrict__ f_row, const int32_t* __restrict__ f_col,
                             int64_t* __restrict__ f_np, const int32_t* __restrict__ f_ksum,
                             const int64_t* __restrict__ mirror, int sym, const int32_t* __restrict__ bs,
                             unsigned long long* __restrict__ flops, unsigned long long* __restrict__ nprod,
                             unsigned long long* __restrict__ shape_cnt, uint8_t* __restrict__ comp,
                             const int32_t* __restrict__ grp) {
    // the shape histogram is gathered per CTA in shared memory (a few shapes take every block,
    // so global atomics per block would serialise on them) and added once per nonzero bin
    constexpr int kBins = (kMaxBlock + 1) * (kMaxBlock + 1);
    __shared__ unsigned int hist[kBins];
    for (int t = threadIdx.x; t < kBins; t += blockDim.x) hist[t] = 0;
    __syncthreads();
    unsigned long long lf = 0, lp = 0;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nform; k += (int64_t)gridDim.x * blockDim.x) {
        const bool computed = block_role(sym, f_row[k], f_col[k], mirror[k], grp) == 0;
        comp[k] = computed ? 1 : 0;
        if (!computed) {
            f_np[k] = 0;
            continue;
        }
        const int m = bs[f_row[k]], n = bs[f_col[k]];
        lf += 2ull * (unsigned long long)m * (unsigned long long)n * (unsigned long long)f_ksum[k];
        lp += (unsigned long long)f_np[k];
        atomicAdd(&hist[m * (kMaxBlock + 1) + n], 1u);
    }
    __syncthreads();
    for (int t = threadIdx.x; t < kBins; t += blockDim.x)
        if (hist[t]) atomicAdd(shape_cnt + t, (unsigned long long)hist[t]);
    for (int o = 16; o > 0; o >>= 1) {
        lf += __shfl_xor_sync(0xffffffffu, lf, o);
        lp += __shfl_xor_sync(0xffffffffu, lp, o);
    }
    if ((threadIdx.x & 31) == 0) {
        if (lf) atomicAdd(flops, lf);
        if (lp) atomicAdd(nprod, lp);
    }
}

// Copied blocks: C_IJ = C_JI^T (after every computed block is written), with their twin's
// norm and distance to 1 (never diagonal); dropped blocks get norm -1 so that the filter
// removes them.
__global__ void k_mirror_copy(int64_t nform, int sym, const int64_t* __restrict__ mirror,
                              const int32_t* __restrict__ f_row, const int32_t* __restrict__ f_col,
                              const int64_t* __restrict__ f_off, const int32_t* __restrict__ bs,
                              double* __restrict__ c_data, double* __restrict__ c_norm, double* __restrict__ c_dev2,
                              const int32_t* __restrict__ grp) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t k = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); k < nform; k += warps) {
        const int role = block_role(sym, f_row[k], f_col[k], mirror[k], grp);
        if (role == 0) continue;
        if (role == 2) {
            if (lane == 0) {
                c_norm[k] = -1.0;
                c_dev2[k] = 0.0;
            }
            continue;
        }
        const int64_t src = mirror[k];
        const int m = bs[f_row[k]], n = bs[f_col[k]];
        const double* S = c_data + f_off[src];
        double* D = c_data + f_off[k];
        // (i, j) of element e = i n + j, stepped by 32 elements without a division per element
        const int di = 32 / n, dj = 32 - di * n;
        int i = lane / n, j = lane - i * n;
        for (int e = lane; e < m * n; e += 32) {
            D[e] = S[j * m + i];
            i += di;
            j += dj;
            if (j >= n) {
                j -= n;
                ++i;
            }
        }
        // the transpose has its twin's norm and (off the diagonal) distance to 1: taken over, so
        // that the pair is kept or dropped together and no FP64 arithmetic bounds the copy
        if (lane == 0) {
            c_norm[k] = c_norm[src];
            c_dev2[k] = c_dev2[src];
        }
    }
}

__global__ void k_form_rp(int32_t nblk, const int64_t* __restrict__ coff, const int64_t* __restrict__ kidx,
                          int64_t* __restrict__ f_rp) {
    for (int32_t I = blockIdx.x * blockDim.x + threadIdx.x; I <= nblk; I += gridDim.x * blockDim.x)
        f_rp[I] = kidx[coff[I]];
}

struct FillArgs {
    const int64_t* coff;
    const int32_t* keep;
    const uint8_t* comp;     // per formed block: 1 if computed (only those get stack entries)
    const int64_t* kidx;
    const int64_t* pbeg;
    int32_t* cursor;
    int32_t* prod_a; int32_t* prod_b;
    int use_smem;
};

__global__ void k_fill_stack(int32_t nblk, RowPattern P, int nwords, FillArgs F) {
    extern __shared__ uint32_t smem[];
    __shared__ int sh_scan[32];
    uint32_t* bm = smem;
    int* wpre = (int*)(smem + nwords);
    // use_smem: per candidate of the row, its stack base (-1 if not formed) and cursor
    int64_t* sh_base = (int64_t*)(smem + 2 * ((nwords + 1) & ~1));
    for (int32_t I = blockIdx.x; I < nblk; I += gridDim.x) {
        const int nc = build_row(P, I, bm, wpre, nwords, sh_scan);
        const int64_t cb = F.coff[I];
        if (F.use_smem) {
            int32_t* cur = (int32_t*)(sh_base + nc);
            for (int r = threadIdx.x; r < nc; r += blockDim.x) {
                const int64_t c = cb + r;
                sh_base[r] = (F.keep[c] && F.comp[F.kidx[c]]) ? F.pbeg[F.kidx[c]] : -1;
                cur[r] = 0;
            }
            __syncthreads();
            for (int64_t p = P.a_rp[I]; p < P.a_rp[I + 1]; ++p) {
                const int32_t K = P.a_col[p];
                for (int64_t q = P.b_rp[K] + threadIdx.x; q < P.b_rp[K + 1]; q += blockDim.x) {
                    const int r = rank_of(bm, wpre, P.b_col[q]);
                    const int64_t b0 = sh_base[r];
                    if (b0 < 0) continue;
                    const int32_t at = cur[r];
                    cur[r] = at + 1;
                    F.prod_a[b0 + at] = (int32_t)p;
                    F.prod_b[b0 + at] = (int32_t)q;
                }
                __syncthreads();
            }
        } else {
            const int64_t kb = F.kidx[cb];
            const int nk = (int)(F.kidx[cb + nc] - kb);
            int32_t* cur = F.cursor + kb;
            for (int r = threadIdx.x; r < nk; r += blockDim.x) cur[r] = 0;
            __syncthreads();
            for (int64_t p = P.a_rp[I]; p < P.a_rp[I + 1]; ++p) {
                const int32_t K = P.a_col[p];
                for (int64_t q = P.b_rp[K] + threadIdx.x; q < P.b_rp[K + 1]; q += blockDim.x) {
                    const int64_t c = cb + rank_of(bm, wpre, P.b_col[q]);
                    if (!F.keep[c]) continue;
                    const int64_t k = F.kidx[c];
                    if (!F.comp[k]) continue;
                    const int32_t at = cur[k - kb];
                    cur[k - kb] = at + 1;
                    const int64_t pos = F.pbeg[k] + at;
                    F.prod_a[pos] = (int32_t)p;
                    F.prod_b[pos] = (int32_t)q;
                }
                __syncthreads();
            }
        }
    }
}

// ----------------------------------------------------------------- FP64 SMM
__device__ __forceinline__ void elem_of(int idx, int m, int n, int colmajor, int& i, int& j) {
    if (colmajor) {
        j = idx / m;
        i = idx - j * m;
    } else {
        i = idx / n;
        j = idx - i * n;
    }
}

struct ProdMeta {
    int64_t ao, bo;
    int kq;
};

__device__ __forceinline__ ProdMeta fetch_meta(const SmmArgs& S, int64_t base, int64_t pe, int lane) {
    ProdMeta m{0, 0, 0};
    if (base + lane < pe) {
        const int32_t ai = S.prod_a[base + lane], bi = S.prod_b[base + lane];
        m.ao = S.a_off[ai];
        m.bo = S.b_off[bi];
        m.kq = S.bs[S.a_col[ai]];
    }
    return m;
}

// One warp per C block of class E (m*n <= 32*E): lane l owns elements l, l+32,
// ..., sums its products in stack order (ascending K, then k) with FMA, and
// writes alpha*sum + beta*C_in plus the block's norm and distance to 1.  The
// lanes first fetch the metadata of 32 products at once (one product each:
// block offsets and inner size) and broadcast it with shuffles, so the
// dependent index loads are not paid product by product.
// C block k by one warp (or, PAIR, by the warp pair `pair`, this warp owning half `part` of
// the element slots; sh_part is the pairs' exchange area, parity its alternating slot).
template <int E, bool PAIR>
__device__ __forceinline__ void smm_block(int64_t k, const SmmArgs& S, int lane, int part, int pair, int parity,
                                          double (*sh_part)[2][2]) {
    constexpr int EL = PAIR ? (E + 1) / 2 : E;
    {
        const int I = S.f_row[k], J = S.f_col[k];
        const int m = S.bs[I], n = S.bs[J];
        const int mn = m * n;
        int ii[EL], jj[EL];
        double acc[EL];
#pragma unroll
        for (int e = 0; e < EL; ++e) {
            const int idx = lane + 32 * (part * EL + e);
            int i = 0, j = 0;
            if (idx < mn) elem_of(idx, m, n, S.colmajor, i, j);
            ii[e] = i;
            jj[e] = j;
            acc[e] = 0.0;
        }
        const int64_t pb = S.f_pbeg[k], pe = S.f_pbeg[k + 1];
        ProdMeta cur = fetch_meta(S, pb, pe, lane);
        for (int64_t base = pb; base < pe; base += 32) {
            const int cnt = (int)min((int64_t)32, pe - base);
            ProdMeta nxt{0, 0, 0};
            if (S.prefetch2) nxt = fetch_meta(S, base + 32, pe, lane);
            for (int q = 0; q < cnt; ++q) {
                const int64_t aoq = __shfl_sync(0xffffffffu, cur.ao, q);
                const int64_t boq = __shfl_sync(0xffffffffu, cur.bo, q);
                const int kk = __shfl_sync(0xffffffffu, cur.kq, q);
                const double* __restrict__ A = S.a_data + aoq;
                const double* __restrict__ B = S.b_data + boq;
                for (int t = 0; t < kk; ++t) {
#pragma unroll
                    for (int e = 0; e < EL; ++e)
                        acc[e] = fma(__ldg(A + ii[e] * kk + t), __ldg(B + t * n + jj[e]), acc[e]);
                }
            }
            cur = S.prefetch2 ? nxt : fetch_meta(S, base + 32, pe, lane);
        }
        const int64_t ci = S.f_cin[k];
        const double* cin = ci >= 0 ? S.ci_data + S.ci_off[ci] : nullptr;
        double* out = S.c_data + S.f_off[k];
        double sq = 0.0, d = 0.0;
#pragma unroll
        for (int e = 0; e < EL; ++e) {
            const int idx = lane + 32 * (part * EL + e);
            if (idx < mn) {
                const int pos = ii[e] * n + jj[e];
                double v = S.alpha * acc[e];
                if (cin) v = v + S.beta * cin[pos];
                out[pos] = v;
                sq = fma(v, v, sq);
                const double wv = (I == J && ii[e] == jj[e]) ? v - 1.0 : v;
                d = fma(wv, wv, d);
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            sq += __shfl_xor_sync(0xffffffffu, sq, o);
            d += __shfl_xor_sync(0xffffffffu, d, o);
        }
        if (PAIR) {
            // slot parity alternates, so one barrier per block suffices: the second half
            // can rewrite this slot only after passing the next block's barrier, which the
            // first half reaches after reading it
            if (part == 1 && lane == 0) {
                sh_part[pair][parity][0] = sq;
                sh_part[pair][parity][1] = d;
            }
            asm volatile("bar.sync %0, 64;" ::"r"(1 + pair) : "memory");
            if (part == 0 && lane == 0) {
                sq += sh_part[pair][parity][0];
                d += sh_part[pair][parity][1];
            }
        }
        if (part == 0 && lane == 0) {
            S.c_norm[k] = sqrt(sq);
            S.c_dev2[k] = d;
        }
    }
}

template <int E, bool PAIR>
__global__ void __launch_bounds__(256) k_smm_f64(int64_t nlist, const int64_t* __restrict__ list, SmmArgs S) {
    // PAIR: two warps (neighbours in the CTA) share one C block, each owning half of its
    // element slots, so a large block needs half the registers per thread; the halves'
    // norm sums meet in shared memory behind a 64-thread named barrier of the pair.
    __shared__ double sh_part[PAIR ? 4 : 1][2][2];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int part = PAIR ? (warp & 1) : 0, pair = PAIR ? (warp >> 1) : warp;
    const int per_cta = PAIR ? (blockDim.x >> 6) : (blockDim.x >> 5);
    const int64_t stride = (int64_t)gridDim.x * per_cta;
    int parity = 0;
    for (int64_t w = (int64_t)blockIdx.x * per_cta + pair; w < nlist; w += stride, parity ^= 1)
        smm_block<E, PAIR>(list[w], S, lane, part, pair, parity, sh_part);
}


// FP64 class with a K-split remainder: the first 32*EF elements of the block are
// spread over the lanes as in k_smm_f64, and the last R elements are summed along
// K instead: lane l takes the products l, l+32, ... of the block (the product
// whose metadata it fetched) for all R elements, and a fixed xor-shuffle tree adds
// the 32 partial sums.  For m*n = 32*EF + 1 (13x5, 5x13, 23x7, 7x23) this removes
// a 32-lane pass that would carry one useful element.
template <int EF, int R>
__device__ __forceinline__ void smm_block_ks(int64_t k, const SmmArgs& S, int lane) {
    {
        const int I = S.f_row[k], J = S.f_col[k];
        const int m = S.bs[I], n = S.bs[J];
        int ii[EF], jj[EF], ir[R], jr[R];
        double acc[EF], rem[R];
#pragma unroll
        for (int e = 0; e < EF; ++e) {
            elem_of(lane + 32 * e, m, n, S.colmajor, ii[e], jj[e]);
            acc[e] = 0.0;
        }
#pragma unroll
        for (int r = 0; r < R; ++r) {
            elem_of(32 * EF + r, m, n, S.colmajor, ir[r], jr[r]);
            rem[r] = 0.0;
        }
        const int64_t pb = S.f_pbeg[k], pe = S.f_pbeg[k + 1];
        ProdMeta cur = fetch_meta(S, pb, pe, lane);
        for (int64_t base = pb; base < pe; base += 32) {
            const int cnt = (int)min((int64_t)32, pe - base);
            ProdMeta nxt{0, 0, 0};
            if (S.prefetch2) nxt = fetch_meta(S, base + 32, pe, lane);
            for (int q = 0; q < cnt; ++q) {
                const int64_t aoq = __shfl_sync(0xffffffffu, cur.ao, q);
                const int64_t boq = __shfl_sync(0xffffffffu, cur.bo, q);
                const int kk = __shfl_sync(0xffffffffu, cur.kq, q);
                const double* __restrict__ A = S.a_data + aoq;
                const double* __restrict__ B = S.b_data + boq;
                for (int t = 0; t < kk; ++t) {
#pragma unroll
                    for (int e = 0; e < EF; ++e)
                        acc[e] = fma(__ldg(A + ii[e] * kk + t), __ldg(B + t * n + jj[e]), acc[e]);
                }
            }
            // remainder: this lane's own product (kq = 0 past the end of the list)
            const double* __restrict__ A = S.a_data + cur.ao;
            const double* __restrict__ B = S.b_data + cur.bo;
            for (int t = 0; t < cur.kq; ++t) {
#pragma unroll
                for (int r = 0; r < R; ++r)
                    rem[r] = fma(__ldg(A + ir[r] * cur.kq + t), __ldg(B + t * n + jr[r]), rem[r]);
            }
            cur = S.prefetch2 ? nxt : fetch_meta(S, base + 32, pe, lane);
        }
#pragma unroll
        for (int r = 0; r < R; ++r)
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) rem[r] += __shfl_xor_sync(0xffffffffu, rem[r], o);
        const int64_t ci = S.f_cin[k];
        const double* cin = ci >= 0 ? S.ci_data + S.ci_off[ci] : nullptr;
        double* out = S.c_data + S.f_off[k];
        double sq = 0.0, d = 0.0;
#pragma unroll
        for (int e = 0; e < EF; ++e) {
            const int pos = ii[e] * n + jj[e];
            double v = S.alpha * acc[e];
            if (cin) v = v + S.beta * cin[pos];
            out[pos] = v;
            sq = fma(v, v, sq);
            const double wv = (I == J && ii[e] == jj[e]) ? v - 1.0 : v;
            d = fma(wv, wv, d);
        }
#pragma unroll
        for (int r = 0; r < R; ++r)
            if (lane == r) {
                const int pos = ir[r] * n + jr[r];
                double v = S.alpha * rem[r];
                if (cin) v = v + S.beta * cin[pos];
                out[pos] = v;
                sq = fma(v, v, sq);
                const double wv = (I == J && ir[r] == jr[r]) ? v - 1.0 : v;
                d = fma(wv, wv, d);
            }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            sq += __shfl_xor_sync(0xffffffffu, sq, o);
            d += __shfl_xor_sync(0xffffffffu, d, o);
        }
        if (lane == 0) {
            S.c_norm[k] = sqrt(sq);
            S.c_dev2[k] = d;
        }
    }
}

template <int EF, int R>
__global__ void __launch_bounds__(256) k_smm_f64_ks(int64_t nlist, const int64_t* __restrict__ list, SmmArgs S) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t w = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); w < nlist; w += warps)
        smm_block_ks<EF, R>(list[w], S, lane);
}

// The five-slot class (23 x 7 and 7 x 23: m n = 32 x 5 + 1) with registers capped for three
// CTAs of 256 threads per SM (80 registers, no spills): at the uncapped 98 registers only two
// fit, and the operand loads' latency showed (FP64 pipe 72% busy).
__global__ void __launch_bounds__(256, 3) k_smm_f64_ks5(int64_t nlist, const int64_t* __restrict__ list, SmmArgs S) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t w = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); w < nlist; w += warps)
        smm_block_ks<5, 1>(list[w], S, lane);
}

// One launch for every block shape of a product: the warps take C blocks from one work queue
// (the shape lists one after another) in chunks of kQueueChunk with an atomic counter, and
// each runs the single-warp body of its block's class (the K-split one where m n = 32 EF + 1).
// Blocks of up to kQueueMaxE element slots per lane (13 x 13, 23 x 7 and smaller: two CTAs of
// 256 threads fit an SM without spills); larger shapes keep their own launches.  Every C
// element and norm is summed as by the single-warp kernels.
constexpr int kQueueChunk = 4;
constexpr int kQueueMaxE = 9;

template <int E>
__device__ __forceinline__ void queue_dispatch(int e, int ks, int64_t k, const SmmArgs& S, int lane) {
    if constexpr (E <= kQueueMaxE) {
        if (e == E) {
            if constexpr (E >= 2) {
                if (ks) {
                    smm_block_ks<E - 1, 1>(k, S, lane);
                    return;
                }
            }
            smm_block<E, false>(k, S, lane, 0, 0, 0, nullptr);
            return;
        }
        queue_dispatch<E + 1>(e, ks, k, S, lane);
    }
}

__global__ void __launch_bounds__(256, 2) k_smm_f64_queue(int64_t nlist, const int64_t* __restrict__ list, SmmArgs S,
                                                      unsigned long long* __restrict__ counter) {
    const int lane = threadIdx.x & 31;
    while (true) {
        unsigned long long base = 0;
        if (lane == 0) base = atomicAdd(counter, (unsigned long long)kQueueChunk);
        base = __shfl_sync(0xffffffffu, base, 0);
        if (base >= (unsigned long long)nlist) break;
        for (int c = 0; c < kQueueChunk && base + c < (unsigned long long)nlist; ++c) {
            const int64_t k = list[base + c];
            const int mn = S.bs[S.f_row[k]] * S.bs[S.f_col[k]];
            const int ks = (mn > 32 && (mn & 31) == 1) ? 1 : 0;
            queue_dispatch<1>((mn + 31) >> 5, ks, k, S, lane);
        }
    }
}


// Stable partition of the formed blocks by shape: flag[k] = (block k is m x n).
__global__ void k_shape_flags(int64_t nform, const int32_t* __restrict__ f_row, const int32_t* __restrict__ f_col,
                              const int32_t* __restrict__ bs, const int64_t* __restrict__ mirror, int sym, int m, int n,
                              int32_t* __restrict__ flag) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nform; k += (int64_t)gridDim.x * blockDim.x) {
        const int32_t I = f_row[k], J = f_col[k];
        flag[k] = (bs[I] == m && bs[J] == n && block_role(sym, I, J, mirror[k], nullptr) == 0) ? 1 : 0;
    }
}

__global__ void k_class_scatter(int64_t nform, const int32_t* __restrict__ flag, const int64_t* __restrict__ pos,
                                int64_t* __restrict__ list) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nform; k += (int64_t)gridDim.x * blockDim.x)
        if (flag[k]) list[pos[k]] = k;
}

using SmmKernel = void (*)(int64_t, const int64_t*, SmmArgs);

// Classes with at least kPairMinE element slots per lane run as warp pairs (PAIR) when
// the CTA holds whole pairs: 23x23 blocks (E = 17) need 164 registers per thread on one
// warp and left 5.5 warps per SM with the FP64 pipe 62% busy.
constexpr int kPairMinE = 6;
template <int... Es>
struct SmmTable {
    static SmmKernel get(int e, bool pair) {
        SmmKernel t[] = {nullptr, &k_smm_f64<Es, false>...};
        SmmKernel tp[] = {nullptr, &k_smm_f64<Es, (Es >= 2)>...};
        if (e < 1 || e > (int)sizeof...(Es)) return nullptr;
        return pair ? tp[e] : t[e];
    }
};
using SmmF64 = SmmTable<1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 11, 12, 13, 14, 15, 16, 17, 18, 19, 20, 21, 22, 23, 24, 25,
                        26, 27, 28, 29, 30, 31, 32>;

template <int... Es>
struct SmmKsTable {
    static SmmKernel get(int ef) {
        SmmKernel t[] = {nullptr, &k_smm_f64_ks<Es, 1>...};
        if (ef == 5) return &k_smm_f64_ks5;
        return (ef >= 1 && ef <= (int)sizeof...(Es)) ? t[ef] : nullptr;
    }
};
using SmmF64Ks1 = SmmKsTable<1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 11, 12, 13, 14, 15, 16, 17, 18, 19, 20, 21, 22, 23, 24, 25,
                             26, 27, 28, 29, 30, 31>;

// pair: the launch's CTAs hold whole warp pairs (threads per CTA a multiple of 64)
SmmKernel f64_kernel(int cls, bool pair) {
    if (cls > kF64ClassKs1 && cls < kF64Classes) return SmmF64Ks1::get(cls - kF64ClassKs1);
    return SmmF64::get(cls, pair);
}


// Planned products keep their pattern: a block (not diagonal) whose norm is below eps
// is set to zero instead of being removed.
__global__ void k_zero_small(int64_t nb, const int32_t* __restrict__ row, const int32_t* __restrict__ col,
                             const int32_t* __restrict__ bs, const int64_t* __restrict__ off,
                             double* __restrict__ data, double* __restrict__ norms, double eps) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t b = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); b < nb; b += warps) {
        if (row[b] == col[b] || !(norms[b] < eps)) continue;
        const int area = bs[row[b]] * bs[col[b]];
        double* x = data + off[b];
        for (int e = lane; e < area; e += 32) x[e] = 0.0;
        if (lane == 0) norms[b] = 0.0;
    }
}

__global__ void k_keep_filter(int64_t nb, const int32_t* __restrict__ row, const int32_t* __restrict__ col,
                              const double* __restrict__ norms, const double* __restrict__ dev2, double eps,
                              int32_t* __restrict__ keep, double* __restrict__ dev2_kept) {
    for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < nb; b += (int64_t)gridDim.x * blockDim.x) {
        const int32_t k = (row[b] == col[b] || norms[b] >= eps) ? 1 : 0;
        keep[b] = k;
        dev2_kept[b] = k ? dev2[b] : 0.0;
    }
}

struct EventSet {
    cudaEvent_t e[4];
    EventSet() {
        for (auto& x : e) DBG_CK(cudaEventCreate(&x));
    }
    ~EventSet() {
        for (auto& x : e) cudaEventDestroy(x);
    }
    float ms(int a, int b) {
        float t = 0.f;
        cudaEventElapsedTime(&t, e[a], e[b]);
        return t;
    }
};

int sym_grid(int32_t nblk) { return std::min<int32_t>(nblk, num_sms() * 8); }

__global__ void k_keep_twinned(int64_t nb, const int64_t* __restrict__ mirror, int32_t* __restrict__ keep) {
    for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < nb; b += (int64_t)gridDim.x * blockDim.x)
        keep[b] = mirror[b] >= 0 ? 1 : 0;
}

}  // namespace

TuneCfg default_cfg(int prec) {
    (void)prec;
    return TuneCfg{};
}

std::atomic<int> g_fp64_schedule{0};

// The whole formed-block list of a product (every shape) in one work-queue launch.
void launch_smm_queue(int64_t cnt, const int64_t* list, const SmmArgs& sa, unsigned long long* counter,
                      cudaStream_t s) {
    if (cnt <= 0) return;
    static int per_sm[64] = {};
    int dev = 0;
    DBG_CK(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) fail(DBCSR_ECAPACITY, "multiply: device ordinal out of range");
    if (!per_sm[dev]) {
        int b = 0;
        DBG_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_smm_f64_queue, 256, 0));
        per_sm[dev] = std::max(b, 1);
    }
    DBG_CK(cudaMemsetAsync(counter, 0, sizeof(unsigned long long), s));
    const int64_t g = std::min<int64_t>(ceil_div(cnt, 8), (int64_t)num_sms() * per_sm[dev]);
    k_smm_f64_queue<<<(unsigned)g, 256, 0, s>>>(cnt, list, sa, counter);
    DBG_LAUNCH_CK();
}

bool cfg_valid(int m, int n, const TuneCfg& c) {
    const int mn = m * n;
    if (c.tpb < 32 || c.tpb > 256 || c.tpb % 32 || c.ctas_per_sm < 1) return false;
    if (c.split == kSplitPair) return mn > 32 && c.tpb % 64 == 0;
    if (c.split == kSplitK) return mn > 32 && (mn & 31) == 1;
    return c.split == kSplitDefault || c.split == kSplitWarp;
}

int resolve_split(int m, int n, const TuneCfg& c) {
    const int mn = m * n;
    if (c.split != kSplitDefault) return c.split;
    if (mn > 32 && (mn & 31) == 1) return kSplitK;
    return ((mn + 31) >> 5) >= kPairMinE && c.tpb % 64 == 0 ? kSplitPair : kSplitWarp;
}

void launch_smm_shape(int m, int n, int64_t cnt, const int64_t* list, const SmmArgs& sa, const TuneCfg& cfg,
                      cudaStream_t s) {
    if (cnt <= 0) return;
    if (!cfg_valid(m, n, cfg)) fail(DBCSR_EINVAL, "launch configuration out of range for this block shape");
    const int wpc = cfg.tpb / 32;
    const int mn = m * n;
    const int split = resolve_split(m, n, cfg);
    const int cls = split == kSplitK ? kF64ClassKs1 + (mn >> 5) : (mn + 31) >> 5;
    const bool pair = split == kSplitPair;
    SmmKernel kern = f64_kernel(cls, pair);
    if (!kern) fail(DBCSR_ECAPACITY, "multiply: block shape beyond the kernel table");
    SmmArgs a = sa;
    a.colmajor = cfg.colmajor;
    a.prefetch2 = cfg.prefetch2;
    const int64_t g = std::min<int64_t>(ceil_div(cnt, pair ? wpc / 2 : wpc), (int64_t)num_sms() * cfg.ctas_per_sm);
    kern<<<(unsigned)g, cfg.tpb, 0, s>>>(cnt, list, a);
    DBG_LAUNCH_CK();
}

void symmetrize(dbcsr_matrix_* m) {
    check_finalized(m);
    check_unplanned(m, "symmetrize");
    cudaStream_t s = m->stream;
    const int64_t nb = m->nnzb;
    if (nb == 0) return;
    DBuf<int64_t> mirror;
    DBuf<double> norm, dev2;
    DBuf<int32_t> keep;
    mirror.alloc(nb, s);
    norm.alloc(nb, s);
    dev2.alloc(nb, s);
    keep.alloc(nb, s);
    k_find_mirror<<<grid_for(nb, 256), 256, 0, s>>>(nb, m->row.p, m->col.p, m->rp.p, mirror.p);
    DBG_LAUNCH_CK();
    k_sym_average<<<grid_for(nb, 8), 256, 0, s>>>(nb, mirror.p, m->row.p, m->col.p, m->off.p, m->bs.p, m->data.p,
                                                 norm.p, dev2.p);
    DBG_LAUNCH_CK();
    k_keep_twinned<<<grid_for(nb, 256), 256, 0, s>>>(nb, mirror.p, keep.p);
    DBG_LAUNCH_CK();
    compact(m, keep.p, nullptr);
}

void multiply(double alpha, dbcsr_matrix_* A, dbcsr_matrix_* B, double beta, dbcsr_matrix_* C, double eps, int prec,
              dbcsr_mult_stats* stats, bool want_dev2, int sym_result, MultPlan* plan) {
    check_finalized(A);
    check_finalized(B);
    if (!C) fail(DBCSR_EINVAL, "multiply: null C");
    check_unplanned(C, "multiply");
    if (plan) {
        if (beta != 0.0 || sym_result) fail(DBCSR_EINVAL, "multiply_plan: only C = alpha A B (beta = 0)");
        if (C == A || C == B) fail(DBCSR_EINVAL, "multiply_plan: C must differ from A and B");
    }
    if (A->h_bs != B->h_bs || A->h_bs != C->h_bs) fail(DBCSR_EINVAL, "multiply: block sizes of A, B and C differ");
    if (prec != DBCSR_FP64 && !is_bf16(prec))
        fail(DBCSR_EINVAL, "multiply: prec must be DBCSR_FP64, DBCSR_BF16 or DBCSR_BF16X3");
    if (!(eps >= 0.0)) fail(DBCSR_EINVAL, "multiply: eps_filter must be >= 0");
    const bool use_c = (beta != 0.0);
    if (use_c) check_finalized(C);
    // compulsory operand traffic of the block-product launches: A and B read once, the computed
    // C blocks written once, a C input that is neither A nor B read once
    double bytes_min = 8.0 * ((double)A->nel + (B != A ? (double)B->nel : 0.0) +
                              (use_c && C != A && C != B ? (double)C->nel : 0.0));
    int32_t n_smm_launches = 0;
    const int32_t nblk = A->nblk;
    if (nblk > kMaxBlockRows) fail(DBCSR_ECAPACITY, "multiply: more than 262144 block rows");
    cudaStream_t s = C->stream;
    if (A->stream != s) DBG_CK(cudaStreamSynchronize(A->stream));
    if (B->stream != s) DBG_CK(cudaStreamSynchronize(B->stream));

    // BF16 products run on the tensor-core tier, on groups of blocks (kept with the matrices)
    const bool bf16 = is_bf16(prec);
    std::shared_ptr<Groups> groups = A->groups ? A->groups : B->groups;
    if (bf16 && (!groups || groups->nblk != nblk)) {
        groups = build_groups(A);
        A->groups = groups;
    }
    if (groups && groups->nblk != nblk) groups.reset();
    const int32_t* grp = bf16 ? groups->g_of.p : nullptr;

    EventSet ev;
    DBG_CK(cudaEventRecord(ev.e[0], s));
    ensure_norms(A);
    ensure_norms(B);
    if (use_c) ensure_norms(C);

    const int nwords = (nblk + 31) / 32;
    const size_t sm_rank = (size_t)2 * ((nwords + 1) & ~1) * sizeof(uint32_t);
    RowPattern P{A->rp.p, A->col.p, B->rp.p, B->col.p, use_c ? C->rp.p : nullptr, use_c ? C->col.p : nullptr};

    // 1. candidate counts
    DBuf<int64_t> ccnt, coff, maxrow;
    ccnt.alloc(nblk, s);
    coff.alloc(nblk + 1, s);
    maxrow.alloc(2, s);                   // largest candidate count and largest A row of a block row
    maxrow.zero();
    {
        const size_t sm = sm_rank;
        allow_dyn_smem(k_cand_count, sm);
        k_cand_count<<<sym_grid(nblk), kSymThreads, sm, s>>>(nblk, P, nwords, ccnt.p, (unsigned long long*)maxrow.p);
        DBG_LAUNCH_CK();
    }
    scan_exclusive(ccnt.p, coff.p, nblk, s);
    int64_t h2[3];
    {
        const int64_t* src[3] = {coff.p + nblk, maxrow.p, maxrow.p + 1};
        read_i64s(src, 3, h2, s);
    }
    const int64_t ncand = h2[0], max_row = h2[1], max_arow = h2[2];

    // 2. candidates, bounds and the prescreen decision
    DBuf<int32_t> cand_row, cand_col, pcnt, ksum, keep;
    DBuf<double> bound;
    DBuf<int64_t> cin, kidx;
    const int64_t nc1 = std::max<int64_t>(ncand, 1);
    cand_row.alloc(nc1, s);
    cand_col.alloc(nc1, s);
    pcnt.alloc(nc1, s);
    ksum.alloc(nc1, s);
    keep.alloc(nc1, s);
    kidx.alloc(ncand + 1, s);
    if (use_c) cin.alloc(nc1, s);
    const size_t sm_acc = sm_rank + (size_t)max_row * (sizeof(double) + 2 * sizeof(int32_t) + sizeof(float));
    const bool acc_smem = sm_acc <= (size_t)kSymSmemBudget;
    // a candidate's bound has at most (largest A row) terms: the FP32 margin covers 4095
    const bool fast_bound = acc_smem && max_arow < 4096;
    if (!acc_smem) bound.alloc(nc1, s);
    if (ncand) {
        DBuf<float> b_norm_ru;
        if (fast_bound && B->nnzb) {
            b_norm_ru.alloc(B->nnzb, s);
            k_norms_f32_ru<<<grid_for(B->nnzb, 256), 256, 0, s>>>(B->nnzb, B->norms.p, b_norm_ru.p);
            DBG_LAUNCH_CK();
        }
        BoundArgs ba{std::fabs(alpha), std::fabs(beta), eps * (1.0 - 1e-12), A->norms.p, B->norms.p,
                     use_c ? C->norms.p : nullptr, A->bs.p, coff.p, cand_row.p, cand_col.p,
                     bound.p, pcnt.p, ksum.p, use_c ? cin.p : nullptr, keep.p, acc_smem ? 1 : 0,
                     fast_bound ? 1 : 0, b_norm_ru.p};
        const size_t sm = acc_smem ? sm_acc : sm_rank;
        allow_dyn_smem(k_cand_bound, sm);
        k_cand_bound<<<sym_grid(nblk), kSymThreads, sm, s>>>(nblk, P, nwords, ba);
        DBG_LAUNCH_CK();
    }
    scan_exclusive(keep.p, kidx.p, ncand, s);
    const int64_t nform = read_i64(kidx.p + ncand, s);

    // 3. formed-block metadata
    const int64_t nf1 = std::max<int64_t>(nform, 1);
    DBuf<int32_t> f_row, f_col, f_ksum;
    DBuf<uint8_t> f_comp;                 // 1: the block is computed (0: copied from its twin or dropped)
    DBuf<int64_t> f_area, f_np, f_cin, f_off, f_pbeg, f_rp, flops, nprod_exec, shape_cnt, mirror;
    f_ksum.alloc(nf1, s);
    f_comp.alloc(nf1, s);
    mirror.alloc(nf1, s);
    nprod_exec.alloc(1, s);
    nprod_exec.zero();
    f_row.alloc(nf1, s);
    f_col.alloc(nf1, s);
    f_area.alloc(nf1, s);
    f_np.alloc(nf1, s);
    f_cin.alloc(nf1, s);
    f_off.alloc(nform + 1, s);
    f_pbeg.alloc(nform + 1, s);
    f_rp.alloc(nblk + 1, s);
    flops.alloc(1, s);
    flops.zero();
    constexpr int kShapes = (kMaxBlock + 1) * (kMaxBlock + 1);     // histogram of formed blocks by (m, n)
    shape_cnt.alloc(kShapes, s);
    shape_cnt.zero();
    if (ncand) {
        k_form_meta<<<grid_for(ncand, 256), 256, 0, s>>>(ncand, keep.p, kidx.p, cand_row.p, cand_col.p, pcnt.p, ksum.p,
                                                         use_c ? cin.p : nullptr, A->bs.p, f_row.p, f_col.p, f_area.p,
                                                         f_np.p, f_cin.p, f_ksum.p);
        DBG_LAUNCH_CK();
    }
    k_form_rp<<<grid_for(nblk + 1, 256), 256, 0, s>>>(nblk, coff.p, kidx.p, f_rp.p);
    DBG_LAUNCH_CK();
    if (nform) {
        if (sym_result) {
            k_find_mirror<<<grid_for(nform, 256), 256, 0, s>>>(nform, f_row.p, f_col.p, f_rp.p, mirror.p);
            DBG_LAUNCH_CK();
        } else {
            DBG_CK(cudaMemsetAsync(mirror.p, 0xff, sizeof(int64_t) * nform, s));   // -1 (unused without sym)
        }
        k_form_stats<<<grid_for(nform, 256, (int64_t)num_sms() * 8), 256, 0, s>>>(nform, f_row.p, f_col.p, f_np.p, f_ksum.p, mirror.p,
                                                          sym_result, A->bs.p,
                                                          (unsigned long long*)flops.p,
                                                          (unsigned long long*)nprod_exec.p,
                                                          (unsigned long long*)shape_cnt.p, f_comp.p, grp);
        DBG_LAUNCH_CK();
    }
    scan_exclusive(f_area.p, f_off.p, nform, s);
    scan_exclusive(f_np.p, f_pbeg.p, nform, s);
    int64_t h3[4];
    std::vector<int64_t> shapes(kShapes);
    {
        const int64_t* src[4] = {f_off.p + nform, f_pbeg.p + nform, flops.p, nprod_exec.p};
        DBG_CK(cudaMemcpyAsync(shapes.data(), shape_cnt.p, sizeof(int64_t) * kShapes, cudaMemcpyDeviceToHost, s));
        read_i64s(src, 4, h3, s);
    }
    const int64_t nel = h3[0], nprod = h3[1];
    const double nflop = (double)(unsigned long long)h3[2];
    const int64_t nprod_done = h3[3];

    // 4. product stacks
    DBuf<int32_t> prod_a, prod_b, cursor;
    prod_a.alloc(std::max<int64_t>(bf16 ? 1 : nprod, 1), s);
    prod_b.alloc(std::max<int64_t>(bf16 ? 1 : nprod, 1), s);
    const size_t sm_fill = sm_rank + (size_t)max_row * (sizeof(int64_t) + sizeof(int32_t));
    const bool fill_smem = sm_fill <= (size_t)kSymSmemBudget;
    if (!fill_smem && !bf16) cursor.alloc(nf1, s);
    if (nprod && !bf16) {
        FillArgs fa{coff.p, keep.p, f_comp.p, kidx.p, f_pbeg.p, cursor.p, prod_a.p, prod_b.p, fill_smem ? 1 : 0};
        const size_t sm = fill_smem ? sm_fill : sm_rank;
        allow_dyn_smem(k_fill_stack, sm);
        k_fill_stack<<<sym_grid(nblk), kSymThreads, sm, s>>>(nblk, P, nwords, fa);
        DBG_LAUNCH_CK();
    }
    // the candidate arrays are no longer needed
    cand_row.release(); cand_col.release(); pcnt.release(); ksum.release(); bound.release(); cursor.release();
    if (!nform) DBG_CK(cudaEventRecord(ev.e[1], s));

    // 5. numeric
    DBuf<double> c_data, c_norm, c_dev2;
    c_data.alloc(std::max<int64_t>(nel, 1), s);
    c_norm.alloc(nf1, s);
    c_dev2.alloc(nf1, s);
    // kept by a plan: the shape lists, the tensor-core tier's patterns and the launch sequence
    DBuf<int64_t> list;
    SmmArgs sa{};
    struct ShapeLaunch { int m, n; int64_t cnt; };
    std::vector<ShapeLaunch> launches;
    std::unique_ptr<LowTierPlan, void (*)(LowTierPlan*)> lt(nullptr, lowtier_plan_delete);
    LowTierOut lto{};
    DBuf<int64_t> qcounter;                 // the work queue's counter (one-launch schedule)
    const int kmax = *std::max_element(A->h_bs.begin(), A->h_bs.end());
    if (nform) {
        sa = SmmArgs{f_row.p, f_col.p, f_off.p, f_pbeg.p, f_cin.p, prod_a.p, prod_b.p, A->col.p, A->off.p, A->data.p,
                     B->off.p, B->data.p, use_c ? C->off.p : nullptr, use_c ? C->data.p : nullptr, A->bs.p,
                     alpha, beta, c_data.p, c_norm.p, c_dev2.p};
        // FP64: one launch per (m, n) block shape over that shape's blocks (kept in CSR order)
        DBuf<int32_t> flag;
        DBuf<int64_t> pos;
        if (!bf16) {
            flag.alloc(nform, s);
            pos.alloc(nform + 1, s);
            list.alloc(nform, s);
        }
        // with the one-launch schedule, the shapes the work queue takes come first in the list
        const bool queue = !bf16 && g_fp64_schedule.load() == 1;
        int64_t at = 0, at_q = 0;
        for (int pass = 0; pass < 2; ++pass)
        for (int m = 1; m <= kMaxBlock; ++m)
            for (int n = 1; n <= kMaxBlock; ++n) {
                const int64_t cnt = shapes[m * (kMaxBlock + 1) + n];
                if (!cnt) continue;
                if ((queue && ((m * n + 31) >> 5) <= kQueueMaxE) != (pass == 0)) continue;
                bytes_min += 8.0 * (double)cnt * m * n;
                if (bf16) continue;
                k_shape_flags<<<grid_for(nform, 256), 256, 0, s>>>(nform, f_row.p, f_col.p, A->bs.p, mirror.p,
                                                                   sym_result, m, n, flag.p);
                DBG_LAUNCH_CK();
                scan_exclusive(flag.p, pos.p, nform, s);
                k_class_scatter<<<grid_for(nform, 256), 256, 0, s>>>(nform, flag.p, pos.p, list.p + at);
                DBG_LAUNCH_CK();
                if (pass == 0) at_q += cnt;
                launches.push_back({m, n, cnt});
                at += cnt;
            }
        if (bf16) {
            // the tensor-core tier on groups of blocks: group tile patterns and stacks, then the
            // operands packed (split) into tiles -- all counted with the symbolic phase
            lt = lowtier_prepare(prec, A, B, groups, sym_result == kSymMirror, nform, f_rp.p, f_row.p, f_col.p,
                                 f_comp.p, s);
            lowtier_pack(*lt, A, B, s);
            lto = LowTierOut{f_rp.p, f_col.p, f_comp.p, f_off.p, use_c ? f_cin.p : nullptr,
                             use_c ? C->off.p : nullptr, use_c ? C->data.p : nullptr, alpha, beta,
                             c_data.p, c_norm.p, c_dev2.p};
        }
        // the tuned configurations are looked up with the largest block edge as the inner size
        DBG_CK(cudaEventRecord(ev.e[1], s));
        if (bf16) {
            lowtier_run(*lt, A, lto, s);
            n_smm_launches = 1;
        }
        if (at_q > 0) {
            // the queue's shapes in one launch, replacing their per-shape entries
            std::vector<ShapeLaunch> rest{{0, 0, at_q}};
            int64_t q = 0;
            for (const ShapeLaunch& L : launches) {
                if (q < at_q) q += L.cnt;
                else rest.push_back(L);
            }
            launches = std::move(rest);
            qcounter.alloc(1, s);
        }
        at = 0;
        for (const ShapeLaunch& L : launches) {
            if (L.m == 0) launch_smm_queue(L.cnt, list.p, sa, (unsigned long long*)qcounter.p, s);
            else launch_smm_shape(L.m, L.n, L.cnt, list.p + at, sa, tune_lookup(prec, L.m, L.n, kmax), s);
            at += L.cnt;
        }
        if (!bf16)         n_smm_launches = (int32_t)launches.size();
        if (sym_result) {
            DBG_CK(cudaEventRecord(ev.e[2], s));     // the copy / averaging is timed with the filter
            k_mirror_copy<<<grid_for(nform, 8), 256, 0, s>>>(nform, sym_result, mirror.p, f_row.p, f_col.p, f_off.p,
                                                            A->bs.p, c_data.p, c_norm.p, c_dev2.p, grp);
            DBG_LAUNCH_CK();
            if (sym_result == 2) {
                k_sym_average<<<grid_for(nform, 8), 256, 0, s>>>(nform, mirror.p, f_row.p, f_col.p, f_off.p, A->bs.p,
                                                                c_data.p, c_norm.p, c_dev2.p);
                DBG_LAUNCH_CK();
            } else {
                k_sym_diag<<<grid_for(nblk, 8), 256, 0, s>>>(nblk, f_rp.p, f_col.p, f_off.p, A->bs.p, c_data.p,
                                                            c_norm.p, c_dev2.p);
                DBG_LAUNCH_CK();
            }
        }
    }
    if (!sym_result || !nform) DBG_CK(cudaEventRecord(ev.e[2], s));
    if (!plan) {
        prod_a.release();
        prod_b.release();
    }

    // install the formed blocks as C (A or B may alias C: every read above is queued before)
    C->rp = std::move(f_rp);
    C->row = std::move(f_row);
    C->col = std::move(f_col);
    C->off = std::move(f_off);
    C->data = std::move(c_data);
    C->nnzb = nform;
    C->nel = nel;
    C->norms = std::move(c_norm);
    C->norms_valid = true;
    C->finalized = true;
    if (groups) C->groups = groups;

    if (plan) {
        // 6'. a plan keeps the formed pattern: blocks under eps are zeroed, not removed, so
        // that every execution writes the same arrays; then the whole numeric phase
        // (packing, block products, zeroing) is captured into one graph
        auto zero_small = [&](cudaStream_t zs) {
            if (!nform) return;
            k_zero_small<<<grid_for(nform, 8), 256, 0, zs>>>(nform, C->row.p, C->col.p, C->bs.p, C->off.p, C->data.p,
                                                            C->norms.p, eps);
            DBG_LAUNCH_CK();
        };
        zero_small(s);
        // captured on a private stream (the legacy default stream cannot be captured); the
        // graph is launched on C's stream
        cudaStream_t cs = nullptr;
        DBG_CK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        cudaGraph_t graph = nullptr;
        const int64_t l0 = g_launches.load();
        try {
            DBG_CK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
            if (lt) {
                lowtier_pack(*lt, A, B, cs);
                lowtier_run(*lt, A, lto, cs);
            }
            int64_t at = 0;
            for (const ShapeLaunch& L : launches) {
                if (L.m == 0) launch_smm_queue(L.cnt, list.p, sa, (unsigned long long*)qcounter.p, cs);
                else launch_smm_shape(L.m, L.n, L.cnt, list.p + at, sa, tune_lookup(prec, L.m, L.n, kmax), cs);
                at += L.cnt;
            }
            zero_small(cs);
            DBG_CK(cudaStreamEndCapture(cs, &graph));
        } catch (...) {
            cudaStreamCaptureStatus cst = cudaStreamCaptureStatusNone;
            if (cudaStreamIsCapturing(cs, &cst) == cudaSuccess && cst != cudaStreamCaptureStatusNone) {
                cudaGraph_t g = nullptr;
                (void)cudaStreamEndCapture(cs, &g);
                if (g) cudaGraphDestroy(g);
            }
            cudaStreamDestroy(cs);
            (void)cudaGetLastError();
            throw;
        }
        cudaStreamDestroy(cs);
        cudaGraphExec_t exec = nullptr;
        const cudaError_t ie = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        DBG_CK(ie);
        plan->exec = exec;
        plan->kernels = g_launches.load() - l0;
        plan->stream = s;
        plan->A = A;
        plan->B = B;
        plan->C = C;
        plan->bufs_i32.push_back(std::move(prod_a));
        plan->bufs_i32.push_back(std::move(prod_b));
        plan->bufs_i64.push_back(std::move(list));
        plan->bufs_i64.push_back(std::move(f_pbeg));
        plan->bufs_i64.push_back(std::move(f_cin));
        plan->bufs_f64.push_back(std::move(c_dev2));
        plan->bufs_i64.push_back(std::move(qcounter));
        plan->bufs_u8.push_back(std::move(f_comp));
        plan->lt = lt.release();
        A->plans++;
        B->plans++;
        C->plans++;
        DBG_CK(cudaEventRecord(ev.e[3], s));
        if (stats) {
            DBG_CK(cudaStreamSynchronize(s));
            stats->n_candidates = ncand;
            stats->n_formed = nform;
            stats->n_kept = C->nnzb;
            stats->n_products = nprod_done;
            stats->flops = nflop;
            stats->ms_symbolic = ev.ms(0, 1);
            stats->ms_numeric = ev.ms(1, 2);
            stats->ms_filter = ev.ms(2, 3);
            stats->bytes_min = bytes_min;
            stats->n_launches = n_smm_launches;
            stats->flops_tensor = plan->lt ? lowtier_tensor_flops(*plan->lt) : 0.0;
            stats->bytes_tensor = plan->lt ? lowtier_copy_bytes(*plan->lt) : 0.0;
            stats->n_tiles = plan->lt ? lowtier_tiles(*plan->lt) : 0;
        }
        return;
    }

    // 6. filter
    DBuf<int32_t> keep2;
    DBuf<double> dev2k, dsum;
    keep2.alloc(nf1, s);
    dev2k.alloc(nf1, s);
    dsum.alloc(1, s);
    if (nform) {
        k_keep_filter<<<grid_for(nform, 256), 256, 0, s>>>(nform, C->row.p, C->col.p, C->norms.p, c_dev2.p, eps,
                                                           keep2.p, dev2k.p);
        DBG_LAUNCH_CK();
    }
    if (want_dev2) det_sum(dev2k.p, nform, dsum.p, s);
    compact(C, keep2.p, C->norms.p);
    DBG_CK(cudaEventRecord(ev.e[3], s));
    if (lt) lowtier_check(*lt, s);

    if (stats) {
        DBG_CK(cudaStreamSynchronize(s));
        stats->n_candidates = ncand;
        stats->n_formed = nform;
        stats->n_kept = C->nnzb;
        stats->n_products = nprod_done;
        stats->flops = nflop;
        stats->dev2_filtered = want_dev2 ? read_f64(dsum.p, s) : 0.0;
        stats->ms_symbolic = ev.ms(0, 1);
        stats->ms_numeric = ev.ms(1, 2);
        stats->ms_filter = ev.ms(2, 3);
        stats->bytes_min = n_smm_launches ? bytes_min : 0.0;
        stats->n_launches = n_smm_launches;
        stats->flops_tensor = lt ? lowtier_tensor_flops(*lt) : 0.0;
        stats->bytes_tensor = lt ? lowtier_copy_bytes(*lt) : 0.0;
        stats->n_tiles = lt ? lowtier_tiles(*lt) : 0;
    }
}

void execute_plan(MultPlan* plan) {
    if (!plan || !plan->exec) fail(DBCSR_EINVAL, "multiply_execute: null plan");
    dbcsr_matrix_* A = plan->A;
    dbcsr_matrix_* B = plan->B;
    if (A->stream != plan->stream) DBG_CK(cudaStreamSynchronize(A->stream));
    if (B->stream != plan->stream) DBG_CK(cudaStreamSynchronize(B->stream));
    DBG_CK(cudaGraphLaunch(plan->exec, plan->stream));
    g_launches.fetch_add(plan->kernels, std::memory_order_relaxed);
    plan->C->norms_valid = true;
}

MultPlan::~MultPlan() {
    if (exec) {
        cudaStreamSynchronize(stream);      // no execution may still use the buffers
        cudaGraphExecDestroy(exec);
    }
    if (lt) lowtier_plan_delete(lt);
    if (A) A->plans--;
    if (B) B->plans--;
    if (C) C->plans--;
}

}  // namespace dbg

extern "C" {

dbcsr_status dbcsr_set_fp64_schedule(int32_t mode) {
    if (mode != DBCSR_SCHEDULE_PER_SHAPE && mode != DBCSR_SCHEDULE_QUEUE) {
        dbg::set_last_error("set_fp64_schedule: mode must be DBCSR_SCHEDULE_PER_SHAPE or DBCSR_SCHEDULE_QUEUE");
        return DBCSR_EINVAL;
    }
    dbg::g_fp64_schedule.store(mode);
    dbg::set_last_error("");
    return DBCSR_OK;
}

int32_t dbcsr_get_fp64_schedule(void) { return dbg::g_fp64_schedule.load(); }

struct dbcsr_plan_ {
    dbg::MultPlan plan;
};

dbcsr_status dbcsr_multiply_plan(double alpha, dbcsr_matrix A, dbcsr_matrix B, dbcsr_matrix C, double eps_filter,
                                 int32_t prec, dbcsr_plan* out, dbcsr_mult_stats* stats) {
    if (!out) {
        dbg::set_last_error("multiply_plan: null output handle");
        return DBCSR_EINVAL;
    }
    *out = nullptr;
    auto* p = new dbcsr_plan_();
    try {
        if (!A || !B) dbg::fail(DBCSR_EINVAL, "multiply_plan: null handle");
        dbg::multiply(alpha, A, B, 0.0, C, eps_filter, prec, stats, false, dbg::kSymNone, &p->plan);
        *out = p;
        dbg::set_last_error("");
        return DBCSR_OK;
    } catch (const dbg::Error& e) {
        delete p;
        dbg::set_last_error(e.what());
        return e.code;
    } catch (const std::exception& e) {
        delete p;
        dbg::set_last_error(e.what());
        return DBCSR_ECUDA;
    }
}

dbcsr_status dbcsr_multiply_execute(dbcsr_plan plan) {
    try {
        if (!plan) dbg::fail(DBCSR_EINVAL, "multiply_execute: null plan");
        dbg::execute_plan(&plan->plan);
        dbg::set_last_error("");
        return DBCSR_OK;
    } catch (const dbg::Error& e) {
        dbg::set_last_error(e.what());
        return e.code;
    } catch (const std::exception& e) {
        dbg::set_last_error(e.what());
        return DBCSR_ECUDA;
    }
}

dbcsr_status dbcsr_plan_destroy(dbcsr_plan plan) {
    delete plan;
    return DBCSR_OK;
}

}  // extern "C"
