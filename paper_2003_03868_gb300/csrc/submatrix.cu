// Density matrix by the submatrix method (section "Submatrix Method": principal
// submatrices of K, one per DBCSR block with the atoms overlapping it, purified densely
// by an iterative sign scheme or an eigendecomposition).
//
//   * submatrix j (one per block column): I_j = the pattern of column j of H,
//     H^(j) = H[I_j, I_j] (dense, zero where H has no block);
//   * X_0 = (H^(j) - mu 1) / alpha, alpha the Gershgorin bound of H - mu 1 (it bounds every
//     principal submatrix too), padded to n_pad with an identity block (already a sign);
//   * dense Newton-Schulz on the whole batch: X2 = X X, r_j = ||X2 - 1||_F / n_pad, stop when
//     every r_j < tol, else X <- 1.5 X - 0.5 X X2;
//   * block (i, j) of P, i in I_j: the rows of i and columns of j of (1 - X) / 2.  P has the
//     pattern of H.
//
// Every kernel is the library's: gather, residual, scatter, and the batched dense products
// (dense.cu).  The submatrices are grouped by padded size and run in chunks of at most
// kChunkBytes of device memory.  FP64 runs on the FP64 pipe; the mixed mode stores FP32 and
// multiplies on the TF32 tensor cores while the largest residual is at least switch_tol,
// then with split TF32 (three products of TF32 halves, close to FP32 arithmetic; the
// iteration corrects the earlier rounding as in the sparse ladder).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <map>
#include <type_traits>
#include <vector>

#include "common.cuh"

namespace dbg {
namespace {

constexpr int kPad = 16;                          // submatrix edges rounded up to 16
constexpr size_t kChunkBytes = size_t(8) << 30;   // X, X2 and the update buffer of one chunk

__device__ __forceinline__ int64_t find_col(const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                                            int64_t row, int32_t c) {
    int64_t lo = rp[row], hi = rp[row + 1];
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (col[mid] < c) lo = mid + 1; else hi = mid;
    }
    return (lo < rp[row + 1] && col[lo] == c) ? lo : -1;
}

// One CTA per submatrix s (block column j = sub_j[s]): the dense, scaled, padded X_0.
// doff[dstart[s] + a] = first row of block I_j[a] inside the submatrix.
template <class T>
__global__ void k_sub_gather(int32_t nsub, const int32_t* __restrict__ sub_j, const int64_t* __restrict__ dstart,
                             const int32_t* __restrict__ doff, const int32_t* __restrict__ sub_n, int n_pad,
                             const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                             const int64_t* __restrict__ off, const double* __restrict__ data,
                             const int32_t* __restrict__ bs, double mu, double inv_alpha, T* __restrict__ X) {
    for (int32_t s = blockIdx.x; s < nsub; s += gridDim.x) {
        T* x = X + (int64_t)s * n_pad * n_pad;
        for (int64_t e = threadIdx.x; e < (int64_t)n_pad * n_pad; e += blockDim.x) x[e] = T(0);
        __syncthreads();
        const int32_t j = sub_j[s];
        const int64_t q0 = rp[j];
        const int L = (int)(rp[j + 1] - q0);
        const int32_t* d = doff + dstart[s];
        for (int p = threadIdx.x; p < L * L; p += blockDim.x) {
            const int a = p / L, c = p - a * L;
            const int32_t i = col[q0 + a], k = col[q0 + c];
            const int64_t q = find_col(rp, col, i, k);
            if (q < 0) continue;
            const int mi = bs[i], mk = bs[k];
            const double* v = data + off[q];
            for (int r = 0; r < mi; ++r)
                for (int t = 0; t < mk; ++t) {
                    double y = v[r * mk + t];
                    if (i == k && r == t) y -= mu;
                    x[(int64_t)(d[a] + r) * n_pad + d[c] + t] = T(y * inv_alpha);
                }
        }
        for (int k = sub_n[s] + threadIdx.x; k < n_pad; k += blockDim.x) x[(int64_t)k * n_pad + k] = T(1);
        __syncthreads();
    }
}

// One CTA per submatrix: ||X2 - 1||_F^2 (fixed thread order, fixed tree).
template <class T>
__global__ void k_sub_residual(int32_t nsub, int n_pad, const T* __restrict__ X2, double* __restrict__ r2) {
    __shared__ double part[256];
    for (int32_t s = blockIdx.x; s < nsub; s += gridDim.x) {
        const T* x = X2 + (int64_t)s * n_pad * n_pad;
        double acc = 0.0;
        for (int64_t e = threadIdx.x; e < (int64_t)n_pad * n_pad; e += blockDim.x) {
            const double v = (double)x[e] - ((e / n_pad) == (e % n_pad) ? 1.0 : 0.0);
            acc = fma(v, v, acc);
        }
        part[threadIdx.x] = acc;
        __syncthreads();
        for (int o = blockDim.x / 2; o > 0; o >>= 1) {
            if ((int)threadIdx.x < o) part[threadIdx.x] += part[threadIdx.x + o];
            __syncthreads();
        }
        if (threadIdx.x == 0) r2[s] = part[0];
        __syncthreads();
    }
}

// One CTA per submatrix: blocks (i, j), i in I_j, of P = (1 - X) / 2 into P's data.
template <class T>
__global__ void k_sub_scatter(int32_t nsub, const int32_t* __restrict__ sub_j, const int64_t* __restrict__ dstart,
                              const int32_t* __restrict__ doff, int n_pad, const int64_t* __restrict__ rp,
                              const int32_t* __restrict__ col, const int64_t* __restrict__ off,
                              const int32_t* __restrict__ bs, const T* __restrict__ X, double* __restrict__ P) {
    for (int32_t s = blockIdx.x; s < nsub; s += gridDim.x) {
        const T* x = X + (int64_t)s * n_pad * n_pad;
        const int32_t j = sub_j[s];
        const int64_t q0 = rp[j];
        const int L = (int)(rp[j + 1] - q0);
        const int32_t* d = doff + dstart[s];
        const int64_t qj = find_col(rp, col, j, j) - q0;      // position of j in I_j
        const int mj = bs[j];
        for (int a = threadIdx.x; a < L; a += blockDim.x) {
            const int32_t i = col[q0 + a];
            const int64_t q = find_col(rp, col, i, j);
            if (q < 0) continue;
            const int mi = bs[i];
            double* p = P + off[q];
            for (int r = 0; r < mi; ++r)
                for (int t = 0; t < mj; ++t) {
                    const double v = (double)x[(int64_t)(d[a] + r) * n_pad + d[qj] + t];
                    p[r * mj + t] = 0.5 * (((i == j && r == t) ? 1.0 : 0.0) - v);
                }
        }
    }
}

struct Chunk {
    int n_pad;
    std::vector<int32_t> sub_j, sub_n, doff;
    std::vector<int64_t> dstart;
};

// C = alpha A B + beta C for every matrix of the chunk: FP64, or FP32 storage in TF32
// (split: three products of TF32 halves).
void batched_gemm(int32_t b, int n, double alpha, const double* A, const double* B, double beta, double* C, bool,
                  cudaStream_t s) {
    dense_gemm_f64(b, n, alpha, A, B, beta, C, s);
}
void batched_gemm(int32_t b, int n, double alpha, const float* A, const float* B, double beta, float* C, bool split,
                  cudaStream_t s) {
    dense_gemm_tf32(b, n, (float)alpha, A, B, (float)beta, C, split, s);
}

struct ChunkResult {
    int iterations = 0, tf32_iterations = 0;
    double r_max = 0.0, flops = 0.0;
};

template <class T>
ChunkResult run_chunk(const Chunk& ck, dbcsr_matrix_* H, dbcsr_matrix_* P, double mu, double inv_alpha,
                      const dbcsr_sign_opts& o, bool mixed, cudaStream_t s) {
    const int32_t b = (int32_t)ck.sub_j.size();
    const int n = ck.n_pad;
    const int64_t elems = (int64_t)b * n * n;
    DBuf<int32_t> d_j, d_n, d_doff;
    DBuf<int64_t> d_start;
    d_j.alloc(b, s);
    d_n.alloc(b, s);
    d_doff.alloc((int64_t)ck.doff.size(), s);
    d_start.alloc(b, s);
    DBG_CK(cudaMemcpyAsync(d_j.p, ck.sub_j.data(), sizeof(int32_t) * b, cudaMemcpyHostToDevice, s));
    DBG_CK(cudaMemcpyAsync(d_n.p, ck.sub_n.data(), sizeof(int32_t) * b, cudaMemcpyHostToDevice, s));
    DBG_CK(cudaMemcpyAsync(d_doff.p, ck.doff.data(), sizeof(int32_t) * ck.doff.size(), cudaMemcpyHostToDevice, s));
    DBG_CK(cudaMemcpyAsync(d_start.p, ck.dstart.data(), sizeof(int64_t) * b, cudaMemcpyHostToDevice, s));
    DBuf<T> X, X2, U;
    X.alloc(elems, s);
    X2.alloc(elems, s);
    U.alloc(elems, s);
    DBuf<double> r2;
    r2.alloc(b, s);
    const unsigned grid = (unsigned)std::min<int64_t>(b, (int64_t)num_sms() * 8);
    k_sub_gather<T><<<grid, 256, 0, s>>>(b, d_j.p, d_start.p, d_doff.p, d_n.p, n, H->rp.p, H->col.p, H->off.p,
                                         H->data.p, H->bs.p, mu, inv_alpha, X.p);
    DBG_LAUNCH_CK();
    std::vector<double> h_r2(b);
    ChunkResult cr;
    bool tf32 = mixed;
    const double gemm_flops = 2.0 * (double)n * n * n * b;
    while (true) {
        batched_gemm(b, n, 1.0, X.p, X.p, 0.0, X2.p, !tf32, s);                // X2 = X X
        cr.flops += gemm_flops;
        k_sub_residual<T><<<grid, 256, 0, s>>>(b, n, X2.p, r2.p);
        DBG_LAUNCH_CK();
        DBG_CK(cudaMemcpyAsync(h_r2.data(), r2.p, sizeof(double) * b, cudaMemcpyDeviceToHost, s));
        DBG_CK(cudaStreamSynchronize(s));
        double rm = 0.0;
        for (double v : h_r2) rm = std::max(rm, std::sqrt(v) / n);
        if (!std::isfinite(rm)) fail(DBCSR_ENAN, "submatrix_sign: residual is not finite");
        cr.r_max = rm;
        ++cr.iterations;
        if (tf32) ++cr.tf32_iterations;
        if (o.verbose)
            std::fprintf(stderr, "[submatrix] n_pad %d batch %d it %d %s r_max %.3e\n", n, b, cr.iterations,
                         std::is_same<T, double>::value ? "fp64" : tf32 ? "tf32" : "fp32", rm);
        // No stall test here: a principal submatrix of a gapped H may hold an eigenvalue inside
        // the gap (Cauchy interlacing), whose slow convergence dominates the batch's largest
        // residual and would look like a stall.  The TF32 floor of that residual (about
        // 1e-4 relative error per product over n ~ 400) lies below the switch.
        if (tf32 && rm < o.switch_tol) {
            tf32 = false;
        }
        if (!tf32 && rm < o.tol) break;
        if (cr.iterations >= o.max_iter) break;
        // X <- 1.5 X - 0.5 X X2
        DBG_CK(cudaMemcpyAsync(U.p, X.p, sizeof(T) * elems, cudaMemcpyDeviceToDevice, s));
        batched_gemm(b, n, -0.5, X.p, X2.p, 1.5, U.p, !tf32, s);
        cr.flops += gemm_flops;
        std::swap(X.p, U.p);
    }
    k_sub_scatter<T><<<grid, 256, 0, s>>>(b, d_j.p, d_start.p, d_doff.p, n, P->rp.p, P->col.p, P->off.p, P->bs.p,
                                          X.p, P->data.p);
    DBG_LAUNCH_CK();
    return cr;
}

}  // namespace

dbcsr_status submatrix_sign(dbcsr_matrix_* H, double mu, const dbcsr_sign_opts* opts, dbcsr_matrix_* P,
                            dbcsr_sign_report* rep) {
    check_finalized(H);
    if (!P) fail(DBCSR_EINVAL, "submatrix_sign: null P_out");
    if (P->h_bs != H->h_bs) fail(DBCSR_EINVAL, "submatrix_sign: P_out block sizes differ from H");
    if (P == H) fail(DBCSR_EINVAL, "submatrix_sign: P_out must differ from H");
    check_unplanned(P, "submatrix_sign");
    dbcsr_sign_opts o{};
    o.tol = 1e-9;
    o.max_iter = 100;
    o.prec = DBCSR_FP64;
    if (opts) o = *opts;
    if (o.max_iter <= 0) o.max_iter = 100;
    if (!(o.tol > 0)) fail(DBCSR_EINVAL, "submatrix_sign: need tol > 0");
    if (o.prec != DBCSR_FP64 && o.prec != DBCSR_MIXED) fail(DBCSR_EINVAL, "submatrix_sign: prec must be FP64 or MIXED");
    const bool mixed = o.prec == DBCSR_MIXED;
    if (mixed && !(o.switch_tol > 0)) o.switch_tol = 1e-3;
    const auto t0 = std::chrono::steady_clock::now();
    cudaStream_t s = H->stream;
    const double alpha = gershgorin(H, mu);
    if (!(alpha > 0) || !std::isfinite(alpha)) fail(DBCSR_EINVAL, "submatrix_sign: Gershgorin bound is zero or not finite");

    // the pattern on the host
    const int32_t nblk = H->nblk;
    std::vector<int64_t> rp(nblk + 1);
    std::vector<int32_t> col(std::max<int64_t>(H->nnzb, 1));
    DBG_CK(cudaMemcpyAsync(rp.data(), H->rp.p, sizeof(int64_t) * (nblk + 1), cudaMemcpyDeviceToHost, s));
    if (H->nnzb) DBG_CK(cudaMemcpyAsync(col.data(), H->col.p, sizeof(int32_t) * H->nnzb, cudaMemcpyDeviceToHost, s));
    DBG_CK(cudaStreamSynchronize(s));

    // P takes H's pattern
    copy_matrix(P, H);
    // chunks of submatrices of one padded size
    const size_t elem = mixed ? sizeof(float) : sizeof(double);
    std::map<int, std::vector<int32_t>> by_size;
    for (int32_t j = 0; j < nblk; ++j) {
        int n = 0;
        bool diag = false;
        for (int64_t q = rp[j]; q < rp[j + 1]; ++q) {
            n += H->h_bs[col[q]];
            diag = diag || col[q] == j;
        }
        // the scatter places block column j by its own position in I_j
        if (!diag) fail(DBCSR_EINVAL, "submatrix_sign: a diagonal block is missing");
        by_size[(n + kPad - 1) / kPad * kPad].push_back(j);
    }
    dbcsr_sign_report r{};
    r.alpha = alpha;
    int max_it = 0, max_tf32 = 0;
    double r_max = 0.0, flops = 0.0;
    int64_t nsub = 0;
    for (auto& kv : by_size) {
        const int n_pad = kv.first;
        const size_t per = (size_t)3 * n_pad * n_pad * elem;
        const size_t cap = std::max<size_t>(1, kChunkBytes / per);
        const auto& js = kv.second;
        for (size_t c0 = 0; c0 < js.size(); c0 += cap) {
            Chunk ck;
            ck.n_pad = n_pad;
            for (size_t t = c0; t < std::min(js.size(), c0 + cap); ++t) {
                const int32_t j = js[t];
                ck.sub_j.push_back(j);
                ck.dstart.push_back((int64_t)ck.doff.size());
                int acc = 0;
                for (int64_t q = rp[j]; q < rp[j + 1]; ++q) {
                    ck.doff.push_back(acc);
                    acc += H->h_bs[col[q]];
                }
                ck.sub_n.push_back(acc);
            }
            const ChunkResult cr = mixed ? run_chunk<float>(ck, H, P, mu, 1.0 / alpha, o, true, s)
                                         : run_chunk<double>(ck, H, P, mu, 1.0 / alpha, o, false, s);
            max_it = std::max(max_it, cr.iterations);
            max_tf32 = std::max(max_tf32, cr.tf32_iterations);
            r_max = std::max(r_max, cr.r_max);
            flops += cr.flops;
            nsub += (int64_t)ck.sub_j.size();
        }
    }
    P->norms_valid = false;
    r.trace_p = trace(P);
    r.e_band = trace_product(P, H);
    DBG_CK(cudaStreamSynchronize(s));
    r.iterations = max_it;
    r.fp64_from = mixed ? max_tf32 + 1 : 1;
    r.converged = r_max < o.tol ? 1 : 0;
    r.stalled = 0;
    r.residual = r_max;
    r.flops = flops;
    r.n_products = nsub;
    r.nnzb_x = P->nnzb;
    r.ms_total = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    r.ms_multiply = r.ms_total;
    if (rep) *rep = r;
    return r.converged ? DBCSR_OK : DBCSR_ENOTCONV;
}

}  // namespace dbg
