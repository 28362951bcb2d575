// Traces and the Gershgorin bound.  All reductions are deterministic: per-block
// or per-row partials in a fixed order, then det_sum's fixed tree.
#include "common.cuh"

namespace dbg {
namespace {

__device__ __forceinline__ int64_t find_block(const int64_t* __restrict__ rp, const int32_t* __restrict__ col, int32_t row,
                                              int32_t c) {
    int64_t lo = rp[row], hi = rp[row + 1];
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (col[mid] < c) lo = mid + 1; else hi = mid;
    }
    return (lo < rp[row + 1] && col[lo] == c) ? lo : -1;
}

// part[I] = trace of diagonal block I (0 if absent).
__global__ void k_trace_rows(int32_t nblk, const int32_t* __restrict__ bs, const int64_t* __restrict__ rp,
                             const int32_t* __restrict__ col, const int64_t* __restrict__ off,
                             const double* __restrict__ data, double* __restrict__ part) {
    for (int32_t I = blockIdx.x * blockDim.x + threadIdx.x; I < nblk; I += gridDim.x * blockDim.x) {
        const int64_t q = find_block(rp, col, I, I);
        double s = 0.0;
        if (q >= 0) {
            const int m = bs[I];
            const double* x = data + off[q];
            for (int i = 0; i < m; ++i) s += x[i * m + i];
        }
        part[I] = s;
    }
}

// One warp per block A_IJ: part[b] = <A_IJ, B_JI^T> (0 if B_JI is absent).
__global__ void k_trace_product_blocks(int64_t nb, const int32_t* __restrict__ bs, const int32_t* __restrict__ a_row,
                                       const int32_t* __restrict__ a_col, const int64_t* __restrict__ a_off,
                                       const double* __restrict__ a_data, const int64_t* __restrict__ b_rp,
                                       const int32_t* __restrict__ b_col, const int64_t* __restrict__ b_off,
                                       const double* __restrict__ b_data, double* __restrict__ part) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t b = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); b < nb; b += warps) {
        const int32_t I = a_row[b], J = a_col[b];
        const int64_t q = find_block(b_rp, b_col, J, I);
        double s = 0.0;
        if (q >= 0) {
            const int m = bs[I], n = bs[J];
            const double* x = a_data + a_off[b];
            const double* y = b_data + b_off[q];
            for (int e = lane; e < m * n; e += 32) {
                const int i = e / n, j = e - i * n;
                s = fma(x[e], y[j * m + i], s);
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) part[b] = s;
    }
}

// One warp per block row I (eight per CTA), one lane per matrix row i of it: sum_j |(A - mu 1)_ij|
// in ascending column order; the maximum over rows is taken with an integer atomicMax on the
// bits of the non-negative sum.
constexpr int kGershWarps = 8;
__global__ void __launch_bounds__(32 * kGershWarps)
    k_gershgorin(int32_t nblk, const int32_t* __restrict__ bs, const int64_t* __restrict__ rp,
                 const int32_t* __restrict__ col, const int64_t* __restrict__ off,
                 const double* __restrict__ data, double mu, unsigned long long* __restrict__ maxbits) {
    const int32_t I = (int32_t)(blockIdx.x * kGershWarps + (threadIdx.x >> 5));
    if (I >= nblk) return;
    const int m = bs[I];
    const int i = threadIdx.x & 31;
    if (i >= m) return;
    double s = 0.0;
    bool has_diag = false;
    for (int64_t q = rp[I]; q < rp[I + 1]; ++q) {
        const int32_t J = col[q];
        const int n = bs[J];
        const double* x = data + off[q] + (int64_t)i * n;
        for (int j = 0; j < n; ++j) {
            double v = x[j];
            if (J == I && j == i) v -= mu;
            s += fabs(v);
        }
        has_diag |= (J == I);
    }
    if (!has_diag) s += fabs(mu);
    atomicMax(maxbits, (unsigned long long)__double_as_longlong(s));
}

}  // namespace

double trace(dbcsr_matrix_* m) {
    check_finalized(m);
    cudaStream_t s = m->stream;
    DBuf<double> part, out;
    part.alloc(m->nblk, s);
    out.alloc(1, s);
    k_trace_rows<<<grid_for(m->nblk, 128), 128, 0, s>>>(m->nblk, m->bs.p, m->rp.p, m->col.p, m->off.p, m->data.p,
                                                        part.p);
    DBG_LAUNCH_CK();
    det_sum(part.p, m->nblk, out.p, s);
    return read_f64(out.p, s);
}

double trace_product(dbcsr_matrix_* a, dbcsr_matrix_* b) {
    check_finalized(a);
    check_finalized(b);
    if (a->h_bs != b->h_bs) fail(DBCSR_EINVAL, "trace_product: block sizes differ");
    cudaStream_t s = a->stream;
    if (b->stream != s) DBG_CK(cudaStreamSynchronize(b->stream));
    DBuf<double> part, out;
    part.alloc(std::max<int64_t>(a->nnzb, 1), s);
    out.alloc(1, s);
    if (a->nnzb) {
        k_trace_product_blocks<<<grid_for(a->nnzb, 8), 256, 0, s>>>(a->nnzb, a->bs.p, a->row.p, a->col.p, a->off.p,
                                                                    a->data.p, b->rp.p, b->col.p, b->off.p, b->data.p,
                                                                    part.p);
        DBG_LAUNCH_CK();
    }
    det_sum(part.p, a->nnzb, out.p, s);
    return read_f64(out.p, s);
}

double gershgorin(dbcsr_matrix_* m, double mu) {
    check_finalized(m);
    cudaStream_t s = m->stream;
    DBuf<double> out;
    out.alloc(1, s);
    out.zero();
    k_gershgorin<<<(unsigned)ceil_div(m->nblk, kGershWarps), 32 * kGershWarps, 0, s>>>(m->nblk, m->bs.p, m->rp.p, m->col.p, m->off.p, m->data.p, mu,
                                               (unsigned long long*)out.p);
    DBG_LAUNCH_CK();
    return read_f64(out.p, s);
}

void trace_product_parts_into(dbcsr_matrix_* a, dbcsr_matrix_* b, double* part, cudaStream_t s) {
    if (a->nnzb == 0) return;
    k_trace_product_blocks<<<grid_for(a->nnzb, 8), 256, 0, s>>>(a->nnzb, a->bs.p, a->row.p, a->col.p, a->off.p,
                                                                a->data.p, b->rp.p, b->col.p, b->off.p, b->data.p,
                                                                part);
    DBG_LAUNCH_CK();
}

}  // namespace dbg
