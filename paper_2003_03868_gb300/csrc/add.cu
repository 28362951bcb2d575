// Block-sparse matrix sum A <- alpha A + beta B on the union of the two patterns
// (DBCSR's add, used to assemble the polynomials of the higher-order sign
// iterations, section "Sign-Method").  No filtering: the paper flushes small
// elements after multiplications only.
//
// Each term is rounded on its own and then added (alpha*a + beta*b with no fused
// multiply-add), so the sum is the same on every run and in every launch shape.
#include "common.cuh"

namespace dbg {
namespace {

// First position p in col[lo, hi) with col[p] >= c.
__device__ __forceinline__ int64_t lower_bound(const int32_t* __restrict__ col, int64_t lo, int64_t hi, int32_t c) {
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (col[mid] < c) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// One warp per block row I: the sorted union of A's and B's columns in row I.
// The union position of a column c is (A columns < c) + (B columns < c) - (common
// columns < c); the common ones are counted with a ballot over the A columns.
// Count pass (c_rp == nullptr): cnt[I] = size of the union.  Fill pass: writes the
// union's columns, rows, areas and the source block in A and B (-1 when absent).
__global__ void k_union_rows(int32_t nblk, const int32_t* __restrict__ bs, const int64_t* __restrict__ a_rp,
                             const int32_t* __restrict__ a_col, const int64_t* __restrict__ b_rp,
                             const int32_t* __restrict__ b_col, const int64_t* __restrict__ c_rp,
                             int64_t* __restrict__ cnt, int32_t* __restrict__ c_col, int32_t* __restrict__ c_row,
                             int64_t* __restrict__ c_area, int64_t* __restrict__ src_a, int64_t* __restrict__ src_b) {
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t I = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); I < nblk; I += warps) {
        const int64_t a0 = a_rp[I], a1 = a_rp[I + 1], b0 = b_rp[I], b1 = b_rp[I + 1];
        const int64_t base = c_rp ? c_rp[I] : 0;
        const int mI = bs[I];
        int64_t common = 0;
        for (int64_t q0 = a0; q0 < a1; q0 += 32) {
            const int64_t q = q0 + lane;
            bool found = false;
            int32_t c = 0;
            int64_t k = b0;
            if (q < a1) {
                c = a_col[q];
                k = lower_bound(b_col, b0, b1, c);
                found = k < b1 && b_col[k] == c;
            }
            const unsigned m = __ballot_sync(0xffffffffu, found);
            if (c_rp && q < a1) {
                const int64_t pos = base + (q - a0) + (k - b0) - (common + __popc(m & lt));
                c_col[pos] = c;
                c_row[pos] = (int32_t)I;
                c_area[pos] = (int64_t)mI * bs[c];
                src_a[pos] = q;
                src_b[pos] = found ? k : -1;
            }
            common += __popc(m);
        }
        if (!c_rp) {
            if (lane == 0) cnt[I] = (a1 - a0) + (b1 - b0) - common;
            continue;
        }
        // B columns that A lacks
        int64_t common_b = 0;
        for (int64_t q0 = b0; q0 < b1; q0 += 32) {
            const int64_t q = q0 + lane;
            bool found = false;
            int32_t c = 0;
            int64_t k = a0;
            if (q < b1) {
                c = b_col[q];
                k = lower_bound(a_col, a0, a1, c);
                found = k < a1 && a_col[k] == c;
            }
            const unsigned m = __ballot_sync(0xffffffffu, found);
            if (q < b1 && !found) {
                const int64_t pos = base + (q - b0) + (k - a0) - (common_b + __popc(m & lt));
                c_col[pos] = c;
                c_row[pos] = (int32_t)I;
                c_area[pos] = (int64_t)mI * bs[c];
                src_a[pos] = -1;
                src_b[pos] = q;
            }
            common_b += __popc(m);
        }
    }
}

// One warp per union block: alpha * A block + beta * B block (a missing one counts as absent,
// not as a zero term).
__global__ void k_add_values(int64_t nb, const int64_t* __restrict__ src_a, const int64_t* __restrict__ src_b,
                             const int64_t* __restrict__ a_off, const double* __restrict__ a_data,
                             const int64_t* __restrict__ b_off, const double* __restrict__ b_data,
                             const int64_t* __restrict__ c_off, double* __restrict__ c_data, double alpha,
                             double beta) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t b = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); b < nb; b += warps) {
        const int64_t sa = src_a[b], sb = src_b[b];
        const int64_t area = c_off[b + 1] - c_off[b];
        const double* x = sa >= 0 ? a_data + a_off[sa] : nullptr;
        const double* y = sb >= 0 ? b_data + b_off[sb] : nullptr;
        double* d = c_data + c_off[b];
        for (int64_t e = lane; e < area; e += 32) {
            double v;
            if (x && y) v = __dadd_rn(__dmul_rn(alpha, x[e]), __dmul_rn(beta, y[e]));
            else if (x) v = __dmul_rn(alpha, x[e]);
            else v = __dmul_rn(beta, y[e]);
            d[e] = v;
        }
    }
}

}  // namespace

void add(dbcsr_matrix_* A, double alpha, const dbcsr_matrix_* B, double beta) {
    if (!A || !B) fail(DBCSR_EINVAL, "add: null matrix handle");
    check_unplanned(A, "add");
    check_finalized(A);
    check_finalized(B);
    if (A->h_bs != B->h_bs) fail(DBCSR_EINVAL, "add: block sizes differ");
    cudaStream_t s = A->stream;
    if (B->stream != s) DBG_CK(cudaStreamSynchronize(B->stream));
    const int32_t nblk = A->nblk;
    DBuf<int64_t> cnt, rp;
    cnt.alloc(std::max<int32_t>(nblk, 1), s);
    rp.alloc(nblk + 1, s);
    if (nblk) {
        k_union_rows<<<grid_for(nblk, 8), 256, 0, s>>>(nblk, A->bs.p, A->rp.p, A->col.p, B->rp.p, B->col.p, nullptr,
                                                      cnt.p, nullptr, nullptr, nullptr, nullptr, nullptr);
        DBG_LAUNCH_CK();
    }
    scan_exclusive(cnt.p, rp.p, nblk, s);
    const int64_t nb = read_i64(rp.p + nblk, s);
    DBuf<int32_t> col, row;
    DBuf<int64_t> area, off, sa, sb;
    col.alloc(std::max<int64_t>(nb, 1), s);
    row.alloc(std::max<int64_t>(nb, 1), s);
    area.alloc(std::max<int64_t>(nb, 1), s);
    sa.alloc(std::max<int64_t>(nb, 1), s);
    sb.alloc(std::max<int64_t>(nb, 1), s);
    off.alloc(nb + 1, s);
    if (nblk) {
        k_union_rows<<<grid_for(nblk, 8), 256, 0, s>>>(nblk, A->bs.p, A->rp.p, A->col.p, B->rp.p, B->col.p, rp.p,
                                                      nullptr, col.p, row.p, area.p, sa.p, sb.p);
        DBG_LAUNCH_CK();
    }
    scan_exclusive(area.p, off.p, nb, s);
    const int64_t nel = read_i64(off.p + nb, s);
    DBuf<double> data;
    data.alloc(std::max<int64_t>(nel, 1), s);
    if (nb) {
        k_add_values<<<grid_for(nb, 8), 256, 0, s>>>(nb, sa.p, sb.p, A->off.p, A->data.p, B->off.p, B->data.p, off.p,
                                                    data.p, alpha, beta);
        DBG_LAUNCH_CK();
    }
    // A's old arrays (B's too when B is A) are released in stream order, after the kernels read them
    A->rp = std::move(rp);
    A->col = std::move(col);
    A->row = std::move(row);
    A->off = std::move(off);
    A->data = std::move(data);
    A->nnzb = nb;
    A->nel = nel;
    A->norms_valid = false;
}

}  // namespace dbg
