// Many independent sign iterations solved as one batch.
//
// The systems' matrices are stacked into one block-diagonal matrix
// H_batch = diag(H_1, ..., H_n) (blocks of system s keep their sizes; block rows
// and columns are shifted by the rows of the systems before it).  A product of
// block-diagonal matrices stays block-diagonal, so one product over the batch
// forms every system's blocks at once: the stack builder lists all systems'
// block products together and each block-shape class runs as one launch for the
// whole batch, instead of one set of launches (and host round trips) per system.
//
// Per system: its own Gershgorin scale alpha_s, X_0 = (H_s - mu_s 1) / alpha_s,
// residual r_s = ||X2_s - 1||_F / N_s from the blocks of its rows, and its own
// convergence / stall record (same tests as the single-system iteration).  A
// system that is done leaves the batch at once: its P is written out and the batch
// matrices are compacted to the systems still running, so later products spend
// nothing on it.  With DBCSR_MIXED the whole batch leaves the low-precision tier
// once any system's residual drops below the switch.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <memory>
#include <vector>

#include "common.cuh"

namespace dbg {
namespace {

__global__ void k_shift_i32(int64_t n, const int32_t* __restrict__ in, int32_t add, int32_t* __restrict__ out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = in[i] + add;
}

__global__ void k_gather_i64(int64_t n, const int64_t* __restrict__ idx, const int64_t* __restrict__ src,
                             int64_t* __restrict__ out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = src[idx[i]];
}

__global__ void k_shift_i64(int64_t n, const int64_t* __restrict__ in, int64_t add, int64_t* __restrict__ out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = in[i] + add;
}

// Per-system Gershgorin bound: one thread per matrix row, max over the system's rows.
__global__ void k_gershgorin_sys(int32_t nblk, const int32_t* __restrict__ bs, const int64_t* __restrict__ rp,
                                 const int32_t* __restrict__ col, const int64_t* __restrict__ off,
                                 const double* __restrict__ data, const int32_t* __restrict__ row_sys,
                                 const double* __restrict__ mu, unsigned long long* __restrict__ maxbits) {
    const int32_t I = blockIdx.x;
    const int m = bs[I];
    const int i = threadIdx.x;
    if (i >= m) return;
    const int32_t sys = row_sys[I];
    const double shift = mu[sys];
    double s = 0.0;
    bool has_diag = false;
    for (int64_t q = rp[I]; q < rp[I + 1]; ++q) {
        const int32_t J = col[q];
        const int n = bs[J];
        const double* x = data + off[q] + (int64_t)i * n;
        for (int j = 0; j < n; ++j) {
            double v = x[j];
            if (J == I && j == i) v -= shift;
            s += fabs(v);
        }
        has_diag |= (J == I);
    }
    if (!has_diag) s += fabs(shift);
    atomicMax(maxbits + sys, (unsigned long long)__double_as_longlong(s));
}

// X = (H - mu_s 1) / alpha_s, one warp per block.
__global__ void k_scale_shift_sys(int64_t nb, const int32_t* __restrict__ row, const int32_t* __restrict__ col,
                                  const int32_t* __restrict__ bs, const int64_t* __restrict__ off,
                                  double* __restrict__ data, const int32_t* __restrict__ row_sys,
                                  const double* __restrict__ scale, const double* __restrict__ shift) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t b = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); b < nb; b += warps) {
        const int I = row[b], J = col[b];
        const int32_t sys = row_sys[I];
        const double sc = scale[sys], sh = shift[sys];
        const int n = bs[J], area = bs[I] * n;
        double* x = data + off[b];
        for (int e = lane; e < area; e += 32) {
            double v = sc * x[e];
            if (I == J && (e / n) == (e % n)) v += sh;
            x[e] = v;
        }
    }
}

// Per-system sum of v over the blocks of the system's rows, [bbeg[s], bbeg[s+1]):
// one CTA per system, fixed thread-strided order and tree (deterministic).
__global__ void k_segment_sum(int32_t nsys, const int64_t* __restrict__ bbeg, const double* __restrict__ v,
                              double* __restrict__ out) {
    __shared__ double sh[256];
    for (int32_t s = blockIdx.x; s < nsys; s += gridDim.x) {
        double acc = 0.0;
        for (int64_t b = bbeg[s] + threadIdx.x; b < bbeg[s + 1]; b += blockDim.x) acc += v[b];
        sh[threadIdx.x] = acc;
        __syncthreads();
        for (int w = 128; w > 0; w >>= 1) {
            if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
            __syncthreads();
        }
        if (threadIdx.x == 0) out[s] = sh[0];
        __syncthreads();
    }
}

__global__ void k_bbeg_from_rows(int32_t nsys, const int64_t* __restrict__ rp, const int32_t* __restrict__ row_beg,
                                 int64_t* __restrict__ bbeg) {
    for (int32_t s = blockIdx.x * blockDim.x + threadIdx.x; s <= nsys; s += gridDim.x * blockDim.x)
        bbeg[s] = rp[row_beg[s]];
}

std::unique_ptr<dbcsr_matrix_> make_matrix(const std::vector<int32_t>& bs, cudaStream_t s) {
    auto x = std::make_unique<dbcsr_matrix_>();
    x->nblk = (int32_t)bs.size();
    x->stream = s;
    x->h_bs = bs;
    x->n = 0;
    for (int32_t b : bs) x->n += b;
    x->bs.alloc(x->nblk, s);
    DBG_CK(cudaMemcpyAsync(x->bs.p, bs.data(), sizeof(int32_t) * bs.size(), cudaMemcpyHostToDevice, s));
    return x;
}

}  // namespace

dbcsr_status sign_iterate_batched(int32_t nsys, dbcsr_matrix_* const* H, const double* mu, const dbcsr_sign_opts* opts,
                                  dbcsr_matrix_* const* P, dbcsr_sign_report* reps) {
    if (nsys < 1 || !H || !mu || !P) fail(DBCSR_EINVAL, "sign_iterate_batched: need nsys >= 1, H, mu and P_out");
    for (int32_t s = 0; s < nsys; ++s) {
        check_finalized(H[s]);
        if (!P[s] || P[s]->h_bs != H[s]->h_bs) fail(DBCSR_EINVAL, "sign_iterate_batched: P_out[s] missing or of other sizes");
    }
    dbcsr_sign_opts o{};
    o.tol = 1e-9;
    o.max_iter = 100;
    o.prec = DBCSR_FP64;
    o.stall_ratio = 0.5;
    if (opts) o = *opts;
    if (o.max_iter <= 0) o.max_iter = 100;
    if (o.stall_ratio <= 0) o.stall_ratio = 0.5;
    if (!(o.eps_filter >= 0) || !(o.tol > 0)) fail(DBCSR_EINVAL, "sign_iterate_batched: need eps_filter >= 0 and tol > 0");
    if (o.prec != DBCSR_FP64 && o.prec != DBCSR_MIXED) fail(DBCSR_EINVAL, "sign_iterate_batched: prec must be FP64 or MIXED");
    if (o.prec == DBCSR_MIXED && !(o.switch_tol > 0)) o.switch_tol = 1e-4;
    if (o.order == 0) o.order = 2;
    if (o.order < 2 || o.order > 7) fail(DBCSR_EINVAL, "sign_iterate_batched: order must be 2 to 7");
    if (o.order != 2 && (o.flags & DBCSR_SIGN_LOW_CORRECTION))
        fail(DBCSR_EINVAL, "sign_iterate_batched: the low-precision correction applies to order 2 only");
    // Every product of the iteration is symmetric in exact arithmetic.  FP64 and split-BF16
    // products compute the blocks I <= J and mirror the rest; a plain BF16 tier forms full
    // products throughout and X's symmetric part is taken at the end.
    const bool full = (o.flags & DBCSR_SIGN_FULL_PRODUCTS) != 0;
    const int low = (o.flags & DBCSR_SIGN_PLAIN_BF16) ? DBCSR_BF16 : DBCSR_BF16X3;
    const bool full_mixed = o.prec == DBCSR_MIXED && low == DBCSR_BF16;
    const bool correction = o.prec == DBCSR_MIXED && (o.flags & DBCSR_SIGN_LOW_CORRECTION) != 0;

    const auto t0 = std::chrono::steady_clock::now();
    cudaStream_t st = H[0]->stream;
    for (int32_t s = 1; s < nsys; ++s)
        if (H[s]->stream != st) DBG_CK(cudaStreamSynchronize(H[s]->stream));

    // ---- stack the systems into one block-diagonal matrix
    std::vector<int32_t> bs, row_beg(nsys + 1, 0), row_sys;
    std::vector<double> nsys_dim(nsys);
    int64_t nnzb = 0, nel = 0;
    for (int32_t s = 0; s < nsys; ++s) {
        row_beg[s] = (int32_t)bs.size();
        bs.insert(bs.end(), H[s]->h_bs.begin(), H[s]->h_bs.end());
        row_sys.insert(row_sys.end(), H[s]->nblk, s);
        nnzb += H[s]->nnzb;
        nel += H[s]->nel;
        nsys_dim[s] = (double)H[s]->n;
    }
    row_beg[nsys] = (int32_t)bs.size();
    const int32_t nblk = (int32_t)bs.size();
    auto HB = make_matrix(bs, st);
    HB->rp.alloc(nblk + 1, st);
    HB->col.alloc(std::max<int64_t>(nnzb, 1), st);
    HB->row.alloc(std::max<int64_t>(nnzb, 1), st);
    HB->off.alloc(nnzb + 1, st);
    HB->data.alloc(std::max<int64_t>(nel, 1), st);
    int64_t bo = 0, eo = 0;
    for (int32_t s = 0; s < nsys; ++s) {
        const dbcsr_matrix_* h = H[s];
        const int32_t ro = row_beg[s];
        k_shift_i64<<<grid_for(h->nblk + 1, 256), 256, 0, st>>>(h->nblk + 1, h->rp.p, bo, HB->rp.p + ro);
        DBG_LAUNCH_CK();
        if (h->nnzb) {
            k_shift_i32<<<grid_for(h->nnzb, 256), 256, 0, st>>>(h->nnzb, h->col.p, ro, HB->col.p + bo);
            DBG_LAUNCH_CK();
            k_shift_i32<<<grid_for(h->nnzb, 256), 256, 0, st>>>(h->nnzb, h->row.p, ro, HB->row.p + bo);
            DBG_LAUNCH_CK();
        }
        k_shift_i64<<<grid_for(h->nnzb + 1, 256), 256, 0, st>>>(h->nnzb + 1, h->off.p, eo, HB->off.p + bo);
        DBG_LAUNCH_CK();
        if (h->nel) DBG_CK(cudaMemcpyAsync(HB->data.p + eo, h->data.p, sizeof(double) * h->nel, cudaMemcpyDeviceToDevice, st));
        bo += h->nnzb;
        eo += h->nel;
    }
    HB->nnzb = nnzb;
    HB->nel = nel;
    HB->finalized = true;

    DBuf<int32_t> d_row_sys, d_row_beg;
    DBuf<double> d_mu, d_scale, d_shift, d_alpha, d_dev2;
    DBuf<int64_t> d_bbeg;
    d_row_sys.alloc(nblk, st);
    d_row_beg.alloc(nsys + 1, st);
    d_mu.alloc(nsys, st);
    d_scale.alloc(nsys, st);
    d_shift.alloc(nsys, st);
    d_alpha.alloc(nsys, st);
    d_dev2.alloc(nsys, st);
    d_bbeg.alloc(nsys + 1, st);
    DBG_CK(cudaMemcpyAsync(d_row_sys.p, row_sys.data(), sizeof(int32_t) * nblk, cudaMemcpyHostToDevice, st));
    DBG_CK(cudaMemcpyAsync(d_row_beg.p, row_beg.data(), sizeof(int32_t) * (nsys + 1), cudaMemcpyHostToDevice, st));
    DBG_CK(cudaMemcpyAsync(d_mu.p, mu, sizeof(double) * nsys, cudaMemcpyHostToDevice, st));

    // ---- per-system scale and X_0
    d_alpha.zero();
    k_gershgorin_sys<<<nblk, kMaxBlock, 0, st>>>(nblk, HB->bs.p, HB->rp.p, HB->col.p, HB->off.p, HB->data.p, d_row_sys.p,
                                                 d_mu.p, (unsigned long long*)d_alpha.p);
    DBG_LAUNCH_CK();
    std::vector<double> alpha(nsys), scale(nsys), shift(nsys);
    DBG_CK(cudaMemcpyAsync(alpha.data(), d_alpha.p, sizeof(double) * nsys, cudaMemcpyDeviceToHost, st));
    DBG_CK(cudaStreamSynchronize(st));
    for (int32_t s = 0; s < nsys; ++s) {
        if (!(alpha[s] > 0) || !std::isfinite(alpha[s]))
            fail(DBCSR_EINVAL, "sign_iterate_batched: Gershgorin bound of system " + std::to_string(s) + " is zero or not finite");
        scale[s] = 1.0 / alpha[s];
        shift[s] = -mu[s] / alpha[s];
    }
    DBG_CK(cudaMemcpyAsync(d_scale.p, scale.data(), sizeof(double) * nsys, cudaMemcpyHostToDevice, st));
    DBG_CK(cudaMemcpyAsync(d_shift.p, shift.data(), sizeof(double) * nsys, cudaMemcpyHostToDevice, st));
    auto X = make_matrix(bs, st);
    auto X2 = make_matrix(bs, st);
    copy_matrix(X.get(), HB.get());
    if (X->nnzb) {
        k_scale_shift_sys<<<grid_for(X->nnzb, 8), 256, 0, st>>>(X->nnzb, X->row.p, X->col.p, X->bs.p, X->off.p,
                                                                X->data.p, d_row_sys.p, d_scale.p, d_shift.p);
        DBG_LAUNCH_CK();
    }
    X->norms_valid = false;

    // ---- iteration
    std::vector<dbcsr_sign_report> rep(nsys);
    std::vector<int> done(nsys, 0);      // 0 running, 1 converged, 2 stalled, 3 max_iter
    for (int32_t s = 0; s < nsys; ++s) {
        rep[s] = dbcsr_sign_report{};
        rep[s].alpha = alpha[s];
    }
    int tier = (o.prec == DBCSR_MIXED) ? low : DBCSR_FP64;
    int first_fp64 = (tier == DBCSR_FP64) ? 1 : 0;
    const int sym = (full || full_mixed) ? kSymNone : kSymMirror;
    double flops = 0.0, ms_mult = 0.0, ms_sym = 0.0, ms_filt = 0.0, ms_low = 0.0, flops_low = 0.0, bytes_min = 0.0;
    int64_t nprod = 0, launches_fp64 = 0;
    auto account = [&](const dbcsr_mult_stats& ms, int tier_of_product) {
        flops += ms.flops;
        nprod += ms.n_products;
        ms_mult += ms.ms_numeric;
        ms_sym += ms.ms_symbolic;
        ms_filt += ms.ms_filter;
        if (tier_of_product != DBCSR_FP64) {
            ms_low += ms.ms_numeric;
            flops_low += ms.flops;
        } else {
            bytes_min += ms.bytes_min;
            launches_fp64 += ms.n_launches;
        }
    };
    // Active systems, in batch order, with their block-row ranges in the current X.  A system
    // that is done leaves the batch at once: its P is written and X (and X2, which the next
    // update reads) are compacted to the systems still running, so no product is spent on
    // a finished system.
    std::vector<int32_t> act(nsys), act_beg(row_beg);
    for (int32_t s = 0; s < nsys; ++s) act[s] = s;
    std::vector<int32_t> cur_bs = bs;
    DBuf<int64_t> d_idx, d_vals;
    // block and element offsets of the active systems' ranges in m: b[a], e[a] for a = 0..nact
    auto range_offsets = [&](const dbcsr_matrix_* m, std::vector<int64_t>& b, std::vector<int64_t>& e) {
        const size_t na = act.size();
        std::vector<int64_t> hrp(m->nblk + 1);
        DBG_CK(cudaMemcpyAsync(hrp.data(), m->rp.p, sizeof(int64_t) * (m->nblk + 1), cudaMemcpyDeviceToHost, st));
        DBG_CK(cudaStreamSynchronize(st));
        b.resize(na + 1);
        for (size_t a = 0; a <= na; ++a) b[a] = hrp[act_beg[a]];
        d_idx.alloc((int64_t)na + 1, st);
        d_vals.alloc((int64_t)na + 1, st);
        DBG_CK(cudaMemcpyAsync(d_idx.p, b.data(), sizeof(int64_t) * (na + 1), cudaMemcpyHostToDevice, st));
        k_gather_i64<<<grid_for((int64_t)na + 1, 256), 256, 0, st>>>((int64_t)na + 1, d_idx.p, m->off.p, d_vals.p);
        DBG_LAUNCH_CK();
        e.resize(na + 1);
        DBG_CK(cudaMemcpyAsync(e.data(), d_vals.p, sizeof(int64_t) * (na + 1), cudaMemcpyDeviceToHost, st));
        DBG_CK(cudaStreamSynchronize(st));
    };
    // copies rows [r0, r1) of the block-diagonal m (blocks [b0, b1), elements [e0, e1)) into
    // dst at block row dr0, block db0, element de0
    auto copy_rows = [&](const dbcsr_matrix_* m, int32_t r0, int32_t r1, int64_t b0, int64_t b1, int64_t e0, int64_t e1,
                         dbcsr_matrix_* dst, int32_t dr0, int64_t db0, int64_t de0, cudaStream_t ds) {
        k_shift_i64<<<grid_for(r1 - r0 + 1, 256), 256, 0, ds>>>(r1 - r0 + 1, m->rp.p + r0, db0 - b0, dst->rp.p + dr0);
        DBG_LAUNCH_CK();
        if (b1 > b0) {
            k_shift_i32<<<grid_for(b1 - b0, 256), 256, 0, ds>>>(b1 - b0, m->col.p + b0, dr0 - r0, dst->col.p + db0);
            DBG_LAUNCH_CK();
            k_shift_i32<<<grid_for(b1 - b0, 256), 256, 0, ds>>>(b1 - b0, m->row.p + b0, dr0 - r0, dst->row.p + db0);
            DBG_LAUNCH_CK();
        }
        k_shift_i64<<<grid_for(b1 - b0 + 1, 256), 256, 0, ds>>>(b1 - b0 + 1, m->off.p + b0, de0 - e0, dst->off.p + db0);
        DBG_LAUNCH_CK();
        if (e1 > e0)
            DBG_CK(cudaMemcpyAsync(dst->data.p + de0, m->data.p + e0, sizeof(double) * (e1 - e0), cudaMemcpyDeviceToDevice, ds));
    };
    // the active systems flagged in `leave` leave the batch: P_s = (1 - X_s) / 2, then X and
    // (when given) X2 keep only the others
    auto retire = [&](const std::vector<char>& leave, dbcsr_matrix_* x2) {
        std::vector<int64_t> xb, xe, yb, ye;
        range_offsets(X.get(), xb, xe);
        if (x2) range_offsets(x2, yb, ye);
        const size_t na = act.size();
        for (size_t a = 0; a < na; ++a) {
            if (!leave[a]) continue;
            const int32_t sid = act[a];
            dbcsr_matrix_* pm = P[sid];
            cudaStream_t ps = pm->stream;
            if (ps != st) DBG_CK(cudaStreamSynchronize(st));
            const int32_t nb_s = act_beg[a + 1] - act_beg[a];
            const int64_t nbk = xb[a + 1] - xb[a], nel_s = xe[a + 1] - xe[a];
            pm->rp.alloc(nb_s + 1, ps);
            pm->col.alloc(std::max<int64_t>(nbk, 1), ps);
            pm->row.alloc(std::max<int64_t>(nbk, 1), ps);
            pm->off.alloc(nbk + 1, ps);
            pm->data.alloc(std::max<int64_t>(nel_s, 1), ps);
            copy_rows(X.get(), act_beg[a], act_beg[a + 1], xb[a], xb[a + 1], xe[a], xe[a + 1], pm, 0, 0, 0, ps);
            pm->nnzb = nbk;
            pm->nel = nel_s;
            pm->norms_valid = false;
            pm->finalized = true;
            // X of a mixed run with a plain BF16 tier is symmetric only to that tier's accuracy: keep
            // its symmetric part (mirrored products keep X exactly symmetric)
            if (full_mixed && !full) symmetrize(pm);
            scale_shift(pm, -0.5, 0.5);
            dbcsr_sign_report& R = rep[sid];
            R.trace_p = trace(pm);
            R.e_band = trace_product(pm, H[sid]);
            R.converged = done[sid] == 1;
            R.stalled = done[sid] == 2;
            R.fp64_from = first_fp64;
            R.nnzb_x = pm->nnzb;
        }
        // (trace_product synchronised each P's stream, so nothing still reads the old X)
        // the systems that stay, renumbered from block row 0
        std::vector<int32_t> nact, nbeg{0}, nbs;
        for (size_t a = 0; a < na; ++a) {
            if (leave[a]) continue;
            nact.push_back(act[a]);
            nbs.insert(nbs.end(), cur_bs.begin() + act_beg[a], cur_bs.begin() + act_beg[a + 1]);
            nbeg.push_back((int32_t)nbs.size());
        }
        auto rebuild = [&](const dbcsr_matrix_* m, const std::vector<int64_t>& b, const std::vector<int64_t>& e) {
            int64_t nnzb_new = 0, nel_new = 0;
            for (size_t a = 0; a < na; ++a)
                if (!leave[a]) {
                    nnzb_new += b[a + 1] - b[a];
                    nel_new += e[a + 1] - e[a];
                }
            auto y = make_matrix(nbs, st);
            y->rp.alloc(y->nblk + 1, st);
            y->col.alloc(std::max<int64_t>(nnzb_new, 1), st);
            y->row.alloc(std::max<int64_t>(nnzb_new, 1), st);
            y->off.alloc(nnzb_new + 1, st);
            y->data.alloc(std::max<int64_t>(nel_new, 1), st);
            int64_t db = 0, de = 0;
            size_t k = 0;
            for (size_t a = 0; a < na; ++a) {
                if (leave[a]) continue;
                copy_rows(m, act_beg[a], act_beg[a + 1], b[a], b[a + 1], e[a], e[a + 1], y.get(), nbeg[k], db, de, st);
                db += b[a + 1] - b[a];
                de += e[a + 1] - e[a];
                ++k;
            }
            y->nnzb = nnzb_new;
            y->nel = nel_new;
            y->norms_valid = false;
            y->finalized = true;
            return y;
        };
        if (!nact.empty()) {
            // each old matrix is freed (stream-ordered, after its copies) before the next is rebuilt
            X = rebuild(X.get(), xb, xe);
            if (x2) X2 = rebuild(x2, yb, ye);
        }
        act = std::move(nact);
        act_beg = std::move(nbeg);
        cur_bs = std::move(nbs);
        if (!act.empty())
            DBG_CK(cudaMemcpyAsync(d_row_beg.p, act_beg.data(), sizeof(int32_t) * act_beg.size(), cudaMemcpyHostToDevice, st));
    };

    std::vector<double> dev2(nsys);
    DBuf<double> blk_dev2;
    int it = 0;
    while (it < o.max_iter && !act.empty()) {
        const int32_t nact = (int32_t)act.size();
        dbcsr_mult_stats ms{};
        multiply(1.0, X.get(), X.get(), 0.0, X2.get(), o.eps_filter, tier, &ms, false, sym);
        account(ms, tier);
        ++it;
        // per-system ||X2_s - 1||_F^2 over the kept blocks of the system's rows
        blk_dev2.alloc(std::max<int64_t>(X2->nnzb, 1), st);
        compute_block_norms(X2.get(), nullptr, blk_dev2.p);
        k_bbeg_from_rows<<<1, 128, 0, st>>>(nact, X2->rp.p, d_row_beg.p, d_bbeg.p);
        DBG_LAUNCH_CK();
        k_segment_sum<<<std::min<int32_t>(nact, 1024), 256, 0, st>>>(nact, d_bbeg.p, blk_dev2.p, d_dev2.p);
        DBG_LAUNCH_CK();
        DBG_CK(cudaMemcpyAsync(dev2.data(), d_dev2.p, sizeof(double) * nact, cudaMemcpyDeviceToHost, st));
        DBG_CK(cudaStreamSynchronize(st));
        bool any_below_switch = false, any_done = false;
        std::vector<char> leave(nact, 0);
        for (int32_t a = 0; a < nact; ++a) {
            const int32_t sid = act[a];
            const double r = std::sqrt(dev2[a]) / nsys_dim[sid];
            dbcsr_sign_report& R = rep[sid];
            if (!std::isfinite(r)) fail(DBCSR_ENAN, "sign_iterate_batched: residual of system " + std::to_string(sid) + " is not finite");
            if (it - 1 < DBCSR_MAX_HISTORY) R.residual_history[it - 1] = r;
            R.iterations = it;
            R.residual = r;
            const bool slow = it >= 3 && it - 1 < DBCSR_MAX_HISTORY &&
                              R.residual_history[it - 2] < o.stall_ratio * R.residual_history[it - 3] &&
                              r > o.stall_ratio * R.residual_history[it - 2];
            if (tier == DBCSR_FP64) {
                if (r < o.tol) done[sid] = 1;
                else if (slow && it >= first_fp64 + 2) done[sid] = 2;
            } else if (r < o.switch_tol || r < o.tol || slow) {
                any_below_switch = true;
            }
            if (done[sid]) {
                leave[a] = 1;
                any_done = true;
            }
        }
        if (o.verbose)
            std::fprintf(stderr, "[batch] it %3d %s systems running %d/%d formed %lld %.1f GF %.2f ms\n", it,
                         tier == DBCSR_FP64 ? "fp64" : tier == DBCSR_BF16 ? "bf16" : "bf16x3", nact, nsys,
                         (long long)ms.n_formed, ms.flops * 1e-9, ms.ms_numeric);
        if (any_done) retire(leave, X2.get());
        if (act.empty()) break;
        if (tier != DBCSR_FP64 && any_below_switch) {
            tier = DBCSR_FP64;
            first_fp64 = it + 1;
        }
        sign_update(X.get(), X2.get(), o.order, correction, o.eps_filter, tier, sym, account);
    }
    // systems still running at max_iter
    for (int32_t sid : act) done[sid] = 3;
    if (!act.empty()) retire(std::vector<char>(act.size(), 1), nullptr);
    DBG_CK(cudaStreamSynchronize(st));
    const double ms_total = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    bool all_conv = true;
    for (int32_t s = 0; s < nsys; ++s) {
        // the work of the batch is shared: every report carries the batch totals
        rep[s].flops = flops;
        rep[s].n_products = nprod;
        rep[s].ms_total = ms_total;
        rep[s].ms_multiply = ms_mult;
        rep[s].ms_symbolic = ms_sym;
        rep[s].ms_filter = ms_filt;
        rep[s].ms_low = ms_low;
        rep[s].flops_low = flops_low;
        rep[s].bytes_min_fp64 = bytes_min;
        rep[s].launches_fp64 = launches_fp64;
        all_conv = all_conv && rep[s].converged;
        if (reps) reps[s] = rep[s];
    }
    return all_conv ? DBCSR_OK : DBCSR_ENOTCONV;
}

}  // namespace dbg

extern "C" dbcsr_status dbcsr_sign_iterate_batched(int32_t nsys, const dbcsr_matrix* H, const double* mu,
                                                   const dbcsr_sign_opts* opts, dbcsr_matrix* P_out,
                                                   dbcsr_sign_report* reps) {
    dbcsr_status st = DBCSR_OK;
    try {
        st = dbg::sign_iterate_batched(nsys, H, mu, opts, P_out, reps);
        dbg::set_last_error(st == DBCSR_OK ? "" : "a system of the batch did not reach the tolerance");
        return st;
    } catch (const dbg::Error& e) {
        dbg::set_last_error(e.what());
        return e.code;
    } catch (const std::exception& e) {
        dbg::set_last_error(e.what());
        return DBCSR_EINVAL;
    }
}
