// Density matrix by the second-order Newton-Schulz sign iteration
// (section "Sign-Method": sign(A) = A (A^2)^(-1/2), P = (1 - sign(H - mu 1)) / 2
// with S = 1, eps_filter truncation after every product).
//
//   X_0 = (H - mu 1) / alpha,  alpha = Gershgorin bound of H - mu 1
//   repeat:  X2 = filter(X X);  r = ||X2 - 1||_F / N;  stop when r < tol
//            X  = filter(1.5 X - 0.5 X X2)       ( = X (3 - X^2) / 2 )
//   P = (1 - X) / 2,  Tr(P),  E_band = Tr(P H)
#include <chrono>
#include <cmath>
#include <cstdio>
#include <memory>

#include "common.cuh"

namespace dbg {

namespace {

std::unique_ptr<dbcsr_matrix_> make_like(const dbcsr_matrix_* m, cudaStream_t s) {
    auto x = std::make_unique<dbcsr_matrix_>();
    x->nblk = m->nblk;
    x->n = m->n;
    x->stream = s;
    x->h_bs = m->h_bs;
    x->bs.alloc(m->nblk, s);
    DBG_CK(cudaMemcpyAsync(x->bs.p, m->bs.p, sizeof(int32_t) * m->nblk, cudaMemcpyDeviceToDevice, s));
    return x;
}

}  // namespace

dbcsr_status sign_iterate(dbcsr_matrix_* H, double mu, const dbcsr_sign_opts* opts, dbcsr_matrix_* P,
                          dbcsr_sign_report* rep) {
    check_finalized(H);
    if (!P) fail(DBCSR_EINVAL, "sign_iterate: null P_out");
    if (P->h_bs != H->h_bs) fail(DBCSR_EINVAL, "sign_iterate: P_out block sizes differ from H");
    dbcsr_sign_opts o{};
    o.eps_filter = 0.0;
    o.tol = 1e-9;
    o.max_iter = 100;
    o.prec = DBCSR_FP64;
    o.stall_ratio = 0.5;
    if (opts) o = *opts;
    if (o.max_iter <= 0) o.max_iter = 100;
    if (o.stall_ratio <= 0) o.stall_ratio = 0.5;
    if (!(o.eps_filter >= 0) || !(o.tol > 0)) fail(DBCSR_EINVAL, "sign_iterate: need eps_filter >= 0 and tol > 0");
    if (o.prec != DBCSR_FP64 && o.prec != DBCSR_MIXED) fail(DBCSR_EINVAL, "sign_iterate: prec must be FP64 or MIXED");
    if (o.prec == DBCSR_MIXED && !(o.switch_tol > 0)) o.switch_tol = 1e-4;
    // Every product of the iteration is symmetric in exact arithmetic.  FP64 and split-BF16
    // products compute the blocks I <= J and mirror the rest.  Plain BF16 products keep both
    // triangles as computed: a BF16 X2 commutes with X only to about 1e-3, so mirrored BF16
    // products would steer X towards a different matrix; a mixed run with a plain BF16 tier
    // therefore forms full products throughout and takes X's symmetric part at the end.
    const bool full = (o.flags & DBCSR_SIGN_FULL_PRODUCTS) != 0;
    const int low = (o.flags & DBCSR_SIGN_PLAIN_BF16) ? DBCSR_BF16 : DBCSR_BF16X3;
    const bool full_mixed = o.prec == DBCSR_MIXED && low == DBCSR_BF16;
    const bool correction = o.prec == DBCSR_MIXED && (o.flags & DBCSR_SIGN_LOW_CORRECTION) != 0;

    const auto t0 = std::chrono::steady_clock::now();
    cudaStream_t s = H->stream;
    const double N = (double)H->n;
    const double alpha = gershgorin(H, mu);
    if (!(alpha > 0) || !std::isfinite(alpha)) fail(DBCSR_EINVAL, "sign_iterate: Gershgorin bound is zero or not finite");

    auto X = make_like(H, s);
    auto X2 = make_like(H, s);
    copy_matrix(X.get(), H);
    scale_shift(X.get(), 1.0 / alpha, -mu / alpha);

    dbcsr_sign_report r{};
    r.alpha = alpha;
    int it = 0;
    bool converged = false, stalled = false;
    double res = 0.0;
    // precision ladder: BF16 operands / FP32 accumulation while r >= switch_tol, then FP64
    int tier = (o.prec == DBCSR_MIXED) ? low : DBCSR_FP64;
    int first_fp64 = (tier == DBCSR_FP64) ? 1 : 0;
    const int sym = (full || full_mixed) ? kSymNone : kSymMirror;
    auto account = [&](const dbcsr_mult_stats& st, int tier_of_product) {
        r.flops += st.flops;
        r.n_products += st.n_products;
        r.ms_multiply += st.ms_numeric;
        r.ms_symbolic += st.ms_symbolic;
        r.ms_filter += st.ms_filter;
        if (tier_of_product != DBCSR_FP64) {
            r.ms_low += st.ms_numeric;
            r.flops_low += st.flops;
        } else {
            r.bytes_min_fp64 += st.bytes_min;
            r.launches_fp64 += st.n_launches;
        }
    };
    while (it < o.max_iter) {
        dbcsr_mult_stats st{};
        multiply(1.0, X.get(), X.get(), 0.0, X2.get(), o.eps_filter, tier, &st, true, sym);
        res = std::sqrt(st.dev2_filtered) / N;
        account(st, tier);
        if (it < DBCSR_MAX_HISTORY) r.residual_history[it] = res;
        ++it;
        if (!std::isfinite(res)) fail(DBCSR_ENAN, "sign_iterate: residual is not finite");
        if (o.verbose)
            std::fprintf(stderr, "[sign] it %3d %s r %.3e nnzb(X) %lld cand %lld formed %lld kept %lld %.1f GF %.2f ms\n",
                         it, tier == DBCSR_FP64 ? "fp64" : tier == DBCSR_BF16 ? "bf16" : "bf16x3", res, (long long)X->nnzb,
                         (long long)st.n_candidates, (long long)st.n_formed, (long long)st.n_kept, st.flops * 1e-9,
                         st.ms_numeric);
        // without filtering r_k / r_{k-1} only falls: a fast step followed by a slow one is a stall
        const bool slow = it >= 3 && it - 1 < DBCSR_MAX_HISTORY &&
                          r.residual_history[it - 2] < o.stall_ratio * r.residual_history[it - 3] &&
                          res > o.stall_ratio * r.residual_history[it - 2];
        if (tier != DBCSR_FP64) {
            // the low-precision tier ends at the switch residual (or when it stops making progress);
            // convergence is only ever declared on an FP64 product
            if (res < o.switch_tol || res < o.tol || slow) {
                tier = DBCSR_FP64;
                first_fp64 = it + 1;
            }
        } else {
            if (res < o.tol) {
                converged = true;
                if (it - 1 < DBCSR_MAX_HISTORY) r.nnzb_history[it - 1] = X->nnzb;
                break;
            }
            if (slow && it >= first_fp64 + 2) {
                stalled = true;
                if (it - 1 < DBCSR_MAX_HISTORY) r.nnzb_history[it - 1] = X->nnzb;
                break;
            }
        }
        if (correction && tier == DBCSR_FP64) {
            // X <- X - 0.5 X (X2 - 1): the small correction in split BF16, X itself in FP64
            scale_shift(X2.get(), 1.0, -1.0);
            multiply(-0.5, X.get(), X2.get(), 1.0, X.get(), o.eps_filter, DBCSR_BF16X3, &st, false, sym);
            account(st, DBCSR_BF16X3);
        } else {
            multiply(-0.5, X.get(), X2.get(), 1.5, X.get(), o.eps_filter, tier, &st, false, sym);
            account(st, tier);
        }
        if (it - 1 < DBCSR_MAX_HISTORY) r.nnzb_history[it - 1] = X->nnzb;
    }
    // X of a mixed run is symmetric only to the low tier's accuracy (both triangles formed with
    // plain BF16; diagonal blocks summed in FP32 with split BF16), so it is replaced by its
    // symmetric part before P is formed
    if (o.prec == DBCSR_MIXED && !full) symmetrize(X.get());
    copy_matrix(P, X.get());
    scale_shift(P, -0.5, 0.5);
    r.trace_p = trace(P);
    r.e_band = trace_product(P, H);
    DBG_CK(cudaStreamSynchronize(s));
    DBG_CK(cudaStreamSynchronize(P->stream));
    r.iterations = it;
    r.fp64_from = first_fp64;
    r.converged = converged ? 1 : 0;
    r.stalled = stalled ? 1 : 0;
    r.residual = res;
    r.nnzb_x = X->nnzb;
    r.ms_total = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    if (rep) *rep = r;
    return converged ? DBCSR_OK : DBCSR_ENOTCONV;
}

}  // namespace dbg
