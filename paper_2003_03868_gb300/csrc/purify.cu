// Canonical density matrices without a known chemical potential (section "Purification
// methods": TRS4, TC2 and the sign method in CP2K; purifications are grand-canonical by
// construction, so the canonical case needs modified steps or extra iterations to place
// mu).  The steps restate the published algorithms (TC2: Niklasson 2002; TRS4:
// Niklasson, Tymczak and Challacombe 2003):
//
//   X_0 = (g 1 - H) / (2 g), g the Gershgorin bound (spectrum in [0, 1], low states near 1)
//   repeat: e = (Tr X - Tr X^2) / N; stop when |e| < tol
//     TC2:  X <- X^2 if Tr X > N_occ, else 2 X - X^2                        (one product)
//     TRS4: X2 = X^2; gamma = (N_occ - Tr F) / Tr G, F = X2 (4 X - 3 X2), G = X2 (1 - X)^2;
//           gamma in [0, 6]: X <- X2 (gamma + (4 - 2 gamma) X + (gamma - 3) X2)
//           gamma > 6: X <- 2 X - X2;  gamma < 0: X <- X2
//
// Tr X^2, Tr X^3 = Tr(X2 X) and Tr X^4 = Tr(X2 X2) come from the factors (no product
// formed).  Every product is filtered and, as all are polynomials in H, mirrored.
// sign_mu_search bisects mu for the sign method until Tr P(mu) is within 1/2 of N_occ.
#include <chrono>
#include <cmath>
#include <cstdio>
#include <memory>

#include "common.cuh"

namespace dbg {

dbcsr_status purify(dbcsr_matrix_* H, double n_occ, int32_t method, const dbcsr_sign_opts* opts, dbcsr_matrix_* P,
                    dbcsr_sign_report* rep) {
    check_finalized(H);
    if (!P) fail(DBCSR_EINVAL, "purify: null P_out");
    if (P->h_bs != H->h_bs) fail(DBCSR_EINVAL, "purify: P_out block sizes differ from H");
    if (P == H) fail(DBCSR_EINVAL, "purify: P_out must differ from H");
    if (method != DBCSR_PURIFY_TC2 && method != DBCSR_PURIFY_TRS4) fail(DBCSR_EINVAL, "purify: unknown method");
    check_unplanned(P, "purify");
    dbcsr_sign_opts o{};
    o.tol = 1e-9;
    o.max_iter = 100;
    o.prec = DBCSR_FP64;
    if (opts) o = *opts;
    if (o.max_iter <= 0) o.max_iter = 100;
    if (!(o.eps_filter >= 0) || !(o.tol > 0)) fail(DBCSR_EINVAL, "purify: need eps_filter >= 0 and tol > 0");
    if (o.prec != DBCSR_FP64) fail(DBCSR_EINVAL, "purify: prec must be FP64");
    const double N = (double)H->n;
    if (!(n_occ >= 0 && n_occ <= N)) fail(DBCSR_EINVAL, "purify: n_occ must lie in [0, N]");
    const int sym = (o.flags & DBCSR_SIGN_FULL_PRODUCTS) ? kSymNone : kSymMirror;

    const auto t0 = std::chrono::steady_clock::now();
    cudaStream_t s = H->stream;
    const double g = gershgorin(H, 0.0);
    if (!(g > 0) || !std::isfinite(g)) fail(DBCSR_EINVAL, "purify: Gershgorin bound is zero or not finite");
    auto X = make_like(H, s);
    copy_matrix(X.get(), H);
    scale_shift(X.get(), -1.0 / (2.0 * g), 0.5);

    dbcsr_sign_report r{};
    r.alpha = g;
    auto account = [&](const dbcsr_mult_stats& st) {
        r.flops += st.flops;
        r.n_products += st.n_products;
        r.ms_multiply += st.ms_numeric;
        r.ms_symbolic += st.ms_symbolic;
        r.ms_filter += st.ms_filter;
        r.bytes_min_fp64 += st.bytes_min;
        r.launches_fp64 += st.n_launches;
    };
    int it = 0, hist = 0;
    bool converged = false;
    double e = 0.0;
    while (true) {
        const double t1 = trace(X.get());
        const double t2 = trace_product(X.get(), X.get());
        e = (t1 - t2) / N;
        if (!std::isfinite(e)) fail(DBCSR_ENAN, "purify: trace is not finite");
        if (hist < DBCSR_MAX_HISTORY) r.residual_history[hist++] = e;
        if (std::fabs(e) < o.tol) {
            converged = true;
            break;
        }
        if (it >= o.max_iter) break;
        ++it;
        dbcsr_mult_stats st{};
        const char* kind;
        if (method == DBCSR_PURIFY_TC2) {
            if (t1 > n_occ) {
                multiply(1.0, X.get(), X.get(), 0.0, X.get(), o.eps_filter, DBCSR_FP64, &st, false, sym);
                kind = "X^2";
            } else {
                multiply(-1.0, X.get(), X.get(), 2.0, X.get(), o.eps_filter, DBCSR_FP64, &st, false, sym);
                kind = "2X-X^2";
            }
            account(st);
        } else {
            auto X2 = make_like(H, s);
            multiply(1.0, X.get(), X.get(), 0.0, X2.get(), o.eps_filter, DBCSR_FP64, &st, false, sym);
            account(st);
            const double s2 = trace(X2.get());
            const double s3 = trace_product(X2.get(), X.get());
            const double s4 = trace_product(X2.get(), X2.get());
            const double tr_f = 4.0 * s3 - 3.0 * s4, tr_g = s2 - 2.0 * s3 + s4;
            const double gamma = tr_g != 0.0 ? (n_occ - tr_f) / tr_g : (n_occ > tr_f ? 7.0 : -1.0);
            if (gamma > 6.0) {
                add(X.get(), 2.0, X2.get(), -1.0);          // 2 X - X2
                kind = "2X-X^2";
            } else if (gamma < 0.0) {
                X = std::move(X2);
                kind = "X^2";
            } else {
                auto Q = make_like(H, s);
                copy_matrix(Q.get(), X.get());
                add(Q.get(), 4.0 - 2.0 * gamma, X2.get(), gamma - 3.0);
                scale_shift(Q.get(), 1.0, gamma);            // gamma + (4 - 2 gamma) X + (gamma - 3) X2
                multiply(1.0, X2.get(), Q.get(), 0.0, X.get(), o.eps_filter, DBCSR_FP64, &st, false, sym);
                account(st);
                kind = "F+gG";
            }
        }
        if (it - 1 < DBCSR_MAX_HISTORY) r.nnzb_history[it - 1] = X->nnzb;
        if (o.verbose)
            std::fprintf(stderr, "[purify] it %3d %s e %.3e tr %.6f nnzb %lld\n", it, kind, e, t1, (long long)X->nnzb);
    }
    copy_matrix(P, X.get());
    r.trace_p = trace(P);
    r.e_band = trace_product(P, H);
    DBG_CK(cudaStreamSynchronize(s));
    DBG_CK(cudaStreamSynchronize(P->stream));
    r.iterations = it;
    r.fp64_from = 1;
    r.converged = converged ? 1 : 0;
    r.residual = e;
    r.nnzb_x = X->nnzb;
    r.ms_total = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    if (rep) *rep = r;
    return converged ? DBCSR_OK : DBCSR_ENOTCONV;
}

dbcsr_status sign_mu_search(dbcsr_matrix_* H, double n_occ, double mu_lo, double mu_hi, const dbcsr_sign_opts* opts,
                            dbcsr_matrix_* P, double* mu_out, int32_t* evaluations, dbcsr_sign_report* rep) {
    check_finalized(H);
    if (!P) fail(DBCSR_EINVAL, "sign_mu_search: null P_out");
    const double N = (double)H->n;
    if (!(n_occ >= 0 && n_occ <= N)) fail(DBCSR_EINVAL, "sign_mu_search: n_occ must lie in [0, N]");
    const auto t0 = std::chrono::steady_clock::now();
    const double g = gershgorin(H, 0.0);
    double lo = std::isnan(mu_lo) ? -g : mu_lo, hi = std::isnan(mu_hi) ? g : mu_hi;
    if (!(lo < hi)) fail(DBCSR_EINVAL, "sign_mu_search: need mu_lo < mu_hi");
    dbcsr_sign_report r{}, acc{};
    dbcsr_status st = DBCSR_ENOTCONV;
    double mu = 0.5 * (lo + hi);
    int k = 0;
    bool found = false;
    for (; k < 60 && !found; ++k) {
        mu = 0.5 * (lo + hi);
        st = sign_iterate(H, mu, opts, P, &r);
        acc.flops += r.flops;
        acc.n_products += r.n_products;
        acc.ms_multiply += r.ms_multiply;
        acc.ms_symbolic += r.ms_symbolic;
        acc.ms_filter += r.ms_filter;
        acc.ms_low += r.ms_low;
        acc.flops_low += r.flops_low;
        acc.bytes_min_fp64 += r.bytes_min_fp64;
        acc.launches_fp64 += r.launches_fp64;
        if (opts && opts->verbose)
            std::fprintf(stderr, "[mu] eval %d mu %.6f Tr P %.6f\n", k + 1, mu, r.trace_p);
        if (std::fabs(r.trace_p - n_occ) < 0.5) found = true;
        else if (r.trace_p > n_occ) hi = mu;
        else lo = mu;
    }
    // the report of the last sign iteration, with the work of every trial
    r.flops = acc.flops;
    r.n_products = acc.n_products;
    r.ms_multiply = acc.ms_multiply;
    r.ms_symbolic = acc.ms_symbolic;
    r.ms_filter = acc.ms_filter;
    r.ms_low = acc.ms_low;
    r.flops_low = acc.flops_low;
    r.bytes_min_fp64 = acc.bytes_min_fp64;
    r.launches_fp64 = acc.launches_fp64;
    r.ms_total = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    if (mu_out) *mu_out = mu;
    if (evaluations) *evaluations = k;
    if (rep) *rep = r;
    return (found && st == DBCSR_OK) ? DBCSR_OK : DBCSR_ENOTCONV;
}

}  // namespace dbg
