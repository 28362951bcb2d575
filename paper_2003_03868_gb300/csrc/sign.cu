// Density matrix by the sign iteration (section "Sign-Method": sign(A) = A (A^2)^(-1/2),
// P = (1 - sign(H - mu 1)) / 2 with S = 1, eps_filter truncation after every product).
//
//   X_0 = (H - mu 1) / alpha,  alpha = Gershgorin bound of H - mu 1
//   repeat:  Y = filter(X X);  r = ||Y - 1||_F / N;  stop when r < tol
//            X = filter(X p_n(Y))
//   P = (1 - X) / 2,  Tr(P),  E_band = Tr(P H)
//
// p_n(y) = sum_{j<=n} c_j (1 - y)^j, c_j = binom(2j, j) / 4^j, is the series of
// (1 - z)^(-1/2) at z = 1 - y cut after j = n, so X p_n(X^2) -> X (X^2)^(-1/2) with
// order n + 1 (the polynomial Pade iterations).  n = 1 is the second-order
// Newton-Schulz step X (3 - X^2) / 2 (the refinement function f_1 of section "OT/IR"),
// n = 2, 3 the functions f_2, f_3, and n = 4 the printed fifth-order step
// X (35 X^8 - 180 X^6 + 378 X^4 - 420 X^2 + 315) / 128, which the paper evaluates with
// four products per iteration.  Here every order n >= 2 sums p_n in powers of
// Z = 1 - Y, over the pairs q_i = c_2i + c_2i+1 Z, with Z2 = Z^2 and a filter after
// every product:
//   Z = 1 - Y;  Z2 = filter(Z Z);
//   R = top pair (plus c_n Z2 when n is even);  R <- filter(Z2 R + q_i) down to i = 1;
//   U = q_0 + filter(Z2 R)  (for n = 2: U = q_0 + c_2 Z2);  X <- filter(X U),
// that is 3, 4, 4, 5, 5 products per iteration for orders 3 to 7.  The c_j are positive
// and at most 1 (no cancelling sums of large terms, as in powers of Y), and every
// filtered product holds a Z2 factor or X: near convergence U - 1 ~ c_1 Z is a matrix of
// residual-sized blocks, and filtering it on its own would drop corrections just above
// eps for good (the iteration then stalls well above the Newton-Schulz floor).
#include <chrono>
#include <cmath>
#include <cstdio>
#include <functional>
#include <memory>
#include <vector>

#include "common.cuh"

namespace dbg {

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

std::vector<double> sign_series_coeffs(int n) {
    std::vector<double> c(n + 1);
    c[0] = 1.0;
    // binom(2j, j) / 4^j = c_j-1 (2j - 1) / (2j); every c_j is a short dyadic fraction, exact
    for (int j = 1; j <= n; ++j) c[j] = c[j - 1] * (2 * j - 1) / (2 * j);
    return c;
}

std::unique_ptr<dbcsr_matrix_> step_polynomial(dbcsr_matrix_* Y, int order, double eps, int tier, int sym,
                                               const std::function<void(const dbcsr_mult_stats&, int)>& account) {
    const int n = order - 1;
    const std::vector<double> c = sign_series_coeffs(n);
    cudaStream_t s = Y->stream;
    dbcsr_mult_stats st{};
    if (n == 1) {
        auto U = make_like(Y, s);
        copy_matrix(U.get(), Y);
        scale_shift(U.get(), -c[1], c[0] + c[1]);         // 1 + (1 - Y) / 2
        return U;
    }
    scale_shift(Y, -1.0, 1.0);                            // Z = 1 - Y, in place
    dbcsr_matrix_* Z = Y;
    auto Z2 = make_like(Y, s);
    multiply(1.0, Z, Z, 0.0, Z2.get(), eps, tier, &st, false, sym);
    account(st, tier);
    // pair i of p_n: c_2i+1 Z + c_2i 1
    auto pair = [&](dbcsr_matrix_* dst, int i) {
        copy_matrix(dst, Z);
        scale_shift(dst, c[2 * i + 1], c[2 * i]);
    };
    const int m = n / 2;
    auto R = make_like(Y, s);
    int i;
    if (n % 2 == 0) {
        pair(R.get(), m - 1);
        add(R.get(), 1.0, Z2.get(), c[n]);               // c_n Z2 + c_n-1 Z + c_n-2
        i = m - 2;
    } else {
        pair(R.get(), m);                                // c_n Z + c_n-1
        i = m - 1;
    }
    if (n == 2) return R;                                // q_0 + c_2 Z2
    for (; i >= 1; --i) {
        auto V = make_like(Y, s);
        pair(V.get(), i);
        multiply(1.0, Z2.get(), R.get(), 1.0, V.get(), eps, tier, &st, false, sym);
        account(st, tier);
        R = std::move(V);
    }
    auto V = make_like(Y, s);
    multiply(1.0, Z2.get(), R.get(), 0.0, V.get(), eps, tier, &st, false, sym);
    account(st, tier);
    R.reset();
    Z2.reset();
    auto U = make_like(Y, s);
    pair(U.get(), 0);
    add(U.get(), 1.0, V.get(), 1.0);                     // q_0 + filter(Z2 R)
    return U;
}

void sign_update(dbcsr_matrix_* X, dbcsr_matrix_* Y, int order, bool correction, double eps, int tier, int sym,
                 const std::function<void(const dbcsr_mult_stats&, int)>& account) {
    dbcsr_mult_stats st{};
    if (order == 2) {
        if (correction && tier == DBCSR_FP64) {
            // X <- X - 0.5 X (Y - 1): the small correction in split BF16, X itself in FP64
            scale_shift(Y, 1.0, -1.0);
            multiply(-0.5, X, Y, 1.0, X, eps, DBCSR_BF16X3, &st, false, sym);
            account(st, DBCSR_BF16X3);
        } else {
            multiply(-0.5, X, Y, 1.5, X, eps, tier, &st, false, sym);    // X (3 - Y) / 2
            account(st, tier);
        }
        return;
    }
    auto U = step_polynomial(Y, order, eps, tier, sym, account);
    multiply(1.0, X, U.get(), 0.0, X, eps, tier, &st, false, sym);
    account(st, tier);
}

namespace {

// Options with their defaults filled in and checked, and what they imply.
struct SignSetup {
    dbcsr_sign_opts o{};
    bool full = false, full_mixed = false, correction = false, return_x = false;
    int low = DBCSR_BF16X3;
};

SignSetup sign_setup(const dbcsr_sign_opts* opts) {
    SignSetup S;
    dbcsr_sign_opts& o = S.o;
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
    if (o.order == 0) o.order = 2;
    if (o.order < 2 || o.order > 7) fail(DBCSR_EINVAL, "sign_iterate: order must be 2 to 7");
    if (o.order != 2 && (o.flags & DBCSR_SIGN_LOW_CORRECTION))
        fail(DBCSR_EINVAL, "sign_iterate: the low-precision correction applies to order 2 only");
    // Every product of the iteration is symmetric in exact arithmetic.  FP64 and split-BF16
    // products compute the blocks I <= J and mirror the rest.  Plain BF16 products keep both
    // triangles as computed: a BF16 X2 commutes with X only to about 1e-3, so mirrored BF16
    // products would steer X towards a different matrix; a mixed run with a plain BF16 tier
    // therefore forms full products throughout and takes X's symmetric part at the end.
    S.full = (o.flags & DBCSR_SIGN_FULL_PRODUCTS) != 0;
    S.low = (o.flags & DBCSR_SIGN_PLAIN_BF16) ? DBCSR_BF16 : DBCSR_BF16X3;
    S.full_mixed = o.prec == DBCSR_MIXED && S.low == DBCSR_BF16;
    S.correction = o.prec == DBCSR_MIXED && (o.flags & DBCSR_SIGN_LOW_CORRECTION) != 0;
    S.return_x = (o.flags & DBCSR_SIGN_RETURN_X) != 0;
    return S;
}

// The iteration from the scaled X after `it` steps, the next X*X in `tier`, the switch to
// FP64 at step first_fp64 (0: not yet), with r holding the report so far (histories of the
// steps taken); fills P (or X itself with DBCSR_SIGN_RETURN_X) and the report.
dbcsr_status sign_run(dbcsr_matrix_* H, std::unique_ptr<dbcsr_matrix_> X, const SignSetup& S, int it, int tier,
                      int first_fp64, dbcsr_sign_report r, dbcsr_matrix_* P, dbcsr_sign_report* rep,
                      std::chrono::steady_clock::time_point t0) {
    const dbcsr_sign_opts& o = S.o;
    cudaStream_t s = H->stream;
    const double N = (double)H->n;
    auto X2 = make_like(H, s);
    bool converged = false, stalled = false;
    double res = it > 0 && it - 1 < DBCSR_MAX_HISTORY ? r.residual_history[it - 1] : 0.0;
    const int sym = (S.full || S.full_mixed) ? kSymNone : kSymMirror;
    auto account = [&](const dbcsr_mult_stats& st, int tier_of_product) {
        r.flops += st.flops;
        r.n_products += st.n_products;
        r.ms_multiply += st.ms_numeric;
        r.ms_symbolic += st.ms_symbolic;
        r.ms_filter += st.ms_filter;
        if (tier_of_product != DBCSR_FP64) {
            r.ms_low += st.ms_numeric;
            r.flops_low += st.flops;
            r.flops_tensor += st.flops_tensor;
            r.bytes_tensor += st.bytes_tensor;
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
        sign_update(X.get(), X2.get(), o.order, S.correction, o.eps_filter, tier, sym, account);
        if (it - 1 < DBCSR_MAX_HISTORY) r.nnzb_history[it - 1] = X->nnzb;
    }
    if (S.return_x) {
        // the iteration's state for a later dbcsr_sign_iterate_resume: X as it stands
        copy_matrix(P, X.get());
        r.trace_p = std::nan("");
        r.e_band = std::nan("");
    } else {
        // X of a mixed run with a plain BF16 tier (both triangles formed) is symmetric only to
        // that tier's accuracy, so it is replaced by its symmetric part before P is formed;
        // mirrored products keep X exactly symmetric
        if (S.full_mixed && !S.full) symmetrize(X.get());
        copy_matrix(P, X.get());
        scale_shift(P, -0.5, 0.5);
        r.trace_p = trace(P);
        r.e_band = trace_product(P, H);
    }
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

}  // namespace

dbcsr_status sign_iterate(dbcsr_matrix_* H, double mu, const dbcsr_sign_opts* opts, dbcsr_matrix_* P,
                          dbcsr_sign_report* rep) {
    check_finalized(H);
    if (!P) fail(DBCSR_EINVAL, "sign_iterate: null P_out");
    if (P->h_bs != H->h_bs) fail(DBCSR_EINVAL, "sign_iterate: P_out block sizes differ from H");
    const SignSetup S = sign_setup(opts);
    const auto t0 = std::chrono::steady_clock::now();
    const double alpha = gershgorin(H, mu);
    if (!(alpha > 0) || !std::isfinite(alpha)) fail(DBCSR_EINVAL, "sign_iterate: Gershgorin bound is zero or not finite");
    auto X = make_like(H, H->stream);
    copy_matrix(X.get(), H);
    scale_shift(X.get(), 1.0 / alpha, -mu / alpha);
    dbcsr_sign_report r{};
    r.alpha = alpha;
    // precision ladder: BF16 operands / FP32 accumulation while r >= switch_tol, then FP64
    const int tier = (S.o.prec == DBCSR_MIXED) ? S.low : DBCSR_FP64;
    return sign_run(H, std::move(X), S, 0, tier, tier == DBCSR_FP64 ? 1 : 0, r, P, rep, t0);
}

dbcsr_status sign_iterate_resume(dbcsr_matrix_* H, dbcsr_matrix_* X0, const dbcsr_sign_report* prev,
                                 const dbcsr_sign_opts* opts, dbcsr_matrix_* P, dbcsr_sign_report* rep) {
    check_finalized(H);
    check_finalized(X0);
    if (!P || !prev) fail(DBCSR_EINVAL, "sign_iterate_resume: null P_out or report");
    if (P->h_bs != H->h_bs || X0->h_bs != H->h_bs)
        fail(DBCSR_EINVAL, "sign_iterate_resume: block sizes of X or P_out differ from H");
    if (prev->iterations < 0 || prev->iterations > DBCSR_MAX_HISTORY || prev->fp64_from < 0)
        fail(DBCSR_EINVAL, "sign_iterate_resume: the report is not one of a sign iteration");
    const SignSetup S = sign_setup(opts);
    const auto t0 = std::chrono::steady_clock::now();
    auto X = make_like(H, H->stream);
    copy_matrix(X.get(), X0);
    const int it = prev->iterations;
    int first_fp64 = prev->fp64_from;
    if (S.o.prec == DBCSR_FP64) first_fp64 = std::max(1, first_fp64 ? first_fp64 : 1);
    // the step after `it` multiplies in FP64 once the switch has come (at or before it)
    const bool fp64_now = S.o.prec == DBCSR_FP64 || (first_fp64 > 0 && first_fp64 <= it + 1);
    dbcsr_sign_report r = *prev;
    r.ms_total = 0.0;
    return sign_run(H, std::move(X), S, it, fp64_now ? DBCSR_FP64 : S.low, fp64_now ? first_fp64 : 0, r, P, rep,
                    t0);
}

}  // namespace dbg
