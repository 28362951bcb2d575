// Non-orthogonal basis (section "Sign-Method"):
//
//   * S^(-1/2) and S^(1/2) from the sign of the block matrix [[0, A], [1, 0]], which is
//     [[0, A^(1/2)], [A^(-1/2), 0]].  The sign iteration keeps the iterate in the form
//     [[0, Y], [Z, 0]], whose square is diag(Y Z, Z Y); Y and Z are functions of A, so
//     Y Z = Z Y and the step X <- X p(X^2) of any order reads
//         W = filter(Z Y);  r = ||W - 1||_F / N;  stop when r < tol;
//         U = p(W);  Y <- filter(Y U);  Z <- filter(U Z),
//     from Y_0 = A = S / g, Z_0 = 1, g the Gershgorin bound of S (spectrum of A in (0, 1]).
//     S^(1/2) = sqrt(g) Y, S^(-1/2) = Z / sqrt(g).
//     Y = A Z holds at every step in exact arithmetic, and the iteration keeps whatever A
//     its iterates imply: unlike the sign, whose value does not move under perturbations
//     smaller than the gap, A^(-1/2) follows every change of A.  So with the precision
//     ladder the low tier's errors would stay in the result (Tr(P S) off by about 1e-3 on
//     1,024 waters); at the switch to FP64, Y <- filter(A Z) restores the relation and the
//     FP64 steps converge to the root of the true A.
//   * A^-1 of a positive definite A by Hotelling's iteration (section "Preconditioners"):
//     X_0 = 1 / g, repeat T = filter(A X), stop when ||T - 1||_F / N < tol,
//     X <- filter(2 X - X T); the residual 1 - A X squares at every step.
//   * P = (1 - sign(S^-1 K - mu 1)) S^-1 / 2, evaluated through the similarity
//     sign(S^-1 K - mu 1) = S^(-1/2) sign(K' - mu 1) S^(1/2), K' = S^(-1/2) K S^(-1/2):
//     P = S^(-1/2) P' S^(-1/2) with P' the density matrix of K'.  Every product is filtered.
#include <chrono>
#include <cmath>
#include <cstdio>
#include <functional>
#include <memory>

#include "common.cuh"

namespace dbg {
namespace {

// Block row I of the identity: one block (I, I) of area bs[I]^2.
__global__ void k_eye_meta(int32_t nblk, const int32_t* __restrict__ bs, int64_t* __restrict__ rp,
                           int32_t* __restrict__ col, int32_t* __restrict__ row, int64_t* __restrict__ area) {
    for (int32_t I = blockIdx.x * blockDim.x + threadIdx.x; I <= nblk; I += gridDim.x * blockDim.x) {
        rp[I] = I;
        if (I < nblk) {
            col[I] = I;
            row[I] = I;
            area[I] = (int64_t)bs[I] * bs[I];
        }
    }
}

// One warp per diagonal block: the identity block.
__global__ void k_eye_data(int32_t nblk, const int32_t* __restrict__ bs, const int64_t* __restrict__ off,
                           double* __restrict__ data) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t I = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); I < nblk; I += warps) {
        const int m = bs[I];
        double* d = data + off[I];
        for (int e = lane; e < m * m; e += 32) d[e] = (e / m == e % m) ? 1.0 : 0.0;
    }
}

// The identity with m's block sizes, on m's stream.
std::unique_ptr<dbcsr_matrix_> make_identity(const dbcsr_matrix_* m) {
    cudaStream_t s = m->stream;
    auto x = make_like(m, s);
    const int32_t nb = m->nblk;
    x->rp.alloc(nb + 1, s);
    x->col.alloc(std::max<int32_t>(nb, 1), s);
    x->row.alloc(std::max<int32_t>(nb, 1), s);
    x->off.alloc(nb + 1, s);
    DBuf<int64_t> area;
    area.alloc(std::max<int32_t>(nb, 1), s);
    k_eye_meta<<<grid_for(nb + 1, 256), 256, 0, s>>>(nb, x->bs.p, x->rp.p, x->col.p, x->row.p, area.p);
    DBG_LAUNCH_CK();
    scan_exclusive(area.p, x->off.p, nb, s);
    x->nel = read_i64(x->off.p + nb, s);
    x->data.alloc(std::max<int64_t>(x->nel, 1), s);
    if (nb) {
        k_eye_data<<<grid_for(nb, 8), 256, 0, s>>>(nb, x->bs.p, x->off.p, x->data.p);
        DBG_LAUNCH_CK();
    }
    x->nnzb = nb;
    x->norms_valid = false;
    x->finalized = true;
    return x;
}

dbcsr_sign_opts checked_opts(const dbcsr_sign_opts* opts, const char* where) {
    dbcsr_sign_opts o{};
    o.tol = 1e-9;
    o.max_iter = 100;
    o.prec = DBCSR_FP64;
    o.stall_ratio = 0.5;
    if (opts) o = *opts;
    if (o.max_iter <= 0) o.max_iter = 100;
    if (o.stall_ratio <= 0) o.stall_ratio = 0.5;
    const std::string w(where);
    if (!(o.eps_filter >= 0) || !(o.tol > 0)) fail(DBCSR_EINVAL, w + ": need eps_filter >= 0 and tol > 0");
    if (o.prec != DBCSR_FP64 && o.prec != DBCSR_MIXED) fail(DBCSR_EINVAL, w + ": prec must be FP64 or MIXED");
    if (o.prec == DBCSR_MIXED && !(o.switch_tol > 0)) o.switch_tol = 1e-4;
    if (o.order == 0) o.order = 2;
    if (o.order < 2 || o.order > 7) fail(DBCSR_EINVAL, w + ": order must be 2 to 7");
    return o;
}

}  // namespace

dbcsr_status inverse_sqrt(dbcsr_matrix_* S, const dbcsr_sign_opts* opts, dbcsr_matrix_* Sinv, dbcsr_matrix_* Ssqrt,
                          dbcsr_sign_report* rep) {
    check_finalized(S);
    if (!Sinv) fail(DBCSR_EINVAL, "inverse_sqrt: null S_invsqrt");
    if (Sinv->h_bs != S->h_bs || (Ssqrt && Ssqrt->h_bs != S->h_bs))
        fail(DBCSR_EINVAL, "inverse_sqrt: output block sizes differ from S");
    if (Sinv == S || Ssqrt == S || (Ssqrt && Ssqrt == Sinv)) fail(DBCSR_EINVAL, "inverse_sqrt: outputs must be distinct from S");
    const dbcsr_sign_opts o = checked_opts(opts, "inverse_sqrt");
    if (o.flags & DBCSR_SIGN_LOW_CORRECTION) fail(DBCSR_EINVAL, "inverse_sqrt: no low-precision correction form");
    check_unplanned(Sinv, "inverse_sqrt");
    if (Ssqrt) check_unplanned(Ssqrt, "inverse_sqrt");
    const bool full = (o.flags & DBCSR_SIGN_FULL_PRODUCTS) != 0;
    const int low = (o.flags & DBCSR_SIGN_PLAIN_BF16) ? DBCSR_BF16 : DBCSR_BF16X3;
    const bool full_mixed = o.prec == DBCSR_MIXED && low == DBCSR_BF16;

    const auto t0 = std::chrono::steady_clock::now();
    cudaStream_t s = S->stream;
    const double N = (double)S->n;
    const double g = gershgorin(S, 0.0);
    if (!(g > 0) || !std::isfinite(g)) fail(DBCSR_EINVAL, "inverse_sqrt: Gershgorin bound is zero or not finite");

    auto Y = make_like(S, s);
    copy_matrix(Y.get(), S);
    scale_shift(Y.get(), 1.0 / g, 0.0);
    std::unique_ptr<dbcsr_matrix_> A;                     // kept for the switch to FP64
    if (o.prec == DBCSR_MIXED) {
        A = make_like(S, s);
        copy_matrix(A.get(), Y.get());
    }
    auto Z = make_identity(S);
    auto W = make_like(S, s);

    dbcsr_sign_report r{};
    r.alpha = g;
    int it = 0;
    bool converged = false, stalled = false;
    double res = 0.0;
    int tier = (o.prec == DBCSR_MIXED) ? low : DBCSR_FP64;
    int first_fp64 = (tier == DBCSR_FP64) ? 1 : 0;
    // Y, Z, W and U are functions of S: every product is symmetric in exact arithmetic
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
        multiply(1.0, Z.get(), Y.get(), 0.0, W.get(), o.eps_filter, tier, &st, true, sym);
        res = std::sqrt(st.dev2_filtered) / N;
        account(st, tier);
        if (it < DBCSR_MAX_HISTORY) r.residual_history[it] = res;
        ++it;
        if (!std::isfinite(res)) fail(DBCSR_ENAN, "inverse_sqrt: residual is not finite");
        if (o.verbose)
            std::fprintf(stderr, "[sqrt] it %3d %s r %.3e nnzb(Z) %lld nnzb(Y) %lld %.1f GF %.2f ms\n", it,
                         tier == DBCSR_FP64 ? "fp64" : tier == DBCSR_BF16 ? "bf16" : "bf16x3", res, (long long)Z->nnzb,
                         (long long)Y->nnzb, st.flops * 1e-9, st.ms_numeric);
        const bool slow = it >= 3 && it - 1 < DBCSR_MAX_HISTORY &&
                          r.residual_history[it - 2] < o.stall_ratio * r.residual_history[it - 3] &&
                          res > o.stall_ratio * r.residual_history[it - 2];
        if (tier != DBCSR_FP64) {
            if (res < o.switch_tol || res < o.tol || slow) {
                tier = DBCSR_FP64;
                first_fp64 = it + 1;
                // re-anchor on the true A: Y = A Z, then the next step tests Z A Z in FP64
                multiply(1.0, A.get(), Z.get(), 0.0, Y.get(), o.eps_filter, DBCSR_FP64, &st, false, sym);
                account(st, DBCSR_FP64);
                if (it - 1 < DBCSR_MAX_HISTORY) r.nnzb_history[it - 1] = Z->nnzb;
                continue;
            }
        } else {
            if (res < o.tol) {
                converged = true;
                if (it - 1 < DBCSR_MAX_HISTORY) r.nnzb_history[it - 1] = Z->nnzb;
                break;
            }
            if (slow && it >= first_fp64 + 2) {
                stalled = true;
                if (it - 1 < DBCSR_MAX_HISTORY) r.nnzb_history[it - 1] = Z->nnzb;
                break;
            }
        }
        auto U = step_polynomial(W.get(), o.order, o.eps_filter, tier, sym, account);
        multiply(1.0, Y.get(), U.get(), 0.0, Y.get(), o.eps_filter, tier, &st, false, sym);
        account(st, tier);
        multiply(1.0, U.get(), Z.get(), 0.0, Z.get(), o.eps_filter, tier, &st, false, sym);
        account(st, tier);
        if (it - 1 < DBCSR_MAX_HISTORY) r.nnzb_history[it - 1] = Z->nnzb;
    }
    if (full_mixed && !full) {
        symmetrize(Z.get());
        symmetrize(Y.get());
    }
    const double rg = std::sqrt(g);
    copy_matrix(Sinv, Z.get());
    scale_shift(Sinv, 1.0 / rg, 0.0);
    if (Ssqrt) {
        copy_matrix(Ssqrt, Y.get());
        scale_shift(Ssqrt, rg, 0.0);
    }
    DBG_CK(cudaStreamSynchronize(s));
    DBG_CK(cudaStreamSynchronize(Sinv->stream));
    if (Ssqrt) DBG_CK(cudaStreamSynchronize(Ssqrt->stream));
    r.iterations = it;
    r.fp64_from = first_fp64;
    r.converged = converged ? 1 : 0;
    r.stalled = stalled ? 1 : 0;
    r.residual = res;
    r.nnzb_x = Z->nnzb;
    r.ms_total = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    if (rep) *rep = r;
    return converged ? DBCSR_OK : DBCSR_ENOTCONV;
}

dbcsr_status inverse_hotelling(dbcsr_matrix_* A, const dbcsr_sign_opts* opts, dbcsr_matrix_* Ainv,
                               dbcsr_sign_report* rep) {
    check_finalized(A);
    if (!Ainv) fail(DBCSR_EINVAL, "inverse_hotelling: null A_inv");
    if (Ainv->h_bs != A->h_bs) fail(DBCSR_EINVAL, "inverse_hotelling: A_inv block sizes differ from A");
    if (Ainv == A) fail(DBCSR_EINVAL, "inverse_hotelling: A_inv must differ from A");
    check_unplanned(Ainv, "inverse_hotelling");
    dbcsr_sign_opts o = checked_opts(opts, "inverse_hotelling");
    if (o.prec != DBCSR_FP64) fail(DBCSR_EINVAL, "inverse_hotelling: prec must be FP64");
    const int sym = (o.flags & DBCSR_SIGN_FULL_PRODUCTS) ? kSymNone : kSymMirror;   // X is a polynomial in A
    const auto t0 = std::chrono::steady_clock::now();
    cudaStream_t s = A->stream;
    const double N = (double)A->n;
    const double g = gershgorin(A, 0.0);
    if (!(g > 0) || !std::isfinite(g)) fail(DBCSR_EINVAL, "inverse_hotelling: Gershgorin bound is zero or not finite");
    auto X = make_identity(A);
    scale_shift(X.get(), 1.0 / g, 0.0);                       // X_0 = 1 / g
    auto T = make_like(A, s);
    dbcsr_sign_report r{};
    r.alpha = g;
    int it = 0;
    bool converged = false, stalled = false;
    double res = 0.0;
    while (it < o.max_iter) {
        dbcsr_mult_stats st{};
        multiply(1.0, A, X.get(), 0.0, T.get(), o.eps_filter, DBCSR_FP64, &st, true, sym);
        res = std::sqrt(st.dev2_filtered) / N;
        r.flops += st.flops;
        r.n_products += st.n_products;
        r.ms_multiply += st.ms_numeric;
        r.ms_symbolic += st.ms_symbolic;
        r.ms_filter += st.ms_filter;
        if (it < DBCSR_MAX_HISTORY) r.residual_history[it] = res;
        ++it;
        if (!std::isfinite(res)) fail(DBCSR_ENAN, "inverse_hotelling: residual is not finite");
        if (o.verbose)
            std::fprintf(stderr, "[inverse] it %3d r %.3e nnzb(X) %lld\n", it, res, (long long)X->nnzb);
        if (res < o.tol) {
            converged = true;
            break;
        }
        if (it >= 3 && it - 1 < DBCSR_MAX_HISTORY && r.residual_history[it - 2] < o.stall_ratio * r.residual_history[it - 3] &&
            res > o.stall_ratio * r.residual_history[it - 2]) {
            stalled = true;
            break;
        }
        multiply(-1.0, X.get(), T.get(), 2.0, X.get(), o.eps_filter, DBCSR_FP64, &st, false, sym);   // 2 X - X A X
        r.flops += st.flops;
        r.n_products += st.n_products;
        r.ms_multiply += st.ms_numeric;
        r.ms_symbolic += st.ms_symbolic;
        r.ms_filter += st.ms_filter;
        if (it - 1 < DBCSR_MAX_HISTORY) r.nnzb_history[it - 1] = X->nnzb;
    }
    copy_matrix(Ainv, X.get());
    DBG_CK(cudaStreamSynchronize(s));
    DBG_CK(cudaStreamSynchronize(Ainv->stream));
    r.iterations = it;
    r.fp64_from = 1;
    r.converged = converged ? 1 : 0;
    r.stalled = stalled ? 1 : 0;
    r.residual = res;
    r.nnzb_x = X->nnzb;
    r.ms_total = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    if (rep) *rep = r;
    return converged ? DBCSR_OK : DBCSR_ENOTCONV;
}

dbcsr_status sign_iterate_nonorth(dbcsr_matrix_* K, dbcsr_matrix_* S, double mu, const dbcsr_sign_opts* opts,
                                  dbcsr_matrix_* P, dbcsr_sign_report* rep, dbcsr_sign_report* rep_sqrt) {
    check_finalized(K);
    check_finalized(S);
    if (!P) fail(DBCSR_EINVAL, "sign_iterate_nonorth: null P_out");
    if (K->h_bs != S->h_bs || P->h_bs != K->h_bs) fail(DBCSR_EINVAL, "sign_iterate_nonorth: block sizes differ");
    if (P == K || P == S) fail(DBCSR_EINVAL, "sign_iterate_nonorth: P_out must differ from K and S");
    const dbcsr_sign_opts o = checked_opts(opts, "sign_iterate_nonorth");
    check_unplanned(P, "sign_iterate_nonorth");
    const auto t0 = std::chrono::steady_clock::now();
    cudaStream_t s = S->stream;
    if (K->stream != s) DBG_CK(cudaStreamSynchronize(K->stream));

    auto Zs = make_like(S, s);
    dbcsr_sign_report rs{};
    dbcsr_sign_opts os = o;
    os.flags &= ~DBCSR_SIGN_LOW_CORRECTION;
    const dbcsr_status st_sqrt = inverse_sqrt(S, &os, Zs.get(), nullptr, &rs);

    // the congruences in FP64; their results are symmetric in exact arithmetic
    const int sym = (o.flags & DBCSR_SIGN_FULL_PRODUCTS) ? kSymNone : kSymMirror;
    double t_flops = 0.0, t_ms = 0.0, t_sym = 0.0, t_filt = 0.0, t_bytes = 0.0;
    int64_t t_prod = 0, t_launch = 0;
    auto transform = [&](dbcsr_matrix_* A, dbcsr_matrix_* out) {
        auto T = make_like(S, s);
        dbcsr_mult_stats st{};
        multiply(1.0, Zs.get(), A, 0.0, T.get(), o.eps_filter, DBCSR_FP64, &st, false, kSymNone);
        t_flops += st.flops; t_ms += st.ms_numeric; t_sym += st.ms_symbolic; t_filt += st.ms_filter;
        t_bytes += st.bytes_min; t_prod += st.n_products; t_launch += st.n_launches;
        multiply(1.0, T.get(), Zs.get(), 0.0, out, o.eps_filter, DBCSR_FP64, &st, false, sym);
        t_flops += st.flops; t_ms += st.ms_numeric; t_sym += st.ms_symbolic; t_filt += st.ms_filter;
        t_bytes += st.bytes_min; t_prod += st.n_products; t_launch += st.n_launches;
    };
    auto Kp = make_like(S, s);
    transform(K, Kp.get());
    auto Pp = make_like(S, s);
    dbcsr_sign_report r{};
    const dbcsr_status st_sign = sign_iterate(Kp.get(), mu, &o, Pp.get(), &r);
    Kp.reset();
    transform(Pp.get(), P);
    r.trace_p = trace_product(P, S);                  // Tr(P S): the occupied count
    r.e_band = trace_product(P, K);                   // Tr(P K)
    DBG_CK(cudaStreamSynchronize(s));
    r.flops += t_flops;
    r.n_products += t_prod;
    r.ms_multiply += t_ms;
    r.ms_symbolic += t_sym;
    r.ms_filter += t_filt;
    r.bytes_min_fp64 += t_bytes;
    r.launches_fp64 += t_launch;
    r.ms_total = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    if (rep) *rep = r;
    if (rep_sqrt) *rep_sqrt = rs;
    return (st_sqrt == DBCSR_OK && st_sign == DBCSR_OK) ? DBCSR_OK : DBCSR_ENOTCONV;
}

}  // namespace dbg
