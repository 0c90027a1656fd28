// Solves of K x = b for blocks of right-hand sides (Sec. IV: even-odd
// preconditioned BiCGStab; this build adds FP64 defect correction around a
// lower-precision inner solve and runs all RHS of a block in one launch).
//
// Even-odd reduction: with K = [[A_ee, D_eo], [D_oe, A_oo]] (A = mass + clover),
//   M = 1 - A_ee^{-1} D_eo A_oo^{-1} D_oe,   bhat = A_ee^{-1} (b_e - D_eo A_oo^{-1} b_o),
//   M x_e = bhat,   x_o = A_oo^{-1} (b_o - D_oe x_e).
// Convergence is always judged on the FP64 true residual ||b - K x|| / ||b|| of
// the full operator.
#include <algorithm>
#include <cmath>
#include <type_traits>
#include <vector>

#include "blas.cuh"
#include "dirac.cuh"
#include "solver.cuh"

extern "C" int laph_precond_size(void);

namespace laph {

// Host-side summary of one inner solve.
struct InnerStats {
    std::vector<int> iters, status;
};

template <typename T>
static void schur_apply(const DiracOp &op, int nr, const cpx<T> *in, cpx<T> *out, cpx<T> *tmp_o, cudaStream_t s) {
    hop<T>(op, 1, HOP_CLOVINV, tmp_o, in, nullptr, nullptr, nr, s);          // tmp = A_oo^{-1} D_oe in
    hop<T>(op, 0, HOP_CLOVINV_XPAY, out, tmp_o, in, nullptr, nr, s);        // out = in - A_ee^{-1} D_eo tmp
}

// t = M s and the two inner products <t, s>, <t, t> into red[0..1][r]; in FP32 the products
// come out of the epilogue of the second hop where that form exists.
template <typename T>
static void schur_apply_tdots(laph_ctx *ctx, const RedPlan &pl, long nrows, const DiracOp &op, int nr,
                              const cpx<T> *sv, cpx<T> *t, cpx<T> *tmp_o, c64 *red, cudaStream_t s) {
    hop<T>(op, 1, HOP_CLOVINV, tmp_o, sv, nullptr, nullptr, nr, s);
    if (std::is_same<T, float>::value &&
        hop_f32_xpay_dots(ctx, op, 0, (c32 *)t, (const c32 *)tmp_o, (const c32 *)sv, nr, red, s))
        return;
    hop<T>(op, 0, HOP_CLOVINV_XPAY, t, tmp_o, sv, nullptr, nr, s);
    mrhs_dots<T>(ctx, pl, nrows, 2, t, sv, t, t, nullptr, nullptr, red, s);
}

// BiCGStab on the Schur operator for nr right-hand sides at once, x = 0 start.
// Per-RHS relative stopping on the recursive residual; host polls every
// `check_every` iterations (device-side scalars, no per-iteration sync).
template <typename T>
static InnerStats bicgstab_schur(laph_ctx *ctx, const DiracOp &op, int nr, const cpx<T> *b, cpx<T> *x,
                                 double rel_tol, int maxiter, int check_every, cudaStream_t s,
                                 const std::string &tag) {
    const Geom &g = op.g;
    long nrows = g.Vh * 12;
    size_t vb = sizeof(cpx<T>) * nrows * nr;
    auto V = [&](const char *n) { return (cpx<T> *)ws_get(ctx, tag + n, vb); };
    // FP32: the shadow vector is the rounded phase of r0 stored as packed 2-bit codes (blas.cuh),
    // and <rhat, v> comes out of the stencil's epilogue; FP64 (the plain solver): rhat = r0, stored
    constexpr bool gen = std::is_same<T, float>::value;
    cpx<T> *r = V(":r"), *rh = gen ? nullptr : V(":rh"), *p = V(":p"), *v = V(":v"), *sv = V(":s"), *t = V(":t");
    cpx<T> *tmp = V(":tmp");
    uint32_t *rc = gen ? (uint32_t *)ws_get(ctx, tag + ":rc", sizeof(uint32_t) * (size_t)(nrows / 12) * nr) : nullptr;
    char *scb = (char *)ws_get(ctx, tag + ":sc", (sizeof(c64) * 4 + sizeof(double) * 2 + sizeof(int) * 3) * nr + 256);
    BicgScalars sc;
    sc.rho = (c64 *)scb;
    sc.alpha = sc.rho + nr;
    sc.omega = sc.alpha + nr;
    sc.beta = sc.omega + nr;
    sc.rr = (double *)(sc.beta + nr);
    sc.rr_stop = sc.rr + nr;
    sc.active = (int *)(sc.rr_stop + nr);
    sc.status = sc.active + nr;
    sc.iters = sc.status + nr;
    c64 *red = (c64 *)ws_get(ctx, tag + ":red", sizeof(c64) * 3 * nr);
    RedPlan pl = red_plan(ctx, nrows, nr);

    LAPH_CUDA(cudaMemsetAsync(x, 0, vb, s));
    LAPH_CUDA(cudaMemsetAsync(p, 0, vb, s));
    LAPH_CUDA(cudaMemsetAsync(v, 0, vb, s));
    LAPH_CUDA(cudaMemcpyAsync(r, b, vb, cudaMemcpyDeviceToDevice, s));
    if constexpr (gen) {
        mrhs_rhat_init(ctx, pl, nrows, (const c32 *)r, rc, red, s);
        bicg_init_scalars_gen(nr, sc, red, rel_tol, s);
    } else {
        LAPH_CUDA(cudaMemcpyAsync(rh, b, vb, cudaMemcpyDeviceToDevice, s));
        mrhs_dots<T>(ctx, pl, nrows, 1, r, r, nullptr, nullptr, nullptr, nullptr, red, s);
        bicg_init_scalars(nr, sc, red, rel_tol, s);
    }

    int *h_flags = (int *)pinned_get(ctx, sizeof(int) * 3 * nr);
    if (check_every < 1) check_every = 5;
    for (int it = 0; it < maxiter; ++it) {
        bicg_p_update<T>(nrows, nr, sc, r, p, v, s);
        if constexpr (gen) {   // v = M p with <rhat, v>
            hop<T>(op, 1, HOP_CLOVINV, tmp, p, nullptr, nullptr, nr, s);
            if (!hop_f32_xpay_rdot(ctx, op, 0, v, tmp, p, nr, rc, red, s)) {
                hop<T>(op, 0, HOP_CLOVINV_XPAY, v, tmp, p, nullptr, nr, s);
                mrhs_rhat_dots(ctx, pl, nrows, v, rc, red, s);
            }
        } else {
            schur_apply<T>(op, nr, p, v, tmp, s);
            mrhs_dots<T>(ctx, pl, nrows, 1, rh, v, nullptr, nullptr, nullptr, nullptr, red, s);
        }
        bicg_alpha(nr, sc, red, s);
        bicg_s_update<T>(nrows, nr, sc, r, v, sv, s);
        schur_apply_tdots<T>(ctx, pl, nrows, op, nr, sv, t, tmp, red, s);
        bicg_omega(nr, sc, red, s);
        if constexpr (gen)
            bicg_xr_update_reduce_gen(ctx, pl, nrows, sc, x, p, sv, t, r, rc, red, s);
        else
            bicg_xr_update_reduce<T>(ctx, pl, nrows, sc, x, p, sv, t, r, rh, red, s);
        bicg_rho(nr, sc, red, s);
        if ((it + 1) % check_every == 0 || it + 1 == maxiter) {
            LAPH_CUDA(cudaMemcpyAsync(h_flags, sc.active, sizeof(int) * nr, cudaMemcpyDeviceToHost, s));
            LAPH_CUDA(cudaStreamSynchronize(s));
            hop_timeout_check(s);
            bool any = false;
            for (int k = 0; k < nr; ++k) any |= h_flags[k] != 0;
            if (!any) break;
        }
    }
    InnerStats st;
    st.iters.resize(nr);
    st.status.resize(nr);
    LAPH_CUDA(cudaMemcpyAsync(h_flags, sc.iters, sizeof(int) * nr, cudaMemcpyDeviceToHost, s));
    LAPH_CUDA(cudaMemcpyAsync(h_flags + nr, sc.status, sizeof(int) * nr, cudaMemcpyDeviceToHost, s));
    LAPH_CUDA(cudaStreamSynchronize(s));
    for (int k = 0; k < nr; ++k) {
        st.iters[k] = h_flags[k];
        st.status[k] = h_flags[nr + k];
    }
    return st;
}

// The same BiCGStab with every Krylov vector stored in BF16 (one complex per bf2) and FP32
// arithmetic (LAPH_SOLVE_MIXED_BF16); the iterate x is FP32.  nr must be 32, 64, 128 or 256 (the
// copy-engine-fed stencil).  Rounding each stored vector to 8 significant bits separates the
// recursive residual from the true one by about 1e-3 of the starting residual, which the FP64
// defect correction around this solve absorbs.
static InnerStats bicgstab_schur_bf16(laph_ctx *ctx, const DiracOp &op, int nr, const bf2 *b, c32 *x,
                                      double rel_tol, int maxiter, int check_every, cudaStream_t s) {
    const Geom &g = op.g;
    long nrows = g.Vh * 12;
    size_t vb = sizeof(bf2) * nrows * nr;
    auto V = [&](const char *n) { return (bf2 *)ws_get(ctx, std::string("in16") + n, vb); };
    bf2 *r = V(":r"), *rh = V(":rh"), *p = V(":p"), *v = V(":v"), *sv = V(":s"), *t = V(":t"), *tmp = V(":tmp");
    char *scb = (char *)ws_get(ctx, "in16:sc", (sizeof(c64) * 4 + sizeof(double) * 2 + sizeof(int) * 3) * nr + 256);
    BicgScalars sc;
    sc.rho = (c64 *)scb;
    sc.alpha = sc.rho + nr;
    sc.omega = sc.alpha + nr;
    sc.beta = sc.omega + nr;
    sc.rr = (double *)(sc.beta + nr);
    sc.rr_stop = sc.rr + nr;
    sc.active = (int *)(sc.rr_stop + nr);
    sc.status = sc.active + nr;
    sc.iters = sc.status + nr;
    c64 *red = (c64 *)ws_get(ctx, "in16:red", sizeof(c64) * 3 * nr);
    RedPlan pl = red_plan(ctx, nrows, nr);

    LAPH_CUDA(cudaMemsetAsync(x, 0, sizeof(c32) * nrows * nr, s));
    LAPH_CUDA(cudaMemsetAsync(p, 0, vb, s));
    LAPH_CUDA(cudaMemsetAsync(v, 0, vb, s));
    LAPH_CUDA(cudaMemcpyAsync(r, b, vb, cudaMemcpyDeviceToDevice, s));
    LAPH_CUDA(cudaMemcpyAsync(rh, b, vb, cudaMemcpyDeviceToDevice, s));
    mrhs_dots_bf16(ctx, pl, nrows, r, r, red, s);
    bicg_init_scalars(nr, sc, red, rel_tol, s);

    int *h_flags = (int *)pinned_get(ctx, sizeof(int) * 3 * nr);
    if (check_every < 1) check_every = 5;
    for (int it = 0; it < maxiter; ++it) {
        bicg_p_update_bf16(nrows, nr, sc, r, p, v, s);
        hop_bf16(op, 1, HOP_CLOVINV, tmp, p, nullptr, nr, s);          // v = M p
        hop_bf16(op, 0, HOP_CLOVINV_XPAY, v, tmp, p, nr, s);
        mrhs_dots_bf16(ctx, pl, nrows, rh, v, red, s);
        bicg_alpha(nr, sc, red, s);
        bicg_s_update_bf16(nrows, nr, sc, r, v, sv, s);
        hop_bf16(op, 1, HOP_CLOVINV, tmp, sv, nullptr, nr, s);         // t = M s, <t, s>, <t, t>
        if (!hop_bf16_xpay_dots(ctx, op, 0, t, tmp, sv, nr, red, s)) {
            hop_bf16(op, 0, HOP_CLOVINV_XPAY, t, tmp, sv, nr, s);
            mrhs_dots_bf16(ctx, pl, nrows, t, sv, red, s);
            mrhs_dots_bf16(ctx, pl, nrows, t, t, red + nr, s);
        }
        bicg_omega(nr, sc, red, s);
        bicg_xr_update_reduce_bf16(ctx, pl, nrows, sc, x, p, sv, t, r, rh, red, s);
        bicg_rho(nr, sc, red, s);
        if ((it + 1) % check_every == 0 || it + 1 == maxiter) {
            LAPH_CUDA(cudaMemcpyAsync(h_flags, sc.active, sizeof(int) * nr, cudaMemcpyDeviceToHost, s));
            LAPH_CUDA(cudaStreamSynchronize(s));
            hop_timeout_check(s);
            bool any = false;
            for (int k = 0; k < nr; ++k) any |= h_flags[k] != 0;
            if (!any) break;
        }
    }
    InnerStats st;
    st.iters.resize(nr);
    st.status.resize(nr);
    LAPH_CUDA(cudaMemcpyAsync(h_flags, sc.iters, sizeof(int) * nr, cudaMemcpyDeviceToHost, s));
    LAPH_CUDA(cudaMemcpyAsync(h_flags + nr, sc.status, sizeof(int) * nr, cudaMemcpyDeviceToHost, s));
    LAPH_CUDA(cudaStreamSynchronize(s));
    for (int k = 0; k < nr; ++k) {
        st.iters[k] = h_flags[k];
        st.status[k] = h_flags[nr + k];
    }
    return st;
}

std::vector<int> cgnr_solve(laph_ctx *ctx, const DiracOp &op, int nr, c64 *r, c64 *e,
                            const std::vector<double> &target, int maxiter, int check_every, std::vector<int> &conv,
                            cudaStream_t s);

// Blocks of the BF16 inner solver: the copy-engine-fed stencil's right-hand-side counts.  Other
// blocks (a short tail) run the FP32 inner solver.
static bool bf16_block_ok(int nr) { return nr == 32 || nr == 64 || nr == 128 || nr == 256; }

// Solves one block of nr right-hand sides, columns [first, first+nr) of the ABI arrays.
// A right-hand side still above the tolerance when the inner budget or the cycle limit is
// spent, or whose residual fell by less than a factor 2 in each of three consecutive
// defect-correction cycles, is finished by FP64 CG on the normal equations (params.fallback).
void solve_block(laph_ctx *ctx, const DiracOp &op, const c64 *rhs, c64 *sol, int first, int nr,
                        const laph_solver_params &prm, laph_solve_report *rep, cudaStream_t s) {
    const Geom &g = op.g;
    long nrows = g.Vh * 12;
    size_t hb = sizeof(c64) * nrows * nr;
    auto V = [&](const char *n) { return (c64 *)ws_get(ctx, std::string("dc:") + n, hb); };
    c64 *be = V("be"), *bo = V("bo"), *xe = V("xe"), *xo = V("xo"), *bh = V("bh"), *to = V("to");
    c64 *re = V("re"), *ro = V("ro"), *tmp = V("tmp");
    double *scale = (double *)ws_get(ctx, "dc:scale", sizeof(double) * 2 * nr);
    c64 *red = (c64 *)ws_get(ctx, "dc:red", sizeof(c64) * 3 * nr);
    RedPlan pl = red_plan(ctx, nrows, nr);
    std::vector<double> h_scale(2 * nr);

    fields_to_eo(g, rhs, first, nr, be, bo, s);
    // bhat = A_ee^{-1} b_e - A_ee^{-1} D_eo A_oo^{-1} b_o
    clov_inv_apply<double>(op, 1, to, bo, nr, s);
    clov_inv_apply<double>(op, 0, tmp, be, nr, s);
    hop<double>(op, 0, HOP_CLOVINV_XPAY, bh, to, tmp, nullptr, nr, s);
    // ||b||^2 of the full field
    mrhs_dots<double>(ctx, pl, nrows, 2, be, be, bo, bo, nullptr, nullptr, red, s);
    std::vector<c64> h_red(3 * nr);
    LAPH_CUDA(cudaMemcpyAsync(h_red.data(), red, sizeof(c64) * 2 * nr, cudaMemcpyDeviceToHost, s));
    LAPH_CUDA(cudaStreamSynchronize(s));
    std::vector<double> bnorm(nr);
    for (int k = 0; k < nr; ++k) bnorm[k] = std::sqrt(h_red[k].re + h_red[nr + k].re);
    // a right-hand side that is not finite cannot be solved: it is reported as not converged
    // (true residual NaN) and takes no further part in the cycles
    std::vector<int> bad(nr, 0);
    for (int k = 0; k < nr; ++k) bad[k] = !std::isfinite(bnorm[k]);
    auto rel_of = [&](int k, double rn) {
        return bad[k] ? std::nan("") : (bnorm[k] > 0 ? rn / bnorm[k] : 0.0);
    };

    LAPH_CUDA(cudaMemsetAsync(xe, 0, hb, s));
    const double tol = prm.tol;
    std::vector<double> rel(nr, 1.0);
    std::vector<int> iters(nr, 0), outer(nr, 0), broke(nr, 0), stall(nr, 0), handed(nr, 0), fell(nr, 0);
    std::vector<double> prev(nr, 1.0);
    int total_iters = 0;
    const int max_outer = 100;
    for (int cyc = 0; cyc <= max_outer; ++cyc) {
        bool all = true;
        double worst = 0.0;
        if (cyc == 0) {
            // x = 0: r = b, x_o = A_oo^{-1} b_o, and the Schur residual is bhat itself
            LAPH_CUDA(cudaMemcpyAsync(xo, to, hb, cudaMemcpyDeviceToDevice, s));
            LAPH_CUDA(cudaMemcpyAsync(re, bh, hb, cudaMemcpyDeviceToDevice, s));
            for (int k = 0; k < nr; ++k) {
                rel[k] = rel_of(k, bnorm[k]);
                if (!bad[k] && rel[k] > tol) {
                    all = false;
                    worst = 1.0;
                }
            }
            if (all) break;
        } else {
            // x_o = A_oo^{-1} b_o - A_oo^{-1} D_oe x_e, then the true residual r = b - K x.  With
            // x_o rebuilt this way r_o = b_o - A_oo x_o - D_oe x_e vanishes up to rounding, so a
            // cycle decides on r_e alone and r_o is computed (and counted) only when the cycle
            // loop is about to stop.
            hop<double>(op, 1, HOP_CLOVINV_XPAY, xo, xe, to, nullptr, nr, s);
            hop<double>(op, 0, HOP_RESID, re, xo, be, xe, nr, s);
            bool with_ro = false;
            for (;;) {
                mrhs_dots<double>(ctx, pl, nrows, with_ro ? 2 : 1, re, re, with_ro ? ro : nullptr,
                                  with_ro ? ro : nullptr, nullptr, nullptr, red, s);
                LAPH_CUDA(cudaMemcpyAsync(h_red.data(), red, sizeof(c64) * (with_ro ? 2 : 1) * nr,
                                          cudaMemcpyDeviceToHost, s));
                LAPH_CUDA(cudaStreamSynchronize(s));
                if (with_ro) break;
                bool stop = cyc == max_outer || total_iters >= prm.maxiter;
                if (!stop) {
                    stop = true;
                    for (int k = 0; k < nr; ++k) {
                        const double rn = std::sqrt(h_red[k].re);
                        const double re_rel = rel_of(k, rn);
                        if (!(re_rel <= tol) && !handed[k] && !bad[k]) stop = false;
                    }
                }
                if (!stop) {
                    for (int k = 0; k < nr; ++k) h_red[nr + k] = c64{0.0, 0.0};
                    break;
                }
                hop<double>(op, 1, HOP_RESID, ro, xe, bo, xo, nr, s);
                with_ro = true;
            }
            for (int k = 0; k < nr; ++k) {
                double rn = std::sqrt(h_red[k].re + h_red[nr + k].re);
                rel[k] = rel_of(k, rn);
                if (!(rel[k] <= tol) && !bad[k]) {
                    stall[k] = (cyc > 1 && !(rel[k] <= 0.5 * prev[k])) ? stall[k] + 1 : 0;
                    if (prm.fallback && stall[k] >= 3) handed[k] = 1;
                    if (!handed[k]) {
                        all = false;
                        worst = std::max(worst, std::isfinite(rel[k]) ? rel[k] : 1e300);
                    }
                }
                prev[k] = rel[k];
            }
            if (all || cyc == max_outer || total_iters >= prm.maxiter) break;
            // With x_o reconstructed from x_e the Schur residual bhat - M x_e equals A_ee^{-1} r_e.
            clov_inv_apply<double>(op, 0, tmp, re, nr, s);
            LAPH_CUDA(cudaMemcpyAsync(re, tmp, hb, cudaMemcpyDeviceToDevice, s));
        }
        mrhs_dots<double>(ctx, pl, nrows, 1, re, re, nullptr, nullptr, nullptr, nullptr, red, s);
        LAPH_CUDA(cudaMemcpyAsync(h_red.data(), red, sizeof(c64) * nr, cudaMemcpyDeviceToHost, s));
        LAPH_CUDA(cudaStreamSynchronize(s));
        for (int k = 0; k < nr; ++k) {
            double rn = std::sqrt(h_red[k].re);
            bool done = rel[k] <= tol || handed[k] || bad[k] || !(rn > 0.0) || !std::isfinite(rn);
            h_scale[k] = done ? 0.0 : 1.0 / rn;   // into the inner precision
            h_scale[nr + k] = done ? 0.0 : rn;    // back into x_e
            if (!done) outer[k] += 1;
        }
        LAPH_CUDA(cudaMemcpyAsync(scale, h_scale.data(), sizeof(double) * 2 * nr, cudaMemcpyHostToDevice, s));
        int budget = std::max(1, prm.maxiter - total_iters);
        InnerStats st;
        if (prm.mode == LAPH_SOLVE_PLAIN_FP64) {
            c64 *rin = (c64 *)ws_get(ctx, "dc:rin", hb);
            c64 *dx = (c64 *)ws_get(ctx, "dc:dx", hb);
            mrhs_copy_scaled<double, double>(nrows, nr, scale, re, rin, s);
            // ask the inner solve for what the true residual still needs (Schur and true residuals
            // differ by the clover factor, hence the margin)
            double want = std::max(1e-15, 0.2 * tol / std::max(worst, tol));
            st = bicgstab_schur<double>(ctx, op, nr, rin, dx, want, budget, prm.check_every, s, "in64");
            mrhs_axpy_scaled<double, double>(nrows, nr, scale + nr, dx, xe, s);
        } else if (prm.mode == LAPH_SOLVE_MIXED_BF16 && bf16_block_ok(nr)) {
            bf2 *rin = (bf2 *)ws_get(ctx, "dc:rin16", sizeof(bf2) * nrows * nr);
            c32 *dx = (c32 *)ws_get(ctx, "dc:dx32", sizeof(c32) * nrows * nr);
            mrhs_copy_scaled_bf16(nrows, nr, scale, re, rin, s);
            double want = std::max(prm.inner_tol, 0.2 * tol / std::max(worst, tol));
            st = bicgstab_schur_bf16(ctx, op, nr, rin, dx, want, budget, prm.check_every, s);
            mrhs_axpy_scaled<float, double>(nrows, nr, scale + nr, dx, xe, s);
        } else {
            c32 *rin = (c32 *)ws_get(ctx, "dc:rin32", sizeof(c32) * nrows * nr);
            c32 *dx = (c32 *)ws_get(ctx, "dc:dx32", sizeof(c32) * nrows * nr);
            mrhs_copy_scaled<double, float>(nrows, nr, scale, re, rin, s);
            double want = std::max(prm.inner_tol, 0.2 * tol / std::max(worst, tol));
            st = bicgstab_schur<float>(ctx, op, nr, rin, dx, want, budget, prm.check_every, s, "in32");
            mrhs_axpy_scaled<float, double>(nrows, nr, scale + nr, dx, xe, s);
        }
        int mx = 0;
        for (int k = 0; k < nr; ++k) {
            iters[k] += st.iters[k];
            mx = std::max(mx, st.iters[k]);
            if (st.status[k] == 2) broke[k] += 1;
        }
        total_iters += mx;
    }
    // re, ro hold the true residual b - K x of the current (xe, xo) here: every exit from the
    // cycle loop after cycle 0 comes right after it is computed, and cycle 0 exits only when
    // every right-hand side is zero.
    bool need = false;
    for (int k = 0; k < nr; ++k) need |= !(rel[k] <= tol);
    if (prm.fallback && need) {
        const long half = nrows * nr;
        c64 *rp = (c64 *)ws_get(ctx, "dc:cg_r", 2 * hb), *ep = (c64 *)ws_get(ctx, "dc:cg_e", 2 * hb);
        std::vector<double> target(nr, 0.0), mask(2 * nr, 0.0);
        for (int k = 0; k < nr; ++k) {
            fell[k] = !(rel[k] <= tol) && std::isfinite(rel[k]);
            target[k] = fell[k] ? 0.5 * tol * bnorm[k] : 0.0;
            mask[k] = fell[k] ? 1.0 : 0.0;
            mask[nr + k] = 1.0;
        }
        LAPH_CUDA(cudaMemcpyAsync(scale, mask.data(), sizeof(double) * 2 * nr, cudaMemcpyHostToDevice, s));
        mrhs_copy_scaled<double, double>(nrows, nr, scale, re, rp, s);
        mrhs_copy_scaled<double, double>(nrows, nr, scale, ro, rp + half, s);
        std::vector<int> conv;
        std::vector<int> cg_it = cgnr_solve(ctx, op, nr, rp, ep, target, 20000, prm.check_every, conv, s);
        mrhs_axpy_scaled<double, double>(nrows, nr, scale + nr, ep, xe, s);
        mrhs_axpy_scaled<double, double>(nrows, nr, scale + nr, ep + half, xo, s);
        // the true residual of the corrected solution
        hop<double>(op, 0, HOP_RESID, re, xo, be, xe, nr, s);
        hop<double>(op, 1, HOP_RESID, ro, xe, bo, xo, nr, s);
        mrhs_dots<double>(ctx, pl, nrows, 2, re, re, ro, ro, nullptr, nullptr, red, s);
        LAPH_CUDA(cudaMemcpyAsync(h_red.data(), red, sizeof(c64) * 2 * nr, cudaMemcpyDeviceToHost, s));
        LAPH_CUDA(cudaStreamSynchronize(s));
        for (int k = 0; k < nr; ++k) {
            if (!fell[k]) continue;
            rel[k] = rel_of(k, std::sqrt(h_red[k].re + h_red[nr + k].re));
            iters[k] += cg_it[k];
        }
    }
    eo_to_fields(g, xe, xo, first, nr, sol, s);
    if (rep) {
        for (int k = 0; k < nr; ++k) {
            laph_solve_report &o = rep[first + k];
            o.iters = iters[k];
            o.outer = outer[k];
            o.true_resid = rel[k];
            o.status = rel[k] <= tol ? LAPH_OK : LAPH_ERR_NOT_CONVERGED;
            o.fallback_used = fell[k];
        }
    }
}

// RHS block of the mixed solver when the caller leaves the choice to the library: among the
// block sizes 16, 32, 64 and 128 that do not exceed nrhs and whose solver vectors fit in 60 % of
// the free device memory, the one with the lowest time per right-hand side of one inner
// iteration's operator work (t = M s with <t, s> and <t, t>, fused where the shape allows), measured
// with CUDA events on scratch fields once per lattice size and candidate set and cached in
// the context.
static int autotune_block(laph_ctx *ctx, const DiracOp &op, int nrhs, cudaStream_t s) {
    if (nrhs <= 16) return nrhs;
    const long nrows = op.g.Vh * 12;
    size_t free_b = 0, total_b = 0;
    LAPH_CUDA(cudaMemGetInfo(&free_b, &total_b));
    const double per_rhs = (double)nrows * (10 * sizeof(c64) + 10 * sizeof(c32));   // FP64 outer + FP32 inner vectors
    std::vector<int> cand;
    for (int c : {16, 32, 64, 128})
        if (c <= nrhs && c * per_rhs <= 0.6 * (double)free_b) cand.push_back(c);
    if (cand.empty()) return 16;
    const std::string key = "mixed_block:" + std::to_string(op.g.Vh) + ":" + std::to_string(cand.back());
    auto it = ctx->tune.find(key);
    if (it != ctx->tune.end()) return it->second;
    const int nmax = cand.back();
    c32 *a = (c32 *)ws_get(ctx, "tune:a", sizeof(c32) * nrows * nmax);
    c32 *b = (c32 *)ws_get(ctx, "tune:b", sizeof(c32) * nrows * nmax);
    c32 *t = (c32 *)ws_get(ctx, "tune:t", sizeof(c32) * nrows * nmax);
    c64 *red = (c64 *)ws_get(ctx, "tune:red", sizeof(c64) * 2 * nmax);
    LAPH_CUDA(cudaMemsetAsync(a, 0, sizeof(c32) * nrows * nmax, s));
    cudaEvent_t e0, e1;
    LAPH_CUDA(cudaEventCreate(&e0));
    LAPH_CUDA(cudaEventCreate(&e1));
    int best = cand.back();
    double best_t = 1e300;
    for (int nr : cand) {
        RedPlan pl = red_plan(ctx, nrows, nr);
        auto once = [&]() { schur_apply_tdots<float>(ctx, pl, nrows, op, nr, a, b, t, red, s); };
        once();
        LAPH_CUDA(cudaEventRecord(e0, s));
        for (int rep = 0; rep < 3; ++rep) once();
        LAPH_CUDA(cudaEventRecord(e1, s));
        LAPH_CUDA(cudaEventSynchronize(e1));
        float ms = 0.f;
        LAPH_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        const double per = ms / (3.0 * nr);
        if (per < best_t * 0.97 || (per <= best_t * 1.03 && nr > best)) {   // ties go to the larger block
            best_t = std::min(per, best_t);
            best = nr;
        }
    }
    LAPH_CUDA(cudaEventDestroy(e0));
    LAPH_CUDA(cudaEventDestroy(e1));
    ctx->tune[key] = best;
    return best;
}

}  // namespace laph

using namespace laph;

extern "C" int laph_tuned_block(laph_ctx *ctx, int vh, int nmax) {
    if (!ctx) return 0;
    auto it = ctx->tune.find("mixed_block:" + std::to_string(vh) + ":" + std::to_string(nmax));
    return it == ctx->tune.end() ? 0 : it->second;
}

extern "C" int dirac_solve_batch(laph_ctx *ctx, const laph_lattice *lat, const void *links,
                                 const laph_dirac_params *dirac, const void *rhs, void *sol, int nrhs,
                                 const laph_solver_params *params, laph_solve_report *report, void *stream) {
    return guard([&] {
        ctx_activate(ctx);
        Geom g = make_geom(lat);
        LAPH_REQUIRE(dirac != nullptr, "dirac params are null");
        LAPH_REQUIRE(nrhs >= 0, "nrhs must be >= 0");
        laph_solver_params prm{};
        prm.mode = LAPH_SOLVE_MIXED_FP32;
        if (params) prm = *params;
        if (!(prm.tol > 0.0)) prm.tol = 1e-10;
        if (prm.maxiter <= 0) prm.maxiter = 100000;
        if (!(prm.inner_tol > 0.0)) prm.inner_tol = prm.mode == LAPH_SOLVE_MIXED_BF16 ? 1e-2 : 3e-4;
        if (prm.check_every <= 0) prm.check_every = 5;
        LAPH_REQUIRE(prm.mode == LAPH_SOLVE_PLAIN_FP64 || prm.mode == LAPH_SOLVE_MIXED_FP32 ||
                         prm.mode == LAPH_SOLVE_MIXED_BF16 || prm.mode == LAPH_SOLVE_LEARNED,
                     "unknown solver mode");
        LAPH_REQUIRE(prm.mode != LAPH_SOLVE_LEARNED || prm.weights != nullptr, "learned mode needs weights");
        if (nrhs == 0) return;
        cudaStream_t s = as_stream(stream);
        size_t lbytes = sizeof(c64) * 36 * g.V;
        size_t fbytes = sizeof(c64) * 12 * g.V * (size_t)nrhs;
        const c64 *L = (const c64 *)stage_in(ctx, links, lbytes, "links", s);
        const c64 *b = (const c64 *)stage_in(ctx, rhs, fbytes, "rhs", s);
        StagedOut o = stage_out(ctx, sol, fbytes, "sol");
        DiracOp op = prepare_dirac(ctx, g, L, dirac->m0, dirac->csw, lat->xi, s);
        const float *wdev = nullptr;
        if (prm.mode == LAPH_SOLVE_LEARNED)
            wdev = (const float *)stage_in(ctx, prm.weights, sizeof(float) * laph_precond_size(), "learned_w", s);
        int blk = prm.rhs_block;
        if (blk <= 0)
            blk = prm.mode == LAPH_SOLVE_PLAIN_FP64 ? 1
                  : prm.mode == LAPH_SOLVE_MIXED_FP32 || prm.mode == LAPH_SOLVE_MIXED_BF16
                      ? autotune_block(ctx, op, nrhs, s)
                      : std::min(nrhs, 64);
        blk = std::min(blk, std::min(nrhs, 256));
        std::vector<laph_solve_report> rep(nrhs);
        for (int first = 0; first < nrhs; first += blk) {
            int nr = std::min(blk, nrhs - first);
            if (prm.mode == LAPH_SOLVE_LEARNED)
                solve_block_learned(ctx, op, wdev, b, (c64 *)o.dev, first, nr, prm, rep.data(), s);
            else
                solve_block(ctx, op, b, (c64 *)o.dev, first, nr, prm, rep.data(), s);
        }
        o.commit(s);
        LAPH_CUDA(cudaStreamSynchronize(s));
        hop_timeout_check(s);
        bool ok = true;
        for (int k = 0; k < nrhs; ++k) ok &= rep[k].status == LAPH_OK;
        if (report) std::copy(rep.begin(), rep.end(), report);
        if (!ok) throw Error(LAPH_ERR_NOT_CONVERGED, "some right-hand sides did not reach the tolerance");
    });
}
