// FP64 conjugate gradient on the normal equations K^dag K e = K^dag r (Sec. IV: where the
// biconjugate-gradient solve does not converge, a slower CG solve of Omega^dag Omega x =
// Omega^dag y finishes the system; with Omega = gamma_4 K this is the same system, since
// Omega^dag Omega = K^dag K and Omega^dag y = K^dag gamma_4 y).
//
// Fields are full-lattice pairs [even half | odd half] of parity-half fields f[cb*12+k][r];
// K is applied parity by parity (A_pp x_p + D_pq x_q) and K^dag = gamma_5 K gamma_5
// (gamma_5-Hermiticity, Sec. II; gamma_5 = diag(1, 1, -1, -1) in the chiral basis).  Every
// right-hand side of the block runs its own recurrence with its own scalars on the device;
// a right-hand side that has reached its target keeps alpha = beta = 0 from then on.
#include <cmath>
#include <vector>

#include "blas.cuh"
#include "dirac.cuh"

namespace laph {

__global__ void gamma5_kernel(long n, int nr, const c64 *x, c64 *y) {
    long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int k = (int)((i / nr) % 12);   // spin * 3 + colour
    const c64 v = x[i];
    y[i] = k >= 6 ? -v : v;
}

// alpha = gamma / |q|^2 on active right-hand sides, else 0
__global__ void cg_alpha_kernel(int nr, const c64 *qq, const double *gamma, const int *active, double *alpha,
                                double *nalpha) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nr) return;
    const double q = qq[r].re;
    double a = 0.0;
    if (active[r] && q > 0.0 && gamma[r] > 0.0 && isfinite(q)) a = gamma[r] / q;
    alpha[r] = a;
    nalpha[r] = -a;
}

// beta = |s_new|^2 / |s_old|^2 and gamma <- |s_new|^2 on active right-hand sides, else 0
__global__ void cg_beta_kernel(int nr, const c64 *ss, double *gamma, const int *active, double *beta) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nr) return;
    const double g = ss[r].re;
    const bool on = active[r] && isfinite(g);
    beta[r] = (on && gamma[r] > 0.0) ? g / gamma[r] : 0.0;
    gamma[r] = on ? g : 0.0;
}

static void gamma5(long n, int nr, const c64 *x, c64 *y, cudaStream_t s) {
    gamma5_kernel<<<grid_for(n, 256), 256, 0, s>>>(n, nr, x, y);
    LAPH_LAUNCH_CHECK();
}

// e = K^{-1} r per right-hand side, to ||r - K e|| <= target[k] (absolute); target[k] <= 0
// skips column k (e = 0).  `r` is overwritten.  Returns per-RHS iterations; conv[k] = 1
// when column k reached its target.  ||r - K e|| decreases monotonically in CG on the
// normal equations; a column whose residual gains less than 1 % over 20 consecutive checks
// (rounding floor) stops there.
std::vector<int> cgnr_solve(laph_ctx *ctx, const DiracOp &op, int nr, c64 *r, c64 *e,
                            const std::vector<double> &target, int maxiter, int check_every, std::vector<int> &conv,
                            cudaStream_t s) {
    const long half = op.g.Vh * 12 * (long)nr;   // elements of one parity half
    const long nrows2 = 2 * op.g.Vh * 12;
    const size_t pb = sizeof(c64) * 2 * half;
    c64 *sv = (c64 *)ws_get(ctx, "cg:s", pb), *p = (c64 *)ws_get(ctx, "cg:p", pb);
    c64 *q = (c64 *)ws_get(ctx, "cg:q", pb), *t = (c64 *)ws_get(ctx, "cg:t", pb);
    double *dsc = (double *)ws_get(ctx, "cg:scal", sizeof(double) * 5 * nr);
    double *gamma = dsc, *alpha = dsc + nr, *nalpha = dsc + 2 * nr, *beta = dsc + 3 * nr, *ones = dsc + 4 * nr;
    int *active = (int *)ws_get(ctx, "cg:active", sizeof(int) * nr);
    c64 *red = (c64 *)ws_get(ctx, "cg:red", sizeof(c64) * nr);
    RedPlan pl = red_plan(ctx, nrows2, nr);

    auto K = [&](const c64 *x, c64 *y) {
        hop<double>(op, 0, HOP_APPLY, y, x + half, nullptr, x, nr, s);
        hop<double>(op, 1, HOP_APPLY, y + half, x, nullptr, x + half, nr, s);
    };
    auto Kdag = [&](const c64 *x, c64 *y) {
        gamma5(2 * half, nr, x, t, s);
        K(t, y);
        gamma5(2 * half, nr, y, y, s);
    };
    auto norms = [&](const c64 *x, std::vector<double> &out) {
        mrhs_dots<double>(ctx, pl, nrows2, 1, x, x, nullptr, nullptr, nullptr, nullptr, red, s);
        std::vector<c64> h(nr);
        LAPH_CUDA(cudaMemcpyAsync(h.data(), red, sizeof(c64) * nr, cudaMemcpyDeviceToHost, s));
        LAPH_CUDA(cudaStreamSynchronize(s));
        for (int k = 0; k < nr; ++k) out[k] = std::sqrt(std::max(h[k].re, 0.0));
    };

    std::vector<int> iters(nr, 0), h_active(nr, 0), flat(nr, 0);
    std::vector<double> rn(nr), h_ones(nr, 1.0), best(nr, 0.0);
    conv.assign(nr, 0);
    LAPH_CUDA(cudaMemsetAsync(e, 0, pb, s));
    norms(r, rn);
    int nact = 0;
    for (int k = 0; k < nr; ++k) {
        conv[k] = target[k] > 0.0 && rn[k] <= target[k];
        h_active[k] = target[k] > 0.0 && !conv[k] && std::isfinite(rn[k]);
        best[k] = rn[k];
        nact += h_active[k];
    }
    if (nact == 0) return iters;
    LAPH_CUDA(cudaMemcpyAsync(active, h_active.data(), sizeof(int) * nr, cudaMemcpyHostToDevice, s));
    LAPH_CUDA(cudaMemcpyAsync(ones, h_ones.data(), sizeof(double) * nr, cudaMemcpyHostToDevice, s));
    LAPH_CUDA(cudaMemsetAsync(gamma, 0, sizeof(double) * nr, s));

    // s = K^dag r, p = s, gamma = |s|^2
    Kdag(r, sv);
    LAPH_CUDA(cudaMemcpyAsync(p, sv, pb, cudaMemcpyDeviceToDevice, s));
    mrhs_dots<double>(ctx, pl, nrows2, 1, sv, sv, nullptr, nullptr, nullptr, nullptr, red, s);
    cg_beta_kernel<<<grid_for(nr, 256), 256, 0, s>>>(nr, red, gamma, active, beta);   // beta unused here
    LAPH_LAUNCH_CHECK();
    if (check_every < 1) check_every = 25;
    for (int it = 0; it < maxiter; ++it) {
        K(p, q);
        mrhs_dots<double>(ctx, pl, nrows2, 1, q, q, nullptr, nullptr, nullptr, nullptr, red, s);
        cg_alpha_kernel<<<grid_for(nr, 256), 256, 0, s>>>(nr, red, gamma, active, alpha, nalpha);
        LAPH_LAUNCH_CHECK();
        mrhs_axpy_scaled<double, double>(nrows2, nr, alpha, p, e, s);
        mrhs_axpy_scaled<double, double>(nrows2, nr, nalpha, q, r, s);
        Kdag(r, sv);
        mrhs_dots<double>(ctx, pl, nrows2, 1, sv, sv, nullptr, nullptr, nullptr, nullptr, red, s);
        cg_beta_kernel<<<grid_for(nr, 256), 256, 0, s>>>(nr, red, gamma, active, beta);
        LAPH_LAUNCH_CHECK();
        mrhs_copy_scaled<double, double>(nrows2, nr, beta, p, p, s);
        mrhs_axpy_scaled<double, double>(nrows2, nr, ones, sv, p, s);
        for (int k = 0; k < nr; ++k) iters[k] += h_active[k];
        if ((it + 1) % check_every == 0 || it + 1 == maxiter) {
            norms(r, rn);
            nact = 0;
            for (int k = 0; k < nr; ++k) {
                if (h_active[k] && rn[k] <= target[k]) {
                    conv[k] = 1;
                    h_active[k] = 0;
                }
                if (h_active[k] && !std::isfinite(rn[k])) h_active[k] = 0;
                if (h_active[k]) {
                    flat[k] = rn[k] > 0.99 * best[k] ? flat[k] + 1 : 0;
                    best[k] = std::min(best[k], rn[k]);
                    if (flat[k] >= 20) h_active[k] = 0;
                }
                nact += h_active[k];
            }
            if (nact == 0) break;
            LAPH_CUDA(cudaMemcpyAsync(active, h_active.data(), sizeof(int) * nr, cudaMemcpyHostToDevice, s));
        }
    }
    return iters;
}

}  // namespace laph
