// Meson and I=2 two-pion correlators in LapH coefficient space (Sec. III,
// meson function Eq. (mesonfunc) at zero momentum without displacement, the
// connected term of Eq. (mesoncorr), gamma_5-swapped lines Eq. (laphpropg5)).
//
// For one quark line, the sink side is phi^[b](t,alpha,n) = coef (V_s^dag x) and
// the source side is rho^[b](t,alpha,n) = [P^(b) rho](t,alpha,n).  Because the
// eigenvectors of a slice are orthonormal, sum_{x,c} a(x)^* b(x) over LapH-smeared
// fields equals the same sum over LapH coordinates, so
//   M^[b1 b2](a, b; t) = sum_n sum_{alpha beta} conj(a^[b1](t,alpha,n)) W_{alpha beta} b^[b2](t,beta,n)
// with W = (gamma_5 gamma_4)^dag c for a barred first argument (rhobar adds a sign),
// c = gamma_4 Gamma.  All arithmetic is FP64.
#include <cmath>
#include <vector>

#include "common.cuh"
#include "gamma_host.cuh"

namespace laph {

// ----------------------------------------------------------------- kernels
// rho_src[b][alpha][n] = mask_b(t0,alpha,n) i^code(t0,alpha,n)
__global__ void rho_at_t0_kernel(int nt, int nv, int nb, int t0, const uint8_t *codes, const uint8_t *mask,
                                 c64 *out) {
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= nb * 4 * nv) return;
    int b = idx / (4 * nv), a = (idx / nv) % 4, n = idx % nv;
    const uint8_t *m = mask + (long)b * (nt + 4 + nv);
    c64 v{0, 0};
    if (m[t0] && m[nt + a] && m[nt + 4 + n]) {
        int code = codes[(t0 * 4 + a) * nv + n];
        v = code == 0 ? c64{1, 0} : code == 1 ? c64{0, 1} : code == 2 ? c64{-1, 0} : c64{0, -1};
    }
    out[idx] = v;
}

// M[t][b1][b2] = sum_n sum_{a,b} conj(A[b1][tA][a][n]) W[a][b] B[b2][tB][b][n]
// A, B: [nb][ntA][4][nv]; the slice used is t (or 0 when the operand has a single slice).
__global__ void meson_fn_kernel(int nv, int nb, int ntA, int ntB, const c64 *__restrict__ A,
                                const c64 *__restrict__ B, W4 W, c64 *__restrict__ M) {
    extern __shared__ c64 aw[];   // [4][nv]
    const int t = blockIdx.x, b1 = blockIdx.y;
    const int tA = ntA == 1 ? 0 : t, tB = ntB == 1 ? 0 : t;
    const c64 *a = A + (((long)b1 * ntA + tA) * 4) * nv;
    for (int e = threadIdx.x; e < 4 * nv; e += blockDim.x) {
        int bb = e / nv, n = e % nv;
        c64 s{0, 0};
#pragma unroll
        for (int aa = 0; aa < 4; ++aa) s += cmul_conj(a[aa * nv + n], c64{1, 0}) * W.w[aa][bb];
        aw[bb * nv + n] = s;
    }
    __syncthreads();
    for (int b2 = threadIdx.x; b2 < nb; b2 += blockDim.x) {
        const c64 *bp = B + (((long)b2 * ntB + tB) * 4) * nv;
        c64 s{0, 0};
        for (int e = 0; e < 4 * nv; ++e) s += aw[e] * bp[e];
        M[((long)t * nb + b1) * nb + b2] = s;
    }
}

// corr[dt] (+)= -scale * sum_{b1 b2} Msink[t0+dt][b1][b2] conj(Msrc[b1][b2])
__global__ void contract2_kernel(int nt, int nb, int t0, const c64 *Msink, const c64 *Msrc, double scale, c64 *corr) {
    __shared__ c64 sm[256];
    int dt = blockIdx.x;
    int t = (t0 + dt) % nt;
    c64 acc{0, 0};
    for (int e = threadIdx.x; e < nb * nb; e += blockDim.x)
        acc += cmul_conj(Msrc[e], Msink[(long)t * nb * nb + e]);
    sm[threadIdx.x] = acc;
    __syncthreads();
    for (int st = blockDim.x / 2; st > 0; st >>= 1) {
        if ((int)threadIdx.x < st) sm[threadIdx.x] += sm[threadIdx.x + st];
        __syncthreads();
    }
    if (threadIdx.x == 0) corr[dt] += (-scale) * sm[0];
}

// R[t][b1][b4] = sum_{b3} (sum_{b2} conj(S12[b1][b2]) M32[t][b3][b2]) conj(S34[b3][b4])
__global__ void pipi_p_kernel(int nb, const c64 *S12, const c64 *M32, c64 *P) {
    int t = blockIdx.x;
    for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
        int b1 = e / nb, b3 = e % nb;
        c64 s{0, 0};
        for (int b2 = 0; b2 < nb; ++b2) s += cmul_conj(S12[b1 * nb + b2], M32[((long)t * nb + b3) * nb + b2]);
        P[(long)t * nb * nb + e] = s;
    }
}

// X[t] = sum_{b1,b4} M14[t][b1][b4] sum_{b3} P[t][b1][b3] conj(S34[b3][b4]);  corr[dt] = D[dt] - X[t0+dt]
__global__ void pipi_x_kernel(int nt, int nb, int t0, const c64 *P, const c64 *S34, const c64 *M14, const c64 *cpi12,
                              const c64 *cpi34, c64 *corr) {
    __shared__ c64 sm[256];
    int dt = blockIdx.x;
    int t = (t0 + dt) % nt;
    c64 acc{0, 0};
    for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
        int b1 = e / nb, b4 = e % nb;
        c64 r{0, 0};
        for (int b3 = 0; b3 < nb; ++b3) r += P[(long)t * nb * nb + b1 * nb + b3] * conj(S34[b3 * nb + b4]);
        acc += M14[(long)t * nb * nb + e] * r;
    }
    sm[threadIdx.x] = acc;
    __syncthreads();
    for (int st = blockDim.x / 2; st > 0; st >>= 1) {
        if ((int)threadIdx.x < st) sm[threadIdx.x] += sm[threadIdx.x + st];
        __syncthreads();
    }
    if (threadIdx.x == 0) corr[dt] = cpi12[dt] * cpi34[dt] - sm[0];
}

struct LineDev {
    const c64 *coef;   // [nb][nt][4][nv]
    c64 *rho;          // [nb][1][4][nv] at t0
};

static void meson_fn(int nt_out, int nv, int nb, int ntA, int ntB, const c64 *A, const c64 *B, const Mat4 &W, c64 *M,
                     cudaStream_t s) {
    dim3 grid(nt_out, nb);
    int threads = nb < 128 ? 128 : 256;
    meson_fn_kernel<<<grid, threads, sizeof(c64) * 4 * nv, s>>>(nv, nb, ntA, ntB, A, B, to_w4(W), M);
    LAPH_LAUNCH_CHECK();
}

// Connected meson correlator of lines (l1 barred, l2), accumulated into corr with weight `scale`.
static void meson_connected(laph_ctx *ctx, int nt, int nv, int nb, int t0, const LineDev &l1, const LineDev &l2,
                            const Mat4 &c, double scale, c64 *corr, cudaStream_t s, const std::string &tag) {
    Mat4 g5g4 = mat_mul(gamma5(), gamma_mat(3));
    Mat4 wsink = mat_mul(mat_dag(g5g4), c);               // phibar = g5 g4 phi
    Mat4 wsrc = mat_scale(-1.0, wsink);                   // rhobar = -g5 g4 rho
    c64 *Msink = (c64 *)ws_get(ctx, "corr:Msink" + tag, sizeof(c64) * nt * nb * nb);
    c64 *Msrc = (c64 *)ws_get(ctx, "corr:Msrc" + tag, sizeof(c64) * nb * nb);
    meson_fn(nt, nv, nb, nt, nt, l1.coef, l2.coef, wsink, Msink, s);
    meson_fn(1, nv, nb, 1, 1, l1.rho, l2.rho, wsrc, Msrc, s);
    contract2_kernel<<<nt, 256, 0, s>>>(nt, nb, t0, Msink, Msrc, scale, corr);
    LAPH_LAUNCH_CHECK();
}

}  // namespace laph

using namespace laph;

extern "C" int correlate(laph_ctx *ctx, const laph_lattice *lat, const laph_corr_spec *spec, const void *const *coef,
                         const uint8_t *const *noise, void *corr, void *stream) {
    return guard([&] {
        ctx_activate(ctx);
        LAPH_REQUIRE(lat != nullptr && spec != nullptr && coef != nullptr && noise != nullptr, "null argument");
        const int nt = lat->nt, nv = spec->nv, nb = spec->nb, t0 = spec->t0;
        LAPH_REQUIRE(nt >= 1 && nv >= 1 && nb >= 1, "bad sizes");
        LAPH_REQUIRE(t0 >= 0 && t0 < nt, "t0 out of range");
        LAPH_REQUIRE(spec->b_list != nullptr, "b_list is null");
        int nlines = spec->channel == LAPH_CH_PIPI_I2 ? 4 : 2;
        LAPH_REQUIRE(spec->channel >= 0 && spec->channel <= LAPH_CH_PIPI_I2, "unknown channel");
        cudaStream_t s = as_stream(stream);
        std::vector<uint8_t> m = dilution_masks(spec->dil, nt, nv, spec->b_list, nb);
        uint8_t *dm = (uint8_t *)ws_get(ctx, "corr:mask", m.size());
        LAPH_CUDA(cudaMemcpyAsync(dm, m.data(), m.size(), cudaMemcpyHostToDevice, s));
        std::vector<LineDev> lines(nlines);
        for (int k = 0; k < nlines; ++k) {
            LAPH_REQUIRE(coef[k] != nullptr && noise[k] != nullptr, "line arrays are null");
            std::string id = std::to_string(k);
            lines[k].coef = (const c64 *)stage_in(ctx, coef[k], sizeof(c64) * (size_t)nb * nt * 4 * nv, "corr:coef" + id, s);
            const uint8_t *codes = (const uint8_t *)stage_in(ctx, noise[k], (size_t)nt * 4 * nv, "corr:noise" + id, s);
            lines[k].rho = (c64 *)ws_get(ctx, "corr:rho" + id, sizeof(c64) * nb * 4 * nv);
            rho_at_t0_kernel<<<grid_for((long)nb * 4 * nv, 256), 256, 0, s>>>(nt, nv, nb, t0, codes, dm, lines[k].rho);
            LAPH_LAUNCH_CHECK();
        }
        StagedOut out = stage_out(ctx, corr, sizeof(c64) * nt, "corr");
        c64 *c = (c64 *)out.dev;
        LAPH_CUDA(cudaMemsetAsync(c, 0, sizeof(c64) * nt, s));
        Mat4 g4 = gamma_mat(3);
        if (spec->channel == LAPH_CH_PION) {
            meson_connected(ctx, nt, nv, nb, t0, lines[0], lines[1], mat_mul(g4, gamma5()), 1.0, c, s, "a");
        } else if (spec->channel == LAPH_CH_SCALAR) {
            meson_connected(ctx, nt, nv, nb, t0, lines[0], lines[1], mat_mul(g4, ident4()), 1.0, c, s, "a");
        } else if (spec->channel == LAPH_CH_RHO) {
            for (int k = 0; k < 3; ++k)
                meson_connected(ctx, nt, nv, nb, t0, lines[0], lines[1], mat_mul(g4, gamma_mat(k)), 1.0 / 3.0, c, s, "a");
        } else {
            Mat4 cpi = mat_mul(g4, gamma5());
            c64 *c12 = (c64 *)ws_get(ctx, "corr:c12", sizeof(c64) * nt);
            c64 *c34 = (c64 *)ws_get(ctx, "corr:c34", sizeof(c64) * nt);
            LAPH_CUDA(cudaMemsetAsync(c12, 0, sizeof(c64) * nt, s));
            LAPH_CUDA(cudaMemsetAsync(c34, 0, sizeof(c64) * nt, s));
            meson_connected(ctx, nt, nv, nb, t0, lines[0], lines[1], cpi, 1.0, c12, s, "a");
            meson_connected(ctx, nt, nv, nb, t0, lines[2], lines[3], cpi, 1.0, c34, s, "b");
            Mat4 g5g4 = mat_mul(gamma5(), g4);
            Mat4 wsink = mat_mul(mat_dag(g5g4), cpi);
            Mat4 wsrc = mat_scale(-1.0, wsink);
            size_t mb = sizeof(c64) * nt * nb * nb;
            c64 *M14 = (c64 *)ws_get(ctx, "corr:M14", mb);
            c64 *M32 = (c64 *)ws_get(ctx, "corr:M32", mb);
            c64 *S12 = (c64 *)ws_get(ctx, "corr:S12", sizeof(c64) * nb * nb);
            c64 *S34 = (c64 *)ws_get(ctx, "corr:S34", sizeof(c64) * nb * nb);
            c64 *P = (c64 *)ws_get(ctx, "corr:P", mb);
            meson_fn(nt, nv, nb, nt, nt, lines[0].coef, lines[3].coef, wsink, M14, s);   // M(phibar_1, phi_4)
            meson_fn(nt, nv, nb, nt, nt, lines[2].coef, lines[1].coef, wsink, M32, s);   // M(phibar_3, phi_2)
            meson_fn(1, nv, nb, 1, 1, lines[0].rho, lines[1].rho, wsrc, S12, s);         // M(rhobar_1, rho_2)
            meson_fn(1, nv, nb, 1, 1, lines[2].rho, lines[3].rho, wsrc, S34, s);         // M(rhobar_3, rho_4)
            pipi_p_kernel<<<nt, 256, 0, s>>>(nb, S12, M32, P);
            LAPH_LAUNCH_CHECK();
            pipi_x_kernel<<<nt, 256, 0, s>>>(nt, nb, t0, P, S34, M14, c12, c34, c);
            LAPH_LAUNCH_CHECK();
        }
        out.commit(s);
        LAPH_CUDA(cudaStreamSynchronize(s));
    });
}
