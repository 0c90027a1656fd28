// Momentum and same-time pieces of the meson correlators, in LapH coefficient space.
//
// Momentum (Sec. III, the phase e^{-ip.x} of Eq. (mesonfunc) without displacement): an operator
// of momentum p = 2 pi (px, py, pz) / N_s carries sum_x e^{-ip.x}; since phi and varrho are
// LapH-smeared fields V a, the phase enters through the overlaps
//     Phi_p(t)[n, n'] = sum_{x,c} conj(V(t,n,x,c)) e^{-ip.x} V(t,n',x,c)        (laph_mom_overlaps)
// so that M^[b1 b2](a, b; t) = sum conj(a^[b1](t,alpha,n)) W_{alpha beta} Phi_p(t)[n,n'] b^[b2](t,beta,n').
// The sink function at t_F and the source function at t_0 take the same p, and Eq. (mesoncorr)
// conjugates the source one (correlate_mom).
//
// Same-time lines (second term of Eq. (mesoncorr), the isoscalar "smt" diagram of Sec. V): each
// line closes on one slice and its b sum runs alone,
//     L_c(t) = sum_b M^[bb](varrho, varphi; t)    or, reversed,   sum_b M^[bb](varphi, varrho; t)
// with c = gamma_4 Gamma and no gamma_5 swap (laph_meson_loops); the disconnected correlator is
// (1 / n_c) sum_c L_1c(t_0 + dt) conj(L_2c(t_0)) minus a vacuum term (correlate_disconnected).
// All arithmetic is FP64.
#include <cmath>
#include <cstdlib>
#include <vector>

#include "gamma_host.cuh"

namespace laph {

namespace {

// e^{-ip.x} for every site of a slice (x fastest) and every momentum; the phase argument is
// reduced mod N_s in integers before the sincospi call.
__global__ void mom_phase_kernel(int ns, int nmom, const int *mom, c64 *ph) {
    const long v3 = (long)ns * ns * ns;
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    const int p = blockIdx.y;
    if (i >= v3) return;
    const int x = (int)(i % ns), y = (int)((i / ns) % ns), z = (int)(i / ((long)ns * ns));
    const int a = ((mom[3 * p] * x + mom[3 * p + 1] * y + mom[3 * p + 2] * z) % ns + ns) % ns;
    double sn, cs;
    sincospi(-2.0 * a / ns, &sn, &cs);
    ph[(long)p * v3 + i] = c64{cs, sn};
}

// Phi[p][t][n][n'] = scale sum_k conj(A[t][n][k]) ph[p][k / 3] B[t][n'][k], k = 3 x + c (A = B = V for
// the plain overlaps).  16 x 16 output tiles, the K sum in shared-memory slabs of 32.
constexpr int OV_T = 16, OV_K = 32;
__global__ void __launch_bounds__(256) overlaps_kernel(long V3, int nv, int nt, const c64 *__restrict__ Av,
                                                       const c64 *__restrict__ Bv, const c64 *__restrict__ ph,
                                                       c64 scale, c64 *__restrict__ phi) {
    __shared__ c64 As[OV_T][OV_K + 1], Bs[OV_T][OV_K + 1];
    const int tx = threadIdx.x % OV_T, ty = threadIdx.x / OV_T;
    const int n0 = blockIdx.x * OV_T, m0 = blockIdx.y * OV_T;
    const int t = blockIdx.z % nt, p = blockIdx.z / nt;
    const long K = 3 * V3;
    const c64 *at = Av + (long)t * nv * K, *bt = Bv + (long)t * nv * K;
    const c64 *pp = ph + (long)p * V3;
    c64 acc{0, 0};
    for (long k0 = 0; k0 < K; k0 += OV_K) {
        for (int e = threadIdx.x; e < OV_T * OV_K; e += blockDim.x) {
            const int r = e / OV_K, kk = e % OV_K;
            const long k = k0 + kk;
            const int na = n0 + r, nb = m0 + r;
            As[r][kk] = (na < nv && k < K) ? conj(at[(long)na * K + k]) : c64{0, 0};
            Bs[r][kk] = (nb < nv && k < K) ? pp[k / 3] * bt[(long)nb * K + k] : c64{0, 0};
        }
        __syncthreads();
#pragma unroll 8
        for (int kk = 0; kk < OV_K; ++kk) acc += As[ty][kk] * Bs[tx][kk];
        __syncthreads();
    }
    const int n = n0 + ty, m = m0 + tx;
    if (n < nv && m < nv) phi[(((long)p * nt + t) * nv + n) * nv + m] = scale * acc;
}

// One gauge-covariant step of the colour vectors V [nt][nv][V3][3] (Sec. II, the paths of D^(j)):
// s = +mu: out(x) = U_mu(x) in(x + mu);  s = -mu: out(x) = U_mu(x - mu)^dag in(x - mu);  mu = 1, 2, 3
// for x, y, z, periodic in space.  U: [V][4][3][3] (the Laplacian's smeared links).
__global__ void disp_step_kernel(Geom g, const c64 *__restrict__ U, int nv, int s, const c64 *__restrict__ in,
                                 c64 *__restrict__ out) {
    const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long)g.nt * nv * g.V3) return;
    const long xs = idx % g.V3;
    const long tn = idx / g.V3;
    const int t = (int)(tn / nv);
    int c[3] = {(int)(xs % g.ns), (int)((xs / g.ns) % g.ns), (int)(xs / ((long)g.ns * g.ns))};
    const int mu = (s > 0 ? s : -s) - 1;
    c[mu] = (c[mu] + (s > 0 ? 1 : g.ns - 1)) % g.ns;
    const long ys = ((long)c[2] * g.ns + c[1]) * g.ns + c[0];          // the neighbour x +- mu
    const c64 *v = in + (tn * g.V3 + ys) * 3;
    const c64 *u = U + (((long)t * g.V3 + (s > 0 ? xs : ys)) * 4 + mu) * 9;
    for (int a = 0; a < 3; ++a) {
        c64 acc{0, 0};
        for (int b = 0; b < 3; ++b) acc += (s > 0 ? u[a * 3 + b] : conj(u[b * 3 + a])) * v[b];
        out[(tn * g.V3 + xs) * 3 + a] = acc;
    }
}

// out[b][t][beta][n] = sum_n' Phi(t_B)[n][n'] in[b][t][beta][n'], t_B = t or the fixed slice t1 when
// the operand has a single slice (nt_in == 1)
__global__ void phi_apply_kernel(int nv, int nt_in, int t1, const c64 *__restrict__ phi, const c64 *__restrict__ in,
                                 c64 *__restrict__ out) {
    const int b = blockIdx.x, t = blockIdx.y;
    const int tp = nt_in == 1 ? t1 : t;
    const c64 *f = phi + (long)tp * nv * nv;
    const c64 *src = in + ((long)b * nt_in + t) * 4 * nv;
    c64 *dst = out + ((long)b * nt_in + t) * 4 * nv;
    for (int e = threadIdx.x; e < 4 * nv; e += blockDim.x) {
        const int be = e / nv, n = e % nv;
        c64 s{0, 0};
        for (int m = 0; m < nv; ++m) s += f[(long)n * nv + m] * src[be * nv + m];
        dst[e] = s;
    }
}

// rho[b][t][alpha][n] = mask_b(t, alpha, n) i^code(t, alpha, n) for every slice
__global__ void rho_all_kernel(int nt, int nv, int nb, const uint8_t *codes, const uint8_t *mask, c64 *out) {
    const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long)nb * nt * 4 * nv) return;
    const int n = (int)(idx % nv), a = (int)((idx / nv) % 4), t = (int)((idx / (4 * nv)) % nt);
    const int b = (int)(idx / ((long)nt * 4 * nv));
    const uint8_t *m = mask + (long)b * (nt + 4 + nv);
    c64 v{0, 0};
    if (m[t] && m[nt + a] && m[nt + 4 + n]) {
        const int code = codes[(t * 4 + a) * nv + n];
        v = code == 0 ? c64{1, 0} : code == 1 ? c64{0, 1} : code == 2 ? c64{-1, 0} : c64{0, -1};
    }
    out[idx] = v;
}

struct W3 {
    W4 w[3];
};

// loops[c][t] = sum_b sum_n sum_{alpha beta} conj(A[b][t][alpha][n]) W_c[alpha][beta] B[b][t][beta][n], one block per t
__global__ void loops_kernel(int nt, int nv, int nb, int nc, const c64 *__restrict__ A, const c64 *__restrict__ B,
                             W3 W, c64 *__restrict__ loops) {
    __shared__ c64 sm[3][256];
    const int t = blockIdx.x;
    c64 acc[3] = {{0, 0}, {0, 0}, {0, 0}};
    for (long e = threadIdx.x; e < (long)nb * nv; e += blockDim.x) {
        const int b = (int)(e / nv), n = (int)(e % nv);
        const c64 *a = A + ((long)b * nt + t) * 4 * nv + n;
        const c64 *bb = B + ((long)b * nt + t) * 4 * nv + n;
        c64 av[4], bv[4];
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            av[s] = conj(a[s * nv]);
            bv[s] = bb[s * nv];
        }
        for (int c = 0; c < nc; ++c)
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[c] += av[i] * (W.w[c].w[i][j] * bv[j]);
    }
    for (int c = 0; c < 3; ++c) sm[c][threadIdx.x] = acc[c];
    __syncthreads();
    for (int st = blockDim.x / 2; st > 0; st >>= 1) {
        if ((int)threadIdx.x < st)
            for (int c = 0; c < 3; ++c) sm[c][threadIdx.x] += sm[c][threadIdx.x + st];
        __syncthreads();
    }
    if (threadIdx.x < nc) loops[(long)threadIdx.x * nt + t] = sm[threadIdx.x][0];
}

// corr[dt] = (1 / nc) sum_c L1[c][(t0 + dt) mod nt] conj(L2[c][t0]) - vev
__global__ void disconnected_kernel(int nt, int nc, int t0, const c64 *L1, const c64 *L2, c64 vev, c64 *corr) {
    const int dt = blockIdx.x * blockDim.x + threadIdx.x;
    if (dt >= nt) return;
    c64 s{0, 0};
    for (int c = 0; c < nc; ++c) s += L1[(long)c * nt + (t0 + dt) % nt] * conj(L2[(long)c * nt + t0]);
    corr[dt] = (1.0 / nc) * s - vev;
}

void check_spec(const laph_lattice *lat, const laph_corr_spec *spec) {
    LAPH_REQUIRE(lat != nullptr && spec != nullptr, "null argument");
    LAPH_REQUIRE(lat->nt >= 1 && spec->nv >= 1 && spec->nb >= 1, "bad sizes");
    LAPH_REQUIRE(spec->b_list != nullptr, "b_list is null");
    LAPH_REQUIRE(spec->channel == LAPH_CH_PION || spec->channel == LAPH_CH_RHO || spec->channel == LAPH_CH_SCALAR,
                 "meson channel expected (pion, rho or scalar)");
}

}  // namespace

}  // namespace laph

using namespace laph;

extern "C" int laph_mom_overlaps(laph_ctx *ctx, const laph_lattice *lat, const void *evecs, int nv, int nmom,
                                 const int *mom, void *phi, void *stream) {
    return guard([&] {
        ctx_activate(ctx);
        Geom g = make_geom(lat);
        LAPH_REQUIRE(nv >= 1 && nv <= 3 * g.V3, "nv out of range");
        LAPH_REQUIRE(nmom >= 0 && (nmom == 0 || mom != nullptr), "momenta are null");
        LAPH_REQUIRE((long)g.nt * nmom <= 65535, "nt * nmom above 65535");
        if (nmom == 0) return;
        cudaStream_t s = as_stream(stream);
        const c64 *V = (const c64 *)stage_in(ctx, evecs, sizeof(c64) * 3 * g.V3 * g.nt * (size_t)nv, "ov:evecs", s);
        int *dmom = (int *)ws_get(ctx, "ov:mom", sizeof(int) * 3 * nmom);
        LAPH_CUDA(cudaMemcpyAsync(dmom, mom, sizeof(int) * 3 * nmom, cudaMemcpyHostToDevice, s));
        c64 *ph = (c64 *)ws_get(ctx, "ov:phase", sizeof(c64) * g.V3 * nmom);
        mom_phase_kernel<<<dim3(grid_for(g.V3, 256), nmom), 256, 0, s>>>(g.ns, nmom, dmom, ph);
        LAPH_LAUNCH_CHECK();
        StagedOut o = stage_out(ctx, phi, sizeof(c64) * nmom * g.nt * (size_t)nv * nv, "ov:phi");
        const dim3 grid((nv + OV_T - 1) / OV_T, (nv + OV_T - 1) / OV_T, g.nt * nmom);
        prof_begin("overlaps", s);
        overlaps_kernel<<<grid, 256, 0, s>>>(g.V3, nv, g.nt, V, V, ph, c64{1.0, 0.0}, (c64 *)o.dev);
        LAPH_LAUNCH_CHECK();
        prof_end("overlaps", s, 16.0 * 3 * g.V3 * g.nt * (double)nv * grid.x * nmom,
                 8.0 * nv * (double)nv * 3 * g.V3 * g.nt * nmom);
        o.commit(s);
        LAPH_CUDA(cudaStreamSynchronize(s));
    });
}

extern "C" int correlate_mom(laph_ctx *ctx, const laph_lattice *lat, const laph_corr_spec *spec,
                             const void *const *coef, const uint8_t *const *noise, const void *phi, void *corr,
                             void *stream) {
    return guard([&] {
        ctx_activate(ctx);
        check_spec(lat, spec);
        LAPH_REQUIRE(coef != nullptr && noise != nullptr && phi != nullptr && corr != nullptr, "null argument");
        const int nt = lat->nt, nv = spec->nv, nb = spec->nb, t0 = spec->t0;
        LAPH_REQUIRE(t0 >= 0 && t0 < nt, "t0 out of range");
        cudaStream_t s = as_stream(stream);
        std::vector<uint8_t> m = dilution_masks(spec->dil, nt, nv, spec->b_list, nb);
        uint8_t *dm = (uint8_t *)ws_get(ctx, "cm:mask", m.size());
        LAPH_CUDA(cudaMemcpyAsync(dm, m.data(), m.size(), cudaMemcpyHostToDevice, s));
        const c64 *dphi = (const c64 *)stage_in(ctx, phi, sizeof(c64) * nt * (size_t)nv * nv, "cm:phi", s);
        const c64 *cf[2];
        c64 *rho[2];
        for (int k = 0; k < 2; ++k) {
            LAPH_REQUIRE(coef[k] != nullptr && noise[k] != nullptr, "line arrays are null");
            const std::string id = std::to_string(k);
            cf[k] = (const c64 *)stage_in(ctx, coef[k], sizeof(c64) * (size_t)nb * nt * 4 * nv, "cm:coef" + id, s);
            const uint8_t *codes = (const uint8_t *)stage_in(ctx, noise[k], (size_t)nt * 4 * nv, "cm:noise" + id, s);
            rho[k] = (c64 *)ws_get(ctx, "cm:rho" + id, sizeof(c64) * nb * 4 * nv);
            rho_at_t0_kernel<<<grid_for((long)nb * 4 * nv, 256), 256, 0, s>>>(nt, nv, nb, t0, codes, dm, rho[k]);
            LAPH_LAUNCH_CHECK();
        }
        // Phi_p on the second line: its coefficients at every slice and its noise at t0
        c64 *cf2 = (c64 *)ws_get(ctx, "cm:coef2p", sizeof(c64) * (size_t)nb * nt * 4 * nv);
        c64 *rho2 = (c64 *)ws_get(ctx, "cm:rho2p", sizeof(c64) * nb * 4 * nv);
        phi_apply_kernel<<<dim3(nb, nt), 128, 0, s>>>(nv, nt, 0, dphi, cf[1], cf2);
        LAPH_LAUNCH_CHECK();
        phi_apply_kernel<<<dim3(nb, 1), 128, 0, s>>>(nv, 1, t0, dphi, rho[1], rho2);
        LAPH_LAUNCH_CHECK();
        StagedOut out = stage_out(ctx, corr, sizeof(c64) * nt, "cm:corr");
        c64 *c = (c64 *)out.dev;
        LAPH_CUDA(cudaMemsetAsync(c, 0, sizeof(c64) * nt, s));
        Mat4 cs[3];
        const int nc = channel_c(spec->channel, cs);
        const Mat4 g5g4 = mat_mul(gamma5(), gamma_mat(3));
        c64 *Msink = (c64 *)ws_get(ctx, "cm:Msink", sizeof(c64) * nt * nb * nb);
        c64 *Msrc = (c64 *)ws_get(ctx, "cm:Msrc", sizeof(c64) * nb * nb);
        const int threads = nb < 128 ? 128 : 256;
        for (int k = 0; k < nc; ++k) {
            const Mat4 wsink = mat_mul(mat_dag(g5g4), cs[k]);   // phibar = g5 g4 phi
            const Mat4 wsrc = mat_scale(-1.0, wsink);           // rhobar = -g5 g4 rho
            meson_fn_kernel<<<dim3(nt, nb), threads, sizeof(c64) * 4 * nv, s>>>(nv, nb, nt, nt, cf[0], cf2,
                                                                                to_w4(wsink), Msink);
            LAPH_LAUNCH_CHECK();
            meson_fn_kernel<<<dim3(1, nb), threads, sizeof(c64) * 4 * nv, s>>>(nv, nb, 1, 1, rho[0], rho2,
                                                                               to_w4(wsrc), Msrc);
            LAPH_LAUNCH_CHECK();
            contract2_kernel<<<nt, 256, 0, s>>>(nt, nb, t0, Msink, Msrc, 1.0 / nc, c);
            LAPH_LAUNCH_CHECK();
        }
        out.commit(s);
        LAPH_CUDA(cudaStreamSynchronize(s));
    });
}

extern "C" int laph_meson_loops(laph_ctx *ctx, const laph_lattice *lat, const laph_corr_spec *spec, const void *coef,
                                const uint8_t *noise, const void *phi, int reverse, void *loops, void *stream) {
    return guard([&] {
        ctx_activate(ctx);
        check_spec(lat, spec);
        LAPH_REQUIRE(coef != nullptr && noise != nullptr && loops != nullptr, "null argument");
        const int nt = lat->nt, nv = spec->nv, nb = spec->nb;
        cudaStream_t s = as_stream(stream);
        std::vector<uint8_t> m = dilution_masks(spec->dil, nt, nv, spec->b_list, nb);
        uint8_t *dm = (uint8_t *)ws_get(ctx, "lp:mask", m.size());
        LAPH_CUDA(cudaMemcpyAsync(dm, m.data(), m.size(), cudaMemcpyHostToDevice, s));
        const size_t fb = sizeof(c64) * (size_t)nb * nt * 4 * nv;
        const c64 *cf = (const c64 *)stage_in(ctx, coef, fb, "lp:coef", s);
        const uint8_t *codes = (const uint8_t *)stage_in(ctx, noise, (size_t)nt * 4 * nv, "lp:noise", s);
        c64 *rho = (c64 *)ws_get(ctx, "lp:rho", fb);
        rho_all_kernel<<<grid_for((long)nb * nt * 4 * nv, 256), 256, 0, s>>>(nt, nv, nb, codes, dm, rho);
        LAPH_LAUNCH_CHECK();
        const c64 *A = reverse ? cf : rho;   // conjugated operand
        const c64 *B = reverse ? rho : cf;
        if (phi != nullptr) {
            const c64 *dphi = (const c64 *)stage_in(ctx, phi, sizeof(c64) * nt * (size_t)nv * nv, "lp:phi", s);
            c64 *Bp = (c64 *)ws_get(ctx, "lp:Bphi", fb);
            phi_apply_kernel<<<dim3(nb, nt), 128, 0, s>>>(nv, nt, 0, dphi, B, Bp);
            LAPH_LAUNCH_CHECK();
            B = Bp;
        }
        Mat4 cs[3];
        const int nc = channel_c(spec->channel, cs);
        W3 w;
        for (int k = 0; k < 3; ++k) w.w[k] = to_w4(cs[k < nc ? k : 0]);
        StagedOut o = stage_out(ctx, loops, sizeof(c64) * nc * nt, "lp:loops");
        loops_kernel<<<nt, 256, 0, s>>>(nt, nv, nb, nc, A, B, w, (c64 *)o.dev);
        LAPH_LAUNCH_CHECK();
        o.commit(s);
        LAPH_CUDA(cudaStreamSynchronize(s));
    });
}

extern "C" int correlate_disconnected(laph_ctx *ctx, const laph_lattice *lat, int t0, int nc, const void *loops1,
                                      const void *loops2, double vev_re, double vev_im, void *corr, void *stream) {
    return guard([&] {
        ctx_activate(ctx);
        LAPH_REQUIRE(lat != nullptr && loops1 != nullptr && loops2 != nullptr && corr != nullptr, "null argument");
        const int nt = lat->nt;
        LAPH_REQUIRE(nt >= 1 && t0 >= 0 && t0 < nt, "t0 out of range");
        LAPH_REQUIRE(nc == 1 || nc == 3, "nc must be 1 (pion, scalar) or 3 (rho)");
        cudaStream_t s = as_stream(stream);
        const c64 *l1 = (const c64 *)stage_in(ctx, loops1, sizeof(c64) * nc * nt, "dc:l1", s);
        const c64 *l2 = (const c64 *)stage_in(ctx, loops2, sizeof(c64) * nc * nt, "dc:l2", s);
        StagedOut o = stage_out(ctx, corr, sizeof(c64) * nt, "dc:corr");
        disconnected_kernel<<<grid_for(nt, 128), 128, 0, s>>>(nt, nc, t0, l1, l2, c64{vev_re, vev_im}, (c64 *)o.dev);
        LAPH_LAUNCH_CHECK();
        o.commit(s);
        LAPH_CUDA(cudaStreamSynchronize(s));
    });
}

extern "C" int laph_displaced_overlaps(laph_ctx *ctx, const laph_lattice *lat, const void *links3d, const void *evecs,
                                       int nv, const int *mom, int len_bar, const int *path_bar, int len,
                                       const int *path, void *phi, void *stream) {
    return guard([&] {
        ctx_activate(ctx);
        Geom g = make_geom(lat);
        LAPH_REQUIRE(nv >= 1 && nv <= 3 * g.V3, "nv out of range");
        LAPH_REQUIRE(mom != nullptr, "momentum is null");
        LAPH_REQUIRE(len_bar >= 0 && len >= 0 && len_bar <= 64 && len <= 64, "paths of 0 .. 64 steps");
        LAPH_REQUIRE((len_bar == 0 || path_bar) && (len == 0 || path), "path is null");
        int d[3] = {0, 0, 0};
        for (int k = 0; k < len_bar; ++k) {
            LAPH_REQUIRE(path_bar[k] != 0 && path_bar[k] >= -3 && path_bar[k] <= 3, "path steps are +-1, +-2, +-3");
            d[abs(path_bar[k]) - 1] += path_bar[k] > 0 ? 1 : -1;
        }
        for (int k = 0; k < len; ++k) {
            LAPH_REQUIRE(path[k] != 0 && path[k] >= -3 && path[k] <= 3, "path steps are +-1, +-2, +-3");
            d[abs(path[k]) - 1] += path[k] > 0 ? 1 : -1;
        }
        LAPH_REQUIRE(g.nt <= 65535, "nt above 65535");
        cudaStream_t s = as_stream(stream);
        const size_t vb = sizeof(c64) * 3 * g.V3 * g.nt * (size_t)nv;
        const c64 *U = (const c64 *)stage_in(ctx, links3d, sizeof(c64) * 36 * g.V, "do:links", s);
        const c64 *V = (const c64 *)stage_in(ctx, evecs, vb, "do:evecs", s);
        c64 *tmp = (c64 *)ws_get(ctx, "do:tmp", vb);
        // D V for a path: the step nearest the field acts first
        // ping-pong between tmp and the result buffer so that the last step (k = 0) writes the result
        auto displaced = [&](int n, const int *steps, const std::string &name) -> const c64 * {
            if (n == 0) return V;
            c64 *dst = (c64 *)ws_get(ctx, "do:" + name, vb);
            const c64 *src = V;
            for (int k = n - 1; k >= 0; --k) {
                c64 *o = (k % 2 == 0) ? dst : tmp;
                disp_step_kernel<<<grid_for((long)g.nt * nv * g.V3, 256), 256, 0, s>>>(g, U, nv, steps[k], src, o);
                LAPH_LAUNCH_CHECK();
                src = o;
            }
            return dst;
        };
        const c64 *Dj = displaced(len_bar, path_bar, "dj");
        const c64 *Dk = displaced(len, path, "dk");
        int *dmom = (int *)ws_get(ctx, "do:mom", sizeof(int) * 3);
        LAPH_CUDA(cudaMemcpyAsync(dmom, mom, sizeof(int) * 3, cudaMemcpyHostToDevice, s));
        c64 *ph = (c64 *)ws_get(ctx, "do:phase", sizeof(c64) * g.V3);
        mom_phase_kernel<<<dim3(grid_for(g.V3, 256), 1), 256, 0, s>>>(g.ns, 1, dmom, ph);
        LAPH_LAUNCH_CHECK();
        // e^{-i p.(d_j + d_k)/2} = e^{-i pi (p . d) / ns}, p . d reduced mod 2 ns
        const int a = (((mom[0] * d[0] + mom[1] * d[1] + mom[2] * d[2]) % (2 * g.ns)) + 2 * g.ns) % (2 * g.ns);
        const double ang = -M_PI * (double)a / g.ns;
        const double cs = std::cos(ang), sn = std::sin(ang);
        StagedOut o = stage_out(ctx, phi, sizeof(c64) * g.nt * (size_t)nv * nv, "do:phi");
        const dim3 grid((nv + OV_T - 1) / OV_T, (nv + OV_T - 1) / OV_T, g.nt);
        overlaps_kernel<<<grid, 256, 0, s>>>(g.V3, nv, g.nt, Dj, Dk, ph, c64{cs, sn}, (c64 *)o.dev);
        LAPH_LAUNCH_CHECK();
        o.commit(s);
        LAPH_CUDA(cudaStreamSynchronize(s));
    });
}
