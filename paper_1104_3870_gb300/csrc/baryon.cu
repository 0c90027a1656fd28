// Baryon functions and correlators in LapH coefficient space (Sec. III: three-quark elemental
// operators, Eq. (baryonfunc) and Eq. (baryoncorr)).
//
// With f = V f-hat for LapH-smeared fields, the spatial sum of a baryon function becomes the
// antisymmetric three-index tensor of each slice (laph_baryon_tensor)
//     T_p(t)[n1][n2][n3] = sum_x e^{-ip.x} eps_abc V_n1(x)_a V_n2(x)_b V_n3(x)_c
// and
//     B^[b1 b2 b3](f1, f2, f3; t) = c_{alpha beta gamma} sum_{n1 n2 n3} T_p(t)[n1][n2][n3]
//                                   f1^[b1](t,alpha,n1) f2^[b2](t,beta,n2) f3^[b3](t,gamma,n3),
// contracted in three steps (n3 with f3, n2 with f2, then n1, the spins and c with f1).  The
// correlator (correlate_baryon) is the sink function of phi_1, phi_2, phi_3 at t_F times the
// conjugate of the signed sum over the six orderings pi of the sources at t_0: source slot s takes
// line pi(s), with the sign of pi, where the flavour of sink quark pi(s) equals that of source slot
// s, the result relabelled so that index k is the dilution index of line k.  All FP64.
#include <cmath>
#include <vector>

#include "gamma_host.cuh"

namespace laph {

namespace {

// T[t][n1][n2][n3]: one block per (n1, n2, t); the cross product w = ph (V_n1 x V_n2) of a chunk of
// sites goes to shared memory, every thread then adds w . V_n3 for its n3.
constexpr int BT_CHUNK = 128;
__global__ void baryon_tensor_kernel(int ns, int nv, int px, int py, int pz, const c64 *__restrict__ V,
                                     c64 *__restrict__ T) {
    __shared__ c64 w[BT_CHUNK][3];
    const int n1 = blockIdx.x, n2 = blockIdx.y, t = blockIdx.z;
    const long v3 = (long)ns * ns * ns;
    const c64 *a = V + ((long)t * nv + n1) * v3 * 3, *b = V + ((long)t * nv + n2) * v3 * 3;
    c64 acc[4] = {{0, 0}, {0, 0}, {0, 0}, {0, 0}};   // n3 = threadIdx.x + k * blockDim.x, k < 4
    for (long x0 = 0; x0 < v3; x0 += BT_CHUNK) {
        for (int e = threadIdx.x; e < BT_CHUNK; e += blockDim.x) {
            const long x = x0 + e;
            if (x < v3) {
                const int xx = (int)(x % ns), yy = (int)((x / ns) % ns), zz = (int)(x / ((long)ns * ns));
                const int arg = ((px * xx + py * yy + pz * zz) % ns + ns) % ns;
                double sn, cs;
                sincospi(-2.0 * arg / ns, &sn, &cs);
                const c64 ph{cs, sn};
                const c64 *u = a + x * 3, *v = b + x * 3;
                w[e][0] = ph * (u[1] * v[2] - u[2] * v[1]);
                w[e][1] = ph * (u[2] * v[0] - u[0] * v[2]);
                w[e][2] = ph * (u[0] * v[1] - u[1] * v[0]);
            } else {
                w[e][0] = w[e][1] = w[e][2] = c64{0, 0};
            }
        }
        __syncthreads();
        const int cnt = (int)((v3 - x0) < BT_CHUNK ? (v3 - x0) : BT_CHUNK);
        for (int k = 0; k < 4; ++k) {
            const int n3 = threadIdx.x + k * blockDim.x;
            if (n3 >= nv) break;
            const c64 *c = V + (((long)t * nv + n3) * v3 + x0) * 3;
            c64 s{0, 0};
            for (int e = 0; e < cnt; ++e) s += w[e][0] * c[3 * e] + w[e][1] * c[3 * e + 1] + w[e][2] * c[3 * e + 2];
            acc[k] += s;
        }
        __syncthreads();
    }
    for (int k = 0; k < 4; ++k) {
        const int n3 = threadIdx.x + k * blockDim.x;
        if (n3 < nv) T[(((long)t * nv + n1) * nv + n2) * nv + n3] = acc[k];
    }
}

// U[t][n1][n2][b3][g] = sum_n3 T[tT][n1][n2][n3] f3[b3][t][g][n3]   (tT = t, or t1 for single-slice operands)
__global__ void bar_u_kernel(int nv, int nb, int ntf, int t1, const c64 *__restrict__ T, const c64 *__restrict__ f3,
                             c64 *__restrict__ U) {
    const int n12 = blockIdx.x, t = blockIdx.y;
    const int tT = ntf == 1 ? t1 : t;
    const c64 *tr = T + ((long)tT * nv * nv + n12) * nv;
    for (int e = threadIdx.x; e < nb * 4; e += blockDim.x) {
        const int b3 = e / 4, g = e % 4;
        const c64 *f = f3 + (((long)b3 * ntf + t) * 4 + g) * nv;
        c64 s{0, 0};
        for (int n3 = 0; n3 < nv; ++n3) s += tr[n3] * f[n3];
        U[(((long)t * nv * nv + n12) * nb + b3) * 4 + g] = s;
    }
}

// W[t][n1][b2][b3][be][g] = sum_n2 U[t][n1][n2][b3][g] f2[b2][t][be][n2]
__global__ void bar_w_kernel(int nv, int nb, int ntf, const c64 *__restrict__ U, const c64 *__restrict__ f2,
                             c64 *__restrict__ W) {
    const int n1 = blockIdx.x, t = blockIdx.y, b2 = blockIdx.z;
    for (int e = threadIdx.x; e < nb * 16; e += blockDim.x) {
        const int b3 = e / 16, be = (e / 4) % 4, g = e % 4;
        const c64 *f = f2 + (((long)b2 * ntf + t) * 4 + be) * nv;
        c64 s{0, 0};
        for (int n2 = 0; n2 < nv; ++n2) s += U[((((long)t * nv + n1) * nv + n2) * nb + b3) * 4 + g] * f[n2];
        W[((((long)t * nv + n1) * nb + b2) * nb + b3) * 16 + be * 4 + g] = s;
    }
}

struct C64x64 {
    c64 c[64];   // c[alpha][beta][gamma]
};

// B[t][b1][b2][b3] = sum_{n1 al be g} c[al][be][g] f1[b1][t][al][n1] W[t][n1][b2][b3][be][g]
__global__ void bar_b_kernel(int nv, int nb, int ntf, C64x64 c, const c64 *__restrict__ f1, const c64 *__restrict__ W,
                             c64 *__restrict__ B) {
    const int b1 = blockIdx.x, t = blockIdx.y, b2 = blockIdx.z;
    for (int b3 = threadIdx.x; b3 < nb; b3 += blockDim.x) {
        c64 s{0, 0};
        for (int n1 = 0; n1 < nv; ++n1) {
            const c64 *w = W + ((((long)t * nv + n1) * nb + b2) * nb + b3) * 16;
            for (int al = 0; al < 4; ++al) {
                const c64 f = f1[(((long)b1 * ntf + t) * 4 + al) * nv + n1];
                c64 inner{0, 0};
                for (int k = 0; k < 16; ++k) inner += c.c[al * 16 + k] * w[k];
                s += f * inner;
            }
        }
        B[(((long)t * nb + b1) * nb + b2) * nb + b3] = s;
    }
}

// src[j0][j1][j2] += sgn * f[j_p0][j_p1][j_p2] (slot s of f carries line p_s's dilution index)
__global__ void bar_relabel_kernel(int nb, int p0, int p1, int p2, double sgn, const c64 *__restrict__ f,
                                   c64 *__restrict__ src) {
    const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (long)nb * nb * nb) return;
    const int j[3] = {(int)(e / ((long)nb * nb)), (int)((e / nb) % nb), (int)(e % nb)};
    src[e] += sgn * f[((long)j[p0] * nb + j[p1]) * nb + j[p2]];
}

// corr[dt] = sum_b snk[(t0 + dt) mod nt][b] conj(src[b])
__global__ void bar_corr_kernel(int nt, long nb3, int t0, const c64 *__restrict__ snk, const c64 *__restrict__ src,
                                c64 *__restrict__ corr) {
    __shared__ c64 sm[256];
    const int dt = blockIdx.x;
    const long t = (t0 + dt) % nt;
    c64 acc{0, 0};
    for (long e = threadIdx.x; e < nb3; e += blockDim.x) acc += snk[t * nb3 + e] * conj(src[e]);
    sm[threadIdx.x] = acc;
    __syncthreads();
    for (int st = blockDim.x / 2; st > 0; st >>= 1) {
        if ((int)threadIdx.x < st) sm[threadIdx.x] += sm[threadIdx.x + st];
        __syncthreads();
    }
    if (threadIdx.x == 0) corr[dt] = sm[0];
}

}  // namespace

}  // namespace laph

using namespace laph;

extern "C" int laph_baryon_tensor(laph_ctx *ctx, const laph_lattice *lat, const void *evecs, int nv, const int *mom,
                                  void *T, void *stream) {
    return guard([&] {
        ctx_activate(ctx);
        Geom g = make_geom(lat);
        LAPH_REQUIRE(nv >= 1 && nv <= 512 && nv <= 3 * g.V3, "nv out of range (1 .. 512)");
        LAPH_REQUIRE(mom != nullptr && T != nullptr, "null argument");
        LAPH_REQUIRE(g.nt <= 65535, "nt above 65535");
        cudaStream_t s = as_stream(stream);
        const c64 *V = (const c64 *)stage_in(ctx, evecs, sizeof(c64) * 3 * g.V3 * g.nt * (size_t)nv, "bt:evecs", s);
        StagedOut o = stage_out(ctx, T, sizeof(c64) * g.nt * (size_t)nv * nv * nv, "bt:T");
        baryon_tensor_kernel<<<dim3(nv, nv, g.nt), 128, 0, s>>>(g.ns, nv, mom[0], mom[1], mom[2], V, (c64 *)o.dev);
        LAPH_LAUNCH_CHECK();
        o.commit(s);
        LAPH_CUDA(cudaStreamSynchronize(s));
    });
}

extern "C" int correlate_baryon(laph_ctx *ctx, const laph_lattice *lat, const laph_baryon_spec *spec,
                                const void *const *coef, const uint8_t *const *noise, const void *T, void *corr,
                                void *stream) {
    return guard([&] {
        ctx_activate(ctx);
        LAPH_REQUIRE(lat != nullptr && spec != nullptr && coef != nullptr && noise != nullptr && T != nullptr &&
                         corr != nullptr,
                     "null argument");
        const int nt = lat->nt, nv = spec->nv, nb = spec->nb, t0 = spec->t0;
        LAPH_REQUIRE(nt >= 1 && nv >= 1 && nb >= 1 && nb <= 1024, "bad sizes (1 <= nb <= 1024)");
        LAPH_REQUIRE(t0 >= 0 && t0 < nt, "t0 out of range");
        LAPH_REQUIRE(spec->b_list != nullptr && spec->c_snk != nullptr && spec->c_src != nullptr, "null spec array");
        cudaStream_t s = as_stream(stream);
        std::vector<uint8_t> m = dilution_masks(spec->dil, nt, nv, spec->b_list, nb);
        uint8_t *dm = (uint8_t *)ws_get(ctx, "bc:mask", m.size());
        LAPH_CUDA(cudaMemcpyAsync(dm, m.data(), m.size(), cudaMemcpyHostToDevice, s));
        const c64 *dT = (const c64 *)stage_in(ctx, T, sizeof(c64) * nt * (size_t)nv * nv * nv, "bc:T", s);
        const c64 *cf[3];
        c64 *rho[3];
        for (int k = 0; k < 3; ++k) {
            LAPH_REQUIRE(coef[k] != nullptr && noise[k] != nullptr, "line arrays are null");
            const std::string id = std::to_string(k);
            cf[k] = (const c64 *)stage_in(ctx, coef[k], sizeof(c64) * (size_t)nb * nt * 4 * nv, "bc:coef" + id, s);
            const uint8_t *codes = (const uint8_t *)stage_in(ctx, noise[k], (size_t)nt * 4 * nv, "bc:noise" + id, s);
            rho[k] = (c64 *)ws_get(ctx, "bc:rho" + id, sizeof(c64) * nb * 4 * nv);
            rho_at_t0_kernel<<<grid_for((long)nb * 4 * nv, 256), 256, 0, s>>>(nt, nv, nb, t0, codes, dm, rho[k]);
            LAPH_LAUNCH_CHECK();
        }
        C64x64 csnk, csrc;
        for (int i = 0; i < 64; ++i) {
            csnk.c[i] = c64{spec->c_snk[2 * i], spec->c_snk[2 * i + 1]};
            csrc.c[i] = c64{spec->c_src[2 * i], spec->c_src[2 * i + 1]};
        }
        const long nb3 = (long)nb * nb * nb;
        c64 *U = (c64 *)ws_get(ctx, "bc:U", sizeof(c64) * nt * (size_t)nv * nv * nb * 4);
        c64 *W = (c64 *)ws_get(ctx, "bc:W", sizeof(c64) * nt * (size_t)nv * nb * nb * 16);
        c64 *snk = (c64 *)ws_get(ctx, "bc:snk", sizeof(c64) * nt * nb3);
        c64 *fsrc = (c64 *)ws_get(ctx, "bc:fsrc", sizeof(c64) * nb3);
        c64 *src = (c64 *)ws_get(ctx, "bc:src", sizeof(c64) * nb3);
        // one baryon function: operands [nb][ntf][4][nv] (ntf = nt, or 1 at t1)
        auto function = [&](const c64 *f1, const c64 *f2, const c64 *f3, int ntf, int t1, const C64x64 &c, c64 *B) {
            bar_u_kernel<<<dim3(nv * nv, ntf), 128, 0, s>>>(nv, nb, ntf, t1, dT, f3, U);
            LAPH_LAUNCH_CHECK();
            bar_w_kernel<<<dim3(nv, ntf, nb), 128, 0, s>>>(nv, nb, ntf, U, f2, W);
            LAPH_LAUNCH_CHECK();
            bar_b_kernel<<<dim3(nb, ntf, nb), 128, 0, s>>>(nv, nb, ntf, c, f1, W, B);
            LAPH_LAUNCH_CHECK();
        };
        function(cf[0], cf[1], cf[2], nt, 0, csnk, snk);
        LAPH_CUDA(cudaMemsetAsync(src, 0, sizeof(c64) * nb3, s));
        const int perms[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
        const double sgn[6] = {1, -1, -1, 1, 1, -1};
        for (int q = 0; q < 6; ++q) {
            const int *p = perms[q];
            bool ok = true;
            for (int sl = 0; sl < 3; ++sl) ok &= spec->flav_snk[p[sl]] == spec->flav_src[sl];
            if (!ok) continue;
            function(rho[p[0]], rho[p[1]], rho[p[2]], 1, t0, csrc, fsrc);
            bar_relabel_kernel<<<grid_for(nb3, 256), 256, 0, s>>>(nb, p[0], p[1], p[2], sgn[q], fsrc, src);
            LAPH_LAUNCH_CHECK();
        }
        StagedOut o = stage_out(ctx, corr, sizeof(c64) * nt, "bc:corr");
        bar_corr_kernel<<<nt, 256, 0, s>>>(nt, nb3, t0, snk, src, (c64 *)o.dev);
        LAPH_LAUNCH_CHECK();
        o.commit(s);
        LAPH_CUDA(cudaStreamSynchronize(s));
    });
}
