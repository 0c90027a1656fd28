// Gauge preparation on the GPU: stout smearing (Sec. II), the clover field
// strength and its chiral 6x6 blocks with their inverses, and the packing of
// links into the even-odd layouts of the Dirac operator.
#include <cmath>

#include "dirac.cuh"
#include "su3.cuh"

namespace laph {

// --------------------------------------------------------------------------
// Stout step.  One thread per (site, mu):
//   C = rho sum_{nu != mu} [U_nu(x) U_mu(x+nu) U_nu(x+mu)^dag + U_nu(x-nu)^dag U_mu(x-nu) U_nu(x-nu+mu)]
//   Omega = C U_mu^dag;  A = Omega^dag - Omega;  iQ = -A/2 + Tr(A)/6
//   U_mu <- exp(iQ) U_mu
// Reads `in`, writes `out` (all links of a step are updated simultaneously).
// --------------------------------------------------------------------------
__global__ void stout_kernel(Geom g, const c64 *__restrict__ in, c64 *__restrict__ out, double rho, int nmu) {
    long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= g.V * nmu) return;
    long s = idx / nmu;
    int mu = (int)(idx % nmu);
    int c[4];
    site_coords(g, s, c);
    int dims[4] = {g.ns, g.ns, g.ns, g.nt};
    auto shift = [&](const int *cc, int d, int step, int *o) {
        o[0] = cc[0]; o[1] = cc[1]; o[2] = cc[2]; o[3] = cc[3];
        o[d] = (cc[d] + step + dims[d]) % dims[d];
    };
    auto link = [&](const int *cc, int d) { return m3_load(in + (site_of(g, cc) * 4 + d) * 9); };
    M3 umu = link(c, mu);
    M3 csum = m3_zero();
    for (int nu = 0; nu < nmu; ++nu) {
        if (nu == mu) continue;
        int xp_nu[4], xp_mu[4], xm_nu[4], xm_nu_p_mu[4];
        shift(c, nu, 1, xp_nu);
        shift(c, mu, 1, xp_mu);
        shift(c, nu, -1, xm_nu);
        shift(xm_nu, mu, 1, xm_nu_p_mu);
        // upper staple
        M3 a = m3_mul(link(c, nu), link(xp_nu, mu));
        m3_add(csum, m3_mul_nd(a, link(xp_mu, nu)));
        // lower staple
        M3 unu_m = link(xm_nu, nu);
        M3 b = m3_mul_dn(unu_m, link(xm_nu, mu));
        m3_add(csum, m3_mul(b, link(xm_nu_p_mu, nu)));
    }
    M3 om = m3_scale(rho, m3_mul_nd(csum, umu));
    M3 x;
    double tr_im = 0.0;   // Tr(A) is purely imaginary for A anti-Hermitian
#pragma unroll
    for (int i = 0; i < 3; ++i) tr_im += -2.0 * om.m[i][i].im;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            c64 a = conj(om.m[j][i]) - om.m[i][j];   // A = Omega^dag - Omega
            x.m[i][j] = -0.5 * a;
        }
#pragma unroll
    for (int i = 0; i < 3; ++i) x.m[i][i].im += tr_im / 6.0;
    M3 e = m3_expm(x);
    m3_store(out + (s * 4 + mu) * 9, m3_mul(e, umu));
}

__global__ void copy_time_links(Geom g, const c64 *__restrict__ in, c64 *__restrict__ out) {
    long s = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= g.V) return;
#pragma unroll
    for (int k = 0; k < 9; ++k) out[(s * 4 + 3) * 9 + k] = in[(s * 4 + 3) * 9 + k];
}

// --------------------------------------------------------------------------
// Clover construction.  sigma_{mu nu} blocks: chirality h (spins 2h, 2h+1).
// Planes ordered (0,1),(0,2),(0,3),(1,2),(1,3),(2,3).
// --------------------------------------------------------------------------
__constant__ c64 c_sigma[6][2][2][2];
__constant__ double c_wpl[6];

static void upload_sigma(double xi, cudaStream_t s) {
    // chiral-basis gamma matrices, gamma_mu = [[0, G], [G^dag, 0]], G_k = -i sigma_k, G_4 = 1
    const c64 I{0, 1}, O{0, 0}, P{1, 0}, Mi{0, -1}, M1{-1, 0};
    c64 G[4][2][2] = {
        {{O, Mi}, {Mi, O}},     // -i sigma_1
        {{O, M1}, {P, O}},      // -i sigma_2
        {{Mi, O}, {O, I}},      // -i sigma_3
        {{P, O}, {O, P}},       // 1
    };
    c64 gam[4][4][4];
    for (int m = 0; m < 4; ++m)
        for (int i = 0; i < 4; ++i)
            for (int j = 0; j < 4; ++j) gam[m][i][j] = O;
    for (int m = 0; m < 4; ++m)
        for (int i = 0; i < 2; ++i)
            for (int j = 0; j < 2; ++j) {
                gam[m][i][2 + j] = G[m][i][j];
                gam[m][2 + i][j] = conj(G[m][j][i]);
            }
    c64 sig[6][2][2][2];
    double w[6];
    int pl = 0;
    for (int mu = 0; mu < 4; ++mu)
        for (int nu = mu + 1; nu < 4; ++nu, ++pl) {
            w[pl] = (mu == 3 || nu == 3) ? 0.5 * (1.0 + 1.0 / xi) : 1.0 / xi;
            c64 full[4][4];
            for (int i = 0; i < 4; ++i)
                for (int j = 0; j < 4; ++j) {
                    c64 acc = O;
                    for (int k = 0; k < 4; ++k) acc += gam[mu][i][k] * gam[nu][k][j] - gam[nu][i][k] * gam[mu][k][j];
                    full[i][j] = c64{0.0, 0.5} * acc;    // (i/2)[g_mu, g_nu]
                }
            for (int h = 0; h < 2; ++h)
                for (int a = 0; a < 2; ++a)
                    for (int b = 0; b < 2; ++b) sig[pl][h][a][b] = full[2 * h + a][2 * h + b];
        }
    LAPH_CUDA(cudaMemcpyToSymbolAsync(c_sigma, sig, sizeof(sig), 0, cudaMemcpyHostToDevice, s));
    LAPH_CUDA(cudaMemcpyToSymbolAsync(c_wpl, w, sizeof(w), 0, cudaMemcpyHostToDevice, s));
}

__device__ __forceinline__ int herm_off(int i, int j) { return 6 + 2 * (i * (i - 1) / 2 + j); }  // i > j

__device__ void pack_herm(double *dst, const c64 b[6][6]) {
    for (int i = 0; i < 6; ++i) dst[i] = b[i][i].re;
    for (int i = 1; i < 6; ++i)
        for (int j = 0; j < i; ++j) {
            // store the Hermitian average of the two triangles
            c64 v = 0.5 * (b[i][j] + conj(b[j][i]));
            dst[herm_off(i, j)] = v.re;
            dst[herm_off(i, j) + 1] = v.im;
        }
}

// Gauss-Jordan inverse with partial pivoting of a 6x6 complex matrix.
__device__ void inv6(const c64 a_in[6][6], c64 inv[6][6]) {
    c64 a[6][6];
    for (int i = 0; i < 6; ++i)
        for (int j = 0; j < 6; ++j) {
            a[i][j] = a_in[i][j];
            inv[i][j] = c64{i == j ? 1.0 : 0.0, 0.0};
        }
    for (int col = 0; col < 6; ++col) {
        int piv = col;
        double best = norm2(a[col][col]);
        for (int r = col + 1; r < 6; ++r)
            if (norm2(a[r][col]) > best) { best = norm2(a[r][col]); piv = r; }
        if (piv != col)
            for (int j = 0; j < 6; ++j) {
                c64 t = a[col][j]; a[col][j] = a[piv][j]; a[piv][j] = t;
                t = inv[col][j]; inv[col][j] = inv[piv][j]; inv[piv][j] = t;
            }
        c64 d = a[col][col];
        double dn = norm2(d);
        c64 di{d.re / dn, -d.im / dn};
        for (int j = 0; j < 6; ++j) { a[col][j] = a[col][j] * di; inv[col][j] = inv[col][j] * di; }
        for (int r = 0; r < 6; ++r) {
            if (r == col) continue;
            c64 f = a[r][col];
            for (int j = 0; j < 6; ++j) { a[r][j] -= f * a[col][j]; inv[r][j] -= f * inv[col][j]; }
        }
    }
}

// One thread per site: F_{mu nu} for the six planes, the two chiral blocks of
// A = diag - (csw/2) sum w_pl sigma_pl (x) F_pl, their inverses; writes packed
// FP64 A, FP64 A^{-1}, FP32 A^{-1} (and BF16 A^{-1} if requested) in even-odd order.
__global__ void clover_kernel(Geom g, const c64 *__restrict__ U, double diag, double csw, double *clov64,
                              double *cinv64, float *cinv32, __nv_bfloat16 *cinv16) {
    long s = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= g.V) return;
    int c[4];
    site_coords(g, s, c);
    int dims[4] = {g.ns, g.ns, g.ns, g.nt};
    auto sh = [&](const int *cc, int d, int step, int *o) {
        o[0] = cc[0]; o[1] = cc[1]; o[2] = cc[2]; o[3] = cc[3];
        o[d] = (cc[d] + step + dims[d]) % dims[d];
    };
    auto link = [&](const int *cc, int d) { return m3_load(U + (site_of(g, cc) * 4 + d) * 9); };
    c64 blk[2][6][6];
    for (int h = 0; h < 2; ++h)
        for (int i = 0; i < 6; ++i)
            for (int j = 0; j < 6; ++j) blk[h][i][j] = c64{i == j ? diag : 0.0, 0.0};
    int pl = 0;
    for (int mu = 0; mu < 4; ++mu)
        for (int nu = mu + 1; nu < 4; ++nu, ++pl) {
            int xpm[4], xpn[4], xmm[4], xmn[4], xmm_pn[4], xmm_mn[4], xmn_pm[4];
            sh(c, mu, 1, xpm);
            sh(c, nu, 1, xpn);
            sh(c, mu, -1, xmm);
            sh(c, nu, -1, xmn);
            sh(xmm, nu, 1, xmm_pn);
            sh(xmm, nu, -1, xmm_mn);
            sh(xmn, mu, 1, xmn_pm);
            M3 umu = link(c, mu), unu = link(c, nu);
            // leaf 1: U_mu(x) U_nu(x+mu) U_mu(x+nu)^dag U_nu(x)^dag
            M3 q = m3_mul_nd(m3_mul_nd(m3_mul(umu, link(xpm, nu)), link(xpn, mu)), unu);
            // leaf 2: U_nu(x) U_mu(x-mu+nu)^dag U_nu(x-mu)^dag U_mu(x-mu)
            M3 umu_m = link(xmm, mu);
            m3_add(q, m3_mul(m3_mul_nd(m3_mul_nd(unu, link(xmm_pn, mu)), link(xmm, nu)), umu_m));
            // leaf 3: U_mu(x-mu)^dag U_nu(x-mu-nu)^dag U_mu(x-mu-nu) U_nu(x-nu)
            M3 unu_n = link(xmn, nu);
            m3_add(q, m3_mul(m3_mul_dn(m3_mul(link(xmm_mn, nu), umu_m), link(xmm_mn, mu)), unu_n));
            // leaf 4: U_nu(x-nu)^dag U_mu(x-nu) U_nu(x-nu+mu) U_mu(x)^dag
            m3_add(q, m3_mul_nd(m3_mul(m3_mul_dn(unu_n, link(xmn, mu)), link(xmn_pm, nu)), umu));
            // F = (Q - Q^dag)/(8i), traceless
            M3 f;
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) {
                    c64 d = q.m[i][j] - conj(q.m[j][i]);
                    f.m[i][j] = c64{d.im / 8.0, -d.re / 8.0};
                }
            double tr = (f.m[0][0].re + f.m[1][1].re + f.m[2][2].re) / 3.0;
            for (int i = 0; i < 3; ++i) { f.m[i][i].re -= tr; f.m[i][i].im = 0.0; }
            double coef = -0.5 * csw * c_wpl[pl];
            for (int h = 0; h < 2; ++h)
                for (int a = 0; a < 2; ++a)
                    for (int b = 0; b < 2; ++b) {
                        c64 sg = c_sigma[pl][h][a][b];
                        if (sg.re == 0.0 && sg.im == 0.0) continue;
                        for (int i = 0; i < 3; ++i)
                            for (int j = 0; j < 3; ++j) blk[h][a * 3 + i][b * 3 + j] += coef * (sg * f.m[i][j]);
                    }
        }
    int p = parity_of(c);
    long cb = s >> 1;
    for (int h = 0; h < 2; ++h) {
        long off = (((long)p * g.Vh + cb) * 2 + h) * CLOV_BLOCK;
        pack_herm(clov64 + off, blk[h]);
        c64 inv[6][6];
        inv6(blk[h], inv);
        pack_herm(cinv64 + off, inv);
        for (int k = 0; k < CLOV_BLOCK; ++k) {
            cinv32[off + k] = (float)cinv64[off + k];
            if (cinv16) cinv16[off + k] = __double2bfloat16(cinv64[off + k]);
        }
    }
}

// Links into the even-odd layouts.
__global__ void pack_links_kernel(Geom g, const c64 *__restrict__ U, c64 *L64, float4 *L32,
                                  __nv_bfloat162 *L16) {
    long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= g.V * 4) return;
    long s = idx >> 2;
    int mu = (int)(idx & 3);
    int c[4];
    site_coords(g, s, c);
    int p = parity_of(c);
    long cb = s >> 1;
    long o = ((long)p * 4 + mu) * g.Vh + cb;
    const c64 *u = U + (s * 4 + mu) * 9;
#pragma unroll
    for (int k = 0; k < 9; ++k) L64[o * 9 + k] = u[k];
    float r[12];
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        r[2 * k] = (float)u[k].re;
        r[2 * k + 1] = (float)u[k].im;
    }
    L32[o * 3 + 0] = make_float4(r[0], r[1], r[2], r[3]);
    L32[o * 3 + 1] = make_float4(r[4], r[5], r[6], r[7]);
    L32[o * 3 + 2] = make_float4(r[8], r[9], r[10], r[11]);
    if (L16) {
#pragma unroll
        for (int k = 0; k < 6; ++k) L16[o * 6 + k] = __floats2bfloat162_rn(r[2 * k], r[2 * k + 1]);
    }
}

DiracOp prepare_dirac(laph_ctx *ctx, const Geom &g, const c64 *links, double m0, double csw, double xi,
                      cudaStream_t s, bool need_bf16) {
    LAPH_REQUIRE(xi > 0.0, "xi must be positive");
    DiracOp op;
    op.g = g;
    op.m0 = m0;
    op.csw = csw;
    op.xi = xi;
    double w[4] = {1.0 / xi, 1.0 / xi, 1.0 / xi, 1.0};
    for (int mu = 0; mu < 4; ++mu) op.hw[mu] = -0.5 * w[mu];
    op.L64 = (c64 *)ws_get(ctx, "dirac:L64", sizeof(c64) * 9 * 8 * g.Vh);
    op.L32 = (float4 *)ws_get(ctx, "dirac:L32", sizeof(float4) * 3 * 8 * g.Vh);
    op.clov64 = (double *)ws_get(ctx, "dirac:clov64", sizeof(double) * CLOV_BLOCK * 4 * g.Vh);
    op.cinv64 = (double *)ws_get(ctx, "dirac:cinv64", sizeof(double) * CLOV_BLOCK * 4 * g.Vh);
    op.cinv32 = (float *)ws_get(ctx, "dirac:cinv32", sizeof(float) * CLOV_BLOCK * 4 * g.Vh);
    if (need_bf16) {
        op.L16 = (__nv_bfloat162 *)ws_get(ctx, "dirac:L16", sizeof(__nv_bfloat162) * 6 * 8 * g.Vh);
        op.cinv16 = (__nv_bfloat16 *)ws_get(ctx, "dirac:cinv16", sizeof(__nv_bfloat16) * CLOV_BLOCK * 4 * g.Vh);
    }
    upload_sigma(xi, s);
    pack_links_kernel<<<grid_for(g.V * 4, 256), 256, 0, s>>>(g, links, op.L64, op.L32, op.L16);
    LAPH_LAUNCH_CHECK();
    double diag = m0 + w[0] + w[1] + w[2] + w[3];
    clover_kernel<<<grid_for(g.V, 64), 64, 0, s>>>(g, links, diag, csw, op.clov64, op.cinv64, op.cinv32, op.cinv16);
    LAPH_LAUNCH_CHECK();
    prepare_f32_operands(ctx, op, s);
    return op;
}

}  // namespace laph

using namespace laph;

extern "C" int laph_stout_smear(laph_ctx *ctx, const laph_lattice *lat, void *links, double rho, int nsteps,
                                int spatial_only, void *stream) {
    return guard([&] {
        ctx_activate(ctx);
        Geom g = make_geom(lat);
        LAPH_REQUIRE(nsteps >= 0, "nsteps must be >= 0");
        cudaStream_t s = as_stream(stream);
        size_t bytes = sizeof(c64) * 9 * 4 * g.V;
        StagedOut out = stage_out(ctx, links, bytes, "stout_links");
        const void *in = stage_in(ctx, links, bytes, "stout_links_in", s);
        c64 *a = (c64 *)ws_get(ctx, "stout:a", bytes);
        c64 *b = (c64 *)ws_get(ctx, "stout:b", bytes);
        LAPH_CUDA(cudaMemcpyAsync(a, in, bytes, cudaMemcpyDeviceToDevice, s));
        int nmu = spatial_only ? 3 : 4;
        for (int k = 0; k < nsteps; ++k) {
            if (spatial_only) {
                copy_time_links<<<grid_for(g.V, 256), 256, 0, s>>>(g, a, b);
                LAPH_LAUNCH_CHECK();
            }
            stout_kernel<<<grid_for(g.V * nmu, 128), 128, 0, s>>>(g, a, b, rho, nmu);
            LAPH_LAUNCH_CHECK();
            std::swap(a, b);
        }
        LAPH_CUDA(cudaMemcpyAsync(out.dev, a, bytes, cudaMemcpyDeviceToDevice, s));
        out.commit(s);
    });
}
