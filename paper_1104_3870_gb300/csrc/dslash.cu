// Even-odd Wilson-clover stencil on many right-hand sides.
//
// D psi(x) = -1/2 sum_mu w_mu [ (1 - gamma_mu) U_mu(x) psi(x+mu) + (1 + gamma_mu) U_mu(x-mu)^dag psi(x-mu) ]
// with the antiperiodic time boundary applied as a sign on hops across t = nt-1 <-> 0.
// The hop kernel computes D_{p pbar} on one parity and fuses the diagonal part:
// the clover inverse (Schur-complement solver) or the clover itself (residuals).
//
// Chiral basis: gamma_mu = [[0, G_mu], [G_mu^dag, 0]] with G_k = -i sigma_k and
// G_4 = 1, so (1 -+ gamma_mu) psi is fixed by the two-spin half h = u -+ G d
// (u = spins 0,1; d = spins 2,3): upper = h, lower = -+ G^dag h.  Only h is
// multiplied by the link (two colour vectors instead of four).
#include "blas.cuh"
#include "dirac.cuh"

namespace laph {

// ------------------------------------------------------------ link loading
template <typename T>
struct LinkLoad;

template <>
struct LinkLoad<double> {
    static __device__ __forceinline__ void load(const DiracOp &op, int p, int mu, long cb, c64 u[3][3]) {
        const c64 *q = op.L64 + (((long)p * 4 + mu) * op.g.Vh + cb) * 9;
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) u[i][j] = q[i * 3 + j];
    }
};

template <typename T>
__device__ __forceinline__ void third_row(cpx<T> u[3][3]) {
    // row2 = conj(row0 x row1)
    u[2][0] = conj(u[0][1] * u[1][2] - u[0][2] * u[1][1]);
    u[2][1] = conj(u[0][2] * u[1][0] - u[0][0] * u[1][2]);
    u[2][2] = conj(u[0][0] * u[1][1] - u[0][1] * u[1][0]);
}

template <>
struct LinkLoad<float> {
    static __device__ __forceinline__ void load(const DiracOp &op, int p, int mu, long cb, c32 u[3][3]) {
        const float4 *q = op.L32 + (((long)p * 4 + mu) * op.g.Vh + cb) * 3;
        float4 a = __ldg(q), b = __ldg(q + 1), c = __ldg(q + 2);
        u[0][0] = {a.x, a.y};
        u[0][1] = {a.z, a.w};
        u[0][2] = {b.x, b.y};
        u[1][0] = {b.z, b.w};
        u[1][1] = {c.x, c.y};
        u[1][2] = {c.z, c.w};
        third_row(u);
    }
};

// ------------------------------------------------------------ spin algebra
// G d for the lower half (d0, d1) of a spinor; colour component c.
template <typename T>
__device__ __forceinline__ void G_mul(int mu, cpx<T> d0, cpx<T> d1, cpx<T> &o0, cpx<T> &o1) {
    switch (mu) {
        case 0: o0 = -times_i(d1); o1 = -times_i(d0); break;       // -i sigma_1
        case 1: o0 = -d1; o1 = d0; break;                           // -i sigma_2
        case 2: o0 = -times_i(d0); o1 = times_i(d1); break;        // -i sigma_3
        default: o0 = d0; o1 = d1; break;                           // 1
    }
}
// G^dag h
template <typename T>
__device__ __forceinline__ void Gd_mul(int mu, cpx<T> h0, cpx<T> h1, cpx<T> &o0, cpx<T> &o1) {
    switch (mu) {
        case 0: o0 = times_i(h1); o1 = times_i(h0); break;
        case 1: o0 = h1; o1 = -h0; break;
        case 2: o0 = times_i(h0); o1 = -times_i(h1); break;
        default: o0 = h0; o1 = h1; break;
    }
}

// acc += coef * (1 - gamma_mu) U psi      (fwd)
// acc += coef * (1 + gamma_mu) U^dag psi  (!fwd)
template <typename T>
__device__ __forceinline__ void hop_dir(int mu, bool fwd, cpx<T> acc[12], const cpx<T> psi[12], const cpx<T> u[3][3],
                                        T coef) {
    cpx<T> h0[3], h1[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        cpx<T> g0, g1;
        G_mul(mu, psi[6 + c], psi[9 + c], g0, g1);
        if (fwd) {
            h0[c] = psi[c] - g0;
            h1[c] = psi[3 + c] - g1;
        } else {
            h0[c] = psi[c] + g0;
            h1[c] = psi[3 + c] + g1;
        }
    }
    cpx<T> k0[3], k1[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        cpx<T> s0{0, 0}, s1{0, 0};
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            if (fwd) {
                s0 += u[a][b] * h0[b];
                s1 += u[a][b] * h1[b];
            } else {
                s0 += cmul_conj(u[b][a], h0[b]);
                s1 += cmul_conj(u[b][a], h1[b]);
            }
        }
        k0[a] = coef * s0;
        k1[a] = coef * s1;
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        cpx<T> l0, l1;
        Gd_mul(mu, k0[c], k1[c], l0, l1);
        acc[c] += k0[c];
        acc[3 + c] += k1[c];
        if (fwd) {
            acc[6 + c] -= l0;
            acc[9 + c] -= l1;
        } else {
            acc[6 + c] += l0;
            acc[9 + c] += l1;
        }
    }
}

// y = B x for a packed Hermitian 6x6 block (6 real diagonals, then the strictly lower part row-major).
template <typename T, typename S>
__device__ __forceinline__ void herm6(const S *__restrict__ b, const cpx<T> x[6], cpx<T> y[6]) {
#pragma unroll
    for (int i = 0; i < 6; ++i) y[i] = (T)b[i] * x[i];
    int o = 6;
#pragma unroll
    for (int i = 1; i < 6; ++i)
#pragma unroll
        for (int j = 0; j < i; ++j) {
            cpx<T> l{(T)b[o], (T)b[o + 1]};
            o += 2;
            y[i] += l * x[j];
            y[j] += cmul_conj(l, x[i]);
        }
}

template <typename T>
struct ClovPtr;
template <>
struct ClovPtr<double> {
    static __device__ __forceinline__ const double *inv(const DiracOp &op) { return op.cinv64; }
};
template <>
struct ClovPtr<float> {
    static __device__ __forceinline__ const float *inv(const DiracOp &op) { return op.cinv32; }
};

template <typename T, int MODE>
__global__ void __launch_bounds__(256) hop_kernel(DiracOp op, int p, cpx<T> *__restrict__ out,
                                                  const cpx<T> *__restrict__ in, const cpx<T> *__restrict__ z,
                                                  const cpx<T> *__restrict__ xp, int nr) {
    const Geom &g = op.g;
    long tid = (long)blockIdx.x * blockDim.x + threadIdx.x;
    long cb = tid / nr;
    int r = (int)(tid - cb * nr);
    if (cb >= g.Vh) return;
    // neighbours from the table of prepare_f32_operands: forward mu then backward mu, ~j marks
    // a hop across the time boundary (antiperiodic sign)
    const int *nb8 = op.nbr + ((long)p * g.Vh + cb) * 8;
    cpx<T> acc[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) acc[k] = {0, 0};
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) {
        cpx<T> u[3][3], psi[12];
        // forward neighbour
        {
            int j = __ldg(nb8 + mu);
            T coef = j < 0 ? -(T)op.hw[mu] : (T)op.hw[mu];
            long nb = j < 0 ? ~j : j;
            const cpx<T> *src = in + nb * 12 * nr + r;
#pragma unroll
            for (int k = 0; k < 12; ++k) psi[k] = src[(long)k * nr];
            LinkLoad<T>::load(op, p, mu, cb, u);
            hop_dir<T>(mu, true, acc, psi, u, coef);
        }
        // backward neighbour
        {
            int j = __ldg(nb8 + 4 + mu);
            T coef = j < 0 ? -(T)op.hw[mu] : (T)op.hw[mu];
            long nb = j < 0 ? ~j : j;
            const cpx<T> *src = in + nb * 12 * nr + r;
#pragma unroll
            for (int k = 0; k < 12; ++k) psi[k] = src[(long)k * nr];
            LinkLoad<T>::load(op, 1 - p, mu, nb, u);
            hop_dir<T>(mu, false, acc, psi, u, coef);
        }
    }
    cpx<T> res[12];
    if (MODE == HOP_CLOVINV || MODE == HOP_CLOVINV_XPAY) {
        const T *ci = ClovPtr<T>::inv(op) + ((long)p * g.Vh + cb) * 2 * CLOV_BLOCK;
        herm6<T, T>(ci, acc, res);
        herm6<T, T>(ci + CLOV_BLOCK, acc + 6, res + 6);
        if (MODE == HOP_CLOVINV_XPAY) {
            const cpx<T> *zz = z + cb * 12 * nr + r;
#pragma unroll
            for (int k = 0; k < 12; ++k) res[k] = zz[(long)k * nr] - res[k];
        }
    } else {
        // FP64 only: diagonal A x + hop
        const double *cl = op.clov64 + ((long)p * g.Vh + cb) * 2 * CLOV_BLOCK;
        cpx<T> xv[12];
        const cpx<T> *xx = xp + cb * 12 * nr + r;
#pragma unroll
        for (int k = 0; k < 12; ++k) xv[k] = xx[(long)k * nr];
        herm6<T, double>(cl, xv, res);
        herm6<T, double>(cl + CLOV_BLOCK, xv + 6, res + 6);
#pragma unroll
        for (int k = 0; k < 12; ++k) res[k] += acc[k];
        if (MODE == HOP_RESID) {
            const cpx<T> *zz = z + cb * 12 * nr + r;
#pragma unroll
            for (int k = 0; k < 12; ++k) res[k] = zz[(long)k * nr] - res[k];
        }
    }
    cpx<T> *dst = out + cb * 12 * nr + r;
#pragma unroll
    for (int k = 0; k < 12; ++k) dst[(long)k * nr] = res[k];
}

// Algorithmic traffic of one hop launch over the Vh output sites of a parity:
// each neighbour spinor is read once per launch (24 reals), the output written
// once (24 reals), the xpay/residual operands read once (24 reals each); the 8
// links touching a site are read once per launch (12 reals compressed for FP32,
// 18 for FP64) and the clover block once (72 reals).
double hop_bytes(const DiracOp &op, HopMode mode, int nr, size_t real_bytes) {
    double spin = 24.0 * real_bytes;
    double per_rhs = 2.0 * spin + (mode == HOP_CLOVINV ? 0.0 : spin) + (mode == HOP_RESID || mode == HOP_APPLY ? spin : 0.0);
    double link_reals = real_bytes == 4 ? 12.0 : 18.0;
    double per_site = 8.0 * link_reals * real_bytes + 72.0 * (mode == HOP_CLOVINV || mode == HOP_CLOVINV_XPAY ? real_bytes : 8.0);
    return (double)op.g.Vh * (nr * per_rhs + per_site);
}

// Conventional flop count per output site and right-hand side: 1320 (Wilson
// hopping term) + 504 (two 6x6 complex clover blocks).
double hop_flops(const DiracOp &op, int nr) { return (double)op.g.Vh * nr * 1824.0; }

template <typename T>
void hop(const DiracOp &op, int p, HopMode mode, cpx<T> *out, const cpx<T> *in, const cpx<T> *z, const cpx<T> *xp,
         int nr, cudaStream_t s) {
    long n = op.g.Vh * nr;
    const int block = 128;
    unsigned grid = grid_for(n, block);
    prof_begin("dslash_fp64", s);
    switch (mode) {
        case HOP_CLOVINV: hop_kernel<T, HOP_CLOVINV><<<grid, block, 0, s>>>(op, p, out, in, z, xp, nr); break;
        case HOP_CLOVINV_XPAY: hop_kernel<T, HOP_CLOVINV_XPAY><<<grid, block, 0, s>>>(op, p, out, in, z, xp, nr); break;
        case HOP_APPLY: hop_kernel<T, HOP_APPLY><<<grid, block, 0, s>>>(op, p, out, in, z, xp, nr); break;
        case HOP_RESID: hop_kernel<T, HOP_RESID><<<grid, block, 0, s>>>(op, p, out, in, z, xp, nr); break;
    }
    LAPH_LAUNCH_CHECK();
    prof_end("dslash_fp64", s, hop_bytes(op, mode, nr, sizeof(T)), hop_flops(op, nr));
}

template void hop<double>(const DiracOp &, int, HopMode, c64 *, const c64 *, const c64 *, const c64 *, int, cudaStream_t);
template <>
void hop<float>(const DiracOp &op, int p, HopMode mode, c32 *out, const c32 *in, const c32 *z, const c32 *xp, int nr,
                cudaStream_t s) {
    // packed-FP32 kernel of dslash_f32.cu; in apply mode the same-parity operand travels as z
    hop_f32(op, p, mode, out, in, mode == HOP_APPLY ? xp : z, nr, s);
}

// ------------------------------------------------------------ clover inverse only
template <typename T>
__global__ void clov_inv_kernel(DiracOp op, int p, cpx<T> *out, const cpx<T> *in, int nr) {
    long tid = (long)blockIdx.x * blockDim.x + threadIdx.x;
    long cb = tid / nr;
    int r = (int)(tid - cb * nr);
    if (cb >= op.g.Vh) return;
    cpx<T> x[12], y[12];
    const cpx<T> *src = in + cb * 12 * nr + r;
#pragma unroll
    for (int k = 0; k < 12; ++k) x[k] = src[(long)k * nr];
    const T *ci = ClovPtr<T>::inv(op) + ((long)p * op.g.Vh + cb) * 2 * CLOV_BLOCK;
    herm6<T, T>(ci, x, y);
    herm6<T, T>(ci + CLOV_BLOCK, x + 6, y + 6);
    cpx<T> *dst = out + cb * 12 * nr + r;
#pragma unroll
    for (int k = 0; k < 12; ++k) dst[(long)k * nr] = y[k];
}

template <typename T>
void clov_inv_apply(const DiracOp &op, int p, cpx<T> *out, const cpx<T> *in, int nr, cudaStream_t s) {
    long n = op.g.Vh * nr;
    clov_inv_kernel<T><<<grid_for(n, 128), 128, 0, s>>>(op, p, out, in, nr);
    LAPH_LAUNCH_CHECK();
}
template void clov_inv_apply<double>(const DiracOp &, int, c64 *, const c64 *, int, cudaStream_t);
template void clov_inv_apply<float>(const DiracOp &, int, c32 *, const c32 *, int, cudaStream_t);

// ------------------------------------------------------------ layout conversion
__global__ void to_eo_kernel(Geom g, const c64 *__restrict__ abi, int first, int nr, c64 *even, c64 *odd) {
    long tid = (long)blockIdx.x * blockDim.x + threadIdx.x;
    long n = g.V * 12 * nr;
    if (tid >= n) return;
    int r = (int)(tid % nr);
    long sk = tid / nr;          // site * 12 + k
    long s = sk / 12;
    int k = (int)(sk % 12);
    int c[4];
    site_coords(g, s, c);
    c64 v = abi[((long)(first + r) * g.V + s) * 12 + k];
    c64 *dst = parity_of(c) ? odd : even;
    dst[((s >> 1) * 12 + k) * nr + r] = v;
}

__global__ void from_eo_kernel(Geom g, const c64 *__restrict__ even, const c64 *__restrict__ odd, int first, int nr,
                               c64 *abi) {
    long tid = (long)blockIdx.x * blockDim.x + threadIdx.x;
    long n = g.V * 12 * nr;
    if (tid >= n) return;
    // output-major order: coalesced writes to the ABI array
    long s12 = tid % (g.V * 12);
    int r = (int)(tid / (g.V * 12));
    long s = s12 / 12;
    int k = (int)(s12 % 12);
    int c[4];
    site_coords(g, s, c);
    const c64 *src = parity_of(c) ? odd : even;
    abi[((long)(first + r) * g.V + s) * 12 + k] = src[((s >> 1) * 12 + k) * nr + r];
}

void fields_to_eo(const Geom &g, const c64 *abi, int first, int nr, c64 *even, c64 *odd, cudaStream_t s) {
    long n = g.V * 12 * nr;
    to_eo_kernel<<<grid_for(n, 256), 256, 0, s>>>(g, abi, first, nr, even, odd);
    LAPH_LAUNCH_CHECK();
}

void eo_to_fields(const Geom &g, const c64 *even, const c64 *odd, int first, int nr, c64 *abi, cudaStream_t s) {
    long n = g.V * 12 * nr;
    from_eo_kernel<<<grid_for(n, 256), 256, 0, s>>>(g, even, odd, first, nr, abi);
    LAPH_LAUNCH_CHECK();
}

}  // namespace laph

using namespace laph;

extern "C" int laph_dirac_apply(laph_ctx *ctx, const laph_lattice *lat, const void *links,
                                const laph_dirac_params *dirac, const void *in, void *out, int nrhs, void *stream) {
    return guard([&] {
        ctx_activate(ctx);
        Geom g = make_geom(lat);
        LAPH_REQUIRE(dirac != nullptr, "dirac params are null");
        LAPH_REQUIRE(nrhs >= 1, "nrhs must be >= 1");
        cudaStream_t s = as_stream(stream);
        size_t lbytes = sizeof(c64) * 36 * g.V;
        size_t fbytes = sizeof(c64) * 12 * g.V * nrhs;
        const c64 *L = (const c64 *)stage_in(ctx, links, lbytes, "links", s);
        const c64 *x = (const c64 *)stage_in(ctx, in, fbytes, "apply_in", s);
        StagedOut o = stage_out(ctx, out, fbytes, "apply_out");
        DiracOp op = prepare_dirac(ctx, g, L, dirac->m0, dirac->csw, lat->xi, s);
        int nr = nrhs;
        size_t hb = sizeof(c64) * 12 * g.Vh * nr;
        c64 *xe = (c64 *)ws_get(ctx, "apply:xe", hb);
        c64 *xo = (c64 *)ws_get(ctx, "apply:xo", hb);
        c64 *ye = (c64 *)ws_get(ctx, "apply:ye", hb);
        c64 *yo = (c64 *)ws_get(ctx, "apply:yo", hb);
        fields_to_eo(g, x, 0, nr, xe, xo, s);
        hop<double>(op, 0, HOP_APPLY, ye, xo, nullptr, xe, nr, s);
        hop<double>(op, 1, HOP_APPLY, yo, xe, nullptr, xo, nr, s);
        eo_to_fields(g, ye, yo, 0, nr, (c64 *)o.dev, s);
        o.commit(s);
    });
}

extern "C" int laph_dslash_eo(laph_ctx *ctx, const laph_lattice *lat, const void *links,
                              const laph_dirac_params *dirac, int parity, int mode, int precision, const void *in,
                              const void *z, void *out, int nrhs, void *stream) {
    return guard([&] {
        ctx_activate(ctx);
        Geom g = make_geom(lat);
        LAPH_REQUIRE(dirac != nullptr, "dirac params are null");
        LAPH_REQUIRE(parity == 0 || parity == 1, "parity must be 0 or 1");
        LAPH_REQUIRE(mode == LAPH_HOP_CLOVINV || mode == LAPH_HOP_CLOVINV_XPAY || mode == LAPH_HOP_APPLY,
                     "unknown hop mode");
        LAPH_REQUIRE(precision == LAPH_PREC_FP64 || precision == LAPH_PREC_FP32 || precision == LAPH_PREC_BF16,
                     "unknown precision");
        LAPH_REQUIRE(precision != LAPH_PREC_BF16 || (nrhs >= 32 && nrhs <= 256 && (nrhs & (nrhs - 1)) == 0),
                     "the BF16 hop takes 32, 64, 128 or 256 right-hand sides");
        LAPH_REQUIRE(nrhs >= 1, "nrhs must be >= 1");
        LAPH_REQUIRE(in != nullptr && out != nullptr, "in/out are null");
        LAPH_REQUIRE(mode == LAPH_HOP_CLOVINV || z != nullptr, "z is required in this mode");
        cudaStream_t s = as_stream(stream);
        const size_t elem = precision == LAPH_PREC_FP64 ? sizeof(c64) : precision == LAPH_PREC_FP32 ? sizeof(c32)
                                                                                                   : sizeof(bf2);
        const size_t hb = elem * 12 * g.Vh * nrhs;
        const c64 *L = (const c64 *)stage_in(ctx, links, sizeof(c64) * 36 * g.V, "links", s);
        const void *x = stage_in(ctx, in, hb, "hop_in", s);
        const void *zz = mode == LAPH_HOP_CLOVINV ? nullptr : stage_in(ctx, z, hb, "hop_z", s);
        StagedOut o = stage_out(ctx, out, hb, "hop_out");
        DiracOp op = prepare_dirac(ctx, g, L, dirac->m0, dirac->csw, lat->xi, s);
        const HopMode hm = mode == LAPH_HOP_CLOVINV ? HOP_CLOVINV : mode == LAPH_HOP_CLOVINV_XPAY ? HOP_CLOVINV_XPAY
                                                                                                : HOP_APPLY;
        if (precision == LAPH_PREC_FP64) {
            const c64 *zp = (const c64 *)zz;
            hop<double>(op, parity, hm, (c64 *)o.dev, (const c64 *)x, hm == HOP_CLOVINV_XPAY ? zp : nullptr,
                        hm == HOP_APPLY ? zp : nullptr, nrhs, s);
        } else if (precision == LAPH_PREC_FP32) {
            hop_f32(op, parity, hm, (c32 *)o.dev, (const c32 *)x, (const c32 *)zz, nrhs, s);
        } else {
            hop_bf16(op, parity, hm, (bf2 *)o.dev, (const bf2 *)x, (const bf2 *)zz, nrhs, s);
        }
        o.commit(s);
        LAPH_CUDA(cudaStreamSynchronize(s));
        hop_timeout_check(s);
    });
}
