// FP32 even-odd Wilson-clover hop for the inner solver (many right-hand sides),
// written for packed FP32 arithmetic: every complex multiply-add is two
// __ffma2_rn on float2 lanes (re, im).
//
//   c += a b   with a a matrix entry stored as (re, re, im, im):
//       c = ffma2((a.re, a.re), (b.re, b.im), c);  c = ffma2((a.im, a.im), (-b.im, b.re), c)
//   c += conj(a) b uses (b.im, -b.re) in the second product.
//
// Operands prepared once per operator (prepare_dirac): a neighbour table with the
// antiperiodic time sign folded in (no coordinate arithmetic in the kernel), full
// 3x3 FP32 links (no third-row rebuild per right-hand side) and the clover
// inverse in the same (re, re, im, im) form.  Layouts:
//   nbr  [p][cb][8] int32: forward mu = 0..3 then backward mu = 0..3; a negative value ~j means
//        neighbour j with a sign flip (a hop across the time boundary).
//   L32w [p][mu][cb][9] float4 (re, re, im, im) of U_mu(x), row-major.
//   C32w [p][cb][2 blocks][6 float2 (d, d) + 15 float4 (re, re, im, im)] (strictly lower part, row-major).
// Thread mapping and spinor layout as in dslash.cu: thread (cb, r), f[cb][spin*3+colour][nr].
#include "dirac.cuh"

namespace laph {

__device__ __forceinline__ float2 ff(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 rot_i(float2 x) { return make_float2(-x.y, x.x); }     // i x
__device__ __forceinline__ float2 rot_mi(float2 x) { return make_float2(x.y, -x.x); }    // -i x
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __fadd2_rn(a, ff(-b.x, -b.y)); }

// k[a] = sum_b U[a][b] h[b] (fwd) or sum_b conj(U[b][a]) h[b] (!fwd), two spin components.
template <bool FWD>
__device__ __forceinline__ void su3_mul2(const float4 *__restrict__ u, const float2 h0[3], const float2 h1[3],
                                         float2 k0[3], float2 k1[3]) {
    float2 r0[3], r1[3];
#pragma unroll
    for (int b = 0; b < 3; ++b) {
        r0[b] = FWD ? rot_i(h0[b]) : rot_mi(h0[b]);
        r1[b] = FWD ? rot_i(h1[b]) : rot_mi(h1[b]);
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        float2 s0 = ff(0.f, 0.f), s1 = ff(0.f, 0.f);
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            float4 e = __ldg(u + (FWD ? a * 3 + b : b * 3 + a));
            float2 rr = ff(e.x, e.y), ii = ff(e.z, e.w);
            s0 = fma2(rr, h0[b], s0);
            s0 = fma2(ii, r0[b], s0);
            s1 = fma2(rr, h1[b], s1);
            s1 = fma2(ii, r1[b], s1);
        }
        k0[a] = s0;
        k1[a] = s1;
    }
}

// One direction: project the neighbour spinor, multiply by the link, accumulate with weight c.
// FWD: (1 - gamma_mu) U psi(x+mu);  !FWD: (1 + gamma_mu) U^dag psi(x-mu).
template <int MU, bool FWD>
__device__ __forceinline__ void hop_dir2(float2 acc[12], const float2 *__restrict__ src, int nr,
                                         const float4 *__restrict__ u, float c) {
    float2 h0[3], h1[3];
#pragma unroll
    for (int col = 0; col < 3; ++col) {
        float2 u0 = src[(long)(0 * 3 + col) * nr], u1 = src[(long)(1 * 3 + col) * nr];
        float2 d0 = src[(long)(2 * 3 + col) * nr], d1 = src[(long)(3 * 3 + col) * nr];
        // h = u -+ G d with G_1 = -i sigma_1, G_2 = -i sigma_2, G_3 = -i sigma_3, G_4 = 1
        if (MU == 0) {
            h0[col] = FWD ? add2(u0, rot_i(d1)) : sub2(u0, rot_i(d1));
            h1[col] = FWD ? add2(u1, rot_i(d0)) : sub2(u1, rot_i(d0));
        } else if (MU == 1) {
            h0[col] = FWD ? add2(u0, d1) : sub2(u0, d1);
            h1[col] = FWD ? sub2(u1, d0) : add2(u1, d0);
        } else if (MU == 2) {
            h0[col] = FWD ? add2(u0, rot_i(d0)) : sub2(u0, rot_i(d0));
            h1[col] = FWD ? sub2(u1, rot_i(d1)) : add2(u1, rot_i(d1));
        } else {
            h0[col] = FWD ? sub2(u0, d0) : add2(u0, d0);
            h1[col] = FWD ? sub2(u1, d1) : add2(u1, d1);
        }
    }
    float2 k0[3], k1[3];
    su3_mul2<FWD>(u, h0, h1, k0, k1);
    const float2 cc = ff(c, c);
#pragma unroll
    for (int col = 0; col < 3; ++col) {
        acc[col] = fma2(cc, k0[col], acc[col]);
        acc[3 + col] = fma2(cc, k1[col], acc[3 + col]);
        // lower = -+ G^dag k:  G_1^dag (k0,k1) = (i k1, i k0), G_2^dag = (k1, -k0),
        //                      G_3^dag = (i k0, -i k1), G_4^dag = (k0, k1)
        float2 l0, l1;
        if (MU == 0) { l0 = rot_i(k1[col]); l1 = rot_i(k0[col]); }
        else if (MU == 1) { l0 = k1[col]; l1 = ff(-k0[col].x, -k0[col].y); }
        else if (MU == 2) { l0 = rot_i(k0[col]); l1 = rot_mi(k1[col]); }
        else { l0 = k0[col]; l1 = k1[col]; }
        const float2 cs = FWD ? ff(-c, -c) : cc;
        acc[6 + col] = fma2(cs, l0, acc[6 + col]);
        acc[9 + col] = fma2(cs, l1, acc[9 + col]);
    }
}

// y = B x for one packed Hermitian 6x6 block: 6 float2 (d, d) then 15 float4 (re, re, im, im).
__device__ __forceinline__ void herm6_f2(const float *__restrict__ blk, const float2 x[6], float2 y[6]) {
    const float2 *dg = reinterpret_cast<const float2 *>(blk);
    const float4 *lo = reinterpret_cast<const float4 *>(blk + 12);
    float2 ix[6], mix[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        y[i] = __fmul2_rn(__ldg(dg + i), x[i]);
        ix[i] = rot_i(x[i]);
        mix[i] = rot_mi(x[i]);
    }
    int o = 0;
#pragma unroll
    for (int i = 1; i < 6; ++i)
#pragma unroll
        for (int j = 0; j < i; ++j) {
            float4 e = __ldg(lo + o++);
            float2 rr = ff(e.x, e.y), ii = ff(e.z, e.w);
            y[i] = fma2(rr, x[j], y[i]);
            y[i] = fma2(ii, ix[j], y[i]);
            y[j] = fma2(rr, x[i], y[j]);
            y[j] = fma2(ii, mix[i], y[j]);
        }
}

template <int MODE>
__global__ void __launch_bounds__(128) hop2_kernel(const int *__restrict__ nbr, const float4 *__restrict__ L,
                                                   const float *__restrict__ C, long Vh, int p, float hws, float hwt,
                                                   float2 *__restrict__ out, const float2 *__restrict__ in,
                                                   const float2 *__restrict__ z, int nr) {
    long tid = (long)blockIdx.x * blockDim.x + threadIdx.x;
    long cb = tid / nr;
    int r = (int)(tid - cb * nr);
    if (cb >= Vh) return;
    const int *nb = nbr + ((long)p * Vh + cb) * 8;
    int nn[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) nn[k] = __ldg(nb + k);
    float2 acc[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) acc[k] = ff(0.f, 0.f);
    const long lstride = Vh * 9;   // float4 per (p, mu) plane
#define HOP_DIR(MU)                                                                                        \
    {                                                                                                      \
        const float w = (MU == 3) ? hwt : hws;                                                             \
        int j = nn[MU];                                                                                    \
        float c = j < 0 ? -w : w;                                                                          \
        j = j < 0 ? ~j : j;                                                                                \
        hop_dir2<MU, true>(acc, in + (long)j * 12 * nr + r, nr, L + ((long)p * 4 + MU) * lstride + cb * 9, c); \
        int jb = nn[4 + MU];                                                                               \
        float cbk = jb < 0 ? -w : w;                                                                       \
        jb = jb < 0 ? ~jb : jb;                                                                            \
        hop_dir2<MU, false>(acc, in + (long)jb * 12 * nr + r, nr,                                          \
                            L + ((long)(1 - p) * 4 + MU) * lstride + (long)jb * 9, cbk);                   \
    }
    HOP_DIR(0)
    HOP_DIR(1)
    HOP_DIR(2)
    HOP_DIR(3)
#undef HOP_DIR
    const float *cl = C + ((long)p * Vh + cb) * 144;
    float2 res[12];
    float2 *dst = out + cb * 12 * nr + r;
    if (MODE == HOP_APPLY) {
        // K restricted to parity p: A_pp z + D in  (C holds the packed clover A itself here)
        const float2 *zz = z + cb * 12 * nr + r;
        float2 xv[12];
#pragma unroll
        for (int k = 0; k < 12; ++k) xv[k] = zz[(long)k * nr];
        herm6_f2(cl, xv, res);
        herm6_f2(cl + 72, xv + 6, res + 6);
#pragma unroll
        for (int k = 0; k < 12; ++k) dst[(long)k * nr] = add2(res[k], acc[k]);
        return;
    }
    herm6_f2(cl, acc, res);
    herm6_f2(cl + 72, acc + 6, res + 6);
    if (MODE == HOP_CLOVINV_XPAY) {
        const float2 *zz = z + cb * 12 * nr + r;
#pragma unroll
        for (int k = 0; k < 12; ++k) dst[(long)k * nr] = sub2(zz[(long)k * nr], res[k]);
    } else {
#pragma unroll
        for (int k = 0; k < 12; ++k) dst[(long)k * nr] = res[k];
    }
}

double hop_bytes(const DiracOp &op, HopMode mode, int nr, size_t real_bytes);
double hop_flops(const DiracOp &op, int nr);

void hop_f32(const DiracOp &op, int p, HopMode mode, c32 *out, const c32 *in, const c32 *z, int nr, cudaStream_t s) {
    LAPH_REQUIRE(mode == HOP_CLOVINV || mode == HOP_CLOVINV_XPAY || mode == HOP_APPLY,
                 "FP32 hop supports the clover-inverse and apply modes");
    long n = op.g.Vh * nr;
    const int block = 128;
    unsigned grid = grid_for(n, block);
    float hws = (float)op.hw[0], hwt = (float)op.hw[3];
    prof_begin("dslash_fp32", s);
    if (mode == HOP_APPLY)
        hop2_kernel<HOP_APPLY><<<grid, block, 0, s>>>(op.nbr, op.L32w, op.C32wA, op.g.Vh, p, hws, hwt, (float2 *)out,
                                                      (const float2 *)in, (const float2 *)z, nr);
    else if (mode == HOP_CLOVINV)
        hop2_kernel<HOP_CLOVINV><<<grid, block, 0, s>>>(op.nbr, op.L32w, op.C32w, op.g.Vh, p, hws, hwt, (float2 *)out,
                                                        (const float2 *)in, (const float2 *)z, nr);
    else
        hop2_kernel<HOP_CLOVINV_XPAY><<<grid, block, 0, s>>>(op.nbr, op.L32w, op.C32w, op.g.Vh, p, hws, hwt,
                                                             (float2 *)out, (const float2 *)in, (const float2 *)z, nr);
    LAPH_LAUNCH_CHECK();
    prof_end("dslash_fp32", s, hop_bytes(op, mode, nr, sizeof(float)), hop_flops(op, nr));
}

// ------------------------------------------------------------------ operand preparation
__global__ void nbr_kernel(Geom g, int *nbr) {
    long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= 2 * g.Vh) return;
    int p = (int)(idx / g.Vh);
    long cb = idx % g.Vh;
    int c[4];
    cb_coords(g, p, cb, c);
    const int dims[4] = {g.ns, g.ns, g.ns, g.nt};
    for (int mu = 0; mu < 4; ++mu) {
        int cf[4] = {c[0], c[1], c[2], c[3]}, cbk[4] = {c[0], c[1], c[2], c[3]};
        cf[mu] = (c[mu] + 1) % dims[mu];
        cbk[mu] = (c[mu] - 1 + dims[mu]) % dims[mu];
        int jf = (int)(site_of(g, cf) >> 1), jb = (int)(site_of(g, cbk) >> 1);
        bool flip_f = (mu == 3 && c[3] == g.nt - 1), flip_b = (mu == 3 && c[3] == 0);
        nbr[idx * 8 + mu] = flip_f ? ~jf : jf;
        nbr[idx * 8 + 4 + mu] = flip_b ? ~jb : jb;
    }
}

__global__ void links_w_kernel(long n4, const c64 *__restrict__ L64, float4 *L32w) {
    long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n4 * 9) return;
    c64 u = L64[idx];
    L32w[idx] = make_float4((float)u.re, (float)u.re, (float)u.im, (float)u.im);
}

__global__ void clov_w_kernel(long nblk, const double *__restrict__ cinv64, float *C32w) {
    long b = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nblk) return;
    const double *src = cinv64 + b * CLOV_BLOCK;
    float *dst = C32w + b * 72;
    for (int i = 0; i < 6; ++i) {
        dst[2 * i] = (float)src[i];
        dst[2 * i + 1] = (float)src[i];
    }
    for (int k = 0; k < 15; ++k) {
        float re = (float)src[6 + 2 * k], im = (float)src[6 + 2 * k + 1];
        dst[12 + 4 * k] = re;
        dst[12 + 4 * k + 1] = re;
        dst[12 + 4 * k + 2] = im;
        dst[12 + 4 * k + 3] = im;
    }
}

void prepare_f32_operands(laph_ctx *ctx, DiracOp &op, cudaStream_t s) {
    const Geom &g = op.g;
    LAPH_REQUIRE(g.Vh < (1L << 31), "lattice too large for 32-bit neighbour indices");
    op.nbr = (int *)ws_get(ctx, "dirac:nbr", sizeof(int) * 16 * g.Vh);
    op.L32w = (float4 *)ws_get(ctx, "dirac:L32w", sizeof(float4) * 9 * 8 * g.Vh);
    op.C32w = (float *)ws_get(ctx, "dirac:C32w", sizeof(float) * 144 * 2 * g.Vh);
    op.C32wA = (float *)ws_get(ctx, "dirac:C32wA", sizeof(float) * 144 * 2 * g.Vh);
    nbr_kernel<<<grid_for(2 * g.Vh, 256), 256, 0, s>>>(g, op.nbr);
    LAPH_LAUNCH_CHECK();
    links_w_kernel<<<grid_for(8 * g.Vh * 9, 256), 256, 0, s>>>(8 * g.Vh, op.L64, op.L32w);
    LAPH_LAUNCH_CHECK();
    clov_w_kernel<<<grid_for(4 * g.Vh, 256), 256, 0, s>>>(4 * g.Vh, op.cinv64, op.C32w);
    LAPH_LAUNCH_CHECK();
    clov_w_kernel<<<grid_for(4 * g.Vh, 256), 256, 0, s>>>(4 * g.Vh, op.clov64, op.C32wA);
    LAPH_LAUNCH_CHECK();
}

}  // namespace laph
