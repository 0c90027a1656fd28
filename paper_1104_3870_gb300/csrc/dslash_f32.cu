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
#include <cuda.h>
#include <cudaTypedefs.h>

#include <cstdlib>

#include "blas.cuh"
#include "dirac.cuh"
#include "tma.cuh"

namespace laph {

__device__ __forceinline__ float2 ff(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 rot_i(float2 x) { return make_float2(-x.y, x.x); }     // i x
__device__ __forceinline__ float2 rot_mi(float2 x) { return make_float2(x.y, -x.x); }    // -i x
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __fadd2_rn(a, ff(-b.x, -b.y)); }
// operand load: read-only global path (G) or plain load (shared-memory staging)
template <bool G, typename T>
__device__ __forceinline__ T ld(const T *p) { return G ? __ldg(p) : *p; }
// spinor elements: FP32 (float2) or BF16 (bf162) storage, FP32 arithmetic
__device__ __forceinline__ float2 to_f2(float2 v) { return v; }
__device__ __forceinline__ float2 to_f2(__nv_bfloat162 v) { return __bfloat1622float2(v); }
template <typename E>
__device__ __forceinline__ E from_f2(float2 v);
template <>
__device__ __forceinline__ float2 from_f2<float2>(float2 v) { return v; }
template <>
__device__ __forceinline__ __nv_bfloat162 from_f2<__nv_bfloat162>(float2 v) { return __float22bfloat162_rn(v); }

// k[a] = sum_b U[a][b] h[b] (fwd) or sum_b conj(U[b][a]) h[b] (!fwd), two spin components.
template <bool FWD, bool G = true>
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
            float4 e = ld<G>(u + (FWD ? a * 3 + b : b * 3 + a));
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
template <int MU, bool FWD, bool G = true, typename E = float2>
__device__ __forceinline__ void hop_dir2(float2 acc[12], const E *__restrict__ src, int nr,
                                         const float4 *__restrict__ u, float c) {
    float2 h0[3], h1[3];
#pragma unroll
    for (int col = 0; col < 3; ++col) {
        float2 u0 = to_f2(src[(long)(0 * 3 + col) * nr]), u1 = to_f2(src[(long)(1 * 3 + col) * nr]);
        float2 d0 = to_f2(src[(long)(2 * 3 + col) * nr]), d1 = to_f2(src[(long)(3 * 3 + col) * nr]);
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
    su3_mul2<FWD, G>(u, h0, h1, k0, k1);
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
template <bool G = true>
__device__ __forceinline__ void herm6_f2(const float *__restrict__ blk, const float2 x[6], float2 y[6]) {
    const float2 *dg = reinterpret_cast<const float2 *>(blk);
    const float4 *lo = reinterpret_cast<const float4 *>(blk + 12);
    float2 ix[6], mix[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        y[i] = __fmul2_rn(ld<G>(dg + i), x[i]);
        ix[i] = rot_i(x[i]);
        mix[i] = rot_mi(x[i]);
    }
    int o = 0;
#pragma unroll
    for (int i = 1; i < 6; ++i)
#pragma unroll
        for (int j = 0; j < i; ++j) {
            float4 e = ld<G>(lo + o++);
            float2 rr = ff(e.x, e.y), ii = ff(e.z, e.w);
            y[i] = fma2(rr, x[j], y[i]);
            y[i] = fma2(ii, ix[j], y[i]);
            y[j] = fma2(rr, x[i], y[j]);
            y[j] = fma2(ii, mix[i], y[j]);
        }
}

template <int MODE>
__global__ void __launch_bounds__(128, MODE == HOP_APPLY ? 6 : 8) hop2_kernel(const int *__restrict__ nbr, const float4 *__restrict__ L,
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

// ------------------------------------------------------------------ TMA-fed hop
// The same arithmetic as hop2_kernel, with the operands of every hop brought into shared
// memory by the copy engine ahead of use.  A work unit is one warp: 32 RPT right-hand sides of
// one output site.  It consumes its jobs in order, each filling one slot of the warp's private
// ring of NS slots:
//   hop job       [12][32 RPT] tile of a neighbour spinor (one 2D tensor copy) + its link (9
//                 float4); with one RHS per lane a job holds both hops of one direction
//   epilogue job  [12][32 RPT] tile of z (modes with z) + the 144-float clover block of the site
// (nine jobs per site with two RHS per lane, five with one; in the clover-inverse mode with one
// RHS per lane the clover rides in the last hop job, whose slot is kept through the epilogue:
// four jobs).  While the warp computes job n, jobs n+1 .. n+NS-1 are in flight; the slot of job n
// is refilled with job n+NS as soon as every lane has read it.  Lane 0 issues all copies, and
// warps never wait on one another.
constexpr int HOP3_WARPS = 4;
#ifndef HOP3_MINB
#define HOP3_MINB 4   // blocks per SM the register allocation targets
#endif
// RPT right-hand sides per lane: a warp owns 32 RPT RHS of its site; the tile of a hop is
// 12 rows x 256 RPT B, followed by the link (144 B) or the clover block (576 B).
// HPJ hops per job: 1, or 2 (the forward and backward hop of one direction: two tiles and two links
// per slot, five jobs per site instead of nine, each covering twice the copy latency).
// CJ (clover-inverse mode with two hops per job): the clover block rides in the last hop job, whose
// slot the warp keeps until its epilogue, so a site takes four jobs instead of five.
#ifndef HOP3_CLOVJ
#define HOP3_CLOVJ 1
#endif
template <int RPT, typename E = float2, int HPJ = 1, bool CJ = false>
struct Hop3Geo {
    static constexpr int SPIN = 12 * 32 * RPT * (int)sizeof(E);     // 3072 RPT B (FP32), 1536 RPT B (BF16)
    static constexpr int PAIRB = HPJ * (SPIN + 144) + (CJ ? 576 : 0);
    static constexpr int BODY = PAIRB > SPIN + 576 ? PAIRB : SPIN + 576;
    static constexpr int SLOT = ((BODY + 127) / 128) * 128;         // 128-byte aligned slots
    static constexpr int JOBS = 8 / HPJ + (CJ ? 0 : 1);             // hop jobs (+ the epilogue job)
};
template <int MODE, int HPJ>
__host__ __device__ constexpr bool hop3_cj() { return HOP3_CLOVJ && MODE == HOP_CLOVINV && HPJ == 2; }
constexpr long long HOP3_WAIT_CYCLES = 1LL << 31;   // about one second at the maximum SM clock

__device__ int g_hop3_timeout;   // set when a copy wait gives up (or the ring is misaligned); read by the host

// DOTS (xpay mode, nr = 32 RPT): the epilogue also accumulates, per right-hand side, the inner
// products <out, z> and <out, out> of the warp's sites in FP32 and writes them as the warp's
// partial sums partial[warp][k][r] (k = 0, 1; FP64) for a fixed-order final sum.
template <int MODE, int NS, int RPT, int DOTS = 0, typename E = float2, int HPJ = 1>
__global__ void __launch_bounds__(HOP3_WARPS * 32, HOP3_MINB)
    hop3_kernel(const __grid_constant__ CUtensorMap tm_in, const __grid_constant__ CUtensorMap tm_z,
                const int *__restrict__ nbr, const int *__restrict__ order, const float4 *__restrict__ L,
                const float *__restrict__ C, int Vh, int p, float hws, float hwt, E *__restrict__ out, int nr, int gshift,
                int nunits, c64 *__restrict__ partial, const uint32_t *__restrict__ rcode) {
    extern __shared__ __align__(128) unsigned char sm3[];
    constexpr bool CJ = hop3_cj<MODE, HPJ>();
    constexpr int HOP3_SPIN = Hop3Geo<RPT, E, HPJ, CJ>::SPIN, HOP3_SLOT = Hop3Geo<RPT, E, HPJ, CJ>::SLOT;
    constexpr int NJ = Hop3Geo<RPT, E, HPJ, CJ>::JOBS;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (smem_u32(sm3) & 127) {   // tensor copies need 128-byte aligned destinations
        if (threadIdx.x == 0) atomicExch(&g_hop3_timeout, 2);
        return;
    }
    unsigned char *ring = sm3 + warp * NS * HOP3_SLOT;
    uint64_t *bar = reinterpret_cast<uint64_t *>(sm3 + HOP3_WARPS * NS * HOP3_SLOT) + warp * NS;
    float *meta = reinterpret_cast<float *>(sm3 + HOP3_WARPS * NS * (HOP3_SLOT + 8)) + warp * NS * 2;
    if (lane < NS) mbar_init(bar + lane, 1);
    mbar_fence_init();
    __syncwarp();
    const int gmask = (1 << gshift) - 1;
    // units of this warp: q = gw, gw + gstride, ...  The whole grid sweeps the lattice in
    // lexicographic bands, so a band's neighbours are in L2 from the bands around it
    // (contiguous per-CTA ranges measured 35 % slower; L2 evict-first/last hints on the
    // copies and stores made no difference).
    const int gw = blockIdx.x * HOP3_WARPS + warp, gstride = gridDim.x * HOP3_WARPS;
    const int nu = gw < nunits ? (nunits - gw + gstride - 1) / gstride : 0;
    const int *nbp = nbr + (long)p * Vh * 8;

    // issue pointer: job ij of the unit iq (the ik-th of this warp) goes to slot islot; lane
    // d < 8 holds neighbour d of unit iq (nb_i) and of the unit after it (nb_n)
    int iq = gw, ik = 0, ij = 0, islot = 0, niss = 0;
    // order[u]: the output site (checkerboard index) of the u-th unit site in visiting order
    int icb = nu > 0 ? __ldg(order + (iq >> gshift)) : 0;
    int nb_i = (nu > 0 && lane < 8) ? __ldg(nbp + icb * 8 + lane) : 0;
    int nb_n = (nu > 1 && lane < 8) ? __ldg(nbp + __ldg(order + ((iq + gstride) >> gshift)) * 8 + lane) : 0;
    auto issue = [&]() {
        if (ik >= nu) return;
        // HPJ = 1: job ij is hop ij of (forward mu = 0, backward mu = 0, forward mu = 1, ...);
        // HPJ = 2: job ij holds the forward and the backward hop of mu = ij
        const int e = __shfl_sync(0xffffffffu, nb_i, HPJ == 2 ? ij : ((ij & 1) ? 4 + (ij >> 1) : (ij >> 1)));
        const int e2 = HPJ == 2 ? __shfl_sync(0xffffffffu, nb_i, 4 + (ij & 3)) : 0;
        if (lane == 0) {
            const int cb = icb, h = iq & gmask;
            unsigned char *sl = ring + islot * HOP3_SLOT;
            uint64_t *b = bar + islot;
            fence_proxy_async_smem();
            if (CJ || ij < NJ - 1) {
                const int mu = HPJ == 2 ? ij : ij >> 1;
                const float w = mu == 3 ? hwt : hws;
                const int jn = e < 0 ? ~e : e;
                meta[2 * islot] = e < 0 ? -w : w;
                if (HPJ == 2) {
                    const int jb = e2 < 0 ? ~e2 : e2;
                    const bool clov = CJ && ij == NJ - 1;
                    meta[2 * islot + 1] = e2 < 0 ? -w : w;
                    mbar_arrive_expect_tx(b, 2 * (HOP3_SPIN + 144) + (clov ? 576 : 0));
                    tma_tile_2d(sl, &tm_in, 64 * RPT * h, 12 * jn, b);
                    tma_tile_2d(sl + HOP3_SPIN, &tm_in, 64 * RPT * h, 12 * jb, b);
                    bulk_g2s(sl + 2 * HOP3_SPIN, L + ((long)(p * 4 + mu) * Vh + cb) * 9, 144, b);
                    bulk_g2s(sl + 2 * HOP3_SPIN + 144, L + ((long)((1 - p) * 4 + mu) * Vh + jb) * 9, 144, b);
                    if (clov) bulk_g2s(sl + 2 * HOP3_SPIN + 288, C + ((long)p * Vh + cb) * 144, 576, b);
                } else {
                    mbar_arrive_expect_tx(b, HOP3_SPIN + 144);
                    tma_tile_2d(sl, &tm_in, 64 * RPT * h, 12 * jn, b);
                    const float4 *u = (ij & 1) ? L + ((long)((1 - p) * 4 + mu) * Vh + jn) * 9
                                               : L + ((long)(p * 4 + mu) * Vh + cb) * 9;
                    bulk_g2s(sl + HOP3_SPIN, u, 144, b);
                }
            } else {
                constexpr bool needz = MODE != HOP_CLOVINV;
                mbar_arrive_expect_tx(b, (needz ? HOP3_SPIN : 0) + 576);
                if (needz) tma_tile_2d(sl, &tm_z, 64 * RPT * h, 12 * cb, b);
                bulk_g2s(sl + HOP3_SPIN, C + ((long)p * Vh + cb) * 144, 576, b);
            }
        }
        ++niss;
        if (++islot == NS) islot = 0;
        if (++ij == NJ) {
            ij = 0;
            ++ik;
            iq += gstride;
            nb_i = nb_n;
            icb = ik < nu ? __ldg(order + (iq >> gshift)) : 0;
            nb_n = (ik + 1 < nu && lane < 8) ? __ldg(nbp + __ldg(order + ((iq + gstride) >> gshift)) * 8 + lane) : 0;
        }
    };
    // consume pointer
    int cslot = 0, ncons = 0;
    uint32_t cpar = 0;
    auto wait = [&]() -> bool {
        return __all_sync(0xffffffffu, mbar_wait_bounded(bar + cslot, cpar, HOP3_WAIT_CYCLES));
    };
    auto release = [&]() {
        __syncwarp();
        issue();
        ++ncons;
        if (++cslot == NS) {
            cslot = 0;
            cpar ^= 1u;
        }
    };

    for (int k = 0; k < NS; ++k) issue();
    float2 dts[RPT];
    float dtt[RPT];
#pragma unroll
    for (int q = 0; q < RPT; ++q) {
        dts[q] = ff(0.f, 0.f);
        dtt[q] = 0.f;
    }
    bool ok = true;
    for (int k = 0, q = gw; k < nu && ok; ++k, q += gstride) {
        const int cb = __ldg(order + (q >> gshift)), h = q & gmask;
        // packed shadow-vector codes, fetched before the hops so that their latency is hidden
        uint32_t rw[RPT];
#pragma unroll
        for (int q = 0; q < RPT; ++q) rw[q] = DOTS == 2 ? __ldg(rcode + (long)cb * nr + 32 * q + lane) : 0u;
        float2 acc[RPT][12];
#pragma unroll
        for (int q = 0; q < RPT; ++q)
#pragma unroll
            for (int c = 0; c < 12; ++c) acc[q][c] = ff(0.f, 0.f);
#define HOP3_DIR(MU, FWD)                                                                                  \
    if (ok) {                                                                                              \
        if (!wait()) {                                                                                     \
            ok = false;                                                                                    \
        } else {                                                                                           \
            const unsigned char *sl_ = ring + cslot * HOP3_SLOT;                                           \
            const float c_ = meta[2 * cslot];                                                              \
            _Pragma("unroll") for (int q = 0; q < RPT; ++q)                                                \
                hop_dir2<MU, FWD, false, E>(acc[q], reinterpret_cast<const E *>(sl_) + 32 * q + lane,      \
                                            32 * RPT, reinterpret_cast<const float4 *>(sl_ + HOP3_SPIN), c_); \
            release();                                                                                     \
        }                                                                                                  \
    }
#define HOP3_PAIR(MU)                                                                                      \
    if (ok) {                                                                                              \
        if (!wait()) {                                                                                     \
            ok = false;                                                                                    \
        } else {                                                                                           \
            const unsigned char *sl_ = ring + cslot * HOP3_SLOT;                                           \
            const float cf_ = meta[2 * cslot], cb_ = meta[2 * cslot + 1];                                  \
            const float4 *lk_ = reinterpret_cast<const float4 *>(sl_ + 2 * HOP3_SPIN);                     \
            _Pragma("unroll") for (int q = 0; q < RPT; ++q) {                                              \
                hop_dir2<MU, true, false, E>(acc[q], reinterpret_cast<const E *>(sl_) + 32 * q + lane,     \
                                             32 * RPT, lk_, cf_);                                          \
                hop_dir2<MU, false, false, E>(acc[q],                                                      \
                                              reinterpret_cast<const E *>(sl_ + HOP3_SPIN) + 32 * q + lane, \
                                              32 * RPT, lk_ + 9, cb_);                                     \
            }                                                                                              \
            if (!(CJ && MU == 3)) release();                                                               \
        }                                                                                                  \
    }
        if (HPJ == 2) {
            HOP3_PAIR(0)
            HOP3_PAIR(1)
            HOP3_PAIR(2)
            HOP3_PAIR(3)
        } else {
            HOP3_DIR(0, true)
            HOP3_DIR(0, false)
            HOP3_DIR(1, true)
            HOP3_DIR(1, false)
            HOP3_DIR(2, true)
            HOP3_DIR(2, false)
            HOP3_DIR(3, true)
            HOP3_DIR(3, false)
        }
#undef HOP3_DIR
#undef HOP3_PAIR
        if (CJ) {
            if (!ok) break;   // the clover came with the last hop job, whose slot is still held
        } else if (!ok || !wait()) {
            ok = false;
            break;
        }
        const unsigned char *sl = ring + cslot * HOP3_SLOT;
        const float *cl = reinterpret_cast<const float *>(sl + (CJ ? 2 * HOP3_SPIN + 288 : HOP3_SPIN));
        float2 res[RPT][12];
#pragma unroll
        for (int q = 0; q < RPT; ++q) {
            const E *zs = reinterpret_cast<const E *>(sl) + 32 * q + lane;
            if (MODE == HOP_APPLY) {
                float2 xv[12];
#pragma unroll
                for (int c = 0; c < 12; ++c) xv[c] = to_f2(zs[c * 32 * RPT]);
                herm6_f2<false>(cl, xv, res[q]);
                herm6_f2<false>(cl + 72, xv + 6, res[q] + 6);
#pragma unroll
                for (int c = 0; c < 12; ++c) res[q][c] = add2(res[q][c], acc[q][c]);
            } else {
                herm6_f2<false>(cl, acc[q], res[q]);
                herm6_f2<false>(cl + 72, acc[q] + 6, res[q] + 6);
                if (MODE == HOP_CLOVINV_XPAY) {
#pragma unroll
                    for (int c = 0; c < 12; ++c) {
                        const float2 zc = to_f2(zs[c * 32 * RPT]);
                        res[q][c] = sub2(zc, res[q][c]);
                        if (DOTS == 1) {   // conj(t) z and |t|^2
                            const float2 t = res[q][c];
                            dts[q].x = fmaf(t.x, zc.x, fmaf(t.y, zc.y, dts[q].x));
                            dts[q].y = fmaf(t.x, zc.y, fmaf(-t.y, zc.x, dts[q].y));
                            dtt[q] = fmaf(t.x, t.x, fmaf(t.y, t.y, dtt[q]));
                        } else if (DOTS == 2) {   // conj(rhat) t with the coded shadow vector (nr = 32 RPT)
                            const c32 v = rhat_conj_mul((rw[q] >> (2 * c)) & 3u, c32{res[q][c].x, res[q][c].y});
                            dts[q].x += v.re;
                            dts[q].y += v.im;
                        }
                    }
                }
            }
        }
        release();
#pragma unroll
        for (int q = 0; q < RPT; ++q) {
            E *dst = out + (long)cb * 12 * nr + 32 * RPT * h + 32 * q + lane;
#pragma unroll
            for (int c = 0; c < 12; ++c) dst[(long)c * nr] = from_f2<E>(res[q][c]);
        }
    }
    if (DOTS != 0) {   // every warp writes, zeros where it had no units
        const int gwarp = blockIdx.x * HOP3_WARPS + warp;
#pragma unroll
        for (int q = 0; q < RPT; ++q) {
            const int r = 32 * q + lane;
            partial[((long)gwarp * 2 + 0) * nr + r] = c64{(double)dts[q].x, (double)dts[q].y};
            partial[((long)gwarp * 2 + 1) * nr + r] = c64{(double)dtt[q], 0.0};
        }
    }
    if (!ok) {
        if (lane == 0) atomicExch(&g_hop3_timeout, 1);
        // wait (bounded) for every job issued and not yet read, so no copy lands after exit
        for (; ncons < niss; ++ncons) {
            mbar_wait_bounded(bar + cslot, cpar, HOP3_WAIT_CYCLES);
            if (++cslot == NS) {
                cslot = 0;
                cpar ^= 1u;
            }
        }
    }
}

// 2D view of a half-lattice FP32 field [cb][12][nr] complex: rows (cb, component) of 2 nr
// floats; a box is the 12 rows x 32 rpt right-hand sides that one warp reads.
template <typename E>
static CUtensorMap spinor_map(const E *base, long Vh, int nr, int rpt) {
    constexpr bool bf = sizeof(E) == 4;   // bf162 (two BF16 reals) or float2 (two FP32 reals)
    static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    if (!encode) {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        LAPH_CUDA(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q));
        LAPH_REQUIRE(q == cudaDriverEntryPointSuccess && fn != nullptr, "cuTensorMapEncodeTiled is unavailable");
        encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    }
    CUtensorMap m;
    const cuuint64_t dims[2] = {(cuuint64_t)(2 * nr), (cuuint64_t)(12 * Vh)};
    const cuuint64_t strides[1] = {(cuuint64_t)(2 * nr) * (bf ? 2 : 4)};
    const cuuint32_t box[2] = {(cuuint32_t)(64 * rpt), 12};
    const cuuint32_t estr[2] = {1, 1};
    CUresult r = encode(&m, bf ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2,
                        const_cast<E *>(base), dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    LAPH_REQUIRE(r == CUDA_SUCCESS, "tensor map encoding failed");
    return m;
}

template <int MODE, int NS, int RPT, int DOTS = 0, typename E = float2>
static long launch_hop3(const DiracOp &op, int p, float hws, float hwt, E *out, const E *in,
                        const E *z, int nr, cudaStream_t s, laph_ctx *ctx = nullptr, c64 *red = nullptr,
                        const uint32_t *rcode = nullptr) {
    // one RHS per lane: two hops per job (the slot still leaves room for four blocks per SM)
    constexpr int HPJ = RPT == 1 ? 2 : 1;
    constexpr size_t smem = (size_t)HOP3_WARPS * NS * (Hop3Geo<RPT, E, HPJ, hop3_cj<MODE, HPJ>()>::SLOT + 8 + 8);
    static int bpsm[64] = {0};
    static int nsm[64] = {0};
    int dev = 0;
    LAPH_CUDA(cudaGetDevice(&dev));
    LAPH_REQUIRE(dev < 64, "device index out of range");
    if (bpsm[dev] == 0) {
        LAPH_CUDA(cudaFuncSetAttribute(hop3_kernel<MODE, NS, RPT, DOTS, E, HPJ>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        LAPH_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bpsm[dev], hop3_kernel<MODE, NS, RPT, DOTS, E, HPJ>,
                                                                HOP3_WARPS * 32, smem));
        LAPH_CUDA(cudaDeviceGetAttribute(&nsm[dev], cudaDevAttrMultiProcessorCount, dev));
        LAPH_REQUIRE(bpsm[dev] > 0, "TMA hop kernel does not fit on this device");
    }
    int gshift = 0;
    while ((32 * RPT << gshift) < nr) ++gshift;
    const CUtensorMap tin = spinor_map(in, op.g.Vh, nr, RPT);
    const CUtensorMap tz = MODE == HOP_CLOVINV ? tin : spinor_map(z, op.g.Vh, nr, RPT);
    const long nunits = op.g.Vh * (nr / (32 * RPT));
    long grid = (nunits + HOP3_WARPS - 1) / HOP3_WARPS;
    const long cap = (long)bpsm[dev] * nsm[dev];
    if (grid > cap) grid = cap;
    c64 *partial = nullptr;
    if (DOTS != 0) partial = (c64 *)ws_get(ctx, "hop3:dots", sizeof(c64) * 2 * nr * grid * HOP3_WARPS);
    hop3_kernel<MODE, NS, RPT, DOTS, E, HPJ><<<(unsigned)grid, HOP3_WARPS * 32, smem, s>>>(
        tin, tz, op.nbr, op.order, op.L32w, MODE == HOP_APPLY ? op.C32wA : op.C32w, (int)op.g.Vh, p, hws, hwt, out, nr,
        gshift, (int)nunits, partial, rcode);
    if (DOTS != 0) {
        LAPH_LAUNCH_CHECK();
        red_final_sum(partial, (int)(grid * HOP3_WARPS), 2, nr, red, s);
    }
    return grid * HOP3_WARPS;
}

// Ring depth per warp of the TMA-fed kernel.  Two slots measured fastest on a 16^3 x 32
// lattice at 32 and 64 right-hand sides: a deeper ring costs more occupancy than its extra
// prefetch gains.  LAPH_HOP_STAGES = 3 selects a deeper ring, 0 the register-fed kernel
// (hop2_kernel) for every shape.  LAPH_HOP_RPT = 1 keeps one right-hand side per lane when
// the block has 64 or more.
static int hop3_stages() {
    static int ns = -1;
    if (ns < 0) {
        const char *e = getenv("LAPH_HOP_STAGES");
        int v = e ? atoi(e) : 2;
        ns = (v == 0 || v == 2 || v == 3) ? v : 2;
    }
    return ns;
}
static int hop3_rpt_max() {
    static int r = -1;
    if (r < 0) {
        const char *e = getenv("LAPH_HOP_RPT");
        r = (e && atoi(e) == 1) ? 1 : 2;
    }
    return r;
}

template <int NS, int RPT>
static void hop3_modes(const DiracOp &op, int p, HopMode mode, float hws, float hwt, float2 *out, const float2 *in,
                       const float2 *z, int nr, cudaStream_t s) {
    if (mode == HOP_APPLY)
        launch_hop3<HOP_APPLY, NS, RPT>(op, p, hws, hwt, out, in, z, nr, s);
    else if (mode == HOP_CLOVINV)
        launch_hop3<HOP_CLOVINV, NS, RPT>(op, p, hws, hwt, out, in, (const float2 *)nullptr, nr, s);
    else
        launch_hop3<HOP_CLOVINV_XPAY, NS, RPT>(op, p, hws, hwt, out, in, z, nr, s);
}

void hop_timeout_check(cudaStream_t s) {
    int v = 0;   // read on the caller's stream, so that other streams are not serialised with it
    LAPH_CUDA(cudaMemcpyFromSymbolAsync(&v, g_hop3_timeout, sizeof(int), 0, cudaMemcpyDeviceToHost, s));
    LAPH_CUDA(cudaStreamSynchronize(s));
    if (v) {   // 1: a copy wait gave up; 2: the shared-memory ring was misaligned (no copy issued)
        const int zero = 0;
        LAPH_CUDA(cudaMemcpyToSymbolAsync(g_hop3_timeout, &zero, sizeof(int), 0, cudaMemcpyHostToDevice, s));
        LAPH_CUDA(cudaStreamSynchronize(s));
        throw Error(LAPH_ERR_TIMEOUT, "a stencil copy wait gave up (device wait cap)");
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
    const bool aligned = ((reinterpret_cast<uintptr_t>(in) | reinterpret_cast<uintptr_t>(z) |
                           reinterpret_cast<uintptr_t>(op.L32w) | reinterpret_cast<uintptr_t>(op.C32w) |
                           reinterpret_cast<uintptr_t>(op.C32wA)) & 15) == 0;
    const int ns = hop3_stages();
    const bool pow2 = nr == 32 || nr == 64 || nr == 128 || nr == 256;
    if (pow2 && aligned && ns > 0 && op.g.Vh * (nr / 32) < (1L << 30)) {
        float2 *o = (float2 *)out;
        const float2 *i = (const float2 *)in, *zz = (const float2 *)z;
        const bool two = hop3_rpt_max() == 2 && nr % 64 == 0;
        if (ns == 3)
            two ? hop3_modes<3, 2>(op, p, mode, hws, hwt, o, i, zz, nr, s)
                : hop3_modes<3, 1>(op, p, mode, hws, hwt, o, i, zz, nr, s);
        else
            two ? hop3_modes<2, 2>(op, p, mode, hws, hwt, o, i, zz, nr, s)
                : hop3_modes<2, 1>(op, p, mode, hws, hwt, o, i, zz, nr, s);
    } else if (mode == HOP_APPLY)
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

bool hop_f32_xpay_dots(laph_ctx *ctx, const DiracOp &op, int p, c32 *out, const c32 *in, const c32 *z, int nr,
                       c64 *red, cudaStream_t s) {
    const bool aligned = ((reinterpret_cast<uintptr_t>(in) | reinterpret_cast<uintptr_t>(z) |
                           reinterpret_cast<uintptr_t>(op.L32w) | reinterpret_cast<uintptr_t>(op.C32w)) & 15) == 0;
    const int ns = hop3_stages();
    const int rpt = (hop3_rpt_max() == 2 && nr == 64) ? 2 : 1;
    if (!aligned || ns != 2 || nr != 32 * rpt) return false;
    float hws = (float)op.hw[0], hwt = (float)op.hw[3];
    prof_begin("dslash_fp32", s);
    if (rpt == 2)
        launch_hop3<HOP_CLOVINV_XPAY, 2, 2, 1>(op, p, hws, hwt, (float2 *)out, (const float2 *)in,
                                                  (const float2 *)z, nr, s, ctx, red);
    else
        launch_hop3<HOP_CLOVINV_XPAY, 2, 1, 1>(op, p, hws, hwt, (float2 *)out, (const float2 *)in,
                                                  (const float2 *)z, nr, s, ctx, red);
    LAPH_LAUNCH_CHECK();
    prof_end("dslash_fp32", s, hop_bytes(op, HOP_CLOVINV_XPAY, nr, sizeof(float)), hop_flops(op, nr));
    return true;
}

// The xpay hop out = z - A_pp^{-1} D in with <rhat, out> of every right-hand side fused into its
// epilogue (rhat the coded shadow vector of blas.cuh, rcode[cb][r] packed words): red[0][r] = <rhat, out>,
// red[1][r] = 0.
bool hop_f32_xpay_rdot(laph_ctx *ctx, const DiracOp &op, int p, c32 *out, const c32 *in, const c32 *z, int nr,
                       const uint32_t *rcode, c64 *red, cudaStream_t s) {
    // one right-hand side per lane only: with two the fused epilogue spills registers
    const bool aligned = ((reinterpret_cast<uintptr_t>(in) | reinterpret_cast<uintptr_t>(z) |
                           reinterpret_cast<uintptr_t>(op.L32w) | reinterpret_cast<uintptr_t>(op.C32w)) & 15) == 0;
    if (!aligned || hop3_stages() != 2 || nr != 32) return false;
    float hws = (float)op.hw[0], hwt = (float)op.hw[3];
    prof_begin("dslash_fp32", s);
    launch_hop3<HOP_CLOVINV_XPAY, 2, 1, 2>(op, p, hws, hwt, (float2 *)out, (const float2 *)in, (const float2 *)z, nr,
                                           s, ctx, red, rcode);
    LAPH_LAUNCH_CHECK();
    prof_end("dslash_fp32", s, hop_bytes(op, HOP_CLOVINV_XPAY, nr, sizeof(float)) + (double)op.g.Vh * 4 * nr,
             hop_flops(op, nr));
    return true;
}

// ------------------------------------------------------------------ BF16-stored spinors
// Algorithmic bytes of one BF16 hop launch: spinors 24 BF16 reals (2 B) in and out (and z),
// the 8 links of a site as 12 FP32 reals and the 72 FP32 clover reals, once per launch.
static double hop_bytes_bf16(const DiracOp &op, HopMode mode, int nr) {
    const double spin = 24.0 * 2.0;
    const double per_rhs = 2.0 * spin + (mode == HOP_CLOVINV ? 0.0 : spin);
    return (double)op.g.Vh * (nr * per_rhs + 8.0 * 12.0 * 4.0 + 72.0 * 4.0);
}

static bool bf16_ok(const DiracOp &op, const void *in, const void *z, int nr) {
    const bool aligned = ((reinterpret_cast<uintptr_t>(in) | reinterpret_cast<uintptr_t>(z) |
                           reinterpret_cast<uintptr_t>(op.L32w) | reinterpret_cast<uintptr_t>(op.C32w) |
                           reinterpret_cast<uintptr_t>(op.C32wA)) & 15) == 0;
    return aligned && nr % 32 == 0 && nr >= 32 && nr <= 256 && (nr & (nr - 1)) == 0 &&
           op.g.Vh * (nr / 32) < (1L << 30);
}

void hop_bf16(const DiracOp &op, int p, HopMode mode, __nv_bfloat162 *out, const __nv_bfloat162 *in,
              const __nv_bfloat162 *z, int nr, cudaStream_t s) {
    LAPH_REQUIRE(mode == HOP_CLOVINV || mode == HOP_CLOVINV_XPAY || mode == HOP_APPLY,
                 "BF16 hop supports the clover-inverse and apply modes");
    LAPH_REQUIRE(bf16_ok(op, in, z, nr), "BF16 hop needs 16-byte aligned operands and 32, 64, 128 or 256 "
                                         "right-hand sides");
    const float hws = (float)op.hw[0], hwt = (float)op.hw[3];
    prof_begin("dslash_bf16", s);
    const bool two = hop3_rpt_max() == 2 && nr % 64 == 0;
    if (mode == HOP_APPLY)
        two ? (void)launch_hop3<HOP_APPLY, 2, 2, 0>(op, p, hws, hwt, out, in, z, nr, s)
            : (void)launch_hop3<HOP_APPLY, 2, 1, 0>(op, p, hws, hwt, out, in, z, nr, s);
    else if (mode == HOP_CLOVINV)
        two ? (void)launch_hop3<HOP_CLOVINV, 2, 2, 0>(op, p, hws, hwt, out, in, (const __nv_bfloat162 *)nullptr,
                                                          nr, s)
            : (void)launch_hop3<HOP_CLOVINV, 2, 1, 0>(op, p, hws, hwt, out, in, (const __nv_bfloat162 *)nullptr,
                                                          nr, s);
    else
        two ? (void)launch_hop3<HOP_CLOVINV_XPAY, 2, 2, 0>(op, p, hws, hwt, out, in, z, nr, s)
            : (void)launch_hop3<HOP_CLOVINV_XPAY, 2, 1, 0>(op, p, hws, hwt, out, in, z, nr, s);
    LAPH_LAUNCH_CHECK();
    prof_end("dslash_bf16", s, hop_bytes_bf16(op, mode, nr), hop_flops(op, nr));
}

bool hop_bf16_xpay_dots(laph_ctx *ctx, const DiracOp &op, int p, __nv_bfloat162 *out, const __nv_bfloat162 *in,
                        const __nv_bfloat162 *z, int nr, c64 *red, cudaStream_t s) {
    const int rpt = (hop3_rpt_max() == 2 && nr == 64) ? 2 : 1;
    if (!bf16_ok(op, in, z, nr) || nr != 32 * rpt) return false;
    const float hws = (float)op.hw[0], hwt = (float)op.hw[3];
    prof_begin("dslash_bf16", s);
    if (rpt == 2)
        launch_hop3<HOP_CLOVINV_XPAY, 2, 2, 1>(op, p, hws, hwt, out, in, z, nr, s, ctx, red);
    else
        launch_hop3<HOP_CLOVINV_XPAY, 2, 1, 1>(op, p, hws, hwt, out, in, z, nr, s, ctx, red);
    LAPH_LAUNCH_CHECK();
    prof_end("dslash_bf16", s, hop_bytes_bf16(op, HOP_CLOVINV_XPAY, nr), hop_flops(op, nr));
    return true;
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

// Visiting order of the output sites of the copy-engine-fed hop: z-blocks of bz planes, and inside
// a block x (half index) fastest, then y, z, t.  The +-t neighbours of consecutive sites are then
// bz ns^2 / 2 sites apart instead of a whole slice (ns^3 / 2), which keeps a neighbour tile in L2
// from its first use to its last (24^3 slices, 32 RHS: 35 MB instead of 108 MB between the two);
// a block's two boundary planes are read once more (1 + 2 / bz of one pass over the input).
// bz = ns is the lexicographic order.
__global__ void order_kernel(Geom g, int bz, int *order) {
    long u = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= g.Vh) return;
    const int nxh = g.ns / 2;
    long v = u;
    const int xh = (int)(v % nxh); v /= nxh;
    const int y = (int)(v % g.ns); v /= g.ns;
    const int zi = (int)(v % bz); v /= bz;
    const int t = (int)(v % g.nt);
    const int z = (int)(v / g.nt) * bz + zi;
    order[u] = (int)((((long)t * g.ns + z) * g.ns + y) * nxh + xh);
}

static int hop_zblock(const Geom &g) {
    static int env = -2;
    if (env == -2) {
        const char *e = getenv("LAPH_HOP_ZBLOCK");
        env = e ? atoi(e) : -1;
    }
    int bz = env >= 0 ? env : 8;
    if (bz <= 0 || g.ns % bz != 0) bz = g.ns;
    return bz;
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
    op.order = (int *)ws_get(ctx, "dirac:order", sizeof(int) * g.Vh);
    order_kernel<<<grid_for(g.Vh, 256), 256, 0, s>>>(g, hop_zblock(g), op.order);
    LAPH_LAUNCH_CHECK();
    links_w_kernel<<<grid_for(8 * g.Vh * 9, 256), 256, 0, s>>>(8 * g.Vh, op.L64, op.L32w);
    LAPH_LAUNCH_CHECK();
    clov_w_kernel<<<grid_for(4 * g.Vh, 256), 256, 0, s>>>(4 * g.Vh, op.cinv64, op.C32w);
    LAPH_LAUNCH_CHECK();
    clov_w_kernel<<<grid_for(4 * g.Vh, 256), 256, 0, s>>>(4 * g.Vh, op.clov64, op.C32wA);
    LAPH_LAUNCH_CHECK();
}

}  // namespace laph
