// Multi-RHS BLAS-1 kernels and the per-RHS BiCGStab scalar updates.
#include <cmath>

#include "blas.cuh"

namespace laph {

RedPlan red_plan(laph_ctx *ctx, long nrows, int nr) {
    LAPH_REQUIRE(nr >= 1 && nr <= 256, "right-hand-side block must be 1..256");
    RedPlan p;
    p.nr = nr;
    p.rpb = 1;
    while (nr * p.rpb * 2 <= 256) p.rpb *= 2;
    p.block = nr * p.rpb;
    long want = (nrows + p.rpb - 1) / p.rpb;
    long cap = 8L * (ctx->sm_count > 0 ? ctx->sm_count : 152);   // enough warps to keep the loads in flight
    p.grid = (unsigned)(want < cap ? (want < 1 ? 1 : want) : cap);
    return p;
}

// ------------------------------------------------------------------ reductions
// Each thread accumulates its rows in the precision of the data (Body::Acc: FP32 for the
// inner solver, FP64 for the outer one; FP64 arithmetic is scarce on this GPU), then the
// block tree and the cross-block sum run in FP64.
template <int NRED, class Body>
__global__ void red_kernel(long nrows, int nr, int rpb, Body body, c64 *partial) {
    using Acc = typename Body::Acc;
    extern __shared__ c64 sm[];
    const int tid = threadIdx.x, bd = blockDim.x;
    const int r = tid % nr, row0 = tid / nr;
    Acc acc[NRED];
#pragma unroll
    for (int k = 0; k < NRED; ++k) acc[k] = {0, 0};
    // two rows per step (Body::two issues both rows' loads before either row's stores)
    const long step = (long)gridDim.x * rpb;
    long row = (long)blockIdx.x * rpb + row0;
    for (; row + step < nrows; row += 2 * step) body.two(row * nr + r, (row + step) * nr + r, r, acc);
    if (row < nrows) body(row * nr + r, r, acc);
#pragma unroll
    for (int k = 0; k < NRED; ++k) sm[k * bd + tid] = cvt<double>(acc[k]);
    __syncthreads();
    for (int st = rpb / 2; st > 0; st >>= 1) {
        if (row0 < st)
#pragma unroll
            for (int k = 0; k < NRED; ++k) sm[k * bd + tid] += sm[k * bd + tid + st * nr];
        __syncthreads();
    }
    if (row0 == 0)
#pragma unroll
        for (int k = 0; k < NRED; ++k) partial[((long)blockIdx.x * NRED + k) * nr + r] = sm[k * bd + r];
}

// out[k][r] = sum_b partial[b][k][r], one block per (k, r), fixed order.
__global__ void red_final(const c64 *partial, int nblk, int nred, int nr, c64 *out) {
    __shared__ c64 sm[256];
    int kr = blockIdx.x;
    int k = kr / nr, r = kr % nr;
    c64 a{0.0, 0.0};
    for (int b = threadIdx.x; b < nblk; b += blockDim.x) a += partial[((long)b * nred + k) * nr + r];
    sm[threadIdx.x] = a;
    __syncthreads();
    for (int st = blockDim.x / 2; st > 0; st >>= 1) {
        if ((int)threadIdx.x < st) sm[threadIdx.x] += sm[threadIdx.x + st];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[k * nr + r] = sm[0];
}

template <int NRED, class Body>
static void run_reduce(laph_ctx *ctx, const RedPlan &pl, long nrows, const Body &body, c64 *out, cudaStream_t s,
                       const char *family = nullptr, double bytes = 0.0) {
    c64 *partial = (c64 *)ws_get(ctx, "red:partial", sizeof(c64) * pl.grid * NRED * pl.nr);
    size_t shm = sizeof(c64) * NRED * pl.block;
    const char *fam = family ? family : sizeof(typename Body::Acc) == 8 ? "blas_fp32" : "blas_fp64";
    prof_begin(fam, s);
    red_kernel<NRED, Body><<<pl.grid, pl.block, shm, s>>>(nrows, pl.nr, pl.rpb, body, partial);
    LAPH_LAUNCH_CHECK();
    red_final<<<NRED * pl.nr, 256, 0, s>>>(partial, (int)pl.grid, NRED, pl.nr, out);
    LAPH_LAUNCH_CHECK();
    prof_end(fam, s, bytes, 0.0);
}

void red_final_sum(const c64 *partial, int nblk, int nred, int nr, c64 *out, cudaStream_t s) {
    red_final<<<nred * nr, 256, 0, s>>>(partial, nblk, nred, nr, out);
    LAPH_LAUNCH_CHECK();
}

template <typename T>
struct Dots1 {
    using Acc = cpx<T>;
    const cpx<T> *a0, *b0;
    __device__ void operator()(long i, int, Acc *acc) const { acc[0] += cmul_conj(a0[i], b0[i]); }
    __device__ void two(long i, long j, int k, Acc *acc) const {
        (*this)(i, k, acc);
        (*this)(j, k, acc);
    }
};
template <typename T>
struct Dots2 {
    using Acc = cpx<T>;
    const cpx<T> *a0, *b0, *a1, *b1;
    __device__ void operator()(long i, int, Acc *acc) const {
        acc[0] += cmul_conj(a0[i], b0[i]);
        acc[1] += cmul_conj(a1[i], b1[i]);
    }
    __device__ void two(long i, long j, int k, Acc *acc) const {
        (*this)(i, k, acc);
        (*this)(j, k, acc);
    }
};
template <typename T>
struct Dots3 {
    using Acc = cpx<T>;
    const cpx<T> *a0, *b0, *a1, *b1, *a2, *b2;
    __device__ void operator()(long i, int, Acc *acc) const {
        acc[0] += cmul_conj(a0[i], b0[i]);
        acc[1] += cmul_conj(a1[i], b1[i]);
        acc[2] += cmul_conj(a2[i], b2[i]);
    }
    __device__ void two(long i, long j, int k, Acc *acc) const {
        (*this)(i, k, acc);
        (*this)(j, k, acc);
    }
};

template <typename T>
void mrhs_dots(laph_ctx *ctx, const RedPlan &pl, long nrows, int nred, const cpx<T> *a0, const cpx<T> *b0,
               const cpx<T> *a1, const cpx<T> *b1, const cpx<T> *a2, const cpx<T> *b2, c64 *out, cudaStream_t s) {
    const double by = 2.0 * nred * (double)nrows * pl.nr * sizeof(cpx<T>);   // two streams per product
    if (nred == 1)
        run_reduce<1>(ctx, pl, nrows, Dots1<T>{a0, b0}, out, s, nullptr, by);
    else if (nred == 2)
        run_reduce<2>(ctx, pl, nrows, Dots2<T>{a0, b0, a1, b1}, out, s, nullptr, by);
    else
        run_reduce<3>(ctx, pl, nrows, Dots3<T>{a0, b0, a1, b1, a2, b2}, out, s, nullptr, by);
}
template void mrhs_dots<float>(laph_ctx *, const RedPlan &, long, int, const c32 *, const c32 *, const c32 *,
                               const c32 *, const c32 *, const c32 *, c64 *, cudaStream_t);
template void mrhs_dots<double>(laph_ctx *, const RedPlan &, long, int, const c64 *, const c64 *, const c64 *,
                                const c64 *, const c64 *, const c64 *, c64 *, cudaStream_t);

// ------------------------------------------------------------------ elementwise
template <typename Tx, typename Ty>
__global__ void axpy_scaled_kernel(long n, int nr, const double *scale, const cpx<Tx> *x, cpx<Ty> *y) {
    long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double a = scale[i % nr];
    cpx<double> v = cvt<double>(y[i]) + a * cvt<double>(x[i]);
    y[i] = cvt<Ty>(v);
}

template <typename Tx, typename Ty>
void mrhs_axpy_scaled(long nrows, int nr, const double *scale, const cpx<Tx> *x, cpx<Ty> *y, cudaStream_t s) {
    long n = nrows * nr;
    prof_begin("blas_convert", s);
    axpy_scaled_kernel<Tx, Ty><<<grid_for(n, 256), 256, 0, s>>>(n, nr, scale, x, y);
    LAPH_LAUNCH_CHECK();
    prof_end("blas_convert", s, 0.0, 0.0);
}
template void mrhs_axpy_scaled<float, double>(long, int, const double *, const c32 *, c64 *, cudaStream_t);
template void mrhs_axpy_scaled<double, double>(long, int, const double *, const c64 *, c64 *, cudaStream_t);

template <typename Tx, typename Ty>
__global__ void copy_scaled_kernel(long n, int nr, const double *scale, const cpx<Tx> *x, cpx<Ty> *y) {
    long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double a = scale[i % nr];
    y[i] = cvt<Ty>(a * cvt<double>(x[i]));
}

template <typename Tx, typename Ty>
void mrhs_copy_scaled(long nrows, int nr, const double *scale, const cpx<Tx> *x, cpx<Ty> *y, cudaStream_t s) {
    long n = nrows * nr;
    prof_begin("blas_convert", s);
    copy_scaled_kernel<Tx, Ty><<<grid_for(n, 256), 256, 0, s>>>(n, nr, scale, x, y);
    LAPH_LAUNCH_CHECK();
    prof_end("blas_convert", s, 0.0, 0.0);
}
template void mrhs_copy_scaled<double, float>(long, int, const double *, const c64 *, c32 *, cudaStream_t);
template void mrhs_copy_scaled<float, double>(long, int, const double *, const c32 *, c64 *, cudaStream_t);
template void mrhs_copy_scaled<float, float>(long, int, const double *, const c32 *, c32 *, cudaStream_t);
template void mrhs_copy_scaled<double, double>(long, int, const double *, const c64 *, c64 *, cudaStream_t);

__global__ void sub_kernel(long n, const c64 *x, const c64 *y, c64 *z) {
    long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) z[i] = x[i] - y[i];
}
void mrhs_sub(long n, const c64 *x, const c64 *y, c64 *z, cudaStream_t s) {
    sub_kernel<<<grid_for(n, 256), 256, 0, s>>>(n, x, y, z);
    LAPH_LAUNCH_CHECK();
}

// ------------------------------------------------------------------ BiCGStab pieces
template <typename T>
__global__ void p_update_kernel(long n, int nr, BicgScalars sc, const cpx<T> *r, cpx<T> *p, const cpx<T> *v) {
    long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int k = (int)(i % nr);
    cpx<T> b = cvt<T>(sc.beta[k]), w = cvt<T>(sc.omega[k]);
    cpx<T> bp = p[i] - w * v[i];
    p[i] = r[i] + b * bp;
}
template <typename T>
void bicg_p_update(long nrows, int nr, const BicgScalars &sc, const cpx<T> *r, cpx<T> *p, const cpx<T> *v,
                   cudaStream_t s) {
    long n = nrows * nr;
    const char *fam = sizeof(T) == 4 ? "blas_fp32" : "blas_fp64";
    prof_begin(fam, s);
    p_update_kernel<T><<<grid_for(n, 256), 256, 0, s>>>(n, nr, sc, r, p, v);
    LAPH_LAUNCH_CHECK();
    prof_end(fam, s, 4.0 * n * sizeof(cpx<T>), 0.0);   // read r, p, v; write p
}

template <typename T>
__global__ void s_update_kernel(long n, int nr, BicgScalars sc, const cpx<T> *r, const cpx<T> *v, cpx<T> *sv) {
    long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    cpx<T> a = cvt<T>(sc.alpha[i % nr]);
    sv[i] = r[i] - a * v[i];
}
template <typename T>
void bicg_s_update(long nrows, int nr, const BicgScalars &sc, const cpx<T> *r, const cpx<T> *v, cpx<T> *sv,
                   cudaStream_t s) {
    long n = nrows * nr;
    const char *fam = sizeof(T) == 4 ? "blas_fp32" : "blas_fp64";
    prof_begin(fam, s);
    s_update_kernel<T><<<grid_for(n, 256), 256, 0, s>>>(n, nr, sc, r, v, sv);
    LAPH_LAUNCH_CHECK();
    prof_end(fam, s, 3.0 * n * sizeof(cpx<T>), 0.0);   // read r, v; write s
}

template <typename T>
struct XRBody {
    BicgScalars sc;
    cpx<T> *x;
    const cpx<T> *p, *sv, *t;
    cpx<T> *r;
    const cpx<T> *rhat;
    using Acc = cpx<T>;
    __device__ void operator()(long i, int k, Acc *acc) const {
        cpx<T> a = cvt<T>(sc.alpha[k]), w = cvt<T>(sc.omega[k]);
        x[i] = x[i] + a * p[i] + w * sv[i];
        cpx<T> rn = sv[i] - w * t[i];
        r[i] = rn;
        acc[0] += cmul_conj(rhat[i], rn);
        acc[1] += cmul_conj(rn, rn);
    }
    __device__ void two(long i, long j, int k, Acc *acc) const {
        const cpx<T> a = cvt<T>(sc.alpha[k]), w = cvt<T>(sc.omega[k]);
        const cpx<T> xi = x[i], pi = p[i], si = sv[i], ti = t[i], hi = rhat[i];
        const cpx<T> xj = x[j], pj = p[j], sj = sv[j], tj = t[j], hj = rhat[j];
        const cpx<T> ri = si - w * ti, rj = sj - w * tj;
        x[i] = xi + a * pi + w * si;
        x[j] = xj + a * pj + w * sj;
        r[i] = ri;
        r[j] = rj;
        acc[0] += cmul_conj(hi, ri);
        acc[1] += cmul_conj(ri, ri);
        acc[0] += cmul_conj(hj, rj);
        acc[1] += cmul_conj(rj, rj);
    }
};

template <typename T>
void bicg_xr_update_reduce(laph_ctx *ctx, const RedPlan &pl, long nrows, const BicgScalars &sc, cpx<T> *x,
                           const cpx<T> *p, const cpx<T> *sv, const cpx<T> *t, cpx<T> *r, const cpx<T> *rhat,
                           c64 *red, cudaStream_t s) {
    // read x, p, s, t, rhat; write x, r
    run_reduce<2>(ctx, pl, nrows, XRBody<T>{sc, x, p, sv, t, r, rhat}, red, s, nullptr,
                  7.0 * nrows * pl.nr * sizeof(cpx<T>));
}

template void bicg_p_update<float>(long, int, const BicgScalars &, const c32 *, c32 *, const c32 *, cudaStream_t);
template void bicg_p_update<double>(long, int, const BicgScalars &, const c64 *, c64 *, const c64 *, cudaStream_t);
template void bicg_s_update<float>(long, int, const BicgScalars &, const c32 *, const c32 *, c32 *, cudaStream_t);
template void bicg_s_update<double>(long, int, const BicgScalars &, const c64 *, const c64 *, c64 *, cudaStream_t);
template void bicg_xr_update_reduce<float>(laph_ctx *, const RedPlan &, long, const BicgScalars &, c32 *, const c32 *,
                                           const c32 *, const c32 *, c32 *, const c32 *, c64 *, cudaStream_t);
template void bicg_xr_update_reduce<double>(laph_ctx *, const RedPlan &, long, const BicgScalars &, c64 *, const c64 *,
                                            const c64 *, const c64 *, c64 *, const c64 *, c64 *, cudaStream_t);

// ------------------------------------------------------------------ BF16-stored vectors
// Inner vectors of LAPH_SOLVE_MIXED_BF16: one complex per __nv_bfloat162, FP32 arithmetic; the
// iterate x stays FP32.  Same element order as the FP32 fields (element i is right-hand side i % nr).
__device__ __forceinline__ c32 bfl(bf2 v) {
    const float2 f = __bfloat1622float2(v);
    return c32{f.x, f.y};
}
__device__ __forceinline__ bf2 bfs(c32 v) { return __float22bfloat162_rn(make_float2(v.re, v.im)); }

__global__ void bf_p_update_kernel(long n, int nr, BicgScalars sc, const bf2 *r, bf2 *p, const bf2 *v) {
    long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int k = (int)(i % nr);
    const c32 b = cvt<float>(sc.beta[k]), w = cvt<float>(sc.omega[k]);
    p[i] = bfs(bfl(r[i]) + b * (bfl(p[i]) - w * bfl(v[i])));
}
void bicg_p_update_bf16(long nrows, int nr, const BicgScalars &sc, const bf2 *r, bf2 *p, const bf2 *v,
                        cudaStream_t s) {
    long n = nrows * nr;
    prof_begin("blas_bf16", s);
    bf_p_update_kernel<<<grid_for(n, 256), 256, 0, s>>>(n, nr, sc, r, p, v);
    LAPH_LAUNCH_CHECK();
    prof_end("blas_bf16", s, 4.0 * n * sizeof(bf2), 0.0);
}

__global__ void bf_s_update_kernel(long n, int nr, BicgScalars sc, const bf2 *r, const bf2 *v, bf2 *sv) {
    long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const c32 a = cvt<float>(sc.alpha[i % nr]);
    sv[i] = bfs(bfl(r[i]) - a * bfl(v[i]));
}
void bicg_s_update_bf16(long nrows, int nr, const BicgScalars &sc, const bf2 *r, const bf2 *v, bf2 *sv,
                        cudaStream_t s) {
    long n = nrows * nr;
    prof_begin("blas_bf16", s);
    bf_s_update_kernel<<<grid_for(n, 256), 256, 0, s>>>(n, nr, sc, r, v, sv);
    LAPH_LAUNCH_CHECK();
    prof_end("blas_bf16", s, 3.0 * n * sizeof(bf2), 0.0);
}

// conj(a) b summed per right-hand side
struct BfDots1 {
    using Acc = c32;
    const bf2 *a0, *b0;
    __device__ void operator()(long i, int, Acc *acc) const { acc[0] += cmul_conj(bfl(a0[i]), bfl(b0[i])); }
    __device__ void two(long i, long j, int k, Acc *acc) const {
        const c32 ai = bfl(a0[i]), bi = bfl(b0[i]), aj = bfl(a0[j]), bj = bfl(b0[j]);
        acc[0] += cmul_conj(ai, bi);
        acc[0] += cmul_conj(aj, bj);
    }
};
// x += alpha p + omega s (x FP32); r = s - omega t stored in BF16; <rhat, r>, <r, r> of the stored r
struct BfXR {
    BicgScalars sc;
    c32 *x;
    const bf2 *p, *sv, *t;
    bf2 *r;
    const bf2 *rhat;
    using Acc = c32;
    __device__ void operator()(long i, int k, Acc *acc) const {
        const c32 a = cvt<float>(sc.alpha[k]), w = cvt<float>(sc.omega[k]);
        const c32 si = bfl(sv[i]);
        x[i] = x[i] + a * bfl(p[i]) + w * si;
        const bf2 rs = bfs(si - w * bfl(t[i]));
        r[i] = rs;
        const c32 rn = bfl(rs);
        acc[0] += cmul_conj(bfl(rhat[i]), rn);
        acc[1] += cmul_conj(rn, rn);
    }
    __device__ void two(long i, long j, int k, Acc *acc) const {
        (*this)(i, k, acc);
        (*this)(j, k, acc);
    }
};

void mrhs_dots_bf16(laph_ctx *ctx, const RedPlan &pl, long nrows, const bf2 *a, const bf2 *b, c64 *out,
                    cudaStream_t s) {
    run_reduce<1>(ctx, pl, nrows, BfDots1{a, b}, out, s, "blas_bf16", 2.0 * nrows * pl.nr * sizeof(bf2));
}
void bicg_xr_update_reduce_bf16(laph_ctx *ctx, const RedPlan &pl, long nrows, const BicgScalars &sc, c32 *x,
                                const bf2 *p, const bf2 *sv, const bf2 *t, bf2 *r, const bf2 *rhat, c64 *red,
                                cudaStream_t s) {
    run_reduce<2>(ctx, pl, nrows, BfXR{sc, x, p, sv, t, r, rhat}, red, s, "blas_bf16",
                  (double)nrows * pl.nr * (5.0 * sizeof(bf2) + 2.0 * sizeof(c32)));
}

__global__ void bf_from64_kernel(long n, int nr, const double *scale, const c64 *x, bf2 *y) {
    long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double a = scale[i % nr];
    y[i] = bfs(c32{(float)(a * x[i].re), (float)(a * x[i].im)});
}
void mrhs_copy_scaled_bf16(long nrows, int nr, const double *scale, const c64 *x, bf2 *y, cudaStream_t s) {
    long n = nrows * nr;
    prof_begin("blas_convert", s);
    bf_from64_kernel<<<grid_for(n, 256), 256, 0, s>>>(n, nr, scale, x, y);
    LAPH_LAUNCH_CHECK();
    prof_end("blas_convert", s, 0.0, 0.0);
}

// ------------------------------------------------------------------ generated shadow vector
// code[cb][r] = packed rhat_quant of the 12 components of site cb, right-hand side r
__global__ void rhat_pack_kernel(long nsite, int nr, const c32 *__restrict__ r, uint32_t *__restrict__ code) {
    const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= nsite * nr) return;
    const long cb = idx / nr, k = idx - cb * nr;
    uint32_t w = 0;
#pragma unroll
    for (int c = 0; c < 12; ++c) {
        const c32 v = r[(cb * 12 + c) * nr + k];
        w |= rhat_quant(v.re, v.im) << (2 * c);
    }
    code[idx] = w;
}

struct RhatDots {
    const c32 *v;
    const uint32_t *code;
    int nr;
    using Acc = c32;
    __device__ void operator()(long i, int, Acc *acc) const {
        const c32 w = v[i];
        acc[0] += rhat_conj_mul(rhat_code_at(code, i, nr), w);
        acc[1] += cmul_conj(w, w);
    }
    __device__ void two(long i, long j, int k, Acc *acc) const {
        (*this)(i, k, acc);
        (*this)(j, k, acc);
    }
};
void mrhs_rhat_dots(laph_ctx *ctx, const RedPlan &pl, long nrows, const c32 *v, const uint32_t *code, c64 *red,
                    cudaStream_t s) {
    run_reduce<2>(ctx, pl, nrows, RhatDots{v, code, pl.nr}, red, s, nullptr,
                  (double)nrows * pl.nr * (sizeof(c32) + 4.0 / 12.0));
}
void mrhs_rhat_init(laph_ctx *ctx, const RedPlan &pl, long nrows, const c32 *r, uint32_t *code, c64 *red,
                    cudaStream_t s) {
    const long nsite = nrows / 12;
    rhat_pack_kernel<<<grid_for(nsite * pl.nr, 256), 256, 0, s>>>(nsite, pl.nr, r, code);
    LAPH_LAUNCH_CHECK();
    mrhs_rhat_dots(ctx, pl, nrows, r, code, red, s);
}

struct XRGenBody {
    BicgScalars sc;
    c32 *x;
    const c32 *p, *sv, *t;
    c32 *r;
    const uint32_t *code;
    int nr;
    using Acc = c32;
    __device__ void operator()(long i, int k, Acc *acc) const {
        const c32 a = cvt<float>(sc.alpha[k]), w = cvt<float>(sc.omega[k]);
        const c32 si = sv[i];
        x[i] = x[i] + a * p[i] + w * si;
        const c32 rn = si - w * t[i];
        r[i] = rn;
        acc[0] += rhat_conj_mul(rhat_code_at(code, i, nr), rn);
        acc[1] += cmul_conj(rn, rn);
    }
    __device__ void two(long i, long j, int k, Acc *acc) const {
        const c32 a = cvt<float>(sc.alpha[k]), w = cvt<float>(sc.omega[k]);
        const c32 xi = x[i], pi = p[i], si = sv[i], ti = t[i];
        const c32 xj = x[j], pj = p[j], sj = sv[j], tj = t[j];
        const uint32_t qi = rhat_code_at(code, i, nr), qj = rhat_code_at(code, j, nr);
        const c32 ri = si - w * ti, rj = sj - w * tj;
        x[i] = xi + a * pi + w * si;
        x[j] = xj + a * pj + w * sj;
        r[i] = ri;
        r[j] = rj;
        acc[0] += rhat_conj_mul(qi, ri);
        acc[1] += cmul_conj(ri, ri);
        acc[0] += rhat_conj_mul(qj, rj);
        acc[1] += cmul_conj(rj, rj);
    }
};
void bicg_xr_update_reduce_gen(laph_ctx *ctx, const RedPlan &pl, long nrows, const BicgScalars &sc, c32 *x,
                               const c32 *p, const c32 *sv, const c32 *t, c32 *r, const uint32_t *code, c64 *red,
                               cudaStream_t s) {
    // read x, p, s, t and the codes; write x, r
    run_reduce<2>(ctx, pl, nrows, XRGenBody{sc, x, p, sv, t, r, code, pl.nr}, red, s, nullptr,
                  (6.0 * sizeof(c32) + 4.0 / 12.0) * nrows * pl.nr);
}

__device__ __forceinline__ c64 cdiv(c64 a, c64 b) {
    double d = norm2(b);
    return c64{(a.re * b.re + a.im * b.im) / d, (a.im * b.re - a.re * b.im) / d};
}

__device__ __forceinline__ void deactivate(const BicgScalars &sc, int k, int status) {
    sc.active[k] = 0;
    sc.status[k] = status;
    sc.alpha[k] = c64{0.0, 0.0};
    sc.omega[k] = c64{0.0, 0.0};
    sc.beta[k] = c64{0.0, 0.0};
}

__global__ void init_scalars_kernel(int nr, BicgScalars sc, const c64 *red_rr, double rel_tol) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nr) return;
    double rr = red_rr[k].re;
    sc.rho[k] = c64{rr, 0.0};   // <rhat, r> with rhat = r
    sc.alpha[k] = c64{1.0, 0.0};
    sc.omega[k] = c64{1.0, 0.0};
    sc.beta[k] = c64{rr, 0.0};  // (rho / rho_old)(alpha / omega) with rho_old = 1: p = r first
    sc.rr[k] = rr;
    sc.rr_stop[k] = rel_tol * rel_tol * rr;
    sc.iters[k] = 0;
    bool run = rr > 0.0 && isfinite(rr);
    sc.active[k] = run ? 1 : 0;
    sc.status[k] = run ? 0 : 1;
    if (!run) deactivate(sc, k, 1);
}
void bicg_init_scalars(int nr, const BicgScalars &sc, const c64 *red_rr, double rel_tol, cudaStream_t s) {
    init_scalars_kernel<<<grid_for(nr, 64), 64, 0, s>>>(nr, sc, red_rr, rel_tol);
    LAPH_LAUNCH_CHECK();
}

// coded shadow vector: rho = <rhat, r0>, rr = <r0, r0>
__global__ void init_scalars_gen_kernel(int nr, BicgScalars sc, const c64 *red, double rel_tol) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nr) return;
    const c64 rho = red[k];
    const double rr = red[nr + k].re;
    sc.rho[k] = rho;
    sc.alpha[k] = c64{1.0, 0.0};
    sc.omega[k] = c64{1.0, 0.0};
    sc.beta[k] = rho;   // (rho / rho_old)(alpha / omega) with rho_old = 1: p = r first
    sc.rr[k] = rr;
    sc.rr_stop[k] = rel_tol * rel_tol * rr;
    sc.iters[k] = 0;
    const bool run = rr > 0.0 && isfinite(rr) && norm2(rho) > 0.0;
    sc.active[k] = run ? 1 : 0;
    sc.status[k] = run ? 0 : (rr > 0.0 ? 2 : 1);
    if (!run) deactivate(sc, k, sc.status[k]);
}
void bicg_init_scalars_gen(int nr, const BicgScalars &sc, const c64 *red, double rel_tol, cudaStream_t s) {
    init_scalars_gen_kernel<<<grid_for(nr, 64), 64, 0, s>>>(nr, sc, red, rel_tol);
    LAPH_LAUNCH_CHECK();
}

// alpha = rho / <rhat, v>
__global__ void alpha_kernel(int nr, BicgScalars sc, const c64 *red) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nr || !sc.active[k]) return;
    sc.iters[k] += 1;
    c64 d = red[k];
    double dn = norm2(d);
    if (!(dn > 0.0) || !isfinite(dn) || dn < 1e-60 * sc.rr[k] * sc.rr[k]) { deactivate(sc, k, 2); return; }
    sc.alpha[k] = cdiv(sc.rho[k], d);
}
void bicg_alpha(int nr, const BicgScalars &sc, const c64 *red, cudaStream_t s) {
    alpha_kernel<<<grid_for(nr, 64), 64, 0, s>>>(nr, sc, red);
    LAPH_LAUNCH_CHECK();
}

// omega = <t, s> / <t, t>
__global__ void omega_kernel(int nr, BicgScalars sc, const c64 *red) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nr || !sc.active[k]) return;
    c64 ts = red[k];
    double tt = red[nr + k].re;
    if (!(tt > 0.0) || !isfinite(tt)) {
        // t = M s = 0 means s = 0: the half step already solved the system
        sc.omega[k] = c64{0.0, 0.0};
        return;
    }
    sc.omega[k] = c64{ts.re / tt, ts.im / tt};
}
void bicg_omega(int nr, const BicgScalars &sc, const c64 *red, cudaStream_t s) {
    omega_kernel<<<grid_for(nr, 64), 64, 0, s>>>(nr, sc, red);
    LAPH_LAUNCH_CHECK();
}

// rho_new = <rhat, r>, rr = <r, r>; beta = (rho_new / rho)(alpha / omega); convergence test
__global__ void rho_kernel(int nr, BicgScalars sc, const c64 *red) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nr || !sc.active[k]) return;
    c64 rn = red[k];
    double rr = red[nr + k].re;
    sc.rr[k] = rr;
    if (!isfinite(rr) || !isfinite(rn.re) || !isfinite(rn.im)) { deactivate(sc, k, 2); return; }
    if (rr <= sc.rr_stop[k]) { deactivate(sc, k, 1); return; }
    c64 w = sc.omega[k];
    if (norm2(w) == 0.0 || norm2(rn) == 0.0) { deactivate(sc, k, 2); return; }
    sc.beta[k] = cdiv(rn, sc.rho[k]) * cdiv(sc.alpha[k], w);
    sc.rho[k] = rn;
}
void bicg_rho(int nr, const BicgScalars &sc, const c64 *red, cudaStream_t s) {
    rho_kernel<<<grid_for(nr, 64), 64, 0, s>>>(nr, sc, red);
    LAPH_LAUNCH_CHECK();
}

}  // namespace laph
