// Multi-right-hand-side BLAS-1 on parity-half fields f[row][r], row = cb*12 + k,
// r fastest.  Reductions are per right-hand side, accumulated in FP64, and
// deterministic: a fixed two-stage tree (block tree over rows with equal r,
// then a fixed-order sum over blocks).
#pragma once
#include "common.cuh"

namespace laph {

struct RedPlan {
    int nr;        // right-hand sides
    int rpb;       // rows per block (power of two)
    int block;     // nr * rpb threads
    unsigned grid; // blocks
};

RedPlan red_plan(laph_ctx *ctx, long nrows, int nr);

// out[k][r] (k < nred) = sum over rows of the k-th product; a and b pairs are (conj(a) b).
// Computes up to three dot products in one pass: pairs (a0,b0), (a1,b1), (a2,b2).
template <typename T>
void mrhs_dots(laph_ctx *ctx, const RedPlan &pl, long nrows, int nred, const cpx<T> *a0, const cpx<T> *b0,
               const cpx<T> *a1, const cpx<T> *b1, const cpx<T> *a2, const cpx<T> *b2, c64 *out, cudaStream_t s);

// out[k][r] = sum over blocks b of partial[b][k][r], in a fixed order (FP64).
void red_final_sum(const c64 *partial, int nblk, int nred, int nr, c64 *out, cudaStream_t s);

// y[row][r] = y + scale[r] * x   (x of type Tx, y of type Ty)
template <typename Tx, typename Ty>
void mrhs_axpy_scaled(long nrows, int nr, const double *scale, const cpx<Tx> *x, cpx<Ty> *y, cudaStream_t s);

// y[row][r] = x * scale[r]   (type conversion allowed)
template <typename Tx, typename Ty>
void mrhs_copy_scaled(long nrows, int nr, const double *scale, const cpx<Tx> *x, cpx<Ty> *y, cudaStream_t s);

// z = x - y (FP64)
void mrhs_sub(long n, const c64 *x, const c64 *y, c64 *z, cudaStream_t s);

// Shadow vector of the FP32 inner BiCGStab: any fixed vector not orthogonal to the first residual
// serves (van der Vorst 1992).  This one is the phase of r0 rounded to the nearest power of i,
// rhat = i^code, code in {0, 1, 2, 3}.  The codes of the 12 spin-colour components of one site
// and right-hand side are packed in one 32-bit word, code[cb][r] bits 2c and 2c + 1 (4 bytes per
// 96 bytes of FP32 spinor), so <rhat, v> can be formed in the stencil's epilogue and <rhat, r>
// in the update kernel at little traffic.  A hashed random phase (no storage at all) measured
// 40 % more iterations on a 24^3 x 128 lattice near the critical mass: its overlap with r is of
// order |r| / sqrt(N), against ||r0||_1 / sqrt(N) for the rounded phase of r0.
__host__ __device__ __forceinline__ uint32_t rhat_quant(float re, float im) {
    return fabsf(re) >= fabsf(im) ? (re >= 0.0f ? 0u : 2u) : (im >= 0.0f ? 1u : 3u);
}
// code of element i = row * nr + r of a [Vh * 12][nr] field, row = cb * 12 + c
__host__ __device__ __forceinline__ uint32_t rhat_code_at(const uint32_t *code, long i, int nr) {
    const long row = i / nr;
    const long r = i - row * nr;
    return (code[(row / 12) * nr + r] >> (2 * (int)(row % 12))) & 3u;
}
// conj(i^code) v
template <typename T>
__host__ __device__ __forceinline__ cpx<T> rhat_conj_mul(uint32_t code, cpx<T> v) {
    return code == 0 ? v : code == 1 ? cpx<T>{v.im, -v.re} : code == 2 ? cpx<T>{-v.re, -v.im} : cpx<T>{-v.im, v.re};
}

// BiCGStab building blocks (T = float or double); scalars per RHS live in `sc`.
// Per-RHS BiCGStab scalars (complex: K is not Hermitian) and flags.
// status: 0 running, 1 converged, 2 breakdown.
struct BicgScalars {
    c64 *rho, *alpha, *omega, *beta;
    double *rr, *rr_stop;
    int *active, *status, *iters;
};

template <typename T>
void bicg_p_update(long nrows, int nr, const BicgScalars &sc, const cpx<T> *r, cpx<T> *p, const cpx<T> *v,
                   cudaStream_t s);
template <typename T>
void bicg_s_update(long nrows, int nr, const BicgScalars &sc, const cpx<T> *r, const cpx<T> *v, cpx<T> *sv,
                   cudaStream_t s);
// x += alpha p + omega s; r = s - omega t; and reduces <rhat, r>, <r, r>
template <typename T>
void bicg_xr_update_reduce(laph_ctx *ctx, const RedPlan &pl, long nrows, const BicgScalars &sc, cpx<T> *x,
                           const cpx<T> *p, const cpx<T> *sv, const cpx<T> *t, cpx<T> *r, const cpx<T> *rhat,
                           c64 *red, cudaStream_t s);

// BF16-stored inner vectors (one complex per bf2), FP32 arithmetic, FP32 iterate x.
using bf2 = __nv_bfloat162;
void bicg_p_update_bf16(long nrows, int nr, const BicgScalars &sc, const bf2 *r, bf2 *p, const bf2 *v,
                        cudaStream_t s);
void bicg_s_update_bf16(long nrows, int nr, const BicgScalars &sc, const bf2 *r, const bf2 *v, bf2 *sv,
                        cudaStream_t s);
void bicg_xr_update_reduce_bf16(laph_ctx *ctx, const RedPlan &pl, long nrows, const BicgScalars &sc, cpx<float> *x,
                                const bf2 *p, const bf2 *sv, const bf2 *t, bf2 *r, const bf2 *rhat, c64 *red,
                                cudaStream_t s);
void mrhs_dots_bf16(laph_ctx *ctx, const RedPlan &pl, long nrows, const bf2 *a, const bf2 *b, c64 *out,
                    cudaStream_t s);
// y = bf16(scale[r] * x) from an FP64 field
void mrhs_copy_scaled_bf16(long nrows, int nr, const double *scale, const c64 *x, bf2 *y, cudaStream_t s);

void bicg_init_scalars(int nr, const BicgScalars &sc, const c64 *red_rr, double rel_tol, cudaStream_t s);
// the same with the coded shadow vector: red[0][r] = <rhat, r0>, red[1][r] = <r0, r0>
void bicg_init_scalars_gen(int nr, const BicgScalars &sc, const c64 *red, double rel_tol, cudaStream_t s);
// code [nrows / 12][nr] = the packed rhat_quant(r0); red[0][r] = <rhat, r0>, red[1][r] = <r0, r0>
void mrhs_rhat_init(laph_ctx *ctx, const RedPlan &pl, long nrows, const cpx<float> *r, uint32_t *code, c64 *red,
                    cudaStream_t s);
// red[0][r] = <rhat, v>, red[1][r] = <v, v> for the stored codes
void mrhs_rhat_dots(laph_ctx *ctx, const RedPlan &pl, long nrows, const cpx<float> *v, const uint32_t *code,
                    c64 *red, cudaStream_t s);
// x += alpha p + omega s; r = s - omega t; red = <rhat, r>, <r, r> with the coded rhat (FP32)
void bicg_xr_update_reduce_gen(laph_ctx *ctx, const RedPlan &pl, long nrows, const BicgScalars &sc, cpx<float> *x,
                               const cpx<float> *p, const cpx<float> *sv, const cpx<float> *t, cpx<float> *r,
                               const uint32_t *code, c64 *red, cudaStream_t s);
void bicg_alpha(int nr, const BicgScalars &sc, const c64 *red, cudaStream_t s);
void bicg_omega(int nr, const BicgScalars &sc, const c64 *red, cudaStream_t s);
void bicg_rho(int nr, const BicgScalars &sc, const c64 *red, cudaStream_t s);

}  // namespace laph
