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
void bicg_alpha(int nr, const BicgScalars &sc, const c64 *red, cudaStream_t s);
void bicg_omega(int nr, const BicgScalars &sc, const c64 *red, cudaStream_t s);
void bicg_rho(int nr, const BicgScalars &sc, const c64 *red, cudaStream_t s);

}  // namespace laph
