// The prepared Wilson-clover operator on the device and the even-odd
// multi-right-hand-side field layout used by the solvers.
//
// Field layout (solver internal): one parity half of nr right-hand sides,
//   f[cb][k][r], k = spin*3 + colour (12 complex), r = 0..nr-1 (fastest).
// A thread owns one (cb, r): consecutive threads are consecutive right-hand
// sides of one site, so spinor loads coalesce and link / clover loads of a
// site are shared by the warp (broadcast).
//
// Links: L64 [parity][mu][cb][3][3] c64;  L32 [parity][mu][cb] 3 float4 holding
// the first two rows (12 reals) -- the third row of an SU(3) matrix is
// conj(row0 x row1).  Clover: per site two Hermitian 6x6 chiral blocks
// (spins {0,1} and {2,3} x colour), packed as 6 real diagonals followed by
// the 15 complex strictly-lower entries (row-major), 36 reals per block.
#pragma once
#include "common.cuh"

namespace laph {

constexpr int CLOV_BLOCK = 36;   // reals per packed 6x6 Hermitian block

struct DiracOp {
    Geom g;
    double m0, csw, xi;
    double hw[4];            // -1/2 w_mu
    c64 *L64 = nullptr;      // [2][4][Vh][9]
    float4 *L32 = nullptr;   // [2][4][Vh][3]
    __nv_bfloat162 *L16 = nullptr;  // [2][4][Vh][6] (12 reals as 6 bf16 pairs)
    double *clov64 = nullptr;  // A       [2][Vh][2][36]
    double *cinv64 = nullptr;  // A^{-1}  [2][Vh][2][36]
    float *cinv32 = nullptr;   // A^{-1}  [2][Vh][2][36]
    __nv_bfloat16 *cinv16 = nullptr;  // A^{-1} [2][Vh][2][36]
    // FP32 inner-operator operands in packed form (dslash_f32.cu)
    int *nbr = nullptr;       // [2][Vh][8] neighbour table, sign-folded
    int *order = nullptr;     // [Vh] visiting order of the output sites (z-blocked), see dslash_f32.cu
    float4 *L32w = nullptr;   // [2][4][Vh][9] (re, re, im, im)
    float *C32w = nullptr;    // [2][Vh][2][72] clover inverse
    float *C32wA = nullptr;   // [2][Vh][2][72] clover A (full-lattice K for the learned solver)
};

// Builds nbr, L32w and C32w from L64 and cinv64 (called by prepare_dirac).
void prepare_f32_operands(laph_ctx *ctx, DiracOp &op, cudaStream_t s);

// Builds links/clover on the device from ABI links [V][4][3][3] c64 (device pointer).
DiracOp prepare_dirac(laph_ctx *ctx, const Geom &g, const c64 *links, double m0, double csw, double xi,
                      cudaStream_t s, bool need_bf16 = false);

// Kernel modes of the hopping term D_{p pbar} (fused diagonal part):
enum HopMode {
    HOP_CLOVINV = 0,       // out = A_pp^{-1} D in
    HOP_CLOVINV_XPAY = 1,  // out = z - A_pp^{-1} D in
    HOP_APPLY = 2,         // out = A_pp xp + D in             (K restricted to parity p)
    HOP_RESID = 3,         // out = z - (A_pp xp + D in)       (residual b - K x)
};

// Launches the hopping kernel for output parity p on nr right-hand sides.
// T = double (FP64 links/clover) or float (FP32 compressed links, FP32 clover inverse).
template <typename T>
void hop(const DiracOp &op, int p, HopMode mode, cpx<T> *out, const cpx<T> *in, const cpx<T> *z,
         const cpx<T> *xp, int nr, cudaStream_t s);

// FP32 hop with the packed operands of prepare_f32_operands (modes HOP_CLOVINV and HOP_CLOVINV_XPAY).
// Throws LAPH_ERR_TIMEOUT (and clears the flag) when a TMA-fed stencil launch gave up waiting for a copy.
void hop_timeout_check(cudaStream_t s);
void hop_f32(const DiracOp &op, int p, HopMode mode, cpx<float> *out, const cpx<float> *in, const cpx<float> *z,
             int nr, cudaStream_t s);
// The xpay hop out = z - A_pp^{-1} D in with the inner products <out, z> and <out, out> of every
// right-hand side fused into its epilogue: red[0][r] = <out, z>, red[1][r] = <out, out>.
// Returns false (launching nothing) where the fused form is not available for this shape.
bool hop_f32_xpay_dots(laph_ctx *ctx, const DiracOp &op, int p, cpx<float> *out, const cpx<float> *in,
                       const cpx<float> *z, int nr, cpx<double> *red, cudaStream_t s);

// The same with <rhat, out> (the coded shadow vector of blas.cuh, rcode [Vh][nr] packed words) fused
// instead: red[0][r] = <rhat, out>.
bool hop_f32_xpay_rdot(laph_ctx *ctx, const DiracOp &op, int p, cpx<float> *out, const cpx<float> *in,
                       const cpx<float> *z, int nr, const uint32_t *rcode, cpx<double> *red, cudaStream_t s);

// BF16-stored spinors ([cb][12][nr] bf162: one complex per element), FP32 links and clover inverse, FP32
// arithmetic: the copy-engine-fed kernel of hop_f32 reading and writing BF16 tiles.  nr must be 32, 64,
// 128 or 256.  The xpay form with the fused <out, z>, <out, out> returns false where unavailable.
void hop_bf16(const DiracOp &op, int p, HopMode mode, __nv_bfloat162 *out, const __nv_bfloat162 *in,
              const __nv_bfloat162 *z, int nr, cudaStream_t s);
bool hop_bf16_xpay_dots(laph_ctx *ctx, const DiracOp &op, int p, __nv_bfloat162 *out, const __nv_bfloat162 *in,
                        const __nv_bfloat162 *z, int nr, cpx<double> *red, cudaStream_t s);

// Multiplies a parity half by A_pp^{-1} (T precision).
template <typename T>
void clov_inv_apply(const DiracOp &op, int p, cpx<T> *out, const cpx<T> *in, int nr, cudaStream_t s);

// ABI full-lattice fields [nrhs][V][12] c64 <-> internal parity halves [Vh][12][nr].
// `first` selects the first right-hand side of the block, `nr` the block size.
void fields_to_eo(const Geom &g, const c64 *abi, int first, int nr, c64 *even, c64 *odd, cudaStream_t s);
void eo_to_fields(const Geom &g, const c64 *even, const c64 *odd, int first, int nr, c64 *abi, cudaStream_t s);

}  // namespace laph
