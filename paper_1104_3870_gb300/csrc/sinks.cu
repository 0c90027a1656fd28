// Sink coefficients (Sec. IV: the quark-propagation coefficients
// V_s^dag Omega^{-1} V_s P^(b) rho are N_t N_v numbers per spin):
//   coef[i][t][alpha][n] = sum_{x in slice t, c} conj(V(t,n,x,c)) sol[i](t,x,alpha,c)
// One GEMM per time slice: (nv x 3 V3) conj-transposed eigenvectors times the
// (3 V3 x 4 nrhs) solution columns.  FP64, shared-memory tiled: a block owns a
// 16 (n) x 32 (i, alpha) tile and walks the 3 V3 reduction in 32-wide slabs.
#include <cstdlib>

#include "common.cuh"

namespace laph {

constexpr int SK_TN = 16, SK_TC = 32, SK_TK = 32;

__global__ void __launch_bounds__(256) sinks_kernel(Geom g, int nv, int ncol, const c64 *__restrict__ ev,
                                                    const c64 *__restrict__ sol, c64 *__restrict__ coef) {
    __shared__ c64 As[SK_TN][SK_TK + 1];
    __shared__ c64 Bs[SK_TK][SK_TC + 1];
    const int t = blockIdx.z;
    const int n0 = blockIdx.x * SK_TN, c0 = blockIdx.y * SK_TC;
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;   // ty: row n, tx: two columns
    const long K = 3 * g.V3;
    c64 acc0{0, 0}, acc1{0, 0};
    for (long k0 = 0; k0 < K; k0 += SK_TK) {
        // A tile: conj(V(t, n0+r, k0+kk))  (k = x*3 + c is contiguous in the eigenvector layout)
        for (int e = threadIdx.x; e < SK_TN * SK_TK; e += blockDim.x) {
            int r = e / SK_TK, kk = e % SK_TK;
            int n = n0 + r;
            long k = k0 + kk;
            c64 v{0, 0};
            if (n < nv && k < K) v = conj(ev[((long)t * nv + n) * K + k]);
            As[r][kk] = v;
        }
        // B tile: sol[i](t, x, alpha, c) for column j = i*4 + alpha, k = x*3 + c
        for (int e = threadIdx.x; e < SK_TK * SK_TC; e += blockDim.x) {
            int kk = e / SK_TC, j = e % SK_TC;
            int col = c0 + j;
            long k = k0 + kk;
            c64 v{0, 0};
            if (col < ncol && k < K) {
                int i = col / 4, a = col % 4;
                long x = k / 3;
                int c = (int)(k % 3);
                v = sol[(((long)i * g.V + (long)t * g.V3 + x) * 4 + a) * 3 + c];
            }
            Bs[kk][j] = v;
        }
        __syncthreads();
#pragma unroll 8
        for (int kk = 0; kk < SK_TK; ++kk) {
            c64 a = As[ty][kk];
            acc0 += a * Bs[kk][tx];
            acc1 += a * Bs[kk][tx + 16];
        }
        __syncthreads();
    }
    int n = n0 + ty;
    if (n < nv) {
        int cols[2] = {c0 + tx, c0 + tx + 16};
        c64 vals[2] = {acc0, acc1};
        for (int q = 0; q < 2; ++q) {
            if (cols[q] >= ncol) continue;
            int i = cols[q] / 4, a = cols[q] % 4;
            coef[(((long)i * g.nt + t) * 4 + a) * nv + n] = vals[q];
        }
    }
}

void sinks(const Geom &g, int nv, int nrhs, const c64 *ev, const c64 *sol, c64 *coef, cudaStream_t s) {
    int ncol = 4 * nrhs;
    dim3 grid((nv + SK_TN - 1) / SK_TN, (ncol + SK_TC - 1) / SK_TC, g.nt);
    prof_begin("sinks", s);
    sinks_kernel<<<grid, 256, 0, s>>>(g, nv, ncol, ev, sol, coef);
    LAPH_LAUNCH_CHECK();
    prof_end("sinks", s, 0.0, 8.0 * nv * (double)ncol * 3.0 * g.V3 * g.nt);
}

void sinks_tensor_core(laph_ctx *ctx, const Geom &g, const c64 *V, int nv, const c64 *X, int nrhs, c64 *coef,
                       cudaStream_t s);
void sinks_tc_check(cudaStream_t s);

// LAPH_SINKS_FP64=1 selects the FP64 CUDA-core kernel above instead of the tensor-core one
// (sinks_tc.cu), for comparisons.
static bool sinks_fp64_forced() {
    static int v = -1;
    if (v < 0) {
        const char *e = getenv("LAPH_SINKS_FP64");
        v = (e && atoi(e) == 1) ? 1 : 0;
    }
    return v == 1;
}

}  // namespace laph

using namespace laph;

extern "C" int laph_sinks(laph_ctx *ctx, const laph_lattice *lat, const void *evecs, int nv, const void *sol, int nrhs,
                          void *coef, void *stream) {
    return guard([&] {
        ctx_activate(ctx);
        Geom g = make_geom(lat);
        LAPH_REQUIRE(nv >= 1 && nv <= 3 * g.V3, "nv out of range");
        LAPH_REQUIRE(nrhs >= 0, "nrhs must be >= 0");
        if (nrhs == 0) return;
        LAPH_REQUIRE((long)g.nt * 65535 >= 0 && g.nt <= 65535, "nt too large");
        cudaStream_t s = as_stream(stream);
        const c64 *ev = (const c64 *)stage_in(ctx, evecs, sizeof(c64) * 3 * g.V3 * g.nt * (size_t)nv, "evecs", s);
        const c64 *x = (const c64 *)stage_in(ctx, sol, sizeof(c64) * 12 * g.V * (size_t)nrhs, "sinks_sol", s);
        StagedOut o = stage_out(ctx, coef, sizeof(c64) * (size_t)nrhs * g.nt * 4 * nv, "coef");
        if (sinks_fp64_forced()) {
            sinks(g, nv, nrhs, ev, x, (c64 *)o.dev, s);
        } else {
            sinks_tensor_core(ctx, g, ev, nv, x, nrhs, (c64 *)o.dev, s);
            sinks_tc_check(s);
        }
        o.commit(s);
    });
}
