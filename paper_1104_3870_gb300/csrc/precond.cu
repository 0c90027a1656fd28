// Learned gauge-covariant preconditioner: network layers, training, and the
// flexible GCR solve that uses it as a right preconditioner.
//
// Network (the paper has none; reading of the workload): L linear layers
// 1 -> C -> ... -> C -> 1 complex channels,
//   out_c(x) = sum_{c'} sum_{d=0..8} W[d][c][c'] (T_d in_{c'})(x),
//   T_0 = 1, T_{1+mu} psi(x) = s U_mu(x) psi(x+mu), T_{5+mu} psi(x) = s U_mu(x-mu)^dag psi(x-mu),
// W a 4x4 complex spin matrix (identity on colour), s = -1 across the time
// boundary.  Gauge covariant by construction: colour only meets links.
// Weights: layers in order, each [9][c_out][c_in][4][4] complex float (re, im).
//
// Fields of the network are full lattices in even-odd halves: channel c of a
// field f is f + c * 2 Vh 12 nr, parity p at + p Vh 12 nr, then [cb][12][nr].
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <vector>

#include "blas.cuh"
#include "dirac.cuh"
#include "solver.cuh"

namespace laph {

constexpr int NN_MAXC = 4;

// tensor-core layers (nn_tc.cu): nr a multiple of 32
bool nn_tc_ok(int nr, int cin, int cout);
void nn_layer_tensor_core(laph_ctx *ctx, const DiracOp &op, long Vh, int nr, int cin, int cout, const float2 *W,
                          const float2 *in, float2 *out, cudaStream_t s);
void nn_tc_check(cudaStream_t s);

struct NNShape {
    int nchan = 4, nlayers = 4;
    int cin(int l) const { return l == 0 ? 1 : nchan; }
    int cout(int l) const { return l == nlayers - 1 ? 1 : nchan; }
    long layer_size(int l) const { return 9L * cout(l) * cin(l) * 16; }   // complex entries
    long offset(int l) const {
        long o = 0;
        for (int k = 0; k < l; ++k) o += layer_size(k);
        return o;
    }
    long total() const { return offset(nlayers); }
};

__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 ri(float2 x) { return make_float2(-x.y, x.x); }     // i x
__device__ __forceinline__ float2 rmi(float2 x) { return make_float2(x.y, -x.x); }    // -i x
__device__ __forceinline__ float2 ffma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

// t = T_d psi for a full 4-spin spinor; u points to 9 float4 (re, re, im, im); dag: use U^dag.
__device__ __forceinline__ void transport12(const float4 *__restrict__ u, bool dag, float sgn, const float2 psi[12],
                                            float2 t[12]) {
#pragma unroll
    for (int s = 0; s < 4; ++s) {
        float2 h[3], r[3];
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            h[b] = psi[s * 3 + b];
            r[b] = dag ? rmi(h[b]) : ri(h[b]);
        }
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            float2 acc = f2(0.f, 0.f);
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                float4 e = __ldg(u + (dag ? b * 3 + a : a * 3 + b));
                acc = ffma(f2(e.x, e.y), h[b], acc);
                acc = ffma(f2(e.z, e.w), r[b], acc);
            }
            t[s * 3 + a] = f2(sgn * acc.x, sgn * acc.y);
        }
    }
}

// One layer for all output channels, weights staged in shared memory as float4 (re, re, im, im),
// [9][cout][cin][16].  One thread per (site, output channel c, RHS): since W[d][c][c'] acts on
// spin and T_d on colour and site, out_c = sum_d T_d (sum_{c'} W[d][c][c'] in_{c'}) — each thread
// mixes the input channels at the source site, then transports the mixed spinor once, with 12
// accumulators (not 12 cout), so many warps fit on an SM.  Thread index ((p Vh + cb) cout + c) nr + r.
__global__ void __launch_bounds__(128, 4) nn_layer2_kernel(const int *__restrict__ nbr, const float4 *__restrict__ L,
                                                        long Vh, int nr, int cin, int cout,
                                                        const float2 *__restrict__ W, const float2 *__restrict__ in,
                                                        float2 *__restrict__ out) {
    extern __shared__ float4 wsm[];
    const int nw = 9 * cout * cin * 16;
    for (int i = threadIdx.x; i < nw; i += blockDim.x) {
        float2 w = W[i];
        wsm[i] = make_float4(w.x, w.x, w.y, w.y);
    }
    __syncthreads();
    const long tid = (long)blockIdx.x * blockDim.x + threadIdx.x;
    const long sc = tid / nr;              // site * cout + c
    const int r = (int)(tid - sc * nr);
    const long site = sc / cout;           // p * Vh + cb
    const int c = (int)(sc - site * cout);
    if (site >= 2 * Vh) return;
    const int p = (int)(site / Vh);
    const long cb = site - (long)p * Vh;
    const long chan = 2 * Vh * 12 * (long)nr;
    const long half = Vh * 12 * (long)nr;
    const int *nb = nbr + site * 8;
    float2 acc[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) acc[k] = f2(0.f, 0.f);
    const long lplane = Vh * 9;
    for (int d = 0; d < 9; ++d) {
        long src_off;
        const float4 *u = nullptr;
        bool dag = false;
        float sgn = 1.f;
        if (d == 0) {
            src_off = (long)p * half + cb * 12 * nr;
        } else {
            const int mu = (d - 1) & 3;
            const bool fwdd = d <= 4;
            int j = __ldg(nb + (fwdd ? mu : 4 + mu));
            sgn = j < 0 ? -1.f : 1.f;
            j = j < 0 ? ~j : j;
            src_off = (long)(1 - p) * half + (long)j * 12 * nr;
            u = fwdd ? L + ((long)p * 4 + mu) * lplane + cb * 9 : L + ((long)(1 - p) * 4 + mu) * lplane + (long)j * 9;
            dag = !fwdd;
        }
        float2 y[12];
#pragma unroll
        for (int k = 0; k < 12; ++k) y[k] = f2(0.f, 0.f);
        for (int cp = 0; cp < cin; ++cp) {
            const float2 *sp = in + cp * chan + src_off + r;
            const float4 *w = wsm + ((d * cout + c) * cin + cp) * 16;
#pragma unroll
            for (int si = 0; si < 4; ++si) {
                float2 ps[3], ip[3];
#pragma unroll
                for (int col = 0; col < 3; ++col) {
                    ps[col] = sp[(long)(si * 3 + col) * nr];
                    ip[col] = ri(ps[col]);
                }
#pragma unroll
                for (int so = 0; so < 4; ++so) {
                    const float4 e = w[so * 4 + si];
                    const float2 rr = f2(e.x, e.y), ii = f2(e.z, e.w);
#pragma unroll
                    for (int col = 0; col < 3; ++col) {
                        y[so * 3 + col] = ffma(rr, ps[col], y[so * 3 + col]);
                        y[so * 3 + col] = ffma(ii, ip[col], y[so * 3 + col]);
                    }
                }
            }
        }
        if (d == 0) {
#pragma unroll
            for (int k = 0; k < 12; ++k) acc[k] = __fadd2_rn(acc[k], y[k]);
        } else {
            float2 t[12];
            transport12(u, dag, sgn, y, t);
#pragma unroll
            for (int k = 0; k < 12; ++k) acc[k] = __fadd2_rn(acc[k], t[k]);
        }
    }
    float2 *o = out + c * chan + (long)p * half + cb * 12 * nr + r;
#pragma unroll
    for (int k = 0; k < 12; ++k) o[(long)k * nr] = acc[k];
}

// W'[d][c'][c] = W[dbar][c][c']^dag (adjoint layer: swapped transports, conjugate-transposed spin matrices)
__global__ void nn_adjoint_weights(int cin, int cout, const float2 *W, float2 *Wa) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    int n = 9 * cout * cin * 16;
    if (i >= n) return;
    int e = i % 16, so = e / 4, si = e % 4;
    // adjoint layout [9][cin][cout][16] (its c_out = cin of W, its c_in = cout of W)
    int cp_adj = (i / 16) % cout;          // adjoint's input channel  (W's output channel)
    int c_adj = (i / (16 * cout)) % cin;   // adjoint's output channel (W's input channel)
    int d = i / (16 * cout * cin);
    const int dbar[9] = {0, 5, 6, 7, 8, 1, 2, 3, 4};
    // Wa[d][c_adj][cp_adj][so][si] = conj(W[dbar][cp_adj][c_adj][si][so])
    float2 w = W[((dbar[d] * cout + cp_adj) * cin + c_adj) * 16 + si * 4 + so];
    Wa[i] = f2(w.x, -w.y);
}

// ------------------------------------------------------------------ weight gradient
// dW[d][c][c'][so][si] = sum_{p, cb, r, col} g_c[so][col] conj((T_d a_{c'})[si][col]).
// Tiles of 32 (site, rhs) rows: the first 128 threads (32 rows x 4 channels) build the transported
// tile in shared memory, then each of the 256 threads owns one (c so, c' si) output and sums the tile.
constexpr int WG_ROWS = 32;   // 2 x 24 KB of shared tiles

__global__ void __launch_bounds__(256) nn_wgrad_kernel(const int *__restrict__ nbr, const float4 *__restrict__ L,
                                                       long Vh, int nr, int cin, int cout, int d,
                                                       const float2 *__restrict__ a, const float2 *__restrict__ g,
                                                       float2 *__restrict__ partial) {
    __shared__ float2 At[WG_ROWS][3][NN_MAXC * 4];
    __shared__ float2 Gt[WG_ROWS][3][NN_MAXC * 4];
    const long nrows = 2 * Vh * (long)nr;
    const long chan = 2 * Vh * 12 * (long)nr;
    const long half = Vh * 12 * (long)nr;
    const long lplane = Vh * 9;
    const int oi = threadIdx.x / 16, oj = threadIdx.x % 16;   // output entry (c so) x (c' si)
    float2 acc = f2(0.f, 0.f);
    for (long r0 = (long)blockIdx.x * WG_ROWS; r0 < nrows; r0 += (long)gridDim.x * WG_ROWS) {
        if (threadIdx.x < WG_ROWS * 4) {
            int row = threadIdx.x / 4, ch = threadIdx.x % 4;
            long gr = r0 + row;
            bool ok = gr < nrows;
            long site = ok ? gr / nr : 0;
            int r = ok ? (int)(gr - site * nr) : 0;
            int p = (int)(site / Vh);
            long cb = site - (long)p * Vh;
            if (ch < cin) {
                float2 t[12];
                if (ok) {
                    long src_off;
                    const float4 *u = nullptr;
                    bool dag = false;
                    float sgn = 1.f;
                    if (d == 0) {
                        src_off = (long)p * half + cb * 12 * nr;
                    } else {
                        int mu = (d - 1) & 3;
                        bool fwdd = d <= 4;
                        int j = __ldg(nbr + site * 8 + (fwdd ? mu : 4 + mu));
                        sgn = j < 0 ? -1.f : 1.f;
                        j = j < 0 ? ~j : j;
                        src_off = (long)(1 - p) * half + (long)j * 12 * nr;
                        u = fwdd ? L + ((long)p * 4 + mu) * lplane + cb * 9
                                 : L + ((long)(1 - p) * 4 + mu) * lplane + (long)j * 9;
                        dag = !fwdd;
                    }
                    float2 psi[12];
                    const float2 *s = a + ch * chan + src_off + r;
#pragma unroll
                    for (int k = 0; k < 12; ++k) psi[k] = s[(long)k * nr];
                    if (d == 0) {
#pragma unroll
                        for (int k = 0; k < 12; ++k) t[k] = psi[k];
                    } else {
                        transport12(u, dag, sgn, psi, t);
                    }
                } else {
#pragma unroll
                    for (int k = 0; k < 12; ++k) t[k] = f2(0.f, 0.f);
                }
#pragma unroll
                for (int sp = 0; sp < 4; ++sp)
#pragma unroll
                    for (int col = 0; col < 3; ++col) At[row][col][ch * 4 + sp] = t[sp * 3 + col];
            }
            if (ch < cout) {
                const float2 *s = g + ch * chan + (long)p * half + cb * 12 * nr + r;
#pragma unroll
                for (int sp = 0; sp < 4; ++sp)
#pragma unroll
                    for (int col = 0; col < 3; ++col) Gt[row][col][ch * 4 + sp] = ok ? s[(long)(sp * 3 + col) * nr] : f2(0.f, 0.f);
            }
        }
        __syncthreads();
        if (oi < cout * 4 && oj < cin * 4) {
            for (int row = 0; row < WG_ROWS; ++row)
#pragma unroll
                for (int col = 0; col < 3; ++col) {
                    float2 gv = Gt[row][col][oi], av = At[row][col][oj];
                    // acc += g * conj(a)
                    acc.x += gv.x * av.x + gv.y * av.y;
                    acc.y += gv.y * av.x - gv.x * av.y;
                }
        }
        __syncthreads();
    }
    if (oi < cout * 4 && oj < cin * 4) {
        int c = oi / 4, so = oi % 4, cp = oj / 4, si = oj % 4;
        partial[(long)blockIdx.x * (cout * cin * 16) + (c * cin + cp) * 16 + so * 4 + si] = acc;
    }
}

// grad[d][i] = sum_b partial[b][i] in FP64 and fixed order; one block per output entry.
__global__ void nn_wgrad_final(int nblk, int n, const float2 *partial, int d, c64 *grad) {
    __shared__ c64 sm[256];
    int i = blockIdx.x;
    c64 a{0, 0};
    for (int b = threadIdx.x; b < nblk; b += blockDim.x) {
        float2 v = partial[(long)b * n + i];
        a += c64{v.x, v.y};
    }
    sm[threadIdx.x] = a;
    __syncthreads();
    for (int st = blockDim.x / 2; st > 0; st >>= 1) {
        if ((int)threadIdx.x < st) sm[threadIdx.x] += sm[threadIdx.x + st];
        __syncthreads();
    }
    if (threadIdx.x == 0) grad[(long)d * n + i] = sm[0];
}

// Adam on the real and imaginary parts: gradient of Re w is 2 Re(dL/d conj w), of Im w is 2 Im.
__global__ void adam_kernel(long n, float2 *w, const c64 *grad, float2 *m, float2 *v, float lr, float b1, float b2,
                            float eps, float bc1, float bc2) {
    long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float gx = (float)(2.0 * grad[i].re), gy = (float)(2.0 * grad[i].im);
    float2 mm = m[i], vv = v[i];
    mm.x = b1 * mm.x + (1 - b1) * gx;
    mm.y = b1 * mm.y + (1 - b1) * gy;
    vv.x = b2 * vv.x + (1 - b2) * gx * gx;
    vv.y = b2 * vv.y + (1 - b2) * gy * gy;
    m[i] = mm;
    v[i] = vv;
    float2 ww = w[i];
    ww.x -= lr * (mm.x / bc1) / (sqrtf(vv.x / bc2) + eps);
    ww.y -= lr * (mm.y / bc1) / (sqrtf(vv.y / bc2) + eps);
    w[i] = ww;
}

// e = (y - phi) * scale[r]  (scale = 1 / (B ||phi_r||^2)), full fields
__global__ void nn_err_kernel(long n, int nr, const float2 *y, const float2 *phi, const double *scale, float2 *e) {
    long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float s = (float)scale[i % nr];
    float2 a = y[i], b = phi[i];
    e[i] = f2(s * (a.x - b.x), s * (a.y - b.y));
}

// ------------------------------------------------------------------ host side
struct Net {
    NNShape sh;
    const DiracOp *op;
    long Vh;
    int nr;
    laph_ctx *tc = nullptr;   // non-null: the layers run on the tensor cores (nn_tc.cu) where they can
};

static void launch_layer(const Net &net, int cin, int cout, const float2 *W, const float2 *in, float2 *out,
                         cudaStream_t s) {
    if (net.tc != nullptr && nn_tc_ok(net.nr, cin, cout)) {
        nn_layer_tensor_core(net.tc, *net.op, net.Vh, net.nr, cin, cout, W, in, out, s);
        return;
    }
    long n = 2 * net.Vh * net.nr * cout;
    size_t shm = sizeof(float4) * 9 * cin * cout * 16;
    if (shm > 48 * 1024) LAPH_CUDA(cudaFuncSetAttribute(nn_layer2_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
    prof_begin("nn_layer", s);
    nn_layer2_kernel<<<grid_for(n, 128), 128, shm, s>>>(net.op->nbr, net.op->L32w, net.Vh, net.nr, cin, cout, W, in, out);
    LAPH_LAUNCH_CHECK();
    prof_end("nn_layer", s, 0.0, 0.0);
}

// Forward pass; acts[l] receives the input of layer l (acts[0] = r must be filled), acts[L] the output.
static void net_forward(const Net &net, const float2 *W, std::vector<float2 *> &acts, cudaStream_t s) {
    for (int l = 0; l < net.sh.nlayers; ++l)
        launch_layer(net, net.sh.cin(l), net.sh.cout(l), W + net.sh.offset(l), acts[l], acts[l + 1], s);
}

// Backward pass from g = dL/d conj(output): accumulates dL/d conj(W) (FP64) into grad.
static void net_backward(laph_ctx *ctx, const Net &net, const float2 *W, const std::vector<float2 *> &acts, float2 *g,
                         float2 *gtmp, c64 *grad, cudaStream_t s) {
    const long nrows = 2 * net.Vh * net.nr;
    unsigned grid = (unsigned)std::min<long>((nrows + WG_ROWS - 1) / WG_ROWS, 4L * (ctx->sm_count ? ctx->sm_count : 152));
    float2 *partial = (float2 *)ws_get(ctx, "nn:partial", sizeof(float2) * grid * NN_MAXC * NN_MAXC * 16);
    float2 *Wa = (float2 *)ws_get(ctx, "nn:Wadj", sizeof(float2) * 9 * NN_MAXC * NN_MAXC * 16);
    float2 *gc = g, *go = gtmp;
    for (int l = net.sh.nlayers - 1; l >= 0; --l) {
        int cin = net.sh.cin(l), cout = net.sh.cout(l);
        int n = cout * cin * 16;
        c64 *gl = grad + net.sh.offset(l);
        prof_begin("nn_wgrad", s);
        for (int d = 0; d < 9; ++d) {
            nn_wgrad_kernel<<<grid, 256, 0, s>>>(net.op->nbr, net.op->L32w, net.Vh, net.nr, cin, cout, d, acts[l], gc,
                                                partial);
            LAPH_LAUNCH_CHECK();
            nn_wgrad_final<<<n, 256, 0, s>>>((int)grid, n, partial, d, gl);
            LAPH_LAUNCH_CHECK();
        }
        prof_end("nn_wgrad", s, 0.0, 0.0);
        if (l > 0) {
            nn_adjoint_weights<<<grid_for(9L * n, 256), 256, 0, s>>>(cin, cout, W + net.sh.offset(l), Wa);
            LAPH_LAUNCH_CHECK();
            launch_layer(net, cout, cin, Wa, gc, go, s);
            std::swap(gc, go);
        }
    }
}

// Full-lattice fields: ABI [n][V][12] c64 -> network layout (FP32), channel 0.
static void abi_to_net(const Geom &g, const c64 *abi, int first, int nr, float2 *out, c64 *tmp_e, c64 *tmp_o,
                       double *ones, cudaStream_t s) {
    fields_to_eo(g, abi, first, nr, tmp_e, tmp_o, s);
    long rows = g.Vh * 12;
    mrhs_copy_scaled<double, float>(rows, nr, ones, tmp_e, (c32 *)out, s);
    mrhs_copy_scaled<double, float>(rows, nr, ones, tmp_o, (c32 *)(out + g.Vh * 12 * (long)nr), s);
}

__global__ void fill_kernel(long n, double v, double *x) {
    long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) x[i] = v;
}

// y[i] += a[i % nr] x[i] with a complex coefficient per right-hand side (FP32 fields)
__global__ void caxpy_rhs_kernel(long n, int nr, const c64 *a, const float2 *x, float2 *y) {
    long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    c64 c = a[i % nr];
    float2 xv = x[i], yv = y[i];
    float cr = (float)c.re, ci = (float)c.im;
    y[i] = make_float2(yv.x + cr * xv.x - ci * xv.y, yv.y + cr * xv.y + ci * xv.x);
}

// Flexible GCR (restart R) for K x = b on full FP32 fields, right-preconditioned by the network:
// z_j = N(r), w_j = K z_j orthonormalised against w_0..w_{j-1} (classical Gram-Schmidt, two
// passes, applied to z_j as well), x += <w_j, r> z_j, r -= <w_j, r> w_j.  Returns iterations.
static int fgcr(laph_ctx *ctx, const Net &net, const float2 *W, const float2 *b, float2 *x, double tol, int maxiter,
                int restart, cudaStream_t s) {
    const int nr = net.nr;
    const long Vh = net.Vh;
    const long half = Vh * 12 * (long)nr, full = 2 * half;
    const long rows = 2 * Vh * 12;
    auto F = [&](const std::string &n, int k) { return (float2 *)ws_get(ctx, "fgcr:" + n + std::to_string(k), sizeof(float2) * full); };
    std::vector<float2 *> Z(restart), Wv(restart);
    for (int j = 0; j < restart; ++j) {
        Z[j] = F("z", j);
        Wv[j] = F("w", j);
    }
    float2 *r = F("r", 0);
    std::vector<float2 *> acts(net.sh.nlayers + 1);
    for (int l = 0; l <= net.sh.nlayers; ++l)
        acts[l] = (float2 *)ws_get(ctx, "nn:act" + std::to_string(l), sizeof(float2) * full * NN_MAXC);
    c64 *red = (c64 *)ws_get(ctx, "fgcr:red", sizeof(c64) * (restart + 2) * nr);
    c64 *coef = (c64 *)ws_get(ctx, "fgcr:coef", sizeof(c64) * (restart + 1) * nr);
    double *sc = (double *)ws_get(ctx, "fgcr:sc", sizeof(double) * nr);
    RedPlan pl = red_plan(ctx, rows, nr);
    std::vector<c64> hred(2 * nr), hc(nr), hgs;
    std::vector<double> hs(nr), rr0(nr);
    LAPH_CUDA(cudaMemcpyAsync(r, b, sizeof(float2) * full, cudaMemcpyDeviceToDevice, s));
    LAPH_CUDA(cudaMemsetAsync(x, 0, sizeof(float2) * full, s));
    auto dot = [&](const float2 *a, const float2 *bb) {
        mrhs_dots<float>(ctx, pl, rows, 1, (const c32 *)a, (const c32 *)bb, nullptr, nullptr, nullptr, nullptr, red, s);
        LAPH_CUDA(cudaMemcpyAsync(hred.data(), red, sizeof(c64) * nr, cudaMemcpyDeviceToHost, s));
        LAPH_CUDA(cudaStreamSynchronize(s));
    };
    auto axpy = [&](const std::vector<c64> &a, const float2 *xx, float2 *yy) {
        LAPH_CUDA(cudaMemcpyAsync(coef, a.data(), sizeof(c64) * nr, cudaMemcpyHostToDevice, s));
        caxpy_rhs_kernel<<<grid_for(full, 256), 256, 0, s>>>(full, nr, coef, xx, yy);
        LAPH_LAUNCH_CHECK();
    };
    dot(r, r);
    for (int k = 0; k < nr; ++k) rr0[k] = hred[k].re;
    std::vector<int> active(nr);
    for (int k = 0; k < nr; ++k) active[k] = rr0[k] > 0.0;
    int it = 0;
    std::vector<double> rr_cycle(rr0);
    while (it < maxiter) {
        if (it > 0) {
            // a restart cycle that gained less than 10% on every active right-hand side: stalled
            dot(r, r);
            bool gained = false;
            for (int k = 0; k < nr; ++k) {
                if (active[k] && hred[k].re < 0.81 * rr_cycle[k]) gained = true;
                rr_cycle[k] = hred[k].re;
            }
            if (!gained) return it;
        }
        for (int j = 0; j < restart && it < maxiter; ++j, ++it) {
            LAPH_CUDA(cudaMemcpyAsync(acts[0], r, sizeof(float2) * full, cudaMemcpyDeviceToDevice, s));
            net_forward(net, W, acts, s);
            LAPH_CUDA(cudaMemcpyAsync(Z[j], acts[net.sh.nlayers], sizeof(float2) * full, cudaMemcpyDeviceToDevice, s));
            // w_j = K z_j on both parities
            hop_f32(*net.op, 0, HOP_APPLY, (c32 *)Wv[j], (const c32 *)(Z[j] + half), (const c32 *)Z[j], nr, s);
            hop_f32(*net.op, 1, HOP_APPLY, (c32 *)(Wv[j] + half), (const c32 *)Z[j], (const c32 *)(Z[j] + half), nr, s);
            // classical Gram-Schmidt, twice: all j projections of a pass in one round trip
            for (int pass = 0; pass < 2 && j > 0; ++pass) {
                for (int i = 0; i < j; i += 3) {
                    const int m = std::min(3, j - i);
                    mrhs_dots<float>(ctx, pl, rows, m, (const c32 *)Wv[i], (const c32 *)Wv[j],
                                     m > 1 ? (const c32 *)Wv[i + 1] : nullptr, m > 1 ? (const c32 *)Wv[j] : nullptr,
                                     m > 2 ? (const c32 *)Wv[i + 2] : nullptr, m > 2 ? (const c32 *)Wv[j] : nullptr,
                                     red + (long)i * nr, s);
                }
                hgs.resize((size_t)j * nr);
                LAPH_CUDA(cudaMemcpyAsync(hgs.data(), red, sizeof(c64) * j * nr, cudaMemcpyDeviceToHost, s));
                LAPH_CUDA(cudaStreamSynchronize(s));
                for (auto &v : hgs) v = c64{-v.re, -v.im};
                LAPH_CUDA(cudaMemcpyAsync(coef, hgs.data(), sizeof(c64) * j * nr, cudaMemcpyHostToDevice, s));
                for (int i = 0; i < j; ++i) {
                    caxpy_rhs_kernel<<<grid_for(full, 256), 256, 0, s>>>(full, nr, coef + (long)i * nr, Wv[i], Wv[j]);
                    LAPH_LAUNCH_CHECK();
                    caxpy_rhs_kernel<<<grid_for(full, 256), 256, 0, s>>>(full, nr, coef + (long)i * nr, Z[i], Z[j]);
                    LAPH_LAUNCH_CHECK();
                }
            }
            dot(Wv[j], Wv[j]);
            for (int k = 0; k < nr; ++k) hs[k] = hred[k].re > 0 ? 1.0 / std::sqrt(hred[k].re) : 0.0;
            LAPH_CUDA(cudaMemcpyAsync(sc, hs.data(), sizeof(double) * nr, cudaMemcpyHostToDevice, s));
            mrhs_copy_scaled<float, float>(rows, nr, sc, (const c32 *)Wv[j], (c32 *)Wv[j], s);
            mrhs_copy_scaled<float, float>(rows, nr, sc, (const c32 *)Z[j], (c32 *)Z[j], s);
            dot(Wv[j], r);
            for (int k = 0; k < nr; ++k) hc[k] = active[k] ? hred[k] : c64{0, 0};
            axpy(hc, Z[j], x);
            for (int k = 0; k < nr; ++k) hc[k] = c64{-hc[k].re, -hc[k].im};
            axpy(hc, Wv[j], r);
            dot(r, r);
            bool any = false;
            for (int k = 0; k < nr; ++k) {
                if (active[k] && hred[k].re <= tol * tol * rr0[k]) active[k] = 0;
                any |= active[k] != 0;
            }
            if (!any) return it + 1;
        }
    }
    return it;
}

void solve_block_learned(laph_ctx *ctx, const DiracOp &op, const float *weights, const c64 *rhs, c64 *sol, int first,
                         int nr, const laph_solver_params &prm, laph_solve_report *rep, cudaStream_t s) {
    const Geom &g = op.g;
    const long rows = g.Vh * 12;
    size_t hb = sizeof(c64) * rows * nr;
    auto V = [&](const char *n) { return (c64 *)ws_get(ctx, std::string("lc:") + n, hb); };
    c64 *be = V("be"), *bo = V("bo"), *xe = V("xe"), *xo = V("xo"), *re = V("re"), *ro = V("ro");
    const long half = rows * nr;
    float2 *b32 = (float2 *)ws_get(ctx, "lc:b32", sizeof(float2) * 2 * half);
    float2 *x32 = (float2 *)ws_get(ctx, "lc:x32", sizeof(float2) * 2 * half);
    double *scale = (double *)ws_get(ctx, "lc:scale", sizeof(double) * 2 * nr);
    c64 *red = (c64 *)ws_get(ctx, "lc:red", sizeof(c64) * 2 * nr);
    RedPlan pl = red_plan(ctx, rows, nr);
    std::vector<c64> h(2 * nr);
    std::vector<double> bn(nr), rel(nr, 1.0), hsc(2 * nr);
    std::vector<int> iters(nr, 0), outer(nr, 0), fell(nr, 0);
    fields_to_eo(g, rhs, first, nr, be, bo, s);
    mrhs_dots<double>(ctx, pl, rows, 2, be, be, bo, bo, nullptr, nullptr, red, s);
    LAPH_CUDA(cudaMemcpyAsync(h.data(), red, sizeof(c64) * 2 * nr, cudaMemcpyDeviceToHost, s));
    LAPH_CUDA(cudaStreamSynchronize(s));
    for (int k = 0; k < nr; ++k) bn[k] = std::sqrt(h[k].re + h[nr + k].re);
    LAPH_CUDA(cudaMemsetAsync(xe, 0, hb, s));
    LAPH_CUDA(cudaMemsetAsync(xo, 0, hb, s));
    LAPH_CUDA(cudaMemcpyAsync(re, be, hb, cudaMemcpyDeviceToDevice, s));
    LAPH_CUDA(cudaMemcpyAsync(ro, bo, hb, cudaMemcpyDeviceToDevice, s));
    // inside FGCR the network runs on the tensor cores (BF16 operands; the flexible method takes an
    // inexact preconditioner); LAPH_NN_FP32=1 keeps the FP32 CUDA-core layers
    static const bool nn_fp32 = [] {
        const char *e = std::getenv("LAPH_NN_FP32");
        return e != nullptr && e[0] == '1';
    }();
    Net net{NNShape(), &op, g.Vh, nr, nn_fp32 ? nullptr : ctx};
    const int restart = prm.gcr_restart > 0 ? prm.gcr_restart : 16;
    int total = 0;
    double prev_worst = 1e300;
    for (int cyc = 0; cyc < 100; ++cyc) {
        if (cyc > 0) {
            hop<double>(op, 0, HOP_RESID, re, xo, be, xe, nr, s);
            hop<double>(op, 1, HOP_RESID, ro, xe, bo, xo, nr, s);
        }
        mrhs_dots<double>(ctx, pl, rows, 2, re, re, ro, ro, nullptr, nullptr, red, s);
        LAPH_CUDA(cudaMemcpyAsync(h.data(), red, sizeof(c64) * 2 * nr, cudaMemcpyDeviceToHost, s));
        LAPH_CUDA(cudaStreamSynchronize(s));
        double worst = 0.0;
        bool all = true;
        for (int k = 0; k < nr; ++k) {
            double rn = std::sqrt(h[k].re + h[nr + k].re);
            // a right-hand side that is not finite is reported as not converged and left alone
            const bool bad = !std::isfinite(bn[k]);
            rel[k] = bad ? std::nan("") : (bn[k] > 0 ? rn / bn[k] : 0.0);
            if (!(rel[k] <= prm.tol) && !bad) {
                all = false;
                worst = std::max(worst, std::isfinite(rel[k]) ? rel[k] : 1e300);
            }
            hsc[k] = (rel[k] <= prm.tol || !(rn > 0)) ? 0.0 : 1.0 / rn;
            hsc[nr + k] = (rel[k] <= prm.tol || !(rn > 0)) ? 0.0 : rn;
        }
        if (all || total >= prm.maxiter) break;
        if (cyc > 0 && !(worst < 0.1 * prev_worst)) {
            // the learned cycle stalled: the plain mixed-precision solver takes over on the
            // residual equation K d = r, then x += d
            c64 *rabi = (c64 *)ws_get(ctx, "lc:rabi", sizeof(c64) * 12 * g.V * nr);
            c64 *dabi = (c64 *)ws_get(ctx, "lc:dabi", sizeof(c64) * 12 * g.V * nr);
            eo_to_fields(g, re, ro, 0, nr, rabi, s);
            laph_solver_params fb = prm;
            fb.mode = LAPH_SOLVE_MIXED_FP32;
            fb.tol = std::max(1e-15, 0.5 * prm.tol / std::max(worst, prm.tol));
            std::vector<laph_solve_report> frep(nr);
            solve_block(ctx, op, rabi, dabi, 0, nr, fb, frep.data(), s);
            c64 *de = V("de"), *dd = V("do");
            fields_to_eo(g, dabi, 0, nr, de, dd, s);
            std::vector<double> one(nr, 1.0);
            LAPH_CUDA(cudaMemcpyAsync(scale, one.data(), sizeof(double) * nr, cudaMemcpyHostToDevice, s));
            mrhs_axpy_scaled<double, double>(rows, nr, scale, de, xe, s);
            mrhs_axpy_scaled<double, double>(rows, nr, scale, dd, xo, s);
            for (int k = 0; k < nr; ++k) {
                fell[k] = 1;
                iters[k] += frep[k].iters;
            }
            prev_worst = 0.0;   // no further fallback decisions: next cycles only verify
            continue;
        }
        prev_worst = worst;
        LAPH_CUDA(cudaMemcpyAsync(scale, hsc.data(), sizeof(double) * 2 * nr, cudaMemcpyHostToDevice, s));
        mrhs_copy_scaled<double, float>(rows, nr, scale, re, (c32 *)b32, s);
        mrhs_copy_scaled<double, float>(rows, nr, scale, ro, (c32 *)(b32 + half), s);
        double want = std::max(prm.inner_tol, 0.2 * prm.tol / std::max(worst, prm.tol));
        int n = fgcr(ctx, net, (const float2 *)weights, b32, x32, want, std::max(1, prm.maxiter - total), restart, s);
        if (net.tc != nullptr) nn_tc_check(s);
        total += n;
        for (int k = 0; k < nr; ++k)
            if (hsc[k] > 0) {
                iters[k] += n;
                outer[k] += 1;
            }
        mrhs_axpy_scaled<float, double>(rows, nr, scale + nr, (const c32 *)x32, xe, s);
        mrhs_axpy_scaled<float, double>(rows, nr, scale + nr, (const c32 *)(x32 + half), xo, s);
    }
    eo_to_fields(g, xe, xo, first, nr, sol, s);
    if (rep)
        for (int k = 0; k < nr; ++k) {
            laph_solve_report &o = rep[first + k];
            o.iters = iters[k];
            o.outer = outer[k];
            o.true_resid = rel[k];
            o.status = rel[k] <= prm.tol ? LAPH_OK : LAPH_ERR_NOT_CONVERGED;
            o.fallback_used = fell[k];
        }
}

}  // namespace laph

using namespace laph;

extern "C" int laph_precond_init(uint64_t seed, double diag, float *weights) {
    return guard([&] {
        LAPH_REQUIRE(weights != nullptr, "weights is null");
        LAPH_REQUIRE(diag != 0.0, "diag must be nonzero");
        NNShape sh;
        // seeded start: channel 0 carries the identity (1/diag in the last layer), every other
        // weight is small; a splitmix64 stream gives reproducible host-side values
        uint64_t st = seed ? seed : 0x9E3779B97F4A7C15ull;
        auto next = [&]() {
            st += 0x9E3779B97F4A7C15ull;
            uint64_t z = st;
            z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
            z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
            z ^= z >> 31;
            return (double)(z >> 11) * (1.0 / 9007199254740992.0) - 0.5;
        };
        long o = 0;
        for (int l = 0; l < sh.nlayers; ++l) {
            int cin = sh.cin(l), cout = sh.cout(l);
            double amp = 0.02 / std::sqrt(9.0 * cin * 4.0);
            for (int d = 0; d < 9; ++d)
                for (int c = 0; c < cout; ++c)
                    for (int cp = 0; cp < cin; ++cp)
                        for (int e = 0; e < 16; ++e, ++o) {
                            double re = amp * next(), im = amp * next();
                            if (d == 0 && c == 0 && cp == 0 && e / 4 == e % 4)
                                re += (l == sh.nlayers - 1) ? 1.0 / diag : 1.0;
                            weights[2 * o] = (float)re;
                            weights[2 * o + 1] = (float)im;
                        }
        }
    });
}

extern "C" int laph_precond_size(void) { return (int)(2 * NNShape().total()); }

// Trains the preconditioner on pairs (rho_i, phi_i), K phi_i = rho_i, on one gauge field.
// weights and adam ([2][nweights] floats: first and second moments) are updated in place.
extern "C" int laph_precond_train(laph_ctx *ctx, const laph_lattice *lat, const void *links,
                                  const laph_dirac_params *dirac, const void *rho, const void *phi, int npairs,
                                  int epochs, int batch, double lr, int step0, float *weights, float *adam,
                                  double *loss_out, void *stream) {
    return guard([&] {
        ctx_activate(ctx);
        Geom g = make_geom(lat);
        LAPH_REQUIRE(npairs >= 1 && batch >= 1 && epochs >= 0, "bad sizes");
        LAPH_REQUIRE(weights && adam, "weights / adam state are null");
        cudaStream_t s = as_stream(stream);
        batch = std::min(batch, npairs);
        NNShape sh;
        const long nw = sh.total();   // complex weights
        size_t fb = sizeof(c64) * 12 * g.V * (size_t)npairs;
        const c64 *L = (const c64 *)stage_in(ctx, links, sizeof(c64) * 36 * g.V, "links", s);
        const c64 *R = (const c64 *)stage_in(ctx, rho, fb, "nn_rho", s);
        const c64 *P = (const c64 *)stage_in(ctx, phi, fb, "nn_phi", s);
        DiracOp op = prepare_dirac(ctx, g, L, dirac->m0, dirac->csw, lat->xi, s);
        float2 *W = (float2 *)ws_get(ctx, "nn:W", sizeof(float2) * nw);
        float2 *M = (float2 *)ws_get(ctx, "nn:m", sizeof(float2) * nw);
        float2 *Vv = (float2 *)ws_get(ctx, "nn:v", sizeof(float2) * nw);
        c64 *grad = (c64 *)ws_get(ctx, "nn:grad", sizeof(c64) * nw);
        StagedOut wout = stage_out(ctx, weights, sizeof(float2) * nw, "nn_w_out");
        StagedOut aout = stage_out(ctx, adam, sizeof(float2) * 2 * nw, "nn_adam_out");
        const void *win = stage_in(ctx, weights, sizeof(float2) * nw, "nn_w_in", s);
        const void *ain = stage_in(ctx, adam, sizeof(float2) * 2 * nw, "nn_adam_in", s);
        LAPH_CUDA(cudaMemcpyAsync(W, win, sizeof(float2) * nw, cudaMemcpyDeviceToDevice, s));
        LAPH_CUDA(cudaMemcpyAsync(M, ain, sizeof(float2) * nw, cudaMemcpyDeviceToDevice, s));
        LAPH_CUDA(cudaMemcpyAsync(Vv, (const float2 *)ain + nw, sizeof(float2) * nw, cudaMemcpyDeviceToDevice, s));
        Net net{sh, &op, g.Vh, batch};
        const long chan = 2 * g.Vh * 12 * (long)batch;
        std::vector<float2 *> acts(sh.nlayers + 1);
        for (int l = 0; l <= sh.nlayers; ++l)
            acts[l] = (float2 *)ws_get(ctx, "nn:act" + std::to_string(l), sizeof(float2) * chan * NN_MAXC);
        float2 *phib = (float2 *)ws_get(ctx, "nn:phib", sizeof(float2) * chan);
        float2 *ga = (float2 *)ws_get(ctx, "nn:ga", sizeof(float2) * chan * NN_MAXC);
        float2 *gb = (float2 *)ws_get(ctx, "nn:gb", sizeof(float2) * chan * NN_MAXC);
        c64 *te = (c64 *)ws_get(ctx, "nn:te", sizeof(c64) * g.Vh * 12 * batch);
        c64 *to = (c64 *)ws_get(ctx, "nn:to", sizeof(c64) * g.Vh * 12 * batch);
        double *ones = (double *)ws_get(ctx, "nn:ones", sizeof(double) * batch);
        double *scale = (double *)ws_get(ctx, "nn:scale", sizeof(double) * batch);
        c64 *red = (c64 *)ws_get(ctx, "nn:red", sizeof(c64) * 2 * batch);
        fill_kernel<<<1, 256, 0, s>>>(batch, 1.0, ones);
        LAPH_LAUNCH_CHECK();
        RedPlan pl = red_plan(ctx, 2 * g.Vh * 12, batch);
        std::vector<c64> hred(2 * batch);
        std::vector<double> hscale(batch);
        double total_loss = 0.0;
        int nbatches = 0, step = step0;
        const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
        for (int ep = 0; ep < epochs; ++ep) {
            for (int first = 0; first + batch <= npairs; first += batch) {
                abi_to_net(g, R, first, batch, acts[0], te, to, ones, s);
                abi_to_net(g, P, first, batch, phib, te, to, ones, s);
                net_forward(net, W, acts, s);
                // per-pair ||phi||^2 and ||y - phi||^2 for the loss; e = (y - phi) / (B ||phi||^2)
                mrhs_dots<float>(ctx, pl, 2 * g.Vh * 12, 1, (c32 *)phib, (c32 *)phib, nullptr, nullptr, nullptr,
                                 nullptr, red, s);
                LAPH_CUDA(cudaMemcpyAsync(hred.data(), red, sizeof(c64) * batch, cudaMemcpyDeviceToHost, s));
                LAPH_CUDA(cudaStreamSynchronize(s));
                for (int k = 0; k < batch; ++k) hscale[k] = 1.0 / (batch * std::max(hred[k].re, 1e-300));
                LAPH_CUDA(cudaMemcpyAsync(scale, hscale.data(), sizeof(double) * batch, cudaMemcpyHostToDevice, s));
                long nf = chan;
                nn_err_kernel<<<grid_for(nf, 256), 256, 0, s>>>(nf, batch, acts[sh.nlayers], phib, scale, ga);
                LAPH_LAUNCH_CHECK();
                mrhs_dots<float>(ctx, pl, 2 * g.Vh * 12, 1, (c32 *)ga, (c32 *)ga, nullptr, nullptr, nullptr, nullptr,
                                 red, s);
                LAPH_CUDA(cudaMemcpyAsync(hred.data(), red, sizeof(c64) * batch, cudaMemcpyDeviceToHost, s));
                LAPH_CUDA(cudaStreamSynchronize(s));
                double bl = 0.0;
                // ||e_k||^2 = s_k^2 ||y_k - phi_k||^2 with s_k = 1/(B ||phi_k||^2), so the batch loss
                // sum_k ||y_k - phi_k||^2 / (B ||phi_k||^2) is sum_k ||e_k||^2 / s_k
                for (int k = 0; k < batch; ++k) bl += hred[k].re / hscale[k];
                total_loss += bl;
                ++nbatches;
                LAPH_CUDA(cudaMemsetAsync(grad, 0, sizeof(c64) * nw, s));
                net_backward(ctx, net, W, acts, ga, gb, grad, s);
                ++step;
                float bc1 = 1.f - powf(b1, (float)step), bc2 = 1.f - powf(b2, (float)step);
                adam_kernel<<<grid_for(nw, 256), 256, 0, s>>>(nw, W, grad, M, Vv, (float)lr, b1, b2, eps, bc1, bc2);
                LAPH_LAUNCH_CHECK();
            }
        }
        LAPH_CUDA(cudaMemcpyAsync(wout.dev, W, sizeof(float2) * nw, cudaMemcpyDeviceToDevice, s));
        LAPH_CUDA(cudaMemcpyAsync(aout.dev, M, sizeof(float2) * nw, cudaMemcpyDeviceToDevice, s));
        LAPH_CUDA(cudaMemcpyAsync((float2 *)aout.dev + nw, Vv, sizeof(float2) * nw, cudaMemcpyDeviceToDevice, s));
        wout.commit(s);
        aout.commit(s);
        LAPH_CUDA(cudaStreamSynchronize(s));
        if (loss_out) *loss_out = nbatches ? total_loss / nbatches : 0.0;
    });
}

// Loss and dL/d conj(W) (c128, layout of the weights) over all npairs in one batch.
extern "C" int laph_precond_grad(laph_ctx *ctx, const laph_lattice *lat, const void *links,
                                 const laph_dirac_params *dirac, const float *weights, const void *rho,
                                 const void *phi, int npairs, double *loss_out, void *grad_out, void *stream) {
    return guard([&] {
        ctx_activate(ctx);
        Geom g = make_geom(lat);
        LAPH_REQUIRE(npairs >= 1 && npairs <= 256, "npairs must be 1..256");
        cudaStream_t s = as_stream(stream);
        NNShape sh;
        const long nw = sh.total();
        const int B = npairs;
        size_t fb = sizeof(c64) * 12 * g.V * (size_t)B;
        const c64 *L = (const c64 *)stage_in(ctx, links, sizeof(c64) * 36 * g.V, "links", s);
        const c64 *R = (const c64 *)stage_in(ctx, rho, fb, "nn_rho", s);
        const c64 *P = (const c64 *)stage_in(ctx, phi, fb, "nn_phi", s);
        const float2 *W = (const float2 *)stage_in(ctx, weights, sizeof(float2) * nw, "nn_grad_w", s);
        StagedOut go = stage_out(ctx, grad_out, sizeof(c64) * nw, "nn_grad_out");
        DiracOp op = prepare_dirac(ctx, g, L, dirac->m0, dirac->csw, lat->xi, s);
        Net net{sh, &op, g.Vh, B};
        const long chan = 2 * g.Vh * 12 * (long)B;
        std::vector<float2 *> acts(sh.nlayers + 1);
        for (int l = 0; l <= sh.nlayers; ++l)
            acts[l] = (float2 *)ws_get(ctx, "nn:act" + std::to_string(l), sizeof(float2) * chan * NN_MAXC);
        float2 *phib = (float2 *)ws_get(ctx, "nn:phib", sizeof(float2) * chan);
        float2 *ga = (float2 *)ws_get(ctx, "nn:ga", sizeof(float2) * chan * NN_MAXC);
        float2 *gb = (float2 *)ws_get(ctx, "nn:gb", sizeof(float2) * chan * NN_MAXC);
        c64 *te = (c64 *)ws_get(ctx, "nn:te", sizeof(c64) * g.Vh * 12 * B);
        c64 *to = (c64 *)ws_get(ctx, "nn:to", sizeof(c64) * g.Vh * 12 * B);
        double *ones = (double *)ws_get(ctx, "nn:ones", sizeof(double) * B);
        double *scale = (double *)ws_get(ctx, "nn:scale", sizeof(double) * B);
        c64 *red = (c64 *)ws_get(ctx, "nn:red", sizeof(c64) * 2 * B);
        fill_kernel<<<1, 256, 0, s>>>(B, 1.0, ones);
        LAPH_LAUNCH_CHECK();
        RedPlan pl = red_plan(ctx, 2 * g.Vh * 12, B);
        std::vector<c64> hred(B);
        std::vector<double> hs(B);
        abi_to_net(g, R, 0, B, acts[0], te, to, ones, s);
        abi_to_net(g, P, 0, B, phib, te, to, ones, s);
        net_forward(net, W, acts, s);
        mrhs_dots<float>(ctx, pl, 2 * g.Vh * 12, 1, (c32 *)phib, (c32 *)phib, nullptr, nullptr, nullptr, nullptr, red, s);
        LAPH_CUDA(cudaMemcpyAsync(hred.data(), red, sizeof(c64) * B, cudaMemcpyDeviceToHost, s));
        LAPH_CUDA(cudaStreamSynchronize(s));
        for (int k = 0; k < B; ++k) hs[k] = 1.0 / (B * std::max(hred[k].re, 1e-300));
        LAPH_CUDA(cudaMemcpyAsync(scale, hs.data(), sizeof(double) * B, cudaMemcpyHostToDevice, s));
        nn_err_kernel<<<grid_for(chan, 256), 256, 0, s>>>(chan, B, acts[sh.nlayers], phib, scale, ga);
        LAPH_LAUNCH_CHECK();
        mrhs_dots<float>(ctx, pl, 2 * g.Vh * 12, 1, (c32 *)ga, (c32 *)ga, nullptr, nullptr, nullptr, nullptr, red, s);
        LAPH_CUDA(cudaMemcpyAsync(hred.data(), red, sizeof(c64) * B, cudaMemcpyDeviceToHost, s));
        LAPH_CUDA(cudaMemsetAsync(go.dev, 0, sizeof(c64) * nw, s));
        net_backward(ctx, net, (const float2 *)W, acts, ga, gb, (c64 *)go.dev, s);
        LAPH_CUDA(cudaStreamSynchronize(s));
        double l = 0.0;
        for (int k = 0; k < B; ++k) l += hred[k].re / hs[k];
        if (loss_out) *loss_out = l;
        go.commit(s);
    });
}

// Applies the network: out = N(in) for nrhs full fields (ABI layout, c128 in and out); tc: the
// layers on the tensor cores (nrhs a multiple of 32).
static void precond_apply(laph_ctx *ctx, const laph_lattice *lat, const void *links, const laph_dirac_params *dirac,
                          const float *weights, const void *in, void *out, int nrhs, void *stream, bool tc) {
    {
        ctx_activate(ctx);
        Geom g = make_geom(lat);
        LAPH_REQUIRE(nrhs >= 1 && nrhs <= 256, "nrhs must be 1..256");
        cudaStream_t s = as_stream(stream);
        NNShape sh;
        const long nw = sh.total();
        size_t fb = sizeof(c64) * 12 * g.V * (size_t)nrhs;
        const c64 *L = (const c64 *)stage_in(ctx, links, sizeof(c64) * 36 * g.V, "links", s);
        const c64 *X = (const c64 *)stage_in(ctx, in, fb, "nn_apply_in", s);
        const float2 *W = (const float2 *)stage_in(ctx, weights, sizeof(float2) * nw, "nn_apply_w", s);
        StagedOut o = stage_out(ctx, out, fb, "nn_apply_out");
        DiracOp op = prepare_dirac(ctx, g, L, dirac->m0, dirac->csw, lat->xi, s);
        if (tc) LAPH_REQUIRE(nn_tc_ok(nrhs, 1, 1), "tensor-core network: nrhs must be a multiple of 32");
        Net net{sh, &op, g.Vh, nrhs, tc ? ctx : nullptr};
        const long chan = 2 * g.Vh * 12 * (long)nrhs;
        std::vector<float2 *> acts(sh.nlayers + 1);
        for (int l = 0; l <= sh.nlayers; ++l)
            acts[l] = (float2 *)ws_get(ctx, "nn:act" + std::to_string(l), sizeof(float2) * chan * NN_MAXC);
        c64 *te = (c64 *)ws_get(ctx, "nn:te", sizeof(c64) * g.Vh * 12 * nrhs);
        c64 *to = (c64 *)ws_get(ctx, "nn:to", sizeof(c64) * g.Vh * 12 * nrhs);
        double *ones = (double *)ws_get(ctx, "nn:ones", sizeof(double) * nrhs);
        fill_kernel<<<1, 256, 0, s>>>(nrhs, 1.0, ones);
        LAPH_LAUNCH_CHECK();
        abi_to_net(g, X, 0, nrhs, acts[0], te, to, ones, s);
        net_forward(net, W, acts, s);
        long rows = g.Vh * 12;
        mrhs_copy_scaled<float, double>(rows, nrhs, ones, (const c32 *)acts[sh.nlayers], te, s);
        mrhs_copy_scaled<float, double>(rows, nrhs, ones, (const c32 *)(acts[sh.nlayers] + g.Vh * 12 * (long)nrhs), to, s);
        eo_to_fields(g, te, to, 0, nrhs, (c64 *)o.dev, s);
        o.commit(s);
        if (tc) nn_tc_check(s);
    }
}

extern "C" int laph_precond_apply(laph_ctx *ctx, const laph_lattice *lat, const void *links,
                                  const laph_dirac_params *dirac, const float *weights, const void *in, void *out,
                                  int nrhs, void *stream) {
    return guard([&] { precond_apply(ctx, lat, links, dirac, weights, in, out, nrhs, stream, false); });
}

extern "C" int laph_precond_apply_tc(laph_ctx *ctx, const laph_lattice *lat, const void *links,
                                     const laph_dirac_params *dirac, const float *weights, const void *in, void *out,
                                     int nrhs, void *stream) {
    return guard([&] { precond_apply(ctx, lat, links, dirac, weights, in, out, nrhs, stream, true); });
}
