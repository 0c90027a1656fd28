// One layer of the learned preconditioner's network on the tensor cores (tcgen05, BF16 operands,
// FP32 accumulation), for the network applications inside the flexible GCR solve, which tolerates
// an inexact preconditioner.
//
// The layer  out_c(x) = sum_{d, c'} W[d][c][c'] (T_d in_{c'})(x)  (W a 4 x 4 complex spin matrix,
// identity on colour; T_0 = 1, T_d a signed link transport) is a GEMM once the transported inputs
// are gathered: for a unit of one site and 32 right-hand sides the rows m = colour * 32 + rhs
// (96 of the 128 MMA rows used), the columns k = (d, c', s_in) and n = (c, s_out), written over
// the reals (k2 = 2 k + part, n2 = 2 n + part):
//   A[m][k2] = (T_d in_{c'})(x)[s_in][colour] (re, im),
//   B[n2][k2]: (re, re) -> Re W, (im, re) -> -Im W, (re, im) -> Im W, (im, im) -> Re W,
// so D = A B^T holds (Re out, Im out).  The CUDA cores do the gathers and the SU(3) transports
// (a sixth of the layer's multiply-adds) and write A in BF16 into shared memory in the no-swizzle
// K-major core-matrix layout (8 rows x 16 B per core matrix, K-adjacent cores 128 B apart, 8-row
// groups KP * 16 B apart); one thread issues the MMAs (M = 128, N = 16 or 32, K = 16) into a
// TMEM accumulator and commits to an mbarrier; the warps read the accumulator back with
// tcgen05.ld and store the FP32 outputs.  Every wait is bounded (about a second); a wait that
// gives up sets a flag the host turns into LAPH_ERR_TIMEOUT, and the CTA stops, waits (bounded)
// for its issued MMAs and frees its TMEM.
#include <cstdint>

#include "blas.cuh"
#include "dirac.cuh"

namespace laph {

namespace {

constexpr int NT_THREADS = 256;
constexpr int NT_M = 128;
constexpr long long NT_WAIT = 1LL << 31;   // ~1 s at the maximum SM clock

__device__ int g_nn_tc_flag;

__host__ __device__ constexpr int nt_kp(int cin) { return (72 * cin + 15) / 16 * 16; }
__host__ __device__ constexpr int nt_np(int cout) { return 8 * cout < 16 ? 16 : 8 * cout; }

// byte offset of (row, k2) in a K-major core-matrix tile of kp columns
__device__ __forceinline__ uint32_t nt_off(int kp, int row, int k2) {
    return (uint32_t)((((row >> 3) * (kp >> 3) + (k2 >> 3)) * 128) + (row & 7) * 16 + (k2 & 7) * 2);
}

__device__ __forceinline__ uint64_t nt_desc(uint32_t saddr, int kp) {
    uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFF);
    d |= (uint64_t)(128 >> 4) << 16;            // K-adjacent core matrices 128 B apart
    d |= (uint64_t)((kp * 16) >> 4) << 32;      // 8-row groups kp * 16 B apart
    d |= (uint64_t)1 << 46;
    return d;
}

__device__ __forceinline__ bool nt_wait(uint32_t bar, uint32_t parity) {
    const long long t0 = clock64();
    for (;;) {
        uint32_t ok;
        asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
                     : "=r"(ok)
                     : "r"(bar), "r"(parity)
                     : "memory");
        if (ok) return true;
        if (clock64() - t0 > NT_WAIT) return false;
    }
}

__device__ __forceinline__ uint32_t bf16_pair(float lo, float hi) {
    const uint32_t a = __bfloat16_as_ushort(__float2bfloat16_rn(lo));
    const uint32_t b = __bfloat16_as_ushort(__float2bfloat16_rn(hi));
    return a | (b << 16);
}

// B operand of one layer in the core-matrix layout ([np][kp] BF16, zero padding), from the
// weights [9][cout][cin][4][4] complex.
__global__ void nn_tc_prep_kernel(int cin, int cout, const float2 *__restrict__ W, uint16_t *__restrict__ B) {
    const int kp = nt_kp(cin), np = nt_np(cout);
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= kp * np) return;
    const int n2 = i / kp, k2 = i % kp;
    float v = 0.f;
    const int n = n2 >> 1, pn = n2 & 1, k = k2 >> 1, pk = k2 & 1;
    if (n < 4 * cout && k < 36 * cin) {
        const int c = n >> 2, so = n & 3;
        const int d = k / (4 * cin), cp = (k >> 2) % cin, si = k & 3;
        const float2 w = W[(((d * cout + c) * cin + cp) * 4 + so) * 4 + si];
        v = pk == pn ? w.x : (pk == 1 ? -w.y : w.y);
    }
    const uint32_t off = nt_off(kp, n2, k2);
    B[off >> 1] = __bfloat16_as_ushort(__float2bfloat16_rn(v));
}

// t = s U psi or s U^dag psi for one colour vector per spin (12 complex), links (re, re, im, im)
__device__ __forceinline__ void nt_transport(const float4 *__restrict__ u, bool dag, float s, const float2 psi[12],
                                             float2 t[12]) {
#pragma unroll
    for (int sp = 0; sp < 4; ++sp)
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            float re = 0.f, im = 0.f;
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                const float4 e = __ldg(u + (dag ? b * 3 + a : a * 3 + b));
                const float ur = e.x, ui = dag ? -e.z : e.z;
                const float2 h = psi[sp * 3 + b];
                re = fmaf(ur, h.x, fmaf(-ui, h.y, re));
                im = fmaf(ur, h.y, fmaf(ui, h.x, im));
            }
            t[sp * 3 + a] = make_float2(s * re, s * im);
        }
}

__global__ void __launch_bounds__(NT_THREADS, 2)
    nn_layer_tc_kernel(const int *__restrict__ nbr, const float4 *__restrict__ L, long Vh, int nr, int cin, int cout,
                       const uint16_t *__restrict__ Bg, const float2 *__restrict__ in, float2 *__restrict__ out) {
    extern __shared__ __align__(1024) unsigned char nsm[];
    const int kp = nt_kp(cin), np = nt_np(cout);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    unsigned char *base = (unsigned char *)(((uintptr_t)nsm + 1023) & ~(uintptr_t)1023);
    unsigned char *As = base, *Bs = base + NT_M * kp * 2;
    uint64_t *bar = (uint64_t *)(Bs + np * kp * 2);
    uint32_t *tslot = (uint32_t *)(bar + 1);
    int *s_nb = (int *)(tslot + 1);   // the 8 neighbours of the current unit's site
    const uint32_t a_s = (uint32_t)__cvta_generic_to_shared(As), b_s = (uint32_t)__cvta_generic_to_shared(Bs);
    const uint32_t bar_s = (uint32_t)__cvta_generic_to_shared(bar);

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         (uint32_t)__cvta_generic_to_shared(tslot)),
                     "r"(32));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar_s));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    // weights once; A's padding columns (k2 >= 72 cin) stay zero for the whole kernel
    for (int i = tid; i < np * kp / 8; i += NT_THREADS)
        reinterpret_cast<uint4 *>(Bs)[i] = reinterpret_cast<const uint4 *>(Bg)[i];
    for (int i = tid; i < NT_M * kp / 8; i += NT_THREADS) reinterpret_cast<uint4 *>(As)[i] = make_uint4(0, 0, 0, 0);
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = *tslot;
    const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(np >> 3) << 17) | ((uint32_t)(NT_M >> 4) << 24);

    const long chan = 2 * Vh * 12 * (long)nr, half = Vh * 12 * (long)nr, lplane = Vh * 9;
    const int nh = nr >> 5;
    const long nunits = 2 * Vh * nh;
    // unit u -> (site, rhs block), sites in checkerboard order (the stencil's z-blocked order cut
    // the DRAM reads by 18 % but measured 5 % slower: the layer waits on latency, not bandwidth)
    auto site_of = [&](long uu) -> long { return uu / nh; };
    // neighbour table of a unit's site in shared memory, loaded one unit ahead (during the MMAs of
    // the unit before), so that no gather waits on it
    if (tid < 8 && (long)blockIdx.x < nunits) s_nb[tid] = __ldg(nbr + site_of(blockIdx.x) * 8 + tid);
    __syncthreads();
    bool bad = false;
    uint32_t phase = 0;
    bool pending = false;
    for (long u = blockIdx.x; u < nunits && !bad; u += gridDim.x) {
        const long site = site_of(u);
        const int h = (int)(u % nh);
        const int p = (int)(site / Vh);
        const long cb = site - (long)p * Vh;
        // A: transported inputs, one (d, c', rhs) item per thread and step (loading two items ahead
        // measured 13 % slower: the extra registers cost more than the overlap gained)
        for (int it = tid; it < 9 * cin * 32; it += NT_THREADS) {
            const int r = it & 31, cp = (it >> 5) % cin, d = it / (32 * cin);
            long src = (long)p * half + cb * 12 * nr;
            const float4 *lk = nullptr;
            bool dag = false;
            float sg = 1.f;
            if (d > 0) {
                const int mu = (d - 1) & 3;
                const bool fw = d <= 4;
                int j = s_nb[fw ? mu : 4 + mu];
                sg = j < 0 ? -1.f : 1.f;
                j = j < 0 ? ~j : j;
                src = (long)(1 - p) * half + (long)j * 12 * nr;
                lk = fw ? L + ((long)p * 4 + mu) * lplane + cb * 9 : L + ((long)(1 - p) * 4 + mu) * lplane + (long)j * 9;
                dag = !fw;
            }
            const float2 *sp = in + cp * chan + src + 32 * h + r;
            float2 psi[12], t[12];
#pragma unroll
            for (int k = 0; k < 12; ++k) psi[k] = __ldg(sp + (long)k * nr);
            if (lk == nullptr) {
#pragma unroll
                for (int k = 0; k < 12; ++k) t[k] = psi[k];
            } else {
                nt_transport(lk, dag, sg, psi, t);
            }
            const int k2 = (d * cin + cp) * 8;
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                uint4 v;
                v.x = bf16_pair(t[0 * 3 + a].x, t[0 * 3 + a].y);
                v.y = bf16_pair(t[1 * 3 + a].x, t[1 * 3 + a].y);
                v.z = bf16_pair(t[2 * 3 + a].x, t[2 * 3 + a].y);
                v.w = bf16_pair(t[3 * 3 + a].x, t[3 * 3 + a].y);
                *reinterpret_cast<uint4 *>(As + nt_off(kp, a * 32 + r, k2)) = v;
            }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;");
        if (tid == 0) {
#pragma unroll 1
            for (int ks = 0; ks < kp / 16; ++ks) {
                const uint64_t ad = nt_desc(a_s + (uint32_t)(ks * 256), kp);
                const uint64_t bd = nt_desc(b_s + (uint32_t)(ks * 256), kp);
                const uint32_t acc = ks > 0 ? 1u : 0u;
                asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                             "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(tmem),
                             "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar_s));
        }
        pending = true;
        if (tid < 8 && u + gridDim.x < nunits) s_nb[tid] = __ldg(nbr + site_of(u + gridDim.x) * 8 + tid);
        const bool ok = nt_wait(bar_s, phase);
        if (__syncthreads_or(!ok)) {
            bad = true;
            break;
        }
        pending = false;
        phase ^= 1u;
        asm volatile("tcgen05.fence::after_thread_sync;");
        // epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31 (colour w % 4, rhs = lane), columns
        // 16 (w / 4) .. + 15; colour 3 is padding
        const int q = warp & 3, cg = (warp >> 2) * 16;
        if (cg < np) {
            uint32_t rr[16];
            const uint32_t ta = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)cg;
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                : "=r"(rr[0]), "=r"(rr[1]), "=r"(rr[2]), "=r"(rr[3]), "=r"(rr[4]), "=r"(rr[5]), "=r"(rr[6]),
                  "=r"(rr[7]), "=r"(rr[8]), "=r"(rr[9]), "=r"(rr[10]), "=r"(rr[11]), "=r"(rr[12]), "=r"(rr[13]),
                  "=r"(rr[14]), "=r"(rr[15])
                : "r"(ta));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            if (q < 3) {
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const int n = (cg >> 1) + j;   // complex column (c, s_out)
                    if (n < 4 * cout) {
                        const int c = n >> 2, so = n & 3;
                        out[c * chan + (long)p * half + (cb * 12 + so * 3 + q) * nr + 32 * h + lane] =
                            make_float2(__uint_as_float(rr[2 * j]), __uint_as_float(rr[2 * j + 1]));
                    }
                }
            }
        }
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncthreads();   // A and the accumulator are free for the next unit
    }
    if (bad) {
        if (tid == 0) atomicExch(&g_nn_tc_flag, 1);
        if (pending) (void)nt_wait(bar_s, phase);
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(32));
}

}  // namespace

bool nn_tc_ok(int nr, int cin, int cout) { return nr % 32 == 0 && cin >= 1 && cin <= 4 && cout >= 1 && cout <= 4; }

// out = layer(in) on the tensor cores; fields as the network's ([c][2][Vh][12][nr] FP32 complex).
void nn_layer_tensor_core(laph_ctx *ctx, const DiracOp &op, long Vh, int nr, int cin, int cout, const float2 *W,
                          const float2 *in, float2 *out, cudaStream_t s) {
    const int kp = nt_kp(cin), np = nt_np(cout);
    uint16_t *B = (uint16_t *)ws_get(ctx, "nn_tc:B", sizeof(uint16_t) * kp * np);
    nn_tc_prep_kernel<<<grid_for((long)kp * np, 256), 256, 0, s>>>(cin, cout, W, B);
    LAPH_LAUNCH_CHECK();
    const size_t smem = (size_t)(NT_M + np) * kp * 2 + 64 + 1024;
    static int attr_dev = -1;
    int dev = 0;
    LAPH_CUDA(cudaGetDevice(&dev));
    if (attr_dev != dev) {
        LAPH_CUDA(cudaFuncSetAttribute(nn_layer_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)((size_t)(NT_M + 32) * nt_kp(4) * 2 + 64 + 1024)));
        attr_dev = dev;
    }
    const long nunits = 2 * Vh * (nr / 32);
    const long cap = 2L * (ctx->sm_count ? ctx->sm_count : 152);
    const unsigned grid = (unsigned)(nunits < cap ? nunits : cap);
    prof_begin("nn_layer_tc", s);
    nn_layer_tc_kernel<<<grid, NT_THREADS, smem, s>>>(op.nbr, op.L32w, Vh, nr, cin, cout, B, in, out);
    LAPH_LAUNCH_CHECK();
    // flops the tensor cores execute (padding included); bytes: inputs gathered once, outputs once
    prof_end("nn_layer_tc", s, 8.0 * 12 * 2 * Vh * nr * (cin + cout),
             2.0 * NT_M * (double)kp * np * (double)nunits);
}

// Throws LAPH_ERR_TIMEOUT (and clears the flag) if a tensor-core layer CTA gave up waiting.
void nn_tc_check(cudaStream_t s) {
    int v = 0;
    LAPH_CUDA(cudaMemcpyFromSymbolAsync(&v, g_nn_tc_flag, sizeof(int), 0, cudaMemcpyDeviceToHost, s));
    LAPH_CUDA(cudaStreamSynchronize(s));
    if (v) {
        const int zero = 0;
        LAPH_CUDA(cudaMemcpyToSymbolAsync(g_nn_tc_flag, &zero, sizeof(int), 0, cudaMemcpyHostToDevice, s));
        LAPH_CUDA(cudaStreamSynchronize(s));
        throw Error(LAPH_ERR_TIMEOUT, "a tensor-core network-layer wait gave up (device wait cap)");
    }
}

}  // namespace laph
