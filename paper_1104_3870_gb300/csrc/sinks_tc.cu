// Sink coefficients on the tensor cores (Sec. IV: the quark-propagation coefficients
// V_s^dag x of every slice), FP64-accurate through exact integer slices.
//
//   coef[i][t][alpha][n] = sum_{x,c} conj(V[t][n][x][c]) X[i][t][x][alpha][c]
//
// Per slice t this is a complex GEMM C = V^H X with K = 3 V3.  Written over the reals
// (k2 = 2k + part): row (n, re) of A holds (Re V, Im V), row (n, im) holds (-Im V, Re V),
// column (i, alpha) of B holds (Re x, Im x), so C_re = A_(n,re) . B and C_im = A_(n,im) . B.
//
// Exact slices (the error-free splitting of Ozaki, Ogita, Oishi and Rump, 2012): every row of A
// is scaled by a power of two 2^-E_n with E_n the exponent of its largest entry, every column of B
// by 2^-E_c, so that the scaled entries lie in (-1, 1).  Each scaled entry is cut into eight
// signed 6-bit digits (|a| = sum_{j=1..8} d_j 2^-6j + O(2^-48), d_j in [0, 63], all with the sign
// of a); a digit is an integer that BF16 holds exactly.  A digit product is at most 63^2 < 2^12,
// and the sums of one diagonal j + l = D over 512 real k take at most 8 * 512 * 63^2 < 2^24, so
// the tensor cores' FP32 accumulation of them is exact.  After each chunk of 512 the nine
// diagonals D = 2..10 (43 digit pairs) are read from TMEM and added, weighted by 2^-6D, into FP64
// registers; the scale 2^(E_n + E_c) is applied at the end.  The pairs left out (j + l >= 11) add
// at most 6 * 63^2 2^-66 + ... < 4e-16 of 2^(E_n + E_c) per real k, a tenth of the 2^-48
// truncation of the entries, so a coefficient is within 2^-46 (max|a| sum|b| + max|b| sum|a|)
// of the exact sum over its real k, plus the FP64 rounding of the sums.
//
// Kernel: one CTA of four warps per (32 output columns, 128 real rows, slice).  Digits of a
// sub-chunk of 32 real k are written by all threads into shared memory in the no-swizzle
// K-major core-matrix layout (8 rows x 16 B per core matrix; K-adjacent cores 128 B apart,
// 8-row groups 512 B apart), double-buffered; thread 0 issues tcgen05.mma kind::f16 (BF16 in,
// FP32 accumulate, M = 128, N = 32, K = 16) into nine TMEM accumulators of 32 columns and
// commits to the buffer's mbarrier.  Every wait is bounded (about a second); a wait that gives
// up sets a flag the host turns into LAPH_ERR_TIMEOUT, and the CTA stops issuing, waits for its
// issued work (bounded) and frees its TMEM.
#include <cstdint>

#include "common.cuh"

namespace laph {

namespace {

constexpr int TC_M = 128;         // real rows per CTA (64 eigenvectors, re and im rows)
constexpr int TC_N = 32;          // columns per CTA (8 right-hand sides x 4 spins)
constexpr int TC_KS = 32;         // real k per shared-memory sub-chunk (16 complex)
constexpr int TC_DIGITS = 8;      // 6-bit digits per value
constexpr int TC_DIAG = 9;        // diagonals j + l = 2 .. 10
constexpr int TC_DRAIN = 16;      // sub-chunks per TMEM drain (512 real k)
constexpr int TC_A_BYTES = TC_DIGITS * TC_M * TC_KS * 2;   // 64 KB
constexpr int TC_B_BYTES = TC_DIGITS * TC_N * TC_KS * 2;   // 16 KB
constexpr int TC_BUF = TC_A_BYTES + TC_B_BYTES;
constexpr size_t TC_SMEM = 2 * (size_t)TC_BUF + 1024;       // two buffers + barriers, aligned
constexpr long long TC_WAIT = 1LL << 31;                    // ~1 s at the maximum SM clock
constexpr int TC_NONFINITE = 4096;                          // exponent marking a row / column with NaN or inf

__device__ int g_sinks_tc_flag;

// |a| 2^-E as a fraction with 48 bits, truncated (|a| < 2^E by the choice of E).
__device__ __forceinline__ uint64_t frac48(double a, int E) {
    const uint64_t bits = (uint64_t)__double_as_longlong(a) & 0x7FFFFFFFFFFFFFFFull;
    const int ex = (int)(bits >> 52);
    if (ex == 0) return 0;
    const uint64_t mant = (bits & 0xFFFFFFFFFFFFFull) | (1ull << 52);
    const int sh = 1027 + E - ex;   // |a| = mant 2^(ex - 1075); times 2^(48 - E)
    return (sh >= 64 || sh < 0) ? 0ull : (mant >> sh);
}
// BF16 bits of the integer v in [0, 63] with sign bit s
__device__ __forceinline__ uint32_t bf16_digit(uint32_t v, uint32_t s) {
    const float f = __uint_as_float(0x4B000000u | v) - 8388608.0f;   // exactly v
    return (__float_as_uint(f) >> 16) | (s << 15);
}
__device__ __forceinline__ uint32_t digit(uint64_t F, int j) { return (uint32_t)(F >> (48 - 6 * j)) & 63u; }

// byte offset of element (row, k2) of digit plane j in a K-major core-matrix tile with rows rows
__device__ __forceinline__ uint32_t core_off(int j, int rows, int row, int k2) {
    return (uint32_t)((((j * (rows / 8) + (row >> 3)) * (TC_KS / 8) + (k2 >> 3)) * 128) + (row & 7) * 16 + (k2 & 7) * 2);
}

__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
    uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFF);
    d |= (uint64_t)(128 >> 4) << 16;                    // K-adjacent core matrices 128 B apart
    d |= (uint64_t)((TC_KS / 8) * 128 >> 4) << 32;      // 8-row groups 512 B apart
    d |= (uint64_t)1 << 46;
    return d;
}

__device__ __forceinline__ bool mbar_wait_parity(uint32_t bar, uint32_t parity) {
    const long long t0 = clock64();
    for (;;) {
        uint32_t ok;
        asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
                     : "=r"(ok)
                     : "r"(bar), "r"(parity)
                     : "memory");
        if (ok) return true;
        if (clock64() - t0 > TC_WAIT) return false;
    }
}

__global__ void __launch_bounds__(128, 1)
    sinks_tc_kernel(const c64 *__restrict__ V, const c64 *__restrict__ X, const int *__restrict__ Erow,
                    const int *__restrict__ Ecol, int nv, int nrhs, long K, int nt, c64 *__restrict__ coef) {
    extern __shared__ __align__(1024) unsigned char tsm[];
    const int tid = threadIdx.x, warp = tid >> 5;
    const int n0 = blockIdx.x * TC_N, m0 = blockIdx.y * TC_M, t = blockIdx.z;
    unsigned char *base = (unsigned char *)(((uintptr_t)tsm + 1023) & ~(uintptr_t)1023);
    uint64_t *bars = (uint64_t *)(base + 2 * TC_BUF);
    uint32_t *tslot = (uint32_t *)(bars + 2);
    const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(base);
    const uint32_t bar0 = (uint32_t)__cvta_generic_to_shared(bars);

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         (uint32_t)__cvta_generic_to_shared(tslot)),
                     "r"(512));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar0));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar0 + 8));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = *tslot;

    const long K2 = 2 * K;
    const int nsub = (int)((K2 + TC_KS - 1) / TC_KS);
    // instruction descriptor: FP32 accumulate, BF16 A and B, both K-major, N = 32, M = 128
    const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TC_N >> 3) << 17) |
                           ((uint32_t)(TC_M >> 4) << 24);
    double acc[TC_N];
#pragma unroll
    for (int c = 0; c < TC_N; ++c) acc[c] = 0.0;
    bool started[TC_DIAG];
#pragma unroll
    for (int d = 0; d < TC_DIAG; ++d) started[d] = false;
    bool bad = false;
    int last = -1;   // last sub-chunk whose MMAs were committed

    for (int kk = 0; kk < nsub; ++kk) {
        const int b = kk & 1;
        if (kk >= 2) {   // the MMAs that read this buffer two sub-chunks ago are done
            const bool ok = mbar_wait_parity(bar0 + 8 * b, (uint32_t)(((kk >> 1) - 1) & 1));
            if (__syncthreads_or(!ok)) {
                bad = true;
                break;
            }
        }
        unsigned char *abuf = base + b * TC_BUF, *bbuf = abuf + TC_A_BYTES;
        const long kc0 = (long)kk * (TC_KS / 2);   // first complex k of the sub-chunk
        // A digits: 64 eigenvectors x 16 complex k, eight items per thread (a half warp per vector)
#pragma unroll 2
        for (int q = 0; q < 8; ++q) {
            const int it = tid + 128 * q, nl = it >> 4, kl = it & 15;
            const int n = (m0 >> 1) + nl;
            const long k = kc0 + kl;
            uint64_t Fr = 0, Fi = 0;
            uint32_t sr = 0, si = 0;
            if (n < nv && k < K) {
                const c64 v = V[((long)t * nv + n) * K + k];
                const int E = Erow[t * nv + n];
                Fr = frac48(v.re, E);
                Fi = frac48(v.im, E);
                sr = v.re < 0.0;
                si = v.im < 0.0;
            }
#pragma unroll
            for (int j = 1; j <= TC_DIGITS; ++j) {
                const uint32_t dr = digit(Fr, j), di = digit(Fi, j);
                const uint32_t re_row = bf16_digit(dr, sr) | (bf16_digit(di, si) << 16);        // (Re V, Im V)
                const uint32_t im_row = bf16_digit(di, si ^ 1u) | (bf16_digit(dr, sr) << 16);   // (-Im V, Re V)
                *(uint32_t *)(abuf + core_off(j - 1, TC_M, 2 * nl, 2 * kl)) = re_row;
                *(uint32_t *)(abuf + core_off(j - 1, TC_M, 2 * nl + 1, 2 * kl)) = im_row;
            }
        }
        // B digits: 32 columns (i, alpha) x 16 complex k (k = x * 3 + c), four items per thread
#pragma unroll 2
        for (int q = 0; q < 4; ++q) {
            const int it = tid + 128 * q, cl = it >> 4, kl = it & 15;
            const int cg = n0 + cl, i = cg >> 2, al = cg & 3;
            const long k = kc0 + kl;
            uint64_t Fr = 0, Fi = 0;
            uint32_t sr = 0, si = 0;
            if (i < nrhs && k < K) {
                const long x = k / 3, c = k - 3 * x;
                const c64 v = X[(((long)i * nt + t) * (K / 3) + x) * 12 + al * 3 + c];
                const int E = Ecol[((long)i * nt + t) * 4 + al];
                Fr = frac48(v.re, E);
                Fi = frac48(v.im, E);
                sr = v.re < 0.0;
                si = v.im < 0.0;
            }
#pragma unroll
            for (int j = 1; j <= TC_DIGITS; ++j)
                *(uint32_t *)(bbuf + core_off(j - 1, TC_N, cl, 2 * kl)) =
                    bf16_digit(digit(Fr, j), sr) | (bf16_digit(digit(Fi, j), si) << 16);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;");
        if (tid == 0) {
            const uint32_t a0 = sbase + b * TC_BUF, b0 = a0 + TC_A_BYTES;
#pragma unroll 1
            for (int d = 0; d < TC_DIAG; ++d)
#pragma unroll 1
                for (int j = 1; j <= TC_DIGITS; ++j) {
                    const int l = d + 2 - j;
                    if (l < 1 || l > TC_DIGITS) continue;
#pragma unroll
                    for (int ks = 0; ks < TC_KS / 16; ++ks) {
                        const uint64_t ad = smem_desc(a0 + (uint32_t)(((j - 1) * (TC_M / 8) * (TC_KS / 8) + 2 * ks) * 128));
                        const uint64_t bd = smem_desc(b0 + (uint32_t)(((l - 1) * (TC_N / 8) * (TC_KS / 8) + 2 * ks) * 128));
                        const uint32_t accum = started[d] ? 1u : 0u;
                        started[d] = true;
                        asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                                     "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(
                                         tmem + (uint32_t)(d * TC_N)),
                                     "l"(ad), "l"(bd), "r"(idesc), "r"(accum));
                    }
                }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                bar0 + 8 * b));
        }
        last = kk;
        if ((kk + 1) % TC_DRAIN == 0 || kk == nsub - 1) {
            // drain: wait for this sub-chunk's MMAs, add the eight diagonals into FP64
            const bool ok = mbar_wait_parity(bar0 + 8 * b, (uint32_t)((kk >> 1) & 1));
            if (__syncthreads_or(!ok)) {
                bad = true;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;");
#pragma unroll 1
            for (int d = 0; d < TC_DIAG; ++d) {
                const double w = ldexp(1.0, -6 * (d + 2));
#pragma unroll
                for (int h = 0; h < TC_N / 32; ++h) {
                    uint32_t r[32];
                    const uint32_t ta = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(d * TC_N + h * 32);
                    asm volatile(
                        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
                          "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]),
                          "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]),
                          "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                        : "r"(ta));
                    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                    for (int c = 0; c < 32; ++c) acc[h * 32 + c] = fma((double)__uint_as_float(r[c]), w, acc[h * 32 + c]);
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;");
#pragma unroll
            for (int d = 0; d < TC_DIAG; ++d) started[d] = false;
        }
    }
    if (bad) {
        if (tid == 0) atomicExch(&g_sinks_tc_flag, 1);
        if (last >= 0) (void)mbar_wait_parity(bar0 + 8 * (last & 1), (uint32_t)((last >> 1) & 1));
    } else {
        // row tid of the tile: eigenvector n, real (even row) or imaginary (odd row) part
        const int r = m0 + tid, n = r >> 1;
        if (n < nv) {
            const int En = Erow[t * nv + n];
#pragma unroll
            for (int c = 0; c < TC_N; ++c) {
                const int cg = n0 + c, i = cg >> 2, al = cg & 3;
                if (i < nrhs) {
                    const int Ec = Ecol[((long)i * nt + t) * 4 + al];
                    // a non-finite input row or column gives a non-finite coefficient, as in FP64
                    const double val = (En >= TC_NONFINITE || Ec >= TC_NONFINITE) ? __longlong_as_double(0x7FF8000000000000ll)
                                                                                : ldexp(acc[c], En + Ec);
                    double *dst = reinterpret_cast<double *>(coef + (((long)i * nt + t) * 4 + al) * nv + n);
                    dst[r & 1] = val;
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
}

// E such that every |entry| of the row / column is below 2^E (frexp exponent of the largest; 0 for
// an all-zero row).
__device__ __forceinline__ int exp_above(double m) {
    if (!isfinite(m)) return TC_NONFINITE;
    if (!(m > 0.0)) return 0;
    int e;
    (void)frexp(m, &e);
    return e;
}

// Erow[t][n] over V[t][n][0..K), one block per (n, t)
__global__ void row_exp_kernel(const c64 *__restrict__ V, long K, int nv, int *Erow) {
    __shared__ double sm[256];
    const int n = blockIdx.x, t = blockIdx.y;
    const c64 *v = V + ((long)t * nv + n) * K;
    double m = 0.0;
    for (long k = threadIdx.x; k < K; k += blockDim.x) {
        const double a = fmax(fabs(v[k].re), fabs(v[k].im));
        m = (isfinite(v[k].re) && isfinite(v[k].im)) ? fmax(m, a) : INFINITY;
    }
    sm[threadIdx.x] = m;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) sm[threadIdx.x] = fmax(sm[threadIdx.x], sm[threadIdx.x + s]);
        __syncthreads();
    }
    if (threadIdx.x == 0) Erow[t * nv + n] = exp_above(sm[0]);
}

// Ecol[i][t][alpha] over X[i][t][x][alpha][c], one block per (i, t)
__global__ void col_exp_kernel(const c64 *__restrict__ X, long V3, int nt, int *Ecol) {
    __shared__ double sm[4][256];
    const int i = blockIdx.x, t = blockIdx.y;
    const c64 *x = X + ((long)i * nt + t) * V3 * 12;
    double m[4] = {0.0, 0.0, 0.0, 0.0};
    for (long e = threadIdx.x; e < V3 * 12; e += blockDim.x) {
        const int al = (int)((e % 12) / 3);
        const double a = fmax(fabs(x[e].re), fabs(x[e].im));
        m[al] = (isfinite(x[e].re) && isfinite(x[e].im)) ? fmax(m[al], a) : INFINITY;
    }
    for (int a = 0; a < 4; ++a) sm[a][threadIdx.x] = m[a];
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s)
            for (int a = 0; a < 4; ++a) sm[a][threadIdx.x] = fmax(sm[a][threadIdx.x], sm[a][threadIdx.x + s]);
        __syncthreads();
    }
    if (threadIdx.x < 4) Ecol[((long)i * nt + t) * 4 + threadIdx.x] = exp_above(sm[threadIdx.x][0]);
}

}  // namespace

// coef[i][t][alpha][n] for nrhs solutions (device arrays; layouts as laph_sinks).
void sinks_tensor_core(laph_ctx *ctx, const Geom &g, const c64 *V, int nv, const c64 *X, int nrhs, c64 *coef,
                       cudaStream_t s) {
    static bool attr = false;
    if (!attr) {
        LAPH_CUDA(cudaFuncSetAttribute(sinks_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TC_SMEM));
        attr = true;
    }
    const long K = 3 * g.V3;
    int *Erow = (int *)ws_get(ctx, "sinks_tc:erow", sizeof(int) * g.nt * (size_t)nv);
    int *Ecol = (int *)ws_get(ctx, "sinks_tc:ecol", sizeof(int) * 4 * g.nt * (size_t)nrhs);
    prof_begin("sinks", s);
    row_exp_kernel<<<dim3(nv, g.nt), 256, 0, s>>>(V, K, nv, Erow);
    LAPH_LAUNCH_CHECK();
    col_exp_kernel<<<dim3(nrhs, g.nt), 256, 0, s>>>(X, g.V3, g.nt, Ecol);
    LAPH_LAUNCH_CHECK();
    const dim3 grid((unsigned)((4 * nrhs + TC_N - 1) / TC_N), (unsigned)((2 * nv + TC_M - 1) / TC_M), (unsigned)g.nt);
    sinks_tc_kernel<<<grid, 128, TC_SMEM, s>>>(V, X, Erow, Ecol, nv, nrhs, K, g.nt, coef);
    LAPH_LAUNCH_CHECK();
    // 43 digit-pair GEMMs of (2 nv) x (6 V3) x (4 nrhs) per slice on the tensor cores
    // algorithmic bytes: the solutions once per row tile, the eigenvectors once per column tile;
    // flops: the 43 digit-pair GEMMs the tensor cores execute, padding included
    const double nsub = (double)((2 * K + TC_KS - 1) / TC_KS) * TC_KS;
    prof_end("sinks", s,
             16.0 * (double)g.V * 12 * nrhs * grid.y + 16.0 * (double)g.nt * nv * K * grid.x +
                 16.0 * (double)nrhs * g.nt * 4 * nv,
             43.0 * 2.0 * (double)TC_M * grid.y * nsub * (double)TC_N * grid.x * g.nt);
}

// Throws LAPH_ERR_TIMEOUT (and clears the flag) if a tensor-core sink CTA gave up waiting.
void sinks_tc_check(cudaStream_t s) {
    int v = 0;
    LAPH_CUDA(cudaMemcpyFromSymbolAsync(&v, g_sinks_tc_flag, sizeof(int), 0, cudaMemcpyDeviceToHost, s));
    LAPH_CUDA(cudaStreamSynchronize(s));
    if (v) {
        const int zero = 0;
        LAPH_CUDA(cudaMemcpyToSymbolAsync(g_sinks_tc_flag, &zero, sizeof(int), 0, cudaMemcpyHostToDevice, s));
        LAPH_CUDA(cudaStreamSynchronize(s));
        throw Error(LAPH_ERR_TIMEOUT, "a tensor-core sink wait gave up (device wait cap)");
    }
}

}  // namespace laph
