// Lowest eigenpairs of -Delta on every time slice (Sec. II: V_s from the N_v
// lowest eigenvalues of -Delta per slice; Sec. IV: Krylov-spectral restarted
// Lanczos with Chebyshev acceleration).
//
//   -Delta psi(x) = 6 psi(x) - sum_k [ U_k(x) psi(x+k) + U_k(x-k)^dag psi(x-k) ]   (k spatial)
//   B = 1 + 2 (Delta + lambda_C)/(lambda_L - lambda_C) = a (-Delta) + b,
//       a = -2/(lambda_L - lambda_C), b = 1 + 2 lambda_C/(lambda_L - lambda_C)
//   A = T_n(B) by T_0 = 1, T_1 = B, T_k = 2 B T_{k-1} - T_{k-2}
// The lowest eigenvalues of -Delta become the largest of A.  Each Lanczos step
// applies A to one vector per slice, orthogonalises it against the whole basis
// (full reorthogonalisation) and repeats while the norm drops by more than
// 1/sqrt(2), at most four repeats.  After m steps the projected matrix is
// diagonalised (batched complex Jacobi, one block per slice), k Ritz vectors
// are kept (thick restart) and the residuals ||(-Delta) y - mu y|| of the
// wanted N_v are checked explicitly on -Delta itself.
//
// All slices advance together (the slice is the batch index); every array has
// a leading slice dimension.  FP64 throughout.
#include <algorithm>
#include <cmath>
#include <vector>

#include "common.cuh"
#include "philox.cuh"

namespace laph {

// Complex Gaussian fill from Philox4x32-10 words by the Box-Muller transform.
__global__ void normal_fill_kernel(long n, uint32_t seed, uint32_t stream, c64 *out) {
    long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint32_t c[4] = {(uint32_t)i, (uint32_t)(i >> 32), stream, 0u};
    philox4x32_10(c, seed, 0x5EEDu);
    double u1 = ((double)c[0] + 0.5) * (1.0 / 4294967296.0);
    double u2 = ((double)c[1] + 0.5) * (1.0 / 4294967296.0);
    double r = sqrt(-2.0 * log(u1));
    double sn, cs;
    sincospi(2.0 * u2, &sn, &cs);
    out[i] = c64{r * cs, r * sn};
}

// Column c of slice t of V ([t][keep][n]) is refilled with a seeded Gaussian vector where
// mask[t * keep + c] is set (Philox counter (element, t keep + c, 1), key (seed, 0x5EED)).
__global__ void randomize_cols_kernel(long n, int keep, const int *mask, uint32_t seed, c64 *V) {
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    const long col = (long)blockIdx.z * keep + blockIdx.y;
    if (i >= n || !mask[col]) return;
    uint32_t c[4] = {(uint32_t)i, (uint32_t)(i >> 32), (uint32_t)col, 1u};
    philox4x32_10(c, seed, 0x5EEDu);
    double u1 = ((double)c[0] + 0.5) * (1.0 / 4294967296.0);
    double u2 = ((double)c[1] + 0.5) * (1.0 / 4294967296.0);
    double r = sqrt(-2.0 * log(u1));
    double sn, cs;
    sincospi(2.0 * u2, &sn, &cs);
    V[col * n + i] = c64{r * cs, r * sn};
}

void philox_normal_fill(c64 *out, long n, uint32_t seed, uint32_t stream, cudaStream_t s) {
    normal_fill_kernel<<<grid_for(n, 256), 256, 0, s>>>(n, seed, stream, out);
    LAPH_LAUNCH_CHECK();
}

struct EigDims {
    int nt;
    long V3, n;   // n = 3 V3
    int m;        // Krylov dimension
};

// ------------------------------------------------------------------ Laplacian / Chebyshev
// out[t][v][x][c] = alpha * (a_t * (-Delta in) + b_t * in) - (use_prev ? prev : 0)
__global__ void cheb_kernel(Geom g, const c64 *__restrict__ U, int nvec, const c64 *__restrict__ in,
                            const c64 *__restrict__ prev, c64 *__restrict__ out, const double *__restrict__ ca,
                            const double *__restrict__ cb, double alpha, int use_prev, long in_tstride,
                            long out_tstride) {
    // vector v of slice t lives at base + t * tstride + v * 3 V3
    long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
    long per_t = (long)nvec * g.V3;
    if (idx >= per_t * g.nt) return;
    int t = (int)(idx / per_t);
    long r = idx % per_t;
    int v = (int)(r / g.V3);
    long x = r % g.V3;
    int c[4];
    site_coords(g, (long)t * g.V3 + x, c);
    const c64 *src = in + (long)t * in_tstride + (long)v * 3 * g.V3;
    c64 psi[3], acc[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        psi[i] = src[x * 3 + i];
        acc[i] = 6.0 * psi[i];
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        int cf[4] = {c[0], c[1], c[2], c[3]};
        cf[k] = (c[k] + 1) % g.ns;
        int cbk[4] = {c[0], c[1], c[2], c[3]};
        cbk[k] = (c[k] - 1 + g.ns) % g.ns;
        long sf = site_of(g, cf), sb = site_of(g, cbk);
        long xf = sf - (long)t * g.V3, xb = sb - (long)t * g.V3;
        const c64 *uf = U + (((long)t * g.V3 + x) * 4 + k) * 9;
        const c64 *ub = U + (sb * 4 + k) * 9;
        c64 pf[3], pb[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            pf[i] = src[xf * 3 + i];
            pb[i] = src[xb * 3 + i];
        }
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            c64 s{0, 0};
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                s += uf[i * 3 + j] * pf[j];
                s += cmul_conj(ub[j * 3 + i], pb[j]);
            }
            acc[i] -= s;
        }
    }
    double a = ca[t], b = cb[t];
    c64 *dst = out + (long)t * out_tstride + (long)v * 3 * g.V3;
    const c64 *pv = prev ? prev + (long)t * out_tstride + (long)v * 3 * g.V3 : nullptr;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        c64 y = alpha * (a * acc[i] + b * psi[i]);
        if (use_prev) y -= pv[x * 3 + i];
        dst[x * 3 + i] = y;
    }
}

// ------------------------------------------------------------------ block reductions
__device__ __forceinline__ c64 block_sum(c64 v, c64 *sm) {
    sm[threadIdx.x] = v;
    __syncthreads();
    for (int st = blockDim.x / 2; st > 0; st >>= 1) {
        if ((int)threadIdx.x < st) sm[threadIdx.x] += sm[threadIdx.x + st];
        __syncthreads();
    }
    c64 r = sm[0];
    __syncthreads();
    return r;
}

// h[t][i] = <V[t][i], w[t]> for i < cnt; blocks (t, i); skipped for slices whose flag is 0 when pass > 0
__global__ void gemv_c_kernel(long n, int ldv, const c64 *__restrict__ V, const c64 *__restrict__ w, int cnt,
                              c64 *h, const int *flag, int pass) {
    __shared__ c64 sm[256];
    int t = blockIdx.y, i = blockIdx.x;
    if (i >= cnt) return;
    if (pass > 0 && !flag[t]) return;
    const c64 *v = V + ((long)t * ldv + i) * n;
    const c64 *ww = w + (long)t * n;
    c64 a{0, 0};
    for (long k = threadIdx.x; k < n; k += blockDim.x) a += cmul_conj(v[k], ww[k]);
    c64 s = block_sum(a, sm);
    if (threadIdx.x == 0) h[(long)t * (ldv + 1) + i] = s;
}

// w[t] -= sum_i V[t][i] h[t][i];  hacc += h
__global__ void gemv_n_kernel(long n, int ldv, const c64 *__restrict__ V, c64 *w, int cnt, const c64 *__restrict__ h,
                              const int *flag, int pass) {
    int t = blockIdx.y;
    if (pass > 0 && !flag[t]) return;
    long k = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const c64 *hh = h + (long)t * (ldv + 1);
    c64 s{0, 0};
    for (int i = 0; i < cnt; ++i) s += V[((long)t * ldv + i) * n + k] * hh[i];
    w[(long)t * n + k] -= s;
}

// nrm[t] = ||w[t]||; flag[t] = another pass needed (norm fell by more than 1/sqrt 2, < 4 repeats);
// accumulates h into column j of H (pass > 0 only for flagged slices).
__global__ void reorth_norm_kernel(long n, int ldv, const c64 *w, const c64 *h, c64 *H, int j, int cnt, double *nrm,
                                   int *flag, int pass) {
    __shared__ c64 sm[256];
    int t = blockIdx.x;
    bool active = pass == 0 || flag[t];
    if (!active) return;
    const c64 *ww = w + (long)t * n;
    c64 a{0, 0};
    for (long k = threadIdx.x; k < n; k += blockDim.x) a += c64{norm2(ww[k]), 0.0};
    c64 s = block_sum(a, sm);
    const c64 *hh = h + (long)t * (ldv + 1);
    c64 *Ht = H + (long)t * ldv * ldv;   // H[t][row][col], ldv x ldv
    for (int i = threadIdx.x; i < cnt; i += blockDim.x) Ht[(long)i * ldv + j] += hh[i];
    if (threadIdx.x == 0) {
        double after = sqrt(s.re);
        double before = nrm[t];
        nrm[t] = after;
        flag[t] = (pass < 4 && after < before * 0.7071067811865476) ? 1 : 0;
    }
}

__global__ void norm_only_kernel(long n, const c64 *w, double *nrm) {
    __shared__ c64 sm[256];
    int t = blockIdx.x;
    const c64 *ww = w + (long)t * n;
    c64 a{0, 0};
    for (long k = threadIdx.x; k < n; k += blockDim.x) a += c64{norm2(ww[k]), 0.0};
    c64 s = block_sum(a, sm);
    if (threadIdx.x == 0) nrm[t] = sqrt(s.re);
}

// V[t][j+1] = w / nrm; H[j+1][j] = nrm (when j+1 < ldv rows)
__global__ void lanczos_next_kernel(long n, int ldv, int j, const c64 *w, const double *nrm, c64 *V, c64 *H) {
    int t = blockIdx.y;
    long k = (long)blockIdx.x * blockDim.x + threadIdx.x;
    double b = nrm[t];
    double inv = b > 0.0 ? 1.0 / b : 0.0;
    if (k < n) V[((long)t * ldv + j + 1) * n + k] = inv * w[(long)t * n + k];
    if (k == 0 && j >= 0 && j + 1 < ldv) H[(long)t * ldv * ldv + (long)(j + 1) * ldv + j] = c64{b, 0.0};
}

__global__ void scale_kernel(long n, c64 *v, const double *nrm) {
    int t = blockIdx.y;
    long k = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    double b = nrm[t];
    v[(long)t * n + k] = (b > 0.0 ? 1.0 / b : 0.0) * v[(long)t * n + k];
}

// ------------------------------------------------------------------ batched complex Jacobi
// One block per slice: eigen-decomposition of the Hermitian m x m leading part of H
// (row stride ldh).  Outputs theta[t][0..m) descending and Y[t][row][col] (eigenvectors in columns).
__global__ void jacobi_kernel(int m, int ldh, const c64 *H, c64 *J, c64 *Y, c64 *Ysorted, double *theta,
                              int max_sweeps, int ascending, int in_smem) {
    extern __shared__ double jsm[];   // reduction scratch, per-pair rotation parameters, [A, Z]
    const int t = blockIdx.x;
    const int mm = (m + 1) & ~1;      // even count of players (a dummy index when m is odd)
    const int npair = mm / 2;
    double *red = jsm;                 // 2 * blockDim doubles (also the sort order at the end)
    double *cs = red + 2 * blockDim.x, *sn = cs + npair;
    c64 *ph = (c64 *)(sn + npair);
    int *pp = (int *)(ph + npair);
    int *qq = pp + npair;
    // the working matrix and the rotations live in shared memory when they fit, else in global
    c64 *sm_mats = (c64 *)(((uintptr_t)(qq + npair) + 15) & ~(uintptr_t)15);
    c64 *A = in_smem ? sm_mats : J + (long)t * m * m;
    c64 *Z = in_smem ? sm_mats + (long)m * m : Y + (long)t * m * m;
    const c64 *Hs = H + (long)t * ldh * ldh;
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
        int i = e / m, j = e % m;
        c64 v = 0.5 * (Hs[(long)i * ldh + j] + conj(Hs[(long)j * ldh + i]));
        if (i == j) v.im = 0.0;
        A[e] = v;
        Z[e] = c64{i == j ? 1.0 : 0.0, 0.0};
    }
    __syncthreads();
    for (int sweep = 0; sweep < max_sweeps; ++sweep) {
        // off-diagonal and total Frobenius norms
        double off = 0.0, tot = 0.0;
        for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
            double v = norm2(A[e]);
            tot += v;
            if (e / m != e % m) off += v;
        }
        red[threadIdx.x] = off;
        red[blockDim.x + threadIdx.x] = tot;
        __syncthreads();
        for (int st = blockDim.x / 2; st > 0; st >>= 1) {
            if ((int)threadIdx.x < st) {
                red[threadIdx.x] += red[threadIdx.x + st];
                red[blockDim.x + threadIdx.x] += red[blockDim.x + threadIdx.x + st];
            }
            __syncthreads();
        }
        double offn = red[0], totn = red[blockDim.x];
        __syncthreads();
        if (offn <= 1e-30 * totn || offn == 0.0) break;
        for (int round = 0; round < mm - 1; ++round) {
            // circle schedule: (mm-1, round) and ((round+k) mod (mm-1), (round-k) mod (mm-1))
            for (int k = threadIdx.x; k < npair; k += blockDim.x) {
                int p, q;
                if (k == 0) {
                    p = mm - 1;
                    q = round;
                } else {
                    p = (round + k) % (mm - 1);
                    q = (round - k + (mm - 1)) % (mm - 1);
                }
                if (p > q) { int tmp = p; p = q; q = tmp; }
                pp[k] = p;
                qq[k] = q;
                double c = 1.0, s = 0.0;
                c64 e{1.0, 0.0};
                if (q < m) {
                    c64 apq = A[(long)p * m + q];
                    double mag = sqrt(norm2(apq));
                    if (mag > 1e-300) {
                        double app = A[(long)p * m + p].re, aqq = A[(long)q * m + q].re;
                        double tau = (aqq - app) / (2.0 * mag);
                        double tt = (tau >= 0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
                        c = 1.0 / sqrt(1.0 + tt * tt);
                        s = -tt * c;   // G = diag(1, e^{-i phi}) [[c, -s], [s, c]] zeroes A_pq
                        e = c64{apq.re / mag, apq.im / mag};   // e^{i phi}
                    }
                }
                cs[k] = c;
                sn[k] = s;
                ph[k] = e;
            }
            __syncthreads();
            // rows: A <- G^dag A, G = [[c, -s], [s e^{-i phi}, c e^{-i phi}]] on (p, q)
            for (int e2 = threadIdx.x; e2 < npair * m; e2 += blockDim.x) {
                int k = e2 / m, j = e2 % m;
                int p = pp[k], q = qq[k];
                if (q >= m || sn[k] == 0.0) continue;
                c64 ep = ph[k];
                c64 apj = A[(long)p * m + j], aqj = A[(long)q * m + j];
                A[(long)p * m + j] = cs[k] * apj + sn[k] * (ep * aqj);
                A[(long)q * m + j] = (-sn[k]) * apj + cs[k] * (ep * aqj);
            }
            __syncthreads();
            // columns: A <- A G,  Z <- Z G
            for (int e2 = threadIdx.x; e2 < npair * m; e2 += blockDim.x) {
                int k = e2 / m, i = e2 % m;
                int p = pp[k], q = qq[k];
                if (q >= m || sn[k] == 0.0) continue;
                c64 em = conj(ph[k]);
                c64 aip = A[(long)i * m + p], aiq = A[(long)i * m + q];
                A[(long)i * m + p] = cs[k] * aip + sn[k] * (aiq * em);
                A[(long)i * m + q] = (-sn[k]) * aip + cs[k] * (aiq * em);
                c64 zip = Z[(long)i * m + p], ziq = Z[(long)i * m + q];
                Z[(long)i * m + p] = cs[k] * zip + sn[k] * (ziq * em);
                Z[(long)i * m + q] = (-sn[k]) * zip + cs[k] * (ziq * em);
            }
            __syncthreads();
            for (int k = threadIdx.x; k < npair; k += blockDim.x) {
                int p = pp[k], q = qq[k];
                if (q >= m || sn[k] == 0.0) continue;
                A[(long)p * m + q] = c64{0, 0};
                A[(long)q * m + p] = c64{0, 0};
                A[(long)p * m + p].im = 0.0;
                A[(long)q * m + q].im = 0.0;
            }
            __syncthreads();
        }
    }
    // sort descending (thread 0 builds the order, all threads permute)
    int *order = (int *)red;
    if (threadIdx.x == 0) {
        for (int i = 0; i < m; ++i) order[i] = i;
        for (int i = 0; i < m; ++i) {
            int best = i;
            for (int j = i + 1; j < m; ++j) {
                double vj = A[(long)order[j] * m + order[j]].re, vb = A[(long)order[best] * m + order[best]].re;
                if (ascending ? vj < vb : vj > vb) best = j;
            }
            int tmp = order[i]; order[i] = order[best]; order[best] = tmp;
        }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
        int i = e / m, j = e % m;
        Ysorted[(long)t * m * m + e] = Z[(long)i * m + order[j]];
    }
    for (int j = threadIdx.x; j < m; j += blockDim.x) theta[(long)t * m + j] = A[(long)order[j] * m + order[j]].re;
}

// ------------------------------------------------------------------ restart GEMM
// Out[t][c] = sum_{j < m} V[t][j] Y[t][j][c] for c < k.  Tiled: 64 rows x 16 columns per block.
__global__ void __launch_bounds__(256) rotate_kernel(long n, int ldv, int m, int k, const c64 *__restrict__ V,
                                                      const c64 *__restrict__ Y, c64 *__restrict__ Out) {
    __shared__ c64 Ys[32][16];
    __shared__ c64 Vs[32][65];
    int t = blockIdx.z;
    long r0 = (long)blockIdx.x * 64;
    int c0 = blockIdx.y * 16;
    int tr = threadIdx.x % 64, tc = threadIdx.x / 64;   // 64 rows x 4 column groups of 4
    c64 acc[4] = {{0, 0}, {0, 0}, {0, 0}, {0, 0}};
    for (int j0 = 0; j0 < m; j0 += 32) {
        for (int e = threadIdx.x; e < 32 * 16; e += blockDim.x) {
            int jj = e / 16, cc = e % 16;
            int j = j0 + jj, c = c0 + cc;
            Ys[jj][cc] = (j < m && c < k) ? Y[((long)t * m + j) * m + c] : c64{0, 0};
        }
        for (int e = threadIdx.x; e < 32 * 64; e += blockDim.x) {
            int jj = e / 64, rr = e % 64;
            int j = j0 + jj;
            long row = r0 + rr;
            Vs[jj][rr] = (j < m && row < n) ? V[((long)t * ldv + j) * n + row] : c64{0, 0};
        }
        __syncthreads();
#pragma unroll 4
        for (int jj = 0; jj < 32; ++jj) {
            c64 v = Vs[jj][tr];
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[q] += v * Ys[jj][tc * 4 + q];
        }
        __syncthreads();
    }
    long row = r0 + tr;
    if (row < n)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            int c = c0 + tc * 4 + q;
            if (c < k) Out[((long)t * k + c) * n + row] = acc[q];
        }
}

// ------------------------------------------------------------------ Ritz residuals on -Delta
// mu[t][i] = <y, L y>, res[t][i] = ||L y - mu y|| for the first nv Ritz vectors (blocks (i, t));
// Yv holds ldy vectors per slice, LY holds ldl vectors per slice.
__global__ void ritz_resid_kernel(long n, int nv, int ldy, int ldl, const c64 *Yv, const c64 *LY, double *mu,
                                  double *res) {
    __shared__ c64 sm[256];
    int i = blockIdx.x, t = blockIdx.y;
    const c64 *y = Yv + ((long)t * ldy + i) * n;
    const c64 *ly = LY + ((long)t * ldl + i) * n;
    c64 a{0, 0};
    for (long k = threadIdx.x; k < n; k += blockDim.x) a += cmul_conj(y[k], ly[k]);
    c64 yy{0, 0};
    for (long k = threadIdx.x; k < n; k += blockDim.x) yy += c64{norm2(y[k]), 0};
    c64 num = block_sum(a, sm);
    c64 den = block_sum(yy, sm);
    double m_ = num.re / den.re;
    c64 r{0, 0};
    for (long k = threadIdx.x; k < n; k += blockDim.x) r += c64{norm2(ly[k] - m_ * y[k]), 0};
    c64 rr = block_sum(r, sm);
    if (threadIdx.x == 0) {
        mu[(long)t * nv + i] = m_;
        res[(long)t * nv + i] = sqrt(rr.re / den.re);
    }
}

// ------------------------------------------------------------------ block operations of the polish
// G[t][a][b] = <A[t][a], B[t][b]> for k vectors of length n per slice; 16 x 16 tile per block.
__global__ void __launch_bounds__(256) gram_kernel(long n, int k, const c64 *__restrict__ A, const c64 *__restrict__ B,
                                                    c64 *__restrict__ G) {
    __shared__ c64 As[16][33], Bs[16][33];
    int t = blockIdx.z, a0 = blockIdx.x * 16, b0 = blockIdx.y * 16;
    int ta = threadIdx.x / 16, tb = threadIdx.x % 16;
    c64 acc{0, 0};
    for (long k0 = 0; k0 < n; k0 += 32) {
        for (int e = threadIdx.x; e < 16 * 32; e += blockDim.x) {
            int r = e / 32, kk = e % 32;
            long col = k0 + kk;
            As[r][kk] = (a0 + r < k && col < n) ? A[((long)t * k + a0 + r) * n + col] : c64{0, 0};
            Bs[r][kk] = (b0 + r < k && col < n) ? B[((long)t * k + b0 + r) * n + col] : c64{0, 0};
        }
        __syncthreads();
#pragma unroll 8
        for (int kk = 0; kk < 32; ++kk) acc += cmul_conj(As[ta][kk], Bs[tb][kk]);
        __syncthreads();
    }
    if (a0 + ta < k && b0 + tb < k) G[((long)t * k + a0 + ta) * k + b0 + tb] = acc;
}

// M[t][j][c] = W[t][j][c] / sqrt(w[t][c])  (Loewdin orthonormalisation Y M, with S = W diag(w) W^dag)
__global__ void lowdin_kernel(int k, const c64 *W, const double *w, c64 *M) {
    int t = blockIdx.x;
    for (int e = threadIdx.x; e < k * k; e += blockDim.x) {
        int c = e % k;
        double s = w[(long)t * k + c];
        M[(long)t * k * k + e] = (s > 0 ? 1.0 / sqrt(s) : 0.0) * W[(long)t * k * k + e];
    }
}

// ------------------------------------------------------------------ phase convention
// Each vector: the first component (storage order) whose modulus is within a relative
// 1e-8 of the largest is made real and positive.  Blocks (i, t); writes output evecs.
__global__ void phase_fix_kernel(long n, int nv, const c64 *in, const int *perm, c64 *out) {
    __shared__ double smax[256];
    __shared__ long sidx[256];
    int i = blockIdx.x, t = blockIdx.y;
    const c64 *v = in + ((long)t * nv + perm[(long)t * nv + i]) * n;
    double mx = 0.0;
    for (long k = threadIdx.x; k < n; k += blockDim.x) mx = fmax(mx, norm2(v[k]));
    smax[threadIdx.x] = mx;
    __syncthreads();
    for (int st = blockDim.x / 2; st > 0; st >>= 1) {
        if ((int)threadIdx.x < st) smax[threadIdx.x] = fmax(smax[threadIdx.x], smax[threadIdx.x + st]);
        __syncthreads();
    }
    double thr = sqrt(smax[0]) * (1.0 - 1e-8);
    __syncthreads();
    long first = n;
    for (long k = threadIdx.x; k < n; k += blockDim.x)
        if (sqrt(norm2(v[k])) >= thr && k < first) { first = k; break; }
    sidx[threadIdx.x] = first;
    __syncthreads();
    for (int st = blockDim.x / 2; st > 0; st >>= 1) {
        if ((int)threadIdx.x < st) sidx[threadIdx.x] = min(sidx[threadIdx.x], sidx[threadIdx.x + st]);
        __syncthreads();
    }
    long j = sidx[0];
    c64 vj = v[j < n ? j : 0];
    double mag = sqrt(norm2(vj));
    c64 rot = mag > 0 ? c64{vj.re / mag, -vj.im / mag} : c64{1.0, 0.0};
    c64 *o = out + ((long)t * nv + i) * n;
    for (long k = threadIdx.x; k < n; k += blockDim.x) o[k] = v[k] * rot;
}

// ------------------------------------------------------------------ start vector
__global__ void const_fill_kernel(long n, int nt, c64 *v, double val) {
    long k = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n * nt) v[k] = c64{val, 0.0};
}

__global__ void copy_slices_kernel(long n, const c64 *src, long src_stride, c64 *dst, long dst_stride) {
    int t = blockIdx.y;
    long k = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) dst[(long)t * dst_stride + k] = src[(long)t * src_stride + k];
}

// ------------------------------------------------------------------ driver
struct Lanczos {
    laph_ctx *ctx;
    Geom g;
    long n;
    int nt, m, ldv;   // ldv = m + 1 basis vectors
    const c64 *U;
    c64 *V, *w, *c0, *c1, *H, *h;
    double *nrm, *ca, *cb;
    int *flag;
    int ncheb;
    cudaStream_t s;
    long matvecs = 0;

    void apply_A(const c64 *x, c64 *y) {
        // y = T_ncheb(B) x.  T_0 = x (read only); T_k goes to bufs[(ncheb - k) % 3] with
        // bufs = {y, c0, c1}, so T_ncheb lands in y and T_k, T_{k-1}, T_{k-2} never share a buffer.
        long tot = (long)nt * g.V3;
        unsigned grid = grid_for(tot, 128);
        c64 *bufs[3] = {y, c0, c1};
        auto buf = [&](int k) { return bufs[(ncheb - k) % 3]; };
        prof_begin("eig_cheb", s);
        cheb_kernel<<<grid, 128, 0, s>>>(g, U, 1, x, nullptr, buf(1), ca, cb, 1.0, 0, n, n);
        LAPH_LAUNCH_CHECK();
        for (int k = 2; k <= ncheb; ++k) {
            const c64 *tm2 = (k == 2) ? x : buf(k - 2);
            cheb_kernel<<<grid, 128, 0, s>>>(g, U, 1, buf(k - 1), tm2, buf(k), ca, cb, 2.0, 1, n, n);
            LAPH_LAUNCH_CHECK();
        }
        prof_end("eig_cheb", s, 0.0, 0.0);
        matvecs += ncheb;
    }

    // One Lanczos step j: V[:, j+1] from A V[:, j], full reorthogonalisation.
    void step(int j) {
        // w = A v_j; v_j (slice t at V + (t*ldv + j)*n) is first gathered into a dense [t][n] block
        copy_slices_kernel<<<dim3(grid_for(n, 256), nt), 256, 0, s>>>(n, V + (long)j * n, (long)ldv * n, h_vec, n);
        LAPH_LAUNCH_CHECK();
        apply_A(h_vec, w);
        norm_only_kernel<<<nt, 256, 0, s>>>(n, w, nrm);
        LAPH_LAUNCH_CHECK();
        int cnt = j + 1;
        prof_begin("eig_reorth", s);
        for (int pass = 0; pass <= 4; ++pass) {
            gemv_c_kernel<<<dim3(cnt, nt), 256, 0, s>>>(n, ldv, V, w, cnt, h, flag, pass);
            LAPH_LAUNCH_CHECK();
            gemv_n_kernel<<<dim3(grid_for(n, 256), nt), 256, 0, s>>>(n, ldv, V, w, cnt, h, flag, pass);
            LAPH_LAUNCH_CHECK();
            reorth_norm_kernel<<<nt, 256, 0, s>>>(n, ldv, w, h, H, j, cnt, nrm, flag, pass);
            LAPH_LAUNCH_CHECK();
        }
        prof_end("eig_reorth", s, 0.0, 0.0);
        lanczos_next_kernel<<<dim3(grid_for(n, 256), nt), 256, 0, s>>>(n, ldv, j, w, nrm, V, H);
        LAPH_LAUNCH_CHECK();
    }
    c64 *h_vec;
};

// Eigen-decomposition of the leading m x m Hermitian part of H[t] (row stride ldh) for every slice.
static void run_jacobi(int nt, int m, int ldh, const c64 *H, c64 *J, c64 *Yraw, c64 *Y, double *theta, bool ascending,
                       cudaStream_t s) {
    int npair = ((m + 1) & ~1) / 2;
    LAPH_REQUIRE(m <= 1024, "Krylov dimension above 1024 is not supported");
    size_t shm = sizeof(double) * 2 * 256 + sizeof(double) * 2 * npair + sizeof(c64) * npair + sizeof(int) * 2 * npair;
    size_t mats = 2 * sizeof(c64) * (size_t)m * m + 16;
    const size_t smem_cap = 220 * 1024;   // below the 227 KB opt-in limit per block
    int in_smem = (shm + mats <= smem_cap) ? 1 : 0;
    if (in_smem) {
        shm += mats;
        LAPH_CUDA(cudaFuncSetAttribute(jacobi_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
    }
    prof_begin("eig_jacobi", s);
    jacobi_kernel<<<nt, 256, shm, s>>>(m, ldh, H, J, Yraw, Y, theta, 60, ascending ? 1 : 0, in_smem);
    LAPH_LAUNCH_CHECK();
    prof_end("eig_jacobi", s, 0.0, 0.0);
}

// Out[t][c] = sum_j In[t][j] C[t][j][c]   (k x k coefficients, ldv input vectors per slice)
static void rotate(long n, int nt, int ldv, int m, int k, const c64 *In, const c64 *C, c64 *Out, cudaStream_t s) {
    dim3 rg((unsigned)((n + 63) / 64), (unsigned)((k + 15) / 16), nt);
    prof_begin("eig_gemm", s);
    rotate_kernel<<<rg, 256, 0, s>>>(n, ldv, m, k, In, C, Out);
    LAPH_LAUNCH_CHECK();
    prof_end("eig_gemm", s, 0.0, 0.0);
}

}  // namespace laph

using namespace laph;

extern "C" int laph_eigvecs(laph_ctx *ctx, const laph_lattice *lat, const void *links3d, int nv,
                            const laph_eig_params *params, double *evals, void *evecs, laph_eig_report *report,
                            void *stream) {
    int not_conv = 0;
    int rc = guard([&] {
        ctx_activate(ctx);
        Geom g = make_geom(lat);
        const long n = 3 * g.V3;
        LAPH_REQUIRE(nv >= 1 && 2 * (long)nv <= n, "nv out of range (1 <= nv <= 3 V3 / 2)");
        laph_eig_params prm{};
        if (params) prm = *params;
        double lamL = prm.lambda_L > 0 ? prm.lambda_L : 15.0;
        int ncheb = prm.cheb_order > 0 ? prm.cheb_order : 16;
        int m = prm.krylov_dim > 0 ? prm.krylov_dim : std::max(2 * nv + 16, nv + 32);
        m = (int)std::min<long>(m, n - 1);
        LAPH_REQUIRE(m > nv, "krylov_dim must exceed nv");
        int max_restarts = prm.max_restarts > 0 ? prm.max_restarts : 50;
        double tol = prm.tol > 0 ? prm.tol : 1e-13;
        uint64_t seed = params ? prm.seed : 12345u;
        cudaStream_t s = as_stream(stream);
        const int nt = g.nt;

        const c64 *U = (const c64 *)stage_in(ctx, links3d, sizeof(c64) * 36 * g.V, "eig_links", s);
        Lanczos lz;
        lz.ctx = ctx;
        lz.g = g;
        lz.n = n;
        lz.nt = nt;
        lz.m = m;
        lz.ldv = m + 1;
        lz.U = U;
        lz.s = s;
        lz.V = (c64 *)ws_get(ctx, "eig:V", sizeof(c64) * nt * (size_t)(m + 1) * n);
        lz.w = (c64 *)ws_get(ctx, "eig:w", sizeof(c64) * nt * n);
        lz.c0 = (c64 *)ws_get(ctx, "eig:c0", sizeof(c64) * nt * n);
        lz.c1 = (c64 *)ws_get(ctx, "eig:c1", sizeof(c64) * nt * n);
        lz.h_vec = (c64 *)ws_get(ctx, "eig:x", sizeof(c64) * nt * n);
        lz.H = (c64 *)ws_get(ctx, "eig:H", sizeof(c64) * nt * (size_t)(m + 1) * (m + 1));
        lz.h = (c64 *)ws_get(ctx, "eig:h", sizeof(c64) * nt * (size_t)(m + 2));
        lz.nrm = (double *)ws_get(ctx, "eig:nrm", sizeof(double) * nt);
        lz.ca = (double *)ws_get(ctx, "eig:ca", sizeof(double) * nt);
        lz.cb = (double *)ws_get(ctx, "eig:cb", sizeof(double) * nt);
        lz.flag = (int *)ws_get(ctx, "eig:flag", sizeof(int) * nt);
        c64 *J = (c64 *)ws_get(ctx, "eig:J", sizeof(c64) * nt * (size_t)m * m);
        c64 *Yraw = (c64 *)ws_get(ctx, "eig:Yraw", sizeof(c64) * nt * (size_t)m * m);
        c64 *Y = (c64 *)ws_get(ctx, "eig:Y", sizeof(c64) * nt * (size_t)m * m);
        double *theta = (double *)ws_get(ctx, "eig:theta", sizeof(double) * nt * m);
        c64 *Vt = (c64 *)ws_get(ctx, "eig:Vt", sizeof(c64) * nt * (size_t)m * n);
        c64 *LY = (c64 *)ws_get(ctx, "eig:LY", sizeof(c64) * nt * (size_t)nv * n);
        double *mu = (double *)ws_get(ctx, "eig:mu", sizeof(double) * nt * nv);
        double *res = (double *)ws_get(ctx, "eig:res", sizeof(double) * nt * nv);
        std::vector<double> ha(nt), hb(nt);
        auto set_map = [&](const std::vector<double> &lamC, int order) {
            for (int t = 0; t < nt; ++t) {
                if (order == 1 && lamC.empty()) {
                    ha[t] = -1.0;   // A = -(-Delta): the lowest of -Delta become the largest
                    hb[t] = 0.0;
                } else {
                    ha[t] = -2.0 / (lamL - lamC[t]);
                    hb[t] = 1.0 + 2.0 * lamC[t] / (lamL - lamC[t]);
                }
            }
            LAPH_CUDA(cudaMemcpyAsync(lz.ca, ha.data(), sizeof(double) * nt, cudaMemcpyHostToDevice, s));
            LAPH_CUDA(cudaMemcpyAsync(lz.cb, hb.data(), sizeof(double) * nt, cudaMemcpyHostToDevice, s));
            lz.ncheb = order;
            LAPH_CUDA(cudaStreamSynchronize(s));
        };
        auto start_vector = [&]() {
            // v0 per slice: all-equal (seed 0) or seeded Gaussian, normalised
            if (seed == 0) {
                const_fill_kernel<<<grid_for(n * nt, 256), 256, 0, s>>>(n, nt, lz.w, 1.0);
                LAPH_LAUNCH_CHECK();
            } else {
                philox_normal_fill(lz.w, n * nt, (uint32_t)seed, (uint32_t)(seed >> 32), s);
            }
            norm_only_kernel<<<nt, 256, 0, s>>>(n, lz.w, lz.nrm);
            LAPH_LAUNCH_CHECK();
            LAPH_CUDA(cudaMemsetAsync(lz.H, 0, sizeof(c64) * nt * (size_t)(m + 1) * (m + 1), s));
            LAPH_CUDA(cudaMemsetAsync(lz.flag, 0, sizeof(int) * nt, s));
            lanczos_next_kernel<<<dim3(grid_for(n, 256), nt), 256, 0, s>>>(n, m + 1, -1, lz.w, lz.nrm, lz.V, lz.H);
            LAPH_LAUNCH_CHECK();
        };
        std::vector<double> h_theta((size_t)nt * m);

        // 1) cutoff lambda_C: a short unaccelerated Lanczos on -(-Delta).  Ritz values bound the
        //    lowest eigenvalues from above, so the (nv+8)-th Ritz value lies above lambda_{nv}.
        std::vector<double> lamC(nt, prm.lambda_C);
        if (!(prm.lambda_C > 0)) {
            set_map({}, 1);
            start_vector();
            int mest = std::min(m, nv + 24);   // enough Ritz values to bound lambda_{nv+8} from above
            for (int j = 0; j < mest; ++j) lz.step(j);
            run_jacobi(nt, mest, m + 1, lz.H, J, Yraw, Y, theta, false, s);
            LAPH_CUDA(cudaMemcpyAsync(h_theta.data(), theta, sizeof(double) * nt * mest, cudaMemcpyDeviceToHost, s));
            LAPH_CUDA(cudaStreamSynchronize(s));
            int idx = std::min(nv + 8, mest - 1);
            for (int t = 0; t < nt; ++t) lamC[t] = std::min(-h_theta[(size_t)t * mest + idx], 0.8 * lamL);
        }
        int keep = std::min(m - 12, std::max(nv, nv + (m - nv) / 2));
        keep = std::max(keep, nv);
        std::vector<double> h_res((size_t)nt * nv), h_mu((size_t)nt * nv);
        // One Lanczos cycle (steps j0 .. m-1) on the current map, its Ritz vectors Vt = V Y[:, :keep]
        // and the Rayleigh quotients mu and residuals of the nv wanted ones on -Delta itself.
        auto cycle = [&](int j0) {
            for (int j = j0; j < m; ++j) lz.step(j);
            run_jacobi(nt, m, m + 1, lz.H, J, Yraw, Y, theta, false, s);
            rotate(n, nt, m + 1, m, keep, lz.V, Y, Vt, s);
            {
                std::vector<double> one(nt, 1.0), zero(nt, 0.0);
                // LY = (-Delta) Y  with a = 1, b = 0 (temporarily swap the map coefficients)
                LAPH_CUDA(cudaMemcpyAsync(lz.ca, one.data(), sizeof(double) * nt, cudaMemcpyHostToDevice, s));
                LAPH_CUDA(cudaMemcpyAsync(lz.cb, zero.data(), sizeof(double) * nt, cudaMemcpyHostToDevice, s));
                long tot = (long)nt * nv * g.V3;
                cheb_kernel<<<grid_for(tot, 128), 128, 0, s>>>(g, U, nv, Vt, nullptr, LY, lz.ca, lz.cb, 1.0, 0,
                                                               (long)keep * n, (long)nv * n);
                LAPH_LAUNCH_CHECK();
                lz.matvecs += nv;
                ritz_resid_kernel<<<dim3(nv, nt), 256, 0, s>>>(n, nv, keep, nv, Vt, LY, mu, res);
                LAPH_LAUNCH_CHECK();
                LAPH_CUDA(cudaMemcpyAsync(lz.ca, ha.data(), sizeof(double) * nt, cudaMemcpyHostToDevice, s));
                LAPH_CUDA(cudaMemcpyAsync(lz.cb, hb.data(), sizeof(double) * nt, cudaMemcpyHostToDevice, s));
                LAPH_CUDA(cudaMemcpyAsync(h_res.data(), res, sizeof(double) * nt * nv, cudaMemcpyDeviceToHost, s));
                LAPH_CUDA(cudaMemcpyAsync(h_mu.data(), mu, sizeof(double) * nt * nv, cudaMemcpyDeviceToHost, s));
                LAPH_CUDA(cudaStreamSynchronize(s));
            }
        };
        // 1b) refined cutoff: the short unaccelerated run bounds lambda_{nv+8} only loosely when the
        //     low end of the spectrum is clustered (on a 24^3 slice it gave about 11 for wanted
        //     eigenvalues near 0.2, which leaves the filter almost flat).  One Chebyshev-filtered
        //     cycle of order 8 on that loose map already points the wanted Ritz vectors at the low
        //     eigenvectors; the cutoff becomes 1.5 times the largest of their Rayleigh quotients on
        //     -Delta (plus 0.02; the paper's 24^3 runs took lambda_C = 0.5 for N_v = 112, about 1.5
        //     lambda_{N_v} there), never above the loose estimate.
        if (!(prm.lambda_C > 0)) {
            set_map(lamC, std::min(ncheb, 8));
            start_vector();
            cycle(0);
            // The cutoff is raised where needed so that the filter amplifies no wanted eigenvalue
            // more than 1e3 times as much as the largest wanted one (T_n(B(0)) / T_n(B(mu_max)), -Delta
            // >= 0): a wider range puts the FP64 rounding floor of the filtered vectors, about
            // eps times that ratio, near the tolerance (seen on 4^3 slices, where N_v = 8 ends
            // inside the shell near 2).
            auto log_t = [&](double x) { return ncheb * std::acosh(std::max(x, 1.0)); };   // ~ log T_n(x), x >= 1
            for (int t = 0; t < nt; ++t) {
                double mx = 0.0;
                for (int i = 0; i < nv; ++i) mx = std::max(mx, h_mu[(size_t)t * nv + i]);
                if (!(std::isfinite(mx) && mx > 0.0)) continue;
                double c = 1.5 * mx + 0.02;
                for (int k = 0; k < 200 && c < lamC[t]; ++k) {
                    const double b0 = 1.0 + 2.0 * c / (lamL - c), bm = 1.0 + 2.0 * (c - mx) / (lamL - c);
                    if (log_t(b0) - log_t(bm) <= std::log(1e3)) break;
                    c *= 1.05;
                }
                lamC[t] = std::min(lamC[t], c);
            }
        }
        // 2) Chebyshev-accelerated thick-restart Lanczos
        set_map(lamC, ncheb);
        start_vector();
        int j0 = 0, restarts = 0;
        double worst = 0.0, prev_worst = 1e300;
        int slow = 0, polish_iters = 0;
        bool done = false;
        for (restarts = 0; restarts <= max_restarts && !done; ++restarts) {
            cycle(j0);
            worst = 0.0;
            for (double r : h_res) worst = std::max(worst, std::isfinite(r) ? r : 1e300);
            if (worst <= tol * 12.0) {
                done = true;
                break;
            }
            // The residual of a Ritz vector of T_n(B) has a floor of order eps ||T_n(B)||, which for a
            // wide wanted spectrum lies above the tolerance on -Delta.  The kept block goes to the
            // polish below once the restarts reach 1e-8 (the polish gains orders of magnitude per
            // pass from there) or stop gaining (twice less than a factor 2).
            slow = (worst > 0.5 * prev_worst) ? slow + 1 : 0;
            prev_worst = std::min(prev_worst, worst);
            if (restarts == max_restarts || worst < 1e-8 || (slow >= 2 && worst < 1e-4) || slow >= 4) break;
            // thick restart: V[:, :keep] = Vt, V[:, keep] = V[:, m]; H = diag(theta) + coupling row
            copy_slices_kernel<<<dim3(grid_for(n, 256), nt), 256, 0, s>>>(n, lz.V + (long)m * n, (long)(m + 1) * n,
                                                                          lz.w, n);
            LAPH_LAUNCH_CHECK();
            for (int c = 0; c < keep; ++c) {
                copy_slices_kernel<<<dim3(grid_for(n, 256), nt), 256, 0, s>>>(n, Vt + (long)c * n, (long)keep * n,
                                                                              lz.V + (long)c * n, (long)(m + 1) * n);
                LAPH_LAUNCH_CHECK();
            }
            copy_slices_kernel<<<dim3(grid_for(n, 256), nt), 256, 0, s>>>(n, lz.w, n, lz.V + (long)keep * n,
                                                                          (long)(m + 1) * n);
            LAPH_LAUNCH_CHECK();
            // host rebuild of H: theta and beta_m * Y[m-1][i]
            std::vector<c64> hY((size_t)nt * m * m), hH((size_t)nt * (m + 1) * (m + 1), c64{0, 0});
            std::vector<c64> hHold((size_t)nt * (m + 1) * (m + 1));
            LAPH_CUDA(cudaMemcpyAsync(hY.data(), Y, sizeof(c64) * hY.size(), cudaMemcpyDeviceToHost, s));
            LAPH_CUDA(cudaMemcpyAsync(hHold.data(), lz.H, sizeof(c64) * hHold.size(), cudaMemcpyDeviceToHost, s));
            LAPH_CUDA(cudaMemcpyAsync(h_theta.data(), theta, sizeof(double) * nt * m, cudaMemcpyDeviceToHost, s));
            LAPH_CUDA(cudaStreamSynchronize(s));
            for (int t = 0; t < nt; ++t) {
                c64 *Ht = hH.data() + (size_t)t * (m + 1) * (m + 1);
                double beta = hHold[(size_t)t * (m + 1) * (m + 1) + (size_t)m * (m + 1) + (m - 1)].re;
                for (int i = 0; i < keep; ++i) {
                    Ht[(size_t)i * (m + 1) + i] = c64{h_theta[(size_t)t * m + i], 0.0};
                    c64 yl = hY[((size_t)t * m + (m - 1)) * m + i];
                    Ht[(size_t)keep * (m + 1) + i] = beta * yl;
                }
            }
            LAPH_CUDA(cudaMemcpyAsync(lz.H, hH.data(), sizeof(c64) * hH.size(), cudaMemcpyHostToDevice, s));
            LAPH_CUDA(cudaStreamSynchronize(s));
            j0 = keep;
        }
        // 3) polish: Chebyshev-filtered subspace iteration on the kept Ritz block Y (keep vectors
        //    per slice): Y <- T_n(B) Y, Loewdin orthonormalisation, Rayleigh-Ritz on -Delta itself.
        //    Components outside the block fall by T_n(B) of the wanted over the rest each pass.
        c64 *cur = Vt;
        if (!done) {
            size_t blk = sizeof(c64) * nt * (size_t)keep * n;
            c64 *F[3] = {(c64 *)ws_get(ctx, "eig:F0", blk), (c64 *)ws_get(ctx, "eig:F1", blk),
                         (c64 *)ws_get(ctx, "eig:F2", blk)};
            c64 *Gk = (c64 *)ws_get(ctx, "eig:Gk", sizeof(c64) * nt * (size_t)keep * keep);
            c64 *LK = (c64 *)ws_get(ctx, "eig:LK", blk);
            long tot = (long)nt * keep * g.V3;
            unsigned cg = grid_for(tot, 128);
            const long ts = (long)keep * n;
            dim3 gg((unsigned)((keep + 15) / 16), (unsigned)((keep + 15) / 16), nt);
            std::vector<double> one(nt, 1.0), zero(nt, 0.0);
            // passes continue while they gain: at most 100, and never after three passes in a row
            // that each cut the worst residual by less than 10 %
            // A single start vector puts only one direction of each exactly degenerate eigenspace
            // into the Krylov space (the free field: every level at least three-fold).  Before the
            // block iteration, every kept column that is not a wanted Ritz vector with residual
            // <= 1e-8 is replaced by a seeded random vector, so the block spans the missing
            // partners; the filter turns the random columns into low modes within a pass or two.
            {
                std::vector<int> hm((size_t)nt * keep, 1);
                for (int t = 0; t < nt; ++t)
                    for (int i = 0; i < nv; ++i) hm[(size_t)t * keep + i] = !(h_res[(size_t)t * nv + i] <= 1e-8);
                int *dm = (int *)ws_get(ctx, "eig:rmask", sizeof(int) * nt * (size_t)keep);
                LAPH_CUDA(cudaMemcpyAsync(dm, hm.data(), sizeof(int) * hm.size(), cudaMemcpyHostToDevice, s));
                randomize_cols_kernel<<<dim3(grid_for(n, 256), keep, nt), 256, 0, s>>>(n, keep, dm,
                                                                                      (uint32_t)(seed ^ 0xA5A5u), Vt);
                LAPH_LAUNCH_CHECK();
                LAPH_CUDA(cudaStreamSynchronize(s));
            }
            double pol_prev = worst;
            int pol_flat = 0;
            for (int it = 0; it < 100 && !done && pol_flat < 3; ++it, ++polish_iters) {
                // filter: T_k into F[(ncheb - k) % 3], T_0 = cur
                const int npol = ncheb;
                auto fb = [&](int k) { return F[(npol - k) % 3]; };
                cheb_kernel<<<cg, 128, 0, s>>>(g, U, keep, cur, nullptr, fb(1), lz.ca, lz.cb, 1.0, 0, ts, ts);
                LAPH_LAUNCH_CHECK();
                for (int k = 2; k <= npol; ++k) {
                    const c64 *tm2 = (k == 2) ? cur : fb(k - 2);
                    cheb_kernel<<<cg, 128, 0, s>>>(g, U, keep, fb(k - 1), tm2, fb(k), lz.ca, lz.cb, 2.0, 1, ts, ts);
                    LAPH_LAUNCH_CHECK();
                }
                lz.matvecs += (long)npol * keep;
                c64 *Yf = F[0];
                // Loewdin: S = Yf^dag Yf = W diag(w) W^dag, Y = Yf W diag(w)^{-1/2}
                gram_kernel<<<gg, 256, 0, s>>>(n, keep, Yf, Yf, Gk);
                LAPH_LAUNCH_CHECK();
                run_jacobi(nt, keep, keep, Gk, J, Yraw, Y, theta, false, s);
                lowdin_kernel<<<nt, 256, 0, s>>>(keep, Y, theta, Yraw);
                LAPH_LAUNCH_CHECK();
                c64 *Yo = (cur == Vt) ? F[1] : Vt;
                rotate(n, nt, keep, keep, keep, Yf, Yraw, Yo, s);
                // Rayleigh-Ritz on -Delta: G = Y^dag L Y, ascending eigenpairs
                LAPH_CUDA(cudaMemcpyAsync(lz.ca, one.data(), sizeof(double) * nt, cudaMemcpyHostToDevice, s));
                LAPH_CUDA(cudaMemcpyAsync(lz.cb, zero.data(), sizeof(double) * nt, cudaMemcpyHostToDevice, s));
                cheb_kernel<<<cg, 128, 0, s>>>(g, U, keep, Yo, nullptr, LK, lz.ca, lz.cb, 1.0, 0, ts, ts);
                LAPH_LAUNCH_CHECK();
                lz.matvecs += keep;
                gram_kernel<<<gg, 256, 0, s>>>(n, keep, Yo, LK, Gk);
                LAPH_LAUNCH_CHECK();
                run_jacobi(nt, keep, keep, Gk, J, Yraw, Y, theta, true, s);
                c64 *Yn = (Yo == Vt) ? F[2] : Vt;
                rotate(n, nt, keep, keep, keep, Yo, Y, Yn, s);
                c64 *LKn = (Yn == F[2]) ? F[0] : F[2];
                rotate(n, nt, keep, keep, keep, LK, Y, LKn, s);
                ritz_resid_kernel<<<dim3(nv, nt), 256, 0, s>>>(n, nv, keep, keep, Yn, LKn, mu, res);
                LAPH_LAUNCH_CHECK();
                LAPH_CUDA(cudaMemcpyAsync(lz.ca, ha.data(), sizeof(double) * nt, cudaMemcpyHostToDevice, s));
                LAPH_CUDA(cudaMemcpyAsync(lz.cb, hb.data(), sizeof(double) * nt, cudaMemcpyHostToDevice, s));
                LAPH_CUDA(cudaMemcpyAsync(h_res.data(), res, sizeof(double) * nt * nv, cudaMemcpyDeviceToHost, s));
                LAPH_CUDA(cudaMemcpyAsync(h_mu.data(), mu, sizeof(double) * nt * nv, cudaMemcpyDeviceToHost, s));
                LAPH_CUDA(cudaStreamSynchronize(s));
                if (Yn != Vt) {
                    LAPH_CUDA(cudaMemcpyAsync(Vt, Yn, blk, cudaMemcpyDeviceToDevice, s));
                }
                cur = Vt;
                worst = 0.0;
                for (double r : h_res) worst = std::max(worst, std::isfinite(r) ? r : 1e300);
                if (worst <= tol * 12.0) done = true;
                pol_flat = (worst > 0.9 * pol_prev) ? pol_flat + 1 : 0;
                pol_prev = std::min(pol_prev, worst);
            }
        }
        // outputs: ascending mu with the phase convention
        std::vector<int> perm((size_t)nt * nv);
        std::vector<double> ev((size_t)nt * nv);
        for (int t = 0; t < nt; ++t) {
            std::vector<int> o(nv);
            for (int i = 0; i < nv; ++i) o[i] = i;
            std::sort(o.begin(), o.end(), [&](int a, int b) { return h_mu[(size_t)t * nv + a] < h_mu[(size_t)t * nv + b]; });
            for (int i = 0; i < nv; ++i) {
                perm[(size_t)t * nv + i] = o[i];
                ev[(size_t)t * nv + i] = h_mu[(size_t)t * nv + o[i]];
            }
        }
        int *dperm = (int *)ws_get(ctx, "eig:perm", sizeof(int) * nt * nv);
        LAPH_CUDA(cudaMemcpyAsync(dperm, perm.data(), sizeof(int) * perm.size(), cudaMemcpyHostToDevice, s));
        // Vt holds [t][keep][n]; gather the nv wanted into a [t][nv][n] block
        for (int c = 0; c < nv; ++c) {
            copy_slices_kernel<<<dim3(grid_for(n, 256), nt), 256, 0, s>>>(n, Vt + (long)c * n, (long)keep * n,
                                                                          LY + (long)c * n, (long)nv * n);
            LAPH_LAUNCH_CHECK();
        }
        StagedOut oe = stage_out(ctx, evecs, sizeof(c64) * nt * (size_t)nv * n, "evecs_out");
        phase_fix_kernel<<<dim3(nv, nt), 256, 0, s>>>(n, nv, LY, dperm, (c64 *)oe.dev);
        LAPH_LAUNCH_CHECK();
        oe.commit(s);
        StagedOut ol = stage_out(ctx, evals, sizeof(double) * nt * nv, "evals_out");
        LAPH_CUDA(cudaMemcpyAsync(ol.dev, ev.data(), sizeof(double) * ev.size(), cudaMemcpyHostToDevice, s));
        ol.commit(s);
        LAPH_CUDA(cudaStreamSynchronize(s));
        if (report) {
            report->restarts = restarts;
            report->matvecs = (int)lz.matvecs;
            int nconv = nv;
            for (int t = 0; t < nt; ++t) {
                int c = 0;
                for (int i = 0; i < nv; ++i) c += h_res[(size_t)t * nv + i] <= tol * 12.0;
                nconv = std::min(nconv, c);
            }
            report->nconv = nconv;
            report->max_resid = worst;
            double lc = 0;
            for (double v : lamC) lc = std::max(lc, v);
            report->lambda_C = lc;
        }
        if (!done) not_conv = 1;
    });
    if (rc == LAPH_OK && not_conv) {
        set_last_error("eigensolver did not reach the tolerance");
        return LAPH_ERR_NOT_CONVERGED;
    }
    return rc;
}
