// Small dense 3x3 complex matrix helpers (FP64) used by the gauge kernels.
#pragma once
#include "common.cuh"

namespace laph {

struct M3 {
    c64 m[3][3];
};

__device__ __forceinline__ M3 m3_load(const c64 *p) {
    M3 r;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) r.m[i][j] = p[i * 3 + j];
    return r;
}

__device__ __forceinline__ void m3_store(c64 *p, const M3 &a) {
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) p[i * 3 + j] = a.m[i][j];
}

__device__ __forceinline__ M3 m3_zero() {
    M3 r;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) r.m[i][j] = c64{0.0, 0.0};
    return r;
}

__device__ __forceinline__ M3 m3_eye() {
    M3 r = m3_zero();
    r.m[0][0].re = r.m[1][1].re = r.m[2][2].re = 1.0;
    return r;
}

// a * b
__device__ __forceinline__ M3 m3_mul(const M3 &a, const M3 &b) {
    M3 r;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            c64 s = a.m[i][0] * b.m[0][j];
            s += a.m[i][1] * b.m[1][j];
            s += a.m[i][2] * b.m[2][j];
            r.m[i][j] = s;
        }
    return r;
}

// a * b^dag
__device__ __forceinline__ M3 m3_mul_nd(const M3 &a, const M3 &b) {
    M3 r;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            c64 s = a.m[i][0] * conj(b.m[j][0]);
            s += a.m[i][1] * conj(b.m[j][1]);
            s += a.m[i][2] * conj(b.m[j][2]);
            r.m[i][j] = s;
        }
    return r;
}

// a^dag * b
__device__ __forceinline__ M3 m3_mul_dn(const M3 &a, const M3 &b) {
    M3 r;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            c64 s = conj(a.m[0][i]) * b.m[0][j];
            s += conj(a.m[1][i]) * b.m[1][j];
            s += conj(a.m[2][i]) * b.m[2][j];
            r.m[i][j] = s;
        }
    return r;
}

__device__ __forceinline__ M3 m3_dag(const M3 &a) {
    M3 r;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) r.m[i][j] = conj(a.m[j][i]);
    return r;
}

__device__ __forceinline__ void m3_add(M3 &a, const M3 &b) {
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) a.m[i][j] += b.m[i][j];
}

__device__ __forceinline__ M3 m3_scale(double s, const M3 &a) {
    M3 r;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) r.m[i][j] = s * a.m[i][j];
    return r;
}

__device__ __forceinline__ double m3_frob(const M3 &a) {
    double s = 0;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) s += norm2(a.m[i][j]);
    return sqrt(s);
}

// exp(X) for a small anti-Hermitian X by scaling and squaring (Moler & Van
// Loan, "Nineteen dubious ways to compute the exponential of a matrix"):
// X / 2^k with ||X / 2^k||_F <= 1/8, Taylor series to order 14, then k squarings.
__device__ __forceinline__ M3 m3_expm(const M3 &x) {
    double nrm = m3_frob(x);
    int k = 0;
    while (nrm > 0.125 && k < 40) {
        nrm *= 0.5;
        ++k;
    }
    M3 xs = m3_scale(ldexp(1.0, -k), x);
    // Horner form of sum_{j=0}^{14} xs^j / j!
    M3 r = m3_eye();
    for (int j = 14; j >= 1; --j) {
        r = m3_mul(xs, r);
        r = m3_scale(1.0 / j, r);
        r.m[0][0].re += 1.0;
        r.m[1][1].re += 1.0;
        r.m[2][2].re += 1.0;
    }
    for (int i = 0; i < k; ++i) r = m3_mul(r, r);
    return r;
}

}  // namespace laph
