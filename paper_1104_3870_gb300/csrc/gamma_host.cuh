// Dirac matrices on the host (chiral basis) and the 4x4 spin weight passed to the meson-function
// kernels, shared by the correlator entry points.
#pragma once
#include "common.cuh"

namespace laph {

struct Mat4 {
    c64 m[4][4];
};

inline Mat4 mat_zero() {
    Mat4 r;
    for (auto &row : r.m)
        for (auto &v : row) v = {0, 0};
    return r;
}
inline Mat4 mat_mul(const Mat4 &a, const Mat4 &b) {
    Mat4 r = mat_zero();
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j)
            for (int k = 0; k < 4; ++k) r.m[i][j] += a.m[i][k] * b.m[k][j];
    return r;
}
inline Mat4 mat_dag(const Mat4 &a) {
    Mat4 r;
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) r.m[i][j] = conj(a.m[j][i]);
    return r;
}
inline Mat4 mat_scale(double s, const Mat4 &a) {
    Mat4 r;
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) r.m[i][j] = s * a.m[i][j];
    return r;
}
// chiral basis: gamma_mu = [[0, G], [G^dag, 0]], G_k = -i sigma_k, G_4 = 1
inline Mat4 gamma_mat(int mu) {
    const c64 O{0, 0}, P{1, 0}, M1{-1, 0}, I{0, 1}, Mi{0, -1};
    c64 G[4][2][2] = {{{O, Mi}, {Mi, O}}, {{O, M1}, {P, O}}, {{Mi, O}, {O, I}}, {{P, O}, {O, P}}};
    Mat4 r = mat_zero();
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) {
            r.m[i][2 + j] = G[mu][i][j];
            r.m[2 + i][j] = conj(G[mu][j][i]);
        }
    return r;
}
inline Mat4 gamma5() { return mat_mul(mat_mul(gamma_mat(0), gamma_mat(1)), mat_mul(gamma_mat(2), gamma_mat(3))); }
inline Mat4 ident4() {
    Mat4 r = mat_zero();
    for (int i = 0; i < 4; ++i) r.m[i][i] = {1, 0};
    return r;
}

// spin weight of the meson-function kernels
struct W4 {
    c64 w[4][4];
};
inline W4 to_w4(const Mat4 &m) {
    W4 w;
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) w.w[i][j] = m.m[i][j];
    return w;
}

// c = gamma_4 Gamma of a meson channel's components (pion gamma_5, rho gamma_1..3, scalar 1);
// returns the number of components
inline int channel_c(int channel, Mat4 out[3]) {
    const Mat4 g4 = gamma_mat(3);
    if (channel == LAPH_CH_RHO) {
        for (int k = 0; k < 3; ++k) out[k] = mat_mul(g4, gamma_mat(k));
        return 3;
    }
    out[0] = mat_mul(g4, channel == LAPH_CH_PION ? gamma5() : ident4());
    return 1;
}

// ABI projector masks (correlate.cu) and the diluted noise of each projector at t0
std::vector<uint8_t> dilution_masks(const laph_dilution &d, int nt, int nv, const int *b_list, int nb);
__global__ void rho_at_t0_kernel(int nt, int nv, int nb, int t0, const uint8_t *codes, const uint8_t *mask, c64 *out);
__global__ void meson_fn_kernel(int nv, int nb, int ntA, int ntB, const c64 *__restrict__ A, const c64 *__restrict__ B,
                                W4 W, c64 *__restrict__ M);
__global__ void contract2_kernel(int nt, int nb, int t0, const c64 *Msink, const c64 *Msrc, double scale, c64 *corr);

}  // namespace laph
