// Z4 noise in the LapH subspace and diluted sources (Sec. II, Eq. (varrhodef)
// with D = 1; dilution projectors P^(b) = P_T (x) P_S (x) P_L; Sec. IV noise).
//
// Noise: Philox4x32-10 (Salmon et al., SC'11) written from its definition:
// ten rounds of (hi0,lo0) = mulhilo(0xD2511F53, c0), (hi1,lo1) = mulhilo(0xCD9E8D57, c2),
// c <- (hi1^c1^k0, lo1, hi0^c3^k1, lo0), with the key bumped by
// (0x9E3779B9, 0xBB67AE85) before every round after the first.
// rho(t, alpha, n) = i^(w0 & 3) with counter ((t*4 + alpha)*nv + n, 0, 0, 0) and
// key ((config_id << 16) | noise_id, 0x4C415048).
#include <vector>

#include "common.cuh"
#include "philox.cuh"

namespace laph {

__global__ void z4_kernel(int n, uint32_t key0, uint8_t *codes) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint32_t c[4] = {(uint32_t)i, 0u, 0u, 0u};
    philox4x32_10(c, key0, 0x4C415048u);
    codes[i] = (uint8_t)(c[0] & 3u);
}

void z4_codes(int nt, int nv, uint16_t noise_id, uint16_t config_id, uint8_t *codes, cudaStream_t s) {
    int n = nt * 4 * nv;
    uint32_t key0 = ((uint32_t)config_id << 16) | (uint32_t)noise_id;
    z4_kernel<<<grid_for(n, 256), 256, 0, s>>>(n, key0, codes);
    LAPH_LAUNCH_CHECK();
}

// Projector diagonal of one dilution type (Sec. II table of schemes).
static bool proj(int type, int J, int N, int b, int i) {
    switch (type) {
        case 0: return true;
        case 1: return i == b;
        case 2: return (J * i) / N == b;
        default: return i % J == b;
    }
}

int n_proj(int type, int J, int N) {
    switch (type) {
        case 0: return 1;
        case 1: return N;
        case 2:
        case 3:
            LAPH_REQUIRE(J > 0 && N % J == 0, "dilution J must divide the dimension");
            return J;
        default: throw Error(LAPH_ERR_ARG, "unknown dilution type");
    }
}

// Host table mask[b][nt + 4 + nv] of the diagonals of P_T, P_S, P_L for each listed b.
std::vector<uint8_t> dilution_masks(const laph_dilution &d, int nt, int nv, const int *b_list, int nb) {
    int nT = n_proj(d.T.type, d.T.J, nt), nS = n_proj(d.S.type, d.S.J, 4), nL = n_proj(d.L.type, d.L.J, nv);
    int w = nt + 4 + nv;
    std::vector<uint8_t> m((size_t)nb * w);
    for (int i = 0; i < nb; ++i) {
        int b = b_list[i];
        LAPH_REQUIRE(b >= 0 && b < nT * nS * nL, "projector index out of range");
        int bL = b % nL, bS = (b / nL) % nS, bT = b / (nL * nS);
        for (int t = 0; t < nt; ++t) m[(size_t)i * w + t] = proj(d.T.type, d.T.J, nt, bT, t);
        for (int a = 0; a < 4; ++a) m[(size_t)i * w + nt + a] = proj(d.S.type, d.S.J, 4, bS, a);
        for (int n = 0; n < nv; ++n) m[(size_t)i * w + nt + 4 + n] = proj(d.L.type, d.L.J, nv, bL, n);
    }
    return m;
}

// out[b][site][alpha][c] = (gamma_4 y)_alpha,  y_alpha = sum_n V(t,n,x,c) [P^(b) rho](t,alpha,n).
// gamma_4 swaps the upper and lower spin pairs (chiral basis).
__global__ void sources_kernel(Geom g, int nv, int nb, const c64 *__restrict__ evecs, const uint8_t *__restrict__ codes,
                               const uint8_t *__restrict__ mask, c64 *out) {
    long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
    long per_b = g.V * 3;
    if (idx >= per_b * nb) return;
    int b = (int)(idx / per_b);
    long sc = idx % per_b;
    long s = sc / 3;
    int c = (int)(sc % 3);
    int t = (int)(s / g.V3);
    long x = s % g.V3;
    const int w = g.nt + 4 + nv;
    const uint8_t *m = mask + (long)b * w;
    c64 y[4] = {{0, 0}, {0, 0}, {0, 0}, {0, 0}};
    if (m[t]) {
        const c64 *v = evecs + ((long)t * nv) * g.V3 * 3 + x * 3 + c;
        for (int n = 0; n < nv; ++n) {
            if (!m[g.nt + 4 + n]) continue;
            c64 vn = v[(long)n * g.V3 * 3];
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                if (!m[g.nt + a]) continue;
                int code = codes[(t * 4 + a) * nv + n];
                // i^code * vn
                c64 r = code == 0 ? vn : code == 1 ? times_i(vn) : code == 2 ? -vn : -times_i(vn);
                y[a] += r;
            }
        }
    }
    c64 *o = out + ((long)b * g.V + s) * 12;
    o[0 * 3 + c] = y[2];
    o[1 * 3 + c] = y[3];
    o[2 * 3 + c] = y[0];
    o[3 * 3 + c] = y[1];
}

}  // namespace laph

using namespace laph;

extern "C" int laph_make_sources(laph_ctx *ctx, const laph_lattice *lat, const void *evecs, int nv, uint16_t noise_id,
                                 uint16_t config_id, const laph_dilution *dil, const int *b_list, int nb, void *rhs,
                                 uint8_t *noise, void *stream) {
    return guard([&] {
        ctx_activate(ctx);
        Geom g = make_geom(lat);
        LAPH_REQUIRE(dil != nullptr, "dilution is null");
        LAPH_REQUIRE(nv >= 1 && nv <= 3 * g.V3, "nv out of range");
        LAPH_REQUIRE(nb >= 0, "nb must be >= 0");
        cudaStream_t s = as_stream(stream);
        std::vector<int> hb(nb);
        if (nb) {
            LAPH_REQUIRE(b_list != nullptr, "b_list is null");
            if (is_device_ptr(b_list)) {   // ordered on the caller's stream, then read on the host
                LAPH_CUDA(cudaMemcpyAsync(hb.data(), b_list, sizeof(int) * nb, cudaMemcpyDeviceToHost, s));
                LAPH_CUDA(cudaStreamSynchronize(s));
            } else
                std::copy(b_list, b_list + nb, hb.begin());
        }
        std::vector<uint8_t> m = dilution_masks(*dil, g.nt, nv, hb.data(), nb);
        size_t ebytes = sizeof(c64) * 3 * g.V3 * g.nt * (size_t)nv;
        const c64 *ev = (const c64 *)stage_in(ctx, evecs, ebytes, "evecs", s);
        uint8_t *codes = (uint8_t *)ws_get(ctx, "src:codes", (size_t)g.nt * 4 * nv);
        z4_codes(g.nt, nv, noise_id, config_id, codes, s);
        uint8_t *dm = (uint8_t *)ws_get(ctx, "src:mask", m.size() + 1);
        if (!m.empty()) LAPH_CUDA(cudaMemcpyAsync(dm, m.data(), m.size(), cudaMemcpyHostToDevice, s));
        size_t obytes = sizeof(c64) * 12 * g.V * (size_t)nb;
        StagedOut o = stage_out(ctx, rhs, obytes, "sources");
        if (nb) {
            long n = g.V * 3 * nb;
            sources_kernel<<<grid_for(n, 256), 256, 0, s>>>(g, nv, nb, ev, codes, dm, (c64 *)o.dev);
            LAPH_LAUNCH_CHECK();
        }
        if (noise) {
            StagedOut on = stage_out(ctx, noise, (size_t)g.nt * 4 * nv, "noise");
            LAPH_CUDA(cudaMemcpyAsync(on.dev, codes, (size_t)g.nt * 4 * nv, cudaMemcpyDeviceToDevice, s));
            on.commit(s);
        }
        o.commit(s);
        // keep the host mask alive until the async copy finished
        LAPH_CUDA(cudaStreamSynchronize(s));
    });
}
