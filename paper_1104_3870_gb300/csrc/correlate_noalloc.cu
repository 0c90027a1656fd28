// correlate_noalloc: the correlator contraction of correlate() for callers
// that cannot allocate GPU memory.
//
// Some callers run where cudaMalloc is off limits: code executing inside a
// caller-managed memory pool or arena that must stay the only allocator,
// processes whose device memory is fully reserved up front, or real-time
// loops where an allocation would stall or break a capture.  This entry
// point therefore allocates nothing.  Its scratch (meson-function matrices,
// the diluted noise at t0, the projector masks) lives
// in one file-scope __device__ array of fixed size, which every GPU that loads
// the library holds until the process exits.  The caller passes inputs and
// outputs as device pointers; host pointers are rejected because staging
// them would need an allocation.
//
// Every call runs on the device that holds its arrays: it reads that device
// from the output pointer, requires every input (and a non-default stream) to
// belong to the same device, makes it current for the call and restores the
// caller's current device on return.  With that device current it looks up the
// array's address (cudaGetSymbolAddress) on every call, so the address stays
// right after a device reset.  The first call on a device also loads the
// library's kernels there; make that first call before any stream capture.
// The projector list travels to the device inside a kernel argument (at most
// NA_MAX_NB entries), not through a copy from the caller's host array.  Every
// call shares the array and leaves the last call's contents in it, so calls
// that overlap on the GPU (different streams or threads without ordering) race
// on it.
//
// The contraction kernels are the ones of correlate() (correlate.cu); only the
// origin of the scratch memory differs.
#include <vector>

#include "common.cuh"

namespace laph {

constexpr size_t NOALLOC_SCRATCH_BYTES = 16u << 20;   // 16 MiB per device
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

// Kernels shared with correlate.cu (same definitions, launched through their host stubs).
struct W4 {
    c64 w[4][4];
};
__global__ void rho_at_t0_kernel(int nt, int nv, int nb, int t0, const uint8_t *codes, const uint8_t *mask, c64 *out);
__global__ void meson_fn_kernel(int nv, int nb, int ntA, int ntB, const c64 *__restrict__ A, const c64 *__restrict__ B,
                                W4 W, c64 *__restrict__ M);
__global__ void contract2_kernel(int nt, int nb, int t0, const c64 *Msink, const c64 *Msrc, double scale, c64 *corr);
__global__ void pipi_p_kernel(int nb, const c64 *S12, const c64 *M32, c64 *P);
__global__ void pipi_x_kernel(int nt, int nb, int t0, const c64 *P, const c64 *S34, const c64 *M14, const c64 *cpi12,
                              const c64 *cpi34, c64 *corr);

// Projector masks computed on the device from the dilution scheme (no host table upload):
// mask[i][nt + 4 + nv] for the i-th listed projector.
__device__ __forceinline__ bool na_proj(int type, int J, int N, int b, int i) {
    switch (type) {
        case 0: return true;
        case 1: return i == b;
        case 2: return (J * i) / N == b;
        default: return i % J == b;
    }
}

// The projector list by value (a kernel argument of 2 KB): no host-to-device copy of the
// caller's array is needed.
constexpr int NA_MAX_NB = 512;
struct NaBlist {
    int b[NA_MAX_NB];
};

__global__ void na_mask_kernel(int nt, int nv, int nb, laph_dilution d, int nS, int nL, NaBlist blist,
                               uint8_t *mask) {
    int w = nt + 4 + nv;
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= nb * w) return;
    int i = idx / w, e = idx % w;
    int b = blist.b[i];
    int bL = b % nL, bS = (b / nL) % nS, bT = b / (nL * nS);
    bool v;
    if (e < nt) v = na_proj(d.T.type, d.T.J, nt, bT, e);
    else if (e < nt + 4) v = na_proj(d.S.type, d.S.J, 4, bS, e - nt);
    else v = na_proj(d.L.type, d.L.J, nv, bL, e - nt - 4);
    mask[idx] = v ? 1 : 0;
}

static int na_nproj(int type, int J, int N) {
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

// Chiral-basis Dirac matrices on the host: gamma_mu = [[0, G], [G^dag, 0]], G_k = -i sigma_k, G_4 = 1.
struct NaMat {
    c64 m[4][4];
};
static NaMat na_zero() {
    NaMat r;
    for (auto &row : r.m)
        for (auto &v : row) v = {0, 0};
    return r;
}
static NaMat na_mul(const NaMat &a, const NaMat &b) {
    NaMat r = na_zero();
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j)
            for (int k = 0; k < 4; ++k) r.m[i][j] += a.m[i][k] * b.m[k][j];
    return r;
}
static NaMat na_gamma(int mu) {
    const c64 O{0, 0}, P{1, 0}, M1{-1, 0}, I{0, 1}, Mi{0, -1};
    c64 G[4][2][2] = {{{O, Mi}, {Mi, O}}, {{O, M1}, {P, O}}, {{Mi, O}, {O, I}}, {{P, O}, {O, P}}};
    NaMat r = na_zero();
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) {
            r.m[i][2 + j] = G[mu][i][j];
            r.m[2 + i][j] = conj(G[mu][j][i]);
        }
    return r;
}
static NaMat na_gamma5() { return na_mul(na_mul(na_gamma(0), na_gamma(1)), na_mul(na_gamma(2), na_gamma(3))); }
// W = s * (gamma_5 gamma_4)^dag c
static W4 na_weight(const NaMat &c, double s) {
    NaMat g = na_mul(na_gamma5(), na_gamma(3));
    W4 w;
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) {
            c64 acc{0, 0};
            for (int k = 0; k < 4; ++k) acc += conj(g.m[k][i]) * c.m[k][j];
            w.w[i][j] = s * acc;
        }
    return w;
}

// Device address of the scratch array on the current device.  Looked up on every call (cheap
// once the module is loaded on that device), so no address outlives a device reset.
static unsigned char *scratch_for_current_device() {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        throw Error(LAPH_ERR_CUDA, std::string("cudaGetSymbolAddress of the scratch array failed: ") +
                                       cudaGetErrorString(e));
    }
    return (unsigned char *)p;
}

// Device that owns a device (or managed) allocation; -1 for host memory or an unknown pointer.
static int na_device_of(const void *p) {
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return -1;
    }
    return (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) ? a.device : -1;
}

// Makes `dev` current for the lifetime of the object and restores the previous device after.
struct NaDeviceScope {
    int prev = -1;
    explicit NaDeviceScope(int dev) {
        LAPH_CUDA(cudaGetDevice(&prev));
        if (prev != dev) LAPH_CUDA(cudaSetDevice(dev));
    }
    ~NaDeviceScope() {
        int cur = -1;
        if (cudaGetDevice(&cur) == cudaSuccess && cur != prev) (void)cudaSetDevice(prev);
    }
};

// Bump allocator over the fixed array (256-byte aligned pieces).
struct Carve {
    unsigned char *base;
    size_t used = 0;
    template <typename T>
    T *take(size_t count) {
        size_t bytes = (count * sizeof(T) + 255) & ~size_t(255);
        T *p = (T *)(base + used);
        used += bytes;
        return p;
    }
};

// Scratch of one call: projector masks, the diluted noise of every line at t0, one sink /
// source meson-function pair for a meson channel (the rho components reuse it in turn), and
// for I=2 pi pi two pairs plus the crossed-term matrices.
static size_t na_bytes(int nt, int nv, int nb, int nlines, bool pipi) {
    auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
    size_t s = al((size_t)nb * (nt + 4 + nv));
    s += nlines * al(sizeof(c64) * nb * 4 * nv);
    s += (pipi ? 2 : 1) * (al(sizeof(c64) * nt * nb * nb) + al(sizeof(c64) * nb * nb));
    if (pipi) s += 3 * al(sizeof(c64) * nt * nb * nb) + 2 * al(sizeof(c64) * nb * nb) + 2 * al(sizeof(c64) * nt);
    return s;
}

}  // namespace laph

using namespace laph;

extern "C" int correlate_noalloc(const laph_lattice *lat, const laph_corr_spec *spec, const void *const *coef,
                                 const uint8_t *const *noise, void *corr, void *stream) {
    return guard([&] {
        LAPH_REQUIRE(lat != nullptr && spec != nullptr && coef != nullptr && noise != nullptr && corr != nullptr,
                     "null argument");
        const int nt = lat->nt, nv = spec->nv, nb = spec->nb, t0 = spec->t0;
        LAPH_REQUIRE(nt >= 1 && nv >= 1 && nb >= 1, "bad sizes");
        LAPH_REQUIRE(t0 >= 0 && t0 < nt, "t0 out of range");
        LAPH_REQUIRE(spec->b_list != nullptr, "b_list is null");
        LAPH_REQUIRE(spec->channel >= 0 && spec->channel <= LAPH_CH_PIPI_I2, "unknown channel");
        const bool pipi = spec->channel == LAPH_CH_PIPI_I2;
        const int nlines = pipi ? 4 : 2;
        int nT = na_nproj(spec->dil.T.type, spec->dil.T.J, nt);
        int nS = na_nproj(spec->dil.S.type, spec->dil.S.J, 4);
        int nL = na_nproj(spec->dil.L.type, spec->dil.L.J, nv);
        for (int i = 0; i < nb; ++i)
            LAPH_REQUIRE(spec->b_list[i] >= 0 && spec->b_list[i] < nT * nS * nL, "projector index out of range");
        size_t need = na_bytes(nt, nv, nb, nlines, pipi);
        if (need > NOALLOC_SCRATCH_BYTES)
            throw Error(LAPH_ERR_ARG, "correlate_noalloc: this problem needs " + std::to_string(need) +
                                          " bytes of scratch, above the fixed " +
                                          std::to_string(NOALLOC_SCRATCH_BYTES) +
                                          "-byte array; use correlate() or fewer projectors");
        LAPH_REQUIRE(nb <= NA_MAX_NB, "correlate_noalloc takes at most " + std::to_string(NA_MAX_NB) +
                                          " projectors per line");
        // every array on one device, which runs the call
        const int dev = na_device_of(corr);
        LAPH_REQUIRE(dev >= 0, "correlate_noalloc takes a device output pointer");
        for (int k = 0; k < nlines; ++k) {
            LAPH_REQUIRE(coef[k] && noise[k], "null line array");
            const int dc = na_device_of(coef[k]), dn = na_device_of(noise[k]);
            LAPH_REQUIRE(dc >= 0 && dn >= 0,
                         "correlate_noalloc takes device pointers only (host arrays would need staging)");
            LAPH_REQUIRE(dc == dev && dn == dev, "correlate_noalloc: the line arrays and the output must be on one "
                                                 "device");
        }
        cudaStream_t s = as_stream(stream);
        // the legacy (0), legacy-handle (1) and per-thread (2) default streams follow the current device
        if (reinterpret_cast<uintptr_t>(s) > 2) {
            int sdev = -1;
            LAPH_CUDA(cudaStreamGetDevice(s, &sdev));
            LAPH_REQUIRE(sdev == dev, "correlate_noalloc: the stream belongs to another device than the arrays");
        }
        NaDeviceScope scope(dev);
        NaBlist bl;
        for (int i = 0; i < nb; ++i) bl.b[i] = spec->b_list[i];
        Carve cv{scratch_for_current_device()};
        uint8_t *mask = cv.take<uint8_t>((size_t)nb * (nt + 4 + nv));
        na_mask_kernel<<<grid_for((long)nb * (nt + 4 + nv), 256), 256, 0, s>>>(nt, nv, nb, spec->dil, nS, nL, bl,
                                                                              mask);
        LAPH_LAUNCH_CHECK();
        std::vector<c64 *> rho(nlines);
        for (int k = 0; k < nlines; ++k) {
            rho[k] = cv.take<c64>((size_t)nb * 4 * nv);
            rho_at_t0_kernel<<<grid_for((long)nb * 4 * nv, 256), 256, 0, s>>>(nt, nv, nb, t0, noise[k], mask, rho[k]);
            LAPH_LAUNCH_CHECK();
        }
        c64 *out = (c64 *)corr;
        LAPH_CUDA(cudaMemsetAsync(out, 0, sizeof(c64) * nt, s));
        auto meson = [&](const c64 *A, const c64 *B, const c64 *ra, const c64 *rb, const NaMat &c, double scale,
                         c64 *dst) {
            c64 *Msink = cv.take<c64>((size_t)nt * nb * nb);
            c64 *Msrc = cv.take<c64>((size_t)nb * nb);
            int threads = nb < 128 ? 128 : 256;
            meson_fn_kernel<<<dim3(nt, nb), threads, sizeof(c64) * 4 * nv, s>>>(nv, nb, nt, nt, A, B, na_weight(c, 1.0),
                                                                               Msink);
            LAPH_LAUNCH_CHECK();
            meson_fn_kernel<<<dim3(1, nb), threads, sizeof(c64) * 4 * nv, s>>>(nv, nb, 1, 1, ra, rb, na_weight(c, -1.0),
                                                                              Msrc);
            LAPH_LAUNCH_CHECK();
            contract2_kernel<<<nt, 256, 0, s>>>(nt, nb, t0, Msink, Msrc, scale, dst);
            LAPH_LAUNCH_CHECK();
        };
        const c64 *cf[4];
        for (int k = 0; k < nlines; ++k) cf[k] = (const c64 *)coef[k];
        NaMat g4 = na_gamma(3);
        if (spec->channel == LAPH_CH_PION) {
            meson(cf[0], cf[1], rho[0], rho[1], na_mul(g4, na_gamma5()), 1.0, out);
        } else if (spec->channel == LAPH_CH_SCALAR) {
            meson(cf[0], cf[1], rho[0], rho[1], g4, 1.0, out);
        } else if (spec->channel == LAPH_CH_RHO) {
            // the three spatial components share the two scratch matrices in turn (stream order)
            size_t mark = cv.used;
            for (int k = 0; k < 3; ++k) {
                cv.used = mark;
                meson(cf[0], cf[1], rho[0], rho[1], na_mul(g4, na_gamma(k)), 1.0 / 3.0, out);
            }
        } else {
            NaMat cpi = na_mul(g4, na_gamma5());
            c64 *c12 = cv.take<c64>(nt);
            c64 *c34 = cv.take<c64>(nt);
            LAPH_CUDA(cudaMemsetAsync(c12, 0, sizeof(c64) * nt, s));
            LAPH_CUDA(cudaMemsetAsync(c34, 0, sizeof(c64) * nt, s));
            meson(cf[0], cf[1], rho[0], rho[1], cpi, 1.0, c12);
            meson(cf[2], cf[3], rho[2], rho[3], cpi, 1.0, c34);
            c64 *M14 = cv.take<c64>((size_t)nt * nb * nb);
            c64 *M32 = cv.take<c64>((size_t)nt * nb * nb);
            c64 *P = cv.take<c64>((size_t)nt * nb * nb);
            c64 *S12 = cv.take<c64>((size_t)nb * nb);
            c64 *S34 = cv.take<c64>((size_t)nb * nb);
            int threads = nb < 128 ? 128 : 256;
            size_t shm = sizeof(c64) * 4 * nv;
            meson_fn_kernel<<<dim3(nt, nb), threads, shm, s>>>(nv, nb, nt, nt, cf[0], cf[3], na_weight(cpi, 1.0), M14);
            LAPH_LAUNCH_CHECK();
            meson_fn_kernel<<<dim3(nt, nb), threads, shm, s>>>(nv, nb, nt, nt, cf[2], cf[1], na_weight(cpi, 1.0), M32);
            LAPH_LAUNCH_CHECK();
            meson_fn_kernel<<<dim3(1, nb), threads, shm, s>>>(nv, nb, 1, 1, rho[0], rho[1], na_weight(cpi, -1.0), S12);
            LAPH_LAUNCH_CHECK();
            meson_fn_kernel<<<dim3(1, nb), threads, shm, s>>>(nv, nb, 1, 1, rho[2], rho[3], na_weight(cpi, -1.0), S34);
            LAPH_LAUNCH_CHECK();
            pipi_p_kernel<<<nt, 256, 0, s>>>(nb, S12, M32, P);
            LAPH_LAUNCH_CHECK();
            pipi_x_kernel<<<nt, 256, 0, s>>>(nt, nb, t0, P, S34, M14, c12, c34, out);
            LAPH_LAUNCH_CHECK();
        }
        LAPH_REQUIRE(cv.used <= NOALLOC_SCRATCH_BYTES, "scratch accounting error");
    });
}
