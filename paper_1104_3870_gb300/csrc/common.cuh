// Internal definitions shared by the CUDA translation units of liblaph.
// Complex arithmetic, lattice geometry (lexicographic and even-odd), the
// context with its grow-only device workspace, host/device staging of ABI
// arrays, and error plumbing (C++ exceptions inside, status codes at the ABI).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <map>
#include <stdexcept>
#include <string>
#include <vector>

#include "../../include/laph.h"

namespace laph {

// ----------------------------------------------------------------- errors
struct Error : std::runtime_error {
    int code;
    Error(int c, const std::string &m) : std::runtime_error(m), code(c) {}
};

void set_last_error(const std::string &msg);

#define LAPH_CUDA(call)                                                                    \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess)                                                             \
            throw ::laph::Error(LAPH_ERR_CUDA, std::string(#call " failed: ") +            \
                                                  cudaGetErrorString(e_) + " at " +        \
                                                  __FILE__ + ":" + std::to_string(__LINE__)); \
    } while (0)

// Every kernel launch of the library is followed by this check; it also counts launches.
void count_launch();
#define LAPH_LAUNCH_CHECK()              \
    do {                                 \
        ::laph::count_launch();          \
        LAPH_CUDA(cudaGetLastError());   \
    } while (0)

// Optional per-kernel-family timing with CUDA events on the launching stream
// (enabled by laph_profile_enable); `bytes` is the algorithmic traffic of the launch.
bool prof_on();
void prof_begin(const char *family, cudaStream_t s);
void prof_end(const char *family, cudaStream_t s, double bytes, double flops);

#define LAPH_REQUIRE(cond, msg)                                                            \
    do {                                                                                   \
        if (!(cond)) throw ::laph::Error(LAPH_ERR_ARG, (msg));                             \
    } while (0)

// Runs `body` and converts exceptions into ABI status codes.
template <typename F>
int guard(F &&body) {
    try {
        set_last_error("");
        body();
        return LAPH_OK;
    } catch (const Error &e) {
        set_last_error(e.what());
        return e.code;
    } catch (const std::bad_alloc &) {
        set_last_error("host allocation failed");
        return LAPH_ERR_NOMEM;
    } catch (const std::exception &e) {
        set_last_error(e.what());
        return LAPH_ERR_CUDA;
    }
}

// ----------------------------------------------------------------- complex
template <typename T>
struct alignas(2 * sizeof(T)) cpx {
    T re, im;
};
using c64 = cpx<double>;
using c32 = cpx<float>;

template <typename T>
__host__ __device__ __forceinline__ cpx<T> mk(T r, T i) { return cpx<T>{r, i}; }
template <typename T>
__host__ __device__ __forceinline__ cpx<T> operator+(cpx<T> a, cpx<T> b) { return {a.re + b.re, a.im + b.im}; }
template <typename T>
__host__ __device__ __forceinline__ cpx<T> operator-(cpx<T> a, cpx<T> b) { return {a.re - b.re, a.im - b.im}; }
template <typename T>
__host__ __device__ __forceinline__ cpx<T> operator-(cpx<T> a) { return {-a.re, -a.im}; }
template <typename T>
__host__ __device__ __forceinline__ cpx<T> operator*(cpx<T> a, cpx<T> b) {
    return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
template <typename T>
__host__ __device__ __forceinline__ cpx<T> operator*(T s, cpx<T> a) { return {s * a.re, s * a.im}; }
template <typename T>
__host__ __device__ __forceinline__ cpx<T> &operator+=(cpx<T> &a, cpx<T> b) { a.re += b.re; a.im += b.im; return a; }
template <typename T>
__host__ __device__ __forceinline__ cpx<T> &operator-=(cpx<T> &a, cpx<T> b) { a.re -= b.re; a.im -= b.im; return a; }
template <typename T>
__host__ __device__ __forceinline__ cpx<T> conj(cpx<T> a) { return {a.re, -a.im}; }
// conj(a) * b
template <typename T>
__host__ __device__ __forceinline__ cpx<T> cmul_conj(cpx<T> a, cpx<T> b) {
    return {a.re * b.re + a.im * b.im, a.re * b.im - a.im * b.re};
}
// i * a
template <typename T>
__host__ __device__ __forceinline__ cpx<T> times_i(cpx<T> a) { return {-a.im, a.re}; }
template <typename T>
__host__ __device__ __forceinline__ T norm2(cpx<T> a) { return a.re * a.re + a.im * a.im; }
template <typename To, typename From>
__host__ __device__ __forceinline__ cpx<To> cvt(cpx<From> a) { return {(To)a.re, (To)a.im}; }

// ----------------------------------------------------------------- geometry
// Site s = ((t*ns + z)*ns + y)*ns + x; parity (x+y+z+t)&1; checkerboard index cb = s >> 1.
struct Geom {
    int ns, nt, hs;   // hs = ns / 2
    long V3, V, Vh;   // Vh = V / 2
};

inline Geom make_geom(const laph_lattice *lat) {
    LAPH_REQUIRE(lat != nullptr, "lattice is null");
    LAPH_REQUIRE(lat->ns >= 2 && lat->nt >= 2, "ns and nt must be >= 2");
    LAPH_REQUIRE(lat->ns % 2 == 0 && lat->nt % 2 == 0, "ns and nt must be even");
    Geom g;
    g.ns = lat->ns;
    g.nt = lat->nt;
    g.hs = lat->ns / 2;
    g.V3 = (long)lat->ns * lat->ns * lat->ns;
    g.V = g.V3 * lat->nt;
    g.Vh = g.V / 2;
    return g;
}

__host__ __device__ __forceinline__ void site_coords(const Geom &g, long s, int c[4]) {
    c[0] = (int)(s % g.ns);
    long r = s / g.ns;
    c[1] = (int)(r % g.ns);
    r /= g.ns;
    c[2] = (int)(r % g.ns);
    c[3] = (int)(r / g.ns);
}

__host__ __device__ __forceinline__ long site_of(const Geom &g, const int c[4]) {
    return (((long)c[3] * g.ns + c[2]) * g.ns + c[1]) * g.ns + c[0];
}

// Coordinates of checkerboard site (p, cb).
__host__ __device__ __forceinline__ void cb_coords(const Geom &g, int p, long cb, int c[4]) {
    int xh = (int)(cb % g.hs);
    long r = cb / g.hs;
    c[1] = (int)(r % g.ns);
    r /= g.ns;
    c[2] = (int)(r % g.ns);
    c[3] = (int)(r / g.ns);
    int b0 = (p + c[1] + c[2] + c[3]) & 1;
    c[0] = 2 * xh + b0;
}

__host__ __device__ __forceinline__ int parity_of(const int c[4]) { return (c[0] + c[1] + c[2] + c[3]) & 1; }

// ----------------------------------------------------------------- context
struct Buf {
    void *ptr = nullptr;
    size_t bytes = 0;
};

}  // namespace laph

struct laph_ctx {
    int device = 0;
    std::map<std::string, laph::Buf> ws;
    void *pinned = nullptr;
    size_t pinned_bytes = 0;
    std::map<std::string, int> tune;   // autotune cache: key -> chosen block size
    int sm_count = 0;
};

namespace laph {

// Grow-only named device buffer of the context.
void *ws_get(laph_ctx *ctx, const std::string &name, size_t bytes);
// Pinned host scratch of at least `bytes`.
void *pinned_get(laph_ctx *ctx, size_t bytes);
void ctx_activate(laph_ctx *ctx);

bool is_device_ptr(const void *p);

// Input staging: returns a device pointer holding `bytes` of `p` (copied
// into workspace `name` when `p` is host memory).
const void *stage_in(laph_ctx *ctx, const void *p, size_t bytes, const std::string &name, cudaStream_t s);

// Output staging: device pointer to write into; commit() copies back to host when needed.
struct StagedOut {
    void *user = nullptr;
    void *dev = nullptr;
    size_t bytes = 0;
    bool host = false;
    void commit(cudaStream_t s);
};
StagedOut stage_out(laph_ctx *ctx, void *p, size_t bytes, const std::string &name);

inline cudaStream_t as_stream(void *s) { return reinterpret_cast<cudaStream_t>(s); }

inline unsigned grid_for(long n, int block, long cap = 1L << 30) {
    long g = (n + block - 1) / block;
    if (g < 1) g = 1;
    if (g > cap) g = cap;
    return (unsigned)g;
}

// Dirac matrices (chiral basis) and sigma_{mu nu} blocks in constant memory.
// gamma_mu = [[0, G_mu], [G_mu^dag, 0]] with G_k = -i sigma_k, G_4 = 1.
}  // namespace laph
