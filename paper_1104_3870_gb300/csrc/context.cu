// Context, workspace, host/device staging and error reporting of liblaph.
#include <cstring>

#include "common.cuh"

namespace laph {

static thread_local std::string g_last_error;

void set_last_error(const std::string &msg) { g_last_error = msg; }

void ctx_activate(laph_ctx *ctx) {
    LAPH_REQUIRE(ctx != nullptr, "context is null");
    LAPH_CUDA(cudaSetDevice(ctx->device));
}

void *ws_get(laph_ctx *ctx, const std::string &name, size_t bytes) {
    if (bytes == 0) bytes = 256;
    Buf &b = ctx->ws[name];
    if (b.bytes < bytes) {
        if (b.ptr) {
            // the buffer may still be in use by queued work on any stream
            LAPH_CUDA(cudaDeviceSynchronize());
            LAPH_CUDA(cudaFree(b.ptr));
            b.ptr = nullptr;
            b.bytes = 0;
        }
        cudaError_t e = cudaMalloc(&b.ptr, bytes);
        if (e != cudaSuccess) {
            (void)cudaGetLastError();
            throw Error(LAPH_ERR_NOMEM, "workspace '" + name + "' of " + std::to_string(bytes) +
                                            " bytes: " + cudaGetErrorString(e));
        }
        b.bytes = bytes;
    }
    return b.ptr;
}

void *pinned_get(laph_ctx *ctx, size_t bytes) {
    if (ctx->pinned_bytes < bytes) {
        if (ctx->pinned) {
            LAPH_CUDA(cudaDeviceSynchronize());
            LAPH_CUDA(cudaFreeHost(ctx->pinned));
        }
        size_t nb = bytes < 65536 ? 65536 : bytes;
        LAPH_CUDA(cudaMallocHost(&ctx->pinned, nb));
        ctx->pinned_bytes = nb;
    }
    return ctx->pinned;
}

bool is_device_ptr(const void *p) {
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

const void *stage_in(laph_ctx *ctx, const void *p, size_t bytes, const std::string &name, cudaStream_t s) {
    LAPH_REQUIRE(p != nullptr || bytes == 0, "input pointer '" + name + "' is null");
    if (bytes == 0 || is_device_ptr(p)) return p;
    void *d = ws_get(ctx, "stage_in:" + name, bytes);
    LAPH_CUDA(cudaMemcpyAsync(d, p, bytes, cudaMemcpyHostToDevice, s));
    return d;
}

StagedOut stage_out(laph_ctx *ctx, void *p, size_t bytes, const std::string &name) {
    LAPH_REQUIRE(p != nullptr || bytes == 0, "output pointer '" + name + "' is null");
    StagedOut o;
    o.user = p;
    o.bytes = bytes;
    if (bytes == 0 || is_device_ptr(p)) {
        o.dev = p;
        o.host = false;
    } else {
        o.dev = ws_get(ctx, "stage_out:" + name, bytes);
        o.host = true;
    }
    return o;
}

void StagedOut::commit(cudaStream_t s) {
    if (host && bytes) {
        LAPH_CUDA(cudaMemcpyAsync(user, dev, bytes, cudaMemcpyDeviceToHost, s));
        LAPH_CUDA(cudaStreamSynchronize(s));
    }
}

}  // namespace laph

using namespace laph;

extern "C" int laph_ctx_create(int device, laph_ctx **out) {
    return guard([&] {
        LAPH_REQUIRE(out != nullptr, "out is null");
        int n = 0;
        LAPH_CUDA(cudaGetDeviceCount(&n));
        LAPH_REQUIRE(device >= 0 && device < n, "device index out of range");
        LAPH_CUDA(cudaSetDevice(device));
        laph_ctx *c = new laph_ctx();
        c->device = device;
        LAPH_CUDA(cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, device));
        *out = c;
    });
}

extern "C" void laph_ctx_destroy(laph_ctx *ctx) {
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    cudaDeviceSynchronize();
    for (auto &kv : ctx->ws)
        if (kv.second.ptr) cudaFree(kv.second.ptr);
    if (ctx->pinned) cudaFreeHost(ctx->pinned);
    delete ctx;
}

extern "C" const char *laph_last_error(void) { return g_last_error.c_str(); }

extern "C" const char *laph_version(void) { return "laph-gb300 0.1 (sm_103a)"; }
