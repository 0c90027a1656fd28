// Context, workspace, host/device staging, error reporting, launch counting and
// optional kernel timing of liblaph.
#include <atomic>
#include <cstring>
#include <mutex>

#include "common.cuh"

namespace laph {

static thread_local std::string g_last_error;

void set_last_error(const std::string &msg) { g_last_error = msg; }

static std::atomic<long> g_launches{0};
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

struct ProfEntry {
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> pending;
    long launches = 0;
    double ms = 0.0, bytes = 0.0, flops = 0.0;
};
static std::mutex g_prof_mu;
static int g_prof = 0;   // 0 off, 1 stencil families only, 2 every instrumented family
static std::map<std::string, ProfEntry> g_prof_tab;
static std::vector<cudaEvent_t> g_event_pool;
static thread_local cudaEvent_t g_open_start = nullptr;

static cudaEvent_t take_event() {
    if (!g_event_pool.empty()) {
        cudaEvent_t e = g_event_pool.back();
        g_event_pool.pop_back();
        return e;
    }
    cudaEvent_t e;
    LAPH_CUDA(cudaEventCreate(&e));
    return e;
}

bool prof_on() { return g_prof != 0; }

void prof_begin(const char *family, cudaStream_t s) {
    if (!g_prof) return;
    if (g_prof == 1 && std::strncmp(family, "dslash", 6) != 0) return;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    g_open_start = take_event();
    LAPH_CUDA(cudaEventRecord(g_open_start, s));
}

static void drain(ProfEntry &e) {
    for (auto &p : e.pending) {
        LAPH_CUDA(cudaEventSynchronize(p.second));
        float ms = 0.f;
        LAPH_CUDA(cudaEventElapsedTime(&ms, p.first, p.second));
        e.ms += ms;
        g_event_pool.push_back(p.first);
        g_event_pool.push_back(p.second);
    }
    e.pending.clear();
}

void prof_end(const char *family, cudaStream_t s, double bytes, double flops) {
    if (!g_prof || !g_open_start) return;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    cudaEvent_t stop = take_event();
    LAPH_CUDA(cudaEventRecord(stop, s));
    ProfEntry &e = g_prof_tab[family];
    e.pending.emplace_back(g_open_start, stop);
    g_open_start = nullptr;
    e.launches += 1;
    e.bytes += bytes;
    e.flops += flops;
    if (e.pending.size() > 4096) drain(e);
}

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

extern "C" long laph_launch_count(void) { return g_launches.load(); }

extern "C" void laph_profile_enable(int level) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    g_prof = level < 0 ? 0 : (level > 2 ? 2 : level);
}

extern "C" void laph_profile_reset(void) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    for (auto &kv : g_prof_tab) {
        try {
            drain(kv.second);
        } catch (...) {
        }
    }
    g_prof_tab.clear();
}

extern "C" int laph_profile_families(char *buf, int len) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    std::string all;
    for (auto &kv : g_prof_tab) all += kv.first + ",";
    if (buf && len > 0) {
        std::strncpy(buf, all.c_str(), (size_t)len - 1);
        buf[len - 1] = 0;
    }
    return (int)all.size();
}

extern "C" int laph_profile_read(const char *family, long *launches, double *ms, double *bytes, double *flops) {
    return guard([&] {
        std::lock_guard<std::mutex> lk(g_prof_mu);
        auto it = g_prof_tab.find(family ? family : "");
        if (it == g_prof_tab.end()) {
            *launches = 0;
            *ms = *bytes = *flops = 0.0;
            return;
        }
        drain(it->second);
        *launches = it->second.launches;
        *ms = it->second.ms;
        *bytes = it->second.bytes;
        *flops = it->second.flops;
    });
}
