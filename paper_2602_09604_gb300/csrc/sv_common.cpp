// Error reporting and small shared helpers.
#include <algorithm>
#include <atomic>
#include <cstdarg>
#include <cstdio>
#include <future>
#include <mutex>
#include <system_error>
#include <thread>

#include "sv_internal.h"

namespace svg {

namespace {
struct DevBuf {
    void *p;
    size_t bytes;
};
std::mutex g_buf_mu;
std::vector<DevBuf> g_buf_cache[64];
constexpr size_t kBufCacheCount = 8;
constexpr size_t kBufCacheBytes = size_t(256) << 20;
}  // namespace

int dev_buffer_get(int device, size_t bytes, void **out, size_t *got_bytes)
{
    *out = nullptr;
    *got_bytes = 0;
    if (device >= 0 && device < 64) {
        std::lock_guard<std::mutex> lk(g_buf_mu);
        std::vector<DevBuf> &c = g_buf_cache[device];
        size_t best = c.size();
        for (size_t i = 0; i < c.size(); ++i)
            if (c[i].bytes >= bytes && c[i].bytes <= 4 * bytes && (best == c.size() || c[i].bytes < c[best].bytes)) best = i;
        if (best < c.size()) {
            *out = c[best].p;
            *got_bytes = c[best].bytes;
            c.erase(c.begin() + (long)best);
            return SV_OK;
        }
    }
    SV_CUDA_TRY(cudaMalloc(out, bytes));
    *got_bytes = bytes;
    return SV_OK;
}

void dev_buffer_put(int device, void *p, size_t bytes)
{
    if (!p) return;
    if (device >= 0 && device < 64) {
        std::lock_guard<std::mutex> lk(g_buf_mu);
        std::vector<DevBuf> &c = g_buf_cache[device];
        size_t held = 0;
        for (const DevBuf &b : c) held += b.bytes;
        if (c.size() < kBufCacheCount && held + bytes <= kBufCacheBytes) {
            c.push_back(DevBuf{p, bytes});
            return;
        }
    }
    int cur = -1;
    cudaGetDevice(&cur);
    if (device >= 0 && cur != device) cudaSetDevice(device);
    cudaFree(p);
    if (device >= 0 && cur >= 0 && cur != device) cudaSetDevice(cur);
}

namespace {
std::mutex g_pin_mu;
unsigned char *g_pin = nullptr;
size_t g_pin_bytes = 0;
}  // namespace

int pinned_staging(size_t bytes, unsigned char **out, std::unique_lock<std::mutex> &lock)
{
    lock = std::unique_lock<std::mutex>(g_pin_mu);
    if (g_pin_bytes < bytes) {
        if (g_pin) cudaFreeHost(g_pin);
        g_pin = nullptr;
        g_pin_bytes = 0;
        const size_t want = std::max(bytes, size_t(4) << 20);
        const cudaError_t e = cudaMallocHost(reinterpret_cast<void **>(&g_pin), want);
        if (e != cudaSuccess) {
            g_pin = nullptr;
            set_error("pinned staging buffer: %s", cudaGetErrorString(e));
            return SV_ECUDA;
        }
        g_pin_bytes = want;
    }
    *out = g_pin;
    return SV_OK;
}

void host_parallel_for(size_t n, size_t threads, const std::function<void(size_t)> &fn)
{
    std::atomic<size_t> next{0};
    auto work = [&]() {
        for (size_t i = next++; i < n; i = next++) fn(i);
    };
    const size_t hw = std::max(1u, std::thread::hardware_concurrency());
    const size_t nt = std::min(std::min(threads, n), hw);
    std::vector<std::future<void>> jobs;
    try {
        for (size_t t = 1; t < nt; ++t) jobs.push_back(std::async(std::launch::async, work));
    } catch (const std::system_error &) {   // no more threads: the ones started and this one finish
    }
    work();
    for (auto &j : jobs) j.get();   // rethrows a worker's exception (e.g. std::bad_alloc)
}

static thread_local char g_err[512] = "";

void set_error(const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    std::vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

void clear_error() { g_err[0] = '\0'; }

int device_sm_count(int device)
{
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return 0;
    return v;
}

}  // namespace svg

extern "C" const char *sv_last_error(void) { return svg::g_err; }

extern "C" const char *sv_version(void) { return "svgb300 0.1 (sm_103a)"; }
