// Error reporting and small shared helpers.
#include <atomic>
#include <cstdarg>
#include <cstdio>
#include <future>
#include <system_error>
#include <thread>

#include "sv_internal.h"

namespace svg {

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
