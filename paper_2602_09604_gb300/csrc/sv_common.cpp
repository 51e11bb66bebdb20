// Error reporting and small shared helpers.
#include <cstdarg>
#include <cstdio>

#include "sv_internal.h"

namespace svg {

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
