// pwl_capi.cu -- library-wide pieces of the C ABI: thread-local error
// strings, the device-property cache and descriptor validation.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>

#include <mutex>
#include <vector>

#include "pwl_common.cuh"

namespace pwl {

static thread_local char g_err[512] = "";

void clear_error() { g_err[0] = 0; }

pwl_status fail(pwl_status s, const char* fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return s;
}

pwl_status cuda_fail(cudaError_t e, const char* what)
{
    snprintf(g_err, sizeof(g_err), "%s: %s (%s)", what, cudaGetErrorString(e), cudaGetErrorName(e));
    return (e == cudaErrorMemoryAllocation) ? PWL_ENOMEM : PWL_ECUDA;
}

const DeviceInfo& device_info()
{
    static std::mutex mu;
    static std::vector<DeviceInfo> cache;
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(mu);
    for (auto& d : cache)
        if (d.device == dev) return d;
    DeviceInfo d{};
    d.device = dev;
    int v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    d.sms = v > 0 ? v : 1;
    cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    d.smem_optin = v > 0 ? (size_t)v : 48 * 1024;
    cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    d.smem_per_sm = v > 0 ? (size_t)v : 100 * 1024;
    cudaDeviceGetAttribute(&v, cudaDevAttrMaxThreadsPerMultiProcessor, dev);
    d.max_threads_sm = v > 0 ? v : 2048;
    cache.push_back(d);
    return cache.back();
}

pwl_status validate_func(const pwl_func* f)
{
    if (!f) return fail(PWL_EINVAL, "function descriptor is NULL");
    if (f->kind < PWL_F_GAUSSIAN || f->kind > PWL_F_EXP)
        return fail(PWL_EINVAL, "unknown function kind %d", f->kind);
    if (f->reserved != 0) return fail(PWL_EINVAL, "pwl_func.reserved must be 0");
    if (!isfinite(f->a) || !isfinite(f->b) || !(f->a < f->b))
        return fail(PWL_EINVAL, "interval [a, b] must be finite with a < b (got [%g, %g])", f->a,
                    f->b);
    for (int i = 0; i < 8; ++i)
        if (!isfinite(f->p[i])) return fail(PWL_EINVAL, "parameter p[%d] is not finite", i);
    if ((f->kind == PWL_F_GAUSSIAN || f->kind == PWL_F_LORENTZIAN) && !(f->p[2] != 0.0))
        return fail(PWL_EINVAL, "width parameter p[2] must be non-zero");
    return PWL_OK;
}

}  // namespace pwl

extern "C" {

const char* pwl_last_error(void) { return pwl::g_err; }

int32_t pwl_version(void) { return 1 * 10000 + 0 * 100 + 0; }

}  // extern "C"
