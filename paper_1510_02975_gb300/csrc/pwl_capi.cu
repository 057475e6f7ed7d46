// pwl_capi.cu -- library-wide pieces of the C ABI: thread-local error
// strings, the device-property cache and descriptor validation.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <atomic>
#include <deque>
#include <map>
#include <mutex>
#include <tuple>
#include <utility>
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

// Failure injection for the allocation paths: < 0 disables; n >= 0 lets
// the next n device allocations through and fails every one after them.
static std::atomic<int64_t> g_alloc_budget{-1};

static bool alloc_allowed()
{
    int64_t b = g_alloc_budget.load();
    while (b >= 0) {
        if (b == 0) return false;
        if (g_alloc_budget.compare_exchange_weak(b, b - 1)) return true;
    }
    return true;
}

cudaError_t dev_malloc(void** p, size_t bytes)
{
    if (!alloc_allowed()) return cudaErrorMemoryAllocation;
    return cudaMalloc(p, bytes);
}

cudaError_t dev_malloc_array(cudaArray_t* a, const cudaChannelFormatDesc* d, size_t width)
{
    if (!alloc_allowed()) return cudaErrorMemoryAllocation;
    return cudaMallocArray(a, d, width, 0);
}

const DeviceInfo& device_info()
{
    static std::mutex mu;
    static std::deque<DeviceInfo> cache;  // references stay valid as devices are added
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

// The dynamic shared-memory limit is a per-function maximum: it is raised
// when a launch needs more and never lowered, so a cached grid stays valid.
// Both it and the occupancy query are host calls that cost more than a small
// launch, hence the caches (per device and kernel).
namespace {
std::mutex g_launch_mu;
std::map<std::pair<int, const void*>, size_t> g_smem_limit;
std::map<std::tuple<int, const void*, int, size_t>, int> g_grid;

cudaError_t ensure_smem_limit_locked(int dev, const void* fn, size_t smem)
{
    size_t& lim = g_smem_limit[std::make_pair(dev, fn)];
    if (lim >= smem && lim != 0) return cudaSuccess;
    const cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) lim = std::max(lim, smem);
    return e;
}
}  // namespace

cudaError_t ensure_smem_limit(const void* fn, size_t smem)
{
    const int dev = device_info().device;
    std::lock_guard<std::mutex> lk(g_launch_mu);
    return ensure_smem_limit_locked(dev, fn, smem);
}

cudaError_t occupancy_grid_fn(const void* fn, int threads, size_t smem, int* grid)
{
    const DeviceInfo& di = device_info();
    std::lock_guard<std::mutex> lk(g_launch_mu);
    cudaError_t e = ensure_smem_limit_locked(di.device, fn, smem);
    if (e != cudaSuccess) return e;
    const auto key = std::make_tuple(di.device, fn, threads, smem);
    const auto it = g_grid.find(key);
    if (it != g_grid.end()) {
        *grid = it->second;
        return cudaSuccess;
    }
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, threads, smem);
    if (e != cudaSuccess) return e;
    *grid = std::max(occ, 1) * di.sms;
    g_grid[key] = *grid;
    return cudaSuccess;
}

pwl_status validate_func(const pwl_func* f)
{
    if (!f) return fail(PWL_EINVAL, "function descriptor is NULL");
    if (f->kind < PWL_F_GAUSSIAN || f->kind > PWL_F_SAMPLED)
        return fail(PWL_EINVAL, "unknown function kind %d", f->kind);
    if (f->reserved != 0) return fail(PWL_EINVAL, "pwl_func.reserved must be 0");
    if (!isfinite(f->a) || !isfinite(f->b) || !(f->a < f->b))
        return fail(PWL_EINVAL, "interval [a, b] must be finite with a < b (got [%g, %g])", f->a,
                    f->b);
    if (f->kind == PWL_F_SAMPLED) {
        const double S = f->p[0];
        if (!(S >= 4.0) || !(S <= 9007199254740992.0) || S != floor(S))
            return fail(PWL_EINVAL, "a sampled function needs an integer sample count >= 4 in p[0]");
        const uint64_t addr = sampled_address(*f);
        if (addr == 0 || (addr & 7u) != 0)
            return fail(PWL_EINVAL, "a sampled function needs an 8-byte aligned sample address in p[1]");
        const double h = (f->b - f->a) / (S - 1.0);
        if (f->p[2] != h || f->p[3] != 1.0 / h || f->p[4] != 1.0 / (h * h))
            return fail(PWL_EINVAL, "a sampled function needs p[2..4] = h, 1/h, 1/h^2 (pwl_func_sampled)");
        return PWL_OK;
    }
    for (int i = 0; i < 8; ++i)
        if (!isfinite(f->p[i])) return fail(PWL_EINVAL, "parameter p[%d] is not finite", i);
    if ((f->kind == PWL_F_GAUSSIAN || f->kind == PWL_F_LORENTZIAN) && !(f->p[2] != 0.0))
        return fail(PWL_EINVAL, "width parameter p[2] must be non-zero");
    return PWL_OK;
}

}  // namespace pwl

using namespace pwl;

extern "C" {

pwl_status pwl_func_sampled(double a, double b, const double* d_samples, int64_t n_samples, pwl_func* out)
{
    clear_error();
    if (!out) return fail(PWL_EINVAL, "out is NULL");
    if (!d_samples) return fail(PWL_EINVAL, "d_samples is NULL");
    if (n_samples < 4) return fail(PWL_EINVAL, "need at least 4 samples (got %lld)", (long long)n_samples);
    if (!isfinite(a) || !isfinite(b) || !(a < b)) return fail(PWL_EINVAL, "need finite a < b");
    pwl_func f;
    memset(&f, 0, sizeof(f));
    f.kind = PWL_F_SAMPLED;
    f.a = a;
    f.b = b;
    f.p[0] = (double)n_samples;
    const uint64_t addr = (uint64_t)(uintptr_t)d_samples;
    memcpy(&f.p[1], &addr, sizeof(addr));
    const double h = (b - a) / ((double)n_samples - 1.0);
    f.p[2] = h;
    f.p[3] = 1.0 / h;
    f.p[4] = 1.0 / (h * h);
    *out = f;
    return validate_func(out);
}

const char* pwl_last_error(void) { return pwl::g_err; }

pwl_status pwl_test_fail_allocations(int64_t succeed_first)
{
    clear_error();
    g_alloc_budget.store(succeed_first < 0 ? -1 : succeed_first);
    return PWL_OK;
}

int32_t pwl_version(void) { return 1 * 10000 + 0 * 100 + 0; }

}  // extern "C"
