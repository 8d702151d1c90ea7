// Error strings, argument validation and device queries for the C ABI.
#include <mutex>

#include "svdlut_internal.cuh"

namespace svdlut {

static thread_local char g_err[512] = "";

void set_error(const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
}

void clear_error() { g_err[0] = '\0'; }

svdlut_status check_dims(const svdlut_dims *d)
{
    if (!d) return fail(SVDLUT_ERR_INVALID_ARG, "dims is NULL");
    if (d->D_t < 2) return fail(SVDLUT_ERR_INVALID_ARG, "D_t=%d must be >= 2", d->D_t);
    if (d->rank < 1 || d->rank > d->D_t)
        return fail(SVDLUT_ERR_INVALID_ARG, "rank=%d must be in [1, D_t=%d]", d->rank, d->D_t);
    if (d->K < 0) return fail(SVDLUT_ERR_INVALID_ARG, "K=%d must be >= 0", d->K);
    if (d->Dsx < 2 || d->Dsy < 2 || d->Dsc < 2)
        return fail(SVDLUT_ERR_INVALID_ARG, "grid sizes Dsx=%d Dsy=%d Dsc=%d must be >= 2", d->Dsx,
                    d->Dsy, d->Dsc);
    if (d->D_t > kMaxDt) return fail(SVDLUT_ERR_UNSUPPORTED, "D_t=%d > %d", d->D_t, kMaxDt);
    if (d->K > kMaxK) return fail(SVDLUT_ERR_UNSUPPORTED, "K=%d > %d", d->K, kMaxK);
    if (d->Dsc > kMaxDsc) return fail(SVDLUT_ERR_UNSUPPORTED, "Dsc=%d > %d", d->Dsc, kMaxDsc);
    return SVDLUT_OK;
}

svdlut_status device_info(DeviceInfo *out)
{
    static std::mutex mu;
    static DeviceInfo cache[64];
    static bool have[64] = {};
    int dev = 0;
    SVDLUT_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return fail(SVDLUT_ERR_UNSUPPORTED, "device index %d", dev);
    std::lock_guard<std::mutex> g(mu);
    if (!have[dev]) {
        DeviceInfo d;
        d.device = dev;
        SVDLUT_CUDA_TRY(cudaDeviceGetAttribute(&d.sm_count, cudaDevAttrMultiProcessorCount, dev));
        SVDLUT_CUDA_TRY(
            cudaDeviceGetAttribute(&d.max_smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
        cache[dev] = d;
        have[dev] = true;
    }
    *out = cache[dev];
    return SVDLUT_OK;
}

#ifdef SVDLUT_CHECK_BOUNDS
// [0] failures, [1] site, [2] index, [3] limit of the first failure
static __device__ unsigned int g_check_words[4];
#endif

svdlut_status check_buffer(unsigned int **out)
{
#ifdef SVDLUT_CHECK_BOUNDS
    static std::mutex mu;
    static unsigned int *addr[64] = {};
    int dev = 0;
    SVDLUT_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return fail(SVDLUT_ERR_UNSUPPORTED, "device index %d", dev);
    std::lock_guard<std::mutex> g(mu);
    if (!addr[dev]) {
        void *p = nullptr;
        SVDLUT_CUDA_TRY(cudaGetSymbolAddress(&p, g_check_words));
        addr[dev] = static_cast<unsigned int *>(p);
    }
    *out = addr[dev];
#else
    *out = nullptr;
#endif
    return SVDLUT_OK;
}

}  // namespace svdlut

extern "C" svdlut_status svdlut_check_report(uint32_t out[4])
{
    svdlut::clear_error();
    if (!out) return svdlut::fail(SVDLUT_ERR_INVALID_ARG, "out is NULL");
#ifdef SVDLUT_CHECK_BOUNDS
    unsigned int h[4] = {0, 0, 0, 0};
    SVDLUT_CUDA_TRY(cudaDeviceSynchronize());
    SVDLUT_CUDA_TRY(cudaMemcpyFromSymbol(h, svdlut::g_check_words, sizeof h));
    const unsigned int zero[4] = {0, 0, 0, 0};
    SVDLUT_CUDA_TRY(cudaMemcpyToSymbol(svdlut::g_check_words, zero, sizeof zero));
    for (int i = 0; i < 4; ++i) out[i] = h[i];
    return SVDLUT_OK;
#else
    for (int i = 0; i < 4; ++i) out[i] = 0;
    return svdlut::fail(SVDLUT_ERR_UNSUPPORTED, "library built without SVDLUT_CHECK_BOUNDS");
#endif
}

extern "C" const char *svdlut_last_error(void) { return svdlut::g_err; }

extern "C" const char *svdlut_version(void) { return "svdlut 0.1.0 sm_103a"; }
