// svdlut_backward_noalloc: the adjoint with its workspace in a fixed,
// library-owned device array, for callers that cannot allocate device memory.
//
// Who needs this: code that must not call cudaMalloc / cudaFree (or any
// allocator that does) on its own -- for example a host application whose
// device memory is owned by another runtime's pool and forbids allocation by
// plugins, or a latency-critical loop where an allocation could block on a
// device-wide synchronisation.  Such callers still pass their own inputs and
// outputs; only the scratch space comes from here.
#include <cuda.h>

#include <mutex>

#include "svdlut_internal.cuh"

namespace {

// Upper bound on the scratch space (bytes).  The array lives as long as the
// library is loaded, on every GPU that loads it.
constexpr size_t kNoAllocScratchBytes = size_t(32) << 20;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// Unique id of the CUDA context current on this thread (0 if none), through
// the driver's cuCtxGetCurrent / cuCtxGetId obtained from the runtime (no
// link against the driver library).
svdlut_status current_context_id(unsigned long long *id)
{
    using GetCurrent = CUresult (*)(CUcontext *);
    using GetId = CUresult (*)(CUcontext, unsigned long long *);
    static std::once_flag once;
    static GetCurrent get_current = nullptr;
    static GetId get_id = nullptr;
    std::call_once(once, [] {
        cudaDriverEntryPointQueryResult q1 = cudaDriverEntryPointSymbolNotFound, q2 = q1;
        void *f1 = nullptr, *f2 = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) == cudaSuccess &&
            cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) == cudaSuccess &&
            q1 == cudaDriverEntryPointSuccess && q2 == cudaDriverEntryPointSuccess) {
            get_current = reinterpret_cast<GetCurrent>(f1);
            get_id = reinterpret_cast<GetId>(f2);
        }
    });
    if (!get_current || !get_id)
        return svdlut::fail(SVDLUT_ERR_CUDA, "svdlut_backward_noalloc: cuCtxGetCurrent/cuCtxGetId not available");
    CUcontext ctx = nullptr;
    if (get_current(&ctx) != CUDA_SUCCESS)
        return svdlut::fail(SVDLUT_ERR_CUDA, "svdlut_backward_noalloc: cuCtxGetCurrent failed");
    *id = 0;
    if (ctx && get_id(ctx, id) != CUDA_SUCCESS)
        return svdlut::fail(SVDLUT_ERR_CUDA, "svdlut_backward_noalloc: cuCtxGetId failed");
    return SVDLUT_OK;
}

// Device address of g_noalloc_scratch, looked up once per device (with that
// device current) and context: after a device reset the array is loaded
// again, possibly elsewhere, in a new context, and is looked up again.  In
// host code the symbol is only a stand-in: the address a kernel may use must
// come from cudaGetSymbolAddress.
svdlut_status scratch_address(void **out)
{
    static std::mutex mu;
    static void *addr[64] = {};
    static unsigned long long ctx_of[64] = {};
    int dev = 0;
    SVDLUT_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return svdlut::fail(SVDLUT_ERR_UNSUPPORTED, "device index %d", dev);
    unsigned long long ctx = 0;
    svdlut_status st = current_context_id(&ctx);
    if (st != SVDLUT_OK) return st;
    std::lock_guard<std::mutex> g(mu);
    if (!addr[dev] || ctx == 0 || ctx != ctx_of[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return svdlut::cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
        // the lookup makes the device's primary context current if none was
        if ((st = current_context_id(&ctx)) != SVDLUT_OK) return st;
        addr[dev] = p;
        ctx_of[dev] = ctx;
    }
    *out = addr[dev];
    return SVDLUT_OK;
}

}  // namespace

extern "C" svdlut_status svdlut_backward_noalloc(const svdlut_dims *dims, const svdlut_params *params, int B,
                                                 int H, int W, const float *x, const float *dy, float *dx,
                                                 const svdlut_grads *grads, svdlut_stream_t stream)
{
    SVDLUT_TRACE("svdlut_backward_noalloc");
    svdlut::clear_error();
    const svdlut_grads g0{};
    const svdlut_grads &g = grads ? *grads : g0;
    const bool needs_ws = g.dU || g.dS || g.dV || g.dlut_w ||
                          (dims && dims->K > 0 && (g.dg_xy || g.dg_xc || g.dg_yc || g.dgrid_w));
    void *ws = nullptr;
    size_t ws_bytes = 0;
    if (needs_ws) {
        const size_t need = svdlut_backward_workspace_size(dims, B, H, W);
        if (need == 0)  // bad arguments: let svdlut_backward report them
            return svdlut_backward(dims, params, B, H, W, x, dy, dx, grads, nullptr, 0, stream);
        if (need > kNoAllocScratchBytes)
            return svdlut::fail(SVDLUT_ERR_UNSUPPORTED,
                                "svdlut_backward_noalloc: these sizes need %zu bytes of scratch, more than the "
                                "fixed %zu; call svdlut_backward with your own workspace",
                                need, kNoAllocScratchBytes);
        svdlut_status st = scratch_address(&ws);
        if (st != SVDLUT_OK) return st;
        ws_bytes = kNoAllocScratchBytes;
    }
    // Nothing in the scratch needs to start at zero: every pass writes the
    // parts it later reads.
    return svdlut_backward(dims, params, B, H, W, x, dy, dx, grads, ws, ws_bytes, stream);
}
