// svdlut_backward_noalloc: the adjoint with its workspace in a fixed,
// library-owned device array, for callers that cannot allocate device memory.
//
// Who needs this: code that must not call cudaMalloc / cudaFree (or any
// allocator that does) on its own -- for example a host application whose
// device memory is owned by another runtime's pool and forbids allocation by
// plugins, a latency-critical loop where an allocation could block on a
// device-wide synchronisation, or code being recorded into a CUDA graph,
// where a plain cudaMalloc is not allowed.  Such callers still pass their own
// inputs and outputs; only the scratch space comes from here.
#include <mutex>

#include "svdlut_internal.cuh"

namespace {

// Upper bound on the scratch space (bytes).  The array lives as long as the
// library is loaded, on every GPU that loads it.
constexpr size_t kNoAllocScratchBytes = size_t(32) << 20;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// Device address of g_noalloc_scratch, looked up once per device (with that
// device current).  In host code the symbol is only a stand-in: the address a
// kernel may use must come from cudaGetSymbolAddress.
svdlut_status scratch_address(void **out)
{
    static std::mutex mu;
    static void *addr[64] = {};
    int dev = 0;
    SVDLUT_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return svdlut::fail(SVDLUT_ERR_UNSUPPORTED, "device index %d", dev);
    std::lock_guard<std::mutex> g(mu);
    if (!addr[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return svdlut::cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
        addr[dev] = p;
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
