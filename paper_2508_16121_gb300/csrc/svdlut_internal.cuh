// Internal helpers shared by the library's translation units (not installed).
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <cstdarg>
#include <cstdint>
#include <utility>
#include <cstdio>

#include "svdlut.h"

namespace svdlut {

// ---- error reporting (thread-local message behind svdlut_last_error) ----
void set_error(const char *fmt, ...);
void clear_error();

inline svdlut_status fail(svdlut_status s, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    set_error("%s", buf);
    return s;
}

inline svdlut_status cuda_fail(cudaError_t e, const char *where)
{
    return fail(SVDLUT_ERR_CUDA, "%s: %s (%s)", where, cudaGetErrorString(e), cudaGetErrorName(e));
}

#define SVDLUT_CUDA_TRY(expr)                                          \
    do {                                                               \
        cudaError_t _e = (expr);                                       \
        if (_e != cudaSuccess) return ::svdlut::cuda_fail(_e, #expr);  \
    } while (0)

// ---- tracing: an NVTX range around each public entry point (a no-op unless
// a profiler such as Nsight Systems is attached) ----
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};
#define SVDLUT_TRACE(name) ::svdlut::NvtxRange svdlut_trace_range_(name)

// ---- size limits of the library ----
constexpr int kMaxDt = 33;
constexpr int kMaxK = 48;
constexpr int kMaxDsc = 64;

// Validate dims against the documented ranges.
svdlut_status check_dims(const svdlut_dims *d);

// Device properties of the current device, cached per device.
struct DeviceInfo {
    int device;
    int sm_count;
    int max_smem_optin;
};
svdlut_status device_info(DeviceInfo *out);

// Device status words of the kernels' index checks for the current device
// (builds with SVDLUT_CHECK_BOUNDS; null otherwise).
svdlut_status check_buffer(unsigned int **out);

inline bool aligned(const void *p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

// Programmatic dependent launch (chains of small kernels).  The kernel waits
// for the preceding kernel's results before it reads anything, then lets the
// next launch in the stream start its launch processing; both are no-ops for
// a kernel launched without the attribute.
__device__ __forceinline__ void pdl_enter()
{
    asm volatile("griddepcontrol.wait;\n" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;\n" :::);
}

// Launches kernel<<<grid, block, smem, s>>>(args...) as a programmatic
// dependent launch: its launch overlaps the end of the preceding kernel in
// the stream (the kernel must call pdl_enter() first).
template <typename... KArgs, typename... Args>
svdlut_status launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                         Args &&...args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    SVDLUT_CUDA_TRY(cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...));
    return SVDLUT_OK;
}

}  // namespace svdlut
