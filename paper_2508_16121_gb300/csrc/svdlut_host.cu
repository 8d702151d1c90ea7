// svdlut_apply_host: the fused transform on images that live in host memory.
//
// Page-locked (pinned) host buffers are mapped into the GPU's address space:
// the transform kernel then reads the input and writes the output over the
// CPU-GPU link directly, with no copies and no device buffers (the fastest
// way on a GB300 with NVLink-C2C: ~310 GB/s of combined traffic, against
// ~340 GB/s for copy engines that cannot overlap the transform fully).
//
// Otherwise (pageable memory) each image is cut into row bands.  Band k is uploaded on a library-owned
// copy stream, transformed on the caller's stream once its upload is done,
// and downloaded on a second copy stream once its transform is done, so the
// upload of band k+1, the transform of band k and the download of band k-1
// overlap.  The copy streams fork from the caller's stream at the start and
// join it at the end, so the call is ordered like any other work on that
// stream (and can be captured in a CUDA graph).
#include <algorithm>
#include <mutex>

#include "apply_kernel.cuh"
#include "apply_launch.cuh"

namespace svdlut {

namespace {

constexpr int kMaxBands = 16;     // row bands per image
constexpr int kMinBandRows = 64;  // smallest band
constexpr size_t kWsAlign = 256;

struct HostPipe {
    bool ready = false;
    cudaStream_t up = nullptr, down = nullptr;
    cudaEvent_t fork = nullptr, up_done[kMaxBands] = {}, tx_done[kMaxBands] = {}, down_done = nullptr;
};

std::mutex g_host_mu;
HostPipe g_pipes[64];

svdlut_status pipe_for(int device, HostPipe **out)
{
    if (device < 0 || device >= 64) return fail(SVDLUT_ERR_UNSUPPORTED, "device %d out of range", device);
    HostPipe &p = g_pipes[device];
    if (!p.ready) {
        SVDLUT_CUDA_TRY(cudaStreamCreateWithFlags(&p.up, cudaStreamNonBlocking));
        SVDLUT_CUDA_TRY(cudaStreamCreateWithFlags(&p.down, cudaStreamNonBlocking));
        SVDLUT_CUDA_TRY(cudaEventCreateWithFlags(&p.fork, cudaEventDisableTiming));
        SVDLUT_CUDA_TRY(cudaEventCreateWithFlags(&p.down_done, cudaEventDisableTiming));
        for (int k = 0; k < kMaxBands; ++k) {
            SVDLUT_CUDA_TRY(cudaEventCreateWithFlags(&p.up_done[k], cudaEventDisableTiming));
            SVDLUT_CUDA_TRY(cudaEventCreateWithFlags(&p.tx_done[k], cudaEventDisableTiming));
        }
        p.ready = true;
    }
    *out = &p;
    return SVDLUT_OK;
}

size_t image_bytes(int H, int W, svdlut_dtype dt)
{
    return static_cast<size_t>(3) * H * W * (dt == SVDLUT_F32 ? 4 : 1);
}

size_t round_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

int band_count(int H) { return std::max(1, std::min(kMaxBands, H / kMinBandRows)); }

// Device address of page-locked host memory mapped into the GPU's address
// space, or null (pageable memory or a lookup error, which is cleared).
void *mapped_device_pointer(const void *p)
{
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return at.type == cudaMemoryTypeHost ? at.devicePointer : nullptr;
}

}  // namespace

}  // namespace svdlut

using namespace svdlut;

extern "C" size_t svdlut_apply_host_workspace_size(int B, int H, int W, svdlut_dtype dtype)
{
    if (B < 1 || H < 1 || W < 1 || (dtype != SVDLUT_F32 && dtype != SVDLUT_U8)) return 0;
    return 2 * round_up(static_cast<size_t>(B) * image_bytes(H, W, dtype), kWsAlign);
}

extern "C" svdlut_status svdlut_apply_host(const svdlut_dims *dims, const svdlut_params *params, int B, int H, int W,
                                           svdlut_dtype dtype, const void *x_host, void *y_host, void *ws,
                                           size_t ws_bytes, svdlut_stream_t stream)
{
    SVDLUT_TRACE("svdlut_apply_host");
    clear_error();
    svdlut_status st = check_dims(dims);
    if (st != SVDLUT_OK) return st;
    if ((st = check_params(dims, params)) != SVDLUT_OK) return st;
    if (B < 1 || H < 1 || W < 1) return fail(SVDLUT_ERR_INVALID_ARG, "B=%d H=%d W=%d must be >= 1", B, H, W);
    if (dtype != SVDLUT_F32 && dtype != SVDLUT_U8) return fail(SVDLUT_ERR_INVALID_ARG, "unknown dtype %d", dtype);
    if (!x_host || !y_host) return fail(SVDLUT_ERR_INVALID_ARG, "x_host and y_host are required");
    const size_t img = image_bytes(H, W, dtype), all = static_cast<size_t>(B) * img;
    const char *xs = static_cast<const char *>(x_host);
    char *ys = static_cast<char *>(y_host);
    if (xs < ys + all && ys < xs + all) return fail(SVDLUT_ERR_INVALID_ARG, "x_host and y_host overlap");
    DeviceInfo di;
    if ((st = device_info(&di)) != SVDLUT_OK) return st;
    const cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);

    // mapped (page-locked) host memory: the kernel works on it in place
    void *xm = mapped_device_pointer(x_host), *ym = mapped_device_pointer(y_host);
    if (xm && ym) {
        for (int b0 = 0; b0 < B; b0 += kPlainChunk) {
            LaunchArgs<kPlainChunk> a{};
            a.n = std::min(kPlainChunk, B - b0);
            for (int i = 0; i < a.n; ++i) a.img[i] = make_desc(dims, params, b0 + i, H, W, dtype, xm, ym);
            size_t smem = 0;
            if ((st = plan_uniform(a, di.sm_count, static_cast<size_t>(di.max_smem_optin), &smem)) != SVDLUT_OK)
                return st;
            if ((st = launch_apply(a, smem, dtype, s, 0)) != SVDLUT_OK) return st;
        }
        return SVDLUT_OK;
    }

    if (!ws || ws_bytes < svdlut_apply_host_workspace_size(B, H, W, dtype))
        return fail(SVDLUT_ERR_WORKSPACE, "workspace of %zu bytes needed", svdlut_apply_host_workspace_size(B, H, W, dtype));
    if (!aligned(ws, kWsAlign)) return fail(SVDLUT_ERR_INVALID_ARG, "workspace must be %zu-byte aligned", kWsAlign);
    std::lock_guard<std::mutex> lock(g_host_mu);  // the copy streams and events are per device
    HostPipe *pp = nullptr;
    if ((st = pipe_for(di.device, &pp)) != SVDLUT_OK) return st;
    HostPipe &p = *pp;
    char *xd = static_cast<char *>(ws), *yd = xd + round_up(all, kWsAlign);
    const size_t es = dtype == SVDLUT_F32 ? 4 : 1, row = static_cast<size_t>(W) * es, plane = row * H;
    const int nb = band_count(H);
    {   // the shared-memory plan of the tallest band must exist before any work is queued
        LaunchArgs<kPlainChunk> a{};
        a.n = 1;
        a.img[0] = make_desc(dims, params, 0, H, W, dtype, xd, yd);
        a.img[0].y_end = (H + nb - 1) / nb;
        size_t smem = 0;
        if ((st = plan_uniform(a, di.sm_count, static_cast<size_t>(di.max_smem_optin), &smem)) != SVDLUT_OK)
            return st;
    }

    // fork: the copy streams start after the caller's earlier work
    SVDLUT_CUDA_TRY(cudaEventRecord(p.fork, s));
    SVDLUT_CUDA_TRY(cudaStreamWaitEvent(p.up, p.fork, 0));
    SVDLUT_CUDA_TRY(cudaStreamWaitEvent(p.down, p.fork, 0));
    for (int b = 0; b < B; ++b) {
        for (int k = 0; k < nb; ++k) {
            const int r0 = static_cast<int>(static_cast<long long>(H) * k / nb);
            const int r1 = static_cast<int>(static_cast<long long>(H) * (k + 1) / nb);
            const size_t off = static_cast<size_t>(b) * img + r0 * row, len = (r1 - r0) * row;
            // upload band k (three plane segments)
            for (int c = 0; c < 3; ++c)
                SVDLUT_CUDA_TRY(cudaMemcpyAsync(xd + off + c * plane, xs + off + c * plane, len,
                                                cudaMemcpyHostToDevice, p.up));
            SVDLUT_CUDA_TRY(cudaEventRecord(p.up_done[k], p.up));
            // transform band k on the caller's stream
            SVDLUT_CUDA_TRY(cudaStreamWaitEvent(s, p.up_done[k], 0));
            LaunchArgs<kPlainChunk> a{};
            a.n = 1;
            a.img[0] = make_desc(dims, params, b, H, W, dtype, xd, yd);
            a.img[0].y_begin = r0;
            a.img[0].y_end = r1;
            size_t smem = 0;
            if ((st = plan_uniform(a, di.sm_count, static_cast<size_t>(di.max_smem_optin), &smem)) != SVDLUT_OK)
                return st;
            if ((st = launch_apply(a, smem, dtype, s, 0)) != SVDLUT_OK) return st;
            SVDLUT_CUDA_TRY(cudaEventRecord(p.tx_done[k], s));
            // download band k once transformed
            SVDLUT_CUDA_TRY(cudaStreamWaitEvent(p.down, p.tx_done[k], 0));
            for (int c = 0; c < 3; ++c)
                SVDLUT_CUDA_TRY(cudaMemcpyAsync(ys + off + c * plane, yd + off + c * plane, len, cudaMemcpyDeviceToHost,
                                                p.down));
        }
    }
    // join: the caller's stream continues after the last download
    SVDLUT_CUDA_TRY(cudaEventRecord(p.down_done, p.down));
    SVDLUT_CUDA_TRY(cudaStreamWaitEvent(s, p.down_done, 0));
    return SVDLUT_OK;
}
