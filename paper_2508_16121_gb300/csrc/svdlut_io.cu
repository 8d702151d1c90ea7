// svdlut_apply_io: the fused transform between pixel formats.  Interleaved
// 8-bit frames are decoded, and 8-bit outputs encoded, inside apply_kernel.
// 16-bit inputs (the tone-mapping and PPR10K photos, Sec. 4.1) are decoded by
// u16_decode_kernel into a stream-ordered FP32 buffer of up to kPlainChunk
// images, which the FP32-input transform then reads: code v becomes
// float(v) * float(1 / 65535), so the result is bitwise that of the FP32 path
// on those values.  Only the pairs listed in svdlut.h are instantiated.
#include <algorithm>
#include <cstdint>

#include "apply_kernel.cuh"
#include "apply_launch.cuh"

namespace svdlut {
namespace {

struct FmtInfo {
    size_t px_bytes;  // one pixel, three channels
    size_t align;     // element alignment required
};

bool fmt_info(svdlut_pixfmt f, FmtInfo *o)
{
    switch (f) {
    case SVDLUT_PIX_F32: *o = {12, 4}; return true;
    case SVDLUT_PIX_U8: *o = {3, 1}; return true;
    case SVDLUT_PIX_U16: *o = {6, 2}; return true;
    case SVDLUT_PIX_U8_HWC: *o = {3, 1}; return true;
    case SVDLUT_PIX_U16_HWC: *o = {6, 2}; return true;
    default: return false;
    }
}

// n images of H x W 16-bit codes (planar [n][3][H][W], or interleaved
// [n][H][W][3] when hwc) to planar FP32 [n][3][H][W]: float(v) * (1 / 65535).
// quad: H W % 4 == 0 and x 8-byte aligned: a thread takes 4 consecutive codes
// of a plane (one 8-byte load) or 4 pixels of an interleaved row (three),
// and writes one float4 per plane; otherwise one code per thread.
__device__ __forceinline__ float u16_code(unsigned int w, int h, float k)
{
    return static_cast<float>(h ? w >> 16 : w & 0xFFFFu) * k;
}

__global__ void u16_decode_kernel(const uint16_t *__restrict__ x, bool hwc, bool quad, int n, size_t plane,
                                  float *__restrict__ out)
{
    const float k = 1.0f / 65535.0f;
    const size_t stride = static_cast<size_t>(gridDim.x) * blockDim.x;
    const size_t first = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x;
    if (quad && !hwc) {
        const size_t quads = static_cast<size_t>(n) * 3 * plane / 4;
        const uint2 *xq = reinterpret_cast<const uint2 *>(x);
        float4 *oq = reinterpret_cast<float4 *>(out);
        for (size_t q = first; q < quads; q += stride) {
            const uint2 w = __ldg(xq + q);
            oq[q] = make_float4(u16_code(w.x, 0, k), u16_code(w.x, 1, k), u16_code(w.y, 0, k), u16_code(w.y, 1, k));
        }
    } else if (quad) {
        const size_t quads = static_cast<size_t>(n) * plane / 4;  // pixel quads
        for (size_t q = first; q < quads; q += stride) {
            const size_t px = 4 * q, b = px / plane, p = px - b * plane;
            // r0 g0 | b0 r1 | g1 b1 | r2 g2 | b2 r3 | g3 b3
            const uint2 *src = reinterpret_cast<const uint2 *>(x + 3 * px);
            const uint2 w0 = __ldg(src), w1 = __ldg(src + 1), w2 = __ldg(src + 2);
            float *o = out + b * 3 * plane + p;
            *reinterpret_cast<float4 *>(o) =
                make_float4(u16_code(w0.x, 0, k), u16_code(w0.y, 1, k), u16_code(w1.y, 0, k), u16_code(w2.x, 1, k));
            *reinterpret_cast<float4 *>(o + plane) =
                make_float4(u16_code(w0.x, 1, k), u16_code(w1.x, 0, k), u16_code(w1.y, 1, k), u16_code(w2.y, 0, k));
            *reinterpret_cast<float4 *>(o + 2 * plane) =
                make_float4(u16_code(w0.y, 0, k), u16_code(w1.x, 1, k), u16_code(w2.x, 0, k), u16_code(w2.y, 1, k));
        }
    } else {
        const size_t total = static_cast<size_t>(n) * 3 * plane;
        for (size_t e = first; e < total; e += stride) {
            size_t src = e;
            if (hwc) {  // e = (b * 3 + c) * plane + p  <-  (b * plane + p) * 3 + c
                const size_t bc = e / plane, p = e - bc * plane, b = bc / 3, c = bc - b * 3;
                src = (b * plane + p) * 3 + c;
            }
            out[e] = static_cast<float>(__ldg(x + src)) * k;
        }
    }
}

template <class IO>
svdlut_status run_io(const svdlut_dims *dims, const svdlut_params *params, int B, int H, int W, const void *x,
                     const FmtInfo &fi, void *y, const FmtInfo &fo, cudaStream_t s)
{
    DeviceInfo di;
    svdlut_status st = device_info(&di);
    if (st != SVDLUT_OK) return st;
    for (int b0 = 0; b0 < B; b0 += kPlainChunk) {
        LaunchArgs<kPlainChunk> a{};
        a.n = std::min(kPlainChunk, B - b0);
        for (int i = 0; i < a.n; ++i)
            a.img[i] = make_desc_io(dims, params, b0 + i, H, W, x, fi.px_bytes, IO::In::kVecAlign, y, fo.px_bytes,
                                    IO::Out::kVecAlign);
        size_t smem = 0;
        if ((st = plan_uniform(a, di.sm_count, static_cast<size_t>(di.max_smem_optin), &smem)) != SVDLUT_OK)
            return st;
        if (a.total_blocks <= 0) continue;
        if ((st = launch_apply_t<IO, kPlainChunk, false>(a, smem, di.sm_count, di.max_smem_optin, di.device, s, 0)) !=
            SVDLUT_OK)
            return st;
    }
    return SVDLUT_OK;
}

// The parameters of images b, b + 1, ... as those of a batch starting at b.
svdlut_params params_from(const svdlut_dims *d, const svdlut_params *p, int b)
{
    svdlut_params q = *p;
    q.U = p->U + b * param_stride(d, 0);
    q.S = p->S + b * param_stride(d, 1);
    q.V = p->V + b * param_stride(d, 2);
    q.lut_w = p->lut_w + b * param_stride(d, 3);
    q.g_xy = p->g_xy ? p->g_xy + b * param_stride(d, 4) : nullptr;
    q.g_xc = p->g_xc ? p->g_xc + b * param_stride(d, 5) : nullptr;
    q.g_yc = p->g_yc ? p->g_yc + b * param_stride(d, 6) : nullptr;
    q.grid_w = p->grid_w ? p->grid_w + b * param_stride(d, 7) : nullptr;
    return q;
}

// 16-bit input: per chunk of up to kPlainChunk images, decode into `tmp`, then
// the FP32-input transform of those images writes their outputs (format
// out_fmt) in place in y.
svdlut_status run_u16(const svdlut_dims *dims, const svdlut_params *params, int B, int H, int W, const void *x,
                      bool hwc, svdlut_pixfmt out_fmt, void *y, const FmtInfo &fo, cudaStream_t s)
{
    const size_t plane = static_cast<size_t>(H) * W;
    const int chunk = std::min(B, kPlainChunk);
    float *tmp = nullptr;
    SVDLUT_CUDA_TRY(cudaMallocAsync(reinterpret_cast<void **>(&tmp), sizeof(float) * chunk * 3 * plane, s));
    const FmtInfo ff{12, 4};
    svdlut_status st = SVDLUT_OK;
    for (int b0 = 0; b0 < B && st == SVDLUT_OK; b0 += chunk) {
        const int n = std::min(chunk, B - b0);
        const uint16_t *xb = static_cast<const uint16_t *>(x) + static_cast<size_t>(b0) * 3 * plane;
        const bool quad = plane % 4 == 0 && aligned(xb, 8);
        const size_t work = static_cast<size_t>(n) * 3 * plane / (quad ? (hwc ? 12 : 4) : 1);
        const int blocks = static_cast<int>(std::min<size_t>((work + 255) / 256, 152 * 32));
        u16_decode_kernel<<<blocks, 256, 0, s>>>(xb, hwc, quad, n, plane, tmp);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) {
            st = fail(SVDLUT_ERR_CUDA, "u16_decode_kernel: %s", cudaGetErrorString(e));
            break;
        }
        // the chunk as a batch of its own: images b0.. of y and of the parameters
        char *yb = static_cast<char *>(y) + static_cast<size_t>(b0) * plane * fo.px_bytes;
        const svdlut_params pb = params_from(dims, params, b0);
        if (out_fmt == SVDLUT_PIX_F32)
            st = run_io<IoF32>(dims, &pb, n, H, W, tmp, ff, yb, fo, s);
        else if (out_fmt == SVDLUT_PIX_U8)
            st = run_io<Io<InF32, OutU8>>(dims, &pb, n, H, W, tmp, ff, yb, fo, s);
        else
            st = run_io<Io<InF32, OutU8Hwc>>(dims, &pb, n, H, W, tmp, ff, yb, fo, s);
    }
    const cudaError_t e = cudaFreeAsync(tmp, s);
    if (st == SVDLUT_OK && e != cudaSuccess) st = fail(SVDLUT_ERR_CUDA, "cudaFreeAsync: %s", cudaGetErrorString(e));
    return st;
}

}  // namespace
}  // namespace svdlut

using namespace svdlut;

extern "C" svdlut_status svdlut_apply_io(const svdlut_dims *dims, const svdlut_params *params, int B, int H, int W,
                                         svdlut_pixfmt in_fmt, const void *x, svdlut_pixfmt out_fmt, void *y,
                                         svdlut_stream_t stream)
{
    SVDLUT_TRACE("svdlut_apply_io");
    clear_error();
    if (in_fmt == SVDLUT_PIX_F32 && out_fmt == SVDLUT_PIX_F32)
        return svdlut_apply(dims, params, B, H, W, SVDLUT_F32, x, y, stream);
    if (in_fmt == SVDLUT_PIX_U8 && out_fmt == SVDLUT_PIX_U8)
        return svdlut_apply(dims, params, B, H, W, SVDLUT_U8, x, y, stream);
    svdlut_status st = check_dims(dims);
    if (st != SVDLUT_OK) return st;
    if ((st = check_params(dims, params)) != SVDLUT_OK) return st;
    if (B < 1 || H < 1 || W < 1) return fail(SVDLUT_ERR_INVALID_ARG, "B=%d H=%d W=%d must be >= 1", B, H, W);
    FmtInfo fi{}, fo{};
    if (!fmt_info(in_fmt, &fi) || !fmt_info(out_fmt, &fo))
        return fail(SVDLUT_ERR_INVALID_ARG, "unknown pixel format %d -> %d", in_fmt, out_fmt);
    if (!x || !y) return fail(SVDLUT_ERR_INVALID_ARG, "x and y are required");
    if (!aligned(x, fi.align) || !aligned(y, fo.align))
        return fail(SVDLUT_ERR_INVALID_ARG, "arrays must be aligned to their element size");
    const size_t px = static_cast<size_t>(B) * H * W;
    const char *xs = static_cast<const char *>(x), *ys = static_cast<const char *>(y);
    if (xs < ys + px * fo.px_bytes && ys < xs + px * fi.px_bytes)
        return fail(SVDLUT_ERR_INVALID_ARG, "x and y overlap");
    const cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (in_fmt == SVDLUT_PIX_U16 && (out_fmt == SVDLUT_PIX_U8 || out_fmt == SVDLUT_PIX_F32))
        return run_u16(dims, params, B, H, W, x, false, out_fmt, y, fo, s);
    if (in_fmt == SVDLUT_PIX_U8_HWC && out_fmt == SVDLUT_PIX_U8_HWC)
        return run_io<Io<InU8Hwc, OutU8Hwc>>(dims, params, B, H, W, x, fi, y, fo, s);
    if (in_fmt == SVDLUT_PIX_U16_HWC && out_fmt == SVDLUT_PIX_U8_HWC)
        return run_u16(dims, params, B, H, W, x, true, out_fmt, y, fo, s);
    return fail(SVDLUT_ERR_UNSUPPORTED, "pixel formats %d -> %d are not supported", in_fmt, out_fmt);
}
