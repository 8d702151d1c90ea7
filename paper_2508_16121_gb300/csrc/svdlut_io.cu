// svdlut_apply_io: the fused transform between pixel formats.  The 16-bit
// inputs (the tone-mapping and PPR10K photos, Sec. 4.1) and interleaved
// 8-bit frames are decoded, and 8-bit outputs encoded, inside apply_kernel,
// so a 16-bit photo goes to an 8-bit result in one pass over HBM with no
// conversion buffers.  Only the pairs listed in svdlut.h are instantiated.
#include <algorithm>

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
    if (in_fmt == SVDLUT_PIX_U16 && out_fmt == SVDLUT_PIX_U8)
        return run_io<Io<InU16, OutU8>>(dims, params, B, H, W, x, fi, y, fo, s);
    if (in_fmt == SVDLUT_PIX_U16 && out_fmt == SVDLUT_PIX_F32)
        return run_io<Io<InU16, OutF32>>(dims, params, B, H, W, x, fi, y, fo, s);
    if (in_fmt == SVDLUT_PIX_U8_HWC && out_fmt == SVDLUT_PIX_U8_HWC)
        return run_io<Io<InU8Hwc, OutU8Hwc>>(dims, params, B, H, W, x, fi, y, fo, s);
    if (in_fmt == SVDLUT_PIX_U16_HWC && out_fmt == SVDLUT_PIX_U8_HWC)
        return run_io<Io<InU16Hwc, OutU8Hwc>>(dims, params, B, H, W, x, fi, y, fo, s);
    return fail(SVDLUT_ERR_UNSUPPORTED, "pixel formats %d -> %d are not supported", in_fmt, out_fmt);
}
