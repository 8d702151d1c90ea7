// svdlut_apply: host entry of the plain (same-size batch) fused apply.
#include <algorithm>
#include <cmath>

#include "apply_kernel.cuh"
#include "apply_launch.cuh"

namespace svdlut {

svdlut_status check_params(const svdlut_dims *d, const svdlut_params *p)
{
    if (!p) return fail(SVDLUT_ERR_INVALID_ARG, "params is NULL");
    if (!p->U || !p->S || !p->V || !p->lut_w)
        return fail(SVDLUT_ERR_INVALID_ARG, "params: U, S, V and lut_w are required");
    if (d->K > 0 && (!p->g_xy || !p->g_xc || !p->g_yc || !p->grid_w))
        return fail(SVDLUT_ERR_INVALID_ARG, "params: g_xy, g_xc, g_yc and grid_w are required when K > 0");
    const void *ptrs[8] = {p->U, p->S, p->V, p->lut_w, p->g_xy, p->g_xc, p->g_yc, p->grid_w};
    for (const void *q : ptrs)
        if (q && !aligned(q, 4)) return fail(SVDLUT_ERR_INVALID_ARG, "params: pointers must be 4-byte aligned");
    return SVDLUT_OK;
}

size_t param_stride(const svdlut_dims *d, int which)
{
    const size_t D = d->D_t, R = d->rank, K = d->K;
    switch (which) {
    case 0: return 9 * D * R;                              // U
    case 1: return 9 * R;                                  // S
    case 2: return 9 * D * R;                              // V
    case 3: return 12;                                     // lut_w
    case 4: return K * d->Dsy * d->Dsx;                    // g_xy
    case 5: return K * d->Dsx * d->Dsc;                    // g_xc
    case 6: return K * d->Dsy * d->Dsc;                    // g_yc
    default: return K * 4;                                 // grid_w
    }
}

ImgDesc make_desc_io(const svdlut_dims *d, const svdlut_params *p, int b, int H, int W, const void *x,
                     size_t x_px_bytes, size_t x_align, void *y, size_t y_px_bytes, size_t y_align)
{
    ImgDesc e{};
    const size_t px = static_cast<size_t>(H) * W;
    e.x = static_cast<const char *>(x) + b * px * x_px_bytes;
    e.y = static_cast<char *>(y) + b * px * y_px_bytes;
    e.U = p->U + b * param_stride(d, 0);
    e.S = p->S + b * param_stride(d, 1);
    e.V = p->V + b * param_stride(d, 2);
    e.lw = p->lut_w + b * param_stride(d, 3);
    e.gxy = p->g_xy ? p->g_xy + b * param_stride(d, 4) : nullptr;
    e.gxc = p->g_xc ? p->g_xc + b * param_stride(d, 5) : nullptr;
    e.gyc = p->g_yc ? p->g_yc + b * param_stride(d, 6) : nullptr;
    e.gw = p->grid_w ? p->grid_w + b * param_stride(d, 7) : nullptr;
    e.H = H;
    e.W = W;
    e.y_begin = 0;
    e.y_end = H;
    e.D = d->D_t;
    e.R = d->rank;
    e.K = d->K;
    e.Dsx = d->Dsx;
    e.Dsy = d->Dsy;
    e.Dsc = d->Dsc;
    e.rW1 = W > 1 ? 1.0f / static_cast<float>(W - 1) : 0.f;
    e.rH1 = H > 1 ? 1.0f / static_cast<float>(H - 1) : 0.f;
    e.vec = (W % 4 == 0) && aligned(e.x, x_align) && aligned(e.y, y_align);
    return e;
}

ImgDesc make_desc(const svdlut_dims *d, const svdlut_params *p, int b, int H, int W, svdlut_dtype dt,
                  const void *x, void *y)
{
    const size_t es = dt == SVDLUT_F32 ? 4 : 1, va = dt == SVDLUT_F32 ? 16 : 4;
    return make_desc_io(d, p, b, H, W, x, 3 * es, va, y, 3 * es, va);
}

}  // namespace svdlut

using namespace svdlut;

static svdlut_status apply_impl(const svdlut_dims *dims, const svdlut_params *params, int B, int H, int W,
                                svdlut_dtype dtype, const void *x, void *y, int ctas, void *ws, size_t ws_bytes,
                                svdlut_stream_t stream);

extern "C" svdlut_status svdlut_apply(const svdlut_dims *dims, const svdlut_params *params, int B, int H,
                                      int W, svdlut_dtype dtype, const void *x, void *y,
                                      svdlut_stream_t stream)
{
    SVDLUT_TRACE("svdlut_apply");
    return apply_impl(dims, params, B, H, W, dtype, x, y, 0, nullptr, 0, stream);
}

extern "C" svdlut_status svdlut_apply_cfg(const svdlut_dims *dims, const svdlut_params *params, int B, int H,
                                          int W, svdlut_dtype dtype, const void *x, void *y,
                                          const svdlut_launch_cfg *cfg, svdlut_stream_t stream)
{
    SVDLUT_TRACE("svdlut_apply_cfg");
    clear_error();
    if (cfg && cfg->ctas < 0) return fail(SVDLUT_ERR_INVALID_ARG, "negative CTA count");
    return apply_impl(dims, params, B, H, W, dtype, x, y, cfg ? cfg->ctas : 0, nullptr, 0, stream);
}

extern "C" size_t svdlut_apply_workspace_size(const svdlut_dims *dims, int B)
{
    if (B < 1 || check_dims(dims) != SVDLUT_OK) return 0;
    return static_cast<size_t>(B) * prep_image_bytes(dims);
}

extern "C" svdlut_status svdlut_apply_ws(const svdlut_dims *dims, const svdlut_params *params, int B, int H, int W,
                                         svdlut_dtype dtype, const void *x, void *y, const svdlut_launch_cfg *cfg,
                                         void *ws, size_t ws_bytes, svdlut_stream_t stream)
{
    SVDLUT_TRACE("svdlut_apply_ws");
    clear_error();
    if (cfg && cfg->ctas < 0) return fail(SVDLUT_ERR_INVALID_ARG, "negative CTA count");
    if (!ws) return fail(SVDLUT_ERR_WORKSPACE, "workspace is NULL");
    return apply_impl(dims, params, B, H, W, dtype, x, y, cfg ? cfg->ctas : 0, ws, ws_bytes, stream);
}

// The launches of a planned batch, N images each: the per-image tables first
// (prep_kernel) when a workspace is given, then apply_kernel.
template <int N>
static svdlut_status apply_chunks(const svdlut_dims *dims, const svdlut_params *params, int B, int H, int W,
                                  svdlut_dtype dtype, const void *x, void *y, int n_cta, void *ws, size_t per_img,
                                  const DeviceInfo &di, cudaStream_t s)
{
    svdlut_status st = SVDLUT_OK;
    for (int b0 = 0; b0 < B; b0 += N) {
        LaunchArgs<N> a{};
        a.n = std::min(N, B - b0);
        for (int i = 0; i < a.n; ++i) {
            a.img[i] = make_desc(dims, params, b0 + i, H, W, dtype, x, y);
            if (ws) set_prep_tables(a.img[i], dims, static_cast<char *>(ws) + static_cast<size_t>(b0 + i) * per_img);
        }
        size_t smem = 0;
        if ((st = plan_uniform(a, n_cta, static_cast<size_t>(di.max_smem_optin), &smem)) != SVDLUT_OK)
            return st;
        if (ws) {
            if ((st = launch_prep(a, di.sm_count, s)) != SVDLUT_OK) return st;
            a.pre = 1;
        }
        if ((st = launch_apply(a, smem, dtype, s, n_cta)) != SVDLUT_OK) return st;
    }
    return SVDLUT_OK;
}

static svdlut_status apply_impl(const svdlut_dims *dims, const svdlut_params *params, int B, int H, int W,
                                svdlut_dtype dtype, const void *x, void *y, int ctas, void *ws, size_t ws_bytes,
                                svdlut_stream_t stream)
{
    clear_error();
    svdlut_status st = check_dims(dims);
    if (st != SVDLUT_OK) return st;
    if ((st = check_params(dims, params)) != SVDLUT_OK) return st;
    if (B < 1 || H < 1 || W < 1) return fail(SVDLUT_ERR_INVALID_ARG, "B=%d H=%d W=%d must be >= 1", B, H, W);
    if (dtype != SVDLUT_F32 && dtype != SVDLUT_U8) return fail(SVDLUT_ERR_INVALID_ARG, "unknown dtype %d", dtype);
    if (!x || !y) return fail(SVDLUT_ERR_INVALID_ARG, "x and y are required");
    const size_t es = dtype == SVDLUT_F32 ? 4 : 1;
    if (dtype == SVDLUT_F32 && (!aligned(x, 4) || !aligned(y, 4)))
        return fail(SVDLUT_ERR_INVALID_ARG, "float images must be 4-byte aligned");
    const size_t bytes = static_cast<size_t>(B) * 3 * H * W * es;
    const char *xs = static_cast<const char *>(x), *ys = static_cast<const char *>(y);
    if (xs < ys + bytes && ys < xs + bytes) return fail(SVDLUT_ERR_INVALID_ARG, "x and y overlap");

    const size_t per_img = prep_image_bytes(dims);
    if (ws) {
        if (ws_bytes < static_cast<size_t>(B) * per_img)
            return fail(SVDLUT_ERR_WORKSPACE, "workspace of %zu bytes needed (got %zu)",
                        static_cast<size_t>(B) * per_img, ws_bytes);
        if (!aligned(ws, 256)) return fail(SVDLUT_ERR_INVALID_ARG, "workspace must be 256-byte aligned");
        char *ws_c = static_cast<char *>(ws);
        if ((ws_c < ys + bytes && ys < ws_c + B * per_img) || (ws_c < xs + bytes && xs < ws_c + B * per_img))
            return fail(SVDLUT_ERR_INVALID_ARG, "workspace overlaps x or y");
    }

    DeviceInfo di;
    if ((st = device_info(&di)) != SVDLUT_OK) return st;
    const int n_cta = ctas > 0 ? std::min(ctas, di.sm_count) : di.sm_count;  // persistent CTAs to plan for
    const cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    // up to 16 images per launch, or 64 when the batch is larger (fewer launches
    // and table precomputations for batches of small images)
    return B > kPlainChunk ? apply_chunks<kRaggedMax>(dims, params, B, H, W, dtype, x, y, n_cta, ws, per_img, di, s)
                           : apply_chunks<kPlainChunk>(dims, params, B, H, W, dtype, x, y, n_cta, ws, per_img, di, s);
}
