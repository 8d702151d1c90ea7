// svdlut_apply_batched: one persistent launch over images of uneven sizes,
// each with its own transform, and its autotuner.
//
// Every image is cut into 128-pixel column strips and row bands (BH rows);
// the blocks of all images form one image-major list.  With the queue
// schedule the CTAs (one per SM) take blocks from an atomic counter, so uneven
// blocks and uneven content (noise-like images cost more shared-memory gathers
// than smooth ones) balance out; with the ranges schedule each CTA takes a
// contiguous range of the list, so it meets fewer images.  A CTA rebuilds its
// LUT tables only when the next block belongs to another image.
#include <algorithm>
#include <cmath>
#include <vector>

#include "apply_kernel.cuh"
#include "apply_launch.cuh"

namespace svdlut {

static svdlut_status check_image(const svdlut_image &im, svdlut_dtype dt, int i)
{
    svdlut_status st = check_dims(&im.dims);
    if (st == SVDLUT_OK) st = check_params(&im.dims, &im.params);
    if (st != SVDLUT_OK) {
        char msg[512];
        snprintf(msg, sizeof msg, "%s", svdlut_last_error());
        return fail(st, "image %d: %s", i, msg);
    }
    if (im.H < 1 || im.W < 1) return fail(SVDLUT_ERR_INVALID_ARG, "image %d: H=%d W=%d", i, im.H, im.W);
    if (!im.x || !im.y) return fail(SVDLUT_ERR_INVALID_ARG, "image %d: x and y are required", i);
    if (dt == SVDLUT_F32 && (!aligned(im.x, 4) || !aligned(im.y, 4)))
        return fail(SVDLUT_ERR_INVALID_ARG, "image %d: float images must be 4-byte aligned", i);
    const size_t bytes = static_cast<size_t>(3) * im.H * im.W * (dt == SVDLUT_F32 ? 4 : 1);
    const char *xs = static_cast<const char *>(im.x), *ys = static_cast<const char *>(im.y);
    if (xs < ys + bytes && ys < xs + bytes) return fail(SVDLUT_ERR_INVALID_ARG, "image %d: x and y overlap", i);
    return SVDLUT_OK;
}

// Plans images [i0, i0 + a.n) with about block_px pixels per block; shrinks a
// block's height until its grid slices fit in shared memory.
static svdlut_status plan_ragged(LaunchArgs<kRaggedMax> &a, const svdlut_image *imgs, int i0, svdlut_dtype dt,
                                 int block_px, size_t smem_limit, size_t *smem_out)
{
    int begin = 0;
    a.nvx_max = 2;
    a.nvy_max = 2;
    a.bh_max = 1;
    a.xcol = 1;
    for (int i = 0; i < a.n; ++i)
        if (imgs[i0 + i].dims.Dsc > kXcolMaxDsc) a.xcol = 0;
    for (int i = 0; i < a.n; ++i) {
        const svdlut_image &im = imgs[i0 + i];
        ImgDesc e = make_desc(&im.dims, &im.params, 0, im.H, im.W, dt, im.x, im.y);
        e.strips = (im.W + kTileW - 1) / kTileW;
        int BH = std::max(kMinBlockH, std::min(im.H, (block_px + kTileW - 1) / kTileW));
        for (;;) {
            const int bands = (im.H + BH - 1) / BH;
            BH = (im.H + bands - 1) / bands;
            const int nvx = span_bound(kTileW, im.W, im.dims.Dsx), nvy = span_bound(BH, im.H, im.dims.Dsy);
            const size_t need =
                sizeof(float) * (static_cast<size_t>(lcell_floats(im.dims.D_t)) + kMiscFloats +
                                 std::max(prologue_floats_n(im.dims.D_t, im.dims.rank, 1),
                                          block_floats(nvx, nvy, im.dims.Dsc, BH, a.xcol != 0)));
            if (need <= smem_limit) break;
            if (BH <= 1)
                return fail(SVDLUT_ERR_UNSUPPORTED, "image %d: grid slices do not fit in shared memory", i0 + i);
            BH = std::max(1, BH / 2);
        }
        e.BH = BH;
        e.block_begin = begin;
        begin += e.strips * ((im.H + BH - 1) / BH);
        a.nvx_max = std::max(a.nvx_max, span_bound(kTileW, im.W, im.dims.Dsx));
        a.nvy_max = std::max(a.nvy_max, span_bound(BH, im.H, im.dims.Dsy));
        a.bh_max = std::max(a.bh_max, BH);
        a.img[i] = e;
    }
    a.total_blocks = begin;
    *smem_out = apply_smem_bytes(a, smem_limit);
    if (*smem_out > smem_limit)
        return fail(SVDLUT_ERR_UNSUPPORTED, "batch needs %zu bytes of shared memory (limit %zu)", *smem_out, smem_limit);
    return SVDLUT_OK;
}

static int auto_block_px(const svdlut_image *imgs, int n, int sm_count)
{
    double px = 0;
    for (int i = 0; i < n; ++i) px += static_cast<double>(imgs[i].H) * imgs[i].W;
    // about four blocks per CTA, within 16 .. 1024 rows of 128 pixels
    const double t = px / (4.0 * sm_count);
    return static_cast<int>(std::min(1024.0 * kTileW, std::max(16.0 * kTileW, t)));
}

// Workspace of the queue counters alone, and with the precomputed per-image
// tables after them (256-byte aligned).
static size_t queue_bytes(int n)
{
    const size_t chunks = (static_cast<size_t>(n) + kRaggedMax - 1) / kRaggedMax;
    return (chunks * sizeof(unsigned int) + 255) & ~static_cast<size_t>(255);
}
static size_t tables_bytes(const svdlut_image *imgs, int n)
{
    size_t t = 0;
    for (int i = 0; i < n; ++i) t += prep_image_bytes(&imgs[i].dims);
    return t;
}

static svdlut_status run_batched(const svdlut_image *imgs, int n, svdlut_dtype dtype, const svdlut_launch_cfg *cfg,
                                 void *ws, size_t ws_bytes, cudaStream_t s)
{
    svdlut_status st;
    DeviceInfo di;
    if ((st = device_info(&di)) != SVDLUT_OK) return st;
    const int block_px = cfg && cfg->block_px > 0 ? cfg->block_px : auto_block_px(imgs, n, di.sm_count);
    const int ctas = cfg && cfg->ctas > 0 ? cfg->ctas : di.sm_count;
    const bool ranges = cfg && cfg->schedule == SVDLUT_SCHED_RANGES;
    unsigned int *queue = static_cast<unsigned int *>(ws);
    // per-image tables precomputed once (prep_kernel) when the workspace holds them
    const bool pre = ws_bytes >= queue_bytes(n) + tables_bytes(imgs, n) && aligned(ws, 256);
    char *tab = static_cast<char *>(ws) + queue_bytes(n);
    for (int i0 = 0, chunk = 0; i0 < n; i0 += kRaggedMax, ++chunk) {
        LaunchArgs<kRaggedMax> a{};
        a.n = std::min(kRaggedMax, n - i0);
        size_t smem = 0;
        if ((st = plan_ragged(a, imgs, i0, dtype, block_px, static_cast<size_t>(di.max_smem_optin), &smem)) !=
            SVDLUT_OK)
            return st;
        if (!ranges) {
            a.queue = queue + chunk;
            SVDLUT_CUDA_TRY(cudaMemsetAsync(a.queue, 0, sizeof(unsigned int), s));
        }
        if (pre) {
            for (int i = 0; i < a.n; ++i) {
                set_prep_tables(a.img[i], &imgs[i0 + i].dims, tab);
                tab += prep_image_bytes(&imgs[i0 + i].dims);
            }
            if ((st = launch_prep(a, di.sm_count, s)) != SVDLUT_OK) return st;
            a.pre = 1;
        }
        if ((st = launch_apply(a, smem, dtype, s, std::min(ctas, a.total_blocks))) != SVDLUT_OK) return st;
    }
    return SVDLUT_OK;
}

}  // namespace svdlut

using namespace svdlut;

extern "C" size_t svdlut_batched_workspace_size(int n)
{
    if (n < 1) return 0;
    return queue_bytes(n);
}

extern "C" size_t svdlut_batched_tables_workspace_size(const svdlut_image *imgs, int n)
{
    if (!imgs || n < 1) return 0;
    for (int i = 0; i < n; ++i)
        if (check_dims(&imgs[i].dims) != SVDLUT_OK) return 0;
    return queue_bytes(n) + tables_bytes(imgs, n);
}

extern "C" svdlut_status svdlut_apply_batched(const svdlut_image *imgs, int n, svdlut_dtype dtype,
                                              const svdlut_launch_cfg *cfg, void *ws, size_t ws_bytes,
                                              svdlut_stream_t stream)
{
    SVDLUT_TRACE("svdlut_apply_batched");
    clear_error();
    if (!imgs || n < 1) return fail(SVDLUT_ERR_INVALID_ARG, "imgs is NULL or n=%d < 1", n);
    if (dtype != SVDLUT_F32 && dtype != SVDLUT_U8) return fail(SVDLUT_ERR_INVALID_ARG, "unknown dtype %d", dtype);
    svdlut_status st;
    for (int i = 0; i < n; ++i)
        if ((st = check_image(imgs[i], dtype, i)) != SVDLUT_OK) return st;
    if (cfg && (cfg->block_px < 0 || cfg->ctas < 0)) return fail(SVDLUT_ERR_INVALID_ARG, "negative launch config");
    if (cfg && cfg->schedule != SVDLUT_SCHED_QUEUE && cfg->schedule != SVDLUT_SCHED_RANGES)
        return fail(SVDLUT_ERR_INVALID_ARG, "unknown schedule %d", cfg->schedule);
    if (!ws || ws_bytes < svdlut_batched_workspace_size(n))
        return fail(SVDLUT_ERR_WORKSPACE, "workspace of %zu bytes needed", svdlut_batched_workspace_size(n));
    if (!aligned(ws, 4)) return fail(SVDLUT_ERR_INVALID_ARG, "workspace must be 4-byte aligned");
    return run_batched(imgs, n, dtype, cfg, ws, ws_bytes, reinterpret_cast<cudaStream_t>(stream));
}

extern "C" svdlut_status svdlut_autotune_batched(const svdlut_image *imgs, int n, svdlut_dtype dtype, void *ws,
                                                 size_t ws_bytes, svdlut_stream_t stream, int reps,
                                                 svdlut_launch_cfg *best, float *best_ms)
{
    SVDLUT_TRACE("svdlut_autotune_batched");
    clear_error();
    if (!best) return fail(SVDLUT_ERR_INVALID_ARG, "best is NULL");
    if (!imgs || n < 1) return fail(SVDLUT_ERR_INVALID_ARG, "imgs is NULL or n=%d < 1", n);
    if (reps < 1) reps = 1;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    DeviceInfo di;
    svdlut_status st = device_info(&di);
    if (st != SVDLUT_OK) return st;
    const int base = auto_block_px(imgs, n, di.sm_count);
    std::vector<svdlut_launch_cfg> cands;
    for (int sched : {SVDLUT_SCHED_QUEUE, SVDLUT_SCHED_RANGES}) {
        for (int rows : {16, 32, 64, 128, 256, 512}) cands.push_back({rows * kTileW, 0, sched});
        cands.push_back({base, 0, sched});
    }
    cudaEvent_t e0, e1;
    SVDLUT_CUDA_TRY(cudaEventCreate(&e0));
    SVDLUT_CUDA_TRY(cudaEventCreate(&e1));
    float best_t = 1e30f;
    svdlut_launch_cfg win = cands.back();
    for (const svdlut_launch_cfg &c : cands) {
        // warm-up, then timed repetitions
        if ((st = svdlut_apply_batched(imgs, n, dtype, &c, ws, ws_bytes, stream)) != SVDLUT_OK) break;
        cudaEventRecord(e0, s);
        for (int r = 0; r < reps && st == SVDLUT_OK; ++r) st = svdlut_apply_batched(imgs, n, dtype, &c, ws, ws_bytes, stream);
        cudaEventRecord(e1, s);
        if (st != SVDLUT_OK) break;
        if (cudaEventSynchronize(e1) != cudaSuccess) {
            st = fail(SVDLUT_ERR_CUDA, "autotune: event synchronize failed");
            break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        ms /= reps;
        if (ms < best_t) {
            best_t = ms;
            win = c;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != SVDLUT_OK) return st;
    *best = win;
    if (best_ms) *best_ms = best_t;
    return SVDLUT_OK;
}
