// Launch helper for apply_kernel (shared by the plain and ragged entries).
#pragma once

#include <algorithm>
#include <mutex>
#include <utility>
#include <vector>

#include "apply_kernel.cuh"

namespace svdlut {

constexpr int kPlainChunk = 16;   // images per launch of svdlut_apply
constexpr int kRaggedMax = 64;    // images per launch of svdlut_apply_batched

svdlut_status check_params(const svdlut_dims *d, const svdlut_params *p);
size_t param_stride(const svdlut_dims *d, int which);
ImgDesc make_desc(const svdlut_dims *d, const svdlut_params *p, int b, int H, int W, svdlut_dtype dt,
                  const void *x, void *y);
// x_px_bytes / y_px_bytes: bytes of one pixel (all three channels) of the
// input / output format; x_align / y_align: alignment of its vector access
ImgDesc make_desc_io(const svdlut_dims *d, const svdlut_params *p, int b, int H, int W, const void *x,
                     size_t x_px_bytes, size_t x_align, void *y, size_t y_px_bytes, size_t y_align);

// Shared-memory bytes of args a for block heights up to bh_max; the
// all-nine-tables prologue is enabled when it fits.  Sets lcell/scratch sizes.
// Shared-memory bytes of args a for block heights up to bh_max; the
// all-nine-tables prologue is enabled when it fits.  Sets lcell/scratch sizes.
template <int N>
size_t apply_smem_bytes(LaunchArgs<N> &a, size_t limit)
{
    int Dmax = 2, pro1 = 0, pro3 = 0, blk = 0;
    for (int i = 0; i < a.n; ++i) {
        const ImgDesc &e = a.img[i];
        Dmax = std::max(Dmax, e.D);
        pro1 = std::max(pro1, prologue_floats_n(e.D, e.R, 1));
        pro3 = std::max(pro3, prologue_floats_n(e.D, e.R, 3));
        blk = std::max(blk, block_floats(a.nvx_max, a.nvy_max, e.Dsc, a.bh_max, a.xcol != 0));
    }
    a.lcell_floats = lcell_floats(Dmax);
    auto bytes = [&](int scratch) {
        return sizeof(float) * (static_cast<size_t>(a.lcell_floats) + kMiscFloats + scratch);
    };
    const int base = std::max(blk, pro1);
    a.scratch_floats = bytes(std::max(base, pro3)) <= limit ? std::max(base, pro3) : base;
    return bytes(a.scratch_floats);
}

// Plans the block split of B same-size images: each image is cut into
// `strips` column strips of kTileW pixels and `bands` row bands; bands
// minimises the estimated time, waves x (rows each warp walks in a block + a
// fixed cost of about one row per block: the block's tables), with ties
// going to the better-filled waves, while the block buffers fit in shared
// memory.  Fills strips/BH/block_begin, total_blocks, nvx_max, nvy_max,
// bh_max and the shared-memory size.
template <int N>
svdlut_status plan_uniform(LaunchArgs<N> &a, int sm_count, size_t smem_limit, size_t *smem_out)
{
    const ImgDesc &e0 = a.img[0];
    // rows to cover (a row range of the image for banded calls); grid
    // spacing still follows the full image height H
    const int H = e0.H, W = e0.W, rows = e0.y_end - e0.y_begin, strips = (W + kTileW - 1) / kTileW;
    const int max_bands = std::max(1, (rows + kMinBlockH - 1) / kMinBlockH);
    int best = -1;
    double best_score = -1e30;
    const int nvx = span_bound(kTileW, W, e0.Dsx);
    a.xcol = e0.Dsc <= kXcolMaxDsc;
    const int fixed = lcell_floats(e0.D) + kMiscFloats;
    const int pro = prologue_floats_n(e0.D, e0.R, 1);  // required; all-pairs-at-once is optional
    for (int bands = 1; bands <= max_bands; ++bands) {
        const int BH = (rows + bands - 1) / bands;
        const int need = fixed + std::max(pro, block_floats(nvx, span_bound(BH, H, e0.Dsy), e0.Dsc, BH, a.xcol != 0));
        if (sizeof(float) * static_cast<size_t>(need) > smem_limit) continue;
        const long long T = static_cast<long long>(a.n) * strips * ((rows + BH - 1) / BH);
        const double waves = std::ceil(static_cast<double>(T) / sm_count - 1e-9);
        const double fill = static_cast<double>(T) / (waves * sm_count);  // share of SM time used
        const double score = -waves * ((BH + kWarps - 1) / kWarps + 1) + 1e-3 * fill;
        if (score > best_score + 1e-12) {
            best_score = score;
            best = bands;
        }
        if (bands >= 4 * sm_count) break;
    }
    if (best < 0)
        return fail(SVDLUT_ERR_UNSUPPORTED,
                    "grid slices of a %dx%d block do not fit in shared memory (%zu bytes): grid vertices too "
                    "dense or D_t/rank too large", kTileW, kMinBlockH, smem_limit);
    const int BH = (rows + best - 1) / best;
    const int bands = (rows + BH - 1) / BH;
    for (int i = 0; i < a.n; ++i) {
        a.img[i].strips = strips;
        a.img[i].BH = BH;
        a.img[i].block_begin = i * strips * bands;
    }
    a.total_blocks = a.n * strips * bands;
    a.nvx_max = span_bound(kTileW, W, e0.Dsx);
    a.nvy_max = span_bound(BH, H, e0.Dsy);
    a.bh_max = BH;
    *smem_out = apply_smem_bytes(a, smem_limit);
    return SVDLUT_OK;
}

// Opts kernel `fn` into max_smem bytes of dynamic shared memory once per
// device.  Keyed by the kernel's host address: every translation unit that
// launches a kernel template has its own instance of it.
inline svdlut_status allow_smem_once(const void *fn, int max_smem, int device)
{
    static std::mutex mu;
    static std::vector<std::pair<int, const void *>> done;
    std::lock_guard<std::mutex> g(mu);
    for (const auto &e : done)
        if (e.first == device && e.second == fn) return SVDLUT_OK;
    SVDLUT_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem));
    done.emplace_back(device, fn);
    return SVDLUT_OK;
}

template <class IO, int N, bool DX>
svdlut_status launch_apply_t(LaunchArgs<N> &a, size_t smem, int sm_count, int max_smem, int device,
                             cudaStream_t s, int grid)
{
    svdlut_status st = allow_smem_once(reinterpret_cast<const void *>(apply_kernel<IO, N, DX>), max_smem, device);
    if (st != SVDLUT_OK) return st;
    if ((st = check_buffer(&a.check)) != SVDLUT_OK) return st;
    if (grid <= 0) grid = std::min(a.total_blocks, sm_count);
    grid = std::max(1, std::min(grid, a.total_blocks));
    if (a.pre) {
        // dependent of the preceding prep_kernel: it may start while that
        // kernel runs and waits for it before reading the tables
        return launch_pdl(apply_kernel<IO, N, DX>, dim3(grid), dim3(kThreads), smem, s, a);
    }
    apply_kernel<IO, N, DX><<<grid, kThreads, smem, s>>>(a);
    SVDLUT_CUDA_TRY(cudaGetLastError());
    return SVDLUT_OK;
}

// Workspace bytes of the precomputed tables of one image, and the launch of
// prep_kernel over a chunk of planned images (pcell / pfold set).
inline size_t prep_image_bytes(const svdlut_dims *d)
{
    auto a256 = [](size_t v) { return (v + 255) & ~static_cast<size_t>(255); };
    return a256(sizeof(float) * static_cast<size_t>(lcell_floats(d->D_t))) +
           a256(sizeof(float) * (pfold_floats(d->Dsx, d->Dsy, d->Dsc) + 3));
}

// Points the descriptor's precomputed tables at w (prep_image_bytes(d) bytes).
inline void set_prep_tables(ImgDesc &e, const svdlut_dims *d, char *w)
{
    e.pcell = reinterpret_cast<float *>(w);
    e.pfold = reinterpret_cast<float *>(
        w + ((sizeof(float) * static_cast<size_t>(lcell_floats(d->D_t)) + 255) & ~static_cast<size_t>(255)));
}

template <int N>
svdlut_status launch_prep(const LaunchArgs<N> &a, int sm_count, cudaStream_t s)
{
    PrepArgs<N> pa{};
    pa.n = a.n;
    double total = 0;
    int smem_fl = 0;
    for (int i = 0; i < a.n; ++i) {
        const ImgDesc &e = a.img[i];
        pa.img[i] = e;
        pa.start[i] = static_cast<int>(total);
        total += static_cast<double>(pfold_floats(e.Dsx, e.Dsy, e.Dsc) + 3);
        if (total >= 2147483647.0)
            return fail(SVDLUT_ERR_UNSUPPORTED, "grids of %d images too large for the workspace path", a.n);
        smem_fl = std::max(smem_fl, prep_smem_floats(e.D, e.R));
    }
    pa.start[a.n] = static_cast<int>(total);
    const int fold_ctas = std::max(sm_count, 2 * sm_count - kLutCtas * a.n);
    const size_t smem = sizeof(float) * static_cast<size_t>(smem_fl);
    // programmatic dependent of the preceding kernel (it waits for it first)
    return launch_pdl(prep_kernel<N>, dim3(kLutCtas * a.n + fold_ctas), dim3(kPrepThreads), smem, s, pa);
}

// Launches apply_kernel for args whose blocks are already planned.  dx_mode
// runs the pixel part of the adjoint (float images only).
template <int N>
svdlut_status launch_apply(LaunchArgs<N> &a, size_t smem, svdlut_dtype dt, cudaStream_t s, int grid,
                           bool dx_mode = false)
{
    if (a.total_blocks <= 0) return SVDLUT_OK;
    DeviceInfo di;
    svdlut_status st = device_info(&di);
    if (st != SVDLUT_OK) return st;
    if (dx_mode) return launch_apply_t<IoF32, N, true>(a, smem, di.sm_count, di.max_smem_optin, di.device, s, grid);
    return dt == SVDLUT_F32
               ? launch_apply_t<IoF32, N, false>(a, smem, di.sm_count, di.max_smem_optin, di.device, s, grid)
               : launch_apply_t<IoU8, N, false>(a, smem, di.sm_count, di.max_smem_optin, di.device, s, grid);
}

}  // namespace svdlut
