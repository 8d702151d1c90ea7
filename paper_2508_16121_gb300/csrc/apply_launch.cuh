// Launch helper for apply_kernel (shared by the plain and ragged entries).
#pragma once

#include <algorithm>
#include <mutex>

#include "apply_kernel.cuh"

namespace svdlut {

constexpr int kPlainChunk = 16;   // images per launch of svdlut_apply
constexpr int kRaggedMax = 64;    // images per launch of svdlut_apply_batched

svdlut_status check_params(const svdlut_dims *d, const svdlut_params *p);
size_t param_stride(const svdlut_dims *d, int which);
ImgDesc make_desc(const svdlut_dims *d, const svdlut_params *p, int b, int H, int W, svdlut_dtype dt,
                  const void *x, void *y);

// Dynamic shared memory (bytes) for args a, given the per-block limit; sets
// a.lcell_floats, a.stage_floats and a.scratch_floats.  The grid-slice
// staging area and the all-tables-at-once prologue are used when they fit.
template <int N>
size_t apply_smem_bytes(LaunchArgs<N> &a, size_t limit)
{
    int Dmax = 2, pro1 = 0, pro3 = 0, til = 0, stg = 0;
    for (int i = 0; i < a.n; ++i) {
        const ImgDesc &e = a.img[i];
        Dmax = std::max(Dmax, e.D);
        pro1 = std::max(pro1, prologue_floats_n(e.D, e.R, 1));
        pro3 = std::max(pro3, prologue_floats_n(e.D, e.R, 3));
        til = std::max(til, tile_floats(a.nvx_max, a.nvy_max, e.Dsc));
        stg = std::max(stg, stage_floats(e.K, a.nvx_max, a.nvy_max, e.Dsc));
    }
    stg = (stg + 3) & ~3;
    a.lcell_floats = lcell_floats(Dmax);
    auto bytes = [&](int stage, int scratch) {
        return sizeof(float) * (static_cast<size_t>(a.lcell_floats) + kMiscFloats + stage + scratch);
    };
    const int base = std::max(til, pro1);
    a.stage_floats = kStage && bytes(stg, base) <= limit ? stg : 0;
    a.scratch_floats = bytes(a.stage_floats, std::max(base, pro3)) <= limit ? std::max(base, pro3) : base;
    return bytes(a.stage_floats, a.scratch_floats);
}

template <typename T, int N>
svdlut_status launch_apply_t(LaunchArgs<N> &a, cudaStream_t s, int grid)
{
    DeviceInfo di;
    svdlut_status st = device_info(&di);
    if (st != SVDLUT_OK) return st;
    const size_t smem = apply_smem_bytes(a, static_cast<size_t>(di.max_smem_optin));
    if (smem > static_cast<size_t>(di.max_smem_optin))
        return fail(SVDLUT_ERR_UNSUPPORTED,
                    "transform needs %zu bytes of shared memory per block (limit %d): grid vertices "
                    "too dense for a %dx%d tile or D_t/rank too large",
                    smem, di.max_smem_optin, kTileW, kTileH);
    static std::mutex mu;
    static bool attr_set[64] = {};
    {
        std::lock_guard<std::mutex> g(mu);
        if (!attr_set[di.device]) {
            SVDLUT_CUDA_TRY(cudaFuncSetAttribute(apply_kernel<T, N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 di.max_smem_optin));
            attr_set[di.device] = true;
        }
    }
    if (grid <= 0) grid = std::min(a.total_tiles, di.sm_count);
    grid = std::max(1, std::min(grid, a.total_tiles));
    apply_kernel<T, N><<<grid, kThreads, smem, s>>>(a);
    SVDLUT_CUDA_TRY(cudaGetLastError());
    return SVDLUT_OK;
}

template <int N>
svdlut_status launch_apply(LaunchArgs<N> &a, svdlut_dtype dt, cudaStream_t s, int grid)
{
    if (a.total_tiles <= 0) return SVDLUT_OK;
    return dt == SVDLUT_F32 ? launch_apply_t<float, N>(a, s, grid) : launch_apply_t<uint8_t, N>(a, s, grid);
}

}  // namespace svdlut
