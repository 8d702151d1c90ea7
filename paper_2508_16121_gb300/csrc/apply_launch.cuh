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

// Dynamic shared memory (bytes) needed for args a; sets a.lcell_floats and
// a.scratch_floats.
template <int N>
size_t apply_smem_bytes(LaunchArgs<N> &a)
{
    int Dmax = 2, pro = 0, til = 0;
    for (int i = 0; i < a.n; ++i) {
        const ImgDesc &e = a.img[i];
        Dmax = std::max(Dmax, e.D);
        pro = std::max(pro, prologue_floats(e.D, e.R));
        til = std::max(til, tile_floats(a.nvx_max, a.nvy_max, e.Dsc));
    }
    a.lcell_floats = lcell_floats(Dmax);
    a.scratch_floats = std::max(pro, til);
    return sizeof(float) * (static_cast<size_t>(a.lcell_floats) + kMiscFloats + a.scratch_floats);
}

template <typename T, int N>
svdlut_status launch_apply_t(LaunchArgs<N> &a, cudaStream_t s, int grid)
{
    DeviceInfo di;
    svdlut_status st = device_info(&di);
    if (st != SVDLUT_OK) return st;
    const size_t smem = apply_smem_bytes(a);
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
