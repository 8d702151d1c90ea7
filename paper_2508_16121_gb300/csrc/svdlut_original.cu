// The paper's original (unfused) structure, the "1x1 conv" model of Table 6,
// run on the GPU as the paper ran it: every intermediate goes through HBM.
//   1. maps_kernel   : K spatial maps f_s[k] = w_xy psi_xy + w_xc psi_xc +
//                      w_yc psi_yc + b_k (Eq. 7), written [B][K][H][W];
//   2. fusion_kernel : Xbar = 1x1 conv (K+3 -> 3) of concat(X, f_s) (Eq. 8),
//                      written [B][3][H][W];
//   3. the 2D LUT transform of Xbar (Eq. 5): apply_kernel with no grids.
// It exists to measure what the fused transform (Eq. 10) saves on this GPU
// (Sec. 3.2.3, Table 2), with results checked against the FP64 oracle.
#include <algorithm>

#include "apply_kernel.cuh"
#include "apply_launch.cuh"

namespace svdlut {
namespace {

struct MapsArgs {
    const float *x;
    const float *gxy, *gxc, *gyc, *gw;  // image 0; per-image strides below
    float *fs;
    size_t sxy, sxc, syc, sgw;
    int B, H, W, K, Dsx, Dsy, Dsc;
    float rW1, rH1;
};

// value at (da, db) of the cell whose corners are v00 = t[0], v10 = t[lda],
// v01 = t[1], v11 = t[lda + 1] (rows along a, columns along b)
__device__ __forceinline__ float bilin(const float *__restrict__ t, int lda, float da, float db)
{
    const float v00 = __ldg(t), v01 = __ldg(t + 1), v10 = __ldg(t + lda), v11 = __ldg(t + lda + 1);
    const float v0 = fmaf(v01 - v00, db, v00), v1 = fmaf(v11 - v10, db, v10);
    return fmaf(v1 - v0, da, v0);
}

// One thread per pixel (row-major over the batch, so a warp reads 32
// adjacent pixels): all K maps of the pixel.
__global__ void __launch_bounds__(256) maps_kernel(const MapsArgs a)
{
    const size_t plane = static_cast<size_t>(a.H) * a.W, n = plane * a.B;
    const float fS1 = static_cast<float>(a.Dsc - 1), fS2 = static_cast<float>(a.Dsc - 2);
    for (size_t e = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; e < n;
         e += static_cast<size_t>(gridDim.x) * blockDim.x) {
        const int b = static_cast<int>(e / plane);
        const size_t o = e - static_cast<size_t>(b) * plane;
        const int y = static_cast<int>(o / a.W), x = static_cast<int>(o - static_cast<size_t>(y) * a.W);
        const float *xb = a.x + static_cast<size_t>(b) * 3 * plane + o;
        float p[3], ec[3];
        int jc[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            p[c] = __saturatef(__ldg(xb + c * plane));
            jc[c] = cell_of(p[c], fS1, fS2, ec[c]);
        }
        int ix, iy;
        float dx, dy;
        spatial_cell(x, a.W, a.Dsx, a.rW1, ix, dx);
        spatial_cell(y, a.H, a.Dsy, a.rH1, iy, dy);
        const float *gxy = a.gxy + b * a.sxy, *gxc = a.gxc + b * a.sxc, *gyc = a.gyc + b * a.syc,
                    *gw = a.gw + b * a.sgw;
        float *fs = a.fs + static_cast<size_t>(b) * a.K * plane + o;
        for (int k = 0; k < a.K; ++k) {
            const int c = k % 3;  // grid k reads channel k mod 3 (selects, not a local-memory index)
            const int j = c == 0 ? jc[0] : (c == 1 ? jc[1] : jc[2]);
            const float e = c == 0 ? ec[0] : (c == 1 ? ec[1] : ec[2]);
            const float *w = gw + 4 * k;
            const float pxy = bilin(gxy + (static_cast<size_t>(k) * a.Dsy + iy) * a.Dsx + ix, a.Dsx, dy, dx);
            const float pxc = bilin(gxc + (static_cast<size_t>(k) * a.Dsx + ix) * a.Dsc + j, a.Dsc, dx, e);
            const float pyc = bilin(gyc + (static_cast<size_t>(k) * a.Dsy + iy) * a.Dsc + j, a.Dsc, dy, e);
            fs[k * plane] = fmaf(__ldg(w), pxy, fmaf(__ldg(w + 1), pxc, fmaf(__ldg(w + 2), pyc, __ldg(w + 3))));
        }
    }
}

// Xbar_c = bf[c] + sum_i Wf[c][i] X_i + sum_k Wf[c][3 + k] f_s[k], one thread per pixel.
__global__ void __launch_bounds__(256) fusion_kernel(const float *__restrict__ x, const float *__restrict__ fs,
                                                     const float *__restrict__ fusion, int B, int H, int W, int K,
                                                     float *__restrict__ xbar)
{
    const size_t plane = static_cast<size_t>(H) * W, n = plane * B;
    const int nf = 3 * (K + 3) + 3;
    for (size_t e = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; e < n;
         e += static_cast<size_t>(gridDim.x) * blockDim.x) {
        const int b = static_cast<int>(e / plane);
        const size_t o = e - static_cast<size_t>(b) * plane;
        const float *Wf = fusion + static_cast<size_t>(b) * nf, *bf = Wf + 3 * (K + 3);
        const float *xb = x + static_cast<size_t>(b) * 3 * plane + o;
        const float *fb = fs + static_cast<size_t>(b) * K * plane + o;
        float v[3] = {__ldg(bf), __ldg(bf + 1), __ldg(bf + 2)};
        for (int i = 0; i < 3; ++i) {
            const float xi = __ldg(xb + i * plane);
#pragma unroll
            for (int c = 0; c < 3; ++c) v[c] = fmaf(__ldg(Wf + c * (K + 3) + i), xi, v[c]);
        }
        for (int k = 0; k < K; ++k) {
            const float f = fb[k * plane];
#pragma unroll
            for (int c = 0; c < 3; ++c) v[c] = fmaf(__ldg(Wf + c * (K + 3) + 3 + k), f, v[c]);
        }
        float *ob = xbar + static_cast<size_t>(b) * 3 * plane + o;
#pragma unroll
        for (int c = 0; c < 3; ++c) ob[c * plane] = v[c];
    }
}

constexpr size_t kWsAlign = 256;

size_t align_up(size_t v) { return (v + kWsAlign - 1) / kWsAlign * kWsAlign; }

int grid_for(size_t n, int sms) { return static_cast<int>(std::min<size_t>((n + 255) / 256, static_cast<size_t>(sms) * 16)); }

}  // namespace
}  // namespace svdlut

using namespace svdlut;

extern "C" size_t svdlut_apply_original_workspace_size(const svdlut_dims *dims, int B, int H, int W)
{
    if (!dims || B < 1 || H < 1 || W < 1 || dims->K < 0) return 0;
    const size_t plane = static_cast<size_t>(H) * W * B * sizeof(float);
    return align_up(plane * dims->K) + align_up(plane * 3);
}

extern "C" svdlut_status svdlut_apply_original(const svdlut_dims *dims, const svdlut_params *params,
                                               const float *fusion, int B, int H, int W, const float *x, float *y,
                                               void *ws, size_t ws_bytes, svdlut_stream_t stream)
{
    SVDLUT_TRACE("svdlut_apply_original");
    clear_error();
    svdlut_status st = check_dims(dims);
    if (st != SVDLUT_OK) return st;
    if ((st = check_params(dims, params)) != SVDLUT_OK) return st;
    if (B < 1 || H < 1 || W < 1) return fail(SVDLUT_ERR_INVALID_ARG, "B=%d H=%d W=%d must be >= 1", B, H, W);
    if (!fusion || !x || !y) return fail(SVDLUT_ERR_INVALID_ARG, "fusion, x and y are required");
    if (!aligned(x, 4) || !aligned(y, 4) || !aligned(fusion, 4))
        return fail(SVDLUT_ERR_INVALID_ARG, "float arrays must be 4-byte aligned");
    const size_t bytes = static_cast<size_t>(B) * 3 * H * W * sizeof(float);
    const char *xs = reinterpret_cast<const char *>(x), *ys = reinterpret_cast<const char *>(y);
    if (xs < ys + bytes && ys < xs + bytes) return fail(SVDLUT_ERR_INVALID_ARG, "x and y overlap");
    if (!ws || ws_bytes < svdlut_apply_original_workspace_size(dims, B, H, W))
        return fail(SVDLUT_ERR_WORKSPACE, "workspace of %zu bytes needed",
                    svdlut_apply_original_workspace_size(dims, B, H, W));
    if (!aligned(ws, kWsAlign)) return fail(SVDLUT_ERR_INVALID_ARG, "workspace must be %zu-byte aligned", kWsAlign);

    DeviceInfo di;
    if ((st = device_info(&di)) != SVDLUT_OK) return st;
    const cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const size_t plane = static_cast<size_t>(H) * W;
    float *fs = static_cast<float *>(ws);
    float *xbar = reinterpret_cast<float *>(static_cast<char *>(ws) + align_up(plane * B * dims->K * sizeof(float)));
    const size_t n = plane * B;
    const int K = dims->K;
    if (K > 0) {
        MapsArgs a{};
        a.x = x;
        a.gxy = params->g_xy;
        a.gxc = params->g_xc;
        a.gyc = params->g_yc;
        a.gw = params->grid_w;
        a.fs = fs;
        a.sxy = param_stride(dims, 4);
        a.sxc = param_stride(dims, 5);
        a.syc = param_stride(dims, 6);
        a.sgw = param_stride(dims, 7);
        a.B = B;
        a.H = H;
        a.W = W;
        a.K = K;
        a.Dsx = dims->Dsx;
        a.Dsy = dims->Dsy;
        a.Dsc = dims->Dsc;
        a.rW1 = W > 1 ? 1.0f / static_cast<float>(W - 1) : 0.f;
        a.rH1 = H > 1 ? 1.0f / static_cast<float>(H - 1) : 0.f;
        maps_kernel<<<grid_for(n, di.sm_count), 256, 0, s>>>(a);
        SVDLUT_CUDA_TRY(cudaGetLastError());
    }
    fusion_kernel<<<grid_for(n, di.sm_count), 256, 0, s>>>(x, fs, fusion, B, H, W, K, xbar);
    SVDLUT_CUDA_TRY(cudaGetLastError());
    // LUT transform of Xbar: the fused kernel with no grids
    svdlut_dims d0 = *dims;
    d0.K = 0;
    svdlut_params p0 = *params;
    p0.g_xy = p0.g_xc = p0.g_yc = p0.grid_w = nullptr;
    for (int b0 = 0; b0 < B; b0 += kPlainChunk) {
        LaunchArgs<kPlainChunk> la{};
        la.n = std::min(kPlainChunk, B - b0);
        for (int i = 0; i < la.n; ++i) la.img[i] = make_desc(&d0, &p0, b0 + i, H, W, SVDLUT_F32, xbar, y);
        size_t smem = 0;
        if ((st = plan_uniform(la, di.sm_count, static_cast<size_t>(di.max_smem_optin), &smem)) != SVDLUT_OK)
            return st;
        if ((st = launch_apply(la, smem, SVDLUT_F32, s, 0)) != SVDLUT_OK) return st;
    }
    return SVDLUT_OK;
}
