// The 3D LUT the paper starts from (Eq. 3) and the test of its hypothesis
// that a sum of 2D LUTs can replace it (Eq. 4):
//  - svdlut_lut3d_apply: trilinear transform of images by per-image 3D LUTs;
//    the tables are repacked to one float4 (r, g, b, pad) per vertex, so a
//    pixel's 8 corners are 8 16-byte gathers through L1/L2 (a 33^3 table is
//    575 KB per channel triple: too large for shared memory);
//  - svdlut_lut3d_fit2d: the least-squares fit of each 3D table by
//    A[i][j] + B[i][k] + C[j][k] on the vertex grid, which is the
//    second-order ANOVA projection fit = m_ij. + m_i.k + m_.jk - m_i.. -
//    m_.j. - m_..k + m_... (m: means over the dotted indices), one CTA per
//    table with the table in shared memory.
#include <algorithm>

#include "apply_kernel.cuh"
#include "apply_launch.cuh"

namespace svdlut {
namespace {

// planar [B][3][D^3] -> packed [B][D^3] float4 (r, g, b, 0)
__global__ void lut3d_pack_kernel(const float *__restrict__ planar, int B, int n3, float4 *__restrict__ packed)
{
    const size_t n = static_cast<size_t>(B) * n3;
    for (size_t e = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; e < n;
         e += static_cast<size_t>(gridDim.x) * blockDim.x) {
        const size_t b = e / n3, v = e - b * n3;
        const float *p = planar + b * 3 * static_cast<size_t>(n3) + v;
        packed[e] = make_float4(__ldg(p), __ldg(p + n3), __ldg(p + 2 * static_cast<size_t>(n3)), 0.f);
    }
}

__device__ __forceinline__ float4 lerp4(const float4 a, const float4 b, float t)
{
    return make_float4(fmaf(b.x - a.x, t, a.x), fmaf(b.y - a.y, t, a.y), fmaf(b.z - a.z, t, a.z), 0.f);
}

// One thread per pixel, row-major over the batch.
__global__ void __launch_bounds__(256) lut3d_apply_kernel(const float4 *__restrict__ lut, int D, int B, int H, int W,
                                                          const float *__restrict__ x, float *__restrict__ y)
{
    const size_t plane = static_cast<size_t>(H) * W, n = plane * B, n3 = static_cast<size_t>(D) * D * D;
    const float fD1 = static_cast<float>(D - 1), fD2 = static_cast<float>(D - 2);
    for (size_t e = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; e < n;
         e += static_cast<size_t>(gridDim.x) * blockDim.x) {
        const size_t b = e / plane, o = e - b * plane;
        const float *xb = x + b * 3 * plane + o;
        float fr, fg, fb;
        const int ir = cell_of(__saturatef(__ldcs(xb)), fD1, fD2, fr);
        const int ig = cell_of(__saturatef(__ldcs(xb + plane)), fD1, fD2, fg);
        const int ib = cell_of(__saturatef(__ldcs(xb + 2 * plane)), fD1, fD2, fb);
        const float4 *t = lut + b * n3 + (static_cast<size_t>(ir) * D + ig) * D + ib;
        const size_t sr = static_cast<size_t>(D) * D, sg = D;
        const float4 c000 = __ldg(t), c001 = __ldg(t + 1), c010 = __ldg(t + sg), c011 = __ldg(t + sg + 1);
        const float4 c100 = __ldg(t + sr), c101 = __ldg(t + sr + 1), c110 = __ldg(t + sr + sg),
                     c111 = __ldg(t + sr + sg + 1);
        const float4 c00 = lerp4(c000, c001, fb), c01 = lerp4(c010, c011, fb);
        const float4 c10 = lerp4(c100, c101, fb), c11 = lerp4(c110, c111, fb);
        const float4 v = lerp4(lerp4(c00, c01, fg), lerp4(c10, c11, fg), fr);
        float *yb = y + b * 3 * plane + o;
        __stcs(yb, v.x);
        __stcs(yb + plane, v.y);
        __stcs(yb + 2 * plane, v.z);
    }
}

// One CTA per (image, channel) table.  Shared memory: the D^3 table, then
// the marginal means m_ij, m_ik, m_jk [D][D] and m_i, m_j, m_k [D], then one
// partial sum per warp (no static shared memory, so the dynamic part may take
// the whole opt-in limit).
constexpr int kFitThreads = 512;

__global__ void __launch_bounds__(kFitThreads) lut3d_fit2d_kernel(const float *__restrict__ planar, int D,
                                                                 float *__restrict__ tables, float *__restrict__ rms)
{
    extern __shared__ __align__(16) float sm[];
    const int tb = blockIdx.x;  // b * 3 + c
    const int n2 = D * D, n3 = n2 * D;
    float *t = sm, *mij = t + n3, *mik = mij + n2, *mjk = mik + n2, *mi = mjk + n2, *mj = mi + D, *mk = mj + D,
          *red = mk + D;
    const float *src = planar + static_cast<size_t>(tb) * n3;
    for (int e = threadIdx.x; e < n3; e += kFitThreads) t[e] = __ldg(src + e);
    __syncthreads();
    const float inv = 1.0f / static_cast<float>(D);
    // two-index means: each thread sums one line of D values in order
    for (int e = threadIdx.x; e < 3 * n2; e += kFitThreads) {
        const int which = e / n2, a = (e - which * n2) / D, b = e - which * n2 - a * D;
        float s = 0.f;
        if (which == 0)
            for (int k = 0; k < D; ++k) s += t[(a * D + b) * D + k];  // m_ij
        else if (which == 1)
            for (int j = 0; j < D; ++j) s += t[(a * D + j) * D + b];  // m_ik
        else
            for (int i = 0; i < D; ++i) s += t[(i * D + a) * D + b];  // m_jk
        (which == 0 ? mij : (which == 1 ? mik : mjk))[a * D + b] = s * inv;
    }
    __syncthreads();
    // one-index means from the two-index ones
    for (int e = threadIdx.x; e < 3 * D; e += kFitThreads) {
        const int which = e / D, a = e - which * D;
        float s = 0.f;
        if (which == 0)
            for (int j = 0; j < D; ++j) s += mij[a * D + j];  // m_i
        else if (which == 1)
            for (int i = 0; i < D; ++i) s += mij[i * D + a];  // m_j
        else
            for (int i = 0; i < D; ++i) s += mik[i * D + a];  // m_k
        (which == 0 ? mi : (which == 1 ? mj : mk))[a] = s * inv;
    }
    __syncthreads();
    float m = 0.f;
    for (int i = 0; i < D; ++i) m += mi[i];
    m *= inv;
    // tables in the svdlut U layout for rank D: [c][pair rg, rb, gb][D][D]
    float *A = tables + static_cast<size_t>(tb) * 3 * n2, *Bt = A + n2, *C = Bt + n2;
    for (int e = threadIdx.x; e < n2; e += kFitThreads) {
        const int a = e / D, b = e - a * D;
        A[e] = mij[e];
        Bt[e] = mik[e] - mi[a];
        C[e] = mjk[e] - mj[a] - mk[b] + m;
    }
    // residual: the three-way interaction
    float ss = 0.f;
    for (int e = threadIdx.x; e < n3; e += kFitThreads) {
        const int i = e / n2, j = (e - i * n2) / D, k = e - i * n2 - j * D;
        const float r = t[e] - (mij[i * D + j] + (mik[i * D + k] - mi[i]) + (mjk[j * D + k] - mj[j] - mk[k] + m));
        ss = fmaf(r, r, ss);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = ss;
    __syncthreads();
    if (threadIdx.x == 0) {
        float s = 0.f;
        for (int w = 0; w < kFitThreads / 32; ++w) s += red[w];
        rms[tb] = sqrtf(s / static_cast<float>(n3));
    }
}

int grid_for(size_t n, int sms) { return static_cast<int>(std::min<size_t>((n + 255) / 256, static_cast<size_t>(sms) * 16)); }

}  // namespace
}  // namespace svdlut

using namespace svdlut;

extern "C" size_t svdlut_lut3d_workspace_size(int D, int B)
{
    if (D < 2 || B < 1) return 0;
    return static_cast<size_t>(B) * D * D * D * sizeof(float4);
}

extern "C" svdlut_status svdlut_lut3d_apply(int D, const float *lut3d, int B, int H, int W, const float *x, float *y,
                                            void *ws, size_t ws_bytes, svdlut_stream_t stream)
{
    SVDLUT_TRACE("svdlut_lut3d_apply");
    clear_error();
    if (D < 2 || D > kMaxDt) return fail(SVDLUT_ERR_INVALID_ARG, "D=%d out of [2, %d]", D, kMaxDt);
    if (B < 1 || H < 1 || W < 1) return fail(SVDLUT_ERR_INVALID_ARG, "B=%d H=%d W=%d must be >= 1", B, H, W);
    if (!lut3d || !x || !y) return fail(SVDLUT_ERR_INVALID_ARG, "lut3d, x and y are required");
    if (!ws || ws_bytes < svdlut_lut3d_workspace_size(D, B))
        return fail(SVDLUT_ERR_WORKSPACE, "workspace of %zu bytes needed", svdlut_lut3d_workspace_size(D, B));
    if (!aligned(ws, 16) || !aligned(x, 4) || !aligned(y, 4) || !aligned(lut3d, 4))
        return fail(SVDLUT_ERR_INVALID_ARG, "misaligned pointer (workspace: 16 bytes, arrays: 4)");
    DeviceInfo di;
    svdlut_status st = device_info(&di);
    if (st != SVDLUT_OK) return st;
    const cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const int n3 = D * D * D;
    float4 *packed = static_cast<float4 *>(ws);
    lut3d_pack_kernel<<<grid_for(static_cast<size_t>(B) * n3, di.sm_count), 256, 0, s>>>(lut3d, B, n3, packed);
    SVDLUT_CUDA_TRY(cudaGetLastError());
    lut3d_apply_kernel<<<grid_for(static_cast<size_t>(B) * H * W, di.sm_count), 256, 0, s>>>(packed, D, B, H, W, x, y);
    SVDLUT_CUDA_TRY(cudaGetLastError());
    return SVDLUT_OK;
}

extern "C" svdlut_status svdlut_lut3d_fit2d(int D, const float *lut3d, int B, float *tables, float *rms,
                                            svdlut_stream_t stream)
{
    SVDLUT_TRACE("svdlut_lut3d_fit2d");
    clear_error();
    if (D < 2 || D > kMaxDt) return fail(SVDLUT_ERR_INVALID_ARG, "D=%d out of [2, %d]", D, kMaxDt);
    if (B < 1) return fail(SVDLUT_ERR_INVALID_ARG, "B=%d must be >= 1", B);
    if (!lut3d || !tables || !rms) return fail(SVDLUT_ERR_INVALID_ARG, "lut3d, tables and rms are required");
    DeviceInfo di;
    svdlut_status st = device_info(&di);
    if (st != SVDLUT_OK) return st;
    const size_t smem = sizeof(float) * (static_cast<size_t>(D) * D * D + 3 * D * D + 3 * D + kFitThreads / 32);
    if (smem > static_cast<size_t>(di.max_smem_optin)) return fail(SVDLUT_ERR_UNSUPPORTED, "D=%d too large", D);
    if ((st = allow_smem_once(reinterpret_cast<const void *>(lut3d_fit2d_kernel), di.max_smem_optin, di.device)) !=
        SVDLUT_OK)
        return st;
    lut3d_fit2d_kernel<<<3 * B, kFitThreads, smem, reinterpret_cast<cudaStream_t>(stream)>>>(lut3d, D, tables, rms);
    SVDLUT_CUDA_TRY(cudaGetLastError());
    return SVDLUT_OK;
}
