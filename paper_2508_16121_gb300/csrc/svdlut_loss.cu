// svdlut_cie94: the colour-difference term of the training loss (Eq. 11,
// weight lambda_c = 0.005): the mean over pixels of the CIE94 difference
// between the prediction and the ground truth in CIELAB, and its gradient
// with respect to the prediction, in one pass over the two images.
//
// Per pixel: sRGB decoding (IEC 61966-2-1) of the raw values, XYZ by the
// matrix derived on the host from the sRGB primaries' and D65's
// chromaticities, CIELAB relative to that white, CIE94 with the graphic-arts
// weights and the ground truth as the reference, Delta H^2 clamped at 0.
// u^2.4 is taken as exp2(2.4 log2 u) through log2f and exp2f, fewer
// instructions than powf.  The gradient walks the same steps backwards,
// reusing the forward values (d lin / dc = (2.4 / 1.055) exp2(1.4 log2 u);
// for f = cbrt(t), f' = 1 / (3 f^2)), with fast reciprocals; it is 0 where
// Delta E = 0.  The sum is reduced per block and then over blocks in a fixed
// order (deterministic).
#include <algorithm>
#include <atomic>
#include <cmath>

#include "svdlut_internal.cuh"

namespace svdlut {
namespace {

constexpr int kLossThreads = 256;
constexpr float kEps = 216.0f / 24389.0f, kKappa = 24389.0f / 27.0f, kK1 = 0.045f, kK2 = 0.015f;

struct ColourConsts {
    float M[9];    // linear sRGB -> XYZ, row-major
    float inv_n[3];  // 1 / white (Xn, Yn, Zn)
};

// M = P diag(s) with P's columns the XYZ (Y = 1) of the primaries and
// P s = the white's XYZ: the standard derivation from chromaticities.
ColourConsts colour_consts()
{
    const double prim[3][2] = {{0.64, 0.33}, {0.30, 0.60}, {0.15, 0.06}}, wxy[2] = {0.3127, 0.3290};
    double P[3][3], w[3] = {wxy[0] / wxy[1], 1.0, (1.0 - wxy[0] - wxy[1]) / wxy[1]};
    for (int j = 0; j < 3; ++j) {
        const double x = prim[j][0], y = prim[j][1];
        P[0][j] = x / y;
        P[1][j] = 1.0;
        P[2][j] = (1.0 - x - y) / y;
    }
    // s = P^-1 w by Cramer's rule
    auto det3 = [](const double A[3][3]) {
        return A[0][0] * (A[1][1] * A[2][2] - A[1][2] * A[2][1]) - A[0][1] * (A[1][0] * A[2][2] - A[1][2] * A[2][0]) +
               A[0][2] * (A[1][0] * A[2][1] - A[1][1] * A[2][0]);
    };
    const double dP = det3(P);
    double s[3];
    for (int j = 0; j < 3; ++j) {
        double A[3][3];
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c) A[r][c] = c == j ? w[r] : P[r][c];
        s[j] = det3(A) / dP;
    }
    ColourConsts k{};
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) k.M[3 * r + c] = static_cast<float>(P[r][c] * s[c]);
    for (int r = 0; r < 3; ++r) k.inv_n[r] = static_cast<float>(1.0 / w[r]);
    return k;
}

struct LabFwd {
    float lin[3], lu[3];  // decoded values; log2 u (u = (c + 0.055) / 1.055) on the power branch
    bool pw[3];           // power branch taken
    float t[3], f[3];     // XYZ / white and f(t)
    float L, a, b;
};

__device__ __forceinline__ void lab_of(const float c[3], const ColourConsts &k, LabFwd &o)
{
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        o.pw[i] = c[i] > 0.04045f;
        o.lu[i] = o.pw[i] ? log2f((c[i] + 0.055f) * (1.0f / 1.055f)) : 0.f;
        o.lin[i] = o.pw[i] ? exp2f(2.4f * o.lu[i]) : c[i] * (1.0f / 12.92f);
    }
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        const float X = fmaf(k.M[3 * r], o.lin[0], fmaf(k.M[3 * r + 1], o.lin[1], k.M[3 * r + 2] * o.lin[2]));
        o.t[r] = X * k.inv_n[r];
        o.f[r] = o.t[r] > kEps ? cbrtf(o.t[r]) : fmaf(kKappa, o.t[r], 16.0f) * (1.0f / 116.0f);
    }
    o.L = fmaf(116.0f, o.f[1], -16.0f);
    o.a = 500.0f * (o.f[0] - o.f[1]);
    o.b = 200.0f * (o.f[1] - o.f[2]);
}

__device__ __forceinline__ float block_sum(float v, float *red)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    float s = 0.f;
    if (threadIdx.x == 0)
        for (int w = 0; w < kLossThreads / 32; ++w) s += red[w];
    return s;
}

__global__ void __launch_bounds__(kLossThreads) cie94_kernel(const float *__restrict__ y, const float *__restrict__ t,
                                                             int B, size_t plane, float gscale, float *__restrict__ dy,
                                                             int accumulate, const ColourConsts k,
                                                             float *__restrict__ part)
{
    __shared__ float red[kLossThreads / 32];
    const size_t n = plane * B;
    float sum = 0.f;
    for (size_t e = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; e < n;
         e += static_cast<size_t>(gridDim.x) * blockDim.x) {
        const size_t b = e / plane, o = e - b * plane, base = b * 3 * plane + o;
        const float cy[3] = {__ldcs(y + base), __ldcs(y + base + plane), __ldcs(y + base + 2 * plane)};
        const float ct[3] = {__ldcs(t + base), __ldcs(t + base + plane), __ldcs(t + base + 2 * plane)};
        LabFwd P, R;  // prediction, reference (ground truth)
        lab_of(cy, k, P);
        lab_of(ct, k, R);
        const float C1 = sqrtf(fmaf(R.a, R.a, R.b * R.b)), C2 = sqrtf(fmaf(P.a, P.a, P.b * P.b));
        const float dL = R.L - P.L, dC = C1 - C2, da = R.a - P.a, db = R.b - P.b;
        const float dH2raw = fmaf(da, da, fmaf(db, db, -dC * dC));
        const float SC = fmaf(kK1, C1, 1.0f), SH = fmaf(kK2, C1, 1.0f);
        const float iSC2 = __frcp_rn(SC * SC), iSH2 = __frcp_rn(SH * SH);
        const float Q = fmaf(dL, dL, fmaf(dC * dC, iSC2, fmaxf(dH2raw, 0.f) * iSH2));
        const float dE = sqrtf(Q);
        sum += dE;
        if (!dy) continue;
        float g[3] = {0.f, 0.f, 0.f};
        if (dE > 0.f) {
            const float sc = gscale * 0.5f * rsqrtf(Q);
            const float iC2 = C2 > 0.f ? __fdividef(1.0f, C2) : 0.f;
            const float ua = P.a * iC2, ub = P.b * iC2;
            const float hon = dH2raw > 0.f ? iSH2 : 0.f;
            const float gL = -2.0f * dL * sc;
            const float ga = (-2.0f * dC * ua * iSC2 + hon * (2.0f * dC * ua - 2.0f * da)) * sc;
            const float gb = (-2.0f * dC * ub * iSC2 + hon * (2.0f * dC * ub - 2.0f * db)) * sc;
            const float gf[3] = {500.0f * ga, fmaf(116.0f, gL, fmaf(-500.0f, ga, 200.0f * gb)), -200.0f * gb};
            float gx[3];
#pragma unroll
            for (int r = 0; r < 3; ++r) {
                const float dfdt = P.t[r] > kEps ? __fdividef(1.0f, 3.0f * P.f[r] * P.f[r]) : kKappa * (1.0f / 116.0f);
                gx[r] = gf[r] * dfdt * k.inv_n[r];
            }
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const float gl = fmaf(k.M[c], gx[0], fmaf(k.M[3 + c], gx[1], k.M[6 + c] * gx[2]));
                const float dl = P.pw[c] ? (2.4f / 1.055f) * exp2f(1.4f * P.lu[c]) : 1.0f / 12.92f;
                g[c] = gl * dl;
            }
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            float *q = dy + base + c * plane;
            *q = accumulate ? *q + g[c] : g[c];
        }
    }
    const float tot = block_sum(sum, red);
    if (threadIdx.x == 0) part[blockIdx.x] = tot;
}

__global__ void mean_final_kernel(const float *part, int nb, size_t n, float *loss)
{
    const int lane = threadIdx.x & 31;
    double s = 0.0;
    for (int i = lane; i < nb; i += 32) s += part[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) *loss = static_cast<float>(s / static_cast<double>(n));
}

constexpr int kMaxBlocks = 1024;

}  // namespace
}  // namespace svdlut

using namespace svdlut;

extern "C" svdlut_status svdlut_cie94(const float *y, const float *target, int B, int H, int W, float weight,
                                      float *dy, int accumulate, float *loss, void *ws, size_t ws_bytes,
                                      svdlut_stream_t stream)
{
    SVDLUT_TRACE("svdlut_cie94");
    clear_error();
    if (!y || !target || !loss) return fail(SVDLUT_ERR_INVALID_ARG, "cie94: y, target and loss are required");
    if (B < 1 || H < 1 || W < 1) return fail(SVDLUT_ERR_INVALID_ARG, "B=%d H=%d W=%d must be >= 1", B, H, W);
    if (!aligned(y, 4) || !aligned(target, 4) || (dy && !aligned(dy, 4)) || !aligned(loss, 4))
        return fail(SVDLUT_ERR_INVALID_ARG, "float arrays must be 4-byte aligned");
    if (!ws || ws_bytes < sizeof(float) * kMaxBlocks)
        return fail(SVDLUT_ERR_WORKSPACE, "cie94: workspace of %zu bytes needed", sizeof(float) * kMaxBlocks);
    DeviceInfo di;
    svdlut_status st = device_info(&di);
    if (st != SVDLUT_OK) return st;
    static const ColourConsts k = colour_consts();
    const size_t plane = static_cast<size_t>(H) * W, n = plane * B;
    // one resident wave: as many blocks per SM as the registers allow
    static std::atomic<int> cached_per_sm{0};
    int per_sm = cached_per_sm.load();
    if (per_sm == 0) {
        SVDLUT_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, cie94_kernel, kLossThreads, 0));
        per_sm = std::max(per_sm, 1);
        cached_per_sm.store(per_sm);
    }
    const int nb = static_cast<int>(std::min<size_t>((n + kLossThreads - 1) / kLossThreads,
                                                     std::min<size_t>(kMaxBlocks, static_cast<size_t>(di.sm_count) * per_sm)));
    const cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    float *part = static_cast<float *>(ws);
    cie94_kernel<<<nb, kLossThreads, 0, s>>>(y, target, B, plane, weight / static_cast<float>(n), dy, accumulate, k,
                                             part);
    SVDLUT_CUDA_TRY(cudaGetLastError());
    mean_final_kernel<<<1, 32, 0, s>>>(part, nb, n, loss);
    SVDLUT_CUDA_TRY(cudaGetLastError());
    return SVDLUT_OK;
}
