// The learned factor generator (Supp. Sec. A, Tables 8-12) on sm_103a: a
// bilinear 256x256 thumbnail, five 3x3 stride-2 convolutions (BF16 tensor-core
// implicit GEMMs, FP32 accumulation) with LeakyReLU and InstanceNorm, average
// pooling to a 256-d context and four two-layer FC heads that emit the SVD
// factors, LUT weights, 2D bilateral grids and grid weights in the layouts
// svdlut_apply reads.  Forward, backward and an Adam step; every reduction is
// done in a fixed order (no atomics), so training is bitwise repeatable.
#include <cuda_bf16.h>

#include <algorithm>
#include <atomic>
#include <vector>
#include <utility>
#include <mutex>
#include <cstdint>

#include "svdlut_internal.cuh"

namespace svdlut {
namespace gen {

constexpr int kCh[6] = {3, 8, 16, 32, 64, 64};
constexpr int kSz[6] = {256, 128, 64, 32, 16, 8};  // spatial size of the input of conv i / output of conv i-1
constexpr int kThumb = 256;
constexpr float kSlope = 0.2f;
constexpr float kEps = 1e-5f;
constexpr int kDT = 33, kNS = 8, kDS = 17, kHidden = 8, kRho = 256;

struct Layout {
    size_t conv_w[5], conv_b[5], in_g[4], in_b[4];
    size_t w1[4], b1[4], w2[4], b2[4];
    int head_n[4];
    size_t total;
};

__host__ __device__ inline int head_n(int K, int h)
{
    return h == 0 ? K * 3 * kDS * kDS : (h == 1 ? K * 4 : (h == 2 ? 9 * (kDT * kNS + kNS + kDT * kNS) : 12));
}

inline Layout make_layout(int K)
{
    Layout L{};
    size_t o = 0;
    for (int i = 0; i < 5; ++i) {
        L.conv_w[i] = o;
        o += static_cast<size_t>(kCh[i + 1]) * kCh[i] * 9;
        L.conv_b[i] = o;
        o += kCh[i + 1];
        if (i < 4) {
            L.in_g[i] = o;
            o += kCh[i + 1];
            L.in_b[i] = o;
            o += kCh[i + 1];
        }
    }
    for (int h = 0; h < 4; ++h) {
        L.head_n[h] = head_n(K, h);
        L.w1[h] = o;
        o += static_cast<size_t>(kHidden) * kRho;
        L.b1[h] = o;
        o += kHidden;
        L.w2[h] = o;
        o += static_cast<size_t>(L.head_n[h]) * kHidden;
        L.b2[h] = o;
        o += L.head_n[h];
    }
    L.total = o;
    return L;
}

// Workspace (floats): forward activations kept for the backward pass, then
// backward temporaries.  InstanceNorm is not materialised: the layer after it
// reads r[i] and applies the per-(b, c) affine map sc * r + sh on load.
struct WsLayout {
    size_t thumb, r[5], mean[4], rstd[4], sc[4], sh[4], part, wbf[5], tstat, dgw[5], rho, hidden;
    size_t dz[2], dact, wpart, dhid, drho, insum;
    size_t total;
};


inline size_t act_size(int B, int i) { return static_cast<size_t>(B) * kCh[i + 1] * kSz[i + 1] * kSz[i + 1]; }

// Weight gradient of conv i (wgrad_kernel): tiles of 126 im2col columns
// (with the bias column) and N = output channels padded to 16, 32 or 64; a
// layer with at most 32 columns (the first) packs four pixel subsets into one
// MMA instead (wgrad_sets = 4, N = 4 Cout).  The batch's output pixels are cut
// into chunks of wgrad_chunk_px pixels (whole stages of 64 x sets pixels) so
// that tiles x chunks fill the resident CTAs of one wave on 152 SMs (a fixed
// split: the summation order, hence the result, does not depend on the
// device); the partials of chunk z and subset r are chunk sets z + r.
inline int wgrad_np(int Cout) { return Cout <= 16 ? 16 : Cout <= 32 ? 32 : 64; }
inline int wgrad_sets(int i) { return kCh[i] * 9 + 1 <= 32 && 4 * kCh[i + 1] <= 64 ? 4 : 1; }
inline int wgrad_np_layer(int i) { return wgrad_np(wgrad_sets(i) * kCh[i + 1]); }
inline int wgrad_tiles(int i) { return wgrad_sets(i) > 1 ? 1 : (kCh[i] * 9 + 1 + 125) / 126; }
inline int wgrad_chunk_px(int B, int i)
{
    const int pix = B * kSz[i + 1] * kSz[i + 1], st = 64 * wgrad_sets(i);
    const int ctas = (wgrad_np_layer(i) == 16 && wgrad_sets(i) == 1 ? 3 : 2) * 152;  // resident CTAs x SMs
    const int want = std::max(1, (ctas + wgrad_tiles(i) - 1) / wgrad_tiles(i));
    const int px = (pix + want - 1) / want;
    return std::max(st, (px + st - 1) / st * st);
}
inline int wgrad_chunks(int B, int i)
{
    const int pix = B * kSz[i + 1] * kSz[i + 1], c = wgrad_chunk_px(B, i);
    return (pix + c - 1) / c;
}

// Forward conv i (conv_umma_kernel): K = 9 Cin in stages of 64 (kWK); the
// CTAs are (128-pixel tile, K split).  Layers with fewer than two tiles per
// SM split K so that tiles x splits give about four CTAs per SM; ks = stages
// per split.  (Fixed numbers, not the device's: the summation order, hence
// the result, does not depend on the GPU.)
inline int conv_stages(int i) { return (kCh[i] * 9 + 63) / 64; }
inline int conv_ks(int B, int i)
{
    const int tiles = (B * kSz[i + 1] * kSz[i + 1] + 127) / 128, nst = conv_stages(i);
    if (tiles >= 2 * 152) return nst;
    const int want = (4 * 152 + tiles - 1) / tiles;
    return std::max(1, (nst + want - 1) / want);
}
inline int conv_split(int B, int i) { return (conv_stages(i) + conv_ks(B, i) - 1) / conv_ks(B, i); }
// BF16 elements of conv i's weights in the B layout (NP x whole stages)
inline size_t conv_wbf_elems(int i) { return static_cast<size_t>(wgrad_np(kCh[i + 1])) * conv_stages(i) * 64; }
// Input gradient of conv i >= 1 (dgrad_umma_kernel): per parity class cls =
// 2 py + px, K = (1 + py)(1 + px) Cout, padded to whole 64-k stages; the
// class's split weights take 2 NP Kpad BF16 elements (hi, then lo).
inline int dgrad_kpad(int i, int cls) { return ((1 + (cls >> 1)) * (1 + (cls & 1)) * kCh[i + 1] + 63) / 64 * 64; }
inline size_t dgrad_w_elems(int i)
{
    size_t n = 0;
    for (int c = 0; c < 4; ++c) n += static_cast<size_t>(2) * wgrad_np(kCh[i]) * dgrad_kpad(i, c);
    return n;
}

inline WsLayout make_ws(int B)
{
    WsLayout w{};
    size_t o = 0;
    auto take = [&](size_t n) {
        const size_t at = o;
        o += (n + 63) & ~static_cast<size_t>(63);
        return at;
    };
    w.thumb = take(static_cast<size_t>(B) * 3 * kThumb * kThumb);
    for (int i = 0; i < 5; ++i) w.r[i] = take(act_size(B, i));
    for (int i = 0; i < 4; ++i) {
        w.mean[i] = take(static_cast<size_t>(B) * kCh[i + 1]);
        w.rstd[i] = take(static_cast<size_t>(B) * kCh[i + 1]);
        w.sc[i] = take(static_cast<size_t>(B) * kCh[i + 1]);
        w.sh[i] = take(static_cast<size_t>(B) * kCh[i + 1]);
    }
    size_t pp = 0;
    for (int i = 0; i < 5; ++i) pp = std::max(pp, static_cast<size_t>(conv_split(B, i)) * act_size(B, i));
    w.part = take(pp);
    for (int i = 0; i < 5; ++i) w.wbf[i] = take((conv_wbf_elems(i) + 1) / 2);
    size_t ts = 0;  // per-tile statistics of the layers with the fused finish
    for (int i = 0; i < 4; ++i)
        ts = std::max(ts, static_cast<size_t>((B * kSz[i + 1] * kSz[i + 1] + 127) / 128) * kCh[i + 1] * 2);
    w.tstat = take(ts);
    for (int i = 1; i < 5; ++i) w.dgw[i] = take(dgrad_w_elems(i) / 2);
    w.rho = take(static_cast<size_t>(B) * kRho);
    w.hidden = take(static_cast<size_t>(B) * 4 * kHidden);
    const size_t amax = act_size(B, 0);
    w.dz[0] = take(amax);
    w.dz[1] = take(amax);
    w.dact = take(amax);
    size_t wp = 0;
    for (int i = 0; i < 5; ++i) {
        wp = std::max(wp, static_cast<size_t>(wgrad_chunks(B, i)) * wgrad_sets(i) * kCh[i + 1] * (kCh[i] * 9 + 1));
    }
    w.wpart = take(wp);
    w.dhid = take(static_cast<size_t>(B) * 4 * kHidden);
    w.drho = take(static_cast<size_t>(B) * kRho);
    w.insum = take(static_cast<size_t>(B) * 64 * 2);
    w.total = o;
    return w;
}

// ---------------------------------------------------------------- kernels

// Bilinear downsample to 256x256 with half-pixel centres, no antialiasing.
__global__ void downsample_kernel(const float *__restrict__ x, int B, int H, int W, float *__restrict__ t)
{
    static_assert(kThumb % 4 == 0, "four outputs of one thumbnail row per thread");
    pdl_enter();
    const size_t n4 = static_cast<size_t>(B) * 3 * kThumb * kThumb / 4;
    const float sy_ = static_cast<float>(H) / kThumb, sx_ = static_cast<float>(W) / kThumb;
    for (size_t e4 = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; e4 < n4;
         e4 += static_cast<size_t>(gridDim.x) * blockDim.x) {
        const size_t e = 4 * e4;
        const int ox0 = static_cast<int>(e % kThumb), oy = static_cast<int>((e / kThumb) % kThumb);
        const size_t bc = e / (kThumb * kThumb);
        const float sy = fminf(fmaxf((oy + 0.5f) * sy_ - 0.5f, 0.f), static_cast<float>(H - 1));
        const int y0 = static_cast<int>(sy), y1 = min(y0 + 1, H - 1);
        const float fy = sy - y0;
        const float *r0 = x + (bc * H + y0) * W, *r1 = x + (bc * H + y1) * W;
        float v[4][4], fx[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {  // every load of the four outputs first
            const float sx = fminf(fmaxf((ox0 + u + 0.5f) * sx_ - 0.5f, 0.f), static_cast<float>(W - 1));
            const int x0 = static_cast<int>(sx), x1 = min(x0 + 1, W - 1);
            fx[u] = sx - x0;
            v[u][0] = __ldg(r0 + x0);
            v[u][1] = __ldg(r0 + x1);
            v[u][2] = __ldg(r1 + x0);
            v[u][3] = __ldg(r1 + x1);
        }
        float o[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const float top = (1.f - fx[u]) * v[u][0] + fx[u] * v[u][1];
            const float bot = (1.f - fx[u]) * v[u][2] + fx[u] * v[u][3];
            o[u] = (1.f - fy) * top + fy * bot;
        }
        *reinterpret_cast<float4 *>(t + e) = make_float4(o[0], o[1], o[2], o[3]);
    }
}

// ---- weight gradients of the stride-2 pad-1 3x3 convolutions on tcgen05 ----
// dW[o][j] = sum over the batch's output pixels p of dz[o][p] im2col[p][j],
// j = (c, ky, kx) < Kd = 9 Cin, and the bias gradient as column j = Kd (an
// all-ones im2col column).  A CTA takes one tile of kWRows = 126 columns j
// (blockIdx.x: 42 whole (c, ky) groups, so the three kx of a group never
// straddle two tiles) and one chunk of pixels (blockIdx.y), and writes that
// chunk's partial [Cout][Kd + 1] slice; wgrad_reduce_kernel sums the chunks
// in a fixed order.  The columns j are the MMA's M = 128 rows (TMEM lanes),
// the output channels its N = NP >= Cout columns, the pixels its K: per
// stage of kWK = 64 pixels both operands are staged K-major in shared memory
// (two stages in flight) as BF16 hi and lo parts, and one thread issues
// lo*hi + hi*lo + hi*hi (three kind::f16 MMAs per 16-wide K step, about 16
// mantissa bits: the gradient sums are long chains of cancelling terms) into
// FP32 accumulators in TMEM.  Shared-memory layout: no swizzle, core
// matrices of 8 rows x 16 bytes; element (r, k) of an R-row operand sits at
// byte (k / 8) * 16 R + 16 r + 2 (k % 8), so the 8 pixels of one octet of
// one row are a single 16-byte store, and a warp's stores of consecutive
// rows are free of bank conflicts.  Staging tasks: an A task is one (c, ky)
// group x one pixel octet, the 16 input values of one input row under it
// (four float4 loads; 2 ox0 is a multiple of 16) and its left neighbour,
// mapped through the InstanceNorm affine, giving the three kx rows; a B task
// is one dz row x one octet (two float4 loads).  Rows that never change (the
// bias row, the padding rows of the tile and of N) are written once.  Every
// wait is bounded: on expiry the outputs are NaN and g_umma_timeouts counts
// the warp.
// threads of a weight-gradient CTA (staging; warps w < 8 read TMEM lanes
// 32 (w % 4) .. + 31): 512, two CTAs per SM; 256 (three per SM) for the
// 16-channel layer with one subset, whose stages fit three CTAs
__host__ __device__ constexpr int wgrad_threads(int NP, int SETS) { return NP == 16 && SETS == 1 ? 256 : 512; }
constexpr int kWK = 64;      // pixels per stage (four K steps of 16)
constexpr int kWRows = 126;  // columns j per tile
__device__ unsigned int g_umma_timeouts;

static_assert(kSz[0] % 16 == 0 && kSz[1] % 16 == 0 && kSz[2] % 16 == 0 && kSz[3] % 16 == 0 && kSz[4] % 16 == 0,
              "input rows of the weight gradient are loaded as float4 from 16-float boundaries");
static_assert(kSz[5] % 8 == 0, "an output row holds whole pixel octets, an image whole stages");
static_assert(kCh[1] <= 64 && kCh[2] <= 64 && kCh[3] <= 64 && kCh[4] <= 64 && kCh[5] <= 64,
              "output channels of a weight gradient: at most the MMA's N = 64");
static_assert((kCh[2] & (kCh[2] - 1)) == 0 && (kCh[3] & (kCh[3] - 1)) == 0 && (kCh[4] & (kCh[4] - 1)) == 0 &&
                  (kCh[5] & (kCh[5] - 1)) == 0 && kCh[2] >= 8,
              "input gradient: output channels a power of two >= 8 (an octet of k is one tap)");

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return static_cast<uint32_t>(__cvta_generic_to_shared(p)); }

// shared-memory matrix descriptor, no swizzle: start, leading (K) and stride
// (M/N) byte offsets between core matrices, descriptor version 1
__device__ __forceinline__ uint64_t umma_sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    return static_cast<uint64_t>((addr >> 4) & 0x3FFFu) | (static_cast<uint64_t>((lbo >> 4) & 0x3FFFu) << 16) |
           (static_cast<uint64_t>((sbo >> 4) & 0x3FFFu) << 32) | (static_cast<uint64_t>(1) << 46);
}

// instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, N and M
__host__ __device__ constexpr uint32_t umma_idesc_bf16(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | (static_cast<uint32_t>(N >> 3) << 17) |
           (static_cast<uint32_t>(M >> 4) << 24);
}

__device__ __forceinline__ void umma_bf16(uint32_t taddr, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc)
{
    asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                 " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(taddr),
                 "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
}

// waits until the mbarrier's phase of the given parity completes; false if
// the bounded wait expired
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity)
{
    uint32_t done = 0;
    for (long it = 0; it < (1L << 26) && !done; ++it)
        asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                     " selp.u32 %0, 1, 0, p;\n}\n"
                     : "=r"(done)
                     : "r"(mbar), "r"(parity)
                     : "memory");
    return done != 0;
}

// 8 FP32 values as BF16 hi and lo = bf16(v - hi): one 16-byte store each
__device__ __forceinline__ void split_store(char *hi, char *lo, const float (&v)[8])
{
    uint32_t h[4], l[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const __nv_bfloat162 hh = __floats2bfloat162_rn(v[2 * q], v[2 * q + 1]);
        const __nv_bfloat162 ll = __floats2bfloat162_rn(v[2 * q] - __low2float(hh), v[2 * q + 1] - __high2float(hh));
        h[q] = *reinterpret_cast<const uint32_t *>(&hh);
        l[q] = *reinterpret_cast<const uint32_t *>(&ll);
    }
    *reinterpret_cast<uint4 *>(hi) = make_uint4(h[0], h[1], h[2], h[3]);
    *reinterpret_cast<uint4 *>(lo) = make_uint4(l[0], l[1], l[2], l[3]);
}

struct WgradArgs {
    const float *in;       // [B][Cin][S][S] layer input (the raw activation when sc is set)
    const float *sc, *sh;  // [B][Cin] InstanceNorm affine applied on load (zero padding after it), or null
    const float *dz;       // [B][Cout][So][So] gradient of the conv output
    float *part;           // [chunks][Cout][Kd + 1] partial sums
    int Cin, Cout, S, So, npix, chunk;
};

// bytes of one stage: hi and lo parts of the 128-row A and the NP-row B operand
__host__ __device__ constexpr int wgrad_stage_bytes(int NP) { return 2 * (128 + NP) * kWK * 2; }
// CTAs per SM that the two stages allow in 227 KB of shared memory
constexpr int wgrad_ctas_per_sm(int NP) { return (227 * 1024) / (2 * wgrad_stage_bytes(NP) + 1024); }

// SETS = 4 (a layer with 9 Cin + 1 <= 32 columns, like the first): the 128
// rows hold four disjoint pixel subsets of the stage, rows 32 r .. 32 r + 31
// the im2col of subset r and B columns Cout r .. Cout r + Cout - 1 its dz, so
// a stage covers 4 x 64 pixels; the diagonal blocks (r, r) of D are the
// subsets' partial sums (the others are discarded), written as chunks
// SETS z + r.
template <int NP, int SETS>
__global__ void __launch_bounds__(wgrad_threads(NP, SETS), wgrad_threads(NP, SETS) == 256 ? 3 : 2) wgrad_kernel(const WgradArgs p)
{
    static_assert(NP % 16 == 0 && NP >= 16 && NP <= 64, "N of an M = 128 MMA: 16 .. 64, multiple of 16");
    static_assert(SETS == 1 || SETS == 4, "one subset (126-column tiles) or four (32 rows each)");
    constexpr int kWT = wgrad_threads(NP, SETS);
    constexpr int RS = SETS == 1 ? kWRows : 128 / SETS;  // rows of one subset
    constexpr uint32_t kCols = NP < 32 ? 32 : NP;  // TMEM columns (power of 2 >= 32)
    constexpr int kA = 128 * kWK * 2, kB = NP * kWK * 2, kStage = wgrad_stage_bytes(NP);
    constexpr uint32_t idesc = umma_idesc_bf16(128, NP);
    extern __shared__ __align__(128) char wsm[];  // stage s % 2: [A hi][A lo][B hi][B lo]
    __shared__ __align__(8) uint64_t mbar[2];
    __shared__ uint32_t taddr_s;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int tile = blockIdx.x, z = blockIdx.y;
    const int Kd = 9 * p.Cin, P = p.So * p.So;
    const int ng = max(0, min(kWRows / 3, 3 * p.Cin - (kWRows / 3) * tile));  // live (c, ky) groups per subset
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_addr(&taddr_s)),
                     "r"(kCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_addr(&mbar[0])));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_addr(&mbar[1])));
        asm volatile("fence.mbarrier_init.release.cluster;\n");
    }
    // rows that never change: everything zero, then the bias row (hi = 1)
    for (int i = tid; i < 2 * kStage / 16; i += kWT) reinterpret_cast<uint4 *>(wsm)[i] = make_uint4(0u, 0u, 0u, 0u);
    __syncthreads();
    const int rb = Kd - kWRows * tile;  // the bias row within a subset
    if (rb >= 0 && rb < RS && tid < 16 * SETS)
        *reinterpret_cast<uint4 *>(wsm + ((tid >> 3) & 1) * kStage + (tid & 7) * 16 * 128 + 16 * ((tid >> 4) * RS + rb)) =
            make_uint4(0x3F803F80u, 0x3F803F80u, 0x3F803F80u, 0x3F803F80u);
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;\n");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n");
    const uint32_t taddr = taddr_s;
    const int m_beg = z * p.chunk;
    const int nst = (min(p.chunk, p.npix - m_beg) + SETS * kWK - 1) / (SETS * kWK);
    const int na = SETS * ng * 8, nt = na + SETS * p.Cout * 8;
    bool ok = true;
    // Two stages per iteration (both buffers): twice the loads in flight per
    // barrier, which the narrow layers need (their stage has fewer tasks
    // than threads).  Buffer b holds the stages s with s % 2 == b.
    for (int s = 0; s < nst; s += 2) {
        const int ns = min(2, nst - s);
        if (s >= 2) {  // the previous iteration's MMAs have read both buffers
            ok = mbar_wait(smem_addr(&mbar[0]), ((s - 2) >> 1) & 1) && ok;
            ok = mbar_wait(smem_addr(&mbar[1]), ((s - 1) >> 1) & 1) && ok;
        }
        for (int t2 = tid; t2 < ns * nt; t2 += kWT) {
            const int si = t2 >= nt ? 1 : 0, t = t2 - si * nt;
            char *stg = wsm + si * kStage;
            const int m0 = m_beg + (s + si) * SETS * kWK;
            if (t < na) {
                const int set = SETS == 1 ? 0 : t / (ng * 8), ts = t - set * ng * 8;
                const int q = ts / ng, g = ts - q * ng;
                const int cg = (kWRows / 3) * tile + g, c = cg / 3, ky = cg - 3 * c;
                const int m = m0 + set * kWK + 8 * q;
                float v[16], left = 0.f;
#pragma unroll
                for (int u = 0; u < 16; ++u) v[u] = 0.f;
                if (m < p.npix) {
                    const int b = m / P, rr = m - b * P, oy = rr / p.So, ox0 = rr - oy * p.So;
                    const int iy = 2 * oy + ky - 1;
                    if (iy >= 0 && iy < p.S) {
                        const float *row =
                            p.in + (static_cast<size_t>(b * p.Cin + c) * p.S + iy) * p.S + 2 * ox0;
#pragma unroll
                        for (int u = 0; u < 4; ++u) {
                            const float4 f = __ldg(reinterpret_cast<const float4 *>(row) + u);
                            v[4 * u] = f.x;
                            v[4 * u + 1] = f.y;
                            v[4 * u + 2] = f.z;
                            v[4 * u + 3] = f.w;
                        }
                        if (ox0 > 0) left = __ldg(row - 1);
                        if (p.sc) {
                            const float a = __ldg(p.sc + b * p.Cin + c), h = __ldg(p.sh + b * p.Cin + c);
#pragma unroll
                            for (int u = 0; u < 16; ++u) v[u] = fmaf(v[u], a, h);
                            if (ox0 > 0) left = fmaf(left, a, h);
                        }
                    }
                }
                // input column 2 ox + kx - 1 of the octet's pixels ox0 + u
                float r0[8], r1[8], r2[8];
                r0[0] = left;
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    if (u > 0) r0[u] = v[2 * u - 1];
                    r1[u] = v[2 * u];
                    r2[u] = v[2 * u + 1];
                }
                char *dst = stg + q * 16 * 128 + 16 * (set * RS + 3 * g);
                split_store(dst, dst + kA, r0);
                split_store(dst + 16, dst + kA + 16, r1);
                split_store(dst + 32, dst + kA + 32, r2);
            } else {
                const int tb = t - na, set = SETS == 1 ? 0 : tb / (p.Cout * 8), ts = tb - set * p.Cout * 8;
                const int q = ts / p.Cout, o = ts - q * p.Cout;
                const int m = m0 + set * kWK + 8 * q;
                float v[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) v[u] = 0.f;
                if (m < p.npix) {
                    const int b = m / P, rr = m - b * P;
                    const float4 *src =
                        reinterpret_cast<const float4 *>(p.dz + (static_cast<size_t>(b) * p.Cout + o) * P + rr);
                    const float4 f0 = __ldg(src), f1 = __ldg(src + 1);
                    v[0] = f0.x, v[1] = f0.y, v[2] = f0.z, v[3] = f0.w;
                    v[4] = f1.x, v[5] = f1.y, v[6] = f1.z, v[7] = f1.w;
                }
                char *dst = stg + 2 * kA + q * 16 * NP + 16 * (set * p.Cout + o);
                split_store(dst, dst + kB, v);
            }
        }
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");  // generic stores -> tensor core
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;\n");
            for (int si = 0; si < ns; ++si) {
                const uint32_t a0 = smem_addr(wsm + si * kStage), b0 = a0 + 2 * kA;
#pragma unroll
                for (int kk = 0; kk < kWK / 16; ++kk) {
                    const uint64_t ahi = umma_sdesc(a0 + kk * 2 * 16 * 128, 16 * 128, 128);
                    const uint64_t alo = umma_sdesc(a0 + kA + kk * 2 * 16 * 128, 16 * 128, 128);
                    const uint64_t bhi = umma_sdesc(b0 + kk * 2 * 16 * NP, 16 * NP, 128);
                    const uint64_t blo = umma_sdesc(b0 + kB + kk * 2 * 16 * NP, 16 * NP, 128);
                    umma_bf16(taddr, alo, bhi, idesc, (s + si > 0 || kk > 0) ? 1u : 0u);
                    umma_bf16(taddr, ahi, blo, idesc, 1u);
                    umma_bf16(taddr, ahi, bhi, idesc, 1u);
                }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                                 smem_addr(&mbar[si]))
                             : "memory");
            }
        }
    }
    if (nst > 0) ok = mbar_wait(smem_addr(&mbar[(nst - 1) & 1]), ((nst - 1) >> 1) & 1) && ok;  // all MMAs
    asm volatile("tcgen05.fence::after_thread_sync;\n");
    if (!ok && lane == 0) atomicAdd(&g_umma_timeouts, 1u);
    if constexpr (SETS > 1) {
        // warp w < 4 holds subset w's rows (its lanes), its block of columns
        if (warp < 4) {
            const int zv = SETS * z + warp;
            for (int c0 = 0; c0 < p.Cout; c0 += 8) {
                uint32_t v[8];
                asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n"
                             : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
                               "=r"(v[7])
                             : "r"(taddr + (static_cast<uint32_t>(32 * warp) << 16) + warp * p.Cout + c0));
                asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const int o = c0 + q;
                    if (lane <= Kd && o < p.Cout)
                        p.part[(static_cast<size_t>(zv) * p.Cout + o) * (Kd + 1) + lane] =
                            ok ? __uint_as_float(v[q]) : __int_as_float(0x7fc00000);
                }
            }
        }
    } else {
    // epilogue: warp w < 8 holds rows 32 (w % 4) + lane of D, columns of half w / 4
    const int r = 32 * (warp & 3) + lane, j = kWRows * tile + r;
    constexpr int kHalf = NP / 2;
    const int cb = (warp >> 2) * kHalf;
#pragma unroll
    for (int c0 = 0; c0 < (warp < 8 ? kHalf : 0); c0 += 8) {
        uint32_t v[8];
        asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n"
                     : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
                     : "r"(taddr + (static_cast<uint32_t>(32 * (warp & 3)) << 16) + cb + c0));
        asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int o = cb + c0 + q;
            if (r < kWRows && j <= Kd && o < p.Cout)
                p.part[(static_cast<size_t>(z) * p.Cout + o) * (Kd + 1) + j] =
                    ok ? __uint_as_float(v[q]) : __int_as_float(0x7fc00000);
        }
    }
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;\n");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(taddr), "r"(kCols));
    }
}

// ---- forward convolution on tcgen05 (implicit GEMM) ----
// D[m][o] = sum_k im2col[m][k] W[o][k] for the output pixels m = (b, oy, ox)
// of a 128-pixel tile (the MMA's M rows, TMEM lanes) and the output channels
// o (N = NP >= Cout), K = 9 Cin.  Reduction order: (tap = 3 ky + kx, c) with c
// fastest when Cin is a power of two >= 8 (C8: an octet of k is 8 channels of
// one tap, decoded once by shift and mask), else (the first layer, Cin = 3)
// the weight tensor's own order (c, ky, kx), decoded at compile time.  Both
// operands are single BF16 (the forward's precision) in the no-swizzle
// K-major layout of wgrad_kernel: element (m, k) of a stage of kWK = 64 k at
// byte (k / 8) * 16 * 128 + 16 m + 2 (k % 8), so a thread writes the 8 k of
// one octet of its pixel as one 16-byte store (conflict-free across a warp's
// consecutive pixels).  conv_wprep_kernel lays the weights out once per call
// in exactly the stage layout of B (element (o, k) at byte (k / 8) * 16 NP +
// 16 o + 2 (k % 8), zero for o >= Cout and k >= Kd), so a stage of B is a
// contiguous copy.  CTA (tile, z) takes the stages [z ks, (z + 1) ks) and
// writes its raw sums to part[z][o][m]; conv_finish_kernel adds the partials
// in z order, the bias, LeakyReLU and the InstanceNorm statistics.  Two
// stages in flight; every wait is bounded (NaN outputs and g_umma_timeouts
// on expiry).
// sum over the 32 lanes (butterfly: every lane gets the same total)
__device__ __forceinline__ float warp_total(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

struct ConvUmma {
    const float *in;       // [B][Cin][S][S]
    const float *sc, *sh;  // [B][Cin] affine map of the input (zero padding after it), or null
    const uint4 *wb;       // BF16 weights in the stage layout (conv_wprep_kernel)
    float *part;           // [Z][Cout][M]
    int Cin, S, So, Cout, M, Kd, ks;  // ks: stages of 64 k per split
    // fused finish (one split, So^2 a multiple of 128, r set): the epilogue
    // writes r = LeakyReLU(D + bias) and the tile's per-channel sum and M2
    const float *bias;  // [Cout]
    float *r;           // [B][Cout][So][So], or null: raw sums to part
    float *tstat;       // [tiles][Cout][2]
};

// NT threads (128 or 256): thread t keeps pixel t % 128 of the tile and the
// octets t / 128 + (NT / 128) j of each stage; NBUF stage buffers (1 or 2).
// The narrow layers take 128 threads, so that more CTAs (tiles in flight)
// fit on an SM.
__host__ __device__ constexpr int conv_stage_bytes(int NP) { return (128 + NP) * kWK * 2; }

template <int NP, bool C8, int NT, int NBUF>
__global__ void __launch_bounds__(NT, NT == 128 ? 8 : (NP == 64 ? 2 : 3)) conv_umma_kernel(const ConvUmma p)
{
    static_assert(NP % 16 == 0 && NP >= 16 && NP <= 64, "N of an M = 128 MMA: 16 .. 64, multiple of 16");
    static_assert((NT == 128 || NT == 256) && (NBUF == 1 || NBUF == 2), "128 or 256 threads, 1 or 2 stages");
    constexpr uint32_t kCols = NP < 32 ? 32 : NP;
    constexpr int kA = 128 * kWK * 2, kStage = conv_stage_bytes(NP);
    constexpr uint32_t idesc = umma_idesc_bf16(128, NP);
    extern __shared__ __align__(128) char csm[];  // stage i % NBUF: [A][B]
    __shared__ __align__(8) uint64_t mbar[2];
    __shared__ uint32_t taddr_s;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int tile = blockIdx.x, z = blockIdx.y;
    const int P = p.So * p.So, S2 = p.S * p.S;
    const int ml = tid & 127, m = tile * 128 + ml;
    const bool mval = m < p.M;
    int b = 0, oy = 0, ox = 0;
    if (mval) {
        b = m / P;
        const int rr = m - b * P;
        oy = rr / p.So;
        ox = rr - oy * p.So;
    }
    const float *inb = p.in + static_cast<size_t>(b) * p.Cin * S2;
    const float *scb = p.sc ? p.sc + b * p.Cin : nullptr;
    const float *shb = p.sh ? p.sh + b * p.Cin : nullptr;
    static_assert(C8 || NT == 128, "the first layer's element decode needs q = j (128 threads)");
    const int cin_lg = 31 - __clz(p.Cin);
    int roff[3], xoff[3];  // first layer: input row offset and column of tap ky / kx, and whether inside
    bool vy[3], vx[3];
#pragma unroll
    for (int t = 0; t < 3; ++t) {
        const int iy = 2 * oy + t - 1, ix = 2 * ox + t - 1;
        vy[t] = iy >= 0 && iy < p.S;
        vx[t] = ix >= 0 && ix < p.S;
        roff[t] = iy * p.S;
        xoff[t] = ix;
    }
    const int nko = (p.Kd + 7) / 8;
    const int st_beg = z * p.ks, st_end = min(st_beg + p.ks, (p.Kd + kWK - 1) / kWK);
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_addr(&taddr_s)),
                     "r"(kCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_addr(&mbar[0])));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_addr(&mbar[1])));
        asm volatile("fence.mbarrier_init.release.cluster;\n");
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n");
    const uint32_t taddr = taddr_s;
    pdl_enter();  // the input and the prepared weights come from earlier kernels
    bool ok = true;
    for (int s = st_beg; s < st_end; ++s) {
        const int i = s - st_beg, buf = i % NBUF;
        char *stg = csm + buf * kStage;
        if (i >= NBUF) ok = mbar_wait(smem_addr(&mbar[buf]), ((i - NBUF) / NBUF) & 1) && ok;  // stage i - NBUF read
        const uint4 *wsrc = p.wb + static_cast<size_t>(s) * NP * 8;
        for (int e = tid; e < NP * 8; e += NT) reinterpret_cast<uint4 *>(stg + kA)[e] = __ldg(wsrc + e);
#pragma unroll
        for (int j = 0; j < 8 * 128 / NT; ++j) {
            const int q = (tid >> 7) + (NT / 128) * j, k0 = s * kWK + 8 * q;
            char *dst = stg + q * 16 * 128 + 16 * ml;
            if (k0 >= p.Kd) {  // past the reduction: zeros (B is zero there too)
                *reinterpret_cast<uint4 *>(dst) = make_uint4(0u, 0u, 0u, 0u);
                continue;
            }
            float v[8];
            if constexpr (C8) {
                // Cin a power of two: tap and first channel by shift and mask
                const int t = k0 >> cin_lg, c0 = k0 & (p.Cin - 1), ky = t / 3, kx = t - 3 * ky;
                const int iy = 2 * oy + ky - 1, ix = 2 * ox + kx - 1;
                const bool in = mval && iy >= 0 && iy < p.S && ix >= 0 && ix < p.S;
                const float *src = inb + static_cast<size_t>(c0) * S2 + iy * p.S + ix;
#pragma unroll
                for (int u = 0; u < 8; ++u) v[u] = in ? __ldg(src + static_cast<size_t>(u) * S2) : 0.f;
                if (scb && in) {
                    const float4 a0 = __ldg(reinterpret_cast<const float4 *>(scb + c0)),
                                 a1 = __ldg(reinterpret_cast<const float4 *>(scb + c0) + 1);
                    const float4 h0 = __ldg(reinterpret_cast<const float4 *>(shb + c0)),
                                 h1 = __ldg(reinterpret_cast<const float4 *>(shb + c0) + 1);
                    const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
                    const float h[8] = {h0.x, h0.y, h0.z, h0.w, h1.x, h1.y, h1.z, h1.w};
#pragma unroll
                    for (int u = 0; u < 8; ++u) v[u] = fmaf(v[u], a[u], h[u]);
                }
            } else {
                // the first layer (Cin = 3, one stage, q = j): k = 9 c + 3 ky + kx
                // is a constant per unrolled element
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int k = 8 * j + u, c = k / 9, ky = (k % 9) / 3, kx = k % 3;
                    const bool in = k < 27 && mval && vy[ky] && vx[kx];
                    float x = in ? __ldg(inb + c * S2 + roff[ky] + xoff[kx]) : 0.f;
                    if (scb && in) x = fmaf(x, __ldg(scb + c), __ldg(shb + c));
                    v[u] = x;
                }
            }
            uint32_t h[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const __nv_bfloat162 hh = __floats2bfloat162_rn(v[2 * u], v[2 * u + 1]);
                h[u] = *reinterpret_cast<const uint32_t *>(&hh);
            }
            *reinterpret_cast<uint4 *>(dst) = make_uint4(h[0], h[1], h[2], h[3]);
        }
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");  // generic stores -> tensor core
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;\n");
            const uint32_t a0 = smem_addr(stg), b0 = a0 + kA;
            const int nk = (min(8, nko - 8 * s) + 1) / 2;  // K steps of 16 holding live k
            for (int kk = 0; kk < nk; ++kk)
                umma_bf16(taddr, umma_sdesc(a0 + kk * 2 * 16 * 128, 16 * 128, 128),
                          umma_sdesc(b0 + kk * 2 * 16 * NP, 16 * NP, 128), idesc, (i > 0 || kk > 0) ? 1u : 0u);
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                             smem_addr(&mbar[buf]))
                         : "memory");
        }
    }
    const int nst = st_end - st_beg;
    if (nst > 0) ok = mbar_wait(smem_addr(&mbar[(nst - 1) % NBUF]), ((nst - 1) / NBUF) & 1) && ok;  // all MMAs
    asm volatile("tcgen05.fence::after_thread_sync;\n");
    if (!ok && lane == 0) atomicAdd(&g_umma_timeouts, 1u);
    // epilogue: warp w holds pixels 32 (w % 4) + lane of the tile and, of
    // the NP channels, the kHalf from (w / 4) kHalf (kHalf = NP with 128 threads)
    const int r = 32 * (warp & 3) + lane, mo = tile * 128 + r;
    constexpr int kHalf = NP * 128 / NT;
    const int cb = (warp >> 2) * kHalf;
    if (p.r) {
        // fused finish: the tile lies in one image b; per channel the tile's
        // sum (fixed order: warps, then the four warps of a half) and its M2
        // about the tile mean (conv_stats_kernel combines the tiles)
        __shared__ float red[2][4][NP];
        const int bimg = (tile * 128) / P, rr = mo - bimg * P;
        float x[kHalf];
#pragma unroll
        for (int c0 = 0; c0 < kHalf; c0 += 8) {
            uint32_t v[8];
            asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n"
                         : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
                           "=r"(v[7])
                         : "r"(taddr + (static_cast<uint32_t>(32 * (warp & 3)) << 16) + cb + c0));
            asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int o = cb + c0 + q;
                float y = 0.f;
                if (o < p.Cout) {
                    y = __uint_as_float(v[q]) + __ldg(p.bias + o);
                    y = y > 0.f ? y : kSlope * y;
                    if (!ok) y = __int_as_float(0x7fc00000);
                    p.r[(static_cast<size_t>(bimg) * p.Cout + o) * P + rr] = y;
                }
                x[c0 + q] = y;
            }
        }
#pragma unroll
        for (int c = 0; c < kHalf; ++c) {
            if (cb + c >= p.Cout) break;  // padding channels (uniform per warp)
            const float t = warp_total(x[c]);
            if (lane == 0) red[0][warp & 3][cb + c] = t;
        }
        __syncthreads();
#pragma unroll
        for (int c = 0; c < kHalf; ++c) {
            const int o = cb + c;
            if (o >= p.Cout) break;
            const float mt = (((red[0][0][o] + red[0][1][o]) + red[0][2][o]) + red[0][3][o]) * (1.f / 128.f);
            const float d = x[c] - mt, t = warp_total(d * d);
            if (lane == 0) red[1][warp & 3][o] = t;
        }
        __syncthreads();
        if (tid < p.Cout) {
            float *e = p.tstat + (static_cast<size_t>(tile) * p.Cout + tid) * 2;
            e[0] = ((red[0][0][tid] + red[0][1][tid]) + red[0][2][tid]) + red[0][3][tid];
            e[1] = ((red[1][0][tid] + red[1][1][tid]) + red[1][2][tid]) + red[1][3][tid];
        }
    } else {
#pragma unroll
    for (int c0 = 0; c0 < kHalf; c0 += 8) {
        uint32_t v[8];
        asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n"
                     : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
                     : "r"(taddr + (static_cast<uint32_t>(32 * (warp & 3)) << 16) + cb + c0));
        asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int o = cb + c0 + q;
            if (mo < p.M && o < p.Cout)
                p.part[(static_cast<size_t>(z) * p.Cout + o) * p.M + mo] =
                    ok ? __uint_as_float(v[q]) : __int_as_float(0x7fc00000);
        }
    }
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;\n");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(taddr), "r"(kCols));
    }
}

// The five convolutions' weights as BF16 in the B stage layout of
// conv_umma_kernel: element (o, k) of layer i at bf16 index (k / 8) * 8 NP +
// 8 o + k % 8 for k < Kpad (whole 64-k stages), zero for o >= Cout or k >= Kd;
// k in the kernel's reduction order ((tap, c) when Cin is a power of two >= 8,
// else (c, tap)).
struct WPrep {
    const float *w[5];
    __nv_bfloat16 *out[5];
    int start[6];  // flattened element ranges per layer
    int cin[5], cout[5], np[5], kpad[5];
};

__global__ void conv_wprep_kernel(const WPrep p)
{
    pdl_enter();  // the outputs may still be read by the previous call's kernels
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < p.start[5]; e += gridDim.x * blockDim.x) {
        int i = 0;
        while (e >= p.start[i + 1]) ++i;
        const int Cin = p.cin[i], Cout = p.cout[i], Kd = 9 * Cin, NP = p.np[i];
        const int l = e - p.start[i], o = l / p.kpad[i], k = l - o * p.kpad[i];
        float v = 0.f;
        if (o < Cout && k < Kd) {
            int c, tap;
            if (Cin >= 8 && (Cin & (Cin - 1)) == 0) {
                tap = k / Cin;
                c = k - tap * Cin;
            } else {
                c = k / 9;
                tap = k - 9 * c;
            }
            v = p.w[i][(static_cast<size_t>(o) * Cin + c) * 9 + tap];
        }
        p.out[i][(k >> 3) * 8 * NP + 8 * o + (k & 7)] = __float2bfloat16_rn(v);
    }
}

// ---- input gradient of the stride-2 3x3 convolution on tcgen05, by input parity ----
// Input pixel (iy, ix) = (2 qy + py, 2 qx + px) only receives the taps with
// iy + 1 - ky and ix + 1 - kx even: ky = 1 (output row qy) when py = 0, ky = 0
// (row qy + 1) or ky = 2 (row qy) when py = 1; likewise along x.  Each parity
// class (blockIdx.y = 2 py + px) is then a dense GEMM: M = the class's input
// pixels m = (b, qy, qx), 128 per CTA (TMEM lanes), N = NP >= Cin input
// channels, K = (tap, o) over its 1, 2 or 4 live taps x Cout (o fastest;
// Cout is a power of two >= 8, so an octet of k is 8 output channels of one
// tap).  No zero tap of the full 3x3 im2col is loaded or multiplied.  Both
// operands are split into BF16 hi and lo parts (lo*hi + hi*lo + hi*hi, the
// weight gradient's precision), staged K-major in the no-swizzle layout
// (element (m, k) at byte (k / 8) 16 * 128 + 16 m + 2 (k % 8)); the weights are
// laid out once per call by dgrad_wprep_kernel in the stage layout of B
// (per layer and class: NP x Kpad hi, then lo).  One stage buffer; every
// wait is bounded (NaN outputs and g_umma_timeouts on expiry).
struct DgradUmma {
    const float *dz;   // [B][Cout][So][So]
    const uint4 *wb;   // this layer's prepared weights; class c at wb + cls_off[c] (uint4 units)
    float *dact;       // [B][Cin][2 So][2 So]
    int Cout, Cin, So, M, cout_lg;  // M = B So^2 pixels per class
    int cls_off[4], kpad[4];        // per class: offset of its hi part, K padded to whole stages
};

constexpr int kDGT = 128;  // threads: pixel tid of the tile, all eight octets of a stage
__host__ __device__ constexpr int dgrad_stage_bytes(int NP) { return 2 * (128 + NP) * kWK * 2; }

// NBUF stage buffers: 2 for the widest layer (up to four K stages per class,
// 128 CTAs), 1 for the others, whose many CTAs need the occupancy more than
// the overlap (measured: two buffers slowed the 32-channel layer 23 -> 31 us).
template <int NP, int NBUF>
__global__ void __launch_bounds__(kDGT, NBUF == 2 ? 2 : (NP == 64 ? 4 : 6)) dgrad_umma_kernel(const DgradUmma p)
{
    static_assert(NBUF == 1 || NBUF == 2, "one or two stage buffers");
    static_assert(NP % 16 == 0 && NP >= 16 && NP <= 64, "N of an M = 128 MMA: 16 .. 64, multiple of 16");
    constexpr uint32_t kCols = NP < 32 ? 32 : NP;
    constexpr int kA = 128 * kWK * 2, kB = NP * kWK * 2;  // one part (hi or lo) of A / B
    constexpr uint32_t idesc = umma_idesc_bf16(128, NP);
    extern __shared__ __align__(128) char dsm0[];  // stage s % NBUF: [A hi][A lo][B hi][B lo]
    __shared__ __align__(8) uint64_t mbar[2];
    __shared__ uint32_t taddr_s;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int tile = blockIdx.x, cls = blockIdx.y, py = cls >> 1, px = cls & 1, ntx = px ? 2 : 1;
    const int Kd = (py ? 2 : 1) * ntx * p.Cout, nst = (Kd + kWK - 1) / kWK, P = p.So * p.So;
    const int m = tile * 128 + tid;
    const bool mval = m < p.M;
    int b = 0, qy = 0, qx = 0;
    if (mval) {
        b = m / P;
        const int rr = m - b * P;
        qy = rr / p.So;
        qx = rr - qy * p.So;
    }
    const float *dzb = p.dz + static_cast<size_t>(b) * p.Cout * P;
    // (selected, not indexed: a runtime index would copy the arrays to local memory)
    const int cls_off = cls == 0 ? p.cls_off[0] : cls == 1 ? p.cls_off[1] : cls == 2 ? p.cls_off[2] : p.cls_off[3];
    const int kpad = cls == 0 ? p.kpad[0] : cls == 1 ? p.kpad[1] : cls == 2 ? p.kpad[2] : p.kpad[3];
    const uint4 *wcls = p.wb + cls_off;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_addr(&taddr_s)),
                     "r"(kCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_addr(&mbar[0])));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_addr(&mbar[1])));
        asm volatile("fence.mbarrier_init.release.cluster;\n");
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n");
    const uint32_t taddr = taddr_s;
    bool ok = true;
    for (int s = 0; s < nst; ++s) {
        const int buf = s % NBUF;
        char *dsm = dsm0 + buf * dgrad_stage_bytes(NP);
        if (s >= NBUF) ok = mbar_wait(smem_addr(&mbar[buf]), ((s - NBUF) / NBUF) & 1) && ok;  // stage s - NBUF read
        // B: hi and lo parts of this stage, contiguous in the prepared layout
        const uint4 *whi = wcls + static_cast<size_t>(s) * NP * 8, *wlo = whi + static_cast<size_t>(kpad) * NP / 8;
        for (int e = tid; e < NP * 8; e += kDGT) {
            reinterpret_cast<uint4 *>(dsm + 2 * kA)[e] = __ldg(whi + e);
            reinterpret_cast<uint4 *>(dsm + 2 * kA + kB)[e] = __ldg(wlo + e);
        }
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int k0 = s * kWK + 8 * q;
            char *dst = dsm + q * 16 * 128 + 16 * tid;
            float v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) v[u] = 0.f;
            if (k0 < Kd && mval) {
                const int tap = k0 >> p.cout_lg, o0 = k0 & (p.Cout - 1);
                const int ty = ntx == 2 ? tap >> 1 : tap, tx = ntx == 2 ? tap & 1 : 0;
                const int oy = qy + (py && ty == 0 ? 1 : 0), ox = qx + (px && tx == 0 ? 1 : 0);
                if (oy < p.So && ox < p.So) {
                    const float *src = dzb + static_cast<size_t>(o0) * P + oy * p.So + ox;
#pragma unroll
                    for (int u = 0; u < 8; ++u) v[u] = __ldg(src + static_cast<size_t>(u) * P);
                }
            }
            split_store(dst, dst + kA, v);
        }
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");  // generic stores -> tensor core
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;\n");
            const uint32_t a0 = smem_addr(dsm), b0 = a0 + 2 * kA;
            const int nk = (min(kWK, Kd - s * kWK) + 15) / 16;  // K steps of 16 holding live k
            for (int kk = 0; kk < nk; ++kk) {
                const uint64_t ahi = umma_sdesc(a0 + kk * 2 * 16 * 128, 16 * 128, 128);
                const uint64_t alo = umma_sdesc(a0 + kA + kk * 2 * 16 * 128, 16 * 128, 128);
                const uint64_t bhi = umma_sdesc(b0 + kk * 2 * 16 * NP, 16 * NP, 128);
                const uint64_t blo = umma_sdesc(b0 + kB + kk * 2 * 16 * NP, 16 * NP, 128);
                umma_bf16(taddr, alo, bhi, idesc, (s > 0 || kk > 0) ? 1u : 0u);
                umma_bf16(taddr, ahi, blo, idesc, 1u);
                umma_bf16(taddr, ahi, bhi, idesc, 1u);
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                             smem_addr(&mbar[buf]))
                         : "memory");
        }
    }
    if (nst > 0) ok = mbar_wait(smem_addr(&mbar[(nst - 1) % NBUF]), ((nst - 1) / NBUF) & 1) && ok;  // all MMAs
    asm volatile("tcgen05.fence::after_thread_sync;\n");
    if (!ok && lane == 0) atomicAdd(&g_umma_timeouts, 1u);
    // epilogue: thread tid holds pixel tid of the tile (TMEM lane), all NP channels
    const int S = 2 * p.So;
    float *out = p.dact + static_cast<size_t>(b) * p.Cin * S * S + static_cast<size_t>(2 * qy + py) * S + 2 * qx + px;
#pragma unroll
    for (int c0 = 0; c0 < NP; c0 += 8) {
        uint32_t v[8];
        asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n"
                     : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
                     : "r"(taddr + (static_cast<uint32_t>(32 * warp) << 16) + c0));
        asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int c = c0 + q;
            if (mval && c < p.Cin)
                out[static_cast<size_t>(c) * S * S] = ok ? __uint_as_float(v[q]) : __int_as_float(0x7fc00000);
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;\n");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(taddr), "r"(kCols));
    }
}

// The input-gradient weights of conv layers 1..4 as split BF16 in the B
// stage layout of dgrad_umma_kernel: per layer and parity class, the hi part
// then the lo part, each with element (c, k = tap * Cout + o) at bf16 index
// (k / 8) * 8 NP + 8 c + k % 8 for k < Kpad (whole 64-k stages); zero for
// c >= Cin or k beyond the class's taps.  Segment g = 4 (layer - 1) + class.
struct DPrep {
    const float *w[4];       // [Cout][Cin][3][3] of layers 1..4
    __nv_bfloat16 *seg[16];  // hi part of each segment (lo follows at + NP Kpad)
    int cin[4], cout[4], np[4], kpad[16];
    int start[17];           // flattened element ranges (NP x Kpad each)
};

__global__ void dgrad_wprep_kernel(const DPrep p)
{
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < p.start[16]; e += gridDim.x * blockDim.x) {
        int g = 0;
        while (e >= p.start[g + 1]) ++g;
        const int l = g >> 2, cls = g & 3, py = cls >> 1, px = cls & 1, ntx = px ? 2 : 1;
        const int Cin = p.cin[l], Cout = p.cout[l], NP = p.np[l], kpad = p.kpad[g];
        const int i = e - p.start[g], c = i / kpad, k = i - c * kpad;
        const int Kd = (py ? 2 : 1) * ntx * Cout;
        float v = 0.f;
        if (c < Cin && k < Kd) {
            const int tap = k / Cout, o = k - tap * Cout;
            const int ty = ntx == 2 ? tap >> 1 : tap, tx = ntx == 2 ? tap & 1 : 0;
            const int ky = py ? (ty == 0 ? 0 : 2) : 1, kx = px ? (tx == 0 ? 0 : 2) : 1;
            v = p.w[l][((static_cast<size_t>(o) * Cin + c) * 3 + ky) * 3 + kx];
        }
        const __nv_bfloat16 h = __float2bfloat16_rn(v);
        const size_t at = static_cast<size_t>(k >> 3) * 8 * NP + 8 * c + (k & 7);
        p.seg[g][at] = h;
        p.seg[g][static_cast<size_t>(NP) * kpad + at] = __float2bfloat16_rn(v - __bfloat162float(h));
    }
}

// Fixed-order sum over the NW warps of a block; every thread gets the total.
template <int NW>
__device__ __forceinline__ float block_sum(float v, float *red)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    float s = 0.f;
#pragma unroll
    for (int w = 0; w < NW; ++w) s += red[w];
    return s;
}

// One CTA of NT threads per (b, n) plane of conv i (the layers whose K is
// split): r = LeakyReLU(sum_z part + bias); with
// gam set, also the InstanceNorm statistics of the plane (two passes, biased
// variance) and its affine map sc = gamma rstd, sh = beta - mean sc.
template <int NT>
__global__ void __launch_bounds__(NT) conv_finish_kernel(const float *__restrict__ part, int Z, int N, int M, int P,
                                                         const float *__restrict__ bias, float *__restrict__ r,
                                                         const float *gam, const float *bet, float *mean, float *rstd,
                                                         float *sc, float *sh)
{
    pdl_enter();
    __shared__ float red[NT / 32];
    const int bn = blockIdx.x, b = bn / N, n = bn - b * N;
    const float *src = part + static_cast<size_t>(n) * M + static_cast<size_t>(b) * P;
    const size_t zs = static_cast<size_t>(N) * M;
    float *dst = r + static_cast<size_t>(bn) * P;
    const float bi = __ldg(bias + n);
    float s = 0.f;
    for (int i0 = threadIdx.x; i0 < P; i0 += 4 * NT) {
        // four pixels, partials taken 8 slices at a time with every load
        // issued before the (in-order) sums
        float v[4] = {0.f, 0.f, 0.f, 0.f};
        for (int z0 = 0; z0 < Z; z0 += 8) {
            float t[8][4];
#pragma unroll
            for (int zz = 0; zz < 8; ++zz)
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    t[zz][u] = z0 + zz < Z && i0 + u * NT < P ? src[(z0 + zz) * zs + i0 + u * NT] : 0.f;
#pragma unroll
            for (int zz = 0; zz < 8; ++zz)
#pragma unroll
                for (int u = 0; u < 4; ++u) v[u] += t[zz][u];
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            if (i0 + u * NT >= P) break;
            float x = v[u] + bi;
            x = x > 0.f ? x : kSlope * x;
            dst[i0 + u * NT] = x;
            s += x;
        }
    }
    if (!gam) return;
    const float mu = block_sum<NT / 32>(s, red) / P;
    float q = 0.f;
#pragma unroll 4
    for (int i = threadIdx.x; i < P; i += NT) {
        const float d = dst[i] - mu;
        q = fmaf(d, d, q);
    }
    const float var = block_sum<NT / 32>(q, red) / P;
    if (threadIdx.x == 0) {
        const float rs = rsqrtf(var + kEps), gs = rs * gam[n];
        mean[bn] = mu;
        rstd[bn] = rs;
        sc[bn] = gs;
        sh[bn] = bet[n] - mu * gs;
    }
}

// InstanceNorm statistics of a convolution with the fused finish: one warp
// per (b, o) plane merges the per-tile (count 128, sum, M2) of image b in a
// fixed order (lane l takes tiles [l T / 32, (l + 1) T / 32) in order, then a
// pairwise tree over the lanes; Chan, Golub and LeVeque's update for a
// union: mean += d nB / n, M2 += M2B + d^2 nA nB / n), then writes mean,
// rstd (biased variance) and the affine map sc = gamma rstd, sh = beta - mean sc.
__global__ void conv_stats_kernel(const float *__restrict__ tstat, int B, int Cout, int tpi, int P,
                                  const float *__restrict__ gam, const float *__restrict__ bet, float *mean,
                                  float *rstd, float *sc, float *sh)
{
    pdl_enter();
    const int wid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (wid >= B * Cout) return;
    const int b = wid / Cout, o = wid - b * Cout;
    float n = 0.f, mu = 0.f, m2 = 0.f;
    auto merge = [&](float nb, float mb, float m2b) {
        if (nb == 0.f) return;
        const float nn = n + nb, d = mb - mu, f = nb / nn;
        m2 = m2 + m2b + d * d * n * f;
        mu = fmaf(d, f, mu);
        n = nn;
    };
    for (int t = lane * tpi / 32; t < (lane + 1) * tpi / 32; ++t) {
        const float *e = tstat + (static_cast<size_t>(b) * tpi + t) * Cout * 2 + 2 * o;
        merge(128.f, e[0] * (1.f / 128.f), e[1]);
    }
#pragma unroll
    for (int s = 1; s < 32; s <<= 1) {
        const float nb = __shfl_down_sync(0xffffffffu, n, s), mb = __shfl_down_sync(0xffffffffu, mu, s),
                    m2b = __shfl_down_sync(0xffffffffu, m2, s);
        if ((lane & (2 * s - 1)) == 0) merge(nb, mb, m2b);
    }
    if (lane == 0) {
        const float var = m2 / static_cast<float>(P);
        const float rs = rsqrtf(var + kEps), gs = rs * gam[o];
        mean[wid] = mu;
        rstd[wid] = rs;
        sc[wid] = gs;
        sh[wid] = bet[o] - mu * gs;
    }
}

// Opts kernel fn into `bytes` of dynamic shared memory, once per device
// (calls from several threads are serialised).
static svdlut_status smem_opt_in(const void *fn, int bytes)
{
    static std::mutex mu;
    static std::vector<std::pair<int, const void *>> done;
    int dev = 0;
    SVDLUT_CUDA_TRY(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> g(mu);
    for (const auto &e : done)
        if (e.first == dev && e.second == fn) return SVDLUT_OK;
    SVDLUT_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    done.emplace_back(dev, fn);
    return SVDLUT_OK;
}

template <int NP, int SETS>
static svdlut_status launch_wgrad(const WgradArgs &a, int tiles, int chunks, cudaStream_t s)
{
    constexpr int smem = 2 * wgrad_stage_bytes(NP);
    const svdlut_status st = smem_opt_in(reinterpret_cast<const void *>(wgrad_kernel<NP, SETS>), smem);
    if (st != SVDLUT_OK) return st;
    wgrad_kernel<NP, SETS><<<dim3(tiles, chunks), wgrad_threads(NP, SETS), smem, s>>>(a);
    SVDLUT_CUDA_TRY(cudaGetLastError());
    return SVDLUT_OK;
}

// Launch of conv_umma_kernel<NP, C8> as a programmatic dependent of the
// kernel before it.
template <int NP, bool C8, int NT, int NBUF>
static svdlut_status launch_conv_t(const ConvUmma &a, dim3 grid, cudaStream_t s)
{
    constexpr int smem = NBUF * conv_stage_bytes(NP);
    const svdlut_status st = smem_opt_in(reinterpret_cast<const void *>(conv_umma_kernel<NP, C8, NT, NBUF>), smem);
    if (st != SVDLUT_OK) return st;
    return launch_pdl(conv_umma_kernel<NP, C8, NT, NBUF>, grid, dim3(NT), smem, s, a);
}
template <int NP, int NBUF>
static svdlut_status launch_dgrad_t(const DgradUmma &a, cudaStream_t s)
{
    constexpr int smem = NBUF * dgrad_stage_bytes(NP);
    const svdlut_status st = smem_opt_in(reinterpret_cast<const void *>(dgrad_umma_kernel<NP, NBUF>), smem);
    if (st != SVDLUT_OK) return st;
    dgrad_umma_kernel<NP, NBUF><<<dim3((a.M + 127) / 128, 4), kDGT, smem, s>>>(a);
    SVDLUT_CUDA_TRY(cudaGetLastError());
    return SVDLUT_OK;
}
static svdlut_status launch_conv(const ConvUmma &a, int Z, cudaStream_t s)
{
    const dim3 grid((a.M + 127) / 128, Z);
    const int np = wgrad_np(a.Cout);
    if ((a.Cin & (a.Cin - 1)) != 0 || a.Cin < 8) {
        // the first layer: 27 k, one stage, one buffer
        if (np == 16 && a.Cin == 3) return launch_conv_t<16, false, 128, 1>(a, grid, s);
        return fail(SVDLUT_ERR_UNSUPPORTED, "convolution with %d inputs and %d outputs", a.Cin, a.Cout);
    }
    return np == 16 ? launch_conv_t<16, true, 128, 2>(a, grid, s)
                    : np == 32 ? launch_conv_t<32, true, 256, 2>(a, grid, s) : launch_conv_t<64, true, 256, 2>(a, grid, s);
}

// Fixed-order block sum (256 threads); every thread gets the total.
__device__ __forceinline__ float block_sum256(float v, float *red) { return block_sum<8>(v, red); }

// SplitMix64 finaliser (Steele, Lea, Flood 2014), the counter-based
// generator of the dropout mask: element e of [B][64][8][8] is kept (x2)
// when the top bit of splitmix64(seed * 2^32 + e) is 0.
__device__ __forceinline__ uint64_t splitmix64(uint64_t x)
{
    uint64_t z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ float drop_scale(int training, uint64_t seed, size_t e)
{
    if (!training) return 1.f;
    return (splitmix64((seed << 32) + e) >> 63) == 0 ? 2.f : 0.f;
}

// Dropout + 4x4 average pooling of the last feature map [B][64][8][8] -> rho
// [B][256], one thread per rho element (kept for the backward pass).
__device__ __forceinline__ float pool_one(const float *__restrict__ r4, int b, int i, int training, uint64_t seed)
{
    const int c = i >> 2, py = (i >> 1) & 1, px = i & 1;
    float s = 0.f;
#pragma unroll
    for (int yy = 0; yy < 4; ++yy)
#pragma unroll
        for (int xx = 0; xx < 4; ++xx) {
            const size_t f = ((static_cast<size_t>(b) * 64 + c) * 8 + py * 4 + yy) * 8 + px * 4 + xx;
            s += __ldg(r4 + f) * drop_scale(training, seed, f);
        }
    return s * (1.f / 16.f);
}

struct HeadW {
    const float *w1[4], *b1[4], *w2[4], *b2[4];
    int n[4];
    int K;
};

struct ParamOut {
    float *U, *S, *V, *lw, *gxy, *gxc, *gyc, *gw;
};

// destination of head h, output n of image b in the svdlut parameter layouts
__device__ __forceinline__ float *head_dst(const ParamOut &o, int K, int h, int b, int n)
{
    if (h == 0) {
        const int k = n / (3 * kDS * kDS), rem = n - k * 3 * kDS * kDS, plane = rem / (kDS * kDS),
                  e = rem - plane * kDS * kDS;
        float *base = plane == 0 ? o.gxy : (plane == 1 ? o.gxc : o.gyc);
        return base + (static_cast<size_t>(b) * K + k) * kDS * kDS + e;
    }
    if (h == 1) return o.gw + static_cast<size_t>(b) * K * 4 + n;
    if (h == 3) return o.lw + static_cast<size_t>(b) * 12 + n;
    const int nu = 9 * kDT * kNS, ns = 9 * kNS;
    if (n < nu) return o.U + static_cast<size_t>(b) * nu + n;
    if (n < nu + ns) return o.S + static_cast<size_t>(b) * ns + (n - nu);
    return o.V + static_cast<size_t>(b) * nu + (n - nu - ns);
}

// Pooling and the first FC layer of the four heads, one CTA (256 threads) per
// image: rho in shared memory, then each warp reduces 4 of the 32 hidden
// units (lane-strided products, butterfly sum: a fixed order).
__global__ void __launch_bounds__(256) pool_fc1_kernel(const float *__restrict__ r4, HeadW hw, int training,
                                                       uint64_t seed, float *__restrict__ rho,
                                                       float *__restrict__ hidden)
{
    pdl_enter();
    __shared__ float sr[kRho];
    const int b = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const float v = pool_one(r4, b, tid, training, seed);
    sr[tid] = v;
    rho[static_cast<size_t>(b) * kRho + tid] = v;
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int o = warp * 4 + q, h = o >> 3, j = o & 7;
        const float *w = hw.w1[h] + j * kRho;
        float s = 0.f;
#pragma unroll
        for (int i = 0; i < kRho / 32; ++i) s = fmaf(__ldg(w + i * 32 + lane), sr[i * 32 + lane], s);
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
        if (lane == 0) hidden[b * 32 + o] = s + hw.b1[h][j];
    }
}

__global__ void fc2_kernel(const float *__restrict__ hidden, HeadW hw, int B, int ntot, ParamOut o)
{
    pdl_enter();
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < B * ntot; e += gridDim.x * blockDim.x) {
        const int b = e / ntot;
        int n = e - b * ntot, h = 0;
        while (n >= hw.n[h]) n -= hw.n[h++];
        const float *w = hw.w2[h] + static_cast<size_t>(n) * kHidden, *x = hidden + b * 32 + h * 8;
        float s = hw.b2[h][n];
#pragma unroll
        for (int j = 0; j < kHidden; ++j) s = fmaf(w[j], x[j], s);
        *head_dst(o, hw.K, h, b, n) = s;
    }
}

struct HeadGrads {  // where the head weight gradients go (passed by value)
    float *dw2[4], *db2[4], *dw1[4], *db1[4];
};

struct ParamIn {
    const float *U, *S, *V, *lw, *gxy, *gxc, *gyc, *gw;
};

__device__ __forceinline__ float head_src(const ParamIn &i, int K, int h, int b, int n)
{
    ParamOut o{const_cast<float *>(i.U), const_cast<float *>(i.S), const_cast<float *>(i.V), const_cast<float *>(i.lw),
               const_cast<float *>(i.gxy), const_cast<float *>(i.gxc), const_cast<float *>(i.gyc),
               const_cast<float *>(i.gw)};
    return *head_dst(o, K, h, b, n);
}

// dW2, db2: one thread per (h, n, j) (j = hidden unit; j = 0 also takes db2),
// each summing over the batch in order.
__global__ void fc2_wgrad_kernel(const float *__restrict__ hidden, ParamIn d, HeadW hw, int B, int ntot, HeadGrads hg)
{
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < ntot * kHidden; e += gridDim.x * blockDim.x) {
        int n = e / kHidden, h = 0;
        const int j = e - n * kHidden;
        while (n >= hw.n[h]) n -= hw.n[h++];
        float sw = 0.f, sb = 0.f;
#pragma unroll 8
        for (int b = 0; b < B; ++b) {  // unrolled: independent loads in flight, the same order of sums
            const float g = head_src(d, hw.K, h, b, n);
            sb += g;
            sw = fmaf(g, hidden[b * 32 + h * 8 + j], sw);
        }
        if (j == 0) hg.db2[h][n] = sb;
        hg.dw2[h][static_cast<size_t>(n) * kHidden + j] = sw;
    }
}

// dhidden[b][h][j] = sum_n dout[b][h][n] w2[h][n][j]: one CTA per (b, h).
__global__ void __launch_bounds__(256) fc2_dgrad_kernel(ParamIn d, HeadW hw, float *__restrict__ dhid)
{
    __shared__ float red[8];
    const int b = blockIdx.x, h = blockIdx.y;
    float s[kHidden] = {};
#pragma unroll 4
    for (int n = threadIdx.x; n < hw.n[h]; n += 256) {
        const float g = head_src(d, hw.K, h, b, n);
#pragma unroll
        for (int j = 0; j < kHidden; ++j) s[j] = fmaf(g, hw.w2[h][static_cast<size_t>(n) * kHidden + j], s[j]);
    }
#pragma unroll
    for (int j = 0; j < kHidden; ++j) {
        const float t = block_sum256(s[j], red);
        if (threadIdx.x == 0) dhid[b * 32 + h * 8 + j] = t;
    }
}

// dW1, db1 (thread per weight, sum over the batch in order) and drho.
__global__ void fc1_bwd_kernel(const float *__restrict__ rho, const float *__restrict__ dhid, HeadW hw, int B,
                               HeadGrads hg, float *__restrict__ drho)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e < 4 * kHidden * kRho) {
        const int h = e / (kHidden * kRho), r = e - h * kHidden * kRho, j = r / kRho, i = r - j * kRho;
        float s = 0.f;
        for (int b = 0; b < B; ++b) s = fmaf(dhid[b * 32 + h * 8 + j], rho[static_cast<size_t>(b) * kRho + i], s);
        hg.dw1[h][r] = s;
        if (i == 0) {
            float sb = 0.f;
            for (int b = 0; b < B; ++b) sb += dhid[b * 32 + h * 8 + j];
            hg.db1[h][j] = sb;
        }
    }
    if (e < B * kRho) {
        const int b = e / kRho, i = e - b * kRho;
        float s = 0.f;
        for (int h = 0; h < 4; ++h)
            for (int j = 0; j < kHidden; ++j) s = fmaf(dhid[b * 32 + h * 8 + j], hw.w1[h][j * kRho + i], s);
        drho[e] = s;
    }
}

// pooling, dropout and LeakyReLU backward: dz4 [B][64][8][8]
__global__ void pool_bwd_kernel(const float *__restrict__ drho, const float *__restrict__ r4, int B, int training,
                                uint64_t seed, float *__restrict__ dz)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= B * 64 * 64) return;
    const int b = e / 4096, r = e - b * 4096, c = r >> 6, y = (r >> 3) & 7, x = r & 7;
    const float g = drho[b * kRho + c * 4 + (y >> 2) * 2 + (x >> 2)] * (1.f / 16.f);
    dz[e] = g * drop_scale(training, seed, e) * (r4[e] > 0.f ? 1.f : kSlope);
}

// Sum of the partial weight gradients over chunks: one warp per output, lane
// l adds chunks l, l + 32, ... in order, then a butterfly (a fixed order).
// Partials are [chunks][N][Kd + 1]; column Kd is the bias gradient.
__global__ void wgrad_reduce_kernel(const float *__restrict__ part, int chunks, int N, int Kd, float *__restrict__ dw,
                                    float *__restrict__ db)
{
    const int lane = threadIdx.x & 31;
    const int e = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, n_out = N * (Kd + 1);
    if (e >= n_out) return;  // whole warps leave together
    float s = 0.f;
    for (int z = lane; z < chunks; z += 32) s += __ldg(part + static_cast<size_t>(z) * n_out + e);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) {
        const int i = e / (Kd + 1), j = e - i * (Kd + 1);
        if (j < Kd) dw[i * Kd + j] = s;
        else db[i] = s;
    }
}

// InstanceNorm backward, pass 1 (one CTA per (b, c)): s1 = sum dA xh, s2 = sum dA
__global__ void __launch_bounds__(256) in_bwd_sums_kernel(const float *__restrict__ da, const float *__restrict__ r,
                                                          const float *mean, const float *rstd, int HW, float *sums)
{
    __shared__ float red[8];
    const size_t o = static_cast<size_t>(blockIdx.x) * HW;
    const float mu = mean[blockIdx.x], rs = rstd[blockIdx.x];
    float s1 = 0.f, s2 = 0.f;
    for (int i = threadIdx.x; i < HW; i += 256) {
        const float g = da[o + i];
        s1 = fmaf(g, (r[o + i] - mu) * rs, s1);
        s2 += g;
    }
    const float t1 = block_sum256(s1, red);
    const float t2 = block_sum256(s2, red);
    if (threadIdx.x == 0) {
        sums[2 * blockIdx.x] = t1;
        sums[2 * blockIdx.x + 1] = t2;
    }
}

// pass 2: dz = LeakyReLU'(r) * rstd * gamma * (dA - s2/n - xh s1/n)
// Four elements per thread (HW % 4 == 0: one plane per quad; float4 I/O).
__global__ void in_bwd_apply_kernel(const float *__restrict__ da, const float *__restrict__ r, const float *mean,
                                    const float *rstd, const float *gam, const float *sums, int C, int HW, size_t n,
                                    float *__restrict__ dz)
{
    const float inv = 1.f / HW;
    const size_t n4 = n / 4;
    for (size_t e4 = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; e4 < n4;
         e4 += static_cast<size_t>(gridDim.x) * blockDim.x) {
        const unsigned int bc = static_cast<unsigned int>(4 * e4 / static_cast<unsigned int>(HW));
        const int c = static_cast<int>(bc % static_cast<unsigned int>(C));
        const float rs = rstd[bc], mu = mean[bc], g = rs * gam[c];
        const float s0 = sums[2 * bc], s1 = sums[2 * bc + 1];
        const float4 a = reinterpret_cast<const float4 *>(da)[e4], x = reinterpret_cast<const float4 *>(r)[e4];
        const float av[4] = {a.x, a.y, a.z, a.w}, xv[4] = {x.x, x.y, x.z, x.w};
        float o[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const float xh = (xv[u] - mu) * rs;
            const float dr = g * (av[u] - s1 * inv - xh * s0 * inv);
            o[u] = xv[u] > 0.f ? dr : kSlope * dr;
        }
        reinterpret_cast<float4 *>(dz)[e4] = make_float4(o[0], o[1], o[2], o[3]);
    }
}

// dgamma[c], dbeta[c] = sums over the batch (in order)
__global__ void in_param_grad_kernel(const float *sums, int B, int C, float *dg, float *db)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= C) return;
    float a = 0.f, b2 = 0.f;
    for (int b = 0; b < B; ++b) {
        a += sums[2 * (b * C + c)];
        b2 += sums[2 * (b * C + c) + 1];
    }
    dg[c] = a;
    db[c] = b2;
}

__global__ void adam_kernel(float *w, const float *__restrict__ g, float *m, float *v, size_t n, float lr, float b1,
                            float b2, float eps, float c1, float c2)
{
    for (size_t e = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; e < n;
         e += static_cast<size_t>(gridDim.x) * blockDim.x) {
        const float gg = g[e];
        const float mm = b1 * m[e] + (1.f - b1) * gg;
        const float vv = b2 * v[e] + (1.f - b2) * gg * gg;
        m[e] = mm;
        v[e] = vv;
        w[e] -= lr * (mm / c1) / (sqrtf(vv / c2) + eps);
    }
}

// MSE loss (Eq. 11, first term): per-CTA partial sums of (y - t)^2 and the
// gradient dy = 2 (y - t) / n; partials are summed in order by mse_final.
__global__ void __launch_bounds__(256) mse_kernel(const float *__restrict__ y, const float *__restrict__ t, size_t n,
                                                  float *__restrict__ dy, float *__restrict__ part)
{
    __shared__ float red[8];
    const float sc = 2.f / static_cast<float>(n);
    float s = 0.f;
    for (size_t e = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; e < n;
         e += static_cast<size_t>(gridDim.x) * blockDim.x) {
        const float d = y[e] - t[e];
        s = fmaf(d, d, s);
        if (dy) dy[e] = sc * d;
    }
    const float tot = block_sum256(s, red);
    if (threadIdx.x == 0) part[blockIdx.x] = tot;
}

__global__ void mse_final_kernel(const float *part, int nb, size_t n, float *loss)
{
    // one warp: lane l adds partials l, l + 32, ... in double, then a butterfly
    const int lane = threadIdx.x & 31;
    double s = 0.0;
    for (int i = lane; i < nb; i += 32) s += part[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) *loss = static_cast<float>(s / static_cast<double>(n));
}

inline int blocks_for(size_t n, int t = 256) { return static_cast<int>(std::min<size_t>((n + t - 1) / t, 152 * 8)); }

inline HeadW head_weights(const float *w, const Layout &L, int K)
{
    HeadW h{};
    for (int i = 0; i < 4; ++i) {
        h.w1[i] = w + L.w1[i];
        h.b1[i] = w + L.b1[i];
        h.w2[i] = w + L.w2[i];
        h.b2[i] = w + L.b2[i];
        h.n[i] = L.head_n[i];
    }
    h.K = K;
    return h;
}

}  // namespace gen
}  // namespace svdlut

extern "C" svdlut_status svdlut_tensor_core_timeouts(uint32_t *count)
{
    svdlut::clear_error();
    if (!count) return svdlut::fail(SVDLUT_ERR_INVALID_ARG, "count is NULL");
    unsigned int h = 0;
    const unsigned int zero = 0;
    SVDLUT_CUDA_TRY(cudaDeviceSynchronize());
    SVDLUT_CUDA_TRY(cudaMemcpyFromSymbol(&h, svdlut::gen::g_umma_timeouts, sizeof h));
    SVDLUT_CUDA_TRY(cudaMemcpyToSymbol(svdlut::gen::g_umma_timeouts, &zero, sizeof zero));
    *count = h;
    return SVDLUT_OK;
}

using namespace svdlut;
using namespace svdlut::gen;

extern "C" size_t svdlut_generator_param_count(int K)
{
    if (K < 0 || K > kMaxK) return 0;
    return make_layout(K).total;
}

extern "C" size_t svdlut_generator_workspace_size(int K, int B)
{
    if (K < 0 || K > kMaxK || B < 1) return 0;
    return make_ws(B).total * sizeof(float);
}

static svdlut_status gen_check(int K, const float *weights, int B, void *ws, size_t ws_bytes)
{
    if (K < 0 || K > kMaxK) return fail(SVDLUT_ERR_INVALID_ARG, "K=%d out of [0, %d]", K, kMaxK);
    if (B < 1) return fail(SVDLUT_ERR_INVALID_ARG, "B=%d must be >= 1", B);
    if (!weights) return fail(SVDLUT_ERR_INVALID_ARG, "weights is NULL");
    if (!ws || ws_bytes < svdlut_generator_workspace_size(K, B))
        return fail(SVDLUT_ERR_WORKSPACE, "generator workspace of %zu bytes needed",
                    svdlut_generator_workspace_size(K, B));
    if (!aligned(ws, 256) || !aligned(weights, 4)) return fail(SVDLUT_ERR_INVALID_ARG, "misaligned weights or workspace");
    return SVDLUT_OK;
}

extern "C" svdlut_status svdlut_generator_forward(int K, const float *weights, int B, int H, int W, const float *x,
                                                  const svdlut_param_buffers *out, int training, uint64_t seed,
                                                  void *ws, size_t ws_bytes, svdlut_stream_t stream)
{
    SVDLUT_TRACE("svdlut_generator_forward");
    clear_error();
    svdlut_status st = gen_check(K, weights, B, ws, ws_bytes);
    if (st != SVDLUT_OK) return st;
    if (!x || !out || H < 1 || W < 1) return fail(SVDLUT_ERR_INVALID_ARG, "x/out missing or H=%d W=%d", H, W);
    if (!out->U || !out->S || !out->V || !out->lut_w || (K > 0 && (!out->g_xy || !out->g_xc || !out->g_yc || !out->grid_w)))
        return fail(SVDLUT_ERR_INVALID_ARG, "every output buffer is required");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const Layout L = make_layout(K);
    const WsLayout wl = make_ws(B);
    float *w = static_cast<float *>(ws);
    // a chain of small kernels, each a programmatic dependent launch of the one before
    if ((st = launch_pdl(downsample_kernel, dim3(static_cast<int>((static_cast<size_t>(B) * 3 * kThumb * kThumb / 4 + 255) / 256)),
                         dim3(256), 0, s, x, B, H, W, w + wl.thumb)) != SVDLUT_OK)
        return st;
    {  // the convolutions' weights in the tensor cores' B layout
        WPrep wp{};
        int e = 0;
        for (int i = 0; i < 5; ++i) {
            wp.w[i] = weights + L.conv_w[i];
            wp.out[i] = reinterpret_cast<__nv_bfloat16 *>(w + wl.wbf[i]);
            wp.cin[i] = kCh[i];
            wp.cout[i] = kCh[i + 1];
            wp.np[i] = wgrad_np(kCh[i + 1]);
            wp.kpad[i] = conv_stages(i) * 64;
            wp.start[i] = e;
            e += static_cast<int>(conv_wbf_elems(i));
        }
        wp.start[5] = e;
        if ((st = launch_pdl(conv_wprep_kernel, dim3((e + 255) / 256), dim3(256), 0, s, wp)) != SVDLUT_OK) return st;
    }
    const float *in = w + wl.thumb, *isc = nullptr, *ish = nullptr;
    for (int i = 0; i < 5; ++i) {
        const int Cin = kCh[i], Cout = kCh[i + 1], S = kSz[i], So = kSz[i + 1];
        const int M = B * So * So, Kd = Cin * 9, Z = conv_split(B, i), P = So * So;
        float *r = w + wl.r[i];
        const bool norm = i < 4, fuse = norm && Z == 1 && P % 128 == 0;
        const float *gam = norm ? weights + L.in_g[i] : nullptr, *bet = norm ? weights + L.in_b[i] : nullptr;
        float *mean = norm ? w + wl.mean[i] : nullptr, *rstd = norm ? w + wl.rstd[i] : nullptr;
        float *scn = norm ? w + wl.sc[i] : nullptr, *shn = norm ? w + wl.sh[i] : nullptr;
        if ((st = launch_conv(ConvUmma{in, isc, ish, reinterpret_cast<const uint4 *>(w + wl.wbf[i]), w + wl.part, Cin,
                                       S, So, Cout, M, Kd, conv_ks(B, i), weights + L.conv_b[i], fuse ? r : nullptr,
                                       w + wl.tstat},
                              Z, s)) != SVDLUT_OK)
            return st;
        if (fuse) {
            st = launch_pdl(conv_stats_kernel, dim3((B * Cout * 32 + 255) / 256), dim3(256), 0, s,
                            static_cast<const float *>(w + wl.tstat), B, Cout, P / 128, P, gam, bet, mean, rstd, scn, shn);
        } else {
            const float *part = w + wl.part, *bias = weights + L.conv_b[i];
            st = P >= 4096 ? launch_pdl(conv_finish_kernel<512>, dim3(B * Cout), dim3(512), 0, s, part, Z, Cout, M, P,
                                        bias, r, gam, bet, mean, rstd, scn, shn)
               : P >= 1024 ? launch_pdl(conv_finish_kernel<256>, dim3(B * Cout), dim3(256), 0, s, part, Z, Cout, M, P,
                                        bias, r, gam, bet, mean, rstd, scn, shn)
                           : launch_pdl(conv_finish_kernel<64>, dim3(B * Cout), dim3(64), 0, s, part, Z, Cout, M, P,
                                        bias, r, gam, bet, mean, rstd, scn, shn);
        }
        if (st != SVDLUT_OK) return st;
        in = r;
        if (norm) {
            isc = w + wl.sc[i];
            ish = w + wl.sh[i];
        }
    }
    const HeadW hw = head_weights(weights, L, K);
    if ((st = launch_pdl(pool_fc1_kernel, dim3(B), dim3(256), 0, s, static_cast<const float *>(w + wl.r[4]), hw,
                         training, seed, w + wl.rho, w + wl.hidden)) != SVDLUT_OK)
        return st;
    const int ntot = L.head_n[0] + L.head_n[1] + L.head_n[2] + L.head_n[3];
    ParamOut po{out->U, out->S, out->V, out->lut_w, out->g_xy, out->g_xc, out->g_yc, out->grid_w};
    if ((st = launch_pdl(fc2_kernel, dim3(blocks_for(static_cast<size_t>(B) * ntot)), dim3(256), 0, s,
                         static_cast<const float *>(w + wl.hidden), hw, B, ntot, po)) != SVDLUT_OK)
        return st;
    return SVDLUT_OK;
}

extern "C" svdlut_status svdlut_generator_backward(int K, const float *weights, int B, const svdlut_params *dparams,
                                                   float *dweights, int training, uint64_t seed, void *ws,
                                                   size_t ws_bytes, svdlut_stream_t stream)
{
    SVDLUT_TRACE("svdlut_generator_backward");
    clear_error();
    svdlut_status st = gen_check(K, weights, B, ws, ws_bytes);
    if (st != SVDLUT_OK) return st;
    if (!dparams || !dweights) return fail(SVDLUT_ERR_INVALID_ARG, "dparams and dweights are required");
    if (!dparams->U || !dparams->S || !dparams->V || !dparams->lut_w ||
        (K > 0 && (!dparams->g_xy || !dparams->g_xc || !dparams->g_yc || !dparams->grid_w)))
        return fail(SVDLUT_ERR_INVALID_ARG, "every output gradient is required");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const Layout L = make_layout(K);
    const WsLayout wl = make_ws(B);
    float *w = static_cast<float *>(ws);
    HeadGrads hg{};
    for (int h = 0; h < 4; ++h) {
        hg.dw2[h] = dweights + L.w2[h];
        hg.db2[h] = dweights + L.b2[h];
        hg.dw1[h] = dweights + L.w1[h];
        hg.db1[h] = dweights + L.b1[h];
    }
    const HeadW hw = head_weights(weights, L, K);
    const ParamIn pin{dparams->U, dparams->S, dparams->V, dparams->lut_w, dparams->g_xy, dparams->g_xc,
                      dparams->g_yc, dparams->grid_w};
    const int ntot = L.head_n[0] + L.head_n[1] + L.head_n[2] + L.head_n[3];
    fc2_wgrad_kernel<<<blocks_for(static_cast<size_t>(ntot) * kHidden), 256, 0, s>>>(w + wl.hidden, pin, hw, B, ntot,
                                                                                    hg);
    fc2_dgrad_kernel<<<dim3(B, 4), 256, 0, s>>>(pin, hw, w + wl.dhid);
    fc1_bwd_kernel<<<(std::max(4 * kHidden * kRho, B * kRho) + 255) / 256, 256, 0, s>>>(
        w + wl.rho, w + wl.dhid, hw, B, hg, w + wl.drho);
    {  // the input-gradient weights of layers 1..4 in the tensor cores' B layout
        DPrep dp{};
        int e = 0;
        for (int l = 0; l < 4; ++l) {
            const int i = l + 1;
            dp.w[l] = weights + L.conv_w[i];
            dp.cin[l] = kCh[i];
            dp.cout[l] = kCh[i + 1];
            dp.np[l] = wgrad_np(kCh[i]);
            __nv_bfloat16 *base = reinterpret_cast<__nv_bfloat16 *>(w + wl.dgw[i]);
            for (int c = 0; c < 4; ++c) {
                const int g = 4 * l + c;
                dp.kpad[g] = dgrad_kpad(i, c);
                dp.seg[g] = base;
                base += static_cast<size_t>(2) * dp.np[l] * dp.kpad[g];
                dp.start[g] = e;
                e += dp.np[l] * dp.kpad[g];
            }
        }
        dp.start[16] = e;
        dgrad_wprep_kernel<<<(e + 255) / 256, 256, 0, s>>>(dp);
    }
    float *dz = w + wl.dz[0];
    pool_bwd_kernel<<<(B * 4096 + 255) / 256, 256, 0, s>>>(w + wl.drho, w + wl.r[4], B, training, seed, dz);
    SVDLUT_CUDA_TRY(cudaGetLastError());
    for (int i = 4; i >= 0; --i) {
        const int Cin = kCh[i], Cout = kCh[i + 1], S = kSz[i], So = kSz[i + 1];
        const int pix = B * So * So, Kd = Cin * 9, chunk = wgrad_chunk_px(B, i), chunks = wgrad_chunks(B, i);
        // weight and bias gradient: partial per pixel chunk (bias = an extra
        // all-ones im2col column), then an ordered sum
        const WgradArgs wa{i == 0 ? w + wl.thumb : w + wl.r[i - 1], i == 0 ? nullptr : w + wl.sc[i - 1],
                           i == 0 ? nullptr : w + wl.sh[i - 1], dz, w + wl.wpart, Cin, Cout, S, So, pix, chunk};
        const int np = wgrad_np_layer(i), tiles = wgrad_tiles(i), sets = wgrad_sets(i);
        if (sets == 4)
            st = np == 16 ? launch_wgrad<16, 4>(wa, tiles, chunks, s) : launch_wgrad<32, 4>(wa, tiles, chunks, s);
        else
            st = np == 16 ? launch_wgrad<16, 1>(wa, tiles, chunks, s)
                          : np == 32 ? launch_wgrad<32, 1>(wa, tiles, chunks, s) : launch_wgrad<64, 1>(wa, tiles, chunks, s);
        if (st != SVDLUT_OK) return st;
        wgrad_reduce_kernel<<<(Cout * (Kd + 1) * 32 + 255) / 256, 256, 0, s>>>(
            w + wl.wpart, chunks * sets, Cout, Kd, dweights + L.conv_w[i], dweights + L.conv_b[i]);
        SVDLUT_CUDA_TRY(cudaGetLastError());
        if (i == 0) break;
        // input gradient, then InstanceNorm + LeakyReLU backward of layer i-1
        float *dact = w + wl.dact;
        {
            DgradUmma da{dz, reinterpret_cast<const uint4 *>(w + wl.dgw[i]), dact, Cout, Cin, So, B * So * So,
                         31 - __builtin_clz(static_cast<unsigned>(Cout)), {}, {}};
            size_t off = 0;
            for (int c = 0; c < 4; ++c) {
                da.cls_off[c] = static_cast<int>(off / 8);  // uint4 units
                da.kpad[c] = dgrad_kpad(i, c);
                off += static_cast<size_t>(2) * wgrad_np(Cin) * da.kpad[c];
            }
            const int np = wgrad_np(Cin);
            st = np == 16 ? launch_dgrad_t<16, 1>(da, s)
                          : np == 32 ? launch_dgrad_t<32, 1>(da, s) : launch_dgrad_t<64, 2>(da, s);
            if (st != SVDLUT_OK) return st;
        }
        const int j = i - 1;
        float *dz_next = dz == w + wl.dz[0] ? w + wl.dz[1] : w + wl.dz[0];
        in_bwd_sums_kernel<<<B * Cin, 256, 0, s>>>(dact, w + wl.r[j], w + wl.mean[j], w + wl.rstd[j], S * S,
                                                   w + wl.insum);
        const size_t n = act_size(B, j);
        in_bwd_apply_kernel<<<blocks_for(n / 4), 256, 0, s>>>(dact, w + wl.r[j], w + wl.mean[j], w + wl.rstd[j],
                                                          weights + L.in_g[j], w + wl.insum, Cin, S * S, n, dz_next);
        in_param_grad_kernel<<<1, 64, 0, s>>>(w + wl.insum, B, Cin, dweights + L.in_g[j], dweights + L.in_b[j]);
        SVDLUT_CUDA_TRY(cudaGetLastError());
        dz = dz_next;
    }
    return SVDLUT_OK;
}

extern "C" svdlut_status svdlut_generator_adam(float *weights, const float *grads, float *m, float *v, size_t n,
                                               float lr, float beta1, float beta2, float eps, int step,
                                               svdlut_stream_t stream)
{
    SVDLUT_TRACE("svdlut_generator_adam");
    clear_error();
    if (!weights || !grads || !m || !v || n == 0 || step < 1)
        return fail(SVDLUT_ERR_INVALID_ARG, "adam: null buffer, n = 0 or step < 1");
    const float c1 = 1.f - powf(beta1, static_cast<float>(step));
    const float c2 = 1.f - powf(beta2, static_cast<float>(step));
    adam_kernel<<<blocks_for(n), 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(weights, grads, m, v, n, lr, beta1,
                                                                                    beta2, eps, c1, c2);
    SVDLUT_CUDA_TRY(cudaGetLastError());
    return SVDLUT_OK;
}

extern "C" svdlut_status svdlut_mse(const float *y, const float *target, size_t n, float *dy, float *loss, void *ws,
                                    size_t ws_bytes, svdlut_stream_t stream)
{
    SVDLUT_TRACE("svdlut_mse");
    clear_error();
    if (!y || !target || !loss || n == 0) return fail(SVDLUT_ERR_INVALID_ARG, "mse: null buffer or n = 0");
    const int nb = std::min(blocks_for(n), 1024);
    if (!ws || ws_bytes < sizeof(float) * static_cast<size_t>(nb))
        return fail(SVDLUT_ERR_WORKSPACE, "mse: workspace of %zu bytes needed", sizeof(float) * static_cast<size_t>(1024));
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    float *part = static_cast<float *>(ws);
    mse_kernel<<<nb, 256, 0, s>>>(y, target, n, dy, part);
    mse_final_kernel<<<1, 32, 0, s>>>(part, nb, n, loss);
    SVDLUT_CUDA_TRY(cudaGetLastError());
    return SVDLUT_OK;
}
