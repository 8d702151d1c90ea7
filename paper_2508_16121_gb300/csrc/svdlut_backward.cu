// svdlut_backward: adjoint of the fused transform (FP32 images).
//
// The paper trains end to end through its slicing + LUT transform (Sec. 4.2)
// and prints no derivative; everything here is the exact derivative of the
// forward map of Eq. 10 / Supp. Eqs. 12-22.  Passes (all on the caller's
// stream, no atomics, every sum in a fixed order -> bitwise repeatable):
//   1. dx      : apply_kernel<IoF32, N, true> (slopes of the same cells).
//   2. lut     : lut_grad_kernel scatters dy * bilinear weights into
//                warp-private tables G_p[i][j][c] (one LUT pair, all three
//                output channels per warp: one key match per pixel and pair),
//                then sums the warps of a CTA into a per-CTA partial.
//   3. grid    : grid_grad_kernel does the same for the folded grid planes
//                (xy, xc, yc per output channel) over 128-px column blocks.
//   4. reduce  : lut_finalize_kernel sums the CTA partials and contracts
//                through T = U diag(S) V^T (Eq. 9) to dU, dS, dV, dlut_w;
//                grid_reduce_kernel sums the block partials per vertex into dg_*
//                and per-CTA partials of dgrid_w, grid_wsum_kernel sums those.
#include <algorithm>
#include <mutex>
#include <utility>
#include <vector>
#include <cmath>

#include "apply_kernel.cuh"
#include "apply_launch.cuh"

namespace svdlut {

// ---------------------------------------------------------------------------
// deterministic warp scatter
// ---------------------------------------------------------------------------

// Position of the n-th (0-based) set bit of m (m has more than n set bits).
__device__ __forceinline__ int nth_set_bit(unsigned int m, int n)
{
    int p = 0;
#pragma unroll
    for (int w = 16; w >= 1; w >>= 1) {
        const unsigned int lo = p + w >= 32 ? 0xffffffffu : ((1u << (p + w)) - 1u);
        if (__popc(m & lo) <= n) p += w;
    }
    return p;
}

// Adds v[corner][ch] to tab[key + off(corner) + ch], corner offsets
// (0, ld, cs, ld + cs) for the (00, 10, 01, 11) corners of a bilinear cell.
// Lanes with equal keys are first summed by a shuffle tree over their ranks
// in the group (fixed order); the lowest lane of each group then writes, one
// corner at a time with a warp barrier between corners, so two groups never
// update one address in the same step.  key < 0 marks an inactive lane.
// Every lane of the warp must call this.  VEC: every key's NC <= 3 values sit
// in one 16-byte slot (tab, key, ld and cs multiples of 4 floats), updated
// with one 16-byte load and store.
template <int NC, bool VEC = false>
__device__ __forceinline__ void warp_scatter(float *tab, int key, int ld, int cs, float (&v)[4][NC])
{
    const unsigned int full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const unsigned int me = 1u << lane;
    const int k = key >= 0 ? key : -1 - lane;
    const unsigned int grp = __match_any_sync(full, k);
    if (!__all_sync(full, grp == me)) {
        if (__all_sync(full, grp == full)) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1)
#pragma unroll
                for (int q = 0; q < 4; ++q)
#pragma unroll
                    for (int c = 0; c < NC; ++c) v[q][c] += __shfl_xor_sync(full, v[q][c], o);
        } else {
            const int rank = __popc(grp & (me - 1));
            const int size = __popc(grp);
            const int maxsize = static_cast<int>(__reduce_max_sync(full, static_cast<unsigned int>(size)));
            for (int s = 1; s < maxsize; s <<= 1) {
                const int src_rank = rank + s;
                const bool take = (rank & (2 * s - 1)) == 0 && src_rank < size;
                const int src = take ? nth_set_bit(grp, src_rank) : lane;
#pragma unroll
                for (int q = 0; q < 4; ++q)
#pragma unroll
                    for (int c = 0; c < NC; ++c) {
                        const float o = __shfl_sync(full, v[q][c], src);
                        if (take) v[q][c] += o;
                    }
            }
        }
    }
    const bool leader = key >= 0 && (grp & (me - 1)) == 0;
    const int off[4] = {0, ld, cs, ld + cs};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        if (leader) {
            if constexpr (VEC) {
                static_assert(NC <= 3, "one 16-byte slot per key");
                float4 *t = reinterpret_cast<float4 *>(tab + key + off[q]);
                float4 o = *t;
                o.x += v[q][0];
                if constexpr (NC > 1) o.y += v[q][1];
                if constexpr (NC > 2) o.z += v[q][2];
                *t = o;
            } else {
                float *t = tab + key + off[q];
#pragma unroll
                for (int c = 0; c < NC; ++c) t[c] += v[q][c];
            }
        }
        __syncwarp();
    }
}

// Fixed-order warp sum (butterfly); every lane gets the total.
__device__ __forceinline__ float warp_sum(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

constexpr int kLutWarps = 12;  // 4 groups x 3 LUT pairs
constexpr int kLutThreads = kLutWarps * 32;

struct BwdArgs {
    const float *x, *dy;
    int B, H, W;
    int D, K, Dsx, Dsy, Dsc;
    float rW1, rH1;
    int strips;
    int vec;  // 16-byte loads allowed
};

// ---------------------------------------------------------------------------
// LUT gradients: G^c_p[i][j] = sum_px dy_c * bilinear weight of vertex (i, j)
// at (x_alpha, x_beta) for pair p = (alpha, beta).
// grid (P, B); CTA (p, b) owns the rows [p H / P, (p+1) H / P) of image b.
// Its work is the sequence of (128-column strip, row) pairs, strip by strip;
// warp group g takes the g-th quarter of it (equal shares to within one row,
// whatever the number of strips: a piece of a strip, whole strips, a piece of
// the next).  Warp (group g, pair q) walks down the rows of each of its
// pieces; lane l takes columns l + 32 k (k = 0..3: coalesced loads) and
// keeps, per column, the four corner contributions
// (three channels each) of its current cell in registers: while the cell
// does not change (smooth regions, where consecutive rows fall in the same
// cell) it only accumulates; when it changes, the warp scatters the finished
// sums into its private table [D][D][3 channels + 1 pad] (deterministic
// warp_scatter).  Rows are loaded two ahead.
// Output: lut_part[b][p][c][pair][D*D], sums_part[b][p][c] (sum of dy_c).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kLutThreads, 1)
    lut_grad_kernel(BwdArgs a, float *__restrict__ lut_part, float *__restrict__ sums_part)
{
    extern __shared__ __align__(16) float sm[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int grp = warp / 3, pair = warp - grp * 3;
    const int A = pair == 2 ? 1 : 0, Bx = pair == 0 ? 1 : 2;  // axes of the pair
    const int P = gridDim.x, p = blockIdx.x, b = blockIdx.y;
    const int D = a.D, DD = D * D;
    float *tab = sm + warp * 4 * DD;  // [D][D][3 channels + 1 pad] of this warp's pair
    float *sums = sm + kLutWarps * 4 * DD;
    for (int e = threadIdx.x; e < kLutWarps * 4 * DD; e += kLutThreads) sm[e] = 0.f;
    __syncthreads();

    const int r0 = static_cast<int>((static_cast<long long>(a.H) * p) / P);
    const int r1 = static_cast<int>((static_cast<long long>(a.H) * (p + 1)) / P);
    constexpr int kGroups = kLutWarps / 3;
    const size_t plane = static_cast<size_t>(a.H) * a.W;
    const float *xb = a.x + static_cast<size_t>(b) * 3 * plane;
    const float *gb = a.dy + static_cast<size_t>(b) * 3 * plane;
    const float fD1 = static_cast<float>(D - 1), fD2 = static_cast<float>(D - 2);
    float dysum[3] = {0.f, 0.f, 0.f};
    float acc[4][4][3];  // [column k][corner][channel]
    int acc_key[4] = {-1, -1, -1, -1};
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
            for (int c = 0; c < 3; ++c) acc[k][q][c] = 0.f;
    const long long nrows = r1 - r0, T = static_cast<long long>(a.strips) * nrows;
    const long long t1 = T * (grp + 1) / kGroups;
    for (long long t = T * grp / kGroups; t < t1;) {
        const int strip = static_cast<int>(t / nrows);
        const long long s0 = strip * nrows;
        const int ra = r0 + static_cast<int>(t - s0), rb = r0 + static_cast<int>(min(t1 - s0, nrows));
        t = s0 + nrows;
        const int x = strip * kTileW + lane;
        const int n = x < a.W ? min(4, (a.W - x + 31) >> 5) : 0;  // this lane's columns x + 32 k, k < n
        struct Row {
            float4 pa, pb, g0, g1, g2;
        };
        auto load = [&](int r, Row &o) {
            const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
            o.pa = o.pb = o.g0 = o.g1 = o.g2 = z;
            if (r < rb && n > 0) {
                const size_t off = static_cast<size_t>(r) * a.W + x;
                o.pa = PixIO<float>::load_s(xb + A * plane + off, n);
                o.pb = PixIO<float>::load_s(xb + Bx * plane + off, n);
                o.g0 = PixIO<float>::load_s(gb + off, n);
                o.g1 = PixIO<float>::load_s(gb + plane + off, n);
                o.g2 = PixIO<float>::load_s(gb + 2 * plane + off, n);
            }
        };
        Row cur, nx1, nx2;
        load(ra, cur);
        load(ra + 1, nx1);
        for (int r = ra; r < rb; ++r) {
            load(r + 2, nx2);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const bool act = k < n;
                const float gy[3] = {get(cur.g0, k), get(cur.g1, k), get(cur.g2, k)};
#pragma unroll
                for (int c = 0; c < 3; ++c) dysum[c] += gy[c];
                float da, db;
                const int ia = cell_of(fminf(fmaxf(get(cur.pa, k), 0.f), 1.f), fD1, fD2, da);
                const int ib = cell_of(fminf(fmaxf(get(cur.pb, k), 0.f), 1.f), fD1, fD2, db);
                const float w[4] = {(1.f - da) * (1.f - db), da * (1.f - db), (1.f - da) * db, da * db};
                const int key = act ? (ia * D + ib) * 4 : -1;
                const bool change = key != acc_key[k];
                if (__any_sync(0xffffffffu, change))
                    warp_scatter<3, true>(tab, change ? acc_key[k] : -1, D * 4, 4, acc[k]);
                if (change) {
#pragma unroll
                    for (int q = 0; q < 4; ++q)
#pragma unroll
                        for (int c = 0; c < 3; ++c) acc[k][q][c] = gy[c] * w[q];
                    acc_key[k] = key;
                } else {
#pragma unroll
                    for (int q = 0; q < 4; ++q)
#pragma unroll
                        for (int c = 0; c < 3; ++c) acc[k][q][c] = fmaf(gy[c], w[q], acc[k][q][c]);
                }
            }
            cur = nx1;
            nx1 = nx2;
        }
        // the piece's runs end here
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            warp_scatter<3, true>(tab, acc_key[k], D * 4, 4, acc[k]);
            acc_key[k] = -1;
        }
    }
    // sum of dy_c: the pair-0 warps' totals (every pair warp of a group sees the same pixels)
#pragma unroll
    for (int c = 0; c < 3; ++c) dysum[c] = warp_sum(dysum[c]);
    if (lane == 0 && pair == 0) {
        sums[grp * 3 + 0] = dysum[0];
        sums[grp * 3 + 1] = dysum[1];
        sums[grp * 3 + 2] = dysum[2];
    }
    __syncthreads();
    // CTA partial [c][pair][cell]: sum the groups in order
    float *out = lut_part + (static_cast<size_t>(b) * P + p) * 9 * DD;
    for (int e = threadIdx.x; e < 9 * DD; e += kLutThreads) {
        const int c = e / (3 * DD), r = e - c * 3 * DD, q = r / DD, cell = r - q * DD;
        float s = 0.f;
        for (int gq = 0; gq < kGroups; ++gq) s += sm[(gq * 3 + q) * 4 * DD + cell * 4 + c];
        out[e] = s;
    }
    if (threadIdx.x < 3) {
        float s = 0.f;
        for (int gq = 0; gq < kGroups; ++gq) s += sums[gq * 3 + threadIdx.x];
        sums_part[(static_cast<size_t>(b) * P + p) * 3 + threadIdx.x] = s;
    }
}

// ---------------------------------------------------------------------------
// grid gradients per output channel c (folded planes F_c = sum_{k=c mod 3}
// w_k g_k): dFxy_c[iy][ix], dFxc_c[ix][j], dFyc_c[iy][j] = scatters of dy_c.
// Blocks: 128-px column strip x BH rows (host plan); warp w owns a contiguous
// run of rows.  Output per block: xy [nvy][nvx][3], xc [3][nvx][Dsc],
// yc [3][nvy][Dsc] in block-local indexing.
// ---------------------------------------------------------------------------
struct GridPlan {
    int BH, bands, nblk;   // per image
    int nvx, nvy, rpw, nvyw;  // maxima
    int blk_stride;        // floats per block partial
    int bins;              // 1: yc through lane-private bins, 0: warp scatter (large Dsc)
};

// Per-warp floats: the xy, xc and yc tables, then the lane-private yc bins
// [3][Dsc][33] (one column per lane, padded so that a lane summing a row of
// bins reads 32 different banks).
__host__ __device__ inline int grid_table_floats(int nvx, int nvyw, int Dsc)
{
    return (3 * nvyw * nvx + 3 * nvx * Dsc + 3 * nvyw * Dsc + 3) & ~3;
}
__host__ __device__ inline int grid_warp_floats(int nvx, int nvyw, int Dsc, int bins)
{
    return grid_table_floats(nvx, nvyw, Dsc) + (bins ? 3 * Dsc * 33 : 0);
}

__host__ __device__ inline int grid_block_floats(int nvx, int nvy, int Dsc)
{
    return 3 * nvy * nvx + 3 * nvx * Dsc + 3 * nvy * Dsc;
}

__global__ void __launch_bounds__(kThreads, 1)
    grid_grad_kernel(BwdArgs a, GridPlan gp, float *__restrict__ grid_part)
{
    extern __shared__ __align__(16) float sm[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int b = blockIdx.y, lb = blockIdx.x;
    const int band = lb / a.strips, strip = lb - band * a.strips;
    const int x0 = strip * kTileW, y0 = band * gp.BH;
    const int rows = min(gp.BH, a.H - y0);
    if (rows <= 0) return;
    const int Dsc = a.Dsc, Dc2 = Dsc - 2;
    // block footprint
    int ixlo, ixhi, iylo, iyhi;
    float t;
    spatial_cell(x0, a.W, a.Dsx, a.rW1, ixlo, t);
    spatial_cell(min(x0 + kTileW - 1, a.W - 1), a.W, a.Dsx, a.rW1, ixhi, t);
    spatial_cell(y0, a.H, a.Dsy, a.rH1, iylo, t);
    spatial_cell(y0 + rows - 1, a.H, a.Dsy, a.rH1, iyhi, t);
    const int nvx = min(min(ixhi + 1, a.Dsx - 1) - ixlo + 1, gp.nvx);
    const int nvy = min(min(iyhi + 1, a.Dsy - 1) - iylo + 1, gp.nvy);
    // this warp's rows and their footprint
    const int rpw = (rows + kWarps - 1) / kWarps;
    const int wr0 = min(warp * rpw, rows), wr1 = min(wr0 + rpw, rows);
    int wylo = iylo, wyhi = iylo;
    if (wr1 > wr0) {
        spatial_cell(y0 + wr0, a.H, a.Dsy, a.rH1, wylo, t);
        spatial_cell(y0 + wr1 - 1, a.H, a.Dsy, a.rH1, wyhi, t);
    }
    const int nvyw = min(min(wyhi + 1, a.Dsy - 1) - wylo + 1, gp.nvyw);

    const int wf = grid_warp_floats(gp.nvx, gp.nvyw, Dsc, gp.bins);
    float *wt = sm + warp * wf;
    float *txy = wt;                             // [nvyw][nvx][3]
    float *txc = txy + 3 * gp.nvyw * gp.nvx;     // [3][nvx][Dsc]
    float *tyc = txc + 3 * gp.nvx * Dsc;         // [3][nvyw][Dsc]
    float *hb = wt + grid_table_floats(gp.nvx, gp.nvyw, Dsc);  // [3][Dsc][33] yc bins of this row
    for (int e = threadIdx.x; e < kWarps * wf; e += kThreads) sm[e] = 0.f;
    __syncthreads();

    const size_t plane = static_cast<size_t>(a.H) * a.W;
    const float *xb = a.x + static_cast<size_t>(b) * 3 * plane;
    const float *gb = a.dy + static_cast<size_t>(b) * 3 * plane;
    const float fS1 = static_cast<float>(Dsc - 1), fS2 = static_cast<float>(Dc2);
    const int x = x0 + lane * 4;
    const int n = min(4, a.W - x);
    int ixl[4];
    float dxk[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        int ix;
        spatial_cell(min(x + k, a.W - 1), a.W, a.Dsx, a.rW1, ix, dxk[k]);
        ixl[k] = max(0, min(ix - ixlo, nvx - 2));
    }
    // xy: the weights factor as (y part) x (x part) and a lane's columns are
    // fixed, so sum_rows dy_c (1 - dy) and sum_rows dy_c dy are kept per
    // pixel while the rows stay in one y-cell and scattered when it changes.
    float sy0[4][3], sy1[4][3];
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
        for (int c = 0; c < 3; ++c) sy0[k][c] = sy1[k][c] = 0.f;
    int iyw_acc = -1;
    auto flush_xy = [&]() {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float dx = dxk[k];
            float v[4][3];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                v[0][c] = sy0[k][c] * (1.f - dx);
                v[1][c] = sy1[k][c] * (1.f - dx);
                v[2][c] = sy0[k][c] * dx;
                v[3][c] = sy1[k][c] * dx;
                sy0[k][c] = sy1[k][c] = 0.f;
            }
            warp_scatter<3>(txy, k < n ? (iyw_acc * gp.nvx + ixl[k]) * 3 : -1, gp.nvx * 3, 3, v);
        }
    };
    for (int r = wr0; r < wr1; ++r) {
        const int y = y0 + r;
        int iy;
        float dy;
        spatial_cell(y, a.H, a.Dsy, a.rH1, iy, dy);
        const int iyw = max(0, min(iy - wylo, nvyw - 2));
        if (iyw != iyw_acc) {
            if (iyw_acc >= 0) flush_xy();
            iyw_acc = iyw;
        }
        const size_t o = static_cast<size_t>(y) * a.W + x;
        float4 P[3], G[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            P[c] = make_float4(0.f, 0.f, 0.f, 0.f);
            G[c] = P[c];
            if (n > 0) {
                P[c] = PixIO<float>::load(xb + c * plane + o, n, a.vec && n == 4);
                G[c] = PixIO<float>::load(gb + c * plane + o, n, a.vec && n == 4);
            }
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const bool act = k < n;
            const float dx = dxk[k];
            float gy[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) gy[c] = act ? get(G[c], k) : 0.f;
#pragma unroll
            for (int c = 0; c < 3; ++c) {  // xy corners (iy, ix), (iy+1, ix), (iy, ix+1), (iy+1, ix+1)
                sy0[k][c] = fmaf(gy[c], 1.f - dy, sy0[k][c]);
                sy1[k][c] = fmaf(gy[c], dy, sy1[k][c]);
            }
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const float pc = fminf(fmaxf(get(P[c], k), 0.f), 1.f);
                float ec;
                const int jc = cell_of(pc, fS1, fS2, ec);
                {   // xc: corners (ix, j), (ix+1, j), (ix, j+1), (ix+1, j+1)
                    float v[4][1] = {{gy[c] * (1.f - dx) * (1.f - ec)}, {gy[c] * dx * (1.f - ec)},
                                     {gy[c] * (1.f - dx) * ec}, {gy[c] * dx * ec}};
                    warp_scatter<1>(txc + c * gp.nvx * Dsc, act ? ixl[k] * Dsc + jc : -1, Dsc, 1, v);
                }
                if (gp.bins) {
                    // yc: the row (hence dy and the y-cell) is common to the warp, so
                    // the intensity weights go to this lane's own bins (no conflicts)
                    // and are spread over the corners (iy, iy+1) once per row
                    hb[(c * Dsc + jc) * 33 + lane] += gy[c] * (1.f - ec);
                    hb[(c * Dsc + jc + 1) * 33 + lane] += gy[c] * ec;
                } else {  // yc: corners (iy, j), (iy+1, j), (iy, j+1), (iy+1, j+1)
                    float v[4][1] = {{gy[c] * (1.f - dy) * (1.f - ec)}, {gy[c] * dy * (1.f - ec)},
                                     {gy[c] * (1.f - dy) * ec}, {gy[c] * dy * ec}};
                    warp_scatter<1>(tyc + c * gp.nvyw * Dsc, act ? iyw * Dsc + jc : -1, Dsc, 1, v);
                }
            }
        }
        // yc bins of this row: lane-ordered sums, spread over rows iy, iy+1
        __syncwarp();
        for (int e = lane; gp.bins && e < 3 * Dsc; e += 32) {
            float *col = hb + e * 33;
            float sum = 0.f;
#pragma unroll 8
            for (int l = 0; l < 32; ++l) {
                sum += col[l];
                col[l] = 0.f;
            }
            const int c = e / Dsc, j = e - c * Dsc;
            float *t0 = tyc + (c * gp.nvyw + iyw) * Dsc + j;
            t0[0] = fmaf(1.f - dy, sum, t0[0]);
            t0[Dsc] = fmaf(dy, sum, t0[Dsc]);
        }
        __syncwarp();
    }
    if (iyw_acc >= 0) flush_xy();
    // the warps' first vertex row relative to the block's
    __shared__ int wy_off[kWarps], wy_n[kWarps];
    if (lane == 0) {
        wy_off[warp] = wylo - iylo;
        wy_n[warp] = wr1 > wr0 ? nvyw : 0;
    }
    __syncthreads();
    // block partial: sum the warps in order (each block entry independently)
    float *out = grid_part + (static_cast<size_t>(b) * gp.nblk + lb) * gp.blk_stride;
    float *oxy = out, *oxc = out + 3 * gp.nvy * gp.nvx, *oyc = oxc + 3 * gp.nvx * Dsc;
    for (int e = threadIdx.x; e < nvy * nvx * 3; e += kThreads) {
        const int iyb = e / (nvx * 3), r = e - iyb * nvx * 3;  // r = ix * 3 + c
        float s = 0.f;
        for (int w = 0; w < kWarps; ++w) {
            const int iw = iyb - wy_off[w];
            if (iw >= 0 && iw < wy_n[w]) s += sm[w * wf + iw * gp.nvx * 3 + r];
        }
        oxy[iyb * gp.nvx * 3 + r] = s;
    }
    for (int e = threadIdx.x; e < 3 * nvx * Dsc; e += kThreads) {
        const int c = e / (nvx * Dsc), r = e - c * nvx * Dsc;
        float s = 0.f;
        for (int w = 0; w < kWarps; ++w) s += sm[w * wf + 3 * gp.nvyw * gp.nvx + c * gp.nvx * Dsc + r];
        oxc[c * gp.nvx * Dsc + r] = s;
    }
    for (int e = threadIdx.x; e < 3 * nvy * Dsc; e += kThreads) {
        const int c = e / (nvy * Dsc), r = e - c * nvy * Dsc, iyb = r / Dsc, j = r - iyb * Dsc;
        float s = 0.f;
        for (int w = 0; w < kWarps; ++w) {
            const int iw = iyb - wy_off[w];
            if (iw >= 0 && iw < wy_n[w])
                s += sm[w * wf + 3 * gp.nvyw * gp.nvx + 3 * gp.nvx * Dsc + (c * gp.nvyw + iw) * Dsc + j];
        }
        oyc[(c * gp.nvy + iyb) * Dsc + j] = s;
    }
}

// ---------------------------------------------------------------------------
// LUT finalize: one CTA per (table c*3+pair, image).
// ---------------------------------------------------------------------------
constexpr int kFinThreads = 256;

__device__ inline float block_sum(float v, float *red)
{
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    float s = 0.f;
    for (int w = 0; w < kFinThreads / 32; ++w) s += red[w];
    return s;
}

struct FinArgs {
    const float *U, *S, *V, *lw;
    float *dU, *dS, *dV, *dlw;
    int D, R, P;
};

__global__ void __launch_bounds__(kFinThreads)
    lut_finalize_kernel(FinArgs f, const float *__restrict__ lut_part, const float *__restrict__ sums_part)
{
    extern __shared__ __align__(16) float sm[];
    const int cp = blockIdx.x, b = blockIdx.y, c = cp / 3, pair = cp - c * 3;
    const int D = f.D, R = f.R, DD = D * D, DR = D * R;
    float *G = sm, *T = sm + DD, *Q = T + DD, *red = Q + DR;  // Q[i][r] = sum_j dT[i][j] V[j][r]
    const float *U = f.U + (static_cast<size_t>(b) * 9 + cp) * DR;
    const float *V = f.V + (static_cast<size_t>(b) * 9 + cp) * DR;
    const float *S = f.S + (static_cast<size_t>(b) * 9 + cp) * R;
    const float w = f.lw[static_cast<size_t>(b) * 12 + c * 4 + pair];
    for (int e = threadIdx.x; e < DD; e += kFinThreads) {
        float s = 0.f;
        for (int p = 0; p < f.P; ++p) s += lut_part[((static_cast<size_t>(b) * f.P + p) * 9 + cp) * DD + e];
        G[e] = s;
        const int i = e / D, j = e - i * D;
        float tv = 0.f;
        for (int r = 0; r < R; ++r) tv = fmaf(U[i * R + r] * S[r], V[j * R + r], tv);
        T[e] = tv;
    }
    __syncthreads();
    // dw = <G, T>
    float part = 0.f;
    for (int e = threadIdx.x; e < DD; e += kFinThreads) part = fmaf(G[e], T[e], part);
    const float dw = block_sum(part, red);
    if (threadIdx.x == 0 && f.dlw) {
        f.dlw[static_cast<size_t>(b) * 12 + c * 4 + pair] = dw;
        if (pair == 0) {
            float s = 0.f;
            for (int p = 0; p < f.P; ++p) s += sums_part[(static_cast<size_t>(b) * f.P + p) * 3 + c];
            f.dlw[static_cast<size_t>(b) * 12 + c * 4 + 3] = s;
        }
    }
    // Q = (w G) V ; dU = Q diag(S) ; dS_r = sum_i U[i][r] Q[i][r]
    for (int e = threadIdx.x; e < DR; e += kFinThreads) {
        const int i = e / R, r = e - i * R;
        float s = 0.f;
        for (int j = 0; j < D; ++j) s = fmaf(G[i * D + j], V[j * R + r], s);
        Q[e] = w * s;
        if (f.dU) f.dU[(static_cast<size_t>(b) * 9 + cp) * DR + e] = w * s * S[r];
    }
    // dV = (w G)^T U diag(S)
    if (f.dV)
        for (int e = threadIdx.x; e < DR; e += kFinThreads) {
            const int j = e / R, r = e - j * R;
            float s = 0.f;
            for (int i = 0; i < D; ++i) s = fmaf(G[i * D + j], U[i * R + r], s);
            f.dV[(static_cast<size_t>(b) * 9 + cp) * DR + e] = w * s * S[r];
        }
    __syncthreads();
    if (f.dS && threadIdx.x < R) {
        const int r = threadIdx.x;
        float s = 0.f;
        for (int i = 0; i < D; ++i) s = fmaf(U[i * R + r], Q[i * R + r], s);
        f.dS[(static_cast<size_t>(b) * 9 + cp) * R + r] = s;
    }
}

// ---------------------------------------------------------------------------
// grid reduce and finalize, fused.  A CTA takes a slice of kGRChunk vertices
// of one folded plane (xy, xc or yc) of one output channel c of one image.
// Per vertex it sums the partials of the blocks whose footprint holds the
// vertex (bands, then strips, in order), which is dF_c at that vertex; then
// for every grid k with k mod 3 = c it writes dg^k_plane = w^k_plane dF_c
// (Supp. Eqs. 21-22: grid k feeds channel k mod 3 with weight w^k_plane) and
// adds dF_c g^k_plane to the CTA's partial of dgrid_w[k][plane].
// grid_wsum_kernel sums those partials over the slices in order.
// ---------------------------------------------------------------------------
constexpr int kGRThreads = 256, kGRChunk = kGRThreads * 2;
constexpr int kMaxKK = (kMaxK + 2) / 3;  // grids per output channel

struct GridRed {
    int B, H, W, K, Dsx, Dsy, Dsc, strips;
    float rW1, rH1;
    GridPlan gp;
    int sl[3];  // slices per channel plane: xy, xc, yc
    int smax;   // max(sl)
    const float *gxy, *gxc, *gyc, *gw;
    float *dgxy, *dgxc, *dgyc;  // any may be null
    float *wpart;               // [B][3 planes][K][smax] partial sums of dgrid_w, or null
};

// block footprint along one axis: first vertex and count (as grid_grad_kernel)
__device__ __forceinline__ void axis_span(int p0, int cnt, int n, int Ds, float rn1, int vmax, int &lo, int &nv)
{
    int hi;
    float t;
    spatial_cell(p0, n, Ds, rn1, lo, t);
    spatial_cell(p0 + cnt - 1, n, Ds, rn1, hi, t);
    nv = min(min(hi + 1, Ds - 1) - lo + 1, vmax);
}

// range of strips / bands whose footprint may contain vertex v (pixel range
// between the neighbouring vertices)
__device__ __forceinline__ void cover_range(int v, int n, int Ds, int unit, int nunits, int &u0, int &u1)
{
    if (n <= 1) {
        u0 = 0;
        u1 = nunits - 1;
        return;
    }
    // a / d for 0 <= a, 1 <= d: a 32-bit division whenever a fits
    auto div = [](long long a, int d) -> long long {
        return a <= 0xffffffffLL ? static_cast<long long>(static_cast<unsigned int>(a) / static_cast<unsigned int>(d))
                                 : a / d;
    };
    const long long lo = div(static_cast<long long>(max(v - 1, 0)) * (n - 1), Ds - 1);
    const long long hi = div(static_cast<long long>(min(v + 1, Ds - 1)) * (n - 1) + (Ds - 2), Ds - 1);
    u0 = max(0, static_cast<int>(div(lo, unit)) - 1);
    u1 = min(nunits - 1, static_cast<int>(div(hi, unit)) + 1);
}

__host__ __device__ inline int grid_plane_size(int plane, int Dsx, int Dsy, int Dsc)
{
    return plane == 0 ? Dsy * Dsx : (plane == 1 ? Dsx * Dsc : Dsy * Dsc);
}

__global__ void __launch_bounds__(kGRThreads, 4)
    grid_reduce_kernel(GridRed g, const float *__restrict__ grid_part)
{
    extern __shared__ int gtab[];  // ylo[bands], nvy[bands], xlo[strips], nvx[strips]
    __shared__ float red[kGRThreads / 32][kMaxKK];
    const GridPlan &gp = g.gp;
    const int b = blockIdx.y;
    int q = blockIdx.x, plane = 0;  // blockIdx.x -> (plane, channel c, slice)
    while (plane < 2 && q >= 3 * g.sl[plane]) {
        q -= 3 * g.sl[plane];
        ++plane;
    }
    const int c = q / g.sl[plane], slice = q - c * g.sl[plane];
    int *ylo = gtab, *nvy = gtab + gp.bands, *xlo = nvy + gp.bands, *nvx = xlo + g.strips;
    for (int t = threadIdx.x; t < gp.bands + g.strips; t += kGRThreads) {
        if (t < gp.bands) {
            const int y0 = t * gp.BH, rows = min(gp.BH, g.H - y0);
            if (rows > 0) axis_span(y0, rows, g.H, g.Dsy, g.rH1, gp.nvy, ylo[t], nvy[t]);
            else ylo[t] = nvy[t] = 0;
        } else {
            const int st = t - gp.bands, x0 = st * kTileW;
            axis_span(x0, min(kTileW, g.W - x0), g.W, g.Dsx, g.rW1, gp.nvx, xlo[st], nvx[st]);
        }
    }
    __syncthreads();
    const int Dsx = g.Dsx, Dsy = g.Dsy, Dsc = g.Dsc, K = g.K;
    const int n = grid_plane_size(plane, Dsx, Dsy, Dsc), ncol = plane == 0 ? Dsx : Dsc;
    const float *gsrc = plane == 0 ? g.gxy : (plane == 1 ? g.gxc : g.gyc);
    float *gdst = plane == 0 ? g.dgxy : (plane == 1 ? g.dgxc : g.dgyc);
    const int oxc = 3 * gp.nvy * gp.nvx, oyc = oxc + 3 * gp.nvx * Dsc;  // plane offsets in a block partial
    float acc[kMaxKK];
#pragma unroll
    for (int kk = 0; kk < kMaxKK; ++kk) acc[kk] = 0.f;
    const int e1 = min(n, (slice + 1) * kGRChunk);
    for (int e = slice * kGRChunk + threadIdx.x; e < e1; e += kGRThreads) {
        // xy: (iy, ix); xc: (ix, j); yc: (iy, j)
        const int r = e / ncol, col = e - r * ncol;
        const int iy = plane == 1 ? -1 : r, ix = plane == 0 ? col : (plane == 1 ? r : -1), j = col;
        int s0 = 0, s1 = g.strips - 1, b0 = 0, b1 = gp.bands - 1;
        if (ix >= 0) cover_range(ix, g.W, Dsx, kTileW, g.strips, s0, s1);
        if (iy >= 0) cover_range(iy, g.H, Dsy, gp.BH, gp.bands, b0, b1);
        float s = 0.f;
        for (int bd = b0; bd <= b1; ++bd) {
            const int yl = ylo[bd], ny = nvy[bd];
            if (ny <= 0 || (iy >= 0 && (iy < yl || iy >= yl + ny))) continue;
            for (int st = s0; st <= s1; ++st) {
                const int xl = xlo[st];
                if (ix >= 0 && (ix < xl || ix >= xl + nvx[st])) continue;
                const float *bp = grid_part + (static_cast<size_t>(b) * gp.nblk + bd * g.strips + st) * gp.blk_stride;
                if (plane == 0)
                    s += bp[((iy - yl) * gp.nvx + (ix - xl)) * 3 + c];
                else if (plane == 1)
                    s += bp[oxc + (c * gp.nvx + (ix - xl)) * Dsc + j];
                else
                    s += bp[oyc + (c * gp.nvy + (iy - yl)) * Dsc + j];
            }
        }
#pragma unroll
        for (int kk = 0; kk < kMaxKK; ++kk) {
            const int k = c + 3 * kk;
            if (k >= K) break;
            const size_t o = (static_cast<size_t>(b) * K + k) * n + e;
            if (gdst) gdst[o] = __ldg(g.gw + (static_cast<size_t>(b) * K + k) * 4 + plane) * s;
            acc[kk] = fmaf(s, __ldg(gsrc + o), acc[kk]);
        }
    }
    if (!g.wpart) return;
    // the CTA's partials of dgrid_w: warp butterflies, then the warps in order
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int kk = 0; kk < kMaxKK; ++kk) {
        if (c + 3 * kk >= K) break;
        const float v = warp_sum(acc[kk]);
        if (lane == 0) red[warp][kk] = v;
    }
    __syncthreads();
    const int k = c + 3 * static_cast<int>(threadIdx.x);
    if (static_cast<int>(threadIdx.x) < kMaxKK && k < K) {
        float s = 0.f;
        for (int w = 0; w < kGRThreads / 32; ++w) s += red[w][threadIdx.x];
        g.wpart[((static_cast<size_t>(b) * 3 + plane) * K + k) * g.smax + slice] = s;
    }
}

// dgrid_w[b][k] = (the slice partials of each plane summed in order, the sum
// of dy_{k mod 3} over the image from the LUT pass partials: the bias).
struct GridWsum {
    int B, K, P, smax;
    int sl[3];
    float *dgw;
};

__global__ void grid_wsum_kernel(GridWsum f, const float *__restrict__ wpart, const float *__restrict__ sums_part)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;  // (b, k, entry)
    if (t >= f.B * f.K * 4) return;
    const int q = t & 3, bk = t >> 2, b = bk / f.K, k = bk - b * f.K;
    float s = 0.f;
    if (q < 3) {
        const float *p = wpart + ((static_cast<size_t>(b) * 3 + q) * f.K + k) * f.smax;
        for (int i = 0; i < f.sl[q]; ++i) s += p[i];
    } else {
        for (int p = 0; p < f.P; ++p) s += sums_part[(static_cast<size_t>(b) * f.P + p) * 3 + k % 3];
    }
    f.dgw[static_cast<size_t>(bk) * 4 + q] = s;
}

// ---------------------------------------------------------------------------
// host planning and workspace
// ---------------------------------------------------------------------------
struct BwdPlan {
    int P;             // LUT-pass CTAs per image
    size_t lut_smem;   // bytes
    GridPlan gp;
    size_t grid_smem;  // bytes
    // workspace layout (bytes); the last part holds the per-image tables of
    // the dx pass (prep_kernel)
    size_t off_lut, off_sums, off_grid, off_wpart, off_prep, prep_img, total;
    int sl[3], smax;  // grid_reduce_kernel slices per channel plane (xy, xc, yc)
};

static size_t align256(size_t v) { return (v + 255) & ~static_cast<size_t>(255); }

// Lets kernel f use dynamic shared memory up to the opt-in limit minus its
// static shared memory.
// Opts kernel f into the largest dynamic shared memory its static shared
// memory leaves, once per device (calls from several threads are serialised).
static svdlut_status allow_dynamic_smem(const void *f, int max_optin, int device)
{
    static std::mutex mu;
    static std::vector<std::pair<int, const void *>> done;
    std::lock_guard<std::mutex> g(mu);
    for (const auto &e : done)
        if (e.first == device && e.second == f) return SVDLUT_OK;
    cudaFuncAttributes fa;
    SVDLUT_CUDA_TRY(cudaFuncGetAttributes(&fa, f));
    SVDLUT_CUDA_TRY(cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         max_optin - static_cast<int>(fa.sharedSizeBytes)));
    done.emplace_back(device, f);
    return SVDLUT_OK;
}

static svdlut_status plan_backward(const svdlut_dims *d, int B, int H, int W, int sm_count, size_t smem_limit,
                                   BwdPlan *pl)
{
    const int D = d->D_t, Dsc = d->Dsc;
    pl->lut_smem = sizeof(float) * (static_cast<size_t>(kLutWarps) * 4 * D * D + kLutWarps);
    if (pl->lut_smem > smem_limit) return fail(SVDLUT_ERR_UNSUPPORTED, "D_t=%d too large for the adjoint", D);
    // LUT pass: P CTAs per image (one CTA per SM); estimated time = waves x
    // (rows a warp group walks: a quarter of strips x rows, + a fixed cost of
    // about 16 rows per CTA: clearing the tables, writing the partial)
    {
        const long long strips = (W + kTileW - 1) / kTileW, G = kLutWarps / 3;
        long long best_cost = -1;
        for (int P = 1; P <= std::min(H, 4 * sm_count); ++P) {
            const long long waves = (static_cast<long long>(B) * P + sm_count - 1) / sm_count;
            const long long rows = (H + P - 1) / P;
            const long long cost = waves * ((strips * rows + G - 1) / G + 16);
            if (best_cost < 0 || cost < best_cost) {
                best_cost = cost;
                pl->P = P;
            }
        }
    }
    // grid pass: blocks of 128 x BH; bands minimise waves x (rows a warp
    // walks + a fixed cost of about 4 rows per block: clearing the tables,
    // writing the partial); ties go to the better-filled waves
    const int strips = (W + kTileW - 1) / kTileW;
    const int max_bands = std::max(1, (H + kMinBlockH - 1) / kMinBlockH);
    int best = -1;
    double best_score = -1e30;
    GridPlan bestgp{};
    for (int bins = 1; bins >= 0 && best < 0; --bins)
    for (int bands = 1; bands <= max_bands; ++bands) {
        GridPlan gp{};
        gp.bins = bins;
        gp.BH = (H + bands - 1) / bands;
        gp.bands = (H + gp.BH - 1) / gp.BH;
        gp.nvx = span_bound(kTileW, W, d->Dsx);
        gp.nvy = span_bound(gp.BH, H, d->Dsy);
        gp.rpw = (gp.BH + kWarps - 1) / kWarps;
        gp.nvyw = span_bound(gp.rpw, H, d->Dsy);
        const size_t need = sizeof(float) * static_cast<size_t>(kWarps) * grid_warp_floats(gp.nvx, gp.nvyw, Dsc, bins);
        if (need + 256 > smem_limit) continue;  // + the kernel's static row offsets
        const long long T = static_cast<long long>(B) * strips * gp.bands;
        const double waves = std::ceil(static_cast<double>(T) / sm_count - 1e-9);
        const double fill = static_cast<double>(T) / (waves * sm_count);
        const double score = -waves * (gp.rpw + 4) + 1e-3 * fill;
        if (score > best_score + 1e-12) {
            best_score = score;
            best = bands;
            bestgp = gp;
        }
        if (bands >= 4 * sm_count) break;
    }
    if (best < 0) return fail(SVDLUT_ERR_UNSUPPORTED, "grid vertices too dense for the adjoint's blocks");
    bestgp.nblk = strips * bestgp.bands;
    bestgp.blk_stride = grid_block_floats(bestgp.nvx, bestgp.nvy, Dsc);
    pl->gp = bestgp;
    pl->grid_smem =
        sizeof(float) * static_cast<size_t>(kWarps) * grid_warp_floats(bestgp.nvx, bestgp.nvyw, Dsc, bestgp.bins);
    size_t off = 0;
    pl->off_lut = off;
    off = align256(off + sizeof(float) * static_cast<size_t>(B) * pl->P * 9 * D * D);
    pl->off_sums = off;
    off = align256(off + sizeof(float) * static_cast<size_t>(B) * pl->P * 3);
    pl->off_grid = off;
    off = align256(off + sizeof(float) * static_cast<size_t>(B) * bestgp.nblk * bestgp.blk_stride);
    pl->smax = 1;
    for (int q = 0; q < 3; ++q) {
        pl->sl[q] = (grid_plane_size(q, d->Dsx, d->Dsy, Dsc) + kGRChunk - 1) / kGRChunk;
        pl->smax = std::max(pl->smax, pl->sl[q]);
    }
    pl->off_wpart = off;
    off = align256(off + sizeof(float) * static_cast<size_t>(B) * 3 * std::max(d->K, 0) * pl->smax);
    pl->off_prep = off;
    pl->prep_img = prep_image_bytes(d);
    off += static_cast<size_t>(B) * pl->prep_img;
    pl->total = off;
    return SVDLUT_OK;
}

static svdlut_status check_backward_args(const svdlut_dims *dims, const svdlut_params *params, int B, int H,
                                         int W, const float *x, const float *dy)
{
    svdlut_status st = check_dims(dims);
    if (st != SVDLUT_OK) return st;
    if ((st = check_params(dims, params)) != SVDLUT_OK) return st;
    if (B < 1 || H < 1 || W < 1) return fail(SVDLUT_ERR_INVALID_ARG, "B=%d H=%d W=%d must be >= 1", B, H, W);
    if (!x || !dy) return fail(SVDLUT_ERR_INVALID_ARG, "x and dy are required");
    if (!aligned(x, 4) || !aligned(dy, 4)) return fail(SVDLUT_ERR_INVALID_ARG, "x and dy must be 4-byte aligned");
    return SVDLUT_OK;
}

}  // namespace svdlut

using namespace svdlut;

extern "C" size_t svdlut_backward_workspace_size(const svdlut_dims *dims, int B, int H, int W)
{
    if (check_dims(dims) != SVDLUT_OK || B < 1 || H < 1 || W < 1) return 0;
    DeviceInfo di;
    if (device_info(&di) != SVDLUT_OK) return 0;
    BwdPlan pl;
    if (plan_backward(dims, B, H, W, di.sm_count, static_cast<size_t>(di.max_smem_optin), &pl) != SVDLUT_OK)
        return 0;
    return pl.total;
}

extern "C" svdlut_status svdlut_backward(const svdlut_dims *dims, const svdlut_params *params, int B, int H,
                                         int W, const float *x, const float *dy, float *dx,
                                         const svdlut_grads *grads, void *ws, size_t ws_bytes,
                                         svdlut_stream_t stream)
{
    SVDLUT_TRACE("svdlut_backward");
    clear_error();
    svdlut_status st = check_backward_args(dims, params, B, H, W, x, dy);
    if (st != SVDLUT_OK) return st;
    if (dx && !aligned(dx, 4)) return fail(SVDLUT_ERR_INVALID_ARG, "dx must be 4-byte aligned");
    const size_t img = static_cast<size_t>(3) * H * W * sizeof(float);
    if (dx) {
        const char *ds = reinterpret_cast<const char *>(dx), *xs = reinterpret_cast<const char *>(x),
                   *gs = reinterpret_cast<const char *>(dy);
        const size_t n = B * img;
        if ((ds < xs + n && xs < ds + n) || (ds < gs + n && gs < ds + n))
            return fail(SVDLUT_ERR_INVALID_ARG, "dx overlaps x or dy");
    }
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    DeviceInfo di;
    if ((st = device_info(&di)) != SVDLUT_OK) return st;
    const size_t smem_limit = static_cast<size_t>(di.max_smem_optin);

    const svdlut_grads g0{};
    const svdlut_grads &g = grads ? *grads : g0;
    const bool want_lut = g.dU || g.dS || g.dV || g.dlut_w;
    const bool want_grid = dims->K > 0 && (g.dg_xy || g.dg_xc || g.dg_yc || g.dgrid_w);
    BwdPlan pl;
    if ((st = plan_backward(dims, B, H, W, di.sm_count, smem_limit, &pl)) != SVDLUT_OK) return st;
    const bool have_ws = ws && ws_bytes >= pl.total;
    if ((want_lut || want_grid) && !have_ws)
        return fail(SVDLUT_ERR_WORKSPACE, "workspace of %zu bytes needed (got %zu)", pl.total, ws ? ws_bytes : 0);
    if (have_ws && !aligned(ws, 256)) return fail(SVDLUT_ERR_INVALID_ARG, "workspace must be 256-byte aligned");

    // 1. dx through the forward kernel's adjoint mode; with a workspace, the
    // per-image tables are precomputed once (prep_kernel) instead of in
    // every CTA
    if (dx) {
        for (int b0 = 0; b0 < B; b0 += kPlainChunk) {
            LaunchArgs<kPlainChunk> a{};
            a.n = std::min(kPlainChunk, B - b0);
            for (int i = 0; i < a.n; ++i) {
                a.img[i] = make_desc(dims, params, b0 + i, H, W, SVDLUT_F32, x, dx);
                a.img[i].dy = dy + static_cast<size_t>(b0 + i) * 3 * H * W;
                a.img[i].vec = a.img[i].vec && aligned(a.img[i].dy, 16);
                if (have_ws)
                    set_prep_tables(a.img[i], dims,
                                    static_cast<char *>(ws) + pl.off_prep + static_cast<size_t>(b0 + i) * pl.prep_img);
            }
            size_t smem = 0;
            if ((st = plan_uniform(a, di.sm_count, smem_limit, &smem)) != SVDLUT_OK) return st;
            if (have_ws) {
                if ((st = launch_prep(a, di.sm_count, s)) != SVDLUT_OK) return st;
                a.pre = 1;
            }
            if ((st = launch_apply(a, smem, SVDLUT_F32, s, 0, true)) != SVDLUT_OK) return st;
        }
    }
    if (!want_lut && !want_grid) return SVDLUT_OK;
    char *w = static_cast<char *>(ws);
    float *lut_part = reinterpret_cast<float *>(w + pl.off_lut);
    float *sums_part = reinterpret_cast<float *>(w + pl.off_sums);
    float *grid_part = reinterpret_cast<float *>(w + pl.off_grid);
    float *wpart = reinterpret_cast<float *>(w + pl.off_wpart);

    BwdArgs a{};
    a.x = x;
    a.dy = dy;
    a.B = B;
    a.H = H;
    a.W = W;
    a.D = dims->D_t;
    a.K = dims->K;
    a.Dsx = dims->Dsx;
    a.Dsy = dims->Dsy;
    a.Dsc = dims->Dsc;
    a.rW1 = W > 1 ? 1.0f / static_cast<float>(W - 1) : 0.f;
    a.rH1 = H > 1 ? 1.0f / static_cast<float>(H - 1) : 0.f;
    a.strips = (W + kTileW - 1) / kTileW;
    a.vec = (W % 4 == 0) && aligned(x, 16) && aligned(dy, 16);

    if ((st = allow_dynamic_smem(reinterpret_cast<const void *>(lut_grad_kernel), di.max_smem_optin, di.device)) !=
        SVDLUT_OK)
        return st;
    if ((st = allow_dynamic_smem(reinterpret_cast<const void *>(grid_grad_kernel), di.max_smem_optin, di.device)) !=
        SVDLUT_OK)
        return st;
    if ((st = allow_dynamic_smem(reinterpret_cast<const void *>(lut_finalize_kernel), di.max_smem_optin,
                                 di.device)) != SVDLUT_OK)
        return st;
    if (pl.grid_smem + 256 > static_cast<size_t>(di.max_smem_optin) || pl.lut_smem > static_cast<size_t>(di.max_smem_optin))
        return fail(SVDLUT_ERR_UNSUPPORTED, "adjoint tables do not fit in shared memory");
    // 2. LUT pass (also produces the dy channel sums used by every bias)
    lut_grad_kernel<<<dim3(pl.P, B), kLutThreads, pl.lut_smem, s>>>(a, lut_part, sums_part);
    SVDLUT_CUDA_TRY(cudaGetLastError());
    if (want_lut) {
        FinArgs f{params->U, params->S, params->V, params->lut_w, g.dU, g.dS, g.dV, g.dlut_w,
                  dims->D_t, dims->rank, pl.P};
        const size_t fsm = sizeof(float) * (2 * dims->D_t * dims->D_t + dims->D_t * dims->rank + kFinThreads / 32);
        lut_finalize_kernel<<<dim3(9, B), kFinThreads, fsm, s>>>(f, lut_part, sums_part);
        SVDLUT_CUDA_TRY(cudaGetLastError());
    }
    if (want_grid) {
        grid_grad_kernel<<<dim3(pl.gp.nblk, B), kThreads, pl.grid_smem, s>>>(a, pl.gp, grid_part);
        SVDLUT_CUDA_TRY(cudaGetLastError());
        GridRed r{};
        r.B = B;
        r.H = H;
        r.W = W;
        r.K = dims->K;
        r.Dsx = dims->Dsx;
        r.Dsy = dims->Dsy;
        r.Dsc = dims->Dsc;
        r.strips = a.strips;
        r.rW1 = a.rW1;
        r.rH1 = a.rH1;
        r.gp = pl.gp;
        r.smax = pl.smax;
        for (int q = 0; q < 3; ++q) r.sl[q] = pl.sl[q];
        r.gxy = params->g_xy;
        r.gxc = params->g_xc;
        r.gyc = params->g_yc;
        r.gw = params->grid_w;
        r.dgxy = g.dg_xy;
        r.dgxc = g.dg_xc;
        r.dgyc = g.dg_yc;
        r.wpart = g.dgrid_w ? wpart : nullptr;
        // the CTA's band and strip footprint tables
        const size_t rsm = sizeof(int) * 2 * static_cast<size_t>(pl.gp.bands + a.strips);
        if (rsm > 48 * 1024) {
            if ((st = allow_dynamic_smem(reinterpret_cast<const void *>(grid_reduce_kernel), di.max_smem_optin,
                                         di.device)) != SVDLUT_OK)
                return st;
            if (rsm + sizeof(float) * (kGRThreads / 32) * kMaxKK > static_cast<size_t>(di.max_smem_optin))
                return fail(SVDLUT_ERR_UNSUPPORTED, "too many column strips and row bands for the grid reduction");
        }
        grid_reduce_kernel<<<dim3(3 * (pl.sl[0] + pl.sl[1] + pl.sl[2]), B), kGRThreads, rsm, s>>>(r, grid_part);
        SVDLUT_CUDA_TRY(cudaGetLastError());
        if (g.dgrid_w) {
            GridWsum f{B, dims->K, pl.P, pl.smax, {pl.sl[0], pl.sl[1], pl.sl[2]}, g.dgrid_w};
            const int n = B * dims->K * 4;
            grid_wsum_kernel<<<(n + 255) / 256, 256, 0, s>>>(f, wpart, sums_part);
            SVDLUT_CUDA_TRY(cudaGetLastError());
        }
    }
    return SVDLUT_OK;
}
