// Fused 2D slicing + 2D LUT transform kernel (Eq. 10, Supp. Eq. 22) for sm_103a.
//
// One persistent CTA per SM walks a contiguous range of pixel blocks (or takes
// blocks from an atomic queue, for ragged batches); a block is a
// 128-pixel-wide column strip of one image, BH rows tall (BH is planned on the
// host so that the blocks cover the SMs evenly).  A lane owns 4 pixels of a
// row: columns lane + 32 k of the tile for float images (every warp-wide
// access covers 32 adjacent pixels, which keeps the table gathers of smooth
// regions on few cells), or 4 adjacent pixels for integer pixel formats (one
// 32- or 64-bit access per plane or word); warp w owns rows w, w + kWarps, ...
// of the block.  The pixel formats (planar float and 8-bit, interleaved
// 8-bit) are template parameters (Io<In, Out> below).
//  - Prologue, once per image a CTA meets: the factor rows arrive by
//    asynchronous copies, the nine 2D LUTs are rebuilt from their SVD factors
//    (Eq. 9) in shared memory, multiplied by their LUT weights (Eq. 5) and
//    turned into per-cell bilinear coefficients (phi = a + b da + c db +
//    d da db, Supp. Eq. 15) for the three output channels: 3 float4 per cell
//    and pair.
//  - Per block: the grid slices of the block's footprint are summed over the
//    grids that feed each output channel (grid k feeds channel k mod 3, Supp.
//    Eq. 22) with their weights (Eq. 21), with the loads of several elements
//    per thread in flight; the xc slice is stored per x-cell and intensity
//    cell in slope form (value, slope along intensity, and their differences
//    to the next x-cell).
//  - Per row: a warp interpolates the xy and yc slices along y for its row
//    (yc as value and slope along intensity).
//  - Per pixel: 9 LDS.128 for the three LUT pairs, 2 LDS.128 (xy), 3 LDS.128
//    (xc) and 3 LDS.64 (yc).  Row data is loaded one row ahead, across block
//    boundaries.
#pragma once

#include <type_traits>

#include "svdlut_internal.cuh"

namespace svdlut {

#ifndef SVDLUT_WARPS
#define SVDLUT_WARPS 16
#endif
constexpr int kWarps = SVDLUT_WARPS;
constexpr int kThreads = kWarps * 32;
constexpr int kTileW = 128;  // 32 lanes x 4 pixels
constexpr int kMinBlockH = 16;
static_assert(kTileW <= kThreads, "column tables need one thread each");

struct ImgDesc {
    const void *x;
    void *y;          // forward: output image; adjoint: dx
    const float *dy;  // adjoint only: upstream gradient
    const float *U, *S, *V, *lw, *gxy, *gxc, *gyc, *gw;
    int H, W;
    int D, R, K, Dsx, Dsy, Dsc;
    int y_begin, y_end;  // rows processed: [y_begin, y_end) of the H-row image
    int strips;       // column strips of kTileW pixels
    int BH;           // block height (rows)
    int block_begin;  // first global block index of this image
    float rW1, rH1;   // 1/(W-1), 1/(H-1); 0 when W or H is 1
    int vec;         // whole-lane vector loads and stores allowed (W % 4 == 0, aligned images)
    // precomputed per image by prep_kernel (workspace path), else null:
    float *pcell;  // the cell table, laid out as in shared memory (lcell_floats(D) floats)
    float *pfold;  // grid slices folded per output channel: xy [3][Dsy][Dsx], xc [3][Dsx][Dsc],
                   // yc [3][Dsy][Dsc], then the three summed biases
};

template <int N>
struct LaunchArgs {
    int n;             // images in img[]
    int total_blocks;  // sum of blocks over images
    int nvx_max, nvy_max, bh_max;
    int lcell_floats;    // floats reserved for the cell table
    int scratch_floats;  // floats of the block buffers / prologue temporaries
    int xcol;            // nonzero: per-column xc tables (every image's Dsc <= kXcolMaxDsc)
    int pre;             // nonzero: cell tables and folded grids precomputed (ImgDesc::pcell, pfold)
    unsigned int *queue;  // non-null: blocks are taken from this counter (must be 0 at launch)
    unsigned int *check;  // index-check status (builds with SVDLUT_CHECK_BOUNDS), else null
    ImgDesc img[N];
};

// Largest intensity-vertex count whose xc slice is tabulated per block column
// (3 x Dsc x 128 floats: 36 KB at 24); larger Dsc use the per-cell slope form.
constexpr int kXcolMaxDsc = 24;

// ---- optional index checks ----
// Built with -DSVDLUT_CHECK_BOUNDS, every shared-memory gather index of the
// kernel is tested against its table size, every lane's run of pixels
// against its image plane, and every vector access and 16-byte asynchronous
// copy against its alignment.  A failure is counted in the status words
// (count, site, index, limit of the first one) and the access is made safe:
// the index replaced by 0, the pixel run dropped, the vector access done with
// scalar ones, the copy skipped.  Otherwise the checks compile to nothing.
enum CheckSite : unsigned int {
    kChkLut = 1, kChkPxc = 2, kChkRyc = 3, kChkRxy = 4,  // shared-memory gathers
    kChkPixel = 5,                                       // pixel run outside the plane (index: offset)
    kChkAlign = 6                                        // misaligned vector access or copy (index: address)
};

__device__ __forceinline__ void check_record(unsigned int *st, unsigned int site, unsigned int idx, unsigned int limit)
{
    if (st && atomicAdd(st, 1u) == 0u) {
        st[1] = site;
        st[2] = idx;
        st[3] = limit;
    }
}

__device__ __forceinline__ int checked_index(unsigned int *st, unsigned int site, int idx, int limit)
{
#ifdef SVDLUT_CHECK_BOUNDS
    if (idx >= 0 && idx < limit) return idx;
    check_record(st, site, static_cast<unsigned int>(idx), static_cast<unsigned int>(limit));
    return 0;
#else
    (void)st;
    (void)site;
    (void)limit;
    return idx;
#endif
}

// A lane's n adjacent pixels from offset off must lie in a plane of `plane`
// pixels; returns n, or 0 after a failure.
__device__ __forceinline__ int checked_run(unsigned int *st, size_t off, int n, size_t plane)
{
#ifdef SVDLUT_CHECK_BOUNDS
    if (n <= 0 || off + static_cast<size_t>(n - 1) < plane) return n;
    check_record(st, kChkPixel, static_cast<unsigned int>(off), static_cast<unsigned int>(plane));
    return 0;
#else
    (void)st;
    (void)off;
    (void)plane;
    return n;
#endif
}

// vec, unless a vector access at p would be misaligned for `align` bytes
__device__ __forceinline__ bool checked_vec(unsigned int *st, bool vec, const void *p, size_t align)
{
#ifdef SVDLUT_CHECK_BOUNDS
    if (!vec || (reinterpret_cast<uintptr_t>(p) % align) == 0) return vec;
    check_record(st, kChkAlign, static_cast<unsigned int>(reinterpret_cast<uintptr_t>(p)),
                 static_cast<unsigned int>(align));
    return false;
#else
    (void)st;
    (void)p;
    (void)align;
    return vec;
#endif
}

// Spatial cell of pixel index x on an axis of n pixels and Ds vertices
// (x' = x/(n-1), u = x' (Ds-1), Supp. Eqs. 17-18), computed exactly in
// integers: i = floor(x (Ds-1) / (n-1)) clamped to Ds-2, delta = remainder
// / (n-1).  A float product x * (Ds-1)/(n-1) would lose up to half an ulp of
// u (1.5e-5 at u ~ 479), too much for the grid term at 4K.
__host__ __device__ __forceinline__ void spatial_cell(int x, int n, int Ds, float rn1, int &i, float &d)
{
    if (n <= 1) {
        i = 0;
        d = 0.f;
        return;
    }
    const long long num = static_cast<long long>(x) * (Ds - 1);
    // exact integer quotient; 32-bit division whenever the numerator fits
    long long q = num <= 0xffffffffLL ? static_cast<long long>(static_cast<unsigned int>(num) /
                                                              static_cast<unsigned int>(n - 1))
                                      : num / (n - 1);
    if (q > Ds - 2) q = Ds - 2;
    i = static_cast<int>(q);
    d = static_cast<float>(num - q * (n - 1)) * rn1;
}

// Upper bound on the grid vertices along an axis that one tile of `extent`
// pixels touches on an image axis of n pixels with Ds vertices.
inline int span_bound(int extent, int n, int Ds)
{
    if (n <= 1) return 2 < Ds ? 2 : Ds;
    double s = static_cast<double>(Ds - 1) / static_cast<double>(n - 1);
    int v = static_cast<int>(ceil((extent - 1) * s)) + 3;
    return v < Ds ? v : Ds;
}

// Cell table: per pair (D-1) rows of cells with a row stride of D cells (one
// cell of padding) so that the bank of a cell depends on both of its indices.
__host__ __device__ inline int lcell_floats(int D) { return 3 * (D - 1) * D * 12; }

constexpr int kMiscFloats = kMaxK * 4 + 4;

// ---- pixel I/O ----
template <typename T>
struct PixIO;

template <>
struct PixIO<float> {
    using Raw = float4;
    static __device__ __forceinline__ Raw load(const float *p, int n, bool vec)
    {
        if (vec && n == 4) return __ldcs(reinterpret_cast<const float4 *>(p));
        Raw v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (n > 0) v.x = __ldcs(p);
        if (n > 1) v.y = __ldcs(p + 1);
        if (n > 2) v.z = __ldcs(p + 2);
        if (n > 3) v.w = __ldcs(p + 3);
        return v;
    }
    static __device__ __forceinline__ float4 to_float(Raw v) { return v; }
    // pixel k of a lane at p + 32 k (k < n): one coalesced 128-byte row per warp instruction
    static __device__ __forceinline__ Raw load_s(const float *p, int n)
    {
        Raw v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (n > 0) v.x = __ldcs(p);
        if (n > 1) v.y = __ldcs(p + 32);
        if (n > 2) v.z = __ldcs(p + 64);
        if (n > 3) v.w = __ldcs(p + 96);
        return v;
    }
    static __device__ __forceinline__ void store_s(float *p, float4 v, int n)
    {
        if (n > 0) __stcs(p, v.x);
        if (n > 1) __stcs(p + 32, v.y);
        if (n > 2) __stcs(p + 64, v.z);
        if (n > 3) __stcs(p + 96, v.w);
    }
    static __device__ __forceinline__ void store(float *p, float4 v, int n, bool vec)
    {
        if (vec && n == 4) {
            __stcs(reinterpret_cast<float4 *>(p), v);
            return;
        }
        if (n > 0) __stcs(p, v.x);
        if (n > 1) __stcs(p + 1, v.y);
        if (n > 2) __stcs(p + 2, v.z);
        if (n > 3) __stcs(p + 3, v.w);
    }
};

// Round-half-even of clamp(y,0,1)*255 on the FMA pipe: after adding 1.5*2^23
// the low byte of the bit pattern is the rounded integer (0..255).
__device__ __forceinline__ unsigned int quant_u8_bits(float y)
{
    y = fminf(fmaxf(y, 0.f), 1.f);
    return static_cast<unsigned int>(__float_as_int(fmaf(y, 255.f, 12582912.0f)));
}

template <>
struct PixIO<uint8_t> {
    // four pixels packed in one 32-bit word, byte k = pixel k
    using Raw = unsigned int;
    static __device__ __forceinline__ Raw load(const uint8_t *p, int n, bool vec)
    {
        if (vec && n == 4) return __ldcs(reinterpret_cast<const unsigned int *>(p));
        unsigned int w = 0;
        if (n > 0) w |= static_cast<unsigned int>(p[0]);
        if (n > 1) w |= static_cast<unsigned int>(p[1]) << 8;
        if (n > 2) w |= static_cast<unsigned int>(p[2]) << 16;
        if (n > 3) w |= static_cast<unsigned int>(p[3]) << 24;
        return w;
    }
    // v/255 with the integer placed in the mantissa of 2^23 (no I2F)
    static __device__ __forceinline__ float4 to_float(Raw w)
    {
        const float k = 1.0f / 255.0f, m = 8388608.0f;
        const float a = __int_as_float(__byte_perm(w, 0x4B000000u, 0x7440)) - m;
        const float b = __int_as_float(__byte_perm(w, 0x4B000000u, 0x7441)) - m;
        const float c = __int_as_float(__byte_perm(w, 0x4B000000u, 0x7442)) - m;
        const float d = __int_as_float(__byte_perm(w, 0x4B000000u, 0x7443)) - m;
        return make_float4(a * k, b * k, c * k, d * k);
    }
    static __device__ __forceinline__ void store(uint8_t *p, float4 v, int n, bool vec)
    {
        const unsigned int w = __byte_perm(__byte_perm(quant_u8_bits(v.x), quant_u8_bits(v.y), 0x0040),
                                           __byte_perm(quant_u8_bits(v.z), quant_u8_bits(v.w), 0x0040), 0x5410);
        if (vec && n == 4) {
            __stcs(reinterpret_cast<unsigned int *>(p), w);
            return;
        }
        if (n > 0) p[0] = w & 0xff;
        if (n > 1) p[1] = (w >> 8) & 0xff;
        if (n > 2) p[2] = (w >> 16) & 0xff;
        if (n > 3) p[3] = w >> 24;
    }
};

// ---- pixel formats of the transform's input and output ----
// A lane handles 4 adjacent pixels of a tile row (columns lane * 4 + k, k <
// n), so a whole lane is one 128-bit access per float plane (one 32-bit
// access per 8-bit plane or interleaved word).  `off` is the
// offset y * W + x of the lane's first pixel, at(base, off) its address,
// `plane` = H * W.  load(at(..), plane, ..) fills Raw r[3] with the lane's
// pixels; unpack() turns them into the channel values (r, g, b) of the 4
// pixels.  kVecAlign: the alignment that makes the whole-lane vector access
// legal (with W % 4 == 0).
struct InF32 {  // planar float [3][H][W]
    using Raw = float4;  // one per channel
    static constexpr size_t kPixelBytes = 12, kVecAlign = 16;
    static __device__ __forceinline__ const void *at(const void *base, size_t off)
    {
        return static_cast<const float *>(base) + off;
    }
    static __device__ __forceinline__ void load(const void *q, size_t plane, int n, bool vec, Raw *r)
    {
        const float *p = static_cast<const float *>(q);
#pragma unroll
        for (int c = 0; c < 3; ++c) r[c] = PixIO<float>::load(p + c * plane, n, vec);
    }
    static __device__ __forceinline__ void unpack(const Raw *r, float4 (&v)[3])
    {
        v[0] = r[0];
        v[1] = r[1];
        v[2] = r[2];
    }
};

struct InU8 {  // planar 8-bit [3][H][W], value v / 255
    using Raw = unsigned int;  // one per channel, byte k = pixel k
    static constexpr size_t kPixelBytes = 3, kVecAlign = 4;
    static __device__ __forceinline__ const void *at(const void *base, size_t off)
    {
        return static_cast<const uint8_t *>(base) + off;
    }
    static __device__ __forceinline__ void load(const void *q, size_t plane, int n, bool vec, Raw *r)
    {
        const uint8_t *p = static_cast<const uint8_t *>(q);
#pragma unroll
        for (int c = 0; c < 3; ++c) r[c] = PixIO<uint8_t>::load(p + c * plane, n, vec);
    }
    static __device__ __forceinline__ void unpack(const Raw *r, float4 (&v)[3])
    {
#pragma unroll
        for (int c = 0; c < 3; ++c) v[c] = PixIO<uint8_t>::to_float(r[c]);
    }
};

// byte b (0..3) of w as a float in [0, 255] (no I2F)
__device__ __forceinline__ float byte_value(unsigned int w, int b)
{
    return __int_as_float(__byte_perm(w, 0x4B000000u, 0x7440 + b)) - 8388608.0f;
}

struct InU8Hwc {  // interleaved 8-bit [H][W][3], value v / 255
    // 12 bytes of 4 pixels: r0 g0 b0 r1 | g1 b1 r2 g2 | b2 r3 g3 b3
    using Raw = unsigned int;
    static constexpr size_t kPixelBytes = 3, kVecAlign = 4;
    static __device__ __forceinline__ const void *at(const void *base, size_t off)
    {
        return static_cast<const uint8_t *>(base) + 3 * off;
    }
    static __device__ __forceinline__ void load(const void *q, size_t, int n, bool vec, Raw *r)
    {
        const uint8_t *p = static_cast<const uint8_t *>(q);
        if (vec && n == 4) {
            const unsigned int *w = reinterpret_cast<const unsigned int *>(p);
            r[0] = __ldcs(w);
            r[1] = __ldcs(w + 1);
            r[2] = __ldcs(w + 2);
            return;
        }
        unsigned int w[3] = {0u, 0u, 0u};
#pragma unroll
        for (int i = 0; i < 12; ++i)
            if (i < 3 * n) w[i >> 2] |= static_cast<unsigned int>(p[i]) << (8 * (i & 3));
        r[0] = w[0];
        r[1] = w[1];
        r[2] = w[2];
    }
    static __device__ __forceinline__ void unpack(const Raw *r, float4 (&v)[3])
    {
        const float k = 1.0f / 255.0f;
        v[0] = make_float4(byte_value(r[0], 0) * k, byte_value(r[0], 3) * k, byte_value(r[1], 2) * k,
                           byte_value(r[2], 1) * k);
        v[1] = make_float4(byte_value(r[0], 1) * k, byte_value(r[1], 0) * k, byte_value(r[1], 3) * k,
                           byte_value(r[2], 2) * k);
        v[2] = make_float4(byte_value(r[0], 2) * k, byte_value(r[1], 1) * k, byte_value(r[2], 0) * k,
                           byte_value(r[2], 3) * k);
    }
};

// Outputs: o[c][k] = channel c of the lane's pixel k.
struct OutF32 {  // planar float
    static constexpr size_t kPixelBytes = 12, kVecAlign = 16;
    static __device__ __forceinline__ const void *at(const void *base, size_t off)
    {
        return static_cast<const float *>(base) + off;
    }
    static __device__ __forceinline__ void store(void *base, size_t plane, size_t off, const float (&o)[3][4], int n,
                                                 bool vec)
    {
        float *p = static_cast<float *>(base) + off;
#pragma unroll
        for (int c = 0; c < 3; ++c)
            PixIO<float>::store(p + c * plane, make_float4(o[c][0], o[c][1], o[c][2], o[c][3]), n, vec);
    }
};

struct OutU8 {  // planar 8-bit, rint(clamp(y, 0, 1) * 255)
    static constexpr size_t kPixelBytes = 3, kVecAlign = 4;
    static __device__ __forceinline__ const void *at(const void *base, size_t off)
    {
        return static_cast<const uint8_t *>(base) + off;
    }
    static __device__ __forceinline__ void store(void *base, size_t plane, size_t off, const float (&o)[3][4], int n,
                                                 bool vec)
    {
        uint8_t *p = static_cast<uint8_t *>(base) + off;
#pragma unroll
        for (int c = 0; c < 3; ++c)
            PixIO<uint8_t>::store(p + c * plane, make_float4(o[c][0], o[c][1], o[c][2], o[c][3]), n, vec);
    }
};

// bytes (a, b, c, d) -> one word, each the low byte of its argument
__device__ __forceinline__ unsigned int pack4(unsigned int a, unsigned int b, unsigned int c, unsigned int d)
{
    return __byte_perm(__byte_perm(a, b, 0x0040), __byte_perm(c, d, 0x0040), 0x5410);
}

struct OutU8Hwc {  // interleaved 8-bit, rint(clamp(y, 0, 1) * 255)
    static constexpr size_t kPixelBytes = 3, kVecAlign = 4;
    static __device__ __forceinline__ const void *at(const void *base, size_t off)
    {
        return static_cast<const uint8_t *>(base) + 3 * off;
    }
    static __device__ __forceinline__ void store(void *base, size_t, size_t off, const float (&o)[3][4], int n,
                                                 bool vec)
    {
        uint8_t *p = static_cast<uint8_t *>(base) + 3 * off;
        unsigned int q[3][4];
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int k = 0; k < 4; ++k) q[c][k] = quant_u8_bits(o[c][k]);
        const unsigned int w0 = pack4(q[0][0], q[1][0], q[2][0], q[0][1]);
        const unsigned int w1 = pack4(q[1][1], q[2][1], q[0][2], q[1][2]);
        const unsigned int w2 = pack4(q[2][2], q[0][3], q[1][3], q[2][3]);
        if (vec && n == 4) {
            unsigned int *w = reinterpret_cast<unsigned int *>(p);
            __stcs(w, w0);
            __stcs(w + 1, w1);
            __stcs(w + 2, w2);
            return;
        }
        const unsigned int w[3] = {w0, w1, w2};
#pragma unroll
        for (int i = 0; i < 12; ++i)
            if (i < 3 * n) p[i] = static_cast<uint8_t>(w[i >> 2] >> (8 * (i & 3)));
    }
};

template <class IN, class OUT>
struct Io {
    using In = IN;
    using Out = OUT;
};

using IoF32 = Io<InF32, OutF32>;
using IoU8 = Io<InU8, OutU8>;

__device__ __forceinline__ float get(const float4 &v, int k)
{
    return k == 0 ? v.x : (k == 1 ? v.y : (k == 2 ? v.z : v.w));
}

// Cell of p in [0,1] on an axis with D vertices (fDm1 = D-1, fDm2 = D-2), on
// the FMA pipe: i = round-to-nearest(min(p (D-1) - 1/2, D-2)) via the
// 1.5 * 2^23 magic constant, frac = p (D-1) - i in [0, 1].  This is the
// Supp. Eq. 13 cell except exactly on a vertex, where the cell below may be
// chosen with frac = 1; bilinear interpolation is continuous there, so the
// value is the same.
__device__ __forceinline__ int cell_of(float p, float fDm1, float fDm2, float &frac)
{
    const float t = fminf(fmaf(p, fDm1, -0.5f), fDm2);
    const float m = t + 12582912.0f;
    frac = fmaf(p, fDm1, -(m - 12582912.0f));
    return __float_as_int(m) - 0x4B400000;
}

// The same cell as cell_of, returned as the bit pattern of 1.5 * 2^23 + i
// (i = bits - kCellBias): callers fold the bias into their address
// arithmetic (unsigned, modulo 2^32).
constexpr unsigned int kCellBias = 0x4B400000u;
__device__ __forceinline__ unsigned int cell_bits(float p, float fDm1, float fDm2, float &frac)
{
    const float t = fminf(fmaf(p, fDm1, -0.5f), fDm2);
    const float m = t + 12582912.0f;
    frac = fmaf(p, fDm1, -(m - 12582912.0f));
    return static_cast<unsigned int>(__float_as_int(m));
}

// ---- LUT prologue: Eq. 9 reconstruction, Eq. 5 weight fold, cell coefficients ----
// Factor rows are padded with zeros to Rp floats, a multiple of 4 with Rp / 4
// odd: rows are read as float4, and the lanes of a quarter warp reading
// consecutive rows hit different 16-byte bank groups.
__host__ __device__ inline int padded_rank(int R)
{
    const int q = (R + 3) / 4;
    return 4 * (q | 1);
}

// Shared-memory floats of the prologue temporaries: factors of all nine
// tables at once (pairs = 3) or of one pair at a time (pairs = 1).
__host__ __device__ inline int prologue_floats_n(int D, int R, int pairs)
{
    return 2 * 3 * pairs * D * padded_rank(R) + D * D * 4;
}

// 16- and 4-byte asynchronous global -> shared copies (cp.async; L2 only for
// 16 bytes) and the wait for all of this thread's copies.
__device__ __forceinline__ void cp_async16(void *dst, const void *src)
{
    const unsigned int s = static_cast<unsigned int>(__cvta_generic_to_shared(dst));
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async4(void *dst, const void *src)
{
    const unsigned int s = static_cast<unsigned int>(__cvta_generic_to_shared(dst));
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all()
{
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

__device__ __forceinline__ bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

__device__ inline void build_luts(const ImgDesc &d, float4 *lcell, float *tmp, float *misc, int tmp_floats,
                                  unsigned int *check)
{
    (void)check;
    const int tid = threadIdx.x;
    const int D = d.D, R = d.R, Rp = padded_rank(R), R4 = (R + 3) / 4, DR = D * R, DRp = D * Rp, Dm1 = D - 1;
    // all nine tables' factors at once when they fit (one global round trip)
    const int pairs_at_once = prologue_floats_n(D, R, 3) <= tmp_floats ? 3 : 1;
    const int nf = 3 * pairs_at_once;  // (c, p) tables held
    float *sU = tmp;                   // [nf][D][Rp] = U * S * w
    float *sV = tmp + nf * DRp;        // [nf][D][Rp]
    float4 *vt = reinterpret_cast<float4 *>(tmp + 2 * nf * DRp);  // [D][D]

    // grid weights and summed biases
    for (int e = tid; e < d.K * 4; e += kThreads) misc[e] = __ldg(d.gw + e);
    if (tid < 3) {
        float b = __ldg(d.lw + tid * 4 + 3);
        for (int k = tid; k < d.K; k += 3) b += __ldg(d.gw + k * 4 + 3);
        misc[kMaxK * 4 + tid] = b;
    }
    const int nc = Dm1 * D;  // padded cells per pair
    const int nrow = nf * D;  // factor rows held (of U, and of V)
    const bool fast = (R & 3) == 0 && aligned16(d.U) && aligned16(d.V);
    for (int p = 0; p < 3; ++p) {
        if ((pairs_at_once == 1 || p == 0) && fast) {
            // slot <-> (c, p): slot = c * 3 + p when all pairs are held, else c.
            // U and V rows (16-byte chunks), S and the pair weights go to
            // shared memory as asynchronous copies (one round trip); S and
            // the weights sit in the vt area until U is scaled by them.
            float *sS = reinterpret_cast<float *>(vt), *sW = sS + nf * R;
            for (int e = tid; e < nrow * R4; e += kThreads) {
                const int row = e / R4, q = e - row * R4, slot = row / D, i = row - slot * D;
                const int c = slot / pairs_at_once, pp = pairs_at_once == 3 ? slot - c * 3 : p;
                const int cp = c * 3 + pp;
                float *du = sU + slot * DRp + i * Rp + 4 * q, *dv = sV + slot * DRp + i * Rp + 4 * q;
                const float *su = d.U + cp * DR + i * R + 4 * q, *sv = d.V + cp * DR + i * R + 4 * q;
#ifdef SVDLUT_CHECK_BOUNDS
                if (((reinterpret_cast<uintptr_t>(du) | reinterpret_cast<uintptr_t>(dv) |
                      reinterpret_cast<uintptr_t>(su) | reinterpret_cast<uintptr_t>(sv)) & 15) != 0) {
                    check_record(check, kChkAlign, static_cast<unsigned int>(reinterpret_cast<uintptr_t>(su)), 16u);
                    continue;
                }
#endif
                cp_async16(du, su);
                cp_async16(dv, sv);
            }
            for (int e = tid; e < nf * (R + 1); e += kThreads) {
                const int slot = e / (R + 1), r = e - slot * (R + 1);
                const int c = slot / pairs_at_once, pp = pairs_at_once == 3 ? slot - c * 3 : p;
                if (r < R) cp_async4(sS + slot * R + r, d.S + (c * 3 + pp) * R + r);
                else cp_async4(sW + slot, d.lw + c * 4 + pp);
            }
            cp_async_wait_all();
            __syncthreads();
            for (int e = tid; e < nrow * R; e += kThreads) {
                const int row = e / R, r = e - row * R, slot = row / D;
                sU[row * Rp + r] = sU[row * Rp + r] * sS[slot * R + r] * sW[slot];  // (U S) w, as below
            }
            __syncthreads();
        } else if (pairs_at_once == 1 || p == 0) {
            // general case (rank not a multiple of 4 or unaligned factors):
            // element e = (slot, i, r) with r < Rp, padding zeroed; the loads
            // of kLoadBatch elements are issued before any of their stores.
            constexpr int kLoadBatch = 4;
            for (int e0 = tid; e0 < nrow * Rp; e0 += kLoadBatch * kThreads) {
                float u[kLoadBatch], v[kLoadBatch];
#pragma unroll
                for (int q = 0; q < kLoadBatch; ++q) {
                    const int e = e0 + q * kThreads;
                    const int row = e / Rp, r = e - row * Rp, slot = row / D, i = row - slot * D;
                    const int c = slot / pairs_at_once, pp = pairs_at_once == 3 ? slot - c * 3 : p;
                    const int cp = c * 3 + pp;
                    const bool ok = e < nrow * Rp && r < R;
                    u[q] = ok ? __ldg(d.U + cp * DR + i * R + r) * __ldg(d.S + cp * R + r) * __ldg(d.lw + c * 4 + pp)
                              : 0.f;
                    v[q] = ok ? __ldg(d.V + cp * DR + i * R + r) : 0.f;
                }
#pragma unroll
                for (int q = 0; q < kLoadBatch; ++q) {
                    const int e = e0 + q * kThreads;
                    if (e < nrow * Rp) {
                        sU[e] = u[q];
                        sV[e] = v[q];
                    }
                }
            }
            __syncthreads();
        }
        for (int e = tid; e < D * D; e += kThreads) {
            const int i = e / D, j = e - i * D;
            float acc[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const int slot = pairs_at_once == 3 ? c * 3 + p : c;
                const float4 *u = reinterpret_cast<const float4 *>(sU + slot * DRp + i * Rp);
                const float4 *v = reinterpret_cast<const float4 *>(sV + slot * DRp + j * Rp);
                float a = 0.f;
                if (R4 == 2) {
#pragma unroll
                    for (int q = 0; q < 2; ++q) {
                        const float4 x = u[q], y = v[q];
                        a = fmaf(x.x, y.x, fmaf(x.y, y.y, fmaf(x.z, y.z, fmaf(x.w, y.w, a))));
                    }
                } else {
                    for (int q = 0; q < R4; ++q) {
                        const float4 x = u[q], y = v[q];
                        a = fmaf(x.x, y.x, fmaf(x.y, y.y, fmaf(x.z, y.z, fmaf(x.w, y.w, a))));
                    }
                }
                acc[c] = a;
            }
            vt[e] = make_float4(acc[0], acc[1], acc[2], 0.f);
        }
        __syncthreads();
        for (int e = tid; e < Dm1 * Dm1; e += kThreads) {
            const int i = e / Dm1, j = e - i * Dm1;
            {
                const float4 v00 = vt[i * D + j], v10 = vt[(i + 1) * D + j];
                const float4 v01 = vt[i * D + j + 1], v11 = vt[(i + 1) * D + j + 1];
                const float bx = v10.x - v00.x, by = v10.y - v00.y, bz = v10.z - v00.z;
                const float cx = v01.x - v00.x, cy = v01.y - v00.y, cz = v01.z - v00.z;
                const float dx = v11.x - v10.x - v01.x + v00.x, dy = v11.y - v10.y - v01.y + v00.y,
                            dz = v11.z - v10.z - v01.z + v00.z;
                float4 *q = lcell + (p * nc + i * D + j) * 3;
                q[0] = make_float4(v00.x, v00.y, v00.z, bx);
                q[1] = make_float4(by, bz, cx, cy);
                q[2] = make_float4(cz, dx, dy, dz);
            }
        }
        __syncthreads();
    }
}

struct BlockGeom {
    int x0, y0, rows, ixlo, iylo, nvx, nvy;
};

__device__ __forceinline__ BlockGeom block_geom(const ImgDesc &d, int lb, int nvx_max, int nvy_max)
{
    BlockGeom g;
    const int band = lb / d.strips, strip = lb - band * d.strips;
    g.x0 = strip * kTileW;
    g.y0 = d.y_begin + band * d.BH;
    g.rows = min(d.BH, d.y_end - g.y0);
    const int x1 = min(g.x0 + kTileW - 1, d.W - 1), y1 = g.y0 + g.rows - 1;
    int ixhi, iyhi;
    float unused;
    spatial_cell(g.x0, d.W, d.Dsx, d.rW1, g.ixlo, unused);
    spatial_cell(x1, d.W, d.Dsx, d.rW1, ixhi, unused);
    spatial_cell(g.y0, d.H, d.Dsy, d.rH1, g.iylo, unused);
    spatial_cell(y1, d.H, d.Dsy, d.rH1, iyhi, unused);
    ixhi = min(ixhi + 1, d.Dsx - 1);
    iyhi = min(iyhi + 1, d.Dsy - 1);
    g.nvx = min(ixhi - g.ixlo + 1, nvx_max);
    g.nvy = min(iyhi - g.iylo + 1, nvy_max);
    return g;
}

// Block buffers (floats, in this order):
//   fxy [3][nvy][nvx], fxc [3][nvx][Dsc], fyc [3][nvy][Dsc]   folded grid slices
//   coli [kTileW] int, cold [kTileW]                           column cells
//   rowi [bh] int, rowd [bh]                                    row cells
//   the xc slice, in one of two forms (LaunchArgs::xcol):
//     xcol [3][Dsc][kTileW]: the folded xc slice interpolated along x at each
//          column of the block, per intensity vertex; column col is stored
//          at (col & 3) * 32 + (col >> 2), so that pixel k of every lane of a
//          warp (column lane * 4 + k) reads consecutive words: no bank
//          conflicts whatever the intensities;
//     pxc [3][nvx-1][Dsc] float4: slope form of x-cell ix and intensity cell
//          j (see block_phase_b), for large Dsc where xcol does not fit; row
//          stride Dsc (one padding entry) to spread banks
//   per warp: rxy [nvx] float4 (xy interpolated along y for the warp's row),
//             ryc [3][Dsc-1] float2 (yc interpolated along y: value at j and
//             slope to j + 1)
struct BlockBufs {
    float *fxy, *fxc, *fyc;
    int *coli, *rowi;
    float *cold, *rowd;
    float *xcol;
    float4 *pxc, *rxy;
    float2 *ryc;
};

// rounded to 4 floats so every warp's float4 table stays 16-byte aligned
__host__ __device__ inline int warp_row_floats(int nvx, int Dsc) { return (nvx * 4 + 3 * (Dsc - 1) * 2 + 3) & ~3; }

__host__ __device__ inline int fold_floats(int nvx, int nvy, int Dsc)
{
    return (3 * nvy * nvx + 3 * nvx * Dsc + 3 * nvy * Dsc + 3) & ~3;
}

__host__ __device__ inline int xc_table_floats(int nvx, int Dsc, bool xcol)
{
    return xcol ? 3 * Dsc * kTileW : 3 * (nvx - 1) * Dsc * 4;
}

__host__ __device__ inline int block_floats(int nvx, int nvy, int Dsc, int bh, bool xcol)
{
    return fold_floats(nvx, nvy, Dsc) + 2 * kTileW + ((2 * bh + 3) & ~3) + xc_table_floats(nvx, Dsc, xcol) +
           kWarps * warp_row_floats(nvx, Dsc);
}

__device__ __forceinline__ BlockBufs block_bufs(float *scratch, int nvx, int nvy, int Dsc, int bh_max, bool xcol)
{
    BlockBufs b;
    const int warp = threadIdx.x >> 5;
    b.fxy = scratch;
    b.fxc = b.fxy + 3 * nvy * nvx;
    b.fyc = b.fxc + 3 * nvx * Dsc;
    float *t = scratch + fold_floats(nvx, nvy, Dsc);
    b.coli = reinterpret_cast<int *>(t);
    b.cold = t + kTileW;
    b.rowi = reinterpret_cast<int *>(t + 2 * kTileW);
    b.rowd = t + 2 * kTileW + bh_max;
    float *xt = t + 2 * kTileW + ((2 * bh_max + 3) & ~3);
    b.xcol = xt;
    b.pxc = reinterpret_cast<float4 *>(xt);
    float *w = xt + xc_table_floats(nvx, Dsc, xcol) + warp * warp_row_floats(nvx, Dsc);
    b.rxy = reinterpret_cast<float4 *>(w);
    b.ryc = reinterpret_cast<float2 *>(w + nvx * 4);
    return b;
}

// Block setup, phase A: grid slices of the block footprint folded per output
// channel (sum over grids k = c mod 3 of w_k times grid k: Supp. Eqs. 21-22);
// column and row cell tables.
__device__ inline void block_phase_a(const ImgDesc &d, const BlockGeom &g, const BlockBufs &b, const float *misc,
                                     bool fold = true)
{
    const int tid = threadIdx.x;
    const int nvx = g.nvx, nvy = g.nvy, Dsc = d.Dsc, K = d.K;
    const size_t kxy = static_cast<size_t>(d.Dsy) * d.Dsx, kxc = static_cast<size_t>(d.Dsx) * Dsc,
                 kyc = static_cast<size_t>(d.Dsy) * Dsc;
    // One index space over the three folded slices (xy, then xc, then yc;
    // each [3 c][rows][cols], consecutive elements adjacent in memory); every
    // thread takes kFoldBatch elements at a time and issues all their loads
    // before the first FMA, so the slices cost a few memory round trips.
    const int nxy = 3 * nvy * nvx, nxc = 3 * nvx * Dsc, nyc = 3 * nvy * Dsc, ntot = nxy + nxc + nyc;
    if (!fold) {
        // the folded slices were copied from the precomputed ones (setup_pre)
    } else if (K > 0) {
        // element e -> its first grid value's address and its channel c (by
        // comparison: one division per element)
        auto locate = [&](int e, int &c, size_t &kst) -> const float * {
            if (e < nxy) {
                const int r = e / nvx, ixl = e - r * nvx;
                c = r >= nvy ? (r >= 2 * nvy ? 2 : 1) : 0;
                kst = kxy;
                return d.gxy + static_cast<size_t>(g.iylo + r - c * nvy) * d.Dsx + g.ixlo + ixl;
            }
            if (e < nxy + nxc) {
                const int f = e - nxy, r = f / Dsc, j = f - r * Dsc;
                c = r >= nvx ? (r >= 2 * nvx ? 2 : 1) : 0;
                kst = kxc;
                return d.gxc + static_cast<size_t>(g.ixlo + r - c * nvx) * Dsc + j;
            }
            const int f = e - nxy - nxc, r = f / Dsc, j = f - r * Dsc;
            c = r >= nvy ? (r >= 2 * nvy ? 2 : 1) : 0;
            kst = kyc;
            return d.gyc + static_cast<size_t>(g.iylo + r - c * nvy) * Dsc + j;
        };
        // kFoldBatch elements per thread at a time, their first kFoldTerms
        // grids (K <= 9: all of them) loaded before the first FMA
        constexpr int kFoldBatch = 8, kFoldTerms = 3;
        for (int e0 = tid; e0 < ntot; e0 += kFoldBatch * kThreads) {
            int ch[kFoldBatch];
            float v[kFoldBatch][kFoldTerms];
#pragma unroll
            for (int q = 0; q < kFoldBatch; ++q) {
                const int e = e0 + q * kThreads;
                int c = 0;
                size_t kst = 0;
                const float *sp = e < ntot ? locate(e, c, kst) : nullptr;
                ch[q] = c;
#pragma unroll
                for (int t = 0; t < kFoldTerms; ++t) {
                    const int k = c + 3 * t;
                    v[q][t] = sp && k < K ? __ldg(sp + k * kst) : 0.f;
                }
            }
#pragma unroll
            for (int q = 0; q < kFoldBatch; ++q) {
                const int e = e0 + q * kThreads;
                if (e >= ntot) continue;
                const int which = e < nxy ? 0 : (e < nxy + nxc ? 1 : 2);
                float acc = 0.f;
#pragma unroll
                for (int t = 0; t < kFoldTerms; ++t) {
                    const int k = ch[q] + 3 * t;
                    if (k < K) acc = fmaf(misc[k * 4 + which], v[q][t], acc);
                }
                if (K > 3 * kFoldTerms) {  // grids beyond the third of a channel
                    int c;
                    size_t kst;
                    const float *sp = locate(e, c, kst);
                    for (int k = c + 3 * kFoldTerms; k < K; k += 3) acc = fmaf(misc[k * 4 + which], __ldg(sp + k * kst), acc);
                }
                float *dst = e < nxy ? b.fxy + e : (e < nxy + nxc ? b.fxc + (e - nxy) : b.fyc + (e - nxy - nxc));
                *dst = acc;
            }
        }
    } else {
        for (int e = tid; e < ntot; e += kThreads)
            (e < nxy ? b.fxy + e : (e < nxy + nxc ? b.fxc + (e - nxy) : b.fyc + (e - nxy - nxc)))[0] = 0.f;
    }
    if (tid < kTileW) {
        int ix;
        float dx;
        spatial_cell(min(g.x0 + tid, d.W - 1), d.W, d.Dsx, d.rW1, ix, dx);
        b.coli[tid] = max(0, min(ix - g.ixlo, nvx - 2));
        b.cold[tid] = dx;
    }
    for (int row = tid; row < g.rows; row += kThreads) {
        int iy;
        float dy;
        spatial_cell(g.y0 + row, d.H, d.Dsy, d.rH1, iy, dy);
        b.rowi[row] = max(0, min(iy - g.iylo, nvy - 2));
        b.rowd[row] = dy;
    }
}

// ---- precomputed per-image tables (workspace path) ----
// Floats of the folded grid slices of one image, and the offset of its three
// summed biases after them.
__host__ __device__ inline size_t pfold_floats(int Dsx, int Dsy, int Dsc)
{
    return 3 * (static_cast<size_t>(Dsy) * Dsx + static_cast<size_t>(Dsx) * Dsc + static_cast<size_t>(Dsy) * Dsc);
}

// q = floor(n / m) for 0 <= n < 2^20, m >= 1, with rm = 1.0f / m: n + 0.5 is
// at least 0.5 away from a multiple of m, far more than the float error.
__device__ __forceinline__ int quot(int n, float rm) { return static_cast<int>((static_cast<float>(n) + 0.5f) * rm); }

// Block setup from the precomputed tables: on an image switch the cell table
// (16-byte asynchronous copies) and the summed biases; for every block the
// folded slices of its footprint (4-byte asynchronous copies).  The caller
// waits for the copies.
__device__ inline void setup_pre(const ImgDesc &d, const BlockGeom &g, const BlockBufs &b, float4 *lcell,
                                 float *misc, bool rebuild)
{
    const int tid = threadIdx.x;
    const int nvx = g.nvx, nvy = g.nvy, Dsc = d.Dsc, Dsx = d.Dsx, Dsy = d.Dsy;
    const float *pxy = d.pfold, *pxc = pxy + 3 * static_cast<size_t>(Dsy) * Dsx,
                *pyc = pxc + 3 * static_cast<size_t>(Dsx) * Dsc;
    if (rebuild) {
        // Every CTA copies the same table: each starts at its own place in it
        // (evenly spread over the CTAs), so that at any moment the copies
        // read different lines rather than all CTAs the same ones.
        const float4 *src = reinterpret_cast<const float4 *>(d.pcell);
        const int n4 = lcell_floats(d.D) / 4;
        const int rot = static_cast<int>((static_cast<long long>(n4) * blockIdx.x) / gridDim.x);
        for (int e = tid; e < n4; e += kThreads) {
            const int f = e + rot < n4 ? e + rot : e + rot - n4;
            cp_async16(lcell + f, src + f);
        }
        if (tid < 3) misc[kMaxK * 4 + tid] = __ldg(d.pfold + pfold_floats(Dsx, Dsy, Dsc) + tid);
    }
    const int nxy = nvy * nvx, nxc = nvx * Dsc, nyc = nvy * Dsc, oxy = 3 * nxy, oxc = 3 * nxc;
    const int ntot = oxy + oxc + 3 * nyc;
    const float rnvx = 1.0f / static_cast<float>(nvx);
    for (int o = tid; o < ntot; o += kThreads) {
        const float *src;
        if (o < oxy) {
            const int c = o >= nxy ? (o >= 2 * nxy ? 2 : 1) : 0, f = o - c * nxy, r = quot(f, rnvx);
            src = pxy + (static_cast<size_t>(c) * Dsy + g.iylo + r) * Dsx + g.ixlo + (f - r * nvx);
        } else if (o < oxy + oxc) {
            const int f0 = o - oxy, c = f0 >= nxc ? (f0 >= 2 * nxc ? 2 : 1) : 0;
            src = pxc + (static_cast<size_t>(c) * Dsx + g.ixlo) * Dsc + (f0 - c * nxc);
        } else {
            const int f0 = o - oxy - oxc, c = f0 >= nyc ? (f0 >= 2 * nyc ? 2 : 1) : 0;
            src = pyc + (static_cast<size_t>(c) * Dsy + g.iylo) * Dsc + (f0 - c * nyc);
        }
        cp_async4(b.fxy + o, src);  // fxy, fxc, fyc are consecutive
    }
}

// Per-image precomputation for the workspace path, one launch per chunk of
// images: the first CTAs build the cell table of each (image, pair) -- T = (U S) w
// V^T of the pair's three channel tables (Eq. 9, Eq. 5 weight) and the
// coefficient form of Supp. Eq. 15, in the same arithmetic order as
// build_luts, so both paths give identical tables; the other CTAs fold the
// grid slices per output channel (Supp. Eqs. 21-22; same order as
// block_phase_a) and sum the biases.  Lets the dependent apply kernel launch
// as soon as it starts.
constexpr int kPrepThreads = 512;
template <int N>
struct PrepArgs {
    int n;
    int start[N + 1];  // first fold output of each image in the flat index (host prefix sums)
    ImgDesc img[N];
};

__host__ __device__ inline int prep_smem_floats(int D, int R) { return 2 * 3 * D * padded_rank(R) + 3 * D * D; }


// CTAs [0, kLutCtas * n) build the cell rows [i0, i1) of (image, pair,
// part): T rows i0 .. i1 of the pair's three channel tables, then the cells.
constexpr int kLutParts = 4, kLutCtas = 3 * kLutParts;

template <int N>
__global__ void __launch_bounds__(kPrepThreads) prep_kernel(const __grid_constant__ PrepArgs<N> a)
{
    // launched as a programmatic dependent of the preceding kernel: wait for
    // its results (e.g. generator outputs) before reading anything
    asm volatile("griddepcontrol.wait;\n" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;\n" :::);
    extern __shared__ __align__(16) float ps[];
    const int tid = threadIdx.x;
    if (static_cast<int>(blockIdx.x) < kLutCtas * a.n) {
        const ImgDesc &d = a.img[blockIdx.x / kLutCtas];
        const int rem = blockIdx.x % kLutCtas, p = rem / kLutParts, part = rem - p * kLutParts;
        const int D = d.D, R = d.R, Rp = padded_rank(R), R4 = (R + 3) / 4, DR = D * R, DRp = D * Rp, Dm1 = D - 1;
        const int i0 = (Dm1 * part) / kLutParts, i1 = (Dm1 * (part + 1)) / kLutParts;  // cell rows
        const int nrow = i1 - i0 + 1;                                                    // T rows i0 .. i1
        if (i1 <= i0) return;
        float *sU = ps, *sV = ps + 3 * DRp, *sT = ps + 6 * DRp;  // [3 c][D][Rp] x 2, [3 c][nrow][D]
        // factor rows (U scaled by S and the pair weight, as build_luts): U
        // rows i0 .. i1 and all V rows; the loads of kBatch elements are
        // issued before any of their stores
        constexpr int kBatch = 4;
        const int nu = 3 * nrow * Rp, nv = 3 * DRp;
        for (int e0 = tid; e0 < nu + nv; e0 += kBatch * kPrepThreads) {
            float val[kBatch];
            int dst[kBatch];
#pragma unroll
            for (int q = 0; q < kBatch; ++q) {
                const int e = e0 + q * kPrepThreads;
                dst[q] = -1;
                val[q] = 0.f;
                if (e < nu) {
                    const int row = e / Rp, r = e - row * Rp, c = row / nrow, i = i0 + row - c * nrow, cp = c * 3 + p;
                    dst[q] = c * DRp + i * Rp + r;
                    if (r < R)
                        val[q] = __ldg(d.U + cp * DR + i * R + r) * __ldg(d.S + cp * R + r) * __ldg(d.lw + c * 4 + p);
                } else if (e < nu + nv) {
                    const int f = e - nu, row = f / Rp, r = f - row * Rp, c = row / D, i = row - c * D;
                    dst[q] = 3 * DRp + f;
                    if (r < R) val[q] = __ldg(d.V + (c * 3 + p) * DR + i * R + r);
                }
            }
#pragma unroll
            for (int q = 0; q < kBatch; ++q)
                if (dst[q] >= 0) ps[dst[q]] = val[q];
        }
        __syncthreads();
        for (int e = tid; e < 3 * nrow * D; e += kPrepThreads) {
            const int row = e / D, j = e - row * D, c = row / nrow, i = i0 + row - c * nrow;
            const float4 *u = reinterpret_cast<const float4 *>(sU + c * DRp + i * Rp);
            const float4 *v = reinterpret_cast<const float4 *>(sV + c * DRp + j * Rp);
            float acc = 0.f;
            for (int q = 0; q < R4; ++q) {
                const float4 x = u[q], y = v[q];
                acc = fmaf(x.x, y.x, fmaf(x.y, y.y, fmaf(x.z, y.z, fmaf(x.w, y.w, acc))));
            }
            sT[e] = acc;
        }
        __syncthreads();
        float4 *out = reinterpret_cast<float4 *>(d.pcell) + static_cast<size_t>(p) * Dm1 * D * 3;
        for (int e = tid; e < (i1 - i0) * Dm1; e += kPrepThreads) {
            const int ii = e / Dm1, j = e - ii * Dm1, i = i0 + ii;
            float v00[3], bb[3], cc[3], dd[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const float *t = sT + (c * nrow + ii) * D + j;
                const float t00 = t[0], t01 = t[1], t10 = t[D], t11 = t[D + 1];
                v00[c] = t00;
                bb[c] = t10 - t00;
                cc[c] = t01 - t00;
                dd[c] = t11 - t10 - t01 + t00;
            }
            float4 *q = out + (i * D + j) * 3;
            q[0] = make_float4(v00[0], v00[1], v00[2], bb[0]);
            q[1] = make_float4(bb[1], bb[2], cc[0], cc[1]);
            q[2] = make_float4(cc[2], dd[0], dd[1], dd[2]);
        }
        return;
    }
    // folded grid slices and summed biases of all images (grid-stride; the
    // loads of kBatch outputs are issued before their sums); image i owns the
    // flat outputs [start[i], start[i + 1])
    const int total = a.start[a.n];
    const int stride = (static_cast<int>(gridDim.x) - kLutCtas * a.n) * kPrepThreads;
    constexpr int kBatch = 4, kTerms = 3;
    for (int t0 = (static_cast<int>(blockIdx.x) - kLutCtas * a.n) * kPrepThreads + tid; t0 < total;
         t0 += kBatch * stride) {
        float g[kBatch][kTerms], w[kBatch][kTerms];
        int which[kBatch], ch[kBatch], im[kBatch], o[kBatch], e[kBatch];
#pragma unroll
        for (int q = 0; q < kBatch; ++q) {
            const int t = t0 + q * stride;
            int i = 0;
            if (t < total)
                while (t >= a.start[i + 1]) ++i;
            im[q] = i;
            o[q] = t - a.start[i];
            const ImgDesc &d = a.img[i];
            const int nxy = d.Dsy * d.Dsx, nxc = d.Dsx * d.Dsc, nyc = d.Dsy * d.Dsc;
            const int per = 3 * (nxy + nxc + nyc) + 3;
            const float *gsrc = nullptr;
            int kst = 0;
            if (t >= total || o[q] >= per - 3) {
                which[q] = 3;  // bias (or nothing)
                ch[q] = t < total ? o[q] - (per - 3) : 0;
                e[q] = 0;
            } else if (o[q] < 3 * nxy) {
                which[q] = 0;
                ch[q] = o[q] >= nxy ? (o[q] >= 2 * nxy ? 2 : 1) : 0;
                e[q] = o[q] - ch[q] * nxy;
                gsrc = d.gxy;
                kst = nxy;
            } else if (o[q] < 3 * (nxy + nxc)) {
                which[q] = 1;
                const int f = o[q] - 3 * nxy;
                ch[q] = f >= nxc ? (f >= 2 * nxc ? 2 : 1) : 0;
                e[q] = f - ch[q] * nxc;
                gsrc = d.gxc;
                kst = nxc;
            } else {
                which[q] = 2;
                const int f = o[q] - 3 * (nxy + nxc);
                ch[q] = f >= nyc ? (f >= 2 * nyc ? 2 : 1) : 0;
                e[q] = f - ch[q] * nyc;
                gsrc = d.gyc;
                kst = nyc;
            }
#pragma unroll
            for (int m = 0; m < kTerms; ++m) {
                const int k = ch[q] + 3 * m;
                const bool ok = which[q] < 3 && k < d.K;
                g[q][m] = ok ? __ldg(gsrc + static_cast<size_t>(k) * kst + e[q]) : 0.f;
                w[q][m] = ok ? __ldg(d.gw + k * 4 + which[q]) : 0.f;
            }
        }
#pragma unroll
        for (int q = 0; q < kBatch; ++q) {
            const int t = t0 + q * stride;
            if (t >= total) continue;
            const ImgDesc &d = a.img[im[q]];
            const int K = d.K;
            float acc;
            if (which[q] == 3) {  // summed bias of channel c: b^c + the grid biases feeding c
                acc = __ldg(d.lw + ch[q] * 4 + 3);
                for (int k = ch[q]; k < K; k += 3) acc += __ldg(d.gw + k * 4 + 3);
            } else {
                acc = 0.f;
#pragma unroll
                for (int m = 0; m < kTerms; ++m)
                    if (ch[q] + 3 * m < K) acc = fmaf(w[q][m], g[q][m], acc);
                const int nxy = d.Dsy * d.Dsx, nxc = d.Dsx * d.Dsc, nyc = d.Dsy * d.Dsc;
                const float *gsrc = which[q] == 0 ? d.gxy : (which[q] == 1 ? d.gxc : d.gyc);
                const int kst = which[q] == 0 ? nxy : (which[q] == 1 ? nxc : nyc);
                for (int k = ch[q] + 3 * kTerms; k < K; k += 3)
                    acc = fmaf(__ldg(d.gw + k * 4 + which[q]), __ldg(gsrc + static_cast<size_t>(k) * kst + e[q]), acc);
            }
            d.pfold[o[q]] = acc;
        }
    }
}

// Block setup, phase B: the xc slice table of the block.
//  xcol: value of the folded xc slice at column col and intensity vertex j,
//        (1 - dx) F(ix, j) + dx F(ix + 1, j) (Supp. Eq. 20 along x), at the
//        permuted position of the column (see BlockBufs).
//  pxc:  the slice of x-cell ix and intensity cell j in slope form (F,
//        F(j+1) - F(j), F(ix+1) - F(ix), [F(ix+1,j+1) - F(ix+1,j)] -
//        [F(ix,j+1) - F(ix,j)]), so that at (dx, e) it is (x + dx z) +
//        e (y + dx w).
__device__ inline void block_phase_b(const ImgDesc &d, const BlockGeom &g, const BlockBufs &b, bool xcol)
{
    const int nvx = g.nvx, Dsc = d.Dsc, Dc1 = Dsc - 1;
    if (xcol) {
        for (int e = threadIdx.x; e < 3 * Dsc * kTileW; e += kThreads) {
            const int col = e & (kTileW - 1), r = e >> 7;  // r = c * Dsc + j
            const int c = r >= Dsc ? (r >= 2 * Dsc ? 2 : 1) : 0, j = r - c * Dsc;
            const int ix = b.coli[col];
            const float *f0 = b.fxc + (c * nvx + ix) * Dsc + j;
            const float v0 = f0[0], v1 = f0[Dsc];
            b.xcol[r * kTileW + (col & 3) * 32 + (col >> 2)] = fmaf(v1 - v0, b.cold[col], v0);
        }
        return;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int r = warp; r < 3 * (nvx - 1); r += kWarps) {
        const int c = r / (nvx - 1), ixl = r - c * (nvx - 1);
        const float *f0 = b.fxc + (c * nvx + ixl) * Dsc;
        const float *f1 = f0 + Dsc;
        for (int j = lane; j < Dc1; j += 32) {
            const float s0 = f0[j + 1] - f0[j], s1 = f1[j + 1] - f1[j];
            b.pxc[r * Dsc + j] = make_float4(f0[j], s0, f1[j] - f0[j], s1 - s0);
        }
    }
}

// Per-warp tables of one block row: xy and yc slices interpolated along y.
__device__ __forceinline__ void warp_row_tables(const BlockGeom &g, const BlockBufs &b, int Dsc, int row)
{
    const int lane = threadIdx.x & 31;
    const int nvx = g.nvx, nvy = g.nvy, Dc1 = Dsc - 1;
    const int iyl = b.rowi[row];
    const float dy = b.rowd[row];
    for (int ixl = lane; ixl < nvx; ixl += 32) {
        float v[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float a0 = b.fxy[(c * nvy + iyl) * nvx + ixl];
            const float a1 = b.fxy[(c * nvy + iyl + 1) * nvx + ixl];
            v[c] = fmaf(a1 - a0, dy, a0);
        }
        b.rxy[ixl] = make_float4(v[0], v[1], v[2], 0.f);
    }
    for (int e = lane; e < 3 * Dc1; e += 32) {
        const int c = e >= Dc1 ? (e >= 2 * Dc1 ? 2 : 1) : 0, j = e - c * Dc1;
        const float *r0 = b.fyc + (c * nvy + iyl) * Dsc + j;
        const float *r1 = r0 + Dsc;
        const float v0 = fmaf(r1[0] - r0[0], dy, r0[0]), v1 = fmaf(r1[1] - r0[1], dy, r0[1]);
        b.ryc[e] = make_float2(v0, v1 - v0);  // value at j and slope to j + 1
    }
}

// One LUT pair: add the folded, weighted bilinear value of the three output
// channels (coefficient form of Supp. Eq. 15) from the cell's 3 float4.
__device__ __forceinline__ void lut_pair(const float4 &q0, const float4 &q1, const float4 &q2, float da, float db,
                                         float &y0, float &y1, float &y2)
{
    y0 += fmaf(fmaf(q2.y, da, q1.z), db, fmaf(q0.w, da, q0.x));
    y1 += fmaf(fmaf(q2.z, da, q1.w), db, fmaf(q1.x, da, q0.y));
    y2 += fmaf(fmaf(q2.w, da, q2.x), db, fmaf(q1.y, da, q0.z));
}

// One LUT pair's part of the adjoint: with upstream gradients g of the three
// output channels, d/dp_alpha and d/dp_beta of sum_c g_c phi_c (weights
// already folded in): (D-1) (b + d db) and (D-1) (c + d da) per channel.
__device__ __forceinline__ void lut_pair_dx(const float4 &q0, const float4 &q1, const float4 &q2, float da, float db,
                                            const float (&g)[3], float fD1, float &ga, float &gb)
{
    // b = (q0.w, q1.x, q1.y), c = (q1.z, q1.w, q2.x), d = (q2.y, q2.z, q2.w)
    const float sa = g[0] * fmaf(q2.y, db, q0.w) + g[1] * fmaf(q2.z, db, q1.x) + g[2] * fmaf(q2.w, db, q1.y);
    const float sb = g[0] * fmaf(q2.y, da, q1.z) + g[1] * fmaf(q2.z, da, q1.w) + g[2] * fmaf(q2.w, da, q2.x);
    ga = fmaf(fD1, sa, ga);
    gb = fmaf(fD1, sb, gb);
}

static_assert(kTileW == 128, "the xcol table and the lane mapping assume 128-pixel tiles");

// Cell at byte offset off of the cell table (3 float4 per cell).
__device__ __forceinline__ const float4 *lut_at(const float4 *lcell, unsigned int off, unsigned int *check, int lim)
{
#ifdef SVDLUT_CHECK_BOUNDS
    return lcell + checked_index(check, kChkLut, static_cast<int>(off >> 4), lim);
#else
    (void)check;
    (void)lim;
    return reinterpret_cast<const float4 *>(reinterpret_cast<const char *>(lcell) + off);
#endif
}

// DX = false: the forward transform, y = f(x).
// DX = true (float images): the pixel part of the adjoint, dx = (df/dx)^T dy,
// from the slopes of the same cell coefficients (lut_pair_dx); the xc / yc
// terms add (Dsc-1) (s1 - s0) for their channel; zero where the input was
// clamped (outside [0,1]).
//
// A lane takes 4 adjacent pixels of a row (one 128-bit access per float
// plane).  Every pixel gathers its own cells: reusing a lane's previous cell
// when unchanged saved shared-memory wavefronts in smooth regions but cost
// more in compares than it saved.
template <class IO, int N, bool DX>
__global__ void __launch_bounds__(kThreads, 1) apply_kernel(const __grid_constant__ LaunchArgs<N> a)
{
    extern __shared__ __align__(16) float smem[];
    float4 *lcell = reinterpret_cast<float4 *>(smem);
    float *misc = smem + a.lcell_floats;
    float *scratch = misc + kMiscFloats;

    // the next kernel of the stream (e.g. the next call's prep_kernel, which
    // waits for this one before reading anything) may begin launching
    asm volatile("griddepcontrol.launch_dependents;\n" :::);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const bool xcol = a.xcol != 0;
    // Block schedule: a contiguous range per CTA, or (queue) blocks taken in
    // order from a global counter so that uneven blocks balance out.
    int *slot = reinterpret_cast<int *>(misc + kMaxK * 4 + 3);
    int blk, b_end;
    if (a.queue) {
        if (threadIdx.x == 0) *slot = static_cast<int>(atomicAdd(a.queue, 1u));
        __syncthreads();
        blk = *slot;
        b_end = a.total_blocks;
    } else {
        const int G = gridDim.x, gi = blockIdx.x;
        blk = static_cast<int>((static_cast<long long>(a.total_blocks) * gi) / G);
        b_end = static_cast<int>((static_cast<long long>(a.total_blocks) * (gi + 1)) / G);
    }
    if (blk >= b_end) return;

    using In = typename IO::In;
    using Out = typename IO::Out;
    using Raw = typename In::Raw;
    static_assert(!DX || std::is_same<IO, IoF32>::value, "the adjoint takes float images");
    // the lane's pixels of a tile row: columns x0 + lane * 4 + k, k < n
    auto lane_px = [&](int W, int x0, int &x) {
        x = x0 + lane * 4;
        return min(4, W - x);
    };

    auto find_image = [&](int blk) {
        int im = 0;
        while (im + 1 < a.n && a.img[im + 1].block_begin <= blk) ++im;
        return im;
    };
    constexpr int NP = DX ? 6 : 3;  // Raw words loaded per row: x (and dy)
    // this lane's pixels at image offset off (n of them, 0 for none)
    auto load_px = [&](const ImgDesc &d, size_t off, int n, size_t plane, Raw (&dst)[NP]) {
        const int nc = n > 0 ? checked_run(a.check, off, n, plane) : 0;
        if (nc > 0) {
            const void *px = In::at(d.x, off);
            In::load(px, plane, nc, checked_vec(a.check, d.vec, px, In::kVecAlign), dst);
        } else {
#pragma unroll
            for (int c = 0; c < 3; ++c) dst[c] = Raw();
        }
        if constexpr (DX) {
            const float *g = d.dy + off;
            const bool v = checked_vec(a.check, d.vec, g, 16);
#pragma unroll
            for (int c = 0; c < 3; ++c) dst[3 + c] = nc > 0 ? PixIO<float>::load(g + c * plane, nc, v) : Raw();
        }
    };
    // loads this lane's pixels of row `row` (block-relative) of block blk
    auto load_row = [&](int blk, int row, Raw (&dst)[NP]) {
        const ImgDesc &d = a.img[find_image(blk)];
        const int lb = blk - d.block_begin;
        const int band = lb / d.strips, strip = lb - band * d.strips;
        int x;
        const int n = lane_px(d.W, strip * kTileW, x);
        const int y = d.y_begin + band * d.BH + row;
        const bool ok = row < d.BH && y < d.y_end;
        load_px(d, static_cast<size_t>(y) * d.W + x, ok ? n : 0, static_cast<size_t>(d.H) * d.W, dst);
    };

    Raw cur[NP], nxt[NP];
    int cur_im = -1;
    bool first = true, pre_wait = a.pre != 0;
    for (;;) {
        const int im = find_image(blk);
        const ImgDesc &d = a.img[im];
        const BlockGeom g = block_geom(d, blk - d.block_begin, a.nvx_max, a.nvy_max);
        const BlockBufs b = block_bufs(scratch, g.nvx, g.nvy, d.Dsc, a.bh_max, xcol);
        // the first row's pixels are requested after the factor copies, so
        // that those do not queue behind them
        auto first_row = [&]() {
            if (first) {
                load_row(blk, warp, cur);
                first = false;
            }
        };
        __syncthreads();  // previous block's rows done with the buffers and the cell table
        if (a.pre) {
            // The pixels are inputs of the call, complete before the launch:
            // the first row is requested while the precomputation may still
            // run (programmatic dependent launch); the tables after it ends.
            first_row();
            if (pre_wait) {
                asm volatile("griddepcontrol.wait;\n" ::: "memory");
                pre_wait = false;
            }
            setup_pre(d, g, b, lcell, misc, im != cur_im);
            cp_async_wait_all();
            __syncthreads();
        } else if (im != cur_im) {
            build_luts(d, lcell, scratch, misc, a.scratch_floats, a.check);
            __syncthreads();
        }
        cur_im = im;
        first_row();
        if (a.queue && threadIdx.x == 0) *slot = static_cast<int>(atomicAdd(a.queue, 1u));
        block_phase_a(d, g, b, misc, !a.pre);
        __syncthreads();
        const int next = a.queue ? *slot : blk + 1;
        const bool has_next = next < b_end;
        block_phase_b(d, g, b, xcol);
        __syncthreads();

        // ---- rows of this warp ----
        const int D = d.D, Dsc = d.Dsc, Dc1 = Dsc - 1;
        const int nc3 = (D - 1) * D * 3;  // float4 per pair table
        const int D3 = D * 3;             // float4 per cell row
        const int lut_lim = 3 * nc3 - 2;  // each cell reads 3 float4
        const float fD1 = static_cast<float>(D - 1), fD2 = static_cast<float>(D - 2);
        const float fS1 = static_cast<float>(Dc1), fS2 = static_cast<float>(Dsc - 2);
        const float bias0 = misc[kMaxK * 4 + 0], bias1 = misc[kMaxK * 4 + 1], bias2 = misc[kMaxK * 4 + 2];
        int xbase;
        const int n = lane_px(d.W, g.x0, xbase);
        int ixl[4];
        float dxk[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            ixl[k] = b.coli[lane * 4 + k];
            dxk[k] = b.cold[lane * 4 + k];
        }
        // 4 adjacent pixels usually span at most two x-cells: 3 xy vertices
        const bool xy_fast = ixl[3] - ixl[0] <= 1;
        const int xcs = (g.nvx - 1) * Dsc;  // float4 per channel of pxc
        const float *xcl = b.xcol + lane;   // + (c * Dsc + j) * kTileW + k * 32
        const size_t plane = static_cast<size_t>(d.H) * d.W;
        // offset of this lane's pixels in row 0 of the block
        const size_t off0 = static_cast<size_t>(g.y0) * d.W + xbase;
        // xc slice of channel c at intensity cell j for pixel k: value at j
        // and slope to j + 1
        auto xc_slice = [&](int c, int j, int k, float &v, float &sl) {
            if (xcol) {
                const float *f = xcl + checked_index(a.check, kChkPxc, (c * Dsc + j) * kTileW + k * 32,
                                                     3 * Dsc * kTileW - kTileW - 31);
                v = f[0];
                sl = f[kTileW] - v;
            } else {
                const float4 q = b.pxc[checked_index(a.check, kChkPxc, c * xcs + ixl[k] * Dsc + j, 3 * xcs)];
                v = fmaf(q.z, dxk[k], q.x);
                sl = fmaf(q.w, dxk[k], q.y);
            }
        };
        // Fast rows (the common case, uniform over the block): per-column xc
        // tables, D - 1 = 2 (Dsc - 1) (the slice cell is the LUT cell halved:
        // the 17 intensity vertices are every other LUT vertex), and x-cells
        // at least 3 pixels wide (a lane's 4 pixels touch at most 2 of them).
        const bool fast = xcol && D - 1 == 2 * Dc1 && d.W - 1 >= 3 * (d.Dsx - 1);
        auto rows = [&](auto fast_tag) {
            constexpr bool FAST = decltype(fast_tag)::value;
            // fast rows: xy of pixel k = xa + w0[k] (xb - xa) + w1[k] (xc - xb)
            float w0[4], w1[4];
            if constexpr (FAST) {
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const bool c0 = ixl[k] == ixl[0];
                    w0[k] = c0 ? dxk[k] : 1.f;
                    w1[k] = c0 ? 0.f : dxk[k];
                }
            }
            const unsigned int rowB = static_cast<unsigned int>(D3) * 16u, pairB = static_cast<unsigned int>(nc3) * 16u;
            const unsigned int kRow = 0u - kCellBias * rowB, kCol = 0u - kCellBias * 48u;
#pragma unroll 1
            for (int row = warp; row < g.rows; row += kWarps) {
                // next row of this warp, possibly in the next block
                if (row + kWarps < g.rows) load_px(d, off0 + static_cast<size_t>(row + kWarps) * d.W, n, plane, nxt);
                else if (has_next) load_row(next, warp, nxt);
                const int y = g.y0 + row;
                warp_row_tables(g, b, Dsc, row);
                __syncwarp();
                float out[3][4];
                if constexpr (FAST) {
                    const float4 xa = b.rxy[ixl[0]], xb = b.rxy[ixl[0] + 1], xc = b.rxy[min(ixl[0] + 2, g.nvx - 1)];
                    const float base[3] = {bias0 + xa.x, bias1 + xa.y, bias2 + xa.z};
                    const float ab[3] = {xb.x - xa.x, xb.y - xa.y, xb.z - xa.z};
                    const float bc[3] = {xc.x - xb.x, xc.y - xb.y, xc.z - xb.z};
                    float4 pv[3];
                    In::unpack(cur, pv);
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        float p[3] = {get(pv[0], k), get(pv[1], k), get(pv[2], k)};
                        unsigned int cb[3];
                        float dc[3];
                        bool inside[3];
#pragma unroll
                        for (int c = 0; c < 3; ++c) {
                            inside[c] = p[c] >= 0.f && p[c] <= 1.f;
                            cb[c] = cell_bits(__saturatef(p[c]), fD1, fD2, dc[c]);
                        }
                        // LUT cells of the pairs rg, rb, gb: row offset of the first
                        // channel of the pair plus column offset of the second
                        const unsigned int Rr = cb[0] * rowB + kRow, Rg = cb[1] * rowB + kRow;
                        const unsigned int Cg = cb[1] * 48u + kCol, Cb = cb[2] * 48u + kCol;
                        const float4 *q0 = lut_at(lcell, Rr + Cg, a.check, lut_lim);
                        const float4 *q1 = lut_at(lcell, pairB + Rr + Cb, a.check, lut_lim);
                        const float4 *q2 = lut_at(lcell, 2u * pairB + Rg + Cb, a.check, lut_lim);
                        float yy[3];
#pragma unroll
                        for (int c = 0; c < 3; ++c) yy[c] = fmaf(w0[k], ab[c], fmaf(w1[k], bc[c], base[c]));
                        // slice cell: the LUT cell halved, e = (i mod 2 + frac) / 2
                        int jc[3];
                        float ec[3];
#pragma unroll
                        for (int c = 0; c < 3; ++c) {
                            jc[c] = static_cast<int>((cb[c] - kCellBias) >> 1);
                            ec[c] = fmaf(dc[c], 0.5f, (cb[c] & 1u) ? 0.5f : 0.f);
                        }
                        if constexpr (!DX) {
                            lut_pair(q0[0], q0[1], q0[2], dc[0], dc[1], yy[0], yy[1], yy[2]);
                            lut_pair(q1[0], q1[1], q1[2], dc[0], dc[2], yy[0], yy[1], yy[2]);
                            lut_pair(q2[0], q2[1], q2[2], dc[1], dc[2], yy[0], yy[1], yy[2]);
#pragma unroll
                            for (int c = 0; c < 3; ++c) {
                                const float *f = xcl + checked_index(a.check, kChkPxc, (c * Dsc + jc[c]) * kTileW + k * 32,
                                                                     3 * Dsc * kTileW - kTileW - 31);
                                const float2 r = b.ryc[checked_index(a.check, kChkRyc, c * Dc1 + jc[c], 3 * Dc1)];
                                const float v = f[0];
                                out[c][k] = fmaf((f[kTileW] - v) + r.y, ec[c], yy[c] + (v + r.x));
                            }
                            (void)inside;
                        } else {
                            const float gy[3] = {get(cur[3], k), get(cur[4], k), get(cur[5], k)};
                            float gp[3] = {0.f, 0.f, 0.f};
                            lut_pair_dx(q0[0], q0[1], q0[2], dc[0], dc[1], gy, fD1, gp[0], gp[1]);
                            lut_pair_dx(q1[0], q1[1], q1[2], dc[0], dc[2], gy, fD1, gp[0], gp[2]);
                            lut_pair_dx(q2[0], q2[1], q2[2], dc[1], dc[2], gy, fD1, gp[1], gp[2]);
#pragma unroll
                            for (int c = 0; c < 3; ++c) {
                                const float *f = xcl + checked_index(a.check, kChkPxc, (c * Dsc + jc[c]) * kTileW + k * 32,
                                                                     3 * Dsc * kTileW - kTileW - 31);
                                const float2 r = b.ryc[checked_index(a.check, kChkRyc, c * Dc1 + jc[c], 3 * Dc1)];
                                gp[c] = fmaf(gy[c] * fS1, (f[kTileW] - f[0]) + r.y, gp[c]);
                                out[c][k] = inside[c] ? gp[c] : 0.f;
                            }
                            (void)yy;
                            (void)ec;
                        }
                    }
                } else {
                    float4 xa, xb, xc;  // xy vertices ixl[0] .. ixl[0] + 2 (fast path)
                    if (xy_fast) {
                        xa = b.rxy[ixl[0]];
                        xb = b.rxy[ixl[0] + 1];
                        xc = b.rxy[min(ixl[0] + 2, g.nvx - 1)];
                    }
                    float4 pv[3];
                    In::unpack(cur, pv);
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        float4 q[3][3];  // cell coefficients of the three pairs
                        float2 ry[3];    // yc entries of the three channels
                        float p[3] = {get(pv[0], k), get(pv[1], k), get(pv[2], k)};
                        int ic[3], jc[3];
                        float dc[3], ec[3];
                        bool inside[3];
#pragma unroll
                        for (int c = 0; c < 3; ++c) {
                            inside[c] = p[c] >= 0.f && p[c] <= 1.f;
                            p[c] = __saturatef(p[c]);
                            ic[c] = cell_of(p[c], fD1, fD2, dc[c]);
                            jc[c] = cell_of(p[c], fS1, fS2, ec[c]);
                        }
                        // LUT pairs (rg, rb, gb): axes (A, B)
                        const int cid[3] = {ic[0] * D3 + ic[1] * 3, nc3 + ic[0] * D3 + ic[2] * 3,
                                            2 * nc3 + ic[1] * D3 + ic[2] * 3};
#pragma unroll
                        for (int pr = 0; pr < 3; ++pr) {
                            const float4 *c4 = lcell + checked_index(a.check, kChkLut, cid[pr], lut_lim);
                            q[pr][0] = c4[0];
                            q[pr][1] = c4[1];
                            q[pr][2] = c4[2];
                        }
#pragma unroll
                        for (int c = 0; c < 3; ++c) ry[c] = b.ryc[checked_index(a.check, kChkRyc, c * Dc1 + jc[c], 3 * Dc1)];
                        if constexpr (!DX) {
                            float y0 = bias0, y1 = bias1, y2 = bias2;
                            lut_pair(q[0][0], q[0][1], q[0][2], dc[0], dc[1], y0, y1, y2);
                            lut_pair(q[1][0], q[1][1], q[1][2], dc[0], dc[2], y0, y1, y2);
                            lut_pair(q[2][0], q[2][1], q[2][2], dc[1], dc[2], y0, y1, y2);
                            // xy slicing: row-interpolated vertices, lerp along x
                            const float4 r0 = xy_fast ? (ixl[k] == ixl[0] ? xa : xb)
                                                      : b.rxy[checked_index(a.check, kChkRxy, ixl[k], g.nvx)];
                            const float4 r1 = xy_fast ? (ixl[k] == ixl[0] ? xb : xc)
                                                      : b.rxy[checked_index(a.check, kChkRxy, ixl[k] + 1, g.nvx)];
                            const float dx = dxk[k];
                            const float yy[3] = {y0 + fmaf(r1.x - r0.x, dx, r0.x), y1 + fmaf(r1.y - r0.y, dx, r0.y),
                                                 y2 + fmaf(r1.z - r0.z, dx, r0.z)};
                            // xc + yc slicing share the intensity cell of channel c
#pragma unroll
                            for (int c = 0; c < 3; ++c) {
                                float v, sl;
                                xc_slice(c, jc[c], k, v, sl);
                                out[c][k] = fmaf(sl + ry[c].y, ec[c], yy[c] + (v + ry[c].x));
                            }
                            (void)inside;
                        } else {
                            const float gy[3] = {get(cur[3], k), get(cur[4], k), get(cur[5], k)};
                            float gp[3] = {0.f, 0.f, 0.f};
                            lut_pair_dx(q[0][0], q[0][1], q[0][2], dc[0], dc[1], gy, fD1, gp[0], gp[1]);
                            lut_pair_dx(q[1][0], q[1][1], q[1][2], dc[0], dc[2], gy, fD1, gp[0], gp[2]);
                            lut_pair_dx(q[2][0], q[2][1], q[2][2], dc[1], dc[2], gy, fD1, gp[1], gp[2]);
#pragma unroll
                            for (int c = 0; c < 3; ++c) {
                                float v, sl;
                                xc_slice(c, jc[c], k, v, sl);
                                gp[c] = fmaf(gy[c] * fS1, sl + ry[c].y, gp[c]);
                                out[c][k] = inside[c] ? gp[c] : 0.f;
                            }
                        }
                    }
                }
                const size_t off = static_cast<size_t>(y) * d.W + xbase;
                const int nc = checked_run(a.check, off, n, plane);
                if (nc > 0) {
                    if constexpr (!DX) {
                        const void *py = Out::at(d.y, off);
                        Out::store(d.y, plane, off, out, nc, checked_vec(a.check, d.vec, py, Out::kVecAlign));
                    } else {
                        float *py = static_cast<float *>(d.y) + off;
                        const bool v = checked_vec(a.check, d.vec, py, 16);
#pragma unroll
                        for (int c = 0; c < 3; ++c)
                            PixIO<float>::store(py + c * plane, make_float4(out[c][0], out[c][1], out[c][2], out[c][3]),
                                                nc, v);
                    }
                }
                __syncwarp();  // row tables are rewritten for the next row
#pragma unroll
                for (int c = 0; c < NP; ++c) cur[c] = nxt[c];
            }
        };
        if (fast) rows(std::true_type{});
        else rows(std::false_type{});
        if (warp >= g.rows && has_next) load_row(next, warp, cur);  // no row here
        if (!has_next) break;
        blk = next;
    }
}

}  // namespace svdlut
