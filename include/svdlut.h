/*
 * svdlut.h -- C ABI of the GB300 (sm_103a) SVDLUT library.
 *
 * SVDLUT (arXiv 2508.16121) enhances an image with an image-adaptive colour
 * transform stored as nine 2D LUTs, each rebuilt from rank-R SVD factors, and
 * adds 2D bilateral-grid slicing for spatial awareness; both are fused into one
 * per-pixel pass (Sec. 3.2.3, Eq. 10; Supp. Sec. C, Eqs. 12-22).
 *
 * Conventions shared by every entry point
 *  - All tensor pointers are DEVICE pointers unless stated otherwise; the
 *    caller owns every buffer.  The library does not allocate on these paths.
 *  - Calls are asynchronous on the given stream (a cudaStream_t, passed as
 *    svdlut_stream_t; NULL = legacy default stream).  Errors found on the host
 *    (bad arguments) are returned before anything is launched; a failed launch
 *    returns SVDLUT_ERR_CUDA.  svdlut_last_error() gives a thread-local message.
 *  - Images are planar (CHW) per image, batch-major: x[b][c][h][w], c = r,g,b.
 *    FP32 values are read as they are and clamped to [0,1] before lookup;
 *    8-bit values v are read as v/255.
 *  - Cell rule on an axis with D vertices: u = p (D-1), i = min(floor(u), D-2),
 *    delta = u - i  (Supp. Eqs. 13 and 18 with the upper edge kept inside).
 *  - Spatial coordinates x' = x/(W-1), y' = y/(H-1) (0 when W or H is 1), pixel
 *    indices as in Supp. Eq. 17.
 */
#ifndef SVDLUT_H
#define SVDLUT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *svdlut_stream_t; /* same type as cudaStream_t */

typedef enum {
    SVDLUT_OK = 0,
    SVDLUT_ERR_INVALID_ARG = 1, /* null pointer, bad size, misaligned pointer */
    SVDLUT_ERR_UNSUPPORTED = 2, /* valid but beyond the library's size limits */
    SVDLUT_ERR_CUDA = 3,        /* a CUDA call or launch failed              */
    SVDLUT_ERR_WORKSPACE = 4,   /* workspace missing or too small            */
    SVDLUT_ERR_TIMEOUT = 5      /* a bounded device-side wait ran out        */
} svdlut_status;

typedef enum {
    SVDLUT_F32 = 0, /* float32 in and out                                    */
    SVDLUT_U8 = 1   /* uint8 in and out; out = rint(clamp(Y,0,1)*255) in FP32 */
} svdlut_dtype;

/*
 * Sizes of one transform.
 *   D_t   LUT vertices per axis (paper: 33, Supp. Sec. A)        2 <= D_t <= 33
 *   rank  SVD rank N_s (paper: 8, Eq. 9)                          1 <= rank <= D_t
 *   K     number of 2D bilateral grids (paper: 6)                 0 <= K <= 48
 *   Dsx, Dsy, Dsc  grid vertices along x, y and intensity (paper: 17 each);
 *         Dsx, Dsy >= 2, 2 <= Dsc <= 64.
 */
typedef struct {
    int32_t D_t, rank, K, Dsx, Dsy, Dsc;
} svdlut_dims;

/*
 * Per-image transform parameters (Supp. Tables 9-12), FP32 device arrays with
 * a leading batch axis B (one set per image):
 *   U      [B][3 c][3 pair][D_t][rank]  pair order (rg, rb, gb); row i of U is
 *                                       vertex i of the pair's first axis
 *   S      [B][3][3][rank]              singular values (any sign)
 *   V      [B][3][3][D_t][rank]         row j is vertex j of the second axis
 *          so that t^c_p[i][j] = sum_r U[i][r] S[r] V[j][r]          (Eq. 9)
 *   lut_w  [B][3 c][4]                  (w_rg, w_rb, w_gb, b)        (Eq. 5)
 *   g_xy   [B][K][Dsy][Dsx]             plane over (y, x)
 *   g_xc   [B][K][Dsx][Dsc]             plane over (x, intensity)
 *   g_yc   [B][K][Dsy][Dsc]             plane over (y, intensity)
 *   grid_w [B][K][4]                    (w_xy, w_xc, w_yc, b)        (Supp. Eq. 21)
 * Grid k uses the intensity of channel k mod 3 and adds to output channel
 * k mod 3 (Eq. 10 / Supp. Eq. 22).  g_* and grid_w may be NULL when K == 0.
 */
typedef struct {
    const float *U, *S, *V, *lut_w, *g_xy, *g_xc, *g_yc, *grid_w;
} svdlut_params;

/*
 * svdlut_apply -- the fused 2D slicing + 2D LUT transform (Eq. 10, Supp. Eq. 22):
 *   Y_c = sum_p w^c_p I_bi(x, t^c_p) + b^c
 *       + sum_{k = c mod 3} [ w_xy I_bi((x',y'), g_xy) + w_xc I_bi((x',x_c), g_xc)
 *                             + w_yc I_bi((y',x_c), g_yc) + b_k ]
 * for B images of H x W.  x and y: [B][3][H][W] of dtype (float or uint8),
 * device, must not overlap.  Pointers must be 4-byte aligned for F32; 16-byte
 * alignment and W % 4 == 0 enable the vectorised path (any other case is
 * handled, more slowly).  Returns INVALID_ARG for null pointers, B, H or W < 1
 * or dims out of range; UNSUPPORTED for dims beyond the limits above, and when
 * the grid slices of one 128-pixel-wide block do not fit in shared memory
 * next to the LUT tables (grids much denser along x than one vertex per 8
 * pixels combined with a large Dsc and D_t).
 */
svdlut_status svdlut_apply(const svdlut_dims *dims, const svdlut_params *params, int B, int H,
                           int W, svdlut_dtype dtype, const void *x, void *y,
                           svdlut_stream_t stream);

/*
 * svdlut_apply_host -- svdlut_apply on images in HOST memory.
 *  - Page-locked (pinned, cudaHostAlloc / cudaHostRegister) x_host and y_host
 *    are mapped into the GPU's address space: the kernel reads and writes them
 *    in place over the CPU-GPU link, no copies, ws unused (may be NULL).
 *  - Otherwise each image is cut into row bands; the upload of a band, the
 *    transform of the previous one and the download of the one before run
 *    concurrently, on two copy streams owned by the library (created once per
 *    device) and on `stream` for the transform.  The copy streams fork from
 *    `stream` at the start and join it at the end.
 * Either way the call is ordered on `stream` like svdlut_apply (and can be
 * captured in a CUDA graph); y_host is complete when `stream` has reached the
 * end of the call.
 *   x_host, y_host  host memory, [B][3][H][W] of dtype, must not overlap
 *   params          DEVICE pointers, as for svdlut_apply
 *   ws, ws_bytes    pageable case: device workspace of
 *                   svdlut_apply_host_workspace_size() bytes, 256-byte aligned
 *                   (device copies of x and y)
 * Errors: those of svdlut_apply; WORKSPACE when ws is needed and missing or
 * too small.  Calls on one device are serialised on the host (the copy streams
 * are shared).
 */
svdlut_status svdlut_apply_host(const svdlut_dims *dims, const svdlut_params *params, int B, int H, int W,
                                svdlut_dtype dtype, const void *x_host, void *y_host, void *ws, size_t ws_bytes,
                                svdlut_stream_t stream);
size_t svdlut_apply_host_workspace_size(int B, int H, int W, svdlut_dtype dtype);

/*
 * One image of a ragged batch for svdlut_apply_batched: its size, transform
 * sizes and parameters (the svdlut_params layouts without the batch axis),
 * and device pointers to its [3][H][W] input and output.
 */
typedef struct {
    int32_t H, W;
    svdlut_dims dims;
    svdlut_params params;
    const void *x;
    void *y;
} svdlut_image;

/* Launch shape of svdlut_apply_batched: target pixels per work block (0 =
 * automatic: about four blocks per SM), persistent CTAs (0 = one per SM) and
 * the block schedule: SVDLUT_SCHED_QUEUE (0) has the CTAs take blocks from an
 * atomic counter (balances uneven blocks); SVDLUT_SCHED_RANGES (1) gives each
 * CTA a contiguous range of the image-major block list (fewer image switches,
 * hence fewer LUT rebuilds per CTA). */
typedef struct {
    int32_t block_px;
    int32_t ctas;
    int32_t schedule;
} svdlut_launch_cfg;

enum { SVDLUT_SCHED_QUEUE = 0, SVDLUT_SCHED_RANGES = 1 };

/*
 * svdlut_apply_cfg -- svdlut_apply with a launch shape: cfg->ctas > 0 plans
 * the work for and launches that many persistent CTAs (at most one per SM),
 * leaving the other SMs to concurrent work on other streams, e.g. the factor
 * generator of the next batch; cfg->block_px and cfg->schedule are not used
 * (the blocks are planned for the CTA count, in contiguous ranges).  cfg may
 * be NULL (= svdlut_apply).
 * Errors: those of svdlut_apply; INVALID_ARG for a negative CTA count.
 */
svdlut_status svdlut_apply_cfg(const svdlut_dims *dims, const svdlut_params *params, int B, int H, int W,
                               svdlut_dtype dtype, const void *x, void *y, const svdlut_launch_cfg *cfg,
                               svdlut_stream_t stream);

/*
 * svdlut_apply_ws -- svdlut_apply (with cfg as in svdlut_apply_cfg) whose
 * per-image tables are computed once per call into a caller workspace instead
 * of by every CTA: one small kernel rebuilds each image's nine 2D LUTs from
 * their factors (Eq. 9) times the pair weights (Eq. 5) in the per-cell
 * coefficient form of the bilinear interpolation (Supp. Eq. 15), folds the
 * grid slices per output channel (Supp. Eqs. 21-22) and sums the biases; the
 * transform kernel, launched as its programmatic dependent, copies its part
 * of those tables into shared memory.  The result is bit-identical to
 * svdlut_apply.
 * ws: device memory of at least svdlut_apply_workspace_size(dims, B) bytes,
 * 256-byte aligned, not overlapping x or y; its contents on entry do not
 * matter and are overwritten; concurrent calls must use different workspaces.
 * cfg may be NULL.
 * Errors: those of svdlut_apply_cfg; WORKSPACE (NULL or too small);
 * INVALID_ARG (misaligned or overlapping workspace).
 */
svdlut_status svdlut_apply_ws(const svdlut_dims *dims, const svdlut_params *params, int B, int H, int W,
                              svdlut_dtype dtype, const void *x, void *y, const svdlut_launch_cfg *cfg, void *ws,
                              size_t ws_bytes, svdlut_stream_t stream);

/* Workspace bytes of svdlut_apply_ws for B images of these dims (0 if the
 * dims are invalid or B < 1): per image 4 * 3 * (D_t-1) * D_t * 12 bytes of
 * cell table plus 4 * (3 * (Dsy*Dsx + Dsx*Dsc + Dsy*Dsc) + 3) bytes of folded
 * grids and biases, each rounded up to 256 bytes. */
size_t svdlut_apply_workspace_size(const svdlut_dims *dims, int B);

/*
 * svdlut_apply_batched -- the fused transform of svdlut_apply (Eq. 10) over n
 * images of uneven sizes, each with its own transform, in one persistent
 * launch per 64 images.  imgs is a HOST array of n descriptors (read during the
 * call only).  With the queue schedule the images' blocks are taken from a
 * counter in ws; either way the call is capturable in a CUDA graph (a 4-byte
 * memset, for the queue, + one kernel per 64 images).
 * ws: device memory of svdlut_batched_workspace_size(n) bytes, 4-byte aligned;
 * concurrent calls must use different workspaces.  cfg may be NULL.
 * Errors: INVALID_ARG (a bad image, reported with its index), WORKSPACE,
 * UNSUPPORTED, CUDA.
 */
svdlut_status svdlut_apply_batched(const svdlut_image *imgs, int n, svdlut_dtype dtype,
                                   const svdlut_launch_cfg *cfg, void *ws, size_t ws_bytes,
                                   svdlut_stream_t stream);

/* Workspace bytes for a batch of n images (0 if n < 1): the block-queue
 * counters.  With this minimum every CTA rebuilds the tables of each image it
 * meets. */
size_t svdlut_batched_workspace_size(int n);

/* Workspace bytes for these n images with their per-image tables (the LUT
 * cell tables and folded grids of svdlut_apply_ws, computed once per call by
 * one small kernel and copied into each CTA); 0 on bad arguments.  A
 * workspace of at least this size, 256-byte aligned, makes
 * svdlut_apply_batched use them (same results, bit for bit). */
size_t svdlut_batched_tables_workspace_size(const svdlut_image *imgs, int n);

/*
 * svdlut_autotune_batched -- times svdlut_apply_batched on this batch for a
 * set of block sizes, each with both schedules (reps timed launches each,
 * after one warm-up) and
 * returns the fastest launch shape in *best (and its time in *best_ms if not
 * NULL).  Synchronises the stream; not capturable.  Writes the images' y.
 */
svdlut_status svdlut_autotune_batched(const svdlut_image *imgs, int n, svdlut_dtype dtype, void *ws,
                                      size_t ws_bytes, svdlut_stream_t stream, int reps,
                                      svdlut_launch_cfg *best, float *best_ms);

/*
 * Gradient outputs of svdlut_backward: device FP32 arrays with the layouts of
 * the matching svdlut_params fields (leading batch axis B).  Any pointer may
 * be NULL (that gradient is not computed).  Wanted outputs are overwritten.
 */
typedef struct {
    float *dU, *dS, *dV, *dlut_w, *dg_xy, *dg_xc, *dg_yc, *dgrid_w;
} svdlut_grads;

/*
 * svdlut_backward -- adjoint of svdlut_apply for FP32 images.
 * The paper trains end to end through the fused transform (Sec. 4.2) without
 * printing its derivative; this is the exact derivative of the map above:
 *   G^c_p = sum_px dy_c * (bilinear weights of (x_a, x_b))   per LUT vertex
 *   dT^c_p = w^c_p G^c_p;  dU = dT V diag(S),  dV = dT^T U diag(S),
 *   dS_r = sum_ij dT_ij U_ir V_jr;  dw^c_p = <G^c_p, T^c_p>;  db^c = sum dy_c
 *   grids likewise (dg^k = w^k * scatter of dy_{k mod 3}, dw^k = <scatter, g^k>);
 *   dx_a = [0 <= x_a <= 1] * (sum of dy-weighted slopes of every bilinear
 *          term that reads x_a).
 * x, dy: [B][3][H][W] FP32 device (x is the forward input).  dx: same shape,
 * may be NULL.  Parameter gradients are deterministic: no atomics, every sum
 * is taken in a fixed order, so repeated calls give identical bits.
 * Workspace: device memory of at least svdlut_backward_workspace_size(...)
 * bytes, 256-byte aligned, owned by the caller; contents on entry are
 * ignored.  Returns SVDLUT_ERR_WORKSPACE if ws is NULL or too small while
 * a parameter gradient is requested (dx alone needs no workspace).
 */
svdlut_status svdlut_backward(const svdlut_dims *dims, const svdlut_params *params, int B, int H,
                              int W, const float *x, const float *dy, float *dx,
                              const svdlut_grads *grads, void *ws, size_t ws_bytes,
                              svdlut_stream_t stream);

/* Bytes of workspace svdlut_backward needs for these sizes (0 on bad args). */
size_t svdlut_backward_workspace_size(const svdlut_dims *dims, int B, int H, int W);

/*
 * ---- learned factor generator (Supp. Sec. A, Tables 8-12) ----
 * A 256x256 bilinear thumbnail of the input goes through five 3x3 stride-2
 * convolutions (3->8->16->32->64->64 channels; LeakyReLU 0.2, then affine
 * InstanceNorm on the first four), Dropout(0.5) while training, average
 * pooling to 64x2x2 = 256 features and four heads of two FC layers (256->8->n):
 * the 2D bilateral grids (K x 3 planes of 17x17), their weights (K x 4), the
 * SVD factors of the nine 2D LUTs (D_t = 33, rank 8: U, S, V) and the LUT
 * weights (3 x 4).  Its outputs are the svdlut_params of svdlut_apply with
 * dims {33, 8, K, 17, 17, 17}.  The convolutions run on the tensor cores
 * (tcgen05) with FP32 accumulation: BF16 operands in the forward pass,
 * split-BF16 operands (about 16 mantissa bits) for the weight and input
 * gradients; all other arithmetic is FP32.
 *
 * Weights: one FP32 device array of svdlut_generator_param_count(K) floats,
 * in this order: for conv i = 0..4: w [Cout][Cin][3][3], b [Cout], and for
 * i < 4 the InstanceNorm scale [Cout] and shift [Cout]; then for the heads
 * grids, grid weights, LUT factors, LUT weights: w1 [8][256], b1 [8],
 * w2 [n][8], b2 [n] with n = K*3*17*17, K*4, 9*(33*8+8+33*8), 12.  The factor
 * head's outputs are U ([3][3][33][8]), then S ([3][3][8]), then V; the grid
 * head's are [K][plane xy, xc, yc][17][17].  At K = 6 there are 160,478
 * parameters (the paper's Table 6).
 */

/* Writable parameter buffers (layouts of svdlut_params, leading batch axis). */
typedef struct {
    float *U, *S, *V, *lut_w, *g_xy, *g_xc, *g_yc, *grid_w;
} svdlut_param_buffers;

/* Number of FP32 weights of the generator with K grids (0 if K is out of range). */
size_t svdlut_generator_param_count(int K);

/* Workspace bytes for a batch of B images (activations kept for backward). */
size_t svdlut_generator_workspace_size(int K, int B);

/*
 * svdlut_generator_forward -- predicts the transform parameters of B images.
 * x: [B][3][H][W] FP32 device, any H, W >= 1 (bilinearly resized to 256x256).
 * training != 0 applies Dropout(0.5) with a mask drawn from SplitMix64 counters
 * (element e of [B][64][8][8] kept when the top bit of splitmix64(seed*2^32+e)
 * is 0).  ws (256-byte aligned, svdlut_generator_workspace_size bytes) keeps
 * the activations for svdlut_generator_backward.
 */
svdlut_status svdlut_generator_forward(int K, const float *weights, int B, int H, int W, const float *x,
                                       const svdlut_param_buffers *out, int training, uint64_t seed,
                                       void *ws, size_t ws_bytes, svdlut_stream_t stream);

/*
 * svdlut_generator_backward -- gradient of sum(dparams * params) with
 * respect to the weights (dweights, overwritten), using the activations the
 * last svdlut_generator_forward left in ws (same K, B, training and seed).
 * Deterministic (fixed-order reductions, no atomics).
 */
svdlut_status svdlut_generator_backward(int K, const float *weights, int B, const svdlut_params *dparams,
                                        float *dweights, int training, uint64_t seed, void *ws,
                                        size_t ws_bytes, svdlut_stream_t stream);

/* One Adam step on n FP32 weights (Sec. 4.2 trains with Adam): m, v are the
 * moment buffers, step >= 1 is the 1-based step count (bias correction). */
svdlut_status svdlut_generator_adam(float *weights, const float *grads, float *m, float *v, size_t n,
                                    float lr, float beta1, float beta2, float eps, int step,
                                    svdlut_stream_t stream);

/* MSE loss (Sec. 3.3, the first term of the training loss): *loss =
 * mean((y - target)^2) over n floats and, if dy is not NULL, dy = 2 (y -
 * target) / n.  ws: at least 4096 bytes of device scratch.  Deterministic. */
svdlut_status svdlut_mse(const float *y, const float *target, size_t n, float *dy, float *loss, void *ws,
                         size_t ws_bytes, svdlut_stream_t stream);

/*
 * svdlut_cie94 -- the colour-difference term of the training loss (Eq. 11,
 * weight lambda_c = 0.005 in the paper): *loss = mean over the B*H*W pixels
 * of the CIE94 difference between y and the reference `target` in CIELAB:
 *   sRGB decoding (IEC 61966-2-1) of the raw values, XYZ by the matrix of the
 *   sRGB primaries and the D65 white (0.3127, 0.3290), CIELAB relative to
 *   that white, CIE94 with kL = kC = kH = 1, K1 = 0.045, K2 = 0.015 and
 *   S_C, S_H from the reference's chroma.
 * If dy is not NULL, weight * d(*loss)/dy is written to dy (accumulate = 0)
 * or added to it (accumulate != 0); the gradient is 0 where the difference
 * is 0.  y, target, dy: [B][3][H][W] float device arrays; loss: one device
 * float; ws: at least 4096 bytes of device scratch.  Deterministic.
 */
svdlut_status svdlut_cie94(const float *y, const float *target, int B, int H, int W, float weight, float *dy,
                           int accumulate, float *loss, void *ws, size_t ws_bytes, svdlut_stream_t stream);

/*
 * svdlut_backward_noalloc -- svdlut_backward for callers that cannot allocate
 * device memory.  The paper has no counterpart; this is a library service.
 *
 * Some callers may not call cudaMalloc / cudaFree or any allocating routine
 * themselves: a host whose device memory belongs to another runtime's pool,
 * or a latency-critical loop where an allocation could stall on a device-wide
 * synchronisation.  This entry takes
 * the same arguments as svdlut_backward minus the workspace; its scratch space
 * is a fixed 32 MiB array inside the library (present on every GPU that loads
 * it, until the process exits), and it allocates nothing.
 *  - Sizes whose svdlut_backward_workspace_size exceeds 32 MiB are rejected
 *    with SVDLUT_ERR_UNSUPPORTED.  The workspace plan depends on the GPU's SM
 *    count; on a 152-SM GB300, 8 x 1920x1080 and one 3840x2160 image (D_t=33,
 *    rank 8, K=8 grids at 1/8 resolution) fit.
 *  - The first call on a device looks up the array's device address (one
 *    cudaGetSymbolAddress with that device current); make that first call
 *    before any stream capture.  The lookup is repeated when the current
 *    context has changed (e.g. after cudaDeviceReset).
 *  - All calls share the one array and leave their data in it.  Calls whose
 *    kernels overlap on the GPU (other streams, other threads) race on it:
 *    serialise them, e.g. on one stream.
 */
svdlut_status svdlut_backward_noalloc(const svdlut_dims *dims, const svdlut_params *params, int B, int H,
                                      int W, const float *x, const float *dy, float *dx,
                                      const svdlut_grads *grads, svdlut_stream_t stream);

/*
 * svdlut_tensor_core_timeouts -- number of warps of the generator's tcgen05
 * kernels (the forward convolutions of svdlut_generator_forward, the weight-
 * and input-gradient GEMMs of svdlut_generator_backward) whose bounded wait
 * for their matrix multiplies expired since the last call, on the current
 * device; the counter is then reset.  A tile whose wait expired writes NaN
 * instead of its result.  count: host pointer, required.  Synchronises the
 * device (errors of earlier asynchronous work are returned).  Not a
 * computation of the paper.
 */
svdlut_status svdlut_tensor_core_timeouts(uint32_t *count);

/* Message of the last error raised on this thread ("" if none). */
const char *svdlut_last_error(void);

/*
 * svdlut_apply_original -- the paper's original, unfused structure (the "1x1
 * conv" model of Table 6; Eqs. 7, 8 and 5), kept for comparison with the fused
 * transform: K spatial maps f_s[k] = w_xy psi_xy + w_xc psi_xc + w_yc psi_yc +
 * b_k are written to the workspace, then Xbar = 1x1 conv (K+3 -> 3) of
 * concat(x, f_s), then y = the 2D LUT transform of Xbar (inputs clamped to
 * [0,1] for the lookups, as in svdlut_apply).
 *   fusion   [B][3 (K+3) + 3] device floats: weights [3 out][K+3 in] (input
 *            channels r, g, b, then the K maps), then biases [3]
 *   x, y     [B][3][H][W] float device arrays, must not overlap
 *   ws       device workspace of svdlut_apply_original_workspace_size()
 *            bytes, 256-byte aligned (f_s and Xbar)
 * Errors: those of svdlut_apply; WORKSPACE when ws is missing or too small.
 */
svdlut_status svdlut_apply_original(const svdlut_dims *dims, const svdlut_params *params, const float *fusion,
                                    int B, int H, int W, const float *x, float *y, void *ws, size_t ws_bytes,
                                    svdlut_stream_t stream);
size_t svdlut_apply_original_workspace_size(const svdlut_dims *dims, int B, int H, int W);

/*
 * Pixel formats of svdlut_apply_io.  Planar formats are [B][3][H][W],
 * interleaved (HWC) ones [B][H][W][3] with channels (r, g, b) per pixel.
 * Integer inputs map code v to v / 255 (8-bit) or v / 65535 (16-bit);
 * 8-bit outputs are rint(clamp(Y, 0, 1) * 255) as for SVDLUT_U8.  The
 * 16-bit inputs are those of the tone-mapping and PPR10K tasks (Sec. 4.1).
 */
typedef enum {
    SVDLUT_PIX_F32 = 0,     /* planar float                    */
    SVDLUT_PIX_U8 = 1,      /* planar 8-bit                    */
    SVDLUT_PIX_U16 = 2,     /* planar 16-bit (input only)      */
    SVDLUT_PIX_U8_HWC = 3,  /* interleaved 8-bit               */
    SVDLUT_PIX_U16_HWC = 4  /* interleaved 16-bit (input only) */
} svdlut_pixfmt;

/*
 * svdlut_apply_io -- svdlut_apply between pixel formats: the same transform
 * (Eq. 10, Supp. Eq. 22) with the input decoded and the output encoded.
 * Supported (input -> output) pairs:
 *   F32 -> F32, U8 -> U8 (as svdlut_apply), U16 -> U8, U16 -> F32,
 *   U8_HWC -> U8_HWC, U16_HWC -> U8_HWC.
 * Interleaved 8-bit frames are decoded and encoded inside the transform
 * kernel.  16-bit inputs are first decoded (float(v) * float(1 / 65535)) into
 * an FP32 frame of up to 16 images (up to 16 * 3 * H * W floats), which this
 * call takes from the device's stream-ordered allocator (cudaMallocAsync /
 * cudaFreeAsync on `stream`) and returns before it ends on the stream; the
 * results equal those of the float path on the decoded values.
 * x and y are device arrays of B images of H x W in their formats and must not
 * overlap; float arrays 4-byte aligned, 16-bit arrays 2-byte aligned.  W % 4
 * == 0 with 16-byte aligned arrays enables the vector path.  Errors: those of
 * svdlut_apply; CUDA when the temporary cannot be allocated; UNSUPPORTED for
 * any other pair of formats.
 */
svdlut_status svdlut_apply_io(const svdlut_dims *dims, const svdlut_params *params, int B, int H, int W,
                              svdlut_pixfmt in_fmt, const void *x, svdlut_pixfmt out_fmt, void *y,
                              svdlut_stream_t stream);

/*
 * svdlut_lut3d_apply -- the 3D LUT transform the paper starts from (Eq. 3):
 * y_c = trilinear interpolation, at the clamped (r, g, b) of each pixel, of
 * the table t^c over the D x D x D vertex grid, for B images of H x W.
 *   lut3d  [B][3 c][D][D][D] device floats, index [r][g][b]
 *   x, y   [B][3][H][W] float device arrays
 *   ws     device workspace of svdlut_lut3d_workspace_size(D, B) bytes,
 *          16-byte aligned (the tables repacked as one float4 per vertex)
 * 2 <= D <= 33.  Errors: INVALID_ARG for null or misaligned pointers, bad
 * sizes; WORKSPACE when ws is missing or too small.
 */
svdlut_status svdlut_lut3d_apply(int D, const float *lut3d, int B, int H, int W, const float *x, float *y,
                                 void *ws, size_t ws_bytes, svdlut_stream_t stream);
size_t svdlut_lut3d_workspace_size(int D, int B);

/*
 * svdlut_lut3d_fit2d -- the best approximation of each 3D table by a sum of
 * 2D tables, the hypothesis behind the 2D LUT (Eq. 4): the least-squares fit
 * over the vertex grid, t[i][j][k] ~ A[i][j] + Bt[i][k] + C[j][k], which is
 * the second-order ANOVA projection (m: means over the dotted indices)
 *   A = m_ij.,  Bt = m_i.k - m_i..,  C = m_.jk - m_.j. - m_..k + m_... .
 *   lut3d   [B][3 c][D][D][D] device floats
 *   tables  [B][3 c][3 pair (A, Bt, C)][D][D] device floats, written: this
 *           is the U array of svdlut_params for rank = D with S = 1, V = the
 *           identity and lut_w = (1, 1, 1, 0), so svdlut_apply can run the fit
 *   rms     [B][3] device floats, written: RMS of the residual over the grid
 * 2 <= D <= 33.  Errors: INVALID_ARG for null pointers or bad sizes.
 */
svdlut_status svdlut_lut3d_fit2d(int D, const float *lut3d, int B, float *tables, float *rms,
                                 svdlut_stream_t stream);

/*
 * svdlut_check_report -- index-check status of a library built with
 * -DSVDLUT_CHECK_BOUNDS (a debugging build in which the transform kernels
 * test every shared-memory gather index, count the ones out of range and
 * replace them by 0 instead of faulting).  Waits for the device, copies
 * out[0] = failures, out[1] = site (1 LUT cell, 2 xc slice, 3 yc slice,
 * 4 xy slice), out[2] = index and out[3] = limit of the first failure, and
 * clears them.  The paper has no counterpart.  Returns UNSUPPORTED (out
 * zeroed) in the normal build.
 */
svdlut_status svdlut_check_report(uint32_t out[4]);

/* Library version, e.g. "svdlut 0.1.0 sm_103a". */
const char *svdlut_version(void);

#ifdef __cplusplus
}
#endif

#endif /* SVDLUT_H */
