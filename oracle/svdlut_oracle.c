/*
 * FP64 CPU oracle for the SVDLUT transform (arXiv 2508.16121).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code,
 * header, table or constant with the CUDA path.
 *
 * It computes, term by term and in double precision, what the paper
 * defines:
 *   - 2D LUTs rebuilt from SVD factors, T = U diag(S) V^T   (Eq. 9)
 *   - 2D LUT transform by bilinear interpolation           (Eq. 5 / Supp. Eqs. 12-16)
 *   - 2D slicing of bilateral grids                         (Eq. 7 / Supp. Eqs. 17-21)
 *   - the fused sum Y_c = Phi^c + sum_{k = c mod 3} Psi^k   (Eq. 10 / Supp. Eq. 22)
 * plus the adjoint of that map (the paper trains end to end through it,
 * Sec. 4.2, but prints no formula: the adjoint below is the derivative of
 * the forward written here).
 *
 * Readings of the paper taken here (each is also listed in the design notes):
 *   - Supp. Eq. 16 repeats w_rb*phi_rb; the third term is w_gb*phi_gb (Eq. 5).
 *   - Cell of a query p on D vertices: u = p (D-1), i = min(floor(u), D-2),
 *     delta = u - i  (Supp. Eq. 13 with the upper edge kept inside the table).
 *   - Inputs are clamped to [0,1] before lookup.
 *   - x' = x/(W-1), y' = y/(H-1) with integer pixel indices; 0 when W or H is 1.
 *   - Grid k feeds output channel k mod 3 and uses that channel's intensity,
 *     for any K >= 0 (Supp. Eq. 22 generalised from K divisible by 3).
 *   - Layouts: U, V [3 c][3 pair][D][R] (pair order rg, rb, gb; U rows index
 *     the first axis of the pair), S [3][3][R], lut_w [3][4] = (w_rg, w_rb,
 *     w_gb, b); g_xy [K][Dsy][Dsx], g_xc [K][Dsx][Dsc], g_yc [K][Dsy][Dsc],
 *     grid_w [K][4] = (w_xy, w_xc, w_yc, b).  Leading batch axis B on all.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

/* dims[6] = {D_t, rank, K, Dsx, Dsy, Dsc} */
enum { O_DT = 0, O_R, O_K, O_DSX, O_DSY, O_DSC };

/* channel on each axis of a pair: rg, rb, gb (Supp. Eq. 12) */
static const int AX_A[3] = {0, 0, 1};
static const int AX_B[3] = {1, 2, 2};

/* ---- Eq. 9: T = U diag(S) V^T for one D x D table ---- */
void oracle_lut_from_svd(int D, int R, const double *U, const double *S,
                         const double *V, double *T)
{
    for (int i = 0; i < D; ++i)
        for (int j = 0; j < D; ++j) {
            double t = 0.0;
            for (int r = 0; r < R; ++r)
                t += U[i * R + r] * S[r] * V[j * R + r];
            T[i * D + j] = t;
        }
}

/* Supp. Eq. 13 cell rule: lower vertex index and fractional position. */
static void cell(double p, int D, int *i, double *d)
{
    double u = p * (double)(D - 1);
    int k = (int)floor(u);
    if (k > D - 2) k = D - 2;
    if (k < 0) k = 0;
    *i = k;
    *d = u - (double)k;
}

/* Supp. Eqs. 13-15 (and 18-20): bilinear read of tab[a][b] with row stride ld,
 * Da x Db vertices, at (pa, pb) in [0,1]^2. */
static double bilinear(const double *tab, int ld, int Da, int Db, double pa, double pb)
{
    int i, j;
    double da, db;
    cell(pa, Da, &i, &da);
    cell(pb, Db, &j, &db);
    double v00 = tab[i * ld + j];
    double v10 = tab[(i + 1) * ld + j];
    double v01 = tab[i * ld + j + 1];
    double v11 = tab[(i + 1) * ld + j + 1];
    return (1.0 - da) * (1.0 - db) * v00 + da * (1.0 - db) * v10
         + (1.0 - da) * db * v01 + da * db * v11;
}

static double clamp01(double v) { return v < 0.0 ? 0.0 : (v > 1.0 ? 1.0 : v); }

static double coord(int x, int W) { return W > 1 ? (double)x / (double)(W - 1) : 0.0; }

typedef struct {
    int D, R, K, Dsx, Dsy, Dsc;
    const double *U, *S, *V, *lw, *gxy, *gxc, *gyc, *gw;
} img_params;

static img_params params_of(const int *dims, int b, const double *U, const double *S,
                            const double *V, const double *lut_w, const double *g_xy,
                            const double *g_xc, const double *g_yc, const double *grid_w)
{
    img_params q;
    q.D = dims[O_DT]; q.R = dims[O_R]; q.K = dims[O_K];
    q.Dsx = dims[O_DSX]; q.Dsy = dims[O_DSY]; q.Dsc = dims[O_DSC];
    size_t nf = (size_t)9 * q.D * q.R;
    q.U = U + (size_t)b * nf;
    q.V = V + (size_t)b * nf;
    q.S = S + (size_t)b * 9 * q.R;
    q.lw = lut_w + (size_t)b * 12;
    q.gxy = g_xy + (size_t)b * q.K * q.Dsy * q.Dsx;
    q.gxc = g_xc + (size_t)b * q.K * q.Dsx * q.Dsc;
    q.gyc = g_yc + (size_t)b * q.K * q.Dsy * q.Dsc;
    q.gw = grid_w + (size_t)b * q.K * 4;
    return q;
}

/* the nine tables T^c_p of one image, [c][p][D][D] */
static double *build_tables(const img_params *q)
{
    int D = q->D, R = q->R;
    double *T = (double *)malloc(sizeof(double) * 9 * D * D);
    for (int cp = 0; cp < 9; ++cp)
        oracle_lut_from_svd(D, R, q->U + (size_t)cp * D * R, q->S + cp * R,
                            q->V + (size_t)cp * D * R, T + (size_t)cp * D * D);
    return T;
}

/* Forward of one pixel: Eq. 5 (LUT transform), Eq. 7 (slicing), Eq. 10 (sum).
 * p[3] clamped colour, (xs, ys) normalised position. */
static void pixel_forward(const img_params *q, const double *T, const double p[3],
                          double xs, double ys, double y[3])
{
    int D = q->D;
    for (int c = 0; c < 3; ++c) {
        /* Phi^c = w_rg phi_rg + w_rb phi_rb + w_gb phi_gb + b^c */
        double Phi = 0.0;
        for (int pr = 0; pr < 3; ++pr) {
            double phi = bilinear(T + (size_t)(c * 3 + pr) * D * D, D, D, D,
                                  p[AX_A[pr]], p[AX_B[pr]]);
            Phi += q->lw[c * 4 + pr] * phi;
        }
        Phi += q->lw[c * 4 + 3];
        y[c] = Phi;
    }
    for (int k = 0; k < q->K; ++k) {
        int c = k % 3;
        const double *w = q->gw + k * 4;
        double psi_xy = bilinear(q->gxy + (size_t)k * q->Dsy * q->Dsx, q->Dsx, q->Dsy, q->Dsx, ys, xs);
        double psi_xc = bilinear(q->gxc + (size_t)k * q->Dsx * q->Dsc, q->Dsc, q->Dsx, q->Dsc, xs, p[c]);
        double psi_yc = bilinear(q->gyc + (size_t)k * q->Dsy * q->Dsc, q->Dsc, q->Dsy, q->Dsc, ys, p[c]);
        y[c] += w[0] * psi_xy + w[1] * psi_xc + w[2] * psi_yc + w[3];
    }
}

/* Forward over a batch.  x, y: [B][3][H][W] doubles (x in [0,1] scale;
 * values outside are clamped).  Returns 0 on success. */
int oracle_forward(const int *dims, int B, int H, int W,
                   const double *U, const double *S, const double *V, const double *lut_w,
                   const double *g_xy, const double *g_xc, const double *g_yc,
                   const double *grid_w, const double *x, double *y, int nthreads)
{
    size_t plane = (size_t)H * W;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
    for (int b = 0; b < B; ++b) {
        img_params q = params_of(dims, b, U, S, V, lut_w, g_xy, g_xc, g_yc, grid_w);
        double *T = build_tables(&q);
        const double *xb = x + (size_t)b * 3 * plane;
        double *yb = y + (size_t)b * 3 * plane;
#pragma omp parallel for schedule(static)
        for (int row = 0; row < H; ++row) {
            for (int col = 0; col < W; ++col) {
                size_t o = (size_t)row * W + col;
                double p[3], out[3];
                for (int c = 0; c < 3; ++c) p[c] = clamp01(xb[c * plane + o]);
                pixel_forward(&q, T, p, coord(col, W), coord(row, H), out);
                for (int c = 0; c < 3; ++c) yb[c * plane + o] = out[c];
            }
        }
        free(T);
    }
    return 0;
}

/* The paper's original (unfused) structure, the "1x1 conv" model of Table 6:
 *   f_s[k] = w_xy psi_xy + w_xc psi_xc + w_yc psi_yc + b_k        (Eq. 7, K maps)
 *   Xbar_c = sum_i Wf[c][i] X_i + sum_k Wf[c][3+k] f_s[k] + bf[c]  (Eq. 8, 1x1 conv)
 *   Y_c    = w_rg phi_rg(Xbar) + w_rb phi_rb(Xbar) + w_gb phi_gb(Xbar) + b^c   (Eq. 5)
 * The slices read the clamped input intensity of channel k mod 3; the conv
 * takes the input as given; the LUT lookup clamps Xbar to [0,1] (reading R6).
 * fusion: [B][3][K+3] weights then [B][3] biases, i.e. [B][3 (K+3) + 3].
 * Grid arguments may be NULL when K == 0. */
int oracle_forward_original(const int *dims, int B, int H, int W,
                            const double *U, const double *S, const double *V, const double *lut_w,
                            const double *g_xy, const double *g_xc, const double *g_yc,
                            const double *grid_w, const double *fusion, const double *x, double *y,
                            int nthreads)
{
    size_t plane = (size_t)H * W;
    const int K = dims[2], nf = 3 * (K + 3) + 3;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
    for (int b = 0; b < B; ++b) {
        img_params q = params_of(dims, b, U, S, V, lut_w, g_xy, g_xc, g_yc, grid_w);
        double *T = build_tables(&q);
        const double *xb = x + (size_t)b * 3 * plane;
        const double *Wf = fusion + (size_t)b * nf, *bf = Wf + 3 * (K + 3);
        double *yb = y + (size_t)b * 3 * plane;
        int D = q.D;
#pragma omp parallel for schedule(static)
        for (int row = 0; row < H; ++row) {
            double *fs = (double *)malloc(sizeof(double) * (K > 0 ? K : 1));
            for (int col = 0; col < W; ++col) {
                size_t o = (size_t)row * W + col;
                double xin[3], p[3], xs = coord(col, W), ys = coord(row, H);
                for (int c = 0; c < 3; ++c) {
                    xin[c] = xb[c * plane + o];
                    p[c] = clamp01(xin[c]);
                }
                for (int k = 0; k < K; ++k) {
                    int c = k % 3;
                    const double *w = q.gw + k * 4;
                    fs[k] = w[0] * bilinear(q.gxy + (size_t)k * q.Dsy * q.Dsx, q.Dsx, q.Dsy, q.Dsx, ys, xs)
                          + w[1] * bilinear(q.gxc + (size_t)k * q.Dsx * q.Dsc, q.Dsc, q.Dsx, q.Dsc, xs, p[c])
                          + w[2] * bilinear(q.gyc + (size_t)k * q.Dsy * q.Dsc, q.Dsc, q.Dsy, q.Dsc, ys, p[c])
                          + w[3];
                }
                double xbar[3];
                for (int c = 0; c < 3; ++c) {
                    double v = bf[c];
                    for (int i = 0; i < 3; ++i) v += Wf[c * (K + 3) + i] * xin[i];
                    for (int k = 0; k < K; ++k) v += Wf[c * (K + 3) + 3 + k] * fs[k];
                    xbar[c] = clamp01(v);
                }
                for (int c = 0; c < 3; ++c) {
                    double Phi = q.lw[c * 4 + 3];
                    for (int pr = 0; pr < 3; ++pr)
                        Phi += q.lw[c * 4 + pr] * bilinear(T + (size_t)(c * 3 + pr) * D * D, D, D, D,
                                                           xbar[AX_A[pr]], xbar[AX_B[pr]]);
                    yb[c * plane + o] = Phi;
                }
            }
            free(fs);
        }
        free(T);
    }
    return 0;
}

/* ---- 3D LUT (Eq. 3) and its best decomposition into 2D LUTs (Eq. 4) ----
 * lut3d: [D][D][D] per output channel, axes (r, g, b); trilinear lookup with
 * the cell rule of Supp. Eq. 13 on each axis. */
static double trilinear(const double *t, int D, double pr, double pg, double pb)
{
    int i, j, k;
    double a, b, c;
    cell(pr, D, &i, &a);
    cell(pg, D, &j, &b);
    cell(pb, D, &k, &c);
    double v = 0.0;
    for (int di = 0; di < 2; ++di)
        for (int dj = 0; dj < 2; ++dj)
            for (int dk = 0; dk < 2; ++dk) {
                double w = (di ? a : 1.0 - a) * (dj ? b : 1.0 - b) * (dk ? c : 1.0 - c);
                v += w * t[((size_t)(i + di) * D + (j + dj)) * D + (k + dk)];
            }
    return v;
}

/* y = I_tri(clamp(x), t^c_rgb) for every channel c.  lut3d: [B][3 c][D][D][D]. */
int oracle_lut3d_apply(int D, int B, int H, int W, const double *lut3d, const double *x, double *y)
{
    size_t plane = (size_t)H * W, nl = (size_t)D * D * D;
    for (int b = 0; b < B; ++b) {
        const double *xb = x + (size_t)b * 3 * plane;
        double *yb = y + (size_t)b * 3 * plane;
#pragma omp parallel for schedule(static)
        for (int row = 0; row < H; ++row)
            for (int col = 0; col < W; ++col) {
                size_t o = (size_t)row * W + col;
                double p[3];
                for (int c = 0; c < 3; ++c) p[c] = clamp01(xb[c * plane + o]);
                for (int c = 0; c < 3; ++c)
                    yb[c * plane + o] = trilinear(lut3d + ((size_t)b * 3 + c) * nl, D, p[0], p[1], p[2]);
            }
    }
    return 0;
}

/* Least-squares fit, over the D^3 vertices, of one 3D table t[i][j][k] by a
 * sum of 2D tables A[i][j] + Bt[i][k] + C[j][k] (the hypothesis of Eq. 4 with
 * the weights and bias absorbed).  The sums of functions of two indices form
 * a linear space whose orthogonal projection is the second-order ANOVA
 * expansion:
 *   fit = m_ij. + m_i.k + m_.jk - m_i.. - m_.j. - m_..k + m_...
 * (m: means over the dotted indices); it is split as A = m_ij.,
 * Bt = m_i.k - m_i.., C = m_.jk - m_.j. - m_..k + m_... .  Returns the RMS
 * of the residual (the three-way interaction). */
double oracle_lut3d_fit2d(int D, const double *t, double *A, double *Bt, double *C)
{
    size_t n2 = (size_t)D * D;
    double *mij = (double *)calloc(n2, sizeof(double)), *mik = (double *)calloc(n2, sizeof(double)),
           *mjk = (double *)calloc(n2, sizeof(double)), *mi = (double *)calloc(D, sizeof(double)),
           *mj = (double *)calloc(D, sizeof(double)), *mk = (double *)calloc(D, sizeof(double));
    double m = 0.0;
    for (int i = 0; i < D; ++i)
        for (int j = 0; j < D; ++j)
            for (int k = 0; k < D; ++k) {
                double v = t[((size_t)i * D + j) * D + k];
                mij[i * D + j] += v;
                mik[i * D + k] += v;
                mjk[j * D + k] += v;
                mi[i] += v;
                mj[j] += v;
                mk[k] += v;
                m += v;
            }
    for (size_t e = 0; e < n2; ++e) {
        mij[e] /= D;
        mik[e] /= D;
        mjk[e] /= D;
    }
    for (int i = 0; i < D; ++i) {
        mi[i] /= (double)D * D;
        mj[i] /= (double)D * D;
        mk[i] /= (double)D * D;
    }
    m /= (double)D * D * D;
    for (int a = 0; a < D; ++a)
        for (int b = 0; b < D; ++b) {
            A[a * D + b] = mij[a * D + b];
            Bt[a * D + b] = mik[a * D + b] - mi[a];
            C[a * D + b] = mjk[a * D + b] - mj[a] - mk[b] + m;
        }
    double ss = 0.0;
    for (int i = 0; i < D; ++i)
        for (int j = 0; j < D; ++j)
            for (int k = 0; k < D; ++k) {
                double r = t[((size_t)i * D + j) * D + k] - A[i * D + j] - Bt[i * D + k] - C[j * D + k];
                ss += r * r;
            }
    free(mij);
    free(mik);
    free(mjk);
    free(mi);
    free(mj);
    free(mk);
    return sqrt(ss / ((double)D * D * D));
}

/* Forward of the LUT part only through the separable form
 * I_bi(U S V^T; a, b) = sum_r s_r I_1d(u_r; a) I_1d(v_r; b),
 * never materialising T.  Independent second route used to cross-check the
 * materialised route; grids are evaluated as in oracle_forward. */
static double lerp1d(const double *col, int stride, int D, double p)
{
    int i;
    double d;
    cell(p, D, &i, &d);
    return (1.0 - d) * col[i * stride] + d * col[(i + 1) * stride];
}

int oracle_forward_separable(const int *dims, int B, int H, int W,
                             const double *U, const double *S, const double *V,
                             const double *lut_w, const double *g_xy, const double *g_xc,
                             const double *g_yc, const double *grid_w, const double *x,
                             double *y)
{
    size_t plane = (size_t)H * W;
    for (int b = 0; b < B; ++b) {
        img_params q = params_of(dims, b, U, S, V, lut_w, g_xy, g_xc, g_yc, grid_w);
        int D = q.D, R = q.R;
        const double *xb = x + (size_t)b * 3 * plane;
        double *yb = y + (size_t)b * 3 * plane;
        for (size_t o = 0; o < plane; ++o) {
            int row = (int)(o / W), col = (int)(o % W);
            double p[3];
            for (int c = 0; c < 3; ++c) p[c] = clamp01(xb[c * plane + o]);
            double xs = coord(col, W), ys = coord(row, H);
            for (int c = 0; c < 3; ++c) {
                double Phi = q.lw[c * 4 + 3];
                for (int pr = 0; pr < 3; ++pr) {
                    const double *Ucp = q.U + (size_t)(c * 3 + pr) * D * R;
                    const double *Vcp = q.V + (size_t)(c * 3 + pr) * D * R;
                    double phi = 0.0;
                    for (int r = 0; r < R; ++r)
                        phi += q.S[(c * 3 + pr) * R + r] * lerp1d(Ucp + r, R, D, p[AX_A[pr]])
                               * lerp1d(Vcp + r, R, D, p[AX_B[pr]]);
                    Phi += q.lw[c * 4 + pr] * phi;
                }
                yb[c * plane + o] = Phi;
            }
            for (int k = 0; k < q.K; ++k) {
                int c = k % 3;
                const double *w = q.gw + k * 4;
                double v = w[0] * bilinear(q.gxy + (size_t)k * q.Dsy * q.Dsx, q.Dsx, q.Dsy, q.Dsx, ys, xs)
                         + w[1] * bilinear(q.gxc + (size_t)k * q.Dsx * q.Dsc, q.Dsc, q.Dsx, q.Dsc, xs, p[c])
                         + w[2] * bilinear(q.gyc + (size_t)k * q.Dsy * q.Dsc, q.Dsc, q.Dsy, q.Dsc, ys, p[c])
                         + w[3];
                yb[c * plane + o] += v;
            }
        }
    }
    return 0;
}

/* ---- adjoint ---- */

/* Scatter g * bilinear weights of (pa, pb) into tab; return the bilinear value
 * of val at (pa, pb) and its partial derivatives w.r.t. pa and pb. */
static double bilinear_adj(const double *val, double *grad, int ld, int Da, int Db,
                           double pa, double pb, double g, double *dpa, double *dpb)
{
    int i, j;
    double da, db;
    cell(pa, Da, &i, &da);
    cell(pb, Db, &j, &db);
    size_t o00 = (size_t)i * ld + j, o10 = (size_t)(i + 1) * ld + j;
    size_t o01 = o00 + 1, o11 = o10 + 1;
    double v00 = val[o00], v10 = val[o10], v01 = val[o01], v11 = val[o11];
    if (grad) {
        grad[o00] += g * (1.0 - da) * (1.0 - db);
        grad[o10] += g * da * (1.0 - db);
        grad[o01] += g * (1.0 - da) * db;
        grad[o11] += g * da * db;
    }
    if (dpa) *dpa = (double)(Da - 1) * ((1.0 - db) * (v10 - v00) + db * (v11 - v01));
    if (dpb) *dpb = (double)(Db - 1) * ((1.0 - da) * (v01 - v00) + da * (v11 - v10));
    return (1.0 - da) * (1.0 - db) * v00 + da * (1.0 - db) * v10
         + (1.0 - da) * db * v01 + da * db * v11;
}

/* Adjoint of oracle_forward under upstream gradient dy.  Every output
 * pointer may be NULL (not wanted); wanted outputs are overwritten.
 * dx gets d/dx of clamp(x) (1 inside [0,1], 0 outside) times dL/dp. */
int oracle_backward(const int *dims, int B, int H, int W,
                    const double *U, const double *S, const double *V, const double *lut_w,
                    const double *g_xy, const double *g_xc, const double *g_yc,
                    const double *grid_w, const double *x, const double *dy, double *dx,
                    double *dU, double *dS, double *dV, double *dlut_w, double *dg_xy,
                    double *dg_xc, double *dg_yc, double *dgrid_w)
{
    int D = dims[O_DT], R = dims[O_R], K = dims[O_K];
    int Dsx = dims[O_DSX], Dsy = dims[O_DSY], Dsc = dims[O_DSC];
    size_t plane = (size_t)H * W;
    for (int b = 0; b < B; ++b) {
        img_params q = params_of(dims, b, U, S, V, lut_w, g_xy, g_xc, g_yc, grid_w);
        double *T = build_tables(&q);
        double *dT = (double *)calloc((size_t)9 * D * D, sizeof(double));
        double dlw[12] = {0};
        size_t nxy = (size_t)K * Dsy * Dsx, nxc = (size_t)K * Dsx * Dsc, nyc = (size_t)K * Dsy * Dsc;
        double *gxy = (double *)calloc(nxy + 1, sizeof(double));
        double *gxc = (double *)calloc(nxc + 1, sizeof(double));
        double *gyc = (double *)calloc(nyc + 1, sizeof(double));
        double *gw = (double *)calloc((size_t)K * 4 + 1, sizeof(double));
        const double *xb = x + (size_t)b * 3 * plane;
        const double *gb = dy + (size_t)b * 3 * plane;
        for (size_t o = 0; o < plane; ++o) {
            int row = (int)(o / W), col = (int)(o % W);
            double p[3], g[3], dp[3] = {0, 0, 0};
            for (int c = 0; c < 3; ++c) {
                p[c] = clamp01(xb[c * plane + o]);
                g[c] = gb[c * plane + o];
            }
            double xs = coord(col, W), ys = coord(row, H);
            for (int c = 0; c < 3; ++c) {
                for (int pr = 0; pr < 3; ++pr) {
                    double w = q.lw[c * 4 + pr];
                    double da_, db_;
                    size_t off = (size_t)(c * 3 + pr) * D * D;
                    double phi = bilinear_adj(T + off, dT + off, D, D, D, p[AX_A[pr]], p[AX_B[pr]],
                                              g[c] * w, &da_, &db_);
                    dlw[c * 4 + pr] += g[c] * phi;
                    dp[AX_A[pr]] += g[c] * w * da_;
                    dp[AX_B[pr]] += g[c] * w * db_;
                }
                dlw[c * 4 + 3] += g[c];
            }
            for (int k = 0; k < K; ++k) {
                int c = k % 3;
                const double *w = q.gw + k * 4;
                double dpc1, dpc2;
                double psi_xy = bilinear_adj(q.gxy + (size_t)k * Dsy * Dsx, gxy + (size_t)k * Dsy * Dsx,
                                             Dsx, Dsy, Dsx, ys, xs, g[c] * w[0], NULL, NULL);
                double psi_xc = bilinear_adj(q.gxc + (size_t)k * Dsx * Dsc, gxc + (size_t)k * Dsx * Dsc,
                                             Dsc, Dsx, Dsc, xs, p[c], g[c] * w[1], NULL, &dpc1);
                double psi_yc = bilinear_adj(q.gyc + (size_t)k * Dsy * Dsc, gyc + (size_t)k * Dsy * Dsc,
                                             Dsc, Dsy, Dsc, ys, p[c], g[c] * w[2], NULL, &dpc2);
                gw[k * 4 + 0] += g[c] * psi_xy;
                gw[k * 4 + 1] += g[c] * psi_xc;
                gw[k * 4 + 2] += g[c] * psi_yc;
                gw[k * 4 + 3] += g[c];
                dp[c] += g[c] * (w[1] * dpc1 + w[2] * dpc2);
            }
            if (dx) {
                double *dxb = dx + (size_t)b * 3 * plane;
                for (int c = 0; c < 3; ++c) {
                    double xv = xb[c * plane + o];
                    dxb[c * plane + o] = (xv >= 0.0 && xv <= 1.0) ? dp[c] : 0.0;
                }
            }
        }
        /* chain rule through T = U diag(S) V^T */
        for (int cp = 0; cp < 9; ++cp) {
            const double *Ui = q.U + (size_t)cp * D * R, *Vi = q.V + (size_t)cp * D * R;
            const double *Si = q.S + cp * R;
            const double *G = dT + (size_t)cp * D * D;
            for (int r = 0; r < R; ++r) {
                if (dU)
                    for (int i = 0; i < D; ++i) {
                        double a = 0.0;
                        for (int j = 0; j < D; ++j) a += G[i * D + j] * Vi[j * R + r];
                        dU[(size_t)b * 9 * D * R + (size_t)cp * D * R + i * R + r] = a * Si[r];
                    }
                if (dV)
                    for (int j = 0; j < D; ++j) {
                        double a = 0.0;
                        for (int i = 0; i < D; ++i) a += G[i * D + j] * Ui[i * R + r];
                        dV[(size_t)b * 9 * D * R + (size_t)cp * D * R + j * R + r] = a * Si[r];
                    }
                if (dS) {
                    double a = 0.0;
                    for (int i = 0; i < D; ++i)
                        for (int j = 0; j < D; ++j) a += G[i * D + j] * Ui[i * R + r] * Vi[j * R + r];
                    dS[(size_t)b * 9 * R + cp * R + r] = a;
                }
            }
        }
        if (dlut_w) memcpy(dlut_w + (size_t)b * 12, dlw, sizeof dlw);
        if (dg_xy) memcpy(dg_xy + (size_t)b * nxy, gxy, sizeof(double) * nxy);
        if (dg_xc) memcpy(dg_xc + (size_t)b * nxc, gxc, sizeof(double) * nxc);
        if (dg_yc) memcpy(dg_yc + (size_t)b * nyc, gyc, sizeof(double) * nyc);
        if (dgrid_w) memcpy(dgrid_w + (size_t)b * K * 4, gw, sizeof(double) * K * 4);
        free(T); free(dT); free(gxy); free(gxc); free(gyc); free(gw);
    }
    return 0;
}

/* 8-bit input: p = v / 255. */
void oracle_u8_to_unit(const uint8_t *v, double *out, size_t n)
{
    for (size_t i = 0; i < n; ++i) out[i] = (double)v[i] / 255.0;
}

/* 16-bit input (the 16-bit photos of Sec. 4.1): p = v / 65535. */
void oracle_u16_to_unit(const uint16_t *v, double *out, size_t n)
{
    for (size_t i = 0; i < n; ++i) out[i] = (double)v[i] / 65535.0;
}

/* 8-bit output: round-half-even of clamp(Y,0,1)*255, in FP64 like the rest
 * of the oracle.  A result that lies within rounding error of a half-integer
 * code may come out one code apart in a lower-precision implementation; the
 * 1-LSB tolerance of the parity tests covers exactly that. */
void oracle_quantize_u8(const double *y, uint8_t *out, size_t n)
{
    for (size_t i = 0; i < n; ++i) {
        double f = y[i];
        f = f < 0.0 ? 0.0 : (f > 1.0 ? 1.0 : f);
        out[i] = (uint8_t)rint(f * 255.0);
    }
}
