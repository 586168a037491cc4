/*
 * dbmp_oracle.c -- plain, slow FP64 CPU reference of the DiffBMP rasterizer.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the correctness oracle for the CUDA
 * library: only the test suite, the smoke check and the benchmark's CPU-baseline
 * leg may load it.  It shares no code, header, helper or constant generator with
 * the CUDA path, and the CUDA path never calls it.
 *
 * What it computes (DiffBMP, "Differentiable Rendering with Bitmap Primitives"):
 *   Eq. 1   canvas -> normalised primitive coords  [u v] = R(theta) [(x-xi)/s (y-yi)/s]
 *   Eq. 2   normalised -> bitmap coords            U = (u+1)/2 (W-1), V = (v+1)/2 (H-1)
 *   Eqs. S1-S3 (Sec. S1.1) bilinear sample M = w^T p over the four lattice taps
 *   Eq. 3   alpha_i = alpha_max sigmoid(nu_i) M_i
 *   Eqs. 4-5 front-to-back Porter-Duff over: T_k = prod_{j<k}(1-alpha_j),
 *           I = sum_k T_k alpha_k sigmoid(c_k)
 *   Eq. 8   background blend  I = I_FG + T_N b ;  I_alpha = 1 - T_N (Sec. 3.3.2)
 *   Eq. 6, Eq. S4, Eq. S5 (Sec. 3.1.2, Sec. S1.2): exact gradients, written here as a
 *           reverse recursion over the layers of one pixel (no division).
 *   Sec. 3.2 "Structure-aware Initialization" (Tab. S1 window 7, base probability 0.1):
 *           local variance, its normalisation, weighted draws of lattice points and the
 *           initial parameters at them (oracle_local_variance, oracle_structure_init).
 *   Sec. 3.1.1 "Parallelization": every primitive is listed in each tile its padded
 *           bounding box overlaps, in front-to-back (index) order; oracle_bin is that
 *           listing written out as a definition (fp32 bounding-box specification).
 *
 * Readings where the paper is silent (each also listed in the design notes):
 *   - pixel (px,py) sits at canvas coordinate x = px, y = py (integer centres, as the
 *     meshgrid of the naive baseline, Algorithm S3);
 *   - taps outside the bitmap are zero (zero padding, as grid_sample in Algorithm S3);
 *   - index 0 is the front layer;
 *   - the "skip if M < eps" test of Algorithm 1 is read with eps = 0: a layer with
 *     M == 0 has alpha == 0 and changes nothing, so skipping it is exact;
 *   - early termination: a layer k is composited only while T_k >= T_stop
 *     (T_stop = 0 composites every layer);
 *   - a primitive with a non-finite parameter or s == 0 is skipped (no tiles, no
 *     contribution, zero gradient);
 *   - structure-aware initialisation: "lattice points" are the pixel centres; the local
 *     variance is the population variance over the 7 x 7 window clipped to the canvas,
 *     averaged over R, G, B; NLV is its min-max normalisation over the canvas; draws
 *     are with replacement, with weights quantised to multiples of 2^-20 so that the
 *     cumulative weights are exact; the colour draw is on the activated colour
 *     (clamped to [1e-4, 1 - 1e-4], stored as its logit); the random numbers are inputs.
 *
 * Parity pins: the tests check this file against closed forms (identity transform,
 * one and two layer over, occlusion, zero opacity, rotation by pi/2), against
 * torch.nn.functional.grid_sample + autograd in float64 (Algorithm S3), against
 * central finite differences in FP64, against Eq. S5 for b = 0, and the binning
 * against brute-force rectangle intersection and the sum_i tau_i = sum_t d_t identity.
 * The initialisation: brute-force windows (numpy) and the checkerboard closed form for
 * the variance, inverse-CDF hits and the law of large numbers for the draws, and the
 * parameter formulas at the drawn pixels.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_BG_NONE 0
#define ORC_BG_CONST 1
#define ORC_BG_BUFFER 2

/* -------------------------------------------------------------------------- */
/* Per-primitive quantities in FP64                                            */
/* -------------------------------------------------------------------------- */
typedef struct {
    int valid;
    double x, y, s, cs, sn;     /* position, scale, cos(theta), sin(theta) */
    double amax, sig_nu, a;     /* alpha_max, sigmoid(nu), alpha_max*sigmoid(nu) */
    double chat[3];             /* sigmoid(c)                                */
    double xlo, xhi, ylo, yhi;  /* conservative canvas support box           */
    const float *bmp;           /* bitmap P_i, row-major [H][W]              */
} orc_prim;

static double sigmoid(double z) { return 1.0 / (1.0 + exp(-z)); }

static int finite_params(const float *p) {
    for (int j = 0; j < 8; ++j)
        if (!isfinite(p[j])) return 0;
    return p[2] != 0.0f;
}

/* Fill one primitive record.  The support box is the canvas region where any of
 * the four bilinear taps can be non-zero: U in (-1, W) and V in (-1, H), i.e.
 * |u| < 1 + 2/(W-1), |v| < 1 + 2/(H-1), widened by one pixel.  It only skips work
 * whose result is exactly zero; it never changes a value. */
static void make_prim(orc_prim *q, const float *p, int32_t bid, const float *atlas,
                      int32_t Hb, int32_t Wb, double alpha_max) {
    q->valid = finite_params(p);
    q->x = p[0];
    q->y = p[1];
    q->s = p[2];
    double th = p[3];
    q->cs = cos(th);
    q->sn = sin(th);
    q->amax = alpha_max;
    q->sig_nu = sigmoid((double)p[4]);
    q->a = alpha_max * q->sig_nu;
    for (int j = 0; j < 3; ++j) q->chat[j] = sigmoid((double)p[5 + j]);
    q->bmp = atlas + (size_t)bid * (size_t)Hb * (size_t)Wb;
    double eu = 1.0 + 2.0 / (double)(Wb - 1), ev = 1.0 + 2.0 / (double)(Hb - 1);
    double as = fabs(q->s);
    double hx = as * (fabs(q->cs) * eu + fabs(q->sn) * ev) + 1.0;
    double hy = as * (fabs(q->sn) * eu + fabs(q->cs) * ev) + 1.0;
    q->xlo = q->x - hx;
    q->xhi = q->x + hx;
    q->ylo = q->y - hy;
    q->yhi = q->y + hy;
}

/* One bitmap tap with zero padding outside [0,W-1] x [0,H-1]. */
static double tap(const float *P, int32_t Hb, int32_t Wb, long v, long u) {
    if (u < 0 || v < 0 || u >= Wb || v >= Hb) return 0.0;
    return (double)P[(size_t)v * (size_t)Wb + (size_t)u];
}

/* Everything the backward needs about one (pixel, layer) evaluation. */
typedef struct {
    int k;
    double u, v, wu, wv;
    double p00, p01, p10, p11;
    double M, alpha, T;  /* T = transmittance in front of this layer */
} orc_layer;

/* Eq. 1, Eq. 2 and Eqs. S1-S3 at canvas point (x, y). */
static void sample(const orc_prim *q, int32_t Hb, int32_t Wb, double x, double y, orc_layer *L) {
    double dx = x - q->x, dy = y - q->y;
    L->u = (q->cs * dx + q->sn * dy) / q->s;
    L->v = (-q->sn * dx + q->cs * dy) / q->s;
    double U = (L->u + 1.0) / 2.0 * (double)(Wb - 1);
    double V = (L->v + 1.0) / 2.0 * (double)(Hb - 1);
    double u0 = floor(U), v0 = floor(V);
    L->wu = U - u0;
    L->wv = V - v0;
    long iu = (long)u0, iv = (long)v0;
    L->p00 = tap(q->bmp, Hb, Wb, iv, iu);
    L->p01 = tap(q->bmp, Hb, Wb, iv, iu + 1);
    L->p10 = tap(q->bmp, Hb, Wb, iv + 1, iu);
    L->p11 = tap(q->bmp, Hb, Wb, iv + 1, iu + 1);
    L->M = (1.0 - L->wu) * (1.0 - L->wv) * L->p00 + L->wu * (1.0 - L->wv) * L->p01 +
           (1.0 - L->wu) * L->wv * L->p10 + L->wu * L->wv * L->p11;
}

static int in_box(const orc_prim *q, double x, double y) {
    return q->valid && x > q->xlo && x < q->xhi && y > q->ylo && y < q->yhi;
}

/* Walk all layers of one pixel front to back (Eqs. 3-5).  Returns the number of
 * contributing layers written to `Ls` (may be NULL), stores C, T_N, last index and
 * the number of (pixel, primitive) pairs whose bitmap was sampled. */
static int walk_pixel(const orc_prim *P, int32_t N, int32_t Hb, int32_t Wb, double x, double y,
                      double T_stop, orc_layer *Ls, double C[3], double *T_out, int32_t *last,
                      int64_t *pairs) {
    double T = 1.0;
    int n = 0;
    C[0] = C[1] = C[2] = 0.0;
    *last = -1;
    for (int32_t k = 0; k < N; ++k) {
        const orc_prim *q = &P[k];
        if (!in_box(q, x, y)) continue;
        if (T < T_stop) break;
        orc_layer L;
        sample(q, Hb, Wb, x, y, &L);
        ++*pairs;
        if (L.M == 0.0) continue;
        L.k = k;
        L.alpha = q->a * L.M;
        L.T = T;
        for (int j = 0; j < 3; ++j) C[j] += T * L.alpha * q->chat[j];
        T *= (1.0 - L.alpha);
        *last = k;
        if (Ls) Ls[n] = L;
        ++n;
    }
    *T_out = T;
    return n;
}

static double bg_value(int32_t bg_mode, const double *bg_rgb, const float *bg_buf, int j,
                       size_t pix, size_t HW) {
    if (bg_mode == ORC_BG_CONST) return bg_rgb[j];
    if (bg_mode == ORC_BG_BUFFER) return (double)bg_buf[(size_t)j * HW + pix];
    return 0.0;
}

static orc_prim *make_prims(int32_t N, const float *params, const int32_t *bitmap_id,
                            const float *atlas, int32_t Hb, int32_t Wb, double alpha_max) {
    orc_prim *P = (orc_prim *)calloc((size_t)(N > 0 ? N : 1), sizeof(orc_prim));
    for (int32_t k = 0; k < N; ++k)
        make_prim(&P[k], params + 8 * (size_t)k, bitmap_id[k], atlas, Hb, Wb, alpha_max);
    return P;
}

/* -------------------------------------------------------------------------- */
/* Forward: whole canvas, or a list of pixels                                  */
/* -------------------------------------------------------------------------- */

/* Renders the pixels (px[i], py[i]), i < n_pix.  If px == NULL, renders the whole
 * H x W canvas in row-major order (n_pix ignored).  Outputs are indexed like the
 * pixel list: image[j * n + i], T_final[i], n_last[i] (index of the last
 * contributing primitive, -1 if none).  Returns the number of sampled pairs; if
 * `contrib` is not NULL it receives the number of contributing pairs: layers with
 * M > 0 that a pixel composites while its transmittance is still >= T_stop. */
int64_t oracle_render(int32_t H, int32_t W, int32_t N, const float *params,
                      const int32_t *bitmap_id, const float *atlas, int32_t n_bmp, int32_t Hb,
                      int32_t Wb, double alpha_max, int32_t bg_mode, const double *bg_rgb,
                      const float *bg_buf, double T_stop, int64_t n_pix, const int32_t *px,
                      const int32_t *py, double *image, double *T_final, int32_t *n_last,
                      int64_t *contrib) {
    (void)n_bmp;
    orc_prim *P = make_prims(N, params, bitmap_id, atlas, Hb, Wb, alpha_max);
    int64_t n = px ? n_pix : (int64_t)H * (int64_t)W;
    size_t HW = (size_t)H * (size_t)W;
    int64_t pairs = 0, n_contrib = 0;
#pragma omp parallel for schedule(dynamic, 64) reduction(+ : pairs, n_contrib)
    for (int64_t i = 0; i < n; ++i) {
        int32_t x = px ? px[i] : (int32_t)(i % W);
        int32_t y = px ? py[i] : (int32_t)(i / W);
        double C[3], T;
        int32_t last;
        int64_t pr = 0;
        n_contrib += walk_pixel(P, N, Hb, Wb, (double)x, (double)y, T_stop, NULL, C, &T, &last, &pr);
        pairs += pr;
        size_t pix = (size_t)y * (size_t)W + (size_t)x;
        for (int j = 0; j < 3; ++j)
            image[(size_t)j * (size_t)n + (size_t)i] =
                C[j] + T * bg_value(bg_mode, bg_rgb, bg_buf, j, pix, HW);
        T_final[i] = T;
        n_last[i] = last;
    }
    free(P);
    if (contrib) *contrib = n_contrib;
    return pairs;
}

/* -------------------------------------------------------------------------- */
/* Backward                                                                    */
/* -------------------------------------------------------------------------- */

/* Adds the gradient of one pixel into G (N x 8, order x y s theta nu c_r c_g c_b).
 * g[3] = dL/dI at the pixel, gA = dL/dI_alpha, b[3] = background at the pixel.
 * Reverse recursion (exact derivative of Eqs. 3-5 and Eq. 8):
 *   dL/dalpha_k = T_k [ sum_j g_j (chat_kj - R_j) + gA * B ],
 *   with R = colour behind layer k normalised by T_{k+1} (starts at b), updated by
 *   R <- alpha_k chat_k + (1 - alpha_k) R, and B = prod_{m>k} (1 - alpha_m).
 * If `only` >= 0, only that primitive's row is accumulated. */
static void pixel_grad(const orc_prim *P, int32_t Hb, int32_t Wb, const orc_layer *Ls, int n,
                       const double g[3], double gA, const double b[3], double *G, int32_t only) {
    double R[3] = {b[0], b[1], b[2]};
    double B = 1.0;
    double kw = 0.5 * (double)(Wb - 1), kv = 0.5 * (double)(Hb - 1);
    for (int l = n - 1; l >= 0; --l) {
        const orc_layer *L = &Ls[l];
        const orc_prim *q = &P[L->k];
        double dA = gA * B;
        for (int j = 0; j < 3; ++j) dA += g[j] * (q->chat[j] - R[j]);
        dA *= L->T;
        if (only < 0 || only == L->k) {
            double *Gk = G + 8 * (size_t)(only < 0 ? L->k : 0);
            /* Eq. S4: colour logits */
            for (int j = 0; j < 3; ++j)
                Gk[5 + j] += g[j] * L->T * L->alpha * q->chat[j] * (1.0 - q->chat[j]);
            /* Eq. 3: opacity logit */
            Gk[4] += dA * q->amax * L->M * q->sig_nu * (1.0 - q->sig_nu);
            /* Eq. 6: geometry through the bilinear sample and Eqs. 1-2 */
            double dM = dA * q->a;
            double dMdU = (1.0 - L->wv) * (L->p01 - L->p00) + L->wv * (L->p11 - L->p10);
            double dMdV = (1.0 - L->wu) * (L->p10 - L->p00) + L->wu * (L->p11 - L->p01);
            double gu = dM * dMdU * kw, gv = dM * dMdV * kv;
            double s = q->s, cs = q->cs, sn = q->sn;
            Gk[0] += gu * (-cs / s) + gv * (sn / s);
            Gk[1] += gu * (-sn / s) + gv * (-cs / s);
            Gk[2] += gu * (-L->u / s) + gv * (-L->v / s);
            Gk[3] += gu * L->v + gv * (-L->u);
        }
        for (int j = 0; j < 3; ++j) R[j] = L->alpha * q->chat[j] + (1.0 - L->alpha) * R[j];
        B *= (1.0 - L->alpha);
    }
}

/* Gradient of L w.r.t. every primitive's raw parameters, summed over the whole
 * canvas.  dL_dimage: 3 x H x W (planar), dL_dalpha: H x W or NULL.  dparams: N x 8,
 * overwritten.  Same T_stop semantics as the forward. */
void oracle_grad_rows(int32_t H, int32_t W, int32_t N, const float *params,
                      const int32_t *bitmap_id, const float *atlas, int32_t n_bmp, int32_t Hb,
                      int32_t Wb, double alpha_max, int32_t bg_mode, const double *bg_rgb,
                      const float *bg_buf, double T_stop, const double *dL_dimage,
                      const double *dL_dalpha, int32_t y0, int32_t y1, double *dparams);

void oracle_grad(int32_t H, int32_t W, int32_t N, const float *params, const int32_t *bitmap_id,
                 const float *atlas, int32_t n_bmp, int32_t Hb, int32_t Wb, double alpha_max,
                 int32_t bg_mode, const double *bg_rgb, const float *bg_buf, double T_stop,
                 const double *dL_dimage, const double *dL_dalpha, double *dparams) {
    oracle_grad_rows(H, W, N, params, bitmap_id, atlas, n_bmp, Hb, Wb, alpha_max, bg_mode, bg_rgb,
                     bg_buf, T_stop, dL_dimage, dL_dalpha, 0, H, dparams);
}

/* The same sum restricted to the canvas rows y0 <= y < y1 (a bounded sample). */
void oracle_grad_rows(int32_t H, int32_t W, int32_t N, const float *params,
                      const int32_t *bitmap_id, const float *atlas, int32_t n_bmp, int32_t Hb,
                      int32_t Wb, double alpha_max, int32_t bg_mode, const double *bg_rgb,
                      const float *bg_buf, double T_stop, const double *dL_dimage,
                      const double *dL_dalpha, int32_t y0, int32_t y1, double *dparams) {
    (void)n_bmp;
    orc_prim *P = make_prims(N, params, bitmap_id, atlas, Hb, Wb, alpha_max);
    size_t HW = (size_t)H * (size_t)W;
    memset(dparams, 0, sizeof(double) * 8 * (size_t)N);
#pragma omp parallel
    {
        double *Gloc = (double *)calloc(8 * (size_t)(N > 0 ? N : 1), sizeof(double));
        orc_layer *Ls = (orc_layer *)malloc(sizeof(orc_layer) * (size_t)(N > 0 ? N : 1));
#pragma omp for schedule(dynamic, 64)
        for (int64_t i = (int64_t)y0 * W; i < (int64_t)y1 * W; ++i) {
            int32_t x = (int32_t)(i % W), y = (int32_t)(i / W);
            double C[3], T, g[3], b[3];
            int32_t last;
            int64_t pr = 0;
            int n = walk_pixel(P, N, Hb, Wb, x, y, T_stop, Ls, C, &T, &last, &pr);
            for (int j = 0; j < 3; ++j) {
                g[j] = dL_dimage[(size_t)j * HW + (size_t)i];
                b[j] = bg_value(bg_mode, bg_rgb, bg_buf, j, (size_t)i, HW);
            }
            double gA = dL_dalpha ? dL_dalpha[i] : 0.0;
            pixel_grad(P, Hb, Wb, Ls, n, g, gA, b, Gloc, -1);
        }
#pragma omp critical
        for (size_t t = 0; t < 8 * (size_t)N; ++t) dparams[t] += Gloc[t];
        free(Gloc);
        free(Ls);
    }
    free(P);
}

/* The same sum over an explicit set of pixels (px[i], py[i]), i < n (each pixel
 * counted as often as it is listed): the gradient of a loss that only those pixels
 * carry, for every primitive at once.  Used for parity on one dense tile of a
 * canvas too large for oracle_grad.  dL_dimage / dL_dalpha are full-canvas maps. */
void oracle_grad_pixels(int32_t H, int32_t W, int32_t N, const float *params,
                        const int32_t *bitmap_id, const float *atlas, int32_t n_bmp, int32_t Hb,
                        int32_t Wb, double alpha_max, int32_t bg_mode, const double *bg_rgb,
                        const float *bg_buf, double T_stop, const double *dL_dimage,
                        const double *dL_dalpha, int64_t n, const int32_t *px, const int32_t *py,
                        double *dparams) {
    (void)n_bmp;
    orc_prim *P = make_prims(N, params, bitmap_id, atlas, Hb, Wb, alpha_max);
    size_t HW = (size_t)H * (size_t)W;
    memset(dparams, 0, sizeof(double) * 8 * (size_t)N);
#pragma omp parallel
    {
        double *Gloc = (double *)calloc(8 * (size_t)(N > 0 ? N : 1), sizeof(double));
        orc_layer *Ls = (orc_layer *)malloc(sizeof(orc_layer) * (size_t)(N > 0 ? N : 1));
#pragma omp for schedule(dynamic, 16)
        for (int64_t i = 0; i < n; ++i) {
            if (px[i] < 0 || px[i] >= W || py[i] < 0 || py[i] >= H) continue;
            size_t pix = (size_t)py[i] * (size_t)W + (size_t)px[i];
            double C[3], T, g[3], b[3];
            int32_t last;
            int64_t pr = 0;
            int nl = walk_pixel(P, N, Hb, Wb, (double)px[i], (double)py[i], T_stop, Ls, C, &T, &last, &pr);
            for (int j = 0; j < 3; ++j) {
                g[j] = dL_dimage[(size_t)j * HW + pix];
                b[j] = bg_value(bg_mode, bg_rgb, bg_buf, j, pix, HW);
            }
            double gA = dL_dalpha ? dL_dalpha[pix] : 0.0;
            pixel_grad(P, Hb, Wb, Ls, nl, g, gA, b, Gloc, -1);
        }
#pragma omp critical
        for (size_t t = 0; t < 8 * (size_t)N; ++t) dparams[t] += Gloc[t];
        free(Gloc);
        free(Ls);
    }
    free(P);
}

/* Gradient of selected primitives only: for each sel[t], sums the per-pixel
 * contributions over the pixels of its support box (all other pixels contribute
 * exactly zero).  Used for sampled parity on canvases too large for oracle_grad.
 * dparams_sel: n_sel x 8. */
void oracle_grad_selected(int32_t H, int32_t W, int32_t N, const float *params,
                          const int32_t *bitmap_id, const float *atlas, int32_t n_bmp, int32_t Hb,
                          int32_t Wb, double alpha_max, int32_t bg_mode, const double *bg_rgb,
                          const float *bg_buf, double T_stop, const float *dL_dimage,
                          const float *dL_dalpha, int32_t n_sel, const int32_t *sel,
                          double *dparams_sel) {
    (void)n_bmp;
    orc_prim *P = make_prims(N, params, bitmap_id, atlas, Hb, Wb, alpha_max);
    size_t HW = (size_t)H * (size_t)W;
    memset(dparams_sel, 0, sizeof(double) * 8 * (size_t)n_sel);
    for (int32_t t = 0; t < n_sel; ++t) {
        const orc_prim *q = &P[sel[t]];
        if (!q->valid) continue;
        long x0 = (long)floor(q->xlo), x1 = (long)ceil(q->xhi);
        long y0 = (long)floor(q->ylo), y1 = (long)ceil(q->yhi);
        if (x0 < 0) x0 = 0;
        if (y0 < 0) y0 = 0;
        if (x1 > W - 1) x1 = W - 1;
        if (y1 > H - 1) y1 = H - 1;
        if (x1 < x0 || y1 < y0) continue;
        double G[8] = {0};
        long bw = x1 - x0 + 1;
        long nb = bw * (y1 - y0 + 1);
#pragma omp parallel
        {
            double Gl[8] = {0};
            orc_layer *Ls = (orc_layer *)malloc(sizeof(orc_layer) * (size_t)(N > 0 ? N : 1));
#pragma omp for schedule(dynamic, 64)
            for (long i = 0; i < nb; ++i) {
                long x = x0 + i % bw, y = y0 + i / bw;
                if (!in_box(q, (double)x, (double)y)) continue;
                double C[3], T, g[3], b[3];
                int32_t last;
                int64_t pr = 0;
                int n = walk_pixel(P, N, Hb, Wb, (double)x, (double)y, T_stop, Ls, C, &T, &last, &pr);
                size_t pix = (size_t)y * (size_t)W + (size_t)x;
                for (int j = 0; j < 3; ++j) {
                    g[j] = (double)dL_dimage[(size_t)j * HW + pix];
                    b[j] = bg_value(bg_mode, bg_rgb, bg_buf, j, pix, HW);
                }
                double gA = dL_dalpha ? (double)dL_dalpha[pix] : 0.0;
                pixel_grad(P, Hb, Wb, Ls, n, g, gA, b, Gl, sel[t]);
            }
#pragma omp critical
            for (int j = 0; j < 8; ++j) G[j] += Gl[j];
            free(Ls);
        }
        for (int j = 0; j < 8; ++j) dparams_sel[8 * (size_t)t + j] = G[j];
    }
    free(P);
}

/* Eq. S5 as printed (suffix sum S_j and back-product B, no background term), for
 * one pixel: writes dL/dalpha_k of the pixel's contributing layers, front to back,
 * into out[] and their primitive indices into ks[].  Returns the layer count.
 * Used only to pin the reverse recursion above when b = 0. */
int32_t oracle_eq_s5_dalpha(int32_t N, const float *params, const int32_t *bitmap_id,
                            const float *atlas, int32_t Hb, int32_t Wb, double alpha_max, int32_t x,
                            int32_t y, const double g[3], double gA, double *out, int32_t *ks) {
    orc_prim *P = make_prims(N, params, bitmap_id, atlas, Hb, Wb, alpha_max);
    orc_layer *Ls = (orc_layer *)malloc(sizeof(orc_layer) * (size_t)(N > 0 ? N : 1));
    double C[3], T;
    int32_t last;
    int64_t pr = 0;
    int n = walk_pixel(P, N, Hb, Wb, x, y, 0.0, Ls, C, &T, &last, &pr);
    for (int l = 0; l < n; ++l) {
        const orc_prim *q = &P[Ls[l].k];
        double S[3] = {0, 0, 0}, B = 1.0;
        for (int m = l + 1; m < n; ++m) {
            for (int j = 0; j < 3; ++j) S[j] += P[Ls[m].k].chat[j] * Ls[m].alpha * Ls[m].T;
            B *= (1.0 - Ls[m].alpha);
        }
        double d = gA * Ls[l].T * B;
        for (int j = 0; j < 3; ++j) d += g[j] * (Ls[l].T * q->chat[j] - S[j] / (1.0 - Ls[l].alpha));
        out[l] = d;
        ks[l] = Ls[l].k;
    }
    free(Ls);
    free(P);
    return n;
}

/* -------------------------------------------------------------------------- */
/* Binning specification (Sec. 3.1.1 "Parallelization"; Sec. S1.3)             */
/* -------------------------------------------------------------------------- */
/* The tile lists are defined by an fp32 bounding box computed with the steps
 * below, one IEEE single-precision operation at a time (this file is compiled
 * with -ffp-contract=off, so no fused multiply-add).  Its sine and cosine come
 * from Cody-Waite reduction by pi/2 (three-part constant) and the Taylor series
 * of sin and cos to degree 9 / 8 on [-pi/4, pi/4].
 *
 * The box holds the pixels where the primitive's sample M can be non-zero.  With
 * zero padding (Sec. S1.1) M > 0 needs a non-zero tap, so only bitmap coordinates
 * U in (u0 - 1, u1 + 1), V in (v0 - 1, v1 + 1) matter, where [u0, u1] x [v0, v1] are
 * the first and last columns and rows of the bitmap holding a texel > 0 (an all-zero
 * bitmap lists the primitive nowhere).  In the normalised coordinates of Eq. 1 that
 * box has centre (uc, vc) and half-extents (eu, ev); the pixel offsets
 * (dx, dy) = s (cos u - sin v, sin u + cos v) of its image form a rotated box with
 * centre s (cos uc - sin vc, sin uc + cos vc) and axis-aligned half-extents
 * hx = |s| (|cos| eu + |sin| ev), hy = |s| (|sin| eu + |cos| ev).  The margin
 * m = 1 + |s| 2^-19 pixels exceeds the rounding of these steps and of the
 * compositors' transform, so the box contains every pixel with M > 0.  For
 * |theta| > 65536 (outside the reduction's range) the box is centred on (x, y)
 * with hx = hy = |s| (|uc| + eu + |vc| + ev), which holds every rotation.
 *
 * A primitive is listed in tile (tx, ty) iff tx0 <= tx <= tx1 and ty0 <= ty <= ty1
 * with tx0 = floor((cx - hx - m)/T), tx1 = floor((cx + hx + m)/T), cx = x + dx_c
 * (same for y), clipped to the canvas' tiles.  Lists hold primitive indices in
 * increasing order (front to back). */

/* sin and cos of the specification; returns 0 (and 1, 1) for |th| > 65536. */
static int spec_sincos(float th, float *sn, float *cs) {
    if (!(fabsf(th) <= 65536.0f)) { /* outside the reduction's exact range */
        *sn = 1.0f;
        *cs = 1.0f;
        return 0;
    }
    const float two_over_pi = 0.636619772367581343f;
    const float C1 = 1.5703125f;               /* pi/2 split in three parts */
    const float C2 = 4.83751296997070312e-4f;
    const float C3 = 7.54978995489188e-8f;
    float k = rintf(th * two_over_pi);
    float r = th - k * C1;
    r = r - k * C2;
    r = r - k * C3;
    float r2 = r * r;
    float sp = 1.0f / 362880.0f;
    sp = sp * r2 + (-1.0f / 5040.0f);
    sp = sp * r2 + (1.0f / 120.0f);
    sp = sp * r2 + (-1.0f / 6.0f);
    float sr = r + (r * r2) * sp;
    float cp = 1.0f / 40320.0f;
    cp = cp * r2 + (-1.0f / 720.0f);
    cp = cp * r2 + (1.0f / 24.0f);
    cp = cp * r2 + (-0.5f);
    float cr = 1.0f + r2 * cp;
    long q = ((long)k % 4 + 4) % 4; /* quadrant: th = k pi/2 + r */
    if (q == 0) {
        *sn = sr;
        *cs = cr;
    } else if (q == 1) {
        *sn = cr;
        *cs = -sr;
    } else if (q == 2) {
        *sn = -sr;
        *cs = -cr;
    } else {
        *sn = -cr;
        *cs = sr;
    }
    return 1;
}

/* |sin|, |cos| of the specification (bounded by 1 outside the reduction's range). */
static void spec_abs_sincos(float th, float *as, float *ac) {
    float sn, cs;
    spec_sincos(th, &sn, &cs);
    *as = fabsf(sn);
    *ac = fabsf(cs);
}

/* First and last column and row of bitmap b holding a texel > 0: box = {u0, u1, v0,
 * v1}; {W_b, -1, H_b, -1} for an all-zero bitmap. */
static void spec_nonzero_box(const float *atlas, int32_t b, int32_t Hb, int32_t Wb, int32_t box[4]) {
    box[0] = Wb;
    box[1] = -1;
    box[2] = Hb;
    box[3] = -1;
    const float *P = atlas + (size_t)b * Hb * Wb;
    for (int32_t v = 0; v < Hb; ++v)
        for (int32_t u = 0; u < Wb; ++u)
            if (P[(size_t)v * Wb + u] > 0.0f) {
                if (u < box[0]) box[0] = u;
                if (u > box[1]) box[1] = u;
                if (v < box[2]) box[2] = v;
                if (v > box[3]) box[3] = v;
            }
}

/* Tile rectangle of one primitive whose bitmap's non-zero box is `box`; returns 0
 * if it touches no tile. */
static int spec_rect(const float *p, const int32_t box[4], int32_t Hb, int32_t Wb, int32_t tile,
                     int32_t ntx, int32_t nty, int32_t r[4]) {
    for (int j = 0; j < 8; ++j)
        if (!isfinite(p[j])) return 0;
    if (p[2] == 0.0f) return 0;
    if (box[0] > box[1]) return 0; /* all-zero bitmap */
    float kw = (float)(Wb - 1) * 0.5f, kv = (float)(Hb - 1) * 0.5f;
    /* centre and half-extent of (u0 - 1, u1 + 1) in texels from the bitmap centre (exact) */
    float cu = ((float)(box[0] + box[1]) - (float)(Wb - 1)) * 0.5f;
    float hu = (float)(box[1] - box[0] + 2) * 0.5f;
    float cv = ((float)(box[2] + box[3]) - (float)(Hb - 1)) * 0.5f;
    float hv = (float)(box[3] - box[2] + 2) * 0.5f;
    float uc = cu / kw, eu = hu / kw, vc = cv / kv, ev = hv / kv;
    float sn, cs;
    float s = p[2], as = fabsf(p[2]);
    float dxc, dyc, hx, hy;
    if (spec_sincos(p[3], &sn, &cs)) {
        dxc = s * (cs * uc - sn * vc);
        dyc = s * (sn * uc + cs * vc);
        hx = as * (fabsf(cs) * eu + fabsf(sn) * ev);
        hy = as * (fabsf(sn) * eu + fabsf(cs) * ev);
    } else {
        dxc = 0.0f;
        dyc = 0.0f;
        hx = as * (((fabsf(uc) + eu) + fabsf(vc)) + ev);
        hy = hx;
    }
    float m = 1.0f + as * 1.9073486328125e-06f; /* 2^-19 */
    float cx = p[0] + dxc, cy = p[1] + dyc;
    float inv_t = 1.0f / (float)tile;
    float fx0 = floorf(((cx - hx) - m) * inv_t);
    float fx1 = floorf(((cx + hx) + m) * inv_t);
    float fy0 = floorf(((cy - hy) - m) * inv_t);
    float fy1 = floorf(((cy + hy) + m) * inv_t);
    if (!(fx1 >= 0.0f) || !(fy1 >= 0.0f)) return 0;
    if (!(fx0 <= (float)(ntx - 1)) || !(fy0 <= (float)(nty - 1))) return 0;
    r[0] = fx0 < 0.0f ? 0 : (int32_t)fx0;
    r[1] = fy0 < 0.0f ? 0 : (int32_t)fy0;
    r[2] = fx1 > (float)(ntx - 1) ? ntx - 1 : (int32_t)fx1;
    r[3] = fy1 > (float)(nty - 1) ? nty - 1 : (int32_t)fy1;
    return 1;
}

/* Padded screen-space box area of each primitive, (2 hx + 2)(2 hy + 2) in FP64, from
 * the fp32 half-extents of the bitmap's whole support with its zero-padding ring
 * (|u| < 1 + 2/(W-1), |v| < 1 + 2/(H-1)) rotated by theta and scaled by |s|: the
 * footprint A_i of the scaling analysis (Sec. S4), whatever the bitmap holds; -1 for
 * a primitive the binning skips as invalid. */
void oracle_bin_footprint(int32_t N, const float *params, int32_t Hb, int32_t Wb, double *area) {
    for (int32_t i = 0; i < N; ++i) {
        const float *p = params + 8 * (size_t)i;
        int ok = p[2] != 0.0f;
        for (int j = 0; j < 8; ++j)
            if (!isfinite(p[j])) ok = 0;
        if (!ok) {
            area[i] = -1.0;
            continue;
        }
        float eu = 1.0f + 2.0f / (float)(Wb - 1);
        float ev = 1.0f + 2.0f / (float)(Hb - 1);
        float as, ac;
        spec_abs_sincos(p[3], &as, &ac);
        float s = fabsf(p[2]);
        float hx = s * (ac * eu + as * ev);
        float hy = s * (as * eu + ac * ev);
        area[i] = (2.0 * (double)hx + 2.0) * (2.0 * (double)hy + 2.0);
    }
}

/* Per-primitive tile rectangles: rects[4*i] = {tx0, ty0, tx1, ty1} or {0,0,-1,-1}
 * when the primitive touches no tile; tau[i] = number of tiles.  A primitive whose
 * bitmap id is outside [0, n_bmp) touches no tile. */
void oracle_bin_rects(int32_t H, int32_t W, int32_t tile, int32_t N, const float *params,
                      const int32_t *bitmap_id, const float *atlas, int32_t n_bmp, int32_t Hb,
                      int32_t Wb, int32_t *rects, int64_t *tau) {
    int32_t ntx = (W + tile - 1) / tile, nty = (H + tile - 1) / tile;
    int32_t *boxes = (int32_t *)malloc(sizeof(int32_t) * 4 * (size_t)(n_bmp > 0 ? n_bmp : 1));
    for (int32_t b = 0; b < n_bmp; ++b) spec_nonzero_box(atlas, b, Hb, Wb, boxes + 4 * (size_t)b);
    for (int32_t i = 0; i < N; ++i) {
        int32_t r[4];
        int32_t b = bitmap_id[i];
        if (b >= 0 && b < n_bmp &&
            spec_rect(params + 8 * (size_t)i, boxes + 4 * (size_t)b, Hb, Wb, tile, ntx, nty, r)) {
            memcpy(rects + 4 * (size_t)i, r, sizeof r);
            tau[i] = (int64_t)(r[2] - r[0] + 1) * (int64_t)(r[3] - r[1] + 1);
        } else {
            rects[4 * (size_t)i + 0] = 0;
            rects[4 * (size_t)i + 1] = 0;
            rects[4 * (size_t)i + 2] = -1;
            rects[4 * (size_t)i + 3] = -1;
            tau[i] = 0;
        }
    }
    free(boxes);
}

/* The non-zero box of each bitmap (testing aid): boxes[4*b] = {u0, u1, v0, v1}. */
void oracle_nonzero_boxes(const float *atlas, int32_t n_bmp, int32_t Hb, int32_t Wb, int32_t *boxes) {
    for (int32_t b = 0; b < n_bmp; ++b) spec_nonzero_box(atlas, b, Hb, Wb, boxes + 4 * (size_t)b);
}

/* The tile lists as a definition: for every tile t (row-major), every primitive
 * whose rectangle contains t, in increasing index order.  Writes the list
 * boundaries (offsets[t] .. offsets[t+1]) and, if `list` is not NULL and K fits
 * in `cap`, the concatenated lists.  Returns K = sum_t d_t. */
int64_t oracle_bin(int32_t H, int32_t W, int32_t tile, int32_t N, const float *params,
                   const int32_t *bitmap_id, const float *atlas, int32_t n_bmp, int32_t Hb, int32_t Wb,
                   int64_t *offsets, int32_t *list, int64_t cap) {
    int32_t ntx = (W + tile - 1) / tile, nty = (H + tile - 1) / tile;
    int32_t *rects = (int32_t *)malloc(sizeof(int32_t) * 4 * (size_t)(N > 0 ? N : 1));
    int64_t *tau = (int64_t *)malloc(sizeof(int64_t) * (size_t)(N > 0 ? N : 1));
    oracle_bin_rects(H, W, tile, N, params, bitmap_id, atlas, n_bmp, Hb, Wb, rects, tau);
    int64_t K = 0;
    for (int32_t ty = 0; ty < nty; ++ty)
        for (int32_t tx = 0; tx < ntx; ++tx) {
            offsets[(size_t)ty * ntx + tx] = K;
            for (int32_t i = 0; i < N; ++i) {
                const int32_t *r = rects + 4 * (size_t)i;
                if (tx >= r[0] && tx <= r[2] && ty >= r[1] && ty <= r[3]) {
                    if (list && K < cap) list[K] = i;
                    ++K;
                }
            }
        }
    offsets[(size_t)ntx * nty] = K;
    free(rects);
    free(tau);
    return K;
}

/* -------------------------------------------------------------------------- */
/* Structure-aware initialisation (Sec. 3.2, "Structure-aware Initialization";  */
/* Tab. S1: variance window 7, base probability 0.1, colour noise std 0.02)    */
/* -------------------------------------------------------------------------- */
/* LV(p): for each channel, the population variance of the image over the 7 x 7
 * window centred on p (clipped to the canvas), averaged over the three channels.
 * The sums run over the window in row-major order, mean first, then the squared
 * deviations. */
void oracle_local_variance(int32_t H, int32_t W, const float *image, double *lv) {
    const size_t HW = (size_t)H * W;
    for (int32_t y = 0; y < H; ++y)
        for (int32_t x = 0; x < W; ++x) {
            const int32_t y0 = y - 3 < 0 ? 0 : y - 3, y1 = y + 3 > H - 1 ? H - 1 : y + 3;
            const int32_t x0 = x - 3 < 0 ? 0 : x - 3, x1 = x + 3 > W - 1 ? W - 1 : x + 3;
            const double n = (double)((y1 - y0 + 1) * (x1 - x0 + 1));
            double acc = 0.0;
            for (int c = 0; c < 3; ++c) {
                const float *P = image + (size_t)c * HW;
                double sum = 0.0;
                for (int32_t yy = y0; yy <= y1; ++yy)
                    for (int32_t xx = x0; xx <= x1; ++xx) sum += (double)P[(size_t)yy * W + xx];
                const double mean = sum / n;
                double ss = 0.0;
                for (int32_t yy = y0; yy <= y1; ++yy)
                    for (int32_t xx = x0; xx <= x1; ++xx) {
                        const double d = (double)P[(size_t)yy * W + xx] - mean;
                        ss += d * d;
                    }
                acc += ss / n;
            }
            lv[(size_t)y * W + x] = acc / 3.0;
        }
}

/* The initialisation itself.  NLV = (LV - min LV) / (max LV - min LV) (0 where the
 * variance is constant over the canvas).  Pixel p is drawn with probability
 * proportional to w(p) = 0.1 + 0.9 NLV(p), quantised to q(p) = floor(w(p) 2^20) so
 * that cumulative weights are exact integers: primitive i takes the pixel p with
 * Q(p) <= floor(u_pos[i] Q_total) < Q(p) + q(p), Q the exclusive prefix sum of q
 * (draws with replacement).  Its parameters: (x, y) = (px, py), the pixel centre;
 * s = s_max - (s_max - s_min) NLV(p); theta = 2 pi u_theta[i]; nu fixed; colour
 * channel j: c_hat = I_j(p) + sigma_c n_color[3i+j] clamped to [1e-4, 1 - 1e-4],
 * stored as the logit.  params_out is [N][8] FP64; nlv_out [H][W] and pix_out [N]
 * may be NULL.  mask (nullable, [H][W]): the spatially constrained variant (Sec.
 * 3.3.2, Sec. S3 "Re-initialization Mechanism") draws only pixels with mask > 0;
 * with an empty mask nothing is drawn (params_out untouched).  Returns Q_total. */
int64_t oracle_structure_init(int32_t H, int32_t W, const float *image, const float *mask, int32_t N,
                              const double *u_pos, const double *u_theta, const double *n_color, double s_min,
                              double s_max, double sigma_c, double nu, double *params_out, double *nlv_out,
                              int32_t *pix_out) {
    const size_t HW = (size_t)H * W;
    double *lv = (double *)malloc(sizeof(double) * HW);
    int64_t *Q = (int64_t *)malloc(sizeof(int64_t) * (HW + 1));
    oracle_local_variance(H, W, image, lv);
    double mn = lv[0], mx = lv[0];
    for (size_t p = 1; p < HW; ++p) {
        if (lv[p] < mn) mn = lv[p];
        if (lv[p] > mx) mx = lv[p];
    }
    Q[0] = 0;
    for (size_t p = 0; p < HW; ++p) {
        lv[p] = mx > mn ? (lv[p] - mn) / (mx - mn) : 0.0; /* NLV */
        const double w = 0.1 + 0.9 * lv[p];
        Q[p + 1] = Q[p] + (mask && !(mask[p] > 0.0f) ? 0 : (int64_t)floor(w * 1048576.0));
    }
    const int64_t total = Q[HW];
    if (total == 0) N = 0; /* an empty mask draws nothing */
    const double two_pi = 6.283185307179586476925286766559;
    for (int32_t i = 0; i < N; ++i) {
        const int64_t t = (int64_t)floor(u_pos[i] * (double)total);
        size_t lo = 0, hi = HW - 1; /* largest p with Q[p] <= t */
        while (lo < hi) {
            const size_t mid = (lo + hi + 1) / 2;
            if (Q[mid] <= t) lo = mid; else hi = mid - 1;
        }
        const size_t p = lo;
        double *o = params_out + 8 * (size_t)i;
        o[0] = (double)(p % (size_t)W);
        o[1] = (double)(p / (size_t)W);
        o[2] = s_max - (s_max - s_min) * lv[p];
        o[3] = two_pi * u_theta[i];
        o[4] = nu;
        for (int j = 0; j < 3; ++j) {
            double c = (double)image[(size_t)j * HW + p] + sigma_c * n_color[3 * (size_t)i + j];
            c = c < 1e-4 ? 1e-4 : (c > 1.0 - 1e-4 ? 1.0 - 1e-4 : c);
            o[5 + j] = log(c / (1.0 - c));
        }
        if (pix_out) pix_out[i] = (int32_t)p;
    }
    if (nlv_out) memcpy(nlv_out, lv, sizeof(double) * HW);
    free(lv);
    free(Q);
    return total;
}

/* The spec's |sin|, |cos| (exported so the tests can bound its error). */
void oracle_spec_abs_sincos(float th, float *as, float *ac) { spec_abs_sincos(th, as, ac); }
int oracle_spec_sincos(float th, float *sn, float *cs) { return spec_sincos(th, sn, cs); }

int32_t oracle_num_threads(void) {
#ifdef _OPENMP
    return (int32_t)omp_get_max_threads();
#else
    return 1;
#endif
}

/* Threads of the calling thread's later parallel regions (n >= 1); for timing the
 * oracle on one core and on all of them.  Changes no result. */
void oracle_set_num_threads(int32_t n) {
#ifdef _OPENMP
    if (n >= 1) omp_set_num_threads((int)n);
#else
    (void)n;
#endif
}
