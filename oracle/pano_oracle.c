/*
 * pano_oracle.c -- plain FP64 CPU oracle for the asymmetric bidirectional
 * optical-flow blend of two overlap strips (Meng & Liu, "High-quality Panorama
 * Stitching based on Asymmetric Bidirectional Optical Flow", Section III-C).
 *
 * TEST INFRASTRUCTURE ONLY. This file is the slow, obviously correct statement
 * of what the GPU path computes. Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg may load it. It shares no code, header, table or
 * constant with the CUDA library, and the CUDA library never calls it.
 *
 * Every function follows one passage of the paper; where the paper is silent
 * (it gives no Lucas-Kanade parameters, no pyramid kernel, no definition of
 * FlowMag and no values for kSoftmaxSharpness / kFlowMagCoef) the reading used
 * is stated at the function. Conventions used throughout:
 *   - images are row-major, row y (the paper's i), column x (the paper's j);
 *   - a flow field is (h, w, 2) with [..., 0] the column offset and [..., 1]
 *     the row offset, in pixels of the grid it lives on;
 *   - FlowAtoB lives on A's grid and satisfies A(p) ~ B(p + FlowAtoB(p))
 *     (Section III-C-1: "optical flow of OverlappedR relative to OverlappedL"
 *     is FlowRtoL);
 *   - every border is replicate (clamp-to-edge).
 *
 * Parity status: all functions are pinned by the CPU tests (closed forms,
 * library special cases and brute force). Not pinned: the accuracy of the
 * chosen Lucas-Kanade defaults against the authors' own tuned parameters,
 * which the paper does not publish.
 *
 * Loops over output rows carry "omp parallel for": every output pixel is
 * computed independently from read-only inputs, so the result does not depend
 * on the thread count.
 */
#include <math.h>
#include <stddef.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define PIX(a, w, y, x) ((a)[(size_t)(y) * (size_t)(w) + (size_t)(x)])

static int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

int oracle_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void oracle_set_num_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* ---------------------------------------------------------------------------
 * Unit scaling. 8-bit samples are mapped to [0, 1] by v / 255 so that every
 * later constant (the Tikhonov term of the flow solve) is in intensity units
 * independent of the storage type. (Reading: the paper works on photos and
 * states no intensity scale.)
 * ------------------------------------------------------------------------- */
void oracle_to_unit_u8(const unsigned char* in, long n, double* out)
{
    for (long i = 0; i < n; ++i) out[i] = (double)in[i] / 255.0;
}

/* ---------------------------------------------------------------------------
 * Luminance for the flow estimate. The paper computes one flow per image pair
 * (Section III-C-1) but does not say which channel; this oracle uses the
 * ITU-R BT.601 luma Y = 0.299 R + 0.587 G + 0.114 B. One channel: identity.
 * img: (h, w, c) interleaved, c in {1, 3}.  Y: (h, w).
 * ------------------------------------------------------------------------- */
void oracle_luma(const double* img, int h, int w, int c, double* Y)
{
    long n = (long)h * w;
    if (c == 1) {
        memcpy(Y, img, (size_t)n * sizeof(double));
        return;
    }
    for (long i = 0; i < n; ++i)
        Y[i] = 0.299 * img[3 * i + 0] + 0.587 * img[3 * i + 1] + 0.114 * img[3 * i + 2];
}

/* ---------------------------------------------------------------------------
 * One REDUCE step of the Gaussian pyramid used by pyramidal Lucas-Kanade
 * (Section III-C-1, which names the "LK pyramid algorithm" and cites
 * Bruhn/Weickert/Schnoerr [20]). Kernel: the 5-tap binomial
 * [1 4 6 4 1] / 16 of Burt and Adelson, applied along rows (y) and then along
 * columns (x) with replicate borders, keeping the even rows and columns.
 * dst has ceil(h/2) x ceil(w/2) pixels.
 * ------------------------------------------------------------------------- */
void oracle_pyr_down(const double* src, int h, int w, double* dst)
{
    static const double k[5] = {1.0 / 16, 4.0 / 16, 6.0 / 16, 4.0 / 16, 1.0 / 16};
    int hd = (h + 1) / 2, wd = (w + 1) / 2;
    double* tmp = (double*)malloc((size_t)h * w * sizeof(double));
    /* blur along y */
#pragma omp parallel for schedule(static)
    for (int y = 0; y < h; ++y)
        for (int x = 0; x < w; ++x) {
            double s = 0.0;
            for (int t = -2; t <= 2; ++t) s += k[t + 2] * PIX(src, w, clampi(y + t, 0, h - 1), x);
            PIX(tmp, w, y, x) = s;
        }
    /* blur along x at the kept columns, keep the even rows */
#pragma omp parallel for schedule(static)
    for (int yd = 0; yd < hd; ++yd)
        for (int xd = 0; xd < wd; ++xd) {
            int y = 2 * yd, x = 2 * xd;
            double s = 0.0;
            for (int t = -2; t <= 2; ++t) s += k[t + 2] * PIX(tmp, w, y, clampi(x + t, 0, w - 1));
            PIX(dst, wd, yd, xd) = s;
        }
    free(tmp);
}

/* ---------------------------------------------------------------------------
 * Bilinear sample of a single-channel image at real position (x, y), with
 * pixel centres at integer coordinates and each of the four taps clamped to
 * the image (clamp-to-edge). This is the sampler of Code 1 (ColorL = L(Lx, Ly),
 * ColorR = R(Rx, Ry)) and of the warp inside each flow update.
 * stride: distance in doubles between horizontally adjacent samples (the
 * channel count of an interleaved image); the row pitch is w * stride.
 * ------------------------------------------------------------------------- */
static double bilinear_strided(const double* I, int h, int w, int stride, double x, double y)
{
    double x0f = floor(x), y0f = floor(y);
    double fx = x - x0f, fy = y - y0f;
    /* positions beyond any tap range clamp to the same edge pixel; limiting
       them first keeps the float->int conversion defined */
    if (x0f < -2.0) x0f = -2.0;
    if (x0f > (double)w + 1.0) x0f = (double)w + 1.0;
    if (y0f < -2.0) y0f = -2.0;
    if (y0f > (double)h + 1.0) y0f = (double)h + 1.0;
    int x0 = (int)x0f, y0 = (int)y0f;
    int xa = clampi(x0, 0, w - 1), xb = clampi(x0 + 1, 0, w - 1);
    int ya = clampi(y0, 0, h - 1), yb = clampi(y0 + 1, 0, h - 1);
    size_t row = (size_t)w * stride;
    double i00 = I[(size_t)ya * row + (size_t)xa * stride];
    double i10 = I[(size_t)ya * row + (size_t)xb * stride];
    double i01 = I[(size_t)yb * row + (size_t)xa * stride];
    double i11 = I[(size_t)yb * row + (size_t)xb * stride];
    return (1.0 - fy) * ((1.0 - fx) * i00 + fx * i10) + fy * ((1.0 - fx) * i01 + fx * i11);
}

double oracle_bilinear(const double* I, int h, int w, double x, double y)
{
    return bilinear_strided(I, h, w, 1, x, y);
}

/* Vectorised form for tests: out[k] = I(xs[k], ys[k]). */
void oracle_bilinear_many(const double* I, int h, int w, const double* xs, const double* ys,
                          long n, double* out)
{
    for (long k = 0; k < n; ++k) out[k] = bilinear_strided(I, h, w, 1, xs[k], ys[k]);
}

/* ---------------------------------------------------------------------------
 * Flow warp: dst(p) = src(p + s * flow(p)) for every pixel p and channel.
 * Code 1 evaluates exactly this with s = 1 - BlendL for L and s = 1 - BlendR
 * for R; the flow update evaluates it with s = 1. src/dst: (h, w, c).
 * ------------------------------------------------------------------------- */
void oracle_warp(const double* src, int h, int w, int c, const double* flow, double s, double* dst)
{
#pragma omp parallel for schedule(static)
    for (int y = 0; y < h; ++y)
        for (int x = 0; x < w; ++x) {
            size_t p = (size_t)y * w + x;
            double px = x + s * flow[2 * p + 0], py = y + s * flow[2 * p + 1];
            for (int ch = 0; ch < c; ++ch)
                dst[p * c + ch] = bilinear_strided(src + ch, h, w, c, px, py);
        }
}

/* ---------------------------------------------------------------------------
 * Spatial gradient of the template: central differences with replicate
 * borders, Ix = (T(x+1) - T(x-1)) / 2, Iy = (T(y+1) - T(y-1)) / 2.
 * (Reading: the paper states no gradient filter.)
 * ------------------------------------------------------------------------- */
void oracle_gradient(const double* T, int h, int w, double* Ix, double* Iy)
{
    for (int y = 0; y < h; ++y)
        for (int x = 0; x < w; ++x) {
            PIX(Ix, w, y, x) = 0.5 * (PIX(T, w, y, clampi(x + 1, 0, w - 1)) - PIX(T, w, y, clampi(x - 1, 0, w - 1)));
            PIX(Iy, w, y, x) = 0.5 * (PIX(T, w, clampi(y + 1, 0, h - 1), x) - PIX(T, w, clampi(y - 1, 0, h - 1), x));
        }
}

/* ---------------------------------------------------------------------------
 * One dense Lucas-Kanade refinement step at one pyramid level (Section
 * III-C-1 "LK pyramid algorithm"; the local least-squares flow of [20],
 * applied with warping).
 *
 * Template T, target J, flow u on T's grid (so T(p) ~ J(p + u(p))). Every
 * pixel p looks for one flow vector v that is constant over the (2r+1)^2 box
 * W(p) around it (the Lucas-Kanade assumption). The brightness constancy of
 * each box sample q is linearised at that sample's own current flow u(q):
 *     J(q + v) ~ J(q + u(q)) + grad T(q) . (v - u(q)).
 * Minimising
 *     sum_{q in W(p)} (It(q) + grad T(q) . (v - u(q)))^2 + lambda |v - u(p)|^2
 * over v gives the 2x2 system solved below:
 *   1. It(q) = J(q + u(q)) - T(q)                      (bilinear, clamp-to-edge)
 *      s(q)  = grad T(q) . u(q) - It(q)
 *   2. window sums over W(p), clipped to the image (pixels outside the image
 *      are left out, not clamped):
 *        G(p) = sum grad T grad T^T,   m(p) = sum grad T * s
 *   3. (G(p) + lambda I) v = m(p) + lambda u(p), solved with the explicit 2x2
 *      inverse, det = (G11 + lambda)(G22 + lambda) - G12^2;
 *   4. u(p) <- v.
 * All pixels are updated from the same old u. Where u is constant over the
 * box this is the classical Gauss-Newton increment v = u - (G + lambda I)^-1
 * sum grad T It. (Reading: the paper gives neither the LK variant nor its
 * parameters; the increment form with It taken at each sample's own flow is
 * not a stable iteration, this form is.)
 * u: (h, w, 2), updated in place.
 * ------------------------------------------------------------------------- */
void oracle_lk_step(const double* T, const double* J, int h, int w, double* u, int r, double lambda)
{
    size_t n = (size_t)h * w;
    double* Ix = (double*)malloc(n * sizeof(double));
    double* Iy = (double*)malloc(n * sizeof(double));
    double* s = (double*)malloc(n * sizeof(double));
    double* v = (double*)malloc(2 * n * sizeof(double));
    oracle_gradient(T, h, w, Ix, Iy);
#pragma omp parallel for schedule(static)
    for (int y = 0; y < h; ++y)
        for (int x = 0; x < w; ++x) {
            size_t q = (size_t)y * w + x;
            double It = bilinear_strided(J, h, w, 1, x + u[2 * q], y + u[2 * q + 1]) - T[q];
            s[q] = Ix[q] * u[2 * q] + Iy[q] * u[2 * q + 1] - It;
        }
#pragma omp parallel for schedule(static)
    for (int y = 0; y < h; ++y)
        for (int x = 0; x < w; ++x) {
            double g11 = 0, g12 = 0, g22 = 0, m1 = 0, m2 = 0;
            for (int qy = y - r; qy <= y + r; ++qy) {
                if (qy < 0 || qy >= h) continue;
                for (int qx = x - r; qx <= x + r; ++qx) {
                    if (qx < 0 || qx >= w) continue;
                    size_t q = (size_t)qy * w + qx;
                    g11 += Ix[q] * Ix[q];
                    g12 += Ix[q] * Iy[q];
                    g22 += Iy[q] * Iy[q];
                    m1 += Ix[q] * s[q];
                    m2 += Iy[q] * s[q];
                }
            }
            size_t p = (size_t)y * w + x;
            double a11 = g11 + lambda, a22 = g22 + lambda;
            double det = a11 * a22 - g12 * g12;
            double r1 = m1 + lambda * u[2 * p], r2 = m2 + lambda * u[2 * p + 1];
            v[2 * p + 0] = (a22 * r1 - g12 * r2) / det;
            v[2 * p + 1] = (-g12 * r1 + a11 * r2) / det;
        }
    memcpy(u, v, 2 * n * sizeof(double));
    free(Ix); free(Iy); free(s); free(v);
}

/* ---------------------------------------------------------------------------
 * Coarse-to-fine propagation of pyramidal LK: the flow of level l+1
 * (hc x wc) becomes the starting flow of level l (h x w) by bilinear
 * upsampling at (x/2, y/2) -- level l+1 pixel i sits on level l pixel 2i --
 * and doubling, because displacements are measured in pixels of each level.
 * ------------------------------------------------------------------------- */
void oracle_upsample_flow(const double* uc, int hc, int wc, double* uf, int h, int w)
{
    for (int y = 0; y < h; ++y)
        for (int x = 0; x < w; ++x) {
            size_t p = (size_t)y * w + x;
            uf[2 * p + 0] = 2.0 * bilinear_strided(uc + 0, hc, wc, 2, 0.5 * x, 0.5 * y);
            uf[2 * p + 1] = 2.0 * bilinear_strided(uc + 1, hc, wc, 2, 0.5 * x, 0.5 * y);
        }
}

/* Number of pixels of every level of a pyramid with the given base size. */
static void level_sizes(int h, int w, int levels, int* hs, int* ws)
{
    hs[0] = h; ws[0] = w;
    for (int l = 1; l < levels; ++l) { hs[l] = (hs[l - 1] + 1) / 2; ws[l] = (ws[l - 1] + 1) / 2; }
}

/* ---------------------------------------------------------------------------
 * Storage precision of the pyramid levels. Not a step of the paper (it states
 * no precision): a build extension that keeps the levels in a 16-bit format.
 * fmt 0 = exact (no rounding), 1 = bfloat16, 2 = IEEE 754 binary16.
 * A format with p significand bits (the leading one included) and smallest
 * normal exponent emin holds, for |v| in [2^e, 2^(e+1)) with e >= emin, the
 * multiples of 2^(e - p + 1); below 2^emin (subnormals) the multiples of
 * 2^(emin - p + 1). Rounding is to the nearest such value, ties to the even
 * multiple; results beyond the largest finite value become +-infinity.
 *   bfloat16: p = 8, emin = -126, largest (2 - 2^-7) 2^127
 *   binary16: p = 11, emin = -14, largest (2 - 2^-10) 2^15 = 65504
 * ------------------------------------------------------------------------- */
static double round_to_format(double v, int p, int emin, double maxv)
{
    if (v == 0.0 || !isfinite(v)) return v;
    int e;
    frexp(fabs(v), &e);              /* |v| = m 2^e with m in [0.5, 1): leading bit 2^(e-1) */
    int lead = e - 1;
    if (lead < emin) lead = emin;    /* subnormal range: fixed spacing */
    double ulp = ldexp(1.0, lead - (p - 1));
    double r = nearbyint(v / ulp) * ulp;   /* default rounding mode: to nearest, ties to even */
    if (fabs(r) > maxv) return v > 0 ? INFINITY : -INFINITY;
    return r;
}

void oracle_round_storage(double* a, long n, int fmt)
{
    if (fmt == 0) return;
    int p = fmt == 1 ? 8 : 11;
    int emin = fmt == 1 ? -126 : -14;
    double maxv = fmt == 1 ? ldexp(2.0 - ldexp(1.0, -7), 127) : 65504.0;
    for (long i = 0; i < n; ++i) a[i] = round_to_format(a[i], p, emin, maxv);
}

/* Pyramid of a single-channel image: levels planes, level 0 = Y. out holds
   the planes back to back (level 0 first). With a storage format every level
   is rounded as it is stored, and the next REDUCE reads the stored level. */
void oracle_pyramid_stored(const double* Y, int h, int w, int levels, int fmt, double* out)
{
    int hs[32], ws[32];
    level_sizes(h, w, levels, hs, ws);
    memcpy(out, Y, (size_t)h * w * sizeof(double));
    oracle_round_storage(out, (long)h * w, fmt);
    double* prev = out;
    for (int l = 1; l < levels; ++l) {
        double* cur = prev + (size_t)hs[l - 1] * ws[l - 1];
        oracle_pyr_down(prev, hs[l - 1], ws[l - 1], cur);
        oracle_round_storage(cur, (long)hs[l] * ws[l], fmt);
        prev = cur;
    }
}

void oracle_pyramid(const double* Y, int h, int w, int levels, double* out)
{
    oracle_pyramid_stored(Y, h, w, levels, 0, out);
}

/* ---------------------------------------------------------------------------
 * Pyramidal LK in one direction: zero flow at the coarsest level, `iters`
 * refinement steps per level, upsample to the next finer level, repeat.
 * Tpyr / Jpyr: pyramids laid out as oracle_pyramid writes them.
 * u0: (h, w, 2) flow at level 0 on T's grid.
 * ------------------------------------------------------------------------- */
void oracle_flow_dir(const double* Tpyr, const double* Jpyr, int h, int w, int levels,
                     int iters, int r, double lambda, double* u0)
{
    int hs[32], ws[32];
    size_t off[32];
    level_sizes(h, w, levels, hs, ws);
    off[0] = 0;
    for (int l = 1; l < levels; ++l) off[l] = off[l - 1] + (size_t)hs[l - 1] * ws[l - 1];
    double* u = (double*)calloc((size_t)2 * hs[levels - 1] * ws[levels - 1], sizeof(double));
    for (int l = levels - 1; l >= 0; --l) {
        if (l < levels - 1) {
            double* uf = (double*)malloc((size_t)2 * hs[l] * ws[l] * sizeof(double));
            oracle_upsample_flow(u, hs[l + 1], ws[l + 1], uf, hs[l], ws[l]);
            free(u);
            u = uf;
        }
        for (int k = 0; k < iters; ++k)
            oracle_lk_step(Tpyr + off[l], Jpyr + off[l], hs[l], ws[l], u, r, lambda);
    }
    memcpy(u0, u, (size_t)2 * h * w * sizeof(double));
    free(u);
}

/* ---------------------------------------------------------------------------
 * Asymmetric bidirectional flow of a pair (Section III-C-1): FlowLtoR with L
 * as template and R as target, FlowRtoL with the roles exchanged. Both use the
 * same procedure, so the pair differs only through the data ("asymmetric").
 * YL, YR: (h, w) luma. flowLR, flowRL: (h, w, 2).
 * ------------------------------------------------------------------------- */
void oracle_flow_pair_stored(const double* YL, const double* YR, int h, int w, int levels, int iters,
                             int r, double lambda, int fmt, double* flowLR, double* flowRL)
{
    int hs[32], ws[32];
    level_sizes(h, w, levels, hs, ws);
    size_t tot = 0;
    for (int l = 0; l < levels; ++l) tot += (size_t)hs[l] * ws[l];
    double* PL = (double*)malloc(tot * sizeof(double));
    double* PR = (double*)malloc(tot * sizeof(double));
    oracle_pyramid_stored(YL, h, w, levels, fmt, PL);
    oracle_pyramid_stored(YR, h, w, levels, fmt, PR);
    oracle_flow_dir(PL, PR, h, w, levels, iters, r, lambda, flowLR);
    oracle_flow_dir(PR, PL, h, w, levels, iters, r, lambda, flowRL);
    free(PL); free(PR);
}

void oracle_flow_pair(const double* YL, const double* YR, int h, int w, int levels, int iters,
                      int r, double lambda, double* flowLR, double* flowRL)
{
    oracle_flow_pair_stored(YL, YR, h, w, levels, iters, r, lambda, 0, flowLR, flowRL);
}

/* ---------------------------------------------------------------------------
 * Global blending coefficient, Eq. (1), by brute force on a labelled canvas.
 * label: 1 = Area1 (L only), 2 = Area2 (R only), 3 = Area3 (overlap),
 * anything else = neither. Lmin / Rmin are the smallest Euclidean distances
 * between pixel centres from (i, j) to any Area1 / Area2 pixel. Cost is
 * O(N^2): tiny canvases only.
 *   Blend = 0 in Area1, 1 in Area2, Lmin / (Lmin + Rmin) in Area3, 0.5 else.
 * Eq. (1) is undefined when the canvas has no Area1 (or no Area2) pixel; the
 * reading used is its limit as that area moves infinitely far away: no
 * Area1 gives Blend = 1 in Area3, no Area2 gives 0, neither gives 0.5.
 * ------------------------------------------------------------------------- */
void oracle_blend_coeff(const unsigned char* label, int h, int w, double* blend)
{
    for (int i = 0; i < h; ++i)
        for (int j = 0; j < w; ++j) {
            unsigned char a = PIX(label, w, i, j);
            double v;
            if (a == 1) v = 0.0;
            else if (a == 2) v = 1.0;
            else if (a == 3) {
                double lmin = INFINITY, rmin = INFINITY;
                for (int y = 0; y < h; ++y)
                    for (int x = 0; x < w; ++x) {
                        unsigned char b = PIX(label, w, y, x);
                        if (b != 1 && b != 2) continue;
                        double d = sqrt((double)(y - i) * (y - i) + (double)(x - j) * (x - j));
                        if (b == 1 && d < lmin) lmin = d;
                        if (b == 2 && d < rmin) rmin = d;
                    }
                if (isinf(lmin) && isinf(rmin)) v = 0.5;
                else if (isinf(lmin)) v = 1.0;
                else if (isinf(rmin)) v = 0.0;
                else v = lmin / (lmin + rmin);
            } else v = 0.5;
            PIX(blend, w, i, j) = v;
        }
}

/* Eq. (1) at n chosen pixels (ys[i], xs[i]) of a labelled canvas, by the same
   brute force: for checks of large canvases at sampled pixels. */
void oracle_blend_coeff_at(const unsigned char* label, int h, int w, const int* ys, const int* xs, long n,
                           double* out)
{
    int has1 = 0, has2 = 0;
    for (long k = 0; k < (long)h * w; ++k) {
        has1 |= label[k] == 1;
        has2 |= label[k] == 2;
    }
#pragma omp parallel for schedule(dynamic, 1)
    for (long k = 0; k < n; ++k) {
        int i = ys[k], j = xs[k];
        unsigned char a = PIX(label, w, i, j);
        double v;
        if (a == 1) v = 0.0;
        else if (a == 2) v = 1.0;
        else if (a == 3) {
            if (!has1 && !has2) v = 0.5;
            else if (!has1) v = 1.0;
            else if (!has2) v = 0.0;
            else {
                double l2 = INFINITY, r2 = INFINITY;
                for (int y = 0; y < h; ++y)
                    for (int x = 0; x < w; ++x) {
                        unsigned char b = PIX(label, w, y, x);
                        if (b != 1 && b != 2) continue;
                        double d2 = (double)(y - i) * (y - i) + (double)(x - j) * (x - j);
                        if (b == 1 && d2 < l2) l2 = d2;
                        if (b == 2 && d2 < r2) r2 = d2;
                    }
                double lmin = sqrt(l2), rmin = sqrt(r2);
                v = lmin / (lmin + rmin);
            }
        } else v = 0.5;
        out[k] = v;
    }
}

/* ---------------------------------------------------------------------------
 * Eq. (1) for an overlap strip of width w that spans the canvas height, with
 * Area1 the column just left of it and Area2 the column just right of it:
 * Lmin = x + 1 and Rmin = w - x, so Blend(x) = (x + 1) / (w + 1).
 * out: (w,) one value per column.
 * ------------------------------------------------------------------------- */
void oracle_blend_ramp(int w, double* out)
{
    for (int x = 0; x < w; ++x) out[x] = (double)(x + 1) / (double)(w + 1);
}

/* ---------------------------------------------------------------------------
 * Code 1, the Area3 branch, for every pixel of the overlap strips.
 * L, R: (h, w, c) unit-scaled. flowLR, flowRL: (h, w, 2). blend: (h, w) or
 * NULL for the Eq. (1) strip ramp. F: (h, w, c).
 *   BlendL = 1 - Blend,  BlendR = Blend
 *   ColorL = L(p + (1 - BlendL) FlowRtoL(p)),  ColorR = R(p + (1 - BlendR) FlowLtoR(p))
 *   FlowL = 1 + kFlowMagCoef FlowMagRL,  ExpL = exp(kSoftmaxSharpness BlendL FlowL)
 *   FlowR = 1 + kFlowMagCoef FlowMagLR,  ExpR = exp(kSoftmaxSharpness BlendR FlowR)
 *   F = ColorL ExpL / (ExpL + ExpR) + ColorR ExpR / (ExpL + ExpR)
 * Reading: FlowMagRL / FlowMagLR (named but not defined in the paper) are
 * the Euclidean lengths of FlowRtoL(p) / FlowLtoR(p) divided by the strip
 * width w, so the exponent stays bounded for any strip size.
 * ------------------------------------------------------------------------- */
void oracle_blend(const double* L, const double* R, int h, int w, int c, const double* flowLR,
                  const double* flowRL, const double* blend, double k_sharp, double k_mag, double* F)
{
#pragma omp parallel for schedule(static)
    for (int y = 0; y < h; ++y)
        for (int x = 0; x < w; ++x) {
            size_t p = (size_t)y * w + x;
            double B = blend ? blend[p] : (double)(x + 1) / (double)(w + 1);
            double blendL = 1.0 - B, blendR = B;
            double rlx = flowRL[2 * p], rly = flowRL[2 * p + 1];
            double lrx = flowLR[2 * p], lry = flowLR[2 * p + 1];
            double Lx = x + rlx * (1.0 - blendL), Ly = y + rly * (1.0 - blendL);
            double Rx = x + lrx * (1.0 - blendR), Ry = y + lry * (1.0 - blendR);
            double magRL = sqrt(rlx * rlx + rly * rly) / (double)w;
            double magLR = sqrt(lrx * lrx + lry * lry) / (double)w;
            double expL = exp(k_sharp * blendL * (1.0 + k_mag * magRL));
            double expR = exp(k_sharp * blendR * (1.0 + k_mag * magLR));
            double sL = expL / (expL + expR), sR = expR / (expL + expR);
            for (int ch = 0; ch < c; ++ch) {
                double colL = bilinear_strided(L + ch, h, w, c, Lx, Ly);
                double colR = bilinear_strided(R + ch, h, w, c, Rx, Ry);
                F[p * c + ch] = colL * sL + colR * sR;
            }
        }
}

/* ---------------------------------------------------------------------------
 * Code 1 on a whole canvas (Section III-C-3), every branch:
 *   Area1 (label 1): F = L(p);  Area2 (label 2): F = R(p);
 *   Area3 (label 3): the blend above, with L and R the canvas images;
 *   any other label: F = 0.
 * L, R: (h, w, c) unit-scaled canvas images. label: (h, w). blend: (h, w),
 * Eq. (1). flowLR, flowRL: (fh, fw, 2), the flows of the overlap crop whose
 * pixel (0, 0) is canvas pixel (fy0, fx0).
 * Readings: the Area3 samples read the canvas images (clamp-to-edge at the
 * canvas border), so a displaced sample near the seam reads L or R beyond
 * the crop, as Code 1 samples the images L and R themselves. FlowMag divides
 * by the crop width fw, the overlap width of the strip form. An Area3 pixel
 * outside the crop has no flow and uses zero.
 * ------------------------------------------------------------------------- */
void oracle_compose(const double* L, const double* R, int h, int w, int c, const unsigned char* label,
                    const double* blend, const double* flowLR, const double* flowRL, int fy0, int fx0, int fh,
                    int fw, double k_sharp, double k_mag, double* F)
{
#pragma omp parallel for schedule(static)
    for (int y = 0; y < h; ++y)
        for (int x = 0; x < w; ++x) {
            size_t p = (size_t)y * w + x;
            double* out = F + p * c;
            unsigned char area = label[p];
            if (area == 1) {                      /* Code 1: F(i, j) = L(i, j) */
                for (int ch = 0; ch < c; ++ch) out[ch] = L[p * c + ch];
            } else if (area == 2) {               /* Code 1: F(i, j) = R(i, j) */
                for (int ch = 0; ch < c; ++ch) out[ch] = R[p * c + ch];
            } else if (area == 3) {
                /* FlowRtoL(i, j), FlowLtoR(i, j) from the crop (zero outside it) */
                double rtol_x = 0.0, rtol_y = 0.0, ltor_x = 0.0, ltor_y = 0.0;
                int qy = y - fy0, qx = x - fx0;
                if (qy >= 0 && qy < fh && qx >= 0 && qx < fw) {
                    size_t q = 2 * ((size_t)qy * fw + qx);
                    rtol_x = flowRL[q];
                    rtol_y = flowRL[q + 1];
                    ltor_x = flowLR[q];
                    ltor_y = flowLR[q + 1];
                }
                double BlendL = 1.0 - blend[p], BlendR = blend[p];
                double Lx_ = x + (1.0 - BlendL) * rtol_x, Ly_ = y + (1.0 - BlendL) * rtol_y;
                double Rx_ = x + (1.0 - BlendR) * ltor_x, Ry_ = y + (1.0 - BlendR) * ltor_y;
                double FlowMagRL = sqrt(rtol_x * rtol_x + rtol_y * rtol_y) / (double)fw;
                double FlowMagLR = sqrt(ltor_x * ltor_x + ltor_y * ltor_y) / (double)fw;
                double FlowL = 1.0 + k_mag * FlowMagRL, FlowR = 1.0 + k_mag * FlowMagLR;
                double ExpL = exp(k_sharp * BlendL * FlowL), ExpR = exp(k_sharp * BlendR * FlowR);
                double SoftmaxL = ExpL / (ExpL + ExpR), SoftmaxR = ExpR / (ExpL + ExpR);
                for (int ch = 0; ch < c; ++ch)
                    out[ch] = bilinear_strided(L + ch, h, w, c, Lx_, Ly_) * SoftmaxL +
                              bilinear_strided(R + ch, h, w, c, Rx_, Ry_) * SoftmaxR;
            } else {                              /* Code 1: F(i, j) = 0 */
                for (int ch = 0; ch < c; ++ch) out[ch] = 0.0;
            }
        }
}

/* Blend weights alone (for tests): sL, sR per pixel. */
void oracle_blend_weights(int h, int w, const double* flowLR, const double* flowRL,
                          const double* blend, double k_sharp, double k_mag, double* sL, double* sR)
{
    for (int y = 0; y < h; ++y)
        for (int x = 0; x < w; ++x) {
            size_t p = (size_t)y * w + x;
            double B = blend ? blend[p] : (double)(x + 1) / (double)(w + 1);
            double magRL = hypot(flowRL[2 * p], flowRL[2 * p + 1]) / (double)w;
            double magLR = hypot(flowLR[2 * p], flowLR[2 * p + 1]) / (double)w;
            double expL = exp(k_sharp * (1.0 - B) * (1.0 + k_mag * magRL));
            double expR = exp(k_sharp * B * (1.0 + k_mag * magLR));
            sL[p] = expL / (expL + expR);
            sR[p] = expR / (expL + expR);
        }
}

/* ---------------------------------------------------------------------------
 * Back to 8 bits: round(255 F) with ties to even, clamped to [0, 255].
 * (Reading: the paper does not state how F is stored.)
 * ------------------------------------------------------------------------- */
void oracle_quantize_u8(const double* F, long n, unsigned char* out)
{
    for (long i = 0; i < n; ++i) {
        double v = nearbyint(255.0 * F[i]);   /* default rounding mode: ties to even */
        if (v < 0.0) v = 0.0;
        if (v > 255.0) v = 255.0;
        out[i] = (unsigned char)v;
    }
}

/* ===========================================================================
 * Differentiable refinement (not in the paper: a build extension whose
 * energy takes its smoothness term from the Horn-Schunck half of [20]).
 *
 *   E(u) = sum_p (J(p + u(p)) - T(p))^2
 *        + alpha sum_p sum_{c in {x,y}} [ (u_c(p + e_x) - u_c(p))^2 [x < w-1]
 *                                       + (u_c(p + e_y) - u_c(p))^2 [y < h-1] ]
 * with J sampled bilinearly with clamp-to-edge taps (the sampler of the LK
 * step) and forward differences that are zero across the image border.
 * ========================================================================= */

/* Bilinear sample and its derivative with respect to the sample position,
   taps clamped to the image (the derivative is that of the interpolant). */
static double bilinear_d(const double* I, int h, int w, double x, double y, double* dx, double* dy)
{
    double x0f = floor(x), y0f = floor(y);
    double fx = x - x0f, fy = y - y0f;
    if (x0f < -2.0) x0f = -2.0;
    if (x0f > (double)w + 1.0) x0f = (double)w + 1.0;
    if (y0f < -2.0) y0f = -2.0;
    if (y0f > (double)h + 1.0) y0f = (double)h + 1.0;
    int x0 = (int)x0f, y0 = (int)y0f;
    int xa = clampi(x0, 0, w - 1), xb = clampi(x0 + 1, 0, w - 1);
    int ya = clampi(y0, 0, h - 1), yb = clampi(y0 + 1, 0, h - 1);
    double i00 = PIX(I, w, ya, xa), i10 = PIX(I, w, ya, xb);
    double i01 = PIX(I, w, yb, xa), i11 = PIX(I, w, yb, xb);
    *dx = (1.0 - fy) * (i10 - i00) + fy * (i11 - i01);
    *dy = (1.0 - fx) * (i01 - i00) + fx * (i11 - i10);
    return (1.0 - fy) * ((1.0 - fx) * i00 + fx * i10) + fy * ((1.0 - fx) * i01 + fx * i11);
}

double oracle_energy(const double* T, const double* J, int h, int w, const double* u, double alpha)
{
    double data = 0.0, smooth = 0.0;
    for (int y = 0; y < h; ++y)
        for (int x = 0; x < w; ++x) {
            size_t p = (size_t)y * w + x;
            double r = bilinear_strided(J, h, w, 1, x + u[2 * p], y + u[2 * p + 1]) - T[p];
            data += r * r;
            for (int c = 0; c < 2; ++c) {
                if (x < w - 1) { double d = u[2 * (p + 1) + c] - u[2 * p + c]; smooth += d * d; }
                if (y < h - 1) { double d = u[2 * (p + w) + c] - u[2 * p + c]; smooth += d * d; }
            }
        }
    return data + alpha * smooth;
}

/* Gradients of oracle_energy: gu (h, w, 2), gT (h, w), gJ (h, w); any may be
   NULL. dE/dJ collects 2 r(p) times each tap's bilinear weight at the tap's
   clamped position. */
void oracle_energy_grad(const double* T, const double* J, int h, int w, const double* u, double alpha,
                        double* gu, double* gT, double* gJ)
{
    size_t n = (size_t)h * w;
    if (gJ) memset(gJ, 0, n * sizeof(double));
    for (int y = 0; y < h; ++y)
        for (int x = 0; x < w; ++x) {
            size_t p = (size_t)y * w + x;
            double sx = x + u[2 * p], sy = y + u[2 * p + 1];
            double jdx, jdy;
            double r = bilinear_d(J, h, w, sx, sy, &jdx, &jdy) - T[p];
            if (gu) {
                gu[2 * p + 0] = 2.0 * r * jdx;
                gu[2 * p + 1] = 2.0 * r * jdy;
                for (int c = 0; c < 2; ++c) {
                    double s = 0.0;
                    if (x > 0) s += u[2 * p + c] - u[2 * (p - 1) + c];
                    if (x < w - 1) s += u[2 * p + c] - u[2 * (p + 1) + c];
                    if (y > 0) s += u[2 * p + c] - u[2 * (p - w) + c];
                    if (y < h - 1) s += u[2 * p + c] - u[2 * (p + w) + c];
                    gu[2 * p + c] += 2.0 * alpha * s;
                }
            }
            if (gT) gT[p] = -2.0 * r;
            if (gJ) {
                double x0f = floor(sx), y0f = floor(sy);
                double fx = sx - x0f, fy = sy - y0f;
                if (x0f < -2.0) x0f = -2.0;
                if (x0f > (double)w + 1.0) x0f = (double)w + 1.0;
                if (y0f < -2.0) y0f = -2.0;
                if (y0f > (double)h + 1.0) y0f = (double)h + 1.0;
                int x0 = (int)x0f, y0 = (int)y0f;
                int xa = clampi(x0, 0, w - 1), xb = clampi(x0 + 1, 0, w - 1);
                int ya = clampi(y0, 0, h - 1), yb = clampi(y0 + 1, 0, h - 1);
                double g = 2.0 * r;
                PIX(gJ, w, ya, xa) += g * (1.0 - fy) * (1.0 - fx);
                PIX(gJ, w, ya, xb) += g * (1.0 - fy) * fx;
                PIX(gJ, w, yb, xa) += g * fy * (1.0 - fx);
                PIX(gJ, w, yb, xb) += g * fy * fx;
            }
        }
}

/* Transpose of oracle_pyr_down: given the gradient of the (ceil(h/2),
   ceil(w/2)) output, the gradient of the (h, w) input. Each output pixel
   spreads its value back along the same 5x5 binomial weights and clamped
   taps that formed it. */
void oracle_pyr_down_adjoint(const double* gdst, int h, int w, double* gsrc)
{
    static const double k[5] = {1.0 / 16, 4.0 / 16, 6.0 / 16, 4.0 / 16, 1.0 / 16};
    int hd = (h + 1) / 2, wd = (w + 1) / 2;
    memset(gsrc, 0, (size_t)h * w * sizeof(double));
    for (int yd = 0; yd < hd; ++yd)
        for (int xd = 0; xd < wd; ++xd) {
            double g = PIX(gdst, wd, yd, xd);
            for (int ty = -2; ty <= 2; ++ty)
                for (int tx = -2; tx <= 2; ++tx) {
                    int sy = clampi(2 * yd + ty, 0, h - 1), sx = clampi(2 * xd + tx, 0, w - 1);
                    PIX(gsrc, w, sy, sx) += k[ty + 2] * k[tx + 2] * g;
                }
        }
}
