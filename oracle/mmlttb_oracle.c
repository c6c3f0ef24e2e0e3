/*
 * MinMaxLTTB oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, single-threaded CPU statement of what the MinMaxLTTB method of
 * "MinMaxLTTB: Leveraging MinMax-Preselection to Scale LTTB" (arXiv 2305.00332)
 * computes.  Only the test suite, the package smoke check and the benchmark's CPU
 * baseline load this file's shared library; the CUDA library never does, and the
 * two share no code.  Build with  -O2 -ffp-contract=off  and no fast-math, so that
 * every floating-point sum, difference and product below is rounded on its own,
 * in the order written (GCC on aarch64 would otherwise contract a*b-c*d to FMA).
 *
 * What the paper states (Sec. 3):
 *   - MinMaxLTTB is two steps: MinMax preselects vertical extrema (the argmin and
 *     argmax of each bin), then LTTB runs on the preselected points only.
 *   - The first and last point of the series are always handed to LTTB.
 *   - r_ps * n_out points are preselected; r_ps/2 MinMax sub-buckets per LTTB
 *     bucket, i.e. n_out * r_ps / 2 MinMax bins.
 * What it takes from Sec. 2.2.1 and the LTTB thesis it cites:
 *   - MinMax: per bin B_i, the vertical extrema via (arg)min and (arg)max.
 *   - LTTB: per bucket B_i, the point forming the largest triangle with the
 *     point selected in B_{i-1} and the average (mean x, mean y) of B_{i+1}.
 *
 * Readings where the paper is silent (numbered R1..R21 wherever they are cited):
 *   R1  LTTB buckets: first and last point fixed, K = n_out-2 buckets over the
 *       interior positions 1..m-2, bucket j = [floor(j(m-2)/K)+1, floor((j+1)(m-2)/K)+1)
 *       in exact integer arithmetic.
 *   R2  MinMax bins, index mode: B = floor(n_out*r_ps/2) bins over the interior
 *       points 1..n-2, bin i = [floor(i(n-2)/B)+1, floor((i+1)(n-2)/B)+1).
 *   R3  MinMax bins, x mode (int64 x, non-decreasing): edges
 *       e_i = x_0 + floor(i (x_{n-1}-x_0) / B); interior point p is in the largest
 *       bin i with e_i <= x_p (so the last bin runs up to and including x_{n-1}).
 *       Empty bins emit nothing.
 *   R4  LTTB over preselected points: buckets are formed over positions in the
 *       preselected list; means and areas use the original coordinates.
 *   R5  The next bucket of the last bucket is the single last point.
 *   R6  Area = |(xa-xc)(yb-ya) - (xa-xb)(yc-ya)| in FP64, each product and
 *       difference rounded separately, without the factor 1/2.  Implicit x is
 *       the index as a double.
 *   R7  Mean = FP64 sum from left to right over the bucket, then one division by
 *       the count.
 *   R8  Ties: the lowest index wins, in MinMax (min and max) and in LTTB.
 *   R9  A bin whose argmin equals its argmax emits that index once.
 *   R10 -0.0 and +0.0 compare equal (IEEE), so they tie.
 *   R11 NaN in y is a precondition violation; the output is then unspecified.
 *   R12 B = floor(n_out*r_ps/2) for odd products.
 *   R13 minmaxlttb rejects r_ps < 2; minmax_preselect alone accepts r_ps >= 1.
 *   R14 When fewer than n_out points are preselected (x mode), all are returned.
 *   R15 When r_ps*n_out >= n, minmaxlttb is plain LTTB on all points; when
 *       n_out >= n it returns every index.
 *   R16 M4 (Sec. 2.2.1, Table 1: the vertical extrema and the first and last point
 *       of each bin): B = floor(n_out/4) bins over ALL points 0..n-1, index bins
 *       [floor(i n/B), floor((i+1) n/B)), x-width bins as R3 but over all points;
 *       per non-empty bin the sorted distinct {first, argmin, argmax, last}.
 *   R17 x-width bins on float64 x: D = x_{n-1} - x_0 and e_i = x_0 + (i*D)/B in FP64,
 *       each operation rounded on its own; point p is in the largest bin i with
 *       e_i <= x_p (FP64 comparison), as R3 otherwise.
 *   R18 NaN-aware MinMax / M4 (binmode | NAN_AWARE): a bin that holds a NaN reports
 *       its first NaN as both argmin and argmax (the convention of numpy's argmin and
 *       argmax); other bins as R8.  Plain MinMax/LTTB keep R11.
 *   R19 Line-chart rasterisation (Sec. 3.1 and the caption of fig:vis_repr: linear
 *       interpolation, lines 2 pixels wide, anti-aliased).  A W x H canvas, pixel
 *       (c, r) covering [c, c+1) x [r, r+1), row 0 at the top.  A data point maps to
 *       px = (x - x0) * (W / (x1 - x0)), py = (y1 - y) * (H / (y1 - y0)) in FP64, each
 *       operation rounded, then rounded to float32 (a zero extent maps to W/2 or H/2).
 *       Each pixel holds 4 x 4 samples at c + (i + 0.5)/4, r + (k + 0.5)/4; a sample is
 *       inked when its distance to a segment between consecutive drawn points is at
 *       most 1 (half the line width), computed in float32 with every operation
 *       rounded in the order written in raster_sample().  Intensity = round(255 x
 *       inked samples / 16), i.e. (16ths * 255 + 8) / 16 in integers.
 *   R20 Conv-mask: the pixels with an inked reference pixel within Chebyshev
 *       distance 1 (a 3 x 3 dilation of the reference).
 *   R21 PEM_20 = (pixels whose intensities differ by more than 20) / |mask|;
 *       MSE = (sum over all pixels of the squared intensity difference) / |mask|; both
 *       0 for an empty mask.  mmo_visual_counts returns the exact integer counts.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define MMO_EINVAL (-1)
#define MMO_ENOMEM (-5)

enum { Y_F32 = 0, Y_F64 = 1 };
enum { X_IMPLICIT = 0, X_I64 = 1, X_F64 = 2 };
enum { BINS_INDEX = 0, BINS_XWIDTH = 1 };
#define NAN_AWARE 0x10 /* flag OR-ed into binmode (R18) */

/* The y value of point i as a double (a float converts exactly). */
static double y_at(const void *y, int ydt, int64_t i)
{
    if (ydt == Y_F32) return (double)((const float *)y)[i];
    return ((const double *)y)[i];
}

/* The x coordinate of point i as a double (R6: implicit x is the index). */
static double x_at(const void *x, int xk, int64_t i)
{
    if (xk == X_IMPLICIT) return (double)i;
    if (xk == X_I64) return (double)((const int64_t *)x)[i];
    return ((const double *)x)[i];
}

/* floor(a*b/c) + 1 for 0 <= a <= c, b >= 0, c > 0: the start of part a when
   b items are split into c equal-count parts (R1, R2). */
static int64_t part_start(int64_t a, int64_t b, int64_t c)
{
    unsigned __int128 num = (unsigned __int128)(uint64_t)a * (uint64_t)b;
    return (int64_t)(num / (uint64_t)c) + 1;
}

static int check_common(const void *y, int ydt, const void *x, int xk, int64_t n)
{
    if (n < 0) return MMO_EINVAL;
    if (n > 0 && y == NULL) return MMO_EINVAL;
    if (ydt != Y_F32 && ydt != Y_F64) return MMO_EINVAL;
    if (xk != X_IMPLICIT && xk != X_I64 && xk != X_F64) return MMO_EINVAL;
    if (xk != X_IMPLICIT && n > 0 && x == NULL) return MMO_EINVAL;
    return 0;
}

/*
 * MinMax per bin (Sec. 2.2.1; the preselection of Sec. 3).  For each of the B
 * bins over the interior points 1..n-2, writes the index of the first minimum and
 * of the first maximum of y, or -1 for both when the bin is empty.
 * Bins follow R2 (index mode) or R3 (x mode).  Returns B, or a negative error.
 */
int64_t mmo_minmax_bins(const void *y, int ydt, const void *x, int xk, int64_t n,
                        int64_t B, int binmode, int64_t *imin, int64_t *imax)
{
    int rc = check_common(y, ydt, x, xk, n);
    if (rc) return rc;
    const int nan_aware = (binmode & NAN_AWARE) != 0;
    binmode &= ~NAN_AWARE;
    if (B < 1) return MMO_EINVAL;
    if (binmode != BINS_INDEX && binmode != BINS_XWIDTH) return MMO_EINVAL;
    if (binmode == BINS_XWIDTH && xk == X_IMPLICIT) return MMO_EINVAL;

    double *vmin = (double *)malloc(sizeof(double) * (size_t)B);
    double *vmax = (double *)malloc(sizeof(double) * (size_t)B);
    char *hasnan = (char *)calloc((size_t)B, 1);
    if (!vmin || !vmax || !hasnan) { free(vmin); free(vmax); free(hasnan); return MMO_ENOMEM; }
    for (int64_t b = 0; b < B; b++) { imin[b] = -1; imax[b] = -1; }

    const int64_t N = n - 2; /* interior points 1..n-2 */
    const int64_t *xi = (const int64_t *)x;
    int64_t x0 = 0, D = 0;
    if (binmode == BINS_XWIDTH && xk == X_I64 && n >= 2) { x0 = xi[0]; D = xi[n - 1] - xi[0]; }

    /* start (index mode) or left edge (x mode) of bin b+1; past the last bin, a bound
       above every int64 */
#define NEXT_BOUND(bb)                                                                  \
    ((bb) + 1 >= B ? (__int128)INT64_MAX + 1                                            \
     : binmode == BINS_INDEX ? (__int128)part_start((bb) + 1, N, B)                     \
     : (__int128)x0 + ((__int128)((bb) + 1) * (__int128)D) / (__int128)B)
    /* float64 x (R17): left edge of bin b+1 in FP64, +inf past the last bin */
    const double *xf = (const double *)x;
    const double xf0 = (binmode == BINS_XWIDTH && xk == X_F64 && n >= 2) ? xf[0] : 0.0;
    const double Df = (binmode == BINS_XWIDTH && xk == X_F64 && n >= 2) ? xf[n - 1] - xf[0] : 0.0;
#define NEXT_EDGE_F(bb) ((bb) + 1 >= B ? INFINITY : xf0 + ((double)((bb) + 1) * Df) / (double)B)
    const int fx = binmode == BINS_XWIDTH && xk == X_F64;
    int64_t b = 0;
    __int128 next = fx ? 0 : NEXT_BOUND(b);
    double nextf = fx ? NEXT_EDGE_F(b) : 0.0;
    for (int64_t p = 1; p <= n - 2; p++) {
        if (fx) {
            while (nextf <= xf[p]) {
                b++;
                nextf = NEXT_EDGE_F(b);
            }
        }
        /* Move to the last bin whose start is at or before p:
           index mode: start(b+1) <= p;  x mode: e_{b+1} = x_0 + floor((b+1) D / B) <= x_p (R3) */
        __int128 here = fx ? 0 : binmode == BINS_INDEX ? (__int128)p : (__int128)xi[p];
        while (!fx && next <= here) {
            b++;
            next = NEXT_BOUND(b);
        }
        double v = y_at(y, ydt, p);
        if (imin[b] < 0) {
            imin[b] = p; imax[b] = p; vmin[b] = v; vmax[b] = v;
            if (nan_aware && isnan(v)) hasnan[b] = 1;
        } else if (nan_aware && hasnan[b]) {
            /* the bin's first NaN decides both extremes (R18) */
        } else if (nan_aware && isnan(v)) {
            hasnan[b] = 1; imin[b] = p; imax[b] = p;
        } else {
            /* strict comparisons keep the first occurrence (R8, R10) */
            if (v < vmin[b]) { vmin[b] = v; imin[b] = p; }
            if (v > vmax[b]) { vmax[b] = v; imax[b] = p; }
        }
    }
#undef NEXT_BOUND
#undef NEXT_EDGE_F
    free(vmin);
    free(vmax);
    free(hasnan);
    return B;
}

/*
 * MinMax preselection (Sec. 3, first step): point 0, then for each non-empty bin
 * its argmin and argmax in increasing index order (once if equal, R9), then point
 * n-1.  B = floor(n_out*r_ps/2) (R12).  out must hold 2B+2 indices.
 * Returns the number of indices written, or a negative error.
 */
int64_t mmo_minmax_preselect(const void *y, int ydt, const void *x, int xk, int64_t n,
                             int64_t n_out, int32_t r_ps, int binmode, int64_t *out)
{
    int rc = check_common(y, ydt, x, xk, n);
    if (rc) return rc;
    if (n_out < 1 || r_ps < 1) return MMO_EINVAL;
    if (n_out > INT64_MAX / r_ps) return MMO_EINVAL;
    int64_t B = n_out * (int64_t)r_ps / 2;
    if (B < 1) return MMO_EINVAL;
    const int bm = binmode & ~NAN_AWARE;
    if (bm != BINS_INDEX && bm != BINS_XWIDTH) return MMO_EINVAL;
    if (bm == BINS_XWIDTH && xk == X_IMPLICIT) return MMO_EINVAL;
    if (n == 0) return 0;
    if (n == 1) { out[0] = 0; return 1; }

    int64_t *imin = (int64_t *)malloc(sizeof(int64_t) * (size_t)B);
    int64_t *imax = (int64_t *)malloc(sizeof(int64_t) * (size_t)B);
    if (!imin || !imax) { free(imin); free(imax); return MMO_ENOMEM; }
    int64_t r = mmo_minmax_bins(y, ydt, x, xk, n, B, binmode, imin, imax);
    if (r < 0) { free(imin); free(imax); return r; }

    int64_t m = 0;
    out[m++] = 0;
    for (int64_t b = 0; b < B; b++) {
        if (imin[b] < 0) continue; /* empty bin (R3) */
        int64_t lo = imin[b] < imax[b] ? imin[b] : imax[b];
        int64_t hi = imin[b] < imax[b] ? imax[b] : imin[b];
        out[m++] = lo;
        if (hi != lo) out[m++] = hi;
    }
    out[m++] = n - 1;
    free(imin);
    free(imax);
    return m;
}

/*
 * LTTB (Sec. 2.2.1 and the thesis it cites) on the m points at positions 0..m-1,
 * where position p is original point idx[p] (idx == NULL: position p is point p).
 * Buckets R1, next-bucket mean R5/R7, area R6, ties R8.  Writes min(n_out, m)
 * original indices to out and returns that count, or a negative error.
 */
int64_t mmo_lttb_positions(const void *y, int ydt, const void *x, int xk,
                           const int64_t *idx, int64_t m, int64_t n_out, int64_t *out)
{
    int rc = check_common(y, ydt, x, xk, m);
    if (rc) return rc;
    if (n_out < 0) return MMO_EINVAL;
#define IDX(p) (idx ? idx[(p)] : (int64_t)(p))
    if (n_out >= m) { /* nothing to drop: every point (R14, R15) */
        for (int64_t p = 0; p < m; p++) out[p] = IDX(p);
        return m;
    }
    if (n_out < 3) return MMO_EINVAL;

    const int64_t K = n_out - 2; /* buckets */
    const int64_t N = m - 2;     /* interior positions, N > K */
    int64_t a = 0;               /* position of the previously selected point */
    out[0] = IDX(0);
    for (int64_t j = 0; j < K; j++) {
        int64_t lo = part_start(j, N, K);
        int64_t hi = part_start(j + 1, N, K);
        int64_t nlo, nhi;
        if (j + 1 < K) { nlo = hi; nhi = part_start(j + 2, N, K); }
        else { nlo = m - 1; nhi = m; } /* R5 */

        /* mean of the next bucket: left-to-right sums, one division (R7) */
        double sx = 0.0, sy = 0.0;
        for (int64_t p = nlo; p < nhi; p++) {
            sx = sx + x_at(x, xk, IDX(p));
            sy = sy + y_at(y, ydt, IDX(p));
        }
        double cnt = (double)(nhi - nlo);
        double xc = sx / cnt, yc = sy / cnt;

        double xa = x_at(x, xk, IDX(a)), ya = y_at(y, ydt, IDX(a));
        double best = -1.0;
        int64_t pick = lo;
        for (int64_t p = lo; p < hi; p++) {
            double xb = x_at(x, xk, IDX(p)), yb = y_at(y, ydt, IDX(p));
            double area = fabs((xa - xc) * (yb - ya) - (xa - xb) * (yc - ya));
            if (p == lo || area > best) { best = area; pick = p; } /* R8 */
        }
        out[j + 1] = IDX(pick);
        a = pick;
    }
    out[K + 1] = IDX(m - 1);
#undef IDX
    return n_out;
}

/* Plain LTTB on all n points. */
int64_t mmo_lttb(const void *y, int ydt, const void *x, int xk, int64_t n, int64_t n_out,
                 int64_t *out)
{
    return mmo_lttb_positions(y, ydt, x, xk, NULL, n, n_out, out);
}

/*
 * MinMaxLTTB (Sec. 3): n_out >= n returns every index; r_ps*n_out >= n runs LTTB
 * on all points (R15); otherwise MinMax preselection followed by LTTB on the
 * preselected points (R4, R14).  out holds min(n_out, n) indices.
 */
int64_t mmo_minmaxlttb(const void *y, int ydt, const void *x, int xk, int64_t n,
                       int64_t n_out, int32_t r_ps, int binmode, int64_t *out)
{
    int rc = check_common(y, ydt, x, xk, n);
    if (rc) return rc;
    if (n_out < 0) return MMO_EINVAL;
    if (binmode != BINS_INDEX && binmode != BINS_XWIDTH) return MMO_EINVAL;
    if (binmode == BINS_XWIDTH && xk == X_IMPLICIT) return MMO_EINVAL;
    if (n_out >= n) {
        for (int64_t p = 0; p < n; p++) out[p] = p;
        return n;
    }
    if (n_out < 3 || r_ps < 2) return MMO_EINVAL;
    if (n_out > INT64_MAX / r_ps) return MMO_EINVAL;
    if ((int64_t)r_ps * n_out >= n) return mmo_lttb(y, ydt, x, xk, n, n_out, out);

    int64_t B = n_out * (int64_t)r_ps / 2;
    int64_t *sel = (int64_t *)malloc(sizeof(int64_t) * (size_t)(2 * B + 2));
    if (!sel) return MMO_ENOMEM;
    int64_t m = mmo_minmax_preselect(y, ydt, x, xk, n, n_out, r_ps, binmode, sel);
    if (m < 0) { free(sel); return m; }
    int64_t r = mmo_lttb_positions(y, ydt, x, xk, sel, m, n_out, out);
    free(sel);
    return r;
}

/*
 * M4 (Sec. 2.2.1, Table 1; reading R16): per bin the first point, the first argmin,
 * the first argmax and the last point, in increasing index order without repeats.
 * out must hold 4B indices.  Returns the number written, or a negative error.
 */
int64_t mmo_m4(const void *y, int ydt, const void *x, int xk, int64_t n, int64_t n_out,
               int binmode, int64_t *out)
{
    int rc = check_common(y, ydt, x, xk, n);
    if (rc) return rc;
    const int nan_aware = (binmode & NAN_AWARE) != 0;
    binmode &= ~NAN_AWARE;
    if (n_out < 4) return MMO_EINVAL;
    if (binmode != BINS_INDEX && binmode != BINS_XWIDTH) return MMO_EINVAL;
    if (binmode == BINS_XWIDTH && xk == X_IMPLICIT) return MMO_EINVAL;
    const int64_t B = n_out / 4;
    if (n == 0) return 0;

    int64_t *first = (int64_t *)malloc(sizeof(int64_t) * (size_t)B);
    int64_t *last = (int64_t *)malloc(sizeof(int64_t) * (size_t)B);
    int64_t *imin = (int64_t *)malloc(sizeof(int64_t) * (size_t)B);
    int64_t *imax = (int64_t *)malloc(sizeof(int64_t) * (size_t)B);
    double *vmin = (double *)malloc(sizeof(double) * (size_t)B);
    double *vmax = (double *)malloc(sizeof(double) * (size_t)B);
    char *hasnan = (char *)calloc((size_t)B, 1);
    if (!first || !last || !imin || !imax || !vmin || !vmax || !hasnan) {
        free(first); free(last); free(imin); free(imax); free(vmin); free(vmax); free(hasnan);
        return MMO_ENOMEM;
    }
    for (int64_t b = 0; b < B; b++) first[b] = -1;
    const int64_t *xi = (const int64_t *)x;
    int64_t x0 = 0, D = 0;
    if (binmode == BINS_XWIDTH && xk == X_I64) { x0 = xi[0]; D = xi[n - 1] - xi[0]; }
    const double *xf = (const double *)x;
    const int fx = binmode == BINS_XWIDTH && xk == X_F64;
    const double xf0 = fx ? xf[0] : 0.0, Df = fx ? xf[n - 1] - xf[0] : 0.0;
#define NEXT_EDGE_F4(bb) ((bb) + 1 >= B ? INFINITY : xf0 + ((double)((bb) + 1) * Df) / (double)B)
    /* start (index mode) or left edge (x mode) of bin b+1; past the last bin, a bound
       above every int64 */
#define NEXT_BOUND4(bb)                                                                 \
    ((bb) + 1 >= B ? (__int128)INT64_MAX + 1                                            \
     : binmode == BINS_INDEX ? (__int128)(((unsigned __int128)((bb) + 1) * (uint64_t)n) / (uint64_t)B) \
     : (__int128)x0 + ((__int128)((bb) + 1) * (__int128)D) / (__int128)B)
    int64_t b = 0;
    __int128 next = fx ? 0 : NEXT_BOUND4(b);
    double nextf = fx ? NEXT_EDGE_F4(b) : 0.0;
    for (int64_t p = 0; p < n; p++) {
        if (fx) {
            while (nextf <= xf[p]) {
                b++;
                nextf = NEXT_EDGE_F4(b);
            }
        }
        __int128 here = fx ? 0 : binmode == BINS_INDEX ? (__int128)p : (__int128)xi[p];
        while (!fx && next <= here) {
            b++;
            next = NEXT_BOUND4(b);
        }
        double v = y_at(y, ydt, p);
        if (first[b] < 0) {
            first[b] = p; last[b] = p; imin[b] = p; imax[b] = p; vmin[b] = v; vmax[b] = v;
            if (nan_aware && isnan(v)) hasnan[b] = 1;
        } else {
            last[b] = p;
            if (nan_aware && hasnan[b]) {
                /* the bin's first NaN decides both extremes (R18) */
            } else if (nan_aware && isnan(v)) {
                hasnan[b] = 1; imin[b] = p; imax[b] = p;
            } else {
                if (v < vmin[b]) { vmin[b] = v; imin[b] = p; }
                if (v > vmax[b]) { vmax[b] = v; imax[b] = p; }
            }
        }
    }
#undef NEXT_BOUND4
#undef NEXT_EDGE_F4
    int64_t m = 0;
    for (b = 0; b < B; b++) {
        if (first[b] < 0) continue;
        int64_t c[4] = {first[b], imin[b] < imax[b] ? imin[b] : imax[b],
                        imin[b] < imax[b] ? imax[b] : imin[b], last[b]};
        for (int k = 0; k < 4; k++)
            if (k == 0 || c[k] != c[k - 1]) out[m++] = c[k];
    }
    free(first); free(last); free(imin); free(imax); free(vmin); free(vmax); free(hasnan);
    return m;
}


/* ---- line-chart rasterisation and visual metrics (R19-R21) ---------------- */

/* Canvas coordinate of a data value: v -> (v - a) * (size / (b - a)), FP64, then
   float32; a zero extent maps to the middle.  `flip` maps to (b - v) * ... (rows). */
static float raster_coord(double v, double a, double b, int size, int flip)
{
    double d = b - a;
    if (d == 0.0) return (float)(0.5 * (double)size);
    double s = (double)size / d;
    double t = flip ? (b - v) : (v - a);
    return (float)(t * s);
}

/* Whether sample (sx, sy) lies within distance 1 of segment (ax, ay)-(bx, by). */
static int raster_sample(float sx, float sy, float ax, float ay, float bx, float by)
{
    float dx = bx - ax, dy = by - ay;
    float len2 = dx * dx + dy * dy;
    float t = 0.0f;
    if (len2 > 0.0f) {
        float num = (sx - ax) * dx + (sy - ay) * dy;
        t = num / len2;
        if (t < 0.0f) t = 0.0f;
        if (t > 1.0f) t = 1.0f;
    }
    float qx = ax + t * dx, qy = ay + t * dy;
    float ex = sx - qx, ey = sy - qy;
    float d2 = ex * ex + ey * ey;
    return d2 <= 1.0f;
}

/* Rasterise the polyline through points idx[0..k) of the series (idx NULL: all n
   points) into `mask`: one 16-bit sample mask per pixel (row-major, W x H), OR-ed
   into what is already there.  Returns the number of segments drawn. */
int64_t mmo_raster(const void *y, int ydt, const void *x, int xk, int64_t n, const int64_t *idx,
                   int64_t k, double x0, double x1, double y0, double y1, int W, int H, uint32_t *mask)
{
    if (check_common(y, ydt, x, xk, n) || W <= 0 || H <= 0 || !mask) return MMO_EINVAL;
    if (!idx) k = n;
    int64_t segs = 0;
    for (int64_t q = 0; q + 1 < k; q++) {
        int64_t ia = idx ? idx[q] : q, ib = idx ? idx[q + 1] : q + 1;
        float ax = raster_coord(x_at(x, xk, ia), x0, x1, W, 0);
        float ay = raster_coord(y_at(y, ydt, ia), y0, y1, H, 1);
        float bx = raster_coord(x_at(x, xk, ib), x0, x1, W, 0);
        float by = raster_coord(y_at(y, ydt, ib), y0, y1, H, 1);
        segs++;
        /* A NaN endpoint makes every sample distance NaN, so the segment inks nothing. */
        if (ax != ax || ay != ay || bx != bx || by != by) continue;
        float lox = ax < bx ? ax : bx, hix = ax < bx ? bx : ax;
        float loy = ay < by ? ay : by, hiy = ay < by ? by : ay;
        double c0 = floor((double)lox - 1.0), c1 = floor((double)hix + 1.0);
        double r0 = floor((double)loy - 1.0), r1 = floor((double)hiy + 1.0);
        /* clip to the canvas (from both sides, so that far-away coordinates leave an
           empty range and every value converts to int64) */
        if (c0 < 0) c0 = 0;
        if (r0 < 0) r0 = 0;
        if (c0 > W) c0 = W;
        if (r0 > H) r0 = H;
        if (c1 > W - 1) c1 = W - 1;
        if (r1 > H - 1) r1 = H - 1;
        if (c1 < -1) c1 = -1;
        if (r1 < -1) r1 = -1;
        for (int64_t r = (int64_t)r0; r <= (int64_t)r1; r++)
            for (int64_t c = (int64_t)c0; c <= (int64_t)c1; c++) {
                uint32_t m = 0;
                for (int kk = 0; kk < 4; kk++)
                    for (int i = 0; i < 4; i++) {
                        float sx = (float)c + (0.25f * (float)i + 0.125f);
                        float sy = (float)r + (0.25f * (float)kk + 0.125f);
                        if (raster_sample(sx, sy, ax, ay, bx, by)) m |= 1u << (kk * 4 + i);
                    }
                mask[r * W + c] |= m;
            }
    }
    return segs;
}

/* Intensities of a canvas of sample masks (R19). */
void mmo_raster_intensity(const uint32_t *mask, int64_t pixels, uint8_t *out)
{
    for (int64_t p = 0; p < pixels; p++) {
        uint32_t v = mask[p] & 0xffffu;
        int inked = 0;
        while (v) { inked += (int)(v & 1u); v >>= 1; }
        out[p] = (uint8_t)((inked * 255 + 8) / 16);
    }
}

/* Exact counts behind PEM_margin and MSE (R20, R21): counts[0] = pixels whose
   intensities differ by more than `margin`, counts[1] = sum of squared differences,
   counts[2] = conv-mask size. */
void mmo_visual_counts(const uint8_t *ref, const uint8_t *img, int W, int H, int margin, int64_t *counts)
{
    int64_t over = 0, sq = 0, msize = 0;
    for (int r = 0; r < H; r++)
        for (int c = 0; c < W; c++) {
            int d = (int)ref[r * W + c] - (int)img[r * W + c];
            if (d < 0) d = -d;
            if (d > margin) over++;
            sq += (int64_t)d * d;
            int inmask = 0;
            for (int rr = r - 1; rr <= r + 1 && !inmask; rr++)
                for (int cc = c - 1; cc <= c + 1; cc++)
                    if (rr >= 0 && rr < H && cc >= 0 && cc < W && ref[rr * W + cc] > 0) { inmask = 1; break; }
            msize += inmask;
        }
    counts[0] = over;
    counts[1] = sq;
    counts[2] = msize;
}
