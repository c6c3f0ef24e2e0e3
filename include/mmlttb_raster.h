/*
 * mmlttb_raster.h -- C ABI of the headless line-chart rasteriser and the visual
 * metrics of libmmlttb.so (arXiv 2305.00332, Sec. 4: downsampled line charts are
 * rendered and compared with the chart of all points by PEM_20 and MSE; the figure
 * on visual representativeness: linear interpolation, 2-pixel-wide anti-aliased
 * lines).  The conventions of mmlttb.h hold: device pointers owned by the caller,
 * asynchronous on `stream`, MMLTTB_OK or a negative MMLTTB_E* code, argument errors
 * detected on the host before anything is enqueued, nothing allocated.
 *
 * The rendering model (fixed so that every pixel is reproducible bit for bit):
 *   - A W x H canvas; pixel (c, r) covers [c, c+1) x [r, r+1), row 0 at the top,
 *     stored row-major.
 *   - A point (x, y) maps to px = (x - x0) * (W / (x1 - x0)) and
 *     py = (y1 - y) * (H / (y1 - y0)), in FP64 with every operation rounded on its
 *     own, then rounded to float32.  A zero extent (x1 == x0 or y1 == y0) maps to
 *     W/2 or H/2.  Implicit x is the index as a double; int64 x converts to the
 *     nearest double.
 *   - Consecutive drawn points are joined by segments.  Each pixel holds 4 x 4
 *     samples at (c + (i + 0.5)/4, r + (k + 0.5)/4), bit k*4 + i of its mask.  A
 *     sample is inked by a segment A-B when its distance to the segment is at most 1
 *     (half the line width), computed in float32 with each operation rounded on its
 *     own, no fused multiply-add:
 *       d = B - A, l2 = dx*dx + dy*dy,
 *       t = ((sx-ax)*dx + (sy-ay)*dy) / l2 clamped to [0, 1] (t = 0 when l2 == 0),
 *       e = S - (A + t*d),  inked iff ex*ex + ey*ey <= 1.
 *     Only pixels in [floor(min px) - 1, floor(max px) + 1] x [floor(min py) - 1,
 *     floor(max py) + 1] (clipped to the canvas) are tested; no sample outside that
 *     box lies within distance 1.  A segment with a NaN endpoint inks nothing.
 *   - Intensity = round(255 * inked samples / 16) = (inked * 255 + 8) / 16.
 *   - Conv-mask = pixels with a reference pixel of intensity > 0 within Chebyshev
 *     distance 1.  PEM_margin = #{pixels with |ref - img| > margin} / |mask| and
 *     MSE = sum (ref - img)^2 / |mask| (all pixels), 0 when the mask is empty.
 */
#ifndef MMLTTB_RASTER_H
#define MMLTTB_RASTER_H

#include "mmlttb.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Largest canvas side the rasteriser accepts; W * H must also stay <= 2^28. */
#define MMLTTB_RASTER_MAX_SIDE 65536

/*
 * The line chart of a (downsampled) series, as rendered for the visual comparison of
 * Sec. 4 (linear interpolation, 2-pixel lines, anti-aliased; readings above).
 * Rasterise the polyline through points idx[0..k) of the series (x, y) -- or
 * through all n_in points when idx is NULL (k is then ignored) -- and OR each
 * pixel's 16-bit sample mask into mask[r * width + c] (device uint32[height *
 * width]; zero it first for a fresh canvas; drawing several polylines into one
 * canvas overlays them).
 *   y, ydtype, x, xkind, n_in  the series, as in mmlttb.h; here x need not be
 *                              monotone (every segment is drawn on its own).
 *   idx        device int64[k], indices into the series (for instance a
 *              downsampling result); an index outside [0, n_in) is a precondition
 *              violation, and the segments that end at it draw nothing.
 *   x0, x1, y0, y1       the data extents mapped onto the canvas (finite; x1 < x0 or
 *                        y1 < y0 mirrors the chart).
 *   width, height        canvas size, 1..MMLTTB_RASTER_MAX_SIDE, width*height <= 2^28.
 * One launch: a warp per segment (per 31 consecutive segments when there are many).
 * Fewer than two drawn points enqueue nothing.
 * MMLTTB_EINVAL for a NULL y/mask, a NULL x that is not implicit, bad enums, n_in or
 * k < 0, a non-finite extent, or a canvas size out of range.
 */
int mmlttb_raster(const void *y, int ydtype, const void *x, int xkind, int64_t n_in,
                  const int64_t *idx, int64_t k, double x0, double x1, double y0, double y1,
                  int32_t width, int32_t height, uint32_t *mask, mmlttb_stream stream);

/*
 * Anti-aliased intensity of a rendered chart (Sec. 4 renders; coverage reading above).
 * 8-bit intensities of a canvas of sample masks: out[p] = (popcount(mask[p] &
 * 0xffff) * 255 + 8) / 16 for p < pixels (device arrays).  MMLTTB_EINVAL for NULL
 * pointers or pixels < 0.
 */
int mmlttb_raster_intensity(const uint32_t *mask, int64_t pixels, uint8_t *out,
                            mmlttb_stream stream);

/*
 * The visual metrics of Sec. 4 (PEM_20 and MSE over the conv-mask, as named in the
 * caption of the visual-representativeness figure; DSSIM is not provided).
 * Exact integer counts behind PEM_margin and MSE for a reference image `ref` and an
 * image `img` (device uint8[height * width], row-major):
 *   counts[0] = pixels with |ref - img| > margin,
 *   counts[1] = sum over all pixels of (ref - img)^2,
 *   counts[2] = conv-mask size (pixels with ref > 0 within Chebyshev distance 1).
 * counts is a device int64[3], overwritten.  PEM = counts[0] / counts[2] and MSE =
 * counts[1] / counts[2] (0 for an empty mask) are left to the caller.
 * MMLTTB_EINVAL for NULL pointers, width or height < 1, width*height > 2^31 - 1, or
 * margin < 0.
 */
int mmlttb_visual_counts(const uint8_t *ref, const uint8_t *img, int32_t width, int32_t height,
                         int32_t margin, int64_t *counts, mmlttb_stream stream);

#ifdef __cplusplus
}
#endif

#endif /* MMLTTB_RASTER_H */
