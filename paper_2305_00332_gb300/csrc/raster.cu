// Headless line-chart rasterisation and the visual metrics (Sec. 4: downsampled
// charts are compared with the chart of all points by PEM_20 and MSE; the figure on
// visual representativeness: linearly interpolated, 2-pixel-wide anti-aliased lines).
//
//  k_raster         a warp per segment, or per 31 consecutive segments when there are
//                   many.  Lanes map the points to canvas coordinates (FP64, then
//                   float32), once per point.  When the union of the group's pixel
//                   boxes is small (dense charts) its masks are read once and each
//                   segment tests only the open pixels of its box; otherwise each box
//                   is read 32 masks at a time.  Pixels are tested two per step: each
//                   half-warp tests the 16 samples of one pixel (one sample per lane,
//                   float32 with every operation rounded on its own), and one ballot
//                   yields both pixels' sample masks, OR-ed into the canvas.
//  k_intensity      16ths of ink -> 8-bit intensity, one thread per pixel.
//  k_visual_counts  per pixel |ref - img| > margin, (ref - img)^2 and whether the
//                   3 x 3 neighbourhood of the reference holds ink; block sums, one
//                   64-bit atomic add per block and count (integers: exact, order-free).
#include <limits.h>

#include <algorithm>
#include <cmath>

#include "host.h"
#include "mmlttb_raster.h"

namespace mmlttb {

namespace {

struct RasterArgs {
  const void* y;
  const void* x;
  const int64_t* idx;  // drawn points (NULL: all n)
  int64_t n;
  int64_t segments;  // drawn points - 1
  double x0, x1, y0, y1;
  uint32_t* mask;
  int32_t W, H;
  int32_t ydt, xk;
  int32_t group;  // consecutive segments per warp step: 1, or 31 for many segments
};

// Canvas coordinates of drawn point p: px = (x - x0) * (W / (x1 - x0)),
// py = (y1 - y) * (H / (y1 - y0)), each FP64 operation rounded on its own, then
// rounded to float32; a zero extent maps to the middle.  NaN for an index outside
// [0, n) (such a point draws nothing).  sx, sy are the scales of canvas_scale, zx, zy
// whether the extent is zero.
__device__ __forceinline__ void canvas_point(const RasterArgs& a, int64_t p, double sx, double sy, bool zx,
                                             bool zy, float* cx, float* cy) {
  const int64_t i = a.idx ? __ldg(a.idx + p) : p;
  if (i < 0 || i >= a.n) {
    *cx = *cy = __int_as_float(0x7fc00000);
    return;
  }
  double xv;
  if (a.xk == MMLTTB_X_I64)
    xv = __ll2double_rn(__ldg((const long long*)a.x + i));
  else if (a.xk == MMLTTB_X_F64)
    xv = __ldg((const double*)a.x + i);
  else
    xv = __ll2double_rn(i);
  const double yv = a.ydt == MMLTTB_F64 ? __ldg((const double*)a.y + i) : (double)__ldg((const float*)a.y + i);
  *cx = zx ? __double2float_rn(0.5 * (double)a.W) : __double2float_rn(__dmul_rn(__dsub_rn(xv, a.x0), sx));
  *cy = zy ? __double2float_rn(0.5 * (double)a.H) : __double2float_rn(__dmul_rn(__dsub_rn(a.y1, yv), sy));
}

// size / (hi - lo) in FP64; *zero tells a zero extent (mapped to the middle).
__device__ __forceinline__ double canvas_scale(double lo, double hi, int size, bool* zero) {
  const double d = __dsub_rn(hi, lo);
  *zero = d == 0.0;
  return *zero ? 0.0 : __ddiv_rn((double)size, d);
}

// Whether sample (sx, sy) is within distance 1 of the segment from (ax, ay) along
// (dx, dy) with squared length len2: float32, every operation rounded on its own.
__device__ __forceinline__ bool sample_inked(float sx, float sy, float ax, float ay, float dx, float dy,
                                             float len2) {
  float t = 0.0f;
  if (len2 > 0.0f) {
    const float num = __fadd_rn(__fmul_rn(__fsub_rn(sx, ax), dx), __fmul_rn(__fsub_rn(sy, ay), dy));
    t = __fdiv_rn(num, len2);
    if (t < 0.0f) t = 0.0f;
    if (t > 1.0f) t = 1.0f;
  }
  const float ex = __fsub_rn(sx, __fadd_rn(ax, __fmul_rn(t, dx)));
  const float ey = __fsub_rn(sy, __fadd_rn(ay, __fmul_rn(t, dy)));
  return __fadd_rn(__fmul_rn(ex, ex), __fmul_rn(ey, ey)) <= 1.0f;
}

// floor(v) for a non-NaN v, after clamping v to [-4, lim + 4]; the pixel box clipped
// to [0, lim - 1] is the same as with the unclamped floor.
__device__ __forceinline__ int floor_clamped(float v, int lim) {
  return (int)floorf(fminf(fmaxf(v, -4.0f), (float)lim + 4.0f));
}

// The pixel box of segment A-B (R: [floor(min) - 1, floor(max) + 1] on both axes),
// clipped to the canvas; false when it is empty or an endpoint is NaN (such a segment
// inks nothing).
__device__ __forceinline__ bool segment_box(const RasterArgs& a, float ax, float ay, float bx, float by, int* c0,
                                            int* c1, int* r0, int* r1) {
  if (isnan(ax) || isnan(ay) || isnan(bx) || isnan(by)) return false;
  const float lox = ax < bx ? ax : bx, hix = ax < bx ? bx : ax;
  const float loy = ay < by ? ay : by, hiy = ay < by ? by : ay;
  *c0 = max(floor_clamped(lox, a.W) - 1, 0);
  *c1 = min(floor_clamped(hix, a.W) + 1, a.W - 1);
  *r0 = max(floor_clamped(loy, a.H) - 1, 0);
  *r1 = min(floor_clamped(hiy, a.H) + 1, a.H - 1);
  return *c0 <= *c1 && *r0 <= *r1;
}

// Test and ink the pixels of `todo` against segment A + t*(dx, dy): bit p is pixel p
// of a listing whose (row << 16 | column) offsets from (r0, c0) lane p holds in rcA
// (p < 32) or lane p - 32 in rcB.  Two pixels per step, one per half-warp, one sample
// per lane; one ballot gives both pixels' masks, OR-ed into the canvas.
__device__ __forceinline__ void ink_pixels(const RasterArgs& a, unsigned long long todo, unsigned rcA,
                                           unsigned rcB, int r0, int c0, float ax, float ay, float dx, float dy,
                                           float len2, int half, int s, float offx, float offy) {
  while (todo) {
    const int first = __ffsll(todo) - 1;
    todo &= todo - 1;
    const int second = todo ? __ffsll(todo) - 1 : -1;
    if (todo) todo &= todo - 1;
    const int mine = half ? second : first;
    const int src = mine < 0 ? 0 : (mine & 31);
    const unsigned pa = __shfl_sync(kFull, rcA, src), pb = __shfl_sync(kFull, rcB, src);
    const unsigned prc = mine >= 32 ? pb : pa;
    const int pr = r0 + (int)(prc >> 16), pc = c0 + (int)(prc & 0xffffu);
    bool ink = false;
    if (mine >= 0) ink = sample_inked(__fadd_rn((float)pc, offx), __fadd_rn((float)pr, offy), ax, ay, dx, dy, len2);
    const unsigned b = __ballot_sync(kFull, ink);
    if (s == 0 && mine >= 0) {
      const unsigned m = half ? b >> 16 : b & 0xffffu;
      if (m) atomicOr(a.mask + (int64_t)pr * a.W + pc, m);
    }
  }
}

// Whether the canvas pixel (r, c) is not fully inked yet.  Masks only grow, so a stale
// read only costs a test that was not needed.
__device__ __forceinline__ bool pixel_open(const RasterArgs& a, int r, int c) {
  return (__ldcg(a.mask + (int64_t)r * a.W + c) & 0xffffu) != 0xffffu;
}

constexpr int kRasterThreads = 256;
constexpr int kUnionPixels = 64;  // the union box of a warp's segments is read at once up to this size

__global__ void __launch_bounds__(kRasterThreads) k_raster(const __grid_constant__ RasterArgs a) {
  const int lane = threadIdx.x & 31;
  const int half = lane >> 4, s = lane & 15;
  // this lane's sample within its pixel: bit s = k*4 + i at (i + 0.5)/4, (k + 0.5)/4
  const float offx = 0.25f * (float)(s & 3) + 0.125f, offy = 0.25f * (float)(s >> 2) + 0.125f;
  bool zx, zy;
  const double sx = canvas_scale(a.x0, a.x1, a.W, &zx), sy = canvas_scale(a.y0, a.y1, a.H, &zy);
  const int64_t warps = (int64_t)gridDim.x * (kRasterThreads / 32);
  const int G = a.group;
  for (int64_t base = (((int64_t)blockIdx.x * kRasterThreads + threadIdx.x) >> 5) * G; base < a.segments;
       base += warps * G) {
    // lanes 0..G map the group's G + 1 points, once each (the FP64 pipe is narrow);
    // lane j < gn holds segment j (its point and the next lane's)
    float cx = 0.0f, cy = 0.0f;
    if (lane <= G && base + lane <= a.segments) canvas_point(a, base + lane, sx, sy, zx, zy, &cx, &cy);
    const int gn = (int)min((int64_t)G, a.segments - base);
    const float nx = __shfl_down_sync(kFull, cx, 1), ny = __shfl_down_sync(kFull, cy, 1);
    int sc0 = 0, sc1 = -1, sr0 = 0, sr1 = -1;
    const bool sv = lane < gn && segment_box(a, cx, cy, nx, ny, &sc0, &sc1, &sr0, &sr1);
    const unsigned live = __ballot_sync(kFull, sv);
    if (!live) continue;
    // the union of the segments' boxes
    const int uc0 = __reduce_min_sync(kFull, sv ? sc0 : INT_MAX), uc1 = __reduce_max_sync(kFull, sv ? sc1 : -1);
    const int ur0 = __reduce_min_sync(kFull, sv ? sr0 : INT_MAX), ur1 = __reduce_max_sync(kFull, sv ? sr1 : -1);
    const int uw = uc1 - uc0 + 1, uh = ur1 - ur0 + 1;
    if (uw <= kUnionPixels && uh <= kUnionPixels && uw * uh <= kUnionPixels) {
      // Small union (dense charts): read its masks once; a segment only tests the open
      // pixels of its own box, and a group whose union is fully inked costs one read.
      const int unp = uw * uh;
      const int pA = lane, pB = lane + 32;
      const int rowA = pA / uw, colA = pA - rowA * uw, rowB = pB / uw, colB = pB - rowB * uw;
      const unsigned rcA = ((unsigned)rowA << 16) | (unsigned)colA, rcB = ((unsigned)rowB << 16) | (unsigned)colB;
      const bool okA = pA < unp, okB = pB < unp;
      const bool openA = okA && pixel_open(a, ur0 + rowA, uc0 + colA);
      const bool openB = okB && pixel_open(a, ur0 + rowB, uc0 + colB);
      const unsigned long long open =
          (unsigned long long)__ballot_sync(kFull, openA) | ((unsigned long long)__ballot_sync(kFull, openB) << 32);
      if (!open) continue;
      for (unsigned segs = live; segs; segs &= segs - 1) {
        const int j = __ffs(segs) - 1;
        const int c0 = __shfl_sync(kFull, sc0, j), c1 = __shfl_sync(kFull, sc1, j);
        const int r0 = __shfl_sync(kFull, sr0, j), r1 = __shfl_sync(kFull, sr1, j);
        const bool inA = okA && uc0 + colA >= c0 && uc0 + colA <= c1 && ur0 + rowA >= r0 && ur0 + rowA <= r1;
        const bool inB = okB && uc0 + colB >= c0 && uc0 + colB <= c1 && ur0 + rowB >= r0 && ur0 + rowB <= r1;
        const unsigned long long todo =
            open & ((unsigned long long)__ballot_sync(kFull, inA) | ((unsigned long long)__ballot_sync(kFull, inB) << 32));
        if (!todo) continue;
        const float ax = __shfl_sync(kFull, cx, j), ay = __shfl_sync(kFull, cy, j);
        const float bx = __shfl_sync(kFull, nx, j), by = __shfl_sync(kFull, ny, j);
        const float dx = __fsub_rn(bx, ax), dy = __fsub_rn(by, ay);
        const float len2 = __fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy));
        ink_pixels(a, todo, rcA, rcB, ur0, uc0, ax, ay, dx, dy, len2, half, s, offx, offy);
      }
      continue;
    }
    // Large union: segment by segment, each box in chunks of 32 pixels whose open
    // pixels are tested.
    for (unsigned segs = live; segs; segs &= segs - 1) {
      const int j = __ffs(segs) - 1;
      const int c0 = __shfl_sync(kFull, sc0, j), c1 = __shfl_sync(kFull, sc1, j);
      const int r0 = __shfl_sync(kFull, sr0, j), r1 = __shfl_sync(kFull, sr1, j);
      const float ax = __shfl_sync(kFull, cx, j), ay = __shfl_sync(kFull, cy, j);
      const float bx = __shfl_sync(kFull, nx, j), by = __shfl_sync(kFull, ny, j);
      const float dx = __fsub_rn(bx, ax), dy = __fsub_rn(by, ay);
      const float len2 = __fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy));
      const int w = c1 - c0 + 1;
      const int npix = w * (r1 - r0 + 1);
      for (int q0 = 0; q0 < npix; q0 += 32) {
        const int p = q0 + lane;
        unsigned rc = 0;  // (row << 16) | column within the box
        bool open = false;
        if (p < npix) {
          const int pr = p / w, pc = p - pr * w;
          rc = ((unsigned)pr << 16) | (unsigned)pc;
          open = pixel_open(a, r0 + pr, c0 + pc);
        }
        ink_pixels(a, __ballot_sync(kFull, open), rc, 0u, r0, c0, ax, ay, dx, dy, len2, half, s, offx, offy);
      }
    }
  }
}

__global__ void __launch_bounds__(256) k_intensity(const uint32_t* __restrict__ mask, int64_t pixels,
                                                   uint8_t* __restrict__ out) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < pixels; p += stride) {
    const int inked = __popc(__ldg(mask + p) & 0xffffu);
    out[p] = (uint8_t)((inked * 255 + 8) >> 4);
  }
}

__global__ void __launch_bounds__(256) k_visual_counts(const uint8_t* __restrict__ ref,
                                                       const uint8_t* __restrict__ img, int W, int H,
                                                       int margin, unsigned long long* counts) {
  __shared__ unsigned long long s_part[3][8];
  unsigned long long over = 0, sq = 0, msize = 0;
  const int64_t pixels = (int64_t)W * H, stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < pixels; p += stride) {
    const int r = (int)(p / W), c = (int)(p - (int64_t)r * W);
    int d = (int)__ldg(ref + p) - (int)__ldg(img + p);
    d = d < 0 ? -d : d;
    over += d > margin;
    sq += (unsigned long long)(d * d);
    bool in = false;
    for (int rr = max(r - 1, 0); rr <= min(r + 1, H - 1); ++rr)
      for (int cc = max(c - 1, 0); cc <= min(c + 1, W - 1); ++cc) in |= __ldg(ref + (int64_t)rr * W + cc) > 0;
    msize += in;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    over += __shfl_xor_sync(kFull, over, o);
    sq += __shfl_xor_sync(kFull, sq, o);
    msize += __shfl_xor_sync(kFull, msize, o);
  }
  const int warp = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) {
    s_part[0][warp] = over;
    s_part[1][warp] = sq;
    s_part[2][warp] = msize;
  }
  __syncthreads();
  if (threadIdx.x < 3) {
    unsigned long long t = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += s_part[threadIdx.x][w];
    if (t) atomicAdd(counts + threadIdx.x, t);
  }
}

int64_t grid_for(int64_t work_ctas, int per_sm) {
  DevInfo d;
  const int sms = get_dev_info(&d) == MMLTTB_OK && d.sms > 0 ? d.sms : 152;
  return std::max<int64_t>(1, std::min<int64_t>(work_ctas, (int64_t)sms * per_sm));
}

}  // namespace

}  // namespace mmlttb

using namespace mmlttb;

extern "C" {

int mmlttb_raster(const void* y, int ydtype, const void* x, int xkind, int64_t n_in, const int64_t* idx,
                  int64_t k, double x0, double x1, double y0, double y1, int32_t width, int32_t height,
                  uint32_t* mask, mmlttb_stream stream) {
  if (!y || !mask || n_in < 0) return MMLTTB_EINVAL;
  if (ydtype != MMLTTB_F32 && ydtype != MMLTTB_F64) return MMLTTB_EINVAL;
  if (xkind != MMLTTB_X_IMPLICIT && xkind != MMLTTB_X_I64 && xkind != MMLTTB_X_F64) return MMLTTB_EINVAL;
  if (xkind != MMLTTB_X_IMPLICIT && !x) return MMLTTB_EINVAL;
  if (idx && k < 0) return MMLTTB_EINVAL;
  if (!std::isfinite(x0) || !std::isfinite(x1) || !std::isfinite(y0) || !std::isfinite(y1)) return MMLTTB_EINVAL;
  if (width < 1 || height < 1 || width > MMLTTB_RASTER_MAX_SIDE || height > MMLTTB_RASTER_MAX_SIDE ||
      (int64_t)width * height > (int64_t(1) << 28))
    return MMLTTB_EINVAL;
  const int64_t drawn = idx ? k : n_in;
  if (drawn < 2) return MMLTTB_OK;
  RasterArgs a;
  a.y = y;
  a.x = x;
  a.idx = idx;
  a.n = n_in;
  a.segments = drawn - 1;
  a.x0 = x0;
  a.x1 = x1;
  a.y0 = y0;
  a.y1 = y1;
  a.mask = mask;
  a.W = width;
  a.H = height;
  a.ydt = ydtype;
  a.xk = xkind;
  // Many short segments: a warp takes 31 consecutive ones, so that each point is
  // mapped once by one lane of a full-warp FP64 instruction.  Few (typically long)
  // segments: one per warp, for parallelism.
  DevInfo d;
  const int sms = get_dev_info(&d) == MMLTTB_OK && d.sms > 0 ? d.sms : 152;
  a.group = a.segments >= (int64_t)31 * sms * 16 ? 31 : 1;
  const int64_t warps_needed = (a.segments + a.group - 1) / a.group;
  const int64_t grid = grid_for((warps_needed + kRasterThreads / 32 - 1) / (kRasterThreads / 32), 8);
  k_raster<<<(unsigned)grid, kRasterThreads, 0, (cudaStream_t)stream>>>(a);
  ++g_launches;
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? MMLTTB_OK : cuda_fail(e);
}

int mmlttb_raster_intensity(const uint32_t* mask, int64_t pixels, uint8_t* out, mmlttb_stream stream) {
  if (!mask || !out || pixels < 0) return MMLTTB_EINVAL;
  if (pixels == 0) return MMLTTB_OK;
  const int64_t grid = grid_for((pixels + 255) / 256, 8);
  k_intensity<<<(unsigned)grid, 256, 0, (cudaStream_t)stream>>>(mask, pixels, out);
  ++g_launches;
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? MMLTTB_OK : cuda_fail(e);
}

int mmlttb_visual_counts(const uint8_t* ref, const uint8_t* img, int32_t width, int32_t height,
                         int32_t margin, int64_t* counts, mmlttb_stream stream) {
  if (!ref || !img || !counts || width < 1 || height < 1 || margin < 0 ||
      (int64_t)width * height > INT32_MAX)
    return MMLTTB_EINVAL;
  cudaError_t e = cudaMemsetAsync(counts, 0, 3 * sizeof(int64_t), (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e);
  const int64_t grid = grid_for(((int64_t)width * height + 255) / 256, 8);
  k_visual_counts<<<(unsigned)grid, 256, 0, (cudaStream_t)stream>>>(ref, img, width, height, margin,
                                                                   (unsigned long long*)counts);
  ++g_launches;
  e = cudaGetLastError();
  return e == cudaSuccess ? MMLTTB_OK : cuda_fail(e);
}

}  // extern "C"
