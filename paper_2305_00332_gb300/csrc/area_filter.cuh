// FP32 bounds on the FP64 LTTB triangle area (reading R6), so that an argmax over a
// large bucket needs FP64 only where two candidates come close.
//
// The area the method compares is A(b) = fl|fl(fl(P*fl(yb-ya)) - fl(fl(xa-xb)*R))|
// with P = fl(xa-xc), R = fl(yc-ya), every FP64 operation rounded on its own.  This part
// has about 1.6 FP64 lane operations per cycle and SM against about 76 FP32 adds, and
// FP64 <-> FP32 or int64 -> FP32 conversions run at FP64 speed, so an FP64 area per
// candidate would dominate.  StepBound (below) gives, for every candidate of a bucket,
// an FP32 value |T| formed from values converted with integer operations only, and one
// error bound E for the whole bucket with |A(b) - |T|| <= E; its comment carries the
// error analysis.  Over a bucket, a candidate whose |T| + E is below the largest |T| - E
// has a strictly smaller area than the candidate attaining it: it can neither win nor
// tie.  When only one candidate remains it is the pick; otherwise the FP64 area
// (tri_area) decides among the remaining ones, with the lowest position on ties (R8),
// which is the sequential result.
#pragma once

#include "common.cuh"

namespace mmlttb {
namespace {

constexpr float kFilterU = 5.9604644775390625e-08f;  // 2^-24
constexpr float kFilterAbs = 7.888609052210118e-31f;  // 2^-100

// FP32 value of an int64, exact below 2^22 in magnitude, else truncated (relative
// error below 2^-23).  Integer operations and one FP32 add only.
__device__ __forceinline__ float f32_of_i64(long long d) {
  if (d > -(1ll << 22) && d < (1ll << 22))  // 1.5*2^23 + d holds d exactly in its low bits
    return __fsub_rn(__int_as_float(0x4B400000 + (int)d), 12582912.0f);
  const unsigned long long a = d < 0 ? 0ull - (unsigned long long)d : (unsigned long long)d;
  const int lz = __clzll((long long)a);
  const unsigned mant = (unsigned)((a << lz) >> 40) & 0x7fffffu;  // 23 bits below the leading one
  const unsigned bits = ((unsigned)(63 - lz + 127) << 23) | mant | (d < 0 ? 0x80000000u : 0u);
  return __uint_as_float(bits);
}

// Whether a float is zero or in [2^-60, 2^60) in magnitude.
__device__ __forceinline__ bool f32_in_range(float v) {
  const unsigned b = __float_as_uint(v) & 0x7fffffffu;
  const unsigned e = b >> 23;
  return b == 0u || (e >= 127u - 60u && e < 127u + 60u);
}

// FP64 -> FP32 by truncation of the significand (relative error below 2^-23), with
// integer operations only; *ok turns false outside {0} and [2^-60, 2^60).
__device__ __forceinline__ float f32_of_f64(double v, bool* ok) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  const unsigned sign = (unsigned)(b >> 32) & 0x80000000u;
  const int be = (int)((b >> 52) & 0x7ff);
  if ((b & 0x7fffffffffffffffull) == 0) return __uint_as_float(sign);
  const int e = be - 1023;
  if (be == 0 || e < -60 || e >= 60) {  // subnormal, tiny, huge, inf or NaN
    *ok = false;
    return 0.0f;
  }
  return __uint_as_float(sign | ((unsigned)(e + 127) << 23) | (unsigned)((b >> 29) & 0x7fffffu));
}

// int64 value of an integer-valued double below 2^63 in magnitude (exact; integer
// operations only).
__device__ __forceinline__ long long i64_of_f64_int(double v) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  const int be = (int)((b >> 52) & 0x7ff);
  if (be < 1023) return 0;  // |v| < 1: an integer-valued double is 0
  const unsigned long long sig = (b & 0xfffffffffffffull) | (1ull << 52);
  const int sh = be - 1075;
  const unsigned long long a = sh >= 0 ? sig << sh : sig >> (-sh);
  return (b >> 63) ? -(long long)a : (long long)a;
}

// A bucket mean as the FP32 filter uses it, with error bounds against the FP64 mean
// (xc, yc) the method forms (R7): |xint + xfrac - xc| <= ex and |y32 - yc| <= ey, xfrac
// in [0, 1) (NaN, or y32 NaN, when the filter cannot take this mean).  Only integer x
// (implicit or int64) is filtered.
struct MeanF {
  long long xint;
  float xfrac, y32, ex, ey;
};

// Whether |v| < 2^k for a double (integer test of the exponent field; false for inf
// and NaN), k in [-1022, 1023].
__device__ __forceinline__ bool f64_below_pow2(double v, int k) {
  const int be = (int)(((unsigned long long)__double_as_longlong(v) >> 52) & 0x7ff);
  return be < 1023 + k;
}

// The split form of an FP64 mean with integer operations: xint = floor(v), and the
// fraction v - xint in [0, 1) as FP32 with an absolute error below 2^-22 (truncated
// significand bits, and for negative v one FP32 subtraction from 1).  *ok turns false
// unless |v| < 2^52.
__device__ __forceinline__ void split_floor(double v, long long* xint, float* xfrac, bool* ok) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  const int e = (int)((b >> 52) & 0x7ff) - 1023;
  const bool neg = (b >> 63) != 0;
  if (e >= 52) {  // integer-valued, or beyond the filter's range
    *ok = false;
    *xint = 0;
    *xfrac = 0.0f;
    return;
  }
  const unsigned long long m = (b & 0xfffffffffffffull) | (1ull << 52);
  unsigned long long ip, fb;
  int fe;  // fraction = fb * 2^fe
  if (e < 0) {
    ip = 0;
    fb = (b & 0x7fffffffffffffffull) ? m : 0;  // |v| < 1 (zero or subnormal: fraction |v|)
    fe = (e < -1022 ? -1022 : e) - 52;
    if (((b >> 52) & 0x7ff) == 0) fb = b & 0xfffffffffffffull;
  } else {
    ip = m >> (52 - e);
    fb = m & ((1ull << (52 - e)) - 1);
    fe = e - 52;
  }
  // fb * 2^fe in FP32: truncate fb, scale by a power of two (exact unless far below 2^-126)
  float f = f32_of_i64((long long)fb);
  const int se = fe < -126 ? -126 : fe;
  f = __fmul_rn(f, __uint_as_float((unsigned)(se + 127) << 23));
  if (fe < -126) f = 0.0f;  // below 2^-126: the fraction's error stays below 2^-100
  if (!neg) {
    *xint = (long long)ip;
    *xfrac = f;
  } else {
    *xint = -(long long)ip - (fb ? 1 : 0);
    *xfrac = fb ? __fsub_rn(1.0f, f) : 0.0f;
  }
}

// FP32 truncation of a double known to be below 2^60 in magnitude; values below 2^-60
// become 0 (absolute error below 2^-60).  Monotone non-decreasing.
__device__ __forceinline__ float f32_trunc(double v) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  const int e = (int)((b >> 52) & 0x7ff) - 1023;
  const unsigned sign = (unsigned)(b >> 32) & 0x80000000u;
  if (e < -60) return __uint_as_float(sign);
  return __uint_as_float(sign | ((unsigned)(e + 127) << 23) | (unsigned)((b >> 29) & 0x7fffffu));
}

// Per-bucket statistics for the step bound below: the smallest and largest y of the
// bucket as the filter sees them (float32 y exactly, float64 y truncated by f32_trunc,
// which is monotone, so every candidate's FP32 y lies between them; NaN when a value is
// NaN or not below 2^60 in magnitude), and the x span x_last - x_first (exact integer;
// for implicit x the position span), and its first x (the origin of the step bound).
struct BucketF {
  float ymin, ymax;
  long long xspan, x0;
};

// One error bound for every candidate of a bucket (a step of a long chain).  With the
// bucket's first x as origin (xb' = xb - x0, xa' = xa - x0, exact integers):
//   area expression  P (yb - ya) + R (xb - xa) = P dy + R xb' + K0,  K0 = -R xa'
//   per candidate    T = fma(P32, fl32(yb32 - ya32), fma(R32, xb'32, K32)),
//                    K32 = -fl32(R32 xa'32)
// and |A(b) - |T|| <= E for every candidate of the bucket, with
//   Dm = max(ymax - ya32, ya32 - ymin)             (bounds |yb32 - ya32|)
//   Xm = X' + |xa'32|                                (bounds |xb - xa|, X' the x span)
//   tY = 2^-22 (max(|ymin|, |ymax|) + |ya32|) for truncated float64 y, else 0
//   M  = (|P32|+eP)(Dm + tY) + (|R32|+eR) Xm
//   E  = (10u + rho) M + 1.02 (eP (Dm + tY) + eR Xm) + (|P32|+eP)(tY + 2^-59) + 2^-100
// The terms: the FP32 roundings of dy, the two FMAs and K32, each at most u M (10u
// leaves room for the FP64 roundings of A, 3.01 2^-53 M); x differences truncated
// beyond 2^22 (rho = 2^-22, on both xb' and xa'); the errors eP, eR of P32, R32 (below);
// truncation of float64 y (tY) and float64 y below 2^-60 taken
// as 0 (2^-59 for yb and ya); subnormal results (2^-100).  The step is unfiltered unless
// P32, R32, the bucket's y range, X' and the pick's values are below 2^60, so M stays far
// from overflow.  Ordering a bucket's candidates by |T| orders their upper bounds.
// P32 = fl32(f32(xa - xint) - xfrac) and R32 = fl32(yc32 - ya32) (the mean c in the
// split form of MeanF) carry absolute error bounds against the FP64 values P, R:
//   eP = 2^-22 |f32(xa - xint)| + 2^-23 |P32| + ex   (truncation of the integer
//        difference; rounding of the subtraction and FP64 rounding of P; the mean's x)
//   eR = ey + tau' |ya32| + 2^-23 |R32|                (the mean's y; truncation of the
//        pick's y, tau' = 2^-22 for float64 y and 0 for float32; the two roundings)
struct StepBound {
  float P32, R32, K32, ya32, E;
  bool ok;

  __device__ __forceinline__ void init(long long xa, float ya, long long x0, const MeanF& c, const BucketF& bk,
                                       bool y_trunc) {
    init_span(xa, ya, x0, c, bk.ymin, bk.ymax, f32_of_i64(bk.xspan), y_trunc);
  }
  // the same with the bucket's y range and FP32 x span (f32_of_i64 of the span) given
  __device__ __forceinline__ void init_span(long long xa, float ya, long long x0, const MeanF& c, float ymin,
                                            float ymax, float xs, bool y_trunc) {
    const float big = 1.152921504606847e18f;  // 2^60
    const float d32 = f32_of_i64(xa - c.xint);
    P32 = __fsub_rn(d32, c.xfrac);
    R32 = __fsub_rn(c.y32, ya);
    ya32 = ya;
    const float xa32 = f32_of_i64(xa - x0);
    const float aP = fabsf(P32), aR = fabsf(R32);
    ok = fabsf(ya) < big && fabsf(c.y32) < big && fabsf(d32) < big && aP < big && aR < big &&
         fabsf(ymin) < big && fabsf(ymax) < big && fabsf(xa32) < big && xs < big && c.xfrac >= 0.0f &&
         c.xfrac < 1.0f && c.ex < 1.0f && c.ey < big;
    K32 = -__fmul_rn(R32, xa32);
    const float eP = __fmaf_ru(4.0f * kFilterU, fabsf(d32), __fmaf_ru(2.0f * kFilterU, aP, c.ex));
    const float eR = __fmaf_ru(y_trunc ? 4.0f * kFilterU : 0.0f, fabsf(ya), __fmaf_ru(2.0f * kFilterU, aR, c.ey));
    const float dm = fmaxf(__fsub_ru(ymax, ya), __fsub_ru(ya, ymin));
    const float tY = y_trunc ? __fmul_ru(4.0f * kFilterU, __fadd_ru(fmaxf(fabsf(ymin), fabsf(ymax)), fabsf(ya)))
                             : 0.0f;
    const float xm = __fadd_ru(xs, fabsf(xa32));
    const float pP = __fadd_ru(aP, eP), pR = __fadd_ru(aR, eR);
    const float dmt = __fadd_ru(dm, tY);
    const float M = __fmaf_ru(pP, dmt, __fmul_ru(pR, xm));
    float e = __fmul_ru(14.0f * kFilterU, M);
    e = __fmaf_ru(1.02f, __fmaf_ru(eP, dmt, __fmul_ru(eR, xm)), e);
    e = __fmaf_ru(pP, __fadd_ru(tY, 1.7347234759768071e-18f), e);  // 2^-59
    E = __fadd_ru(e, kFilterAbs);
    ok = ok && E < 3.0e38f;
  }
  // |T| of a candidate (see above)
  __device__ __forceinline__ float t_abs(float yb, float xb_rel) const {
    return fabsf(__fmaf_rn(P32, __fsub_rn(yb, ya32), __fmaf_rn(R32, xb_rel, K32)));
  }
};

// The x of position p as an exact integer for the filter (implicit x: the index).
__device__ __forceinline__ long long filter_x(const SeriesPlan& sp, int64_t p) {
  if (sp.xk == MMLTTB_X_IMPLICIT) return sp.sel ? sp.sel[p] : p;
  if (sp.xk == MMLTTB_X_I64) return sp.px ? i64_of_f64_int(sp.px[p]) : __ldg((const long long*)sp.x + p);
  return 0;  // float64 x is not filtered
}

// The y of position p as the chain's FP32 filter sees it (float32 exactly, float64
// truncated), with a flag for values the filter cannot take (NaN, beyond 2^60).
__device__ __forceinline__ float filter_y(const SeriesPlan& sp, int64_t p, bool* ok) {
  if (!sp.py && sp.ydt == MMLTTB_F32) {
    const float v = __ldg((const float*)sp.y + p);
    *ok = *ok && fabsf(v) < 1.152921504606847e18f;
    return v;
  }
  const double v = sp.py ? __ldg(sp.py + p) : __ldg((const double*)sp.y + p);
  *ok = *ok && f64_below_pow2(v, 60);
  return f32_trunc(v);
}

// The filter form of the FP64 mean (xc, yc) of positions [lo, hi) (R7), without an
// FP64 instruction.  With integer x below 2^45 and at most 255 positions, every
// partial FP64 x sum is an integer below 2^53, so the FP64 sum is the exact integer
// sum S and xc = fl64(S/n): xint = floor(S/n) by integer division, xfrac = fl32(r/n)
// with r = S - n*xint, and ex = 2^-24 (the fraction) + 2^-53 |xc|.  The y sum runs
// left to right in FP32 over the filter's y (float32 exact, float64 truncated with
// relative error tau < 2^-23); against the FP64 mean, with A = max |y|:
//   |fl32 sum - sum of filter y| <= gamma32(n-1) n A,  |that - exact sum| <= tau n A,
//   |exact sum - FP64 sum| <= gamma64(n-1) n A,  and the two divisions contribute
//   2^-24 |y32| and 2^-53 |yc|,
// so ey = 2^-24 |y32| + (n 2^-24 + tau + 2^-44)(1 + 2^-10) A' covers them (A' the largest
// |filter y|; gamma(k) = k u / (1 - k u); the last factor covers A <= A' (1 + 2^-22)
// and gamma's denominator).  False when the filter cannot take the mean.
__device__ __forceinline__ bool mean_filter_form(const SeriesPlan& sp, int64_t lo, int64_t hi, MeanF* c) {
  const long long n = hi - lo;
  if (sp.xk == MMLTTB_X_F64 || n <= 0 || n > 255) return false;
  bool ok = true;
  unsigned long long sx = 0, xmax = 0;  // two's complement sum: exact once |x| < 2^45 is known
  float sy = 0.0f, amax = 0.0f;
  for (int64_t p = lo; p < hi; ++p) {
    const long long x = filter_x(sp, p);
    const unsigned long long ax = x < 0 ? 0ull - (unsigned long long)x : (unsigned long long)x;
    xmax = ax > xmax ? ax : xmax;
    sx += (unsigned long long)x;
    const float v = filter_y(sp, p, &ok);
    amax = fmaxf(amax, fabsf(v));
    sy = __fadd_rn(sy, v);
  }
  if (!ok || xmax >= (1ull << 45)) return false;
  const long long S = (long long)sx;
  long long q, r;
  if (S > -(1ll << 31) && S < (1ll << 31)) {
    const int q32 = (int)S / (int)n;
    q = q32;
    r = S - q * n;
  } else {
    q = S / n;
    r = S - q * n;
  }
  if (r < 0) {
    q -= 1;
    r += n;
  }
  c->xint = q;
  c->xfrac = __fdiv_rn((float)(int)r, (float)(int)n);  // r/n <= 254/255: below 1 after rounding
  const unsigned long long aq = q < 0 ? 0ull - (unsigned long long)q : (unsigned long long)q;
  c->ex = __fmaf_ru(2.220446049250313e-16f, f32_of_i64((long long)aq), 2.0f * kFilterU);  // 2^-52
  c->y32 = __fdiv_rn(sy, (float)(int)n);
  const float tau = sp.ydt != MMLTTB_F32 ? 4.0f * kFilterU : 0.0f;
  const float cn = __fmul_ru(__fmaf_ru((float)(int)n, kFilterU, __fadd_ru(tau, 5.684341886080802e-14f)),  // 2^-44
                             1.0009765625f);
  c->ey = __fmaf_ru(cn, amax, __fmul_ru(kFilterU, fabsf(c->y32)));
  return true;
}

}  // namespace
}  // namespace mmlttb
