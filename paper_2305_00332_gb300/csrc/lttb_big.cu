// LTTB on large buckets (Sec. 2.2.1 LTTB; plain LTTB on every point, or MinMaxLTTB
// with a large r_ps): two launches.
//
//   k_lttb_means    every next-bucket mean (R5, R7), a warp per bucket over all SMs.
//                   The means do not depend on the picks.  Each sum is the left-to-
//                   right FP64 sum of R7, formed 256 terms at a time: when every
//                   partial sum of a chunk is provably exact (all terms and the
//                   running sum are multiples of 2^q and stay below 2^(53+q)), the
//                   chunk is added as one integer total; otherwise 32 terms at a
//                   time, and only a 32-term piece that can round is added term by
//                   term, in order.  Either way the result is the sequential sum.
//   k_lttb_fix      the chain of picks as a fixpoint over all SMs (cooperative launch):
//                   every bucket's pick is the argmax given the previous bucket's current
//                   pick; passes re-evaluate only buckets whose previous pick changed,
//                   until none does, which is the sequential result (the proof is at
//                   the kernel).  A CTA evaluates a bucket with FP32 bounds on the
//                   areas (area_filter.cuh) and forms FP64 areas only on near ties.
#include <type_traits>

#include "area_filter.cuh"
#include "lttb.cuh"

namespace mmlttb {
namespace {

// ---------------------------------------------------------------- exact sums (R7)

// A term as an exact significand and scale: value = sig * 2^scale, |sig| < 2^53.
// `special` marks terms the integer path cannot carry (inf, NaN, int64 beyond 2^53,
// whose FP64 value is rounded).
struct Term {
  long long sig;
  int scale;
  bool special;
};

__device__ __forceinline__ Term term_of(float v) {
  const unsigned b = __float_as_uint(v);
  const int be = (int)((b >> 23) & 0xffu);
  const long long sig = be ? (long long)((b & 0x7fffffu) | 0x800000u) : (long long)(b & 0x7fffffu);
  return Term{(b >> 31) ? -sig : sig, (be ? be : 1) - 150, be == 0xff};
}
__device__ __forceinline__ Term term_of(double v) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  const int be = (int)((b >> 52) & 0x7ff);
  const unsigned long long m = b & 0xfffffffffffffull;
  const long long sig = be ? (long long)(m | (1ull << 52)) : (long long)m;
  return Term{(b >> 63) ? -sig : sig, (be ? be : 1) - 1075, be == 0x7ff};
}
__device__ __forceinline__ Term term_of(long long v) {
  const bool big = v >= (1ll << 53) || v <= -(1ll << 53);
  return Term{big ? 0 : v, 0, big};
}
// The FP64 value the sequential sum adds (as x_of / y_of form it).
__device__ __forceinline__ double dval(float v) { return (double)v; }
__device__ __forceinline__ double dval(double v) { return v; }
__device__ __forceinline__ double dval(long long v) { return (double)v; }

// Weight of the lowest and of the highest set bit of a nonzero term.
__device__ __forceinline__ int low_bit(const Term& t) {
  const unsigned long long a = t.sig < 0 ? 0ull - (unsigned long long)t.sig : (unsigned long long)t.sig;
  return t.scale + __ffsll((long long)a) - 1;
}
__device__ __forceinline__ int high_bit(const Term& t) {
  const unsigned long long a = t.sig < 0 ? 0ull - (unsigned long long)t.sig : (unsigned long long)t.sig;
  return t.scale + 63 - __clzll((long long)a);
}

// s * 2^q as a double, exactly (|s| < 2^53, q >= -1074), with integer operations.
__device__ __forceinline__ double dbl_scaled(long long s, int q) {
  if (s == 0) return 0.0;
  const unsigned long long sign = s < 0 ? (1ull << 63) : 0ull;
  const unsigned long long a = s < 0 ? 0ull - (unsigned long long)s : (unsigned long long)s;
  const int top = 63 - __clzll((long long)a);
  const int E = top + q;
  unsigned long long bits;
  if (E >= -1022)
    bits = sign | ((unsigned long long)(E + 1023) << 52) | ((a << (52 - top)) & 0xfffffffffffffull);
  else
    bits = sign | (a << (q + 1074));  // subnormal: a multiple of 2^-1074 below 2^-1022
  return __longlong_as_double((long long)bits);
}

__device__ __forceinline__ long long warp_sum_i64(long long v) {
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(kFull, v, d);
  return v;
}

// Add the terms t[0..cnt) of every lane (all valid terms, positions in order inside
// the chunk do not matter) to S exactly, if every partial sum in every order is
// representable: terms and S multiples of 2^q, |S| < 2^(52+q) and the terms' total
// magnitude below 2^(52+q) (at most 2^lg terms, each below 2^(e+1)).  Warp-uniform.
template <int CNT>
__device__ __forceinline__ bool try_exact_add(double* S, const Term (&t)[CNT], const bool (&in)[CNT], int lg) {
  int g = INT_MAX, e = INT_MIN;
  bool sp = false;
#pragma unroll
  for (int i = 0; i < CNT; ++i) {
    if (!in[i]) continue;
    sp |= t[i].special;
    if (t[i].sig != 0 && !t[i].special) {
      g = min(g, low_bit(t[i]));
      e = max(e, high_bit(t[i]));
    }
  }
  g = __reduce_min_sync(kFull, g);
  e = __reduce_max_sync(kFull, e);
  if (__any_sync(kFull, sp)) return false;
  if (g == INT_MAX) return true;  // every term is zero: S is unchanged (S is never -0)
  int q = g, eS = INT_MIN;
  if (*S != 0.0) {
    const Term ts = term_of(*S);
    q = min(q, low_bit(ts));
    eS = high_bit(ts);
  }
  if (eS != INT_MIN && (eS + 1 > 52 + q || eS + 2 > 1020)) return false;
  if (e + 1 + lg > 52 + q || e + 1 + lg > 1020) return false;
  long long s = 0;
#pragma unroll
  for (int i = 0; i < CNT; ++i) {
    if (!in[i] || t[i].sig == 0) continue;
    const int sh = t[i].scale - q;  // >= -(trailing zeros of sig): the shift drops only zeros
    s += sh >= 0 ? (t[i].sig << sh) : (t[i].sig >> (-sh));
  }
  s = warp_sum_i64(s);
  *S = __dadd_rn(*S, dbl_scaled(s, q));  // exact: the total is representable
  return true;
}

// ---- 128-bit exact prefix sums (a row of 32 terms that may round somewhere)

using i128 = __int128;
using u128 = unsigned __int128;

__device__ __forceinline__ i128 shfl_up_i128(i128 v, int d) {
  const unsigned long long lo = (unsigned long long)v, hi = (unsigned long long)((u128)v >> 64);
  const unsigned long long olo = __shfl_up_sync(kFull, lo, d), ohi = __shfl_up_sync(kFull, hi, d);
  return (i128)(((u128)ohi << 64) | olo);
}
__device__ __forceinline__ i128 shfl_i128(i128 v, int src) {
  const unsigned long long lo = (unsigned long long)v, hi = (unsigned long long)((u128)v >> 64);
  const unsigned long long olo = __shfl_sync(kFull, lo, src), ohi = __shfl_sync(kFull, hi, src);
  return (i128)(((u128)ohi << 64) | olo);
}
__device__ __forceinline__ int bitlen_u128(u128 a) {
  const unsigned long long hi = (unsigned long long)(a >> 64), lo = (unsigned long long)a;
  return hi ? 128 - __clzll((long long)hi) : (lo ? 64 - __clzll((long long)lo) : 0);
}
__device__ __forceinline__ int ctz_u128(u128 a) {
  const unsigned long long lo = (unsigned long long)a, hi = (unsigned long long)(a >> 64);
  return lo ? __ffsll((long long)lo) - 1 : 64 + __ffsll((long long)hi) - 1;
}
// A term (or a double) as an integer in units of 2^q (q at most its lowest set bit).
__device__ __forceinline__ i128 units_of(const Term& t, int q) {
  if (t.sig == 0) return 0;
  const int sh = t.scale - q;
  return sh >= 0 ? (i128)t.sig << sh : (i128)(t.sig >> (-sh));
}
// Whether v * 2^q is a double (|v| * 2^q below 2^1024; q >= -1074).
__device__ __forceinline__ bool representable(i128 v, int q) {
  if (v == 0) return true;
  const u128 a = v < 0 ? (u128)(-v) : (u128)v;
  const int b = bitlen_u128(a), E = q + b - 1;
  if (E > 1023) return false;
  if (E < -1022) return true;  // subnormal range: every multiple of 2^-1074 is a double
  return b - ctz_u128(a) <= 53;
}
// v * 2^q rounded to the nearest double, ties to even (the rounding of an FP64 add).
__device__ __forceinline__ double round_units(i128 v, int q) {
  if (v == 0) return 0.0;
  const bool neg = v < 0;
  const u128 a = neg ? (u128)(-v) : (u128)v;
  const int b = bitlen_u128(a);
  int d = b - 53;
  if (-1074 - q > d) d = -1074 - q;
  if (d < 0) d = 0;
  u128 mm = d ? a >> d : a;
  if (d) {
    const u128 rem = a & (((u128)1 << d) - 1), half = (u128)1 << (d - 1);
    if (rem > half || (rem == half && (mm & 1))) mm += 1;
  }
  long long m = (long long)mm;
  int e = q + d;
  if (m == (1ll << 53)) {
    m >>= 1;
    e += 1;
  }
  if (e + 52 > 1023) return neg ? -INFINITY : INFINITY;
  const double r = dbl_scaled(m, e);
  return neg ? -r : r;
}

// Add a 32-term row (lane l holds the term at index c + l, in index order) to S exactly
// as the left-to-right FP64 sum does (R7): the partial sums are formed exactly in 128-bit
// integers (a warp scan), and at the first partial sum that is not a double it is rounded
// and the rest continue from there; a row costs one pass plus one per rounding.  Returns
// false when the terms and S do not fit 128-bit units (the caller adds term by term).
__device__ __noinline__ bool row_add_exact(double* S, const Term& t, bool in, int lane) {
  int g = (in && t.sig != 0 && !t.special) ? low_bit(t) : INT_MAX;
  int e = (in && t.sig != 0 && !t.special) ? high_bit(t) : INT_MIN;
  if (__any_sync(kFull, in && t.special)) return false;
  g = __reduce_min_sync(kFull, g);
  e = __reduce_max_sync(kFull, e);
  if (g == INT_MAX) return true;  // every term is zero
  int q = g, eS = INT_MIN;
  Term ts{0, 0, false};
  if (*S != 0.0) {
    ts = term_of(*S);
    q = min(q, low_bit(ts));
    eS = high_bit(ts);
  }
  if (max(e, eS) + 8 - q > 125) return false;  // partial sums below 2^(max + 7) in 2^q units
  i128 P = in ? units_of(t, q) : 0;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const i128 o = shfl_up_i128(P, d);
    if (lane >= d) P += o;
  }
  const i128 T = units_of(ts, q) + P;
  i128 delta = 0;
  int done = -1;  // lanes up to here are final
  for (;;) {
    const bool bad = in && lane > done && !representable(T + delta, q);
    const unsigned mask = __ballot_sync(kFull, bad);
    if (!mask) break;
    const int k = __ffs(mask) - 1;
    const i128 Tk = shfl_i128(T + delta, k);
    const double r = round_units(Tk, q);  // the FP64 add at term k rounds here
    if (!isfinite(r)) return false;       // overflow: let the term-by-term sum produce it
    delta += units_of(term_of(r), q) - Tk;
    done = k;
  }
  *S = round_units(shfl_i128(T + delta, 31), q);  // exact: a double by construction
  return true;
}

// The rows of a 256-term chunk that may round (out of line: rare).  Each row: first
// the cheap exactness test, then the 128-bit prefix (row_add_exact), and beyond 128-bit
// units the terms one by one in index order.
// dv[i]: the FP64 value of the lane's term in row i (exact: float32, float64, or an
// int64 below 2^53 in magnitude); special[i]: a term the integer paths cannot carry.
__device__ __noinline__ void chunk_rows(double* S, const double* dv, const bool* special, int64_t c, int64_t hi,
                                        int lane) {
  for (int i = 0; i < 8; ++i) {
    if (c + 32 * i >= hi) break;
    Term t = term_of(dv[i]);
    t.special = t.special || special[i];
    const bool in = c + 32 * i + lane < hi;
    Term ti[1] = {t};
    bool ini[1] = {in};
    if (try_exact_add<1>(S, ti, ini, 5)) continue;
    if (row_add_exact(S, t, in, lane)) continue;
    for (int k = 0; k < 32 && c + 32 * i + k < hi; ++k) *S = __dadd_rn(*S, __shfl_sync(kFull, dv[i], k));
  }
}

// try_exact_add for a 256-term chunk of float or double terms (lane l holds v[i] at
// c + 32i + l; `full`: all 256 exist), from magnitudes only: the smallest nonzero |v|
// has the smallest exponent, whose significand scale qs (biased exponent - 150 for
// float, - 1075 for double; a multiple of 2^qs for every term, possibly finer than the
// lowest set bit, which only makes the test stricter) is a unit of every term, and
// the largest |v| bounds the magnitudes.  The integer total shifts each significand by
// its scale - q.  Also returns the chunk's signed y range for the bucket statistics.
template <class T>
__device__ __forceinline__ bool try_exact_chunk_fp(double* S, const T (&v)[8], int64_t c, int64_t hi, int lane,
                                                   bool full, T* vmin, T* vmax) {
  constexpr bool F = sizeof(T) == 4;
  constexpr int kBias = F ? 150 : 1075, kTop = F ? 23 : 52, kExpMask = F ? 0xff : 0x7ff;
  using U = typename std::conditional<F, unsigned, unsigned long long>::type;
  constexpr U kAbs = F ? (U)0x7fffffffu : (U)0x7fffffffffffffffull;
  // magnitudes as integers (order-preserving for non-negative values); signed y range
  // in FP32 for float, as order-preserving keys for double (no FP64 instructions)
  U amin = ~(U)0, amax = 0;
  T lo_ = (T)INFINITY, hi_ = (T)-INFINITY;
  long long klo = LLONG_MAX, khi = LLONG_MIN;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    if (!full && c + 32 * i + lane >= hi) continue;
    U b;
    if constexpr (F) b = __float_as_uint(v[i]);
    else b = (U)__double_as_longlong(v[i]);
    const U a = b & kAbs;
    amax = a > amax ? a : amax;
    amin = (a != 0 && a < amin) ? a : amin;
    if constexpr (F) {
      lo_ = fminf(lo_, v[i]);
      hi_ = fmaxf(hi_, v[i]);
    } else {
      const long long k = (long long)b < 0 ? (long long)(b ^ kAbs) : (long long)b;  // order-preserving key
      klo = k < klo ? k : klo;
      khi = k > khi ? k : khi;
    }
  }
  if constexpr (!F) {
    auto unkey = [&](long long k) { return __longlong_as_double(k < 0 ? (long long)((U)k ^ kAbs) : k); };
    lo_ = klo == LLONG_MAX ? (T)INFINITY : unkey(klo);
    hi_ = khi == LLONG_MIN ? (T)-INFINITY : unkey(khi);
  }
  const bool special = ((amax >> kTop) & kExpMask) == kExpMask;  // an inf or NaN in this lane
  if (special) hi_ = (T)NAN;  // flags the bucket's range
  *vmin = lo_;
  *vmax = hi_;
  int bmin = amin == ~(U)0 ? kExpMask + 1 : (int)(amin >> kTop);  // no nonzero term: above every exponent
  int bmax = amax == 0 ? -1 : (int)(amax >> kTop);
  bmin = __reduce_min_sync(kFull, bmin);
  bmax = __reduce_max_sync(kFull, bmax);
  if (bmax == kExpMask) return false;  // an inf or NaN somewhere
  if (bmax < 0) return true;           // every term is zero: S is unchanged (S is never -0)
  const int qs = (bmin ? bmin : 1) - kBias, et = (bmax ? bmax : 1) - kBias + kTop;
  int q = qs, eS = INT_MIN;
  if (*S != 0.0) {
    const Term ts = term_of(*S);
    q = min(q, low_bit(ts));
    eS = high_bit(ts);
  }
  if (eS != INT_MIN && (eS + 1 > 52 + q || eS + 2 > 1020)) return false;
  if (et + 9 > 52 + q || et + 9 > 1020) return false;  // 256 terms below 2^(et+1)
  long long sum = 0;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    if (!full && c + 32 * i + lane >= hi) continue;
    U b;
    if constexpr (F) b = __float_as_uint(v[i]);
    else b = (U)__double_as_longlong(v[i]);
    const int be = (int)(b >> kTop) & kExpMask;
    long long sig = (long long)(b & (((U)1 << kTop) - 1)) | (be ? (1ll << kTop) : 0ll);
    sig <<= ((be ? be : 1) - kBias) - q;  // exact: below 2^(et + 1 - q) <= 2^44
    sum += (b >> (F ? 31 : 63)) ? -sig : sig;
  }
  sum = warp_sum_i64(sum);
  *S = __dadd_rn(*S, dbl_scaled(sum, q));  // exact: the total is representable
  return true;
}

// Left-to-right FP64 sum of load(lo) .. load(hi-1) (R7), by a warp (all lanes call it;
// every lane returns the sum).  Chunks of 256 terms, lane l holding terms c + 32i + l,
// with the next chunk's loads in flight.  A chunk whose partial sums provably
// never round is added as one integer total; otherwise each 32-term row is added by
// row_add_exact (or, beyond 128-bit units, term by term).  obs(v, valid) sees every
// loaded value (bucket statistics in the same pass).
template <class Load, class Obs>
__device__ double warp_sum_ltr(int64_t lo, int64_t hi, int lane, Load load, Obs obs) {
  using T = decltype(load(lo));
  double S = 0.0;
  T va[8], vb[8];
  auto fetch = [&](int64_t c, T (&v)[8]) {
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int64_t p = c + 32 * i + lane;
      v[i] = p < hi ? load(p) : T(0);
    }
  };
  auto chunk = [&](int64_t c, T (&v)[8]) {
    T cmin, cmax;
    const bool ex = c + 256 <= hi ? try_exact_chunk_fp(&S, v, c, hi, lane, true, &cmin, &cmax)
                                  : try_exact_chunk_fp(&S, v, c, hi, lane, false, &cmin, &cmax);
    obs(cmin, cmax);
    if (ex) return;
    double dv[8];
    bool sp[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      dv[i] = dval(v[i]);
      sp[i] = term_of(v[i]).special;
    }
    chunk_rows(&S, dv, sp, c, hi, lane);
  };
  if (lo < hi) fetch(lo, va);
  if (lo + 256 < hi) fetch(lo + 256, vb);
  for (int64_t c = lo; c < hi; c += 512) {  // two buffers in turn: no register copy waits
    chunk(c, va);
    if (c + 256 >= hi) break;
    if (c + 512 < hi) fetch(c + 512, va);
    chunk(c + 256, vb);
    if (c + 768 < hi) fetch(c + 768, vb);
  }
  return S;
}

struct NoObs {
  template <class T>
  __device__ void operator()(T, T) const {}
};

// Whether the x sum of positions [lo, hi) has the closed form: implicit x on every
// point, all partial sums integers below 2^53, so the sequential FP64 sum is exact.
__device__ __forceinline__ bool x_closed(const SeriesPlan& sp, int64_t lo, int64_t hi) {
  return !sp.px && sp.xk == MMLTTB_X_IMPLICIT && hi > 0 && hi - lo <= ((1ll << 53) - 1) / hi;
}

// Sum of the x of positions [lo, hi) as LTTB's mean forms it, where it has no closed
// form (out of line: its registers stay out of the y path's).
__device__ __noinline__ double sum_x(const SeriesPlan& sp, int64_t lo, int64_t hi, int lane) {
  if (sp.px) return warp_sum_ltr(lo, hi, lane, [&](int64_t p) { return __ldg(sp.px + p); }, NoObs{});
  if (sp.xk == MMLTTB_X_IMPLICIT)
    return warp_sum_ltr(lo, hi, lane, [&](int64_t p) { return (double)p; }, NoObs{});
  // the method adds x as FP64 (x_of): int64 x enters the sum as its double
  if (sp.xk == MMLTTB_X_I64)
    return warp_sum_ltr(lo, hi, lane, [&](int64_t p) { return (double)__ldg((const long long*)sp.x + p); },
                        NoObs{});
  return warp_sum_ltr(lo, hi, lane, [&](int64_t p) { return __ldg((const double*)sp.x + p); }, NoObs{});
}

// The y range of a bucket as the chain's FP32 filter sees it (float32 exactly, float64
// truncated by f32_trunc), and whether every value is within its range (below 2^60).
struct YRange {
  float lo = INFINITY, hi = -INFINITY;
  bool ok = true;
  // a lane's range over a chunk (empty: lo = +inf, hi = -inf)
  __device__ void operator()(float mn, float mx) {
    if (!(mn <= mx)) {
      if (mn == mn && mx == mx) return;  // empty
      ok = false;                        // NaN
      return;
    }
    ok = ok && fabsf(mn) < 1.152921504606847e18f && fabsf(mx) < 1.152921504606847e18f;
    lo = fminf(lo, mn);
    hi = fmaxf(hi, mx);
  }
  __device__ void operator()(double mn, double mx) {
    if (!(mn <= mx)) {
      if (mn == mn && mx == mx) return;
      ok = false;
      return;
    }
    ok = ok && fabs(mn) < 1.152921504606847e18 && fabs(mx) < 1.152921504606847e18;
    lo = fminf(lo, f32_trunc(mn));  // f32_trunc is monotone
    hi = fmaxf(hi, f32_trunc(mx));
  }
};

// Sum of the y of positions [lo, hi) (R7), with the bucket's y range.  YS: 0 float32
// series, 1 float64 series, 2 the FP64 copies of preselected points.
template <int YS>
__device__ double sum_y(const SeriesPlan& sp, int64_t lo, int64_t hi, int lane, YRange& yr) {
  auto obs = [&](auto mn, auto mx) { yr(mn, mx); };
  if constexpr (YS == 2) return warp_sum_ltr(lo, hi, lane, [&](int64_t p) { return __ldg(sp.py + p); }, obs);
  else if constexpr (YS == 0)
    return warp_sum_ltr(lo, hi, lane, [&](int64_t p) { return __ldg((const float*)sp.y + p); }, obs);
  else return warp_sum_ltr(lo, hi, lane, [&](int64_t p) { return __ldg((const double*)sp.y + p); }, obs);
}

constexpr int kMeansThreads = 256;

// For t in [0, K]: bucket t's statistics for the chain's filter (t < K) and the mean
// after bucket t-1, that is of bucket t or, for t = K, of the last point (R1, R5, R7):
// means[2(t-1)], means[2(t-1)+1] and their split form.  A warp per t; bucket t's y is
// read once for both.
template <int YS>
__global__ void __launch_bounds__(kMeansThreads) k_lttb_means(const __grid_constant__ Batch bt) {
  const SeriesPlan& sp = bt.one;
  const int64_t m = lttb_m(sp);
  if (m <= sp.n_out) return;
  const int64_t K = sp.n_out - 2, N = m - 2;
  MeanF* mf = (MeanF*)(sp.means + 2 * K);
  BucketF* bf = (BucketF*)(mf + K);
  const int lane = threadIdx.x & 31;
  const int64_t w0 = ((int64_t)blockIdx.x * kMeansThreads + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * kMeansThreads) >> 5;
  for (int64_t t = w0; t <= K; t += nw) {
    int64_t lo = m - 1, hi = m;
    if (t < K) {
      lo = part_start(t, N, sp.dK);
      hi = part_start(t + 1, N, sp.dK);
    }
    YRange yr;
    const double sy = sum_y<YS>(sp, lo, hi, lane, yr);
    if (t < K) {
      float ymin = yr.lo, ymax = yr.hi;
#pragma unroll
      for (int d = 16; d > 0; d >>= 1) {
        ymin = fminf(ymin, __shfl_xor_sync(kFull, ymin, d));
        ymax = fmaxf(ymax, __shfl_xor_sync(kFull, ymax, d));
      }
      const bool ok = __all_sync(kFull, yr.ok);
      if (lane == 0) {
        BucketF b;
        b.ymin = ok ? ymin : __int_as_float(0x7fc00000);
        b.ymax = ok ? ymax : __int_as_float(0x7fc00000);
        b.x0 = filter_x(sp, lo);
        b.xspan = filter_x(sp, hi - 1) - b.x0;
        bf[t] = b;
      }
      if (t == 0) continue;  // bucket 0 is nobody's next bucket
    }
    const double sx = x_closed(sp, lo, hi) ? (double)((lo + hi - 1) * (hi - lo) / 2) : sum_x(sp, lo, hi, lane);
    if (lane == 0) {
      const double cnt = (double)(hi - lo);
      const double xc = __ddiv_rn(sx, cnt), yc = __ddiv_rn(sy, cnt);
      sp.means[2 * (t - 1)] = xc;
      sp.means[2 * (t - 1) + 1] = yc;
      // the split form the chain's FP32 filter uses (integer x)
      MeanF f;
      bool fits = true;
      split_floor(xc, &f.xint, &f.xfrac, &fits);
      if (!fits) f.xfrac = __int_as_float(0x7fc00000);  // NaN: unfiltered
      f.y32 = f64_below_pow2(yc, 60) ? f32_trunc(yc) : __int_as_float(0x7fc00000);
      f.ex = 4.0f * kFilterU;                     // split_floor's fraction
      f.ey = __fmul_ru(4.0f * kFilterU, fabsf(f.y32));  // truncation of yc
      mf[t - 1] = f;
    }
  }
}

// ---------------------------------------------------------------- the chain (fixpoint)

constexpr int kFixThreads = 512;
constexpr int kFixWarps = kFixThreads / 32;
constexpr int kFixUnroll = 8;  // positions per thread whose loads are in flight together

__device__ __forceinline__ bool beats(long long ab, long long pos, long long ob, long long op) {
  return ob > ab || (ob == ab && op < pos);
}

// Warp-wide merge of (t1, t2, p1): largest t1 first (lowest position on ties), t2 the
// largest of everything else.  Every lane ends with the same values.
__device__ __forceinline__ void warp_top2(float& t1, float& t2, long long& p1) {
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) {
    const float o1 = __shfl_xor_sync(kFull, t1, d), o2 = __shfl_xor_sync(kFull, t2, d);
    const long long op = __shfl_xor_sync(kFull, p1, d);
    if (o1 > t1 || (o1 == t1 && op < p1)) {
      t2 = fmaxf(fmaxf(t2, o2), t1);
      t1 = o1;
      p1 = op;
    } else {
      t2 = fmaxf(fmaxf(t2, o2), o1);
    }
  }
}

// Warp argmax of (ab, pos): largest area, then lowest position.
__device__ __forceinline__ void warp_argmax(long long& ab, long long& pos) {
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) {
    const long long ob = __shfl_xor_sync(kFull, ab, d), op = __shfl_xor_sync(kFull, pos, d);
    if (beats(ab, pos, ob, op)) {
      ab = ob;
      pos = op;
    }
  }
}

struct FixShared {
  float t1[kFixWarps], t2[kFixWarps];
  long long p1[kFixWarps], ab[kFixWarps];
  long long pick;
  int mode;
};

// The pick of bucket j after the point at position a (R1, R5-R8): the position in
// bucket j with the largest FP64 area against a and the mean after bucket j, the
// lowest position on ties.  Block-collective (all threads call it, every thread gets
// the result).  FP32 step bound first (StepBound, one bound E for the bucket): when
// the largest |T| minus E exceeds every other |T| plus E the first is the pick and no
// FP64 area is formed; otherwise the FP64 area of every candidate whose |T| + E reaches
// it decides.
__device__ long long bucket_argmax(const SeriesPlan& sp, int64_t j, long long a, const MeanF* mf,
                                   const BucketF* bf, FixShared& sh) {
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  const int64_t K = sp.n_out - 2, N = lttb_m(sp) - 2;
  const int64_t lo = part_start(j, N, sp.dK), hi = part_start(j + 1, N, sp.dK);
  const bool ytrunc = sp.py || sp.ydt != MMLTTB_F32;
  bool aok = true;
  const float ay32 = filter_y(sp, a, &aok);
  const BucketF bk = bf[j];
  StepBound sb;
  sb.init(filter_x(sp, a), aok ? ay32 : __int_as_float(0x7fc00000), bk.x0, mf[j], bk, ytrunc);
  sb.ok = sb.ok && sp.xk != MMLTTB_X_F64 && aok;
  // ---- filter round
  float t1 = -1.0f, t2 = -1.0f;
  long long p1 = LLONG_MAX;
  if (sb.ok) {
    for (int64_t q0 = lo + t; q0 < hi; q0 += (int64_t)kFixThreads * kFixUnroll) {
      float yv[kFixUnroll];
      long long xv[kFixUnroll];
#pragma unroll
      for (int u = 0; u < kFixUnroll; ++u) {
        const int64_t q = q0 + (int64_t)u * kFixThreads;
        bool ok = true;
        yv[u] = q < hi ? filter_y(sp, q, &ok) : 0.0f;
        xv[u] = q < hi ? filter_x(sp, q) : 0;
      }
#pragma unroll
      for (int u = 0; u < kFixUnroll; ++u) {
        const int64_t q = q0 + (int64_t)u * kFixThreads;
        const float ta = q < hi ? sb.t_abs(yv[u], f32_of_i64(xv[u] - bk.x0)) : -1.0f;
        t2 = fmaxf(t2, fminf(ta, t1));
        if (ta > t1) {
          t1 = ta;
          p1 = q;
        }
      }
    }
  }
  warp_top2(t1, t2, p1);
  if (lane == 0) {
    sh.t1[w] = t1;
    sh.t2[w] = t2;
    sh.p1[w] = p1;
  }
  __syncthreads();
  if (w == 0) {
    float u1 = lane < kFixWarps ? sh.t1[lane] : -1.0f, u2 = lane < kFixWarps ? sh.t2[lane] : -1.0f;
    long long up = lane < kFixWarps ? sh.p1[lane] : LLONG_MAX;
    warp_top2(u1, u2, up);
    if (lane == 0) {
      // decided: every other candidate's area is below the first's
      const bool dec = sb.ok && __fadd_ru(u2, sb.E) < __fsub_rd(u1, sb.E);
      sh.mode = dec ? 0 : 1;
      sh.pick = up;
      sh.t1[0] = u1;  // read by the exact round
    }
  }
  __syncthreads();
  if (sh.mode == 0) {
    const long long r = sh.pick;
    __syncthreads();  // sh is reused by the next call
    return r;
  }
  // ---- exact round (a near tie, or an unfiltered step): FP64 areas of the candidates
  // whose bound reaches the first's lower bound
  const float thr = sb.ok ? __fsub_rd(__fsub_rd(sh.t1[0], sb.E), sb.E) : -INFINITY;
  double xa, ya;
  pos_xy(sp, a, &xa, &ya);
  const double xc = sp.means[2 * j], yc = sp.means[2 * j + 1];
  long long ab = -1, pos = LLONG_MAX;
  for (int64_t q = lo + t; q < hi; q += kFixThreads) {
    if (sb.ok) {
      bool ok = true;
      const float yq = filter_y(sp, q, &ok);
      if (!(sb.t_abs(yq, f32_of_i64(filter_x(sp, q) - bk.x0)) >= thr)) continue;
    }
    double xb, yb;
    pos_xy(sp, q, &xb, &yb);
    const long long v = __double_as_longlong(tri_area(xa, ya, xb, yb, xc, yc));
    if (beats(ab, pos, v, q)) {
      ab = v;
      pos = q;
    }
  }
  warp_argmax(ab, pos);
  __syncthreads();  // every thread has read sh.t1[0]
  if (lane == 0) {
    sh.ab[w] = ab;
    sh.p1[w] = pos;
  }
  __syncthreads();
  if (w == 0) {
    long long wab = lane < kFixWarps ? sh.ab[lane] : -1, wpos = lane < kFixWarps ? sh.p1[lane] : LLONG_MAX;
    warp_argmax(wab, wpos);
    if (lane == 0) sh.pick = wpos;
  }
  __syncthreads();
  const long long r = sh.pick;
  __syncthreads();  // sh is reused by the next call
  (void)K;
  return r;
}

__device__ __forceinline__ long long ld_volatile(const long long* p) { return *(const volatile long long*)p; }
__device__ __forceinline__ int ld_volatile(const int* p) { return *(const volatile int*)p; }

// The LTTB chain as a fixpoint over all SMs.  b[j] is the pick the evaluation of
// bucket j takes as its previous pick (b[0] = position 0; b[j+1] = pick of bucket j).
// Start: b[j] = the first position of bucket j-1 (a guess) for j >= 1.  Pass 1 evaluates
// every bucket; each later pass evaluates the buckets whose b[j] changed in the pass
// before (a worklist), a CTA per bucket, and writes b[j+1] when it changes.  Whenever a
// bucket is not on the next worklist, b[j+1] = (pick of bucket j after b[j]); so the
// smallest wrong b[J] always has a correct b[J-1] on the next worklist, the correct
// prefix grows by at least one bucket a pass, and an empty worklist (at most K passes)
// means every b is the sequential method's pick: the result is bit-identical to the
// serial chain.  A bucket evaluated while its b[j] changes is on the next worklist
// anyway, so reading either value is safe.  Cooperative launch (all CTAs resident).
__global__ void __launch_bounds__(kFixThreads) k_lttb_fix(const __grid_constant__ Batch bt) {
  const SeriesPlan& sp = bt.one;
  const int64_t m = lttb_m(sp);
  if (m <= sp.n_out) return;  // uniform over the grid: no barrier was passed
  const int64_t K = sp.n_out - 2, N = m - 2;
  const MeanF* mf = (const MeanF*)(sp.means + 2 * K);
  const BucketF* bf = (const BucketF*)(mf + K);
  long long* b = (long long*)(bf + K);            // K+1 picks
  int* wl = (int*)(b + K + 1);                     // 2 worklists of K entries
  int* cnt = wl + 2 * K;                           // entries per pass, K+2 counters
  const int64_t G = gridDim.x, c = blockIdx.x;
  __shared__ FixShared sh;
  for (int64_t j = c * kFixThreads + threadIdx.x; j <= K + 1; j += G * kFixThreads) {
    if (j <= K) b[j] = j == 0 ? 0 : part_start(j - 1, N, sp.dK);
    cnt[j] = 0;
  }
  unsigned phase = 1;
  if (!grid_barrier(bt.barrier, (unsigned)G * phase, bt.status)) return;
  int64_t nitems = K;
  for (int64_t p = 0; nitems > 0 && p <= K; ++p) {
    const int* items = p == 0 ? nullptr : wl + (p & 1) * K;
    int* next = wl + ((p + 1) & 1) * K;
    for (int64_t i = c; i < nitems; i += G) {
      const int64_t j = items ? (int64_t)ld_volatile(items + i) : i;
      const long long a = ld_volatile(b + j);
      const long long v = bucket_argmax(sp, j, a, mf, bf, sh);
      if (threadIdx.x == 0 && v != ld_volatile(b + j + 1)) {
        *(volatile long long*)(b + j + 1) = v;
        if (j + 1 < K) next[atomicAdd(cnt + p + 1, 1)] = (int)(j + 1);
      }
    }
    ++phase;
    if (!grid_barrier(bt.barrier, (unsigned)G * phase, bt.status)) return;
    nitems = ld_volatile(cnt + p + 1);
  }
  for (int64_t j = c * kFixThreads + threadIdx.x; j < K; j += G * kFixThreads)
    sp.out[j + 1] = index_of(sp, ld_volatile(b + j + 1));
  if (c == 0 && threadIdx.x == 0) {
    sp.out[0] = index_of(sp, 0);
    sp.out[K + 1] = index_of(sp, m - 1);
    if (sp.out_count) *sp.out_count = sp.n_out;
  }
}

}  // namespace

cudaError_t launch_lttb_means(const Batch& bt, int sms, cudaStream_t st) {
  const int64_t K = bt.one.n_out - 2;
  int64_t blocks = ((K + 1) * 32 + kMeansThreads - 1) / kMeansThreads;
  const int64_t cap = (int64_t)sms * (2048 / kMeansThreads);
  if (blocks > cap) blocks = cap;
  if (blocks < 1) blocks = 1;
  const SeriesPlan& sp = bt.one;
  if (sp.py) k_lttb_means<2><<<(unsigned)blocks, kMeansThreads, 0, st>>>(bt);
  else if (sp.ydt == MMLTTB_F32) k_lttb_means<0><<<(unsigned)blocks, kMeansThreads, 0, st>>>(bt);
  else k_lttb_means<1><<<(unsigned)blocks, kMeansThreads, 0, st>>>(bt);
  return cudaGetLastError();
}

// Workspace bytes of the large-bucket engine for K buckets: FP64 means, their split
// form, bucket statistics, the picks, two worklists and the per-pass counters.
size_t lttb_big_bytes(int64_t K) {
  return (size_t)K * 16 + (size_t)K * sizeof(MeanF) + (size_t)K * sizeof(BucketF) + (size_t)(K + 1) * 8 +
         (size_t)2 * K * 4 + (size_t)(K + 2) * 4;
}

cudaError_t launch_lttb_fix(const Batch& bt, int sms, cudaStream_t st) {
  static int bps[64];
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  if (bps[dev] == 0) {
    int n = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_lttb_fix, kFixThreads, 0);
    if (e != cudaSuccess) return e;
    bps[dev] = n < 1 ? 1 : (n > 2 ? 2 : n);
  }
  Batch copy = bt;
  void* args[] = {&copy};
  return cudaLaunchCooperativeKernel((const void*)k_lttb_fix, dim3((unsigned)(sms * bps[dev])), dim3(kFixThreads),
                                     args, 0, st);
}

}  // namespace mmlttb
