// Device code of the MinMax preselection pass (Sec. 3 first step; MinMax of
// Sec. 2.2.1, Table 1), shared by the split kernels (k_edges, k_stream) and the
// fused single-cluster kernel.
//
// The interior points of every series are laid end to end in one global work space
// (series_work in common.cuh), cut into W equal ranges, one per warp.  A warp walks
// the bins that meet its range; for each piece it streams y with 16-byte coalesced
// loads and keeps a per-lane first-occurrence argmin/argmax, then reduces across its
// lane group and writes one Record at slot (global bin + warp).  x is never streamed:
// bin bounds come from integer arithmetic (index bins) or from the bin-edge search.
#pragma once

#include "common.cuh"

namespace mmlttb {
namespace {

__device__ __forceinline__ float4 ld_stream4(const float4* p) {
  float4 v;
  asm("ld.global.nc.L1::no_allocate.L2::256B.v4.f32 {%0,%1,%2,%3}, [%4];"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
               : "l"(p));
  return v;
}

__device__ __forceinline__ uint4 ld_stream4u(const void* p) {
  uint4 v;
  asm("ld.global.nc.L1::no_allocate.L2::256B.v4.u32 {%0,%1,%2,%3}, [%4];"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "l"(p));
  return v;
}

// Where a segment routine reads y from: straight from global memory (16-byte
// streaming loads), or from a window of y staged in shared memory.  Both take the
// global address of a 16-byte aligned vector of y.
struct GlobalSrc {
  __device__ __forceinline__ float4 ld4(uintptr_t a) const { return ld_stream4((const float4*)a); }
  __device__ __forceinline__ uint4 ld4u(uintptr_t a) const { return ld_stream4u((const void*)a); }
};
// A copy of global bytes [g0, g0 + size) at shared address s0 (g0 and s0 16-byte
// aligned); only vectors inside the copy are read.
struct SharedSrc {
  uintptr_t g0;
  uint32_t s0;
  __device__ __forceinline__ float4 ld4(uintptr_t a) const {
    float4 v;
    asm volatile("ld.shared.v4.f32 {%0,%1,%2,%3}, [%4];"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                 : "r"(s0 + (uint32_t)(a - g0)));
    return v;
  }
  __device__ __forceinline__ uint4 ld4u(uintptr_t a) const {
    uint4 v;
    asm volatile("ld.shared.v4.u32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "r"(s0 + (uint32_t)(a - g0)));
    return v;
  }
};

// NaN-propagating float min/max (a NaN operand makes the result NaN).
__device__ __forceinline__ float fmin_nan(float a, float b) {
  float r;
  asm("min.NaN.f32 %0, %1, %2;" : "=f"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ float fmax_nan(float a, float b) {
  float r;
  asm("max.NaN.f32 %0, %1, %2;" : "=f"(r) : "f"(a), "f"(b));
  return r;
}

// The high 32 bits of a double read as a float.  For doubles below 2^1017 in
// magnitude this is a non-decreasing function of the double's value (the bit
// patterns of both formats order like sign-magnitude integers), so
// proxy(e) > proxy(m) implies e > m.  Larger magnitudes, inf and NaN map to NaN or
// inf proxies, which the callers treat as "compare exactly".
__device__ __forceinline__ float proxy_of_hi(unsigned hi) { return __uint_as_float(hi); }

// Bin bounds of series sp (R2 index bins; R3 x-width bins via the edge array).
// Bins cover the points [p0, p0 + nb): the interior for MinMax, all points for M4.
__device__ __forceinline__ int64_t bin_start(const Batch& bt, const SeriesPlan& sp, int64_t b) {
  if (sp.binmode == MMLTTB_BINS_INDEX) return sp.p0 + muldiv(b, sp.nb, sp.dB);
  return bt.edges[sp.edge_off + b];
}
// The bin holding binned point p; warp-collective (every lane passes the same p).
// x-width bins: a 32-ary search of the bin starts (three rounds for 8000 bins where
// a binary search takes thirteen dependent loads).
__device__ __forceinline__ int64_t bin_containing(const Batch& bt, const SeriesPlan& sp, int64_t p,
                                                  int lane) {
  if (sp.binmode == MMLTTB_BINS_INDEX) return part_of(p - sp.p0 + 1, sp.dnb, sp.B);
  const int64_t* E = bt.edges + sp.edge_off;
  int64_t lo = 0, hi = sp.B;  // the largest i < B with E[i] <= p lies in [lo, hi); E[0] <= p
  while (hi - lo > 1) {
    const int64_t step = (hi - lo + 31) >> 5;
    const int64_t q = lo + (int64_t)lane * step;
    const unsigned le = __ballot_sync(kFull, q < hi && E[q] <= p);  // a prefix of the lanes
    const int64_t last = lo + (int64_t)(31 - __clz(le)) * step;
    hi = last + step < hi ? last + step : hi;
    lo = last;
  }
  return lo;
}

// (key, offset) reductions over the aligned group of G lanes holding this lane (G a
// power of two), every lane of the warp taking part: the smallest key with its
// smallest offset (argmin, first occurrence on ties) and the largest key with its
// smallest offset.  A whole warp (G = 32) uses the warp reduction instructions;
// smaller groups exchange with log2(G) xor shuffles, one instruction serving every
// group of the warp (reductions over a sub-warp mask are issued once per group).
__device__ __forceinline__ void group_arg32(int& kmn, unsigned& omn, int& kmx, unsigned& omx, int G) {
  if (G == 32) {
    const int wmn = __reduce_min_sync(kFull, kmn);
    omn = __reduce_min_sync(kFull, kmn == wmn ? omn : 0xffffffffu);
    kmn = wmn;
    const int wmx = __reduce_max_sync(kFull, kmx);
    omx = __reduce_min_sync(kFull, kmx == wmx ? omx : 0xffffffffu);
    kmx = wmx;
    return;
  }
  for (int d = 1; d < G; d <<= 1) {
    const int a = __shfl_xor_sync(kFull, kmn, d);
    const unsigned ao = __shfl_xor_sync(kFull, omn, d);
    if (a < kmn || (a == kmn && ao < omn)) {
      kmn = a;
      omn = ao;
    }
    const int c = __shfl_xor_sync(kFull, kmx, d);
    const unsigned co = __shfl_xor_sync(kFull, omx, d);
    if (c > kmx || (c == kmx && co < omx)) {
      kmx = c;
      omx = co;
    }
  }
}
__device__ __forceinline__ void group_arg64(long long& kmn, unsigned& omn, long long& kmx, unsigned& omx,
                                            int G) {
  if (G == 32) {  // int64 order = (signed high word, unsigned low word)
    const int hmn = (int)(kmn >> 32);
    const unsigned lmn = (unsigned)kmn;
    const int whm = __reduce_min_sync(kFull, hmn);
    const unsigned wlm = __reduce_min_sync(kFull, hmn == whm ? lmn : 0xffffffffu);
    const bool eqm = (hmn == whm) && (lmn == wlm);
    omn = __reduce_min_sync(kFull, eqm ? omn : 0xffffffffu);
    kmn = (long long)(((unsigned long long)(unsigned)whm << 32) | wlm);
    const int hmx = (int)(kmx >> 32);
    const unsigned lmx = (unsigned)kmx;
    const int whx = __reduce_max_sync(kFull, hmx);
    const unsigned wlx = __reduce_max_sync(kFull, hmx == whx ? lmx : 0u);
    const bool eqx = (hmx == whx) && (lmx == wlx);
    omx = __reduce_min_sync(kFull, eqx ? omx : 0xffffffffu);
    kmx = (long long)(((unsigned long long)(unsigned)whx << 32) | wlx);
    return;
  }
  for (int d = 1; d < G; d <<= 1) {
    const long long a = __shfl_xor_sync(kFull, kmn, d);
    const unsigned ao = __shfl_xor_sync(kFull, omn, d);
    if (a < kmn || (a == kmn && ao < omn)) {
      kmn = a;
      omn = ao;
    }
    const long long c = __shfl_xor_sync(kFull, kmx, d);
    const unsigned co = __shfl_xor_sync(kFull, omx, d);
    if (c > kmx || (c == kmx && co < omx)) {
      kmx = c;
      omx = co;
    }
  }
}
__device__ __forceinline__ unsigned group_min_u32(unsigned v, int G) {
  if (G == 32) return __reduce_min_sync(kFull, v);
  for (int d = 1; d < G; d <<= 1) {
    const unsigned o = __shfl_xor_sync(kFull, v, d);
    v = o < v ? o : v;
  }
  return v;
}

// First-occurrence argmin/argmax of y[lo, hi) for float32 y by one group of G lanes
// (gl = lane within the group; G = 32: the whole warp).  Every lane of the warp calls
// it (a group with nothing to do passes lo == hi).
// kNanAware: NaN-aware mode (R18): a bin holding a NaN reports its first NaN as both
// extremes; its record carries the keys LLONG_MIN / LLONG_MAX, which no value has,
// so merging records keeps the first NaN of the bin.
template <int kUnroll, bool kNanAware, class Src = GlobalSrc>
__device__ Record segment_f32(const float* y, int64_t lo, int64_t hi, int gl, int G, const Src& src = Src()) {
  const uint32_t len = (uint32_t)(hi - lo);
  const float inf = __int_as_float(0x7f800000);
  // Empty state: only strictly smaller (larger) values are recorded, so a lane that
  // sees nothing but +inf (-inf) keeps offset ~0u; if every lane does, the extreme is
  // the first point (offset 0).
  float mn = inf, mx = -inf;
  uint32_t omn = 0xffffffffu, omx = 0xffffffffu, onan = 0xffffffffu;
  const uintptr_t ybase = (uintptr_t)y;
  const uintptr_t a0 = (ybase + (uintptr_t)lo * 4u) & ~(uintptr_t)15;
  const int32_t rel0 = (int32_t)((int64_t)(a0 - ybase) / 4 - lo);  // offset of vector 0's first element: -3..0
  // vectors 0..nvec-1 cover the piece; those in [vf, vl) lie wholly inside it, the
  // others (the first when the piece starts mid-vector, the last when it ends
  // mid-vector) are masked
  const int32_t span = (int32_t)len - rel0;
  const int32_t nvec = len ? (span + 3) >> 2 : 0;
  const int32_t vf = rel0 < 0 ? 1 : 0, vl = span >> 2;
  // one vector with its out-of-piece elements masked out (in offset order)
  auto masked = [&](const float4 b, int32_t r) {
    const float e[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
    for (int k = 0; k < 4; k++) {
      if ((uint32_t)(r + k) >= len) continue;
      if (kNanAware && onan == 0xffffffffu && e[k] != e[k]) onan = (uint32_t)(r + k);
      if (e[k] < mn) { mn = e[k]; omn = (uint32_t)(r + k); }
      if (e[k] > mx) { mx = e[k]; omx = (uint32_t)(r + k); }
    }
  };
  if (gl == 0 && vf == 1 && nvec > 0) masked(src.ld4(a0), rel0);  // the lowest offsets first
  for (int32_t v = vf + gl; v < vl; v += G * kUnroll) {
    float4 buf[kUnroll];
#pragma unroll
    for (int u = 0; u < kUnroll; u++)
      if (v + G * u < vl) buf[u] = src.ld4(a0 + (uintptr_t)(v + G * u) * 16u);
#pragma unroll
    for (int u = 0; u < kUnroll; u++) {
      if (v + G * u >= vl) break;
      const float4 b = buf[u];
      if (kNanAware && onan == 0xffffffffu) {
        if ((b.x != b.x) | (b.y != b.y) | (b.z != b.z) | (b.w != b.w)) {
          const int32_t r = rel0 + 4 * (v + G * u);
          onan = (uint32_t)(b.x != b.x ? r : b.y != b.y ? r + 1 : b.z != b.z ? r + 2 : r + 3);
        }
      }
      const float m4 = fminf(fminf(b.x, b.y), fminf(b.z, b.w));
      const float x4 = fmaxf(fmaxf(b.x, b.y), fmaxf(b.z, b.w));
      if (m4 < mn) {  // rare: some element is a new strict minimum
        const int32_t r = rel0 + 4 * (v + G * u);
        if (b.x < mn) { mn = b.x; omn = (uint32_t)r; }
        if (b.y < mn) { mn = b.y; omn = (uint32_t)(r + 1); }
        if (b.z < mn) { mn = b.z; omn = (uint32_t)(r + 2); }
        if (b.w < mn) { mn = b.w; omn = (uint32_t)(r + 3); }
      }
      if (x4 > mx) {
        const int32_t r = rel0 + 4 * (v + G * u);
        if (b.x > mx) { mx = b.x; omx = (uint32_t)r; }
        if (b.y > mx) { mx = b.y; omx = (uint32_t)(r + 1); }
        if (b.z > mx) { mx = b.z; omx = (uint32_t)(r + 2); }
        if (b.w > mx) { mx = b.w; omx = (uint32_t)(r + 3); }
      }
    }
  }
  if (gl == 0 && nvec - 1 >= vl && nvec - 1 >= vf) masked(src.ld4(a0 + (uintptr_t)(nvec - 1) * 16u), rel0 + 4 * (nvec - 1));
  int wmn = key32(mn), wmx = key32(mx);
  unsigned wo = omn, wx = omx;
  group_arg32(wmn, wo, wmx, wx, G);
  Record r;
  r.kmin = wmn;
  r.kmax = wmx;
  r.imin = lo + (int64_t)(wo == 0xffffffffu ? 0u : wo);
  r.imax = lo + (int64_t)(wx == 0xffffffffu ? 0u : wx);
  if (kNanAware) {
    const unsigned wn = group_min_u32(onan, G);
    if (wn != 0xffffffffu) {
      r.kmin = LLONG_MIN;
      r.kmax = LLONG_MAX;
      r.imin = r.imax = lo + (int64_t)wn;
    }
  }
  return r;
}

// Warp-wide first-occurrence argmin/argmax of y[lo, hi) for float64 y.  The hot
// loop issues no FP64 instruction (FP64 is a narrow pipe on this part): a float
// compare of the high-word proxies rules out almost every element, and the rest
// are compared exactly through order-preserving int64 keys.
template <int kUnroll, bool kNanAware, class Src = GlobalSrc>
__device__ Record segment_f64(const double* y, int64_t lo, int64_t hi, int gl, int G, const Src& src = Src()) {
  const uint32_t len = (uint32_t)(hi - lo);
  // Empty state: keys beyond every double's key and NaN proxies, so the first
  // element a lane sees takes the exact path and is recorded.
  long long kmn = LLONG_MAX, kmx = LLONG_MIN;
  float pmn = __int_as_float(0x7fc00000), pmx = pmn;
  uint32_t omn = 0xffffffffu, omx = 0xffffffffu, onan = 0xffffffffu;
  const uintptr_t ybase = (uintptr_t)y;
  const uintptr_t a0 = (ybase + (uintptr_t)lo * 8u) & ~(uintptr_t)15;
  const int32_t rel0 = (int32_t)((int64_t)(a0 - ybase) / 8 - lo);  // offset of vector 0's first element: -1..0
  const float inf = __int_as_float(0x7f800000);
  // vectors in [vf, vl) lie wholly inside the piece; a first or last vector that is
  // only partly inside is masked
  const int32_t span = (int32_t)len - rel0;
  const int32_t nvec = len ? (span + 1) >> 1 : 0;
  const int32_t vf = rel0 < 0 ? 1 : 0, vl = span >> 1;
  // the two elements of vector b at offsets r, r + 1 (ok0/ok1: inside the piece)
  auto update = [&](const uint4 b, int32_t r, bool ok0, bool ok1) {
    const float p0 = proxy_of_hi(b.y), p1 = proxy_of_hi(b.w);
    const float pm = fmin_nan(ok0 ? p0 : inf, ok1 ? p1 : inf);
    const float px = fmax_nan(ok0 ? p0 : -inf, ok1 ? p1 : -inf);
    if (!(pm > pmn) || !(px < pmx)) {  // rare: exact comparison through int64 keys
      const long long e0 = ((long long)b.y << 32) | b.x;
      const long long e1 = ((long long)b.w << 32) | b.z;
      const long long k0 = key64(__longlong_as_double(e0));
      const long long k1 = key64(__longlong_as_double(e1));
      if (kNanAware && onan == 0xffffffffu) {  // NaN proxies always take this path
        const long long m = 0x7fffffffffffffffLL, inf_bits = 0x7ff0000000000000LL;
        if (ok1 && (e1 & m) > inf_bits) onan = (uint32_t)(r + 1);
        if (ok0 && (e0 & m) > inf_bits) onan = (uint32_t)r;
      }
      if (ok0 && k0 < kmn) { kmn = k0; omn = (uint32_t)r; pmn = p0; }
      if (ok1 && k1 < kmn) { kmn = k1; omn = (uint32_t)(r + 1); pmn = p1; }
      if (ok0 && k0 > kmx) { kmx = k0; omx = (uint32_t)r; pmx = p0; }
      if (ok1 && k1 > kmx) { kmx = k1; omx = (uint32_t)(r + 1); pmx = p1; }
    }
  };
  auto masked = [&](int32_t vi) {
    const int32_t r = rel0 + 2 * vi;
    update(src.ld4u(a0 + (uintptr_t)vi * 16u), r, (uint32_t)r < len, (uint32_t)(r + 1) < len);
  };
  if (gl == 0 && vf == 1 && nvec > 0) masked(0);  // the lowest offsets first
  for (int32_t v = vf + gl; v < vl; v += G * kUnroll) {
    uint4 buf[kUnroll];
#pragma unroll
    for (int u = 0; u < kUnroll; u++)
      if (v + G * u < vl) buf[u] = src.ld4u(a0 + (uintptr_t)(v + G * u) * 16u);
#pragma unroll
    for (int u = 0; u < kUnroll; u++) {
      if (v + G * u >= vl) break;
      update(buf[u], rel0 + 2 * (v + G * u), true, true);
    }
  }
  if (gl == 0 && nvec - 1 >= vl && nvec - 1 >= vf) masked(nvec - 1);
  unsigned wo = omn, wx = omx;
  group_arg64(kmn, wo, kmx, wx, G);
  Record r;
  r.kmin = kmn;
  r.kmax = kmx;
  r.imin = lo + (int64_t)(wo == 0xffffffffu ? 0u : wo);
  r.imax = lo + (int64_t)(wx == 0xffffffffu ? 0u : wx);
  if (kNanAware) {
    const unsigned wn = group_min_u32(onan, G);
    if (wn != 0xffffffffu) {
      r.kmin = LLONG_MIN;
      r.kmax = LLONG_MAX;
      r.imin = r.imax = lo + (int64_t)wn;
    }
  }
  return r;
}

// The segment routine for the plan's y type and NaN rule, for kernels compiled for
// any y.  Each routine stays a separate function: inlined together, the four of
// them spill their state.
template <int kUnroll, bool kNan>
__device__ __noinline__ Record segment_f32_call(const float* y, int64_t lo, int64_t hi, int gl, int G) {
  return segment_f32<kUnroll, kNan>(y, lo, hi, gl, G);
}
template <int kUnroll, bool kNan>
__device__ __noinline__ Record segment_f64_call(const double* y, int64_t lo, int64_t hi, int gl, int G) {
  return segment_f64<kUnroll, kNan>(y, lo, hi, gl, G);
}
template <int kUnroll>
__device__ __forceinline__ Record segment_any(const SeriesPlan& sp, int64_t lo, int64_t hi, int gl, int G) {
  if (sp.nan_aware)
    return sp.ydt == MMLTTB_F32 ? segment_f32_call<kUnroll, true>((const float*)sp.y, lo, hi, gl, G)
                                : segment_f64_call<kUnroll, true>((const double*)sp.y, lo, hi, gl, G);
  return sp.ydt == MMLTTB_F32 ? segment_f32_call<kUnroll, false>((const float*)sp.y, lo, hi, gl, G)
                              : segment_f64_call<kUnroll, false>((const double*)sp.y, lo, hi, gl, G);
}

// Smallest interior point q in [0, N] whose work unit floor(q*D/N) is >= t, for
// 0 <= t <= D: ceil(t*N/D).
__device__ __forceinline__ int64_t point_at_work(int64_t t, int64_t N, const Div& D) {
  return muldiv_ceil(t, N, D);
}

// y kinds a stream kernel is compiled for: any (dispatch on the plan's type and
// NaN-aware flag), or one type with or without the NaN-aware rule.  A kernel
// specialised to one kind inlines one segment routine instead of calling one of four
// and keeps its state in registers.
enum YMode : int { kYAny = 0, kYF32 = 1, kYF64 = 2, kYF32Nan = 3, kYF64Nan = 4 };

// One warp over the binned points [p_lo, p_hi) of one series.  The warp splits into
// 32/G groups of G lanes (G chosen per series from its mean bin size) and each group
// works on its own bin, so small bins are processed 32/G at a time.
template <int kUnroll, int kY>
__device__ void warp_series_range(const Batch& bt, const SeriesPlan& sp, int64_t p_lo,
                                  int64_t p_hi, int64_t w, int lane) {
  const int G = sp.group;
  const int ngroups = 32 / G;
  const int grp = lane / G, gl = lane - grp * G;
  const bool ib = sp.binmode == MMLTTB_BINS_INDEX;
  int64_t b = bin_containing(bt, sp, p_lo, lane);
  // index bins: L = floor(mb*nb/B) and rem = mb*nb - L*B for this group's bin mb,
  // stepped by 32/G bins per round with the plan's constants (no division per bin)
  int64_t L = 0;
  int32_t rem = 0;
  if (ib) {
    const int64_t mb0 = b + grp;
    L = muldiv(mb0, sp.nb, sp.dB);
    rem = (int32_t)((uint64_t)mb0 * (uint64_t)sp.nb - (uint64_t)L * (uint64_t)sp.B);
  }
  for (;;) {
    const int64_t mb = b + grp;
    int64_t lo = p_hi, hi = p_hi, sb1 = sp.p0 + sp.nb;
    if (mb < sp.B) {
      int64_t sb;
      if (ib) {
        sb = sp.p0 + L;
        if (mb + 1 < sp.B) sb1 = sb + sp.bin_q1 + (rem + sp.bin_r1 >= sp.B ? 1 : 0);
      } else {
        sb = bin_start(bt, sp, mb);
        if (mb + 1 < sp.B) sb1 = bin_start(bt, sp, mb + 1);
      }
      lo = sb > p_lo ? sb : p_lo;
      hi = sb1 < p_hi ? sb1 : p_hi;
      if (hi < lo) hi = lo;
    }
    {  // every group takes part in the group reductions; empty groups have lo == hi
      Record r;
      if constexpr (kY == kYF32) {
        r = segment_f32<kUnroll, false>((const float*)sp.y, lo, hi, gl, G);
      } else if constexpr (kY == kYF64) {
        r = segment_f64<kUnroll, false>((const double*)sp.y, lo, hi, gl, G);
      } else if constexpr (kY == kYF32Nan) {
        r = segment_f32<kUnroll, true>((const float*)sp.y, lo, hi, gl, G);
      } else if constexpr (kY == kYF64Nan) {
        r = segment_f64<kUnroll, true>((const double*)sp.y, lo, hi, gl, G);
      } else {
        r = segment_any<kUnroll>(sp, lo, hi, gl, G);
      }
      if (gl == 0 && lo < hi) bt.rec[sp.bin_off + mb + w] = r;
    }
    // the round ends with bin b + ngroups - 1 (held by the last group)
    const int64_t last_end = __shfl_sync(kFull, sb1, 31);
    if (last_end >= p_hi || b + ngroups >= sp.B) break;
    b += ngroups;
    if (ib) {
      L += sp.bin_qs;
      rem += sp.bin_rs;
      if (rem >= sp.B) {
        rem -= (int32_t)sp.B;
        L += 1;
      }
    }
  }
}


// Streaming warp w of the launch: every bin piece of every series in its range.
template <int U, int kY = kYAny>
__device__ void stream_warp(const Batch& bt, int64_t w, int lane) {
  int64_t g = warp_begin(w, bt.total_pos, bt.dwarps);
  const int64_t g_end = warp_begin(w + 1, bt.total_pos, bt.dwarps);
  int s = bt.pos_offs ? upper_index(bt.pos_offs, bt.n_series, g) : 0;
  while (g < g_end && s < bt.n_series) {
    const SeriesPlan& sp = plan_of(bt, s);
    const int64_t send = sp.pos_off + sp.npos;
    const int64_t seg_end = send < g_end ? send : g_end;
    if (seg_end > g) {
      // binned points whose work unit lies in [g, seg_end): p0 + q, q in [q_lo, q_hi)
      const int64_t q_lo = point_at_work(g - sp.pos_off, sp.nb, sp.dnpos);
      const int64_t q_hi = point_at_work(seg_end - sp.pos_off, sp.nb, sp.dnpos);
      if (q_hi > q_lo) warp_series_range<U, kY>(bt, sp, sp.p0 + q_lo, sp.p0 + q_hi, w, lane);
      g = seg_end;
    }
    ++s;
  }
}

// ---- staged stream (k_stream_bulk) ----
// mbarrier and bulk-copy primitives (shared addresses of this CTA).
__device__ __forceinline__ void mbar_init(uint32_t bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.release.cta.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_copy_g2s(uint32_t dst, uintptr_t src, uint32_t bytes, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
      "l"(src), "r"(bytes), "r"(bar)
      : "memory");
}
// Test for the completion of phase `parity`; the warp may be suspended (without
// issuing) until it completes or about `hint_ns` pass.
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, unsigned parity, unsigned hint_ns) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cta.shared::cta.b64 p, [%1], %2, %3;\n"
      " selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(bar), "r"(parity), "r"(hint_ns)
      : "memory");
  return ok != 0;
}
// Wait for phase `parity` of a barrier to complete, for at most 2 s.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, unsigned parity) {
  if (mbar_try_wait(bar, parity, 20000u)) return true;
  const unsigned long long t0 = global_ns();
  for (;;) {
    if (mbar_try_wait(bar, parity, 20000u)) return true;
    if (global_ns() - t0 > 2000000000ull) return false;
  }
}

// The bins, y window and copy of tile t of a staged series: bins [b0, b1), points
// [e0, e1), and the 16-byte aligned global bytes [g0, g0 + bytes) holding them (every
// 16-byte vector of it holds a point of the series, as with the register stream's
// vector loads).
struct TileWin {
  int64_t b0, b1, e0, e1;
  uintptr_t g0;
  uint32_t bytes;
};
__device__ __forceinline__ TileWin tile_window(const SeriesPlan& sp, int64_t t) {
  TileWin w;
  w.b0 = t * sp.bulk_bpt;
  w.b1 = w.b0 + sp.bulk_bpt < sp.B ? w.b0 + sp.bulk_bpt : sp.B;
  const int64_t e0 = sp.p0 + muldiv(w.b0, sp.nb, sp.dB);
  const int64_t e1 = w.b1 >= sp.B ? sp.p0 + sp.nb : sp.p0 + muldiv(w.b1, sp.nb, sp.dB);
  w.e0 = e0;
  w.e1 = e1;
  const uintptr_t es = sp.ydt == MMLTTB_F32 ? 4u : 8u, y = (uintptr_t)sp.y;
  w.g0 = (y + (uintptr_t)e0 * es) & ~(uintptr_t)15;
  const uintptr_t g1 = (y + (uintptr_t)e1 * es + 15u) & ~(uintptr_t)15;
  w.bytes = e1 > e0 ? (uint32_t)(g1 - w.g0) : 0u;
  return w;
}

// The tiles a warp takes, in order: those whose first unit lies in the warp's range
// [c0, c1) of the tile cost space (series s holds units [tcost_off, tcost_off +
// tiles * tcost)).
struct TileCursor {
  int s;
  int64_t t, t_end, c0, c1;
  bool done;
  __device__ void span(const Batch& bt) {  // the tiles of series s in [c0, c1)
    const SeriesPlan& sp = plan_of(bt, s);
    t = t_end = 0;
    if (sp.bulk_bpt <= 0 || sp.tcost <= 0) return;
    const int64_t nt = (sp.B + sp.bulk_bpt - 1) / sp.bulk_bpt;
    const int64_t a = c0 - sp.tcost_off, b = c1 - sp.tcost_off;
    t = a <= 0 ? 0 : (a + sp.tcost - 1) / sp.tcost;
    t_end = b <= 0 ? 0 : (b + sp.tcost - 1) / sp.tcost;
    if (t_end > nt) t_end = nt;
  }
  __device__ void advance(const Batch& bt) {  // to the next series with a tile in range
    while (t >= t_end) {
      if (++s >= bt.n_series || plan_of(bt, s).tcost_off >= c1) {
        done = true;
        return;
      }
      span(bt);
    }
  }
  __device__ void init(const Batch& bt, int64_t c0_, int64_t c1_) {
    c0 = c0_;
    c1 = c1_;
    done = c0 >= c1;
    s = bt.tcost_offs ? upper_index(bt.tcost_offs, bt.n_series, c0) : 0;
    if (done) return;
    span(bt);
    advance(bt);
  }
  __device__ void next(const Batch& bt) {
    ++t;
    advance(bt);
  }
};

// Partial MinMax state of a piece of a bin (float32): the smallest and largest value
// recorded and their first offsets in the tile (kNone: nothing recorded; as in the
// register stream only values below +inf / above -inf are recorded, so NaN never is),
// and the first NaN (NaN-aware rule).
constexpr uint32_t kNone = 0xffffffffu;
struct Part {
  float mn, mx;
  uint32_t imn, imx, inan;
};
__device__ __forceinline__ void part_reset(Part& c) {
  c.mn = __int_as_float(0x7f800000);
  c.mx = -c.mn;
  c.imn = c.imx = c.inan = kNone;
}
// a and b cover disjoint pieces of one bin: the first occurrence over both
__device__ __forceinline__ void part_merge(Part& a, const Part& b) {
  if (b.imn != kNone && (a.imn == kNone || b.mn < a.mn || (b.mn == a.mn && b.imn < a.imn))) {
    a.mn = b.mn;
    a.imn = b.imn;
  }
  if (b.imx != kNone && (a.imx == kNone || b.mx > a.mx || (b.mx == a.mx && b.imx < a.imx))) {
    a.mx = b.mx;
    a.imx = b.imx;
  }
  a.inan = b.inan < a.inan ? b.inan : a.inan;
}
__device__ __forceinline__ Part part_shfl_down(const Part& c, int d) {
  Part r;
  r.mn = __shfl_down_sync(kFull, c.mn, d);
  r.mx = __shfl_down_sync(kFull, c.mx, d);
  r.imn = __shfl_down_sync(kFull, c.imn, d);
  r.imx = __shfl_down_sync(kFull, c.imx, d);
  r.inan = __shfl_down_sync(kFull, c.inan, d);
  return r;
}
template <bool kNan>
__device__ __forceinline__ void part_add(Part& c, float v, uint32_t off) {
  if (kNan && c.inan == kNone && v != v) c.inan = off;
  if (v < c.mn) {
    c.mn = v;
    c.imn = off;
  }
  if (v > c.mx) {
    c.mx = v;
    c.imx = off;
  }
}
// four consecutive points (offsets off..off+3) of one bin
template <bool kNan>
__device__ __forceinline__ void part_add4(Part& c, const float4 b, uint32_t off) {
  if (kNan && c.inan == kNone && ((b.x != b.x) | (b.y != b.y) | (b.z != b.z) | (b.w != b.w)))
    c.inan = off + (b.x != b.x ? 0u : b.y != b.y ? 1u : b.z != b.z ? 2u : 3u);
  const float m4 = fminf(fminf(b.x, b.y), fminf(b.z, b.w));
  const float x4 = fmaxf(fmaxf(b.x, b.y), fmaxf(b.z, b.w));
  if (m4 < c.mn) {  // its first occurrence among the four (a NaN equals nothing)
    c.mn = m4;
    c.imn = off + (b.x == m4 ? 0u : b.y == m4 ? 1u : b.z == m4 ? 2u : 3u);
  }
  if (x4 > c.mx) {
    c.mx = x4;
    c.imx = off + (b.x == x4 ? 0u : b.y == x4 ? 1u : b.z == x4 ? 2u : 3u);
  }
}

// Record of bin b of a staged series from its complete state (bin first point bstart,
// tile first point e0): only the indices matter to the compaction.
template <bool kNan>
__device__ __forceinline__ void emit_bin(const Batch& bt, const SeriesPlan& sp, int64_t b, const Part& c,
                                         int64_t bstart, int64_t e0) {
  Record r;
  r.kmin = key32(c.mn);
  r.kmax = key32(c.mx);
  r.imin = c.imn == kNone ? bstart : e0 + c.imn;
  r.imax = c.imx == kNone ? bstart : e0 + c.imx;
  if (kNan && c.inan != kNone) {
    r.kmin = LLONG_MIN;
    r.kmax = LLONG_MAX;
    r.imin = r.imax = e0 + c.inan;
  }
  bt.rec[sp.bin_off + b + sp.rec_w] = r;
}

// Bounds of index bin b: its first point, and the first point after it.
__device__ __forceinline__ int64_t ibin_start(const SeriesPlan& sp, int64_t b) {
  return sp.p0 + muldiv(b, sp.nb, sp.dB);
}
__device__ __forceinline__ int64_t ibin_end(const SeriesPlan& sp, int64_t b) {
  return b + 1 >= sp.B ? sp.p0 + sp.nb : sp.p0 + muldiv(b + 1, sp.nb, sp.dB);
}

// The bins of one staged float32 tile, read from shared memory: groups of G lanes
// (sp.group) take 32/G bins per round, bin bounds stepped from the series' constants
// (no division per bin).  Within a bin the G lanes read its whole 16-byte vectors in
// turn (consecutive lanes, consecutive vectors) with no range test; the group's first
// lane also takes the partial vectors at the bin's two ends, masked.  A butterfly over the
// group joins the lanes' Parts and the first lane writes the bin's record.
template <bool kNan>
__device__ void bulk_tile_f32(const Batch& bt, const SeriesPlan& sp, const TileWin& tw, uint32_t sdst, int lane) {
  const int G = sp.group, ngroups = 32 / G;
  const int grp = lane / G, gl = lane - grp * G;
  const int64_t e0 = tw.e0;
  const int64_t pbase = ((int64_t)tw.g0 - (int64_t)(uintptr_t)sp.y) / 4;  // point of the window's first float
  auto ld = [&](int64_t k) {
    float4 v;
    asm volatile("ld.shared.v4.f32 {%0,%1,%2,%3}, [%4];"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                 : "r"(sdst + 16u * (uint32_t)k));
    return v;
  };
  // bin mb = b0 + grp: lo = p0 + floor(mb*nb/B), rem = mb*nb mod B; later bins by
  // steps of one bin (q1, r1) and of 32/G bins (qs, rs)
  const int64_t mb0 = tw.b0 + grp;
  int64_t lo = ibin_start(sp, mb0);
  uint64_t rem = (uint64_t)mb0 * (uint64_t)sp.nb - (uint64_t)(lo - sp.p0) * (uint64_t)sp.B;
  const uint64_t Bu = (uint64_t)sp.B, r1 = (uint64_t)sp.bin_r1, rs = (uint64_t)sp.bin_rs;
  for (int64_t bb = tw.b0; bb < tw.b1; bb += ngroups) {
    const int64_t mb = bb + grp;
    const int64_t hi = lo + sp.bin_q1 + (rem + r1 >= Bu ? 1 : 0);  // start of bin mb + 1
    Part c;
    part_reset(c);
    const bool active = mb < tw.b1 && lo < hi;
    if (active) {
      const int64_t ka = (lo - pbase) >> 2, kb = (hi - 1 - pbase) >> 2;  // first and last vector
      const int64_t kf = (lo - pbase) & 3 ? ka + 1 : ka;                 // whole vectors [kf, kl)
      const int64_t kl = (hi - pbase) & 3 ? kb : kb + 1;
      // each lane takes its points in increasing order: the partial first vector,
      // the whole vectors, the partial last vector
      auto masked = [&](int64_t k) {
        const float4 v = ld(k);
        const float e[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int64_t p = pbase + 4 * k + j;
          if (p >= lo && p < hi) part_add<kNan>(c, e[j], (uint32_t)(p - e0));
        }
      };
      if (gl == 0 && kf != ka) masked(ka);
      int64_t k = kf + gl;
      for (; k + 3 * G < kl; k += 4 * G) {  // four reads in flight, then their reductions
        const float4 a0 = ld(k), a1 = ld(k + G), a2 = ld(k + 2 * G), a3 = ld(k + 3 * G);
        const uint32_t o = (uint32_t)(pbase + 4 * k - e0), og = 4u * (uint32_t)G;
        part_add4<kNan>(c, a0, o);
        part_add4<kNan>(c, a1, o + og);
        part_add4<kNan>(c, a2, o + 2 * og);
        part_add4<kNan>(c, a3, o + 3 * og);
      }
      for (; k < kl; k += G) part_add4<kNan>(c, ld(k), (uint32_t)(pbase + 4 * k - e0));
      if (gl == 0 && kl == kb && !(kf != ka && kb == ka)) masked(kb);
    }
    for (int d = 1; d < G; d <<= 1) {  // every lane takes part
      Part o;
      o.mn = __shfl_xor_sync(kFull, c.mn, d);
      o.mx = __shfl_xor_sync(kFull, c.mx, d);
      o.imn = __shfl_xor_sync(kFull, c.imn, d);
      o.imx = __shfl_xor_sync(kFull, c.imx, d);
      o.inan = __shfl_xor_sync(kFull, c.inan, d);
      part_merge(c, o);
    }
    if (active && gl == 0) emit_bin<kNan>(bt, sp, mb, c, lo, e0);
    // the next round: bin mb + 32/G
    lo += sp.bin_qs;
    rem += rs;
    if (rem >= Bu) {
      rem -= Bu;
      lo += 1;
    }
  }
}

// Staged-stream warp w: its tiles, each copied by one cp.async.bulk (lane 0 issues;
// an mbarrier per stage counts the bytes) into the next of its kBulkStages stages
// while the lanes reduce an earlier one, so that kBulkStages - 1 copies are in flight.
// Every wait is bounded: on a timeout the warp sets status bit 1, waits (bounded) for
// its copies still in flight and returns.
template <int kY>
__device__ void bulk_warp(const Batch& bt, int64_t w, int lane, uint32_t sbase, uint32_t bbase) {
  TileCursor cons;
  cons.init(bt, warp_begin(w, bt.total_tcost, bt.dbwarps), warp_begin(w + 1, bt.total_tcost, bt.dbwarps));
  if (cons.done) return;
  if (lane == 0) {
    for (int i = 0; i < kBulkStages; ++i) mbar_init(bbase + 8u * i, 1);
    fence_mbar_init();
  }
  __syncwarp();
  TileCursor prod = cons;
  auto issue = [&](int st) {
    if (lane == 0) {
      const TileWin pw = tile_window(plan_of(bt, prod.s), prod.t);
      const uint32_t bar = bbase + 8u * st;
      mbar_arrive_tx(bar, pw.bytes);
      if (pw.bytes) bulk_copy_g2s(sbase + (uint32_t)st * kBulkStageBytes, pw.g0, pw.bytes, bar);
    }
    prod.next(bt);
  };
  int inflight = 0;
  for (int i = 0; i < kBulkStages && !prod.done; ++i, ++inflight) issue(i);
  int st = 0;
  unsigned phase = 0;
  while (!cons.done) {
    if (!mbar_wait_bounded(bbase + 8u * st, phase)) {
      if (lane == 0) atomicOr(bt.status, 1u);
      for (int i = 1; i < inflight; ++i) {  // the copies issued after this stage
        const int s2 = (st + i) % kBulkStages;
        mbar_wait_bounded(bbase + 8u * s2, phase ^ (s2 < st ? 1u : 0u));
      }
      return;
    }
    const SeriesPlan& sp = plan_of(bt, cons.s);
    const TileWin tw = tile_window(sp, cons.t);
    const bool nan = kY == kYF32Nan || (kY == kYAny && sp.nan_aware);
    if (nan)
      bulk_tile_f32<true>(bt, sp, tw, sbase + (uint32_t)st * kBulkStageBytes, lane);
    else
      bulk_tile_f32<false>(bt, sp, tw, sbase + (uint32_t)st * kBulkStageBytes, lane);
    cons.next(bt);
    __syncwarp();
    --inflight;
    if (!prod.done) {
      if (lane == 0) fence_proxy_async();  // the lanes' reads of this stage before its refill
      issue(st);
      ++inflight;
    }
    if (++st == kBulkStages) {
      st = 0;
      phase ^= 1u;
    }
  }
}

// Bin edge e of the launch (all 32 lanes of a warp call it with the same e):
// S_b = first binned point with x >= e_b, e_b = x_0 + floor(b (x_{n-1} - x_0) / B)
// (R3, R16; FP64 edges on float64 x, R17); S_0 = p0, S_B = p0 + nb.  A 32-ary search:
// each round the lanes probe 32 equally spaced points and keep the interval that
// holds the first probe at or after the edge.
__device__ int64_t edge_at(const Batch& bt, int64_t e, int lane) {
  const int s = bt.edge_offs ? upper_index(bt.edge_offs, bt.n_series, e) : 0;
  const SeriesPlan& sp = plan_of(bt, s);
  const int64_t b = e - sp.edge_off;
  int64_t res;
  if (sp.nb < 1 || b == 0) {
    res = sp.p0;
  } else if (b >= sp.B) {
    res = sp.p0 + sp.nb;
  } else {
    // left edge e_b: int64 x exact (R3); float64 x with every operation rounded (R17)
    const bool fx = sp.xk == MMLTTB_X_F64;
    const long long* x = (const long long*)sp.x;
    const double* xd = (const double*)sp.x;
    long long eb = 0;
    double ebf = 0.0;
    if (fx) {
      const double x0 = __ldg(xd), D = __dsub_rn(__ldg(xd + sp.n - 1), x0);
      ebf = __dadd_rn(x0, __ddiv_rn(__dmul_rn((double)b, D), (double)sp.B));
    } else {
      const long long x0 = __ldg(x), xl = __ldg(x + sp.n - 1);
      eb = x0 + (long long)muldiv(b, xl - x0, sp.dB);
    }
    auto at_or_after = [&](int64_t q) { return fx ? __ldg(xd + q) >= ebf : __ldg(x + q) >= eb; };
    int64_t lo = sp.p0, hi = sp.p0 + sp.nb;  // answer in [lo, hi]
    while (hi - lo > 32) {
      const int64_t step = (hi - lo + 31) / 32;
      const int64_t q = lo + (int64_t)lane * step;
      const bool pred = q < hi && at_or_after(q);
      const unsigned m = __ballot_sync(kFull, pred);
      if (m == 0) {
        const int64_t last = lo + ((hi - lo - 1) / step) * step;  // last sampled point
        lo = last + 1;
      } else {
        const int f = __ffs(m) - 1;
        const int64_t qf = lo + (int64_t)f * step;
        lo = f > 0 ? qf - step + 1 : lo;
        hi = qf;
      }
    }
    const int64_t q = lo + lane;
    const bool pred = q < hi && at_or_after(q);
    const unsigned m = __ballot_sync(kFull, pred);
    res = m ? lo + (__ffs(m) - 1) : hi;
  }
  return res;
}

}  // namespace
}  // namespace mmlttb
