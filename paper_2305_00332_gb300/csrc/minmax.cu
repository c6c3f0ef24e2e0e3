// MinMax preselection kernels (Sec. 3 first step; MinMax of Sec. 2.2.1, Table 1).
//
//  k_edges   x-width bins: one warp per bin edge, 32-ary search for the first
//            interior point with x >= e_b (x is non-decreasing).
//  k_stream  the HBM-bound pass.  The interior points of every series are laid end
//            to end in one global position space, cut into W equal ranges, one per
//            warp.  A warp walks the bins that meet its range; for each piece it
//            streams y with 16-byte coalesced loads (4 in flight per lane) and keeps
//            a per-lane first-occurrence argmin/argmax, then reduces across the warp
//            and writes one Record at slot (global bin + warp).  x is never streamed:
//            bin bounds come from integer arithmetic (index bins) or from k_edges.
//  k_bins / k_binscan / k_place   compaction: combine each bin's records (they sit
//            in consecutive slots), drop empty bins, dedupe argmin == argmax and place
//            [0, per-bin pairs..., n-1] with a scan restarted at every series.
#include "common.cuh"

namespace mmlttb {

namespace {

constexpr unsigned kFull = 0xffffffffu;
// Stream-kernel variants the autotuner chooses from: 16-byte vectors in flight per
// lane (U) and resident CTAs per SM the register budget is set for (MINB).
template <int U, int MINB>
struct StreamCfg {
  static constexpr int kUnroll = U;
  static constexpr int kMinBlocks = MINB;
};

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
  if (sp.binmode == MMLTTB_BINS_INDEX) return sp.p0 + muldiv(b, sp.nb, sp.B);
  return bt.edges[sp.edge_off + b];
}
__device__ __forceinline__ int64_t bin_containing(const Batch& bt, const SeriesPlan& sp, int64_t p) {
  if (sp.binmode == MMLTTB_BINS_INDEX) return part_of(p - sp.p0 + 1, sp.nb, sp.B);
  return upper_index(bt.edges + sp.edge_off, (int)sp.B, p);
}

// First-occurrence argmin/argmax of y[lo, hi) for float32 y by one group of G lanes
// (gl = lane within the group, gmask = the group's lanes; G = 32: the whole warp).
// kNanAware: NaN-aware mode (R18): a bin holding a NaN reports its first NaN as both
// extremes; its record carries the keys LLONG_MIN / LLONG_MAX, which no value has,
// so merging records keeps the first NaN of the bin.
template <int kUnroll, bool kNanAware>
__device__ Record segment_f32(const float* y, int64_t lo, int64_t hi, int gl, int G, unsigned gmask) {
  const uint32_t len = (uint32_t)(hi - lo);
  const float inf = __int_as_float(0x7f800000);
  // Empty state: only strictly smaller (larger) values are recorded, so a lane that
  // sees nothing but +inf (-inf) keeps offset ~0u; if every lane does, the extreme is
  // the first point (offset 0).
  float mn = inf, mx = -inf;
  uint32_t omn = 0xffffffffu, omx = 0xffffffffu, onan = 0xffffffffu;
  const uintptr_t ybase = (uintptr_t)y;
  const uintptr_t a0 = (ybase + (uintptr_t)lo * 4u) & ~(uintptr_t)15;
  const uintptr_t aend = ybase + (uintptr_t)hi * 4u;
  const int64_t nvec = hi > lo ? (int64_t)((aend - a0 + 15u) >> 4) : 0;
  const int32_t rel0 = (int32_t)(((int64_t)a0 - (int64_t)ybase) / 4 - lo);  // in [-3, 0]
  const float4* vp = (const float4*)a0;
  for (int64_t v = gl; v < nvec; v += G * kUnroll) {
    float4 buf[kUnroll];
#pragma unroll
    for (int u = 0; u < kUnroll; u++) {
      int64_t vi = v + G * u;
      if (vi < nvec) buf[u] = ld_stream4(vp + vi);
    }
#pragma unroll
    for (int u = 0; u < kUnroll; u++) {
      int64_t vi = v + G * u;
      if (vi < nvec) {
        const int32_t r = rel0 + 4 * (int32_t)vi;
        const float e[4] = {buf[u].x, buf[u].y, buf[u].z, buf[u].w};
        float fm[4], fx[4];
#pragma unroll
        for (int k = 0; k < 4; k++) {
          const bool ok = (uint32_t)(r + k) < len;
          fm[k] = ok ? e[k] : inf;
          fx[k] = ok ? e[k] : -inf;
        }
        if (kNanAware && onan == 0xffffffffu) {
          const bool any = (e[0] != e[0]) | (e[1] != e[1]) | (e[2] != e[2]) | (e[3] != e[3]);
          if (any) {
#pragma unroll
            for (int k = 3; k >= 0; k--)  // lowest valid NaN of the vector
              if ((uint32_t)(r + k) < len && e[k] != e[k]) onan = (uint32_t)(r + k);
          }
        }
        const float m4 = fminf(fminf(fm[0], fm[1]), fminf(fm[2], fm[3]));
        const float x4 = fmaxf(fmaxf(fx[0], fx[1]), fmaxf(fx[2], fx[3]));
        if (m4 < mn) {  // rare: some element is a new strict minimum
#pragma unroll
          for (int k = 0; k < 4; k++)
            if (fm[k] < mn) { mn = fm[k]; omn = (uint32_t)(r + k); }
        }
        if (x4 > mx) {
#pragma unroll
          for (int k = 0; k < 4; k++)
            if (fx[k] > mx) { mx = fx[k]; omx = (uint32_t)(r + k); }
        }
      }
    }
  }
  const int kmn = key32(mn), kmx = key32(mx);
  const int wmn = __reduce_min_sync(gmask, kmn);
  const unsigned wo = __reduce_min_sync(gmask, kmn == wmn ? omn : 0xffffffffu);
  const int wmx = __reduce_max_sync(gmask, kmx);
  const unsigned wx = __reduce_min_sync(gmask, kmx == wmx ? omx : 0xffffffffu);
  Record r;
  r.kmin = wmn;
  r.kmax = wmx;
  r.imin = lo + (int64_t)(wo == 0xffffffffu ? 0u : wo);
  r.imax = lo + (int64_t)(wx == 0xffffffffu ? 0u : wx);
  if (kNanAware) {
    const unsigned wn = __reduce_min_sync(gmask, onan);
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
template <int kUnroll, bool kNanAware>
__device__ Record segment_f64(const double* y, int64_t lo, int64_t hi, int gl, int G, unsigned gmask) {
  const uint32_t len = (uint32_t)(hi - lo);
  // Empty state: keys beyond every double's key and NaN proxies, so the first
  // element a lane sees takes the exact path and is recorded.
  long long kmn = LLONG_MAX, kmx = LLONG_MIN;
  float pmn = __int_as_float(0x7fc00000), pmx = pmn;
  uint32_t omn = 0xffffffffu, omx = 0xffffffffu, onan = 0xffffffffu;
  const uintptr_t ybase = (uintptr_t)y;
  const uintptr_t a0 = (ybase + (uintptr_t)lo * 8u) & ~(uintptr_t)15;
  const uintptr_t aend = ybase + (uintptr_t)hi * 8u;
  const int64_t nvec = hi > lo ? (int64_t)((aend - a0 + 15u) >> 4) : 0;
  const int32_t rel0 = (int32_t)(((int64_t)a0 - (int64_t)ybase) / 8 - lo);  // in [-1, 0]
  const float inf = __int_as_float(0x7f800000);
  for (int64_t v = gl; v < nvec; v += G * kUnroll) {
    uint4 buf[kUnroll];
#pragma unroll
    for (int u = 0; u < kUnroll; u++) {
      int64_t vi = v + G * u;
      if (vi < nvec) buf[u] = ld_stream4u((const void*)(a0 + (uintptr_t)vi * 16u));
    }
#pragma unroll
    for (int u = 0; u < kUnroll; u++) {
      int64_t vi = v + G * u;
      if (vi < nvec) {
        const int32_t r = rel0 + 2 * (int32_t)vi;
        const bool ok0 = (uint32_t)r < len, ok1 = (uint32_t)(r + 1) < len;
        const float p0 = proxy_of_hi(buf[u].y), p1 = proxy_of_hi(buf[u].w);
        const float pm = fmin_nan(ok0 ? p0 : inf, ok1 ? p1 : inf);
        const float px = fmax_nan(ok0 ? p0 : -inf, ok1 ? p1 : -inf);
        const bool need_min = !(pm > pmn);
        const bool need_max = !(px < pmx);
        if (need_min || need_max) {  // rare: exact comparison through int64 keys
          const long long e0 = ((long long)buf[u].y << 32) | buf[u].x;
          const long long e1 = ((long long)buf[u].w << 32) | buf[u].z;
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
      }
    }
  }
  // int64 order = (signed high word, unsigned low word)
  const int hmn = (int)(kmn >> 32);
  const unsigned lmn = (unsigned)kmn;
  const int whm = __reduce_min_sync(gmask, hmn);
  const unsigned wlm = __reduce_min_sync(gmask, hmn == whm ? lmn : 0xffffffffu);
  const bool eqm = (hmn == whm) && (lmn == wlm);
  const unsigned wo = __reduce_min_sync(gmask, eqm ? omn : 0xffffffffu);
  const int hmx = (int)(kmx >> 32);
  const unsigned lmx = (unsigned)kmx;
  const int whx = __reduce_max_sync(gmask, hmx);
  const unsigned wlx = __reduce_max_sync(gmask, hmx == whx ? lmx : 0u);
  const bool eqx = (hmx == whx) && (lmx == wlx);
  const unsigned wx = __reduce_min_sync(gmask, eqx ? omx : 0xffffffffu);
  Record r;
  r.kmin = ((long long)whm << 32) | wlm;
  r.kmax = ((long long)whx << 32) | wlx;
  r.imin = lo + (int64_t)(wo == 0xffffffffu ? 0u : wo);
  r.imax = lo + (int64_t)(wx == 0xffffffffu ? 0u : wx);
  if (kNanAware) {
    const unsigned wn = __reduce_min_sync(gmask, onan);
    if (wn != 0xffffffffu) {
      r.kmin = LLONG_MIN;
      r.kmax = LLONG_MAX;
      r.imin = r.imax = lo + (int64_t)wn;
    }
  }
  return r;
}

// Smallest interior point q in [0, N] whose work unit floor(q*D/N) is >= t, for
// 0 <= t <= D: ceil(t*N/D).
__device__ __forceinline__ int64_t point_at_work(int64_t t, int64_t N, int64_t D) {
  return muldiv_ceil(t, N, D);
}

// One warp over the binned points [p_lo, p_hi) of one series.  The warp splits into
// 32/G groups of G lanes (G chosen per series from its mean bin size) and each group
// works on its own bin, so small bins are processed 32/G at a time.
template <int kUnroll>
__device__ void warp_series_range(const Batch& bt, const SeriesPlan& sp, int64_t p_lo,
                                  int64_t p_hi, int64_t w, int lane) {
  const int G = sp.group;
  const int ngroups = 32 / G;
  const int grp = lane / G, gl = lane - grp * G;
  const unsigned gmask = G == 32 ? kFull : (((1u << G) - 1u) << (grp * G));
  int64_t b = bin_containing(bt, sp, p_lo);
  for (;;) {
    const int64_t mb = b + grp;
    int64_t lo = p_hi, hi = p_hi, sb1 = sp.p0 + sp.nb;
    if (mb < sp.B) {
      const int64_t sb = bin_start(bt, sp, mb);
      sb1 = (mb + 1 >= sp.B) ? sp.p0 + sp.nb : bin_start(bt, sp, mb + 1);
      lo = sb > p_lo ? sb : p_lo;
      hi = sb1 < p_hi ? sb1 : p_hi;
    }
    if (lo < hi) {
      Record r;
      if (sp.nan_aware)
        r = (sp.ydt == MMLTTB_F32) ? segment_f32<kUnroll, true>((const float*)sp.y, lo, hi, gl, G, gmask)
                                   : segment_f64<kUnroll, true>((const double*)sp.y, lo, hi, gl, G, gmask);
      else
        r = (sp.ydt == MMLTTB_F32) ? segment_f32<kUnroll, false>((const float*)sp.y, lo, hi, gl, G, gmask)
                                   : segment_f64<kUnroll, false>((const double*)sp.y, lo, hi, gl, G, gmask);
      if (gl == 0) bt.rec[sp.bin_off + mb + w] = r;
    }
    // the round ends with bin b + ngroups - 1 (held by the last group)
    const int64_t last_end = __shfl_sync(kFull, sb1, 31);
    if (last_end >= p_hi || b + ngroups >= sp.B) break;
    b += ngroups;
  }
}

template <int U, int MINB>
__global__ void __launch_bounds__(kStreamThreads, MINB) k_stream(const __grid_constant__ Batch bt) {
  pdl_wait();
  pdl_trigger();
  const int lane = threadIdx.x & 31;
  const int64_t w = (int64_t)blockIdx.x * kStreamWarps + (threadIdx.x >> 5);
  if (w >= bt.n_warps) return;
  int64_t g = warp_begin(w, bt.total_pos, bt.n_warps);
  const int64_t g_end = warp_begin(w + 1, bt.total_pos, bt.n_warps);
  int s = bt.pos_offs ? upper_index(bt.pos_offs, bt.n_series, g) : 0;
  while (g < g_end && s < bt.n_series) {
    const SeriesPlan& sp = plan_of(bt, s);
    const int64_t send = sp.pos_off + sp.npos;
    const int64_t seg_end = send < g_end ? send : g_end;
    if (seg_end > g) {
      // binned points whose work unit lies in [g, seg_end): p0 + q, q in [q_lo, q_hi)
      const int64_t q_lo = point_at_work(g - sp.pos_off, sp.nb, sp.npos);
      const int64_t q_hi = point_at_work(seg_end - sp.pos_off, sp.nb, sp.npos);
      if (q_hi > q_lo) warp_series_range<U>(bt, sp, sp.p0 + q_lo, sp.p0 + q_hi, w, lane);
      g = seg_end;
    }
    ++s;
  }
}

// One warp per bin edge of every x-width series: S_b = first binned point with
// x >= e_b, e_b = x_0 + floor(b (x_{n-1} - x_0) / B) (R3, R16); S_0 = p0, S_B = p0 + nb.
__global__ void __launch_bounds__(256) k_edges(const __grid_constant__ Batch bt) {
  pdl_wait();
  pdl_trigger();
  const int lane = threadIdx.x & 31;
  const int64_t e = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (e >= bt.total_edges) return;
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
      eb = x0 + (long long)muldiv(b, xl - x0, sp.B);
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
  if (lane == 0) bt.edges[e] = res;
}

__device__ __forceinline__ void combine(Record& a, const Record& b) {
  if (b.kmin < a.kmin || (b.kmin == a.kmin && b.imin < a.imin)) { a.kmin = b.kmin; a.imin = b.imin; }
  if (b.kmax > a.kmax || (b.kmax == a.kmax && b.imax < a.imax)) { a.kmax = b.kmax; a.imax = b.imax; }
}

// Exclusive block scan of small non-negative counts; returns the block total.
template <int NT>
__device__ int block_excl_scan(int v, int* excl) {
  __shared__ int wsum[NT / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int inc = v;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    int t = __shfl_up_sync(kFull, inc, d);
    if (lane >= d) inc += t;
  }
  if (lane == 31) wsum[wid] = inc;
  __syncthreads();
  if (wid == 0) {
    int t = lane < NT / 32 ? wsum[lane] : 0;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      int u = __shfl_up_sync(kFull, t, d);
      if (lane >= d) t += u;
    }
    if (lane < NT / 32) wsum[lane] = t;  // inclusive warp prefix
  }
  __syncthreads();
  const int before = wid > 0 ? wsum[wid - 1] : 0;
  const int total = wsum[NT / 32 - 1];
  *excl = before + inc - v;
  __syncthreads();
  return total;
}

// ---- compaction (A-2): three grid-wide kernels --------------------------------
// Every series' bins are laid out from a CTA boundary (kBinsPerCta bins per CTA).
//   k_bins     one thread per bin: combine the bin's records (consecutive slots)
//              into (lower, higher) of argmin/argmax, -1 for an empty bin; each CTA
//              writes how many indices its bins emit.
//   k_binscan  one CTA: exclusive scan of the CTA totals, restarted at every
//              series; the last CTA of a series fixes its count m and the first
//              and last entries of its preselected list.
//   k_place    one thread per bin: block scan + CTA offset place the bin's indices
//              (and, before LTTB, their x and y as FP64) in the preselected list.

__device__ __forceinline__ int emit_count(int64_t lo, int64_t hi) {
  return lo < 0 ? 0 : (lo == hi ? 1 : 2);
}
// M4 emits the sorted distinct {first, lo, hi, last} (first <= lo <= hi <= last).
__device__ __forceinline__ int m4_count(int64_t first, int64_t lo, int64_t hi, int64_t last) {
  return lo < 0 ? 0 : 1 + (lo != first) + (hi != lo) + (last != hi);
}

__global__ void __launch_bounds__(kBinsPerCta) k_bins(const __grid_constant__ Batch bt) {
  __shared__ int s_series;
  pdl_wait();
  pdl_trigger();
  const int64_t c = blockIdx.x;
  if (threadIdx.x == 0) s_series = bt.cta_offs ? upper_index(bt.cta_offs, bt.n_series, c) : 0;
  __syncthreads();
  const SeriesPlan& sp = plan_of(bt, s_series);
  const int64_t b = (c - sp.bincta_off) * kBinsPerCta + threadIdx.x;
  int64_t lo = -1, hi = -1, first = -1, last = -1;
  if (sp.nb > 0 && b < sp.B) {
    const int64_t sb = bin_start(bt, sp, b);
    const int64_t sb1 = (b + 1 >= sp.B) ? sp.p0 + sp.nb : bin_start(bt, sp, b + 1);
    if (sb < sb1) {
      first = sb;
      last = sb1 - 1;
      const int64_t wf = warp_of(sp.pos_off + muldiv(sb - sp.p0, sp.npos, sp.nb), bt.total_pos, bt.n_warps);
      const int64_t wl = warp_of(sp.pos_off + muldiv(sb1 - 1 - sp.p0, sp.npos, sp.nb), bt.total_pos, bt.n_warps);
      const Record* rb = bt.rec + sp.bin_off + b;
      Record r = rb[wf];
      for (int64_t w = wf + 1; w <= wl; ++w) combine(r, rb[w]);
      lo = r.imin < r.imax ? r.imin : r.imax;
      hi = r.imin < r.imax ? r.imax : r.imin;
    }
  }
  const int64_t slot = c * kBinsPerCta + threadIdx.x;
  bt.binres[2 * slot] = lo;
  bt.binres[2 * slot + 1] = hi;
  int cnt = sp.branch == BR_M4 ? m4_count(first, lo, hi, last) : emit_count(lo, hi);
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) cnt += __shfl_xor_sync(kFull, cnt, d);
  __shared__ int s_warp[kBinsPerCta / 32];
  if ((threadIdx.x & 31) == 0) s_warp[threadIdx.x >> 5] = cnt;
  __syncthreads();
  if (threadIdx.x == 0) {
    int t = 0;
#pragma unroll
    for (int w = 0; w < kBinsPerCta / 32; ++w) t += s_warp[w];
    bt.cta_sum[c] = t;
    bt.cta_series[c] = s_series;
  }
}

constexpr int kScanThreads = 1024;

// Write the list head/tail of series s once its count m is known.
__device__ void finish_series(const SeriesPlan& sp, int64_t emitted) {
  int64_t* P = sp.sel;
  const int64_t n = sp.n;
  int64_t m;
  if (sp.branch == BR_M4) {  // M4 keeps no extra points
    m = emitted;
  } else if (n <= 2) {  // no interior points: [0] or [0, 1]
    m = n;
    for (int64_t i = 0; i < n; ++i) P[i] = i;
  } else {
    m = emitted + 2;
    P[0] = 0;
    P[m - 1] = n - 1;
  }
  if (sp.px && m > 0) {
    sp.px[0] = x_of(sp, 0);
    sp.py[0] = y_of(sp, 0);
    sp.px[m - 1] = x_of(sp, n - 1);
    sp.py[m - 1] = y_of(sp, n - 1);
  }
  *sp.m_ptr = m;
  if ((sp.branch == BR_PRESELECT || sp.branch == BR_M4) && sp.out_count) *sp.out_count = m;
}

__global__ void __launch_bounds__(kScanThreads) k_binscan(const __grid_constant__ Batch bt) {
  __shared__ int64_t s_inc[kScanThreads];
  __shared__ int s_head[kScanThreads];
  pdl_wait();
  pdl_trigger();
  const int tid = threadIdx.x;
  const int64_t total = bt.total_bin_ctas;
  int64_t carry = 0;  // running sum of the segment that continues into the next tile
  for (int64_t tile = 0; tile < total; tile += kScanThreads) {
    const int64_t c = tile + tid;
    const bool valid = c < total;
    const int s = valid ? bt.cta_series[c] : -1;
    const int64_t v = valid ? bt.cta_sum[c] : 0;
    const bool head = valid && (c == 0 || bt.cta_series[c - 1] != s);
    s_inc[tid] = v;
    s_head[tid] = head ? tid : -1;
    __syncthreads();
    // Hillis-Steele inclusive sum and max-scan of segment heads over the tile
    for (int d = 1; d < kScanThreads; d <<= 1) {
      const int64_t a = tid >= d ? s_inc[tid - d] : 0;
      const int h = tid >= d ? s_head[tid - d] : -1;
      __syncthreads();
      s_inc[tid] += a;
      if (h > s_head[tid]) s_head[tid] = h;
      __syncthreads();
    }
    const int start = s_head[tid];  // this element's segment start in the tile, or -1
    int64_t excl = s_inc[tid] - v;
    if (start >= 0) excl -= start > 0 ? s_inc[start - 1] : 0;
    else excl += carry;
    const int last = (int)((total - tile < kScanThreads ? total - tile : kScanThreads) - 1);
    const int last_start = s_head[last];
    const int64_t new_carry = last_start >= 0
                                  ? s_inc[last] - (last_start > 0 ? s_inc[last_start - 1] : 0)
                                  : carry + s_inc[last];
    if (valid) {
      bt.cta_off[c] = excl;
      const bool tail = c + 1 == total || bt.cta_series[c + 1] != s;
      if (tail) finish_series(plan_of(bt, s), excl + v);
    }
    __syncthreads();
    carry = new_carry;
  }
}

__global__ void __launch_bounds__(kBinsPerCta) k_place(const __grid_constant__ Batch bt) {
  pdl_wait();
  pdl_trigger();
  const int64_t c = blockIdx.x;
  const int s = bt.cta_series[c];
  const SeriesPlan& sp = plan_of(bt, s);
  const int64_t slot = c * kBinsPerCta + threadIdx.x;
  const int64_t lo = bt.binres[2 * slot], hi = bt.binres[2 * slot + 1];
  const bool m4 = sp.branch == BR_M4;
  int64_t first = -1, last = -1;
  if (m4 && lo >= 0) {
    const int64_t b = (c - sp.bincta_off) * kBinsPerCta + threadIdx.x;
    first = bin_start(bt, sp, b);
    last = ((b + 1 >= sp.B) ? sp.p0 + sp.nb : bin_start(bt, sp, b + 1)) - 1;
  }
  const int cnt = m4 ? m4_count(first, lo, hi, last) : emit_count(lo, hi);
  int excl;
  block_excl_scan<kBinsPerCta>(cnt, &excl);
  if (cnt == 0 || (!m4 && sp.n <= 2)) return;
  if (m4) {
    int64_t o = bt.cta_off[c] + excl;
    sp.sel[o++] = first;
    if (lo != first) sp.sel[o++] = lo;
    if (hi != lo) sp.sel[o++] = hi;
    if (last != hi) sp.sel[o++] = last;
    return;
  }
  const int64_t pos = 1 + bt.cta_off[c] + excl;
  sp.sel[pos] = lo;
  if (cnt == 2) sp.sel[pos + 1] = hi;
  if (sp.px) {
    sp.px[pos] = x_of(sp, lo);
    sp.py[pos] = y_of(sp, lo);
    if (cnt == 2) {
      sp.px[pos + 1] = x_of(sp, hi);
      sp.py[pos + 1] = y_of(sp, hi);
    }
  }
}

}  // namespace

// The compiled variants: (U, MINB) = (4, 4), (8, 3), (2, 6).
static const void* stream_kernel(int v) {
  switch (v) {
    case 1: return (const void*)k_stream<8, 3>;
    case 2: return (const void*)k_stream<2, 6>;
    default: return (const void*)k_stream<4, 4>;
  }
}

int stream_variant_info(int v, int* unroll, int* min_blocks) {
  static const int U[kStreamVariants] = {4, 8, 2}, M[kStreamVariants] = {4, 3, 6};
  if (v < 0 || v >= kStreamVariants) return -1;
  *unroll = U[v];
  *min_blocks = M[v];
  return 0;
}

int stream_blocks_per_sm(int v) {
  int bps = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, stream_kernel(v), kStreamThreads, 0) !=
      cudaSuccess)
    return 1;
  return bps > 0 ? bps : 1;
}

cudaError_t launch_edges(const Batch& bt, cudaStream_t st) {
  if (bt.total_edges <= 0) return cudaSuccess;
  const int64_t threads = bt.total_edges * 32;
  const int64_t grid = (threads + 255) / 256;
  return launch_pdl(k_edges, dim3((unsigned)grid), dim3(256), 0, st, bt);
}

cudaError_t launch_stream(const Batch& bt, int64_t grid, int variant, cudaStream_t st) {
  if (bt.n_warps <= 0) return cudaSuccess;
  const dim3 g((unsigned)grid), b(kStreamThreads);
  switch (variant) {
    case 1: return launch_pdl(k_stream<8, 3>, g, b, 0, st, bt);
    case 2: return launch_pdl(k_stream<2, 6>, g, b, 0, st, bt);
    default: return launch_pdl(k_stream<4, 4>, g, b, 0, st, bt);
  }
}

cudaError_t launch_compact(const Batch& bt, cudaStream_t st) {
  if (bt.total_bin_ctas <= 0) return cudaSuccess;
  const dim3 grid((unsigned)bt.total_bin_ctas);
  cudaError_t e = launch_pdl(k_bins, grid, dim3(kBinsPerCta), 0, st, bt);
  if (e != cudaSuccess) return e;
  e = launch_pdl(k_binscan, dim3(1), dim3(kScanThreads), 0, st, bt);
  if (e != cudaSuccess) return e;
  return launch_pdl(k_place, grid, dim3(kBinsPerCta), 0, st, bt);
}

}  // namespace mmlttb
