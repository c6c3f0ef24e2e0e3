// Device code of the compaction step (A-2) of MinMax preselection (Sec. 3): the
// records of each bin are combined, empty bins dropped, argmin == argmax emitted
// once (R9), and the survivors placed in order after the first point, with the last
// point appended: the preselected list [0, per-bin pairs..., n-1].  Shared by the
// split compaction kernels and the fused single-cluster kernel.
#pragma once

#include "stream.cuh"

namespace mmlttb {
namespace {

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

__device__ __forceinline__ int emit_count(int64_t lo, int64_t hi) {
  return lo < 0 ? 0 : (lo == hi ? 1 : 2);
}
// M4 emits the sorted distinct {first, lo, hi, last} (first <= lo <= hi <= last).
__device__ __forceinline__ int m4_count(int64_t first, int64_t lo, int64_t hi, int64_t last) {
  return lo < 0 ? 0 : 1 + (lo != first) + (hi != lo) + (last != hi);
}

// The y value (FP64) a record key stands for: keys are order-preserving images of the
// values (key32 / key64), so this inverts them, with -0.0 coming back as +0.0 (they
// compare equal, and every LTTB area takes an absolute value, so no pick changes).
__device__ __forceinline__ double value_of_key(const SeriesPlan& sp, long long k) {
  if (sp.ydt == MMLTTB_F32) {
    const int k32 = (int)k;
    const unsigned bits = k32 >= 0 ? (unsigned)k32 : ((0u - (unsigned)k32) | 0x80000000u);
    return (double)__uint_as_float(bits);
  }
  const unsigned long long bits =
      k >= 0 ? (unsigned long long)k : ((0ull - (unsigned long long)k) | 0x8000000000000000ull);
  return __longlong_as_double((long long)bits);
}

// Resolve bin b of series sp from its records (consecutive slots, one per warp that
// streamed part of it; one slot for a series of the staged stream): lo/hi = the lower
// and higher of (first argmin, first argmax) and klo/khi the record keys of their y
// values, first/last = the bin's first and last point; all -1 (keys 0) for an empty bin.
__device__ __forceinline__ void resolve_bin(const Batch& bt, const SeriesPlan& sp, int64_t b, int64_t* lo,
                                            int64_t* hi, long long* klo, long long* khi, int64_t* first,
                                            int64_t* last) {
  *lo = *hi = *first = *last = -1;
  *klo = *khi = 0;
  if (sp.nb <= 0 || b >= sp.B) return;
  const int64_t sb = bin_start(bt, sp, b);
  const int64_t sb1 = (b + 1 >= sp.B) ? sp.p0 + sp.nb : bin_start(bt, sp, b + 1);
  if (sb >= sb1) return;
  *first = sb;
  *last = sb1 - 1;
  Record r;
  if (sp.bulk_bpt > 0) {  // staged stream: one record per bin
    r = bt.rec[sp.bin_off + b + sp.rec_w];
  } else {
    const int64_t wf = warp_of(sp.pos_off + muldiv(sb - sp.p0, sp.npos, sp.dnb), bt.dtotal, bt.n_warps);
    const int64_t wl = warp_of(sp.pos_off + muldiv(sb1 - 1 - sp.p0, sp.npos, sp.dnb), bt.dtotal, bt.n_warps);
    const Record* rb = bt.rec + sp.bin_off + b;
    r = rb[wf];
    for (int64_t w = wf + 1; w <= wl; ++w) combine(r, rb[w]);
  }
  const bool min_first = r.imin < r.imax;
  *lo = min_first ? r.imin : r.imax;
  *hi = min_first ? r.imax : r.imin;
  *klo = min_first ? r.kmin : r.kmax;
  *khi = min_first ? r.kmax : r.kmin;
}

// Indices bin b of series sp contributes to the list: MinMax (lo, hi) deduplicated
// (R9), or M4's sorted distinct {first, lo, hi, last} (R16).
__device__ __forceinline__ int bin_count(const SeriesPlan& sp, int64_t lo, int64_t hi,
                                         int64_t first, int64_t last) {
  return sp.branch == BR_M4 ? m4_count(first, lo, hi, last) : emit_count(lo, hi);
}

// Write bin b's indices at list offset o (the exclusive prefix of the counts of the
// bins before it); MinMax lists start after the first point and carry FP64 copies of
// x and y for LTTB, y from the record keys klo/khi (no gather of y).
__device__ __forceinline__ void place_bin(const SeriesPlan& sp, int64_t lo, int64_t hi, long long klo,
                                          long long khi, int64_t first, int64_t last, int cnt, int64_t o) {
  if (cnt == 0) return;
  if (sp.branch == BR_M4) {
    sp.sel[o++] = first;
    if (lo != first) sp.sel[o++] = lo;
    if (hi != lo) sp.sel[o++] = hi;
    if (last != hi) sp.sel[o++] = last;
    return;
  }
  if (sp.n <= 2) return;
  const int64_t pos = 1 + o;
  sp.sel[pos] = lo;
  if (cnt == 2) sp.sel[pos + 1] = hi;
  if (sp.px) {
    sp.px[pos] = x_of(sp, lo);
    sp.py[pos] = value_of_key(sp, klo);
    if (cnt == 2) {
      sp.px[pos + 1] = x_of(sp, hi);
      sp.py[pos + 1] = value_of_key(sp, khi);
    }
  }
}

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

}  // namespace
}  // namespace mmlttb
