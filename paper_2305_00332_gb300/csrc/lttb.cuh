// Device code of the LTTB step (Sec. 2.2.1 LTTB; Sec. 3 second step of MinMaxLTTB)
// on small buckets, shared by the split kernels (k_tables, k_chain) and the fused
// single-cluster kernel.
//
// LTTB is a chain: the pick b_j of bucket j depends on the pick of bucket j-1.  When
// buckets are small (MinMaxLTTB puts about r_ps points in each), the chain is cut
// into independent pieces:
//   bucket_pick    every position p that can be the previous pick of bucket j (p in
//                  bucket j-1, or p = 0 for j = 0) gets T[p] = the offset in bucket j
//                  of the point with the largest area against p and the mean of
//                  bucket j+1.  Each area is the same FP64 expression the sequential
//                  method evaluates, so every entry equals the sequential choice for p.
//   chain_series   one CTA resolves b_j = T[L_{j-1} + b_{j-1}] for all j by a
//                  parallel prefix over function composition (Hillis-Steele), then
//                  writes the picked indices.
#pragma once

#include "area_filter.cuh"
#include "common.cuh"

namespace mmlttb {
namespace {

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Grid-wide barrier on a monotone counter with a 2 s bound.  Returns false (and
// sets status bit 1) when the other CTAs did not all arrive in time.
__device__ bool grid_barrier(unsigned* ctr, unsigned target, unsigned* status) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(ctr, 1u);
    ok = 1;
    const unsigned long long t0 = global_ns();
    while (ld_acquire(ctr) < target) {
      if (global_ns() - t0 > 2000000000ull) {
        set_status(status, 1u);
        ok = 0;
        break;
      }
    }
    __threadfence();
  }
  __syncthreads();
  return ok != 0;
}

__device__ __forceinline__ int64_t lttb_m(const SeriesPlan& sp) {
  return sp.branch == BR_LTTB_ALL ? sp.n : *sp.m_ptr;
}

// Mean of LTTB positions [lo, hi): left-to-right FP64 sums, one division each (R7).
__device__ void bucket_mean(const SeriesPlan& sp, int64_t lo, int64_t hi, double* xc, double* yc) {
  double sx = 0.0, sy = 0.0;
  if (sp.xk == MMLTTB_X_IMPLICIT && !sp.sel && hi > 0 && hi - lo <= ((1ll << 53) - 1) / hi) {
    // Implicit x on all points: the indices lo..hi-1 and all their partial sums are
    // integers below 2^53, so the sequential FP64 sum is exact and equals the
    // closed form.
    sx = (double)((lo + hi - 1) * (hi - lo) / 2);
    for (int64_t p = lo; p < hi; ++p) sy = __dadd_rn(sy, y_of(sp, p));
  } else if (hi - lo > 8) {
    for (int64_t p = lo; p < hi; ++p) {
      double xp, yp;
      pos_xy(sp, p, &xp, &yp);
      sx = __dadd_rn(sx, xp);
      sy = __dadd_rn(sy, yp);
    }
  } else {
    // a small bucket (after preselection): its loads in flight together, then the
    // sums in order (left to right)
    double xv[8], yv[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      xv[u] = yv[u] = 0.0;
      if (lo + u < hi) pos_xy(sp, lo + u, &xv[u], &yv[u]);
    }
#pragma unroll
    for (int u = 0; u < 8; ++u)
      if (lo + u < hi) {
        sx = __dadd_rn(sx, xv[u]);
        sy = __dadd_rn(sy, yv[u]);
      }
  }
  const double cnt = (double)(hi - lo);
  *xc = __ddiv_rn(sx, cnt);
  *yc = __ddiv_rn(sy, cnt);
}

// Exponent bookkeeping for exact sums.  A finite double v != 0 is a multiple of
// 2^g(v) (g = the weight of its lowest set significand bit) and below 2^(e(v)+1) in
// magnitude (e = its unbiased exponent).  If every term of a sum is a multiple of 2^G
// and n * 2^(E+1) <= 2^(53+G) (G, E the smallest g and largest e), every partial sum
// in ANY order is a multiple of 2^G below 2^(53+G): representable, so no addition
// rounds and all orders give the same, exact sum -- the left-to-right FP64 sum of R7.
struct ExactSum {
  int gmin = INT_MAX, emax = INT_MIN;
  bool bad = false;  // inf or NaN seen
  __device__ void add(double v) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    const int be = (int)((b >> 52) & 0x7ff);
    const unsigned long long m = b & 0xfffffffffffffull;
    if (be == 0x7ff) {
      bad = true;
    } else if (be != 0 || m != 0) {
      const unsigned long long sig = be ? (m | (1ull << 52)) : m;  // value = sig * 2^(max(be,1) - 1075)
      const int scale = (be ? be : 1) - 1075;
      const int g = scale + __ffsll((long long)sig) - 1;
      const int e = scale + 63 - __clzll((long long)sig);
      gmin = g < gmin ? g : gmin;
      emax = e > emax ? e : emax;
    }
  }
  // warp-wide: whether a sum of n terms is exact in any order (every lane gets it)
  __device__ bool exact(int64_t n) {
    const int g = __reduce_min_sync(kFull, gmin), e = __reduce_max_sync(kFull, emax);
    const bool anybad = __any_sync(kFull, bad);
    if (anybad) return false;
    if (g == INT_MAX) return true;  // all terms zero
    const int lg = 64 - __clzll((long long)(n > 1 ? n - 1 : 1));  // ceil(log2 n)
    return lg + e + 1 <= 53 + g;
  }
};

__device__ __forceinline__ double warp_sum_f64(double v) {
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) v = __dadd_rn(v, __shfl_xor_sync(kFull, v, d));
  return v;
}

// Mean of LTTB positions [lo, hi) formed by a whole warp (all lanes call it): when the
// bucket's sums are exact in any order (ExactSum) the lanes add strided terms and the
// warp combines them, which equals the left-to-right sums of R7 bit for bit; otherwise
// lane 0 forms the sequential sums.  One IEEE division each.  Results in every lane.
__device__ void bucket_mean_warp(const SeriesPlan& sp, int64_t lo, int64_t hi, int lane, double* xc, double* yc) {
  const bool xclosed = sp.xk == MMLTTB_X_IMPLICIT && !sp.sel && hi > 0 && hi - lo <= ((1ll << 53) - 1) / hi;
  double sx = 0.0, sy = 0.0;
  ExactSum ex, ey;
  for (int64_t p = lo + lane; p < hi; p += 32) {
    double xp, yp;
    pos_xy(sp, p, &xp, &yp);
    if (!xclosed) {
      ex.add(xp);
      sx = __dadd_rn(sx, xp);
    }
    ey.add(yp);
    sy = __dadd_rn(sy, yp);
  }
  const bool fast = (xclosed || ex.exact(hi - lo)) && ey.exact(hi - lo);
  if (fast) {
    sy = warp_sum_f64(sy);
    sx = xclosed ? (double)((lo + hi - 1) * (hi - lo) / 2) : warp_sum_f64(sx);
    const double cnt = (double)(hi - lo);
    *xc = __ddiv_rn(sx, cnt);
    *yc = __ddiv_rn(sy, cnt);
    return;
  }
  double a = 0.0, b = 0.0;
  if (lane == 0) bucket_mean(sp, lo, hi, &a, &b);
  *xc = __shfl_sync(kFull, a, 0);
  *yc = __shfl_sync(kFull, b, 0);
}

// Bounds of the bucket after bucket j (R1), or the last point for the last bucket (R5).
__device__ __forceinline__ void next_bucket(int64_t j, const Div& dK, int64_t N, int64_t m,
                                            int64_t* lo, int64_t* hi) {
  if (j + 1 < (int64_t)dK.d) {
    *lo = part_start(j + 1, N, dK);
    *hi = part_start(j + 2, N, dK);
  } else {
    *lo = m - 1;
    *hi = m;
  }
}

// Slots a warp of k_tables fills: up to kTableRounds rounds of 32 (bt.tab_rounds; one
// round when there are too few slots to fill the GPU).
constexpr int kTableRounds = kTableRoundsMax;
constexpr int kTableBlock = 32 * kTableRounds;
constexpr int kTableCache = 8;  // candidates kept in shared memory per bucket

struct TableReq {  // a bucket that picks of the warp's slots fall in
  int64_t jt;      // the bucket (its picks follow picks in bucket jt - 1)
  int32_t s;       // series
  int32_t o;       // offset in the block of its first slot
};

// Up to 32 buckets of a table prepared for the entries whose picks fall in them, one
// per lane, structure of arrays (lanes that read different buckets hit different
// banks): candidates [lo, lo + cnt), the bucket after it [nlo, nlo + ncnt) and, with
// integer x, the FP32 filter data of StepBound: the mean after the bucket in filter
// form (ex < 0 where the filter does not apply), the candidates' y range, x origin
// and x span, and for buckets of up to kTableCache positions their FP32 y and x offsets.
struct TableChunk {
  long long lo[32], nlo[32], x0[32], xint[32];
  int cnt[32], ncnt[32];
  float xfrac[32], ym[32], ex[32], ey[32], ymin[32], ymax[32], xs[32];
  float cy[kTableCache][32], cx[kTableCache][32];
};

struct TableShared {  // a warp's shared memory in k_tables
  TableReq req[kTableBlock];
  uint8_t dreq[kTableBlock];  // the request of each slot of the block (0xff: no entry)
  TableChunk ch;
};

// Lane i of a chunk: bucket [lo, hi) prepared with the bucket after it [nlo, nhi),
// using integer and FP32 operations only.
__device__ void table_prepare(const SeriesPlan& sp, int64_t lo, int64_t hi, int64_t nlo, int64_t nhi,
                              TableChunk& ch, int i) {
  MeanF c;
  bool ok = mean_filter_form(sp, nlo, nhi, &c);
  float ymin = INFINITY, ymax = -INFINITY;
  const long long x0 = filter_x(sp, lo);
  const bool cached = hi - lo <= kTableCache;
  for (int64_t q = lo; q < hi; ++q) {
    const float v = filter_y(sp, q, &ok);
    ymin = fminf(ymin, v);
    ymax = fmaxf(ymax, v);
    if (cached) {
      ch.cy[q - lo][i] = v;
      ch.cx[q - lo][i] = f32_of_i64(filter_x(sp, q) - x0);
    }
  }
  const long long xl = filter_x(sp, hi - 1), lim = 1ll << 53;
  ok = ok && x0 > -lim && x0 < lim && xl > -lim && xl < lim;
  ch.lo[i] = lo;
  ch.nlo[i] = nlo;
  ch.cnt[i] = (int)(hi - lo);
  ch.ncnt[i] = (int)(nhi - nlo);
  ch.x0[i] = x0;
  ch.xint[i] = c.xint;
  ch.xfrac[i] = c.xfrac;
  ch.ym[i] = c.y32;
  ch.ex[i] = ok ? c.ex : -1.0f;
  ch.ey[i] = c.ey;
  ch.ymin[i] = ymin;
  ch.ymax[i] = ymax;
  ch.xs[i] = f32_of_i64(xl - x0);
}

// The offset in bucket i of the chunk of the pick after position pa: the largest FP64
// area (tri_area), the lowest offset on ties (R6, R8).  FP32 bounds first (StepBound);
// when the first candidate's lower bound exceeds every other upper bound it is the
// pick without any FP64 operation, otherwise the FP64 mean (R7) and the FP64 areas of
// the candidates that may be largest decide.
__device__ int table_pick(const SeriesPlan& sp, const TableChunk& ch, int i, int64_t pa) {
  const int64_t lo = ch.lo[i];
  const int cnt = ch.cnt[i];
  const long long x0 = ch.x0[i];
  StepBound sb;
  sb.ok = false;
  float thr = -INFINITY;
  if (ch.ex[i] >= 0.0f) {
    bool aok = true;
    const long long xa = filter_x(sp, pa);
    const float ya = filter_y(sp, pa, &aok);
    if (aok && xa > -(1ll << 53) && xa < (1ll << 53)) {
      MeanF c;
      c.xint = ch.xint[i];
      c.xfrac = ch.xfrac[i];
      c.y32 = ch.ym[i];
      c.ex = ch.ex[i];
      c.ey = ch.ey[i];
      sb.init_span(xa, ya, x0, c, ch.ymin[i], ch.ymax[i], ch.xs[i], sp.ydt != MMLTTB_F32);
      if (sb.ok) {
        float t1 = -1.0f, t2 = -1.0f;
        int p1 = 0;
        if (cnt <= kTableCache) {
#pragma unroll
          for (int u = 0; u < kTableCache; ++u) {
            if (u >= cnt) break;
            const float ta = sb.t_abs(ch.cy[u][i], ch.cx[u][i]);
            t2 = fmaxf(t2, fminf(ta, t1));
            if (ta > t1) {
              t1 = ta;
              p1 = u;
            }
          }
        } else {
          for (int u = 0; u < cnt; ++u) {
            bool qok = true;
            const float ta = sb.t_abs(filter_y(sp, lo + u, &qok), f32_of_i64(filter_x(sp, lo + u) - x0));
            t2 = fmaxf(t2, fminf(ta, t1));
            if (ta > t1) {
              t1 = ta;
              p1 = u;
            }
          }
        }
        if (__fadd_ru(t2, sb.E) < __fsub_rd(t1, sb.E)) return p1;  // decided without FP64
        thr = __fsub_rd(__fsub_rd(t1, sb.E), sb.E);
      }
    }
  }
  double xc, yc, xa, ya;
  bucket_mean(sp, ch.nlo[i], ch.nlo[i] + ch.ncnt[i], &xc, &yc);
  pos_xy(sp, pa, &xa, &ya);
  long long best = -1;  // bits of a non-negative double order like the double
  int pk = 0;
  for (int u = 0; u < cnt; ++u) {
    if (sb.ok) {
      bool qok = true;
      if (!(sb.t_abs(filter_y(sp, lo + u, &qok), f32_of_i64(filter_x(sp, lo + u) - x0)) >= thr)) continue;
    }
    double xb, yb;
    pos_xy(sp, lo + u, &xb, &yb);
    const long long ab = __double_as_longlong(tri_area(xa, ya, xb, yb, xc, yc));
    if (best < 0 || ab > best) {  // R8: the first largest wins
      best = ab;
      pk = u;
    }
  }
  return pk;
}

// Table entries of the warp's block of slots [base, base + 32*rounds).  Warp-
// collective; `s0` is the series of slot `base`; sh is the warp's shared memory.
__device__ void table_block(const Batch& bt, int64_t base, int rounds, int s0, int lane, TableShared& sh) {
  // 1. every slot's bucket; the first slot of each distinct (series, bucket) files a
  //    request, and every slot notes the request it belongs to (requests follow slot
  //    order, so that is the last one filed at or before it)
  int s = s0, nreq = 0;
  int64_t carry_jt = -1;
  int carry_s = -1;
  // the lane's current series, cached: its next series' first slot, table offset,
  // position count m, bucket count K and a divisor for m - 2 (no load or division per
  // slot while the series stays the same)
  int cs = -1;
  int64_t c_next = 0, c_off = 0, c_m = 0, c_K = 0;
  bool c_tab = false;
  Div c_dN;
#pragma unroll
  for (int r = 0; r < kTableRounds; ++r) {
    if (r >= rounds) continue;
    const int64_t slot = base + 32 * r + lane;
    if (cs < 0 || slot >= c_next) {
      if (bt.tab_offs)
        while (s + 1 < bt.n_series && bt.tab_offs[s + 1] <= slot) ++s;
      const SeriesPlan& sp = plan_of(bt, s);
      cs = s;
      c_next = bt.tab_offs && s + 1 < bt.n_series ? bt.tab_offs[s + 1] : INT64_MAX;
      c_off = sp.tab_off;
      c_tab = sp.engine == EN_TABLES;
      c_m = c_tab ? lttb_m(sp) : 0;
      c_K = sp.n_out - 2;
      c_tab = c_tab && c_m > sp.n_out;
      c_dN = make_div(c_m - 2 > 0 ? c_m - 2 : 1);
    }
    int64_t jt = -1;
    bool work = false;
    if (slot < bt.total_slots && c_tab) {  // the bucket its pick falls in (R1): jt
      const int64_t p = slot - c_off;
      if (p == 0) {
        jt = 0;
        work = true;
      } else if (p <= c_m - 2) {
        jt = part_of(p, c_dN, c_K) + 1;
        work = true;
      }
      work = work && jt < c_K;
    }
    const int ks = work ? s : -1;
    int64_t pjt = __shfl_up_sync(kFull, work ? jt : -1, 1);
    int ps = __shfl_up_sync(kFull, ks, 1);
    if (lane == 0) {
      pjt = carry_jt;
      ps = carry_s;
    }
    const bool first = work && (ps != ks || pjt != jt);
    const unsigned fl = __ballot_sync(kFull, first);
    const int d = nreq + __popc(fl & ((2u << lane) - 1u)) - 1;
    if (first) {
      sh.req[d].jt = jt;
      sh.req[d].s = ks;
      sh.req[d].o = 32 * r + lane;
    }
    sh.dreq[32 * r + lane] = work ? (uint8_t)d : (uint8_t)0xff;
    nreq += __popc(fl);
    carry_jt = __shfl_sync(kFull, work ? jt : -1, 31);
    carry_s = __shfl_sync(kFull, ks, 31);
  }
  __syncwarp();
  // 2. chunks of 32 requests: one lane per bucket prepares it, with the mean of the
  //    bucket after it (R5, R7); then one lane per slot picks (the slots of a chunk's
  //    buckets are the block's slots from its first request's to the next chunk's)
  for (int c0 = 0; c0 < nreq; c0 += 32) {
    const int d = c0 + lane;
    if (d < nreq) {
      const TableReq q = sh.req[d];
      const SeriesPlan& sp = plan_of(bt, q.s);
      const int64_t m = lttb_m(sp), K = sp.n_out - 2, N = m - 2;
      StepDiv bs;
      bs.init(q.jt == 0 ? 0 : q.jt - 1, N, sp.dK, 1);
      if (q.jt > 0) bs.next();
      const int64_t lo = bs.L + 1;  // bucket jt = [lo, hi) (R1)
      bs.next();
      const int64_t hi = bs.L + 1;
      int64_t nlo = m - 1, nhi = m;  // after the last bucket: the last point (R5)
      if (q.jt + 1 < K) {
        nlo = hi;
        bs.next();
        nhi = bs.L + 1;
      }
      table_prepare(sp, lo, hi, nlo, nhi, sh.ch, lane);
    }
    __syncwarp();
    const int o0 = sh.req[c0].o;
    const int o1 = c0 + 32 < nreq ? sh.req[c0 + 32].o : 32 * rounds;
    for (int o = o0 + lane; o < o1; o += 32) {
      const int dd = sh.dreq[o];
      if (dd == 0xff) continue;
      const SeriesPlan& sp = plan_of(bt, sh.req[dd].s);
      const int64_t p = base + o - sp.tab_off;
      sp.tab[p] = (uint8_t)table_pick(sp, sh.ch, dd - c0, p);
    }
    __syncwarp();
  }
}

// The LTTB pick that follows the k-th position of bucket j-1 (position 0 for j = 0):
// the offset in bucket j of the point with the largest area against that position
// and the mean of bucket j+1 (R1, R5-R8).  Warp-collective: all 32 lanes call it,
// the 2^lgS lanes of a bucket (lane groups aligned to 2^lgS) with the same j; the
// first lane of a bucket forms the mean (R7) for all of them.  The bucket starts
// step from one floor(j*N/K), so nothing divides by the position count.  *pos
// receives the position whose entry this is; the result is meaningful only where
// *valid (j < K and k inside bucket j-1).
__device__ int bucket_pick(const SeriesPlan& sp, int64_t m, int64_t j, int k, int lgS, int lane,
                           int64_t* pos, bool* valid) {
  const int S = 1 << lgS;
  const int64_t K = sp.n_out - 2, N = m - 2;
  bool work = false;
  int64_t p = 0, lo = 0, hi = 0;
  double xc = 0.0, yc = 0.0, xa = 0.0, ya = 0.0;
  double xb[8], yb[8];  // candidates; buckets of up to 8 load before the mean is formed
#pragma unroll
  for (int u = 0; u < 8; ++u) xb[u] = yb[u] = 0.0;
  if (j < K) {
    StepDiv bs;
    int64_t lprev = 0;
    if (j == 0) {
      bs.init(0, N, sp.dK, 1);
    } else {
      bs.init(j - 1, N, sp.dK, 1);
      lprev = bs.L + 1;  // start of bucket j-1
      bs.next();
    }
    lo = bs.L + 1;  // bucket j = [lo, hi) (R1)
    bs.next();
    hi = bs.L + 1;
    p = j == 0 ? 0 : lprev + k;
    work = k < (j == 0 ? 1 : lo - lprev);
    if (work) {
      pos_xy(sp, p, &xa, &ya);
#pragma unroll
      for (int u = 0; u < 8; ++u)
        if (lo + u < hi) pos_xy(sp, lo + u, &xb[u], &yb[u]);
    }
    if (k == 0) {
      int64_t nlo = m - 1, nhi = m;  // after the last bucket: the last point (R5)
      if (j + 1 < K) {
        nlo = hi;
        bs.next();
        nhi = bs.L + 1;
      }
      bucket_mean(sp, nlo, nhi, &xc, &yc);
    }
  }
  const int leader = lane & ~(S - 1);
  xc = __shfl_sync(kFull, xc, leader);
  yc = __shfl_sync(kFull, yc, leader);
  *pos = p;
  *valid = work;
  if (!work) return 0;
  long long best = -1;  // bits of a non-negative double order like the double
  int pick = 0;
  for (int64_t q0 = lo; q0 < hi; q0 += 8) {
    if (q0 > lo) {
#pragma unroll
      for (int u = 0; u < 8; ++u)
        if (q0 + u < hi) pos_xy(sp, q0 + u, &xb[u], &yb[u]);
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      if (q0 + u >= hi) break;
      const long long ab = __double_as_longlong(tri_area(xa, ya, xb[u], yb[u], xc, yc));
      if (q0 + u == lo || ab > best) {  // R8: the first largest wins
        best = ab;
        pick = (int)(q0 + u - lo);
      }
    }
  }
  return pick;
}

// Table entries of one series laid out bucket-major: slot j*S + k (S = 2^tab_lgS,
// at least the largest bucket) holds the pick after the k-th position of bucket j-1.
__device__ void table_bucket_entry(const SeriesPlan& sp, int64_t m, int64_t slot, int lane) {
  const int lgS = sp.tab_lgS;
  int64_t p;
  bool valid;
  const int pick = bucket_pick(sp, m, slot >> lgS, (int)(slot & ((1 << lgS) - 1)), lgS, lane, &p, &valid);
  if (valid) sp.tab[p] = (uint8_t)pick;
}

// Bucket starts L_j = floor(j*N/K)+1 for consecutive j without a division per step.
struct PartIter {
  StepDiv sd;
  int64_t L = 0;
  __device__ PartIter() {}
  __device__ PartIter(int64_t j, int64_t N, const Div& dK) {
    sd.init(j, N, dK, 1);
    L = sd.L + 1;
  }
  __device__ void next() {  // j -> j+1
    sd.next();
    L = sd.L + 1;
  }
};

// A map of at most 8 entries with values below 8, one byte per entry (entry i in
// byte i of {hi:lo}), so that composing two maps is two byte permutations.
struct Map8 {
  unsigned lo, hi;
};
// Selector nibbles for __byte_perm from four bytes (each below 8).
__device__ __forceinline__ unsigned nibbles(unsigned w) {
  return (w & 0x7u) | ((w >> 4) & 0x70u) | ((w >> 8) & 0x700u) | ((w >> 12) & 0x7000u);
}
// (a after b)(i) = a[b[i]]
__device__ __forceinline__ Map8 compose(Map8 a, Map8 b) {
  return {__byte_perm(a.lo, a.hi, nibbles(b.lo)), __byte_perm(a.lo, a.hi, nibbles(b.hi))};
}
__device__ __forceinline__ int map_at(Map8 a, int i) {
  return (int)(((i < 4 ? a.lo : a.hi) >> (8 * (i & 3))) & 0xffu);
}
__device__ __forceinline__ Map8 shfl_up_map(Map8 a, int d) {
  return {__shfl_up_sync(kFull, a.lo, d), __shfl_up_sync(kFull, a.hi, d)};
}
__device__ __forceinline__ Map8 shfl_down_map(Map8 a, int d) {
  return {__shfl_down_sync(kFull, a.lo, d), __shfl_down_sync(kFull, a.hi, d)};
}
__device__ __forceinline__ Map8 shfl_map(Map8 a, int src) {
  return {__shfl_sync(kFull, a.lo, src), __shfl_sync(kFull, a.hi, src)};
}
constexpr Map8 kIdentity8 = {0x03020100u, 0x07060504u};

// The LTTB output of series sp once its tables are written.  Block-collective over
// NT threads.  F ([2][kTableMaxBucket][NT]) and dom ([2][NT]) are shared scratch;
// s_tab4 holds up to tab_smem bytes of shared memory for staging the tables
// (staged_tab_bytes(m) of them when they fit).
//   Phase 1: thread t composes the steps of its segment of buckets [j0, j1) for
//            every entry offset in bucket j0-1 (four entries at a time, so four
//            independent table loads are in flight).
//   Phase 2: the prefix of the segment maps under composition, evaluated at the
//            chain's start (position 0): with buckets of at most 8 positions the
//            maps live in registers (warp shuffle scan, then one pass over the
//            warps' totals); otherwise a Hillis-Steele scan over shared memory.
//   Phase 3: each segment is walked from its resolved entry, writing positions;
//            then positions become indices with independent loads.
template <int NT>
__device__ void chain_series(const SeriesPlan& sp, uint4* s_tab4, int64_t tab_smem,
                             uint8_t (*F)[kTableMaxBucket][NT], uint8_t (*dom)[NT]) {
  __shared__ unsigned s_wlo[NT / 32], s_whi[NT / 32];
  __shared__ int s_went[NT / 32];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  if (sp.branch == BR_ARANGE) {
    for (int64_t i = tid; i < sp.n; i += NT) sp.out[i] = i;
    if (tid == 0 && sp.out_count) *sp.out_count = sp.n;
    return;
  }
  if (sp.branch != BR_LTTB_ALL && sp.branch != BR_MINMAX_LTTB) return;
  const int64_t m = lttb_m(sp);
  if (m <= sp.n_out) {  // nothing to drop (R14)
    for (int64_t i = tid; i < m; i += NT) sp.out[i] = index_of(sp, i);
    if (tid == 0 && sp.out_count) *sp.out_count = m;
    return;
  }
  if (sp.engine != EN_TABLES) return;
  const int64_t K = sp.n_out - 2, N = m - 2;
  const int T = K < NT ? (int)K : NT;
  const bool packed = (N + K - 1) / K <= 8;  // every bucket holds at most 8 positions
  // Staged tables keep byte q at q + 4*(q/32): the threads walk segments about 32
  // positions apart, and without the pad word per 32 bytes a warp's lookups would
  // fall into 4 of the 32 banks.
  const uint8_t* tab = sp.tab;
  int64_t padw = 0;
  if (staged_tab_bytes(m) <= tab_smem) {
    const int64_t nw4 = (m + 3) / 4;  // 4-byte words (the storage is padded to 16 bytes)
    const unsigned* src = (const unsigned*)sp.tab;
    unsigned* dst = (unsigned*)s_tab4;
    for (int64_t i0 = tid; i0 < nw4; i0 += 4 * NT) {  // four L2 loads in flight per thread
      unsigned w[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) w[u] = i0 + u * NT < nw4 ? __ldcg(src + i0 + u * NT) : 0u;
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int64_t i = i0 + u * NT;
        if (i < nw4) dst[i + (i >> 3)] = w[u];
      }
    }
    __syncthreads();
    tab = (const uint8_t*)s_tab4;
    padw = 4;
  }
  static_assert((NT & (NT - 1)) == 0, "NT must be a power of two");
  int64_t j0 = 0, j1 = 0;
  Map8 P = {0x03020100u, 0x07060504u};  // identity (threads without a segment keep it)
  PartIter it0;
  int64_t l0 = 0;
  if (tid < T) {
    // segment [floor(t*K/T), floor((t+1)*K/T)): T = NT (a power of two) or T = K
    if (T == NT) {
      j0 = (int64_t)(((uint64_t)tid * (uint64_t)K) / (uint64_t)NT);
      j1 = (int64_t)(((uint64_t)(tid + 1) * (uint64_t)K) / (uint64_t)NT);
    } else {
      j0 = tid;
      j1 = tid + 1;
    }
    it0 = PartIter(j0 > 0 ? j0 - 1 : 0, N, sp.dK);  // start of bucket j0-1 (or of bucket 0)
    int d0 = 1;
    if (j0 > 0) {
      l0 = it0.L;
      it0.next();
      d0 = (int)(it0.L - l0);
    }
    for (int ia = 0; ia < d0; ia += 4) {
      int v0 = ia, v1 = ia + 1 < d0 ? ia + 1 : ia, v2 = ia + 2 < d0 ? ia + 2 : ia;
      int v3 = ia + 3 < d0 ? ia + 3 : ia;
      PartIter it = it0;
      int64_t lprev = l0;
      for (int64_t j = j0; j < j1; ++j) {
        v0 = tab[lprev + v0 + (((lprev + v0) >> 5) * padw)];
        v1 = tab[lprev + v1 + (((lprev + v1) >> 5) * padw)];
        v2 = tab[lprev + v2 + (((lprev + v2) >> 5) * padw)];
        v3 = tab[lprev + v3 + (((lprev + v3) >> 5) * padw)];
        lprev = it.L;  // start of bucket j
        it.next();
      }
      if (packed) {
        const unsigned w = (unsigned)v0 | ((unsigned)v1 << 8) | ((unsigned)v2 << 16) | ((unsigned)v3 << 24);
        if (ia == 0) P.lo = w; else P.hi = w;
      } else {
        F[0][ia][tid] = (uint8_t)v0;
        if (ia + 1 < d0) F[0][ia + 1][tid] = (uint8_t)v1;
        if (ia + 2 < d0) F[0][ia + 2][tid] = (uint8_t)v2;
        if (ia + 3 < d0) F[0][ia + 3][tid] = (uint8_t)v3;
      }
    }
    if (!packed) dom[0][tid] = (uint8_t)d0;
  }
  int v;  // entry offset of this thread's segment (in bucket j0-1)
  if (packed) {
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const Map8 o = shfl_up_map(P, d);
      if (lane >= d) P = compose(P, o);
    }
    // P: this warp's segments up to and including this thread's, composed
    if (lane == 31) {
      s_wlo[wid] = P.lo;
      s_whi[wid] = P.hi;
    }
    __syncthreads();
    if (tid == 0) {
      int e = 0;  // the chain starts at position 0
      for (int w = 0; w < NT / 32; ++w) {
        s_went[w] = e;
        e = map_at(Map8{s_wlo[w], s_whi[w]}, e);
      }
    }
    __syncthreads();
    const Map8 prev = shfl_up_map(P, 1);
    v = lane == 0 ? s_went[wid] : map_at(prev, s_went[wid]);
  } else {
    int c = 0;
    for (int d = 1; d < T; d <<= 1) {
      __syncthreads();
      if (tid < T) {
        if (tid >= d) {
          const int dd = dom[c][tid - d];
          for (int ia = 0; ia < dd; ++ia) F[c ^ 1][ia][tid] = F[c][F[c][ia][tid - d]][tid];
          dom[c ^ 1][tid] = (uint8_t)dd;
        } else {
          const int dd = dom[c][tid];
          for (int ia = 0; ia < dd; ++ia) F[c ^ 1][ia][tid] = F[c][ia][tid];
          dom[c ^ 1][tid] = (uint8_t)dd;
        }
      }
      c ^= 1;
    }
    __syncthreads();
    v = (tid == 0 || tid >= T) ? 0 : F[c][0][tid - 1];
  }
  if (tid < T) {
    PartIter it = it0;  // as after phase 1's set-up: L = start of bucket j0
    int64_t lprev = l0;
    for (int64_t j = j0; j < j1; ++j) {
      v = tab[lprev + v + (((lprev + v) >> 5) * padw)];
      sp.out[j + 1] = it.L + v;  // position in bucket j
      lprev = it.L;
      it.next();
    }
  }
  if (sp.sel) {  // positions -> original indices, four independent gathers per round
    __syncthreads();
    for (int64_t i = 1 + tid; i <= K; i += 4 * NT) {
      int64_t q[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) q[u] = i + u * NT <= K ? sp.out[i + u * NT] : 0;
#pragma unroll
      for (int u = 0; u < 4; ++u) q[u] = sp.sel[q[u]];
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (i + u * NT <= K) sp.out[i + u * NT] = q[u];
    }
  }
  if (tid == 0) {
    sp.out[0] = index_of(sp, 0);
    sp.out[K + 1] = index_of(sp, m - 1);
    if (sp.out_count) *sp.out_count = sp.n_out;
  }
}

}  // namespace
}  // namespace mmlttb
