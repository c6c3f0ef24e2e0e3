// Shared structures and device helpers of libmmlttb (MinMaxLTTB, arXiv 2305.00332).
//
// One launch sequence serves a single series and a batch of series alike: every
// kernel receives a `Batch` holding the per-series plans, and the MinMax stream
// walks one global "interior position" space that concatenates the interior points
// 1..n-2 of every series that needs preselection.
#pragma once

#include <cuda_runtime.h>
#include <limits.h>
#include <stdint.h>

#include "mmlttb.h"

namespace mmlttb {

// What a series needs, decided on the host from its sizes alone (Sec. 3).
enum Branch : int32_t {
  BR_ARANGE = 0,       // n_out >= n: every index
  BR_LTTB_ALL = 1,     // LTTB on all n points (plain LTTB, or r_ps*n_out >= n)
  BR_MINMAX_LTTB = 2,  // MinMax preselection, then LTTB on the preselected points
  BR_PRESELECT = 3,    // MinMax preselection only; the list goes to the output
  BR_M4 = 4,           // M4: first, argmin, argmax, last of each bin over all points
};

// Which LTTB engine resolves the serial bucket chain.
enum Engine : int32_t {
  EN_NONE = 0,
  EN_TABLES = 1,  // per-position transition tables + parallel chain composition
  EN_GRID = 2,    // one grid-wide step per bucket (cooperative launch)
  EN_BLOCK = 3,   // one CTA per series, one block-wide step per bucket
};

constexpr unsigned kFull = 0xffffffffu;

// Largest LTTB bucket (in points) the transition-table engine accepts.
constexpr int kTableMaxBucket = 32;
// Shared memory that m table bytes take when staged for the chain: one 4-byte pad
// word after every 32 bytes (bank spread), rounded up to 16 bytes.
__host__ __device__ inline int64_t staged_tab_bytes(int64_t m) {
  const int64_t w = (m + 3) / 4;
  return ((w + (w + 7) / 8) * 4 + 15) & ~int64_t(15);
}
// Bins per CTA of the compaction kernels; every series' bins start on a CTA boundary.
constexpr int kBinsPerCta = 256;
// Threads of the streaming MinMax kernel's CTAs.
// Staged stream (k_stream_bulk) for float32 index bins of at most kBulkMaxBinBytes:
// every warp runs its own pipeline of kBulkStages shared-memory stages, each filled by
// one cp.async.bulk copy of a tile (whole bins of one series, at most kBulkTileBytes
// of y, widened to 16-byte boundaries).  CTAs of kBulkWarps warps, as many per SM as
// fit.  Measured on 1e8 float32 points it matches or passes the register stream for
// bins of 16 to 128 points and falls behind it above (fewer bins per tile, per-tile
// costs less amortised), hence the bin limit.
constexpr int kBulkWarps = 1;
constexpr int kBulkStages = 2;
constexpr int64_t kBulkTileBytes = 8192;
constexpr int kBulkStageBytes = 8192 + 64;
constexpr int kBulkSmemBytes = kBulkWarps * kBulkStages * (kBulkStageBytes + 8);
constexpr int64_t kBulkMaxBinBytes = 512;
constexpr int64_t kBulkBinCost = 64;  // tile cost of a bin beyond its bytes (record, reduction)
// Bins per tile of the staged stream for a series with nb binned points of elem_bytes
// in B index bins (0: the register stream).  Bins hold floor(nb/B) or ceil(nb/B)
// points, so bpt bins of ceil(nb/B) points fit a tile.
__host__ __device__ inline int64_t bulk_bins_per_tile(int64_t nb, int64_t B, int elem_bytes) {
  if (B <= 0 || nb <= 0) return 0;
  const int64_t smax = (nb + B - 1) / B;
  if (smax * elem_bytes > kBulkMaxBinBytes) return 0;
  const int64_t bpt = kBulkTileBytes / elem_bytes / smax;
  return bpt < B ? bpt : B;
}
// Lanes per bin of the staged stream: the 32 lanes cover a tile's bpt bins in one round
// (a lane per bin from 17 bins per tile on, a whole warp for a one-bin tile).  From
// shared memory a lane reads its share of a bin at no extra latency, so fewer lanes per
// bin cost fewer per-bin rounds (bounds, group reduction, record store).
__host__ __device__ inline int bulk_group(int64_t bpt) {
  int c = 1;
  while (c < 32 && c < bpt) c <<= 1;
  return 32 / c;
}

// Division by a divisor fixed ahead of the kernel (bins, points, work units, warps,
// buckets).  An integer division costs hundreds of cycles of latency on this part;
// with inv = floor((2^64-1)/d), computed once where d is set (on the host),
// umulhi(a, inv) is floor(a/d) or one less, and one compare fixes it.
struct Div {
  uint64_t d = 1, inv = ~0ull;
};
__host__ __device__ inline Div make_div(int64_t d) {
  Div r;
  r.d = d > 0 ? (uint64_t)d : 1ull;
  r.inv = ~0ull / r.d;
  return r;
}
__host__ __device__ inline uint64_t div_by(uint64_t a, const Div& D) {
#ifdef __CUDA_ARCH__
  uint64_t q = __umul64hi(a, D.inv);
  uint64_t r = a - q * D.d;
  if (r >= D.d) {
    ++q;
    r -= D.d;
  }
  if (r >= D.d) ++q;
  return q;
#else
  return a / D.d;
#endif
}

// Result of one warp over one bin (or the part of a bin inside the warp's range):
// order-preserving integer keys of the extreme y values and their point indices.
struct Record {
  long long kmin, kmax;
  long long imin, imax;
};

struct SeriesPlan {
  const void* y;
  const void* x;
  int32_t ydt, xk, binmode, branch, engine, r_ps;
  int32_t group;     // lanes per bin in the MinMax stream (1..32, a power of two)
  int32_t bin_r1, bin_rs;  // index bins: nb mod B and (32/group)*nb mod B (set_bin_steps)
  int64_t bin_q1, bin_qs;  // index bins: floor(nb/B) and floor((32/group)*nb/B)
  Div dB, dnb, dnpos, dK;  // divisors B, nb, npos and K = n_out - 2 (set_bin_steps)
  int32_t tab_lgS;         // fused tables: log2 of the slots per bucket (>= largest bucket)
  int32_t nan_aware; // NaN-aware MinMax / M4 (R18)
  int64_t n, n_out;
  int64_t B;         // MinMax bins (minmax branches), else 0
  int64_t p0;        // first binned point: 1 (MinMax over the interior) or 0 (M4)
  int64_t nb;        // binned points: n-2 (MinMax) or n (M4)
  int64_t bin_off;   // global index of this series' bin 0 in the record space
  int64_t edge_off;  // index of this series' S_0 in the edge array (x-width bins)
  int64_t pos_off;   // offset of this series in the global work (cost) space
  int64_t npos;      // its extent there: D = N + kBinCost*min(B, N) for N = n-2 > 0, else 0
  int64_t tab_off;   // first slot of this series in the table-slot space
  int64_t tab_cap;   // slots reserved (positions that may need a table entry)
  int64_t bincta_off; // first compaction CTA of this series (minmax branches)
  // staged stream (k_stream_bulk), index bins of at most kBulkTileBytes: bins per tile
  // (0: the register stream), the series' first unit in the launch's tile cost space
  // and the cost of one of its tiles, and the record slot offset of its bins (bin b's
  // record at bin_off + b + rec_w)
  int64_t bulk_bpt, tcost_off, tcost, rec_w;
  int64_t* sel;      // preselected list (capacity 2B+2), NULL for BR_LTTB_ALL
  double* px;        // x of each preselected position as FP64 (BR_MINMAX_LTTB), else NULL
  double* py;        // y of each preselected position as FP64 (BR_MINMAX_LTTB), else NULL
  int64_t* m_ptr;    // number of preselected points (device), minmax branches
  uint8_t* tab;      // one transition-table byte per position (EN_TABLES)
  double* means;     // 2*K doubles: next-bucket means (EN_GRID / EN_BLOCK)
  int64_t* out;
  int64_t* out_count;
};

struct Batch {
  const SeriesPlan* plans;  // device array of n_series plans; NULL: the single plan `one`
  SeriesPlan one;
  const int64_t* pos_offs;   // n_series+1 prefix of npos, the work space (NULL for a single series)
  const int64_t* edge_offs;  // n_series+1 prefix of edge counts
  const int64_t* tab_offs;   // n_series+1 prefix of tab_cap
  const int64_t* cta_offs;   // n_series+1 prefix of compaction CTAs
  int32_t n_series;
  int64_t total_pos;   // sum of npos: the total work the streaming warps split evenly
  int64_t n_warps;     // streaming warps, each with at least one interior point
  Div dtotal, dwarps;  // divisors total_pos and n_warps (set_warp_divs)
  Div dgrid;           // divisor gridDim.x of the fused kernel
  int64_t total_edges; // sum over x-width series of B+1
  int64_t total_slots; // sum of tab_cap
  int64_t total_bin_ctas;  // compaction CTAs over all minmax series
  Record* rec;         // total bins + n_warps records
  int64_t* edges;      // bin starts S_b of x-width series
  int64_t* binres;     // per padded bin: (first argmin/argmax lower, higher, their keys) or (-1, -1, 0, 0)
  int32_t* cta_sum;    // per compaction CTA: number of indices its bins emit
  int32_t* cta_series; // per compaction CTA: its series
  int64_t* cta_off;    // per compaction CTA: exclusive prefix of cta_sum within its series
  unsigned* status;    // error bits (1: a bounded wait timed out, 2: device check failed)
  unsigned* barrier;   // grid barrier counter (EN_GRID and the fused kernel)
  int64_t* fused_tot;  // per CTA of the fused kernel: indices its bins emit
  int64_t chain_smem;  // dynamic shared memory of k_chain for the tables (bytes)
  int32_t zero_status; // the launch clears the status and barrier words first (first kernel of a call)
  int32_t tab_rounds;  // k_tables: rounds of 32 slots per warp (1..kTableRoundsMax)
  int32_t tab_rounds_req;  // the tuning's rounds for k_tables (0: from the slot count)
  const int64_t* tcost_offs;  // n_series+1 prefix of the staged stream's tile costs (NULL: single)
  int64_t total_tcost;  // the tile cost space k_stream_bulk's warps split evenly
  int64_t n_bulk_warps; // warps of k_stream_bulk
  Div dtcost, dbwarps;  // divisors total_tcost and n_bulk_warps
};

__host__ __device__ inline void set_bin_steps(SeriesPlan& sp) {
  sp.dB = make_div(sp.B);
  sp.dnb = make_div(sp.nb);
  sp.dnpos = make_div(sp.npos);
  sp.dK = make_div(sp.n_out - 2);
  sp.bin_q1 = sp.bin_qs = 0;
  sp.bin_r1 = sp.bin_rs = 0;
  if (sp.B <= 0 || sp.nb < 0 || sp.group <= 0) return;
  const int64_t s = 32 / sp.group;
  sp.bin_q1 = sp.nb / sp.B;
  sp.bin_r1 = (int32_t)(sp.nb - sp.bin_q1 * sp.B);
  sp.bin_qs = (s * sp.nb) / sp.B;
  sp.bin_rs = (int32_t)(s * sp.nb - sp.bin_qs * sp.B);
}

// Divisors of the streams' warp partitions, after total_pos, n_warps, total_tcost and
// n_bulk_warps are set.
__host__ __device__ inline void set_warp_divs(Batch& bt) {
  bt.dtotal = make_div(bt.total_pos);
  bt.dwarps = make_div(bt.n_warps);
  bt.dtcost = make_div(bt.total_tcost);
  bt.dbwarps = make_div(bt.n_bulk_warps);
}

__host__ __device__ inline const SeriesPlan& plan_of(const Batch& bt, int s) {
  return bt.plans ? bt.plans[s] : bt.one;
}

// Last index i in [0, count) with offs[i] <= v (offs non-decreasing, offs[0] <= v).
__device__ inline int upper_index(const int64_t* offs, int count, int64_t v) {
  int lo = 0, hi = count;  // answer in [lo, hi)
  while (hi - lo > 1) {
    int mid = (lo + hi) >> 1;
    if (offs[mid] <= v) lo = mid; else hi = mid;
  }
  return lo;
}

// The same, warp-collective (every lane passes the same v): a 32-ary search, two or
// three rounds of parallel loads for a few thousand entries.
__device__ inline int warp_upper_index(const int64_t* offs, int count, int64_t v, int lane) {
  int lo = 0, hi = count;  // answer in [lo, hi)
  while (hi - lo > 1) {
    const int step = (hi - lo + 31) >> 5;
    const int q = lo + lane * step;
    const unsigned le = __ballot_sync(kFull, q < hi && offs[q] <= v);  // a prefix of the lanes
    const int last = lo + (31 - __clz(le)) * step;
    hi = last + step < hi ? last + step : hi;
    lo = last;
  }
  return lo;
}

// floor(a*b/c) for a, b >= 0, c > 0, exact for any int64 inputs whose quotient fits.
__host__ __device__ inline int64_t muldiv(int64_t a, int64_t b, int64_t c) {
#ifdef __CUDA_ARCH__
  unsigned long long lo = (unsigned long long)a * (unsigned long long)b;
  unsigned long long hi = __umul64hi((unsigned long long)a, (unsigned long long)b);
  if (hi == 0) return (int64_t)(lo / (unsigned long long)c);
  unsigned __int128 num = ((unsigned __int128)hi << 64) | lo;
  return (int64_t)(num / (unsigned long long)c);
#else
  unsigned __int128 num = (unsigned __int128)(uint64_t)a * (uint64_t)b;
  return (int64_t)(num / (uint64_t)c);
#endif
}

// ceil(a*b/c) for a, b >= 0, c > 0 (exact, 128-bit intermediate when needed).
__host__ __device__ inline int64_t muldiv_ceil(int64_t a, int64_t b, int64_t c) {
#ifdef __CUDA_ARCH__
  unsigned long long lo = (unsigned long long)a * (unsigned long long)b;
  unsigned long long hi = __umul64hi((unsigned long long)a, (unsigned long long)b);
  if (hi == 0) {
    const unsigned long long q = lo / (unsigned long long)c;
    return (int64_t)(q + (q * (unsigned long long)c != lo ? 1 : 0));
  }
  const unsigned __int128 num = ((unsigned __int128)hi << 64) | lo;
  const unsigned __int128 q = num / (unsigned long long)c;
  return (int64_t)(q + (q * (unsigned long long)c != num ? 1 : 0));
#else
  const unsigned __int128 num = (unsigned __int128)(uint64_t)a * (uint64_t)b;
  const unsigned __int128 q = num / (uint64_t)c;
  return (int64_t)(q + (q * (uint64_t)c != num ? 1 : 0));
#endif
}

// Start of part j when `items` items are split into `parts` equal-count parts,
// counting from 1: floor(j*items/parts)+1.  Used for MinMax index bins over the
// interior points and for LTTB buckets over the interior positions.
__host__ __device__ inline int64_t part_start(int64_t j, int64_t items, int64_t parts) {
  return muldiv(j, items, parts) + 1;
}

// The part that contains position p (1 <= p <= items): the largest j with
// part_start(j) <= p, i.e. floor((p*parts - 1) / items).
__host__ __device__ inline int64_t part_of(int64_t p, int64_t items, int64_t parts) {
#ifdef __CUDA_ARCH__
  unsigned long long lo = (unsigned long long)p * (unsigned long long)parts;
  unsigned long long hi = __umul64hi((unsigned long long)p, (unsigned long long)parts);
  if (hi == 0) return (int64_t)((lo - 1ull) / (unsigned long long)items);
  unsigned __int128 num = (((unsigned __int128)hi << 64) | lo) - 1u;
  return (int64_t)(num / (unsigned long long)items);
#else
  unsigned __int128 num = (unsigned __int128)(uint64_t)p * (uint64_t)parts - 1u;
  return (int64_t)(num / (uint64_t)items);
#endif
}

// The same with a prepared divisor (the fast path when the product fits 64 bits).
__host__ __device__ inline int64_t muldiv(int64_t a, int64_t b, const Div& c) {
#ifdef __CUDA_ARCH__
  const unsigned long long lo = (unsigned long long)a * (unsigned long long)b;
  const unsigned long long hi = __umul64hi((unsigned long long)a, (unsigned long long)b);
  if (hi == 0) return (int64_t)div_by(lo, c);
  const unsigned __int128 num = ((unsigned __int128)hi << 64) | lo;
  return (int64_t)(num / c.d);
#else
  return muldiv(a, b, (int64_t)c.d);
#endif
}
__host__ __device__ inline int64_t muldiv_ceil(int64_t a, int64_t b, const Div& c) {
#ifdef __CUDA_ARCH__
  const unsigned long long lo = (unsigned long long)a * (unsigned long long)b;
  const unsigned long long hi = __umul64hi((unsigned long long)a, (unsigned long long)b);
  if (hi == 0) {
    const unsigned long long q = div_by(lo, c);
    return (int64_t)(q + (q * c.d != lo ? 1 : 0));
  }
  return muldiv_ceil(a, b, (int64_t)c.d);
#else
  return muldiv_ceil(a, b, (int64_t)c.d);
#endif
}
__host__ __device__ inline int64_t part_start(int64_t j, int64_t items, const Div& parts) {
  return muldiv(j, items, parts) + 1;
}
__host__ __device__ inline int64_t part_of(int64_t p, const Div& items, int64_t parts) {
#ifdef __CUDA_ARCH__
  const unsigned long long lo = (unsigned long long)p * (unsigned long long)parts;
  const unsigned long long hi = __umul64hi((unsigned long long)p, (unsigned long long)parts);
  if (hi == 0) return (int64_t)div_by(lo - 1ull, items);
  return part_of(p, (int64_t)items.d, parts);
#else
  return part_of(p, (int64_t)items.d, parts);
#endif
}

// floor(j*N/K) for j = j0, j0 + s, j0 + 2s, ... (N >= 0, K >= 1, s*N < 2^63) with
// no division per step: an integer division costs hundreds of cycles of latency on
// this part, a step a few adds.
struct StepDiv {
  int64_t L = 0, rem = 0;   // floor(j*N/K) and j*N - L*K, in [0, K)
  int64_t qs = 0, rs = 0;   // floor(s*N/K) and s*N - qs*K
  int64_t K = 1;
  __host__ __device__ void init(int64_t j, int64_t N, const Div& dK, int64_t s) {
    K = (int64_t)dK.d;
    L = muldiv(j, N, dK);
    // the true remainder lies in [0, K): exact in wrapping 64-bit arithmetic
    rem = (int64_t)((uint64_t)j * (uint64_t)N - (uint64_t)L * (uint64_t)K);
    qs = (int64_t)div_by((uint64_t)(s * N), dK);
    rs = s * N - qs * K;
  }
  __host__ __device__ void next() {  // j -> j + s
    L += qs;
    rem += rs;
    if (rem >= K) {
      rem -= K;
      L += 1;
    }
  }
};

// Index-bin step constants of a plan (after nb, B and group are set): a lane group of
// the stream moves from bin mb to mb + 32/group per round and needs bin starts
// floor(mb*nb/B) without a division per round.
struct SeriesPlan;
__host__ __device__ inline void set_bin_steps(SeriesPlan& sp);

// Work balance of the MinMax stream.  A bin has a fixed cost (a load round trip and a
// reduction by its group of lanes), so every series occupies D = N + c*min(B, N)
// units of a global work space, c = kBinCostPerLane * G, in which binned point q
// (0-based) sits at unit floor(q*D/N): strictly increasing, steps of at most c+1.
// Warps split the work space evenly, so a warp covering short series with small
// bins gets fewer points.
// A bin handled by a group of G lanes costs about 16*G points of work (a full warp
// per bin: one load round trip and one reduction per 512 points of float32).
constexpr int64_t kBinCostPerLane = 16;
constexpr int64_t kBinCostMax = 32 * kBinCostPerLane;
__host__ __device__ inline int64_t series_work(int64_t N, int64_t B, int G) {
  return N > 0 ? N + kBinCostPerLane * G * (B < N ? B : N) : 0;
}
// Lanes per bin for a series, a power of two.  A bin costs a fixed round of bounds,
// reduction and record store.  For launches that stream at least
// kStreamThroughputBytes the lanes read about 512 bytes (32 loads of 16 bytes) each
// per bin, at least 2 lanes above 128-byte bins, which amortises that round (on 1e8
// float32 points: 125-point bins 2.5 -> 3.3 TB/s, 1024-point bins 3.2 -> 3.8 TB/s).
// Smaller launches are latency-bound: about one 64-byte round trip per lane per bin.
constexpr int64_t kStreamThroughputBytes = int64_t(64) << 20;
__host__ __device__ inline int stream_group(int64_t N, int64_t B, int elem_bytes, bool throughput) {
  const int64_t per_bin_bytes = (B > 0 ? N / B : N) * elem_bytes;
  int G = 1;
  if (!throughput) {
    while (G < 32 && (int64_t)G * 64 < per_bin_bytes) G <<= 1;
    return G;
  }
  if (per_bin_bytes <= 128) return 1;
  G = 2;
  while (G < 32 && (int64_t)G * 512 < per_bin_bytes) G <<= 1;
  return G;
}

// Lanes per bin for a single series that streams at least kStreamThroughputBytes.
// Alone on the GPU, small bins want more lanes than the batch rule gives: on 1e9
// float32 points, 4 lanes for bins of 128 B to 1 KiB (125-point bins 2.5 -> 3.9 TB/s,
// 256-point 2.9 -> 4.5) and 8 up to 4 KiB (512-point 4.2 -> 5.2), then about 512 bytes
// per lane.  In a batch the same choice measured slower (3.8 -> 4.9 ms on the
// 4096-series mix, also with the work space charged as for stream_group), so batches
// keep stream_group.
__host__ __device__ inline int stream_group_single(int64_t N, int64_t B, int elem_bytes) {
  const int64_t per_bin_bytes = (B > 0 ? N / B : N) * elem_bytes;
  if (per_bin_bytes <= 128) return 1;
  if (per_bin_bytes <= 1024) return 4;
  if (per_bin_bytes <= 4096) return 8;
  int G = 16;
  while (G < 32 && (int64_t)G * 512 < per_bin_bytes) G <<= 1;
  return G;
}

// Streaming warp w covers global work units [floor(w*T/W), floor((w+1)*T/W)).
__host__ __device__ inline int64_t warp_begin(int64_t w, int64_t total, const Div& warps) {
  return muldiv(w, total, warps);
}
// The warp whose range holds global work unit g: floor(((g+1)*W - 1) / T).
__host__ __device__ inline int64_t warp_of(int64_t g, const Div& total, int64_t warps) {
  return part_of(g + 1, total, warps);
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Order-preserving integer keys of y values; -0.0 and +0.0 share key 0.
__device__ __forceinline__ int key32(float v) {
  int s = __float_as_int(v);
  return s >= 0 ? s : -(s & 0x7fffffff);
}
__device__ __forceinline__ long long key64(double v) {
  long long s = __double_as_longlong(v);
  return s >= 0 ? s : -(s & 0x7fffffffffffffffLL);
}

// Programmatic dependent launch: a kernel launched with programmatic stream
// serialization may start while its predecessor drains; it waits here (before it
// reads anything the predecessor wrote) and lets its own successor launch early.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" :::); }

__device__ __forceinline__ void set_status(unsigned* status, unsigned bit) {
  if (status) atomicOr(status, bit);
}

// Branches that run the MinMax stream and the compaction.
__host__ __device__ inline bool binned(int32_t branch) {
  return branch == BR_MINMAX_LTTB || branch == BR_PRESELECT || branch == BR_M4;
}

// Coordinates of original point i as FP64 (implicit x is the index).
__device__ __forceinline__ double x_of(const SeriesPlan& sp, int64_t i) {
  if (sp.xk == MMLTTB_X_IMPLICIT) return (double)i;
  if (sp.xk == MMLTTB_X_I64) return (double)__ldg((const long long*)sp.x + i);
  return __ldg((const double*)sp.x + i);
}
__device__ __forceinline__ double y_of(const SeriesPlan& sp, int64_t i) {
  if (sp.ydt == MMLTTB_F32) return (double)__ldg((const float*)sp.y + i);
  return __ldg((const double*)sp.y + i);
}
// Original index of LTTB position p (identity when LTTB runs on all points).
__device__ __forceinline__ int64_t index_of(const SeriesPlan& sp, int64_t p) {
  return sp.sel ? sp.sel[p] : p;
}
// Coordinates of LTTB position p: the compacted copies after preselection, else the
// original point p.
__device__ __forceinline__ void pos_xy(const SeriesPlan& sp, int64_t p, double* x, double* y) {
  if (sp.px) {
    *x = sp.px[p];
    *y = sp.py[p];
  } else {
    const int64_t i = index_of(sp, p);
    *x = x_of(sp, i);
    *y = y_of(sp, i);
  }
}

// LTTB triangle area (Sec. 2.2.1): |(xa-xc)(yb-ya) - (xa-xb)(yc-ya)|, every
// operation rounded on its own (no contraction into FMA).
__device__ __forceinline__ double tri_area(double xa, double ya, double xb, double yb,
                                           double xc, double yc) {
  double p1 = __dmul_rn(__dsub_rn(xa, xc), __dsub_rn(yb, ya));
  double p2 = __dmul_rn(__dsub_rn(xa, xb), __dsub_rn(yc, ya));
  return fabs(__dsub_rn(p1, p2));
}

// ---- host launchers (defined in minmax.cu / lttb.cu) ----
// Launch `kernel(bt)` with programmatic stream serialization allowed.
template <typename K>
inline cudaError_t launch_pdl(K kernel, dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                              const Batch& bt) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, bt);
}
cudaError_t launch_edges(const Batch& bt, cudaStream_t st);
constexpr int kTableRoundsMax = 7;  // k_tables: rounds of 32 slots per warp at most
// Stream-kernel variants (see stream_variant_info); launch_stream runs one of them
// over bt.n_warps warps.
constexpr int kStreamVariants = 6;
// ymode: 0 any y (dispatch per series), 1 float32 only, 2 float64 only, 3 float32
// NaN-aware only, 4 float64 NaN-aware only; see stream_ymode.
cudaError_t launch_stream(const Batch& bt, int variant, int ymode, cudaStream_t st);
// The staged stream over the series with bulk_bpt > 0 (bt.n_bulk_warps warps), and
// its resident CTAs per SM.
cudaError_t launch_stream_bulk(const Batch& bt, int ymode, cudaStream_t st);
int stream_bulk_blocks_per_sm();
// The stream-kernel y mode for series of y type ydt: the specialised kernel unless the
// NaN-aware rule applies.
inline int stream_ymode(int ydt, bool nan_aware) {
  if (nan_aware) return ydt == MMLTTB_F32 ? 3 : 4;
  return ydt == MMLTTB_F32 ? 1 : 2;
}
int stream_variant_info(int variant, int* unroll, int* min_blocks);
int stream_variant_threads(int variant);  // threads per CTA
// Compaction (A-2): per-bin resolve, per-series scan of CTA totals, placement.
cudaError_t launch_compact(const Batch& bt, cudaStream_t st);
cudaError_t launch_tables(const Batch& bt, cudaStream_t st);
cudaError_t launch_chain(const Batch& bt, int n_blocks, int64_t max_positions, cudaStream_t st);
cudaError_t launch_iota(int64_t* out, int64_t n, int64_t* out_count, cudaStream_t st);
// Large-bucket LTTB of the single series bt.one (lttb_big.cu): the next-bucket means and
// bucket statistics on every SM, then the chain as a fixpoint over all SMs (cooperative
// launch).  lttb_big_bytes(K): the workspace both need at sp.means.
cudaError_t launch_lttb_means(const Batch& bt, int sms, cudaStream_t st);
cudaError_t launch_lttb_fix(const Batch& bt, int sms, cudaStream_t st);
size_t lttb_big_bytes(int64_t K);
cudaError_t launch_lttb_block(const Batch& bt, int n_blocks, cudaStream_t st);
int stream_blocks_per_sm(int variant);
// Fused single-series kernel, one CTA per SM (fused.cu): its grid on a device with
// `sms` SMs (0 when it does not fit), the dynamic shared memory it stages tables in,
// its streaming warps, and the launch (with or without the edge search and the
// MinMax stream).
int fused_grid_size(int sms);
int64_t fused_tab_smem(int64_t tab_cap);
int fused_warps(int grid);
cudaError_t launch_fused(const Batch& bt, int grid, bool with_stream, cudaStream_t st);
// Clear the workspace header words a call's kernels use (status word and barrier
// counter); run by the first kernel of a call that has no header memset.
__device__ __forceinline__ void zero_header(const Batch& bt) {
  *bt.status = 0u;
  *bt.barrier = 0u;
}
constexpr int kGridThreads = 256;

}  // namespace mmlttb
