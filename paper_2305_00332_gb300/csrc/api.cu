// C ABI of libmmlttb: argument checks, planning, workspace layout and the launch
// sequence of the MinMaxLTTB hot path (arXiv 2305.00332, Sec. 3).
//
// Launch sequences for one series (all on the caller's stream, no host sync), by
// launch path (single_path):
//   split:       memset(header) -> [k_edges] -> k_stream -> k_bins -> k_binscan ->
//                k_place -> k_tables -> k_chain, or, when LTTB buckets are large,
//                [k_chain] -> k_lttb_means -> k_lttb_fix (a batch: k_lttb_block)
//   fused tail:  [k_edges] -> k_stream -> k_fused<0> (compaction and LTTB, one launch)
//   fused:       memset(header) -> k_fused<1> (the whole call in one persistent launch)
// or k_iota when every index is kept.
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <mutex>
#include <new>
#include <vector>

#include "host.h"

namespace mmlttb {


thread_local int g_last_cuda_error = 0;
thread_local unsigned long long g_launches = 0;
thread_local cudaEvent_t g_ev_start = nullptr;     // one-shot events around k_stream
thread_local cudaEvent_t g_ev_stop = nullptr;
thread_local cudaEvent_t g_stage_ev[16];            // one-shot events between the kernels
thread_local int g_stage_n = 0, g_stage_i = 0;

// Record the next armed stage event (if any) on `st`.
void stage_mark(cudaStream_t st) {
  if (g_stage_i < g_stage_n) cudaEventRecord(g_stage_ev[g_stage_i++], st);
}

void stage_disarm() { g_stage_n = g_stage_i = 0; }

int cuda_fail(cudaError_t e) {
  g_last_cuda_error = (int)e;
  return MMLTTB_ECUDA;
}

std::mutex g_dev_mu;
DevInfo g_dev[64];

int get_dev_info(DevInfo* out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e);
  std::lock_guard<std::mutex> lk(g_dev_mu);
  if (dev >= 0 && dev < 64 && g_dev[dev].ok) {
    *out = g_dev[dev];
    return MMLTTB_OK;
  }
  DevInfo d;
  d.device = dev;
  e = cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return cuda_fail(e);
  for (int v = 0; v < kStreamVariants; ++v) d.stream_bps[v] = stream_blocks_per_sm(v);
  d.fused_grid = fused_grid_size(d.sms);
  d.bulk_bps = stream_bulk_blocks_per_sm();
  d.ok = true;
  if (dev >= 0 && dev < 64) g_dev[dev] = d;
  *out = d;
  return MMLTTB_OK;
}

// Tuned stream variant per device and y type; a per-thread override while tuning.
std::atomic<int> g_variant[64][2];
thread_local int g_variant_override = -1;

int stream_variant(const DevInfo& d, int ydt) {
  if (g_variant_override >= 0) return g_variant_override;
  if (d.device < 0 || d.device >= 64 || ydt < 0 || ydt > 1) return 0;
  return g_variant[d.device][ydt].load();
}

// ---- tunings (mmlttb_tuning), per process under (device, y type, x kind, bin mode,
// size class)
constexpr int kSizeClasses = 13;
std::mutex g_tune_mu;
bool g_tune_set[64][2][3][2][kSizeClasses];
mmlttb_tuning g_tune[64][2][3][2][kSizeClasses];
thread_local const mmlttb_tuning* g_tune_override = nullptr;  // while tuning

int size_class(int64_t n) {
  int c = 0;
  while (n >= 10 && c < kSizeClasses - 1) {
    n /= 10;
    ++c;
  }
  return c;
}

bool tuning_valid(const mmlttb_tuning& t) {
  return t.variant >= 0 && t.variant < kStreamVariants && t.group_shift >= -1 && t.group_shift <= 1 &&
         t.tab_rounds >= 0 && t.tab_rounds <= kTableRoundsMax && t.reserved == 0;
}

bool tune_key_ok(const DevInfo& d, int ydt, int xk, int binmode) {
  return d.device >= 0 && d.device < 64 && (ydt == MMLTTB_F32 || ydt == MMLTTB_F64) && xk >= 0 && xk <= 2 &&
         (binmode == MMLTTB_BINS_INDEX || binmode == MMLTTB_BINS_XWIDTH);
}

mmlttb_tuning tuning_for(const DevInfo& d, int ydt, int xk, int binmode, int64_t n) {
  if (g_tune_override) return *g_tune_override;
  mmlttb_tuning t{stream_variant(d, ydt), 0, 0, 0};
  binmode &= ~MMLTTB_NAN_AWARE;
  if (tune_key_ok(d, ydt, xk, binmode)) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    const int c = size_class(n);
    if (g_tune_set[d.device][ydt][xk][binmode][c]) t = g_tune[d.device][ydt][xk][binmode][c];
  }
  if (g_variant_override >= 0) t.variant = g_variant_override;
  return t;
}

int shift_group(int G, int shift) {
  if (shift > 0) return G < 32 ? G << 1 : 32;
  if (shift < 0) return G > 1 ? G >> 1 : 1;
  return G;
}

int64_t stream_warp_cap(const DevInfo& d) {
  int64_t c = 0;
  for (int v = 0; v < kStreamVariants; ++v) {
    const int64_t w = (int64_t)d.sms * d.stream_bps[v] * (stream_variant_threads(v) / 32);
    if (w > c) c = w;
  }
  return c;
}

int64_t stream_warps(const DevInfo& d, int variant, int64_t work) {
  int64_t W = work / (kBinCostMax + 1);
  const int64_t cap = (int64_t)d.sms * d.stream_bps[variant] * (stream_variant_threads(variant) / 32);
  if (W > cap) W = cap;
  if (W < 1 && work > 0) W = 1;
  return W;
}

int64_t bulk_warps(const DevInfo& d, int64_t tiles) {
  const int64_t cap = (int64_t)d.sms * d.bulk_bps * kBulkWarps;
  return tiles < cap ? tiles : cap;
}

int64_t bulk_rec_w(int64_t pos_off, int64_t total, int64_t W) {
  if (total <= 0 || W <= 0) return 0;
  const int64_t w = warp_of(pos_off, make_div(total), W);
  return w < W ? w : W;
}

std::atomic<int> g_bulk_on{0};  // measured no faster overall: opt-in
bool bulk_enabled() { return g_bulk_on.load() != 0; }

struct SinglePlan {
  int32_t branch = BR_ARANGE, engine = EN_NONE;
  int64_t B = 0, K = 0, npos = 0, W = 0, Wcap = 0, tab_cap = 0;
  size_t off_edges = 0, off_rec = 0, off_sel = 0, off_tab = 0, off_means = 0;
  size_t off_binres = 0, off_ctasum = 0, off_ctaser = 0, off_ctaoff = 0, off_px = 0, off_py = 0;
  size_t off_ftot = 0;
  int64_t nct = 0;  // compaction CTAs
  int64_t nb = 0;   // binned points
  int group = 32;   // lanes per bin in the stream
  int tab_lgS = 0;  // log2 of the fused tables' slots per bucket
  int variant = 0;  // stream-kernel variant
  int tab_rounds = 0;  // k_tables rounds per warp (0: from the slot count)
  int64_t bulk_bpt = 0, tcost = 0, tiles = 0, Wb = 0;  // staged stream (bulk_bpt > 0)
  size_t total = kHeader;
};

int classify(int op, int ydt, int xk, int64_t n, int64_t n_out, int32_t r_ps, int binmode,
             int32_t* branch, int64_t* bins) {
  if (ydt != MMLTTB_F32 && ydt != MMLTTB_F64) return MMLTTB_EINVAL;
  if (xk != MMLTTB_X_IMPLICIT && xk != MMLTTB_X_I64 && xk != MMLTTB_X_F64) return MMLTTB_EINVAL;
  if (n < 0 || n_out < 0) return MMLTTB_EINVAL;
  const bool uses_bins = op == MMLTTB_OP_PRESELECT || op == MMLTTB_OP_MINMAXLTTB || op == MMLTTB_OP_M4;
  if (binmode & MMLTTB_NAN_AWARE) {  // NaN-aware aggregation: MinMax preselection and M4 only
    if (op != MMLTTB_OP_PRESELECT && op != MMLTTB_OP_M4) return MMLTTB_EINVAL;
    binmode &= ~MMLTTB_NAN_AWARE;
  }
  if (uses_bins) {
    if (binmode != MMLTTB_BINS_INDEX && binmode != MMLTTB_BINS_XWIDTH) return MMLTTB_EINVAL;
    if (binmode == MMLTTB_BINS_XWIDTH && xk == MMLTTB_X_IMPLICIT) return MMLTTB_EINVAL;
  }
  int64_t B = 0;
  int32_t br;
  switch (op) {
    case MMLTTB_OP_PRESELECT:
      if (n_out < 1 || r_ps < 1) return MMLTTB_EINVAL;
      if (n_out > INT64_MAX / r_ps) return MMLTTB_EINVAL;
      B = n_out * (int64_t)r_ps / 2;
      if (B < 1) return MMLTTB_EINVAL;
      br = BR_PRESELECT;
      break;
    case MMLTTB_OP_M4:
      if (n_out < 4) return MMLTTB_EINVAL;
      B = n_out / 4;
      br = BR_M4;
      break;
    case MMLTTB_OP_LTTB:
      if (n_out >= n) br = BR_ARANGE;
      else if (n_out < 3) return MMLTTB_EINVAL;
      else br = BR_LTTB_ALL;
      break;
    case MMLTTB_OP_MINMAXLTTB:
      if (n_out >= n) { br = BR_ARANGE; break; }
      if (n_out < 3 || r_ps < 2) return MMLTTB_EINVAL;
      if (n_out > INT64_MAX / r_ps) return MMLTTB_EINVAL;
      if ((int64_t)r_ps * n_out >= n) { br = BR_LTTB_ALL; break; }
      B = n_out * (int64_t)r_ps / 2;
      br = BR_MINMAX_LTTB;
      break;
    default:
      return MMLTTB_EINVAL;
  }
  if (B >= (int64_t(1) << 30)) return MMLTTB_EINVAL;  // bins are indexed with int on device
  *branch = br;
  *bins = B;
  return MMLTTB_OK;
}

int plan_single(int op, int ydt, int xk, int64_t n, int64_t n_out, int32_t r_ps, int binmode,
                const DevInfo& d, SinglePlan* P) {
  SinglePlan p;
  int rc = classify(op, ydt, xk, n, n_out, r_ps, binmode, &p.branch, &p.B);
  if (rc) return rc;
  binmode &= ~MMLTTB_NAN_AWARE;
  size_t off = kHeader;
  if (binned(p.branch)) {
    const int64_t N = p.branch == BR_M4 ? n : (n > 2 ? n - 2 : 0);
    p.nb = N;
    // x-width bins can be very uneven: keep whole warps per bin there
    const int eb = ydt == MMLTTB_F32 ? 4 : 8;
    const mmlttb_tuning tu = tuning_for(d, ydt, xk, binmode, n);
    p.variant = tu.variant;
    p.tab_rounds = tu.tab_rounds;
    const bool large = N * eb >= kStreamThroughputBytes;
    p.group = binmode == MMLTTB_BINS_XWIDTH
                  ? 32
                  : shift_group(large ? stream_group_single(N, p.B, eb) : stream_group(N, p.B, eb, false),
                                tu.group_shift);
    if (binmode == MMLTTB_BINS_INDEX && ydt == MMLTTB_F32 && N * eb >= kStreamThroughputBytes && bulk_enabled())
      p.bulk_bpt = bulk_bins_per_tile(N, p.B, eb);
    if (p.bulk_bpt > 0) {  // the staged stream: no register-stream work
      p.group = bulk_group(p.bulk_bpt);
      p.tiles = (p.B + p.bulk_bpt - 1) / p.bulk_bpt;
      p.tcost = p.bulk_bpt * (((N + p.B - 1) / p.B) * eb + kBulkBinCost);
      p.Wb = bulk_warps(d, p.tiles);
    }
    p.npos = p.bulk_bpt > 0 ? 0 : series_work(N, p.B, p.group);
    p.Wcap = stream_warp_cap(d);
    p.W = stream_warps(d, p.variant, p.npos);
    if (p.W > 0 && N / p.W >= (int64_t(1) << 30)) return MMLTTB_EINVAL;  // per-warp span
    if (binmode == MMLTTB_BINS_XWIDTH) {
      p.off_edges = off;
      off = align256(off + (size_t)(p.B + 1) * 8);
    }
    p.off_rec = off;
    off = align256(off + (size_t)(p.B + p.Wcap) * sizeof(Record));
    p.nct = (p.B + kBinsPerCta - 1) / kBinsPerCta;
    p.off_binres = off;
    off = align256(off + (size_t)p.nct * kBinsPerCta * 32);
    p.off_ctasum = off;
    off = align256(off + (size_t)p.nct * 4);
    p.off_ctaser = off;
    off = align256(off + (size_t)p.nct * 4);
    p.off_ctaoff = off;
    off = align256(off + (size_t)p.nct * 8);
  }
  if (p.branch != BR_ARANGE) {  // per-CTA words of the fused kernel
    p.off_ftot = off;
    off = align256(off + (size_t)d.sms * 8);
  }
  if (p.branch == BR_MINMAX_LTTB) {
    p.off_sel = off;
    off = align256(off + (size_t)(2 * p.B + 2) * 8);
    p.off_px = off;
    off = align256(off + (size_t)(2 * p.B + 2) * 8);
    p.off_py = off;
    off = align256(off + (size_t)(2 * p.B + 2) * 8);
  }
  if (p.branch == BR_LTTB_ALL || p.branch == BR_MINMAX_LTTB) {
    p.K = n_out - 2;
    const int64_t mcap = p.branch == BR_LTTB_ALL ? n : 2 * p.B + 2;
    p.engine = max_bucket(mcap, p.K) <= kTableMaxBucket ? EN_TABLES : EN_GRID;
    if (p.engine == EN_TABLES) {
      p.tab_cap = mcap;
      while ((int64_t(1) << p.tab_lgS) < max_bucket(mcap, p.K)) ++p.tab_lgS;
      p.off_tab = off;
      off = align256(off + (size_t)mcap);
    } else {
      p.off_means = off;  // means, bucket statistics, picks and worklists of the large-bucket engine
      off = align256(off + lttb_big_bytes(p.K));
    }
  }
  p.total = off;
  *P = p;
  return MMLTTB_OK;
}

// Single-series launch path.  The fused persistent kernel replaces the split
// compaction/LTTB kernels when the bins and table positions are few enough for its
// grid; series of up to kFusedStreamBytes of y also run the edge search and the
// MinMax stream inside it (one launch), larger ones run k_edges/k_stream first.
constexpr int64_t kFusedMaxBins = int64_t(1) << 18;
constexpr int64_t kFusedMaxSlots = int64_t(1) << 20;
constexpr int64_t kFusedStreamBytes = int64_t(8) << 20;
thread_local int g_path_override = MMLTTB_PATH_AUTO;

int single_path(const SinglePlan& p, const DevInfo& d, int64_t n, int ydt) {
  if (p.branch == BR_ARANGE || d.fused_grid <= 0 || g_path_override == MMLTTB_PATH_SPLIT)
    return MMLTTB_PATH_SPLIT;
  const bool lttb = p.branch == BR_LTTB_ALL || p.branch == BR_MINMAX_LTTB;
  if (lttb && p.engine != EN_TABLES) return MMLTTB_PATH_SPLIT;
  if (p.B > kFusedMaxBins || p.tab_cap > kFusedMaxSlots) return MMLTTB_PATH_SPLIT;
  if (!binned(p.branch)) return MMLTTB_PATH_FUSED_TAIL;  // LTTB on all points: tables + chain
  if (g_path_override == MMLTTB_PATH_FUSED_TAIL || g_path_override == MMLTTB_PATH_FUSED)
    return g_path_override;
  const int64_t bytes = n * (ydt == MMLTTB_F32 ? 4 : 8);
  return bytes <= kFusedStreamBytes ? MMLTTB_PATH_FUSED : MMLTTB_PATH_FUSED_TAIL;
}

int run_single(int op, const void* y, int ydt, const void* x, int xk, int64_t n, int64_t n_out,
               int32_t r_ps, int binmode, int64_t* out, int64_t out_cap, int64_t* out_count,
               void* ws, size_t ws_bytes, cudaStream_t st) {
  int32_t branch;
  int64_t bins;
  int rc = classify(op, ydt, xk, n, n_out, r_ps, binmode, &branch, &bins);
  if (rc) return rc;
  if (n > 0 && y == nullptr) return MMLTTB_EINVAL;
  if (xk != MMLTTB_X_IMPLICIT && n > 0 && x == nullptr) return MMLTTB_EINVAL;
  const int64_t need = branch == BR_PRESELECT ? (n < 2 * bins + 2 ? n : 2 * bins + 2)
                       : branch == BR_M4      ? (n < 4 * bins ? n : 4 * bins)
                                              : (n_out < n ? n_out : n);
  if (need > 0 && out == nullptr) return MMLTTB_EINVAL;
  if (out_cap < need) return MMLTTB_ERANGE;
  DevInfo d;
  rc = get_dev_info(&d);
  if (rc) return rc;
  SinglePlan p;
  rc = plan_single(op, ydt, xk, n, n_out, r_ps, binmode, d, &p);
  if (rc) return rc;
  if (ws == nullptr || ws_bytes < p.total) return MMLTTB_ENOSPC;

  char* w = (char*)ws;
  Batch bt;
  memset(&bt, 0, sizeof(bt));
  bt.plans = nullptr;
  bt.n_series = 1;
  bt.status = (unsigned*)w;
  bt.barrier = (unsigned*)(w + 4);
  SeriesPlan& sp = bt.one;
  sp.y = y;
  sp.x = xk == MMLTTB_X_IMPLICIT ? nullptr : x;
  sp.ydt = ydt;
  sp.xk = xk;
  sp.nan_aware = (binmode & MMLTTB_NAN_AWARE) ? 1 : 0;
  binmode &= ~MMLTTB_NAN_AWARE;
  sp.binmode = binmode;
  sp.branch = p.branch;
  sp.engine = p.engine;
  sp.r_ps = r_ps;
  sp.n = n;
  sp.n_out = n_out;
  sp.B = p.B;
  sp.bin_off = 0;
  sp.edge_off = 0;
  sp.pos_off = 0;
  sp.npos = p.npos;
  sp.tab_off = 0;
  sp.tab_cap = p.tab_cap;
  sp.m_ptr = (int64_t*)(w + 8);
  sp.p0 = p.branch == BR_M4 ? 0 : 1;
  sp.nb = p.nb;
  sp.group = p.group;
  sp.sel = (p.branch == BR_PRESELECT || p.branch == BR_M4) ? out
           : (p.branch == BR_MINMAX_LTTB ? (int64_t*)(w + p.off_sel) : nullptr);
  sp.px = p.branch == BR_MINMAX_LTTB ? (double*)(w + p.off_px) : nullptr;
  sp.py = p.branch == BR_MINMAX_LTTB ? (double*)(w + p.off_py) : nullptr;
  sp.bincta_off = 0;
  sp.tab = p.engine == EN_TABLES ? (uint8_t*)(w + p.off_tab) : nullptr;
  sp.means = p.engine == EN_GRID ? (double*)(w + p.off_means) : nullptr;
  sp.out = out;
  sp.out_count = out_count;
  sp.tab_lgS = p.tab_lgS;
  sp.bulk_bpt = p.bulk_bpt;
  sp.tcost_off = 0;
  sp.tcost = p.tcost;
  sp.rec_w = 0;
  set_bin_steps(sp);
  bt.total_pos = p.npos;
  bt.n_warps = p.W;
  bt.tcost_offs = nullptr;
  bt.tab_rounds_req = p.tab_rounds;
  bt.total_tcost = p.tiles * p.tcost;
  bt.n_bulk_warps = p.Wb;
  set_warp_divs(bt);
  bt.total_edges = (p.B > 0 && sp.binmode == MMLTTB_BINS_XWIDTH) ? p.B + 1 : 0;
  bt.total_slots = p.tab_cap;  // k_tables: one slot per position
  bt.rec = p.off_rec ? (Record*)(w + p.off_rec) : nullptr;
  bt.edges = p.off_edges ? (int64_t*)(w + p.off_edges) : nullptr;
  bt.total_bin_ctas = p.nct;
  bt.binres = p.off_binres ? (int64_t*)(w + p.off_binres) : nullptr;
  bt.cta_sum = p.off_ctasum ? (int32_t*)(w + p.off_ctasum) : nullptr;
  bt.cta_series = p.off_ctaser ? (int32_t*)(w + p.off_ctaser) : nullptr;
  bt.cta_off = p.off_ctaoff ? (int64_t*)(w + p.off_ctaoff) : nullptr;
  bt.fused_tot = p.off_ftot ? (int64_t*)(w + p.off_ftot) : nullptr;

  struct StageReset {  // the stage events are one-shot: disarm when this call returns
    ~StageReset() { g_stage_n = g_stage_i = 0; }
  } stage_reset;
  cudaError_t e;
  const int path = single_path(p, d, n, ydt);
  if (path != MMLTTB_PATH_SPLIT) {
    const int G = d.fused_grid;
    bt.chain_smem = fused_tab_smem(p.tab_cap);
    bt.dgrid = make_div(G);
    // the header words (status, barrier) are cleared by the first kernel of the
    // call, or by a memset when the fused kernel is the first
    const bool lead = path == MMLTTB_PATH_FUSED_TAIL && (bt.total_edges > 0 || p.W > 0 || p.Wb > 0);
    if (!lead && (e = cudaMemsetAsync(ws, 0, kHeader, st)) != cudaSuccess) return cuda_fail(e);
    stage_mark(st);
    if (path == MMLTTB_PATH_FUSED) {
      int64_t W = p.npos / (kBinCostMax + 1);
      if (W > fused_warps(G)) W = fused_warps(G);
      if (W < 1 && p.npos > 0) W = 1;
      bt.n_warps = W;
      set_warp_divs(bt);
      if ((e = launch_fused(bt, G, true, st)) != cudaSuccess) return cuda_fail(e);
      stage_mark(st);
      ++g_launches;
      return MMLTTB_OK;
    }
    bt.zero_status = lead ? 1 : 0;  // cleared by the first kernel launched
    if (bt.total_edges > 0) {
      if ((e = launch_edges(bt, st)) != cudaSuccess) return cuda_fail(e);
      stage_mark(st);
      ++g_launches;
      bt.zero_status = 0;
    }
    if (g_ev_start && (e = cudaEventRecord(g_ev_start, st)) != cudaSuccess) return cuda_fail(e);
    if (p.W > 0) {
      if ((e = launch_stream(bt, p.variant, stream_ymode(ydt, sp.nan_aware != 0), st)) != cudaSuccess)
        return cuda_fail(e);
      ++g_launches;
      bt.zero_status = 0;
    }
    if (p.Wb > 0) {
      if ((e = launch_stream_bulk(bt, stream_ymode(ydt, sp.nan_aware != 0), st)) != cudaSuccess)
        return cuda_fail(e);
      ++g_launches;
      bt.zero_status = 0;
    }
    if (p.Wb > 0 || p.W > 0) stage_mark(st);
    if (g_ev_stop && (e = cudaEventRecord(g_ev_stop, st)) != cudaSuccess) return cuda_fail(e);
    g_ev_start = g_ev_stop = nullptr;
    if ((e = launch_fused(bt, G, false, st)) != cudaSuccess) return cuda_fail(e);
    stage_mark(st);
    ++g_launches;
    return MMLTTB_OK;
  }
  e = cudaMemsetAsync(ws, 0, kHeader, st);
  if (e != cudaSuccess) return cuda_fail(e);
  stage_mark(st);
  if (p.branch == BR_ARANGE) {
    e = launch_iota(out, n, out_count, st);
    if (e != cudaSuccess) return cuda_fail(e);
    ++g_launches;
    return MMLTTB_OK;
  }
  if (binned(p.branch)) {
    if (bt.total_edges > 0) {
      if ((e = launch_edges(bt, st)) != cudaSuccess) return cuda_fail(e);
      stage_mark(st);
      ++g_launches;
    }
    if (g_ev_start && (e = cudaEventRecord(g_ev_start, st)) != cudaSuccess) return cuda_fail(e);
    if (p.W > 0) {
      if ((e = launch_stream(bt, p.variant, stream_ymode(ydt, sp.nan_aware != 0), st)) != cudaSuccess)
        return cuda_fail(e);
      ++g_launches;
    }
    if (p.Wb > 0) {
      if ((e = launch_stream_bulk(bt, stream_ymode(ydt, sp.nan_aware != 0), st)) != cudaSuccess)
        return cuda_fail(e);
      ++g_launches;
    }
    if (p.Wb > 0 || p.W > 0) stage_mark(st);
    if (g_ev_stop && (e = cudaEventRecord(g_ev_stop, st)) != cudaSuccess) return cuda_fail(e);
    g_ev_start = g_ev_stop = nullptr;
    if ((e = launch_compact(bt, st)) != cudaSuccess) return cuda_fail(e);
    stage_mark(st);
    g_launches += 3;
  }
  if (p.branch == BR_PRESELECT || p.branch == BR_M4) return MMLTTB_OK;
  if (p.engine == EN_TABLES) {
    if ((e = launch_tables(bt, st)) != cudaSuccess) return cuda_fail(e);
    stage_mark(st);
    if ((e = launch_chain(bt, 1, p.tab_cap, st)) != cudaSuccess) return cuda_fail(e);
    stage_mark(st);
    g_launches += 2;
  } else {
    if (p.branch == BR_MINMAX_LTTB) {
      if ((e = launch_chain(bt, 1, 0, st)) != cudaSuccess) return cuda_fail(e);
      ++g_launches;
    }
    // the means and bucket statistics on every SM, then the chain as a fixpoint
    if ((e = launch_lttb_means(bt, d.sms, st)) != cudaSuccess) return cuda_fail(e);
    stage_mark(st);
    ++g_launches;
    if ((e = launch_lttb_fix(bt, d.sms, st)) != cudaSuccess) return cuda_fail(e);
    stage_mark(st);
    ++g_launches;
  }
  return MMLTTB_OK;
}

// Device address of host memory the GPU may read in place (pinned or registered;
// with unified addressing it is the same address), or NULL.
const void* host_device_view(const void* p) {
  if (!p) return nullptr;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();  // clear the sticky-free error of an unknown pointer
    return nullptr;
  }
  if (a.type == cudaMemoryTypeHost && a.devicePointer) return a.devicePointer;
  return nullptr;
}

// Device layout of mmlttb_minmaxlttb_host: out | count | workspace | y | x.  Inputs
// read in place need only the part before y (inplace_total); pageable inputs are
// staged in y | x (total).
struct HostLayout {
  size_t y = 0, x = 0, out = 0, count = 0, ws = 0, ws_bytes = 0, inplace_total = 0, total = 0;
};

int host_layout(int ydt, int xk, int64_t n, int64_t n_out, int32_t r_ps, int binmode,
                HostLayout* L) {
  int32_t branch;
  int64_t bins;
  int rc = classify(MMLTTB_OP_MINMAXLTTB, ydt, xk, n, n_out, r_ps, binmode, &branch, &bins);
  if (rc) return rc;
  DevInfo d;
  rc = get_dev_info(&d);
  if (rc) return rc;
  SinglePlan p;
  rc = plan_single(MMLTTB_OP_MINMAXLTTB, ydt, xk, n, n_out, r_ps, binmode, d, &p);
  if (rc) return rc;
  const size_t es = ydt == MMLTTB_F32 ? 4 : 8;
  const int64_t cap = n_out < n ? n_out : n;
  HostLayout l;
  size_t off = 0;
  l.out = off;
  off = align256(off + (size_t)(cap > 0 ? cap : 1) * 8);
  l.count = off;
  off = align256(off + 8);
  l.ws = off;
  l.ws_bytes = p.total;
  off = align256(off + p.total);
  l.inplace_total = off;
  l.y = off;
  off = align256(off + (size_t)n * es);
  l.x = off;
  off = align256(off + (xk == MMLTTB_X_IMPLICIT ? 0 : (size_t)n * 8));
  l.total = off;
  *L = l;
  return MMLTTB_OK;
}


}  // namespace mmlttb

using namespace mmlttb;

extern "C" {

const char* mmlttb_strerror(int code) {
  switch (code) {
    case MMLTTB_OK: return "success";
    case MMLTTB_EINVAL: return "invalid argument";
    case MMLTTB_ENOSPC: return "workspace too small";
    case MMLTTB_ECUDA: return "CUDA error";
    case MMLTTB_ETIMEOUT: return "device-side wait timed out";
    case MMLTTB_ERANGE: return "output capacity too small";
    case MMLTTB_EDEVICE: return "device-side check failed";
    case MMLTTB_ENOMEM: return "host memory allocation failed";
    case MMLTTB_ESCRATCH: return "sizes exceed the 4 MiB static scratch of mmlttb_minmaxlttb_noalloc";
    case MMLTTB_EBUSY: return "server queue full";
    default: return "unknown error";
  }
}

int mmlttb_last_cuda_error(void) { return g_last_cuda_error; }

int mmlttb_version(void) { return 100; }

int mmlttb_workspace_bytes(int op, int ydtype, int xkind, int64_t n_in, int64_t n_out, int32_t r_ps,
                           int binmode, size_t* bytes) {
  if (!bytes) return MMLTTB_EINVAL;
  int32_t branch;
  int64_t bins;
  int rc = classify(op, ydtype, xkind, n_in, n_out, r_ps, binmode, &branch, &bins);
  if (rc) return rc;
  DevInfo d;
  rc = get_dev_info(&d);
  if (rc) return rc;
  SinglePlan p;
  rc = plan_single(op, ydtype, xkind, n_in, n_out, r_ps, binmode, d, &p);
  if (rc) return rc;
  *bytes = p.total;
  return MMLTTB_OK;
}

int mmlttb_minmax_preselect(const void* y, int ydtype, const void* x, int xkind, int64_t n_in,
                            int64_t n_out, int32_t r_ps, int binmode, int64_t* out_idx,
                            int64_t out_cap, int64_t* out_count, void* workspace,
                            size_t workspace_bytes, mmlttb_stream stream) {
  return run_single(MMLTTB_OP_PRESELECT, y, ydtype, x, xkind, n_in, n_out, r_ps, binmode, out_idx,
                    out_cap, out_count, workspace, workspace_bytes, (cudaStream_t)stream);
}

int mmlttb_m4(const void* y, int ydtype, const void* x, int xkind, int64_t n_in, int64_t n_out,
              int binmode, int64_t* out_idx, int64_t out_cap, int64_t* out_count, void* workspace,
              size_t workspace_bytes, mmlttb_stream stream) {
  return run_single(MMLTTB_OP_M4, y, ydtype, x, xkind, n_in, n_out, 4, binmode, out_idx, out_cap,
                    out_count, workspace, workspace_bytes, (cudaStream_t)stream);
}

int mmlttb_lttb(const void* y, int ydtype, const void* x, int xkind, int64_t n_in, int64_t n_out,
                int64_t* out_idx, int64_t out_cap, int64_t* out_count, void* workspace,
                size_t workspace_bytes, mmlttb_stream stream) {
  return run_single(MMLTTB_OP_LTTB, y, ydtype, x, xkind, n_in, n_out, 2, MMLTTB_BINS_INDEX, out_idx,
                    out_cap, out_count, workspace, workspace_bytes, (cudaStream_t)stream);
}

int mmlttb_minmaxlttb(const void* y, int ydtype, const void* x, int xkind, int64_t n_in,
                      int64_t n_out, int32_t r_ps, int binmode, int64_t* out_idx, int64_t out_cap,
                      int64_t* out_count, void* workspace, size_t workspace_bytes,
                      mmlttb_stream stream) {
  return run_single(MMLTTB_OP_MINMAXLTTB, y, ydtype, x, xkind, n_in, n_out, r_ps, binmode, out_idx,
                    out_cap, out_count, workspace, workspace_bytes, (cudaStream_t)stream);
}

int mmlttb_host_buffer_bytes(int ydtype, int xkind, int64_t n_in, int64_t n_out, int32_t r_ps,
                             int binmode, size_t* bytes) {
  if (!bytes) return MMLTTB_EINVAL;
  HostLayout l;
  int rc = host_layout(ydtype, xkind, n_in, n_out, r_ps, binmode, &l);
  if (rc) return rc;
  *bytes = l.total;
  return MMLTTB_OK;
}

int mmlttb_host_buffer_bytes_inplace(int ydtype, int xkind, int64_t n_in, int64_t n_out, int32_t r_ps,
                                     int binmode, size_t* bytes) {
  if (!bytes) return MMLTTB_EINVAL;
  HostLayout l;
  int rc = host_layout(ydtype, xkind, n_in, n_out, r_ps, binmode, &l);
  if (rc) return rc;
  *bytes = l.inplace_total;
  return MMLTTB_OK;
}

int mmlttb_minmaxlttb_host(const void* y_host, int ydtype, const void* x_host, int xkind,
                           int64_t n_in, int64_t n_out, int32_t r_ps, int binmode,
                           int64_t* out_host, int64_t out_cap, int64_t* out_count_host,
                           void* device_buffer, size_t device_bytes, mmlttb_stream stream) {
  HostLayout l;
  int rc = host_layout(ydtype, xkind, n_in, n_out, r_ps, binmode, &l);
  if (rc) return rc;
  if (n_in > 0 && y_host == nullptr) return MMLTTB_EINVAL;
  if (xkind != MMLTTB_X_IMPLICIT && n_in > 0 && x_host == nullptr) return MMLTTB_EINVAL;
  const int64_t need = n_out < n_in ? n_out : n_in;
  if (need > 0 && out_host == nullptr) return MMLTTB_EINVAL;
  if (out_cap < need) return MMLTTB_ERANGE;
  cudaStream_t st = (cudaStream_t)stream;
  char* b = (char*)device_buffer;
  const size_t es = ydtype == MMLTTB_F32 ? 4 : 8;
  cudaError_t e;
  // Pinned or registered host memory is read in place by the kernels (over the
  // CPU-GPU link): only the bytes the path touches cross it, i.e. every y once and x
  // only at bin-edge probes and preselected points, and the device buffer holds no
  // copy of the series.  Pageable memory is staged.
  const void* yd = host_device_view(y_host);
  const void* xd = xkind == MMLTTB_X_IMPLICIT ? nullptr : host_device_view(x_host);
  const bool staged = n_in > 0 && (!yd || (xkind != MMLTTB_X_IMPLICIT && !xd));
  if (device_buffer == nullptr || device_bytes < (staged ? l.total : l.inplace_total)) return MMLTTB_ENOSPC;
  if (staged) {
    if ((e = cudaMemcpyAsync(b + l.y, y_host, (size_t)n_in * es, cudaMemcpyHostToDevice, st)))
      return cuda_fail(e);
    yd = b + l.y;
    if (xkind != MMLTTB_X_IMPLICIT) {
      if ((e = cudaMemcpyAsync(b + l.x, x_host, (size_t)n_in * 8, cudaMemcpyHostToDevice, st)))
        return cuda_fail(e);
      xd = b + l.x;
    }
  }
  rc = run_single(MMLTTB_OP_MINMAXLTTB, yd, ydtype, xd, xkind, n_in, n_out, r_ps, binmode,
                  (int64_t*)(b + l.out), out_cap < need ? out_cap : need, (int64_t*)(b + l.count),
                  b + l.ws, l.ws_bytes, st);
  if (rc) return rc;
  if (need > 0 && (e = cudaMemcpyAsync(out_host, b + l.out, (size_t)need * 8, cudaMemcpyDeviceToHost, st)))
    return cuda_fail(e);
  if (out_count_host && (e = cudaMemcpyAsync(out_count_host, b + l.count, 8, cudaMemcpyDeviceToHost, st)))
    return cuda_fail(e);
  if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_fail(e);
  return MMLTTB_OK;
}



int mmlttb_stream_variant_info(int variant, int* unroll, int* min_blocks) {
  if (!unroll || !min_blocks) return MMLTTB_EINVAL;
  return stream_variant_info(variant, unroll, min_blocks) == 0 ? MMLTTB_OK : MMLTTB_EINVAL;
}

int mmlttb_get_stream_variant(int ydtype, int* variant) {
  if (!variant || (ydtype != MMLTTB_F32 && ydtype != MMLTTB_F64)) return MMLTTB_EINVAL;
  DevInfo d;
  int rc = get_dev_info(&d);
  if (rc) return rc;
  *variant = stream_variant(d, ydtype);
  return MMLTTB_OK;
}

int mmlttb_set_stream_variant(int ydtype, int variant) {
  if (ydtype != MMLTTB_F32 && ydtype != MMLTTB_F64) return MMLTTB_EINVAL;
  if (variant < 0 || variant >= kStreamVariants) return MMLTTB_EINVAL;
  DevInfo d;
  int rc = get_dev_info(&d);
  if (rc) return rc;
  if (d.device < 0 || d.device >= 64) return MMLTTB_EINVAL;
  g_variant[d.device][ydtype].store(variant);
  return MMLTTB_OK;
}

int mmlttb_autotune(int ydtype, const void* y, int64_t n_in, int64_t n_out, int32_t r_ps,
                    int64_t* out_idx, int64_t out_cap, void* workspace, size_t workspace_bytes,
                    mmlttb_stream stream, int* best_variant, float* best_ms) {
  if (!best_variant || (ydtype != MMLTTB_F32 && ydtype != MMLTTB_F64)) return MMLTTB_EINVAL;
  DevInfo d;
  int rc = get_dev_info(&d);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  cudaEvent_t a = nullptr, b = nullptr;
  cudaError_t e;
  if ((e = cudaEventCreate(&a)) != cudaSuccess || (e = cudaEventCreate(&b)) != cudaSuccess) {
    if (a) cudaEventDestroy(a);
    return cuda_fail(e);
  }
  float best = 3.0e38f;
  int bv = -1;
  const int saved_path = g_path_override;
  g_path_override = MMLTTB_PATH_SPLIT;  // time the stream kernel on its own
  for (int v = 0; v < kStreamVariants && !rc; ++v) {
    g_variant_override = v;
    float t[7];
    for (int r = 0; r < 3 + 7 && !rc; ++r) {
      if (r >= 3) {
        g_ev_start = a;
        g_ev_stop = b;
      }
      rc = run_single(MMLTTB_OP_PRESELECT, y, ydtype, nullptr, MMLTTB_X_IMPLICIT, n_in, n_out, r_ps,
                      MMLTTB_BINS_INDEX, out_idx, out_cap, nullptr, workspace, workspace_bytes, st);
      g_ev_start = g_ev_stop = nullptr;
      if (!rc && r >= 3) {
        if ((e = cudaEventSynchronize(b)) != cudaSuccess) rc = cuda_fail(e);
        else if ((e = cudaEventElapsedTime(&t[r - 3], a, b)) != cudaSuccess) rc = cuda_fail(e);
      }
    }
    if (rc) break;
    std::sort(t, t + 7);
    if (t[3] < best) {
      best = t[3];
      bv = v;
    }
  }
  g_variant_override = -1;
  g_path_override = saved_path;
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (rc) return rc;
  if (d.device >= 0 && d.device < 64) g_variant[d.device][ydtype].store(bv);
  *best_variant = bv;
  if (best_ms) *best_ms = best;
  return MMLTTB_OK;
}

int mmlttb_stream_variant_threads(int variant, int* threads) {
  if (!threads || variant < 0 || variant >= kStreamVariants) return MMLTTB_EINVAL;
  *threads = stream_variant_threads(variant);
  return MMLTTB_OK;
}

int mmlttb_set_tuning(int ydtype, int xkind, int binmode, int64_t n_in, const mmlttb_tuning* tuning) {
  if (!tuning || !tuning_valid(*tuning)) return MMLTTB_EINVAL;
  DevInfo d;
  int rc = get_dev_info(&d);
  if (rc) return rc;
  binmode &= ~MMLTTB_NAN_AWARE;
  if (!tune_key_ok(d, ydtype, xkind, binmode)) return MMLTTB_EINVAL;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  const int c = size_class(n_in);
  g_tune[d.device][ydtype][xkind][binmode][c] = *tuning;
  g_tune_set[d.device][ydtype][xkind][binmode][c] = true;
  return MMLTTB_OK;
}

int mmlttb_get_tuning(int ydtype, int xkind, int binmode, int64_t n_in, mmlttb_tuning* tuning) {
  if (!tuning) return MMLTTB_EINVAL;
  DevInfo d;
  int rc = get_dev_info(&d);
  if (rc) return rc;
  if (!tune_key_ok(d, ydtype, xkind, binmode & ~MMLTTB_NAN_AWARE)) return MMLTTB_EINVAL;
  *tuning = tuning_for(d, ydtype, xkind, binmode, n_in);
  return MMLTTB_OK;
}

int mmlttb_clear_tunings(void) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  memset(g_tune_set, 0, sizeof(g_tune_set));
  return MMLTTB_OK;
}

int mmlttb_autotune_tuple(int ydtype, const void* y, int xkind, const void* x, int64_t n_in, int64_t n_out,
                          int32_t r_ps, int binmode, int64_t* out_idx, int64_t out_cap, void* workspace,
                          size_t workspace_bytes, mmlttb_stream stream, mmlttb_tuning* best, float* best_ms) {
  if (!best) return MMLTTB_EINVAL;
  DevInfo d;
  int rc = get_dev_info(&d);
  if (rc) return rc;
  if (!tune_key_ok(d, ydtype, xkind, binmode & ~MMLTTB_NAN_AWARE)) return MMLTTB_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  cudaEvent_t a = nullptr, b = nullptr;
  cudaError_t e;
  if ((e = cudaEventCreate(&a)) != cudaSuccess || (e = cudaEventCreate(&b)) != cudaSuccess) {
    if (a) cudaEventDestroy(a);
    return cuda_fail(e);
  }
  mmlttb_tuning cand{0, 0, 0, 0}, win{0, 0, 0, 0};
  float win_ms = 3.0e38f;
  const int saved_path = g_path_override;
  g_path_override = MMLTTB_PATH_SPLIT;  // the stream and k_tables as kernels of their own
  g_tune_override = &cand;
  // the median of 7 timed runs after 3 untimed ones: the stream kernel (events armed
  // around it) or, with whole = true, the whole call
  auto timed = [&](int op, bool whole, float* ms) -> int {
    float t[7];
    for (int r = 0; r < 10; ++r) {
      if (r >= 3 && !whole) {
        g_ev_start = a;
        g_ev_stop = b;
      }
      if (r >= 3 && whole && (e = cudaEventRecord(a, st)) != cudaSuccess) return cuda_fail(e);
      int q = run_single(op, y, ydtype, x, xkind, n_in, n_out, r_ps, binmode, out_idx, out_cap, nullptr, workspace,
                         workspace_bytes, st);
      g_ev_start = g_ev_stop = nullptr;
      if (q) return q;
      if (r >= 3 && whole && (e = cudaEventRecord(b, st)) != cudaSuccess) return cuda_fail(e);
      if (r >= 3) {
        if ((e = cudaEventSynchronize(b)) != cudaSuccess) return cuda_fail(e);
        if ((e = cudaEventElapsedTime(&t[r - 3], a, b)) != cudaSuccess) return cuda_fail(e);
      }
    }
    std::sort(t, t + 7);
    *ms = t[3];
    return MMLTTB_OK;
  };
  for (int v = 0; v < kStreamVariants && !rc; ++v)
    for (int g = -1; g <= 1 && !rc; ++g) {
      cand = mmlttb_tuning{v, g, 0, 0};
      float ms = 0.0f;
      rc = timed(MMLTTB_OP_PRESELECT, false, &ms);
      if (!rc && ms < win_ms) {
        win_ms = ms;
        win = cand;
      }
    }
  float best_whole = 3.0e38f;
  const int rounds[4] = {0, 2, 4, 7};
  mmlttb_tuning win2 = win;
  for (int i = 0; i < 4 && !rc; ++i) {
    cand = win;
    cand.tab_rounds = rounds[i];
    float ms = 0.0f;
    rc = timed(MMLTTB_OP_MINMAXLTTB, true, &ms);
    if (!rc && ms < best_whole) {
      best_whole = ms;
      win2 = cand;
    }
  }
  g_tune_override = nullptr;
  g_path_override = saved_path;
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (rc) return rc;
  rc = mmlttb_set_tuning(ydtype, xkind, binmode, n_in, &win2);
  if (rc) return rc;
  *best = win2;
  if (best_ms) *best_ms = win_ms;
  return MMLTTB_OK;
}

int mmlttb_set_stage_events(void* const* events, int count) {
  if (count < 0 || count > 16 || (count > 0 && !events)) return MMLTTB_EINVAL;
  for (int i = 0; i < count; ++i) g_stage_ev[i] = (cudaEvent_t)events[i];
  g_stage_n = count;
  g_stage_i = 0;
  return MMLTTB_OK;
}

int mmlttb_set_timing_events(void* start_event, void* stop_event) {
  g_ev_start = (cudaEvent_t)start_event;
  g_ev_stop = (cudaEvent_t)stop_event;
  return MMLTTB_OK;
}

unsigned long long mmlttb_launch_count(void) { return g_launches; }

int mmlttb_set_stream_staging(int enable) {
  if (enable != 0 && enable != 1) return MMLTTB_EINVAL;
  g_bulk_on.store(enable);
  return MMLTTB_OK;
}

int mmlttb_get_stream_staging(int* enable) {
  if (!enable) return MMLTTB_EINVAL;
  *enable = g_bulk_on.load();
  return MMLTTB_OK;
}

int mmlttb_set_single_path(int path) {
  if (path < MMLTTB_PATH_AUTO || path > MMLTTB_PATH_FUSED) return MMLTTB_EINVAL;
  g_path_override = path;
  return MMLTTB_OK;
}

int mmlttb_single_path(int op, int ydtype, int xkind, int64_t n_in, int64_t n_out, int32_t r_ps,
                       int binmode) {
  DevInfo d;
  int rc = get_dev_info(&d);
  if (rc) return rc;
  SinglePlan p;
  rc = plan_single(op, ydtype, xkind, n_in, n_out, r_ps, binmode, d, &p);
  if (rc) return rc;
  return single_path(p, d, n_in, ydtype);
}

int mmlttb_stream_tiles(int op, int ydtype, int xkind, int64_t n_in, int64_t n_out, int32_t r_ps, int binmode,
                       int64_t* bins_per_tile) {
  if (!bins_per_tile) return MMLTTB_EINVAL;
  DevInfo d;
  int rc = get_dev_info(&d);
  if (rc) return rc;
  SinglePlan p;
  rc = plan_single(op, ydtype, xkind, n_in, n_out, r_ps, binmode, d, &p);
  if (rc) return rc;
  *bins_per_tile = p.bulk_bpt;
  return MMLTTB_OK;
}

int mmlttb_workspace_status(const void* workspace, int* status, mmlttb_stream stream) {
  if (!workspace || !status) return MMLTTB_EINVAL;
  unsigned v = 0;
  cudaError_t e = cudaMemcpyAsync(&v, workspace, sizeof(v), cudaMemcpyDeviceToHost, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e);
  e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e);
  *status = (int)v;
  return MMLTTB_OK;
}

}  // extern "C"

// ---------------------------------------------------------------- no-allocation variant
// Some callers cannot allocate device memory at the moment they need a result:
// latency-critical loops whose owners forbid allocation because cudaMalloc/cudaFree
// can synchronize the whole device and stall unrelated streams, and plugin hosts
// (a database function, a chart server extension) that hand out no allocator at all.
// For them mmlttb_minmaxlttb_noalloc runs on a scratch array that is part of the
// library image itself: every GPU that loads the library keeps these bytes reserved
// until the process exits.
namespace {

constexpr size_t kNoAllocScratchBytes = size_t(4) << 20;  // 4 MiB
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_noalloc_mu;
void* g_noalloc_addr[64] = {};

// Device address of the scratch array on the current device.  In host code the
// symbol g_noalloc_scratch is only a host-side stand-in, so the address is taken
// once per device, with that device current, through cudaGetSymbolAddress.
int noalloc_scratch(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e);
  if (dev < 0 || dev >= 64) return MMLTTB_EINVAL;
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(e);
    g_noalloc_addr[dev] = p;
  }
  *out = g_noalloc_addr[dev];
  return MMLTTB_OK;
}

}  // namespace

extern "C" int mmlttb_minmaxlttb_noalloc(const void* y, int ydtype, const void* x, int xkind,
                                         int64_t n_in, int64_t n_out, int32_t r_ps, int binmode,
                                         int64_t* out_idx, int64_t out_cap, int64_t* out_count,
                                         mmlttb_stream stream) {
  int32_t branch;
  int64_t bins;
  int rc = classify(MMLTTB_OP_MINMAXLTTB, ydtype, xkind, n_in, n_out, r_ps, binmode, &branch, &bins);
  if (rc) return rc;
  DevInfo d;
  rc = get_dev_info(&d);
  if (rc) return rc;
  SinglePlan p;
  rc = plan_single(MMLTTB_OP_MINMAXLTTB, ydtype, xkind, n_in, n_out, r_ps, binmode, d, &p);
  if (rc) return rc;
  if (p.total > kNoAllocScratchBytes) return MMLTTB_ESCRATCH;
  void* scratch = nullptr;
  rc = noalloc_scratch(&scratch);
  if (rc) return rc;
  // run_single clears the scratch header (status word, barrier counter, counts) on
  // the stream before its first kernel; every other byte it reads is written first.
  return run_single(MMLTTB_OP_MINMAXLTTB, y, ydtype, x, xkind, n_in, n_out, r_ps, binmode, out_idx,
                    out_cap, out_count, scratch, kNoAllocScratchBytes, (cudaStream_t)stream);
}

extern "C" int mmlttb_noalloc_status(int* status, mmlttb_stream stream) {
  if (!status) return MMLTTB_EINVAL;
  void* scratch = nullptr;
  int rc = noalloc_scratch(&scratch);
  if (rc) return rc;
  // The status word is the first word of the header, as in a caller's workspace.
  return mmlttb_workspace_status(scratch, status, stream);
}
