// C ABI of libmmlttb: argument checks, planning, workspace layout and the launch
// sequence of the MinMaxLTTB hot path (arXiv 2305.00332, Sec. 3).
//
// Launch sequence for one series (all on the caller's stream, no host sync):
//   memset(header) -> [k_edges] -> k_stream -> k_merge -> k_tables -> k_chain
// (or k_lttb_grid instead of the table pair when LTTB buckets are large), or
// k_iota when every index is kept.
#include <stdio.h>
#include <string.h>

#include <mutex>
#include <new>
#include <vector>

#include "common.cuh"

using namespace mmlttb;

namespace {

thread_local int g_last_cuda_error = 0;
thread_local unsigned long long g_launches = 0;   // kernels launched by this thread
thread_local cudaEvent_t g_ev_start = nullptr;     // one-shot events around k_stream
thread_local cudaEvent_t g_ev_stop = nullptr;

int cuda_fail(cudaError_t e) {
  g_last_cuda_error = (int)e;
  return MMLTTB_ECUDA;
}

struct DevInfo {
  int sms = 0;
  int stream_bps = 0;
  int grid_bps = 0;
  bool ok = false;
};

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
  e = cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return cuda_fail(e);
  d.stream_bps = stream_blocks_per_sm();
  d.grid_bps = lttb_grid_blocks_per_sm();
  d.ok = true;
  if (dev >= 0 && dev < 64) g_dev[dev] = d;
  *out = d;
  return MMLTTB_OK;
}

size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

constexpr size_t kHeader = 256;  // status word @0, barrier counter @4, m @8

struct SinglePlan {
  int32_t branch = BR_ARANGE, engine = EN_NONE;
  int64_t B = 0, K = 0, npos = 0, W = 0, Wcap = 0, tab_cap = 0;
  int grid_lttb = 0;
  size_t off_edges = 0, off_rec = 0, off_sel = 0, off_tab = 0, off_means = 0, off_partial = 0;
  size_t total = kHeader;
};

// Largest LTTB bucket over m positions with K buckets: ceil((m-2)/K).
int64_t max_bucket(int64_t m, int64_t K) { return (m - 2 + K - 1) / K; }

// Host-only validation and branch choice (Sec. 3 dispatch); needs no device.
int classify(int op, int ydt, int xk, int64_t n, int64_t n_out, int32_t r_ps, int binmode,
             int32_t* branch, int64_t* bins) {
  if (ydt != MMLTTB_F32 && ydt != MMLTTB_F64) return MMLTTB_EINVAL;
  if (xk != MMLTTB_X_IMPLICIT && xk != MMLTTB_X_I64 && xk != MMLTTB_X_F64) return MMLTTB_EINVAL;
  if (n < 0 || n_out < 0) return MMLTTB_EINVAL;
  const bool uses_bins = op == MMLTTB_OP_PRESELECT || op == MMLTTB_OP_MINMAXLTTB;
  if (uses_bins) {
    if (binmode != MMLTTB_BINS_INDEX && binmode != MMLTTB_BINS_XWIDTH) return MMLTTB_EINVAL;
    if (binmode == MMLTTB_BINS_XWIDTH && xk != MMLTTB_X_I64) return MMLTTB_EINVAL;
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
  size_t off = kHeader;
  if (p.branch == BR_PRESELECT || p.branch == BR_MINMAX_LTTB) {
    p.npos = n > 2 ? n - 2 : 0;
    p.Wcap = (int64_t)d.sms * d.stream_bps * kStreamWarps;
    p.W = p.npos < p.Wcap ? p.npos : p.Wcap;
    if (p.W > 0 && p.npos / p.W >= (int64_t(1) << 30)) return MMLTTB_EINVAL;  // per-warp span
    if (binmode == MMLTTB_BINS_XWIDTH) {
      p.off_edges = off;
      off = align256(off + (size_t)(p.B + 1) * 8);
    }
    p.off_rec = off;
    off = align256(off + (size_t)(p.B + p.Wcap) * sizeof(Record));
  }
  if (p.branch == BR_MINMAX_LTTB) {
    p.off_sel = off;
    off = align256(off + (size_t)(2 * p.B + 2) * 8);
  }
  if (p.branch == BR_LTTB_ALL || p.branch == BR_MINMAX_LTTB) {
    p.K = n_out - 2;
    const int64_t mcap = p.branch == BR_LTTB_ALL ? n : 2 * p.B + 2;
    p.engine = max_bucket(mcap, p.K) <= kTableMaxBucket ? EN_TABLES : EN_GRID;
    if (p.engine == EN_TABLES) {
      p.tab_cap = mcap;
      p.off_tab = off;
      off = align256(off + (size_t)mcap);
    } else {
      p.grid_lttb = d.sms * d.grid_bps;
      p.off_means = off;
      off = align256(off + (size_t)p.K * 16);
      p.off_partial = off;
      off = align256(off + (size_t)p.grid_lttb * 32);
    }
  }
  p.total = off;
  *P = p;
  return MMLTTB_OK;
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
  sp.sel = p.branch == BR_PRESELECT ? out : (p.branch == BR_MINMAX_LTTB ? (int64_t*)(w + p.off_sel) : nullptr);
  sp.tab = p.engine == EN_TABLES ? (uint8_t*)(w + p.off_tab) : nullptr;
  sp.means = p.engine == EN_GRID ? (double*)(w + p.off_means) : nullptr;
  sp.out = out;
  sp.out_count = out_count;
  bt.total_pos = p.npos;
  bt.n_warps = p.W;
  bt.total_edges = (p.B > 0 && binmode == MMLTTB_BINS_XWIDTH) ? p.B + 1 : 0;
  bt.total_slots = p.tab_cap;
  bt.rec = p.off_rec ? (Record*)(w + p.off_rec) : nullptr;
  bt.edges = p.off_edges ? (int64_t*)(w + p.off_edges) : nullptr;
  bt.partial = p.off_partial ? (double*)(w + p.off_partial) : nullptr;

  cudaError_t e = cudaMemsetAsync(ws, 0, kHeader, st);
  if (e != cudaSuccess) return cuda_fail(e);
  if (p.branch == BR_ARANGE) {
    e = launch_iota(out, n, out_count, st);
    if (e != cudaSuccess) return cuda_fail(e);
    ++g_launches;
    return MMLTTB_OK;
  }
  if (p.branch == BR_PRESELECT || p.branch == BR_MINMAX_LTTB) {
    if (bt.total_edges > 0) {
      if ((e = launch_edges(bt, st)) != cudaSuccess) return cuda_fail(e);
      ++g_launches;
    }
    if (g_ev_start && (e = cudaEventRecord(g_ev_start, st)) != cudaSuccess) return cuda_fail(e);
    if (p.W > 0) {
      const int64_t grid = (p.W + kStreamWarps - 1) / kStreamWarps;
      if ((e = launch_stream(bt, grid, st)) != cudaSuccess) return cuda_fail(e);
      ++g_launches;
    }
    if (g_ev_stop && (e = cudaEventRecord(g_ev_stop, st)) != cudaSuccess) return cuda_fail(e);
    g_ev_start = g_ev_stop = nullptr;
    if ((e = launch_merge(bt, 1, st)) != cudaSuccess) return cuda_fail(e);
    ++g_launches;
  }
  if (p.branch == BR_PRESELECT) return MMLTTB_OK;
  if (p.engine == EN_TABLES) {
    if ((e = launch_tables(bt, st)) != cudaSuccess) return cuda_fail(e);
    if ((e = launch_chain(bt, 1, st)) != cudaSuccess) return cuda_fail(e);
    g_launches += 2;
  } else {
    if (p.branch == BR_MINMAX_LTTB) {
      if ((e = launch_chain(bt, 1, st)) != cudaSuccess) return cuda_fail(e);
      ++g_launches;
    }
    if ((e = launch_lttb_grid(bt, p.grid_lttb, st)) != cudaSuccess) return cuda_fail(e);
    ++g_launches;
  }
  return MMLTTB_OK;
}

// Device staging layout of mmlttb_minmaxlttb_host: y | x | out | count | workspace.
struct HostLayout {
  size_t y = 0, x = 0, out = 0, count = 0, ws = 0, ws_bytes = 0, total = 0;
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
  l.y = off;
  off = align256(off + (size_t)n * es);
  l.x = off;
  off = align256(off + (xk == MMLTTB_X_IMPLICIT ? 0 : (size_t)n * 8));
  l.out = off;
  off = align256(off + (size_t)(cap > 0 ? cap : 1) * 8);
  l.count = off;
  off = align256(off + 8);
  l.ws = off;
  l.ws_bytes = p.total;
  off = align256(off + p.total);
  l.total = off;
  *L = l;
  return MMLTTB_OK;
}


// ---------------------------------------------------------------- batches
// A batch plans many series once (host), lays them out in one caller-owned
// workspace, uploads the plan table with one copy from pinned host memory, and runs
// the same kernels as a single series over all of them: one MinMax stream over the
// concatenated interior points, one merge CTA per series, one table pass over all
// positions, one chain CTA per series.  The launch sequence can be captured into a
// CUDA graph once and replayed.
struct BatchImpl {
  std::vector<mmlttb_series_desc> descs;
  std::vector<SeriesPlan> plans;  // pointer fields filled per workspace address
  int64_t n = 0;
  int64_t total_pos = 0, total_bins = 0, total_edges = 0, total_slots = 0;
  int64_t Wcap = 0, W = 0;
  bool any_block = false;
  size_t off_plans = 0, off_pos = 0, off_edge = 0, off_tab = 0, off_m = 0, off_edges = 0,
         off_rec = 0, off_sel = 0, off_tabs = 0, off_means = 0, total = kHeader, upload_bytes = 0;
  std::vector<int64_t> sel_off, tab_byte_off, mean_off;
  char* pinned = nullptr;       // upload image: plans | pos_offs | edge_offs | tab_offs
  const void* bound_ws = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  const void* graph_ws = nullptr;
  cudaStream_t capture_stream = nullptr;
  int graph_launches = 0;
  ~BatchImpl() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    if (capture_stream) cudaStreamDestroy(capture_stream);
    if (pinned) cudaFreeHost(pinned);
  }
};

int batch_plan(BatchImpl* b, const DevInfo& d) {
  const int64_t n = b->n;
  b->plans.assign(n, SeriesPlan{});
  b->sel_off.assign(n, -1);
  b->tab_byte_off.assign(n, -1);
  b->mean_off.assign(n, -1);
  int64_t pos = 0, bins = 0, edges = 0, slots = 0, sel = 0, means = 0;
  for (int64_t s = 0; s < n; ++s) {
    const mmlttb_series_desc& D = b->descs[s];
    int32_t br;
    int64_t B;
    int rc = classify(D.op, D.ydtype, D.xkind, D.n_in, D.n_out, D.r_ps, D.binmode, &br, &B);
    if (rc) return rc;
    if (D.n_in > 0 && D.y == nullptr) return MMLTTB_EINVAL;
    if (D.xkind != MMLTTB_X_IMPLICIT && D.n_in > 0 && D.x == nullptr) return MMLTTB_EINVAL;
    const int64_t need = br == BR_PRESELECT ? (D.n_in < 2 * B + 2 ? D.n_in : 2 * B + 2)
                                            : (D.n_out < D.n_in ? D.n_out : D.n_in);
    if (need > 0 && D.out_idx == nullptr) return MMLTTB_EINVAL;
    if (D.out_cap < need) return MMLTTB_ERANGE;
    SeriesPlan& sp = b->plans[s];
    sp.y = D.y;
    sp.x = D.xkind == MMLTTB_X_IMPLICIT ? nullptr : D.x;
    sp.ydt = D.ydtype;
    sp.xk = D.xkind;
    sp.binmode = D.binmode;
    sp.branch = br;
    sp.r_ps = D.r_ps;
    sp.n = D.n_in;
    sp.n_out = D.n_out;
    sp.B = B;
    sp.out = D.out_idx;
    sp.out_count = D.out_count;
    sp.bin_off = bins;
    sp.pos_off = pos;
    sp.edge_off = edges;
    sp.tab_off = slots;
    const bool mm = br == BR_PRESELECT || br == BR_MINMAX_LTTB;
    if (mm) {
      sp.npos = D.n_in > 2 ? D.n_in - 2 : 0;
      pos += sp.npos;
      bins += B;
      if (D.binmode == MMLTTB_BINS_XWIDTH) edges += B + 1;
    }
    if (br == BR_MINMAX_LTTB) {
      b->sel_off[s] = sel;
      sel += 2 * B + 2;
    }
    if (br == BR_LTTB_ALL || br == BR_MINMAX_LTTB) {
      const int64_t K = D.n_out - 2;
      const int64_t mcap = br == BR_LTTB_ALL ? D.n_in : 2 * B + 2;
      if (max_bucket(mcap, K) <= kTableMaxBucket) {
        sp.engine = EN_TABLES;
        sp.tab_cap = mcap;
        b->tab_byte_off[s] = slots;
        slots += mcap;
      } else {
        sp.engine = EN_BLOCK;
        b->any_block = true;
        b->mean_off[s] = means;
        means += 2 * K;
      }
    }
  }
  b->total_pos = pos;
  b->total_bins = bins;
  b->total_edges = edges;
  b->total_slots = slots;
  b->Wcap = (int64_t)d.sms * d.stream_bps * kStreamWarps;
  b->W = pos < b->Wcap ? pos : b->Wcap;
  if (b->W > 0 && pos / b->W >= (int64_t(1) << 30)) return MMLTTB_EINVAL;
  size_t off = kHeader;
  auto take = [&](size_t bytes) { size_t o = off; off = align256(off + bytes); return o; };
  b->off_plans = take((size_t)n * sizeof(SeriesPlan));
  b->off_pos = take((size_t)(n + 1) * 8);
  b->off_edge = take((size_t)(n + 1) * 8);
  b->off_tab = take((size_t)(n + 1) * 8);
  b->upload_bytes = off - b->off_plans;
  b->off_m = take((size_t)n * 8);
  b->off_edges = take((size_t)edges * 8);
  b->off_rec = take((size_t)(bins + b->Wcap) * sizeof(Record));
  b->off_sel = take((size_t)sel * 8);
  b->off_tabs = take((size_t)slots);
  b->off_means = take((size_t)means * 8);
  b->total = off;
  cudaError_t e = cudaHostAlloc((void**)&b->pinned, b->upload_bytes, cudaHostAllocDefault);
  if (e != cudaSuccess) return cuda_fail(e);
  // the offset tables never depend on the workspace address
  int64_t* po = (int64_t*)(b->pinned + (b->off_pos - b->off_plans));
  int64_t* eo = (int64_t*)(b->pinned + (b->off_edge - b->off_plans));
  int64_t* to = (int64_t*)(b->pinned + (b->off_tab - b->off_plans));
  for (int64_t s = 0; s < n; ++s) {
    po[s] = b->plans[s].pos_off;
    eo[s] = b->plans[s].edge_off;
    to[s] = b->plans[s].tab_off;
  }
  po[n] = pos;
  eo[n] = edges;
  to[n] = slots;
  return MMLTTB_OK;
}

// Point every plan at its sections of workspace `ws` and refresh the upload image.
void batch_bind(BatchImpl* b, void* ws) {
  char* w = (char*)ws;
  for (int64_t s = 0; s < b->n; ++s) {
    SeriesPlan& sp = b->plans[s];
    sp.m_ptr = (int64_t*)(w + b->off_m) + s;
    sp.sel = sp.branch == BR_PRESELECT ? sp.out
             : sp.branch == BR_MINMAX_LTTB ? (int64_t*)(w + b->off_sel) + b->sel_off[s] : nullptr;
    sp.tab = sp.engine == EN_TABLES ? (uint8_t*)(w + b->off_tabs) + b->tab_byte_off[s] : nullptr;
    sp.means = sp.engine == EN_BLOCK ? (double*)(w + b->off_means) + b->mean_off[s] : nullptr;
  }
  memcpy(b->pinned, b->plans.data(), (size_t)b->n * sizeof(SeriesPlan));
  b->bound_ws = ws;
}

Batch batch_args(const BatchImpl* b, void* ws) {
  char* w = (char*)ws;
  Batch bt;
  memset(&bt, 0, sizeof(bt));
  bt.plans = (const SeriesPlan*)(w + b->off_plans);
  bt.pos_offs = (const int64_t*)(w + b->off_pos);
  bt.edge_offs = (const int64_t*)(w + b->off_edge);
  bt.tab_offs = (const int64_t*)(w + b->off_tab);
  bt.n_series = (int32_t)b->n;
  bt.total_pos = b->total_pos;
  bt.n_warps = b->W;
  bt.total_edges = b->total_edges;
  bt.total_slots = b->total_slots;
  bt.rec = (Record*)(w + b->off_rec);
  bt.edges = (int64_t*)(w + b->off_edges);
  bt.status = (unsigned*)w;
  bt.barrier = (unsigned*)(w + 4);
  return bt;
}

// Enqueue the whole batch on `st`: upload, then the kernels (capturable).
int batch_enqueue(BatchImpl* b, void* ws, cudaStream_t st) {
  if (b->bound_ws != ws) batch_bind(b, ws);
  const Batch bt = batch_args(b, ws);
  cudaError_t e;
  if ((e = cudaMemsetAsync(ws, 0, kHeader, st)) != cudaSuccess) return cuda_fail(e);
  if ((e = cudaMemcpyAsync((char*)ws + b->off_plans, b->pinned, b->upload_bytes,
                           cudaMemcpyHostToDevice, st)) != cudaSuccess)
    return cuda_fail(e);
  const int nb = (int)b->n;
  if (bt.total_edges > 0) {
    if ((e = launch_edges(bt, st)) != cudaSuccess) return cuda_fail(e);
    ++g_launches;
  }
  if (b->W > 0) {
    const int64_t grid = (b->W + kStreamWarps - 1) / kStreamWarps;
    if ((e = launch_stream(bt, grid, st)) != cudaSuccess) return cuda_fail(e);
    if ((e = launch_merge(bt, nb, st)) != cudaSuccess) return cuda_fail(e);
    g_launches += 2;
  } else if (b->total_bins > 0 || b->total_pos == 0) {
    // series with n <= 2 still need their trivial preselected list
    if ((e = launch_merge(bt, nb, st)) != cudaSuccess) return cuda_fail(e);
    ++g_launches;
  }
  if (bt.total_slots > 0) {
    if ((e = launch_tables(bt, st)) != cudaSuccess) return cuda_fail(e);
    ++g_launches;
  }
  if ((e = launch_chain(bt, nb, st)) != cudaSuccess) return cuda_fail(e);
  ++g_launches;
  if (b->any_block) {
    if ((e = launch_lttb_block(bt, nb, st)) != cudaSuccess) return cuda_fail(e);
    ++g_launches;
  }
  return MMLTTB_OK;
}

}  // namespace

struct mmlttb_batch {
  BatchImpl impl;
};

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
  if (device_buffer == nullptr || device_bytes < l.total) return MMLTTB_ENOSPC;
  cudaStream_t st = (cudaStream_t)stream;
  char* b = (char*)device_buffer;
  const size_t es = ydtype == MMLTTB_F32 ? 4 : 8;
  cudaError_t e;
  if (n_in > 0 && (e = cudaMemcpyAsync(b + l.y, y_host, (size_t)n_in * es, cudaMemcpyHostToDevice, st)))
    return cuda_fail(e);
  if (xkind != MMLTTB_X_IMPLICIT && n_in > 0 &&
      (e = cudaMemcpyAsync(b + l.x, x_host, (size_t)n_in * 8, cudaMemcpyHostToDevice, st)))
    return cuda_fail(e);
  rc = run_single(MMLTTB_OP_MINMAXLTTB, b + l.y, ydtype, xkind == MMLTTB_X_IMPLICIT ? nullptr : b + l.x,
                  xkind, n_in, n_out, r_ps, binmode, (int64_t*)(b + l.out), out_cap < need ? out_cap : need,
                  (int64_t*)(b + l.count), b + l.ws, l.ws_bytes, st);
  if (rc) return rc;
  if (need > 0 && (e = cudaMemcpyAsync(out_host, b + l.out, (size_t)need * 8, cudaMemcpyDeviceToHost, st)))
    return cuda_fail(e);
  if (out_count_host && (e = cudaMemcpyAsync(out_count_host, b + l.count, 8, cudaMemcpyDeviceToHost, st)))
    return cuda_fail(e);
  if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_fail(e);
  return MMLTTB_OK;
}


int mmlttb_batch_create(const mmlttb_series_desc* descs, int64_t n_series, mmlttb_batch_t* out) {
  if (!out || n_series < 1 || n_series > INT32_MAX || !descs) return MMLTTB_EINVAL;
  *out = nullptr;
  DevInfo d;
  int rc = get_dev_info(&d);
  if (rc) return rc;
  mmlttb_batch* b = new (std::nothrow) mmlttb_batch;
  if (!b) return MMLTTB_ENOMEM;
  b->impl.n = n_series;
  b->impl.descs.assign(descs, descs + n_series);
  rc = batch_plan(&b->impl, d);
  if (rc) {
    delete b;
    return rc;
  }
  *out = b;
  return MMLTTB_OK;
}

int mmlttb_batch_workspace_bytes(mmlttb_batch_t batch, size_t* bytes) {
  if (!batch || !bytes) return MMLTTB_EINVAL;
  *bytes = batch->impl.total;
  return MMLTTB_OK;
}

int mmlttb_batch_run(mmlttb_batch_t batch, void* workspace, size_t workspace_bytes,
                     mmlttb_stream stream) {
  if (!batch) return MMLTTB_EINVAL;
  if (!workspace || workspace_bytes < batch->impl.total) return MMLTTB_ENOSPC;
  return batch_enqueue(&batch->impl, workspace, (cudaStream_t)stream);
}

int mmlttb_batch_run_graph(mmlttb_batch_t batch, void* workspace, size_t workspace_bytes,
                           mmlttb_stream stream) {
  if (!batch) return MMLTTB_EINVAL;
  if (!workspace || workspace_bytes < batch->impl.total) return MMLTTB_ENOSPC;
  BatchImpl& b = batch->impl;
  cudaError_t e;
  if (!b.exec || b.graph_ws != workspace) {
    if (b.exec) { cudaGraphExecDestroy(b.exec); b.exec = nullptr; }
    if (b.graph) { cudaGraphDestroy(b.graph); b.graph = nullptr; }
    if (!b.capture_stream &&
        (e = cudaStreamCreateWithFlags(&b.capture_stream, cudaStreamNonBlocking)) != cudaSuccess)
      return cuda_fail(e);
    if ((e = cudaStreamBeginCapture(b.capture_stream, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
      return cuda_fail(e);
    const unsigned long long before = g_launches;
    int rc = batch_enqueue(&b, workspace, b.capture_stream);
    g_launches = before;  // captured, not launched
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(b.capture_stream, &g);
    if (rc) {
      if (g) cudaGraphDestroy(g);
      return rc;
    }
    if (e != cudaSuccess) return cuda_fail(e);
    b.graph = g;
    if ((e = cudaGraphInstantiate(&b.exec, b.graph, 0)) != cudaSuccess) return cuda_fail(e);
    b.graph_ws = workspace;
    b.graph_launches = 0;
    for (auto k : {b.total_edges > 0, b.W > 0, b.W > 0 || b.total_bins > 0 || b.total_pos == 0,
                   b.total_slots > 0, true, b.any_block})
      b.graph_launches += k ? 1 : 0;
  }
  if ((e = cudaGraphLaunch(b.exec, (cudaStream_t)stream)) != cudaSuccess) return cuda_fail(e);
  g_launches += b.graph_launches;
  return MMLTTB_OK;
}

int mmlttb_batch_destroy(mmlttb_batch_t batch) {
  delete batch;
  return MMLTTB_OK;
}

int mmlttb_set_timing_events(void* start_event, void* stop_event) {
  g_ev_start = (cudaEvent_t)start_event;
  g_ev_stop = (cudaEvent_t)stop_event;
  return MMLTTB_OK;
}

unsigned long long mmlttb_launch_count(void) { return g_launches; }

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
// Some callers cannot allocate device memory at the moment they need a result: code
// that runs while a CUDA stream is being captured (cudaMalloc is not allowed there),
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
