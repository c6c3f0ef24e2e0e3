// Batches of series (host side): planning, workspace layout, upload and launch
// sequence, plus the mmlttb_batch_* C ABI and CUDA-graph capture.
#include <string.h>

#include <new>
#include <vector>

#include "host.h"

namespace mmlttb {

// ---------------------------------------------------------------- batches
// A batch plans many series once (host), lays them out in one caller-owned
// workspace, uploads the plan table with one copy from pinned host memory, and runs
// the same kernels as a single series over all of them: one MinMax stream over the
// concatenated interior points, one merge CTA per series, one table pass over all
// positions, one chain CTA per series.  The launch sequence can be captured into a
// CUDA graph once and replayed.

size_t batch_upload_bytes(int64_t n) {
  return align256((size_t)n * sizeof(SeriesPlan)) + 5 * align256((size_t)(n + 1) * 8);
}

int batch_plan(BatchImpl* b, const DevInfo& d, char* lend, size_t lend_bytes) {
  const int64_t n = b->n;
  b->plans.assign(n, SeriesPlan{});
  b->sel_off.assign(n, -1);
  b->tab_byte_off.assign(n, -1);
  b->mean_off.assign(n, -1);
  int64_t pos = 0, bins = 0, edges = 0, slots = 0, sel = 0, means = 0, ctas = 0, tcost = 0, tiles = 0;
  int64_t y_bytes = 0;  // the batch's y, which the stream reads about once
  for (int64_t s = 0; s < n; ++s)
    if (b->descs[s].n_in > 0) y_bytes += b->descs[s].n_in * (b->descs[s].ydtype == MMLTTB_F32 ? 4 : 8);
  const bool throughput = y_bytes >= kStreamThroughputBytes;
  const bool bulk_on = bulk_enabled();
  // the tuning of the key (y type, x kind, bin mode) that holds most binned points, its
  // size class from the batch's binned points
  int64_t key_pts[2][3][2] = {};
  int64_t binned_pts = 0;
  for (int64_t s = 0; s < n; ++s) {
    const mmlttb_series_desc& D = b->descs[s];
    int32_t br;
    int64_t B;
    const int bm = D.binmode & ~MMLTTB_NAN_AWARE;
    if (classify(D.op, D.ydtype, D.xkind, D.n_in, D.n_out, D.r_ps, D.binmode, &br, &B) || !binned(br)) continue;
    key_pts[D.ydtype][D.xkind][bm] += D.n_in;
    binned_pts += D.n_in;
  }
  int ky = MMLTTB_F32, kx = MMLTTB_X_IMPLICIT, kb = MMLTTB_BINS_INDEX;
  for (int a = 0; a < 2; ++a)
    for (int c = 0; c < 3; ++c)
      for (int e = 0; e < 2; ++e)
        if (key_pts[a][c][e] > key_pts[ky][kx][kb]) {
          ky = a;
          kx = c;
          kb = e;
        }
  const mmlttb_tuning tu = tuning_for(d, ky, kx, kb, binned_pts);
  b->tuning = tu;
  b->key_ydt = ky;
  b->key_xk = kx;
  b->key_bm = kb;
  b->key_n = binned_pts;
  for (int64_t s = 0; s < n; ++s) {
    const mmlttb_series_desc& D = b->descs[s];
    int32_t br;
    int64_t B;
    int rc = classify(D.op, D.ydtype, D.xkind, D.n_in, D.n_out, D.r_ps, D.binmode, &br, &B);
    if (rc) return rc;
    if (D.n_in > 0 && D.y == nullptr) return MMLTTB_EINVAL;
    if (D.xkind != MMLTTB_X_IMPLICIT && D.n_in > 0 && D.x == nullptr) return MMLTTB_EINVAL;
    const int64_t need = br == BR_PRESELECT ? (D.n_in < 2 * B + 2 ? D.n_in : 2 * B + 2)
                         : br == BR_M4      ? (D.n_in < 4 * B ? D.n_in : 4 * B)
                                            : (D.n_out < D.n_in ? D.n_out : D.n_in);
    if (need > 0 && D.out_idx == nullptr) return MMLTTB_EINVAL;
    if (D.out_cap < need) return MMLTTB_ERANGE;
    SeriesPlan& sp = b->plans[s];
    sp.y = D.y;
    sp.x = D.xkind == MMLTTB_X_IMPLICIT ? nullptr : D.x;
    sp.ydt = D.ydtype;
    sp.xk = D.xkind;
    sp.nan_aware = (D.binmode & MMLTTB_NAN_AWARE) ? 1 : 0;
    sp.binmode = D.binmode & ~MMLTTB_NAN_AWARE;
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
    const bool mm = binned(br);
    sp.bincta_off = ctas;
    sp.p0 = br == BR_M4 ? 0 : 1;
    sp.nb = br == BR_M4 ? D.n_in : (D.n_in > 2 ? D.n_in - 2 : 0);
    // x-width bins can be very uneven: keep whole warps per bin there
    const int eb = D.ydtype == MMLTTB_F32 ? 4 : 8;
    sp.group = sp.binmode == MMLTTB_BINS_XWIDTH ? 32 : shift_group(stream_group(sp.nb, B, eb, throughput), tu.group_shift);
    sp.tcost_off = tcost;
    if (mm && throughput && bulk_on && sp.binmode == MMLTTB_BINS_INDEX && D.ydtype == MMLTTB_F32)
      sp.bulk_bpt = bulk_bins_per_tile(sp.nb, B, eb);
    if (sp.bulk_bpt > 0) {  // the staged stream: no share of the register stream's work
      sp.group = bulk_group(sp.bulk_bpt);
      const int64_t nt = (B + sp.bulk_bpt - 1) / sp.bulk_bpt;
      sp.tcost = sp.bulk_bpt * (((sp.nb + B - 1) / B) * eb + kBulkBinCost);
      tcost += nt * sp.tcost;
      tiles += nt;
    }
    if (mm) {
      sp.npos = sp.bulk_bpt > 0 ? 0 : series_work(sp.nb, B, sp.group);
      pos += sp.npos;
      bins += B;
      ctas += (B + kBinsPerCta - 1) / kBinsPerCta;
      if (sp.binmode == MMLTTB_BINS_XWIDTH) edges += B + 1;
    }
    set_bin_steps(sp);
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
        // one table byte per position, 16-byte aligned and padded; the slots of
        // k_tables are these positions
        b->tab_byte_off[s] = slots;
        slots += (mcap + 15) & ~int64_t(15);
        if (mcap > b->max_tab) b->max_tab = mcap;
        int lgS = 0;
        while ((int64_t(1) << lgS) < max_bucket(mcap, K)) ++lgS;
        sp.tab_lgS = lgS;
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
  b->total_bin_ctas = ctas;
  b->variant = tu.variant;
  b->ymode = -1;  // the specialised stream kernel when every binned series shares one y mode
  for (int64_t s = 0; s < n; ++s) {
    const SeriesPlan& sp = b->plans[s];
    if (!binned(sp.branch)) continue;
    const int y = stream_ymode(sp.ydt, sp.nan_aware != 0);
    b->ymode = (b->ymode < 0 || b->ymode == y) ? y : 0;
  }
  if (b->ymode < 0) b->ymode = 0;
  b->Wcap = stream_warp_cap(d);
  b->W = stream_warps(d, b->variant, pos);
  if (b->W > 0 && pos / b->W >= (int64_t(1) << 30)) return MMLTTB_EINVAL;
  b->total_tcost = tcost;
  b->Wb = bulk_warps(d, tiles);
  for (int64_t s = 0; s < n; ++s)
    if (b->plans[s].bulk_bpt > 0) b->plans[s].rec_w = bulk_rec_w(b->plans[s].pos_off, pos, b->W);
  size_t off = kHeader;
  auto take = [&](size_t bytes) { size_t o = off; off = align256(off + bytes); return o; };
  b->off_plans = take((size_t)n * sizeof(SeriesPlan));
  b->off_pos = take((size_t)(n + 1) * 8);
  b->off_edge = take((size_t)(n + 1) * 8);
  b->off_tab = take((size_t)(n + 1) * 8);
  b->off_cta = take((size_t)(n + 1) * 8);
  b->off_tcost = take((size_t)(n + 1) * 8);
  b->upload_bytes = off - b->off_plans;
  b->off_m = take((size_t)n * 8);
  b->off_edges = take((size_t)edges * 8);
  b->off_rec = take((size_t)(bins + b->Wcap) * sizeof(Record));
  b->off_sel = take((size_t)sel * 8);
  b->off_px = take((size_t)sel * 8);
  b->off_py = take((size_t)sel * 8);
  b->off_binres = take((size_t)ctas * kBinsPerCta * 32);
  b->off_ctasum = take((size_t)ctas * 4);
  b->off_ctaser = take((size_t)ctas * 4);
  b->off_ctaoff = take((size_t)ctas * 8);
  b->off_tabs = take((size_t)slots);
  b->off_means = take((size_t)means * 8);
  b->total = off;
  if (lend && lend_bytes >= b->upload_bytes) {
    b->pinned = lend;
    b->own_pinned = false;
  } else {
    cudaError_t e = cudaHostAlloc((void**)&b->pinned, b->upload_bytes, cudaHostAllocDefault);
    if (e != cudaSuccess) return cuda_fail(e);
  }
  // the offset tables never depend on the workspace address
  int64_t* po = (int64_t*)(b->pinned + (b->off_pos - b->off_plans));
  int64_t* eo = (int64_t*)(b->pinned + (b->off_edge - b->off_plans));
  int64_t* to = (int64_t*)(b->pinned + (b->off_tab - b->off_plans));
  int64_t* co = (int64_t*)(b->pinned + (b->off_cta - b->off_plans));
  int64_t* ko = (int64_t*)(b->pinned + (b->off_tcost - b->off_plans));
  for (int64_t s = 0; s < n; ++s) {
    po[s] = b->plans[s].pos_off;
    eo[s] = b->plans[s].edge_off;
    to[s] = b->plans[s].tab_off;
    co[s] = b->plans[s].bincta_off;
    ko[s] = b->plans[s].tcost_off;
  }
  po[n] = pos;
  eo[n] = edges;
  to[n] = slots;
  co[n] = ctas;
  ko[n] = tcost;
  return MMLTTB_OK;
}

// Point every plan at its sections of workspace `ws` and refresh the upload image.
void batch_bind(BatchImpl* b, void* ws) {
  char* w = (char*)ws;
  for (int64_t s = 0; s < b->n; ++s) {
    SeriesPlan& sp = b->plans[s];
    sp.m_ptr = (int64_t*)(w + b->off_m) + s;
    sp.sel = (sp.branch == BR_PRESELECT || sp.branch == BR_M4) ? sp.out
             : sp.branch == BR_MINMAX_LTTB ? (int64_t*)(w + b->off_sel) + b->sel_off[s] : nullptr;
    sp.px = sp.branch == BR_MINMAX_LTTB ? (double*)(w + b->off_px) + b->sel_off[s] : nullptr;
    sp.py = sp.branch == BR_MINMAX_LTTB ? (double*)(w + b->off_py) + b->sel_off[s] : nullptr;
    sp.tab = sp.engine == EN_TABLES ? (uint8_t*)(w + b->off_tabs) + b->tab_byte_off[s] : nullptr;
    sp.means = sp.engine == EN_BLOCK ? (double*)(w + b->off_means) + b->mean_off[s] : nullptr;
  }
  memcpy(b->pinned, b->plans.data(), (size_t)b->n * sizeof(SeriesPlan));
  b->bound_ws = ws;
}

static Batch batch_args(const BatchImpl* b, void* ws) {
  char* w = (char*)ws;
  Batch bt;
  memset(&bt, 0, sizeof(bt));
  bt.plans = (const SeriesPlan*)(w + b->off_plans);
  bt.pos_offs = (const int64_t*)(w + b->off_pos);
  bt.edge_offs = (const int64_t*)(w + b->off_edge);
  bt.tab_offs = (const int64_t*)(w + b->off_tab);
  bt.cta_offs = (const int64_t*)(w + b->off_cta);
  bt.tcost_offs = (const int64_t*)(w + b->off_tcost);
  bt.tab_rounds_req = b->tuning.tab_rounds;
  bt.total_tcost = b->total_tcost;
  bt.n_bulk_warps = b->Wb;
  bt.total_bin_ctas = b->total_bin_ctas;
  bt.binres = (int64_t*)(w + b->off_binres);
  bt.cta_sum = (int32_t*)(w + b->off_ctasum);
  bt.cta_series = (int32_t*)(w + b->off_ctaser);
  bt.cta_off = (int64_t*)(w + b->off_ctaoff);
  bt.n_series = (int32_t)b->n;
  bt.total_pos = b->total_pos;
  bt.n_warps = b->W;
  set_warp_divs(bt);
  bt.total_edges = b->total_edges;
  bt.total_slots = b->total_slots;
  bt.rec = (Record*)(w + b->off_rec);
  bt.edges = (int64_t*)(w + b->off_edges);
  bt.status = (unsigned*)w;
  bt.barrier = (unsigned*)(w + 4);
  return bt;
}

// Enqueue the whole batch on `st`: upload, then the kernels (capturable).  An armed
// set of stage events (mmlttb_set_stage_events, uncaptured runs) is recorded at seven
// fixed points: after the upload, then after the edge search, the stream, the
// compaction, the tables, the chain and the block engine, whether or not each ran.
int batch_enqueue(BatchImpl* b, void* ws, cudaStream_t st) {
  struct StageReset {  // the stage events are one-shot: disarm when this call returns
    ~StageReset() { stage_disarm(); }
  } stage_reset;
  if (b->bound_ws != ws) batch_bind(b, ws);
  const Batch bt = batch_args(b, ws);
  cudaError_t e;
  if ((e = cudaMemsetAsync(ws, 0, kHeader, st)) != cudaSuccess) return cuda_fail(e);
  if ((e = cudaMemcpyAsync((char*)ws + b->off_plans, b->pinned, b->upload_bytes,
                           cudaMemcpyHostToDevice, st)) != cudaSuccess)
    return cuda_fail(e);
  stage_mark(st);
  const int nb = (int)b->n;
  if (bt.total_edges > 0) {
    if ((e = launch_edges(bt, st)) != cudaSuccess) return cuda_fail(e);
    ++g_launches;
  }
  stage_mark(st);
  if (b->W > 0) {
    if ((e = launch_stream(bt, b->variant, b->ymode, st)) != cudaSuccess) return cuda_fail(e);
    ++g_launches;
  }
  // the staged stream after the register stream: launched first, its resident CTAs
  // delayed part of the register stream's persistent grid (6.9 against 3.7 ms)
  if (b->Wb > 0) {
    if ((e = launch_stream_bulk(bt, b->ymode, st)) != cudaSuccess) return cuda_fail(e);
    ++g_launches;
  }
  stage_mark(st);
  if (b->total_bin_ctas > 0) {
    if ((e = launch_compact(bt, st)) != cudaSuccess) return cuda_fail(e);
    g_launches += 3;
  }
  stage_mark(st);
  if (bt.total_slots > 0) {
    if ((e = launch_tables(bt, st)) != cudaSuccess) return cuda_fail(e);
    ++g_launches;
  }
  stage_mark(st);
  if ((e = launch_chain(bt, nb, b->max_tab, st)) != cudaSuccess) return cuda_fail(e);
  ++g_launches;
  stage_mark(st);
  if (b->any_block) {
    if ((e = launch_lttb_block(bt, nb, st)) != cudaSuccess) return cuda_fail(e);
    ++g_launches;
  }
  stage_mark(st);
  return MMLTTB_OK;
}

}  // namespace mmlttb

using namespace mmlttb;

struct mmlttb_batch {
  BatchImpl impl;
};

extern "C" {

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

int mmlttb_batch_tuning(mmlttb_batch_t batch, mmlttb_tuning* tuning) {
  if (!batch || !tuning) return MMLTTB_EINVAL;
  *tuning = batch->impl.tuning;
  return MMLTTB_OK;
}

int mmlttb_batch_tuning_key(mmlttb_batch_t batch, int* ydtype, int* xkind, int* binmode, int64_t* n_in) {
  if (!batch || !ydtype || !xkind || !binmode || !n_in) return MMLTTB_EINVAL;
  *ydtype = batch->impl.key_ydt;
  *xkind = batch->impl.key_xk;
  *binmode = batch->impl.key_bm;
  *n_in = batch->impl.key_n;
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
    for (auto k : {b.total_edges > 0, b.W > 0, b.total_slots > 0, true, b.any_block})
      b.graph_launches += k ? 1 : 0;
    b.graph_launches += b.total_bin_ctas > 0 ? 3 : 0;
  }
  if ((e = cudaGraphLaunch(b.exec, (cudaStream_t)stream)) != cudaSuccess) return cuda_fail(e);
  g_launches += b.graph_launches;
  return MMLTTB_OK;
}

int mmlttb_batch_destroy(mmlttb_batch_t batch) {
  delete batch;
  return MMLTTB_OK;
}

}  // extern "C"
