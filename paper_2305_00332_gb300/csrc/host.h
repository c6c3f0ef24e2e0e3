// Host-side internals shared by the C ABI translation units (not part of the ABI).
#pragma once

#include <mutex>
#include <vector>

#include "common.cuh"

namespace mmlttb {

extern thread_local int g_last_cuda_error;
extern thread_local unsigned long long g_launches;  // kernels launched by this thread

// Record the next armed per-stage profiling event (if any) on `st`.
void stage_mark(cudaStream_t st);
// Disarm the per-stage profiling events (they are one-shot per call).
void stage_disarm();
// Remember `e` as the thread's last CUDA error and return MMLTTB_ECUDA.
int cuda_fail(cudaError_t e);

struct DevInfo {
  int device = 0;
  int sms = 0;
  int stream_bps[kStreamVariants] = {};  // resident stream CTAs per SM, per variant
  int fused_grid = 0;  // CTAs of the fused single-series kernel (0: unavailable)
  int bulk_bps = 1;    // resident staged-stream CTAs per SM
  bool ok = false;
};
// SM count and kernel occupancies of the current device (cached per device).
int get_dev_info(DevInfo* out);
// Stream variant used for y of type ydt on this device (tuned or default).
int stream_variant(const DevInfo& d, int ydt);
// The tuning of a key (mmlttb_tuning; the thread's override while tuning, else the
// stored one, else the default), the lanes-per-bin shift it applies, and the size
// class of n (its decimal digits less one, at most 12).
mmlttb_tuning tuning_for(const DevInfo& d, int ydt, int xk, int binmode, int64_t n);
int shift_group(int G, int shift);
int size_class(int64_t n);
// Most streaming warps any variant runs (sizes the record array).
int64_t stream_warp_cap(const DevInfo& d);
// Streaming warps of `variant` for `work` units: every warp gets at least one point.
int64_t stream_warps(const DevInfo& d, int variant, int64_t work);
// Warps of the staged stream for `tiles` tiles: one wave of resident CTAs at most.
int64_t bulk_warps(const DevInfo& d, int64_t tiles);
// Record slot offset of a staged series at pos_off of a register work space of
// `total` units split over W warps: the slots of its bins lie after those of every
// register-streamed series before it and before those of every one after it.
int64_t bulk_rec_w(int64_t pos_off, int64_t total, int64_t W);
// Whether the staged stream is enabled for new plans (mmlttb_set_stream_staging).
bool bulk_enabled();

// Failure-detection probes (a bounded wait that nothing satisfies; see mmlttb_diag.h).
cudaError_t launch_sync_probe(const Batch& bt, cudaStream_t st);     // fused.cu grid_sync
cudaError_t launch_barrier_probe(const Batch& bt, cudaStream_t st);  // lttb.cu grid_barrier
cudaError_t launch_mbarrier_probe(const Batch& bt, cudaStream_t st); // minmax.cu staged-stream wait

inline size_t align256(size_t v) { return (v + 255) & ~size_t(255); }
constexpr size_t kHeader = 256;  // workspace header: status word @0, barrier counter @4, m @8

// Largest LTTB bucket over m positions with K buckets: ceil((m-2)/K).
inline int64_t max_bucket(int64_t m, int64_t K) { return (m - 2 + K - 1) / K; }

// Host-only validation and branch choice (Sec. 3 dispatch); needs no device.
int classify(int op, int ydt, int xk, int64_t n, int64_t n_out, int32_t r_ps, int binmode,
             int32_t* branch, int64_t* bins);

struct BatchImpl {
  std::vector<mmlttb_series_desc> descs;
  std::vector<SeriesPlan> plans;  // pointer fields filled per workspace address
  int64_t n = 0;
  int64_t total_pos = 0, total_bins = 0, total_edges = 0, total_slots = 0;
  int64_t Wcap = 0, W = 0;
  int64_t total_tcost = 0, Wb = 0;  // staged stream: tile cost space and warps
  int variant = 0;
  mmlttb_tuning tuning = {0, 0, 0, 0};  // the tuning the batch was planned with
  int key_ydt = 0, key_xk = 0, key_bm = 0;  // its key: the (y type, x kind, bin mode) of most
  int64_t key_n = 0;                        // binned points, and those points
  int ymode = 0;  // stream-kernel y mode (stream_ymode) shared by every binned series, else 0
  bool any_block = false;
  int64_t max_tab = 0;  // largest per-series table storage (positions)
  int64_t total_bin_ctas = 0;
  size_t off_plans = 0, off_pos = 0, off_edge = 0, off_tab = 0, off_cta = 0, off_m = 0, off_edges = 0,
         off_rec = 0, off_sel = 0, off_px = 0, off_py = 0, off_tabs = 0, off_means = 0,
         off_binres = 0, off_ctasum = 0, off_ctaser = 0, off_ctaoff = 0, off_tcost = 0, total = kHeader,
         upload_bytes = 0;
  std::vector<int64_t> sel_off, tab_byte_off, mean_off;
  char* pinned = nullptr;  // upload image: plans | pos_offs | edge_offs | tab_offs | cta_offs | tcost_offs
  bool own_pinned = true;       // false: the image lives in a buffer lent by the caller
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
    if (pinned && own_pinned) cudaFreeHost(pinned);
  }
};

// Plan every series of b->descs (validation, branches, engines, workspace layout)
// and fill the offset tables of the upload image.  `lend`, when not NULL, is a
// pinned buffer of `lend_bytes` the image may use instead of its own allocation.
int batch_plan(BatchImpl* b, const DevInfo& d, char* lend = nullptr, size_t lend_bytes = 0);
// Bytes of the upload image batch_plan needs for n series.
size_t batch_upload_bytes(int64_t n);
// Point every plan at its sections of workspace `ws` and refresh the upload image.
void batch_bind(BatchImpl* b, void* ws);
// Enqueue the whole batch on `st`: header clear, upload, kernels (capturable).
int batch_enqueue(BatchImpl* b, void* ws, cudaStream_t st);

}  // namespace mmlttb
