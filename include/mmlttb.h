/*
 * mmlttb.h -- C ABI of the GB300 (sm_103a) MinMaxLTTB library, libmmlttb.so.
 *
 * MinMaxLTTB (arXiv 2305.00332, Sec. 3) downsamples a time series of n_in points
 * to n_out indices in two steps: MinMax preselection keeps the argmin and argmax
 * of y in each of floor(n_out*r_ps/2) bins (plus the first and last point), then
 * LTTB (Sec. 2.2.1) picks one point per bucket among the preselected points.
 * Every result is a selection, returned as strictly increasing int64 indices into
 * the input series.
 *
 * Conventions shared by every entry point:
 *   - Pointers named y, x, out_idx, out_count and workspace are DEVICE pointers
 *     (or host memory the device can address); the caller allocates and owns them.
 *     Nothing is allocated or freed by these calls.
 *   - Calls are asynchronous on `stream` (a cudaStream_t; NULL = legacy default
 *     stream) unless stated otherwise.  Results are valid once the stream has
 *     reached the call.  Calls that overlap on the GPU must not share a workspace.
 *   - The return value is MMLTTB_OK (0) or a negative MMLTTB_E* code; argument
 *     errors are detected on the host before anything is enqueued.  No C++
 *     exception crosses this interface.
 *   - y is float32 or float64, contiguous.  x is implicit (the index 0..n_in-1),
 *     int64 or float64, contiguous, and non-decreasing (a precondition that is not
 *     checked).  y must contain no NaN (precondition, not checked).
 *   - Ties go to the lowest index; -0.0 and +0.0 are equal.  The LTTB areas and
 *     bucket means are computed in FP64 exactly as
 *       area = |(xa-xc)*(yb-ya) - (xa-xb)*(yc-ya)|   (each operation rounded on its own)
 *       mean = (((v0 + v1) + v2) + ...) / count       (left to right)
 *     so results are bit-identical to a sequential CPU statement of the method.
 */
#ifndef MMLTTB_H
#define MMLTTB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Return codes. */
#define MMLTTB_OK 0
#define MMLTTB_EINVAL (-1)   /* invalid argument (null pointer, size, enum, r_ps, n_out) */
#define MMLTTB_ENOSPC (-2)   /* workspace smaller than the size query returned */
#define MMLTTB_ECUDA (-3)    /* a CUDA runtime call or kernel launch failed */
#define MMLTTB_ETIMEOUT (-4) /* a bounded device-side wait gave up (status word) */
#define MMLTTB_ERANGE (-6)   /* output capacity too small */
#define MMLTTB_EDEVICE (-7)  /* a device-side check failed (status word) */
#define MMLTTB_ENOMEM (-8)   /* host memory for a batch object could not be allocated */
#define MMLTTB_ESCRATCH (-9) /* sizes need more than the static scratch of mmlttb_minmaxlttb_noalloc */
#define MMLTTB_EBUSY (-10)   /* server queue full: resubmit later */

/* Element type of y. */
#define MMLTTB_F32 0
#define MMLTTB_F64 1

/* Kind of x. */
#define MMLTTB_X_IMPLICIT 0 /* x = index; the x pointer is ignored (may be NULL) */
#define MMLTTB_X_I64 1      /* int64, non-decreasing */
#define MMLTTB_X_F64 2      /* float64, non-decreasing, finite */

/* How MinMax bins partition the interior points 1..n_in-2. */
#define MMLTTB_BINS_INDEX 0  /* equal count: bin i = [floor(i(n-2)/B)+1, floor((i+1)(n-2)/B)+1) */
#define MMLTTB_BINS_XWIDTH 1 /* equal x width: edges e_i = x0 + floor(i(x_{n-1}-x0)/B) for int64 x,
                                e_i = x0 + (i*(x_{n-1}-x0))/B in FP64 (each operation rounded) for
                                float64 x; point p is in the largest bin i with e_i <= x_p;
                                empty bins emit nothing */

/* Flag OR-ed into binmode of mmlttb_minmax_preselect and mmlttb_m4 (only): NaN-aware
   bins.  A bin holding a NaN reports its first NaN as both argmin and argmax (the
   convention of numpy's argmin/argmax), so a plot of the selection shows the gap. */
#define MMLTTB_NAN_AWARE 0x10

/* Operation selector for mmlttb_workspace_bytes. */
#define MMLTTB_OP_PRESELECT 0
#define MMLTTB_OP_LTTB 1
#define MMLTTB_OP_MINMAXLTTB 2
#define MMLTTB_OP_M4 3

/* Opaque CUDA stream handle; binary-compatible with cudaStream_t. */
typedef struct CUstream_st *mmlttb_stream;

/* Library infrastructure (no counterpart in the paper): return-code text, the last
   CUDA error and the version. */
/* Human-readable text for a return code; never NULL, static storage. */
const char *mmlttb_strerror(int code);

/* The cudaError_t value of the most recent MMLTTB_ECUDA on the calling thread. */
int mmlttb_last_cuda_error(void);

/* Library version as MAJOR*10000 + MINOR*100 + PATCH. */
int mmlttb_version(void);

/*
 * Workspace size (bytes, on the current device) needed by `op` for these sizes (no
 * counterpart in the paper: the caller-owned scratch of the operations below).
 * Writes the size to *bytes.  The size depends only on the arguments and on the
 * current device's SM count.  Returns MMLTTB_OK or MMLTTB_EINVAL.
 */
int mmlttb_workspace_bytes(int op, int ydtype, int xkind, int64_t n_in, int64_t n_out,
                           int32_t r_ps, int binmode, size_t *bytes);

/*
 * MinMax preselection (Sec. 3, first step; MinMax of Sec. 2.2.1 and Table 1).
 * B = floor(n_out*r_ps/2) bins (r_ps >= 1, B >= 1) over the interior points
 * 1..n_in-2.  Writes point 0, then per non-empty bin its argmin and argmax of y in
 * increasing index order (once when they coincide), then point n_in-1: at most
 * 2B+2 strictly increasing indices.
 *   out_idx   device int64[out_cap]; out_cap must be >= min(n_in, 2B+2), else MMLTTB_ERANGE.
 *   out_count device int64 (nullable): receives the number of indices written.
 *   workspace device memory of at least mmlttb_workspace_bytes(MMLTTB_OP_PRESELECT, ...) bytes.
 */
int mmlttb_minmax_preselect(const void *y, int ydtype, const void *x, int xkind, int64_t n_in,
                            int64_t n_out, int32_t r_ps, int binmode, int64_t *out_idx,
                            int64_t out_cap, int64_t *out_count, void *workspace,
                            size_t workspace_bytes, mmlttb_stream stream);

/*
 * M4 (Sec. 2.2.1 and Table 1: per bin the vertical extrema and the first and last
 * point).  B = floor(n_out/4) bins (n_out >= 4) over ALL points 0..n_in-1: index
 * bins [floor(i n/B), floor((i+1) n/B)), or equal-width x bins as for MinMax.  Per
 * non-empty bin, its first point, first argmin, first argmax and last point, in
 * increasing order without repeats: at most 4B indices.
 *   out_idx   device int64[out_cap], out_cap >= min(n_in, 4B).
 *   out_count device int64 (nullable): receives the number of indices written.
 *   workspace at least mmlttb_workspace_bytes(MMLTTB_OP_M4, ...) bytes.
 */
int mmlttb_m4(const void *y, int ydtype, const void *x, int xkind, int64_t n_in, int64_t n_out,
              int binmode, int64_t *out_idx, int64_t out_cap, int64_t *out_count, void *workspace,
              size_t workspace_bytes, mmlttb_stream stream);

/*
 * LTTB (Largest-Triangle-Three-Buckets; Sec. 2.2.1 and Table 1 of the paper, after
 * Steinarsson's thesis) on all n_in points.  n_out >= n_in returns 0..n_in-1;
 * otherwise n_out >= 3 is required: first and last point are kept and each of the
 * n_out-2 buckets [floor(j(n-2)/K)+1, floor((j+1)(n-2)/K)+1) contributes the point
 * with the largest triangle area against the previous pick and the mean of the next
 * bucket (the last bucket's next bucket is the last point).
 *   out_idx   device int64[out_cap], out_cap >= min(n_out, n_in).
 *   out_count device int64 (nullable): receives min(n_out, n_in).
 */
int mmlttb_lttb(const void *y, int ydtype, const void *x, int xkind, int64_t n_in,
                int64_t n_out, int64_t *out_idx, int64_t out_cap, int64_t *out_count,
                void *workspace, size_t workspace_bytes, mmlttb_stream stream);

/*
 * MinMaxLTTB (Sec. 3): n_out >= n_in returns every index; n_out < 3 or r_ps < 2 is
 * MMLTTB_EINVAL; r_ps*n_out >= n_in runs LTTB on all points; otherwise MinMax
 * preselection (as mmlttb_minmax_preselect) followed by LTTB on the preselected
 * points, buckets formed over positions in the preselected list and areas/means
 * taken from the original x and y.  When fewer than n_out points are preselected
 * (possible with x-width bins) all of them are returned.
 *   out_idx   device int64[out_cap], out_cap >= min(n_out, n_in).
 *   out_count device int64 (nullable): number of indices written (min(n_out, n_in)
 *             with index bins).
 */
int mmlttb_minmaxlttb(const void *y, int ydtype, const void *x, int xkind, int64_t n_in,
                      int64_t n_out, int32_t r_ps, int binmode, int64_t *out_idx,
                      int64_t out_cap, int64_t *out_count, void *workspace,
                      size_t workspace_bytes, mmlttb_stream stream);

/*
 * MinMaxLTTB without a workspace argument and without any allocation.  The paper
 * has no counterpart: this entry point exists for callers that cannot allocate
 * device memory when they need a result -- latency-critical loops that forbid
 * cudaMalloc/cudaFree because those can synchronize the whole device and stall
 * unrelated streams, and plugin hosts (a database function, a chart-server
 * extension) that offer no allocator.  Same arguments, semantics and results as
 * mmlttb_minmaxlttb, minus the workspace pair; the caller still provides the
 * inputs and out_idx/out_count.
 *   Scratch: a 4 MiB array compiled into the library (a static __device__
 *   variable), so every GPU that loads the library holds those 4 MiB until the
 *   process exits.  Sizes whose workspace (mmlttb_workspace_bytes) exceeds 4 MiB
 *   return MMLTTB_ESCRATCH and enqueue nothing; about 34 000 MinMax bins
 *   (n_out * r_ps / 2) fit.
 *   Set-up: the first call on each device looks up the array's device address
 *   (cudaGetSymbolAddress, with that device current) and caches it; make that first
 *   call before any stream capture begins.
 *   Sharing: every call on a device uses the same array and leaves its contents
 *   behind; each call clears what must start at zero.  Calls whose work overlaps on
 *   the GPU (different streams, or different host threads) race on the array and
 *   must be serialized by the caller.
 *   Status: the status word (bounded-wait timeouts, device checks) lives in the
 *   array too; read it with mmlttb_noalloc_status.
 */
int mmlttb_minmaxlttb_noalloc(const void *y, int ydtype, const void *x, int xkind, int64_t n_in,
                              int64_t n_out, int32_t r_ps, int binmode, int64_t *out_idx,
                              int64_t out_cap, int64_t *out_count, mmlttb_stream stream);

/*
 * Status word of the most recent mmlttb_minmaxlttb_noalloc call on the current
 * device (no counterpart in the paper).  The caller cannot address that entry
 * point's scratch, so this reads the word for it: the same bits as
 * mmlttb_workspace_status (0 = fine, 1 = a bounded device wait timed out and the
 * indices are not valid, 2 = a device check failed).  It waits for `stream` (pass
 * the stream of the call to check) and copies 4 bytes to the host; it allocates
 * nothing.  The next mmlttb_minmaxlttb_noalloc call on the device clears the word.
 * Before the first such call on the device it reports 0.  Returns MMLTTB_OK,
 * MMLTTB_EINVAL (status NULL) or MMLTTB_ECUDA.
 */
int mmlttb_noalloc_status(int *status, mmlttb_stream stream);

/*
 * MinMaxLTTB (Sec. 3) on HOST buffers, end to end (blocking): the setting of series
 * of billions of points held outside the accelerator (Sec. 1).  Pinned or registered host
 * memory (cudaHostAlloc / cudaHostRegister) is read in place by the kernels over
 * the CPU-GPU link, so only what the path touches crosses it: every y value once,
 * x only at the bin-edge probes and the preselected points.  This also serves
 * series larger than device memory.  Pageable host memory is first copied into
 * `device_buffer`.  The indices and the count are copied back to out_host /
 * out_count_host and `stream` is synchronized before returning.
 *   device_buffer  device memory owned by the caller, holding the output, the
 *                  workspace and, for pageable inputs, the staged series: at least
 *                  mmlttb_host_buffer_bytes(...) bytes, or, when y (and x) are
 *                  pinned or registered, mmlttb_host_buffer_bytes_inplace(...) bytes,
 *                  which do not grow with the series beyond its workspace (records
 *                  per bin and warp, LTTB tables).  A smaller buffer: MMLTTB_ENOSPC.
 *   out_host       host int64[out_cap], out_cap >= min(n_out, n_in).
 *   out_count_host host int64 (nullable).
 */
int mmlttb_host_buffer_bytes(int ydtype, int xkind, int64_t n_in, int64_t n_out, int32_t r_ps,
                             int binmode, size_t *bytes);
int mmlttb_host_buffer_bytes_inplace(int ydtype, int xkind, int64_t n_in, int64_t n_out, int32_t r_ps,
                                     int binmode, size_t *bytes);
int mmlttb_minmaxlttb_host(const void *y_host, int ydtype, const void *x_host, int xkind,
                           int64_t n_in, int64_t n_out, int32_t r_ps, int binmode,
                           int64_t *out_host, int64_t out_cap, int64_t *out_count_host,
                           void *device_buffer, size_t device_bytes, mmlttb_stream stream);

/*
 * Batches (many series in one launch sequence; the paper treats one series at a
 * time, batching is this library's).  Each series is described by a
 * mmlttb_series_desc; its op selects MinMaxLTTB (Sec. 3), plain LTTB (Sec. 2.2.1),
 * M4 (Sec. 2.2.1, Table 1) or preselection only (Sec. 3),
 * with the same semantics and argument rules as the single-series entry points.
 * All series run in one sequence of kernels: one MinMax stream over the interior
 * points of every series (cut into equal slices, one per warp, whatever the series
 * lengths), then per-series compaction, LTTB tables and chains.  The batch object
 * owns a pinned host copy of its plan table (allocated by mmlttb_batch_create,
 * freed by mmlttb_batch_destroy); device memory is the caller's workspace.
 */
typedef struct mmlttb_series_desc {
  const void *y;      /* device: n_in float32/float64 values */
  const void *x;      /* device: n_in int64/float64 values, or NULL with MMLTTB_X_IMPLICIT */
  int32_t op;         /* MMLTTB_OP_MINMAXLTTB, MMLTTB_OP_LTTB, MMLTTB_OP_PRESELECT or MMLTTB_OP_M4 */
  int32_t ydtype;     /* MMLTTB_F32 / MMLTTB_F64 */
  int32_t xkind;      /* MMLTTB_X_* */
  int32_t binmode;    /* MMLTTB_BINS_* */
  int32_t r_ps;
  int32_t reserved;   /* set to 0 */
  int64_t n_in, n_out;
  int64_t *out_idx;   /* device int64[out_cap] */
  int64_t out_cap;
  int64_t *out_count; /* device int64, nullable */
} mmlttb_series_desc;

typedef struct mmlttb_batch *mmlttb_batch_t;

/* Validate and plan n_series series (host side; reads only the descriptors).
   Returns MMLTTB_EINVAL / MMLTTB_ERANGE for the first invalid series. */
int mmlttb_batch_create(const mmlttb_series_desc *descs, int64_t n_series, mmlttb_batch_t *out);
/* Workspace bytes the batch needs (on the device current at creation). */
int mmlttb_batch_workspace_bytes(mmlttb_batch_t batch, size_t *bytes);
/* Enqueue the batch on `stream` (asynchronous; capturable into a CUDA graph). */
int mmlttb_batch_run(mmlttb_batch_t batch, void *workspace, size_t workspace_bytes,
                     mmlttb_stream stream);
/* Same work through a CUDA graph captured on the first call (per workspace address)
   and replayed afterwards: one graph launch instead of about six API calls. */
int mmlttb_batch_run_graph(mmlttb_batch_t batch, void *workspace, size_t workspace_bytes,
                           mmlttb_stream stream);
/* Release the batch (its graph and pinned plan table).  No call may be in flight. */
int mmlttb_batch_destroy(mmlttb_batch_t batch);

/*
 * Zoom-window server (continuous batching).  A visualisation front end asks for
 * MinMaxLTTB of windows [start, end) of series that stay resident on the device
 * (the interactive zoom/pan use case of Sec. 1 and Sec. 2.1).  Requests are queued;
 * a scheduler thread owned by the server forms batches first come, first served
 * whenever one of `streams` slots is free, admitting requests while the batch's
 * workspace fits the slot's budget, and runs each batch as one batched launch
 * sequence on the slot's stream.  Requests that arrive while batches are on the
 * GPU join the next batch, so batches overlap on the device.  Results are the
 * same as a single mmlttb_minmaxlttb call on the window (indices are absolute in
 * the resident series).  Device memory comes from a caller-owned pool; the server
 * allocates pinned host buffers for results and plan uploads.
 */
typedef struct mmlttb_server_config {
  int32_t streams;                    /* batches in flight at once (>= 1), one stream each */
  int32_t reserved;                   /* set to 0 */
  int64_t max_batch;                  /* requests per batch at most */
  int64_t max_n_out;                  /* largest n_out a request may ask for */
  int64_t max_pending;                /* queue capacity; beyond it submit returns MMLTTB_EBUSY */
  int64_t workspace_bytes_per_stream; /* device workspace per batch: the admission budget */
} mmlttb_server_config;

typedef struct mmlttb_request {
  int64_t series;     /* id returned by mmlttb_server_add_series */
  int64_t start, end; /* window [start, end) of the resident series, 0 <= start < end <= n */
  int64_t n_out;      /* 3 <= n_out <= max_n_out */
  int32_t r_ps;       /* >= 2 */
  int32_t binmode;    /* MMLTTB_BINS_* */
} mmlttb_request;

typedef struct mmlttb_server_stats {
  int64_t submitted, completed, rejected, batches, gpu_launches;
  double mean_batch;
  double latency_p50_s, latency_p99_s, latency_max_s, latency_mean_s;
  /* continuous batching: batches launched while at least one other batch of this
     server was still in flight (enqueued and not yet completed on the device), and
     the most batches in flight at once */
  int64_t overlapped_batches, max_batches_in_flight;
} mmlttb_server_stats;

typedef struct mmlttb_server *mmlttb_server_t;

/* Device pool bytes a configuration needs (workspace, outputs and counts per stream). */
int mmlttb_server_pool_bytes(const mmlttb_server_config *cfg, size_t *bytes);
/* Start a server on the current device over a caller-owned device pool. */
int mmlttb_server_create(const mmlttb_server_config *cfg, void *device_pool, size_t pool_bytes,
                         mmlttb_server_t *out);
/* Register a resident series (device pointers, owned by the caller, kept valid
   until the server is destroyed). */
int mmlttb_server_add_series(mmlttb_server_t server, const void *y, int ydtype, const void *x,
                             int xkind, int64_t n, int64_t *series_id);
/* Queue a request (thread-safe, returns at once).  MMLTTB_EINVAL for a malformed
   request, MMLTTB_ENOSPC when it cannot fit a slot's workspace even alone,
   MMLTTB_EBUSY when the queue is full. */
int mmlttb_server_submit(mmlttb_server_t server, const mmlttb_request *req, uint64_t *request_id);
/* Block until the request completes; copy its indices (host int64[out_cap]) and
   release it.  latency_s (nullable) receives completion minus submission time. */
int mmlttb_server_wait(mmlttb_server_t server, uint64_t request_id, int64_t *out_host,
                       int64_t out_cap, int64_t *count, double *latency_s);
/* Block until every submitted request has completed. */
int mmlttb_server_drain(mmlttb_server_t server);
/* Trace replay: submit reqs[i] at t_offset_s[i] seconds after the call starts
   (offsets non-decreasing); ids[i] receives the id (0 when rejected) and status[i]
   (nullable) the submit result.  Returns after the last submission. */
int mmlttb_server_replay(mmlttb_server_t server, const mmlttb_request *reqs,
                         const double *t_offset_s, int64_t n, uint64_t *ids, int *status);
int mmlttb_server_get_stats(mmlttb_server_t server, mmlttb_server_stats *stats);
int mmlttb_server_reset_stats(mmlttb_server_t server);
/* Finish queued work, stop the scheduler and release the server's host buffers. */
int mmlttb_server_destroy(mmlttb_server_t server);

/*
 * Measurement support (no counterpart in the paper).
 * Profiling hook (per calling thread, one shot): the next call that runs MinMax
 * preselection records `start_event` on its stream just before the streaming
 * MinMax kernel and `stop_event` just after it, then forgets both.  The events
 * are cudaEvent_t handles created by the caller (NULL, NULL disarms).  The time
 * between them is that kernel's device time.
 */
int mmlttb_set_timing_events(void *start_event, void *stop_event);

/*
 * Profiling hook (per calling thread, one shot): the next single-series call
 * records events[0] on its stream before its first kernel and events[k] after its
 * k-th launch step, for as many events as given (at most 16), then forgets them.
 * For MinMaxLTTB with x-width bins the steps are, on the split path: edge search,
 * MinMax stream, compaction, LTTB tables, LTTB chain; on the fused-tail path: edge
 * search, MinMax stream, fused tail; on the fused path: the one fused kernel.
 * An uncaptured batch run (mmlttb_batch_run) records seven events at fixed points:
 * after the header clear and upload, then after the edge search, the MinMax
 * stream, the compaction, the LTTB tables, the LTTB chain and the one-CTA-per-series
 * LTTB, whether or not each of these kernels ran for that batch.
 */
int mmlttb_set_stage_events(void *const *events, int count);

/*
 * Autotuning (no counterpart in the paper, which fixes results, not launches; every
 * tuning returns the same indices).  A tuning is the tuple
 *   variant      the streaming MinMax kernel: 16-byte loads in flight per lane, resident
 *                CTAs per SM and threads per CTA (mmlttb_stream_variant_info,
 *                mmlttb_stream_variant_threads), 0 .. MMLTTB_STREAM_VARIANTS - 1;
 *   group_shift  lanes per index bin of the register stream: the size-based choice
 *                doubled (+1), kept (0) or halved (-1), within 1 .. 32;
 *   tab_rounds   rounds of 32 table slots per warp of k_tables, 1 .. 7 (0: chosen from
 *                the slot count).
 * Tunings are kept per process under a key: the current device, the y type, the x
 * kind, the bin mode and the size class (the decimal digits of n_in less one, at most
 * 12).  Single-series calls use the tuning of their key; a batch, the one of the key
 * that holds most of its binned points, its size class from its total points
 * (mmlttb_batch_tuning reports it, mmlttb_batch_tuning_key that key with the batch's
 * binned points as n_in).  Keys never set use the default {0 or the variant
 * set for the y type by mmlttb_set_stream_variant, 0, 0}.
 * mmlttb_autotune_tuple times, blocking, every variant x group_shift on MinMax
 * preselection of the caller's series (device y and, for int64/float64 x, x; n_in,
 * n_out, r_ps, bin mode as given; workspace as for mmlttb_minmaxlttb, which must also
 * fit out_idx's needs), then tab_rounds in {0, 2, 4, 7} on MinMaxLTTB of it, stores
 * the fastest tuple under the series' key and returns it (*best_ms: the median stream
 * kernel time of the chosen variant).  mmlttb_autotune is the older entry point: it
 * tunes the variant alone for implicit x and index bins and also makes it the
 * variant of that y type.  set/get let a caller persist and restore tunings.
 * MMLTTB_EINVAL for a NULL pointer, an unknown type or kind, or a field out of range.
 */
#define MMLTTB_STREAM_VARIANTS 6
typedef struct mmlttb_tuning {
  int32_t variant;
  int32_t group_shift;
  int32_t tab_rounds;
  int32_t reserved; /* 0 */
} mmlttb_tuning;
int mmlttb_stream_variant_info(int variant, int *unroll, int *min_blocks);
int mmlttb_stream_variant_threads(int variant, int *threads);
int mmlttb_autotune(int ydtype, const void *y, int64_t n_in, int64_t n_out, int32_t r_ps,
                    int64_t *out_idx, int64_t out_cap, void *workspace, size_t workspace_bytes,
                    mmlttb_stream stream, int *best_variant, float *best_ms);
int mmlttb_autotune_tuple(int ydtype, const void *y, int xkind, const void *x, int64_t n_in, int64_t n_out,
                          int32_t r_ps, int binmode, int64_t *out_idx, int64_t out_cap, void *workspace,
                          size_t workspace_bytes, mmlttb_stream stream, mmlttb_tuning *best, float *best_ms);
int mmlttb_set_tuning(int ydtype, int xkind, int binmode, int64_t n_in, const mmlttb_tuning *tuning);
int mmlttb_get_tuning(int ydtype, int xkind, int binmode, int64_t n_in, mmlttb_tuning *tuning);
int mmlttb_clear_tunings(void);
int mmlttb_batch_tuning(mmlttb_batch_t batch, mmlttb_tuning *tuning);
int mmlttb_batch_tuning_key(mmlttb_batch_t batch, int *ydtype, int *xkind, int *binmode, int64_t *n_in);
int mmlttb_get_stream_variant(int ydtype, int *variant);
int mmlttb_set_stream_variant(int ydtype, int variant);

/*
 * Staged MinMax stream (no counterpart in the paper; results are the same either way).
 * With staging on, index bins of at most 512 bytes of float32 y (128 points) in
 * launches that stream at least 64 MiB are read by k_stream_bulk: each warp copies
 * tiles of whole bins (8 KiB) into shared memory with cp.async.bulk behind an mbarrier
 * pipeline and reduces them there; other bins take the register stream (16-byte loads
 * into registers).  Staging is off by default: on 1e8 float32 points it runs from
 * 0.96x to 1.25x the register stream at 16- to 128-point bins and slower above, and
 * the 4096-series batch replays 2% slower with it.  mmlttb_set_stream_staging(1)
 * turns it on for plans made afterwards (0 turns it off); process-wide.
 * MMLTTB_EINVAL for another value or a NULL pointer.
 */
int mmlttb_set_stream_staging(int enable);
int mmlttb_get_stream_staging(int *enable);
/* Bins per staged tile of a single-series call with these arguments on the current
 * device (*bins_per_tile = 0: the register stream), or a negative error code. */
int mmlttb_stream_tiles(int op, int ydtype, int xkind, int64_t n_in, int64_t n_out, int32_t r_ps, int binmode,
                       int64_t *bins_per_tile);

/* Number of kernels this library has launched from the calling thread so far. */
unsigned long long mmlttb_launch_count(void);

/*
 * Launch paths of the single-series calls (no counterpart in the paper, which
 * specifies results, not launches; every path returns the same result).
 *   MMLTTB_PATH_SPLIT       one grid-wide kernel per step: edge search, MinMax
 *                           stream, compaction (3 kernels), LTTB tables, LTTB chain.
 *   MMLTTB_PATH_FUSED_TAIL  edge search and MinMax stream as their own kernels, then
 *                           ONE persistent kernel (one CTA per SM, cooperative
 *                           launch) for compaction, tables and chain, with grid-wide
 *                           barriers between the steps.
 *   MMLTTB_PATH_FUSED       the whole call as that one persistent kernel (edge
 *                           search and stream included): the lowest latency for
 *                           small n.
 * The barriers wait at most 2 s (then status bit 1, see mmlttb_workspace_status).
 * AUTO picks FUSED for y of at most 8 MiB, FUSED_TAIL above, and SPLIT where the
 * fused kernel does not apply (LTTB buckets above 32 points, more than 262144 bins
 * or 1048576 table positions, or a device where its CTA does not fit).
 * mmlttb_set_single_path sets a preference for the calling thread (a forced fused
 * path still falls back to SPLIT where it does not apply); MMLTTB_EINVAL for an
 * unknown value.  mmlttb_single_path returns the path a call with these arguments
 * takes on the current device (>= 0), or a negative error code.
 */
#define MMLTTB_PATH_AUTO 0
#define MMLTTB_PATH_SPLIT 1
#define MMLTTB_PATH_FUSED_TAIL 2
#define MMLTTB_PATH_FUSED 3
int mmlttb_set_single_path(int path);
int mmlttb_single_path(int op, int ydtype, int xkind, int64_t n_in, int64_t n_out, int32_t r_ps,
                       int binmode);

/*
 * Read the workspace's status word (blocking: synchronizes `stream`).  *status
 * receives 0 when no device-side wait timed out and no device check failed since
 * the workspace was last cleared; otherwise a bitmask (1 = a bounded wait timed
 * out, 2 = a device check failed).  Returns MMLTTB_OK, or MMLTTB_ECUDA.
 */
int mmlttb_workspace_status(const void *workspace, int *status, mmlttb_stream stream);

#ifdef __cplusplus
}
#endif

#endif /* MMLTTB_H */
