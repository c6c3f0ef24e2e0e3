// Compaction kernels (A-2) of MinMax preselection (Sec. 3), grid-wide: used for
// batches and for single series on the split launch path.
//
// Every series' bins are laid out from a CTA boundary (kBinsPerCta bins per CTA).
//   k_bins     one thread per bin: combine the bin's records (consecutive slots)
//              into (lower, higher) of argmin/argmax, -1 for an empty bin; each CTA
//              writes how many indices its bins emit.
//   k_binscan  one CTA: exclusive scan of the CTA totals, restarted at every
//              series; the last CTA of a series fixes its count m and the first
//              and last entries of its preselected list.
//   k_place    one thread per bin: block scan + CTA offset place the bin's indices
//              (and, before LTTB, their x and y as FP64) in the preselected list.
#include "compact.cuh"

namespace mmlttb {

namespace {

__global__ void __launch_bounds__(kBinsPerCta) k_bins(const __grid_constant__ Batch bt) {
  __shared__ int s_series;
  __shared__ int s_warp[kBinsPerCta / 32];
  pdl_wait();
  pdl_trigger();
  const int64_t c = blockIdx.x;
  if (threadIdx.x == 0) s_series = bt.cta_offs ? upper_index(bt.cta_offs, bt.n_series, c) : 0;
  __syncthreads();
  const SeriesPlan& sp = plan_of(bt, s_series);
  const int64_t b = (c - sp.bincta_off) * kBinsPerCta + threadIdx.x;
  int64_t lo, hi, first, last;
  resolve_bin(bt, sp, b, &lo, &hi, &first, &last);
  const int64_t slot = c * kBinsPerCta + threadIdx.x;
  bt.binres[2 * slot] = lo;
  bt.binres[2 * slot + 1] = hi;
  int cnt = bin_count(sp, lo, hi, first, last);
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) cnt += __shfl_xor_sync(kFull, cnt, d);
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
  int64_t first = -1, last = -1;
  if (sp.branch == BR_M4 && lo >= 0) {
    const int64_t b = (c - sp.bincta_off) * kBinsPerCta + threadIdx.x;
    first = bin_start(bt, sp, b);
    last = ((b + 1 >= sp.B) ? sp.p0 + sp.nb : bin_start(bt, sp, b + 1)) - 1;
  }
  const int cnt = bin_count(sp, lo, hi, first, last);
  int excl;
  block_excl_scan<kBinsPerCta>(cnt, &excl);
  place_bin(sp, lo, hi, first, last, cnt, bt.cta_off[c] + excl);
}

}  // namespace

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
