// Compaction kernels (A-2) of MinMax preselection (Sec. 3), grid-wide: used for
// batches and for single series on the split launch path.
//
// Every series' bins are laid out from a CTA boundary (kBinsPerCta bins per CTA).
//   k_bins     one thread per bin: combine the bin's records (consecutive slots)
//              into (lower, higher) of argmin/argmax with their keys, -1 for an empty
//              bin; each CTA
//              writes how many indices its bins emit.
//   k_binscan  one warp per series: exclusive scan of the series' CTA totals; the
//              series' count m and the first and last entries of its list.
//   k_place    one thread per bin: block scan + CTA offset place the bin's indices
//              (and, before LTTB, their x and y as FP64, y from the record keys) in
//              the preselected list.
#include "compact.cuh"

namespace mmlttb {

namespace {

__global__ void __launch_bounds__(kBinsPerCta) k_bins(const __grid_constant__ Batch bt) {
  __shared__ int s_series;
  __shared__ int s_warp[kBinsPerCta / 32];
  pdl_wait();
  pdl_trigger();
  const int64_t c = blockIdx.x;
  if (threadIdx.x < 32) {  // the CTA's series: a 32-ary warp search (3 rounds for 4096 series)
    const int s = bt.cta_offs ? warp_upper_index(bt.cta_offs, bt.n_series, c, threadIdx.x) : 0;
    if (threadIdx.x == 0) s_series = s;
  }
  __syncthreads();
  const SeriesPlan& sp = plan_of(bt, s_series);
  const int64_t b = (c - sp.bincta_off) * kBinsPerCta + threadIdx.x;
  int64_t lo, hi, first, last;
  long long klo, khi;
  resolve_bin(bt, sp, b, &lo, &hi, &klo, &khi, &first, &last);
  const int64_t slot = c * kBinsPerCta + threadIdx.x;
  bt.binres[4 * slot] = lo;
  bt.binres[4 * slot + 1] = hi;
  bt.binres[4 * slot + 2] = klo;
  bt.binres[4 * slot + 3] = khi;
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

constexpr int kScanThreads = 256;

// One warp per series: exclusive scan of the series' CTA totals, 32 at a time with
// shuffles, then the series' count m and the ends of its list (finish_series).
__global__ void __launch_bounds__(kScanThreads) k_binscan(const __grid_constant__ Batch bt) {
  pdl_wait();
  pdl_trigger();
  const int lane = threadIdx.x & 31;
  const int64_t s = ((int64_t)blockIdx.x * kScanThreads + threadIdx.x) >> 5;
  if (s >= bt.n_series) return;
  const SeriesPlan& sp = plan_of(bt, (int)s);
  if (!binned(sp.branch)) return;
  const int64_t c0 = sp.bincta_off, c1 = c0 + (sp.B + kBinsPerCta - 1) / kBinsPerCta;
  int64_t carry = 0;
  for (int64_t c = c0; c < c1; c += 32) {
    const int64_t ci = c + lane;
    const int64_t v = ci < c1 ? (int64_t)bt.cta_sum[ci] : 0;
    int64_t inc = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const int64_t t = __shfl_up_sync(kFull, inc, d);
      if (lane >= d) inc += t;
    }
    if (ci < c1) bt.cta_off[ci] = carry + inc - v;
    carry += __shfl_sync(kFull, inc, 31);
  }
  if (lane == 0) finish_series(sp, carry);
}

__global__ void __launch_bounds__(kBinsPerCta) k_place(const __grid_constant__ Batch bt) {
  pdl_wait();
  pdl_trigger();
  const int64_t c = blockIdx.x;
  const int s = bt.cta_series[c];
  const SeriesPlan& sp = plan_of(bt, s);
  const int64_t slot = c * kBinsPerCta + threadIdx.x;
  const int64_t lo = bt.binres[4 * slot], hi = bt.binres[4 * slot + 1];
  const long long klo = bt.binres[4 * slot + 2], khi = bt.binres[4 * slot + 3];
  int64_t first = -1, last = -1;
  if (sp.branch == BR_M4 && lo >= 0) {
    const int64_t b = (c - sp.bincta_off) * kBinsPerCta + threadIdx.x;
    first = bin_start(bt, sp, b);
    last = ((b + 1 >= sp.B) ? sp.p0 + sp.nb : bin_start(bt, sp, b + 1)) - 1;
  }
  const int cnt = bin_count(sp, lo, hi, first, last);
  int excl;
  block_excl_scan<kBinsPerCta>(cnt, &excl);
  place_bin(sp, lo, hi, klo, khi, first, last, cnt, bt.cta_off[c] + excl);
}

}  // namespace

cudaError_t launch_compact(const Batch& bt, cudaStream_t st) {
  if (bt.total_bin_ctas <= 0) return cudaSuccess;
  const dim3 grid((unsigned)bt.total_bin_ctas);
  cudaError_t e = launch_pdl(k_bins, grid, dim3(kBinsPerCta), 0, st, bt);
  if (e != cudaSuccess) return e;
  const int64_t scan_ctas = ((int64_t)bt.n_series * 32 + kScanThreads - 1) / kScanThreads;
  e = launch_pdl(k_binscan, dim3((unsigned)scan_ctas), dim3(kScanThreads), 0, st, bt);
  if (e != cudaSuccess) return e;
  return launch_pdl(k_place, grid, dim3(kBinsPerCta), 0, st, bt);
}

}  // namespace mmlttb
