// LTTB stage kernels (Sec. 2.2.1 LTTB; Sec. 3 second step of MinMaxLTTB).
//
// Small buckets (lttb.cuh): k_tables fills one transition-table entry per position,
// k_chain resolves the chain by a parallel prefix over function composition.
// Large buckets of a single series use lttb_big.cu; in a batch, k_lttb_block runs one
// CTA per series.
#include "lttb.cuh"

namespace mmlttb {

namespace {

constexpr int kChainThreads = 512;
constexpr int64_t kChainSmemMax = 160 * 1024;  // tables staged in shared memory up to this size
constexpr int kTableThreads = 64;  // small CTAs: the positions spread over every SM

// A warp per kTableBlock consecutive table slots (one slot per position); the warp
// finds the series of its first slot with a 32-ary search.
__global__ void __launch_bounds__(kTableThreads) k_tables(const __grid_constant__ Batch bt) {
  __shared__ TableShared s_tab[kTableThreads / 32];
  pdl_wait();
  pdl_trigger();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int rounds = bt.tab_rounds;
  const int64_t base = ((int64_t)blockIdx.x * (kTableThreads / 32) + wid) * 32 * rounds;
  if (base >= bt.total_slots) return;
  const int s0 = bt.tab_offs ? warp_upper_index(bt.tab_offs, bt.n_series, base, lane) : 0;
  table_block(bt, base, rounds, s0, lane, s_tab[wid]);
}

__global__ void __launch_bounds__(kChainThreads) k_chain(const __grid_constant__ Batch bt) {
  // F[c][ia][t]: thread t's map, entry ia (entry-major, so a warp touches 32
  // consecutive bytes per entry instead of 32 bytes apart)
  __shared__ uint8_t F[2][kTableMaxBucket][kChainThreads];
  __shared__ uint8_t dom[2][kChainThreads];
  extern __shared__ uint4 s_tab4[];
  pdl_wait();
  pdl_trigger();
  chain_series<kChainThreads>(plan_of(bt, blockIdx.x), s_tab4, bt.chain_smem, F, dom);
}

// Failure-detection probe: a two-CTA launch in which CTA 1 never arrives, so CTA 0's
// grid_barrier wait runs out (2 s), sets status bit 1 and the kernel returns.
__global__ void k_barrier_probe(unsigned* ctr, unsigned* status) {
  if (blockIdx.x == 1) return;
  grid_barrier(ctr, 2u, status);
}

// Block-wide argmax of (area bits, position): the largest area, lowest position.
__device__ void block_argmax(long long& ab, long long& pos) {
  __shared__ long long s_ab[32], s_pos[32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) {
    const long long oab = __shfl_xor_sync(kFull, ab, d);
    const long long opos = __shfl_xor_sync(kFull, pos, d);
    if (oab > ab || (oab == ab && opos < pos)) { ab = oab; pos = opos; }
  }
  __syncthreads();
  if (lane == 0) { s_ab[wid] = ab; s_pos[wid] = pos; }
  __syncthreads();
  if (wid == 0) {
    ab = lane < nw ? s_ab[lane] : -1;
    pos = lane < nw ? s_pos[lane] : LLONG_MAX;
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
      const long long oab = __shfl_xor_sync(kFull, ab, d);
      const long long opos = __shfl_xor_sync(kFull, pos, d);
      if (oab > ab || (oab == ab && opos < pos)) { ab = oab; pos = opos; }
    }
    if (lane == 0) { s_ab[0] = ab; s_pos[0] = pos; }
  }
  __syncthreads();
  ab = s_ab[0];
  pos = s_pos[0];
}

// Sequential LTTB with one CTA per series (batched series with large buckets).
__global__ void __launch_bounds__(kGridThreads) k_lttb_block(const __grid_constant__ Batch bt) {
  pdl_wait();
  pdl_trigger();
  const SeriesPlan& sp = plan_of(bt, blockIdx.x);
  if (sp.engine != EN_BLOCK) return;
  if (sp.branch != BR_LTTB_ALL && sp.branch != BR_MINMAX_LTTB) return;
  const int64_t m = lttb_m(sp);
  if (m <= sp.n_out) return;
  const int64_t K = sp.n_out - 2, N = m - 2;
  const int lane = threadIdx.x & 31;
  for (int64_t j = threadIdx.x >> 5; j < K; j += blockDim.x >> 5) {  // a warp per bucket mean
    int64_t lo, hi;
    next_bucket(j, sp.dK, N, m, &lo, &hi);
    double xc, yc;
    bucket_mean_warp(sp, lo, hi, lane, &xc, &yc);
    if (lane == 0) {
      sp.means[2 * j] = xc;
      sp.means[2 * j + 1] = yc;
    }
  }
  __syncthreads();
  int64_t a = 0;
  for (int64_t j = 0; j < K; ++j) {
    const int64_t lj = part_start(j, N, sp.dK), lj1 = part_start(j + 1, N, sp.dK);
    const double xc = sp.means[2 * j], yc = sp.means[2 * j + 1];
    const int64_t ia = index_of(sp, a);
    const double xa = x_of(sp, ia), ya = y_of(sp, ia);
    long long ab = -1, pos = LLONG_MAX;
    for (int64_t q = lj + threadIdx.x; q < lj1; q += blockDim.x) {
      const int64_t ib = index_of(sp, q);
      const long long v = __double_as_longlong(tri_area(xa, ya, x_of(sp, ib), y_of(sp, ib), xc, yc));
      if (v > ab) { ab = v; pos = q; }
    }
    block_argmax(ab, pos);
    a = pos;
    if (threadIdx.x == 0) sp.out[j + 1] = index_of(sp, a);
  }
  if (threadIdx.x == 0) {
    sp.out[0] = index_of(sp, 0);
    sp.out[K + 1] = index_of(sp, m - 1);
    if (sp.out_count) *sp.out_count = sp.n_out;
  }
}

__global__ void k_iota(int64_t* out, int64_t n, int64_t* out_count) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = i;
  if (blockIdx.x == 0 && threadIdx.x == 0 && out_count) *out_count = n;
}

}  // namespace

cudaError_t launch_barrier_probe(const Batch& bt, cudaStream_t st) {
  k_barrier_probe<<<2, 32, 0, st>>>(bt.barrier, bt.status);
  return cudaGetLastError();
}

cudaError_t launch_tables(const Batch& bt, cudaStream_t st) {
  if (bt.total_slots <= 0) return cudaSuccess;
  // the tuning's rounds, else as many rounds per warp as keep about 16 warps per SM
  // busy, at most kTableRounds
  int dev = 0, sms = 152;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  Batch b = bt;
  const int64_t r = bt.tab_rounds_req > 0 ? bt.tab_rounds_req : bt.total_slots / ((int64_t)sms * 16 * 32);
  b.tab_rounds = (int32_t)(r < 1 ? 1 : r > kTableRounds ? kTableRounds : r);
  const int64_t per_cta = (int64_t)(kTableThreads / 32) * 32 * b.tab_rounds;
  const int64_t grid = (bt.total_slots + per_cta - 1) / per_cta;
  return launch_pdl(k_tables, dim3((unsigned)grid), dim3(kTableThreads), 0, st, b);
}

cudaError_t launch_chain(const Batch& bt, int n_blocks, int64_t max_positions, cudaStream_t st) {
  if (n_blocks <= 0) return cudaSuccess;
  static bool configured[64] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev >= 0 && dev < 64 && !configured[dev]) {
    e = cudaFuncSetAttribute(k_chain, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kChainSmemMax);
    if (e != cudaSuccess) return e;
    configured[dev] = true;
  }
  Batch b = bt;
  const int64_t bytes = staged_tab_bytes(max_positions);
  b.chain_smem = bytes <= kChainSmemMax ? bytes : 0;
  return launch_pdl(k_chain, dim3(n_blocks), dim3(kChainThreads), (size_t)b.chain_smem, st, b);
}

cudaError_t launch_iota(int64_t* out, int64_t n, int64_t* out_count, cudaStream_t st) {
  int64_t blocks = (n + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  if (blocks < 1) blocks = 1;
  k_iota<<<(unsigned)blocks, 256, 0, st>>>(out, n, out_count);
  return cudaGetLastError();
}

cudaError_t launch_lttb_block(const Batch& bt, int n_blocks, cudaStream_t st) {
  if (n_blocks <= 0) return cudaSuccess;
  return launch_pdl(k_lttb_block, dim3(n_blocks), dim3(kGridThreads), 0, st, bt);
}

}  // namespace mmlttb
