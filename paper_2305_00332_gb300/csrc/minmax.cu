// MinMax preselection kernels (Sec. 3 first step; MinMax of Sec. 2.2.1, Table 1).
//
//  k_edges   x-width bins: one warp per bin edge, 32-ary search for the first
//            binned point with x >= e_b (x is non-decreasing).
//  k_stream  the HBM-bound pass (stream.cuh): warps over equal ranges of the global
//            work space, 16-byte coalesced loads of y, one Record per bin piece.
#include "stream.cuh"

namespace mmlttb {

namespace {

template <int U, int MINB, int kY, int NT>
__global__ void __launch_bounds__(NT, MINB) k_stream(const __grid_constant__ Batch bt) {
  pdl_wait();
  pdl_trigger();
  if (bt.zero_status && blockIdx.x == 0 && threadIdx.x == 0) zero_header(bt);
  const int64_t w = (int64_t)blockIdx.x * (NT / 32) + (threadIdx.x >> 5);
  if (w >= bt.n_warps) return;
  stream_warp<U, kY>(bt, w, threadIdx.x & 31);
}

// The staged stream: CTAs of kBulkWarps warps, every warp with its own kBulkStages
// shared-memory stages and mbarriers (dynamic shared memory: the stages, then the
// barriers).
template <int kY>
__global__ void __launch_bounds__(kBulkWarps * 32) k_stream_bulk(const __grid_constant__ Batch bt) {
  extern __shared__ __align__(128) unsigned char s_bulk[];
  pdl_wait();
  pdl_trigger();
  if (bt.zero_status && blockIdx.x == 0 && threadIdx.x == 0) zero_header(bt);
  const int wid = threadIdx.x >> 5;
  const int64_t w = (int64_t)blockIdx.x * kBulkWarps + wid;
  if (w >= bt.n_bulk_warps) return;
  const uint32_t s0 = (uint32_t)__cvta_generic_to_shared(s_bulk);
  const uint32_t sbase = s0 + (uint32_t)(wid * kBulkStages * kBulkStageBytes);
  const uint32_t bbase = s0 + (uint32_t)(kBulkWarps * kBulkStages * kBulkStageBytes + wid * kBulkStages * 8);
  bulk_warp<kY>(bt, w, threadIdx.x & 31, sbase, bbase);
}

// Failure-detection probe of the staged stream's stage wait: one warp waits on an
// mbarrier that expects one arrival, which never comes (no copy is issued), so the
// bounded wait runs out (2 s); lane 0 sets status bit 1 and the kernel returns.
__global__ void k_mbarrier_probe(unsigned* status) {
  __shared__ __align__(8) unsigned long long bar;
  const uint32_t b = (uint32_t)__cvta_generic_to_shared(&bar);
  if (threadIdx.x == 0) {
    mbar_init(b, 1);
    fence_mbar_init();
  }
  __syncwarp();
  if (!mbar_wait_bounded(b, 0) && threadIdx.x == 0) atomicOr(status, 1u);
}

__global__ void __launch_bounds__(256) k_edges(const __grid_constant__ Batch bt) {
  pdl_wait();
  pdl_trigger();
  if (bt.zero_status && blockIdx.x == 0 && threadIdx.x == 0) zero_header(bt);
  const int64_t e = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (e >= bt.total_edges) return;
  const int64_t res = edge_at(bt, e, threadIdx.x & 31);
  if ((threadIdx.x & 31) == 0) bt.edges[e] = res;
}

}  // namespace

// The compiled variants (loads in flight per lane U, CTAs per SM MINB, threads per CTA
// NT): (4, 4, 256), (8, 3, 256), (2, 6, 256), (4, 8, 128), (8, 6, 128), (2, 12, 128),
// each for any y and for float32 and float64 y with and without the NaN-aware rule.
constexpr int kVarU[kStreamVariants] = {4, 8, 2, 4, 8, 2};
constexpr int kVarMinB[kStreamVariants] = {4, 3, 6, 8, 6, 12};
constexpr int kVarThreads[kStreamVariants] = {256, 256, 256, 128, 128, 128};
template <int kY>
static const void* stream_kernel_y(int v) {
  switch (v) {
    case 1: return (const void*)k_stream<8, 3, kY, 256>;
    case 2: return (const void*)k_stream<2, 6, kY, 256>;
    case 3: return (const void*)k_stream<4, 8, kY, 128>;
    case 4: return (const void*)k_stream<8, 6, kY, 128>;
    case 5: return (const void*)k_stream<2, 12, kY, 128>;
    default: return (const void*)k_stream<4, 4, kY, 256>;
  }
}
static const void* stream_kernel(int v, int ymode) {
  switch (ymode) {
    case kYF32: return stream_kernel_y<kYF32>(v);
    case kYF64: return stream_kernel_y<kYF64>(v);
    case kYF32Nan: return stream_kernel_y<kYF32Nan>(v);
    case kYF64Nan: return stream_kernel_y<kYF64Nan>(v);
    default: return stream_kernel_y<kYAny>(v);
  }
}

int stream_variant_info(int v, int* unroll, int* min_blocks) {
  if (v < 0 || v >= kStreamVariants) return -1;
  *unroll = kVarU[v];
  *min_blocks = kVarMinB[v];
  return 0;
}

int stream_variant_threads(int v) { return v >= 0 && v < kStreamVariants ? kVarThreads[v] : 256; }

int stream_blocks_per_sm(int v) {
  int bps = 0;
  int b0 = 0;
  for (int y = kYAny; y <= kYF64Nan; ++y) {  // the smallest occupancy of the variant's kernels
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, stream_kernel(v, y), kVarThreads[v], 0) != cudaSuccess)
      return 1;
    if (y == kYAny || bps < b0) b0 = bps;
  }
  return b0 > 0 ? b0 : 1;
}

cudaError_t launch_edges(const Batch& bt, cudaStream_t st) {
  if (bt.total_edges <= 0) return cudaSuccess;
  const int64_t threads = bt.total_edges * 32;
  const int64_t grid = (threads + 255) / 256;
  return launch_pdl(k_edges, dim3((unsigned)grid), dim3(256), 0, st, bt);
}

template <int kY>
static cudaError_t launch_stream_y(const Batch& bt, int64_t grid, int variant, cudaStream_t st) {
  const dim3 g((unsigned)grid), b(kVarThreads[variant]);
  switch (variant) {
    case 1: return launch_pdl(k_stream<8, 3, kY, 256>, g, b, 0, st, bt);
    case 2: return launch_pdl(k_stream<2, 6, kY, 256>, g, b, 0, st, bt);
    case 3: return launch_pdl(k_stream<4, 8, kY, 128>, g, b, 0, st, bt);
    case 4: return launch_pdl(k_stream<8, 6, kY, 128>, g, b, 0, st, bt);
    case 5: return launch_pdl(k_stream<2, 12, kY, 128>, g, b, 0, st, bt);
    default: return launch_pdl(k_stream<4, 4, kY, 256>, g, b, 0, st, bt);
  }
}

cudaError_t launch_stream(const Batch& bt, int variant, int ymode, cudaStream_t st) {
  if (bt.n_warps <= 0) return cudaSuccess;
  if (variant < 0 || variant >= kStreamVariants) variant = 0;
  const int wpc = kVarThreads[variant] / 32;
  const int64_t grid = (bt.n_warps + wpc - 1) / wpc;
  switch (ymode) {
    case kYF32: return launch_stream_y<kYF32>(bt, grid, variant, st);
    case kYF64: return launch_stream_y<kYF64>(bt, grid, variant, st);
    case kYF32Nan: return launch_stream_y<kYF32Nan>(bt, grid, variant, st);
    case kYF64Nan: return launch_stream_y<kYF64Nan>(bt, grid, variant, st);
    default: return launch_stream_y<kYAny>(bt, grid, variant, st);
  }
}

template <int kY>
static cudaError_t launch_bulk_y(const Batch& bt, cudaStream_t st) {
  static bool configured[64] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  if (!configured[dev]) {
    e = cudaFuncSetAttribute(k_stream_bulk<kY>, cudaFuncAttributeMaxDynamicSharedMemorySize, kBulkSmemBytes);
    if (e != cudaSuccess) return e;
    configured[dev] = true;
  }
  const int64_t grid = (bt.n_bulk_warps + kBulkWarps - 1) / kBulkWarps;
  return launch_pdl(k_stream_bulk<kY>, dim3((unsigned)grid), dim3(kBulkWarps * 32), kBulkSmemBytes, st, bt);
}

int stream_bulk_blocks_per_sm() {
  const void* ks[3] = {(const void*)k_stream_bulk<kYAny>, (const void*)k_stream_bulk<kYF32>,
                       (const void*)k_stream_bulk<kYF32Nan>};
  int b0 = 0;
  for (int i = 0; i < 3; ++i) {  // the smallest occupancy of the y modes
    int bps = 0;
    if (cudaFuncSetAttribute(ks[i], cudaFuncAttributeMaxDynamicSharedMemorySize, kBulkSmemBytes) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, ks[i], kBulkWarps * 32, kBulkSmemBytes) != cudaSuccess)
      return 1;
    if (i == 0 || bps < b0) b0 = bps;
  }
  return b0 > 0 ? b0 : 1;
}

cudaError_t launch_mbarrier_probe(const Batch& bt, cudaStream_t st) {
  k_mbarrier_probe<<<1, 32, 0, st>>>(bt.status);
  return cudaGetLastError();
}

cudaError_t launch_stream_bulk(const Batch& bt, int ymode, cudaStream_t st) {
  if (bt.n_bulk_warps <= 0) return cudaSuccess;
  switch (ymode) {  // staged series hold float32 y
    case kYF32: return launch_bulk_y<kYF32>(bt, st);
    case kYF32Nan: return launch_bulk_y<kYF32Nan>(bt, st);
    default: return launch_bulk_y<kYAny>(bt, st);
  }
}

}  // namespace mmlttb
