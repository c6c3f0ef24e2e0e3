// Fused MinMaxLTTB for one series in one persistent launch (Sec. 3: MinMax
// preselection, then LTTB on the preselected points).
//
// The split path launches up to seven dependent kernels; each launch boundary costs
// microseconds, which dominates small series and the tail of large ones.  k_fused
// is a cooperative launch of one 512-thread CTA per SM that runs the steps in turn,
// separated by a grid-wide barrier:
//
//   [edges]     x-width bins: the grid's warps search the bin edges (kStream)
//   [stream]    MinMax records over the whole series (kStream)
//   compaction  pass 1: CTA c resolves its contiguous share of the bins and
//               publishes how many indices they emit; pass 2: every CTA sums the
//               totals before it and places its bins' indices
//   LTTB        buckets of at most 8 positions: every CTA forms the picks of its
//               buckets, composes them and, after one barrier, resolves its share
//               of the chain (lttb_by_ctas).  Larger buckets: the transition tables
//               over every SM, a barrier, then CTA 0 resolves the chain.  (The FP64
//               areas are the costly part, and the FP64 pipe is narrow.)
//
// With kStream = false the kernel is the tail of a large series: k_edges and
// k_stream run before it, and it starts on their records.
//
// The barrier counter is a workspace header word that is zero when the call starts
// (cleared by the call's first kernel or by a memset); every wait on it gives up
// after 2 s (status bit 1, and the kernel returns).
#include "compact.cuh"
#include "lttb.cuh"

namespace mmlttb {

namespace {

constexpr int kFusedThreads = 512;
constexpr int kFusedWarps = kFusedThreads / 32;
constexpr int kFusedUnroll = 4;                   // 16-byte loads in flight per lane
constexpr int64_t kFusedTabSmemMax = 160 * 1024;  // tables staged in shared memory up to this size
constexpr unsigned long long kWaitNs = 2000000000ull;

__device__ __forceinline__ unsigned long long now_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Grid-wide barrier (all CTAs of a cooperative launch) on one counter whose low 31
// bits start below 2^31 - gridDim.x: CTA 0 adds 2^31 - (gridDim.x - 1), every other
// CTA adds 1, so the top bit flips exactly when the last CTA arrives and the low
// bits return to their start (the counter is ready for the next barrier).  Returns
// false when the wait timed out (status bit 1 set); the caller then returns.
__device__ bool grid_sync(const Batch& bt) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned inc = blockIdx.x == 0 ? 0x80000000u - (gridDim.x - 1u) : 1u;
    __threadfence();  // this CTA's writes are visible before it arrives
    const unsigned old = atomicAdd(bt.barrier, inc);
    s_ok = 1;
    const unsigned long long t0 = now_ns();
    while (((ld_acquire_u32(bt.barrier) ^ old) & 0x80000000u) == 0u) {
      if (now_ns() - t0 > kWaitNs) {
        set_status(bt.status, 1u);
        s_ok = 0;
        break;
      }
    }
  }
  __syncthreads();
  return s_ok != 0;
}

// Failure-detection probe: a two-CTA launch in which CTA 1 never arrives, so CTA 0's
// grid_sync wait runs out (kWaitNs), sets status bit 1 and the kernel returns.
__global__ void k_sync_probe(const __grid_constant__ Batch bt) {
  if (blockIdx.x == 1) return;
  grid_sync(bt);
}

__device__ __forceinline__ long long warp_sum64(long long v) {
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(kFull, v, d);
  return v;
}

// LTTB on the preselected positions of a single series whose buckets hold at most 8
// positions (MinMaxLTTB with r_ps up to 7), on every CTA of the grid at once.  CTA c
// owns buckets [jc0, jc1):
//   1. the picks after every position of the bucket before (bucket_pick), packed
//      into one map of 8 bytes per bucket (entry offset -> pick offset);
//   2. an inclusive block scan of the bucket maps under composition, so each bucket
//      holds the map from the pick before jc0 to its own pick;
//   3. the CTA publishes its total map; after a grid barrier every CTA composes the
//      maps of the CTAs before it (a warp reduction in CTA order) and evaluates the
//      result at the chain's start, position 0: the pick before jc0;
//   4. every bucket's pick is one byte lookup; the picks become indices.
// The sequential chain of Sec. 2.2.1 is resolved exactly: every map entry is a pick
// the sequential method would make from that previous pick.  s_lo/s_hi hold 4096
// maps each.  Returns false when the barrier timed out.
__device__ bool lttb_by_ctas(const Batch& bt, const SeriesPlan& sp, int64_t m, int lgS,
                             unsigned* s_lo, unsigned* s_hi) {
  __shared__ unsigned s_wl[kFusedWarps], s_wh[kFusedWarps];
  __shared__ unsigned s_cl, s_ch;
  __shared__ int s_entry;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t c = blockIdx.x;
  const int64_t K = sp.n_out - 2, N = m - 2;
  const int64_t jc0 = muldiv(c, K, bt.dgrid), jc1 = muldiv(c + 1, K, bt.dgrid);
  const int64_t nbk = jc1 - jc0;
  const int S = 1 << lgS;
  // 1. bucket maps
  for (int64_t base = (int64_t)warp * 32; base < (nbk << lgS); base += kFusedThreads) {
    const int64_t slot = base + lane;
    const int64_t jj = slot >> lgS;
    const int k = (int)(slot & (S - 1));
    int64_t p;
    bool valid;
    const int pick = bucket_pick(sp, m, jj < nbk ? jc0 + jj : K, k, lgS, lane, &p, &valid);
    unsigned wl = 0u, wh = 0u;
    if (valid) {
      if (k < 4) wl = (unsigned)pick << (8 * k);
      else wh = (unsigned)pick << (8 * (k - 4));
    }
    for (int d = 1; d < S; d <<= 1) {
      wl |= __shfl_xor_sync(kFull, wl, d);
      wh |= __shfl_xor_sync(kFull, wh, d);
    }
    if (k == 0 && jj < nbk) {
      s_lo[jj] = wl;
      s_hi[jj] = wh;
    }
  }
  __syncthreads();
  // 2. prefix of the bucket maps within the CTA
  Map8 carry = kIdentity8;
  for (int64_t t0 = 0; t0 < nbk; t0 += kFusedThreads) {
    const int64_t i = t0 + tid;
    Map8 P = i < nbk ? Map8{s_lo[i], s_hi[i]} : kIdentity8;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const Map8 o = shfl_up_map(P, d);
      if (lane >= d) P = compose(P, o);
    }
    if (lane == 31) {
      s_wl[warp] = P.lo;
      s_wh[warp] = P.hi;
    }
    __syncthreads();
    if (warp == 0) {
      Map8 W = lane < kFusedWarps ? Map8{s_wl[lane], s_wh[lane]} : kIdentity8;
#pragma unroll
      for (int d = 1; d < kFusedWarps; d <<= 1) {
        const Map8 o = shfl_up_map(W, d);
        if (lane >= d) W = compose(W, o);
      }
      Map8 E = shfl_up_map(W, 1);
      if (lane == 0) E = kIdentity8;
      E = compose(E, carry);  // everything before this warp, earlier tiles first
      const Map8 total = compose(shfl_map(W, kFusedWarps - 1), carry);
      if (lane < kFusedWarps) {
        s_wl[lane] = E.lo;
        s_wh[lane] = E.hi;
      }
      if (lane == 0) {
        s_cl = total.lo;
        s_ch = total.hi;
      }
    }
    __syncthreads();
    P = compose(P, Map8{s_wl[warp], s_wh[warp]});
    if (i < nbk) {
      s_lo[i] = P.lo;
      s_hi[i] = P.hi;
    }
    carry = Map8{s_cl, s_ch};
    __syncthreads();
  }
  // 3. the CTA's map for the others, then the pick before this CTA's first bucket
  if (tid == 0) bt.fused_tot[c] = (long long)(((unsigned long long)carry.hi << 32) | carry.lo);
  if (!grid_sync(bt)) return false;
  if (warp == 0) {
    const int64_t q = (c + 31) >> 5;  // CTAs per lane, in order
    Map8 A = kIdentity8;
    for (int64_t k2 = (int64_t)lane * q; k2 < (int64_t)(lane + 1) * q && k2 < c; ++k2) {
      const unsigned long long v = (unsigned long long)bt.fused_tot[k2];
      A = compose(Map8{(unsigned)v, (unsigned)(v >> 32)}, A);
    }
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {  // lane i (earlier CTAs) then lane i + d
      const Map8 o = shfl_down_map(A, d);
      if ((lane & (2 * d - 1)) == 0) A = compose(o, A);
    }
    if (lane == 0) s_entry = map_at(A, 0);  // the chain starts at position 0
  }
  __syncthreads();
  const int e = s_entry;
  // 4. picks -> output indices
  for (int64_t jj = tid; jj < nbk; jj += kFusedThreads) {
    const int64_t j = jc0 + jj;
    const int off = map_at(Map8{s_lo[jj], s_hi[jj]}, e);
    sp.out[j + 1] = index_of(sp, part_start(j, N, sp.dK) + off);
  }
  if (c == 0 && tid == 0) {
    sp.out[0] = index_of(sp, 0);
    sp.out[K + 1] = index_of(sp, m - 1);
    if (sp.out_count) *sp.out_count = sp.n_out;
  }
  return true;
}

template <bool kStream>
__global__ void __launch_bounds__(kFusedThreads, 1) k_fused(const __grid_constant__ Batch bt) {
  // chain scratch: F[c][ia][t] = thread t's map, entry ia (CTA 0), or the bucket maps
  // of lttb_by_ctas (every CTA)
  __shared__ __align__(16) uint8_t F[2][kTableMaxBucket][kFusedThreads];
  __shared__ uint8_t dom[2][kFusedThreads];
  __shared__ long long s_warp[kFusedWarps];
  __shared__ long long s_base, s_grand;
  extern __shared__ uint4 s_tab4[];
  const int64_t c = blockIdx.x, G = gridDim.x;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t gw = c * kFusedWarps + warp, nw = G * kFusedWarps;
  const SeriesPlan& sp = bt.one;
  pdl_wait();
  pdl_trigger();
  if constexpr (kStream) {
    if (bt.total_edges > 0) {
      for (int64_t e = gw; e < bt.total_edges; e += nw) {
        const int64_t r = edge_at(bt, e, lane);
        if (lane == 0) bt.edges[e] = r;
      }
      if (!grid_sync(bt)) return;
    }
    for (int64_t w = gw; w < bt.n_warps; w += nw) stream_warp<kFusedUnroll>(bt, w, lane);
    if (!grid_sync(bt)) return;
  }
  if (binned(sp.branch)) {
    // CTA c owns the contiguous bins [b0, b1)
    const int64_t Bc = (sp.B + G - 1) / G;
    const int64_t b0 = c * Bc < sp.B ? c * Bc : sp.B;
    const int64_t b1 = b0 + Bc < sp.B ? b0 + Bc : sp.B;
    long long acc = 0;
    for (int64_t t = b0; t < b1; t += kFusedThreads) {
      const int64_t b = t + tid;
      if (b < b1) {
        int64_t lo, hi, first, last;
        long long klo, khi;
        resolve_bin(bt, sp, b, &lo, &hi, &klo, &khi, &first, &last);
        bt.binres[4 * b] = lo;
        bt.binres[4 * b + 1] = hi;
        bt.binres[4 * b + 2] = klo;
        bt.binres[4 * b + 3] = khi;
        acc += bin_count(sp, lo, hi, first, last);
      }
    }
    acc = warp_sum64(acc);
    if (lane == 0) s_warp[warp] = acc;
    __syncthreads();
    if (tid == 0) {
      long long t = 0;
      for (int w = 0; w < kFusedWarps; ++w) t += s_warp[w];
      bt.fused_tot[c] = t;
    }
    if (!grid_sync(bt)) return;
    if (warp == 0) {
      long long before = 0, grand = 0;
      for (int64_t k = lane; k < G; k += 32) {
        const long long v = bt.fused_tot[k];
        grand += v;
        if (k < c) before += v;
      }
      before = warp_sum64(before);
      grand = warp_sum64(grand);
      if (lane == 0) {
        s_base = before;
        s_grand = grand;
      }
    }
    __syncthreads();
    if (c == 0 && tid == 0) finish_series(sp, s_grand);
    long long carry = s_base;
    for (int64_t t = b0; t < b1; t += kFusedThreads) {
      const int64_t b = t + tid;
      int64_t lo = -1, hi = -1, first = -1, last = -1;
      long long klo = 0, khi = 0;
      if (b < b1) {
        lo = bt.binres[4 * b];
        hi = bt.binres[4 * b + 1];
        klo = bt.binres[4 * b + 2];
        khi = bt.binres[4 * b + 3];
        if (sp.branch == BR_M4 && lo >= 0) {
          first = bin_start(bt, sp, b);
          last = ((b + 1 >= sp.B) ? sp.p0 + sp.nb : bin_start(bt, sp, b + 1)) - 1;
        }
      }
      const int cnt = bin_count(sp, lo, hi, first, last);
      int excl;
      const int tile = block_excl_scan<kFusedThreads>(cnt, &excl);
      place_bin(sp, lo, hi, klo, khi, first, last, cnt, carry + excl);
      carry += tile;
    }
    if (sp.branch == BR_PRESELECT || sp.branch == BR_M4 || sp.engine != EN_TABLES) return;
    if (!grid_sync(bt)) return;  // the list is complete
  }
  if (sp.engine != EN_TABLES) return;
  {
    const int64_t m = lttb_m(sp);
    if (m > sp.n_out) {
      const int64_t K = sp.n_out - 2;
      const int64_t bmax = (int64_t)div_by((uint64_t)(m - 2 + K - 1), sp.dK);  // largest bucket
      int lgS = 0;
      while ((int64_t(1) << lgS) < bmax) ++lgS;
      const int64_t per_cta = (int64_t)div_by((uint64_t)(K + G - 1), bt.dgrid);
      if (lgS <= 3 && per_cta <= 4096) {
        lttb_by_ctas(bt, sp, m, lgS, (unsigned*)&F[0][0][0], (unsigned*)&F[0][0][0] + 4096);
        return;
      }
    }
    const int64_t nslots = m > sp.n_out ? (sp.n_out - 2) << sp.tab_lgS : 0;
    // warp-sized slot blocks dealt round-robin over the CTAs, so the FP64 area work
    // of a small table spreads over every SM
    for (int64_t base = ((int64_t)warp * G + c) * 32; base < nslots; base += nw * 32)
      table_bucket_entry(sp, m, base + lane, lane);
  }
  if (!grid_sync(bt)) return;  // every table entry is visible
  if (c != 0) return;
  chain_series<kFusedThreads>(sp, s_tab4, bt.chain_smem, F, dom);
}

template <bool kStream>
cudaError_t launch_fused_t(const Batch& bt, int grid, cudaStream_t st) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3(kFusedThreads);
  cfg.dynamicSmemBytes = (size_t)bt.chain_smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[2];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[1].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 2;
  return cudaLaunchKernelEx(&cfg, k_fused<kStream>, bt);
}

}  // namespace

cudaError_t launch_sync_probe(const Batch& bt, cudaStream_t st) {
  k_sync_probe<<<2, 32, 0, st>>>(bt);
  return cudaGetLastError();
}

// CTAs of the fused kernel: one per SM when one 512-thread CTA with the largest
// staged table fits on an SM, else 0 (the fused path is then not used).
int fused_grid_size(int sms) {
  for (const void* k : {(const void*)k_fused<true>, (const void*)k_fused<false>}) {
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFusedTabSmemMax) !=
        cudaSuccess) {
      cudaGetLastError();
      return 0;
    }
    int bps = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k, kFusedThreads, (size_t)kFusedTabSmemMax) !=
            cudaSuccess ||
        bps < 1) {
      cudaGetLastError();
      return 0;
    }
  }
  return sms;
}

int64_t fused_tab_smem(int64_t tab_cap) {
  const int64_t b = staged_tab_bytes(tab_cap);
  return b <= kFusedTabSmemMax ? b : 0;
}

int fused_warps(int grid) { return grid * kFusedWarps; }

cudaError_t launch_fused(const Batch& bt, int grid, bool with_stream, cudaStream_t st) {
  return with_stream ? launch_fused_t<true>(bt, grid, st) : launch_fused_t<false>(bt, grid, st);
}

}  // namespace mmlttb
