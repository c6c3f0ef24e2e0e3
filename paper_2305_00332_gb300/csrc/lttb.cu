// LTTB stage kernels (Sec. 2.2.1 LTTB; Sec. 3 second step of MinMaxLTTB).
//
// LTTB is a chain: the pick b_j of bucket j depends on the pick of bucket j-1.
// When buckets are small (MinMaxLTTB puts about r_ps points in each), the chain is
// cut into independent pieces:
//   k_tables  every position p that can be the previous pick of bucket j (p in
//             bucket j-1, or p = 0 for j = 0) gets T[p] = the offset in bucket j of
//             the point with the largest area against p and the mean of bucket j+1.
//             Each area is the same FP64 expression the sequential method evaluates,
//             so every table entry equals the sequential choice for that p.
//   k_chain   one CTA per series resolves b_j = T[L_{j-1} + b_{j-1}] for all j by a
//             parallel prefix over function composition (Hillis-Steele), then writes
//             the picked indices.
// Large buckets use k_lttb_grid: one grid-wide argmax per bucket (cooperative
// launch, bounded spin barrier), or k_lttb_block: one CTA per series.
#include "common.cuh"

namespace mmlttb {

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kChainThreads = 512;
constexpr int64_t kChainSmemMax = 160 * 1024;  // tables staged in shared memory up to this size

__device__ __forceinline__ int64_t lttb_m(const SeriesPlan& sp) {
  return sp.branch == BR_LTTB_ALL ? sp.n : *sp.m_ptr;
}

// Mean of LTTB positions [lo, hi): left-to-right FP64 sums, one division each (R7).
__device__ void bucket_mean(const SeriesPlan& sp, int64_t lo, int64_t hi, double* xc, double* yc) {
  double sx = 0.0, sy = 0.0;
  if (sp.xk == MMLTTB_X_IMPLICIT && !sp.sel && hi > 0 && hi - lo <= ((1ll << 53) - 1) / hi) {
    // Implicit x on all points: the indices lo..hi-1 and all their partial sums are
    // integers below 2^53, so the sequential FP64 sum is exact and equals the
    // closed form.
    sx = (double)((lo + hi - 1) * (hi - lo) / 2);
    for (int64_t p = lo; p < hi; ++p) sy = __dadd_rn(sy, y_of(sp, p));
  } else {
    for (int64_t p = lo; p < hi; ++p) {
      double xp, yp;
      pos_xy(sp, p, &xp, &yp);
      sx = __dadd_rn(sx, xp);
      sy = __dadd_rn(sy, yp);
    }
  }
  const double cnt = (double)(hi - lo);
  *xc = __ddiv_rn(sx, cnt);
  *yc = __ddiv_rn(sy, cnt);
}

// Bounds of the bucket after bucket j (R1), or the last point for the last bucket (R5).
__device__ __forceinline__ void next_bucket(int64_t j, int64_t K, int64_t N, int64_t m,
                                            int64_t* lo, int64_t* hi) {
  if (j + 1 < K) {
    *lo = part_start(j + 1, N, K);
    *hi = part_start(j + 2, N, K);
  } else {
    *lo = m - 1;
    *hi = m;
  }
}

constexpr int kTableThreads = 64;  // small CTAs: the positions spread over every SM

__global__ void __launch_bounds__(kTableThreads) k_tables(const __grid_constant__ Batch bt) {
  pdl_wait();
  pdl_trigger();
  const int lane = threadIdx.x & 31;
  const int64_t slot = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  // Every lane stays to the warp-wide steps below; `work` marks lanes with a table
  // entry to fill.
  bool work = slot < bt.total_slots;
  int s = 0;
  int64_t p = 0, m = 0, K = 0, N = 0, jt = 0;
  const SeriesPlan* spp = nullptr;
  if (work) {
    s = bt.tab_offs ? upper_index(bt.tab_offs, bt.n_series, slot) : 0;
    spp = &plan_of(bt, s);
    p = slot - spp->tab_off;
    work = spp->engine == EN_TABLES;
    if (work) {
      m = lttb_m(*spp);
      work = p < m && m > spp->n_out;
    }
    if (work) {
      K = spp->n_out - 2;
      N = m - 2;
      if (p == 0) jt = 0;               // the bucket whose pick follows a pick at p
      else if (p <= m - 2) jt = part_of(p, N, K) + 1;
      else work = false;
      if (jt >= K) work = false;
    }
  }
  // Lanes that target the same bucket of the same series share its next-bucket mean:
  // the lowest such lane computes it (R7) and broadcasts it.
  const unsigned long long key = work ? ((unsigned long long)s << 40) ^ (unsigned long long)jt
                                      : ~0ull - (unsigned long long)lane;
  const unsigned group = __match_any_sync(0xffffffffu, key);
  const int leader = __ffs(group) - 1;
  double xc = 0.0, yc = 0.0;
  int64_t lo = 0, hi = 0;
  if (work) {
    const SeriesPlan& sp = *spp;
    lo = part_start(jt, N, K);
    hi = part_start(jt + 1, N, K);
    if (lane == leader) {
      int64_t nlo, nhi;
      next_bucket(jt, K, N, m, &nlo, &nhi);
      bucket_mean(sp, nlo, nhi, &xc, &yc);
    }
  }
  xc = __shfl_sync(0xffffffffu, xc, leader);
  yc = __shfl_sync(0xffffffffu, yc, leader);
  if (!work) return;
  const SeriesPlan& sp = *spp;
  double xa, ya;
  pos_xy(sp, p, &xa, &ya);
  long long best = -1;  // bits of a non-negative double order like the double
  int pick = 0;
  for (int64_t q = lo; q < hi; ++q) {
    double xb, yb;
    pos_xy(sp, q, &xb, &yb);
    const double area = tri_area(xa, ya, xb, yb, xc, yc);
    const long long ab = __double_as_longlong(area);
    if (q == lo || ab > best) { best = ab; pick = (int)(q - lo); }  // R8: first wins
  }
  sp.tab[p] = (uint8_t)pick;
}

// Bucket starts L_j = floor(j*N/K)+1 for consecutive j without a division per step.
struct PartIter {
  int64_t L, rem, q, r, K;
  __device__ PartIter(int64_t j, int64_t N, int64_t K_) : K(K_) {
    q = N / K;
    r = N - q * K;
    const unsigned __int128 jn = (unsigned __int128)(uint64_t)j * (uint64_t)N;
    const int64_t f = (int64_t)(jn / (uint64_t)K);
    L = f + 1;
    rem = (int64_t)(jn - (unsigned __int128)(uint64_t)f * (uint64_t)K);
  }
  __device__ void next() {  // j -> j+1
    L += q;
    rem += r;
    if (rem >= K) {
      rem -= K;
      L += 1;
    }
  }
};

__global__ void __launch_bounds__(kChainThreads) k_chain(const __grid_constant__ Batch bt) {
  // F[c][ia][t]: thread t's map, entry ia (entry-major, so a warp touches 32
  // consecutive bytes per entry instead of 32 bytes apart)
  __shared__ uint8_t F[2][kTableMaxBucket][kChainThreads];
  __shared__ uint8_t dom[2][kChainThreads];
  extern __shared__ uint4 s_tab4[];
  pdl_wait();
  pdl_trigger();
  const SeriesPlan& sp = plan_of(bt, blockIdx.x);
  const int tid = threadIdx.x;
  if (sp.branch == BR_ARANGE) {
    for (int64_t i = tid; i < sp.n; i += blockDim.x) sp.out[i] = i;
    if (tid == 0 && sp.out_count) *sp.out_count = sp.n;
    return;
  }
  if (sp.branch != BR_LTTB_ALL && sp.branch != BR_MINMAX_LTTB) return;
  const int64_t m = lttb_m(sp);
  if (m <= sp.n_out) {  // nothing to drop (R14)
    for (int64_t i = tid; i < m; i += blockDim.x) sp.out[i] = index_of(sp, i);
    if (tid == 0 && sp.out_count) *sp.out_count = m;
    return;
  }
  if (sp.engine != EN_TABLES) return;
  const int64_t K = sp.n_out - 2, N = m - 2;
  const int T = K < kChainThreads ? (int)K : kChainThreads;
  const uint8_t* tab = sp.tab;
  if (m <= bt.chain_smem) {  // stage the tables (16-byte aligned storage, padded to 16)
    const int64_t nv = (m + 15) / 16;
    const uint4* src = (const uint4*)sp.tab;
    for (int64_t i = tid; i < nv; i += blockDim.x) s_tab4[i] = src[i];
    __syncthreads();
    tab = (const uint8_t*)s_tab4;
  }
  int64_t j0 = 0, j1 = 0;
  if (tid < T) {
    j0 = muldiv(tid, K, T);
    j1 = muldiv(tid + 1, K, T);
    // Phase 1: compose this segment's steps for every possible entry offset.
    PartIter it(j0 > 0 ? j0 - 1 : 0, N, K);  // start of bucket j0-1 (or of bucket 0)
    int d0 = 1;
    int64_t lprev = 0;
    if (j0 > 0) {
      lprev = it.L;
      it.next();
      d0 = (int)(it.L - lprev);
    }
    for (int ia = 0; ia < d0; ++ia) F[0][ia][tid] = (uint8_t)ia;
    for (int64_t j = j0; j < j1; ++j) {
      for (int ia = 0; ia < d0; ++ia) F[0][ia][tid] = tab[lprev + F[0][ia][tid]];
      lprev = it.L;  // start of bucket j
      it.next();
    }
    dom[0][tid] = (uint8_t)d0;
  }
  // Phase 2: inclusive prefix of the segment maps under composition.
  int c = 0;
  for (int d = 1; d < T; d <<= 1) {
    __syncthreads();
    if (tid < T) {
      if (tid >= d) {
        const int dd = dom[c][tid - d];
        for (int ia = 0; ia < dd; ++ia) F[c ^ 1][ia][tid] = F[c][F[c][ia][tid - d]][tid];
        dom[c ^ 1][tid] = (uint8_t)dd;
      } else {
        const int dd = dom[c][tid];
        for (int ia = 0; ia < dd; ++ia) F[c ^ 1][ia][tid] = F[c][ia][tid];
        dom[c ^ 1][tid] = (uint8_t)dd;
      }
    }
    c ^= 1;
  }
  __syncthreads();
  // Phase 3: walk each segment from its resolved entry; first record the picked
  // positions, then translate them to indices with independent loads.
  if (tid < T) {
    int v = tid == 0 ? 0 : F[c][0][tid - 1];
    PartIter it(j0 > 0 ? j0 - 1 : 0, N, K);
    int64_t lprev = 0;
    if (j0 > 0) {
      lprev = it.L;
      it.next();
    }
    for (int64_t j = j0; j < j1; ++j) {
      v = tab[lprev + v];
      sp.out[j + 1] = it.L + v;  // position in bucket j
      lprev = it.L;
      it.next();
    }
    if (sp.sel)
      for (int64_t j = j0; j < j1; ++j) sp.out[j + 1] = sp.sel[sp.out[j + 1]];
  }
  if (tid == 0) {
    sp.out[0] = index_of(sp, 0);
    sp.out[K + 1] = index_of(sp, m - 1);
    if (sp.out_count) *sp.out_count = sp.n_out;
  }
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Grid-wide barrier on a monotone counter with a 2 s bound.  Returns false (and
// sets status bit 1) when the other CTAs did not all arrive in time.
__device__ bool grid_barrier(unsigned* ctr, unsigned target, unsigned* status) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(ctr, 1u);
    ok = 1;
    const unsigned long long t0 = global_ns();
    while (ld_acquire(ctr) < target) {
      if (global_ns() - t0 > 2000000000ull) {
        set_status(status, 1u);
        ok = 0;
        break;
      }
    }
    __threadfence();
  }
  __syncthreads();
  return ok != 0;
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

// Sequential LTTB with one grid-wide argmax per bucket (single series).
__global__ void __launch_bounds__(kGridThreads) k_lttb_grid(const __grid_constant__ Batch bt) {
  const SeriesPlan& sp = bt.one;
  const int64_t m = lttb_m(sp);
  if (m <= sp.n_out) return;  // k_chain copied the points
  const int64_t K = sp.n_out - 2, N = m - 2;
  const int64_t G = gridDim.x, c = blockIdx.x;
  // Phase A: every next-bucket mean, one thread per bucket.
  for (int64_t j = c * blockDim.x + threadIdx.x; j < K; j += G * blockDim.x) {
    int64_t lo, hi;
    next_bucket(j, K, N, m, &lo, &hi);
    bucket_mean(sp, lo, hi, &sp.means[2 * j], &sp.means[2 * j + 1]);
  }
  if (!grid_barrier(bt.barrier, (unsigned)G, bt.status)) return;
  __shared__ long long s_pick;
  int64_t a = 0;
  long long* part = (long long*)bt.partial;
  for (int64_t j = 0; j < K; ++j) {
    const int64_t lj = part_start(j, N, K), lj1 = part_start(j + 1, N, K);
    const int64_t len = lj1 - lj;
    const int64_t q0 = lj + muldiv(c, len, G), q1 = lj + muldiv(c + 1, len, G);
    const double xc = sp.means[2 * j], yc = sp.means[2 * j + 1];
    const int64_t ia = index_of(sp, a);
    const double xa = x_of(sp, ia), ya = y_of(sp, ia);
    long long ab = -1, pos = LLONG_MAX;
    for (int64_t q = q0 + threadIdx.x; q < q1; q += blockDim.x) {
      const int64_t ib = index_of(sp, q);
      const long long v = __double_as_longlong(tri_area(xa, ya, x_of(sp, ib), y_of(sp, ib), xc, yc));
      if (v > ab) { ab = v; pos = q; }  // increasing q: strict keeps the first
    }
    block_argmax(ab, pos);
    long long* pj = part + (j & 1) * 2 * G;
    if (threadIdx.x == 0) { pj[2 * c] = ab; pj[2 * c + 1] = pos; }
    if (!grid_barrier(bt.barrier, (unsigned)((j + 2) * G), bt.status)) return;
    ab = -1;
    pos = LLONG_MAX;
    for (int64_t k = threadIdx.x; k < G; k += blockDim.x) {
      const long long oab = ((volatile long long*)pj)[2 * k];
      const long long opos = ((volatile long long*)pj)[2 * k + 1];
      if (oab > ab || (oab == ab && opos < pos)) { ab = oab; pos = opos; }
    }
    block_argmax(ab, pos);
    if (threadIdx.x == 0) s_pick = pos;
    __syncthreads();
    a = s_pick;
    if (c == 0 && threadIdx.x == 0) sp.out[j + 1] = index_of(sp, a);
  }
  if (c == 0 && threadIdx.x == 0) {
    sp.out[0] = index_of(sp, 0);
    sp.out[K + 1] = index_of(sp, m - 1);
    if (sp.out_count) *sp.out_count = sp.n_out;
  }
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
  for (int64_t j = threadIdx.x; j < K; j += blockDim.x) {
    int64_t lo, hi;
    next_bucket(j, K, N, m, &lo, &hi);
    bucket_mean(sp, lo, hi, &sp.means[2 * j], &sp.means[2 * j + 1]);
  }
  __syncthreads();
  int64_t a = 0;
  for (int64_t j = 0; j < K; ++j) {
    const int64_t lj = part_start(j, N, K), lj1 = part_start(j + 1, N, K);
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

int lttb_grid_blocks_per_sm() {
  int bps = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k_lttb_grid, kGridThreads, 0) != cudaSuccess)
    return 1;
  if (bps > 2) bps = 2;
  return bps > 0 ? bps : 1;
}

cudaError_t launch_tables(const Batch& bt, cudaStream_t st) {
  if (bt.total_slots <= 0) return cudaSuccess;
  const int64_t grid = (bt.total_slots + kTableThreads - 1) / kTableThreads;
  return launch_pdl(k_tables, dim3((unsigned)grid), dim3(kTableThreads), 0, st, bt);
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
  b.chain_smem = max_positions <= kChainSmemMax ? ((max_positions + 15) & ~int64_t(15)) : 0;
  return launch_pdl(k_chain, dim3(n_blocks), dim3(kChainThreads), (size_t)b.chain_smem, st, b);
}

cudaError_t launch_iota(int64_t* out, int64_t n, int64_t* out_count, cudaStream_t st) {
  int64_t blocks = (n + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  if (blocks < 1) blocks = 1;
  k_iota<<<(unsigned)blocks, 256, 0, st>>>(out, n, out_count);
  return cudaGetLastError();
}

cudaError_t launch_lttb_grid(const Batch& bt, int grid, cudaStream_t st) {
  Batch copy = bt;
  void* args[] = {&copy};
  return cudaLaunchCooperativeKernel((const void*)k_lttb_grid, dim3(grid), dim3(kGridThreads), args,
                                     0, st);
}

cudaError_t launch_lttb_block(const Batch& bt, int n_blocks, cudaStream_t st) {
  if (n_blocks <= 0) return cudaSuccess;
  return launch_pdl(k_lttb_block, dim3(n_blocks), dim3(kGridThreads), 0, st, bt);
}

}  // namespace mmlttb
