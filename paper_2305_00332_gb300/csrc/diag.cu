// Diagnostics: bounded device waits that nothing satisfies (failure detection), and a
// device-side check of a series' documented preconditions.
#include <algorithm>

#include "host.h"
#include "mmlttb_diag.h"

namespace mmlttb {
namespace {

// Grid-stride scan of the series: NaN in y, a decrease of x, a non-finite float64 x.
// One atomicOr per warp that found something.
__global__ void __launch_bounds__(256) k_check_series(const void* __restrict__ y, int ydt, const void* __restrict__ x,
                                                      int xk, int64_t n, unsigned* flags) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  unsigned f = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    if (ydt == MMLTTB_F32) {
      const float v = __ldg((const float*)y + i);
      if (v != v) f |= MMLTTB_CHECK_Y_NAN;
    } else {
      const double v = __ldg((const double*)y + i);
      if (v != v) f |= MMLTTB_CHECK_Y_NAN;
    }
    if (xk == MMLTTB_X_I64 && i + 1 < n) {
      if (__ldg((const long long*)x + i + 1) < __ldg((const long long*)x + i)) f |= MMLTTB_CHECK_X_DECREASES;
    } else if (xk == MMLTTB_X_F64) {
      const double a = __ldg((const double*)x + i);
      if (!isfinite(a)) f |= MMLTTB_CHECK_X_NONFINITE;
      if (i + 1 < n && __ldg((const double*)x + i + 1) < a) f |= MMLTTB_CHECK_X_DECREASES;
    }
  }
  const unsigned any = __reduce_or_sync(kFull, f);
  if (any && (threadIdx.x & 31) == 0) atomicOr(flags, any);
}

}  // namespace
}  // namespace mmlttb

using namespace mmlttb;

extern "C" int mmlttb_check_series(const void* y, int ydtype, const void* x, int xkind, int64_t n_in,
                                   uint32_t* flags, mmlttb_stream stream) {
  if (!flags || n_in < 0 || (n_in > 0 && !y)) return MMLTTB_EINVAL;
  if (ydtype != MMLTTB_F32 && ydtype != MMLTTB_F64) return MMLTTB_EINVAL;
  if (xkind != MMLTTB_X_IMPLICIT && xkind != MMLTTB_X_I64 && xkind != MMLTTB_X_F64) return MMLTTB_EINVAL;
  if (xkind != MMLTTB_X_IMPLICIT && n_in > 0 && !x) return MMLTTB_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaMemsetAsync(flags, 0, sizeof(uint32_t), st);
  if (e != cudaSuccess) return cuda_fail(e);
  if (n_in == 0) return MMLTTB_OK;
  DevInfo d;
  const int sms = get_dev_info(&d) == MMLTTB_OK && d.sms > 0 ? d.sms : 152;
  const int64_t grid = std::max<int64_t>(1, std::min<int64_t>((n_in + 255) / 256, (int64_t)sms * 8));
  k_check_series<<<(unsigned)grid, 256, 0, st>>>(y, ydtype, x, xkind, n_in, (unsigned*)flags);
  ++g_launches;
  e = cudaGetLastError();
  return e == cudaSuccess ? MMLTTB_OK : cuda_fail(e);
}

extern "C" int mmlttb_diag_wait_timeout(int which, void* workspace, size_t workspace_bytes,
                                        mmlttb_stream stream) {
  if (which != MMLTTB_DIAG_FUSED_BARRIER && which != MMLTTB_DIAG_GRID_BARRIER && which != MMLTTB_DIAG_MBARRIER)
    return MMLTTB_EINVAL;
  if (!workspace || workspace_bytes < kHeader) return MMLTTB_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaMemsetAsync(workspace, 0, kHeader, st);
  if (e != cudaSuccess) return cuda_fail(e);
  Batch bt = {};
  bt.status = (unsigned*)workspace;
  bt.barrier = (unsigned*)((char*)workspace + 4);
  e = which == MMLTTB_DIAG_FUSED_BARRIER ? launch_sync_probe(bt, st)
      : which == MMLTTB_DIAG_GRID_BARRIER ? launch_barrier_probe(bt, st)
                                          : launch_mbarrier_probe(bt, st);
  if (e != cudaSuccess) return cuda_fail(e);
  ++g_launches;
  return MMLTTB_OK;
}
