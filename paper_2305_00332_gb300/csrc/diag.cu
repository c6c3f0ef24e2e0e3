// Failure-detection diagnostics: bounded device waits that nothing satisfies.
#include "host.h"
#include "mmlttb_diag.h"

using namespace mmlttb;

extern "C" int mmlttb_diag_wait_timeout(int which, void* workspace, size_t workspace_bytes,
                                        mmlttb_stream stream) {
  if (which != MMLTTB_DIAG_FUSED_BARRIER && which != MMLTTB_DIAG_GRID_BARRIER) return MMLTTB_EINVAL;
  if (!workspace || workspace_bytes < kHeader) return MMLTTB_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaMemsetAsync(workspace, 0, kHeader, st);
  if (e != cudaSuccess) return cuda_fail(e);
  Batch bt = {};
  bt.status = (unsigned*)workspace;
  bt.barrier = (unsigned*)((char*)workspace + 4);
  e = which == MMLTTB_DIAG_FUSED_BARRIER ? launch_sync_probe(bt, st) : launch_barrier_probe(bt, st);
  if (e != cudaSuccess) return cuda_fail(e);
  ++g_launches;
  return MMLTTB_OK;
}
