/*
 * mmlttb_diag.h -- failure-detection diagnostics of libmmlttb.so (no counterpart in
 * the paper).  The library's device-side waits (the grid barriers of the fused
 * single-series kernel and of the grid-wide LTTB engine) are bounded: a wait that is
 * not satisfied within 2 s sets bit 1 of the workspace status word
 * (mmlttb_workspace_status) and the kernel returns, leaving the context usable.
 * The conventions of mmlttb.h hold.
 */
#ifndef MMLTTB_DIAG_H
#define MMLTTB_DIAG_H

#include "mmlttb.h"

#ifdef __cplusplus
extern "C" {
#endif

#define MMLTTB_DIAG_FUSED_BARRIER 0 /* the fused kernel's grid barrier */
#define MMLTTB_DIAG_GRID_BARRIER 1  /* the grid-wide LTTB engine's barrier */

/*
 * Run one barrier of kind `which` on a two-CTA launch in which the second CTA never
 * arrives, so the first CTA's wait runs out after its 2 s bound.  `workspace` is a
 * device buffer of at least 256 bytes whose first 256 bytes (the header) are cleared
 * first; afterwards mmlttb_workspace_status reports bit 1 (a wait timed out).
 * Asynchronous on `stream` (the kernel runs about 2 s).  MMLTTB_EINVAL for an unknown
 * `which`, a NULL workspace or fewer than 256 bytes.
 */
int mmlttb_diag_wait_timeout(int which, void *workspace, size_t workspace_bytes, mmlttb_stream stream);

#ifdef __cplusplus
}
#endif

#endif /* MMLTTB_DIAG_H */
