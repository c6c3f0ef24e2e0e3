/*
 * mmlttb_diag.h -- diagnostics of libmmlttb.so (no counterpart in the paper):
 * failure detection and a precondition check.  The library's device-side waits (the grid barriers of the fused
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
#define MMLTTB_DIAG_GRID_BARRIER 1  /* the large-bucket LTTB engine's grid barrier */
#define MMLTTB_DIAG_MBARRIER 2      /* the staged MinMax stream's stage wait (mbarrier) */

/*
 * Run one wait of kind `which` that nothing satisfies: a grid barrier on a two-CTA
 * launch in which the second CTA never arrives, or an mbarrier that expects one
 * arrival that never comes (no copy is issued), so the wait runs out after its 2 s
 * bound.  `workspace` is a
 * device buffer of at least 256 bytes whose first 256 bytes (the header) are cleared
 * first; afterwards mmlttb_workspace_status reports bit 1 (a wait timed out).
 * Asynchronous on `stream` (the kernel runs about 2 s).  MMLTTB_EINVAL for an unknown
 * `which`, a NULL workspace or fewer than 256 bytes.
 */
int mmlttb_diag_wait_timeout(int which, void *workspace, size_t workspace_bytes, mmlttb_stream stream);

/* Bits of mmlttb_check_series. */
#define MMLTTB_CHECK_Y_NAN 0x1       /* y holds a NaN (MinMaxLTTB, LTTB and plain MinMax
                                        then return unspecified indices) */
#define MMLTTB_CHECK_X_DECREASES 0x2 /* x[i+1] < x[i] for some i (x must be non-decreasing) */
#define MMLTTB_CHECK_X_NONFINITE 0x4 /* float64 x holds NaN or +-inf */

/*
 * Check the documented preconditions of a series (mmlttb.h) on the device: one
 * read of y and x.  *flags (device uint32) is overwritten with the MMLTTB_CHECK_*
 * bits of the violations found (0: none).  x is ignored for MMLTTB_X_IMPLICIT.
 * MMLTTB_EINVAL for a NULL y (n_in > 0) or flags, a NULL x that is not implicit, bad
 * enums or n_in < 0.
 */
int mmlttb_check_series(const void *y, int ydtype, const void *x, int xkind, int64_t n_in, uint32_t *flags,
                        mmlttb_stream stream);

#ifdef __cplusplus
}
#endif

#endif /* MMLTTB_DIAG_H */
