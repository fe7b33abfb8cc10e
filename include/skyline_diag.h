/*
 * skyline_diag.h -- measurement entry points of libskyline (not part of the
 * skyline method itself; the paper has no counterpart).
 *
 * The dominance kernels of the library are bound by FP32 comparisons
 * (Def. 1 of Section 2 tests t[A] <= s[A] per attribute), not by tensor
 * cores or memory.  There is no published comparison-throughput figure for
 * the GPU, so the roofline denominator of those kernels is measured here.
 */
#ifndef SKYLINE_DIAG_H_
#define SKYLINE_DIAG_H_

#include <stdint.h>
#include "skyline.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Runs a register-only kernel on the context's device and stream whose
   inner loop is FP32 compares accumulated into predicates (the instruction
   form of a dominance test), on every SM at full occupancy, for about
   `iterations` x 64 compares per thread.  *compares_per_s receives the
   measured FP32 compares per second of the whole GPU; *sm_count the number
   of SMs used.  Blocks until done.  Errors: SKY_EINVAL (NULL outputs or
   iterations == 0), SKY_ECUDA. */
sky_status sky_probe_compare_rate(sky_ctx* ctx, uint32_t iterations, double* compares_per_s,
                                  uint32_t* sm_count);

#ifdef __cplusplus
}
#endif
#endif /* SKYLINE_DIAG_H_ */
