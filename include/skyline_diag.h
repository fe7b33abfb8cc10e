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

/* Runs the dominance engine's first test as a throughput loop on the
   context's device and stream: 128-thread CTAs, four per SM (as the engine
   runs), each lane holding four candidates' FP16 images (d = 6, duplicated
   per word) and scanning a staged shared-memory block two dominator pairs
   per step -- one f16x2 subtraction per attribute and candidate, the sign
   words OR-ed per test and AND-ed per step, a branch on the result -- the
   instruction sequence of the engine's scan when every test fails (a
   confirmation), about `iterations` x 512 tests per thread.
   *dim_compares_per_s receives the tests per second x 6 (the practical
   ceiling of the engine's compare loop); *sm_count the SMs used.  Blocks
   until done.  Errors: SKY_EINVAL (NULL outputs or iterations == 0),
   SKY_ENOMEM, SKY_ECUDA. */
sky_status sky_probe_reject_rate(sky_ctx* ctx, uint32_t iterations, double* dim_compares_per_s,
                                 uint32_t* sm_count);
/* Test hook of the engine's bounded waits (the paper has no counterpart; it
   exists so that a test can show that a device-side wait which never ends
   is turned into an error status without faulting or hanging the GPU).
   Arms the context's next sky_skyline / sky_skyline_ex / sky_skyline_batch
   call only (the call after it runs normally again): every wait of the
   persistent engine -- for a bulk copy, for a ticket's task, for a
   preceding tile's count -- gives up after wait_limit_ns nanoseconds
   without progress anywhere in the launch (instead of 4 s), and, when
   withhold_task >= 1, the withhold_task-th task that an engine launch of
   that call publishes keeps its tickets but is never marked published, so
   the CTAs that draw those tickets wait until the limit runs out.  The
   armed call then returns SKY_ETIMEOUT (or SKY_OK when the launch has
   fewer tasks); the context stays usable.  Errors: SKY_EINVAL (NULL
   context, wait_limit_ns below 1 ms). */
sky_status sky_diag_engine_wait_test(sky_ctx* ctx, uint64_t wait_limit_ns, uint32_t withhold_task);

#ifdef __cplusplus
}
#endif
#endif /* SKYLINE_DIAG_H_ */
