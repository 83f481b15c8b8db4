/*
 * fcirc_prof.h -- launch tracing of the f-circulant library.
 *
 * While tracing is on, every kernel the library launches is bracketed by two
 * CUDA events recorded on the stream it is launched on, so per-kernel device
 * time can be read back without a profiler.  The paper has no counterpart
 * (its timings are wall-clock minima, Section 3.1); this is measurement
 * plumbing for the kernels of the C ABI in fcirc.h.
 *
 * Events are recorded only between fcirc_prof_start() and fcirc_prof_stop();
 * tracing must be off while a stream is captured into a CUDA graph.  The
 * copies that stage host arguments are traced too, as "copy_h2d" and
 * "copy_d2h" (they are not kernel launches).
 */
#ifndef FCIRC_PROF_H
#define FCIRC_PROF_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Clears previous records and turns tracing on (all threads, all devices). */
int fcirc_prof_start(void);

/* Turns tracing off; records are kept until the next fcirc_prof_start(). */
int fcirc_prof_stop(void);

/* Waits for the recorded events and writes one line per kernel name,
 *   "<name> <launches> <total_ms>\n",
 * into buf (NUL-terminated, truncated to len bytes).  Returns FCIRC_OK or an
 * fcirc_status code. */
int fcirc_prof_report(char *buf, uint64_t len);

/* Number of records (kernel launches and staging copies) since
 * fcirc_prof_start(). */
uint64_t fcirc_prof_launches(void);

/*
 * Measures the SM's integer-multiply throughput, the unit that bounds the
 * modular kernels (each butterfly is one Shoup product: a high-half and two
 * low-half 32-bit multiplies).  Launches ctas_per_sm (1..8) CTAs of 256
 * threads per SM of the current device; every thread runs 16 independent
 * chains of `iters` multiplies of one kind (kind 0: low-half v * a + b;
 * kind 1: high-half hi(v * a) + b), so the multiply pipe and not latency sets
 * the rate.  Times five launches with CUDA events on a stream of its own
 * (synchronising) and writes the fastest launch's time in *ms and its rate
 * in multiplies per second in *mul_per_s.  Allocates and frees a 1 KiB
 * sink.  Returns FCIRC_OK, FCIRC_EINVAL (bad arguments), FCIRC_ENOMEM or
 * FCIRC_ECUDA.
 */
int fcirc_prof_mul_probe(int kind, uint32_t ctas_per_sm, uint32_t iters, double *ms, double *mul_per_s);

#ifdef __cplusplus
}
#endif

#endif /* FCIRC_PROF_H */
