/*
 * awo_probe.h -- measurement kernels for the roofline of the particle kernel.
 *
 * The particle step of the avalanche workflow (Sec. 5.2) gathers a 2x2
 * height footprint and scatters two reductions per visit, into rasters that
 * are L2-resident at the working set of a persistent launch.  The relevant
 * ceilings are therefore the L2 throughput of scattered 4-byte loads and of
 * scattered 4-byte reductions, which no vendor table lists.  These kernels
 * measure them on the running GPU; the caller times each call with CUDA
 * events on `stream`.  Same conventions as awo.h (caller-owned device
 * buffers, asynchronous, status codes).
 */
#ifndef AWO_PROBE_H
#define AWO_PROBE_H

#include <stddef.h>
#include <stdint.h>

#include "awo.h"

#ifdef __cplusplus
extern "C" {
#endif

/*
 * Scattered loads: every thread of a persistent grid performs `iters`
 * rounds; each round loads 4 independent 4-byte words at hashed positions in
 * d_buf[0 .. n_words) (n_words a power of two, <= 2^30) and folds them into a
 * checksum, written to d_sink (one uint32 per thread of the grid, at least
 * awo_probe_threads() entries).  Loads issued: awo_probe_threads() * iters * 4.
 */
awo_status awo_probe_l2_gather(const uint32_t* d_buf, uint32_t n_words, uint32_t iters, uint32_t* d_sink,
                               void* stream);

/*
 * Scattered reductions: like the gather probe, but each round issues one
 * fire-and-forget 32-bit add (RED.ADD) and one 32-bit max (RED.MAX) at hashed
 * positions of d_buf.  Reductions issued: awo_probe_threads() * iters * 2.
 */
awo_status awo_probe_l2_red(uint32_t* d_buf, uint32_t n_words, uint32_t iters, void* stream);

/* Threads of the persistent probe grid on the current device. */
uint64_t awo_probe_threads(void);

/*
 * Self-test of the particle kernels' normalisation (a check of this library's
 * own arithmetic; the paper has no counterpart).  The kernels form
 * 1 / sqrt(x) as two correctly rounded steps, s = RN(sqrt x) and
 * r = RN(1 / s), with one hardware approximation each refined by Markstein's
 * method inside [2^-100, 2^100] and by the IEEE intrinsics outside it.  This
 * call compares that function with __frcp_rn(__fsqrt_rn(x)) bit for bit for
 * x = every FP32 bit pattern b in [first, first + count) except +0 and -0,
 * on the current device, and writes the number of mismatches to
 * *d_mismatches (device uint64, 8-byte aligned, overwritten; zero means the
 * particle kernels' directions are the IEEE ones on this GPU).  first = 0 and
 * count = 2^32 check every input.  Asynchronous on `stream`.
 * AWO_EINVAL: d_mismatches NULL or misaligned, or first + count > 2^32.
 */
awo_status awo_selftest_rcp_sqrt(uint32_t first, uint64_t count, uint64_t* d_mismatches, void* stream);

/*
 * Self-test of the particle kernels' visited cell (a check of this library's
 * own arithmetic; the paper has no counterpart).  A visit goes to the cell
 * whose centre is nearest, floor(u) + [u - floor(u) >= 1/2] per axis; the
 * kernels form it as floor(u + 1/2) with the sum rounded toward zero.  This
 * call compares the two for every FP32 bit pattern b in [first, first +
 * count) whose value lies in [0, 2^23) (others are skipped) and writes the
 * number of mismatches to *d_mismatches (as in awo_selftest_rcp_sqrt).
 * AWO_EINVAL: d_mismatches NULL or misaligned, or first + count > 2^32.
 */
awo_status awo_selftest_visit_cell(uint32_t first, uint64_t count, uint64_t* d_mismatches, void* stream);

/*
 * Self-test of the correctly rounded division of the compose pass (a check
 * of this library's own arithmetic; the paper has no counterpart).  The
 * colour ramp divides by each segment's width through its correctly rounded
 * reciprocal and two quotient corrections (Markstein's method) instead of
 * the IEEE division intrinsic, and so do the normals' central differences
 * (dividends of either sign).  For each of the n_divisors divisors b in
 * d_divisors (device, FP32; entries that are not positive and finite are
 * skipped), this call compares the two for every FP32 a whose bit pattern
 * lies in [bits(b) - span, bits(b)] (clamped at +0: span >= bits(b) covers
 * all of [0, b], span = 2^23 the binade below b), and for -a, and writes the
 * number of mismatches (bit patterns that differ) to *d_mismatches (device
 * uint64, 8-byte aligned; set to 0 first), in stream order.
 * AWO_EINVAL: d_divisors or d_mismatches NULL or misaligned, n_divisors = 0.
 */
awo_status awo_selftest_div_rn(const float* d_divisors, uint32_t n_divisors, uint32_t span, uint64_t* d_mismatches,
                               void* stream);

/*
 * Random words of the particle kernels (a check of this library's own
 * generator; Philox4x32-10 is defined by Salmon, Moraes, Dror and Shaw,
 * "Parallel Random Numbers: As Easy as 1, 2, 3", SC'11).  For i in [0, n):
 *   d_out[4i .. 4i+3] = Philox4x32-10(counter d_counters[4i .. 4i+3],
 *                                     key (seed low word, seed high word)),
 * computed on the current device by the device function that the particle
 * kernels draw their moves from (awo_simulate: counter (cell, j, n >> 1, 0)).
 * Round keys: weyl_keys == 0 takes them from a table filled on the host (the
 * single-request kernel's form), weyl_keys != 0 generates them in registers
 * by the Weyl schedule (the batched kernel's form when its requests have
 * different seeds).  d_counters and d_out: device uint32 [4n], 16-byte
 * aligned, caller-owned; d_out is overwritten.  Asynchronous on `stream`.
 * AWO_EINVAL: d_counters or d_out NULL or misaligned, or n < 0.
 */
awo_status awo_probe_philox(const uint32_t* d_counters, int64_t n, uint64_t seed, int32_t weyl_keys,
                            uint32_t* d_out, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* AWO_PROBE_H */
