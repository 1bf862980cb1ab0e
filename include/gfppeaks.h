/*
 * libgfppeaks — the hardware ceilings that the rooflines of libgfpdot are
 * stated against, measured by this project's own kernels on the GPU in use.
 *
 * A measurement component, not part of the dot-product library: no gfp_*
 * entry point of libgfpdot calls it and libgfpdot does not contain it.  The
 * paper has no counterpart (its timings are on CPUs).  Each probe allocates
 * its own device buffers with cudaMalloc, runs `reps` timed launches after
 * two warm-up launches on a stream of its own, synchronises, frees what it
 * allocated and returns.  Timing is by CUDA events around each launch.
 *
 * Probes (`kind`):
 *  GFP_PEAK_READ_HBM   read-only stream of `bytes` (rounded down to a
 *                      multiple of 16; use several times the L2 size) with
 *                      16-byte streaming loads, eight in flight per thread,
 *                      one persistent CTA set per SM: the ceiling of a
 *                      kernel that only reads, like the dot products
 *                      (8 bytes read per multiply-add).  rate = GB/s.
 *  GFP_PEAK_COPY_HBM   copy of bytes/2 into another bytes/2 (read + write
 *                      counted): the same kind of figure as a device copy.
 *                      rate = GB/s.
 *  GFP_PEAK_READ_L2    `bytes` (choose well below the L2 size) read 64 times
 *                      per launch with loads that bypass L1 (ld.global.cg),
 *                      after one untimed pass has brought them into L2.
 *                      rate = GB/s from L2 to the SMs.
 *  GFP_PEAK_DFMA       independent chains of double-precision fma per
 *                      thread, every SM full: rate = TFLOP/s (2 per fma).
 *                      The floating-point representation's loop is one
 *                      fma per multiply-add (Section 3.1, m = 53).
 *  GFP_PEAK_IMMA_SYNC  warp-level mma.sync m16n8k32 with signed 8-bit
 *                      operands and 32-bit accumulators (the pre-tcgen05
 *                      integer tensor path), four accumulator chains per
 *                      warp, every SM full: rate = TOP/s (2 per multiply-add).
 *  GFP_PEAK_LAUNCH     `reps` empty launches captured in one CUDA graph and
 *                      replayed: rate = microseconds per launch (the floor
 *                      of any one-launch-per-call entry point in a graph).
 *
 * Errors: GFP_PEAK_ERR_ARG for an unknown kind, a NULL result, reps < 1 or
 * bytes too small for the probe; GFP_PEAK_ERR_CUDA when a CUDA call fails
 * (allocation included).  Nothing is left allocated on error.
 */
#ifndef GFPPEAKS_H
#define GFPPEAKS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    GFP_PEAK_READ_HBM = 0,
    GFP_PEAK_COPY_HBM = 1,
    GFP_PEAK_READ_L2 = 2,
    GFP_PEAK_DFMA = 3,
    GFP_PEAK_IMMA_SYNC = 4,
    GFP_PEAK_LAUNCH = 5,
    GFP_PEAK_KINDS_ = 6
};

enum { GFP_PEAK_OK = 0, GFP_PEAK_ERR_ARG = -1, GFP_PEAK_ERR_CUDA = -2 };

typedef struct gfp_peak_result {
    double rate;        /* best launch: GB/s, TFLOP/s, TOP/s or us per launch (see kind) */
    double rate_median; /* median launch, same unit */
    double ms_best;     /* fastest launch, milliseconds */
    double ms_median;   /* median launch, milliseconds */
    double work;        /* bytes, flops or ops per launch (launches for GFP_PEAK_LAUNCH) */
    int grid;           /* CTAs per launch */
    int threads;        /* threads per CTA */
} gfp_peak_result;

/* Run probe `kind` on the current device (see above).  `bytes` is ignored by
 * the arithmetic and launch probes. */
int gfp_peak_measure(int kind, uint64_t bytes, int reps, gfp_peak_result *out);

/* Static name of a probe kind ("read_hbm", ...), or NULL if unknown. */
const char *gfp_peak_name(int kind);

#ifdef __cplusplus
}
#endif

#endif
