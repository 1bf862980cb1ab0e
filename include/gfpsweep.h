/*
 * libgfpsweep: host (CPU) implementations of the dot-product representations
 * that J.-G. Dumas, "Efficient dot product over word-size finite fields"
 * compares in its Section 3 (Figures 5-8), for timing sweeps over the modulus
 * on the host cores.  A measurement component: none of the gfp_* entry points
 * of libgfpdot calls it, and it is not a fallback for them.
 *
 * Every variant computes the exact residue (sum_i x_i y_i) mod p of canonical
 * inputs (0 <= x_i, y_i < p); representations other than the classical one
 * (centred, Montgomery, double) are converted into before and out of after
 * the timed dot products, as the paper excludes conversions from its timings.
 *
 * Errors: every function returns 0 on success, GFP_SWEEP_ERR_DOMAIN (-1) when
 * p lies outside the variant's domain (gfp_sweep_supported), and
 * GFP_SWEEP_ERR_ARG (-2) for a null pointer with n > 0, an unknown variant or
 * a failed allocation.  Inputs are not range-checked: entries >= p are outside
 * the contract.  Buffers belong to the caller; the library keeps no state.
 */
#ifndef GFPSWEEP_H
#define GFPSWEEP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    GFP_SWEEP_ERR_DOMAIN = -1,
    GFP_SWEEP_ERR_ARG = -2,
};

/* Variants.  "32" = the 32-bit unsigned machine word of the paper's Pentium III
 * experiments, "64" = 64-bit words, "53" = the double significand. */
typedef enum {
    /* Section 2.1: one remainder per term (Zpz AXPY); p(p-1) < 2^32 */
    GFP_SWEEP_ZPZ32 = 0,
    /* Section 3.2 blocked dot product: a remainder every lambda terms, with
     * lambda (p-1)^2 + (p-1) < 2^32 (the residue is carried, Eq. (2) form) */
    GFP_SWEEP_BLOCK32 = 1,
    /* Section 3.3 division on demand: add CORR = 2^32 mod p when t + ab < ab */
    GFP_SWEEP_OVERFLOW32 = 2,
    /* Section 3.4 hybrid (block-overflow): one wrap test per block of lambda
     * terms, lambda p (p-1) < 2^32 read as lambda (p-1)^2 + (p-1) < 2^32 */
    GFP_SWEEP_HYBRID32 = 3,
    /* Section 3.2.2 centred blocks in signed 32-bit words:
     * lambda ((p-1)/2)^2 + (p-1) <= 2^31 - 1 */
    GFP_SWEEP_CENTERED_BLOCK32 = 4,
    /* Section 3.3 signed overflow detection on centred values (two tests per
     * term), computed in unsigned arithmetic with explicit wrap tests */
    GFP_SWEEP_CENTERED_OVERFLOW32 = 5,
    /* Sections 2.2 and 3.2.1 Montgomery form aB mod p with B = 2^16 (half the
     * word): blocks of products reduced by one REDC each, lambda (p-1)^2 < pB;
     * odd p only */
    GFP_SWEEP_MONTGOMERY_BLOCK16 = 6,
    /* Section 2.1 with 64-bit words: one remainder per term */
    GFP_SWEEP_ZPZ64 = 7,
    /* Section 3.1 delayed division with 64-bit words (Eq. (2) carried form) */
    GFP_SWEEP_BLOCK64 = 8,
    /* Section 3.3 division on demand with CORR = 2^64 mod p */
    GFP_SWEEP_OVERFLOW64 = 9,
    /* Section 3.4 hybrid with 64-bit words */
    GFP_SWEEP_HYBRID64 = 10,
    /* Sections 2.3 and 3.1 doubles: exact integer sums below 2^53 reduced
     * every lambda terms by T - floor(T / p) p with a +-p fix-up */
    GFP_SWEEP_FP53_BLOCK = 11,
    /* Sections 2.2 and 3.2.1 Montgomery form with B = 2^32 in 64-bit words:
     * lambda (p-1)^2 < pB; odd p only */
    GFP_SWEEP_MONTGOMERY_BLOCK32 = 12,
    GFP_SWEEP_COUNT = 13
} gfp_sweep_variant;

/* Short name of a variant ("zpz32", "block32", ...), or NULL. */
const char *gfp_sweep_name(int variant);

/* 1 if the variant handles modulus p (2 <= p <= 2^32 - 1 and the variant's own
 * bound above), else 0. */
int gfp_sweep_supported(int variant, uint32_t p);

/* The variant's block length lambda for p (terms between reductions or wrap
 * tests; 1 for the per-term and overflow variants), 0 outside the domain. */
uint64_t gfp_sweep_block(int variant, uint32_t p);

/* One dot product of host vectors x, y (n entries each, canonical residues)
 * in the variant's representation; writes the canonical residue to *out. */
int gfp_sweep_dot(int variant, uint32_t p, uint64_t n, const uint32_t *x, const uint32_t *y,
                  uint32_t *out);

/* Converts x, y into the variant's representation once, then runs the dot
 * product `reps` times back to back on one host thread and reports the
 * wall-clock seconds of that loop (CLOCK_MONOTONIC) in *seconds and the
 * residue in *out.  reps >= 1. */
int gfp_sweep_time(int variant, uint32_t p, uint64_t n, const uint32_t *x, const uint32_t *y,
                   uint64_t reps, double *seconds, uint32_t *out);

#ifdef __cplusplus
}
#endif

#endif /* GFPSWEEP_H */
