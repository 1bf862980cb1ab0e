/*
 * Host (CPU) implementations of the dot-product representations compared in
 * Section 3 of J.-G. Dumas, "Efficient dot product over word-size finite
 * fields" (Figures 5-8), used to time sweeps over the modulus on the host
 * cores.  Interface and contracts: include/gfpsweep.h.
 *
 * Plain C, no intrinsics and no -march, so that it builds and behaves the same
 * on x86-64 and on Arm.  Each dot-product routine is compiled `noipa` so that
 * a timing loop cannot hoist a call with unchanged arguments.
 */
#define _POSIX_C_SOURCE 199309L   /* clock_gettime under -std=c11 */
#include "gfpsweep.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#include <time.h>

#define NOIPA __attribute__((noipa))

/* ---------------- parameters ---------------- */

static uint64_t pm1sq(uint32_t p) { return (uint64_t)(p - 1) * (uint64_t)(p - 1); }

/* largest lambda with lambda (p-1)^2 + (p-1) <= limit (p >= 2); the residue
 * carried from block to block is at most p - 1 (Eq. (2) form) */
static uint64_t lambda_carried(uint32_t p, uint64_t limit)
{
    const uint64_t sq = pm1sq(p);
    if (sq == 0) return UINT64_MAX;           /* p = 1 is rejected earlier */
    if (limit < (uint64_t)(p - 1)) return 0;
    return (limit - (uint64_t)(p - 1)) / sq;
}

/* magnitude bound of centred values: a > (p-1)/2 maps to a - p, so the
 * largest magnitude is floor(p/2) */
static uint64_t centred_max(uint32_t p) { return (uint64_t)(p / 2); }

static uint64_t lambda_centred32(uint32_t p)
{
    const uint64_t h = centred_max(p), lim = 2147483647ull;   /* 2^31 - 1 */
    if (h == 0) return UINT64_MAX;
    if (h * h + (uint64_t)(p - 1) > lim) return 0;
    return (lim - (uint64_t)(p - 1)) / (h * h);
}

static uint64_t lambda_mont16(uint32_t p)
{
    /* lambda (p-1)^2 <= p 2^16 - 1 keeps every block sum a valid REDC input */
    if ((p & 1u) == 0 || p < 3 || p > 65535u) return 0;
    return (((uint64_t)p << 16) - 1) / pm1sq(p);
}

static uint64_t lambda_mont32(uint32_t p)
{
    if ((p & 1u) == 0 || p < 3) return 0;
    return (((uint64_t)p << 32) - 1) / pm1sq(p);
}

static uint64_t lambda_fp53(uint32_t p)
{
    return lambda_carried(p, 9007199254740992ull);           /* 2^53 */
}

static const char *const NAMES[GFP_SWEEP_COUNT] = {
    "zpz32",    "block32", "overflow32", "hybrid32", "centered_block32", "centered_overflow32",
    "montgomery_block16", "zpz64", "block64", "overflow64", "hybrid64", "fp53_block",
    "montgomery_block32"};

const char *gfp_sweep_name(int v) { return (v >= 0 && v < GFP_SWEEP_COUNT) ? NAMES[v] : NULL; }

uint64_t gfp_sweep_block(int v, uint32_t p)
{
    if (p < 2) return 0;
    switch (v) {
    case GFP_SWEEP_ZPZ32:
    case GFP_SWEEP_OVERFLOW32:
        /* the AXPY value r + ab <= p (p - 1) must fit 32 bits */
        return ((uint64_t)p * (uint64_t)(p - 1) <= 0xFFFFFFFFull) ? 1 : 0;
    case GFP_SWEEP_BLOCK32:
    case GFP_SWEEP_HYBRID32:
        return lambda_carried(p, 0xFFFFFFFFull);
    case GFP_SWEEP_CENTERED_BLOCK32:
        return lambda_centred32(p);
    case GFP_SWEEP_CENTERED_OVERFLOW32:
        return lambda_centred32(p) ? 1 : 0;
    case GFP_SWEEP_MONTGOMERY_BLOCK16:
        return lambda_mont16(p);
    case GFP_SWEEP_ZPZ64:
    case GFP_SWEEP_OVERFLOW64:
        return 1;
    case GFP_SWEEP_BLOCK64:
    case GFP_SWEEP_HYBRID64:
        return lambda_carried(p, 0xFFFFFFFFFFFFFFFFull);
    case GFP_SWEEP_FP53_BLOCK:
        return lambda_fp53(p);
    case GFP_SWEEP_MONTGOMERY_BLOCK32:
        return lambda_mont32(p);
    default:
        return 0;
    }
}

int gfp_sweep_supported(int v, uint32_t p) { return gfp_sweep_block(v, p) > 0 ? 1 : 0; }

/* -p^{-1} mod 2^bits for odd p (Newton: each step doubles the correct low bits) */
static uint32_t neg_inv_pow2(uint32_t p, int bits)
{
    uint32_t inv = p;                       /* correct to 3 bits: p p = 1 mod 8 */
    for (int i = 0; i < 5; ++i) inv *= 2u - p * inv;
    const uint32_t r = 0u - inv;
    return bits == 32 ? r : (r & 0xFFFFu);
}

/* end of the block that starts at i (lam may be close to 2^64 for tiny p, so
 * i + lam is not formed when it could wrap) */
static uint64_t block_end(uint64_t i, uint64_t lam, uint64_t n) { return lam >= n - i ? n : i + lam; }

/* ---------------- 32-bit words ---------------- */

/* Section 2.1: r <- (r + x_i y_i) mod p every term */
NOIPA static uint32_t dot_zpz32(uint32_t p, uint64_t n, const uint32_t *x, const uint32_t *y)
{
    uint32_t r = 0;
    for (uint64_t i = 0; i < n; ++i) r = (r + x[i] * y[i]) % p;
    return r;
}

/* Section 3.2: lam terms, then one remainder */
NOIPA static uint32_t dot_block32(uint32_t p, uint64_t lam, uint64_t n, const uint32_t *x,
                                  const uint32_t *y)
{
    uint32_t r = 0;
    uint64_t i = 0;
    while (i < n) {
        const uint64_t end = block_end(i, lam, n);
        for (; i < end; ++i) r += x[i] * y[i];
        r %= p;
    }
    return r;
}

/* Section 3.3: a wrap of t + ab shows as t + ab < ab; it stands for 2^32 = CORR */
NOIPA static uint32_t dot_overflow32(uint32_t p, uint32_t corr, uint64_t n, const uint32_t *x,
                                     const uint32_t *y)
{
    uint32_t s = 0;
    for (uint64_t i = 0; i < n; ++i) {
        const uint32_t pr = x[i] * y[i];
        s += pr;
        if (s < pr) s += corr;
    }
    return s % p;
}

/* Section 3.4: lam products (sum < 2^32) wrap a block at most once; one test
 * per block, and CORR added after a wrap cannot wrap again by the bound */
NOIPA static uint32_t dot_hybrid32(uint32_t p, uint32_t corr, uint64_t lam, uint64_t n,
                                   const uint32_t *x, const uint32_t *y)
{
    uint32_t s = 0;
    uint64_t i = 0;
    while (i < n) {
        const uint64_t end = block_end(i, lam, n);
        const uint32_t s0 = s;
        for (; i < end; ++i) s += x[i] * y[i];
        if (s < s0) s += corr;
    }
    return s % p;
}

/* Section 3.2.2: centred values, signed blocks; C's remainder keeps the sign,
 * so the carried residue lies in (-p, p) */
NOIPA static int32_t dot_centred_block32(int32_t p, uint64_t lam, uint64_t n, const int32_t *x,
                                         const int32_t *y)
{
    int32_t r = 0;
    uint64_t i = 0;
    while (i < n) {
        const uint64_t end = block_end(i, lam, n);
        for (; i < end; ++i) r += x[i] * y[i];
        r %= p;
    }
    return r;
}

/* Section 3.3 on centred values: the running sum is a 32-bit two's-complement
 * word; a positive product that turns a non-negative sum negative wrapped
 * past 2^31 (add CORR = 2^32 mod p), a negative product that turns a negative
 * sum non-negative wrapped the other way (subtract CORR).  Kept in unsigned
 * arithmetic, so no signed overflow occurs. */
NOIPA static uint32_t dot_centred_overflow32(uint32_t corr, uint64_t n, const int32_t *x,
                                             const int32_t *y)
{
    uint32_t s = 0;
    for (uint64_t i = 0; i < n; ++i) {
        const int32_t pr = x[i] * y[i];
        const uint32_t t = s + (uint32_t)pr;
        if (pr > 0) {
            if (!(s >> 31) && (t >> 31)) s = t + corr;
            else s = t;
        } else if (pr < 0) {
            if ((s >> 31) && !(t >> 31)) s = t - corr;
            else s = t;
        }
    }
    return s;
}

/* REDC with B = 2^16 for T < p B: (T + U p) / B with U = T n' mod B, computed
 * as high parts so that nothing exceeds 32 bits; result < 2p, = T B^-1 mod p */
static inline uint32_t redc16(uint32_t T, uint32_t p, uint32_t nprime)
{
    const uint32_t lo = T & 0xFFFFu;
    const uint32_t U = (lo * nprime) & 0xFFFFu;
    return (T >> 16) + ((lo + U * p) >> 16);
}

/* Sections 2.2, 3.2.1: elements stored as aB mod p; a product of two is abB^2,
 * so the products of a block add up before one REDC brings the block to the
 * form (sum) B; the block results add up as well */
NOIPA static uint32_t dot_mont16(uint32_t p, uint32_t nprime, uint64_t lam, uint64_t n,
                                 const uint32_t *xm, const uint32_t *ym)
{
    uint64_t acc = 0;
    uint64_t i = 0;
    while (i < n) {
        const uint64_t end = block_end(i, lam, n);
        uint32_t T = 0;
        for (; i < end; ++i) T += xm[i] * ym[i];
        acc += redc16(T, p, nprime);
    }
    return (uint32_t)(acc % p);   /* the dot product in Montgomery form */
}

/* ---------------- 64-bit words ---------------- */

NOIPA static uint32_t dot_zpz64(uint32_t p, uint64_t n, const uint32_t *x, const uint32_t *y)
{
    uint64_t r = 0;
    for (uint64_t i = 0; i < n; ++i) r = (r + (uint64_t)x[i] * y[i]) % p;
    return (uint32_t)r;
}

NOIPA static uint32_t dot_block64(uint32_t p, uint64_t lam, uint64_t n, const uint32_t *x,
                                  const uint32_t *y)
{
    uint64_t r = 0;
    uint64_t i = 0;
    while (i < n) {
        const uint64_t end = block_end(i, lam, n);
        for (; i < end; ++i) r += (uint64_t)x[i] * y[i];
        r %= p;
    }
    return (uint32_t)r;
}

NOIPA static uint32_t dot_overflow64(uint32_t p, uint64_t corr, uint64_t n, const uint32_t *x,
                                     const uint32_t *y)
{
    uint64_t s = 0;
    for (uint64_t i = 0; i < n; ++i) {
        const uint64_t pr = (uint64_t)x[i] * y[i];
        s += pr;
        if (s < pr) s += corr;
    }
    return (uint32_t)(s % p);
}

NOIPA static uint32_t dot_hybrid64(uint32_t p, uint64_t corr, uint64_t lam, uint64_t n,
                                   const uint32_t *x, const uint32_t *y)
{
    uint64_t s = 0;
    uint64_t i = 0;
    while (i < n) {
        const uint64_t end = block_end(i, lam, n);
        const uint64_t s0 = s;
        for (; i < end; ++i) s += (uint64_t)x[i] * y[i];
        if (s < s0) s += corr;
    }
    return (uint32_t)(s % p);
}

/* Sections 2.3, 3.1: integer sums in doubles stay exact below 2^53; every lam
 * terms T <- T - floor(T / p) p (the quotient from a precomputed 1/p), then
 * the +-p fix-up for a quotient off by one.  T - q p is taken with one fused
 * multiply-add: its exact value is below 2p in magnitude, so the fma returns
 * it exactly even where q p itself would round above 2^53. */
static inline double fp_reduce(double T, double P, double invP)
{
    const double q = floor(T * invP);
    double r = fma(-q, P, T);
    if (r >= P) r -= P;
    else if (r < 0) r += P;
    return r;
}

NOIPA static uint32_t dot_fp53(double P, double invP, uint64_t lam, uint64_t n, const double *x,
                               const double *y)
{
    double T = 0.0;
    uint64_t i = 0;
    while (i < n) {
        const uint64_t end = block_end(i, lam, n);
        for (; i < end; ++i) T += x[i] * y[i];
        T = fp_reduce(T, P, invP);
    }
    return (uint32_t)T;
}

/* REDC with B = 2^32 for T < p B, as high parts of 64-bit values; result < 2p */
static inline uint64_t redc32(uint64_t T, uint32_t p, uint32_t nprime)
{
    const uint32_t lo = (uint32_t)T;
    const uint32_t U = lo * nprime;
    return (T >> 32) + (((uint64_t)U * p + lo) >> 32);
}

NOIPA static uint32_t dot_mont32(uint32_t p, uint32_t nprime, uint64_t lam, uint64_t n,
                                 const uint32_t *xm, const uint32_t *ym)
{
    uint64_t acc = 0;
    uint64_t i = 0;
    while (i < n) {
        const uint64_t end = block_end(i, lam, n);
        uint64_t T = 0;
        for (; i < end; ++i) T += (uint64_t)xm[i] * ym[i];
        acc += redc32(T, p, nprime);
    }
    return (uint32_t)(acc % p);
}

/* ---------------- conversions and dispatch ---------------- */

typedef struct {
    int v;
    uint32_t p;
    uint64_t lam;
    uint32_t corr32;
    uint64_t corr64;
    uint32_t nprime;
    double P, invP;
    uint64_t n;
    const uint32_t *x, *y;      /* caller's canonical residues */
    void *cx, *cy;              /* converted copies (centred, Montgomery, double) */
} prepared;

static void release(prepared *w)
{
    free(w->cx);
    free(w->cy);
    w->cx = w->cy = NULL;
}

static int prepare(prepared *w, int v, uint32_t p, uint64_t n, const uint32_t *x, const uint32_t *y)
{
    memset(w, 0, sizeof *w);
    if (v < 0 || v >= GFP_SWEEP_COUNT) return GFP_SWEEP_ERR_ARG;
    if (n > 0 && (!x || !y)) return GFP_SWEEP_ERR_ARG;
    if (!gfp_sweep_supported(v, p)) return GFP_SWEEP_ERR_DOMAIN;
    w->v = v;
    w->p = p;
    w->n = n;
    w->x = x;
    w->y = y;
    w->lam = gfp_sweep_block(v, p);
    w->corr32 = (uint32_t)((1ull << 32) % p);
    w->corr64 = (uint64_t)((0xFFFFFFFFFFFFFFFFull % p + 1) % p);
    const size_t cnt = n ? (size_t)n : 1;
    switch (v) {
    case GFP_SWEEP_CENTERED_BLOCK32:
    case GFP_SWEEP_CENTERED_OVERFLOW32: {
        int32_t *a = malloc(cnt * sizeof *a), *b = malloc(cnt * sizeof *b);
        w->cx = a;
        w->cy = b;
        if (!a || !b) {
            release(w);
            return GFP_SWEEP_ERR_ARG;
        }
        const uint32_t half = (p - 1) / 2;
        for (uint64_t i = 0; i < n; ++i) {
            a[i] = x[i] > half ? (int32_t)x[i] - (int32_t)p : (int32_t)x[i];
            b[i] = y[i] > half ? (int32_t)y[i] - (int32_t)p : (int32_t)y[i];
        }
        break;
    }
    case GFP_SWEEP_MONTGOMERY_BLOCK16:
    case GFP_SWEEP_MONTGOMERY_BLOCK32: {
        const int sh = v == GFP_SWEEP_MONTGOMERY_BLOCK16 ? 16 : 32;
        uint32_t *a = malloc(cnt * sizeof *a), *b = malloc(cnt * sizeof *b);
        w->cx = a;
        w->cy = b;
        if (!a || !b) {
            release(w);
            return GFP_SWEEP_ERR_ARG;
        }
        w->nprime = neg_inv_pow2(p, sh);
        for (uint64_t i = 0; i < n; ++i) {
            a[i] = (uint32_t)(((uint64_t)x[i] << sh) % p);
            b[i] = (uint32_t)(((uint64_t)y[i] << sh) % p);
        }
        break;
    }
    case GFP_SWEEP_FP53_BLOCK: {
        double *a = malloc(cnt * sizeof *a), *b = malloc(cnt * sizeof *b);
        w->cx = a;
        w->cy = b;
        if (!a || !b) {
            release(w);
            return GFP_SWEEP_ERR_ARG;
        }
        for (uint64_t i = 0; i < n; ++i) {
            a[i] = (double)x[i];
            b[i] = (double)y[i];
        }
        w->P = (double)p;
        w->invP = 1.0 / (double)p;
        break;
    }
    default:
        break;
    }
    return 0;
}

/* one dot product in the prepared representation; the result in that
 * representation (Montgomery form, signed centred value, ...) */
static uint64_t run_raw(const prepared *w)
{
    const uint32_t p = w->p;
    switch (w->v) {
    case GFP_SWEEP_ZPZ32: return dot_zpz32(p, w->n, w->x, w->y);
    case GFP_SWEEP_BLOCK32: return dot_block32(p, w->lam, w->n, w->x, w->y);
    case GFP_SWEEP_OVERFLOW32: return dot_overflow32(p, w->corr32, w->n, w->x, w->y);
    case GFP_SWEEP_HYBRID32: return dot_hybrid32(p, w->corr32, w->lam, w->n, w->x, w->y);
    case GFP_SWEEP_CENTERED_BLOCK32:
        return (uint64_t)(uint32_t)dot_centred_block32((int32_t)p, w->lam, w->n, w->cx, w->cy);
    case GFP_SWEEP_CENTERED_OVERFLOW32: return dot_centred_overflow32(w->corr32, w->n, w->cx, w->cy);
    case GFP_SWEEP_MONTGOMERY_BLOCK16: return dot_mont16(p, w->nprime, w->lam, w->n, w->cx, w->cy);
    case GFP_SWEEP_ZPZ64: return dot_zpz64(p, w->n, w->x, w->y);
    case GFP_SWEEP_BLOCK64: return dot_block64(p, w->lam, w->n, w->x, w->y);
    case GFP_SWEEP_OVERFLOW64: return dot_overflow64(p, w->corr64, w->n, w->x, w->y);
    case GFP_SWEEP_HYBRID64: return dot_hybrid64(p, w->corr64, w->lam, w->n, w->x, w->y);
    case GFP_SWEEP_FP53_BLOCK: return dot_fp53(w->P, w->invP, w->lam, w->n, w->cx, w->cy);
    case GFP_SWEEP_MONTGOMERY_BLOCK32: return dot_mont32(p, w->nprime, w->lam, w->n, w->cx, w->cy);
    default: return 0;
    }
}

/* the canonical residue of a raw result */
static uint32_t to_canonical(const prepared *w, uint64_t raw)
{
    const uint32_t p = w->p;
    switch (w->v) {
    case GFP_SWEEP_CENTERED_BLOCK32:
    case GFP_SWEEP_CENTERED_OVERFLOW32: {
        const int64_t s = (int64_t)(int32_t)(uint32_t)raw;   /* the two's-complement word */
        int64_t r = s % (int64_t)p;
        if (r < 0) r += p;
        return (uint32_t)r;
    }
    case GFP_SWEEP_MONTGOMERY_BLOCK16: {
        uint32_t r = redc16((uint32_t)raw, p, w->nprime);     /* (dot B) B^-1 */
        return r >= p ? r - p : r;
    }
    case GFP_SWEEP_MONTGOMERY_BLOCK32: {
        uint64_t r = redc32(raw, p, w->nprime);
        return (uint32_t)(r >= p ? r - p : r);
    }
    default:
        return (uint32_t)raw;
    }
}

int gfp_sweep_dot(int v, uint32_t p, uint64_t n, const uint32_t *x, const uint32_t *y, uint32_t *out)
{
    if (!out) return GFP_SWEEP_ERR_ARG;
    prepared w;
    const int st = prepare(&w, v, p, n, x, y);
    if (st) return st;
    *out = to_canonical(&w, run_raw(&w));
    release(&w);
    return 0;
}

static double now_seconds(void)
{
    struct timespec ts;
    clock_gettime(CLOCK_MONOTONIC, &ts);
    return (double)ts.tv_sec + 1e-9 * (double)ts.tv_nsec;
}

int gfp_sweep_time(int v, uint32_t p, uint64_t n, const uint32_t *x, const uint32_t *y,
                   uint64_t reps, double *seconds, uint32_t *out)
{
    if (!seconds || !out || reps == 0) return GFP_SWEEP_ERR_ARG;
    prepared w;
    const int st = prepare(&w, v, p, n, x, y);
    if (st) return st;
    volatile uint64_t sink = 0;
    uint64_t raw = run_raw(&w);   /* warm caches and branch predictors */
    const double t0 = now_seconds();
    for (uint64_t r = 0; r < reps; ++r) {
        raw = run_raw(&w);
        sink = sink + raw;
    }
    *seconds = now_seconds() - t0;
    *out = to_canonical(&w, raw);
    release(&w);
    return 0;
}
