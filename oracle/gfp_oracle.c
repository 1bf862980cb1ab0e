/*
 * Oracle for the exact dot product over a word-size prime field GF(p).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the library calls, links or loads
 * this file; only the tests, the smoke check and the CPU-baseline leg of the
 * benchmark do.  It shares no code with the CUDA path.
 *
 * Definition implemented (the plain one, since every delayed-reduction method
 * of the paper reaches exactly the same residue):
 *
 *      dot(x, y) = ( sum_{i<n} x_i * y_i ) mod p,   result in [0, p)
 *
 * computed term by term in the paper's classical "Zpz" representation
 * (Section 2.1): residues in [0, p), and AXPY  r <- (r + x_i*y_i) mod p  is one
 * machine multiplication, one machine addition and one machine remainder.
 * Overflow argument: inputs are canonical (x_i, y_i < p) and p <= 2^32-1, so
 * r + x_i*y_i <= (p-1) + (p-1)^2 = p(p-1) < 2^64: the unsigned 64-bit Zpz
 * limit of Section 2.1 (largest admissible prime 4294967291).
 *
 * Derived products (matrix-vector, block and sparse-row block) apply the same
 * per-term definition to each output entry; the iterative matrix-vector use is
 * the Wiedemann-style iteration the introduction names as a consumer of the
 * dot product.
 *
 * Restatements of the paper's own dot-product variants (blocked delayed
 * division, Section 3.2; division on demand by overflow detection,
 * Section 3.3; floating-point reduction, Section 2.3) are included as separate
 * functions so that tests can check them against the plain definition; they
 * are written from the descriptions, with bounds from Eq. (1) and Eq. (2).
 *
 * Finite fields GF(p^k) (Section 2.4: the discrete-logarithm representation
 * and field extensions): field addition, multiplication and the term-by-term
 * field dot product in GF(p)[x]/(f), at the end of this file.
 *
 * Parity status: every function here is pinned by tests against arbitrary
 * precision brute force, closed forms, invariants and, for GF(2^8), the
 * worked examples published in FIPS 197 (no function is "parity unpinned").
 */
#include <stdint.h>
#include <stddef.h>
#include <math.h>

/* Zpz AXPY (Section 2.1): one multiply, one add, one remainder. */
static inline uint64_t zpz_axpy(uint64_t r, uint32_t a, uint32_t b, uint64_t p)
{
    return (r + (uint64_t)a * (uint64_t)b) % p;
}

/* dot(x, y) mod p, term by term. */
uint32_t oracle_dot(uint32_t p, uint64_t n, const uint32_t *x, const uint32_t *y)
{
    uint64_t r = 0;
    for (uint64_t i = 0; i < n; ++i)
        r = zpz_axpy(r, x[i], y[i], p);
    return (uint32_t)r;
}

/* Strided form: dot over x[i*incx], y[i*incy]. */
uint32_t oracle_dot_strided(uint32_t p, uint64_t n, const uint32_t *x, uint64_t incx,
                            const uint32_t *y, uint64_t incy)
{
    uint64_t r = 0;
    for (uint64_t i = 0; i < n; ++i)
        r = zpz_axpy(r, x[i * incx], y[i * incy], p);
    return (uint32_t)r;
}

/* count independent pairs packed in flat buffers: pair j is
 * x[off[j] .. off[j]+n[j]) and y[...] with prime p[j]; out[j] its residue. */
void oracle_dot_batch(uint64_t count, const uint32_t *p, const uint64_t *n,
                      const uint64_t *off, const uint32_t *x, const uint32_t *y,
                      uint32_t *out)
{
    for (uint64_t j = 0; j < count; ++j)
        out[j] = oracle_dot(p[j], n[j], x + off[j], y + off[j]);
}

/* y_i = sum_j A[i*lda + j] * x_j mod p, for rows r0 <= i < r1. */
void oracle_matvec_rows(uint32_t p, uint64_t r0, uint64_t r1, uint64_t cols,
                        const uint32_t *A, uint64_t lda, const uint32_t *x, uint32_t *y)
{
    for (uint64_t i = r0; i < r1; ++i)
        y[i] = oracle_dot(p, cols, A + i * lda, x);
}

/* C[i*ldc + j] = sum_t A[i*lda + t] * B[t*ldb + j] mod p, rows r0 <= i < r1,
 * all nb columns.  A is m x k row-major, B is k x nb row-major. */
void oracle_block_rows(uint32_t p, uint64_t r0, uint64_t r1, uint64_t k, uint64_t nb,
                       const uint32_t *A, uint64_t lda, const uint32_t *B, uint64_t ldb,
                       uint32_t *C, uint64_t ldc)
{
    for (uint64_t i = r0; i < r1; ++i)
        for (uint64_t j = 0; j < nb; ++j)
            C[i * ldc + j] = oracle_dot_strided(p, k, A + i * lda, 1, B + j, ldb);
}

/* Sparse-row (CSR) block product: row i has nonzeros val[q] at columns col[q]
 * for row_ptr[i] <= q < row_ptr[i+1]; C[i*ldc + j] = sum_q val[q]*B[col[q]*ldb + j]. */
void oracle_csr_rows(uint32_t p, uint64_t r0, uint64_t r1, uint64_t nb,
                     const uint32_t *row_ptr, const uint32_t *col, const uint32_t *val,
                     const uint32_t *B, uint64_t ldb, uint32_t *C, uint64_t ldc)
{
    for (uint64_t i = r0; i < r1; ++i)
        for (uint64_t j = 0; j < nb; ++j) {
            uint64_t r = 0;
            for (uint64_t q = row_ptr[i]; q < row_ptr[i + 1]; ++q)
                r = zpz_axpy(r, val[q], B[(uint64_t)col[q] * ldb + j], p);
            C[i * ldc + j] = (uint32_t)r;
        }
}

/* ------------------------------------------------------------------------
 * The paper's dot-product variants, restated (checked against oracle_dot).
 * ---------------------------------------------------------------------- */

/* Blocked delayed division, "block-XXX" (Section 3.2): accumulate K products
 * in an acc_bits-wide unsigned accumulator (32 or 64), take one remainder per
 * full block of K terms, then the tail, then one final remainder.  The caller
 * chooses K; it is correct when K*(p-1)^2 + (p-1) < 2^acc_bits (Eq. (2) form,
 * since the residue of one block is carried into the next).  Returns the
 * residue, or UINT64_MAX when K violates that bound. */
uint64_t oracle_paper_block_dot(uint32_t p, uint64_t n, const uint32_t *a, const uint32_t *b,
                                uint64_t K, int acc_bits)
{
    if (K == 0 || (acc_bits != 32 && acc_bits != 64)) return UINT64_MAX;
    const unsigned __int128 lim = (acc_bits == 64) ? ((unsigned __int128)1 << 64)
                                                    : ((unsigned __int128)1 << 32);
    const unsigned __int128 pm1 = p - 1;
    if ((unsigned __int128)K * pm1 * pm1 + pm1 >= lim) return UINT64_MAX;
    const uint64_t mask = (acc_bits == 64) ? UINT64_MAX : 0xFFFFFFFFull;
    uint64_t res = 0, i = 0;
    if (K < n) {
        uint64_t full = (n / K) * K;
        while (i < full) {
            for (uint64_t j = 0; j < K; ++j, ++i)
                res = (res + (uint64_t)a[i] * b[i]) & mask;
            res %= p;
        }
    }
    for (; i < n; ++i)
        res = (res + (uint64_t)a[i] * b[i]) & mask;
    return res % p;
}

/* Division on demand (Section 3.3): let the m-bit unsigned sum wrap, detect
 * the wrap by comparing the new sum with the product just added, and add the
 * correction CORR = 2^m mod p when it happened.  Valid here for m = 64 and
 * p <= 2^32-1: every product is at most (p-1)^2 < 2^64 - 2^33, and after a
 * wrap the sum is below the product, so adding CORR < 2^32 cannot wrap again.
 * One final remainder at the end. */
uint32_t oracle_paper_overflow_dot(uint32_t p, uint64_t n, const uint32_t *a, const uint32_t *b)
{
    /* CORR = 2^64 mod p, from (2^64 - 1) mod p + 1. */
    const uint64_t corr = (UINT64_MAX % p + 1) % p;
    uint64_t sum = 0;
    for (uint64_t i = 0; i < n; ++i) {
        uint64_t product = (uint64_t)a[i] * b[i];
        sum += product;
        if (sum < product) sum += corr;
    }
    return (uint32_t)(sum % p);
}

/* Floating-point reduction (Section 2.3): T mod P = T - floor(T * 1/P) * P,
 * followed by a one-step adjustment for the rounding of the floor.  Valid for
 * integral 0 <= T <= 2^53.  The product floor(.)*P is formed with fma so that
 * no intermediate rounds (the remainder is a small exact integer). */
double oracle_paper_fp_reduce(double T, double P)
{
    double invP = 1.0 / P;
    double q = floor(T * invP);
    double r = fma(-q, P, T);
    if (r >= P) r -= P;
    else if (r < 0) r += P;
    return r;
}

/* Dot product in the floating-point representation with delayed division
 * (Section 3.1, m = 53): accumulate exactly in a double and reduce every K
 * terms with the floating-point reduction; K*(p-1)^2 + (p-1) <= 2^53 keeps
 * every partial sum an exactly representable integer.  Returns the residue,
 * or UINT32_MAX when K violates that bound. */
uint32_t oracle_paper_fp_dot(uint32_t p, uint64_t n, const uint32_t *a, const uint32_t *b,
                             uint64_t K)
{
    const unsigned __int128 pm1 = p - 1;
    if (K == 0 || (unsigned __int128)K * pm1 * pm1 + pm1 > ((unsigned __int128)1 << 53))
        return UINT32_MAX;
    double P = (double)p, acc = 0.0;
    uint64_t left = K;
    for (uint64_t i = 0; i < n; ++i) {
        if (left == 0) { acc = oracle_paper_fp_reduce(acc, P); left = K; }
        acc += (double)a[i] * (double)b[i];
        --left;
    }
    return (uint32_t)oracle_paper_fp_reduce(acc, P);
}

/*
 * Finite fields GF(q), q = p^k, for the discrete-logarithm (Zech) dot product
 * of Section 2.4 ("Discrete logarithms" and "Field extensions").  Plain
 * definition: an element is a polynomial of degree < k over GF(p), encoded as
 * the integer sum_j c_j p^j (c_j in [0, p) the coefficient of x^j); the field
 * is GF(p)[x] / (f) for a monic f = x^k + f_{k-1} x^{k-1} + ... + f_0 given
 * by its low coefficients f[0..k-1].  Addition adds coefficients mod p;
 * multiplication is the schoolbook product reduced by x^k = -(f_{k-1} x^{k-1}
 * + ... + f_0).  The dot product applies these field operations term by term.
 * For k = 1 (f = x + f_0) the encoding is the residue itself and the
 * operations are those of GF(p).
 */
#define ORACLE_GFQ_MAXK 32

static void gfq_digits(uint32_t p, uint32_t k, uint32_t v, uint32_t *c)
{
    for (uint32_t j = 0; j < k; ++j) {
        c[j] = v % p;
        v /= p;
    }
}

static uint32_t gfq_value(uint32_t p, uint32_t k, const uint32_t *c)
{
    uint32_t v = 0;
    for (uint32_t j = k; j-- > 0;) v = v * p + c[j];
    return v;
}

uint32_t oracle_gfq_add(uint32_t p, uint32_t k, uint32_t a, uint32_t b)
{
    uint32_t ca[ORACLE_GFQ_MAXK], cb[ORACLE_GFQ_MAXK];
    gfq_digits(p, k, a, ca);
    gfq_digits(p, k, b, cb);
    for (uint32_t j = 0; j < k; ++j) ca[j] = (uint32_t)(((uint64_t)ca[j] + cb[j]) % p);
    return gfq_value(p, k, ca);
}

uint32_t oracle_gfq_mul(uint32_t p, uint32_t k, const uint32_t *f, uint32_t a, uint32_t b)
{
    uint32_t ca[ORACLE_GFQ_MAXK], cb[ORACLE_GFQ_MAXK];
    uint64_t prod[2 * ORACLE_GFQ_MAXK];
    gfq_digits(p, k, a, ca);
    gfq_digits(p, k, b, cb);
    for (uint32_t m = 0; m < 2 * k; ++m) prod[m] = 0;
    for (uint32_t i = 0; i < k; ++i)
        for (uint32_t j = 0; j < k; ++j) prod[i + j] = (prod[i + j] + (uint64_t)ca[i] * cb[j]) % p;
    /* reduce from the top degree down: t x^m = t x^{m-k} x^k = -t sum_j f_j x^{m-k+j} */
    for (uint32_t m = 2 * k - 1; m-- > k;) {
        const uint64_t t = prod[m];
        prod[m] = 0;
        for (uint32_t j = 0; j < k; ++j)
            prod[m - k + j] = (prod[m - k + j] + (uint64_t)(p - f[j] % p) % p * t) % p;
    }
    uint32_t c[ORACLE_GFQ_MAXK];
    for (uint32_t j = 0; j < k; ++j) c[j] = (uint32_t)prod[j];
    return gfq_value(p, k, c);
}

uint32_t oracle_gfq_dot(uint32_t p, uint32_t k, const uint32_t *f, uint64_t n, const uint32_t *x,
                        const uint32_t *y)
{
    uint32_t r = 0;
    for (uint64_t i = 0; i < n; ++i) r = oracle_gfq_add(p, k, r, oracle_gfq_mul(p, k, f, x[i], y[i]));
    return r;
}
