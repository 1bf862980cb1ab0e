// Field arithmetic shared by the kernels and the host entry points of
// libgfpdot: per-modulus constants, the reductions into [0, p), and the
// unreduced accumulators of the dot-product method (Dumas, "Efficient dot
// product over word-size finite fields", Sections 2.1, 2.3 and 3.1-3.4).
#pragma once
#include <stdint.h>
#include <math.h>

#if defined(__CUDACC__)
#define GFP_HD __host__ __device__ __forceinline__
#define GFP_D __device__ __forceinline__
#else
#define GFP_HD inline
#define GFP_D inline
#endif

namespace gfp {

enum Repr : uint32_t {
    PERTERM = 1, U64_BLOCK = 2, U64_CARRY = 3, FP64 = 4, CENTERED = 6, MONTGOMERY = 7
};

// Constants for one modulus p (2 <= p <= 2^32-1).
struct Mod {
    uint32_t p;
    uint32_t corr;   // 2^64 mod p: the correction of a wrapped 64-bit sum (Section 3.3)
    uint64_t mu;     // floor(2^64 / p) for Barrett's reduction
    double pd;       // p as a double
    double invp;     // 1/p rounded to double (Section 2.3)
};

GFP_HD uint64_t mulhi64(uint64_t a, uint64_t b)
{
#if defined(__CUDA_ARCH__)
    return __umul64hi(a, b);
#else
    return (uint64_t)(((unsigned __int128)a * b) >> 64);
#endif
}

// x mod p by Barrett's method (P. Barrett, CRYPTO '86; Menezes et al.,
// Handbook of Applied Cryptography, Alg. 14.42) specialised to a 64-bit x and
// mu = floor(2^64/p).  With Q = floor(x/p): q = floor(x*mu / 2^64) <= x/p, and
// since mu > 2^64/p - 1, q > x/p - x/2^64 - 1 > x/p - 2, so q is Q or Q-1 and
// one conditional subtraction finishes the reduction.
GFP_HD uint32_t reduce64(uint64_t x, const Mod &m)
{
    uint64_t q = mulhi64(x, m.mu);
    uint64_t r = x - q * (uint64_t)m.p;
    if (r >= m.p) r -= m.p;
    return (uint32_t)r;
}

// Floating-point reduction of Section 2.3 for an integral 0 <= T <= 2^53:
// T - floor(T/p)*p with 1/p precomputed.  T*invp is within 2/p < 1 of T/p,
// so the floor is off by at most one and one adjustment each way suffices.
// fma forms T - q*p with a single rounding of an exact small integer, so the
// remainder itself is exact (no intermediate q*p rounding near 2^53).
GFP_HD double reduce_f64(double T, const Mod &m)
{
    double q = floor(T * m.invp);
    double r = fma(-q, m.pd, T);
    if (r >= m.pd) r -= m.pd;
    else if (r < 0.0) r += m.pd;
    return r;
}

// ---------------------------------------------------------------------------
// Per-thread accumulators.  Each consumes products of canonical residues and
// yields the residue of their sum.  `add4` takes four terms at once (one
// 128-bit load of each operand).
// ---------------------------------------------------------------------------

// Classical representation (Section 2.1): one remainder per term.  This is the
// per-term baseline the delayed forms are measured against.
struct AccPerTerm {
    uint64_t r;
    GFP_D void init(const Mod &, uint64_t) { r = 0; }
    GFP_D void add(uint32_t a, uint32_t b, const Mod &m) { r = (r + (uint64_t)a * b) % m.p; }
    GFP_D void add4(uint4 a, uint4 b, const Mod &m)
    {
        add(a.x, b.x, m); add(a.y, b.y, m); add(a.z, b.z, m); add(a.w, b.w, m);
    }
    GFP_D uint32_t residue(const Mod &) const { return (uint32_t)r; }
};

// Blocked delayed division (Sections 3.1-3.2): a 64-bit accumulator absorbs
// up to k products, then is reduced; the residue carries into the next block,
// so k is the Eq. (2) bound k(p-1)^2 + (p-1) < 2^64.  For p < 2^16, k exceeds
// 2^32 and no reduction ever happens inside a kernel.
struct AccBlock {
    uint64_t acc, left, k;
    GFP_D void init(const Mod &, uint64_t kk) { acc = 0; k = kk; left = kk; }
    GFP_D void add(uint32_t a, uint32_t b, const Mod &m)
    {
        if (left == 0) { acc = reduce64(acc, m); left = k; }
        acc += (uint64_t)a * b;
        --left;
    }
    GFP_D void add4(uint4 a, uint4 b, const Mod &m)
    {
        if (left >= 4) {
            acc += (uint64_t)a.x * b.x;
            acc += (uint64_t)a.y * b.y;
            acc += (uint64_t)a.z * b.z;
            acc += (uint64_t)a.w * b.w;
            left -= 4;
        } else {
            add(a.x, b.x, m); add(a.y, b.y, m); add(a.z, b.z, m); add(a.w, b.w, m);
        }
    }
    GFP_D uint32_t residue(const Mod &m) const { return reduce64(acc, m); }
};

// Division on demand (Section 3.3), hybrid form: the 64-bit sum is allowed to
// wrap; instead of adding CORR = 2^64 mod p at each wrap, the wraps are
// counted (a wrap happened iff the new sum is below the product just added)
// and CORR is applied once at the end: value = lo + c*2^64 = lo + c*CORR
// (mod p).  Exact for any p <= 2^32-1 and up to 2^32-1 wraps per thread,
// with no remainder inside the loop.
struct AccCarry {
    uint32_t lo0, lo1, c;
    GFP_D void init(const Mod &, uint64_t) { lo0 = lo1 = c = 0; }
    GFP_D void add(uint32_t a, uint32_t b, const Mod &)
    {
#if defined(__CUDA_ARCH__)
        asm("mad.lo.cc.u32 %0, %3, %4, %0;\n\t"
            "madc.hi.cc.u32 %1, %3, %4, %1;\n\t"
            "addc.u32 %2, %2, 0;"
            : "+r"(lo0), "+r"(lo1), "+r"(c) : "r"(a), "r"(b));
#else
        uint64_t lo = ((uint64_t)lo1 << 32) | lo0, t = (uint64_t)a * b;
        lo += t; c += (lo < t);
        lo0 = (uint32_t)lo; lo1 = (uint32_t)(lo >> 32);
#endif
    }
    GFP_D void add4(uint4 a, uint4 b, const Mod &m)
    {
        add(a.x, b.x, m); add(a.y, b.y, m); add(a.z, b.z, m); add(a.w, b.w, m);
    }
    GFP_D uint32_t residue(const Mod &m) const
    {
        uint64_t lo = ((uint64_t)lo1 << 32) | lo0;
        uint32_t r1 = reduce64(lo, m);
        uint32_t r2 = reduce64((uint64_t)c * m.corr, m);   // c, corr < 2^32
        uint64_t s = (uint64_t)r1 + r2;
        return (uint32_t)(s >= m.p ? s - m.p : s);
    }
};

// Floating-point representation with delayed division (Section 3.1, m = 53):
// products of residues below 2^26 accumulate exactly in a double (fma forms
// a*b + acc with one rounding of an exact integer <= 2^53) and the sum is
// reduced with the Section 2.3 reduction every k terms, k the Eq. (2) bound for
// m = 53.
struct AccF64 {
    double acc;
    uint64_t left, k;
    GFP_D void init(const Mod &, uint64_t kk) { acc = 0.0; k = kk; left = kk; }
    GFP_D void add(uint32_t a, uint32_t b, const Mod &m)
    {
        if (left == 0) { acc = reduce_f64(acc, m); left = k; }
        acc = fma((double)a, (double)b, acc);
        --left;
    }
    GFP_D void add4(uint4 a, uint4 b, const Mod &m)
    {
        if (left >= 4) {
            acc = fma((double)a.x, (double)b.x, acc);
            acc = fma((double)a.y, (double)b.y, acc);
            acc = fma((double)a.z, (double)b.z, acc);
            acc = fma((double)a.w, (double)b.w, acc);
            left -= 4;
        } else {
            add(a.x, b.x, m); add(a.y, b.y, m); add(a.z, b.z, m); add(a.w, b.w, m);
        }
    }
    GFP_D uint32_t residue(const Mod &m) const { return (uint32_t)reduce_f64(acc, m); }
};

// Centred representation (Section 3.2.2): residues are read as
// s in [-(p-1)/2, (p-1)/2] and signed products accumulate in 64 bits; with
// h = (p-1)/2 the block bound is k h^2 + (p-1) <= 2^63 - 1, about twice the
// unsigned Eq. (2) block for the same modulus.  Reduction of a signed sum
// into [0, p) uses the Barrett reduction of its magnitude.
struct AccCentered {
    long long acc;
    uint64_t left, k;
    GFP_D void init(const Mod &, uint64_t kk) { acc = 0; k = kk; left = kk; }
    static GFP_D long long centre(uint32_t a, const Mod &m)
    {
        return (a > ((m.p - 1) >> 1)) ? (long long)a - (long long)m.p : (long long)a;
    }
    static GFP_D uint32_t residue_of(long long v, const Mod &m)
    {
        if (v >= 0) return reduce64((uint64_t)v, m);
        const uint32_t t = reduce64((uint64_t)(-v), m);
        return t ? m.p - t : 0u;
    }
    GFP_D void add(uint32_t a, uint32_t b, const Mod &m)
    {
        if (left == 0) { acc = (long long)residue_of(acc, m); left = k; }
        acc += centre(a, m) * centre(b, m);
        --left;
    }
    GFP_D void add4(uint4 a, uint4 b, const Mod &m)
    {
        if (left >= 4) {
            acc += centre(a.x, m) * centre(b.x, m);
            acc += centre(a.y, m) * centre(b.y, m);
            acc += centre(a.z, m) * centre(b.z, m);
            acc += centre(a.w, m) * centre(b.w, m);
            left -= 4;
        } else {
            add(a.x, b.x, m); add(a.y, b.y, m); add(a.z, b.z, m); add(a.w, b.w, m);
        }
    }
    GFP_D uint32_t residue(const Mod &m) const { return residue_of(acc, m); }
};

// Montgomery reduction (Section 2.2; blocked as in Section 3.2.1) with
// B = 2^32 for odd p: a block of products T < pB is reduced by
// REDC(T) = T B^-1 mod p (Montgomery, Math. Comp. 1985), the block results
// are summed, and the total, which carries a factor B^-1, is multiplied back
// by REDC(total * (B^2 mod p)).  B^2 mod p = 2^64 mod p is the CORR constant.
struct AccMontgomery {
    uint64_t acc, sum;
    uint64_t left, k;
    uint32_t ninv;   // -p^-1 mod 2^32
    GFP_D void init(const Mod &m, uint64_t kk)
    {
        acc = 0; sum = 0; k = kk; left = kk;
        uint32_t x = m.p;                       // p^-1 mod 2^32 by Newton's iteration
        for (int i = 0; i < 5; ++i) x *= 2u - m.p * x;
        ninv = 0u - x;
    }
    GFP_D uint32_t redc(uint64_t T, const Mod &m) const
    {
        const uint32_t lo = (uint32_t)T;
        const uint32_t q = lo * ninv;           // T + q p = 0 (mod 2^32)
        // (T + q p) / 2^32 without the 65-bit sum: the low words cancel exactly
        uint64_t t = (T >> 32) + (uint64_t)(((uint64_t)q * m.p) >> 32) + (lo != 0u ? 1u : 0u);
        if (t >= m.p) t -= m.p;
        return (uint32_t)t;
    }
    GFP_D void flush(const Mod &m) { sum += redc(acc, m); acc = 0; left = k; }
    GFP_D void add(uint32_t a, uint32_t b, const Mod &m)
    {
        if (left == 0) flush(m);
        acc += (uint64_t)a * b;
        --left;
    }
    GFP_D void add4(uint4 a, uint4 b, const Mod &m)
    {
        if (left >= 4) {
            acc += (uint64_t)a.x * b.x;
            acc += (uint64_t)a.y * b.y;
            acc += (uint64_t)a.z * b.z;
            acc += (uint64_t)a.w * b.w;
            left -= 4;
        } else {
            add(a.x, b.x, m); add(a.y, b.y, m); add(a.z, b.z, m); add(a.w, b.w, m);
        }
    }
    GFP_D uint32_t residue(const Mod &m) const
    {
        // sum < (blocks + 1) p; reduce, then multiply back by B: REDC(x * B^2 mod p) = x B
        const uint64_t total = (uint64_t)reduce64(sum + redc(acc, m), m);
        return redc(total * m.corr, m);
    }
};

}  // namespace gfp
