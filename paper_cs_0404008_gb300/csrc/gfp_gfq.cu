// Dot product over a finite field GF(q), q = p^k <= 2^16, in the discrete-
// logarithm ("Zech logarithm") representation of Section 2.4, which stays the
// same for prime fields and their extensions.
//
// Codes: the zero element is code 0, the element g^e (g = x, the class of x
// in GF(p)[x]/(f) for a primitive f) is code e for 1 <= e <= q-2, and 1 = g^0
// is code q-1 (= qbar).  Hence every non-zero code is congruent to its
// exponent modulo qbar, and
//   g^i * g^j = g^(i+j):         code i + j, less qbar when above qbar;
//   g^i + g^j = g^i (1 + g^(j-i)): code i + Z[(j - i) mod qbar], less qbar when
//                                 above qbar, where Z[t] is the code of 1 + g^t
//                                 (Z[t] = 0 when 1 + g^t is zero)
// with one table Z of qbar entries, as the paper's operation table lays out.
//
// The dot-product kernel keeps Z in shared memory (a 64K-entry uint16 table,
// so every index a masked 16-bit difference can form stays inside it), streams
// the two code vectors with 16-byte loads, and runs four independent
// accumulation chains per thread (each addition waits on its table lookup).
// Warps, then the CTA, combine their partial sums with the same Zech addition;
// the last CTA to finish (ticket counter) combines the CTA partials.
//
// Prime fields and fields of characteristic 2 take a cheaper route to the
// same sum: a product is still a code addition, but each product is turned
// back into its element value by one lookup in the code-to-value table and
// the values are added in the additive representation, as integers for
// GF(p) (a 64-bit sum of values below 2^16 needs no reduction before 2^48
// terms) and by XOR for GF(2^k) (coefficient-wise addition mod 2); the total
// is converted to a code once.  That replaces the Zech addition, the costly
// step of the representation, by one lookup and one add.
#include <algorithm>
#include <cstring>
#include <vector>

#include "gfp_internal.h"

struct gfp_gfq {
    int device = 0;
    uint32_t p = 0, k = 0, q = 0, qbar = 0;
    uint32_t f[16] = {0};
    uint16_t *d_zech = nullptr;      // 65536 entries; Z[t] for t < qbar, zero beyond
    uint32_t *d_log = nullptr;       // q entries: element value -> code
    uint32_t *d_exp = nullptr;       // qbar + 1 entries: code -> element value
    uint32_t *d_partials = nullptr;  // one per CTA of the dot kernel
    uint32_t *d_ticket = nullptr;    // finished CTAs (zero outside calls)
    uint32_t *d_err = nullptr;       // bit 0: a value >= q or a code > qbar was converted
    uint16_t *d_exp16 = nullptr;     // 65536 entries: code -> element value (entry 0: 1; 0 beyond qbar)
    unsigned long long *d_acc = nullptr;   // value-domain sum of the dot kernel (zero outside calls)
    uint8_t *d_tab8 = nullptr;       // q <= 256, k > 1: code -> value and value addition tables
    uint32_t tab8_bytes = 0;
    int mode = 0;                    // 0: Zech additions; 1: integer sum (k = 1); 2: XOR (p = 2);
                                     // 3: value-addition table (odd p, k > 1, q <= 256)
    int grid = 0;
};

namespace gfp {
namespace gfq {

constexpr int THREADS = 1024;
constexpr uint32_t TABLE = 65536;
constexpr size_t SMEM = TABLE * sizeof(uint16_t);   // 128 KiB
// fields from this size on take the Zech kernel with the rare zero branch
// (measured at 2^27 codes: faster from q = 1331 on, slower up to q = 729,
// where a warp's four updates of 32 lanes meet a zero element too often)
constexpr uint32_t RARE_Q = 1024;
// grid strides per loop iteration: with one 1024-thread CTA per SM (the table
// takes 128 KiB of shared memory) and 64 registers per thread, eight 16-byte
// loads in flight per thread are what keeps HBM busy (one stride: 0.75-0.77 of
// the copy bandwidth for the value-domain sums, four: 0.88-0.94)
#ifndef GFQ_NS
#define GFQ_NS 4
#endif

__device__ __forceinline__ uint32_t zmul(uint32_t a, uint32_t b, uint32_t qbar)
{
    uint32_t r = a + b;
    r = r > qbar ? r - qbar : r;
    return (a == 0u || b == 0u) ? 0u : r;
}

// a + c in codes; the table index is masked to 16 bits, so codes outside
// [0, qbar] (out of contract) give an unspecified code but never leave Z
__device__ __forceinline__ uint32_t zadd(uint32_t a, uint32_t c, const uint16_t *Z, uint32_t qbar)
{
    uint32_t t = c - a;
    t = c < a ? t + qbar : t;
    const uint32_t z = Z[t & 0xFFFFu];
    uint32_t r = a + z;
    r = r > qbar ? r - qbar : r;
    r = z == 0u ? 0u : r;
    r = a == 0u ? c : r;
    return c == 0u ? a : r;
}

// acc + (code a) * (code b) for fields whose zero element is rare, common
// case only (a, b, acc nonzero, no cancellation), without selects: returns the
// new code and sets m to a value that is 0 exactly when the case is not the
// common one (a zero code, a zero accumulator, or Z[t] = 0 when the sum
// cancels: a zero factor shows as a zero product, all four being below 2^16).
// Codes are 1..qbar for nonzero elements, 0 for zero.
__device__ __forceinline__ uint32_t zfast(uint32_t acc, uint32_t a, uint32_t b, const uint16_t *Z,
                                          uint32_t qbar, uint32_t &m)
{
    uint32_t c = a + b;                         // code of the product, modulo qbar:
    c = min(c, c - qbar);                       // qbar becomes 0, the same index below
    const uint32_t d = c - acc;                 // (c - acc) mod qbar by an unsigned min
    const uint32_t t = min(d, d + qbar);
    const uint32_t z = Z[t & 0xFFFFu];
    uint32_t r = acc + z;
    r = r > qbar ? r - qbar : r;
    m = min(a * b, acc * z);
    return r;
}

// Four independent chains advanced by one term each, with one test for the
// rare cases of all four (if any needs it, all four take the general code on
// that rarely taken branch); the four common-case updates interleave.
__device__ __forceinline__ void zstep4(uint32_t &x0, uint32_t &x1, uint32_t &x2, uint32_t &x3,
                                       uint32_t a0, uint32_t b0, uint32_t a1, uint32_t b1,
                                       uint32_t a2, uint32_t b2, uint32_t a3, uint32_t b3,
                                       const uint16_t *Z, uint32_t qbar)
{
    uint32_t m0, m1, m2, m3;
    const uint32_t r0 = zfast(x0, a0, b0, Z, qbar, m0), r1 = zfast(x1, a1, b1, Z, qbar, m1);
    const uint32_t r2 = zfast(x2, a2, b2, Z, qbar, m2), r3 = zfast(x3, a3, b3, Z, qbar, m3);
    if (min(min(m0, m1), min(m2, m3)) == 0u) {
        x0 = zadd(x0, zmul(a0, b0, qbar), Z, qbar);
        x1 = zadd(x1, zmul(a1, b1, qbar), Z, qbar);
        x2 = zadd(x2, zmul(a2, b2, qbar), Z, qbar);
        x3 = zadd(x3, zmul(a3, b3, qbar), Z, qbar);
    } else {
        x0 = r0;
        x1 = r1;
        x2 = r2;
        x3 = r3;
    }
}

__device__ __forceinline__ uint32_t warp_zsum(uint32_t v, const uint16_t *Z, uint32_t qbar)
{
#pragma unroll
    for (int o = 16; o; o >>= 1) v = zadd(v, __shfl_xor_sync(0xffffffffu, v, o), Z, qbar);
    return v;
}

__device__ __forceinline__ uint4 ldcs4(const uint16_t *p, uint64_t v)
{
    return __ldcs(reinterpret_cast<const uint4 *>(p) + v);
}

// RARE: zstep4 (zero elements handled on a rare branch), for large fields;
// otherwise the select form of zadd(zmul), for small fields where zeros are
// frequent enough to make the branch diverge.
template <bool RARE>
__global__ void __launch_bounds__(THREADS, 1)
    k_gfq_dot(const uint16_t *__restrict__ x, const uint16_t *__restrict__ y, uint64_t n,
              int vec, const uint16_t *__restrict__ Zg, uint32_t qbar, uint32_t *partials,
              uint32_t *ticket, uint16_t *out)
{
    extern __shared__ uint16_t Z[];
    __shared__ uint32_t wpart[THREADS / 32];
    __shared__ uint32_t last;
    // Z[0 .. qbar] is all the arithmetic of valid codes reads
    // programmatic dependent launch: placed while the previous kernel of the
    // stream drains, a CTA loads the field's table (constant) first and only
    // then waits for that kernel, which may have produced the codes
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    const uint32_t nload = (qbar + 8u) / 8u;
    for (uint32_t i = threadIdx.x; i < nload; i += blockDim.x)
        reinterpret_cast<uint4 *>(Z)[i] = reinterpret_cast<const uint4 *>(Zg)[i];
    asm volatile("griddepcontrol.wait;" ::: "memory");
    __syncthreads();

    const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint64_t nthreads = (uint64_t)gridDim.x * blockDim.x;
    uint32_t a0 = 0, a1 = 0, a2 = 0, a3 = 0;
    const uint64_t nvec = vec ? n / 8 : 0;
    auto step = [&](const uint4 &u, const uint4 &w) {
        if constexpr (RARE) {
            zstep4(a0, a1, a2, a3, u.x & 0xFFFFu, w.x & 0xFFFFu, u.x >> 16, w.x >> 16,
                   u.y & 0xFFFFu, w.y & 0xFFFFu, u.y >> 16, w.y >> 16, Z, qbar);
            zstep4(a0, a1, a2, a3, u.z & 0xFFFFu, w.z & 0xFFFFu, u.z >> 16, w.z >> 16,
                   u.w & 0xFFFFu, w.w & 0xFFFFu, u.w >> 16, w.w >> 16, Z, qbar);
        } else {
            a0 = zadd(a0, zmul(u.x & 0xFFFFu, w.x & 0xFFFFu, qbar), Z, qbar);
            a1 = zadd(a1, zmul(u.x >> 16, w.x >> 16, qbar), Z, qbar);
            a2 = zadd(a2, zmul(u.y & 0xFFFFu, w.y & 0xFFFFu, qbar), Z, qbar);
            a3 = zadd(a3, zmul(u.y >> 16, w.y >> 16, qbar), Z, qbar);
            a0 = zadd(a0, zmul(u.z & 0xFFFFu, w.z & 0xFFFFu, qbar), Z, qbar);
            a1 = zadd(a1, zmul(u.z >> 16, w.z >> 16, qbar), Z, qbar);
            a2 = zadd(a2, zmul(u.w & 0xFFFFu, w.w & 0xFFFFu, qbar), Z, qbar);
            a3 = zadd(a3, zmul(u.w >> 16, w.w >> 16, qbar), Z, qbar);
        }
    };
    // GFQ_NS strides per iteration: 2 GFQ_NS 16-byte loads in flight per thread
    uint64_t v = tid;
    for (; v + (GFQ_NS - 1) * nthreads < nvec; v += GFQ_NS * nthreads) {
        uint4 u[GFQ_NS], w[GFQ_NS];
#pragma unroll
        for (int j = 0; j < GFQ_NS; ++j) {
            u[j] = ldcs4(x, v + j * nthreads);
            w[j] = ldcs4(y, v + j * nthreads);
        }
#pragma unroll
        for (int j = 0; j < GFQ_NS; ++j) step(u[j], w[j]);
    }
    for (; v < nvec; v += nthreads) step(ldcs4(x, v), ldcs4(y, v));
    for (uint64_t i = nvec * 8 + tid; i < n; i += nthreads) a0 = zadd(a0, zmul(x[i], y[i], qbar), Z, qbar);
    uint32_t acc = zadd(zadd(a0, a1, Z, qbar), zadd(a2, a3, Z, qbar), Z, qbar);

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    acc = warp_zsum(acc, Z, qbar);
    if (lane == 0) wpart[warp] = acc;
    __syncthreads();
    if (warp == 0) {
        acc = lane < (int)(blockDim.x >> 5) ? wpart[lane] : 0u;
        acc = warp_zsum(acc, Z, qbar);
        if (lane == 0) {
            partials[blockIdx.x] = acc;
            __threadfence();
            last = atomicAdd(ticket, 1u) == gridDim.x - 1 ? 1u : 0u;
        }
    }
    __syncthreads();
    if (last && warp == 0) {
        __threadfence();
        acc = 0;
        for (uint32_t b = lane; b < gridDim.x; b += 32) acc = zadd(acc, __ldcg(partials + b), Z, qbar);
        acc = warp_zsum(acc, Z, qbar);
        if (lane == 0) {
            *out = (uint16_t)acc;
            *ticket = 0u;   // ready for the next call
        }
    }
}

// Value-domain dot product for GF(p) (XOR = false: integer sum, reduced mod p
// once) and GF(2^k) (XOR = true): acc += exp(code(x_i) + code(y_i)).
template <bool XOR>
__global__ void __launch_bounds__(THREADS, 1)
    k_gfq_dot_exp(const uint16_t *__restrict__ x, const uint16_t *__restrict__ y, uint64_t n, int vec,
                  const uint16_t *__restrict__ Eg, uint32_t qbar, uint32_t p, const uint32_t *__restrict__ logt,
                  unsigned long long *acc_slot, uint32_t *ticket, uint16_t *out)
{
    extern __shared__ uint16_t E[];
    __shared__ unsigned long long wpart[THREADS / 32];
    __shared__ uint32_t last;
    // programmatic dependent launch: placed while the previous kernel of the
    // stream drains, a CTA loads the field's table (constant) first and only
    // then waits for that kernel, which may have produced the codes
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    const uint32_t nload = (qbar + 8u) / 8u;   // E[0 .. qbar]
    for (uint32_t i = threadIdx.x; i < nload; i += blockDim.x)
        reinterpret_cast<uint4 *>(E)[i] = reinterpret_cast<const uint4 *>(Eg)[i];
    asm volatile("griddepcontrol.wait;" ::: "memory");
    __syncthreads();

    // value of the product of codes a and b (0 if either is the zero element)
    auto prod = [&](uint32_t a, uint32_t b) -> uint32_t {
        uint32_t c = a + b;
        c = min(c, c - qbar);   // a + b mod qbar, qbar itself becoming 0 (E[0] = E[qbar] = 1)
        const uint32_t v = E[c & 0xFFFFu];
        return (a == 0u || b == 0u) ? 0u : v;
    };
    const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint64_t nthreads = (uint64_t)gridDim.x * blockDim.x;
    unsigned long long s0 = 0, s1 = 0;
    uint32_t x0 = 0, x1 = 0;
    const uint64_t nvec = vec ? n / 8 : 0;
    auto step = [&](const uint4 &u, const uint4 &w) {
        const uint32_t a0 = prod(u.x & 0xFFFFu, w.x & 0xFFFFu), a1 = prod(u.x >> 16, w.x >> 16);
        const uint32_t a2 = prod(u.y & 0xFFFFu, w.y & 0xFFFFu), a3 = prod(u.y >> 16, w.y >> 16);
        const uint32_t a4 = prod(u.z & 0xFFFFu, w.z & 0xFFFFu), a5 = prod(u.z >> 16, w.z >> 16);
        const uint32_t a6 = prod(u.w & 0xFFFFu, w.w & 0xFFFFu), a7 = prod(u.w >> 16, w.w >> 16);
        if (XOR) {
            x0 ^= a0 ^ a1 ^ a2 ^ a3;
            x1 ^= a4 ^ a5 ^ a6 ^ a7;
        } else {
            s0 += (a0 + a1) + (a2 + a3);   // each below 2^16: the 32-bit partial sums cannot wrap
            s1 += (a4 + a5) + (a6 + a7);
        }
    };
    // GFQ_NS strides per iteration: 2 GFQ_NS 16-byte loads in flight per thread
    uint64_t v = tid;
    for (; v + (GFQ_NS - 1) * nthreads < nvec; v += GFQ_NS * nthreads) {
        uint4 u[GFQ_NS], w[GFQ_NS];
#pragma unroll
        for (int j = 0; j < GFQ_NS; ++j) {
            u[j] = ldcs4(x, v + j * nthreads);
            w[j] = ldcs4(y, v + j * nthreads);
        }
#pragma unroll
        for (int j = 0; j < GFQ_NS; ++j) step(u[j], w[j]);
    }
    for (; v < nvec; v += nthreads) step(ldcs4(x, v), ldcs4(y, v));
    for (uint64_t i = nvec * 8 + tid; i < n; i += nthreads) {
        if (XOR) x0 ^= prod(x[i], y[i]);
        else s0 += prod(x[i], y[i]);
    }
    unsigned long long acc = XOR ? (unsigned long long)(x0 ^ x1) : s0 + s1;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        const unsigned long long t = __shfl_xor_sync(0xffffffffu, acc, o);
        acc = XOR ? (acc ^ t) : (acc + t);
    }
    if (lane == 0) wpart[warp] = acc;
    __syncthreads();
    if (warp == 0) {
        acc = lane < (int)(blockDim.x >> 5) ? wpart[lane] : 0ull;
#pragma unroll
        for (int o = 16; o; o >>= 1) {
            const unsigned long long t = __shfl_xor_sync(0xffffffffu, acc, o);
            acc = XOR ? (acc ^ t) : (acc + t);
        }
        if (lane == 0) {
            if (XOR) atomicXor(reinterpret_cast<unsigned int *>(acc_slot), (unsigned int)acc);
            else atomicAdd(acc_slot, acc);
            __threadfence();
            last = atomicAdd(ticket, 1u) == gridDim.x - 1 ? 1u : 0u;
        }
    }
    __syncthreads();
    if (last && threadIdx.x == 0) {
        __threadfence();
        const unsigned long long tot = XOR ? (unsigned long long)__ldcg(reinterpret_cast<const unsigned int *>(acc_slot))
                                           : __ldcg(acc_slot);
        const uint32_t val = XOR ? (uint32_t)tot : (uint32_t)(tot % p);
        *out = (uint16_t)logt[val];
        *acc_slot = 0ull;   // ready for the next call
        *ticket = 0u;
    }
}

// Value-domain dot product for small odd-characteristic extension fields
// (k > 1, q <= 256): a product's code becomes its element value by one lookup
// and values are added by one lookup in the q x q field-addition table, both
// in shared memory: T[0, 256) code -> value (entry 0 holds x^0 = 1, entries
// past q-1 hold 0), T[256 + s q + v] = value of s + v.  Four chains per
// thread, then the warp, the CTA and the last CTA, all through the table.
// Every table entry is below q, so indices stay inside it for any input.
__global__ void __launch_bounds__(THREADS, 1)
    k_gfq_dot_add(const uint16_t *__restrict__ x, const uint16_t *__restrict__ y, uint64_t n, int vec,
                  const uint8_t *__restrict__ Tg, uint32_t tbytes, uint32_t q, uint32_t qbar,
                  const uint32_t *__restrict__ logt, uint32_t *partials, uint32_t *ticket, uint16_t *out)
{
    extern __shared__ uint8_t T[];
    __shared__ uint32_t wpart[THREADS / 32];
    __shared__ uint32_t last;
    // programmatic dependent launch: placed while the previous kernel of the
    // stream drains, a CTA loads the field's table (constant) first and only
    // then waits for that kernel, which may have produced the codes
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    for (uint32_t i = threadIdx.x; i < tbytes / 16u; i += blockDim.x)
        reinterpret_cast<uint4 *>(T)[i] = reinterpret_cast<const uint4 *>(Tg)[i];
    asm volatile("griddepcontrol.wait;" ::: "memory");
    __syncthreads();
    const uint8_t *E = T, *ADD = T + 256;

    auto prod = [&](uint32_t a, uint32_t b) -> uint32_t {
        uint32_t c = a + b;
        c = min(c, c - qbar);   // a + b mod qbar, qbar itself becoming 0 (E[0] = 1)
        const uint32_t v = E[c & 0xFFu];
        return (a == 0u || b == 0u) ? 0u : v;
    };
    auto add = [&](uint32_t s, uint32_t v) -> uint32_t { return ADD[s * q + v]; };
    const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint64_t nthreads = (uint64_t)gridDim.x * blockDim.x;
    uint32_t s0 = 0, s1 = 0, s2 = 0, s3 = 0;
    auto step = [&](const uint4 &u, const uint4 &w) {
        s0 = add(s0, prod(u.x & 0xFFFFu, w.x & 0xFFFFu));
        s1 = add(s1, prod(u.x >> 16, w.x >> 16));
        s2 = add(s2, prod(u.y & 0xFFFFu, w.y & 0xFFFFu));
        s3 = add(s3, prod(u.y >> 16, w.y >> 16));
        s0 = add(s0, prod(u.z & 0xFFFFu, w.z & 0xFFFFu));
        s1 = add(s1, prod(u.z >> 16, w.z >> 16));
        s2 = add(s2, prod(u.w & 0xFFFFu, w.w & 0xFFFFu));
        s3 = add(s3, prod(u.w >> 16, w.w >> 16));
    };
    const uint64_t nvec = vec ? n / 8 : 0;
    uint64_t v = tid;
    for (; v + (GFQ_NS - 1) * nthreads < nvec; v += GFQ_NS * nthreads) {
        uint4 u[GFQ_NS], w[GFQ_NS];
#pragma unroll
        for (int j = 0; j < GFQ_NS; ++j) {
            u[j] = ldcs4(x, v + j * nthreads);
            w[j] = ldcs4(y, v + j * nthreads);
        }
#pragma unroll
        for (int j = 0; j < GFQ_NS; ++j) step(u[j], w[j]);
    }
    for (; v < nvec; v += nthreads) step(ldcs4(x, v), ldcs4(y, v));
    for (uint64_t i = nvec * 8 + tid; i < n; i += nthreads) s0 = add(s0, prod(x[i], y[i]));
    uint32_t acc = add(add(s0, s1), add(s2, s3));
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o; o >>= 1) acc = add(acc, __shfl_xor_sync(0xffffffffu, acc, o));
    if (lane == 0) wpart[warp] = acc;
    __syncthreads();
    if (warp == 0) {
        acc = lane < (int)(blockDim.x >> 5) ? wpart[lane] : 0u;
#pragma unroll
        for (int o = 16; o; o >>= 1) acc = add(acc, __shfl_xor_sync(0xffffffffu, acc, o));
        if (lane == 0) {
            partials[blockIdx.x] = acc;
            __threadfence();
            last = atomicAdd(ticket, 1u) == gridDim.x - 1 ? 1u : 0u;
        }
    }
    __syncthreads();
    if (last && warp == 0) {
        __threadfence();
        acc = 0;
        for (uint32_t b = lane; b < gridDim.x; b += 32) acc = add(acc, __ldcg(partials + b));
#pragma unroll
        for (int o = 16; o; o >>= 1) acc = add(acc, __shfl_xor_sync(0xffffffffu, acc, o));
        if (lane == 0) {
            *out = (uint16_t)logt[acc];
            *ticket = 0u;   // ready for the next call
        }
    }
}

__global__ void k_gfq_to_log(const uint32_t *__restrict__ v, uint64_t n, const uint32_t *__restrict__ logt,
                             uint32_t q, uint16_t *__restrict__ codes, uint32_t *err)
{
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t a = v[i];
        if (a >= q) {
            atomicOr(err, 1u);
            codes[i] = 0;
        } else {
            codes[i] = (uint16_t)logt[a];
        }
    }
}

__global__ void k_gfq_from_log(const uint16_t *__restrict__ c, uint64_t n, const uint32_t *__restrict__ expt,
                               uint32_t qbar, uint32_t *__restrict__ v, uint32_t *err)
{
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t a = c[i];
        if (a > qbar) {
            atomicOr(err, 1u);
            v[i] = 0;
        } else {
            v[i] = expt[a];
        }
    }
}

// ---------------- host: field construction ----------------

// element with base-p digits c[0..k-1] times x, modulo f (x^k = -sum f_j x^j)
static void times_x(uint32_t p, uint32_t k, const uint32_t *f, uint32_t *c)
{
    if (k == 1) {   // x = -f_0
        c[0] = (uint32_t)((uint64_t)c[0] * ((p - f[0]) % p) % p);
        return;
    }
    const uint64_t t = c[k - 1];
    for (uint32_t j = k - 1; j >= 1; --j) c[j] = c[j - 1];
    c[0] = 0;
    for (uint32_t j = 0; j < k; ++j) c[j] = (uint32_t)((c[j] + (uint64_t)((p - f[j]) % p) * t) % p);
}

static uint32_t digits_value(uint32_t p, uint32_t k, const uint32_t *c)
{
    uint32_t v = 0;
    for (uint32_t j = k; j-- > 0;) v = v * p + c[j];
    return v;
}

// powers of x: expv[e] = value of x^e for e < q-1; false unless x generates
// all q-1 non-zero elements (so that the quotient ring is a field)
static bool powers_of_x(uint32_t p, uint32_t k, const uint32_t *f, uint32_t q, std::vector<uint32_t> &expv,
                        std::vector<uint32_t> &logv)
{
    expv.assign(q - 1, 0);
    logv.assign(q, 0);
    std::vector<uint8_t> seen(q, 0);
    uint32_t c[16] = {0};
    c[0] = 1;
    for (uint32_t e = 0; e + 1 < q; ++e) {
        const uint32_t v = digits_value(p, k, c);
        if (v == 0 || seen[v]) return false;
        seen[v] = 1;
        expv[e] = v;
        logv[v] = e == 0 ? q - 1 : e;
        times_x(p, k, f, c);
    }
    return digits_value(p, k, c) == 1;
}

static bool order_params(uint32_t p, uint32_t k, uint32_t &q)
{
    if (p < 2 || k < 1 || k > 16) return false;
    uint64_t qq = 1;
    for (uint32_t i = 0; i < k; ++i) {
        qq *= p;
        if (qq > 65536) return false;
    }
    q = (uint32_t)qq;
    return q >= 2;
}

}  // namespace gfq
}  // namespace gfp

using namespace gfp;

#define GFQ_TRY(expr)                       \
    do {                                    \
        cudaError_t e_ = (expr);            \
        if (e_ != cudaSuccess) {            \
            note_cuda_error(e_);            \
            return GFP_ERR_CUDA;            \
        }                                   \
    } while (0)

extern "C" {

GFP_API gfp_status gfp_gfq_find_primitive(uint32_t p, uint32_t k, uint32_t *f)
{
    GFP_TRACE();
    uint32_t q;
    if (!f || !gfq::order_params(p, k, q)) return GFP_ERR_INVALID;
    std::vector<uint32_t> expv, logv;
    std::vector<uint32_t> cand(k, 0);
    // candidates in lexicographic order of (f[k-1], ..., f[1]), then f[0] = 1 .. p-1
    for (;;) {
        for (uint32_t f0 = 1; f0 < p; ++f0) {
            cand[0] = f0;
            if (gfq::powers_of_x(p, k, cand.data(), q, expv, logv)) {
                std::copy(cand.begin(), cand.end(), f);
                return GFP_OK;
            }
        }
        uint32_t j = 1;
        while (j < k && ++cand[j] == p) cand[j++] = 0;
        if (j >= k) return GFP_ERR_INVALID;   // no primitive polynomial: p is not prime
    }
}

GFP_API gfp_status gfp_gfq_create(int device, uint32_t p, uint32_t k, const uint32_t *f, gfp_gfq **out)
{
    GFP_TRACE();
    uint32_t q;
    if (!out || !f || !gfq::order_params(p, k, q)) return GFP_ERR_INVALID;
    *out = nullptr;
    for (uint32_t j = 0; j < k; ++j)
        if (f[j] >= p) return GFP_ERR_INVALID;
    std::vector<uint32_t> expv, logv;
    if (!gfq::powers_of_x(p, k, f, q, expv, logv)) return GFP_ERR_INVALID;
    const uint32_t qbar = q - 1;
    // Z[t] = code of 1 + x^t: add 1 to the constant digit of x^t
    std::vector<uint16_t> zech(gfq::TABLE, 0);
    for (uint32_t t = 0; t < qbar; ++t) {
        uint32_t v = expv[t];
        const uint32_t d0 = v % p;
        v = v - d0 + (d0 + 1) % p;
        zech[t] = (uint16_t)(v == 0 ? 0 : logv[v]);
    }
    std::vector<uint32_t> expc(qbar + 1, 0);   // code -> value
    for (uint32_t c = 1; c <= qbar; ++c) expc[c] = expv[c % qbar];
    // the same as uint16 (values < q <= 2^16); entry 0 holds x^0 = 1 like entry
    // qbar, so that a product code reduced by min(c, c - qbar) may land on 0
    std::vector<uint16_t> exp16(gfq::TABLE, 0);
    for (uint32_t c = 1; c <= qbar; ++c) exp16[c] = (uint16_t)expc[c];
    exp16[0] = (uint16_t)expc[qbar];
    // small odd-characteristic extensions: code -> value (uint8) and the value
    // addition table (digit-wise sums mod p of the base-p values)
    const bool small_ext = p != 2 && k > 1 && q <= 256;
    std::vector<uint8_t> tab8;
    if (small_ext) {
        tab8.assign(((size_t)256 + (size_t)q * q + 15) & ~(size_t)15, 0);
        for (uint32_t c = 1; c <= qbar; ++c) tab8[c] = (uint8_t)expc[c];
        tab8[0] = (uint8_t)expc[qbar];
        for (uint32_t a = 0; a < q; ++a)
            for (uint32_t b = 0; b < q; ++b) {
                uint32_t r = 0, pw = 1, u = a, w = b;
                for (uint32_t j = 0; j < k; ++j, pw *= p, u /= p, w /= p) r += ((u % p + w % p) % p) * pw;
                tab8[256 + (size_t)a * q + b] = (uint8_t)r;
            }
    }

    int sms = 0;
    GFQ_TRY(cudaSetDevice(device));
    GFQ_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
    GFQ_TRY(cudaFuncSetAttribute(gfq::k_gfq_dot<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)gfq::SMEM));
    GFQ_TRY(cudaFuncSetAttribute(gfq::k_gfq_dot<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)gfq::SMEM));
    GFQ_TRY(cudaFuncSetAttribute(gfq::k_gfq_dot_exp<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)gfq::SMEM));
    GFQ_TRY(cudaFuncSetAttribute(gfq::k_gfq_dot_exp<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)gfq::SMEM));
    GFQ_TRY(cudaFuncSetAttribute(gfq::k_gfq_dot_add, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 256 + 256 * 256));
    gfp_gfq *fq = new gfp_gfq;
    fq->device = device;
    fq->p = p;
    fq->k = k;
    fq->q = q;
    fq->qbar = qbar;
    for (uint32_t j = 0; j < k; ++j) fq->f[j] = f[j];
    fq->grid = std::max(1, sms);
    fq->mode = p == 2 ? 2 : (k == 1 ? 1 : (small_ext ? 3 : 0));
    cudaError_t e = cudaSuccess;
    auto alloc = [&](void **ptr, size_t bytes) {
        if (e == cudaSuccess) e = cudaMalloc(ptr, bytes);
    };
    alloc((void **)&fq->d_zech, gfq::SMEM);
    alloc((void **)&fq->d_log, (size_t)q * 4);
    alloc((void **)&fq->d_exp, (size_t)(qbar + 1) * 4);
    alloc((void **)&fq->d_partials, (size_t)fq->grid * 4);
    alloc((void **)&fq->d_ticket, 4);
    alloc((void **)&fq->d_err, 4);
    alloc((void **)&fq->d_exp16, gfq::SMEM);
    alloc((void **)&fq->d_acc, 8);
    if (small_ext) {
        fq->tab8_bytes = (uint32_t)tab8.size();
        alloc((void **)&fq->d_tab8, tab8.size());
    }
    if (e == cudaSuccess) e = cudaMemcpy(fq->d_zech, zech.data(), gfq::SMEM, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(fq->d_log, logv.data(), (size_t)q * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(fq->d_exp, expc.data(), (size_t)(qbar + 1) * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(fq->d_ticket, 0, 4);
    if (e == cudaSuccess) e = cudaMemset(fq->d_err, 0, 4);
    if (e == cudaSuccess) e = cudaMemcpy(fq->d_exp16, exp16.data(), gfq::SMEM, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(fq->d_acc, 0, 8);
    if (e == cudaSuccess && small_ext)
        e = cudaMemcpy(fq->d_tab8, tab8.data(), tab8.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        note_cuda_error(e);
        gfp_gfq_destroy(fq);
        return e == cudaErrorMemoryAllocation ? GFP_ERR_NOMEM : GFP_ERR_CUDA;
    }
    *out = fq;
    return GFP_OK;
}

GFP_API gfp_status gfp_gfq_destroy(gfp_gfq *fq)
{
    GFP_TRACE();
    if (!fq) return GFP_ERR_INVALID;
    cudaSetDevice(fq->device);
    cudaFree(fq->d_zech);
    cudaFree(fq->d_log);
    cudaFree(fq->d_exp);
    cudaFree(fq->d_partials);
    cudaFree(fq->d_ticket);
    cudaFree(fq->d_err);
    cudaFree(fq->d_exp16);
    cudaFree(fq->d_tab8);
    cudaFree(fq->d_acc);
    delete fq;
    return GFP_OK;
}

GFP_API gfp_status gfp_gfq_info(const gfp_gfq *fq, uint32_t *p, uint32_t *k, uint32_t *q)
{
    if (!fq) return GFP_ERR_INVALID;
    if (p) *p = fq->p;
    if (k) *k = fq->k;
    if (q) *q = fq->q;
    return GFP_OK;
}

static int conv_grid(const gfp_gfq *fq, uint64_t n)
{
    const uint64_t want = (n + 255) / 256;
    return (int)std::max<uint64_t>(1, std::min<uint64_t>(want, (uint64_t)fq->grid * 8));
}

GFP_API gfp_status gfp_gfq_to_log(gfp_gfq *fq, uint64_t n, const uint32_t *values, uint16_t *codes,
                                  void *stream)
{
    GFP_TRACE();
    if (!fq || (n && (!values || !codes))) return GFP_ERR_INVALID;
    if (n == 0) return GFP_OK;
    GFQ_TRY(cudaSetDevice(fq->device));
    gfq::k_gfq_to_log<<<conv_grid(fq, n), 256, 0, (cudaStream_t)stream>>>(values, n, fq->d_log, fq->q,
                                                                          codes, fq->d_err);
    GFQ_TRY(cudaGetLastError());
    return GFP_OK;
}

GFP_API gfp_status gfp_gfq_from_log(gfp_gfq *fq, uint64_t n, const uint16_t *codes, uint32_t *values,
                                    void *stream)
{
    GFP_TRACE();
    if (!fq || (n && (!values || !codes))) return GFP_ERR_INVALID;
    if (n == 0) return GFP_OK;
    GFQ_TRY(cudaSetDevice(fq->device));
    gfq::k_gfq_from_log<<<conv_grid(fq, n), 256, 0, (cudaStream_t)stream>>>(codes, n, fq->d_exp, fq->qbar,
                                                                            values, fq->d_err);
    GFQ_TRY(cudaGetLastError());
    return GFP_OK;
}

GFP_API gfp_status gfp_gfq_dot(gfp_gfq *fq, uint64_t n, const uint16_t *x, const uint16_t *y, uint16_t *out,
                               void *stream)
{
    GFP_TRACE();
    if (!fq || !out || (n && (!x || !y))) return GFP_ERR_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    GFQ_TRY(cudaSetDevice(fq->device));
    if (n == 0) {
        GFQ_TRY(cudaMemsetAsync(out, 0, sizeof(uint16_t), s));
        return GFP_OK;
    }
    const int vec = ((((uintptr_t)x) | ((uintptr_t)y)) & 15u) == 0 ? 1 : 0;
    const uint64_t work = vec ? (n + 7) / 8 : n;
    const int grid = (int)std::max<uint64_t>(1, std::min<uint64_t>((uint64_t)fq->grid,
                                                                    (work + gfq::THREADS - 1) / gfq::THREADS));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(gfq::THREADS);
    cfg.dynamicSmemBytes = gfq::SMEM;
    cfg.stream = s;
    cudaLaunchAttribute pdl[1];
    pdl[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    pdl[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = pdl;
    cfg.numAttrs = 1;
    if (fq->mode == 1) {
        GFQ_TRY(cudaLaunchKernelEx(&cfg, gfq::k_gfq_dot_exp<false>, x, y, n, vec,
                                   (const uint16_t *)fq->d_exp16, fq->qbar, fq->p,
                                   (const uint32_t *)fq->d_log, fq->d_acc, fq->d_ticket, out));
    } else if (fq->mode == 2) {
        GFQ_TRY(cudaLaunchKernelEx(&cfg, gfq::k_gfq_dot_exp<true>, x, y, n, vec,
                                   (const uint16_t *)fq->d_exp16, fq->qbar, fq->p,
                                   (const uint32_t *)fq->d_log, fq->d_acc, fq->d_ticket, out));
    } else if (fq->mode == 3) {
        cfg.dynamicSmemBytes = fq->tab8_bytes;
        GFQ_TRY(cudaLaunchKernelEx(&cfg, gfq::k_gfq_dot_add, x, y, n, vec, (const uint8_t *)fq->d_tab8,
                                   (uint32_t)fq->tab8_bytes, (uint32_t)fq->q, fq->qbar,
                                   (const uint32_t *)fq->d_log, fq->d_partials, fq->d_ticket, out));
    } else if (fq->q >= gfq::RARE_Q) {
        GFQ_TRY(cudaLaunchKernelEx(&cfg, gfq::k_gfq_dot<true>, x, y, n, vec,
                                   (const uint16_t *)fq->d_zech, fq->qbar, fq->d_partials,
                                   fq->d_ticket, out));
    } else {
        GFQ_TRY(cudaLaunchKernelEx(&cfg, gfq::k_gfq_dot<false>, x, y, n, vec,
                                   (const uint16_t *)fq->d_zech, fq->qbar, fq->d_partials,
                                   fq->d_ticket, out));
    }
    GFQ_TRY(cudaGetLastError());
    return GFP_OK;
}

GFP_API gfp_status gfp_gfq_check(gfp_gfq *fq)
{
    GFP_TRACE();
    if (!fq) return GFP_ERR_INVALID;
    GFQ_TRY(cudaSetDevice(fq->device));
    GFQ_TRY(cudaDeviceSynchronize());
    uint32_t err = 0;
    GFQ_TRY(cudaMemcpy(&err, fq->d_err, 4, cudaMemcpyDeviceToHost));
    if (err) {
        GFQ_TRY(cudaMemset(fq->d_err, 0, 4));
        return GFP_ERR_RANGE;
    }
    return GFP_OK;
}

}  // extern "C"
