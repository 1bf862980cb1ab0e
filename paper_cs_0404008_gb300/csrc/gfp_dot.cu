// Dot-product kernels of libgfpdot: single dot, persistent batched dot over
// uneven (pair, chunk) work units with mixed moduli, the device input
// generator and the input range check.
//
// Data path (all representations): 128-bit coalesced loads of uint32
// residues, a per-thread unreduced accumulator (Section 3 of the paper),
// one reduction per thread, a warp-shuffle plus shared-memory combine of the
// thread residues, one 64-bit atomic add per CTA into the output's slot, and a
// single final reduction by the last CTA to finish (found by a ticket counter
// in the batched kernel, by a CTA count packed into the slot itself in the
// single-dot kernel).  The last CTA returns slots and tickets to zero, so the
// scratch is reusable by the next launch without a memset.
#include "gfp_internal.h"

namespace gfp {

#ifdef GFP_DEVICE_CHECKS
__device__ uint32_t g_dot_check;
uint32_t dot_check_bits()
{
    uint32_t h = 0, z = 0;
    if (cudaMemcpyFromSymbol(&h, g_dot_check, 4) != cudaSuccess) return 0;
    cudaMemcpyToSymbol(g_dot_check, &z, 4);
    return h;
}
#else
uint32_t dot_check_bits() { return 0; }
#endif

__device__ __forceinline__ uint4 ld_stream4(const uint4 *p) { return __ldcs(p); }
__device__ __forceinline__ uint32_t ld_stream1(const uint32_t *p) { return __ldcs(p); }

// Thread `t` of a group of T threads accumulates its share of elements
// [b, e) of x and y.  When x+b and y+b are 16-byte aligned (b is a multiple of
// 4 for every caller) the loop issues U 128-bit loads of each operand before
// consuming them; otherwise 32-bit loads (still coalesced across a warp).
template <class Acc, int U>
__device__ __forceinline__ void accumulate_range(Acc &acc, const Mod &m, const uint32_t *x,
                                                 const uint32_t *y, uint64_t b, uint64_t e,
                                                 uint64_t t, uint64_t T)
{
    if (e <= b) return;
    const bool vec = ((((uintptr_t)(x + b)) | ((uintptr_t)(y + b))) & 15u) == 0;
    if (vec) {
        const uint4 *xv = reinterpret_cast<const uint4 *>(x + b);
        const uint4 *yv = reinterpret_cast<const uint4 *>(y + b);
        const uint64_t nv = (e - b) >> 2;
        uint64_t v = t;
        for (; v + (U - 1) * T < nv; v += U * T) {
            uint4 a[U], c[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                a[u] = ld_stream4(xv + v + u * T);
                c[u] = ld_stream4(yv + v + u * T);
            }
#pragma unroll
            for (int u = 0; u < U; ++u) acc.add4(a[u], c[u], m);
        }
        for (; v < nv; v += T) acc.add4(ld_stream4(xv + v), ld_stream4(yv + v), m);
        const uint64_t i = b + (nv << 2) + t;   // fewer than 4 tail elements, T >= 4
        if (i < e) acc.add(ld_stream1(x + i), ld_stream1(y + i), m);
    } else {
        constexpr int S = 4 * U;
        uint64_t i = b + t;
        for (; i + (S - 1) * T < e; i += S * T) {
            uint32_t a[S], c[S];
#pragma unroll
            for (int u = 0; u < S; ++u) {
                a[u] = ld_stream1(x + i + u * T);
                c[u] = ld_stream1(y + i + u * T);
            }
#pragma unroll
            for (int u = 0; u < S; ++u) acc.add(a[u], c[u], m);
        }
        for (; i < e; i += T) acc.add(ld_stream1(x + i), ld_stream1(y + i), m);
    }
}

// Sum of one uint64 per thread over the CTA; the result is valid in thread 0.
// Ends with a barrier so the shared buffer may be reused immediately.
__device__ __forceinline__ uint64_t cta_sum(uint64_t v)
{
    __shared__ uint64_t sh[32];
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) sh[w] = v;
    __syncthreads();
    if (w == 0) {
        v = (l < (int)(blockDim.x >> 5)) ? sh[l] : 0;
#pragma unroll
        for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    }
    __syncthreads();
    return v;
}

// Called by thread 0 with the CTA's residue sum for one output: adds it to the
// slot; the CTA that brings the ticket to `expected` reduces the slot into
// *out and returns slot and ticket to zero.
__device__ __forceinline__ void combine_and_finish(uint64_t cta_total, const Mod &m,
                                                   unsigned long long *slot, uint32_t *ticket,
                                                   uint32_t expected, uint32_t *out)
{
    atomicAdd(slot, (unsigned long long)reduce64(cta_total, m));
    __threadfence();
    const uint32_t done = atomicAdd(ticket, 1u);
    if (done == expected - 1) {
        __threadfence();
        const unsigned long long v = atomicExch(slot, 0ull);
        atomicExch(ticket, 0u);
        *out = reduce64((uint64_t)v, m);
    }
}

// Single-dot combine in one atomic: each CTA adds its residue (below 2^32)
// plus 2^48 to a 64-bit slot, so the low 48 bits collect the residue sum and
// the high 16 bits count the CTAs (a grid of at most 2^16 - 1 CTAs keeps the
// sum below 2^48).  The CTA whose add returns a count of grid - 1 holds every
// other contribution in the returned value: it reduces the total into *out
// and returns the slot to zero; no fence or second atomic is needed.
__device__ __forceinline__ void combine_packed(uint64_t cta_total, const Mod &m,
                                               unsigned long long *slot, uint32_t ctas,
                                               uint32_t *out)
{
    const uint64_t r = reduce64(cta_total, m);
    const unsigned long long old = atomicAdd(slot, (unsigned long long)r + (1ull << 48));
    if ((uint32_t)(old >> 48) == ctas - 1) {
        *slot = 0ull;
        *out = reduce64((old & ((1ull << 48) - 1)) + r, m);
    }
}

template <class Acc>
__global__ void __launch_bounds__(DOT_THREADS)
    k_dot_single(Mod m, uint64_t k, uint64_t n, const uint32_t *__restrict__ x,
                 const uint32_t *__restrict__ y, unsigned long long *slot, uint32_t *out)
{
    // Programmatic dependent launch: let the next kernel of the stream be
    // scheduled now, and wait here until the previous one has finished and
    // its writes are visible (it may have produced x or y).
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    asm volatile("griddepcontrol.wait;" ::: "memory");
    Acc acc;
    acc.init(m, k);
    const uint64_t T = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    accumulate_range<Acc, 4>(acc, m, x, y, 0, n, t, T);
    const uint64_t s = cta_sum(acc.residue(m));
    if (threadIdx.x == 0) combine_packed(s, m, slot, gridDim.x, out);
}

template <class Acc>
__device__ __forceinline__ uint32_t unit_residue(const DevPair &pr, const DevUnit &un)
{
    Acc acc;
    acc.init(pr.m, pr.k);
    accumulate_range<Acc, 4>(acc, pr.m, pr.x, pr.y, un.begin, un.end, threadIdx.x, blockDim.x);
    return acc.residue(pr.m);
}

// Persistent batched kernel: CTAs pull work units from a global counter until
// the list is exhausted; the representation is chosen per pair.  The last CTA
// to leave returns both counters to zero.
__global__ void __launch_bounds__(DOT_THREADS)
    k_dot_batched(const DevPair *__restrict__ pairs, const DevPairAux *__restrict__ aux,
                  const DevUnit *__restrict__ units, uint32_t n_units, BatchScratch sc,
                  uint32_t *__restrict__ out)
{
    __shared__ uint32_t s_u;
    for (;;) {
        if (threadIdx.x == 0) s_u = atomicAdd(&sc.ctr[0], 1u);
        __syncthreads();
        const uint32_t u = s_u;
        if (u >= n_units) break;
        const DevUnit un = units[u];
        const DevPair pr = pairs[un.pair];
        const DevPairAux ax = aux[un.pair];
        GFP_DCHECK(g_dot_check, un.begin <= un.end && un.end <= pr.n, DCHECK_DOT_UNIT);
        uint32_t r;
        switch (ax.repr) {
        case U64_BLOCK: r = unit_residue<AccBlock>(pr, un); break;
        case U64_CARRY: r = unit_residue<AccCarry>(pr, un); break;
        case FP64: r = unit_residue<AccF64>(pr, un); break;
        case CENTERED: r = unit_residue<AccCentered>(pr, un); break;
        case MONTGOMERY: r = unit_residue<AccMontgomery>(pr, un); break;
        default: r = unit_residue<AccPerTerm>(pr, un); break;
        }
        const uint64_t s = cta_sum(r);   // its barriers also order the reuse of s_u
        if (threadIdx.x == 0)
            combine_and_finish(s, pr.m, sc.slots + un.pair, sc.tickets + un.pair, ax.units,
                               out + un.pair);
    }
    if (threadIdx.x == 0) {
        __threadfence();
        const uint32_t d = atomicAdd(&sc.ctr[1], 1u);
        if (d == gridDim.x - 1) {
            atomicExch(&sc.ctr[0], 0u);
            atomicExch(&sc.ctr[1], 0u);
        }
    }
}

// ---- synthetic inputs: counter-based SplitMix64 (see gfp_fill_uniform) ----

__device__ __forceinline__ uint64_t mix64(uint64_t z)
{
    z ^= z >> 30;
    z *= 0xBF58476D1CE4E5B9ull;
    z ^= z >> 27;
    z *= 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__global__ void k_fill_uniform(uint32_t p, uint64_t key, uint64_t offset, uint64_t n,
                               uint32_t *out)
{
    const uint64_t T = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += T)
        out[i] = (uint32_t)(mix64(key + 0x9E3779B97F4A7C15ull * (offset + i + 1)) % p);
}

// the same sequence laid out as a rows x cols matrix with leading dimension ld:
// out[r*ld + c] = word(r*cols + c) mod p
__global__ void k_fill_uniform_2d(uint32_t p, uint64_t key, uint64_t rows, uint64_t cols, uint64_t ld,
                                  uint32_t *out)
{
    const uint64_t T = (uint64_t)gridDim.x * blockDim.x, n = rows * cols;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += T)
        out[(i / cols) * ld + i % cols] = (uint32_t)(mix64(key + 0x9E3779B97F4A7C15ull * (i + 1)) % p);
}

__global__ void k_check_range(const uint32_t *v, uint64_t n, uint32_t p, uint32_t *flag)
{
    const uint64_t T = (uint64_t)gridDim.x * blockDim.x;
    bool bad = false;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += T)
        bad |= (v[i] >= p);
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(flag, 1u);
}

// ---- launchers ----

template <class Acc>
static int occupancy_single()
{
    static int occ = 0;
    if (!occ) {
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_dot_single<Acc>, DOT_THREADS,
                                                          0) != cudaSuccess || occ < 1)
            occ = 1;
    }
    return occ;
}

static int occupancy_for(Repr r)
{
    switch (r) {
    case U64_BLOCK: return occupancy_single<AccBlock>();
    case U64_CARRY: return occupancy_single<AccCarry>();
    case FP64: return occupancy_single<AccF64>();
    case CENTERED: return occupancy_single<AccCentered>();
    case MONTGOMERY: return occupancy_single<AccMontgomery>();
    default: return occupancy_single<AccPerTerm>();
    }
}

int dot_single_grid(Repr r, uint64_t n, int sm_count)
{
    const uint64_t per_cta = (uint64_t)DOT_THREADS * 16;   // 4 vectors of 4 per thread
    uint64_t want = (n + per_cta - 1) / per_cta;
    const uint64_t cap = (uint64_t)sm_count * occupancy_for(r);
    if (want < 1) want = 1;
    want = want < cap ? want : cap;
    return (int)(want < 65535 ? want : 65535);   // the packed combine counts CTAs in 16 bits
}

template <class Acc>
static cudaError_t launch_single_pdl(const Mod &m, uint64_t k, uint64_t n, const uint32_t *x,
                                     const uint32_t *y, unsigned long long *slot, uint32_t *out,
                                     int grid, cudaStream_t s)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(DOT_THREADS);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_dot_single<Acc>, m, k, n, x, y, slot, out);
}

cudaError_t launch_dot_single(Repr r, const Mod &m, uint64_t k, uint64_t n, const uint32_t *x,
                              const uint32_t *y, unsigned long long *slot, uint32_t *out, int grid,
                              cudaStream_t s)
{
    cudaError_t e;
    switch (r) {
    case U64_BLOCK: e = launch_single_pdl<AccBlock>(m, k, n, x, y, slot, out, grid, s); break;
    case U64_CARRY: e = launch_single_pdl<AccCarry>(m, k, n, x, y, slot, out, grid, s); break;
    case FP64: e = launch_single_pdl<AccF64>(m, k, n, x, y, slot, out, grid, s); break;
    case CENTERED: e = launch_single_pdl<AccCentered>(m, k, n, x, y, slot, out, grid, s); break;
    case MONTGOMERY: e = launch_single_pdl<AccMontgomery>(m, k, n, x, y, slot, out, grid, s); break;
    default: e = launch_single_pdl<AccPerTerm>(m, k, n, x, y, slot, out, grid, s); break;
    }
    return e != cudaSuccess ? e : cudaGetLastError();
}

int dot_batched_grid(int sm_count)
{
    static int occ = 0;
    if (!occ) {
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_dot_batched, DOT_THREADS, 0) !=
                cudaSuccess || occ < 1)
            occ = 1;
    }
    return sm_count * occ;
}

cudaError_t launch_dot_batched(const DevPair *pairs, const DevPairAux *aux, const DevUnit *units,
                               uint32_t n_units, BatchScratch sc, uint32_t *out, int grid,
                               cudaStream_t s)
{
    k_dot_batched<<<grid, DOT_THREADS, 0, s>>>(pairs, aux, units, n_units, sc, out);
    return cudaGetLastError();
}

static uint64_t fill_key(uint64_t seed, uint64_t stream_id)
{
    uint64_t z = seed + 0x9E3779B97F4A7C15ull * (stream_id + 1);
    z ^= z >> 30; z *= 0xBF58476D1CE4E5B9ull; z ^= z >> 27; z *= 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

cudaError_t launch_fill_uniform(uint32_t p, uint64_t seed, uint64_t stream_id, uint64_t offset,
                                uint64_t n, uint32_t *out, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    uint64_t blocks = (n + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    k_fill_uniform<<<(unsigned)blocks, 256, 0, s>>>(p, fill_key(seed, stream_id), offset, n, out);
    return cudaGetLastError();
}

cudaError_t launch_fill_uniform_2d(uint32_t p, uint64_t seed, uint64_t stream_id, uint64_t rows,
                                   uint64_t cols, uint64_t ld, uint32_t *out, cudaStream_t s)
{
    const uint64_t n = rows * cols;
    if (n == 0) return cudaSuccess;
    uint64_t blocks = (n + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    k_fill_uniform_2d<<<(unsigned)blocks, 256, 0, s>>>(p, fill_key(seed, stream_id), rows, cols, ld, out);
    return cudaGetLastError();
}

cudaError_t launch_check_range(const uint32_t *v, uint64_t n, uint32_t p, uint32_t *flag,
                               cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    uint64_t blocks = (n + 255) / 256;
    if (blocks > 2048) blocks = 2048;
    k_check_range<<<(unsigned)blocks, 256, 0, s>>>(v, n, p, flag);
    return cudaGetLastError();
}

}  // namespace gfp
