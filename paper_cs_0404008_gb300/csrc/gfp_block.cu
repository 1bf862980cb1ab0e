// Block product over GF(p): C = A B mod p, A m x k, B k x nb (row-major
// uint32 residues), the dense contraction at the heart of block methods.
//
// Tensor-core path (p <= 65791, the centred residues of Section 3.2.2 then
// fit two balanced 8-bit digits):
//   a in [0, p) is centred to s in [-(p-1)/2, (p-1)/2] and split exactly as
//   s = 256 h + l with l in [-128, 127], h in [-128, 128].  Every digit is an
//   exact fp16 value and every digit product is an integer of magnitude at
//   most 2^14, so 1024 of them sum to at most 2^24: exact in an fp32
//   accumulator.  A and B digits therefore go through tcgen05.mma kind::f16
//   with fp32 accumulation in TMEM, and every 1024 terms (the exact chunk,
//   Eq. (1) read with m = 24 for the fp32 significand) the four digit-product
//   accumulators are recombined as hh*2^16 + (hl + lh)*2^8 + ll in int64,
//   reduced mod p, and summed as residues.  Nothing is approximated.
//   Roles per CTA (one CTA per SM, persistent over (tile, chunk) units):
//     warp 0      TMA-loads uint32 A boxes (two 64-deep k-blocks per slot)
//                 from HBM into a ring of shared-memory slots (a prepared A:
//                 bulk-copies its 8-bit digit planes, one k-block per slot)
//     warp 1      owns TMEM and issues the MMAs (one thread)
//     warp 2      bulk-copies the pre-split B digit tiles (own ring)
//     warps 3-10  read a landed A box into registers, centre and split it,
//                 and write the two fp16 digit tiles in place over it
//                 (128-byte-swizzled, K-major), the same 32 KiB per k-block
//                 (a prepared A: widen its 8-bit digits to the same tiles)
//     warps 11-14 drain the accumulators (tcgen05.ld), recombine, reduce
//   B's digits are stacked [hi | lo] along N (N = 128 per MMA), so one MMA
//   per A digit yields both products with that digit; the two MMAs of a K
//   step accumulate into separate TMEM columns (two independent chains).
//   Units of one output tile may be split over several CTAs: each adds its
//   residue sums for the tile into a column-major u32 workspace (coalesced
//   atomics, one transaction per column and warp), and a small kernel behind
//   this one reduces the sums mod p, writes C through a shared-memory
//   transpose and clears the workspace.
//
// Larger moduli on the tensor cores (p > 65791): the exact integer products
// sum_t A[i][t] B[t][j] are below k (p-1)^2, so they are fixed by their
// residues modulo a few small primes p' <= 65536 whose product exceeds that
// bound (a residue number system).  Each pass runs the tensor-core kernel
// above modulo one p', reducing every input a < 2^32 to a mod p' while it is
// split into digits; a last kernel recombines the residues with Garner's
// mixed-radix method and evaluates the integer modulo p.
//
// CUDA-core path (any p <= 2^32-1): shared-memory tiled product with the
// per-thread unreduced accumulators of the dot-product kernels.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <cstring>
#include <mutex>

#include "gfp_internal.h"
#include "gfp_tc.cuh"

namespace gfp {
namespace blk {

constexpr int BM = 128;            // rows per tile (MMA M)
constexpr int BK = 64;             // K per k-block: one 128-byte swizzle row of fp16
constexpr int NT = 64;             // output columns per n-tile
constexpr int MMA_N = 2 * NT;      // hi and lo digits of B stacked along N
constexpr int KC = 16;             // k-blocks per exact chunk (1024 terms)
constexpr int A_TILE_BYTES = BM * BK * 4;                     // 32 KiB of uint32 per k-block
constexpr int A_DIGIT_BYTES = BM * BK * 2;                    // 16 KiB per digit
constexpr int B_TILE_BYTES = MMA_N * BK * 2;                  // 16 KiB
static_assert(A_TILE_BYTES == 2 * A_DIGIT_BYTES, "in-place conversion needs equal sizes");
constexpr int CONV_WARPS = 8;
constexpr int EPI_WARPS = 4;
constexpr int W_APROD = 0, W_MMA = 1, W_BPROD = 2, W_CONV0 = 3, W_EPI0 = W_CONV0 + CONV_WARPS;
constexpr int THREADS = 32 * (W_EPI0 + EPI_WARPS);            // 480
constexpr uint32_t TMEM_COLS = 512;   // 2 accumulator sets x 2 digits x 128 columns
constexpr uint64_t WAIT_NS = 2000000000ull;   // bounded waits: 2 s
constexpr uint32_t IDESC = ptx::idesc_f16_f32(BM, MMA_N);

// Pipeline depths: SLOTS shared-memory slots of KBB k-blocks of A each, and
// BSTAGES B digit tiles.  A slot receives a uint32 box (TMA) that the
// converter warps turn into fp16 digit tiles in place, or, for a prepared A,
// a tile of 8-bit digit planes (bulk copy) that they widen in place.  The
// uint32 path measured fastest with three two-k-block slots (longer TMA row
// bursts) and two B stages; the prepared path with five one-k-block slots
// and four B stages.
template <int SLOTS_, int BSTAGES_, int KBB_>
struct Pipe {
    static constexpr int SLOTS = SLOTS_, BSTAGES = BSTAGES_, KBB = KBB_;
    static constexpr int SLOT_BYTES = KBB * A_TILE_BYTES;
    struct Bars {
        uint64_t a_full[SLOTS];    // A tile landed (1 arrival + tx bytes)
        uint64_t conv[SLOTS];      // digits written in place (one arrival per converter warp)
        uint64_t a_empty[SLOTS];   // MMAs reading the digits completed (tcgen05.commit)
        uint64_t full_b[BSTAGES];  // B digit tile landed (1 arrival + tx bytes)
        uint64_t empty_b[BSTAGES]; // MMAs reading the B tile completed (tcgen05.commit)
        uint64_t acc_full[2];      // accumulator set ready (tcgen05.commit)
        uint64_t acc_empty[2];     // accumulator set drained (one arrival per epilogue warp)
        uint64_t drain;            // all MMAs issued by this CTA completed
        uint32_t tmem_base;
        uint32_t abort;
    };
    static constexpr size_t SMEM_BYTES = 1024 /*alignment slack*/ + (size_t)SLOTS * SLOT_BYTES +
                                         (size_t)BSTAGES * B_TILE_BYTES + 1024;
    static_assert(sizeof(Bars) <= 1024, "barriers fit their reserve");
    static_assert(SMEM_BYTES <= 232448, "shared memory per block");
};
using PipeU32 = Pipe<3, 2, 2>;    // uint32 A, converted in place
using PipePrep = Pipe<5, 4, 1>;   // prepared A: 8-bit digit planes, widened in place
static_assert(PipePrep::KBB == 1, "one prepared tile per slot");

// Prepared A (gfp_block_prepare): per (m-tile, k-block) two planes of 8-bit
// digits, high then low, each 128 rows x 64 K, row-major, every digit stored
// with a bias of 128.  A residue a of p <= 65536 is represented by s = a or
// a - p in [-32896, 32639] (s = a when a <= min((p-1)/2, 32639)), split as
// s = 256 h + l with h, l in [-128, 127]: u = s + 32896 in [0, 65535] holds
// h + 128 in its high byte and l + 128 in its low byte.  Every digit is still
// at most 128 in magnitude, so the 1024-term fp32 chunks stay exact.
constexpr int A8_PLANE_BYTES = BM * BK;           // 8 KiB per digit plane
constexpr int A8_TILE_BYTES = 2 * A8_PLANE_BYTES; // 16 KiB per (m-tile, k-block)
constexpr uint32_t DIGIT8_MAX_P = 65536;

struct Args {
    CUtensorMap tmap_a;       // A as a 2-D uint32 tensor {k, m}, box {BK*KBB, BM} (uint32 pipe), zero fill
    uint64_t m, k, nb;
    const uint8_t *Bimg;      // [n_tiles][kblocks] tiles of B_TILE_BYTES
    const uint8_t *Aimg;      // prepared A: [m_tiles][kblocks] tiles of A8_TILE_BYTES (PREP)
    uint32_t *C;
    uint64_t ldc;
    uint32_t *Cacc;           // (n_tiles*NT) x m u32 partial residue sums, column-major: the
                              // entry of row i, column j at j*m + i (zero outside calls)
    uint32_t *err;            // bit 0: a bounded wait expired
    Mod mod;
    uint64_t off;             // multiple of p >= 2^41 making recombined values non-negative
    uint32_t pre_magic;       // floor(2^32 / p) for the input reduction of the residue passes
    uint32_t half;            // (p-1)/2
    uint32_t m_tiles, n_tiles, kblocks, chunks;
    uint64_t units;
};

// Bounded wait on an mbarrier phase: gives up after limit_ns (or as soon as
// another role of the CTA has given up), sets the CTA abort flag and bit 0 of
// the error word, and returns false.
__device__ __forceinline__ bool wait_bar(uint32_t bar, uint32_t parity, volatile uint32_t *abort,
                                         uint32_t *err, uint64_t limit_ns = WAIT_NS)
{
    uint64_t t0 = 0;
    for (uint32_t i = 0;; ++i) {
        if (ptx::mbar_try_wait(bar, parity)) return true;
        if ((i & 255u) == 255u) {
            if (*abort) return false;
            const uint64_t t = ptx::globaltimer();
            if (t0 == 0) t0 = t;
            else if (t - t0 > limit_ns) {
                *abort = 1u;
                atomicOr(err, 1u);
                return false;
            }
        }
    }
}

// Failure-detection self test: one thread waits on an mbarrier that nothing
// arrives on; the bounded wait must expire and report it in *err.
__global__ void k_wait_selftest(uint64_t limit_ns, uint32_t *err)
{
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t abort;
    if (threadIdx.x == 0) {
        ptx::mbar_init(ptx::smem_u32(&bar), 1);
        abort = 0;
        ptx::fence_barrier_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if (!wait_bar(ptx::smem_u32(&bar), 0, &abort, err, limit_ns)) atomicOr(err, 2u);
    }
}

__device__ uint32_t g_selftest_err;

// warp-uniform bounded wait: lane 0 polls, the result is broadcast
__device__ __forceinline__ bool warp_wait(uint32_t bar, uint32_t parity, volatile uint32_t *abort,
                                          uint32_t *err)
{
    bool ok = true;
    if ((threadIdx.x & 31) == 0) ok = wait_bar(bar, parity, abort, err);
    return __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
}

struct UnitPos {
    uint32_t nt, mt, c, kb0, kb1;
};

__device__ __forceinline__ UnitPos unit_pos(const Args &a, uint64_t u)
{
    UnitPos q;
    q.c = (uint32_t)(u % a.chunks);
    const uint64_t tile = u / a.chunks;
    q.mt = (uint32_t)(tile % a.m_tiles);
    q.nt = (uint32_t)(tile / a.m_tiles);
    q.kb0 = q.c * KC;
    q.kb1 = min(q.kb0 + (uint32_t)KC, a.kblocks);
    return q;
}

// Centre two residues and split each into balanced 8-bit digits, returned
// as packed fp16 pairs (element 0 in the low half).  With u = s + 32896, where
// s in [-32895, 32895] is the centred residue, the digits of s = 256 h + l are
// l = (u & 255) - 128 and h = (u >> 8) - 128.  The fp16 encoding of 1536 + d
// for an integer |d| <= 512 is the 16-bit integer 0x6600 + d (exponent of
// [1024, 2048), unit spacing), so a byte permute plus one integer add builds
// 1536 + d for both lanes and one exact fp16 subtraction leaves d.
__device__ __forceinline__ void split_pair(uint32_t a0, uint32_t a1, uint32_t p, uint32_t half,
                                           uint32_t &hi2, uint32_t &lo2)
{
    const uint32_t u0 = a0 + 32896u - (a0 > half ? p : 0u);
    const uint32_t u1 = a1 + 32896u - (a1 > half ? p : 0u);
    const uint32_t lo_bits = __byte_perm(u0, u1, 0x3430) + 0x65806580u;   // [u0 & 255, u1 & 255]
    const uint32_t hi_bits = __byte_perm(u0, u1, 0x6521) + 0x65806580u;   // [u0 >> 8, u1 >> 8]
    const __half2 bias = __halves2half2(__ushort_as_half(0x6600), __ushort_as_half(0x6600));
    const __half2 lo = __hsub2(*reinterpret_cast<const __half2 *>(&lo_bits), bias);
    const __half2 hi = __hsub2(*reinterpret_cast<const __half2 *>(&hi_bits), bias);
    lo2 = *reinterpret_cast<const uint32_t *>(&lo);
    hi2 = *reinterpret_cast<const uint32_t *>(&hi);
}

// Converter thread ct (0..255) handles 8 chunks of 4 consecutive K of one row.
// load_tile copies them from the landed uint32 tile (row-major, 256 bytes per
// row) into registers; once every converter thread has done so, store_digits
// overwrites the same 32 KiB with the two 128-byte-swizzled K-major fp16
// digit tiles (high digits first).
struct ARegs {
    uint4 v[8];
};

// sub-tile `sub` of a slot holding KBB k-blocks (row stride BK*4*KBB bytes)
template <int KBB>
__device__ __forceinline__ void load_tile(const uint8_t *slot, int sub, int ct, ARegs &r)
{
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int q = ct + 256 * i;
        const int row = q >> 4, c4 = q & 15;
        r.v[i] = *reinterpret_cast<const uint4 *>(slot + row * (BK * 4 * KBB) + sub * (BK * 4) + c4 * 16);
    }
}

// a mod p for any 32-bit a and p <= 65791: q = floor(a * floor(2^32/p) / 2^32)
// is floor(a/p) or one less, so one conditional subtraction finishes it
__device__ __forceinline__ uint32_t reduce_small(uint32_t a, uint32_t p, uint32_t magic)
{
    uint32_t r = a - __umulhi(a, magic) * p;
    return r >= p ? r - p : r;
}

template <bool PRE>
__device__ __forceinline__ void store_digits(const Args &a, const ARegs &r, uint8_t *stage, int ct)
{
    uint8_t *th = stage;                    // high digits
    uint8_t *tl = stage + A_DIGIT_BYTES;    // low digits
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int q = ct + 256 * i;
        const int row = q >> 4, c4 = q & 15;
        uint32_t h01, l01, h23, l23;
        uint4 w = r.v[i];
        if (PRE) {
            w.x = reduce_small(w.x, a.mod.p, a.pre_magic);
            w.y = reduce_small(w.y, a.mod.p, a.pre_magic);
            w.z = reduce_small(w.z, a.mod.p, a.pre_magic);
            w.w = reduce_small(w.w, a.mod.p, a.pre_magic);
        }
        split_pair(w.x, w.y, a.mod.p, a.half, h01, l01);
        split_pair(w.z, w.w, a.mod.p, a.half, h23, l23);
        // 128-byte swizzle: 16-byte chunk j of row r sits at chunk j ^ (r & 7)
        const int j = c4 >> 1, halfsel = c4 & 1;
        const uint32_t off = (uint32_t)row * 128u + ((uint32_t)(j ^ (row & 7)) << 4) + (halfsel << 3);
        *reinterpret_cast<uint2 *>(th + off) = make_uint2(h01, h23);
        *reinterpret_cast<uint2 *>(tl + off) = make_uint2(l01, l23);
    }
}

// A prepared tile's 16-byte chunk c of 1024 (thread ct takes c = ct + 256 i):
// plane c / 512, row (c / 4) mod 128, K columns 16 (c mod 4) .. + 15.  Its
// 16 biased bytes become 16 fp16 digits: the fp16 encoding of 1408 + b for a
// byte b is the 16-bit integer 0x6580 + b, and one exact subtraction of 1536
// leaves b - 128.  The two 8-digit halves land at their 128-byte-swizzled
// places of the plane's fp16 tile (high digits at slot offset 0, low at
// A_DIGIT_BYTES), the layout the MMAs read.
__device__ __forceinline__ void widen_store(uint8_t *slot, int c, uint4 w)
{
    const int d = c >> 9, row = (c >> 2) & 127, j = c & 3;
    const __half2 bias = __halves2half2(__ushort_as_half(0x6600), __ushort_as_half(0x6600));
    const uint32_t in[4] = {w.x, w.y, w.z, w.w};
    uint32_t o[8];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        const uint32_t b01 = __byte_perm(in[e], 0u, 0x4140) + 0x65806580u;   // bytes 0, 1
        const uint32_t b23 = __byte_perm(in[e], 0u, 0x4342) + 0x65806580u;   // bytes 2, 3
        const __half2 h01 = __hsub2(*reinterpret_cast<const __half2 *>(&b01), bias);
        const __half2 h23 = __hsub2(*reinterpret_cast<const __half2 *>(&b23), bias);
        o[2 * e] = *reinterpret_cast<const uint32_t *>(&h01);
        o[2 * e + 1] = *reinterpret_cast<const uint32_t *>(&h23);
    }
    uint8_t *tile = slot + (size_t)d * A_DIGIT_BYTES;
    const uint32_t r7 = (uint32_t)(row & 7), base = (uint32_t)row * 128u;
    *reinterpret_cast<uint4 *>(tile + base + (((uint32_t)(2 * j) ^ r7) << 4)) = make_uint4(o[0], o[1], o[2], o[3]);
    *reinterpret_cast<uint4 *>(tile + base + (((uint32_t)(2 * j + 1) ^ r7) << 4)) = make_uint4(o[4], o[5], o[6], o[7]);
}

// (x + y) mod p for x, y < p: the per-thread sums of chunk residues stay
// below p however many chunks a long K holds, and the u32 partial sums that
// meet in the workspace then add at most one such sum per contributing CTA
__device__ __forceinline__ uint32_t add_mod(uint32_t x, uint32_t y, uint32_t p)
{
    const uint32_t t = x + y;
    return t >= p ? t - p : t;
}

// PRE: reduce each input modulo p while splitting it (the residue passes).
// PREP: A arrives prepared, as 8-bit digit planes (k_block_prep_a); the
// producer bulk-copies a 16 KiB tile into the upper half of a slot and the
// converter warps widen it in place into the two fp16 digit tiles.
template <bool PRE, bool PREP, class P>
__global__ void __launch_bounds__(THREADS, 1) k_block_tc(const __grid_constant__ Args a)
{
    constexpr int SLOTS = P::SLOTS, BSTAGES = P::BSTAGES, KBB = P::KBB;
    constexpr int SLOT_BYTES = P::SLOT_BYTES;
    using Bars = typename P::Bars;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t *slot_mem = smem;                                  // SLOTS A slots
    uint8_t *bst = smem + (size_t)SLOTS * SLOT_BYTES;          // BSTAGES B digit tiles
    Bars *bars = reinterpret_cast<Bars *>(bst + (size_t)BSTAGES * B_TILE_BYTES);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    const uint64_t u0 = a.units * blockIdx.x / gridDim.x;
    const uint64_t u1 = a.units * (blockIdx.x + 1) / gridDim.x;

    if (threadIdx.x == 0) {
        for (int s = 0; s < SLOTS; ++s) {
            ptx::mbar_init(ptx::smem_u32(&bars->a_full[s]), 1);
            ptx::mbar_init(ptx::smem_u32(&bars->conv[s]), CONV_WARPS);
            ptx::mbar_init(ptx::smem_u32(&bars->a_empty[s]), 1);
        }
        for (int s = 0; s < BSTAGES; ++s) {
            ptx::mbar_init(ptx::smem_u32(&bars->full_b[s]), 1);
            ptx::mbar_init(ptx::smem_u32(&bars->empty_b[s]), 1);
        }
        for (int b = 0; b < 2; ++b) {
            ptx::mbar_init(ptx::smem_u32(&bars->acc_full[b]), 1);
            ptx::mbar_init(ptx::smem_u32(&bars->acc_empty[b]), EPI_WARPS);
        }
        ptx::mbar_init(ptx::smem_u32(&bars->drain), 1);
        bars->abort = 0;
        ptx::fence_barrier_init();
    }
    if (warp == W_MMA) {
        ptx::tmem_alloc(ptx::smem_u32(&bars->tmem_base), TMEM_COLS);
        ptx::tmem_relinquish();
    }
    ptx::tc_fence_before();
    __syncthreads();
    ptx::tc_fence_after();
    const uint32_t tmem = bars->tmem_base;
    volatile uint32_t *abort = &bars->abort;

    if (warp == W_APROD) {
        // ---------------- producer: uint32 A tiles (TMA) into free slots ----------------
        if (lane == 0) {
            int armed[SLOTS];
            for (int s = 0; s < SLOTS; ++s) armed[s] = -1;
            uint32_t si = 0;   // slot sequence number
            bool ok = true;
            if (!PREP) ptx::prefetch_tensormap(&a.tmap_a);
            for (uint64_t u = u0; u < u1 && ok; ++u) {
                const UnitPos q = unit_pos(a, u);
                for (uint32_t kb = q.kb0; kb < q.kb1; kb += KBB, ++si) {
                    const uint32_t s = si % SLOTS, round = si / SLOTS;
                    if (round > 0 &&
                        !wait_bar(ptx::smem_u32(&bars->a_empty[s]), (round - 1) & 1, abort, a.err)) {
                        ok = false;
                        break;
                    }
                    const uint32_t fb = ptx::smem_u32(&bars->a_full[s]);
                    if (PREP) {
                        // one prepared tile, into the slot's upper half
                        ptx::mbar_arrive_expect_tx(fb, A8_TILE_BYTES);
                        ptx::bulk_g2s(ptx::smem_u32(slot_mem + (size_t)s * SLOT_BYTES + A_DIGIT_BYTES),
                                      a.Aimg + ((uint64_t)q.mt * a.kblocks + kb) * A8_TILE_BYTES,
                                      A8_TILE_BYTES, fb);
                    } else {
                        ptx::mbar_arrive_expect_tx(fb, SLOT_BYTES);
                        ptx::tma_load_2d(ptx::smem_u32(slot_mem + (size_t)s * SLOT_BYTES), &a.tmap_a,
                                         (int)(kb * BK), (int)(q.mt * BM), fb);
                    }
                    armed[s] = (int)round;
                }
            }
            // copies already issued must land before the CTA can exit
            for (int s = 0; s < SLOTS; ++s) {
                if (armed[s] < 0) continue;
                const uint32_t fb = ptx::smem_u32(&bars->a_full[s]);
                const uint64_t t0 = ptx::globaltimer();
                while (!ptx::mbar_try_wait(fb, armed[s] & 1) && ptx::globaltimer() - t0 < WAIT_NS) {
                }
            }
        }
    } else if (warp == W_BPROD) {
        // ---------------- producer: B digit tiles (bulk copies from the prepared image) ----------------
        if (lane == 0) {
            // the image is written by the B-digit kernel launched just before
            // this one (programmatic dependent launch): the only read of its
            // output, so the only role that waits for it; A's copies, barrier
            // set-up and TMEM allocation overlap its run
            asm volatile("griddepcontrol.wait;" ::: "memory");
            int armed[BSTAGES];
            for (int s = 0; s < BSTAGES; ++s) armed[s] = -1;
            uint32_t it = 0;
            bool ok = true;
            for (uint64_t u = u0; u < u1 && ok; ++u) {
                const UnitPos q = unit_pos(a, u);
                for (uint32_t kb = q.kb0; kb < q.kb1; ++kb, ++it) {
                    const uint32_t s = it % BSTAGES, round = it / BSTAGES;
                    if (round > 0 &&
                        !wait_bar(ptx::smem_u32(&bars->empty_b[s]), (round - 1) & 1, abort, a.err)) {
                        ok = false;
                        break;
                    }
                    const uint32_t fb = ptx::smem_u32(&bars->full_b[s]);
                    ptx::mbar_arrive_expect_tx(fb, B_TILE_BYTES);
                    ptx::bulk_g2s(ptx::smem_u32(bst + (size_t)s * B_TILE_BYTES),
                                  a.Bimg + ((uint64_t)q.nt * a.kblocks + kb) * B_TILE_BYTES,
                                  B_TILE_BYTES, fb);
                    armed[s] = (int)round;
                }
            }
            for (int s = 0; s < BSTAGES; ++s) {
                if (armed[s] < 0) continue;
                const uint32_t fb = ptx::smem_u32(&bars->full_b[s]);
                const uint64_t t0 = ptx::globaltimer();
                while (!ptx::mbar_try_wait(fb, armed[s] & 1) && ptx::globaltimer() - t0 < WAIT_NS) {
                }
            }
        }
    } else if (warp == W_MMA) {
        // ---------------- MMA issue (one thread) ----------------
        if (lane == 0) {
            uint32_t it = 0, si = 0;
            bool ok = true;
            uint64_t idx = 0;
            for (uint64_t u = u0; u < u1 && ok; ++u, ++idx) {
                const UnitPos q = unit_pos(a, u);
                const uint32_t b = (uint32_t)(idx & 1), use = (uint32_t)(idx >> 1);
                if (use > 0 &&
                    !wait_bar(ptx::smem_u32(&bars->acc_empty[b]), (use - 1) & 1, abort, a.err)) {
                    ok = false;
                    break;
                }
                ptx::tc_fence_after();
                const uint32_t d_hi = tmem + b * 256u;         // A high digit x [B hi | B lo]
                const uint32_t d_lo = tmem + b * 256u + 128u;  // A low digit  x [B hi | B lo]
                for (uint32_t kb = q.kb0; kb < q.kb1; ++kb, ++it) {
                    const uint32_t sub = (kb - q.kb0) % KBB;
                    const uint32_t s = si % SLOTS, round = si / SLOTS;
                    const uint32_t sb = it % BSTAGES, roundb = it / BSTAGES;
                    // the slot's fp16 digits: converted or widened in place
                    if (!wait_bar(ptx::smem_u32(&bars->full_b[sb]), roundb & 1, abort, a.err) ||
                        (sub == 0 && !wait_bar(ptx::smem_u32(&bars->conv[s]), round & 1, abort, a.err))) {
                        ok = false;
                        break;
                    }
                    ptx::tc_fence_after();
                    const uint32_t base =
                        ptx::smem_u32(slot_mem + (size_t)s * SLOT_BYTES + (size_t)sub * A_TILE_BYTES);
                    const uint64_t dah = ptx::sdesc_k_sw128(base);
                    const uint64_t dal = ptx::sdesc_k_sw128(base + A_DIGIT_BYTES);
                    const uint64_t db = ptx::sdesc_k_sw128(ptx::smem_u32(bst + (size_t)sb * B_TILE_BYTES));
#pragma unroll
                    for (int kk = 0; kk < BK / 16; ++kk) {
                        const uint32_t acc = (kb > q.kb0 || kk > 0) ? 1u : 0u;
                        // advance 16 fp16 (32 bytes) along K inside the swizzle atom
                        ptx::mma_f16(d_hi, dah + 2 * kk, db + 2 * kk, IDESC, acc);
                        ptx::mma_f16(d_lo, dal + 2 * kk, db + 2 * kk, IDESC, acc);
                    }
                    ptx::mma_commit(ptx::smem_u32(&bars->empty_b[sb]));
                    if (sub == KBB - 1 || kb + 1 == q.kb1) {   // last k-block of this slot
                        ptx::mma_commit(ptx::smem_u32(&bars->a_empty[s]));
                        ++si;
                    }
                }
                if (!ok) break;
                ptx::mma_commit(ptx::smem_u32(&bars->acc_full[b]));
            }
            // every MMA issued by this CTA has completed before TMEM is freed
            ptx::mma_commit(ptx::smem_u32(&bars->drain));
            const uint64_t t0 = ptx::globaltimer();
            while (!ptx::mbar_try_wait(ptx::smem_u32(&bars->drain), 0) &&
                   ptx::globaltimer() - t0 < WAIT_NS) {
            }
        }
    } else if (PREP && warp < W_EPI0) {
        // ---------------- converters: 8-bit digit planes -> fp16 digit tiles, in place ----------------
        const int ct = threadIdx.x - 32 * W_CONV0;   // 0..255
        uint32_t si = 0;
        for (uint64_t u = u0; u < u1; ++u) {
            const UnitPos q = unit_pos(a, u);
            bool ok = true;
            for (uint32_t kb = q.kb0; kb < q.kb1; ++kb, ++si) {
                const uint32_t s = si % SLOTS, round = si / SLOTS;
                const bool got = warp_wait(ptx::smem_u32(&bars->a_full[s]), round & 1, abort, a.err);
                // every converter warp reads its chunks before any overwrites them
                if (ptx::bar_red_or<2, CONV_WARPS * 32>(!got || *abort != 0)) {
                    ok = false;
                    break;
                }
                uint8_t *slot = slot_mem + (size_t)s * SLOT_BYTES;
                const uint4 *src = reinterpret_cast<const uint4 *>(slot + A_DIGIT_BYTES);
                uint4 w[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) w[i] = src[ct + 256 * i];
                asm volatile("bar.sync 2, %0;" ::"n"(CONV_WARPS * 32) : "memory");
#pragma unroll
                for (int i = 0; i < 4; ++i) widen_store(slot, ct + 256 * i, w[i]);
                ptx::fence_proxy_async_smem();
                __syncwarp();
                if (lane == 0) ptx::mbar_arrive(ptx::smem_u32(&bars->conv[s]));
            }
            if (!ok) break;
        }
    } else if (warp < W_EPI0) {
        // ---------------- converters: uint32 tiles -> centred fp16 digits, in place ----------------
        const int ct = threadIdx.x - 32 * W_CONV0;   // 0..255
        uint32_t si = 0;
        for (uint64_t u = u0; u < u1; ++u) {
            const UnitPos q = unit_pos(a, u);
            bool ok = true;
            for (uint32_t kb = q.kb0; kb < q.kb1; kb += KBB, ++si) {
                const uint32_t s = si % SLOTS, round = si / SLOTS;
                const bool got = warp_wait(ptx::smem_u32(&bars->a_full[s]), round & 1, abort, a.err);
                // all converter warps read the box before any overwrites it; decide together
                if (ptx::bar_red_or<2, CONV_WARPS * 32>(!got || *abort != 0)) {
                    ok = false;
                    break;
                }
                uint8_t *slot = slot_mem + (size_t)s * SLOT_BYTES;
                const uint32_t nsub = min((uint32_t)KBB, q.kb1 - kb);
                ARegs r[KBB];
#pragma unroll
                for (int sub = 0; sub < KBB; ++sub)
                    if ((uint32_t)sub < nsub) load_tile<KBB>(slot, sub, ct, r[sub]);
                asm volatile("bar.sync 2, %0;" ::"n"(CONV_WARPS * 32) : "memory");
#pragma unroll
                for (int sub = 0; sub < KBB; ++sub)
                    if ((uint32_t)sub < nsub) store_digits<PRE>(a, r[sub], slot + (size_t)sub * A_TILE_BYTES, ct);
                ptx::fence_proxy_async_smem();
                __syncwarp();
                if (lane == 0) ptx::mbar_arrive(ptx::smem_u32(&bars->conv[s]));
            }
            if (!ok) break;
        }
    } else {
        // ---------------- epilogue: TMEM -> residues ----------------
        const int quarter = warp & 3;               // TMEM lanes 32*quarter .. +31
        const int row_in_tile = quarter * 32 + lane;
        const uint32_t lane_bits = (uint32_t)(quarter * 32) << 16;
        uint32_t res[NT];
#pragma unroll
        for (int j = 0; j < NT; ++j) res[j] = 0;
        uint64_t idx = 0;
        for (uint64_t u = u0; u < u1; ++u, ++idx) {
            const UnitPos q = unit_pos(a, u);
            const uint32_t b = (uint32_t)(idx & 1), use = (uint32_t)(idx >> 1);
            const bool got = warp_wait(ptx::smem_u32(&bars->acc_full[b]), use & 1, abort, a.err);
            // decide together: the epilogue warps meet at named barriers below
            if (ptx::bar_red_or<1, EPI_WARPS * 32>(!got || *abort != 0)) break;
            ptx::tc_fence_after();
            const uint32_t d_hi = tmem + lane_bits + b * 256u;
            const uint32_t d_lo = d_hi + 128u;
#pragma unroll
            for (int g = 0; g < NT / 8; ++g) {
                uint32_t hh[8], hl[8], lh[8], ll[8];
                ptx::tmem_ld8(d_hi + g * 8, hh);
                ptx::tmem_ld8(d_hi + NT + g * 8, hl);
                ptx::tmem_ld8(d_lo + g * 8, lh);
                ptx::tmem_ld8(d_lo + NT + g * 8, ll);
                ptx::tmem_ld_wait();
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const long long vhh = __float2int_rn(__uint_as_float(hh[j]));
                    const long long vx = (long long)__float2int_rn(__uint_as_float(hl[j])) +
                                         (long long)__float2int_rn(__uint_as_float(lh[j]));
                    const long long vll = __float2int_rn(__uint_as_float(ll[j]));
                    const long long v = vhh * 65536ll + vx * 256ll + vll;
                    res[g * 8 + j] = add_mod(res[g * 8 + j], reduce64((uint64_t)(v + (long long)a.off), a.mod),
                                             a.mod.p);
                }
            }
            ptx::tc_fence_before();
            __syncwarp();
            if (lane == 0) ptx::mbar_arrive(ptx::smem_u32(&bars->acc_empty[b]));
            // end of this CTA's run of units on the output tile?
            bool flush = (u + 1 == u1);
            if (!flush) {
                const UnitPos nq = unit_pos(a, u + 1);
                flush = (nq.mt != q.mt) || (nq.nt != q.nt);
            }
            if (flush) {
                // column-major partial sums: the 32 lanes of a warp (consecutive
                // rows) add to 128 consecutive bytes, one L2 transaction per
                // column; k_block_finish reduces them into C after this kernel
                const uint64_t grow = (uint64_t)q.mt * BM + row_in_tile;
                const uint64_t col0 = (uint64_t)q.nt * NT;
                if (grow < a.m) {
#pragma unroll
                    for (int j = 0; j < NT; ++j)
                        if (col0 + j < a.nb) atomicAdd(&a.Cacc[(col0 + j) * a.m + grow], res[j]);
                }
#pragma unroll
                for (int j = 0; j < NT; ++j) res[j] = 0;
                // the epilogue warps meet after a flush: without this barrier the
                // compiler carries the flush into the next unit's drain and the
                // kernel spills about 440 bytes per thread at 128 registers
                asm volatile("bar.sync 1, %0;" ::"n"(EPI_WARPS * 32));
            }
        }
        // the kernel that reduces the partial sums may be launched now (it
        // waits for this grid to complete before reading them)
        asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    }

    ptx::tc_fence_before();
    __syncthreads();
    if (warp == W_MMA) {
        ptx::tc_fence_after();
        ptx::tmem_dealloc(tmem, TMEM_COLS);
    }
}

constexpr int FIN_THREADS = 512;
__global__ void __launch_bounds__(FIN_THREADS)
    k_block_finish(uint32_t *__restrict__ Cacc, uint64_t m, uint64_t nb, uint32_t *__restrict__ C,
                   uint64_t ldc, uint32_t p, uint32_t magic)
{
    __shared__ uint32_t t[NT][BM + 1];   // [column][row], padded against bank conflicts
    constexpr int PER = NT * BM / FIN_THREADS;
    asm volatile("griddepcontrol.wait;" ::: "memory");
    const uint64_t r0 = (uint64_t)blockIdx.x * BM, c0 = (uint64_t)blockIdx.y * NT;
    // all of a thread's loads are issued before any is used or cleared (one
    // memory latency, not one per element); consecutive threads take
    // consecutive rows of one column
    uint32_t v[PER];
#pragma unroll
    for (int e = 0; e < PER; ++e) {
        const int i = threadIdx.x + e * FIN_THREADS, c = i / BM, r = i % BM;
        v[e] = (r0 + r < m && c0 + c < nb) ? __ldcg(&Cacc[(c0 + c) * m + r0 + r]) : 0u;
    }
#pragma unroll
    for (int e = 0; e < PER; ++e) {
        const int i = threadIdx.x + e * FIN_THREADS, c = i / BM, r = i % BM;
        if (r0 + r < m && c0 + c < nb) __stcg(&Cacc[(c0 + c) * m + r0 + r], 0u);
        t[c][r] = reduce_small(v[e], p, magic);   // the sums are below 2^32
    }
    __syncthreads();
    for (int i = threadIdx.x; i < NT * BM; i += FIN_THREADS) {
        const int r = i / NT, c = i % NT;   // consecutive threads: consecutive columns of one row
        if (r0 + r < m && c0 + c < nb) C[(r0 + r) * ldc + c0 + c] = t[c][r];
    }
}


// B (k x nb, row-major) -> per (n-tile, k-block) tiles of 128 rows x 64 K
// fp16 digits in the 128-byte swizzled K-major layout: rows 0..63 hold the
// high digits of output columns nt*64 + r, rows 64..127 the low digits.
__global__ void k_block_prep_b(const uint32_t *B, uint64_t ldb, uint64_t k, uint64_t nb, Mod mod,
                               uint32_t half, uint32_t kblocks, int pre, uint8_t *img)
{
    // the product kernel that follows may be placed now (it waits for this
    // grid only where it reads the image)
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    const uint32_t tile = blockIdx.x;            // nt * kblocks + kb
    const uint32_t nt = tile / kblocks, kb = tile % kblocks;
    uint8_t *out = img + (uint64_t)tile * B_TILE_BYTES;
    for (int t = threadIdx.x; t < 64 * 8; t += blockDim.x) {
        const int col = t >> 3, j = t & 7;       // output column within the tile, 16-byte chunk
        const uint64_t gcol = (uint64_t)nt * NT + col;
        uint32_t v[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const uint64_t gk = (uint64_t)kb * BK + j * 8 + e;
            v[e] = (gk < k && gcol < nb) ? B[gk * ldb + gcol] : 0u;
            if (pre) v[e] %= mod.p;
        }
        uint4 wh, wl;
        split_pair(v[0], v[1], mod.p, half, wh.x, wl.x);
        split_pair(v[2], v[3], mod.p, half, wh.y, wl.y);
        split_pair(v[4], v[5], mod.p, half, wh.z, wl.z);
        split_pair(v[6], v[7], mod.p, half, wh.w, wl.w);
        const int rh = col, rl = col + 64;
        *reinterpret_cast<uint4 *>(out + rh * 128 + ((j ^ (rh & 7)) << 4)) = wh;
        *reinterpret_cast<uint4 *>(out + rl * 128 + ((j ^ (rl & 7)) << 4)) = wl;
    }
}

// A (m x k, row-major uint32 residues, leading dimension lda) -> prepared
// tiles for one modulus p <= 65536: per (m-tile, k-block) the two 8-bit digit
// planes described at A8_TILE_BYTES.  Entries outside the matrix are 0
// (bytes 0x80, 0x80).  With pre != 0 each entry is first reduced modulo p (a
// residue pass).  Thread q of a tile handles 4 consecutive K of one row.
__global__ void __launch_bounds__(256)
    k_block_prep_a(const uint32_t *__restrict__ A, uint64_t lda, uint64_t m, uint64_t k, Mod mod,
                   uint32_t pre_magic, int pre, uint32_t kblocks, uint8_t *img)
{
    const uint64_t tile = blockIdx.x;   // mt * kblocks + kb
    const uint64_t mt = tile / kblocks, kb = tile % kblocks;
    uint8_t *hi = img + tile * A8_TILE_BYTES;
    uint8_t *lo = hi + A8_PLANE_BYTES;
    const uint32_t p = mod.p;
    const uint32_t thr = min((p - 1) / 2, 32639u);   // largest residue kept as itself
    for (int q = threadIdx.x; q < BM * 16; q += blockDim.x) {
        const int row = q >> 4, c4 = q & 15;
        const uint64_t gr = mt * BM + row, gk = kb * BK + (uint64_t)c4 * 4;
        uint32_t hb = 0, lb = 0;
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            uint32_t v = (gr < m && gk + e < k) ? __ldg(A + gr * lda + gk + e) : 0u;
            if (pre) v = reduce_small(v, p, pre_magic);
            const uint32_t u = v + 32896u - (v > thr ? p : 0u);   // in [0, 65535]
            hb |= (u >> 8) << (8 * e);
            lb |= (u & 255u) << (8 * e);
        }
        *reinterpret_cast<uint32_t *>(hi + row * BK + c4 * 4) = hb;
        *reinterpret_cast<uint32_t *>(lo + row * BK + c4 * 4) = lb;
    }
}

// x mod m for x < 2^40 and m < 2^17, minv = floor((2^64 - 1) / m): the
// multiply-high quotient is floor(x / m) or one less
__device__ __forceinline__ uint32_t mod_small64(uint64_t x, uint32_t m, uint64_t minv)
{
    const uint64_t r = x - __umul64hi(x, minv) * m;
    return (uint32_t)(r >= m ? r - m : r);
}

// Garner recombination of L residue matrices R[l] (m x nb, dense) into
// C = X mod p, where X is the unique integer in [0, prod m_l) with X = R[l]
// mod m_l: mixed-radix digits v_l in [0, m_l), X = v_0 + m_0 (v_1 + m_1 (v_2
// + ...)), evaluated modulo p from the innermost term out.  The moduli are
// the largest primes <= 65536, all above 65000, so a digit v_j < m_j is below
// 2 m_l and reduces modulo m_l by one conditional subtraction.
__global__ void k_block_crt(const uint32_t *R, uint64_t m, uint64_t nb, uint32_t *C, uint64_t ldc, RnsConst rc)
{
    const uint64_t count = m * nb;
    for (uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; e < count;
         e += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t v[RNS_MAX];
#pragma unroll
        for (int l = 0; l < RNS_MAX; ++l) {
            if (l >= rc.L) break;
            const uint32_t ml = rc.mod[l];
            uint32_t t = R[(uint64_t)l * count + e];   // below ml
#pragma unroll
            for (int j = 0; j < RNS_MAX; ++j) {
                if (j >= l) break;
                const uint32_t vj = v[j] >= ml ? v[j] - ml : v[j];
                t = t >= vj ? t - vj : t + ml - vj;     // (t - v_j) mod m_l
                t = mod_small64((uint64_t)t * rc.inv[l][j], ml, rc.minv[l]);
            }
            v[l] = t;
        }
        uint64_t acc = reduce64(v[rc.L - 1], rc.modp);
        for (int l = rc.L - 2; l >= 0; --l) acc = reduce64(acc * rc.mod[l] + v[l], rc.modp);
        C[(e / nb) * ldc + e % nb] = (uint32_t)acc;
    }
}

// ---------------- CUDA-core path ----------------
constexpr int CC_TM = 64, CC_TN = 64, CC_TK = 32, CC_THREADS = 256;

template <class Acc>
__global__ void __launch_bounds__(CC_THREADS)
    k_block_cc(Mod mod, uint64_t kk_bound, uint64_t m, uint64_t k, uint64_t nb,
               const uint32_t *__restrict__ A, uint64_t lda, const uint32_t *__restrict__ B,
               uint64_t ldb, uint32_t *__restrict__ C, uint64_t ldc)
{
    __shared__ __align__(16) uint32_t As[CC_TK][CC_TM];   // transposed: [k][row]
    __shared__ __align__(16) uint32_t Bs[CC_TK][CC_TN];
    const int t = threadIdx.x, tx = t & 15, ty = t >> 4;
    const uint64_t row0 = (uint64_t)blockIdx.y * CC_TM, col0 = (uint64_t)blockIdx.x * CC_TN;
    Acc acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j].init(mod, kk_bound);
    for (uint64_t k0 = 0; k0 < k; k0 += CC_TK) {
        // A tile: 64 rows x 32 K; thread -> row t/4, 8 consecutive K
        {
            const int r = t >> 2, kc = (t & 3) * 8;
            const uint64_t gr = row0 + r;
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                const uint64_t gk = k0 + kc + e;
                As[kc + e][r] = (gr < m && gk < k) ? __ldg(A + gr * lda + gk) : 0u;
            }
        }
        // B tile: 32 K x 64 columns; thread -> K t/8, 8 consecutive columns
        {
            const int r = t >> 3, cc = (t & 7) * 8;
            const uint64_t gk = k0 + r;
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                const uint64_t gc = col0 + cc + e;
                Bs[r][cc + e] = (gk < k && gc < nb) ? __ldg(B + gk * ldb + gc) : 0u;
            }
        }
        __syncthreads();
        const int kmax = (int)min((uint64_t)CC_TK, k - k0);
        for (int kk = 0; kk < kmax; ++kk) {
            const uint4 av = *reinterpret_cast<const uint4 *>(&As[kk][ty * 4]);
            const uint4 bv = *reinterpret_cast<const uint4 *>(&Bs[kk][tx * 4]);
            const uint32_t ar[4] = {av.x, av.y, av.z, av.w};
            const uint32_t br[4] = {bv.x, bv.y, bv.z, bv.w};
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j].add(ar[i], br[j], mod);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const uint64_t gr = row0 + ty * 4 + i;
        if (gr >= m) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const uint64_t gc = col0 + tx * 4 + j;
            if (gc < nb) C[gr * ldc + gc] = acc[i][j].residue(mod);
        }
    }
}

}  // namespace blk

// ---------------- launchers ----------------

bool block_tc_layout_ok(const uint32_t *A, uint64_t lda)
{
    return ((((uintptr_t)A) & 15u) == 0) && (lda % 4 == 0);
}

bool block_tc_eligible(uint32_t p, const uint32_t *A, uint64_t lda)
{
    return p >= 2 && p <= BLOCK_TC_MAX_P && block_tc_layout_ok(A, lda);
}

static uint32_t pow_mod_small(uint64_t b, uint64_t e, uint32_t m)
{
    uint64_t r = 1 % m;
    b %= m;
    while (e) {
        if (e & 1) r = r * b % m;
        b = b * b % m;
        e >>= 1;
    }
    return (uint32_t)r;
}

bool block_rns_plan(uint32_t p, uint64_t k, RnsConst *rc)
{
    // the RNS_MAX largest primes not above 65536, by trial division: every
    // residue modulus then also fits the 8-bit digit planes of a prepared A
    static uint32_t primes[RNS_MAX];
    static bool ready = false;
    static std::mutex mu;
    {
        std::lock_guard<std::mutex> g(mu);
        if (!ready) {
            int found = 0;
            for (uint32_t c = RNS_PRIME_MAX; found < RNS_MAX; --c) {
                bool prime = c > 1;
                for (uint32_t d = 2; prime && d * d <= c; ++d) prime = (c % d) != 0;
                if (prime) primes[found++] = c;
            }
            ready = true;
        }
    }
    if (p < 2) return false;
    // every exact entry sum_t a_t b_t lies in [0, k (p-1)^2]; the moduli's
    // product must exceed that to fix it
    const unsigned __int128 bound = (unsigned __int128)k * (uint64_t)(p - 1) * (uint64_t)(p - 1);
    unsigned __int128 M = 1;
    int L = 0;
    while (L < RNS_MAX && M <= bound) M *= primes[L++];
    if (M <= bound) return false;
    rc->L = L;
    rc->p = p;
    for (int l = 0; l < RNS_MAX; ++l) {
        rc->mod[l] = l < L ? primes[l] : 1;
        for (int j = 0; j < RNS_MAX; ++j)
            rc->inv[l][j] = (l < L && j < l) ? pow_mod_small(primes[j], primes[l] - 2, primes[l]) : 0;
        rc->minv[l] = UINT64_MAX / rc->mod[l];
    }
    rc->modp = make_mod(p);
    return true;
}

size_t block_tc_bimg_bytes(uint64_t k, uint64_t nb)
{
    const uint64_t kblocks = (k + blk::BK - 1) / blk::BK;
    const uint64_t n_tiles = (nb + blk::NT - 1) / blk::NT;
    return (n_tiles * kblocks * (uint64_t)blk::B_TILE_BYTES + 255) & ~(size_t)255;
}

size_t block_tc_workspace_bytes(uint64_t m, uint64_t k, uint64_t nb)
{
    const uint64_t kblocks = (k + blk::BK - 1) / blk::BK;
    const uint64_t n_tiles = (nb + blk::NT - 1) / blk::NT;
    size_t b = n_tiles * kblocks * (uint64_t)blk::B_TILE_BYTES;
    b = (b + 255) & ~(size_t)255;
    b += ((m * n_tiles * blk::NT * 4 + 255) & ~(size_t)255);
    b += 256;   // error flag
    return b;
}

uint32_t *block_tc_err_flag(void *ws, uint64_t m, uint64_t k, uint64_t nb)
{
    return (uint32_t *)((uint8_t *)ws + block_tc_workspace_bytes(m, k, nb) - 256);
}

static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    }
    return fn;
}

size_t block_prep_a_bytes(uint64_t m, uint64_t k)
{
    const uint64_t kblocks = (k + blk::BK - 1) / blk::BK;
    const uint64_t m_tiles = (m + blk::BM - 1) / blk::BM;
    return (size_t)(m_tiles * kblocks) * blk::A8_TILE_BYTES;
}

cudaError_t launch_block_prep_a(const Mod &mod, uint64_t m, uint64_t k, const uint32_t *A,
                                uint64_t lda, bool reduce_inputs, uint8_t *img, cudaStream_t s)
{
    using namespace blk;
    const uint64_t kblocks = (k + BK - 1) / BK, m_tiles = (m + BM - 1) / BM;
    if (m_tiles * kblocks == 0) return cudaSuccess;
    if (m_tiles * kblocks > 0x7FFFFFFFull) return cudaErrorInvalidValue;
    if (mod.p > DIGIT8_MAX_P) return cudaErrorInvalidValue;
    k_block_prep_a<<<(unsigned)(m_tiles * kblocks), 256, 0, s>>>(
        A, lda, m, k, mod, (uint32_t)((1ull << 32) / mod.p), reduce_inputs ? 1 : 0, (uint32_t)kblocks,
        img);
    return cudaGetLastError();
}

cudaError_t launch_block_tc(const Mod &mod, uint64_t m, uint64_t k, uint64_t nb, const uint32_t *A,
                            uint64_t lda, const uint32_t *B, uint64_t ldb, uint32_t *C, uint64_t ldc,
                            void *ws, int sm_count, cudaStream_t s, int *launches, bool reduce_inputs,
                            const uint8_t *Aimg)
{
    using namespace blk;
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_block_tc<false, false, PipeU32>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)PipeU32::SMEM_BYTES);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_block_tc<true, false, PipeU32>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)PipeU32::SMEM_BYTES);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_block_tc<false, true, PipePrep>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)PipePrep::SMEM_BYTES);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    Args a;
    memset(&a, 0, sizeof a);
    if (Aimg) {
        // prepared digits (16-byte aligned tiles of a device allocation): no tensor map
        if (((uintptr_t)Aimg) & 15u) return cudaErrorInvalidValue;
        a.Aimg = Aimg;
    } else {
        PFN_cuTensorMapEncodeTiled_v12000 encode = tensor_map_encoder();
        if (!encode) return cudaErrorNotSupported;
        // A: innermost dimension k (elements), then m rows lda*4 bytes apart
        const cuuint64_t gdim[2] = {(cuuint64_t)k, (cuuint64_t)m};
        const cuuint64_t gstride[1] = {(cuuint64_t)lda * 4};
        const cuuint32_t box[2] = {(cuuint32_t)(BK * PipeU32::KBB), (cuuint32_t)BM};
        const cuuint32_t estride[2] = {1, 1};
        if (encode(&a.tmap_a, CU_TENSOR_MAP_DATA_TYPE_UINT32, 2, (void *)A, gdim, gstride, box, estride,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return cudaErrorInvalidValue;
    }
    a.m = m;
    a.k = k;
    a.nb = nb;
    a.C = C;
    a.ldc = ldc;
    a.mod = mod;
    a.half = (mod.p - 1) / 2;
    a.kblocks = (uint32_t)((k + BK - 1) / BK);
    a.n_tiles = (uint32_t)((nb + NT - 1) / NT);
    a.m_tiles = (uint32_t)((m + BM - 1) / BM);
    a.chunks = (a.kblocks + KC - 1) / KC;
    a.units = (uint64_t)a.n_tiles * a.m_tiles * a.chunks;
    if (a.n_tiles > 65535) return cudaErrorInvalidValue;   // grid y of the finishing kernel
    const uint64_t two41 = 1ull << 41;
    a.off = (two41 / mod.p + 1) * (uint64_t)mod.p;
    a.pre_magic = (uint32_t)((1ull << 32) / mod.p);
    uint8_t *w = (uint8_t *)ws;
    size_t o = (size_t)a.n_tiles * a.kblocks * B_TILE_BYTES;
    o = (o + 255) & ~(size_t)255;
    a.Bimg = w;
    a.Cacc = (uint32_t *)(w + o);
    o += ((m * a.n_tiles * NT * 4 + 255) & ~(size_t)255);
    a.err = (uint32_t *)(w + o);
    k_block_prep_b<<<a.n_tiles * a.kblocks, 256, 0, s>>>(B, ldb, k, nb, mod, a.half, a.kblocks,
                                                         reduce_inputs ? 1 : 0, (uint8_t *)a.Bimg);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const uint64_t grid = std::min<uint64_t>(a.units, (uint64_t)sm_count);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(THREADS);
    cfg.stream = s;
    cudaLaunchAttribute pdl[1];
    pdl[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    pdl[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = pdl;
    cfg.numAttrs = 1;
    if (Aimg) {   // the image already holds the residues of this pass's modulus
        cfg.dynamicSmemBytes = PipePrep::SMEM_BYTES;
        e = cudaLaunchKernelEx(&cfg, k_block_tc<false, true, PipePrep>, a);
    } else if (reduce_inputs) {
        cfg.dynamicSmemBytes = PipeU32::SMEM_BYTES;
        e = cudaLaunchKernelEx(&cfg, k_block_tc<true, false, PipeU32>, a);
    } else {
        cfg.dynamicSmemBytes = PipeU32::SMEM_BYTES;
        e = cudaLaunchKernelEx(&cfg, k_block_tc<false, false, PipeU32>, a);
    }
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t fcfg = {};
    fcfg.gridDim = dim3(a.m_tiles, a.n_tiles);
    fcfg.blockDim = dim3(FIN_THREADS);
    fcfg.stream = s;
    fcfg.attrs = pdl;
    fcfg.numAttrs = 1;
    e = cudaLaunchKernelEx(&fcfg, k_block_finish, a.Cacc, m, nb, C, ldc, mod.p, a.pre_magic);
    if (e != cudaSuccess) return e;
    *launches += 3;
    return cudaGetLastError();
}

cudaError_t launch_block_crt(const uint32_t *R, uint64_t m, uint64_t nb, uint32_t *C, uint64_t ldc,
                             const RnsConst &rc, int sm_count, cudaStream_t s)
{
    const uint64_t count = m * nb;
    const uint64_t blocks = std::max<uint64_t>(1, std::min<uint64_t>((count + 255) / 256, (uint64_t)sm_count * 8));
    blk::k_block_crt<<<(unsigned)blocks, 256, 0, s>>>(R, m, nb, C, ldc, rc);
    return cudaGetLastError();
}

template <class Acc>
static cudaError_t cc_launch(const Mod &mod, uint64_t kb, uint64_t m, uint64_t k, uint64_t nb,
                             const uint32_t *A, uint64_t lda, const uint32_t *B, uint64_t ldb,
                             uint32_t *C, uint64_t ldc, cudaStream_t s)
{
    using namespace blk;
    dim3 grid((unsigned)((nb + CC_TN - 1) / CC_TN), (unsigned)((m + CC_TM - 1) / CC_TM));
    k_block_cc<Acc><<<grid, CC_THREADS, 0, s>>>(mod, kb, m, k, nb, A, lda, B, ldb, C, ldc);
    return cudaGetLastError();
}

cudaError_t wait_selftest(uint64_t limit_ns, cudaStream_t s, uint32_t *status_bits)
{
    uint32_t zero = 0;
    cudaError_t e = cudaMemcpyToSymbolAsync(blk::g_selftest_err, &zero, 4, 0, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return e;
    uint32_t *dptr = nullptr;
    e = cudaGetSymbolAddress((void **)&dptr, blk::g_selftest_err);
    if (e != cudaSuccess) return e;
    blk::k_wait_selftest<<<1, 32, 0, s>>>(limit_ns, dptr);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    e = cudaMemcpyFromSymbolAsync(status_bits, blk::g_selftest_err, 4, 0, cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return e;
    return cudaStreamSynchronize(s);
}

cudaError_t launch_block_cc(Repr r, const Mod &mod, uint64_t kbound, uint64_t m, uint64_t k,
                            uint64_t nb, const uint32_t *A, uint64_t lda, const uint32_t *B,
                            uint64_t ldb, uint32_t *C, uint64_t ldc, cudaStream_t s)
{
    switch (r) {
    case U64_BLOCK: return cc_launch<AccBlock>(mod, kbound, m, k, nb, A, lda, B, ldb, C, ldc, s);
    case U64_CARRY: return cc_launch<AccCarry>(mod, kbound, m, k, nb, A, lda, B, ldb, C, ldc, s);
    case FP64: return cc_launch<AccF64>(mod, kbound, m, k, nb, A, lda, B, ldb, C, ldc, s);
    case CENTERED: return cc_launch<AccCentered>(mod, kbound, m, k, nb, A, lda, B, ldb, C, ldc, s);
    case MONTGOMERY: return cc_launch<AccMontgomery>(mod, kbound, m, k, nb, A, lda, B, ldb, C, ldc, s);
    default: return cc_launch<AccPerTerm>(mod, kbound, m, k, nb, A, lda, B, ldb, C, ldc, s);
    }
}

}  // namespace gfp
