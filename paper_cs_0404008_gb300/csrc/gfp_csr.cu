// Sparse-row block product over GF(p): C = A B mod p with A in CSR form
// (row_ptr, col, val) and B dense k x nb.  Two kernels: the wide form below
// (16-byte gathers, for B rows 16-byte aligned) and this general one for any
// layout.  One warp per row and 64-column
// group: the warp reads 32 nonzeros at a time (coalesced), broadcasts each
// (column, value) pair with shuffles, and lane j accumulates output columns
// 2j and 2j+1 from one 8-byte load of the selected B row (a 256-byte coalesced
// segment per nonzero, L2-resident for moderate k*nb), four nonzeros per step
// so that four B-row loads are in flight, with the unreduced accumulators of
// the dot-product kernels and one reduction per output.
#include "gfp_internal.h"

#include <algorithm>
#include <type_traits>

namespace gfp {

#ifdef GFP_DEVICE_CHECKS
__device__ uint32_t g_csr_check;
uint32_t csr_check_bits()
{
    uint32_t h = 0, z = 0;
    if (cudaMemcpyFromSymbol(&h, g_csr_check, 4) != cudaSuccess) return 0;
    cudaMemcpyToSymbol(g_csr_check, &z, 4);
    return h;
}
#else
uint32_t csr_check_bits() { return 0; }
#endif

template <class Acc>
__global__ void __launch_bounds__(256)
    k_block_csr(Mod mod, uint64_t kbound, uint64_t m, uint64_t k, uint64_t nb,
                const uint32_t *__restrict__ row_ptr, const uint32_t *__restrict__ col,
                const uint32_t *__restrict__ val, const uint32_t *__restrict__ B, uint64_t ldb,
                uint32_t *__restrict__ C, uint64_t ldc)
{
    const int lane = threadIdx.x & 31;
    const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x >> 5);
    // 8-byte loads of column pairs need 8-byte aligned rows
    const bool pair_ok = ((((uintptr_t)B) & 7u) == 0) && (ldb % 2 == 0);
    for (uint64_t row = (uint64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); row < m;
         row += warps) {
        const uint32_t q0 = __ldg(row_ptr + row), q1 = __ldg(row_ptr + row + 1);
        GFP_DCHECK(g_csr_check, q0 <= q1, DCHECK_CSR_ROW_PTR);
        for (uint64_t c0 = 0; c0 < nb; c0 += 64) {
            const uint64_t ca = c0 + 2 * lane;             // this lane's columns ca, ca+1
            const bool va = ca < nb, vb = ca + 1 < nb;
            Acc a0, a1;
            a0.init(mod, kbound);
            a1.init(mod, kbound);
            for (uint32_t q = q0; q < q1; q += 32) {
                const uint32_t cnt = min(32u, q1 - q);
                uint32_t mycol = 0, myval = 0;
                if ((uint32_t)lane < cnt) {
                    mycol = __ldg(col + q + lane);
                    myval = __ldg(val + q + lane);
                    GFP_DCHECK(g_csr_check, mycol < k, DCHECK_CSR_COLUMN);
                    if (mycol >= k) {   // outside the matrix: contributes nothing, reads row 0
                        mycol = 0;
                        myval = 0;
                    }
                }
                uint32_t t = 0;
                for (; t + 4 <= cnt; t += 4) {
                    uint32_t cc[4], vv[4], bx[4], by[4];
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        cc[e] = __shfl_sync(0xffffffffu, mycol, t + e);
                        vv[e] = __shfl_sync(0xffffffffu, myval, t + e);
                    }
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const uint32_t *br = B + (uint64_t)cc[e] * ldb + ca;
                        if (pair_ok && vb) {
                            const uint2 w = __ldg(reinterpret_cast<const uint2 *>(br));
                            bx[e] = w.x;
                            by[e] = w.y;
                        } else {
                            bx[e] = va ? __ldg(br) : 0u;
                            by[e] = vb ? __ldg(br + 1) : 0u;
                        }
                    }
                    a0.add4(make_uint4(vv[0], vv[1], vv[2], vv[3]), make_uint4(bx[0], bx[1], bx[2], bx[3]),
                            mod);
                    a1.add4(make_uint4(vv[0], vv[1], vv[2], vv[3]), make_uint4(by[0], by[1], by[2], by[3]),
                            mod);
                }
                for (; t < cnt; ++t) {
                    const uint32_t c = __shfl_sync(0xffffffffu, mycol, t);
                    const uint32_t v = __shfl_sync(0xffffffffu, myval, t);
                    const uint32_t *br = B + (uint64_t)c * ldb + ca;
                    if (va) a0.add(v, __ldg(br), mod);
                    if (vb) a1.add(v, __ldg(br + 1), mod);
                }
            }
            if (va) C[row * ldc + ca] = a0.residue(mod);
            if (vb) C[row * ldc + ca + 1] = a1.residue(mod);
        }
    }
}

// Wide form, for B 16-byte aligned with ldb and nb multiples of 4: the two
// half-warps take alternate groups of four nonzeros of the row, and lane l of
// a half owns output columns 4l..4l+3 of the 64-column group, which it gathers
// with one 16-byte load per nonzero.  The (column, value) pairs of 32 nonzeros
// are staged in shared memory so that a lane fetches its four pairs with two
// 16-byte loads; the two halves' residues are added modulo p at the end.
//
// PLAIN (blocked representation, lambda >= 16): plain 64-bit sums with no
// per-term bookkeeping.  A half adds at most 16 products per chunk of 32
// nonzeros, so reducing the sums after every floor(lambda / 16) chunks keeps
// each at most a value below p plus lambda products (the carried bound).
// Otherwise one accumulator of the representation per output column.

// Visits nonzeros q0 <= q < q1 in steps of eight (four per half), calling
// fn(values, B quads of the four nonzeros) for each step and done() after each
// chunk of 32.  Padding and columns outside [0, k) enter as value 0 at column
// 0 (k >= 1).
template <class F, class G>
__device__ __forceinline__ void csr_row_quads(uint32_t q0, uint32_t q1, uint64_t k,
                                              const uint32_t *__restrict__ col,
                                              const uint32_t *__restrict__ val, uint2 *st,
                                              int lane, int half, const char *bcol,
                                              uint32_t ldb_bytes, F &&fn, G &&done)
{
    const uint4 *st4 = reinterpret_cast<const uint4 *>(st);
    // the pairs of the next chunk are loaded while the current one is gathered
    uint32_t cn = 0, vn = 0;
    if (q0 < q1 && (uint32_t)lane < q1 - q0) {
        cn = __ldg(col + q0 + lane);
        vn = __ldg(val + q0 + lane);
    }
    for (uint32_t q = q0; q < q1; q += 32) {
        const uint32_t cnt = min(32u, q1 - q);
        uint32_t c = cn, v = vn;
        cn = 0;
        vn = 0;
        if (q1 - q > 32 && (uint32_t)lane < q1 - q - 32) {
            cn = __ldg(col + q + 32 + lane);
            vn = __ldg(val + q + 32 + lane);
        }
        GFP_DCHECK(g_csr_check, c < k, DCHECK_CSR_COLUMN);
        if (c >= k) {   // lanes past the end hold (0, 0)
            c = 0;
            v = 0;
        }
        st[lane] = make_uint2(c, v);
        __syncwarp();
        const uint32_t steps = (cnt + 7) >> 3;
        for (uint32_t t = 0; t < steps; ++t) {
            const uint4 e01 = st4[4 * t + 2 * half];       // pairs 8t+4h, 8t+4h+1
            const uint4 e23 = st4[4 * t + 2 * half + 1];   // pairs 8t+4h+2, 8t+4h+3
            const uint4 b0 = __ldg(reinterpret_cast<const uint4 *>(bcol + (uint64_t)e01.x * ldb_bytes));
            const uint4 b1 = __ldg(reinterpret_cast<const uint4 *>(bcol + (uint64_t)e01.z * ldb_bytes));
            const uint4 b2 = __ldg(reinterpret_cast<const uint4 *>(bcol + (uint64_t)e23.x * ldb_bytes));
            const uint4 b3 = __ldg(reinterpret_cast<const uint4 *>(bcol + (uint64_t)e23.z * ldb_bytes));
            fn(make_uint4(e01.y, e01.w, e23.y, e23.w), b0, b1, b2, b3);
        }
        __syncwarp();
        done();
    }
}

template <class Acc, bool PLAIN>
__global__ void __launch_bounds__(256, PLAIN ? 4 : 3)
    k_block_csr_wide(Mod mod, uint64_t kbound, uint32_t segc, uint64_t m, uint64_t k, uint64_t nb,
                     const uint32_t *__restrict__ row_ptr, const uint32_t *__restrict__ col,
                     const uint32_t *__restrict__ val, const uint32_t *__restrict__ B,
                     uint32_t ldb_bytes, uint32_t *__restrict__ C, uint64_t ldc)
{
    __shared__ __align__(16) uint2 stage[8][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int half = lane >> 4, hl = lane & 15;
    uint2 *st = stage[w];
    const uint64_t warps = (uint64_t)gridDim.x * 8;
    const bool cvec = ((((uintptr_t)C) & 15u) == 0) && (ldc % 4 == 0);
    for (uint64_t row = (uint64_t)blockIdx.x * 8 + w; row < m; row += warps) {
        const uint32_t q0 = __ldg(row_ptr + row), q1 = __ldg(row_ptr + row + 1);
        GFP_DCHECK(g_csr_check, q0 <= q1, DCHECK_CSR_ROW_PTR);
        for (uint64_t c0 = 0; c0 < nb; c0 += 64) {
            const uint64_t ca = c0 + 4 * (uint64_t)hl;
            const bool va = ca < nb;   // nb % 4 == 0: the whole quad is valid
            const char *bcol = reinterpret_cast<const char *>(B + (va ? ca : 0));
            uint32_t r[4];
            if constexpr (PLAIN) {
                uint64_t s0 = 0, s1 = 0, s2 = 0, s3 = 0;
                uint32_t chunks = 0;
                csr_row_quads(
                    q0, q1, k, col, val, st, lane, half, bcol, ldb_bytes,
                    [&](uint4 v, uint4 b0, uint4 b1, uint4 b2, uint4 b3) {
                        s0 += (uint64_t)v.x * b0.x + (uint64_t)v.y * b1.x + (uint64_t)v.z * b2.x +
                              (uint64_t)v.w * b3.x;
                        s1 += (uint64_t)v.x * b0.y + (uint64_t)v.y * b1.y + (uint64_t)v.z * b2.y +
                              (uint64_t)v.w * b3.y;
                        s2 += (uint64_t)v.x * b0.z + (uint64_t)v.y * b1.z + (uint64_t)v.z * b2.z +
                              (uint64_t)v.w * b3.z;
                        s3 += (uint64_t)v.x * b0.w + (uint64_t)v.y * b1.w + (uint64_t)v.z * b2.w +
                              (uint64_t)v.w * b3.w;
                    },
                    [&]() {
                        if (++chunks == segc) {
                            chunks = 0;
                            s0 = reduce64(s0, mod);
                            s1 = reduce64(s1, mod);
                            s2 = reduce64(s2, mod);
                            s3 = reduce64(s3, mod);
                        }
                    });
                r[0] = reduce64(s0, mod);
                r[1] = reduce64(s1, mod);
                r[2] = reduce64(s2, mod);
                r[3] = reduce64(s3, mod);
            } else {
                Acc a[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) a[j].init(mod, kbound);
                csr_row_quads(
                    q0, q1, k, col, val, st, lane, half, bcol, ldb_bytes,
                    [&](uint4 v, uint4 b0, uint4 b1, uint4 b2, uint4 b3) {
                        a[0].add4(v, make_uint4(b0.x, b1.x, b2.x, b3.x), mod);
                        a[1].add4(v, make_uint4(b0.y, b1.y, b2.y, b3.y), mod);
                        a[2].add4(v, make_uint4(b0.z, b1.z, b2.z, b3.z), mod);
                        a[3].add4(v, make_uint4(b0.w, b1.w, b2.w, b3.w), mod);
                    },
                    [] {});
#pragma unroll
                for (int j = 0; j < 4; ++j) r[j] = a[j].residue(mod);
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const uint64_t t = (uint64_t)r[j] + __shfl_xor_sync(0xffffffffu, r[j], 16);
                r[j] = (uint32_t)(t >= mod.p ? t - mod.p : t);
            }
            if (half == 0 && va) {
                uint32_t *out = C + row * ldc + ca;
                if (cvec) {
                    *reinterpret_cast<uint4 *>(out) = make_uint4(r[0], r[1], r[2], r[3]);
                } else {
                    out[0] = r[0];
                    out[1] = r[1];
                    out[2] = r[2];
                    out[3] = r[3];
                }
            }
        }
    }
}

template <class Acc, bool PLAIN>
static int csr_wide_blocks_per_sm()
{
    static int cached = 0;
    if (!cached) {
        int b = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_block_csr_wide<Acc, PLAIN>, 256, 0) !=
                cudaSuccess ||
            b < 1)
            b = 1;
        cached = b;
    }
    return cached;
}

template <class Acc, bool PLAIN>
static cudaError_t csr_wide_launch(const Mod &mod, uint64_t kbound, uint32_t segc, uint64_t m,
                                   uint64_t k, uint64_t nb, const uint32_t *row_ptr,
                                   const uint32_t *col, const uint32_t *val, const uint32_t *B,
                                   uint64_t ldb, uint32_t *C, uint64_t ldc, int sm_count,
                                   cudaStream_t s)
{
    uint64_t blocks = (m + 7) / 8;
    const uint64_t cap = (uint64_t)sm_count * csr_wide_blocks_per_sm<Acc, PLAIN>();
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    k_block_csr_wide<Acc, PLAIN><<<(unsigned)blocks, 256, 0, s>>>(
        mod, kbound, segc, m, k, nb, row_ptr, col, val, B, (uint32_t)(ldb * 4), C, ldc);
    return cudaGetLastError();
}

template <class Acc>
static cudaError_t csr_launch(const Mod &mod, uint64_t kbound, uint64_t m, uint64_t k, uint64_t nb,
                              const uint32_t *row_ptr, const uint32_t *col, const uint32_t *val,
                              const uint32_t *B, uint64_t ldb, uint32_t *C, uint64_t ldc,
                              int sm_count, cudaStream_t s)
{
    const bool wide = nb % 4 == 0 && ldb % 4 == 0 && ((uintptr_t)B & 15u) == 0 && ldb < (1ull << 30);
    if (wide) {
        if constexpr (std::is_same<Acc, AccBlock>::value) {
            if (kbound >= 16) {
                // chunks of 32 nonzeros between reductions (at most 16 products each)
                const uint64_t segc = std::min<uint64_t>(kbound / 16, 0xFFFFFFFFull);
                return csr_wide_launch<Acc, true>(mod, kbound, (uint32_t)segc, m, k, nb, row_ptr,
                                                  col, val, B, ldb, C, ldc, sm_count, s);
            }
        }
        return csr_wide_launch<Acc, false>(mod, kbound, 0, m, k, nb, row_ptr, col, val, B, ldb, C,
                                           ldc, sm_count, s);
    }
    uint64_t blocks = (m + 7) / 8;
    const uint64_t cap = (uint64_t)sm_count * 8;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    k_block_csr<Acc><<<(unsigned)blocks, 256, 0, s>>>(mod, kbound, m, k, nb, row_ptr, col, val, B,
                                                      ldb, C, ldc);
    return cudaGetLastError();
}

cudaError_t launch_block_csr(Repr r, const Mod &mod, uint64_t kbound, uint64_t m, uint64_t k,
                             uint64_t nb, const uint32_t *row_ptr, const uint32_t *col,
                             const uint32_t *val, const uint32_t *B, uint64_t ldb, uint32_t *C,
                             uint64_t ldc, int sm_count, cudaStream_t s)
{
    switch (r) {
    case U64_BLOCK:
        return csr_launch<AccBlock>(mod, kbound, m, k, nb, row_ptr, col, val, B, ldb, C, ldc, sm_count, s);
    case U64_CARRY:
        return csr_launch<AccCarry>(mod, kbound, m, k, nb, row_ptr, col, val, B, ldb, C, ldc, sm_count, s);
    case FP64:
        return csr_launch<AccF64>(mod, kbound, m, k, nb, row_ptr, col, val, B, ldb, C, ldc, sm_count, s);
    case CENTERED:
        return csr_launch<AccCentered>(mod, kbound, m, k, nb, row_ptr, col, val, B, ldb, C, ldc, sm_count, s);
    case MONTGOMERY:
        return csr_launch<AccMontgomery>(mod, kbound, m, k, nb, row_ptr, col, val, B, ldb, C, ldc, sm_count, s);
    default:
        return csr_launch<AccPerTerm>(mod, kbound, m, k, nb, row_ptr, col, val, B, ldb, C, ldc, sm_count, s);
    }
}

}  // namespace gfp
