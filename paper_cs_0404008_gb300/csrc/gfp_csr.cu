// Sparse-row block product over GF(p): C = A B mod p with A in CSR form
// (row_ptr, col, val) and B dense k x nb.  One warp per row and 64-column
// group: the warp reads 32 nonzeros at a time (coalesced), broadcasts each
// (column, value) pair with shuffles, and lane j accumulates output columns
// 2j and 2j+1 from one 8-byte load of the selected B row (a 256-byte coalesced
// segment per nonzero, L2-resident for moderate k*nb), four nonzeros per step
// so that four B-row loads are in flight, with the unreduced accumulators of
// the dot-product kernels and one reduction per output.
#include "gfp_internal.h"

namespace gfp {

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

template <class Acc>
static cudaError_t csr_launch(const Mod &mod, uint64_t kbound, uint64_t m, uint64_t k, uint64_t nb,
                              const uint32_t *row_ptr, const uint32_t *col, const uint32_t *val,
                              const uint32_t *B, uint64_t ldb, uint32_t *C, uint64_t ldc,
                              int sm_count, cudaStream_t s)
{
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
