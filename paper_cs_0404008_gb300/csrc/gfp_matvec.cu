// Dense matrix-vector product over GF(p): y_i = (sum_j A_ij x_j) mod p.
//
// Each CTA owns a contiguous range of rows (ranges differ by at most one row
// over the grid, one CTA per SM).  x is staged once per CTA in shared memory.
// Inside a CTA the warps form G groups of W warps: a group works on one row at
// a time and warp s of the group streams column segment s of that row with
// 128-bit loads, accumulating unreduced (Section 3 of the paper) and leaving
// one residue per (row, segment) in shared memory.  After a batch of RB rows
// the CTA sums the W segment residues of each row and writes y.  No atomics,
// no per-row barrier; A is read exactly once.
#include "gfp_internal.h"

namespace gfp {

constexpr int MV_RB = 64;   // rows per batch (multiple of every group count G)
constexpr int MV_PREFETCH_ROWS = 4;   // rows of A requested into L2 before the dependency wait

// Sum of one uint64 per thread over the CTA, valid in thread 0.
__device__ __forceinline__ uint64_t cta_sum_mv(uint64_t v)
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

// Projection of the product onto a vector u, fused into the epilogue (the
// scalar sequence u^T A^t x of a Wiedemann-style iteration): every CTA adds
// the residue of sum_i u_i y_i over its rows to a slot; the last CTA reduces
// it into *sout.  Inactive when u is null.
struct MvProj {
    const uint32_t *u;
    unsigned long long *slot;
    uint32_t *ticket;
    uint32_t *sout;
};

template <class Acc, bool XS, int U>
__global__ void __launch_bounds__(MV_THREADS, 1)
    k_matvec(Mod m, uint64_t k, uint64_t rows, uint64_t cols, const uint32_t *__restrict__ A,
             uint64_t lda, const uint32_t *__restrict__ x, uint32_t *__restrict__ y, int W,
             MvProj proj)
{
    extern __shared__ __align__(16) uint32_t smem[];
    const uint64_t colsp = (cols + 3) & ~3ull;
    // Programmatic dependent launch: the next kernel of the stream may be
    // scheduled on SMs this grid has left (its tail).  A never changes, so
    // before waiting for the previous kernel (which may have produced x) the
    // CTA asks L2 for the first rows it will stream; everything that reads
    // x or writes y comes after the wait.
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    {
        const uint64_t r0 = rows * blockIdx.x / gridDim.x, r1 = rows * (blockIdx.x + 1) / gridDim.x;
        const uint64_t row_bytes = cols * 4;
        if (threadIdx.x < MV_PREFETCH_ROWS && r0 + threadIdx.x < r1 &&
            ((((uintptr_t)A) | (lda * 4) | row_bytes) & 15u) == 0 && row_bytes <= 0xFFFFFFF0ull)
            asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(A + (r0 + threadIdx.x) * lda),
                         "r"((uint32_t)row_bytes)
                         : "memory");
    }
    asm volatile("griddepcontrol.wait;" ::: "memory");
    uint32_t *xs = smem;
    uint32_t *part = smem + (XS ? colsp : 0);
    const int nw = blockDim.x >> 5, w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int G = nw / W, g = w / W, sgm = w % W;

    if (XS) {
        for (uint64_t j = threadIdx.x; j < colsp; j += blockDim.x) xs[j] = (j < cols) ? x[j] : 0u;
        __syncthreads();
    }
    const uint32_t *xsrc = XS ? xs : x;
    const bool vec = ((((uintptr_t)A) & 15u) == 0) && (lda % 4 == 0) &&
                     (XS || ((((uintptr_t)x) & 15u) == 0));

    // column segment of this warp: [c0, c1), c0 a multiple of 4
    const uint64_t seg = ((cols + W - 1) / W + 3) & ~3ull;
    const uint64_t c0 = (uint64_t)sgm * seg;
    const uint64_t c1 = (c0 + seg < cols) ? c0 + seg : cols;

    const uint64_t r_begin = rows * blockIdx.x / gridDim.x;
    const uint64_t r_end = rows * (blockIdx.x + 1) / gridDim.x;
    uint64_t pacc = 0;   // projection partial (sum of residues)

    for (uint64_t rb = r_begin; rb < r_end; rb += MV_RB) {
        const uint64_t rcount = (r_end - rb < (uint64_t)MV_RB) ? r_end - rb : (uint64_t)MV_RB;
        for (uint64_t i = g; i < rcount; i += G) {
            const uint32_t *Ar = A + (rb + i) * lda;
            Acc acc;
            acc.init(m, k);
            if (c0 < c1) {
                if (vec) {
                    const uint4 *av = reinterpret_cast<const uint4 *>(Ar + c0);
                    const uint4 *xv = reinterpret_cast<const uint4 *>(xsrc + c0);
                    const uint64_t nv = (c1 - c0) >> 2;
                    uint64_t v = lane;
                    for (; v + (U - 1) * 32 < nv; v += U * 32) {
                        uint4 a[U];
#pragma unroll
                        for (int u = 0; u < U; ++u) a[u] = __ldcs(av + v + u * 32);
#pragma unroll
                        for (int u = 0; u < U; ++u)
                            acc.add4(a[u], XS ? xv[v + u * 32] : __ldg(xv + v + u * 32), m);
                    }
                    for (; v < nv; v += 32)
                        acc.add4(__ldcs(av + v), XS ? xv[v] : __ldg(xv + v), m);
                    const uint64_t j = c0 + (nv << 2) + lane;
                    if (j < c1) acc.add(__ldcs(Ar + j), XS ? xsrc[j] : __ldg(xsrc + j), m);
                } else {
                    for (uint64_t j = c0 + lane; j < c1; j += 32)
                        acc.add(__ldcs(Ar + j), XS ? xsrc[j] : __ldg(xsrc + j), m);
                }
            }
            uint64_t s = acc.residue(m);
#pragma unroll
            for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            if (lane == 0) part[i * W + sgm] = reduce64(s, m);
        }
        __syncthreads();
        for (uint64_t i = threadIdx.x; i < rcount; i += blockDim.x) {
            uint64_t s = 0;
            for (int q = 0; q < W; ++q) s += part[i * W + q];
            const uint32_t yi = reduce64(s, m);
            y[rb + i] = yi;
            if (proj.u) pacc += reduce64((uint64_t)yi * __ldg(proj.u + rb + i), m);
        }
        __syncthreads();
    }
    if (proj.u) {
        const uint64_t s = cta_sum_mv(pacc);
        if (threadIdx.x == 0) {
            atomicAdd(proj.slot, (unsigned long long)reduce64(s, m));
            __threadfence();
            if (atomicAdd(proj.ticket, 1u) == gridDim.x - 1) {
                __threadfence();
                const unsigned long long v = atomicExch(proj.slot, 0ull);
                atomicExch(proj.ticket, 0u);
                *proj.sout = reduce64((uint64_t)v, m);
            }
        }
    }
}

// Shared memory above which x is read through the L1/L2 path instead.
constexpr size_t MV_XS_MAX = 200 * 1024;

template <class Acc, bool XS>
static cudaError_t mv_launch(const Mod &m, uint64_t k, uint64_t rows, uint64_t cols,
                             const uint32_t *A, uint64_t lda, const uint32_t *x, uint32_t *y,
                             int sm_count, cudaStream_t s, const MvProj &proj)
{
    constexpr int U = 4;
    const int nw = MV_THREADS / 32;
    // warps per row: enough that each warp streams >= U*32 vectors, at most nw
    uint64_t nv = cols / 4;
    int W = 1;
    while (W < nw && nv / (uint64_t)(2 * W) >= (uint64_t)U * 32) W *= 2;
    const size_t colsp = (cols + 3) & ~3ull;
    const size_t smem = (XS ? colsp * 4 : 0) + (size_t)MV_RB * W * 4;
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(k_matvec<Acc, XS, U>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)(MV_XS_MAX + MV_RB * nw * 4));
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    uint64_t grid = (uint64_t)sm_count;
    if (grid > rows) grid = rows ? rows : 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(MV_THREADS);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const cudaError_t e = cudaLaunchKernelEx(&cfg, k_matvec<Acc, XS, U>, m, k, rows, cols, A, lda, x,
                                             y, W, proj);
    return e != cudaSuccess ? e : cudaGetLastError();
}

template <class Acc>
static cudaError_t mv_dispatch(const Mod &m, uint64_t k, uint64_t rows, uint64_t cols,
                               const uint32_t *A, uint64_t lda, const uint32_t *x, uint32_t *y,
                               int sm_count, cudaStream_t s, const MvProj &proj)
{
    if (((cols + 3) & ~3ull) * 4 <= MV_XS_MAX)
        return mv_launch<Acc, true>(m, k, rows, cols, A, lda, x, y, sm_count, s, proj);
    return mv_launch<Acc, false>(m, k, rows, cols, A, lda, x, y, sm_count, s, proj);
}

cudaError_t launch_matvec(Repr r, const Mod &m, uint64_t k, uint64_t rows, uint64_t cols,
                          const uint32_t *A, uint64_t lda, const uint32_t *x, uint32_t *y,
                          int sm_count, cudaStream_t s, const uint32_t *u,
                          unsigned long long *slot, uint32_t *ticket, uint32_t *sout)
{
    const MvProj proj{u, slot, ticket, sout};
    switch (r) {
    case U64_BLOCK: return mv_dispatch<AccBlock>(m, k, rows, cols, A, lda, x, y, sm_count, s, proj);
    case U64_CARRY: return mv_dispatch<AccCarry>(m, k, rows, cols, A, lda, x, y, sm_count, s, proj);
    case FP64: return mv_dispatch<AccF64>(m, k, rows, cols, A, lda, x, y, sm_count, s, proj);
    case CENTERED: return mv_dispatch<AccCentered>(m, k, rows, cols, A, lda, x, y, sm_count, s, proj);
    case MONTGOMERY: return mv_dispatch<AccMontgomery>(m, k, rows, cols, A, lda, x, y, sm_count, s, proj);
    default: return mv_dispatch<AccPerTerm>(m, k, rows, cols, A, lda, x, y, sm_count, s, proj);
    }
}

}  // namespace gfp
