// libgfppeaks: ceilings for the rooflines of libgfpdot, measured by this
// project's own kernels (interface and probe definitions in gfppeaks.h).
//
// Every probe keeps its loads or arithmetic alive by folding the results
// into one word that is stored only if it equals an unlikely constant, so
// the compiler cannot drop the work and the probe writes nothing else.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <vector>

#include "gfppeaks.h"

namespace {

constexpr int RD_THREADS = 512;
constexpr uint32_t KEEP = 0x9E3779B9u;

__device__ __forceinline__ uint32_t fold(uint4 a) { return a.x ^ a.y ^ a.z ^ a.w; }

// read-only stream, eight 16-byte streaming loads in flight per thread
__global__ void __launch_bounds__(RD_THREADS) k_read(const uint4 *__restrict__ v, uint64_t nv,
                                                     uint32_t *sink)
{
    const uint64_t T = (uint64_t)gridDim.x * blockDim.x;
    uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t acc = 0;
    for (; i + 7 * T < nv; i += 8 * T) {
        uint4 a[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) a[u] = __ldcs(v + i + u * T);
#pragma unroll
        for (int u = 0; u < 8; ++u) acc ^= fold(a[u]);
    }
    for (; i < nv; i += T) acc ^= fold(__ldcs(v + i));
    if (acc == KEEP) sink[0] = acc;
}

// copy, four 16-byte loads in flight per thread
__global__ void __launch_bounds__(RD_THREADS) k_copy(const uint4 *__restrict__ s, uint4 *__restrict__ d,
                                                     uint64_t nv)
{
    const uint64_t T = (uint64_t)gridDim.x * blockDim.x;
    uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (; i + 3 * T < nv; i += 4 * T) {
        uint4 a[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) a[u] = __ldcs(s + i + u * T);
#pragma unroll
        for (int u = 0; u < 4; ++u) __stcs(d + i + u * T, a[u]);
    }
    for (; i < nv; i += T) __stcs(d + i, __ldcs(s + i));
}

// L2-resident reads: `passes` sweeps over the same words, L1 bypassed
__global__ void __launch_bounds__(RD_THREADS) k_read_l2(const uint4 *__restrict__ v, uint64_t nv,
                                                        int passes, uint32_t *sink)
{
    const uint64_t T = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t t0 = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t acc = 0;
    for (int pass = 0; pass < passes; ++pass) {
        uint64_t i = t0;
        for (; i + 7 * T < nv; i += 8 * T) {
            uint4 a[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) a[u] = __ldcg(v + i + u * T);
#pragma unroll
            for (int u = 0; u < 8; ++u) acc ^= fold(a[u]);
        }
        for (; i < nv; i += T) acc ^= fold(__ldcg(v + i));
        acc = (acc << 1) | (acc >> 31);
    }
    if (acc == KEEP) sink[0] = acc;
}

// eight independent fma chains per thread
__global__ void __launch_bounds__(256) k_dfma(int iters, double s, uint32_t *sink)
{
    double a[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) a[c] = 1e-3 * (threadIdx.x + c);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < 8; ++c) a[c] = fma(a[c], s, 1e-7);
    }
    double t = 0;
#pragma unroll
    for (int c = 0; c < 8; ++c) t += a[c];
    if (t == 123456.75) sink[0] = KEEP;
}

// four independent m16n8k32 s8 accumulator chains per warp
__global__ void __launch_bounds__(256) k_imma(int iters, uint32_t seed, uint32_t *sink)
{
    const uint32_t l = threadIdx.x & 31;
    uint32_t a0 = seed ^ l, a1 = a0 * 3u, a2 = a0 * 5u, a3 = a0 * 7u;
    uint32_t b0 = seed + l, b1 = b0 * 11u;
    int32_t c[4][4] = {};
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int ch = 0; ch < 4; ++ch)
            asm volatile(
                "mma.sync.aligned.m16n8k32.row.col.s32.s8.s8.s32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
                "{%8,%9}, {%0,%1,%2,%3};"
                : "+r"(c[ch][0]), "+r"(c[ch][1]), "+r"(c[ch][2]), "+r"(c[ch][3])
                : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
    }
    int32_t t = 0;
#pragma unroll
    for (int ch = 0; ch < 4; ++ch) t ^= c[ch][0] ^ c[ch][1] ^ c[ch][2] ^ c[ch][3];
    if ((uint32_t)t == KEEP) sink[0] = (uint32_t)t;
}

__global__ void k_empty() {}

template <class K>
int persistent_grid(K kern, int threads, int sms)
{
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, threads, 0) != cudaSuccess ||
        occ < 1)
        occ = 1;
    return sms * occ;
}

struct Probe {
    cudaStream_t s = nullptr;
    std::vector<void *> bufs;
    cudaError_t err = cudaSuccess;
    ~Probe()
    {
        if (s) cudaStreamSynchronize(s);
        for (void *b : bufs) cudaFree(b);
        if (s) cudaStreamDestroy(s);
    }
    void *alloc(size_t n)
    {
        void *p = nullptr;
        cudaError_t e = cudaMalloc(&p, n);
        if (e != cudaSuccess) {
            err = e;
            return nullptr;
        }
        bufs.push_back(p);
        return p;
    }
};

// times `reps` launches of `launch` (after two warm-ups); fills ms_best/median
template <class L>
cudaError_t time_launches(cudaStream_t s, int reps, L launch, gfp_peak_result *r)
{
    std::vector<cudaEvent_t> ev(reps + 1);
    for (auto &e : ev)
        if (cudaEventCreate(&e) != cudaSuccess) return cudaErrorUnknown;
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < 2 && e == cudaSuccess; ++i) e = launch();
    for (int i = 0; i < reps && e == cudaSuccess; ++i) {
        cudaEventRecord(ev[i], s);
        e = launch();
        cudaEventRecord(ev[i + 1], s);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    std::vector<double> ms;
    for (int i = 0; i < reps && e == cudaSuccess; ++i) {
        float t = 0;
        e = cudaEventElapsedTime(&t, ev[i], ev[i + 1]);
        ms.push_back(t);
    }
    for (auto &x : ev) cudaEventDestroy(x);
    if (e != cudaSuccess) return e;
    std::sort(ms.begin(), ms.end());
    r->ms_best = ms.front();
    r->ms_median = ms[ms.size() / 2];
    return cudaSuccess;
}

}  // namespace

extern "C" __attribute__((visibility("default"))) const char *gfp_peak_name(int kind)
{
    static const char *names[GFP_PEAK_KINDS_] = {"read_hbm", "copy_hbm", "read_l2",
                                                 "dfma", "imma_sync_s8", "launch"};
    return (kind >= 0 && kind < GFP_PEAK_KINDS_) ? names[kind] : nullptr;
}

extern "C" __attribute__((visibility("default"))) int gfp_peak_measure(int kind, uint64_t bytes,
                                                                       int reps,
                                                                       gfp_peak_result *out)
{
    if (!out || reps < 1 || kind < 0 || kind >= GFP_PEAK_KINDS_) return GFP_PEAK_ERR_ARG;
    const bool needs_bytes = kind <= GFP_PEAK_READ_L2;
    if (needs_bytes && bytes < (1u << 20)) return GFP_PEAK_ERR_ARG;
    *out = gfp_peak_result{};
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return GFP_PEAK_ERR_CUDA;
    Probe pr;
    if (cudaStreamCreateWithFlags(&pr.s, cudaStreamNonBlocking) != cudaSuccess) {
        pr.s = nullptr;
        return GFP_PEAK_ERR_CUDA;
    }
    uint32_t *sink = (uint32_t *)pr.alloc(256);
    if (!sink) return GFP_PEAK_ERR_CUDA;
    cudaStream_t s = pr.s;
    cudaError_t e = cudaSuccess;
    double work = 0;
    switch (kind) {
    case GFP_PEAK_READ_HBM:
    case GFP_PEAK_READ_L2: {
        const uint64_t nv = bytes / 16;
        uint4 *v = (uint4 *)pr.alloc(nv * 16);
        if (!v) return GFP_PEAK_ERR_CUDA;
        if (cudaMemsetAsync(v, 0x5A, nv * 16, s) != cudaSuccess) return GFP_PEAK_ERR_CUDA;
        if (kind == GFP_PEAK_READ_HBM) {
            const int grid = persistent_grid(k_read, RD_THREADS, sms);
            out->grid = grid;
            out->threads = RD_THREADS;
            work = (double)nv * 16;
            e = time_launches(s, reps, [&] {
                k_read<<<grid, RD_THREADS, 0, s>>>(v, nv, sink);
                return cudaGetLastError();
            }, out);
        } else {
            const int grid = persistent_grid(k_read_l2, RD_THREADS, sms), passes = 64;
            out->grid = grid;
            out->threads = RD_THREADS;
            k_read_l2<<<grid, RD_THREADS, 0, s>>>(v, nv, 1, sink);   // bring into L2
            work = (double)nv * 16 * passes;
            e = time_launches(s, reps, [&] {
                k_read_l2<<<grid, RD_THREADS, 0, s>>>(v, nv, passes, sink);
                return cudaGetLastError();
            }, out);
        }
        break;
    }
    case GFP_PEAK_COPY_HBM: {
        const uint64_t nv = bytes / 32;
        uint4 *a = (uint4 *)pr.alloc(nv * 16), *b = (uint4 *)pr.alloc(nv * 16);
        if (!a || !b) return GFP_PEAK_ERR_CUDA;
        if (cudaMemsetAsync(a, 0x5A, nv * 16, s) != cudaSuccess) return GFP_PEAK_ERR_CUDA;
        const int grid = persistent_grid(k_copy, RD_THREADS, sms);
        out->grid = grid;
        out->threads = RD_THREADS;
        work = (double)nv * 32;
        e = time_launches(s, reps, [&] {
            k_copy<<<grid, RD_THREADS, 0, s>>>(a, b, nv);
            return cudaGetLastError();
        }, out);
        break;
    }
    case GFP_PEAK_DFMA: {
        const int grid = persistent_grid(k_dfma, 256, sms), iters = 1024;
        out->grid = grid;
        out->threads = 256;
        work = 2.0 * 8 * iters * (double)grid * 256;
        e = time_launches(s, reps, [&] {
            k_dfma<<<grid, 256, 0, s>>>(iters, 0.9999999, sink);
            return cudaGetLastError();
        }, out);
        break;
    }
    case GFP_PEAK_IMMA_SYNC: {
        const int grid = persistent_grid(k_imma, 256, sms), iters = 4096;
        out->grid = grid;
        out->threads = 256;
        work = 2.0 * 16 * 8 * 32 * 4 * (double)iters * grid * (256 / 32);
        e = time_launches(s, reps, [&] {
            k_imma<<<grid, 256, 0, s>>>(iters, 0x1234567u, sink);
            return cudaGetLastError();
        }, out);
        break;
    }
    case GFP_PEAK_LAUNCH: {
        cudaGraph_t g = nullptr;
        cudaGraphExec_t ge = nullptr;
        out->grid = sms;
        out->threads = 256;
        e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
        for (int i = 0; i < reps && e == cudaSuccess; ++i) {
            k_empty<<<sms, 256, 0, s>>>();
            e = cudaGetLastError();
        }
        cudaError_t e2 = cudaStreamEndCapture(s, &g);
        if (e == cudaSuccess) e = e2;
        if (e == cudaSuccess) e = cudaGraphInstantiate(&ge, g, 0);
        work = reps;
        if (e == cudaSuccess)
            e = time_launches(s, 5, [&] { return cudaGraphLaunch(ge, s); }, out);
        if (ge) cudaGraphExecDestroy(ge);
        if (g) cudaGraphDestroy(g);
        if (e != cudaSuccess) return GFP_PEAK_ERR_CUDA;
        out->work = work;
        out->rate = out->ms_best * 1e3 / reps;
        out->rate_median = out->ms_median * 1e3 / reps;
        return GFP_PEAK_OK;
    }
    }
    if (e != cudaSuccess || pr.err != cudaSuccess) return GFP_PEAK_ERR_CUDA;
    out->work = work;
    const double scale = (kind == GFP_PEAK_DFMA || kind == GFP_PEAK_IMMA_SYNC) ? 1e12 : 1e9;
    out->rate = work / (out->ms_best * 1e-3) / scale;
    out->rate_median = work / (out->ms_median * 1e-3) / scale;
    return GFP_PEAK_OK;
}
