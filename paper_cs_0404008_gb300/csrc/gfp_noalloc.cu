// gfp_dot_batched_noalloc: the batched dot product for callers that cannot
// allocate device memory.
//
// Some callers cannot call cudaMalloc at the point where they need a result:
// code running inside a real-time or interrupt-like host path where an
// allocation may block or fail, plug-ins whose host application owns the
// device memory budget and forbids allocations of its own, and code that must
// keep a fixed, pre-declared device footprint.  For them this entry point runs
// the same persistent batched kernel as gfp_dot_batched, but keeps every
// piece of scratch it needs (pair descriptors, work list, per-pair partial
// sums and completion tickets, work counters) in one file-scope device array
// of fixed size, so a call allocates nothing: no cudaMalloc, no cudaFree, no
// host heap allocation and no allocating library routine.
//
// Every device that loads the library holds the array until the process
// exits.  All calls share it and it keeps the last call's contents; the parts
// that must start at zero are cleared by every call.  Two calls whose work
// overlaps on the GPU race on the array, so a caller must order them (one
// stream, or events).
#include <algorithm>
#include <mutex>

#include "gfp_internal.h"

namespace gfp {
namespace {

constexpr uint64_t NA_MAX_PAIRS = 1024;    // GFP_NOALLOC_MAX_PAIRS
constexpr uint64_t NA_MAX_UNITS = 16384;   // GFP_NOALLOC_MAX_UNITS
constexpr uint64_t NA_CHUNK = 65536;       // elements per work unit
constexpr int NA_MAX_DEVICES = 64;

struct NoAllocScratch {
    DevPair pairs[NA_MAX_PAIRS];
    DevPairAux aux[NA_MAX_PAIRS];
    DevUnit units[NA_MAX_UNITS];
    unsigned long long slots[NA_MAX_PAIRS];   // zero at launch
    uint32_t tickets[NA_MAX_PAIRS];           // zero at launch
    uint32_t ctr[2];                          // zero at launch
};

static __device__ __align__(256) NoAllocScratch g_noalloc_scratch;

// Host staging for the descriptors (static: no host allocation either);
// guarded by na_mutex together with the per-device symbol addresses.
NoAllocScratch h_stage;
NoAllocScratch *d_addr[NA_MAX_DEVICES];
int d_sms[NA_MAX_DEVICES];
std::mutex na_mutex;

gfp_status fail(cudaError_t e)
{
    note_cuda_error(e);
    return GFP_ERR_CUDA;
}

double unit_cost(const DevUnit &u, const DevPairAux *aux)
{
    const uint32_t r = aux[u.pair].repr;
    const double c = r == FP64 ? 8.0 : r == PERTERM ? 6.0 : 1.0;
    return c * (double)(u.end - u.begin);
}

}  // namespace
}  // namespace gfp

using namespace gfp;

extern "C" GFP_API gfp_status gfp_dot_batched_noalloc(const gfp_dot_desc *d, uint64_t count,
                                                      uint32_t *out, void *stream)
{
    if (count && (!d || !out)) return GFP_ERR_INVALID;
    if (count == 0) return GFP_OK;
    if (count > NA_MAX_PAIRS) return GFP_ERR_INVALID;
    int dev = 0;
    cudaError_t e0 = cudaGetDevice(&dev);
    if (e0 != cudaSuccess) return fail(e0);
    if (dev < 0 || dev >= NA_MAX_DEVICES) return GFP_ERR_CUDA;

    std::lock_guard<std::mutex> g(na_mutex);
    // set-up, once per device, with that device current: the device address
    // of the scratch array (its host-side name is only a stand-in)
    if (!d_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) return fail(e != cudaSuccess ? e : cudaErrorInvalidSymbol);
        int sms = 0;
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return fail(e);
        d_sms[dev] = sms;
        d_addr[dev] = (NoAllocScratch *)p;
    }
    NoAllocScratch *dsc = d_addr[dev];

    // first pass: check every descriptor and count the work units, writing
    // nothing, so a refused batch leaves the staging and the device untouched
    uint64_t nu = 0;
    for (uint64_t j = 0; j < count; ++j) {
        const gfp_dot_desc &q = d[j];
        if (q.p < 2 || (q.n && (!q.x || !q.y))) return GFP_ERR_INVALID;
        if ((((uintptr_t)q.x) | ((uintptr_t)q.y)) & 3u) return GFP_ERR_INVALID;
        uint32_t r = q.repr;
        if (r == GFP_REPR_AUTO) r = gfp_choose_repr(nullptr, q.p, q.n);
        if (r < GFP_REPR_PERTERM || r >= GFP_REPR_COUNT_ || !repr_eligible((Repr)r, q.p))
            return GFP_ERR_UNSUPPORTED;
        const uint64_t units = q.n ? (q.n + NA_CHUNK - 1) / NA_CHUNK : 1;
        if (units > NA_MAX_UNITS - nu) return GFP_ERR_INVALID;   // work list would not fit
        nu += units;
    }

    // second pass: descriptors and work list in the static host staging
    uint64_t w = 0;
    for (uint64_t j = 0; j < count; ++j) {
        const gfp_dot_desc &q = d[j];
        uint32_t r = q.repr;
        if (r == GFP_REPR_AUTO) r = gfp_choose_repr(nullptr, q.p, q.n);
        const uint64_t units = q.n ? (q.n + NA_CHUNK - 1) / NA_CHUNK : 1;
        DevPair &pr = h_stage.pairs[j];
        pr.x = q.x;
        pr.y = q.y;
        pr.n = q.n;
        pr.k = k_for((Repr)r, q.p);
        pr.m = make_mod(q.p);
        h_stage.aux[j].repr = r;
        h_stage.aux[j].units = (uint32_t)units;
        if (q.n == 0) {
            h_stage.units[w++] = DevUnit{0, 0, (uint32_t)j, 0};
        } else {
            for (uint64_t b = 0; b < q.n; b += NA_CHUNK)
                h_stage.units[w++] = DevUnit{b, std::min<uint64_t>(q.n, b + NA_CHUNK), (uint32_t)j, 0};
        }
    }
    // largest units first; ties in (pair, start) order so the order is total.
    // std::sort sorts in place (std::stable_sort may take a heap buffer).
    std::sort(h_stage.units, h_stage.units + nu, [](const DevUnit &a, const DevUnit &b) {
        const double ca = unit_cost(a, h_stage.aux), cb = unit_cost(b, h_stage.aux);
        if (ca != cb) return ca > cb;
        if (a.pair != b.pair) return a.pair < b.pair;
        return a.begin < b.begin;
    });

    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    // pageable copies: the staging may be reused as soon as these return
    cudaError_t e = cudaMemcpyAsync(dsc->pairs, h_stage.pairs, count * sizeof(DevPair),
                                    cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(dsc->aux, h_stage.aux, count * sizeof(DevPairAux),
                            cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(dsc->units, h_stage.units, nu * sizeof(DevUnit),
                            cudaMemcpyHostToDevice, s);
    // clear what must start at zero (the kernel also leaves it zero, but a
    // previous launch that failed would not have)
    if (e == cudaSuccess)
        e = cudaMemsetAsync(dsc->slots, 0, count * sizeof(unsigned long long), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(dsc->tickets, 0, count * sizeof(uint32_t), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(dsc->ctr, 0, sizeof(dsc->ctr), s);
    if (e != cudaSuccess) return fail(e);
    BatchScratch sc;
    sc.slots = dsc->slots;
    sc.tickets = dsc->tickets;
    sc.ctr = dsc->ctr;
    e = launch_dot_batched(dsc->pairs, dsc->aux, dsc->units, (uint32_t)nu, sc, out,
                           dot_batched_grid(d_sms[dev]), s);
    if (e != cudaSuccess) return fail(e);
    return GFP_OK;
}
