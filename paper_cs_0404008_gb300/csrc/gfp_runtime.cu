// Host side of libgfpdot: per-modulus parameters (delay bounds of Eq. (1)
// and Eq. (2), the overflow correction of Section 3.3, Barrett and
// floating-point constants), the context and its scratch, representation
// choice, batch work lists, and the C entry points of the dot-product and
// matrix-vector paths.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>

#include "gfp_internal.h"

namespace gfp {

uint64_t delay_bound(uint32_t p, int acc_bits, int carried)
{
    if (p < 2 || acc_bits < 1 || acc_bits > 64) return 0;
    typedef unsigned __int128 u128;
    const u128 pm1 = (u128)(p - 1), sq = pm1 * pm1;
    const u128 lim = ((u128)1 << acc_bits) - 1;   // the sum must stay <= 2^m - 1
    const u128 extra = carried ? pm1 : 0;
    if (lim < extra + sq) return 0;
    const u128 k = (lim - extra) / sq;
    return k > (u128)UINT64_MAX ? UINT64_MAX : (uint64_t)k;
}

Mod make_mod(uint32_t p)
{
    Mod m;
    m.p = p;
    m.corr = (uint32_t)((UINT64_MAX % p + 1) % p);
    if ((p & (p - 1)) == 0) {   // power of two: floor(2^64/p) = 2^(64 - log2 p)
        int lg = 0;
        while ((1u << lg) != p) ++lg;
        m.mu = 1ull << (64 - lg);
    } else {
        m.mu = UINT64_MAX / p;  // equals floor(2^64/p) when p does not divide 2^64
    }
    m.pd = (double)p;
    m.invp = 1.0 / (double)p;
    return m;
}

// Centred accumulator (Section 3.2.2): largest k with k h^2 + (p-1) <= 2^63 - 1,
// h = (p-1)/2 (a carried residue in [0, p) plus k signed products).
uint64_t centered_bound(uint32_t p)
{
    if (p < 2) return 0;
    typedef unsigned __int128 u128;
    const u128 h = (u128)((p - 1) / 2), sq = h * h, lim = ((u128)1 << 63) - 1 - (u128)(p - 1);
    if (sq == 0) return UINT64_MAX;
    const u128 k = lim / sq;
    return k > (u128)UINT64_MAX ? UINT64_MAX : (uint64_t)k;
}

// Montgomery blocks (Sections 2.2, 3.2.1) with B = 2^32: a block sum T of k
// products must stay below p B for REDC: largest k with k (p-1)^2 < p 2^32.
uint64_t montgomery_bound(uint32_t p)
{
    if (p < 3 || (p & 1u) == 0) return 0;
    typedef unsigned __int128 u128;
    const u128 sq = (u128)(p - 1) * (p - 1), lim = ((u128)p << 32) - 1;
    const u128 k = lim / sq;
    return k > (u128)UINT64_MAX ? UINT64_MAX : (uint64_t)k;
}

uint64_t k_for(Repr r, uint32_t p)
{
    switch (r) {
    case U64_BLOCK: return delay_bound(p, 64, 1);
    case FP64: return delay_bound(p, 53, 1);
    case CENTERED: return centered_bound(p);
    case MONTGOMERY: return montgomery_bound(p);
    default: return 0;
    }
}

bool repr_eligible(Repr r, uint32_t p)
{
    if (p < 2) return false;
    switch (r) {
    case PERTERM:
    case U64_CARRY: return true;
    case U64_BLOCK: return delay_bound(p, 64, 1) >= 1;
    case FP64: return delay_bound(p, 53, 1) >= 1;
    case CENTERED: return centered_bound(p) >= 1;
    case MONTGOMERY: return montgomery_bound(p) >= 1;
    default: return false;
    }
}

}  // namespace gfp

using namespace gfp;

// ---------------------------------------------------------------------------
// helpers
// ---------------------------------------------------------------------------

// The last CUDA error seen by an entry point of this thread (diagnostics).
static thread_local cudaError_t g_last_cuda_error = cudaSuccess;

#define GFP_CUDA_TRY(expr)                                   \
    do {                                                     \
        cudaError_t e_ = (expr);                             \
        if (e_ != cudaSuccess) {                             \
            g_last_cuda_error = e_;                          \
            return GFP_ERR_CUDA;                             \
        }                                                    \
    } while (0)

void gfp::note_cuda_error(cudaError_t e) { g_last_cuda_error = e; }

static inline cudaStream_t as_stream(void *s) { return reinterpret_cast<cudaStream_t>(s); }

static inline uint32_t lg2_floor(uint64_t n)
{
    uint32_t l = 0;
    while (n >>= 1) ++l;
    return l;
}

// Built-in rule: the blocked 64-bit form when its interval is so long that no
// reduction happens inside a kernel, the wrap-counting form otherwise.
static Repr default_repr(uint32_t p)
{
    return delay_bound(p, 64, 1) >= (1ull << 20) ? U64_BLOCK : U64_CARRY;
}

static const gfp_plan_entry *plan_lookup(const gfp_ctx *ctx, uint32_t p, uint64_t n)
{
    if (!ctx || ctx->plan.empty()) return nullptr;
    auto it = ctx->plan.find({p, lg2_floor(n ? n : 1)});
    if (it != ctx->plan.end()) return &it->second;
    // nearest bucket of the same modulus
    const gfp_plan_entry *best = nullptr;
    uint32_t lg = lg2_floor(n ? n : 1), bd = 1000;
    for (auto &kv : ctx->plan) {
        if (kv.first.first != p) continue;
        uint32_t d = kv.first.second > lg ? kv.first.second - lg : lg - kv.first.second;
        if (d < bd) { bd = d; best = &kv.second; }
    }
    return best;
}

// Resolve the representation of one call; returns false if not eligible.
static bool resolve_repr(const gfp_ctx *ctx, uint32_t requested, uint32_t p, uint64_t n, Repr *out)
{
    uint32_t r = requested;
    if (r == GFP_REPR_AUTO && ctx) r = ctx->forced;
    if (r == GFP_REPR_AUTO) {
        const gfp_plan_entry *e = plan_lookup(ctx, p, n);
        r = (e && repr_eligible((Repr)e->repr, p)) ? e->repr : default_repr(p);
    }
    if (r < GFP_REPR_PERTERM || r >= GFP_REPR_COUNT_ || r == GFP_REPR_F16TC) return false;
    if (!repr_eligible((Repr)r, p)) return false;
    *out = (Repr)r;
    return true;
}

// The same without the tuned plan: the plan times the dot-product kernels, so
// products with other inner loops (sparse-row, CUDA-core block) take the
// forced representation if one is set, else the built-in rule.
static bool resolve_repr_untuned(const gfp_ctx *ctx, uint32_t p, Repr *out)
{
    uint32_t r = ctx ? (uint32_t)ctx->forced : (uint32_t)GFP_REPR_AUTO;
    if (r == GFP_REPR_AUTO) r = default_repr(p);
    if (r < GFP_REPR_PERTERM || r >= GFP_REPR_COUNT_ || r == GFP_REPR_F16TC) return false;
    if (!repr_eligible((Repr)r, p)) return false;
    *out = (Repr)r;
    return true;
}

static uint32_t chunk_for(const gfp_ctx *ctx, uint32_t p, uint64_t n)
{
    const gfp_plan_entry *e = plan_lookup(ctx, p, n);
    uint32_t c = (e && e->chunk) ? e->chunk : (ctx ? ctx->default_chunk : 65536u);
    return std::max<uint32_t>(4096u, c & ~3u);
}

static gfp_status check_range(gfp_ctx *ctx, const uint32_t *v, uint64_t n, uint32_t p,
                              cudaStream_t s)
{
    if (!ctx->validate || n == 0) return GFP_OK;
    GFP_CUDA_TRY(cudaMemsetAsync(ctx->d_flag, 0, sizeof(uint32_t), s));
    GFP_CUDA_TRY(launch_check_range(v, n, p, ctx->d_flag, s));
    ctx->launches++;
    uint32_t h = 0;
    GFP_CUDA_TRY(cudaMemcpyAsync(&h, ctx->d_flag, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    GFP_CUDA_TRY(cudaStreamSynchronize(s));
    return h ? GFP_ERR_RANGE : GFP_OK;
}

// ---------------------------------------------------------------------------
// batch work lists
// ---------------------------------------------------------------------------

namespace {

struct HostBatch {
    std::vector<DevPair> pairs;
    std::vector<DevPairAux> aux;
    std::vector<DevUnit> units;
    uint64_t bytes = 0;
};

// Relative per-element cost used to order units (longest processing time
// first): the floating-point form is bound by FP64 throughput and the
// per-term form by the remainder, both well above the streaming cost.
double repr_cost(Repr r)
{
    switch (r) {
    case FP64: return 8.0;
    case PERTERM: return 6.0;
    case CENTERED:
    case MONTGOMERY: return 1.5;
    default: return 1.0;
    }
}

gfp_status build_batch(const gfp_ctx *ctx, const gfp_dot_desc *d, uint64_t count, HostBatch &hb)
{
    if (count > 0xFFFFFFFFull) return GFP_ERR_INVALID;
    hb.pairs.resize(count);
    hb.aux.resize(count);
    std::vector<double> cost;
    uint64_t total_units = 0;
    for (uint64_t j = 0; j < count; ++j) {
        const gfp_dot_desc &q = d[j];
        if (q.p < 2) return GFP_ERR_INVALID;
        if (q.n && (!q.x || !q.y)) return GFP_ERR_INVALID;
        if ((((uintptr_t)q.x) | ((uintptr_t)q.y)) & 3u) return GFP_ERR_INVALID;
        Repr r;
        if (!resolve_repr(ctx, q.repr, q.p, q.n, &r)) return GFP_ERR_UNSUPPORTED;
        const uint32_t chunk = chunk_for(ctx, q.p, q.n);
        const uint64_t nu = q.n ? (q.n + chunk - 1) / chunk : 1;
        if (nu > 0xFFFFFFFFull) return GFP_ERR_INVALID;
        DevPair &pr = hb.pairs[j];
        pr.x = q.x;
        pr.y = q.y;
        pr.n = q.n;
        pr.m = make_mod(q.p);
        pr.k = k_for(r, q.p);
        hb.aux[j].repr = (uint32_t)r;
        hb.aux[j].units = (uint32_t)nu;
        total_units += nu;
        hb.bytes += q.n * 8;
    }
    if (total_units > 0xFFFFFFFFull) return GFP_ERR_INVALID;
    hb.units.resize(total_units);
    cost.resize(total_units);
    uint64_t u = 0;
    for (uint64_t j = 0; j < count; ++j) {
        const uint64_t n = d[j].n;
        const uint32_t chunk = chunk_for(ctx, d[j].p, n);
        const double c = repr_cost((Repr)hb.aux[j].repr);
        if (n == 0) {
            hb.units[u] = DevUnit{0, 0, (uint32_t)j, 0};
            cost[u++] = 0.0;
            continue;
        }
        for (uint64_t b = 0; b < n; b += chunk) {
            const uint64_t e = std::min<uint64_t>(n, b + chunk);
            hb.units[u] = DevUnit{b, e, (uint32_t)j, 0};
            cost[u++] = c * (double)(e - b);
        }
    }
    // longest processing time first (stable: equal costs keep pair order)
    std::vector<uint32_t> order(total_units);
    for (uint64_t i = 0; i < total_units; ++i) order[i] = (uint32_t)i;
    std::stable_sort(order.begin(), order.end(),
                     [&](uint32_t a, uint32_t b) { return cost[a] > cost[b]; });
    std::vector<DevUnit> sorted(total_units);
    for (uint64_t i = 0; i < total_units; ++i) sorted[i] = hb.units[order[i]];
    hb.units.swap(sorted);
    return GFP_OK;
}

inline size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

// Device image of a batch: [pairs | aux | units | slots | tickets | ctr].
struct BatchLayout {
    size_t pairs, aux, units, slots, tickets, ctr, total;
    BatchLayout(uint64_t count, uint64_t n_units)
    {
        pairs = 0;
        aux = align256(pairs + count * sizeof(DevPair));
        units = align256(aux + count * sizeof(DevPairAux));
        slots = align256(units + n_units * sizeof(DevUnit));
        tickets = align256(slots + count * sizeof(unsigned long long));
        ctr = align256(tickets + count * sizeof(uint32_t));
        total = align256(ctr + 2 * sizeof(uint32_t));
    }
};

}  // namespace

struct gfp_batch_plan {
    gfp_ctx *ctx = nullptr;
    void *mem = nullptr;
    uint64_t count = 0, n_units = 0, bytes = 0;
    const DevPair *pairs = nullptr;
    const DevPairAux *aux = nullptr;
    const DevUnit *units = nullptr;
    BatchScratch sc;
    int grid = 0;
};

static gfp_status upload_batch(const HostBatch &hb, void *mem, const BatchLayout &L,
                               bool zero_scratch, cudaStream_t s)
{
    char *base = (char *)mem;
    const uint64_t count = hb.pairs.size();
    if (count) {
        GFP_CUDA_TRY(cudaMemcpyAsync(base + L.pairs, hb.pairs.data(), count * sizeof(DevPair),
                                     cudaMemcpyHostToDevice, s));
        GFP_CUDA_TRY(cudaMemcpyAsync(base + L.aux, hb.aux.data(), count * sizeof(DevPairAux),
                                     cudaMemcpyHostToDevice, s));
    }
    if (!hb.units.empty())
        GFP_CUDA_TRY(cudaMemcpyAsync(base + L.units, hb.units.data(),
                                     hb.units.size() * sizeof(DevUnit), cudaMemcpyHostToDevice, s));
    if (zero_scratch) GFP_CUDA_TRY(cudaMemsetAsync(base + L.slots, 0, L.total - L.slots, s));
    return GFP_OK;
}

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------

extern "C" {

GFP_API const char *gfp_status_string(int st)
{
    switch (st) {
    case GFP_OK: return "GFP_OK";
    case GFP_PENDING: return "GFP_PENDING";
    case GFP_ERR_INVALID: return "GFP_ERR_INVALID";
    case GFP_ERR_RANGE: return "GFP_ERR_RANGE";
    case GFP_ERR_UNSUPPORTED: return "GFP_ERR_UNSUPPORTED";
    case GFP_ERR_NOMEM: return "GFP_ERR_NOMEM";
    case GFP_ERR_CUDA: return "GFP_ERR_CUDA";
    case GFP_ERR_AGAIN: return "GFP_ERR_AGAIN";
    case GFP_ERR_TIMEOUT: return "GFP_ERR_TIMEOUT";
    case GFP_ERR_UNKNOWN_TICKET: return "GFP_ERR_UNKNOWN_TICKET";
    case GFP_ERR_CANCELLED: return "GFP_ERR_CANCELLED";
    default: return "GFP_UNKNOWN_STATUS";
    }
}

GFP_API const char *gfp_last_cuda_error(void)
{
    return g_last_cuda_error == cudaSuccess ? "no CUDA error" : cudaGetErrorString(g_last_cuda_error);
}

GFP_API uint64_t gfp_delay_bound(uint32_t p, int acc_bits, int carried)
{
    return delay_bound(p, acc_bits, carried);
}

GFP_API gfp_status gfp_get_params(uint32_t p, gfp_params *out)
{
    if (p < 2 || !out) return GFP_ERR_INVALID;
    const Mod m = make_mod(p);
    out->p = p;
    out->corr = m.corr;
    out->k_u64 = delay_bound(p, 64, 1);
    out->k_fp64 = delay_bound(p, 53, 1);
    out->barrett_mu = m.mu;
    out->inv_p = m.invp;
    out->fp64_ok = out->k_fp64 >= 1;
    out->k_centered = centered_bound(p);
    out->k_montgomery = montgomery_bound(p);
    return GFP_OK;
}

GFP_API uint32_t gfp_reduce_u64(uint64_t x, uint32_t p)
{
    if (p < 2) return 0;
    return reduce64(x, make_mod(p));
}

GFP_API double gfp_reduce_f64(double T, uint32_t p)
{
    if (p < 2) return 0.0;
    return reduce_f64(T, make_mod(p));
}

GFP_API gfp_repr gfp_choose_repr(const gfp_ctx *ctx, uint32_t p, uint64_t n)
{
    Repr r;
    if (p < 2 || !resolve_repr(ctx, GFP_REPR_AUTO, p, n, &r)) return GFP_REPR_AUTO;
    return (gfp_repr)r;
}

GFP_API gfp_status gfp_plan_load(gfp_ctx *ctx, const char *path);   // gfp_tune.cu

GFP_API gfp_status gfp_context_create(int device, gfp_ctx **out)
{
    GFP_TRACE();
    if (!out) return GFP_ERR_INVALID;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev)
        return GFP_ERR_CUDA;
    GFP_CUDA_TRY(cudaSetDevice(device));
    gfp_ctx *c = new (std::nothrow) gfp_ctx();
    if (!c) return GFP_ERR_NOMEM;
    c->device = device;
    if (cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, device) !=
        cudaSuccess) {
        delete c;
        return GFP_ERR_CUDA;
    }
    const size_t ring_bytes = (size_t)c->ring_size * sizeof(unsigned long long);
    void *mem = nullptr;
    if (cudaMalloc(&mem, ring_bytes + 256) != cudaSuccess) {
        delete c;
        return GFP_ERR_NOMEM;
    }
    cudaMemset(mem, 0, ring_bytes + 256);
    c->ring_slots = (unsigned long long *)mem;
    c->d_flag = (uint32_t *)((char *)mem + ring_bytes);
    if (cudaDeviceSynchronize() != cudaSuccess) {
        cudaFree(mem);
        delete c;
        return GFP_ERR_CUDA;
    }
    if (const char *e = getenv("GFP_FORCE_REPR")) {
        int r = atoi(e);
        if (r >= 0 && r < GFP_REPR_COUNT_) c->forced = (gfp_repr)r;
    }
    if (const char *e = getenv("GFP_VALIDATE")) c->validate = atoi(e) != 0;
    if (const char *e = getenv("GFP_PLAN_FILE")) gfp_plan_load(c, e);
    *out = c;
    return GFP_OK;
}

GFP_API gfp_status gfp_context_destroy(gfp_ctx *ctx)
{
    GFP_TRACE();
    if (!ctx) return GFP_ERR_INVALID;
    cudaSetDevice(ctx->device);
    cudaDeviceSynchronize();
    for (auto &kv : ctx->graphs) cudaGraphExecDestroy(kv.second);
    for (auto &kv : ctx->seq_graphs) cudaGraphExecDestroy(kv.second);
    if (ctx->pingpong) cudaFree(ctx->pingpong);
    if (ctx->seq_slots) cudaFree(ctx->seq_slots);
    for (int i = 0; i < gfp_ctx::kCopyStreams; ++i)
        if (ctx->copy_streams[i]) cudaStreamDestroy(ctx->copy_streams[i]);
    for (int i = 0; i <= gfp_ctx::kCopyStreams; ++i)
        if (ctx->copy_events[i]) cudaEventDestroy(ctx->copy_events[i]);
    cudaFree(ctx->ring_slots);
    if (ctx->bw) cudaFree(ctx->bw);
    if (ctx->stage) cudaFree(ctx->stage);
    if (ctx->stage_out) cudaFree(ctx->stage_out);
    if (ctx->blk_ws) cudaFree(ctx->blk_ws);
    delete ctx;
    return GFP_OK;
}

GFP_API gfp_status gfp_set_repr(gfp_ctx *ctx, gfp_repr repr)
{
    GFP_TRACE();
    if (!ctx || repr < GFP_REPR_AUTO || repr >= GFP_REPR_COUNT_) return GFP_ERR_INVALID;
    ctx->forced = repr;
    return GFP_OK;
}

GFP_API gfp_status gfp_set_validate(gfp_ctx *ctx, int on)
{
    GFP_TRACE();
    if (!ctx) return GFP_ERR_INVALID;
    ctx->validate = on != 0;
    return GFP_OK;
}

GFP_API uint64_t gfp_launch_count(const gfp_ctx *ctx) { return ctx ? ctx->launches.load() : 0; }

GFP_API gfp_status gfp_dot(gfp_ctx *ctx, uint32_t p, uint64_t n, const uint32_t *x,
                           const uint32_t *y, uint32_t *out, void *stream)
{
    GFP_TRACE();
    if (!ctx || p < 2 || !out || (n && (!x || !y))) return GFP_ERR_INVALID;
    if ((((uintptr_t)x) | ((uintptr_t)y) | ((uintptr_t)out)) & 3u) return GFP_ERR_INVALID;
    Repr r;
    if (!resolve_repr(ctx, GFP_REPR_AUTO, p, n, &r)) return GFP_ERR_UNSUPPORTED;
    cudaStream_t s = as_stream(stream);
    if (ctx->validate) {
        gfp_status st = check_range(ctx, x, n, p, s);
        if (st == GFP_OK) st = check_range(ctx, y, n, p, s);
        if (st != GFP_OK) return st;
    }
    const uint32_t slot = ctx->ring_pos.fetch_add(1) % ctx->ring_size;
    const int grid = dot_single_grid(r, n, ctx->sm_count);
    GFP_CUDA_TRY(launch_dot_single(r, make_mod(p), k_for(r, p), n, x, y, ctx->ring_slots + slot,
                                   out, grid, s));
    ctx->launches++;
    return GFP_OK;
}

GFP_API gfp_status gfp_batch_plan_create(gfp_ctx *ctx, const gfp_dot_desc *d, uint64_t count,
                                         gfp_batch_plan **out)
{
    GFP_TRACE();
    if (!ctx || !out || (count && !d)) return GFP_ERR_INVALID;
    *out = nullptr;
    HostBatch hb;
    gfp_status st = build_batch(ctx, d, count, hb);
    if (st != GFP_OK) return st;
    BatchLayout L(count, hb.units.size());
    gfp_batch_plan *pl = new (std::nothrow) gfp_batch_plan();
    if (!pl) return GFP_ERR_NOMEM;
    if (cudaMalloc(&pl->mem, L.total) != cudaSuccess) {
        delete pl;
        return GFP_ERR_NOMEM;
    }
    st = upload_batch(hb, pl->mem, L, true, 0);
    if (st == GFP_OK && cudaDeviceSynchronize() != cudaSuccess) st = GFP_ERR_CUDA;
    if (st != GFP_OK) {
        cudaFree(pl->mem);
        delete pl;
        return st;
    }
    char *base = (char *)pl->mem;
    pl->ctx = ctx;
    pl->count = count;
    pl->n_units = hb.units.size();
    pl->bytes = hb.bytes;
    pl->pairs = (const DevPair *)(base + L.pairs);
    pl->aux = (const DevPairAux *)(base + L.aux);
    pl->units = (const DevUnit *)(base + L.units);
    pl->sc.slots = (unsigned long long *)(base + L.slots);
    pl->sc.tickets = (uint32_t *)(base + L.tickets);
    pl->sc.ctr = (uint32_t *)(base + L.ctr);
    pl->grid = dot_batched_grid(ctx->sm_count);
    *out = pl;
    return GFP_OK;
}

GFP_API gfp_status gfp_batch_plan_exec(gfp_batch_plan *pl, uint32_t *out, void *stream)
{
    GFP_TRACE();
    if (!pl || (pl->count && !out)) return GFP_ERR_INVALID;
    if (pl->count == 0) return GFP_OK;
    GFP_CUDA_TRY(launch_dot_batched(pl->pairs, pl->aux, pl->units, (uint32_t)pl->n_units, pl->sc,
                                    out, pl->grid, as_stream(stream)));
    pl->ctx->launches++;
    return GFP_OK;
}

GFP_API gfp_status gfp_batch_plan_info(const gfp_batch_plan *pl, uint64_t *units, uint64_t *bytes)
{
    GFP_TRACE();
    if (!pl) return GFP_ERR_INVALID;
    if (units) *units = pl->n_units;
    if (bytes) *bytes = pl->bytes;
    return GFP_OK;
}

GFP_API gfp_status gfp_batch_plan_destroy(gfp_batch_plan *pl)
{
    GFP_TRACE();
    if (!pl) return GFP_ERR_INVALID;
    cudaFree(pl->mem);
    delete pl;
    return GFP_OK;
}

static gfp_status batched_oneshot(gfp_ctx *ctx, const gfp_dot_desc *d, uint64_t count,
                                  uint32_t *out, cudaStream_t s)
{
    HostBatch hb;
    gfp_status st = build_batch(ctx, d, count, hb);
    if (st != GFP_OK) return st;
    if (ctx->validate)
        for (uint64_t j = 0; j < count; ++j) {
            st = check_range(ctx, d[j].x, d[j].n, d[j].p, s);
            if (st == GFP_OK) st = check_range(ctx, d[j].y, d[j].n, d[j].p, s);
            if (st != GFP_OK) return st;
        }
    BatchLayout L(count, hb.units.size());
    bool fresh = false;
    if (L.total > ctx->bw_bytes) {
        if (ctx->bw) {
            GFP_CUDA_TRY(cudaStreamSynchronize(s));
            cudaFree(ctx->bw);
            ctx->bw = nullptr;
            ctx->bw_bytes = 0;
        }
        const size_t want = std::max<size_t>(L.total, (size_t)1 << 20);
        if (cudaMalloc(&ctx->bw, want) != cudaSuccess) return GFP_ERR_NOMEM;
        ctx->bw_bytes = want;
        fresh = true;
    }
    // the scratch region moves with the layout: clear it whenever it may hold
    // stale values (fresh buffer, or a layout with a different offset)
    const bool zero = fresh || ctx->bw_slots_off != L.slots;
    st = upload_batch(hb, ctx->bw, L, false, s);
    if (st != GFP_OK) return st;
    char *base = (char *)ctx->bw;
    if (zero) GFP_CUDA_TRY(cudaMemsetAsync(base + L.slots, 0, ctx->bw_bytes - L.slots, s));
    ctx->bw_slots_off = L.slots;
    BatchScratch sc;
    sc.slots = (unsigned long long *)(base + L.slots);
    sc.tickets = (uint32_t *)(base + L.tickets);
    sc.ctr = (uint32_t *)(base + L.ctr);
    GFP_CUDA_TRY(launch_dot_batched((const DevPair *)(base + L.pairs),
                                    (const DevPairAux *)(base + L.aux),
                                    (const DevUnit *)(base + L.units), (uint32_t)hb.units.size(),
                                    sc, out, dot_batched_grid(ctx->sm_count), s));
    ctx->launches++;
    return GFP_OK;
}

GFP_API gfp_status gfp_dot_batched(gfp_ctx *ctx, const gfp_dot_desc *d, uint64_t count,
                                   uint32_t *out, void *stream)
{
    GFP_TRACE();
    if (!ctx || (count && (!d || !out))) return GFP_ERR_INVALID;
    if (count == 0) return GFP_OK;
    std::lock_guard<std::mutex> g(ctx->mu);
    return batched_oneshot(ctx, d, count, out, as_stream(stream));
}

GFP_API gfp_status gfp_dot_batched_host(gfp_ctx *ctx, uint64_t count, const uint32_t *p,
                                        const uint64_t *n, const uint64_t *off,
                                        const uint32_t *x_host, const uint32_t *y_host,
                                        uint64_t total, uint32_t *out_host, void *stream)
{
    GFP_TRACE();
    if (!ctx || (count && (!p || !n || !off || !out_host))) return GFP_ERR_INVALID;
    if (count == 0) return GFP_OK;
    if (total && (!x_host || !y_host)) return GFP_ERR_INVALID;
    for (uint64_t j = 0; j < count; ++j)
        if ((off[j] & 3u) || off[j] > total || n[j] > total - off[j] || p[j] < 2)
            return GFP_ERR_INVALID;
    std::lock_guard<std::mutex> g(ctx->mu);
    cudaStream_t s = as_stream(stream);
    const size_t need = (size_t)2 * (total ? total : 1);
    if (need > ctx->stage_elems) {
        GFP_CUDA_TRY(cudaStreamSynchronize(s));
        if (ctx->stage) cudaFree(ctx->stage);
        ctx->stage = nullptr;
        ctx->stage_elems = 0;
        if (cudaMalloc(&ctx->stage, need * 4) != cudaSuccess) return GFP_ERR_NOMEM;
        ctx->stage_elems = need;
    }
    if (count > ctx->stage_out_elems) {
        GFP_CUDA_TRY(cudaStreamSynchronize(s));
        if (ctx->stage_out) cudaFree(ctx->stage_out);
        ctx->stage_out = nullptr;
        ctx->stage_out_elems = 0;
        if (cudaMalloc(&ctx->stage_out, count * 4) != cudaSuccess) return GFP_ERR_NOMEM;
        ctx->stage_out_elems = count;
    }
    uint32_t *dx = ctx->stage, *dy = ctx->stage + (total ? total : 1);
    if (total) {
        if (!ctx->copy_streams[0]) {
            for (int i = 0; i < gfp_ctx::kCopyStreams; ++i)
                GFP_CUDA_TRY(cudaStreamCreateWithFlags(&ctx->copy_streams[i], cudaStreamNonBlocking));
            for (int i = 0; i <= gfp_ctx::kCopyStreams; ++i)
                GFP_CUDA_TRY(cudaEventCreateWithFlags(&ctx->copy_events[i], cudaEventDisableTiming));
        }
        // the copies may overwrite staging that earlier work on `s` still reads
        GFP_CUDA_TRY(cudaEventRecord(ctx->copy_events[gfp_ctx::kCopyStreams], s));
        const uint64_t per = (total + gfp_ctx::kCopyStreams - 1) / gfp_ctx::kCopyStreams;
        for (int i = 0; i < gfp_ctx::kCopyStreams; ++i) {
            const uint64_t b = (uint64_t)i * per;
            if (b >= total) break;
            const uint64_t len = std::min<uint64_t>(per, total - b);
            cudaStream_t cs = ctx->copy_streams[i];
            GFP_CUDA_TRY(cudaStreamWaitEvent(cs, ctx->copy_events[gfp_ctx::kCopyStreams], 0));
            GFP_CUDA_TRY(cudaMemcpyAsync(dx + b, x_host + b, len * 4, cudaMemcpyHostToDevice, cs));
            GFP_CUDA_TRY(cudaMemcpyAsync(dy + b, y_host + b, len * 4, cudaMemcpyHostToDevice, cs));
            GFP_CUDA_TRY(cudaEventRecord(ctx->copy_events[i], cs));
            GFP_CUDA_TRY(cudaStreamWaitEvent(s, ctx->copy_events[i], 0));
        }
    }
    std::vector<gfp_dot_desc> d(count);
    for (uint64_t j = 0; j < count; ++j)
        d[j] = gfp_dot_desc{p[j], GFP_REPR_AUTO, n[j], dx + off[j], dy + off[j]};
    gfp_status st = batched_oneshot(ctx, d.data(), count, ctx->stage_out, s);
    if (st != GFP_OK) return st;
    GFP_CUDA_TRY(cudaMemcpyAsync(out_host, ctx->stage_out, count * 4, cudaMemcpyDeviceToHost, s));
    GFP_CUDA_TRY(cudaStreamSynchronize(s));
    return GFP_OK;
}

GFP_API gfp_status gfp_matvec(gfp_ctx *ctx, uint32_t p, uint64_t rows, uint64_t cols,
                              const uint32_t *A, uint64_t lda, const uint32_t *x, uint32_t *y,
                              void *stream)
{
    GFP_TRACE();
    if (!ctx || p < 2 || lda < cols || (rows && !y) || (rows && cols && (!A || !x)))
        return GFP_ERR_INVALID;
    if ((((uintptr_t)A) | ((uintptr_t)x) | ((uintptr_t)y)) & 3u) return GFP_ERR_INVALID;
    if (rows == 0) return GFP_OK;
    Repr r;
    if (!resolve_repr(ctx, GFP_REPR_AUTO, p, cols, &r)) return GFP_ERR_UNSUPPORTED;
    cudaStream_t s = as_stream(stream);
    if (ctx->validate) {
        gfp_status st = check_range(ctx, x, cols, p, s);
        for (uint64_t i = 0; st == GFP_OK && i < rows; ++i) st = check_range(ctx, A + i * lda, cols, p, s);
        if (st != GFP_OK) return st;
    }
    GFP_CUDA_TRY(launch_matvec(r, make_mod(p), k_for(r, p), rows, cols, A, lda, x, y,
                               ctx->sm_count, s));
    ctx->launches++;
    return GFP_OK;
}

GFP_API gfp_status gfp_matvec_iterate(gfp_ctx *ctx, uint32_t p, uint64_t n, const uint32_t *A,
                                      uint64_t lda, const uint32_t *x0, uint32_t *Y,
                                      uint32_t iters, void *stream)
{
    GFP_TRACE();
    if (!ctx || p < 2 || lda < n || (n && (!A || !x0 || !Y))) return GFP_ERR_INVALID;
    if ((((uintptr_t)A) | ((uintptr_t)x0) | ((uintptr_t)Y)) & 3u) return GFP_ERR_INVALID;
    if (n == 0 || iters == 0) return GFP_OK;
    Repr r;
    if (!resolve_repr(ctx, GFP_REPR_AUTO, p, n, &r)) return GFP_ERR_UNSUPPORTED;
    cudaStream_t s = as_stream(stream);
    std::lock_guard<std::mutex> g(ctx->mu);
    gfp_ctx::GraphKey key{p, n, A, lda, x0, Y, iters, (int)r};
    auto it = ctx->graphs.find(key);
    if (it == ctx->graphs.end()) {
        // warm the launch path (function attributes) outside capture
        cudaStream_t cs;
        GFP_CUDA_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        const Mod m = make_mod(p);
        const uint64_t k = k_for(r, p);
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        for (uint32_t t = 0; e == cudaSuccess && t < iters; ++t) {
            const uint32_t *xt = t ? Y + (uint64_t)(t - 1) * n : x0;
            e = launch_matvec(r, m, k, n, n, A, lda, xt, Y + (uint64_t)t * n, ctx->sm_count, cs);
        }
        cudaError_t e2 = cudaStreamEndCapture(cs, &graph);
        if (e == cudaSuccess) e = e2;
        cudaGraphExec_t exec = nullptr;
        if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        cudaStreamDestroy(cs);
        if (e != cudaSuccess) return GFP_ERR_CUDA;
        it = ctx->graphs.emplace(key, exec).first;
    }
    GFP_CUDA_TRY(cudaGraphLaunch(it->second, s));
    ctx->launches += iters;
    return GFP_OK;
}

static gfp_status check_range_rows(gfp_ctx *ctx, const uint32_t *M, uint64_t rows, uint64_t cols,
                                   uint64_t ld, uint32_t p, cudaStream_t s)
{
    if (!ctx->validate) return GFP_OK;
    if (ld == cols) return check_range(ctx, M, rows * cols, p, s);
    for (uint64_t i = 0; i < rows; ++i) {
        gfp_status st = check_range(ctx, M + i * ld, cols, p, s);
        if (st != GFP_OK) return st;
    }
    return GFP_OK;
}

// CTAs of one tensor-core block kernel: one per SM, or the context's cap
static int block_sms(const gfp_ctx *ctx)
{
    return (ctx->blk_sms > 0 && ctx->blk_sms < ctx->sm_count) ? ctx->blk_sms : ctx->sm_count;
}

// Block-product workspace of the context for shape (m, k, nb) followed by
// `passes` residue matrices (m x nb uint32 each); the caller holds ctx->mu.
static gfp_status ensure_block_ws(gfp_ctx *ctx, uint64_t m, uint64_t k, uint64_t nb, int passes,
                                  cudaStream_t s)
{
    const size_t tc_need = block_tc_workspace_bytes(m, k, nb);
    const size_t need = tc_need + (size_t)passes * m * nb * 4;
    if (need > ctx->blk_ws_bytes) {
        GFP_CUDA_TRY(cudaDeviceSynchronize());
        if (ctx->blk_ws) cudaFree(ctx->blk_ws);
        ctx->blk_ws = nullptr;
        ctx->blk_ws_bytes = 0;
        if (cudaMalloc(&ctx->blk_ws, need) != cudaSuccess) return GFP_ERR_NOMEM;
        GFP_CUDA_TRY(cudaMemset(ctx->blk_ws, 0, need));
        ctx->blk_ws_bytes = need;
    }
    if (m != ctx->blk_m || k != ctx->blk_k || nb != ctx->blk_nb) {
        // the partial-sum region moves with the shape: clear it
        const size_t z = block_tc_bimg_bytes(k, nb);
        GFP_CUDA_TRY(cudaMemsetAsync((uint8_t *)ctx->blk_ws + z, 0, tc_need - z, s));
        ctx->blk_m = m;
        ctx->blk_k = k;
        ctx->blk_nb = nb;
    }
    return GFP_OK;
}

GFP_API gfp_status gfp_matmul_block(gfp_ctx *ctx, uint32_t p, uint64_t m, uint64_t k, uint64_t nb,
                                    const uint32_t *A, uint64_t lda, const uint32_t *B,
                                    uint64_t ldb, uint32_t *C, uint64_t ldc, void *stream)
{
    GFP_TRACE();
    if (!ctx || p < 2 || lda < k || ldb < nb || ldc < nb) return GFP_ERR_INVALID;
    if ((m && nb && !C) || (m && k && !A) || (k && nb && !B)) return GFP_ERR_INVALID;
    if ((((uintptr_t)A) | ((uintptr_t)B) | ((uintptr_t)C)) & 3u) return GFP_ERR_INVALID;
    if (m == 0 || nb == 0) return GFP_OK;
    cudaStream_t s = as_stream(stream);
    if (k == 0) {
        GFP_CUDA_TRY(cudaMemset2DAsync(C, ldc * 4, 0, nb * 4, m, s));
        return GFP_OK;
    }
    // tensor cores: directly for p <= 65791, through residues modulo small
    // primes (one pass each, then a Garner recombination) above that
    const bool layout_ok = block_tc_layout_ok(A, lda);
    RnsConst rc;
    const bool direct_ok = layout_ok && p <= BLOCK_TC_MAX_P;
    bool rns_ok = layout_ok && p > BLOCK_TC_MAX_P && block_rns_plan(p, k, &rc);
    if (rns_ok && ctx->forced == GFP_REPR_AUTO) {
        // the residue passes each stream A once (about 4 TB/s) after two
        // launches; the CUDA-core kernel pays per multiply-add (about 4.5e12/s
        // at best): keep the residues only where they are expected to win
        const double t_rns = rc.L * (25e-6 + 4.0 * (double)m * (double)k / 4.0e12);
        const double t_cc = (double)m * (double)k * (double)nb / 4.5e12;
        if (t_cc <= t_rns) rns_ok = false;
    }
    const bool tc_ok = direct_ok || rns_ok;
    bool use_tc = false;
    Repr r = U64_CARRY;
    if (ctx->forced == GFP_REPR_F16TC) {
        if (!tc_ok) return GFP_ERR_UNSUPPORTED;
        use_tc = true;
    } else if (ctx->forced == GFP_REPR_AUTO && tc_ok) {
        use_tc = true;
    } else if (!resolve_repr_untuned(ctx, p, &r)) {
        return GFP_ERR_UNSUPPORTED;
    }
    if (ctx->validate) {
        gfp_status st = check_range_rows(ctx, A, m, k, lda, p, s);
        if (st == GFP_OK) st = check_range_rows(ctx, B, k, nb, ldb, p, s);
        if (st != GFP_OK) return st;
    }
    const Mod mod = make_mod(p);
    if (!use_tc) {
        GFP_CUDA_TRY(launch_block_cc(r, mod, k_for(r, p), m, k, nb, A, lda, B, ldb, C, ldc, s));
        ctx->launches++;
        return GFP_OK;
    }
    std::lock_guard<std::mutex> g(ctx->mu);
    const size_t tc_need = block_tc_workspace_bytes(m, k, nb);
    {
        const gfp_status st = ensure_block_ws(ctx, m, k, nb, rns_ok ? rc.L : 0, s);
        if (st != GFP_OK) return st;
    }
    int launches = 0;
    if (!rns_ok) {
        GFP_CUDA_TRY(launch_block_tc(mod, m, k, nb, A, lda, B, ldb, C, ldc, ctx->blk_ws, block_sms(ctx),
                                     s, &launches));
    } else {
        uint32_t *R = (uint32_t *)((uint8_t *)ctx->blk_ws + tc_need);
        for (int l = 0; l < rc.L; ++l)
            GFP_CUDA_TRY(launch_block_tc(make_mod(rc.mod[l]), m, k, nb, A, lda, B, ldb, R + (size_t)l * m * nb,
                                         nb, ctx->blk_ws, block_sms(ctx), s, &launches, true));
        GFP_CUDA_TRY(launch_block_crt(R, m, nb, C, ldc, rc, ctx->sm_count, s));
        ++launches;
    }
    ctx->launches += launches;
    return GFP_OK;
}

// A prepared once for repeated block products: its tensor-core digit
// images, one per modulus (p itself, or each residue-pass modulus).
struct gfp_block_prep {
    uint32_t p = 0;
    uint64_t m = 0, k = 0;
    int passes = 0;          // 1: p <= 65536 directly; more: residue passes
    RnsConst rc{};
    void *mem = nullptr;
    size_t per = 0;          // bytes of one image
};

GFP_API gfp_status gfp_block_prepare(gfp_ctx *ctx, uint32_t p, uint64_t m, uint64_t k,
                                     const uint32_t *A, uint64_t lda, gfp_block_prep **out)
{
    GFP_TRACE();
    if (!out) return GFP_ERR_INVALID;
    *out = nullptr;
    if (!ctx || p < 2 || m == 0 || k == 0 || lda < k || !A || (((uintptr_t)A) & 3u))
        return GFP_ERR_INVALID;
    RnsConst rc{};
    int passes = 1;
    if (p > RNS_PRIME_MAX) {   // beyond the 8-bit digit planes: residue passes
        if (!block_rns_plan(p, k, &rc)) return GFP_ERR_UNSUPPORTED;
        passes = rc.L;
    }
    if (ctx->validate) {
        const gfp_status st = check_range_rows(ctx, A, m, k, lda, p, nullptr);
        if (st != GFP_OK) return st;
    }
    gfp_block_prep *pp = new (std::nothrow) gfp_block_prep();
    if (!pp) return GFP_ERR_NOMEM;
    pp->per = block_prep_a_bytes(m, k);
    if (cudaMalloc(&pp->mem, pp->per * passes) != cudaSuccess) {
        delete pp;
        return GFP_ERR_NOMEM;
    }
    cudaError_t e = cudaSuccess;
    for (int l = 0; l < passes && e == cudaSuccess; ++l)
        e = launch_block_prep_a(make_mod(passes == 1 ? p : rc.mod[l]), m, k, A, lda, passes > 1,
                                (uint8_t *)pp->mem + pp->per * l, nullptr);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        note_cuda_error(e);
        cudaFree(pp->mem);
        delete pp;
        return GFP_ERR_CUDA;
    }
    ctx->launches += passes;
    pp->p = p;
    pp->m = m;
    pp->k = k;
    pp->passes = passes;
    pp->rc = rc;
    *out = pp;
    return GFP_OK;
}

GFP_API gfp_status gfp_block_prep_info(const gfp_block_prep *pp, uint64_t *bytes, uint32_t *passes)
{
    if (!pp) return GFP_ERR_INVALID;
    if (bytes) *bytes = (uint64_t)pp->per * pp->passes;
    if (passes) *passes = (uint32_t)pp->passes;
    return GFP_OK;
}

GFP_API gfp_status gfp_block_prep_destroy(gfp_block_prep *pp)
{
    GFP_TRACE();
    if (!pp) return GFP_ERR_INVALID;
    cudaDeviceSynchronize();
    cudaFree(pp->mem);
    delete pp;
    return GFP_OK;
}

GFP_API gfp_status gfp_matmul_block_prepared(gfp_ctx *ctx, const gfp_block_prep *pp, uint64_t nb,
                                             const uint32_t *B, uint64_t ldb, uint32_t *C,
                                             uint64_t ldc, void *stream)
{
    GFP_TRACE();
    if (!ctx || !pp || ldb < nb || ldc < nb) return GFP_ERR_INVALID;
    if (nb && (!B || !C)) return GFP_ERR_INVALID;
    if ((((uintptr_t)B) | ((uintptr_t)C)) & 3u) return GFP_ERR_INVALID;
    if (nb == 0) return GFP_OK;
    cudaStream_t s = as_stream(stream);
    const uint64_t m = pp->m, k = pp->k;
    if (ctx->validate) {
        const gfp_status st = check_range_rows(ctx, B, k, nb, ldb, pp->p, s);
        if (st != GFP_OK) return st;
    }
    std::lock_guard<std::mutex> g(ctx->mu);
    const gfp_status st = ensure_block_ws(ctx, m, k, nb, pp->passes > 1 ? pp->passes : 0, s);
    if (st != GFP_OK) return st;
    int launches = 0;
    const uint8_t *img = (const uint8_t *)pp->mem;
    if (pp->passes == 1) {
        GFP_CUDA_TRY(launch_block_tc(make_mod(pp->p), m, k, nb, nullptr, 0, B, ldb, C, ldc,
                                     ctx->blk_ws, block_sms(ctx), s, &launches, false, img));
    } else {
        uint32_t *R = (uint32_t *)((uint8_t *)ctx->blk_ws + block_tc_workspace_bytes(m, k, nb));
        for (int l = 0; l < pp->passes; ++l)
            GFP_CUDA_TRY(launch_block_tc(make_mod(pp->rc.mod[l]), m, k, nb, nullptr, 0, B, ldb,
                                         R + (size_t)l * m * nb, nb, ctx->blk_ws, block_sms(ctx), s,
                                         &launches, true, img + pp->per * l));
        GFP_CUDA_TRY(launch_block_crt(R, m, nb, C, ldc, pp->rc, ctx->sm_count, s));
        ++launches;
    }
    ctx->launches += launches;
    return GFP_OK;
}

GFP_API gfp_status gfp_matmul_block_csr(gfp_ctx *ctx, uint32_t p, uint64_t m, uint64_t k,
                                        uint64_t nb, const uint32_t *row_ptr, const uint32_t *col,
                                        const uint32_t *val, const uint32_t *B, uint64_t ldb,
                                        uint32_t *C, uint64_t ldc, void *stream)
{
    GFP_TRACE();
    if (!ctx || p < 2 || ldb < nb || ldc < nb) return GFP_ERR_INVALID;
    if (m && (!row_ptr || (nb && !C))) return GFP_ERR_INVALID;
    if ((((uintptr_t)row_ptr) | ((uintptr_t)col) | ((uintptr_t)val) | ((uintptr_t)B) |
         ((uintptr_t)C)) & 3u)
        return GFP_ERR_INVALID;
    if (m == 0 || nb == 0) return GFP_OK;
    cudaStream_t s = as_stream(stream);
    Repr r;
    if (!resolve_repr_untuned(ctx, p, &r)) return GFP_ERR_UNSUPPORTED;
    if (ctx->validate) {
        // structure: row_ptr read back on the host (validation mode synchronises anyway)
        std::vector<uint32_t> rp(m + 1);
        GFP_CUDA_TRY(cudaMemcpyAsync(rp.data(), row_ptr, (m + 1) * 4, cudaMemcpyDeviceToHost, s));
        GFP_CUDA_TRY(cudaStreamSynchronize(s));
        if (rp[0] != 0) return GFP_ERR_INVALID;
        for (uint64_t i = 0; i < m; ++i)
            if (rp[i + 1] < rp[i]) return GFP_ERR_INVALID;
        const uint64_t nnz = rp[m];
        if (nnz && (!col || !val)) return GFP_ERR_INVALID;
        gfp_status st = check_range(ctx, col, nnz, k ? (uint32_t)std::min<uint64_t>(k, 0xFFFFFFFFull) : 0u, s);
        if (st == GFP_ERR_RANGE) return GFP_ERR_INVALID;
        if (st == GFP_OK) st = check_range(ctx, val, nnz, p, s);
        if (st == GFP_OK) st = check_range_rows(ctx, B, k, nb, ldb, p, s);
        if (st != GFP_OK) return st;
    }
    if (k == 0) {   // no column can hold a nonzero: C = 0 (B has no rows to read)
        GFP_CUDA_TRY(cudaMemset2DAsync(C, ldc * 4, 0, nb * 4, m, s));
        return GFP_OK;
    }
    GFP_CUDA_TRY(launch_block_csr(r, make_mod(p), k_for(r, p), m, k, nb, row_ptr, col, val, B, ldb,
                                  C, ldc, ctx->sm_count, s));
    ctx->launches++;
    return GFP_OK;
}

GFP_API gfp_status gfp_context_check(gfp_ctx *ctx)
{
    if (!ctx) return GFP_ERR_INVALID;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return GFP_ERR_CUDA;
    if (cudaDeviceSynchronize() != cudaSuccess) return GFP_ERR_CUDA;
    // device-side checks (GFP_DEVICE_CHECKS builds; always 0 otherwise)
    const uint32_t dbits = csr_check_bits() | dot_check_bits();
    if (!ctx->blk_ws) return dbits ? GFP_ERR_INVALID : GFP_OK;
    uint32_t *flag = block_tc_err_flag(ctx->blk_ws, ctx->blk_m, ctx->blk_k, ctx->blk_nb);
    uint32_t h = 0;
    GFP_CUDA_TRY(cudaMemcpy(&h, flag, 4, cudaMemcpyDeviceToHost));
    if (h) {
        GFP_CUDA_TRY(cudaMemset(ctx->blk_ws, 0, ctx->blk_ws_bytes));
        return GFP_ERR_TIMEOUT;
    }
    return dbits ? GFP_ERR_INVALID : GFP_OK;
}

GFP_API gfp_status gfp_wait_selftest(uint64_t limit_ns, void *stream)
{
    GFP_TRACE();
    if (limit_ns < 1000000ull || limit_ns > 2000000000ull) return GFP_ERR_INVALID;
    uint32_t bits = 0;
    GFP_CUDA_TRY(wait_selftest(limit_ns, as_stream(stream), &bits));
    return (bits & 1u) ? GFP_ERR_TIMEOUT : GFP_OK;
}

GFP_API gfp_status gfp_matvec_sequence(gfp_ctx *ctx, uint32_t p, uint64_t n, const uint32_t *A,
                                       uint64_t lda, const uint32_t *x0, const uint32_t *u,
                                       uint32_t iters, uint32_t *seq, uint32_t *Y, void *stream)
{
    GFP_TRACE();
    if (!ctx || p < 2 || lda < n || !seq || (n && (!A || !x0 || !u))) return GFP_ERR_INVALID;
    if ((((uintptr_t)A) | ((uintptr_t)x0) | ((uintptr_t)u) | ((uintptr_t)seq) | ((uintptr_t)Y)) & 3u)
        return GFP_ERR_INVALID;
    if (iters > 65535) return GFP_ERR_INVALID;
    cudaStream_t s = as_stream(stream);
    if (n == 0) {
        GFP_CUDA_TRY(cudaMemsetAsync(seq, 0, 4ull * (iters + 1), s));
        return GFP_OK;
    }
    Repr r;
    if (!resolve_repr(ctx, GFP_REPR_AUTO, p, n, &r)) return GFP_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> g(ctx->mu);
    // scratch, grown outside any capture: projection slots and ping-pong vectors
    if (iters + 1 > ctx->seq_cap) {
        GFP_CUDA_TRY(cudaStreamSynchronize(s));
        if (ctx->seq_slots) cudaFree(ctx->seq_slots);
        ctx->seq_slots = nullptr;
        ctx->seq_cap = 0;
        const uint32_t cap = std::max<uint32_t>(iters + 1, 256);
        void *mem = nullptr;
        if (cudaMalloc(&mem, (size_t)cap * 12) != cudaSuccess) return GFP_ERR_NOMEM;
        GFP_CUDA_TRY(cudaMemset(mem, 0, (size_t)cap * 12));
        ctx->seq_slots = (unsigned long long *)mem;
        ctx->seq_tickets = (uint32_t *)((char *)mem + (size_t)cap * 8);
        ctx->seq_cap = cap;
    }
    if (!Y && 2 * n > ctx->pingpong_n) {
        GFP_CUDA_TRY(cudaStreamSynchronize(s));
        if (ctx->pingpong) cudaFree(ctx->pingpong);
        ctx->pingpong = nullptr;
        ctx->pingpong_n = 0;
        if (cudaMalloc(&ctx->pingpong, 2 * n * 4) != cudaSuccess) return GFP_ERR_NOMEM;
        ctx->pingpong_n = 2 * n;
    }
    gfp_ctx::SeqKey key{p, n, A, lda, x0, u, seq, Y, iters, (int)r};
    auto it = ctx->seq_graphs.find(key);
    if (it == ctx->seq_graphs.end()) {
        cudaStream_t cs;
        GFP_CUDA_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        const Mod m = make_mod(p);
        const uint64_t k = k_for(r, p);
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess)
            e = launch_dot_single(r, m, k, n, u, x0, ctx->seq_slots, seq,
                                  dot_single_grid(r, n, ctx->sm_count), cs);
        for (uint32_t t = 1; e == cudaSuccess && t <= iters; ++t) {
            const uint32_t *xin = (t == 1) ? x0
                                  : (Y ? Y + (uint64_t)(t - 2) * n : ctx->pingpong + (uint64_t)(t % 2) * n);
            uint32_t *xout = Y ? Y + (uint64_t)(t - 1) * n : ctx->pingpong + (uint64_t)((t + 1) % 2) * n;
            e = launch_matvec(r, m, k, n, n, A, lda, xin, xout, ctx->sm_count, cs, u,
                              ctx->seq_slots + t, ctx->seq_tickets + t, seq + t);
        }
        cudaError_t e2 = cudaStreamEndCapture(cs, &graph);
        if (e == cudaSuccess) e = e2;
        cudaGraphExec_t exec = nullptr;
        if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        cudaStreamDestroy(cs);
        if (e != cudaSuccess) {
            g_last_cuda_error = e;
            return GFP_ERR_CUDA;
        }
        it = ctx->seq_graphs.emplace(key, exec).first;
    }
    GFP_CUDA_TRY(cudaGraphLaunch(it->second, s));
    ctx->launches += iters + 1;
    return GFP_OK;
}

GFP_API gfp_status gfp_fill_uniform(uint32_t p, uint64_t seed, uint64_t stream_id,
                                    uint64_t offset, uint64_t n, uint32_t *out, void *stream)
{
    GFP_TRACE();
    if (p < 2 || (n && !out)) return GFP_ERR_INVALID;
    GFP_CUDA_TRY(launch_fill_uniform(p, seed, stream_id, offset, n, out, as_stream(stream)));
    return GFP_OK;
}

}  // extern "C"
