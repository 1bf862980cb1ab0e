// Install-time selection of the dot-product representation and work-unit
// length per (p, n), following the automated empirical optimisation proposed
// in the paper's conclusion: every eligible candidate is timed on the device
// and the fastest one is recorded in a plan table, which later calls consult.
//
// Plan file format (JSON):
//   {"version": 1, "entries": [{"p": 65521, "lg_n": 20, "repr": 2, "chunk": 65536}, ...]}
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "gfp_internal.h"

using namespace gfp;

namespace {

// Minimal reader for the plan format above: scans objects for the four keys.
bool parse_plan(const std::string &txt, std::vector<gfp_plan_entry> &out)
{
    size_t pos = txt.find("\"entries\"");
    if (pos == std::string::npos) return false;
    for (;;) {
        const size_t ob = txt.find('{', pos);
        if (ob == std::string::npos) break;
        const size_t cb = txt.find('}', ob);
        if (cb == std::string::npos) return false;
        const std::string obj = txt.substr(ob, cb - ob + 1);
        auto num = [&](const char *key, unsigned long long &v) {
            const std::string k = std::string("\"") + key + "\"";
            size_t q = obj.find(k);
            if (q == std::string::npos) return false;
            q = obj.find(':', q);
            if (q == std::string::npos) return false;
            v = strtoull(obj.c_str() + q + 1, nullptr, 10);
            return true;
        };
        unsigned long long p, lg, r, c;
        if (!num("p", p) || !num("lg_n", lg) || !num("repr", r) || !num("chunk", c)) return false;
        if (p < 2 || p > 0xFFFFFFFFull || lg > 63 || r >= GFP_REPR_COUNT_ || c > 0xFFFFFFFFull)
            return false;
        out.push_back(gfp_plan_entry{(uint32_t)p, (uint32_t)lg, (uint32_t)r, (uint32_t)c});
        pos = cb + 1;
    }
    return true;
}

struct DevBuf {
    void *p = nullptr;
    ~DevBuf() { if (p) cudaFree(p); }
};

}  // namespace

extern "C" {

GFP_API gfp_status gfp_plan_load(gfp_ctx *ctx, const char *path)
{
    GFP_TRACE();
    if (!ctx || !path) return GFP_ERR_INVALID;
    FILE *f = fopen(path, "rb");
    if (!f) return GFP_ERR_INVALID;
    std::string txt;
    char buf[4096];
    size_t got;
    while ((got = fread(buf, 1, sizeof buf, f)) > 0) txt.append(buf, got);
    fclose(f);
    std::vector<gfp_plan_entry> es;
    if (!parse_plan(txt, es)) return GFP_ERR_INVALID;
    std::lock_guard<std::mutex> g(ctx->mu);
    ctx->plan.clear();
    for (auto &e : es) ctx->plan[{e.p, e.lg_n}] = e;
    return GFP_OK;
}

GFP_API gfp_status gfp_plan_save(const gfp_ctx *ctx, const char *path)
{
    GFP_TRACE();
    if (!ctx || !path) return GFP_ERR_INVALID;
    FILE *f = fopen(path, "wb");
    if (!f) return GFP_ERR_INVALID;
    fprintf(f, "{\"version\": 1, \"entries\": [");
    bool first = true;
    for (auto &kv : ctx->plan) {
        const gfp_plan_entry &e = kv.second;
        fprintf(f, "%s\n  {\"p\": %u, \"lg_n\": %u, \"repr\": %u, \"chunk\": %u}", first ? "" : ",",
                e.p, e.lg_n, e.repr, e.chunk);
        first = false;
    }
    fprintf(f, "\n]}\n");
    fclose(f);
    return GFP_OK;
}

GFP_API uint64_t gfp_plan_size(const gfp_ctx *ctx) { return ctx ? ctx->plan.size() : 0; }

GFP_API gfp_status gfp_tune(gfp_ctx *ctx, const uint32_t *primes, uint32_t nprimes,
                            uint32_t lg_lo, uint32_t lg_hi, const char *plan_path)
{
    GFP_TRACE();
    static const uint32_t kDefault[] = {32749u, 65521u, 67108859u, 2147483647u, 4294967291u};
    if (!ctx || lg_lo > lg_hi || lg_hi > 26) return GFP_ERR_INVALID;
    if (!primes || nprimes == 0) {
        primes = kDefault;
        nprimes = 5;
    }
    for (uint32_t i = 0; i < nprimes; ++i)
        if (primes[i] < 2) return GFP_ERR_INVALID;
    // operand pool: 2 x 2^28 bytes (larger than L2, so each timing run is cold)
    const uint64_t pool_elems = 1ull << 26;
    DevBuf xb, yb, ob;
    if (cudaMalloc(&xb.p, pool_elems * 4) != cudaSuccess) return GFP_ERR_NOMEM;
    if (cudaMalloc(&yb.p, pool_elems * 4) != cudaSuccess) return GFP_ERR_NOMEM;
    if (cudaMalloc(&ob.p, 1 << 20) != cudaSuccess) return GFP_ERR_NOMEM;
    cudaStream_t s;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return GFP_ERR_CUDA;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const gfp_repr saved_forced = ctx->forced;
    ctx->forced = GFP_REPR_AUTO;
    std::map<std::pair<uint32_t, uint32_t>, gfp_plan_entry> table;
    gfp_status result = GFP_OK;
    static const uint32_t chunks[] = {16384u, 65536u, 262144u};
    static const uint32_t reprs[] = {GFP_REPR_U64_BLOCK, GFP_REPR_U64_CARRY, GFP_REPR_FP64,
                                     GFP_REPR_CENTERED, GFP_REPR_MONTGOMERY};
    for (uint32_t pi = 0; pi < nprimes && result == GFP_OK; ++pi) {
        const uint32_t p = primes[pi];
        gfp_fill_uniform(p, 0x7157ull, 0, 0, pool_elems, (uint32_t *)xb.p, s);
        gfp_fill_uniform(p, 0x7157ull, 1, 0, pool_elems, (uint32_t *)yb.p, s);
        for (uint32_t lg = lg_lo; lg <= lg_hi && result == GFP_OK; lg += 2) {
            const uint64_t n = 1ull << lg;
            uint64_t count = pool_elems / n;
            if (count > 262144) count = 262144;
            std::vector<gfp_dot_desc> d(count);
            for (uint64_t j = 0; j < count; ++j)
                d[j] = gfp_dot_desc{p, 0, n, (uint32_t *)xb.p + j * n, (uint32_t *)yb.p + j * n};
            float best = 1e30f;
            gfp_plan_entry be{p, lg, (uint32_t)GFP_REPR_U64_CARRY, 65536u};
            for (uint32_t r : reprs) {
                if (!repr_eligible((Repr)r, p)) continue;
                for (uint32_t c : chunks) {
                    if (c > 4 * n && c != chunks[0]) continue;   // chunk irrelevant below n
                    for (auto &q : d) q.repr = r;
                    // temporary single-entry plan steering the chunk length
                    ctx->plan[{p, lg}] = gfp_plan_entry{p, lg, r, c};
                    gfp_batch_plan *pl = nullptr;
                    if (gfp_batch_plan_create(ctx, d.data(), count, &pl) != GFP_OK) {
                        result = GFP_ERR_CUDA;
                        break;
                    }
                    float ms = 1e30f;
                    for (int it = 0; it < 6; ++it) {
                        cudaEventRecord(e0, s);
                        gfp_batch_plan_exec(pl, (uint32_t *)ob.p, s);
                        cudaEventRecord(e1, s);
                        if (cudaEventSynchronize(e1) != cudaSuccess) {
                            result = GFP_ERR_CUDA;
                            break;
                        }
                        float t = 0;
                        cudaEventElapsedTime(&t, e0, e1);
                        if (it >= 1 && t < ms) ms = t;   // first run warms up
                    }
                    gfp_batch_plan_destroy(pl);
                    if (result != GFP_OK) break;
                    if (ms < best) {
                        best = ms;
                        be = gfp_plan_entry{p, lg, r, c};
                    }
                }
                if (result != GFP_OK) break;
            }
            ctx->plan.erase({p, lg});
            table[{p, lg}] = be;
        }
    }
    ctx->forced = saved_forced;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamSynchronize(s);
    cudaStreamDestroy(s);
    if (result != GFP_OK) return result;
    {
        std::lock_guard<std::mutex> g(ctx->mu);
        for (auto &kv : table) ctx->plan[kv.first] = kv.second;
    }
    if (plan_path) return gfp_plan_save(ctx, plan_path);
    return GFP_OK;
}

}  // extern "C"
