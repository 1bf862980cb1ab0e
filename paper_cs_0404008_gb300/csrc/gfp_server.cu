// Service layer of libgfpdot: continuous batching of dot, matrix-vector and
// block jobs with mixed moduli.
//
//   submit  -> FIFO queue (bounded; GFP_ERR_AGAIN when full)
//   admit   -> head-of-line job enters when a slot is free and its operand and
//              output bytes fit in the device arena (memory-based admission)
//   launch  -> all dot jobs admitted in one dispatcher pass share ONE
//              persistent batched kernel launch; matrix-vector and block jobs
//              launch individually; launches rotate over a pool of streams
//              (dot and matrix-vector on high-priority streams, block jobs on
//              low-priority ones), so work of different jobs overlaps on the
//              device and short jobs' CTAs are scheduled first
//   complete-> the dispatcher polls a completion event per launch, frees the
//              operands, publishes the result and wakes waiters
// A simulation mode runs the same dispatcher without a GPU: a job "completes"
// after a time proportional to its work, which lets the admission, batching
// and API logic be tested on a host without CUDA devices.
#include <algorithm>
#include <chrono>
#include <cstdlib>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "gfp_internal.h"

namespace {

uint64_t now_ns()
{
    return (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(
               std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

inline uint64_t a256(uint64_t b) { return (b + 255) & ~(uint64_t)255; }

// First-fit allocator over one device range, 256-byte granules, coalescing.
struct Arena {
    uint64_t size = 0, in_use = 0, peak = 0;
    std::map<uint64_t, uint64_t> free_;   // offset -> length

    void init(uint64_t bytes)
    {
        size = bytes;
        free_.clear();
        free_[0] = bytes;
    }
    bool alloc(uint64_t bytes, uint64_t *off)
    {
        bytes = a256(bytes ? bytes : 1);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < bytes) continue;
            *off = it->first;
            const uint64_t rest = it->second - bytes, roff = it->first + bytes;
            free_.erase(it);
            if (rest) free_[roff] = rest;
            in_use += bytes;
            if (in_use > peak) peak = in_use;
            return true;
        }
        return false;
    }
    void release(uint64_t off, uint64_t bytes)
    {
        bytes = a256(bytes ? bytes : 1);
        in_use -= bytes;
        auto it = free_.emplace(off, bytes).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
};

struct Matrix {
    uint32_t p;
    uint64_t rows, cols;
    const uint32_t *dev;
    void *owned;
    uint64_t ld;   // leading dimension (server-generated matrices pad rows to 16 bytes)
    gfp_block_prep *prep = nullptr;   // digit images for block jobs (gfp_prepare_matrix)
};

enum class State { Queued, Running, Done };

struct Launch;

struct JobRec {
    gfp_job job;
    State state = State::Queued;
    gfp_result res{};
    uint64_t op_off = 0, op_bytes = 0;     // operands generated by the server
    uint64_t out_off = 0, out_bytes = 0;   // MATVEC / BLOCK outputs
    bool has_op = false, has_out = false;
    bool release_when_done = false;
    uint32_t dot_index = 0;                // position in its launch's result array
};

struct Launch {
    std::vector<uint64_t> tickets;
    int stream = 0;
    cudaEvent_t ev = nullptr;
    uint64_t res_off = 0, res_bytes = 0;   // DOT: device results
    int pinned = -1;                       // DOT: pinned host block index
    uint64_t sim_done = 0;
    int32_t status = GFP_OK;
};

constexpr uint32_t kPinnedBlocks = 64, kPinnedElems = 4096;   // dots per launch <= 4096
constexpr uint64_t kDotResBytes = 4ull * kPinnedElems;          // device results of one launch

}  // namespace

struct gfp_server {
    gfp_server_cfg cfg{};
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::thread disp;
    bool stop = false;

    std::deque<uint64_t> queue;
    std::unordered_map<uint64_t, JobRec> jobs;
    std::vector<Launch> running;
    std::map<uint64_t, Matrix> mats;
    uint64_t next_ticket = 1, next_mat = 1;
    uint64_t admit_attempts = 0;

    Arena arena;
    uint8_t *base = nullptr;   // device arena (nullptr in simulation)
    std::vector<cudaStream_t> streams;
    std::vector<gfp_ctx *> ctxs;
    uint32_t *pinned = nullptr;
    std::vector<int> pinned_free;
    int rr = 0, rr_blk = 0;   // next stream of each class
    int n_fast = 0;           // streams [0, n_fast) carry dot and matrix-vector launches
    gfp_server_stats st{};

    uint64_t footprint(const gfp_job &j, uint64_t *op, uint64_t *out) const;
    void dispatcher();
    void poll_completions();
    void finish(Launch &L, int32_t status);
    bool admit_and_launch();
    int32_t launch_dots(std::vector<uint64_t> &dots, Launch &L);
    int32_t launch_one(uint64_t t, Launch &L);
    double sim_seconds(const gfp_job &j) const;
};

uint64_t gfp_server::footprint(const gfp_job &j, uint64_t *op, uint64_t *out) const
{
    *op = 0;
    *out = 0;
    if (j.kind == GFP_JOB_DOT) {
        if (!j.x) *op += a256(4 * j.n);
        if (!j.y) *op += a256(4 * j.n);
    } else {
        const Matrix &M = mats.at(j.matrix);
        if (j.kind == GFP_JOB_MATVEC) {
            if (!j.v) *op += a256(4 * M.cols);
            *out = a256(4 * M.rows);
        } else {
            if (!j.v) *op += a256(4 * M.cols * j.nb);
            *out = a256(4 * M.rows * j.nb);
        }
    }
    return *op + *out;
}

double gfp_server::sim_seconds(const gfp_job &j) const
{
    // bandwidth-bound estimate: operand bytes at 6 TB/s, plus a 5 us launch cost
    double bytes = 0;
    if (j.kind == GFP_JOB_DOT) {
        bytes = 8.0 * j.n;
    } else {
        const Matrix &M = mats.at(j.matrix);
        bytes = 4.0 * M.rows * M.cols + (j.kind == GFP_JOB_BLOCK ? 4.0 * M.cols * j.nb : 4.0 * M.cols);
    }
    return 5e-6 + bytes / 6e12;
}

void gfp_server::finish(Launch &L, int32_t status)
{
    const uint64_t t = now_ns();
    for (uint64_t tk : L.tickets) {
        auto it = jobs.find(tk);
        if (it == jobs.end()) continue;
        JobRec &r = it->second;
        if (r.has_op) {
            arena.release(r.op_off, r.op_bytes);
            r.has_op = false;
        }
        r.res.status = status;
        r.res.t_done_ns = t;
        if (status == GFP_OK && r.job.kind == GFP_JOB_DOT)
            r.res.value = (cfg.simulate || L.pinned < 0)
                              ? 0u
                              : pinned[(size_t)L.pinned * kPinnedElems + r.dot_index];
        if (status != GFP_OK && r.has_out) {
            arena.release(r.out_off, r.out_bytes);
            r.has_out = false;
            r.res.out_elems = 0;
        }
        r.state = State::Done;
        if (status == GFP_OK) st.completed++;
        else st.failed++;
        if (r.release_when_done) {
            if (r.has_out) arena.release(r.out_off, r.out_bytes);
            jobs.erase(it);
        }
    }
    if (L.res_bytes) arena.release(L.res_off, L.res_bytes);
    if (L.pinned >= 0) pinned_free.push_back(L.pinned);
    if (L.ev) cudaEventDestroy(L.ev);
    L.ev = nullptr;
}

void gfp_server::poll_completions()
{
    const uint64_t t = now_ns();
    bool any = false;
    for (size_t i = 0; i < running.size();) {
        Launch &L = running[i];
        int32_t status = GFP_PENDING;
        if (L.status != GFP_OK) {
            status = L.status;
        } else if (cfg.simulate) {
            if (t >= L.sim_done) status = GFP_OK;
        } else {
            const cudaError_t e = cudaEventQuery(L.ev);
            if (e == cudaSuccess) status = GFP_OK;
            else if (e != cudaErrorNotReady) status = GFP_ERR_CUDA;
        }
        if (status == GFP_PENDING) {
            ++i;
            continue;
        }
        finish(L, status);
        running[i] = std::move(running.back());
        running.pop_back();
        any = true;
    }
    if (any) cv_done.notify_all();
}

int32_t gfp_server::launch_dots(std::vector<uint64_t> &dots, Launch &L)
{
    cudaStream_t s = streams[L.stream];
    gfp_ctx *ctx = ctxs[L.stream];
    std::vector<gfp_dot_desc> d(dots.size());
    for (size_t i = 0; i < dots.size(); ++i) {
        JobRec &r = jobs.at(dots[i]);
        const gfp_job &j = r.job;
        const uint32_t *x = j.x, *y = j.y;
        uint64_t off = r.op_off;
        if (!x) {
            uint32_t *gx = (uint32_t *)(base + off);
            if (gfp_fill_uniform(j.p, j.seed, 0, 0, j.n, gx, s) != GFP_OK) return GFP_ERR_CUDA;
            st.kernel_launches++;
            x = gx;
            off += a256(4 * j.n);
        }
        if (!y) {
            uint32_t *gy = (uint32_t *)(base + off);
            if (gfp_fill_uniform(j.p, j.seed, 1, 0, j.n, gy, s) != GFP_OK) return GFP_ERR_CUDA;
            st.kernel_launches++;
            y = gy;
        }
        d[i] = gfp_dot_desc{j.p, GFP_REPR_AUTO, j.n, x, y};
        r.dot_index = (uint32_t)i;
    }
    uint32_t *dres = (uint32_t *)(base + L.res_off);
    const gfp_status stt = gfp_dot_batched(ctx, d.data(), d.size(), dres, s);
    if (stt != GFP_OK) return stt;
    st.kernel_launches++;
    if (cudaMemcpyAsync(pinned + (size_t)L.pinned * kPinnedElems, dres, 4 * d.size(),
                        cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return GFP_ERR_CUDA;
    return GFP_OK;
}

int32_t gfp_server::launch_one(uint64_t t, Launch &L)
{
    cudaStream_t s = streams[L.stream];
    gfp_ctx *ctx = ctxs[L.stream];
    JobRec &r = jobs.at(t);
    const gfp_job &j = r.job;
    const Matrix &M = mats.at(j.matrix);
    const uint32_t *v = j.v;
    if (!v) {
        uint32_t *gv = (uint32_t *)(base + r.op_off);
        const uint64_t n = (j.kind == GFP_JOB_MATVEC) ? M.cols : M.cols * j.nb;
        if (gfp_fill_uniform(j.p, j.seed, 0, 0, n, gv, s) != GFP_OK) return GFP_ERR_CUDA;
        st.kernel_launches++;
        v = gv;
    }
    uint32_t *outp = (uint32_t *)(base + r.out_off);
    const uint64_t before = gfp_launch_count(ctx);
    gfp_status stt;
    if (j.kind == GFP_JOB_MATVEC)
        stt = gfp_matvec(ctx, j.p, M.rows, M.cols, M.dev, M.ld, v, outp, s);
    else if (M.prep)
        stt = gfp_matmul_block_prepared(ctx, M.prep, j.nb, v, j.nb, outp, j.nb, s);
    else
        stt = gfp_matmul_block(ctx, j.p, M.rows, M.cols, j.nb, M.dev, M.ld, v, j.nb, outp, j.nb, s);
    st.kernel_launches += gfp_launch_count(ctx) - before;
    return stt;
}

// One dispatcher pass: admit head-of-line jobs while they fit, launch them.
// Returns true if anything was admitted.
bool gfp_server::admit_and_launch()
{
    const uint64_t t = now_ns();
    std::vector<uint64_t> dots, others;
    uint64_t dres_off = 0;            // results of this pass's dot launch
    bool have_dres = false;
    while (!queue.empty()) {
        const uint64_t tk = queue.front();
        auto it = jobs.find(tk);
        if (it == jobs.end() || it->second.state != State::Queued) {
            queue.pop_front();
            continue;
        }
        JobRec &r = it->second;
        const size_t slots = running.size() + (dots.empty() ? 0 : 1) + others.size();
        if (slots >= cfg.max_inflight) {
            st.admission_stalls++;
            break;
        }
        if (r.job.kind == GFP_JOB_DOT && cfg.batch_window_us && dots.empty() &&
            t - r.res.t_submit_ns < (uint64_t)cfg.batch_window_us * 1000ull && queue.size() < 64)
            break;   // let more dot jobs arrive for this launch
        if (r.job.kind == GFP_JOB_DOT && dots.size() >= kPinnedElems) break;
        if (r.job.kind == GFP_JOB_DOT && !have_dres && !cfg.simulate) {
            // a dot launch needs a pinned result block and a device result array
            if (pinned_free.empty() || !arena.alloc(kDotResBytes, &dres_off)) {
                st.admission_stalls++;
                break;
            }
            have_dres = true;
        }
        uint64_t op, out;
        footprint(r.job, &op, &out);
        ++admit_attempts;
        bool ok = !(cfg.fail_every && admit_attempts % cfg.fail_every == 0);
        uint64_t op_off = 0, out_off = 0;
        if (ok && op && !arena.alloc(op, &op_off)) ok = false;
        if (ok && out && !arena.alloc(out, &out_off)) {
            if (op) arena.release(op_off, op);
            ok = false;
        }
        if (!ok) {
            if (cfg.fail_every && admit_attempts % cfg.fail_every == 0) {
                // injected allocation failure: the job fails, the queue moves on
                queue.pop_front();
                r.state = State::Done;
                r.res.status = GFP_ERR_NOMEM;
                r.res.t_done_ns = t;
                st.failed++;
                cv_done.notify_all();
                continue;
            }
            st.admission_stalls++;
            break;   // wait for memory to free
        }
        queue.pop_front();
        r.op_off = op_off;
        r.op_bytes = op;
        r.has_op = op != 0;
        r.out_off = out_off;
        r.out_bytes = out;
        r.has_out = out != 0;
        r.state = State::Running;
        r.res.t_admit_ns = t;
        st.admitted++;
        (r.job.kind == GFP_JOB_DOT ? dots : others).push_back(tk);
    }
    if (have_dres && dots.empty()) {
        arena.release(dres_off, kDotResBytes);
        have_dres = false;
    }
    if (dots.empty() && others.empty()) return false;

    // dot and matrix-vector launches rotate over the high-priority streams,
    // block launches over the low-priority ones (all of them when there is one)
    auto start = [&](Launch &L, bool block) {
        const int nf = n_fast, ns = (int)streams.size();
        if (block && ns > nf) {
            L.stream = nf + rr_blk;
            rr_blk = (rr_blk + 1) % (ns - nf);
        } else {
            L.stream = rr;
            rr = (rr + 1) % nf;
        }
        if (!cfg.simulate && cudaEventCreateWithFlags(&L.ev, cudaEventDisableTiming) != cudaSuccess)
            L.status = GFP_ERR_CUDA;
    };
    const uint64_t t_start = now_ns();
    if (!dots.empty()) {
        Launch L;
        L.tickets = dots;
        start(L, false);
        double sim = 0;
        for (uint64_t tk : dots) {
            JobRec &r = jobs.at(tk);
            r.res.t_start_ns = t_start;
            r.res.batch = (uint32_t)dots.size();
            sim += sim_seconds(r.job) - 5e-6;
        }
        st.dot_launches++;
        if (cfg.simulate) {
            L.sim_done = t_start + (uint64_t)((sim + 5e-6) * 1e9);
        } else {
            L.res_off = dres_off;
            L.res_bytes = kDotResBytes;
        }
        if (!cfg.simulate && L.status == GFP_OK) {
            if (pinned_free.empty()) {
                L.status = GFP_ERR_NOMEM;
            } else {
                L.pinned = pinned_free.back();
                pinned_free.pop_back();
                L.status = launch_dots(dots, L);
                if (L.status == GFP_OK &&
                    cudaEventRecord(L.ev, streams[L.stream]) != cudaSuccess)
                    L.status = GFP_ERR_CUDA;
            }
            const uint64_t t_q = now_ns();   // every launch of the batch is enqueued
            for (uint64_t tk : dots) jobs.at(tk).res.t_start_ns = t_q;
        }
        running.push_back(std::move(L));
    }
    for (uint64_t tk : others) {
        Launch L;
        L.tickets = {tk};
        start(L, jobs.at(tk).job.kind == GFP_JOB_BLOCK);
        JobRec &r = jobs.at(tk);
        r.res.t_start_ns = t_start;
        r.res.batch = 1;
        if (cfg.simulate) {
            L.sim_done = t_start + (uint64_t)(sim_seconds(r.job) * 1e9);
        } else if (L.status == GFP_OK) {
            L.status = launch_one(tk, L);
            if (L.status == GFP_OK && cudaEventRecord(L.ev, streams[L.stream]) != cudaSuccess)
                L.status = GFP_ERR_CUDA;
            r.res.t_start_ns = now_ns();   // the job's launches are enqueued
        }
        running.push_back(std::move(L));
    }
    return true;
}

void gfp_server::dispatcher()
{
    if (!cfg.simulate) cudaSetDevice(cfg.device);
    std::unique_lock<std::mutex> lk(mu);
    while (!stop) {
        poll_completions();
        const bool launched = admit_and_launch();
        if (launched) continue;
        // idle: wake on a submission, or poll completions again shortly
        cv_work.wait_for(lk, std::chrono::microseconds(running.empty() ? 2000 : 20));
    }
}

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------

extern "C" {

GFP_API gfp_status gfp_server_create(const gfp_server_cfg *cfg, gfp_server **out)
{
    GFP_TRACE();
    if (!cfg || !out) return GFP_ERR_INVALID;
    *out = nullptr;
    gfp_server *s = new (std::nothrow) gfp_server();
    if (!s) return GFP_ERR_NOMEM;
    s->cfg = *cfg;
    if (!s->cfg.mem_budget) {
        const char *e = getenv("GFP_MEM_BUDGET");   // bytes; the default is 4 GiB
        const unsigned long long b = e ? strtoull(e, nullptr, 10) : 0ull;
        s->cfg.mem_budget = b ? (uint64_t)b : 4ull << 30;
    }
    if (!s->cfg.max_inflight) s->cfg.max_inflight = 256;
    if (!s->cfg.n_streams) s->cfg.n_streams = 4;
    if (!s->cfg.queue_capacity) s->cfg.queue_capacity = 65536;
    s->arena.init(s->cfg.mem_budget);
    s->st.mem_budget = s->cfg.mem_budget;
    if (!s->cfg.simulate) {
        gfp_status stt = GFP_OK;
        if (cudaSetDevice(s->cfg.device) != cudaSuccess) stt = GFP_ERR_CUDA;
        if (stt == GFP_OK && cudaMalloc(&s->base, s->cfg.mem_budget) != cudaSuccess) {
            s->base = nullptr;
            stt = GFP_ERR_NOMEM;
        }
        if (stt == GFP_OK && cudaHostAlloc((void **)&s->pinned, (size_t)kPinnedBlocks * kPinnedElems * 4,
                                           cudaHostAllocDefault) != cudaSuccess) {
            s->pinned = nullptr;
            stt = GFP_ERR_NOMEM;
        }
        // with two or more streams, the first half get the highest priority
        // (dot and matrix-vector jobs) and the rest the lowest (block jobs):
        // CTAs of short jobs are scheduled ahead of a block kernel's
        int lo_prio = 0, hi_prio = 0;
        if (cudaDeviceGetStreamPriorityRange(&lo_prio, &hi_prio) != cudaSuccess) lo_prio = hi_prio = 0;
        s->n_fast = s->cfg.n_streams >= 2 ? (int)(s->cfg.n_streams + 1) / 2 : 1;
        for (uint32_t i = 0; stt == GFP_OK && i < s->cfg.n_streams; ++i) {
            cudaStream_t cs;
            const int prio = (int)i < s->n_fast ? hi_prio : lo_prio;
            if (cudaStreamCreateWithPriority(&cs, cudaStreamNonBlocking, prio) != cudaSuccess) {
                stt = GFP_ERR_CUDA;
                break;
            }
            s->streams.push_back(cs);
            gfp_ctx *c = nullptr;
            stt = gfp_context_create(s->cfg.device, &c);
            if (stt == GFP_OK) {
                if (s->cfg.block_sm_percent > 0 && s->cfg.block_sm_percent < 100)
                    c->blk_sms = std::max(1, (int)((uint64_t)c->sm_count * s->cfg.block_sm_percent / 100));
                s->ctxs.push_back(c);
            }
        }
        if (stt != GFP_OK) {
            for (auto c : s->ctxs) gfp_context_destroy(c);
            for (auto cs : s->streams) cudaStreamDestroy(cs);
            if (s->pinned) cudaFreeHost(s->pinned);
            if (s->base) cudaFree(s->base);
            delete s;
            return stt;
        }
    } else {
        s->streams.resize(s->cfg.n_streams, nullptr);
        s->n_fast = s->cfg.n_streams >= 2 ? (int)(s->cfg.n_streams + 1) / 2 : 1;
    }
    for (int i = (int)kPinnedBlocks - 1; i >= 0; --i) s->pinned_free.push_back(i);
    s->disp = std::thread([s] { s->dispatcher(); });
    *out = s;
    return GFP_OK;
}

GFP_API gfp_status gfp_server_destroy(gfp_server *s)
{
    GFP_TRACE();
    if (!s) return GFP_ERR_INVALID;
    {
        std::lock_guard<std::mutex> g(s->mu);
        s->stop = true;
        for (uint64_t tk : s->queue) {
            auto it = s->jobs.find(tk);
            if (it != s->jobs.end() && it->second.state == State::Queued) {
                it->second.state = State::Done;
                it->second.res.status = GFP_ERR_CANCELLED;
                s->st.cancelled++;
            }
        }
        s->queue.clear();
    }
    s->cv_work.notify_all();
    s->disp.join();
    // jobs still on the device: wait for them (bounded), then release everything
    const uint64_t t0 = now_ns();
    for (;;) {
        {
            std::lock_guard<std::mutex> g(s->mu);
            s->poll_completions();
            if (s->running.empty() || now_ns() - t0 > 10000000000ull) break;
        }
        std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
    s->cv_done.notify_all();
    if (!s->cfg.simulate) {
        for (auto c : s->ctxs) gfp_context_destroy(c);
        for (auto cs : s->streams) cudaStreamDestroy(cs);
        for (auto &kv : s->mats) {
            if (kv.second.prep) gfp_block_prep_destroy(kv.second.prep);
            if (kv.second.owned) cudaFree(kv.second.owned);
        }
        if (s->pinned) cudaFreeHost(s->pinned);
        if (s->base) cudaFree(s->base);
    }
    delete s;
    return GFP_OK;
}

GFP_API gfp_status gfp_register_matrix(gfp_server *s, uint32_t p, uint64_t rows, uint64_t cols,
                                       const uint32_t *dev, uint64_t seed, uint64_t *handle)
{
    GFP_TRACE();
    if (!s || !handle || p < 2 || rows == 0 || cols == 0) return GFP_ERR_INVALID;
    if (dev && (((uintptr_t)dev) & 3u)) return GFP_ERR_INVALID;
    Matrix M{p, rows, cols, dev, nullptr, cols};
    if (!dev && !s->cfg.simulate) {
        // rows start on 16-byte boundaries so that the tensor-core block
        // product (which copies A by TMA) can take the matrix
        M.ld = (cols + 3) / 4 * 4;
        void *mem = nullptr;
        if (cudaSetDevice(s->cfg.device) != cudaSuccess) return GFP_ERR_CUDA;
        if (cudaMalloc(&mem, 4 * rows * M.ld) != cudaSuccess) return GFP_ERR_NOMEM;
        if (gfp::launch_fill_uniform_2d(p, seed, 0, rows, cols, M.ld, (uint32_t *)mem, nullptr) != cudaSuccess ||
            cudaDeviceSynchronize() != cudaSuccess) {
            cudaFree(mem);
            return GFP_ERR_CUDA;
        }
        M.dev = (const uint32_t *)mem;
        M.owned = mem;
    }
    std::lock_guard<std::mutex> g(s->mu);
    *handle = s->next_mat++;
    s->mats[*handle] = M;
    return GFP_OK;
}

GFP_API gfp_status gfp_prepare_matrix(gfp_server *s, uint64_t handle)
{
    GFP_TRACE();
    if (!s) return GFP_ERR_INVALID;
    Matrix M;
    {
        std::lock_guard<std::mutex> g(s->mu);
        auto it = s->mats.find(handle);
        if (it == s->mats.end()) return GFP_ERR_INVALID;
        if (it->second.prep || s->cfg.simulate) return GFP_OK;
        M = it->second;
    }
    if (cudaSetDevice(s->cfg.device) != cudaSuccess) return GFP_ERR_CUDA;
    gfp_block_prep *pp = nullptr;
    const gfp_status st = gfp_block_prepare(s->ctxs[0], M.p, M.rows, M.cols, M.dev, M.ld, &pp);
    if (st != GFP_OK) return st;
    std::lock_guard<std::mutex> g(s->mu);
    auto it = s->mats.find(handle);
    if (it == s->mats.end() || it->second.prep) {
        gfp_block_prep_destroy(pp);
        return it == s->mats.end() ? GFP_ERR_INVALID : GFP_OK;
    }
    it->second.prep = pp;
    return GFP_OK;
}

GFP_API gfp_status gfp_submit(gfp_server *s, const gfp_job *job, uint64_t *ticket)
{
    GFP_TRACE();
    if (!s || !job || !ticket) return GFP_ERR_INVALID;
    const gfp_job &j = *job;
    if (j.kind > GFP_JOB_BLOCK || j.p < 2) return GFP_ERR_INVALID;
    std::lock_guard<std::mutex> g(s->mu);
    if (j.kind == GFP_JOB_DOT) {
        if (j.n && ((j.x && (((uintptr_t)j.x) & 3u)) || (j.y && (((uintptr_t)j.y) & 3u))))
            return GFP_ERR_INVALID;
    } else {
        auto it = s->mats.find(j.matrix);
        if (it == s->mats.end() || it->second.p != j.p) return GFP_ERR_INVALID;
        if (j.kind == GFP_JOB_BLOCK && j.nb == 0) return GFP_ERR_INVALID;
        if (j.v && (((uintptr_t)j.v) & 3u)) return GFP_ERR_INVALID;
    }
    uint64_t op, out;
    if (s->footprint(j, &op, &out) + (j.kind == GFP_JOB_DOT ? kDotResBytes : 0) > s->cfg.mem_budget)
        return GFP_ERR_NOMEM;
    if (s->queue.size() >= s->cfg.queue_capacity) return GFP_ERR_AGAIN;
    if (s->stop) return GFP_ERR_CANCELLED;
    const uint64_t tk = s->next_ticket++;
    JobRec r;
    r.job = j;
    r.res.kind = j.kind;
    r.res.status = GFP_PENDING;
    r.res.t_submit_ns = now_ns();
    if (j.kind != GFP_JOB_DOT) {
        const Matrix &M = s->mats.at(j.matrix);
        r.res.out_elems = (j.kind == GFP_JOB_MATVEC) ? M.rows : M.rows * j.nb;
    }
    s->jobs.emplace(tk, r);
    s->queue.push_back(tk);
    s->st.submitted++;
    *ticket = tk;
    s->cv_work.notify_one();
    return GFP_OK;
}

GFP_API gfp_status gfp_poll(gfp_server *s, uint64_t ticket, gfp_result *res)
{
    if (!s) return GFP_ERR_INVALID;
    std::lock_guard<std::mutex> g(s->mu);
    auto it = s->jobs.find(ticket);
    if (it == s->jobs.end()) return GFP_ERR_UNKNOWN_TICKET;
    if (it->second.state != State::Done) return GFP_PENDING;
    if (res) *res = it->second.res;
    return GFP_OK;
}

GFP_API gfp_status gfp_wait(gfp_server *s, uint64_t ticket, uint64_t timeout_us, gfp_result *res)
{
    GFP_TRACE();
    if (!s) return GFP_ERR_INVALID;
    std::unique_lock<std::mutex> lk(s->mu);
    const auto deadline = std::chrono::steady_clock::now() + std::chrono::microseconds(timeout_us);
    for (;;) {
        auto it = s->jobs.find(ticket);
        if (it == s->jobs.end()) return GFP_ERR_UNKNOWN_TICKET;
        if (it->second.state == State::Done) {
            if (res) *res = it->second.res;
            return GFP_OK;
        }
        if (s->cv_done.wait_until(lk, deadline) == std::cv_status::timeout) {
            it = s->jobs.find(ticket);
            if (it != s->jobs.end() && it->second.state == State::Done) {
                if (res) *res = it->second.res;
                return GFP_OK;
            }
            return it == s->jobs.end() ? GFP_ERR_UNKNOWN_TICKET : GFP_ERR_TIMEOUT;
        }
    }
}

GFP_API gfp_status gfp_result_copy(gfp_server *s, uint64_t ticket, uint32_t *host, uint64_t count)
{
    GFP_TRACE();
    if (!s || (count && !host)) return GFP_ERR_INVALID;
    uint64_t off;
    {
        std::lock_guard<std::mutex> g(s->mu);
        auto it = s->jobs.find(ticket);
        if (it == s->jobs.end()) return GFP_ERR_UNKNOWN_TICKET;
        const JobRec &r = it->second;
        if (r.state != State::Done) return GFP_PENDING;
        if (r.res.status != GFP_OK || !r.has_out || count > r.res.out_elems) return GFP_ERR_INVALID;
        off = r.out_off;
    }
    if (s->cfg.simulate || count == 0) return GFP_OK;
    // the output region stays allocated until gfp_release, which the caller
    // does not call concurrently with this copy
    if (cudaMemcpy(host, s->base + off, 4 * count, cudaMemcpyDeviceToHost) != cudaSuccess)
        return GFP_ERR_CUDA;
    return GFP_OK;
}

GFP_API gfp_status gfp_release(gfp_server *s, uint64_t ticket)
{
    GFP_TRACE();
    if (!s) return GFP_ERR_INVALID;
    std::lock_guard<std::mutex> g(s->mu);
    auto it = s->jobs.find(ticket);
    if (it == s->jobs.end()) return GFP_ERR_UNKNOWN_TICKET;
    JobRec &r = it->second;
    if (r.state == State::Queued) {
        r.state = State::Done;
        r.res.status = GFP_ERR_CANCELLED;
        s->st.cancelled++;
        s->jobs.erase(it);   // the queue skips tickets it no longer finds
        return GFP_OK;
    }
    if (r.state == State::Running) {
        r.release_when_done = true;
        return GFP_OK;
    }
    if (r.has_out) s->arena.release(r.out_off, r.out_bytes);
    s->jobs.erase(it);
    return GFP_OK;
}

GFP_API gfp_status gfp_server_get_stats(gfp_server *s, gfp_server_stats *out)
{
    if (!s || !out) return GFP_ERR_INVALID;
    std::lock_guard<std::mutex> g(s->mu);
    *out = s->st;
    out->mem_in_use = s->arena.in_use;
    out->mem_peak = s->arena.peak;
    return GFP_OK;
}

}  // extern "C"
