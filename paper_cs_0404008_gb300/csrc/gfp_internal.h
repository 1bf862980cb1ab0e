// Internal declarations shared by the translation units of libgfpdot.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <atomic>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "gfp_arith.cuh"
#include "../../include/gfpdot.h"

namespace gfp {

// NVTX range spanning one entry point, named after it, so that a profiler
// timeline (Nsight Systems, ncu --nvtx) shows each library call around the
// kernels it launched.  Without an attached tool the push and pop return at
// once (NVTX v3 is header-only and loads nothing unless a tool asks).
struct TraceRange {
    explicit TraceRange(const char *name) { nvtxRangePushA(name); }
    ~TraceRange() { nvtxRangePop(); }
    TraceRange(const TraceRange &) = delete;
    TraceRange &operator=(const TraceRange &) = delete;
};
#define GFP_TRACE() ::gfp::TraceRange gfp_trace_range_(__func__)

// Device-side checks (builds with GFP_DEVICE_CHECKS only): a kernel that
// meets an input its contract excludes, or an index outside what its launch
// set up, records a bit in its translation unit's error word instead of
// faulting or trapping; gfp_context_check reports the bits (GFP_ERR_INVALID)
// and clears them.  Release builds compile the checks away.
#ifdef GFP_DEVICE_CHECKS
#define GFP_DCHECK(word, cond, bit)                              \
    do {                                                          \
        if (!(cond)) atomicOr(&(word), (uint32_t)(bit));         \
    } while (0)
#else
#define GFP_DCHECK(word, cond, bit) \
    do {                            \
    } while (0)
#endif
// bits of the device-check words
constexpr uint32_t DCHECK_CSR_COLUMN = 1u;     // a column index >= k
constexpr uint32_t DCHECK_CSR_ROW_PTR = 2u;    // row_ptr decreases
constexpr uint32_t DCHECK_DOT_UNIT = 4u;       // a work unit outside its pair
// Reads and clears the words of gfp_csr.cu and gfp_dot.cu (0 in release builds).
uint32_t csr_check_bits();
uint32_t dot_check_bits();

// One pair of a batch as the persistent kernel sees it (64 bytes).
struct DevPair {
    const uint32_t *x;
    const uint32_t *y;
    uint64_t n;
    uint64_t k;        // reduction interval for the chosen representation
    Mod m;             // 32 bytes
};
static_assert(sizeof(Mod) == 32, "Mod layout");

// Representation and unit count are kept beside the pair (read once per unit).
struct DevPairAux {
    uint32_t repr;
    uint32_t units;
};

// One work unit: elements [begin, end) of pair `pair`.
struct DevUnit {
    uint64_t begin;
    uint64_t end;
    uint32_t pair;
    uint32_t pad;
};

// Records a CUDA error for gfp_last_cuda_error (entry points in other units).
void note_cuda_error(cudaError_t e);

Mod make_mod(uint32_t p);
uint64_t delay_bound(uint32_t p, int acc_bits, int carried);
uint64_t k_for(Repr r, uint32_t p);
uint64_t centered_bound(uint32_t p);
uint64_t montgomery_bound(uint32_t p);
bool repr_eligible(Repr r, uint32_t p);

// Launch configuration constants of the dot kernels.
constexpr int DOT_THREADS = 256;
constexpr int MV_THREADS = 1024;

// Device scratch of one batched execution.
struct BatchScratch {
    unsigned long long *slots = nullptr;  // per pair: sum of unit residues
    uint32_t *tickets = nullptr;          // per pair: finished units
    uint32_t *ctr = nullptr;              // [0] next unit, [1] finished CTAs
};

// Kernel launchers (gfp_dot.cu, gfp_matvec.cu).
cudaError_t launch_dot_single(Repr r, const Mod &m, uint64_t k, uint64_t n, const uint32_t *x,
                              const uint32_t *y, unsigned long long *slot, uint32_t *out, int grid,
                              cudaStream_t s);
int dot_single_grid(Repr r, uint64_t n, int sm_count);
cudaError_t launch_dot_batched(const DevPair *pairs, const DevPairAux *aux, const DevUnit *units,
                               uint32_t n_units, BatchScratch sc, uint32_t *out, int grid,
                               cudaStream_t s);
int dot_batched_grid(int sm_count);
cudaError_t launch_fill_uniform(uint32_t p, uint64_t seed, uint64_t stream_id, uint64_t offset,
                                uint64_t n, uint32_t *out, cudaStream_t s);
// rows x cols of the same sequence (element r*cols + c) at out[r*ld + c]
cudaError_t launch_fill_uniform_2d(uint32_t p, uint64_t seed, uint64_t stream_id, uint64_t rows,
                                   uint64_t cols, uint64_t ld, uint32_t *out, cudaStream_t s);
cudaError_t launch_check_range(const uint32_t *v, uint64_t n, uint32_t p, uint32_t *flag,
                               cudaStream_t s);
// u non-null: also *sout = (sum_i u_i y_i) mod p, combined through slot/ticket
cudaError_t launch_matvec(Repr r, const Mod &m, uint64_t k, uint64_t rows, uint64_t cols,
                          const uint32_t *A, uint64_t lda, const uint32_t *x, uint32_t *y,
                          int sm_count, cudaStream_t s, const uint32_t *u = nullptr,
                          unsigned long long *slot = nullptr, uint32_t *ticket = nullptr,
                          uint32_t *sout = nullptr);

// Block product (gfp_block.cu).  The tensor-core path needs the centred
// residues to fit two balanced 8-bit digits: (p-1)/2 <= 32895.
constexpr uint32_t BLOCK_TC_MAX_P = 65791;
// Moduli of the residue passes, and of prepared operands taken directly: at
// most 65536, so that every residue has two 8-bit balanced digits.
constexpr uint32_t RNS_PRIME_MAX = 65536;
bool block_tc_eligible(uint32_t p, const uint32_t *A, uint64_t lda);
// A's layout suits the tensor-core kernel (TMA: 16-byte base, rows 16-byte apart)
bool block_tc_layout_ok(const uint32_t *A, uint64_t lda);

// Residue-number-system constants of a large-p tensor-core block product:
// moduli mod[0..L-1] (primes <= RNS_PRIME_MAX), inv[l][j] = mod[j]^-1 mod
// mod[l] for j < l, and the target modulus p.
constexpr int RNS_MAX = 6;
struct RnsConst {
    int L;
    uint32_t p;
    uint32_t mod[RNS_MAX];
    uint32_t inv[RNS_MAX][RNS_MAX];
    uint64_t minv[RNS_MAX];   // floor((2^64 - 1) / mod[l]), for remainders by multiply-high
    Mod modp;                 // Barrett constants of p
};
// Chooses the moduli for k-term sums of products of residues below p; false
// when RNS_MAX moduli do not cover k (p-1)^2.
bool block_rns_plan(uint32_t p, uint64_t k, RnsConst *rc);
cudaError_t launch_block_crt(const uint32_t *R, uint64_t m, uint64_t nb, uint32_t *C, uint64_t ldc,
                             const RnsConst &rc, int sm_count, cudaStream_t s);
size_t block_tc_workspace_bytes(uint64_t m, uint64_t k, uint64_t nb);
size_t block_tc_bimg_bytes(uint64_t k, uint64_t nb);   // the rest must be zero at launch
cudaError_t launch_block_tc(const Mod &mod, uint64_t m, uint64_t k, uint64_t nb, const uint32_t *A,
                            uint64_t lda, const uint32_t *B, uint64_t ldb, uint32_t *C, uint64_t ldc,
                            void *ws, int sm_count, cudaStream_t s, int *launches,
                            bool reduce_inputs = false, const uint8_t *Aimg = nullptr);
// Prepared A: digit image of A for one modulus (block_prep_a_bytes(m, k)
// bytes), consumed by launch_block_tc through Aimg (A and lda then unused).
size_t block_prep_a_bytes(uint64_t m, uint64_t k);
cudaError_t launch_block_prep_a(const Mod &mod, uint64_t m, uint64_t k, const uint32_t *A,
                                uint64_t lda, bool reduce_inputs, uint8_t *img, cudaStream_t s);
uint32_t *block_tc_err_flag(void *ws, uint64_t m, uint64_t k, uint64_t nb);
// Runs the bounded-wait self test; *status_bits gets the device error word.
cudaError_t wait_selftest(uint64_t limit_ns, cudaStream_t s, uint32_t *status_bits);
cudaError_t launch_block_cc(Repr r, const Mod &mod, uint64_t kbound, uint64_t m, uint64_t k,
                            uint64_t nb, const uint32_t *A, uint64_t lda, const uint32_t *B,
                            uint64_t ldb, uint32_t *C, uint64_t ldc, cudaStream_t s);
// Sparse-row block product (gfp_csr.cu).
cudaError_t launch_block_csr(Repr r, const Mod &mod, uint64_t kbound, uint64_t m, uint64_t k,
                             uint64_t nb,
                             const uint32_t *row_ptr, const uint32_t *col, const uint32_t *val,
                             const uint32_t *B, uint64_t ldb, uint32_t *C, uint64_t ldc,
                             int sm_count, cudaStream_t s);

}  // namespace gfp

// Tuned plan entry: representation and unit chunk per (p, length bucket).
struct gfp_plan_entry {
    uint32_t p;
    uint32_t lg_n;      // bucket: floor(log2(n)), 0..63
    uint32_t repr;
    uint32_t chunk;     // work-unit length in elements for batched execution
};

struct gfp_ctx {
    int device = 0;
    int sm_count = 0;
    int blk_sms = 0;   // CTAs of a tensor-core block kernel (0: one per SM); set by the service
    gfp_repr forced = GFP_REPR_AUTO;
    bool validate = false;
    std::atomic<uint64_t> launches{0};
    std::mutex mu;

    // single-dot scratch ring: one packed (residue sum, CTA count) word per slot
    unsigned long long *ring_slots = nullptr;
    uint32_t ring_size = 1024;
    std::atomic<uint32_t> ring_pos{0};

    // validation flag (device) and pinned host mirror
    uint32_t *d_flag = nullptr;

    // one-shot batched workspace (grown on demand)
    void *bw = nullptr;
    size_t bw_bytes = 0;
    size_t bw_slots_off = (size_t)-1;   // offset of the scratch region last cleared
    // host-buffer staging for gfp_dot_batched_host; copies are split over
    // several streams so that more than one copy engine moves them
    static constexpr int kCopyStreams = 4;
    cudaStream_t copy_streams[kCopyStreams] = {};
    cudaEvent_t copy_events[kCopyStreams + 1] = {};
    uint32_t *stage = nullptr;
    size_t stage_elems = 0;
    uint32_t *stage_out = nullptr;
    size_t stage_out_elems = 0;

    // block-product workspace (B digit image, column-major partial sums,
    // error flag); zero outside calls except the B image; grown on demand
    void *blk_ws = nullptr;
    size_t blk_ws_bytes = 0;
    uint64_t blk_m = 0, blk_k = 0, blk_nb = 0;   // shape whose error flag is live

    // tuned plan: (p, lg_n) -> entry
    std::map<std::pair<uint32_t, uint32_t>, gfp_plan_entry> plan;
    uint32_t default_chunk = 65536;

    // cached matvec iteration graphs
    struct GraphKey {
        uint32_t p; uint64_t n; const uint32_t *A; uint64_t lda; const uint32_t *x0; uint32_t *Y;
        uint32_t iters; int repr;
        bool operator<(const GraphKey &o) const
        {
            return std::tie(p, n, A, lda, x0, Y, iters, repr) <
                   std::tie(o.p, o.n, o.A, o.lda, o.x0, o.Y, o.iters, o.repr);
        }
    };
    std::map<GraphKey, cudaGraphExec_t> graphs;
    // sequence graphs (x0, u, A, ...) and their ping-pong vectors
    struct SeqKey {
        uint32_t p; uint64_t n; const uint32_t *A; uint64_t lda; const uint32_t *x0;
        const uint32_t *u; uint32_t *seq; uint32_t *Y; uint32_t iters; int repr;
        bool operator<(const SeqKey &o) const
        {
            return std::tie(p, n, A, lda, x0, u, seq, Y, iters, repr) <
                   std::tie(o.p, o.n, o.A, o.lda, o.x0, o.u, o.seq, o.Y, o.iters, o.repr);
        }
    };
    std::map<SeqKey, cudaGraphExec_t> seq_graphs;
    uint32_t *pingpong = nullptr;
    uint64_t pingpong_n = 0;
    unsigned long long *seq_slots = nullptr;   // per-iteration projection scratch
    uint32_t *seq_tickets = nullptr;
    uint32_t seq_cap = 0;
};
