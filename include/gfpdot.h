/*
 * libgfpdot — exact dot products over word-size prime fields GF(p) on GB300.
 *
 * The method is J.-G. Dumas, "Efficient dot product over word-size finite
 * fields": residues are multiplied and accumulated unreduced and reduced
 * modulo p only when the accumulator could overflow (delayed division,
 * Section 3.1, Eq. (1); blocked form, Section 3.2; division on demand by
 * overflow detection, Section 3.3; hybrid, Section 3.4, Eq. (2)), with one
 * final reduction into [0, p).  Every call returns the exact residue: the
 * result of each entry point is bit-identical to the plain definition
 * (sum x_i*y_i) mod p, whatever representation computes it.
 *
 * Conventions (all entry points)
 *  - Residues are uint32_t and must be canonical (0 <= v < p).  Non-canonical
 *    inputs are outside the contract; with validation enabled
 *    (gfp_set_validate or GFP_VALIDATE=1) the operand-checking entry points
 *    detect them on the device and return GFP_ERR_RANGE (this adds a device
 *    synchronisation, so it is not usable under stream capture).
 *  - The modulus p satisfies 2 <= p <= 2^32-1.  Primality is not required by
 *    the arithmetic (results are residues modulo p), but the method is stated
 *    for prime fields and the tests use primes.
 *  - Pointer arguments named "device" are CUDA device pointers (4-byte
 *    aligned; 16-byte alignment enables the 128-bit load path, other
 *    alignments fall back to 32-bit loads inside the same kernel).  Pointers
 *    named "host" are host memory.  The caller owns every operand and output
 *    buffer; they must stay alive until the work queued on `stream` completes.
 *    The library owns only the context/plan/server objects it creates and
 *    never frees caller memory.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Compute entry points only enqueue work: they return before the
 *    result is ready unless documented otherwise.
 *  - Errors: argument checks happen before any launch and return a negative
 *    status with nothing enqueued.  Launch failures return GFP_ERR_CUDA.
 *    Asynchronous device errors surface on a later call that synchronises.
 *    No exception crosses this interface and nothing aborts the process.
 */
#ifndef GFPDOT_H
#define GFPDOT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define GFP_API __attribute__((visibility("default")))
#else
#define GFP_API
#endif

typedef enum gfp_status {
    GFP_OK = 0,
    GFP_PENDING = 1,             /* service: job not finished yet */
    GFP_ERR_INVALID = -1,        /* NULL pointer, p < 2, bad dimensions or strides */
    GFP_ERR_RANGE = -2,          /* an input residue >= p (validation enabled) */
    GFP_ERR_UNSUPPORTED = -3,    /* requested representation not eligible for p */
    GFP_ERR_NOMEM = -4,          /* device or host allocation failed */
    GFP_ERR_CUDA = -5,           /* a CUDA runtime call or launch failed */
    GFP_ERR_AGAIN = -6,          /* service queue full */
    GFP_ERR_TIMEOUT = -7,        /* a bounded wait ran out */
    GFP_ERR_UNKNOWN_TICKET = -8, /* service: no such ticket */
    GFP_ERR_CANCELLED = -9       /* service: job cancelled or server shut down */
} gfp_status;

/* Accumulation representation of the dot-product kernels. */
typedef enum gfp_repr {
    GFP_REPR_AUTO = 0,      /* per-(p, n) choice from the tuned plan or the default rules */
    GFP_REPR_PERTERM = 1,   /* classical Zpz: one remainder per term (Section 2.1); baseline */
    GFP_REPR_U64_BLOCK = 2, /* 64-bit accumulator reduced every k terms (Sections 3.1-3.2,
                               k from Eq. (2) with the residue carried between blocks) */
    GFP_REPR_U64_CARRY = 3, /* division on demand (Section 3.3): 64-bit sum that may wrap, a
                               32-bit wrap count, and one correction by 2^64 mod p at the end */
    GFP_REPR_FP64 = 4,      /* 53-bit exact double accumulator reduced every k terms with the
                               floating-point reduction of Section 2.3 (p <= 94906266 only) */
    GFP_REPR_F16TC = 5,     /* block product only: centred residues (Section 3.2.2) split into
                               two balanced 8-bit digits, exact fp16 tensor-core products with
                               fp32 accumulation over chunks of 1024 terms (p <= 65791; larger
                               p through residues modulo primes <= 65536) */
    GFP_REPR_CENTERED = 6,  /* centred representation (Section 3.2.2): signed residues in
                               [-(p-1)/2, (p-1)/2], signed 64-bit accumulator reduced every
                               k terms, k h^2 + (p-1) <= 2^63 - 1 with h = (p-1)/2 */
    GFP_REPR_MONTGOMERY = 7,/* Montgomery reduction (Sections 2.2, 3.2.1), B = 2^32, odd p:
                               blocks of k products with k (p-1)^2 < p B reduced by REDC,
                               the B^-1 factor removed once at the end */
    GFP_REPR_COUNT_ = 8
} gfp_repr;

typedef struct gfp_ctx gfp_ctx;

/* Per-modulus constants (Section 3, host side). */
typedef struct gfp_params {
    uint32_t p;
    uint32_t corr;        /* CORR = 2^64 mod p (Section 3.3 with m = 64) */
    uint64_t k_u64;       /* Eq. (2), m = 64: largest k with k(p-1)^2 + (p-1) < 2^64 */
    uint64_t k_fp64;      /* Eq. (2), m = 53: largest k with k(p-1)^2 + (p-1) < 2^53; 0 if none */
    uint64_t barrett_mu;  /* floor(2^64 / p), Barrett's reduction constant */
    double   inv_p;       /* 1/p rounded to double (Section 2.3) */
    int      fp64_ok;     /* 1 when k_fp64 >= 1 */
    uint64_t k_centered;  /* GFP_REPR_CENTERED block length (see gfp_repr) */
    uint64_t k_montgomery;/* GFP_REPR_MONTGOMERY block length; 0 for even p */
} gfp_params;

/* ---- status and parameters (host only; usable without a GPU) ---- */

/* Static string naming a status code. */
GFP_API const char *gfp_status_string(int status);
/* Description of the last CUDA error that made an entry point of the calling
 * thread return GFP_ERR_CUDA ("no CUDA error" if none). */
GFP_API const char *gfp_last_cuda_error(void);

/* Largest number of products lambda that an acc_bits-wide unsigned
 * accumulator can absorb before a reduction is required (Section 3.1,
 * Eq. (1): lambda (p-1)^2 < 2^m; with carried != 0, Section 3.4, Eq. (2) in its
 * tight form lambda (p-1)^2 + (p-1) < 2^m, for a block that starts from a
 * residue already reduced below p).  acc_bits in [1, 64].  Returns 0 when no
 * product fits, or for invalid arguments (p < 2, acc_bits out of range). */
GFP_API uint64_t gfp_delay_bound(uint32_t p, int acc_bits, int carried);

/* Fill *out with the constants above.  GFP_ERR_INVALID if p < 2 or out NULL. */
GFP_API gfp_status gfp_get_params(uint32_t p, gfp_params *out);

/* Host evaluation of the library's reductions (the same inline code the
 * kernels use), for testing: x mod p by Barrett's method, and the
 * floating-point reduction of Section 2.3 of an integral 0 <= T <= 2^53. */
GFP_API uint32_t gfp_reduce_u64(uint64_t x, uint32_t p);
GFP_API double   gfp_reduce_f64(double T, uint32_t p);

/* Representation that GFP_REPR_AUTO resolves to for (p, n) in `ctx`
 * (ctx may be NULL for the built-in rules). */
GFP_API gfp_repr gfp_choose_repr(const gfp_ctx *ctx, uint32_t p, uint64_t n);

/* ---- context ---- */

/* Create a context bound to CUDA device `device`; allocates its workspace
 * (a few MB).  *out receives the handle.  GFP_ERR_CUDA if the device is
 * unavailable.  Reads GFP_PLAN_FILE (tuned plan), GFP_FORCE_REPR (0..4) and
 * GFP_VALIDATE (0/1) from the environment. */
GFP_API gfp_status gfp_context_create(int device, gfp_ctx **out);
/* Synchronise the context's work, free its workspace and the handle. */
GFP_API gfp_status gfp_context_destroy(gfp_ctx *ctx);
/* Force a representation for later calls (GFP_REPR_AUTO restores the
 * automatic choice).  Calls whose p is not eligible then fail with
 * GFP_ERR_UNSUPPORTED. */
GFP_API gfp_status gfp_set_repr(gfp_ctx *ctx, gfp_repr repr);
/* Enable (1) or disable (0) device-side input validation. */
GFP_API gfp_status gfp_set_validate(gfp_ctx *ctx, int on);
/* Number of kernels this context has launched so far (diagnostics). */
GFP_API uint64_t gfp_launch_count(const gfp_ctx *ctx);

/* ---- dot products ---- */

/* out[0] = (sum_{i<n} x[i]*y[i]) mod p.
 *   x, y: device, n residues each.  out: device, one uint32_t.
 * n == 0 writes 0.  One kernel launch; uses one slot of the context's scratch
 * ring (calls in flight at the same time on different streams take different
 * slots; more than 1024 such calls in flight at once would share a slot). */
GFP_API gfp_status gfp_dot(gfp_ctx *ctx, uint32_t p, uint64_t n, const uint32_t *x,
                           const uint32_t *y, uint32_t *out, void *stream);

/* One pair of a batch: x, y device pointers of n residues modulo p. */
typedef struct gfp_dot_desc {
    uint32_t p;
    uint32_t repr;          /* gfp_repr for this pair; GFP_REPR_AUTO for the context's choice */
    uint64_t n;
    const uint32_t *x;
    const uint32_t *y;
} gfp_dot_desc;

/* out[j] = dot of pair d[j] modulo d[j].p for 0 <= j < count, in ONE
 * persistent kernel launch over a work list of (pair, chunk) units of uneven
 * lengths and mixed moduli.  d: host array.  out: device, count uint32_t.
 * Builds the work list on the host and uploads it into the context's
 * workspace (pageable copy: not usable under stream capture; use a plan).
 * Calls sharing one context must not overlap on different streams. */
GFP_API gfp_status gfp_dot_batched(gfp_ctx *ctx, const gfp_dot_desc *d, uint64_t count,
                                   uint32_t *out, void *stream);

/* Reusable batch plan: the work list and its scratch live on the device, so
 * gfp_batch_plan_exec is a single kernel launch, capture-safe, with no host
 * work.  The descriptors (pointers, lengths, moduli) are fixed at creation;
 * the operand contents may change between executions.  One plan must not be
 * executed concurrently on two streams (its scratch counters are shared). */
typedef struct gfp_batch_plan gfp_batch_plan;
GFP_API gfp_status gfp_batch_plan_create(gfp_ctx *ctx, const gfp_dot_desc *d, uint64_t count,
                                         gfp_batch_plan **out);
GFP_API gfp_status gfp_batch_plan_exec(gfp_batch_plan *plan, uint32_t *out, void *stream);
/* Units in the plan's work list and algorithmic operand bytes per execution. */
GFP_API gfp_status gfp_batch_plan_info(const gfp_batch_plan *plan, uint64_t *units,
                                       uint64_t *bytes);
GFP_API gfp_status gfp_batch_plan_destroy(gfp_batch_plan *plan);

/* Batched dot products from HOST buffers (end-to-end form): pair j is
 * x_host[off[j] .. off[j]+n[j]) and y_host[...] modulo p[j]; all arrays are
 * host memory (pinned memory gives full copy bandwidth).  The call copies
 * the `total` elements of x_host and y_host to the device, runs the batched
 * kernel, copies the count residues back into out_host and synchronises
 * `stream` before returning.  off[j] must be a multiple of 4 and
 * off[j] + n[j] <= total.  Device staging is held by the context and grown on
 * demand. */
GFP_API gfp_status gfp_dot_batched_host(gfp_ctx *ctx, uint64_t count, const uint32_t *p,
                                        const uint64_t *n, const uint64_t *off,
                                        const uint32_t *x_host, const uint32_t *y_host,
                                        uint64_t total, uint32_t *out_host, void *stream);

/* Batched dot products that allocate nothing (no counterpart in the paper:
 * an interface convenience).  For callers that cannot call cudaMalloc where
 * they need the result (fixed device-memory budgets owned by a host
 * application, paths where an allocation may block or fail): same result
 * and same kernel as gfp_dot_batched, but all scratch lives in one
 * file-scope device array of fixed size that every device loading the
 * library holds until process exit.  No context is needed; the current CUDA
 * device is used and GFP_REPR_AUTO follows the built-in rules.
 *   d: host array of count descriptors (operands on the current device).
 *   out: device, count uint32_t.
 * Limits: count <= 1024 pairs and at most 16384 work units of 65536
 * elements (about 2^30 elements in total); beyond either, GFP_ERR_INVALID
 * with nothing enqueued.  The first call on a device looks up the array's
 * device address (a failure there is returned as GFP_ERR_CUDA).  All calls
 * share the array (each clears the parts that must start at zero): calls
 * whose work overlaps on the GPU race, so order them on one stream. */
GFP_API gfp_status gfp_dot_batched_noalloc(const gfp_dot_desc *d, uint64_t count, uint32_t *out,
                                           void *stream);

/* ---- matrix-vector (the iterative use named in Section 1) ---- */

/* y[i] = (sum_j A[i*lda + j] * x[j]) mod p for 0 <= i < rows.
 *   A: device, row-major, lda >= cols.  x: device, cols.  y: device, rows.
 * y must not overlap A or x.  One kernel launch. */
GFP_API gfp_status gfp_matvec(gfp_ctx *ctx, uint32_t p, uint64_t rows, uint64_t cols,
                              const uint32_t *A, uint64_t lda, const uint32_t *x, uint32_t *y,
                              void *stream);

/* Wiedemann-style iteration x_{t+1} = A x_t for t = 0 .. iters-1 with a square
 * n x n matrix, all launches captured once in a CUDA graph (cached in the
 * context per argument set) and replayed with one graph launch.
 *   x0: device, n.  Y: device, iters*n; row t receives x_{t+1}. */
GFP_API gfp_status gfp_matvec_iterate(gfp_ctx *ctx, uint32_t p, uint64_t n, const uint32_t *A,
                                      uint64_t lda, const uint32_t *x0, uint32_t *Y,
                                      uint32_t iters, void *stream);

/* The scalar sequence of a Wiedemann-style iteration (the iterative methods
 * the introduction names as users of the dot product): seq[t] = u^T A^t x0
 * mod p for t = 0 .. iters, with x_{t+1} = A x_t.  Each product's projection
 * onto u is fused into the matrix-vector kernel's epilogue (no second pass
 * over y).  A: device n x n (lda >= n); x0, u: device, n; seq: device,
 * iters + 1; Y: device iters x n receiving x_1 .. x_iters, or NULL to keep
 * them in context scratch.  The launches are captured once in a CUDA graph
 * (cached per argument set) and replayed with one graph launch; scratch is
 * grown on the first call, so make it outside stream capture.  Calls sharing
 * one context must not overlap on different streams.  iters <= 65535. */
GFP_API gfp_status gfp_matvec_sequence(gfp_ctx *ctx, uint32_t p, uint64_t n, const uint32_t *A,
                                       uint64_t lda, const uint32_t *x0, const uint32_t *u,
                                       uint32_t iters, uint32_t *seq, uint32_t *Y, void *stream);

/* ---- block products (dense contraction of many dot products) ---- */

/* C[i*ldc + j] = (sum_t A[i*lda + t] * B[t*ldb + j]) mod p, 0 <= i < m,
 * 0 <= j < nb.  A (m x k), B (k x nb), C (m x nb): device, row-major,
 * lda >= k, ldb >= nb, ldc >= nb; C must not overlap A or B.
 * Path: with GFP_REPR_AUTO or GFP_REPR_F16TC, A 16-byte aligned and lda a
 * multiple of 4, the tensor cores: for p <= 65791 the digit kernel directly
 * (three launches: B digit split, the persistent product, the reduction of
 * its partial sums into C); for larger p
 * one such pass per modulus of a residue number system (the L <= 6 largest
 * primes <= 65536 whose product exceeds k (p-1)^2, each pass reducing the
 * inputs modulo its prime) and one launch recombining the residues with
 * Garner's method modulo p.  Otherwise the CUDA-core kernel with the
 * representation forced on the context, else the built-in rule for p (tuned
 * plans time the dot-product kernels and do not apply here; forcing F16TC
 * where the tensor cores are not eligible gives GFP_ERR_UNSUPPORTED).  The tensor-core path
 * uses the context's workspace (grown on demand, so call once outside stream
 * capture for the largest shape) and must not run concurrently with another
 * block product of the same context.  k == 0 writes zeros. */
GFP_API gfp_status gfp_matmul_block(gfp_ctx *ctx, uint32_t p, uint64_t m, uint64_t k, uint64_t nb,
                                    const uint32_t *A, uint64_t lda, const uint32_t *B,
                                    uint64_t ldb, uint32_t *C, uint64_t ldc, void *stream);

/* A prepared once for repeated block products with the same A (block
 * Wiedemann-style iterations, a resident matrix serving many requests): the
 * residues of A split once into the two balanced 8-bit digits the tensor-core
 * product multiplies (the centred representation of Section 3.2.2, with the
 * representative of each residue taken in [-32896, 32639] so that both
 * digits fit a byte), stored as two 8-bit digit planes per tile, 2 bytes per
 * entry of A: each product reads half the bytes of the uint32 A and only
 * widens the digits to fp16 in shared memory.  For p <= 65536 one image; for
 * larger p one image per residue-pass modulus (A reduced modulo each, 2 bytes
 * per entry each; gfp_block_prep_info gives the bytes and the pass count).
 *   A: device, m x k row-major, lda >= k, canonical residues; not referenced
 *   after the call returns (it synchronises the device).  m, k >= 1.
 * GFP_ERR_UNSUPPORTED when no residue passes cover k (p-1)^2; GFP_ERR_NOMEM
 * when the image does not fit.  The prepared object owns its device memory
 * until gfp_block_prep_destroy. */
typedef struct gfp_block_prep gfp_block_prep;
GFP_API gfp_status gfp_block_prepare(gfp_ctx *ctx, uint32_t p, uint64_t m, uint64_t k,
                                     const uint32_t *A, uint64_t lda, gfp_block_prep **out);
/* C = A B mod p for the prepared A (m x k): B device k x nb (ldb >= nb),
 * C device m x nb (ldc >= nb); the same result as gfp_matmul_block on the
 * original A.  Three launches (B's digits, the product, its partial sums
 * into C), or three per residue pass plus one recombination.  Uses the
 * context's block workspace (grown on first use of a shape: make that call
 * outside stream capture); calls sharing one context must not run
 * concurrently on different streams. */
GFP_API gfp_status gfp_matmul_block_prepared(gfp_ctx *ctx, const gfp_block_prep *prep, uint64_t nb,
                                             const uint32_t *B, uint64_t ldb, uint32_t *C,
                                             uint64_t ldc, void *stream);
/* Device bytes held and residue passes per product (1 for p <= 65536). */
GFP_API gfp_status gfp_block_prep_info(const gfp_block_prep *prep, uint64_t *bytes,
                                       uint32_t *passes);
/* Synchronises the device and frees the prepared images. */
GFP_API gfp_status gfp_block_prep_destroy(gfp_block_prep *prep);

/* Sparse-row block product: A is m x k in CSR form (row_ptr[m+1] offsets
 * into col[] and val[], column indices < k, values canonical residues), B is
 * k x nb dense.  C[i*ldc + j] = (sum_q val[q] * B[col[q]*ldb + j]) mod p for
 * row_ptr[i] <= q < row_ptr[i+1].  All arrays on the device; row_ptr must be
 * non-decreasing with row_ptr[0] = 0 (checked on the device only when
 * validation is enabled, together with col < k and the residues).  One launch;
 * k == 0 writes zeros.  Representation: the one forced on the context, else
 * the built-in rule for p (tuned plans do not apply). */
GFP_API gfp_status gfp_matmul_block_csr(gfp_ctx *ctx, uint32_t p, uint64_t m, uint64_t k,
                                        uint64_t nb, const uint32_t *row_ptr, const uint32_t *col,
                                        const uint32_t *val, const uint32_t *B, uint64_t ldb,
                                        uint32_t *C, uint64_t ldc, void *stream);

/* Synchronise the context's device and report whether a kernel of the
 * context gave up on a bounded wait since the last check (GFP_ERR_TIMEOUT,
 * after which the workspace is cleared so later calls start clean), or a
 * CUDA error is pending (GFP_ERR_CUDA).  In a library built with device-side
 * checks (GFP_DEVICE_CHECKS), also GFP_ERR_INVALID when a kernel met input
 * outside its contract since the last check (a sparse-row column >= k or a
 * decreasing row_ptr, a batched work unit outside its pair); the kernels
 * skip such input instead of faulting, and the check clears the record.
 * GFP_OK otherwise. */
GFP_API gfp_status gfp_context_check(gfp_ctx *ctx);

/* Failure-detection self test (no counterpart in the paper): launches one
 * thread that waits, with the same bounded wait the tensor-core kernel uses
 * for its pipeline barriers, on a barrier nothing arrives on.  The wait must
 * give up after limit_ns (1 ms <= limit_ns <= 2 s) and report it: the call
 * synchronises `stream` and returns GFP_ERR_TIMEOUT when the expiry was
 * detected (the expected outcome; the context stays usable), GFP_OK if the
 * wait somehow completed, GFP_ERR_INVALID for a limit out of range. */
GFP_API gfp_status gfp_wait_selftest(uint64_t limit_ns, void *stream);

/* ---- install-time tuning (automated empirical optimisation, Section 4) ---- */

/* Time every eligible representation (U64_BLOCK, U64_CARRY, FP64, CENTERED,
 * MONTGOMERY) and
 * work-unit length (16Ki, 64Ki, 256Ki elements) for each prime of
 * primes[0..nprimes) (NULL: 32749, 65521, 67108859, 2^31-1, 2^32-5) and
 * each length 2^lg, lg = lg_lo, lg_lo+2, ..., <= lg_hi (lg_hi <= 26), on
 * batches of resident synthetic vectors (512 MiB of operands), and record the
 * fastest choice per (p, floor(log2 n)) in the context's plan; GFP_REPR_AUTO
 * calls consult it (nearest length bucket of the same p).  Writes the plan to
 * plan_path when it is not NULL.  Synchronous; allocates while it runs. */
GFP_API gfp_status gfp_tune(gfp_ctx *ctx, const uint32_t *primes, uint32_t nprimes,
                            uint32_t lg_lo, uint32_t lg_hi, const char *plan_path);
/* Replace the context's plan by the one in `path` / write it to `path`
 * (format: {"version": 1, "entries": [{"p":P, "lg_n":L, "repr":R, "chunk":C}, ...]}).
 * GFP_ERR_INVALID if the file cannot be read or parsed (plan unchanged). */
GFP_API gfp_status gfp_plan_load(gfp_ctx *ctx, const char *path);
GFP_API gfp_status gfp_plan_save(const gfp_ctx *ctx, const char *path);
/* Number of (p, length bucket) entries in the context's plan. */
GFP_API uint64_t gfp_plan_size(const gfp_ctx *ctx);

/* ---- service: continuous batching of dot, matrix-vector and block jobs ---- */

typedef struct gfp_server gfp_server;

typedef enum gfp_job_kind { GFP_JOB_DOT = 0, GFP_JOB_MATVEC = 1, GFP_JOB_BLOCK = 2 } gfp_job_kind;

typedef struct gfp_server_cfg {
    int device;                 /* CUDA device */
    uint64_t mem_budget;        /* device bytes for job operands and results (0: the
                                   environment variable GFP_MEM_BUDGET, in bytes, else 4 GiB) */
    uint32_t max_inflight;      /* launches on the GPU at once; a batched dot launch counts once (0: 256) */
    uint32_t n_streams;         /* stream pool size (0: 4); with two or more, the first half
                                   (rounded up) run at the highest stream priority and take
                                   dot and matrix-vector launches, the rest take block jobs at
                                   the lowest priority */
    uint32_t queue_capacity;    /* submitted but not admitted jobs before GFP_ERR_AGAIN (0: 65536) */
    uint32_t batch_window_us;   /* dot jobs arriving within this window share one launch (0: none) */
    uint32_t simulate;          /* 1: no GPU; jobs "run" on the host for a time proportional to
                                   their work (scheduling, admission and API tests without a GPU) */
    uint32_t fail_every;        /* fault injection: every n-th admission attempt fails as if the
                                   device allocation failed (0: off) */
    uint32_t block_sm_percent;  /* share of the SMs that one BLOCK job's tensor-core kernel may
                                   occupy, in percent (0 or >= 100: all).  Its persistent CTAs
                                   fill an SM each; leaving some SMs to the other jobs keeps dot
                                   and matrix-vector jobs from waiting behind a block job */
} gfp_server_cfg;

/* A job.  Operands are either caller device pointers (which must stay valid
 * until the job completes) or, when a pointer is NULL, generated by the server
 * in its own memory with gfp_fill_uniform(p, seed, stream, 0, ...), stream 0
 * for x / the vector / B and stream 1 for y.
 *   DOT:    n, x, y.  The residue is returned in gfp_result.value.
 *   MATVEC: matrix (handle of a registered rows x cols matrix), v (cols).
 *           Output: rows residues in server memory.
 *   BLOCK:  matrix (m x k), v = B (k x nb, row-major), nb.  Output m x nb.
 * Outputs of MATVEC and BLOCK stay in server memory (counted against the
 * budget) until gfp_release; read them with gfp_result_copy. */
typedef struct gfp_job {
    uint32_t kind;
    uint32_t p;
    uint64_t n;
    uint64_t nb;
    uint64_t matrix;
    const uint32_t *x;
    const uint32_t *y;
    const uint32_t *v;
    uint64_t seed;
} gfp_job;

typedef struct gfp_result {
    int32_t status;             /* GFP_OK, GFP_ERR_* of the job */
    uint32_t kind;
    uint32_t value;             /* DOT: the residue */
    uint32_t batch;             /* DOT: number of dot jobs that shared its launch */
    uint64_t out_elems;         /* MATVEC / BLOCK: output residues held for gfp_result_copy */
    uint64_t t_submit_ns, t_admit_ns, t_start_ns, t_done_ns;   /* steady clock: submitted,
                                   admitted, its launches enqueued on the GPU (simulation: launch
                                   decided), completion seen by the dispatcher */
} gfp_result;

typedef struct gfp_server_stats {
    uint64_t submitted, admitted, completed, failed, cancelled;
    uint64_t admission_stalls;  /* dispatcher passes that left a job waiting for memory or a slot */
    uint64_t dot_launches;      /* batched launches carrying dot jobs */
    uint64_t mem_in_use, mem_peak, mem_budget;
    uint64_t kernel_launches;
} gfp_server_stats;

/* Start a server: allocates the memory budget as one device arena, the stream
 * pool and one context per stream, and starts the dispatcher thread. */
GFP_API gfp_status gfp_server_create(const gfp_server_cfg *cfg, gfp_server **out);
/* Stop the dispatcher, cancel jobs not yet admitted (GFP_ERR_CANCELLED),
 * wait (bounded, 10 s) for jobs on the GPU, free everything. */
GFP_API gfp_status gfp_server_destroy(gfp_server *srv);
/* Register a resident rows x cols matrix: `dev` (caller-owned device memory,
 * row-major, leading dimension cols) or, when dev is NULL, generated into
 * server memory outside the job budget from (p, seed, stream 0).  *handle
 * identifies it in MATVEC and BLOCK jobs. */
GFP_API gfp_status gfp_register_matrix(gfp_server *srv, uint32_t p, uint64_t rows, uint64_t cols,
                                       const uint32_t *dev, uint64_t seed, uint64_t *handle);
/* Prepare a registered matrix for BLOCK jobs: its tensor-core digit images
 * (gfp_block_prepare) are built now, held outside the job budget until the
 * server is destroyed, and every later BLOCK job on it reads them instead of
 * converting the matrix on each product (results are identical).  Optional;
 * synchronises the device.  A no-op in simulation mode or when already
 * prepared.  GFP_ERR_INVALID for an unknown handle, the errors of
 * gfp_block_prepare otherwise. */
GFP_API gfp_status gfp_prepare_matrix(gfp_server *srv, uint64_t handle);
/* Queue a job; never blocks.  GFP_ERR_INVALID for malformed jobs (unknown
 * kind or matrix, p mismatch, zero sizes), GFP_ERR_NOMEM if the job alone
 * exceeds the budget, GFP_ERR_AGAIN if the queue is full. */
GFP_API gfp_status gfp_submit(gfp_server *srv, const gfp_job *job, uint64_t *ticket);
/* Non-blocking: GFP_PENDING while queued or running; otherwise fills *res and
 * returns GFP_OK (the job's own status is res->status). */
GFP_API gfp_status gfp_poll(gfp_server *srv, uint64_t ticket, gfp_result *res);
/* Blocking poll with a bound: GFP_ERR_TIMEOUT if not done within timeout_us. */
GFP_API gfp_status gfp_wait(gfp_server *srv, uint64_t ticket, uint64_t timeout_us, gfp_result *res);
/* Copy a finished MATVEC / BLOCK job's outputs (count residues) to host memory. */
GFP_API gfp_status gfp_result_copy(gfp_server *srv, uint64_t ticket, uint32_t *host, uint64_t count);
/* Forget a finished job and free its outputs; cancel it if still queued. */
GFP_API gfp_status gfp_release(gfp_server *srv, uint64_t ticket);
GFP_API gfp_status gfp_server_get_stats(gfp_server *srv, gfp_server_stats *out);

/* ---- finite fields GF(p^k) in the discrete-logarithm representation ---- */

/* Section 2.4 ("Discrete logarithms", "Field extensions"): a dot product over
 * GF(q), q = p^k <= 2^16, prime field or extension, with every element stored
 * as a 16-bit code: 0 for zero, e for x^e (1 <= e <= q-2) and q-1 for 1,
 * where x is the class of x in GF(p)[x]/(f) for a monic f = x^k + f[k-1]
 * x^(k-1) + ... + f[0] whose powers of x run through all q-1 non-zero
 * elements (a primitive polynomial).  A product is one code addition modulo
 * q-1 and a sum one lookup in the table Z[t] = code of 1 + x^t (the paper's
 * "plus one" table of q entries), so the arithmetic is the same whatever k.
 *
 * Element values (the other end of the conversions) encode the polynomial
 * sum_j c_j x^j (0 <= c_j < p) as the integer sum_j c_j p^j; for k = 1 that is
 * the residue itself and f = x + f[0] makes x = -f[0] mod p, which must be a
 * primitive root.
 *
 * A field object owns its tables (host-built, resident on `device`) and the
 * dot product's scratch: dot products and conversions on one field object
 * must not run concurrently on several streams. */
typedef struct gfp_gfq gfp_gfq;

/* Writes to f[0..k-1] the first primitive polynomial of degree k over GF(p)
 * (candidates in lexicographic order of f[k-1..1], then f[0] = 1, 2, ...),
 * searched on the host.  GFP_ERR_INVALID if p^k > 2^16, p < 2, k < 1, or no
 * candidate qualifies (p not prime). */
GFP_API gfp_status gfp_gfq_find_primitive(uint32_t p, uint32_t k, uint32_t *f);

/* Builds GF(p^k) from f[0..k-1] (host array, entries < p) on `device`.
 * GFP_ERR_INVALID if p^k > 2^16, an entry of f is >= p, or x does not
 * generate all q-1 non-zero elements modulo f (f reducible or not
 * primitive, or p not prime); GFP_ERR_NOMEM / GFP_ERR_CUDA on device
 * failures.  Device memory: two 128 KiB tables (Zech logarithms, code to
 * value) + 8 q bytes + scratch, plus 256 + q^2 bytes for odd p, k > 1 and
 * q <= 256. */
GFP_API gfp_status gfp_gfq_create(int device, uint32_t p, uint32_t k, const uint32_t *f, gfp_gfq **out);
GFP_API gfp_status gfp_gfq_destroy(gfp_gfq *fq);
/* p, k and q = p^k of a field (any output pointer may be NULL). */
GFP_API gfp_status gfp_gfq_info(const gfp_gfq *fq, uint32_t *p, uint32_t *k, uint32_t *q);

/* codes[i] = code of the element values[i] (device arrays, n entries).  A value
 * >= q yields code 0 and sets the field's error flag (gfp_gfq_check). */
GFP_API gfp_status gfp_gfq_to_log(gfp_gfq *fq, uint64_t n, const uint32_t *values, uint16_t *codes,
                                  void *stream);
/* values[i] = element value of codes[i].  A code > q-1 yields 0 and sets the
 * error flag. */
GFP_API gfp_status gfp_gfq_from_log(gfp_gfq *fq, uint64_t n, const uint16_t *codes, uint32_t *values,
                                    void *stream);

/* *out (device) = code of sum_{i<n} x_i y_i in GF(q), x and y device arrays of
 * n codes in [0, q-1]; 16-byte aligned x and y take the vectorised path.
 * Each product is a code addition (Section 2.4); the sum is formed from
 * element values for prime fields (integers, reduced mod p once),
 * characteristic 2 (XOR) and odd characteristic with k > 1 and q <= 256 (a
 * table of the field's value addition), and by Zech additions for larger odd
 * characteristic extensions.  n = 0 gives code 0.  Codes above q-1 are outside the contract: the
 * result is then unspecified (no out-of-bounds access occurs). */
GFP_API gfp_status gfp_gfq_dot(gfp_gfq *fq, uint64_t n, const uint16_t *x, const uint16_t *y, uint16_t *out,
                               void *stream);

/* Synchronise the field's device; GFP_ERR_RANGE (and clear the flag) if a
 * conversion met an out-of-range value or code since the last check. */
GFP_API gfp_status gfp_gfq_check(gfp_gfq *fq);

/* ---- synthetic inputs (device generator) ---- */

/* out[i] = word(seed, stream_id, offset + i) mod p for 0 <= i < n, where
 * word is the counter-based SplitMix64 sequence
 *   key = mix64(seed + G*(stream_id+1)),  word(i) = mix64(key + G*(i+1)),
 *   G = 0x9E3779B97F4A7C15  (arithmetic modulo 2^64).
 * Input synthesis only (the benchmark and service generate operands with
 * it); it is not part of the dot-product method. */
GFP_API gfp_status gfp_fill_uniform(uint32_t p, uint64_t seed, uint64_t stream_id,
                                    uint64_t offset, uint64_t n, uint32_t *out, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* GFPDOT_H */
