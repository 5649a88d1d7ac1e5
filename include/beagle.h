/*
 * beagle.h -- C ABI of the GB300 population-scoring library (libbeagle.so).
 *
 * What the library computes follows the Beagle tutorial (arXiv 2607.06731), cited by section
 * title:
 *   - A genome is a GCL program in reverse Polish notation run on a value stack (the GCL
 *     section and Table 3). Unary ops replace the top value; binary ops pop the top b and the
 *     value below it a and push a (op) b (SUB is a - b, DIV is a / b, POW is a ^ b).
 *   - The GPU evaluates each program on every fitness case and returns one aggregated
 *     fitness per program; the CPU keeps the genetic operators ("Dividing Tasks Between CPU
 *     and GPU"). Genomes go to the device once per generation and datasets stay resident.
 *   - Fitness: the mean squared error and 1 - r^2, r being the Pearson correlation of Eq. 1
 *     between outputs and targets, squared ("Fitness Functions"); and the paper's own fitness
 *     functions, Eqs. 2 and 5 (beagle_score_fit).
 *
 * Readings of points the paper leaves open (the paper's own DIV, LN, SQRT are unprotected):
 *   pdiv(a, b) = a / b if |b| > 1e-3, else 1;  plog(a) = ln|a| if |a| > 1e-3, else 0;
 *   psqrt(a) = sqrt|a|; the rest of Table 3 is unprotected. A program is INVALID when any
 *   value it produces is non-finite or has |v| > 1e30; an invalid program scores +inf for
 *   both fitness values. When a program's output is the same on every case, r is undefined
 *   and 1 - r^2 is reported as 1 (flag DEGENERATE). Thresholds are compared in the
 *   arithmetic's own precision (the fp32 value nearest 1e30 and 1e-3 on the FP32 path).
 *
 * Conventions for every call:
 *   - Return value: BEAGLE_OK (0) or a negative BEAGLE_ERR_* code; beagle_last_error()
 *     returns a message for the calling thread's last failure.
 *   - "device" pointers are CUDA device (or managed) memory of the current device; "host"
 *     pointers are ordinary or pinned host memory. The caller owns every buffer it passes;
 *     the library owns resident datasets (until released) and its serving state.
 *   - A stream argument is a cudaStream_t cast to void* (NULL = the legacy default stream).
 *     Scoring calls are asynchronous on that stream unless stated otherwise: results are
 *     valid once the stream reaches the call's position.
 *   - Calls are thread-safe.
 */
#ifndef BEAGLE_H
#define BEAGLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t beagle_status;

#define BEAGLE_OK             0
#define BEAGLE_ERR_ARG       -1   /* null pointer, bad size, unknown precision */
#define BEAGLE_ERR_PROGRAM   -2   /* a program failed the structural check */
#define BEAGLE_ERR_DATASET   -3   /* unknown dataset id, or dataset values rejected */
#define BEAGLE_ERR_OOM       -4   /* device memory or serving budget exhausted */
#define BEAGLE_ERR_CUDA      -5   /* a CUDA runtime call failed */
#define BEAGLE_ERR_TIMEOUT   -6   /* a bounded wait ran out */
#define BEAGLE_ERR_BUSY      -7   /* resource still in use */
#define BEAGLE_ERR_LIMIT     -8   /* a size above a documented maximum */

/* ---- Wire format: one byte per token (Table 3 op names; protected forms as above) ---- */
#define BEAGLE_OP_CONST   0   /* push consts[token] */
#define BEAGLE_OP_ADD     1
#define BEAGLE_OP_SUB     2   /* second - top */
#define BEAGLE_OP_MUL     3
#define BEAGLE_OP_PDIV    4   /* second / top, protected */
#define BEAGLE_OP_SIN     5
#define BEAGLE_OP_COS     6
#define BEAGLE_OP_EXP     7
#define BEAGLE_OP_PLOG    8
#define BEAGLE_OP_PSQRT   9
#define BEAGLE_OP_SQUARE 10
#define BEAGLE_OP_DUP    11   /* push a copy of the top */
#define BEAGLE_OP_SWAP   12   /* exchange the top two */
#define BEAGLE_OP_DEL    13   /* pop the top */
/* The rest of Table 3, unprotected: a value outside an operator's domain is NaN (invalid). */
#define BEAGLE_OP_POW    14   /* second ^ top */
#define BEAGLE_OP_SIGN   15   /* -top ("changes the sign") */
#define BEAGLE_OP_CUBE   16   /* (top top) top, each product rounded */
#define BEAGLE_OP_CBRT   17
#define BEAGLE_OP_TAN    18
#define BEAGLE_OP_ASIN   19   /* ARCSIN */
#define BEAGLE_OP_ACOS   20   /* ARCCOS */
#define BEAGLE_OP_ATAN   21   /* ARCTAN */
#define BEAGLE_OP_TANH   22
#define BEAGLE_OP_LOAD0  32   /* BEAGLE_OP_LOAD0 + k pushes input x_k (k zero-based) */
/* Table 3's variables: COPY @k copies the top into variable k (the stack is unchanged);
 * PASTE @k pushes it and empties the variable. Each COPY @k must be followed by exactly one
 * PASTE @k before the next COPY @k, and every variable must be empty at the end. On the GPU a
 * live variable k occupies a stack slot: the stack depth plus (highest live k + 1) must not
 * exceed the stack limit. */
#define BEAGLE_OP_COPY0  64   /* BEAGLE_OP_COPY0 + k, k < BEAGLE_MAX_REGS */
#define BEAGLE_OP_PASTE0 80   /* BEAGLE_OP_PASTE0 + k */
#define BEAGLE_MAX_REGS   8

#define BEAGLE_MAX_VARS    16    /* inputs per dataset (d) */
#define BEAGLE_MAX_DEPTH   32    /* values on the stack: the paper's StackSize (the GCL
                                    section); programs deeper than 16 run in a second pass */
#define BEAGLE_MAX_LENGTH  256   /* tokens per program */

/* ---- Result flags ---- */
#define BEAGLE_FLAG_INVALID     1u  /* a value was non-finite or |v| > 1e30: both fitnesses +inf */
#define BEAGLE_FLAG_DEGENERATE  2u  /* output identical on every case: one_minus_r2 = 1 */
#define BEAGLE_FLAG_MALFORMED   4u  /* failed the structural check on the device: both +inf */
#define BEAGLE_FLAG_TIMEOUT     8u  /* a bounded device wait ran out: result not computed */
/* Every wait inside the scoring kernels is bounded (4 s by default; the environment variable
 * BEAGLE_WAIT_LIMIT_US, read at each launch, sets another bound). A wait that runs out ends
 * the launch early and every result of that launch carries BEAGLE_FLAG_TIMEOUT with NaN
 * fitness; the device context stays usable. BEAGLE_TEST_STALL=1 is a test hook that makes
 * the waits run out (the producer warp publishes no work). */

/* ---- Precision of program arithmetic ---- */
#define BEAGLE_FP32_COMPENSATED 0   /* fp32 ops; fp32 compensated sums; fp64 cross-tile merge */
#define BEAGLE_FP64             1   /* every op and sum in fp64 (plain sums) */

/* One aggregated fitness per program ("Dividing Tasks Between CPU and GPU"), 24 bytes. */
typedef struct beagle_fitness {
    double mse;           /* (1/N) sum_i (f(x_i) - y_i)^2 */
    double one_minus_r2;  /* 1 - r^2, r from Eq. 1 */
    uint32_t flags;       /* BEAGLE_FLAG_* */
    uint32_t reserved;
} beagle_fitness;

/*
 * Upload a dataset and keep it resident on the current device ("Dividing Tasks Between CPU
 * and GPU": data is sent once; the MLSetup mandatory overrides: one (inputs, output) point
 * per fitness case).
 *   X      [d][N] fp32, row k holds input x_k of every case (column-major by case).
 *   y      [N] fp32 targets.
 *   N >= 2, 1 <= d <= BEAGLE_MAX_VARS. inputs_on_device: 0 = host pointers, 1 = device.
 * Every value must be finite with |v| <= 1e30, and y must not be constant, else
 * BEAGLE_ERR_DATASET. The library computes the target mean and sum of squares in fp64 and
 * stores X, y and y - mean(y) in its own padded layout. The call returns once the data is
 * on the device. *dataset_id receives a positive id.
 */
beagle_status beagle_upload_dataset(const float *X, const float *y, int64_t N, int32_t d,
                                    int32_t inputs_on_device, void *stream,
                                    int32_t *dataset_id);

/*
 * beagle_upload_dataset with flags. BEAGLE_DATASET_INVALID_TARGETS: y may hold invalid
 * targets (NaN, +-inf, |y| > 1e30), as the paper allows ("Fitness Functions": invalid values in
 * the dataset are matched, not removed); X must still be valid. Such a dataset is scored with
 * beagle_score_fit only (beagle_score returns BEAGLE_ERR_DATASET); its stored mean and sum of
 * squares are over the valid targets, and it may hold a constant or empty set of valid targets.
 */
#define BEAGLE_DATASET_INVALID_TARGETS 1u
beagle_status beagle_upload_dataset_ex(const float *X, const float *y, int64_t N, int32_t d,
                                       int32_t inputs_on_device, uint32_t flags, void *stream,
                                       int32_t *dataset_id);

/* Release a dataset. Work already enqueued that uses it completes first (the call
 * synchronises the device). BEAGLE_ERR_DATASET for an unknown id, BEAGLE_ERR_BUSY while a
 * serving run still holds it. */
beagle_status beagle_release_dataset(int32_t dataset_id);

/* N, d, mean of y and sum_i (y_i - mean)^2 of a resident dataset (any pointer may be NULL). */
beagle_status beagle_dataset_info(int32_t dataset_id, int64_t *N, int32_t *d, double *ybar,
                                  double *syy);

/*
 * Host-side structural check of a population in the wire format (the GCL section): every
 * token finds its operands, the stack never holds more than max_depth values, inputs exist,
 * COPY and PASTE pair up, exactly one value remains, and 1 <= length <= BEAGLE_MAX_LENGTH. All
 * pointers are host pointers. Returns BEAGLE_ERR_PROGRAM and the index of the first bad
 * program in *first_bad (if not NULL), else BEAGLE_OK and -1. (max_depth: the GPU's depth limit
 * and the paper's StackSize differ; the index is 64-bit like P.)
 */
beagle_status beagle_validate_programs(const uint8_t *programs, const int64_t *offsets,
                                       const int32_t *lengths, int64_t P, int32_t d,
                                       int32_t max_depth, int64_t *first_bad);

/*
 * beagle_validate_programs with an operator whitelist ("Subclassing MLSetup - optional
 * overrides": GetAllowedOperations restricts the operators a run may use). allowed lists
 * n_allowed opcodes (host array); BEAGLE_OP_LOAD0 admits every LOAD, BEAGLE_OP_COPY0 every
 * COPY and PASTE. n_allowed = 0 admits every operator. A program using another operator fails
 * the check like a malformed one.
 */
beagle_status beagle_validate_programs_ex(const uint8_t *programs, const int64_t *offsets,
                                          const int32_t *lengths, int64_t P, int32_t d,
                                          int32_t max_depth, const uint8_t *allowed,
                                          int32_t n_allowed, int64_t *first_bad);

/*
 * Score a population against a resident dataset ("Dividing Tasks Between CPU and GPU"). All
 * array pointers are device pointers:
 *   programs  concatenated tokens; program p is programs[offsets[p] .. offsets[p]+lengths[p])
 *   offsets   [P] int64, lengths [P] int32
 *   consts    token-aligned fp32: consts[offsets[p] + j] is read when token j is CONST
 *   fitness_out [P] beagle_fitness, written by the call
 * precision is BEAGLE_FP32_COMPENSATED or BEAGLE_FP64. Programs are not checked on the
 * host; a program that fails the structural check (or is deeper than BEAGLE_MAX_DEPTH or
 * longer than BEAGLE_MAX_LENGTH) gets BEAGLE_FLAG_MALFORMED instead of a fitness.
 * Asynchronous on stream; the call uses stream-ordered scratch memory that it frees itself.
 * Results are deterministic: the same program and dataset give the same bits in any
 * population and any batch. A program found invalid on one case is not evaluated on its
 * remaining cases (see beagle_set_invalid_early_exit): the results are the same bits, the
 * work done depends on how many programs are invalid.
 */
beagle_status beagle_score(const uint8_t *programs, const int64_t *offsets,
                           const int32_t *lengths, const float *consts, int64_t P,
                           int32_t dataset_id, beagle_fitness *fitness_out,
                           int32_t precision, void *stream);

/*
 * The paper's own fitness functions ("Fitness Functions" in the framework overview, Eqs. 1-2;
 * the configuration section's fitness functions, Eqs. 3-5; "Creating Custom Fit Functions":
 * the IFitFunc interface, selected here per call by kind). Each fitness case is judged on its
 * own: a case whose evaluation produced an invalid value (non-finite or |v| > 1e30, the rule
 * above applied per case) is an invalid output; a target that is non-finite or above 1e30 is an
 * invalid target (datasets uploaded with BEAGLE_DATASET_INVALID_TARGETS may hold them).
 *   BEAGLE_FIT_CORRELATION  CorrelationFitFunc: r of Eq. 1 over the pairs where output and
 *        target are both valid, then Eq. 2: score = M r^4 (N - (c1 + c2)) - M (c1 - c2), c1 =
 *        pairs with exactly one invalid member, c2 = pairs with both invalid. r := 0 when it is
 *        undefined (no valid pair, or outputs or targets constant over the valid pairs; flag
 *        DEGENERATE).
 *   BEAGLE_FIT_STD, _STD_SQUARE, _STD_CUBE, _STD_HYPER  Eq. 5 per case, summed (integer):
 *        q = min(|f|,|y|) / max(|f|,|y|); M when both are 0; round(M q^k - M/11) when f and y
 *        have opposite signs; round(M q^k) otherwise; k = 1, 2, 3, 8 (reading: the variants'
 *        power applies to the ratio, so the best case still earns M). Pairs with an invalid
 *        member (FitFunctionIfInvalid, reading): +M when both are invalid, -M when one is.
 *        round() is to nearest, ties to even, in the path's precision (fp32 on the
 *        FP32-compensated path).
 *   BEAGLE_FIT_VALIDATE  the interactive V command's test ("Interacting with Beagle During a
 *        Run"): a case passes when output and target are valid and |f - y| <= 0.001 |y|
 *        (decided in fp64); score = passing cases; flag PERFECT when all N pass.
 * asr = score / (M N) (the average score ratio of the sample run output; score / N for
 * VALIDATE). taxed_score = score - tax_per_token * length: the parsimony pressure of
 * ScriptLengthTaxRateInternal; tax_per_token < 0 selects its default rate M N / 85 (a
 * perfect program of length 85 is taxed to zero). A malformed program scores -inf.
 */
#define BEAGLE_FIT_MSE_R2        0   /* beagle_score's MSE and 1 - r^2 (not for beagle_score_fit) */
#define BEAGLE_FIT_CORRELATION   1
#define BEAGLE_FIT_STD           2
#define BEAGLE_FIT_STD_SQUARE    3
#define BEAGLE_FIT_STD_CUBE      4
#define BEAGLE_FIT_STD_HYPER     5
#define BEAGLE_FIT_VALIDATE      6
#define BEAGLE_FLAG_PERFECT     16u  /* VALIDATE: every case passed */

typedef struct beagle_fit_config {
    int32_t kind;            /* BEAGLE_FIT_* (not MSE_R2) */
    int32_t max_score;       /* M, 1 .. 2^22 (the paper's sample run: 10,000 per case) */
    double tax_per_token;    /* length tax; < 0: M N / 85 */
} beagle_fit_config;

typedef struct beagle_fit_result {   /* 56 bytes */
    double score;            /* Eq. 2 score, sum of Eq. 5 rewards, or passing cases */
    double asr;              /* score / (M N) (VALIDATE: score / N) */
    double r2;               /* CORRELATION: r^2 over the valid pairs; else 0 */
    double taxed_score;      /* score - tax_per_token * length */
    int64_t c1;              /* pairs with exactly one invalid member */
    int64_t c2;              /* pairs with both members invalid */
    uint32_t flags;          /* BEAGLE_FLAG_DEGENERATE / MALFORMED / TIMEOUT / PERFECT */
    uint32_t reserved;
} beagle_fit_result;

/*
 * Score a population with one of the paper's fitness functions. Arguments as for beagle_score
 * (device pointers), plus cfg (host pointer) and fit_out, a device array of P
 * beagle_fit_result. Works on any dataset, including ones uploaded with
 * BEAGLE_DATASET_INVALID_TARGETS. Asynchronous on stream.
 */
beagle_status beagle_score_fit(const uint8_t *programs, const int64_t *offsets,
                               const int32_t *lengths, const float *consts, int64_t P,
                               int32_t dataset_id, const beagle_fit_config *cfg,
                               beagle_fit_result *fit_out, int32_t precision, void *stream);

/*
 * Run each program on every case and keep the outputs (the paper's ExecuteGenome utility,
 * "Useful Utilities"): same arguments and results as beagle_score, plus outputs, a device array of
 * P x N values (row p holds program p's output on every case), fp32 for
 * BEAGLE_FP32_COMPENSATED and fp64 for BEAGLE_FP64. Outputs of malformed programs are not
 * written. Asynchronous on stream.
 */
beagle_status beagle_eval(const uint8_t *programs, const int64_t *offsets,
                          const int32_t *lengths, const float *consts, int64_t P,
                          int32_t dataset_id, void *outputs, beagle_fitness *fitness_out,
                          int32_t precision, void *stream);

/*
 * Same as beagle_score with HOST arrays (pinned memory gives the fastest copies): copies the
 * inputs to the device, scores, copies the fitness back and synchronises the stream before
 * returning. consts_len is the number of floats in consts (the total token count).
 */
beagle_status beagle_score_host(const uint8_t *programs, const int64_t *offsets,
                                const int32_t *lengths, const float *consts, int64_t P,
                                int64_t n_tokens, int32_t dataset_id,
                                beagle_fitness *fitness_out, int32_t precision, void *stream);

/*
 * beagle_score_static: beagle_score that allocates no device memory. The paper has no
 * counterpart; this is for callers that cannot allocate while they score -- a loop that must
 * never block on the device (cudaMalloc and cudaFree may synchronise it), a process that
 * reserves its whole device-memory budget up front, or code that runs while another
 * component owns the allocator. Same arguments, results and asynchrony as beagle_score, with
 * a fixed launch shape: tiles of 512 cases, 4 cases per lane on the FP32 path, programs in
 * the caller's order. beagle_set_launch_config and the autotuner's choices are ignored; with
 * the automatic shape, beagle_score gives the same bits. Its scratch (a 256-byte header plus
 * 44 bytes per program and tile of 512 cases) lives in one fixed array of
 * BEAGLE_STATIC_SCRATCH_BYTES inside the library, held on every device that loads the library
 * until the process exits; a call that needs more (or P >= 2^31) fails with BEAGLE_ERR_LIMIT
 * before enqueuing anything. The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current, so make that first call before any stream
 * capture. All calls share the one array and each zeroes its header on its stream: calls
 * whose work overlaps on the GPU (other streams or threads) race, so the caller must
 * serialise them.
 */
#define BEAGLE_STATIC_SCRATCH_BYTES (32u << 20)
beagle_status beagle_score_static(const uint8_t *programs, const int64_t *offsets,
                                  const int32_t *lengths, const float *consts, int64_t P,
                                  int32_t dataset_id, beagle_fitness *fitness_out,
                                  int32_t precision, void *stream);

/*
 * Serving (continuous batching on the device). Many concurrent evolutionary runs each submit one
 * generation at a time -- a population in the wire format in HOST memory, scored against the
 * run's resident dataset ("Dividing Tasks Between CPU and GPU": genomes go to the device once
 * per generation, one fitness per genome comes back). The server copies each request into
 * pinned staging recycled from a pool (the dead pool of "CPU Optimizations"), admits queued
 * requests in arrival order while their device bytes (inputs and scoring scratch) fit
 * hbm_budget_bytes ("Hardware Optimized": batches fit device memory), and appends each as a
 * job to the work queue of ONE persistent kernel that keeps running while requests arrive:
 * a request admitted while others are on the GPU is scored between their work items, so a
 * small request does not wait for a large one, and the kernel writes every program's fitness
 * straight into the request's pinned output as soon as the program's last tile is done. The
 * kernel exits when the server has no work and is launched again when work arrives. A
 * request's results are the same bits alone, in any mix, and through beagle_score (tiles of
 * 512 cases). Datasets are held resident while a request uses them; datasets with invalid
 * targets are refused (BEAGLE_ERR_DATASET).
 *   submit   non-blocking; returns a ticket. A request larger than the budget fails with
 *            BEAGLE_ERR_OOM when it reaches the head of the queue.
 *   poll     *done = 1 and the results copied to host_out (P records) once finished; the
 *            ticket is then retired.
 *   wait     blocks until finished (timeout_us < 0: no limit); BEAGLE_ERR_TIMEOUT if not done
 *            in time (the ticket stays valid); on success retires the ticket.
 *   timing   for a finished request (retired or not; the last 65,536 are kept): time queued
 *            before admission and submit-to-result latency (microseconds, host clock), and
 *            the device's %globaltimer stamps (ns) when its first work item was claimed and
 *            when its last unit finished.
 *   stats    counters, node evaluations per second between the first submission and the last
 *            completion, and p50 / p99 / max latency (submit to result) of completed requests;
 *            inflight_launches counts admitted requests not yet finished and launches the
 *            persistent kernel's launches.
 *   destroy  finishes every queued and running request, then frees the server.
 */
typedef struct beagle_serve_config {
    int64_t hbm_budget_bytes;   /* 0: half of the free device memory at creation */
    int32_t max_inflight;       /* unused (0-8 accepted): the queue feeds one running kernel */
    int32_t max_batch_jobs;     /* requests admitted per round of the serving thread; 0: 64 */
    int32_t precision;          /* BEAGLE_FP32_COMPENSATED or BEAGLE_FP64 */
    int32_t reserved;
} beagle_serve_config;

typedef struct beagle_request {
    const uint8_t *programs;    /* host, as for beagle_score */
    const int64_t *offsets;
    const int32_t *lengths;
    const float *consts;
    int64_t P;
    int64_t n_tokens;           /* total tokens (length of programs and consts) */
    int32_t dataset_id;
    int32_t reserved;
} beagle_request;

typedef struct beagle_serve_counters {
    int64_t submitted, completed, rejected, queued, inflight_launches, launches;
    int64_t node_evals, bytes_in_use, peak_bytes, budget_bytes;
    double gpops, p50_us, p99_us, max_us;
} beagle_serve_counters;

typedef struct beagle_server beagle_server;
beagle_status beagle_serve_create(const beagle_serve_config *cfg, beagle_server **server);
beagle_status beagle_serve_submit(beagle_server *server, const beagle_request *req,
                                  uint64_t *ticket);
beagle_status beagle_serve_poll(beagle_server *server, uint64_t ticket,
                                beagle_fitness *host_out, int32_t *done);
beagle_status beagle_serve_wait(beagle_server *server, uint64_t ticket,
                                beagle_fitness *host_out, int64_t timeout_us);
beagle_status beagle_serve_timing(beagle_server *server, uint64_t ticket, double *queue_us,
                                  double *latency_us, uint64_t *gpu_start_ns,
                                  uint64_t *gpu_end_ns);
beagle_status beagle_serve_stats(beagle_server *server, beagle_serve_counters *stats);
beagle_status beagle_serve_destroy(beagle_server *server);

/*
 * Launch shape of the scoring kernel (no counterpart in the paper). All fields 0 = chosen
 * automatically. cases_per_lane: fitness cases each lane evaluates per pass on the FP32 path
 * (2, 4 or 8); tile: cases per staged tile (256 or 512); group: programs per work item;
 * warps: upper bound on consumer warps per CTA (1-31); grid: CTAs (default one per SM);
 * keep_order: 0 automatic -- on launches of at least 2^24 program-cases (P x N summed) the
 * programs run in the length-bucketed order (longest first), each packed once for the call
 * by a packing kernel that also folds their constant subexpressions (FP32 path); smaller
 * launches keep the caller's order and pack per work item; 1 always the caller's order (no
 * packing kernel); 2 always the length-bucketed order with the packing kernel.
 * beagle_set_launch_config sets the process-wide configuration used by every later scoring
 * call (NULL restores automatic); results do not depend on it beyond the rounding of sums
 * over differently sized tiles (tile) -- with a fixed tile they are bit-identical.
 */
typedef struct beagle_launch_config {
    int32_t cases_per_lane;
    int32_t tile;
    int32_t group;
    int32_t warps;
    int32_t grid;
    int32_t keep_order;
} beagle_launch_config;
beagle_status beagle_set_launch_config(const beagle_launch_config *cfg);
beagle_status beagle_get_launch_config(beagle_launch_config *cfg);

/*
 * Measurement support (not part of scoring).
 * beagle_measure_op_rates: throughput of each operator on the current device, in operator
 * evaluations per second, written to rates[opcode] for the ten arithmetic opcodes (other
 * entries 0). Each evaluation includes the validity check the scoring kernels do; eight
 * independent chains per thread at full occupancy, so the figure is what straight-line
 * compiled code reaches. Synchronous; runs about seconds_hint seconds. n_rates >= 11.
 * beagle_kernel_timing: enable (1) or disable (0) CUDA-event timing around every scoring
 * kernel launch. beagle_kernel_time: synchronises on the recorded events, returns the summed
 * kernel time (ms) and the number of launches since the previous query, and clears them.
 */
beagle_status beagle_measure_op_rates(double *rates, int32_t n_rates, double seconds_hint,
                                      void *stream);

/*
 * Early exit on invalid programs (MSE / 1 - r^2 scoring). A program with one invalid value on
 * one fitness case is invalid (the validity rule above), whatever its other cases give. By
 * default the scoring kernels use that: a case tile stops at the first 128-case pass (256 at 8
 * cases per lane) that meets an invalid case, and once some tile has found a program invalid
 * its later tiles are not run. The results are the same bits either way; the work done, and
 * so the time, depends on how many programs are invalid and where. enable = 0 turns this off
 * (every case of every program runs) for the calls that follow, 1 turns it back on.
 * The serving loop takes the setting when a request is submitted. beagle_score_fit,
 * beagle_eval and beagle_score_static always run every case. Process-wide setting.
 *
 * beagle_count_cases: while cases_run (a device array of P int64) is set, every following
 * single-population scoring call with exactly P programs adds to cases_run[p] the fitness
 * cases it ran for program p (N with the early exit off; fewer for invalid programs with it
 * on, and 0 for malformed ones). Costs one atomic add per program and tile. NULL turns it off.
 * BEAGLE_ERR_ARG for a non-null array with P <= 0.
 */
beagle_status beagle_set_invalid_early_exit(int32_t enable);
beagle_status beagle_count_cases(int64_t *cases_run, int64_t P);
beagle_status beagle_kernel_timing(int32_t enable);
beagle_status beagle_kernel_time(double *total_ms, int64_t *launches);

/*
 * Ragged batches (the paper batches populations to fit device memory, "Hardware Optimized";
 * here many (population, dataset) pairs share one persistent launch). A job is one
 * beagle_score call's
 * arguments (device pointers, as for beagle_score). Jobs may use different datasets, sizes
 * and program lengths; programs are processed in a length-bucketed order (longest first).
 * Results are the same bits as scoring each job alone.
 */
typedef struct beagle_job {
    const uint8_t *programs;
    const int64_t *offsets;
    const int32_t *lengths;
    const float *consts;
    int64_t P;
    int32_t dataset_id;
    int32_t reserved;
    beagle_fitness *fitness_out;
} beagle_job;

/* Score n_jobs jobs (host array of job descriptors) on stream. Jobs are grouped into
 * persistent launches of at most 64 jobs, in ascending order of input count d; a launch is
 * cut where d changes once it holds 2^24 program-cases (sum of P x N), since its shared memory
 * is sized by its widest dataset. Asynchronous. */
beagle_status beagle_score_batch(const beagle_job *jobs, int32_t n_jobs, int32_t precision,
                                 void *stream);

/*
 * A batch captured once into a CUDA graph and replayed: for an evolutionary loop that refills
 * the same device buffers every generation. The plan keeps the job descriptors as given
 * (same pointers, same sizes) and holds its datasets resident (beagle_release_dataset returns
 * BEAGLE_ERR_BUSY until the plan is destroyed). beagle_batch_plan_launch enqueues one replay
 * on stream (asynchronous).
 */
typedef struct beagle_batch_plan beagle_batch_plan;
beagle_status beagle_batch_plan_create(const beagle_job *jobs, int32_t n_jobs,
                                       int32_t precision, beagle_batch_plan **plan);
beagle_status beagle_batch_plan_launch(beagle_batch_plan *plan, void *stream);
beagle_status beagle_batch_plan_destroy(beagle_batch_plan *plan);

/*
 * Autotuner: time candidate launch shapes (cases per lane 2/4/8 x tile 512/256 x programs per
 * item) on the given jobs (it runs them, overwriting fitness_out) and remember the fastest for
 * this shape class (precision, d, floor(log2 of the largest N)); later calls of that class
 * with an automatic configuration use it. max_trials <= 0 tries all candidates. Synchronous.
 * best / best_ms (may be NULL) receive the chosen shape and its time per call.
 * beagle_autotune_clear forgets every tuned entry.
 */
beagle_status beagle_autotune(const beagle_job *jobs, int32_t n_jobs, int32_t precision,
                              int32_t max_trials, void *stream, beagle_launch_config *best,
                              double *best_ms);
beagle_status beagle_autotune_clear(void);

/*
 * Monte-Carlo ranking ("Monte-Carlo Ranking" in the overview; Table 2): the host side of a
 * generation ranks the population without sorting it. A sample of 100 individuals (indices in
 * sample, device [100], drawn by the caller) estimates the percentiles: its keys sorted
 * ascending give thresholds t_q = the q-th order statistic, q = 10, 20, ..., 90. One pass then
 * gives individual p its group g = the number of thresholds with key >= t_q (0-9; 9 is the
 * ">= 90" row) and its children: floor(E_g) + (u[p] < E_g - floor(E_g)), E_g = Table 2's
 * expected children (0.01, 0.03, 0.06, 0.15, 0.25, 0.5, 1, 1.5, 2.5, 4 for g = 0..9) and
 * u[p] a uniform number in [0, 1) (device [P], drawn by the caller).
 *   key               device pointer to the first record's key field, e.g. &fitness[0].mse
 *                     or &fit_results[0].taxed_score; key_stride_bytes apart (24 / 56)
 *   negate            1: lower values are better (MSE, 1 - r^2): the key is -value
 * Higher keys are better; a NaN key ranks below every other (group 0), and a sample index
 * outside [0, P) reads as NaN. Outputs: group_out [P] uint8, children_out [P] int32, device.
 * n_sample must be 100. Asynchronous on stream.
 */
beagle_status beagle_rank(const double *key, int64_t key_stride_bytes, int32_t negate, int64_t P,
                          const int64_t *sample, int32_t n_sample, const float *u,
                          uint8_t *group_out, int32_t *children_out, void *stream);

/*
 * Population sharding by cost ("Hardware Optimized": the work of a generation is spread over
 * every GPU of the machine): split programs [0, P) into n_shards contiguous ranges of nearly
 * equal cost, a program's cost being its length (every program runs on the same cases).
 * bounds_out[0..n_shards] (host) receives the range edges: shard k is [bounds[k],
 * bounds[k+1]). Each shard's cost is within the longest program's length of total / n_shards.
 * lengths is a host array. Each GPU then scores its shard with its own copy of the dataset; no
 * collective is needed until the fitness records are gathered.
 */
beagle_status beagle_shard_by_cost(const int32_t *lengths, int64_t P, int32_t n_shards,
                                   int64_t *bounds_out);

/* Message of the calling thread's most recent failure ("" if none). */
const char *beagle_last_error(void);

/* Library version, major * 10000 + minor * 100 + patch. */
int32_t beagle_version(void);

#ifdef __cplusplus
}
#endif

#endif /* BEAGLE_H */
