/*
 * ltl.h -- C ABI of the GB300 enumerative LTL learner (sm_103a).
 *
 * The library learns a minimal LTL formula separating positive from negative
 * finite traces ("LTL learning on GPUs", arXiv 2402.12373): bottom-up,
 * size-by-size enumeration over !, &, |, X, F, G and U (Section 3, the
 * `enum` / `handleOp` / check-and-cache steps), each formula represented by
 * its characteristic matrix of bit-vectors (Section 4), F, G and U computed
 * branch-free -- by default as an integer carry chain over the bit-reversed
 * trace, or (ltl_opts.propagation) by the paper's exponential propagation in
 * O(log n) shifts (Section 4, Appendix B), with identical results -- and
 * every candidate deduplicated exactly by observational equivalence modulo the
 * suffixes of the input traces (Section 5 with an exact, not relaxed, check).
 *
 * Conventions shared by every entry point
 *  - Traces.  A trace is a finite string over the powerset of the alphabet
 *    {p0 .. p(n_props-1)}, n_props <= 32 (Section 2).  Position i of a trace
 *    is one uint32: bit p set iff p holds there.  A trace set is `letters`
 *    (all positions of all traces, concatenated) plus `offsets` (n_traces+1
 *    non-decreasing prefix offsets, offsets[0] == 0).  Empty traces are legal
 *    and satisfy no formula (every formula is false at i >= |tr|, Section 2).
 *  - Characteristic sequences.  Bit t of word w of a trace's sequence is
 *    position 64*w + t (least significant bit = position 0); positions at or
 *    beyond the trace's length are always 0.  A trace of length L uses
 *    ceil(L / 64) words.
 *  - Formula text.  Fully parenthesised infix: `p3`, `!f`, `X f`, `F f`,
 *    `G f`, `(f & g)`, `(f | g)`, `(f U g)`; extra parentheses `(f)` and
 *    whitespace are accepted on input.
 *  - Connective masks: LTL_NOT | LTL_AND | ... ; LTL_ALL selects all seven.
 *  - Ownership.  The caller owns every buffer it passes; the library copies
 *    what it needs and never keeps a caller pointer past the call (except
 *    `ltl_opts.workspace`, which a context uses until it is destroyed).
 *  - Errors.  No call returns silently: a CUDA error gives LTL_ERR_CUDA and
 *    leaves the context usable; LTL_ERR_BUFSIZE reports a too-small output
 *    buffer (the required size is written where stated).
 *  - Threads.  A context may be used by one host thread at a time.
 *  - Process-wide state.  The library keeps, for the life of the process,
 *    page-locked host blocks that contexts, batches and servers release (the
 *    next one reuses them instead of pinning memory again), the launch
 *    properties of its kernels per device, and a few idle host threads for
 *    copying large submitted inputs.  Do not reset a device
 *    (cudaDeviceReset) while the library is loaded: the cached blocks and
 *    properties belong to the device's context.
 */
#ifndef LTL_GB300_H
#define LTL_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    LTL_OK = 0,            /* a separating formula was found                  */
    LTL_NOT_FOUND = 1,     /* none up to max_size (or P and N intersect)      */
    LTL_CAP_REACHED = 2,   /* the language cache filled its memory first      */
    LTL_ERR_INVALID = -1,  /* bad argument, malformed traces or formula       */
    LTL_ERR_CUDA = -2,     /* a CUDA call failed (message: ltl_last_error)    */
    LTL_ERR_OOM = -3,      /* workspace / allocator could not supply memory   */
    LTL_ERR_TIMEOUT = -4,  /* a bounded device wait ran out (see spin_limit)  */
    LTL_ERR_BUFSIZE = -5   /* output buffer too small                         */
} ltl_status;

enum {
    LTL_NOT = 1, LTL_AND = 2, LTL_OR = 4, LTL_X = 8,
    LTL_F = 16, LTL_G = 32, LTL_U = 64, LTL_ALL = 127,
    /* restriction flag in the same mask: negation normal form, i.e. negation
     * applied to atoms only (Section 2; used for the comparisons of Section 7) */
    LTL_NNF = 256
};

/* stop_on_solution values */
enum {
    LTL_STOP_NONE = 0,     /* enumerate every level up to max_size           */
    LTL_STOP_FIRST = 1,    /* return at the first separating candidate       */
    LTL_STOP_LEVEL = 2     /* finish the level where a separator was found   */
};

/* ruc values: the cache admission policy (relaxed uniqueness checks, Section 5).
 * A candidate enters the cache only if its admission key is new.
 *   LTL_RUC_EXACT  key = the whole characteristic matrix (fingerprint, then a
 *                  full compare): every distinct matrix is kept.
 *   LTL_RUC_HASH   key = 63 bits of a hash of the matrix, no compare: a key
 *                  collision drops a matrix (false positive, never a false
 *                  negative).  A matrix of at most 63 bits in all (the sum of
 *                  the trace lengths; traces x max_len for device-resident
 *                  traces) is checked exactly instead.
 *   LTL_RUC_FKP    key = the first b positions of every trace concatenated in
 *                  trace order, b = max(1, 63 / n_traces), truncated to 63 bits
 *                  (the "first k percent" map of Section 7).
 * Relaxed modes stay sound (every returned formula separates) but may miss the
 * minimal size, and results may vary between runs: which of two colliding
 * matrices is kept depends on timing. */
enum {
    LTL_RUC_EXACT = 0,
    LTL_RUC_HASH = 1,
    LTL_RUC_FKP = 2
};

typedef struct {
    const uint32_t *letters;   /* concatenated positions (host memory)        */
    const uint64_t *offsets;   /* n_traces + 1 prefix offsets (host memory)   */
    uint64_t n_traces;
} ltl_traces;

/* Options; a NULL pointer or a zero field selects the default. */
typedef struct {
    uint64_t mem_budget_bytes;   /* device bytes for cache + hash set; default:
                                    workspace_bytes, else 40% of free memory  */
    int stop_on_solution;        /* LTL_STOP_*, default LTL_STOP_FIRST when the
                                    whole struct is absent                    */
    uint64_t spin_limit;         /* bound on every device wait loop, in
                                    iterations (about 1 us each); default 2^20 */
    void *(*alloc)(size_t bytes, void *stream, void *user); /* optional device
                                    allocator (e.g. a framework's caching one) */
    void (*free)(void *ptr, void *stream, void *user);
    void *user;                  /* passed back to alloc / free               */
    void *stream;                /* cudaStream_t to run on; NULL: the
                                    context creates its own stream           */
    void *workspace;             /* optional caller-owned device buffer used
                                    for all device state (>= 256-byte aligned) */
    uint64_t workspace_bytes;
    const char *autotune_path;   /* online autotuning of the size-level
                                    launches (tiles per resident CTA: 2, 4 or
                                    8; resident CTAs per SM: the occupancy
                                    maximum or one fewer), per kernel shape,
                                    connective and candidate-count bucket,
                                    from the launches' own event times.  NULL:
                                    off (4 tiles per CTA, full occupancy);
                                    "": tune in memory for the lifetime of the
                                    context, batch call or server; a file
                                    path: also read when created and written
                                    when destroyed.  The string is copied.    */
    uint32_t max_chunks;         /* launch-shape cap: at most this many 16-byte
                                    chunks per thread (rounded up to a power of
                                    two); 0 = automatic                        */
    uint32_t costs[8];           /* cost homomorphism (Section 2): cost of the
                                    atoms, !, &, |, X, F, G, U in this order;
                                    0 = 1.  Size levels become cost levels and
                                    max_size is then the largest cost; a cost
                                    above max_size bans a connective          */
    uint32_t max_errors;         /* noisy learning (Section 3): a formula that
                                    misclassifies at most this many traces
                                    counts as separating; 0 = exact           */
    uint32_t ruc;                /* cache admission (Section 5): LTL_RUC_EXACT
                                    (default), LTL_RUC_HASH or LTL_RUC_FKP    */
    uint32_t ruc_mask_bits;      /* relaxed modes: zero this many of the 63
                                    admission-key bits, the highest first
                                    (0..62; the masking experiment, Sec. 7).
                                    LTL_RUC_EXACT: the same bits of the
                                    fingerprint key are zeroed, so that more
                                    candidates meet an equal key of a
                                    different matrix; the full compare still
                                    decides, results stay exact (a stress
                                    setting for the collision path)          */
    uint32_t level_kernel;       /* LTL_KERNEL_*: which size-level kernel runs
                                    matrices that fit one CTA                 */
    uint32_t level_planning;     /* LTL_PLAN_*: where the segments and tiles
                                    of a size level are planned              */
    uint32_t propagation;        /* LTL_PROP_*: how the level kernels compute
                                    F, G and U                               */
} ltl_opts;

/* level_kernel values.  All kernels compute the same candidates, counts and
 * cache; they differ in how the check-and-cache step is scheduled.
 *   LTL_KERNEL_AUTO   for matrices that fit one CTA, per launch: the
 *                     warp-specialised kernel when the problem's round has at
 *                     least 2^15 candidates and the shape's ring fits shared
 *                     memory, the fused kernel otherwise (small rounds are
 *                     bound by launch latency); for
 *                     larger matrices, rounds with fewer candidates than SMs
 *                     run the cluster kernel (a thread-block cluster holds one
 *                     candidate in its CTAs' shared memory) when a slice
 *                     fits, the others the two-pass streaming kernel (faster
 *                     when every SM has candidates of its own)
 *   LTL_KERNEL_FUSED  all warps compute a batch, then probe and store it;
 *                     larger matrices by the two-pass streaming kernel
 *   LTL_KERNEL_WS     compute warps hand each batch to dedicated hash warps
 *                     through a shared-memory ring and compute the next one
 *                     while the hash warps probe, store and compare it (when
 *                     the ring fits in shared memory; else the fused kernel),
 *                     in every launch; larger matrices by the cluster kernel
 *                     in every round (when a slice fits) */
enum { LTL_KERNEL_AUTO = 0, LTL_KERNEL_FUSED = 1, LTL_KERNEL_WS = 2 };

/* level_planning values.  A level's candidate space (Section 3) depends on how
 * many formulas every earlier level added.
 *   LTL_PLAN_AUTO  for one problem on the fused kernel: the levels that stay
 *                  below 2^17 candidates even if every earlier candidate were
 *                  new are planned on the device, one after another, and run
 *                  back to back with one read-back for the whole chain; the
 *                  other levels (and batches, servers, divide and conquer) are
 *                  planned on the host after reading back the previous level
 *   LTL_PLAN_HOST  every level planned on the host.
 * Results, counts and formulas are the same either way. */
enum { LTL_PLAN_AUTO = 0, LTL_PLAN_HOST = 1 };

/* propagation values: two evaluations of the same operators (Section 4), so
 * results, counts and formulas are the same either way.
 *   LTL_PROP_CARRY    (default) the positions of each trace reversed, U's
 *                     recursion g | (f & next) becomes the carry chain of the
 *                     integer sum (f | g) + g, and F(x) = x | -x: a fixed
 *                     handful of integer operations per trace word
 *   LTL_PROP_LOGSTEP  the paper's exponential propagation: ceil(log2 Lmax)
 *                     shift-by-2^i steps (Lemmas 1 and 2 of Appendix B)
 * ltl_eval always uses the exponential propagation. */
enum { LTL_PROP_CARRY = 0, LTL_PROP_LOGSTEP = 1 };

#define LTL_MAX_LEVELS 64

/* Per-level statistics.  Unique counts of a level are exact only when the
 * level completed (levels 1 .. levels_done). */
typedef struct {
    int levels_done;                      /* last fully enumerated size level   */
    int found_size;                       /* size of the returned formula, or 0 */
    uint64_t unique[LTL_MAX_LEVELS];      /* new characteristic matrices by size */
    uint64_t candidates[LTL_MAX_LEVELS];  /* candidates built at each size      */
    double ms[LTL_MAX_LEVELS];            /* device time of each level's kernel */
    uint64_t entries;                     /* language-cache entries at the end  */
    uint64_t n_traces;                    /* |P| + |N|                          */
    uint32_t words_per_trace;             /* characteristic words per trace     */
    uint32_t threads_per_cta;             /* launch shape chosen               */
    uint32_t traces_per_thread;
    uint32_t chunk_groups;                /* 1: candidates kept in registers   */
    uint32_t batch;                       /* candidates per CTA batch          */
    uint32_t traces_per_word;             /* 2: narrow layout (traces <= 32)   */
    uint32_t ctas_per_sm;                 /* resident CTAs per SM              */
    uint64_t launches;                    /* kernels launched by the call       */
    uint64_t h2d_bytes, d2h_bytes;        /* host<->device bytes copied         */
    uint64_t max_entries;                 /* cache capacity in entries          */
    double total_ms;                      /* wall time of the call              */
    float op_ms[LTL_MAX_LEVELS][8];       /* device time of each connective's
                                             launch: [level][op], op = 0 atoms,
                                             1 Not, 2 And, 3 Or, 4 X, 5 F, 6 G,
                                             7 U.  Its own time where op_alone
                                             is set.  Levels that run their
                                             launches concurrently (fewer than
                                             2^18 candidates, or several
                                             problems): the time from the
                                             level's start.  Larger levels of
                                             one problem run U alone first, then
                                             the others concurrently: theirs is
                                             the time from U's end.  Levels
                                             planned on the device
                                             (LTL_PLAN_AUTO) are timed by the
                                             device clock from one planner
                                             call to the next; each launched
                                             connective gets the level's time */
    uint32_t device_planned_levels;       /* levels planned on the device       */
    uint32_t graph_levels;                /* of those, levels run by replaying a
                                             captured CUDA graph               */
    uint64_t compares;                    /* full-matrix compares after an
                                             equal key (exact admission)       */
    uint64_t collisions;                  /* compares that found a different
                                             matrix (probing went on)          */
    uint64_t op_staged[LTL_MAX_LEVELS][8];/* operand matrices each connective's
                                             launch copied into shared memory
                                             ([level][op] as op_ms): counted by
                                             the fused and warp-specialised
                                             level kernels on levels planned
                                             on the host, 0 elsewhere;
                                             a launch shared by several
                                             problems reports its total to each */
    uint8_t op_kernel[LTL_MAX_LEVELS][8]; /* which level kernel ran each
                                             launch ([level][op] as op_ms):
                                             LTL_LAUNCH_*, 0 where none ran   */
    uint8_t op_alone[LTL_MAX_LEVELS][8];  /* 1 where the launch ran alone on the
                                             device, so that op_ms is its own
                                             duration                          */
} ltl_stats;

/* op_kernel values */
enum { LTL_LAUNCH_NONE = 0, LTL_LAUNCH_FUSED = 1, LTL_LAUNCH_WS = 2, LTL_LAUNCH_STREAM = 3,
       LTL_LAUNCH_CLUSTER = 4 };

/* ---------------------------------------------------------------------------
 * ltl_learn -- learn a minimal separating formula (Section 2, the LTL learning
 * problem; Section 3, `enum`).
 *   P, N       positive and negative traces (host memory).  P and N should be
 *              disjoint; a trace in both makes the problem unsolvable and the
 *              result is LTL_NOT_FOUND.
 *   n_props    alphabet size, 1..32; every letter must be < 2^n_props.
 *   ops        connectives allowed (mask of LTL_NOT .. LTL_U), optionally
 *              with LTL_NNF.
 *   max_size   largest formula size (syntax-tree nodes) tried, 1..63.
 *   opts       may be NULL.
 *   formula_out, formula_cap  receive the NUL-terminated text of a separating
 *              formula of minimal size (any one of them; "" when none).  A
 *              capacity of 8 * max_size + 1 bytes always suffices; a smaller
 *              buffer that cannot hold the text gives LTL_ERR_BUFSIZE.
 *   stats      may be NULL.
 * Returns LTL_OK, LTL_NOT_FOUND, LTL_CAP_REACHED or an error.
 * -------------------------------------------------------------------------*/
ltl_status ltl_learn(const ltl_traces *P, const ltl_traces *N, int n_props, uint32_t ops,
                     int max_size, const ltl_opts *opts, char *formula_out, size_t formula_cap,
                     ltl_stats *stats);

/* ---------------------------------------------------------------------------
 * ltl_eval -- characteristic sequences of a formula over traces (Section 4,
 * the characteristic matrix; F, G and U by exponential propagation).
 *   formula          text as above; atoms must be < n_props.
 *   traces           host memory.
 *   cs_out           host buffer of n_traces * words_per_trace uint64, trace
 *                    major: word w of trace t at cs_out[t * words_per_trace + w].
 *   words_per_trace  must be >= ceil(max trace length / 64).
 * -------------------------------------------------------------------------*/
ltl_status ltl_eval(const char *formula, const ltl_traces *traces, int n_props,
                    uint64_t *cs_out, int words_per_trace);

/* ---------------------------------------------------------------------------
 * Contexts: reusable device state (stream, workspace, language cache).  After
 * a learn call the context keeps the enumerated cache until the next call, so
 * it can be inspected.
 * -------------------------------------------------------------------------*/
typedef struct ltl_ctx ltl_ctx;

ltl_status ltl_ctx_create(const ltl_opts *opts, ltl_ctx **out);
void ltl_ctx_destroy(ltl_ctx *ctx);

/* Device bytes for the cache and hash set of the context's next learn calls
 * (as ltl_opts.mem_budget_bytes; 0 = all of the workspace). */
ltl_status ltl_ctx_set_mem_budget(ltl_ctx *ctx, uint64_t bytes);

/* As ltl_learn, on a context (host traces). */
ltl_status ltl_ctx_learn(ltl_ctx *ctx, const ltl_traces *P, const ltl_traces *N, int n_props,
                         uint32_t ops, int max_size, char *formula_out, size_t formula_cap,
                         ltl_stats *stats);

/* As ltl_ctx_learn with the traces already in device memory: d_letters and
 * d_offsets describe n_pos positive traces followed by n_neg negative ones;
 * max_len must be >= the longest trace.  The device buffers are only read
 * during the call. */
ltl_status ltl_ctx_learn_device(ltl_ctx *ctx, const uint32_t *d_letters, const uint64_t *d_offsets,
                                uint64_t n_pos, uint64_t n_neg, uint32_t max_len, int n_props,
                                uint32_t ops, int max_size, char *formula_out, size_t formula_cap,
                                ltl_stats *stats);

/* Entries of size level `level` of the last learn call are the cache indices
 * [*begin, *begin + *count). */
ltl_status ltl_ctx_level_range(ltl_ctx *ctx, int level, uint64_t *begin, uint64_t *count);

/* Formula text and characteristic matrix of cache entry `idx` of the last
 * learn call.  cs_out (host, may be NULL) receives n_traces * words_per_trace
 * uint64 in the layout of ltl_eval; words_per_trace must equal
 * stats.words_per_trace of that call.  LTL_ERR_BUFSIZE if formula_cap is too
 * small. */
ltl_status ltl_ctx_entry(ltl_ctx *ctx, uint64_t idx, char *formula_out, size_t formula_cap,
                         uint64_t *cs_out, int words_per_trace);

/* ---------------------------------------------------------------------------
 * Batched and served learning.  Many independent learning problems share one
 * device workspace; each keeps its language cache and hash set resident in
 * its own region of the workspace while it runs.  Work advances in rounds:
 * in one round every resident problem enumerates its next size level, and the
 * candidates of all of them are processed by one launch per connective and
 * launch shape (persistent CTAs pull tiles of any problem).  Problems are
 * admitted into free memory between rounds, so problems that arrive while
 * others run join the next round (continuous batching).  Each problem's result
 * is the same as ltl_learn's on it alone: same status, minimal size and
 * per-level counts (the formula text may be another minimal separator).
 * The paper has no batching; its D&C unit notes that sub-problems can be
 * learned in parallel (Section 6).
 * -------------------------------------------------------------------------*/
#define LTL_FORMULA_MAX 512

typedef struct {
    ltl_traces P, N;              /* host traces (copied at submission)        */
    int n_props;
    uint32_t ops;
    int max_size;
    uint64_t mem_budget_bytes;    /* device bytes for this problem's cache and
                                     hash set; 0 = the engine's default share  */
} ltl_problem;

typedef struct {
    uint64_t id;                  /* submission id (batch: the input index)    */
    ltl_status status;            /* as ltl_learn; LTL_ERR_OOM if the budget
                                     exceeds the whole workspace               */
    int found_size;
    int levels_done;
    char formula[LTL_FORMULA_MAX];
    uint64_t unique[LTL_MAX_LEVELS];
    uint64_t candidates[LTL_MAX_LEVELS];
    uint64_t n_traces;
    uint32_t rounds;              /* rounds the problem took part in           */
    double queue_ms;              /* entry of the submitting call -> admission */
    double latency_ms;            /* entry of the submitting call -> result
                                     (the library's copy of the traces
                                     included)                                 */
} ltl_result;

/* Learns n problems together; out[i] is problem i's result.  opts as for
 * ltl_learn (stop_on_solution applies to every problem; opts->workspace, if
 * given, holds all of them).  Returns LTL_OK if every problem was processed
 * (look at out[i].status), or an error. */
ltl_status ltl_learn_batch(int n, const ltl_problem *problems, const ltl_opts *opts, ltl_result *out);

/* A learning server: a host worker thread runs rounds while problems are
 * resident and admits submitted problems between rounds as their memory
 * budget fits (max_resident caps how many are resident at once, <= 4096). */
typedef struct ltl_server ltl_server;
ltl_status ltl_server_create(const ltl_opts *opts, int max_resident, ltl_server **out);
/* Queues a problem (its traces are copied); *id receives its id. */
ltl_status ltl_server_submit(ltl_server *srv, const ltl_problem *problem, uint64_t *id);
/* Moves up to max finished results into out (in completion order), waiting up
 * to wait_ms milliseconds for at least one; *n_out receives the count. */
ltl_status ltl_server_poll(ltl_server *srv, ltl_result *out, int max, int *n_out, int wait_ms);
/* Number of problems queued or resident (not yet polled as results). */
ltl_status ltl_server_pending(ltl_server *srv, uint64_t *queued, uint64_t *resident);
void ltl_server_destroy(ltl_server *srv);

/* ---------------------------------------------------------------------------
 * ltl_eval_noalloc -- ltl_eval for callers that cannot allocate device memory.
 * The paper has no counterpart; this is a deployment variant of ltl_eval.
 *
 * Who needs it: code that runs where allocation is not allowed -- inside a
 * framework that owns all device memory through its own pool, in a real-time
 * loop that must not allocate after start-up, or where the implicit
 * synchronisation of cudaMalloc / cudaFree is unacceptable.  This call
 * allocates nothing: no cudaMalloc, cudaFree or allocating library routine.
 *
 *   formula          text as for ltl_eval; atoms must be < n_props.
 *   d_letters,       the traces, already in DEVICE memory (layout as in
 *   d_offsets        ltl_traces); read only.
 *   n_traces         number of traces.
 *   max_len          >= the longest trace (<= 1024).  A trace longer than
 *                    max_len but within 64 * ceil(max_len / 64) positions is
 *                    still evaluated exactly; a longer one is rejected with
 *                    LTL_ERR_INVALID.
 *   d_cs_out         DEVICE buffer of n_traces * words_per_trace uint64, trace
 *                    major as for ltl_eval, written by the call.
 *   words_per_trace  >= ceil(max_len / 64).
 *   stream           cudaStream_t the work runs on (NULL: legacy default
 *                    stream); the call returns after the stream has finished it.
 *
 * Scratch: one file-scope static device array of LTL_NOALLOC_SCRATCH_BYTES
 * (64 MiB), held by every GPU that loads the library until the process exits.
 * A call needing more (about 8 * (1 + n_props + stack depth) * ceil(max_len/64)
 * * n_traces bytes) is rejected with LTL_ERR_OOM and a message giving the
 * size.  All calls on a device share the array and it keeps the last call's
 * contents; each call clears what must start at zero.  Calls whose work
 * overlaps on the GPU (other streams or host threads) race on the array: the
 * caller must serialise them.  The first call on a device looks up the
 * array's device address (cudaGetSymbolAddress, with that device current).
 * Every call also reads a status word back to the host and synchronises the
 * stream, so no call may be made while a stream is being captured.
 * -------------------------------------------------------------------------*/
#define LTL_NOALLOC_SCRATCH_BYTES (64ull << 20)
ltl_status ltl_eval_noalloc(const char *formula, const uint32_t *d_letters, const uint64_t *d_offsets,
                            uint64_t n_traces, uint32_t max_len, int n_props, uint64_t *d_cs_out,
                            int words_per_trace, void *stream);

/* -------------------------------------------------------------------------
 * ltl_learn_dc -- divide and conquer over the enumerator (Section 6).
 *
 * A specification with more traces than the split window is split, each part
 * of at most `window` traces is learned by the enumerator (all parts that are
 * ready at once share launches, as in ltl_learn_batch), and the partial
 * formulae are combined as (f11 & f12) | (f21 & f22).  The result separates
 * (P, N) -- the call checks it on every trace before returning -- but is not
 * minimal in general.
 *   LTL_DC_DETERMINISTIC  detSplit: P and N halved in list order; f11 on
 *                         (P1, N1), f12 on (P1, N2 accepted by f11), f21 on
 *                         (P2 not accepted by f11 & f12, N1), f22 on (that
 *                         P2, N2 accepted by f21), one after another.
 *   LTL_DC_RANDOM         randSplit: f11 on a random balanced sample of at
 *                         most `window` traces; then, concurrently, f12 on the
 *                         traces f11 accepts, f21 on those it rejects, f22 on
 *                         the positives it rejects against the negatives it
 *                         accepts.
 * A part the enumerator cannot solve within max_size or its memory budget is
 * closed by the overfitting formula of its positive trace when it has only
 * one (Section 3's fallback: that trace's letters under nested X's), else
 * retried with half the window; a part of one positive and one negative trace
 * that still fails is closed by a formula telling the two traces apart (their
 * first differing position, or the end of the shorter one).
 *
 * Arguments as ltl_learn; ops must allow & and | (the combination uses them);
 * opts->stop_on_solution is ignored (each part stops at its first
 * separator); opts->max_errors must be 0; costs, NNF and relaxed admission
 * apply to every part.  Results may vary between runs (which minimal formula
 * a part returns depends on timing); with LTL_DC_RANDOM the samples are drawn
 * from `seed`.  Traces may have at most 1024 positions.
 * Returns LTL_OK with the formula; LTL_NOT_FOUND when no formula over the
 * allowed connectives can separate (a trace in both P and N, an empty
 * positive trace, or a positive trace that is a prefix of a negative one
 * under LTL_NNF); LTL_ERR_BUFSIZE when formula_cap is too small
 * (stats->formula_len holds the length).
 * -------------------------------------------------------------------------*/
enum { LTL_DC_DETERMINISTIC = 0, LTL_DC_RANDOM = 1 };

typedef struct {
    int mode;              /* LTL_DC_DETERMINISTIC or LTL_DC_RANDOM             */
    uint64_t window;       /* split window: most traces (|P| + |N|) sent to one
                              enumeration; at least 2                          */
    uint64_t seed;         /* LTL_DC_RANDOM: seed of the sample draws          */
    int max_resident;      /* parts enumerated concurrently; 0 = 64            */
} ltl_dc_opts;

typedef struct {
    uint64_t enum_calls;   /* parts sent to the enumerator                    */
    uint64_t enum_failed;  /* of which found no formula (window halved)       */
    uint64_t fallbacks;    /* parts closed by an overfitting or distinguishing
                              formula                                         */
    uint64_t evals;        /* formulae evaluated on all traces (membership)   */
    uint64_t rounds;       /* enumeration rounds (shared launch groups)       */
    uint64_t min_window;   /* smallest split window used                      */
    int max_depth;         /* depth of the deepest part enumerated or split
                              (0: the whole specification in one enumeration) */
    uint64_t formula_size; /* syntax-tree nodes of the returned formula       */
    uint64_t formula_len;  /* its text length, without the terminating NUL    */
    double total_ms;
} ltl_dc_stats;

ltl_status ltl_learn_dc(const ltl_traces *P, const ltl_traces *N, int n_props, uint32_t ops, int max_size,
                        const ltl_opts *opts, const ltl_dc_opts *dc, char *formula_out, size_t formula_cap,
                        ltl_dc_stats *stats);

/* The autotuner's measurements on a context (see ltl_opts.autotune_path), as
 * text: one line per launch class -- its key, then for each of the six
 * configurations (tiles per CTA 2, 4, 8 at full occupancy, then the same with
 * one CTA per SM fewer) "best ns per candidate:runs" (0:0 = untried).
 * LTL_ERR_BUFSIZE when `cap` bytes do not hold it (*needed is set either way,
 * terminating NUL included). */
ltl_status ltl_ctx_autotune_dump(ltl_ctx *ctx, char *out, size_t cap, size_t *needed);

/* Integer throughput of the current device, the roof for candidate launches
 * that memory does not hold back.  The log-step loops of F, G and U (Section
 * 4) consist of 32-bit shifts and three-input bitwise operations; this runs
 * `iters` steps of eight independent chains of one shift and one three-input
 * operation in every thread of 8 CTAs x 256 threads per SM, `repeats` times
 * after one warm-up launch, on a stream of its own.
 *   *ops_per_s  32-bit integer operations (shifts + logic operations, per
 *               thread) per second of the fastest repeat.
 *   *best_ms    that repeat's CUDA-event time (may be NULL).
 * LTL_ERR_INVALID for NULL ops_per_s, iters < 4 or repeats < 1;
 * LTL_ERR_CUDA when the device cannot run it.  Allocates 4 bytes per CTA of
 * device memory for the duration of the call. */
ltl_status ltl_int32_peak(int iters, int repeats, double *ops_per_s, double *best_ms);

/* Message of the last error on this host thread (static storage). */
const char *ltl_last_error(void);

/* Library build information (static storage). */
const char *ltl_version(void);

#ifdef __cplusplus
}
#endif
#endif /* LTL_GB300_H */
