/*
 * imm.h — C ABI of the GB300 IMM hot path (EfficientIMM, arXiv 2411.09473).
 *
 * The library samples random reverse-reachable (RRR) sets on the GPU and runs
 * greedy max-coverage seed selection over them, under the Independent Cascade
 * (IC) and Linear Threshold (LT) models.  Every kernel is hand-written CUDA for
 * sm_103a; this header is the only interface (plain C types, no torch types).
 *
 * Conventions shared by every call
 *   - Return value: IMM_OK (0) or one of the IMM_E* codes below.  On error the
 *     context stays usable; imm_last_error() describes the failure.
 *   - Host pointers are caller-owned and only read (or written, for outputs)
 *     during the call; the library never keeps them.
 *   - Device memory is library-owned.  It comes from the optional allocator
 *     given to imm_create (e.g. PyTorch's caching allocator), otherwise from
 *     stream-ordered allocations (cudaMallocFromPoolAsync on the context's
 *     stream) in a memory pool the library keeps per device; that pool
 *     retains freed memory for reuse until the process exits.
 *   - All GPU work of a context is issued on the stream given to imm_create
 *     (NULL = the legacy default stream).  Calls that return host results
 *     synchronise that stream before returning.
 *   - Vertex ids are uint32 (n < 2^32 - 1); edge ids are uint32 positions in
 *     the in-edge array (m < 2^32); set ids are uint64 but a stream holds fewer
 *     than 2^32 - 1 sets (occurrence counts are uint32).
 *   - Randomness: Philox4x32-10 (Salmon et al., SC'11) keyed by the 64-bit
 *     rng seed.  Root of set s: words 0,1 of Philox(ctr=(s_lo,s_hi,0,1));
 *     IC coin of in-edge e: word e&3 of Philox(ctr=(s_lo,s_hi,e>>2,2));
 *     LT draw at vertex v: word 0 of Philox(ctr=(s_lo,s_hi,v,3)).  Each set is
 *     therefore a pure function of (graph, seed, set id), whatever the
 *     traversal order, launch shape or batching.
 *   - Not thread-safe: one host thread drives a context at a time.
 */
#ifndef IMM_H
#define IMM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---- */
#define IMM_OK        0
#define IMM_EINVAL    1  /* bad argument or malformed graph */
#define IMM_ENOMEM    2  /* device allocation failed or arena limit reached */
#define IMM_ECUDA     3  /* a CUDA runtime call or kernel failed */
#define IMM_ETIMEOUT  4  /* a bounded device wait gave up */
#define IMM_ESTATE    5  /* call not valid in the context's current state */

/* ---- diffusion models (Sec. II-A) ---- */
#define IMM_IC 0
#define IMM_LT 1

typedef struct imm_ctx imm_ctx;

/* Optional device allocator.  alloc returns a device pointer of at least
 * `bytes` bytes usable on `stream`, or NULL on failure; free releases it. */
typedef struct imm_alloc {
    void* (*alloc)(void* user, size_t bytes, void* stream);
    void (*free)(void* user, void* ptr, size_t bytes, void* stream);
    void* user;
} imm_alloc;

#define IMM_MAX_ROUNDS 64

/* Statistics of one imm_run (all fields written by the call). */
typedef struct imm_stats {
    uint32_t rounds;                      /* sampling-phase rounds executed (Alg. 1 loop) */
    uint32_t stopped_early;               /* 1 if the OPT lower-bound test fired */
    uint64_t theta_i[IMM_MAX_ROUNDS];     /* theta_i of each round */
    uint64_t covered_i[IMM_MAX_ROUNDS];   /* sets covered by that round's selection */
    uint64_t sets_i[IMM_MAX_ROUNDS];      /* stream size at that round's selection */
    double lb;                            /* lower bound on OPT (1 if the test never fired) */
    uint64_t theta;                       /* Set_Theta result, ceil(lambda* / LB) */
    uint64_t num_sets;                    /* final stream size, max(theta, sets so far) */
    uint64_t covered;                     /* sets covered by the final seed set */
    double lambda_prime;
    double lambda_star;
    uint64_t members;                     /* sum of set sizes over the final stream */
    uint64_t edges_examined;              /* IC: in-edges whose coin was read; LT: walk steps */
    double ms_total;                      /* host wall time of the call */
    double ms_sample;                     /* device time of sampling kernels (CUDA events) */
    double ms_select;                     /* device time of selection kernels (CUDA events) */
    double ms_index;                      /* device time of compaction + inverted-index kernels */
    uint64_t sample_launches;             /* sampler kernel launches (timed by ms_sample) */
    uint64_t kernel_launches;             /* all kernel launches issued by the call */
    uint64_t sample_edges;                /* same as edges_examined, for the timed launches */
    uint64_t sample_members;              /* members produced by the timed sampler launches */
    uint64_t reused_sets;                 /* served queries: sets already resident when the query
                                             started (a stream drawn with the same seed) */
} imm_stats;

/* Create a context on CUDA device `device`.  `alloc` may be NULL (then
 * the library's memory pool is used); `stream` is a cudaStream_t or NULL.
 * Errors: EINVAL (out==NULL or bad device), ECUDA. */
int imm_create(imm_ctx** out, int device, const imm_alloc* alloc, void* stream);

/* Destroy a context and free all its device memory.  NULL is a no-op. */
void imm_destroy(imm_ctx* ctx);

/* Message describing the context's most recent error (owned by the context,
 * valid until the next call on it).  Never NULL. */
const char* imm_last_error(imm_ctx* ctx);

/* Load a directed graph G = (V, E) (Sec. II-A) as CSR of its transpose, i.e.
 * in-edges grouped by head v: in-edges of v are positions
 * in_row[v] .. in_row[v+1]-1 of in_src (their tails u) and weight.
 * weight[e] is p_uv for IMM_IC (edge live with that probability) or w_uv for
 * IMM_LT (sum over a head's in-edges <= 1 + 1e-6).  Host pointers, copied in.
 * The library derives per-edge integer thresholds on the device:
 *   IC: thr[e] = ceilf(p_e * 2^24) (fp32, exact);
 *   LT: cthr[e] = min(ceil(cw_e * 2^24), 2^24), cw_e the fp64 left-to-right
 *       running sum of the head's weights in CSR order.
 * Replaces any previous graph and drops the current RRR-set stream.
 * Errors: EINVAL (n < 2, in_row[0] != 0, in_row[n] != m, in_row not
 * monotone, in_src[e] >= n, weight NaN/<0/>1, LT head sum > 1 + 1e-6,
 * m >= 2^32), ENOMEM, ECUDA. */
int imm_load_graph(imm_ctx* ctx, uint32_t n, uint64_t m, const uint64_t* in_row,
                   const uint32_t* in_src, const float* weight, int model);

/* Same as imm_load_graph with DEVICE pointers (on the context's device,
 * readable on its stream).  The data is copied into library memory. */
int imm_load_graph_device(imm_ctx* ctx, uint32_t n, uint64_t m, const uint64_t* d_in_row,
                          const uint32_t* d_in_src, const float* d_weight, int model);

/* Generate_RRRsets (Alg. 1 lines 3 and 9; Alg. 3): extend the RRR-set stream
 * to `theta` sets by sampling set ids |R| .. theta-1 with `rng_seed`
 * (no-op if theta <= |R|).  Each set: a root drawn uniformly from V, then
 *   IC: every vertex that reaches the root through live in-edges (reverse
 *       probabilistic BFS; in-edge e live iff (coin >> 8) < thr[e]);
 *   LT: the reverse walk that at vertex v picks the first in-edge j with
 *       (draw >> 8) < cthr[j], stopping when none is picked or the picked
 *       tail is already in the set.
 * Members are stored contiguously per set in set-id order (prefix-sum
 * compaction into the device arena) and counted into the per-vertex
 * occurrence counter (Alg. 3, fused count).
 * Errors: EINVAL (model differs from the loaded graph's, theta >= 2^32-1),
 * ESTATE (no graph, or rng_seed differs from the current stream's: call
 * imm_reset_sets first), ENOMEM (arena limit or allocation), ECUDA. */
int imm_sample(imm_ctx* ctx, int model, uint64_t theta, uint64_t rng_seed);

/* Find_Most_Influential_Set (Alg. 2): greedy max coverage over the current
 * stream.  k rounds; each picks the vertex not yet picked with the most
 * occurrences among uncovered sets (ties -> lowest id; picking continues at
 * count 0), marks every uncovered set holding it covered and removes those
 * sets' members from the counts (by decrement, or by recounting the
 * uncovered sets when that is less work: Sec. IV-C adaptive counter update;
 * the result is identical).  Writes the k picks in order to seeds_out (host,
 * k entries) and the number of covered sets to *covered_out (host, nullable).
 * Errors: EINVAL (k == 0, k > n, seeds_out NULL), ESTATE (no graph), ECUDA. */
int imm_select(imm_ctx* ctx, uint32_t k, uint32_t* seeds_out, uint64_t* covered_out);

/* IMM (Alg. 1 with Tang, Shi & Xiao 2015's Theta_Estimation,
 * OPT_Lower_Bound and Set_Theta): drops the current stream, then
 *   ell' = ell (1 + ln2 / ln n), eps' = sqrt(2) eps,
 *   for i = 1 .. ceil(log2 n) - 1: x = n / 2^i, sample to ceil(lambda'/x),
 *     select k; stop with LB = nF/(1+eps') once nF = n*covered/|R| >= (1+eps') x;
 *   theta = ceil(lambda* / LB); sample to max(theta, |R|); select k.
 * lambda' and lambda* as in Tang et al.; host fp64, no FMA contraction.
 * Writes k seeds to seeds_out (host) and, if stats_out != NULL, *stats_out.
 * Errors: EINVAL (k == 0, k > n, eps not in (0,1), ell <= 0, model differs
 * from the graph's, theta would reach 2^32-1), ESTATE, ENOMEM, ECUDA. */
int imm_run(imm_ctx* ctx, int model, uint32_t k, double epsilon, double ell,
            uint64_t rng_seed, uint32_t* seeds_out, imm_stats* stats_out);

/* imm_run with options (flags: OR of IMM_RUN_*).
 * IMM_RUN_FRESH_FINAL: the final selection runs on a fresh stream.  Once the
 * estimation rounds have fixed LB and theta, their sets are dropped, and
 * exactly theta new sets are sampled under the key rng_seed ^
 * IMM_FRESH_FINAL_KEY.  They are independent of the sets that fixed theta.
 * This is Chen's 2018 correction of Alg. 1's reuse of those sets; the paper
 * reuses them.  The estimation rounds, LB and theta are the same as
 * imm_run's.  stats_out->num_sets is theta, and the stream left in the
 * context is the fresh one.
 * flags == 0 is imm_run.  Errors: as imm_run, and EINVAL for unknown flags. */
#define IMM_RUN_FRESH_FINAL 1u
#define IMM_FRESH_FINAL_KEY 0x9E3779B97F4A7C15ull
int imm_run_ex(imm_ctx* ctx, int model, uint32_t k, double epsilon, double ell,
               uint64_t rng_seed, uint32_t flags, uint32_t* seeds_out, imm_stats* stats_out);

/* OPIM-style early stop (Sec. VI cites OPIM: Tang, Tang, Xiao, Yuan,
 * SIGMOD 2018; this follows its OPIM-C procedure).  Two independent RR-set
 * collections of equal size double each round: R1 is the context's stream
 * under rng_seed, R2 a second stream on the same graph under rng_seed ^
 * IMM_OPIM_KEY (held by the call, freed before it returns).  Per round i:
 *   theta_i = ceil(theta_0) * 2^(i-1) sets per collection, i = 1 .. i_max;
 *   S = the greedy's k picks over R1 (as imm_select), cov1 = its R1
 *   coverage, cov2 = the number of R2 sets holding a member of S;
 *   upper = (sqrt(cov1 / (1 - (1-1/k)^k) + a1/2) + sqrt(a1/2))^2 * n / theta_i
 *   lower = ((sqrt(cov2 + 2 a2/9) - sqrt(a2/2))^2 - a2/18) * n / theta_i
 *   stop with S once lower / upper >= 1 - 1/e - epsilon, or at i_max.
 * With delta = n^-ell, g = 1 - 1/e, L = ln(6/delta):
 *   theta_max = 2n (g sqrt(L) + sqrt(g (ln C(n,k) + L)))^2 / (eps^2 k),
 *   theta_0 = theta_max eps^2 k / n, i_max = max(1, ceil(log2(theta_max /
 *   theta_0))), a2 = ln(3 i_max / delta), a1 = a2 + ln C(n,k).
 * Host fp64, no FMA contraction.  Writes k seeds to seeds_out (host) and, if
 * stats_out != NULL, *stats_out; the context keeps R1 as its stream.
 * Errors: EINVAL (k == 0, k > n, eps not in (0,1), ell <= 0, model differs
 * from the graph's, collections would reach 2^32-1 sets), ESTATE, ENOMEM,
 * ECUDA. */
#define IMM_OPIM_KEY 0xD1B54A32D192ED03ull
typedef struct imm_opim_stats {
    uint32_t rounds;                  /* rounds run */
    uint32_t stopped_early;           /* 1 if the ratio test fired before round i_max */
    uint32_t i_max;
    uint64_t sets_i[IMM_MAX_ROUNDS];  /* sets per collection in round i */
    uint64_t cov1_i[IMM_MAX_ROUNDS];  /* R1 coverage of that round's picks */
    uint64_t cov2_i[IMM_MAX_ROUNDS];  /* R2 coverage of the same picks */
    double upper_i[IMM_MAX_ROUNDS];   /* upper confidence bound on OPT */
    double lower_i[IMM_MAX_ROUNDS];   /* lower confidence bound on the picks' spread */
    double theta_max;
    double theta_0;
    double alpha;                     /* lower / upper of the last round */
    double ms_total;                  /* host wall time of the call */
    double ms_sample;                 /* device time of R1's sampling kernels */
    double ms_select;                 /* device time of the selections */
    uint64_t kernel_launches;
} imm_opim_stats;
int imm_run_opim(imm_ctx* ctx, int model, uint32_t k, double epsilon, double ell, uint64_t rng_seed,
                 uint32_t* seeds_out, imm_opim_stats* stats_out);

/* ---- tuning (knobs that change speed, never results) ----
 * Every RRR set is a pure function of (graph, seed, set id) and the greedy's
 * picks do not depend on how the work is scheduled, so these knobs change
 * how fast a run goes, not what it returns.
 *   batch_sets        most sets sampled per batch (the arena grows by
 *                     batches; smaller batches reuse less memory per step)
 *   group_min_mean    mean size of the large IC sets (from earlier batches)
 *                     from which solo runs sample them 64 at a time as one
 *                     multi-source BFS (also needs >= n/64)
 *   select_cta_max_n  solo selections on graphs up to this many vertices run
 *                     on one CTA, larger ones on the cooperative grid
 *   cluster_min_n     batched and served selections on graphs of at least
 *                     this many vertices run on an 8-CTA thread-block
 *                     cluster, smaller ones on one CTA
 *   select_cand       nonzero: one-CTA and cluster selections scan a
 *                     candidate list in rounds where it is exact
 *   solo_cluster      nonzero: solo selections above select_cta_max_n over
 *                     streams without bitmap-stored sets run on one 8-CTA
 *                     cluster instead of the cooperative grid (default 0)
 * Batch and server workers take the tuning of their graph's context. */
typedef struct imm_tuning {
    uint32_t batch_sets;
    uint32_t group_min_mean;
    uint32_t select_cta_max_n;
    uint32_t cluster_min_n;
    uint32_t select_cand;
    uint32_t solo_cluster;
} imm_tuning;
/* Errors: EINVAL (ctx or tuning NULL, batch_sets < 256). */
int imm_set_tuning(imm_ctx* ctx, const imm_tuning* tuning);
int imm_get_tuning(imm_ctx* ctx, imm_tuning* tuning_out);

/* One query of a batch: the context holding its graph (loaded with
 * imm_load_graph; the model is the graph's), and IMM's parameters. */
typedef struct imm_query {
    imm_ctx* graph;
    uint32_t k;
    double epsilon;
    double ell;
    uint64_t rng_seed;
} imm_query;

/* Batched IMM (Alg. 1 per query, as imm_run): nq queries over one or more
 * loaded graphs advance together.  Each wave runs one sampling batch of every
 * query still sampling (each on its own stream) and one selection launch for
 * every query that reached its sampling target (one CTA per query).  Each
 * query's seeds, theta ladder, LB and theta equal imm_run's on the same
 * inputs.  seeds_out (host) receives the queries' seeds concatenated in query
 * order (sum of k entries); stats_out (host, nq entries, nullable) and
 * status_out (host, nq entries, nullable) receive per-query statistics and
 * status.  The graph contexts' RRR-set streams are not touched.  The
 * queries' own buffers come from their graph context's allocator (the
 * library's memory pool if it has none), on the queries' own streams, and
 * selections of instances on graphs of >= 2^15 vertices run on thread-block
 * clusters.
 * Errors: EINVAL (a query's graph missing or not loaded, contexts on
 * different devices, bad k/epsilon/ell); a query that fails on its own
 * (ENOMEM under the graph context's arena limit, ...) reports its status in
 * status_out while the others complete. */
int imm_run_batch(const imm_query* queries, uint32_t nq, uint32_t* seeds_out, imm_stats* stats_out,
                  int* status_out);

/* Autotuner for batched IMM: runs the batch (imm_run_batch) once per
 * candidate tuning of a fixed grid, each applied to every graph context of
 * the batch, `reps` times each (the first run of each candidate is not
 * timed when reps > 1), and keeps the fastest by host wall time: it is set
 * on every graph context of the batch and written to *best_out (nullable).
 * times_ms_out (host, nullable, IMM_TUNE_CANDIDATES entries) receives each
 * candidate's mean time, and candidates_out (host, nullable, same count) the
 * candidates.  The batch's results are the same under every candidate.
 * Errors: as imm_run_batch (a query that fails fails the call). */
#define IMM_TUNE_CANDIDATES 12
int imm_autotune_batch(const imm_query* queries, uint32_t nq, uint32_t reps, imm_tuning* best_out,
                       double* times_ms_out, imm_tuning* candidates_out);

/* ---- served IMM (continuous batching) ----
 * A server keeps the given graphs resident (caller-owned contexts that must
 * outlive it) and runs IMM queries on a host thread in waves (as
 * imm_run_batch).  Between waves it admits submitted queries while fewer
 * than max_active are in flight and its workers' device memory is under
 * memory_budget_bytes (0 = no limit; each query's arena is then limited to
 * half the budget), so queries that arrive while others are on the GPU join
 * the next wave and overlap with them.  Every result equals the query's solo
 * imm_run.  Server workers allocate from the library's memory pool on their own
 * streams (never through the contexts' allocator callbacks). */
typedef struct imm_server imm_server;

typedef struct imm_server_config {
    uint64_t memory_budget_bytes;
    uint32_t max_active;  /* 0 = 64 */
    /* Nonzero: prefix-stable stream sharing.  A finished query's RRR-set
     * stream stays resident in its idle worker, and a later query on the same
     * graph with the same rng seed reuses it (Alg. 1 extends a stream by
     * appending set ids, and a set is a function of graph, seed and set id
     * only): its selections see the prefix of the resident stream that the
     * query would have sampled, and it samples only the sets beyond it.
     * Results are those of the query run alone; imm_stats.reused_sets counts
     * the sets it found resident.  Resident streams count against the memory
     * budget, and idle workers are reclaimed when admission needs memory. */
    uint32_t share_streams;
} imm_server_config;

typedef struct imm_completion {
    uint64_t id;
    int status;          /* IMM_OK or the query's error */
    double latency_ms;   /* submission to completion */
    double queue_ms;     /* submission to admission */
} imm_completion;

/* Errors: EINVAL (no graphs, a graph not loaded, contexts on different
 * devices), ECUDA, ENOMEM. */
int imm_server_create(imm_server** out, imm_ctx* const* graphs, uint32_t ngraphs, const imm_server_config* cfg);
/* Queue a query on graph index `graph` (position in the create call's list);
 * *id_out receives its id.  Errors: EINVAL (bad graph index, k, eps, ell),
 * or the status of a failure that stopped the server. */
int imm_server_submit(imm_server* s, uint32_t graph, uint32_t k, double epsilon, double ell, uint64_t rng_seed,
                      uint64_t* id_out);
/* Non-blocking: up to cap completions (oldest first) into out (host). */
int imm_server_poll(imm_server* s, imm_completion* out, uint32_t cap, uint32_t* n_out);
/* Results of a completed query (seeds_out: host, k >= the query's k;
 * stats_out nullable); the query is then forgotten.  Errors: ESTATE (id not
 * completed or unknown), EINVAL (k too small), or the query's own error. */
int imm_server_take(imm_server* s, uint64_t id, uint32_t* seeds_out, uint32_t k, imm_stats* stats_out);
/* Queue depth, queries in flight, waves run, device bytes held; returns the
 * status of a failure that stopped the server (IMM_OK if none). */
int imm_server_info(imm_server* s, uint64_t* pending, uint64_t* active, uint64_t* waves, uint64_t* device_bytes);
/* Stop the loop (the wave in progress finishes), free everything. */
void imm_server_destroy(imm_server* s);

/* Drop the RRR-set stream (counts, arena, index); keeps the graph. */
int imm_reset_sets(imm_ctx* ctx);

/* Number of sets in the stream and total members (either pointer nullable). */
int imm_stream_size(imm_ctx* ctx, uint64_t* num_sets, uint64_t* num_members);

/* Test hook: members of stored set `set_id`, sorted ascending, into buf
 * (host, cap entries); *len receives the set's size.
 * Errors: EINVAL (set_id >= |R|, len NULL, or size > cap). */
int imm_get_set(imm_ctx* ctx, uint64_t set_id, uint32_t* buf, uint32_t cap, uint32_t* len);

/* Test hook: sets first .. first+count-1 in stored layout.  off_out (host,
 * count+1 entries) receives offsets relative to the first set's start;
 * mem_out (host, cap entries) receives the members (traversal order inside
 * each set, not sorted).  off_out is filled even when the members do not
 * fit, so a call with cap = 0 sizes the buffer.  Errors: EINVAL (range
 * outside the stream, or members > cap). */
int imm_get_sets(imm_ctx* ctx, uint64_t first, uint64_t count, uint64_t* off_out,
                 uint32_t* mem_out, uint64_t cap);

/* Test hook: per-vertex occurrence counts over the whole stream (host, n). */
int imm_get_counts(imm_ctx* ctx, uint32_t* cnt_out);

/* Limit on device bytes for the RRR-set arena and its inverted index
 * (0 = unlimited).  imm_sample returns ENOMEM instead of growing past it. */
int imm_set_arena_limit(imm_ctx* ctx, uint64_t bytes);

/* Properties of the loaded build: IMM_BUILD_BOUNDS_CHECK is set when the
 * library was compiled with index checks (-DIMM_BOUNDS_CHECK).  That build
 * compares indices into the stream arena, the sampling staging and output
 * buffers, the per-set queues, the grouped sampler's lists and the
 * selection's lists with their bounds; the first index out of range is not
 * used, the kernels record it, and the call returns IMM_ECUDA naming the
 * check, the index and the bound. */
#define IMM_BUILD_BOUNDS_CHECK 1
int imm_build_flags(void);

/* ---- selection without device allocation ----
 * No counterpart in the paper: this entry point exists for callers that
 * cannot allocate device memory at run time, for example a plugin inside
 * another framework whose memory pool owns the whole GPU, or a service whose
 * memory footprint is fixed when it starts.
 *
 * Same greedy max coverage as imm_select (k rounds, ties to the lowest vertex
 * id, picked vertices excluded, picking continues at count 0), over a set
 * system the caller already holds on the device:
 *   d_off      device uint64[nsets + 1], member offsets (nondecreasing, d_off[0] = 0)
 *   d_members  device uint32[d_off[nsets]], vertex ids < n, distinct within a set
 *   d_seeds_out   device uint32[k]: the picks in order
 *   d_covered_out device uint64 (nullable): number of sets covered
 *   stream     cudaStream_t (NULL = legacy default stream); the call is
 *              asynchronous on it and returns once the work is enqueued.
 * It allocates and frees nothing (no cudaMalloc/cudaFree, no allocating
 * library routine).  Its scratch is one fixed array compiled into the library
 * (about 9 MB), held on every GPU that loads the library until the process
 * exits.  Limits: n <= IMM_NOALLOC_MAX_N, nsets <= IMM_NOALLOC_MAX_SETS,
 * k <= IMM_NOALLOC_MAX_K.
 * The first call on a device looks up that array's device address and the
 * device's SM count (with the device current) and keeps them for the life of
 * the process; make that first call before any stream capture, and do not
 * call it again after a cudaDeviceReset of that device.  Every call shares
 * the array and clears what must start at zero; calls that overlap on the GPU
 * (other streams, other host threads) race on it and must be serialised by
 * the caller.
 * A member id >= n is never used as an index: the kernels skip it, and the
 * call then writes 0xFFFFFFFF to every seed and 2^64 - 1 to *d_covered_out
 * (the check happens on the GPU, so it cannot be returned as a status).
 * A launch error pending on the calling thread from earlier work is cleared
 * on entry.
 * Errors: EINVAL (n == 0, k == 0, k > n, a size above its limit, a NULL
 * required pointer), ECUDA (device lookup or a launch failed; no later round
 * is enqueued after a failed launch). */
#define IMM_NOALLOC_MAX_N    (1u << 20)
#define IMM_NOALLOC_MAX_SETS (1u << 22)
#define IMM_NOALLOC_MAX_K    4096u
int imm_select_noalloc(uint32_t n, uint64_t nsets, const uint64_t* d_off, const uint32_t* d_members,
                       uint32_t k, uint32_t* d_seeds_out, unsigned long long* d_covered_out, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* IMM_H */
