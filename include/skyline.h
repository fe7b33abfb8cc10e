/*
 * skyline.h -- C ABI of libskyline, a GB300 (sm_103a) implementation of the
 * partitioned skyline method of Ciaccia & Martinenghi, "Optimization
 * Strategies for Parallel Computation of Skylines" (arXiv 2411.14968).
 *
 * Problem (Section 2, Def. 1): given a relation r of N tuples with d numeric
 * attributes, all to be minimised, a tuple t dominates s (t < s) iff
 * t[A] <= s[A] for every attribute A and t[A'] < s[A'] for at least one A'.
 * The skyline Sky(r) is the set of tuples that no tuple of r dominates.  Exact
 * duplicates never dominate each other, so every copy of a skyline tuple is
 * returned.  Comparisons are exact IEEE FP32 comparisons (no reduced
 * precision, no flush-to-zero); -0.0 equals +0.0; +-inf are allowed; NaN is
 * rejected.
 *
 * Method (Algorithm 2, Section 3): Partition r into r_1..r_p (Random 3.1,
 * Grid 3.2, Angular 3.3, Sliced 3.4), optionally drop grid-dominated cells
 * (Grid Filtering, 3.2) and tuples dominated by representatives (4.1),
 * compute every local skyline u_i = Sky(r_i) with the sort-filter-skyline
 * order of Algorithm 1, then merge: Sky(u) over u = union of u_i (sequential
 * final phase) or the NoSeq identity Sky(r) = union_i Sky_{pd_i}(u_i)
 * (Section 4.2, Prop. 2).  Every variant returns the same set (Prop. 1,
 * Prop. 2), so the result never depends on the parameters.
 *
 * Conventions of every call:
 *  - status codes are returned; nothing is thrown across the ABI;
 *  - `points` is row-major N x d FP32, caller-owned and read-only; it may be
 *    host memory (pageable or pinned) or device memory of the context's
 *    device -- the library asks the CUDA runtime which;
 *  - index outputs are caller-owned u32 arrays of capacity >= N in host or
 *    device memory (again detected); indices are 0-based and ascending;
 *  - a context owns its device scratch memory, grows it on demand within
 *    its memory budget and frees it in sky_destroy;
 *  - calls on one context must not run concurrently from several host
 *    threads, except sky_submit / sky_poll / sky_wait.
 */
#ifndef SKYLINE_H_
#define SKYLINE_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  SKY_OK = 0,
  SKY_EINVAL = 1,     /* bad argument: d outside 1..8, N >= 2^32, NaN, bad params */
  SKY_ENOMEM = 2,     /* scratch memory beyond the context budget or cudaMalloc failed */
  SKY_ECUDA = 3,      /* a CUDA runtime call failed; sky_last_error says which */
  SKY_ETIMEOUT = 4,   /* a bounded device-side wait gave up (the GPU stays usable) */
  SKY_EBUSY = 5,      /* a ticket is still in flight (sky_poll) */
  SKY_ECANCELLED = 6  /* unknown or already collected ticket */
} sky_status;

typedef enum {
  SKY_RANDOM = 0,   /* Section 3.1: random, equi-numerous partitions */
  SKY_GRID = 1,     /* Section 3.2: m_i slices per attribute, p = prod m_i cells */
  SKY_ANGULAR = 2,  /* Section 3.3: m_i slices per hyperspherical angle (d-1 angles) */
  SKY_SLICED = 3,   /* Section 3.4: p equal slices along one attribute */
  SKY_NONE = 4      /* one partition: plain SFS (Algorithm 1) over the whole input */
} sky_partitioning;

/* Representative filtering (Section 4.1): Sorted = the first points of each
   partition in score order; Region = the points with the largest volume of
   the dominance region inside the unit cube (prod (1 - x_i), attributes
   clamped to [0, 1], or divided by the column maximum first when
   `normalize` is set; at most 64 per partition). */
typedef enum { SKY_REP_NONE = 0, SKY_REP_SORTED = 1, SKY_REP_REGION = 2 } sky_rep;
typedef enum { SKY_MERGE_SEQUENTIAL = 0, SKY_MERGE_NOSEQ = 1 } sky_merge;
typedef enum {
  SKY_EXEC_PERSISTENT = 0, /* all partitions' local skylines in one cooperative launch */
  SKY_EXEC_PLAIN = 1       /* one launch per partition, in partition order */
} sky_exec;

/* The 16-bit images the dominance engine tests before its FP32 test (a
   filter that never changes a result, only how many pairs reach the FP32
   test; Def. 1 is invariant under any strictly increasing map of each
   attribute, and the images need only be non-decreasing):
   SKY_IMAGES_VALUES: each attribute rounded down to FP16 (clamped to the
     finite FP16 range).  Free, and sharp for values of moderate magnitude
     spread over many FP16 steps (e.g. [0, 1]); blunt when a column's values
     share few FP16 numbers -- a large common offset, magnitudes above
     65504 or below about 1e-5 -- and the engine then runs several times
     slower (every pair reaches the FP32 test).
   SKY_IMAGES_RANKS: each attribute's dense rank in its column (sky_rank_space),
     used as an order-preserving 15-bit code: exact (distinct values keep
     distinct codes) for columns of at most 31,744 distinct values, scaled
     down otherwise.  Costs one sort per attribute; the engine's speed then
     no longer depends on the value range. */
typedef enum { SKY_IMAGES_VALUES = 0, SKY_IMAGES_RANKS = 1 } sky_images;

typedef struct {
  uint32_t struct_size;        /* sizeof(sky_params); filled by sky_params_init */
  sky_partitioning scheme;
  uint32_t num_partitions;     /* Random / Sliced: p (clamped to [1, N]) */
  uint32_t slices[8];          /* Grid: m per attribute (d used); Angular: m per angle (d-1 used) */
  uint32_t normalize;          /* Grid / Angular keys and Region volumes: divide each attribute by
                                  its column maximum first (dominance uses raw values) */
  uint32_t slice_dim;          /* Sliced: attribute to slice on (default 0) */
  uint64_t seed;               /* Random: SplitMix64 seed */
  uint32_t grid_filter;        /* Grid: drop cells a non-empty cell grid-dominates (default 1) */
  sky_rep rep;                 /* representative filtering (Section 4.1) */
  uint32_t reps_per_partition; /* Sorted representatives per partition (default 1) */
  sky_merge merge;             /* final phase (Section 4.2) */
  sky_exec exec;               /* launch form of the local-skyline phase */
  /* tuning knobs of the dominance engine; 0 selects the built-in default */
  uint32_t chunk_min;          /* smallest SFS chunk of a partition (points; default 1024) */
  uint32_t chunk_max;          /* largest SFS chunk of a partition (points; default 262144) */
  uint32_t chunk_alpha_x4;     /* next chunk = alpha/4 x current window size, clamped (default 32) */
  uint32_t dom_block;          /* dominator block per work item (points, multiple of 32, <= 2048; default 1024) */
  uint32_t engine_warps;       /* warps per CTA of the engine's work items: 4 or 8 (default 4) */
  uint32_t engine_cands;       /* candidates per lane: 2 or 4 (default 4); a work item's tile is
                                  32 x engine_warps x engine_cands candidates */
  sky_images images;           /* images of the engine's first test (default SKY_IMAGES_VALUES) */
} sky_params;

/* Per-call statistics (sky_get_stats). */
typedef struct {
  uint64_t n;                  /* input points */
  uint32_t d;
  uint32_t partitions;         /* p after clamping */
  uint32_t nonempty_partitions; /* partitions holding at least one point (before Grid Filtering) */
  uint32_t rounds_local;       /* SFS rounds of the local phase (max over partitions) */
  uint32_t rounds_merge;       /* SFS rounds of the sequential merge */
  uint32_t reps_kept;          /* representatives left after removing dominated ones */
  uint64_t grid_dropped;       /* points in cells removed by Grid Filtering */
  uint64_t rep_dropped;        /* points removed by representatives */
  uint64_t local_union;        /* |u| = sum of local skyline sizes */
  uint64_t skyline;            /* |Sky(r)| */
  double ms_total;             /* device time of the whole call (0 unless timing is on) */
  double ms_phase[6];          /* prep+sort (after a host input's copy to the device), filters, local,
                                  merge, output, host copies */
  uint64_t launches;           /* CUDA kernels the call launched */
  double ms_dom_local;         /* device time of the local-skyline dominance launches (timing on) */
  double ms_dom_merge;         /* device time of the final-phase dominance launch (timing on) */
  uint64_t tests_fp16;         /* dominance tests of the engine's launches (local phase and sequential
                                  merge; not NoSeq's): candidate slots x staged dominators its 16-bit
                                  image test covered, slots of candidates already dead included */
  uint64_t tests_fp16_local;   /* the part of tests_fp16 made by the local phase */
} sky_stats;

typedef struct sky_ctx sky_ctx;

/* Fills *p with the defaults: SKY_NONE, p = 1, slices 1, grid_filter 1,
   reps_per_partition 1, sequential merge, persistent launch. */
void sky_params_init(sky_params* p);

/* Creates a context on CUDA device `device` whose scratch memory may grow up
   to mem_budget_bytes (0 = no limit but the device's).  The context starts
   on the legacy default stream.  On failure *ctx is NULL. */
sky_status sky_create(sky_ctx** ctx, int device, size_t mem_budget_bytes);

/* Runs every later call of the context on `cuda_stream` (a cudaStream_t of
   the context's device; NULL = legacy default stream).  The stream is not
   owned by the context. */
sky_status sky_set_stream(sky_ctx* ctx, void* cuda_stream);

/* Turns per-phase CUDA-event timing of the statistics on (1) or off (0). */
sky_status sky_set_timing(sky_ctx* ctx, int on);

/* Sky(points) by Algorithm 2 with the given parameters (NULL = defaults).
   points: N x d FP32 row-major (host or device).  out_idx: capacity >= N
   (host or device); receives the |Sky| ascending indices.  *out_count
   (host) receives |Sky|.  N = 0 returns SKY_OK with count 0.  Blocks until
   the result is in out_idx. */
sky_status sky_skyline(sky_ctx* ctx, const float* points, uint64_t n, uint32_t d,
                       const sky_params* params, uint32_t* out_idx, uint64_t* out_count);

/* sky_skyline plus per-point diagnostics in input order (each may be NULL;
   host or device, capacity >= N):
     out_pid[i]   partition of point i (Section 3 index formula of the scheme);
     out_stage[i] where point i left the method: 1 in Sky(r), 2 in a cell
                  removed by Grid Filtering, 3 dominated by a representative,
                  4 dominated inside its partition, 5 in u but not in Sky(r). */
sky_status sky_skyline_ex(sky_ctx* ctx, const float* points, uint64_t n, uint32_t d,
                          const sky_params* params, uint32_t* out_idx, uint64_t* out_count,
                          uint32_t* out_pid, uint8_t* out_stage);

/* One query of a batch (sky_skyline_batch). */
typedef struct {
  const float* points;       /* N x d FP32 row-major, host or device */
  uint64_t n;
  uint32_t d;
  const sky_params* params;  /* NULL = defaults */
  uint32_t* out_idx;         /* capacity >= N, host or device */
  uint64_t* out_count;       /* host */
  sky_status status;         /* out: this query's status */
} sky_query;

/* Runs nq independent skyline queries as one batch: the partitions of all
   queries are computed in one persistent launch of the dominance engine
   (Algorithm 2's local phase for every query at once) and the sequential
   final phases of all queries in a second one, so that many queries of
   uneven size fill the GPU together.  Each query's result equals what
   sky_skyline returns for it alone.  Arguments are checked before any work
   starts: an invalid query fails the whole call (its status says which).
   Queries asking for SKY_EXEC_PLAIN get their own launches.  Blocks until
   every result is in its out_idx.  The statistics of the context become
   the batch's (sums over queries; maxima of round counts). */
sky_status sky_skyline_batch(sky_ctx* ctx, sky_query* queries, uint32_t nq);

/* Autotuner of the dominance engine's knobs (chunk_min, chunk_max,
   chunk_alpha_x4, dom_block, engine_warps, engine_cands of sky_params):
   the SFS chunk sizes of the engine's rounds, the dominator block a CTA
   stages in shared memory, and the launch shape (warps per CTA and
   candidates per lane, i.e. the tile width of a work item and the warps
   that share a partition's tile).  They decide how Algorithm 1 is cut into
   parallel work, never the result.
   Runs the query (points, n, d with the method parameters in *params) up
   to max_trials times (0 = 48) with candidate knobs, timing each run with
   CUDA events on the context's stream (coordinate descent from the
   defaults, two sweeps), and writes the fastest knobs into *params;
   *best_ms receives its time.  Blocks; allocates one N-index device buffer
   for the trial outputs. */
sky_status sky_autotune(sky_ctx* ctx, const float* points, uint64_t n, uint32_t d, sky_params* params,
                        uint32_t max_trials, double* best_ms);

/* sky_autotune for a batch run by sky_skyline_batch: one set of knobs for
   all queries (the queries share the engine's launches, so the best knobs
   of a batch differ from those of its queries alone).  queries[i].params
   hold the method parameters (their knobs are ignored); out_idx and
   out_count of the queries are not used.  The six knob fields of *knobs
   (struct_size set, e.g. by sky_params_init) receive the result. */
sky_status sky_autotune_batch(sky_ctx* ctx, const sky_query* queries, uint32_t nq, uint32_t max_trials,
                              sky_params* knobs, double* best_ms);

/* ---- CUDA graphs ------------------------------------------------------
   A batch (as sky_skyline_batch would run it) captured into a CUDA graph and
   replayed with one graph launch: for a batch that is run again and again
   over the same device buffers (inputs rewritten in place between runs),
   the host's per-launch cost is paid once, at capture.  The graph owns its
   own workspace, pinned staging and stream, so later calls on the context
   cannot move its buffers.  Inputs and outputs must be device memory (the
   per-point diagnostics are not captured); shapes, parameters and pointers
   are fixed at capture.  Results equal sky_skyline_batch's. */
typedef struct sky_graph sky_graph;

/* Captures the batch (queries[i].out_count are ignored).  SKY_EINVAL for
   invalid queries or host pointers; SKY_ECUDA if capture or instantiation
   fails; *graph is NULL on failure.  The context's memory budget applies to
   the graph's workspace. */
sky_status sky_graph_capture(sky_ctx* ctx, const sky_query* queries, uint32_t nq, sky_graph** graph);

/* Replays the graph after the work already queued on the context's stream
   (at capture time) and waits for it.  out_counts (host, nq entries, may be
   NULL) receive each query's |Sky|; *ms (may be NULL) the device time of
   the replay.  Returns the first failing query's status. */
sky_status sky_graph_launch(sky_graph* graph, uint64_t* out_counts, double* ms);

void sky_graph_destroy(sky_graph* graph);

/* ---- serving: a request loop with continuous batching ----------------
   sky_submit queues a query and returns at once.  Worker threads of the
   context take queued queries in arrival order into batches whose device
   memory fits their share of the serving budget, run each batch like
   sky_skyline_batch on their own stream (the workspaces stay resident
   between batches), and publish every query's result.  Queries that arrive
   while a batch is on the GPU join the next batch of the first worker that
   frees up; with two or more workers one batch's copies and memory-bound
   stages overlap another's dominance kernel.  Each result equals what
   sky_skyline returns for the query alone.  sky_submit, sky_poll and
   sky_wait may be called from several host threads at once. */
typedef struct {
  uint32_t struct_size;       /* sizeof(sky_serve_config); set by sky_serve_config_init */
  uint32_t workers;           /* batches in flight (streams); default 2 */
  uint32_t max_batch;         /* queries per batch; default 64 */
  uint64_t mem_budget_bytes;  /* device memory of all workers' workspaces; 0 = half the free memory */
} sky_serve_config;

typedef struct {
  double queue_us;            /* submit to the start of its batch */
  double run_us;              /* start of its batch to its result */
  double latency_us;          /* submit to result */
  uint32_t batch_queries;     /* queries in its batch */
} sky_ticket_info;

void sky_serve_config_init(sky_serve_config* cfg);

/* Device memory (bytes) that one query of this shape takes in a batch: the
   figure the serving loop admits queries by.  0 if the arguments are
   invalid. */
uint64_t sky_query_bytes(uint64_t n, uint32_t d, const sky_params* params);

/* Starts the serving loop of the context (cfg NULL = defaults).  Called
   implicitly with the defaults by the first sky_submit.  SKY_EBUSY if it
   is already running. */
sky_status sky_serve_start(sky_ctx* ctx, const sky_serve_config* cfg);

/* Queues Sky(points) with the given parameters (NULL = defaults); *ticket
   receives its handle.  points (host or device, N x d FP32 row-major) must
   stay valid and unchanged until the ticket completes.  Arguments are
   checked here (SKY_EINVAL); device-side failures are reported by
   sky_wait. */
sky_status sky_submit(sky_ctx* ctx, const float* points, uint64_t n, uint32_t d, const sky_params* params,
                      uint64_t* ticket);

/* SKY_OK if the ticket has completed, SKY_EBUSY if it has not,
   SKY_ECANCELLED if it is unknown or already collected. */
sky_status sky_poll(sky_ctx* ctx, uint64_t ticket);

/* Waits up to timeout_us (negative = no limit) for the ticket, copies its
   |Sky| ascending indices to out_idx (host or device, capacity >= N),
   *out_count = |Sky|, fills *info if not NULL, and releases the ticket.
   SKY_EBUSY on timeout (the ticket stays valid), SKY_ECANCELLED for an
   unknown or collected ticket, else the query's own status. */
sky_status sky_wait(sky_ctx* ctx, uint64_t ticket, uint32_t* out_idx, uint64_t* out_count, int64_t timeout_us,
                    sky_ticket_info* info);

/* Runs the queued queries to completion and stops the workers (their
   workspaces are freed).  Uncollected tickets stay collectable. */
sky_status sky_serve_stop(sky_ctx* ctx);

/* Rank space of a point set (Def. 1 compares each attribute only by order,
   so replacing every value by its rank in its column keeps every dominance
   relation and the skyline).  points: N x d FP32 row-major (host or
   device); -0.0 and +0.0 are one value.  Outputs (each may be NULL; host or
   device):
     out_ranks[i*d + a]  dense rank of points[i*d + a] in column a: the
                         number of distinct values of column a below it
                         (0 .. distinct - 1; equal values, equal ranks);
     out_distinct[a]     number of distinct values of column a;
     out_codes[i*d + a]  the 15-bit code that SKY_IMAGES_RANKS gives the
                         engine: the rank itself when the column has at most
                         31,744 distinct values, else floor(rank x 31,743 /
                         (distinct - 1)); read as the bits of an FP16
                         number, the codes are finite, non-negative and
                         non-decreasing in the value.
   Blocks until the outputs are written.  Errors: SKY_EINVAL for d outside
   1..8, N >= 2^32 - 1, NULL points with N > 0, memory of another GPU, or a
   NaN attribute; SKY_ENOMEM; SKY_ECUDA.  N = 0 writes only out_distinct
   (zeros). */
sky_status sky_rank_space(sky_ctx* ctx, const float* points, uint64_t n, uint32_t d, uint32_t* out_ranks,
                          uint32_t* out_distinct, uint16_t* out_codes);

/* Statistics of a call.  ticket_or_0 = 0: the last completed sky_skyline,
   sky_skyline_ex or sky_skyline_batch call of the context (a batch's sizes
   and counts are sums over its queries, its round counts maxima).  A
   serving ticket: that query's own sizes and counts (Section 3 partitions,
   filtered points, |u|, |Sky|), with the launches, engine test counts and
   device times of the batch it ran in (device times only when
   sky_set_timing was on when the serving loop started); available from completion until long after
   sky_wait collects the ticket (the last 4096 collected tickets are kept).
   SKY_EBUSY if the ticket has not completed, SKY_ECANCELLED if it is
   unknown, SKY_EINVAL for NULL arguments. */
sky_status sky_get_stats(sky_ctx* ctx, uint64_t ticket_or_0, sky_stats* out);

/* Text of a status code (static storage). */
const char* sky_status_str(sky_status s);

/* Message of the last failing call of the context (static while the context lives). */
const char* sky_last_error(sky_ctx* ctx);

/* Frees the context and its device memory (synchronises its stream first). */
void sky_destroy(sky_ctx* ctx);

/* Largest N accepted by sky_skyline_static. */
#define SKY_STATIC_MAX_POINTS 65536u

/* The paper has no counterpart to this call: it serves callers that cannot
   allocate device memory when they need a skyline -- code running under an
   allocator that owns all of the GPU's memory and forbids cudaMalloc, a
   latency-critical loop in which an allocation or the synchronisation of a
   cudaFree is not acceptable, or code that must keep a fixed footprint.
   It needs no context and allocates nothing: its scratch (about 2.4 MB) is
   one file-scope device array of the library, reserved on every GPU that
   loads the library until the process exits.

   The skyline of a small point set, the same set sky_skyline returns:
   points is device memory of the current device (or managed memory),
   row-major N x d FP32, read-only; out_idx is device memory of the current
   device of capacity >= N and receives the |Sky| ascending indices;
   *out_count (host) receives |Sky|.  The work runs on cuda_stream (NULL =
   legacy default stream); the call copies the count to the host and waits
   for the stream before it returns.  Errors: SKY_EINVAL for d outside 1..8,
   N > SKY_STATIC_MAX_POINTS, NULL pointers, host memory or memory of
   another GPU, or a NaN attribute; SKY_ECUDA if a CUDA call fails.  N = 0
   returns SKY_OK with count 0.

   The first call on a device looks up the array's device address on that
   device (the current one) and caches it, so it should come before any
   stream capture; after a cudaDeviceReset the next call looks it up again.
   Every call reuses the same array, so calls whose work overlaps on the
   GPU -- from several host threads or on several streams at once -- race
   and must not be made. */
sky_status sky_skyline_static(const float* points, uint64_t n, uint32_t d, uint32_t* out_idx,
                              uint64_t* out_count, void* cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* SKYLINE_H_ */
