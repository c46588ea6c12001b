/*
 * mpdp.h - C ABI of the GB300 (sm_103a) MPDP join-order optimizer.
 *
 * The library finds the cheapest bushy join tree without cross products for a
 * query join graph, with the MPDP dynamic program of "Efficient Massively
 * Parallel Join Optimization for Large Queries" (arXiv 2202.13511):
 *   - the DP runs level by level over relation-set sizes k = 2..n (Sec. 2.1.1,
 *     the level dependency rule; Sec. 5, Algorithm "MPDP on GPU");
 *   - each level unranks every k-subset, keeps the connected ones (Sec. 5,
 *     "Unrank", "Filter"), enumerates their CCP pairs either by removing each
 *     edge (tree join graphs, Algorithm 2, Sec. 3.1) or block by block
 *     (Algorithm 4, Sec. 3.2), costs every pair, keeps the best per set
 *     ("Prune", fused) and stores it in the memo ("Scatter");
 *   - the plan is fetched recursively from the memo (Sec. 5, last paragraph).
 *
 * Cost model (the paper's own is unspecified, Sec. 7.1): C_out.
 *   cost({R_i}) = 0;  cost(L join R) = (cost(L) + cost(R)) + card(L u R).
 *   card(S) is a product taken in an order fixed by S alone ("peeling"):
 *   card({r}) = card[r]; otherwise v is the highest-index relation of S
 *   whose removal leaves G[S] with no more components (for a connected S its
 *   highest non-cut vertex) and card(S) = ((card(S \ {v}) * card[v]) *
 *   sel(j1, v)) * sel(j2, v) ... over v's neighbours j1 < j2 < ... in S.
 *   All arithmetic is IEEE-754 binary64, round to nearest, no fused
 *   multiply-add.
 * Ties: the chosen split of S is the lexicographic minimum of (x, left),
 * x = cost(S_left) + cost(S_right) and left the numerically smaller of the
 * two relation bitmaps; cost(S) = x + card(S).
 * Results are therefore bit-identical to any exact DP with the same rules.
 *
 * Relation sets are bitmaps: bit i is relation i.
 * All functions return 0 (MPDP_OK) or a negative MPDP_ERR_* code; none of them
 * aborts.  A context is used by one host thread at a time.
 */
#ifndef MPDP_H
#define MPDP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MPDP_ABI_VERSION 6
/* Exact mode uses 32-bit relation bitmaps; memory grows as 2^n (see
 * mpdp_workspace_bytes), so n is further capped by the memo budget. */
#define MPDP_MAX_EXACT_RELS 30
/* Heuristic modes (IDP2, UnionDP): relations of one query. */
#define MPDP_MAX_HEURISTIC_RELS 4096
#define MPDP_MAX_LEVELS 33
/* Concurrent sub-batches of one device batch (mpdp_config.lanes). */
#define MPDP_MAX_LANES 8

enum {
    MPDP_OK = 0,
    MPDP_ERR_INVALID_ARG = -1,      /* bad index, duplicate edge, non-finite or <= 0 value */
    MPDP_ERR_DISCONNECTED = -2,     /* no plan without cross products exists */
    MPDP_ERR_TOO_LARGE = -3,        /* n above the mode's limit */
    MPDP_ERR_OOM = -4,              /* device allocation failed or memo arena full */
    MPDP_ERR_ADMISSION = -5,        /* request exceeds the memo budget */
    MPDP_ERR_BUFFER_TOO_SMALL = -6, /* caller's node buffer has fewer than 2n-1 entries */
    MPDP_ERR_TIMEOUT = -7,          /* a bounded device wait gave up */
    MPDP_ERR_PROBE_LIMIT = -8,      /* memo probe found no entry within the table */
    MPDP_ERR_CUDA = -9,             /* a CUDA runtime call failed */
    MPDP_ERR_BAD_HANDLE = -10,      /* unknown or released handle */
    MPDP_ERR_NOT_IMPLEMENTED = -11,
    MPDP_ERR_STALE = -12,           /* the handle's memo was overwritten by a later query */
    MPDP_ERR_INTERNAL = -13,        /* an internal consistency check failed */
    MPDP_ERR_NOT_READY = -14        /* the result is not available yet (server) */
};

enum { MPDP_COST_COUT = 0 };

enum {
    MPDP_MODE_EXACT = 0,
    MPDP_MODE_IDP2 = 1,
    MPDP_MODE_UNIONDP = 2,
    MPDP_MODE_IDP2_LEARNED = 3,
    MPDP_MODE_UNIONDP_LEARNED = 4,
    MPDP_MODE_UNIONDP_SIZEFIRST = 5,
    MPDP_MODE_IDP2_WEIGHT_START = 6
};

/* CCP enumeration: AUTO picks TREE when the join graph is a tree
 * (connected with n-1 edges), BLOCKS otherwise.  BLOCKS is correct on trees
 * too (every block is one edge). */
enum { MPDP_ENUM_AUTO = 0, MPDP_ENUM_TREE = 1, MPDP_ENUM_BLOCKS = 2, MPDP_ENUM_DPSUB = 3 };
/* MPDP_ENUM_DPSUB (an ablation baseline, not MPDP): the vertex-based
 * enumeration of DPSUB (Algorithm 1) on the same kernels: every bipartition
 * of a connected S with min(S) on the left is tested for a CCP, 2^(|S|-1) - 1
 * per set; same results, more pairs evaluated (reported as such). */

/* Memo layout.  DENSE: arrays indexed directly by the relation bitmap
 * (20 bytes x 2^n: {cost, card} and left); a tree-mode query whose connected
 * sets the filter unranks uses the bit-reversed bitmap instead (relation 0
 * the top bit), so that the sets the unranking lists side by side sit side
 * by side (an address permutation only).  HASH: one open-addressing table
 * per level, Murmur3 fmix32 hash, linear probing, 32-byte slots {key, left,
 * cost, card}, capacity the power of two >= 2x the level's connected-set
 * count (Sec. 5, memo of "MPDP on GPU"). */
enum { MPDP_MEMO_DENSE = 0, MPDP_MEMO_HASH = 1 };

/* Connected-set filter.  UNRANK: every k-subset of every level is unranked
 * with the combinatorial number system and stepped with the next bit
 * permutation (Sec. 5, "Unrank", "Filter").  BITMAPS: every bitmap below 2^n
 * is visited in index order (all levels at once, no unranking) and each
 * connected one goes straight into the list of its level.  CONNECTED
 * (default): a tree join graph whose connected sets number at most 2^n / 4
 * unranks them themselves (no disconnected set is ever formed); other
 * queries as BITMAPS.  The same sets reach the level lists in every mode.
 * sets_unranked counts the sets of two or more relations the filter forms:
 * 2^n - n - 1 for a sweep, the connected ones for the unranking. */
enum { MPDP_FILTER_BITMAPS = 0, MPDP_FILTER_UNRANK = 1, MPDP_FILTER_CONNECTED = 2 };

typedef struct mpdp_ctx mpdp_ctx; /* opaque, owned by the library */

/* One join predicate between relations u and v (0 <= u, v < n, u != v) with
 * selectivity 0 < sel <= 1.  No duplicate pairs. 16 bytes. */
typedef struct {
    int32_t u, v;
    double sel;
} mpdp_edge;

/* A query as host arrays.  The library copies everything it needs before
 * mpdp_optimize returns; the caller keeps ownership. */
typedef struct {
    int32_t n_rels;          /* number of relations, >= 1 */
    int32_t n_edges;         /* number of join predicates */
    const double *card;      /* [n_rels] base cardinalities, finite and > 0 */
    const mpdp_edge *edges;  /* [n_edges] */
    int32_t cost_model;      /* MPDP_COST_COUT */
    int32_t mode;            /* MPDP_MODE_* */
    int32_t k;               /* heuristic sub-problem size (IDP2 / UnionDP), <= 25;
                                IDP2 with k <= 1 returns GOO's plan */
    int32_t t;               /* UnionDP partition threshold, 2..k (0: k); 0 in
                                the other modes */
} mpdp_query;

/* One node of the result plan.  Node 0 is the root; children have larger
 * indices than their parent (breadth-first order).  40 bytes. */
typedef struct {
    int32_t left, right;  /* child node indices; -1 for a leaf */
    int32_t rel;          /* leaf: relation index; join: -1 */
    int32_t n_leaves;     /* relations under this node */
    uint64_t set;         /* relation bitmap of the node (0 if n > 64) */
    double card;          /* card(set) */
    double cost;          /* C_out cost of the subtree (0 for a leaf) */
} mpdp_plan_node;

/* Counters of one optimization (Sec. 2.2: EvaluatedCounter and CCP-Counter).
 * pairs_evaluated counts the join pairs the enumeration examined: one per
 * edge of G[S] in tree mode (Algorithm 2), one per unordered bipartition
 * {lb, rb} of each block in block mode (Algorithm 4's loop over every
 * non-empty proper lb visits each of these twice).  ccp_pairs counts each
 * unordered CCP pair once. */
typedef struct {
    uint64_t sets_unranked;    /* sets of k = 2..n relations formed by the filter */
    uint64_t sets_connected;   /* connected sets, k = 2..n */
    uint64_t pairs_evaluated;
    uint64_t ccp_pairs;
    uint64_t memo_bytes;       /* device bytes of the memo used by this query */
    uint64_t heavy_sets;       /* block mode: sets evaluated by the chunked heavy-set kernel */
    double device_ms;          /* device time of the batch's DP, from after its
                                  upload and staging to the end of plan fetch (CUDA
                                  events) */
    int32_t enumeration;       /* MPDP_ENUM_TREE or MPDP_ENUM_BLOCKS as run */
    int32_t memo_kind;         /* MPDP_MEMO_* as run */
    uint64_t h2d_bytes;        /* host -> device bytes copied for this query: its
                                  descriptor, cards and edges in the batch's one
                                  upload copy; the batch's first query also carries
                                  the filter prefixes and alignment padding, so the
                                  batch's queries sum to the copy's size */
    uint64_t d2h_bytes;        /* device -> host bytes copied for this query */
    uint64_t filter_steps;     /* BFS rounds run by the filter for sets with no isolated vertex */
    uint64_t connected_per_level[MPDP_MAX_LEVELS];
    uint64_t evaluated_per_level[MPDP_MAX_LEVELS];
    uint64_t ccp_per_level[MPDP_MAX_LEVELS];
} mpdp_stats;

/* Tuning knobs; mpdp_get_config returns the defaults of a new context. */
typedef struct {
    int32_t memo_kind;        /* MPDP_MEMO_DENSE (default) or MPDP_MEMO_HASH */
    int32_t enumeration;      /* MPDP_ENUM_AUTO (default), _TREE, _BLOCKS */
    int32_t heavy_threshold;  /* block mode: a set whose work exceeds this goes
                                 to the heavy-set kernel, one warp per chunk of
                                 at most 2048 pairs (default 64).  Clique
                                 blocks: their pairs, / 16 on a level of at
                                 least 16384 sets, against this limit (half of
                                 it on a smaller level).  Other blocks: their
                                 bipartitions, or their CCPs where listed,
                                 against this limit x the level's sets / 65536,
                                 kept within a quarter and twice this limit.
                                 A set with both weighs each part against its
                                 own limit.  Results do not depend on it. */
    int32_t use_ccc;          /* 1 (default): collaborative context collection
                                 in the heavy-set kernel (Sec. 5) */
    int32_t use_graphs;       /* 1 (default): replay a captured CUDA graph per shape */
    int32_t run_length;       /* MPDP_FILTER_UNRANK: k-subsets unranked per lane
                                 (1..32, default 32) */
    int32_t filter;           /* MPDP_FILTER_CONNECTED (default), _BITMAPS or _UNRANK */
    int32_t grid_blocks_per_sm; /* evaluate grids: at most this many 256-thread
                                 blocks per SM (1..32, default 8) */
    int32_t lanes;            /* a device batch runs as up to this many
                                 sub-batches of consecutive queries, balanced
                                 by 2^n, on concurrent streams, so that one
                                 sub-batch's filter (integer-issue bound)
                                 overlaps another's evaluation (memo-traffic
                                 bound); 1..MPDP_MAX_LANES, default 4.
                                 Results do not depend on it. */
    int32_t fuse_prune;       /* 1 (default): tree-mode levels evaluate, prune
                                 and scatter in one kernel.  0: an ablation of
                                 that fusion (Sec. 5): one kernel writes every
                                 CCP pair's (cost sum, left) to a buffer of
                                 16 B x the largest level's sets x (k - 1),
                                 a second prunes and scatters.  Same results. */
    int32_t group_threads_log2; /* per-level work split of tree-mode levels: a
                                 level with k >= 4 whose sets x G stay within
                                 2^group_threads_log2 threads (G, the power of
                                 two at or above k - 1) runs G lanes per set,
                                 one split each; other levels run a thread per
                                 set.  0 (never groups) or 8..24; default 18.
                                 Results do not depend on it. */
} mpdp_config;

/* Create a context on CUDA device `device`.  memo_budget_bytes caps the device
 * workspace (0 = 64 GiB).  cuda_stream is a cudaStream_t borrowed for all work
 * of the context; NULL means the CUDA default stream.  The caller keeps the
 * stream alive for the life of the context. */
int mpdp_create(mpdp_ctx **out, int device, size_t memo_budget_bytes, void *cuda_stream);
void mpdp_destroy(mpdp_ctx *ctx);
int mpdp_set_config(mpdp_ctx *ctx, const mpdp_config *cfg);
int mpdp_get_config(const mpdp_ctx *ctx, mpdp_config *cfg);

/* Device workspace the exact mode needs for n relations under cfg. */
size_t mpdp_workspace_bytes(int32_t n_rels, const mpdp_config *cfg);

/* Validate the query on the host, enqueue its optimization on the context's
 * stream and return a handle at once (asynchronous).  Exact mode: n <= 30.
 * Heuristic modes (Sec. 4): MPDP_MODE_IDP2 (GOO's plan, then IDP2 with
 * sub-problems of at most k <= 25 relations) and MPDP_MODE_UNIONDP
 * (Algorithm 5 with partitions of at most t and a final DP of at most k:
 * each round orders its edges once, before the union loop, by increasing
 * weight = the card of joining the edge's two nodes, ties by node ids, and
 * unites the sets across each edge in one pass while their size sum stays
 * within t), n <= MPDP_MAX_HEURISTIC_RELS.  MPDP_MODE_UNIONDP_SIZEFIRST is
 * a comparison reading of the same algorithm: after every union the next
 * edge is the one between different sets with the least (current size
 * sum, weight, node ids), and an edge whose sum exceeds t is dropped.
 * n <= MPDP_MAX_HEURISTIC_RELS.  Every sub-problem is solved exactly on the
 * device in extended range; these modes run to completion before the call
 * returns.  Plan nodes of n > 64 relations carry set = 0.
 * MPDP_MODE_UNIONDP_LEARNED: UnionDP whose partitions follow the learned
 * proposal set with mpdp_set_model (edges united in the order of the
 * model's scores), with plain UnionDP as the fallback: both plans are
 * costed exactly and the cheaper is returned (the plain one on ties, and
 * always when no model is set).  In the heuristic modes mpdp_stats carries
 * the number of exact sub-problems in heavy_sets and, for the learned
 * modes, filter_steps = 1 when the learned plan was kept.
 * MPDP_MODE_IDP2_LEARNED: IDP2 started from the learned proposal's plan
 * instead of GOO's (the query's edges in ascending score, each joining the
 * plans of its two ends while they are apart; equal scores in edge order
 * (min(u, v), max(u, v))), with IDP2 from GOO's plan as the fallback: the
 * cheaper plan is returned (GOO's on ties, and always when no model is
 * set).  t must be 0, as for MPDP_MODE_IDP2.
 * MPDP_MODE_IDP2_WEIGHT_START: the same rule with a start that needs no
 * model, a control for what the learned start adds: the query's edges in
 * ascending join card (card(u) * card(v) * sel(u, v)), each joining the
 * plans of its two ends while they are apart; IDP2 from GOO's plan is the
 * fallback, the cheaper plan is returned (GOO's on ties).  t must be 0.
 * mpdp_optimize_batch returns MPDP_ERR_NOT_IMPLEMENTED for any mode but
 * exact. */
int mpdp_optimize(mpdp_ctx *ctx, const mpdp_query *q, int64_t *handle);

/* Enqueue nq queries as device batches (all queries of a batch share every
 * kernel launch; a batch is split only when it would exceed the memo budget
 * or 1024 queries); handles[i] receives each one's handle.  The whole call is
 * validated first: on an error nothing is enqueued. */
int mpdp_optimize_batch(mpdp_ctx *ctx, const mpdp_query *qs, int32_t nq, int64_t *handles);

/* Block until the handle's optimization is done and copy out its plan.
 * nodes: caller buffer of cap >= 2n-1 entries (may be NULL when cap == 0 to
 * read only cost / stats).  n_nodes, cost, st may be NULL. */
int mpdp_get_plan(mpdp_ctx *ctx, int64_t handle, mpdp_plan_node *nodes, int32_t cap,
                  int32_t *n_nodes, double *cost, mpdp_stats *st);

/* Forget a handle (its host result buffer is reused). */
int mpdp_release(mpdp_ctx *ctx, int64_t handle);

/* The plan cost of a handle in extended range: cost = mant * 2^exp2 with
 * mant = 0 or 1 <= mant < 2 (heuristic plans of hundreds of relations cost
 * more than binary64 holds; mpdp_get_plan's cost is then +inf).  No
 * counterpart in the paper.  Blocks like mpdp_get_plan. */
int mpdp_get_cost_xd(mpdp_ctx *ctx, int64_t handle, double *mant, int32_t *exp2);

/* mpdp_get_plan + mpdp_release for `count` handles in one call (no
 * counterpart in the paper; it saves a host round trip per query when a
 * batch is collected).  Handle i's plan goes to nodes + i * stride (stride
 * >= 2n - 1 of every query, or nodes NULL and stride 0 to read only costs
 * and stats); n_nodes[i], costs[i] and status[i] (0 or that handle's
 * MPDP_ERR_*) are always written; stats may be NULL, else `count` records.
 * Every known handle is released, whatever its status.  Returns MPDP_OK,
 * or MPDP_ERR_BAD_HANDLE if a handle was unknown (its status says so too). */
int mpdp_get_plans(mpdp_ctx *ctx, const int64_t *handles, int32_t count, mpdp_plan_node *nodes,
                   int32_t stride, int32_t *n_nodes, double *costs, int32_t *status,
                   mpdp_stats *stats);

/* Plan nodes reserved per query in the device-path output arrays. */
#define MPDP_PLAN_STRIDE 63

/* Device-resident batch: the nq queries' inputs and outputs are device
 * pointers; everything is enqueued on the context's stream as one device
 * batch (shared launches) and nothing waits for the device.
 *   n_rels[nq], n_edges[nq]: HOST arrays of the queries' sizes (they size the
 *     launches; exact mode needs n <= 30);
 *   d_card: device, the queries' cardinalities back to back (sum of n_rels);
 *   d_edges: device, the queries' edges back to back (sum of n_edges);
 *     contents are validated on the device;
 *   d_nodes: device, nq * MPDP_PLAN_STRIDE plan nodes (query i at
 *     i * MPDP_PLAN_STRIDE); d_cost: nq doubles; d_status: nq int32 receiving
 *     0 or an MPDP_ERR_* code once the work has run.
 * Returns MPDP_OK when the work was enqueued, MPDP_ERR_ADMISSION when the
 * batch does not fit the memo budget, MPDP_ERR_TOO_LARGE for nq > 1024. */
int mpdp_optimize_batch_device(mpdp_ctx *ctx, int32_t nq, const int32_t *n_rels,
                               const int32_t *n_edges, const double *d_card,
                               const mpdp_edge *d_edges, int32_t cost_model,
                               mpdp_plan_node *d_nodes, double *d_cost, int32_t *d_status);

/* Device-resident form of one query (a batch of one). */
int mpdp_optimize_device(mpdp_ctx *ctx, int32_t n_rels, int32_t n_edges, const double *d_card,
                         const mpdp_edge *d_edges, int32_t cost_model, mpdp_plan_node *d_nodes,
                         double *d_cost, int32_t *d_status);

/* Allocation-free exact optimization of one small query.  The paper has no
 * counterpart: it is for callers that cannot allocate device memory.  No
 * context is involved and nothing is allocated: the dense memo is a fixed
 * device array inside the library of MPDP_NOALLOC_SCRATCH_BYTES
 * (2^16 sets x 20 bytes), which caps n_rels at MPDP_NOALLOC_MAX_RELS.  One
 * kernel of one block runs the whole DP (levels 2..n) and the plan fetch;
 * cost, plan and status are bit-identical to mpdp_optimize_device for the
 * same query.
 *   n_rels, n_edges: host values; d_card (n_rels doubles), d_edges (n_edges
 *     edges, may be NULL when 0): device, validated on the device as in the
 *     batched path; cost_model: MPDP_COST_COUT;
 *   d_nodes: device, at least 2 * n_rels - 1 plan nodes (breadth-first, as
 *     mpdp_optimize_device writes them); d_cost: 1 double; d_status: 1 int32
 *     receiving 0 or an MPDP_ERR_* code (on an error d_cost is 0 and d_nodes
 *     is not written);
 *   cuda_stream: a cudaStream_t of the current device (NULL: legacy default).
 * Returns MPDP_OK once the kernel is enqueued (nothing waits for it),
 * MPDP_ERR_TOO_LARGE for n_rels > MPDP_NOALLOC_MAX_RELS, MPDP_ERR_INVALID_ARG
 * for a NULL pointer, n_rels < 1, a bad n_edges or cost model, and
 * MPDP_ERR_CUDA when a runtime call fails.
 * Set-up: the first call in each context (in practice, on each device)
 * looks up the array's device address (cudaGetSymbolAddress) with that
 * device current; make that first call before any stream capture.  The
 * address is kept with the context's unique id, so after a device reset the
 * next call, in the new context, looks it up again.  Nothing in the array has to start at zero (a
 * call writes every entry before reading it).  Concurrency: every call on a
 * device uses the same array, so calls whose kernels can overlap on the GPU
 * (different streams, unordered host threads) race; order them on one
 * stream. */
#define MPDP_NOALLOC_MAX_RELS 16
#define MPDP_NOALLOC_SCRATCH_BYTES 1310720
int mpdp_optimize_device_noalloc(int32_t n_rels, int32_t n_edges, const double *d_card,
                                 const mpdp_edge *d_edges, int32_t cost_model,
                                 mpdp_plan_node *d_nodes, double *d_cost, int32_t *d_status,
                                 void *cuda_stream);

/* Wait for all work enqueued on the context's stream.  Device-reported
 * errors are delivered per query (mpdp_get_plan, or the d_status outputs). */
int mpdp_sync(mpdp_ctx *ctx);

/* Read memo entries of the most recent exact optimization of the context
 * (the handle must be that one, else MPDP_ERR_STALE).  sets: host array of
 * connected relation bitmaps; costs / lefts: host outputs.  A singleton reads
 * (0, 0).  Used to check every connected set against a reference. */
int mpdp_memo_lookup(mpdp_ctx *ctx, int64_t handle, const uint64_t *sets, int32_t count,
                     double *costs, uint64_t *lefts);

/* Number of kernel launches the last mpdp_optimize / _device call enqueued. */
int32_t mpdp_last_launch_count(const mpdp_ctx *ctx);

/* Kernel classes timed by the profiling mode. */
enum {
    MPDP_KC_STAGE = 0,   /* device-path input gather */
    MPDP_KC_INGEST = 1,  /* graph build and validation */
    MPDP_KC_FILTER = 2,  /* connectivity filter, all levels (with the level sort) */
    MPDP_KC_MEMO_INIT = 3, /* hash memo layout and clear; per-level tile prefixes */
    MPDP_KC_EVAL = 4,    /* per-level evaluate + prune + scatter (thread per set) */
    MPDP_KC_HEAVY = 5,   /* per-level block-per-set evaluation (block mode) */
    MPDP_KC_EXTRACT = 6, /* plan fetch */
    MPDP_KC_PUBLISH = 7, /* device-path output copy */
    MPDP_KC_COUNT = 8
};

/* Profiling modes (off by default).  While on, work is launched kernel by
 * kernel (no graph replay) with a pair of CUDA events around every launch, on
 * the stream it is launched on.  SERIAL runs a batch's lanes one after the
 * other on the context's stream, so that per-class times add up to the batch
 * (as a profiler's serialised launch list does); CONCURRENT runs them on
 * their own streams as in normal operation.  Any nonzero `mode` other than
 * these is invalid; 1 is SERIAL.
 * mpdp_profile_read waits for the stream, adds the elapsed times per kernel
 * class since the previous read into ms[MPDP_KC_COUNT] and the launch counts
 * into launches[MPDP_KC_COUNT], and resets them.  mpdp_profile_read_active
 * also returns, per class, the wall time during which at least one of its
 * launches was in flight (the union of the launch intervals within each
 * batch; equal to ms in SERIAL mode). */
enum { MPDP_PROFILE_OFF = 0, MPDP_PROFILE_SERIAL = 1, MPDP_PROFILE_CONCURRENT = 2 };
int mpdp_profile(mpdp_ctx *ctx, int mode);
int mpdp_profile_read(mpdp_ctx *ctx, double *ms, uint64_t *launches);
int mpdp_profile_read_active(mpdp_ctx *ctx, double *ms, double *active_ms, uint64_t *launches);

/* Static text for an error code. */
/* Measurement (not part of the method): read bandwidth of this GPU in GB/s,
 * the best of five launches that each read a `bytes` buffer `passes` times
 * (16-byte loads that bypass L1).  A buffer well below the L2 capacity
 * measures the L2; one far above it, HBM.  The buffer is allocated and freed
 * by the call; synchronous on the legacy stream. */
int mpdp_probe_read_gbs(int device, size_t bytes, int passes, double *gbs);

const char *mpdp_strerror(int code);
/* Text of the last CUDA error seen by this context (or ""). */
const char *mpdp_last_error(const mpdp_ctx *ctx);
int32_t mpdp_abi_version(void);

/* ---------------------------------------------------------------------
 * Serving loop (no counterpart in the paper): continuous batching of
 * optimization requests.  A server owns `slots` contexts, each with its own
 * CUDA stream and device workspace of slot_budget_bytes.  mpdp_server_submit
 * copies a request and queues it.  Whenever a slot is free, the queue's head
 * forms that slot's next device batch: requests join in arrival order while
 * the batch stays within max_batch queries and the slot's budget (admission
 * by memo memory).  Batches of different slots run concurrently on the GPU.
 * A request's plan is bit-identical to the same query optimized alone.
 * Progress happens inside submit / poll / drain; the library runs no
 * background thread.  A server is used by one host thread at a time.
 *
 * Persistent mode (persistent = 1): one resident kernel serves every request.
 * `slots` is then the number of query slots (1..1024), each holding one
 * query of up to the relations its slot_budget_bytes of workspace allows
 * (0: 25 relations; larger requests get MPDP_ERR_ADMISSION); max_batch is
 * not used.  A request goes to the device as soon as a slot is free, through
 * a ring in pinned, device-mapped memory that the running kernel polls; the
 * kernel advances every slot through ingest, filter, each DP level and the
 * plan fetch on its own, so requests that arrive while others are on the
 * GPU start at once and their levels overlap.  The kernel ends itself after
 * about 20 ms without work and is started again by the next submit or poll.
 * Needs the dense memo and the CONNECTED or BITMAPS filter. */
typedef struct mpdp_server mpdp_server; /* opaque, owned by the library */

typedef struct {
    int32_t slots;                /* concurrent device batches (1..16; default 4) */
    int32_t max_batch;            /* queries per device batch (1..1024; default 256) */
    uint64_t slot_budget_bytes;   /* device workspace per slot (0: 16 GiB) */
    mpdp_config kernel;           /* kernel configuration of every slot (default:
                                     context defaults with use_graphs = 0, since
                                     mixed batches rarely repeat a shape) */
    int32_t persistent;           /* 0 (default): device batches per slot; 1: one
                                     persistent kernel over query slots */
    int32_t pad;
} mpdp_server_config;

/* Fill *cfg with the defaults. */
int mpdp_server_default_config(mpdp_server_config *cfg);

/* Create a server on CUDA device `device` (cfg NULL: defaults). */
int mpdp_server_create(mpdp_server **out, int device, const mpdp_server_config *cfg);
void mpdp_server_destroy(mpdp_server *s);

/* Queue one exact-mode request (inputs copied before return) and make
 * progress.  *ticket identifies it.  The request is checked here as
 * mpdp_optimize checks a query (MPDP_ERR_INVALID_ARG, _DISCONNECTED,
 * _TOO_LARGE), so one bad request never fails a batch;
 * MPDP_ERR_ADMISSION: the query alone exceeds a slot's budget. */
int mpdp_server_submit(mpdp_server *s, const mpdp_query *q, int64_t *ticket);

/* Make progress without blocking: collect finished batches, start batches
 * on free slots.  The tickets finished by this call go to done[0..cap)
 * (done may be NULL when cap == 0); *count receives how many (count may be
 * NULL). */
int mpdp_server_poll(mpdp_server *s, int64_t *done, int32_t cap, int32_t *count);

/* Block until every submitted request has finished. */
int mpdp_server_drain(mpdp_server *s);

/* Requests waiting in the queue and on the device (either may be NULL). */
int mpdp_server_pending(const mpdp_server *s, int32_t *queued, int32_t *running);

/* Read and forget a finished request: its plan (cap >= 2n-1 nodes, nodes
 * may be NULL), cost, and latency from submit to the poll that saw it done,
 * in microseconds.  Returns the request's status (0 or its MPDP_ERR_*; the
 * request is forgotten either way), MPDP_ERR_NOT_READY if it has not
 * finished (it is kept), MPDP_ERR_BAD_HANDLE if unknown. */
int mpdp_server_result(mpdp_server *s, int64_t ticket, mpdp_plan_node *nodes, int32_t cap,
                       int32_t *n_nodes, double *cost, double *latency_us);

/* ---------------------------------------------------------------------
 * Learned proposal (a project addition; the paper only cites learned
 * optimizers): a 3 x 256 MLP that scores the edges of a query graph, trained
 * and run on the GPU by the library's own BF16 kernels (tensor-core
 * m16n8k16 products, FP32 accumulation, FP32 Adam).  Parameters (f32): W1
 * [n_in x 256], b1 [256], W2 [256 x 256], b2, W3 [256 x 256], b3, w4 [256],
 * b4 [1].  x and targets are device arrays of rows x n_in / rows floats. */
typedef struct mpdp_mlp mpdp_mlp;
int mpdp_mlp_create(mpdp_mlp **out, int device, int32_t n_in, void *cuda_stream);
void mpdp_mlp_destroy(mpdp_mlp *m);
int64_t mpdp_mlp_param_count(const mpdp_mlp *m);
/* Copy parameters in (resets the optimizer state) / out; host arrays. */
int mpdp_mlp_set_params(mpdp_mlp *m, const float *host, int64_t count);
int mpdp_mlp_get_params(mpdp_mlp *m, float *host, int64_t count);
/* y[rows] = MLP(x); device arrays; enqueued on the model's stream. */
int mpdp_mlp_forward(mpdp_mlp *m, const float *d_x, int32_t rows, float *d_y);
/* Gradients of L = sum (y - t)^2 / (2 rows) into host_grads (param_count
 * floats, may be NULL) and L into *loss (may be NULL); waits. */
int mpdp_mlp_gradients(mpdp_mlp *m, const float *d_x, const float *d_t, int32_t rows,
                       float *host_grads, double *loss);
/* One Adam step (beta 0.9 / 0.999) on L; enqueued. */
int mpdp_mlp_train_step(mpdp_mlp *m, const float *d_x, const float *d_t, int32_t rows, float lr);

/* Use `model` (MPDP_EDGE_FEATURES inputs; borrowed, NULL to detach) for
 * MPDP_MODE_UNIONDP_LEARNED and MPDP_MODE_IDP2_LEARNED on this context. */
#define MPDP_EDGE_FEATURES 12
int mpdp_set_model(mpdp_ctx *ctx, mpdp_mlp *model);
/* The model's input rows for the edges of a query graph, in edge order
 * (MPDP_EDGE_FEATURES floats each; cap_rows >= n_edges): the features the
 * learned UnionDP computes at every round and the learned IDP2 start
 * computes once, here for the base graph, so that training data uses the
 * same code. */
int mpdp_edge_features(const mpdp_query *q, float *out, int32_t cap_rows);

#ifdef __cplusplus
}
#endif
#endif /* MPDP_H */
