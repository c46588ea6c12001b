/* Multi-threaded CPU MPDP: the paper's own CPU implementation of the method
 * (Sec. 3.3 "MPDP on CPU"), the "MPDP (24CPU)" system its experiments
 * compare the GPU against (Sec. 7.2).  A comparison baseline that runs on
 * the host cores; it shares no code with the GPU library and is not a
 * fallback of it.
 *
 * It computes the same exact result as mpdp_optimize in MPDP_MODE_EXACT
 * with the C_out cost model: the optimal cross-product-free bushy plan,
 * with card(S) by peeling the highest non-cut vertex (selectivities of its
 * neighbours in ascending order), and among equally cheap splits the one
 * whose smaller side has the smallest relation bitmap.  Costs are IEEE
 * binary64 with every addition and multiplication rounded on its own.
 *
 * Build: libmpdp_cpu.so (plain C11 + pthreads), next to libmpdp.so.
 */
#ifndef MPDP_CPU_H
#define MPDP_CPU_H

#include <stdint.h>

#include "mpdp.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Largest query the dense memo of this baseline takes (2^n entries of
 * 20 bytes: 671 MB at 25 relations, 21 GB at 30). */
#define MPDP_CPU_MAX_RELS 30

typedef struct {
    uint64_t sets_unranked;   /* k-subsets (k >= 2) unranked by the workers */
    uint64_t sets_connected;  /* of those, connected */
    uint64_t pairs_evaluated; /* unordered block bipartitions examined (Algorithm 4) */
    uint64_t ccp_pairs;       /* unordered CCP pairs */
    int32_t threads;          /* worker threads used */
    int32_t reserved;
    double wall_ms;           /* wall time of the level loop */
} mpdp_cpu_stats;

/* Optimize one query on `threads` host threads (0: every online core).
 *
 * card: [n_rels] base cardinalities, finite and > 0.  edges: [n_edges]
 * join predicates (0 <= u, v < n, u != v, 0 < sel <= 1, no duplicates).
 * The caller owns every array; nothing is kept after the call returns.
 * nodes: caller buffer of cap >= 2n - 1 plan nodes (may be NULL with cap 0
 * to read only the cost); the plan is written in breadth-first order from
 * the root, the left child being the side with the smaller relation bitmap.
 * n_nodes, cost and st may be NULL.
 *
 * Returns MPDP_OK; MPDP_ERR_INVALID_ARG for a bad value, index or duplicate
 * edge; MPDP_ERR_DISCONNECTED when the join graph is not connected;
 * MPDP_ERR_TOO_LARGE for n_rels > MPDP_CPU_MAX_RELS; MPDP_ERR_OOM when the
 * memo cannot be allocated; MPDP_ERR_BUFFER_TOO_SMALL when 0 < cap < 2n-1.
 * Level k is a barrier: every worker finishes level k before any starts
 * k + 1; within a level workers take chunks of consecutive ranks from a
 * shared atomic counter. */
int mpdp_cpu_optimize(int32_t n_rels, const double *card, int32_t n_edges, const mpdp_edge *edges,
                      int32_t threads, mpdp_plan_node *nodes, int32_t cap, int32_t *n_nodes, double *cost,
                      mpdp_cpu_stats *st);

#ifdef __cplusplus
}
#endif

#endif /* MPDP_CPU_H */
