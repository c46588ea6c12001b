// Heuristic modes for queries too large for the exact DP (Sec. 4): IDP2
// with GOO's plan as the start (Sec. 4.1) and UnionDP (Algorithm 5).  Both
// run on the host and hand their sub-problems (at most 25 plans each) to the
// exact DP on the device in extended range (XD, mpdp_xd.cuh).
//
// Readings where the paper is silent:
//   * card of a join of plans L and R: ((card(L) * card(R)) * sel(e1)) *
//     sel(e2) ... over the query edges between them, ascending (min(u, v),
//     max(u, v)); cost(leaf) = 0, cost(L join R) = (cost(L) + cost(R)) +
//     card(L join R) (C_out), all in XD.
//   * a sub-problem over plans P_1..P_m numbers them by their smallest base
//     relation; relation i has card(P_i); one edge (i, j) when query edges
//     join P_i and P_j, with sel the product of their sels in the order above.
//   * GOO joins, while more than one tree is left, the two trees joined by an
//     edge whose join has the least card; ties by (smaller tree id, larger
//     tree id), a tree being named by its smallest relation; the tree with the
//     smaller relation goes left.
//   * IDP2(k) picks, while the working tree has more than one leaf, the
//     subtree with 2..k leaves whose joins cost most (leaves at cost 0: they
//     cannot change), the first in pre-order on ties, and replaces it by the
//     exact plan over its leaves.  k <= 1 returns GOO's plan.
//   * UnionDP(k, t) (Algorithm 5): at most k nodes -> one exact DP.
//     Otherwise each edge between nodes weighs the card of joining them;
//     union-find over nodes (size = nodes).  The edges are ordered once,
//     before the union loop, by (size of the sets across the edge, weight,
//     smaller node, larger node); every set is one node then, so this is
//     increasing weight.  One pass in that order unites the two sets across
//     an edge when they differ and their size sum is at most t.  Every set is
//     re-planned exactly and becomes a node of the next round.  t = k unless
//     given.
//   * UnionDP, size-first variant (MPDP_MODE_UNIONDP_SIZEFIRST): the next
//     edge is re-picked after every union as the one between different sets
//     with the least (current size sum, weight, smaller node, larger node),
//     united when the sum is at most t, else dropped (sizes only grow).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <functional>
#include <map>
#include <queue>
#include <vector>

#include "../../include/mpdp.h"
#include "mpdp_heuristic.h"
#include "mpdp_xd_exec.h"

namespace mpdp {

namespace {

struct PNode {
    int left = -1, right = -1, rel = -1;
    int minrel = 0, leaves = 1;
    XD card, cost;
    std::vector<int> rels;  // base relations, ascending
};

struct CutEdge {
    int u, v;  // u < v
    double sel;
    bool operator<(const CutEdge& o) const { return u != o.u ? u < o.u : v < o.v; }
};

class Heuristic {
public:
    Heuristic(const HeuristicQuery& q, XdExecutor& ex, cudaStream_t st, int sms)
        : n_(q.n), exec_(ex), st_(st), sms_(sms), mark_(q.n, 0), adj_(q.n)
    {
        for (int r = 0; r < n_; r++) card_.push_back(xd_make(q.card[r], 0));
        for (size_t e = 0; e < q.eu.size(); e++) {
            const int u = std::min(q.eu[e], q.ev[e]), v = std::max(q.eu[e], q.ev[e]);
            edges_.push_back(CutEdge{u, v, q.sel[e]});
            adj_[u].push_back({v, q.sel[e]});
            adj_[v].push_back({u, q.sel[e]});
        }
        std::sort(edges_.begin(), edges_.end());
    }

    int leaf(int r)
    {
        PNode p;
        p.rel = r;
        p.minrel = r;
        p.leaves = 1;
        p.card = card_[r];
        p.cost = xd_zero();
        p.rels = {r};
        nodes_.push_back(std::move(p));
        return (int)nodes_.size() - 1;
    }

    // query edges between the relation sets of plans a and b, ascending
    std::vector<CutEdge> cut(int a, int b)
    {
        const std::vector<int>* sa = &nodes_[a].rels;
        const std::vector<int>* sb = &nodes_[b].rels;
        if (sb->size() < sa->size()) std::swap(sa, sb);
        ++stamp_;
        for (int r : *sb) mark_[r] = stamp_;
        std::vector<CutEdge> out;
        for (int u : *sa)
            for (const auto& nb : adj_[u])
                if (mark_[nb.first] == stamp_) out.push_back(CutEdge{std::min(u, nb.first), std::max(u, nb.first), nb.second});
        std::sort(out.begin(), out.end());
        return out;
    }

    static XD sel_product(const std::vector<CutEdge>& c)
    {
        XD p = xd_make(c[0].sel, 0);
        for (size_t i = 1; i < c.size(); i++) p = xd_mul(p, xd_make(c[i].sel, 0));
        return p;
    }

    static XD join_card(XD a, XD b, const std::vector<CutEdge>& c)
    {
        XD x = xd_mul(a, b);
        for (const CutEdge& e : c) x = xd_mul(x, xd_make(e.sel, 0));
        return x;
    }

    int join(int a, int b)
    {
        if (nodes_[b].minrel < nodes_[a].minrel) std::swap(a, b);
        const std::vector<CutEdge> c = cut(a, b);
        PNode p;
        p.left = a;
        p.right = b;
        p.minrel = nodes_[a].minrel;
        p.leaves = nodes_[a].leaves + nodes_[b].leaves;
        p.card = join_card(nodes_[a].card, nodes_[b].card, c);
        p.cost = xd_add(xd_add(nodes_[a].cost, nodes_[b].cost), p.card);
        p.rels.resize(nodes_[a].rels.size() + nodes_[b].rels.size());
        std::merge(nodes_[a].rels.begin(), nodes_[a].rels.end(), nodes_[b].rels.begin(), nodes_[b].rels.end(),
                   p.rels.begin());
        nodes_.push_back(std::move(p));
        return (int)nodes_.size() - 1;
    }

    // The sub-problem over these plans (ordered by smallest relation).
    XdSubQuery subproblem(std::vector<int>& parts)
    {
        std::sort(parts.begin(), parts.end(), [&](int a, int b) { return nodes_[a].minrel < nodes_[b].minrel; });
        XdSubQuery q;
        q.n = (int)parts.size();
        for (int p : parts) q.card.push_back(nodes_[p].card);
        for (int i = 0; i < q.n; i++)
            for (int j = i + 1; j < q.n; j++) {
                const std::vector<CutEdge> c = cut(parts[i], parts[j]);
                if (c.empty()) continue;
                q.eu.push_back(i);
                q.ev.push_back(j);
                q.sel.push_back(sel_product(c));
            }
        return q;
    }

    int build(const XdSubPlan& sp, int i, const std::vector<int>& parts)
    {
        if (sp.left[i] < 0) return parts[__builtin_ctz(sp.set[i])];
        return join(build(sp, sp.left[i], parts), build(sp, sp.right[i], parts));
    }

    // exact plans over several groups of plans, solved in one device call
    int exact_many(std::vector<std::vector<int>>& groups, std::vector<int>& out)
    {
        std::vector<XdSubQuery> qs;
        std::vector<int> which;
        out.assign(groups.size(), -1);
        for (size_t g = 0; g < groups.size(); g++) {
            if (groups[g].size() == 1) {
                out[g] = groups[g][0];
                continue;
            }
            if ((int)groups[g].size() > kXdMaxRels) return MPDP_ERR_INTERNAL;
            qs.push_back(subproblem(groups[g]));
            which.push_back((int)g);
        }
        if (qs.empty()) return MPDP_OK;
        std::vector<XdSubPlan> plans;
        const int rc = exec_.run(qs, plans, st_, sms_);
        if (rc != MPDP_OK) return rc;
        subproblems_ += (int)qs.size();
        for (size_t i = 0; i < which.size(); i++) out[which[i]] = build(plans[i], 0, groups[which[i]]);
        return MPDP_OK;
    }

    int goo(int& result);
    int learned_start(int& result);
    int idp2(int k, int& result, bool learned = false);
    int uniondp(int k, int t, int& result, bool size_first = false);
    int scores(int m, const std::vector<int>& cur, const std::vector<std::pair<int, int>>& ij,
               const std::vector<XD>& sel, std::vector<float>& out);

    mpdp_mlp* model_ = nullptr;
    bool weight_scores_ = false;  // score edges by log2 of their join card instead of the model

    int n_;
    std::vector<PNode> nodes_;
    int subproblems_ = 0;

private:
    XdExecutor& exec_;
    cudaStream_t st_;
    int sms_;
    std::vector<int> mark_;
    int stamp_ = 0;
    std::vector<XD> card_;
    std::vector<CutEdge> edges_;
    std::vector<std::vector<std::pair<int, double>>> adj_;
};

// --------------------------------------------------------------------------
// GOO

struct GooCand {
    XD card;
    int lo, hi;  // tree ids (smallest relations), lo < hi
    int va, vb;  // versions when pushed
};

struct GooWorse {
    bool operator()(const GooCand& a, const GooCand& b) const
    {
        // true when a comes after b
        if (xd_less(b.card, a.card)) return true;
        if (xd_less(a.card, b.card)) return false;
        if (a.lo != b.lo) return a.lo > b.lo;
        return a.hi > b.hi;
    }
};

int Heuristic::goo(int& result)
{
    // a tree is named by its smallest relation; plan[id] is its plan node
    std::vector<int> plan(n_), version(n_, 0);
    std::vector<char> alive(n_, 1);
    std::vector<std::map<int, std::vector<CutEdge>>> nbr(n_);
    for (int r = 0; r < n_; r++) plan[r] = leaf(r);
    for (const CutEdge& e : edges_) {
        nbr[e.u][e.v].push_back(e);
        nbr[e.v][e.u].push_back(e);
    }
    std::priority_queue<GooCand, std::vector<GooCand>, GooWorse> heap;
    auto push = [&](int a, int b) {
        const int lo = std::min(a, b), hi = std::max(a, b);
        const XD c = join_card(nodes_[plan[lo]].card, nodes_[plan[hi]].card, nbr[lo][hi]);
        heap.push(GooCand{c, lo, hi, version[lo], version[hi]});
    };
    for (int a = 0; a < n_; a++)
        for (const auto& kv : nbr[a])
            if (a < kv.first) push(a, kv.first);
    int trees = n_;
    while (trees > 1) {
        if (heap.empty()) return MPDP_ERR_DISCONNECTED;
        const GooCand c = heap.top();
        heap.pop();
        if (!alive[c.lo] || !alive[c.hi] || version[c.lo] != c.va || version[c.hi] != c.vb) continue;
        // merge hi into lo (lo keeps the smaller relation, so the name stays)
        const int a = c.lo, b = c.hi;
        plan[a] = join(plan[a], plan[b]);
        alive[b] = 0;
        version[a]++;
        nbr[a].erase(b);
        nbr[b].erase(a);
        for (auto& kv : nbr[b]) {
            const int x = kv.first;
            std::vector<CutEdge>& into = nbr[a][x];
            std::vector<CutEdge> merged(into.size() + kv.second.size());
            std::merge(into.begin(), into.end(), kv.second.begin(), kv.second.end(), merged.begin());
            into = merged;
            nbr[x].erase(b);
            nbr[x][a] = merged;
        }
        nbr[b].clear();
        for (const auto& kv : nbr[a]) push(a, kv.first);
        trees--;
    }
    for (int r = 0; r < n_; r++)
        if (alive[r]) result = plan[r];
    return MPDP_OK;
}

// --------------------------------------------------------------------------
// Learned start for IDP2: the query's edges in ascending predicted score
// (the share of the query under the edge's join in an optimal plan), each
// joining the plans of its two ends when they are still apart (union-find):
// the plan that joins first what the model expects an optimal plan to join
// first.  Equal scores keep the edge order (min(u, v), max(u, v)).

int Heuristic::learned_start(int& result)
{
    std::vector<int> cur(n_), plan(n_), parent(n_);
    for (int r = 0; r < n_; r++) {
        cur[r] = leaf(r);
        plan[r] = cur[r];
        parent[r] = r;
    }
    std::vector<std::pair<int, int>> ij;
    std::vector<XD> sels;
    for (const CutEdge& e : edges_) {
        ij.push_back({e.u, e.v});
        sels.push_back(xd_make(e.sel, 0));
    }
    std::vector<float> sc;
    const int rc = scores(n_, cur, ij, sels, sc);
    if (rc != MPDP_OK) return rc;
    std::vector<int> order(ij.size());
    for (size_t i = 0; i < order.size(); i++) order[i] = (int)i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return sc[a] < sc[b]; });
    auto find = [&](int x) {
        while (parent[x] != x) x = parent[x] = parent[parent[x]];
        return x;
    };
    int trees = n_;
    for (int idx : order) {
        const int a = find(ij[idx].first), b = find(ij[idx].second);
        if (a == b) continue;
        const int lo = std::min(a, b), hi = std::max(a, b);
        plan[lo] = join(plan[lo], plan[hi]);
        parent[hi] = lo;
        trees--;
    }
    if (trees != 1) return MPDP_ERR_DISCONNECTED;
    result = plan[find(0)];
    return MPDP_OK;
}

// --------------------------------------------------------------------------
// IDP2

int Heuristic::idp2(int k, int& result, bool learned)
{
    int rc = learned ? learned_start(result) : goo(result);
    if (rc != MPDP_OK || k <= 1) return rc;
    // working tree: leaves hold plan nodes; internal nodes are joins of the
    // working tree whose cards are recomputed every round
    struct W {
        int l = -1, r = -1, parent = -1, plan = -1;
        int leaves = 0, pre = 0, end = 0;
        XD card, jc;
        std::vector<CutEdge> cut;
    };
    std::vector<W> w;
    // copy GOO's plan as the working tree
    {
        w.reserve(2 * n_);
        std::function<int(int, int)> copy = [&](int p, int parent) -> int {
            const int id = (int)w.size();
            w.push_back(W());
            w[id].parent = parent;
            if (nodes_[p].left < 0) {
                w[id].plan = p;
            } else {
                const int a = copy(nodes_[p].left, id);
                const int b = copy(nodes_[p].right, id);
                w[id].l = a;
                w[id].r = b;
            }
            return id;
        };
        copy(result, -1);
    }
    int root = 0;
    std::vector<int> leaf_of(n_, -1);
    while (w[root].l >= 0) {
        // pre-order numbering, leaf of every relation
        std::vector<int> pre_nodes;
        {
            std::vector<int> st = {root};
            while (!st.empty()) {
                const int v = st.back();
                st.pop_back();
                w[v].pre = (int)pre_nodes.size();
                pre_nodes.push_back(v);
                if (w[v].l >= 0) {
                    st.push_back(w[v].r);
                    st.push_back(w[v].l);
                } else {
                    for (int r : nodes_[w[v].plan].rels) leaf_of[r] = v;
                }
            }
            // subtree end (pre-order index past the subtree), bottom-up
            for (int i = (int)pre_nodes.size() - 1; i >= 0; i--) {
                const int v = pre_nodes[i];
                w[v].end = w[v].l >= 0 ? w[w[v].r].end : w[v].pre + 1;
                w[v].cut.clear();
            }
        }
        // every query edge between two leaves belongs to their lowest common ancestor
        for (const CutEdge& e : edges_) {
            const int a = leaf_of[e.u], b = leaf_of[e.v];
            if (a == b) continue;
            int v = a;
            while (!(w[v].pre <= w[b].pre && w[b].pre < w[v].end)) v = w[v].parent;
            w[v].cut.push_back(e);
        }
        // cards, joins-only costs and leaf counts, bottom-up
        for (int i = (int)pre_nodes.size() - 1; i >= 0; i--) {
            W& v = w[pre_nodes[i]];
            if (v.l < 0) {
                v.card = nodes_[v.plan].card;
                v.jc = xd_zero();
                v.leaves = 1;
                continue;
            }
            std::sort(v.cut.begin(), v.cut.end());
            v.card = join_card(w[v.l].card, w[v.r].card, v.cut);
            v.jc = xd_add(xd_add(w[v.l].jc, w[v.r].jc), v.card);
            v.leaves = w[v.l].leaves + w[v.r].leaves;
        }
        // the costliest subtree with 2..k leaves, first in pre-order on ties
        int best = -1;
        for (int v : pre_nodes)
            if (w[v].l >= 0 && w[v].leaves <= k && (best < 0 || xd_less(w[best].jc, w[v].jc))) best = v;
        std::vector<int> parts;
        {
            std::vector<int> st = {best};
            while (!st.empty()) {
                const int v = st.back();
                st.pop_back();
                if (w[v].l < 0) parts.push_back(w[v].plan);
                else {
                    st.push_back(w[v].r);
                    st.push_back(w[v].l);
                }
            }
        }
        std::vector<std::vector<int>> groups = {parts};
        std::vector<int> out;
        rc = exact_many(groups, out);
        if (rc != MPDP_OK) return rc;
        w[best].l = w[best].r = -1;
        w[best].plan = out[0];
    }
    result = w[root].plan;
    return MPDP_OK;
}

// --------------------------------------------------------------------------
// UnionDP

int Heuristic::uniondp(int k, int t, int& result, bool size_first)
{
    std::vector<int> cur(n_);
    for (int r = 0; r < n_; r++) cur[r] = leaf(r);
    std::vector<int> owner(n_);
    while ((int)cur.size() > k) {
        const int m = (int)cur.size();
        for (int i = 0; i < m; i++)
            for (int r : nodes_[cur[i]].rels) owner[r] = i;
        // edges between nodes, each with its query edges ascending
        std::map<std::pair<int, int>, std::vector<CutEdge>> between;
        for (const CutEdge& e : edges_) {
            const int a = owner[e.u], b = owner[e.v];
            if (a == b) continue;
            between[{std::min(a, b), std::max(a, b)}].push_back(e);
        }
        struct E {
            int i, j;
            XD w;
        };
        std::vector<E> es;
        for (auto& kv : between) {
            std::sort(kv.second.begin(), kv.second.end());
            const XD s = sel_product(kv.second);
            es.push_back(E{kv.first.first, kv.first.second,
                           xd_mul(xd_mul(nodes_[cur[kv.first.first]].card, nodes_[cur[kv.first.second]].card), s)});
        }
        std::vector<int> parent(m), size(m, 1);
        for (int i = 0; i < m; i++) parent[i] = i;
        auto find = [&](int x) {
            while (parent[x] != x) x = parent[x] = parent[parent[x]];
            return x;
        };
        std::vector<char> dropped(es.size(), 0);
        if (!model_ && !size_first) {
            // Algorithm 5's order, fixed before the loop: (size sum of the
            // sets across the edge, weight, i, j); every set is one node here
            std::vector<int> order(es.size());
            for (size_t i = 0; i < order.size(); i++) order[i] = (int)i;
            std::sort(order.begin(), order.end(), [&](int x, int y) {
                const E& a = es[x];
                const E& b = es[y];
                const int sa = size[a.i] + size[a.j], sb = size[b.i] + size[b.j];
                if (sa != sb) return sa < sb;
                if (!xd_equal(a.w, b.w)) return xd_less(a.w, b.w);
                if (a.i != b.i) return a.i < b.i;
                return a.j < b.j;
            });
            for (int idx : order) {
                const int a = find(es[idx].i), b = find(es[idx].j);
                if (a != b && size[a] + size[b] <= t) {
                    parent[b] = a;
                    size[a] += size[b];
                }
            }
            std::fill(dropped.begin(), dropped.end(), 1);
        }
        if (model_) {
            // learned proposal: edges by predicted score (the share of the
            // query under the edge's join in an optimal plan), lowest first,
            // united while the partition stays within t
            std::vector<std::pair<int, int>> ij;
            std::vector<XD> sels;
            for (auto& kv : between) {
                ij.push_back(kv.first);
                sels.push_back(sel_product(kv.second));
            }
            std::vector<float> sc;
            const int rc = scores(m, cur, ij, sels, sc);
            if (rc != MPDP_OK) return rc;
            std::vector<int> order(es.size());
            for (size_t i = 0; i < order.size(); i++) order[i] = (int)i;
            std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return sc[a] < sc[b]; });
            for (int idx : order) {
                const int a = find(es[idx].i), b = find(es[idx].j);
                if (a != b && size[a] + size[b] <= t) {
                    parent[b] = a;
                    size[a] += size[b];
                }
            }
            std::fill(dropped.begin(), dropped.end(), 1);
        }
        for (;;) {
            int best = -1, ba = 0, bb = 0, bs = 0;
            for (size_t idx = 0; idx < es.size(); idx++) {
                if (dropped[idx]) continue;
                const int a = find(es[idx].i), b = find(es[idx].j);
                if (a == b) continue;
                const int ssum = size[a] + size[b];
                bool better = best < 0;
                if (!better) {
                    const E& o = es[best];
                    if (ssum != bs) better = ssum < bs;
                    else if (!xd_equal(es[idx].w, o.w)) better = xd_less(es[idx].w, o.w);
                    else if (es[idx].i != o.i) better = es[idx].i < o.i;
                    else better = es[idx].j < o.j;
                }
                if (better) {
                    best = (int)idx;
                    ba = a;
                    bb = b;
                    bs = ssum;
                }
            }
            if (best < 0) break;
            if (bs <= t) {
                parent[bb] = ba;
                size[ba] += size[bb];
            } else {
                dropped[best] = 1;
            }
        }
        std::map<int, std::vector<int>> by_root;
        for (int i = 0; i < m; i++) by_root[find(i)].push_back(cur[i]);
        std::vector<std::vector<int>> groups;
        for (auto& kv : by_root) groups.push_back(kv.second);
        std::vector<int> out;
        const int rc = exact_many(groups, out);
        if (rc != MPDP_OK) return rc;
        std::sort(out.begin(), out.end(), [&](int a, int b) { return nodes_[a].minrel < nodes_[b].minrel; });
        if ((int)out.size() >= m) return MPDP_ERR_INTERNAL;  // no progress: cannot happen for t >= 2
        cur = out;
    }
    std::vector<std::vector<int>> groups = {cur};
    std::vector<int> out;
    const int rc = exact_many(groups, out);
    if (rc != MPDP_OK) return rc;
    result = out[0];
    return MPDP_OK;
}

double xd_to_double(XD x)
{
    if (x.m == 0.0) return 0.0;
    return std::ldexp(x.m, x.e);
}

}  // namespace

double xd_log2(XD x) { return x.m == 0.0 ? -1e300 : (double)x.e + std::log2(x.m); }

void edge_features(int n, const std::vector<double>& lcard, const std::vector<int>& eu, const std::vector<int>& ev,
                   const std::vector<double>& lsel, std::vector<float>& out)
{
    const int m = (int)eu.size();
    out.assign((size_t)m * kEdgeFeatures, 0.f);
    if (m == 0) return;
    std::vector<int> deg(n, 0);
    std::vector<std::vector<std::pair<int, int>>> adj(n);  // (neighbour, edge)
    for (int e = 0; e < m; e++) {
        deg[eu[e]]++;
        deg[ev[e]]++;
        adj[eu[e]].push_back({ev[e], e});
        adj[ev[e]].push_back({eu[e], e});
    }
    std::vector<double> lj(m);
    for (int e = 0; e < m; e++) lj[e] = lcard[eu[e]] + lcard[ev[e]] + lsel[e];
    std::vector<double> sorted_lj = lj;
    std::sort(sorted_lj.begin(), sorted_lj.end());
    const double median = sorted_lj[m / 2];
    // bridges (iterative lowlink search)
    std::vector<char> bridge(m, 0);
    {
        std::vector<int> disc(n, -1), low(n, 0), parent_edge(n, -1), it(n, 0);
        int timer = 0;
        for (int root = 0; root < n; root++) {
            if (disc[root] >= 0) continue;
            std::vector<int> st = {root};
            disc[root] = low[root] = timer++;
            while (!st.empty()) {
                const int v = st.back();
                if (it[v] < (int)adj[v].size()) {
                    const auto [w, e] = adj[v][it[v]++];
                    if (e == parent_edge[v]) continue;
                    if (disc[w] < 0) {
                        disc[w] = low[w] = timer++;
                        parent_edge[w] = e;
                        st.push_back(w);
                    } else {
                        low[v] = std::min(low[v], disc[w]);
                    }
                } else {
                    st.pop_back();
                    if (!st.empty()) {
                        const int u = st.back();
                        low[u] = std::min(low[u], low[v]);
                        if (low[v] > disc[u]) bridge[parent_edge[v]] = 1;
                    }
                }
            }
        }
    }
    const double ln = std::log2((double)std::max(n, 1));
    for (int e = 0; e < m; e++) {
        const int u = eu[e], v = ev[e];
        double inc_lo = lj[e], inc_hi = lj[e];
        for (int x : {u, v})
            for (const auto& nb : adj[x]) {
                inc_lo = std::min(inc_lo, lj[nb.second]);
                inc_hi = std::max(inc_hi, lj[nb.second]);
            }
        const int rank = (int)(std::lower_bound(sorted_lj.begin(), sorted_lj.end(), lj[e]) - sorted_lj.begin());
        float* f = &out[(size_t)e * kEdgeFeatures];
        f[0] = (float)(std::min(lcard[u], lcard[v]) / 32.0);
        f[1] = (float)(std::max(lcard[u], lcard[v]) / 32.0);
        f[2] = (float)(lsel[e] / 32.0);
        f[3] = (float)(lj[e] / 32.0);
        f[4] = (float)((lj[e] - median) / 32.0);
        f[5] = (float)(m > 1 ? (double)rank / (double)(m - 1) : 0.0);
        f[6] = (float)(std::log2(1.0 + std::min(deg[u], deg[v])) / 4.0);
        f[7] = (float)(std::log2(1.0 + std::max(deg[u], deg[v])) / 4.0);
        f[8] = (float)((lj[e] - inc_lo) / 32.0);
        f[9] = (float)((inc_hi - lj[e]) / 32.0);
        f[10] = bridge[e] ? 1.f : 0.f;
        f[11] = (float)(ln / 12.0);
    }
}


namespace {

int Heuristic::scores(int m, const std::vector<int>& cur, const std::vector<std::pair<int, int>>& ij,
                      const std::vector<XD>& sel, std::vector<float>& out)
{
    std::vector<double> lcard(m), lsel(sel.size());
    std::vector<int> eu(ij.size()), ev(ij.size());
    for (int i = 0; i < m; i++) lcard[i] = xd_log2(nodes_[cur[i]].card);
    for (size_t e = 0; e < ij.size(); e++) {
        eu[e] = ij[e].first;
        ev[e] = ij[e].second;
        lsel[e] = xd_log2(sel[e]);
    }
    if (weight_scores_) {
        // the non-learned control: log2 of each edge's join card
        out.resize(ij.size());
        for (size_t e = 0; e < ij.size(); e++) out[e] = (float)(lcard[eu[e]] + lcard[ev[e]] + lsel[e]);
        return MPDP_OK;
    }
    std::vector<float> feat;
    edge_features(m, lcard, eu, ev, lsel, feat);
    const int rows = (int)ij.size();
    out.assign(rows, 0.f);
    if (rows == 0) return MPDP_OK;
    float *dx = nullptr, *dy = nullptr;
    if (cudaMalloc(&dx, feat.size() * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&dy, (size_t)rows * sizeof(float)) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(dx);
        return MPDP_ERR_OOM;
    }
    int rc = MPDP_OK;
    if (cudaMemcpy(dx, feat.data(), feat.size() * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess)
        rc = MPDP_ERR_CUDA;
    if (rc == MPDP_OK) rc = mpdp_mlp_forward(model_, dx, rows, dy);
    if (rc == MPDP_OK && cudaDeviceSynchronize() != cudaSuccess) rc = MPDP_ERR_CUDA;
    if (rc == MPDP_OK && cudaMemcpy(out.data(), dy, (size_t)rows * sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess)
        rc = MPDP_ERR_CUDA;
    cudaFree(dx);
    cudaFree(dy);
    cudaGetLastError();
    return rc;
}

}  // namespace

int run_heuristic(const HeuristicQuery& q, XdExecutor& ex, cudaStream_t st, int num_sms, HeuristicResult& res)
{
    Heuristic h(q, ex, st, num_sms);
    int root = -1, rc;
    res.learned_won = false;
    if (q.mode == MPDP_MODE_IDP2) rc = h.idp2(q.k, root);
    else if (q.mode == MPDP_MODE_UNIONDP) rc = h.uniondp(q.k, q.t > 0 ? q.t : q.k, root);
    else if (q.mode == MPDP_MODE_UNIONDP_SIZEFIRST) rc = h.uniondp(q.k, q.t > 0 ? q.t : q.k, root, true);
    else if (q.mode == MPDP_MODE_UNIONDP_LEARNED) {
        // the learned proposal's plan, with plain UnionDP as the fallback:
        // both are costed exactly and the cheaper one (plain on ties) wins
        const int t = q.t > 0 ? q.t : q.k;
        rc = h.uniondp(q.k, t, root);
        if (rc == MPDP_OK && q.model) {
            int learned = -1;
            h.model_ = q.model;
            rc = h.uniondp(q.k, t, learned);
            h.model_ = nullptr;
            if (rc == MPDP_OK && xd_less(h.nodes_[learned].cost, h.nodes_[root].cost)) {
                root = learned;
                res.learned_won = true;
            }
        }
    } else if (q.mode == MPDP_MODE_IDP2_LEARNED) {
        // IDP2 from the learned start, with IDP2 from GOO's plan as the
        // fallback: the cheaper plan wins (GOO's on ties)
        rc = h.idp2(q.k, root);
        if (rc == MPDP_OK && q.model) {
            int learned = -1;
            h.model_ = q.model;
            rc = h.idp2(q.k, learned, true);
            h.model_ = nullptr;
            if (rc == MPDP_OK && xd_less(h.nodes_[learned].cost, h.nodes_[root].cost)) {
                root = learned;
                res.learned_won = true;
            }
        }
    } else if (q.mode == MPDP_MODE_IDP2_WEIGHT_START) {
        // the learned mode's rule with a non-learned second start: IDP2 from
        // the plan that joins the edges in ascending join card, IDP2 from
        // GOO's plan as the fallback, the cheaper plan wins (GOO's on ties)
        rc = h.idp2(q.k, root);
        if (rc == MPDP_OK) {
            int alt = -1;
            h.weight_scores_ = true;
            rc = h.idp2(q.k, alt, true);
            h.weight_scores_ = false;
            if (rc == MPDP_OK && xd_less(h.nodes_[alt].cost, h.nodes_[root].cost)) {
                root = alt;
                res.learned_won = true;
            }
        }
    } else return MPDP_ERR_NOT_IMPLEMENTED;
    if (rc != MPDP_OK) return rc;
    // breadth-first node list from the root
    res.nodes.clear();
    std::vector<int> ids = {root};
    for (size_t i = 0; i < ids.size(); i++) {
        const PNode& p = h.nodes_[ids[i]];
        mpdp_plan_node nd;
        nd.n_leaves = p.leaves;
        nd.set = 0;
        if (h.n_ <= 64)
            for (int r : p.rels) nd.set |= 1ull << r;
        nd.card = xd_to_double(p.card);
        nd.cost = xd_to_double(p.cost);
        if (p.left < 0) {
            nd.left = nd.right = -1;
            nd.rel = p.rel;
        } else {
            nd.rel = -1;
            nd.left = (int)ids.size();
            nd.right = (int)ids.size() + 1;
            ids.push_back(p.left);
            ids.push_back(p.right);
        }
        res.nodes.push_back(nd);
    }
    res.cost = h.nodes_[root].cost;
    res.subproblems = h.subproblems_;
    return MPDP_OK;
}

}  // namespace mpdp
