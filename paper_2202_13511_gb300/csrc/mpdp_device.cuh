// Device-side data layout and helpers of the MPDP path (sm_103a).
//
// Relation sets are 32-bit bitmaps (bit i = relation i), the fixed-width
// bitmap sets of the paper (Sec. 2.2, "Implementation Details"; Sec. 5).
// Every kernel works on a batch of queries; one query is a batch of one.
#pragma once

#include <cstddef>
#include <cstdint>

#include "../../include/mpdp.h"

// Loads of data that stays unchanged for a whole launch go through the
// read-only path (MPDP_LDG) and pointers to it are restrict-qualified.  A
// kernel that writes and reads the same memory across its own lifetime (the
// persistent serving kernel) defines MPDP_COHERENT_LOADS before including
// this header: its loads are then plain global loads (never the
// non-coherent read-only path) and no pointer is marked restrict.  Such a
// kernel reads memory that another block wrote only after acquiring it: the
// writer fences before it publishes (a phase word, an arrival count) and
// the reader fences (__threadfence, a GPU-scope fence) after it observes the
// publication, so under the PTX memory model its later loads, L1 hits
// included, see the published writes.
#ifdef MPDP_COHERENT_LOADS
#define MPDP_LDG(p) (*(p))
#define MPDP_RESTRICT
#else
#define MPDP_LDG(p) __ldg(p)
#define MPDP_RESTRICT __restrict__
#endif

namespace mpdp {

constexpr int kMaxRels = 32;        // bitmap width
constexpr int kLevels = MPDP_MAX_LEVELS;
constexpr int kMaxEdges = kMaxRels * (kMaxRels - 1) / 2;
constexpr int kEvalThreads = 256;
constexpr int kFilterThreads = 256;
constexpr int kMaxBatch = 1024;     // queries per device batch
constexpr int kPlanNodes = 2 * kMaxRels - 1;
constexpr unsigned kFull = 0xffffffffu;

// Query as staged from the host (or gathered from caller device buffers).
struct StagedQuery {
    int32_t n, n_edges, cost_model, pad;
    double card[kMaxRels];
    mpdp_edge edges[kMaxEdges];
};

// Query as the kernels read it.  Built on the device by k_ingest.
struct DevQuery {
    int32_t n, n_edges, pad[2];
    uint32_t adj[kMaxRels];          // adjacency bitmaps
    uint32_t nbase[kMaxRels];        // first entry of relation r's neighbour list in nsel
    double card[kMaxRels];
    double nsel[2 * kMaxEdges];      // nsel[nbase[r] + i]: sel of r's i-th neighbour (ascending)
    // nbt[b][x]: union of the adjacency bitmaps of relations 8b + i for every
    // bit i of the byte x, so N(S) = OR_b nbt[b][byte b of S] (4 lookups)
    uint32_t nbt[4][256];
    // Spanning tree T of G, rooted at relation 0 (breadth first; T = G when G
    // is a tree).  ctt[b][x]: union of the children in T of relations 8b + i
    // for every bit i of the byte x, so C(S) = OR_b ctt[b][byte b of S] is
    // the set of relations whose T-parent lies in S.
    uint32_t ctt[4][256];
    uint32_t desc[kMaxRels];         // desc[v]: v and its descendants in T
    int32_t is_tree;                 // G itself is a tree (n - 1 edges)
    int32_t pad2[3];
    // Bitmap-filter run tables for the low relations r < 5 of T (a run is
    // the 32 bitmaps base | i, i < 32):  [r] children of r;  [5 + r] the
    // run mask of "r is in S and its parent is not" when r is the root or
    // its parent is low;  [10 + r] r's parent when it is a high relation,
    // else 0xffffffff;  [15] the relations whose parent is low.
    uint32_t lowrun[16];
    // Connected-set unranking for tree join graphs (zero otherwise).  The
    // connected sets whose top (the member nearest the root) is v are {v}
    // with, for each child c of v, nothing or a connected set whose top is c:
    // nsub[v] = prod over children c of (1 + nsub[c]) of them.  top_pref[v]
    // = sum of nsub[u] for u < v, top_pref[n] = every connected set.
    uint32_t chmask[kMaxRels];       // children of v in T
    uint32_t nsub[kMaxRels];
    uint32_t top_pref[kMaxRels + 1];
    uint32_t leaves;                 // relations without children in T
    uint32_t use_connected;          // filter CONNECTED chose unranking for this query
    uint32_t pad3;
    // x / (1 + nsub[c]) as (t + ((x - t) >> s1)) >> s2 with t = umulhi(x,
    // dmag[c]), s1 = dsh[c] & 1, s2 = dsh[c] >> 1 (Granlund and Montgomery,
    // "Division by invariant integers using multiplication", 1994, Fig. 4.1)
    uint32_t dmag[kMaxRels];
    uint8_t dsh[kMaxRels];
};

// T[S] has one component per member of S whose T-parent is outside S, so
// popcount(S & ~C(S)) == 1 exactly when T[S] is connected: connected(S) in
// a tree join graph, and a sufficient condition in any join graph (T[S] is a
// spanning subgraph of G[S]).
__device__ __forceinline__ uint32_t tops_of(uint32_t s, uint32_t children)
{
    return s & ~children;
}

// low_bit(r): the i in [0, 32) whose bit r is set, as a 32-bit mask (the
// membership of relation r < 5 along a run of 32 bitmaps, bit-sliced over i).
__host__ __device__ constexpr uint32_t low_bit(int r)
{
    return r == 0 ? 0xaaaaaaaau
                  : r == 1 ? 0xccccccccu : r == 2 ? 0xf0f0f0f0u : r == 3 ? 0xff00ff00u : 0xffff0000u;
}

// Per-query device counters and status word.
struct DevCounters {
    unsigned long long unranked;
    unsigned long long heavy;
    unsigned long long memo_slots;
    unsigned long long filter_steps;    // BFS rounds run by the filter's connectivity tests
    unsigned long long connected[kLevels];
    unsigned long long evaluated[kLevels];
    unsigned long long ccp[kLevels];
    unsigned int list_count[kLevels];   // connected sets of level k in the list
    unsigned int heavy_count[kLevels];  // sets of level k sent to the heavy-set kernel
    unsigned int extra_count[kLevels];  // extra pair chunks reserved at level k (may exceed the capacity)
    int status;                         // first MPDP_ERR_* raised on the device
    int pad;
};

struct DevResult {
    double cost;
    int32_t n_nodes;
    int32_t status;
    mpdp_plan_node nodes[kPlanNodes];
};

// Device twin of one query's result + counters: one copy reads both back.
struct DevOut {
    DevResult result;
    DevCounters counters;
};

// Open-addressing memo slot: one 32-byte sector per probe.
struct alignas(32) HashSlot {
    uint32_t key;    // relation bitmap; 0 = empty (the empty set is never stored)
    uint32_t left;   // left child bitmap of the best split
    double cost;     // C_out cost of the best plan
    double card;     // card(S)
    double pad;
};
// The probes read {key, left, cost} and {card, pad} as two 16-byte words.
static_assert(sizeof(HashSlot) == 32 && offsetof(HashSlot, cost) == 8 && offsetof(HashSlot, card) == 16,
              "HashSlot layout");

struct HashLayout {
    unsigned long long base[kLevels];  // first slot of level k's table
    unsigned int mask[kLevels];        // capacity - 1 (capacity a power of two)
    unsigned long long total_slots;
};

// Where one query of a batch lives in the batch workspace.
struct QDesc {
    int32_t n, n_edges, enumeration, cost_model;
    unsigned long long memo_base;      // dense memo: entry of bitmap 0
    unsigned long long list_base;      // first list word of the query
    unsigned long long card_off;       // device path: offset of the query in the caller arrays
    unsigned long long edge_off;
    uint32_t list_off[kLevels];        // level k's region, relative to list_base
    uint32_t warp_begin[kLevels + 1];  // first filter warp of level k, relative to the query
    uint32_t filter_block_base;        // first filter block of the query
    uint32_t heavy_cap;                // heavy-set entries (and extra chunks) of one level: max_k C(n, k)
    unsigned long long heavy_base;     // first heavy-set entry of the query (block mode only)
    // Connectivity bitmap (block mode with the bitmap sweep): bit S of word
    // S / 32 is 1 when G[S] is connected (single relations included, the
    // empty set not), 2^n bits from list word conn_base on; the sweep writes
    // every word.  use_conn = 0: no bitmap, the evaluation tests sets itself.
    unsigned long long conn_base;
    uint32_t use_conn;
    // Block CCP lists (block mode, batched path; see kBlTab): use_bl = 1 when
    // the query has the area at list word bl_base, else every lookup misses.
    uint32_t use_bl;
    unsigned long long bl_base;
};

// Block CCP lists.  The CCP bipartitions of a block B of G[S] depend on B
// alone, and a block of three or more relations is itself a connected,
// 2-connected set of an earlier level; a cyclic query has few of those
// (about 15 at 20 relations with 10-30 % extra edges, 85 at 25) against
// the 10^5-10^6 connected sets that contain them.  Before the levels, the
// query's 2-connected sets that are not cliques (a clique's bipartitions are
// all CCPs) are found and each one's CCP left sides listed once; a set's
// evaluation then folds a listed block's CCPs instead of enumerating its
// 2^(|B|-1) - 1 bipartitions.  The lists are a cache: a block that is not
// listed (larger than kBlMaxBlock, or the table or the store full) is
// enumerated as before, with the same result.
// Area words: [0] sets found, [1] left sides reserved, [2, 4) unused,
// [4, kBlHead) slots {key B, first left side, count, 0} (open addressing on
// fmix32(B), key 0 empty), then room for kBlTab sets found (kBlSets used),
// then kBlLbs left sides.
constexpr uint32_t kBlTab = 1024;
// Sets listed at most: the table stays at most half full, so that a lookup
// of an unlisted block ends at an empty slot within a few probes.
constexpr uint32_t kBlSets = kBlTab / 2;
constexpr uint32_t kBlLbs = 65536;
constexpr uint32_t kBlHead = 4u + 4u * kBlTab;
constexpr uint32_t kBlWords = kBlHead + kBlTab + kBlLbs;
// Queries below kBlMinRels have no lists (on cyclic-16 the two extra
// launches cost more than they save), and blocks above kBlMaxBlock are not
// listed (one thread block lists a block, and every level waits for the
// listing: a block of 18 relations would hold them back longer than its
// enumeration costs the sets that contain it).
constexpr int kBlMinRels = 18;
constexpr int kBlMaxBlock = 14;

// A heavy set (more than heavy_threshold pairs) is cut into nch chunks of
// its pair index space, each taken by one warp.  Chunk 0 is the main entry;
// chunks 1..nch-1 are extra entries [ebase, ebase + nch - 1).  Each chunk
// leaves its best (x, left) in its own entry; the warp whose arrival
// completes the count folds them and writes the memo.
constexpr uint32_t kChunkPairs = 2048;   // pairs per chunk (64 rounds of a warp)
constexpr uint32_t kMaxChunks = 4096;    // chunks per set; with the capacity check before each
                                         // reservation the extra counter stays below 2^32
struct HeavyMain {
    uint32_t set;
    uint32_t nch;
    uint32_t ebase;
    uint32_t arrived;                  // chunks finished; starts at 0
    unsigned long long x;              // chunk 0's best x
    uint32_t left;                     // chunk 0's best left
    uint32_t pad;
};
struct HeavyExtra {
    uint32_t main;                     // index of the set's main entry
    uint32_t left;
    unsigned long long x;
};

// Everything a batch launch needs (passed by value).
struct BatchArgs {
    int nq;
    int max_n;
    const QDesc* desc;
    const uint32_t* filter_block_prefix;  // [nq + 1]
    StagedQuery* staged;
    DevQuery* query;
    DevOut* out;
    uint32_t* lists;
    HeavyMain* hmain;
    HeavyExtra* hextra;
    double2* memo;       // dense memo {cost, card}[S]
    uint32_t* left;      // dense memo left[S]
    HashSlot* arena;     // hash memo slots
    HashLayout* layout;  // [nq]
    unsigned long long arena_begin;  // hash memo: this batch's slots are [arena_begin, arena_slots)
    unsigned long long arena_slots;
    int run;             // ranks per lane in the filter (<= 32)
    int heavy_threshold;
    int use_ccc;
    int dpsub;           // block mode enumerates each set as one block (DPSUB ablation)
    int filter_mode;     // MPDP_FILTER_BITMAPS or MPDP_FILTER_UNRANK (the filter_block_prefix
                         // counts the blocks of the chosen filter)
};

// Record the first device error; later errors keep the first code.
__device__ __forceinline__ void raise_status(DevCounters* c, int code) { atomicCAS(&c->status, 0, code); }

__device__ __forceinline__ int lowest(uint32_t s) { return __ffs(s) - 1; }

// grow(source, restriction) of Sec. 3.2.1: every vertex of the restriction
// reachable from the source.  The loop pops one frontier vertex per step.
__device__ __forceinline__ uint32_t grow(uint32_t source, uint32_t restriction,
                                         const uint32_t* MPDP_RESTRICT adj)
{
    uint32_t seen = source, frontier = source;
    while (frontier) {
        int x = lowest(frontier);
        frontier &= frontier - 1;
        uint32_t nb = adj[x] & restriction & ~seen;
        seen |= nb;
        frontier |= nb;
    }
    return seen;
}

// connected(S): grow from the lowest member of S inside S reaches all of S.
__device__ __forceinline__ bool connected(uint32_t s, const uint32_t* MPDP_RESTRICT adj)
{
    uint32_t seen = s & (0u - s), frontier = seen;
    while (frontier) {
        int x = lowest(frontier);
        frontier &= frontier - 1;
        uint32_t nb = adj[x] & s & ~seen;
        seen |= nb;
        frontier |= nb;
        if (seen == s) return true;
    }
    return seen == s;
}

// The query's connectivity bitmap, when the bitmap sweep wrote one (block
// mode; a tree unranked by the connected-set filter has none).
__device__ __forceinline__ const uint32_t* conn_bitmap(const BatchArgs& a, int q);

// G[X] connected, for a non-empty X: one bit of the connectivity bitmap,
// a single relation at once, or (no bitmap) the search from min(X).
__device__ __forceinline__ bool conn_of(uint32_t x, const uint32_t* MPDP_RESTRICT cw, const uint32_t* MPDP_RESTRICT adj)
{
    if ((x & (x - 1u)) == 0u) return true;
    return cw ? ((MPDP_LDG(&cw[x >> 5]) >> (x & 31u)) & 1u) != 0u : connected(x, adj);
}

// Neighbourhood N(S) (every relation adjacent to a member of S) by byte tables.
__device__ __forceinline__ uint32_t nbhd(uint32_t s, const uint32_t (*MPDP_RESTRICT t)[256])
{
    return t[0][s & 255u] | t[1][(s >> 8) & 255u] | t[2][(s >> 16) & 255u] | t[3][s >> 24];
}

// connected(S) by whole-frontier rounds, for S (|S| >= 2) with no isolated
// vertex in G[S]: grow from min(S) one BFS layer per round until S is
// reached or growth stops.
__device__ __forceinline__ bool connected_rounds_from(uint32_t s, const uint32_t (*MPDP_RESTRICT t)[256],
                                                      uint32_t& rounds)
{
    uint32_t seen = s & (0u - s);
    while (true) {
        rounds++;
        const uint32_t nxt = (seen | nbhd(seen, t)) & s;
        if (nxt == s) return true;
        if (nxt == seen) return false;
        seen = nxt;
    }
}

// connected(S) for |S| >= 2: first reject S when a member has no neighbour
// inside S (an isolated vertex of G[S]), then BFS rounds.
__device__ __forceinline__ bool connected_rounds(uint32_t s, const uint32_t (*MPDP_RESTRICT t)[256],
                                                 uint32_t& rounds)
{
    if (s & ~nbhd(s, t)) return false;
    uint32_t seen = s & (0u - s);
    while (true) {
        rounds++;
        const uint32_t nxt = (seen | nbhd(seen, t)) & s;
        if (nxt == s) return true;
        if (nxt == seen) return false;
        seen = nxt;
    }
}

// Shared-memory copy of one query for the evaluate kernels.
struct SharedQuery {
    uint32_t adj[kMaxRels];
    uint32_t nbase[kMaxRels];
    uint32_t desc[kMaxRels];
    double card[kMaxRels];
    double nsel[2 * kMaxEdges];
};

// sel(j, r) for an edge (j, r): entry of j in r's ascending neighbour list.
__device__ __forceinline__ double sel_of(const SharedQuery& sq, int j, int r)
{
    return sq.nsel[sq.nbase[r] + __popc(sq.adj[r] & ((1u << j) - 1u))];
}

// Highest member of S.
__device__ __forceinline__ int highest(uint32_t s) { return 31 - __clz(s); }

// Peel vertex of a connected S (|S| >= 2) whose G[S] is a tree: its highest
// leaf (a vertex of degree 1 in G[S]), i.e. its highest non-cut vertex.
__device__ __forceinline__ int tree_peel_vertex(uint32_t s, const uint32_t* MPDP_RESTRICT adj)
{
    uint32_t t = s;
    while (t) {
        const int v = highest(t);
        if (__popc(adj[v] & s) == 1) return v;
        t &= ~(1u << v);
    }
    return highest(s);
}

// Peel vertex of a connected S from its blocks: the highest vertex that lies
// in exactly one block (a non-cut vertex).
__device__ __forceinline__ int block_peel_vertex(uint32_t s, const uint32_t* blk, int nb)
{
    uint32_t once = 0u, twice = 0u;
    for (int j = 0; j < nb; j++) {
        twice |= once & blk[j];
        once |= blk[j];
    }
    return highest(s & ~twice);
}

// Lexicographic order of candidate splits on (x, left), x = cost(S_l) +
// cost(S_r) >= 0 compared through its IEEE bit pattern (monotone for
// non-negative doubles, and no FP64 pipe involved).
__device__ __forceinline__ bool better_x(unsigned long long x, uint32_t l, unsigned long long bx, uint32_t bl)
{
    return x < bx || (x == bx && l < bl);
}

// Warp-wide lexicographic min of (x, left); every lane ends with the min.
__device__ __forceinline__ void warp_min_x(unsigned long long& bx, uint32_t& bl)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long ox = __shfl_xor_sync(0xffffffffu, bx, o);
        const uint32_t ol = __shfl_xor_sync(0xffffffffu, bl, o);
        if (better_x(ox, ol, bx, bl)) {
            bx = ox;
            bl = ol;
        }
    }
}

__device__ __forceinline__ const uint32_t* conn_bitmap(const BatchArgs& a, int q)
{
    const QDesc& d = a.desc[q];
    return (d.use_conn && !a.query[q].use_connected) ? a.lists + d.conn_base : nullptr;
}

// Murmur3's 32-bit finaliser (fmix32), the hash the paper names for the memo.
__device__ __forceinline__ uint32_t fmix32(uint32_t h)
{
    h ^= h >> 16;
    h *= 0x85ebca6bu;
    h ^= h >> 13;
    h *= 0xc2b2ae35u;
    h ^= h >> 16;
    return h;
}

// Memo indexed directly by the relation bitmap: a 16-byte entry {cost, card}
// (cost read by every pair, card by the peeling of the next level; one
// sector either way, and one sector written per set) and left[S], read by
// the plan fetch only.
struct DenseMemo {
    double2* cc0;      // batch arena
    uint32_t* left0;
    double2* cc;       // bound to one query
    uint32_t* left;
    int shift;         // bound query: 32 - n when its entries sit at bit-reversed bitmaps, else -1

    static constexpr size_t kSharedBytes = 16;

    // Entry of set S.  A tree-mode query whose connected sets are unranked
    // keeps them at the bit-reversed bitmap (relation 0 the top bit): the
    // unranking lists them with the high-numbered relations varying fastest,
    // so sets evaluated side by side then read and write neighbouring
    // entries.  The bitmap sweep lists sets in bitmap order, which the plain
    // bitmap keeps.
    __device__ __forceinline__ uint32_t at(uint32_t s) const { return shift >= 0 ? __brev(s) >> shift : s; }
    __device__ __forceinline__ void setup(char*) {}
    // per thread; no shared memory involved
    __device__ __forceinline__ void bind(const BatchArgs& a, int q)
    {
        const unsigned long long b = a.desc[q].memo_base;
        cc = cc0 + b;
        left = left0 + b;
        shift = (a.query[q].use_connected && a.desc[q].enumeration == MPDP_ENUM_TREE) ? 32 - a.desc[q].n : -1;
    }
    __device__ __forceinline__ double get_cost(uint32_t s, DevCounters*) const { return MPDP_LDG(&cc[at(s)].x); }
    __device__ __forceinline__ double get_card(uint32_t s, DevCounters*) const { return MPDP_LDG(&cc[at(s)].y); }
    __device__ __forceinline__ void get(uint32_t s, double& c, double& cd, uint32_t& l, DevCounters*) const
    {
        const uint32_t i = at(s);
        const double2 v = cc[i];
        c = v.x;
        cd = v.y;
        l = left[i];
    }
    __device__ __forceinline__ void put(uint32_t s, int, double c, double cd, uint32_t l, DevCounters*)
    {
        const uint32_t i = at(s);
        cc[i] = make_double2(c, cd);
        left[i] = l;
    }
};

// The dense memo as the block-mode kernels see it: their queries (block
// enumeration) always keep entries at the plain bitmap.
struct DensePlainMemo {
    double2* cc0;
    uint32_t* left0;
    double2* cc;
    uint32_t* left;

    static constexpr size_t kSharedBytes = 16;

    __device__ __forceinline__ void setup(char*) {}
    __device__ __forceinline__ void bind(const BatchArgs& a, int q)
    {
        const unsigned long long b = a.desc[q].memo_base;
        cc = cc0 + b;
        left = left0 + b;
    }
    __device__ __forceinline__ double get_cost(uint32_t s, DevCounters*) const { return MPDP_LDG(&cc[s].x); }
    __device__ __forceinline__ double get_card(uint32_t s, DevCounters*) const { return MPDP_LDG(&cc[s].y); }
    __device__ __forceinline__ void get(uint32_t s, double& c, double& cd, uint32_t& l, DevCounters*) const
    {
        const double2 v = cc[s];
        c = v.x;
        cd = v.y;
        l = left[s];
    }
    __device__ __forceinline__ void put(uint32_t s, int, double c, double cd, uint32_t l, DevCounters*)
    {
        cc[s] = make_double2(c, cd);
        left[s] = l;
    }
};

// Memo as one open-addressing table per level (linear probing).
struct HashMemo {
    HashSlot* arena;
    const HashLayout* lay;  // the bound query's table bases and masks

    static constexpr size_t kSharedBytes = 16;

    __device__ __forceinline__ void setup(char*) {}
    // per thread; no shared memory involved
    __device__ __forceinline__ void bind(const BatchArgs& a, int q) { lay = a.layout + q; }
    // Probe for S: each step is one 16-byte load of the slot's {key, left,
    // cost} (and, with `whole`, a second one of its card, issued together:
    // the same sector), so a hit costs one round of memory latency per probe
    // step rather than a key load and then a value load.  False (and the
    // status PROBE_LIMIT) when S is missing.
    __device__ __forceinline__ bool probe(uint32_t s, bool whole, uint4& head, uint4& tail, DevCounters* cnt) const
    {
        const int lvl = __popc(s);
        const HashSlot* t = arena + MPDP_LDG(&lay->base[lvl]);
        const uint32_t m = MPDP_LDG(&lay->mask[lvl]);
        uint32_t h = fmix32(s) & m;
        for (uint32_t i = 0; i <= m; i++) {
            const uint4* e = reinterpret_cast<const uint4*>(t + h);
            head = MPDP_LDG(e);
            if (whole) tail = MPDP_LDG(e + 1);
            if (head.x == s) return true;
            if (head.x == 0u) break;
            h = (h + 1u) & m;
        }
        raise_status(cnt, MPDP_ERR_PROBE_LIMIT);
        return false;
    }
    __device__ __forceinline__ double get_cost(uint32_t s, DevCounters* cnt) const
    {
        uint4 head, tail;
        return probe(s, false, head, tail, cnt) ? __hiloint2double((int)head.w, (int)head.z)
                                                : __longlong_as_double(0x7ff8000000000000ll);
    }
    __device__ __forceinline__ double get_card(uint32_t s, DevCounters* cnt) const
    {
        uint4 head, tail;
        return probe(s, true, head, tail, cnt) ? __hiloint2double((int)tail.y, (int)tail.x)
                                               : __longlong_as_double(0x7ff8000000000000ll);
    }
    __device__ __forceinline__ void get(uint32_t s, double& c, double& card, uint32_t& l, DevCounters* cnt) const
    {
        uint4 head, tail;
        if (probe(s, true, head, tail, cnt)) {
            c = __hiloint2double((int)head.w, (int)head.z);
            card = __hiloint2double((int)tail.y, (int)tail.x);
            l = head.y;
        } else {
            c = card = __longlong_as_double(0x7ff8000000000000ll);
            l = 0xffffffffu;
        }
    }
    __device__ __forceinline__ void put(uint32_t s, int lvl, double c, double card, uint32_t l,
                                        DevCounters* cnt)
    {
        HashSlot* t = arena + MPDP_LDG(&lay->base[lvl]);
        const uint32_t m = MPDP_LDG(&lay->mask[lvl]);
        uint32_t h = fmix32(s) & m;
        for (uint32_t i = 0; i <= m; i++) {
            if (atomicCAS(&t[h].key, 0u, s) == 0u) {
                t[h].left = l;
                t[h].cost = c;
                t[h].card = card;
                return;
            }
            h = (h + 1u) & m;
        }
        raise_status(cnt, MPDP_ERR_OOM);
    }
};

}  // namespace mpdp

namespace mpdp {

// card(S) by peeling vertex v: card(S \ {v}) (from the memo; a single
// relation's card directly; peel_base), times card[v], times sel(j, v) for
// the neighbours j of v in S in ascending order (peel_finish).  __dmul_rn
// keeps every step a separately rounded IEEE multiply.
template <class Memo, class Q>
__device__ __forceinline__ double peel_base(uint32_t s, int v, const Q& sq, const Memo& memo, DevCounters* cnt)
{
    const uint32_t rest = s & ~(1u << v);
    return (rest & (rest - 1u)) ? memo.get_card(rest, cnt) : sq.card[lowest(rest)];
}

template <class Q>
__device__ __forceinline__ double peel_finish(double p, uint32_t s, int v, const Q& sq)
{
    p = __dmul_rn(p, sq.card[v]);
    const uint32_t nv = sq.adj[v];
    uint32_t nb = nv & s;
    while (nb) {
        const int j = lowest(nb);
        nb &= nb - 1u;
        p = __dmul_rn(p, sq.nsel[sq.nbase[v] + __popc(nv & ((1u << j) - 1u))]);
    }
    return p;
}

template <class Memo, class Q>
__device__ __forceinline__ double peel_card(uint32_t s, int v, const Q& sq, const Memo& memo, DevCounters* cnt)
{
    return peel_finish(peel_base(s, v, sq, memo, cnt), s, v, sq);
}

// Fold one CCP pair (S_l, S_r) into the running best (x, left).  x is
// cost(S_l) + cost(S_r); a single relation costs 0 (C_out base case), so a
// pair with a single-relation side needs no addition and no memo read for it.
// Fold one split whose side costs are loaded (cost 0 for a single relation).
__device__ __forceinline__ void fold_costs(uint32_t sl, uint32_t sr, double cl, double cr, unsigned long long& bx,
                                           uint32_t& bl)
{
    const bool ml = (sl & (sl - 1u)) != 0u, mr = (sr & (sr - 1u)) != 0u;
    // with one side a single relation (cost +0.0) the sum is the other cost
    // exactly: OR of the bit patterns, no FP64 instruction
    const unsigned long long xb =
        (ml && mr) ? (unsigned long long)__double_as_longlong(__dadd_rn(cl, cr))
                   : ((unsigned long long)__double_as_longlong(cl) | (unsigned long long)__double_as_longlong(cr));
    const uint32_t l = sl < sr ? sl : sr;
    if (better_x(xb, l, bx, bl)) {
        bx = xb;
        bl = l;
    }
}

template <class Memo>
__device__ __forceinline__ void fold_pair(uint32_t sl, uint32_t sr, const Memo& memo, DevCounters* cnt,
                                          unsigned long long& bx, uint32_t& bl)
{
    const double cl = (sl & (sl - 1u)) ? memo.get_cost(sl, cnt) : 0.0;
    const double cr = (sr & (sr - 1u)) ? memo.get_cost(sr, cnt) : 0.0;
    fold_costs(sl, sr, cl, cr, bx, bl);
}

// cost(S) = x* + card(S) for the chosen split.
__device__ __forceinline__ double set_cost(unsigned long long bx, double card_s)
{
    return __dadd_rn(__longlong_as_double((long long)bx), card_s);
}

constexpr unsigned long long kNoX = 0xffffffffffffffffull;

// Find-Blocks (Sec. 3.2.2; Algorithm 4): the blocks of G[S] as bitmaps.
// A search from min(S) gives a spanning tree (parent of each vertex; anc[v] =
// the tree edges on the path root..v, each edge named by its child vertex).
// Every non-tree edge (x, y) closes the fundamental cycle whose tree edges are
// anc[x] xor anc[y].  Two tree edges lie in one block exactly when a chain of
// fundamental cycles sharing tree edges joins them, so merging overlapping
// cycle edge-sets gives one class per block with a cycle; its vertices are
// the class's child vertices plus their parents.  A tree edge on no cycle is
// a bridge, a block of its own two vertices.  Returns the number of blocks.
//
// With `side` given, a bridge block j also gets side[j]: the side of S that
// holds its lower vertex once the bridge is removed (grow({min}, S \ {max})
// for that block's only pair).  A bridge is a tree edge (x, par[x]) and its
// removal cuts off exactly x's subtree, computed for every x bottom-up over
// the discovery order.  Other blocks get side[j] = 0.
__device__ __forceinline__ int find_blocks(uint32_t s, const uint32_t* MPDP_RESTRICT adj,
                                           uint32_t* MPDP_RESTRICT blk, uint32_t* MPDP_RESTRICT side = nullptr)
{
    uint8_t par[kMaxRels];
    uint32_t anc[kMaxRels];
    uint8_t ord[kMaxRels];
    int nord = 0;
    const int root = lowest(s);
    par[root] = 0xff;
    anc[root] = 0u;
    ord[nord++] = (uint8_t)root;
    uint32_t vis = 1u << root, queue = vis;
    while (queue) {
        const int x = lowest(queue);
        queue &= queue - 1u;
        uint32_t ch = adj[x] & s & ~vis;
        vis |= ch;
        queue |= ch;
        while (ch) {
            const int v = lowest(ch);
            ch &= ch - 1u;
            par[v] = (uint8_t)x;
            anc[v] = anc[x] | (1u << v);
            ord[nord++] = (uint8_t)v;
        }
    }
    uint32_t cls[kMaxRels];
    int nc = 0;
    uint32_t t = s;
    while (t) {
        const int x = lowest(t);
        t &= t - 1u;
        uint32_t ys = adj[x] & s & ~((2u << x) - 1u);  // neighbours y > x
        while (ys) {
            const int y = lowest(ys);
            ys &= ys - 1u;
            if (par[y] == x || par[x] == y) continue;  // tree edge
            uint32_t c = anc[x] ^ anc[y];
            int j = 0;
            while (j < nc) {
                if (cls[j] & c) {
                    c |= cls[j];
                    cls[j] = cls[--nc];
                } else {
                    j++;
                }
            }
            cls[nc++] = c;
        }
    }
    int nb = 0;
    uint32_t in_cycle = 0u;
    for (int j = 0; j < nc; j++) {
        uint32_t c = cls[j], b = c;
        in_cycle |= c;
        while (c) {
            const int v = lowest(c);
            c &= c - 1u;
            b |= 1u << par[v];
        }
        blk[nb++] = b;
    }
    uint32_t br = s & ~in_cycle & ~(1u << root);
    if (side) {
        for (int j = 0; j < nb; j++) side[j] = 0u;
        if (br) {
            // subtree masks, children before parents (reverse discovery order)
            uint32_t sub[kMaxRels];
            for (int i = 0; i < nord; i++) sub[ord[i]] = 1u << ord[i];
            for (int i = nord - 1; i > 0; i--) sub[par[ord[i]]] |= sub[ord[i]];
            while (br) {
                const int v = lowest(br);
                br &= br - 1u;
                const int p = par[v];
                blk[nb] = (1u << v) | (1u << p);
                side[nb++] = v < p ? sub[v] : s ^ sub[v];
            }
        }
        return nb;
    }
    while (br) {
        const int v = lowest(br);
        br &= br - 1u;
        blk[nb++] = (1u << v) | (1u << par[v]);
    }
    return nb;
}

// Every pair of B's vertices adjacent (then every bipartition of B is a CCP).
__device__ __forceinline__ bool is_clique(uint32_t b, const uint32_t* MPDP_RESTRICT adj)
{
    uint32_t t = b;
    while (t) {
        const int v = lowest(t);
        t &= t - 1u;
        if ((adj[v] & b) != (b ^ (1u << v))) return false;
    }
    return true;
}

// S_l of a CCP (lb, rb) of a block of S: grow(lb, S \ rb), which is lb
// itself when the block is all of S.
__device__ __forceinline__ uint32_t left_side(uint32_t s, uint32_t lb, uint32_t rb, const uint32_t* MPDP_RESTRICT adj)
{
    return (lb | rb) == s ? lb : grow(lb, s & ~rb, adj);
}

// Unordered bipartitions of a block B visited by the enumeration: every lb
// holding min(B), except lb = B: 2^(|B|-1) - 1.
__device__ __forceinline__ uint32_t block_pairs(uint32_t b) { return (1u << (__popc(b) - 1)) - 1u; }

// Deposit the low bits of t into the set bits of mask, lowest first.
__device__ __forceinline__ uint32_t deposit(uint32_t t, uint32_t mask)
{
    uint32_t r = 0u;
    while (t && mask) {
        const uint32_t low = mask & (0u - mask);
        if (t & 1u) r |= low;
        t >>= 1;
        mask ^= low;
    }
    return r;
}

}  // namespace mpdp
