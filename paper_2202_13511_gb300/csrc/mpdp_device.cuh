// Device-side data layout and helpers of the MPDP path (sm_103a).
//
// Relation sets are 32-bit bitmaps (bit i = relation i), the fixed-width
// bitmap sets of the paper (Sec. 2.2, "Implementation Details"; Sec. 5).
#pragma once

#include <cstddef>
#include <cstdint>

#include "../../include/mpdp.h"

namespace mpdp {

constexpr int kMaxRels = 32;        // bitmap width
constexpr int kLevels = MPDP_MAX_LEVELS;
constexpr int kMaxEdges = kMaxRels * (kMaxRels - 1) / 2;
constexpr int kEvalThreads = 256;

// Query as staged from the host (or gathered from caller device buffers).
struct StagedQuery {
    int32_t n, n_edges, cost_model, pad;
    double card[kMaxRels];
    mpdp_edge edges[kMaxEdges];
};

// Query as the kernels read it: adjacency bitmaps and a dense selectivity
// matrix (1.0 where there is no edge).  Built on the device by k_ingest.
struct DevQuery {
    int32_t n, n_edges, pad[2];
    uint32_t adj[kMaxRels];
    double card[kMaxRels];
    double sel[kMaxRels * kMaxRels];  // sel[j * 32 + r]
};

// Per-query device counters and status word.
struct DevCounters {
    unsigned long long unranked;
    unsigned long long heavy;
    unsigned long long memo_slots;
    unsigned long long filter_steps;    // vertices expanded by the filter's tests
    unsigned long long connected[kLevels];
    unsigned long long evaluated[kLevels];
    unsigned long long ccp[kLevels];
    unsigned int list_count[kLevels];   // connected sets of level k in the list
    unsigned int heavy_count[kLevels];  // sets of level k sent to the warp kernel
    int status;                         // first MPDP_ERR_* raised on the device
    int pad;
};

struct DevResult {
    double cost;
    int32_t n_nodes;
    int32_t status;
    mpdp_plan_node nodes[2 * kMaxRels - 1];
};

// Host copy of one finished query: result and counters, read back together.
struct HostResult {
    DevResult result;
    DevCounters counters;
};

// Open-addressing memo: one table per level inside one arena.
struct alignas(16) HashSlot {
    uint32_t key;    // relation bitmap; 0 = empty (the empty set is never stored)
    uint32_t left;   // left child bitmap of the best split
    double cost;     // C_out cost of the best plan
};

struct HashLayout {
    unsigned long long base[kLevels];  // first slot of level k's table
    unsigned int mask[kLevels];        // capacity - 1 (capacity a power of two)
    unsigned long long total_slots;
};

// Record the first device error; later errors keep the first code.
__device__ __forceinline__ void raise_status(DevCounters* c, int code)
{
    atomicCAS(&c->status, 0, code);
}

__device__ __forceinline__ int lowest(uint32_t s) { return __ffs(s) - 1; }

// grow(source, restriction) of Sec. 3.2.1: every vertex of the restriction
// reachable from the source.  The loop pops one frontier vertex per step.
__device__ __forceinline__ uint32_t grow(uint32_t source, uint32_t restriction,
                                         const uint32_t* __restrict__ adj)
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
// Stops as soon as every member has been reached.
__device__ __forceinline__ bool connected(uint32_t s, const uint32_t* __restrict__ adj)
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

// card(S): product in the fixed order (relations ascending; after each
// relation r, the selectivities of its edges to smaller members j ascending).
// __dmul_rn keeps every step a separately rounded IEEE multiply.
__device__ __forceinline__ double card_of(uint32_t s, const uint32_t* __restrict__ adj,
                                          const double* __restrict__ card,
                                          const double* __restrict__ sel)
{
    double p = 1.0;
    uint32_t t = s;
    while (t) {
        int r = lowest(t);
        t &= t - 1;
        p = __dmul_rn(p, card[r]);
        uint32_t nb = adj[r] & s & ((1u << r) - 1u);
        while (nb) {
            int j = lowest(nb);
            nb &= nb - 1;
            p = __dmul_rn(p, sel[j * kMaxRels + r]);
        }
    }
    return p;
}

// Lexicographic (cost, left) order of candidate plans.
__device__ __forceinline__ bool better(double c, uint32_t l, double bc, uint32_t bl)
{
    return c < bc || (c == bc && l < bl);
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

// Memo indexed directly by the relation bitmap.
struct DenseMemo {
    double* cost;
    uint32_t* left;

    __device__ __forceinline__ void setup(char*) {}
    __device__ __forceinline__ double get_cost(uint32_t s, DevCounters*) const
    {
        return __ldg(cost + s);
    }
    __device__ __forceinline__ void get(uint32_t s, double& c, uint32_t& l, DevCounters*) const
    {
        c = cost[s];
        l = left[s];
    }
    __device__ __forceinline__ void put(uint32_t s, int, double c, uint32_t l, DevCounters*)
    {
        cost[s] = c;
        left[s] = l;
    }
};

// Memo as one open-addressing table per level (linear probing).
struct HashMemo {
    HashSlot* arena;
    const HashLayout* layout;
    // per-block copy of the level table bases and masks (shared memory)
    unsigned long long* s_base;
    unsigned int* s_mask;

    static constexpr size_t kSharedBytes = kLevels * (sizeof(unsigned long long) + sizeof(unsigned int));

    __device__ __forceinline__ void setup(char* smem)
    {
        s_base = reinterpret_cast<unsigned long long*>(smem);
        s_mask = reinterpret_cast<unsigned int*>(smem + kLevels * sizeof(unsigned long long));
        for (int i = threadIdx.x; i < kLevels; i += blockDim.x) {
            s_base[i] = layout->base[i];
            s_mask[i] = layout->mask[i];
        }
    }

    __device__ __forceinline__ bool find(uint32_t s, double& c, uint32_t& l, DevCounters* cnt) const
    {
        int lvl = __popc(s);
        const HashSlot* t = arena + s_base[lvl];
        uint32_t m = s_mask[lvl];
        uint32_t h = fmix32(s) & m;
        for (uint32_t i = 0; i <= m; i++) {
            uint4 v = __ldg(reinterpret_cast<const uint4*>(t + h));  // one 16-byte probe
            if (v.x == s) {
                l = v.y;
                c = __hiloint2double(static_cast<int>(v.w), static_cast<int>(v.z));
                return true;
            }
            if (v.x == 0u) break;
            h = (h + 1u) & m;
        }
        raise_status(cnt, MPDP_ERR_PROBE_LIMIT);
        c = __longlong_as_double(0x7ff8000000000000ll);
        l = 0xffffffffu;
        return false;
    }
    __device__ __forceinline__ double get_cost(uint32_t s, DevCounters* cnt) const
    {
        double c;
        uint32_t l;
        find(s, c, l, cnt);
        return c;
    }
    __device__ __forceinline__ void get(uint32_t s, double& c, uint32_t& l, DevCounters* cnt) const
    {
        find(s, c, l, cnt);
    }
    __device__ __forceinline__ void put(uint32_t s, int lvl, double c, uint32_t l, DevCounters* cnt)
    {
        HashSlot* t = arena + s_base[lvl];
        uint32_t m = s_mask[lvl];
        uint32_t h = fmix32(s) & m;
        for (uint32_t i = 0; i <= m; i++) {
            uint32_t old = atomicCAS(&t[h].key, 0u, s);
            if (old == 0u) {
                t[h].left = l;
                t[h].cost = c;
                return;
            }
            h = (h + 1u) & m;
        }
        raise_status(cnt, MPDP_ERR_OOM);
    }
};

}  // namespace mpdp
