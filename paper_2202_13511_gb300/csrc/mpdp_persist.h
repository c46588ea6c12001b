// Host interface of the persistent serving engine (mpdp_persist.cu): one
// resident kernel optimizes many exact-mode queries at once, each in its own
// query slot, while the host keeps adding requests through a ring in pinned,
// device-mapped memory.
#pragma once

#include <cstdint>
#include <vector>

#include "../../include/mpdp.h"

namespace mpdp {

struct PersistEngine;

struct PersistResult {
    int32_t slot = -1;
    int64_t ticket = -1;
    int32_t status = MPDP_OK;
    double cost = 0.0;
    std::vector<mpdp_plan_node> nodes;
};

// Largest query (relations) a slot of `slot_budget_bytes` holds (0: 25); 0 if
// none fits.
int persist_max_rels(uint64_t slot_budget_bytes);

// `slots` query slots sized for queries of at most max_rels relations, with
// the kernel knobs of `kernel` (dense memo only).
int persist_create(PersistEngine** out, int device, int slots, int max_rels, const mpdp_config& kernel);
void persist_destroy(PersistEngine* e);

int persist_slots(const PersistEngine* e);
int persist_max_rels(const PersistEngine* e);

// Hand a validated request to free slot `slot`; starts the kernel when it is
// not running.
int persist_submit(PersistEngine* e, int slot, int64_t ticket, int n, int m, const double* card,
                   const mpdp_edge* edges);

// Finished requests since the last call (their slots are free again); keeps
// the kernel running while a slot is busy.
int persist_poll(PersistEngine* e, std::vector<PersistResult>& done);

// Slots with a request on the device.
int persist_busy(const PersistEngine* e);

}  // namespace mpdp
