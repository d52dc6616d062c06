// persist.h -- the control block of a persistent serving kernel and its protocol.
//
// A persistent kernel stays resident on its stream and advances its group's resident
// requests one chunk per generation, instead of one launch per chunk.  The host and
// the kernel talk through pinned host memory mapped into the device (PersistCtl, the
// slot table, the slot-id list and the status words):
//   host:   writes the generation's slot ids, n_items and chunk, then (release) the
//           doorbell = generation number;
//   device: thread 0 of every CTA waits (bounded, %globaltimer) until the doorbell
//           reaches the next generation or `quit` is set, then every CTA advances its
//           share of the items; each instance that finishes (or goes non-finite) is
//           appended to the completion ring; each CTA then adds one to `done`;
//   host:   the generation is complete when done == grid x generation; it reads the
//           ring, the status words and the slot table's remaining counts.
// A wait that runs out (about a second with no doorbell and no quit) writes CHO_ETIMEOUT
// into `status` and ends the kernel, so a stalled host never hangs the device.
#pragma once

#include <cstdint>

#include "cho_internal.h"

namespace cho {

struct PersistCtl {
    uint64_t doorbell;      // host -> device: generation to run (1, 2, ...)
    int32_t quit;           // host -> device: leave the loop at the next wait
    int32_t pad0;
    int64_t n_items;        // host -> device: slot ids of this generation
    int64_t chunk;          // host -> device: steps per slot (min with its remaining)
    unsigned long long done;        // device -> host: CTAs that finished a generation (cumulative)
    int32_t status;                 // device -> host: CHO_ETIMEOUT after a wait ran out
    uint32_t pad1;
    unsigned long long ring_head;   // device -> host: completions appended (cumulative)
};

// Device-side views of the mapped arrays of one persistent group.
struct PersistIO {
    PersistCtl* ctl;
    const int32_t* slot_ids;    // [n_items] of the current generation
    SlotDesc* slots;            // the engine's slot table
    int32_t* status;            // per slot
    int32_t* ring;              // completion ring of slot ids
    uint32_t ring_cap;
};

constexpr unsigned long long kPersistWaitNs = 1000000000ull;

// Persistent kernels of the rk4_small family (padded size S, 64 threads per CTA) and of
// the chain family (P DOFs per thread; chain_persist_threads(P) threads per CTA, which
// holds chains of s < 64 P for P < 8 and s <= 2048 for P = 8).
cudaError_t launch_rk4_small_persist(int S, const PersistIO& pio, bool fp64, int grid, cudaStream_t st);
cudaError_t launch_rk4_chain_persist(int P, const PersistIO& pio, bool fp64, int grid, cudaStream_t st);
int chain_persist_threads(int P);

}  // namespace cho
