// Batched stepping of several simulations of one kernel combination (internal to the library).
//
// A Batch holds a device table of up to kBatchSlots simulations and one CUDA graph of a
// batched time step: every stage of the step (moments, force, u-solve loop, derivatives,
// collision) is one persistent launch whose blocks walk the tiles of all simulations in the
// table, and the u-solve loop runs until every simulation's solve has stopped.  A chunk of
// steps is that graph launched once per step; each simulation takes its own number of steps
// (it idles once they are done).  Results are bitwise those of lbm_step on each simulation.
#pragma once

#include <cstdint>

#include "lbm.h"
#include "lbm_common.h"

namespace lbm {

struct Batch;

// Batch key of a simulation: its kernel combination and its size class (sites within a factor
// of 4).  Simulations batch together only when their keys are equal: a batch steps in lockstep,
// so a small simulation beside a much larger one would wait for it at every stage.
int batch_key(int lattice, const int64_t dims[3], const lbm_params& prm);
int batch_key_of(const lbm_sim* s);

// A batch for the key of `proto` whose launches go to `stream`.
int batch_create(const lbm_sim* proto, cudaStream_t stream, Batch** out);
// Put simulation s (same key, no work in flight) into a free slot.
int batch_attach(Batch* b, int slot, lbm_sim* s);
void batch_detach(Batch* b, int slot);
// Launch a chunk: slot k takes steps[k] steps (0: idle).  Asynchronous on the batch stream.
int batch_launch(Batch* b, const int64_t* steps);
// Once the chunk has completed: record the steps on each simulation (buffer parity, count).
void batch_account(Batch* b, const int64_t* steps);
void batch_destroy(Batch* b);

}  // namespace lbm
