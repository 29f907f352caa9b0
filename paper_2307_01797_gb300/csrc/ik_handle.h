// ik_handle.h -- access to a handle's state for the translation units of
// libitokmc beside ik_api.cu (checkpoints, seeding).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/itokmc.h"
#include "ik_state.h"

namespace ik {

struct HandleView {
    itokmc_config* cfg;
    Params* P;
    Dev* d;
    cudaStream_t s;
    uint32_t* N;          // particle count (host copy)
    uint32_t cap;         // particle capacity
    int64_t* step;        // step counter
    uint64_t G;           // cells of all realizations
    int field_prec;
    uint64_t Gp;          // particle cells (G per species block)
    int* stage;           // stage order: 0 particles not deposited since they
                          // last changed, 1 transported, 2 KMC done
};

// Fills *v after waiting for the handle's streams (nothing of a step may be
// in flight while the state is read or replaced).  ITOKMC_ERR_ARG /
// ITOKMC_ERR_POISONED / ITOKMC_ERR_CUDA as the other entry points.
int handle_view(itokmc_handle* h, HandleView* v);
// Records msg as the handle's last error and returns code.
int handle_fail(itokmc_handle* h, int code, const char* msg);
// Re-deposits the particles and solves the field of the current state.
int handle_solve_field(itokmc_handle* h);
// Samples the particles of every realization from Gaussian seeds (ik_seed.cu;
// the blobs validated by the caller).
int seed_blobs(itokmc_handle* h, const itokmc_seed_blob* blobs, int nb, int flags);

}  // namespace ik
