// batch.h -- launch description of the batched multi-shot 2D kernels.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include "acoustic_common.cuh"

namespace wave {

// One shot of a batch, resident in device memory.
struct BatchShot {
    AcParams prm;   // the shot's grid, fields, multipliers, source, energy slot
    int64_t step;   // global step index of the shot (source time index)
};

struct BatchLaunch {
    BatchShot *shots;   // device array [nshots]
    const int *item0;   // device array [nshots + 1]: first work item of each shot
    double *item_part;  // device array [nitems]: per-item energy partials
    int nshots, nitems;
    int bx, by;         // tile (= thread block) shape, bx * by threads
    int grid;           // persistent grid size
};

// One batched step (velocity and pressure half steps of every shot, optional
// per-shot energy, step counters advanced).
cudaError_t batch_step(const BatchLaunch &L, int prec, int comp, bool energy, cudaStream_t st);
int batch_max_shots();

}  // namespace wave
