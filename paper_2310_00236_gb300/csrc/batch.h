// batch.h -- launch description of the batched multi-shot 2D kernels.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include "acoustic_common.cuh"

namespace wave {

// One shot of a batch, resident in device memory.
struct BatchShot {
    AcParams prm;   // the shot's grid, fields, multipliers, source, energy slot
    int64_t step;   // index of the shot's last step taken (the next step's velocity
                    // launch advances it before the pressure launch reads it; the
                    // one-pass launch reads it and a small launch advances it after)
    // one-pass strips: the alternate buffer set of p, v_x, v_y, t_vx, t_vy
    // (t_p is updated in place) and the number of one-pass steps taken since
    // the parameters were uploaded: the set prm points to holds the state
    // when it is even, the alternate set when it is odd (the other kinds
    // update in place and leave it alone)
    void *alt_p, *alt_v[2], *alt_tv[2];
    int64_t fsteps;
    int *err;       // the context's device error word (set when a bounded wait of
                    // the persistent launch expires)
};

// Four kinds of work item:
//   BATCH_POINTS:  a bx x by tile of points, one thread per point (one block per item);
//   BATCH_STRIPS:  a strip of 32 vectors (32 * vec_width x points) by yc rows,
//                  one warp per item, streaming down the rows (two launches per step);
//   BATCH_FUSED:   the same strips with both half steps in one launch (new
//                  velocities of row j, then p of row j - 1), old state read from
//                  one buffer set and the new state written to the other;
//   BATCH_PERSIST: the same strips, every step of a call but the last (which
//                  reduces the energy, on the two-launch strips) in one
//                  cooperative launch (grid barriers between the half steps).
enum { BATCH_POINTS = 0, BATCH_STRIPS = 1, BATCH_FUSED = 2, BATCH_PERSIST = 3 };

struct BatchLaunch {
    BatchShot *shots;   // device array [nshots]
    const int *item0;   // device array [nshots + 1]: first work item of each shot
    double *item_part;  // device array [nitems]: per-item energy partials
    int nshots, nitems;
    int kind;           // BATCH_POINTS or BATCH_STRIPS
    int bx, by;         // BATCH_POINTS: tile (= thread block) shape, bx * by threads
    int yc, wpb;        // BATCH_STRIPS: rows per item, warps per block
    int grid;           // persistent grid size (blocks; BATCH_PERSIST: chosen at launch)
    unsigned int *bar;  // BATCH_PERSIST: grid-barrier counter (device)
    int *err;           // BATCH_PERSIST: set to 1 when a barrier wait expires (device)
};

// Work items of one shot of nx x ny points under a launch shape.
int64_t batch_items_of(int kind, int bx, int by, int yc, int prec, int64_t nx, int64_t ny);

// One batched step (velocity and pressure half steps of every shot, optional
// per-shot energy, step counters advanced).
cudaError_t batch_step(const BatchLaunch &L, int prec, int comp, bool energy, cudaStream_t st);
// nsteps steps of a BATCH_PERSIST launch shape in cooperative launches (the
// last step with the per-shot energy when energy_last), then the error word
// copied to every shot's context.
cudaError_t batch_persist(const BatchLaunch &L, int prec, int comp, int64_t nsteps, bool energy_last,
                          cudaStream_t st);
int batch_max_shots();

}  // namespace wave
