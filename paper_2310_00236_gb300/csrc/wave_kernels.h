// wave_kernels.h -- internal interface between the C ABI and the kernels.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace wave {

// Same values as wave_precision in include/wave.h.
enum { PREC_FP64 = 0, PREC_FP32 = 1, PREC_FP16 = 2, PREC_BF16 = 3,
       PREC_FP16_F32ARITH = 4, PREC_BF16_F32ARITH = 5, PREC_FP16_PAIRS = 6 };

struct AcParams;

// One acoustic half step with the one-thread-per-point kernels:
// half_step 0 = velocities, 1 = pressure (with source and optional energy).
cudaError_t acoustic_generic_half_step(const AcParams &prm, int ndim, int prec, int comp,
                                       int half_step, cudaStream_t st);
// Number of blocks the generic pressure kernel launches (energy partials).
unsigned acoustic_generic_blocks(const AcParams &prm, int ndim);

// Streaming 3D kernels (n[0] a multiple of the vector width, 3D only).
bool acoustic_stream_supported(const AcParams &prm, int ndim, int prec);
unsigned acoustic_stream_blocks(const AcParams &prm, int prec, int zchunk);
cudaError_t acoustic_stream_half_step(const AcParams &prm, int prec, int comp, int half_step,
                                      int zchunk, cudaStream_t st);

// One-pass 3D step (fused velocity and pressure half steps) with a TMA
// shared-memory pipeline; reads in[] (p, vx, vy, vz, tvx, tvy, tvz) and tp,
// writes out[] and tp_out (= tp: t_p in place; the pair precision, whose
// stencils read t_p in the halos, gives the other set's t_p). maps: the tensor
// maps of the input set (from acoustic_fused_encode, with that set's t_p). err:
// device word set to 1 if a bounded wait expires.
bool acoustic_fused_supported(const AcParams &prm, int ndim, int prec);
unsigned acoustic_fused_blocks(const AcParams &prm, int prec, int zchunk);
size_t fused_maps_bytes();
bool acoustic_fused_encode(void *out_maps, const AcParams &prm, const void *const in[7], const void *tp,
                           int prec, int comp);
cudaError_t acoustic_fused_step(const AcParams &prm, const void *maps, const void *const in[7],
                                void *const out[7], void *tp, void *tp_out, int prec, int comp, int zchunk,
                                int *err, cudaStream_t st);

// Cluster-resident 2D steps (acoustic2d_cluster.cu): the whole state of a
// small 2D grid in the shared memory of one cluster of up to 16 CTAs, any
// number of steps per launch.
struct ClusterRun {
    AcParams prm;           // global arrays (pitch prm.sy); prm.step: global index of the first step
    int64_t nsteps;
    double *e_trace;        // energies after steps 0 .. e_trace_n - 1 (physical units), or nullptr
    int64_t e_trace_n;
    double *e_last;         // energy after the last step, or nullptr
    const int64_t *rec_q;   // receivers: pitched linear indices of field rec_field (0 p, 1 v_x, 2 v_y)
    int nrec, rec_field;
    float *traces;          // traces[s * nrec + r] for steps s < rec_n
    int64_t rec_n;
};
struct ClusterPlan {
    int ctas = 0, rows = 0, rpi = 1;  // CTAs (= bands), rows per band, rows per work item
    size_t smem = 0;                  // dynamic shared memory per CTA
};
// A cluster shape that holds the grid's state and that the device can run;
// false if none (the grid is too large, or the precision has no such kernel).
bool acoustic_cluster_plan(const AcParams &prm, int prec, int comp, ClusterPlan &pl);
cudaError_t acoustic_cluster_steps(const ClusterRun &run, const ClusterPlan &pl, int prec, int comp,
                                   cudaStream_t st);

// A bounded mbarrier wait that nothing completes (polls iterations), setting
// *err to 1 when it expires: the self-test of the device error path.
cudaError_t selftest_wait(int *err, uint32_t polls, cudaStream_t st);

// Receiver sampling: traces[r] = float(field[q[r]]) for r < nrec.
cudaError_t sample_receivers(const void *field, int elem_bytes, int is_bf16, const int64_t *q,
                             int nrec, float *traces, cudaStream_t st);

}  // namespace wave
