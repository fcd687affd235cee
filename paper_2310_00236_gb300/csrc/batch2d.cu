// batch2d.cu -- many independent 2D acoustic problems ("shots") advanced by
// the same launches.
//
// One leapfrog step of every shot is two persistent launches over a single
// work list of (shot, tile) items: the velocity half step of every tile of
// every shot, then the pressure half step. The per-point arithmetic is the one
// of the one-thread-per-point kernels (acoustic_point.cuh), so a shot advanced
// in a batch carries the same bits as when advanced alone. Each shot's step
// counter (the time index of its source wavelet) lives in device memory and
// is advanced by a small kernel after each step, so a sequence of steps can be
// captured once into a CUDA graph and replayed. Energies are reduced per item
// and then per shot in item order (deterministic).
#include <cuda_runtime.h>

#include "acoustic_point.cuh"
#include "batch.h"
#include "wave_kernels.h"

namespace wave {

constexpr int kMaxShots = 1024;

// Shot index of a work item: the last s with item0[s] <= item (binary search).
__device__ __forceinline__ int shot_of(const int *item0, int nshots, int item) {
    int lo = 0, hi = nshots - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (item0[mid] <= item) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

template <class P, int COMP, int HALF>
__global__ void __launch_bounds__(256) batch_half_step(BatchShot *shots, const int *item0, int nshots,
                                                      int nitems, int bx, int by, int energy,
                                                      double *item_part) {
    __shared__ int s_item0[kMaxShots + 1];
    __shared__ AcParams s_prm;
    __shared__ int64_t s_step;
    __shared__ int s_tiles_x, s_start;
    __shared__ double warp_sums[8];
    for (int t = threadIdx.x; t <= nshots; t += blockDim.x) s_item0[t] = item0[t];
    __syncthreads();
    for (int item = blockIdx.x; item < nitems; item += gridDim.x) {
        if (threadIdx.x == 0) {
            const int s = shot_of(s_item0, nshots, item);
            s_prm = shots[s].prm;
            s_step = shots[s].step;
            s_tiles_x = (s_prm.n[0] + bx - 1) / bx;
            s_start = s_item0[s];
        }
        __syncthreads();
        const int local = item - s_start;
        const int i = (local % s_tiles_x) * bx + (int)threadIdx.x % bx;
        const int j = (local / s_tiles_x) * by + (int)threadIdx.x / bx;
        const bool inside = i < s_prm.n[0] && j < s_prm.n[1];
        if (HALF == 0) {
            if (inside) kv_point<P, COMP, 2>(s_prm, i, j, 0);
        } else {
            double e = 0.0;
            if (inside) e = kp_point<P, COMP, 2>(s_prm, i, j, 0, s_step, energy != 0);
            if (energy) {
                for (int off = 16; off > 0; off >>= 1) e += __shfl_down_sync(0xffffffffu, e, off);
                if ((threadIdx.x & 31) == 0) warp_sums[threadIdx.x >> 5] = e;
                __syncthreads();
                if (threadIdx.x == 0) {
                    double t = 0.0;
                    for (int w = 0; w < (int)(blockDim.x >> 5); w++) t += warp_sums[w];
                    item_part[item] = t;
                }
            }
        }
        __syncthreads();
    }
}

// Per-shot energy: the item partials of each shot summed in item order.
__global__ void batch_energy_reduce(BatchShot *shots, const int *item0, const double *item_part) {
    const int s = blockIdx.x;
    __shared__ double warp_sums[8];
    double e = 0.0;
    for (int it = item0[s] + threadIdx.x; it < item0[s + 1]; it += blockDim.x) e += item_part[it];
    for (int off = 16; off > 0; off >>= 1) e += __shfl_down_sync(0xffffffffu, e, off);
    if ((threadIdx.x & 31) == 0) warp_sums[threadIdx.x >> 5] = e;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) t += warp_sums[w];
        *shots[s].prm.e_out = t * shots[s].prm.e_factor;
    }
}

__global__ void batch_advance(BatchShot *shots, int nshots) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s < nshots) shots[s].step++;
}

template <class P, int COMP>
static cudaError_t launch_pc(const BatchLaunch &L, bool energy, cudaStream_t st) {
    const int threads = L.bx * L.by;
    batch_half_step<P, COMP, 0><<<L.grid, threads, 0, st>>>(L.shots, L.item0, L.nshots, L.nitems, L.bx,
                                                            L.by, 0, L.item_part);
    batch_half_step<P, COMP, 1><<<L.grid, threads, 0, st>>>(L.shots, L.item0, L.nshots, L.nitems, L.bx,
                                                            L.by, energy ? 1 : 0, L.item_part);
    if (energy) batch_energy_reduce<<<L.nshots, 256, 0, st>>>(L.shots, L.item0, L.item_part);
    batch_advance<<<(L.nshots + 127) / 128, 128, 0, st>>>(L.shots, L.nshots);
    return cudaGetLastError();
}

template <class P>
static cudaError_t launch_p(const BatchLaunch &L, int comp, bool energy, cudaStream_t st) {
    switch (comp) {
    case 0: return launch_pc<P, 0>(L, energy, st);
    case 3: return launch_pc<P, 3>(L, energy, st);
    default: return launch_pc<P, 6>(L, energy, st);
    }
}

int batch_max_shots() { return kMaxShots; }

cudaError_t batch_step(const BatchLaunch &L, int prec, int comp, bool energy, cudaStream_t st) {
    if (L.bx * L.by > 256 || (L.bx * L.by) % 32 != 0) return cudaErrorInvalidValue;
    switch (prec) {
    case PREC_FP32: return launch_p<F32>(L, comp, energy, st);
    case PREC_FP16: return launch_p<F16>(L, comp, energy, st);
    case PREC_BF16: return launch_p<BF16>(L, comp, energy, st);
    case PREC_FP16_F32ARITH: return launch_p<F16W>(L, comp ? 3 : 0, energy, st);
    case PREC_BF16_F32ARITH: return launch_p<BF16W>(L, comp ? 3 : 0, energy, st);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace wave
