// acoustic_common.cuh -- parameters, boundary images and the energy reduction
// shared by the acoustic kernels.
#pragma once
#include <stdint.h>
#include "wave_arith.cuh"

namespace wave {

enum { BC_PERIODIC = 0, BC_RIGID = 1 };

// Everything one acoustic step needs. Fields are pitched arrays of the
// storage type: element (i, j, k) at i + sy*j + sz*k.
struct AcParams {
    int n[3];
    int bc[3];                 // per axis
    int64_t sy, sz;
    void *p, *tp;
    void *v[3], *tv[3];
    const void *a[3];          // per-point multipliers (storage type; binary32 for
                               // the pair precision) or nullptr
    const void *b;
    uint32_t a_uni[3], b_uni;  // uniform multipliers (the same type's bits)
    // source (arithmetic-format table indexed by global step)
    int64_t src_q;             // linear pitched index of the source point, -1 none
    int src_i, src_j, src_k;   // its grid coordinates (-1 none)
    const void *src;
    int64_t src_nt;
    int64_t step;              // global index of the step being taken
    // energy
    int energy;                // accumulate E^{n+1/2} in this launch
    double *e_part;            // one partial per block
    unsigned int *e_count;     // blocks finished (reset by the last block)
    double *e_out;             // result slot (physical units)
    double e_factor;           // 0.5 h^(d-1) P0^2 dt / Z0
    // z slab of a larger grid (3D streaming kernels): two ghost planes of the
    // field this half step differentiates along z (p for the velocities, v_z
    // for the pressure), pitched like the fields; zg_lo holds the grid planes
    // z0-2, z0-1 below the slab, zg_hi the planes z1, z1+1 above it. nullptr:
    // that face is a face of the grid and its boundary image applies.
    const void *zg_lo, *zg_hi;
};

// Boundary images along one axis with N cells (Section 3 periodic wrap; rigid
// p = 0 walls at nodes 0 and N read p odd and the normal velocity even).
// Returns +1 / -1 (sign of the image) or 0 (the wall node itself).
__device__ __forceinline__ int img_node(int m, int N, int bc, int &out) {
    if (m >= 0 && m < N) { out = m; return 1; }
    if (bc == BC_PERIODIC) { out = m < 0 ? m + N : m - N; return 1; }
    if (m < 0) { out = -m; return -1; }
    if (m == N) { out = 0; return 0; }
    out = 2 * N - m; return -1;
}
__device__ __forceinline__ int img_half(int m, int N, int bc, int &out) {
    if (m >= 0 && m < N) { out = m; return 1; }
    if (bc == BC_PERIODIC) { out = m < 0 ? m + N : m - N; return 1; }
    out = m < 0 ? -1 - m : 2 * N - 1 - m;
    return 1;
}

// Bits of a uniform multiplier as the storage type.
__device__ __forceinline__ void from_bits(uint32_t u, uint16_t &s) { s = static_cast<uint16_t>(u); }
__device__ __forceinline__ void from_bits(uint32_t u, float &s) { s = __uint_as_float(u); }

// Multiplier at point q: per-point array when present, else the uniform value
// (both in the policy's multiplier storage, CoefOf<P>).
template <class P>
__device__ __forceinline__ typename P::A coef(const void *arr, uint32_t uni, int64_t q) {
    typename CoefOf<P>::S s;
    if (arr) s = static_cast<const typename CoefOf<P>::S *>(arr)[q];
    else from_bits(uni, s);
    return CoefOf<P>::ld(s);
}

template <class P>
__device__ __forceinline__ float coef_f32(const void *arr, uint32_t uni, int64_t q) {
    typename CoefOf<P>::S s;
    if (arr) s = static_cast<const typename CoefOf<P>::S *>(arr)[q];
    else from_bits(uni, s);
    return CoefOf<P>::f32(s);
}

// Energy term helpers: products in binary32 (exact for half / bfloat16
// operands), one correctly rounded division.
__device__ __forceinline__ float e_term(float x, float y, float w) {
    return __fdiv_rn(__fmul_rn(x, y), w);
}

// Block sum of a double, then a deterministic last-block reduction of the
// per-block partials in block order. Writes factor * total to *e_out.
// Must be called by every thread of the block.
__device__ __forceinline__ void energy_reduce(double val, double *e_part, unsigned int *e_count,
                                              double *e_out, double factor) {
    __shared__ double warp_sums[32];
    __shared__ bool is_last;
    const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
    const int nthreads = blockDim.x * blockDim.y * blockDim.z;
    for (int off = 16; off > 0; off >>= 1) val += __shfl_down_sync(0xffffffffu, val, off);
    if ((tid & 31) == 0) warp_sums[tid >> 5] = val;
    __syncthreads();
    const unsigned nblocks = gridDim.x * gridDim.y * gridDim.z;
    const unsigned bid = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
    if (tid == 0) {
        double s = 0.0;
        for (int w = 0; w < (nthreads + 31) / 32; w++) s += warp_sums[w];
        e_part[bid] = s;
        __threadfence();
        unsigned prev = atomicAdd(e_count, 1u);
        is_last = (prev == nblocks - 1);
    }
    __syncthreads();
    if (is_last) {
        __threadfence();
        double s = 0.0;
        for (unsigned b = tid; b < nblocks; b += nthreads) s += __ldcg(&e_part[b]);
        for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
        __syncthreads();
        if ((tid & 31) == 0) warp_sums[tid >> 5] = s;
        __syncthreads();
        if (tid == 0) {
            double tot = 0.0;
            for (int w = 0; w < (nthreads + 31) / 32; w++) tot += warp_sums[w];
            *e_out = tot * factor;
            *e_count = 0u;
        }
    }
}

__device__ __forceinline__ void energy_reduce(double val, const AcParams &prm) {
    energy_reduce(val, prm.e_part, prm.e_count, prm.e_out, prm.e_factor);
}

}  // namespace wave
