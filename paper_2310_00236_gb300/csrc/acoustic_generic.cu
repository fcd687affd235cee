// acoustic_generic.cu -- one-thread-per-point acoustic leapfrog kernels.
//
// These handle every grid size, both boundary kinds and every precision. They
// are the reference shape of the computation on the GPU and the path for 2D
// grids and sizes the streaming 3D kernels do not take.
//
// Per step (Algorithm 1 / 2 of Section 4, extended to 3D):
//   K-v: v_c^{n+1/2} = v_c^{n-1/2} + a_c * D_c(p^n)           for c < ndim
//   K-p: R = D_x(v_x) + D_y(v_y) [+ D_z(v_z)] [+ s]; p^{n+1} = p^n + b * R
// with D the fourth-order staggered difference of Section 3 and "+" the plain
// or compensated update.
#include <cuda_runtime.h>
#include "acoustic_common.cuh"
#include "acoustic_point.cuh"
#include "wave_kernels.h"

namespace wave {

template <class P, int COMP, int NDIM>
__global__ void __launch_bounds__(128) kv_generic(AcParams prm) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = (NDIM == 3) ? blockIdx.z : 0;
    if (i >= prm.n[0] || j >= prm.n[1]) return;
    kv_point<P, COMP, NDIM>(prm, i, j, k);
}

template <class P, int COMP, int NDIM>
__global__ void __launch_bounds__(128) kp_generic(AcParams prm) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = (NDIM == 3) ? blockIdx.z : 0;
    double e = 0.0;
    if (i < prm.n[0] && j < prm.n[1]) e = kp_point<P, COMP, NDIM>(prm, i, j, k, prm.step, prm.energy != 0);
    if (prm.energy) energy_reduce(e, prm);
}

template <class P, int COMP, int NDIM>
static cudaError_t launch_t(const AcParams &prm, int half_step, cudaStream_t st) {
    dim3 block(32, 4, 1);
    dim3 grid((prm.n[0] + 31) / 32, (prm.n[1] + 3) / 4, NDIM == 3 ? prm.n[2] : 1);
    if (half_step == 0) kv_generic<P, COMP, NDIM><<<grid, block, 0, st>>>(prm);
    else kp_generic<P, COMP, NDIM><<<grid, block, 0, st>>>(prm);
    return cudaGetLastError();
}

template <class P, int NDIM>
static cudaError_t launch_c(const AcParams &prm, int comp, int half_step, cudaStream_t st) {
    switch (comp) {
    case 0: return launch_t<P, 0, NDIM>(prm, half_step, st);
    case 3: return launch_t<P, 3, NDIM>(prm, half_step, st);
    default: return launch_t<P, 6, NDIM>(prm, half_step, st);
    }
}

template <int NDIM>
static cudaError_t launch_p(const AcParams &prm, int prec, int comp, int half_step,
                            cudaStream_t st) {
    switch (prec) {
    case PREC_FP32: return launch_c<F32, NDIM>(prm, comp, half_step, st);
    case PREC_FP16: return launch_c<F16, NDIM>(prm, comp, half_step, st);
    case PREC_BF16: return launch_c<BF16, NDIM>(prm, comp, half_step, st);
    case PREC_FP16_F32ARITH: return launch_c<F16W, NDIM>(prm, comp ? 3 : 0, half_step, st);
    case PREC_BF16_F32ARITH: return launch_c<BF16W, NDIM>(prm, comp ? 3 : 0, half_step, st);
    case PREC_FP16_PAIRS: return launch_t<F16WP, 3, NDIM>(prm, half_step, st);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t acoustic_generic_half_step(const AcParams &prm, int ndim, int prec, int comp,
                                       int half_step, cudaStream_t st) {
    return ndim == 3 ? launch_p<3>(prm, prec, comp, half_step, st)
                     : launch_p<2>(prm, prec, comp, half_step, st);
}

unsigned acoustic_generic_blocks(const AcParams &prm, int ndim) {
    return ((prm.n[0] + 31) / 32) * ((prm.n[1] + 3) / 4) * (ndim == 3 ? prm.n[2] : 1);
}

}  // namespace wave
