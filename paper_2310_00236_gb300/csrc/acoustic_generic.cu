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
#include "wave_kernels.h"

namespace wave {

template <class P>
__device__ __forceinline__ typename P::A read_signed(const typename P::S *f, int64_t q, int sign) {
    if (sign == 0) return P::zero();
    typename P::A v = P::ld(f[q]);
    return sign > 0 ? v : P::neg(v);
}

template <class P, int COMP, int NDIM>
__global__ void __launch_bounds__(128) kv_generic(AcParams prm) {
    using S = typename P::S;
    using A = typename P::A;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = (NDIM == 3) ? blockIdx.z : 0;
    if (i >= prm.n[0] || j >= prm.n[1]) return;
    const int idx[3] = {i, j, k};
    const int64_t str[3] = {1, prm.sy, prm.sz};
    const int64_t q = i + prm.sy * j + prm.sz * k;
    const S *p = static_cast<const S *>(prm.p);
#pragma unroll
    for (int c = 0; c < NDIM; c++) {
        // v_c at m + 1/2 along axis c reads p at nodes m-1, m, m+1, m+2
        const int m = idx[c];
        const int64_t base = q - str[c] * m;
        A f[4];
#pragma unroll
        for (int t = 0; t < 4; t++) {
            int mm;
            int sg = img_node(m - 1 + t, prm.n[c], prm.bc[c], mm);
            f[t] = read_signed<P>(p, base + str[c] * mm, sg);
        }
        A D = stencil<P>(f[0], f[1], f[2], f[3]);
        A inc = P::mul(coef<P>(prm.a[c], prm.a_uni[c], q), D);
        S *v = static_cast<S *>(prm.v[c]);
        S *tv = static_cast<S *>(prm.tv[c]);
        S V = v[q];
        S T = COMP ? tv[q] : S(0);
        update<P, COMP>(V, T, inc);
        v[q] = V;
        if (COMP) tv[q] = T;
    }
}

template <class P, int COMP, int NDIM>
__global__ void __launch_bounds__(128) kp_generic(AcParams prm) {
    using S = typename P::S;
    using A = typename P::A;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = (NDIM == 3) ? blockIdx.z : 0;
    const bool inside = i < prm.n[0] && j < prm.n[1];
    double e = 0.0;
    if (inside) {
        const int idx[3] = {i, j, k};
        const int64_t str[3] = {1, prm.sy, prm.sz};
        const int64_t q = i + prm.sy * j + prm.sz * k;
        A R = P::zero();
#pragma unroll
        for (int c = 0; c < NDIM; c++) {
            // p at node m along c reads v_c at m-2, m-1, m, m+1 (+1/2)
            const int m = idx[c];
            const int64_t base = q - str[c] * m;
            const S *v = static_cast<const S *>(prm.v[c]);
            A f[4];
#pragma unroll
            for (int t = 0; t < 4; t++) {
                int mm;
                img_half(m - 2 + t, prm.n[c], prm.bc[c], mm);
                f[t] = P::ld(v[base + str[c] * mm]);
            }
            A D = stencil<P>(f[0], f[1], f[2], f[3]);
            R = (c == 0) ? D : P::add(R, D);
        }
        if (q == prm.src_q && prm.step < prm.src_nt)
            R = P::add(R, static_cast<const A *>(prm.src)[prm.step]);
        A inc = P::mul(coef<P>(prm.b, prm.b_uni, q), R);
        S *p = static_cast<S *>(prm.p);
        S *tp = static_cast<S *>(prm.tp);
        const S p_old = p[q];
        S V = p_old;
        S T = COMP ? tp[q] : S(0);
        update<P, COMP>(V, T, inc);
        p[q] = V;
        if (COMP) tp[q] = T;
        if (prm.energy) {
            e = (double)e_term(P::to_f32(p_old), P::to_f32(V), coef_f32<P>(prm.b, prm.b_uni, q));
#pragma unroll
            for (int c = 0; c < NDIM; c++) {
                float vc = P::to_f32(static_cast<const S *>(prm.v[c])[q]);
                e += (double)e_term(vc, vc, coef_f32<P>(prm.a[c], prm.a_uni[c], q));
            }
        }
    }
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
