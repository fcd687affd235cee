// elastic2d.cu -- 2D isotropic elastic velocity-stress leapfrog (Eq. 2,
// Appendix A), one thread per grid point, every precision and update variant.
//
// Per step:
//   vx += bx * (Dx sxx + Dy sxy)
//   vy += by * (Dx sxy + Dy syy)   [+ s, added to the increment]
//   sxx += (l2m * Dx vx) + (lam * Dy vy)
//   syy += (lam * Dx vx) + (l2m * Dy vy)
//   sxy += mu * (Dx vy + Dy vx)
// with the fourth-order staggered difference of Section 3 and the plain or
// compensated update of Algorithms 1 / 2. Staggering: sxx, syy on nodes, vx at
// (i+1/2, j), vy at (i, j+1/2), sxy at (i+1/2, j+1/2).
#include <cuda_runtime.h>
#include "acoustic_common.cuh"
#include "elastic.h"
#include "elastic_common.cuh"
#include "wave_kernels.h"

namespace wave {

// Stencil of field fi along axis ax at point (i, j): f node-type along ax read at
// indices m-1..m+2, half-type at m-2..m+1. Taps: the stored values, or for the
// pair policies RN(V + T) (the image's sign applied to the sum).
template <class P>
__device__ __forceinline__ typename P::A estencil(int fi, const ElParams &e, int ax, bool node,
                                                  bool odd, bool odd_free, int i, int j) {
    using S = typename P::S;
    using A = typename P::A;
    const S *f = static_cast<const S *>(e.f[fi]);
    const S *tf = static_cast<const S *>(e.t[fi]);
    const int m = ax == 0 ? i : j;
    const int first = node ? m - 1 : m - 2;
    A v[4];
#pragma unroll
    for (int t = 0; t < 4; t++) {
        int mm;
        const int sg = emap(first + t, e.n[ax], e.bc[2 * ax], e.bc[2 * ax + 1], node, odd, odd_free, mm);
        if (sg == 0) {
            v[t] = P::zero();
        } else {
            const int64_t q = ax == 0 ? (mm + e.sy * (int64_t)j) : (i + e.sy * (int64_t)mm);
            const A x = IsPairs<P>::value ? P::add(P::ld(f[q]), P::ld(tf[q])) : P::ld(f[q]);
            v[t] = sg > 0 ? x : P::neg(x);
        }
    }
    return stencil<P>(v[0], v[1], v[2], v[3]);
}


template <class P, int COMP>
__global__ void __launch_bounds__(128) el_v(ElParams e) {
    using S = typename P::S;
    using A = typename P::A;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= e.n[0] || j >= e.n[1]) return;
    const int64_t q = i + e.sy * (int64_t)j;
    // vx: sxx node-type in x (even), sxy half-type in y (odd at walls and surface)
    A R = P::add(estencil<P>(F_SXX, e, 0, true, false, true, i, j),
                 estencil<P>(F_SXY, e, 1, false, true, true, i, j));
    A inc = P::mul(coef<P>(e.c[C_BX], e.c_uni[C_BX], q), R);
    S *vx = static_cast<S *>(e.f[F_VX]), *tvx = static_cast<S *>(e.t[F_VX]);
    S V = vx[q], T = COMP ? tvx[q] : S(0);
    update<P, COMP>(V, T, inc);
    vx[q] = V;
    if (COMP) tvx[q] = T;
    // vy: sxy half-type in x (odd), syy node-type in y (even at walls, odd at the surface)
    R = P::add(estencil<P>(F_SXY, e, 0, false, true, true, i, j),
               estencil<P>(F_SYY, e, 1, true, false, true, i, j));
    inc = P::mul(coef<P>(e.c[C_BY], e.c_uni[C_BY], q), R);
    if (q == e.src_q && e.step < e.src_nt) inc = P::add(inc, static_cast<const A *>(e.src)[e.step]);
    S *vy = static_cast<S *>(e.f[F_VY]), *tvy = static_cast<S *>(e.t[F_VY]);
    V = vy[q];
    T = COMP ? tvy[q] : S(0);
    update<P, COMP>(V, T, inc);
    vy[q] = V;
    if (COMP) tvy[q] = T;
}

template <class P, int COMP>
__global__ void __launch_bounds__(128) el_s(ElParams e) {
    using S = typename P::S;
    using A = typename P::A;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    double en = 0.0;
    if (i < e.n[0] && j < e.n[1]) {
        const int64_t q = i + e.sy * (int64_t)j;
        // nodes: vx half-type in x (odd), vy half-type in y (odd at walls, even at the surface)
        const A dxvx = estencil<P>(F_VX, e, 0, false, true, false, i, j);
        const A dyvy = estencil<P>(F_VY, e, 1, false, true, false, i, j);
        const A l2m = coef<P>(e.c[C_L2M], e.c_uni[C_L2M], q);
        const A lam = coef<P>(e.c[C_LAM], e.c_uni[C_LAM], q);
        S *sxx = static_cast<S *>(e.f[F_SXX]), *tsxx = static_cast<S *>(e.t[F_SXX]);
        S *syy = static_cast<S *>(e.f[F_SYY]), *tsyy = static_cast<S *>(e.t[F_SYY]);
        S *sxy = static_cast<S *>(e.f[F_SXY]), *tsxy = static_cast<S *>(e.t[F_SXY]);
        const S sxx0 = sxx[q], syy0 = syy[q], sxy0 = sxy[q];
        A inc = P::add(P::mul(l2m, dxvx), P::mul(lam, dyvy));
        S V = sxx0, T = COMP ? tsxx[q] : S(0);
        update<P, COMP>(V, T, inc);
        sxx[q] = V;
        if (COMP) tsxx[q] = T;
        const S sxx1 = V;
        inc = P::add(P::mul(lam, dxvx), P::mul(l2m, dyvy));
        V = syy0;
        T = COMP ? tsyy[q] : S(0);
        update<P, COMP>(V, T, inc);
        syy[q] = V;
        if (COMP) tsyy[q] = T;
        const S syy1 = V;
        // sxy: vy node-type in x (even), vx node-type in y (even)
        const A R = P::add(estencil<P>(F_VY, e, 0, true, false, false, i, j),
                           estencil<P>(F_VX, e, 1, true, false, false, i, j));
        inc = P::mul(coef<P>(e.c[C_MU], e.c_uni[C_MU], q), R);
        V = sxy0;
        T = COMP ? tsxy[q] : S(0);
        update<P, COMP>(V, T, inc);
        sxy[q] = V;
        if (COMP) tsxy[q] = T;
        if (e.energy) {
            // binary64 terms (a diagnostic reduction over a 2D grid)
            const double bx = coef_f32<P>(e.c[C_BX], e.c_uni[C_BX], q);
            const double by = coef_f32<P>(e.c[C_BY], e.c_uni[C_BY], q);
            const double L = coef_f32<P>(e.c[C_L2M], e.c_uni[C_L2M], q);
            const double M = coef_f32<P>(e.c[C_LAM], e.c_uni[C_LAM], q);
            const double mu = coef_f32<P>(e.c[C_MU], e.c_uni[C_MU], q);
            const double vxv = P::to_f32(static_cast<const S *>(e.f[F_VX])[q]);
            const double vyv = P::to_f32(static_cast<const S *>(e.f[F_VY])[q]);
            const double a0 = P::to_f32(sxx0), a1 = P::to_f32(sxx1);
            const double b0 = P::to_f32(syy0), b1 = P::to_f32(syy1);
            // weight 1/2 for vx and the normal stresses on a free surface row
            const double w = (e.bc[2] == EBC_FREE && j == 0) ? 0.5 : 1.0;
            en = w * (vxv * vxv / bx) + vyv * vyv / by;
            en += w * ((L * (a0 * a1 + b0 * b1) - M * (a0 * b1 + b0 * a1)) / (L * L - M * M));
            if (mu > 0.0) en += (double)P::to_f32(sxy0) * (double)P::to_f32(V) / mu;
        }
    }
    if (e.energy) energy_reduce(en, e.e_part, e.e_count, e.e_out, e.e_factor);
}

template <class P, int COMP>
static cudaError_t launch_t(const ElParams &e, int half, cudaStream_t st) {
    dim3 block(32, 4);
    dim3 grid((e.n[0] + 31) / 32, (e.n[1] + 3) / 4);
    if (half == 0) el_v<P, COMP><<<grid, block, 0, st>>>(e);
    else el_s<P, COMP><<<grid, block, 0, st>>>(e);
    return cudaGetLastError();
}

template <class P>
static cudaError_t launch_c(const ElParams &e, int comp, int half, cudaStream_t st) {
    switch (comp) {
    case 0: return launch_t<P, 0>(e, half, st);
    case 3: return launch_t<P, 3>(e, half, st);
    default: return launch_t<P, 6>(e, half, st);
    }
}

cudaError_t elastic_half_step(const ElParams &e, int prec, int comp, int half, cudaStream_t st) {
    switch (prec) {
    case PREC_FP32: return launch_c<F32>(e, comp, half, st);
    case PREC_FP16: return launch_c<F16>(e, comp, half, st);
    case PREC_BF16: return launch_c<BF16>(e, comp, half, st);
    case PREC_FP16_F32ARITH: return launch_c<F16W>(e, comp ? 3 : 0, half, st);
    case PREC_BF16_F32ARITH: return launch_c<BF16W>(e, comp ? 3 : 0, half, st);
    case PREC_FP16_PAIRS: return comp ? launch_t<F16WP, 3>(e, half, st) : cudaErrorInvalidValue;
    default: return cudaErrorInvalidValue;
    }
}

unsigned elastic_blocks(const int n[2]) { return ((n[0] + 31) / 32) * ((n[1] + 3) / 4); }

}  // namespace wave
