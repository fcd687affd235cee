// acoustic_point.cuh -- the acoustic leapfrog at one grid point, shared by
// the one-thread-per-point kernels and the batched multi-shot kernels, so that
// both produce the same bits.
#pragma once
#include "acoustic_common.cuh"

namespace wave {

template <class P>
__device__ __forceinline__ typename P::A read_signed(const typename P::S *f, int64_t q, int sign) {
    if (sign == 0) return P::zero();
    typename P::A v = P::ld(f[q]);
    return sign > 0 ? v : P::neg(v);
}

// A stencil tap: the stored value, or for the pair policies RN(V + T) (the
// image's sign applied to the sum, which negation commutes with).
template <class P>
__device__ __forceinline__ typename P::A read_tap(const typename P::S *f, const typename P::S *t, int64_t q,
                                                  int sign) {
    if (!IsPairs<P>::value) return read_signed<P>(f, q, sign);
    if (sign == 0) return P::zero();
    const typename P::A v = P::add(P::ld(f[q]), P::ld(t[q]));
    return sign > 0 ? v : P::neg(v);
}

// Velocity half step at point (i, j, k): for each axis c, v_c at m + 1/2
// reads p at nodes m-1, m, m+1, m+2 along c.
template <class P, int COMP, int NDIM>
__device__ __forceinline__ void kv_point(const AcParams &prm, int i, int j, int k) {
    using S = typename P::S;
    using A = typename P::A;
    const int idx[3] = {i, j, k};
    const int64_t str[3] = {1, prm.sy, prm.sz};
    const int64_t q = i + prm.sy * j + prm.sz * k;
    const S *p = static_cast<const S *>(prm.p);
    const S *tp = static_cast<const S *>(prm.tp);
#pragma unroll
    for (int c = 0; c < NDIM; c++) {
        const int m = idx[c];
        const int64_t base = q - str[c] * m;
        A f[4];
#pragma unroll
        for (int t = 0; t < 4; t++) {
            int mm;
            int sg = img_node(m - 1 + t, prm.n[c], prm.bc[c], mm);
            f[t] = read_tap<P>(p, tp, base + str[c] * mm, sg);
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

// Pressure half step at point (i, j, k): R = sum over axes of D_c(v_c) (left
// to right) [+ source], p += b * R. Returns the point's energy terms
// p^n p^{n+1} / b + sum v_c^2 / a_c when `energy` is set, else 0.
template <class P, int COMP, int NDIM>
__device__ __forceinline__ double kp_point(const AcParams &prm, int i, int j, int k, int64_t step,
                                           bool energy) {
    using S = typename P::S;
    using A = typename P::A;
    const int idx[3] = {i, j, k};
    const int64_t str[3] = {1, prm.sy, prm.sz};
    const int64_t q = i + prm.sy * j + prm.sz * k;
    A R = P::zero();
#pragma unroll
    for (int c = 0; c < NDIM; c++) {
        const int m = idx[c];
        const int64_t base = q - str[c] * m;
        const S *v = static_cast<const S *>(prm.v[c]);
        const S *tv = static_cast<const S *>(prm.tv[c]);
        A f[4];
#pragma unroll
        for (int t = 0; t < 4; t++) {
            int mm;
            img_half(m - 2 + t, prm.n[c], prm.bc[c], mm);
            f[t] = read_tap<P>(v, tv, base + str[c] * mm, 1);
        }
        A D = stencil<P>(f[0], f[1], f[2], f[3]);
        R = (c == 0) ? D : P::add(R, D);
    }
    if (q == prm.src_q && step < prm.src_nt) R = P::add(R, static_cast<const A *>(prm.src)[step]);
    A inc = P::mul(coef<P>(prm.b, prm.b_uni, q), R);
    S *p = static_cast<S *>(prm.p);
    S *tp = static_cast<S *>(prm.tp);
    const S p_old = p[q];
    S V = p_old;
    S T = COMP ? tp[q] : S(0);
    update<P, COMP>(V, T, inc);
    p[q] = V;
    if (COMP) tp[q] = T;
    double e = 0.0;
    if (energy) {
        e = (double)e_term(P::to_f32(p_old), P::to_f32(V), coef_f32<P>(prm.b, prm.b_uni, q));
#pragma unroll
        for (int c = 0; c < NDIM; c++) {
            float vc = P::to_f32(static_cast<const S *>(prm.v[c])[q]);
            e += (double)e_term(vc, vc, coef_f32<P>(prm.a[c], prm.a_uni[c], q));
        }
    }
    return e;
}

}  // namespace wave
