// elastic_strips.cu -- the 2D elastic velocity-stress step (Eq. 2, Appendix A)
// on row strips: one warp per strip of 32 16-byte vectors (8 x points per lane
// for 16-bit storage, 4 for binary32) and a chunk of rows, walking down the
// rows. The arithmetic is that of elastic2d.cu, operation for operation, on
// packed pairs (or per element for binary32 and for binary32 registers):
//   vx += bx * (Dx sxx + Dy sxy)
//   vy += by * (Dx sxy + Dy syy)   [+ s, added to the increment]
//   sxx += (l2m * Dx vx) + (lam * Dy vy)
//   syy += (lam * Dx vx) + (l2m * Dy vy)
//   sxy += mu * (Dx vy + Dy vx)
// x neighbours come from the adjacent lanes by shuffle (from memory with the
// boundary images at the grid's x faces and for the last, ragged vector); the
// y stencils read a 4-row register queue per field, each row loaded once with
// its y image. No shared memory, no barriers. The energy (binary64 terms, as
// in elastic2d.cu) is reduced per work item and then over the items in order.
#include <cuda_runtime.h>

#include "acoustic_common.cuh"
#include "elastic.h"
#include "elastic_common.cuh"
#include "strip_common.cuh"
#include "vec_policy.cuh"
#include "wave_kernels.h"

namespace wave {

namespace {

template <class V>
struct ElStrip {
    using Raw = typename V::Raw;
    using AV = typename V::AV;
    using RS = typename V::RS;
    static constexpr int N = V::N;

    // Row my of field f at x (whole vector) with the y image; zero past the grid.
    static __device__ __forceinline__ Raw row(const void *f, const ElParams &e, int x, int my, bool node,
                                              bool odd, bool odd_free, bool active) {
        int jy;
        const int sg = emap(my, e.n[1], e.bc[2], e.bc[3], node, odd, odd_free, jy);
        if (!active || sg == 0 || jy < 0 || jy >= e.n[1]) return V::zero();
        const Raw r = *reinterpret_cast<const Raw *>(static_cast<const char *>(f) +
                                                     (x + e.sy * (int64_t)jy) * sizeof(RS));
        return sg < 0 ? V::rneg(r) : r;
    }
    // Value of field f at x index mx of row j, with the x image.
    static __device__ __forceinline__ RS xval(const void *f, const ElParams &e, int mx, int j, bool node,
                                              bool odd) {
        int ix;
        // x faces are periodic or rigid (a free surface is a y face)
        const int sg = emap(mx, e.n[0], e.bc[0], e.bc[1], node, odd, false, ix);
        if (sg == 0 || ix < 0 || ix >= e.n[0]) return RS(0);
        const RS v = static_cast<const RS *>(f)[ix + e.sy * (int64_t)j];
        return sg < 0 ? V::rneg_s(v) : v;
    }
    static __device__ __forceinline__ RS shfl(RS v, bool up) {
        uint32_t u;
        if (sizeof(RS) == 2) u = (uint32_t)(*reinterpret_cast<const uint16_t *>(&v));
        else u = *reinterpret_cast<const uint32_t *>(&v);
        u = up ? __shfl_up_sync(0xffffffffu, u, 1) : __shfl_down_sync(0xffffffffu, u, 1);
        RS r;
        if (sizeof(RS) == 2) *reinterpret_cast<uint16_t *>(&r) = (uint16_t)u;
        else *reinterpret_cast<uint32_t *>(&r) = u;
        return r;
    }
    static __device__ __forceinline__ void set_raw(Raw &r, int k, RS s);
    // Own vector of row j with the elements past the grid replaced by their
    // x images (only the right-edge lane has any).
    static __device__ __forceinline__ Raw fix(Raw own, const void *f, const ElParams &e, int x, int j,
                                              int nvalid, bool node, bool odd) {
#pragma unroll
        for (int k = 1; k < N; k++)
            if (k >= nvalid) set_raw(own, k, xval(f, e, x + k, j, node, odd));
        return own;
    }
    // x neighbours x-1, x+N, x+N+1 of a node-type row (lanes, or the x images)
    static __device__ __forceinline__ void nb_node(const Raw &own, const void *f, const ElParams &e, int x, int j,
                                                   bool odd, bool left_edge, bool right_edge, RS &l0, RS &r0,
                                                   RS &r1) {
        const RS sl0 = shfl(V::get(own, N - 1), true);
        const RS sr0 = shfl(V::get(own, 0), false);
        const RS sr1 = shfl(V::get(own, 1), false);
        l0 = left_edge ? xval(f, e, x - 1, j, true, odd) : sl0;
        r0 = right_edge ? xval(f, e, x + N, j, true, odd) : sr0;
        r1 = right_edge ? xval(f, e, x + N + 1, j, true, odd) : sr1;
    }
    // x neighbours x-2, x-1, x+N of a half-type row
    static __device__ __forceinline__ void nb_half(const Raw &own, const void *f, const ElParams &e, int x, int j,
                                                   bool odd, bool left_edge, bool right_edge, RS &l1, RS &l0,
                                                   RS &rr) {
        const RS sl1 = shfl(V::get(own, N - 2), true);
        const RS sl0 = shfl(V::get(own, N - 1), true);
        const RS srr = shfl(V::get(own, 0), false);
        l1 = left_edge ? xval(f, e, x - 2, j, false, odd) : sl1;
        l0 = left_edge ? xval(f, e, x - 1, j, false, odd) : sl0;
        rr = right_edge ? xval(f, e, x + N, j, false, odd) : srr;
    }
    // D_x of a field that sits on the x nodes: reads x-1 .. x+N+1. With PAIRS
    // the taps are RN(V + T) (own_t, ft: the field's compensation).
    template <class P, bool PAIRS>
    static __device__ __forceinline__ AV dx_node(const Raw &own, const Raw &own_t, const void *f, const void *ft,
                                                 const ElParams &e, int x, int j, bool odd, bool left_edge,
                                                 bool right_edge) {
        RS l0, r0, r1;
        nb_node(own, f, e, x, j, odd, left_edge, right_edge, l0, r0, r1);
        AV o = V::ld(own);
        typename V::AS al0 = V::lds(l0), ar0 = V::lds(r0), ar1 = V::lds(r1);
        if constexpr (PAIRS) {
            RS t0, t1, t2;
            nb_node(own_t, ft, e, x, j, odd, left_edge, right_edge, t0, t1, t2);
            o = V::add(o, V::ld(own_t));
            al0 = P::add(al0, V::lds(t0));
            ar0 = P::add(ar0, V::lds(t1));
            ar1 = P::add(ar1, V::lds(t2));
        }
        return vstencil<V>(V::shr1(o, al0), o, V::shl1(o, ar0), V::shl2(o, ar0, ar1));
    }
    // D_x of a field that sits on the x half points: reads x-2 .. x+N.
    template <class P, bool PAIRS>
    static __device__ __forceinline__ AV dx_half(const Raw &own, const Raw &own_t, const void *f, const void *ft,
                                                 const ElParams &e, int x, int j, bool odd, bool left_edge,
                                                 bool right_edge) {
        RS l1, l0, rr;
        nb_half(own, f, e, x, j, odd, left_edge, right_edge, l1, l0, rr);
        AV o = V::ld(own);
        typename V::AS al1 = V::lds(l1), al0 = V::lds(l0), arr = V::lds(rr);
        if constexpr (PAIRS) {
            RS t0, t1, t2;
            nb_half(own_t, ft, e, x, j, odd, left_edge, right_edge, t0, t1, t2);
            o = V::add(o, V::ld(own_t));
            al1 = P::add(al1, V::lds(t0));
            al0 = P::add(al0, V::lds(t1));
            arr = P::add(arr, V::lds(t2));
        }
        return vstencil<V>(V::shr2(o, al1, al0), V::shr1(o, al0), o, V::shl1(o, arr));
    }
    // multipliers of the vector at q (binary32 for the pair precision)
    static __device__ __forceinline__ AV coefv(const void *arr, uint32_t uni, int64_t q) {
        return coef_v<V>(arr, uni, q);
    }
    static __device__ __forceinline__ void store(void *f, int64_t q, const Raw &r, int nvalid) {
        if (nvalid >= N) {
            *reinterpret_cast<Raw *>(static_cast<char *>(f) + q * sizeof(RS)) = r;
        } else {
            RS *s = static_cast<RS *>(f) + q;
#pragma unroll
            for (int k = 0; k < N; k++)
                if (k < nvalid) s[k] = V::get(r, k);
        }
    }
    static __device__ __forceinline__ Raw load(const void *f, int64_t q) {
        return *reinterpret_cast<const Raw *>(static_cast<const char *>(f) + q * sizeof(RS));
    }
};

template <class V>
__device__ __forceinline__ void ElStrip<V>::set_raw(Raw &r, int k, RS s) {
    if constexpr (sizeof(RS) == 2) {
        uint32_t *w = (k >> 1) == 0 ? &r.x : (k >> 1) == 1 ? &r.y : (k >> 1) == 2 ? &r.z : &r.w;
        *w = (k & 1) ? ((*w & 0xFFFFu) | ((uint32_t)s << 16)) : ((*w & 0xFFFF0000u) | s);
    } else {
        if (k == 0) r.x = s; else if (k == 1) r.y = s; else if (k == 2) r.z = s; else r.w = s;
    }
}

struct Item {
    int x0, y0, y1;
};
template <int N>
__device__ __forceinline__ Item item_of(const ElParams &e, int item, int yc) {
    const int nstrips = (e.n[0] + 32 * N - 1) / (32 * N);
    Item it;
    it.x0 = (item % nstrips) * 32 * N;
    it.y0 = (item / nstrips) * yc;
    it.y1 = min(it.y0 + yc, e.n[1]);
    return it;
}

}  // namespace

// Velocity half step on row strips.
template <class P, int COMP>
__global__ void __launch_bounds__(256) el_v_strip(const ElParams e, int nitems, int yc) {
    using V = typename VecOf<P>::T;
    using X = ElStrip<V>;
    using Raw = typename V::Raw;
    using AV = typename V::AV;
    constexpr int N = V::N;
    const int lane = threadIdx.x & 31;
    const int wpb = blockDim.x >> 5;
    const int src_i = e.src_q >= 0 ? (int)(e.src_q % e.sy) : -1;
    const int src_j = e.src_q >= 0 ? (int)(e.src_q / e.sy) : -1;
    const int64_t step = e.step_dev ? *e.step_dev : e.step;
    for (int item = blockIdx.x * wpb + (threadIdx.x >> 5); item < nitems; item += gridDim.x * wpb) {
        const Item it = item_of<N>(e, item, yc);
        const int x = it.x0 + lane * N;
        const bool active = x < e.n[0];
        const int nvalid = active ? min(N, e.n[0] - x) : 0;
        const bool le = active && lane == 0;
        const bool re = active && (lane == 31 || x + N >= e.n[0]);
        // sxy rows j-2 .. j+1 (half points in y; odd at walls and surface); syy rows
        // j-1 .. j+2 (nodes; even at walls, odd at the surface); with the pair
        // policies the same queues of their compensations (taps RN(S + T))
        constexpr bool PAIRS = IsPairs<P>::value;
        Raw a0 = X::row(e.f[F_SXY], e, x, it.y0 - 2, false, true, true, active);
        Raw a1 = X::row(e.f[F_SXY], e, x, it.y0 - 1, false, true, true, active);
        Raw a2 = X::row(e.f[F_SXY], e, x, it.y0, false, true, true, active);
        Raw b0 = X::row(e.f[F_SYY], e, x, it.y0 - 1, true, false, true, active);
        Raw b1 = X::row(e.f[F_SYY], e, x, it.y0, true, false, true, active);
        Raw b2 = X::row(e.f[F_SYY], e, x, it.y0 + 1, true, false, true, active);
        Raw ta0 = V::zero(), ta1 = V::zero(), ta2 = V::zero(), tb0 = V::zero(), tb1 = V::zero(), tb2 = V::zero();
        if (PAIRS) {
            ta0 = X::row(e.t[F_SXY], e, x, it.y0 - 2, false, true, true, active);
            ta1 = X::row(e.t[F_SXY], e, x, it.y0 - 1, false, true, true, active);
            ta2 = X::row(e.t[F_SXY], e, x, it.y0, false, true, true, active);
            tb0 = X::row(e.t[F_SYY], e, x, it.y0 - 1, true, false, true, active);
            tb1 = X::row(e.t[F_SYY], e, x, it.y0, true, false, true, active);
            tb2 = X::row(e.t[F_SYY], e, x, it.y0 + 1, true, false, true, active);
        }
        auto tap = [&](const Raw &v, const Raw &t) -> AV { return PAIRS ? V::add(V::ld(v), V::ld(t)) : V::ld(v); };
        for (int j = it.y0; j < it.y1; j++) {
            const Raw a3 = X::row(e.f[F_SXY], e, x, j + 1, false, true, true, active);
            const Raw b3 = X::row(e.f[F_SYY], e, x, j + 2, true, false, true, active);
            const Raw ta3 = PAIRS ? X::row(e.t[F_SXY], e, x, j + 1, false, true, true, active) : V::zero();
            const Raw tb3 = PAIRS ? X::row(e.t[F_SYY], e, x, j + 2, true, false, true, active) : V::zero();
            const int64_t q = x + e.sy * (int64_t)j;
            Raw sxx = V::zero(), vx = V::zero(), vy = V::zero(), tx = V::zero(), ty = V::zero(), tsxx = V::zero();
            if (active) {
                if (PAIRS) tsxx = X::load(e.t[F_SXX], q);
                sxx = X::load(e.f[F_SXX], q);
                vx = X::load(e.f[F_VX], q);
                vy = X::load(e.f[F_VY], q);
                if (COMP) {
                    tx = X::load(e.t[F_VX], q);
                    ty = X::load(e.t[F_VY], q);
                }
            }
            Raw sxx_f = sxx, sxy_f = a2, tsxx_f = tsxx, tsxy_f = ta2;
            if (re) {
                sxx_f = X::fix(sxx, e.f[F_SXX], e, x, j, nvalid, true, false);
                sxy_f = X::fix(a2, e.f[F_SXY], e, x, j, nvalid, false, true);
                if (PAIRS) {
                    tsxx_f = X::fix(tsxx, e.t[F_SXX], e, x, j, nvalid, true, false);
                    tsxy_f = X::fix(ta2, e.t[F_SXY], e, x, j, nvalid, false, true);
                }
            }
            const AV dxsxx =
                X::template dx_node<P, PAIRS>(sxx_f, tsxx_f, e.f[F_SXX], e.t[F_SXX], e, x, j, false, le, re);
            const AV dxsxy =
                X::template dx_half<P, PAIRS>(sxy_f, tsxy_f, e.f[F_SXY], e.t[F_SXY], e, x, j, true, le, re);
            if (active) {
                // vx: Dx sxx + Dy sxy
                AV R = V::add(dxsxx, vstencil<V>(tap(a0, ta0), tap(a1, ta1), tap(a2, ta2), tap(a3, ta3)));
                V::template update<COMP>(vx, tx, V::mul(X::coefv(e.c[C_BX], e.c_uni[C_BX], q), R));
                // vy: Dx sxy + Dy syy [+ s]
                R = V::add(dxsxy, vstencil<V>(tap(b0, tb0), tap(b1, tb1), tap(b2, tb2), tap(b3, tb3)));
                AV inc = V::mul(X::coefv(e.c[C_BY], e.c_uni[C_BY], q), R);
                if (j == src_j && src_i >= x && src_i < x + N && step < e.src_nt) {
                    const typename V::AS sv = static_cast<const typename V::AS *>(e.src)[step];
#pragma unroll
                    for (int k = 0; k < N; k++)
                        if (k == src_i - x) V::set(inc, k, P::add(V::aget(inc, k), sv));
                }
                V::template update<COMP>(vy, ty, inc);
                X::store(e.f[F_VX], q, vx, nvalid);
                X::store(e.f[F_VY], q, vy, nvalid);
                if (COMP) {
                    X::store(e.t[F_VX], q, tx, nvalid);
                    X::store(e.t[F_VY], q, ty, nvalid);
                }
            }
            a0 = a1; a1 = a2; a2 = a3;
            b0 = b1; b1 = b2; b2 = b3;
            ta0 = ta1; ta1 = ta2; ta2 = ta3;
            tb0 = tb1; tb1 = tb2; tb2 = tb3;
        }
    }
}

// Stress half step on row strips, with the item's energy terms.
template <class P, int COMP, bool ENERGY>
__global__ void __launch_bounds__(256) el_s_strip(const ElParams e, int nitems, int yc, double *item_part) {
    // the velocity launch of this step has read the step index: advance it
    if (e.step_dev && blockIdx.x == 0 && threadIdx.x == 0) ++*e.step_dev;
    using V = typename VecOf<P>::T;
    using X = ElStrip<V>;
    using Raw = typename V::Raw;
    using AV = typename V::AV;
    using RS = typename V::RS;
    constexpr int N = V::N;
    const int lane = threadIdx.x & 31;
    const int wpb = blockDim.x >> 5;
    for (int item = blockIdx.x * wpb + (threadIdx.x >> 5); item < nitems; item += gridDim.x * wpb) {
        const Item it = item_of<N>(e, item, yc);
        const int x = it.x0 + lane * N;
        const bool active = x < e.n[0];
        const int nvalid = active ? min(N, e.n[0] - x) : 0;
        const bool le = active && lane == 0;
        const bool re = active && (lane == 31 || x + N >= e.n[0]);
        // vy rows j-2 .. j+1 (half points in y; odd at walls, even at the surface); vx
        // rows j-1 .. j+2 (nodes, even); with the pair policies the same queues
        // of their compensations (taps RN(V + T))
        constexpr bool PAIRS = IsPairs<P>::value;
        Raw c0 = X::row(e.f[F_VY], e, x, it.y0 - 2, false, true, false, active);
        Raw c1 = X::row(e.f[F_VY], e, x, it.y0 - 1, false, true, false, active);
        Raw c2 = X::row(e.f[F_VY], e, x, it.y0, false, true, false, active);
        Raw d0 = X::row(e.f[F_VX], e, x, it.y0 - 1, true, false, false, active);
        Raw d1 = X::row(e.f[F_VX], e, x, it.y0, true, false, false, active);
        Raw d2 = X::row(e.f[F_VX], e, x, it.y0 + 1, true, false, false, active);
        Raw tc0 = V::zero(), tc1 = V::zero(), tc2 = V::zero(), td0 = V::zero(), td1 = V::zero(), td2 = V::zero();
        if (PAIRS) {
            tc0 = X::row(e.t[F_VY], e, x, it.y0 - 2, false, true, false, active);
            tc1 = X::row(e.t[F_VY], e, x, it.y0 - 1, false, true, false, active);
            tc2 = X::row(e.t[F_VY], e, x, it.y0, false, true, false, active);
            td0 = X::row(e.t[F_VX], e, x, it.y0 - 1, true, false, false, active);
            td1 = X::row(e.t[F_VX], e, x, it.y0, true, false, false, active);
            td2 = X::row(e.t[F_VX], e, x, it.y0 + 1, true, false, false, active);
        }
        auto tap = [&](const Raw &v, const Raw &t) -> AV { return PAIRS ? V::add(V::ld(v), V::ld(t)) : V::ld(v); };
        double en = 0.0;
        for (int j = it.y0; j < it.y1; j++) {
            const Raw c3 = X::row(e.f[F_VY], e, x, j + 1, false, true, false, active);
            const Raw d3 = X::row(e.f[F_VX], e, x, j + 2, true, false, false, active);
            const Raw tc3 = PAIRS ? X::row(e.t[F_VY], e, x, j + 1, false, true, false, active) : V::zero();
            const Raw td3 = PAIRS ? X::row(e.t[F_VX], e, x, j + 2, true, false, false, active) : V::zero();
            const int64_t q = x + e.sy * (int64_t)j;
            Raw sxx = V::zero(), syy = V::zero(), sxy = V::zero();
            Raw txx = V::zero(), tyy = V::zero(), txy = V::zero();
            if (active) {
                sxx = X::load(e.f[F_SXX], q);
                syy = X::load(e.f[F_SYY], q);
                sxy = X::load(e.f[F_SXY], q);
                if (COMP) {
                    txx = X::load(e.t[F_SXX], q);
                    tyy = X::load(e.t[F_SYY], q);
                    txy = X::load(e.t[F_SXY], q);
                }
            }
            Raw vx_f = d1, vy_f = c2, tvx_f = td1, tvy_f = tc2;
            if (re) {
                vx_f = X::fix(d1, e.f[F_VX], e, x, j, nvalid, false, true);
                vy_f = X::fix(c2, e.f[F_VY], e, x, j, nvalid, true, false);
                if (PAIRS) {
                    tvx_f = X::fix(td1, e.t[F_VX], e, x, j, nvalid, false, true);
                    tvy_f = X::fix(tc2, e.t[F_VY], e, x, j, nvalid, true, false);
                }
            }
            const AV dxvx = X::template dx_half<P, PAIRS>(vx_f, tvx_f, e.f[F_VX], e.t[F_VX], e, x, j, true, le, re);
            const AV dxvy = X::template dx_node<P, PAIRS>(vy_f, tvy_f, e.f[F_VY], e.t[F_VY], e, x, j, false, le, re);
            if (active) {
                const AV dyvy = vstencil<V>(tap(c0, tc0), tap(c1, tc1), tap(c2, tc2), tap(c3, tc3));
                const AV l2m = X::coefv(e.c[C_L2M], e.c_uni[C_L2M], q);
                const AV lam = X::coefv(e.c[C_LAM], e.c_uni[C_LAM], q);
                const Raw sxx0 = sxx, syy0 = syy, sxy0 = sxy;
                V::template update<COMP>(sxx, txx, V::add(V::mul(l2m, dxvx), V::mul(lam, dyvy)));
                V::template update<COMP>(syy, tyy, V::add(V::mul(lam, dxvx), V::mul(l2m, dyvy)));
                const AV R = V::add(dxvy, vstencil<V>(tap(d0, td0), tap(d1, td1), tap(d2, td2), tap(d3, td3)));
                V::template update<COMP>(sxy, txy, V::mul(X::coefv(e.c[C_MU], e.c_uni[C_MU], q), R));
                X::store(e.f[F_SXX], q, sxx, nvalid);
                X::store(e.f[F_SYY], q, syy, nvalid);
                X::store(e.f[F_SXY], q, sxy, nvalid);
                if (COMP) {
                    X::store(e.t[F_SXX], q, txx, nvalid);
                    X::store(e.t[F_SYY], q, tyy, nvalid);
                    X::store(e.t[F_SXY], q, txy, nvalid);
                }
                if (ENERGY && PAIRS) {
                    // binary64 terms with the binary32 multipliers (CoefOf)
                    const double wrow = (e.bc[2] == EBC_FREE && j == 0) ? 0.5 : 1.0;
#pragma unroll
                    for (int k = 0; k < N; k++) {
                        if (k < nvalid) {
                            const double bx = coef_f32<P>(e.c[0], e.c_uni[0], q + k);
                            const double by = coef_f32<P>(e.c[1], e.c_uni[1], q + k);
                            const double L = coef_f32<P>(e.c[2], e.c_uni[2], q + k);
                            const double M = coef_f32<P>(e.c[3], e.c_uni[3], q + k);
                            const double mu = coef_f32<P>(e.c[4], e.c_uni[4], q + k);
                            const double vxv = V::f32(d1, k), vyv = V::f32(c2, k);
                            const double a0 = V::f32(sxx0, k), a1 = V::f32(sxx, k);
                            const double b0 = V::f32(syy0, k), b1 = V::f32(syy, k);
                            double t = wrow * (vxv * vxv / bx) + vyv * vyv / by;
                            t += wrow * ((L * (a0 * a1 + b0 * b1) - M * (a0 * b1 + b0 * a1)) / (L * L - M * M));
                            if (mu > 0.0) t += (double)V::f32(sxy0, k) * (double)V::f32(sxy, k) / mu;
                            en += t;
                        }
                    }
                } else if (ENERGY) {
                    // binary64 terms, as in the one-thread-per-point kernel
                    const Raw cb[5] = {e.c[0] ? X::load(e.c[0], q) : V::zero(), e.c[1] ? X::load(e.c[1], q) : V::zero(),
                                       e.c[2] ? X::load(e.c[2], q) : V::zero(), e.c[3] ? X::load(e.c[3], q) : V::zero(),
                                       e.c[4] ? X::load(e.c[4], q) : V::zero()};
                    float cu[5];
#pragma unroll
                    for (int w = 0; w < 5; w++) cu[w] = coef_f32<P>(nullptr, e.c_uni[w], 0);
                    // weight 1/2 for vx and the normal stresses on a free surface row
                    const double wrow = (e.bc[2] == EBC_FREE && j == 0) ? 0.5 : 1.0;
#pragma unroll
                    for (int k = 0; k < N; k++) {
                        if (k < nvalid) {
                            const double bx = e.c[0] ? V::f32(cb[0], k) : cu[0];
                            const double by = e.c[1] ? V::f32(cb[1], k) : cu[1];
                            const double L = e.c[2] ? V::f32(cb[2], k) : cu[2];
                            const double M = e.c[3] ? V::f32(cb[3], k) : cu[3];
                            const double mu = e.c[4] ? V::f32(cb[4], k) : cu[4];
                            const double vxv = V::f32(d1, k), vyv = V::f32(c2, k);
                            const double a0 = V::f32(sxx0, k), a1 = V::f32(sxx, k);
                            const double b0 = V::f32(syy0, k), b1 = V::f32(syy, k);
                            double t = wrow * (vxv * vxv / bx) + vyv * vyv / by;
                            t += wrow * ((L * (a0 * a1 + b0 * b1) - M * (a0 * b1 + b0 * a1)) / (L * L - M * M));
                            if (mu > 0.0) t += (double)V::f32(sxy0, k) * (double)V::f32(sxy, k) / mu;
                            en += t;
                        }
                    }
                }
            }
            c0 = c1; c1 = c2; c2 = c3;
            d0 = d1; d1 = d2; d2 = d3;
            tc0 = tc1; tc1 = tc2; tc2 = tc3;
            td0 = td1; td1 = td2; td2 = td3;
        }
        if (ENERGY) {
            for (int off = 16; off > 0; off >>= 1) en += __shfl_down_sync(0xffffffffu, en, off);
            if (lane == 0) item_part[item] = en;
        }
    }
}

// Sum of the item partials in item order, times the physical factor.
__global__ void el_strip_energy(const double *part, int nitems, double *e_out, double factor) {
    __shared__ double ws[8];
    double s = 0.0;
    for (int i = threadIdx.x; i < nitems; i += blockDim.x) s += part[i];
    for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) t += ws[w];
        *e_out = t * factor;
    }
}

template <class P, int COMP>
static cudaError_t launch_t(const ElParams &e, int half, const ElStripLaunch &L, cudaStream_t st) {
    const int threads = 32 * L.wpb;
    if (half == 0) {
        el_v_strip<P, COMP><<<L.grid, threads, 0, st>>>(e, L.nitems, L.yc);
    } else if (e.energy) {
        el_s_strip<P, COMP, true><<<L.grid, threads, 0, st>>>(e, L.nitems, L.yc, L.item_part);
        el_strip_energy<<<1, 256, 0, st>>>(L.item_part, L.nitems, e.e_out, e.e_factor);
    } else {
        el_s_strip<P, COMP, false><<<L.grid, threads, 0, st>>>(e, L.nitems, L.yc, L.item_part);
    }
    return cudaGetLastError();
}

template <class P>
static cudaError_t launch_c(const ElParams &e, int comp, int half, const ElStripLaunch &L, cudaStream_t st) {
    switch (comp) {
    case 0: return launch_t<P, 0>(e, half, L, st);
    case 3: return launch_t<P, 3>(e, half, L, st);
    default: return launch_t<P, 6>(e, half, L, st);
    }
}

int elastic_strip_items(int prec, int nx, int ny, int yc) {
    const int tx = 32 * (prec == PREC_FP32 ? 4 : 8);
    return ((nx + tx - 1) / tx) * ((ny + yc - 1) / yc);
}

cudaError_t elastic_strip_half_step(const ElParams &e, int prec, int comp, int half, const ElStripLaunch &L,
                                    cudaStream_t st) {
    if (L.wpb < 1 || L.wpb > 8 || L.yc < 1) return cudaErrorInvalidValue;
    switch (prec) {
    case PREC_FP32: return launch_c<F32>(e, comp, half, L, st);
    case PREC_FP16: return launch_c<F16>(e, comp, half, L, st);
    case PREC_BF16: return launch_c<BF16>(e, comp, half, L, st);
    case PREC_FP16_F32ARITH: return launch_c<F16W>(e, comp ? 3 : 0, half, L, st);
    case PREC_BF16_F32ARITH: return launch_c<BF16W>(e, comp ? 3 : 0, half, L, st);
    case PREC_FP16_PAIRS: return comp ? launch_t<F16WP, 3>(e, half, L, st) : cudaErrorInvalidValue;
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace wave
