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
//
// Two item kinds: tiles of points with one thread per point (the arithmetic of
// acoustic_point.cuh), and row strips with one warp per strip, 16-byte vectors
// of 8 (binary16 / bfloat16) or 4 (binary32) x points per lane, x neighbours
// by warp shuffle and a register queue down the rows for the y stencil, so
// each array is read about once. Both give the same bits.
#include <cuda_runtime.h>

#include <algorithm>

#include "acoustic_point.cuh"
#include "batch.h"
#include "strip_common.cuh"
#include "vec_policy.cuh"
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

// The velocity launch of a step advances every shot's step counter first (block
// 0): the counters hold the previous step's index between steps, and the
// pressure launch, which reads them for the source, runs after this launch
// has completed.
__device__ __forceinline__ void advance_counters(BatchShot *shots, int nshots) {
    if (blockIdx.x == 0)
        for (int s = threadIdx.x; s < nshots; s += blockDim.x) shots[s].step++;
}

template <class P, int COMP, int HALF>
__global__ void __launch_bounds__(256) batch_half_step(BatchShot *shots, const int *item0, int nshots,
                                                      int nitems, int bx, int by, int energy,
                                                      double *item_part) {
    if (HALF == 0) advance_counters(shots, nshots);
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

// ------------------------------------------------------------------------
// Row-strip kernels (one warp per item)
// ------------------------------------------------------------------------

// Row my of a field at x (a whole vector), with the y boundary image; zero
// for lanes past the grid. node_y: the field sits on nodes along y (odd
// image for the p = 0 walls) or on half points (even image).
template <class V>
__device__ __forceinline__ typename V::Raw row_vec(const void *f, const AcParams &prm, int x, int my,
                                                   bool node_y, bool active) {
    int jy;
    const int sg = node_y ? img_node(my, prm.n[1], prm.bc[1], jy) : img_half(my, prm.n[1], prm.bc[1], jy);
    if (!active || sg == 0 || jy < 0 || jy >= prm.n[1]) return V::zero();
    const typename V::Raw r = *reinterpret_cast<const typename V::Raw *>(
        static_cast<const char *>(f) + (x + prm.sy * (int64_t)jy) * sizeof(typename V::RS));
    return sg < 0 ? V::rneg(r) : r;
}

// One value of row j at x index mx, with the x boundary image.
template <class V>
__device__ __forceinline__ typename V::RS x_val(const void *f, const AcParams &prm, int mx, int j, bool node_x) {
    int ix;
    const int sg = node_x ? img_node(mx, prm.n[0], prm.bc[0], ix) : img_half(mx, prm.n[0], prm.bc[0], ix);
    if (sg == 0 || ix < 0 || ix >= prm.n[0]) return typename V::RS(0);
    const typename V::RS v = static_cast<const typename V::RS *>(f)[ix + prm.sy * (int64_t)j];
    return sg < 0 ? V::rneg_s(v) : v;
}

// Work item -> (shot, strip origin x0, first row y0, end row y1).
struct StripItem {
    int s, x0, y0, y1;
};
template <int N>
__device__ __forceinline__ StripItem strip_of(const int *s_item0, int nshots, int item, const BatchShot *shots,
                                              int yc) {
    StripItem it;
    it.s = shot_of(s_item0, nshots, item);
    const int nx = shots[it.s].prm.n[0], ny = shots[it.s].prm.n[1];
    const int nstrips = (nx + 32 * N - 1) / (32 * N);
    const int local = item - s_item0[it.s];
    it.x0 = (local % nstrips) * (32 * N);
    it.y0 = (local / nstrips) * yc;
    it.y1 = min(it.y0 + yc, ny);
    return it;
}

// Velocity half step of one strip: v_x += a_x Dx(p), v_y += a_y Dy(p), row by row.
// (Both strip kernels are bounded to 80 registers, three blocks of 256 threads
// per SM: the strips wait on global loads, and 24 warps per SM instead of 16
// hide more of it: 64 shots 136 -> 152 Gpt/s, 8192^2 171 -> 183, at a few
// bytes of spills.)
template <class P, int COMP>
__device__ __forceinline__ void kv_strip_item(const AcParams &prm, const StripItem &it, int lane) {
    using V = typename VecOf<P>::T;
    using Raw = typename V::Raw;
    using AV = typename V::AV;
    using RS = typename V::RS;
    constexpr int N = V::N;
    {
        const int nx = prm.n[0];
        const int x = it.x0 + lane * N;
        const bool active = x < nx;
        const int nvalid = active ? min(N, nx - x) : 0;
        const bool left_edge = active && lane == 0;
        const bool right_edge = active && (lane == 31 || x + N >= nx);
        // row queue of the own p vector: rows j-1, j, j+1 (j+2 loaded in the
        // loop); with the pair policies the same queue of t_p (the taps read
        // RN(p + t_p))
        constexpr bool PAIRS = IsPairs<P>::value;
        Raw q0 = row_vec<V>(prm.p, prm, x, it.y0 - 1, true, active);
        Raw q1 = row_vec<V>(prm.p, prm, x, it.y0, true, active);
        Raw q2 = row_vec<V>(prm.p, prm, x, it.y0 + 1, true, active);
        Raw u0 = V::zero(), u1 = V::zero(), u2 = V::zero();
        if (PAIRS) {
            u0 = row_vec<V>(prm.tp, prm, x, it.y0 - 1, true, active);
            u1 = row_vec<V>(prm.tp, prm, x, it.y0, true, active);
            u2 = row_vec<V>(prm.tp, prm, x, it.y0 + 1, true, active);
        }
        for (int j = it.y0; j < it.y1; j++) {
            const Raw q3 = row_vec<V>(prm.p, prm, x, j + 2, true, active);
            const Raw u3 = PAIRS ? row_vec<V>(prm.tp, prm, x, j + 2, true, active) : V::zero();
            const int64_t q = x + prm.sy * (int64_t)j;
            Raw vx = V::zero(), vy = V::zero(), tx = V::zero(), ty = V::zero();
            if (active) {
                vx = at<V>(prm.v[0], q);
                vy = at<V>(prm.v[1], q);
                if (COMP) {
                    tx = at<V>(prm.tv[0], q);
                    ty = at<V>(prm.tv[1], q);
                }
            }
            // x neighbours p[x-1], p[x+N], p[x+N+1] of a row of field f (p, or
            // t_p for the pairs); at strip and grid edges from memory with the
            // x image, and the own vector's elements past the grid replaced by
            // their images
            auto xnb = [&](const void *f, Raw &own, RS &l0, RS &r0, RS &r1) {
                l0 = r0 = r1 = RS(0);
                if (left_edge) l0 = x_val<V>(f, prm, x - 1, j, true);
                if (right_edge) {
                    r0 = x_val<V>(f, prm, x + N, j, true);
                    r1 = x_val<V>(f, prm, x + N + 1, j, true);
#pragma unroll
                    for (int e = 1; e < N; e++)
                        if (e >= nvalid) raw_set<RS, Raw>(own, e, x_val<V>(f, prm, x + e, j, true));
                }
                // (from the fixed-up vector: the lane left of a partial vector
                // reads its element 1, which may lie past the grid)
                const RS sl0 = shfl_rs(V::get(own, N - 1), 1, true);
                const RS sr0 = shfl_rs(V::get(own, 0), 1, false);
                const RS sr1 = shfl_rs(V::get(own, 1), 1, false);
                if (!left_edge) l0 = sl0;
                if (!right_edge) {
                    r0 = sr0;
                    r1 = sr1;
                }
            };
            Raw own = q1, ownt = u1;
            RS l0, r0, r1, l0t = RS(0), r0t = RS(0), r1t = RS(0);
            xnb(prm.p, own, l0, r0, r1);
            if (PAIRS) xnb(prm.tp, ownt, l0t, r0t, r1t);
            if (active) {
                // taps: the stored values, or RN(V + T) for the pairs
                auto tap = [&](const Raw &v, const Raw &t) -> AV { return PAIRS ? V::add(V::ld(v), V::ld(t)) : V::ld(v); };
                auto tap_s = [&](RS v, RS t) -> typename V::AS {
                    return PAIRS ? P::add(V::lds(v), V::lds(t)) : V::lds(v);
                };
                const AV o = tap(own, ownt);
                const typename V::AS a_l0 = tap_s(l0, l0t), a_r0 = tap_s(r0, r0t), a_r1 = tap_s(r1, r1t);
                // v_x at i + 1/2: p[i-1], p[i], p[i+1], p[i+2]
                const AV Dx = vstencil<V>(V::shr1(o, a_l0), o, V::shl1(o, a_r0), V::shl2(o, a_r0, a_r1));
                // v_y at j + 1/2: rows j-1, j, j+1, j+2
                const AV Dy = vstencil<V>(tap(q0, u0), tap(q1, u1), tap(q2, u2), tap(q3, u3));
                V::template update<COMP>(vx, tx, V::mul(coef_v<V>(prm.a[0], prm.a_uni[0], q), Dx));
                V::template update<COMP>(vy, ty, V::mul(coef_v<V>(prm.a[1], prm.a_uni[1], q), Dy));
                store_vec<V>(prm.v[0], q, vx, nvalid);
                store_vec<V>(prm.v[1], q, vy, nvalid);
                if (COMP) {
                    store_vec<V>(prm.tv[0], q, tx, nvalid);
                    store_vec<V>(prm.tv[1], q, ty, nvalid);
                }
            }
            q0 = q1;
            q1 = q2;
            q2 = q3;
            u0 = u1;
            u1 = u2;
            u2 = u3;
        }
    }
}

template <class P, int COMP>
__global__ void __launch_bounds__(256, 3) batch_kv_strip(BatchShot *shots, const int *item0,
                                                      int nshots, int nitems, int yc) {
    advance_counters(shots, nshots);
    constexpr int N = VecOf<P>::T::N;
    __shared__ int s_item0[kMaxShots + 1];
    for (int t = threadIdx.x; t <= nshots; t += blockDim.x) s_item0[t] = item0[t];
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int wpb = blockDim.x >> 5;
    for (int item = blockIdx.x * wpb + (threadIdx.x >> 5); item < nitems; item += gridDim.x * wpb) {
        const StripItem it = strip_of<N>(s_item0, nshots, item, shots, yc);
        const AcParams prm = shots[it.s].prm;
        kv_strip_item<P, COMP>(prm, it, lane);
    }
}

// Pressure half step of one strip: p += b (Dx v_x + Dy v_y [+ s]), with the
// item's energy terms p^n p^{n+1} / b + v_x^2 / a_x + v_y^2 / a_y.
template <class P, int COMP, bool ENERGY>
__device__ __forceinline__ double kp_strip_item(const AcParams &prm, int64_t step, const StripItem &it, int lane) {
    using V = typename VecOf<P>::T;
    using Raw = typename V::Raw;
    using AV = typename V::AV;
    using RS = typename V::RS;
    constexpr int N = V::N;
    {
        const int nx = prm.n[0];
        const int x = it.x0 + lane * N;
        const bool active = x < nx;
        const int nvalid = active ? min(N, nx - x) : 0;
        const bool left_edge = active && lane == 0;
        const bool right_edge = active && (lane == 31 || x + N >= nx);
        // row queue of the own v_y vector: rows j-2, j-1, j (j+1 loaded in
        // the loop); with the pair policies the same queue of t_vy (the taps
        // read RN(v + t_v))
        constexpr bool PAIRS = IsPairs<P>::value;
        Raw r0 = row_vec<V>(prm.v[1], prm, x, it.y0 - 2, false, active);
        Raw r1 = row_vec<V>(prm.v[1], prm, x, it.y0 - 1, false, active);
        Raw r2 = row_vec<V>(prm.v[1], prm, x, it.y0, false, active);
        Raw u0 = V::zero(), u1 = V::zero(), u2 = V::zero();
        if (PAIRS) {
            u0 = row_vec<V>(prm.tv[1], prm, x, it.y0 - 2, false, active);
            u1 = row_vec<V>(prm.tv[1], prm, x, it.y0 - 1, false, active);
            u2 = row_vec<V>(prm.tv[1], prm, x, it.y0, false, active);
        }
        double e_acc = 0.0;
        for (int j = it.y0; j < it.y1; j++) {
            const Raw r3 = row_vec<V>(prm.v[1], prm, x, j + 1, false, active);
            const Raw u3 = PAIRS ? row_vec<V>(prm.tv[1], prm, x, j + 1, false, active) : V::zero();
            const int64_t q = x + prm.sy * (int64_t)j;
            Raw vx = V::zero(), pv = V::zero(), tv = V::zero(), tx = V::zero();
            if (active) {
                vx = at<V>(prm.v[0], q);
                pv = at<V>(prm.p, q);
                if (COMP) tv = at<V>(prm.tp, q);
                if (PAIRS) tx = at<V>(prm.tv[0], q);
            }
            // x neighbours v_x[x-2], v_x[x-1], v_x[x+N] (half-point images) of
            // a row of field f (v_x, or t_vx for the pairs)
            auto xnb = [&](const void *f, const Raw &row, Raw &own, RS &l1, RS &l0, RS &rr) {
                own = row;
                l1 = l0 = rr = RS(0);
                if (left_edge) {
                    l1 = x_val<V>(f, prm, x - 2, j, false);
                    l0 = x_val<V>(f, prm, x - 1, j, false);
                }
                if (right_edge) {
                    rr = x_val<V>(f, prm, x + N, j, false);
#pragma unroll
                    for (int e = 1; e < N; e++)
                        if (e >= nvalid) raw_set<RS, Raw>(own, e, x_val<V>(f, prm, x + e, j, false));
                }
                const RS sl1 = shfl_rs(V::get(row, N - 2), 1, true);
                const RS sl0 = shfl_rs(V::get(row, N - 1), 1, true);
                const RS srr = shfl_rs(V::get(row, 0), 1, false);
                if (!left_edge) {
                    l1 = sl1;
                    l0 = sl0;
                }
                if (!right_edge) rr = srr;
            };
            Raw own, ownt = V::zero();
            RS l1, l0, rr, l1t = RS(0), l0t = RS(0), rrt = RS(0);
            xnb(prm.v[0], vx, own, l1, l0, rr);
            if (PAIRS) xnb(prm.tv[0], tx, ownt, l1t, l0t, rrt);
            if (active) {
                // taps: the stored values, or RN(V + T) for the pairs
                auto tap = [&](const Raw &v, const Raw &t) -> AV { return PAIRS ? V::add(V::ld(v), V::ld(t)) : V::ld(v); };
                auto tap_s = [&](RS v, RS t) -> typename V::AS {
                    return PAIRS ? P::add(V::lds(v), V::lds(t)) : V::lds(v);
                };
                const AV o = tap(own, ownt);
                const typename V::AS a_l1 = tap_s(l1, l1t), a_l0 = tap_s(l0, l0t), a_rr = tap_s(rr, rrt);
                // node i reads v_x at i-2, i-1, i, i+1 (+1/2)
                AV R = vstencil<V>(V::shr2(o, a_l1, a_l0), V::shr1(o, a_l0), o, V::shl1(o, a_rr));
                R = V::add(R, vstencil<V>(tap(r0, u0), tap(r1, u1), tap(r2, u2), tap(r3, u3)));
                if (j == prm.src_j && prm.src_i >= x && prm.src_i < x + N && step < prm.src_nt) {
                    const typename V::AS s_ = static_cast<const typename V::AS *>(prm.src)[step];
#pragma unroll
                    for (int e = 0; e < N; e++)
                        if (e == prm.src_i - x) V::set(R, e, P::add(V::aget(R, e), s_));
                }
                const Raw pold = pv;
                V::template update<COMP>(pv, tv, V::mul(coef_v<V>(prm.b, prm.b_uni, q), R));
                store_vec<V>(prm.p, q, pv, nvalid);
                if (COMP) store_vec<V>(prm.tp, q, tv, nvalid);
                if constexpr (ENERGY && PAIRS) {
                    // (binary32 multipliers, CoefOf)
#pragma unroll
                    for (int e = 0; e < N; e++) {
                        if (e >= nvalid) break;
                        const float fx = V::f32(vx, e), fy = V::f32(r2, e);
                        e_acc += (double)e_term(V::f32(pold, e), V::f32(pv, e), coef_f32<P>(prm.b, prm.b_uni, q + e));
                        e_acc += (double)e_term(fx, fx, coef_f32<P>(prm.a[0], prm.a_uni[0], q + e));
                        e_acc += (double)e_term(fy, fy, coef_f32<P>(prm.a[1], prm.a_uni[1], q + e));
                    }
                } else if constexpr (ENERGY) {
                    RS bs, as0, as1;
                    from_bits(prm.b_uni, bs);
                    from_bits(prm.a_uni[0], as0);
                    from_bits(prm.a_uni[1], as1);
                    const Raw bv = prm.b ? at<V>(const_cast<void *>(prm.b), q) : V::zero();
                    const Raw av0 = prm.a[0] ? at<V>(const_cast<void *>(prm.a[0]), q) : V::zero();
                    const Raw av1 = prm.a[1] ? at<V>(const_cast<void *>(prm.a[1]), q) : V::zero();
#pragma unroll
                    for (int e = 0; e < N; e++) {
                        if (e >= nvalid) break;
                        const float bw = prm.b ? V::f32(bv, e) : P::to_f32(bs);
                        const float aw0 = prm.a[0] ? V::f32(av0, e) : P::to_f32(as0);
                        const float aw1 = prm.a[1] ? V::f32(av1, e) : P::to_f32(as1);
                        const float fx = V::f32(vx, e), fy = V::f32(r2, e);
                        e_acc += (double)e_term(V::f32(pold, e), V::f32(pv, e), bw);
                        e_acc += (double)e_term(fx, fx, aw0);
                        e_acc += (double)e_term(fy, fy, aw1);
                    }
                }
            }
            r0 = r1;
            r1 = r2;
            r2 = r3;
            u0 = u1;
            u1 = u2;
            u2 = u3;
        }
        return e_acc;
    }
}

template <class P, int COMP, bool ENERGY>
__global__ void __launch_bounds__(256, 3) batch_kp_strip(const BatchShot *__restrict__ shots, const int *item0,
                                                      int nshots, int nitems, int yc, double *item_part) {
    constexpr int N = VecOf<P>::T::N;
    __shared__ int s_item0[kMaxShots + 1];
    for (int t = threadIdx.x; t <= nshots; t += blockDim.x) s_item0[t] = item0[t];
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int wpb = blockDim.x >> 5;
    for (int item = blockIdx.x * wpb + (threadIdx.x >> 5); item < nitems; item += gridDim.x * wpb) {
        const StripItem it = strip_of<N>(s_item0, nshots, item, shots, yc);
        const AcParams prm = shots[it.s].prm;
        const int64_t step = shots[it.s].step;
        double e_acc = kp_strip_item<P, COMP, ENERGY>(prm, step, it, lane);
        if (ENERGY) {
            for (int off = 16; off > 0; off >>= 1) e_acc += __shfl_down_sync(0xffffffffu, e_acc, off);
            if (lane == 0) item_part[item] = e_acc;
        }
    }
}

// ------------------------------------------------------------------------
// One-pass row strips: both half steps of a strip in one launch
// ------------------------------------------------------------------------

// New v_x at grid point (m, j), m inside the grid, from the old set: the
// one-point arithmetic of the strips (stencil over p at m-1 .. m+2 with the x
// images, the multiplier, the plain or compensated update).
template <class V, class P, int COMP>
__device__ __forceinline__ typename V::RS vx_new_scalar(const AcParams &prm, const void *pin, const void *vxin,
                                                        const void *txin, int m, int j) {
    using RS = typename V::RS;
    const typename P::A D = stencil<P>(P::ld(x_val<V>(pin, prm, m - 1, j, true)), P::ld(x_val<V>(pin, prm, m, j, true)),
                                       P::ld(x_val<V>(pin, prm, m + 1, j, true)),
                                       P::ld(x_val<V>(pin, prm, m + 2, j, true)));
    const int64_t q = m + prm.sy * (int64_t)j;
    RS Vv = static_cast<const RS *>(vxin)[q];
    RS Tv = COMP ? static_cast<const RS *>(txin)[q] : RS(0);
    update<P, COMP>(Vv, Tv, P::mul(coef<P>(prm.a[0], prm.a_uni[0], q), D));
    return Vv;
}

// One strip item per warp, walking down its rows j = y0-2 .. y1 (from row 0
// at a rigid top face): the new v_y of row j (rows y0-2, y0-1 and y1 are the
// halo this strip recomputes rather than reads), the new v_x of row j, then
// p of row j-1, which reads v_y of rows j-3 .. j and v_x of row j-1 with its
// x neighbours. Rows past a rigid y face take the images of computed rows
// (v_y is even about the walls), as do the x neighbours past a rigid x face;
// neighbours that belong to another strip, or that wrap around a periodic
// face, are recomputed with the one-point arithmetic. The operations are
// those of the two-kernel strips, in the same order, so the bits are too.
template <class P, int COMP, bool ENERGY>
__global__ void __launch_bounds__(128, 4) batch_fused_strip(const BatchShot *__restrict__ shots, const int *item0,
                                                         int nshots, int nitems, int yc, double *item_part) {
    using V = typename VecOf<P>::T;
    using Raw = typename V::Raw;
    using AV = typename V::AV;
    using RS = typename V::RS;
    constexpr int N = V::N;
    __shared__ int s_item0[kMaxShots + 1];
    for (int t = threadIdx.x; t <= nshots; t += blockDim.x) s_item0[t] = item0[t];
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int wpb = blockDim.x >> 5;
    for (int item = blockIdx.x * wpb + (threadIdx.x >> 5); item < nitems; item += gridDim.x * wpb) {
        const StripItem it = strip_of<N>(s_item0, nshots, item, shots, yc);
        const BatchShot &sh = shots[it.s];
        const AcParams prm = sh.prm;
        const int64_t last = sh.step;   // the index of the last step taken
        const int64_t step = last + 1;  // this step (time index of the source)
        const bool a_in = (sh.fsteps & 1) == 0;
        const void *pin = a_in ? prm.p : sh.alt_p;
        void *pout = a_in ? sh.alt_p : prm.p;
        const void *vin0 = a_in ? prm.v[0] : sh.alt_v[0], *vin1 = a_in ? prm.v[1] : sh.alt_v[1];
        void *vout0 = a_in ? sh.alt_v[0] : prm.v[0], *vout1 = a_in ? sh.alt_v[1] : prm.v[1];
        const void *tin0 = a_in ? prm.tv[0] : sh.alt_tv[0], *tin1 = a_in ? prm.tv[1] : sh.alt_tv[1];
        void *tout0 = a_in ? sh.alt_tv[0] : prm.tv[0], *tout1 = a_in ? sh.alt_tv[1] : prm.tv[1];
        const int nx = prm.n[0], ny = prm.n[1];
        const bool rigid_x = prm.bc[0] == BC_RIGID, rigid_y = prm.bc[1] == BC_RIGID;
        const int x = it.x0 + lane * N;
        const bool active = x < nx;
        const int nvalid = active ? min(N, nx - x) : 0;
        const bool left_edge = active && lane == 0;
        const bool right_edge = active && (lane == 31 || x + N >= nx);
        const int jstart = (it.y0 == 0 && rigid_y) ? 0 : it.y0 - 2;
        // old p rows j-1, j, j+1 (row j+2 loaded in the loop)
        Raw pq0 = row_vec<V>(pin, prm, x, jstart - 1, true, active);
        Raw pq1 = row_vec<V>(pin, prm, x, jstart, true, active);
        Raw pq2 = row_vec<V>(pin, prm, x, jstart + 1, true, active);
        // new v_y rows j-3, j-2, j-1
        Raw vq0 = V::zero(), vq1 = V::zero(), vq2 = V::zero();
        // new v_x of row j-1 (elements past the grid replaced by their images)
        // and its x neighbours at x-2, x-1, x+N
        Raw vxo = V::zero();
        RS xl1 = RS(0), xl0 = RS(0), xrr = RS(0);
        double e_acc = 0.0;
        for (int j = jstart; j <= it.y1; j++) {
            const Raw pq3 = row_vec<V>(pin, prm, x, j + 2, true, active);
            // ---- new v_y of row j (half point j + 1/2)
            Raw vyn = V::zero();
            if (j >= ny && rigid_y) {
                vyn = vq2;  // the image of row ny - 1 (even about the wall)
            } else if (active) {
                int jm;
                img_half(j, ny, prm.bc[1], jm);  // the row itself, or its periodic wrap
                const int64_t qy = x + prm.sy * (int64_t)jm;
                Raw vo = at<V>(const_cast<void *>(vin1), qy);
                Raw to = COMP ? at<V>(const_cast<void *>(tin1), qy) : V::zero();
                const AV Dy = vstencil<V>(V::ld(pq0), V::ld(pq1), V::ld(pq2), V::ld(pq3));
                V::template update<COMP>(vo, to, V::mul(coef_v<V>(prm.a[1], prm.a_uni[1], qy), Dy));
                vyn = vo;
                if (j >= it.y0 && j < it.y1) {
                    store_vec<V>(vout1, qy, vo, nvalid);
                    if (COMP) store_vec<V>(tout1, qy, to, nvalid);
                }
            }
            // ---- new v_x of row j (stored rows only)
            Raw vxn = V::zero();
            RS nl1 = RS(0), nl0 = RS(0), nrr = RS(0);
            if (j >= it.y0 && j < it.y1) {
                const int64_t q = x + prm.sy * (int64_t)j;
                // strip edges inside the grid: the neighbouring vector of p, v_x,
                // t_vx (and a_x when it varies) of this row, loaded at once
                // (left: x-N .. x-1; right: x+N .. x+2N-1 when x+N+2 lies inside)
                const bool lh = left_edge && x > 0;
                const bool rh = right_edge && x + N + 2 < nx;
                Raw hp = V::zero(), hvx = V::zero(), htx = V::zero(), ha = V::zero();
                if (lh || rh) {
                    const int64_t qh = q + (lh ? -N : N);
                    hp = at<V>(const_cast<void *>(pin), qh);
                    hvx = at<V>(const_cast<void *>(vin0), qh);
                    if (COMP) htx = at<V>(const_cast<void *>(tin0), qh);
                    if (prm.a[0]) ha = at<V>(const_cast<void *>(prm.a[0]), qh);
                }
                Raw own = pq1;
                RS l0 = RS(0), r0 = RS(0), r1 = RS(0);
                if (left_edge) l0 = lh ? V::get(hp, N - 1) : x_val<V>(pin, prm, x - 1, j, true);
                if (right_edge) {
                    r0 = rh ? V::get(hp, 0) : x_val<V>(pin, prm, x + N, j, true);
                    r1 = rh ? V::get(hp, 1) : x_val<V>(pin, prm, x + N + 1, j, true);
#pragma unroll
                    for (int e = 1; e < N; e++)
                        if (e >= nvalid) raw_set<RS, Raw>(own, e, x_val<V>(pin, prm, x + e, j, true));
                }
                const RS sl0 = shfl_rs(V::get(own, N - 1), 1, true);
                const RS sr0 = shfl_rs(V::get(own, 0), 1, false);
                const RS sr1 = shfl_rs(V::get(own, 1), 1, false);
                if (!left_edge) l0 = sl0;
                if (!right_edge) {
                    r0 = sr0;
                    r1 = sr1;
                }
                if (active) {
                    const AV o = V::ld(own);
                    const AV Dx = vstencil<V>(V::shr1(o, V::lds(l0)), o, V::shl1(o, V::lds(r0)),
                                              V::shl2(o, V::lds(r0), V::lds(r1)));
                    Raw vo = at<V>(const_cast<void *>(vin0), q);
                    Raw to = COMP ? at<V>(const_cast<void *>(tin0), q) : V::zero();
                    V::template update<COMP>(vo, to, V::mul(coef_v<V>(prm.a[0], prm.a_uni[0], q), Dx));
                    vxn = vo;
                    store_vec<V>(vout0, q, vo, nvalid);
                    if (COMP) store_vec<V>(tout0, q, to, nvalid);
                }
                // the x neighbours of the new v_x of this row, for p of this row
                // at the next iteration: element nvalid of a vector cut by the
                // grid's right face holds the image of v_x(nx)
                if (right_edge && nvalid < N) {
                    const RS img = rigid_x ? V::get(vxn, nvalid - 1)
                                           : vx_new_scalar<V, P, COMP>(prm, pin, vin0, tin0, 0, j);
                    raw_set<RS, Raw>(vxn, nvalid, img);
                }
                nl1 = shfl_rs(V::get(vxn, N - 2), 1, true);
                nl0 = shfl_rs(V::get(vxn, N - 1), 1, true);
                nrr = shfl_rs(V::get(vxn, 0), 1, false);
                // new v_x at one point from registers: p at e-1 .. e+2 of the
                // concatenation (halo vector, own vector), the old v_x, t_vx and
                // a_x of the halo vector's element h
                auto edge_vx = [&](RS pm1, RS p0, RS p1, RS p2, int h) -> RS {
                    const typename P::A D = stencil<P>(P::ld(pm1), P::ld(p0), P::ld(p1), P::ld(p2));
                    RS Vv = V::get(hvx, h);
                    RS Tv = COMP ? V::get(htx, h) : RS(0);
                    RS a_s;
                    if (prm.a[0]) a_s = V::get(ha, h);
                    else from_bits(prm.a_uni[0], a_s);
                    update<P, COMP>(Vv, Tv, P::mul(P::ld(a_s), D));
                    return Vv;
                };
                if (left_edge) {
                    if (lh) {
                        // v_x at x-2: p at x-3 .. x; at x-1: p at x-2 .. x+1
                        // (own: the row's p vector with the elements past the grid
                        // replaced by their images)
                        nl1 = edge_vx(V::get(hp, N - 3), V::get(hp, N - 2), V::get(hp, N - 1), V::get(own, 0), N - 2);
                        nl0 = edge_vx(V::get(hp, N - 2), V::get(hp, N - 1), V::get(own, 0), V::get(own, 1), N - 1);
                    } else if (x > 0) {
                        nl1 = vx_new_scalar<V, P, COMP>(prm, pin, vin0, tin0, x - 2, j);
                        nl0 = vx_new_scalar<V, P, COMP>(prm, pin, vin0, tin0, x - 1, j);
                    } else if (rigid_x) {  // v_x even about the wall at -1/2
                        nl1 = V::get(vxn, 1);
                        nl0 = V::get(vxn, 0);
                    } else {
                        nl1 = vx_new_scalar<V, P, COMP>(prm, pin, vin0, tin0, nx - 2, j);
                        nl0 = vx_new_scalar<V, P, COMP>(prm, pin, vin0, tin0, nx - 1, j);
                    }
                }
                if (right_edge) {
                    // v_x at x+N: p at x+N-1 .. x+N+2
                    if (rh) nrr = edge_vx(V::get(own, N - 1), V::get(hp, 0), V::get(hp, 1), V::get(hp, 2), 0);
                    else if (x + N < nx) nrr = vx_new_scalar<V, P, COMP>(prm, pin, vin0, tin0, x + N, j);
                    else if (rigid_x) nrr = V::get(vxn, N - 1);  // v_x(nx) = v_x(nx - 1) when nvalid == N
                    else nrr = vx_new_scalar<V, P, COMP>(prm, pin, vin0, tin0, x + N - nx, j);
                }
            }
            if (j == 1 && it.y0 == 0 && rigid_y) {
                // rows -2 and -1 are the images of rows 1 and 0
                vq0 = vyn;
                vq1 = vq2;
            }
            // ---- p of row j - 1
            const int jp = j - 1;
            if (jp >= it.y0 && jp < it.y1 && active) {
                const int64_t q = x + prm.sy * (int64_t)jp;
                const AV o = V::ld(vxo);
                AV R = vstencil<V>(V::shr2(o, V::lds(xl1), V::lds(xl0)), V::shr1(o, V::lds(xl0)), o,
                                   V::shl1(o, V::lds(xrr)));
                R = V::add(R, vstencil<V>(V::ld(vq0), V::ld(vq1), V::ld(vq2), V::ld(vyn)));
                if (jp == prm.src_j && prm.src_i >= x && prm.src_i < x + N && step < prm.src_nt) {
                    const typename V::AS s_ = static_cast<const typename V::AS *>(prm.src)[step];
#pragma unroll
                    for (int e = 0; e < N; e++)
                        if (e == prm.src_i - x) V::set(R, e, P::add(V::aget(R, e), s_));
                }
                Raw pv = pq0;
                Raw tv = COMP ? at<V>(prm.tp, q) : V::zero();
                const Raw pold = pv;
                V::template update<COMP>(pv, tv, V::mul(coef_v<V>(prm.b, prm.b_uni, q), R));
                store_vec<V>(pout, q, pv, nvalid);
                if (COMP) store_vec<V>(prm.tp, q, tv, nvalid);
                if (ENERGY) {
                    RS bs, as0, as1;
                    from_bits(prm.b_uni, bs);
                    from_bits(prm.a_uni[0], as0);
                    from_bits(prm.a_uni[1], as1);
                    const Raw bv = prm.b ? at<V>(const_cast<void *>(prm.b), q) : V::zero();
                    const Raw av0 = prm.a[0] ? at<V>(const_cast<void *>(prm.a[0]), q) : V::zero();
                    const Raw av1 = prm.a[1] ? at<V>(const_cast<void *>(prm.a[1]), q) : V::zero();
#pragma unroll
                    for (int e = 0; e < N; e++) {
                        if (e >= nvalid) break;
                        const float bw = prm.b ? V::f32(bv, e) : P::to_f32(bs);
                        const float aw0 = prm.a[0] ? V::f32(av0, e) : P::to_f32(as0);
                        const float aw1 = prm.a[1] ? V::f32(av1, e) : P::to_f32(as1);
                        const float fx = V::f32(vxo, e), fy = V::f32(vq2, e);
                        e_acc += (double)e_term(V::f32(pold, e), V::f32(pv, e), bw);
                        e_acc += (double)e_term(fx, fx, aw0);
                        e_acc += (double)e_term(fy, fy, aw1);
                    }
                }
            }
            pq0 = pq1;
            pq1 = pq2;
            pq2 = pq3;
            vq0 = vq1;
            vq1 = vq2;
            vq2 = vyn;
            vxo = vxn;
            xl1 = nl1;
            xl0 = nl0;
            xrr = nrr;
        }
        if (ENERGY) {
            for (int off = 16; off > 0; off >>= 1) e_acc += __shfl_down_sync(0xffffffffu, e_acc, off);
            if (lane == 0) item_part[item] = e_acc;
        }
    }
}

// Advance every shot's step counter and one-pass count after a one-pass launch.
__global__ void batch_advance(BatchShot *shots, int nshots) {
    for (int s = threadIdx.x; s < nshots; s += blockDim.x) {
        shots[s].step++;
        shots[s].fsteps++;
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

// ------------------------------------------------------------------------
// Every step of a call in one cooperative launch (BATCH_PERSIST)
// ------------------------------------------------------------------------

// Grid-wide barrier on a counter that only grows within a launch (zeroed
// before it): each block's thread 0 adds one and waits until every block has
// arrived at this and the earlier barriers. The fences order the blocks'
// writes before the barrier with the reads after it. The wait is bounded
// (2^24 polls of about 64 ns): on expiry it sets *err, and every block leaves
// at its next check (the others then expire in turn).
__device__ __forceinline__ bool grid_barrier(unsigned int *bar, int *err, unsigned int &gen) {
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(bar, 1u);
        const unsigned int target = (gen + 1u) * gridDim.x;
        for (uint32_t polls = 0;; polls++) {
            unsigned int v;
            asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(bar) : "memory");
            if (v >= target) break;
            if (polls > (1u << 24)) {
                atomicExch(err, 1);
                break;
            }
            __nanosleep(64);
        }
        __threadfence();
    }
    gen++;
    __syncthreads();
    return *reinterpret_cast<volatile int *>(err) == 0;
}

// nsteps plain steps of every shot: velocity strips, barrier, pressure
// strips, barrier; block 0 advances the step counters at the start of each
// step (the pressure phase reads them after the barrier). (The step that
// reduces the energy runs on the two-launch strips: with the energy terms
// inlined too, this kernel would spill at its 80-register bound.)
template <class P, int COMP>
__global__ void __launch_bounds__(256, 3) batch_persist_strips(BatchShot *shots, const int *item0, int nshots,
                                                            int nitems, int yc, int64_t nsteps,
                                                            unsigned int *bar, int *err) {
    constexpr int N = VecOf<P>::T::N;
    __shared__ int s_item0[kMaxShots + 1];
    for (int t = threadIdx.x; t <= nshots; t += blockDim.x) s_item0[t] = item0[t];
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int wpb = blockDim.x >> 5;
    const int w0 = blockIdx.x * wpb + (threadIdx.x >> 5), gw = gridDim.x * wpb;
    unsigned int gen = 0;
    for (int64_t s = 0; s < nsteps; s++) {
        if (blockIdx.x == 0)
            for (int t = threadIdx.x; t < nshots; t += blockDim.x) shots[t].step++;
        for (int item = w0; item < nitems; item += gw) {
            const StripItem it = strip_of<N>(s_item0, nshots, item, shots, yc);
            const AcParams prm = shots[it.s].prm;
            kv_strip_item<P, COMP>(prm, it, lane);
        }
        if (!grid_barrier(bar, err, gen)) return;
        for (int item = w0; item < nitems; item += gw) {
            const StripItem it = strip_of<N>(s_item0, nshots, item, shots, yc);
            const AcParams prm = shots[it.s].prm;
            const int64_t step = shots[it.s].step;
            kp_strip_item<P, COMP, false>(prm, step, it, lane);
        }
        if (!grid_barrier(bar, err, gen)) return;
    }
}

// After a persistent launch: an expired barrier marks every shot's context.
__global__ void batch_err_propagate(BatchShot *shots, int nshots, const int *err) {
    if (*err == 0) return;
    for (int s = threadIdx.x; s < nshots; s += blockDim.x)
        if (shots[s].err) *shots[s].err = 1;
}

template <class P, int COMP>
static cudaError_t launch_pc(const BatchLaunch &L, bool energy, cudaStream_t st);

template <class P, int COMP>
static cudaError_t persist_pc(const BatchLaunch &L, int64_t nsteps, bool energy_last, cudaStream_t st) {
    void *fn = reinterpret_cast<void *>(&batch_persist_strips<P, COMP>);
    const int threads = 32 * L.wpb;
    int dev = 0, sms = 1, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, 0);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    // every block resident at once (a cooperative launch refuses more)
    const int grid = std::max(1, std::min((L.nitems + L.wpb - 1) / L.wpb, per_sm * sms));
    // the barrier counter grows by grid per barrier, two barriers a step: keep
    // it below 2^31 within a launch
    const int64_t chunk = std::max<int64_t>(1, ((int64_t)1 << 30) / grid);
    // the plain steps in cooperative launches; the last step, which reduces
    // the energy, on the two-launch strips of the same rows and warps
    const int64_t plain = energy_last ? nsteps - 1 : nsteps;
    e = cudaMemsetAsync(L.err, 0, sizeof(int), st);
    for (int64_t done = 0; done < plain && e == cudaSuccess;) {
        const int64_t n = std::min(chunk, plain - done);
        e = cudaMemsetAsync(L.bar, 0, sizeof(unsigned int), st);
        if (e != cudaSuccess) break;
        BatchShot *shots = L.shots;
        const int *item0 = L.item0;
        int nshots = L.nshots, nitems = L.nitems, yc = L.yc;
        int64_t ns = n;
        unsigned int *bar = L.bar;
        int *err = L.err;
        void *args[] = {&shots, &item0, &nshots, &nitems, &yc, &ns, &bar, &err};
        e = cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(threads), args, 0, st);
        done += n;
    }
    if (e == cudaSuccess && plain > 0) {
        batch_err_propagate<<<1, 256, 0, st>>>(L.shots, L.nshots, L.err);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && energy_last) {
        BatchLaunch S = L;
        S.kind = BATCH_STRIPS;
        S.grid = 16 * sms * 4 / L.wpb;  // a grid-stride loop: any size works
        e = launch_pc<P, COMP>(S, true, st);
    }
    return e;
}

cudaError_t batch_persist(const BatchLaunch &L, int prec, int comp, int64_t nsteps, bool energy_last,
                          cudaStream_t st) {
    if (L.kind != BATCH_PERSIST || L.wpb < 1 || L.wpb > 8 || L.yc < 1 || !L.bar || !L.err)
        return cudaErrorInvalidValue;
    if (nsteps < 1) return cudaSuccess;
    switch (prec) {
    case PREC_FP32:
        return comp == 0 ? persist_pc<F32, 0>(L, nsteps, energy_last, st)
                         : comp == 3 ? persist_pc<F32, 3>(L, nsteps, energy_last, st)
                                     : persist_pc<F32, 6>(L, nsteps, energy_last, st);
    case PREC_FP16:
        return comp == 0 ? persist_pc<F16, 0>(L, nsteps, energy_last, st)
                         : comp == 3 ? persist_pc<F16, 3>(L, nsteps, energy_last, st)
                                     : persist_pc<F16, 6>(L, nsteps, energy_last, st);
    case PREC_BF16:
        return comp == 0 ? persist_pc<BF16, 0>(L, nsteps, energy_last, st)
                         : comp == 3 ? persist_pc<BF16, 3>(L, nsteps, energy_last, st)
                                     : persist_pc<BF16, 6>(L, nsteps, energy_last, st);
    case PREC_FP16_F32ARITH:
        return comp ? persist_pc<F16W, 3>(L, nsteps, energy_last, st) : persist_pc<F16W, 0>(L, nsteps, energy_last, st);
    case PREC_BF16_F32ARITH:
        return comp ? persist_pc<BF16W, 3>(L, nsteps, energy_last, st)
                    : persist_pc<BF16W, 0>(L, nsteps, energy_last, st);
    case PREC_FP16_PAIRS:
        return comp ? persist_pc<F16WP, 3>(L, nsteps, energy_last, st) : cudaErrorInvalidValue;
    default: return cudaErrorInvalidValue;
    }
}

template <class P, int COMP>
static cudaError_t launch_pc(const BatchLaunch &L, bool energy, cudaStream_t st) {
    if (L.kind == BATCH_FUSED) {
        // (the one-pass strips read the stored values only)
        if constexpr (IsPairs<P>::value) {
            return cudaErrorInvalidValue;
        } else {
            const int threads = 32 * L.wpb;
            if (energy)
                batch_fused_strip<P, COMP, true><<<L.grid, threads, 0, st>>>(L.shots, L.item0, L.nshots,
                                                                             L.nitems, L.yc, L.item_part);
            else
                batch_fused_strip<P, COMP, false><<<L.grid, threads, 0, st>>>(L.shots, L.item0, L.nshots,
                                                                              L.nitems, L.yc, L.item_part);
            batch_advance<<<1, 256, 0, st>>>(L.shots, L.nshots);
        }
    } else if (L.kind == BATCH_STRIPS) {
        const int threads = 32 * L.wpb;
        batch_kv_strip<P, COMP><<<L.grid, threads, 0, st>>>(L.shots, L.item0, L.nshots, L.nitems, L.yc);
        if (energy)
            batch_kp_strip<P, COMP, true><<<L.grid, threads, 0, st>>>(L.shots, L.item0, L.nshots, L.nitems, L.yc,
                                                                      L.item_part);
        else
            batch_kp_strip<P, COMP, false><<<L.grid, threads, 0, st>>>(L.shots, L.item0, L.nshots, L.nitems,
                                                                       L.yc, L.item_part);
    } else {
        const int threads = L.bx * L.by;
        batch_half_step<P, COMP, 0><<<L.grid, threads, 0, st>>>(L.shots, L.item0, L.nshots, L.nitems, L.bx,
                                                                L.by, 0, L.item_part);
        batch_half_step<P, COMP, 1><<<L.grid, threads, 0, st>>>(L.shots, L.item0, L.nshots, L.nitems, L.bx,
                                                                L.by, energy ? 1 : 0, L.item_part);
    }
    if (energy) batch_energy_reduce<<<L.nshots, 256, 0, st>>>(L.shots, L.item0, L.item_part);
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

int64_t batch_items_of(int kind, int bx, int by, int yc, int prec, int64_t nx, int64_t ny) {
    if (kind == BATCH_STRIPS || kind == BATCH_FUSED || kind == BATCH_PERSIST) {
        const int64_t tx = 32 * (prec == PREC_FP32 ? 4 : 8);
        return ((nx + tx - 1) / tx) * ((ny + yc - 1) / yc);
    }
    return ((nx + bx - 1) / bx) * ((ny + by - 1) / by);
}

cudaError_t batch_step(const BatchLaunch &L, int prec, int comp, bool energy, cudaStream_t st) {
    if (L.kind == BATCH_PERSIST) return batch_persist(L, prec, comp, 1, energy, st);
    if (L.kind == BATCH_STRIPS || L.kind == BATCH_FUSED) {
        if (L.wpb < 1 || L.wpb > 8 || L.yc < 1) return cudaErrorInvalidValue;
    } else if (L.bx * L.by > 256 || (L.bx * L.by) % 32 != 0) {
        return cudaErrorInvalidValue;
    }
    switch (prec) {
    case PREC_FP32: return launch_p<F32>(L, comp, energy, st);
    case PREC_FP16: return launch_p<F16>(L, comp, energy, st);
    case PREC_BF16: return launch_p<BF16>(L, comp, energy, st);
    case PREC_FP16_F32ARITH: return launch_p<F16W>(L, comp ? 3 : 0, energy, st);
    case PREC_BF16_F32ARITH: return launch_p<BF16W>(L, comp ? 3 : 0, energy, st);
    case PREC_FP16_PAIRS: return comp ? launch_pc<F16WP, 3>(L, energy, st) : cudaErrorInvalidValue;
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace wave
