// acoustic2d_cluster.cu -- 2D acoustic leapfrog steps with the whole state
// resident in the shared memory of one thread-block cluster.
//
// A small 2D grid (one that the shared memory of up to 16 CTAs holds) is
// launch-bound on the row strips: a step is two launches of a few
// microseconds each. Here one launch runs any number of steps. The grid's rows
// are cut into C bands, one per CTA of a cluster of C CTAs. Each CTA copies its
// band of p, v_x, v_y (and their compensations) into shared memory, runs the
// launch's steps, and copies the band back. Per step (Algorithm 1 / 2):
//   velocity half step of every strip of the band      (reads p, rows j-1 .. j+2)
//   cluster barrier
//   pressure half step, source, energy terms           (reads v_y, rows j-2 .. j+1)
//   cluster barrier
//   rank 0 sums the bands' energies; the band holding a receiver samples it
// The stencil rows past a band's edge are read from the neighbouring CTA's
// shared memory (distributed shared memory); the barriers (release / acquire at
// cluster scope) order those reads after the writes of the previous half step.
// The barriers are the hardware cluster barrier: every CTA of a cluster is
// resident at once, and no wait here depends on anything but the cluster.
//
// The per-vector arithmetic is that of the row-strip kernels (batch2d.cu): 32
// lanes x 8 (binary16 / bfloat16) or 4 (binary32) x points per strip, x
// neighbours by warp shuffle, the same boundary images, multiplier vectors and
// updates, so the stored bits equal theirs and the oracle's. Energies are the
// same binary32 terms summed in binary64 in another order.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <algorithm>

#include "acoustic_common.cuh"
#include "strip_common.cuh"
#include "wave_kernels.h"

namespace wave {
namespace cg = cooperative_groups;

namespace {

constexpr int kWarps = 16;       // warps per CTA
constexpr int kMaxCluster = 16;  // CTAs per cluster (above 8: a non-portable size)

// Shared-memory slots of a band: p, v_x, v_y, then (with compensation) t_p,
// t_vx, t_vy; each rows x pitch elements of the storage type.
enum { S_P = 0, S_VX = 1, S_VY = 2, S_TP = 3, S_TVX = 4, S_TVY = 5 };

template <class V>
struct Band {
    using Raw = typename V::Raw;
    using RS = typename V::RS;
    RS *base;      // this CTA's slots
    int slot;      // elements per slot (R * pitch; a band fits in shared memory)
    int sp;        // row pitch (elements), that of the global arrays
    int R;         // rows per band
    int r0, r1;    // this band's rows [r0, r1)
    int rank;

    __device__ __forceinline__ RS *own_row(int a, int j) const { return base + (a * slot + (j - r0) * sp); }
    // Row jy of slot a (0 <= jy < ny), in whichever band holds it. A row
    // less than one band height above or below this band is in the
    // neighbouring band (bands start at multiples of R); others (the images
    // of periodic y walls wrap across the grid) take the division.
    __device__ __forceinline__ const RS *row(int a, int jy) const {
        if (jy >= r0 && jy < r1) return own_row(a, jy);
        const int owner = (jy >= r0 - R && jy < r0 + 2 * R) ? (jy < r0 ? rank - 1 : rank + 1) : jy / R;
        RS *p = base + (a * slot + (jy - owner * R) * sp);
        return cg::this_cluster().map_shared_rank(p, (unsigned)owner);
    }
    // Row my at x (a whole vector) with the y boundary image (as row_vec of
    // the strips): zero for inactive lanes and on the p = 0 wall rows.
    __device__ __forceinline__ Raw rvec(const AcParams &prm, int a, int x, int my, bool node_y, bool active) const {
        int jy;
        const int sg = node_y ? img_node(my, prm.n[1], prm.bc[1], jy) : img_half(my, prm.n[1], prm.bc[1], jy);
        if (!active || sg == 0 || jy < 0 || jy >= prm.n[1]) return V::zero();
        const Raw r = *reinterpret_cast<const Raw *>(row(a, jy) + x);
        return sg < 0 ? V::rneg(r) : r;
    }
    // One value of this band's row j at x index mx, with the x image.
    __device__ __forceinline__ RS xval(const AcParams &prm, int a, int mx, int j, bool node_x) const {
        int ix;
        const int sg = node_x ? img_node(mx, prm.n[0], prm.bc[0], ix) : img_half(mx, prm.n[0], prm.bc[0], ix);
        if (sg == 0 || ix < 0 || ix >= prm.n[0]) return RS(0);
        const RS v = own_row(a, j)[ix];
        return sg < 0 ? V::rneg_s(v) : v;
    }
};

// Velocity half step of strip x0, rows [y0, y1) of the band:
// v_x += a_x Dx(p), v_y += a_y Dy(p) (taps RN(p + t_p) for the pair policies).
template <class P, int COMP, class V>
__device__ __forceinline__ void kv_band(const Band<V> &B, const AcParams &prm, int x0, int y0, int y1, int lane) {
    using Raw = typename V::Raw;
    using AV = typename V::AV;
    using RS = typename V::RS;
    using AS = typename V::AS;
    constexpr int N = V::N;
    constexpr bool PAIRS = IsPairs<P>::value;
    const int nx = prm.n[0];
    const int x = x0 + lane * N;
    const bool active = x < nx;
    const int nvalid = active ? min(N, nx - x) : 0;
    const bool left_edge = active && lane == 0;
    const bool right_edge = active && (lane == 31 || x + N >= nx);
    // row queues of p (and t_p): rows j-1, j, j+1; j+2 loaded in the loop
    Raw q0 = B.rvec(prm, S_P, x, y0 - 1, true, active);
    Raw q1 = B.rvec(prm, S_P, x, y0, true, active);
    Raw q2 = B.rvec(prm, S_P, x, y0 + 1, true, active);
    Raw u0 = V::zero(), u1 = V::zero(), u2 = V::zero();
    if (PAIRS) {
        u0 = B.rvec(prm, S_TP, x, y0 - 1, true, active);
        u1 = B.rvec(prm, S_TP, x, y0, true, active);
        u2 = B.rvec(prm, S_TP, x, y0 + 1, true, active);
    }
    for (int j = y0; j < y1; j++) {
        const Raw q3 = B.rvec(prm, S_P, x, j + 2, true, active);
        const Raw u3 = PAIRS ? B.rvec(prm, S_TP, x, j + 2, true, active) : V::zero();
        RS *rvx = B.own_row(S_VX, j), *rvy = B.own_row(S_VY, j);
        RS *rtx = COMP ? B.own_row(S_TVX, j) : nullptr, *rty = COMP ? B.own_row(S_TVY, j) : nullptr;
        Raw vx = V::zero(), vy = V::zero(), tx = V::zero(), ty = V::zero();
        if (active) {
            vx = *reinterpret_cast<const Raw *>(rvx + x);
            vy = *reinterpret_cast<const Raw *>(rvy + x);
            if (COMP) {
                tx = *reinterpret_cast<const Raw *>(rtx + x);
                ty = *reinterpret_cast<const Raw *>(rty + x);
            }
        }
        // x neighbours p[x-1], p[x+N], p[x+N+1] of row j of slot a, from the
        // neighbouring lanes, or at strip and grid edges from the band with
        // the x image (the own vector's elements past the grid replaced by
        // their images)
        auto xnb = [&](int a, Raw &own, RS &l0, RS &r0, RS &r1) {
            l0 = r0 = r1 = RS(0);
            if (left_edge) l0 = B.xval(prm, a, x - 1, j, true);
            if (right_edge) {
                r0 = B.xval(prm, a, x + N, j, true);
                r1 = B.xval(prm, a, x + N + 1, j, true);
#pragma unroll
                for (int e = 1; e < N; e++)
                    if (e >= nvalid) raw_set<RS, Raw>(own, e, B.xval(prm, a, x + e, j, true));
            }
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
        xnb(S_P, own, l0, r0, r1);
        if (PAIRS) xnb(S_TP, ownt, l0t, r0t, r1t);
        if (active) {
            auto tap = [&](const Raw &v, const Raw &t) -> AV { return PAIRS ? V::add(V::ld(v), V::ld(t)) : V::ld(v); };
            auto tap_s = [&](RS v, RS t) -> AS { return PAIRS ? P::add(V::lds(v), V::lds(t)) : V::lds(v); };
            const AV o = tap(own, ownt);
            const AS a_l0 = tap_s(l0, l0t), a_r0 = tap_s(r0, r0t), a_r1 = tap_s(r1, r1t);
            const AV Dx = vstencil<V>(V::shr1(o, a_l0), o, V::shl1(o, a_r0), V::shl2(o, a_r0, a_r1));
            const AV Dy = vstencil<V>(tap(q0, u0), tap(q1, u1), tap(q2, u2), tap(q3, u3));
            const int64_t q = x + prm.sy * (int64_t)j;  // index of the global multiplier arrays
            V::template update<COMP>(vx, tx, V::mul(coef_v<V>(prm.a[0], prm.a_uni[0], q), Dx));
            V::template update<COMP>(vy, ty, V::mul(coef_v<V>(prm.a[1], prm.a_uni[1], q), Dy));
            store_vec<V>(rvx, x, vx, nvalid);
            store_vec<V>(rvy, x, vy, nvalid);
            if (COMP) {
                store_vec<V>(rtx, x, tx, nvalid);
                store_vec<V>(rty, x, ty, nvalid);
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

// Pressure half step of strip x0, rows [y0, y1) of the band at global step
// `step`: p += b (Dx v_x + Dy v_y [+ s]); with `energy`, adds the energy terms
// p^n p^{n+1} / b + v_x^2 / a_x + v_y^2 / a_y of the strip's points to e_acc.
template <class P, int COMP, class V>
__device__ __forceinline__ void kp_band(const Band<V> &B, const AcParams &prm, int x0, int y0, int y1, int lane,
                                        int64_t step, bool energy, double &e_acc) {
    using Raw = typename V::Raw;
    using AV = typename V::AV;
    using RS = typename V::RS;
    using AS = typename V::AS;
    constexpr int N = V::N;
    constexpr bool PAIRS = IsPairs<P>::value;
    const int nx = prm.n[0];
    const int x = x0 + lane * N;
    const bool active = x < nx;
    const int nvalid = active ? min(N, nx - x) : 0;
    const bool left_edge = active && lane == 0;
    const bool right_edge = active && (lane == 31 || x + N >= nx);
    // row queues of v_y (and t_vy): rows j-2, j-1, j; j+1 loaded in the loop
    Raw r0 = B.rvec(prm, S_VY, x, y0 - 2, false, active);
    Raw r1 = B.rvec(prm, S_VY, x, y0 - 1, false, active);
    Raw r2 = B.rvec(prm, S_VY, x, y0, false, active);
    Raw u0 = V::zero(), u1 = V::zero(), u2 = V::zero();
    if (PAIRS) {
        u0 = B.rvec(prm, S_TVY, x, y0 - 2, false, active);
        u1 = B.rvec(prm, S_TVY, x, y0 - 1, false, active);
        u2 = B.rvec(prm, S_TVY, x, y0, false, active);
    }
    for (int j = y0; j < y1; j++) {
        const Raw r3 = B.rvec(prm, S_VY, x, j + 1, false, active);
        const Raw u3 = PAIRS ? B.rvec(prm, S_TVY, x, j + 1, false, active) : V::zero();
        RS *rp = B.own_row(S_P, j), *rtp = COMP ? B.own_row(S_TP, j) : nullptr;
        const RS *rvx = B.own_row(S_VX, j);
        Raw vx = V::zero(), pv = V::zero(), tv = V::zero(), tx = V::zero();
        if (active) {
            vx = *reinterpret_cast<const Raw *>(rvx + x);
            pv = *reinterpret_cast<const Raw *>(rp + x);
            if (COMP) tv = *reinterpret_cast<const Raw *>(rtp + x);
            if (PAIRS) tx = *reinterpret_cast<const Raw *>(B.own_row(S_TVX, j) + x);
        }
        // x neighbours v_x[x-2], v_x[x-1], v_x[x+N] (half-point images) of row j of slot a
        auto xnb = [&](int a, const Raw &rw, Raw &own, RS &l1, RS &l0, RS &rr) {
            own = rw;
            l1 = l0 = rr = RS(0);
            if (left_edge) {
                l1 = B.xval(prm, a, x - 2, j, false);
                l0 = B.xval(prm, a, x - 1, j, false);
            }
            if (right_edge) {
                rr = B.xval(prm, a, x + N, j, false);
#pragma unroll
                for (int e = 1; e < N; e++)
                    if (e >= nvalid) raw_set<RS, Raw>(own, e, B.xval(prm, a, x + e, j, false));
            }
            const RS sl1 = shfl_rs(V::get(rw, N - 2), 1, true);
            const RS sl0 = shfl_rs(V::get(rw, N - 1), 1, true);
            const RS srr = shfl_rs(V::get(rw, 0), 1, false);
            if (!left_edge) {
                l1 = sl1;
                l0 = sl0;
            }
            if (!right_edge) rr = srr;
        };
        Raw own, ownt = V::zero();
        RS l1, l0, rr, l1t = RS(0), l0t = RS(0), rrt = RS(0);
        xnb(S_VX, vx, own, l1, l0, rr);
        if (PAIRS) xnb(S_TVX, tx, ownt, l1t, l0t, rrt);
        if (active) {
            auto tap = [&](const Raw &v, const Raw &t) -> AV { return PAIRS ? V::add(V::ld(v), V::ld(t)) : V::ld(v); };
            auto tap_s = [&](RS v, RS t) -> AS { return PAIRS ? P::add(V::lds(v), V::lds(t)) : V::lds(v); };
            const AV o = tap(own, ownt);
            const AS a_l1 = tap_s(l1, l1t), a_l0 = tap_s(l0, l0t), a_rr = tap_s(rr, rrt);
            // node i reads v_x at i-2, i-1, i, i+1 (+1/2), v_y at rows j-2 .. j+1
            AV R = vstencil<V>(V::shr2(o, a_l1, a_l0), V::shr1(o, a_l0), o, V::shl1(o, a_rr));
            R = V::add(R, vstencil<V>(tap(r0, u0), tap(r1, u1), tap(r2, u2), tap(r3, u3)));
            if (j == prm.src_j && prm.src_i >= x && prm.src_i < x + N && step < prm.src_nt) {
                const AS s_ = static_cast<const AS *>(prm.src)[step];
#pragma unroll
                for (int e = 0; e < N; e++)
                    if (e == prm.src_i - x) V::set(R, e, P::add(V::aget(R, e), s_));
            }
            const int64_t q = x + prm.sy * (int64_t)j;  // index of the global multiplier arrays
            const Raw pold = pv;
            V::template update<COMP>(pv, tv, V::mul(coef_v<V>(prm.b, prm.b_uni, q), R));
            store_vec<V>(rp, x, pv, nvalid);
            if (COMP) store_vec<V>(rtp, x, tv, nvalid);
            if (energy) {
#pragma unroll
                for (int e = 0; e < N; e++) {
                    if (e >= nvalid) break;
                    const float fx = V::f32(vx, e), fy = V::f32(r2, e);
                    e_acc += (double)e_term(V::f32(pold, e), V::f32(pv, e), coef_f32<P>(prm.b, prm.b_uni, q + e));
                    e_acc += (double)e_term(fx, fx, coef_f32<P>(prm.a[0], prm.a_uni[0], q + e));
                    e_acc += (double)e_term(fy, fy, coef_f32<P>(prm.a[1], prm.a_uni[1], q + e));
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
}

// All steps of one launch. R: rows per band; rpi: rows per work item (one
// warp streams an item's rows).
template <class P, int COMP>
__global__ void __launch_bounds__(kWarps * 32, 1) cluster_steps(ClusterRun run, int R, int rpi) {
    using V = typename VecOf<P>::T;
    using RS = typename V::RS;
    constexpr int N = V::N;
    constexpr int NA = COMP ? 6 : 3;
    cg::cluster_group cl = cg::this_cluster();
    const AcParams &prm = run.prm;
    const int nx = prm.n[0], ny = prm.n[1];
    const int rank = (int)cl.block_rank();
    extern __shared__ __align__(16) unsigned char smem[];
    Band<V> B;
    B.base = reinterpret_cast<RS *>(smem);
    B.sp = (int)prm.sy;
    B.slot = R * (int)prm.sy;
    B.R = R;
    B.r0 = min(rank * R, ny);
    B.r1 = min(B.r0 + R, ny);
    B.rank = rank;
    double *e_part = reinterpret_cast<double *>(smem + (size_t)NA * (size_t)B.slot * sizeof(RS));  // kWarps + 1
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    // this band of every array into shared memory (16-byte copies: the pitch
    // is a multiple of 16 elements)
    void *const gf[6] = {prm.p, prm.v[0], prm.v[1], prm.tp, prm.tv[0], prm.tv[1]};
    const int64_t band_vecs = (int64_t)(B.r1 - B.r0) * prm.sy * (int64_t)sizeof(RS) / 16;
    for (int a = 0; a < NA; a++) {
        const uint4 *src = reinterpret_cast<const uint4 *>(static_cast<const RS *>(gf[a]) + (int64_t)B.r0 * prm.sy);
        uint4 *dst = reinterpret_cast<uint4 *>(B.base + a * B.slot);
        for (int64_t i = tid; i < band_vecs; i += blockDim.x) dst[i] = src[i];
    }
    cl.sync();  // every band is loaded before any row past a band edge is read

    const int nstrips = (nx + 32 * N - 1) / (32 * N);
    const int nitems = nstrips * ((B.r1 - B.r0 + rpi - 1) / rpi);
    const int rec_slot = run.rec_field == 1 ? S_VX : run.rec_field == 2 ? S_VY : S_P;
    for (int64_t s = 0; s < run.nsteps; s++) {
        const int64_t step = prm.step + s;
        for (int it = warp; it < nitems; it += kWarps) {
            const int x0 = (it % nstrips) * 32 * N, y0 = B.r0 + (it / nstrips) * rpi;
            kv_band<P, COMP>(B, prm, x0, y0, min(y0 + rpi, B.r1), lane);
        }
        cl.sync();  // new velocities of every band before the pressure half step reads them
        const bool energy = s < run.e_trace_n || (s == run.nsteps - 1 && run.e_last);
        double e_acc = 0.0;
        for (int it = warp; it < nitems; it += kWarps) {
            const int x0 = (it % nstrips) * 32 * N, y0 = B.r0 + (it / nstrips) * rpi;
            kp_band<P, COMP>(B, prm, x0, y0, min(y0 + rpi, B.r1), lane, step, energy, e_acc);
        }
        if (energy) {
            for (int off = 16; off > 0; off >>= 1) e_acc += __shfl_down_sync(0xffffffffu, e_acc, off);
            if (lane == 0) e_part[warp] = e_acc;
            __syncthreads();
            if (tid == 0) {
                double t = 0.0;
                for (int w = 0; w < kWarps; w++) t += e_part[w];
                e_part[kWarps] = t;
            }
        }
        cl.sync();  // new p of every band (and the bands' energies) before the next step
        if (energy && rank == 0 && tid == 0) {
            // the bands' sums in band order; no band rewrites its sum before
            // the next step's first barrier, which waits for this thread
            double t = 0.0;
            for (unsigned r = 0; r < cl.num_blocks(); r++) t += *cl.map_shared_rank(e_part + kWarps, r);
            t *= prm.e_factor;
            if (s < run.e_trace_n) run.e_trace[s] = t;
            if (s == run.nsteps - 1 && run.e_last) *run.e_last = t;
        }
        if (s < run.rec_n) {
            for (int r = tid; r < run.nrec; r += blockDim.x) {
                const int64_t q = run.rec_q[r];
                const int y = (int)(q / prm.sy);
                if (y >= B.r0 && y < B.r1)
                    run.traces[s * run.nrec + r] = P::to_f32(B.own_row(rec_slot, y)[q % prm.sy]);
            }
            __syncthreads();  // sampled before the next velocity half step rewrites v
        }
    }

    // the band back to global memory (only this CTA wrote it)
    for (int a = 0; a < NA; a++) {
        uint4 *dst = reinterpret_cast<uint4 *>(static_cast<RS *>(gf[a]) + (int64_t)B.r0 * prm.sy);
        const uint4 *src = reinterpret_cast<const uint4 *>(B.base + a * B.slot);
        for (int64_t i = tid; i < band_vecs; i += blockDim.x) dst[i] = src[i];
    }
    cl.sync();  // no CTA exits while another may still read its shared memory
}

template <class P, int COMP>
struct Kern {
    static void *fn() { return reinterpret_cast<void *>(&cluster_steps<P, COMP>); }
};

template <class F>
auto dispatch(int prec, int comp, F &&f) -> decltype(f(Kern<F32, 0>())) {
    switch (prec) {
    case PREC_FP32:
        return comp == 0 ? f(Kern<F32, 0>()) : comp == 3 ? f(Kern<F32, 3>()) : f(Kern<F32, 6>());
    case PREC_FP16:
        return comp == 0 ? f(Kern<F16, 0>()) : comp == 3 ? f(Kern<F16, 3>()) : f(Kern<F16, 6>());
    case PREC_BF16:
        return comp == 0 ? f(Kern<BF16, 0>()) : comp == 3 ? f(Kern<BF16, 3>()) : f(Kern<BF16, 6>());
    case PREC_FP16_F32ARITH: return comp == 0 ? f(Kern<F16W, 0>()) : f(Kern<F16W, 3>());
    case PREC_BF16_F32ARITH: return comp == 0 ? f(Kern<BF16W, 0>()) : f(Kern<BF16W, 3>());
    default: return f(Kern<F16WP, 3>());  // PREC_FP16_PAIRS (compensation required)
    }
}

cudaLaunchConfig_t config_of(const ClusterPlan &pl, cudaLaunchAttribute *attr, cudaStream_t st) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)pl.ctas, 1, 1);
    cfg.blockDim = dim3(kWarps * 32, 1, 1);
    cfg.dynamicSmemBytes = pl.smem;
    cfg.stream = st;
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)pl.ctas;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cfg;
}

}  // namespace

bool acoustic_cluster_plan(const AcParams &prm, int prec, int comp, ClusterPlan &pl) {
    if (prec != PREC_FP32 && prec != PREC_FP16 && prec != PREC_BF16 && prec != PREC_FP16_F32ARITH &&
        prec != PREC_BF16_F32ARITH && prec != PREC_FP16_PAIRS)
        return false;
    if (prec == PREC_FP16_PAIRS && !comp) return false;
    const int64_t eb = prec == PREC_FP32 ? 4 : 2, na = comp ? 6 : 3;
    const int vec = prec == PREC_FP32 ? 4 : 8;
    const int ny = prm.n[1];
    if ((prm.sy * eb) % 16 != 0) return false;
    int dev = 0, optin = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return false;
    if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) return false;
    const int nstrips = (prm.n[0] + 32 * vec - 1) / (32 * vec);
    for (int c = kMaxCluster; c >= 1; c--) {
        const int R = (ny + c - 1) / c;
        if ((ny + R - 1) / R != c) continue;  // no empty band
        const size_t smem = (size_t)(R * prm.sy * eb * na) + sizeof(double) * (kWarps + 1);
        if (smem > (size_t)optin) return false;  // fewer CTAs only need more
        ClusterPlan cand;
        cand.ctas = c;
        cand.rows = R;
        cand.rpi = (int)std::max<int64_t>(1, (int64_t)R * nstrips / kWarps);
        cand.smem = smem;
        const bool ok = dispatch(prec, comp, [&](auto k) {
            void *fn = decltype(k)::fn();
            // (the device's limit, so that any plan's size launches later)
            if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, optin) != cudaSuccess ||
                cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess)
                return false;
            cudaLaunchAttribute attr[1];
            cudaLaunchConfig_t cfg = config_of(cand, attr, nullptr);
            int nclusters = 0;
            return cudaOccupancyMaxActiveClusters(&nclusters, fn, &cfg) == cudaSuccess && nclusters >= 1;
        });
        if (!ok) {
            cudaGetLastError();
            continue;
        }
        pl = cand;
        return true;
    }
    return false;
}

cudaError_t acoustic_cluster_steps(const ClusterRun &run, const ClusterPlan &pl, int prec, int comp,
                                   cudaStream_t st) {
    if (run.nsteps < 1) return cudaSuccess;
    return dispatch(prec, comp, [&](auto k) {
        cudaLaunchAttribute attr[1];
        cudaLaunchConfig_t cfg = config_of(pl, attr, st);
        void *args[3] = {const_cast<ClusterRun *>(&run), const_cast<int *>(&pl.rows), const_cast<int *>(&pl.rpi)};
        return cudaLaunchKernelExC(&cfg, decltype(k)::fn(), args);
    });
}

}  // namespace wave
