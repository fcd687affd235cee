// acoustic3d_stream.cu -- 2.5D streaming kernels for the 3D acoustic leapfrog.
//
// Same arithmetic, operation for operation, as the one-thread-per-point
// kernels (fourth-order staggered difference of Section 3, plain or
// compensated update of Algorithms 1 / 2), laid out for HBM bandwidth:
//   * a CTA owns a TX x TY tile of (x, y) columns and walks a chunk of z planes;
//   * each thread owns VEC consecutive x points of one row (one 16-byte vector
//     of the storage format) and keeps the z-neighbour planes of its own
//     vector in registers (a 4-deep queue), so every array is read once;
//   * x neighbours come from the adjacent lanes by warp shuffle (global loads
//     only at tile edges), y neighbours from a double-buffered shared-memory
//     plane (one __syncthreads per plane);
//   * what a plane's barrier would otherwise wait for (the velocity kernel's
//     halo rows, the pressure kernel's v_x and v_y planes) is copied into
//     shared memory by cp.async one plane ahead;
//   * half and bfloat16 arithmetic is done on packed pairs (f16x2 / bf16x2);
//     the pair precision adds a T queue, plane and x neighbours per field.
// Requirements: 3D, n[0] a multiple of VEC. Boundary images (periodic, or the
// odd / even images of the p = 0 walls) are applied on every halo load.
#include <cuda_runtime.h>
#include "acoustic_common.cuh"
#include "strip_common.cuh"
#include "vec_policy.cuh"
#include "wave_kernels.h"

namespace wave {

// Load the raw vector of a field at (x, row m_y, plane m_z) applying the
// boundary images along y and z. node_y / node_z: the field sits on nodes
// (odd image, wall at N) or half points (even image) along that axis. Past a
// cut z face of a slab (prm.zg_lo / zg_hi) the plane comes from the ghost
// planes instead (the y image still applies).
template <class V>
__device__ __forceinline__ typename V::Raw load_vec_img(const void *f, const AcParams &prm, int x,
                                                        int my, int mz, bool node_y, bool node_z) {
    int jy, kz;
    int sy = node_y ? img_node(my, prm.n[1], prm.bc[1], jy) : img_half(my, prm.n[1], prm.bc[1], jy);
    if ((mz < 0 && prm.zg_lo) || (mz >= prm.n[2] && prm.zg_hi)) {
        // ghost planes: lo holds planes -2, -1, hi holds n, n+1 (the kernels read no farther)
        const bool lo = mz < 0;
        const int gk = lo ? mz + 2 : mz - prm.n[2];
        if (sy == 0 || x >= prm.n[0] || my > prm.n[1] + 2 || my < -3 || gk < 0 || gk > 1) return V::zero();
        const typename V::Raw r = *reinterpret_cast<const typename V::Raw *>(
            static_cast<const char *>(lo ? prm.zg_lo : prm.zg_hi) +
            (x + prm.sy * jy + prm.sz * (int64_t)gk) * sizeof(typename V::RS));
        return sy < 0 ? V::rneg(r) : r;
    }
    int sz = node_z ? img_node(mz, prm.n[2], prm.bc[2], kz) : img_half(mz, prm.n[2], prm.bc[2], kz);
    if (sy == 0 || sz == 0 || x >= prm.n[0] || my > prm.n[1] + 2 || my < -3 || mz > prm.n[2] + 2 || mz < -3)
        return V::zero();
    const typename V::Raw *p = reinterpret_cast<const typename V::Raw *>(
        static_cast<const char *>(f) + (x + prm.sy * jy + prm.sz * (int64_t)kz) * sizeof(typename V::RS));
    typename V::Raw r = *p;
    return (sy * sz < 0) ? V::rneg(r) : r;
}

// One scalar of a field at (mx, row j, plane k) with the x boundary image.
template <class V>
__device__ __forceinline__ typename V::RS load_x_img(const void *f, const AcParams &prm, int mx, int j,
                                                     int k, bool node_x) {
    int ix;
    int s = node_x ? img_node(mx, prm.n[0], prm.bc[0], ix) : img_half(mx, prm.n[0], prm.bc[0], ix);
    if (s == 0) return typename V::RS(0);
    typename V::RS v = static_cast<const typename V::RS *>(f)[ix + prm.sy * j + prm.sz * (int64_t)k];
    return s < 0 ? V::rneg_s(v) : v;
}

// (multipliers: coef_v of strip_common.cuh, binary32 for the pair precision)

// 16-byte asynchronous copy global -> shared (cp.async, cached in L2 only);
// src_bytes 0 reads nothing and writes zeros. Completion: cp_wait_all by the
// issuing thread, then a barrier before other threads read the bytes.
__device__ __forceinline__ void cp16(void *smem, const void *gmem, int src_bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(
                     static_cast<uint32_t>(__cvta_generic_to_shared(smem))),
                 "l"(gmem), "r"(src_bytes)
                 : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }


constexpr int TXV = 8;  // threads per tile row

// ------------------------------------------------------------------------
// Velocity half step: v_c += a_c * D_c(p), c = x, y, z.
// ------------------------------------------------------------------------
template <class P, int COMP, int TY>
// (bounded to 64 registers: eight blocks of 128 threads per SM; the kernels
// wait on global loads, and 32 warps per SM hide more of it than the 20 of the
// unbounded 96 registers: 512^3 fp16 + sum_3op 92.5 -> 112.3 Gpt/s)
// (the pair precision, with the T queues, planes and neighbours beside each
// field's, at four blocks per SM)
__global__ void __launch_bounds__(TXV *TY, IsPairs<P>::value ? 4 : 8) kv_stream(AcParams prm, int zchunk) {
    using V = typename VecOf<P>::T;
    using Raw = typename V::Raw;
    using AV = typename V::AV;
    using RS = typename V::RS;
    using AS = typename V::AS;
    constexpr int N = V::N;
    constexpr int TX = TXV * N;
    constexpr bool PAIRS = IsPairs<P>::value;
    __shared__ Raw sp[2][TY + 3][TXV];  // local row r <-> global row y0 - 1 + r
    __shared__ Raw stp[PAIRS ? 2 : 1][PAIRS ? TY + 3 : 1][TXV];  // the pairs: t_p likewise

    const int tid = threadIdx.x;
    const int lx = tid % TXV, row = tid / TXV;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int z0 = blockIdx.z * zchunk;
    const int z1 = min(z0 + zchunk, prm.n[2]);
    const int x = x0 + lx * N;
    const int j = y0 + row;
    const bool active = x < prm.n[0] && j < prm.n[1];
    // halo rows of the shared plane: local rows 0, TY+1, TY+2
    const bool halo_loader = tid < 3 * TXV;
    const int hr = tid / TXV;                       // 0, 1, 2
    const int h_local = hr == 0 ? 0 : TY + hr;
    const int h_row = y0 - 1 + h_local;
    const int h_x = x0 + (tid % TXV) * N;

    // z queue of the own p vector: planes k-1, k, k+1 (k+2 loaded in the
    // loop); the pairs: the same queue of t_p (taps RN(p + t_p))
    Raw q0 = load_vec_img<V>(prm.p, prm, x, j, z0 - 1, true, true);
    Raw q1 = load_vec_img<V>(prm.p, prm, x, j, z0, true, true);
    Raw q2 = load_vec_img<V>(prm.p, prm, x, j, z0 + 1, true, true);
    Raw u0 = V::zero(), u1 = V::zero(), u2 = V::zero();
    if (PAIRS) {
        u0 = load_vec_img<V>(prm.tp, prm, x, j, z0 - 1, true, true);
        u1 = load_vec_img<V>(prm.tp, prm, x, j, z0, true, true);
        u2 = load_vec_img<V>(prm.tp, prm, x, j, z0 + 1, true, true);
    }
    auto tap = [&](const Raw &v, const Raw &t) -> AV { return PAIRS ? V::add(V::ld(v), V::ld(t)) : V::ld(v); };
    auto tap_s = [&](RS v, RS t) -> AS { return PAIRS ? P::add(V::lds(v), V::lds(t)) : V::lds(v); };
    // Halo rows of the shared plane by cp.async one plane ahead (planes inside
    // the grid or slab: only the y image applies, the same on every plane; the
    // odd image's sign is applied in shared memory after the copy lands, zeros
    // at the wall node and past x or the image range, as load_vec_img gives)
    int h_jy = 0;
    const int h_sg = halo_loader ? img_node(h_row, prm.n[1], prm.bc[1], h_jy) : 0;
    const bool h_ok = halo_loader && h_sg != 0 && h_x < prm.n[0] && h_row >= -3 && h_row <= prm.n[1] + 2;
    auto issue_halo = [&](int kk, int bb) {
        if (!halo_loader) return;
        const int64_t qq = h_x + prm.sy * (int64_t)h_jy + prm.sz * (int64_t)kk;
        cp16(&sp[bb][h_local][tid % TXV], h_ok ? static_cast<const char *>(prm.p) + qq * (int64_t)sizeof(RS) : prm.p,
             h_ok ? 16 : 0);
        if (PAIRS)
            cp16(&stp[PAIRS ? bb : 0][PAIRS ? h_local : 0][tid % TXV],
                 h_ok ? static_cast<const char *>(prm.tp) + qq * (int64_t)sizeof(RS) : prm.tp, h_ok ? 16 : 0);
        cp_commit();
    };
    issue_halo(z0, 0);
    int buf = 0;
    for (int k = z0; k < z1; k++) {
        Raw q3 = load_vec_img<V>(prm.p, prm, x, j, k + 2, true, true);
        Raw u3 = PAIRS ? load_vec_img<V>(prm.tp, prm, x, j, k + 2, true, true) : V::zero();
        const int64_t q = x + prm.sy * j + prm.sz * (int64_t)k;
        Raw vv[3], tt[3];
        if (active) {
#pragma unroll
            for (int c = 0; c < 3; c++) {
                vv[c] = at<V>(prm.v[c], q);
                tt[c] = COMP ? at<V>(prm.tv[c], q) : V::zero();
            }
        }
        // x neighbours of the own plane-k vector: p[x-1], p[x+N], p[x+N+1]
        // (of t_p too for the pairs)
        auto xnb = [&](const void *f, const Raw &own_r, RS &l0, RS &r0, RS &r1) {
            l0 = shfl_rs(V::get(own_r, N - 1), 1, true);
            r0 = shfl_rs(V::get(own_r, 0), 1, false);
            r1 = shfl_rs(V::get(own_r, 1), 1, false);
            if (active) {
                if (lx == 0) l0 = load_x_img<V>(f, prm, x - 1, j, k, true);
                if (lx == TXV - 1 || x + N >= prm.n[0]) {
                    r0 = load_x_img<V>(f, prm, x + N, j, k, true);
                    r1 = load_x_img<V>(f, prm, x + N + 1, j, k, true);
                }
            }
        };
        RS l0, r0, r1, l0t = RS(0), r0t = RS(0), r1t = RS(0);
        xnb(prm.p, q1, l0, r0, r1);
        if (PAIRS) xnb(prm.tp, u1, l0t, r0t, r1t);
        sp[buf][row + 1][lx] = q1;
        if (PAIRS) stp[PAIRS ? buf : 0][PAIRS ? row + 1 : 0][lx] = u1;
        cp_wait_all();
        if (h_ok && h_sg < 0) {
            sp[buf][h_local][tid % TXV] = V::rneg(sp[buf][h_local][tid % TXV]);
            if (PAIRS)
                stp[PAIRS ? buf : 0][PAIRS ? h_local : 0][tid % TXV] =
                    V::rneg(stp[PAIRS ? buf : 0][PAIRS ? h_local : 0][tid % TXV]);
        }
        // past the barrier every thread is done with plane k - 1: buffer
        // buf ^ 1 takes plane k + 1's halo rows
        __syncthreads();
        if (k + 1 < z1) issue_halo(k + 1, buf ^ 1);
        if (active) {
            const AV own = tap(q1, u1);
            const AS a_l0 = tap_s(l0, l0t), a_r0 = tap_s(r0, r0t), a_r1 = tap_s(r1, r1t);
            // v_x at i + 1/2: p[i-1], p[i], p[i+1], p[i+2]
            AV Dx = vstencil<V>(V::shr1(own, a_l0), own, V::shl1(own, a_r0), V::shl2(own, a_r0, a_r1));
            // v_y at j + 1/2: rows j-1, j, j+1, j+2 (local rows row, row+1, row+2, row+3)
            auto prow = [&](int r) -> AV {
                return PAIRS ? tap(sp[buf][r][lx], stp[PAIRS ? buf : 0][PAIRS ? r : 0][lx]) : V::ld(sp[buf][r][lx]);
            };
            AV Dy = vstencil<V>(prow(row), own, prow(row + 2), prow(row + 3));
            // v_z at k + 1/2: planes k-1, k, k+1, k+2
            AV Dz = vstencil<V>(tap(q0, u0), own, tap(q2, u2), tap(q3, u3));
            AV D[3] = {Dx, Dy, Dz};
#pragma unroll
            for (int c = 0; c < 3; c++) {
                AV inc = V::mul(coef_v<V>(prm.a[c], prm.a_uni[c], q), D[c]);
                V::template update<COMP>(vv[c], tt[c], inc);
                at<V>(prm.v[c], q) = vv[c];
                if (COMP) at<V>(prm.tv[c], q) = tt[c];
            }
        }
        q0 = q1;
        q1 = q2;
        q2 = q3;
        u0 = u1;
        u1 = u2;
        u2 = u3;
        buf ^= 1;
    }
}

// Compensated binary32 accumulation for the energy (TwoSum per term).
struct KSum {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float x) {
        float t = __fadd_rn(s, x);
        float pa = __fsub_rn(t, x);
        float pb = __fsub_rn(t, pa);
        float da = __fsub_rn(s, pa);
        float db = __fsub_rn(x, pb);
        c = __fadd_rn(c, __fadd_rn(da, db));
        s = t;
    }
};

// ------------------------------------------------------------------------
// Pressure half step: p += b * (Dx vx + Dy vy + Dz vz [+ s]), optional energy.
// ------------------------------------------------------------------------
template <class P, int COMP, int TY, bool ENERGY>
// (64 registers as kv_stream, the pairs four blocks per SM; the energy variant,
// a call's last step, unbounded)
__global__ void __launch_bounds__(TXV *TY, ENERGY ? 1 : (IsPairs<P>::value ? 4 : 8))
    kp_stream(AcParams prm, int zchunk) {
    using V = typename VecOf<P>::T;
    using Raw = typename V::Raw;
    using AV = typename V::AV;
    using RS = typename V::RS;
    using AS = typename V::AS;
    constexpr int N = V::N;
    constexpr int TX = TXV * N;
    constexpr bool PAIRS = IsPairs<P>::value;
    static_assert(sizeof(Raw) == 16, "one 16-byte vector per thread");
    // v_x and v_y planes, filled by cp.async one plane ahead (the copies of
    // plane k + 1 run while plane k is computed, so the plane's barrier waits
    // on no fresh load); the pairs: t_vx, t_vy likewise
    __shared__ Raw sv[2][TY + 3][TXV];  // v_y, local row r <-> global row y0 - 2 + r
    __shared__ Raw sx[2][TY][TXV];      // v_x of the own rows
    __shared__ Raw stv[PAIRS ? 2 : 1][PAIRS ? TY + 3 : 1][TXV];
    __shared__ Raw stx[PAIRS ? 2 : 1][PAIRS ? TY : 1][TXV];

    const int tid = threadIdx.x;
    const int lx = tid % TXV, row = tid / TXV;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int z0 = blockIdx.z * zchunk;
    const int z1 = min(z0 + zchunk, prm.n[2]);
    const int x = x0 + lx * N;
    const int j = y0 + row;
    const bool active = x < prm.n[0] && j < prm.n[1];
    const bool halo_loader = tid < 3 * TXV;
    const int hr = tid / TXV;
    const int h_local = hr == 0 ? 0 : hr == 1 ? 1 : TY + 2;
    const int h_row = y0 - 2 + h_local;
    const int h_x = x0 + (tid % TXV) * N;

    // z queue of the own v_z vector: planes k-2, k-1, k (k+1 loaded in the
    // loop); the pairs: the same queue of t_vz (taps RN(v + t_v))
    Raw r0 = load_vec_img<V>(prm.v[2], prm, x, j, z0 - 2, true, false);
    Raw r1 = load_vec_img<V>(prm.v[2], prm, x, j, z0 - 1, true, false);
    Raw r2 = load_vec_img<V>(prm.v[2], prm, x, j, z0, true, false);
    Raw u0 = V::zero(), u1 = V::zero(), u2 = V::zero();
    if (PAIRS) {
        u0 = load_vec_img<V>(prm.tv[2], prm, x, j, z0 - 2, true, false);
        u1 = load_vec_img<V>(prm.tv[2], prm, x, j, z0 - 1, true, false);
        u2 = load_vec_img<V>(prm.tv[2], prm, x, j, z0, true, false);
    }
    auto tap = [&](const Raw &v, const Raw &t) -> AV { return PAIRS ? V::add(V::ld(v), V::ld(t)) : V::ld(v); };
    auto tap_s = [&](RS v, RS t) -> AS { return PAIRS ? P::add(V::lds(v), V::lds(t)) : V::lds(v); };
    auto gptr = [&](const void *f, int64_t qq) -> const void * {
        return static_cast<const char *>(f) + qq * (int64_t)sizeof(RS);
    };
    // Copies of plane kk (inside the grid or slab: no z image) into buffer bb:
    // the own v_x vector (zeros outside the grid: those lanes' results are not
    // kept and no kept lane reads them), the own and halo v_y rows (rows past
    // the y faces take the even image, which has sign +1; zeros past x or past
    // the image range, as load_vec_img gives).
    auto issue_plane = [&](int kk, int bb) {
        const int64_t zoff = prm.sz * (int64_t)kk;
        const int64_t qo = x + prm.sy * j + zoff;
        cp16(&sx[bb][row][lx], active ? gptr(prm.v[0], qo) : prm.v[0], active ? 16 : 0);
        if (PAIRS)
            cp16(&stx[PAIRS ? bb : 0][PAIRS ? row : 0][lx], active ? gptr(prm.tv[0], qo) : prm.tv[0],
                 active ? 16 : 0);
        auto vy_row = [&](int xx, int my, int lrow, int lcol) {
            int jy;
            img_half(my, prm.n[1], prm.bc[1], jy);
            const bool ok = xx < prm.n[0] && my >= -3 && my <= prm.n[1] + 2;
            const int64_t qq = xx + prm.sy * jy + zoff;
            cp16(&sv[bb][lrow][lcol], ok ? gptr(prm.v[1], qq) : prm.v[1], ok ? 16 : 0);
            if (PAIRS)
                cp16(&stv[PAIRS ? bb : 0][PAIRS ? lrow : 0][lcol], ok ? gptr(prm.tv[1], qq) : prm.tv[1],
                     ok ? 16 : 0);
        };
        vy_row(x, j, row + 2, lx);
        if (halo_loader) vy_row(h_x, h_row, h_local, tid % TXV);
        cp_commit();
    };
    issue_plane(z0, 0);
    KSum acc;
    int buf = 0;
    for (int k = z0; k < z1; k++) {
        Raw r3 = load_vec_img<V>(prm.v[2], prm, x, j, k + 1, true, false);
        Raw u3 = PAIRS ? load_vec_img<V>(prm.tv[2], prm, x, j, k + 1, true, false) : V::zero();
        const int64_t q = x + prm.sy * j + prm.sz * (int64_t)k;
        Raw pv, tv;
        AV bco;  // the multiplier b, loaded with the fields (not after the barrier)
        if (active) {
            pv = at<V>(prm.p, q);
            tv = COMP ? at<V>(prm.tp, q) : V::zero();
            bco = coef_v<V>(prm.b, prm.b_uni, q);
        }
        // x neighbours of v_x: vx[x-2], vx[x-1], vx[x+N]: the tile-edge lanes
        // load theirs from global memory here, the others take them from the
        // adjacent lanes after the barrier (of t_vx too for the pairs)
        const bool left_edge = active && lx == 0;
        const bool right_edge = active && (lx == TXV - 1 || x + N >= prm.n[0]);
        RS el1 = RS(0), el0 = RS(0), err = RS(0), el1t = RS(0), el0t = RS(0), errt = RS(0);
        if (left_edge) {
            el1 = load_x_img<V>(prm.v[0], prm, x - 2, j, k, false);
            el0 = load_x_img<V>(prm.v[0], prm, x - 1, j, k, false);
            if (PAIRS) {
                el1t = load_x_img<V>(prm.tv[0], prm, x - 2, j, k, false);
                el0t = load_x_img<V>(prm.tv[0], prm, x - 1, j, k, false);
            }
        }
        if (right_edge) {
            err = load_x_img<V>(prm.v[0], prm, x + N, j, k, false);
            if (PAIRS) errt = load_x_img<V>(prm.tv[0], prm, x + N, j, k, false);
        }
        // plane k's copies (issued one plane earlier) are in; once every
        // thread is past the barrier, buffer buf ^ 1 (plane k - 1) is free
        cp_wait_all();
        __syncthreads();
        if (k + 1 < z1) issue_plane(k + 1, buf ^ 1);
        const Raw vx = sx[buf][row][lx];
        const Raw vy = sv[buf][row + 2][lx];
        const Raw tx = PAIRS ? stx[PAIRS ? buf : 0][PAIRS ? row : 0][lx] : V::zero();
        const Raw ty = PAIRS ? stv[PAIRS ? buf : 0][PAIRS ? row + 2 : 0][lx] : V::zero();
        auto xnb = [&](const Raw &own_r, RS e1, RS e0, RS er, RS &l1, RS &l0, RS &rr) {
            l1 = shfl_rs(V::get(own_r, N - 2), 1, true);
            l0 = shfl_rs(V::get(own_r, N - 1), 1, true);
            rr = shfl_rs(V::get(own_r, 0), 1, false);
            if (left_edge) { l1 = e1; l0 = e0; }
            if (right_edge) rr = er;
        };
        RS l1, l0, rr, l1t = RS(0), l0t = RS(0), rrt = RS(0);
        xnb(vx, el1, el0, err, l1, l0, rr);
        if (PAIRS) xnb(tx, el1t, el0t, errt, l1t, l0t, rrt);
        if (active) {
            const AV ownx = tap(vx, tx);
            const AS a_l1 = tap_s(l1, l1t), a_l0 = tap_s(l0, l0t), a_rr = tap_s(rr, rrt);
            // node i reads v_x at i-2, i-1, i, i+1 (+1/2)
            AV R = vstencil<V>(V::shr2(ownx, a_l1, a_l0), V::shr1(ownx, a_l0), ownx, V::shl1(ownx, a_rr));
            auto vrow = [&](int r) -> AV {
                return PAIRS ? tap(sv[buf][r][lx], stv[PAIRS ? buf : 0][PAIRS ? r : 0][lx]) : V::ld(sv[buf][r][lx]);
            };
            AV Dy = vstencil<V>(vrow(row), vrow(row + 1), tap(vy, ty), vrow(row + 3));
            R = V::add(R, Dy);
            AV Dz = vstencil<V>(tap(r0, u0), tap(r1, u1), tap(r2, u2), tap(r3, u3));
            R = V::add(R, Dz);
            if (k == prm.src_k && j == prm.src_j && prm.src_i >= x && prm.src_i < x + N &&
                prm.step < prm.src_nt) {
                const typename V::AS sv_ = static_cast<const typename V::AS *>(prm.src)[prm.step];
                // element index known at compile time: R stays in registers
#pragma unroll
                for (int e = 0; e < N; e++)
                    if (e == prm.src_i - x) V::set(R, e, P::add(V::aget(R, e), sv_));
            }
            AV inc = V::mul(bco, R);
            Raw pold = pv;
            V::template update<COMP>(pv, tv, inc);
            at<V>(prm.p, q) = pv;
            if (COMP) at<V>(prm.tp, q) = tv;
            // Energy terms as the one-pass step forms them: v^2 / a with a
            // uniform a as a product by its reciprocal (a per-point a: the
            // division), the four terms of a point summed in binary32, then
            // added to the compensated accumulator
            if constexpr (ENERGY && PAIRS) {
                // (binary32 multipliers, CoefOf)
                const Raw vc[3] = {vx, vy, r2};
                float ia[3];
#pragma unroll
                for (int c = 0; c < 3; c++) ia[c] = __frcp_rn(coef_f32<P>(nullptr, prm.a_uni[c], 0));
#pragma unroll
                for (int e = 0; e < N; e++) {
                    float t = e_term(V::f32(pold, e), V::f32(pv, e), coef_f32<P>(prm.b, prm.b_uni, q + e));
#pragma unroll
                    for (int c = 0; c < 3; c++) {
                        const float vf = V::f32(vc[c], e);
                        t = __fadd_rn(t, prm.a[c] ? e_term(vf, vf, coef_f32<P>(prm.a[c], prm.a_uni[c], q + e))
                                                  : __fmul_rn(__fmul_rn(vf, vf), ia[c]));
                    }
                    acc.add(t);
                }
            } else if constexpr (ENERGY) {
                typename V::RS bs, as[3];
                const Raw *bvec = prm.b ? reinterpret_cast<const Raw *>(
                                              static_cast<const char *>(prm.b) + q * sizeof(RS)) : nullptr;
                Raw bv = bvec ? *bvec : V::zero();
                Raw avv[3];
#pragma unroll
                for (int c = 0; c < 3; c++)
                    avv[c] = prm.a[c] ? *reinterpret_cast<const Raw *>(static_cast<const char *>(prm.a[c]) +
                                                                      q * sizeof(RS)) : V::zero();
                from_bits(prm.b_uni, bs);
                float ia[3];
#pragma unroll
                for (int c = 0; c < 3; c++) {
                    from_bits(prm.a_uni[c], as[c]);
                    ia[c] = __frcp_rn(P::to_f32(as[c]));
                }
                const Raw vz_own = r2;
#pragma unroll
                for (int e = 0; e < N; e++) {
                    const float bw = prm.b ? V::f32(bv, e) : P::to_f32(bs);
                    float t = e_term(V::f32(pold, e), V::f32(pv, e), bw);
                    const Raw vc[3] = {vx, vy, vz_own};
#pragma unroll
                    for (int c = 0; c < 3; c++) {
                        const float vf = V::f32(vc[c], e);
                        t = __fadd_rn(t, prm.a[c] ? e_term(vf, vf, V::f32(avv[c], e))
                                                  : __fmul_rn(__fmul_rn(vf, vf), ia[c]));
                    }
                    acc.add(t);
                }
            }
        }
        r0 = r1;
        r1 = r2;
        r2 = r3;
        u0 = u1;
        u1 = u2;
        u2 = u3;
        buf ^= 1;
    }
    if (ENERGY) energy_reduce((double)acc.s + (double)acc.c, prm);
}

// ------------------------------------------------------------------------
template <class P, int COMP, int TY>
static cudaError_t launch_t(const AcParams &prm, int half_step, int zchunk, bool energy,
                            cudaStream_t st) {
    using V = typename VecOf<P>::T;
    constexpr int TX = TXV * V::N;
    dim3 grid((prm.n[0] + TX - 1) / TX, (prm.n[1] + TY - 1) / TY, (prm.n[2] + zchunk - 1) / zchunk);
    dim3 block(TXV * TY);
    if (half_step == 0) kv_stream<P, COMP, TY><<<grid, block, 0, st>>>(prm, zchunk);
    else if (energy) kp_stream<P, COMP, TY, true><<<grid, block, 0, st>>>(prm, zchunk);
    else kp_stream<P, COMP, TY, false><<<grid, block, 0, st>>>(prm, zchunk);
    return cudaGetLastError();
}

template <class P>
static cudaError_t launch_c(const AcParams &prm, int comp, int half_step, int zchunk, bool energy,
                            cudaStream_t st) {
    switch (comp) {
    case 0: return launch_t<P, 0, 16>(prm, half_step, zchunk, energy, st);
    case 3: return launch_t<P, 3, 16>(prm, half_step, zchunk, energy, st);
    default: return launch_t<P, 6, 16>(prm, half_step, zchunk, energy, st);
    }
}

int stream_vec_width(int prec) { return prec == PREC_FP32 ? 4 : 8; }

bool acoustic_stream_supported(const AcParams &prm, int ndim, int prec) {
    return ndim == 3 && prec != PREC_FP64 && prm.n[0] % stream_vec_width(prec) == 0 &&
           prm.n[2] >= 4;
}

unsigned acoustic_stream_blocks(const AcParams &prm, int prec, int zchunk) {
    const int tx = TXV * stream_vec_width(prec);
    return ((prm.n[0] + tx - 1) / tx) * ((prm.n[1] + 15) / 16) * ((prm.n[2] + zchunk - 1) / zchunk);
}

cudaError_t acoustic_stream_half_step(const AcParams &prm, int prec, int comp, int half_step,
                                      int zchunk, cudaStream_t st) {
    const bool energy = prm.energy != 0;
    switch (prec) {
    case PREC_FP32: return launch_c<F32>(prm, comp, half_step, zchunk, energy, st);
    case PREC_FP16: return launch_c<F16>(prm, comp, half_step, zchunk, energy, st);
    case PREC_BF16: return launch_c<BF16>(prm, comp, half_step, zchunk, energy, st);
    case PREC_FP16_F32ARITH: return launch_c<F16W>(prm, comp ? 3 : 0, half_step, zchunk, energy, st);
    case PREC_BF16_F32ARITH: return launch_c<BF16W>(prm, comp ? 3 : 0, half_step, zchunk, energy, st);
    case PREC_FP16_PAIRS:
        return comp ? launch_t<F16WP, 3, 16>(prm, half_step, zchunk, energy, st) : cudaErrorInvalidValue;
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace wave
