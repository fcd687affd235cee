// acoustic3d_fused.cu -- one-pass 3D acoustic leapfrog step with an
// asynchronous shared-memory pipeline.
//
// The step of Algorithm 1 / 2 (Section 4) extended to 3D,
//   v_c^{n+1/2} = v_c^{n-1/2} + a_c D_c(p^n)                 (c = x, y, z)
//   p^{n+1}     = p^n + b (Dx vx + Dy vy + Dz vz [+ s])       (v at n+1/2)
// is done in a single sweep: each CTA recomputes the new velocities it needs
// in a halo around its tile (x: 2 left, 1 right; y: 2 above, 1 below; z: the
// previous planes of its own columns), so p is updated without a second pass
// over the velocities. Every operation is the same, in the same order, as in
// the two-kernel path, so the results are bit-identical.
//
// Data movement: old state is read from one set of buffers and the new state
// written to the other (the context swaps them each step), because
// neighbouring CTAs read old values in their halos. A producer warp streams
// rows of the old state into two shared-memory rings with bulk asynchronous
// copies (cp.async.bulk, completion counted on mbarriers): a ring of p^n
// planes running three or more planes ahead (the z stencil of v_z needs
// planes k..k+3) and a ring of the other arrays of plane k. Four consumer
// warps compute. Every mbarrier wait is bounded; on expiry the kernel sets an
// error word and leaves.
//
// Layout of a CTA: TX x TY = (8 lanes x VEC) x 16 rows of (x, y) columns and a
// chunk of z planes; one 16-byte vector per consumer thread.
// Requirements (else the two-kernel path is used): 3D, n[0] a multiple of TX,
// uniform a_c (constant density).
#include <cuda_runtime.h>
#include "acoustic_common.cuh"
#include "wave_kernels.h"

namespace wave {

// -------------------------------------------------------------- PTX helpers
__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                 "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ void bulk_copy(void *dst_smem, const void *src_gmem, uint32_t bytes,
                                          uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst_smem)),
        "l"(src_gmem), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

// Bounded wait: about 2^22 polls (each poll may suspend briefly), then the
// error word is set and false returned. Once any block has set the error
// word, waits give up at their next check so that the whole grid leaves fast.
constexpr uint32_t kWaitPolls = 1u << 22;
__device__ __forceinline__ bool wait_phase(uint64_t *bar, uint32_t parity, int *err) {
    for (uint32_t it = 0; it < kWaitPolls; it++) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 1023u) == 1023u && *reinterpret_cast<volatile int *>(err)) return false;
    }
    atomicExch(err, 1);
    return false;
}

// Shorter bounded wait that ignores the error word (draining copies in flight).
__device__ __forceinline__ void drain_phase(uint64_t *bar, uint32_t parity) {
    for (uint32_t it = 0; it < (1u << 16); it++)
        if (mbar_try_wait(bar, parity)) return;
}

// ------------------------------------------------------------ the kernel
template <class P>
struct FusedShape {
    using S = typename P::S;
    static constexpr int VEC = 16 / sizeof(S);  // elements per 16-byte vector
    static constexpr int LANES = 8;             // consumer lanes per row
    static constexpr int TX = LANES * VEC;      // tile width (elements)
    static constexpr int TY = 16;               // tile rows
    static constexpr int HALO = VEC;            // x halo per side in the wide rows (16 bytes)
    static constexpr int WIDE = TX + 2 * HALO;
    static constexpr int SP = 6;                // p ring depth (planes)
    static constexpr int SO = 3;                // other-array ring depth
    // p plane: own rows wide, 3 halo rows above and below narrow
    static constexpr int P_ELEMS = TY * WIDE + 6 * TX;
    // other arrays of plane k: vx, tvx wide (own rows); vy, tvy rows y0-2..y0+TY;
    // vz, tvz (plane k+1), tp, b own
    static constexpr int O_VX = 0;
    static constexpr int O_TVX = O_VX + TY * WIDE;
    static constexpr int O_VY = O_TVX + TY * WIDE;
    static constexpr int O_TVY = O_VY + (TY + 3) * TX;
    static constexpr int O_VZ = O_TVY + (TY + 3) * TX;
    static constexpr int O_TVZ = O_VZ + TY * TX;
    static constexpr int O_TP = O_TVZ + TY * TX;
    static constexpr int O_B = O_TP + TY * TX;
    static constexpr int O_ELEMS = O_B + TY * TX;
    // new-velocity exchange buffers (double buffered): vx wide own rows, vy rows y0-2..y0+TY
    static constexpr int N_VX = 0;
    static constexpr int N_VY = TY * WIDE;
    static constexpr int N_ELEMS = N_VY + (TY + 3) * TX;
    static constexpr size_t SMEM =
        sizeof(S) * ((size_t)SP * P_ELEMS + (size_t)SO * O_ELEMS + 2 * (size_t)N_ELEMS) +
        sizeof(uint64_t) * (2 * (SP + SO) + 1) + 128;
};

struct FusedParams {
    AcParams a;            // n, bc, strides, coefficients, source, energy (p/v fields unused)
    const void *p_in, *vx_in, *vy_in, *vz_in, *tvx_in, *tvy_in, *tvz_in;
    void *p_out, *vx_out, *vy_out, *vz_out, *tvx_out, *tvy_out, *tvz_out;
    void *tp;              // in place
    int zchunk;
    int *err;              // set to 1 when a bounded wait expires
};

template <class P>
__device__ __forceinline__ typename P::A sgn_ld(typename P::S s, int sign) {
    if (sign == 0) return P::zero();
    typename P::A v = P::ld(s);
    return sign > 0 ? v : P::neg(v);
}

template <class P, int COMP, bool ENERGY>
__global__ void __launch_bounds__(160, 2) fused_step(FusedParams fp) {
    using SH = FusedShape<P>;
    using S = typename P::S;
    using A = typename P::A;
    constexpr int VEC = SH::VEC, TX = SH::TX, TY = SH::TY, WIDE = SH::WIDE, HALO = SH::HALO;
    constexpr int SP = SH::SP, SO = SH::SO;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    S *pring = reinterpret_cast<S *>(smem_raw);
    S *oring = pring + SP * SH::P_ELEMS;
    S *nbuf = oring + SO * SH::O_ELEMS;
    uint64_t *bars = reinterpret_cast<uint64_t *>(nbuf + 2 * SH::N_ELEMS);
    uint64_t *p_full = bars, *p_empty = bars + SP, *o_full = bars + 2 * SP, *o_empty = bars + 2 * SP + SO;
    // barrier of the four consumer warps (an mbarrier, so that its waits are bounded too)
    uint64_t *c_bar = bars + 2 * (SP + SO);

    const AcParams &prm = fp.a;
    const int nx = prm.n[0], ny = prm.n[1], nz = prm.n[2];
    const int bcx = prm.bc[0], bcy = prm.bc[1], bcz = prm.bc[2];
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int z0 = blockIdx.z * fp.zchunk;
    const int z1 = min(z0 + fp.zchunk, nz);
    const int tid = threadIdx.x;
    const int warp = tid >> 5;

    if (tid == 0) {
        for (int s = 0; s < SP; s++) { mbar_init(&p_full[s], 1); mbar_init(&p_empty[s], 4); }
        for (int s = 0; s < SO; s++) { mbar_init(&o_full[s], 1); mbar_init(&o_empty[s], 4); }
        mbar_init(c_bar, 128);
        mbar_fence_init();
    }
    __syncthreads();

    const int64_t sy = prm.sy, sz = prm.sz;
    const int eb = sizeof(S);

    if (warp == 4) {
        // ================================================= producer warp
        const int lane = tid & 31;
        // mapped global row start (element index) for field kind along y/z;
        // wall rows (sign 0) copy row 0 of plane 0 (any valid memory).
        auto row_src = [&](int my, int mz, bool node_y, bool node_z) -> int64_t {
            // rows and planes farther than two past the grid are never read by
            // the consumers (and one reflection does not reach them): copy row 0
            if (my < -3 || my > ny + 2 || mz < -3 || mz > nz + 2) return 0;
            int jy, kz;
            int s1 = node_y ? img_node(my, ny, bcy, jy) : img_half(my, ny, bcy, jy);
            int s2 = node_z ? img_node(mz, nz, bcz, kz) : img_half(mz, nz, bcz, kz);
            if (s1 == 0 || s2 == 0) return 0;
            return sy * jy + sz * (int64_t)kz;
        };
        // Issue the copies of one wide row: the own part [x0, x0+TX) plus the
        // 16-byte halo blocks left and right when they are inside the grid or
        // wrap around it (periodic). Returns bytes issued.
        auto wide_row = [&](S *dst, const S *base, int64_t rowoff, uint64_t *bar, bool issue) -> uint32_t {
            uint32_t bytes = TX * eb;
            if (issue) bulk_copy(dst + HALO, base + rowoff + x0, TX * eb, bar);
            int lx0 = x0 - HALO;
            if (lx0 >= 0 || bcx == BC_PERIODIC) {
                int src = lx0 >= 0 ? lx0 : lx0 + nx;
                if (issue) bulk_copy(dst, base + rowoff + src, HALO * eb, bar);
                bytes += HALO * eb;
            }
            int rx0 = x0 + TX;
            if (rx0 < nx || bcx == BC_PERIODIC) {
                int src = rx0 < nx ? rx0 : rx0 - nx;
                if (issue) bulk_copy(dst + HALO + TX, base + rowoff + src, HALO * eb, bar);
                bytes += HALO * eb;
            }
            return bytes;
        };
        // Work items of one p plane m: TY wide own rows + 6 narrow halo rows.
        auto p_plane = [&](int m, S *dst, uint64_t *bar, bool issue, int part) -> uint32_t {
            const S *pin = static_cast<const S *>(fp.p_in);
            uint32_t bytes = 0;
            for (int r = part; r < TY + 6; r += 32) {
                if (r < TY) {
                    int my = y0 + r;
                    bytes += wide_row(dst + r * WIDE, pin, row_src(my, m, true, true), bar, issue);
                } else {
                    int h = r - TY;  // 0..5 -> rows y0-3, y0-2, y0-1, y0+TY, y0+TY+1, y0+TY+2
                    int my = h < 3 ? y0 - 3 + h : y0 + TY + (h - 3);
                    if (issue) bulk_copy(dst + TY * WIDE + h * TX, pin + row_src(my, m, true, true) + x0,
                                         TX * eb, bar);
                    bytes += TX * eb;
                }
            }
            return bytes;
        };
        auto o_stage = [&](int k, S *dst, uint64_t *bar, bool issue, int part) -> uint32_t {
            uint32_t bytes = 0;
            const bool full_set = k >= z0;
            // rows: 0..TY-1 vx, TY..2TY-1 tvx, then 19 vy, 19 tvy, then TY each vz, tvz, tp, b
            const int nrows = full_set ? (2 * TY + 2 * (TY + 3) + 4 * TY) : 2 * TY;
            for (int r = part; r < nrows; r += 32) {
                if (!full_set) {
                    // warm-up planes: only vz, tvz of plane k+1
                    const bool is_t = r >= TY;
                    const int rr = is_t ? r - TY : r;
                    if (is_t && !COMP) continue;
                    const S *src = static_cast<const S *>(is_t ? fp.tvz_in : fp.vz_in);
                    S *d = dst + (is_t ? SH::O_TVZ : SH::O_VZ) + rr * TX;
                    if (issue) bulk_copy(d, src + row_src(y0 + rr, k + 1, true, false) + x0, TX * eb, bar);
                    bytes += TX * eb;
                    continue;
                }
                int rr = r;
                if (rr < 2 * TY) {
                    const bool is_t = rr >= TY;
                    if (is_t && !COMP) continue;
                    const int row = is_t ? rr - TY : rr;
                    const S *src = static_cast<const S *>(is_t ? fp.tvx_in : fp.vx_in);
                    bytes += wide_row(dst + (is_t ? SH::O_TVX : SH::O_VX) + row * WIDE, src,
                                      row_src(y0 + row, k, true, true), bar, issue);
                    continue;
                }
                rr -= 2 * TY;
                if (rr < 2 * (TY + 3)) {
                    const bool is_t = rr >= TY + 3;
                    if (is_t && !COMP) continue;
                    const int row = is_t ? rr - (TY + 3) : rr;   // row 0 <-> y0 - 2
                    const S *src = static_cast<const S *>(is_t ? fp.tvy_in : fp.vy_in);
                    S *d = dst + (is_t ? SH::O_TVY : SH::O_VY) + row * TX;
                    if (issue) bulk_copy(d, src + row_src(y0 - 2 + row, k, false, true) + x0, TX * eb, bar);
                    bytes += TX * eb;
                    continue;
                }
                rr -= 2 * (TY + 3);
                const int which = rr / TY, row = rr % TY;  // 0 vz, 1 tvz, 2 tp, 3 b
                if (which == 1 && !COMP) continue;
                if (which == 2 && !COMP) continue;
                if (which == 3 && !prm.b) continue;
                const S *src = which == 0 ? static_cast<const S *>(fp.vz_in)
                             : which == 1 ? static_cast<const S *>(fp.tvz_in)
                             : which == 2 ? static_cast<const S *>(fp.tp)
                                          : static_cast<const S *>(prm.b);
                const int off = which == 0 ? SH::O_VZ : which == 1 ? SH::O_TVZ : which == 2 ? SH::O_TP : SH::O_B;
                const int64_t ro = which <= 1 ? row_src(y0 + row, k + 1, true, false)
                                              : row_src(y0 + row, k, true, true);
                if (issue) bulk_copy(dst + off + row * TX, src + ro + x0, TX * eb, bar);
                bytes += TX * eb;
            }
            return bytes;
        };
        auto issue_p = [&](int m, int cnt) -> bool {
            const int slot = cnt % SP;
            if (cnt >= SP && !wait_phase(&p_empty[slot], ((cnt / SP) - 1) & 1, fp.err)) return false;
            S *dst = pring + slot * SH::P_ELEMS;
            uint32_t total = 0;
            for (int part = 0; part < 32; part++) total += p_plane(m, dst, nullptr, false, part);
            if (lane == 0) mbar_expect_tx(&p_full[slot], total);
            __syncwarp();
            p_plane(m, dst, &p_full[slot], true, lane);
            return true;
        };
        auto issue_o = [&](int k, int cnt) -> bool {
            const int slot = cnt % SO;
            if (cnt >= SO && !wait_phase(&o_empty[slot], ((cnt / SO) - 1) & 1, fp.err)) return false;
            S *dst = oring + slot * SH::O_ELEMS;
            uint32_t total = 0;
            for (int part = 0; part < 32; part++) total += o_stage(k, dst, nullptr, false, part);
            if (lane == 0) mbar_expect_tx(&o_full[slot], total);
            __syncwarp();
            o_stage(k, dst, &o_full[slot], true, lane);
            return true;
        };
        int pc = 0, oc = 0;
        bool ok = true;
        for (int m = z0 - 3; m <= z1 + 2 && ok; m++) {
            ok = issue_p(m, pc++);
            if (ok && m >= z0) ok = issue_o(m - 3, oc++);
        }
        // before leaving, let the copies this warp issued land (bounded)
        if (lane == 0) {
            for (int c = (pc > SP ? pc - SP : 0); c < pc; c++) drain_phase(&p_full[c % SP], (c / SP) & 1);
            for (int c = (oc > SO ? oc - SO : 0); c < oc; c++) drain_phase(&o_full[c % SO], (c / SO) & 1);
        }
        return;
    }

    // ===================================================== consumer warps
    const int lx = tid % SH::LANES, row = tid / SH::LANES;
    const int x = x0 + lx * VEC;
    const int j = y0 + row;
    const bool active = j < ny;  // n[0] is a multiple of TX
    A a_uni[3];
#pragma unroll
    for (int c = 0; c < 3; c++) {
        S s;
        from_bits(prm.a_uni[c], s);
        a_uni[c] = P::ld(s);
    }
    S b_s;
    from_bits(prm.b_uni, b_s);

    // v_z^{n+1/2} of the own vector, planes k-2, k-1, k, k+1 (ring of 4)
    A vzq[4][VEC];
    float e_s = 0.f, e_c = 0.f;
    auto eadd = [&](float x_) {
        const float t = __fadd_rn(e_s, x_);
        const float pa = __fsub_rn(t, x_);
        const float pb = __fsub_rn(t, pa);
        e_c = __fadd_rn(e_c, __fadd_rn(__fsub_rn(e_s, pa), __fsub_rn(x_, pb)));
        e_s = t;
    };

    // p sample of plane slot at local row lr (-3..TY+2) and column x (global)
    auto p_row_ptr = [&](const S *pst, int lr) -> const S * {
        if (lr >= 0 && lr < TY) return pst + lr * WIDE + HALO - x0;  // index by global x
        const int h = lr < 0 ? lr + 3 : 3 + (lr - TY);
        return pst + TY * WIDE + h * TX - x0;
    };
    // sign of the image for the p row my in plane m (node type in y and z)
    auto p_sign = [&](int my, int m) -> int {
        int t1, t2;
        return img_node(my, ny, bcy, t1) * img_node(m, nz, bcz, t2);
    };
    // x image for a value of a wide row of a node-type (p) or half-type (vx) field
    auto x_img = [&](int mx, bool node, int &sgn) -> int {
        if (mx >= 0 && mx < nx) { sgn = 1; return mx; }
        if (bcx == BC_PERIODIC) { sgn = 1; return mx; }  // halo block holds the wrapped values
        int out;
        sgn = node ? img_node(mx, nx, bcx, out) : img_half(mx, nx, bcx, out);
        return out;
    };

    int pc = 0, oc = 0, nb = 0;
    bool ok = true;
    uint32_t c_phase = 0;
    auto consumer_sync = [&]() -> bool {
        mbar_arrive(c_bar);
        const bool r = wait_phase(c_bar, c_phase & 1, fp.err);
        c_phase++;
        return r;
    };
    // p planes waited so far (the consumer waits for plane m when first needed)
    int p_waited = 0;
    auto wait_p_upto = [&](int cnt_needed) -> bool {
        while (p_waited < cnt_needed) {
            if (!wait_phase(&p_full[p_waited % SP], (p_waited / SP) & 1, fp.err)) return false;
            p_waited++;
        }
        return true;
    };

    for (int k = z0 - 3; k < z1 && ok; k++) {
        // planes k..k+3 of p: ring counts (k - (z0-3)) .. +3
        const int pbase = k - (z0 - 3);
        if (!wait_p_upto(pbase + 4)) { ok = false; break; }
        const int oslot = oc % SO;
        if (!wait_phase(&o_full[oslot], (oc / SO) & 1, fp.err)) { ok = false; break; }
        const S *ost = oring + oslot * SH::O_ELEMS;
        const S *pst[4];
        for (int t = 0; t < 4; t++) pst[t] = pring + ((pbase + t) % SP) * SH::P_ELEMS;

        // ---- v_z^{n+1/2} at plane k+1 for the own vector (from p^n planes k..k+3)
        if (active) {
            int sg[4];
#pragma unroll
            for (int t = 0; t < 4; t++) sg[t] = p_sign(j, k + t);
            const S *vzrow = ost + SH::O_VZ + row * TX + lx * VEC;
            const S *tzrow = ost + SH::O_TVZ + row * TX + lx * VEC;
            const int64_t qz = x + sy * j + sz * (int64_t)(k + 1);
            const bool write_vz = (k + 1 >= z0) && (k + 1 < z1);
            S vn[VEC], tn[VEC];
#pragma unroll
            for (int e = 0; e < VEC; e++) {
                A f[4];
#pragma unroll
                for (int t = 0; t < 4; t++) f[t] = sgn_ld<P>(p_row_ptr(pst[t], row)[x + e], sg[t]);
                const A D = stencil<P>(f[0], f[1], f[2], f[3]);
                const A inc = P::mul(a_uni[2], D);
                // the v_z image along z is even: same stored values at the mapped plane
                S V = vzrow[e];
                S T = COMP ? tzrow[e] : S(0);
                update<P, COMP>(V, T, inc);
                vn[e] = V;
                tn[e] = T;
                vzq[3][e] = P::ld(V);
            }
            if (write_vz) {
                S *vo = static_cast<S *>(fp.vz_out) + qz;
                S *to = static_cast<S *>(fp.tvz_out) + qz;
#pragma unroll
                for (int e = 0; e < VEC; e++) {
                    vo[e] = vn[e];
                    if (COMP) to[e] = tn[e];
                }
            }
        }

        if (k >= z0) {
            S *nvx = nbuf + nb * SH::N_ELEMS + SH::N_VX;
            S *nvy = nbuf + nb * SH::N_ELEMS + SH::N_VY;
            S vxn[VEC], txn[VEC], vyn[VEC], tyn[VEC];
            // ---- v_x^{n+1/2} at own points and the x halo (lane 0: x0-2, x0-1;
            //      last lane: x0+TX), from p^n plane k of the own row
            if (active) {
                const S *prow = p_row_ptr(pst[0], row);
                const int sgr = p_sign(j, k);
                const S *vxr = ost + SH::O_VX + row * WIDE + HALO - x0;
                const S *txr = ost + SH::O_TVX + row * WIDE + HALO - x0;
                auto pval = [&](int mx) -> A {
                    int s2;
                    const int ix = x_img(mx, true, s2);
                    if (s2 == 0) return P::zero();  // the wall node itself: not read
                    return sgn_ld<P>(prow[ix], s2 * sgr);
                };
                auto vx_at = [&](int ix, S &V, S &T) {
                    // v_x at ix + 1/2 from p at ix-1..ix+2; v_x and t_vx read with the
                    // even x image (half-type field)
                    const A D = stencil<P>(pval(ix - 1), pval(ix), pval(ix + 1), pval(ix + 2));
                    const A inc = P::mul(a_uni[0], D);
                    int s2;
                    const int iv = x_img(ix, false, s2);
                    V = vxr[iv];
                    T = COMP ? txr[iv] : S(0);
                    update<P, COMP>(V, T, inc);
                };
#pragma unroll
                for (int e = 0; e < VEC; e++) vx_at(x + e, vxn[e], txn[e]);
                S *nrow = nvx + row * WIDE + HALO - x0;
#pragma unroll
                for (int e = 0; e < VEC; e++) nrow[x + e] = vxn[e];
                if (lx == 0) {
                    S V, T;
                    vx_at(x0 - 2, V, T);
                    nrow[x0 - 2] = V;
                    vx_at(x0 - 1, V, T);
                    nrow[x0 - 1] = V;
                }
                if (lx == SH::LANES - 1) {
                    S V, T;
                    vx_at(x0 + TX, V, T);
                    nrow[x0 + TX] = V;
                }
            }
            // ---- v_y^{n+1/2} at own rows and the halo rows y0-2, y0-1, y0+TY
            auto vy_at = [&](int lr /* local row of the v_y point, -2..TY */, S *V, S *T) {
                const int my = y0 + lr;
                int sg[4];
                const S *pr[4];
#pragma unroll
                for (int t = 0; t < 4; t++) {
                    pr[t] = p_row_ptr(pst[0], lr - 1 + t);
                    sg[t] = p_sign(my - 1 + t, k);
                }
                const S *vyr = ost + SH::O_VY + (lr + 2) * TX - x0;
                const S *tyr = ost + SH::O_TVY + (lr + 2) * TX - x0;
#pragma unroll
                for (int e = 0; e < VEC; e++) {
                    const A D = stencil<P>(sgn_ld<P>(pr[0][x + e], sg[0]), sgn_ld<P>(pr[1][x + e], sg[1]),
                                           sgn_ld<P>(pr[2][x + e], sg[2]), sgn_ld<P>(pr[3][x + e], sg[3]));
                    const A inc = P::mul(a_uni[1], D);
                    S Vv = vyr[x + e];
                    S Tv = COMP ? tyr[x + e] : S(0);
                    update<P, COMP>(Vv, Tv, inc);
                    V[e] = Vv;
                    T[e] = Tv;
                }
            };
            // own rows, and the first row past the grid (row ny, the image row
            // that the last grid row's stencil reads)
            if (j <= ny) {
                vy_at(row, vyn, tyn);
                S *nr = nvy + (row + 2) * TX - x0;
#pragma unroll
                for (int e = 0; e < VEC; e++) nr[x + e] = vyn[e];
            }
            if (tid < 3 * SH::LANES) {
                // halo rows: local -2, -1, TY (the images of rows outside the grid
                // come out right because the inputs are read with their images)
                const int hr = tid / SH::LANES;
                const int lr = hr == 0 ? -2 : hr == 1 ? -1 : TY;
                if (y0 + lr < ny + 2) {
                    S V[VEC], T[VEC];
                    vy_at(lr, V, T);
                    S *nr = nvy + (lr + 2) * TX - x0;
#pragma unroll
                    for (int e = 0; e < VEC; e++) nr[x + e] = V[e];
                }
            }
            if (!consumer_sync()) { ok = false; break; }
            // ---- p^{n+1}
            if (active) {
                const S *vxr = nvx + row * WIDE + HALO - x0;
                const S *tpr = ost + SH::O_TP + row * TX - x0;
                const S *br = ost + SH::O_B + row * TX - x0;
                const S *prow = p_row_ptr(pst[0], row);
                const int sgr = p_sign(j, k);
                const int64_t q = x + sy * j + sz * (int64_t)k;
                S pn[VEC], tpn[VEC];
#pragma unroll
                for (int e = 0; e < VEC; e++) {
                    const int i = x + e;
                    // node i reads v_x at i-2, i-1, i, i+1 (+1/2); outside the grid the
                    // even image (rigid) or the wrapped halo (periodic)
                    // v_x^{n+1/2} at i-2 .. i+1 (+1/2): own values and the halo values
                    // computed above (outside the grid they were computed from the
                    // images of their inputs, which reproduces the images of v_x)
                    A R = stencil<P>(P::ld(vxr[i - 2]), P::ld(vxr[i - 1]), P::ld(vxr[i]),
                                     P::ld(vxr[i + 1]));
                    const S *vyc = nvy - x0 + i;
                    const A Dy = stencil<P>(P::ld(vyc[(row) * TX]), P::ld(vyc[(row + 1) * TX]),
                                            P::ld(vyc[(row + 2) * TX]), P::ld(vyc[(row + 3) * TX]));
                    R = P::add(R, Dy);
                    const A Dz = stencil<P>(vzq[0][e], vzq[1][e], vzq[2][e], vzq[3][e]);
                    R = P::add(R, Dz);
                    if (k == prm.src_k && j == prm.src_j && i == prm.src_i && prm.step < prm.src_nt)
                        R = P::add(R, static_cast<const A *>(prm.src)[prm.step]);
                    const S bq = prm.b ? br[i] : b_s;
                    const A inc = P::mul(P::ld(bq), R);
                    const S pold = (sgr == 0) ? S(0) : prow[i];
                    S V = pold;
                    S T = COMP ? tpr[i] : S(0);
                    update<P, COMP>(V, T, inc);
                    pn[e] = V;
                    tpn[e] = T;
                    if (ENERGY) {
                        eadd(e_term(P::to_f32(pold), P::to_f32(V), P::to_f32(bq)));
                        const float fx = P::to_f32(vxn[e]), fy = P::to_f32(vyn[e]);
                        eadd(e_term(fx, fx, P::to_f32(P::st(a_uni[0]))));
                        eadd(e_term(fy, fy, P::to_f32(P::st(a_uni[1]))));
                    }
                }
                // stores: p, t_p (in place), v_x, t_vx, v_y, t_vy of plane k
                S *po = static_cast<S *>(fp.p_out) + q;
                S *to = static_cast<S *>(fp.tp) + q;
                S *vxo = static_cast<S *>(fp.vx_out) + q;
                S *txo = static_cast<S *>(fp.tvx_out) + q;
                S *vyo = static_cast<S *>(fp.vy_out) + q;
                S *tyo = static_cast<S *>(fp.tvy_out) + q;
#pragma unroll
                for (int e = 0; e < VEC; e++) {
                    po[e] = pn[e];
                    vxo[e] = vxn[e];
                    vyo[e] = vyn[e];
                    if (COMP) {
                        to[e] = tpn[e];
                        txo[e] = txn[e];
                        tyo[e] = tyn[e];
                    }
                }
                if (ENERGY) {
#pragma unroll
                    for (int e = 0; e < VEC; e++) {
                        const float fz = P::to_f32(P::st(vzq[2][e]));
                        eadd(e_term(fz, fz, P::to_f32(P::st(a_uni[2]))));
                    }
                }
            }
            nb ^= 1;
        }
        // release the stages this iteration consumed: the other arrays of k, p plane k
        __syncwarp();
        if ((tid & 31) == 0) {
            mbar_arrive(&o_empty[oslot]);
            mbar_arrive(&p_empty[pbase % SP]);
        }
        oc++;
        // shift the v_z queue
#pragma unroll
        for (int t = 0; t < 3; t++)
#pragma unroll
            for (int e = 0; e < VEC; e++) vzq[t][e] = vzq[t + 1][e];
    }
    (void)pc;
    if (ENERGY) {
        // every consumer thread of every block takes part in the reduction;
        // the producer warp has left, so reduce over the consumer warps only
        double val = ok ? (double)e_s + (double)e_c : 0.0;
        for (int off = 16; off > 0; off >>= 1) val += __shfl_down_sync(0xffffffffu, val, off);
        __shared__ double wsum[4];
        __shared__ bool last;
        if ((tid & 31) == 0) wsum[warp] = val;
        if (!consumer_sync()) return;
        const unsigned nblocks = gridDim.x * gridDim.y * gridDim.z;
        const unsigned bid = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
        if (tid == 0) {
            prm.e_part[bid] = wsum[0] + wsum[1] + wsum[2] + wsum[3];
            __threadfence();
            last = atomicAdd(prm.e_count, 1u) == nblocks - 1;
        }
        if (!consumer_sync()) return;
        if (last) {
            __threadfence();
            double s = 0.0;
            for (unsigned b = tid; b < nblocks; b += 128) s += __ldcg(&prm.e_part[b]);
            for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
            if (!consumer_sync()) return;
            if ((tid & 31) == 0) wsum[warp] = s;
            if (!consumer_sync()) return;
            if (tid == 0) {
                *prm.e_out = (wsum[0] + wsum[1] + wsum[2] + wsum[3]) * prm.e_factor;
                *prm.e_count = 0u;
            }
        }
    }
}

// ------------------------------------------------------------------------
template <class P, int COMP>
static cudaError_t launch_t(const FusedParams &fp, bool energy, cudaStream_t st) {
    using SH = FusedShape<P>;
    dim3 grid(fp.a.n[0] / SH::TX, (fp.a.n[1] + SH::TY - 1) / SH::TY,
              (fp.a.n[2] + fp.zchunk - 1) / fp.zchunk);
    const size_t smem = SH::SMEM;
    cudaError_t e;
    if (energy) {
        e = cudaFuncSetAttribute(fused_step<P, COMP, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        fused_step<P, COMP, true><<<grid, 160, smem, st>>>(fp);
    } else {
        e = cudaFuncSetAttribute(fused_step<P, COMP, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        fused_step<P, COMP, false><<<grid, 160, smem, st>>>(fp);
    }
    return cudaGetLastError();
}

template <class P>
static cudaError_t launch_c(const FusedParams &fp, int comp, bool energy, cudaStream_t st) {
    switch (comp) {
    case 0: return launch_t<P, 0>(fp, energy, st);
    case 3: return launch_t<P, 3>(fp, energy, st);
    default: return launch_t<P, 6>(fp, energy, st);
    }
}

int fused_tile_x(int prec) { return prec == PREC_FP32 ? 32 : 64; }

bool acoustic_fused_supported(const AcParams &prm, int ndim, int prec) {
    if (ndim != 3 || prec == PREC_FP64) return false;
    if (prm.n[0] % fused_tile_x(prec) != 0 || prm.n[1] < 8 || prm.n[2] < 8) return false;
    return prm.a[0] == nullptr && prm.a[1] == nullptr && prm.a[2] == nullptr;
}

unsigned acoustic_fused_blocks(const AcParams &prm, int prec, int zchunk) {
    return (prm.n[0] / fused_tile_x(prec)) * ((prm.n[1] + 15) / 16) * ((prm.n[2] + zchunk - 1) / zchunk);
}

cudaError_t acoustic_fused_step(const AcParams &prm, const void *const in[7], void *const out[7],
                                void *tp, int prec, int comp, int zchunk, int *err, cudaStream_t st) {
    FusedParams fp;
    fp.a = prm;
    fp.p_in = in[0]; fp.vx_in = in[1]; fp.vy_in = in[2]; fp.vz_in = in[3];
    fp.tvx_in = in[4]; fp.tvy_in = in[5]; fp.tvz_in = in[6];
    fp.p_out = out[0]; fp.vx_out = out[1]; fp.vy_out = out[2]; fp.vz_out = out[3];
    fp.tvx_out = out[4]; fp.tvy_out = out[5]; fp.tvz_out = out[6];
    fp.tp = tp;
    fp.zchunk = zchunk;
    fp.err = err;
    const bool energy = prm.energy != 0;
    switch (prec) {
    case PREC_FP32: return launch_c<F32>(fp, comp, energy, st);
    case PREC_FP16: return launch_c<F16>(fp, comp, energy, st);
    case PREC_BF16: return launch_c<BF16>(fp, comp, energy, st);
    case PREC_FP16_F32ARITH: return launch_c<F16W>(fp, comp ? 3 : 0, energy, st);
    case PREC_BF16_F32ARITH: return launch_c<BF16W>(fp, comp ? 3 : 0, energy, st);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace wave
