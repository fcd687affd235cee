// acoustic3d_fused.cu -- one-pass 3D acoustic leapfrog step with a TMA
// shared-memory pipeline.
//
// The step of Algorithm 1 / 2 (Section 4) extended to 3D,
//   v_c^{n+1/2} = v_c^{n-1/2} + a_c D_c(p^n)                 (c = x, y, z)
//   p^{n+1}     = p^n + b (Dx vx + Dy vy + Dz vz [+ s])       (v at n+1/2)
// in a single sweep: each CTA recomputes the new velocities it needs in a halo
// around its tile (x: 2 left, 1 right; y: 2 above, 1 below; z: the previous
// planes of its own columns), so p is updated without a second pass over the
// velocities. Every operation is the same, in the same order, as in the
// two-kernel path, so the results are bit-identical.
//
// Data movement: the old state is read from one set of buffers and the new
// state written to the other (the context swaps them after each step),
// because neighbouring CTAs read old values in their halos. A producer warp
// streams tiles of the old state into two shared-memory rings with tensor
// TMA copies (cp.async.bulk.tensor, one box per array and plane; completion
// counted on mbarriers): a ring of p^n planes running ahead of the compute
// (the z stencil of v_z needs planes k..k+3) and a ring of the other arrays of
// plane k. With rigid y walls the boxes are used at the y faces too: the rows
// past a face are filled with zeros and the consumers read the mirror rows,
// which lie inside the tile, with the image's sign. With periodic y walls the
// row groups that cross a face are copied row by row (bulk copies) from the
// wrapped rows. (Row-by-row copies made the face tiles 4x slower than the
// interior ones.) Four consumer warps
// compute on 16-byte vectors with packed-pair arithmetic; each warp owns four
// rows of the tile and recomputes the v_y rows it needs from its neighbours
// (two above, one below), so the new velocities are exchanged only inside a
// warp (__syncwarp) and the warps never wait for each other. t_p and b are
// read by each thread from global memory. Every mbarrier wait is bounded; on
// expiry the kernel sets an error word and leaves.
//
// Tile: TX x TY = (8 lanes x VEC) x 16 rows of (x, y) columns, a chunk of z
// planes. Requirements (else the two-kernel path is used): 3D, n[0] a multiple
// of TX, rigid x faces, uniform a_c (constant density).
#include <cuda.h>
#include <cuda_runtime.h>
#include <string.h>

#include "acoustic_common.cuh"
#include "fused_common.cuh"
#include "vec_policy.cuh"
#include "wave_kernels.h"

namespace wave {

// ------------------------------------------------------------ the layout
template <class P>
struct FShape {
    using S = typename P::S;
    // the pair precision: every p slot also holds the t_p tile (at P_ELEMS),
    // and the exchange buffers hold the new velocities' T beside them (at
    // N_ELEMS); the stencil taps are RN32(V + T)
    static constexpr bool PAIRS = IsPairs<P>::value;
    static constexpr int VEC = 16 / sizeof(S);
    static constexpr int LANES = 8;
    static constexpr int TX = LANES * VEC;
    static constexpr int TY = 16;
    static constexpr int HALO = VEC;              // 16-byte x halo blocks of the wide rows
    static constexpr int WIDE = TX + 2 * HALO;
    static constexpr int SP = 5;                  // p ring depth (planes k..k+3 and one ahead)
    static constexpr int SO = 2;                  // other-array ring depth (one ahead)
    // p plane: TY wide own rows, 3 narrow halo rows above, 3 below
    static constexpr int P_HALO = TY * WIDE;
    static constexpr int P_ELEMS = TY * WIDE + 6 * TX;
    // other arrays: vx, tvx wide own rows; vy, tvy rows y0-2..y0+TY; vz, tvz
    // (plane k+1). Every region starts on a 128-byte boundary. (t_p and b are
    // read by the consumers straight from global memory: each thread needs only
    // its own vector, and leaving them out of the ring lets four CTAs share an
    // SM.)
    static constexpr int O_VX = 0;
    static constexpr int O_TVX = O_VX + TY * WIDE;
    static constexpr int O_VY = O_TVX + TY * WIDE;
    static constexpr int O_TVY = O_VY + (TY + 3) * TX;
    static constexpr int O_VZ = O_TVY + (TY + 3) * TX;
    static constexpr int O_TVZ = O_VZ + TY * TX;
    static constexpr int O_ELEMS = O_TVZ + TY * TX;
    // new-velocity exchange: vx wide rows of the tile (each warp writes and
    // reads only its own rows), then two buffers (alternate planes) of the
    // tile's new v_y rows -2 .. TY, shared by the four consumer warps (one
    // bounded CTA sync per plane between writing and reading them)
    static constexpr int N_VY = TY * WIDE;
    static constexpr int N_YROWS = TY + 3;
    static constexpr int N_ELEMS = N_VY + 2 * N_YROWS * TX;
    static constexpr int P_SLOT = PAIRS ? 2 * P_ELEMS : P_ELEMS;
    static constexpr int N_TOT = PAIRS ? 2 * N_ELEMS : N_ELEMS;
    static constexpr size_t RING_BYTES =
        sizeof(S) * ((size_t)SP * P_SLOT + (size_t)SO * O_ELEMS + (size_t)N_TOT);
    static constexpr size_t SMEM = RING_BYTES + sizeof(uint64_t) * (2 * (SP + SO) + 2) + 128;
    static_assert((P_ELEMS * sizeof(S)) % 128 == 0 && (O_ELEMS * sizeof(S)) % 128 == 0 &&
                      (N_ELEMS * sizeof(S)) % 128 == 0 && (O_VY * sizeof(S)) % 128 == 0 &&
                      (O_TVY * sizeof(S)) % 128 == 0 && (O_VZ * sizeof(S)) % 128 == 0 &&
                      (P_HALO * sizeof(S)) % 128 == 0 && ((P_HALO + 3 * TX) * sizeof(S)) % 128 == 0,
                  "TMA destinations must be 128-byte aligned");
};

template <class P, int COMP, bool ENERGY>
// (the pair kernel: three CTAs per SM at 128 registers; its energy variant,
// launched on a call's last step, two, to stay free of spills)
__global__ void __launch_bounds__(160, IsPairs<P>::value ? (ENERGY ? 2 : 3) : 4)
    fused_step(const __grid_constant__ FusedParams fp, const __grid_constant__ FusedMaps maps) {
    using SH = FShape<P>;
    constexpr bool PAIRS = SH::PAIRS;
    using S = typename P::S;
    using V = typename VecOf<P>::T;
    using Raw = typename V::Raw;
    using AV = typename V::AV;
    using RS = typename V::RS;
    constexpr int VEC = SH::VEC, TX = SH::TX, TY = SH::TY, WIDE = SH::WIDE, HALO = SH::HALO;
    constexpr int SP = SH::SP, SO = SH::SO;
    static_assert(V::N == VEC, "vector width");
    extern __shared__ unsigned char smem_raw[];
    unsigned char *base = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~static_cast<uintptr_t>(127));
    S *pring = reinterpret_cast<S *>(base);
    S *oring = pring + SP * SH::P_SLOT;
    S *nbuf = oring + SO * SH::O_ELEMS;
    uint64_t *bars = reinterpret_cast<uint64_t *>(base + SH::RING_BYTES);
    uint64_t *p_full = bars, *p_empty = bars + SP, *o_full = bars + 2 * SP, *o_empty = bars + 2 * SP + SO;
    uint64_t *c_bar = bars + 2 * (SP + SO);
    // v_y rows of a plane complete: the four consumer warps' own rows and the
    // producer warp's halo rows (160 arrivals per plane)
    uint64_t *v_bar = bars + 2 * (SP + SO) + 1;

    const AcParams &prm = fp.a;
    const int nx = prm.n[0], ny = prm.n[1], nz = prm.n[2];
    const int bcy = prm.bc[1], bcz = prm.bc[2];
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int z0 = blockIdx.z * fp.zchunk;
    const int z1 = min(z0 + fp.zchunk, nz);
    const int tid = threadIdx.x;
    const int warp = tid >> 5;
    const int64_t sy = prm.sy, sz = prm.sz;
    constexpr int eb = sizeof(S);

    if (tid == 0) {
        for (int s = 0; s < SP; s++) { mbar_init(&p_full[s], 1); mbar_init(&p_empty[s], 4); }
        for (int s = 0; s < SO; s++) { mbar_init(&o_full[s], 1); mbar_init(&o_empty[s], 4); }
        mbar_init(c_bar, 128);
        mbar_init(v_bar, 160);
        mbar_fence_init();
    }
    __syncthreads();

    // uniform multipliers in their storage (CoefOf: binary32 for the pairs)
    using CS = typename CoefOf<P>::S;
    CS a_raw[3], b_raw;
#pragma unroll
    for (int c = 0; c < 3; c++) from_bits(prm.a_uni[c], a_raw[c]);
    from_bits(prm.b_uni, b_raw);
    const AV ay = V::splat(CoefOf<P>::ld(a_raw[1]));
    // a stencil tap: the stored value, or RN(V + T) for the pairs
    auto tap = [&](const Raw &v, const Raw &t) -> AV { return PAIRS ? V::add(V::ld(v), V::ld(t)) : V::ld(v); };
    auto tap_s = [&](RS v, RS t) -> typename V::AS { return PAIRS ? P::add(V::lds(v), V::lds(t)) : V::lds(v); };
    // tiles whose p rows y0-3..y0+TY+2 are all inside the grid read no images in y
    const bool inner_y = y0 >= 3 && y0 + TY + 3 <= ny;
    // rigid y walls: rows past the y faces were loaded as zeros; the images are
    // read from the mirror rows, which lie inside the tile's rows (p: odd
    // about the wall nodes 0 and ny, the wall row itself zero; v_y: even)
    const bool rigid_y = bcy == BC_RIGID;
    // the tile's new v_y rows -2 .. TY of plane k (two buffers alternating with
    // the planes)
    auto nvy_of = [&](int k) -> S * { return nbuf + SH::N_VY + (k & 1) * SH::N_YROWS * TX; };
    // new v_y at local row lr (-2..TY), lane ln: from the p^n plane pk (rows
    // lr-1..lr+2) and the old v_y, t_vy of the stage ost; stored into nvy
    auto vy_new = [&](const S *pk, const S *ost, S *nvy, int lr, int ln, Raw &Vv, Raw &Tv) {
        Raw pr[4], tr[4];
#pragma unroll
        for (int t = 0; t < 4; t++) {
            int l = lr - 1 + t, sg = 1;
            if (!inner_y) {
                int jm;
                if (rigid_y) {
                    sg = img_node(y0 + l, ny, bcy, jm);
                    l = sg == 0 ? 0 : jm - y0;  // the wall row reads as zero
                } else {
                    sg = img_node(y0 + l, ny, bcy, jm);  // the rows hold their images
                }
            }
            const S *ptr = (l >= 0 && l < TY) ? pk + l * WIDE + HALO + ln * VEC
                                              : pk + SH::P_HALO + (l < 0 ? l + 3 : 3 + l - TY) * TX + ln * VEC;
            const Raw r = *reinterpret_cast<const Raw *>(ptr);
            pr[t] = inner_y ? r : signed_raw<V>(r, sg);
            tr[t] = V::zero();
            if (PAIRS) {
                const Raw rt = *reinterpret_cast<const Raw *>(ptr + SH::P_ELEMS);
                tr[t] = inner_y ? rt : signed_raw<V>(rt, sg);
            }
        }
        const AV D = vstencil<V>(tap(pr[0], tr[0]), tap(pr[1], tr[1]), tap(pr[2], tr[2]), tap(pr[3], tr[3]));
        int lv = lr;
        if (!inner_y && rigid_y) {
            int jm;
            img_half(y0 + lr, ny, bcy, jm);
            lv = jm - y0;
        }
        Vv = *reinterpret_cast<const Raw *>(ost + SH::O_VY + (lv + 2) * TX + ln * VEC);
        Tv = COMP ? *reinterpret_cast<const Raw *>(ost + SH::O_TVY + (lv + 2) * TX + ln * VEC) : V::zero();
        V::template update<COMP>(Vv, Tv, V::mul(ay, D));
        *reinterpret_cast<Raw *>(nvy + (lr + 2) * TX + ln * VEC) = Vv;
        if (PAIRS) *reinterpret_cast<Raw *>(nvy + SH::N_ELEMS + (lr + 2) * TX + ln * VEC) = Tv;
    };

    if (warp == 4) {
        // ================================================= producer warp
        const int lane = tid & 31;
        // element offset of the (mapped) source row; rows and planes farther
        // than two past the grid are never read and copy row 0
        auto row_src = [&](int my, int mz, bool node_y, bool node_z) -> int64_t {
            if (my < -3 || my > ny + 2 || mz < -3 || mz > nz + 2) return 0;
            int jy, kz;
            const int s1 = node_y ? img_node(my, ny, bcy, jy) : img_half(my, ny, bcy, jy);
            const int s2 = node_z ? img_node(mz, nz, bcz, kz) : img_half(mz, nz, bcz, kz);
            if (s1 == 0 || s2 == 0) return 0;
            return sy * jy + sz * (int64_t)kz;
        };
        auto plane_of = [&](int m, bool node) -> int {
            if (m < -3 || m > nz + 2) return 0;
            int kz;
            const int s = node ? img_node(m, nz, bcz, kz) : img_half(m, nz, bcz, kz);
            return s == 0 ? 0 : kz;
        };
        // a wide row by bulk copies: the own part and the halo blocks that lie
        // inside the grid (at the grid's x faces the consumers read images)
        auto wide_row = [&](S *dst, const S *src, int64_t rowoff, uint64_t *bar, bool issue) -> uint32_t {
            uint32_t bytes = TX * eb;
            if (issue) bulk_copy(dst + HALO, src + rowoff + x0, TX * eb, bar);
            if (x0 - HALO >= 0) {
                if (issue) bulk_copy(dst, src + rowoff + x0 - HALO, HALO * eb, bar);
                bytes += HALO * eb;
            }
            if (x0 + TX < nx) {
                if (issue) bulk_copy(dst + HALO + TX, src + rowoff + x0 + TX, HALO * eb, bar);
                bytes += HALO * eb;
            }
            return bytes;
        };
        // Boxes wherever their rows lie inside the grid. With rigid y walls
        // boxes are used everywhere: the rows past the y faces are filled with
        // zeros and the consumers read the mirror rows inside the tile instead;
        // periodic y faces copy the wrapped rows row by row.
        const bool rigid_y = bcy == BC_RIGID;
        const bool own_box = rigid_y || y0 + TY <= ny;            // all own rows inside the grid
        const bool top_box = rigid_y || y0 >= 3;                  // p rows y0-3..y0-1 inside
        const bool bot_box = rigid_y || y0 + TY + 3 <= ny;        // p rows y0+TY..y0+TY+2 inside
        const bool vy_box = rigid_y || (y0 >= 2 && y0 + TY + 1 <= ny);  // v_y rows y0-2..y0+TY inside
        // one p plane: the boxes (lane 0) and the row-by-row groups (spread over lanes)
        auto p_plane1 = [&](int m, S *dst, uint64_t *bar, bool issue, const void *src_arr, const CUtensorMap *m_own,
                            const CUtensorMap *m_halo) -> uint32_t {
            const S *pin = static_cast<const S *>(src_arr);
            const int mz = plane_of(m, true);
            uint32_t bytes = 0;
            if (own_box) {
                if (issue && lane == 0) tma_box(dst, m_own, x0 - HALO, y0, mz, bar);
                bytes += TY * WIDE * eb;
            } else {
                for (int r = 0; r < TY; r++)
                    bytes += wide_row(dst + r * WIDE, pin, row_src(y0 + r, m, true, true), bar,
                                      issue && lane == r);
            }
            for (int side = 0; side < 2; side++) {
                S *hd = dst + SH::P_HALO + side * 3 * TX;
                const int ybase = side == 0 ? y0 - 3 : y0 + TY;
                if (side == 0 ? top_box : bot_box) {
                    if (issue && lane == 0) tma_box(hd, m_halo, x0, ybase, mz, bar);
                } else {
                    for (int h = 0; h < 3; h++)
                        if (issue && lane == 16 + side * 3 + h)
                            bulk_copy(hd + h * TX, pin + row_src(ybase + h, m, true, true) + x0, TX * eb, bar);
                }
                bytes += 3 * TX * eb;
            }
            return bytes;
        };
        auto p_plane = [&](int m, S *dst, uint64_t *bar, bool issue) -> uint32_t {
            uint32_t bytes = p_plane1(m, dst, bar, issue, fp.p_in, &maps.p_own, &maps.p_halo);
            if (PAIRS) bytes += p_plane1(m, dst + SH::P_ELEMS, bar, issue, fp.tp, &maps.tp_own, &maps.tp_halo);
            return bytes;
        };
        // the other arrays of iteration k (warm-up iterations k < z0: v_z, t_vz only)
        auto o_stage = [&](int k, S *dst, uint64_t *bar, bool issue) -> uint32_t {
            uint32_t bytes = 0;
            const int kz1 = plane_of(k + 1, false);
            if (issue && lane == 0) tma_box(dst + SH::O_VZ, &maps.vz, x0, y0, kz1, bar);
            bytes += TY * TX * eb;
            if (COMP) {
                if (issue && lane == 0) tma_box(dst + SH::O_TVZ, &maps.tvz, x0, y0, kz1, bar);
                bytes += TY * TX * eb;
            }
            if (k < z0) return bytes;
            if (issue && lane == 0) tma_box(dst + SH::O_VX, &maps.vx, x0 - HALO, y0, k, bar);
            bytes += TY * WIDE * eb;
            if (COMP) {
                if (issue && lane == 0) tma_box(dst + SH::O_TVX, &maps.tvx, x0 - HALO, y0, k, bar);
                bytes += TY * WIDE * eb;
            }
            for (int ca = 0; ca < (COMP ? 2 : 1); ca++) {
                S *d = dst + (ca ? SH::O_TVY : SH::O_VY);
                if (vy_box) {
                    if (issue && lane == 0) tma_box(d, ca ? &maps.tvy : &maps.vy, x0, y0 - 2, k, bar);
                } else {
                    const S *src = static_cast<const S *>(ca ? fp.tvy_in : fp.vy_in);
                    for (int r = 0; r < TY + 3; r++)
                        if (issue && ((r + ca * 7) % 32) == lane)
                            bulk_copy(d + r * TX, src + row_src(y0 - 2 + r, k, false, true) + x0, TX * eb, bar);
                }
                bytes += (TY + 3) * TX * eb;
            }
            return bytes;
        };
        auto issue_p = [&](int m, int cnt) -> bool {
            const int slot = cnt % SP;
            if (cnt >= SP && !wait_phase(&p_empty[slot], ((cnt / SP) - 1) & 1, fp.err)) return false;
            S *dst = pring + slot * SH::P_SLOT;
            const uint32_t total = p_plane(m, dst, nullptr, false);
            if (lane == 0) mbar_expect_tx(&p_full[slot], total);
            __syncwarp();
            p_plane(m, dst, &p_full[slot], true);
            return true;
        };
        auto issue_o = [&](int k, int cnt) -> bool {
            const int slot = cnt % SO;
            if (cnt >= SO && !wait_phase(&o_empty[slot], ((cnt / SO) - 1) & 1, fp.err)) return false;
            S *dst = oring + slot * SH::O_ELEMS;
            const uint32_t total = o_stage(k, dst, nullptr, false);
            if (lane == 0) mbar_expect_tx(&o_full[slot], total);
            __syncwarp();
            o_stage(k, dst, &o_full[slot], true);
            return true;
        };
        // the tile's halo rows -2, -1 (above) and TY (below) of the new v_y of
        // plane k, for the four consumer warps: 3 x LANES vectors on lanes
        // 0..23, once the stages of plane k have landed and every warp has
        // passed the v_y sync of plane k-1 (so the buffer of plane k-2,
        // rewritten now, has been read)
        auto halo_vy = [&](int k) -> bool {
            // both rings count from the first warm-up plane z0 - 3
            const int pcnt = k - (z0 - 3), ocnt = pcnt;
            if (!wait_phase(&p_full[pcnt % SP], (pcnt / SP) & 1, fp.err)) return false;
            if (!wait_phase(&o_full[ocnt % SO], (ocnt / SO) & 1, fp.err)) return false;
            if (k > z0 && !wait_phase(v_bar, (k - 1 - z0) & 1, fp.err)) return false;
            if (lane < 3 * SH::LANES) {
                const int hr = lane / SH::LANES, ln = lane % SH::LANES;
                const int lr = hr == 0 ? -2 : (hr == 1 ? -1 : TY);
                if (y0 + lr <= ny) {
                    Raw Vh, Th;
                    vy_new(pring + (pcnt % SP) * SH::P_SLOT, oring + (ocnt % SO) * SH::O_ELEMS, nvy_of(k), lr,
                           ln, Vh, Th);
                }
            }
            mbar_arrive(v_bar);
            return true;
        };
        int pc = 0, oc = 0;
        bool ok = true;
        for (int m = z0 - 3; m <= z1 + 2 && ok; m++) {
            ok = issue_p(m, pc++);
            if (ok && m >= z0) ok = issue_o(m - 3, oc++);
            // the halo of the plane whose stages were issued an iteration ago
            if (ok && m - 4 >= z0 && m - 4 < z1) ok = halo_vy(m - 4);
        }
        for (int k = max(z1 + 2 - 3, z0); k < z1 && ok; k++) ok = halo_vy(k);
        if (lane == 0) {  // let the copies issued by this warp land before leaving
            for (int c = (pc > SP ? pc - SP : 0); c < pc; c++) drain_phase(&p_full[c % SP], (c / SP) & 1);
            for (int c = (oc > SO ? oc - SO : 0); c < oc; c++) drain_phase(&o_full[c % SO], (c / SO) & 1);
        }
        return;
    }

    // ===================================================== consumer warps
    const int lx = tid % SH::LANES, row = tid / SH::LANES;
    const int x = x0 + lx * VEC;
    const int j = y0 + row;
    const bool active = j < ny;
    const AV ax = V::splat(CoefOf<P>::ld(a_raw[0])), az = V::splat(CoefOf<P>::ld(a_raw[2]));
    const typename P::A ax_s = CoefOf<P>::ld(a_raw[0]);

    auto plane_sign = [&](int m) -> int { int t; return img_node(m, nz, bcz, t); };
    // raw p vector of local row lr (-3..TY+2) at the own lane
    auto p_vec = [&](const S *pst, int lr) -> Raw {
        const S *ptr = (lr >= 0 && lr < TY) ? pst + lr * WIDE + HALO + lx * VEC
                                            : pst + SH::P_HALO + (lr < 0 ? lr + 3 : 3 + lr - TY) * TX + lx * VEC;
        return *reinterpret_cast<const Raw *>(ptr);
    };
    auto vec_at = [&](const S *p) -> Raw { return *reinterpret_cast<const Raw *>(p); };

    float e_s = 0.f, e_c = 0.f;
    auto eadd = [&](float x_) {
        const float t = __fadd_rn(e_s, x_);
        const float pa = __fsub_rn(t, x_);
        const float pb = __fsub_rn(t, pa);
        e_c = __fadd_rn(e_c, __fadd_rn(__fsub_rn(e_s, pa), __fsub_rn(x_, pb)));
        e_s = t;
    };

    Raw vzq0 = V::zero(), vzq1 = V::zero(), vzq2 = V::zero(), vzq3 = V::zero();
    // the pairs: queues of the taps RN(V + T) themselves (each formed once):
    // p of planes k .. k+3 and the new v_z of planes k-2 .. k+1
    AV ps0{}, ps1{}, ps2{}, ps3{}, zs0{}, zs1{}, zs2{}, zs3{};
    int oc = 0, p_waited = 0;
    // ring positions kept incrementally (no division by the ring depth):
    // the next p stage to wait for and its phase, the slot of plane k
    int pw_slot = 0, pk_slot = 0;
    uint32_t pw_phase = 0;
    // own-column p^n of planes k, k+1, k+2 (z images applied), plane k+3 loaded each iteration
    Raw pq0 = V::zero(), pq1 = V::zero(), pq2 = V::zero();
    uint32_t c_phase = 0;
    bool ok = true;
    auto consumer_sync = [&]() -> bool {
        mbar_arrive(c_bar);
        const bool r = wait_phase(c_bar, c_phase & 1, fp.err);
        c_phase++;
        return r;
    };

    for (int k = z0 - 3; k < z1 && ok; k++) {
        const int pbase = k - (z0 - 3);
        while (p_waited < pbase + 4) {
            if (!wait_phase(&p_full[pw_slot], pw_phase, fp.err)) { ok = false; break; }
            p_waited++;
            if (++pw_slot == SP) { pw_slot = 0; pw_phase ^= 1u; }
        }
        if (!ok) break;
        const int oslot = oc % SO;
        if (!wait_phase(&o_full[oslot], (oc / SO) & 1, fp.err)) { ok = false; break; }
        const S *ost = oring + oslot * SH::O_ELEMS;
        const S *pk = pring + pk_slot * SH::P_SLOT;

        // ---- v_z^{n+1/2} at plane k+1 of the own vector (p^n planes k..k+3)
        Raw vzn = V::zero(), tzn = V::zero();
        const bool inner_z = k >= 0 && k + 3 < nz;  // planes k..k+3 inside the grid
        Raw pq3 = V::zero();
        if (active) {
            // plane k + t of p (off = 0) or t_p (off = P_ELEMS)
            auto plane = [&](int t, int off) -> Raw {
                int sl = pk_slot + t;
                if (sl >= SP) sl -= SP;
                const Raw r = p_vec(pring + sl * SH::P_SLOT + off, row);
                return inner_z ? r : signed_raw<V>(r, plane_sign(k + t));
            };
            AV D;
            if constexpr (PAIRS) {
                if (k == z0 - 3) {
                    ps0 = tap(plane(0, 0), plane(0, SH::P_ELEMS));
                    ps1 = tap(plane(1, 0), plane(1, SH::P_ELEMS));
                    ps2 = tap(plane(2, 0), plane(2, SH::P_ELEMS));
                }
                ps3 = tap(plane(3, 0), plane(3, SH::P_ELEMS));
                D = vstencil<V>(ps0, ps1, ps2, ps3);
            } else {
                if (k == z0 - 3) {
                    pq0 = plane(0, 0);
                    pq1 = plane(1, 0);
                    pq2 = plane(2, 0);
                }
                pq3 = plane(3, 0);
                D = vstencil<V>(V::ld(pq0), V::ld(pq1), V::ld(pq2), V::ld(pq3));
            }
            vzn = vec_at(ost + SH::O_VZ + row * TX + lx * VEC);
            tzn = COMP ? vec_at(ost + SH::O_TVZ + row * TX + lx * VEC) : V::zero();
            V::template update<COMP>(vzn, tzn, V::mul(az, D));
            if (k + 1 >= z0 && k + 1 < z1) {
                const int64_t qz = x + sy * j + sz * (int64_t)(k + 1);
                at<V>(fp.vz_out, qz) = vzn;
                if (COMP) at<V>(fp.tvz_out, qz) = tzn;
            }
        }
        vzq3 = vzn;
        if constexpr (PAIRS) zs3 = tap(vzn, tzn);

        if (k >= z0) {
            S *nvx = nbuf;
            // the tile's v_y rows -2 .. TY of this plane (buffers alternate
            // with the planes: a buffer is rewritten only after every warp
            // has passed the next plane's sync, i.e. finished reading it)
            S *nvy = nvy_of(k);
            constexpr int wr0 = -2;
            __syncwarp();  // this warp's reads of the previous plane's v_x rows are done
            Raw vxn = V::zero(), txn = V::zero(), vyn = V::zero(), tyn = V::zero();
            // ---- v_x^{n+1/2}: own vector, and the x halo of the tile edge lanes
            if (active) {
                const S *prow = pk + row * WIDE + HALO - x0;  // indexed by global x
                const S *trow = prow + SH::P_ELEMS;             // t_p (the pairs)
                // plane k is inside the grid: no image; p[-1] = -p[1] and the
                // wall node and its image at the x faces
                auto xn = [&](const S *r, RS &l0, RS &r0, RS &r1) {
                    if (x == 0) l0 = V::rneg_s(r[1]);
                    else l0 = r[x - 1];
                    if (x + VEC == nx) { r0 = RS(0); r1 = V::rneg_s(r[nx - 1]); }
                    else { r0 = r[x + VEC]; r1 = r[x + VEC + 1]; }
                };
                RS l0, r0, r1, l0t = RS(0), r0t = RS(0), r1t = RS(0);
                xn(prow, l0, r0, r1);
                if (PAIRS) xn(trow, l0t, r0t, r1t);
                AV own;
                if constexpr (PAIRS) own = ps0;
                else own = V::ld(pq0);
                const typename V::AS al0 = tap_s(l0, l0t), ar0 = tap_s(r0, r0t), ar1 = tap_s(r1, r1t);
                const AV D = vstencil<V>(V::shr1(own, al0), own, V::shl1(own, ar0), V::shl2(own, ar0, ar1));
                vxn = vec_at(ost + SH::O_VX + row * WIDE + HALO + lx * VEC);
                txn = COMP ? vec_at(ost + SH::O_TVX + row * WIDE + HALO + lx * VEC) : V::zero();
                V::template update<COMP>(vxn, txn, V::mul(ax, D));
                S *nrow = nvx + row * WIDE + HALO - x0;
                *reinterpret_cast<Raw *>(nrow + x) = vxn;
                if (PAIRS) *reinterpret_cast<Raw *>(nrow + SH::N_ELEMS + x) = txn;
                // final: store now, so that the registers are free for the rest of the plane
                const int64_t qv = x + sy * j + sz * (int64_t)k;
                at<V>(fp.vx_out, qv) = vxn;
                if (COMP) at<V>(fp.tvx_out, qv) = txn;
                // the x halo of the tile (v_x at x0-2, x0-1, x0+TX), one value per
                // lane 0, 1, 2, where it lies inside the grid; at the grid's x faces
                // the reads below take the even images of v_x instead
                if (lx < 3) {
                    const int ix = lx == 0 ? x0 - 2 : (lx == 1 ? x0 - 1 : x0 + TX);
                    if (ix >= 0 && ix < nx) {
                        const S *vxr = ost + SH::O_VX + row * WIDE + HALO - x0;
                        const S *txr = ost + SH::O_TVX + row * WIDE + HALO - x0;
                        auto tp1 = [&](int m) -> typename P::A {
                            return PAIRS ? P::add(P::ld(prow[m]), P::ld(trow[m])) : P::ld(prow[m]);
                        };
                        const typename P::A D1 = stencil<P>(tp1(ix - 1), tp1(ix), tp1(ix + 1), tp1(ix + 2));
                        S Vv = vxr[ix];
                        S Tv = COMP ? txr[ix] : S(0);
                        update<P, COMP>(Vv, Tv, P::mul(ax_s, D1));
                        nrow[ix] = Vv;
                        if (PAIRS) nrow[SH::N_ELEMS + ix] = Tv;
                    }
                }
            }
            // ---- v_y^{n+1/2}: own rows, and row ny (the image row the last
            // grid row reads); the producer warp adds the tile's halo rows
            if (j <= ny) vy_new(pk, ost, nvy, row, lx, vyn, tyn);
            if (active) {
                const int64_t qv = x + sy * j + sz * (int64_t)k;
                at<V>(fp.vy_out, qv) = vyn;
                if (COMP) at<V>(fp.tvy_out, qv) = tyn;
            }
            // own t_p and b vectors from global memory, issued before the
            // exchange reads so that their latency overlaps them
            const int64_t q = x + sy * j + sz * (int64_t)k;
            Raw tpn = V::zero(), bv = V::zero();
            float4 bf0 = make_float4(0.f, 0.f, 0.f, 0.f), bf1 = bf0;  // the pairs: binary32 b
            if (active) {
                if (COMP) tpn = *reinterpret_cast<const Raw *>(static_cast<const S *>(fp.tp) + q);
                if (prm.b) {
                    if (PAIRS) {
                        const float4 *bp = reinterpret_cast<const float4 *>(static_cast<const float *>(prm.b) + q);
                        bf0 = __ldg(bp);
                        bf1 = __ldg(bp + 1);
                    } else {
                        bv = __ldg(reinterpret_cast<const Raw *>(static_cast<const S *>(prm.b) + q));
                    }
                }
            }
            // every warp's v_y rows and the producer's halo rows of this plane
            // are in nvy (bounded wait)
            mbar_arrive(v_bar);
            if (!wait_phase(v_bar, (k - z0) & 1, fp.err)) { ok = false; break; }
            // ---- p^{n+1}
            if (active) {
                const S *vrow = nvx + row * WIDE + HALO - x0;
                const S *tvrow = vrow + SH::N_ELEMS;  // the pairs: T of the new v_x
                const AV ownx = tap(*reinterpret_cast<const Raw *>(vrow + x),
                                    PAIRS ? *reinterpret_cast<const Raw *>(tvrow + x) : V::zero());
                // v_x at x-2, x-1, x+VEC; at the x faces the even images (v_x at 1, 0; nx-1)
                const int il1 = x == 0 ? 1 : x - 2, il0 = x == 0 ? 0 : x - 1, irr = x + VEC == nx ? nx - 1 : x + VEC;
                const typename V::AS l1 = tap_s(vrow[il1], PAIRS ? tvrow[il1] : RS(0));
                const typename V::AS l0 = tap_s(vrow[il0], PAIRS ? tvrow[il0] : RS(0));
                const typename V::AS rr = tap_s(vrow[irr], PAIRS ? tvrow[irr] : RS(0));
                AV R = vstencil<V>(V::shr2(ownx, l1, l0), V::shr1(ownx, l0), ownx, V::shl1(ownx, rr));
                const S *vyc = nvy + (row - 2 - wr0) * TX + lx * VEC;  // rows row-2 .. row+1
                auto vy_tap = [&](int r) -> AV {
                    return tap(vec_at(vyc + r * TX), PAIRS ? vec_at(vyc + SH::N_ELEMS + r * TX) : V::zero());
                };
                const AV Dy = vstencil<V>(vy_tap(0), vy_tap(1), vy_tap(2), vy_tap(3));
                R = V::add(R, Dy);
                AV Dz;
                if constexpr (PAIRS) Dz = vstencil<V>(zs0, zs1, zs2, zs3);
                else Dz = vstencil<V>(V::ld(vzq0), V::ld(vzq1), V::ld(vzq2), V::ld(vzq3));
                R = V::add(R, Dz);
                if (k == prm.src_k && j == prm.src_j && prm.src_i >= x && prm.src_i < x + VEC &&
                    prm.step < prm.src_nt) {
                    const typename V::AS sv_ = static_cast<const typename V::AS *>(prm.src)[prm.step];
                    // element index known at compile time: R stays in registers
#pragma unroll
                    for (int e = 0; e < VEC; e++)
                        if (e == prm.src_i - x) V::set(R, e, P::add(V::aget(R, e), sv_));
                }
                AV bc;
                if constexpr (PAIRS) {
                    if (prm.b) {
                        const float bb[8] = {bf0.x, bf0.y, bf0.z, bf0.w, bf1.x, bf1.y, bf1.z, bf1.w};
#pragma unroll
                        for (int e = 0; e < VEC; e++) V::set(bc, e, bb[e]);
                    } else {
                        bc = V::splat(CoefOf<P>::ld(b_raw));
                    }
                } else {
                    bc = prm.b ? V::ld(bv) : V::splat(V::lds(b_raw));
                }
                // p^n of the own vector (the pairs keep only the taps in
                // registers: p from the ring's plane k, inside the grid)
                Raw pold;
                if constexpr (PAIRS) pold = p_vec(pk, row);
                else pold = pq0;
                Raw pn = pold;
                V::template update<COMP>(pn, tpn, V::mul(bc, R));
                at<V>(fp.p_out, q) = pn;
                if (COMP) at<V>(fp.tp_out, q) = tpn;
                if (ENERGY) {
                    // v^2 / a with the uniform a as a product by its reciprocal;
                    // the four terms of a point summed in binary32, then added
                    // to the compensated accumulator
                    const float ia0 = __frcp_rn(CoefOf<P>::f32(a_raw[0])), ia1 = __frcp_rn(CoefOf<P>::f32(a_raw[1])),
                                ia2 = __frcp_rn(CoefOf<P>::f32(a_raw[2]));
#pragma unroll
                    for (int e = 0; e < VEC; e++) {
                        float bw;
                        if constexpr (PAIRS) bw = V::aget(bc, e);
                        else bw = prm.b ? V::f32(bv, e) : P::to_f32(b_raw);
                        // (the pairs keep only the v_z taps in registers: the
                        // stored v_z of plane k, written by this thread one
                        // plane ago)
                        const float fx = V::f32(vxn, e), fy = V::f32(vyn, e),
                                    fz = V::f32(PAIRS ? at<V>(fp.vz_out, q) : vzq2, e);
                        float t = e_term(V::f32(pold, e), V::f32(pn, e), bw);
                        t = __fadd_rn(t, __fmul_rn(__fmul_rn(fx, fx), ia0));
                        t = __fadd_rn(t, __fmul_rn(__fmul_rn(fy, fy), ia1));
                        t = __fadd_rn(t, __fmul_rn(__fmul_rn(fz, fz), ia2));
                        eadd(t);
                    }
                }
            }
        }
        // release the stages this iteration consumed: the other arrays of k, p plane k
        __syncwarp();
        if ((tid & 31) == 0) {
            mbar_arrive(&o_empty[oslot]);
            mbar_arrive(&p_empty[pk_slot]);
        }
        oc++;
        if (++pk_slot == SP) pk_slot = 0;
        vzq0 = vzq1;
        vzq1 = vzq2;
        vzq2 = vzq3;
        zs0 = zs1;
        zs1 = zs2;
        zs2 = zs3;
        pq0 = pq1;
        pq1 = pq2;
        pq2 = pq3;
        ps0 = ps1;
        ps1 = ps2;
        ps2 = ps3;
    }
    if (ENERGY) {
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
static cudaError_t launch_t(const FusedParams &fp, const FusedMaps &maps, bool energy, cudaStream_t st) {
    using SH = FShape<P>;
    dim3 grid(fp.a.n[0] / SH::TX, (fp.a.n[1] + SH::TY - 1) / SH::TY,
              (fp.a.n[2] + fp.zchunk - 1) / fp.zchunk);
    const int smem = (int)SH::SMEM;
    // the pair kernel (74.75 KiB, at most 128 registers) fits three CTAs per SM
    // only with the whole shared-memory carveout (3 x 75.75 of 228 KiB)
    const int carveout = SH::PAIRS ? 100 : -1;
    cudaError_t e;
    if (energy) {
        e = cudaFuncSetAttribute(fused_step<P, COMP, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e == cudaSuccess && carveout >= 0)
            e = cudaFuncSetAttribute(fused_step<P, COMP, true>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                     carveout);
        if (e != cudaSuccess) return e;
        fused_step<P, COMP, true><<<grid, 160, smem, st>>>(fp, maps);
    } else {
        e = cudaFuncSetAttribute(fused_step<P, COMP, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e == cudaSuccess && carveout >= 0)
            e = cudaFuncSetAttribute(fused_step<P, COMP, false>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                     carveout);
        if (e != cudaSuccess) return e;
        fused_step<P, COMP, false><<<grid, 160, smem, st>>>(fp, maps);
    }
    return cudaGetLastError();
}

template <class P>
static cudaError_t launch_c(const FusedParams &fp, const FusedMaps &maps, int comp, bool energy,
                            cudaStream_t st) {
    switch (comp) {
    case 0: return launch_t<P, 0>(fp, maps, energy, st);
    case 3: return launch_t<P, 3>(fp, maps, energy, st);
    default: return launch_t<P, 6>(fp, maps, energy, st);
    }
}

int fused_tile_x(int prec) { return prec == PREC_FP32 ? 32 : 64; }

bool acoustic_fused_supported(const AcParams &prm, int ndim, int prec) {
    if (ndim != 3 || prec == PREC_FP64) return false;
    if (prm.n[0] % fused_tile_x(prec) != 0 || prm.n[1] < 8 || prm.n[2] < 8) return false;
    if (prm.bc[0] != BC_RIGID) return false;
    return prm.a[0] == nullptr && prm.a[1] == nullptr && prm.a[2] == nullptr;
}

unsigned acoustic_fused_blocks(const AcParams &prm, int prec, int zchunk) {
    return (prm.n[0] / fused_tile_x(prec)) * ((prm.n[1] + 15) / 16) * ((prm.n[2] + zchunk - 1) / zchunk);
}

// ------------------------------------------------------------ tensor maps
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                  const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                  const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encoder() {
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    }
    return fn;
}

// One 3D map over an array of the grid (x extent n[0], row pitch in elements).
static bool encode(CUtensorMap *m, const void *ptr, const int n[3], int64_t pitch, int eb, int bx,
                   int by) {
    EncodeTiledFn fn = encoder();
    if (!fn || !ptr) return false;
    const cuuint64_t dims[3] = {(cuuint64_t)n[0], (cuuint64_t)n[1], (cuuint64_t)n[2]};
    const cuuint64_t strides[2] = {(cuuint64_t)(pitch * eb), (cuuint64_t)(pitch * n[1] * eb)};
    const cuuint32_t box[3] = {(cuuint32_t)bx, (cuuint32_t)by, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    const CUresult r = fn(m, eb == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_UINT16, 3,
                          const_cast<void *>(ptr), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                          CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

size_t fused_maps_bytes() { return sizeof(FusedMaps); }

// Fill the maps for one input set: in[] = p, vx, vy, vz, tvx, tvy, tvz.
bool acoustic_fused_encode(void *out_maps, const AcParams &prm, const void *const in[7], const void *tp,
                           int prec, int comp) {
    FusedMaps mp;
    memset(&mp, 0, sizeof mp);
    const int eb = prec == PREC_FP32 ? 4 : 2;
    const int vec = 16 / eb, tx = 8 * vec, wide = tx + 2 * vec, ty = 16;
    bool ok = encode(&mp.p_own, in[0], prm.n, prm.sy, eb, wide, ty) &&
              encode(&mp.p_halo, in[0], prm.n, prm.sy, eb, tx, 3) &&
              encode(&mp.vx, in[1], prm.n, prm.sy, eb, wide, ty) &&
              encode(&mp.vy, in[2], prm.n, prm.sy, eb, tx, ty + 3) &&
              encode(&mp.vz, in[3], prm.n, prm.sy, eb, tx, ty);
    if (ok && comp)
        ok = encode(&mp.tvx, in[4], prm.n, prm.sy, eb, wide, ty) &&
             encode(&mp.tvy, in[5], prm.n, prm.sy, eb, tx, ty + 3) &&
             encode(&mp.tvz, in[6], prm.n, prm.sy, eb, tx, ty);
    // the pairs read t_p tiles like p's (tp: the input set's t_p)
    if (ok && prec == PREC_FP16_PAIRS)
        ok = encode(&mp.tp_own, tp, prm.n, prm.sy, eb, wide, ty) && encode(&mp.tp_halo, tp, prm.n, prm.sy, eb, tx, 3);
    if (ok) memcpy(out_maps, &mp, sizeof mp);
    return ok;
}

cudaError_t acoustic_fused_step(const AcParams &prm, const void *maps, const void *const in[7],
                                void *const out[7], void *tp, void *tp_out, int prec, int comp, int zchunk,
                                int *err, cudaStream_t st) {
    FusedParams fp;
    fp.a = prm;
    fp.p_in = in[0]; fp.vx_in = in[1]; fp.vy_in = in[2]; fp.vz_in = in[3];
    fp.tvx_in = in[4]; fp.tvy_in = in[5]; fp.tvz_in = in[6];
    fp.p_out = out[0]; fp.vx_out = out[1]; fp.vy_out = out[2]; fp.vz_out = out[3];
    fp.tvx_out = out[4]; fp.tvy_out = out[5]; fp.tvz_out = out[6];
    fp.tp = tp;
    fp.tp_out = tp_out;
    fp.zchunk = zchunk;
    fp.err = err;
    const FusedMaps &mp = *static_cast<const FusedMaps *>(maps);
    const bool energy = prm.energy != 0;
    switch (prec) {
    case PREC_FP32: return launch_c<F32>(fp, mp, comp, energy, st);
    case PREC_FP16: return launch_c<F16>(fp, mp, comp, energy, st);
    case PREC_BF16: return launch_c<BF16>(fp, mp, comp, energy, st);
    case PREC_FP16_F32ARITH: return launch_c<F16W>(fp, mp, comp ? 3 : 0, energy, st);
    case PREC_BF16_F32ARITH: return launch_c<BF16W>(fp, mp, comp ? 3 : 0, energy, st);
    case PREC_FP16_PAIRS: return comp ? launch_t<F16WP, 3>(fp, mp, energy, st) : cudaErrorInvalidValue;
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace wave
