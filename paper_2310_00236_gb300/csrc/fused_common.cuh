// fused_common.cuh -- pieces shared by the one-pass 3D kernels: inline-PTX
// wrappers for mbarriers and bulk / tensor copies, bounded waits, the kernel
// parameter blocks.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "acoustic_common.cuh"

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
__device__ __forceinline__ void tma_box(void *dst_smem, const CUtensorMap *map, int x, int y, int z,
                                        uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
        "[%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_addr(dst_smem)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_addr(bar))
        : "memory");
}

// Bounded wait: about 2^22 polls (each poll may suspend briefly), then the
// error word is set and false returned. Once any block has set the error
// word, waits give up at their next check so that the whole grid leaves fast.
constexpr uint32_t kWaitPolls = 1u << 22;
__device__ __forceinline__ bool wait_phase_limit(uint64_t *bar, uint32_t parity, int *err, uint32_t polls) {
    for (uint32_t it = 0; it < polls; it++) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 1023u) == 1023u && *reinterpret_cast<volatile int *>(err)) return false;
    }
    atomicExch(err, 1);
    return false;
}
__device__ __forceinline__ bool wait_phase(uint64_t *bar, uint32_t parity, int *err) {
    return wait_phase_limit(bar, parity, err, kWaitPolls);
}
// Shorter bounded wait that ignores the error word (draining copies in flight).
__device__ __forceinline__ void drain_phase(uint64_t *bar, uint32_t parity) {
    for (uint32_t it = 0; it < (1u << 16); it++)
        if (mbar_try_wait(bar, parity)) return;
}

struct FusedMaps {
    CUtensorMap p_own, p_halo, vx, tvx, vy, tvy, vz, tvz;
    CUtensorMap tp_own, tp_halo;  // the pair precision: t_p tiles like p's
};

struct FusedParams {
    AcParams a;  // grid, boundaries, strides, multipliers, source, energy
    const void *p_in, *vx_in, *vy_in, *vz_in, *tvx_in, *tvy_in, *tvz_in;
    void *p_out, *vx_out, *vy_out, *vz_out, *tvx_out, *tvy_out, *tvz_out;
    void *tp;       // t_p read (own point; the pair precision: also the stencil taps)
    void *tp_out;   // t_p written: tp itself (in place), except for the pair
                    // precision, whose neighbours read the old t_p in their halos
    int zchunk;
    int *err;    // set to 1 when a bounded wait expires
};

template <class V>
__device__ __forceinline__ typename V::Raw signed_raw(const typename V::Raw &r, int sign) {
    return sign > 0 ? r : (sign < 0 ? V::rneg(r) : V::zero());
}

}  // namespace wave
