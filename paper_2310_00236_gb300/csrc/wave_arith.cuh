// wave_arith.cuh -- per-format arithmetic for the stencil kernels.
//
// Every +, -, * is issued as one PTX instruction with an explicit .rn
// rounding modifier. PTX never fuses an instruction that carries a rounding
// modifier into an FMA, so each operation is a single correctly rounded IEEE
// operation of the format (Section 2's model), independent of -fmad.
// The library is also compiled with -fmad=false for the remaining code.
//
// A policy provides:
//   S        storage type (16-bit bits or float)
//   A        arithmetic type
//   S2 / A2  packed pairs (x-neighbour points processed together)
//   load/store conversions, add/sub/mul on A and A2, and the constants of the
//   stencil: C1 = 9/8 (exact in every format), C2 = 1/24 rounded to the format
//   of the stencil arithmetic.
#pragma once
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <stdint.h>

namespace wave {

// ---------------------------------------------------------------- binary16
struct F16 {
    using S = uint16_t;           // stored bits
    using A = uint16_t;           // arithmetic value (bits of a binary16)
    using A2 = uint32_t;          // two binary16 in one register, low = first
    static constexpr bool kWideArith = false;
    static __device__ __forceinline__ A add(A a, A b) {
        A d; asm("add.rn.f16 %0, %1, %2;" : "=h"(d) : "h"(a), "h"(b)); return d; }
    static __device__ __forceinline__ A sub(A a, A b) {
        A d; asm("sub.rn.f16 %0, %1, %2;" : "=h"(d) : "h"(a), "h"(b)); return d; }
    static __device__ __forceinline__ A mul(A a, A b) {
        A d; asm("mul.rn.f16 %0, %1, %2;" : "=h"(d) : "h"(a), "h"(b)); return d; }
    static __device__ __forceinline__ A2 add2(A2 a, A2 b) {
        A2 d; asm("add.rn.f16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b)); return d; }
    static __device__ __forceinline__ A2 sub2(A2 a, A2 b) {
        A2 d; asm("sub.rn.f16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b)); return d; }
    static __device__ __forceinline__ A2 mul2(A2 a, A2 b) {
        A2 d; asm("mul.rn.f16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b)); return d; }
    static __device__ __forceinline__ A neg(A a) { return a ^ 0x8000u; }
    static __device__ __forceinline__ A2 neg2(A2 a) { return a ^ 0x80008000u; }
    static __device__ __forceinline__ A ld(S s) { return s; }
    static __device__ __forceinline__ S st(A a) { return a; }
    static __device__ __forceinline__ A c1() { return 0x3C80u; }   // 1.125
    static __device__ __forceinline__ A c2() { return 0x2955u; }   // RN16(1/24)
    static __device__ __forceinline__ float to_f32(S s) {
        return __half2float(__ushort_as_half(s)); }
    static __device__ __forceinline__ A zero() { return 0; }
};

// ---------------------------------------------------------------- bfloat16
struct BF16 {
    using S = uint16_t;
    using A = uint16_t;
    using A2 = uint32_t;
    static constexpr bool kWideArith = false;
    static __device__ __forceinline__ A add(A a, A b) {
        A d; asm("add.rn.bf16 %0, %1, %2;" : "=h"(d) : "h"(a), "h"(b)); return d; }
    static __device__ __forceinline__ A sub(A a, A b) {
        A d; asm("sub.rn.bf16 %0, %1, %2;" : "=h"(d) : "h"(a), "h"(b)); return d; }
    static __device__ __forceinline__ A mul(A a, A b) {
        A d; asm("mul.rn.bf16 %0, %1, %2;" : "=h"(d) : "h"(a), "h"(b)); return d; }
    static __device__ __forceinline__ A2 add2(A2 a, A2 b) {
        A2 d; asm("add.rn.bf16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b)); return d; }
    static __device__ __forceinline__ A2 sub2(A2 a, A2 b) {
        A2 d; asm("sub.rn.bf16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b)); return d; }
    static __device__ __forceinline__ A2 mul2(A2 a, A2 b) {
        A2 d; asm("mul.rn.bf16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b)); return d; }
    static __device__ __forceinline__ A neg(A a) { return a ^ 0x8000u; }
    static __device__ __forceinline__ A2 neg2(A2 a) { return a ^ 0x80008000u; }
    static __device__ __forceinline__ A ld(S s) { return s; }
    static __device__ __forceinline__ S st(A a) { return a; }
    static __device__ __forceinline__ A c1() { return 0x3F90u; }   // 1.125
    static __device__ __forceinline__ A c2() { return 0x3D2Bu; }   // RNbf(1/24) = 0.041748046875
    static __device__ __forceinline__ float to_f32(S s) {
        return __uint_as_float(static_cast<uint32_t>(s) << 16); }
    static __device__ __forceinline__ A zero() { return 0; }
};

// ---------------------------------------------------------------- binary32
struct F32 {
    using S = float;
    using A = float;
    static constexpr bool kWideArith = false;
    static __device__ __forceinline__ A add(A a, A b) { return __fadd_rn(a, b); }
    static __device__ __forceinline__ A sub(A a, A b) { return __fsub_rn(a, b); }
    static __device__ __forceinline__ A mul(A a, A b) { return __fmul_rn(a, b); }
    static __device__ __forceinline__ A neg(A a) { return -a; }
    static __device__ __forceinline__ A ld(S s) { return s; }
    static __device__ __forceinline__ S st(A a) { return a; }
    static __device__ __forceinline__ A c1() { return 1.125f; }
    static __device__ __forceinline__ A c2() { return __uint_as_float(0x3D2AAAABu); } // RN32(1/24)
    static __device__ __forceinline__ float to_f32(S s) { return s; }
    static __device__ __forceinline__ A zero() { return 0.0f; }
};

// ------------------------------------- half / bfloat16 storage, binary32 arithmetic
template <class Store>
struct WideArith {
    using S = uint16_t;
    using A = float;
    static constexpr bool kWideArith = true;
    static __device__ __forceinline__ A add(A a, A b) { return __fadd_rn(a, b); }
    static __device__ __forceinline__ A sub(A a, A b) { return __fsub_rn(a, b); }
    static __device__ __forceinline__ A mul(A a, A b) { return __fmul_rn(a, b); }
    static __device__ __forceinline__ A neg(A a) { return -a; }
    static __device__ __forceinline__ A ld(S s) { return Store::to_f32(s); }
    static __device__ __forceinline__ S st(A a);
    static __device__ __forceinline__ A c1() { return 1.125f; }
    static __device__ __forceinline__ A c2() { return __uint_as_float(0x3D2AAAABu); }
    static __device__ __forceinline__ float to_f32(S s) { return Store::to_f32(s); }
    static __device__ __forceinline__ A zero() { return 0.0f; }
};
template <>
__device__ __forceinline__ uint16_t WideArith<F16>::st(float a) {
    return __half_as_ushort(__float2half_rn(a)); }
template <>
__device__ __forceinline__ uint16_t WideArith<BF16>::st(float a) {
    return __bfloat16_as_ushort(__float2bfloat16_rn(a)); }

using F16W = WideArith<F16>;
using BF16W = WideArith<BF16>;

// The binary32-register arithmetic with stencils that read the stored pair:
// every stencil tap is RN32(V + T), the stored value plus its carried
// compensation, instead of V (not the paper's scheme, where the stencil reads
// V: reading the pair removes the error of the rounded stored value; the
// update is WideArith's compensated one).
template <class Store>
struct PairArith : WideArith<Store> {};
using F16WP = PairArith<F16>;

template <class P> struct IsPairs { static constexpr bool value = false; };
template <class Store> struct IsPairs<PairArith<Store>> { static constexpr bool value = true; };

// Storage of the multipliers a and b: the field storage type, except for the
// pair policies, which keep them in binary32 (their rounding to binary16 is
// the error the pair stencil does not remove).
template <class P>
struct CoefOf {
    using S = typename P::S;
    static __device__ __forceinline__ typename P::A ld(S s) { return P::ld(s); }
    static __device__ __forceinline__ float f32(S s) { return P::to_f32(s); }
};
template <class Store>
struct CoefOf<PairArith<Store>> {
    using S = float;
    static __device__ __forceinline__ float ld(float s) { return s; }
    static __device__ __forceinline__ float f32(float s) { return s; }
};

// ------------------------------------------------------------ the method's ops
// Fourth-order staggered difference (Section 3):
//   D = C1 * (f[+1/2] - f[-1/2]) - C2 * (f[+3/2] - f[-3/2])
template <class P>
__device__ __forceinline__ typename P::A stencil(typename P::A fm3, typename P::A fm1,
                                                 typename P::A fp1, typename P::A fp3) {
    typename P::A t1 = P::sub(fp1, fm1);
    typename P::A t2 = P::sub(fp3, fm3);
    return P::sub(P::mul(P::c1(), t1), P::mul(P::c2(), t2));
}

// Solution update V += inc: plain (Algorithm 1) or compensated (Algorithm 2):
// R = T + inc; then sum_3op(V, R) (Code 1) or sum_6op(V, R) (Code 2) gives the
// new V and the new carried term T. With binary32 arithmetic on half storage
// the compensated form is s = V + R, V' = RN(s), T' = RN(s - V').
template <class P, int COMP>
__device__ __forceinline__ void update(typename P::S &V, typename P::S &T, typename P::A inc) {
    using A = typename P::A;
    if (COMP == 0) {
        V = P::st(P::add(P::ld(V), inc));
        return;
    }
    A R = P::add(P::ld(T), inc);
    A v = P::ld(V);
    if (P::kWideArith) {
        A s = P::add(v, R);
        typename P::S vs = P::st(s);
        T = P::st(P::sub(s, P::ld(vs)));
        V = vs;
    } else if (COMP == 3) {
        A s = P::add(v, R);
        A z = P::sub(s, v);
        T = P::st(P::sub(R, z));
        V = P::st(s);
    } else {
        A s = P::add(v, R);
        A pa = P::sub(s, R);
        A pb = P::sub(s, pa);
        A da = P::sub(v, pa);
        A db = P::sub(R, pb);
        T = P::st(P::add(da, db));
        V = P::st(s);
    }
}

}  // namespace wave
