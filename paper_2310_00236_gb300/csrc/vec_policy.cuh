// vec_policy.cuh -- 16-byte vector policies shared by the 3D streaming kernels:
// VEC consecutive x values of one thread, loaded and stored as one 16-byte
// vector, with packed-pair arithmetic for half / bfloat16 (f16x2 / bf16x2) and
// per-element arithmetic for binary32 and for half storage with binary32
// registers. The operations are those of wave_arith.cuh, element for element.
#pragma once
#include "acoustic_common.cuh"

namespace wave {

// ------------------------------------------------------------------------
// Vector policies: VEC consecutive values of one thread.
//   Raw: the 16-byte storage vector.   AV: the arithmetic vector.
//   RS / AS: raw / arithmetic scalar.
// ------------------------------------------------------------------------
template <class P>
struct VPacked {  // binary16 / bfloat16 stored and computed in pairs
    static constexpr int N = 8;
    using Raw = uint4;
    using AV = uint4;
    using RS = uint16_t;
    using AS = uint16_t;
    static __device__ __forceinline__ AV ld(const Raw &r) { return r; }
    static __device__ __forceinline__ AS lds(RS s) { return s; }
    static __device__ __forceinline__ Raw zero() { return make_uint4(0, 0, 0, 0); }
    static __device__ __forceinline__ Raw rneg(const Raw &r) {
        return make_uint4(r.x ^ 0x80008000u, r.y ^ 0x80008000u, r.z ^ 0x80008000u,
                          r.w ^ 0x80008000u);
    }
    static __device__ __forceinline__ RS rneg_s(RS s) { return s ^ 0x8000u; }
    static __device__ __forceinline__ AV add(const AV &a, const AV &b) {
        return make_uint4(P::add2(a.x, b.x), P::add2(a.y, b.y), P::add2(a.z, b.z), P::add2(a.w, b.w)); }
    static __device__ __forceinline__ AV sub(const AV &a, const AV &b) {
        return make_uint4(P::sub2(a.x, b.x), P::sub2(a.y, b.y), P::sub2(a.z, b.z), P::sub2(a.w, b.w)); }
    static __device__ __forceinline__ AV mul(const AV &a, const AV &b) {
        return make_uint4(P::mul2(a.x, b.x), P::mul2(a.y, b.y), P::mul2(a.z, b.z), P::mul2(a.w, b.w)); }
    static __device__ __forceinline__ AV splat(AS s) {
        uint32_t w = (uint32_t)s | ((uint32_t)s << 16);
        return make_uint4(w, w, w, w);
    }
    static __device__ __forceinline__ RS get(const Raw &r, int i) {
        uint32_t w = (i >> 1) == 0 ? r.x : (i >> 1) == 1 ? r.y : (i >> 1) == 2 ? r.z : r.w;
        return (RS)((i & 1) ? (w >> 16) : (w & 0xFFFFu));
    }
    static __device__ __forceinline__ void set(AV &r, int i, AS s) {
        uint32_t *w = (i >> 1) == 0 ? &r.x : (i >> 1) == 1 ? &r.y : (i >> 1) == 2 ? &r.z : &r.w;
        *w = (i & 1) ? ((*w & 0xFFFFu) | ((uint32_t)s << 16)) : ((*w & 0xFFFF0000u) | s);
    }
    static __device__ __forceinline__ AS aget(const AV &r, int i) { return get(r, i); }
    static __device__ __forceinline__ float f32(const Raw &r, int i) { return P::to_f32(get(r, i)); }
    // values at offsets +1, +2, -1, -2 from the own vector
    static __device__ __forceinline__ AV shl1(const AV &o, AS r0) {
        return make_uint4(__byte_perm(o.x, o.y, 0x5432), __byte_perm(o.y, o.z, 0x5432),
                          __byte_perm(o.z, o.w, 0x5432), __byte_perm(o.w, (uint32_t)r0, 0x5432));
    }
    static __device__ __forceinline__ AV shl2(const AV &o, AS r0, AS r1) {
        return make_uint4(o.y, o.z, o.w, (uint32_t)r0 | ((uint32_t)r1 << 16));
    }
    static __device__ __forceinline__ AV shr1(const AV &o, AS l0) {
        return make_uint4(__byte_perm((uint32_t)l0, o.x, 0x5410), __byte_perm(o.x, o.y, 0x5432),
                          __byte_perm(o.y, o.z, 0x5432), __byte_perm(o.z, o.w, 0x5432));
    }
    static __device__ __forceinline__ AV shr2(const AV &o, AS l1, AS l0) {
        return make_uint4((uint32_t)l1 | ((uint32_t)l0 << 16), o.x, o.y, o.z);
    }
    // compensated / plain update on packed pairs (Algorithm 1 / 2)
    template <int COMP>
    static __device__ __forceinline__ void update(Raw &V, Raw &T, const AV &inc) {
        if (COMP == 0) { V = add(V, inc); return; }
        AV R = add(T, inc);
        AV s = add(V, R);
        if (COMP == 3) {
            AV z = sub(s, V);
            T = sub(R, z);
        } else {
            AV pa = sub(s, R);
            AV pb = sub(s, pa);
            AV da = sub(V, pa);
            AV db = sub(R, pb);
            T = add(da, db);
        }
        V = s;
    }
    static __device__ __forceinline__ AV c1() { return splat(P::c1()); }
    static __device__ __forceinline__ AV c2() { return splat(P::c2()); }
};

struct VF32 {  // binary32 stored and computed, 4 per vector
    static constexpr int N = 4;
    using P = F32;
    using Raw = float4;
    using AV = float4;
    using RS = float;
    using AS = float;
    static __device__ __forceinline__ AV ld(const Raw &r) { return r; }
    static __device__ __forceinline__ AS lds(RS s) { return s; }
    static __device__ __forceinline__ Raw zero() { return make_float4(0.f, 0.f, 0.f, 0.f); }
    static __device__ __forceinline__ Raw rneg(const Raw &r) { return make_float4(-r.x, -r.y, -r.z, -r.w); }
    static __device__ __forceinline__ RS rneg_s(RS s) { return -s; }
    static __device__ __forceinline__ AV add(const AV &a, const AV &b) {
        return make_float4(__fadd_rn(a.x, b.x), __fadd_rn(a.y, b.y), __fadd_rn(a.z, b.z), __fadd_rn(a.w, b.w)); }
    static __device__ __forceinline__ AV sub(const AV &a, const AV &b) {
        return make_float4(__fsub_rn(a.x, b.x), __fsub_rn(a.y, b.y), __fsub_rn(a.z, b.z), __fsub_rn(a.w, b.w)); }
    static __device__ __forceinline__ AV mul(const AV &a, const AV &b) {
        return make_float4(__fmul_rn(a.x, b.x), __fmul_rn(a.y, b.y), __fmul_rn(a.z, b.z), __fmul_rn(a.w, b.w)); }
    static __device__ __forceinline__ AV splat(AS s) { return make_float4(s, s, s, s); }
    static __device__ __forceinline__ RS get(const Raw &r, int i) {
        return i == 0 ? r.x : i == 1 ? r.y : i == 2 ? r.z : r.w; }
    static __device__ __forceinline__ void set(AV &r, int i, AS s) {
        if (i == 0) r.x = s; else if (i == 1) r.y = s; else if (i == 2) r.z = s; else r.w = s; }
    static __device__ __forceinline__ AS aget(const AV &r, int i) { return get(r, i); }
    static __device__ __forceinline__ float f32(const Raw &r, int i) { return get(r, i); }
    static __device__ __forceinline__ AV shl1(const AV &o, AS r0) { return make_float4(o.y, o.z, o.w, r0); }
    static __device__ __forceinline__ AV shl2(const AV &o, AS r0, AS r1) { return make_float4(o.z, o.w, r0, r1); }
    static __device__ __forceinline__ AV shr1(const AV &o, AS l0) { return make_float4(l0, o.x, o.y, o.z); }
    static __device__ __forceinline__ AV shr2(const AV &o, AS l1, AS l0) { return make_float4(l1, l0, o.x, o.y); }
    template <int COMP>
    static __device__ __forceinline__ void update(Raw &V, Raw &T, const AV &inc) {
        float v[4] = {V.x, V.y, V.z, V.w}, t[4] = {T.x, T.y, T.z, T.w};
        float in[4] = {inc.x, inc.y, inc.z, inc.w};
#pragma unroll
        for (int i = 0; i < 4; i++) wave::update<F32, COMP>(v[i], t[i], in[i]);
        V = make_float4(v[0], v[1], v[2], v[3]);
        T = make_float4(t[0], t[1], t[2], t[3]);
    }
    static __device__ __forceinline__ AV c1() { return splat(1.125f); }
    static __device__ __forceinline__ AV c2() { return splat(F32::c2()); }
};

template <class P, class Store>
struct VWide {  // half / bfloat16 stored, binary32 arithmetic, 8 per vector
    static constexpr int N = 8;
    using Raw = uint4;
    struct AV { float f[8]; };
    using RS = uint16_t;
    using AS = float;
    static __device__ __forceinline__ RS get(const Raw &r, int i) { return VPacked<Store>::get(r, i); }
    static __device__ __forceinline__ AV ld(const Raw &r) {
        AV a;
#pragma unroll
        for (int i = 0; i < 8; i++) a.f[i] = P::ld(get(r, i));
        return a;
    }
    static __device__ __forceinline__ AS lds(RS s) { return P::ld(s); }
    static __device__ __forceinline__ Raw zero() { return make_uint4(0, 0, 0, 0); }
    static __device__ __forceinline__ Raw rneg(const Raw &r) { return VPacked<Store>::rneg(r); }
    static __device__ __forceinline__ RS rneg_s(RS s) { return s ^ 0x8000u; }
#define WAVE_VW_OP(name, fn)                                                     \
    static __device__ __forceinline__ AV name(const AV &a, const AV &b) {        \
        AV r;                                                                    \
        _Pragma("unroll") for (int i = 0; i < 8; i++) r.f[i] = fn(a.f[i], b.f[i]); \
        return r;                                                                \
    }
    WAVE_VW_OP(add, __fadd_rn)
    WAVE_VW_OP(sub, __fsub_rn)
    WAVE_VW_OP(mul, __fmul_rn)
#undef WAVE_VW_OP
    static __device__ __forceinline__ AV splat(AS s) {
        AV a;
#pragma unroll
        for (int i = 0; i < 8; i++) a.f[i] = s;
        return a;
    }
    static __device__ __forceinline__ void set(AV &r, int i, AS s) { r.f[i] = s; }
    static __device__ __forceinline__ AS aget(const AV &r, int i) { return r.f[i]; }
    static __device__ __forceinline__ float f32(const Raw &r, int i) { return Store::to_f32(get(r, i)); }
    static __device__ __forceinline__ AV shl1(const AV &o, AS r0) {
        AV a;
#pragma unroll
        for (int i = 0; i < 7; i++) a.f[i] = o.f[i + 1];
        a.f[7] = r0;
        return a;
    }
    static __device__ __forceinline__ AV shl2(const AV &o, AS r0, AS r1) {
        AV a;
#pragma unroll
        for (int i = 0; i < 6; i++) a.f[i] = o.f[i + 2];
        a.f[6] = r0;
        a.f[7] = r1;
        return a;
    }
    static __device__ __forceinline__ AV shr1(const AV &o, AS l0) {
        AV a;
        a.f[0] = l0;
#pragma unroll
        for (int i = 1; i < 8; i++) a.f[i] = o.f[i - 1];
        return a;
    }
    static __device__ __forceinline__ AV shr2(const AV &o, AS l1, AS l0) {
        AV a;
        a.f[0] = l1;
        a.f[1] = l0;
#pragma unroll
        for (int i = 2; i < 8; i++) a.f[i] = o.f[i - 2];
        return a;
    }
    template <int COMP>
    static __device__ __forceinline__ void update(Raw &V, Raw &T, const AV &inc) {
        Raw v2 = V, t2 = T;
#pragma unroll
        for (int i = 0; i < 8; i++) {
            uint16_t v = get(V, i), t = get(T, i);
            wave::update<P, COMP>(v, t, inc.f[i]);
            VPacked<Store>::set(v2, i, v);
            VPacked<Store>::set(t2, i, t);
        }
        V = v2;
        T = t2;
    }
    static __device__ __forceinline__ AV c1() { return splat(1.125f); }
    static __device__ __forceinline__ AV c2() { return splat(P::c2()); }
};

template <class P> struct VecOf;
template <> struct VecOf<F16> { using T = VPacked<F16>; };
template <> struct VecOf<BF16> { using T = VPacked<BF16>; };
template <> struct VecOf<F32> { using T = VF32; };
template <> struct VecOf<F16W> { using T = VWide<F16W, F16>; };
template <> struct VecOf<BF16W> { using T = VWide<BF16W, BF16>; };
template <> struct VecOf<F16WP> { using T = VWide<F16WP, F16>; };

// Vector policies of the pair precision (binary32 multipliers, CoefOf).
template <class V> struct VPairs { static constexpr bool value = false; };
template <class Store> struct VPairs<VWide<PairArith<Store>, Store>> { static constexpr bool value = true; };

template <class V>
__device__ __forceinline__ typename V::AV vstencil(const typename V::AV &fm3, const typename V::AV &fm1,
                                                   const typename V::AV &fp1, const typename V::AV &fp3) {
    typename V::AV t1 = V::sub(fp1, fm1);
    typename V::AV t2 = V::sub(fp3, fm3);
    return V::sub(V::mul(V::c1(), t1), V::mul(V::c2(), t2));
}

// The 16-byte vector of a field at element index q.
template <class V>
__device__ __forceinline__ typename V::Raw &at(void *f, int64_t q) {
    return *reinterpret_cast<typename V::Raw *>(static_cast<char *>(f) + q * sizeof(typename V::RS));
}

}  // namespace wave
