// strip_common.cuh -- helpers of the 2D row-strip kernels (one warp per strip
// of 32 vectors, x neighbours by warp shuffle): shuffles of raw scalars,
// element replacement in raw vectors, multiplier vectors and partial stores.
#pragma once
#include "vec_policy.cuh"

namespace wave {

// A raw scalar moved delta lanes up or down the warp (bit moves only).
template <class RS>
__device__ __forceinline__ RS shfl_rs(RS v, int delta, bool up) {
    uint32_t u;
    if (sizeof(RS) == 2) u = (uint32_t)(*reinterpret_cast<const uint16_t *>(&v));
    else u = *reinterpret_cast<const uint32_t *>(&v);
    u = up ? __shfl_up_sync(0xffffffffu, u, delta) : __shfl_down_sync(0xffffffffu, u, delta);
    RS r;
    if (sizeof(RS) == 2) *reinterpret_cast<uint16_t *>(&r) = (uint16_t)u;
    else *reinterpret_cast<uint32_t *>(&r) = u;
    return r;
}

// Element e of a raw vector replaced (bit moves only).
template <class RS, class Raw>
__device__ __forceinline__ void raw_set(Raw &r, int e, RS s);
template <>
__device__ __forceinline__ void raw_set<uint16_t, uint4>(uint4 &r, int e, uint16_t s) {
    uint32_t *w = (e >> 1) == 0 ? &r.x : (e >> 1) == 1 ? &r.y : (e >> 1) == 2 ? &r.z : &r.w;
    *w = (e & 1) ? ((*w & 0xFFFFu) | ((uint32_t)s << 16)) : ((*w & 0xFFFF0000u) | s);
}
template <>
__device__ __forceinline__ void raw_set<float, float4>(float4 &r, int e, float s) {
    if (e == 0) r.x = s; else if (e == 1) r.y = s; else if (e == 2) r.z = s; else r.w = s;
}

// Multipliers of the vector at q (per-point array or uniform value); the pair
// precision keeps them in binary32 (two 16-byte loads per vector of 8).
template <class V>
__device__ __forceinline__ typename V::AV coef_v(const void *arr, uint32_t uni, int64_t q) {
    if constexpr (VPairs<V>::value) {
        typename V::AV a;
        if (arr) {
            const float4 *f = reinterpret_cast<const float4 *>(static_cast<const float *>(arr) + q);
            const float4 lo = f[0], hi = f[1];
            a.f[0] = lo.x; a.f[1] = lo.y; a.f[2] = lo.z; a.f[3] = lo.w;
            a.f[4] = hi.x; a.f[5] = hi.y; a.f[6] = hi.z; a.f[7] = hi.w;
            return a;
        }
        return V::splat(__uint_as_float(uni));
    } else {
        if (arr) return V::ld(*reinterpret_cast<const typename V::Raw *>(
                     static_cast<const char *>(arr) + q * sizeof(typename V::RS)));
        typename V::RS s;
        from_bits(uni, s);
        return V::splat(V::lds(s));
    }
}

// Store the first nvalid elements of a vector (all of it when nvalid == N).
template <class V>
__device__ __forceinline__ void store_vec(void *f, int64_t q, const typename V::Raw &r, int nvalid) {
    if (nvalid >= V::N) {
        at<V>(f, q) = r;
    } else {
        typename V::RS *s = static_cast<typename V::RS *>(f) + q;
#pragma unroll
        for (int e = 0; e < V::N; e++)
            if (e < nvalid) s[e] = V::get(r, e);
    }
}

}  // namespace wave
