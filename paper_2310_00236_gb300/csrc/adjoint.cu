// adjoint.cu -- kernels of the discrete adjoint (gradient of a trace misfit
// with respect to the velocity model). Not in the paper.
//
// Forward step n (scaled variables, rounded multipliers a, b):
//   v^{n+1/2} = v^{n-1/2} + a G p^n,    p^{n+1} = p^n + b (Dv v^{n+1/2} + s^n)
// with G the staggered gradient and Dv the staggered divergence. On the
// unknowns the scheme updates, Dv^T = -G and G^T = -Dv (the discrete
// operator is skew). Reverse-mode differentiation of the step, written for
// mu~ = b * pbar and nu~ = a * vbar, is therefore the same leapfrog with the
// multipliers negated, run backwards in time:
//   mu~ += b r^n at the receivers (r^n: dJ/dtrace of step n)
//   g   += mu~ * (Dv v^{n+1/2} + s^n)                 (dJ/db = g / b)
//   nu~ = nu~ - a G mu~,   mu~ = mu~ - b Dv nu~
// and dJ/dc = (2 / c) g, since b is proportional to c^2. The rigid-wall nodes
// (p held at zero) take no residual, which keeps mu~ zero there and makes the
// skew form exact. The leapfrog half steps reuse the binary32 forward kernels;
// this file holds the residual injection, the gradient accumulation and the
// final scaling.
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "acoustic_common.cuh"
#include "adjoint.h"

namespace wave {

// mu[q_r] += w_r * res[r] for every receiver. One thread per distinct point:
// group g holds receivers order[start[g] .. start[g+1]) (ascending receiver
// index), so points shared by several receivers add them in receiver order.
__global__ void adj_inject_kernel(float *mu, const int64_t *rec_q, const float *rec_w, const int *order,
                                  const int *start, int ngroups, const float *res) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= ngroups) return;
    const int r0 = order[start[g]];
    float acc = mu[rec_q[r0]];
    for (int u = start[g]; u < start[g + 1]; u++) {
        const int r = order[u];
        const float w = rec_w[r];
        if (w != 0.f) acc = __fadd_rn(acc, __fmul_rn(w, res[r]));
    }
    mu[rec_q[r0]] = acc;
}

template <int FMT>
__device__ __forceinline__ float ld_f32(const void *f, int64_t q) {
    if (FMT == ADJ_F32) return static_cast<const float *>(f)[q];
    const uint16_t u = static_cast<const uint16_t *>(f)[q];
    if (FMT == ADJ_BF16) return __uint_as_float((uint32_t)u << 16);
    __half_raw hr;
    hr.x = u;
    return __half2float(__half(hr));
}

// Eight consecutive storage values from v at q (q a multiple of 8: 16-byte
// aligned for 16-bit storage, 32-byte for binary32), as binary32.
template <int FMT>
__device__ __forceinline__ void ld8(const void *v, int64_t q, float f[8]) {
    if (FMT == ADJ_F32) {
        const float4 *p = reinterpret_cast<const float4 *>(static_cast<const float *>(v) + q);
        const float4 a = __ldg(p), b = __ldg(p + 1);
        f[0] = a.x; f[1] = a.y; f[2] = a.z; f[3] = a.w;
        f[4] = b.x; f[5] = b.y; f[6] = b.z; f[7] = b.w;
        return;
    }
    const uint4 u = __ldg(reinterpret_cast<const uint4 *>(static_cast<const uint16_t *>(v) + q));
    const uint32_t w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
    for (int e = 0; e < 8; e++) {
        const uint16_t h = (uint16_t)(e & 1 ? w[e >> 1] >> 16 : w[e >> 1] & 0xFFFFu);
        if (FMT == ADJ_BF16) {
            f[e] = __uint_as_float((uint32_t)h << 16);
        } else {
            __half_raw hr;
            hr.x = h;
            f[e] = __half2float(__half(hr));
        }
    }
}

// g += mu * (sum_c D_c v_c + s) at every p node, in binary32, from the forward
// velocities of the step (storage format FMT) and the scaled source value.
// One thread per 8 consecutive x nodes: the x stencils share 11 values of v_x,
// the y and z stencils read 4 rows / planes of 8 values each. Per node the
// operations and their order are those of one stencil per axis, x then y then z.
template <int FMT, int NDIM>
__global__ void __launch_bounds__(128) adj_grad_kernel(AdjGradParams P) {
    const int i0 = (blockIdx.x * blockDim.x + threadIdx.x) * 8;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = NDIM == 3 ? (int)blockIdx.z : 0;
    const int nx = P.n[0];
    if (i0 >= nx || j >= P.n[1]) return;
    const int64_t row = P.sy * j + P.sz * k;  // element (0, j, k)
    const float c1 = 1.125f, c2 = 1.0f / 24.0f;
    float R[8];
    // x: v_x at i0-2 .. i0+8 (images outside 0..nx-1)
    {
        float f[11];
        if (i0 >= 2 && i0 + 9 <= nx) {
            ld8<FMT>(P.v[0], row + i0, f + 2);
            f[0] = ld_f32<FMT>(P.v[0], row + i0 - 2);
            f[1] = ld_f32<FMT>(P.v[0], row + i0 - 1);
            f[10] = ld_f32<FMT>(P.v[0], row + i0 + 8);
        } else {
            // the nodes below nx read x indices up to nx; past that the
            // values only feed nodes that are not stored, and are not loaded
#pragma unroll
            for (int t = 0; t < 11; t++) {
                f[t] = 0.f;
                if (i0 - 2 + t <= nx) {
                    int mm;
                    img_half(i0 - 2 + t, nx, P.bc[0], mm);
                    f[t] = ld_f32<FMT>(P.v[0], row + mm);
                }
            }
        }
#pragma unroll
        for (int e = 0; e < 8; e++) R[e] = 0.f + (c1 * (f[e + 2] - f[e + 1]) - c2 * (f[e + 3] - f[e]));
    }
    // y and z: rows j-2 .. j+1 and planes k-2 .. k+1 of the own 8 columns
#pragma unroll
    for (int c = 1; c < NDIM; c++) {
        const int m = c == 1 ? j : k;
        const int64_t str = c == 1 ? P.sy : P.sz;
        float f[4][8];
#pragma unroll
        for (int t = 0; t < 4; t++) {
            int mm;
            img_half(m - 2 + t, P.n[c], P.bc[c], mm);
            ld8<FMT>(P.v[c], row - str * m + str * mm + i0, f[t]);
        }
#pragma unroll
        for (int e = 0; e < 8; e++) R[e] += c1 * (f[2][e] - f[1][e]) - c2 * (f[3][e] - f[0][e]);
    }
    const int64_t q0 = row + i0;
    if (P.src_q >= q0 && P.src_q < q0 + 8) {
#pragma unroll
        for (int e = 0; e < 8; e++)
            if (q0 + e == P.src_q) R[e] += P.src_value;
    }
    float4 *g4 = reinterpret_cast<float4 *>(P.g + q0);
    const float4 *m4 = reinterpret_cast<const float4 *>(P.mu + q0);
    if (i0 + 8 <= nx) {
        const float4 ma = m4[0], mb = m4[1];
        float4 ga = g4[0], gb = g4[1];
        ga.x += ma.x * R[0]; ga.y += ma.y * R[1]; ga.z += ma.z * R[2]; ga.w += ma.w * R[3];
        gb.x += mb.x * R[4]; gb.y += mb.y * R[5]; gb.z += mb.z * R[6]; gb.w += mb.w * R[7];
        g4[0] = ga;
        g4[1] = gb;
    } else {
#pragma unroll
        for (int e = 0; e < 8; e++)
            if (i0 + e < nx) P.g[q0 + e] += P.mu[q0 + e] * R[e];
    }
}

// out[i + nx (j + ny k)] = g[q] * two_over_c[...]: dJ/dc, unpitched.
__global__ void adj_finish_kernel(float *out, const float *g, const float *two_over_c, int nx, int ny,
                                  int nz, int64_t sy, int64_t sz) {
    const int64_t npts = (int64_t)nx * ny * nz;
    for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < npts;
         u += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(u % nx);
        const int j = (int)((u / nx) % ny);
        const int k = (int)(u / ((int64_t)nx * ny));
        out[u] = g[i + sy * j + sz * k] * two_over_c[u];
    }
}

// dst[i] = -(binary32 value of the multiplier src[i]), over the pitched array.
template <int FMT>
__global__ void adj_neg_coef_kernel(const void *src, float *dst, int64_t total) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = -ld_f32<FMT>(src, i);
}

cudaError_t adj_neg_coef(const void *src, int fmt, float *dst, int64_t total, cudaStream_t st) {
    const int blocks = (int)std::min<int64_t>((total + 255) / 256, 65535);
    if (fmt == ADJ_F32) adj_neg_coef_kernel<ADJ_F32><<<blocks, 256, 0, st>>>(src, dst, total);
    else if (fmt == ADJ_BF16) adj_neg_coef_kernel<ADJ_BF16><<<blocks, 256, 0, st>>>(src, dst, total);
    else adj_neg_coef_kernel<ADJ_F16><<<blocks, 256, 0, st>>>(src, dst, total);
    return cudaGetLastError();
}

cudaError_t adj_inject(float *mu, const int64_t *rec_q, const float *rec_w, const int *order, const int *start,
                       int ngroups, const float *res, cudaStream_t st) {
    if (ngroups <= 0) return cudaSuccess;
    adj_inject_kernel<<<(ngroups + 127) / 128, 128, 0, st>>>(mu, rec_q, rec_w, order, start, ngroups, res);
    return cudaGetLastError();
}

template <int FMT>
static void launch_grad(const AdjGradParams &P, int ndim, cudaStream_t st) {
    // 32 x 4 threads of 8 x nodes each: 256 x 4 nodes per block
    dim3 block(32, 4, 1);
    dim3 grid((P.n[0] + 255) / 256, (P.n[1] + 3) / 4, ndim == 3 ? P.n[2] : 1);
    if (ndim == 3) adj_grad_kernel<FMT, 3><<<grid, block, 0, st>>>(P);
    else adj_grad_kernel<FMT, 2><<<grid, block, 0, st>>>(P);
}

cudaError_t adj_grad(const AdjGradParams &P, int ndim, int fmt, cudaStream_t st) {
    switch (fmt) {
    case ADJ_F32: launch_grad<ADJ_F32>(P, ndim, st); break;
    case ADJ_BF16: launch_grad<ADJ_BF16>(P, ndim, st); break;
    default: launch_grad<ADJ_F16>(P, ndim, st); break;
    }
    return cudaGetLastError();
}

cudaError_t adj_finish(float *out, const float *g, const float *two_over_c, const int n[3], int64_t sy,
                       int64_t sz, cudaStream_t st) {
    const int64_t npts = (int64_t)n[0] * n[1] * n[2];
    const int blocks = (int)std::min<int64_t>((npts + 255) / 256, 65535);
    adj_finish_kernel<<<blocks, 256, 0, st>>>(out, g, two_over_c, n[0], n[1], n[2], sy, sz);
    return cudaGetLastError();
}

}  // namespace wave
