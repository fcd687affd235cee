// adjoint.h -- kernels of the discrete adjoint used by the C ABI.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace wave {

enum { ADJ_F16 = 0, ADJ_BF16 = 1, ADJ_F32 = 2 };  // storage format of the forward velocities

struct AdjGradParams {
    int n[3];
    int bc[3];              // BC_PERIODIC / BC_RIGID per axis
    int64_t sy, sz;         // pitches (elements)
    const void *v[3];       // forward v_c^{n+1/2}, storage format
    const float *mu;        // adjoint pressure mu~ (binary32, pitched)
    float *g;               // gradient accumulator (binary32, pitched)
    int64_t src_q;          // source point (pitched index) or -1
    float src_value;        // scaled source value of the step (0 past the table)
};

// order / start: receivers grouped by point (see adjoint.cu), ngroups points
cudaError_t adj_inject(float *mu, const int64_t *rec_q, const float *rec_w, const int *order, const int *start,
                       int ngroups, const float *res, cudaStream_t st);
// dst[i] = -src[i] as binary32 (src in storage format fmt), i < total
cudaError_t adj_neg_coef(const void *src, int fmt, float *dst, int64_t total, cudaStream_t st);
cudaError_t adj_grad(const AdjGradParams &P, int ndim, int fmt, cudaStream_t st);
cudaError_t adj_finish(float *out, const float *g, const float *two_over_c, const int n[3], int64_t sy,
                       int64_t sz, cudaStream_t st);

}  // namespace wave
