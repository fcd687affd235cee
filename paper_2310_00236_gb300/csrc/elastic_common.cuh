// elastic_common.cuh -- boundary images and field / coefficient indices
// shared by the 2D elastic kernels.
#pragma once
#include "elastic.h"

namespace wave {

enum { EBC_PERIODIC = 0, EBC_RIGID = 1, EBC_FREE = 2 };
enum { F_VX = 0, F_VY = 1, F_SXX = 2, F_SYY = 3, F_SXY = 4 };
enum { C_BX = 0, C_BY = 1, C_L2M = 2, C_LAM = 3, C_MU = 4 };

// Image of index m along an axis with N points (see elastic.h for the rules).
// node: the field sits on the axis' nodes (else on its half points); odd: the
// field is odd about a rigid wall (normal velocity, shear stress); odd_free:
// the field is odd about a free surface (the stresses; velocities are even).
// Returns +1 / -1 (sign) or 0 (reads zero).
__device__ __forceinline__ int emap(int m, int N, int lo, int hi, bool node, bool odd, bool odd_free,
                                    int &out) {
    if (m >= 0 && m < N) { out = m; return 1; }
    const int bc = m < 0 ? lo : hi;
    if (bc == EBC_PERIODIC) { out = m < 0 ? m + N : m - N; return 1; }
    if (bc == EBC_FREE) {
        // mirror plane: node row 0 (a free surface is a low face)
        out = node ? -m : -1 - m;
        return odd_free ? -1 : 1;
    }
    if (node) {
        out = m < 0 ? -1 - m : 2 * N - 1 - m;
        return odd ? -1 : 1;
    }
    if (m == -1) {
        if (odd) return 0;
        out = 0;
        return 1;
    }
    out = m < 0 ? -2 - m : 2 * N - 2 - m;
    return odd ? -1 : 1;
}

}  // namespace wave
