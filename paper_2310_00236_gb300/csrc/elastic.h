// elastic.h -- parameters of the 2D elastic kernels.
//
// Boundary kinds per face (x-lo, x-hi, y-lo, y-hi):
//   periodic (both faces of an axis): wrap;
//   rigid: frictionless rigid wall on the half points -1/2 and N-1/2: the
//     normal velocity and the shear stress are odd about it (zero on it; the
//     stored point N-1 lies on the high wall and is held at zero), the
//     tangential velocity and the normal stresses are even;
//   free (y-lo only): traction-free surface on the node row 0 by stress
//     imaging: syy is held at zero on row 0 and, above it, syy and sxy are odd
//     images and vx, vy even images of the rows below; on row 0 the host puts
//     the modulus of sxx under zero normal traction into l2m and zero into lam.
// Each keeps the stress-to-velocity map the exact negative adjoint of the
// velocity-to-strain-rate map (with weight 1/2 on the vx and sxx points of a
// free surface row), so the discrete energy is exactly conserved in exact
// arithmetic.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace wave {

struct ElParams {
    int n[2];
    int bc[4];
    int64_t sy;                 // row pitch in elements
    void *f[5], *t[5];          // vx, vy, sxx, syy, sxy and their compensations
    const void *c[5];           // bx, by, l2m, lam, mu (arrays) or nullptr
    uint32_t c_uni[5];          // uniform values (storage bits)
    int64_t src_q;              // pitched index of the v_y source, -1 none
    const void *src;            // arithmetic-format increments per global step
    int64_t src_nt;
    int64_t step;
    int64_t *step_dev;          // strips: the step index in device memory (read by the
                                // velocity launch, advanced by the stress launch), or nullptr
    int energy;
    double *e_part;
    unsigned int *e_count;
    double *e_out;
    double e_factor;
};

cudaError_t elastic_half_step(const ElParams &e, int prec, int comp, int half, cudaStream_t st);
unsigned elastic_blocks(const int n[2]);

// Row-strip kernels (elastic_strips.cu): one warp per strip of 32 16-byte
// vectors by yc rows; the energy goes through item partials.
struct ElStripLaunch {
    int nitems, yc, wpb, grid;
    double *item_part;  // [nitems]
};
int elastic_strip_items(int prec, int nx, int ny, int yc);
cudaError_t elastic_strip_half_step(const ElParams &e, int prec, int comp, int half, const ElStripLaunch &L,
                                    cudaStream_t st);

}  // namespace wave
