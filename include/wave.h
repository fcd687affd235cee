/*
 * wave.h -- C ABI of the GB300 half-precision staggered-grid wave library.
 *
 * The library advances the first-order acoustic system (Eq. 1 of Gao & Harms,
 * "Half precision wave simulation", arXiv 2310.00236; extended to 3D by adding
 * v_z and d/dz) and the 2D isotropic elastic velocity-stress system (Eq. 2,
 * Appendix A) with the fourth-order staggered stencil [1/24, -9/8, 9/8, -1/24]
 * of Section 3 and the staggered leapfrog in time, storing every field in a
 * chosen format and doing every solution update either as a plain sum
 * (Algorithm 1) or as a compensated sum (Algorithm 2 with sum_3op / sum_6op,
 * Code 1 / Code 2 of Section 4).
 *
 * Conventions for every entry point:
 *  - Nothing is thrown across the ABI; every call returns a wave_status and,
 *    on failure, wave_last_error() describes it (thread-local string).
 *  - Host arrays passed in are owned by the caller and copied before return.
 *  - Grid arrays are x fastest: value (i, j, k) sits at i + n[0]*(j + n[1]*k).
 *  - Work is queued on the CUDA stream given to wave_create. wave_step returns
 *    before the GPU finishes; CUDA errors it causes surface at the next call
 *    that synchronises (wave_energy, wave_get_*, wave_sync) as WAVE_ECUDA.
 *  - After any error other than WAVE_EINVAL, WAVE_ERANGE on input data, or
 *    WAVE_ENOTIMPL, the context is poisoned: later calls on it return
 *    WAVE_ESTATE until it is destroyed.
 *  - A context is not thread-safe; distinct contexts are independent.
 *
 * Grid layout (the reading of Fig. 1, whose image is not available): along
 * an axis with N cells of spacing h, pressure (and the normal stresses) sit
 * on the nodes m*h, m = 0..N-1; the velocity component along that axis sits
 * at (m + 1/2)*h. Every field is stored as an N-point array per axis with the
 * same (i, j, k) indexing. Boundaries per axis:
 *  - WAVE_BC_PERIODIC: the stencil wraps around the domain (Section 3).
 *  - WAVE_BC_RIGID (acoustic): p = 0 on walls at node 0 and node N. The
 *    scheme reads p as odd and the normal velocity as even about each wall,
 *    which is the periodic scheme on the doubled domain, so the discrete
 *    energy stays exactly conserved. Node 0 is stored and held at 0, node N
 *    is not stored.
 * Elastic boundaries are described at wave_create.
 */
#ifndef WAVE_H
#define WAVE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct wave_ctx wave_ctx;

typedef enum {
    WAVE_OK = 0,
    WAVE_EINVAL = 1,    /* bad argument; context unchanged */
    WAVE_ENOMEM = 2,    /* device or host allocation failed */
    WAVE_ERANGE = 3,    /* coefficient or input value outside the storage format's normal range */
    WAVE_ECUDA = 4,     /* a CUDA call failed (message has the CUDA error) */
    WAVE_ETIMEOUT = 5,  /* a bounded device wait expired */
    WAVE_ESTATE = 6,    /* context poisoned by an earlier error */
    WAVE_ENOTIMPL = 7   /* valid request this build does not implement */
} wave_status;

typedef enum { WAVE_ACOUSTIC = 0, WAVE_ELASTIC = 1 } wave_physics;

/* Storage format of fields, compensations and coefficients, and the format
 * the arithmetic is done in.
 *   WAVE_FP32, WAVE_FP16, WAVE_BF16: store and compute in that format; every
 *     +, -, * is one correctly rounded operation of the format (Section 2).
 *   WAVE_FP16_F32ARITH, WAVE_BF16_F32ARITH: store in half / bfloat16, compute
 *     in binary32 registers; with compensation the update forms s = V + (T +
 *     inc) in binary32 and stores V' = RN(s), T' = RN(s - V') (not in the paper).
 *   WAVE_FP16_PAIRS: as WAVE_FP16_F32ARITH with compensation, except that
 *     every stencil tap reads RN32(V + T), the stored value plus its carried
 *     compensation, instead of V (not the paper's scheme, where the stencil
 *     reads V: the binary16 pair then acts as a ~22-bit value in the stencil,
 *     which removes the rounding error of the stored value from the
 *     differences); the multipliers (acoustic a, b; elastic bx, by, l2m, lam,
 *     mu) are kept in binary32 (their rounding to binary16 would then be the
 *     largest error left; per-point arrays cost 4 bytes a point). Needs
 *     compensation (WAVE_EINVAL without). Acoustic 3D: the one-pass step
 *     where it applies (t_p then alternates between two buffers), else the
 *     two-kernel streaming step, else one thread per point (the same choice
 *     as the other precisions); 2D: the cluster-resident steps or the two-launch row
 *     strips (not kernel 3). No z slabs and no adjoint (WAVE_ENOTIMPL);
 *     wave_energy_acoustic_static does not take it (WAVE_EINVAL).
 *   WAVE_FP64 is accepted only by the CPU oracle; wave_create returns
 *     WAVE_ENOTIMPL for it. */
typedef enum {
    WAVE_FP64 = 0,
    WAVE_FP32 = 1,
    WAVE_FP16 = 2,
    WAVE_BF16 = 3,
    WAVE_FP16_F32ARITH = 4,
    WAVE_BF16_F32ARITH = 5,
    WAVE_FP16_PAIRS = 6
} wave_precision;

/* Solution update: plain V += inc (Algorithm 1), or the compensated update of
 * Algorithm 2 with the carried term added after the coefficient multiply:
 * R = T + inc; (V, T) = sum(V, R) with sum_3op (Code 1) or sum_6op (Code 2).
 * For the *_F32ARITH precisions WAVE_COMP_3OP and WAVE_COMP_6OP both select
 * the binary32 compensated form described above. */
typedef enum { WAVE_COMP_NONE = 0, WAVE_COMP_3OP = 3, WAVE_COMP_6OP = 6 } wave_comp;

typedef enum { WAVE_BC_PERIODIC = 0, WAVE_BC_RIGID = 1, WAVE_BC_FREE = 2 } wave_bc;

typedef enum {
    WAVE_F_P = 0, WAVE_F_VX = 1, WAVE_F_VY = 2, WAVE_F_VZ = 3,
    WAVE_F_SXX = 4, WAVE_F_SYY = 5, WAVE_F_SXY = 6
} wave_field;

typedef struct {
    int32_t ndim;   /* 2 or 3 (elastic: 2) */
    int64_t n[3];   /* cells per axis, x first; n[2] ignored in 2D. Each >= 8. */
} wave_grid;

typedef struct {
    wave_physics kind;
    const double *rho;  /* density, host, one value per p node (x fastest) */
    const double *vp;   /* sound speed (acoustic) or P-wave speed (elastic), host */
    const double *vs;   /* S-wave speed (elastic), host; NULL for acoustic */
    int32_t bc[6];      /* per face: x-lo, x-hi, y-lo, y-hi, z-lo, z-hi.
                           Acoustic: each axis uses one code on both faces. */
} wave_materials;

typedef struct {
    double field_scale;  /* P0 > 0: stored p^ = p / P0 and v^ = v * Z0 / P0
                            (Z0 = max(rho) * max(vp)); default 1.0 */
    int32_t kernel;      /* 0: automatic (3D: the one-pass step where it applies, else
                            the two-kernel streaming step when n[0] is a multiple of
                            the 16-byte vector width, else one thread per point;
                            2D acoustic: the cluster-resident steps of kernel 4
                            for small grids (a band of at most 5120 points, e.g.
                            256^2), else the row strips of kernel 2);
                            1: one-thread-per-point kernels only; 2: two-kernel
                            streaming step (2D acoustic: row strips, one warp per
                            strip of 16-byte vectors, one launch per half step,
                            any size); 3: one-pass step (3D: both half steps in
                            one kernel; needs n[0] a multiple of 64 (32 for binary32),
                            rigid x faces and a uniform density, else as 0; 2D
                            acoustic: one-pass row strips, both half steps in one
                            launch, keeping a second buffer set of p, v and t_v; a
                            batch of such contexts also tries them in its tuner);
                            4: 2D acoustic only, cluster-resident steps: the rows
                            cut into bands over one thread-block cluster of up to
                            16 CTAs, the whole state in their shared memory, rows
                            past a band's edge read from the neighbouring CTA's
                            shared memory, a cluster barrier after each half step,
                            and every step of a wave_step call (energies, receivers
                            and source included) in one launch; WAVE_EINVAL if the
                            state does not fit (about 3.6 MB: 300k points at 12
                            bytes a point). Every choice gives the same bits. */
    int32_t zchunk;      /* z planes per thread block of the 3D kernels; rows per
                            work item of the 2D row strips (0: automatic) */
    int32_t z_cut;       /* 3D acoustic only: the context is a z slab of a larger
                            grid (domain decomposition along z, for a problem split
                            over several GPUs). Bit 0: the z-lo face is a cut, bit 1:
                            the z-hi face is a cut; a cut face reads the two ghost
                            planes set by wave_set_z_ghosts instead of a boundary
                            image, and the slab steps by wave_half_step. 0: the
                            context is the whole grid. */
    int32_t reserved[5];
    double z0;           /* > 0: the impedance scale Z0 to use instead of
                            max(rho) * max(vp) of this context's materials (every slab
                            of a grid must use the grid's Z0); 0: computed */
    const double *rho_above;  /* z_cut bit 1: the density of the grid plane just above
                            the slab (host, n[0] * n[1], x fastest), for the z
                            multiplier of the slab's last plane (rho averaged
                            across the cut); else NULL */
} wave_options;

/* Optional device allocator for the context's memory (for instance a caching
 * allocator of the host application). alloc returns NULL on failure. Process
 * wide; passing NULLs restores cudaMallocAsync / cudaFreeAsync on the
 * context's stream. */
typedef void *(*wave_alloc_fn)(size_t bytes, void *stream, void *user);
typedef void (*wave_free_fn)(void *ptr, size_t bytes, void *stream, void *user);
wave_status wave_set_allocator(wave_alloc_fn alloc, wave_free_fn free_fn, void *user);

/*
 * wave_create -- Section 3 (problem statement), Section 5 "Range" (units).
 * Builds a context: validates the arguments, nondimensionalises the materials
 * into per-point multipliers, rounds each once to the storage format, checks
 * their range, and allocates the device state (all fields zero).
 *   grid      cells per axis (>= 8 each)
 *   spacing   h per axis in metres; all used axes must be equal (else EINVAL)
 *   mat       host material arrays (copied) and boundary codes
 *   dt        time step in seconds (> 0). Stability needs
 *             max(vp) * dt / h <= 1 / (sqrt(ndim) * (9/8 + 1/24)).
 *   prec, compensated   see the enums above
 *   opt       NULL for defaults
 *   cuda_stream  cudaStream_t to queue work on (NULL = legacy default stream)
 *   out       receives the context
 * Acoustic multipliers (binary64 in exactly this order, then one rounding):
 *   Z0 = max(rho) * max(vp)
 *   b   = (((dt * rho) * vp) * vp) / (Z0 * h)          at p nodes
 *   a_c = ((dt * Z0) / h) / rho_c                      at v_c points
 *   rho_c = (rho[m] + rho[m+1]) * 0.5 along axis c; at the last cell the
 *   neighbour wraps (periodic) or is the cell itself (rigid).
 * Elastic multipliers (WAVE_ELASTIC, 2D, Eq. 2), same rules:
 *   Z0 = max(rho) * max(vp); bx = ((dt * Z0) / h) / rho_x, by likewise, with
 *   rho_x, rho_y two-point averages as rho_c above;
 *   mu = (rho * vs) * vs, lambda = ((rho * vp) * vp) - (2 * mu) at each node;
 *   l2m = ((dt * (lambda + 2 * mu)) / Z0) / h, lam = ((dt * lambda) / Z0) / h;
 *   at the shear points mu_xy = 4 / (1/mu00 + 1/mu10 + 1/mu01 + 1/mu11), the
 *   harmonic mean of the four surrounding nodes (0 if any is 0), and
 *   mu = ((dt * mu_xy) / Z0) / h. Neighbours past the last point wrap
 *   (periodic) or are clamped. On the row of a free surface (j = 0):
 *   l2m = ((dt * M) / Z0) / h with M = ((4 * mu) * (lambda + mu)) /
 *   (lambda + 2 * mu), the modulus of sxx under zero normal traction, and
 *   lam = 0.
 * Elastic boundaries: x faces PERIODIC/PERIODIC or RIGID/RIGID; y faces
 * PERIODIC/PERIODIC or (RIGID or FREE)/RIGID. RIGID is a frictionless rigid
 * wall on the half points -1/2 and N-1/2 (normal velocity and shear stress odd
 * about it and zero on it, the other fields even); the stored points on the
 * high wall are held at zero. FREE (y-lo) is the traction-free surface of
 * Appendix A, on the node row 0, by stress imaging: syy is held at zero on
 * row 0, and above it syy and sxy read as odd images and vx, vy as even images
 * of the rows below. Both keep the discrete operator skew (with weight 1/2 on
 * the vx and sxx points of the surface row), so the energy is conserved in
 * exact arithmetic.
 * Errors: EINVAL (bad grid, spacing, dt, enum, NULL pointer, unsupported BC),
 * ERANGE (a multiplier is not a positive normal number of the storage format,
 * or a material value is not positive and finite; a free surface needs
 * vs > 0 on its row), ENOTIMPL (WAVE_FP64), ENOMEM, ECUDA.
 */
wave_status wave_create(const wave_grid *grid, const double spacing[3],
                        const wave_materials *mat, double dt, wave_precision prec,
                        wave_comp compensated, const wave_options *opt, void *cuda_stream,
                        wave_ctx **out);

/* wave_set_initial -- initial state (Section 3: the paper starts at rest; the
 * benchmark configurations start from a Gaussian pressure). host_values holds
 * one physical value per grid point (x fastest). Stored values are
 * RN(p / P0) for pressure and stresses, RN((v * Z0) / P0) for velocities,
 * rounded once to the storage format. Values a rigid wall or a free surface
 * holds at zero are set to zero. The field's compensation is reset to zero. Acoustic p is
 * p^0; velocities are v^{-1/2}. Synchronous with respect to host_values.
 * Errors: EINVAL (field not in this physics, NULL), ERANGE (non-finite input
 * or a value that overflows the storage format). */
wave_status wave_set_initial(wave_ctx *ctx, wave_field field, const double *host_values);

/* wave_set_source -- point source (Section 3: a Ricker wavelet on p at one
 * point; Appendix A: a vertical force on v_y). wavelet[s] is the physical
 * source amplitude at global step s, for s < nt; later steps have none. It is
 * stored as s^ = RN(w * (Z0 / (P0 * h^(d-1)))) in the arithmetic format and
 * added to the right-hand side before the coefficient multiply (Algorithm 1,
 * the source line of the pressure loop). The elastic v_y force (Eq. 2 puts it
 * outside the 1/rho factor) is stored as s^ = RN(w * ((dt * Z0) / (P0 * h^2)))
 * and added to the v_y increment after the multiply. idx is the grid point
 * (i, j, k).
 * Acoustic: field must be WAVE_F_P. Elastic: WAVE_F_VY. */
wave_status wave_set_source(wave_ctx *ctx, wave_field field, const int64_t idx[3],
                            const double *wavelet, int64_t nt);

/* wave_set_receivers -- receiver time histories (Section 3: traces recorded
 * at a receiver point). After every step s (counted from this call), the
 * stored value of `field` at each of the nrec points idx[3*r..3*r+2] is
 * written, converted exactly to binary32 and still in scaled units, to
 * device_traces[s * nrec + r] for s < capacity_steps. device_traces is caller
 * owned device memory of capacity_steps * nrec floats. nrec = 0 disables. */
wave_status wave_set_receivers(wave_ctx *ctx, wave_field field, const int64_t *idx,
                               int64_t nrec, float *device_traces, int64_t capacity_steps);

/* wave_step -- advance n >= 0 leapfrog steps (Algorithm 1 / 2 per step:
 * velocities from p^n, then p^{n+1} from the new velocities; elastic:
 * velocities from the stresses, then the stresses). Asynchronous. The last
 * step of each call also accumulates the discrete energy (wave_energy). */
wave_status wave_step(wave_ctx *ctx, int64_t n);

/* wave_set_energy_trace -- record the energy of every step into caller owned
 * device memory: device_energy[s] (binary64, physical units) for steps s
 * counted from this call, s < capacity. capacity = 0 disables. */
wave_status wave_set_energy_trace(wave_ctx *ctx, double *device_energy, int64_t capacity);

/* wave_energy -- discrete energy after the most recent step (Section 3 states
 * the discrete system conserves an energy; its formula is the leapfrog form):
 *   acoustic  E = 0.5 h^(d-1) P0^2 dt / Z0 * ( sum v^2 / a + sum p^n p^{n+1} / b )
 *   elastic   E = 0.5 h P0^2 dt / Z0 * ( sum v^2 / b_v + sum sigma^n . C^-1 sigma^{n+1} )
 * with the stored (rounded) values and multipliers (the vx and normal-stress
 * terms of a free surface row weighted 1/2); compensations are not
 * included. Products are formed in binary32 (exact for half and bfloat16
 * operands), divided once, summed with compensation per thread and in binary64
 * across threads. Synchronises the stream. ESTATE if no step has run yet. */
wave_status wave_energy(wave_ctx *ctx, double *E);

/* wave_get_field -- physical values of a field (inverse of the scaling of
 * wave_set_initial, in binary64), one per grid point. Synchronises. */
wave_status wave_get_field(wave_ctx *ctx, wave_field field, double *host_out);

/* wave_get_raw -- the stored bits of a field (compensation = 0) or of its
 * compensation (compensation = 1): n[0]*n[1]*n[2] elements of the storage
 * format (2 bytes for half / bfloat16, 4 for binary32), x fastest, no pitch.
 * Synchronises. */
wave_status wave_get_raw(wave_ctx *ctx, wave_field field, int32_t compensation, void *host_out);

/* wave_set_raw -- inverse of wave_get_raw (no scaling, no wall masking). */
wave_status wave_set_raw(wave_ctx *ctx, wave_field field, int32_t compensation,
                         const void *host_in);

/* wave_get_coefficient -- the rounded multipliers as binary64, one per grid
 * point: acoustic which = 0 b, 1..3 a_x..a_z; elastic which = 0 bx, 1 by,
 * 2 l2m, 3 lam, 4 mu. Also returns Z0 when Z0 != NULL. */
wave_status wave_get_coefficient(wave_ctx *ctx, int32_t which, double *host_out, double *Z0);

/* wave_get_state / wave_set_state -- checkpoint and resume: every field, its
 * compensation, the step counter. *size is in/out (bytes); blob = NULL
 * queries the size. The blob is only meaningful for a context created with
 * the same arguments. Synchronises. */
wave_status wave_get_state(wave_ctx *ctx, void *blob, size_t *size);
wave_status wave_set_state(wave_ctx *ctx, const void *blob, size_t size);

/* wave_sync -- wait for the queued work and report its errors. */
wave_status wave_sync(wave_ctx *ctx);

/* wave_steps_done -- global step counter. */
wave_status wave_steps_done(wave_ctx *ctx, int64_t *steps);

/* wave_set_timing / wave_get_timing -- per-kernel device time. While timing
 * is enabled, wave_step brackets every kernel launch with CUDA events recorded
 * on the context's stream. wave_get_timing synchronises and returns, for one
 * kernel kind, the launches and their summed device time (milliseconds) since
 * timing was last enabled. Kinds: 0 velocity half step, 1 pressure (or stress)
 * half step including source and energy, 2 receiver sampling, 3 a whole step
 * in one launch sequence (3D one-pass kernel, 2D row strips; for the 2D
 * cluster-resident steps, every step of one wave_step call). Enabling resets
 * the totals. Not part of the method; a measurement aid. */
wave_status wave_set_timing(wave_ctx *ctx, int32_t enable);
wave_status wave_get_timing(wave_ctx *ctx, int32_t kind, int64_t *launches, double *ms);

/* wave_selftest_timeout -- run the device error path on purpose: a kernel
 * waits on an mbarrier that nothing completes, with a short poll limit, sets
 * the context's error word when the wait expires and returns. The call then
 * reports what a stalled pipeline reports: WAVE_ETIMEOUT, and the context is
 * poisoned (WAVE_ESTATE afterwards); the CUDA context and other wave contexts
 * stay usable. Nothing faults or hangs. Not part of the method; a test aid. */
wave_status wave_selftest_timeout(wave_ctx *ctx);

/* wave_reset -- zero every field and compensation and the step counter, and
 * restart the receiver and energy traces at their first row; the medium,
 * source, receivers and any adjoint buffers are kept (for running many shots
 * on one context). Asynchronous. */
wave_status wave_reset(wave_ctx *ctx);

/*
 * Gradient of a trace misfit with respect to the velocity model, by the
 * discrete adjoint of the acoustic scheme (not in the paper; acoustic only).
 *
 * wave_record -- run nsteps forward steps from the current state exactly as
 * wave_step does (receivers and the energy trace record as usual), keeping
 * ncheckpoints snapshots of the state (0: ceil(sqrt(nsteps))), one at the start
 * of each segment of K = ceil(nsteps / ncheckpoints) steps, and the end state.
 * Receivers, if set, must record p. Resets the adjoint: the adjoint fields
 * and the gradient start at zero at step nsteps. Memory: (ncheckpoints + 1)
 * states + K velocity fields + 3-5 binary32 fields (6-9 where the context
 * runs the one-pass 3D step: the adjoint leapfrog then uses it too, on a
 * second set of adjoint fields). Errors: ENOTIMPL (elastic), EINVAL, ENOMEM,
 * ECUDA.
 *
 * wave_adjoint_step -- n steps of the adjoint backwards in time from the
 * current adjoint step t (t = nsteps after wave_record; n <= t). residual:
 * device array [nsteps][nrec] (binary32), residual[s * nrec + r] = dJ/dd_sr,
 * the derivative of the misfit J with respect to sample r of step s of the
 * recorded traces (for J = 1/2 sum (d - d_obs)^2 it is d - d_obs); it may be
 * NULL when no receivers are set. Each step injects its residual row at the
 * receivers, accumulates the gradient and takes one leapfrog step of the
 * adjoint fields (binary32) with the multipliers negated. The forward
 * velocities of the step are replayed from the nearest checkpoint (one
 * segment at a time, bit-identical to the recorded run). On return the
 * forward fields again hold the end state of the recorded run.
 * Errors: ESTATE (no recorded run), EINVAL, ECUDA.
 *
 * wave_get_gradient -- dJ/dc at every node (binary32, x fastest, unpitched,
 * n[0]*n[1]*n[2] values) into the caller's device array device_out, for the
 * adjoint steps taken so far; the full gradient once steps_left is 0.
 * device_out may be NULL to query steps_left only. Asynchronous.
 */
wave_status wave_record(wave_ctx *ctx, int64_t nsteps, int64_t ncheckpoints);
wave_status wave_adjoint_step(wave_ctx *ctx, int64_t n, const float *residual_traces);
wave_status wave_get_gradient(wave_ctx *ctx, float *device_out, int64_t *steps_left);

/*
 * Batched stepping of many independent 2D acoustic problems ("shots"), for
 * example the sources of a seismic survey, each with its own grid size,
 * medium and source. Not in the paper (it runs one problem at a time).
 *
 * wave_batch_create -- group nctx existing contexts. All must be 2D acoustic,
 * share the precision, the compensation and the CUDA stream, and have no
 * receivers set. The contexts stay valid and owned by the caller; they must
 * outlive the batch. Errors: EINVAL (mixed contexts, nctx outside 1..1024),
 * ENOMEM, ECUDA.
 * wave_batch_step -- advance every context of the batch n steps over one work
 * list of (shot, tile) items, with each shot's arithmetic identical to
 * wave_step on that context alone (the same bits). Launch kinds: two launches
 * per step (tiles of points, or row strips), one launch per step (one-pass
 * row strips), or every step of the call but the last in one cooperative
 * launch (row strips with a grid barrier between the half steps; every block
 * resident; the last step, which reduces the energy, on the row strips;
 * a barrier wait is bounded, about a second, and on expiry every context's
 * error word is set: wave_energy then returns ETIMEOUT). The first call with
 * enough steps (25) times the candidate launch shapes on its first steps
 * (real steps of the problems) and keeps the fastest; runs of steps of the
 * two-launch kinds are then replayed from a captured CUDA graph when the
 * stream is not the legacy default stream. The energy of the last step is
 * available per context through wave_energy. Asynchronous.
 * wave_batch_set_shape -- use candidate launch shape `shape` (0 .. 23, the
 * tuner's list: 0-1 tiles of points, 2-13 two-launch strips, 14-17 the
 * persistent cooperative launch, 18-23 one-pass strips) instead of tuning.
 * Errors: EINVAL (index out of range; a one-pass shape without every
 * context's second buffer set, or with WAVE_FP16_PAIRS).
 * wave_batch_info -- the launch configuration in use, written to
 * info[0 .. min(ninfo, 7) - 1]: kind (0 one thread per point, 1 one warp per
 * row strip, 2 one-pass row strips, 3 persistent row strips), tile width in
 * points, tile height in rows, threads per block, blocks (0 for kind 3: as
 * many as are resident at once), steps per graph replay (0 when no graph is
 * in use), tuned (0/1).
 */
typedef struct wave_batch wave_batch;
wave_status wave_batch_create(int32_t nctx, wave_ctx *const *ctxs, wave_batch **out);
wave_status wave_batch_step(wave_batch *batch, int64_t n);
wave_status wave_batch_set_shape(wave_batch *batch, int32_t shape);
wave_status wave_batch_info(wave_batch *batch, int32_t *info, int32_t ninfo);
void wave_batch_destroy(wave_batch *batch);

/* Domain decomposition along z (not in the paper; the stencil radius of 2 of
 * Section 3 fixes the ghost width). A 3D acoustic grid of nz planes is split
 * into slabs, one context each (wave_options.z_cut, z0, rho_above), and every
 * step is taken in two halves with an exchange of two planes per cut face in
 * between:
 *   wave_half_step(ctx, 0)  velocities from p (reads the p ghost planes)
 *   exchange v_z            each slab's first two and last two planes of v_z go
 *                           to the neighbours' ghost buffers
 *   wave_half_step(ctx, 1)  pressure from the velocities (reads the v_z ghosts)
 *   exchange p              likewise for p
 * (p is exchanged once before the first step as well). Compensations are
 * point-local and never exchanged. A slab computes exactly the values the
 * whole grid's context computes on its planes (the same operations in the same
 * order). The exchange is the caller's: peer copies or NCCL send/recv into the
 * receiving GPU's own ghost buffers; the library never reads another GPU's
 * memory.
 *
 * wave_set_z_ghosts -- device buffers of the ghost planes, caller owned, each
 * two planes laid out like the context's fields (wave_get_layout): p_lo and
 * vz_lo hold the grid planes z0-2, z0-1 below the slab, p_hi and vz_hi the
 * planes z1, z1+1 above it. Exactly the cut faces' pointers are non-NULL, each
 * 16-byte aligned. EINVAL otherwise or for a context that is not a slab.
 *
 * wave_half_step -- which = 0: the velocity half step; which = 1: the pressure
 * half step with the source, the energy of the step (wave_energy) and the
 * receivers; the pair advances the step count by one. For contexts that run
 * two-kernel steps (slabs always do; others with wave_options.kernel = 1 or 2);
 * ESTATE for a context stepping with a fused kernel, or when the halves are
 * called out of order. wave_step is refused (ESTATE) on a slab.
 *
 * wave_copy_planes -- copy planes z_first .. z_first + nplanes - 1 of a field
 * (storage format, laid out as wave_get_layout says) into device memory dst,
 * asynchronously on the context's stream: the planes a slab sends to its
 * neighbours. EINVAL for a range outside the context or a NULL dst.
 *
 * wave_get_layout -- out[0] row pitch in elements, out[1] elements per plane
 * (pitch * n[1]), out[2] bytes per element of the storage format. */
wave_status wave_set_z_ghosts(wave_ctx *ctx, const void *p_lo, const void *p_hi, const void *vz_lo,
                              const void *vz_hi);
wave_status wave_half_step(wave_ctx *ctx, int32_t which);
wave_status wave_copy_planes(wave_ctx *ctx, wave_field field, int64_t z_first, int64_t nplanes,
                             void *dst);
wave_status wave_get_layout(wave_ctx *ctx, int64_t out[3]);

/* wave_energy_acoustic_static -- the acoustic discrete energy (the quantity
 * wave_energy reports) computed from device arrays the caller already owns,
 * without allocating any device memory. The paper has no counterpart: this is
 * an entry point for callers that cannot call cudaMalloc, such as a host
 * framework that reserves the whole device heap at start-up and hands out only
 * views of it (its own cudaMalloc would fail or break the framework's
 * accounting), or a real-time loop whose memory budget forbids allocation
 * after start-up (an allocation can block, fragment the heap or fail).
 *   ndim, n      grid (2D or 3D), cells per axis
 *   prec         storage format of every array below (the *_F32ARITH codes
 *                mean half / bfloat16 storage)
 *   p_old, p_new pressure p^n and p^{n+1}; v[c] velocities v_c^{n+1/2} (c < ndim)
 *   a[c], b      the multipliers a_c and b, one per point
 *                (all arrays packed, x fastest, no pitch, in device memory)
 *   factor       multiplies the sum; 0.5 h^(d-1) P0^2 dt / Z0 gives wave_energy's units
 *   device_out   one double in device memory, written by the GPU
 *   cuda_stream  stream to run on (asynchronous; synchronise before reading)
 * Its block partials live in a static device array of WAVE_ENERGY_STATIC_MAX_BLOCKS
 * doubles (64 KiB plus a counter) that every GPU loading the library holds until
 * the process exits; each block covers 2048 points, so grids above
 * WAVE_ENERGY_STATIC_MAX_BLOCKS * 2048 = 16,777,216 points are rejected with
 * WAVE_EINVAL. The first call on a device (and the first after the device's
 * context is replaced, e.g. by cudaDeviceReset) looks up the array's device
 * address with that device current: make that first call before any stream
 * capture. Each call clears the array's block counter before its kernel runs.
 * All calls share the one array: calls that overlap on the GPU (two streams,
 * two host threads) race and return wrong sums. */
#define WAVE_ENERGY_STATIC_MAX_BLOCKS 8192
wave_status wave_energy_acoustic_static(int32_t ndim, const int64_t n[3], wave_precision prec,
                                        const void *p_old, const void *p_new,
                                        const void *const v[3], const void *const a[3],
                                        const void *b, double factor, double *device_out,
                                        void *cuda_stream);

void wave_destroy(wave_ctx *ctx);
const char *wave_last_error(void);

/* Build description: "sm_103a ..." plus the compile options that matter for
 * bit-exactness (-fmad=false). */
const char *wave_build_info(void);

#ifdef __cplusplus
}
#endif
#endif /* WAVE_H */
