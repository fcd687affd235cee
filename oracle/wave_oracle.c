/*
 * wave_oracle.c -- TEST INFRASTRUCTURE, NOT PART OF THE PRODUCT.
 *
 * A plain, slow CPU restatement of the method of Gao & Harms, "Half precision
 * wave simulation" (arXiv 2310.00236): the staggered-grid, fourth-order,
 * leapfrog discretisation of the first-order acoustic system (Eq. 1) and of the
 * 2D isotropic elastic velocity-stress system (Eq. 2, Appendix A), with every
 * arithmetic operation rounded to a chosen IEEE format and the solution update
 * done either as a plain sum (Algorithm 1) or as a compensated sum
 * (Algorithm 2, with the 3-operation or 6-operation error-free sum of Code 1 /
 * Code 2 in Section 4).
 *
 * Only the test-suite, the smoke check and the benchmark's CPU-baseline leg
 * load this library. It shares no code with the CUDA path.
 *
 * Representation: every field, compensation and coefficient value is held in a
 * C double that is exactly representable in the field's storage format. Every
 * operation "x op y" in a format F is evaluated as RN_F(x op y) where the
 * inner op is the host's IEEE binary64 operation and RN_F is the
 * round-to-nearest-even conversion below. For binary16 operands the binary64
 * sum, difference and product are exact, so this is a single rounding. For
 * bfloat16 and binary32 operands binary64 has at least 2p+2 bits, so rounding
 * twice gives the same result as rounding once (the classical double-rounding
 * condition for +, -, *; Section 2 of the paper states the correctly-rounded
 * IEEE model that this reproduces).
 *
 * Build: gcc -O2 -std=c11 -ffp-contract=off -fPIC -shared -fopenmp
 * (no -ffast-math: the rounding and the order of every operation matter).
 */
#include <math.h>
#include <float.h>
#include <omp.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Formats (Table 1 of Section 2; bfloat16 added).                          */
/* ------------------------------------------------------------------------ */

enum { ORC_FP64 = 0, ORC_FP32 = 1, ORC_FP16 = 2, ORC_BF16 = 3 };

typedef struct {
    int precision;  /* significand bits including the hidden bit */
    int emin;       /* exponent of the smallest normal number */
    double maxv;    /* largest finite value */
} orc_format;

static const orc_format FORMATS[4] = {
    {53, -1022, DBL_MAX},
    {24, -126, FLT_MAX},
    {11, -14, 65504.0},
    {8, -126, 3.38953138925153547590470800371487866880e38}, /* (2 - 2^-7) * 2^127 */
};

/* Round x to the nearest value of format fmt, ties to even (IEEE 754
 * roundTiesToEven), with gradual underflow and overflow to infinity.
 * Scaling by a power of two is exact, and nearbyint() rounds to the nearest
 * integer with ties to even in the default rounding mode. */
double orc_round(double x, int fmt)
{
    if (fmt == ORC_FP64 || x == 0.0 || !isfinite(x)) return x;
    const orc_format *f = &FORMATS[fmt];
    double ax = fabs(x);
    int e = ilogb(ax);                       /* floor(log2 |x|) */
    if (e < f->emin) e = f->emin;            /* subnormal range: fixed quantum */
    double quantum = ldexp(1.0, e - (f->precision - 1));
    double r = nearbyint(ax / quantum) * quantum;
    if (r > f->maxv) r = INFINITY;
    return copysign(r, x);
}

/* Element-wise rounding to a format (Section 2's IEEE model), exposed for the
 * rounding pins. */
void orc_round_array(int64_t n, const double *x, int fmt, double *out)
{
    for (int64_t i = 0; i < n; i++) out[i] = orc_round(x[i], fmt);
}

/* Element-wise rounded operations, exposed for the arithmetic pins. */
void orc_op_array(int64_t n, int op, const double *a, const double *b, int fmt, double *out)
{
    for (int64_t i = 0; i < n; i++) {
        double r;
        switch (op) {
        case 0: r = a[i] + b[i]; break;
        case 1: r = a[i] - b[i]; break;
        default: r = a[i] * b[i]; break;
        }
        out[i] = orc_round(r, fmt);
    }
}

static inline double add_f(double a, double b, int f) { return orc_round(a + b, f); }
static inline double sub_f(double a, double b, int f) { return orc_round(a - b, f); }
static inline double mul_f(double a, double b, int f) { return orc_round(a * b, f); }

/* Compensated sums of Section 4.
 * sum_3op (Code 1): s = a + b; z = s - a; t = b - z.  Error free when |a| >= |b|.
 * sum_6op (Code 2): s = a + b; pa = s - b; pb = s - pa; da = a - pa; db = b - pb;
 *                   t = da + db.  Error free for any order of magnitudes. */
static void sum_3op(double a, double b, int f, double *s, double *t)
{
    double s_ = add_f(a, b, f);
    double z = sub_f(s_, a, f);
    *t = sub_f(b, z, f);
    *s = s_;
}

static void sum_6op(double a, double b, int f, double *s, double *t)
{
    double s_ = add_f(a, b, f);
    double pa = sub_f(s_, b, f);
    double pb = sub_f(s_, pa, f);
    double da = sub_f(a, pa, f);
    double db = sub_f(b, pb, f);
    *t = add_f(da, db, f);
    *s = s_;
}

void orc_sum_op_array(int64_t n, int variant, const double *a, const double *b, int fmt,
                      double *s, double *t)
{
    for (int64_t i = 0; i < n; i++) {
        if (variant == 3) sum_3op(a[i], b[i], fmt, &s[i], &t[i]);
        else sum_6op(a[i], b[i], fmt, &s[i], &t[i]);
    }
}

/* ------------------------------------------------------------------------ */
/* Grid, boundaries and the stencil (Section 3, Fig. 1 reading).            */
/* ------------------------------------------------------------------------ */

enum { ORC_BC_PERIODIC = 0, ORC_BC_RIGID = 1 };

/* Along one axis with N cells, a field lives either on the nodes m = 0..N-1
 * (node N is the wall or, periodically, node 0) or at the half points
 * m + 1/2, m = 0..N-1. Reading index m outside 0..N-1:
 *   periodic: wrap around the domain (Section 3);
 *   rigid (p = 0 on the walls at nodes 0 and N): node fields are odd about
 *     the walls, half-point fields are even about them.
 * Returns the sign (+1, -1, or 0 for the wall node N itself) and the index. */
static int map_axis(int64_t m, int64_t N, int bc, int node, int64_t *out)
{
    if (m >= 0 && m < N) { *out = m; return 1; }
    if (bc == ORC_BC_PERIODIC) { *out = ((m % N) + N) % N; return 1; }
    if (node) {
        if (m < 0) { *out = -m; return -1; }
        if (m == N) { *out = 0; return 0; }
        *out = 2 * N - m; return -1;
    }
    if (m < 0) { *out = -1 - m; return 1; }
    *out = 2 * N - 1 - m; return 1;
}

typedef struct {
    int32_t ndim;
    int32_t bc[3];
    int64_t n[3];
    int32_t store_fmt;
    int32_t arith_fmt;
    int32_t stencil_fmt;
    int32_t comp;
    /* 0: C2 = RN(1/24) in the stencil format (the scheme). 1 + F: C2 rounded
     * to format F instead, every other operation unchanged -- an experiment
     * that separates the rounding of the operator's weight from the rest
     * (the "Operator" remark of Section 5). */
    int32_t c2_override;
    /* 0: the stencils read the stored values V (the scheme of Algorithms 1
     * and 2). 1: they read RN(V + T) in the stencil format, the stored value
     * plus its carried compensation -- not the paper's scheme: an experiment
     * that measures what the stencil's reading of the rounded stored value
     * costs. */
    int32_t pair_stencil;
} orc_acoustic_cfg;

static inline int64_t lin(const int64_t n[3], int64_t i, int64_t j, int64_t k)
{
    return i + n[0] * (j + n[1] * k);
}

/* Value of field f at the point whose coordinate along axis ax is replaced by m. */
static double read_axis(const double *f, const int64_t n[3], const int32_t bc[3], int ax,
                        int node, int64_t i, int64_t j, int64_t k, int64_t m)
{
    int64_t idx[3] = {i, j, k}, mm;
    int sign = map_axis(m, n[ax], bc[ax], node, &mm);
    if (sign == 0) return 0.0;
    idx[ax] = mm;
    double v = f[lin(n, idx[0], idx[1], idx[2])];
    return sign > 0 ? v : -v;
}

/* Fourth-order staggered difference, coefficients [1/24, -9/8, 9/8, -1/24]
 * (Section 3), evaluated as D = C1*(f[+1/2] - f[-1/2]) - C2*(f[+3/2] - f[-3/2])
 * with C1 = 9/8 and C2 = 1/24 rounded to the stencil format. The value is the
 * undivided difference (the 1/h factor lives in the coefficient). */
static double stencil_w(double fm3, double fm1, double fp1, double fp3, int f, double c2)
{
    const double c1 = 9.0 / 8.0;
    double t1 = sub_f(fp1, fm1, f);
    double t2 = sub_f(fp3, fm3, f);
    return sub_f(mul_f(c1, t1, f), mul_f(c2, t2, f), f);
}

static double stencil(double fm3, double fm1, double fp1, double fp3, int f)
{
    return stencil_w(fm3, fm1, fp1, fp3, f, orc_round(1.0 / 24.0, f));
}

double orc_stencil_c2(int fmt) { return orc_round(1.0 / 24.0, fmt); }

/* Threads used by the OpenMP loops of the solvers (n <= 0: leave unchanged).
 * Returns the count now in force. Timing only: the results do not depend on
 * it, since every parallel loop writes disjoint points and the energy sums
 * are taken in a fixed order. */
int orc_set_threads(int n)
{
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
}

/* Solution update V += inc of Algorithm 1 (comp = 0) or the compensated update
 * of Algorithm 2 (comp = 3 or 6). The carried compensation T is added to the
 * scaled increment before the error-free sum, R = T + inc; sum(V, R) -> (V, T).
 * When the arithmetic format is wider than the storage format (half storage
 * with binary32 registers), the sum is formed in the arithmetic format and
 * the lost part is the difference between that sum and its stored rounding. */
static void update(double *V, double *T, double inc, int comp, int af, int sf)
{
    if (comp == 0) {
        *V = orc_round(add_f(*V, inc, af), sf);
        return;
    }
    double R = add_f(*T, inc, af);
    if (af == sf) {
        double s, t;
        if (comp == 3) sum_3op(*V, R, af, &s, &t);
        else sum_6op(*V, R, af, &s, &t);
        *V = s;
        *T = t;
    } else {
        double s = add_f(*V, R, af);
        double vs = orc_round(s, sf);
        *T = orc_round(sub_f(s, vs, af), sf);
        *V = vs;
    }
}

/* Element-wise solution update (the function above), exposed for its pins:
 * (Vout, Tout) = update of (V, T) by inc. */
void orc_update_array(int64_t n, int comp, int af, int sf, const double *V, const double *T,
                      const double *inc, double *Vout, double *Tout)
{
    for (int64_t i = 0; i < n; i++) {
        double v = V[i], t = T[i];
        update(&v, &t, inc[i], comp, af, sf);
        Vout[i] = v;
        Tout[i] = t;
    }
}

/* Neumaier-compensated binary64 accumulation, for energies. */
typedef struct { double s, c; } acc_t;
static inline void acc_add(acc_t *a, double x)
{
    double t = a->s + x;
    if (fabs(a->s) >= fabs(x)) a->c += (a->s - t) + x;
    else a->c += (x - t) + a->s;
    a->s = t;
}
static inline double acc_val(const acc_t *a) { return a->s + a->c; }

/* ------------------------------------------------------------------------ */
/* Acoustic leapfrog (Eq. 1, Algorithms 1 and 2; 3D by adding vz and d/dz). */
/* ------------------------------------------------------------------------ */

/* Set the values that the rigid walls hold at zero: p on every wall node
 * plane, and each velocity component on the wall planes of the axes it is
 * not staggered along. */
void orc_acoustic_apply_walls(const orc_acoustic_cfg *cfg, double *p, double *vx, double *vy,
                              double *vz)
{
    const int64_t *n = cfg->n;
    double *v[3] = {vx, vy, vz};
    for (int64_t k = 0; k < n[2]; k++)
        for (int64_t j = 0; j < n[1]; j++)
            for (int64_t i = 0; i < n[0]; i++) {
                int64_t idx[3] = {i, j, k};
                int64_t q = lin(n, i, j, k);
                int on_wall[3];
                for (int ax = 0; ax < 3; ax++)
                    on_wall[ax] = ax < cfg->ndim && cfg->bc[ax] == ORC_BC_RIGID && idx[ax] == 0;
                if (on_wall[0] || on_wall[1] || on_wall[2]) p[q] = 0.0;
                for (int c = 0; c < cfg->ndim; c++) {
                    if (!v[c]) continue;
                    for (int ax = 0; ax < cfg->ndim; ax++)
                        if (ax != c && on_wall[ax]) v[c][q] = 0.0;
                }
            }
}

/* Ghost planes along z for a slab of a larger grid (domain decomposition
 * along z; not in the paper): lo holds the global planes z0-2, z0-1 below the
 * slab, hi the planes z1, z1+1 above it, each n[0]*n[1] values x fastest, of
 * the field a half step differentiates along z. NULL: that face is a face of
 * the grid and its boundary rule applies. */
typedef struct { const double *lo, *hi; } zghost;

/* read_axis, except that along z a face with ghost planes reads them */
static double read_axis_g(const double *f, const int64_t n[3], const int32_t bc[3], int ax, int node,
                          int64_t i, int64_t j, int64_t k, int64_t m, const zghost *g)
{
    if (ax == 2 && g) {
        if (m < 0 && g->lo) return g->lo[i + n[0] * (j + n[1] * (m + 2))];
        if (m >= n[2] && g->hi) return g->hi[i + n[0] * (j + n[1] * (m - n[2]))];
    }
    return read_axis(f, n, bc, ax, node, i, j, k, m);
}

/* Velocity half step of Algorithms 1 / 2: v_c^{n+1/2} = v_c^{n-1/2} + a_c D_c(p^n),
 * with D_c reading pr (the stored p, or RN(p + t_p) for pair_stencil). */
static void velocity_half(const orc_acoustic_cfg *cfg, const double *pr, double *const v[3],
                          double *const tv[3], const double *const a[3], double c2, const zghost *g)
{
    const int64_t *n = cfg->n;
    const int nd = cfg->ndim;
    const int sf = cfg->store_fmt, af = cfg->arith_fmt, stf = cfg->stencil_fmt, comp = cfg->comp;
#pragma omp parallel for schedule(static)
    for (int64_t jk = 0; jk < n[1] * n[2]; jk++) {
        const int64_t j = jk % n[1], k = jk / n[1];
        for (int64_t i = 0; i < n[0]; i++) {
            const int64_t q = lin(n, i, j, k);
            const int64_t idx[3] = {i, j, k};
            for (int c = 0; c < nd; c++) {
                /* v_c sits at m + 1/2 along axis c; p at nodes m-1, m, m+1, m+2 */
                const int64_t m = idx[c];
                double fm3 = read_axis_g(pr, n, cfg->bc, c, 1, i, j, k, m - 1, g);
                double fm1 = read_axis_g(pr, n, cfg->bc, c, 1, i, j, k, m, g);
                double fp1 = read_axis_g(pr, n, cfg->bc, c, 1, i, j, k, m + 1, g);
                double fp3 = read_axis_g(pr, n, cfg->bc, c, 1, i, j, k, m + 2, g);
                double D = stencil_w(fm3, fm1, fp1, fp3, stf, c2);
                double inc = orc_round(mul_f(a[c][q], D, stf), af);
                update(&v[c][q], &tv[c][q], inc, comp, af, sf);
            }
        }
    }
}

/* Pressure half step: p^{n+1} = p^n + b (Dx vx + Dy vy [+ Dz vz] [+ s]) with
 * the divergence reading vr, summed left to right, the source at global step
 * gstep. With rowacc, each (j, k) row's energy terms (velocity, pressure). */
static void pressure_half(const orc_acoustic_cfg *cfg, double *p, double *tp, double *const vr[3],
                          double *const v[3], const double *const a[3], const double *b_c, double c2,
                          int64_t src_index, int64_t src_nt, const double *src, int64_t gstep,
                          double *rowacc, const zghost *g)
{
    const int64_t *n = cfg->n;
    const int nd = cfg->ndim;
    const int sf = cfg->store_fmt, af = cfg->arith_fmt, stf = cfg->stencil_fmt, comp = cfg->comp;
#pragma omp parallel for schedule(static)
    for (int64_t jk = 0; jk < n[1] * n[2]; jk++) {
        const int64_t j = jk % n[1], k = jk / n[1];
        acc_t ep = {0.0, 0.0}, ev = {0.0, 0.0};
        for (int64_t i = 0; i < n[0]; i++) {
            const int64_t q = lin(n, i, j, k);
            const int64_t idx[3] = {i, j, k};
            double R = 0.0;
            for (int c = 0; c < nd; c++) {
                /* p sits on node m along axis c; v_c at m-2, m-1, m, m+1 (+1/2) */
                const int64_t m = idx[c];
                double fm3 = read_axis_g(vr[c], n, cfg->bc, c, 0, i, j, k, m - 2, g);
                double fm1 = read_axis_g(vr[c], n, cfg->bc, c, 0, i, j, k, m - 1, g);
                double fp1 = read_axis_g(vr[c], n, cfg->bc, c, 0, i, j, k, m, g);
                double fp3 = read_axis_g(vr[c], n, cfg->bc, c, 0, i, j, k, m + 1, g);
                double D = stencil_w(fm3, fm1, fp1, fp3, stf, c2);
                R = (c == 0) ? D : add_f(R, D, stf);
            }
            if (src && q == src_index && gstep < src_nt) R = add_f(R, src[gstep], stf);
            double inc = orc_round(mul_f(b_c[q], R, stf), af);
            const double p_old = p[q];
            update(&p[q], &tp[q], inc, comp, af, sf);
            if (rowacc) {
                acc_add(&ep, p_old * p[q] / b_c[q]);
                for (int c = 0; c < nd; c++) acc_add(&ev, v[c][q] * v[c][q] / a[c][q]);
            }
        }
        if (rowacc) {
            rowacc[2 * jk] = acc_val(&ev);
            rowacc[2 * jk + 1] = acc_val(&ep);
        }
    }
}

/* Advance nsteps leapfrog steps. State on entry: p^n, v^{n-1/2} and their
 * compensations; on exit p^{n+nsteps}, v^{n+nsteps-1/2}.
 * Per step (Algorithm 1/2 order): all velocity components from p^n, then p
 * from the new velocities. The pressure right-hand side is
 * R = Dx(vx) + Dy(vy) [+ Dz(vz)] [+ source], summed left to right.
 * Energy (scaled units) after step n: E^{n+1/2} = sum v^2/a + sum p^n p^{n+1}/b
 * over all stored points, with the rounded coefficients the scheme uses.
 * src: scaled source values (already rounded to the arithmetic format) for
 * global steps 0..src_nt-1, added at p point src_index; NULL for none.
 * Receivers sample field rec_field (0 p, 1 vx, 2 vy, 3 vz) after each step. */
int orc_acoustic_run(const orc_acoustic_cfg *cfg, double *p, double *tp, double *vx, double *tvx,
                     double *vy, double *tvy, double *vz, double *tvz, const double *ax_c,
                     const double *ay_c, const double *az_c, const double *b_c, int64_t nsteps,
                     int64_t step0, int64_t src_index, int64_t src_nt, const double *src,
                     int32_t rec_field, int64_t nrec, const int64_t *rec_index, double *traces,
                     double *energy)
{
    const int64_t *n = cfg->n;
    const int nd = cfg->ndim;
    const int stf = cfg->stencil_fmt;
    const int comp = cfg->comp;
    const double c2 = orc_round(1.0 / 24.0, cfg->c2_override > 0 ? cfg->c2_override - 1 : stf);
    double *const v[3] = {vx, vy, vz}, *const tv[3] = {tvx, tvy, tvz};
    const double *const a[3] = {ax_c, ay_c, az_c};
    const int64_t npts = n[0] * n[1] * n[2];
    double *rowacc = (double *)calloc((size_t)(n[1] * n[2]) * 2, sizeof(double));
    if (!rowacc) return -1;
    /* what the stencils read: the stored values, or RN(V + T) (pair_stencil) */
    double *pr = p, *vr[3] = {vx, vy, vz};
    double *pairs = NULL;
    if (cfg->pair_stencil && comp) {
        pairs = (double *)malloc(sizeof(double) * (size_t)npts * (size_t)(1 + nd));
        if (!pairs) { free(rowacc); return -1; }
        pr = pairs;
        for (int c = 0; c < nd; c++) vr[c] = pairs + (size_t)npts * (size_t)(1 + c);
    }

    for (int64_t s = 0; s < nsteps; s++) {
        const int64_t gstep = step0 + s;
        if (pairs)
            for (int64_t q = 0; q < npts; q++) pairs[q] = add_f(p[q], tp[q], stf);
        velocity_half(cfg, pr, v, tv, a, c2, NULL);
        if (pairs)
            for (int c = 0; c < nd; c++)
                for (int64_t q = 0; q < npts; q++) vr[c][q] = add_f(v[c][q], tv[c][q], stf);
        pressure_half(cfg, p, tp, vr, v, a, b_c, c2, src_index, src_nt, src, gstep,
                      energy ? rowacc : NULL, NULL);
        if (energy) {
            acc_t e = {0.0, 0.0};
            for (int64_t jk = 0; jk < n[1] * n[2]; jk++) {
                acc_add(&e, rowacc[2 * jk]);
                acc_add(&e, rowacc[2 * jk + 1]);
            }
            energy[s] = acc_val(&e);
        }
        if (traces && nrec > 0) {
            const double *f = rec_field == 0 ? p : v[rec_field - 1];
            for (int64_t r = 0; r < nrec; r++) {
                int64_t q = rec_index[r];
                traces[s * nrec + r] = (q >= 0 && q < npts) ? f[q] : 0.0;
            }
        }
    }
    free(rowacc);
    free(pairs);
    return 0;
}

/* One half step of a 3D z slab (domain decomposition along z; not in the
 * paper): half = 0 the velocity half step (ghosts: planes of p), half = 1 the
 * pressure half step at global step gstep (ghosts: planes of v_z), with the
 * same operations as orc_acoustic_run. ghost_lo / ghost_hi as in zghost; the
 * stored-value scheme only (no pair_stencil). Returns 0, or -2 for a cfg
 * this does not cover. */
int orc_acoustic_half_step(const orc_acoustic_cfg *cfg, int32_t half, double *p, double *tp,
                           double *vx, double *tvx, double *vy, double *tvy, double *vz,
                           double *tvz, const double *ax_c, const double *ay_c, const double *az_c,
                           const double *b_c, const double *ghost_lo, const double *ghost_hi,
                           int64_t gstep, int64_t src_index, int64_t src_nt, const double *src)
{
    if (cfg->ndim != 3 || cfg->pair_stencil) return -2;
    const double c2 =
        orc_round(1.0 / 24.0, cfg->c2_override > 0 ? cfg->c2_override - 1 : cfg->stencil_fmt);
    double *const v[3] = {vx, vy, vz}, *const tv[3] = {tvx, tvy, tvz};
    const double *const a[3] = {ax_c, ay_c, az_c};
    const zghost g = {ghost_lo, ghost_hi};
    if (half == 0) velocity_half(cfg, p, v, tv, a, c2, &g);
    else pressure_half(cfg, p, tp, v, v, a, b_c, c2, src_index, src_nt, src, gstep, NULL, &g);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Discrete adjoint of the acoustic leapfrog (not in the paper).            */
/* ------------------------------------------------------------------------ */

/* Misfit J = 1/2 sum_s sum_r (trace[s][r] - d_obs[s][r])^2 of the pressure
 * traces that orc_acoustic_run records (trace[s] = p^(s+1) at the receivers),
 * and its derivatives, by reverse-mode differentiation of the binary64
 * scheme (store, arithmetic and stencil formats binary64, no compensation).
 *
 * Forward step s (as orc_acoustic_run):
 *   v_c^(s+1/2) = v_c^(s-1/2) + a_c * D_c p^s              (gather over 4 taps)
 *   p^(s+1)     = p^s + b * R^s,  R^s = sum_c D_c v_c^(s+1/2) + src^s
 * Reverse of step s, with adjoints pbar (of p^(s+1)) and vbar (of v^(s+1/2)):
 *   pbar += the residual of step s at the receiver points;
 *   bbar += pbar * R^s;   vbar_c += D_c^T (b * pbar)       (scatter over 4 taps)
 *   pbar += sum_c D_c^T (a_c * vbar_c)
 * Every transpose is the scatter of the forward gather, tap by tap, with the
 * boundary images' signs; pbar then holds the adjoint of p^s. The forward
 * velocity history is kept in full (small problems only).
 * Outputs (any may be NULL): traces [nsteps][nrec]; grad_b = dJ/db;
 * grad_c = dJ/dc through b = dt rho c^2 / (Z0 h), i.e. grad_b * 2 b / c with
 * Z0 held fixed (J does not depend on Z0: it only scales the velocity unit);
 * p0_bar = dJ/dp^0 (the adjoint state at step 0).
 * residual: dJ/dtrace [nsteps][nrec] (= trace - d_obs for the L2 misfit).
 * Returns 0, -1 (allocation), -2 (cfg not binary64 without compensation). */
int orc_acoustic_adjoint(const orc_acoustic_cfg *cfg, const double *p_init, const double *vx_init,
                         const double *vy_init, const double *vz_init, const double *ax_c,
                         const double *ay_c, const double *az_c, const double *b_c, const double *c,
                         int64_t nsteps, int64_t step0, int64_t src_index, int64_t src_nt,
                         const double *src, int64_t nrec, const int64_t *rec_index,
                         const double *residual, double *traces, double *grad_b, double *grad_c,
                         double *p0_bar)
{
    if (cfg->store_fmt != ORC_FP64 || cfg->arith_fmt != ORC_FP64 || cfg->stencil_fmt != ORC_FP64 ||
        cfg->comp != 0)
        return -2;
    const int64_t *n = cfg->n;
    const int nd = cfg->ndim;
    const int64_t npts = n[0] * n[1] * n[2];
    const double *a[3] = {ax_c, ay_c, az_c};
    const double *vinit[3] = {vx_init, vy_init, vz_init};
    const double c1 = 9.0 / 8.0, c2 = 1.0 / 24.0;
    /* forward taps: weights of D = c1 (f[+1/2] - f[-1/2]) - c2 (f[+3/2] - f[-3/2]) */
    const double w[4] = {c2, -c1, c1, -c2};

    double *work = (double *)calloc((size_t)npts * 9, sizeof(double));
    double *hist = (double *)malloc((size_t)npts * nd * (size_t)(nsteps > 0 ? nsteps : 1) * sizeof(double));
    double *tr = (double *)calloc((size_t)(nsteps * nrec > 0 ? nsteps * nrec : 1), sizeof(double));
    if (!work || !hist || !tr) {
        free(work);
        free(hist);
        free(tr);
        return -1;
    }
    double *p = work, *tp = work + npts, *v[3], *tv[3];
    for (int ax = 0; ax < 3; ax++) {
        v[ax] = work + (2 + 2 * ax) * npts;
        tv[ax] = work + (3 + 2 * ax) * npts;
    }
    double *pbar = work + 8 * npts;
    memcpy(p, p_init, (size_t)npts * sizeof(double));
    for (int ax = 0; ax < nd; ax++)
        if (vinit[ax]) memcpy(v[ax], vinit[ax], (size_t)npts * sizeof(double));

    /* forward, keeping v^(s+1/2) and the traces */
    for (int64_t s = 0; s < nsteps; s++) {
        int rc = orc_acoustic_run(cfg, p, tp, v[0], tv[0], v[1], tv[1], v[2], tv[2], a[0], a[1], a[2],
                                  b_c, 1, step0 + s, src_index, src_nt, src, 0, nrec, rec_index,
                                  nrec ? tr + s * nrec : NULL, NULL);
        if (rc) {
            free(work);
            free(hist);
            free(tr);
            return -1;
        }
        for (int ax = 0; ax < nd; ax++)
            memcpy(hist + ((size_t)s * nd + ax) * npts, v[ax], (size_t)npts * sizeof(double));
    }
    if (traces && nrec) memcpy(traces, tr, (size_t)(nsteps * nrec) * sizeof(double));

    /* reverse sweep; the buffers p, tp and v are reused as pbar scratch and vbar */
    double *vbar[3] = {v[0], v[1], v[2]};
    double *Rbar = tp;
    memset(pbar, 0, (size_t)npts * sizeof(double));
    for (int ax = 0; ax < 3; ax++) memset(vbar[ax], 0, (size_t)npts * sizeof(double));
    double *gb = grad_b ? grad_b : tv[0];
    memset(gb, 0, (size_t)npts * sizeof(double));
    for (int64_t s = nsteps - 1; s >= 0; s--) {
        const int64_t gstep = step0 + s;
        for (int64_t r = 0; r < nrec; r++) {
            const int64_t q = rec_index[r];
            if (q >= 0 && q < npts) pbar[q] += residual[s * nrec + r];
        }
        /* reverse of the pressure half step */
        for (int64_t k = 0; k < n[2]; k++)
            for (int64_t j = 0; j < n[1]; j++)
                for (int64_t i = 0; i < n[0]; i++) {
                    const int64_t q = lin(n, i, j, k);
                    const int64_t idx[3] = {i, j, k};
                    double R = 0.0;
                    for (int cx = 0; cx < nd; cx++) {
                        const double *vh = hist + ((size_t)s * nd + cx) * npts;
                        const int64_t m = idx[cx];
                        double f[4];
                        for (int t = 0; t < 4; t++) f[t] = read_axis(vh, n, cfg->bc, cx, 0, i, j, k, m - 2 + t);
                        R += c1 * (f[2] - f[1]) - c2 * (f[3] - f[0]);
                    }
                    if (src && q == src_index && gstep < src_nt) R += src[gstep];
                    gb[q] += pbar[q] * R;
                    Rbar[q] = b_c[q] * pbar[q];
                }
        for (int64_t k = 0; k < n[2]; k++)
            for (int64_t j = 0; j < n[1]; j++)
                for (int64_t i = 0; i < n[0]; i++) {
                    const int64_t q = lin(n, i, j, k);
                    const int64_t idx[3] = {i, j, k};
                    for (int cx = 0; cx < nd; cx++) {
                        const int64_t m = idx[cx];
                        for (int t = 0; t < 4; t++) {
                            int64_t mm, at[3] = {i, j, k};
                            int sg = map_axis(m - 2 + t, n[cx], cfg->bc[cx], 0, &mm);
                            if (sg == 0) continue;
                            at[cx] = mm;
                            vbar[cx][lin(n, at[0], at[1], at[2])] += sg * w[t] * Rbar[q];
                        }
                    }
                }
        /* reverse of the velocity half step: v_c at m + 1/2 read p at m-1 .. m+2 */
        for (int64_t k = 0; k < n[2]; k++)
            for (int64_t j = 0; j < n[1]; j++)
                for (int64_t i = 0; i < n[0]; i++) {
                    const int64_t q = lin(n, i, j, k);
                    const int64_t idx[3] = {i, j, k};
                    for (int cx = 0; cx < nd; cx++) {
                        const double g = a[cx][q] * vbar[cx][q];
                        const int64_t m = idx[cx];
                        for (int t = 0; t < 4; t++) {
                            int64_t mm, at[3] = {i, j, k};
                            int sg = map_axis(m - 1 + t, n[cx], cfg->bc[cx], 1, &mm);
                            if (sg == 0) continue;
                            at[cx] = mm;
                            pbar[lin(n, at[0], at[1], at[2])] += sg * w[t] * g;
                        }
                    }
                }
    }
    if (grad_c)
        for (int64_t q = 0; q < npts; q++) grad_c[q] = gb[q] * 2.0 * b_c[q] / c[q];
    if (p0_bar) memcpy(p0_bar, pbar, (size_t)npts * sizeof(double));
    free(work);
    free(hist);
    free(tr);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Coefficient preparation and scaling (Section 5 "Range"; units chosen so  */
/* that coefficients and fields stay inside the half-precision range).      */
/* ------------------------------------------------------------------------ */

/* Z0 = rho0 * c0 with rho0 = max rho, c0 = max c; field scales: p^ = p / P0,
 * v^ = v * Z0 / P0. Per-point multipliers, computed in binary64 in exactly
 * this order and rounded once to the storage format:
 *   b   = (((dt * rho) * c) * c) / (Z0 * h)          at p nodes
 *   a_c = ((dt * Z0) / h) / rho_c                     at v_c points
 *   rho_c = (rho[m] + rho[m+1]) * 0.5 along axis c, where the neighbour m+1
 *           wraps (periodic) or is clamped to m (rigid) at the last cell.
 * Returns 0, or 1 if some coefficient is not a positive normal number of the
 * storage format. */
int orc_acoustic_coefficients(const orc_acoustic_cfg *cfg, double h, double dt, double P0,
                              const double *rho, const double *c, double *ax_c, double *ay_c,
                              double *az_c, double *b_c, double *Z0_out)
{
    const int64_t *n = cfg->n;
    const int64_t npts = n[0] * n[1] * n[2];
    const int sf = cfg->store_fmt;
    double rho0 = 0.0, c0 = 0.0;
    (void)P0;
    for (int64_t q = 0; q < npts; q++) {
        if (rho[q] > rho0) rho0 = rho[q];
        if (c[q] > c0) c0 = c[q];
    }
    const double Z0 = rho0 * c0;
    *Z0_out = Z0;
    double *a[3] = {ax_c, ay_c, az_c};
    int bad = 0;
    const double tiny = ldexp(1.0, FORMATS[sf].emin);
    for (int64_t k = 0; k < n[2]; k++)
        for (int64_t j = 0; j < n[1]; j++)
            for (int64_t i = 0; i < n[0]; i++) {
                const int64_t q = lin(n, i, j, k);
                const int64_t idx[3] = {i, j, k};
                double bq = orc_round((((dt * rho[q]) * c[q]) * c[q]) / (Z0 * h), sf);
                b_c[q] = bq;
                if (!(bq >= tiny && isfinite(bq))) bad = 1;
                for (int ax = 0; ax < cfg->ndim; ax++) {
                    int64_t nb[3] = {i, j, k};
                    int64_t m = idx[ax] + 1;
                    if (m >= n[ax]) m = (cfg->bc[ax] == ORC_BC_PERIODIC) ? 0 : idx[ax];
                    nb[ax] = m;
                    double rho_c = (rho[q] + rho[lin(n, nb[0], nb[1], nb[2])]) * 0.5;
                    double aq = orc_round(((dt * Z0) / h) / rho_c, sf);
                    a[ax][q] = aq;
                    if (!(aq >= tiny && isfinite(aq))) bad = 1;
                }
            }
    return bad;
}

/* Scaled pressure p^ = RN(p / P0): the unit scaling that keeps the values and
 * multipliers inside the half formats' range (Section 5, "Range"). */
void orc_scale_pressure(int64_t n, const double *in, double P0, int fmt, double *out)
{
    for (int64_t i = 0; i < n; i++) out[i] = orc_round(in[i] / P0, fmt);
}

/* Scaled velocity v^ = RN((v * Z0) / P0), Z0 = max rho * max c (the same
 * scaling, Section 5, "Range"). */
void orc_scale_velocity(int64_t n, const double *in, double Z0, double P0, int fmt, double *out)
{
    for (int64_t i = 0; i < n; i++) out[i] = orc_round((in[i] * Z0) / P0, fmt);
}

/* A point source of strength w(t) on the pressure equation, as a discrete
 * delta w / h^d, enters R (undivided-difference units) as
 * s^ = RN(w * (Z0 / (P0 * h^(d-1)))), with h^(d-1) = h (2D) or h * h (3D). */
void orc_scale_source(int64_t nt, const double *w, double Z0, double P0, double h, int ndim,
                      int fmt, double *out)
{
    const double hd1 = (ndim == 2) ? h : h * h;
    const double scale = Z0 / (P0 * hd1);
    for (int64_t i = 0; i < nt; i++) out[i] = orc_round(w[i] * scale, fmt);
}

/* Physical energy from the scaled one (the discrete energy of Section 3):
 * E = 0.5 * h^(d-1) * P0^2 * dt / Z0 * E^ */
double orc_energy_factor(double h, double dt, double P0, double Z0, int ndim)
{
    const double hd1 = (ndim == 2) ? h : h * h;
    return 0.5 * hd1 * P0 * P0 * dt / Z0;
}

/* ------------------------------------------------------------------------ */
/* 2D isotropic elastic velocity-stress leapfrog (Eq. 2, Appendix A).       */
/* ------------------------------------------------------------------------ */
/* Grid (Virieux staggering, the reading of the missing Fig. 1 extended to
 * Eq. 2): sxx, syy at nodes (i, j); vx at (i+1/2, j); vy at (i, j+1/2);
 * sxy at (i+1/2, j+1/2). All fields stored n[0] x n[1], x fastest; y grows
 * downwards, row 0 is the top.
 * Boundary kinds per face (x-lo, x-hi, y-lo, y-hi):
 *   ORC_BC_PERIODIC (both faces of an axis): wrap.
 *   ORC_EBC_RIGID: frictionless rigid wall on the half points -1/2 and
 *     N-1/2: the normal velocity and the shear stress are odd about the wall
 *     (zero on it; the stored point at N-1 is held at zero), the tangential
 *     velocity and the normal stresses are even.
 *   ORC_EBC_FREE (y-lo only): traction-free surface (the free surface in y
 *     of Appendix A) on the node row j = 0, by stress imaging: syy is held at
 *     zero on that row, and above it syy and sxy are odd images of the rows
 *     below (so both tractions vanish on the surface), while vx and vy are
 *     even images. On the surface row itself syy = 0 leaves
 *     d(sxx)/dt = (lambda + 2 mu - lambda^2 / (lambda + 2 mu)) d(vx)/dx, so the
 *     multipliers there are l2m <- that reduced modulus and lam <- 0 (Dy vy
 *     vanishes on the row because vy is even about it, so syy stays zero).
 * Each closure keeps the map from stress to velocity the exact negative
 * adjoint of the map from velocity to strain rate, in an inner product with
 * unit weights except weight 1/2 on the vx and sxx points of a free surface
 * row (that row lies on the mirror plane of the images), so the discrete
 * energy with those weights is exactly conserved. */
enum { ORC_EBC_RIGID = 1, ORC_EBC_FREE = 2, ORC_EBC_ZERO = 3 };
/* ORC_EBC_ZERO is not a physical boundary: every field reads zero beyond the
 * face. It lets a sub-box of a larger grid be stepped over the domain of
 * dependence of its centre (the values near a cut face are wrong, the centre
 * is not). */

typedef struct {
    int64_t n[2];
    int32_t bc[4];
    int32_t store_fmt, arith_fmt, stencil_fmt, comp;
    int32_t pair_stencil;  /* with comp: the stencils read RN(V + T) (not the paper) */
} orc_elastic_cfg;

/* Image of index m along an axis of N points for a field that is node-type
 * (node = 1) or half-type (node = 0) along that axis. odd: parity about a
 * rigid wall (normal velocity, shear stress); odd_free: parity about a free
 * surface (the stresses syy and sxy that carry a y traction; the velocities
 * are even). lo_bc / hi_bc are the two faces' kinds.
 * Returns the sign (+1, -1) or 0 for "reads zero". */
static int e_map(int64_t m, int64_t N, int lo_bc, int hi_bc, int node, int odd, int odd_free,
                 int64_t *out)
{
    if (m >= 0 && m < N) { *out = m; return 1; }
    int bc = m < 0 ? lo_bc : hi_bc;
    if (bc == ORC_BC_PERIODIC) { *out = ((m % N) + N) % N; return 1; }
    if (bc == ORC_EBC_ZERO) return 0;
    if (bc == ORC_EBC_FREE) {
        /* mirror plane: the node row 0 (free surfaces are low faces only);
         * node m <-> -m, half point m + 1/2 <-> -1-m */
        *out = node ? -m : -1 - m;
        return odd_free ? -1 : 1;
    }
    /* rigid wall at -1/2 (low) or N-1/2 (high) */
    if (node) {                       /* node m <-> -1-m, 2N-1-m */
        *out = m < 0 ? -1 - m : 2 * N - 1 - m;
        return odd ? -1 : 1;
    }
    /* half point m + 1/2 <-> -2-m (low), 2N-2-m (high); -1 is on the wall */
    if (m == -1) { if (odd) return 0; *out = 0; return 1; }
    *out = m < 0 ? -2 - m : 2 * N - 2 - m;
    return odd ? -1 : 1;
}

static double e_read(const double *f, const orc_elastic_cfg *c, int ax, int node, int odd,
                     int odd_free, int64_t i, int64_t j, int64_t m)
{
    int64_t idx[2] = {i, j}, mm;
    int s = e_map(m, c->n[ax], c->bc[2 * ax], c->bc[2 * ax + 1], node, odd, odd_free, &mm);
    if (s == 0) return 0.0;
    idx[ax] = mm;
    double v = f[idx[0] + c->n[0] * idx[1]];
    return s > 0 ? v : -v;
}

/* Points a boundary holds at zero (the elastic boundaries of Appendix A as
 * read here): vx and sxy on column N-1 (rigid x, frictionless walls on the
 * half points), vy and sxy on row N-1 (rigid y-hi), syy on row 0 (free
 * surface at y-lo). */
void orc_elastic_apply_walls(const orc_elastic_cfg *c, double *vx, double *vy, double *syy,
                             double *sxy)
{
    const int64_t nx = c->n[0], ny = c->n[1];
    for (int64_t j = 0; j < ny; j++)
        for (int64_t i = 0; i < nx; i++) {
            int64_t q = i + nx * j;
            if (c->bc[1] == ORC_EBC_RIGID && i == nx - 1) { vx[q] = 0.0; sxy[q] = 0.0; }
            if (c->bc[3] == ORC_EBC_RIGID && j == ny - 1) { vy[q] = 0.0; sxy[q] = 0.0; }
            if (c->bc[2] == ORC_EBC_FREE && j == 0) syy[q] = 0.0;
        }
}

/* Stencil of field f along axis ax around the target, whose offsets to f's
 * points are -3/2..+3/2: f's indices base-1..base+2 (node-type f targeted at a
 * half point, base = target index) or base-2..base+1 (half-type f targeted at
 * a node, base = target index). */
static double e_stencil(const double *f, const orc_elastic_cfg *c, int ax, int node, int odd,
                        int odd_free, int64_t i, int64_t j, int fmt)
{
    const int64_t m = ax == 0 ? i : j;
    const int64_t first = node ? m - 1 : m - 2;
    double a0 = e_read(f, c, ax, node, odd, odd_free, i, j, first);
    double a1 = e_read(f, c, ax, node, odd, odd_free, i, j, first + 1);
    double a2 = e_read(f, c, ax, node, odd, odd_free, i, j, first + 2);
    double a3 = e_read(f, c, ax, node, odd, odd_free, i, j, first + 3);
    return stencil(a0, a1, a2, a3, fmt);
}

/* One elastic leapfrog step per iteration, Eq. 2 in Algorithm 1 / 2 form:
 *   vx += bx * (Dx sxx + Dy sxy)
 *   vy += by * (Dx sxy + Dy syy)            [+ s, added to the increment]
 *   sxx += (l2m * Dx vx) + (lam * Dy vy)
 *   syy += (lam * Dx vx) + (l2m * Dy vy)
 *   sxy += mu * (Dx vy + Dy vx)
 * Energy (scaled) after each step, with the rounded multipliers:
 *   E = sum w vx^2/bx + sum vy^2/by
 *     + sum over nodes w (l2m (sxx sxx' + syy syy') - lam (sxx syy' + syy sxx')) / (l2m^2 - lam^2)
 *     + sum sxy sxy' / mu              (primes: after the step)
 * with w = 1/2 on the row of a free surface (there lam = 0 and syy = 0, so the
 * node term is sxx sxx' / l2m with the reduced modulus) and w = 1 elsewhere.
 * With pair_stencil (and comp) the stencils read RN(V + T) in the stencil
 * format, formed for the stresses before the velocity half step and for the
 * velocities before the stress half step; the energy reads the stored V. */
int orc_elastic_run(const orc_elastic_cfg *c, double *vx, double *tvx, double *vy, double *tvy,
                    double *sxx, double *tsxx, double *syy, double *tsyy, double *sxy,
                    double *tsxy, const double *bx, const double *by, const double *l2m,
                    const double *lam, const double *mu, int64_t nsteps, int64_t step0,
                    int64_t src_index, int64_t src_nt, const double *src, int32_t rec_field,
                    int64_t nrec, const int64_t *rec_index, double *traces, double *energy)
{
    const int64_t nx = c->n[0], ny = c->n[1], npts = nx * ny;
    const int sf = c->store_fmt, af = c->arith_fmt, stf = c->stencil_fmt, comp = c->comp;
    double *rowacc = (double *)calloc((size_t)ny, sizeof(double));
    if (!rowacc) return -1;
    /* what the stencils read: the stored values, or RN(V + T) (pair_stencil) */
    const double *rxx = sxx, *ryy = syy, *rxy = sxy, *rvx = vx, *rvy = vy;
    double *pairs = NULL;
    if (c->pair_stencil && comp) {
        pairs = (double *)malloc(sizeof(double) * (size_t)npts * 5);
        if (!pairs) { free(rowacc); return -1; }
        rxx = pairs; ryy = pairs + npts; rxy = pairs + 2 * npts; rvx = pairs + 3 * npts; rvy = pairs + 4 * npts;
    }
    for (int64_t s = 0; s < nsteps; s++) {
        const int64_t gstep = step0 + s;
        if (pairs)
            for (int64_t q = 0; q < npts; q++) {
                pairs[q] = add_f(sxx[q], tsxx[q], stf);
                pairs[npts + q] = add_f(syy[q], tsyy[q], stf);
                pairs[2 * npts + q] = add_f(sxy[q], tsxy[q], stf);
            }
#pragma omp parallel for schedule(static)
        for (int64_t j = 0; j < ny; j++)
            for (int64_t i = 0; i < nx; i++) {
                const int64_t q = i + nx * j;
                /* vx at (i+1/2, j): sxx node-type in x (even); sxy half-type in y (odd at
                 * rigid walls and at the free surface) */
                double R = add_f(e_stencil(rxx, c, 0, 1, 0, 1, i, j, stf),
                                 e_stencil(rxy, c, 1, 0, 1, 1, i, j, stf), stf);
                double inc = orc_round(mul_f(bx[q], R, stf), af);
                update(&vx[q], &tvx[q], inc, comp, af, sf);
                /* vy at (i, j+1/2): sxy half-type in x (odd); syy node-type in y (even at
                 * rigid walls, odd at the free surface) */
                R = add_f(e_stencil(rxy, c, 0, 0, 1, 1, i, j, stf),
                          e_stencil(ryy, c, 1, 1, 0, 1, i, j, stf), stf);
                inc = orc_round(mul_f(by[q], R, stf), af);
                if (src && q == src_index && gstep < src_nt) inc = add_f(inc, src[gstep], af);
                update(&vy[q], &tvy[q], inc, comp, af, sf);
            }
        if (pairs)
            for (int64_t q = 0; q < npts; q++) {
                pairs[3 * npts + q] = add_f(vx[q], tvx[q], stf);
                pairs[4 * npts + q] = add_f(vy[q], tvy[q], stf);
            }
#pragma omp parallel for schedule(static)
        for (int64_t j = 0; j < ny; j++) {
            acc_t e = {0.0, 0.0};
            for (int64_t i = 0; i < nx; i++) {
                const int64_t q = i + nx * j;
                /* nodes: vx half-type in x (odd), vy half-type in y (odd at rigid walls,
                 * even at the free surface) */
                const double dxvx = e_stencil(rvx, c, 0, 0, 1, 0, i, j, stf);
                const double dyvy = e_stencil(rvy, c, 1, 0, 1, 0, i, j, stf);
                const double sxx0 = sxx[q], syy0 = syy[q], sxy0 = sxy[q];
                double inc = orc_round(add_f(mul_f(l2m[q], dxvx, stf), mul_f(lam[q], dyvy, stf), stf), af);
                update(&sxx[q], &tsxx[q], inc, comp, af, sf);
                inc = orc_round(add_f(mul_f(lam[q], dxvx, stf), mul_f(l2m[q], dyvy, stf), stf), af);
                update(&syy[q], &tsyy[q], inc, comp, af, sf);
                /* sxy at (i+1/2, j+1/2): vy node-type in x (even), vx node-type in y (even) */
                double R = add_f(e_stencil(rvy, c, 0, 1, 0, 0, i, j, stf),
                                 e_stencil(rvx, c, 1, 1, 0, 0, i, j, stf), stf);
                inc = orc_round(mul_f(mu[q], R, stf), af);
                update(&sxy[q], &tsxy[q], inc, comp, af, sf);
                if (energy) {
                    const double w = (c->bc[2] == ORC_EBC_FREE && j == 0) ? 0.5 : 1.0;
                    acc_add(&e, w * (vx[q] * vx[q] / bx[q]));
                    acc_add(&e, vy[q] * vy[q] / by[q]);
                    const double det = l2m[q] * l2m[q] - lam[q] * lam[q];
                    acc_add(&e, w * ((l2m[q] * (sxx0 * sxx[q] + syy0 * syy[q]) -
                                      lam[q] * (sxx0 * syy[q] + syy0 * sxx[q])) / det));
                    if (mu[q] > 0.0) acc_add(&e, sxy0 * sxy[q] / mu[q]);
                }
            }
            rowacc[j] = acc_val(&e);
        }
        if (energy) {
            acc_t e = {0.0, 0.0};
            for (int64_t j = 0; j < ny; j++) acc_add(&e, rowacc[j]);
            energy[s] = acc_val(&e);
        }
        if (traces && nrec > 0) {
            const double *f = rec_field == 1 ? vx : rec_field == 2 ? vy : rec_field == 4 ? sxx
                              : rec_field == 5 ? syy : sxy;
            for (int64_t r = 0; r < nrec; r++) traces[s * nrec + r] = f[rec_index[r]];
        }
    }
    free(rowacc);
    free(pairs);
    return 0;
}

/* Elastic multipliers, binary64 in exactly this order, each rounded once:
 *   Z0 = max(rho) * max(vp)
 *   bx = ((dt * Z0) / h) / rho_x,   rho_x = (rho[i] + rho[i+1]) * 0.5
 *   by = ((dt * Z0) / h) / rho_y,   rho_y = (rho[j] + rho[j+1]) * 0.5
 *   mu = (rho * vs) * vs,  lambda = ((rho * vp) * vp) - (2.0 * mu)
 *   l2m = ((dt * (lambda + 2.0 * mu)) / Z0) / h,  lam = ((dt * lambda) / Z0) / h
 *   mu_xy = 4 / (1/mu00 + 1/mu10 + 1/mu01 + 1/mu11) (0 if any is 0)
 *   mu = ((dt * mu_xy) / Z0) / h
 * On the row of a free surface (y-lo FREE, j = 0), where syy = 0:
 *   M = ((4.0 * mu) * (lambda + mu)) / (lambda + 2.0 * mu)
 *     (= lambda + 2 mu - lambda^2 / (lambda + 2 mu), the modulus of sxx
 *     under zero normal traction)
 *   l2m = ((dt * M) / Z0) / h,  lam = 0
 * The neighbour index i+1 (j+1) wraps on periodic axes and is clamped to the
 * last point otherwise. Returns 0, or 1 if bx, by, l2m are not positive
 * normal numbers or lam, mu are neither zero nor normal, or l2m <= |lam|. */
int orc_elastic_coefficients(const orc_elastic_cfg *c, double h, double dt, const double *rho,
                             const double *vp, const double *vs, double *bx, double *by,
                             double *l2m, double *lam, double *mu, double *Z0_out)
{
    const int64_t nx = c->n[0], ny = c->n[1], npts = nx * ny;
    const int sf = c->store_fmt;
    double rho0 = 0.0, c0 = 0.0;
    for (int64_t q = 0; q < npts; q++) {
        if (rho[q] > rho0) rho0 = rho[q];
        if (vp[q] > c0) c0 = vp[q];
    }
    const double Z0 = rho0 * c0;
    *Z0_out = Z0;
    const double tiny = ldexp(1.0, FORMATS[sf].emin);
    int bad = 0;
#define LAMEMU(q, m_, l_) do { m_ = (rho[q] * vs[q]) * vs[q]; l_ = ((rho[q] * vp[q]) * vp[q]) - (2.0 * m_); } while (0)
    for (int64_t j = 0; j < ny; j++)
        for (int64_t i = 0; i < nx; i++) {
            const int64_t q = i + nx * j;
            int64_t i1 = i + 1 < nx ? i + 1 : (c->bc[1] == ORC_BC_PERIODIC ? 0 : i);
            int64_t j1 = j + 1 < ny ? j + 1 : (c->bc[3] == ORC_BC_PERIODIC ? 0 : j);
            const double rx = (rho[q] + rho[i1 + nx * j]) * 0.5;
            const double ry = (rho[q] + rho[i + nx * j1]) * 0.5;
            bx[q] = orc_round(((dt * Z0) / h) / rx, sf);
            by[q] = orc_round(((dt * Z0) / h) / ry, sf);
            double m00, l00, m10, l10, m01, l01, m11, l11;
            LAMEMU(q, m00, l00);
            LAMEMU(i1 + nx * j, m10, l10);
            LAMEMU(i + nx * j1, m01, l01);
            LAMEMU(i1 + nx * j1, m11, l11);
            (void)l10; (void)l01; (void)l11;
            if (c->bc[2] == ORC_EBC_FREE && j == 0) {
                const double M = ((4.0 * m00) * (l00 + m00)) / (l00 + 2.0 * m00);
                l2m[q] = orc_round(((dt * M) / Z0) / h, sf);
                lam[q] = 0.0;
            } else {
                l2m[q] = orc_round(((dt * (l00 + 2.0 * m00)) / Z0) / h, sf);
                lam[q] = orc_round(((dt * l00) / Z0) / h, sf);
            }
            double mh = 0.0;
            if (m00 > 0.0 && m10 > 0.0 && m01 > 0.0 && m11 > 0.0)
                mh = 4.0 / (1.0 / m00 + 1.0 / m10 + 1.0 / m01 + 1.0 / m11);
            mu[q] = orc_round(((dt * mh) / Z0) / h, sf);
            if (!(bx[q] >= tiny && isfinite(bx[q])) || !(by[q] >= tiny && isfinite(by[q])) ||
                !(l2m[q] >= tiny && isfinite(l2m[q])) ||
                !((lam[q] == 0.0 || fabs(lam[q]) >= tiny) && isfinite(lam[q])) ||
                !((mu[q] == 0.0 || mu[q] >= tiny) && isfinite(mu[q])) || !(l2m[q] > fabs(lam[q])))
                bad = 1;
        }
#undef LAMEMU
    return bad;
}

/* Elastic v_y source in increment units: s^ = RN(w * ((dt * Z0) / (P0 * (h * h)))) */
void orc_elastic_scale_source(int64_t nt, const double *w, double dt, double Z0, double P0,
                              double h, int fmt, double *out)
{
    const double scale = (dt * Z0) / (P0 * (h * h));
    for (int64_t i = 0; i < nt; i++) out[i] = orc_round(w[i] * scale, fmt);
}
