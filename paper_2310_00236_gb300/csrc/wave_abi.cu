// wave_abi.cu -- the C ABI of include/wave.h: argument checking, coefficient
// preparation (binary64, rounded once), device state, step launches, I/O.
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <thread>
#include <vector>

#include "../../include/wave.h"
#include "acoustic_common.cuh"
#include "adjoint.h"
#include "batch.h"
#include "elastic.h"
#include "wave_kernels.h"

using namespace wave;

// ------------------------------------------------------------------ errors
static thread_local char g_err[512] = "";

static wave_status fail(wave_status st, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
    return st;
}

extern "C" const char *wave_last_error(void) { return g_err; }

namespace wave {
void set_last_error_text(const char *msg) { snprintf(g_err, sizeof g_err, "%s", msg); }
}  // namespace wave

extern "C" const char *wave_build_info(void) {
    return "libwave: sm_103a, -fmad=false, explicit .rn half/bfloat16/binary32 arithmetic";
}

// ------------------------------------------------------------- allocation
static wave_alloc_fn g_alloc = nullptr;
static wave_free_fn g_free = nullptr;
static void *g_alloc_user = nullptr;

extern "C" wave_status wave_set_allocator(wave_alloc_fn alloc, wave_free_fn free_fn, void *user) {
    if ((alloc == nullptr) != (free_fn == nullptr))
        return fail(WAVE_EINVAL, "wave_set_allocator: give both functions or neither");
    g_alloc = alloc;
    g_free = free_fn;
    g_alloc_user = user;
    return WAVE_OK;
}

struct DevBuf {
    void *ptr = nullptr;
    size_t bytes = 0;
    wave_free_fn free_fn = nullptr;  // allocator that owns it (nullptr: cudaFreeAsync)
    void *user = nullptr;
};

// ------------------------------------------------------------ host rounding
// Round a binary64 value to a binary format with `mant` fraction bits and
// `expb` exponent bits, to nearest with ties to even, with gradual underflow
// and overflow to infinity. Works on the integer fields of the binary64.
static uint16_t round_bits16(double x, int mant, int expb) {
    uint64_t u;
    memcpy(&u, &x, 8);
    const uint32_t sign = (u >> 63) ? (1u << (mant + expb)) : 0u;
    const uint32_t ex = (uint32_t)((u >> 52) & 0x7FF);
    const uint64_t fr = u & ((1ull << 52) - 1);
    const int bias = (1 << (expb - 1)) - 1;
    const uint32_t inf = ((1u << expb) - 1) << mant;
    if (ex == 0x7FF) return (uint16_t)(sign | inf | (fr ? (1u << (mant - 1)) : 0u));
    if (ex == 0) return (uint16_t)sign;
    const int e = (int)ex - 1023;
    const uint64_t m = fr | (1ull << 52);
    const int emin = 1 - bias;
    const int shift = 52 - mant + (e < emin ? emin - e : 0);
    if (shift > 53) return (uint16_t)sign;
    uint64_t q = m >> shift;
    const uint64_t rem = m & ((1ull << shift) - 1);
    const uint64_t halfway = 1ull << (shift - 1);
    if (rem > halfway || (rem == halfway && (q & 1))) q++;
    uint32_t bits = (e < emin) ? (uint32_t)q
                               : ((uint32_t)(e + bias) << mant) + (uint32_t)q - (1u << mant);
    if (bits >= inf) bits = inf;
    return (uint16_t)(sign | bits);
}

static double half_to_double(uint16_t h) {
    const int s = h >> 15, e = (h >> 10) & 0x1F, m = h & 0x3FF;
    double v;
    if (e == 0) v = ldexp((double)m, -24);
    else if (e == 31) v = m ? NAN : INFINITY;
    else v = ldexp((double)(m + 1024), e - 25);
    return s ? -v : v;
}

static double bf16_to_double(uint16_t b) {
    uint32_t u = (uint32_t)b << 16;
    float f;
    memcpy(&f, &u, 4);
    return (double)f;
}

// Storage-format helpers keyed by precision.
static int elem_bytes(int prec) { return prec == PREC_FP32 ? 4 : 2; }
static bool is_bf16_storage(int prec) { return prec == PREC_BF16 || prec == PREC_BF16_F32ARITH; }
static bool arith_is_f32(int prec) {
    return prec == PREC_FP32 || prec == PREC_FP16_F32ARITH || prec == PREC_BF16_F32ARITH ||
           prec == PREC_FP16_PAIRS;
}

// Format of the multipliers a and b: the storage format, except binary32 for
// the pair precision (whose stencils read V + T; the multipliers' rounding to
// binary16 would then be the largest error left).
static int coef_prec(int prec) { return prec == PREC_FP16_PAIRS ? PREC_FP32 : prec; }

// value -> storage bits (uint16 or float bits) ; returns false if not finite
static inline void store_value(int prec, double x, void *dst, int64_t i) {
    if (prec == PREC_FP32) {
        static_cast<float *>(dst)[i] = (float)x;
    } else if (is_bf16_storage(prec)) {
        static_cast<uint16_t *>(dst)[i] = round_bits16(x, 7, 8);
    } else {
        static_cast<uint16_t *>(dst)[i] = round_bits16(x, 10, 5);
    }
}

static inline double load_value(int prec, const void *src, int64_t i) {
    if (prec == PREC_FP32) return (double)static_cast<const float *>(src)[i];
    if (is_bf16_storage(prec)) return bf16_to_double(static_cast<const uint16_t *>(src)[i]);
    return half_to_double(static_cast<const uint16_t *>(src)[i]);
}

// Smallest positive normal number of the storage format.
static double min_normal(int prec) {
    return (prec == PREC_FP16 || prec == PREC_FP16_F32ARITH || prec == PREC_FP16_PAIRS) ? ldexp(1.0, -14)
                                                                                           : ldexp(1.0, -126);
}

// Parallel loop over [0, n) on the host.
template <class F>
static void parallel_for(int64_t n, F f) {
    unsigned nt = std::thread::hardware_concurrency();
    if (nt == 0) nt = 1;
    if (nt > 32) nt = 32;
    if (n < (int64_t)1 << 20 || nt == 1) {
        f((int64_t)0, n);
        return;
    }
    std::vector<std::thread> th;
    int64_t chunk = (n + nt - 1) / nt;
    for (unsigned t = 0; t < nt; t++) {
        int64_t lo = t * chunk, hi = std::min(n, lo + chunk);
        if (lo >= hi) break;
        th.emplace_back([=]() { f(lo, hi); });
    }
    for (auto &x : th) x.join();
}

// z planes per block of the one-pass 3D step: 32 (each block recomputes 3
// warm-up planes, so longer chunks waste less; at 512^3 16 / 20 / 24 / 28 /
// 32 / 40 planes gave 152.6 / 158.2 / 160.6 / 161.8 / 162.5 / 161.9 Gpt/s),
// halved while the grid would have fewer blocks than the GPU runs at once
// (4 per SM), down to 6.
static int fused_zchunk_for(const AcParams &prm, int prec, int sms) {
    int zc = 32;
    while (zc > 6 && (int64_t)acoustic_fused_blocks(prm, prec, zc) < 4 * (int64_t)sms) zc /= 2;
    return zc;
}

// Launch shape of the row-strip kernels for single 2D problems: 4 warps per
// block; rows per work item from the options (zchunk) or chosen so that the
// grid yields about 12 warps per SM (at most 16 rows: small grids get short
// items, large grids long ones that re-read fewer halo rows). Measured on
// 1024^2: 2 rows per item 50.6 (elastic) and 71.5 (acoustic) Gpt/s, 16 rows
// 16.4 and 31.9.
constexpr int kStripWarps = 4, kStripGraphLevels = 6;  // graphs of 1, 2, 4, ..., 32 steps
static int strip_rows_for(int64_t nstrips, int64_t ny, int sms) {
    const int64_t r = nstrips * ny / (12 * (int64_t)sms);
    return (int)std::max<int64_t>(1, std::min<int64_t>(16, r));
}

// ---------------------------------------------------------------- context
struct wave_ctx {
    int kind = WAVE_ACOUSTIC;
    int ndim = 2;
    int64_t n[3] = {1, 1, 1};
    int64_t pitch = 0, plane = 0, total = 0;  // elements
    int bc[6] = {0, 0, 0, 0, 0, 0};
    int prec = PREC_FP16, comp = 0;
    int kernel_choice = 0;
    int zchunk = 16;
    bool zchunk_set = false;
    bool use_stream = false;
    bool use_fused = false;
    // 2D: the row-strip kernels of the batches, as a batch of one; acoustic
    // strip_fused: the one-pass strips (both half steps in one launch, the
    // state alternating between f / t and alt_f / alt_t)
    bool use_strips = false;
    bool strip_fused = false;
    // 2D acoustic: the cluster-resident steps (the whole state in the shared
    // memory of one cluster, one launch per wave_step call)
    bool use_cluster = false;
    ClusterPlan cplan;
    int strip_items = 0, strip_grid = 0, strip_rows = 16;
    // plain strip steps replayed from captured graphs of 2^j steps (j < kStripGraphLevels)
    cudaGraphExec_t strip_graph[kStripGraphLevels] = {};
    DevBuf strip_shot, strip_item0, strip_part;
    // second set of p, vx, vy, vz and t_vx, t_vy, t_vz for the one-pass step,
    // and the tensor maps of both sets (fset: the set the fields point to now)
    DevBuf alt_f[4], alt_t[4];
    struct alignas(64) MapBlob { unsigned char b[2048]; } fmaps[2];
    int fset = 0;
    double h = 0, dt = 0, P0 = 1.0, Z0 = 1.0;
    // z slab of a larger grid: cut faces (bit 0 z-lo, bit 1 z-hi), the ghost
    // planes (p lo, p hi, v_z lo, v_z hi), whether a velocity half step awaits
    // its pressure half
    int z_cut = 0;
    const void *zg[4] = {nullptr, nullptr, nullptr, nullptr};
    bool half_open = false;
    cudaStream_t stream = nullptr;
    bool poisoned = false;
    int64_t step = 0;
    bool have_energy = false;

    // fields and compensations; acoustic: 0 p, 1 vx, 2 vy, 3 vz
    // elastic: 1 vx, 2 vy, 4 sxx, 5 syy, 6 sxy
    DevBuf f[7], t[7];
    // coefficients (per-point arrays when not uniform)
    DevBuf coef[6];
    uint32_t coef_uni[6] = {0, 0, 0, 0, 0, 0};
    bool coef_is_uniform[6] = {false, false, false, false, false, false};
    std::vector<double> coef_host[6];

    DevBuf e_part, e_misc;   // e_misc: [double e_last][unsigned counter]
    unsigned e_blocks = 0;
    double *e_trace = nullptr;
    int64_t e_trace_cap = 0, e_trace_pos = 0;

    DevBuf src_table;
    int64_t src_q = -1, src_nt = 0;
    int src_field = -1;

    // per-kernel timing (measurement aid)
    bool timing = false;
    struct TimedLaunch { int kind; cudaEvent_t a, b; };
    std::vector<TimedLaunch> pending;
    std::vector<cudaEvent_t> event_pool;
    int64_t t_launches[4] = {0, 0, 0, 0};
    double t_ms[4] = {0, 0, 0, 0};

    DevBuf rec_q;
    int64_t nrec = 0;
    int rec_field = 0;
    float *rec_traces = nullptr;
    int64_t rec_cap = 0, rec_pos = 0;

    std::vector<float> src_host;    // scaled source values (arithmetic format, as binary32)
    std::vector<float> two_over_c;  // acoustic: 2 / c per node (dJ/dc = (2 / c) dJ/db * b)

    // recorded forward run and adjoint state (wave_record / wave_adjoint_step)
    struct Adjoint {
        bool active = false;
        int64_t nsteps = 0, step0 = 0, K = 0, ncp = 0, t = 0;
        int narr = 0;
        DevBuf cps;                   // ncp + 1 snapshots of narr arrays; slot ncp: the end state
        std::vector<int64_t> cp_step;
        DevBuf seg;                   // v^{n+1/2} of up to K steps (ndim arrays each)
        int64_t seg_lo = -1, seg_n = 0;
        DevBuf mu, nu[3], g;          // binary32, pitched like the fields
        // one-pass adjoint leapfrog (3D, uniform a_c): the second buffer set
        // of mu~, nu~ and the tensor maps of both sets (fm[fset]: current)
        bool fused = false;
        DevBuf mu_alt, nu_alt[3];
        MapBlob fm[2];
        int fset = 0;
        uint32_t na_uni[3] = {0, 0, 0}, nb_uni = 0;
        DevBuf rec_w;                 // residual weight per receiver (b, 0 on rigid walls)
        DevBuf rec_order, rec_start;  // receivers grouped by point, in receiver order
        int ngroups = 0;
    } adj;
    // made by the first wave_record, kept for the context's lifetime
    DevBuf adj_na[3], adj_nb;         // negated multipliers (binary32) where per-point
    DevBuf adj_two_over_c;            // 2 / c, unpitched
};

static bool field_valid(const wave_ctx *c, int field) {
    if (c->kind == WAVE_ACOUSTIC) return field >= 0 && field <= (c->ndim == 3 ? 3 : 2);
    return field == WAVE_F_VX || field == WAVE_F_VY || field == WAVE_F_SXX ||
           field == WAVE_F_SYY || field == WAVE_F_SXY;
}

static wave_status dev_alloc(wave_ctx *c, DevBuf &b, size_t bytes, bool zero = true) {
    b.bytes = bytes;
    if (bytes == 0) return WAVE_OK;
    if (g_alloc) {
        b.ptr = g_alloc(bytes, (void *)c->stream, g_alloc_user);
        b.free_fn = g_free;
        b.user = g_alloc_user;
        if (!b.ptr) return fail(WAVE_ENOMEM, "allocator returned NULL for %zu bytes", bytes);
    } else {
        cudaError_t e = cudaMallocAsync(&b.ptr, bytes, c->stream);
        if (e != cudaSuccess) {
            b.ptr = nullptr;
            cudaGetLastError();
            return fail(e == cudaErrorMemoryAllocation ? WAVE_ENOMEM : WAVE_ECUDA,
                        "cudaMallocAsync(%zu): %s", bytes, cudaGetErrorString(e));
        }
    }
    if (!zero) return WAVE_OK;
    cudaError_t e = cudaMemsetAsync(b.ptr, 0, bytes, c->stream);
    if (e != cudaSuccess) return fail(WAVE_ECUDA, "cudaMemsetAsync: %s", cudaGetErrorString(e));
    return WAVE_OK;
}

static void dev_free(wave_ctx *c, DevBuf &b) {
    if (!b.ptr) return;
    if (b.free_fn) b.free_fn(b.ptr, b.bytes, (void *)c->stream, b.user);
    else cudaFreeAsync(b.ptr, c->stream);
    b.ptr = nullptr;
    b.bytes = 0;
}

static wave_status cuda_check(wave_ctx *c, cudaError_t e, const char *what) {
    if (e == cudaSuccess) return WAVE_OK;
    c->poisoned = true;
    return fail(WAVE_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

static wave_status check_device_error(wave_ctx *c);

#define CHECK_CTX(c)                                                                  \
    do {                                                                              \
        if (!(c)) return fail(WAVE_EINVAL, "%s: NULL context", __func__);             \
        if ((c)->poisoned) return fail(WAVE_ESTATE, "%s: context poisoned", __func__); \
    } while (0)

// Copy a packed host array (n[0]*n[1]*n[2] elements) into a pitched field.
static wave_status upload_packed(wave_ctx *c, void *dev, const void *host, size_t eb = 0) {
    if (!eb) eb = elem_bytes(c->prec);
    cudaError_t e = cudaMemcpy2DAsync(dev, c->pitch * eb, host, c->n[0] * eb, c->n[0] * eb,
                                      c->n[1] * c->n[2], cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    return cuda_check(c, e, "upload");
}

static wave_status download_packed(wave_ctx *c, const void *dev, void *host) {
    const size_t eb = elem_bytes(c->prec);
    cudaError_t e = cudaMemcpy2DAsync(host, c->n[0] * eb, dev, c->pitch * eb, c->n[0] * eb,
                                      c->n[1] * c->n[2], cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    return cuda_check(c, e, "download");
}

// ------------------------------------------------------- acoustic creation
static wave_status acoustic_coefficients(wave_ctx *c, const wave_materials *mat, double z0_opt,
                                         const double *rho_above) {
    const int64_t npts = c->n[0] * c->n[1] * c->n[2];
    double rho0 = 0.0, c0 = 0.0;
    for (int64_t q = 0; q < npts; q++) {
        if (!(mat->rho[q] > 0.0) || !isfinite(mat->rho[q]) || !(mat->vp[q] > 0.0) ||
            !isfinite(mat->vp[q]))
            return fail(WAVE_ERANGE, "material value at point %lld is not positive and finite",
                        (long long)q);
        if (mat->rho[q] > rho0) rho0 = mat->rho[q];
        if (mat->vp[q] > c0) c0 = mat->vp[q];
    }
    const double Z0 = z0_opt > 0.0 ? z0_opt : rho0 * c0;
    c->Z0 = Z0;
    const double h = c->h, dt = c->dt;
    const int cp = coef_prec(c->prec);
    const double tiny = min_normal(cp);
    if (rho_above)
        for (int64_t q = 0; q < c->n[0] * c->n[1]; q++)
            if (!(rho_above[q] > 0.0) || !isfinite(rho_above[q]))
                return fail(WAVE_ERANGE, "rho_above at point %lld is not positive and finite", (long long)q);
    for (int w = 0; w < 4; w++) c->coef_host[w].assign(npts, 0.0);
    c->two_over_c.resize(npts);
    for (int64_t q = 0; q < npts; q++) c->two_over_c[q] = (float)(2.0 / mat->vp[q]);
    std::vector<double> &b = c->coef_host[0];
    const int64_t nx = c->n[0], ny = c->n[1];
    const int64_t str[3] = {1, nx, nx * ny};
    bool bad = false;
    int64_t bad_q = -1;
    for (int64_t q = 0; q < npts; q++) {
        const int64_t idx[3] = {q % nx, (q / nx) % ny, q / (nx * ny)};
        double v = (((dt * mat->rho[q]) * mat->vp[q]) * mat->vp[q]) / (Z0 * h);
        double r;
        {
            uint16_t tmp16;
            float tmp32;
            if (cp == PREC_FP32) { tmp32 = (float)v; r = tmp32; }
            else { store_value(cp, v, &tmp16, 0); r = load_value(cp, &tmp16, 0); }
        }
        b[q] = r;
        if (!(r >= tiny) || !isfinite(r)) { bad = true; bad_q = q; }
        for (int ax = 0; ax < c->ndim; ax++) {
            int64_t m = idx[ax] + 1;
            if (m >= c->n[ax]) m = (c->bc[2 * ax] == WAVE_BC_PERIODIC) ? 0 : idx[ax];
            const int64_t nb = q + (m - idx[ax]) * str[ax];
            // a slab's last plane averages with the grid plane above a cut face
            const bool across = ax == 2 && (c->z_cut & 2) && idx[2] == c->n[2] - 1;
            const double rho_c = (mat->rho[q] + (across ? rho_above[q % (nx * ny)] : mat->rho[nb])) * 0.5;
            double av = ((dt * Z0) / h) / rho_c;
            double ar;
            uint16_t tmp16;
            float tmp32;
            if (cp == PREC_FP32) { tmp32 = (float)av; ar = tmp32; }
            else { store_value(cp, av, &tmp16, 0); ar = load_value(cp, &tmp16, 0); }
            c->coef_host[1 + ax][q] = ar;
            if (!(ar >= tiny) || !isfinite(ar)) { bad = true; bad_q = q; }
        }
    }
    if (bad)
        return fail(WAVE_ERANGE,
                    "multiplier at point %lld is not a positive normal number of the storage "
                    "format (rescale units or change dt)", (long long)bad_q);
    return WAVE_OK;
}

// Round a binary64 value once to the storage format and return it as binary64.
static double round_store(int prec, double v) {
    if (prec == PREC_FP32) return (double)(float)v;
    uint16_t t;
    store_value(prec, v, &t, 0);
    return load_value(prec, &t, 0);
}

// Elastic multipliers (Eq. 2 scaled as in Section 5 "Range"), binary64 in this
// order, each rounded once: Z0 = max(rho) max(vp); bx = ((dt Z0)/h)/rho_x,
// by likewise, rho_x = (rho[i] + rho[i+1]) * 0.5; mu = (rho vs) vs,
// lambda = ((rho vp) vp) - 2 mu; l2m = ((dt (lambda + 2 mu))/Z0)/h,
// lam = ((dt lambda)/Z0)/h; mu_xy = 4 / (sum of 1/mu over the four nodes
// around the shear point, 0 if any is 0), mu = ((dt mu_xy)/Z0)/h. The
// neighbour i+1 (j+1) wraps on periodic axes and is clamped otherwise.
// On the row of a free surface (y-lo FREE, j = 0) syy is zero, so sxx obeys
// d(sxx)/dt = M d(vx)/dx with M = ((4 mu)(lambda + mu))/(lambda + 2 mu), the
// modulus under zero normal traction: l2m = ((dt M)/Z0)/h and lam = 0 there
// (the stress kernels then leave syy at zero on that row, since D_y v_y
// vanishes on it by the even image of v_y).
static wave_status elastic_coefficients(wave_ctx *c, const wave_materials *mat) {
    const int64_t nx = c->n[0], ny = c->n[1], npts = nx * ny;
    double rho0 = 0.0, c0 = 0.0;
    for (int64_t q = 0; q < npts; q++) {
        if (!(mat->rho[q] > 0.0) || !isfinite(mat->rho[q]) || !(mat->vp[q] > 0.0) ||
            !isfinite(mat->vp[q]) || !(mat->vs[q] >= 0.0) || !isfinite(mat->vs[q]))
            return fail(WAVE_ERANGE, "material value at point %lld is out of range", (long long)q);
        if (mat->rho[q] > rho0) rho0 = mat->rho[q];
        if (mat->vp[q] > c0) c0 = mat->vp[q];
    }
    const double Z0 = rho0 * c0, h = c->h, dt = c->dt;
    c->Z0 = Z0;
    const int cp = coef_prec(c->prec);  // binary32 for the pair precision
    const double tiny = min_normal(cp);
    for (int w = 0; w < 5; w++) c->coef_host[w].assign(npts, 0.0);
    auto lame = [&](int64_t q, double &m, double &l) {
        m = (mat->rho[q] * mat->vs[q]) * mat->vs[q];
        l = ((mat->rho[q] * mat->vp[q]) * mat->vp[q]) - (2.0 * m);
    };
    for (int64_t j = 0; j < ny; j++)
        for (int64_t i = 0; i < nx; i++) {
            const int64_t q = i + nx * j;
            const int64_t i1 = i + 1 < nx ? i + 1 : (c->bc[1] == WAVE_BC_PERIODIC ? 0 : i);
            const int64_t j1 = j + 1 < ny ? j + 1 : (c->bc[3] == WAVE_BC_PERIODIC ? 0 : j);
            const double rx = (mat->rho[q] + mat->rho[i1 + nx * j]) * 0.5;
            const double ry = (mat->rho[q] + mat->rho[i + nx * j1]) * 0.5;
            const double bx = round_store(cp, ((dt * Z0) / h) / rx);
            const double by = round_store(cp, ((dt * Z0) / h) / ry);
            double m00, l00, m10, l10, m01, l01, m11, l11;
            lame(q, m00, l00);
            lame(i1 + nx * j, m10, l10);
            lame(i + nx * j1, m01, l01);
            lame(i1 + nx * j1, m11, l11);
            const bool surface = c->bc[2] == WAVE_BC_FREE && j == 0;
            const double msurf = ((4.0 * m00) * (l00 + m00)) / (l00 + 2.0 * m00);
            const double l2m = round_store(cp, ((dt * (surface ? msurf : l00 + 2.0 * m00)) / Z0) / h);
            const double lam = surface ? 0.0 : round_store(cp, ((dt * l00) / Z0) / h);
            double mh = 0.0;
            if (m00 > 0.0 && m10 > 0.0 && m01 > 0.0 && m11 > 0.0)
                mh = 4.0 / (1.0 / m00 + 1.0 / m10 + 1.0 / m01 + 1.0 / m11);
            const double mu = round_store(cp, ((dt * mh) / Z0) / h);
            c->coef_host[0][q] = bx;
            c->coef_host[1][q] = by;
            c->coef_host[2][q] = l2m;
            c->coef_host[3][q] = lam;
            c->coef_host[4][q] = mu;
            const bool ok = bx >= tiny && isfinite(bx) && by >= tiny && isfinite(by) &&
                            l2m >= tiny && isfinite(l2m) &&
                            (lam == 0.0 || fabs(lam) >= tiny) && isfinite(lam) &&
                            (mu == 0.0 || mu >= tiny) && isfinite(mu) && l2m > fabs(lam);
            if (!ok)
                return fail(WAVE_ERANGE,
                            "elastic multiplier at point %lld outside the storage format's range "
                            "(rescale units or change dt%s)", (long long)q,
                            surface ? "; a free surface needs vs > 0 on its row" : "");
        }
    return WAVE_OK;
}

// Upload coefficient w (0 b, 1..3 a_x..a_z) as a uniform value or an array.
static wave_status upload_coef(wave_ctx *c, int w) {
    const std::vector<double> &v = c->coef_host[w];
    const int64_t npts = (int64_t)v.size();
    bool uni = true;
    for (int64_t q = 1; q < npts && uni; q++) uni = (v[q] == v[0]);
    c->coef_is_uniform[w] = uni;
    const int cp = coef_prec(c->prec);
    if (uni) {
        if (cp == PREC_FP32) {
            float f = (float)v[0];
            memcpy(&c->coef_uni[w], &f, 4);
        } else {
            uint16_t hb;
            store_value(cp, v[0], &hb, 0);
            c->coef_uni[w] = hb;
        }
        return WAVE_OK;
    }
    const size_t eb = elem_bytes(cp);
    wave_status st = dev_alloc(c, c->coef[w], c->total * eb);
    if (st) return st;
    std::vector<unsigned char> tmp(npts * eb);
    for (int64_t q = 0; q < npts; q++) store_value(cp, v[q], tmp.data(), q);
    return upload_packed(c, c->coef[w].ptr, tmp.data(), eb);
}

static void fill_acoustic_params(wave_ctx *c, AcParams &prm) {
    memset(&prm, 0, sizeof prm);
    for (int ax = 0; ax < 3; ax++) {
        prm.n[ax] = (int)c->n[ax];
        prm.bc[ax] = ax < c->ndim ? (c->bc[2 * ax] == WAVE_BC_PERIODIC ? BC_PERIODIC : BC_RIGID)
                                  : BC_PERIODIC;
    }
    prm.sy = c->pitch;
    prm.sz = c->plane;
    prm.p = c->f[0].ptr;
    prm.tp = c->t[0].ptr;
    for (int ax = 0; ax < 3; ax++) {
        prm.v[ax] = c->f[1 + ax].ptr;
        prm.tv[ax] = c->t[1 + ax].ptr;
        prm.a[ax] = c->coef_is_uniform[1 + ax] ? nullptr : c->coef[1 + ax].ptr;
        prm.a_uni[ax] = c->coef_uni[1 + ax];
    }
    prm.b = c->coef_is_uniform[0] ? nullptr : c->coef[0].ptr;
    prm.b_uni = c->coef_uni[0];
    prm.src_q = c->src_field == WAVE_F_P ? c->src_q : -1;
    prm.src_i = prm.src_j = prm.src_k = -1;
    if (prm.src_q >= 0) {
        prm.src_k = (int)(c->src_q / c->plane);
        prm.src_j = (int)((c->src_q % c->plane) / c->pitch);
        prm.src_i = (int)(c->src_q % c->pitch);
    }
    prm.src = c->src_table.ptr;
    prm.src_nt = c->src_nt;
    prm.e_part = static_cast<double *>(c->e_part.ptr);
    prm.e_count = reinterpret_cast<unsigned *>(static_cast<char *>(c->e_misc.ptr) + 8);
    prm.e_out = static_cast<double *>(c->e_misc.ptr);
    const double hd1 = c->ndim == 2 ? c->h : c->h * c->h;
    prm.e_factor = 0.5 * hd1 * c->P0 * c->P0 * c->dt / c->Z0;
}

static cudaEvent_t take_event(wave_ctx *c) {
    if (!c->event_pool.empty()) {
        cudaEvent_t e = c->event_pool.back();
        c->event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// Record an event on the context stream when timing is on; returns it (or null).
static cudaEvent_t mark(wave_ctx *c) {
    if (!c->timing) return nullptr;
    cudaEvent_t e = take_event(c);
    cudaEventRecord(e, c->stream);
    return e;
}

static void timed(wave_ctx *c, int kind, cudaEvent_t a, cudaEvent_t b) {
    if (a && b) c->pending.push_back({kind, a, b});
}

// Sum the elapsed times of finished launch pairs (stream must be synchronised).
static void collect_timing(wave_ctx *c) {
    std::vector<cudaEvent_t> seen;
    for (auto &t : c->pending) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, t.a, t.b);
        c->t_launches[t.kind]++;
        c->t_ms[t.kind] += ms;
        seen.push_back(t.a);
        seen.push_back(t.b);
    }
    c->pending.clear();
    std::sort(seen.begin(), seen.end());
    seen.erase(std::unique(seen.begin(), seen.end()), seen.end());
    for (auto e : seen) c->event_pool.push_back(e);
}

static void adjoint_free(wave_ctx *c) {
    auto &A = c->adj;
    dev_free(c, A.cps);
    dev_free(c, A.seg);
    dev_free(c, A.mu);
    dev_free(c, A.mu_alt);
    dev_free(c, A.g);
    dev_free(c, A.rec_w);
    dev_free(c, A.rec_order);
    dev_free(c, A.rec_start);
    for (int ax = 0; ax < 3; ax++) {
        dev_free(c, A.nu[ax]);
        dev_free(c, A.nu_alt[ax]);
    }
    A = wave_ctx::Adjoint();
}

static void destroy_ctx(wave_ctx *c) {
    if (!c) return;
    for (auto g : c->strip_graph)
        if (g) cudaGraphExecDestroy(g);
    dev_free(c, c->strip_shot);
    dev_free(c, c->strip_item0);
    dev_free(c, c->strip_part);
    for (auto &b : c->f) dev_free(c, b);
    for (auto &b : c->t) dev_free(c, b);
    for (auto &b : c->coef) dev_free(c, b);
    for (auto &b : c->alt_f) dev_free(c, b);
    for (auto &b : c->alt_t) dev_free(c, b);
    dev_free(c, c->e_part);
    dev_free(c, c->e_misc);
    dev_free(c, c->src_table);
    dev_free(c, c->rec_q);
    adjoint_free(c);
    for (auto &b : c->adj_na) dev_free(c, b);
    dev_free(c, c->adj_nb);
    dev_free(c, c->adj_two_over_c);
    cudaStreamSynchronize(c->stream);
    collect_timing(c);
    for (auto e : c->event_pool) cudaEventDestroy(e);
    delete c;
}

extern "C" void wave_destroy(wave_ctx *c) { destroy_ctx(c); }

extern "C" wave_status wave_create(const wave_grid *grid, const double spacing[3],
                                   const wave_materials *mat, double dt, wave_precision prec,
                                   wave_comp compensated, const wave_options *opt,
                                   void *cuda_stream, wave_ctx **out) {
    if (!grid || !spacing || !mat || !out) return fail(WAVE_EINVAL, "wave_create: NULL argument");
    *out = nullptr;
    if (grid->ndim != 2 && grid->ndim != 3) return fail(WAVE_EINVAL, "ndim must be 2 or 3");
    if (mat->kind != WAVE_ACOUSTIC && mat->kind != WAVE_ELASTIC)
        return fail(WAVE_EINVAL, "unknown physics %d", (int)mat->kind);
    if (mat->kind == WAVE_ELASTIC && grid->ndim != 2)
        return fail(WAVE_ENOTIMPL, "the elastic system is 2D (Eq. 2)");
    for (int ax = 0; ax < grid->ndim; ax++) {
        if (grid->n[ax] < 8) return fail(WAVE_EINVAL, "n[%d] = %lld < 8", ax, (long long)grid->n[ax]);
        if (grid->n[ax] > (1 << 20)) return fail(WAVE_EINVAL, "n[%d] too large", ax);
        if (!(spacing[ax] > 0.0) || !isfinite(spacing[ax]))
            return fail(WAVE_EINVAL, "spacing[%d] must be positive", ax);
        if (spacing[ax] != spacing[0]) return fail(WAVE_EINVAL, "spacing must be isotropic");
    }
    if (!(dt > 0.0) || !isfinite(dt)) return fail(WAVE_EINVAL, "dt must be positive and finite");
    if (prec == WAVE_FP64) return fail(WAVE_ENOTIMPL, "WAVE_FP64 runs only in the CPU oracle");
    if (prec < WAVE_FP32 || prec > WAVE_FP16_PAIRS) return fail(WAVE_EINVAL, "bad precision");
    if (compensated != WAVE_COMP_NONE && compensated != WAVE_COMP_3OP &&
        compensated != WAVE_COMP_6OP)
        return fail(WAVE_EINVAL, "bad compensation %d", (int)compensated);
    if (prec == WAVE_FP16_PAIRS) {
        // the stencils read V + T: nothing to read without the compensation
        if (compensated == WAVE_COMP_NONE) return fail(WAVE_EINVAL, "WAVE_FP16_PAIRS needs a compensation");
    }
    if (!mat->rho || !mat->vp) return fail(WAVE_EINVAL, "material arrays are NULL");
    if (mat->kind == WAVE_ELASTIC && !mat->vs) return fail(WAVE_EINVAL, "elastic needs vs");
    double P0 = 1.0, z0_opt = 0.0;
    int kchoice = 0, zchunk = 0, z_cut = 0;
    const double *rho_above = nullptr;
    if (opt) {
        if (opt->field_scale != 0.0) P0 = opt->field_scale;
        kchoice = opt->kernel;
        zchunk = opt->zchunk;
        z_cut = opt->z_cut;
        z0_opt = opt->z0;
        rho_above = opt->rho_above;
    }
    if (kchoice < 0 || kchoice > 4 || zchunk < 0) return fail(WAVE_EINVAL, "bad kernel options");
    if (kchoice == 4 && (mat->kind != WAVE_ACOUSTIC || grid->ndim != 2))
        return fail(WAVE_EINVAL, "kernel 4 (cluster-resident steps) takes 2D acoustic grids");
    if (z_cut < 0 || z_cut > 3) return fail(WAVE_EINVAL, "z_cut takes bits 0 and 1 only");
    if (z_cut && (mat->kind != WAVE_ACOUSTIC || grid->ndim != 3))
        return fail(WAVE_EINVAL, "z slabs are 3D acoustic contexts");
    if (z_cut && (kchoice == 1 || kchoice == 3))
        return fail(WAVE_EINVAL, "z slabs step with the two-kernel streaming path (kernel 0 or 2)");
    if ((z_cut & 2) && !rho_above) return fail(WAVE_EINVAL, "a cut z-hi face needs rho_above");
    if (prec == WAVE_FP16_PAIRS && z_cut) return fail(WAVE_ENOTIMPL, "WAVE_FP16_PAIRS covers whole grids");
    if (prec == WAVE_FP16_PAIRS && grid->ndim == 2 && kchoice == 3)
        return fail(WAVE_ENOTIMPL, "WAVE_FP16_PAIRS steps 2D grids with the two-launch strips");
    if (!(z0_opt >= 0.0) || !isfinite(z0_opt)) return fail(WAVE_EINVAL, "z0 must be >= 0 and finite");
    if (!(P0 > 0.0) || !isfinite(P0)) return fail(WAVE_EINVAL, "field_scale must be positive");
    const int64_t npts = grid->n[0] * grid->n[1] * (grid->ndim == 3 ? grid->n[2] : 1);
    if (npts > ((int64_t)1 << 31) - 1) return fail(WAVE_EINVAL, "grid too large (>= 2^31 points)");

    wave_ctx *c = new (std::nothrow) wave_ctx();
    if (!c) return fail(WAVE_ENOMEM, "host allocation failed");
    c->kind = mat->kind;
    c->ndim = grid->ndim;
    for (int ax = 0; ax < 3; ax++) c->n[ax] = ax < grid->ndim ? grid->n[ax] : 1;
    for (int fc = 0; fc < 6; fc++) c->bc[fc] = mat->bc[fc];
    c->prec = prec;
    c->comp = compensated;
    c->kernel_choice = kchoice;
    c->z_cut = z_cut;
    if (zchunk > 0) { c->zchunk = zchunk; c->zchunk_set = true; }
    c->h = spacing[0];
    c->dt = dt;
    c->P0 = P0;
    c->stream = static_cast<cudaStream_t>(cuda_stream);
    // pitch: x extent rounded up to 16 elements (>= 32 bytes, 16-byte aligned rows)
    c->pitch = (c->n[0] + 15) / 16 * 16;
    c->plane = c->pitch * c->n[1];
    c->total = c->plane * c->n[2];

    wave_status st;
    if (c->kind == WAVE_ACOUSTIC) {
        for (int ax = 0; ax < 3; ax++) {
            if (ax >= c->ndim) continue;
            int lo = c->bc[2 * ax], hi = c->bc[2 * ax + 1];
            if (lo != hi || (lo != WAVE_BC_PERIODIC && lo != WAVE_BC_RIGID)) {
                delete c;
                return fail(WAVE_EINVAL, "acoustic axis %d: faces must both be PERIODIC or RIGID",
                            ax);
            }
        }
        st = acoustic_coefficients(c, mat, z0_opt, (z_cut & 2) ? rho_above : nullptr);
        if (st) { delete c; return st; }
        const size_t eb = elem_bytes(prec);
        int nf = 1 + c->ndim;
        for (int fi = 0; fi < nf && !st; fi++) {
            st = dev_alloc(c, c->f[fi], c->total * eb);
            if (!st && compensated) st = dev_alloc(c, c->t[fi], c->total * eb);
        }
        for (int w = 0; w < 1 + c->ndim && !st; w++) st = upload_coef(c, w);
        AcParams prm;
        fill_acoustic_params(c, prm);
        c->e_blocks = acoustic_generic_blocks(prm, c->ndim);
        // (3D grids of WAVE_FP16_PAIRS take the same kernels as the stored-value
        // precisions: the one-pass step, else the streaming kernels, else one
        // thread per point)
        const bool pairs = prec == WAVE_FP16_PAIRS;
        c->use_fused = !z_cut && (kchoice == 0 || kchoice == 3) &&
                       acoustic_fused_supported(prm, c->ndim, c->prec);
        c->use_stream = !c->use_fused && kchoice != 1 &&
                        acoustic_stream_supported(prm, c->ndim, c->prec);
        if (z_cut && !c->use_stream && !st)
            st = fail(WAVE_EINVAL, "z slabs need n[0] a multiple of the 16-byte vector width");
        if (c->use_fused && !c->zchunk_set) {
            int dev = 0, sms = 1;
            cudaGetDevice(&dev);
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            c->zchunk = fused_zchunk_for(prm, c->prec, sms);
        }
        if (c->ndim == 2 && kchoice != 1) {
            // row strips of 16 rows, 4 warps per block, at most 16 blocks per SM
            c->use_strips = true;
            int dev = 0, sms = 1;
            cudaGetDevice(&dev);
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            const int64_t tx = 32 * (c->prec == PREC_FP32 ? 4 : 8);
            c->strip_rows = c->zchunk_set ? c->zchunk : strip_rows_for((c->n[0] + tx - 1) / tx, c->n[1], sms);
            c->strip_items = (int)batch_items_of(BATCH_STRIPS, 0, 0, c->strip_rows, c->prec, c->n[0], c->n[1]);
            c->strip_grid = std::max(1, std::min((c->strip_items + kStripWarps - 1) / kStripWarps, 16 * sms));
            const int item0[2] = {0, c->strip_items};
            // kernel 3: the one-pass strips, which read the state from one
            // buffer set and write the other (the two-launch strips are the
            // default: faster on this hardware, see the notes on the kernels)
            c->strip_fused = kchoice == 3;
            // kernel 4: the cluster-resident steps (the state in the shared
            // memory of one cluster); kernel 0 (the default) takes them while
            // a band holds at most 5120 points: a warp walks a row in about
            // 2500 cycles, so a step costs about 3 us plus 0.85 us per 1000
            // points of a band, against about 6.3 us for the two strip
            // launches (256^2: 4.9 against 6.2 us; 384^2: 9.2 against 6.2).
            // The strips stay set up: batches step the context with them.
            if ((kchoice == 0 || kchoice == 4) && !st) {
                c->use_cluster = acoustic_cluster_plan(prm, c->prec, compensated, c->cplan) &&
                                 (kchoice == 4 || (int64_t)c->cplan.rows * c->n[0] <= 5120);
                cudaGetLastError();
                if (kchoice == 4 && !c->use_cluster)
                    st = fail(WAVE_EINVAL, "kernel 4: the grid's state does not fit one cluster's shared memory");
            }
            for (int fi = 0; fi < 3 && c->strip_fused && !st; fi++) {
                st = dev_alloc(c, c->alt_f[fi], c->total * eb);
                if (!st && fi > 0 && compensated) st = dev_alloc(c, c->alt_t[fi], c->total * eb);
            }
            if (!st) st = dev_alloc(c, c->strip_shot, sizeof(BatchShot));
            if (!st) st = dev_alloc(c, c->strip_item0, sizeof(item0));
            if (!st) st = dev_alloc(c, c->strip_part, sizeof(double) * (size_t)c->strip_items);
            if (!st) {
                cudaError_t e = cudaMemcpyAsync(c->strip_item0.ptr, item0, sizeof(item0), cudaMemcpyHostToDevice,
                                                c->stream);
                if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
                if (e != cudaSuccess) st = fail(WAVE_ECUDA, "wave_create: %s", cudaGetErrorString(e));
            }
        }
        if (c->use_stream)
            c->e_blocks = std::max(c->e_blocks, acoustic_stream_blocks(prm, c->prec, c->zchunk));
        if (c->use_fused) {
            c->e_blocks = std::max(c->e_blocks, acoustic_fused_blocks(prm, c->prec, c->zchunk));
            // (the pair precision alternates t_p between the sets too)
            for (int fi = 0; fi < 4 && !st; fi++) {
                st = dev_alloc(c, c->alt_f[fi], c->total * eb);
                if (!st && (fi > 0 || pairs) && compensated) st = dev_alloc(c, c->alt_t[fi], c->total * eb);
            }
            if (!st && fused_maps_bytes() > sizeof(c->fmaps[0].b))
                st = fail(WAVE_ECUDA, "tensor map block too large");
            for (int set = 0; set < 2 && !st; set++) {
                DevBuf *F = set == 0 ? c->f : c->alt_f;
                DevBuf *T = set == 0 ? c->t : c->alt_t;
                const void *in[7] = {F[0].ptr, F[1].ptr, F[2].ptr, F[3].ptr, T[1].ptr, T[2].ptr, T[3].ptr};
                if (!acoustic_fused_encode(c->fmaps[set].b, prm, in, pairs ? T[0].ptr : c->t[0].ptr, c->prec,
                                           compensated))
                    st = fail(WAVE_ECUDA, "cuTensorMapEncodeTiled failed for the one-pass step");
            }
        }
    } else {
        const int *b = c->bc;
        const bool x_ok = (b[0] == WAVE_BC_PERIODIC && b[1] == WAVE_BC_PERIODIC) ||
                          (b[0] == WAVE_BC_RIGID && b[1] == WAVE_BC_RIGID);
        const bool y_ok = (b[2] == WAVE_BC_PERIODIC && b[3] == WAVE_BC_PERIODIC) ||
                          ((b[2] == WAVE_BC_RIGID || b[2] == WAVE_BC_FREE) && b[3] == WAVE_BC_RIGID);
        if (!x_ok || !y_ok) {
            delete c;
            return fail(WAVE_EINVAL, "elastic faces: x PERIODIC/PERIODIC or RIGID/RIGID; "
                                     "y PERIODIC/PERIODIC or (RIGID|FREE)/RIGID");
        }
        st = elastic_coefficients(c, mat);
        if (st) { delete c; return st; }
        const size_t eb = elem_bytes(prec);
        const int fields[5] = {WAVE_F_VX, WAVE_F_VY, WAVE_F_SXX, WAVE_F_SYY, WAVE_F_SXY};
        for (int fi = 0; fi < 5 && !st; fi++) {
            st = dev_alloc(c, c->f[fields[fi]], c->total * eb);
            if (!st && compensated) st = dev_alloc(c, c->t[fields[fi]], c->total * eb);
        }
        for (int w = 0; w < 5 && !st; w++) st = upload_coef(c, w);
        const int nn[2] = {(int)c->n[0], (int)c->n[1]};
        c->e_blocks = elastic_blocks(nn);
        if (kchoice != 1 && !st) {
            c->use_strips = true;
            int dev = 0, sms = 1;
            cudaGetDevice(&dev);
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            const int tx = 32 * (c->prec == PREC_FP32 ? 4 : 8);
            c->strip_rows = c->zchunk_set ? c->zchunk : strip_rows_for((nn[0] + tx - 1) / tx, nn[1], sms);
            c->strip_items = elastic_strip_items(c->prec, nn[0], nn[1], c->strip_rows);
            c->strip_grid = std::max(1, std::min((c->strip_items + kStripWarps - 1) / kStripWarps, 16 * sms));
            st = dev_alloc(c, c->strip_part, sizeof(double) * (size_t)c->strip_items);
        }
    }
    if (!st) st = dev_alloc(c, c->e_part, sizeof(double) * (size_t)std::max(1u, c->e_blocks));
    if (!st) st = dev_alloc(c, c->e_misc, 32);  // [energy][block counter][error word][step index]
    if (!st) {
        cudaError_t e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) st = fail(WAVE_ECUDA, "wave_create: %s", cudaGetErrorString(e));
    }
    if (st) {
        destroy_ctx(c);
        return st;
    }
    *out = c;
    return WAVE_OK;
}

// --------------------------------------------------------------- field I/O
static bool on_rigid_wall_zeroed(const wave_ctx *c, int field, const int64_t idx[3]) {
    // acoustic: p is zero on every rigid wall node plane; v_c on the wall
    // planes of the rigid axes other than c
    for (int ax = 0; ax < c->ndim; ax++) {
        if (c->bc[2 * ax] != WAVE_BC_RIGID || idx[ax] != 0) continue;
        if (ax == 2 && (c->z_cut & 1)) continue;  // a cut, not the grid's wall
        if (field == WAVE_F_P) return true;
        if (field - 1 != ax) return true;
    }
    return false;
}

extern "C" wave_status wave_set_initial(wave_ctx *c, wave_field field, const double *host) {
    CHECK_CTX(c);
    if (!host) return fail(WAVE_EINVAL, "wave_set_initial: NULL values");
    if (!field_valid(c, field)) return fail(WAVE_EINVAL, "field %d not in this physics", field);
    const int64_t npts = c->n[0] * c->n[1] * c->n[2];
    const size_t eb = elem_bytes(c->prec);
    std::vector<unsigned char> tmp;
    try { tmp.resize(npts * eb); } catch (...) { return fail(WAVE_ENOMEM, "host buffer"); }
    const bool is_vel = (field == WAVE_F_VX || field == WAVE_F_VY || field == WAVE_F_VZ);
    const double P0 = c->P0, Z0 = c->Z0;
    const int prec = c->prec;
    const int64_t nx = c->n[0], ny = c->n[1];
    std::vector<int64_t> badv(1, -1);
    int64_t *bad = badv.data();
    unsigned char *dst = tmp.data();
    const wave_ctx *cc = c;
    parallel_for(npts, [=](int64_t lo, int64_t hi) {
        for (int64_t q = lo; q < hi; q++) {
            double x = host[q];
            double s = is_vel ? (x * Z0) / P0 : x / P0;
            if (!isfinite(x)) { *bad = q; s = 0.0; }
            if (cc->kind == WAVE_ACOUSTIC) {
                const int64_t idx[3] = {q % nx, (q / nx) % ny, q / (nx * ny)};
                if (on_rigid_wall_zeroed(cc, field, idx)) s = 0.0;
            } else {
                // frictionless rigid walls hold the normal velocity and the
                // shear stress at zero on the stored wall points; a free
                // surface holds syy at zero on its row
                const int64_t i = q % nx, j = q / nx;
                if (cc->bc[1] == WAVE_BC_RIGID && i == nx - 1 &&
                    (field == WAVE_F_VX || field == WAVE_F_SXY)) s = 0.0;
                if (cc->bc[3] == WAVE_BC_RIGID && j == ny - 1 &&
                    (field == WAVE_F_VY || field == WAVE_F_SXY)) s = 0.0;
                if (cc->bc[2] == WAVE_BC_FREE && j == 0 && field == WAVE_F_SYY) s = 0.0;
            }
            store_value(prec, s, dst, q);
            if (!isfinite(load_value(prec, dst, q))) *bad = q;
        }
    });
    if (*bad >= 0)
        return fail(WAVE_ERANGE, "initial value at point %lld is not finite in the storage format",
                    (long long)*bad);
    wave_status st = upload_packed(c, c->f[field].ptr, tmp.data());
    if (st) return st;
    if (c->t[field].ptr) {
        cudaError_t e = cudaMemsetAsync(c->t[field].ptr, 0, c->t[field].bytes, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        return cuda_check(c, e, "reset compensation");
    }
    return WAVE_OK;
}

extern "C" wave_status wave_get_raw(wave_ctx *c, wave_field field, int32_t compensation,
                                    void *host) {
    CHECK_CTX(c);
    if (!host) return fail(WAVE_EINVAL, "wave_get_raw: NULL output");
    if (!field_valid(c, field)) return fail(WAVE_EINVAL, "field %d not in this physics", field);
    const int64_t npts = c->n[0] * c->n[1] * c->n[2];
    if (compensation && !c->t[field].ptr) {
        memset(host, 0, npts * elem_bytes(c->prec));
        return WAVE_OK;
    }
    return download_packed(c, compensation ? c->t[field].ptr : c->f[field].ptr, host);
}

extern "C" wave_status wave_set_raw(wave_ctx *c, wave_field field, int32_t compensation,
                                    const void *host) {
    CHECK_CTX(c);
    if (!host) return fail(WAVE_EINVAL, "wave_set_raw: NULL input");
    if (!field_valid(c, field)) return fail(WAVE_EINVAL, "field %d not in this physics", field);
    if (compensation && !c->t[field].ptr)
        return fail(WAVE_EINVAL, "context has no compensation arrays");
    return upload_packed(c, compensation ? c->t[field].ptr : c->f[field].ptr, host);
}

extern "C" wave_status wave_get_field(wave_ctx *c, wave_field field, double *host) {
    CHECK_CTX(c);
    if (!host) return fail(WAVE_EINVAL, "wave_get_field: NULL output");
    if (!field_valid(c, field)) return fail(WAVE_EINVAL, "field %d not in this physics", field);
    const int64_t npts = c->n[0] * c->n[1] * c->n[2];
    std::vector<unsigned char> tmp(npts * elem_bytes(c->prec));
    wave_status st = download_packed(c, c->f[field].ptr, tmp.data());
    if (st) return st;
    const bool is_vel = (field == WAVE_F_VX || field == WAVE_F_VY || field == WAVE_F_VZ);
    const double P0 = c->P0, Z0 = c->Z0;
    const int prec = c->prec;
    const unsigned char *src = tmp.data();
    parallel_for(npts, [=](int64_t lo, int64_t hi) {
        for (int64_t q = lo; q < hi; q++) {
            double s = load_value(prec, src, q);
            host[q] = is_vel ? (s * P0) / Z0 : s * P0;
        }
    });
    return WAVE_OK;
}

extern "C" wave_status wave_get_coefficient(wave_ctx *c, int32_t which, double *host, double *Z0) {
    CHECK_CTX(c);
    if (Z0) *Z0 = c->Z0;
    if (!host) return WAVE_OK;
    const std::vector<double> *v = nullptr;
    if (c->kind == WAVE_ACOUSTIC) {
        if (which < 0 || which > c->ndim) return fail(WAVE_EINVAL, "bad coefficient index");
        v = &c->coef_host[which];
    } else {
        if (which < 0 || which > 4) return fail(WAVE_EINVAL, "bad coefficient index");
        v = &c->coef_host[which];
    }
    memcpy(host, v->data(), v->size() * sizeof(double));
    return WAVE_OK;
}

// ----------------------------------------------------------------- source
extern "C" wave_status wave_set_source(wave_ctx *c, wave_field field, const int64_t idx[3],
                                       const double *wavelet, int64_t nt) {
    CHECK_CTX(c);
    if (nt < 0 || (nt > 0 && (!wavelet || !idx))) return fail(WAVE_EINVAL, "bad source arguments");
    if (c->kind == WAVE_ACOUSTIC && field != WAVE_F_P)
        return fail(WAVE_EINVAL, "acoustic sources act on p");
    if (c->kind == WAVE_ELASTIC && field != WAVE_F_VY)
        return fail(WAVE_EINVAL, "elastic sources act on v_y");
    dev_free(c, c->src_table);
    c->src_q = -1;
    c->src_nt = 0;
    c->src_field = -1;
    if (nt == 0) return WAVE_OK;
    for (int ax = 0; ax < c->ndim; ax++)
        if (idx[ax] < 0 || idx[ax] >= c->n[ax]) return fail(WAVE_EINVAL, "source outside grid");
    const double hd1 = c->ndim == 2 ? c->h : c->h * c->h;
    // acoustic: added to R before the multiplier; elastic v_y force: added to
    // the increment after the multiplier, s^ = w * ((dt * Z0) / (P0 * (h * h)))
    const double scale = c->kind == WAVE_ACOUSTIC ? c->Z0 / (c->P0 * hd1)
                                                  : (c->dt * c->Z0) / (c->P0 * (c->h * c->h));
    const bool f32 = arith_is_f32(c->prec);
    std::vector<unsigned char> tab(nt * (f32 ? 4 : 2));
    std::vector<float> host(nt);
    for (int64_t s = 0; s < nt; s++) {
        if (!isfinite(wavelet[s])) return fail(WAVE_ERANGE, "wavelet sample %lld", (long long)s);
        double v = wavelet[s] * scale;
        if (f32) {
            float x = (float)v;
            memcpy(&tab[4 * s], &x, 4);
            host[s] = x;
        } else {
            uint16_t hb = is_bf16_storage(c->prec) ? round_bits16(v, 7, 8) : round_bits16(v, 10, 5);
            memcpy(&tab[2 * s], &hb, 2);
            host[s] = (float)(is_bf16_storage(c->prec) ? bf16_to_double(hb) : half_to_double(hb));
        }
    }
    wave_status st = dev_alloc(c, c->src_table, tab.size());
    if (st) return st;
    cudaError_t e = cudaMemcpyAsync(c->src_table.ptr, tab.data(), tab.size(),
                                    cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_check(c, e, "source upload");
    c->src_q = idx[0] + c->pitch * idx[1] + (c->ndim == 3 ? c->plane * idx[2] : 0);
    c->src_nt = nt;
    c->src_field = field;
    c->src_host.swap(host);
    return WAVE_OK;
}

// -------------------------------------------------------------- receivers
extern "C" wave_status wave_set_receivers(wave_ctx *c, wave_field field, const int64_t *idx,
                                          int64_t nrec, float *traces, int64_t cap) {
    CHECK_CTX(c);
    dev_free(c, c->rec_q);
    c->nrec = 0;
    c->rec_traces = nullptr;
    if (nrec == 0) return WAVE_OK;
    if (nrec < 0 || nrec > 65536 || !idx || !traces || cap < 0)
        return fail(WAVE_EINVAL, "bad receiver arguments");
    if (!field_valid(c, field)) return fail(WAVE_EINVAL, "field %d not in this physics", field);
    std::vector<int64_t> q(nrec);
    for (int64_t r = 0; r < nrec; r++) {
        for (int ax = 0; ax < c->ndim; ax++)
            if (idx[3 * r + ax] < 0 || idx[3 * r + ax] >= c->n[ax])
                return fail(WAVE_EINVAL, "receiver %lld outside grid", (long long)r);
        q[r] = idx[3 * r] + c->pitch * idx[3 * r + 1] +
               (c->ndim == 3 ? c->plane * idx[3 * r + 2] : 0);
    }
    wave_status st = dev_alloc(c, c->rec_q, nrec * sizeof(int64_t));
    if (st) return st;
    cudaError_t e = cudaMemcpyAsync(c->rec_q.ptr, q.data(), nrec * sizeof(int64_t),
                                    cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_check(c, e, "receiver upload");
    c->nrec = nrec;
    c->rec_field = field;
    c->rec_traces = traces;
    c->rec_cap = cap;
    c->rec_pos = 0;
    return WAVE_OK;
}

namespace wave {
__global__ void receivers_kernel(const void *field, int eb, int is_bf16, const int64_t *q, int nrec,
                                 float *out) {
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nrec) return;
    float v;
    if (eb == 4) v = static_cast<const float *>(field)[q[r]];
    else if (is_bf16) v = BF16::to_f32(static_cast<const uint16_t *>(field)[q[r]]);
    else v = F16::to_f32(static_cast<const uint16_t *>(field)[q[r]]);
    out[r] = v;
}

cudaError_t sample_receivers(const void *field, int eb, int is_bf16, const int64_t *q, int nrec,
                             float *traces, cudaStream_t st) {
    receivers_kernel<<<(nrec + 127) / 128, 128, 0, st>>>(field, eb, is_bf16, q, nrec, traces);
    return cudaGetLastError();
}
}  // namespace wave

// ------------------------------------------------------------------ energy
extern "C" wave_status wave_set_energy_trace(wave_ctx *c, double *dev, int64_t cap) {
    CHECK_CTX(c);
    if (cap < 0 || (cap > 0 && !dev)) return fail(WAVE_EINVAL, "bad energy trace");
    c->e_trace = cap ? dev : nullptr;
    c->e_trace_cap = cap;
    c->e_trace_pos = 0;
    return WAVE_OK;
}

extern "C" wave_status wave_energy(wave_ctx *c, double *E) {
    CHECK_CTX(c);
    if (!E) return fail(WAVE_EINVAL, "wave_energy: NULL output");
    if (!c->have_energy) return fail(WAVE_ESTATE, "no step has run yet");
    double e = 0.0;
    cudaError_t err = cudaMemcpyAsync(&e, c->e_misc.ptr, sizeof(double), cudaMemcpyDeviceToHost,
                                      c->stream);
    if (err == cudaSuccess) err = cudaStreamSynchronize(c->stream);
    if (err != cudaSuccess) return cuda_check(c, err, "wave_energy");
    wave_status st = check_device_error(c);
    if (st) return st;
    *E = e;
    return WAVE_OK;
}

// -------------------------------------------------------------------- step
// energy_last: reduce the discrete energy on the last step (wave_energy reads it)
// Run m plain steps (no energy, receivers or trace; the step index lives in
// device memory) from captured graphs of 2^j steps: m = 32 q + (binary digits
// of the rest), so any run length takes at most q + 5 replays. All sizes are
// captured at the first use (63 steps' worth of launches, once), so that no
// later call pays for a capture. one_step() queues one step on the context's
// stream. Returns the number of steps replayed (fewer than m if a capture
// failed; the caller takes the rest with plain launches).
template <class F>
static int64_t strip_graph_run(wave_ctx *c, int64_t m, F one_step, cudaError_t &err) {
    err = cudaSuccess;
    int64_t done = 0;
    for (int j = kStripGraphLevels - 1; j >= 0; j--) {
        const int64_t len = (int64_t)1 << j;
        if (!c->strip_graph[j]) {
            cudaGraph_t g = nullptr;
            cudaError_t e = cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal);
            if (e == cudaSuccess) {
                for (int64_t t = 0; t < len && e == cudaSuccess; t++) e = one_step();
                cudaError_t e2 = cudaStreamEndCapture(c->stream, &g);
                if (e == cudaSuccess) e = e2;
            }
            if (e == cudaSuccess) e = cudaGraphInstantiate(&c->strip_graph[j], g, 0);
            if (g) cudaGraphDestroy(g);
            if (e != cudaSuccess) {  // no graph: the caller launches the rest
                cudaGetLastError();
                c->strip_graph[j] = nullptr;
                return done;
            }
        }
        if (m - done < len) continue;
        // the largest size as often as it fits; below it, each binary digit of the rest once
        do {
            err = cudaGraphLaunch(c->strip_graph[j], c->stream);
            if (err != cudaSuccess) return done;
            done += len;
        } while (j == kStripGraphLevels - 1 && m - done >= len);
    }
    return done;
}

// The current and the alternate buffer sets of p and the velocities (and their
// compensations, t_p excepted) exchange roles after a step that wrote the new
// state into the alternate set.
static void swap_sets(wave_ctx *c) {
    for (int fi = 0; fi <= c->ndim; fi++) {
        std::swap(c->f[fi], c->alt_f[fi]);
        if (fi > 0) std::swap(c->t[fi], c->alt_t[fi]);
    }
}

// A shot's parameters for the strip kernels: the current set, the alternate
// set, the index of the last step taken, no one-pass steps yet.
static void fill_shot(wave_ctx *c, BatchShot &shot) {
    memset(&shot, 0, sizeof shot);
    fill_acoustic_params(c, shot.prm);
    shot.step = c->step - 1;  // the velocity launch of the step advances it
    shot.alt_p = c->alt_f[0].ptr;
    for (int ax = 0; ax < 2; ax++) {
        shot.alt_v[ax] = c->alt_f[1 + ax].ptr;
        shot.alt_tv[ax] = c->alt_t[1 + ax].ptr;
    }
    shot.fsteps = 0;
    shot.err = reinterpret_cast<int *>(static_cast<char *>(c->e_misc.ptr) + 16);
}

static wave_status acoustic_steps(wave_ctx *c, int64_t n, bool energy_last = true) {
    AcParams prm;
    fill_acoustic_params(c, prm);
    const size_t eb = elem_bytes(c->prec);
    BatchLaunch L;
    if (c->use_cluster) {
        // all n steps in one launch: energies, receivers and the source's
        // step index handled inside it
        ClusterRun run;
        memset(&run, 0, sizeof run);
        run.prm = prm;
        run.prm.step = c->step;
        run.nsteps = n;
        const int64_t tn = c->e_trace ? std::min<int64_t>(n, c->e_trace_cap - c->e_trace_pos) : 0;
        run.e_trace = tn > 0 ? c->e_trace + c->e_trace_pos : nullptr;
        run.e_trace_n = std::max<int64_t>(tn, 0);
        run.e_last = energy_last ? static_cast<double *>(c->e_misc.ptr) : nullptr;
        const int64_t rn = c->nrec ? std::min<int64_t>(n, c->rec_cap - c->rec_pos) : 0;
        run.rec_q = static_cast<const int64_t *>(c->rec_q.ptr);
        run.nrec = (int)c->nrec;
        run.rec_field = c->rec_field;
        run.traces = rn > 0 ? c->rec_traces + c->rec_pos * c->nrec : nullptr;
        run.rec_n = std::max<int64_t>(rn, 0);
        cudaEvent_t m0 = mark(c);
        cudaError_t e = acoustic_cluster_steps(run, c->cplan, c->prec, c->comp, c->stream);
        cudaEvent_t m1 = mark(c);
        timed(c, 3, m0, m1);
        if (e != cudaSuccess) return cuda_check(c, e, "wave_step launch");
        c->e_trace_pos += run.e_trace_n;
        c->rec_pos += run.rec_n;
        c->step += n;
        return WAVE_OK;
    }
    if (c->use_strips) {
        BatchShot shot;
        fill_shot(c, shot);
        cudaError_t e = cudaMemcpyAsync(c->strip_shot.ptr, &shot, sizeof shot, cudaMemcpyHostToDevice, c->stream);
        if (e != cudaSuccess) return cuda_check(c, e, "wave_step upload");
        L.shots = static_cast<BatchShot *>(c->strip_shot.ptr);
        L.item0 = static_cast<const int *>(c->strip_item0.ptr);
        L.item_part = static_cast<double *>(c->strip_part.ptr);
        L.nshots = 1;
        L.nitems = c->strip_items;
        L.kind = c->strip_fused ? BATCH_FUSED : BATCH_STRIPS;
        L.bx = L.by = 0;
        L.yc = c->strip_rows;
        L.wpb = kStripWarps;
        L.grid = c->strip_grid;
        // plain runs (no receivers, no energy trace) on a created stream: the
        // steps before the last are replayed from captured graphs (the
        // source's step index lives in device memory)
        const bool plain = !c->nrec && !c->e_trace && c->stream != nullptr && !c->timing;
        if (plain && n > 1) {
            const int64_t done = strip_graph_run(
                c, n - 1, [&]() { return batch_step(L, c->prec, c->comp, false, c->stream); }, e);
            if (e != cudaSuccess) return cuda_check(c, e, "graph launch");
            n -= done;
            c->step += done;
            if (c->strip_fused && (done & 1)) swap_sets(c);
        }
    }
    for (int64_t s = 0; s < n; s++) {
        prm.step = c->step;
        const bool trace = c->e_trace && c->e_trace_pos < c->e_trace_cap;
        prm.energy = (energy_last && s == n - 1) || trace;
        prm.e_out = static_cast<double *>(c->e_misc.ptr);
        if (c->use_strips) {
            cudaEvent_t m0 = mark(c);
            cudaError_t e = batch_step(L, c->prec, c->comp, prm.energy != 0, c->stream);
            cudaEvent_t m1 = mark(c);
            timed(c, 3, m0, m1);
            if (c->strip_fused) swap_sets(c);
            if (e == cudaSuccess && trace)
                e = cudaMemcpyAsync(c->e_trace + c->e_trace_pos, c->e_misc.ptr, sizeof(double),
                                    cudaMemcpyDeviceToDevice, c->stream);
            if (e == cudaSuccess && c->nrec && c->rec_pos < c->rec_cap)
                e = sample_receivers(c->f[c->rec_field].ptr, (int)eb, is_bf16_storage(c->prec),
                                     static_cast<const int64_t *>(c->rec_q.ptr), (int)c->nrec,
                                     c->rec_traces + c->rec_pos * c->nrec, c->stream);
            if (e != cudaSuccess) return cuda_check(c, e, "wave_step launch");
            if (trace) c->e_trace_pos++;
            if (c->nrec && c->rec_pos < c->rec_cap) c->rec_pos++;
            c->step++;
            continue;
        }
        if (c->use_fused) {
            const void *in[7] = {c->f[0].ptr, c->f[1].ptr, c->f[2].ptr, c->f[3].ptr,
                                 c->t[1].ptr, c->t[2].ptr, c->t[3].ptr};
            void *out[7] = {c->alt_f[0].ptr, c->alt_f[1].ptr, c->alt_f[2].ptr, c->alt_f[3].ptr,
                            c->alt_t[1].ptr, c->alt_t[2].ptr, c->alt_t[3].ptr};
            int *err = reinterpret_cast<int *>(static_cast<char *>(c->e_misc.ptr) + 16);
            cudaEvent_t m0 = mark(c);
            const bool pairs = c->prec == PREC_FP16_PAIRS;
            cudaError_t e = acoustic_fused_step(prm, c->fmaps[c->fset].b, in, out, c->t[0].ptr,
                                                pairs ? c->alt_t[0].ptr : c->t[0].ptr, c->prec, c->comp,
                                                c->zchunk, err, c->stream);
            c->fset ^= 1;
            cudaEvent_t m1 = mark(c);
            timed(c, 3, m0, m1);
            for (int fi = 0; fi < 4; fi++) {
                std::swap(c->f[fi], c->alt_f[fi]);
                if (fi > 0 || pairs) std::swap(c->t[fi], c->alt_t[fi]);
            }
            if (e == cudaSuccess && trace)
                e = cudaMemcpyAsync(c->e_trace + c->e_trace_pos, c->e_misc.ptr, sizeof(double),
                                    cudaMemcpyDeviceToDevice, c->stream);
            if (e == cudaSuccess && c->nrec && c->rec_pos < c->rec_cap)
                e = sample_receivers(c->f[c->rec_field].ptr, (int)eb, is_bf16_storage(c->prec),
                                     static_cast<const int64_t *>(c->rec_q.ptr), (int)c->nrec,
                                     c->rec_traces + c->rec_pos * c->nrec, c->stream);
            if (e != cudaSuccess) return cuda_check(c, e, "wave_step launch");
            if (trace) c->e_trace_pos++;
            if (c->nrec && c->rec_pos < c->rec_cap) c->rec_pos++;
            c->step++;
            continue;
        }
        cudaEvent_t m0 = mark(c);
        cudaError_t e = c->use_stream
                            ? acoustic_stream_half_step(prm, c->prec, c->comp, 0, c->zchunk, c->stream)
                            : acoustic_generic_half_step(prm, c->ndim, c->prec, c->comp, 0, c->stream);
        cudaEvent_t m1 = mark(c);
        timed(c, 0, m0, m1);
        if (e == cudaSuccess)
            e = c->use_stream
                    ? acoustic_stream_half_step(prm, c->prec, c->comp, 1, c->zchunk, c->stream)
                    : acoustic_generic_half_step(prm, c->ndim, c->prec, c->comp, 1, c->stream);
        cudaEvent_t m2 = mark(c);
        timed(c, 1, m1, m2);
        if (e == cudaSuccess && trace)
            e = cudaMemcpyAsync(c->e_trace + c->e_trace_pos, c->e_misc.ptr, sizeof(double),
                                cudaMemcpyDeviceToDevice, c->stream);
        if (e == cudaSuccess && c->nrec && c->rec_pos < c->rec_cap)
            e = sample_receivers(c->f[c->rec_field].ptr, (int)eb, is_bf16_storage(c->prec),
                                 static_cast<const int64_t *>(c->rec_q.ptr), (int)c->nrec,
                                 c->rec_traces + c->rec_pos * c->nrec, c->stream);
        if (e != cudaSuccess) return cuda_check(c, e, "wave_step launch");
        if (trace) c->e_trace_pos++;
        if (c->nrec && c->rec_pos < c->rec_cap) c->rec_pos++;
        c->step++;
    }
    return WAVE_OK;
}

static wave_status elastic_steps(wave_ctx *c, int64_t n) {
    ElParams e;
    memset(&e, 0, sizeof e);
    e.n[0] = (int)c->n[0];
    e.n[1] = (int)c->n[1];
    for (int i = 0; i < 4; i++) e.bc[i] = c->bc[i];
    e.sy = c->pitch;
    const int fields[5] = {WAVE_F_VX, WAVE_F_VY, WAVE_F_SXX, WAVE_F_SYY, WAVE_F_SXY};
    for (int i = 0; i < 5; i++) {
        e.f[i] = c->f[fields[i]].ptr;
        e.t[i] = c->t[fields[i]].ptr;
        e.c[i] = c->coef_is_uniform[i] ? nullptr : c->coef[i].ptr;
        e.c_uni[i] = c->coef_uni[i];
    }
    e.src_q = c->src_field == WAVE_F_VY ? c->src_q : -1;
    e.src = c->src_table.ptr;
    e.src_nt = c->src_nt;
    e.e_part = static_cast<double *>(c->e_part.ptr);
    e.e_count = reinterpret_cast<unsigned *>(static_cast<char *>(c->e_misc.ptr) + 8);
    e.e_out = static_cast<double *>(c->e_misc.ptr);
    e.e_factor = 0.5 * c->h * c->P0 * c->P0 * c->dt / c->Z0;
    const size_t eb = elem_bytes(c->prec);
    ElStripLaunch L;
    L.nitems = c->strip_items;
    L.yc = c->strip_rows;
    L.wpb = kStripWarps;
    L.grid = c->strip_grid;
    L.item_part = static_cast<double *>(c->strip_part.ptr);
    if (c->use_strips) {
        // the step index lives in device memory, so runs of steps can be
        // replayed from a graph (plain runs on a created stream)
        e.step_dev = reinterpret_cast<int64_t *>(static_cast<char *>(c->e_misc.ptr) + 24);
        cudaError_t err = cudaMemcpyAsync(e.step_dev, &c->step, sizeof(int64_t), cudaMemcpyHostToDevice, c->stream);
        if (err == cudaSuccess) err = cudaStreamSynchronize(c->stream);
        if (err != cudaSuccess) return cuda_check(c, err, "wave_step upload");
        const bool plain = !c->nrec && !c->e_trace && c->stream != nullptr && !c->timing;
        if (plain && n > 1) {
            e.energy = 0;
            const int64_t done = strip_graph_run(
                c, n - 1,
                [&]() {
                    cudaError_t r = elastic_strip_half_step(e, c->prec, c->comp, 0, L, c->stream);
                    return r == cudaSuccess ? elastic_strip_half_step(e, c->prec, c->comp, 1, L, c->stream) : r;
                },
                err);
            if (err != cudaSuccess) return cuda_check(c, err, "graph launch");
            n -= done;
            c->step += done;
        }
    }
    for (int64_t s = 0; s < n; s++) {
        e.step = c->step;
        const bool trace = c->e_trace && c->e_trace_pos < c->e_trace_cap;
        e.energy = (s == n - 1) || trace;
        cudaEvent_t m0 = mark(c);
        cudaError_t err = c->use_strips ? elastic_strip_half_step(e, c->prec, c->comp, 0, L, c->stream)
                                        : elastic_half_step(e, c->prec, c->comp, 0, c->stream);
        cudaEvent_t m1 = mark(c);
        timed(c, 0, m0, m1);
        if (err == cudaSuccess)
            err = c->use_strips ? elastic_strip_half_step(e, c->prec, c->comp, 1, L, c->stream)
                                : elastic_half_step(e, c->prec, c->comp, 1, c->stream);
        cudaEvent_t m2 = mark(c);
        timed(c, 1, m1, m2);
        if (err == cudaSuccess && trace)
            err = cudaMemcpyAsync(c->e_trace + c->e_trace_pos, c->e_misc.ptr, sizeof(double),
                                  cudaMemcpyDeviceToDevice, c->stream);
        if (err == cudaSuccess && c->nrec && c->rec_pos < c->rec_cap)
            err = sample_receivers(c->f[c->rec_field].ptr, (int)eb, is_bf16_storage(c->prec),
                                   static_cast<const int64_t *>(c->rec_q.ptr), (int)c->nrec,
                                   c->rec_traces + c->rec_pos * c->nrec, c->stream);
        if (err != cudaSuccess) return cuda_check(c, err, "wave_step launch");
        if (trace) c->e_trace_pos++;
        if (c->nrec && c->rec_pos < c->rec_cap) c->rec_pos++;
        c->step++;
    }
    return WAVE_OK;
}

extern "C" wave_status wave_step(wave_ctx *c, int64_t n) {
    CHECK_CTX(c);
    if (n < 0) return fail(WAVE_EINVAL, "negative step count");
    if (c->z_cut) return fail(WAVE_ESTATE, "a z slab steps by wave_half_step, with exchanges in between");
    if (c->half_open) return fail(WAVE_ESTATE, "a velocity half step awaits its pressure half step");
    if (n == 0) return WAVE_OK;
    wave_status st;
    if (c->kind == WAVE_ACOUSTIC) {
        st = acoustic_steps(c, n);
    } else {
        st = elastic_steps(c, n);
    }
    if (!st) c->have_energy = true;
    return st;
}

// ------------------------------------------------- z slabs and half steps
extern "C" wave_status wave_set_z_ghosts(wave_ctx *c, const void *p_lo, const void *p_hi,
                                         const void *vz_lo, const void *vz_hi) {
    CHECK_CTX(c);
    if (!c->z_cut) return fail(WAVE_EINVAL, "wave_set_z_ghosts: the context is not a z slab");
    const void *g[4] = {p_lo, p_hi, vz_lo, vz_hi};
    for (int i = 0; i < 4; i++) {
        const bool cut = (c->z_cut >> (i & 1)) & 1;
        if (cut != (g[i] != nullptr))
            return fail(WAVE_EINVAL, "wave_set_z_ghosts: give the ghost buffers of exactly the cut faces");
        if (g[i] && (reinterpret_cast<uintptr_t>(g[i]) & 15))
            return fail(WAVE_EINVAL, "wave_set_z_ghosts: ghost buffers must be 16-byte aligned");
    }
    for (int i = 0; i < 4; i++) c->zg[i] = g[i];
    return WAVE_OK;
}

extern "C" wave_status wave_half_step(wave_ctx *c, int32_t which) {
    CHECK_CTX(c);
    if (which != 0 && which != 1) return fail(WAVE_EINVAL, "wave_half_step: which is 0 or 1");
    if (c->kind != WAVE_ACOUSTIC || c->use_fused || c->use_strips)
        return fail(WAVE_ESTATE, "wave_half_step: this context steps with a fused kernel "
                                 "(create it with kernel 1 or 2 for half steps)");
    if ((which == 1) != c->half_open)
        return fail(WAVE_ESTATE, "wave_half_step: the halves alternate, velocities first");
    for (int i = 0; i < 4; i++)
        if (((c->z_cut >> (i & 1)) & 1) && !c->zg[i])
            return fail(WAVE_ESTATE, "wave_half_step: set the ghost buffers first");
    AcParams prm;
    fill_acoustic_params(c, prm);
    prm.step = c->step;
    prm.zg_lo = c->zg[which == 0 ? 0 : 2];
    prm.zg_hi = c->zg[which == 0 ? 1 : 3];
    const size_t eb = elem_bytes(c->prec);
    cudaEvent_t m0 = mark(c);
    cudaError_t e;
    if (which == 0) {
        e = c->use_stream ? acoustic_stream_half_step(prm, c->prec, c->comp, 0, c->zchunk, c->stream)
                          : acoustic_generic_half_step(prm, c->ndim, c->prec, c->comp, 0, c->stream);
        cudaEvent_t m1 = mark(c);
        timed(c, 0, m0, m1);
        if (e != cudaSuccess) return cuda_check(c, e, "wave_half_step launch");
        c->half_open = true;
        return WAVE_OK;
    }
    prm.energy = 1;
    e = c->use_stream ? acoustic_stream_half_step(prm, c->prec, c->comp, 1, c->zchunk, c->stream)
                      : acoustic_generic_half_step(prm, c->ndim, c->prec, c->comp, 1, c->stream);
    cudaEvent_t m1 = mark(c);
    timed(c, 1, m0, m1);
    const bool trace = c->e_trace && c->e_trace_pos < c->e_trace_cap;
    if (e == cudaSuccess && trace)
        e = cudaMemcpyAsync(c->e_trace + c->e_trace_pos, c->e_misc.ptr, sizeof(double),
                            cudaMemcpyDeviceToDevice, c->stream);
    if (e == cudaSuccess && c->nrec && c->rec_pos < c->rec_cap)
        e = sample_receivers(c->f[c->rec_field].ptr, (int)eb, is_bf16_storage(c->prec),
                             static_cast<const int64_t *>(c->rec_q.ptr), (int)c->nrec,
                             c->rec_traces + c->rec_pos * c->nrec, c->stream);
    if (e != cudaSuccess) return cuda_check(c, e, "wave_half_step launch");
    if (trace) c->e_trace_pos++;
    if (c->nrec && c->rec_pos < c->rec_cap) c->rec_pos++;
    c->step++;
    c->half_open = false;
    c->have_energy = true;
    return WAVE_OK;
}

extern "C" wave_status wave_copy_planes(wave_ctx *c, wave_field field, int64_t z_first, int64_t nplanes,
                                        void *dst) {
    CHECK_CTX(c);
    if (!field_valid(c, field) || !dst) return fail(WAVE_EINVAL, "wave_copy_planes: bad field or NULL dst");
    if (z_first < 0 || nplanes < 0 || z_first + nplanes > c->n[2])
        return fail(WAVE_EINVAL, "wave_copy_planes: planes %lld..%lld outside 0..%lld", (long long)z_first,
                    (long long)(z_first + nplanes - 1), (long long)(c->n[2] - 1));
    const size_t eb = elem_bytes(c->prec);
    cudaError_t e = cudaMemcpyAsync(dst, static_cast<const char *>(c->f[field].ptr) + z_first * c->plane * eb,
                                    (size_t)(nplanes * c->plane) * eb, cudaMemcpyDeviceToDevice, c->stream);
    return cuda_check(c, e, "wave_copy_planes");
}

extern "C" wave_status wave_get_layout(wave_ctx *c, int64_t out[3]) {
    CHECK_CTX(c);
    if (!out) return fail(WAVE_EINVAL, "wave_get_layout: NULL out");
    out[0] = c->pitch;
    out[1] = c->plane;
    out[2] = (int64_t)elem_bytes(c->prec);
    return WAVE_OK;
}

// Read the device error word (set by a bounded wait that expired).
static wave_status check_device_error(wave_ctx *c) {
    int err = 0;
    cudaError_t e = cudaMemcpyAsync(&err, static_cast<char *>(c->e_misc.ptr) + 16, sizeof(int),
                                    cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_check(c, e, "error word");
    if (err) {
        c->poisoned = true;
        return fail(WAVE_ETIMEOUT, "a bounded device wait expired (pipeline stalled)");
    }
    return WAVE_OK;
}

extern "C" wave_status wave_selftest_timeout(wave_ctx *c) {
    CHECK_CTX(c);
    int *err = reinterpret_cast<int *>(static_cast<char *>(c->e_misc.ptr) + 16);
    cudaError_t e = selftest_wait(err, 1024, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_check(c, e, "self-test");
    return check_device_error(c);
}

extern "C" wave_status wave_sync(wave_ctx *c) {
    CHECK_CTX(c);
    wave_status st = cuda_check(c, cudaStreamSynchronize(c->stream), "wave_sync");
    return st ? st : check_device_error(c);
}

extern "C" wave_status wave_steps_done(wave_ctx *c, int64_t *steps) {
    CHECK_CTX(c);
    if (!steps) return fail(WAVE_EINVAL, "NULL output");
    *steps = c->step;
    return WAVE_OK;
}

// ------------------------------------------------------- checkpoint/resume
struct StateHeader {
    uint64_t magic;
    int64_t step;
    int64_t n[3];
    int32_t prec, comp, kind, nfields;
};
static const uint64_t kMagic = 0x31564157454C4657ull;

static int state_fields(const wave_ctx *c, int *list) {
    int k = 0;
    if (c->kind == WAVE_ACOUSTIC) {
        for (int f = 0; f <= c->ndim; f++) list[k++] = f;
    } else {
        const int ef[5] = {WAVE_F_VX, WAVE_F_VY, WAVE_F_SXX, WAVE_F_SYY, WAVE_F_SXY};
        for (int f : ef) list[k++] = f;
    }
    return k;
}

extern "C" wave_status wave_get_state(wave_ctx *c, void *blob, size_t *size) {
    CHECK_CTX(c);
    if (!size) return fail(WAVE_EINVAL, "NULL size");
    int list[7];
    const int nf = state_fields(c, list);
    const size_t arr = (size_t)(c->n[0] * c->n[1] * c->n[2]) * elem_bytes(c->prec);
    const size_t need = sizeof(StateHeader) + 2 * nf * arr;
    if (!blob) { *size = need; return WAVE_OK; }
    if (*size < need) return fail(WAVE_EINVAL, "state buffer too small (%zu < %zu)", *size, need);
    StateHeader hd{kMagic, c->step, {c->n[0], c->n[1], c->n[2]}, c->prec, c->comp, c->kind, nf};
    memcpy(blob, &hd, sizeof hd);
    unsigned char *p = static_cast<unsigned char *>(blob) + sizeof hd;
    for (int i = 0; i < nf; i++) {
        for (int comp = 0; comp < 2; comp++) {
            wave_status st = wave_get_raw(c, (wave_field)list[i], comp, p);
            if (st) return st;
            p += arr;
        }
    }
    *size = need;
    return WAVE_OK;
}

extern "C" wave_status wave_set_state(wave_ctx *c, const void *blob, size_t size) {
    CHECK_CTX(c);
    if (!blob || size < sizeof(StateHeader)) return fail(WAVE_EINVAL, "bad state blob");
    StateHeader hd;
    memcpy(&hd, blob, sizeof hd);
    int list[7];
    const int nf = state_fields(c, list);
    const size_t arr = (size_t)(c->n[0] * c->n[1] * c->n[2]) * elem_bytes(c->prec);
    if (hd.magic != kMagic || hd.n[0] != c->n[0] || hd.n[1] != c->n[1] || hd.n[2] != c->n[2] ||
        hd.prec != c->prec || hd.comp != c->comp || hd.kind != c->kind || hd.nfields != nf ||
        size < sizeof hd + 2 * nf * arr)
        return fail(WAVE_EINVAL, "state blob does not match this context");
    const unsigned char *p = static_cast<const unsigned char *>(blob) + sizeof hd;
    for (int i = 0; i < nf; i++) {
        wave_status st = wave_set_raw(c, (wave_field)list[i], 0, p);
        if (st) return st;
        p += arr;
        if (c->t[list[i]].ptr) {
            st = wave_set_raw(c, (wave_field)list[i], 1, p);
            if (st) return st;
        }
        p += arr;
    }
    c->step = hd.step;
    c->have_energy = false;
    return WAVE_OK;
}

extern "C" wave_status wave_set_timing(wave_ctx *c, int32_t enable) {
    CHECK_CTX(c);
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_check(c, e, "wave_set_timing");
    collect_timing(c);
    for (int k = 0; k < 4; k++) { c->t_launches[k] = 0; c->t_ms[k] = 0.0; }
    c->timing = enable != 0;
    return WAVE_OK;
}

extern "C" wave_status wave_get_timing(wave_ctx *c, int32_t kind, int64_t *launches, double *ms) {
    CHECK_CTX(c);
    if (kind < 0 || kind > 3 || !launches || !ms) return fail(WAVE_EINVAL, "bad timing query");
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_check(c, e, "wave_get_timing");
    collect_timing(c);
    *launches = c->t_launches[kind];
    *ms = c->t_ms[kind];
    return WAVE_OK;
}

// Zero every field and compensation (both buffer sets) and the step counter.
extern "C" wave_status wave_reset(wave_ctx *c) {
    CHECK_CTX(c);
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < 7 && e == cudaSuccess; i++) {
        if (c->f[i].ptr) e = cudaMemsetAsync(c->f[i].ptr, 0, c->f[i].bytes, c->stream);
        if (e == cudaSuccess && c->t[i].ptr) e = cudaMemsetAsync(c->t[i].ptr, 0, c->t[i].bytes, c->stream);
    }
    for (int i = 0; i < 4 && e == cudaSuccess; i++) {
        if (c->alt_f[i].ptr) e = cudaMemsetAsync(c->alt_f[i].ptr, 0, c->alt_f[i].bytes, c->stream);
        if (e == cudaSuccess && c->alt_t[i].ptr) e = cudaMemsetAsync(c->alt_t[i].ptr, 0, c->alt_t[i].bytes, c->stream);
    }
    if (e != cudaSuccess) return cuda_check(c, e, "wave_reset");
    c->step = 0;
    c->have_energy = false;
    c->half_open = false;
    c->rec_pos = 0;
    c->e_trace_pos = 0;
    c->adj.active = false;
    return WAVE_OK;
}

// ------------------------------------------------------------------ adjoint
// Arrays of a snapshot: p, v_c and, with compensation, t_p, t_v_c.
static int snapshot_arrays(wave_ctx *c, DevBuf **out) {
    int k = 0;
    for (int a = 0; a <= c->ndim; a++) out[k++] = &c->f[a];
    if (c->comp)
        for (int a = 0; a <= c->ndim; a++) out[k++] = &c->t[a];
    return k;
}

// save (to_slot) or restore (from slot) the forward state
static cudaError_t snapshot_copy(wave_ctx *c, int64_t slot, bool save) {
    DevBuf *arr[8];
    const int na = snapshot_arrays(c, arr);
    const size_t bytes = (size_t)c->total * elem_bytes(c->prec);
    char *base = static_cast<char *>(c->adj.cps.ptr) + (size_t)slot * na * bytes;
    for (int a = 0; a < na; a++) {
        void *dst = save ? (void *)(base + a * bytes) : arr[a]->ptr;
        const void *src = save ? arr[a]->ptr : (const void *)(base + a * bytes);
        cudaError_t e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, c->stream);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// binary32 copy of a per-point multiplier, negated, converted on the device
static wave_status make_neg_coef(wave_ctx *c, DevBuf &dst, int w) {
    if (dst.ptr) return WAVE_OK;
    wave_status st = dev_alloc(c, dst, (size_t)c->total * sizeof(float), false);
    if (st) return st;
    const int fmt = c->prec == PREC_FP32 ? ADJ_F32 : is_bf16_storage(c->prec) ? ADJ_BF16 : ADJ_F16;
    return cuda_check(c, adj_neg_coef(c->coef[w].ptr, fmt, static_cast<float *>(dst.ptr), c->total, c->stream),
                      "adjoint multipliers");
}

static wave_status adjoint_fused_setup(wave_ctx *c);

extern "C" wave_status wave_record(wave_ctx *c, int64_t nsteps, int64_t ncheckpoints) {
    CHECK_CTX(c);
    if (c->kind != WAVE_ACOUSTIC) return fail(WAVE_ENOTIMPL, "the adjoint covers the acoustic system");
    if (c->z_cut) return fail(WAVE_ENOTIMPL, "the adjoint covers whole grids, not z slabs");
    if (c->prec == PREC_FP16_PAIRS) return fail(WAVE_ENOTIMPL, "the adjoint covers the stored-value stencils");
    if (c->half_open) return fail(WAVE_ESTATE, "a velocity half step awaits its pressure half step");
    if (nsteps < 1) return fail(WAVE_EINVAL, "nsteps must be positive");
    if (c->nrec && c->rec_field != WAVE_F_P) return fail(WAVE_EINVAL, "adjoint receivers must record p");
    // the snapshot and replay buffers of a previous record are kept when they
    // are large enough (re-allocating gigabytes per shot costs more than a step)
    DevBuf keep_cps = c->adj.cps, keep_seg = c->adj.seg;
    c->adj.cps = DevBuf();
    c->adj.seg = DevBuf();
    adjoint_free(c);
    auto &A = c->adj;
    int64_t ncp = ncheckpoints > 0 ? ncheckpoints : (int64_t)ceil(sqrt((double)nsteps));
    ncp = std::max<int64_t>(1, std::min(ncp, nsteps));
    A.K = (nsteps + ncp - 1) / ncp;
    A.ncp = (nsteps + A.K - 1) / A.K;
    A.nsteps = nsteps;
    A.step0 = c->step;
    DevBuf *arr[8];
    A.narr = snapshot_arrays(c, arr);
    const size_t eb = elem_bytes(c->prec);
    const size_t abytes = (size_t)c->total * eb, fbytes = (size_t)c->total * sizeof(float);
    // snapshots and replayed velocities are written before they are read
    const size_t cps_bytes = (size_t)(A.ncp + 1) * A.narr * abytes, seg_bytes = (size_t)A.K * c->ndim * abytes;
    wave_status st = WAVE_OK;
    if (keep_cps.ptr && keep_cps.bytes >= cps_bytes) A.cps = keep_cps;
    else {
        dev_free(c, keep_cps);
        st = dev_alloc(c, A.cps, cps_bytes, false);
    }
    if (keep_seg.ptr && keep_seg.bytes >= seg_bytes) A.seg = keep_seg;
    else {
        dev_free(c, keep_seg);
        if (!st) st = dev_alloc(c, A.seg, seg_bytes, false);
    }
    if (!st) st = dev_alloc(c, A.mu, fbytes);
    if (!st) st = dev_alloc(c, A.g, fbytes);
    for (int ax = 0; ax < c->ndim && !st; ax++) st = dev_alloc(c, A.nu[ax], fbytes);
    if (st) {
        adjoint_free(c);
        return st;
    }
    // negated binary32 multipliers of the adjoint leapfrog
    for (int ax = 0; ax < c->ndim && !st; ax++) {
        if (c->coef_is_uniform[1 + ax]) {
            const float v = -(float)c->coef_host[1 + ax][0];
            memcpy(&A.na_uni[ax], &v, 4);
        } else {
            st = make_neg_coef(c, c->adj_na[ax], 1 + ax);
        }
    }
    if (!st) {
        if (c->coef_is_uniform[0]) {
            const float v = -(float)c->coef_host[0][0];
            memcpy(&A.nb_uni, &v, 4);
        } else {
            st = make_neg_coef(c, c->adj_nb, 0);
        }
    }
    // residual weights: b at each receiver, 0 on the rigid-wall nodes
    if (!st && c->nrec) {
        std::vector<int64_t> q(c->nrec);
        cudaError_t e = cudaMemcpy(q.data(), c->rec_q.ptr, c->nrec * sizeof(int64_t), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_check(c, e, "receiver read-back");
        std::vector<float> w(c->nrec);
        for (int64_t r = 0; r < c->nrec; r++) {
            const int64_t idx[3] = {q[r] % c->pitch, (q[r] / c->pitch) % c->n[1], q[r] / c->plane};
            bool wall = false;
            for (int ax = 0; ax < c->ndim; ax++) wall |= c->bc[2 * ax] == WAVE_BC_RIGID && idx[ax] == 0;
            const int64_t u = idx[0] + c->n[0] * (idx[1] + c->n[1] * idx[2]);
            w[r] = wall ? 0.f : (float)c->coef_host[0][c->coef_is_uniform[0] ? 0 : u];
        }
        // group the receivers by point (stable: receiver order within a point)
        std::vector<int> order(c->nrec), start;
        for (int64_t r = 0; r < c->nrec; r++) order[r] = (int)r;
        std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return q[a] < q[b]; });
        for (int64_t u = 0; u < c->nrec; u++)
            if (u == 0 || q[order[u]] != q[order[u - 1]]) start.push_back((int)u);
        A.ngroups = (int)start.size();
        start.push_back((int)c->nrec);
        st = dev_alloc(c, A.rec_w, w.size() * sizeof(float));
        if (!st) st = dev_alloc(c, A.rec_order, order.size() * sizeof(int));
        if (!st) st = dev_alloc(c, A.rec_start, start.size() * sizeof(int));
        if (!st) {
            e = cudaMemcpyAsync(A.rec_w.ptr, w.data(), w.size() * sizeof(float), cudaMemcpyHostToDevice, c->stream);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(A.rec_order.ptr, order.data(), order.size() * sizeof(int), cudaMemcpyHostToDevice,
                                    c->stream);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(A.rec_start.ptr, start.data(), start.size() * sizeof(int), cudaMemcpyHostToDevice,
                                    c->stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
            st = cuda_check(c, e, "receiver weights");
        }
    }
    if (!st && !c->adj_two_over_c.ptr) {
        st = dev_alloc(c, c->adj_two_over_c, c->two_over_c.size() * sizeof(float), false);
        if (!st) {
            cudaError_t e = cudaMemcpyAsync(c->adj_two_over_c.ptr, c->two_over_c.data(),
                                            c->two_over_c.size() * sizeof(float), cudaMemcpyHostToDevice,
                                            c->stream);
            st = cuda_check(c, e, "velocity upload");
        }
    }
    if (!st) st = adjoint_fused_setup(c);
    if (st) {
        adjoint_free(c);
        return st;
    }
    // forward run with a snapshot at the start of every segment of K steps
    A.cp_step.assign(A.ncp + 1, 0);
    for (int64_t i = 0; i < A.ncp; i++) {
        A.cp_step[i] = c->step;
        cudaError_t e = snapshot_copy(c, i, true);
        if (e != cudaSuccess) return cuda_check(c, e, "checkpoint");
        st = acoustic_steps(c, std::min(A.K, nsteps - i * A.K), i == A.ncp - 1);
        if (st) return st;
    }
    A.cp_step[A.ncp] = c->step;
    cudaError_t e = snapshot_copy(c, A.ncp, true);
    if (e != cudaSuccess) return cuda_check(c, e, "end state");
    c->have_energy = true;
    A.t = nsteps;
    A.active = true;
    return WAVE_OK;
}

// Replay segment si from its checkpoint, keeping v^{n+1/2} of every step.
static wave_status adjoint_replay(wave_ctx *c, int64_t si) {
    auto &A = c->adj;
    cudaError_t e = snapshot_copy(c, si, false);
    if (e != cudaSuccess) return cuda_check(c, e, "checkpoint restore");
    c->step = A.cp_step[si];
    const int64_t lo = si * A.K, len = std::min(A.K, A.nsteps - lo);
    const int64_t nrec = c->nrec;
    double *etr = c->e_trace;
    c->nrec = 0;
    c->e_trace = nullptr;
    const size_t bytes = (size_t)c->total * elem_bytes(c->prec);
    wave_status st = WAVE_OK;
    for (int64_t m = 0; m < len && !st; m++) {
        st = acoustic_steps(c, 1, false);
        for (int ax = 0; ax < c->ndim && !st; ax++) {
            e = cudaMemcpyAsync(static_cast<char *>(A.seg.ptr) + (size_t)(m * c->ndim + ax) * bytes, c->f[1 + ax].ptr,
                                bytes, cudaMemcpyDeviceToDevice, c->stream);
            st = cuda_check(c, e, "replay copy");
        }
    }
    c->nrec = nrec;
    c->e_trace = etr;
    if (st) return st;
    A.seg_lo = lo;
    A.seg_n = len;
    return WAVE_OK;
}

// Leapfrog parameters of the adjoint sweep on the current mu~, nu~: the
// negated binary32 multipliers, no source, no energy.
static void adjoint_params(const wave_ctx *c, AcParams &prm) {
    const auto &A = c->adj;
    memset(&prm, 0, sizeof prm);
    for (int ax = 0; ax < 3; ax++) {
        prm.n[ax] = (int)c->n[ax];
        prm.bc[ax] = ax < c->ndim ? (c->bc[2 * ax] == WAVE_BC_PERIODIC ? BC_PERIODIC : BC_RIGID) : BC_PERIODIC;
        prm.v[ax] = A.nu[ax].ptr;
        prm.a[ax] = c->adj_na[ax].ptr;
        prm.a_uni[ax] = A.na_uni[ax];
    }
    prm.sy = c->pitch;
    prm.sz = c->plane;
    prm.p = A.mu.ptr;
    prm.b = c->adj_nb.ptr;
    prm.b_uni = A.nb_uni;
    prm.src_q = -1;
    prm.src_i = prm.src_j = prm.src_k = -1;
}

// Second buffer set and tensor maps for the one-pass adjoint leapfrog, where
// the one-pass step applies (3D, uniform a_c, rigid x faces). Without them the
// sweep runs the two half-step kernels; both give the same bits.
static wave_status adjoint_fused_setup(wave_ctx *c) {
    auto &A = c->adj;
    AcParams prm;
    adjoint_params(c, prm);
    A.fused = false;
    if (!c->use_fused || !acoustic_fused_supported(prm, c->ndim, PREC_FP32) ||
        fused_maps_bytes() > sizeof(A.fm[0].b))
        return WAVE_OK;
    const size_t fbytes = (size_t)c->total * sizeof(float);
    wave_status st = dev_alloc(c, A.mu_alt, fbytes);
    for (int ax = 0; ax < c->ndim && !st; ax++) st = dev_alloc(c, A.nu_alt[ax], fbytes);
    if (st) return st;
    for (int set = 0; set < 2; set++) {
        const void *in[7] = {set ? A.mu_alt.ptr : A.mu.ptr, set ? A.nu_alt[0].ptr : A.nu[0].ptr,
                             set ? A.nu_alt[1].ptr : A.nu[1].ptr, set ? A.nu_alt[2].ptr : A.nu[2].ptr,
                             nullptr, nullptr, nullptr};
        if (!acoustic_fused_encode(A.fm[set].b, prm, in, nullptr, PREC_FP32, 0)) return WAVE_OK;
    }
    A.fset = 0;
    A.fused = true;
    return WAVE_OK;
}

extern "C" wave_status wave_adjoint_step(wave_ctx *c, int64_t n, const float *residual) {
    CHECK_CTX(c);
    auto &A = c->adj;
    if (!A.active) return fail(WAVE_ESTATE, "no recorded run: call wave_record first");
    if (n < 0 || n > A.t) return fail(WAVE_EINVAL, "n = %lld outside 0..%lld", (long long)n, (long long)A.t);
    if (c->nrec && !residual) return fail(WAVE_EINVAL, "residual traces are NULL");
    if (n == 0) return WAVE_OK;
    AcParams prm;
    adjoint_params(c, prm);
    const bool stream_ok = acoustic_stream_supported(prm, c->ndim, PREC_FP32);
    AdjGradParams gp;
    memset(&gp, 0, sizeof gp);
    for (int ax = 0; ax < 3; ax++) {
        gp.n[ax] = prm.n[ax];
        gp.bc[ax] = prm.bc[ax];
    }
    gp.sy = c->pitch;
    gp.sz = c->plane;
    gp.g = static_cast<float *>(A.g.ptr);
    const int fmt = c->prec == PREC_FP32 ? ADJ_F32 : is_bf16_storage(c->prec) ? ADJ_BF16 : ADJ_F16;
    const size_t bytes = (size_t)c->total * elem_bytes(c->prec);
    for (int64_t r = 0; r < n; r++) {
        const int64_t s = A.t - 1;  // recorded step being reversed
        if (!(s >= A.seg_lo && s < A.seg_lo + A.seg_n)) {
            wave_status st = adjoint_replay(c, s / A.K);
            if (st) return st;
        }
        cudaError_t e = adj_inject(static_cast<float *>(A.mu.ptr), static_cast<const int64_t *>(c->rec_q.ptr),
                                   static_cast<const float *>(A.rec_w.ptr), static_cast<const int *>(A.rec_order.ptr),
                                   static_cast<const int *>(A.rec_start.ptr), A.ngroups, residual + s * c->nrec,
                                   c->stream);
        const int64_t gstep = A.step0 + s;
        gp.src_q = (c->src_q >= 0 && gstep < c->src_nt) ? c->src_q : -1;
        gp.src_value = gp.src_q >= 0 ? c->src_host[gstep] : 0.f;
        gp.mu = static_cast<const float *>(A.mu.ptr);
        for (int ax = 0; ax < c->ndim; ax++)
            gp.v[ax] = static_cast<const char *>(A.seg.ptr) + (size_t)((s - A.seg_lo) * c->ndim + ax) * bytes;
        if (A.fused) {
            // g reads mu~ after the injection and before the pressure update,
            // as in the two-kernel order below (the velocity update leaves mu~)
            if (e == cudaSuccess) e = adj_grad(gp, c->ndim, fmt, c->stream);
            const void *in[7] = {A.mu.ptr, A.nu[0].ptr, A.nu[1].ptr, A.nu[2].ptr, nullptr, nullptr, nullptr};
            void *out[7] = {A.mu_alt.ptr, A.nu_alt[0].ptr, A.nu_alt[1].ptr, A.nu_alt[2].ptr,
                            nullptr, nullptr, nullptr};
            int *err = reinterpret_cast<int *>(static_cast<char *>(c->e_misc.ptr) + 16);
            prm.p = A.mu.ptr;
            for (int ax = 0; ax < 3; ax++) prm.v[ax] = A.nu[ax].ptr;
            if (e == cudaSuccess)
                e = acoustic_fused_step(prm, A.fm[A.fset].b, in, out, nullptr, nullptr, PREC_FP32, 0, c->zchunk,
                                        err, c->stream);
            A.fset ^= 1;
            std::swap(A.mu, A.mu_alt);
            for (int ax = 0; ax < 3; ax++) std::swap(A.nu[ax], A.nu_alt[ax]);
        } else {
            if (e == cudaSuccess)
                e = stream_ok ? acoustic_stream_half_step(prm, PREC_FP32, 0, 0, c->zchunk, c->stream)
                              : acoustic_generic_half_step(prm, c->ndim, PREC_FP32, 0, 0, c->stream);
            if (e == cudaSuccess) e = adj_grad(gp, c->ndim, fmt, c->stream);
            if (e == cudaSuccess)
                e = stream_ok ? acoustic_stream_half_step(prm, PREC_FP32, 0, 1, c->zchunk, c->stream)
                              : acoustic_generic_half_step(prm, c->ndim, PREC_FP32, 0, 1, c->stream);
        }
        if (e != cudaSuccess) return cuda_check(c, e, "adjoint step");
        A.t--;
    }
    // the forward fields show the end of the recorded run again
    cudaError_t e = snapshot_copy(c, A.ncp, false);
    c->step = A.cp_step[A.ncp];
    return cuda_check(c, e, "end state restore");
}

extern "C" wave_status wave_get_gradient(wave_ctx *c, float *device_out, int64_t *steps_left) {
    CHECK_CTX(c);
    auto &A = c->adj;
    if (!A.active) return fail(WAVE_ESTATE, "no recorded run: call wave_record first");
    if (steps_left) *steps_left = A.t;
    if (!device_out) return WAVE_OK;
    int n[3] = {(int)c->n[0], (int)c->n[1], (int)c->n[2]};
    cudaError_t e = adj_finish(device_out, static_cast<const float *>(A.g.ptr),
                               static_cast<const float *>(c->adj_two_over_c.ptr), n, c->pitch, c->plane, c->stream);
    return cuda_check(c, e, "gradient");
}

// ------------------------------------------------------------------ batches
struct wave_batch {
    std::vector<wave_ctx *> ctx;
    cudaStream_t stream = nullptr;
    int prec = 0, comp = 0;
    BatchShot *d_shots = nullptr;
    int *d_item0 = nullptr;
    double *d_part = nullptr;
    unsigned int *d_sync = nullptr;  // [barrier counter][error word] of the persistent launches
    std::vector<BatchShot> h_shots;
    int shape = 0, nitems = 0, sms = 1;
    bool tuned = false;
    cudaGraphExec_t gexec = nullptr;
    int gsteps = 0;
};

// Launch shapes the autotuner tries (every one computes the same bits).
struct BatchShape {
    int kind, bx, by, yc, wpb, grid_per_sm;
};
static const BatchShape kShapes[] = {
    {BATCH_POINTS, 32, 8, 0, 0, 4},  {BATCH_POINTS, 32, 8, 0, 0, 8},
    {BATCH_STRIPS, 0, 0, 16, 8, 4},  {BATCH_STRIPS, 0, 0, 16, 8, 8},
    {BATCH_STRIPS, 0, 0, 32, 8, 4},  {BATCH_STRIPS, 0, 0, 32, 8, 8},
    {BATCH_STRIPS, 0, 0, 64, 8, 4},  {BATCH_STRIPS, 0, 0, 64, 8, 8},
    {BATCH_STRIPS, 0, 0, 16, 4, 8},  {BATCH_STRIPS, 0, 0, 16, 4, 16},
    {BATCH_STRIPS, 0, 0, 32, 4, 8},  {BATCH_STRIPS, 0, 0, 32, 4, 16},
    {BATCH_STRIPS, 0, 0, 64, 4, 8},  {BATCH_STRIPS, 0, 0, 64, 4, 16},
    // every step of a call in one cooperative launch (grid: as many blocks as
    // are resident at once)
    {BATCH_PERSIST, 0, 0, 16, 8, 0}, {BATCH_PERSIST, 0, 0, 32, 8, 0},
    {BATCH_PERSIST, 0, 0, 16, 4, 0}, {BATCH_PERSIST, 0, 0, 32, 4, 0},
    // one-pass strips last (the tuner runs the candidates in this order)
    {BATCH_FUSED, 0, 0, 16, 4, 8},   {BATCH_FUSED, 0, 0, 16, 4, 16},
    {BATCH_FUSED, 0, 0, 32, 4, 8},   {BATCH_FUSED, 0, 0, 32, 4, 16},
    {BATCH_FUSED, 0, 0, 64, 4, 8},   {BATCH_FUSED, 0, 0, 64, 4, 16},
};
constexpr int kNumShapes = (int)(sizeof(kShapes) / sizeof(kShapes[0]));
constexpr int kDefaultShape = 5;

// work list of a launch shape: first item of each shot
static int batch_items(wave_batch *b, const BatchShape &sh, std::vector<int> &item0) {
    item0.assign(b->ctx.size() + 1, 0);
    for (size_t s = 0; s < b->ctx.size(); s++)
        item0[s + 1] = item0[s] + (int)batch_items_of(sh.kind, sh.bx, sh.by, sh.yc, b->prec, b->ctx[s]->n[0],
                                                      b->ctx[s]->n[1]);
    return item0.back();
}

static cudaError_t batch_set_shape(wave_batch *b, int shape) {
    std::vector<int> item0;
    b->shape = shape;
    b->nitems = batch_items(b, kShapes[shape], item0);
    cudaError_t e = cudaMemcpyAsync(b->d_item0, item0.data(), item0.size() * sizeof(int),
                                    cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    return e;
}

static BatchLaunch batch_launch(wave_batch *b) {
    const BatchShape &sh = kShapes[b->shape];
    BatchLaunch L;
    L.shots = b->d_shots;
    L.item0 = b->d_item0;
    L.item_part = b->d_part;
    L.nshots = (int)b->ctx.size();
    L.nitems = b->nitems;
    L.kind = sh.kind;
    L.bx = sh.bx;
    L.by = sh.by;
    L.yc = sh.yc;
    L.wpb = sh.wpb;
    L.grid = sh.grid_per_sm * b->sms;
    L.bar = b->d_sync;
    L.err = reinterpret_cast<int *>(b->d_sync + 1);
    return L;
}

extern "C" void wave_batch_destroy(wave_batch *b) {
    if (!b) return;
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    cudaStreamSynchronize(b->stream);
    if (b->d_shots) cudaFree(b->d_shots);
    if (b->d_item0) cudaFree(b->d_item0);
    if (b->d_part) cudaFree(b->d_part);
    if (b->d_sync) cudaFree(b->d_sync);
    delete b;
}

extern "C" wave_status wave_batch_create(int32_t nctx, wave_ctx *const *ctxs, wave_batch **out) {
    if (!out || !ctxs) return fail(WAVE_EINVAL, "wave_batch_create: NULL argument");
    *out = nullptr;
    if (nctx < 1 || nctx > batch_max_shots()) return fail(WAVE_EINVAL, "nctx must be 1..%d", batch_max_shots());
    for (int i = 0; i < nctx; i++) {
        const wave_ctx *c = ctxs[i];
        if (!c) return fail(WAVE_EINVAL, "context %d is NULL", i);
        if (c->poisoned) return fail(WAVE_ESTATE, "context %d poisoned", i);
        if (c->kind != WAVE_ACOUSTIC || c->ndim != 2)
            return fail(WAVE_EINVAL, "context %d: batches take 2D acoustic contexts", i);
        if (c->prec != ctxs[0]->prec || c->comp != ctxs[0]->comp || c->stream != ctxs[0]->stream)
            return fail(WAVE_EINVAL, "context %d: precision, compensation and stream must match", i);
        if (c->nrec) return fail(WAVE_EINVAL, "context %d has receivers (not supported in batches)", i);
        if (c->e_trace) return fail(WAVE_EINVAL, "context %d has an energy trace (not supported in batches)", i);
        for (int j = 0; j < i; j++)
            if (ctxs[j] == c) return fail(WAVE_EINVAL, "context %d appears twice", i);
    }
    wave_batch *b = new (std::nothrow) wave_batch();
    if (!b) return fail(WAVE_ENOMEM, "host allocation failed");
    b->ctx.assign(ctxs, ctxs + nctx);
    b->stream = ctxs[0]->stream;
    b->prec = ctxs[0]->prec;
    b->comp = ctxs[0]->comp;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev);
    int max_items = 0;
    std::vector<int> tmp;
    for (const auto &sh : kShapes) max_items = std::max(max_items, batch_items(b, sh, tmp));
    cudaError_t e = cudaMalloc(&b->d_shots, sizeof(BatchShot) * nctx);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_item0, sizeof(int) * (nctx + 1));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_part, sizeof(double) * (size_t)max_items);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_sync, 2 * sizeof(unsigned int));
    if (e == cudaSuccess) e = batch_set_shape(b, kDefaultShape);
    if (e != cudaSuccess) {
        wave_batch_destroy(b);
        cudaGetLastError();
        return fail(e == cudaErrorMemoryAllocation ? WAVE_ENOMEM : WAVE_ECUDA, "wave_batch_create: %s",
                    cudaGetErrorString(e));
    }
    *out = b;
    return WAVE_OK;
}

// upload every shot's parameters, step counter and alternate set
static cudaError_t batch_refresh(wave_batch *b) {
    b->h_shots.resize(b->ctx.size());
    for (size_t s = 0; s < b->ctx.size(); s++) fill_shot(b->ctx[s], b->h_shots[s]);
    return cudaMemcpyAsync(b->d_shots, b->h_shots.data(), sizeof(BatchShot) * b->ctx.size(),
                           cudaMemcpyHostToDevice, b->stream);
}

// The one-pass strips need every context's alternate buffer set.
static bool batch_shape_allowed(const wave_batch *b, int shape) {
    if (kShapes[shape].kind != BATCH_FUSED) return true;
    for (const auto *c : b->ctx)
        if (!c->strip_fused) return false;
    return true;
}

// After nf one-pass steps the contexts' state lives in the alternate sets
// when nf is odd: the host's set pointers follow.
static void batch_follow_sets(wave_batch *b, int64_t nf) {
    if (nf & 1)
        for (auto *c : b->ctx) swap_sets(c);
}

static wave_status batch_fail(wave_batch *b, cudaError_t e, const char *what) {
    for (auto *c : b->ctx) c->poisoned = true;
    cudaGetLastError();
    return fail(WAVE_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

extern "C" wave_status wave_batch_step(wave_batch *b, int64_t n) {
    if (!b) return fail(WAVE_EINVAL, "wave_batch_step: NULL batch");
    if (n < 0) return fail(WAVE_EINVAL, "negative step count");
    for (auto *c : b->ctx)
        if (c->poisoned) return fail(WAVE_ESTATE, "a context of the batch is poisoned");
    if (n == 0) return WAVE_OK;
    cudaError_t e = batch_refresh(b);
    if (e != cudaSuccess) return batch_fail(b, e, "batch upload");
    int64_t left = n;
    if (!b->tuned && left - 1 >= kNumShapes) {
        int64_t nf = 0;  // one-pass steps among the candidates
        // autotune on real steps: every candidate computes the same bits
        float best = 1e30f;
        int bi = kDefaultShape;
        cudaEvent_t e0, e1;
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        for (int si = 0; si < kNumShapes && e == cudaSuccess; si++) {
            if (!batch_shape_allowed(b, si)) continue;
            e = batch_set_shape(b, si);
            if (e != cudaSuccess) break;
            if (kShapes[si].kind == BATCH_FUSED) nf++;
            cudaEventRecord(e0, b->stream);
            e = batch_step(batch_launch(b), b->prec, b->comp, false, b->stream);
            cudaEventRecord(e1, b->stream);
            if (e != cudaSuccess) break;
            e = cudaEventSynchronize(e1);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (ms < best) {
                best = ms;
                bi = si;
            }
            left--;
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        if (e != cudaSuccess) return batch_fail(b, e, "batch autotune");
        // the candidate steps count as steps of the contexts; the one-pass
        // ones may have moved the state to the alternate sets: follow it and
        // upload the parameters again for the steps below
        const int64_t tuned_steps = n - left;
        for (auto *c : b->ctx) c->step += tuned_steps;
        batch_follow_sets(b, nf);
        e = batch_refresh(b);
        if (e == cudaSuccess) e = batch_set_shape(b, bi);
        if (e != cudaSuccess) return batch_fail(b, e, "batch shape");
        for (auto *c : b->ctx) c->step -= tuned_steps;  // added back with the rest below
        b->tuned = true;
    }
    const BatchLaunch L = batch_launch(b);
    if (kShapes[b->shape].kind == BATCH_PERSIST) {
        // every remaining step in one cooperative launch (the last with the energy)
        e = batch_persist(L, b->prec, b->comp, left, true, b->stream);
        if (e != cudaSuccess) return batch_fail(b, e, "batch persistent launch");
        for (auto *c : b->ctx) {
            c->step += n;
            c->have_energy = true;
        }
        return WAVE_OK;
    }
    int64_t plain = left - 1;  // steps without energy; the last step reduces it
    const int G = 32;
    if (b->tuned && b->stream != nullptr && plain >= G) {
        if (!b->gexec) {
            cudaGraph_t g = nullptr;
            e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
            if (e == cudaSuccess) {
                for (int s = 0; s < G && e == cudaSuccess; s++) e = batch_step(L, b->prec, b->comp, false, b->stream);
                cudaError_t e2 = cudaStreamEndCapture(b->stream, &g);
                if (e == cudaSuccess) e = e2;
            }
            if (e == cudaSuccess) e = cudaGraphInstantiate(&b->gexec, g, 0);
            if (g) cudaGraphDestroy(g);
            if (e != cudaSuccess) {  // no graph: fall back to plain launches
                cudaGetLastError();
                b->gexec = nullptr;
            } else {
                b->gsteps = G;
            }
        }
        while (b->gexec && plain >= G) {
            e = cudaGraphLaunch(b->gexec, b->stream);
            if (e != cudaSuccess) return batch_fail(b, e, "graph launch");
            plain -= G;
        }
    }
    for (int64_t s = 0; s < plain; s++) {
        e = batch_step(L, b->prec, b->comp, false, b->stream);
        if (e != cudaSuccess) return batch_fail(b, e, "batch launch");
    }
    e = batch_step(L, b->prec, b->comp, true, b->stream);
    if (e != cudaSuccess) return batch_fail(b, e, "batch launch");
    if (kShapes[b->shape].kind == BATCH_FUSED) batch_follow_sets(b, left);
    for (auto *c : b->ctx) {
        c->step += n;
        c->have_energy = true;
    }
    return WAVE_OK;
}

extern "C" wave_status wave_batch_set_shape(wave_batch *b, int32_t shape) {
    if (!b) return fail(WAVE_EINVAL, "wave_batch_set_shape: NULL batch");
    if (shape < 0 || shape >= kNumShapes) return fail(WAVE_EINVAL, "launch shape %d not in 0..%d", shape, kNumShapes - 1);
    if (!batch_shape_allowed(b, shape))
        return fail(WAVE_EINVAL, "launch shape %d needs every context's second buffer set (kernel 3)", shape);
    if (b->prec == WAVE_FP16_PAIRS && kShapes[shape].kind == BATCH_FUSED)
        return fail(WAVE_EINVAL, "the one-pass strips read the stored values only");
    cudaError_t e = batch_set_shape(b, shape);
    if (e != cudaSuccess) return batch_fail(b, e, "batch shape");
    if (b->gexec) {  // the captured graph belongs to the previous shape
        cudaGraphExecDestroy(b->gexec);
        b->gexec = nullptr;
        b->gsteps = 0;
    }
    b->tuned = true;
    return WAVE_OK;
}

extern "C" wave_status wave_batch_info(wave_batch *b, int32_t *info, int32_t ninfo) {
    if (!b || !info) return fail(WAVE_EINVAL, "NULL argument");
    const BatchShape &sh = kShapes[b->shape];
    const bool strips = sh.kind == BATCH_STRIPS || sh.kind == BATCH_FUSED || sh.kind == BATCH_PERSIST;
    const int32_t v[7] = {sh.kind, strips ? 32 * (b->prec == WAVE_FP32 ? 4 : 8) : sh.bx,
                          strips ? sh.yc : sh.by, strips ? 32 * sh.wpb : sh.bx * sh.by,
                          sh.grid_per_sm * b->sms, b->gexec ? b->gsteps : 0, b->tuned ? 1 : 0};
    for (int i = 0; i < ninfo && i < 7; i++) info[i] = v[i];
    return WAVE_OK;
}
