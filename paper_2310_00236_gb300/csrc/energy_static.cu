// energy_static.cu -- the discrete acoustic energy on caller-owned arrays,
// with no device allocation: the reduction's scratch is a fixed-size static
// device array of this file.
//
// Some callers cannot allocate device memory: a host framework that reserves
// the whole device heap at start-up and hands out only views of it (a
// cudaMalloc of its own would fail or break the framework's accounting), or a
// real-time loop with a fixed memory budget that forbids any allocation after
// start-up (an allocation can block, fragment the heap or fail mid-run).
// wave_energy_acoustic_static serves them: they pass the fields and
// multipliers they already hold, and the per-block partial sums go to
// g_energy_scratch below instead of a buffer from cudaMalloc.
#include <cuda.h>
#include <cuda_runtime.h>
#include <mutex>
#include <stdio.h>

#include "../../include/wave.h"
#include "wave_arith.cuh"

namespace wave {
void set_last_error_text(const char *msg);  // defined with the other ABI entry points
}

namespace {

constexpr int kThreads = 256;
constexpr int kPointsPerThread = 8;
constexpr int kPointsPerBlock = kThreads * kPointsPerThread;  // 2048

struct EnergyScratch {
    double part[WAVE_ENERGY_STATIC_MAX_BLOCKS];
    unsigned int count;
};

// Every GPU that loads the library holds one of these until the process exits.
static __device__ __align__(256) EnergyScratch g_energy_scratch;

enum { TAG_F32 = 0, TAG_F16 = 1, TAG_BF16 = 2 };

thread_local char g_static_err[256];

// Report through wave_last_error().
void set_error(const char *msg) { wave::set_last_error_text(msg); }

template <int PREC>
__device__ __forceinline__ float load_f32(const void *f, int64_t q) {
    if (PREC == TAG_F32) return static_cast<const float *>(f)[q];
    const uint16_t s = static_cast<const uint16_t *>(f)[q];
    if (PREC == TAG_BF16) return wave::BF16::to_f32(s);
    return wave::F16::to_f32(s);
}

// The same terms as the energy of the stepping kernels, with a per-point
// division where the fused one-pass step multiplies by rounded reciprocals of
// a uniform a: products in binary32 (exact for half / bfloat16), one correctly
// rounded division per term, a compensated binary32 sum per thread, binary64
// across threads and blocks.
template <int PREC, int NDIM>
__global__ void __launch_bounds__(kThreads)
energy_static_kernel(int64_t npts, const void *p_old, const void *p_new, const void *v0,
                     const void *v1, const void *v2, const void *a0, const void *a1,
                     const void *a2, const void *b, double factor, double *out,
                     EnergyScratch *scratch) {
    const void *v[3] = {v0, v1, v2};
    const void *a[3] = {a0, a1, a2};
    float s = 0.f, c = 0.f;
    const int64_t base = (int64_t)blockIdx.x * kPointsPerBlock + threadIdx.x;
#pragma unroll
    for (int r = 0; r < kPointsPerThread; r++) {
        const int64_t q = base + (int64_t)r * kThreads;
        if (q >= npts) break;
        float terms[4];
        terms[0] = __fdiv_rn(__fmul_rn(load_f32<PREC>(p_old, q), load_f32<PREC>(p_new, q)),
                             load_f32<PREC>(b, q));
#pragma unroll
        for (int d = 0; d < 3; d++) {
            if (d >= NDIM) { terms[1 + d] = 0.f; continue; }
            const float vv = load_f32<PREC>(v[d], q);
            terms[1 + d] = __fdiv_rn(__fmul_rn(vv, vv), load_f32<PREC>(a[d], q));
        }
#pragma unroll
        for (int t = 0; t < 4; t++) {
            const float x = terms[t];
            const float y = __fadd_rn(s, x);
            const float pa = __fsub_rn(y, x);
            const float pb = __fsub_rn(y, pa);
            c = __fadd_rn(c, __fadd_rn(__fsub_rn(s, pa), __fsub_rn(x, pb)));
            s = y;
        }
    }
    double val = (double)s + (double)c;
    __shared__ double warp_sums[kThreads / 32];
    __shared__ bool is_last;
    for (int off = 16; off > 0; off >>= 1) val += __shfl_down_sync(0xffffffffu, val, off);
    if ((threadIdx.x & 31) == 0) warp_sums[threadIdx.x >> 5] = val;
    __syncthreads();
    if (threadIdx.x == 0) {
        double bs = 0.0;
        for (int w = 0; w < kThreads / 32; w++) bs += warp_sums[w];
        scratch->part[blockIdx.x] = bs;
        __threadfence();
        const unsigned prev = atomicAdd(&scratch->count, 1u);
        is_last = (prev == gridDim.x - 1);
    }
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    double tot = 0.0;
    for (unsigned i = threadIdx.x; i < gridDim.x; i += kThreads) tot += __ldcg(&scratch->part[i]);
    for (int off = 16; off > 0; off >>= 1) tot += __shfl_down_sync(0xffffffffu, tot, off);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) warp_sums[threadIdx.x >> 5] = tot;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < kThreads / 32; w++) t += warp_sums[w];
        *out = t * factor;
        scratch->count = 0u;
    }
}

// Device address of g_energy_scratch, looked up with the device current (the
// host-side name is only a stand-in for the symbol) and cached per device
// together with the identity of the CUDA context it was looked up in: a new
// context on the device (after cudaDeviceReset, say) loads the module afresh
// at another address, so the lookup is repeated then.
typedef CUresult (*CtxGetCurrentFn)(CUcontext *);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long *);

struct ScratchSlot {
    unsigned long long ctx_id;
    void *addr;
};
std::mutex g_scratch_mu;
ScratchSlot g_scratch_slot[256] = {};
CtxGetCurrentFn g_ctx_get_current = nullptr;
CtxGetIdFn g_ctx_get_id = nullptr;

// Identity of the current context, 0 if there is none yet (or the driver
// entry points are unavailable).
unsigned long long current_ctx_id() {
    if (!g_ctx_get_current || !g_ctx_get_id) {
        void *p1 = nullptr, *p2 = nullptr;
        cudaDriverEntryPointQueryResult q1, q2;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p1, 12000, cudaEnableDefault, &q1) !=
                cudaSuccess || q1 != cudaDriverEntryPointSuccess ||
            cudaGetDriverEntryPointByVersion("cuCtxGetId", &p2, 12000, cudaEnableDefault, &q2) !=
                cudaSuccess || q2 != cudaDriverEntryPointSuccess)
            return 0;
        g_ctx_get_current = reinterpret_cast<CtxGetCurrentFn>(p1);
        g_ctx_get_id = reinterpret_cast<CtxGetIdFn>(p2);
    }
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (g_ctx_get_current(&ctx) != CUDA_SUCCESS || !ctx) return 0;
    if (g_ctx_get_id(ctx, &id) != CUDA_SUCCESS) return 0;
    return id;
}

wave_status scratch_address(EnergyScratch **out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= 256) {
        snprintf(g_static_err, sizeof g_static_err, "wave_energy_acoustic_static: no current device (%s)",
                 cudaGetErrorString(e));
        set_error(g_static_err);
        return WAVE_ECUDA;
    }
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    const unsigned long long id = current_ctx_id();
    ScratchSlot &slot = g_scratch_slot[dev];
    if (!slot.addr || id == 0 || slot.ctx_id != id) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_energy_scratch);
        if (e != cudaSuccess || !p) {
            snprintf(g_static_err, sizeof g_static_err,
                     "wave_energy_acoustic_static: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
            set_error(g_static_err);
            return WAVE_ECUDA;
        }
        slot.addr = p;
        slot.ctx_id = current_ctx_id();  // the lookup has made the context current
    }
    *out = static_cast<EnergyScratch *>(slot.addr);
    return WAVE_OK;
}

template <int PREC>
cudaError_t launch(int ndim, int64_t npts, unsigned blocks, const void *p_old, const void *p_new,
                   const void *const v[3], const void *const a[3], const void *b, double factor,
                   double *out, EnergyScratch *scr, cudaStream_t st) {
    if (ndim == 3)
        energy_static_kernel<PREC, 3><<<blocks, kThreads, 0, st>>>(
            npts, p_old, p_new, v[0], v[1], v[2], a[0], a[1], a[2], b, factor, out, scr);
    else
        energy_static_kernel<PREC, 2><<<blocks, kThreads, 0, st>>>(
            npts, p_old, p_new, v[0], v[1], nullptr, a[0], a[1], nullptr, b, factor, out, scr);
    return cudaGetLastError();
}

}  // namespace

extern "C" wave_status wave_energy_acoustic_static(int32_t ndim, const int64_t n[3],
                                                   wave_precision prec, const void *p_old,
                                                   const void *p_new, const void *const v[3],
                                                   const void *const a[3], const void *b,
                                                   double factor, double *device_out,
                                                   void *cuda_stream) {
    if ((ndim != 2 && ndim != 3) || !n || !p_old || !p_new || !v || !a || !b || !device_out) {
        snprintf(g_static_err, sizeof g_static_err, "wave_energy_acoustic_static: bad arguments");
        set_error(g_static_err);
        return WAVE_EINVAL;
    }
    const int64_t maxp = (int64_t)WAVE_ENERGY_STATIC_MAX_BLOCKS * kPointsPerBlock;
    int64_t npts = 1;
    for (int d = 0; d < ndim; d++) {
        if (!v[d] || !a[d] || n[d] < 1) {
            snprintf(g_static_err, sizeof g_static_err, "wave_energy_acoustic_static: bad arguments");
            set_error(g_static_err);
            return WAVE_EINVAL;
        }
        // the product of the extents, stopped at the limit before it can overflow
        if (npts <= maxp) npts = n[d] > maxp ? maxp + 1 : npts * n[d];
    }
    if (prec != WAVE_FP32 && prec != WAVE_FP16 && prec != WAVE_BF16 && prec != WAVE_FP16_F32ARITH &&
        prec != WAVE_BF16_F32ARITH) {
        snprintf(g_static_err, sizeof g_static_err, "wave_energy_acoustic_static: bad precision %d",
                 (int)prec);
        set_error(g_static_err);
        return WAVE_EINVAL;
    }
    if (npts > maxp) {
        snprintf(g_static_err, sizeof g_static_err,
                 "wave_energy_acoustic_static: the grid exceeds the static scratch limit of %lld "
                 "points (%d blocks of %d)", (long long)maxp, WAVE_ENERGY_STATIC_MAX_BLOCKS,
                 kPointsPerBlock);
        set_error(g_static_err);
        return WAVE_EINVAL;
    }
    EnergyScratch *scr = nullptr;
    wave_status ws = scratch_address(&scr);
    if (ws) return ws;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    // the counter must start at zero; a previous call leaves it at zero, but an
    // interrupted one might not
    cudaError_t e = cudaMemsetAsync(&scr->count, 0, sizeof(unsigned int), st);
    const unsigned blocks = (unsigned)((npts + kPointsPerBlock - 1) / kPointsPerBlock);
    if (e == cudaSuccess) {
        if (prec == WAVE_FP32)
            e = launch<TAG_F32>(ndim, npts, blocks, p_old, p_new, v, a, b, factor,
                                            device_out, scr, st);
        else if (prec == WAVE_BF16 || prec == WAVE_BF16_F32ARITH)
            e = launch<TAG_BF16>(ndim, npts, blocks, p_old, p_new, v, a, b, factor,
                                            device_out, scr, st);
        else
            e = launch<TAG_F16>(ndim, npts, blocks, p_old, p_new, v, a, b, factor,
                                            device_out, scr, st);
    }
    if (e != cudaSuccess) {
        snprintf(g_static_err, sizeof g_static_err, "wave_energy_acoustic_static: %s",
                 cudaGetErrorString(e));
        set_error(g_static_err);
        return WAVE_ECUDA;
    }
    return WAVE_OK;
}
