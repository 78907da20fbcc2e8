// Plan-free l2-ball projection (Sec. 3.2, functions g_l; Algorithm 2 steps
// 10-12) whose scratch is a fixed file-scope device array, so a call performs
// no device allocation of any kind.
//
// Scratch layout (doubles): [0, L * nb) per-CTA partial sums of ||z - y||^2,
// nb CTAs per channel; [L * nb, L * nb + L) the per-channel scale factors.
// Every slot is written by this call before it is read, so nothing has to
// start at zero. The array is shared by all calls in the process on a device:
// two calls whose executions overlap (different streams or host threads)
// race on it and give wrong results.
//
// Set-up: the first call on a device (with that device current) resolves the
// array's device address with cudaGetSymbolAddress, which may load this
// library's device code, and caches it per device together with the unique
// id of the CUDA context it belongs to; make that first call before any stream
// capture that is meant to contain these launches. A call that finds a
// different context current on the device (after cudaDeviceReset, or a
// context destroyed and created again) resolves the address again, so a
// cached address never outlives its context.
#include <cuda.h>

#include <mutex>

#include "hs_device.cuh"
#include "hs_internal.h"
#include "hypersara.h"

namespace hs {

constexpr int STATIC_MAX_DEVICES = 64;
constexpr int BALL_CTAS_PER_CHANNEL = 32;

static __device__ __align__(256) double g_ball_scratch[HS_L2BALL_STATIC_DOUBLES];

static std::mutex g_scratch_mu;
static double* g_scratch_ptr[STATIC_MAX_DEVICES] = {};
static unsigned long long g_scratch_ctx[STATIC_MAX_DEVICES] = {};

// Unique id of the calling thread's current CUDA context (0 when none is
// current). The two driver functions are looked up through the runtime, so
// the library has no link-time dependency on the driver library.
static hs_status current_context_id(unsigned long long* id) {
    using get_current_t = CUresult (*)(CUcontext*);
    using get_id_t = CUresult (*)(CUcontext, unsigned long long*);
    static get_current_t get_current = nullptr;
    static get_id_t get_id = nullptr;
    if (!get_current || !get_id) {
        void* f0 = nullptr;
        void* f1 = nullptr;
        cudaDriverEntryPointQueryResult q0, q1;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f0, 12000, cudaEnableDefault, &q0) != cudaSuccess ||
            cudaGetDriverEntryPointByVersion("cuCtxGetId", &f1, 12000, cudaEnableDefault, &q1) != cudaSuccess ||
            q0 != cudaDriverEntryPointSuccess || q1 != cudaDriverEntryPointSuccess || !f0 || !f1)
            return fail(HS_ERR_CUDA, "hs_proj_l2ball_static: driver context queries unavailable");
        get_current = reinterpret_cast<get_current_t>(f0);
        get_id = reinterpret_cast<get_id_t>(f1);
    }
    CUcontext ctx = nullptr;
    *id = 0;
    if (get_current(&ctx) != CUDA_SUCCESS)
        return fail(HS_ERR_CUDA, "hs_proj_l2ball_static: cuCtxGetCurrent failed");
    if (ctx && get_id(ctx, id) != CUDA_SUCCESS)
        return fail(HS_ERR_CUDA, "hs_proj_l2ball_static: cuCtxGetId failed");
    return HS_OK;
}

static hs_status static_scratch(double** out) {
    int dev = -1;
    HS_CHECK_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= STATIC_MAX_DEVICES)
        return fail(HS_ERR_ARG, "hs_proj_l2ball_static: device %d beyond the supported %d", dev,
                    STATIC_MAX_DEVICES);
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    unsigned long long ctx = 0;
    HS_TRY(current_context_id(&ctx));
    if (g_scratch_ptr[dev] == nullptr || ctx == 0 || ctx != g_scratch_ctx[dev]) {
        void* ptr = nullptr;
        const cudaError_t rc = cudaGetSymbolAddress(&ptr, g_ball_scratch);
        if (rc != cudaSuccess || ptr == nullptr)
            return fail(HS_ERR_CUDA, "hs_proj_l2ball_static: cudaGetSymbolAddress: %s", cudaGetErrorString(rc));
        HS_TRY(current_context_id(&ctx));   // the lookup above makes the device's context current
        g_scratch_ptr[dev] = static_cast<double*>(ptr);
        g_scratch_ctx[dev] = ctx;
    }
    *out = g_scratch_ptr[dev];
    return HS_OK;
}

// Partial ||z - y||^2 of channel l over a grid-stride sweep of its range.
template <typename R>
__global__ void __launch_bounds__(256) k_sball_norm(const Cx<R>* __restrict__ Z, const Cx<R>* __restrict__ Y,
                                                   const int64_t* __restrict__ off, int nb,
                                                   double* __restrict__ part) {
    __shared__ double red[32];
    const int l = blockIdx.y;
    const int64_t end = off[l + 1];
    double s = 0.0;
    for (int64_t i = off[l] + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < end;
         i += (int64_t)nb * blockDim.x) {
        const Cx<R> d = csub(Z[i], Y[i]);
        s += (double)d.x * d.x + (double)d.y * d.y;
    }
    s = block_sum(s, red);
    if (threadIdx.x == 0) part[(int64_t)l * nb + blockIdx.x] = s;
}

// rho_l = sqrt(sum of the channel's partials); scale_l = max(0, 1 - eps_l / rho_l).
__global__ void __launch_bounds__(32) k_sball_scale(const double* __restrict__ part, int nb,
                                                   const double* __restrict__ eps, double* __restrict__ rho,
                                                   double* __restrict__ scale) {
    const int l = blockIdx.x;
    double s = 0.0;
    for (int b = threadIdx.x; b < nb; b += 32) s += part[(int64_t)l * nb + b];
    s = warp_sum(s);
    if (threadIdx.x == 0) {
        const double r = sqrt(s);
        if (rho) rho[l] = r;
        const double e = eps[l];
        scale[l] = (r > e) ? (1.0 - e / r) : 0.0;
    }
}

// Z and out may be the same buffer (in-place projection), so neither is
// declared __restrict__; each thread reads z before writing the same index.
template <typename R>
__global__ void __launch_bounds__(256) k_sball_apply(const Cx<R>* Z, const Cx<R>* __restrict__ Y,
                                                    const int64_t* __restrict__ off, int L,
                                                    const double* __restrict__ scale, int dual,
                                                    Cx<R>* out) {
    const int l = blockIdx.y;
    const int64_t end = off[l + 1];
    const R sc = (R)scale[l];
    for (int64_t i = off[l] + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < end;
         i += (int64_t)gridDim.x * blockDim.x) {
        const Cx<R> z = Z[i];
        const Cx<R> r = cscale(csub(z, Y[i]), sc);   // z - P_B(z)
        out[i] = dual ? r : csub(z, r);
    }
}

template <typename R>
static hs_status sball(int L, const int64_t* off, const void* Z, const void* Yd, const double* eps, int dual,
                       void* out, double* rho_out, double* scratch, cudaStream_t s) {
    const int nb = std::min(BALL_CTAS_PER_CHANNEL, (HS_L2BALL_STATIC_DOUBLES - L) / L);
    double* part = scratch;
    double* scale = scratch + (int64_t)L * nb;
    k_sball_norm<R><<<dim3(nb, L), 256, 0, s>>>((const Cx<R>*)Z, (const Cx<R>*)Yd, off, nb, part);
    HS_CHECK_LAUNCH();
    k_sball_scale<<<L, 32, 0, s>>>(part, nb, eps, rho_out, scale);
    HS_CHECK_LAUNCH();
    k_sball_apply<R><<<dim3(nb, L), 256, 0, s>>>((const Cx<R>*)Z, (const Cx<R>*)Yd, off, L, scale, dual,
                                                 (Cx<R>*)out);
    HS_CHECK_LAUNCH();
    return HS_OK;
}

}  // namespace hs

using namespace hs;

extern "C" hs_status hs_proj_l2ball_static(int L, const int64_t* vis_offsets, const void* Z, const void* Yd,
                                           const double* eps, hs_prec prec, int dual, void* out,
                                           double* rho_out, void* stream) {
    clear_error();
    if (L < 1 || L > HS_L2BALL_STATIC_MAX_L)
        return fail(HS_ERR_ARG, "hs_proj_l2ball_static: L = %d outside [1, %d]", L, HS_L2BALL_STATIC_MAX_L);
    if (prec != HS_F32 && prec != HS_F64) return fail(HS_ERR_ARG, "hs_proj_l2ball_static: bad precision");
    if (dual != 0 && dual != 1) return fail(HS_ERR_ARG, "hs_proj_l2ball_static: dual must be 0 or 1");
    if (!vis_offsets || !Z || !Yd || !eps || !out) return fail(HS_ERR_ARG, "hs_proj_l2ball_static: null buffer");
    double* scratch = nullptr;
    HS_TRY(static_scratch(&scratch));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (prec == HS_F32) return sball<float>(L, vis_offsets, Z, Yd, eps, dual, out, rho_out, scratch, s);
    return sball<double>(L, vis_offsets, Z, Yd, eps, dual, out, rho_out, scratch, s);
}
