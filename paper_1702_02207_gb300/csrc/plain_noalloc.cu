// plain_noalloc.cu -- the plain form of RK4 with no allocation at call time.
//
// Some callers must not allocate device memory once they are running: a
// real-time or hardware-in-the-loop simulation loop, for instance, where
// cudaMalloc may block on the device and add unbounded latency to a step with
// a deadline, or an application that hands all device memory to its own pool
// up front.  cho_integrate_plain keeps its state and stage buffers in a
// workspace that the context grows with cudaMalloc on demand;
// cho_integrate_plain_noalloc runs the same plain form with that scratch in a
// fixed array compiled into this file instead, and the step size read on the
// device, so the call itself allocates nothing (host or device).
//
// The scratch array is static device memory: every GPU that loads the library
// holds it until the process exits, and every call shares it, so calls whose
// work overlaps on the GPU (different streams, different threads) race on it.
// Each call overwrites all of the scratch it reads before reading it (the
// state from x0/v0, each stage buffer before the next stage uses it), so no
// part of it has to start at zero.
//
// The step size stays on the device (reading it on the host would need a
// synchronisation), so the host cannot reject a bad one.  The stage kernel
// checks it instead: an h that is not finite and > 0, or that puts the
// instance's fastest mode outside RK4's stability interval on the imaginary
// axis (omega_max h > 2 sqrt 2), makes every stage value NaN, and the call
// returns NaN states for that instance where cho_integrate_plain would return
// CHO_EINVAL or CHO_EUNSTABLE.
#include "../../include/cho.h"
#include "ctx.h"
#include "plain_common.cuh"

#include <mutex>

namespace cho {
namespace {

// State y = (x, v) and the four stage derivatives of one instance: 10 s doubles.
constexpr int kNoAllocMaxS = 4096;
static __device__ __align__(256) double g_plain_scratch[10 * kNoAllocMaxS];

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
double* g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch on the current device, looked up once per device
// (the host-side name of the array is not a device address).
cudaError_t scratch_ptr(int dev, double** out)
{
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_plain_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = (double*)p;
    }
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
}

// Stage j of the plain form for one instance, with c = factor * h and h read on the
// device; omega is the fastest angular frequency of the instance's parameter set.
__global__ void plain_stage_dh_kernel(PlainSys sys, const double* __restrict__ y, const double* __restrict__ kprev,
                                      double factor, const double* __restrict__ h, double omega,
                                      double* __restrict__ kout)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 2 * sys.s) return;
    const double hv = h[0];
    const bool h_ok = hv > 0.0 && hv < INFINITY && omega * hv <= 2.0 * 1.4142135623730951;
    kout[i] = h_ok ? plain_stage_elem(sys, y, kprev, factor * hv, i) : __longlong_as_double(0x7ff8000000000000ll);
}

__global__ void plain_update_dh_kernel(int n, double* __restrict__ y, const double* __restrict__ k,
                                       const double* __restrict__ h)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    y[i] = plain_update_elem(y[i], k, n, i, h[0] / 6.0);
}

}  // namespace
}  // namespace cho

using namespace cho;

extern "C" cho_status cho_integrate_plain_noalloc(cho_ctx* ctx, const cho_batch_desc* b, void* stream)
{
    clear_error();
    if (!ctx || !b || !b->system) return fail(CHO_EINVAL, "cho_integrate_plain_noalloc: NULL argument");
    cho_system_impl* sys = b->system;
    if (sys->ctx != ctx) return fail(CHO_EINVAL, "cho_integrate_plain_noalloc: system belongs to another context");
    if (b->mem != CHO_MEM_DEVICE)
        return fail(CHO_EINVAL, "cho_integrate_plain_noalloc: device pointers only (host arrays would need staging)");
    if (b->prec != CHO_FP64) return fail(CHO_EINVAL, "cho_integrate_plain_noalloc: the plain form is FP64 only");
    if (b->poly_jump != 0)
        return fail(CHO_EINVAL, "cho_integrate_plain_noalloc: the plain form runs RK4 stage by stage");
    if (sys->damped() || sys->forced())
        return fail(CHO_EINVAL, "cho_integrate_plain_noalloc: damped or forced systems run in the batch kernels");
    if (sys->s > kNoAllocMaxS)
        return fail(CHO_EINVAL, "cho_integrate_plain_noalloc: s = %d exceeds the fixed scratch limit of %d DOF",
                    sys->s, kNoAllocMaxS);
    if (b->n_inst < 0 || b->n_steps < 0) return fail(CHO_EINVAL, "cho_integrate_plain_noalloc: negative size");
    if (sys->n_sys != 1 && sys->n_sys != b->n_inst)
        return fail(CHO_EINVAL, "cho_integrate_plain_noalloc: parameter sets do not match n_inst");
    if (b->x_traj || b->v_traj || b->energy || b->ckpt_every != 0)
        return fail(CHO_EINVAL, "cho_integrate_plain_noalloc: no checkpoints in the plain form");
    if (b->n_inst > 0 && (!b->x0 || !b->v0 || !b->h || !b->x_out || !b->v_out))
        return fail(CHO_EINVAL, "cho_integrate_plain_noalloc: x0, v0, h, x_out and v_out are required");
    DeviceGuard g(ctx->device);
    if (!g.ok()) return fail(CHO_ECUDA, "cho_integrate_plain_noalloc: cudaSetDevice failed");
    double* work = nullptr;
    cudaError_t e = scratch_ptr(ctx->device, &work);
    if (e != cudaSuccess) return fail(CHO_ECUDA, "cho_integrate_plain_noalloc: cudaGetSymbolAddress: %s", cudaGetErrorString(e));
    cudaStream_t st = (cudaStream_t)stream;
    const int s = sys->s;
    const int n = 2 * s;
    const bool dense = sys->kind == CHO_DENSE;
    double* k = work;                    // k1..k4: 8 s doubles
    double* y = work + 8 * (size_t)s;    // state: 2 s doubles
    const int threads = 128, blocks = (n + threads - 1) / threads;
    const double factor[4] = {0.0, 0.5, 0.5, 1.0};
    for (int64_t q = 0; q < b->n_inst && e == cudaSuccess; ++q) {
        const int64_t set = sys->n_sys == 1 ? 0 : q;
        PlainSys ps{s, dense ? 1 : 0, sys->d_plain + set * (dense ? (int64_t)s * s : 3 * (int64_t)s)};
        const double* hq = b->h + (b->h_per_inst ? q : 0);
        const double omega = sys->omegas[(size_t)set];
        e = cudaMemcpyAsync(y, b->x0 + q * s, sizeof(double) * s, cudaMemcpyDeviceToDevice, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(y + s, b->v0 + q * s, sizeof(double) * s, cudaMemcpyDeviceToDevice, st);
        for (int64_t step = 0; step < b->n_steps && e == cudaSuccess; ++step) {
            for (int j = 0; j < 4; ++j)
                plain_stage_dh_kernel<<<blocks, threads, 0, st>>>(ps, y, j ? k + (j - 1) * n : nullptr, factor[j], hq,
                                                                  omega, k + j * n);
            plain_update_dh_kernel<<<blocks, threads, 0, st>>>(n, y, k, hq);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaMemcpyAsync(b->x_out + q * s, y, sizeof(double) * s, cudaMemcpyDeviceToDevice, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(b->v_out + q * s, y + s, sizeof(double) * s, cudaMemcpyDeviceToDevice, st);
    }
    if (e != cudaSuccess) return fail(CHO_ECUDA, "cho_integrate_plain_noalloc: %s", cudaGetErrorString(e));
    return CHO_OK;
}
