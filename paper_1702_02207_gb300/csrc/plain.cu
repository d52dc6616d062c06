// plain.cu -- the plain (un-batched) form of RK4, kept as the baseline.
//
// One system at a time, one kernel launch per RK stage plus one for the
// update, FP64 throughout, with the state y = (x, v) and the four stage
// derivatives k1..k4 in device memory between launches:
//   stage j:  k_j = D(y + c_j h k_{j-1}),  c = (0, 1/2, 1/2, 1),  D(y) = (v, -B x)
//   update:   y += h/6 (k1 + 2 k2 + 2 k3 + k4)
// This is how a direct port of a per-equation CPU integrator looks on a GPU;
// the batched kernels are measured against it.
#include "cho_internal.h"

namespace cho {
namespace {

__device__ __forceinline__ double stage_x(const double* y, const double* kp, double c, int j)
{
    return kp ? y[j] + c * kp[j] : y[j];
}

__global__ void plain_stage_kernel(PlainSys sys, const double* __restrict__ y,
                                   const double* __restrict__ kprev, double c, double* __restrict__ kout)
{
    const int s = sys.s;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 2 * s) return;
    if (i < s) {                       // D(1), D(2): x' = v of the stage state
        kout[i] = kprev ? y[s + i] + c * kprev[s + i] : y[s + i];
        return;
    }
    const int r = i - s;               // D(3), D(4): v' = -(B x) of the stage state
    double a;
    if (sys.dense) {
        const double* B = sys.coef + (int64_t)r * s;
        a = 0.0;
        for (int j = 0; j < s; ++j) a = fma(B[j], stage_x(y, kprev, c, j), a);
    } else {
        const double* C = sys.coef;    // [3][s]: sub, main, super
        a = C[s + r] * stage_x(y, kprev, c, r);
        if (r > 0) a = fma(C[r], stage_x(y, kprev, c, r - 1), a);
        if (r + 1 < s) a = fma(C[2 * s + r], stage_x(y, kprev, c, r + 1), a);
    }
    kout[i] = -a;
}

__global__ void plain_update_kernel(int n, double* __restrict__ y, const double* __restrict__ k, double h6)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double* k1 = k;
    const double* k2 = k + n;
    const double* k3 = k + 2 * n;
    const double* k4 = k + 3 * n;
    y[i] = y[i] + h6 * (k1[i] + 2.0 * k2[i] + 2.0 * k3[i] + k4[i]);
}

}  // namespace

cudaError_t launch_plain_step(const PlainSys& sys, double* y, double* work, double h, cudaStream_t st)
{
    const int n = 2 * sys.s;
    const int threads = 128;
    const int blocks = (n + threads - 1) / threads;
    double* k = work;  // k1..k4, each n doubles
    const double c[4] = {0.0, 0.5 * h, 0.5 * h, h};
    for (int j = 0; j < 4; ++j) {
        plain_stage_kernel<<<blocks, threads, 0, st>>>(sys, y, j ? k + (j - 1) * n : nullptr, c[j], k + j * n);
    }
    plain_update_kernel<<<blocks, threads, 0, st>>>(n, y, k, h / 6.0);
    return cudaGetLastError();
}

}  // namespace cho
