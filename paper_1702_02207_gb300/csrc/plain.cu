// plain.cu -- the plain (un-batched) form of RK4, kept as the baseline.
//
// One system at a time, one kernel launch per RK stage plus one for the
// update, FP64 throughout, with the state y = (x, v) and the four stage
// derivatives k1..k4 in device memory between launches:
//   stage j:  k_j = D(y + c_j h k_{j-1}),  c = (0, 1/2, 1/2, 1),  D(y) = (v, -B x)
//   update:   y += h/6 (k1 + 2 k2 + 2 k3 + k4)
// This is how a direct port of a per-equation CPU integrator looks on a GPU;
// the batched kernels are measured against it.
#include "plain_common.cuh"

namespace cho {
namespace {

__global__ void plain_stage_kernel(PlainSys sys, const double* __restrict__ y,
                                   const double* __restrict__ kprev, double c, double* __restrict__ kout)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 2 * sys.s) return;
    kout[i] = plain_stage_elem(sys, y, kprev, c, i);
}

__global__ void plain_update_kernel(int n, double* __restrict__ y, const double* __restrict__ k, double h6)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    y[i] = plain_update_elem(y[i], k, n, i, h6);
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
