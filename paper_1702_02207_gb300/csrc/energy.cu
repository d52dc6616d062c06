// energy.cu -- FP64 mechanical energy of oscillator states (step a5).
//
// Eq. 1 with symmetric M and K conserves E = 1/2 v^T M v + 1/2 x^T K x.  For
// spring systems (eq. 2 and its chain generalisation) the same quantity is
// summed per element: kinetic 1/2 m_i v_i^2 and the potential 1/2 C_i e_i^2 of
// each spring, e_0 = x_0 (wall spring), e_i = x_i - x_{i-1}.  The drift of E
// over a run measures the integrator's dissipation (RK4 loses energy at a rate
// fixed by its stability polynomial).
#include "cho_internal.h"
#include "../../include/cho.h"

namespace cho {
namespace {

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// One warp per state.
__global__ void energy_springs_kernel(EnergySys sys, const double* __restrict__ x,
                                      const double* __restrict__ v, int64_t n_states, int64_t n_per,
                                      double* __restrict__ E)
{
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= n_states) return;
    const int s = sys.s;
    const int64_t set = sys.per_inst_sys ? w / n_per : 0;
    const double* m = sys.masses + set * s;
    const double* C = sys.springs + set * s;
    const double* xs = x + w * s;
    const double* vs = v + w * s;
    double acc = 0.0;
    for (int i = lane; i < s; i += 32) {
        const double e = i == 0 ? xs[0] : xs[i] - xs[i - 1];
        acc += 0.5 * m[i] * vs[i] * vs[i] + 0.5 * C[i] * e * e;
    }
    acc = warp_sum(acc);
    if (lane == 0) E[w] = acc;
}

// One block per state; x and v staged in shared memory.
__global__ void energy_dense_kernel(EnergySys sys, const double* __restrict__ x,
                                    const double* __restrict__ v, int64_t n_per, double* __restrict__ E)
{
    extern __shared__ double sh[];
    const int64_t w = blockIdx.x;
    const int s = sys.s;
    const int64_t set = sys.per_inst_sys ? w / n_per : 0;
    const double* M = sys.M + set * (int64_t)s * s;
    const double* K = sys.K + set * (int64_t)s * s;
    double* xs = sh;
    double* vs = sh + s;
    for (int i = threadIdx.x; i < s; i += blockDim.x) {
        xs[i] = x[w * s + i];
        vs[i] = v[w * s + i];
    }
    __syncthreads();
    double acc = 0.0;
    for (int i = threadIdx.x; i < s; i += blockDim.x) {
        double mv = 0.0, kx = 0.0;
        for (int j = 0; j < s; ++j) {
            mv = fma(M[(int64_t)i * s + j], vs[j], mv);
            kx = fma(K[(int64_t)i * s + j], xs[j], kx);
        }
        acc += 0.5 * (vs[i] * mv + xs[i] * kx);
    }
    acc = warp_sum(acc);
    __shared__ double part[32];
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        double p = threadIdx.x < (blockDim.x >> 5) ? part[threadIdx.x] : 0.0;
        p = warp_sum(p);
        if (threadIdx.x == 0) E[w] = p;
    }
}

}  // namespace

cudaError_t launch_energy(const EnergySys& sys, const double* x, const double* v, int64_t n_inst,
                          int64_t n_per, double* E, cudaStream_t st)
{
    const int64_t n_states = n_inst * n_per;
    if (n_states <= 0) return cudaSuccess;
    if (sys.kind == CHO_DENSE) {
        if (n_states > 0x7fffffffLL) return cudaErrorInvalidValue;
        const size_t smem = 2 * sizeof(double) * (size_t)sys.s;
        if (smem > 48 * 1024) return cudaErrorInvalidValue;
        energy_dense_kernel<<<(unsigned)n_states, 128, smem, st>>>(sys, x, v, n_per, E);
    } else {
        const int64_t blocks = (n_states * 32 + 255) / 256;
        if (blocks > 0x7fffffffLL) return cudaErrorInvalidValue;
        energy_springs_kernel<<<(unsigned)blocks, 256, 0, st>>>(sys, x, v, n_states, n_per, E);
    }
    return cudaGetLastError();
}

}  // namespace cho
