// serve_kernels.cu -- small device helpers of the serving loop.
#include "cho_internal.h"

namespace cho {
namespace {

__global__ void gather_status_kernel(const int32_t* __restrict__ ids, const int32_t* __restrict__ status,
                                     int32_t* __restrict__ out, int64_t n)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = status[ids[i]];
}

}  // namespace

// out[i] = status[ids[i]] for i < n: the per-slot status words of one launch's slots.
cudaError_t launch_gather_status(const int32_t* ids, const int32_t* status, int32_t* out, int64_t n,
                                 cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    const int64_t blocks = (n + 255) / 256;
    gather_status_kernel<<<(unsigned)blocks, 256, 0, st>>>(ids, status, out, n);
    return cudaGetLastError();
}

}  // namespace cho
