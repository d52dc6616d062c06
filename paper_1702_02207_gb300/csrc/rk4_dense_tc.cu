// rk4_dense_tc.cu -- tensor-core (tcgen05) split-BF16 variant of rk4_dense.
#include "cho_internal.h"
#include "ctx.h"

namespace cho {

cudaError_t launch_rk4_dense_tc(const DenseSys&, const BatchIO&, int, cudaStream_t)
{
    return cudaErrorNotSupported;
}

cudaError_t build_dense_tc_device(cho_system_impl*, const double*) { return cudaSuccess; }

}  // namespace cho
