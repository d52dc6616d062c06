// rk4_common.cuh -- device helpers shared by the RK4 kernel families.
#pragma once

#include <cstdint>
#include <type_traits>
#include <cuda_runtime.h>

namespace cho {

// Kahan-compensated x += inc.  `c` carries the rounding error of the running
// sum with the sign convention "represented value = x - c".  The _rn
// intrinsics keep the compiler from contracting or reassociating the steps.
__device__ __forceinline__ void kahan_add(float& x, float& c, float inc)
{
    const float y = __fsub_rn(inc, c);
    const float t = __fadd_rn(x, y);
    c = __fsub_rn(__fsub_rn(t, x), y);
    x = t;
}

// Fused multiply-add in the precision of the operands.
__device__ __forceinline__ double fmar(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float fmar(float a, float b, float c) { return __fmaf_rn(a, b, c); }

// Split an FP64 value into an unevaluated FP32 pair hi + lo.
__host__ __device__ __forceinline__ void split_ff(double d, float& hi, float& lo)
{
    hi = (float)d;
    lo = (float)(d - (double)hi);
}

// Per-instance step constants.  FP64: h, h/2, h/6.  FP32: h and h/2 rounded
// to FP32 (exact when h is an FP32 number), h/6 as an FP32 pair.
template <bool F64>
struct StepSize {
    using Real = std::conditional_t<F64, double, float>;
    Real h, h2, h6;
    float h6lo;
    __device__ __forceinline__ explicit StepSize(double hd)
    {
        h = (Real)hd;
        h2 = (Real)(0.5 * hd);
        const double s6 = hd / 6.0;
        h6 = (Real)s6;
        h6lo = F64 ? 0.f : (float)(s6 - (double)(float)s6);
    }
    // increment h/6 * k for the state update
    __device__ __forceinline__ Real inc(Real k) const
    {
        if constexpr (F64) {
            return h6 * k;
        } else {
            return fmaf(h6, k, h6lo * k);
        }
    }
};

// State update of the RK4 step (both precisions).
template <bool F64>
__device__ __forceinline__ void state_add(std::conditional_t<F64, double, float>& x, float& c,
                                          std::conditional_t<F64, double, float> inc)
{
    if constexpr (F64) {
        x = x + inc;
        (void)c;
    } else {
        kahan_add(x, c, inc);
    }
}

}  // namespace cho
