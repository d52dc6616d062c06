// plain_common.cuh -- the per-element arithmetic of the plain form of RK4, shared
// by cho_integrate_plain (plain.cu) and cho_integrate_plain_noalloc
// (plain_noalloc.cu) so that both compute every value with the same operations.
//
//   stage j:  k_j = D(y + c_j k_{j-1}),  c = (0, h/2, h/2, h),  D(y) = (v, -B x)
//             (Section 3: D(1), D(2) are the velocity rows, D(3), D(4) the
//             acceleration rows of the first-order form)
//   update:   y += h/6 (k1 + 2 k2 + 2 k3 + k4)
#pragma once

#include "cho_internal.h"

namespace cho {

__device__ __forceinline__ double plain_stage_x(const double* y, const double* kp, double c, int j)
{
    return kp ? y[j] + c * kp[j] : y[j];
}

// Element i (0 <= i < 2 s) of stage k_j, with c the stage's multiple of h and kprev the
// previous stage (null for stage 1).
__device__ __forceinline__ double plain_stage_elem(const PlainSys& sys, const double* __restrict__ y,
                                                   const double* __restrict__ kprev, double c, int i)
{
    const int s = sys.s;
    if (i < s) return kprev ? y[s + i] + c * kprev[s + i] : y[s + i];   // D(1), D(2): x' = v
    const int r = i - s;                                                // D(3), D(4): v' = -(B x)
    double a;
    if (sys.dense) {
        const double* B = sys.coef + (int64_t)r * s;
        a = 0.0;
        for (int j = 0; j < s; ++j) a = fma(B[j], plain_stage_x(y, kprev, c, j), a);
    } else {
        const double* C = sys.coef;    // [3][s]: sub, main, super
        a = C[s + r] * plain_stage_x(y, kprev, c, r);
        if (r > 0) a = fma(C[r], plain_stage_x(y, kprev, c, r - 1), a);
        if (r + 1 < s) a = fma(C[2 * s + r], plain_stage_x(y, kprev, c, r + 1), a);
    }
    return -a;
}

// Element i of the update, k holding k1..k4 (n doubles each).
__device__ __forceinline__ double plain_update_elem(double yi, const double* __restrict__ k, int n, int i, double h6)
{
    return yi + h6 * (k[i] + 2.0 * k[n + i] + 2.0 * k[2 * n + i] + k[3 * n + i]);
}

}  // namespace cho
