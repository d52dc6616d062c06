// rk4_common.cuh -- device helpers shared by the RK4 kernel families.
#pragma once

#include <cstdint>
#include <type_traits>
#include <cuda_runtime.h>

namespace cho {

// Compensated state update x += (h6 + h6lo) k in FP32.  The state is carried
// as the unevaluated sum x + e (e holds what the rounded sum x has lost, as
// in Kahan summation).  The operations are the explicit round-to-nearest
// intrinsics, so the compiler neither fuses nor reorders them and every kernel
// that uses this sequence (packed or not) rounds identically.
__device__ __forceinline__ void comp_update(float& x, float& e, float k, float h6, float h6lo)
{
    float y = __fmaf_rn(h6lo, k, e);
    y = __fmaf_rn(h6, k, y);
    const float t = __fadd_rn(x, y);
    e = __fsub_rn(y, __fsub_rn(t, x));
    x = t;
}

// Compensated x += k in FP32 (the increment already scaled): the state is the
// unevaluated sum x + e, as in comp_update.
__device__ __forceinline__ void comp_add(float& x, float& e, float k)
{
    const float y = __fadd_rn(k, e);
    const float t = __fadd_rn(x, y);
    e = __fsub_rn(y, __fsub_rn(t, x));
    x = t;
}

// Compensated x += y in FP32 where y already holds the compensation e (the increment
// was summed onto e): the last two steps of comp_add.
__device__ __forceinline__ void comp_add_folded(float& x, float& e, float y)
{
    const float t = __fadd_rn(x, y);
    e = __fsub_rn(y, __fsub_rn(t, x));
    x = t;
}

// FP32 small systems integrate the scaled velocity u = (h/6) v (scaled_velocity,
// cho_internal.h) with the scaled iteration matrix B'' = (h^2/36) B, an FP32 pair
// formed from B's pair in FP64: then h/2 v = 3 u and h v = 6 u, and the state update
// adds the stage sums without a multiply.
__host__ __device__ __forceinline__ void scaled_coef(float& hi, float& lo, double h)
{
    const double b = ((double)hi + (double)lo) * (h * h / 36.0);
    hi = (float)b;
    lo = (float)(b - (double)hi);
}

// Fused multiply-add in the precision of the operands.
__device__ __forceinline__ double fmar(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float fmar(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double addr(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float addr(float a, float b) { return __fadd_rn(a, b); }

// Split an FP64 value into an unevaluated FP32 pair hi + lo.
__host__ __device__ __forceinline__ void split_ff(double d, float& hi, float& lo)
{
    hi = (float)d;
    lo = (float)(d - (double)hi);
}

// Per-instance step constants.  FP64: h, h/2, h/6.  FP32: h and h/2 rounded
// to FP32 (exact when h is an FP32 number), h/6 as the FP32 pair h6 + h6lo.
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
};

// State update of the RK4 step: x += h/6 k (FP64), compensated in FP32.
template <bool F64>
__device__ __forceinline__ void state_update(std::conditional_t<F64, double, float>& x, float& e,
                                             std::conditional_t<F64, double, float> k, const StepSize<F64>& hs)
{
    if constexpr (F64) {
        x = __fma_rn(hs.h6, k, x);
        (void)e;
    } else {
        comp_update(x, e, k, hs.h6, hs.h6lo);
    }
}

// ---- double-FP32 ("double-word") arithmetic -----------------------------------------
//
// GB300 runs FP64 at about 1/64 of the FP32 rate (a dependent FP64 FMA takes 64
// cycles), so FP64-class accuracy is cheaper as unevaluated pairs hi + lo of FP32
// numbers.  The pieces are the classical error-free transformations: Knuth's TwoSum,
// FastTwoSum (|a| >= |b|) and the FMA form of TwoProd (a b = p + e exactly with
// e = fma(a, b, -p)).  Sums use one TwoSum of the high parts plus the low parts
// ("sloppy" double-word addition: its error is a few units of 2^-48 of the larger
// operand); products use TwoProd of the high parts and the two cross terms.
struct dw {
    float hi, lo;
};

__device__ __forceinline__ dw dw_split(double d)
{
    const float h = (float)d;
    return {h, (float)(d - (double)h)};
}
__device__ __forceinline__ double dw_value(dw a) { return (double)a.hi + (double)a.lo; }
__device__ __forceinline__ dw fast_two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ dw two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}
__device__ __forceinline__ dw dw_add(dw x, dw y)
{
    const dw s = two_sum(x.hi, y.hi);
    return fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo)));
}
__device__ __forceinline__ dw dw_mul(dw x, dw y)
{
    const float p = __fmul_rn(x.hi, y.hi);
    float e = __fmaf_rn(x.hi, y.hi, -p);
    e = __fmaf_rn(x.hi, y.lo, e);
    e = __fmaf_rn(x.lo, y.hi, e);
    return fast_two_sum(p, e);
}
__device__ __forceinline__ dw dw_fma(dw a, dw b, dw c) { return dw_add(dw_mul(a, b), c); }
__device__ __forceinline__ dw dw_neg(dw a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ dw dw_twice(dw a) { return {2.f * a.hi, 2.f * a.lo}; }


// ---- thread-block clusters ------------------------------------------------------
__device__ __forceinline__ uint32_t cluster_rank()
{
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

// Address of the same shared-memory location in CTA `rank` of the cluster.
__device__ __forceinline__ uint32_t mapa(uint32_t addr, uint32_t rank)
{
    uint32_t out;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(out) : "r"(addr), "r"(rank));
    return out;
}

__device__ __forceinline__ void st_cluster_v4(uint32_t addr, uint4 v)
{
    asm volatile("st.shared::cluster.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(v.x), "r"(v.y), "r"(v.z), "r"(v.w)
                 : "memory");
}

__device__ __forceinline__ void st_cluster_f32(uint32_t addr, float v)
{
    asm volatile("st.shared::cluster.f32 [%0], %1;" ::"r"(addr), "f"(v) : "memory");
}

__device__ __forceinline__ void st_cluster_u32(uint32_t addr, uint32_t v)
{
    asm volatile("st.shared::cluster.u32 [%0], %1;" ::"r"(addr), "r"(v) : "memory");
}

// All threads of all CTAs of the cluster; shared-memory writes (local or remote)
// before it are visible to every thread after it.
__device__ __forceinline__ void cluster_sync()
{
    asm volatile("barrier.cluster.arrive.release.aligned;\nbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// ---- mbarriers with transaction counts (distributed shared memory transfers) ------
__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbarrier_init_one(uint64_t* bar)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"((uint32_t)__cvta_generic_to_shared(bar)) : "memory");
}

// The barrier's single arrival, expecting `bytes` of transfers for the current phase.
__device__ __forceinline__ void mbarrier_arm(uint64_t* bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(
                     (uint32_t)__cvta_generic_to_shared(bar)),
                 "r"(bytes)
                 : "memory");
}

// Wait for the phase of the given parity; false after about `limit_ns`.
__device__ __forceinline__ bool mbarrier_wait_bounded(uint64_t* bar, uint32_t parity, uint64_t limit_ns)
{
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(bar);
    const uint64_t t0 = global_ns();
    while (true) {
        uint32_t done;
        asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
                     : "=r"(done)
                     : "r"(a), "r"(parity)
                     : "memory");
        if (done) return true;
        if (global_ns() - t0 > limit_ns) return false;
    }
}

// 4-byte store into (possibly another CTA's) shared memory that completes 4 bytes on
// that CTA's mbarrier `bar` (both addresses from mapa).
__device__ __forceinline__ void st_async_f32(uint32_t addr, float v, uint32_t bar)
{
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.b32 [%0], %1, [%2];" ::"r"(addr),
                 "r"(__float_as_uint(v)), "r"(bar)
                 : "memory");
}

// Run f() n times with a 32-bit inner counter (64-bit compares cost extra
// instructions and a branch every step), the inner loop unrolled U times.
template <int U = 1, class F>
__device__ __forceinline__ void repeat_steps(int64_t n, F&& f)
{
    for (int64_t base = 0; base < n; base += 0x40000000LL) {
        const int32_t m = (int32_t)(n - base < 0x40000000LL ? n - base : 0x40000000LL);
#pragma unroll U
        for (int32_t i = 0; i < m; ++i) f();
    }
}

}  // namespace cho
