// rk4_dense.cu -- classical RK4 for dense systems (eq. 1) whose instances share
// one (M, K), on the CUDA cores (FP64, or FP32 with FP32-pair coefficients).
//
// Each stage needs A = -B Xs for a tile of instances: a matrix product of the
// shared iteration matrix B = M^{-1}K (s x s) with the tile's stage
// displacements Xs (s x NT).  A CTA owns NT instances for the whole horizon.
// Thread (r, n) holds rows [r RI, r RI + RI) of instance n: its state, stage
// values and accumulators stay in registers.  Per stage the threads publish
// their stage displacements to shared memory (double-buffered, one barrier
// per stage), then each thread forms its RI rows of B Xs column by column,
// reading B transposed from global memory (L1/L2 resident, four rows per
// vector load) and Xs from shared memory.
//
// The tensor-core split-BF16 variant lives in rk4_dense_tc.cu.
#include "cho_internal.h"
#include "ctx.h"
#include "rk4_common.cuh"

#include <cmath>
#include <vector>

namespace cho {
namespace {

constexpr int kDenseThreads = 256;

template <int RI, int NT, bool F64>
__global__ void __launch_bounds__(kDenseThreads) rk4_dense_simt_kernel(DenseSys sys, BatchIO io)
{
    using Real = std::conditional_t<F64, double, float>;
    constexpr int RG = kDenseThreads / NT;          // row groups
    constexpr int SP = RG * RI;                     // padded size handled by this instantiation
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Real* xsh = (Real*)smem_raw;                    // [2][SP][NT]

    const int t = threadIdx.x;
    const int n = t % NT;
    const int r = t / NT;
    const int row0 = r * RI;
    const int64_t q = (int64_t)blockIdx.x * NT + n;
    const bool live = q < io.n_inst;
    const int s = sys.s;
    const int ld = sys.s_pad;                       // leading dimension of the transposed B
    const Real* Bt = F64 ? (const Real*)sys.B64 : (const Real*)sys.B32;   // [SP][SP] = B^T
    const float* Btl = sys.B32 + (size_t)ld * ld;                          // lo part (FP32 only)

    const StepSize<F64> hs(live ? io.h[io.h_per_inst ? q : 0] : 1.0);
    Real x[RI], v[RI];
    float cx[RI], cv[RI];
#pragma unroll
    for (int k = 0; k < RI; ++k) {
        const int i = row0 + k;
        const double xd = (live && i < s) ? io.x0[q * s + i] : 0.0;
        const double vd = (live && i < s) ? io.v0[q * s + i] : 0.0;
        x[k] = (Real)xd;
        v[k] = (Real)vd;
        cx[k] = F64 ? 0.f : (float)((double)x[k] - xd);
        cv[k] = F64 ? 0.f : (float)((double)v[k] - vd);
    }

    int buf = 0;
    auto accel = [&](const Real (&xs)[RI], Real (&acc)[RI]) {
        Real* X = xsh + buf * SP * NT;
#pragma unroll
        for (int k = 0; k < RI; ++k) X[(row0 + k) * NT + n] = xs[k];
        __syncthreads();
        Real t0[RI];
#pragma unroll
        for (int k = 0; k < RI; ++k) t0[k] = 0;
        const int jmax = s;                          // columns beyond s are zero
        for (int j = 0; j < jmax; ++j) {
            const Real xj = X[j * NT + n];
            const Real* col = Bt + (size_t)j * ld + row0;
            if constexpr (F64) {
#pragma unroll
                for (int k = 0; k < RI; k += 2) {
                    const double2 b = __ldg((const double2*)(col + k));
                    t0[k] = fmar(b.x, xj, t0[k]);
                    t0[k + 1] = fmar(b.y, xj, t0[k + 1]);
                }
            } else {
                const float* coll = Btl + (size_t)j * ld + row0;
#pragma unroll
                for (int k = 0; k < RI; k += 4) {
                    const float4 bh = __ldg((const float4*)(col + k));
                    const float4 bl = __ldg((const float4*)(coll + k));
                    t0[k] = fmaf(bh.x, xj, fmaf(bl.x, xj, t0[k]));
                    t0[k + 1] = fmaf(bh.y, xj, fmaf(bl.y, xj, t0[k + 1]));
                    t0[k + 2] = fmaf(bh.z, xj, fmaf(bl.z, xj, t0[k + 2]));
                    t0[k + 3] = fmaf(bh.w, xj, fmaf(bl.w, xj, t0[k + 3]));
                }
            }
        }
#pragma unroll
        for (int k = 0; k < RI; ++k) acc[k] = -t0[k];
        buf ^= 1;
    };

    const int64_t nsteps = io.n_steps;
    const int64_t every = io.ckpt_every > 0 ? io.ckpt_every : (nsteps > 0 ? nsteps : 1);
    int64_t ck = 0;
    for (int64_t done = 0; done < nsteps; done += every) {
        for (int64_t it = 0; it < every; ++it) {
            Real a[RI], xs[RI], kx[RI], kv[RI], vs[RI];
            accel(x, a);
#pragma unroll
            for (int k = 0; k < RI; ++k) {
                kx[k] = v[k];
                kv[k] = a[k];
                xs[k] = x[k] + hs.h2 * v[k];
                vs[k] = v[k] + hs.h2 * a[k];
            }
            accel(xs, a);
#pragma unroll
            for (int k = 0; k < RI; ++k) {
                kx[k] = kx[k] + (Real)2 * vs[k];
                kv[k] = kv[k] + (Real)2 * a[k];
                xs[k] = x[k] + hs.h2 * vs[k];
                vs[k] = v[k] + hs.h2 * a[k];
            }
            accel(xs, a);
#pragma unroll
            for (int k = 0; k < RI; ++k) {
                kx[k] = kx[k] + (Real)2 * vs[k];
                kv[k] = kv[k] + (Real)2 * a[k];
                xs[k] = x[k] + hs.h * vs[k];
                vs[k] = v[k] + hs.h * a[k];
            }
            accel(xs, a);
#pragma unroll
            for (int k = 0; k < RI; ++k) {
                kx[k] = kx[k] + vs[k];
                kv[k] = kv[k] + a[k];
                state_add<F64>(x[k], cx[k], hs.inc(kx[k]));
                state_add<F64>(v[k], cv[k], hs.inc(kv[k]));
            }
        }
        if (io.ckpt_every > 0) {
            if (live && io.x_traj) {
#pragma unroll
                for (int k = 0; k < RI; ++k) {
                    const int i = row0 + k;
                    if (i < s) {
                        const int64_t o = (q * io.n_ck + ck) * s + i;
                        io.x_traj[o] = (double)x[k] - (double)cx[k];
                        if (io.v_traj) io.v_traj[o] = (double)v[k] - (double)cv[k];
                    }
                }
            }
            ++ck;
        }
    }
    if (live) {
#pragma unroll
        for (int k = 0; k < RI; ++k) {
            const int i = row0 + k;
            if (i < s) {
                io.x_out[q * s + i] = (double)x[k] - (double)cx[k];
                io.v_out[q * s + i] = (double)v[k] - (double)cv[k];
            }
        }
    }
}

template <int RI, int NT, bool F64>
cudaError_t launch_simt(const DenseSys& sys, const BatchIO& io, cudaStream_t st)
{
    using Real = std::conditional_t<F64, double, float>;
    constexpr int SP = (kDenseThreads / NT) * RI;
    if (sys.s_pad != SP) return cudaErrorInvalidValue;
    const size_t smem = 2 * sizeof(Real) * SP * NT;
    auto kern = rk4_dense_simt_kernel<RI, NT, F64>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int64_t blocks = (io.n_inst + NT - 1) / NT;
    if (blocks <= 0) return cudaSuccess;
    kern<<<(unsigned)blocks, kDenseThreads, smem, st>>>(sys, io);
    return cudaGetLastError();
}

}  // namespace

// s_pad: next power of two >= max(s, 64); the SIMT kernels cover s_pad <= 512.
int dense_pad(int s)
{
    int p = 64;
    while (p < s) p *= 2;
    return p;
}

cudaError_t launch_rk4_dense(const DenseSys& sys, const BatchIO& io, int prec, cudaStream_t st)
{
    if (io.n_inst == 0) return cudaSuccess;
    if (prec == CHO_DENSE_BF16X3 || prec == CHO_DENSE_BF16X5 || prec == CHO_DENSE_BF16X6)
        return launch_rk4_dense_tc(sys, io, prec, st);
    const bool fp64 = prec == CHO_FP64;
    switch (sys.s_pad) {
        case 64: return fp64 ? launch_simt<2, 8, true>(sys, io, st) : launch_simt<4, 16, false>(sys, io, st);
        case 128: return fp64 ? launch_simt<4, 8, true>(sys, io, st) : launch_simt<8, 16, false>(sys, io, st);
        case 256: return fp64 ? launch_simt<8, 8, true>(sys, io, st) : launch_simt<16, 16, false>(sys, io, st);
        case 512: return fp64 ? launch_simt<8, 4, true>(sys, io, st) : launch_simt<16, 8, false>(sys, io, st);
        default: return cudaErrorInvalidValue;
    }
}

// Device data of a dense system: B^T padded to s_pad in FP64 and as FP32 pairs
// (hi block then lo block), plus the BF16 pieces the tensor-core kernel reads.
cudaError_t build_dense_device(cho_system_impl* sys, const double* B)
{
    const int s = sys->s;
    const int sp = dense_pad(s);
    if (sp > 512) return cudaErrorInvalidValue;
    sys->s_pad = sp;
    const size_t n = (size_t)sp * sp;
    std::vector<double> Bt(n, 0.0);
    for (int i = 0; i < s; ++i)
        for (int j = 0; j < s; ++j) Bt[(size_t)j * sp + i] = B[(size_t)i * s + j];
    std::vector<float> B32(2 * n);
    for (size_t k = 0; k < n; ++k) split_ff(Bt[k], B32[k], B32[n + k]);
    cudaError_t e = cudaMalloc(&sys->d_B64, n * sizeof(double));
    if (e == cudaSuccess) e = cudaMemcpy(sys->d_B64, Bt.data(), n * sizeof(double), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc(&sys->d_B32, 2 * n * sizeof(float));
    if (e == cudaSuccess) e = cudaMemcpy(sys->d_B32, B32.data(), 2 * n * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = build_dense_tc_device(sys, B);
    return e;
}

}  // namespace cho
