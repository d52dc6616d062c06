// rk4_dense.cu -- classical RK4 for dense systems (eq. 1) whose instances share
// one (M, K), on the CUDA cores (FP64, or FP32 with FP32-pair coefficients).
//
// Each stage needs A = -B Xs for a tile of instances: a matrix product of the
// shared iteration matrix B = M^{-1}K (s x s) with the tile's stage
// displacements Xs (s x NT).  A CTA owns NT instances for the whole horizon.
// Thread (r, n) holds rows [r RI, r RI + RI) of instance n: its state, stage
// values and accumulators stay in registers.  Per stage the threads publish
// their stage displacements to shared memory (double-buffered, one barrier
// per stage), then each thread forms its RI rows of B Xs column by column.
// B (transposed, L2-resident) is streamed through shared memory in chunks of
// kJC columns with cp.async, double-buffered so that the copy of the next
// chunk overlaps the products of the current one; each thread reads its rows
// of a column with vector shared-memory loads.
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
constexpr int kJC = 8;               // columns of B^T per shared-memory chunk

__device__ __forceinline__ void cp_async16(void* dst, const void* src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// Batch form: FP64 x0/v0 in, FP64 outputs, shared step count, checkpoints.
template <bool F64>
struct DenseBatchSrc {
    BatchIO io;
    int s;
    using Real = std::conditional_t<F64, double, float>;
    __device__ int64_t count() const { return io.n_inst; }
    __device__ double h(int64_t q) const { return io.h[io.h_per_inst ? q : 0]; }
    __device__ int64_t steps(int64_t) const { return io.n_steps; }
    __device__ int64_t ckpt_every() const { return io.ckpt_every; }
    __device__ void load(int64_t q, int i, Real& x, Real& v, float& cx, float& cv) const
    {
        const double xd = io.x0[q * s + i];
        const double vd = io.v0[q * s + i];
        x = (Real)xd;
        v = (Real)vd;
        cx = F64 ? 0.f : (float)(xd - (double)x);
        cv = F64 ? 0.f : (float)(vd - (double)v);
    }
    __device__ void checkpoint(int64_t q, int64_t ck, int i, Real x, Real v, float cx, float cv) const
    {
        if (io.x_traj == nullptr) return;
        const int64_t o = (q * io.n_ck + ck) * s + i;
        io.x_traj[o] = (double)x + (double)cx;
        if (io.v_traj) io.v_traj[o] = (double)v + (double)cv;
    }
    __device__ void store(int64_t q, int i, Real x, Real v, float cx, float cv) const
    {
        io.x_out[q * s + i] = (double)x + (double)cx;
        io.v_out[q * s + i] = (double)v + (double)cv;
    }
    __device__ void finish(int64_t, int64_t, bool) const {}
};

// Slot form (serving): state block [x(s), v(s), cx(s), cv(s)] in kernel precision;
// each slot runs min(chunk, remaining) steps.
template <bool F64>
struct DenseSlotSrc {
    SlotIO io;
    int s;
    using Real = std::conditional_t<F64, double, float>;
    __device__ const SlotDesc& d(int64_t q) const { return io.slots[io.slot_ids[q]]; }
    __device__ int64_t count() const { return io.n_inst; }
    __device__ double h(int64_t q) const { return d(q).h; }
    __device__ int64_t steps(int64_t q) const { return d(q).remaining < io.chunk ? d(q).remaining : io.chunk; }
    __device__ int64_t ckpt_every() const { return 0; }
    __device__ void load(int64_t q, int i, Real& x, Real& v, float& cx, float& cv) const
    {
        const Real* st = (const Real*)d(q).state;
        x = st[i];
        v = st[s + i];
        if constexpr (F64) {
            cx = cv = 0.f;
        } else {
            cx = st[2 * s + i];
            cv = st[3 * s + i];
        }
    }
    __device__ void checkpoint(int64_t, int64_t, int, Real, Real, float, float) const {}
    __device__ void store(int64_t q, int i, Real x, Real v, float cx, float cv) const
    {
        Real* st = (Real*)d(q).state;
        st[i] = x;
        st[s + i] = v;
        if constexpr (!F64) {
            st[2 * s + i] = cx;
            st[3 * s + i] = cv;
        }
    }
    __device__ void finish(int64_t q, int64_t ran, bool bad) const
    {
        const int32_t slot = io.slot_ids[q];
        io.slots[slot].remaining -= ran;
        if (bad) io.status[slot] = CHO_ENONFINITE;
    }
};

template <int RI, int NT, bool F64, class Src>
__global__ void __launch_bounds__(kDenseThreads) rk4_dense_simt_kernel(DenseSys sys, const Src src)
{
    using Real = std::conditional_t<F64, double, float>;
    constexpr int RG = kDenseThreads / NT;          // row groups
    constexpr int SP = RG * RI;                     // padded size handled by this instantiation
    constexpr int NB = F64 ? 1 : 2;                 // B pieces: FP64, or FP32 hi and lo
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Real* xsh = (Real*)smem_raw;                    // [2][SP][NT]
    Real* bsh = xsh + 2 * SP * NT;                  // [2 buffers][NB][kJC][SP]
    __shared__ long long max_steps;
    __shared__ int any_bad[NT];

    const int t = threadIdx.x;
    const int n = t % NT;
    const int r = t / NT;
    const int row0 = r * RI;
    const int64_t q = (int64_t)blockIdx.x * NT + n;
    const bool live = q < src.count();
    const int s = sys.s;
    const Real* Bt = F64 ? (const Real*)sys.B64 : (const Real*)sys.B32;   // [SP][SP] = B^T (then lo, FP32)

    // every instance of the tile runs its own step count; the tile loops to the largest
    const int64_t my_steps = live ? src.steps(q) : 0;
    if (t == 0) max_steps = 0;
    if (t < NT) any_bad[t] = 0;
    __syncthreads();
    if (r == 0) atomicMax(&max_steps, (long long)my_steps);
    __syncthreads();
    const int64_t nsteps = max_steps;

    const StepSize<F64> hs(live ? src.h(q) : 1.0);
    Real x[RI], v[RI];
    float cx[RI], cv[RI];
#pragma unroll
    for (int k = 0; k < RI; ++k) {
        const int i = row0 + k;
        if (live && i < s) {
            src.load(q, i, x[k], v[k], cx[k], cv[k]);
        } else {
            x[k] = v[k] = 0;
            cx[k] = cv[k] = 0.f;
        }
    }

    // copy columns [c kJC, c kJC + kJC) of B^T (each piece) into chunk buffer b
    constexpr int CHUNK = kJC * SP;                 // elements per piece per chunk
    constexpr int VEC = 16 / sizeof(Real);
    const int n_chunks = (s + kJC - 1) / kJC;
    auto load_chunk = [&](int c, int b) {
#pragma unroll
        for (int pc = 0; pc < NB; ++pc) {
            const Real* src_c = Bt + (size_t)pc * SP * SP + (size_t)c * CHUNK;
            Real* dst = bsh + ((size_t)b * NB + pc) * CHUNK;
            for (int e = t * VEC; e < CHUNK; e += kDenseThreads * VEC) cp_async16(dst + e, src_c + e);
        }
        cp_async_commit();
    };

    int buf = 0;
    auto accel = [&](const Real (&xs)[RI], Real (&acc)[RI]) {
        Real* X = xsh + buf * SP * NT;
#pragma unroll
        for (int k = 0; k < RI; ++k) X[(row0 + k) * NT + n] = xs[k];
        Real t0[RI];
#pragma unroll
        for (int k = 0; k < RI; ++k) t0[k] = 0;
        load_chunk(0, 0);
        for (int c = 0; c < n_chunks; ++c) {
            if (c + 1 < n_chunks) {
                load_chunk(c + 1, (c + 1) & 1);
                cp_async_wait<1>();
            } else {
                cp_async_wait<0>();
            }
            __syncthreads();                         // chunk c (and, at c = 0, Xs) visible to all
            const Real* bh = bsh + (size_t)(c & 1) * NB * CHUNK;
            const int jn = s - c * kJC < kJC ? s - c * kJC : kJC;   // columns beyond s are zero
            for (int jj = 0; jj < jn; ++jj) {
                const Real xj = X[(c * kJC + jj) * NT + n];
                const Real* col = bh + jj * SP + row0;
                if constexpr (F64) {
#pragma unroll
                    for (int k = 0; k < RI; k += 2) {
                        const double2 b = *(const double2*)(col + k);
                        t0[k] = fmar(b.x, xj, t0[k]);
                        t0[k + 1] = fmar(b.y, xj, t0[k + 1]);
                    }
                } else {
                    const float* coll = col + CHUNK;
#pragma unroll
                    for (int k = 0; k < RI; k += 4) {
                        const float4 b_hi = *(const float4*)(col + k);
                        const float4 b_lo = *(const float4*)(coll + k);
                        t0[k] = fmaf(b_hi.x, xj, fmaf(b_lo.x, xj, t0[k]));
                        t0[k + 1] = fmaf(b_hi.y, xj, fmaf(b_lo.y, xj, t0[k + 1]));
                        t0[k + 2] = fmaf(b_hi.z, xj, fmaf(b_lo.z, xj, t0[k + 2]));
                        t0[k + 3] = fmaf(b_hi.w, xj, fmaf(b_lo.w, xj, t0[k + 3]));
                    }
                }
            }
            __syncthreads();                         // buffer c & 1 free for chunk c + 2
        }
#pragma unroll
        for (int k = 0; k < RI; ++k) acc[k] = -t0[k];
        buf ^= 1;
    };

    const int64_t every = src.ckpt_every() > 0 ? src.ckpt_every() : (nsteps > 0 ? nsteps : 1);
    int64_t ck = 0;
    int64_t step = 0;
    for (int64_t done = 0; done < nsteps; done += every) {
        for (int64_t it = 0; it < every; ++it, ++step) {
            Real a[RI], xs[RI], kx[RI], kv[RI], vs[RI];
            accel(x, a);
#pragma unroll
            for (int k = 0; k < RI; ++k) {
                kx[k] = v[k];
                kv[k] = a[k];
                xs[k] = fmar(hs.h2, v[k], x[k]);
                vs[k] = fmar(hs.h2, a[k], v[k]);
            }
            accel(xs, a);
#pragma unroll
            for (int k = 0; k < RI; ++k) {
                kx[k] = fmar((Real)2, vs[k], kx[k]);
                kv[k] = fmar((Real)2, a[k], kv[k]);
                xs[k] = fmar(hs.h2, vs[k], x[k]);
                vs[k] = fmar(hs.h2, a[k], v[k]);
            }
            accel(xs, a);
#pragma unroll
            for (int k = 0; k < RI; ++k) {
                kx[k] = fmar((Real)2, vs[k], kx[k]);
                kv[k] = fmar((Real)2, a[k], kv[k]);
                xs[k] = fmar(hs.h, vs[k], x[k]);
                vs[k] = fmar(hs.h, a[k], v[k]);
            }
            accel(xs, a);
            if (step < my_steps) {                   // instances past their horizon hold still
#pragma unroll
                for (int k = 0; k < RI; ++k) {
                    kx[k] = addr(kx[k], vs[k]);
                    kv[k] = addr(kv[k], a[k]);
                    state_update<F64>(x[k], cx[k], kx[k], hs);
                    state_update<F64>(v[k], cv[k], kv[k], hs);
                }
            }
        }
        if (src.ckpt_every() > 0) {
            if (live) {
#pragma unroll
                for (int k = 0; k < RI; ++k)
                    if (row0 + k < s) src.checkpoint(q, ck, row0 + k, x[k], v[k], cx[k], cv[k]);
            }
            ++ck;
        }
    }
    bool bad = false;
    if (live) {
#pragma unroll
        for (int k = 0; k < RI; ++k) {
            if (row0 + k < s) {
                src.store(q, row0 + k, x[k], v[k], cx[k], cv[k]);
                bad |= !(isfinite((double)x[k]) && isfinite((double)v[k]));
            }
        }
    }
    if (bad) any_bad[n] = 1;
    __syncthreads();
    if (live && r == 0) src.finish(q, my_steps, any_bad[n] != 0);
}

template <int RI, int NT, bool F64, class Src>
cudaError_t launch_simt(const DenseSys& sys, const Src& src, int64_t n_inst, cudaStream_t st)
{
    using Real = std::conditional_t<F64, double, float>;
    constexpr int SP = (kDenseThreads / NT) * RI;
    constexpr int NB = F64 ? 1 : 2;
    if (sys.s_pad != SP) return cudaErrorInvalidValue;
    const size_t smem = sizeof(Real) * (2 * (size_t)SP * NT + 2 * (size_t)NB * kJC * SP);
    auto kern = rk4_dense_simt_kernel<RI, NT, F64, Src>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int64_t blocks = (n_inst + NT - 1) / NT;
    if (blocks <= 0) return cudaSuccess;
    kern<<<(unsigned)blocks, kDenseThreads, smem, st>>>(sys, src);
    return cudaGetLastError();
}

template <template <bool> class SrcT, class Init>
cudaError_t dispatch_simt(const DenseSys& sys, bool fp64, int64_t n_inst, cudaStream_t st, const Init& init)
{
#define CHO_DENSE_CASE(SPV, RI64, NT64, RI32, NT32)                                                   \
    case SPV:                                                                                         \
        if (fp64) { SrcT<true> src; init(src); return launch_simt<RI64, NT64, true>(sys, src, n_inst, st); } \
        else { SrcT<false> src; init(src); return launch_simt<RI32, NT32, false>(sys, src, n_inst, st); }
    switch (sys.s_pad) {
        CHO_DENSE_CASE(64, 2, 8, 4, 16)
        CHO_DENSE_CASE(128, 4, 8, 8, 16)
        CHO_DENSE_CASE(256, 8, 8, 16, 16)
        CHO_DENSE_CASE(512, 8, 4, 16, 8)
        default: return cudaErrorInvalidValue;
    }
#undef CHO_DENSE_CASE
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
    return dispatch_simt<DenseBatchSrc>(sys, prec == CHO_FP64, io.n_inst, st, [&](auto& src) {
        src.io = io;
        src.s = sys.s;
    });
}

cudaError_t launch_rk4_dense_slots(const DenseSys& sys, const SlotIO& io, bool fp64, cudaStream_t st)
{
    if (io.n_inst == 0) return cudaSuccess;
    return dispatch_simt<DenseSlotSrc>(sys, fp64, io.n_inst, st, [&](auto& src) {
        src.io = io;
        src.s = sys.s;
    });
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
