// rk4_dense.cu -- classical RK4 for dense systems (eq. 1) on the CUDA cores
// (FP64, or FP32 with FP32-pair coefficients), for instances that share one
// (M, K) or that each have their own.
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
// One (M, K) per instance, FP64: the same kernel with one instance per CTA (NT = 1)
// and the CTA's own B^T streamed through the chunk buffers (read from L2 or HBM
// every stage, so this form is bound by memory bandwidth).  In FP32, instances with
// their own (M, K), and batches of few instances, run on rk4_dense_own_kernel
// (s_pad = 64: one CTA per instance, B held in registers and shared memory) or
// rk4_dense_split_kernel (s_pad >= 128: one CTA or cluster of CTAs per instance,
// B's rows split over it); every FP32 kernel here forms the products in the same
// order, so the choice between them never changes a result's bits.
//
// The tensor-core split-BF16 variants live in rk4_dense_tc.cu.
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
    __device__ void timed_out(int64_t) const {}     // reported through the system's error word
    // B^T (FP64) or its FP32 pair of instance q's parameter set
    __device__ const void* bt(const DenseSys& sys, int64_t q) const
    {
        const int64_t set = sys.per_inst ? q : 0;
        const size_t n = (size_t)sys.s_pad * sys.s_pad;
        if constexpr (F64) return sys.B64 + (size_t)set * n;
        else return sys.B32 + (size_t)set * 2 * n;
    }
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
    __device__ void timed_out(int64_t q) const { io.status[io.slot_ids[q]] = CHO_ETIMEOUT; }
    // the slot's coefficient block (its parameter set's B^T) or the shared one
    __device__ const void* bt(const DenseSys& sys, int64_t q) const
    {
        if (q < io.n_inst && d(q).coef) return d(q).coef;
        if constexpr (F64) return sys.B64;
        else return sys.B32;
    }
};

// acc[k] += col[k] * xj for k < RI, reading col with the widest vector loads that
// RI allows (col is aligned to RI elements: rows are split in blocks of RI).
template <int RI, class Real>
__device__ __forceinline__ void col_fma(const Real* col, Real xj, Real (&acc)[RI])
{
    if constexpr (sizeof(Real) == 8 && RI % 2 == 0) {
#pragma unroll
        for (int k = 0; k < RI; k += 2) {
            const double2 b = *(const double2*)(col + k);
            acc[k] = fmar(b.x, xj, acc[k]);
            acc[k + 1] = fmar(b.y, xj, acc[k + 1]);
        }
    } else if constexpr (sizeof(Real) == 4 && RI % 4 == 0) {
#pragma unroll
        for (int k = 0; k < RI; k += 4) {
            const float4 b = *(const float4*)(col + k);
            acc[k] = fmar(b.x, xj, acc[k]);
            acc[k + 1] = fmar(b.y, xj, acc[k + 1]);
            acc[k + 2] = fmar(b.z, xj, acc[k + 2]);
            acc[k + 3] = fmar(b.w, xj, acc[k + 3]);
        }
    } else if constexpr (sizeof(Real) == 4 && RI % 2 == 0) {
#pragma unroll
        for (int k = 0; k < RI; k += 2) {
            const float2 b = *(const float2*)(col + k);
            acc[k] = fmar(b.x, xj, acc[k]);
            acc[k + 1] = fmar(b.y, xj, acc[k + 1]);
        }
    } else {
#pragma unroll
        for (int k = 0; k < RI; ++k) acc[k] = fmar(col[k], xj, acc[k]);
    }
}

template <int RI, int NT, bool F64, class Src, int NTHR = kDenseThreads>
__global__ void __launch_bounds__(NTHR) rk4_dense_simt_kernel(DenseSys sys, const Src src)
{
    using Real = std::conditional_t<F64, double, float>;
    constexpr int RG = NTHR / NT;                   // row groups
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
    // [SP][SP] = B^T (then lo, FP32): shared, or the CTA's own instance (NT = 1)
    const Real* Bt = (const Real*)src.bt(sys, (int64_t)blockIdx.x * NT);

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

    // copy columns [c kJC, c kJC + kJC) of B^T (np pieces) into chunk buffer b
    constexpr int CHUNK = kJC * SP;                 // elements per piece per chunk
    constexpr int VEC = 16 / sizeof(Real);
    const int n_chunks = (s + kJC - 1) / kJC;
    auto load_chunk = [&](int c, int b, int np) {
        for (int pc = 0; pc < np; ++pc) {
            const Real* src_c = Bt + (size_t)pc * SP * SP + (size_t)c * CHUNK;
            Real* dst = bsh + ((size_t)b * NB + pc) * CHUNK;
            for (int e = t * VEC; e < CHUNK; e += NTHR * VEC) cp_async16(dst + e, src_c + e);
        }
        cp_async_commit();
    };

    int buf = 0;
    // FP32: B = hi + lo.  The lo product is formed at stage 1 only, in its own
    // accumulator, and reused by stages 2-4 ("frozen lo", as rk4_small.cu): those
    // stages stream and multiply the hi piece alone.  Both products are summed in
    // blocks of kJC columns (a partial per block, the partials added in column
    // order): every FP32 dense kernel (streaming, resident, cluster-split) keeps
    // this order, so all of them give the same bits for the same instance.
    Real lo1[RI];
    auto accel = [&](const Real (&xs)[RI], Real (&acc)[RI], bool first) {
        Real* X = xsh + buf * SP * NT;
#pragma unroll
        for (int k = 0; k < RI; ++k) X[(row0 + k) * NT + n] = xs[k];
        Real t0[RI];
#pragma unroll
        for (int k = 0; k < RI; ++k) {
            t0[k] = 0;
            if (first) lo1[k] = 0;
        }
        const int np = (!F64 && first) ? 2 : 1;
        load_chunk(0, 0, np);
        for (int c = 0; c < n_chunks; ++c) {
            if (c + 1 < n_chunks) {
                load_chunk(c + 1, (c + 1) & 1, np);
                cp_async_wait<1>();
            } else {
                cp_async_wait<0>();
            }
            __syncthreads();                         // chunk c (and, at c = 0, Xs) visible to all
            const Real* bh = bsh + (size_t)(c & 1) * NB * CHUNK;
            const int jn = s - c * kJC < kJC ? s - c * kJC : kJC;   // columns beyond s are zero
            // blocked summation: the chunk's kJC terms go into a partial sum that is then
            // added to the total, so the rounding error grows with kJC + s / kJC, not with s
            Real part[RI], lpart[RI];
#pragma unroll
            for (int k = 0; k < RI; ++k) part[k] = lpart[k] = 0;
            for (int jj = 0; jj < jn; ++jj) {
                const Real xj = X[(c * kJC + jj) * NT + n];
                const Real* col = bh + jj * SP + row0;
                col_fma(col, xj, part);
                if constexpr (!F64) {
                    if (first) col_fma(col + CHUNK, xj, lpart);
                }
            }
#pragma unroll
            for (int k = 0; k < RI; ++k) {
                t0[k] = addr(t0[k], part[k]);
                if (!F64 && first) lo1[k] = addr(lo1[k], lpart[k]);
            }
            __syncthreads();                         // buffer c & 1 free for chunk c + 2
        }
#pragma unroll
        for (int k = 0; k < RI; ++k) acc[k] = F64 ? -t0[k] : -addr(t0[k], lo1[k]);
        buf ^= 1;
    };

    const int64_t every = src.ckpt_every() > 0 ? src.ckpt_every() : (nsteps > 0 ? nsteps : 1);
    int64_t ck = 0;
    int64_t step = 0;
    for (int64_t done = 0; done < nsteps; done += every) {
        for (int64_t it = 0; it < every; ++it, ++step) {
            Real a[RI], xs[RI], kx[RI], kv[RI], vs[RI];
            accel(x, a, true);
#pragma unroll
            for (int k = 0; k < RI; ++k) {
                kx[k] = v[k];
                kv[k] = a[k];
                xs[k] = fmar(hs.h2, v[k], x[k]);
                vs[k] = fmar(hs.h2, a[k], v[k]);
            }
            accel(xs, a, false);
#pragma unroll
            for (int k = 0; k < RI; ++k) {
                kx[k] = fmar((Real)2, vs[k], kx[k]);
                kv[k] = fmar((Real)2, a[k], kv[k]);
                xs[k] = fmar(hs.h2, vs[k], x[k]);
                vs[k] = fmar(hs.h2, a[k], v[k]);
            }
            accel(xs, a, false);
#pragma unroll
            for (int k = 0; k < RI; ++k) {
                kx[k] = fmar((Real)2, vs[k], kx[k]);
                kv[k] = fmar((Real)2, a[k], kv[k]);
                xs[k] = fmar(hs.h, vs[k], x[k]);
                vs[k] = fmar(hs.h, a[k], v[k]);
            }
            accel(xs, a, false);
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

// One instance per CTA, s_pad = 64, FP32 (systems with one (M, K) per instance, or a
// few instances of a shared one): thread = 1 row, the thread's row of B's hi piece
// in 64 registers for the whole horizon and the lo piece (used at stage 1) in shared
// memory, row-major with each row padded by 16 bytes (the eight threads of a
// shared-memory phase fall in distinct banks).  Streaming B from shared memory
// instead needed 4 bytes of it per FMA, which held the FMA pipe near a quarter of
// its rate.  The products keep the streaming kernel's order (blocks of kJC columns
// into partials added in column order; the lo piece at stage 1 alone), so both give
// the same bits.
template <class Src>
__global__ void __launch_bounds__(64) rk4_dense_own_kernel(DenseSys sys, const Src src)
{
    using Real = float;
    constexpr bool F64 = false;
    constexpr int SP = 64;
    constexpr int LD = SP + 4;                      // padded row length
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float* Bs = (float*)smem_raw;                   // [SP][LD]: lo piece of B, row-major
    float* X = Bs + (size_t)SP * LD;                // [2][SP]
    __shared__ int any_bad;

    const int t = threadIdx.x;
    const int64_t q = blockIdx.x;
    const int s = sys.s;
    const int64_t my_steps = src.steps(q);
    if (t == 0) any_bad = 0;
    float breg[SP];
    {
        const float* Bt = (const float*)src.bt(sys, q);   // [2][SP][SP] = B^T (hi, lo)
#pragma unroll
        for (int j = 0; j < SP; ++j) breg[j] = Bt[(size_t)j * SP + t];       // hi row t, coalesced
        for (int e = t; e < SP * SP; e += SP) {
            const int j = e / SP, i = e % SP;
            Bs[(size_t)i * LD + j] = Bt[(size_t)SP * SP + e];              // lo piece
        }
    }
    const StepSize<false> hs(src.h(q));
    float x = 0.f, v = 0.f, cx = 0.f, cv = 0.f;
    if (t < s) src.load(q, t, x, v, cx, cv);
    __syncthreads();

    const float* brow_lo = Bs + (size_t)t * LD;
    int buf = 0;
    float lo1 = 0.f;
    auto accel = [&](float xs, bool first) -> float {
        float* Xb = X + buf * SP;
        Xb[t] = xs;
        __syncthreads();
        float acc = 0.f;
        if (first) lo1 = 0.f;
        // every block full: columns beyond s hold zeros in B and X (adds of +0)
#pragma unroll
        for (int c = 0; c < SP / kJC; ++c) {
            float part = 0.f, lpart = 0.f;
#pragma unroll
            for (int jj = 0; jj < kJC; jj += 4) {
                const int j = c * kJC + jj;
                const float4 xx = *(const float4*)(Xb + j);
                part = fmar(breg[j], xx.x, part);
                part = fmar(breg[j + 1], xx.y, part);
                part = fmar(breg[j + 2], xx.z, part);
                part = fmar(breg[j + 3], xx.w, part);
                if (first) {
                    const float4 bl = *(const float4*)(brow_lo + j);
                    lpart = fmar(bl.x, xx.x, lpart);
                    lpart = fmar(bl.y, xx.y, lpart);
                    lpart = fmar(bl.z, xx.z, lpart);
                    lpart = fmar(bl.w, xx.w, lpart);
                }
            }
            acc = addr(acc, part);
            if (first) lo1 = addr(lo1, lpart);
        }
        buf ^= 1;
        return -addr(acc, lo1);
    };

    // the block's step count: every instance is alone in its CTA
    const int64_t nsteps = my_steps;
    const int64_t every = src.ckpt_every() > 0 ? src.ckpt_every() : (nsteps > 0 ? nsteps : 1);
    int64_t ck = 0;
    for (int64_t done = 0; done < nsteps; done += every) {
        for (int64_t it = 0; it < every; ++it) {
            Real a, xs, kx, kv, vs;
            a = accel(x, true);
            kx = v;
            kv = a;
            xs = fmar(hs.h2, v, x);
            vs = fmar(hs.h2, a, v);
            a = accel(xs, false);
            kx = fmar((Real)2, vs, kx);
            kv = fmar((Real)2, a, kv);
            xs = fmar(hs.h2, vs, x);
            vs = fmar(hs.h2, a, v);
            a = accel(xs, false);
            kx = fmar((Real)2, vs, kx);
            kv = fmar((Real)2, a, kv);
            xs = fmar(hs.h, vs, x);
            vs = fmar(hs.h, a, v);
            a = accel(xs, false);
            kx = addr(kx, vs);
            kv = addr(kv, a);
            state_update<F64>(x, cx, kx, hs);
            state_update<F64>(v, cv, kv, hs);
        }
        if (src.ckpt_every() > 0) {
            if (t < s) src.checkpoint(q, ck, t, x, v, cx, cv);
            ++ck;
        }
    }
    bool bad = false;
    if (t < s) {
        src.store(q, t, x, v, cx, cv);
        bad = !(isfinite((double)x) && isfinite((double)v));
    }
    if (bad) any_bad = 1;
    __syncthreads();
    if (t == 0) src.finish(q, my_steps, any_bad != 0);
}

// ---- one instance spread over a cluster of CTAs (FP32, s_pad >= 128) ---------------
//
// With few instances (a serving request, a periodic real-time task) the kernels
// above run each instance's stages one after the other on one SM while the other
// SMs idle.  Here one instance spans a cluster of CS CTAs, each owning R = s_pad / CS
// rows of B: the hi piece of its rows in registers (CPT consecutive blocks of kJC
// columns per thread), the lo piece (stage 1 only) in shared memory.  For x'' = -B x
// the displacement of stage 3, x + h/2 v2, needs only stage 1's product and that of
// stage 4, x + h v3, only stage 2's, so the kernel forms the products of two stages
// per round (stages 1 and 2, then 3 and 4): every CTA forms the block partials of
// its rows for both displacements (a thread per row and block range, B read once
// for the two), the owner thread of each row adds them in column order, completes
// the row's stage values and sends the round's next two displacements to every CTA's
// copy of Xs (st.async into distributed shared memory, double-buffered); each CTA
// waits on its own mbarrier until the round's 2 s_pad values have arrived.  Two
// exchanges per step instead of four.  This is the paper's decomposition of one
// system's RK4 step over parallel workers with a synchronisation between stages
// (Section 3), at the scale of a cluster of SMs.  The block partials and their
// order, and every stage value, are those of the other FP32 dense kernels, so an
// instance gets the same bits whichever of them runs it.  (A cluster barrier per
// stage, whose release waits for the remote stores to be acknowledged before the
// barrier itself, cost about 60 % of the warps' time.)
template <int SP, int R, int NTHR, class Src>
__global__ void __launch_bounds__(NTHR, NTHR >= 512 ? 1 : 2) rk4_dense_split_kernel(DenseSys sys, const Src src)
{
    constexpr int CS = SP / R;                      // CTAs per cluster
    constexpr int NCH = SP / kJC;                   // column blocks
    constexpr int NRG = R / 32;                     // row groups (a warp's lanes are 32 rows)
    constexpr int WPG = (NTHR / 32) / NRG;          // warps per row group
    constexpr int CPT = NCH / WPG;                  // consecutive column blocks per thread
    constexpr int LD = SP + 4;                      // padded row of the lo piece
    constexpr int PLD = NCH + 4;                    // padded row of the partials
    static_assert(R % 32 == 0 && (NTHR / 32) % NRG == 0 && NCH % WPG == 0 && R <= NTHR, "split shape");
    static_assert(CPT % 4 == 0 && NCH % 4 == 0, "partials move as float4");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float* Lo = (float*)smem_raw;                   // [R][LD]: lo piece of this CTA's rows
    float* X = Lo + (size_t)R * LD;                 // [2 rounds][2 displacements][SP], all rows
    float* Ph = X + 4 * SP;                         // [2][R][PLD]: block partials of the two displacements
    float* Pl = Ph + 2 * (size_t)R * PLD;           // [R][PLD]: block partials, lo piece (stage 1)
    __shared__ int any_bad;
    __shared__ __align__(8) uint64_t xbar[2];       // Xs buffer set b complete (clusters)

    const int t = threadIdx.x;
    const int lane = t & 31, w = t >> 5;
    const int lr = (w % NRG) * 32 + lane;           // local row of this thread's partials
    const int c0 = (w / NRG) * CPT;                 // its blocks: c0 .. c0 + CPT - 1
    const uint32_t rank = CS > 1 ? cluster_rank() : 0;
    const int64_t q = blockIdx.x / CS;
    const int s = sys.s;
    // blocks at or past column s hold zero partials; a warp whose blocks all lie
    // there never forms them (its partials keep the zeros written below)
    const bool active = c0 * kJC < s;
    const bool owner = t < R;                       // thread t < R owns local row t (its lr is t)
    const int i = (int)rank * R + t;                // the owner's global row

    const float* Bt = (const float*)src.bt(sys, q);   // [2][SP][SP]: B^T hi, then lo
    float bh[CPT][kJC];
#pragma unroll
    for (int k = 0; k < CPT; ++k)
#pragma unroll
        for (int jj = 0; jj < kJC; ++jj) bh[k][jj] = Bt[(size_t)((c0 + k) * kJC + jj) * SP + (int)rank * R + lr];
    for (int e = t; e < R * SP; e += NTHR) {
        const int j = e / R, r = e % R;             // B^T[j][rank R + r], coalesced over r
        Lo[(size_t)r * LD + j] = Bt[(size_t)SP * SP + (size_t)j * SP + (int)rank * R + r];
    }
    for (int e = t; e < 3 * R * PLD; e += NTHR) Ph[e] = 0.f;   // Ph (both) and Pl
    const int64_t my_steps = src.steps(q);
    const StepSize<false> hs(src.h(q));
    float x = 0.f, v = 0.f, cx = 0.f, cv = 0.f;
    if (owner && i < s) src.load(q, i, x, v, cx, cv);
    if (t == 0) {
        any_bad = 0;
        if constexpr (CS > 1) {
            mbarrier_init_one(&xbar[0]);
            mbarrier_init_one(&xbar[1]);
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
            mbarrier_arm(&xbar[0], 8u * SP);        // each round brings two displacements of s_pad rows
            mbarrier_arm(&xbar[1], 8u * SP);
        }
    }
    // the owner's row of Xs (set 0, first displacement) and the sets' mbarriers; mapa
    // gives their addresses in each CTA of the cluster
    const uint32_t xloc = (uint32_t)__cvta_generic_to_shared(X) + 4u * (uint32_t)(owner ? i : 0);
    const uint32_t bloc = (uint32_t)__cvta_generic_to_shared(&xbar[0]);
    uint32_t xphase[2] = {0u, 0u};
    bool ok = true;
    // every CTA of the cluster is running and has initialised its shared memory
    if (CS > 1) cluster_sync(); else __syncthreads();

    int set = 0;
    float lo1 = 0.f;
    // One round: aa = -(B xa), ab = -(B xb) for this thread's row (owners); the first
    // round of a step also forms the lo product of xa (= x), reused by every stage.
    auto round = [&](float xa, float xb, bool first, float& aa, float& ab) {
        if (owner) {
            const uint32_t off = (uint32_t)(set * 2 * SP * 4);
            if constexpr (CS > 1) {
#pragma unroll
                for (int c = 0; c < CS; ++c) {
                    const uint32_t bar = mapa(bloc + 8u * (uint32_t)set, (uint32_t)c);
                    st_async_f32(mapa(xloc + off, (uint32_t)c), xa, bar);
                    st_async_f32(mapa(xloc + off + 4u * SP, (uint32_t)c), xb, bar);
                }
            } else {
                X[set * 2 * SP + i] = xa;
                X[(set * 2 + 1) * SP + i] = xb;
            }
        }
        if constexpr (CS > 1) {
            // both displacements of every row have arrived (bounded wait, agreed by the CTA)
            ok = __syncthreads_and(mbarrier_wait_bounded(&xbar[set], xphase[set], 1000000000ull));
            if (!ok) {
                aa = ab = 0.f;
                return;
            }
            xphase[set] ^= 1u;
            // the set's next use is two rounds on; its data can only be sent after this
            // CTA's next round of values, so arming it here precedes every transfer
            if (t == 0) mbarrier_arm(&xbar[set], 8u * SP);
        } else {
            __syncthreads();
        }
        if (active) {
            const float* Xa = X + set * 2 * SP + c0 * kJC;
            const float* Xb = Xa + SP;
            const float* lrow = Lo + (size_t)lr * LD + c0 * kJC;
            // each block's columns in order, for both displacements; four blocks at a time
#pragma unroll
            for (int k4 = 0; k4 < CPT; k4 += 4) {
                float pa[4], pb[4], pl[4];
#pragma unroll
                for (int kk = 0; kk < 4; ++kk) {
                    const int k = k4 + kk;
                    const float4 a0 = *(const float4*)(Xa + k * kJC);
                    const float4 a1 = *(const float4*)(Xa + k * kJC + 4);
                    const float4 b0 = *(const float4*)(Xb + k * kJC);
                    const float4 b1 = *(const float4*)(Xb + k * kJC + 4);
                    float u = 0.f, z = 0.f;
                    u = fmar(bh[k][0], a0.x, u);
                    z = fmar(bh[k][0], b0.x, z);
                    u = fmar(bh[k][1], a0.y, u);
                    z = fmar(bh[k][1], b0.y, z);
                    u = fmar(bh[k][2], a0.z, u);
                    z = fmar(bh[k][2], b0.z, z);
                    u = fmar(bh[k][3], a0.w, u);
                    z = fmar(bh[k][3], b0.w, z);
                    u = fmar(bh[k][4], a1.x, u);
                    z = fmar(bh[k][4], b1.x, z);
                    u = fmar(bh[k][5], a1.y, u);
                    z = fmar(bh[k][5], b1.y, z);
                    u = fmar(bh[k][6], a1.z, u);
                    z = fmar(bh[k][6], b1.z, z);
                    u = fmar(bh[k][7], a1.w, u);
                    z = fmar(bh[k][7], b1.w, z);
                    pa[kk] = u;
                    pb[kk] = z;
                    if (first) {
                        const float4 l0 = *(const float4*)(lrow + k * kJC);
                        const float4 l1 = *(const float4*)(lrow + k * kJC + 4);
                        float y = 0.f;
                        y = fmar(l0.x, a0.x, y);
                        y = fmar(l0.y, a0.y, y);
                        y = fmar(l0.z, a0.z, y);
                        y = fmar(l0.w, a0.w, y);
                        y = fmar(l1.x, a1.x, y);
                        y = fmar(l1.y, a1.y, y);
                        y = fmar(l1.z, a1.z, y);
                        y = fmar(l1.w, a1.w, y);
                        pl[kk] = y;
                    }
                }
                *(float4*)(Ph + (size_t)lr * PLD + c0 + k4) = make_float4(pa[0], pa[1], pa[2], pa[3]);
                *(float4*)(Ph + ((size_t)R + lr) * PLD + c0 + k4) = make_float4(pb[0], pb[1], pb[2], pb[3]);
                if (first) *(float4*)(Pl + (size_t)lr * PLD + c0 + k4) = make_float4(pl[0], pl[1], pl[2], pl[3]);
            }
        }
        __syncthreads();
        if (owner) {
            // all NCH blocks in column order (the zero ones leave the sums unchanged)
            float ta = 0.f, tb = 0.f, l = 0.f;
#pragma unroll
            for (int c = 0; c < NCH; c += 4) {
                const float4 ua = *(const float4*)(Ph + (size_t)t * PLD + c);
                const float4 ub = *(const float4*)(Ph + ((size_t)R + t) * PLD + c);
                ta = addr(addr(addr(addr(ta, ua.x), ua.y), ua.z), ua.w);
                tb = addr(addr(addr(addr(tb, ub.x), ub.y), ub.z), ub.w);
                if (first) {
                    const float4 ul = *(const float4*)(Pl + (size_t)t * PLD + c);
                    l = addr(addr(addr(addr(l, ul.x), ul.y), ul.z), ul.w);
                }
            }
            if (first) lo1 = l;
            aa = -addr(ta, lo1);
            ab = -addr(tb, lo1);
        }
        set ^= 1;
    };

    const int64_t every = src.ckpt_every() > 0 ? src.ckpt_every() : (my_steps > 0 ? my_steps : 1);
    int64_t ck = 0;
    for (int64_t done = 0; done < my_steps && ok; done += every) {
        for (int64_t it = 0; it < every && ok; ++it) {
            // stages 1 and 2: x and x2 = x + h/2 v
            float a1 = 0.f, a2 = 0.f, a3 = 0.f, a4 = 0.f;
            const float x2 = fmar(hs.h2, v, x);
            round(x, x2, true, a1, a2);
            if (!ok) break;
            float kx = v, kv = a1;
            const float v2 = fmar(hs.h2, a1, v);
            kx = fmar(2.f, v2, kx);
            kv = fmar(2.f, a2, kv);
            const float x3 = fmar(hs.h2, v2, x);
            const float v3 = fmar(hs.h2, a2, v);
            const float x4 = fmar(hs.h, v3, x);
            // stages 3 and 4: x3 = x + h/2 v2 and x4 = x + h v3
            round(x3, x4, false, a3, a4);
            if (!ok) break;
            kx = fmar(2.f, v3, kx);
            kv = fmar(2.f, a3, kv);
            const float v4 = fmar(hs.h, a3, v);
            kx = addr(kx, v4);
            kv = addr(kv, a4);
            state_update<false>(x, cx, kx, hs);
            state_update<false>(v, cv, kv, hs);
        }
        if (src.ckpt_every() > 0 && ok) {
            if (owner && i < s) src.checkpoint(q, ck, i, x, v, cx, cv);
            ++ck;
        }
    }
    // a wait that gave up: the peers give up on this CTA's values in turn; all meet
    // at the cluster barrier below, after which no transfer is in flight
    if (!ok && t == 0 && sys.err) atomicExch(sys.err, 1);
    bool bad = false;
    if (owner && i < s) {
        src.store(q, i, x, v, cx, cv);
        bad = !(isfinite(x) && isfinite(v));
    }
    if (bad) {
        if constexpr (CS > 1) st_cluster_u32(mapa((uint32_t)__cvta_generic_to_shared(&any_bad), 0u), 1u);
        else any_bad = 1;
    }
    if (CS > 1) cluster_sync(); else __syncthreads();
    if (!ok && t == 0) src.timed_out(q);
    if (rank == 0 && t == 0) src.finish(q, ok ? my_steps : 0, any_bad != 0);
}

// Shapes of the split kernel: s_pad 128 -> one CTA of 256 threads (two per SM),
// 256 -> 2 CTAs and 512 -> 8 CTAs of 512 threads; every thread holds 64 hi values.
template <int SP> struct SplitShape;
template <> struct SplitShape<128> { static constexpr int R = 128, NTHR = 256; };
template <> struct SplitShape<256> { static constexpr int R = 128, NTHR = 512; };
template <> struct SplitShape<512> { static constexpr int R = 64, NTHR = 512; };

template <int SP>
size_t split_smem()
{
    constexpr int R = SplitShape<SP>::R;
    return sizeof(float) * ((size_t)R * (SP + 4) + 4 * (size_t)SP + 3 * (size_t)R * (SP / kJC + 4));
}

template <int SP, class Src>
cudaLaunchConfig_t split_config(int64_t n_inst, cudaStream_t st, cudaLaunchAttribute* attr)
{
    constexpr int CS = SP / SplitShape<SP>::R;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(n_inst * CS), 1, 1);
    cfg.blockDim = dim3(SplitShape<SP>::NTHR, 1, 1);
    cfg.dynamicSmemBytes = split_smem<SP>();
    cfg.stream = st;
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = CS;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cfg;
}

// How many clusters of the split kernel are resident at once on this device (asked
// once per device and shape; 0 if none fits, and its callers keep the other kernels).
template <int SP, class Src>
int split_capacity()
{
    static int known[64];                           // cluster count + 1; 0 unknown
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
    if (known[dev] == 0) {
        auto kern = rk4_dense_split_kernel<SP, SplitShape<SP>::R, SplitShape<SP>::NTHR, Src>;
        int n = 0;
        cudaLaunchAttribute attr[1];
        const cudaLaunchConfig_t cfg = split_config<SP, Src>(1, nullptr, attr);
        bool ok = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)split_smem<SP>()) ==
                  cudaSuccess;
        ok = ok && cudaOccupancyMaxActiveClusters(&n, kern, &cfg) == cudaSuccess;
        if (!ok) {
            (void)cudaGetLastError();
            n = 0;
        }
        known[dev] = n + 1;
    }
    return known[dev] - 1;
}

template <int SP, class Src>
cudaError_t launch_split(const DenseSys& sys, const Src& src, int64_t n_inst, cudaStream_t st)
{
    constexpr int CS = SP / SplitShape<SP>::R;
    if (sys.s_pad != SP) return cudaErrorInvalidValue;
    if (n_inst <= 0) return cudaSuccess;
    if (n_inst > 0x7fffffffLL / CS) return cudaErrorInvalidValue;
    auto kern = rk4_dense_split_kernel<SP, SplitShape<SP>::R, SplitShape<SP>::NTHR, Src>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)split_smem<SP>());
    if (e != cudaSuccess) return e;
    cudaLaunchAttribute attr[1];
    const cudaLaunchConfig_t cfg = split_config<SP, Src>(n_inst, st, attr);
    return cudaLaunchKernelEx(&cfg, kern, sys, src);
}

int device_sm_count()
{
    static int known[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 1;
    if (known[dev] == 0) {
        int n = 0;
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 1;
        known[dev] = n;
    }
    return known[dev];
}

template <class Src>
cudaError_t launch_own(const DenseSys& sys, const Src& src, int64_t n_inst, cudaStream_t st)
{
    constexpr int SP = 64;
    if (sys.s_pad != SP) return cudaErrorInvalidValue;
    const size_t smem = sizeof(float) * ((size_t)SP * (SP + 4) + 2 * (size_t)SP);
    auto kern = rk4_dense_own_kernel<Src>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if (n_inst <= 0) return cudaSuccess;
    if (n_inst > 0x7fffffffLL) return cudaErrorInvalidValue;
    kern<<<(unsigned)n_inst, SP, smem, st>>>(sys, src);
    return cudaGetLastError();
}

template <int RI, int NT, bool F64, class Src, int NTHR = kDenseThreads>
cudaError_t launch_simt(const DenseSys& sys, const Src& src, int64_t n_inst, cudaStream_t st)
{
    using Real = std::conditional_t<F64, double, float>;
    constexpr int SP = (NTHR / NT) * RI;
    constexpr int NB = F64 ? 1 : 2;
    if (sys.s_pad != SP) return cudaErrorInvalidValue;
    const size_t smem = sizeof(Real) * (2 * (size_t)SP * NT + 2 * (size_t)NB * kJC * SP);
    auto kern = rk4_dense_simt_kernel<RI, NT, F64, Src, NTHR>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int64_t blocks = (n_inst + NT - 1) / NT;
    if (blocks <= 0) return cudaSuccess;
    kern<<<(unsigned)blocks, NTHR, smem, st>>>(sys, src);
    return cudaGetLastError();
}

template <template <bool> class SrcT, class Init>
cudaError_t dispatch_simt(const DenseSys& sys, bool fp64, int64_t n_inst, cudaStream_t st, const Init& init)
{
#define CHO_DENSE_CASE(SPV, RI64, NT64, RI32, NT32)                                                   \
    case SPV:                                                                                         \
        if (fp64) { SrcT<true> src; init(src); return launch_simt<RI64, NT64, true>(sys, src, n_inst, st); } \
        else { SrcT<false> src; init(src); return launch_simt<RI32, NT32, false>(sys, src, n_inst, st); }
#define CHO_DENSE_OWN_CASE(SPV, RI)                                                                   \
    case SPV:                                                                                         \
        if (fp64) { SrcT<true> src; init(src); return launch_simt<RI, 1, true, SrcT<true>, SPV / RI>(sys, src, n_inst, st); } \
        else { SrcT<false> src; init(src); return launch_simt<RI, 1, false, SrcT<false>, SPV / RI>(sys, src, n_inst, st); }
    // FP32 with one (M, K) per instance, or few instances of a shared one (up to eight
    // waves of what fits at once): one instance per CTA (s_pad = 64, B resident) or per
    // cluster (larger s, B split over the cluster).  All FP32 kernels give the same bits,
    // so the choice may follow the instance count.
    if (!fp64) {
        SrcT<false> src;
        init(src);
        int cap = 0;
        switch (sys.s_pad) {
            case 64: cap = device_sm_count(); break;
            case 128: cap = split_capacity<128, SrcT<false>>(); break;
            case 256: cap = split_capacity<256, SrcT<false>>(); break;
            case 512: cap = split_capacity<512, SrcT<false>>(); break;
            default: return cudaErrorInvalidValue;
        }
        const bool few = sys.few == 1 || (sys.few < 0 && (sys.per_inst || n_inst <= 8 * (int64_t)cap));
        if (cap > 0 && few) {
            switch (sys.s_pad) {
                case 64: return launch_own(sys, src, n_inst, st);
                case 128: return launch_split<128>(sys, src, n_inst, st);
                case 256: return launch_split<256>(sys, src, n_inst, st);
                default: return launch_split<512>(sys, src, n_inst, st);
            }
        }
    }
    if (sys.per_inst) {                             // one instance (and its own B) per CTA, streamed
        switch (sys.s_pad) {
            CHO_DENSE_OWN_CASE(64, 1)
            CHO_DENSE_OWN_CASE(128, 2)
            CHO_DENSE_OWN_CASE(256, 4)
            CHO_DENSE_OWN_CASE(512, 8)
            default: return cudaErrorInvalidValue;
        }
    }
    switch (sys.s_pad) {
        CHO_DENSE_CASE(64, 2, 8, 4, 16)
        CHO_DENSE_CASE(128, 4, 8, 8, 16)
        CHO_DENSE_CASE(256, 8, 8, 16, 16)
        CHO_DENSE_CASE(512, 8, 4, 16, 8)
        default: return cudaErrorInvalidValue;
    }
#undef CHO_DENSE_CASE
#undef CHO_DENSE_OWN_CASE
}

// ---- polynomial form with k-step jumps (one shared (M, K), one shared h) ------------
//
// For y = (x, v), one RK4 step is y <- P y with P = [[C, H], [G, C]] (blocks
// polynomials in B; see rk4_jump_blocks), and k steps are P^k = [[C_k, H_k], [G_k, C_k]].
// With E_xx = C_k - I, E_xv = H_k, E_vx = G_k formed in FP64 on the host, a jump is
//     x <- x + E_xx x + E_xv v,    v <- v + E_vx x + E_xx v,
// four products of s x s matrices with the tile's x and v per k steps, against
// four B-products per step for the stage form.  Same tiling as rk4_dense_simt:
// the three matrices (transposed; FP32 as hi/lo pairs) are streamed through
// shared memory in chunks of kJP columns; x and v of the tile are published
// once per jump; the state update is compensated in FP32.
constexpr int kJP = 4;

template <int RI, int NT, bool F64>
__global__ void __launch_bounds__(kDenseThreads) rk4_dense_poly_kernel(DenseSys sys, const void* Ev, BatchIO io)
{
    using Real = std::conditional_t<F64, double, float>;
    constexpr int RG = kDenseThreads / NT;
    constexpr int SP = RG * RI;
    constexpr int NB = F64 ? 1 : 2;
    constexpr int NPC = 3 * NB;                     // pieces: E_xx, E_xv, E_vx (hi, lo)
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Real* xv = (Real*)smem_raw;                     // [2 buffers][x | v][SP][NT]
    Real* csh = xv + 4 * SP * NT;                   // [2 buffers][NPC][kJP][SP]

    const int t = threadIdx.x;
    const int n = t % NT;
    const int r = t / NT;
    const int row0 = r * RI;
    const int64_t q = (int64_t)blockIdx.x * NT + n;
    const bool live = q < io.n_inst;
    const int s = sys.s;
    const Real* E = (const Real*)Ev;               // [NPC][SP][SP]

    Real x[RI], v[RI];
    float cx[RI], cv[RI];
#pragma unroll
    for (int k = 0; k < RI; ++k) {
        const int i = row0 + k;
        x[k] = v[k] = 0;
        cx[k] = cv[k] = 0.f;
        if (live && i < s) {
            const double xd = io.x0[q * s + i], vd = io.v0[q * s + i];
            x[k] = (Real)xd;
            v[k] = (Real)vd;
            if constexpr (!F64) {
                cx[k] = (float)(xd - (double)x[k]);
                cv[k] = (float)(vd - (double)v[k]);
            }
        }
    }

    constexpr int CHUNK = kJP * SP;
    constexpr int VEC = 16 / sizeof(Real);
    const int n_chunks = (s + kJP - 1) / kJP;
    auto load_chunk = [&](int c, int b) {
#pragma unroll
        for (int pc = 0; pc < NPC; ++pc) {
            const Real* src_c = E + (size_t)pc * SP * SP + (size_t)c * CHUNK;
            Real* dst = csh + ((size_t)b * NPC + pc) * CHUNK;
            for (int e = t * VEC; e < CHUNK; e += kDenseThreads * VEC) cp_async16(dst + e, src_c + e);
        }
        cp_async_commit();
    };
    int buf = 0;
    auto jump = [&]() {
        Real* X = xv + (size_t)buf * 2 * SP * NT;
        Real* V = X + SP * NT;
#pragma unroll
        for (int k = 0; k < RI; ++k) {
            X[(row0 + k) * NT + n] = x[k];
            V[(row0 + k) * NT + n] = v[k];
        }
        Real zx[RI], zv[RI];
#pragma unroll
        for (int k = 0; k < RI; ++k) zx[k] = zv[k] = 0;
        load_chunk(0, 0);
        for (int c = 0; c < n_chunks; ++c) {
            if (c + 1 < n_chunks) {
                load_chunk(c + 1, (c + 1) & 1);
                cp_async_wait<1>();
            } else {
                cp_async_wait<0>();
            }
            __syncthreads();                         // chunk c (and, at c = 0, x and v) visible to all
            const Real* ch = csh + (size_t)(c & 1) * NPC * CHUNK;
            const int jn = s - c * kJP < kJP ? s - c * kJP : kJP;
            // blocked summation: each chunk's 4 kJP terms per output go into a partial sum
            // that is then added to the total (the rounding error of the 4 s-term sums grows
            // with the chunk length plus the number of chunks, not with 4 s)
            Real px[RI], pv[RI];
#pragma unroll
            for (int k = 0; k < RI; ++k) px[k] = pv[k] = 0;
            for (int jj = 0; jj < jn; ++jj) {
                const int j = c * kJP + jj;
                const Real xj = X[j * NT + n], vj = V[j * NT + n];
                const Real* exx = ch + (0 * NB) * CHUNK + jj * SP + row0;
                const Real* exv = ch + (1 * NB) * CHUNK + jj * SP + row0;
                const Real* evx = ch + (2 * NB) * CHUNK + jj * SP + row0;
                if constexpr (!F64) {                // lo pieces first
                    col_fma(exx + CHUNK, xj, px);
                    col_fma(exv + CHUNK, vj, px);
                    col_fma(evx + CHUNK, xj, pv);
                    col_fma(exx + CHUNK, vj, pv);
                }
                col_fma(exx, xj, px);
                col_fma(exv, vj, px);
                col_fma(evx, xj, pv);
                col_fma(exx, vj, pv);
            }
#pragma unroll
            for (int k = 0; k < RI; ++k) {
                zx[k] = addr(zx[k], px[k]);
                zv[k] = addr(zv[k], pv[k]);
            }
            __syncthreads();                         // buffer c & 1 free for chunk c + 2
        }
#pragma unroll
        for (int k = 0; k < RI; ++k) {
            if constexpr (F64) {
                x[k] = addr(x[k], zx[k]);
                v[k] = addr(v[k], zv[k]);
            } else {
                const float yx = addr(zx[k], cx[k]), tx = addr(x[k], yx);
                cx[k] = __fsub_rn(yx, __fsub_rn(tx, x[k]));
                x[k] = tx;
                const float yv = addr(zv[k], cv[k]), tv = addr(v[k], yv);
                cv[k] = __fsub_rn(yv, __fsub_rn(tv, v[k]));
                v[k] = tv;
            }
        }
        buf ^= 1;
    };

    const int64_t kj = io.poly_jump;
    const int64_t jumps = io.n_steps / kj;
    const int64_t per_ck = io.ckpt_every > 0 && io.x_traj ? io.ckpt_every / kj : (jumps > 0 ? jumps : 1);
    int64_t ck = 0;
    for (int64_t done = 0; done < jumps; done += per_ck) {
        for (int64_t it = 0; it < per_ck; ++it) jump();
        if (io.ckpt_every > 0 && io.x_traj && live) {
#pragma unroll
            for (int k = 0; k < RI; ++k) {
                const int i = row0 + k;
                if (i >= s) continue;
                const int64_t o = (q * io.n_ck + ck) * s + i;
                io.x_traj[o] = (double)x[k] + (double)cx[k];
                if (io.v_traj) io.v_traj[o] = (double)v[k] + (double)cv[k];
            }
        }
        ++ck;
    }
    if (live) {
#pragma unroll
        for (int k = 0; k < RI; ++k) {
            const int i = row0 + k;
            if (i >= s) continue;
            io.x_out[q * s + i] = (double)x[k] + (double)cx[k];
            io.v_out[q * s + i] = (double)v[k] + (double)cv[k];
        }
    }
}

template <int RI, int NT, bool F64>
cudaError_t launch_poly(const DenseSys& sys, const void* E, const BatchIO& io, cudaStream_t st)
{
    using Real = std::conditional_t<F64, double, float>;
    constexpr int SP = (kDenseThreads / NT) * RI;
    constexpr int NPC = 3 * (F64 ? 1 : 2);
    if (sys.s_pad != SP) return cudaErrorInvalidValue;
    const size_t smem = sizeof(Real) * (4 * (size_t)SP * NT + 2 * (size_t)NPC * kJP * SP);
    auto kern = rk4_dense_poly_kernel<RI, NT, F64>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int64_t blocks = (io.n_inst + NT - 1) / NT;
    if (blocks <= 0) return cudaSuccess;
    kern<<<(unsigned)blocks, kDenseThreads, smem, st>>>(sys, E, io);
    return cudaGetLastError();
}

}  // namespace

bool dense_few_default(const DenseSys& sys, int64_t n_inst)
{
    int cap = 0;
    switch (sys.s_pad) {
        case 64: cap = device_sm_count(); break;
        case 128: cap = split_capacity<128, DenseBatchSrc<false>>(); break;
        case 256: cap = split_capacity<256, DenseBatchSrc<false>>(); break;
        case 512: cap = split_capacity<512, DenseBatchSrc<false>>(); break;
        default: return false;
    }
    return cap > 0 && (sys.per_inst || n_inst <= 8 * (int64_t)cap);
}

bool dense_few_capable(const DenseSys& sys)
{
    switch (sys.s_pad) {
        case 64: return true;
        case 128: return split_capacity<128, DenseBatchSrc<false>>() > 0;
        case 256: return split_capacity<256, DenseBatchSrc<false>>() > 0;
        case 512: return split_capacity<512, DenseBatchSrc<false>>() > 0;
        default: return false;
    }
}

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

cudaError_t launch_rk4_dense_poly(const DenseSys& sys, const void* E, const BatchIO& io, bool fp64, cudaStream_t st)
{
    if (io.n_inst == 0) return cudaSuccess;
#define CHO_POLY_CASE(SPV, RI64, NT64, RI32, NT32)                                                  \
    case SPV:                                                                                        \
        return fp64 ? launch_poly<RI64, NT64, true>(sys, E, io, st) : launch_poly<RI32, NT32, false>(sys, E, io, st);
    switch (sys.s_pad) {
        CHO_POLY_CASE(64, 2, 8, 4, 16)
        CHO_POLY_CASE(128, 4, 8, 8, 16)
        CHO_POLY_CASE(256, 8, 8, 16, 16)
        CHO_POLY_CASE(512, 8, 4, 16, 8)
        default: return cudaErrorInvalidValue;
    }
#undef CHO_POLY_CASE
}

cudaError_t launch_rk4_dense_slots(const DenseSys& sys, const SlotIO& io, bool fp64, cudaStream_t st)
{
    if (io.n_inst == 0) return cudaSuccess;
    return dispatch_simt<DenseSlotSrc>(sys, fp64, io.n_inst, st, [&](auto& src) {
        src.io = io;
        src.s = sys.s;
    });
}

namespace {

template <class K>
int blocks_per_sm(K kern, int threads, size_t smem)
{
    int n = 0;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, threads, smem) != cudaSuccess) {
        (void)cudaGetLastError();
        return 0;
    }
    return n;
}

template <int RI, int NT, bool F64, class Src, int NTHR = kDenseThreads>
int simt_resident()
{
    using Real = std::conditional_t<F64, double, float>;
    constexpr int SP = (NTHR / NT) * RI;
    constexpr int NB = F64 ? 1 : 2;
    const size_t smem = sizeof(Real) * (2 * (size_t)SP * NT + 2 * (size_t)NB * kJC * SP);
    return blocks_per_sm(rk4_dense_simt_kernel<RI, NT, F64, Src, NTHR>, NTHR, smem) * device_sm_count() * NT;
}

}  // namespace

// Instances the slot kernels of a dense system hold resident at once on this device: the
// one-instance-per-CTA-or-cluster kernels for FP32 (the choice for up to eight times as
// many instances), else the streaming kernels.  0 if none fits.
int dense_slot_resident(const DenseSys& sys, bool fp64)
{
    using S32 = DenseSlotSrc<false>;
    using S64 = DenseSlotSrc<true>;
    if (!fp64) {
        int cap = 0;
        switch (sys.s_pad) {
            case 64:
                cap = blocks_per_sm(rk4_dense_own_kernel<S32>, 64, sizeof(float) * ((size_t)64 * 68 + 2 * 64)) *
                      device_sm_count();
                break;
            case 128: cap = split_capacity<128, S32>(); break;
            case 256: cap = split_capacity<256, S32>(); break;
            case 512: cap = split_capacity<512, S32>(); break;
            default: return 0;
        }
        if (cap > 0) return cap;
    }
#define CHO_RES_OWN(SPV, RI)                                                                         \
    case SPV: return fp64 ? simt_resident<RI, 1, true, S64, SPV / RI>() : simt_resident<RI, 1, false, S32, SPV / RI>();
#define CHO_RES(SPV, RI64, NT64, RI32, NT32)                                                         \
    case SPV: return fp64 ? simt_resident<RI64, NT64, true, S64>() : simt_resident<RI32, NT32, false, S32>();
    if (sys.per_inst) {
        switch (sys.s_pad) {
            CHO_RES_OWN(64, 1)
            CHO_RES_OWN(128, 2)
            CHO_RES_OWN(256, 4)
            CHO_RES_OWN(512, 8)
            default: return 0;
        }
    }
    switch (sys.s_pad) {
        CHO_RES(64, 2, 8, 4, 16)
        CHO_RES(128, 4, 8, 8, 16)
        CHO_RES(256, 8, 8, 16, 16)
        CHO_RES(512, 8, 4, 16, 8)
        default: return 0;
    }
#undef CHO_RES
#undef CHO_RES_OWN
}

// Device data of a dense system: for each of its n_sys parameter sets B^T padded
// to s_pad in FP64 and as FP32 pairs (hi block then lo block), back to back; for a
// single shared set also the BF16 pieces the tensor-core kernel reads.
cudaError_t build_dense_device(cho_system_impl* sys, const double* B)
{
    const int s = sys->s;
    const int sp = dense_pad(s);
    if (sp > 512) return cudaErrorInvalidValue;
    sys->s_pad = sp;
    const size_t n = (size_t)sp * sp;
    const size_t sets = (size_t)sys->n_sys;
    std::vector<double> Bt(sets * n, 0.0);
    std::vector<float> B32(sets * 2 * n);
    for (size_t p = 0; p < sets; ++p) {
        const double* Bp = B + p * (size_t)s * s;
        double* T = &Bt[p * n];
        for (int i = 0; i < s; ++i)
            for (int j = 0; j < s; ++j) T[(size_t)j * sp + i] = Bp[(size_t)i * s + j];
        float* F = &B32[p * 2 * n];
        for (size_t k = 0; k < n; ++k) split_ff(T[k], F[k], F[n + k]);
    }
    cudaError_t e = cudaMalloc(&sys->d_B64, Bt.size() * sizeof(double));
    if (e == cudaSuccess) e = cudaMemcpy(sys->d_B64, Bt.data(), Bt.size() * sizeof(double), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc(&sys->d_B32, B32.size() * sizeof(float));
    if (e == cudaSuccess) e = cudaMemcpy(sys->d_B32, B32.data(), B32.size() * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        if (sets == 1) {
            e = build_dense_tc_device(sys, B);
        } else {
            sys->s_tc = 0;
            e = cudaMalloc(&sys->d_err, sizeof(int));
            if (e == cudaSuccess) e = cudaMemset(sys->d_err, 0, sizeof(int));
        }
    }
    return e;
}

}  // namespace cho
