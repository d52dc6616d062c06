// rk4_small.cu -- classical RK4 for systems of s <= 32 degrees of freedom.
//
// Each instance is integrated by a group of G = S/R lanes of one warp (S = s
// padded to a power of two, R rows of B = M^{-1}K per lane).  For S <= 4 a
// single thread holds the whole instance (G = 1): state, stage values and all
// of B live in registers and no data is exchanged.  For S >= 8 each lane
// holds R rows of B and R degrees of freedom; the stage displacement is
// published to a per-group shared-memory slot once per stage and read back
// as a broadcast, so that every lane can form its rows of B x.
//
// One RK4 step on y = (x, v) (Section 3, first-order form; right-hand side
// D = (v, -B x) as D(1)..D(4) for eq. 2):
//   a1 = -B x                    k1 = (v,   a1)
//   a2 = -B (x + h/2 v)          k2 = (v2,  a2),  v2 = v + h/2 a1
//   a3 = -B (x + h/2 v2)         k3 = (v3,  a3),  v3 = v + h/2 a2
//   a4 = -B (x + h v3)           k4 = (v4,  a4),  v4 = v + h a3
//   x += h/6 (v + 2 v2 + 2 v3 + v4),  v += h/6 (a1 + 2 a2 + 2 a3 + a4)
// The whole horizon runs with the state in registers; only checkpoints and
// the final state are written to memory.
#include "cho_internal.h"
#include "persist.cuh"
#include "rk4_common.cuh"
#include "../../include/cho.h"

#include <algorithm>
#include <mutex>
#include <type_traits>
#include <cstdlib>
#include <cstring>

namespace cho {
namespace {

constexpr int rows_per_lane(int S) { return S <= 4 ? S : (S == 8 ? 2 : 1); }
constexpr int kDwThreads = 128;   // threads per CTA of the double-FP32 kernel

// ---- instance sources ----------------------------------------------------------

// Batch form: FP64 arrays in and out, shared step count, optional checkpoints.
template <bool F64, int S>
struct BatchSrc {
    SmallSys sys;
    BatchIO io;
    using Real = std::conditional_t<F64, double, float>;

    __device__ int64_t count() const { return io.n_inst; }
    __device__ int s(int64_t) const { return sys.s; }
    __device__ double h(int64_t q) const { return io.h[io.h_per_inst ? q : 0]; }
    __device__ int64_t steps(int64_t) const { return io.n_steps; }
    __device__ int64_t ckpt_every() const { return io.ckpt_every; }

    __device__ void coef(int64_t q, int row, int j, Real& hi, float& lo) const
    {
        const int64_t set = sys.per_inst_sys ? q : 0;
        if constexpr (F64) {
            hi = sys.B64[(set * S + row) * S + j];
            lo = 0.f;
        } else {
            const float* b = sys.B32 + set * 2 * S * S;
            hi = b[row * S + j];
            lo = b[S * S + row * S + j];
        }
    }
    // FP32: v is held as the scaled velocity u = (h/6) v (see scaled_velocity)
    __device__ void load(int64_t q, int row, Real& x, Real& v, float& cx, float& cv) const
    {
        const int sz = sys.s;
        const double xd = row < sz ? io.x0[q * sz + row] : 0.0;
        const double vd0 = row < sz ? io.v0[q * sz + row] : 0.0;
        const double vd = F64 ? vd0 : scaled_velocity(vd0, h(q));
        x = (Real)xd;
        v = (Real)vd;
        // the state is the unevaluated sum x + c
        cx = F64 ? 0.f : (float)(xd - (double)x);
        cv = F64 ? 0.f : (float)(vd - (double)v);
    }
    __device__ double vout(int64_t q, Real v, float cv) const
    {
        const double u = (double)v + (double)cv;
        return F64 ? u : unscaled_velocity(u, h(q));
    }
    __device__ void checkpoint(int64_t q, int64_t ck, int row, Real x, Real v, float cx, float cv) const
    {
        const int sz = sys.s;
        if (row >= sz || io.x_traj == nullptr) return;
        const int64_t o = (q * io.n_ck + ck) * sz + row;
        io.x_traj[o] = (double)x + (double)cx;
        if (io.v_traj) io.v_traj[o] = vout(q, v, cv);
    }
    __device__ void store(int64_t q, int row, Real x, Real v, float cx, float cv, bool) const
    {
        const int sz = sys.s;
        if (row >= sz) return;
        io.x_out[q * sz + row] = (double)x + (double)cx;
        io.v_out[q * sz + row] = vout(q, v, cv);
    }
    __device__ void finish(int64_t, int64_t, bool) const {}
};

// Slot form (serving): resident state block [x(S), v(S), cx(S), cv(S)] in the
// kernel's precision (FP32: the scaled velocity u = (h/6) v in place of v, converted
// by the serving engine at admission and retirement), coefficient block in the batch
// layout of one set.  FRESH (persistent kernels): the slot table and ids live in mapped
// host memory and change between generations, so they are read with volatile loads and
// the state blocks through L2 only (a block may hold another request's state than the
// last time this SM's L1 saw it); finished slots go to the completion ring.
template <bool F64, int S, bool FRESH = false>
struct SlotSrc {
    SlotIO io;
    const PersistIO* pio = nullptr;
    using Real = std::conditional_t<F64, double, float>;

    __device__ int32_t id(int64_t q) const
    {
        if constexpr (FRESH) return ((const volatile int32_t*)io.slot_ids)[q];
        else return io.slot_ids[q];
    }
    __device__ const SlotDesc& d(int64_t q) const { return io.slots[io.slot_ids[q]]; }
    __device__ const void* f_coef(int64_t q) const
    {
        if constexpr (FRESH) return ((const volatile SlotDesc*)io.slots)[id(q)].coef;
        else return d(q).coef;
    }
    __device__ void* f_state(int64_t q) const
    {
        if constexpr (FRESH) return ((const volatile SlotDesc*)io.slots)[id(q)].state;
        else return d(q).state;
    }
    __device__ int64_t count() const { return io.n_inst; }
    __device__ int s(int64_t q) const
    {
        if constexpr (FRESH) return ((const volatile SlotDesc*)io.slots)[id(q)].s;
        else return d(q).s;
    }
    __device__ double h(int64_t q) const
    {
        if constexpr (FRESH) return ((const volatile SlotDesc*)io.slots)[id(q)].h;
        else return d(q).h;
    }
    __device__ int64_t steps(int64_t q) const
    {
        int64_t rem;
        if constexpr (FRESH) rem = ((const volatile SlotDesc*)io.slots)[id(q)].remaining;
        else rem = d(q).remaining;
        return rem < io.chunk ? rem : io.chunk;
    }
    __device__ int64_t ckpt_every() const { return 0; }

    __device__ void coef(int64_t q, int row, int j, Real& hi, float& lo) const
    {
        if constexpr (F64) {
            hi = ((const double*)f_coef(q))[row * S + j];
            lo = 0.f;
        } else {
            const float* b = (const float*)f_coef(q);
            hi = b[row * S + j];
            lo = b[S * S + row * S + j];
        }
    }
    __device__ Real ld(const Real* p) const
    {
        if constexpr (FRESH) return __ldcg(p);
        else return *p;
    }
    __device__ void load(int64_t q, int row, Real& x, Real& v, float& cx, float& cv) const
    {
        const Real* st = (const Real*)f_state(q);
        x = ld(st + row);
        v = ld(st + S + row);
        if constexpr (F64) {
            cx = cv = 0.f;
        } else {
            cx = ld(st + 2 * S + row);
            cv = ld(st + 3 * S + row);
        }
    }
    __device__ void checkpoint(int64_t, int64_t, int, Real, Real, float, float) const {}
    __device__ void store(int64_t q, int row, Real x, Real v, float cx, float cv, bool) const
    {
        Real* st = (Real*)f_state(q);
        st[row] = x;
        st[S + row] = v;
        if constexpr (!F64) {
            st[2 * S + row] = cx;
            st[3 * S + row] = cv;
        }
    }
    // once per instance, after every lane has stored: book the steps run, flag a bad state
    __device__ void finish(int64_t q, int64_t ran, bool bad) const
    {
        const int32_t slot = id(q);
        if constexpr (FRESH) {
            volatile SlotDesc* sd = (volatile SlotDesc*)io.slots + slot;
            const int64_t left = sd->remaining - ran;
            sd->remaining = left;
            if (bad) ((volatile int32_t*)io.status)[slot] = CHO_ENONFINITE;
            if (left == 0 || bad) persist_complete(*pio, slot);
        } else {
            io.slots[slot].remaining -= ran;
            if (bad) io.status[slot] = CHO_ENONFINITE;
        }
    }
};

// ---- the kernel ------------------------------------------------------------------

// The work of CTA `cta` of a launch (the kernel below; the persistent kernel calls it
// for every CTA-sized share of a generation).
template <int S, bool F64, class Src>
__device__ __forceinline__ void rk4_small_body(const Src& src, int64_t cta)
{
    using Real = std::conditional_t<F64, double, float>;
    constexpr int R = rows_per_lane(S);
    constexpr int G = S / R;                      // lanes per instance
    constexpr int GPB = kSmallThreads / G;        // groups per block
    __shared__ Real xch[G > 1 ? 2 : 1][G > 1 ? GPB : 1][G > 1 ? S : 1];

    const int64_t tid = cta * kSmallThreads + threadIdx.x;
    const int64_t q = tid / G;
    const int g = (int)(tid % G);
    const int grp = threadIdx.x / G;
    const unsigned lane = threadIdx.x & 31u;
    const unsigned gmask = (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << (lane & ~(unsigned)(G - 1)));
    if (q >= src.count()) return;                 // whole groups leave together

    // rows g*R .. g*R+R-1 of B (hi, lo)
    Real bh[R][S];
    float bl[R][S];
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
        for (int j = 0; j < S; ++j) {
            src.coef(q, g * R + r, j, bh[r][j], bl[r][j]);
            if constexpr (!F64) scaled_coef(bh[r][j], bl[r][j], src.h(q));   // B'' = h^2/36 B
        }

    const StepSize<F64> hs(src.h(q));
    // stage constants: FP64 h/2, h; FP32 (scaled velocity) 3, 6
    const Real c_half = F64 ? hs.h2 : (Real)3, c_full = F64 ? hs.h : (Real)6;
    Real x[R], v[R];
    float cx[R], cv[R];
#pragma unroll
    for (int r = 0; r < R; ++r) src.load(q, g * R + r, x[r], v[r], cx[r], cv[r]);

    int buf = 0;
    // acc[r] = -(B xs)[row g*R + r].  FP32: B = hi + lo; the lo product is formed
    // at stage 1 (first == true) and reused by stages 2-4 ("frozen lo"): it
    // differs from lo * xs by lo * (xs - x), a relative 2^-24 * omega h of the
    // acceleration, far below the rounding of the hi product, and saves 3/4 of
    // the lo multiply-adds.
    Real lo1[R];
    auto accel = [&](const Real (&xs)[R], Real (&acc)[R], bool first) {
        if constexpr (G == 1) {
            // row r sums its columns starting at the diagonal: j = r, r+1, ... (mod S)
#pragma unroll
            for (int r = 0; r < R; ++r) {
                Real t = 0;
                if constexpr (!F64) {
                    if (first) {
#pragma unroll
                        for (int jj = 0; jj < S; ++jj) t = fmaf(bl[r][(r + jj) % S], xs[(r + jj) % S], t);
                        lo1[r] = t;
                    } else {
                        t = lo1[r];
                    }
                }
#pragma unroll
                for (int jj = 0; jj < S; ++jj) t = fmar(bh[r][(r + jj) % S], xs[(r + jj) % S], t);
                acc[r] = -t;
            }
        } else {
#pragma unroll
            for (int r = 0; r < R; ++r) xch[buf][grp][g * R + r] = xs[r];
            __syncwarp(gmask);
#pragma unroll
            for (int r = 0; r < R; ++r) {
                Real t = 0;
                if constexpr (!F64) {
                    if (first) {
#pragma unroll
                        for (int j = 0; j < S; ++j) t = fmaf(bl[r][j], xch[buf][grp][j], t);
                        lo1[r] = t;
                    } else {
                        t = lo1[r];
                    }
                }
#pragma unroll
                for (int j = 0; j < S; ++j) t = fmar(bh[r][j], xch[buf][grp][j], t);
                acc[r] = -t;
            }
            buf ^= 1;
        }
    };

    const int64_t n = src.steps(q);
    const int64_t every = src.ckpt_every() > 0 ? src.ckpt_every() : (n > 0 ? n : 1);
    int64_t ck = 0;
    for (int64_t done = 0; done < n; done += every) {
        repeat_steps(every, [&]() {
            Real a[R], xs[R], kx[R], kv[R], vs[R];
            accel(x, a, true);                             // stage 1
#pragma unroll
            for (int r = 0; r < R; ++r) {
                if constexpr (F64) kx[r] = v[r];
                else kx[r] = fmar((Real)2, v[r], cx[r]);   // FP32: the x sum starts on its compensation
                kv[r] = a[r];
                xs[r] = fmar(c_half, v[r], x[r]);
                vs[r] = fmar(c_half, a[r], v[r]);
            }
            accel(xs, a, false);                           // stage 2
#pragma unroll
            for (int r = 0; r < R; ++r) {
                kx[r] = fmar((Real)2, vs[r], kx[r]);
                kv[r] = fmar((Real)2, a[r], kv[r]);
                xs[r] = fmar(c_half, vs[r], x[r]);
                vs[r] = fmar(c_half, a[r], v[r]);
            }
            accel(xs, a, false);                           // stage 3
#pragma unroll
            for (int r = 0; r < R; ++r) {
                kx[r] = fmar((Real)2, vs[r], kx[r]);
                kv[r] = fmar((Real)2, a[r], kv[r]);
                xs[r] = fmar(c_full, vs[r], x[r]);
                // FP32: the stage-4 velocity v + 6 a3 enters only the x sum, which takes 2v + 6 a3
                if constexpr (F64) vs[r] = fmar(c_full, a[r], v[r]);
                else kx[r] = fmar(c_full, a[r], kx[r]);
            }
            accel(xs, a, false);                           // stage 4
#pragma unroll
            for (int r = 0; r < R; ++r) {
                if constexpr (F64) {
                    kx[r] = addr(kx[r], vs[r]);
                    kv[r] = addr(kv[r], a[r]);
                    state_update<true>(x[r], cx[r], kx[r], hs);
                    state_update<true>(v[r], cv[r], kv[r], hs);
                } else {
                    kv[r] = addr(kv[r], a[r]);
                    comp_add_folded(x[r], cx[r], kx[r]);   // the scaled sums are the increments
                    comp_add(v[r], cv[r], kv[r]);
                }
            }
        });
        if (src.ckpt_every() > 0) {
#pragma unroll
            for (int r = 0; r < R; ++r) src.checkpoint(q, ck, g * R + r, x[r], v[r], cx[r], cv[r]);
            ++ck;
        }
    }
    bool bad = false;
#pragma unroll
    for (int r = 0; r < R; ++r) bad |= !(isfinite((double)x[r]) && isfinite((double)v[r]));
#pragma unroll
    for (int r = 0; r < R; ++r) src.store(q, g * R + r, x[r], v[r], cx[r], cv[r], bad);
    if constexpr (G > 1) bad = __any_sync(gmask, bad);
    if (g == 0) src.finish(q, n, bad);
}

template <int S, bool F64, class Src>
__global__ void __launch_bounds__(kSmallThreads) rk4_small_kernel(const Src src)
{
    rk4_small_body<S, F64>(src, blockIdx.x);
}

// Persistent form for the serving engine: the generation loop of persist.cuh around
// the same body, over the generation's slot ids.
template <int S, bool F64>
__global__ void __launch_bounds__(kSmallThreads) rk4_small_persist_kernel(const PersistIO pio)
{
    constexpr int G = S / rows_per_lane(S);
    persist_loop(pio, [&](int64_t n, int64_t chunk) {
        SlotSrc<F64, S, true> src;
        src.io = SlotIO{n, pio.slot_ids, pio.slots, pio.status, chunk};
        src.pio = &pio;
        const int64_t ctas = (n * G + kSmallThreads - 1) / kSmallThreads;
        for (int64_t c = blockIdx.x; c < ctas; c += gridDim.x) rk4_small_body<S, F64>(src, c);
    });
}

template <int S, bool F64, class Src>
cudaError_t launch_one(const Src& src, int64_t n, cudaStream_t st)
{
    constexpr int G = S / rows_per_lane(S);
    const int64_t threads = n * G;
    const int64_t blocks = (threads + kSmallThreads - 1) / kSmallThreads;
    if (blocks <= 0) return cudaSuccess;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidValue;
    rk4_small_kernel<S, F64, Src><<<(unsigned)blocks, kSmallThreads, 0, st>>>(src);
    return cudaGetLastError();
}

template <template <bool, int> class SrcT, class Init>
cudaError_t dispatch(int S, bool fp64, int64_t n, cudaStream_t st, const Init& init)
{
#define CHO_SMALL_CASE(SV)                                                                 \
    case SV:                                                                               \
        if (fp64) { SrcT<true, SV> s; init(s); return launch_one<SV, true>(s, n, st); }    \
        else { SrcT<false, SV> s; init(s); return launch_one<SV, false>(s, n, st); }
    switch (S) {
        CHO_SMALL_CASE(2)
        CHO_SMALL_CASE(4)
        CHO_SMALL_CASE(8)
        CHO_SMALL_CASE(16)
        CHO_SMALL_CASE(32)
        default: return cudaErrorInvalidValue;
    }
#undef CHO_SMALL_CASE
}

// ---- 2-DOF systems in FP32, two instances per thread in packed FP32x2 arithmetic ----
//
// The same step as rk4_small_kernel<2, false> (identical rounding: every packed
// operation rounds each lane as the scalar intrinsic does), with lane 0 and
// lane 1 of every float2 holding instances 2t and 2t+1.  Packing halves the
// instructions issued per instance; the coefficients are stored negated so
// that the packed accumulation yields a = -B'' x directly.

constexpr int kPairThreads = 32;

__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }

// Compensated x += k (the increment without a step-size factor).
// x += y with y already holding the compensation (comp_add_folded on both lanes).
__device__ __forceinline__ void pair_add_folded(float2& x, float2& e, float2 y)
{
    const float2 m1 = f2(-1.f, -1.f);
    const float2 t = __fadd2_rn(x, y);
    const float2 d = __ffma2_rn(x, m1, t);       // t - x
    e = __ffma2_rn(d, m1, y);                    // y - (t - x)
    x = t;
}

__device__ __forceinline__ void pair_add(float2& x, float2& e, float2 k) { pair_add_folded(x, e, __fadd2_rn(k, e)); }

// State of two 2-DOF instances held by one thread (lanes .x and .y of every
// float2): x, v and their compensations, FP32.  An odd instance count repeats
// the last instance in lane .y, which is never stored.
struct Pair2State {
    float2 x[2], v[2], ex[2], ev[2];
    int64_t q0, q1;
    bool has1;

    __device__ __forceinline__ void set_instances(const BatchIO& io, int64_t q)
    {
        q0 = q;
        has1 = q0 + 1 < io.n_inst;
        q1 = has1 ? q0 + 1 : q0;
    }
    __device__ __forceinline__ void load_initial(const BatchIO& io)
    {
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            const double xa = io.x0[q0 * 2 + r], xb = io.x0[q1 * 2 + r];
            const double va = io.v0[q0 * 2 + r], vb = io.v0[q1 * 2 + r];
            x[r] = f2((float)xa, (float)xb);
            v[r] = f2((float)va, (float)vb);
            ex[r] = f2((float)(xa - (double)x[r].x), (float)(xb - (double)x[r].y));
            ev[r] = f2((float)(va - (double)v[r].x), (float)(vb - (double)v[r].y));
        }
    }
    // The eight state registers in a fixed order (hand-over between warps).
    __device__ __forceinline__ float2& reg(int i)
    {
        return i < 2 ? x[i] : (i < 4 ? v[i - 2] : (i < 6 ? ex[i - 4] : ev[i - 6]));
    }
    // Checkpoint ck (state after (ck + 1) * ckpt_every steps).
    __device__ __forceinline__ void store_ckpt(const BatchIO& io, int64_t ck) const
    {
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            io.x_traj[(q0 * io.n_ck + ck) * 2 + r] = (double)x[r].x + (double)ex[r].x;
            if (io.v_traj) io.v_traj[(q0 * io.n_ck + ck) * 2 + r] = (double)v[r].x + (double)ev[r].x;
            if (has1) {
                io.x_traj[(q1 * io.n_ck + ck) * 2 + r] = (double)x[r].y + (double)ex[r].y;
                if (io.v_traj) io.v_traj[(q1 * io.n_ck + ck) * 2 + r] = (double)v[r].y + (double)ev[r].y;
            }
        }
    }
    __device__ __forceinline__ void store_final(const BatchIO& io) const
    {
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            io.x_out[q0 * 2 + r] = (double)x[r].x + (double)ex[r].x;
            io.v_out[q0 * 2 + r] = (double)v[r].x + (double)ev[r].x;
            if (has1) {
                io.x_out[q1 * 2 + r] = (double)x[r].y + (double)ex[r].y;
                io.v_out[q1 * 2 + r] = (double)v[r].y + (double)ev[r].y;
            }
        }
    }
};

// RK4 stage by stage (Section 3): the same step as rk4_small_kernel<2, false>,
// on the scaled velocity u = (h/6) v with B'' = (h^2/36) B (see scaled_velocity).
// Shared by the one-launch kernel and the balanced kernel so that both issue
// exactly the same operations.  The v registers of the state hold u.
struct Pair2 : Pair2State {
    float2 nbh[2][2], nbl[2][2];
    double hd0, hd1;

    __device__ __forceinline__ void init(const SmallSys& sys, const BatchIO& io, int64_t q)
    {
        set_instances(io, q);
        const int64_t s0 = sys.per_inst_sys ? q0 : 0, s1 = sys.per_inst_sys ? q1 : 0;
        const float* b0 = sys.B32 + s0 * 8;      // [hi 2x2][lo 2x2]
        const float* b1 = sys.B32 + s1 * 8;
        hd0 = io.h[io.h_per_inst ? q0 : 0];
        hd1 = io.h[io.h_per_inst ? q1 : 0];
#pragma unroll
        for (int r = 0; r < 2; ++r)
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                float h0 = b0[r * 2 + j], l0 = b0[4 + r * 2 + j], h1 = b1[r * 2 + j], l1 = b1[4 + r * 2 + j];
                scaled_coef(h0, l0, hd0);
                scaled_coef(h1, l1, hd1);
                nbh[r][j] = f2(-h0, -h1);
                nbl[r][j] = f2(-l0, -l1);
            }
    }
    __device__ __forceinline__ int64_t quantum() const { return 1; }
    __device__ __forceinline__ void load_initial(const BatchIO& io)
    {
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            const double xa = io.x0[q0 * 2 + r], xb = io.x0[q1 * 2 + r];
            const double ua = scaled_velocity(io.v0[q0 * 2 + r], hd0), ub = scaled_velocity(io.v0[q1 * 2 + r], hd1);
            x[r] = f2((float)xa, (float)xb);
            v[r] = f2((float)ua, (float)ub);
            ex[r] = f2((float)(xa - (double)x[r].x), (float)(xb - (double)x[r].y));
            ev[r] = f2((float)(ua - (double)v[r].x), (float)(ub - (double)v[r].y));
        }
    }
    __device__ __forceinline__ void store_ckpt(const BatchIO& io, int64_t ck) const
    {
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            io.x_traj[(q0 * io.n_ck + ck) * 2 + r] = (double)x[r].x + (double)ex[r].x;
            if (io.v_traj)
                io.v_traj[(q0 * io.n_ck + ck) * 2 + r] = unscaled_velocity((double)v[r].x + (double)ev[r].x, hd0);
            if (has1) {
                io.x_traj[(q1 * io.n_ck + ck) * 2 + r] = (double)x[r].y + (double)ex[r].y;
                if (io.v_traj)
                    io.v_traj[(q1 * io.n_ck + ck) * 2 + r] = unscaled_velocity((double)v[r].y + (double)ev[r].y, hd1);
            }
        }
    }
    __device__ __forceinline__ void store_final(const BatchIO& io) const
    {
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            io.x_out[q0 * 2 + r] = (double)x[r].x + (double)ex[r].x;
            io.v_out[q0 * 2 + r] = unscaled_velocity((double)v[r].x + (double)ev[r].x, hd0);
            if (has1) {
                io.x_out[q1 * 2 + r] = (double)x[r].y + (double)ex[r].y;
                io.v_out[q1 * 2 + r] = unscaled_velocity((double)v[r].y + (double)ev[r].y, hd1);
            }
        }
    }
    // Stage 1 forms the lo product and keeps it; stages 2-4 reuse it (frozen lo,
    // as rk4_small_kernel).
    __device__ __forceinline__ void accel(const float2 (&xs)[2], float2 (&a)[2], float2 (&lo)[2], bool first) const
    {
#pragma unroll
        for (int r = 0; r < 2; ++r) {            // diagonal first, as rk4_small_kernel
            if (first) {
                lo[r] = __fmul2_rn(nbl[r][r], xs[r]);
                lo[r] = __ffma2_rn(nbl[r][1 - r], xs[1 - r], lo[r]);
            }
            const float2 acc = __ffma2_rn(nbh[r][r], xs[r], lo[r]);
            a[r] = __ffma2_rn(nbh[r][1 - r], xs[1 - r], acc);
        }
    }
    // The stage accelerations two at a time: stage 2's displacement x + 3u does not
    // depend on a1, nor stage 4's x + 6 (u + 3 a2) on a3, so {a1, a2} and {a3, a4} are
    // independent pairs (twice the independent work for the one warp of the
    // sub-partition).  Every value keeps its operations and their order.  The x sum
    // starts on its compensation and takes the stage-4 velocity u + 6 a3 as 2u + 6 a3
    // (as rk4_small_kernel in FP32).
    __device__ __forceinline__ void step()
    {
        const float2 two = f2(2.f, 2.f), three = f2(3.f, 3.f), six = f2(6.f, 6.f);
        float2 a1[2], a2[2], xs[2], xt[2], kx[2], kv[2], lo[2];
#pragma unroll
        for (int r = 0; r < 2; ++r) xs[r] = __ffma2_rn(three, v[r], x[r]);
        accel(x, a1, lo, true);
        accel(xs, a2, lo, false);
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            const float2 vs2 = __ffma2_rn(three, a1[r], v[r]);
            const float2 vs3 = __ffma2_rn(three, a2[r], v[r]);
            kx[r] = __ffma2_rn(two, vs2, __ffma2_rn(two, v[r], ex[r]));
            kv[r] = __ffma2_rn(two, a2[r], a1[r]);
            kx[r] = __ffma2_rn(two, vs3, kx[r]);
            xs[r] = __ffma2_rn(three, vs2, x[r]);
            xt[r] = __ffma2_rn(six, vs3, x[r]);
        }
        accel(xs, a1, lo, false);                // a3
        accel(xt, a2, lo, false);                // a4
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            kx[r] = __ffma2_rn(six, a1[r], kx[r]);
            kv[r] = __ffma2_rn(two, a1[r], kv[r]);
            kv[r] = __fadd2_rn(kv[r], a2[r]);
            pair_add_folded(x[r], ex[r], kx[r]);
            pair_add(v[r], ev[r], kv[r]);
        }
    }
};

// ---- polynomial form of the same map ----------------------------------------------
//
// For the linear system y' = A y, y = (x0, x1, v0, v1), A = [[0, I], [-B, 0]], one
// classical RK4 step is exactly y <- P(hA) y with
//     P(hA) = I + hA + (hA)^2/2 + (hA)^3/6 + (hA)^4/24
// (the stage values of Section 3 are linear in y; composing them gives P).  k
// steps are y <- P(hA)^k y.  The jump matrix E = P(hA)^k - I is formed in FP64 per
// instance (Horner for P, binary powers for the k-th power), so the update is
// y <- y + E y: with E as an unevaluated FP32 pair and the compensated state of
// the stage form, 48 FP32 operations per k steps against 64 per step.
struct Mat4 {
    double m[4][4];
};

__device__ __forceinline__ Mat4 mat4_mul(const Mat4& a, const Mat4& b)
{
    Mat4 c;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            double t = 0.0;
#pragma unroll
            for (int l = 0; l < 4; ++l) t = __fma_rn(a.m[i][l], b.m[l][j], t);
            c.m[i][j] = t;
        }
    return c;
}

// E = P(hA)^k - I for the 2 x 2 matrix B (row-major b[4]).
__device__ Mat4 poly_jump_matrix(const double (&b)[4], double h, int k)
{
    Mat4 hA{}, I{};
#pragma unroll
    for (int i = 0; i < 4; ++i) I.m[i][i] = 1.0;
    hA.m[0][2] = h;
    hA.m[1][3] = h;
    hA.m[2][0] = -h * b[0];
    hA.m[2][1] = -h * b[1];
    hA.m[3][0] = -h * b[2];
    hA.m[3][1] = -h * b[3];
    // P = I + hA (I + hA/2 (I + hA/3 (I + hA/4)))
    Mat4 P = I;
    for (int d = 4; d >= 1; --d) {
        Mat4 T = mat4_mul(hA, P);
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) P.m[i][j] = I.m[i][j] + T.m[i][j] / (double)d;
    }
    Mat4 R = I, base = P;
    for (int kk = k; kk > 0; kk >>= 1) {
        if (kk & 1) R = mat4_mul(R, base);
        if (kk > 1) base = mat4_mul(base, base);
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) R.m[i][i] -= 1.0;
    return R;
}

struct Pair2Poly : Pair2State {
    float2 eh[4][4], el[4][4];
    int32_t k;

    // E of both instances from the set-up kernel's FP64 table, split into FP32 pairs.
    __device__ __forceinline__ void init(const SmallSys&, const BatchIO& io, int64_t q)
    {
        set_instances(io, q);
        k = io.poly_jump;
        const double* E0 = io.poly_E + q0 * 16;
        const double* E1 = io.poly_E + q1 * 16;
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const double d0 = E0[i * 4 + j], d1 = E1[i * 4 + j];
                const float h0 = (float)d0, h1 = (float)d1;
                eh[i][j] = f2(h0, h1);
                el[i][j] = f2((float)(d0 - (double)h0), (float)(d1 - (double)h1));
            }
    }
    __device__ __forceinline__ int64_t quantum() const { return k; }
    // k RK4 steps: y <- y + E y (lo products first), compensated.
    __device__ __forceinline__ void step()
    {
        const float2 y[4] = {x[0], x[1], v[0], v[1]};
        float2 z[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            float2 acc = __fmul2_rn(el[i][0], y[0]);
#pragma unroll
            for (int j = 1; j < 4; ++j) acc = __ffma2_rn(el[i][j], y[j], acc);
#pragma unroll
            for (int j = 0; j < 4; ++j) acc = __ffma2_rn(eh[i][j], y[j], acc);
            z[i] = acc;
        }
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            pair_add(x[r], ex[r], z[r]);
            pair_add(v[r], ev[r], z[2 + r]);
        }
    }
};

// Steps [first, last) of the horizon (multiples of the thread type's quantum),
// checkpoints where ckpt_every divides the step count reached (first and last
// are then multiples of ckpt_every).
template <class T>
__device__ __forceinline__ void advance(T& p, int64_t n_steps)
{
    const int64_t n = n_steps / p.quantum();
    for (int64_t base = 0; base < n; base += 0x40000000LL) {
        const int32_t m = (int32_t)(n - base < 0x40000000LL ? n - base : 0x40000000LL);
#pragma unroll 2
        for (int32_t it = 0; it < m; ++it) p.step();
    }
}

template <class T>
__device__ __forceinline__ void run_steps(T& p, const BatchIO& io, int64_t first, int64_t last, bool store)
{
    if (io.ckpt_every > 0 && io.x_traj) {
        for (int64_t done = first; done < last; done += io.ckpt_every) {
            advance(p, io.ckpt_every);
            if (store) p.store_ckpt(io, done / io.ckpt_every);
        }
    } else {
        advance(p, last - first);
    }
}

// Set-up of the polynomial form: E = P(hA)^k - I of every instance in FP64,
// [n_inst][4][4], one instance per thread at full occupancy (the FP64 matrix
// products are latency bound; inside the integration kernels they ran on one
// warp per sub-partition and cost more than the integration at k >= 5).  B is
// the FP32 pair (FP32 mode, as the stage form uses) or the FP64 matrix.
__global__ void __launch_bounds__(64) poly_setup_kernel(const SmallSys sys, const BatchIO io, bool fp64,
                                                        double* E)
{
    const int64_t q = (int64_t)blockIdx.x * 64 + threadIdx.x;
    if (q >= io.n_inst) return;
    const int64_t set = sys.per_inst_sys ? q : 0;
    double b[4];
    if (fp64) {
#pragma unroll
        for (int i = 0; i < 4; ++i) b[i] = sys.B64[set * 4 + i];
    } else {
#pragma unroll
        for (int i = 0; i < 4; ++i) b[i] = (double)sys.B32[set * 8 + i] + (double)sys.B32[set * 8 + 4 + i];
    }
    const Mat4 m = poly_jump_matrix(b, io.h[io.h_per_inst ? q : 0], io.poly_jump);
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) E[q * 16 + i * 4 + j] = m.m[i][j];
}

// The polynomial form in FP64: one instance per thread, y <- y + E y.
__global__ void __launch_bounds__(64) rk4_poly64_kernel(const SmallSys sys, const BatchIO io)
{
    const int64_t q = (int64_t)blockIdx.x * 64 + threadIdx.x;
    if (q >= io.n_inst) return;
    Mat4 E;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) E.m[i][j] = io.poly_E[q * 16 + i * 4 + j];
    double y[4] = {io.x0[q * 2], io.x0[q * 2 + 1], io.v0[q * 2], io.v0[q * 2 + 1]};
    auto jumps = [&](int64_t n) {
        for (int64_t it = 0; it < n; ++it) {
            double z[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                double t = 0.0;
#pragma unroll
                for (int j = 0; j < 4; ++j) t = __fma_rn(E.m[i][j], y[j], t);
                z[i] = t;
            }
#pragma unroll
            for (int i = 0; i < 4; ++i) y[i] = __dadd_rn(y[i], z[i]);
        }
    };
    const int64_t k = io.poly_jump;
    if (io.ckpt_every > 0 && io.x_traj) {
        for (int64_t done = 0; done < io.n_steps; done += io.ckpt_every) {
            jumps(io.ckpt_every / k);
            const int64_t o = (q * io.n_ck + done / io.ckpt_every) * 2;
            io.x_traj[o] = y[0];
            io.x_traj[o + 1] = y[1];
            if (io.v_traj) {
                io.v_traj[o] = y[2];
                io.v_traj[o + 1] = y[3];
            }
        }
    } else {
        jumps(io.n_steps / k);
    }
    io.x_out[q * 2] = y[0];
    io.x_out[q * 2 + 1] = y[1];
    io.v_out[q * 2] = y[2];
    io.v_out[q * 2 + 1] = y[3];
}

// ---- polynomial form for every system of the small family (s <= 32) ---------------
//
// The same map for S = 2 .. 32 (s padded to S with zero rows and columns of B, so the
// padded coordinates keep E's zero rows and never move): y = (x, v) of 2S rows,
// E = P(hA)^k - I of 2S x 2S.  Set-up: one CTA per matrix forms E in FP64 in shared
// memory (hA from B, Horner for P, binary powers for the k-th power, the s = 2 set-up's
// order of operations).  Integration: one thread per row of y; a CTA holds NI = 128/2S
// instances, their E transposed in shared memory (FP64, or FP32 hi and lo pieces), and
// exchanges y through shared memory once per update: thread i forms (E y)_i (FP32: the
// lo products first) and adds it to its row (compensated in FP32).  One E serves every
// instance when they share B and h.

constexpr int kPolySetupThreads = 256;
constexpr int kPolyThreads = 128;

// C = A B for n x n row-major FP64 matrices in shared memory; every thread of the CTA
// takes part, and C is complete (and A, B free) when it returns.
__device__ void smem_matmul(const double* A, const double* B, double* C, int n)
{
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
        const int i = e / n, j = e % n;
        double t = 0.0;
        for (int l = 0; l < n; ++l) t = __fma_rn(A[i * n + l], B[l * n + j], t);
        C[e] = t;
    }
    __syncthreads();
}

// E (n_E matrices of 2S x 2S, row-major) for instance blockIdx.x (or the shared one).
template <int S>
__global__ void __launch_bounds__(kPolySetupThreads) small_poly_setup_kernel(const SmallSys sys, const BatchIO io,
                                                                              bool fp64, double* E)
{
    constexpr int n = 2 * S;
    extern __shared__ __align__(16) double pm[];
    double* hA = pm;
    double* base = pm + n * n;
    double* R = pm + 2 * n * n;
    double* T = pm + 3 * n * n;
    const int64_t q = blockIdx.x;
    const int64_t set = sys.per_inst_sys ? q : 0;
    const double h = io.h[io.h_per_inst ? q : 0];
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
        const int i = e / n, j = e % n;
        double a = 0.0;
        if (i < S) {
            a = (j == S + i) ? h : 0.0;                          // x' = v
        } else if (j < S) {
            const int r = i - S;                                // v' = -B x
            const double b = fp64 ? sys.B64[(set * S + r) * S + j]
                                  : (double)sys.B32[set * 2 * S * S + r * S + j] +
                                        (double)sys.B32[set * 2 * S * S + S * S + r * S + j];
            a = -h * b;
        }
        hA[e] = a;
        base[e] = (i == j) ? 1.0 : 0.0;                           // P starts at I
        R[e] = (i == j) ? 1.0 : 0.0;
    }
    __syncthreads();
    // P = I + hA (I + hA/2 (I + hA/3 (I + hA/4)))
    for (int d = 4; d >= 1; --d) {
        smem_matmul(hA, base, T, n);
        for (int e = threadIdx.x; e < n * n; e += blockDim.x)
            base[e] = ((e / n == e % n) ? 1.0 : 0.0) + T[e] / (double)d;
        __syncthreads();
    }
    // R = P^k by binary powers (T is scratch; hA is free now)
    double* tmp = hA;
    for (int kk = io.poly_jump; kk > 0; kk >>= 1) {
        if (kk & 1) {
            smem_matmul(R, base, T, n);
            double* sw = R;
            R = T;
            T = sw;
        }
        if (kk > 1) {
            smem_matmul(base, base, tmp, n);
            double* sw = base;
            base = tmp;
            tmp = sw;
        }
    }
    double* out = E + (size_t)q * n * n;
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) out[e] = R[e] - ((e / n == e % n) ? 1.0 : 0.0);
}

template <int S, bool F64>
__global__ void __launch_bounds__(kPolyThreads) rk4_small_poly_kernel(const SmallSys sys, const BatchIO io,
                                                                      const double* __restrict__ E, int shared_E)
{
    using Real = std::conditional_t<F64, double, float>;
    constexpr int n = 2 * S;                     // rows of y per instance
    constexpr int NI = kPolyThreads / n;         // instances per CTA
    extern __shared__ __align__(16) unsigned char poly_sm[];
    const int nmat = shared_E ? 1 : NI;
    // E^T per instance slot: FP64 [nmat][n][n], FP32 hi [nmat][n][n] then lo
    Real* Eh = (Real*)poly_sm;
    float* El = (float*)(Eh + (size_t)nmat * n * n);
    Real* ybuf = F64 ? (Real*)(Eh + (size_t)nmat * n * n) : (Real*)(El + (size_t)nmat * n * n);   // [2][NI][n]

    const int li = threadIdx.x / n;
    const int i = threadIdx.x % n;
    const int64_t q0 = (int64_t)blockIdx.x * NI;
    const int64_t q = q0 + li;
    const bool live = q < io.n_inst;
    const int s = sys.s;
    // E of the CTA's instances into shared memory, transposed: Et[m][j][r] = E_m[r][j]
    for (int e = threadIdx.x; e < nmat * n * n; e += kPolyThreads) {
        const int m = e / (n * n), r = (e / n) % n, j = e % n;
        const int64_t src = shared_E ? 0 : q0 + m;
        double d = 0.0;
        if (src < io.n_inst) d = E[(size_t)src * n * n + (size_t)r * n + j];
        const size_t o = (size_t)m * n * n + (size_t)j * n + r;
        if constexpr (F64) {
            Eh[o] = d;
        } else {
            const float hi = (float)d;
            Eh[o] = hi;
            El[o] = (float)(d - (double)hi);
        }
    }
    // row i of this instance's y: x_i (i < S) or v_{i-S}
    const int dof = i < S ? i : i - S;
    Real y = 0;
    float c = 0.f;
    if (live && dof < s) {
        const double d = i < S ? io.x0[q * s + dof] : io.v0[q * s + dof];
        y = (Real)d;
        c = F64 ? 0.f : (float)(d - (double)y);
    }
    __syncthreads();
    const int m = shared_E ? 0 : li;
    const Real* eh = Eh + (size_t)m * n * n + i;
    const float* el = El + (size_t)m * n * n + i;
    int b = 0;
    auto jumps = [&](int64_t count) {
        for (int64_t it = 0; it < count; ++it) {
            Real* yb = ybuf + (size_t)(b * NI + li) * n;
            yb[i] = y;
            __syncthreads();
            Real z;
            if constexpr (F64) {
                z = 0.0;
#pragma unroll 8
                for (int j = 0; j < n; ++j) z = __fma_rn(eh[(size_t)j * n], yb[j], z);
                y = __dadd_rn(y, z);
            } else {
                z = 0.f;
#pragma unroll 8
                for (int j = 0; j < n; ++j) z = __fmaf_rn(el[(size_t)j * n], yb[j], z);
#pragma unroll 8
                for (int j = 0; j < n; ++j) z = __fmaf_rn(eh[(size_t)j * n], yb[j], z);
                comp_add(y, c, z);
            }
            b ^= 1;
        }
    };
    const int64_t k = io.poly_jump;
    auto put = [&](double* xo, double* vo, int64_t off) {
        if (!live || dof >= s) return;
        const double val = (double)y + (double)c;
        if (i < S) xo[off + dof] = val;
        else if (vo) vo[off + dof] = val;
    };
    if (io.ckpt_every > 0 && io.x_traj) {
        for (int64_t done = 0; done < io.n_steps; done += io.ckpt_every) {
            jumps(io.ckpt_every / k);
            put(io.x_traj, io.v_traj, (q * io.n_ck + done / io.ckpt_every) * s);
        }
    } else {
        jumps(io.n_steps / k);
    }
    put(io.x_out, io.v_out, q * s);
}

template <int S>
cudaError_t launch_small_poly(const SmallSys& sys, const BatchIO& io, bool fp64, cudaStream_t st)
{
    constexpr int n = 2 * S;
    constexpr int NI = kPolyThreads / n;
    const bool shared_E = !sys.per_inst_sys && !io.h_per_inst;
    const int64_t n_E = shared_E ? 1 : io.n_inst;
    void* buf = nullptr;
    cudaError_t e = scratch_alloc(&buf, (size_t)n_E * n * n * sizeof(double), st);
    if (e != cudaSuccess) return e;
    const size_t setup_smem = 4 * (size_t)n * n * sizeof(double);
    e = cudaFuncSetAttribute(small_poly_setup_kernel<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)setup_smem);
    if (e == cudaSuccess) {
        small_poly_setup_kernel<S><<<(unsigned)n_E, kPolySetupThreads, setup_smem, st>>>(sys, io, fp64, (double*)buf);
        e = cudaGetLastError();
    }
    const int nmat = shared_E ? 1 : NI;
    const size_t esz = fp64 ? sizeof(double) : 2 * sizeof(float);
    const size_t smem = (size_t)nmat * n * n * esz + 2 * (size_t)NI * n * (fp64 ? sizeof(double) : sizeof(float));
    const int64_t blocks = (io.n_inst + NI - 1) / NI;
    if (e == cudaSuccess && blocks > 0x7fffffffLL) e = cudaErrorInvalidValue;
    if (e == cudaSuccess) {
        if (fp64) {
            e = cudaFuncSetAttribute(rk4_small_poly_kernel<S, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e == cudaSuccess)
                rk4_small_poly_kernel<S, true><<<(unsigned)blocks, kPolyThreads, smem, st>>>(sys, io, (const double*)buf,
                                                                                             shared_E ? 1 : 0);
        } else {
            e = cudaFuncSetAttribute(rk4_small_poly_kernel<S, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e == cudaSuccess)
                rk4_small_poly_kernel<S, false><<<(unsigned)blocks, kPolyThreads, smem, st>>>(sys, io, (const double*)buf,
                                                                                              shared_E ? 1 : 0);
        }
        if (e == cudaSuccess) e = cudaGetLastError();
    }
    const cudaError_t ef = cudaFreeAsync(buf, st);
    return e != cudaSuccess ? e : ef;
}

template <class T>
__global__ void __launch_bounds__(kPairThreads) rk4_pair2_kernel(const SmallSys sys, const BatchIO io)
{
    const int64_t t = (int64_t)blockIdx.x * kPairThreads + threadIdx.x;
    if (2 * t >= io.n_inst) return;
    T p;
    p.init(sys, io, 2 * t);
    p.load_initial(io);
    run_steps(p, io, 0, io.n_steps, true);
    p.store_final(io);
}

// ---- balanced schedule for the 2-DOF FP32 batch --------------------------------
//
// A unit is 64 instances (one warp of Pair2 threads); one warp per SM
// sub-partition already keeps the FP32 pipe busy.  With U units on P warps a
// launch of one warp per unit leaves some sub-partitions with one unit more
// than others (65,536 instances: 1,024 units on 608 sub-partitions, 2 against
// an average of 1.68).  Instead the horizon of every unit is cut in blocks
// (of ckpt_every steps, or single steps) and the U x Tb blocks are dealt to the
// P warps in order, C = max(Tb, ceil(U Tb / P)) blocks each (McNaughton's
// wrap-around rule for preemptive scheduling on identical machines).  A unit
// cut between warps m and m+1 runs its first part at the start of warp m+1,
// which then publishes the state; warp m runs the rest at its end.  Because
// C >= Tb, warp m reaches that point no earlier (in its own progress) than
// warp m+1 finishes the first part, so the wait is normally empty.  It is
// bounded all the same: after 1 s plus the time the warp has run so far it
// gives up, marks the error word and finishes the unit with NaN.
constexpr int kBalWarps = 4;                 // one warp per sub-partition; one CTA per SM
constexpr int kBalSmemBytes = 120 * 1024;    // reserves more than half the SM's shared memory

struct BalanceSched {
    int64_t units;          // U
    int64_t blocks;         // Tb, blocks per unit
    int64_t block_steps;    // steps per block
    int64_t cap;            // C, blocks per warp
    float2* xfer;           // [P][8][32] state of the unit cut at the start of warp p
    unsigned* flag;         // [P], zero before the launch
    int* err;               // error word (may be null)
    int withhold;           // test hook: publish no hand-over, so that every wait runs out
};

__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

template <class T>
__global__ void __launch_bounds__(kBalWarps * 32, 1)
rk4_pair2_balanced_kernel(const SmallSys sys, const BatchIO io, const BalanceSched sc)
{
    const int lane = threadIdx.x & 31;
    const int64_t m = (int64_t)blockIdx.x * kBalWarps + (threadIdx.x >> 5);
    const int64_t total = sc.units * sc.blocks;
    const int64_t p0 = m * sc.cap;
    const int64_t p1 = p0 + sc.cap < total ? p0 + sc.cap : total;
    const uint64_t t_start = global_ns();
    for (int64_t pos = p0; pos < p1;) {
        const int64_t u = pos / sc.blocks;
        const int64_t j0 = u * sc.blocks, j1 = j0 + sc.blocks;
        const int64_t end = j1 < p1 ? j1 : p1;
        const int64_t q = u * 64 + 2 * lane;
        const bool live = q < io.n_inst;
        T p;
        p.init(sys, io, live ? q : (io.n_inst - 1) & ~(int64_t)1);
        if (pos > j0) {
            // Started on warp m - 1's range: the first blocks of the unit, then hand over.
            const int64_t nb = end - pos;
            p.load_initial(io);
            run_steps(p, io, 0, nb * sc.block_steps, live);
            float2* dst = sc.xfer + m * 8 * 32 + lane;
#pragma unroll
            for (int i = 0; i < 8; ++i) dst[i * 32] = p.reg(i);
            __threadfence();
            __syncwarp();
            if (lane == 0 && !sc.withhold)
                asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(sc.flag + m), "r"(1u) : "memory");
        } else if (j1 > p1) {
            // Continues on warp m + 1, which runs its first blocks: wait for them, finish.
            const int64_t nb = end - pos;
            const int64_t first = sc.blocks - nb;
            const unsigned* f = sc.flag + m + 1;
            const uint64_t t_wait = global_ns();
            const uint64_t limit = 1000000000ull + (t_wait - t_start);
            unsigned seen = 0;
            for (;;) {
                asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(seen) : "l"(f) : "memory");
                if (seen) break;
                if (global_ns() - t_wait > limit) break;
                __nanosleep(256);
            }
            const bool ok = __all_sync(0xffffffffu, seen != 0);
            if (ok) {
                const float2* src = sc.xfer + (m + 1) * 8 * 32 + lane;
#pragma unroll
                for (int i = 0; i < 8; ++i) p.reg(i) = src[i * 32];
            } else {
                if (lane == 0 && sc.err) atomicExch(sc.err, 1);
                const float nan = __int_as_float(0x7fc00000);
#pragma unroll
                for (int i = 0; i < 8; ++i) p.reg(i) = f2(nan, nan);
            }
            run_steps(p, io, first * sc.block_steps, sc.blocks * sc.block_steps, live);
            if (live) p.store_final(io);
        } else {
            // The whole unit.
            p.load_initial(io);
            run_steps(p, io, 0, sc.blocks * sc.block_steps, live);
            if (live) p.store_final(io);
        }
        pos = end;
    }
}

// Which 2-DOF FP32 kernel runs: "balanced" (the default: two instances per
// thread on the balanced schedule), "pair" (two instances per thread, one warp
// per 64 instances) or "generic" (rk4_small_kernel<2>); all give the same bits.
// CHO_TWO_DOF_KERNEL overrides the default.
// FP32 s = 2 kernel forced by CHO_TWO_DOF_KERNEL (test hook: "generic", "pair"), else -1.
int two_dof_env_variant()
{
    static int v = -2;
    if (v == -2) {
        const char* e = std::getenv("CHO_TWO_DOF_KERNEL");
        v = -1;
        if (e && std::strcmp(e, "generic") == 0) v = 2;
        if (e && std::strcmp(e, "pair") == 0) v = 3;
    }
    return v;
}

}  // namespace

// Per-call device scratch (hand-over buffers, jump matrices, packed work tables) comes
// from a memory pool of the library's own that keeps up to 256 MiB when freed: the
// default pool returns freed memory to the driver at every synchronisation, and
// mapping it again cost ~0.18 ms per synchronous call.  Stream-ordered, so concurrent
// calls on other streams never share a block.
cudaError_t scratch_alloc(void** p, size_t bytes, cudaStream_t st)
{
    static std::mutex mu;
    static cudaMemPool_t pools[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaMallocAsync(p, bytes, st);
    cudaMemPool_t pool;
    {
        std::lock_guard<std::mutex> lk(mu);
        if (!pools[dev]) {
            cudaMemPoolProps props{};
            props.allocType = cudaMemAllocationTypePinned;
            props.location.type = cudaMemLocationTypeDevice;
            props.location.id = dev;
            e = cudaMemPoolCreate(&pools[dev], &props);
            if (e != cudaSuccess) {
                pools[dev] = nullptr;
                return e;
            }
            uint64_t keep = (uint64_t)256 << 20;
            e = cudaMemPoolSetAttribute(pools[dev], cudaMemPoolAttrReleaseThreshold, &keep);
            if (e != cudaSuccess) return e;
        }
        pool = pools[dev];
    }
    return cudaMallocFromPoolAsync(p, bytes, pool, st);
}

namespace {

template <class T>
cudaError_t launch_pair2(const SmallSys& sys, const BatchIO& io, cudaStream_t st)
{
    const int64_t threads = (io.n_inst + 1) / 2;
    const int64_t blocks = (threads + kPairThreads - 1) / kPairThreads;
    if (blocks <= 0) return cudaSuccess;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidValue;
    rk4_pair2_kernel<T><<<(unsigned)blocks, kPairThreads, 0, st>>>(sys, io);
    return cudaGetLastError();
}

// The balanced schedule when it helps (more units than warps, a cooperative
// launch is available); otherwise the one-launch pair kernel.  The hand-over
// buffer and flags are taken from the stream-ordered allocator and freed after
// the kernel on the same stream, so concurrent calls on other streams do not
// share them.
template <class T>
cudaError_t launch_pair2_balanced(const SmallSys& sys, const BatchIO& io, cudaStream_t st)
{
    int dev = 0, sms = 0, coop = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    if (e != cudaSuccess) return e;
    const int64_t P = (int64_t)sms * kBalWarps;
    const int64_t U = (io.n_inst + 63) / 64;
    const bool ckpt = io.ckpt_every > 0 && io.x_traj;
    // blocks of ckpt_every steps, else of one update (one step, or poly_jump steps)
    const int64_t g = ckpt ? io.ckpt_every : (io.poly_jump > 0 ? io.poly_jump : 1);
    const int64_t Tb = io.n_steps / g;
    if (!coop || U <= P || Tb <= 0 || Tb > ((int64_t)1 << 62) / U) return launch_pair2<T>(sys, io, st);
    auto kern = rk4_pair2_balanced_kernel<T>;
    static bool attr_set[2][64] = {};
    bool& done = attr_set[std::is_same<T, Pair2>::value ? 0 : 1][dev < 64 ? dev : 63];
    if (!done) {
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, kBalSmemBytes);
        if (e != cudaSuccess) return e;
        done = true;
    }
    BalanceSched sc{};
    sc.units = U;
    sc.blocks = Tb;
    sc.block_steps = g;
    sc.cap = std::max(Tb, (U * Tb + P - 1) / P);
    sc.err = sys.err;
    const char* hook = std::getenv("CHO_TEST_WITHHOLD_HANDOVER");
    sc.withhold = hook && hook[0] == '1' ? 1 : 0;
    const size_t xfer_bytes = (size_t)P * 8 * 32 * sizeof(float2);
    void* buf = nullptr;
    e = scratch_alloc(&buf, xfer_bytes + (size_t)P * sizeof(unsigned), st);
    if (e != cudaSuccess) return e;
    sc.xfer = (float2*)buf;
    sc.flag = (unsigned*)((char*)buf + xfer_bytes);
    e = cudaMemsetAsync(sc.flag, 0, (size_t)P * sizeof(unsigned), st);
    if (e == cudaSuccess) {
        SmallSys a0 = sys;
        BatchIO a1 = io;
        void* args[] = {&a0, &a1, &sc};
        e = cudaLaunchCooperativeKernel((const void*)kern, dim3((unsigned)sms), dim3(kBalWarps * 32), args,
                                        (size_t)kBalSmemBytes, st);
    }
    const cudaError_t ef = cudaFreeAsync(buf, st);
    return e != cudaSuccess ? e : ef;
}


// ---- double-FP32: s <= 32 systems with about 48 significant bits on the FP32 pipe ----
//
// The step is the FP64 mode's stage form (rk4_small_kernel<S, true>), operation for
// operation, in the pair arithmetic of rk4_common.cuh (dw): the same lanes per instance
// and rows per lane, and the same column order of B x (S <= 4: one lane per instance,
// each row from its diagonal onwards; S >= 8: lane groups that exchange x as (hi, lo)
// through shared memory, each row from column 0).  B, h, h/2 and h/6 are split from
// FP64.  Batch form only.
template <int S>
__global__ void __launch_bounds__(kDwThreads) rk4_dw_small_kernel(const SmallSys sys, const BatchIO io)
{
    constexpr int R = rows_per_lane(S);
    constexpr int G = S / R;                      // lanes per instance
    constexpr int GPB = kDwThreads / G;           // groups per block
    __shared__ float2 xch[G > 1 ? 2 : 1][G > 1 ? GPB : 1][G > 1 ? S : 1];

    const int64_t tid = (int64_t)blockIdx.x * kDwThreads + threadIdx.x;
    const int64_t q = tid / G;
    const int g = (int)(tid % G);
    const int grp = threadIdx.x / G;
    const unsigned lane = threadIdx.x & 31u;
    const unsigned gmask = (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << (lane & ~(unsigned)(G - 1)));
    if (q >= io.n_inst) return;                   // whole groups leave together

    const int64_t set = sys.per_inst_sys ? q : 0;
    const double* Bq = sys.B64 + set * S * S;     // padded [S][S]
    dw b[R][S];
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
        for (int j = 0; j < S; ++j) b[r][j] = dw_split(Bq[(g * R + r) * S + j]);
    const double hd = io.h[io.h_per_inst ? q : 0];
    const dw h = dw_split(hd), h2 = dw_split(0.5 * hd), h6 = dw_split(hd / 6.0);
    const int s = sys.s;
    dw x[R], v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int row = g * R + r;
        x[r] = dw_split(row < s ? io.x0[q * s + row] : 0.0);
        v[r] = dw_split(row < s ? io.v0[q * s + row] : 0.0);
    }
    int buf = 0;
    // a = -(B xs): the first product rounded (the FP64 mode's fma onto zero), then fmas
    auto accel = [&](const dw (&xs)[R], dw (&a)[R]) {
        if constexpr (G == 1) {
#pragma unroll
            for (int r = 0; r < R; ++r) {
                dw t = dw_mul(b[r][r], xs[r]);
#pragma unroll
                for (int jj = 1; jj < S; ++jj) t = dw_fma(b[r][(r + jj) % S], xs[(r + jj) % S], t);
                a[r] = dw_neg(t);
            }
        } else {
#pragma unroll
            for (int r = 0; r < R; ++r) xch[buf][grp][g * R + r] = make_float2(xs[r].hi, xs[r].lo);
            __syncwarp(gmask);
#pragma unroll
            for (int r = 0; r < R; ++r) {
                float2 c = xch[buf][grp][0];
                dw t = dw_mul(b[r][0], dw{c.x, c.y});
#pragma unroll
                for (int j = 1; j < S; ++j) {
                    c = xch[buf][grp][j];
                    t = dw_fma(b[r][j], dw{c.x, c.y}, t);
                }
                a[r] = dw_neg(t);
            }
            buf ^= 1;
        }
    };
    const int64_t every = io.ckpt_every > 0 ? io.ckpt_every : (io.n_steps > 0 ? io.n_steps : 1);
    int64_t ck = 0;
    for (int64_t done = 0; done < io.n_steps; done += every) {
        repeat_steps(every, [&]() {
            dw a[R], xs[R], kx[R], kv[R], vs[R];
            accel(x, a);
#pragma unroll
            for (int r = 0; r < R; ++r) {
                kx[r] = v[r];
                kv[r] = a[r];
                xs[r] = dw_fma(h2, v[r], x[r]);
                vs[r] = dw_fma(h2, a[r], v[r]);
            }
            accel(xs, a);
#pragma unroll
            for (int r = 0; r < R; ++r) {
                kx[r] = dw_add(dw_twice(vs[r]), kx[r]);
                kv[r] = dw_add(dw_twice(a[r]), kv[r]);
                xs[r] = dw_fma(h2, vs[r], x[r]);
                vs[r] = dw_fma(h2, a[r], v[r]);
            }
            accel(xs, a);
#pragma unroll
            for (int r = 0; r < R; ++r) {
                kx[r] = dw_add(dw_twice(vs[r]), kx[r]);
                kv[r] = dw_add(dw_twice(a[r]), kv[r]);
                xs[r] = dw_fma(h, vs[r], x[r]);
                vs[r] = dw_fma(h, a[r], v[r]);
            }
            accel(xs, a);
#pragma unroll
            for (int r = 0; r < R; ++r) {
                kx[r] = dw_add(kx[r], vs[r]);
                kv[r] = dw_add(kv[r], a[r]);
                x[r] = dw_fma(h6, kx[r], x[r]);
                v[r] = dw_fma(h6, kv[r], v[r]);
            }
        });
        if (io.ckpt_every > 0 && io.x_traj) {
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int row = g * R + r;
                if (row >= s) continue;
                const int64_t o = (q * io.n_ck + ck) * s + row;
                io.x_traj[o] = dw_value(x[r]);
                if (io.v_traj) io.v_traj[o] = dw_value(v[r]);
            }
        }
        ++ck;
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int row = g * R + r;
        if (row >= s) continue;
        io.x_out[q * s + row] = dw_value(x[r]);
        io.v_out[q * s + row] = dw_value(v[r]);
    }
}

template <int S>
cudaError_t launch_dw_one(const SmallSys& sys, const BatchIO& io, cudaStream_t st)
{
    constexpr int G = S / rows_per_lane(S);
    const int64_t blocks = (io.n_inst * G + kDwThreads - 1) / kDwThreads;
    if (blocks <= 0) return cudaSuccess;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidValue;
    rk4_dw_small_kernel<S><<<(unsigned)blocks, kDwThreads, 0, st>>>(sys, io);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_rk4_small(const SmallSys& sys, const BatchIO& io, bool fp64, cudaStream_t st)
{
    if (io.poly_jump > 0 && sys.s != 2) {        // polynomial form, any other s <= 32
        if (io.n_inst == 0) return cudaSuccess;
        switch (sys.S) {
            case 2: return launch_small_poly<2>(sys, io, fp64, st);
            case 4: return launch_small_poly<4>(sys, io, fp64, st);
            case 8: return launch_small_poly<8>(sys, io, fp64, st);
            case 16: return launch_small_poly<16>(sys, io, fp64, st);
            case 32: return launch_small_poly<32>(sys, io, fp64, st);
            default: return cudaErrorInvalidValue;
        }
    }
    if (io.poly_jump > 0) {                      // polynomial form, s = 2
        const int64_t blocks = (io.n_inst + 63) / 64;
        if (blocks <= 0) return cudaSuccess;
        if (blocks > 0x7fffffffLL) return cudaErrorInvalidValue;
        // the jump matrices live for this call only, in stream order
        void* buf = nullptr;
        cudaError_t e = scratch_alloc(&buf, (size_t)io.n_inst * 16 * sizeof(double), st);
        if (e != cudaSuccess) return e;
        BatchIO pio = io;
        pio.poly_E = (const double*)buf;
        poly_setup_kernel<<<(unsigned)blocks, 64, 0, st>>>(sys, io, fp64, (double*)buf);
        e = cudaGetLastError();
        if (e == cudaSuccess) {
            if (fp64) {
                rk4_poly64_kernel<<<(unsigned)blocks, 64, 0, st>>>(sys, pio);
                e = cudaGetLastError();
            } else {
                const int pv = two_dof_env_variant() >= 0 ? two_dof_env_variant() : sys.variant;
                e = pv == 3 ? launch_pair2<Pair2Poly>(sys, pio, st) : launch_pair2_balanced<Pair2Poly>(sys, pio, st);
            }
        }
        const cudaError_t ef = cudaFreeAsync(buf, st);
        return e != cudaSuccess ? e : ef;
    }
    // the test hook, else the caller's (tuned) choice, else the balanced kernel
    const int variant = two_dof_env_variant() >= 0 ? two_dof_env_variant() : (sys.variant >= 0 ? sys.variant : 0);
    // s = 1 is also padded to S = 2 but keeps the generic layout
    if (sys.s == 2 && !fp64 && variant == 3) return launch_pair2<Pair2>(sys, io, st);
    if (sys.s == 2 && !fp64 && variant == 0) return launch_pair2_balanced<Pair2>(sys, io, st);
    return dispatch<BatchSrc>(sys.S, fp64, io.n_inst, st, [&](auto& s) {
        s.sys = sys;
        s.io = io;
    });
}

cudaError_t launch_rk4_small_dw(const SmallSys& sys, const BatchIO& io, cudaStream_t st)
{
    if (!sys.B64) return cudaErrorInvalidValue;
    switch (sys.S) {
        case 2: return launch_dw_one<2>(sys, io, st);
        case 4: return launch_dw_one<4>(sys, io, st);
        case 8: return launch_dw_one<8>(sys, io, st);
        case 16: return launch_dw_one<16>(sys, io, st);
        case 32: return launch_dw_one<32>(sys, io, st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_rk4_small_slots(int S, const SlotIO& io, bool fp64, cudaStream_t st)
{
    return dispatch<SlotSrc>(S, fp64, io.n_inst, st, [&](auto& s) { s.io = io; });
}

// Instances of padded size S the slot kernel holds resident at once on this device.
int small_slot_resident(int S, bool fp64)
{
    int n = 0, lanes = 1;
    cudaError_t e = cudaErrorInvalidValue;
#define CHO_RES_CASE(SV)                                                                                           \
    case SV:                                                                                                       \
        lanes = SV / rows_per_lane(SV);                                                                            \
        e = fp64 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, rk4_small_kernel<SV, true, SlotSrc<true, SV>>, \
                                                                  kSmallThreads, 0)                                \
                 : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, rk4_small_kernel<SV, false, SlotSrc<false, SV>>, \
                                                                  kSmallThreads, 0);                               \
        break;
    switch (S) {
        CHO_RES_CASE(2)
        CHO_RES_CASE(4)
        CHO_RES_CASE(8)
        CHO_RES_CASE(16)
        CHO_RES_CASE(32)
        default: break;
    }
#undef CHO_RES_CASE
    int dev = 0, sms = 0;
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return 0;
    }
    return n * sms * (kSmallThreads / lanes);
}

cudaError_t launch_rk4_small_persist(int S, const PersistIO& pio, bool fp64, int grid, cudaStream_t st)
{
#define CHO_PERSIST_CASE(SV)                                                                            \
    case SV:                                                                                            \
        if (fp64) rk4_small_persist_kernel<SV, true><<<grid, kSmallThreads, 0, st>>>(pio);             \
        else rk4_small_persist_kernel<SV, false><<<grid, kSmallThreads, 0, st>>>(pio);                 \
        return cudaGetLastError();
    if (grid <= 0) return cudaErrorInvalidValue;
    switch (S) {
        CHO_PERSIST_CASE(2)
        CHO_PERSIST_CASE(4)
        CHO_PERSIST_CASE(8)
        CHO_PERSIST_CASE(16)
        CHO_PERSIST_CASE(32)
        default: return cudaErrorInvalidValue;
    }
#undef CHO_PERSIST_CASE
}

}  // namespace cho
