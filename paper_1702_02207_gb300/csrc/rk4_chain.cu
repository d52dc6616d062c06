// rk4_chain.cu -- classical RK4 for fixed-free spring chains (eq. 2 generalised).
//
// Eq. 2 written per mass gives the acceleration from the spring extensions
// e_i = x_i - x_{i-1} (e_0 = x_0, the wall spring):
//     a_i = -g_i e_i + u_i e_{i+1},   g_i = C_i / m_i,  u_i = C_{i+1} / m_i,
// with u_{s-1} = 0 (the free end).  This is B x for the tridiagonal
// B = M^{-1} K, evaluated in the factored form M^{-1} D^T diag(C) D x (D the
// difference operator): neighbouring displacements are subtracted first, which
// is exact when they are close, so slow modes of stiff chains keep their
// accuracy in FP32.
//
// One CTA integrates one instance for the whole horizon.  Thread t owns P
// consecutive DOFs [tP, tP + P) with their coefficients and state in
// registers.  Per stage it needs one displacement from each neighbouring
// thread: every thread stores its first and last displacement in a
// double-buffered shared-memory slot array and, after the stage's single
// __syncthreads, loads its neighbours' slots (zero slots stand for the wall
// and for the space past the free end).  Stage order and the state update are
// those of rk4_small.cu.
//
// Kernels: rk4_chain_kernel (FP64 at every P; FP32 at P = 1), rk4_chain_pk_kernel
// (FP32 at P >= 2: the same operations on packed pairs of DOFs, the same bits) and
// rk4_chain_dw_kernel (double-FP32, CHO_FP32X2).
#include "cho_internal.h"
#include "persist.cuh"
#include "rk4_common.cuh"
#include "../../include/cho.h"

namespace cho {
namespace {

constexpr int kChainUnroll = 2;   // steps per pass of the packed kernel's step loop

// Batch form: coefficient set per instance or shared; FP64 in and out.
template <bool F64>
struct ChainBatchSrc {
    ChainSys sys;
    BatchIO io;
    using Real = std::conditional_t<F64, double, float>;

    __device__ int s(int64_t) const { return sys.s; }
    __device__ double h(int64_t q) const { return io.h[io.h_per_inst ? q : 0]; }
    __device__ int64_t steps(int64_t) const { return io.n_steps; }
    __device__ int64_t ckpt_every() const { return io.ckpt_every; }
    __device__ const void* coef(int64_t q) const
    {
        const int64_t set = sys.per_inst_sys ? q : 0;
        if constexpr (F64) return sys.C64 + set * 2 * sys.s;
        else return sys.C32 + set * 4 * sys.s;
    }
    // FP32: v is held as the scaled velocity u = (h/6) v (scaled_velocity)
    __device__ void load(int64_t q, int i, Real& x, Real& v, float& cx, float& cv) const
    {
        const double xd = io.x0[q * sys.s + i];
        const double vd = F64 ? io.v0[q * sys.s + i] : scaled_velocity(io.v0[q * sys.s + i], h(q));
        x = (Real)xd;
        v = (Real)vd;
        cx = F64 ? 0.f : (float)(xd - (double)x);
        cv = F64 ? 0.f : (float)(vd - (double)v);
    }
    __device__ double vout(int64_t q, Real v, float cv) const
    {
        const double u = (double)v + (double)cv;
        return F64 ? u : unscaled_velocity(u, h(q));
    }
    __device__ void checkpoint(int64_t q, int64_t ck, int i, Real x, Real v, float cx, float cv) const
    {
        if (io.x_traj == nullptr) return;
        const int64_t o = (q * io.n_ck + ck) * sys.s + i;
        io.x_traj[o] = (double)x + (double)cx;
        if (io.v_traj) io.v_traj[o] = vout(q, v, cv);
    }
    __device__ void store(int64_t q, int i, Real x, Real v, float cx, float cv) const
    {
        io.x_out[q * sys.s + i] = (double)x + (double)cx;
        io.v_out[q * sys.s + i] = vout(q, v, cv);
    }
    __device__ void finish(int64_t, int64_t, bool) const {}
};

// Slot form: state block [x(s), v(s), cx(s), cv(s)] in kernel precision (FP32: the
// scaled velocity in place of v, converted by the serving engine).  FRESH (persistent
// kernels): table and ids in mapped host memory read with volatile loads, state blocks
// through L2 only, finished slots to the completion ring (as SlotSrc in rk4_small.cu).
template <bool F64, bool FRESH = false>
struct ChainSlotSrc {
    SlotIO io;
    const PersistIO* pio = nullptr;
    using Real = std::conditional_t<F64, double, float>;

    __device__ int32_t id(int64_t q) const
    {
        if constexpr (FRESH) return ((const volatile int32_t*)io.slot_ids)[q];
        else return io.slot_ids[q];
    }
    __device__ const SlotDesc& d(int64_t q) const { return io.slots[io.slot_ids[q]]; }
    __device__ const volatile SlotDesc& vd(int64_t q) const { return ((const volatile SlotDesc*)io.slots)[id(q)]; }
    __device__ int s(int64_t q) const
    {
        if constexpr (FRESH) return vd(q).s;
        else return d(q).s;
    }
    __device__ double h(int64_t q) const
    {
        if constexpr (FRESH) return vd(q).h;
        else return d(q).h;
    }
    __device__ int64_t steps(int64_t q) const
    {
        int64_t rem;
        if constexpr (FRESH) rem = vd(q).remaining;
        else rem = d(q).remaining;
        return rem < io.chunk ? rem : io.chunk;
    }
    __device__ int64_t ckpt_every() const { return 0; }
    __device__ const void* coef(int64_t q) const
    {
        if constexpr (FRESH) return vd(q).coef;
        else return d(q).coef;
    }
    __device__ Real* state(int64_t q) const
    {
        if constexpr (FRESH) return (Real*)vd(q).state;
        else return (Real*)d(q).state;
    }
    __device__ Real ld(const Real* p) const
    {
        if constexpr (FRESH) return __ldcg(p);
        else return *p;
    }
    __device__ void load(int64_t q, int i, Real& x, Real& v, float& cx, float& cv) const
    {
        const int sz = s(q);
        const Real* st = state(q);
        x = ld(st + i);
        v = ld(st + sz + i);
        if constexpr (F64) {
            cx = cv = 0.f;
        } else {
            cx = ld(st + 2 * sz + i);
            cv = ld(st + 3 * sz + i);
        }
    }
    __device__ void checkpoint(int64_t, int64_t, int, Real, Real, float, float) const {}
    __device__ void store(int64_t q, int i, Real x, Real v, float cx, float cv) const
    {
        const int sz = s(q);
        Real* st = state(q);
        st[i] = x;
        st[sz + i] = v;
        if constexpr (!F64) {
            st[2 * sz + i] = cx;
            st[3 * sz + i] = cv;
        }
    }
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

// One instance per CTA: the work of instance q (the kernel's CTA blockIdx.x, or an item
// of a persistent kernel's generation).
template <int P, bool F64, int MAXT, class Src>
__device__ __forceinline__ void rk4_chain_body(const Src& src, int64_t q)
{
    using Real = std::conditional_t<F64, double, float>;
    // edge displacements, [buffer][slot]: thread t stores its last DOF in edge_last[.][t + 1]
    // and its first in edge_first[.][t]; edge_last[.][0] (the wall) and
    // edge_first[.][blockDim.x] (past the free end) stay zero
    __shared__ Real edge_last[2][MAXT + 1];
    __shared__ Real edge_first[2][MAXT + 1];
    __shared__ int any_bad;

    const int t = threadIdx.x;
    const int s = src.s(q);
    const int i0 = t * P;
    if (t == 0) {
        any_bad = 0;
        edge_last[0][0] = edge_last[1][0] = (Real)0;
        edge_first[0][blockDim.x] = edge_first[1][blockDim.x] = (Real)0;
    }
    __syncthreads();

    // coefficients of DOFs i0 .. i0+P-1 (zero beyond s: padded DOFs stay at rest)
    Real gh[P], uh[P];
    float gl[P], ul[P];
    const void* cb = src.coef(q);
#pragma unroll
    for (int p = 0; p < P; ++p) {
        const int i = i0 + p;
        const bool in = i < s;
        if constexpr (F64) {
            const double* c = (const double*)cb;
            gh[p] = in ? c[i] : 0.0;
            uh[p] = in ? c[s + i] : 0.0;
            gl[p] = ul[p] = 0.f;
        } else {
            const float* c = (const float*)cb;
            gh[p] = in ? c[i] : 0.f;
            uh[p] = in ? c[s + i] : 0.f;
            gl[p] = in ? c[2 * s + i] : 0.f;
            ul[p] = in ? c[3 * s + i] : 0.f;
            scaled_coef(gh[p], gl[p], src.h(q));     // g'' = h^2/36 g, u'' = h^2/36 u
            scaled_coef(uh[p], ul[p], src.h(q));
        }
    }

    const StepSize<F64> hs(src.h(q));
    // stage constants: FP64 h/2, h; FP32 (scaled velocity) 3, 6
    const Real c_half = F64 ? hs.h2 : (Real)3, c_full = F64 ? hs.h : (Real)6;
    Real x[P], v[P];
    float cx[P], cv[P];
#pragma unroll
    for (int p = 0; p < P; ++p) {
        const int i = i0 + p;
        if (i < s) {
            src.load(q, i, x[p], v[p], cx[p], cv[p]);
        } else {
            x[p] = v[p] = 0;
            cx[p] = cv[p] = 0.f;
        }
    }

    int buf = 0;
    // FP32: the lo parts of g and u multiply the stage-1 extensions and the sum is
    // reused by stages 2-4 (frozen lo, as in rk4_small.cu).
    float lo1[P];
    // the neighbours' edge displacements come through shared memory: one store and one
    // load per side and stage, the zero slots standing in for the wall and the free end
    auto accel = [&](const Real (&xs)[P], Real (&acc)[P], bool first) {
        edge_last[buf][t + 1] = xs[P - 1];
        edge_first[buf][t] = xs[0];
        __syncthreads();
        const Real left = edge_last[buf][t];
        const Real right = edge_first[buf][t + 1];
        buf ^= 1;
        Real e[P + 1];                       // spring extensions e_{i0} .. e_{i0+P}
        e[0] = xs[0] - left;
#pragma unroll
        for (int p = 1; p < P; ++p) e[p] = xs[p] - xs[p - 1];
        e[P] = right - xs[P - 1];
#pragma unroll
        for (int p = 0; p < P; ++p) {
            Real a;
            if constexpr (F64) {
                a = fmar(uh[p], e[p + 1], -gh[p] * e[p]);
            } else {
                if (first) lo1[p] = fmaf(ul[p], e[p + 1], -gl[p] * e[p]);
                a = fmaf(uh[p], e[p + 1], fmaf(-gh[p], e[p], lo1[p]));
            }
            acc[p] = a;
        }
    };

    const int64_t n = src.steps(q);
    const int64_t every = src.ckpt_every() > 0 ? src.ckpt_every() : (n > 0 ? n : 1);
    int64_t ck = 0;
    for (int64_t done = 0; done < n; done += every) {
        repeat_steps(every, [&]() {
            Real a[P], xs[P], kx[P], kv[P], vs[P];
            accel(x, a, true);
#pragma unroll
            for (int p = 0; p < P; ++p) {
                if constexpr (F64) kx[p] = v[p];
                else kx[p] = fmar((Real)2, v[p], cx[p]);   // FP32: the x sum starts on its compensation
                kv[p] = a[p];
                xs[p] = fmar(c_half, v[p], x[p]);
                vs[p] = fmar(c_half, a[p], v[p]);
            }
            accel(xs, a, false);
#pragma unroll
            for (int p = 0; p < P; ++p) {
                kx[p] = fmar((Real)2, vs[p], kx[p]);
                kv[p] = fmar((Real)2, a[p], kv[p]);
                xs[p] = fmar(c_half, vs[p], x[p]);
                vs[p] = fmar(c_half, a[p], v[p]);
            }
            accel(xs, a, false);
#pragma unroll
            for (int p = 0; p < P; ++p) {
                kx[p] = fmar((Real)2, vs[p], kx[p]);
                kv[p] = fmar((Real)2, a[p], kv[p]);
                xs[p] = fmar(c_full, vs[p], x[p]);
                // FP32: the stage-4 velocity v + 6 a3 enters only the x sum, which takes 2v + 6 a3
                if constexpr (F64) vs[p] = fmar(c_full, a[p], v[p]);
                else kx[p] = fmar(c_full, a[p], kx[p]);
            }
            accel(xs, a, false);
#pragma unroll
            for (int p = 0; p < P; ++p) {
                if constexpr (F64) {
                    kx[p] = addr(kx[p], vs[p]);
                    kv[p] = addr(kv[p], a[p]);
                    state_update<true>(x[p], cx[p], kx[p], hs);
                    state_update<true>(v[p], cv[p], kv[p], hs);
                } else {
                    kv[p] = addr(kv[p], a[p]);
                    comp_add_folded(x[p], cx[p], kx[p]);
                    comp_add(v[p], cv[p], kv[p]);
                }
            }
        });
        if (src.ckpt_every() > 0) {
#pragma unroll
            for (int p = 0; p < P; ++p)
                if (i0 + p < s) src.checkpoint(q, ck, i0 + p, x[p], v[p], cx[p], cv[p]);
            ++ck;
        }
    }
    bool bad = false;
#pragma unroll
    for (int p = 0; p < P; ++p) {
        if (i0 + p < s) {
            src.store(q, i0 + p, x[p], v[p], cx[p], cv[p]);
            bad |= !(isfinite((double)x[p]) && isfinite((double)v[p]));
        }
    }
    if (bad) any_bad = 1;
    __syncthreads();
    if (t == 0) src.finish(q, n, any_bad != 0);
}

template <int P, bool F64, int MAXT, class Src>
__global__ void __launch_bounds__(MAXT) rk4_chain_kernel(const Src src)
{
    rk4_chain_body<P, F64, MAXT>(src, blockIdx.x);
}

// FP32 with P >= 2 DOFs per thread in packed FP32x2 arithmetic: the step of
// rk4_chain_kernel<P, false>, every packed operation rounding each lane as the scalar
// one does (the same bits), with DOF p of the thread in lane .x and DOF p + P/2 in
// lane .y of pair p.  That pairing keeps the spring extensions on aligned pairs,
// E_k = (e_k, e_{k+P/2}) = X_k - X_{k-1}, and leaves two pairs per stage to assemble
// from scalars: (left neighbour, x_{P/2-1}) for E_0 and (x_{P/2}, right neighbour)
// for E_{P/2}.  Packing halves the FP32 instructions the stage issues.
//
// PAIR: the four stage accelerations are formed two at a time.  For x'' = -B x the
// stage-2 displacement x + (h/2) v does not depend on a1, nor the stage-4
// displacement x + h (v + (h/2) a2) on a3, so {a1, a2} and then {a3, a4} are
// independent pairs: one neighbour exchange and one barrier serve two stages, and
// each thread has twice the independent work between barriers.  Every value keeps
// its operations and their order, so the bits are those of the stage-by-stage form.
// The paired form needs about 2P more registers; CTAs wider than 256 threads (64
// registers a thread) run stage by stage.
template <int P, bool PAIR, int MAXT, class Src>
__device__ __forceinline__ void rk4_chain_pk_body(const Src& src, int64_t q)
{
    static_assert(P >= 2 && P % 2 == 0, "pairs of DOFs");
    constexpr int H = P / 2;
    constexpr int NS = PAIR ? 2 : 1;          // stages evaluated per exchange
    using Edge = std::conditional_t<PAIR, float2, float>;   // one value per stage in flight
    // edge displacements, [buffer][slot]: thread t stores its last DOF in edge_last[.][t + 1]
    // and its first in edge_first[.][t]; edge_last[.][0] (the wall) and
    // edge_first[.][blockDim.x] (past the free end) stay zero
    __shared__ Edge edge_last[2][MAXT + 1];
    __shared__ Edge edge_first[2][MAXT + 1];
    __shared__ int any_bad;

    const int t = threadIdx.x;
    const int s = src.s(q);
    const int i0 = t * P;
    if (t == 0) {
        any_bad = 0;
        edge_last[0][0] = edge_last[1][0] = Edge{};
        edge_first[0][blockDim.x] = edge_first[1][blockDim.x] = Edge{};
    }
    __syncthreads();

    // coefficients, negated g (zero beyond s: padded DOFs stay at rest)
    float2 ngh[H], uh[H], ngl[H], ul[H];
    {
        const float* c = (const float*)src.coef(q);
        float gh_[P], uh_[P], gl_[P], ul_[P];
#pragma unroll
        for (int p = 0; p < P; ++p) {
            const int i = i0 + p;
            const bool in = i < s;
            gh_[p] = in ? c[i] : 0.f;
            uh_[p] = in ? c[s + i] : 0.f;
            gl_[p] = in ? c[2 * s + i] : 0.f;
            ul_[p] = in ? c[3 * s + i] : 0.f;
            scaled_coef(gh_[p], gl_[p], src.h(q));     // g'' = h^2/36 g, u'' = h^2/36 u
            scaled_coef(uh_[p], ul_[p], src.h(q));
        }
#pragma unroll
        for (int k = 0; k < H; ++k) {
            ngh[k] = make_float2(-gh_[k], -gh_[k + H]);
            uh[k] = make_float2(uh_[k], uh_[k + H]);
            ngl[k] = make_float2(-gl_[k], -gl_[k + H]);
            ul[k] = make_float2(ul_[k], ul_[k + H]);
        }
    }
    const float2 m1 = make_float2(-1.f, -1.f), two = make_float2(2.f, 2.f);
    const float2 three = make_float2(3.f, 3.f), six = make_float2(6.f, 6.f);
    float2 x[H], v[H], cx[H], cv[H];
#pragma unroll
    for (int k = 0; k < H; ++k) {
        float a[2], b[2], ca[2], cb[2];
#pragma unroll
        for (int l = 0; l < 2; ++l) {
            const int i = i0 + k + l * H;
            if (i < s) {
                src.load(q, i, a[l], b[l], ca[l], cb[l]);
            } else {
                a[l] = b[l] = ca[l] = cb[l] = 0.f;
            }
        }
        x[k] = make_float2(a[0], a[1]);
        v[k] = make_float2(b[0], b[1]);
        cx[k] = make_float2(ca[0], ca[1]);
        cv[k] = make_float2(cb[0], cb[1]);
    }

    int buf = 0;
    float2 lo1[H];   // lo parts of g and u times the stage-1 extensions (frozen lo)
    auto edge_of = [](const Edge& v, int j) -> float {
        if constexpr (PAIR) return j == 0 ? v.x : v.y;
        else return v;
    };
    // Accelerations of NS stages, xs[j] their displacements (xs[0] = x when first).
    // The neighbours' edge displacements come through shared memory (one store and one
    // load per side for the NS stages).  The extensions and accelerations of the interior
    // pairs use only this thread's displacements: they are formed before the barrier.
    auto accel = [&](const float2 (&xs)[NS][H], float2 (&acc)[NS][H], bool first) {
        if constexpr (PAIR) {
            edge_last[buf][t + 1] = make_float2(xs[0][H - 1].y, xs[1][H - 1].y);
            edge_first[buf][t] = make_float2(xs[0][0].x, xs[1][0].x);
        } else {
            edge_last[buf][t + 1] = xs[0][H - 1].y;
            edge_first[buf][t] = xs[0][0].x;
        }
        float2 e[NS][H + 1];                 // e[j][k] = (e_k, e_{k+H}); e[j][H] = (e_H, e_P)
#pragma unroll
        for (int j = 0; j < NS; ++j)
#pragma unroll
            for (int k = 1; k < H; ++k) e[j][k] = __ffma2_rn(xs[j][k - 1], m1, xs[j][k]);
#pragma unroll
        for (int k = 1; k + 1 < H; ++k) {
            if (first) lo1[k] = __ffma2_rn(ul[k], e[0][k + 1], __fmul2_rn(ngl[k], e[0][k]));
#pragma unroll
            for (int j = 0; j < NS; ++j)
                acc[j][k] = __ffma2_rn(uh[k], e[j][k + 1], __ffma2_rn(ngh[k], e[j][k], lo1[k]));
        }
        __syncthreads();
        const Edge l = edge_last[buf][t];          // thread t - 1's last DOF (zero at the wall)
        const Edge r = edge_first[buf][t + 1];     // thread t + 1's first DOF
        buf ^= 1;
        // the two boundary pairs (e_0, e_H) and (e_H, e_P) from scalar differences (the
        // values of the packed lanes; no pair of operands to assemble)
#pragma unroll
        for (int j = 0; j < NS; ++j) {
            const float e0 = __fsub_rn(xs[j][0].x, edge_of(l, j));
            const float eH = __fsub_rn(xs[j][0].y, xs[j][H - 1].x);
            const float eP = __fsub_rn(edge_of(r, j), xs[j][H - 1].y);
            e[j][0] = make_float2(e0, eH);
            e[j][H] = make_float2(eH, eP);
        }
#pragma unroll
        for (int k = 0; k < H; k += (H > 1 ? H - 1 : 1)) {
            if (first) lo1[k] = __ffma2_rn(ul[k], e[0][k + 1], __fmul2_rn(ngl[k], e[0][k]));
#pragma unroll
            for (int j = 0; j < NS; ++j)
                acc[j][k] = __ffma2_rn(uh[k], e[j][k + 1], __ffma2_rn(ngh[k], e[j][k], lo1[k]));
        }
    };
    // compensated x += y, y already holding the compensation (comp_add_folded)
    auto comp_add2_folded = [&](float2& xx, float2& ee, float2 y) {
        const float2 tt = __fadd2_rn(xx, y);
        ee = __ffma2_rn(__ffma2_rn(xx, m1, tt), m1, y);     // y - (t - x)
        xx = tt;
    };
    // compensated x += k (comp_add)
    auto comp_add2 = [&](float2& xx, float2& ee, float2 kk) { comp_add2_folded(xx, ee, __fadd2_rn(kk, ee)); };

    const int64_t n = src.steps(q);
    const int64_t every = src.ckpt_every() > 0 ? src.ckpt_every() : (n > 0 ? n : 1);
    int64_t ck = 0;
    for (int64_t done = 0; done < n; done += every) {
        // The x sum starts on its compensation and takes the stage-4 velocity v + 6 a3 as
        // 2v + 6 a3 (the stage-4 velocity enters nothing else): kx = 2v + cx + 2 vs2 + 2 vs3
        // + 6 a3, and the update adds it to x without a further sum (comp_add_folded).
        repeat_steps<kChainUnroll>(every, [&]() {
            float2 xs[NS][H], a[NS][H], kx[H], kv[H];
            if constexpr (PAIR) {
                // stages 1 and 2: a1 = A(x), a2 = A(x + 3v)
#pragma unroll
                for (int k = 0; k < H; ++k) {
                    xs[0][k] = x[k];
                    xs[1][k] = __ffma2_rn(three, v[k], x[k]);
                }
                accel(xs, a, true);
                // stages 3 and 4: a3 = A(x + 3 vs2), a4 = A(x + 6 vs3)
#pragma unroll
                for (int k = 0; k < H; ++k) {
                    const float2 vs2 = __ffma2_rn(three, a[0][k], v[k]);
                    const float2 vs3 = __ffma2_rn(three, a[1][k], v[k]);
                    kx[k] = __ffma2_rn(two, vs2, __ffma2_rn(two, v[k], cx[k]));
                    kv[k] = __ffma2_rn(two, a[1][k], a[0][k]);
                    kx[k] = __ffma2_rn(two, vs3, kx[k]);
                    xs[0][k] = __ffma2_rn(three, vs2, x[k]);
                    xs[1][k] = __ffma2_rn(six, vs3, x[k]);
                }
                accel(xs, a, false);
#pragma unroll
                for (int k = 0; k < H; ++k) {
                    kx[k] = __ffma2_rn(six, a[0][k], kx[k]);
                    kv[k] = __ffma2_rn(two, a[0][k], kv[k]);
                    kv[k] = __fadd2_rn(kv[k], a[1][k]);
                    comp_add2_folded(x[k], cx[k], kx[k]);
                    comp_add2(v[k], cv[k], kv[k]);
                }
            } else {
                float2 vs[H];
#pragma unroll
                for (int k = 0; k < H; ++k) xs[0][k] = x[k];
                accel(xs, a, true);
#pragma unroll
                for (int k = 0; k < H; ++k) {
                    kx[k] = __ffma2_rn(two, v[k], cx[k]);
                    kv[k] = a[0][k];
                    xs[0][k] = __ffma2_rn(three, v[k], x[k]);
                    vs[k] = __ffma2_rn(three, a[0][k], v[k]);
                }
                accel(xs, a, false);
#pragma unroll
                for (int k = 0; k < H; ++k) {
                    kx[k] = __ffma2_rn(two, vs[k], kx[k]);
                    kv[k] = __ffma2_rn(two, a[0][k], kv[k]);
                    xs[0][k] = __ffma2_rn(three, vs[k], x[k]);
                    vs[k] = __ffma2_rn(three, a[0][k], v[k]);
                }
                accel(xs, a, false);
#pragma unroll
                for (int k = 0; k < H; ++k) {
                    kx[k] = __ffma2_rn(two, vs[k], kx[k]);
                    kv[k] = __ffma2_rn(two, a[0][k], kv[k]);
                    xs[0][k] = __ffma2_rn(six, vs[k], x[k]);
                    kx[k] = __ffma2_rn(six, a[0][k], kx[k]);
                }
                accel(xs, a, false);
#pragma unroll
                for (int k = 0; k < H; ++k) {
                    kv[k] = __fadd2_rn(kv[k], a[0][k]);
                    comp_add2_folded(x[k], cx[k], kx[k]);
                    comp_add2(v[k], cv[k], kv[k]);
                }
            }
        });
        if (src.ckpt_every() > 0) {
#pragma unroll
            for (int k = 0; k < H; ++k) {
                if (i0 + k < s) src.checkpoint(q, ck, i0 + k, x[k].x, v[k].x, cx[k].x, cv[k].x);
                if (i0 + k + H < s) src.checkpoint(q, ck, i0 + k + H, x[k].y, v[k].y, cx[k].y, cv[k].y);
            }
            ++ck;
        }
    }
    bool bad = false;
#pragma unroll
    for (int k = 0; k < H; ++k) {
        if (i0 + k < s) {
            src.store(q, i0 + k, x[k].x, v[k].x, cx[k].x, cv[k].x);
            bad |= !(isfinite(x[k].x) && isfinite(v[k].x));
        }
        if (i0 + k + H < s) {
            src.store(q, i0 + k + H, x[k].y, v[k].y, cx[k].y, cv[k].y);
            bad |= !(isfinite(x[k].y) && isfinite(v[k].y));
        }
    }
    if (bad) any_bad = 1;
    __syncthreads();
    if (t == 0) src.finish(q, n, any_bad != 0);
}

// At most 128 registers a thread for CTAs of up to 256 threads: the paired body keeps
// four 128-thread CTAs (16 warps) on an SM without spilling.
template <int P, int MAXT, class Src>
__global__ void __launch_bounds__(MAXT, MAXT <= 256 ? 2 : 1) rk4_chain_pk_kernel(const Src src)
{
    rk4_chain_pk_body<P, (MAXT <= 256), MAXT>(src, blockIdx.x);
}

// Persistent form for the serving engine: the generation loop of persist.cuh around the
// body of rk4_chain_kernel (FP64, or FP32 at P = 1) or rk4_chain_pk_kernel (FP32, P >= 2),
// one generation item per CTA in turn.  The CTA has the thread count of the size class
// (64 threads for P = 1, 2, 4: s < 256; 256 for P = 8: s <= 2048).
template <int P, bool F64, int MAXT>
__global__ void __launch_bounds__(MAXT, (!F64 && P >= 2) ? 2 : 1) rk4_chain_persist_kernel(const PersistIO pio)
{
    persist_loop(pio, [&](int64_t n, int64_t chunk) {
        ChainSlotSrc<F64, true> src;
        src.io = SlotIO{n, pio.slot_ids, pio.slots, pio.status, chunk};
        src.pio = &pio;
        for (int64_t q = blockIdx.x; q < n; q += gridDim.x) {
            if constexpr (!F64 && P >= 2) rk4_chain_pk_body<P, true, MAXT>(src, q);
            else rk4_chain_body<P, F64, MAXT>(src, q);
        }
    });
}

// Double-FP32 (CHO_FP32X2): the FP64 form of rk4_chain_kernel, operation for
// operation, in the pair arithmetic of rk4_common.cuh (dw).  P = 4 DOFs per thread
// (a pair state takes twice the registers of FP32).  The spring extensions
// e_i = x_i - x_{i-1} start with an exact TwoSum of the high parts, so close
// neighbours keep their difference to about 2^-48 of the displacement.
template <int P>
__global__ void __launch_bounds__(256) rk4_chain_dw_kernel(const ChainBatchSrc<true> src)
{
    __shared__ float2 edge_last[2][8][32];   // last DOF of every thread (hi, lo), [buffer][warp][lane]
    __shared__ float2 edge_first[2][8][32];  // first DOF of every thread
    const int64_t q = blockIdx.x;
    const int t = threadIdx.x;
    const int lane = t & 31;
    const int warp = t >> 5;
    const int nwarp = blockDim.x >> 5;
    const int s = src.s(q);
    const int i0 = t * P;

    dw g[P], u[P];
    {
        const double* c = (const double*)src.coef(q);   // [2][s]: g, u
#pragma unroll
        for (int p = 0; p < P; ++p) {
            const int i = i0 + p;
            g[p] = dw_split(i < s ? c[i] : 0.0);
            u[p] = dw_split(i < s ? c[s + i] : 0.0);
        }
    }
    const double hd = src.h(q);
    const dw h = dw_split(hd), h2 = dw_split(0.5 * hd), h6 = dw_split(hd / 6.0);
    dw x[P], v[P];
#pragma unroll
    for (int p = 0; p < P; ++p) {
        double xd = 0.0, vd = 0.0;
        float e0, e1;
        if (i0 + p < s) src.load(q, i0 + p, xd, vd, e0, e1);
        x[p] = dw_split(xd);
        v[p] = dw_split(vd);
    }

    int buf = 0;
    const int wl = warp > 0 ? warp - 1 : 0;
    const int wr = warp + 1 < nwarp ? warp + 1 : warp;
    const bool has_left = warp > 0, has_right = warp + 1 < nwarp;
    auto shfl = [&](dw a, int d, bool up) -> dw {
        return up ? dw{__shfl_up_sync(0xffffffffu, a.hi, d), __shfl_up_sync(0xffffffffu, a.lo, d)}
                  : dw{__shfl_down_sync(0xffffffffu, a.hi, d), __shfl_down_sync(0xffffffffu, a.lo, d)};
    };
    // a_i = u_i e_{i+1} - g_i e_i, as the FP64 form's fma(u, e_{i+1}, -g e_i)
    auto accel = [&](const dw (&xs)[P], dw (&acc)[P]) {
        const dw up = shfl(xs[P - 1], 1, true);
        const dw dn = shfl(xs[0], 1, false);
        edge_last[buf][warp][lane] = make_float2(xs[P - 1].hi, xs[P - 1].lo);
        edge_first[buf][warp][lane] = make_float2(xs[0].hi, xs[0].lo);
        __syncthreads();
        const float2 el2 = edge_last[buf][wl][31], ef2 = edge_first[buf][wr][0];
        const dw el = has_left ? dw{el2.x, el2.y} : dw{0.f, 0.f};
        const dw ef = has_right ? dw{ef2.x, ef2.y} : dw{0.f, 0.f};
        const dw left = lane == 0 ? el : up;
        const dw right = lane == 31 ? ef : dn;
        buf ^= 1;
        dw e[P + 1];
        e[0] = dw_add(xs[0], dw_neg(left));
#pragma unroll
        for (int p = 1; p < P; ++p) e[p] = dw_add(xs[p], dw_neg(xs[p - 1]));
        e[P] = dw_add(right, dw_neg(xs[P - 1]));
#pragma unroll
        for (int p = 0; p < P; ++p) acc[p] = dw_fma(u[p], e[p + 1], dw_neg(dw_mul(g[p], e[p])));
    };

    const int64_t n = src.steps(q);
    const int64_t every = src.ckpt_every() > 0 ? src.ckpt_every() : (n > 0 ? n : 1);
    int64_t ck = 0;
    for (int64_t done = 0; done < n; done += every) {
        repeat_steps(every, [&]() {
            dw a[P], xs[P], kx[P], kv[P], vs[P];
            accel(x, a);
#pragma unroll
            for (int p = 0; p < P; ++p) {
                kx[p] = v[p];
                kv[p] = a[p];
                xs[p] = dw_fma(h2, v[p], x[p]);
                vs[p] = dw_fma(h2, a[p], v[p]);
            }
            accel(xs, a);
#pragma unroll
            for (int p = 0; p < P; ++p) {
                kx[p] = dw_add(dw_twice(vs[p]), kx[p]);
                kv[p] = dw_add(dw_twice(a[p]), kv[p]);
                xs[p] = dw_fma(h2, vs[p], x[p]);
                vs[p] = dw_fma(h2, a[p], v[p]);
            }
            accel(xs, a);
#pragma unroll
            for (int p = 0; p < P; ++p) {
                kx[p] = dw_add(dw_twice(vs[p]), kx[p]);
                kv[p] = dw_add(dw_twice(a[p]), kv[p]);
                xs[p] = dw_fma(h, vs[p], x[p]);
                vs[p] = dw_fma(h, a[p], v[p]);
            }
            accel(xs, a);
#pragma unroll
            for (int p = 0; p < P; ++p) {
                kx[p] = dw_add(kx[p], vs[p]);
                kv[p] = dw_add(kv[p], a[p]);
                x[p] = dw_fma(h6, kx[p], x[p]);
                v[p] = dw_fma(h6, kv[p], v[p]);
            }
        });
        if (src.ckpt_every() > 0) {
#pragma unroll
            for (int p = 0; p < P; ++p)
                if (i0 + p < s) src.checkpoint(q, ck, i0 + p, dw_value(x[p]), dw_value(v[p]), 0.f, 0.f);
            ++ck;
        }
    }
#pragma unroll
    for (int p = 0; p < P; ++p)
        if (i0 + p < s) src.store(q, i0 + p, dw_value(x[p]), dw_value(v[p]), 0.f, 0.f);
}

template <int P, bool F64, class Src>
cudaError_t launch_p(const Src& src, int64_t n_inst, int s_max, cudaStream_t st)
{
    int threads = (s_max + P - 1) / P;
    threads = ((threads + 31) / 32) * 32;
    if (threads > kChainMaxThreads) return cudaErrorInvalidValue;
    if (n_inst <= 0) return cudaSuccess;
    if (n_inst > 0x7fffffffLL) return cudaErrorInvalidValue;
    if constexpr (P == 8) {
        if (threads > 256) {   // s > 2048: wide CTAs, 64 registers per thread
            if constexpr (F64) rk4_chain_kernel<P, F64, kChainMaxThreads, Src><<<(unsigned)n_inst, threads, 0, st>>>(src);
            else rk4_chain_pk_kernel<P, kChainMaxThreads, Src><<<(unsigned)n_inst, threads, 0, st>>>(src);
            return cudaGetLastError();
        }
    }
    if constexpr (!F64 && P >= 2) rk4_chain_pk_kernel<P, 256, Src><<<(unsigned)n_inst, threads, 0, st>>>(src);
    else rk4_chain_kernel<P, F64, 256, Src><<<(unsigned)n_inst, threads, 0, st>>>(src);
    return cudaGetLastError();
}

template <bool F64, class Src>
cudaError_t launch_any(const Src& src, int64_t n_inst, int s_max, cudaStream_t st, int P = 0)
{
    if (P == 0 || !chain_dofs_valid(s_max, P)) P = chain_dofs_per_thread(s_max);
    switch (P) {
        case 1: return launch_p<1, F64>(src, n_inst, s_max, st);
        case 2: return launch_p<2, F64>(src, n_inst, s_max, st);
        case 4: return launch_p<4, F64>(src, n_inst, s_max, st);
        case 8: return launch_p<8, F64>(src, n_inst, s_max, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

// DOFs per thread: the most (up to 8) that still leaves a full warp, so that the
// per-stage exchange (two shared-memory stores and loads, one barrier)
// is shared by as many DOFs as possible.  s = 1024: 8 DOFs on 128 threads ran
// 55.2 ms against 64.4 ms with 4 on 256 (4096 chains, 1e4 steps).  Up to s =
// 2048 at most 256 threads; above, 8 DOFs per thread on up to 1024 threads.
int chain_dofs_per_thread(int s)
{
    if (s < 64) return 1;
    if (s < 128) return 2;
    if (s < 256) return 4;
    return 8;
}

bool chain_dofs_valid(int s, int P)
{
    if (P != 1 && P != 2 && P != 4 && P != 8) return false;
    const int threads = (((s + P - 1) / P + 31) / 32) * 32;
    return threads <= (P == 8 ? kChainMaxThreads : 256);
}

cudaError_t launch_rk4_chain(const ChainSys& sys, const BatchIO& io, bool fp64, cudaStream_t st)
{
    if (fp64) {
        ChainBatchSrc<true> s{sys, io};
        return launch_any<true>(s, io.n_inst, sys.s, st, sys.dofs_per_thread);
    }
    ChainBatchSrc<false> s{sys, io};
    return launch_any<false>(s, io.n_inst, sys.s, st, sys.dofs_per_thread);
}

cudaError_t launch_rk4_chain_slots(int s_max, const SlotIO& io, bool fp64, cudaStream_t st)
{
    if (fp64) {
        ChainSlotSrc<true> s{io};
        return launch_any<true>(s, io.n_inst, s_max, st);
    }
    ChainSlotSrc<false> s{io};
    return launch_any<false>(s, io.n_inst, s_max, st);
}

namespace {

template <int P, bool F64>
int chain_resident_p(int s)
{
    int threads = (s + P - 1) / P;
    threads = ((threads + 31) / 32) * 32;
    if (threads > kChainMaxThreads) return 0;
    int n = 0;
    cudaError_t e = cudaSuccess;
    using Src = ChainSlotSrc<F64>;
    bool wide = false;
    if constexpr (P == 8) {
        wide = threads > 256;                       // s > 2048: the wide CTAs of launch_p
        if (wide) {
            if constexpr (F64)
                e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, rk4_chain_kernel<P, F64, kChainMaxThreads, Src>,
                                                                  threads, 0);
            else
                e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, rk4_chain_pk_kernel<P, kChainMaxThreads, Src>,
                                                                  threads, 0);
        }
    }
    if (!wide) {
        if constexpr (F64 || P < 2)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, rk4_chain_kernel<P, F64, 256, Src>, threads, 0);
        else
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, rk4_chain_pk_kernel<P, 256, Src>, threads, 0);
    }
    int dev = 0, sms = 0;
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return 0;
    }
    return n * sms;
}

}  // namespace

// Chains of s masses the slot kernel holds resident at once on this device (one per CTA).
int chain_slot_resident(int s, bool fp64)
{
    switch (chain_dofs_per_thread(s)) {
        case 1: return fp64 ? chain_resident_p<1, true>(s) : chain_resident_p<1, false>(s);
        case 2: return fp64 ? chain_resident_p<2, true>(s) : chain_resident_p<2, false>(s);
        case 4: return fp64 ? chain_resident_p<4, true>(s) : chain_resident_p<4, false>(s);
        default: return fp64 ? chain_resident_p<8, true>(s) : chain_resident_p<8, false>(s);
    }
}

int chain_persist_threads(int P) { return P == 8 ? 256 : 64; }

cudaError_t launch_rk4_chain_persist(int P, const PersistIO& pio, bool fp64, int grid, cudaStream_t st)
{
    if (grid <= 0) return cudaErrorInvalidValue;
    const int th = chain_persist_threads(P);
    switch (P) {
        case 1:
            if (fp64) rk4_chain_persist_kernel<1, true, 64><<<grid, th, 0, st>>>(pio);
            else rk4_chain_persist_kernel<1, false, 64><<<grid, th, 0, st>>>(pio);
            break;
        case 2:
            if (fp64) rk4_chain_persist_kernel<2, true, 64><<<grid, th, 0, st>>>(pio);
            else rk4_chain_persist_kernel<2, false, 64><<<grid, th, 0, st>>>(pio);
            break;
        case 4:
            if (fp64) rk4_chain_persist_kernel<4, true, 64><<<grid, th, 0, st>>>(pio);
            else rk4_chain_persist_kernel<4, false, 64><<<grid, th, 0, st>>>(pio);
            break;
        case 8:
            if (fp64) rk4_chain_persist_kernel<8, true, 256><<<grid, th, 0, st>>>(pio);
            else rk4_chain_persist_kernel<8, false, 256><<<grid, th, 0, st>>>(pio);
            break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_rk4_chain_dw(const ChainSys& sys, const BatchIO& io, cudaStream_t st)
{
    constexpr int P = 4;
    int threads = (sys.s + P - 1) / P;
    threads = ((threads + 31) / 32) * 32;
    if (threads > 256 || !sys.C64) return cudaErrorInvalidValue;
    if (io.n_inst <= 0) return cudaSuccess;
    if (io.n_inst > 0x7fffffffLL) return cudaErrorInvalidValue;
    ChainBatchSrc<true> src{sys, io};
    rk4_chain_dw_kernel<P><<<(unsigned)io.n_inst, threads, 0, st>>>(src);
    return cudaGetLastError();
}

}  // namespace cho
