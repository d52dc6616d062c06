// rk4_chain_ext.cu -- classical RK4 for the spring chain with a dashpot beside
// every spring and a harmonic force on every mass (beyond the paper's undamped
// eqs. 1-3):
//     m_i x_i'' = -C_i e_i + C_{i+1} e_{i+1} - c_i e_i' + c_{i+1} e_{i+1}' + F_i cos(omega t + phase),
// e_i = x_i - x_{i-1} (e_0 = x_0, the wall), e_i' = v_i - v_{i-1}, nothing to the
// right of the last mass.  The layout is rk4_chain's (one CTA per instance, P
// consecutive DOFs per thread, the neighbours' edge values through a
// double-buffered shared-memory slot array with one barrier per stage); here each
// stage also exchanges the stage velocities, and takes the force at its own time
// t, t + h/2, t + h/2, t + h.
//
// FP32: coefficients as FP32 pairs with the lo products of springs and dashpots
// formed at stage 1 and reused by stages 2-4 (as rk4_chain); the force phase in
// cycles, (omega t + phase) / 2 pi, is carried as an FP32 pair advanced by
// omega h / 2 pi each step and reduced to [0, 1), so the cosine (cospif) keeps
// its accuracy over long horizons.  FP64: the phase is omega t + phase directly.
#include "cho_internal.h"
#include "rk4_common.cuh"
#include "../../include/cho.h"

#include <cmath>

namespace cho {
namespace {

constexpr int kExtThreads = 256;

// Phase in cycles as an unevaluated FP32 pair, advanced by a pair increment.
struct Phase32 {
    float hi, lo, dhi, dlo;
    __device__ void init(double phase, double omega, double h)
    {
        const double two_pi = 6.283185307179586476925286766559;
        double c = phase / two_pi;
        c -= floor(c);
        split_ff(c, hi, lo);
        split_ff(omega * h / two_pi, dhi, dlo);
    }
    // cos(2 pi (phase + frac * step)) for frac = 0, 1/2, 1 (j = 0, 1, 2)
    __device__ __forceinline__ float cosine(int j) const
    {
        const float r0 = __fadd_rn(hi, lo);
        const float d = __fadd_rn(dhi, dlo);
        const float r = j == 0 ? r0 : (j == 1 ? __fmaf_rn(0.5f, d, r0) : __fadd_rn(r0, d));
        return cospif(2.f * r);
    }
    __device__ __forceinline__ void advance()
    {
        // two-sum of the hi parts, lo parts added into the error, renormalised
        const float s = __fadd_rn(hi, dhi);
        const float bb = __fsub_rn(s, hi);
        const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(dhi, bb));
        const float l = __fadd_rn(__fadd_rn(lo, dlo), err);
        const float h2 = __fadd_rn(s, l);
        lo = __fsub_rn(l, __fsub_rn(h2, s));
        hi = __fsub_rn(h2, rintf(h2));           // drop whole cycles (exact)
    }
};

template <int P, bool F64>
__global__ void __launch_bounds__(kExtThreads) rk4_chain_ext_kernel(const ChainExtSys sys, const BatchIO io)
{
    using Real = std::conditional_t<F64, double, float>;
    struct XV {
        Real x, v;
    };
    // stage displacement and velocity at the edges, [buffer][slot]: thread t stores its
    // last DOF's in edge_l[.][t + 1] and its first DOF's in edge_f[.][t]; edge_l[.][0]
    // (the wall) and edge_f[.][blockDim.x] (past the free end) stay zero
    __shared__ XV edge_l[2][kExtThreads + 1], edge_f[2][kExtThreads + 1];

    const int64_t q = blockIdx.x;
    const int t = threadIdx.x;
    const int lane = t & 31;
    const int s = sys.s;
    if (t == 0) {
        edge_l[0][0] = edge_l[1][0] = XV{0, 0};
        edge_f[0][blockDim.x] = edge_f[1][blockDim.x] = XV{0, 0};
    }
    const int i0 = t * P;
    const int64_t set = sys.per_inst_sys ? q : 0;

    // coefficients g, u (springs), y, w (dashpots), p (force) of DOFs i0 .. i0+P-1
    Real gh[P], uh[P], yh[P], wh[P], ph[P];
    float gl[P], ul[P], yl[P], wl[P], pl[P];
#pragma unroll
    for (int p = 0; p < P; ++p) {
        const int i = i0 + p;
        const bool in = i < s;
        if constexpr (F64) {
            const double* c = sys.E64 + set * 5 * (int64_t)s;
            gh[p] = in ? c[i] : 0.0;
            uh[p] = in ? c[s + i] : 0.0;
            yh[p] = in ? c[2 * s + i] : 0.0;
            wh[p] = in ? c[3 * s + i] : 0.0;
            ph[p] = in ? c[4 * s + i] : 0.0;
            gl[p] = ul[p] = yl[p] = wl[p] = pl[p] = 0.f;
        } else {
            const float* c = sys.E32 + set * 10 * (int64_t)s;
            gh[p] = in ? c[i] : 0.f;
            uh[p] = in ? c[s + i] : 0.f;
            yh[p] = in ? c[2 * s + i] : 0.f;
            wh[p] = in ? c[3 * s + i] : 0.f;
            ph[p] = in ? c[4 * s + i] : 0.f;
            gl[p] = in ? c[5 * s + i] : 0.f;
            ul[p] = in ? c[6 * s + i] : 0.f;
            yl[p] = in ? c[7 * s + i] : 0.f;
            wl[p] = in ? c[8 * s + i] : 0.f;
            pl[p] = in ? c[9 * s + i] : 0.f;
        }
    }
    const double hd = io.h[io.h_per_inst ? q : 0];
    const StepSize<F64> hs(hd);
    const bool forced = sys.force != nullptr;
    const double omega = forced ? sys.force[set * 2] : 0.0;
    const double phase0 = forced ? sys.force[set * 2 + 1] : 0.0;
    Phase32 ph32;
    if constexpr (!F64) ph32.init(phase0, omega, hd);

    Real x[P], v[P];
    float cx[P], cv[P];
#pragma unroll
    for (int p = 0; p < P; ++p) {
        const int i = i0 + p;
        x[p] = v[p] = 0;
        cx[p] = cv[p] = 0.f;
        if (i < s) {
            const double xd = io.x0[q * s + i], vd = io.v0[q * s + i];
            x[p] = (Real)xd;
            v[p] = (Real)vd;
            if constexpr (!F64) {
                cx[p] = (float)(xd - (double)x[p]);
                cv[p] = (float)(vd - (double)v[p]);
            }
        }
    }

    int buf = 0;
    float lo1[P];
    // the neighbours' edge values come through shared memory: one store and one load per
    // side and stage, the zero slots standing in for the wall and the free end
    auto accel = [&](const Real (&xs)[P], const Real (&vs)[P], Real fst, Real (&acc)[P], bool first) {
        edge_l[buf][t + 1] = XV{xs[P - 1], vs[P - 1]};
        edge_f[buf][t] = XV{xs[0], vs[0]};
        __syncthreads();
        const XV l = edge_l[buf][t];
        const XV r_ = edge_f[buf][t + 1];
        const Real xleft = l.x, vleft = l.v, xright = r_.x, vright = r_.v;
        buf ^= 1;
        Real e[P + 1], r[P + 1];                 // extensions and their rates
        e[0] = xs[0] - xleft;
        r[0] = vs[0] - vleft;
#pragma unroll
        for (int p = 1; p < P; ++p) {
            e[p] = xs[p] - xs[p - 1];
            r[p] = vs[p] - vs[p - 1];
        }
        e[P] = xright - xs[P - 1];
        r[P] = vright - vs[P - 1];
#pragma unroll
        for (int p = 0; p < P; ++p) {
            Real a;
            if constexpr (F64) {
                a = fmar(uh[p], e[p + 1], -gh[p] * e[p]);
                a = fmar(wh[p], r[p + 1], a);
                a = fmar(-yh[p], r[p], a);
                a = fmar(ph[p], fst, a);
            } else {
                if (first) {
                    float lo = fmaf(ul[p], e[p + 1], -gl[p] * e[p]);
                    lo = fmaf(wl[p], r[p + 1], lo);
                    lo1[p] = fmaf(-yl[p], r[p], lo);
                }
                a = fmaf(uh[p], e[p + 1], fmaf(-gh[p], e[p], lo1[p]));
                a = fmaf(wh[p], r[p + 1], a);
                a = fmaf(-yh[p], r[p], a);
                a = fmaf(ph[p], fst, fmaf(pl[p], fst, a));
            }
            acc[p] = a;
        }
    };

    const int64_t n = io.n_steps;
    const int64_t every = io.ckpt_every > 0 ? io.ckpt_every : (n > 0 ? n : 1);
    int64_t ck = 0;
    int64_t step = 0;
    // the step's three force cosines: lane j of every warp evaluates cosine j, then all
    // lanes take the three by shuffle (the same values as three evaluations per thread)
    const int jc = lane < 3 ? lane : 0;
    for (int64_t done = 0; done < n; done += every) {
#pragma unroll 2
        for (int64_t it = 0; it < every; ++it, ++step) {
            Real f0 = 0, f1 = 0, f2 = 0;
            if (forced) {
                Real c;
                if constexpr (F64) {
                    const double tn = (double)step * hd;
                    const double tj = jc == 0 ? tn : (jc == 1 ? tn + hd / 2.0 : tn + hd);
                    c = cos(omega * tj + phase0);
                } else {
                    c = ph32.cosine(jc);
                    ph32.advance();
                }
                f0 = __shfl_sync(0xffffffffu, c, 0);
                f1 = __shfl_sync(0xffffffffu, c, 1);
                f2 = __shfl_sync(0xffffffffu, c, 2);
            }
            Real a[P], xs[P], kx[P], kv[P], vs[P];
            accel(x, v, f0, a, true);
#pragma unroll
            for (int p = 0; p < P; ++p) {
                kx[p] = v[p];
                kv[p] = a[p];
                xs[p] = fmar(hs.h2, v[p], x[p]);
                vs[p] = fmar(hs.h2, a[p], v[p]);
            }
            accel(xs, vs, f1, a, false);
#pragma unroll
            for (int p = 0; p < P; ++p) {
                kx[p] = fmar((Real)2, vs[p], kx[p]);
                kv[p] = fmar((Real)2, a[p], kv[p]);
                xs[p] = fmar(hs.h2, vs[p], x[p]);
                vs[p] = fmar(hs.h2, a[p], v[p]);
            }
            accel(xs, vs, f1, a, false);
#pragma unroll
            for (int p = 0; p < P; ++p) {
                kx[p] = fmar((Real)2, vs[p], kx[p]);
                kv[p] = fmar((Real)2, a[p], kv[p]);
                xs[p] = fmar(hs.h, vs[p], x[p]);
                vs[p] = fmar(hs.h, a[p], v[p]);
            }
            accel(xs, vs, f2, a, false);
#pragma unroll
            for (int p = 0; p < P; ++p) {
                kx[p] = addr(kx[p], vs[p]);
                kv[p] = addr(kv[p], a[p]);
                state_update<F64>(x[p], cx[p], kx[p], hs);
                state_update<F64>(v[p], cv[p], kv[p], hs);
            }
        }
        if (io.ckpt_every > 0 && io.x_traj) {
#pragma unroll
            for (int p = 0; p < P; ++p) {
                const int i = i0 + p;
                if (i >= s) continue;
                const int64_t o = (q * io.n_ck + ck) * s + i;
                io.x_traj[o] = (double)x[p] + (double)cx[p];
                if (io.v_traj) io.v_traj[o] = (double)v[p] + (double)cv[p];
            }
        }
        ++ck;
    }
#pragma unroll
    for (int p = 0; p < P; ++p) {
        const int i = i0 + p;
        if (i >= s) continue;
        io.x_out[q * s + i] = (double)x[p] + (double)cx[p];
        io.v_out[q * s + i] = (double)v[p] + (double)cv[p];
    }
}

template <int P, bool F64>
cudaError_t launch_ext(const ChainExtSys& sys, const BatchIO& io, cudaStream_t st)
{
    int threads = (sys.s + P - 1) / P;
    threads = ((threads + 31) / 32) * 32;
    if (threads > kExtThreads) return cudaErrorInvalidValue;
    if (io.n_inst <= 0) return cudaSuccess;
    if (io.n_inst > 0x7fffffffLL) return cudaErrorInvalidValue;
    rk4_chain_ext_kernel<P, F64><<<(unsigned)io.n_inst, threads, 0, st>>>(sys, io);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_rk4_chain_ext(const ChainExtSys& sys, const BatchIO& io, bool fp64, cudaStream_t st)
{
    if (sys.s < 1 || sys.s > kChainExtMaxS) return cudaErrorInvalidValue;
    if (sys.s <= 256) return fp64 ? launch_ext<1, true>(sys, io, st) : launch_ext<1, false>(sys, io, st);
    if (sys.s <= 512) return fp64 ? launch_ext<2, true>(sys, io, st) : launch_ext<2, false>(sys, io, st);
    return fp64 ? launch_ext<4, true>(sys, io, st) : launch_ext<4, false>(sys, io, st);
}

}  // namespace cho
