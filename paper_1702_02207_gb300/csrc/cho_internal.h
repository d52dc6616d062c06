// cho_internal.h -- declarations shared by the library's translation units.
// Not part of the public ABI (include/cho.h is).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace cho {

// Kernel family chosen for a (kind, s, n_sys) system.
enum Path : int32_t {
    PATH_SMALL = 0,   // s <= 32, any kind, any number of parameter sets
    PATH_CHAIN = 1,   // CHAIN / TWO_DOF with s > 32
    PATH_DENSE = 2,   // DENSE with s > 32 and one shared parameter set
};

constexpr int kSmallThreads = 64;    // threads per CTA of rk4_small (small CTAs balance the SMs)
constexpr int kChainMaxThreads = 1024;

#ifdef __CUDACC__
#define CHO_HD __host__ __device__
#else
#define CHO_HD
#endif

// The FP32 small-system kernels carry the scaled velocity u = (h/6) v (exact step
// constants 3 and 6 replace h/2 and h, and no h/6 multiply in the state update);
// the batch kernels and the serving engine convert with these, identically.
CHO_HD inline double scaled_velocity(double v, double h) { return v * (h / 6.0); }
CHO_HD inline double unscaled_velocity(double u, double h) { return u * (6.0 / h); }

// Host-side split of an FP64 value into an unevaluated FP32 pair hi + lo.
inline void split_pair(double d, float& hi, float& lo)
{
    hi = (float)d;
    lo = (float)(d - (double)hi);
}

// Padded size of the rk4_small family for s <= 32.
inline int small_S(int s) { return s <= 2 ? 2 : s <= 4 ? 4 : s <= 8 ? 8 : s <= 16 ? 16 : 32; }

// ----------------------------------------------------------------------------
// Where a kernel's instances get their state, step size and step count.
//
// Batch form: x0/v0 (n_inst, s) FP64 in, x_out/v_out FP64 out, optional
// checkpoint trajectories.  Slot form (serving): instance q is slot
// slot_ids[q]; its resident state block and step count come from the slot
// table, and the block is read and written back in the kernel's own precision
// so that a run split into chunks is bitwise equal to an unsplit run.
// ----------------------------------------------------------------------------
struct BatchIO {
    int64_t n_inst;
    const double* x0;
    const double* v0;
    const double* h;
    int32_t h_per_inst;
    int64_t n_steps;
    int64_t ckpt_every;     // 0: no checkpoints
    int64_t n_ck;
    int32_t poly_jump;      // 0: RK4 stages; k >= 1: polynomial form, k steps per update (s = 2)
    const double* poly_E;   // polynomial form: E = P(hA)^k - I per instance, [n_inst][4][4] (set by the launcher)
    double* x_out;
    double* v_out;
    double* x_traj;
    double* v_traj;
};

// One resident request in the serving slot table (device memory).  Written by
// the host when the request is admitted; `remaining` is decremented by the
// kernel that advances the slot.
struct SlotDesc {
    const void* coef;       // coefficient block of its parameter set (kernel-family layout)
    void* state;            // resident state block (kernel-family layout, kernel precision)
    double h;
    int64_t remaining;      // RK4 steps still to run
    int32_t s;
    int32_t pad;
};

struct SlotIO {
    int64_t n_inst;         // slots advanced by this launch
    const int32_t* slot_ids;
    SlotDesc* slots;
    int32_t* status;        // per slot: set to CHO_ENONFINITE on a non-finite state
    int64_t chunk;          // each slot runs min(chunk, remaining) steps
};

// Stream-ordered per-call device scratch from the library's own memory pool (rk4_small.cu);
// release it with cudaFreeAsync on the same stream.
cudaError_t scratch_alloc(void** p, size_t bytes, cudaStream_t st);

cudaError_t launch_gather_status(const int32_t* ids, const int32_t* status, int32_t* out, int64_t n,
                                 cudaStream_t st);

// ---- rk4_small ----------------------------------------------------------------
// Coefficients per parameter set: FP64 B (S*S), or FP32 hi (S*S) followed by lo (S*S).
struct SmallSys {
    int32_t s;
    int32_t S;
    int32_t per_inst_sys;   // 1: set = instance index, 0: set 0
    const double* B64;      // [n_sys][S][S]
    const float* B32;       // [n_sys][2][S][S] (hi then lo)
    int* err;               // device error word: set when a bounded wait gives up (may be null)
    int32_t variant = -1;   // FP32 s = 2 kernel: -1 default, 0 balanced, 2 lane-group form, 3 pair form
};

cudaError_t launch_rk4_small(const SmallSys& sys, const BatchIO& io, bool fp64, cudaStream_t st);
// Double-FP32 (CHO_FP32X2) for s <= 32 systems (padded S = 2 .. 32), the lanes of rk4_small.
cudaError_t launch_rk4_small_dw(const SmallSys& sys, const BatchIO& io, cudaStream_t st);
cudaError_t launch_rk4_small_slots(int S, const SlotIO& io, bool fp64, cudaStream_t st);
// Instances the slot kernel holds resident at once on this device (0: none fits).
int small_slot_resident(int S, bool fp64);

// ---- rk4_chain ----------------------------------------------------------------
// Coefficients per parameter set, spring form of eq. 2: g_i = C_i/m_i and
// u_i = C_{i+1}/m_i (u_{s-1} = 0): FP64 [2][s] (g, u) or FP32 [4][s] (g, u hi; then lo).
struct ChainSys {
    int32_t s;
    int32_t per_inst_sys;
    const double* C64;      // [n_sys][2][s]
    const float* C32;       // [n_sys][4][s]
    int32_t dofs_per_thread = 0;   // 1, 2, 4 or 8 (chain_dofs_valid); 0: chain_dofs_per_thread(s)
};

int chain_dofs_per_thread(int s);
// Whether P DOFs per thread fit the chain kernel for s DOFs (P < 8: at most 256
// threads; P = 8: at most 1024).
bool chain_dofs_valid(int s, int P);
cudaError_t launch_rk4_chain(const ChainSys& sys, const BatchIO& io, bool fp64, cudaStream_t st);
// Double-FP32 (CHO_FP32X2) for chains of s <= 1024, 4 DOFs per thread, batch form.
cudaError_t launch_rk4_chain_dw(const ChainSys& sys, const BatchIO& io, cudaStream_t st);

// ---- rk4_chain_ext: the chain with dashpots and harmonic forcing -------------------
// Per parameter set and DOF i (FP64 [n_sys][5][s], FP32 [n_sys][10][s]: the five hi
// rows, then the five lo rows): g_i = C_i/m_i, u_i = C_{i+1}/m_i, y_i = c_i/m_i,
// w_i = c_{i+1}/m_i, p_i = F_i/m_i (u, w = 0 at the free end).  Per set: omega, phase
// (FP64 [n_sys][2]).
struct ChainExtSys {
    int32_t s;
    int32_t per_inst_sys;
    const double* E64;
    const float* E32;
    const double* force;    // [n_sys][2]: omega, phase (null: no forcing)
};
constexpr int kChainExtMaxS = 1024;
cudaError_t launch_rk4_chain_ext(const ChainExtSys& sys, const BatchIO& io, bool fp64, cudaStream_t st);
cudaError_t launch_rk4_chain_slots(int s_max, const SlotIO& io, bool fp64, cudaStream_t st);
int chain_slot_resident(int s, bool fp64);

// ---- rk4_dense (shared B, s > 32) ------------------------------------------------
struct DenseSys {
    int32_t s;
    int32_t s_pad;          // SIMT kernels: next power of two >= max(s, 64), <= 512
    const double* B64;      // [s_pad][s_pad] = B^T, zero padded
    const float* B32;       // [2][s_pad][s_pad] (hi, lo) of B^T, zero padded
    const uint16_t* Bbf;    // tensor-core kernel: shared-memory images of the BF16 pieces of B
    int32_t s_tc;           // tensor-core layout: 64 (two tiles on a block diagonal), 128 or 256 (0: none)
    int* err;               // device error word of the tensor-core kernel (bounded waits)
    int32_t stall_mma;      // test hook: issue no MMA, so the bounded wait on it runs out
    int32_t per_inst;       // 1: one (M, K) per instance, B64/B32 hold n_sys matrices back to back
    int32_t few = -1;       // FP32: 1 one instance per CTA or cluster, 0 the streaming kernel, -1 by count
};

// Whether the FP32 one-instance-per-CTA-or-cluster kernels can run this system here,
// and whether the default rule picks them for n_inst instances.
bool dense_few_capable(const DenseSys& sys);
bool dense_few_default(const DenseSys& sys, int64_t n_inst);

// Test hook for the bounded device waits: CHO_TEST_STALL_MMA=1 in the environment makes
// the tensor-core kernel skip its MMAs, so its wait on their completion gives up after
// about a second and the run reports CHO_ETIMEOUT.  Read at every launch.
int test_stall_mma();
int dense_pad(int s);
cudaError_t launch_rk4_dense(const DenseSys& sys, const BatchIO& io, int prec, cudaStream_t st);
// Polynomial form with k-step jumps (io.poly_jump = k) of a shared dense system: E holds
// the transposed jump blocks [3][s_pad][s_pad] (FP64) or [3][2][s_pad][s_pad] (FP32 pairs).
cudaError_t launch_rk4_dense_poly(const DenseSys& sys, const void* E, const BatchIO& io, bool fp64, cudaStream_t st);
cudaError_t launch_rk4_dense_slots(const DenseSys& sys, const SlotIO& io, bool fp64, cudaStream_t st);
int dense_slot_resident(const DenseSys& sys, bool fp64);
// tensor-core split-BF16 variant (rk4_dense_tc.cu)
cudaError_t launch_rk4_dense_tc(const DenseSys& sys, const BatchIO& io, int prec, cudaStream_t st);
cudaError_t launch_rk4_dense_tc_slots(const DenseSys& sys, const SlotIO& io, int prec, cudaStream_t st);
int dense_tc_slot_resident(const DenseSys& sys, int prec);

// ---- energy -------------------------------------------------------------------
struct EnergySys {
    int32_t kind;           // cho_kind
    int32_t s;
    int32_t per_inst_sys;
    const double* masses;   // [n_sys][s]  (TWO_DOF / CHAIN)
    const double* springs;  // [n_sys][s]
    const double* M;        // [n_sys][s][s] (DENSE)
    const double* K;
};
cudaError_t launch_energy(const EnergySys& sys, const double* x, const double* v, int64_t n_inst,
                          int64_t n_per, double* E, cudaStream_t st);

// ---- plain form (baseline) -----------------------------------------------------
// One system at a time; y = (x, v) in device memory; k buffers in `work` (8 s doubles).
struct PlainSys {
    int32_t s;
    int32_t dense;          // 0: tridiagonal coefficients, 1: dense B
    const double* coef;     // tridiagonal [3][s] or dense [s][s] of this parameter set
};
cudaError_t launch_plain_step(const PlainSys& sys, double* y, double* work, double h, cudaStream_t st);

}  // namespace cho
