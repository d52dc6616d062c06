// ctx.h -- the library's context and system objects (internal).
#pragma once

#include "../../include/cho.h"
#include "cho_internal.h"

#include <array>
#include <cstdint>
#include <map>
#include <mutex>
#include <set>
#include <vector>

namespace cho {

// Sets the thread-local message returned by cho_last_error() and returns st.
cho_status fail(cho_status st, const char* fmt, ...);
void clear_error();

// Makes `dev` current for the scope and restores the caller's device after.
class DeviceGuard {
public:
    explicit DeviceGuard(int dev);
    ~DeviceGuard();
    bool ok() const { return ok_; }

private:
    int prev_ = -1;
    bool ok_ = false;
};

// Grow-only device buffer owned by a context.
class Workspace {
public:
    void* get(size_t bytes, cudaError_t* err);
    void release();

private:
    void* ptr_ = nullptr;
    size_t cap_ = 0;
};

struct ServeEngine;

}  // namespace cho

struct cho_system_impl {
    cho_ctx* ctx = nullptr;
    int32_t kind = 0;
    int32_t s = 0;
    int64_t n_sys = 0;
    int32_t path = 0;
    int32_t S = 0;          // rk4_small padded size
    int32_t s_pad = 0;      // rk4_dense padded size (CUDA cores)
    int32_t s_tc = 0;       // rk4_dense tensor-core layout: 64, 128 or 256 (0: none)
    double omega_max = 0.0;
    std::vector<double> omegas;
    // host copies of the description
    std::vector<double> h_masses, h_springs, h_M, h_K;
    // device data (see cho_internal.h for layouts)
    double* d_B64 = nullptr;
    float* d_B32 = nullptr;
    uint16_t* d_Bbf = nullptr;
    double* d_masses = nullptr;
    double* d_springs = nullptr;
    double* d_M = nullptr;
    double* d_K = nullptr;
    int* d_err = nullptr;               // device error word of the kernels with bounded waits
    double* d_plain = nullptr;          // FP64 plain-form coefficients: tridiagonal [3][s] or dense [s][s]
    // dense, one shared (M, K): B row-major FP64 (host) and the k-step jump blocks of the
    // polynomial form per (h, k): [3][s_pad][s_pad] transposed FP64 and [3][2][s_pad][s_pad] FP32 pairs
    std::vector<double> h_B;
    struct PolyBlocks {
        double h;
        int32_t k;
        double* d64;
        float* d32;
    };
    std::mutex poly_mu;
    std::vector<PolyBlocks> poly;
    // spring kinds: dashpots and harmonic forcing (see cho_system_set_damping/_forcing)
    std::vector<double> h_dampers, h_famp, h_fomega, h_fphase;
    double* d_ext64 = nullptr;          // ChainExtSys coefficients
    float* d_ext32 = nullptr;
    double* d_force = nullptr;          // [n_sys][2] omega, phase
    bool damped() const { return !h_dampers.empty(); }
    bool forced() const { return !h_famp.empty(); }
};

namespace cho {
// Kernel variants that give the same bits for a batch, chosen by the tuner or forced.
struct KernelChoice {
    int32_t small_variant = -1;     // SmallSys::variant
    int32_t chain_dofs = 0;         // ChainSys::dofs_per_thread
    int32_t dense_few = -1;         // DenseSys::few
};
// Tune table key: kernel family, its size (S, s or s_pad), precision, one (M, K) per
// instance, floor(log2(n_inst)).
using TuneKey = std::array<int32_t, 5>;
}  // namespace cho

struct cho_ctx {
    int device = 0;
    int sm_count = 0;
    int cc_major = 0, cc_minor = 0;
    char device_name[256] = {};
    std::mutex tune_mu;                 // guards `tune`
    std::map<cho::TuneKey, int32_t> tune;   // chosen variant per batch shape (tuner's code)
    cho_config cfg{};
    std::mutex mu;                      // guards `systems`
    std::set<cho_system_impl*> systems;
    std::mutex ws_mu;                   // guards `ws` and `err_host`
    cho::Workspace ws;                  // host-memory batch staging
    int* err_host = nullptr;            // pinned word: a system's device error word, read in stream order
    std::mutex plain_mu;
    cho::Workspace plain_ws;            // plain-form state and stage buffers
    cho::ServeEngine* serve = nullptr;
    std::mutex serve_mu;
};

namespace cho {
// Builds the dense-path device data (B in FP64, FP32 pairs and BF16 pieces).
cudaError_t build_dense_device(cho_system_impl* sys, const double* B);
// BF16 pieces of B for the tensor-core kernel (rk4_dense_tc.cu).
cudaError_t build_dense_tc_device(cho_system_impl* sys, const double* B);
// Stops the serving thread of a context, if any.
void serve_stop(cho_ctx* ctx);
// The argument checks of cho_integrate_batch.
cho_status validate_batch(const cho_batch_desc* b, const char* who, cudaStream_t st);
// One batch with device arrays (validated by the caller); `force` overrides the tune table.
cho_status run_device_batch(cho_ctx* ctx, const cho_batch_desc* b, cudaStream_t st, const KernelChoice* force);
// Tune key of a batch shape; false for shapes with a single variant.
bool tune_key(const cho_system_impl* sys, int64_t n_inst, int32_t prec, int32_t poly_jump, TuneKey* key);
}  // namespace cho
