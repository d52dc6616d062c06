// packed.cu -- several batches of uneven sizes in as few kernel launches as possible.
//
// cho_integrate_packed takes a list of batches (any systems, sizes and step counts)
// and runs every set of batches that share a kernel family and size class in ONE
// launch: rk4_small by padded size S (chains, 2-DOF and dense systems of s <= 32 alike),
// rk4_chain by DOFs per thread (the CTA is sized for the group's largest chain), and
// rk4_dense by system.  The launch goes over a work table with one entry per instance
// -- its coefficients (its parameter set), its state block, h, its step count and its
// own s -- the table the serving engine's slot-form kernels read.  On the device, in
// stream order and without a host synchronisation:
//   1. packed_in_kernel writes each batch's table entries and converts its FP64
//      x0, v0 into state blocks in the kernel's precision (the same FP64 expressions as
//      the batch kernels' loads, so the bits are those of separate calls);
//   2. one slot-form launch per group advances every instance its own step count;
//   3. packed_out_kernel converts the blocks back into each batch's x_out, v_out.
// Every family's slot form computes each instance with the operations of its batch
// form, so each batch's result is bitwise equal to a separate cho_integrate_batch.
#include "../../include/cho.h"
#include "cho_internal.h"
#include "ctx.h"

#include <algorithm>
#include <map>
#include <tuple>
#include <vector>

namespace cho {
namespace {

constexpr int kPackThreads = 256;

// One batch of a group, as the conversion kernels see it.
struct PackBatch {
    const double* x0;
    const double* v0;
    const double* h;
    int32_t h_per_inst;
    double* x_out;
    double* v_out;
    int64_t n_inst;
    int64_t first;          // its first entry in the group's work table
    int64_t n_steps;
    int32_t s;              // DOFs per instance
    int32_t n;              // state rows per instance (S for rk4_small, else s)
    int32_t scaled;         // FP32 rk4_small / rk4_chain: the state holds u = (h/6) v
    const char* coef;       // coefficients of parameter set 0 (null: the kernel reads the system's)
    int64_t coef_stride;    // bytes between parameter sets (0: one set for every instance)
    char* state;            // state block of entry `first`
    int64_t block_bytes;    // bytes per state block
};

template <bool F64>
__global__ void __launch_bounds__(kPackThreads) packed_in_kernel(const PackBatch b, SlotDesc* slots, int32_t* ids,
                                                                 int32_t* status)
{
    const int64_t t = (int64_t)blockIdx.x * kPackThreads + threadIdx.x;
    if (t >= b.n_inst * b.n) return;
    const int64_t q = t / b.n;
    const int i = (int)(t % b.n);
    const double h = b.h[b.h_per_inst ? q : 0];
    char* blk = b.state + q * b.block_bytes;
    if (i == 0) {
        SlotDesc d;
        d.coef = b.coef ? (const void*)(b.coef + q * b.coef_stride) : nullptr;
        d.state = blk;
        d.h = h;
        d.remaining = b.n_steps;
        d.s = b.s;
        d.pad = 0;
        slots[b.first + q] = d;
        ids[b.first + q] = (int32_t)(b.first + q);
        status[b.first + q] = 0;
    }
    const double xd = i < b.s ? b.x0[q * b.s + i] : 0.0;
    const double v0 = i < b.s ? b.v0[q * b.s + i] : 0.0;
    if constexpr (F64) {
        double* st = (double*)blk;
        st[i] = xd;
        st[b.n + i] = v0;
    } else {
        const double vd = b.scaled ? scaled_velocity(v0, h) : v0;
        float* st = (float*)blk;
        const float x = (float)xd, v = (float)vd;
        st[i] = x;
        st[b.n + i] = v;
        st[2 * b.n + i] = (float)(xd - (double)x);      // the state is the unevaluated sum x + c
        st[3 * b.n + i] = (float)(vd - (double)v);
    }
}

template <bool F64>
__global__ void __launch_bounds__(kPackThreads) packed_out_kernel(const PackBatch b)
{
    const int64_t t = (int64_t)blockIdx.x * kPackThreads + threadIdx.x;
    if (t >= b.n_inst * b.s) return;
    const int64_t q = t / b.s;
    const int i = (int)(t % b.s);
    const char* blk = b.state + q * b.block_bytes;
    if constexpr (F64) {
        const double* st = (const double*)blk;
        b.x_out[q * b.s + i] = st[i];
        b.v_out[q * b.s + i] = st[b.n + i];
    } else {
        const float* st = (const float*)blk;
        const double u = (double)st[b.n + i] + (double)st[3 * b.n + i];
        b.x_out[q * b.s + i] = (double)st[i] + (double)st[2 * b.n + i];
        b.v_out[q * b.s + i] = b.scaled ? unscaled_velocity(u, b.h[b.h_per_inst ? q : 0]) : u;
    }
}

bool bf16_prec(int32_t p) { return p == CHO_DENSE_BF16X3 || p == CHO_DENSE_BF16X5 || p == CHO_DENSE_BF16X6; }

// Batches that share one launch: kernel family, size class, arithmetic, and (dense) the system.
using PackKey = std::tuple<int, int, int, const cho_system_impl*>;

}  // namespace
}  // namespace cho

using namespace cho;

extern "C" cho_status cho_integrate_packed(cho_ctx* ctx, const cho_batch_desc* batches, int32_t n_batches,
                                           void* stream)
{
    clear_error();
    const char* who = "cho_integrate_packed";
    if (!ctx) return fail(CHO_EINVAL, "%s: NULL ctx", who);
    if (n_batches < 0 || (n_batches > 0 && !batches)) return fail(CHO_EINVAL, "%s: bad batch list", who);
    DeviceGuard g(ctx->device);
    if (!g.ok()) return fail(CHO_ECUDA, "%s: cudaSetDevice failed", who);
    cudaStream_t st = (cudaStream_t)stream;
    std::map<PackKey, std::vector<int>> groups;
    for (int k = 0; k < n_batches; ++k) {
        const cho_batch_desc* b = &batches[k];
        cho_status rc = validate_batch(b, who, st);
        if (rc != CHO_OK) return rc;
        const cho_system_impl* sys = b->system;
        if (sys->ctx != ctx) return fail(CHO_EINVAL, "%s: batch %d: system belongs to another context", who, k);
        if (b->mem != CHO_MEM_DEVICE) return fail(CHO_EINVAL, "%s: batch %d: device arrays only", who, k);
        if (b->poly_jump != 0) return fail(CHO_EINVAL, "%s: batch %d: RK4 stage by stage only", who, k);
        if (b->ckpt_every != 0 || b->x_traj || b->v_traj || b->energy)
            return fail(CHO_EINVAL, "%s: batch %d: final states only (no checkpoints or energy)", who, k);
        if (sys->damped() || sys->forced())
            return fail(CHO_EINVAL, "%s: batch %d: damped or forced systems run in cho_integrate_batch", who, k);
        const int32_t p = b->prec;
        if (p == CHO_FP32X2) return fail(CHO_EINVAL, "%s: batch %d: CHO_FP32X2 runs in cho_integrate_batch", who, k);
        if (b->n_inst == 0) continue;
        const int64_t rows = sys->path == PATH_SMALL ? sys->S : sys->s;   // conversion threads per instance
        if (b->n_inst > 0x7fffffffLL || b->n_inst * rows > ((int64_t)0x7fffffff) * kPackThreads)
            return fail(CHO_EINVAL, "%s: batch %d: too many instances", who, k);
        const int size = sys->path == PATH_SMALL ? sys->S
                                                 : (sys->path == PATH_CHAIN ? chain_dofs_per_thread(sys->s) : sys->s);
        const int arith = p == CHO_FP64 ? 0 : (bf16_prec(p) ? p : 1);   // FP32 dense: one family for both names
        groups[PackKey(sys->path, size, arith, sys->path == PATH_DENSE ? sys : nullptr)].push_back(k);
    }
    if (groups.empty()) return CHO_OK;

    // layout of the scratch: per group its table, ids, status words and state blocks
    struct Plan {
        PackKey key;
        std::vector<PackBatch> pb;
        int64_t n = 0;
        size_t off_slots = 0, off_ids = 0, off_status = 0, off_state = 0, state_bytes = 0;
    };
    std::vector<Plan> plans;
    size_t total = 0;
    auto take = [&](size_t bytes) {
        const size_t o = total;
        total += (bytes + 255) / 256 * 256;
        return o;
    };
    for (auto& kv : groups) {
        Plan pl;
        pl.key = kv.first;
        const bool f64 = std::get<2>(kv.first) == 0;
        for (int k : kv.second) {
            const cho_batch_desc* b = &batches[k];
            const cho_system_impl* sys = b->system;
            PackBatch x{};
            x.x0 = b->x0;
            x.v0 = b->v0;
            x.h = b->h;
            x.h_per_inst = b->h_per_inst;
            x.x_out = b->x_out;
            x.v_out = b->v_out;
            x.n_inst = b->n_inst;
            x.first = pl.n;
            x.n_steps = b->n_steps;
            x.s = sys->s;
            x.n = sys->path == PATH_SMALL ? sys->S : sys->s;
            x.scaled = !f64 && sys->path != PATH_DENSE;
            x.block_bytes = f64 ? 2 * (int64_t)x.n * 8 : 4 * (int64_t)x.n * 4;
            const bool per_set = sys->n_sys != 1;
            if (sys->path == PATH_SMALL) {
                const int64_t SS = (int64_t)sys->S * sys->S;
                x.coef = f64 ? (const char*)sys->d_B64 : (const char*)sys->d_B32;
                x.coef_stride = per_set ? (f64 ? SS * 8 : 2 * SS * 4) : 0;
            } else if (sys->path == PATH_CHAIN) {
                x.coef = f64 ? (const char*)sys->d_B64 : (const char*)sys->d_B32;
                x.coef_stride = per_set ? (f64 ? 2 * (int64_t)sys->s * 8 : 4 * (int64_t)sys->s * 4) : 0;
            } else if (per_set && !bf16_prec(b->prec)) {                 // dense, one (M, K) per instance
                const int64_t n2 = (int64_t)sys->s_pad * sys->s_pad;
                x.coef = f64 ? (const char*)sys->d_B64 : (const char*)sys->d_B32;
                x.coef_stride = f64 ? n2 * 8 : 2 * n2 * 4;
            } else {
                x.coef = nullptr;                                          // shared dense: the system's B
                x.coef_stride = 0;
            }
            pl.n += b->n_inst;
            pl.state_bytes += (size_t)b->n_inst * (size_t)x.block_bytes;
            pl.pb.push_back(x);
        }
        if (pl.n > 0x7fffffffLL) return fail(CHO_EINVAL, "%s: more than 2^31 - 1 instances in one group", who);
        pl.off_slots = take((size_t)pl.n * sizeof(SlotDesc));
        pl.off_ids = take((size_t)pl.n * sizeof(int32_t));
        pl.off_status = take((size_t)pl.n * sizeof(int32_t));
        pl.off_state = take(pl.state_bytes);
        plans.push_back(std::move(pl));
    }
    char* base = nullptr;
    cudaError_t e = scratch_alloc((void**)&base, total, st);
    if (e != cudaSuccess) return fail(CHO_ENOMEM, "%s: %zu bytes of scratch: %s", who, total, cudaGetErrorString(e));
    for (Plan& pl : plans) {
        if (e != cudaSuccess) break;
        const int path = std::get<0>(pl.key), size = std::get<1>(pl.key), arith = std::get<2>(pl.key);
        const bool f64 = arith == 0;
        SlotDesc* slots = (SlotDesc*)(base + pl.off_slots);
        int32_t* ids = (int32_t*)(base + pl.off_ids);
        int32_t* status = (int32_t*)(base + pl.off_status);
        char* state = base + pl.off_state;
        int64_t chunk = 0;
        int s_max = 0;
        for (PackBatch& x : pl.pb) {
            x.state = state;
            state += x.n_inst * x.block_bytes;
            chunk = std::max(chunk, x.n_steps);
            s_max = std::max(s_max, x.s);
            const int64_t threads = x.n_inst * x.n;
            const unsigned blocks = (unsigned)((threads + kPackThreads - 1) / kPackThreads);
            if (f64) packed_in_kernel<true><<<blocks, kPackThreads, 0, st>>>(x, slots, ids, status);
            else packed_in_kernel<false><<<blocks, kPackThreads, 0, st>>>(x, slots, ids, status);
            e = cudaGetLastError();
            if (e != cudaSuccess) break;
        }
        if (e != cudaSuccess) break;
        SlotIO io{pl.n, ids, slots, status, chunk};
        if (chunk > 0) {
            if (path == PATH_SMALL) {
                e = launch_rk4_small_slots(size, io, f64, st);
            } else if (path == PATH_CHAIN) {
                e = launch_rk4_chain_slots(s_max, io, f64, st);
            } else {
                cho_system_impl* sys = const_cast<cho_system_impl*>(std::get<3>(pl.key));
                DenseSys ds{sys->s, sys->s_pad, sys->d_B64, sys->d_B32, sys->d_Bbf, sys->s_tc, sys->d_err, 0,
                            sys->n_sys != 1 ? 1 : 0};
                if (bf16_prec(arith)) {
                    ds.stall_mma = test_stall_mma();
                    e = launch_rk4_dense_tc_slots(ds, io, arith, st);
                } else {
                    e = launch_rk4_dense_slots(ds, io, f64, st);
                }
            }
        }
        for (const PackBatch& x : pl.pb) {
            if (e != cudaSuccess) break;
            const int64_t threads = x.n_inst * x.s;
            const unsigned blocks = (unsigned)((threads + kPackThreads - 1) / kPackThreads);
            if (f64) packed_out_kernel<true><<<blocks, kPackThreads, 0, st>>>(x);
            else packed_out_kernel<false><<<blocks, kPackThreads, 0, st>>>(x);
            e = cudaGetLastError();
        }
    }
    const cudaError_t ef = cudaFreeAsync(base, st);
    if (e != cudaSuccess) return fail(CHO_ECUDA, "%s: %s", who, cudaGetErrorString(e));
    if (ef != cudaSuccess) return fail(CHO_ECUDA, "%s: %s", who, cudaGetErrorString(ef));
    return CHO_OK;
}
