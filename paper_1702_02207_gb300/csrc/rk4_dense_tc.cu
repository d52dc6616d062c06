// rk4_dense_tc.cu -- rk4_dense on the tensor cores: each RK4 stage's B Xs
// (B = M^{-1}K shared by all instances, Xs the stage displacements of a tile of
// 32 instances) is a tcgen05.mma contraction with split-BF16 operands and FP32
// accumulation in tensor memory; the stage combinations and the Kahan-
// compensated FP32 state update run on the CUDA cores.
//
// Split-BF16.  B = b0 + b1 + b2 and Xs = p0 + p1 + p2 with each piece the BF16
// rounding of what the previous pieces leave (8 significant bits each).  The
// product keeps the partial products down to a chosen order:
//   bf16x3: b0 p0 + b0 p1 + b1 p0                 (operands to 16 bits)
//   bf16x5: bf16x3 + b1 p1 + b2 p0                (B to 24 bits, Xs to 16)
//   bf16x6: bf16x5 + b0 p2                        (both to 24 bits; s <= 128)
// Grouped issue (grp_a below): one MMA per piece of B covers every piece of Xs that
// piece pairs with, the Xs pieces laid side by side along N, so bf16x5 issues 3 MMAs
// per K chunk instead of 5 at the same ~45-cycle cost each, and every accumulator holds
// the products of each order in its own group of 32 columns.
//
// Accumulation.  Summing all K/16 chunk products of a stage into one TMEM
// accumulator lets the tensor core's accumulation rounding build up a bias that
// acts like a frequency shift, so the error grew with the horizon (bf16x5 at
// s = 256: 2.4e-5 after 5e3 steps).  bf16x5 and bf16x6 therefore spread the K chunks
// over several accumulators, and the column groups keep the large order-0 products
// apart from the small ones: each order is summed over the accumulators and the
// orders added smallest first, on the CUDA cores in FP32 round-to-nearest.  One CTA
// (two accumulator sets): two accumulators of 96 columns per set, four K chunks each
// (s = 128, 5e3 steps: 8.0e-6; one accumulator per set was 7 % faster and reached
// 1.5e-5 in v); 2-CTA clusters: five accumulators (s = 256, 5e3 steps: 1.0e-5 with four,
// 9.96e-6 with five over 30 sampled instances); bf16x3, whose truncation error
// dominates, keeps one.

// Work split.  s <= 64: one CTA per 64 instances, two tiles of 32 stacked along
// the 128 rows against the block-diagonal [B 0; 0 B] (the MMA shape is fixed at
// 128 rows; a padded 64 x 64 B would leave half of every MMA idle).  64 < s <=
// 128: one CTA per tile of 32 instances.  Both pair the stages (the products of
// stages 1 and 2 go to the tensor cores together, then those of 3 and 4; see
// rk4_dense_tc_pair_kernel) on two accumulator sets.  128 < s <= 256: a cluster
// of two CTAs per tile, one stage at a time; CTA r owns rows [128 r, 128 r + 128)
// of B and of the state and writes its rows of each stage's Xs into both CTAs'
// shared memory, so each CTA multiplies its 128 rows of B by the full Xs.  B's
// pieces are fetched once with bulk (TMA) copies and stay in shared memory.
//
// Measured cost (GB300, back-to-back tcgen05.mma of M = 128, K = 16 from one
// thread): about 45 cycles per MMA for N <= 64 whether A comes from shared or
// tensor memory, 64 at N = 128 and 128 at N = 256 (the full BF16 rate, about
// 8,150 flop per cycle per SM); the issuing thread is held for about as long as
// its MMAs run.  A stage here issues 24 MMAs (bf16x5, s = 128: 8 K chunks x 3 grouped
// products of N = 64, 64 and 32), about 1,080 cycles a stage (40 MMAs of N = 32 before
// the grouping: 1,800), and the epilogue (TMEM loads, FP32 sums, stage update,
// publishing Xs, barrier) runs on packed pairs of instances (FADD2 / FFMA2).  Wider tiles
// would need the state of 64 instances per SM, which fits neither the register file nor
// tensor memory beside the accumulators.  A warp that only issues MMAs was measured slower
// in both forms tried: with setmaxnreg (the epilogue then spilled) and with 17 warps and
// the state in tensor memory (the mbarrier hand-over and the state traffic cost more than
// the issuing thread's wait).
//
// Per CTA: 16 warps.  Warp w reads TMEM lanes 32 (w % 4) .. +31 (rows of its
// 128-row block) and columns 8 (w / 4) .. +7 (instances); each thread keeps the
// state of one row for eight instances in registers.  Thread 0 issues the MMAs.
// (Splitting a CTA into two independent 16-instance tiles that share B, so that
// one tile's MMAs overlap the other's epilogue, was measured slower: the MMAs are
// half as wide and twice as many, s = 128 bf16x3 75.8 ms against 61.4 ms.)
//
// Operand layouts in shared memory (no swizzle, 16-byte core matrices of
// 8 rows x 16 bytes):
//   B (A operand, K-major): row m, column k of a 16-column chunk at
//     (m / 8) * 256 + ((k % 16) / 8) * 128 + (m % 8) * 16 + (k % 8) * 2, chunks 4096 B
//     apart: descriptor LBO = 128 (K direction), SBO = 256 (M direction).
//   Xs (B operand, MN-major): instance n, DOF k of a 16-DOF chunk at
//     ((k % 16) / 8) * 512 + (n / 8) * 128 + (k % 8) * 16 + (n % 8) * 2, chunks 1024 B
//     apart: descriptor LBO = 512 (K direction), SBO = 128 (N direction).
// Every wait on an mbarrier gives up after about a second; the kernel then
// records the failure in an error word and leaves the integration.
#include "cho_internal.h"
#include "ctx.h"
#include "rk4_common.cuh"

#include <cuda_bf16.h>
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <vector>

namespace cho {
namespace {

constexpr int kTcWarps = 16;
constexpr int kTcThreads = kTcWarps * 32;
constexpr int kNT = 32;            // instances per tile (MMA N)
constexpr int kCPT = 8;            // instances per thread
constexpr int kAChunk = 4096;      // bytes of one 128 x 16 chunk of B
constexpr int kXChunk = 1024;      // bytes of one 16 x 32 chunk of Xs
constexpr int kBPieces = 3;        // BF16 pieces of B kept per CTA rank
constexpr unsigned long long kWaitNs = 1000000000ull;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t globaltimer()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFF);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;          // descriptor version of tcgen05
    return d;                        // base offset 0, no swizzle
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

// Bounded wait for the phase with the given parity; false after kWaitNs.  The
// suspend-time hint lets a waiting warp sleep until the phase completes (or the hint
// runs out) instead of spinning: the warps that wait for the MMAs share the SM's
// issue slots with the one that issues them.
constexpr uint32_t kSuspendNs = 20000;

__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity)
{
    const uint64_t t0 = globaltimer();
    while (true) {
        uint32_t done;
        asm volatile(
            "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\nselp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(smem_u32(bar)), "r"(parity), "r"(kSuspendNs)
            : "memory");
        if (done) return true;
        if (globaltimer() - t0 > kWaitNs) return false;
    }
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accumulate)
{
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\ntcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void mma_commit(uint64_t* bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float (&v)[8])
{
    uint32_t r[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

// Four accumulators' x8 column groups (kNT columns apart) with a single wait.
__device__ __forceinline__ void tmem_ld8_x4(uint32_t taddr, float (&v)[4][8])
{
    uint32_t r[4][8];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%32];\n"
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%8,%9,%10,%11,%12,%13,%14,%15}, [%33];\n"
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%16,%17,%18,%19,%20,%21,%22,%23}, [%34];\n"
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%24,%25,%26,%27,%28,%29,%30,%31}, [%35];\n"
        "tcgen05.wait::ld.sync.aligned;\n"
        : "=r"(r[0][0]), "=r"(r[0][1]), "=r"(r[0][2]), "=r"(r[0][3]), "=r"(r[0][4]), "=r"(r[0][5]), "=r"(r[0][6]),
          "=r"(r[0][7]), "=r"(r[1][0]), "=r"(r[1][1]), "=r"(r[1][2]), "=r"(r[1][3]), "=r"(r[1][4]), "=r"(r[1][5]),
          "=r"(r[1][6]), "=r"(r[1][7]), "=r"(r[2][0]), "=r"(r[2][1]), "=r"(r[2][2]), "=r"(r[2][3]), "=r"(r[2][4]),
          "=r"(r[2][5]), "=r"(r[2][6]), "=r"(r[2][7]), "=r"(r[3][0]), "=r"(r[3][1]), "=r"(r[3][2]), "=r"(r[3][3]),
          "=r"(r[3][4]), "=r"(r[3][5]), "=r"(r[3][6]), "=r"(r[3][7])
        : "r"(taddr), "r"(taddr + (uint32_t)kNT), "r"(taddr + (uint32_t)(2 * kNT)), "r"(taddr + (uint32_t)(3 * kNT))
        : "memory");
#pragma unroll
    for (int g = 0; g < 4; ++g)
#pragma unroll
        for (int i = 0; i < 8; ++i) v[g][i] = __uint_as_float(r[g][i]);
}

// Grouped products.  An MMA of N <= 64 costs about as much as one of
// N = 32, so the MMA of B piece a covers all the Xs pieces paired with it, laid side by
// side along N (32 columns per piece), and writes accumulator columns from 32 a on:
// column group g of an accumulator then collects the products of order g (b0 p0; b0 p1 +
// b1 p0; b1 p1 + b2 p0 [+ b0 p2]), added smallest first in FP32.  Per K chunk, in an order
// where every MMA that starts its columns starts all of them:
//   x3 (PA 2, PB 2): b0.[p0 p1], b1.[p0]            (2 MMAs instead of 3)
//   x5 (PA 3, PB 2): b0.[p0 p1], b2.[p0], b1.[p0 p1] (3 instead of 5)
//   x6 (PA 3, PB 3): b0.[p0 p1 p2], b1.[p0 p1], b2.[p0] (3 instead of 6)
__host__ __device__ constexpr int grp_a(int PA, int PB, int m)       // B piece of the m-th MMA
{
    return PA == 2 ? m : (PB == 2 ? (m == 0 ? 0 : (m == 1 ? 2 : 1)) : m);
}
__host__ __device__ constexpr int grp_np(int PA, int PB, int a)      // Xs pieces paired with B piece a
{
    return PA == 2 ? (a == 0 ? 2 : 1) : (PB == 2 ? (a == 2 ? 1 : 2) : 3 - a);
}
__host__ __device__ constexpr bool grp_starts(int PA, int PB, int m) // the m-th MMA may start its columns
{
    return PA == 2 ? m == 0 : (PB == 2 ? m <= 1 : m == 0);
}
constexpr int grp_width(int PA) { return PA == 2 ? 64 : 96; }         // columns of one accumulator
// Accumulators of the cluster kernel (one set, no stage pairing): bf16x3 one of two column
// groups (its truncation error dominates); bf16x5 five of three groups, 480 of the 512 TMEM
// columns, the 16 K chunks of s = 256 dealt round-robin (four, then three per accumulator)
constexpr int cluster_nacc(int PA) { return PA == 2 ? 1 : 5; }

__device__ __forceinline__ uint32_t tc_idesc(int n)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | (1u << 16) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

// Two accumulators' x8 column groups (kNT columns apart) with a single wait.
__device__ __forceinline__ void tmem_ld8_x2(uint32_t taddr, float (&v)[2][8])
{
    uint32_t r[2][8];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%16];\n"
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%8,%9,%10,%11,%12,%13,%14,%15}, [%17];\n"
        "tcgen05.wait::ld.sync.aligned;\n"
        : "=r"(r[0][0]), "=r"(r[0][1]), "=r"(r[0][2]), "=r"(r[0][3]), "=r"(r[0][4]), "=r"(r[0][5]), "=r"(r[0][6]),
          "=r"(r[0][7]), "=r"(r[1][0]), "=r"(r[1][1]), "=r"(r[1][2]), "=r"(r[1][3]), "=r"(r[1][4]), "=r"(r[1][5]),
          "=r"(r[1][6]), "=r"(r[1][7])
        : "r"(taddr), "r"(taddr + (uint32_t)kNT)
        : "memory");
#pragma unroll
    for (int g = 0; g < 2; ++g)
#pragma unroll
        for (int i = 0; i < 8; ++i) v[g][i] = __uint_as_float(r[g][i]);
}

// comp_update on packed pairs: each lane rounds as the scalar form in rk4_common.cuh.
__device__ __forceinline__ void comp_update2(float2& x, float2& e, float2 k, float2 h6, float2 h6lo)
{
    float2 y = __ffma2_rn(h6lo, k, e);
    y = __ffma2_rn(h6, k, y);
    const float2 t = __fadd2_rn(x, y);
    const float2 d = __fadd2_rn(t, make_float2(-x.x, -x.y));
    e = __fadd2_rn(y, make_float2(-d.x, -d.y));
    x = t;
}

// Batch form: FP64 arrays in and out, shared step count, checkpoints.
struct TcBatchSrc {
    BatchIO io;
    int s;
    __device__ int64_t count() const { return io.n_inst; }
    __device__ double h(int64_t q) const { return io.h[io.h_per_inst ? q : 0]; }
    __device__ int64_t steps(int64_t) const { return io.n_steps; }
    __device__ int64_t ckpt_every() const { return io.ckpt_every; }
    __device__ void load(int64_t q, int k, float& x, float& v, float& cx, float& cv) const
    {
        const double xd = io.x0[q * s + k], vd = io.v0[q * s + k];
        x = (float)xd;
        v = (float)vd;
        cx = (float)(xd - (double)x);
        cv = (float)(vd - (double)v);
    }
    __device__ void checkpoint(int64_t q, int64_t ck, int k, float x, float v, float cx, float cv) const
    {
        if (!io.x_traj) return;
        const int64_t o = (q * io.n_ck + ck) * s + k;
        io.x_traj[o] = (double)x + (double)cx;
        if (io.v_traj) io.v_traj[o] = (double)v + (double)cv;
    }
    __device__ void store(int64_t q, int k, float x, float v, float cx, float cv) const
    {
        io.x_out[q * s + k] = (double)x + (double)cx;
        io.v_out[q * s + k] = (double)v + (double)cv;
    }
    __device__ void flag(int64_t, int) const {}
    __device__ void book(int64_t, int64_t) const {}
};

// Slot form (serving): FP32 state block [x(s), v(s), cx(s), cv(s)]; each slot runs
// min(chunk, remaining) steps, the tile loops to its largest count.
struct TcSlotSrc {
    SlotIO io;
    int s;
    __device__ const SlotDesc& d(int64_t q) const { return io.slots[io.slot_ids[q]]; }
    __device__ int64_t count() const { return io.n_inst; }
    __device__ double h(int64_t q) const { return d(q).h; }
    __device__ int64_t steps(int64_t q) const { return d(q).remaining < io.chunk ? d(q).remaining : io.chunk; }
    __device__ int64_t ckpt_every() const { return 0; }
    __device__ void load(int64_t q, int k, float& x, float& v, float& cx, float& cv) const
    {
        const float* st = (const float*)d(q).state;
        x = st[k];
        v = st[s + k];
        cx = st[2 * s + k];
        cv = st[3 * s + k];
    }
    __device__ void checkpoint(int64_t, int64_t, int, float, float, float, float) const {}
    __device__ void store(int64_t q, int k, float x, float v, float cx, float cv) const
    {
        float* st = (float*)d(q).state;
        st[k] = x;
        st[s + k] = v;
        st[2 * s + k] = cx;
        st[3 * s + k] = cv;
    }
    __device__ void flag(int64_t q, int code) const { io.status[io.slot_ids[q]] = code; }
    __device__ void book(int64_t q, int64_t ran) const { io.slots[io.slot_ids[q]].remaining -= ran; }
};

constexpr uint32_t tc_pow2(uint32_t n) { return n <= 32 ? 32 : (n <= 64 ? 64 : (n <= 128 ? 128 : (n <= 256 ? 256 : 512))); }

// Balanced schedule (batch form, more tiles than CTAs or clusters fit at once).  A launch
// of one CTA (or cluster) per tile runs ceil(U / P) waves (8,192 instances of s = 128: 256
// tiles on 152 SMs, two waves of which the second is 68 % full).  Instead P resident units
// (one CTA per SM, or one cluster per SM pair) take the tiles' horizons cut in blocks (of
// ckpt_every steps, or single steps), the U x Tb blocks dealt in order, C = max(Tb,
// ceil(U Tb / P)) to each unit (McNaughton's wrap-around rule, as for the 2-DOF kernel in
// rk4_small.cu).  A tile cut between units g and g + 1 runs its first blocks at the start
// of unit g + 1, which then publishes the state of all its threads; unit g runs the
// remaining blocks at its end, after a bounded wait (a second plus the time it has run)
// that is normally empty because C >= Tb.  The pieces run exactly the operations of the
// whole-tile launch: the same bits.
struct TcSched {
    int64_t units;          // U tiles; 0: one tile per CTA (blockIdx.x), its whole horizon
    int64_t blocks;         // Tb blocks per tile
    int64_t block_steps;    // steps per block
    int64_t cap;            // C blocks per CTA
    float* xfer;            // [CTAs][4 kCPT][kTcThreads]: the state of the tile cut at the start of a CTA's unit
    unsigned* flag;         // [CTAs], zero before the launch: 1 published, 2 published after a failure
    int withhold;           // test hook: publish no hand-over, so that every wait runs out
};

// A cluster of CS CTAs per tile (128 < s <= 256): PA pieces of B, PB pieces of Xs,
// NACC accumulators; one stage at a time (two accumulator sets of 16 would not fit
// the 512 TMEM columns).
template <int PA, int PB, int CS, int NACC, class Src>
__global__ void __launch_bounds__(kTcThreads, 1) rk4_dense_tc_kernel(DenseSys sys, const Src src, const TcSched sc)
{
    static_assert(CS > 1, "one CTA per tile: rk4_dense_tc_pair_kernel");
    constexpr int NI = kNT;                          // instances per tile
    constexpr int KC = 8 * CS;                       // 16-wide K chunks (K = 128 CS)
    constexpr int A_BYTES = PA * KC * kAChunk;
    constexpr int XCH = PB * kXChunk;                // one K chunk of Xs: its PB pieces side by side
    constexpr int W = grp_width(PA);                 // columns of one accumulator (grouped products)
    constexpr uint32_t TCOLS = tc_pow2((uint32_t)(NACC * W));
    static_assert(NACC * W <= 512, "the accumulators fit tensor memory");
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char* sA = smem;                        // this CTA's 128 rows of B, PA pieces (shared-memory form)
    unsigned char* sX = smem + A_BYTES;              // Xs, PB pieces
    __shared__ __align__(8) uint64_t bar_load;
    __shared__ __align__(8) uint64_t bar_mma;
    __shared__ uint32_t tmem_slot;
    __shared__ int abort_flag[2];
    __shared__ __align__(16) float sh_h[4][NI];      // h, h/2, h/6 hi, h/6 lo of each instance
    __shared__ long long sh_steps[NI];               // steps of each instance in this launch
    __shared__ long long sh_max_steps;
    __shared__ int sh_bad[NI];
    __shared__ unsigned sh_in;                       // hand-over flag seen by thread 0
    __shared__ long long sh_pos;                     // balanced schedule: first block of the next piece
    __shared__ long long sh_tile;                    // tile of the current piece
    __shared__ int sh_to_xfer;                       // the current piece hands its state over
    __shared__ unsigned long long sh_t_start;

    const int tid = threadIdx.x;
    const int warp = tid >> 5;
    const int lane = tid & 31;
    const uint32_t rank = cluster_rank();
    const int quad = warp & 3;
    const int colgrp = warp >> 2;
    const int row = 32 * quad + lane;                // row of this CTA's block
    const int k = 128 * (int)rank + row;             // K index of the MMA (row of Xs)
    const int kio = k;                               // DOF
    const int ib = 0;
    const int s = sys.s;
    const bool live_row = kio < s;
    const int n0 = colgrp * kCPT;                    // first instance column of this thread
    constexpr int kP = kCPT / 2;                     // instance pairs of this thread
    // (h, h/2, h/6 hi, h/6 lo)[c] of the thread's instance pair j
    auto hpair = [&](int c, int j) { return *reinterpret_cast<const float2*>(&sh_h[c][ib + n0 + 2 * j]); };

    // ---- set-up: barriers, TMEM, B into shared memory ----
    if (tid == 0) {
        mbar_init(&bar_load, 1);
        mbar_init(&bar_mma, 1);
        abort_flag[0] = abort_flag[1] = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (tid == 0) {
        sh_t_start = globaltimer();
        sh_pos = sc.units > 0 ? (long long)(blockIdx.x / CS) * sc.cap : -1;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                     "r"(TCOLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_slot;
    cluster_sync();               // the peer's shared memory is initialised before any remote write

    // Cluster-wide agreement on a local outcome: a failing thread flags its own CTA and
    // the peer, then every thread passes the same barrier and reads the same flags.
    auto agree = [&](bool mine) -> bool {
        if (!mine) {
            atomicExch(&abort_flag[0], 1);
            const uint32_t peer = mapa(smem_u32(&abort_flag[1]), rank ^ 1u);
            asm volatile("st.shared::cluster.u32 [%0], %1;" ::"r"(peer), "r"(1) : "memory");
        }
        cluster_sync();
        return abort_flag[0] == 0 && abort_flag[1] == 0;
    };
    bool ok = true;
    {
        if (tid == 0) {
            const unsigned char* src = (const unsigned char*)sys.Bbf + (size_t)rank * kBPieces * KC * kAChunk;
            mbar_expect_tx(&bar_load, A_BYTES);
            for (int off = 0; off < A_BYTES; off += 16384) {
                const int n = A_BYTES - off < 16384 ? A_BYTES - off : 16384;
                bulk_g2s(sA + off, src + off, (uint32_t)n, &bar_load);
            }
        }
        ok = agree(mbar_wait(&bar_load, 0));
    }

    // Xs addresses of this thread's DOF k in every CTA of the cluster (layout of the one-CTA
    // kernel: the PB pieces side by side along N)
    const int kc = k / 16, kk = k % 16;
    const uint32_t xoff = (uint32_t)(kc * XCH + (kk / 8) * (PB * 512) + (n0 / 8) * 128 + (kk % 8) * 16);
    uint32_t xdst[CS];
#pragma unroll
    for (int c = 0; c < CS; ++c) xdst[c] = mapa(smem_u32(sX) + xoff, (uint32_t)c);

    const uint32_t taddr = tmem + ((uint32_t)(32 * quad) << 16) + (uint32_t)n0;
    // operand descriptors of chunk 0; the others add their byte offset / 16
    // (shared-memory addresses stay below 2^18, inside the 14-bit field)
    const uint64_t bdesc0 = smem_desc(smem_u32(sX), PB * 512, 128);
    const uint64_t adesc0 = smem_desc(smem_u32(sA), 128, 256);
    uint32_t phase = 0;
    bool inflight = false;                           // a commit whose wait ran out (same in every thread)
    uint32_t inflight_phase = 0;

    // One stage: publish Xs pieces, MMA, return a = -(B Xs) for this thread's cells.
    auto stage = [&](const float2 (&xs)[kP], float2 (&a)[kP]) -> bool {
        float2 r[kP];
#pragma unroll
        for (int j = 0; j < kP; ++j) r[j] = xs[j];
#pragma unroll
        for (int p = 0; p < PB; ++p) {
            __nv_bfloat162 q[kP];
#pragma unroll
            for (int j = 0; j < kP; ++j) q[j] = __float22bfloat162_rn(r[j]);
            uint4 w;
            w.x = reinterpret_cast<const uint32_t&>(q[0]);
            w.y = reinterpret_cast<const uint32_t&>(q[1]);
            w.z = reinterpret_cast<const uint32_t&>(q[2]);
            w.w = reinterpret_cast<const uint32_t&>(q[3]);
#pragma unroll
            for (int c = 0; c < CS; ++c) st_cluster_v4(xdst[c] + (uint32_t)(p * 512), w);
            if (p + 1 < PB) {
#pragma unroll
                for (int j = 0; j < kP; ++j) {
                    const float2 back = __bfloat1622float2(q[j]);
                    r[j] = __fadd2_rn(r[j], make_float2(-back.x, -back.y));
                }
            }
        }
        // the Xs stores (this CTA's and the peer's) visible to the tensor cores (the async proxy)
        asm volatile("fence.proxy.async.shared::cluster;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        cluster_sync();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (tid == 0 && !sys.stall_mma) {
            // grouped products, B piece by B piece (see grp_a): the MMAs that start columns
            // of an accumulator come before those that only add to them
#pragma unroll
            for (int m = 0; m < PA; ++m) {
                const int a = grp_a(PA, PB, m);
                const uint32_t idesc = tc_idesc(32 * grp_np(PA, PB, a));
                // descriptor address fields count 16-byte units; fully unrolled, so that each
                // chunk's accumulator (c % NACC) is a constant
                uint64_t bd = bdesc0;
                uint64_t ad = adesc0 + (uint64_t)((a * KC * kAChunk) >> 4);
#pragma unroll
                for (int c = 0; c < KC; ++c) {
                    const uint32_t acc = grp_starts(PA, PB, m) ? (c >= NACC ? 1u : 0u) : 1u;
                    mma_bf16(tmem + (uint32_t)((c % NACC) * W + 32 * a), ad, bd, idesc, acc);
                    bd += XCH >> 4;
                    ad += kAChunk >> 4;
                }
            }
            mma_commit(&bar_mma);
        }
        // the whole warp takes the same branch around the .sync.aligned TMEM load
        const bool done = __all_sync(0xffffffffu, mbar_wait(&bar_mma, phase));
        if (!done && !sys.stall_mma) {
            inflight = true;
            inflight_phase = phase;
        }
        phase ^= 1;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        auto pr = [](const float (&g)[kCPT], int j) { return make_float2(g[2 * j], g[2 * j + 1]); };
        float2 acc[kP];
        if (done) {
            if constexpr (PA == 2) {
                // accumulators of two column groups: b0 p0 | b0 p1 + b1 p0
                float2 big[kP], mid[kP];
#pragma unroll
                for (int sl = 0; sl < NACC; ++sl) {
                    float g[2][kCPT];
                    tmem_ld8_x2(taddr + (uint32_t)(sl * W), g);
#pragma unroll
                    for (int j = 0; j < kP; ++j) {
                        big[j] = sl == 0 ? pr(g[0], j) : __fadd2_rn(big[j], pr(g[0], j));
                        mid[j] = sl == 0 ? pr(g[1], j) : __fadd2_rn(mid[j], pr(g[1], j));
                    }
                }
#pragma unroll
                for (int j = 0; j < kP; ++j) acc[j] = __fadd2_rn(big[j], mid[j]);
            } else {
                // accumulators of three column groups: each order summed over the
                // accumulators, the smaller orders then added to the largest
                float2 big[kP], mid[kP], small[kP];
#pragma unroll
                for (int sl = 0; sl < NACC; ++sl) {
                    float g[2][kCPT], g2[kCPT];
                    tmem_ld8_x2(taddr + (uint32_t)(sl * W), g);
                    tmem_ld8(taddr + (uint32_t)(sl * W + 64), g2);
#pragma unroll
                    for (int j = 0; j < kP; ++j) {
                        big[j] = sl == 0 ? pr(g[0], j) : __fadd2_rn(big[j], pr(g[0], j));
                        mid[j] = sl == 0 ? pr(g[1], j) : __fadd2_rn(mid[j], pr(g[1], j));
                        small[j] = sl == 0 ? pr(g2, j) : __fadd2_rn(small[j], pr(g2, j));
                    }
                }
#pragma unroll
                for (int j = 0; j < kP; ++j) acc[j] = __fadd2_rn(big[j], __fadd2_rn(mid[j], small[j]));
            }
        }
#pragma unroll
        for (int j = 0; j < kP; ++j) a[j] = done ? make_float2(-acc[j].x, -acc[j].y) : make_float2(0.f, 0.f);
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        // every CTA has its MMA done (so Xs may be rewritten) and agrees on aborts
        return agree(done);
    };

    float2 x[kP], v[kP], cx[kP], cv[kP];            // instance columns 2j and 2j + 1 of pair j
    // the value of instance column j of a pair array
    auto at = [](float2 (&arr)[kP], int j) -> float& { return (j & 1) ? arr[j >> 1].y : arr[j >> 1].x; };
    // the pieces of this cluster (see TcSched); the piece's description is kept in shared
    // memory, not in registers across the steps
    for (;;) {
        const int64_t g = blockIdx.x / CS;
        const int64_t pos = sh_pos;
        const int64_t pend = sc.units > 0 ? (g * sc.cap + sc.cap < sc.units * sc.blocks ? g * sc.cap + sc.cap
                                                                                        : sc.units * sc.blocks)
                                          : 0;
        if (sc.units > 0 ? pos >= pend : pos == -2) break;
        int64_t tile = g, st0 = 0, st1 = -1, next = -2;   // st1 < 0: the tile's largest step count
        bool from_xfer = false, to_xfer = false;
        if (sc.units > 0) {
            const int64_t u = pos / sc.blocks;
            const int64_t j0 = u * sc.blocks, j1 = j0 + sc.blocks;
            const int64_t end = j1 < pend ? j1 : pend;
            tile = u;
            if (pos > j0) {                         // the first blocks of a tile cut with cluster g - 1
                st1 = (end - pos) * sc.block_steps;
                to_xfer = true;
            } else if (j1 > pend) {                 // the last blocks of a tile cut with cluster g + 1
                st0 = (sc.blocks - (end - pos)) * sc.block_steps;
                st1 = sc.blocks * sc.block_steps;
                from_xfer = true;
            }
            next = end;
        }
        if (tid < NI) {
            const int64_t q = tile * NI + tid;
            const bool live = q < src.count();
            const double hd = live ? src.h(q) : 1.0;
            sh_steps[tid] = live ? (long long)src.steps(q) : 0;
            sh_bad[tid] = 0;
            const double h6 = hd / 6.0;
            sh_h[0][tid] = (float)hd;
            sh_h[1][tid] = (float)(0.5 * hd);
            sh_h[2][tid] = (float)h6;
            sh_h[3][tid] = (float)(h6 - (double)(float)h6);
        }
        if (tid == 0) {
            sh_tile = tile;
            sh_to_xfer = to_xfer ? 1 : 0;
            sh_in = 1u;
        }
        const int64_t me = g * CS + rank;           // this CTA's hand-over slot
        if (from_xfer && tid == 0) {
            // bounded wait for the hand-over of the same rank in cluster g + 1
            const unsigned* f = sc.flag + me + CS;
            const uint64_t t_wait = globaltimer();
            const uint64_t limit = kWaitNs + (t_wait - sh_t_start);
            unsigned seen = 0;
            for (;;) {
                asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(seen) : "l"(f) : "memory");
                if (seen) break;
                if (globaltimer() - t_wait > limit) break;
                __nanosleep(1024);
            }
            __threadfence();
            sh_in = seen;
        }
        __syncthreads();
        if (tid == 0) sh_pos = next;                // read again after this piece's last barrier
        const bool in_ok = sh_in == 1u;
        if (from_xfer) {
            const float* xf = sc.xfer + (size_t)(me + CS) * (4 * kCPT * kTcThreads) + tid;
            const float nan = __int_as_float(0x7fc00000);
#pragma unroll
            for (int j = 0; j < kCPT; ++j) {
                at(x, j) = in_ok ? __ldcg(xf + (0 * kCPT + j) * kTcThreads) : nan;
                at(v, j) = in_ok ? __ldcg(xf + (1 * kCPT + j) * kTcThreads) : nan;
                at(cx, j) = in_ok ? __ldcg(xf + (2 * kCPT + j) * kTcThreads) : nan;
                at(cv, j) = in_ok ? __ldcg(xf + (3 * kCPT + j) * kTcThreads) : nan;
            }
        } else {
#pragma unroll
            for (int j = 0; j < kCPT; ++j) {
                const int64_t q = tile * NI + ib + n0 + j;
                if (live_row && q < src.count()) {
                    src.load(q, kio, at(x, j), at(v, j), at(cx, j), at(cv, j));
                } else {
                    at(x, j) = at(v, j) = at(cx, j) = at(cv, j) = 0.f;
                }
            }
        }
        if (tid == 0) {
            long long m = 0;
            for (int j = 0; j < NI; ++j) m = sh_steps[j] > m ? sh_steps[j] : m;
            sh_max_steps = m;
        }
        // both CTAs of the cluster run the piece, or neither (a failed hand-over ends the
        // cluster's last piece; the abort flags stay set)
        const bool piece_ok = agree(in_ok);

        if (st1 < 0) st1 = ok ? (int64_t)sh_max_steps : 0;
        const int64_t len = st1 - st0;
        const int64_t every = src.ckpt_every() > 0 ? src.ckpt_every() : (len > 0 ? len : 1);
        int64_t ck = src.ckpt_every() > 0 ? st0 / src.ckpt_every() : 0, step = st0;
        for (int64_t done_steps = st0; done_steps < st1 && ok && piece_ok; done_steps += every) {
            for (int64_t it = 0; it < every && ok; ++it, ++step) {
            float2 a[kP], xs[kP], kx[kP], kv[kP], vs[kP];
            const float2 two = make_float2(2.f, 2.f);
            ok = stage(x, a);
#pragma unroll
            for (int j = 0; j < kP; ++j) {
                const float2 h2 = hpair(1, j);
                kx[j] = v[j];
                kv[j] = a[j];
                xs[j] = __ffma2_rn(h2, v[j], x[j]);
                vs[j] = __ffma2_rn(h2, a[j], v[j]);
            }
            if (ok) ok = stage(xs, a);
#pragma unroll
            for (int j = 0; j < kP; ++j) {
                const float2 h2 = hpair(1, j);
                kx[j] = __ffma2_rn(two, vs[j], kx[j]);
                kv[j] = __ffma2_rn(two, a[j], kv[j]);
                xs[j] = __ffma2_rn(h2, vs[j], x[j]);
                vs[j] = __ffma2_rn(h2, a[j], v[j]);
            }
            if (ok) ok = stage(xs, a);
#pragma unroll
            for (int j = 0; j < kP; ++j) {
                const float2 h = hpair(0, j);
                kx[j] = __ffma2_rn(two, vs[j], kx[j]);
                kv[j] = __ffma2_rn(two, a[j], kv[j]);
                xs[j] = __ffma2_rn(h, vs[j], x[j]);
                vs[j] = __ffma2_rn(h, a[j], v[j]);
            }
            if (ok) ok = stage(xs, a);
#pragma unroll
            for (int j = 0; j < kP; ++j) {
                const float2 h6 = hpair(2, j), h6l = hpair(3, j);
                kx[j] = __fadd2_rn(kx[j], vs[j]);
                kv[j] = __fadd2_rn(kv[j], a[j]);
                float2 nx = x[j], ncx = cx[j], nv = v[j], ncv = cv[j];
                comp_update2(nx, ncx, kx[j], h6, h6l);
                comp_update2(nv, ncv, kv[j], h6, h6l);
                if (step < sh_steps[ib + n0 + 2 * j]) {       // instances past their count hold still
                    x[j].x = nx.x;
                    cx[j].x = ncx.x;
                    v[j].x = nv.x;
                    cv[j].x = ncv.x;
                }
                if (step < sh_steps[ib + n0 + 2 * j + 1]) {
                    x[j].y = nx.y;
                    cx[j].y = ncx.y;
                    v[j].y = nv.y;
                    cv[j].y = ncv.y;
                }
            }
        }
            if (src.ckpt_every() > 0 && ok) {
                if (live_row) {
                    const int64_t tq = *(volatile long long*)&sh_tile;
#pragma unroll
                    for (int j = 0; j < kCPT; ++j) {
                        const int64_t q = tq * NI + ib + n0 + j;
                        if (q < src.count()) src.checkpoint(q, ck, kio, at(x, j), at(v, j), at(cx, j), at(cv, j));
                    }
                }
                ++ck;
            }
        }
        const int64_t tile_out = *(volatile long long*)&sh_tile;
        if (*(volatile int*)&sh_to_xfer) {
            // publish the state of every thread for cluster g - 1 (2 after a failure)
            float* xf = sc.xfer + (size_t)(blockIdx.x) * (4 * kCPT * kTcThreads) + tid;
#pragma unroll
            for (int j = 0; j < kCPT; ++j) {
                __stcg(xf + (0 * kCPT + j) * kTcThreads, at(x, j));
                __stcg(xf + (1 * kCPT + j) * kTcThreads, at(v, j));
                __stcg(xf + (2 * kCPT + j) * kTcThreads, at(cx, j));
                __stcg(xf + (3 * kCPT + j) * kTcThreads, at(cv, j));
            }
            __threadfence();
            __syncthreads();
            if (tid == 0 && !sc.withhold) {
                const unsigned val = ok ? 1u : 2u;
                asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(sc.flag + blockIdx.x), "r"(val) : "memory");
            }
            continue;
        }
        if (live_row) {
#pragma unroll
            for (int j = 0; j < kCPT; ++j) {
                const int64_t q = tile_out * NI + ib + n0 + j;
                if (q < src.count()) {
                    src.store(q, kio, at(x, j), at(v, j), at(cx, j), at(cv, j));
                    if (!(isfinite(at(x, j)) && isfinite(at(v, j)))) sh_bad[ib + n0 + j] = 1;
                }
            }
        }
        __syncthreads();
        if (tid < NI) {
            const int64_t q = tile_out * NI + tid;
            if (q < src.count()) {
                if (!(ok && piece_ok)) src.flag(q, CHO_ETIMEOUT);
                else if (sh_bad[tid]) src.flag(q, CHO_ENONFINITE);
                if (rank == 0) src.book(q, ok && piece_ok ? (int64_t)sh_steps[tid] : 0);
            }
        }
        if (!piece_ok && tid == 0 && sys.err) atomicExch(sys.err, 1);
        __syncthreads();                            // sh_* free for the next piece
    }
    // after a failed wait: wait once more (bounded) for the MMAs still in flight before
    // the accumulators are freed
    if (inflight) (void)mbar_wait(&bar_mma, inflight_phase);
    if (!ok && tid == 0 && sys.err) atomicExch(sys.err, 1);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TCOLS));
    cluster_sync();               // the peer may still write into this CTA's shared memory until here
}

// One CTA per tile (s <= 128), stages paired.  For x'' = -B x the RK4 stage
// displacements are x, x + h/2 v, x + h/2 v2 and x + h v3 with v2 = v + h/2 a1 and
// v3 = v + h/2 a2: the third needs only the first product and the fourth only the
// second.  So the products of stages 1 and 2 go to the tensor cores together,
// each into its own set of accumulators and from its own Xs buffers; the epilogue
// of stage 1 (which yields stage 3's Xs) runs while stage 2's MMAs execute, and
// that of stage 2 (stage 4's Xs) while stage 3's do.  The tensor cores then
// wait only for the step's final update.  Every value is formed by the same
// operations as in rk4_dense_tc_kernel, so both give the same bits.  B's pieces
// stay in shared memory: two accumulator sets fill the 512 TMEM columns, and an
// MMA this narrow costs the same with A from shared memory.
template <int PA, int PB, int NACC, int PK, class Src>
__global__ void __launch_bounds__(kTcThreads, 1) rk4_dense_tc_pair_kernel(DenseSys sys, const Src src, const TcSched sc)
{
    constexpr int NI = kNT * PK;                     // instances per CTA
    constexpr int KC = 8;                            // 16-wide K chunks (K = 128)
    constexpr int A_BYTES = PA * KC * kAChunk;
    constexpr int XCH = PB * kXChunk;                // one K chunk of Xs: its PB pieces side by side
    constexpr int X_BYTES = KC * XCH;                // one Xs buffer set
    constexpr int W = grp_width(PA);                 // columns of one accumulator
    constexpr uint32_t TCOLS = tc_pow2((uint32_t)(2 * NACC * W));
    static_assert(2 * NACC * W <= 512, "two accumulator sets fit tensor memory");
    static_assert((PA == 2 && NACC == 1) || (PA == 3 && (NACC == 1 || NACC == 2)), "accumulators read by collect()");
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char* sA = smem;                        // B, PA pieces
    unsigned char* sX = smem + A_BYTES;              // two Xs buffer sets of PB pieces
    __shared__ __align__(8) uint64_t bar_load;
    __shared__ __align__(8) uint64_t bar_mma[2];
    __shared__ uint32_t tmem_slot;
    __shared__ int abort_flag;
    __shared__ __align__(16) float sh_h[4][NI];      // h, h/2, h/6 hi, h/6 lo of each instance
    __shared__ long long sh_steps[NI];               // steps of each instance in this launch
    __shared__ long long sh_max_steps;
    __shared__ int sh_bad[NI];
    __shared__ unsigned sh_in;                       // hand-over flag seen by thread 0
    __shared__ long long sh_pos;                     // balanced schedule: first block of the next piece
    __shared__ long long sh_tile;                    // tile of the current piece
    __shared__ int sh_to_xfer;                       // the current piece hands its state over
    __shared__ unsigned long long sh_t_start;

    const int tid = threadIdx.x;
    const int warp = tid >> 5;
    const int lane = tid & 31;
    const int quad = warp & 3;
    const int colgrp = warp >> 2;
    const int row = 32 * quad + lane;                // row of the 128-row block = K index of the MMA
    const int kio = PK == 2 ? (row & 63) : row;      // DOF
    const int ib = PK == 2 ? (row >> 6) * kNT : 0;   // first instance slot of this row's tile half
    const int s = sys.s;
    const bool live_row = kio < s;
    const int n0 = colgrp * kCPT;                    // first instance column of this thread
    constexpr int kP = kCPT / 2;                     // instance pairs of this thread
    // (h, h/2, h/6 hi, h/6 lo)[c] of the thread's instance pair j
    auto hpair = [&](int c, int j) { return *reinterpret_cast<const float2*>(&sh_h[c][ib + n0 + 2 * j]); };

    if (tid == 0) {
        mbar_init(&bar_load, 1);
        mbar_init(&bar_mma[0], 1);
        mbar_init(&bar_mma[1], 1);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                     "r"(TCOLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_slot;

    // agreement on a local outcome: every thread passes the barrier and reads the flag
    auto agree = [&](bool mine) -> bool {
        if (!mine) atomicExch(&abort_flag, 1);
        __syncthreads();
        return abort_flag == 0;
    };
    if (tid == 0) {
        const unsigned char* img = (const unsigned char*)sys.Bbf;
        mbar_expect_tx(&bar_load, A_BYTES);
        for (int off = 0; off < A_BYTES; off += 16384) {
            const int n = A_BYTES - off < 16384 ? A_BYTES - off : 16384;
            bulk_g2s(sA + off, img + off, (uint32_t)n, &bar_load);
        }
    }
    if (tid == 0) {
        sh_t_start = globaltimer();
        sh_pos = sc.units > 0 ? (long long)blockIdx.x * sc.cap : -1;
    }
    bool ok = agree(mbar_wait(&bar_load, 0));

    // Xs chunk layout (MN-major, no swizzle): instance column n of piece p at N index 32 p + n;
    // the two 8-row K halves LBO = PB * 512 bytes apart, 8-column groups SBO = 128 apart
    const int kc = row / 16, kk = row % 16;
    const uint32_t xoff = (uint32_t)(kc * XCH + (kk / 8) * (PB * 512) + (n0 / 8) * 128 + (kk % 8) * 16);
    const uint32_t xdst = smem_u32(sX) + xoff;      // this thread's cells of piece 0 in buffer set 0
    const uint32_t tlane = tmem + ((uint32_t)(32 * quad) << 16) + (uint32_t)n0;
    const uint64_t adesc0 = smem_desc(smem_u32(sA), 128, 256);
    uint32_t phase[2] = {0u, 0u};
    bool inflight[2] = {false, false};               // a commit not yet waited for (same in every thread)

    // Xs pieces of xs into buffer set b (instance columns in pairs: one conversion
    // instruction per pair, the residual in packed FP32; the same roundings as per value)
    auto publish = [&](int b, const float2 (&xs)[kP]) {
        float2 r[kP];
#pragma unroll
        for (int j = 0; j < kP; ++j) r[j] = xs[j];
#pragma unroll
        for (int p = 0; p < PB; ++p) {
            __nv_bfloat162 q[kP];
#pragma unroll
            for (int j = 0; j < kP; ++j) q[j] = __float22bfloat162_rn(r[j]);
            uint4 w;
            w.x = reinterpret_cast<const uint32_t&>(q[0]);
            w.y = reinterpret_cast<const uint32_t&>(q[1]);
            w.z = reinterpret_cast<const uint32_t&>(q[2]);
            w.w = reinterpret_cast<const uint32_t&>(q[3]);
            st_cluster_v4(xdst + (uint32_t)(b * X_BYTES + p * 512), w);
            if (p + 1 < PB) {
#pragma unroll
                for (int j = 0; j < kP; ++j) {
                    const float2 back = __bfloat1622float2(q[j]);
                    r[j] = __fadd2_rn(r[j], make_float2(-back.x, -back.y));
                }
            }
        }
    };
    // every thread's Xs stores visible to the tensor cores and its TMEM loads done; agree
    auto sync = [&](bool mine) -> bool {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        const bool go = agree(mine);
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        return go;
    };
    // thread 0: the stage's products from buffer set b into accumulator set b
    auto issue = [&](int b) {
        if (tid == 0 && !sys.stall_mma) {
            const uint64_t bdesc0 = smem_desc(smem_u32(sX + b * X_BYTES), PB * 512, 128);
            const uint32_t dcol = tmem + (uint32_t)(b * NACC * W);
            // B piece by B piece, K chunk by K chunk: in each accumulator the MMAs that start
            // columns (m = 0, and for x5 m = 1) come before those that only add to them
#pragma unroll
            for (int m = 0; m < PA; ++m) {
                const int a = grp_a(PA, PB, m);
                const uint32_t idesc = tc_idesc(32 * grp_np(PA, PB, a));
                uint64_t bd = bdesc0;
                uint64_t ad = adesc0 + (uint64_t)((a * KC * kAChunk) >> 4);
#pragma unroll
                for (int c = 0; c < KC; ++c) {
                    const uint32_t acc = grp_starts(PA, PB, m) ? (c >= NACC ? 1u : 0u) : 1u;
                    mma_bf16(dcol + (uint32_t)((c % NACC) * W + 32 * a), ad, bd, idesc, acc);
                    bd += XCH >> 4;
                    ad += kAChunk >> 4;
                }
            }
            mma_commit(&bar_mma[b]);
        }
        inflight[b] = !sys.stall_mma;
    };
    // wait for accumulator set b and return a = -(B Xs) for this thread's cells, the column
    // groups summed in packed FP32 (pairs of instances; each lane rounds as a scalar add)
    auto collect = [&](int b, float2 (&a)[kP]) -> bool {
        const bool done = __all_sync(0xffffffffu, mbar_wait(&bar_mma[b], phase[b]));
        if (done) {
            phase[b] ^= 1u;
            inflight[b] = false;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        auto pr = [](const float (&g)[kCPT], int j) { return make_float2(g[2 * j], g[2 * j + 1]); };
        float2 acc[kP];
        if (done) {
            const uint32_t taddr = tlane + (uint32_t)(b * NACC * W);
            if constexpr (PA == 2) {
                // one accumulator: b0 p0 | b0 p1 + b1 p0
                float g[2][kCPT];
                tmem_ld8_x2(taddr, g);
#pragma unroll
                for (int j = 0; j < kP; ++j) acc[j] = __fadd2_rn(pr(g[0], j), pr(g[1], j));
            } else if constexpr (NACC == 1) {
                // one accumulator of three column groups, the smaller orders first
                float g[2][kCPT], g2[kCPT];
                tmem_ld8_x2(taddr, g);
                tmem_ld8(taddr + 64u, g2);
#pragma unroll
                for (int j = 0; j < kP; ++j) acc[j] = __fadd2_rn(pr(g[0], j), __fadd2_rn(pr(g[1], j), pr(g2, j)));
            } else {
                // two accumulators of three column groups: each order summed over the two,
                // then the smaller orders added to the largest
                float g[4][kCPT];
                tmem_ld8_x4(taddr, g);                          // slot 0: G0 G1 G2; slot 1: G0
                float h[2][kCPT];
                tmem_ld8_x2(taddr + (uint32_t)(W + 32), h);      // slot 1: G1 G2
#pragma unroll
                for (int j = 0; j < kP; ++j) {
                    const float2 big = __fadd2_rn(pr(g[0], j), pr(g[3], j));
                    acc[j] = __fadd2_rn(big, __fadd2_rn(__fadd2_rn(pr(g[1], j), pr(h[0], j)),
                                                       __fadd2_rn(pr(g[2], j), pr(h[1], j))));
                }
            }
        }
#pragma unroll
        for (int j = 0; j < kP; ++j) a[j] = done ? make_float2(-acc[j].x, -acc[j].y) : make_float2(0.f, 0.f);
        return done;
    };

    float2 x[kP], v[kP], cx[kP], cv[kP];            // instance columns 2j and 2j + 1 of pair j
    // the value of instance column j of a pair array
    auto at = [](float2 (&arr)[kP], int j) -> float& { return (j & 1) ? arr[j >> 1].y : arr[j >> 1].x; };
    // the pieces of this CTA: (tile, steps [st0, st1), state from the hand-over of CTA
    // g + 1 or from the input, state to the hand-over of this CTA or to the output).  The
    // piece's description is kept in shared memory, not in registers across the steps.
    for (;;) {
        const int64_t g = blockIdx.x;
        const int64_t pos = sh_pos;
        const int64_t pend = sc.units > 0 ? (g * sc.cap + sc.cap < sc.units * sc.blocks ? g * sc.cap + sc.cap
                                                                                        : sc.units * sc.blocks)
                                          : 0;
        if (sc.units > 0 ? pos >= pend : pos == -2) break;
        int64_t tile = g, st0 = 0, st1 = -1, next = -2;   // st1 < 0: the tile's largest step count
        bool from_xfer = false, to_xfer = false;
        if (sc.units > 0) {
            const int64_t u = pos / sc.blocks;
            const int64_t j0 = u * sc.blocks, j1 = j0 + sc.blocks;
            const int64_t end = j1 < pend ? j1 : pend;
            tile = u;
            if (pos > j0) {                         // the first blocks of a tile cut with CTA g - 1
                st1 = (end - pos) * sc.block_steps;
                to_xfer = true;
            } else if (j1 > pend) {                 // the last blocks of a tile cut with CTA g + 1
                st0 = (sc.blocks - (end - pos)) * sc.block_steps;
                st1 = sc.blocks * sc.block_steps;
                from_xfer = true;
            }
            next = end;
        }
        if (tid < NI) {
            const int64_t q = tile * NI + tid;
            const bool live = q < src.count();
            const double hd = live ? src.h(q) : 1.0;
            sh_steps[tid] = live ? (long long)src.steps(q) : 0;
            sh_bad[tid] = 0;
            const double h6 = hd / 6.0;
            sh_h[0][tid] = (float)hd;
            sh_h[1][tid] = (float)(0.5 * hd);
            sh_h[2][tid] = (float)h6;
            sh_h[3][tid] = (float)(h6 - (double)(float)h6);
        }
        if (tid == 0) {
            sh_tile = tile;
            sh_to_xfer = to_xfer ? 1 : 0;
        }
        if (from_xfer && tid == 0) {
            // bounded wait for CTA g + 1's hand-over
            const unsigned* f = sc.flag + g + 1;
            const uint64_t t_wait = globaltimer();
            const uint64_t limit = kWaitNs + (t_wait - sh_t_start);
            unsigned seen = 0;
            for (;;) {
                asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(seen) : "l"(f) : "memory");
                if (seen) break;
                if (globaltimer() - t_wait > limit) break;
                __nanosleep(1024);
            }
            __threadfence();
            sh_in = seen;
        }
        __syncthreads();
        if (tid == 0) sh_pos = next;                // read again after this piece's last barrier
        bool piece_ok = ok;
        if (from_xfer) {
            piece_ok = ok && sh_in == 1u;
            const float* xf = sc.xfer + (size_t)(g + 1) * (4 * kCPT * kTcThreads) + tid;
            const float nan = __int_as_float(0x7fc00000);
#pragma unroll
            for (int j = 0; j < kCPT; ++j) {
                at(x, j) = piece_ok ? __ldcg(xf + (0 * kCPT + j) * kTcThreads) : nan;
                at(v, j) = piece_ok ? __ldcg(xf + (1 * kCPT + j) * kTcThreads) : nan;
                at(cx, j) = piece_ok ? __ldcg(xf + (2 * kCPT + j) * kTcThreads) : nan;
                at(cv, j) = piece_ok ? __ldcg(xf + (3 * kCPT + j) * kTcThreads) : nan;
            }
        } else {
#pragma unroll
            for (int j = 0; j < kCPT; ++j) {
                const int64_t q = tile * NI + ib + n0 + j;
                if (live_row && q < src.count()) {
                    src.load(q, kio, at(x, j), at(v, j), at(cx, j), at(cv, j));
                } else {
                    at(x, j) = at(v, j) = at(cx, j) = at(cv, j) = 0.f;
                }
            }
        }
        if (tid == 0) {
            long long m = 0;
            for (int j = 0; j < NI; ++j) m = sh_steps[j] > m ? sh_steps[j] : m;
            sh_max_steps = m;
        }
        __syncthreads();

        if (st1 < 0) st1 = ok ? (int64_t)sh_max_steps : 0;
        const int64_t len = st1 - st0;
        const int64_t every = src.ckpt_every() > 0 ? src.ckpt_every() : (len > 0 ? len : 1);
        int64_t ck = src.ckpt_every() > 0 ? st0 / src.ckpt_every() : 0, step = st0;
        for (int64_t done_steps = st0; done_steps < st1 && ok && piece_ok; done_steps += every) {
            // the last product of a step is agreed on at the next step's first barrier (or after
            // the block, before its results are written): a failure there ends the run
            bool good_prev = true;
            for (int64_t it = 0; it < every && ok; ++it, ++step) {
            float2 a[kP], xs[kP], kx[kP], kv[kP], vm[kP];
            const float2 two = make_float2(2.f, 2.f);
            // stages 1 and 2 together: Xs = x and x + h/2 v
#pragma unroll
            for (int j = 0; j < kP; ++j) xs[j] = __ffma2_rn(hpair(1, j), v[j], x[j]);
            publish(0, x);
            publish(1, xs);
            if (!(ok = sync(good_prev))) break;
            issue(0);
            issue(1);
            // stage 1 result: a1; stage 3's Xs = x + h/2 v2 with v2 = v + h/2 a1
            bool good = collect(0, a);
#pragma unroll
            for (int j = 0; j < kP; ++j) {
                const float2 h2 = hpair(1, j);
                kx[j] = v[j];
                kv[j] = a[j];
                vm[j] = __ffma2_rn(h2, a[j], v[j]);     // v2
                xs[j] = __ffma2_rn(h2, vm[j], x[j]);    // x3
            }
            publish(0, xs);
            if (!(ok = sync(good))) break;
            issue(0);
            // stage 2 result: a2; stage 4's Xs = x + h v3 with v3 = v + h/2 a2
            good = collect(1, a);
#pragma unroll
            for (int j = 0; j < kP; ++j) {
                const float2 h2 = hpair(1, j), h = hpair(0, j);
                kx[j] = __ffma2_rn(two, vm[j], kx[j]);
                kv[j] = __ffma2_rn(two, a[j], kv[j]);
                vm[j] = __ffma2_rn(h2, a[j], v[j]);     // v3
                xs[j] = __ffma2_rn(h, vm[j], x[j]);     // x4
            }
            publish(1, xs);
            if (!(ok = sync(good))) break;
            issue(1);
            // stage 3 result: a3; v4 = v + h a3
            good = collect(0, a);
#pragma unroll
            for (int j = 0; j < kP; ++j) {
                const float2 h = hpair(0, j);
                kx[j] = __ffma2_rn(two, vm[j], kx[j]);
                kv[j] = __ffma2_rn(two, a[j], kv[j]);
                vm[j] = __ffma2_rn(h, a[j], v[j]);      // v4
            }
            // stage 4 result: a4, then the step's update (compensated, in packed pairs; an
            // instance past its step count holds still)
            if (good) good = collect(1, a);
            good_prev = good;
#pragma unroll
            for (int j = 0; j < kP; ++j) {
                const float2 h6 = hpair(2, j), h6l = hpair(3, j);
                kx[j] = __fadd2_rn(kx[j], vm[j]);
                kv[j] = __fadd2_rn(kv[j], a[j]);
                float2 nx = x[j], ncx = cx[j], nv = v[j], ncv = cv[j];
                comp_update2(nx, ncx, kx[j], h6, h6l);
                comp_update2(nv, ncv, kv[j], h6, h6l);
                if (step < sh_steps[ib + n0 + 2 * j]) {
                    x[j].x = nx.x;
                    cx[j].x = ncx.x;
                    v[j].x = nv.x;
                    cv[j].x = ncv.x;
                }
                if (step < sh_steps[ib + n0 + 2 * j + 1]) {
                    x[j].y = nx.y;
                    cx[j].y = ncx.y;
                    v[j].y = nv.y;
                    cv[j].y = ncv.y;
                }
            }
        }
            if (ok) ok = agree(good_prev);
            if (src.ckpt_every() > 0 && ok) {
                if (live_row) {
                    const int64_t tq = *(volatile long long*)&sh_tile;
#pragma unroll
                    for (int j = 0; j < kCPT; ++j) {
                        const int64_t q = tq * NI + ib + n0 + j;
                        if (q < src.count()) src.checkpoint(q, ck, kio, at(x, j), at(v, j), at(cx, j), at(cv, j));
                    }
                }
                ++ck;
            }
        }
        const int64_t tile_out = *(volatile long long*)&sh_tile;
        if (*(volatile int*)&sh_to_xfer) {
            // publish the state of every thread for CTA g - 1 (2 after a failure)
            float* xf = sc.xfer + (size_t)blockIdx.x * (4 * kCPT * kTcThreads) + tid;
#pragma unroll
            for (int j = 0; j < kCPT; ++j) {
                __stcg(xf + (0 * kCPT + j) * kTcThreads, at(x, j));
                __stcg(xf + (1 * kCPT + j) * kTcThreads, at(v, j));
                __stcg(xf + (2 * kCPT + j) * kTcThreads, at(cx, j));
                __stcg(xf + (3 * kCPT + j) * kTcThreads, at(cv, j));
            }
            __threadfence();
            __syncthreads();
            if (tid == 0 && !sc.withhold) {
                const unsigned val = ok ? 1u : 2u;
                asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(sc.flag + blockIdx.x), "r"(val) : "memory");
            }
            continue;
        }
        if (live_row) {
#pragma unroll
            for (int j = 0; j < kCPT; ++j) {
                const int64_t q = tile_out * NI + ib + n0 + j;
                if (q < src.count()) {
                    src.store(q, kio, at(x, j), at(v, j), at(cx, j), at(cv, j));
                    if (!(isfinite(at(x, j)) && isfinite(at(v, j)))) sh_bad[ib + n0 + j] = 1;
                }
            }
        }
        __syncthreads();
        if (tid < NI) {
            const int64_t q = tile_out * NI + tid;
            if (q < src.count()) {
                if (!(ok && piece_ok)) src.flag(q, CHO_ETIMEOUT);
                else if (sh_bad[tid]) src.flag(q, CHO_ENONFINITE);
                src.book(q, ok && piece_ok ? (int64_t)sh_steps[tid] : 0);
            }
        }
        if (!piece_ok && tid == 0 && sys.err) atomicExch(sys.err, 1);
        __syncthreads();                            // sh_* free for the next piece
    }
    // after a failed wait: wait once more (bounded) for what is still in flight
    // before the accumulators are freed
#pragma unroll
    for (int b = 0; b < 2; ++b)
        if (inflight[b]) (void)mbar_wait(&bar_mma[b], phase[b]);
    if (!ok && tid == 0 && sys.err) atomicExch(sys.err, 1);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TCOLS));
}

// The balanced schedule when it helps: batch form, more tiles than resident units (CTAs
// or clusters) and not a whole number of waves, a cooperative launch available (it
// guarantees that every unit is resident, so each hand-over wait ends).  The hand-over
// buffer and flags come from the stream-ordered scratch pool and are freed after the
// kernel on the same stream.
template <class Src>
bool tc_balance(const Src&, int64_t, int64_t, int, TcSched*)
{
    return false;
}

bool tc_balance(const TcBatchSrc& src, int64_t tiles, int64_t units, int coop, TcSched* sc)
{
    const BatchIO& io = src.io;
    const int64_t g = io.ckpt_every > 0 ? io.ckpt_every : 1;
    const int64_t Tb = io.n_steps / g;
    if (!coop || tiles <= units || tiles % units == 0 || Tb <= 0 || Tb > ((int64_t)1 << 62) / tiles) return false;
    sc->units = tiles;
    sc->blocks = Tb;
    sc->block_steps = g;
    sc->cap = std::max(Tb, (tiles * Tb + units - 1) / units);
    return true;
}

template <int PA, int PB, int NACC, int PK, class Src>
cudaError_t launch_tc_pair(const DenseSys& sys, const Src& src, int64_t n_inst, cudaStream_t st)
{
    const size_t smem = (size_t)PA * 8 * kAChunk + 2 * (size_t)PB * 8 * kXChunk;
    auto kern = rk4_dense_tc_pair_kernel<PA, PB, NACC, PK, Src>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int64_t tiles = (n_inst + kNT * PK - 1) / (kNT * PK);
    if (tiles <= 0) return cudaSuccess;
    if (tiles > 0x7fffffffLL) return cudaErrorInvalidValue;
    int dev = 0, sms = 0, coop = 0, per_sm = 0;
    e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kTcThreads, smem);
    if (e != cudaSuccess) return e;
    TcSched sc{};
    if (per_sm < 1 || !tc_balance(src, tiles, (int64_t)sms, coop, &sc)) {
        kern<<<(unsigned)tiles, kTcThreads, smem, st>>>(sys, src, sc);
        return cudaGetLastError();
    }
    const char* hook = std::getenv("CHO_TEST_WITHHOLD_HANDOVER");
    sc.withhold = hook && hook[0] == '1' ? 1 : 0;
    const size_t xfer_bytes = (size_t)sms * 4 * kCPT * kTcThreads * sizeof(float);
    void* buf = nullptr;
    e = scratch_alloc(&buf, xfer_bytes + (size_t)sms * sizeof(unsigned), st);
    if (e != cudaSuccess) return e;
    sc.xfer = (float*)buf;
    sc.flag = (unsigned*)((char*)buf + xfer_bytes);
    e = cudaMemsetAsync(sc.flag, 0, (size_t)sms * sizeof(unsigned), st);
    if (e == cudaSuccess) {
        DenseSys a0 = sys;
        Src a1 = src;
        void* args[] = {&a0, &a1, &sc};
        e = cudaLaunchCooperativeKernel((const void*)kern, dim3((unsigned)sms), dim3(kTcThreads), args, smem, st);
    }
    const cudaError_t ef = cudaFreeAsync(buf, st);
    return e != cudaSuccess ? e : ef;
}

// Clusters: the balanced schedule needs every cluster resident at once, which a
// cooperative launch of as many clusters as fit guarantees; where the launch refuses the
// combination of cooperative launch and clusters, one cluster per tile as before.
template <int PA, int PB, int CS, class Src>
cudaError_t launch_tc(const DenseSys& sys, const Src& src, int64_t n_inst, cudaStream_t st)
{
    constexpr int KC = 8 * CS;
    constexpr int NACC = cluster_nacc(PA);
    const size_t smem = (size_t)PA * KC * kAChunk + (size_t)PB * KC * kXChunk;
    auto kern = rk4_dense_tc_kernel<PA, PB, CS, NACC, Src>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int64_t tiles = (n_inst + kNT - 1) / kNT;
    if (tiles <= 0) return cudaSuccess;
    if (tiles * CS > 0x7fffffffLL) return cudaErrorInvalidValue;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(tiles * CS), 1, 1);
    cfg.blockDim = dim3(kTcThreads, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = CS;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    TcSched sc{};
    int dev = 0, coop = 0, clusters = 0;
    e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveClusters(&clusters, kern, &cfg);
    if (e != cudaSuccess) return e;
    if (clusters < 1 || !tc_balance(src, tiles, (int64_t)clusters, coop, &sc))
        return cudaLaunchKernelEx(&cfg, kern, sys, src, sc);
    const char* hook = std::getenv("CHO_TEST_WITHHOLD_HANDOVER");
    sc.withhold = hook && hook[0] == '1' ? 1 : 0;
    const int64_t ctas = (int64_t)clusters * CS;
    const size_t xfer_bytes = (size_t)ctas * 4 * kCPT * kTcThreads * sizeof(float);
    void* buf = nullptr;
    e = scratch_alloc(&buf, xfer_bytes + (size_t)ctas * sizeof(unsigned), st);
    if (e != cudaSuccess) return e;
    sc.xfer = (float*)buf;
    sc.flag = (unsigned*)((char*)buf + xfer_bytes);
    e = cudaMemsetAsync(sc.flag, 0, (size_t)ctas * sizeof(unsigned), st);
    if (e == cudaSuccess) {
        cudaLaunchConfig_t bc = cfg;
        bc.gridDim = dim3((unsigned)ctas, 1, 1);
        attr[1].id = cudaLaunchAttributeCooperative;
        attr[1].val.cooperative = 1;
        bc.numAttrs = 2;
        e = cudaLaunchKernelEx(&bc, kern, sys, src, sc);
        if (e != cudaSuccess) {
            (void)cudaGetLastError();               // the refusal is not sticky: run one cluster per tile
            TcSched none{};
            e = cudaLaunchKernelEx(&cfg, kern, sys, src, none);
        }
    }
    const cudaError_t ef = cudaFreeAsync(buf, st);
    return e != cudaSuccess ? e : ef;
}

template <class Src>
cudaError_t dispatch_tc(const DenseSys& sys, const Src& src, int64_t n_inst, int prec, cudaStream_t st)
{
    if (n_inst == 0) return cudaSuccess;
    if (!sys.Bbf || sys.s_tc == 0) return cudaErrorNotSupported;
    // one CTA per tile (s <= 128): stages paired on two accumulator sets; 2-CTA clusters
    // (s <= 256): one stage at a time
    const bool two = sys.s_tc == 256, pack = sys.s_tc == 64;
    switch (prec) {
        case CHO_DENSE_BF16X3:
            if (two) return launch_tc<2, 2, 2>(sys, src, n_inst, st);
            return pack ? launch_tc_pair<2, 2, 1, 2>(sys, src, n_inst, st) : launch_tc_pair<2, 2, 1, 1>(sys, src, n_inst, st);
        case CHO_DENSE_BF16X5:
            if (two) return launch_tc<3, 2, 2>(sys, src, n_inst, st);
            return pack ? launch_tc_pair<3, 2, 2, 2>(sys, src, n_inst, st) : launch_tc_pair<3, 2, 2, 1>(sys, src, n_inst, st);
        case CHO_DENSE_BF16X6:
            if (two) return cudaErrorNotSupported;   // 192 KB of B plus 48 KB of Xs exceed shared memory
            return pack ? launch_tc_pair<3, 3, 2, 2>(sys, src, n_inst, st) : launch_tc_pair<3, 3, 2, 1>(sys, src, n_inst, st);
        default: return cudaErrorInvalidValue;
    }
}

// Round to the nearest BF16 (ties to even) of an FP32 value, as bits.
uint16_t bf16_bits(float f)
{
    uint32_t u;
    std::memcpy(&u, &f, 4);
    const uint32_t lsb = (u >> 16) & 1u;
    u += 0x7FFFu + lsb;
    return (uint16_t)(u >> 16);
}

float bf16_value(uint16_t b)
{
    const uint32_t u = (uint32_t)b << 16;
    float f;
    std::memcpy(&f, &u, 4);
    return f;
}

}  // namespace

int test_stall_mma()
{
    const char* e = std::getenv("CHO_TEST_STALL_MMA");
    return e && e[0] == '1' ? 1 : 0;
}

cudaError_t launch_rk4_dense_tc(const DenseSys& sys, const BatchIO& io, int prec, cudaStream_t st)
{
    DenseSys d = sys;
    d.stall_mma = test_stall_mma();
    return dispatch_tc(d, TcBatchSrc{io, sys.s}, io.n_inst, prec, st);
}

namespace {

template <int PA, int PB, int NACC, int PK>
int pair_resident()
{
    const size_t smem = (size_t)PA * 8 * kAChunk + 2 * (size_t)PB * 8 * kXChunk;
    auto kern = rk4_dense_tc_pair_kernel<PA, PB, NACC, PK, TcSlotSrc>;
    int n = 0, dev = 0, sms = 0;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, kTcThreads, smem) != cudaSuccess ||
        cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        (void)cudaGetLastError();
        return 0;
    }
    return n * sms * kNT * PK;
}

template <int PA, int PB, int CS>
int cluster_resident()
{
    constexpr int KC = 8 * CS;
    constexpr int NACC = cluster_nacc(PA);
    const size_t smem = (size_t)PA * KC * kAChunk + (size_t)PB * KC * kXChunk;
    auto kern = rk4_dense_tc_kernel<PA, PB, CS, NACC, TcSlotSrc>;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(CS, 1, 1);
    cfg.blockDim = dim3(kTcThreads, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = CS;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
        cudaOccupancyMaxActiveClusters(&n, kern, &cfg) != cudaSuccess) {
        (void)cudaGetLastError();
        return 0;
    }
    return n * kNT;
}

}  // namespace

// Instances the tensor-core slot kernels hold resident at once on this device (0: none).
int dense_tc_slot_resident(const DenseSys& sys, int prec)
{
    const bool two = sys.s_tc == 256, pack = sys.s_tc == 64;
    switch (prec) {
        case CHO_DENSE_BF16X3:
            if (two) return cluster_resident<2, 2, 2>();
            return pack ? pair_resident<2, 2, 1, 2>() : pair_resident<2, 2, 1, 1>();
        case CHO_DENSE_BF16X5:
            if (two) return cluster_resident<3, 2, 2>();
            return pack ? pair_resident<3, 2, 2, 2>() : pair_resident<3, 2, 2, 1>();
        case CHO_DENSE_BF16X6:
            if (two) return 0;
            return pack ? pair_resident<3, 3, 2, 2>() : pair_resident<3, 3, 2, 1>();
        default: return 0;
    }
}

cudaError_t launch_rk4_dense_tc_slots(const DenseSys& sys, const SlotIO& io, int prec, cudaStream_t st)
{
    DenseSys d = sys;
    d.stall_mma = test_stall_mma();
    return dispatch_tc(d, TcSlotSrc{io, sys.s}, io.n_inst, prec, st);
}

// BF16 pieces of B for the tensor-core kernel, laid out per CTA rank as the exact
// shared-memory image the kernel copies: [rank][piece 0..2][K chunk][4096 B].
cudaError_t build_dense_tc_device(cho_system_impl* sys, const double* B)
{
    const int s = sys->s;
    if (s > 256) {
        sys->s_tc = 0;
        return cudaSuccess;
    }
    // s <= 64: two copies of B on the diagonal of a 128 x 128 block (two tiles of
    // instances stacked along the rows); else B padded to 128 or 256.
    const int st = s <= 64 ? 64 : (s <= 128 ? 128 : 256);
    const int CS = st == 256 ? 2 : 1, KC = st == 256 ? 16 : 8;
    sys->s_tc = st;
    const size_t per_rank = (size_t)kBPieces * KC * kAChunk;
    std::vector<unsigned char> img((size_t)CS * per_rank, 0);
    for (int r = 0; r < CS; ++r)
        for (int m = 0; m < 128; ++m) {
            for (int kk = 0; kk < 16 * KC; ++kk) {
                int i = 128 * r + m, j = kk;
                if (st == 64) {
                    if (m / 64 != kk / 64) continue;
                    i = m % 64;
                    j = kk % 64;
                }
                double rem = (i < s && j < s) ? B[(size_t)i * s + j] : 0.0;
                for (int p = 0; p < kBPieces; ++p) {
                    const uint16_t b = bf16_bits((float)rem);
                    rem -= (double)bf16_value(b);
                    const int c = kk / 16, k16 = kk % 16;
                    const size_t off = (size_t)r * per_rank + ((size_t)p * KC + c) * kAChunk + (m / 8) * 256 +
                                       (k16 / 8) * 128 + (m % 8) * 16 + (k16 % 8) * 2;
                    std::memcpy(&img[off], &b, 2);
                }
            }
        }
    cudaError_t e = cudaMalloc(&sys->d_Bbf, img.size());
    if (e == cudaSuccess) e = cudaMemcpy(sys->d_Bbf, img.data(), img.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc(&sys->d_err, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(sys->d_err, 0, sizeof(int));
    return e;
}

}  // namespace cho
