// persist.cuh -- device side of the persistent serving kernels (protocol in persist.h).
#pragma once

#include "cho_internal.h"
#include "persist.h"
#include "rk4_common.cuh"
#include "../../include/cho.h"

namespace cho {

__device__ __forceinline__ uint64_t ld_acquire_sys(const uint64_t* p)
{
    uint64_t v;
    asm volatile("ld.acquire.sys.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ int32_t ld_acquire_sys(const int32_t* p)
{
    int32_t v;
    asm volatile("ld.acquire.sys.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Thread 0: wait for generation `gen`.  1: run it; 0: quit; -1: the wait ran out.  A rung
// generation is run even when quit is set too: the host writes the doorbell before quit,
// so once quit is seen (acquire) a doorbell rung before it is seen as well.
__device__ __forceinline__ int persist_wait(PersistCtl* ctl, uint64_t gen)
{
    const uint64_t t0 = global_ns();
    while (true) {
        if (ld_acquire_sys(&ctl->doorbell) >= gen) return 1;
        if (ld_acquire_sys(&ctl->quit)) return ld_acquire_sys(&ctl->doorbell) >= gen ? 1 : 0;
        if (global_ns() - t0 > kPersistWaitNs) return -1;
        __nanosleep(2000);
    }
}

// Append a finished slot to the completion ring (one thread per slot).
__device__ __forceinline__ void persist_complete(const PersistIO& pio, int32_t slot)
{
    const unsigned long long k = atomicAdd_system(&pio.ctl->ring_head, 1ull);
    ((volatile int32_t*)pio.ring)[k % pio.ring_cap] = slot;
    __threadfence_system();
}

// The generation loop of a persistent kernel: run(n_items, chunk) advances this CTA's
// share of the generation's items.
template <class Run>
__device__ __forceinline__ void persist_loop(const PersistIO& pio, Run&& run)
{
    __shared__ int sh_go;
    __shared__ long long sh_n, sh_chunk;
    for (uint64_t gen = 1;; ++gen) {
        if (threadIdx.x == 0) {
            const int go = persist_wait(pio.ctl, gen);
            if (go < 0) atomicExch_system(&pio.ctl->status, (int)CHO_ETIMEOUT);
            sh_go = go;
            sh_n = ((volatile long long*)&pio.ctl->n_items)[0];
            sh_chunk = ((volatile long long*)&pio.ctl->chunk)[0];
        }
        __syncthreads();
        if (sh_go <= 0) break;
        const int64_t n = sh_n, chunk = sh_chunk;
        __threadfence_system();             // what the host wrote before the doorbell is seen below
        run(n, chunk);
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence_system();
            atomicAdd_system(&pio.ctl->done, 1ull);
        }
    }
}

}  // namespace cho
