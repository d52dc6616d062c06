// serve.cpp -- continuous batching of single-instance integration requests.
//
// cho_submit queues a request (one instance of one parameter set); a worker
// thread owned by the context runs the request loop:
//   1. admission: requests leave three fixed-priority FIFO queues (class 0
//      first; strict priority, no ageing) while a slot is free and their state
//      fits the device-memory budget; each admitted request gets a slot in the
//      device slot table and a resident state block in its kernel's precision;
//   2. one chunk: every active resident request advances min(chunk, remaining) RK4
//      steps; requests are grouped by kernel family (rk4_small by padded size,
//      rk4_chain by threads per CTA, rk4_dense by shared system) and each group
//      is one kernel launch over a list of slot ids.  The active set is chosen in
//      priority order (class, then admission order) up to about one wave of the device
//      (cho_config.active_pct of the instances every kernel holds resident at once);
//      the other resident requests keep their state on the device and wait at their
//      chunk boundary until there is room (fixed-priority preemption at chunk
//      granularity);
//   3. retirement: finished requests are read back, converted to FP64 and
//      handed to cho_poll; their slots and memory go back to the pool, so the
//      next chunk admits more work while the others keep running.
// The state stays on the device between chunks in the kernel's own precision
// (x, v and the Kahan compensations), so a request's result does not depend on
// how its horizon is cut into chunks or on which requests share its launches.
// This follows the paper's use of the model as a fixed-priority real-time
// workload (Section 5) with the GPU as the executor.
//
// Persistent mode (cho_config.persistent): rk4_small groups and chain groups (s <= 2048)
// are served by a kernel that stays resident on the group's stream and runs one chunk
// per generation (persist.h): the slot table, the status words, each group's slot-id
// list and its completion ring live in pinned host memory mapped into the device, the
// host rings a doorbell instead of launching, and the kernel appends finished slots to
// the ring.  State blocks are copied on a second stream of the group while its kernel
// holds the first.  The resident kernels together hold at most half the SMs' worth of
// CTAs (each CTA on one SM at most) and 60 % of the register file, so they stay
// co-resident with each other and at least half the SMs stay whole for the relaunched
// kernels (dense groups, which allocate clusters and tensor memory per launch, and any
// group beyond the cap, which falls back to relaunching); a group with no resident
// request tells its kernel to quit.  Results are bitwise those of the relaunch mode.
#include "../../include/cho.h"
#include "cho_internal.h"
#include "ctx.h"
#include "persist.h"

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cstdlib>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <list>
#include <map>
#include <mutex>
#include <thread>
#include <tuple>
#include <unordered_map>
#include <vector>

namespace cho {

// Called by the serving buffers before they allocate.  An allocation of device or
// page-locked host memory serialises all streams; a resident serving kernel waits for the
// serving thread's next doorbell, so on the serving thread every resident kernel is first
// told to quit (it finishes any generation in flight without the host, then leaves) and is
// started again at its group's next generation.
void serving_before_alloc();

static double now_s()
{
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

namespace {

enum ReqState { RQ_QUEUED = 0, RQ_RESIDENT = 1, RQ_DONE = 2 };

struct Req {
    uint64_t ticket = 0;
    cho_system_impl* sys = nullptr;
    int64_t set = 0;
    int32_t s = 0, prec = 0, priority = 0;
    double h = 0.0;
    int64_t n_steps = 0, remaining = 0;
    std::vector<double> x0, v0, x, v;
    ReqState state = RQ_QUEUED;
    cho_status status = CHO_OK;
    bool cancel = false;
    double t_submit = 0, t_admit = 0, t_done = 0;
    int32_t slot = -1;
    size_t bytes = 0;
    void* block = nullptr;
    size_t readback_off = 0;
    bool reading_back = false;
    int64_t weight = 0;             // occupancy weight (ServeEngine::footprint)
    bool active = false;            // advanced by the next launch of its group
    std::list<Req*>::iterator res_it;   // place in its class's resident list
};

bool fp64_prec(int32_t prec) { return prec == CHO_FP64; }

// Bytes of the resident state block of a request.
size_t state_bytes(const cho_system_impl* sys, int32_t prec)
{
    const size_t n = sys->path == PATH_SMALL ? (size_t)sys->S : (size_t)sys->s;
    return fp64_prec(prec) ? 2 * n * sizeof(double) : 4 * n * sizeof(float);
}

size_t round_class(size_t b)
{
    size_t c = 256;
    while (c < b) c <<= 1;
    return c;
}

// Device blocks of power-of-two size classes carved from 64 MiB arenas.  Arenas come from
// stream-ordered allocation on the pool's own stream (no wait for other streams, where
// resident serving kernels may be waiting for the serving thread) and are freed at release.
class BlockPool {
public:
    BlockPool() = default;
    BlockPool(const BlockPool&) = delete;
    BlockPool& operator=(const BlockPool&) = delete;
    ~BlockPool() { release(); }
    void* get(size_t cls, cudaError_t* err)
    {
        *err = cudaSuccess;
        auto& fl = free_[cls];
        if (!fl.empty()) {
            void* p = fl.back();
            fl.pop_back();
            return p;
        }
        if (!st_) {
            *err = cudaStreamCreateWithFlags(&st_, cudaStreamNonBlocking);
            if (*err != cudaSuccess) {
                st_ = nullptr;
                return nullptr;
            }
        }
        const size_t arena = std::max<size_t>((size_t)64 << 20, cls);
        void* base = nullptr;
        serving_before_alloc();
        *err = cudaMallocAsync(&base, arena, st_);
        if (*err == cudaSuccess) *err = cudaStreamSynchronize(st_);
        if (*err != cudaSuccess) return nullptr;
        arenas_.push_back(base);
        for (size_t off = cls; off + cls <= arena; off += cls) fl.push_back((char*)base + off);
        return base;
    }
    void put(size_t cls, void* p) { free_[cls].push_back(p); }
    void release()
    {
        for (void* a : arenas_) cudaFreeAsync(a, st_);
        if (st_) {
            cudaStreamSynchronize(st_);
            cudaStreamDestroy(st_);
        }
        st_ = nullptr;
        arenas_.clear();
        free_.clear();
    }

private:
    std::map<size_t, std::vector<void*>> free_;
    std::vector<void*> arenas_;
    cudaStream_t st_ = nullptr;
};

// Growth of the serving loop's buffers never frees: cudaFree and cudaFreeHost wait for
// the whole device, and a resident (persistent) kernel is waiting for the serving thread's
// next doorbell, so a free there would stall both until the kernel's wait runs out.  A
// buffer that grows (at least doubling) keeps its old allocations until release().
template <class T>
class PinnedBuf {
public:
    PinnedBuf() = default;
    PinnedBuf(const PinnedBuf&) = delete;
    PinnedBuf& operator=(const PinnedBuf&) = delete;
    ~PinnedBuf() { release(); }
    T* get(size_t n, cudaError_t* err)
    {
        *err = cudaSuccess;
        if (n <= cap_) return p_;
        size_t want = std::max(std::max(n, (size_t)4096), 2 * cap_);
        T* p = nullptr;
        serving_before_alloc();
        *err = cudaHostAlloc((void**)&p, want * sizeof(T), cudaHostAllocDefault);
        if (*err != cudaSuccess) return nullptr;
        if (p_) old_.push_back(p_);
        p_ = p;
        cap_ = want;
        return p_;
    }
    T* ptr() const { return p_; }
    void release()
    {
        if (p_) cudaFreeHost(p_);
        for (T* o : old_) cudaFreeHost(o);
        old_.clear();
        p_ = nullptr;
        cap_ = 0;
    }

private:
    T* p_ = nullptr;
    size_t cap_ = 0;
    std::vector<T*> old_;
};

template <class T>
class DevBuf {
public:
    DevBuf() = default;
    DevBuf(const DevBuf&) = delete;
    DevBuf& operator=(const DevBuf&) = delete;
    ~DevBuf() { release(); }
    T* get(size_t n, cudaError_t* err)
    {
        *err = cudaSuccess;
        if (n <= cap_) return p_;
        size_t want = std::max(std::max(n, (size_t)1024), 2 * cap_);
        T* p = nullptr;
        serving_before_alloc();
        *err = cudaMalloc((void**)&p, want * sizeof(T));
        if (*err != cudaSuccess) return nullptr;
        if (p_) old_.push_back(p_);            // kept until release(): see PinnedBuf
        p_ = p;
        cap_ = want;
        return p_;
    }
    T* ptr() const { return p_; }
    size_t cap() const { return cap_; }
    void release()
    {
        if (p_) cudaFree(p_);
        for (T* o : old_) cudaFree(o);
        old_.clear();
        p_ = nullptr;
        cap_ = 0;
    }

private:
    T* p_ = nullptr;
    size_t cap_ = 0;
    std::vector<T*> old_;
};

// Pinned host memory mapped into the device (host and device pointer).
template <class T>
class Mapped {
public:
    Mapped() = default;
    Mapped(const Mapped&) = delete;
    Mapped& operator=(const Mapped&) = delete;
    ~Mapped() { release(); }
    cudaError_t alloc(size_t n)
    {
        release();
        serving_before_alloc();
        cudaError_t e = cudaHostAlloc((void**)&h, std::max<size_t>(n, 1) * sizeof(T), cudaHostAllocMapped);
        if (e != cudaSuccess) {
            h = nullptr;
            return e;
        }
        std::memset((void*)h, 0, std::max<size_t>(n, 1) * sizeof(T));
        e = cudaHostGetDevicePointer((void**)&d, (void*)h, 0);
        n_ = n;
        return e;
    }
    void release()
    {
        if (h) cudaFreeHost((void*)h);
        h = nullptr;
        d = nullptr;
        n_ = 0;
    }
    size_t size() const { return n_; }
    T* h = nullptr;
    T* d = nullptr;

private:
    size_t n_ = 0;
};

// Lanes per instance of rk4_small at padded size S (rows_per_lane of rk4_small.cu).
int small_lanes(int S) { return S <= 4 ? 1 : (S == 8 ? 4 : S); }

}  // namespace

// Requests that run in one kernel launch: same kernel family, size class and
// precision (and, for dense systems, the same shared B).
using GroupKey = std::tuple<int, int, int, cho_system_impl*>;

struct Group {
    GroupKey key;
    cudaStream_t st = nullptr;
    cudaEvent_t ev = nullptr;
    bool busy = false;
    int64_t chunk = 0;
    cudaEvent_t k0 = nullptr, k1 = nullptr;   // around the kernel of a launch (chunk tuning only)
    int64_t max_run = 0;            // most steps a member runs in the launch in flight
    std::vector<Req*> members;      // resident
    std::vector<Req*> incoming;     // admitted, state not uploaded yet
    std::vector<Req*> launched;     // advanced by the launch in flight
    PinnedBuf<int32_t> h_ids;
    DevBuf<int32_t> d_ids;
    DevBuf<int32_t> d_st;
    PinnedBuf<int32_t> h_st;
    PinnedBuf<unsigned char> h_up;
    PinnedBuf<unsigned char> h_down;
    PinnedBuf<SlotDesc> h_desc;
    // persistent mode
    bool persist = false;           // the group can be served by a resident kernel
    bool running = false;           // its kernel takes doorbells (launched, not told to quit)
    bool resident = false;          // its kernel may still be on `st` (until synchronised)
    bool inflight = false;          // a generation rung on the resident kernel, not yet retired
    int grid = 0;
    int64_t footprint = 0;          // registers the resident kernel holds
    uint64_t gen = 0;               // last generation rung
    unsigned long long ring_tail = 0;
    double t_ring = 0.0;
    double t_last = 0.0;            // last start or completed generation of the resident kernel
    cudaStream_t cst = nullptr;     // state copies while the kernel holds `st`
    Mapped<PersistCtl> ctl;
    Mapped<int32_t> ids;
    Mapped<int32_t> ring;
};

struct ServeEngine {
    cho_ctx* ctx = nullptr;
    std::thread worker;
    std::mutex mu;
    std::condition_variable cv;
    bool stop = false;
    bool failed = false;
    std::deque<Req*> queue[3];
    std::list<Req*> resident_by_class[3];   // resident requests, admission order per class
    bool active_dirty = false;              // the active set needs choosing again
    int64_t active_cap = 0;                 // occupancy weight of the active set; <= 0: no cap
    std::map<std::tuple<int, int, int, bool>, int64_t> weight_cache;
    std::unordered_map<uint64_t, Req*> reqs;
    int64_t n_resident = 0;
    uint64_t next_ticket = 1;
    int64_t resident_bytes = 0;
    int64_t completed = 0;
    int64_t n_queued = 0;
    // chunk-boundary traffic: state bytes each chunk reads and writes back (the resident
    // block of every advanced request, once each way) and the DOF-steps it advances
    int64_t traffic_bytes = 0, traffic_dof_steps = 0;
    // device side (worker thread only)
    int32_t slot_cap = 0;
    std::vector<int32_t> free_slots;
    DevBuf<SlotDesc> d_slots;       // slot table, allocated once (kernels in flight read it)
    DevBuf<int32_t> d_status;
    BlockPool pool;
    std::map<GroupKey, Group*> groups;
    // persistent mode: slot table and status words in mapped host memory
    bool persistent = false;
    bool withhold_doorbell = false;  // test hook (CHO_TEST_WITHHOLD_DOORBELL=1)
    Mapped<SlotDesc> m_slots;
    Mapped<int32_t> m_status;
    int64_t persist_regs = 0, persist_cap = 0;     // registers held by resident kernels, and the cap
    int64_t persist_ctas = 0, persist_cta_cap = 0; // their CTAs, and the cap (half the SMs)
    SlotDesc* slots_d() { return persistent ? m_slots.d : d_slots.ptr(); }
    int32_t* status_d() { return persistent ? m_status.d : d_status.ptr(); }

    void run();
    Group* group_for(Req* r, cudaError_t* e);
    cudaError_t upload(Group* g, cudaStream_t copy_st);
    cudaError_t launch(Group* g);
    cudaError_t launch_persist(Group* g, bool* fell_back);
    void retire(Group* g);          // caller holds mu
    void retire_persist(Group* g);  // caller holds mu
    void timed_out(Group* g);       // caller holds mu
    void quit(Group* g);
    void park();                    // quit every resident kernel (before an allocation)
    void fail_all(cho_status st_code);
    void release(Req* r);           // caller holds mu
    void choose_active();           // caller holds mu
    int64_t footprint(const Req* r);  // caller holds mu
    // finished requests in the order they finished (cho_poll_any); caller holds mu
    std::deque<uint64_t> done_fifo;
    void mark_done(Req* r)
    {
        r->state = RQ_DONE;
        done_fifo.push_back(r->ticket);
        // tickets collected by cho_poll stay in the queue until cho_poll_any passes them;
        // drop them when they dominate, so a client that only calls cho_poll holds no memory
        if (done_fifo.size() > 2 * reqs.size() + 4096) {
            std::deque<uint64_t> keep;
            for (uint64_t t : done_fifo)
                if (reqs.count(t)) keep.push_back(t);
            done_fifo.swap(keep);
        }
    }
};

void ServeEngine::fail_all(cho_status code)
{
    // caller holds mu
    failed = true;
    const double t = now_s();
    for (auto& kv : groups) {
        Group* g = kv.second;
        quit(g);
        for (auto* list : {&g->members, &g->incoming})
            for (Req* r : *list) {
                mark_done(r);
                r->status = code;
                r->t_done = t;
            }
        g->members.clear();
        g->incoming.clear();
        g->launched.clear();
    }
    for (auto& q : queue) {
        for (Req* r : q) {
            mark_done(r);
            r->status = code;
            r->t_done = t;
        }
        q.clear();
    }
    for (auto& l : resident_by_class) l.clear();
    n_queued = 0;
    n_resident = 0;
    cv.notify_all();
}

// Occupancy weight of a request: its share of the device, D / (instances its slot kernel
// holds resident at once), with D = SMs x 2048 the unit of the active-set cap; so a cap
// of 100 % takes about one wave of every kernel family together (a dense s = 512 request
// on an 8-CTA cluster weighs as much as eight full SMs, a 2-DOF lane next to nothing).
// Asked once per kernel shape.
int64_t ServeEngine::footprint(const Req* r)
{
    const cho_system_impl* sys = r->sys;
    const bool f64 = fp64_prec(r->prec);
    const bool tc = r->prec == CHO_DENSE_BF16X3 || r->prec == CHO_DENSE_BF16X5 || r->prec == CHO_DENSE_BF16X6;
    const int size = sys->path == PATH_SMALL ? sys->S : (sys->path == PATH_CHAIN ? sys->s : sys->s_pad);
    const auto key = std::make_tuple((int)sys->path, size, (int)r->prec, sys->path == PATH_DENSE && sys->n_sys != 1);
    auto it = weight_cache.find(key);
    if (it != weight_cache.end()) return it->second;
    int resident = 0;
    if (sys->path == PATH_SMALL) {
        resident = small_slot_resident(sys->S, f64);
    } else if (sys->path == PATH_CHAIN) {
        resident = chain_slot_resident(sys->s, f64);
    } else {
        DenseSys ds{sys->s, sys->s_pad, sys->d_B64, sys->d_B32, sys->d_Bbf, sys->s_tc, sys->d_err, 0,
                    sys->n_sys != 1 ? 1 : 0};
        resident = tc ? dense_tc_slot_resident(ds, r->prec) : dense_slot_resident(ds, f64);
    }
    const int64_t D = (int64_t)ctx->sm_count * 2048;
    const int64_t w = resident > 0 ? std::max<int64_t>(1, (D + resident - 1) / resident) : D;
    weight_cache[key] = w;
    return w;
}

// The active set: resident requests in priority order (class 0 first, admission order
// within a class), each taken while the set's weight stays within the cap (the first one
// always), so that under load the higher classes run as on a device of their own and the
// lower ones wait at their chunk boundaries.
void ServeEngine::choose_active()
{
    int64_t used = 0;
    for (auto& l : resident_by_class)
        for (Req* r : l) {
            r->active = active_cap <= 0 || used == 0 || used + r->weight <= active_cap;
            if (r->active) used += r->weight;
        }
    active_dirty = false;
}

void ServeEngine::release(Req* r)
{
    if (r->slot >= 0) resident_by_class[r->priority].erase(r->res_it);
    active_dirty = true;
    resident_bytes -= (int64_t)r->bytes;
    if (r->block) pool.put(r->bytes, r->block);
    r->block = nullptr;
    if (r->slot >= 0) free_slots.push_back(r->slot);
    r->slot = -1;
    --n_resident;
    ++completed;
}

static int64_t group_chunk(const cho_ctx* ctx) { return ctx->cfg.chunk_steps; }

Group* ServeEngine::group_for(Req* r, cudaError_t* e)
{
    *e = cudaSuccess;
    const cho_system_impl* sys = r->sys;
    // chains of more than 2048 masses need wider CTAs than the persistent chain kernel's
    const bool wide_chain = sys->path == PATH_CHAIN && sys->s > 2048;
    const int size = sys->path == PATH_SMALL
                         ? sys->S
                         : (sys->path == PATH_CHAIN ? (wide_chain ? 16 : chain_dofs_per_thread(sys->s)) : sys->s);
    GroupKey key(sys->path, size, r->prec, sys->path == PATH_DENSE ? r->sys : nullptr);
    auto it = groups.find(key);
    if (it != groups.end()) return it->second;
    Group* g = new (std::nothrow) Group();
    if (!g) {
        *e = cudaErrorMemoryAllocation;
        return nullptr;
    }
    g->key = key;
    g->chunk = group_chunk(ctx);
    *e = cudaStreamCreateWithFlags(&g->st, cudaStreamNonBlocking);
    if (*e == cudaSuccess) *e = cudaEventCreateWithFlags(&g->ev, cudaEventDisableTiming);
    if (*e == cudaSuccess && ctx->cfg.chunk_us > 0) {
        *e = cudaEventCreate(&g->k0);
        if (*e == cudaSuccess) *e = cudaEventCreate(&g->k1);
    }
    g->persist = persistent && (sys->path == PATH_SMALL || (sys->path == PATH_CHAIN && !wide_chain));
    if (*e == cudaSuccess && g->persist) {
        *e = cudaStreamCreateWithFlags(&g->cst, cudaStreamNonBlocking);
        if (*e == cudaSuccess) *e = g->ctl.alloc(1);
        if (*e == cudaSuccess) *e = g->ids.alloc((size_t)slot_cap);
        if (*e == cudaSuccess) *e = g->ring.alloc((size_t)slot_cap);
    }
    if (*e != cudaSuccess) {
        if (g->st) cudaStreamDestroy(g->st);
        if (g->cst) cudaStreamDestroy(g->cst);
        delete g;
        return nullptr;
    }
    groups[key] = g;
    return g;
}

// Upload the group's new requests (state blocks on copy_st, table entries and status
// words: mapped host memory in persistent mode, else copies on copy_st) and make them
// members.
cudaError_t ServeEngine::upload(Group* g, cudaStream_t copy_st)
{
    cudaError_t e = cudaSuccess;
    size_t up_bytes = 0;
    for (Req* r : g->incoming) up_bytes += r->bytes;
    unsigned char* up = g->h_up.get(std::max<size_t>(up_bytes, 1), &e);
    SlotDesc* hd = e == cudaSuccess ? g->h_desc.get(std::max<size_t>(g->incoming.size(), 1), &e) : nullptr;
    size_t off = 0;
    for (size_t k = 0; k < g->incoming.size() && e == cudaSuccess; ++k) {
        Req* r = g->incoming[k];
        const cho_system_impl* sys = r->sys;
        const int n = sys->path == PATH_SMALL ? sys->S : sys->s;
        const int s = sys->s;
        unsigned char* dst = up + off;
        if (fp64_prec(r->prec)) {
            double* d = (double*)dst;
            for (int i = 0; i < n; ++i) {
                d[i] = i < s ? r->x0[i] : 0.0;
                d[n + i] = i < s ? r->v0[i] : 0.0;
            }
        } else {
            // FP32 small systems and chains hold the scaled velocity u = (h/6) v
            const bool scaled = sys->path == PATH_SMALL || sys->path == PATH_CHAIN;
            float* f = (float*)dst;
            for (int i = 0; i < n; ++i) {
                const double xd = i < s ? r->x0[i] : 0.0, v0 = i < s ? r->v0[i] : 0.0;
                const double vd = scaled ? scaled_velocity(v0, r->h) : v0;
                f[i] = (float)xd;
                f[n + i] = (float)vd;
                f[2 * n + i] = (float)(xd - (double)f[i]);          // compensation: x + e
                f[3 * n + i] = (float)(vd - (double)f[n + i]);
            }
        }
        e = cudaMemcpyAsync(r->block, dst, state_bytes(sys, r->prec), cudaMemcpyHostToDevice, copy_st);
        off += r->bytes;
        SlotDesc sd{};
        if (sys->path == PATH_SMALL) {
            const size_t SS = (size_t)sys->S * sys->S;
            sd.coef = fp64_prec(r->prec) ? (const void*)(sys->d_B64 + r->set * SS)
                                          : (const void*)(sys->d_B32 + r->set * 2 * SS);
        } else if (sys->path == PATH_CHAIN) {
            sd.coef = fp64_prec(r->prec) ? (const void*)(sys->d_B64 + r->set * 2 * s)
                                          : (const void*)(sys->d_B32 + r->set * 4 * s);
        } else if (sys->n_sys != 1 && (fp64_prec(r->prec) || r->prec == CHO_FP32_KAHAN)) {
            const size_t n = (size_t)sys->s_pad * sys->s_pad;   // dense, one (M, K) per set: its B^T
            sd.coef = fp64_prec(r->prec) ? (const void*)(sys->d_B64 + r->set * n)
                                          : (const void*)(sys->d_B32 + r->set * 2 * n);
        }
        sd.state = r->block;
        sd.h = r->h;
        sd.remaining = r->n_steps;
        sd.s = s;
        hd[k] = sd;
        if (persistent) {
            // the slot is free: no kernel reads its entry until the host hands it out
            m_slots.h[r->slot] = sd;
            ((volatile int32_t*)m_status.h)[r->slot] = 0;
        } else {
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(d_slots.ptr() + r->slot, &hd[k], sizeof(SlotDesc), cudaMemcpyHostToDevice, copy_st);
            if (e == cudaSuccess) e = cudaMemsetAsync(d_status.ptr() + r->slot, 0, sizeof(int32_t), copy_st);
        }
    }
    if (e != cudaSuccess) return e;
    g->members.insert(g->members.end(), g->incoming.begin(), g->incoming.end());
    g->incoming.clear();
    return cudaSuccess;
}

// Upload the group's new requests, advance every member by one chunk (one launch), and
// queue the read-back of status words and of the states that finish in this chunk.
cudaError_t ServeEngine::launch(Group* g)
{
    const int64_t L = g->chunk;
    cudaError_t e = upload(g, g->st);
    if (e != cudaSuccess) return e;
    g->launched.clear();
    for (Req* r : g->members)
        if (r->active) g->launched.push_back(r);
    const size_t n_ids = g->launched.size();
    if (n_ids == 0) return cudaSuccess;
    int32_t* ids = g->h_ids.get(n_ids, &e);
    if (e == cudaSuccess) g->d_ids.get(n_ids, &e);
    if (e == cudaSuccess) g->d_st.get(n_ids, &e);
    int32_t* hst = e == cudaSuccess ? g->h_st.get(n_ids, &e) : nullptr;
    if (e != cudaSuccess) return e;
    for (size_t i = 0; i < n_ids; ++i) ids[i] = g->launched[i]->slot;
    e = cudaMemcpyAsync(g->d_ids.ptr(), ids, n_ids * sizeof(int32_t), cudaMemcpyHostToDevice, g->st);
    if (e != cudaSuccess) return e;
    const int path = std::get<0>(g->key), size = std::get<1>(g->key), prec = std::get<2>(g->key);
    const bool f64 = fp64_prec(prec);
    SlotIO io{(int64_t)n_ids, g->d_ids.ptr(), slots_d(), status_d(), L};
    g->max_run = 0;
    for (Req* r : g->launched) g->max_run = std::max(g->max_run, std::min(L, r->remaining));
    if (g->k0) e = cudaEventRecord(g->k0, g->st);
    if (e != cudaSuccess) return e;
    if (path == PATH_SMALL) {
        e = launch_rk4_small_slots(size, io, f64, g->st);
    } else if (path == PATH_CHAIN) {
        int s_max = 0;
        for (Req* r : g->launched) s_max = std::max(s_max, r->sys->s);
        e = launch_rk4_chain_slots(s_max, io, f64, g->st);
    } else {
        cho_system_impl* sys = std::get<3>(g->key);
        DenseSys ds{sys->s, sys->s_pad, sys->d_B64, sys->d_B32, sys->d_Bbf, sys->s_tc, sys->d_err, 0,
                    sys->n_sys != 1 ? 1 : 0};
        if (prec == CHO_DENSE_BF16X3 || prec == CHO_DENSE_BF16X5 || prec == CHO_DENSE_BF16X6)
            e = launch_rk4_dense_tc_slots(ds, io, prec, g->st);
        else
            e = launch_rk4_dense_slots(ds, io, f64, g->st);
    }
    if (e == cudaSuccess && g->k1) e = cudaEventRecord(g->k1, g->st);
    if (e == cudaSuccess) e = launch_gather_status(g->d_ids.ptr(), status_d(), g->d_st.ptr(), (int64_t)n_ids, g->st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(hst, g->d_st.ptr(), n_ids * sizeof(int32_t), cudaMemcpyDeviceToHost, g->st);
    size_t down_bytes = 0;
    for (Req* r : g->launched)
        if (r->remaining <= L) down_bytes += r->bytes;
    unsigned char* down = e == cudaSuccess ? g->h_down.get(std::max<size_t>(down_bytes, 1), &e) : nullptr;
    size_t doff = 0;
    for (Req* r : g->launched) {
        if (e != cudaSuccess) break;
        r->reading_back = r->remaining <= L;
        if (r->reading_back) {
            r->readback_off = doff;
            e = cudaMemcpyAsync(down + doff, r->block, state_bytes(r->sys, r->prec), cudaMemcpyDeviceToHost, g->st);
            doff += r->bytes;
        }
    }
    if (e == cudaSuccess) e = cudaEventRecord(g->ev, g->st);
    if (e == cudaSuccess) g->busy = true;
    return e;
}

// The group's launch has finished: book the steps, hand out finished results,
// return their slots and memory.  Caller holds mu.
void ServeEngine::retire(Group* g)
{
    const double t = now_s();
    const int64_t L = g->chunk;
    const int32_t* hst = g->h_st.ptr();
    const unsigned char* down = g->h_down.ptr();
    for (size_t i = 0; i < g->launched.size(); ++i) {
        Req* r = g->launched[i];
        const int64_t ran = std::min<int64_t>(L, r->remaining);
        traffic_bytes += 2 * (int64_t)state_bytes(r->sys, r->prec);
        traffic_dof_steps += (int64_t)r->sys->s * ran;
        r->remaining -= ran;
        const int32_t code = hst ? hst[i] : 0;
        if (code != 0) {
            r->status = (cho_status)code;
            mark_done(r);
            r->t_done = t;
        } else if (r->remaining == 0 && r->reading_back) {
            const cho_system_impl* sys = r->sys;
            const int n = sys->path == PATH_SMALL ? sys->S : sys->s;
            const int s = sys->s;
            r->x.resize(s);
            r->v.resize(s);
            const unsigned char* src = down + r->readback_off;
            if (fp64_prec(r->prec)) {
                const double* d = (const double*)src;
                for (int k = 0; k < s; ++k) {
                    r->x[k] = d[k];
                    r->v[k] = d[n + k];
                }
            } else {
                const float* f = (const float*)src;
                const bool scaled = sys->path == PATH_SMALL || sys->path == PATH_CHAIN;
                for (int k = 0; k < s; ++k) {
                    r->x[k] = (double)f[k] + (double)f[2 * n + k];
                    const double u = (double)f[n + k] + (double)f[3 * n + k];
                    r->v[k] = scaled ? unscaled_velocity(u, r->h) : u;
                }
            }
            r->status = CHO_OK;
            mark_done(r);
            r->t_done = t;
        } else if (r->cancel) {
            r->status = CHO_ECANCELLED;
            mark_done(r);
            r->t_done = t;
        }
    }
    auto it = std::remove_if(g->members.begin(), g->members.end(), [&](Req* r) {
        if (r->state != RQ_DONE) return false;
        release(r);
        return true;
    });
    g->members.erase(it, g->members.end());
    g->launched.clear();
    g->busy = false;
    // chunk-length tuning: from the kernel's device time per step in this launch, the
    // chunk that would take chunk_us, moving at most a factor of two per launch
    float ms = 0.f;
    if (g->k0 && g->max_run > 0 && cudaEventElapsedTime(&ms, g->k0, g->k1) == cudaSuccess && ms > 0.f) {
        const double per_step_us = 1e3 * (double)ms / (double)g->max_run;
        double target = (double)ctx->cfg.chunk_us / per_step_us;
        target = std::min(std::max(target, 0.5 * (double)L), 2.0 * (double)L);
        g->chunk = std::min<int64_t>(std::max<int64_t>(std::llround(target), 16), (int64_t)1 << 22);
    }
}

// Persistent mode: upload the new members (which may allocate, and so park every resident
// kernel: first), start the group's resident kernel if it takes no doorbells (within the
// caps; *fell_back when it does not fit, and the caller relaunches instead), write the
// generation's slot ids and ring the doorbell.
cudaError_t ServeEngine::launch_persist(Group* g, bool* fell_back)
{
    *fell_back = false;
    const int path = std::get<0>(g->key), size = std::get<1>(g->key), prec = std::get<2>(g->key);
    const bool f64 = fp64_prec(prec);
    size_t n = 0;
    for (auto* list : {&g->members, &g->incoming})
        for (Req* r : *list) n += r->active ? 1 : 0;
    if (n == 0) return cudaSuccess;
    cudaError_t e = upload(g, g->cst);
    if (e == cudaSuccess) e = cudaStreamSynchronize(g->cst);     // blocks on the device before the doorbell
    if (e != cudaSuccess) return e;
    const int threads = path == PATH_SMALL ? kSmallThreads : chain_persist_threads(size);
    const int64_t per_cta = (int64_t)threads * 128;              // registers a CTA may hold
    const int64_t want = path == PATH_SMALL
                             ? ((int64_t)n * small_lanes(size) + kSmallThreads - 1) / kSmallThreads
                             : (int64_t)n;
    const int64_t most = path == PATH_SMALL ? 2 * (int64_t)ctx->sm_count : (int64_t)ctx->sm_count;
    // each resident CTA sits on its own SM at most, so capping their number at half the SMs
    // leaves the other half whole for the launched kernels (a 512-thread dense CTA needs a
    // full register file)
    auto room = [&]() {
        return std::min((persist_cap - persist_regs) / per_cta, persist_cta_cap - persist_ctas);
    };
    // a kernel idle for half its doorbell wait may leave before the next ring: replace it;
    // so is one whose group has outgrown its grid by a quarter when a larger grid fits
    if (g->running && (g->ctl.h->status == CHO_ETIMEOUT || now_s() - g->t_last > 0.5)) quit(g);
    if (g->running && want > g->grid) {
        const int64_t bigger = std::min(std::min(want, most), room() + g->grid);
        if (4 * bigger >= 5 * (int64_t)g->grid) quit(g);
    }
    if (!g->running) {
        const int64_t grid = std::min(std::min(want, most), room());
        if (grid < 1) {
            *fell_back = true;
            return cudaSuccess;
        }
        // the group's previous kernel (told to quit, or timed out) has left its stream
        if (g->resident) {
            e = cudaStreamSynchronize(g->st);
            if (e != cudaSuccess) return e;
            g->resident = false;
        }
        PersistCtl* c = g->ctl.h;
        std::memset((void*)c, 0, sizeof(PersistCtl));
        g->gen = 0;
        g->ring_tail = 0;
        g->grid = (int)grid;
        g->footprint = grid * per_cta;
        std::atomic_thread_fence(std::memory_order_seq_cst);
        PersistIO pio{g->ctl.d, g->ids.d, m_slots.d, m_status.d, g->ring.d, (uint32_t)g->ring.size()};
        e = path == PATH_SMALL ? launch_rk4_small_persist(size, pio, f64, g->grid, g->st)
                               : launch_rk4_chain_persist(size, pio, f64, g->grid, g->st);
        if (e != cudaSuccess) return e;
        g->running = true;
        g->resident = true;
        g->t_last = now_s();
        persist_regs += g->footprint;
        persist_ctas += g->grid;
    }
    g->launched.clear();
    for (Req* r : g->members)
        if (r->active) g->launched.push_back(r);
    const int64_t L = g->chunk;
    g->max_run = 0;
    for (size_t i = 0; i < g->launched.size(); ++i) {
        Req* r = g->launched[i];
        g->ids.h[i] = r->slot;
        g->max_run = std::max(g->max_run, std::min(L, r->remaining));
    }
    PersistCtl* c = g->ctl.h;
    ((volatile int64_t*)&c->n_items)[0] = (int64_t)g->launched.size();
    ((volatile int64_t*)&c->chunk)[0] = L;
    std::atomic_thread_fence(std::memory_order_seq_cst);        // payload before the doorbell
    ++g->gen;
    if (!withhold_doorbell) ((volatile uint64_t*)&c->doorbell)[0] = g->gen;
    std::atomic_thread_fence(std::memory_order_seq_cst);
    g->t_ring = now_s();
    g->busy = true;
    g->inflight = true;
    return cudaSuccess;
}

// Tell the group's resident kernel to leave: it finishes a generation in flight, then
// leaves at its next doorbell wait.  Its CTAs no longer count against the caps.
void ServeEngine::quit(Group* g)
{
    if (!g->running) return;
    std::atomic_thread_fence(std::memory_order_seq_cst);
    ((volatile int32_t*)&g->ctl.h->quit)[0] = 1;
    std::atomic_thread_fence(std::memory_order_seq_cst);
    g->running = false;
    persist_regs -= g->footprint;
    persist_ctas -= g->grid;
    g->footprint = 0;
}

void ServeEngine::park()
{
    if (withhold_doorbell) return;   // test hook: the withheld kernels are to time out by themselves
    for (auto& kv : groups) quit(kv.second);
}

// The resident kernel's doorbell wait ran out (it has left): every request of the
// generation in flight ends with CHO_ETIMEOUT.  Caller holds mu.
void ServeEngine::timed_out(Group* g)
{
    const double t = now_s();
    for (Req* r : g->launched) {
        r->status = CHO_ETIMEOUT;
        mark_done(r);
        r->t_done = t;
    }
    auto it = std::remove_if(g->members.begin(), g->members.end(), [&](Req* r) {
        if (r->state != RQ_DONE) return false;
        release(r);
        return true;
    });
    g->members.erase(it, g->members.end());
    g->launched.clear();
    g->busy = false;
    g->inflight = false;
    quit(g);                        // releases the caps if the kernel still counted
}

// A generation of the resident kernel is complete: read the completion ring, book the
// steps, read back finished states (copy stream) and hand them out.  Caller holds mu.
void ServeEngine::retire_persist(Group* g)
{
    const double t = now_s();
    const int64_t L = g->chunk;
    PersistCtl* c = g->ctl.h;
    std::atomic_thread_fence(std::memory_order_seq_cst);
    const unsigned long long head = ((volatile unsigned long long*)&c->ring_head)[0];
    std::vector<char> finished(g->launched.size(), 0);
    {
        std::unordered_map<int32_t, size_t> pos;
        for (size_t i = 0; i < g->launched.size(); ++i) pos[g->launched[i]->slot] = i;
        for (unsigned long long k = g->ring_tail; k < head; ++k) {
            const int32_t slot = ((volatile int32_t*)g->ring.h)[k % g->ring.size()];
            auto it = pos.find(slot);
            if (it != pos.end()) finished[it->second] = 1;
        }
        g->ring_tail = head;
    }
    cudaError_t e = cudaSuccess;
    size_t down_bytes = 0;
    for (size_t i = 0; i < g->launched.size(); ++i)
        if (finished[i]) down_bytes += g->launched[i]->bytes;
    unsigned char* down = g->h_down.get(std::max<size_t>(down_bytes, 1), &e);
    size_t doff = 0;
    for (size_t i = 0; i < g->launched.size() && e == cudaSuccess; ++i) {
        Req* r = g->launched[i];
        const int64_t ran = std::min<int64_t>(L, r->remaining);
        traffic_bytes += 2 * (int64_t)state_bytes(r->sys, r->prec);
        traffic_dof_steps += (int64_t)r->sys->s * ran;
        r->remaining -= ran;
        const int32_t code = ((volatile int32_t*)m_status.h)[r->slot];
        r->reading_back = finished[i] && code == 0 && r->remaining == 0;
        if (r->reading_back) {
            r->readback_off = doff;
            e = cudaMemcpyAsync(down + doff, r->block, state_bytes(r->sys, r->prec), cudaMemcpyDeviceToHost, g->cst);
            doff += r->bytes;
        }
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(g->cst);
    if (e != cudaSuccess) {
        fail_all(CHO_ECUDA);
        return;
    }
    for (Req* r : g->launched) {
        const int32_t code = ((volatile int32_t*)m_status.h)[r->slot];
        if (code != 0) {
            r->status = (cho_status)code;
            mark_done(r);
            r->t_done = t;
        } else if (r->remaining == 0 && r->reading_back) {
            const cho_system_impl* sys = r->sys;
            const int nn = sys->path == PATH_SMALL ? sys->S : sys->s;
            const int sz = sys->s;
            r->x.resize(sz);
            r->v.resize(sz);
            const unsigned char* src = down + r->readback_off;
            if (fp64_prec(r->prec)) {
                const double* d = (const double*)src;
                for (int k = 0; k < sz; ++k) {
                    r->x[k] = d[k];
                    r->v[k] = d[nn + k];
                }
            } else {
                const float* f = (const float*)src;
                for (int k = 0; k < sz; ++k) {           // small and chain families: scaled velocity
                    r->x[k] = (double)f[k] + (double)f[2 * nn + k];
                    r->v[k] = unscaled_velocity((double)f[nn + k] + (double)f[3 * nn + k], r->h);
                }
            }
            r->status = CHO_OK;
            mark_done(r);
            r->t_done = t;
        } else if (r->remaining == 0) {
            r->status = CHO_EINTERNAL;                   // finished without a completion entry
            mark_done(r);
            r->t_done = t;
        } else if (r->cancel) {
            r->status = CHO_ECANCELLED;
            mark_done(r);
            r->t_done = t;
        }
    }
    auto it = std::remove_if(g->members.begin(), g->members.end(), [&](Req* r) {
        if (r->state != RQ_DONE) return false;
        release(r);
        return true;
    });
    g->members.erase(it, g->members.end());
    g->launched.clear();
    g->busy = false;
    g->inflight = false;
    g->t_last = t;
    // chunk-length tuning from the generation's wall time (doorbell to completion)
    if (ctx->cfg.chunk_us > 0 && g->max_run > 0) {
        const double per_step_us = 1e6 * (t - g->t_ring) / (double)g->max_run;
        if (per_step_us > 0.0) {
            double target = (double)ctx->cfg.chunk_us / per_step_us;
            target = std::min(std::max(target, 0.5 * (double)L), 2.0 * (double)L);
            g->chunk = std::min<int64_t>(std::max<int64_t>(std::llround(target), 16), (int64_t)1 << 22);
        }
    }
}

namespace {
thread_local ServeEngine* t_serving = nullptr;   // the engine whose serving thread this is
}

void serving_before_alloc()
{
    if (t_serving) t_serving->park();
}

void ServeEngine::run()
{
    DeviceGuard dg(ctx->device);
    t_serving = this;
    std::vector<Group*> to_launch;
    while (true) {
        bool progressed = false;
        to_launch.clear();
        {
            std::unique_lock<std::mutex> lk(mu);
            while (!stop && n_resident == 0 && n_queued == 0) cv.wait(lk);
            if (stop) break;
            // finished launches
            for (auto& kv : groups) {
                Group* g = kv.second;
                if (!g->inflight) continue;
                // persistent: the generation is complete when every CTA has counted it
                volatile PersistCtl* c = g->ctl.h;
                if (c->status == CHO_ETIMEOUT) {
                    timed_out(g);
                    progressed = true;
                } else if (now_s() - g->t_ring > 10.0 && c->done < (unsigned long long)g->grid * g->gen) {
                    // host-side deadline: the kernel is told to leave and its stream drained
                    // before the generation's blocks are given back
                    quit(g);
                    if (cudaStreamSynchronize(g->st) != cudaSuccess) {
                        fail_all(CHO_ECUDA);
                        return;
                    }
                    g->resident = false;
                    if (c->done >= (unsigned long long)g->grid * g->gen) retire_persist(g);
                    else timed_out(g);
                    if (failed) return;
                    progressed = true;
                } else if (c->done >= (unsigned long long)g->grid * g->gen) {
                    retire_persist(g);
                    if (failed) return;
                    progressed = true;
                }
            }
            for (auto& kv : groups) {
                Group* g = kv.second;
                if (!g->busy || g->inflight) continue;
                const cudaError_t q = cudaEventQuery(g->ev);
                if (q == cudaErrorNotReady) continue;
                if (q != cudaSuccess) {
                    fail_all(CHO_ECUDA);
                    return;
                }
                retire(g);
                progressed = true;
            }
            // cancelled requests leave: those not yet on the device (admitted, waiting for their
            // group's next launch, possibly paused) at once, members of idle groups before their
            // next launch
            for (auto& kv : groups) {
                Group* g = kv.second;
                auto cancel = [&](Req* r) {
                    if (!r->cancel) return false;
                    mark_done(r);
                    r->status = CHO_ECANCELLED;
                    r->t_done = now_s();
                    release(r);
                    return true;
                };
                auto in = std::remove_if(g->incoming.begin(), g->incoming.end(), cancel);
                if (in != g->incoming.end()) progressed = true;
                g->incoming.erase(in, g->incoming.end());
                if (g->busy) continue;
                auto it = std::remove_if(g->members.begin(), g->members.end(), cancel);
                if (it != g->members.end()) progressed = true;
                g->members.erase(it, g->members.end());
            }
            // admission: strict fixed priority, FIFO within a class, slots and budget permitting
            const int64_t budget = ctx->cfg.budget_bytes;
            for (int p = 0; p < 3; ++p) {
                bool blocked = false;
                while (!queue[p].empty()) {
                    Req* r = queue[p].front();
                    if (r->cancel) {
                        queue[p].pop_front();
                        --n_queued;
                        mark_done(r);
                        r->status = CHO_ECANCELLED;
                        r->t_done = now_s();
                        ++completed;
                        continue;
                    }
                    if (free_slots.empty() || resident_bytes + (int64_t)r->bytes > budget) {
                        blocked = true;
                        break;
                    }
                    cudaError_t e;
                    Group* g = group_for(r, &e);
                    void* block = g ? pool.get(r->bytes, &e) : nullptr;
                    if (!block) {
                        fail_all(e == cudaErrorMemoryAllocation ? CHO_ENOMEM : CHO_ECUDA);
                        return;
                    }
                    queue[p].pop_front();
                    --n_queued;
                    r->block = block;
                    r->slot = free_slots.back();
                    free_slots.pop_back();
                    resident_bytes += (int64_t)r->bytes;
                    ++n_resident;
                    r->state = RQ_RESIDENT;
                    r->remaining = r->n_steps;
                    r->t_admit = now_s();
                    r->weight = footprint(r);
                    resident_by_class[p].push_back(r);
                    r->res_it = std::prev(resident_by_class[p].end());
                    active_dirty = true;
                    g->incoming.push_back(r);
                    progressed = true;
                }
                if (blocked) break;
            }
            if (active_dirty) choose_active();
            for (auto& kv : groups) {
                Group* g = kv.second;
                if (g->busy) continue;
                bool any = false;
                for (auto* list : {&g->members, &g->incoming})
                    for (Req* r : *list) any = any || r->active;
                if (any) to_launch.push_back(g);
                // a resident kernel with nothing to run leaves its SMs to the others
                else if (g->running) quit(g);
            }
            if (progressed) cv.notify_all();
        }
        // launches outside the lock (only this thread touches the groups' device side)
        for (Group* g : to_launch) {
            cudaError_t e = cudaSuccess;
            bool relaunch = !g->persist;
            if (g->persist) {
                bool fell_back = false;
                e = launch_persist(g, &fell_back);
                relaunch = fell_back;
            }
            if (e == cudaSuccess && relaunch) e = launch(g);
            if (e != cudaSuccess) {
                std::lock_guard<std::mutex> lk(mu);
                fail_all(CHO_ECUDA);
                return;
            }
            progressed = true;
        }
        if (!progressed) std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
}

static ServeEngine* engine(cho_ctx* ctx, cho_status* err)
{
    std::lock_guard<std::mutex> lk(ctx->serve_mu);
    if (ctx->serve) return ctx->serve;
    ServeEngine* en = new (std::nothrow) ServeEngine();
    if (!en) {
        *err = fail(CHO_ENOMEM, "cho_submit: out of host memory");
        return nullptr;
    }
    en->ctx = ctx;
    DeviceGuard g(ctx->device);
    cudaError_t e = cudaSuccess;
    en->slot_cap = ctx->cfg.max_slots;
    en->persistent = ctx->cfg.persistent != 0;
    en->active_cap = ctx->cfg.active_pct > 0 ? (int64_t)ctx->cfg.active_pct * ctx->sm_count * 2048 / 100 : 0;
    if (en->persistent) {
        e = en->m_slots.alloc((size_t)en->slot_cap);
        if (e == cudaSuccess) e = en->m_status.alloc((size_t)en->slot_cap);
        en->persist_cap = (int64_t)(0.6 * (double)ctx->sm_count * 65536.0);
        en->persist_cta_cap = std::max(1, ctx->sm_count / 2);
        const char* hook = std::getenv("CHO_TEST_WITHHOLD_DOORBELL");
        en->withhold_doorbell = hook && hook[0] == '1';
    } else {
        en->d_slots.get((size_t)en->slot_cap, &e);
        if (e == cudaSuccess) en->d_status.get((size_t)en->slot_cap, &e);
    }
    if (e != cudaSuccess) {
        delete en;
        *err = fail(CHO_ENOMEM, "cho_submit: slot table of %d slots: %s", ctx->cfg.max_slots, cudaGetErrorString(e));
        return nullptr;
    }
    for (int32_t i = en->slot_cap - 1; i >= 0; --i) en->free_slots.push_back(i);
    en->worker = std::thread([en] { en->run(); });
    ctx->serve = en;
    return en;
}

void serve_stop(cho_ctx* ctx)
{
    ServeEngine* en = nullptr;
    {
        std::lock_guard<std::mutex> lk(ctx->serve_mu);
        en = ctx->serve;
        ctx->serve = nullptr;
    }
    if (!en) return;
    {
        std::lock_guard<std::mutex> lk(en->mu);
        en->stop = true;
        en->cv.notify_all();
    }
    if (en->worker.joinable()) en->worker.join();
    {
        DeviceGuard g(ctx->device);
        for (auto& kv : en->groups) en->quit(kv.second);
        for (auto& kv : en->groups) {
            Group* gr = kv.second;
            cudaStreamSynchronize(gr->st);
            if (gr->cst) {
                cudaStreamSynchronize(gr->cst);
                cudaStreamDestroy(gr->cst);
            }
            gr->ctl.release();
            gr->ids.release();
            gr->ring.release();
            cudaEventDestroy(gr->ev);
            if (gr->k0) cudaEventDestroy(gr->k0);
            if (gr->k1) cudaEventDestroy(gr->k1);
            cudaStreamDestroy(gr->st);
            delete gr;
        }
        en->groups.clear();
        for (auto& kv : en->reqs) delete kv.second;
        en->reqs.clear();
        en->pool.release();
        en->d_slots.release();
        en->d_status.release();
        en->m_slots.release();
        en->m_status.release();
    }
    delete en;
}

}  // namespace cho

using namespace cho;

extern "C" cho_status cho_submit(cho_ctx* ctx, const cho_request* rq, uint64_t* ticket)
{
    clear_error();
    if (!ctx || !rq || !ticket || !rq->system) return fail(CHO_EINVAL, "cho_submit: NULL argument");
    cho_system_impl* sys = rq->system;
    if (sys->ctx != ctx) return fail(CHO_EINVAL, "cho_submit: system belongs to another context");
    if (rq->sys_index < 0 || rq->sys_index >= sys->n_sys) return fail(CHO_EINVAL, "cho_submit: sys_index out of range");
    if (!rq->x0 || !rq->v0) return fail(CHO_EINVAL, "cho_submit: x0/v0 required");
    if (rq->n_steps < 0) return fail(CHO_EINVAL, "cho_submit: n_steps < 0");
    if (rq->priority < 0 || rq->priority > 2) return fail(CHO_EINVAL, "cho_submit: priority must be 0, 1 or 2");
    if (sys->damped() || sys->forced())
        return fail(CHO_EINVAL, "cho_submit: damped or forced systems run through cho_integrate_batch");
    const bool dense_simt = rq->prec == CHO_DENSE_FP32_SIMT && sys->kind == CHO_DENSE;
    const bool bf16 = rq->prec == CHO_DENSE_BF16X3 || rq->prec == CHO_DENSE_BF16X5 || rq->prec == CHO_DENSE_BF16X6;
    if (bf16 && (sys->path != PATH_DENSE || sys->s_tc == 0 || (rq->prec == CHO_DENSE_BF16X6 && sys->s_tc > 128)))
        return fail(CHO_EINVAL, "cho_submit: BF16 modes need a shared dense system with 32 < s <= 256 (x6: s <= 128)");
    if (rq->prec != CHO_FP64 && rq->prec != CHO_FP32_KAHAN && !dense_simt && !bf16)
        return fail(CHO_EINVAL, "cho_submit: unknown or unsupported precision %d", rq->prec);
    if (!(rq->h > 0.0) || !std::isfinite(rq->h)) return fail(CHO_EINVAL, "cho_submit: h must be finite and > 0");
    const double w = sys->omegas[(size_t)rq->sys_index];
    if (w * rq->h > 2.0 * std::sqrt(2.0))
        return fail(CHO_EUNSTABLE, "cho_submit: omega_max*h = %g > 2 sqrt 2", w * rq->h);
    for (int i = 0; i < sys->s; ++i)
        if (!std::isfinite(rq->x0[i]) || !std::isfinite(rq->v0[i]))
            return fail(CHO_ENONFINITE, "cho_submit: non-finite initial state");
    const int32_t prec = dense_simt ? CHO_FP32_KAHAN : rq->prec;
    const size_t bytes = round_class(state_bytes(sys, prec));
    if ((int64_t)bytes > ctx->cfg.budget_bytes)
        return fail(CHO_EBUDGET, "cho_submit: %zu bytes of state exceed the budget", bytes);
    cho_status err = CHO_OK;
    ServeEngine* en = engine(ctx, &err);
    if (!en) return err;
    Req* r = new (std::nothrow) Req();
    if (!r) return fail(CHO_ENOMEM, "cho_submit: out of host memory");
    r->sys = sys;
    r->set = rq->sys_index;
    r->s = sys->s;
    r->prec = prec;
    r->priority = rq->priority;
    r->h = rq->h;
    r->n_steps = rq->n_steps;
    r->x0.assign(rq->x0, rq->x0 + sys->s);
    r->v0.assign(rq->v0, rq->v0 + sys->s);
    r->bytes = bytes;
    r->t_submit = now_s();
    {
        std::lock_guard<std::mutex> lk(en->mu);
        if (en->failed) {
            delete r;
            return fail(CHO_ECUDA, "cho_submit: the serving loop stopped after a CUDA error");
        }
        r->ticket = en->next_ticket++;
        en->reqs[r->ticket] = r;
        en->queue[r->priority].push_back(r);
        ++en->n_queued;
        en->cv.notify_all();
    }
    *ticket = r->ticket;
    return CHO_OK;
}

extern "C" cho_status cho_poll(cho_ctx* ctx, uint64_t ticket, cho_result* out)
{
    clear_error();
    if (!ctx) return fail(CHO_EINVAL, "cho_poll: NULL ctx");
    ServeEngine* en;
    {
        std::lock_guard<std::mutex> lk(ctx->serve_mu);
        en = ctx->serve;
    }
    if (!en) return fail(CHO_ENOTFOUND, "cho_poll: unknown ticket %llu", (unsigned long long)ticket);
    std::lock_guard<std::mutex> lk(en->mu);
    auto it = en->reqs.find(ticket);
    if (it == en->reqs.end()) return fail(CHO_ENOTFOUND, "cho_poll: unknown ticket %llu", (unsigned long long)ticket);
    Req* r = it->second;
    if (r->state != RQ_DONE) return CHO_PENDING;
    const cho_status st = r->status;
    if (out) {
        if (st == CHO_OK) {
            if (out->x) std::memcpy(out->x, r->x.data(), sizeof(double) * r->x.size());
            if (out->v) std::memcpy(out->v, r->v.data(), sizeof(double) * r->v.size());
        }
        out->t_submit = r->t_submit;
        out->t_admit = r->t_admit;
        out->t_done = r->t_done;
    }
    en->reqs.erase(it);
    delete r;
    if (st != CHO_OK) return fail(st, "cho_poll: request %llu ended with status %d", (unsigned long long)ticket, (int)st);
    return CHO_OK;
}

extern "C" cho_status cho_poll_any(cho_ctx* ctx, uint64_t* ticket, cho_result* out)
{
    clear_error();
    if (!ctx || !ticket) return fail(CHO_EINVAL, "cho_poll_any: NULL argument");
    ServeEngine* en;
    {
        std::lock_guard<std::mutex> lk(ctx->serve_mu);
        en = ctx->serve;
    }
    if (!en) return CHO_PENDING;
    std::lock_guard<std::mutex> lk(en->mu);
    while (!en->done_fifo.empty()) {
        const uint64_t t = en->done_fifo.front();
        en->done_fifo.pop_front();
        auto it = en->reqs.find(t);
        if (it == en->reqs.end()) continue;            // already collected by cho_poll
        Req* r = it->second;
        const cho_status st = r->status;
        if (out) {
            if (st == CHO_OK) {
                if (out->x) std::memcpy(out->x, r->x.data(), sizeof(double) * r->x.size());
                if (out->v) std::memcpy(out->v, r->v.data(), sizeof(double) * r->v.size());
            }
            out->t_submit = r->t_submit;
            out->t_admit = r->t_admit;
            out->t_done = r->t_done;
        }
        *ticket = t;
        en->reqs.erase(it);
        delete r;
        return st;
    }
    return CHO_PENDING;
}

extern "C" cho_status cho_cancel(cho_ctx* ctx, uint64_t ticket)
{
    clear_error();
    if (!ctx) return fail(CHO_EINVAL, "cho_cancel: NULL ctx");
    ServeEngine* en;
    {
        std::lock_guard<std::mutex> lk(ctx->serve_mu);
        en = ctx->serve;
    }
    if (!en) return fail(CHO_ENOTFOUND, "cho_cancel: unknown ticket");
    std::lock_guard<std::mutex> lk(en->mu);
    auto it = en->reqs.find(ticket);
    if (it == en->reqs.end()) return fail(CHO_ENOTFOUND, "cho_cancel: unknown ticket");
    it->second->cancel = true;
    en->cv.notify_all();
    return CHO_OK;
}

extern "C" cho_status cho_serve_stats(cho_ctx* ctx, int64_t* queued, int64_t* resident, int64_t* completed,
                                      int64_t* resident_bytes)
{
    clear_error();
    if (!ctx) return fail(CHO_EINVAL, "cho_serve_stats: NULL ctx");
    ServeEngine* en;
    {
        std::lock_guard<std::mutex> lk(ctx->serve_mu);
        en = ctx->serve;
    }
    int64_t q = 0, r = 0, c = 0, b = 0;
    if (en) {
        std::lock_guard<std::mutex> lk(en->mu);
        q = en->n_queued;
        r = en->n_resident;
        c = en->completed;
        b = en->resident_bytes;
    }
    if (queued) *queued = q;
    if (resident) *resident = r;
    if (completed) *completed = c;
    if (resident_bytes) *resident_bytes = b;
    return CHO_OK;
}

extern "C" cho_status cho_serve_traffic(cho_ctx* ctx, int64_t* state_bytes_moved, int64_t* dof_steps)
{
    clear_error();
    if (!ctx) return fail(CHO_EINVAL, "cho_serve_traffic: NULL ctx");
    ServeEngine* en;
    {
        std::lock_guard<std::mutex> lk(ctx->serve_mu);
        en = ctx->serve;
    }
    int64_t b = 0, d = 0;
    if (en) {
        std::lock_guard<std::mutex> lk(en->mu);
        b = en->traffic_bytes;
        d = en->traffic_dof_steps;
    }
    if (state_bytes_moved) *state_bytes_moved = b;
    if (dof_steps) *dof_steps = d;
    return CHO_OK;
}
