// serve.cpp -- continuous batching of single-instance integration requests.
//
// cho_submit queues a request (one instance of one parameter set); a worker
// thread owned by the context runs the request loop:
//   1. admission: requests leave three fixed-priority FIFO queues (class 0
//      first; strict priority, no ageing) while a slot is free and their state
//      fits the device-memory budget; each admitted request gets a slot in the
//      device slot table and a resident state block in its kernel's precision;
//   2. one chunk: every resident request advances min(chunk, remaining) RK4 steps;
//      requests are grouped by kernel family (rk4_small by padded size,
//      rk4_chain by threads per CTA, rk4_dense by shared system) and each group
//      is one kernel launch over a list of slot ids;
//   3. retirement: finished requests are read back, converted to FP64 and
//      handed to cho_poll; their slots and memory go back to the pool, so the
//      next chunk admits more work while the others keep running.
// The state stays on the device between chunks in the kernel's own precision
// (x, v and the Kahan compensations), so a request's result does not depend on
// how its horizon is cut into chunks or on which requests share its launches.
// This follows the paper's use of the model as a fixed-priority real-time
// workload (Section 5) with the GPU as the executor.
#include "../../include/cho.h"
#include "cho_internal.h"
#include "ctx.h"

#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <tuple>
#include <unordered_map>
#include <vector>

namespace cho {

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

// Device blocks of power-of-two size classes carved from 64 MiB arenas.
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
        const size_t arena = std::max<size_t>((size_t)64 << 20, cls);
        void* base = nullptr;
        *err = cudaMalloc(&base, arena);
        if (*err != cudaSuccess) return nullptr;
        arenas_.push_back(base);
        for (size_t off = cls; off + cls <= arena; off += cls) fl.push_back((char*)base + off);
        return base;
    }
    void put(size_t cls, void* p) { free_[cls].push_back(p); }
    void release()
    {
        for (void* a : arenas_) cudaFree(a);
        arenas_.clear();
        free_.clear();
    }

private:
    std::map<size_t, std::vector<void*>> free_;
    std::vector<void*> arenas_;
};

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
        release();
        size_t want = std::max(n, (size_t)4096);
        *err = cudaHostAlloc((void**)&p_, want * sizeof(T), cudaHostAllocDefault);
        if (*err != cudaSuccess) {
            p_ = nullptr;
            return nullptr;
        }
        cap_ = want;
        return p_;
    }
    void release()
    {
        if (p_) cudaFreeHost(p_);
        p_ = nullptr;
        cap_ = 0;
    }

private:
    T* p_ = nullptr;
    size_t cap_ = 0;
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
        release();
        size_t want = std::max(n, (size_t)1024);
        *err = cudaMalloc((void**)&p_, want * sizeof(T));
        if (*err != cudaSuccess) {
            p_ = nullptr;
            return nullptr;
        }
        cap_ = want;
        return p_;
    }
    T* ptr() const { return p_; }
    size_t cap() const { return cap_; }
    void swap(DevBuf& o)
    {
        std::swap(p_, o.p_);
        std::swap(cap_, o.cap_);
    }
    void release()
    {
        if (p_) cudaFree(p_);
        p_ = nullptr;
        cap_ = 0;
    }

private:
    T* p_ = nullptr;
    size_t cap_ = 0;
};

}  // namespace

struct ServeEngine {
    cho_ctx* ctx = nullptr;
    std::thread worker;
    std::mutex mu;
    std::condition_variable cv;
    bool stop = false;
    bool failed = false;
    std::deque<Req*> queue[3];
    std::unordered_map<uint64_t, Req*> reqs;
    std::vector<Req*> resident;
    uint64_t next_ticket = 1;
    int64_t resident_bytes = 0;
    int64_t completed = 0;
    int64_t n_queued = 0;
    // device side (worker thread only)
    cudaStream_t st = nullptr;
    int32_t slot_cap = 0;
    std::vector<int32_t> free_slots;
    DevBuf<SlotDesc> d_slots;
    DevBuf<int32_t> d_status;
    DevBuf<int32_t> d_ids;
    PinnedBuf<SlotDesc> h_slot_stage;
    PinnedBuf<int32_t> h_ids;
    PinnedBuf<int32_t> h_status;
    PinnedBuf<unsigned char> h_up;
    PinnedBuf<unsigned char> h_down;
    BlockPool pool;

    void run();
    bool grow_slots(int32_t need, cudaError_t* err);
    void fail_all(cho_status st_code);
};

bool ServeEngine::grow_slots(int32_t need, cudaError_t* err)
{
    *err = cudaSuccess;
    if (need <= slot_cap) return true;
    int32_t cap = std::max<int32_t>(1024, slot_cap);
    while (cap < need) cap *= 2;
    cap = std::min<int32_t>(cap, std::max<int32_t>(ctx->cfg.max_slots, need));
    // preserve the descriptors of resident slots
    SlotDesc* old = d_slots.ptr();
    int32_t* olds = d_status.ptr();
    DevBuf<SlotDesc> ns;
    DevBuf<int32_t> nst;
    if (!ns.get((size_t)cap, err) || !nst.get((size_t)cap, err)) return false;
    if (old && slot_cap > 0) {
        *err = cudaMemcpyAsync(ns.ptr(), old, sizeof(SlotDesc) * slot_cap, cudaMemcpyDeviceToDevice, st);
        if (*err == cudaSuccess)
            *err = cudaMemcpyAsync(nst.ptr(), olds, sizeof(int32_t) * slot_cap, cudaMemcpyDeviceToDevice, st);
        if (*err == cudaSuccess) *err = cudaStreamSynchronize(st);
        if (*err != cudaSuccess) return false;
    }
    d_slots.swap(ns);     // the old buffers are freed when ns/nst leave scope
    d_status.swap(nst);
    for (int32_t i = cap - 1; i >= slot_cap; --i) free_slots.push_back(i);
    slot_cap = cap;
    return true;
}

void ServeEngine::fail_all(cho_status code)
{
    // caller holds mu
    failed = true;
    for (Req* r : resident) {
        r->state = RQ_DONE;
        r->status = code;
        r->t_done = now_s();
    }
    resident.clear();
    for (auto& q : queue) {
        for (Req* r : q) {
            r->state = RQ_DONE;
            r->status = code;
            r->t_done = now_s();
        }
        q.clear();
    }
    n_queued = 0;
    cv.notify_all();
}

void ServeEngine::run()
{
    DeviceGuard g(ctx->device);
    const int64_t L = ctx->cfg.chunk_steps;
    std::vector<Req*> admitted, batch, finished;
    // group key: (path, size, fp64, system for dense)
    using Key = std::tuple<int, int, int, cho_system_impl*>;
    std::map<Key, std::vector<int32_t>> groups;
    while (true) {
        cudaError_t e = cudaSuccess;
        admitted.clear();
        {
            std::unique_lock<std::mutex> lk(mu);
            while (!stop && resident.empty() && n_queued == 0) cv.wait(lk);
            if (stop) break;
            // drop cancelled requests
            for (Req* r : resident)
                if (r->cancel) {
                    r->state = RQ_DONE;
                    r->status = CHO_ECANCELLED;
                    r->t_done = now_s();
                }
            auto it = std::remove_if(resident.begin(), resident.end(), [&](Req* r) {
                if (r->state != RQ_DONE) return false;
                resident_bytes -= (int64_t)r->bytes;
                pool.put(r->bytes, r->block);
                free_slots.push_back(r->slot);
                ++completed;
                return true;
            });
            resident.erase(it, resident.end());
            // admission: strict fixed priority, FIFO within a class
            const int64_t budget = ctx->cfg.budget_bytes;
            for (int p = 0; p < 3; ++p) {
                bool blocked = false;
                while (!queue[p].empty()) {
                    Req* r = queue[p].front();
                    if (r->cancel) {
                        queue[p].pop_front();
                        --n_queued;
                        r->state = RQ_DONE;
                        r->status = CHO_ECANCELLED;
                        r->t_done = now_s();
                        ++completed;
                        continue;
                    }
                    if ((int64_t)resident.size() + (int64_t)admitted.size() >= ctx->cfg.max_slots ||
                        resident_bytes + (int64_t)r->bytes > budget) {
                        blocked = true;
                        break;
                    }
                    queue[p].pop_front();
                    --n_queued;
                    resident_bytes += (int64_t)r->bytes;
                    admitted.push_back(r);
                }
                if (blocked) break;
            }
            cv.notify_all();
        }
        // ---- device work of this chunk (no lock held) ----
        size_t up_bytes = 0;
        for (Req* r : admitted) up_bytes += r->bytes;
        unsigned char* up = h_up.get(std::max<size_t>(up_bytes, 1), &e);
        if (e == cudaSuccess) grow_slots((int32_t)(resident.size() + admitted.size()), &e);
        SlotDesc* hs = e == cudaSuccess ? h_slot_stage.get(std::max<size_t>(admitted.size(), 1), &e) : nullptr;
        size_t off = 0;
        for (size_t k = 0; k < admitted.size() && e == cudaSuccess; ++k) {
            Req* r = admitted[k];
            r->block = pool.get(r->bytes, &e);
            if (!r->block) break;
            r->slot = free_slots.back();
            free_slots.pop_back();
            // initial state in kernel precision and layout
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
                float* f = (float*)dst;
                for (int i = 0; i < n; ++i) {
                    const double xd = i < s ? r->x0[i] : 0.0, vd = i < s ? r->v0[i] : 0.0;
                    f[i] = (float)xd;
                    f[n + i] = (float)vd;
                    f[2 * n + i] = (float)(xd - (double)f[i]);          // compensation: x + e
                    f[3 * n + i] = (float)(vd - (double)f[n + i]);
                }
            }
            e = cudaMemcpyAsync(r->block, dst, state_bytes(sys, r->prec), cudaMemcpyHostToDevice, st);
            off += r->bytes;
            if (e != cudaSuccess) break;
            SlotDesc sd{};
            if (sys->path == PATH_SMALL) {
                const size_t SS = (size_t)sys->S * sys->S;
                sd.coef = fp64_prec(r->prec) ? (const void*)(sys->d_B64 + r->set * SS)
                                              : (const void*)(sys->d_B32 + r->set * 2 * SS);
            } else if (sys->path == PATH_CHAIN) {
                sd.coef = fp64_prec(r->prec) ? (const void*)(sys->d_B64 + r->set * 2 * s)
                                              : (const void*)(sys->d_B32 + r->set * 4 * s);
            } else {
                sd.coef = nullptr;
            }
            sd.state = r->block;
            sd.h = r->h;
            sd.remaining = r->n_steps;
            sd.s = s;
            hs[k] = sd;
            e = cudaMemcpyAsync(d_slots.ptr() + r->slot, &hs[k], sizeof(SlotDesc), cudaMemcpyHostToDevice, st);
            if (e == cudaSuccess) e = cudaMemsetAsync(d_status.ptr() + r->slot, 0, sizeof(int32_t), st);
            if (e != cudaSuccess) break;
        }
        {
            std::lock_guard<std::mutex> lk(mu);
            const double t = now_s();
            for (Req* r : admitted) {
                r->state = RQ_RESIDENT;
                r->remaining = r->n_steps;
                r->t_admit = t;
                resident.push_back(r);
            }
            if (e != cudaSuccess) {
                fail_all(CHO_ECUDA);
                return;
            }
            batch.assign(resident.begin(), resident.end());
        }
        // launches: one per kernel group
        groups.clear();
        int32_t max_slot = 0;
        for (Req* r : batch) {
            const cho_system_impl* sys = r->sys;
            int size = sys->path == PATH_SMALL ? sys->S : (sys->path == PATH_CHAIN ? chain_dofs_per_thread(sys->s) : sys->s_pad);
            cho_system_impl* key_sys = sys->path == PATH_DENSE ? r->sys : nullptr;
            groups[Key(sys->path, size, fp64_prec(r->prec) ? 1 : 0, key_sys)].push_back(r->slot);
            max_slot = std::max(max_slot, r->slot + 1);
        }
        size_t n_ids = 0;
        for (auto& kv : groups) n_ids += kv.second.size();
        int32_t* ids = e == cudaSuccess ? h_ids.get(std::max<size_t>(n_ids, 1), &e) : nullptr;
        if (e == cudaSuccess) d_ids.get(std::max<size_t>(n_ids, 1), &e);
        if (e == cudaSuccess && n_ids > 0) {
            size_t o = 0;
            for (auto& kv : groups) {
                std::memcpy(ids + o, kv.second.data(), kv.second.size() * sizeof(int32_t));
                o += kv.second.size();
            }
            e = cudaMemcpyAsync(d_ids.ptr(), ids, n_ids * sizeof(int32_t), cudaMemcpyHostToDevice, st);
            o = 0;
            for (auto& kv : groups) {
                if (e != cudaSuccess) break;
                const int path = std::get<0>(kv.first), size = std::get<1>(kv.first);
                const bool f64 = std::get<2>(kv.first) != 0;
                SlotIO io{(int64_t)kv.second.size(), d_ids.ptr() + o, d_slots.ptr(), d_status.ptr(), L};
                if (path == PATH_SMALL) {
                    e = launch_rk4_small_slots(size, io, f64, st);
                } else if (path == PATH_CHAIN) {
                    int s_max = 0;
                    for (Req* r : batch)
                        if (r->sys->path == PATH_CHAIN && chain_dofs_per_thread(r->sys->s) == size)
                            s_max = std::max(s_max, r->sys->s);
                    e = launch_rk4_chain_slots(s_max, io, f64, st);
                } else {
                    cho_system_impl* sys = std::get<3>(kv.first);
                    DenseSys ds{sys->s, sys->s_pad, sys->d_B64, sys->d_B32, sys->d_Bbf, sys->s_tc, sys->d_err};
                    e = launch_rk4_dense_slots(ds, io, f64, st);
                }
                o += kv.second.size();
            }
        }
        // read back: per-slot status, and the state of requests that finish in this chunk
        int32_t* hst = nullptr;
        finished.clear();
        if (e == cudaSuccess && max_slot > 0) {
            hst = h_status.get((size_t)max_slot, &e);
            if (hst) e = cudaMemcpyAsync(hst, d_status.ptr(), sizeof(int32_t) * max_slot, cudaMemcpyDeviceToHost, st);
        }
        size_t down_bytes = 0;
        for (Req* r : batch)
            if (r->remaining <= L) down_bytes += r->bytes;
        unsigned char* down = e == cudaSuccess ? h_down.get(std::max<size_t>(down_bytes, 1), &e) : nullptr;
        size_t doff = 0;
        for (Req* r : batch) {
            if (e != cudaSuccess) break;
            if (r->remaining <= L) {
                r->readback_off = doff;
                r->reading_back = true;
                e = cudaMemcpyAsync(down + doff, r->block, state_bytes(r->sys, r->prec), cudaMemcpyDeviceToHost, st);
                doff += r->bytes;
                finished.push_back(r);
            }
        }
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        // ---- retire ----
        {
            std::lock_guard<std::mutex> lk(mu);
            if (e != cudaSuccess) {
                fail_all(CHO_ECUDA);
                return;
            }
            const double t = now_s();
            for (Req* r : batch) {
                r->remaining -= std::min<int64_t>(L, r->remaining);
                const bool bad = hst && hst[r->slot] != 0;
                if (r->remaining == 0 || bad) {
                    if (bad) {
                        r->status = CHO_ENONFINITE;
                    } else {
                        const cho_system_impl* sys = r->sys;
                        const int n = sys->path == PATH_SMALL ? sys->S : sys->s;
                        const int s = sys->s;
                        r->x.resize(s);
                        r->v.resize(s);
                        const unsigned char* src = down + r->readback_off;
                        if (fp64_prec(r->prec)) {
                            const double* d = (const double*)src;
                            for (int i = 0; i < s; ++i) {
                                r->x[i] = d[i];
                                r->v[i] = d[n + i];
                            }
                        } else {
                            const float* f = (const float*)src;
                            for (int i = 0; i < s; ++i) {
                                r->x[i] = (double)f[i] + (double)f[2 * n + i];
                                r->v[i] = (double)f[n + i] + (double)f[3 * n + i];
                            }
                        }
                        r->status = CHO_OK;
                    }
                    r->state = RQ_DONE;
                    r->t_done = t;
                }
            }
            auto it = std::remove_if(resident.begin(), resident.end(), [&](Req* r) {
                if (r->state != RQ_DONE) return false;
                resident_bytes -= (int64_t)r->bytes;
                pool.put(r->bytes, r->block);
                free_slots.push_back(r->slot);
                ++completed;
                return true;
            });
            resident.erase(it, resident.end());
            cv.notify_all();
        }
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
    cudaError_t e = cudaStreamCreateWithFlags(&en->st, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        delete en;
        *err = fail(CHO_ECUDA, "cho_submit: cudaStreamCreate: %s", cudaGetErrorString(e));
        return nullptr;
    }
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
        if (en->st) {
            cudaStreamSynchronize(en->st);
            cudaStreamDestroy(en->st);
        }
        for (auto& kv : en->reqs) delete kv.second;
        en->reqs.clear();
        en->pool.release();
        en->d_slots.release();
        en->d_status.release();
        en->d_ids.release();
        en->h_slot_stage.release();
        en->h_ids.release();
        en->h_status.release();
        en->h_up.release();
        en->h_down.release();
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
    const bool dense_simt = rq->prec == CHO_DENSE_FP32_SIMT && sys->kind == CHO_DENSE;
    if (rq->prec != CHO_FP64 && rq->prec != CHO_FP32_KAHAN && !dense_simt)
        return fail(CHO_EINVAL, "cho_submit: serving runs CHO_FP64 or CHO_FP32_KAHAN");
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
        r = (int64_t)en->resident.size();
        c = en->completed;
        b = en->resident_bytes;
    }
    if (queued) *queued = q;
    if (resident) *resident = r;
    if (completed) *completed = c;
    if (resident_bytes) *resident_bytes = b;
    return CHO_OK;
}
