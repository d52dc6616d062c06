// tune.cpp -- the autotuner.  For one batch shape (system, instance count,
// precision, step form) several kernels compute the same bits: the FP32 2-DOF
// kernel in its balanced, pair and lane-group forms; the chain kernel with 1, 2,
// 4 or 8 DOFs per thread; FP32 dense instances one per CTA or cluster or on the
// streaming kernel.  cho_autotune runs each on seeded inputs of that shape, keeps
// those whose outputs equal the first one's bit for bit, times them with CUDA
// events and records the fastest in the context's tune table, which
// cho_integrate_batch consults for every later batch of the same shape (the
// instance count by its power of two).  The table can be written to and read from
// a text file.
#include "../../include/cho.h"
#include "cho_internal.h"
#include "ctx.h"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

using namespace cho;

namespace {

struct Candidate {
    int32_t code;
    char name[24];
};

// The first candidate is the kernel the default rules pick for the shape.
std::vector<Candidate> candidates(const cho_system_impl* sys, int64_t n_inst, int32_t prec, int32_t poly_jump)
{
    std::vector<Candidate> c;
    auto add = [&](int32_t code, const char* name) {
        Candidate k{code, {}};
        std::snprintf(k.name, sizeof(k.name), "%s", name);
        c.push_back(k);
    };
    if (sys->path == PATH_SMALL) {
        add(0, "balanced");
        add(3, "pair");
        if (poly_jump == 0) add(2, "lane_group");
    } else if (sys->path == PATH_CHAIN) {
        const int def = chain_dofs_per_thread(sys->s);
        char nm[24];
        std::snprintf(nm, sizeof(nm), "dofs_per_thread_%d", def);
        add(def, nm);
        for (int P : {1, 2, 4, 8}) {
            if (P == def || !chain_dofs_valid(sys->s, P)) continue;
            std::snprintf(nm, sizeof(nm), "dofs_per_thread_%d", P);
            add(P, nm);
        }
    } else if (sys->path == PATH_DENSE) {
        DenseSys ds{sys->s, sys->s_pad, sys->d_B64, sys->d_B32, sys->d_Bbf, sys->s_tc, sys->d_err, 0,
                    sys->n_sys != 1 ? 1 : 0};
        const bool few_ok = dense_few_capable(ds);
        if (few_ok && dense_few_default(ds, n_inst)) {
            add(1, "one_per_cta_or_cluster");
            add(0, "streaming");
        } else {
            add(0, "streaming");
            if (few_ok) add(1, "one_per_cta_or_cluster");
        }
    }
    (void)prec;
    return c;
}

KernelChoice choice_for(const cho_system_impl* sys, int32_t code)
{
    KernelChoice kc;
    if (sys->path == PATH_SMALL) kc.small_variant = code;
    if (sys->path == PATH_CHAIN) kc.chain_dofs = code;
    if (sys->path == PATH_DENSE) kc.dense_few = code;
    return kc;
}

template <class T>
struct DeviceArray {
    T* p = nullptr;
    ~DeviceArray()
    {
        if (p) cudaFree(p);
    }
    cudaError_t alloc(size_t n) { return cudaMalloc(&p, std::max<size_t>(n, 1) * sizeof(T)); }
};

}  // namespace

extern "C" cho_status cho_autotune(cho_ctx* ctx, cho_system sys, int64_t n_inst, int32_t prec, int32_t poly_jump,
                                   cho_tune_result* out)
{
    clear_error();
    if (!ctx || !sys) return fail(CHO_EINVAL, "cho_autotune: NULL ctx or system");
    if (n_inst <= 0 || n_inst > ((int64_t)1 << 31)) return fail(CHO_EINVAL, "cho_autotune: n_inst must be in 1..2^31");
    if (poly_jump < 0) return fail(CHO_EINVAL, "cho_autotune: poly_jump must be >= 0");
    DeviceGuard g(ctx->device);
    if (!g.ok()) return fail(CHO_ECUDA, "cho_autotune: cudaSetDevice failed");
    cho_tune_result res;
    std::memset(&res, 0, sizeof(res));
    TuneKey key;
    std::vector<Candidate> cand;
    if (tune_key(sys, n_inst, prec, poly_jump, &key)) cand = candidates(sys, n_inst, prec, poly_jump);
    if (cand.size() > 8) cand.resize(8);

    // seeded inputs of the shape: x0 in [-1, 1), v0 = 0, h = T_min / 32 of each set
    const int s = sys->s;
    const size_t ns = (size_t)n_inst * s;
    std::vector<double> hx(ns), hh((size_t)n_inst);
    uint64_t st64 = 0x9E3779B97F4A7C15ull;
    for (size_t k = 0; k < ns; ++k) {
        st64 = st64 * 6364136223846793005ull + 1442695040888963407ull;
        hx[k] = (double)(st64 >> 11) * (2.0 / 9007199254740992.0) - 1.0;
    }
    for (int64_t q = 0; q < n_inst; ++q) {
        const size_t set = sys->n_sys != 1 ? (size_t)(q % sys->n_sys) : 0;
        const double w = set < sys->omegas.size() ? sys->omegas[set] : sys->omega_max;
        hh[(size_t)q] = (double)(float)(6.283185307179586 / (w > 0 ? w : 1.0) / 32.0);
    }
    const int64_t n_run = sys->n_sys != 1 ? std::min<int64_t>(n_inst, sys->n_sys) : n_inst;
    if (n_run != n_inst) return fail(CHO_EINVAL, "cho_autotune: a system with one (M, K) per instance has %lld sets",
                                     (long long)sys->n_sys);
    DeviceArray<double> x0, v0, h, xo, vo, xr, vr;
    cudaError_t e = x0.alloc(ns);
    if (e == cudaSuccess) e = v0.alloc(ns);
    if (e == cudaSuccess) e = h.alloc((size_t)n_inst);
    if (e == cudaSuccess) e = xo.alloc(ns);
    if (e == cudaSuccess) e = vo.alloc(ns);
    if (e == cudaSuccess) e = xr.alloc(ns);
    if (e == cudaSuccess) e = vr.alloc(ns);
    if (e != cudaSuccess) return fail(CHO_ENOMEM, "cho_autotune: %s", cudaGetErrorString(e));
    e = cudaMemcpy(x0.p, hx.data(), ns * sizeof(double), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(v0.p, 0, ns * sizeof(double));
    if (e == cudaSuccess) e = cudaMemcpy(h.p, hh.data(), hh.size() * sizeof(double), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return fail(CHO_ECUDA, "cho_autotune: upload: %s", cudaGetErrorString(e));

    cho_batch_desc b;
    std::memset(&b, 0, sizeof(b));
    b.system = sys;
    b.n_inst = n_inst;
    b.prec = prec;
    b.mem = CHO_MEM_DEVICE;
    b.x0 = x0.p;
    b.v0 = v0.p;
    b.h = h.p;
    b.h_per_inst = 1;
    b.poly_jump = poly_jump;
    const int64_t quantum = poly_jump > 0 ? poly_jump : 1;
    b.n_steps = 16 * quantum;
    b.x_out = xo.p;
    b.v_out = vo.p;
    cho_status rc = validate_batch(&b, "cho_autotune", nullptr);
    if (rc != CHO_OK) return rc;
    if (cand.empty()) {                              // one kernel for this shape: nothing to choose
        res.n_variants = 1;
        res.chosen = 0;
        res.code[0] = -1;
        std::snprintf(res.name[0], sizeof(res.name[0]), "default");
        if (out) *out = res;
        return CHO_OK;
    }
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    e = cudaEventCreate(&ev0);
    if (e == cudaSuccess) e = cudaEventCreate(&ev1);
    auto run_once = [&](const KernelChoice& kc, double* us) -> cho_status {
        cudaError_t ee = cudaEventRecord(ev0, nullptr);
        cho_status r = ee == cudaSuccess ? run_device_batch(ctx, &b, nullptr, &kc) : CHO_ECUDA;
        if (r != CHO_OK) return r;
        ee = cudaEventRecord(ev1, nullptr);
        if (ee == cudaSuccess) ee = cudaEventSynchronize(ev1);
        float ms = 0.f;
        if (ee == cudaSuccess) ee = cudaEventElapsedTime(&ms, ev0, ev1);
        if (ee != cudaSuccess) return fail(CHO_ECUDA, "cho_autotune: %s", cudaGetErrorString(ee));
        *us = 1e3 * (double)ms;
        return CHO_OK;
    };
    // calibrate: runs of about 3 ms with the first candidate
    double us = 0.0;
    const KernelChoice first = choice_for(sys, cand[0].code);
    if (e == cudaSuccess) rc = run_once(first, &us);
    if (e == cudaSuccess && rc == CHO_OK) rc = run_once(first, &us);
    if (e == cudaSuccess && rc == CHO_OK) {
        const double per = std::max(us, 1.0) / (double)b.n_steps;
        int64_t n = (int64_t)std::llround(3000.0 / per);
        n = std::max<int64_t>(16, std::min<int64_t>(n, (int64_t)1 << 20));
        b.n_steps = (n + quantum - 1) / quantum * quantum;
    }
    std::vector<double> ref_x, ref_v, got_x(ns), got_v(ns);
    for (size_t k = 0; k < cand.size() && e == cudaSuccess && rc == CHO_OK; ++k) {
        const KernelChoice kc = choice_for(sys, cand[k].code);
        double best = 1e300;
        rc = run_once(kc, &us);                      // warm-up
        for (int rep = 0; rep < 3 && rc == CHO_OK; ++rep) {
            rc = run_once(kc, &us);
            best = std::min(best, us);
        }
        if (rc != CHO_OK) break;
        e = cudaMemcpy(got_x.data(), xo.p, ns * sizeof(double), cudaMemcpyDeviceToHost);
        if (e == cudaSuccess) e = cudaMemcpy(got_v.data(), vo.p, ns * sizeof(double), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) break;
        if (k == 0) {
            ref_x = got_x;
            ref_v = got_v;
        }
        const bool same = std::memcmp(got_x.data(), ref_x.data(), ns * sizeof(double)) == 0 &&
                          std::memcmp(got_v.data(), ref_v.data(), ns * sizeof(double)) == 0;
        res.code[k] = cand[k].code;
        std::snprintf(res.name[k], sizeof(res.name[k]), "%s", cand[k].name);
        res.us_per_step[k] = same ? best / (double)b.n_steps : -1.0;
    }
    if (ev0) cudaEventDestroy(ev0);
    if (ev1) cudaEventDestroy(ev1);
    if (e != cudaSuccess) return fail(CHO_ECUDA, "cho_autotune: %s", cudaGetErrorString(e));
    if (rc != CHO_OK) return rc;
    res.n_variants = (int32_t)cand.size();
    res.sample_steps = b.n_steps;
    // the default kernel (candidate 0) stays unless another is at least 3 % faster, so that
    // timing noise between near-equal kernels does not flip the choice
    res.chosen = 0;
    double best = res.us_per_step[0] * 0.97;
    for (int k = 1; k < res.n_variants; ++k)
        if (res.us_per_step[k] > 0 && res.us_per_step[k] < best) {
            res.chosen = k;
            best = res.us_per_step[k];
        }
    {
        std::lock_guard<std::mutex> lk(ctx->tune_mu);
        ctx->tune[key] = res.code[res.chosen];
    }
    if (out) *out = res;
    return CHO_OK;
}

extern "C" cho_status cho_tune_query(cho_ctx* ctx, cho_system sys, int64_t n_inst, int32_t prec, int32_t poly_jump,
                                     int32_t* code)
{
    clear_error();
    if (!ctx || !sys || !code) return fail(CHO_EINVAL, "cho_tune_query: NULL argument");
    *code = -1;
    TuneKey key;
    if (!tune_key(sys, n_inst, prec, poly_jump, &key)) return CHO_OK;
    std::lock_guard<std::mutex> lk(ctx->tune_mu);
    auto it = ctx->tune.find(key);
    if (it != ctx->tune.end()) *code = it->second;
    return CHO_OK;
}

// File format: a first line "cho-tune 1", then one entry per line, tab separated:
// device name, kernel family, size, precision, per-instance flag, log2 instance
// bucket, variant code.  Entries for other devices are kept in the file but not loaded.
extern "C" cho_status cho_tune_save(cho_ctx* ctx, const char* path)
{
    clear_error();
    if (!ctx || !path) return fail(CHO_EINVAL, "cho_tune_save: NULL argument");
    FILE* f = std::fopen(path, "w");
    if (!f) return fail(CHO_EINVAL, "cho_tune_save: cannot open %s", path);
    std::fprintf(f, "cho-tune 1\n");
    {
        std::lock_guard<std::mutex> lk(ctx->tune_mu);
        for (const auto& kv : ctx->tune)
            std::fprintf(f, "%s\t%d\t%d\t%d\t%d\t%d\t%d\n", ctx->device_name, kv.first[0], kv.first[1], kv.first[2],
                         kv.first[3], kv.first[4], kv.second);
    }
    const bool ok = std::fclose(f) == 0;
    return ok ? CHO_OK : fail(CHO_EINVAL, "cho_tune_save: writing %s failed", path);
}

extern "C" cho_status cho_tune_load(cho_ctx* ctx, const char* path, int32_t* n_loaded)
{
    clear_error();
    if (!ctx || !path) return fail(CHO_EINVAL, "cho_tune_load: NULL argument");
    FILE* f = std::fopen(path, "r");
    if (!f) return fail(CHO_EINVAL, "cho_tune_load: cannot open %s", path);
    char line[512];
    int32_t n = 0;
    bool ok = std::fgets(line, sizeof(line), f) && std::strncmp(line, "cho-tune 1", 10) == 0;
    std::vector<std::pair<TuneKey, int32_t>> entries;
    while (ok && std::fgets(line, sizeof(line), f)) {
        char* tab = std::strchr(line, '\t');
        if (!tab) {
            ok = false;
            break;
        }
        *tab = '\0';
        int v[7];
        if (std::sscanf(tab + 1, "%d %d %d %d %d %d", &v[0], &v[1], &v[2], &v[3], &v[4], &v[5]) != 6) {
            ok = false;
            break;
        }
        if (std::strcmp(line, ctx->device_name) != 0) continue;
        entries.push_back({TuneKey{v[0], v[1], v[2], v[3], v[4]}, v[5]});
    }
    std::fclose(f);
    if (!ok) return fail(CHO_EINVAL, "cho_tune_load: %s is not a tune file", path);
    {
        std::lock_guard<std::mutex> lk(ctx->tune_mu);
        for (const auto& kv : entries) {
            ctx->tune[kv.first] = kv.second;
            ++n;
        }
    }
    if (n_loaded) *n_loaded = n;
    return CHO_OK;
}
