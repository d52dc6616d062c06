// api.cpp -- the C ABI: contexts, system set-up (step a0), batch dispatch.
#include "../../include/cho.h"
#include "cho_internal.h"
#include "ctx.h"
#include "linalg.h"

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

namespace cho {

static thread_local std::string g_last_error;

cho_status fail(cho_status st, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    std::vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return st;
}

void clear_error() { g_last_error.clear(); }

DeviceGuard::DeviceGuard(int dev)
{
    if (cudaGetDevice(&prev_) != cudaSuccess) prev_ = -1;
    ok_ = cudaSetDevice(dev) == cudaSuccess;
}
DeviceGuard::~DeviceGuard()
{
    if (prev_ >= 0) cudaSetDevice(prev_);
}

void* Workspace::get(size_t bytes, cudaError_t* err)
{
    *err = cudaSuccess;
    if (bytes <= cap_) return ptr_;
    if (ptr_) cudaFree(ptr_);
    ptr_ = nullptr;
    cap_ = 0;
    size_t want = std::max(bytes, (size_t)1 << 20);
    *err = cudaMalloc(&ptr_, want);
    if (*err != cudaSuccess) {
        ptr_ = nullptr;
        return nullptr;
    }
    cap_ = want;
    return ptr_;
}
void Workspace::release()
{
    if (ptr_) cudaFree(ptr_);
    ptr_ = nullptr;
    cap_ = 0;
}

template <class T>
static cudaError_t upload(T** dst, const T* src, size_t n)
{
    *dst = nullptr;
    if (n == 0) return cudaSuccess;
    cudaError_t e = cudaMalloc((void**)dst, n * sizeof(T));
    if (e != cudaSuccess) {
        *dst = nullptr;
        return e;
    }
    e = cudaMemcpy(*dst, src, n * sizeof(T), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(*dst);
        *dst = nullptr;
    }
    return e;
}

static void free_system_device(cho_system_impl* s)
{
    for (auto& pb : s->poly) {
        if (pb.d64) cudaFree(pb.d64);
        if (pb.d32) cudaFree(pb.d32);
    }
    s->poly.clear();
    for (void* p : {(void*)s->d_ext64, (void*)s->d_ext32, (void*)s->d_force})
        if (p) cudaFree(p);
    s->d_ext64 = nullptr;
    s->d_ext32 = nullptr;
    s->d_force = nullptr;
    void* ptrs[] = {s->d_B64, s->d_B32, s->d_Bbf, s->d_masses, s->d_springs, s->d_M, s->d_K, s->d_plain, s->d_err};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    s->d_B64 = nullptr;
    s->d_B32 = nullptr;
    s->d_Bbf = nullptr;
    s->d_masses = s->d_springs = s->d_M = s->d_K = s->d_plain = nullptr;
    s->d_err = nullptr;
}

// Tridiagonal B = M^{-1} K of a chain (also eq. 2 at s = 2), FP64 [3][s]: sub, main, super.
static void chain_B(int s, const double* m, const double* C, double* out)
{
    for (int i = 0; i < s; ++i) {
        const double right = i + 1 < s ? C[i + 1] : 0.0;
        out[i] = i > 0 ? -C[i] / m[i] : 0.0;
        out[s + i] = (C[i] + right) / m[i];
        out[2 * s + i] = i + 1 < s ? -right / m[i] : 0.0;
    }
}

static bool all_finite(const double* p, size_t n)
{
    for (size_t i = 0; i < n; ++i)
        if (!std::isfinite(p[i])) return false;
    return true;
}

// Read and clear the device error word of a system (the tensor-core kernel and
// the balanced 2-DOF kernel set it when one of their bounded waits gives up).
// Synchronous; CHO_OK or CHO_ETIMEOUT.
static cho_status take_device_error(cho_system_impl* sys, const char* who)
{
    if (!sys->d_err) return CHO_OK;
    int h = 0;
    cudaError_t e = cudaMemcpy(&h, sys->d_err, sizeof(int), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && h) e = cudaMemset(sys->d_err, 0, sizeof(int));
    if (e != cudaSuccess) return fail(CHO_ECUDA, "%s: reading the device error word: %s", who, cudaGetErrorString(e));
    if (h) return fail(CHO_ETIMEOUT, "%s: a bounded device wait gave up after its time limit; results are invalid", who);
    return CHO_OK;
}


}  // namespace cho

using namespace cho;

// ------------------------------------------------------------------------------
// context
// ------------------------------------------------------------------------------

extern "C" const char* cho_last_error(void) { return g_last_error.c_str(); }

extern "C" cho_status cho_init(cho_ctx** out, int device, const cho_config* cfg)
{
    clear_error();
    if (!out) return fail(CHO_EINVAL, "cho_init: out is NULL");
    int n = 0;
    cudaError_t e = cudaGetDeviceCount(&n);
    if (e != cudaSuccess) return fail(CHO_ECUDA, "cho_init: cudaGetDeviceCount: %s", cudaGetErrorString(e));
    if (device < 0 || device >= n) return fail(CHO_EINVAL, "cho_init: device %d not in [0, %d)", device, n);
    cho_ctx* c = new (std::nothrow) cho_ctx();
    if (!c) return fail(CHO_ENOMEM, "cho_init: out of host memory");
    c->device = device;
    c->cfg.budget_bytes = (int64_t)40 << 30;
    c->cfg.chunk_steps = 1000;
    c->cfg.max_slots = 1 << 20;
    if (cfg) {
        if (cfg->budget_bytes > 0) c->cfg.budget_bytes = cfg->budget_bytes;
        if (cfg->chunk_steps > 0) c->cfg.chunk_steps = cfg->chunk_steps;
        if (cfg->max_slots > 0) c->cfg.max_slots = cfg->max_slots;
        if (cfg->chunk_us > 0) c->cfg.chunk_us = cfg->chunk_us;
        c->cfg.persistent = cfg->persistent != 0 ? 1 : 0;
        c->cfg.active_pct = cfg->active_pct;
    }
    if (c->cfg.active_pct == 0) c->cfg.active_pct = 100;
    {
        DeviceGuard g(device);
        if (!g.ok()) {
            delete c;
            return fail(CHO_ECUDA, "cho_init: cudaSetDevice(%d) failed", device);
        }
        cudaDeviceProp prop;
        e = cudaGetDeviceProperties(&prop, device);
        if (e != cudaSuccess) {
            delete c;
            return fail(CHO_ECUDA, "cho_init: cudaGetDeviceProperties: %s", cudaGetErrorString(e));
        }
        c->sm_count = prop.multiProcessorCount;
        std::snprintf(c->device_name, sizeof(c->device_name), "%s", prop.name);
        c->cc_major = prop.major;
        c->cc_minor = prop.minor;
    }
    *out = c;
    return CHO_OK;
}

extern "C" void cho_shutdown(cho_ctx* ctx)
{
    if (!ctx) return;
    serve_stop(ctx);
    DeviceGuard g(ctx->device);
    std::vector<cho_system_impl*> systems;
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        systems.assign(ctx->systems.begin(), ctx->systems.end());
        ctx->systems.clear();
    }
    for (cho_system_impl* s : systems) {
        free_system_device(s);
        delete s;
    }
    ctx->ws.release();
    ctx->plain_ws.release();
    if (ctx->err_host) cudaFreeHost(ctx->err_host);
    delete ctx;
}

// ------------------------------------------------------------------------------
// systems
// ------------------------------------------------------------------------------

extern "C" cho_status cho_create_system(cho_ctx* ctx, const cho_system_desc* d_in, cho_system* out)
{
    clear_error();
    if (!ctx || !d_in || !out) return fail(CHO_EINVAL, "cho_create_system: NULL argument");
    // a spring system with coupled masses is eq. 1 with a tridiagonal M: assemble M and K
    // (K of the chain: K_ii = C_i + C_{i+1}, K_{i,i+1} = -C_{i+1}) and build a dense system
    cho_system_desc dd = *d_in;
    const cho_system_desc* d = &dd;
    std::vector<double> cM, cK;
    if (d_in->kind != CHO_DENSE && d_in->mass_coupling) {
        const int s = d_in->s;
        if (s < 1 || s > 512) return fail(CHO_EINVAL, "cho_create_system: coupled masses need 1 <= s <= 512");
        if (d_in->n_sys < 1) return fail(CHO_EINVAL, "cho_create_system: n_sys < 1");
        if (!d_in->masses || !d_in->springs) return fail(CHO_EINVAL, "cho_create_system: masses/springs required");
        const size_t ss = (size_t)s * s;
        cM.assign((size_t)d_in->n_sys * ss, 0.0);
        cK.assign((size_t)d_in->n_sys * ss, 0.0);
        for (int64_t p = 0; p < d_in->n_sys; ++p) {
            const double* m = d_in->masses + p * s;
            const double* c = d_in->springs + p * s;
            const double* mu = d_in->mass_coupling + p * s;
            double* M = &cM[(size_t)p * ss];
            double* K = &cK[(size_t)p * ss];
            for (int i = 0; i < s; ++i) {
                if (!std::isfinite(m[i]) || !(m[i] > 0.0) || !std::isfinite(c[i]) || !(c[i] >= 0.0) ||
                    (i + 1 < s && !std::isfinite(mu[i])))
                    return fail(CHO_EINVAL, "cho_create_system: set %lld: masses > 0, springs >= 0 and finite "
                                "couplings required", (long long)p);
                M[(size_t)i * s + i] = m[i];
                K[(size_t)i * s + i] = c[i] + (i + 1 < s ? c[i + 1] : 0.0);
                if (i + 1 < s) {
                    M[(size_t)i * s + i + 1] = M[(size_t)(i + 1) * s + i] = mu[i];
                    K[(size_t)i * s + i + 1] = K[(size_t)(i + 1) * s + i] = -c[i + 1];
                }
            }
        }
        dd.kind = CHO_DENSE;
        dd.masses = dd.springs = nullptr;
        dd.M = cM.data();
        dd.K = cK.data();
    }
    const int s = d->s;
    const int64_t n_sys = d->n_sys;
    if (s < 1 || s > 8192) return fail(CHO_EINVAL, "cho_create_system: s = %d outside [1, 8192]", s);
    if (n_sys < 1) return fail(CHO_EINVAL, "cho_create_system: n_sys = %lld < 1", (long long)n_sys);
    if (d->kind != CHO_TWO_DOF && d->kind != CHO_CHAIN && d->kind != CHO_DENSE)
        return fail(CHO_EINVAL, "cho_create_system: unknown kind %d", d->kind);
    if (d->kind == CHO_TWO_DOF && s != 2) return fail(CHO_EINVAL, "cho_create_system: TWO_DOF needs s == 2");

    cho_system_impl* sys = new (std::nothrow) cho_system_impl();
    if (!sys) return fail(CHO_ENOMEM, "cho_create_system: out of host memory");
    sys->ctx = ctx;
    sys->kind = d->kind;
    sys->s = s;
    sys->n_sys = n_sys;
    sys->omegas.resize((size_t)n_sys);

    const bool springs = d->kind != CHO_DENSE;
    const size_t ss = (size_t)s * s;
    std::vector<double> plain;     // FP64 coefficients per set: [3][s] or [s][s]
    if (springs) {
        if (!d->masses || !d->springs) {
            delete sys;
            return fail(CHO_EINVAL, "cho_create_system: masses/springs required");
        }
        const size_t n = (size_t)n_sys * s;
        for (size_t i = 0; i < n; ++i) {
            if (!std::isfinite(d->masses[i]) || !(d->masses[i] > 0.0)) {
                delete sys;
                return fail(CHO_EINVAL, "cho_create_system: mass %zu is not finite and > 0", i);
            }
            if (!std::isfinite(d->springs[i]) || !(d->springs[i] >= 0.0)) {
                delete sys;
                return fail(CHO_EINVAL, "cho_create_system: spring %zu is not finite and >= 0", i);
            }
        }
        sys->h_masses.assign(d->masses, d->masses + n);
        sys->h_springs.assign(d->springs, d->springs + n);
        plain.resize((size_t)n_sys * 3 * s);
        for (int64_t p = 0; p < n_sys; ++p) {
            chain_B(s, d->masses + p * s, d->springs + p * s, &plain[(size_t)p * 3 * s]);
            sys->omegas[(size_t)p] = linalg::omega_max_chain(s, d->masses + p * s, d->springs + p * s);
        }
    } else {
        if (!d->M || !d->K) {
            delete sys;
            return fail(CHO_EINVAL, "cho_create_system: M/K required");
        }
        if (!all_finite(d->M, (size_t)n_sys * ss) || !all_finite(d->K, (size_t)n_sys * ss)) {
            delete sys;
            return fail(CHO_EINVAL, "cho_create_system: M or K has a non-finite entry");
        }
        plain.resize((size_t)n_sys * ss);
        std::vector<double> L;
        for (int64_t p = 0; p < n_sys; ++p) {
            const double* M = d->M + p * ss;
            const double* K = d->K + p * ss;
            double kmax = 0.0, mmax = 0.0;
            for (size_t i = 0; i < ss; ++i) {
                kmax = std::max(kmax, std::fabs(K[i]));
                mmax = std::max(mmax, std::fabs(M[i]));
            }
            for (int i = 0; i < s; ++i)
                for (int j = 0; j < i; ++j) {
                    if (std::fabs(K[(size_t)i * s + j] - K[(size_t)j * s + i]) > 1e-12 * kmax) {
                        delete sys;
                        return fail(CHO_EINVAL, "cho_create_system: K of set %lld is not symmetric", (long long)p);
                    }
                    if (std::fabs(M[(size_t)i * s + j] - M[(size_t)j * s + i]) > 1e-12 * mmax) {
                        delete sys;
                        return fail(CHO_ENOTSPD, "cho_create_system: M of set %lld is not symmetric", (long long)p);
                    }
                }
            if (!linalg::cholesky(s, M, L)) {
                delete sys;
                return fail(CHO_ENOTSPD, "cho_create_system: M of set %lld is not positive definite", (long long)p);
            }
            linalg::dense_B(s, L, K, &plain[(size_t)p * ss]);
            sys->omegas[(size_t)p] = linalg::omega_max_dense(s, L, K);
        }
        sys->h_M.assign(d->M, d->M + (size_t)n_sys * ss);
        sys->h_K.assign(d->K, d->K + (size_t)n_sys * ss);
    }
    sys->omega_max = *std::max_element(sys->omegas.begin(), sys->omegas.end());

    // kernel family and its coefficient layout
    if (s <= 32) {
        sys->path = PATH_SMALL;
    } else if (springs) {
        sys->path = PATH_CHAIN;
    } else {
        sys->path = PATH_DENSE;     // one shared (M, K), or one per instance (CUDA cores only)
    }

    DeviceGuard g(ctx->device);
    if (!g.ok()) {
        delete sys;
        return fail(CHO_ECUDA, "cho_create_system: cudaSetDevice failed");
    }
    cudaError_t e = cudaSuccess;
    if (sys->path == PATH_SMALL) {
        const int S = small_S(s);
        sys->S = S;
        const size_t SS = (size_t)S * S;
        std::vector<double> B64((size_t)n_sys * SS, 0.0);
        for (int64_t p = 0; p < n_sys; ++p) {
            double* Bp = &B64[(size_t)p * SS];
            if (springs) {
                const double* c = &plain[(size_t)p * 3 * s];
                for (int i = 0; i < s; ++i) {
                    if (i > 0) Bp[(size_t)i * S + i - 1] = c[i];
                    Bp[(size_t)i * S + i] = c[s + i];
                    if (i + 1 < s) Bp[(size_t)i * S + i + 1] = c[2 * s + i];
                }
            } else {
                const double* b = &plain[(size_t)p * ss];
                for (int i = 0; i < s; ++i)
                    for (int j = 0; j < s; ++j) Bp[(size_t)i * S + j] = b[(size_t)i * s + j];
            }
        }
        std::vector<float> B32((size_t)n_sys * 2 * SS);
        for (int64_t p = 0; p < n_sys; ++p)
            for (size_t k = 0; k < SS; ++k)
                split_pair(B64[(size_t)p * SS + k], B32[(size_t)p * 2 * SS + k], B32[(size_t)p * 2 * SS + SS + k]);
        e = upload(&sys->d_B64, B64.data(), B64.size());
        if (e == cudaSuccess) e = upload(&sys->d_B32, B32.data(), B32.size());
        if (e == cudaSuccess) e = cudaMalloc(&sys->d_err, sizeof(int));
        if (e == cudaSuccess) e = cudaMemset(sys->d_err, 0, sizeof(int));
    } else if (sys->path == PATH_CHAIN) {
        // spring form of eq. 2: g_i = C_i / m_i, u_i = C_{i+1} / m_i
        std::vector<double> C64((size_t)n_sys * 2 * s);
        std::vector<float> C32((size_t)n_sys * 4 * s);
        for (int64_t p = 0; p < n_sys; ++p) {
            const double* m = d->masses + p * s;
            const double* C = d->springs + p * s;
            double* c = &C64[(size_t)p * 2 * s];
            for (int i = 0; i < s; ++i) {
                c[i] = C[i] / m[i];
                c[s + i] = i + 1 < s ? C[i + 1] / m[i] : 0.0;
            }
            float* f = &C32[(size_t)p * 4 * s];
            for (int k = 0; k < 2 * s; ++k) split_pair(c[k], f[k], f[2 * s + k]);
        }
        e = upload(&sys->d_B64, C64.data(), C64.size());
        if (e == cudaSuccess) e = upload(&sys->d_B32, C32.data(), C32.size());
    } else {
        e = build_dense_device(sys, plain.data());
        if (n_sys == 1) sys->h_B = plain;
    }
    if (e == cudaSuccess) {
        if (springs) {
            e = upload(&sys->d_masses, sys->h_masses.data(), sys->h_masses.size());
            if (e == cudaSuccess) e = upload(&sys->d_springs, sys->h_springs.data(), sys->h_springs.size());
        } else {
            e = upload(&sys->d_M, sys->h_M.data(), sys->h_M.size());
            if (e == cudaSuccess) e = upload(&sys->d_K, sys->h_K.data(), sys->h_K.size());
        }
    }
    if (e == cudaSuccess) e = upload(&sys->d_plain, plain.data(), plain.size());
    if (e != cudaSuccess) {
        free_system_device(sys);
        delete sys;
        return fail(e == cudaErrorMemoryAllocation ? CHO_ENOMEM : CHO_ECUDA, "cho_create_system: %s",
                    cudaGetErrorString(e));
    }
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        ctx->systems.insert(sys);
    }
    *out = sys;
    return CHO_OK;
}

// Coefficients of the damped / forced chain kernel from the system's masses, springs,
// dashpots and force amplitudes (absent parts as zeros), FP64 and FP32 pairs, per set.
static cho_status build_chain_ext(cho_system_impl* sys, const char* who)
{
    for (void* p : {(void*)sys->d_ext64, (void*)sys->d_ext32, (void*)sys->d_force})
        if (p) cudaFree(p);
    sys->d_ext64 = nullptr;
    sys->d_ext32 = nullptr;
    sys->d_force = nullptr;
    if (!sys->damped() && !sys->forced()) return CHO_OK;
    const int s = sys->s;
    const int64_t n_sys = sys->n_sys;
    std::vector<double> E64((size_t)n_sys * 5 * s, 0.0);
    std::vector<float> E32((size_t)n_sys * 10 * s, 0.0f);
    for (int64_t p = 0; p < n_sys; ++p) {
        const double* m = &sys->h_masses[(size_t)p * s];
        const double* C = &sys->h_springs[(size_t)p * s];
        const double* c = sys->damped() ? &sys->h_dampers[(size_t)p * s] : nullptr;
        const double* F = sys->forced() ? &sys->h_famp[(size_t)p * s] : nullptr;
        double* e = &E64[(size_t)p * 5 * s];
        for (int i = 0; i < s; ++i) {
            e[i] = C[i] / m[i];
            e[s + i] = i + 1 < s ? C[i + 1] / m[i] : 0.0;
            e[2 * s + i] = c ? c[i] / m[i] : 0.0;
            e[3 * s + i] = c && i + 1 < s ? c[i + 1] / m[i] : 0.0;
            e[4 * s + i] = F ? F[i] / m[i] : 0.0;
        }
        float* f = &E32[(size_t)p * 10 * s];
        for (int k = 0; k < 5 * s; ++k) split_pair(e[k], f[k], f[5 * s + k]);
    }
    cudaError_t err = upload(&sys->d_ext64, E64.data(), E64.size());
    if (err == cudaSuccess) err = upload(&sys->d_ext32, E32.data(), E32.size());
    if (err == cudaSuccess && sys->forced()) {
        std::vector<double> fw((size_t)n_sys * 2);
        for (int64_t p = 0; p < n_sys; ++p) {
            fw[(size_t)p * 2] = sys->h_fomega[(size_t)p];
            fw[(size_t)p * 2 + 1] = sys->h_fphase[(size_t)p];
        }
        err = upload(&sys->d_force, fw.data(), fw.size());
    }
    if (err != cudaSuccess)
        return fail(err == cudaErrorMemoryAllocation ? CHO_ENOMEM : CHO_ECUDA, "%s: %s", who, cudaGetErrorString(err));
    return CHO_OK;
}

static cho_status check_spring_system(cho_system sys, const char* who)
{
    if (!sys) return fail(CHO_EINVAL, "%s: NULL system", who);
    if (sys->kind == CHO_DENSE) return fail(CHO_EINVAL, "%s: damping and forcing are built for spring systems", who);
    if (sys->s > kChainExtMaxS) return fail(CHO_EINVAL, "%s: s = %d above %d", who, sys->s, kChainExtMaxS);
    return CHO_OK;
}

extern "C" cho_status cho_system_set_damping(cho_system sys, const double* dampers)
{
    clear_error();
    cho_status rc = check_spring_system(sys, "cho_system_set_damping");
    if (rc != CHO_OK) return rc;
    const size_t n = (size_t)sys->n_sys * sys->s;
    if (dampers) {
        for (size_t i = 0; i < n; ++i)
            if (!std::isfinite(dampers[i]) || dampers[i] < 0.0)
                return fail(CHO_EINVAL, "cho_system_set_damping: damper %zu is not finite and >= 0", i);
    }
    DeviceGuard g(sys->ctx->device);
    if (!g.ok()) return fail(CHO_ECUDA, "cho_system_set_damping: cudaSetDevice failed");
    if (dampers) sys->h_dampers.assign(dampers, dampers + n);
    else sys->h_dampers.clear();
    return build_chain_ext(sys, "cho_system_set_damping");
}

extern "C" cho_status cho_system_set_forcing(cho_system sys, const double* amplitude, const double* omega,
                                             const double* phase)
{
    clear_error();
    cho_status rc = check_spring_system(sys, "cho_system_set_forcing");
    if (rc != CHO_OK) return rc;
    const size_t n = (size_t)sys->n_sys * sys->s;
    const size_t ns = (size_t)sys->n_sys;
    if (amplitude) {
        if (!omega) return fail(CHO_EINVAL, "cho_system_set_forcing: omega required");
        if (!all_finite(amplitude, n) || !all_finite(omega, ns) || (phase && !all_finite(phase, ns)))
            return fail(CHO_EINVAL, "cho_system_set_forcing: non-finite amplitude, omega or phase");
    }
    DeviceGuard g(sys->ctx->device);
    if (!g.ok()) return fail(CHO_ECUDA, "cho_system_set_forcing: cudaSetDevice failed");
    if (amplitude) {
        sys->h_famp.assign(amplitude, amplitude + n);
        sys->h_fomega.assign(omega, omega + ns);
        if (phase) sys->h_fphase.assign(phase, phase + ns);
        else sys->h_fphase.assign(ns, 0.0);
    } else {
        sys->h_famp.clear();
        sys->h_fomega.clear();
        sys->h_fphase.clear();
    }
    return build_chain_ext(sys, "cho_system_set_forcing");
}

extern "C" cho_status cho_system_info(cho_system sys, double* omega_max, int32_t* s, int64_t* n_sys)
{
    clear_error();
    if (!sys) return fail(CHO_EINVAL, "cho_system_info: NULL system");
    if (omega_max) *omega_max = sys->omega_max;
    if (s) *s = sys->s;
    if (n_sys) *n_sys = sys->n_sys;
    return CHO_OK;
}

extern "C" cho_status cho_system_omegas(cho_system sys, double* omega)
{
    clear_error();
    if (!sys || !omega) return fail(CHO_EINVAL, "cho_system_omegas: NULL argument");
    std::memcpy(omega, sys->omegas.data(), sizeof(double) * sys->omegas.size());
    return CHO_OK;
}

extern "C" cho_status cho_system_status(cho_system sys)
{
    clear_error();
    if (!sys) return fail(CHO_EINVAL, "cho_system_status: NULL system");
    DeviceGuard g(sys->ctx->device);
    if (!g.ok()) return fail(CHO_ECUDA, "cho_system_status: cudaSetDevice failed");
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return fail(CHO_ECUDA, "cho_system_status: %s", cudaGetErrorString(e));
    return take_device_error(sys, "cho_system_status");
}

extern "C" void cho_destroy_system(cho_system sys)
{
    if (!sys) return;
    cho_ctx* ctx = sys->ctx;
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        ctx->systems.erase(sys);
    }
    DeviceGuard g(ctx->device);
    free_system_device(sys);
    delete sys;
}

// ------------------------------------------------------------------------------
// batch integration
// ------------------------------------------------------------------------------

namespace cho {

static cho_status check_batch(const cho_batch_desc* b, const char* who, bool plain_form, cudaStream_t st)
{
    if (!b || !b->system) return fail(CHO_EINVAL, "%s: NULL batch or system", who);
    const cho_system_impl* sys = b->system;
    if (b->n_inst < 0) return fail(CHO_EINVAL, "%s: n_inst < 0", who);
    if (sys->n_sys != 1 && sys->n_sys != b->n_inst)
        return fail(CHO_EINVAL, "%s: system has %lld parameter sets for %lld instances", who,
                    (long long)sys->n_sys, (long long)b->n_inst);
    if (b->n_steps < 0) return fail(CHO_EINVAL, "%s: n_steps < 0", who);
    if (b->ckpt_every < 0 || (b->ckpt_every > 0 && b->n_steps % b->ckpt_every != 0))
        return fail(CHO_EINVAL, "%s: ckpt_every must be 0 or divide n_steps", who);
    if (b->mem != CHO_MEM_DEVICE && b->mem != CHO_MEM_HOST) return fail(CHO_EINVAL, "%s: bad mem", who);
    if (b->n_inst > 0 && (!b->x0 || !b->v0 || !b->h || !b->x_out || !b->v_out))
        return fail(CHO_EINVAL, "%s: x0, v0, h, x_out and v_out are required", who);
    if (b->energy && (!b->x_traj || !b->v_traj || b->ckpt_every == 0))
        return fail(CHO_EINVAL, "%s: energy needs x_traj, v_traj and ckpt_every > 0", who);
    if ((b->x_traj || b->v_traj) && b->ckpt_every == 0)
        return fail(CHO_EINVAL, "%s: trajectories need ckpt_every > 0", who);
    const int p = b->prec;
    if (b->poly_jump < 0) return fail(CHO_EINVAL, "%s: poly_jump < 0", who);
    if (sys->damped() || sys->forced()) {
        if (plain_form || b->poly_jump != 0)
            return fail(CHO_EINVAL, "%s: damped or forced systems run RK4 stage by stage in the batch kernels", who);
        if (p != CHO_FP64 && p != CHO_FP32_KAHAN)
            return fail(CHO_EINVAL, "%s: damped or forced systems run in CHO_FP64 or CHO_FP32_KAHAN", who);
    }
    if (b->poly_jump > 0) {
        if (plain_form) return fail(CHO_EINVAL, "%s: the plain form runs RK4 stage by stage", who);
        const bool small = sys->path == PATH_SMALL;
        const bool dense1 = sys->path == PATH_DENSE && sys->n_sys == 1;
        if (!small && !dense1)
            return fail(CHO_EINVAL, "%s: the polynomial form is built for systems of s <= 32 and shared dense systems",
                        who);
        if (p != CHO_FP64 && p != CHO_FP32_KAHAN && !(dense1 && p == CHO_DENSE_FP32_SIMT))
            return fail(CHO_EINVAL, "%s: the polynomial form runs in CHO_FP64 or FP32 (compensated)", who);
        if (b->n_steps % b->poly_jump != 0 || (b->ckpt_every > 0 && b->ckpt_every % b->poly_jump != 0))
            return fail(CHO_EINVAL, "%s: poly_jump must divide n_steps and ckpt_every", who);
    }
    if (plain_form) {
        if (p != CHO_FP64) return fail(CHO_EINVAL, "%s: the plain form is FP64 only", who);
        if (b->x_traj || b->v_traj || b->energy) return fail(CHO_EINVAL, "%s: no checkpoints in the plain form", who);
    } else if (p == CHO_FP64 || p == CHO_FP32_KAHAN) {
    } else if (p == CHO_FP32X2) {
        const bool small = sys->path == PATH_SMALL;
        const bool chain = sys->path == PATH_CHAIN && sys->s <= 1024;
        if (!small && !chain)
            return fail(CHO_EINVAL, "%s: CHO_FP32X2 integrates systems of s <= 32 and spring chains of s <= 1024", who);
    } else if (p == CHO_DENSE_FP32_SIMT || p == CHO_DENSE_BF16X3 || p == CHO_DENSE_BF16X5 || p == CHO_DENSE_BF16X6) {
        if (sys->kind != CHO_DENSE) return fail(CHO_EINVAL, "%s: precision %d is for dense systems", who, p);
        if ((p != CHO_DENSE_FP32_SIMT) && (sys->path != PATH_DENSE || sys->s_tc == 0))
            return fail(CHO_EINVAL, "%s: BF16 tensor-core modes need one shared dense system with 32 < s <= 256", who);
        if (p == CHO_DENSE_BF16X6 && sys->s_tc > 128)
            return fail(CHO_EINVAL, "%s: bf16x6 needs s <= 128 (its operands exceed shared memory above)", who);
    } else {
        return fail(CHO_EINVAL, "%s: unknown precision %d", who, p);
    }
    // stability: RK4 is stable on the imaginary axis for |omega h| <= 2 sqrt 2
    const double lim = 2.0 * std::sqrt(2.0);
    const bool host_h = b->mem == CHO_MEM_HOST || !b->h_per_inst;
    if (host_h && b->n_inst > 0) {
        if (b->mem == CHO_MEM_DEVICE && !b->h_per_inst) {
            // shared h on the device: a single value, read synchronously
            double hv = 0.0;
            if (cudaMemcpyAsync(&hv, b->h, sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                cudaStreamSynchronize(st) != cudaSuccess)
                return fail(CHO_ECUDA, "%s: reading h failed", who);
            if (!(hv > 0.0) || !std::isfinite(hv)) return fail(CHO_EINVAL, "%s: h must be finite and > 0", who);
            if (sys->omega_max * hv > lim)
                return fail(CHO_EUNSTABLE, "%s: omega_max*h = %g > 2 sqrt 2", who, sys->omega_max * hv);
        } else {
            // one branch-free pass (it vectorises; a batch of 65,536 instances is checked in
            // microseconds), then a second pass only to name the first offender
            const int64_t nh = b->h_per_inst ? b->n_inst : 1;
            const bool per_set = sys->n_sys != 1 && b->h_per_inst;   // one h: check the largest omega
            const double w0 = b->h_per_inst ? sys->omegas[0] : sys->omega_max;
            const double* w = sys->omegas.data();
            const double* hp = b->h;
            // count the step sizes out of range (a NaN fails every comparison), one plain loop
            // per case so that each vectorises
            int64_t nbad = 0;
            if (per_set) {
                for (int64_t i = 0; i < nh; ++i) {
                    const double hv = hp[i];
                    nbad += (int64_t)((hv > 0.0) & (hv < INFINITY) & (w[i] * hv <= lim)) ^ 1;
                }
            } else {
                for (int64_t i = 0; i < nh; ++i) {
                    const double hv = hp[i];
                    nbad += (int64_t)((hv > 0.0) & (hv < INFINITY) & (w0 * hv <= lim)) ^ 1;
                }
            }
            const bool bad = nbad != 0;
            if (bad) {
                for (int64_t i = 0; i < nh; ++i) {
                    const double hv = b->h[i];
                    if (!(hv > 0.0) || !std::isfinite(hv))
                        return fail(CHO_EINVAL, "%s: h[%lld] must be finite and > 0", who, (long long)i);
                    const double wv = per_set ? w[i] : w0;
                    if (wv * hv > lim)
                        return fail(CHO_EUNSTABLE, "%s: instance %lld has omega_max*h = %g > 2 sqrt 2", who,
                                    (long long)i, wv * hv);
                }
            }
        }
    }
    return CHO_OK;
}

// The k-step jump blocks of a shared dense system for step h (polynomial form), built
// on first use in FP64 on the host (O(s^3 log k)), uploaded transposed and padded to
// s_pad, FP64 and FP32 pairs, and kept with the system.
static cho_status dense_poly_blocks(cho_system_impl* sys, double h, int k, bool fp64, const void** out)
{
    std::lock_guard<std::mutex> lk(sys->poly_mu);
    for (const auto& pb : sys->poly)
        if (pb.h == h && pb.k == k) {
            *out = fp64 ? (const void*)pb.d64 : (const void*)pb.d32;
            return CHO_OK;
        }
    const int s = sys->s, sp = sys->s_pad;
    std::vector<double> blk[3];
    linalg::rk4_jump_blocks(s, sys->h_B.data(), h, k, blk[0], blk[1], blk[2]);
    const size_t n = (size_t)sp * sp;
    std::vector<double> T64(3 * n, 0.0);
    std::vector<float> T32(6 * n, 0.0f);
    for (int m = 0; m < 3; ++m)
        for (int i = 0; i < s; ++i)
            for (int j = 0; j < s; ++j) {
                const double e = blk[m][(size_t)i * s + j];
                T64[m * n + (size_t)j * sp + i] = e;
                split_pair(e, T32[2 * m * n + (size_t)j * sp + i], T32[(2 * m + 1) * n + (size_t)j * sp + i]);
            }
    cho_system_impl::PolyBlocks pb{h, k, nullptr, nullptr};
    cudaError_t e = cudaMalloc(&pb.d64, T64.size() * sizeof(double));
    if (e == cudaSuccess) e = cudaMemcpy(pb.d64, T64.data(), T64.size() * sizeof(double), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc(&pb.d32, T32.size() * sizeof(float));
    if (e == cudaSuccess) e = cudaMemcpy(pb.d32, T32.data(), T32.size() * sizeof(float), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        if (pb.d64) cudaFree(pb.d64);
        if (pb.d32) cudaFree(pb.d32);
        return fail(e == cudaErrorMemoryAllocation ? CHO_ENOMEM : CHO_ECUDA, "integrate: jump blocks: %s",
                    cudaGetErrorString(e));
    }
    sys->poly.push_back(pb);
    *out = fp64 ? (const void*)pb.d64 : (const void*)pb.d32;
    return CHO_OK;
}

bool tune_key(const cho_system_impl* sys, int64_t n_inst, int32_t prec, int32_t poly_jump, TuneKey* key)
{
    if (sys->damped() || sys->forced() || n_inst <= 0) return false;
    int bucket = 0;
    while (bucket < 62 && ((int64_t)1 << (bucket + 1)) <= n_inst) ++bucket;
    const int32_t per = sys->n_sys != 1 ? 1 : 0;
    const bool fp32 = prec == CHO_FP32_KAHAN || prec == CHO_DENSE_FP32_SIMT;
    if (sys->path == PATH_SMALL && sys->s == 2 && prec == CHO_FP32_KAHAN) {
        *key = {PATH_SMALL, sys->S, prec, per, bucket + (poly_jump > 0 ? 64 : 0)};
        return true;
    }
    if (sys->path == PATH_CHAIN && poly_jump == 0 && prec != CHO_FP32X2) {   // double-FP32: one kernel
        *key = {PATH_CHAIN, sys->s, prec, per, bucket};
        return true;
    }
    if (sys->path == PATH_DENSE && fp32 && poly_jump == 0) {
        *key = {PATH_DENSE, sys->s_pad, prec, per, bucket};
        return true;
    }
    return false;
}

// Run one batch whose arrays are all device pointers.
cho_status run_device_batch(cho_ctx* ctx, const cho_batch_desc* b, cudaStream_t st, const KernelChoice* force)
{
    cho_system_impl* sys = b->system;
    KernelChoice kc;
    if (force) {
        kc = *force;
    } else {
        TuneKey key;
        if (tune_key(sys, b->n_inst, b->prec, b->poly_jump, &key)) {
            std::lock_guard<std::mutex> lk(ctx->tune_mu);
            auto it = ctx->tune.find(key);
            if (it != ctx->tune.end()) {
                if (sys->path == PATH_SMALL) kc.small_variant = it->second;
                if (sys->path == PATH_CHAIN) kc.chain_dofs = it->second;
                if (sys->path == PATH_DENSE) kc.dense_few = it->second;
            }
        }
    }
    BatchIO io{};
    io.n_inst = b->n_inst;
    io.x0 = b->x0;
    io.v0 = b->v0;
    io.h = b->h;
    io.h_per_inst = b->h_per_inst;
    io.n_steps = b->n_steps;
    io.ckpt_every = b->ckpt_every;
    io.n_ck = b->ckpt_every > 0 ? b->n_steps / b->ckpt_every : 0;
    io.poly_jump = b->poly_jump;
    io.x_out = b->x_out;
    io.v_out = b->v_out;
    io.x_traj = b->x_traj;
    io.v_traj = b->v_traj;
    if (b->n_inst == 0) return CHO_OK;
    const bool fp64 = b->prec == CHO_FP64;
    cudaError_t e;
    if (sys->damped() || sys->forced()) {
        ChainExtSys cs{sys->s, sys->n_sys != 1 ? 1 : 0, sys->d_ext64, sys->d_ext32,
                       sys->forced() ? sys->d_force : nullptr};
        e = launch_rk4_chain_ext(cs, io, fp64, st);
    } else if (sys->path == PATH_SMALL) {
        SmallSys ss{sys->s, sys->S, sys->n_sys != 1 ? 1 : 0, sys->d_B64, sys->d_B32, sys->d_err};
        ss.variant = kc.small_variant;
        e = b->prec == CHO_FP32X2 ? launch_rk4_small_dw(ss, io, st) : launch_rk4_small(ss, io, fp64, st);
    } else if (sys->path == PATH_CHAIN) {
        ChainSys cs{sys->s, sys->n_sys != 1 ? 1 : 0, sys->d_B64, sys->d_B32};
        cs.dofs_per_thread = kc.chain_dofs;
        e = b->prec == CHO_FP32X2 ? launch_rk4_chain_dw(cs, io, st) : launch_rk4_chain(cs, io, fp64, st);
    } else if (b->poly_jump > 0) {
        // polynomial form of a shared dense system: one h for the whole batch
        const size_t nh = b->h_per_inst ? (size_t)b->n_inst : 1;
        std::vector<double> hv(nh);
        e = cudaMemcpyAsync(hv.data(), b->h, nh * sizeof(double), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return fail(CHO_ECUDA, "integrate: reading h: %s", cudaGetErrorString(e));
        for (double hh : hv)
            if (hh != hv[0]) return fail(CHO_EINVAL, "integrate: the dense polynomial form needs one h for the batch");
        const void* E = nullptr;
        cho_status rc = dense_poly_blocks(sys, hv[0], b->poly_jump, fp64, &E);
        if (rc != CHO_OK) return rc;
        DenseSys ds{sys->s, sys->s_pad, sys->d_B64, sys->d_B32, sys->d_Bbf, sys->s_tc, sys->d_err, 0, 0};
        e = launch_rk4_dense_poly(ds, E, io, fp64, st);
    } else {
        DenseSys ds{sys->s, sys->s_pad, sys->d_B64, sys->d_B32, sys->d_Bbf, sys->s_tc, sys->d_err, 0,
                    sys->n_sys != 1 ? 1 : 0};
        ds.few = kc.dense_few;
        e = launch_rk4_dense(ds, io, b->prec, st);
    }
    if (e != cudaSuccess) return fail(CHO_ECUDA, "integrate: kernel launch: %s", cudaGetErrorString(e));
    if (b->energy) {
        EnergySys es{sys->kind, sys->s, sys->n_sys != 1 ? 1 : 0, sys->d_masses, sys->d_springs, sys->d_M, sys->d_K};
        e = launch_energy(es, b->x_traj, b->v_traj, b->n_inst, io.n_ck, b->energy, st);
        if (e != cudaSuccess) return fail(CHO_ECUDA, "integrate: energy launch: %s", cudaGetErrorString(e));
    }
    return CHO_OK;
}

// Stage host arrays through the context workspace, run, copy back, synchronise.
template <class Run>
static cho_status run_staged(cho_ctx* ctx, const cho_batch_desc* b, cudaStream_t st, Run run)
{
    const int64_t n = b->n_inst;
    const int s = b->system->s;
    const int64_t n_ck = b->ckpt_every > 0 ? b->n_steps / b->ckpt_every : 0;
    const size_t ns = (size_t)n * s;
    const size_t nh = b->h_per_inst ? (size_t)n : 1;
    const size_t ntr = (size_t)n * n_ck * s;
    size_t off[8], total = 0;
    auto take = [&](int k, size_t count) {
        off[k] = total;
        total += ((count * sizeof(double) + 255) / 256) * 256;
    };
    take(0, ns);                      // x0
    take(1, ns);                      // v0
    take(2, nh);                      // h
    take(3, ns);                      // x_out
    take(4, ns);                      // v_out
    take(5, b->x_traj ? ntr : 0);
    take(6, b->v_traj ? ntr : 0);
    take(7, b->energy ? (size_t)n * n_ck : 0);
    std::lock_guard<std::mutex> lk(ctx->ws_mu);
    cudaError_t e;
    char* base = (char*)ctx->ws.get(total, &e);
    if (!base) return fail(CHO_ENOMEM, "integrate: staging %zu bytes: %s", total, cudaGetErrorString(e));
    auto P = [&](int k) { return (double*)(base + off[k]); };
    cho_batch_desc d = *b;
    d.mem = CHO_MEM_DEVICE;
    d.x0 = P(0);
    d.v0 = P(1);
    d.h = P(2);
    d.x_out = P(3);
    d.v_out = P(4);
    d.x_traj = b->x_traj ? P(5) : nullptr;
    d.v_traj = b->v_traj ? P(6) : nullptr;
    d.energy = b->energy ? P(7) : nullptr;
#define CHO_STAGE(dst, src, bytes, kind)                                                        \
    do {                                                                                        \
        if ((bytes) > 0) {                                                                      \
            e = cudaMemcpyAsync((void*)(dst), (const void*)(src), (bytes), kind, st);          \
            if (e != cudaSuccess) return fail(CHO_ECUDA, "integrate: copy: %s", cudaGetErrorString(e)); \
        }                                                                                       \
    } while (0)
    CHO_STAGE(d.x0, b->x0, ns * 8, cudaMemcpyHostToDevice);
    CHO_STAGE(d.v0, b->v0, ns * 8, cudaMemcpyHostToDevice);
    CHO_STAGE(d.h, b->h, nh * 8, cudaMemcpyHostToDevice);
    cho_status rc = run(&d);
    if (rc != CHO_OK) return rc;
    CHO_STAGE(b->x_out, d.x_out, ns * 8, cudaMemcpyDeviceToHost);
    CHO_STAGE(b->v_out, d.v_out, ns * 8, cudaMemcpyDeviceToHost);
    if (b->x_traj) CHO_STAGE(b->x_traj, d.x_traj, ntr * 8, cudaMemcpyDeviceToHost);
    if (b->v_traj) CHO_STAGE(b->v_traj, d.v_traj, ntr * 8, cudaMemcpyDeviceToHost);
    if (b->energy) CHO_STAGE(b->energy, d.energy, (size_t)n * n_ck * 8, cudaMemcpyDeviceToHost);
#undef CHO_STAGE
    // the system's device error word comes back with the results (one synchronisation);
    // it is reset only in the rare case that a bounded wait gave up
    cho_system_impl* sys = b->system;
    const bool err_async = sys->d_err && (ctx->err_host || cudaHostAlloc((void**)&ctx->err_host, sizeof(int),
                                                                         cudaHostAllocDefault) == cudaSuccess);
    if (err_async) {
        e = cudaMemcpyAsync(ctx->err_host, sys->d_err, sizeof(int), cudaMemcpyDeviceToHost, st);
        if (e != cudaSuccess) return fail(CHO_ECUDA, "integrate: %s", cudaGetErrorString(e));
    }
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fail(CHO_ECUDA, "integrate: %s", cudaGetErrorString(e));
    if (!err_async) return take_device_error(sys, "integrate");
    if (*ctx->err_host == 0) return CHO_OK;
    e = cudaMemset(sys->d_err, 0, sizeof(int));
    if (e != cudaSuccess) return fail(CHO_ECUDA, "integrate: resetting the device error word: %s", cudaGetErrorString(e));
    return fail(CHO_ETIMEOUT, "integrate: a bounded device wait gave up after its time limit; results are invalid");
}

static cho_status run_plain_device(cho_ctx* ctx, const cho_batch_desc* b, cudaStream_t st)
{
    cho_system_impl* sys = b->system;
    const int s = sys->s;
    const bool dense = sys->kind == CHO_DENSE;
    const double* coef = sys->d_plain;
    cudaError_t e;
    std::lock_guard<std::mutex> lk(ctx->plain_mu);
    double* work = (double*)ctx->plain_ws.get(sizeof(double) * 10 * (size_t)s, &e);
    if (!work) return fail(CHO_ENOMEM, "integrate_plain: %s", cudaGetErrorString(e));
    double* y = work + 8 * (size_t)s;
    std::vector<double> hbuf;
    const double* hh = b->h;
    if (b->mem == CHO_MEM_DEVICE) {      // the host loop needs h values
        const size_t nh = b->h_per_inst ? (size_t)b->n_inst : 1;
        hbuf.resize(nh);
        e = cudaMemcpyAsync(hbuf.data(), b->h, nh * 8, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return fail(CHO_ECUDA, "integrate_plain: %s", cudaGetErrorString(e));
        hh = hbuf.data();
    }
    for (int64_t q = 0; q < b->n_inst; ++q) {
        const int64_t set = sys->n_sys == 1 ? 0 : q;
        PlainSys ps{s, dense ? 1 : 0, coef + set * (dense ? (int64_t)s * s : 3 * (int64_t)s)};
        e = cudaMemcpyAsync(y, b->x0 + q * s, sizeof(double) * s, cudaMemcpyDeviceToDevice, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(y + s, b->v0 + q * s, sizeof(double) * s, cudaMemcpyDeviceToDevice, st);
        const double h = hh[b->h_per_inst ? q : 0];
        for (int64_t n = 0; n < b->n_steps && e == cudaSuccess; ++n) e = launch_plain_step(ps, y, work, h, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(b->x_out + q * s, y, sizeof(double) * s, cudaMemcpyDeviceToDevice, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(b->v_out + q * s, y + s, sizeof(double) * s, cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) return fail(CHO_ECUDA, "integrate_plain: %s", cudaGetErrorString(e));
    }
    return CHO_OK;
}

}  // namespace cho

cho_status cho::validate_batch(const cho_batch_desc* b, const char* who, cudaStream_t st)
{
    return check_batch(b, who, false, st);
}

extern "C" cho_status cho_integrate_batch(cho_ctx* ctx, const cho_batch_desc* b, void* stream)
{
    clear_error();
    if (!ctx) return fail(CHO_EINVAL, "cho_integrate_batch: NULL ctx");
    DeviceGuard g(ctx->device);
    if (!g.ok()) return fail(CHO_ECUDA, "cho_integrate_batch: cudaSetDevice failed");
    cudaStream_t st = (cudaStream_t)stream;
    cho_status rc = check_batch(b, "cho_integrate_batch", false, st);
    if (rc != CHO_OK) return rc;
    if (b->mem == CHO_MEM_DEVICE) return run_device_batch(ctx, b, st, nullptr);
    return run_staged(ctx, b, st, [&](const cho_batch_desc* d) { return run_device_batch(ctx, d, st, nullptr); });
}

extern "C" cho_status cho_integrate_plain(cho_ctx* ctx, const cho_batch_desc* b, void* stream)
{
    clear_error();
    if (!ctx) return fail(CHO_EINVAL, "cho_integrate_plain: NULL ctx");
    DeviceGuard g(ctx->device);
    if (!g.ok()) return fail(CHO_ECUDA, "cho_integrate_plain: cudaSetDevice failed");
    cudaStream_t st = (cudaStream_t)stream;
    cho_status rc = check_batch(b, "cho_integrate_plain", true, st);
    if (rc != CHO_OK) return rc;
    if (b->mem == CHO_MEM_DEVICE) return run_plain_device(ctx, b, st);
    return run_staged(ctx, b, st, [&](const cho_batch_desc* d) { return run_plain_device(ctx, d, st); });
}

extern "C" cho_status cho_energy(cho_ctx* ctx, cho_system sys, const double* x, const double* v, int64_t n_inst,
                                 int64_t n_per, int32_t mem, double* E, void* stream)
{
    clear_error();
    if (!ctx || !sys) return fail(CHO_EINVAL, "cho_energy: NULL argument");
    if (n_inst < 0 || n_per < 0) return fail(CHO_EINVAL, "cho_energy: negative size");
    if (n_inst * n_per > 0 && (!x || !v || !E)) return fail(CHO_EINVAL, "cho_energy: NULL array");
    if (sys->n_sys != 1 && sys->n_sys != n_inst)
        return fail(CHO_EINVAL, "cho_energy: system has %lld parameter sets for %lld instances",
                    (long long)sys->n_sys, (long long)n_inst);
    if (mem != CHO_MEM_DEVICE && mem != CHO_MEM_HOST) return fail(CHO_EINVAL, "cho_energy: bad mem");
    if (sys->kind == CHO_DENSE && sys->s > 3072) return fail(CHO_EINVAL, "cho_energy: s > 3072");
    DeviceGuard g(ctx->device);
    if (!g.ok()) return fail(CHO_ECUDA, "cho_energy: cudaSetDevice failed");
    cudaStream_t st = (cudaStream_t)stream;
    EnergySys es{sys->kind, sys->s, sys->n_sys != 1 ? 1 : 0, sys->d_masses, sys->d_springs, sys->d_M, sys->d_K};
    const size_t nst = (size_t)n_inst * n_per;
    if (mem == CHO_MEM_DEVICE) {
        cudaError_t e = launch_energy(es, x, v, n_inst, n_per, E, st);
        if (e != cudaSuccess) return fail(CHO_ECUDA, "cho_energy: %s", cudaGetErrorString(e));
        return CHO_OK;
    }
    const size_t xb = ((nst * sys->s * 8 + 255) / 256) * 256;
    std::lock_guard<std::mutex> lk(ctx->ws_mu);
    cudaError_t e;
    char* base = (char*)ctx->ws.get(2 * xb + nst * 8 + 256, &e);
    if (!base) return fail(CHO_ENOMEM, "cho_energy: %s", cudaGetErrorString(e));
    double* dx = (double*)base;
    double* dv = (double*)(base + xb);
    double* dE = (double*)(base + 2 * xb);
    e = cudaMemcpyAsync(dx, x, nst * sys->s * 8, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dv, v, nst * sys->s * 8, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = launch_energy(es, dx, dv, n_inst, n_per, dE, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(E, dE, nst * 8, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fail(CHO_ECUDA, "cho_energy: %s", cudaGetErrorString(e));
    return CHO_OK;
}
