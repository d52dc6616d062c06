/*
 * cho_oracle.c -- FP64 reference integrator for coupled linear oscillators.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the oracle that the GPU library is
 * checked against.  Only the test suite, the smoke check and the CPU-baseline
 * leg of the benchmark load it.  It shares no code, header, table or helper
 * with the CUDA path and must never be linked into it.
 *
 * What it computes (Sections 2-3 of the paper):
 *   - the model is eq. 1,  sum_j (m_ij x_j'' + k_ij x_j) = 0, i.e. M x'' + K x = 0;
 *   - the spring system of eq. 2 (ground spring C1 on mass 1, spring C2 between
 *     masses 1 and 2, mass 2 free) generalised to a fixed-free chain of s
 *     masses: spring i joins mass i-1 and mass i, spring 0 joins mass 0 to the
 *     wall, the last mass is free; at s = 2 this is eq. 2 term by term, and with
 *     equal masses and springs it is eq. 3;
 *   - the first-order form of Section 3: the state is (x, v) with v = x',
 *     and the right-hand side is D = (v, x'') as in the D(1)..D(4) listing;
 *   - classical fourth-order Runge-Kutta with a fixed step h (the paper names
 *     Runge-Kutta integration without the order; the classical scheme with
 *     weights 1/6, 1/3, 1/3, 1/6 at nodes 0, 1/2, 1/2, 1 is the reading used).
 *   - the mechanical energy 1/2 v^T M v + 1/2 x^T K x, which eq. 1 conserves for
 *     symmetric M and K;
 *   - beyond the paper (which treats the undamped case only): the chain with a
 *     dashpot beside every spring and a harmonic force on every mass,
 *     M x'' + D x' + K x = F cos(Om t + phi), integrated by the same RK4 with the
 *     stage times t, t + h/2, t + h/2, t + h (oracle_rk4_chain_ext).
 *
 * Plain loops, FP64, single-threaded, built with -O2 -ffp-contract=off and no
 * fast-math so that every rounding is the one written here.
 *
 * Parity pins: every function here is pinned by the not-gpu tests (closed
 * forms of eqs. 6-7, the exact discrete RK4 modal map, brute-force matrix
 * powers, energy laws); none is "parity unpinned".
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_OK 0
#define ORACLE_EINVAL -1
#define ORACLE_ENOTSPD -5
#define ORACLE_ENOMEM -2

/* Planted mistakes, compiled in only by the mutation tests (-DORACLE_MUTANT=k)
 * to show that the pins catch each of them.  The default build has none. */
#ifndef ORACLE_MUTANT
#define ORACLE_MUTANT 0
#endif

/* ------------------------------------------------------------------------- */
/* Model: acceleration x'' for a given displacement x                         */
/* ------------------------------------------------------------------------- */

typedef struct {
    int kind;              /* 0 = spring chain (eq. 2 generalised), 1 = dense (eq. 1) */
    int s;
    const double* m;       /* chain: s masses */
    const double* C;       /* chain: s spring rates, C[0] is the wall spring */
    const double* c;       /* chain, optional: s dashpot rates, dashpot i beside spring i */
    const double* F;       /* chain, optional: s force amplitudes, f_i(t) = F_i cos(Om t + phi) */
    double Om, phi;        /* forcing frequency (rad/s) and phase */
    const double* M;       /* dense: s*s row-major mass matrix */
    const double* K;       /* dense: s*s row-major stiffness matrix */
    double* L;             /* dense: Cholesky factor of M (lower, row-major), owned */
    double* work;          /* dense: s scratch values, owned */
} model_t;

/* Eq. 2 written per mass: m_i x_i'' = -C_i (x_i - x_{i-1}) + C_{i+1} (x_{i+1} - x_i),
 * with x_{-1} = 0 (the wall) and no spring to the right of the last mass.
 * For s = 2: m1 x1'' = -C1 x1 + C2 (x2 - x1) and m2 x2'' = -C2 (x2 - x1). */
static void chain_accel(const model_t* md, const double* x, double* a)
{
    const int s = md->s;
    for (int i = 0; i < s; ++i) {
        double ext_left = (i == 0) ? x[0] : (x[i] - x[i - 1]);
        double force = -md->C[i] * ext_left;
        if (i + 1 < s) {
#if ORACLE_MUTANT == 1
            force -= md->C[i + 1] * (x[i + 1] - x[i]);      /* wrong sign */
#else
            force += md->C[i + 1] * (x[i + 1] - x[i]);
#endif
        }
        a[i] = force / md->m[i];
    }
}

/* Cholesky factorisation M = L L^T of a symmetric positive definite matrix. */
static int cholesky(int s, const double* M, double* L)
{
    memset(L, 0, sizeof(double) * (size_t)s * (size_t)s);
    for (int j = 0; j < s; ++j) {
        double d = M[j * s + j];
        for (int k = 0; k < j; ++k) d -= L[j * s + k] * L[j * s + k];
        if (!(d > 0.0)) return ORACLE_ENOTSPD;
        double ljj = sqrt(d);
        L[j * s + j] = ljj;
        for (int i = j + 1; i < s; ++i) {
            double t = M[i * s + j];
            for (int k = 0; k < j; ++k) t -= L[i * s + k] * L[j * s + k];
            L[i * s + j] = t / ljj;
        }
    }
    return ORACLE_OK;
}

/* Eq. 1 solved for x'':  M a = -K x.  First f = K x, then L y = -f, then L^T a = y. */
static void dense_accel(const model_t* md, const double* x, double* a)
{
    const int s = md->s;
    double* y = md->work;
    for (int i = 0; i < s; ++i) {
        double f = 0.0;
        for (int j = 0; j < s; ++j) f += md->K[i * s + j] * x[j];
        y[i] = -f;
    }
    for (int i = 0; i < s; ++i) {            /* forward substitution */
        double t = y[i];
        for (int k = 0; k < i; ++k) t -= md->L[i * s + k] * y[k];
        y[i] = t / md->L[i * s + i];
    }
    for (int i = s - 1; i >= 0; --i) {       /* back substitution with L^T */
        double t = y[i];
        for (int k = i + 1; k < s; ++k) t -= md->L[k * s + i] * a[k];
        a[i] = t / md->L[i * s + i];
    }
}

static void accel(const model_t* md, const double* x, double* a)
{
    if (md->kind == 0) chain_accel(md, x, a);
    else dense_accel(md, x, a);
}

/* Beyond the paper (its undamped eq. 1-3): M x'' + D x' + K x = f(t) for the chain,
 * a dashpot c_i beside every spring (same attachment) and a harmonic force on every
 * mass.  Per mass:
 *   m_i x_i'' = -C_i e_i + C_{i+1} e_{i+1} - c_i e_i' + c_{i+1} e_{i+1}' + F_i cos(Om t + phi),
 * e_i = x_i - x_{i-1} (x_{-1} = 0), e_i' = v_i - v_{i-1}; nothing right of the last mass. */
static void chain_accel_ext(const model_t* md, const double* x, const double* v, double t, double* a)
{
    const int s = md->s;
    const double f = md->F ? cos(md->Om * t + md->phi) : 0.0;
    for (int i = 0; i < s; ++i) {
        double ext_left = (i == 0) ? x[0] : (x[i] - x[i - 1]);
        double force = -md->C[i] * ext_left;
        if (i + 1 < s) force += md->C[i + 1] * (x[i + 1] - x[i]);
        if (md->c) {
            double rate_left = (i == 0) ? v[0] : (v[i] - v[i - 1]);
#if ORACLE_MUTANT == 4
            force += md->c[i] * rate_left;                      /* wrong sign */
#else
            force -= md->c[i] * rate_left;
#endif
            if (i + 1 < s) force += md->c[i + 1] * (v[i + 1] - v[i]);
        }
        if (md->F) force += md->F[i] * f;
        a[i] = force / md->m[i];
    }
}

/* First-order right-hand side of Section 3: y = (x, v), D(y) = (v, x''); t is the
 * stage time (used only by the forced model). */
static void rhs(const model_t* md, const double* y, double t, double* D)
{
    const int s = md->s;
    for (int i = 0; i < s; ++i) D[i] = y[s + i];            /* D(1), D(2): x' = v   */
    if (md->kind == 0 && (md->c || md->F)) chain_accel_ext(md, y, y + s, t, D + s);
    else accel(md, y, D + s);                                 /* D(3), D(4): v' = x'' */
}

/* ------------------------------------------------------------------------- */
/* Classical RK4 on y' = D(y)                                                 */
/* ------------------------------------------------------------------------- */

static int rk4_run(const model_t* md, const double* x0, const double* v0, double h,
                   long n_steps, long ckpt_every, double* x_traj, double* v_traj,
                   double* x_out, double* v_out)
{
    const int s = md->s;
    const int n = 2 * s;
    double* buf = (double*)malloc(sizeof(double) * (size_t)n * 6);
    if (!buf) return ORACLE_ENOMEM;
    double* y = buf;
    double* k1 = buf + n;
    double* k2 = buf + 2 * n;
    double* k3 = buf + 3 * n;
    double* k4 = buf + 4 * n;
    double* yt = buf + 5 * n;

    for (int i = 0; i < s; ++i) { y[i] = x0[i]; y[s + i] = v0[i]; }
    long ck = 0;
    for (long step = 1; step <= n_steps; ++step) {
        const double t = (double)(step - 1) * h;            /* stage times t, t + h/2, t + h/2, t + h */
        rhs(md, y, t, k1);
        for (int i = 0; i < n; ++i) yt[i] = y[i] + (h / 2.0) * k1[i];
        rhs(md, yt, t + h / 2.0, k2);
        for (int i = 0; i < n; ++i) yt[i] = y[i] + (h / 2.0) * k2[i];
        rhs(md, yt, t + h / 2.0, k3);
#if ORACLE_MUTANT == 2
        for (int i = 0; i < n; ++i) yt[i] = y[i] + (h / 2.0) * k3[i];   /* wrong node */
#else
        for (int i = 0; i < n; ++i) yt[i] = y[i] + h * k3[i];
#endif
        rhs(md, yt, t + h, k4);
        for (int i = 0; i < n; ++i) {
#if ORACLE_MUTANT == 3
            y[i] = y[i] + (h / 6.0) * (k1[i] + 2.0 * k2[i] + k3[i] + k4[i]);  /* dropped weight */
#else
            y[i] = y[i] + (h / 6.0) * (k1[i] + 2.0 * k2[i] + 2.0 * k3[i] + k4[i]);
#endif
        }
        if (ckpt_every > 0 && step % ckpt_every == 0) {
            if (x_traj) memcpy(x_traj + ck * s, y, sizeof(double) * (size_t)s);
            if (v_traj) memcpy(v_traj + ck * s, y + s, sizeof(double) * (size_t)s);
            ++ck;
        }
    }
    if (x_out) memcpy(x_out, y, sizeof(double) * (size_t)s);
    if (v_out) memcpy(v_out, y + s, sizeof(double) * (size_t)s);
    free(buf);
    return ORACLE_OK;
}

/* ------------------------------------------------------------------------- */
/* Public entry points: a batch of independent instances                      */
/*                                                                            */
/* Parameter sets: n_sys == 1 shares one set among all instances, otherwise   */
/* n_sys == n_inst and instance i uses set i.  Arrays are row-major:          */
/*   masses/springs (n_sys, s); M/K (n_sys, s, s); x0/v0/x_out/v_out          */
/*   (n_inst, s); h (n_inst); x_traj/v_traj (n_inst, n_steps/ckpt_every, s).  */
/* Checkpoint c holds the state after (c+1)*ckpt_every steps.                 */
/* ------------------------------------------------------------------------- */

static int check_common(int s, long n_inst, long n_sys, long n_steps, long ckpt_every)
{
    if (s < 1 || n_inst < 0 || n_steps < 0 || ckpt_every < 0) return ORACLE_EINVAL;
    if (!(n_sys == 1 || n_sys == n_inst)) return ORACLE_EINVAL;
    if (ckpt_every > 0 && n_steps % ckpt_every != 0) return ORACLE_EINVAL;
    return ORACLE_OK;
}

int oracle_rk4_chain(int s, long n_inst, long n_sys, const double* masses, const double* springs,
                     const double* x0, const double* v0, const double* h, long n_steps,
                     long ckpt_every, double* x_traj, double* v_traj, double* x_out, double* v_out)
{
    int rc = check_common(s, n_inst, n_sys, n_steps, ckpt_every);
    if (rc) return rc;
    long n_ck = ckpt_every > 0 ? n_steps / ckpt_every : 0;
    for (long q = 0; q < n_inst; ++q) {
        long p = (n_sys == 1) ? 0 : q;
        model_t md;
        memset(&md, 0, sizeof md);
        md.kind = 0;
        md.s = s;
        md.m = masses + p * s;
        md.C = springs + p * s;
        rc = rk4_run(&md, x0 + q * s, v0 + q * s, h[q], n_steps, ckpt_every,
                     x_traj ? x_traj + q * n_ck * s : NULL, v_traj ? v_traj + q * n_ck * s : NULL,
                     x_out ? x_out + q * s : NULL, v_out ? v_out + q * s : NULL);
        if (rc) return rc;
    }
    return ORACLE_OK;
}

/* The damped and forced chain (chain_accel_ext); dampers and famp (n_sys, s) may be NULL,
 * fomega and fphase (n_sys) are read only when famp is given. */
int oracle_rk4_chain_ext(int s, long n_inst, long n_sys, const double* masses, const double* springs,
                         const double* dampers, const double* famp, const double* fomega, const double* fphase,
                         const double* x0, const double* v0, const double* h, long n_steps,
                         long ckpt_every, double* x_traj, double* v_traj, double* x_out, double* v_out)
{
    int rc = check_common(s, n_inst, n_sys, n_steps, ckpt_every);
    if (rc) return rc;
    if (famp && (!fomega || !fphase)) return ORACLE_EINVAL;
    long n_ck = ckpt_every > 0 ? n_steps / ckpt_every : 0;
    for (long q = 0; q < n_inst; ++q) {
        long p = (n_sys == 1) ? 0 : q;
        model_t md;
        memset(&md, 0, sizeof md);
        md.kind = 0;
        md.s = s;
        md.m = masses + p * s;
        md.C = springs + p * s;
        md.c = dampers ? dampers + p * s : NULL;
        md.F = famp ? famp + p * s : NULL;
        md.Om = famp ? fomega[p] : 0.0;
        md.phi = famp ? fphase[p] : 0.0;
        rc = rk4_run(&md, x0 + q * s, v0 + q * s, h[q], n_steps, ckpt_every,
                     x_traj ? x_traj + q * n_ck * s : NULL, v_traj ? v_traj + q * n_ck * s : NULL,
                     x_out ? x_out + q * s : NULL, v_out ? v_out + q * s : NULL);
        if (rc) return rc;
    }
    return ORACLE_OK;
}

int oracle_rk4_dense(int s, long n_inst, long n_sys, const double* M, const double* K,
                     const double* x0, const double* v0, const double* h, long n_steps,
                     long ckpt_every, double* x_traj, double* v_traj, double* x_out, double* v_out)
{
    int rc = check_common(s, n_inst, n_sys, n_steps, ckpt_every);
    if (rc) return rc;
    long n_ck = ckpt_every > 0 ? n_steps / ckpt_every : 0;
    double* L = (double*)malloc(sizeof(double) * (size_t)s * (size_t)s);
    double* work = (double*)malloc(sizeof(double) * (size_t)s);
    if (!L || !work) { free(L); free(work); return ORACLE_ENOMEM; }
    long factored = -1;
    for (long q = 0; q < n_inst && rc == ORACLE_OK; ++q) {
        long p = (n_sys == 1) ? 0 : q;
        model_t md;
        memset(&md, 0, sizeof md);
        md.kind = 1;
        md.s = s;
        md.M = M + p * (long)s * s;
        md.K = K + p * (long)s * s;
        md.L = L;
        md.work = work;
        if (factored != p) {
            rc = cholesky(s, md.M, L);
            if (rc) break;
            factored = p;
        }
        rc = rk4_run(&md, x0 + q * s, v0 + q * s, h[q], n_steps, ckpt_every,
                     x_traj ? x_traj + q * n_ck * s : NULL, v_traj ? v_traj + q * n_ck * s : NULL,
                     x_out ? x_out + q * s : NULL, v_out ? v_out + q * s : NULL);
    }
    free(L);
    free(work);
    return rc;
}

/* Energy of the chain, written per element: kinetic 1/2 m_i v_i^2 plus the
 * potential 1/2 C_i e_i^2 stored in each spring, e_i being its extension. */
int oracle_energy_chain(int s, long n_inst, long n_sys, const double* masses, const double* springs,
                        const double* x, const double* v, double* E)
{
    if (s < 1 || n_inst < 0 || !(n_sys == 1 || n_sys == n_inst)) return ORACLE_EINVAL;
    for (long q = 0; q < n_inst; ++q) {
        long p = (n_sys == 1) ? 0 : q;
        const double* m = masses + p * s;
        const double* C = springs + p * s;
        const double* xq = x + q * s;
        const double* vq = v + q * s;
        double kin = 0.0, pot = 0.0;
        for (int i = 0; i < s; ++i) {
            kin += 0.5 * m[i] * vq[i] * vq[i];
            double e = (i == 0) ? xq[0] : (xq[i] - xq[i - 1]);
            pot += 0.5 * C[i] * e * e;
        }
        E[q] = kin + pot;
    }
    return ORACLE_OK;
}

/* Energy of eq. 1 with full matrices: 1/2 v^T M v + 1/2 x^T K x. */
int oracle_energy_dense(int s, long n_inst, long n_sys, const double* M, const double* K,
                        const double* x, const double* v, double* E)
{
    if (s < 1 || n_inst < 0 || !(n_sys == 1 || n_sys == n_inst)) return ORACLE_EINVAL;
    for (long q = 0; q < n_inst; ++q) {
        long p = (n_sys == 1) ? 0 : q;
        const double* Mp = M + p * (long)s * s;
        const double* Kp = K + p * (long)s * s;
        const double* xq = x + q * s;
        const double* vq = v + q * s;
        double kin = 0.0, pot = 0.0;
        for (int i = 0; i < s; ++i) {
            for (int j = 0; j < s; ++j) {
                kin += 0.5 * vq[i] * Mp[i * s + j] * vq[j];
                pot += 0.5 * xq[i] * Kp[i * s + j] * xq[j];
            }
        }
        E[q] = kin + pot;
    }
    return ORACLE_OK;
}

int oracle_version(void) { return 1; }
