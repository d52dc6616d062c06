/*
 * cho.h -- C ABI of the batched coupled-harmonic-oscillator integrator.
 *
 * The library integrates many independent instances of eq. 1 of "Parallel
 * Implementation of the Coupled Harmonic Oscillator" (arXiv 1702.02207),
 *
 *     sum_j (m_ij x_j'' + k_ij x_j) = 0,   i.e.  M x'' + K x = 0,        (eq. 1)
 *
 * with fixed-step classical fourth-order Runge-Kutta on the first-order form
 * y = (x, v), v = x' (Section 3: x3 = x1', x4 = x2', right-hand side D(1)..D(4)).
 * Each RK4 step evaluates the acceleration a = -M^{-1} K x four times (the
 * D(3), D(4) rows of Section 3), forms the stage states, and adds the weighted
 * sum h/6 (k1 + 2 k2 + 2 k3 + k4) to the state.
 *
 * Three kinds of system are accepted:
 *   CHO_TWO_DOF  the spring system of eq. 2 (Section 2, Figure 1): mass 1 on a
 *                wall spring C1, spring C2 between masses 1 and 2, mass 2 free.
 *                Eq. 3 is the case m1 = m2, C1 = C2.
 *   CHO_CHAIN    eq. 2 generalised to s masses: spring i joins mass i-1 and i,
 *                spring 0 joins mass 0 to the wall, the last mass is free.
 *                K is tridiagonal with K_ii = C_i + C_{i+1}, K_{i,i+1} = -C_{i+1}.
 *   CHO_DENSE    eq. 1 with full symmetric positive definite M and symmetric K.
 *
 * Conventions for every call:
 *   - every function returns a cho_status and never aborts the process;
 *   - on error, output parameters are left untouched and cho_last_error()
 *     returns a message for the calling thread;
 *   - handles are opaque and owned by the library;
 *   - arrays passed in are owned by the caller; the library copies what it keeps;
 *   - all floating-point inputs and outputs are IEEE binary64, row-major;
 *   - device pointers must be CUDA device memory of the context's device (or
 *     managed memory); "stream" is a cudaStream_t (NULL = legacy default stream).
 *
 * Test-only environment switches.  Three variables exist only so that the test suite
 * can reach code paths that normal inputs never take; applications must leave them
 * unset, and no result depends on them except as stated:
 *   CHO_TWO_DOF_KERNEL=generic|pair         forces the lane-group or the pair form of the
 *       FP32 s = 2 batch kernels instead of the default choice (all give the same bits;
 *       read once, at the first such launch of the process);
 *   CHO_TEST_STALL_MMA=1                    the tensor-core dense kernel issues no MMA,
 *       so its bounded wait runs out and the call reports CHO_ETIMEOUT (read per launch);
 *   CHO_TEST_WITHHOLD_HANDOVER=1            the balanced kernels (s = 2, and the
 *       one-CTA tensor-core kernel for s <= 128) publish no hand-over flag, so every
 *       hand-over wait runs out (CHO_ETIMEOUT, NaN states; read per launch);
 *   CHO_TEST_WITHHOLD_DOORBELL=1            persistent serving never rings its kernels'
 *       doorbell, so their bounded waits run out (requests end with CHO_ETIMEOUT; read when
 *       a context's serving engine starts).
 */
#ifndef CHO_H
#define CHO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum cho_status {
    CHO_OK = 0,
    CHO_PENDING = 1,        /* cho_poll: the request has not finished yet            */
    CHO_EINVAL = -1,        /* bad argument (null pointer, size, kind, precision)    */
    CHO_ENOMEM = -2,        /* device or host allocation failed                       */
    CHO_EBUDGET = -3,       /* a request can never fit in the serving memory budget  */
    CHO_EUNSTABLE = -4,     /* omega_max * h exceeds the RK4 stability limit 2*sqrt 2 */
    CHO_ENOTSPD = -5,       /* M is not symmetric positive definite                   */
    CHO_ETIMEOUT = -6,      /* a bounded wait gave up                                 */
    CHO_ENONFINITE = -7,    /* a non-finite input or state                            */
    CHO_ECANCELLED = -8,    /* the request was cancelled                              */
    CHO_ECUDA = -9,         /* a CUDA runtime call failed                             */
    CHO_EINTERNAL = -10,    /* an internal consistency check failed                   */
    CHO_ENOTFOUND = -11     /* unknown ticket                                         */
} cho_status;

typedef enum cho_kind {
    CHO_TWO_DOF = 0,
    CHO_CHAIN = 1,
    CHO_DENSE = 2
} cho_kind;

/* Arithmetic of the integration (the state is always returned in FP64).
 *   CHO_FP64             FP64 state and stages.
 *   CHO_FP32_KAHAN       FP32 state and stages, Kahan-compensated state update,
 *                        M^{-1}K and h/6 carried as unevaluated FP32 pairs (hi + lo).
 *   CHO_DENSE_FP32_SIMT  dense systems: like CHO_FP32_KAHAN (the same kernel family).
 *   CHO_DENSE_BF16X3/X5/X6  dense systems with a shared (M, K): the product
 *                        M^{-1}K X on tensor cores with M^{-1}K and X split into
 *                        BF16 pieces, FP32 accumulation, FP32 + Kahan state.
 *                        x3: 3 partial products, operands to 16 bits (~1e-3 error);
 *                        x5: 5 products, M^{-1}K to 24 bits, X to 16; x6: 6 products,
 *                        both to 24 bits (s <= 128).  x5/x6 keep each 16-wide K chunk
 *                        in its own accumulator and add the chunks in FP32 (<= 1e-5
 *                        over 5e3 steps at h = T_min/100).
 *   CHO_FP32X2           systems of s <= 32 (any kind) and spring chains of s <= 1024:
 *                        state, coefficients
 *                        and every operation as unevaluated pairs of FP32 numbers
 *                        (about 48 significant bits; error-free TwoSum / TwoProd on the
 *                        FP32 pipe), the stage form of CHO_FP64.  Within the FP64 mode's
 *                        tolerance of the FP64 oracle on this GPU's much faster FP32 pipe.
 *                        Batch calls only (not the polynomial form, serving or the
 *                        plain form).                                               */
typedef enum cho_prec {
    CHO_FP64 = 0,
    CHO_FP32_KAHAN = 1,
    CHO_DENSE_BF16X3 = 2,
    CHO_DENSE_BF16X5 = 3,
    CHO_DENSE_BF16X6 = 4,
    CHO_DENSE_FP32_SIMT = 5,
    CHO_FP32X2 = 6
} cho_prec;

/* Where the state arrays of a batch live. */
typedef enum cho_mem {
    CHO_MEM_DEVICE = 0,     /* device pointers; the call is asynchronous on the stream  */
    CHO_MEM_HOST = 1        /* host pointers; the library stages them through device
                               memory and returns after the results are in host memory */
} cho_mem;

typedef struct cho_ctx cho_ctx;
typedef struct cho_system_impl* cho_system;

/* Optional context settings (pass NULL for defaults).  Zero fields take defaults. */
typedef struct cho_config {
    int64_t budget_bytes;   /* serving: device bytes for resident request state (default 40 GiB) */
    int32_t chunk_steps;    /* serving: RK4 steps per chunk between scheduling points (default 1000) */
    int32_t max_slots;      /* serving: maximum resident requests (default 1 << 20)       */
    int32_t chunk_us;       /* serving: > 0 tunes each kernel group's chunk length while it runs so
                               that a chunk takes about this many microseconds of device time
                               (chunk_steps is the first guess); 0 keeps chunk_steps.  Results do
                               not depend on the chunk length. */
    int32_t persistent;     /* serving: 1 serves rk4_small groups and chain groups (s <= 2048) with
                               resident kernels driven through pinned mapped memory (doorbell per
                               chunk, completion ring; see cho_submit), 0 launches every chunk.
                               Results are bitwise the same. */
    int32_t active_pct;     /* serving: the requests advanced by each chunk (the active set) are
                               chosen in priority order (class, then admission order) up to this
                               percentage of one wave of the device, each request weighing
                               1 / (instances its kernel holds resident at once); the others
                               stay resident and wait at their chunk boundary.  0: 100;
                               < 0: no cap (every resident request advances every chunk).
                               Results do not depend on it. */
    int32_t reserved[1];
} cho_config;

/* Description of one system kind and size, with n_sys parameter sets.
 * TWO_DOF / CHAIN: masses (n_sys, s) in kg and springs (n_sys, s) in N/m, springs[.,0]
 *   is the wall spring; every value must be finite and > 0.  TWO_DOF requires s == 2.
 * DENSE: M and K (n_sys, s, s), row-major; M symmetric positive definite, K symmetric
 *   (relative asymmetry <= 1e-12), all finite.
 * All pointers are host memory; the library copies them. */
typedef struct cho_system_desc {
    int32_t kind;           /* cho_kind */
    int32_t s;              /* degrees of freedom, >= 1 */
    int64_t n_sys;          /* parameter sets, >= 1 */
    const double* masses;
    const double* springs;
    const double* M;
    const double* K;
    const double* mass_coupling;   /* TWO_DOF / CHAIN, optional (NULL: diagonal M): (n_sys, s),
                                      entry i the off-diagonal mass m_{i,i+1} = m_{i+1,i} coupling
                                      mass i and mass i + 1 (the last entry of each set is unused).
                                      M is then tridiagonal -- eq. 1 with general m_ij, as a
                                      consistent mass matrix of a discretised rod has -- and the
                                      system is built and integrated as a DENSE system of that M and
                                      the chain's K (s <= 512; cho_system_info reports CHO_DENSE);
                                      M must be positive definite (CHO_ENOTSPD otherwise). */
} cho_system_desc;

/* One batch of independent instances of one system.
 * Instance i uses parameter set i when the system has n_inst sets, or set 0 when it
 * has one.  Layouts (row-major, FP64):
 *   x0, v0, x_out, v_out      (n_inst, s)
 *   h                         (n_inst) when h_per_inst != 0, else (1)
 *   x_traj, v_traj (optional) (n_inst, n_steps / ckpt_every, s): checkpoint c holds the
 *                             state after (c + 1) * ckpt_every steps
 *   energy (optional)         (n_inst, n_steps / ckpt_every): energy of each checkpoint,
 *                             1/2 v^T M v + 1/2 x^T K x in FP64; needs x_traj and v_traj
 * x_out/v_out may alias x0/v0.  ckpt_every must divide n_steps when it is non-zero.
 *
 * Polynomial form (poly_jump = k >= 1).  For the linear system y' = A y, A = [[0, I], [-B, 0]],
 * one classical RK4 step is exactly y <- P(hA) y with P(z) = 1 + z + z^2/2 + z^3/6 + z^4/24
 * (the four stages of Section 3 composed).  The library forms E = P(hA)^k - I per instance in
 * FP64 and advances y <- y + E y (FP32: E as FP32 pairs, compensated state), k steps per
 * update: the same result up to rounding with fewer dependent operations.  Supported for
 *   - every system of s <= 32 (any kind; one parameter set or one per instance) in CHO_FP64
 *     and CHO_FP32_KAHAN.  s = 2: E (4 x 4) per instance in registers.  Other s: E is
 *     2 S x 2 S (S = s padded to 2, 4, 8, 16 or 32), formed per instance by a set-up kernel
 *     (one matrix for the batch when the system has one parameter set and h_per_inst == 0)
 *     and kept in shared memory by the integration kernel; device scratch of
 *     (matrices) x 4 S^2 doubles for the call, from the library's stream-ordered pool;
 *   - DENSE systems with one shared (M, K) and one h for the whole batch: the blocks of
 *     P(hA)^k formed in FP64 on the host and cached per (h, k), in CHO_FP64, CHO_FP32_KAHAN
 *     or CHO_DENSE_FP32_SIMT on the CUDA cores (reading h synchronises the stream).
 * k must divide n_steps and ckpt_every.  In FP32, k omega_max h <= 1 keeps the rounding of
 * the increments within the FP32 tolerance.  Errors: CHO_EINVAL otherwise. */
typedef struct cho_batch_desc {
    cho_system system;
    int64_t n_inst;
    int32_t prec;           /* cho_prec */
    int32_t mem;            /* cho_mem: where x0, v0, h and all outputs live */
    const double* x0;
    const double* v0;
    const double* h;
    int32_t h_per_inst;
    int32_t poly_jump;      /* 0: RK4 stage by stage (Section 3's D(1)..D(4)).  k >= 1: the
                               polynomial form of the same map, k steps at a time (see below) */
    int64_t n_steps;
    int64_t ckpt_every;
    double* x_out;
    double* v_out;
    double* x_traj;
    double* v_traj;
    double* energy;
} cho_batch_desc;

/* One serving request: a single instance of one parameter set of a system. */
typedef struct cho_request {
    cho_system system;
    int64_t sys_index;      /* which parameter set of the system */
    const double* x0;       /* host, (s) */
    const double* v0;       /* host, (s) */
    double h;
    int64_t n_steps;
    int32_t prec;           /* CHO_FP64, CHO_FP32_KAHAN, or for shared dense systems with
                               32 < s <= 256 a BF16 tensor-core mode */
    int32_t priority;       /* 0 (highest), 1, 2 */
} cho_request;

typedef struct cho_result {
    double* x;              /* caller-owned host buffer of s values, filled on CHO_OK */
    double* v;              /* caller-owned host buffer of s values, filled on CHO_OK */
    double t_submit;        /* seconds on the library's monotonic clock */
    double t_admit;
    double t_done;
} cho_result;

/* ---- context -------------------------------------------------------------------- */

/* Create a context on CUDA device `device`.  Errors: CHO_EINVAL (bad device),
 * CHO_ECUDA.  The context owns its device buffers and its serving thread. */
cho_status cho_init(cho_ctx** out, int device, const cho_config* cfg);

/* Stop serving (pending requests finish as CHO_ECANCELLED), free everything.
 * Systems created on the context must be destroyed first or are freed here. */
void cho_shutdown(cho_ctx* ctx);

/* Thread-local message of the last failed call on this thread ("" if none). */
const char* cho_last_error(void);

/* ---- systems (step a0: set-up, off the integration loop) -------------------------- */

/* Validate a system description and build the iteration matrix B = M^{-1} K of every
 * parameter set (eqs. 1-3; for TWO_DOF/CHAIN from the spring rates per mass, for DENSE
 * by a Cholesky solve), its largest natural frequency omega_max (the square root of the
 * largest eigenvalue of the pencil (K, M)), and the FP32/BF16 splittings the kernels
 * use; upload them to the device.  Errors: CHO_EINVAL, CHO_ENOTSPD, CHO_ENOMEM, CHO_ECUDA. */
cho_status cho_create_system(cho_ctx* ctx, const cho_system_desc* desc, cho_system* out);

/* Damping and forcing -- beyond the paper, whose eqs. 1-3 are undamped; its introduction
 * motivates hardware-in-the-loop simulation, where both appear.  For TWO_DOF and CHAIN
 * systems only, integrated by rk4_chain for any s <= 1024 in CHO_FP64 or CHO_FP32_KAHAN:
 *   M x'' + D x' + K x = f(t),  m_i x_i'' = -C_i e_i + C_{i+1} e_{i+1} - c_i e_i' + c_{i+1} e_{i+1}'
 *                                          + F_i cos(omega t + phase),  e_i = x_i - x_{i-1},
 * classical RK4 with the stage times t, t + h/2, t + h/2, t + h; t = 0 at the first step of
 * every batch (a resumed run carries its time in the phase).  Damped or forced systems are
 * not accepted by cho_submit, the polynomial form, the plain form or the BF16 modes
 * (CHO_EINVAL there).
 *
 * cho_system_set_damping: dampers (n_sys, s) host array in N s/m, finite and >= 0, dashpot i
 * attached like spring i; NULL removes the damping.
 * cho_system_set_forcing: amplitude (n_sys, s) in N (finite), omega and phase (n_sys) in rad/s
 * and rad (finite; phase may be NULL for 0); NULL amplitude removes the forcing.
 * Both replace earlier values and copy the arrays.  Errors: CHO_EINVAL, CHO_ENOMEM, CHO_ECUDA. */
cho_status cho_system_set_damping(cho_system sys, const double* dampers);
cho_status cho_system_set_forcing(cho_system sys, const double* amplitude, const double* omega, const double* phase);

/* omega_max: the largest natural frequency over all parameter sets (rad/s). */
cho_status cho_system_info(cho_system sys, double* omega_max, int32_t* s, int64_t* n_sys);

/* Largest natural frequency of each parameter set, omega (n_sys), host memory. */
cho_status cho_system_omegas(cho_system sys, double* omega);

/* Device-side status of a system: waits for the device, then returns CHO_ETIMEOUT (and
 * clears it) if a run on this system gave up one of its bounded waits (the tensor-core
 * kernel's waits on its MMAs, about a second each, after which it stops; the balanced 2-DOF
 * kernel's wait for a hand-over between warps, one second plus the time run so far, after
 * which that unit finishes as NaN); its results are then invalid.  Otherwise
 * CHO_OK.  Host-memory batches report this themselves; device-memory batches, which return
 * before the kernel ends, report it here.  Errors: CHO_EINVAL, CHO_ECUDA. */
cho_status cho_system_status(cho_system sys);

void cho_destroy_system(cho_system sys);

/* ---- batched integration (steps a1-a5) -------------------------------------------- */

/* Integrate every instance of the batch for n_steps classical RK4 steps (Section 3's
 * first-order form, eq. 1 right-hand side), writing the final state, optional
 * checkpoints and optional FP64 energies.  Kernel choice: s <= 32 any kind -> rk4_small;
 * CHAIN/TWO_DOF s > 32 -> rk4_chain; DENSE s > 32 with one shared parameter set ->
 * rk4_dense.  Errors: CHO_EINVAL, CHO_EUNSTABLE (omega_max * h > 2 sqrt 2 for some
 * instance; checked on host values only, i.e. for CHO_MEM_HOST or h_per_inst == 0),
 * CHO_ECUDA, CHO_ENOMEM.  CHO_MEM_DEVICE: asynchronous on `stream`.  CHO_MEM_HOST: the arrays
 * are staged through the context's device workspace on `stream` (NULL: the legacy default
 * stream) and the call returns once the results are in host memory. */
cho_status cho_integrate_batch(cho_ctx* ctx, const cho_batch_desc* batch, void* stream);

/* CUDA graphs.  With device arrays and h_per_inst = 1 (and not the dense polynomial form,
 * which reads h on the host), cho_integrate_batch neither synchronises nor allocates outside
 * stream-ordered memory pools, so a sequence of calls -- batches of different systems, sizes
 * and precisions -- can be captured on a stream into a CUDA graph and replayed: each replay
 * runs the captured batches on the current contents of their arrays, with the bits of direct
 * calls.  Make one call of each shape before capturing (first calls set kernel attributes
 * and query cluster occupancy). */

/* The same integration in the plain form: one system at a time, one kernel launch per
 * RK stage and one per update, FP64 state kept in device memory between launches.
 * This is the un-batched baseline the batched kernels are measured against.  Only
 * prec == CHO_FP64; checkpoints and energy are not supported (pass NULL / 0).
 * Uses a device work buffer of 10 s doubles held by the context. */
cho_status cho_integrate_plain(cho_ctx* ctx, const cho_batch_desc* batch, void* stream);

/* The plain form without allocating: the same integration as cho_integrate_plain, for
 * callers that must not allocate device memory once they run -- a real-time or
 * hardware-in-the-loop stepping loop, where cudaMalloc can block on the device and break
 * a step's deadline, or an application that hands all device memory to its own pool.
 * The paper has no counterpart; this is a deployment variant.
 * Its scratch (state and stage buffers of one instance, 10 s doubles) is a fixed array
 * compiled into the library, so s must be <= 4096 (CHO_EINVAL above).  Every GPU that
 * loads the library holds that array (320 KiB) until the process exits.  All calls share
 * it: calls whose work overlaps on the GPU race on it and must be serialised by the
 * caller (same stream, or synchronised streams).  Each call rewrites all scratch it
 * reads, so nothing in it has to start at zero.
 * The first call on a device looks up the array's device address (this loads it onto
 * that device) and keeps it for the life of the process; make that first call before any
 * stream capture.  The kept address does not survive cudaDeviceReset (or any other
 * teardown of the device's primary context): do not call this entry point after one.
 * Arrays: device pointers only (batch->mem == CHO_MEM_DEVICE), prec == CHO_FP64, no
 * checkpoints or energy, no damped or forced systems.  h is read on the device only, so
 * the host cannot check it: an h that is not finite and > 0, or with omega_max * h >
 * 2 sqrt 2 for the instance's parameter set, yields NaN in that instance's x_out and
 * v_out (where cho_integrate_plain returns CHO_EINVAL or CHO_EUNSTABLE) once at least
 * one step runs.  Asynchronous on `stream`; no allocation, host or device, at any call.
 * Errors: CHO_EINVAL, CHO_ECUDA. */
cho_status cho_integrate_plain_noalloc(cho_ctx* ctx, const cho_batch_desc* batch, void* stream);

/* Several batches packed into as few kernel launches as possible.  Batches whose systems fall
 * into one kernel family and size class run in ONE launch over a device work table with one
 * entry per instance (its parameter set's coefficients, its state, h, its step count and its
 * own s): rk4_small by padded size S (any kind of s <= 32 together: 2-DOF systems, chains of
 * 3 and 4 masses and dense systems of s = 4 share S = 4), rk4_chain by DOFs per thread (s < 64,
 * < 128, < 256, >= 256; the CTA is sized for the group's largest chain) and rk4_dense by
 * system.  Each batch's x_out, v_out are bitwise equal to a separate cho_integrate_batch call
 * of that batch (every family computes an instance with the same operations in both forms).
 * Eq. 1 and eq. 2 with uneven sizes and horizons in one launch: the instance, not the batch,
 * is the unit of work.
 * Every batch: device arrays (mem == CHO_MEM_DEVICE), poly_jump == 0, no checkpoints or energy,
 * not damped or forced, prec CHO_FP64, CHO_FP32_KAHAN, CHO_DENSE_FP32_SIMT or (one shared dense
 * system) CHO_DENSE_BF16X3/X5/X6; each batch is otherwise checked as cho_integrate_batch checks
 * it (a batch with one h on the device is read synchronously for the stability check).
 * Asynchronous on `stream`; the work table and state blocks come from the library's
 * stream-ordered scratch pool for the call.  Errors: CHO_EINVAL, CHO_EUNSTABLE, CHO_ENOMEM,
 * CHO_ECUDA. */
cho_status cho_integrate_packed(cho_ctx* ctx, const cho_batch_desc* batches, int32_t n_batches, void* stream);

/* FP64 energy 1/2 v^T M v + 1/2 x^T K x of states x, v (n_inst, n_per, s); state (i, c)
 * uses parameter set i (or 0 when the system has one set).  E is (n_inst, n_per).
 * mem selects host or device pointers as in cho_batch_desc.  Errors: CHO_EINVAL, CHO_ECUDA. */
cho_status cho_energy(cho_ctx* ctx, cho_system sys, const double* x, const double* v,
                      int64_t n_inst, int64_t n_per, int32_t mem, double* E, void* stream);

/* ---- autotuning of the batch kernels ------------------------------------------------- */

/* For some batch shapes several kernels compute the same bits: FP32 TWO_DOF systems
 * (balanced schedule, pair form, lane-group form), CHAIN systems (1, 2, 4 or 8 DOFs per
 * thread), FP32 DENSE systems (one instance per CTA or cluster of CTAs, or the streaming
 * kernel).  cho_autotune runs each candidate for the shape (system, n_inst, prec,
 * poly_jump) on seeded inputs on the context's device, keeps those whose final states
 * equal the first candidate's bit for bit, times them with CUDA events (best of three
 * runs of about 3 ms after a warm-up) and records the fastest in the context's tune
 * table; the first candidate is the kernel the default rules pick, and it is kept unless
 * another is at least 3 % faster.  Later cho_integrate_batch calls of the same shape use it; the instance count
 * is matched by floor(log2(n_inst)).  Shapes with a single kernel report one variant
 * and record nothing.  A system with one parameter set per instance needs n_inst equal
 * to its set count.  Synchronous; allocates 7 n_inst s doubles of device memory for the
 * call.  Errors: CHO_EINVAL (as cho_integrate_batch for the shape), CHO_ENOMEM, CHO_ECUDA. */
typedef struct cho_tune_result {
    int32_t n_variants;         /* candidates timed (1: the shape has a single kernel)           */
    int32_t chosen;             /* index of the fastest eligible candidate                        */
    int32_t code[8];            /* variant code as stored in the tune table (-1: default kernel)  */
    double us_per_step[8];      /* device time per RK4 step of the whole batch; < 0: its bits
                                   differed from the first candidate's, so it was not eligible  */
    char name[8][24];           /* candidate names                                                */
    int64_t sample_steps;       /* RK4 steps per timed run                                        */
} cho_tune_result;

cho_status cho_autotune(cho_ctx* ctx, cho_system sys, int64_t n_inst, int32_t prec, int32_t poly_jump,
                        cho_tune_result* out);

/* The variant code recorded for a shape (-1: none; the default rules apply). */
cho_status cho_tune_query(cho_ctx* ctx, cho_system sys, int64_t n_inst, int32_t prec, int32_t poly_jump,
                          int32_t* code);

/* Write the tune table to a text file ("cho-tune 1", then one tab-separated entry per line
 * led by the device name), or read one and add the entries recorded for this context's
 * device (n_loaded may be NULL).  Errors: CHO_EINVAL (cannot open, or not a tune file). */
cho_status cho_tune_save(cho_ctx* ctx, const char* path);
cho_status cho_tune_load(cho_ctx* ctx, const char* path, int32_t* n_loaded);

/* ---- measurement ---------------------------------------------------------------------- */

/* Measured arithmetic peak of the CUDA cores on the context's device: every thread of a
 * full-occupancy grid runs 8 independent fused multiply-add chains for iters x 16 rounds
 * (kind 0: scalar FP32 fma.rn.f32; 1: packed FP32 pairs fma.rn.f32x2; 2: FP64 fma.rn.f64),
 * timed with CUDA events after one warm-up launch.  *flops_per_s = 2 x FMAs / time, the
 * denominator of the batched kernels' "alu" roofline fractions; *seconds (may be NULL) is
 * the timed launch's duration.  Not part of the paper's method: the hardware's own rate.
 * Synchronous; allocates no device memory.  Errors: CHO_EINVAL, CHO_ECUDA. */
cho_status cho_measure_fma_peak(cho_ctx* ctx, int32_t kind, int32_t iters, double* flops_per_s, double* seconds);

/* ---- serving: continuous batching of single-instance requests --------------------- */

/* Persistent serving (cho_config.persistent = 1).  rk4_small groups (any kind of s <= 32) and
 * chain groups (s <= 2048) are served by a kernel that stays resident on the group's stream
 * and runs one chunk per generation instead of one launch per chunk (Section 5's real-time
 * use: no launch on the per-chunk path).  The slot table, the status words, each group's
 * slot-id list and completion ring are pinned host memory mapped into the device; the
 * serving thread writes a generation's slot ids and rings a doorbell, the kernel's CTAs
 * advance their share, append finished slots to the ring and count the generation done.
 * Every doorbell wait on the device is bounded (about a second): a kernel left without a
 * doorbell stops, reports CHO_ETIMEOUT, and the requests of its pending generation end
 * with CHO_ETIMEOUT; the context stays usable.  Resident kernels together hold at most half
 * the SMs' worth of CTAs and 60 % of the registers, so at least half the SMs stay whole for
 * launched kernels; a group beyond that, and every dense group, is launched per chunk as in
 * the default mode.  A group with no resident request releases its kernel. */

/* Fixed priorities (Section 5's fixed-priority real-time use).  Queued requests are admitted
 * class 0 first, FIFO within a class, while a slot is free and their state fits the budget.
 * Each chunk then advances the active set: the resident requests taken in the same order
 * (class, then admission) while their weights, each the request's share of one wave of the
 * device (1 / the instances its kernel holds resident at once), stay within
 * cho_config.active_pct; the other resident requests keep their state on the device and
 * wait at their chunk boundary, so a higher-class arrival takes the place of lower-class
 * work at the next boundary.  A request's result does not depend on when it ran. */

/* Queue one request.  Inputs are copied; returns at once with a ticket.
 * Errors: CHO_EINVAL, CHO_EUNSTABLE, CHO_EBUDGET (the request alone exceeds the budget). */
cho_status cho_submit(cho_ctx* ctx, const cho_request* req, uint64_t* ticket);

/* CHO_PENDING while queued or running; CHO_OK with out->x, out->v filled once done
 * (the ticket is then released); or the request's error (CHO_ECANCELLED,
 * CHO_ENONFINITE, CHO_ECUDA).  CHO_ENOTFOUND for an unknown or released ticket. */
cho_status cho_poll(cho_ctx* ctx, uint64_t ticket, cho_result* out);

/* The next finished request of any ticket, in the order requests finish: *ticket is set
 * and its status returned (CHO_OK with out->x, out->v filled when not NULL -- they must
 * hold s values of that request's system -- or the request's error); the ticket is then
 * released as by cho_poll.  CHO_PENDING when no finished request is waiting.  A serving
 * client collects results this way without polling every ticket it holds. */
cho_status cho_poll_any(cho_ctx* ctx, uint64_t* ticket, cho_result* out);

/* Cancel a queued or running request (it stops at its next chunk boundary). */
cho_status cho_cancel(cho_ctx* ctx, uint64_t ticket);

/* Serving counters: queued, resident, completed requests and resident device bytes. */
cho_status cho_serve_stats(cho_ctx* ctx, int64_t* queued, int64_t* resident, int64_t* completed,
                           int64_t* resident_bytes);

/* Serving traffic at chunk boundaries (cumulative since the engine started): the resident
 * state bytes the chunks read and wrote back (each advanced request's state block once each
 * way per chunk) and the DOF-steps they advanced, so that bytes / DOF-steps is the engine's
 * memory term per DOF-step (about 2 x 16 B / L for FP32 state and chunks of L steps). */
cho_status cho_serve_traffic(cho_ctx* ctx, int64_t* state_bytes_moved, int64_t* dof_steps);

#ifdef __cplusplus
}
#endif

#endif /* CHO_H */
