"""Seeded synthetic workloads for coupled linear oscillators.

This module produces inputs only: masses, spring rates, mass and stiffness
matrices, initial states, step sizes and request streams, all in FP64 numpy
arrays.  It contains no integration arithmetic.  The tests, the benchmark,
the smoke check and the oracle's callers all draw from it, so the GPU path and
the oracle are fed the same numbers.

Workloads (sizes, distributions and seeds):

* ``eq3_single``     -- eq. 3 with m = 2 kg, C = 2025 N/m, x(0) = (1, 0), v(0) = 0,
                        h = 1e-4 s, 1e5 steps (the 2-DOF system of Section 2).
* ``two_dof_batch``  -- 65,536 independent systems of eq. 2 with masses and spring
                        rates log-uniform in [0.1, 10] kg and [1e2, 1e4] N/m,
                        x(0) ~ U(-1, 1), v(0) = 0, h = T_min/200 per instance, 1e4 steps.
* ``chain_batch``    -- fixed-free chains of s = 1024 masses (eq. 2 generalised),
                        masses log-uniform [0.5, 2] kg, spring rates log-uniform
                        [1e2, 1e3] N/m, x(0) ~ N(0, 0.1^2), v(0) = 0, h = T_min/100,
                        1e4 steps, 4096 instances.
* ``dense_group``    -- eq. 1 with M = I + 0.1 G G^T / s, K = Q diag(lam) Q^T (Q Haar
                        orthogonal, lam log-uniform [1, 1e4]), one (M, K) shared by 8192
                        instances, x(0) ~ N(0, 1), v(0) = 0, h = T_min/100, 5e3 steps.
* ``request_stream`` -- Poisson arrivals of mixed 2-DOF / chain / dense solves with
                        log-uniform sizes and horizons and three priority classes.

T_min = 2 pi / omega_max, with omega_max^2 the largest eigenvalue of the pencil
(K, M), found with a library eigensolver.  Every step size except eq. 3's is
rounded to FP32 so that FP64 and FP32 computations use the identical h.
"""
from __future__ import annotations

import math

import numpy as np

SEED_BASE = 1702


def _rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def _log_uniform(rng, lo, hi, size):
    return np.exp(rng.uniform(math.log(lo), math.log(hi), size=size))


def fp32_exact(h):
    """Round step sizes to the nearest FP32 value (returned as FP64)."""
    return np.asarray(h, dtype=np.float64).astype(np.float32).astype(np.float64)


# ---------------------------------------------------------------------------
# Top frequency of each system (used only to choose h = T_min / k)
# ---------------------------------------------------------------------------

def stiffness_chain(springs):
    """Tridiagonal stiffness of the fixed-free chain as (diag, offdiag) arrays.

    Spring 0 ties mass 0 to the wall, spring i joins masses i-1 and i, the last
    mass is free: K_ii = C_i + C_{i+1} (C_s = 0), K_{i,i+1} = -C_{i+1}.
    """
    springs = np.atleast_2d(np.asarray(springs, dtype=np.float64))
    diag = springs.copy()
    diag[:, :-1] += springs[:, 1:]
    off = -springs[:, 1:]
    return diag, off


def dense_stiffness_chain(springs):
    """Full (n, s, s) stiffness matrices of fixed-free chains."""
    diag, off = stiffness_chain(springs)
    n, s = diag.shape
    K = np.zeros((n, s, s))
    idx = np.arange(s)
    K[:, idx, idx] = diag
    K[:, idx[:-1], idx[1:]] = off
    K[:, idx[1:], idx[:-1]] = off
    return K


def omega_max_chain(masses, springs):
    """Largest natural frequency of each chain (library tridiagonal eigensolver)."""
    from scipy.linalg import eigvalsh_tridiagonal

    masses = np.atleast_2d(np.asarray(masses, dtype=np.float64))
    diag, off = stiffness_chain(springs)
    s = masses.shape[1]
    if s == 1:
        return np.sqrt(diag[:, 0] / masses[:, 0])
    d = diag / masses
    e = off / np.sqrt(masses[:, :-1] * masses[:, 1:])
    if s == 2:
        # stacked 2x2 symmetric eigenproblems in one library call
        A = np.empty((masses.shape[0], 2, 2))
        A[:, 0, 0] = d[:, 0]
        A[:, 1, 1] = d[:, 1]
        A[:, 0, 1] = A[:, 1, 0] = e[:, 0]
        return np.sqrt(np.linalg.eigvalsh(A)[:, -1])
    out = np.empty(masses.shape[0])
    for i in range(masses.shape[0]):
        lam = eigvalsh_tridiagonal(d[i], e[i], select="i", select_range=(s - 1, s - 1))
        out[i] = math.sqrt(lam[0])
    return out


def omega_max_dense(M, K):
    """Largest natural frequency of M x'' + K x = 0 (library generalised eigensolver)."""
    from scipy.linalg import eigh

    M = np.asarray(M, dtype=np.float64)
    K = np.asarray(K, dtype=np.float64)
    if M.ndim == 2:
        lam = eigh(K, M, eigvals_only=True)
        return math.sqrt(lam[-1])
    return np.array([math.sqrt(eigh(K[i], M[i], eigvals_only=True)[-1]) for i in range(M.shape[0])])


# ---------------------------------------------------------------------------
# Workloads
# ---------------------------------------------------------------------------

def eq3_single(x0=(1.0, 0.0)):
    """Eq. 3: equal masses m = 2 kg, equal springs C = 2025 N/m, h = 1e-4 s, 1e5 steps."""
    return {
        "kind": "two_dof",
        "s": 2,
        "masses": np.array([[2.0, 2.0]]),
        "springs": np.array([[2025.0, 2025.0]]),
        "x0": np.array([list(x0)], dtype=np.float64),
        "v0": np.zeros((1, 2)),
        "h": np.array([1e-4]),
        "n_steps": 100_000,
    }


def two_dof_batch(n_inst=65_536, n_steps=10_000, steps_per_period=200, seed=SEED_BASE + 1):
    """Independent systems of eq. 2 (m1 != m2, C1 != C2), one parameter set per instance."""
    rng = _rng(seed)
    masses = _log_uniform(rng, 0.1, 10.0, (n_inst, 2))
    springs = _log_uniform(rng, 1e2, 1e4, (n_inst, 2))
    x0 = rng.uniform(-1.0, 1.0, size=(n_inst, 2))
    v0 = np.zeros((n_inst, 2))
    w = omega_max_chain(masses, springs)
    h = fp32_exact(2.0 * math.pi / w / steps_per_period)
    return {"kind": "two_dof", "s": 2, "masses": masses, "springs": springs, "x0": x0, "v0": v0,
            "h": h, "n_steps": int(n_steps), "omega_max": w}


def chain_batch(n_inst=4096, s=1024, n_steps=10_000, steps_per_period=100, seed=SEED_BASE + 2,
                sigma=0.1):
    """Fixed-free spring chains of s masses, one parameter set per instance."""
    rng = _rng(seed)
    masses = _log_uniform(rng, 0.5, 2.0, (n_inst, s))
    springs = _log_uniform(rng, 1e2, 1e3, (n_inst, s))
    x0 = rng.normal(0.0, sigma, size=(n_inst, s))
    v0 = np.zeros((n_inst, s))
    w = omega_max_chain(masses, springs)
    h = fp32_exact(2.0 * math.pi / w / steps_per_period)
    return {"kind": "chain", "s": s, "masses": masses, "springs": springs, "x0": x0, "v0": v0,
            "h": h, "n_steps": int(n_steps), "omega_max": w}


def haar_orthogonal(rng, s):
    """Haar-distributed orthogonal matrix: QR of a Gaussian matrix with the sign fix."""
    Z = rng.normal(size=(s, s))
    Q, R = np.linalg.qr(Z)
    return Q * np.sign(np.diag(R))[None, :]


def dense_system(s, seed, lam_lo=1.0, lam_hi=1e4):
    """One (M, K) pair: M = I + 0.1 G G^T / s, K = Q diag(lam) Q^T."""
    rng = _rng(seed)
    G = rng.normal(size=(s, s))
    M = np.eye(s) + 0.1 * (G @ G.T) / s
    M = 0.5 * (M + M.T)
    Q = haar_orthogonal(rng, s)
    lam = _log_uniform(rng, lam_lo, lam_hi, s)
    K = (Q * lam[None, :]) @ Q.T
    K = 0.5 * (K + K.T)
    return M, K, Q, lam


def dense_group(s=128, n_inst=8192, n_steps=5000, steps_per_period=100, seed=None):
    """One shared (M, K) of size s and n_inst seeded initial displacements."""
    if seed is None:
        seed = SEED_BASE + 3 + 1000 * s
    M, K, Q, lam = dense_system(s, seed)
    rng = _rng(seed + 7)
    x0 = rng.normal(0.0, 1.0, size=(n_inst, s))
    v0 = np.zeros((n_inst, s))
    w = omega_max_dense(M, K)
    h = float(fp32_exact(2.0 * math.pi / w / steps_per_period))
    return {"kind": "dense", "s": s, "M": M[None], "K": K[None], "Q": Q, "lam": lam, "x0": x0,
            "v0": v0, "h": np.full(n_inst, h), "n_steps": int(n_steps), "omega_max": w}


def dense_own(s=128, n_inst=64, n_steps=1000, steps_per_period=100, seed=None):
    """n_inst independent dense systems of size s, each with its own (M, K) drawn as in
    ``dense_system`` (seed + instance index), h = T_min/steps_per_period per instance."""
    if seed is None:
        seed = SEED_BASE + 5 + 1000 * s
    Ms, Ks, ws = [], [], []
    for i in range(n_inst):
        M, K, _, _ = dense_system(s, seed + i)
        Ms.append(M)
        Ks.append(K)
        ws.append(omega_max_dense(M, K))
    rng = _rng(seed + 10 ** 6)
    x0 = rng.normal(0.0, 1.0, size=(n_inst, s))
    v0 = np.zeros((n_inst, s))
    w = np.asarray(ws)
    h = fp32_exact(2.0 * math.pi / w / steps_per_period)
    return {"kind": "dense", "s": s, "M": np.stack(Ms), "K": np.stack(Ks), "x0": x0, "v0": v0, "h": h,
            "n_steps": int(n_steps), "omega_max": w}


def uniform_chain(s, m=1.0, C=1.0):
    """Uniform fixed-free chain: all masses m, all springs C."""
    return np.full((1, s), float(m)), np.full((1, s), float(C))


def request_stream(n_req=200_000, rate_per_s=1000.0, s_lo=2, s_hi=512, n_lo=1_000, n_hi=100_000,
                   class_mix=(0.2, 0.3, 0.5), seed=SEED_BASE + 4, dense_sizes=(4, 8, 16, 32, 64, 128, 256, 512)):
    """Poisson request stream of mixed solves.

    Each request gets an arrival time (exponential gaps at ``rate_per_s``), a
    priority class (0 highest, drawn with ``class_mix``), a size s log-uniform
    over the integers [s_lo, s_hi], a horizon log-uniform over [n_lo, n_hi]
    steps, and a type: s = 2 is an eq. 2 system; larger s is a spring chain or
    (half of the time) a dense system, whose s is snapped to the nearest of
    ``dense_sizes`` so that dense requests share a few pre-built (M, K) groups.
    Parameters of each request are drawn lazily by ``request_params``.
    """
    rng = _rng(seed)
    gaps = rng.exponential(1.0 / rate_per_s, size=n_req)
    t = np.cumsum(gaps)
    cls = rng.choice(3, size=n_req, p=np.asarray(class_mix) / sum(class_mix))
    s = np.floor(np.exp(rng.uniform(math.log(s_lo), math.log(s_hi + 1), size=n_req))).astype(np.int64)
    s = np.clip(s, s_lo, s_hi)
    n = np.round(_log_uniform(rng, n_lo, n_hi, n_req)).astype(np.int64)
    is_dense = (s > 2) & (rng.uniform(size=n_req) < 0.5)
    dense_sizes = np.asarray(dense_sizes)
    snapped = dense_sizes[np.argmin(np.abs(np.log(s[:, None]) - np.log(dense_sizes[None, :])), axis=1)]
    s = np.where(is_dense, snapped, s)
    kind = np.where(s == 2, 0, np.where(is_dense, 2, 1))
    return {"t_arrive": t, "priority": cls, "s": s, "n_steps": n, "kind": kind,
            "seed": seed, "n_req": n_req}


def request_params(stream, i):
    """Parameters of request i of a ``request_stream`` (chain/2-DOF: its own masses and springs)."""
    rng = _rng(int(stream["seed"]) * 1_000_003 + int(i))
    s = int(stream["s"][i])
    kind = int(stream["kind"][i])
    x0 = rng.uniform(-1.0, 1.0, size=(1, s))
    v0 = np.zeros((1, s))
    if kind == 2:
        return {"kind": "dense", "s": s, "x0": x0, "v0": v0}
    lo_m, hi_m, lo_c, hi_c = (0.1, 10.0, 1e2, 1e4) if s == 2 else (0.5, 2.0, 1e2, 1e3)
    masses = _log_uniform(rng, lo_m, hi_m, (1, s))
    springs = _log_uniform(rng, lo_c, hi_c, (1, s))
    w = omega_max_chain(masses, springs)
    h = fp32_exact(2.0 * math.pi / w / (200 if s == 2 else 100))
    return {"kind": "two_dof" if s == 2 else "chain", "s": s, "masses": masses, "springs": springs,
            "x0": x0, "v0": v0, "h": h}
