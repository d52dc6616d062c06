"""Shared helpers of the GPU parity tests: error metric, sampling, oracle calls."""
import os

import numpy as np

import oracle

THREADS = max(1, min(16, os.cpu_count() or 1))

# Tolerances (relative max-norm over the checkpoints of the horizon):
TOL_FP64 = 1e-10
TOL_FP32 = 1e-5


def rel_err(got, ref):
    """Per instance: max_t |got - ref|_inf / max_t |ref|_inf over (n_inst, n_ck, s) trajectories."""
    got = np.asarray(got)
    ref = np.asarray(ref)
    axes = tuple(range(1, ref.ndim))
    num = np.max(np.abs(got - ref), axis=axes)
    den = np.maximum(np.max(np.abs(ref), axis=axes), 1e-300)
    return num / den


def sample_indices(n, k, seed=0):
    """First, last and a seeded random sample of instance indices (sorted, unique)."""
    if n <= k:
        return np.arange(n)
    rng = np.random.default_rng(seed)
    idx = np.concatenate([[0, n - 1], rng.choice(n, size=k - 2, replace=False)])
    return np.unique(idx)


def oracle_run(cfg, idx=None, n_steps=None, ckpt_every=0):
    """Run the oracle on a workload dict (optionally a subset of instances)."""
    n_steps = cfg["n_steps"] if n_steps is None else n_steps
    sel = slice(None) if idx is None else idx
    if cfg["kind"] == "dense":
        M, K = cfg["M"], cfg["K"]
        if M.shape[0] != 1:
            M, K = M[sel], K[sel]
        return oracle.rk4_dense(M if M.shape[0] != 1 else M[0], K if K.shape[0] != 1 else K[0],
                                cfg["x0"][sel], cfg["v0"][sel], cfg["h"][sel], n_steps, ckpt_every,
                                threads=THREADS)
    m, C = cfg["masses"], cfg["springs"]
    if m.shape[0] != 1:
        m, C = m[sel], C[sel]
    return oracle.rk4_chain(m, C, cfg["x0"][sel], cfg["v0"][sel], cfg["h"][sel], n_steps, ckpt_every,
                            threads=THREADS)


def with_ends(traj, final):
    """Trajectory checkpoints plus the final state, (n_inst, n_ck + 1, s)."""
    if traj is None:
        return np.asarray(final)[:, None, :]
    return np.concatenate([np.asarray(traj), np.asarray(final)[:, None, :]], axis=1)
