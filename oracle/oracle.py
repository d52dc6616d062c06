"""ctypes wrapper around the FP64 C oracle.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The C code does all the arithmetic; this module compiles it with gcc
(``-O2 -ffp-contract=off``, no fast-math), marshals numpy arrays, and may split
a batch of independent instances over host threads.  ctypes releases the GIL
during each foreign call, so every thread runs the same single-threaded C
function on its own slice of instances; the result does not depend on the
number of threads.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from concurrent.futures import ThreadPoolExecutor

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cho_oracle.c")
_LIB_DIR = os.path.join(_HERE, "_build")
_lock = threading.Lock()
_libs: dict[int, ctypes.CDLL] = {}

_dp = ctypes.POINTER(ctypes.c_double)


def _lib_path(mutant: int) -> str:
    name = "libcho_oracle.so" if mutant == 0 else f"libcho_oracle_mut{mutant}.so"
    return os.path.join(_LIB_DIR, name)


def build(mutant: int = 0, force: bool = False) -> str:
    """Compile the oracle into a shared library and return its path.

    ``mutant`` > 0 compiles a copy with one deliberately planted mistake; only
    the mutation tests use it, to show that the pins catch that mistake.
    """
    os.makedirs(_LIB_DIR, exist_ok=True)
    out = _lib_path(mutant)
    if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(_SRC):
        return out
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c99", "-fPIC", "-shared",
           f"-DORACLE_MUTANT={int(mutant)}", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def load(mutant: int = 0) -> ctypes.CDLL:
    with _lock:
        if mutant in _libs:
            return _libs[mutant]
        lib = ctypes.CDLL(build(mutant))
        L, I, D = ctypes.c_long, ctypes.c_int, ctypes.c_double
        for fn in ("oracle_rk4_chain", "oracle_rk4_dense"):
            f = getattr(lib, fn)
            f.restype = I
            f.argtypes = [I, L, L, _dp, _dp, _dp, _dp, _dp, L, L, _dp, _dp, _dp, _dp]
        f = lib.oracle_rk4_chain_ext
        f.restype = I
        f.argtypes = [I, L, L, _dp, _dp, _dp, _dp, _dp, _dp, _dp, _dp, _dp, L, L, _dp, _dp, _dp, _dp]
        for fn in ("oracle_energy_chain", "oracle_energy_dense"):
            f = getattr(lib, fn)
            f.restype = I
            f.argtypes = [I, L, L, _dp, _dp, _dp, _dp, _dp]
        _libs[mutant] = lib
        return lib


def _ptr(a):
    if a is None:
        return None
    return a.ctypes.data_as(_dp)


def _f64(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _run_rk4(fn_name, s, p1, p2, x0, v0, h, n_steps, ckpt_every, threads, mutant):
    lib = load(mutant)
    fn = getattr(lib, fn_name)
    x0 = _f64(x0).reshape(-1, s)
    v0 = _f64(v0).reshape(-1, s)
    n_inst = x0.shape[0]
    h = _f64(np.broadcast_to(np.asarray(h, dtype=np.float64), (n_inst,)))
    per = s if fn_name == "oracle_rk4_chain" else s * s
    p1 = _f64(p1).reshape(-1, per)
    p2 = _f64(p2).reshape(-1, per)
    n_sys = p1.shape[0]
    if n_sys not in (1, n_inst):
        raise ValueError("parameter sets must be 1 or one per instance")
    n_ck = n_steps // ckpt_every if ckpt_every else 0
    x_out = np.empty((n_inst, s))
    v_out = np.empty((n_inst, s))
    x_tr = np.empty((n_inst, n_ck, s)) if n_ck else None
    v_tr = np.empty((n_inst, n_ck, s)) if n_ck else None

    def part(lo, hi):
        if hi <= lo:
            return 0
        ps = slice(0, 1) if n_sys == 1 else slice(lo, hi)
        nsys_part = 1 if n_sys == 1 else hi - lo
        return fn(s, hi - lo, nsys_part, _ptr(p1[ps]), _ptr(p2[ps]), _ptr(x0[lo:hi]), _ptr(v0[lo:hi]),
                  _ptr(h[lo:hi]), int(n_steps), int(ckpt_every),
                  _ptr(x_tr[lo:hi]) if n_ck else None, _ptr(v_tr[lo:hi]) if n_ck else None,
                  _ptr(x_out[lo:hi]), _ptr(v_out[lo:hi]))

    threads = max(1, min(int(threads), n_inst))
    if threads == 1:
        rcs = [part(0, n_inst)]
    else:
        bounds = np.linspace(0, n_inst, threads + 1).astype(int)
        with ThreadPoolExecutor(threads) as ex:
            rcs = list(ex.map(lambda i: part(bounds[i], bounds[i + 1]), range(threads)))
    for rc in rcs:
        if rc != 0:
            raise RuntimeError(f"{fn_name} failed with status {rc}")
    return {"x": x_out, "v": v_out, "x_traj": x_tr, "v_traj": v_tr}


def rk4_chain(masses, springs, x0, v0, h, n_steps, ckpt_every=0, threads=1, mutant=0):
    """Classical RK4 on the fixed-free spring chain (eq. 2 generalised to s masses).

    masses, springs: (n_sys, s) with n_sys 1 or n_inst; springs[:, 0] is the wall spring.
    x0, v0: (n_inst, s).  h: scalar or (n_inst,).  Returns final x, v and, when
    ``ckpt_every`` > 0, trajectories (n_inst, n_steps // ckpt_every, s).
    """
    masses = np.atleast_2d(masses)
    s = masses.shape[1]
    return _run_rk4("oracle_rk4_chain", s, masses, springs, x0, v0, h, n_steps, ckpt_every,
                    threads, mutant)


def rk4_chain_ext(masses, springs, x0, v0, h, n_steps, ckpt_every=0, dampers=None, force_amp=None,
                  force_omega=None, force_phase=None, threads=1, mutant=0):
    """Classical RK4 on the chain with a dashpot beside every spring and a harmonic force
    F_i cos(omega t + phase) on every mass: M x'' + D x' + K x = f(t) (beyond the paper's
    undamped eqs. 1-3).  dampers, force_amp: (n_sys, s) or None; force_omega, force_phase:
    (n_sys,) (phase defaults to 0).  t = 0 at the first step.  Other arguments as ``rk4_chain``."""
    lib = load(mutant)
    masses = _f64(np.atleast_2d(masses))
    s = masses.shape[1]
    springs = _f64(springs).reshape(-1, s)
    n_sys = masses.shape[0]
    x0 = _f64(x0).reshape(-1, s)
    v0 = _f64(v0).reshape(-1, s)
    n_inst = x0.shape[0]
    if n_sys not in (1, n_inst):
        raise ValueError("parameter sets must be 1 or one per instance")
    h = _f64(np.broadcast_to(np.asarray(h, dtype=np.float64), (n_inst,)))
    damp = None if dampers is None else _f64(dampers).reshape(-1, s)
    famp = None if force_amp is None else _f64(force_amp).reshape(-1, s)
    fom = None if famp is None else _f64(np.broadcast_to(np.asarray(force_omega, dtype=np.float64), (n_sys,)))
    fph = None if famp is None else _f64(np.broadcast_to(
        np.asarray(0.0 if force_phase is None else force_phase, dtype=np.float64), (n_sys,)))
    n_ck = n_steps // ckpt_every if ckpt_every else 0
    x_out = np.empty((n_inst, s))
    v_out = np.empty((n_inst, s))
    x_tr = np.empty((n_inst, n_ck, s)) if n_ck else None
    v_tr = np.empty((n_inst, n_ck, s)) if n_ck else None

    def sl(a, lo, hi):
        if a is None:
            return None
        return _ptr(a[0:1] if n_sys == 1 else a[lo:hi])

    def part(lo, hi):
        if hi <= lo:
            return 0
        nsys_part = 1 if n_sys == 1 else hi - lo
        return lib.oracle_rk4_chain_ext(s, hi - lo, nsys_part, sl(masses, lo, hi), sl(springs, lo, hi),
                                        sl(damp, lo, hi), sl(famp, lo, hi), sl(fom, lo, hi), sl(fph, lo, hi),
                                        _ptr(x0[lo:hi]), _ptr(v0[lo:hi]), _ptr(h[lo:hi]), int(n_steps),
                                        int(ckpt_every), _ptr(x_tr[lo:hi]) if n_ck else None,
                                        _ptr(v_tr[lo:hi]) if n_ck else None, _ptr(x_out[lo:hi]),
                                        _ptr(v_out[lo:hi]))

    threads = max(1, min(int(threads), n_inst))
    if threads == 1:
        rcs = [part(0, n_inst)]
    else:
        bounds = np.linspace(0, n_inst, threads + 1).astype(int)
        with ThreadPoolExecutor(threads) as ex:
            rcs = list(ex.map(lambda i: part(bounds[i], bounds[i + 1]), range(threads)))
    for rc in rcs:
        if rc != 0:
            raise RuntimeError(f"oracle_rk4_chain_ext failed with status {rc}")
    return {"x": x_out, "v": v_out, "x_traj": x_tr, "v_traj": v_tr}


def rk4_dense(M, K, x0, v0, h, n_steps, ckpt_every=0, threads=1, mutant=0):
    """Classical RK4 on M x'' + K x = 0 (eq. 1) with full SPD M and symmetric K.

    M, K: (s, s) shared or (n_inst, s, s).  Other arguments as ``rk4_chain``.
    """
    M = np.asarray(M, dtype=np.float64)
    s = M.shape[-1]
    return _run_rk4("oracle_rk4_dense", s, M, K, x0, v0, h, n_steps, ckpt_every, threads, mutant)


def _energy(fn_name, s, p1, p2, x, v, per):
    lib = load(0)
    x = _f64(x).reshape(-1, s)
    v = _f64(v).reshape(-1, s)
    p1 = _f64(p1).reshape(-1, per)
    p2 = _f64(p2).reshape(-1, per)
    n_inst = x.shape[0]
    n_sys = p1.shape[0]
    if n_sys not in (1, n_inst):
        raise ValueError("parameter sets must be 1 or one per state")
    E = np.empty(n_inst)
    rc = getattr(lib, fn_name)(s, n_inst, n_sys, _ptr(p1), _ptr(p2), _ptr(x), _ptr(v), _ptr(E))
    if rc != 0:
        raise RuntimeError(f"{fn_name} failed with status {rc}")
    return E


def energy_chain(masses, springs, x, v):
    """Mechanical energy of chain states: sum 1/2 m v^2 + sum 1/2 C (spring extension)^2."""
    masses = np.atleast_2d(masses)
    s = masses.shape[1]
    return _energy("oracle_energy_chain", s, masses, springs, x, v, s)


def energy_dense(M, K, x, v):
    """Mechanical energy 1/2 v^T M v + 1/2 x^T K x of states of eq. 1."""
    M = np.asarray(M, dtype=np.float64)
    s = M.shape[-1]
    return _energy("oracle_energy_dense", s, M, K, x, v, s * s)
