"""ctypes binding of ``libcho.so`` (the C ABI declared in ``include/cho.h``).

The functions carry the C names and only marshal arguments: numpy arrays are
passed as host memory (``CHO_MEM_HOST``), CUDA ``torch.Tensor`` objects as
device memory (``CHO_MEM_DEVICE``) on torch's current stream.  Every step of
the integration runs in the library's CUDA kernels; there is no Python or CPU
fallback, and ``load()`` raises if the library has not been built.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libcho.so")

# ---- constants (mirror include/cho.h) --------------------------------------------
CHO_OK, CHO_PENDING = 0, 1
CHO_EINVAL, CHO_ENOMEM, CHO_EBUDGET, CHO_EUNSTABLE, CHO_ENOTSPD = -1, -2, -3, -4, -5
CHO_ETIMEOUT, CHO_ENONFINITE, CHO_ECANCELLED, CHO_ECUDA, CHO_EINTERNAL, CHO_ENOTFOUND = -6, -7, -8, -9, -10, -11
STATUS_NAMES = {
    0: "CHO_OK", 1: "CHO_PENDING", -1: "CHO_EINVAL", -2: "CHO_ENOMEM", -3: "CHO_EBUDGET",
    -4: "CHO_EUNSTABLE", -5: "CHO_ENOTSPD", -6: "CHO_ETIMEOUT", -7: "CHO_ENONFINITE",
    -8: "CHO_ECANCELLED", -9: "CHO_ECUDA", -10: "CHO_EINTERNAL", -11: "CHO_ENOTFOUND",
}
CHO_TWO_DOF, CHO_CHAIN, CHO_DENSE = 0, 1, 2
CHO_FP64, CHO_FP32_KAHAN, CHO_DENSE_BF16X3, CHO_DENSE_BF16X5, CHO_DENSE_BF16X6, CHO_DENSE_FP32_SIMT = 0, 1, 2, 3, 4, 5
CHO_FP32X2 = 6
CHO_MEM_DEVICE, CHO_MEM_HOST = 0, 1

KINDS = {"two_dof": CHO_TWO_DOF, "chain": CHO_CHAIN, "dense": CHO_DENSE}
PRECS = {"fp64": CHO_FP64, "fp32_kahan": CHO_FP32_KAHAN, "bf16x3": CHO_DENSE_BF16X3,
         "bf16x5": CHO_DENSE_BF16X5, "bf16x6": CHO_DENSE_BF16X6, "fp32_simt": CHO_DENSE_FP32_SIMT,
         "fp32x2": CHO_FP32X2}

EXPORTED = [
    "cho_init", "cho_shutdown", "cho_last_error", "cho_create_system", "cho_system_info",
    "cho_system_omegas", "cho_system_status", "cho_system_set_damping", "cho_system_set_forcing",
    "cho_destroy_system", "cho_integrate_batch", "cho_integrate_plain",
    "cho_integrate_plain_noalloc",
    "cho_energy", "cho_submit", "cho_poll", "cho_cancel", "cho_serve_stats",
    "cho_autotune", "cho_tune_query", "cho_tune_save", "cho_tune_load", "cho_measure_fma_peak",
    "cho_integrate_packed", "cho_poll_any", "cho_serve_traffic",
]

_dp = ctypes.POINTER(ctypes.c_double)


class cho_config(ctypes.Structure):
    _fields_ = [("budget_bytes", ctypes.c_int64), ("chunk_steps", ctypes.c_int32),
                ("max_slots", ctypes.c_int32), ("chunk_us", ctypes.c_int32), ("persistent", ctypes.c_int32),
                ("active_pct", ctypes.c_int32), ("reserved", ctypes.c_int32 * 1)]


class cho_tune_result(ctypes.Structure):
    _fields_ = [("n_variants", ctypes.c_int32), ("chosen", ctypes.c_int32), ("code", ctypes.c_int32 * 8),
                ("us_per_step", ctypes.c_double * 8), ("name", (ctypes.c_char * 24) * 8),
                ("sample_steps", ctypes.c_int64)]


class cho_system_desc(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("s", ctypes.c_int32), ("n_sys", ctypes.c_int64),
                ("masses", ctypes.c_void_p), ("springs", ctypes.c_void_p),
                ("M", ctypes.c_void_p), ("K", ctypes.c_void_p), ("mass_coupling", ctypes.c_void_p)]


class cho_batch_desc(ctypes.Structure):
    _fields_ = [("system", ctypes.c_void_p), ("n_inst", ctypes.c_int64), ("prec", ctypes.c_int32),
                ("mem", ctypes.c_int32), ("x0", ctypes.c_void_p), ("v0", ctypes.c_void_p),
                ("h", ctypes.c_void_p), ("h_per_inst", ctypes.c_int32), ("poly_jump", ctypes.c_int32),
                ("n_steps", ctypes.c_int64), ("ckpt_every", ctypes.c_int64),
                ("x_out", ctypes.c_void_p), ("v_out", ctypes.c_void_p), ("x_traj", ctypes.c_void_p),
                ("v_traj", ctypes.c_void_p), ("energy", ctypes.c_void_p)]


class cho_request(ctypes.Structure):
    _fields_ = [("system", ctypes.c_void_p), ("sys_index", ctypes.c_int64), ("x0", ctypes.c_void_p),
                ("v0", ctypes.c_void_p), ("h", ctypes.c_double), ("n_steps", ctypes.c_int64),
                ("prec", ctypes.c_int32), ("priority", ctypes.c_int32)]


class cho_result(ctypes.Structure):
    _fields_ = [("x", ctypes.c_void_p), ("v", ctypes.c_void_p), ("t_submit", ctypes.c_double),
                ("t_admit", ctypes.c_double), ("t_done", ctypes.c_double)]


class ChoError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status
        self.message = message


_lib = None
_lock = threading.Lock()


def load(path: str | None = None) -> ctypes.CDLL:
    """Load ``libcho.so``; raises ``ChoError`` if it is missing (build it with ``__graft_entry__.build()``)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise ChoError(CHO_EINTERNAL, f"libcho.so not built ({p}); the CUDA library is required")
        lib = ctypes.CDLL(p)
        V, I32, I64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
        sig = {
            "cho_init": ([ctypes.POINTER(V), ctypes.c_int, ctypes.POINTER(cho_config)], I32),
            "cho_shutdown": ([V], None),
            "cho_last_error": ([], ctypes.c_char_p),
            "cho_create_system": ([V, ctypes.POINTER(cho_system_desc), ctypes.POINTER(V)], I32),
            "cho_system_info": ([V, _dp, ctypes.POINTER(I32), ctypes.POINTER(I64)], I32),
            "cho_system_omegas": ([V, _dp], I32),
            "cho_system_status": ([V], I32),
            "cho_system_set_damping": ([V, V], I32),
            "cho_system_set_forcing": ([V, V, V, V], I32),
            "cho_destroy_system": ([V], None),
            "cho_integrate_batch": ([V, ctypes.POINTER(cho_batch_desc), V], I32),
            "cho_integrate_plain": ([V, ctypes.POINTER(cho_batch_desc), V], I32),
            "cho_integrate_plain_noalloc": ([V, ctypes.POINTER(cho_batch_desc), V], I32),
            "cho_energy": ([V, V, V, V, I64, I64, I32, V, V], I32),
            "cho_submit": ([V, ctypes.POINTER(cho_request), ctypes.POINTER(ctypes.c_uint64)], I32),
            "cho_poll": ([V, ctypes.c_uint64, ctypes.POINTER(cho_result)], I32),
            "cho_cancel": ([V, ctypes.c_uint64], I32),
            "cho_serve_stats": ([V] + [ctypes.POINTER(I64)] * 4, I32),
            "cho_serve_traffic": ([V] + [ctypes.POINTER(I64)] * 2, I32),
            "cho_autotune": ([V, V, I64, I32, I32, ctypes.POINTER(cho_tune_result)], I32),
            "cho_tune_query": ([V, V, I64, I32, I32, ctypes.POINTER(I32)], I32),
            "cho_tune_save": ([V, ctypes.c_char_p], I32),
            "cho_tune_load": ([V, ctypes.c_char_p, ctypes.POINTER(I32)], I32),
            "cho_measure_fma_peak": ([V, I32, I32, _dp, _dp], I32),
            "cho_integrate_packed": ([V, ctypes.POINTER(cho_batch_desc), I32, V], I32),
            "cho_poll_any": ([V, ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(cho_result)], I32),
        }
        for name, (args, res) in sig.items():
            f = getattr(lib, name)
            f.argtypes = args
            f.restype = res
        _lib = lib
        return lib


def _check(status, ok=(CHO_OK,)):
    if status not in ok:
        msg = load().cho_last_error()
        raise ChoError(status, msg.decode() if msg else "")
    return status


# ---- array marshalling ---------------------------------------------------------------

def _is_cuda(a):
    return getattr(a, "is_cuda", False)


def _ptr(a):
    if a is None:
        return None
    if _is_cuda(a) or hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr()
    return a.ctypes.data


def _host_f64(a, shape=None):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if shape is not None:
        a = a.reshape(shape)
    return a


def _cuda_f64(a):
    import torch

    if a.dtype != torch.float64:
        raise ValueError("device arrays must be float64")
    return a.contiguous()


def _stream_ptr(stream):
    if stream is not None:
        return getattr(stream, "cuda_stream", stream)
    import torch

    return torch.cuda.current_stream().cuda_stream


# ---- context -----------------------------------------------------------------------

def cho_init(device=0, budget_bytes=0, chunk_steps=0, max_slots=0, chunk_us=0, persistent=0, active_pct=0):
    lib = load()
    ctx = ctypes.c_void_p()
    cfg = cho_config(int(budget_bytes), int(chunk_steps), int(max_slots), int(chunk_us), int(persistent),
                     int(active_pct))
    _check(lib.cho_init(ctypes.byref(ctx), int(device), ctypes.byref(cfg)))
    return ctx


def cho_shutdown(ctx):
    load().cho_shutdown(ctx)


def cho_last_error():
    m = load().cho_last_error()
    return m.decode() if m else ""


# ---- systems -----------------------------------------------------------------------

def cho_create_system(ctx, kind, masses=None, springs=None, M=None, K=None, mass_coupling=None):
    """Create a system from host arrays: masses/springs (n_sys, s) or M/K (n_sys, s, s).
    mass_coupling (n_sys, s), spring kinds only: off-diagonal masses m_{i,i+1} (a tridiagonal
    M; the system is then built as a dense system, see include/cho.h)."""
    kind = KINDS.get(kind, kind)
    keep = []
    if kind == CHO_DENSE:
        M = _host_f64(M)
        K = _host_f64(K)
        if M.ndim == 2:
            M, K = M[None], K[None]
        n_sys, s = M.shape[0], M.shape[-1]
        keep += [M, K]
        d = cho_system_desc(kind, s, n_sys, None, None, M.ctypes.data, K.ctypes.data)
    else:
        masses = np.atleast_2d(_host_f64(masses))
        springs = np.atleast_2d(_host_f64(springs))
        n_sys, s = masses.shape
        keep += [masses, springs]
        mc = None
        if mass_coupling is not None:
            mc = np.atleast_2d(_host_f64(mass_coupling))
            if mc.shape != masses.shape:
                raise ValueError("mass_coupling must have the shape of masses")
            keep.append(mc)
        d = cho_system_desc(kind, s, n_sys, masses.ctypes.data, springs.ctypes.data, None, None,
                            None if mc is None else mc.ctypes.data)
    out = ctypes.c_void_p()
    _check(load().cho_create_system(ctx, ctypes.byref(d), ctypes.byref(out)))
    del keep
    return out


def cho_system_info(system):
    w = ctypes.c_double()
    s = ctypes.c_int32()
    n = ctypes.c_int64()
    _check(load().cho_system_info(system, ctypes.byref(w), ctypes.byref(s), ctypes.byref(n)))
    return w.value, s.value, n.value


def cho_system_omegas(system):
    _, _, n = cho_system_info(system)
    out = np.empty(n)
    _check(load().cho_system_omegas(system, out.ctypes.data_as(_dp)))
    return out


def cho_system_status(system):
    """CHO_OK, or raises ChoError(CHO_ETIMEOUT) if a tensor-core run on the system gave up a wait."""
    return _check(load().cho_system_status(system))


def cho_system_set_damping(system, dampers):
    """A dashpot beside every spring: dampers (n_sys, s) in N s/m, or None to remove them."""
    if dampers is None:
        return _check(load().cho_system_set_damping(system, None))
    d = _host_f64(dampers)
    return _check(load().cho_system_set_damping(system, d.ctypes.data))


def cho_system_set_forcing(system, amplitude, omega=None, phase=None):
    """Harmonic force amplitude_i cos(omega t + phase) on every mass: amplitude (n_sys, s) in N,
    omega and phase (n_sys) or scalars; amplitude None removes the forcing."""
    if amplitude is None:
        return _check(load().cho_system_set_forcing(system, None, None, None))
    _, s, n = cho_system_info(system)
    a = _host_f64(amplitude).reshape(-1)
    w = _host_f64(np.broadcast_to(np.asarray(omega, dtype=np.float64), (n,)))
    p = None if phase is None else _host_f64(np.broadcast_to(np.asarray(phase, dtype=np.float64), (n,)))
    return _check(load().cho_system_set_forcing(system, a.ctypes.data, w.ctypes.data,
                                                None if p is None else p.ctypes.data))


def cho_destroy_system(system):
    load().cho_destroy_system(system)


# ---- batches -----------------------------------------------------------------------

def _batch(fn_name, ctx, system, x0, v0, h, n_steps, prec=CHO_FP64, ckpt_every=0, trajectory=False,
           energy=False, out=None, stream=None, poly_jump=0):
    prec = PRECS.get(prec, prec)
    _, s, _ = cho_system_info(system)
    device = _is_cuda(x0)
    n_ck = n_steps // ckpt_every if ckpt_every else 0
    res = dict(out or {})
    if device:
        import torch

        x0 = _cuda_f64(x0)
        v0 = _cuda_f64(v0)
        n_inst = x0.shape[0] if x0.dim() > 1 else 1
        if not _is_cuda(h):
            h = torch.as_tensor(np.asarray(h, dtype=np.float64).reshape(-1), device=x0.device)
        h = _cuda_f64(h)
        new = lambda *shape: torch.empty(shape, dtype=torch.float64, device=x0.device)  # noqa: E731
        mem = CHO_MEM_DEVICE
    else:
        x0 = _host_f64(x0).reshape(-1, s)
        v0 = _host_f64(v0).reshape(-1, s)
        n_inst = x0.shape[0]
        h = _host_f64(h).reshape(-1)
        new = lambda *shape: np.empty(shape)  # noqa: E731
        mem = CHO_MEM_HOST
    h_per_inst = int(h.shape[0] != 1 or n_inst == 1)
    if h.shape[0] not in (1, n_inst):
        raise ValueError("h must have 1 or n_inst values")
    for k, shape in (("x", (n_inst, s)), ("v", (n_inst, s))):
        if k not in res:
            res[k] = new(*shape)
    if trajectory or energy:
        res.setdefault("x_traj", new(n_inst, n_ck, s))
        res.setdefault("v_traj", new(n_inst, n_ck, s))
    if energy:
        res.setdefault("energy", new(n_inst, n_ck))
    b = cho_batch_desc()
    b.system = system
    b.n_inst = n_inst
    b.prec = prec
    b.mem = mem
    b.x0, b.v0, b.h = _ptr(x0), _ptr(v0), _ptr(h)
    b.h_per_inst = h_per_inst
    b.poly_jump = int(poly_jump)
    b.n_steps = int(n_steps)
    b.ckpt_every = int(ckpt_every)
    b.x_out, b.v_out = _ptr(res["x"]), _ptr(res["v"])
    b.x_traj, b.v_traj = _ptr(res.get("x_traj")), _ptr(res.get("v_traj"))
    b.energy = _ptr(res.get("energy"))
    # host arrays are staged on the caller's stream when one is given (NULL: the default stream)
    st = _stream_ptr(stream) if (device or stream is not None) else None
    _check(getattr(load(), fn_name)(ctx, ctypes.byref(b), st))
    return res


def cho_integrate_batch(ctx, system, x0, v0, h, n_steps, prec=CHO_FP64, ckpt_every=0, trajectory=False,
                        energy=False, out=None, stream=None, poly_jump=0):
    """Integrate a batch (see include/cho.h).  Returns a dict with x, v and, when asked, x_traj,
    v_traj (n_inst, n_steps // ckpt_every, s) and energy (n_inst, n_steps // ckpt_every).
    ``poly_jump`` = k >= 1 selects the polynomial form (k RK4 steps per update, s = 2)."""
    return _batch("cho_integrate_batch", ctx, system, x0, v0, h, n_steps, prec, ckpt_every, trajectory,
                  energy, out, stream, poly_jump)


def cho_integrate_plain(ctx, system, x0, v0, h, n_steps, out=None, stream=None):
    """The plain form: one launch per stage, one system at a time, FP64."""
    return _batch("cho_integrate_plain", ctx, system, x0, v0, h, n_steps, CHO_FP64, 0, False, False,
                  out, stream)


def cho_integrate_plain_noalloc(ctx, system, x0, v0, h, n_steps, out=None, stream=None):
    """The plain form with its scratch in the library's fixed device array (no allocation
    in the call).  Device (CUDA tensor) arrays only; pass ``out`` to avoid the binding
    allocating the result tensors."""
    if not _is_cuda(x0):
        raise ValueError("cho_integrate_plain_noalloc takes device arrays")
    return _batch("cho_integrate_plain_noalloc", ctx, system, x0, v0, h, n_steps, CHO_FP64, 0, False, False,
                  out, stream)


def cho_integrate_packed(ctx, batches, stream=None):
    """Several batches in as few launches as possible (see include/cho.h).  ``batches`` is a
    list of dicts with keys system, x0, v0, h (CUDA tensors; h of 1 or n_inst values),
    n_steps, prec and optionally out ({"x", "v"} tensors).  Returns one {"x", "v"} dict per
    batch."""
    import torch

    descs = (cho_batch_desc * max(1, len(batches)))()
    results, keep = [], []
    for k, bt in enumerate(batches):
        _, s, _ = cho_system_info(bt["system"])
        x0 = _cuda_f64(bt["x0"])
        v0 = _cuda_f64(bt["v0"])
        h = bt["h"]
        if not _is_cuda(h):
            h = torch.as_tensor(np.asarray(h, dtype=np.float64).reshape(-1), device=x0.device)
        h = _cuda_f64(h)
        n_inst = x0.shape[0] if x0.dim() > 1 else 1
        if h.shape[0] not in (1, n_inst):
            raise ValueError("h must have 1 or n_inst values")
        res = dict(bt.get("out") or {})
        for key in ("x", "v"):
            if key not in res:
                res[key] = torch.empty((n_inst, s), dtype=torch.float64, device=x0.device)
        d = descs[k]
        d.system = bt["system"]
        d.n_inst = n_inst
        d.prec = PRECS.get(bt.get("prec", CHO_FP64), bt.get("prec", CHO_FP64))
        d.mem = CHO_MEM_DEVICE
        d.x0, d.v0, d.h = _ptr(x0), _ptr(v0), _ptr(h)
        d.h_per_inst = int(h.shape[0] != 1 or n_inst == 1)
        d.poly_jump = 0
        d.n_steps = int(bt["n_steps"])
        d.ckpt_every = 0
        d.x_out, d.v_out = _ptr(res["x"]), _ptr(res["v"])
        d.x_traj = d.v_traj = d.energy = None
        keep += [x0, v0, h]
        results.append(res)
    st = _stream_ptr(stream)
    _check(load().cho_integrate_packed(ctx, descs, len(batches), st))
    return results


def cho_energy(ctx, system, x, v, stream=None):
    """FP64 energy of states x, v shaped (n_inst, s) or (n_inst, n_per, s)."""
    _, s, _ = cho_system_info(system)
    device = _is_cuda(x)
    if device:
        import torch

        x = _cuda_f64(x)
        v = _cuda_f64(v)
        shape = tuple(x.shape[:-1])
        E = torch.empty(shape, dtype=torch.float64, device=x.device)
        mem = CHO_MEM_DEVICE
    else:
        x = _host_f64(x)
        v = _host_f64(v)
        shape = x.shape[:-1]
        E = np.empty(shape)
        mem = CHO_MEM_HOST
    n_inst = shape[0] if len(shape) else 1
    n_per = shape[1] if len(shape) > 1 else 1
    st = _stream_ptr(stream) if device else None
    _check(load().cho_energy(ctx, system, _ptr(x), _ptr(v), n_inst, n_per, mem, _ptr(E), st))
    return E


# ---- serving -----------------------------------------------------------------------

def cho_submit(ctx, system, x0, v0, h, n_steps, prec=CHO_FP32_KAHAN, priority=2, sys_index=0):
    x0 = _host_f64(x0).reshape(-1)
    v0 = _host_f64(v0).reshape(-1)
    r = cho_request(system, int(sys_index), x0.ctypes.data, v0.ctypes.data, float(h), int(n_steps),
                    PRECS.get(prec, prec), int(priority))
    t = ctypes.c_uint64()
    _check(load().cho_submit(ctx, ctypes.byref(r), ctypes.byref(t)))
    return t.value


def cho_poll(ctx, ticket, s):
    """Returns (status, result) with result = dict(x, v, t_submit, t_admit, t_done) once CHO_OK."""
    x = np.empty(s)
    v = np.empty(s)
    r = cho_result(x.ctypes.data, v.ctypes.data, 0.0, 0.0, 0.0)
    st = load().cho_poll(ctx, ctypes.c_uint64(ticket), ctypes.byref(r))
    if st == CHO_OK:
        return st, {"x": x, "v": v, "t_submit": r.t_submit, "t_admit": r.t_admit, "t_done": r.t_done}
    if st == CHO_PENDING:
        return st, None
    _check(st)
    return st, None


def cho_poll_any(ctx):
    """The next finished request of any ticket: (status, ticket, times) with times a dict of
    t_submit, t_admit, t_done; (CHO_PENDING, None, None) when none is waiting.  Results of
    failed requests come back as their status code, not as an exception."""
    t = ctypes.c_uint64()
    r = cho_result(None, None, 0.0, 0.0, 0.0)
    st = load().cho_poll_any(ctx, ctypes.byref(t), ctypes.byref(r))
    if st == CHO_PENDING:
        return st, None, None
    return st, t.value, {"t_submit": r.t_submit, "t_admit": r.t_admit, "t_done": r.t_done}


def cho_cancel(ctx, ticket):
    return _check(load().cho_cancel(ctx, ctypes.c_uint64(ticket)))


def cho_serve_stats(ctx):
    vals = [ctypes.c_int64() for _ in range(4)]
    _check(load().cho_serve_stats(ctx, *[ctypes.byref(v) for v in vals]))
    return dict(zip(("queued", "resident", "completed", "resident_bytes"), (v.value for v in vals)))


def cho_serve_traffic(ctx):
    """Cumulative chunk-boundary traffic of the serving engine: state bytes read and written
    back by the chunks and the DOF-steps they advanced (include/cho.h)."""
    vals = [ctypes.c_int64() for _ in range(2)]
    _check(load().cho_serve_traffic(ctx, *[ctypes.byref(v) for v in vals]))
    return {"state_bytes": vals[0].value, "dof_steps": vals[1].value}


# ---- autotuning ------------------------------------------------------------------------

def cho_autotune(ctx, system, n_inst, prec=CHO_FP32_KAHAN, poly_jump=0):
    """Time the same-bits kernel variants of a batch shape and record the fastest (see
    include/cho.h).  Returns a dict: variants [(name, code, us_per_step)], chosen (name),
    code and sample_steps."""
    r = cho_tune_result()
    _check(load().cho_autotune(ctx, system, int(n_inst), int(PRECS.get(prec, prec)), int(poly_jump),
                               ctypes.byref(r)))
    variants = [(bytes(r.name[k]).split(b"\0")[0].decode(), int(r.code[k]), float(r.us_per_step[k]))
                for k in range(r.n_variants)]
    return {"variants": variants, "chosen": variants[r.chosen][0], "code": variants[r.chosen][1],
            "sample_steps": int(r.sample_steps)}


def cho_tune_query(ctx, system, n_inst, prec=CHO_FP32_KAHAN, poly_jump=0):
    """The variant code recorded for a batch shape, or -1."""
    code = ctypes.c_int32()
    _check(load().cho_tune_query(ctx, system, int(n_inst), int(PRECS.get(prec, prec)), int(poly_jump),
                                 ctypes.byref(code)))
    return code.value


def cho_tune_save(ctx, path):
    _check(load().cho_tune_save(ctx, os.fsencode(path)))


def cho_tune_load(ctx, path):
    n = ctypes.c_int32()
    _check(load().cho_tune_load(ctx, os.fsencode(path), ctypes.byref(n)))
    return n.value


# ---- measurement -----------------------------------------------------------------------

FMA_KINDS = {"fp32": 0, "fp32x2": 1, "fp64": 2}


def cho_measure_fma_peak(ctx, kind="fp32", iters=20000):
    """Measured FMA throughput of the CUDA cores (see include/cho.h): returns
    (flop/s, seconds of the timed launch)."""
    f, t = ctypes.c_double(), ctypes.c_double()
    _check(load().cho_measure_fma_peak(ctx, int(FMA_KINDS.get(kind, kind)), int(iters), ctypes.byref(f),
                                       ctypes.byref(t)))
    return f.value, t.value
