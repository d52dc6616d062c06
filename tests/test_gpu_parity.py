"""GPU parity: every kernel family against the FP64 oracle on the same seeded inputs.

Error metric (per instance): max over checkpoints of |x_gpu - x_ref|_inf divided by
max over checkpoints of |x_ref|_inf, and the same for v.  Bars: FP64 mode 1e-10,
FP32 + Kahan mode 1e-5.  Checkpoints are every 125 steps: the workloads' step is
T_min/200 or T_min/100, so a stride of 100 steps would sample the fastest mode at
the same phase every time (e.g. always at its turning points, where v ~ 0) and the
normalisation would not see the horizon's true maximum.
"""
import math
import os

import numpy as np
import pytest

from paper_1702_02207_gb300 import cho, inputs
from parity_util import TOL_FP32, TOL_FP64, oracle_run, rel_err, sample_indices

pytestmark = pytest.mark.gpu
ROOT_DIR = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def ctx():
    c = cho.cho_init(0)
    yield c
    cho.cho_shutdown(c)


def make_system(ctx, cfg):
    if cfg["kind"] == "dense":
        return cho.cho_create_system(ctx, "dense", M=cfg["M"], K=cfg["K"])
    return cho.cho_create_system(ctx, cfg["kind"], masses=cfg["masses"], springs=cfg["springs"])


def run_gpu(ctx, cfg, prec, ckpt_every, device=True, n_steps=None):
    import torch

    n_steps = cfg["n_steps"] if n_steps is None else n_steps
    sys_ = make_system(ctx, cfg)
    try:
        if device:
            dev = torch.device("cuda:0")
            x0 = torch.as_tensor(cfg["x0"], device=dev)
            v0 = torch.as_tensor(cfg["v0"], device=dev)
            h = torch.as_tensor(cfg["h"], device=dev)
            out = cho.cho_integrate_batch(ctx, sys_, x0, v0, h, n_steps, prec, ckpt_every,
                                          trajectory=ckpt_every > 0)
            torch.cuda.synchronize()
            out = {k: v.cpu().numpy() for k, v in out.items()}
        else:
            out = cho.cho_integrate_batch(ctx, sys_, cfg["x0"], cfg["v0"], cfg["h"], n_steps, prec,
                                          ckpt_every, trajectory=ckpt_every > 0)
    finally:
        cho.cho_destroy_system(sys_)
    return out


def check(out, ref, tol, idx=None):
    sel = slice(None) if idx is None else idx
    ex = rel_err(out["x_traj"][sel], ref["x_traj"])
    ev = rel_err(out["v_traj"][sel], ref["v_traj"])
    assert np.all(np.isfinite(out["x"][sel]))
    assert ex.max() <= tol, (ex.max(), int(np.argmax(ex)))
    assert ev.max() <= tol, (ev.max(), int(np.argmax(ev)))
    return ex.max(), ev.max()


# ---- eq. 3 (the paper's 2-DOF example) -----------------------------------------------

def test_eq3_fp64_full_horizon(ctx):
    cfg = inputs.eq3_single()
    out = run_gpu(ctx, cfg, "fp64", 1000)
    ref = oracle_run(cfg, ckpt_every=1000)
    check(out, ref, TOL_FP64)
    assert np.allclose(out["x"][0], [0.5919944669044028, -0.55303750830408224], atol=1e-10)


@pytest.mark.parametrize("x0", [(2.0, -3.0)])
def test_eq3_fig2_start_fp32(ctx, x0):
    cfg = inputs.eq3_single(x0)
    cfg["n_steps"] = 20_000
    out = run_gpu(ctx, cfg, "fp32_kahan", 200)
    ref = oracle_run(cfg, ckpt_every=200)
    check(out, ref, TOL_FP32)


# ---- eq. 2 batches --------------------------------------------------------------------

@pytest.mark.parametrize("prec,tol", [("fp64", TOL_FP64), ("fp32_kahan", TOL_FP32)])
@pytest.mark.parametrize("n_inst", [1, 7, 1000])
def test_two_dof_batch_ragged(ctx, prec, tol, n_inst):
    cfg = inputs.two_dof_batch(n_inst=n_inst, n_steps=10_000)
    out = run_gpu(ctx, cfg, prec, 125)
    ref = oracle_run(cfg, ckpt_every=125)
    check(out, ref, tol)


@pytest.mark.parametrize("prec,tol", [("fp32_kahan", TOL_FP32), ("fp64", TOL_FP64)])
def test_two_dof_full_size_sampled(ctx, prec, tol):
    """65,536 systems x 1e4 steps in one launch (the benchmark's configuration), sampled."""
    cfg = inputs.two_dof_batch()
    out = run_gpu(ctx, cfg, prec, 125)
    idx = sample_indices(cfg["x0"].shape[0], 256)
    ref = oracle_run(cfg, idx=idx, ckpt_every=125)
    check(out, ref, tol, idx)


def test_host_and_device_memory_agree(ctx):
    cfg = inputs.two_dof_batch(n_inst=300, n_steps=2000)
    a = run_gpu(ctx, cfg, "fp32_kahan", 125, device=True)
    b = run_gpu(ctx, cfg, "fp32_kahan", 125, device=False)
    assert np.array_equal(a["x"], b["x"]) and np.array_equal(a["v_traj"], b["v_traj"])


@pytest.mark.parametrize("case", ["two_dof", "chain", "dense_tc", "dense_simt"])
def test_pinned_and_pageable_host_arrays_agree_with_device_arrays(ctx, case):
    """Host arrays, page-locked (as the benchmark's end-to-end call passes them) or pageable,
    are staged through the context's workspace: the results, trajectories and energies are
    bitwise those of device arrays, for every kernel family."""
    import torch

    if case == "two_dof":
        cfg, prec = inputs.two_dof_batch(n_inst=5000, n_steps=400), "fp32_kahan"
    elif case == "chain":
        cfg, prec = inputs.chain_batch(n_inst=9, s=300, n_steps=400, seed=301), "fp32_kahan"
    elif case == "dense_tc":
        cfg, prec = inputs.dense_group(s=128, n_inst=70, n_steps=400, seed=128), "bf16x5"
    else:
        cfg, prec = inputs.dense_group(s=100, n_inst=20, n_steps=400, seed=100), "fp32_simt"
    sys_ = make_system(ctx, cfg)
    d = torch.device("cuda:0")
    try:
        n, s = cfg["x0"].shape
        h = np.asarray(cfg["h"], dtype=np.float64).reshape(-1)
        energy = case != "dense_tc"
        ref = cho.cho_integrate_batch(ctx, sys_, torch.as_tensor(cfg["x0"], device=d),
                                      torch.as_tensor(cfg["v0"], device=d), torch.as_tensor(h, device=d), 400, prec,
                                      100, trajectory=True, energy=energy)
        pin = lambda a: torch.as_tensor(np.ascontiguousarray(a)).pin_memory()  # noqa: E731
        out = {"x": pin(np.zeros((n, s))), "v": pin(np.zeros((n, s))), "x_traj": pin(np.zeros((n, 4, s))),
               "v_traj": pin(np.zeros((n, 4, s)))}
        if energy:
            out["energy"] = pin(np.zeros((n, 4)))
        got = cho.cho_integrate_batch(ctx, sys_, pin(cfg["x0"]), pin(cfg["v0"]), pin(h), 400, prec, 100,
                                      trajectory=True, energy=energy, out=out)
        staged = cho.cho_integrate_batch(ctx, sys_, cfg["x0"], cfg["v0"], h, 400, prec, 100, trajectory=True,
                                         energy=energy)
        for key in ("x", "v", "x_traj", "v_traj") + (("energy",) if energy else ()):
            r = ref[key].cpu().numpy()
            assert np.array_equal(np.asarray(got[key]), r), key
            assert np.array_equal(np.asarray(staged[key]), r), key
    finally:
        cho.cho_destroy_system(sys_)


# ---- small systems (rk4_small) ----------------------------------------------------------

@pytest.mark.parametrize("s", [1, 3, 4, 5, 8, 9, 16, 17, 31, 32])
@pytest.mark.parametrize("prec,tol", [("fp64", TOL_FP64), ("fp32_kahan", TOL_FP32)])
def test_small_chains(ctx, s, prec, tol):
    cfg = inputs.chain_batch(n_inst=37, s=s, n_steps=3000, seed=500 + s)
    out = run_gpu(ctx, cfg, prec, 125)
    ref = oracle_run(cfg, ckpt_every=125)
    check(out, ref, tol)


def dense_per_instance(s, n_inst, seed, n_steps=2000):
    rng = np.random.default_rng(seed)
    Ms, Ks = [], []
    for i in range(n_inst):
        M, K, _, _ = inputs.dense_system(s, seed * 1000 + i)
        Ms.append(M)
        Ks.append(K)
    M = np.stack(Ms)
    K = np.stack(Ks)
    w = inputs.omega_max_dense(M, K)
    h = inputs.fp32_exact(2 * math.pi / w / 100)
    return {"kind": "dense", "s": s, "M": M, "K": K, "x0": rng.normal(size=(n_inst, s)),
            "v0": np.zeros((n_inst, s)), "h": h, "n_steps": n_steps}


@pytest.mark.parametrize("s", [2, 6, 8, 13, 32])
@pytest.mark.parametrize("prec,tol", [("fp64", TOL_FP64), ("fp32_kahan", TOL_FP32)])
def test_small_dense_per_instance(ctx, s, prec, tol):
    cfg = dense_per_instance(s, 21, 40 + s)
    out = run_gpu(ctx, cfg, prec, 125)
    ref = oracle_run(cfg, ckpt_every=125)
    check(out, ref, tol)


# ---- chains (rk4_chain) -----------------------------------------------------------------

@pytest.mark.parametrize("s", [33, 64, 255, 256, 257, 1023, 1024, 1025, 2100])
@pytest.mark.parametrize("prec,tol", [("fp64", TOL_FP64), ("fp32_kahan", TOL_FP32)])
def test_chains(ctx, s, prec, tol):
    n_inst = 7 if s < 2000 else 2
    cfg = inputs.chain_batch(n_inst=n_inst, s=s, n_steps=2000, seed=900 + s)
    out = run_gpu(ctx, cfg, prec, 125)
    ref = oracle_run(cfg, ckpt_every=125)
    check(out, ref, tol)


def test_chain_full_size_sampled_fp32(ctx):
    """4096 chains of 1024 masses x 1e4 steps, FP32 + Kahan, sampled against the oracle."""
    cfg = inputs.chain_batch()
    out = run_gpu(ctx, cfg, "fp32_kahan", 625)
    idx = sample_indices(cfg["x0"].shape[0], 12)
    ref = oracle_run(cfg, idx=idx, ckpt_every=625)
    check(out, ref, TOL_FP32, idx)


# ---- dense shared systems (rk4_dense, CUDA cores) -----------------------------------------

@pytest.mark.parametrize("s", [33, 64, 100, 128, 256])
@pytest.mark.parametrize("prec,tol", [("fp64", TOL_FP64), ("fp32_simt", TOL_FP32), ("fp32_kahan", TOL_FP32)])
def test_dense_shared(ctx, s, prec, tol):
    cfg = inputs.dense_group(s=s, n_inst=37, n_steps=1000)
    out = run_gpu(ctx, cfg, prec, 125)
    ref = oracle_run(cfg, ckpt_every=125)
    check(out, ref, tol)


# ---- energy -----------------------------------------------------------------------------

def test_energy_matches_oracle(ctx):
    import oracle

    cfg = inputs.two_dof_batch(n_inst=50, n_steps=1000)
    sys_ = make_system(ctx, cfg)
    try:
        out = cho.cho_integrate_batch(ctx, sys_, cfg["x0"], cfg["v0"], cfg["h"], 1000, "fp64", 100, energy=True)
    finally:
        cho.cho_destroy_system(sys_)
    n_ck = out["x_traj"].shape[1]
    E_ref = oracle.energy_chain(np.repeat(cfg["masses"], n_ck, 0), np.repeat(cfg["springs"], n_ck, 0),
                                out["x_traj"].reshape(-1, 2), out["v_traj"].reshape(-1, 2)).reshape(50, n_ck)
    assert np.allclose(out["energy"], E_ref, rtol=1e-13)


def test_energy_dense_and_chain_api(ctx):
    import oracle

    cfg = inputs.dense_group(s=64, n_inst=9, n_steps=10)
    sys_ = make_system(ctx, cfg)
    try:
        rng = np.random.default_rng(1)
        x = rng.normal(size=(9, 64))
        v = rng.normal(size=(9, 64))
        E = cho.cho_energy(ctx, sys_, x, v)
    finally:
        cho.cho_destroy_system(sys_)
    assert np.allclose(E, oracle.energy_dense(cfg["M"][0], cfg["K"][0], x, v), rtol=1e-13)
    cfg = inputs.chain_batch(n_inst=5, s=300)
    sys_ = make_system(ctx, cfg)
    try:
        E = cho.cho_energy(ctx, sys_, cfg["x0"], cfg["x0"])
    finally:
        cho.cho_destroy_system(sys_)
    assert np.allclose(E, oracle.energy_chain(cfg["masses"], cfg["springs"], cfg["x0"], cfg["x0"]), rtol=1e-13)


def test_energy_drift_config1_on_gpu(ctx):
    """GPU FP64 energy after 1e5 steps of eq. 3 shows RK4's drift -2.4508e-11."""
    cfg = inputs.eq3_single()
    sys_ = make_system(ctx, cfg)
    try:
        out = cho.cho_integrate_batch(ctx, sys_, cfg["x0"], cfg["v0"], cfg["h"], cfg["n_steps"], "fp64",
                                      cfg["n_steps"], energy=True)
    finally:
        cho.cho_destroy_system(sys_)
    drift = (out["energy"][0, -1] - 2025.0) / 2025.0
    assert drift == pytest.approx(-2.4508e-11, rel=2e-3)


# ---- plain form --------------------------------------------------------------------------

@pytest.mark.parametrize("kind", ["two_dof", "chain", "dense"])
def test_plain_form_matches_oracle(ctx, kind):
    if kind == "two_dof":
        cfg = inputs.two_dof_batch(n_inst=3, n_steps=300)
    elif kind == "chain":
        cfg = inputs.chain_batch(n_inst=2, s=300, n_steps=200)
    else:
        cfg = inputs.dense_group(s=40, n_inst=2, n_steps=200)
    sys_ = make_system(ctx, cfg)
    try:
        out = cho.cho_integrate_plain(ctx, sys_, cfg["x0"], cfg["v0"], cfg["h"], cfg["n_steps"])
    finally:
        cho.cho_destroy_system(sys_)
    ref = oracle_run(cfg)
    assert rel_err(out["x"][:, None], ref["x"][:, None]).max() < TOL_FP64


# ---- edge cases and errors ----------------------------------------------------------------

def test_zero_steps_and_zero_instances(ctx):
    cfg = inputs.chain_batch(n_inst=4, s=40, n_steps=0)
    out = run_gpu(ctx, cfg, "fp64", 0, n_steps=0)
    assert np.array_equal(out["x"], cfg["x0"]) and np.array_equal(out["v"], cfg["v0"])
    out = run_gpu(ctx, cfg, "fp32_kahan", 0, n_steps=0)
    # FP32 value plus FP32 compensation carry the FP64 input to about 2^-48
    assert np.allclose(out["x"], cfg["x0"], rtol=2e-14, atol=0)
    sys_ = make_system(ctx, inputs.chain_batch(n_inst=1, s=40))
    try:
        r = cho.cho_integrate_batch(ctx, sys_, np.zeros((0, 40)), np.zeros((0, 40)), [1e-3], 10)
        assert r["x"].shape == (0, 40)
    finally:
        cho.cho_destroy_system(sys_)


def test_resume_is_bitwise_in_fp64(ctx):
    cfg = inputs.chain_batch(n_inst=5, s=50, n_steps=400, seed=77)
    full = run_gpu(ctx, cfg, "fp64", 0)
    half = run_gpu(ctx, cfg, "fp64", 0, n_steps=200)
    cfg2 = dict(cfg, x0=half["x"], v0=half["v"])
    rest = run_gpu(ctx, cfg2, "fp64", 0, n_steps=200)
    assert np.array_equal(rest["x"], full["x"]) and np.array_equal(rest["v"], full["v"])


def test_errors_are_reported(ctx):
    with pytest.raises(cho.ChoError) as ei:
        cho.cho_create_system(ctx, "chain", masses=[[1.0, -1.0]], springs=[[1.0, 1.0]])
    assert ei.value.status == cho.CHO_EINVAL
    with pytest.raises(cho.ChoError) as ei:
        cho.cho_create_system(ctx, "dense", M=[[1.0, 2.0], [2.0, 1.0]], K=np.eye(2))
    assert ei.value.status == cho.CHO_ENOTSPD
    with pytest.raises(cho.ChoError) as ei:
        cho.cho_create_system(ctx, "two_dof", masses=[[1.0, 1.0, 1.0]], springs=[[1.0, 1.0, 1.0]])
    assert ei.value.status == cho.CHO_EINVAL
    cfg = inputs.eq3_single()
    sys_ = make_system(ctx, cfg)
    try:
        w, s, n = cho.cho_system_info(sys_)
        assert (s, n) == (2, 1)
        assert w == pytest.approx(math.sqrt(1012.5 * (3 + math.sqrt(5)) / 2), rel=1e-12)
        with pytest.raises(cho.ChoError) as ei:      # |omega h| > 2 sqrt 2
            cho.cho_integrate_batch(ctx, sys_, cfg["x0"], cfg["v0"], [3.0 / w], 10)
        assert ei.value.status == cho.CHO_EUNSTABLE
        with pytest.raises(cho.ChoError) as ei:
            cho.cho_integrate_batch(ctx, sys_, cfg["x0"], cfg["v0"], cfg["h"], 10, ckpt_every=3)
        assert ei.value.status == cho.CHO_EINVAL
        with pytest.raises(cho.ChoError) as ei:
            cho.cho_integrate_batch(ctx, sys_, cfg["x0"], cfg["v0"], cfg["h"], 10, prec="bf16x3")
        assert ei.value.status == cho.CHO_EINVAL
    finally:
        cho.cho_destroy_system(sys_)


def test_omega_max_matches_library_eigensolvers(ctx):
    cfg = inputs.chain_batch(n_inst=3, s=200)
    sys_ = make_system(ctx, cfg)
    try:
        assert np.allclose(cho.cho_system_omegas(sys_), cfg["omega_max"], rtol=1e-12)
    finally:
        cho.cho_destroy_system(sys_)
    cfg = inputs.dense_group(s=96, n_inst=1)
    sys_ = make_system(ctx, cfg)
    try:
        assert cho.cho_system_info(sys_)[0] == pytest.approx(cfg["omega_max"], rel=1e-10)
    finally:
        cho.cho_destroy_system(sys_)


# ---- dense shared systems on the tensor cores (split BF16) ---------------------------------

# bf16x3 drops the 2^-16-relative partial products, so its error is stated, not 1e-5:
# about n * theta * 2^-16 of phase after n steps of angle theta (1e-3 at 1000 steps here).
TOL_BF16 = {"bf16x3": 3e-3, "bf16x5": TOL_FP32, "bf16x6": TOL_FP32}


def test_dense_tensor_core_first_light(ctx):
    """One tile, s = 128, a few steps: the tensor-core path agrees with the FP32 CUDA-core path."""
    cfg = inputs.dense_group(s=128, n_inst=32, n_steps=10)
    simt = run_gpu(ctx, cfg, "fp32_simt", 0)
    tc = run_gpu(ctx, cfg, "bf16x5", 0)
    assert rel_err(tc["x"][:, None], simt["x"][:, None]).max() < 1e-5


@pytest.mark.parametrize("s", [33, 64, 100, 128, 129, 200, 256])
@pytest.mark.parametrize("prec", ["bf16x3", "bf16x5", "bf16x6"])
def test_dense_tensor_core(ctx, s, prec):
    if prec == "bf16x6" and s > 128:
        cfg = inputs.dense_group(s=s, n_inst=3, n_steps=10)
        with pytest.raises(cho.ChoError) as ei:
            run_gpu(ctx, cfg, prec, 0)
        assert ei.value.status == cho.CHO_EINVAL
        return
    cfg = inputs.dense_group(s=s, n_inst=45, n_steps=1000)
    out = run_gpu(ctx, cfg, prec, 125)
    ref = oracle_run(cfg, ckpt_every=125)
    ex, ev = check(out, ref, TOL_BF16[prec])
    print(f"dense s={s} {prec}: max rel err x {ex:.3e} v {ev:.3e}")


def test_two_dof_kernel_variants_are_bitwise_equal(tmp_path):
    """The pair-packed and generic 2-DOF FP32 kernels round identically."""
    import subprocess
    import sys as _sys

    code = (
        "import sys, numpy as np, torch\n"
        "sys.path.insert(0, %r)\n"
        "from paper_1702_02207_gb300 import cho, inputs\n"
        "cfg = inputs.two_dof_batch(n_inst=999, n_steps=3000)\n"
        "ctx = cho.cho_init(0)\n"
        "s = cho.cho_create_system(ctx, 'two_dof', masses=cfg['masses'], springs=cfg['springs'])\n"
        "d = torch.device('cuda:0')\n"
        "o = cho.cho_integrate_batch(ctx, s, torch.as_tensor(cfg['x0'], device=d), torch.as_tensor(cfg['v0'], device=d),"
        " torch.as_tensor(cfg['h'], device=d), 3000, 'fp32_kahan', 1000, trajectory=True)\n"
        "torch.cuda.synchronize()\n"
        "np.savez(sys.argv[1], **{k: v.cpu().numpy() for k, v in o.items()})\n"
    ) % ROOT_DIR
    res = {}
    for variant in ("pair", "generic"):
        path = str(tmp_path / f"{variant}.npz")
        env = dict(os.environ, CHO_TWO_DOF_KERNEL=variant)
        subprocess.run([_sys.executable, "-c", code, path], check=True, env=env, timeout=300)
        res[variant] = np.load(path)
    for variant in ("generic",):
        for k in ("x", "v", "x_traj", "v_traj"):
            assert np.array_equal(res["pair"][k], res[variant][k]), (variant, k)


_VARIANT_RUN = (
    "import sys, numpy as np, torch\n"
    "sys.path.insert(0, %r)\n"
    "from paper_1702_02207_gb300 import cho, inputs\n"
    "n_inst, n_steps, every = int(sys.argv[2]), int(sys.argv[3]), int(sys.argv[4])\n"
    "cfg = inputs.two_dof_batch(n_inst=n_inst, n_steps=n_steps)\n"
    "ctx = cho.cho_init(0)\n"
    "s = cho.cho_create_system(ctx, 'two_dof', masses=cfg['masses'], springs=cfg['springs'])\n"
    "d = torch.device('cuda:0')\n"
    "o = cho.cho_integrate_batch(ctx, s, torch.as_tensor(cfg['x0'], device=d), torch.as_tensor(cfg['v0'], device=d),"
    " torch.as_tensor(cfg['h'], device=d), n_steps, 'fp32_kahan', every, trajectory=every > 0)\n"
    "torch.cuda.synchronize()\n"
    "assert cho.cho_system_status(s) == cho.CHO_OK\n"
    "np.savez(sys.argv[1], **{k: v.cpu().numpy() for k, v in o.items()})\n"
) % ROOT_DIR


@pytest.mark.parametrize("n_inst,n_steps,every", [(45001, 3000, 1000), (45001, 3000, 0), (38913, 7, 0),
                                                  (100000, 13, 0)])
def test_two_dof_balanced_schedule_is_bitwise_equal(tmp_path, n_inst, n_steps, every):
    """The balanced schedule (instances' horizons cut between warps, state handed over through
    global memory) gives the same bits as one warp per 64 instances: ragged last unit, odd
    instance count, hand-over at checkpoint blocks and at single steps."""
    import subprocess
    import sys as _sys

    res = {}
    for variant in ("balanced", "pair"):
        path = str(tmp_path / f"{variant}.npz")
        env = dict(os.environ, CHO_TWO_DOF_KERNEL=variant)
        subprocess.run([_sys.executable, "-c", _VARIANT_RUN, path, str(n_inst), str(n_steps), str(every)],
                       check=True, env=env, timeout=300)
        res[variant] = np.load(path)
    for k in res["pair"].files:
        assert np.isfinite(res["balanced"][k]).all(), k
        assert np.array_equal(res["pair"][k], res["balanced"][k]), k


def test_balanced_handover_wait_gives_up_and_reports(ctx):
    """Test hook CHO_TEST_WITHHOLD_HANDOVER=1: no warp publishes its hand-over, every wait runs
    out (after about a second), the units concerned finish as NaN, the call reports
    CHO_ETIMEOUT, and the context stays usable."""
    import torch

    cfg = inputs.two_dof_batch(n_inst=45001, n_steps=300)
    sys_ = make_system(ctx, cfg)
    d = torch.device("cuda:0")
    try:
        os.environ["CHO_TEST_WITHHOLD_HANDOVER"] = "1"
        try:
            with pytest.raises(cho.ChoError) as ei:
                cho.cho_integrate_batch(ctx, sys_, cfg["x0"], cfg["v0"], cfg["h"], 300, "fp32_kahan")
            assert ei.value.status == cho.CHO_ETIMEOUT
            o = cho.cho_integrate_batch(ctx, sys_, torch.as_tensor(cfg["x0"], device=d),
                                        torch.as_tensor(cfg["v0"], device=d), torch.as_tensor(cfg["h"], device=d),
                                        300, "fp32_kahan")
            with pytest.raises(cho.ChoError) as ei:
                cho.cho_system_status(sys_)
            assert ei.value.status == cho.CHO_ETIMEOUT
            assert np.isnan(o["x"].cpu().numpy()).any()
        finally:
            del os.environ["CHO_TEST_WITHHOLD_HANDOVER"]
        assert cho.cho_system_status(sys_) == cho.CHO_OK
        out = cho.cho_integrate_batch(ctx, sys_, cfg["x0"], cfg["v0"], cfg["h"], 300, "fp32_kahan")
        idx = sample_indices(45001, 64)
        ref = oracle_run(cfg, idx=idx)
        assert rel_err(out["x"][idx][:, None], ref["x"][:, None]).max() < TOL_FP32
    finally:
        cho.cho_destroy_system(sys_)


# ---- dense systems with one (M, K) per instance (CUDA cores) ----------------------------------

@pytest.mark.parametrize("s", [33, 64, 100, 128, 256, 300])
@pytest.mark.parametrize("prec,tol", [("fp64", TOL_FP64), ("fp32_kahan", TOL_FP32)])
def test_dense_per_instance(ctx, s, prec, tol):
    """Seven instances, each with its own M and K (and its own h = T_min/100), 1000 steps."""
    cfg = inputs.dense_own(s=s, n_inst=7, n_steps=1000)
    out = run_gpu(ctx, cfg, prec, 125)
    ref = oracle_run(cfg, ckpt_every=125)
    ex, ev = check(out, ref, tol)
    print(f"dense own-K s={s} {prec}: x {ex:.3e} v {ev:.3e}")


def _beyond_few(s, sms):
    """An instance count above what the FP32 few-instance dense kernels take (eight waves of
    one instance per CTA at s_pad = 64, one per SM; at 128, at most two per SM; per 2- or 8-CTA
    cluster at 256 and 512), so that the streaming kernel runs it."""
    sp = 64
    while sp < s:
        sp *= 2
    return 8 * {64: sms, 128: 2 * sms, 256: sms // 2, 512: sms // 8}[sp] + 5


@pytest.mark.parametrize("s", [64, 100, 200, 333, 512])
def test_dense_few_instances_same_bits_as_many(ctx, s):
    """A few instances of a shared dense system run one per CTA (s_pad = 64: B resident) or
    one per cluster of CTAs (larger s: B's rows split over the cluster, stage displacements
    exchanged through distributed shared memory); many instances run on the streaming
    kernel.  All FP32 dense kernels sum the products in the same order, so the shared
    instances agree bit for bit, trajectories included, and with the oracle."""
    import torch

    sms = torch.cuda.get_device_properties(0).multi_processor_count
    many = _beyond_few(s, sms)
    cfg = inputs.dense_group(s=s, n_inst=many, n_steps=400)
    few = dict(cfg, x0=cfg["x0"][:3], v0=cfg["v0"][:3], h=cfg["h"][:3])
    out_few = run_gpu(ctx, few, "fp32_kahan", 100)
    out_many = run_gpu(ctx, cfg, "fp32_kahan", 100)
    for k in ("x", "v", "x_traj", "v_traj"):
        assert np.array_equal(out_few[k], out_many[k][:3]), k
    ref = oracle_run(few, ckpt_every=100)
    ex, ev = check(out_few, ref, TOL_FP32)
    print(f"dense few-instance s={s}: x {ex:.3e} v {ev:.3e}")


@pytest.mark.parametrize("s", [100, 300])
def test_dense_per_instance_same_bits_as_shared(ctx, s):
    """Instance i of a system with one (M, K) per instance (cluster kernel) gives the bits of
    the same instance in a large batch of a shared system built from its M and K (streaming
    kernel)."""
    import torch

    cfg = inputs.dense_own(s=s, n_inst=3, n_steps=300)
    out = run_gpu(ctx, cfg, "fp32_kahan", 100)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    many = _beyond_few(s, sms)
    i = 1
    shared = dict(kind="dense", s=s, M=cfg["M"][i:i + 1], K=cfg["K"][i:i + 1],
                  x0=np.repeat(cfg["x0"][i:i + 1], many, 0), v0=np.repeat(cfg["v0"][i:i + 1], many, 0),
                  h=np.full(many, cfg["h"][i]), n_steps=300)
    out_sh = run_gpu(ctx, shared, "fp32_kahan", 100)
    for k in ("x", "v", "x_traj", "v_traj"):
        assert np.array_equal(out[k][i], out_sh[k][0]), k
        assert np.array_equal(out_sh[k][0], out_sh[k][many - 1]), k


def test_dense_per_instance_energy_and_errors(ctx):
    """FP64 energy per checkpoint from each instance's own M and K; BF16 modes are refused."""
    import oracle

    cfg = inputs.dense_own(s=48, n_inst=3, n_steps=500)
    sys_ = make_system(ctx, cfg)
    try:
        out = cho.cho_integrate_batch(ctx, sys_, cfg["x0"], cfg["v0"], cfg["h"], 500, "fp64", 100, energy=True)
        for i in range(3):
            e_ref = oracle.energy_dense(cfg["M"][i], cfg["K"][i], out["x_traj"][i], out["v_traj"][i])
            assert np.allclose(out["energy"][i], e_ref, rtol=1e-12)
        for prec in ("bf16x3", "bf16x5"):
            with pytest.raises(cho.ChoError) as ei:
                cho.cho_integrate_batch(ctx, sys_, cfg["x0"], cfg["v0"], cfg["h"], 10, prec)
            assert ei.value.status == cho.CHO_EINVAL
    finally:
        cho.cho_destroy_system(sys_)


# ---- damped and forced spring systems (rk4_chain_ext) -------------------------------------------

def _damped_forced_case(s, n_inst, n_steps, seed, damped, forced):
    cfg = inputs.chain_batch(n_inst=n_inst, s=s, n_steps=n_steps, seed=seed)
    if s == 2:
        cfg["kind"] = "two_dof"
    rng = np.random.default_rng(seed + 1)
    m, C = cfg["masses"], cfg["springs"]
    ext = {"dampers": None, "force_amp": None, "force_omega": None, "force_phase": None}
    if damped:       # damping ratios of a few percent
        ext["dampers"] = 0.04 * np.sqrt(C * m) * rng.uniform(0.5, 2.0, C.shape)
    if forced:
        ext["force_amp"] = C * rng.normal(0.0, 0.01, C.shape)
        ext["force_omega"] = cfg["omega_max"] * rng.uniform(0.05, 0.5, n_inst)
        ext["force_phase"] = rng.uniform(-np.pi, np.pi, n_inst)
    return cfg, ext


def _run_ext(ctx, cfg, ext, prec, every):
    import torch

    sys_ = cho.cho_create_system(ctx, cfg["kind"], masses=cfg["masses"], springs=cfg["springs"])
    try:
        if ext["dampers"] is not None:
            cho.cho_system_set_damping(sys_, ext["dampers"])
        if ext["force_amp"] is not None:
            cho.cho_system_set_forcing(sys_, ext["force_amp"], ext["force_omega"], ext["force_phase"])
        d = torch.device("cuda:0")
        out = cho.cho_integrate_batch(ctx, sys_, torch.as_tensor(cfg["x0"], device=d),
                                      torch.as_tensor(cfg["v0"], device=d), torch.as_tensor(cfg["h"], device=d),
                                      cfg["n_steps"], prec, every, trajectory=True)
        torch.cuda.synchronize()
        return {k: v.cpu().numpy() for k, v in out.items()}
    finally:
        cho.cho_destroy_system(sys_)


@pytest.mark.parametrize("s", [1, 2, 3, 64, 300, 513, 1024])
@pytest.mark.parametrize("mode", ["damped", "forced", "both"])
@pytest.mark.parametrize("prec,tol", [("fp64", TOL_FP64), ("fp32_kahan", TOL_FP32)])
def test_damped_forced_chain_matches_oracle(ctx, s, mode, prec, tol):
    import oracle

    cfg, ext = _damped_forced_case(s, 5, 2000, 500 + s, mode != "forced", mode != "damped")
    out = _run_ext(ctx, cfg, ext, prec, 125)
    ref = oracle.rk4_chain_ext(cfg["masses"], cfg["springs"], cfg["x0"], cfg["v0"], cfg["h"], cfg["n_steps"], 125,
                               threads=5, **ext)
    ex, ev = check(out, ref, tol)
    print(f"{mode} s={s} {prec}: x {ex:.3e} v {ev:.3e}")


def test_damping_and_forcing_api(ctx):
    """Removing damping and forcing gives back the undamped kernels' bits; what the extended
    model does not cover is refused with CHO_EINVAL."""
    cfg, ext = _damped_forced_case(8, 3, 200, 77, True, True)
    plain = cho.cho_create_system(ctx, "chain", masses=cfg["masses"], springs=cfg["springs"])
    sys_ = cho.cho_create_system(ctx, "chain", masses=cfg["masses"], springs=cfg["springs"])
    dn = inputs.dense_group(s=40, n_inst=1, n_steps=1)
    dense = cho.cho_create_system(ctx, "dense", M=dn["M"], K=dn["K"])
    try:
        ref = cho.cho_integrate_batch(ctx, plain, cfg["x0"], cfg["v0"], cfg["h"], 200, "fp32_kahan")
        cho.cho_system_set_damping(sys_, ext["dampers"])
        cho.cho_system_set_forcing(sys_, ext["force_amp"], ext["force_omega"], ext["force_phase"])
        moved = cho.cho_integrate_batch(ctx, sys_, cfg["x0"], cfg["v0"], cfg["h"], 200, "fp32_kahan")
        assert not np.array_equal(moved["x"], ref["x"])
        for call in (lambda: cho.cho_integrate_batch(ctx, sys_, cfg["x0"], cfg["v0"], cfg["h"], 200, "fp32_kahan",
                                                     poly_jump=1),
                     lambda: cho.cho_submit(ctx, sys_, cfg["x0"][0], cfg["v0"][0], float(cfg["h"][0]), 10),
                     lambda: cho.cho_system_set_damping(dense, np.ones((1, 40))),
                     lambda: cho.cho_system_set_damping(sys_, -np.ones((3, 8))),
                     lambda: cho.cho_system_set_forcing(sys_, np.full((3, 8), np.nan), 1.0)):
            with pytest.raises(cho.ChoError) as ei:
                call()
            assert ei.value.status == cho.CHO_EINVAL
        cho.cho_system_set_damping(sys_, None)
        cho.cho_system_set_forcing(sys_, None)
        back = cho.cho_integrate_batch(ctx, sys_, cfg["x0"], cfg["v0"], cfg["h"], 200, "fp32_kahan")
        assert np.array_equal(back["x"], ref["x"]) and np.array_equal(back["v"], ref["v"])
    finally:
        for sy in (plain, sys_, dense):
            cho.cho_destroy_system(sy)


# ---- polynomial form (k RK4 steps per update with P(hA)^k) ---------------------------------------

@pytest.mark.parametrize("prec,tol,k", [("fp32_kahan", TOL_FP32, 1), ("fp32_kahan", TOL_FP32, 5),
                                        ("fp32_kahan", TOL_FP32, 25), ("fp64", TOL_FP64, 1),
                                        ("fp64", TOL_FP64, 5), ("fp64", TOL_FP64, 125)])
def test_poly_form_matches_oracle(ctx, prec, tol, k):
    """y <- y + (P(hA)^k - I) y reproduces the stage-by-stage FP64 oracle (999 systems, odd count).
    FP32 stays within 1e-5 while k omega h <= 1 (here k <= 25 at h = T_min/200); at k = 125
    (k omega h = 3.9) the increment E y is as large as y and its rounding reached 1.2e-5."""
    import torch

    cfg = inputs.two_dof_batch(n_inst=999, n_steps=10000)
    sys_ = make_system(ctx, cfg)
    d = torch.device("cuda:0")
    try:
        out = cho.cho_integrate_batch(ctx, sys_, torch.as_tensor(cfg["x0"], device=d),
                                      torch.as_tensor(cfg["v0"], device=d), torch.as_tensor(cfg["h"], device=d),
                                      10000, prec, 125, trajectory=True, poly_jump=k)
        torch.cuda.synchronize()
        out = {key: val.cpu().numpy() for key, val in out.items()}
    finally:
        cho.cho_destroy_system(sys_)
    ref = oracle_run(cfg, ckpt_every=125)
    ex, ev = check(out, ref, tol)
    print(f"poly k={k} {prec}: x {ex:.3e} v {ev:.3e}")


@pytest.mark.parametrize("s", [1, 3, 8, 17, 32])
@pytest.mark.parametrize("kind", ["chain", "dense_own", "dense_shared"])
@pytest.mark.parametrize("prec,tol,k", [("fp64", TOL_FP64, 1), ("fp64", TOL_FP64, 25), ("fp64", TOL_FP64, 125),
                                        ("fp32_kahan", TOL_FP32, 1), ("fp32_kahan", TOL_FP32, 5)])
def test_poly_form_small_systems(ctx, s, kind, prec, tol, k):
    """Systems of s <= 32 other than s = 2 in the polynomial form: a 2S x 2S jump matrix per
    instance (chains and dense systems with their own parameters and h) or one for the batch
    (a shared dense system with one h), 21 instances x 1000 steps against the stage-by-stage
    oracle, checkpoints every 125 steps (a stride of 250 = 2.5 periods of the fastest mode
    samples a single-mode velocity only at its zeros).  FP32: k omega h <= 0.32 at h = T_min/100."""
    import torch

    n_steps = 1000
    if kind == "chain":
        cfg = inputs.chain_batch(n_inst=21, s=s, n_steps=n_steps, seed=700 + s)
    elif kind == "dense_own":
        cfg = inputs.dense_own(s=s, n_inst=21, n_steps=n_steps, seed=7000 + s)
    else:
        cfg = inputs.dense_group(s=s, n_inst=21, n_steps=n_steps, seed=8000 + s)
    sys_ = make_system(ctx, cfg)
    d = torch.device("cuda:0")
    h = cfg["h"] if kind != "dense_shared" else cfg["h"][:1]
    try:
        out = cho.cho_integrate_batch(ctx, sys_, torch.as_tensor(cfg["x0"], device=d),
                                      torch.as_tensor(cfg["v0"], device=d), torch.as_tensor(h, device=d),
                                      n_steps, prec, 125, trajectory=True, poly_jump=k)
        torch.cuda.synchronize()
        out = {key: val.cpu().numpy() for key, val in out.items()}
    finally:
        cho.cho_destroy_system(sys_)
    if kind == "dense_shared":
        cfg = dict(cfg, h=np.full(21, cfg["h"][0]))
    ref = oracle_run(cfg, ckpt_every=125)
    ex, ev = check(out, ref, tol)
    print(f"small poly s={s} {kind} k={k} {prec}: x {ex:.3e} v {ev:.3e}")


@pytest.mark.parametrize("s", [33, 64, 128, 256, 300])
@pytest.mark.parametrize("prec,tol,k", [("fp64", TOL_FP64, 1), ("fp64", TOL_FP64, 25), ("fp32_kahan", TOL_FP32, 1),
                                        ("fp32_kahan", TOL_FP32, 5)])
def test_dense_poly_form_matches_oracle(ctx, s, prec, tol, k):
    """Shared dense system, jumps x <- x + E_xx x + E_xv v, v <- v + E_vx x + E_xx v built from
    P(hA)^k in FP64 on the host; 9 instances, 1000 steps against the stage-by-stage oracle."""
    import torch

    cfg = inputs.dense_group(s=s, n_inst=9, n_steps=1000)
    sys_ = make_system(ctx, cfg)
    d = torch.device("cuda:0")
    try:
        out = cho.cho_integrate_batch(ctx, sys_, torch.as_tensor(cfg["x0"], device=d),
                                      torch.as_tensor(cfg["v0"], device=d), torch.as_tensor(cfg["h"], device=d),
                                      1000, prec, 125, trajectory=True, poly_jump=k)
        torch.cuda.synchronize()
        out = {key: val.cpu().numpy() for key, val in out.items()}
    finally:
        cho.cho_destroy_system(sys_)
    ref = oracle_run(cfg, ckpt_every=125)
    ex, ev = check(out, ref, tol)
    print(f"dense poly s={s} k={k} {prec}: x {ex:.3e} v {ev:.3e}")


def test_dense_poly_form_needs_one_h(ctx):
    cfg = inputs.dense_group(s=40, n_inst=3, n_steps=100)
    h = cfg["h"].copy()
    h[1] *= 0.5
    sys_ = make_system(ctx, cfg)
    try:
        with pytest.raises(cho.ChoError) as ei:
            cho.cho_integrate_batch(ctx, sys_, cfg["x0"], cfg["v0"], h, 100, "fp32_kahan", poly_jump=5)
        assert ei.value.status == cho.CHO_EINVAL
        own = inputs.dense_own(s=40, n_inst=2, n_steps=10)
        s2 = make_system(ctx, own)
        try:
            with pytest.raises(cho.ChoError) as ei:
                cho.cho_integrate_batch(ctx, s2, own["x0"], own["v0"], own["h"], 10, "fp32_kahan", poly_jump=5)
            assert ei.value.status == cho.CHO_EINVAL
        finally:
            cho.cho_destroy_system(s2)
    finally:
        cho.cho_destroy_system(sys_)


def test_dense_poly_form_full_size_sampled(ctx):
    """8192 instances of s = 128, 5e3 steps, k = 5, sampled against the oracle."""
    import torch

    cfg = inputs.dense_group(s=128, n_inst=8192, n_steps=5000)
    sys_ = make_system(ctx, cfg)
    d = torch.device("cuda:0")
    try:
        out = cho.cho_integrate_batch(ctx, sys_, torch.as_tensor(cfg["x0"], device=d),
                                      torch.as_tensor(cfg["v0"], device=d), torch.as_tensor(cfg["h"], device=d),
                                      5000, "fp32_kahan", 625, trajectory=True, poly_jump=5)
        torch.cuda.synchronize()
        out = {key: val.cpu().numpy() for key, val in out.items()}
    finally:
        cho.cho_destroy_system(sys_)
    idx = sample_indices(8192, 6)
    ref = oracle_run(cfg, idx=idx, ckpt_every=625)
    check(out, ref, TOL_FP32, idx)


@pytest.mark.parametrize("k", [1, 5, 25])
def test_poly_form_full_size_sampled(ctx, k):
    """65,536 systems x 1e4 steps in the polynomial form on the balanced schedule, sampled
    (checkpoints every 125 steps: a multiple of T_min / h = 200 would see the fastest mode
    only at its turning points)."""
    cfg = inputs.two_dof_batch()
    import torch

    sys_ = make_system(ctx, cfg)
    d = torch.device("cuda:0")
    try:
        out = cho.cho_integrate_batch(ctx, sys_, torch.as_tensor(cfg["x0"], device=d),
                                      torch.as_tensor(cfg["v0"], device=d), torch.as_tensor(cfg["h"], device=d),
                                      10000, "fp32_kahan", 125, trajectory=True, poly_jump=k)
        torch.cuda.synchronize()
        out = {key: val.cpu().numpy() for key, val in out.items()}
    finally:
        cho.cho_destroy_system(sys_)
    idx = sample_indices(cfg["x0"].shape[0], 128)
    ref = oracle_run(cfg, idx=idx, ckpt_every=125)
    check(out, ref, TOL_FP32, idx)


def test_poly_form_balanced_is_bitwise_equal(tmp_path):
    """The polynomial form on the balanced schedule gives the bits of one warp per 64 instances."""
    import subprocess
    import sys as _sys

    code = _VARIANT_RUN.replace("'fp32_kahan', every, trajectory=every > 0)",
                                "'fp32_kahan', every, trajectory=every > 0, poly_jump=5)")
    assert code != _VARIANT_RUN
    res = {}
    for variant in ("balanced", "pair"):
        path = str(tmp_path / f"{variant}.npz")
        env = dict(os.environ, CHO_TWO_DOF_KERNEL=variant)
        subprocess.run([_sys.executable, "-c", code, path, "45001", "3000", "1000"], check=True, env=env,
                       timeout=300)
        res[variant] = np.load(path)
    for key in res["pair"].files:
        assert np.isfinite(res["balanced"][key]).all(), key
        assert np.array_equal(res["pair"][key], res["balanced"][key]), key


def test_poly_form_rejects_what_it_does_not_cover(ctx):
    cfg = inputs.two_dof_batch(n_inst=4, n_steps=100)
    two = make_system(ctx, cfg)
    ch = inputs.chain_batch(n_inst=2, s=5, n_steps=100)
    chain = cho.cho_create_system(ctx, "chain", masses=ch["masses"], springs=ch["springs"])
    try:
        bad = [
            lambda: cho.cho_integrate_batch(ctx, two, cfg["x0"], cfg["v0"], cfg["h"], 100, "fp32_kahan",
                                            poly_jump=3),                       # 3 does not divide 100
            lambda: cho.cho_integrate_batch(ctx, two, cfg["x0"], cfg["v0"], cfg["h"], 100, "fp32_kahan", 50,
                                            trajectory=True, poly_jump=20),     # 20 does not divide 50
            lambda: cho.cho_integrate_batch(ctx, two, cfg["x0"], cfg["v0"], cfg["h"], 100, "fp32_kahan",
                                            poly_jump=-1),
            lambda: cho.cho_integrate_batch(ctx, chain, ch["x0"], ch["v0"], ch["h"], 100, "fp32x2",
                                            poly_jump=1),                       # not in double-FP32
        ]
        for call in bad:
            with pytest.raises(cho.ChoError) as ei:
                call()
            assert ei.value.status == cho.CHO_EINVAL
        # zero instances and zero steps are accepted
        out = cho.cho_integrate_batch(ctx, two, cfg["x0"], cfg["v0"], cfg["h"], 0, "fp32_kahan", poly_jump=4)
        assert np.allclose(out["x"], cfg["x0"], rtol=0, atol=1e-7)
    finally:
        cho.cho_destroy_system(chain)
        cho.cho_destroy_system(two)


# ---- full-size workloads, sampled against the oracle ------------------------------------------

# Over the full 5e3-step horizon bf16x5 and bf16x6 stay within 1e-5 (each K chunk in its own
# accumulator, chunks added in FP32 round-to-nearest).
TOL_BF16_FULL = {"bf16x5": TOL_FP32, "bf16x6": TOL_FP32}


@pytest.mark.parametrize("s,prec", [(64, "bf16x5"), (128, "bf16x5"), (256, "bf16x5"), (64, "bf16x6"),
                                    (128, "bf16x6")])
def test_dense_full_size_sampled(ctx, s, prec):
    """8192 instances sharing one (M, K), 5e3 steps on the tensor cores (the benchmark launch)."""
    cfg = inputs.dense_group(s=s, n_inst=8192, n_steps=5000)
    out = run_gpu(ctx, cfg, prec, 625)
    idx = sample_indices(8192, 16)
    ref = oracle_run(cfg, idx=idx, ckpt_every=625)
    ex, ev = check(out, ref, TOL_BF16_FULL[prec], idx)
    print(f"dense s={s} 8192 x 5000 {prec} sampled: x {ex:.3e} v {ev:.3e}")


@pytest.mark.parametrize("s", [64, 128, 256])
@pytest.mark.parametrize("prec,tol", [("fp32_simt", TOL_FP32), ("fp64", TOL_FP64)])
def test_dense_full_horizon_cuda_cores(ctx, s, prec, tol):
    """The dense workload at its full size and horizon (8192 instances sharing one (M, K),
    5e3 steps) on the CUDA cores, FP32 + compensation and FP64, sampled against the oracle
    on 16 instances (first, last and a seeded sample)."""
    cfg = inputs.dense_group(s=s, n_inst=8192, n_steps=5000)
    out = run_gpu(ctx, cfg, prec, 625)
    idx = sample_indices(8192, 16)
    ref = oracle_run(cfg, idx=idx, ckpt_every=625)
    ex, ev = check(out, ref, tol, idx)
    print(f"dense s={s} 8192 x 5000 {prec} sampled: x {ex:.3e} v {ev:.3e}")


def test_chain_full_size_sampled_fp64(ctx):
    """4096 chains of 1024 masses x 1e4 steps in FP64, sampled against the oracle."""
    cfg = inputs.chain_batch()
    out = run_gpu(ctx, cfg, "fp64", 625)
    idx = sample_indices(cfg["x0"].shape[0], 8)
    ref = oracle_run(cfg, idx=idx, ckpt_every=625)
    check(out, ref, TOL_FP64, idx)


@pytest.mark.parametrize("prec,tol", [("fp64", TOL_FP64), ("fp32_kahan", TOL_FP32)])
def test_largest_chain(ctx, prec, tol):
    """s = 8192 (eight DOFs per thread on 1024 threads), the largest chain the library takes."""
    cfg = inputs.chain_batch(n_inst=2, s=8192, n_steps=250, seed=8192)
    out = run_gpu(ctx, cfg, prec, 125)
    ref = oracle_run(cfg, ckpt_every=125)
    check(out, ref, tol)


@pytest.mark.parametrize("prec,tol", [("fp64", TOL_FP64), ("fp32_simt", TOL_FP32)])
def test_largest_dense_simt(ctx, prec, tol):
    """s = 512 (the largest dense system on the CUDA cores)."""
    cfg = inputs.dense_group(s=512, n_inst=9, n_steps=250)
    out = run_gpu(ctx, cfg, prec, 125)
    ref = oracle_run(cfg, ckpt_every=125)
    check(out, ref, tol)


def test_energy_dense_checkpoints(ctx):
    import oracle

    cfg = inputs.dense_group(s=100, n_inst=6, n_steps=500)
    sys_ = make_system(ctx, cfg)
    try:
        out = cho.cho_integrate_batch(ctx, sys_, cfg["x0"], cfg["v0"], cfg["h"], 500, "fp64", 125, energy=True)
    finally:
        cho.cho_destroy_system(sys_)
    E_ref = oracle.energy_dense(cfg["M"][0], cfg["K"][0], out["x_traj"].reshape(-1, 100),
                                out["v_traj"].reshape(-1, 100)).reshape(6, -1)
    assert np.allclose(out["energy"], E_ref, rtol=1e-12)
    # RK4 loses energy: every instance's energy decreases monotonically over the checkpoints
    assert np.all(np.diff(out["energy"], axis=1) <= 0)


def test_many_parameter_sets_small_dense(ctx):
    """S = 32 lane groups with 4099 distinct parameter sets (ragged last block)."""
    n = 4099
    rng = np.random.default_rng(31)
    s = 20
    M, K = [], []
    base_M, base_K, _, _ = inputs.dense_system(s, 2020)
    for i in range(n):
        scale = rng.uniform(0.5, 2.0)
        M.append(base_M)
        K.append(base_K * scale)
    M = np.stack(M)
    K = np.stack(K)
    w = inputs.omega_max_dense(base_M, base_K) * np.sqrt(2.0)
    cfg = {"kind": "dense", "s": s, "M": M, "K": K, "x0": rng.normal(size=(n, s)), "v0": np.zeros((n, s)),
           "h": np.full(n, float(inputs.fp32_exact(2 * math.pi / w / 100))), "n_steps": 500}
    out = run_gpu(ctx, cfg, "fp32_kahan", 125)
    idx = sample_indices(n, 40)
    ref = oracle_run(cfg, idx=idx, ckpt_every=125)
    check(out, ref, TOL_FP32, idx)


def test_tensor_core_wait_gives_up_and_reports(ctx):
    """Bounded device waits: with the MMAs withheld (test hook), the wait for their completion
    runs out after about a second, the kernel leaves cleanly and the call reports
    CHO_ETIMEOUT; the context stays usable and the next run is correct."""
    cfg = inputs.dense_group(s=64, n_inst=40, n_steps=20)
    sys_ = make_system(ctx, cfg)
    try:
        os.environ["CHO_TEST_STALL_MMA"] = "1"
        try:
            with pytest.raises(cho.ChoError) as ei:
                cho.cho_integrate_batch(ctx, sys_, cfg["x0"], cfg["v0"], cfg["h"], 20, "bf16x5")
            assert ei.value.status == cho.CHO_ETIMEOUT
            import torch

            d = torch.device("cuda:0")
            cho.cho_integrate_batch(ctx, sys_, torch.as_tensor(cfg["x0"], device=d),
                                    torch.as_tensor(cfg["v0"], device=d), torch.as_tensor(cfg["h"], device=d),
                                    20, "bf16x5")
            with pytest.raises(cho.ChoError) as ei:
                cho.cho_system_status(sys_)
            assert ei.value.status == cho.CHO_ETIMEOUT
        finally:
            del os.environ["CHO_TEST_STALL_MMA"]
        assert cho.cho_system_status(sys_) == cho.CHO_OK
        out = cho.cho_integrate_batch(ctx, sys_, cfg["x0"], cfg["v0"], cfg["h"], 20, "bf16x5")
        ref = oracle_run(cfg)
        assert rel_err(out["x"][:, None], ref["x"][:, None]).max() < TOL_FP32
    finally:
        cho.cho_destroy_system(sys_)


@pytest.mark.parametrize("s,prec,ckpt", [(128, "bf16x5", 0), (128, "bf16x3", 50), (128, "bf16x6", 0),
                                         (256, "bf16x5", 0), (256, "bf16x3", 50)])
def test_tensor_core_balanced_schedule_gives_the_bits_of_whole_tiles(ctx, s, prec, ckpt):
    """8185 instances: 256 tiles, more than the CTAs (s = 128) or 2-CTA clusters (s = 256)
    that fit at once, run on the balanced schedule (tiles cut between CTAs or clusters,
    their state handed over); parts of 4096 (s = 128: 128 tiles) or 2048 instances (s = 256:
    64 clusters), the last one ragged, run one CTA or cluster per tile for the whole horizon
    and give the same bits.  With checkpoints the cuts fall on checkpoint blocks and the
    trajectories agree."""
    import torch

    n, steps = 8185, 300
    part_n = 4096 if s == 128 else 2048
    cfg = inputs.dense_group(s=s, n_inst=n, n_steps=steps)
    sys_ = make_system(ctx, cfg)
    d = torch.device("cuda:0")
    try:
        x0 = torch.as_tensor(cfg["x0"], device=d)
        v0 = torch.as_tensor(np.random.default_rng(s).normal(0, 0.1, cfg["x0"].shape), device=d)
        h = torch.as_tensor(cfg["h"], device=d)
        full = cho.cho_integrate_batch(ctx, sys_, x0, v0, h, steps, prec, ckpt, trajectory=ckpt > 0)
        keys = ("x", "v", "x_traj", "v_traj") if ckpt else ("x", "v")
        for part in [slice(i, min(i + part_n, n)) for i in range(0, n, part_n)]:
            sep = cho.cho_integrate_batch(ctx, sys_, x0[part], v0[part], h[part], steps, prec, ckpt,
                                          trajectory=ckpt > 0)
            for key in keys:
                a, b = full[key][part].cpu().numpy(), sep[key].cpu().numpy()
                assert np.all(np.isfinite(a)), key
                assert np.array_equal(a, b), (key, float(np.max(np.abs(a - b))))
    finally:
        cho.cho_destroy_system(sys_)


@pytest.mark.parametrize("s", [128, 256])
def test_tensor_core_handover_wait_gives_up_and_reports(ctx, s):
    """Test hook CHO_TEST_WITHHOLD_HANDOVER=1 on the balanced tensor-core schedule: no CTA
    publishes the state of its first tile, each wait for it runs out (after about a second),
    those tiles finish as NaN, the call reports CHO_ETIMEOUT and the context stays usable."""
    import torch

    n, steps = 8192, 200
    cfg = inputs.dense_group(s=s, n_inst=n, n_steps=steps)
    sys_ = make_system(ctx, cfg)
    d = torch.device("cuda:0")
    try:
        os.environ["CHO_TEST_WITHHOLD_HANDOVER"] = "1"
        try:
            with pytest.raises(cho.ChoError) as ei:
                cho.cho_integrate_batch(ctx, sys_, cfg["x0"], cfg["v0"], cfg["h"], steps, "bf16x5")
            assert ei.value.status == cho.CHO_ETIMEOUT
            o = cho.cho_integrate_batch(ctx, sys_, torch.as_tensor(cfg["x0"], device=d),
                                        torch.as_tensor(cfg["v0"], device=d), torch.as_tensor(cfg["h"], device=d),
                                        steps, "bf16x5")
            with pytest.raises(cho.ChoError) as ei:
                cho.cho_system_status(sys_)
            assert ei.value.status == cho.CHO_ETIMEOUT
            xo = o["x"].cpu().numpy()
            assert np.isnan(xo).any() and np.isfinite(xo).any()
        finally:
            del os.environ["CHO_TEST_WITHHOLD_HANDOVER"]
        assert cho.cho_system_status(sys_) == cho.CHO_OK
        out = cho.cho_integrate_batch(ctx, sys_, cfg["x0"], cfg["v0"], cfg["h"], steps, "bf16x5")
        idx = sample_indices(n, 8)
        ref = oracle_run(cfg, idx=idx)
        assert rel_err(out["x"][idx][:, None], ref["x"][:, None]).max() < TOL_FP32
    finally:
        cho.cho_destroy_system(sys_)


# ---- autotuning among kernels that give the same bits ----------------------------------------

def _device_run(ctx, sys_, cfg, prec, n_steps):
    import torch

    dev = torch.device("cuda:0")
    out = cho.cho_integrate_batch(ctx, sys_, torch.as_tensor(cfg["x0"], device=dev),
                                  torch.as_tensor(cfg["v0"], device=dev), torch.as_tensor(cfg["h"], device=dev),
                                  n_steps, prec)
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in out.items()}


@pytest.mark.parametrize("case", ["two_dof", "chain_fp32", "chain_fp32_s40", "chain_fp32_s200", "chain_fp64",
                                  "dense_fp32"])
def test_autotune_chooses_among_same_bit_kernels(tmp_path, case):
    """cho_autotune times every candidate kernel of the shape; all give the bits of the first,
    the fastest is recorded, later batches of the shape use it (same bits as an untuned
    context), and the table survives a save / load into another context."""
    if case == "two_dof":
        cfg, prec, n_cand = inputs.two_dof_batch(n_inst=4096, n_steps=300), "fp32_kahan", 3
    elif case == "chain_fp32_s40":
        # 1 DOF per thread (the default, scalar FP32) against 2, 4 and 8 (packed FP32x2 pairs)
        cfg, prec, n_cand = inputs.chain_batch(n_inst=64, s=40, n_steps=200), "fp32_kahan", 4
    elif case == "chain_fp32_s200":
        # 4 DOFs per thread (the default: 2 warps) against the scalar kernel on 7 warps and the
        # packed kernel at 2 (4 warps) and 8 (1 warp): the packed kernels evaluate two stages per
        # neighbour exchange, the scalar kernel one, and the warp-edge exchange differs in each
        cfg, prec, n_cand = inputs.chain_batch(n_inst=64, s=200, n_steps=200), "fp32_kahan", 4
    elif case.startswith("chain"):
        cfg = inputs.chain_batch(n_inst=64, s=300, n_steps=200)
        prec, n_cand = ("fp32_kahan" if case == "chain_fp32" else "fp64"), 3     # 8 (default), 2, 4 DOFs per thread
    else:
        cfg, prec, n_cand = inputs.dense_group(s=200, n_inst=12, n_steps=200), "fp32_kahan", 2
    n_inst = cfg["x0"].shape[0]
    ctx, ctx2 = cho.cho_init(0), cho.cho_init(0)
    try:
        sys1, sys2 = make_system(ctx, cfg), make_system(ctx2, cfg)
        assert cho.cho_tune_query(ctx, sys1, n_inst, prec) == -1
        r = cho.cho_autotune(ctx, sys1, n_inst, prec)
        print(case, r)
        assert len(r["variants"]) == n_cand
        times = [us for _, _, us in r["variants"]]
        assert all(us > 0 for us in times), "a candidate gave different bits"
        best = int(np.argmin(times))
        expect = best if times[best] < 0.97 * times[0] else 0          # the default stays unless 3 % slower
        assert r["chosen"] == r["variants"][expect][0]
        assert cho.cho_tune_query(ctx, sys1, n_inst, prec) == r["code"]
        tuned = _device_run(ctx, sys1, cfg, prec, cfg["n_steps"])
        default = _device_run(ctx2, sys2, cfg, prec, cfg["n_steps"])
        assert np.array_equal(tuned["x"], default["x"]) and np.array_equal(tuned["v"], default["v"])
        path = tmp_path / "tune.txt"
        cho.cho_tune_save(ctx, str(path))
        assert cho.cho_tune_load(ctx2, str(path)) >= 1
        assert cho.cho_tune_query(ctx2, sys2, n_inst, prec) == r["code"]
        # one kernel only (FP64 dense, or the tensor cores): nothing to choose, nothing recorded
        if case == "dense_fp32":
            r64 = cho.cho_autotune(ctx, sys1, n_inst, "fp64")
            assert len(r64["variants"]) == 1 and cho.cho_tune_query(ctx, sys1, n_inst, "fp64") == -1
        bad = tmp_path / "bad.txt"
        bad.write_text("not a tune file\n")
        with pytest.raises(cho.ChoError):
            cho.cho_tune_load(ctx2, str(bad))
        cho.cho_destroy_system(sys1)
        cho.cho_destroy_system(sys2)
    finally:
        cho.cho_shutdown(ctx)
        cho.cho_shutdown(ctx2)


def test_uneven_batches_replay_from_a_cuda_graph():
    """A period's worth of uneven batches (2-DOF FP32, a chain, few dense instances on a
    cluster, dense on the tensor cores) captured on one stream into a CUDA graph: each
    replay gives the bits of direct calls, also after the inputs are rewritten in place."""
    import torch

    dev = torch.device("cuda:0")
    ctx = cho.cho_init(0)
    cases = [(inputs.two_dof_batch(n_inst=4096, n_steps=1), "fp32_kahan", 200),
             (inputs.chain_batch(n_inst=16, s=300, n_steps=1), "fp32_kahan", 100),
             (inputs.dense_group(s=200, n_inst=3, n_steps=1), "fp32_kahan", 100),
             (inputs.dense_group(s=128, n_inst=40, n_steps=1), "bf16x5", 100)]
    try:
        batches = []
        for cfg, prec, n in cases:
            sys_ = make_system(ctx, cfg)
            t = {k: torch.as_tensor(cfg[k], device=dev).clone() for k in ("x0", "v0", "h")}
            out = {"x": torch.empty_like(t["x0"]), "v": torch.empty_like(t["v0"])}
            batches.append((sys_, t, out, prec, n))
        s = torch.cuda.Stream()

        def run_all():
            for sys_, t, out, prec, n in batches:
                cho.cho_integrate_batch(ctx, sys_, t["x0"], t["v0"], t["h"], n, prec, out=out, stream=s)

        with torch.cuda.stream(s):
            run_all()                                  # first calls outside the capture
        torch.cuda.synchronize()
        direct = [(out["x"].clone(), out["v"].clone()) for _, _, out, _, _ in batches]
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s, capture_error_mode="thread_local"):
            run_all()
        for _, _, out, _, _ in batches:
            out["x"].zero_()
        g.replay()
        torch.cuda.synchronize()
        for (_, _, out, _, _), (x, v) in zip(batches, direct):
            assert torch.equal(out["x"], x) and torch.equal(out["v"], v)
        # new initial states in place: the replay follows them
        for _, t, _, _, _ in batches:
            t["x0"].mul_(0.5)
        g.replay()
        torch.cuda.synchronize()
        replayed = [(out["x"].clone(), out["v"].clone()) for _, _, out, _, _ in batches]
        with torch.cuda.stream(s):
            run_all()
        torch.cuda.synchronize()
        for (_, _, out, _, _), (x, v) in zip(batches, replayed):
            assert torch.equal(out["x"], x) and torch.equal(out["v"], v)
        del g
        for sys_, _, _, _, _ in batches:
            cho.cho_destroy_system(sys_)
    finally:
        cho.cho_shutdown(ctx)


# ---- double-FP32 (CHO_FP32X2): FP64-class accuracy on the FP32 pipe -----------------------------

def test_fp32x2_eq3_full_horizon():
    """Eq. 3 for 1e5 steps in double-FP32: within the FP64 mode's bar of the oracle and of the
    discrete closed form."""
    c = cho.cho_init(0)
    try:
        cfg = inputs.eq3_single()
        out = run_gpu(c, cfg, "fp32x2", 1000)
        ref = oracle_run(cfg, ckpt_every=1000)
        ex, ev = check(out, ref, TOL_FP64)
        print(f"fp32x2 eq3: x {ex:.3e} v {ev:.3e}")
        assert np.allclose(out["x"][0], [0.5919944669044028, -0.55303750830408224], atol=1e-10)
    finally:
        cho.cho_shutdown(c)


@pytest.mark.parametrize("n_inst", [1, 37, 1000])
def test_fp32x2_two_dof_batch(n_inst):
    c = cho.cho_init(0)
    try:
        cfg = inputs.two_dof_batch(n_inst=n_inst, n_steps=2000)
        out = run_gpu(c, cfg, "fp32x2", 250)
        ref = oracle_run(cfg, ckpt_every=250)
        ex, ev = check(out, ref, TOL_FP64)
        print(f"fp32x2 two_dof x{n_inst}: x {ex:.3e} v {ev:.3e}")
    finally:
        cho.cho_shutdown(c)


@pytest.mark.parametrize("s", [1, 3, 4, 5, 8, 9, 13, 16, 17, 31, 32])
def test_fp32x2_small_chains(s):
    """Chains of s <= 32 in double-FP32 on the small-system lanes (padded S = 2 .. 32: one
    lane holds S <= 4 rows, S = 8 two rows per lane, S >= 16 one): within the FP64 mode's bar."""
    c = cho.cho_init(0)
    try:
        cfg = inputs.chain_batch(n_inst=67, s=s, n_steps=2000, seed=2900 + s)
        # checkpoints every 125 steps: at 100 steps per period of the fastest mode a 250-step
        # stride meets s = 1 (one mode) at v = 0 every time
        out = run_gpu(c, cfg, "fp32x2", 125)
        ref = oracle_run(cfg, ckpt_every=125)
        ex, ev = check(out, ref, TOL_FP64)
        print(f"fp32x2 small chain s={s}: x {ex:.3e} v {ev:.3e}")
    finally:
        cho.cho_shutdown(c)


@pytest.mark.parametrize("s", [3, 6, 8, 13, 32])
def test_fp32x2_small_dense(s):
    """Dense (M, K) of s <= 32 in double-FP32: one (M, K) per instance, and one shared."""
    c = cho.cho_init(0)
    try:
        cfg = dense_per_instance(s, 21, 40 + s)
        out = run_gpu(c, cfg, "fp32x2", 125)
        check(out, oracle_run(cfg, ckpt_every=125), TOL_FP64)
        cfg = inputs.dense_group(s=s, n_inst=37, n_steps=1000)
        out = run_gpu(c, cfg, "fp32x2", 125)
        ex, ev = check(out, oracle_run(cfg, ckpt_every=125), TOL_FP64)
        print(f"fp32x2 small dense s={s}: x {ex:.3e} v {ev:.3e}")
    finally:
        cho.cho_shutdown(c)


@pytest.mark.parametrize("s", [33, 64, 127, 128, 129, 255, 256, 500, 1023, 1024])
def test_fp32x2_chains(s):
    """Spring chains in double-FP32 (four DOFs per thread, one CTA per chain; s not a
    multiple of 4 or of 128 leaves ragged threads and warps): within the FP64 mode's bar."""
    c = cho.cho_init(0)
    try:
        cfg = inputs.chain_batch(n_inst=5, s=s, n_steps=2000, seed=1900 + s)
        out = run_gpu(c, cfg, "fp32x2", 250)
        ref = oracle_run(cfg, ckpt_every=250)
        ex, ev = check(out, ref, TOL_FP64)
        print(f"fp32x2 chain s={s}: x {ex:.3e} v {ev:.3e}")
    finally:
        cho.cho_shutdown(c)


def test_fp32x2_chain_shared_parameters_and_host_arrays():
    """One (masses, springs) set for the whole batch, per-instance h, host arrays."""
    c = cho.cho_init(0)
    try:
        cfg = inputs.chain_batch(n_inst=9, s=300, n_steps=1000, seed=77)
        cfg = dict(cfg, masses=cfg["masses"][:1], springs=cfg["springs"][:1])
        out = run_gpu(c, cfg, "fp32x2", 125, device=False)
        ref = oracle_run(cfg, ckpt_every=125)
        check(out, ref, TOL_FP64)
        # one double-FP32 chain kernel: nothing for the tuner to choose or record
        sys_ = make_system(c, cfg)
        r = cho.cho_autotune(c, sys_, 9, "fp32x2")
        assert len(r["variants"]) == 1 and cho.cho_tune_query(c, sys_, 9, "fp32x2") == -1
        cho.cho_destroy_system(sys_)
    finally:
        cho.cho_shutdown(c)


def test_fp32x2_chain_full_size_sampled():
    """4096 chains of 1024 masses x 1e4 steps in double-FP32, sampled against the oracle."""
    c = cho.cho_init(0)
    try:
        cfg = inputs.chain_batch()
        out = run_gpu(c, cfg, "fp32x2", 625)
        idx = sample_indices(cfg["x0"].shape[0], 6)
        ref = oracle_run(cfg, idx=idx, ckpt_every=625)
        ex, ev = check(out, ref, TOL_FP64, idx)
        print(f"fp32x2 chain 4096 x 1024 sampled: x {ex:.3e} v {ev:.3e}")
    finally:
        cho.cho_shutdown(c)


def test_fp32x2_is_refused_outside_its_scope():
    c = cho.cho_init(0)
    try:
        ch = inputs.chain_batch(n_inst=2, s=1040, n_steps=10)      # chains beyond 1024 DOFs
        sys_ = make_system(c, ch)
        with pytest.raises(cho.ChoError) as ei:
            cho.cho_integrate_batch(c, sys_, ch["x0"], ch["v0"], ch["h"], 10, "fp32x2")
        assert ei.value.status == cho.CHO_EINVAL
        cho.cho_destroy_system(sys_)
        dn = inputs.dense_group(s=64, n_inst=2, n_steps=10)
        sysd = cho.cho_create_system(c, "dense", M=dn["M"], K=dn["K"])
        with pytest.raises(cho.ChoError):
            cho.cho_integrate_batch(c, sysd, dn["x0"], dn["v0"], dn["h"], 10, "fp32x2")
        cho.cho_destroy_system(sysd)
        two = inputs.two_dof_batch(n_inst=2, n_steps=10)
        sys2 = make_system(c, two)
        with pytest.raises(cho.ChoError):
            cho.cho_integrate_batch(c, sys2, two["x0"], two["v0"], two["h"], 10, "fp32x2", poly_jump=5)
        with pytest.raises(cho.ChoError):
            cho.cho_submit(c, sys2, two["x0"][0], two["v0"][0], float(two["h"][0]), 10, "fp32x2", 0, 0)
        cho.cho_destroy_system(sys2)
    finally:
        cho.cho_shutdown(c)


# ---- chains with coupled masses (eq. 1 with a tridiagonal M) ------------------------------

def coupled_chain(s, n_inst, seed, per_instance=True, n_steps=1000):
    """Chains whose mass matrix is tridiagonal: diagonal m_i, off-diagonal m_{i,i+1} =
    0.2 min(m_i, m_{i+1}) (a consistent-mass-like coupling), springs as in chain_batch; the
    dense M and K the library assembles, for the oracle."""
    cfg = inputs.chain_batch(n_inst=n_inst if per_instance else 1, s=s, n_steps=n_steps, seed=seed)
    m, c = cfg["masses"], cfg["springs"]
    mu = np.zeros_like(m)
    mu[:, :-1] = 0.2 * np.minimum(m[:, :-1], m[:, 1:])
    Ms, Ks = [], []
    for p in range(m.shape[0]):
        M = np.diag(m[p]) + np.diag(mu[p, :-1], 1) + np.diag(mu[p, :-1], -1)
        Ms.append(M)
        Ks.append(inputs.dense_stiffness_chain(c[p:p + 1])[0])
    M, K = np.stack(Ms), np.stack(Ks)
    w = inputs.omega_max_dense(M, K)
    h = inputs.fp32_exact(2 * math.pi / np.atleast_1d(w) / 100)
    rng = np.random.default_rng(seed + 1)
    x0 = rng.normal(0, 0.1, (n_inst, s))
    h = np.resize(h, n_inst) if per_instance else np.full(n_inst, h[0])
    return {"kind": "dense", "s": s, "M": M, "K": K, "masses": m, "springs": c, "mu": mu, "x0": x0,
            "v0": np.zeros((n_inst, s)), "h": h, "n_steps": n_steps}


@pytest.mark.parametrize("s", [3, 17, 40, 100, 300])
@pytest.mark.parametrize("per_instance", [True, False])
@pytest.mark.parametrize("prec,tol", [("fp64", TOL_FP64), ("fp32_kahan", TOL_FP32)])
def test_chain_with_coupled_masses_matches_dense_oracle(ctx, s, per_instance, prec, tol):
    cfg = coupled_chain(s, 7, 1300 + s, per_instance)
    sys_ = cho.cho_create_system(ctx, "chain", masses=cfg["masses"], springs=cfg["springs"],
                                 mass_coupling=cfg["mu"])
    try:
        w, s_info, n_sys = cho.cho_system_info(sys_)
        assert s_info == s and n_sys == cfg["masses"].shape[0]
        assert np.isclose(w, np.max(inputs.omega_max_dense(cfg["M"], cfg["K"])), rtol=1e-9)
        out = cho.cho_integrate_batch(ctx, sys_, cfg["x0"], cfg["v0"], cfg["h"], cfg["n_steps"], prec, 125,
                                      trajectory=True, energy=True)
        E = cho.cho_energy(ctx, sys_, out["x_traj"][:, -1], out["v_traj"][:, -1])
    finally:
        cho.cho_destroy_system(sys_)
    ref = oracle_run(cfg, ckpt_every=125)
    check(out, ref, tol)
    import oracle

    M = cfg["M"] if per_instance else np.repeat(cfg["M"], 7, 0)
    K = cfg["K"] if per_instance else np.repeat(cfg["K"], 7, 0)
    E_ref = np.array([oracle.energy_dense(M[i], K[i], out["x_traj"][i, -1:], out["v_traj"][i, -1:])[0]
                      for i in range(7)])
    assert np.allclose(E, E_ref, rtol=1e-12)


def test_chain_with_coupled_masses_rejects_bad_input(ctx):
    cfg = inputs.chain_batch(n_inst=1, s=6, n_steps=1)
    mu = np.full_like(cfg["masses"], 0.0)
    mu[0, 2] = 10.0 * cfg["masses"].max()              # M not positive definite
    with pytest.raises(cho.ChoError) as ei:
        cho.cho_create_system(ctx, "chain", masses=cfg["masses"], springs=cfg["springs"], mass_coupling=mu)
    assert ei.value.status == cho.CHO_ENOTSPD
    big = inputs.chain_batch(n_inst=1, s=600, n_steps=1)
    with pytest.raises(cho.ChoError) as ei:
        cho.cho_create_system(ctx, "chain", masses=big["masses"], springs=big["springs"],
                              mass_coupling=0.1 * big["masses"])
    assert ei.value.status == cho.CHO_EINVAL
