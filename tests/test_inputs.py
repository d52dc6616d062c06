"""Seeded workload generators: determinism, shapes, ranges and step-size recipe."""
import math

import numpy as np

from paper_1702_02207_gb300 import inputs


def test_two_dof_batch_recipe():
    a = inputs.two_dof_batch(n_inst=4096)
    b = inputs.two_dof_batch(n_inst=4096)
    assert np.array_equal(a["masses"], b["masses"]) and np.array_equal(a["x0"], b["x0"])
    assert a["masses"].shape == (4096, 2) and a["springs"].shape == (4096, 2)
    assert a["masses"].min() >= 0.1 and a["masses"].max() <= 10.0
    assert a["springs"].min() >= 1e2 and a["springs"].max() <= 1e4
    assert np.all(np.abs(a["x0"]) <= 1.0) and np.all(a["v0"] == 0)
    # h is FP32-representable and equals T_min / 200 to FP32 rounding
    assert np.array_equal(a["h"].astype(np.float32).astype(np.float64), a["h"])
    theta = a["omega_max"] * a["h"]
    assert np.allclose(theta, 2 * math.pi / 200, rtol=1e-7)
    # log-uniform: the median of log(m) sits mid-range
    assert abs(np.median(np.log(a["masses"]))) < 0.1


def test_chain_batch_recipe_small():
    c = inputs.chain_batch(n_inst=3, s=64)
    assert c["x0"].shape == (3, 64)
    assert np.allclose(c["omega_max"] * c["h"], 2 * math.pi / 100, rtol=1e-7)
    # omega_max agrees with a dense generalised eigensolve
    K = inputs.dense_stiffness_chain(c["springs"][:1])[0]
    w = inputs.omega_max_dense(np.diag(c["masses"][0]), K)
    assert w == np.float64(w) and abs(w - c["omega_max"][0]) < 1e-9 * w


def test_dense_group_recipe():
    d = inputs.dense_group(s=32, n_inst=5)
    M, K = d["M"][0], d["K"][0]
    assert np.allclose(M, M.T) and np.allclose(K, K.T)
    assert np.linalg.eigvalsh(M).min() > 0.99
    lam = np.linalg.eigvalsh(K)
    assert lam.min() >= 1.0 - 1e-9 and lam.max() <= 1e4 * (1 + 1e-9)
    assert np.allclose(d["Q"].T @ d["Q"], np.eye(32), atol=1e-12)


def test_request_stream_recipe():
    st = inputs.request_stream(n_req=20_000)
    assert np.all(np.diff(st["t_arrive"]) > 0)
    assert st["s"].min() >= 2 and st["s"].max() <= 512
    assert st["n_steps"].min() >= 1000 and st["n_steps"].max() <= 100_000
    frac = np.bincount(st["priority"], minlength=3) / st["n_req"]
    assert np.allclose(frac, [0.2, 0.3, 0.5], atol=0.02)
    assert np.all(st["kind"][st["s"] == 2] == 0)
    p = inputs.request_params(st, 5)
    q = inputs.request_params(st, 5)
    assert np.array_equal(p["x0"], q["x0"])
