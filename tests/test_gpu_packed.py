"""cho_integrate_packed: batches of uneven sizes and horizons in as few launches as possible.

Each batch's result must be bitwise equal to a separate cho_integrate_batch call of the
same batch (eq. 1 and eq. 2 with uneven s: the instance, not the batch, is the unit of
work), whichever other batches share its launch.
"""
import numpy as np
import pytest

from paper_1702_02207_gb300 import cho, inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = cho.cho_init(0)
    yield c
    cho.cho_shutdown(c)


def _mk(ctx, cfg):
    if cfg["kind"] == "dense":
        return cho.cho_create_system(ctx, "dense", M=cfg["M"], K=cfg["K"])
    return cho.cho_create_system(ctx, cfg["kind"], masses=cfg["masses"], springs=cfg["springs"])


def _workloads():
    """(config, steps) of batches spanning every packing group: s = 2 (S = 2); chains of 3 and
    dense of 4 (both S = 4); chains of 5 and 8 (S = 8); chains of 40 and 63 (one DOF per thread),
    100 (two), 300 (eight); dense shared s = 100, dense with one (M, K) per instance s = 50."""
    return [
        (inputs.two_dof_batch(n_inst=300, n_steps=1), 700),
        (inputs.chain_batch(n_inst=50, s=3, n_steps=1, seed=31), 400),
        (inputs.dense_group(s=4, n_inst=20, n_steps=1, seed=41), 250),
        (inputs.chain_batch(n_inst=40, s=5, n_steps=1, seed=51), 300),
        (inputs.chain_batch(n_inst=30, s=8, n_steps=1, seed=81), 500),
        (inputs.chain_batch(n_inst=10, s=40, n_steps=1, seed=401), 350),
        (inputs.chain_batch(n_inst=7, s=63, n_steps=1, seed=631), 120),
        (inputs.chain_batch(n_inst=5, s=100, n_steps=1, seed=1001), 200),
        (inputs.chain_batch(n_inst=3, s=300, n_steps=1, seed=3001), 150),
        (inputs.dense_group(s=100, n_inst=9, n_steps=1, seed=1002), 180),
        (inputs.dense_own(s=50, n_inst=4, n_steps=1, seed=502), 160),
    ]


@pytest.mark.parametrize("prec", ["fp32_kahan", "fp64"])
def test_packed_batches_match_separate_calls_bitwise(ctx, prec):
    import torch

    d = torch.device("cuda:0")
    work = _workloads()
    systems = [_mk(ctx, cfg) for cfg, _ in work]
    try:
        batches, separate = [], []
        for (cfg, n), sy in zip(work, systems):
            x0 = torch.as_tensor(cfg["x0"], device=d)
            v0 = torch.as_tensor(np.random.default_rng(cfg["s"]).normal(0, 0.1, cfg["x0"].shape), device=d)
            h = torch.as_tensor(np.asarray(cfg["h"]).reshape(-1), device=d)
            batches.append({"system": sy, "x0": x0, "v0": v0, "h": h, "n_steps": n, "prec": prec})
            separate.append(cho.cho_integrate_batch(ctx, sy, x0, v0, h, n, prec))
        packed = cho.cho_integrate_packed(ctx, batches)
        torch.cuda.synchronize()
        for k, (a, b) in enumerate(zip(packed, separate)):
            for key in ("x", "v"):
                ga, gb = a[key].cpu().numpy(), b[key].cpu().numpy()
                assert np.all(np.isfinite(gb)), (k, key)
                assert np.array_equal(ga, gb), (k, key, float(np.max(np.abs(ga - gb))))
        # a second call in another order (other group membership order) gives the same bits
        again = cho.cho_integrate_packed(ctx, batches[::-1])[::-1]
        torch.cuda.synchronize()
        for a, b in zip(again, separate):
            assert np.array_equal(a["x"].cpu().numpy(), b["x"].cpu().numpy())
    finally:
        for sy in systems:
            cho.cho_destroy_system(sy)


def test_packed_tensor_core_and_zero_steps(ctx):
    """A shared dense system on the tensor cores (bf16x5) beside a chain group, and a batch of
    zero steps, which returns its input."""
    import torch

    d = torch.device("cuda:0")
    dn = inputs.dense_group(s=128, n_inst=40, n_steps=1, seed=1280)
    ch = inputs.chain_batch(n_inst=6, s=64, n_steps=1, seed=640)
    sd, sc = _mk(ctx, dn), _mk(ctx, ch)
    try:
        b1 = {"system": sd, "x0": torch.as_tensor(dn["x0"], device=d), "v0": torch.as_tensor(dn["v0"], device=d),
              "h": torch.as_tensor(dn["h"][:1], device=d), "n_steps": 100, "prec": "bf16x5"}
        b2 = {"system": sc, "x0": torch.as_tensor(ch["x0"], device=d), "v0": torch.as_tensor(ch["v0"], device=d),
              "h": torch.as_tensor(ch["h"], device=d), "n_steps": 0, "prec": "fp32_kahan"}
        sep = cho.cho_integrate_batch(ctx, sd, b1["x0"], b1["v0"], b1["h"], 100, "bf16x5")
        sep0 = cho.cho_integrate_batch(ctx, sc, b2["x0"], b2["v0"], b2["h"], 0, "fp32_kahan")
        out = cho.cho_integrate_packed(ctx, [b1, b2])
        torch.cuda.synchronize()
        assert np.array_equal(out[0]["x"].cpu().numpy(), sep["x"].cpu().numpy())
        assert np.array_equal(out[0]["v"].cpu().numpy(), sep["v"].cpu().numpy())
        assert np.array_equal(out[1]["x"].cpu().numpy(), sep0["x"].cpu().numpy())
    finally:
        cho.cho_destroy_system(sd)
        cho.cho_destroy_system(sc)


def test_packed_rejects_what_it_does_not_cover(ctx):
    import torch

    d = torch.device("cuda:0")
    ch = inputs.chain_batch(n_inst=2, s=40, n_steps=1)
    sc = _mk(ctx, ch)
    try:
        base = {"system": sc, "x0": torch.as_tensor(ch["x0"], device=d), "v0": torch.as_tensor(ch["v0"], device=d),
                "h": torch.as_tensor(ch["h"], device=d), "n_steps": 10, "prec": "fp32x2"}
        with pytest.raises(cho.ChoError) as ei:
            cho.cho_integrate_packed(ctx, [base])
        assert ei.value.status == cho.CHO_EINVAL
        cho.cho_system_set_damping(sc, 0.01 * ch["springs"])
        with pytest.raises(cho.ChoError) as ei:
            cho.cho_integrate_packed(ctx, [dict(base, prec="fp32_kahan")])
        assert ei.value.status == cho.CHO_EINVAL
        cho.cho_system_set_damping(sc, None)
        bad_h = dict(base, prec="fp32_kahan", h=torch.full((2,), 10.0, dtype=torch.float64, device=d))
        assert cho.cho_integrate_packed(ctx, []) == []
        # an unstable h on the device with one h per instance is not checked on the host
        # (as cho_integrate_batch); a single device h is
        with pytest.raises(cho.ChoError) as ei:
            cho.cho_integrate_packed(ctx, [dict(bad_h, h=bad_h["h"][:1])])
        assert ei.value.status == cho.CHO_EUNSTABLE
    finally:
        cho.cho_destroy_system(sc)
