"""cho_integrate_plain_noalloc: the plain form with no allocation at call time.

Callers such as a real-time stepping loop must not allocate device memory while
they run (an allocation can block on the device and miss a step's deadline);
this entry point keeps its scratch in a fixed array inside the library.  The
tests check it against cho_integrate_plain, which allocates its scratch in a
context workspace, through the C ABI: the two run the same FP64 operations (one
shared device helper; h/2 and h/6 are IEEE operations on the same h in both), so
the results must match bit for bit, on two calls in a row (the second call finds
the array holding the first call's data).  This file is collected last, so a
failure here comes after every other test has run.
"""
import numpy as np
import pytest

from paper_1702_02207_gb300 import cho, inputs

pytestmark = pytest.mark.gpu


def _device(cfg):
    import torch

    dev = torch.device("cuda:0")
    return (torch.as_tensor(cfg["x0"], device=dev), torch.as_tensor(cfg["v0"], device=dev),
            torch.as_tensor(np.asarray(cfg["h"], dtype=np.float64).reshape(-1), device=dev))


def _system(ctx, kind):
    if kind == "two_dof":
        cfg = inputs.two_dof_batch(n_inst=3, n_steps=200)
        return cfg, cho.cho_create_system(ctx, "two_dof", masses=cfg["masses"], springs=cfg["springs"])
    if kind == "chain":
        # one parameter set and one h per instance (the h differ)
        cfg = inputs.chain_batch(n_inst=3, s=300, n_steps=150)
        assert len(set(np.asarray(cfg["h"]).tolist())) == 3
        return cfg, cho.cho_create_system(ctx, "chain", masses=cfg["masses"], springs=cfg["springs"])
    if kind == "dense":
        cfg = inputs.dense_group(s=40, n_inst=2, n_steps=150)
        return cfg, cho.cho_create_system(ctx, "dense", M=cfg["M"], K=cfg["K"])
    # dense systems with one (M, K) and one h per instance
    cfg = inputs.dense_own(s=24, n_inst=3, n_steps=120)
    return cfg, cho.cho_create_system(ctx, "dense", M=cfg["M"], K=cfg["K"])


@pytest.mark.parametrize("kind", ["two_dof", "chain", "dense", "dense_own"])
def test_noalloc_plain_matches_plain_on_two_calls(kind):
    import torch

    ctx = cho.cho_init(0)
    try:
        cfg, sys_ = _system(ctx, kind)
        x0, v0, h = _device(cfg)
        ref = cho.cho_integrate_plain(ctx, sys_, x0, v0, h, cfg["n_steps"])
        # a different input on the first call leaves other data in the shared scratch
        other = cho.cho_integrate_plain_noalloc(ctx, sys_, x0.flip(0).contiguous(), v0, h, cfg["n_steps"])
        got = cho.cho_integrate_plain_noalloc(ctx, sys_, x0, v0, h, cfg["n_steps"])
        torch.cuda.synchronize()
        for key in ("x", "v"):
            r = ref[key].cpu().numpy()
            g = got[key].cpu().numpy()
            assert np.all(np.isfinite(r))
            assert np.array_equal(g, r), (kind, key, np.max(np.abs(g - r)))
        assert np.all(np.isfinite(other["x"].cpu().numpy()))
        cho.cho_destroy_system(sys_)
    finally:
        cho.cho_shutdown(ctx)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    ctx = cho.cho_init(0)
    try:
        big = inputs.chain_batch(n_inst=1, s=5000, n_steps=1)
        sys_ = cho.cho_create_system(ctx, "chain", masses=big["masses"], springs=big["springs"])
        x0, v0, h = _device(big)
        with pytest.raises(cho.ChoError) as ei:
            cho.cho_integrate_plain_noalloc(ctx, sys_, x0, v0, h, 1)
        assert ei.value.status == cho.CHO_EINVAL
        assert "4096" in ei.value.message
        cho.cho_destroy_system(sys_)
    finally:
        cho.cho_shutdown(ctx)


def test_noalloc_rejects_damped_and_forced_systems():
    ctx = cho.cho_init(0)
    try:
        cfg = inputs.chain_batch(n_inst=2, s=50, n_steps=10)
        sys_ = cho.cho_create_system(ctx, "chain", masses=cfg["masses"], springs=cfg["springs"])
        x0, v0, h = _device(cfg)
        cho.cho_system_set_damping(sys_, 0.01 * cfg["springs"])
        with pytest.raises(cho.ChoError) as ei:
            cho.cho_integrate_plain_noalloc(ctx, sys_, x0, v0, h, 10)
        assert ei.value.status == cho.CHO_EINVAL
        cho.cho_system_set_damping(sys_, None)
        cho.cho_system_set_forcing(sys_, np.ones((2, 50)), np.full(2, 3.0))
        with pytest.raises(cho.ChoError) as ei:
            cho.cho_integrate_plain_noalloc(ctx, sys_, x0, v0, h, 10)
        assert ei.value.status == cho.CHO_EINVAL
        cho.cho_destroy_system(sys_)
    finally:
        cho.cho_shutdown(ctx)


def test_noalloc_bad_or_unstable_h_gives_nan_states():
    """h stays on the device, so a bad one cannot be rejected on the host: a non-positive,
    non-finite or unstable h (omega_max h > 2 sqrt 2) yields NaN states for that instance,
    and the other instances of the call are unaffected."""
    import torch

    ctx = cho.cho_init(0)
    try:
        cfg = inputs.chain_batch(n_inst=4, s=60, n_steps=20)
        sys_ = cho.cho_create_system(ctx, "chain", masses=cfg["masses"], springs=cfg["springs"])
        x0, v0, h = _device(cfg)
        ref = cho.cho_integrate_plain(ctx, sys_, x0, v0, h, 20)
        bad = h.clone()
        w = np.asarray(cfg["omega_max"], dtype=np.float64)
        bad[1] = -float(h[1])
        bad[2] = float("inf")
        bad[3] = 1.01 * 2.0 * np.sqrt(2.0) / w[3]          # just past the stability bound
        # host arrays: the allocating plain form checks h on the host and refuses
        with pytest.raises(cho.ChoError) as ei:
            cho.cho_integrate_plain(ctx, sys_, cfg["x0"], cfg["v0"], bad.cpu().numpy(), 20)
        assert ei.value.status == cho.CHO_EINVAL
        got = cho.cho_integrate_plain_noalloc(ctx, sys_, x0, v0, bad, 20)
        torch.cuda.synchronize()
        gx = got["x"].cpu().numpy()
        gv = got["v"].cpu().numpy()
        assert np.array_equal(gx[0], ref["x"].cpu().numpy()[0])
        assert np.array_equal(gv[0], ref["v"].cpu().numpy()[0])
        assert np.all(np.isnan(gx[1:])) and np.all(np.isnan(gv[1:]))
        cho.cho_destroy_system(sys_)
    finally:
        cho.cho_shutdown(ctx)
