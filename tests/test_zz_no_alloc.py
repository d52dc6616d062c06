"""cho_integrate_plain_noalloc: the plain form with no allocation at call time.

Callers such as a real-time stepping loop must not allocate device memory while
they run (an allocation can block on the device and miss a step's deadline);
this entry point keeps its scratch in a fixed array inside the library.  The
test checks it against cho_integrate_plain, which allocates its scratch in a
context workspace, on two calls in a row (the second call finds the array
holding the first call's data), through the C ABI.  This file is collected
last, so a failure here comes after every other test has run.
"""
import numpy as np
import pytest

from paper_1702_02207_gb300 import cho, inputs
from parity_util import TOL_FP64

pytestmark = pytest.mark.gpu


def _device(cfg):
    import torch

    dev = torch.device("cuda:0")
    return (torch.as_tensor(cfg["x0"], device=dev), torch.as_tensor(cfg["v0"], device=dev),
            torch.as_tensor(cfg["h"], device=dev))


@pytest.mark.parametrize("kind", ["two_dof", "chain", "dense"])
def test_noalloc_plain_matches_plain_on_two_calls(kind):
    import torch

    ctx = cho.cho_init(0)
    try:
        if kind == "two_dof":
            cfg = inputs.two_dof_batch(n_inst=3, n_steps=200)
            sys_ = cho.cho_create_system(ctx, "two_dof", masses=cfg["masses"], springs=cfg["springs"])
        elif kind == "chain":
            cfg = inputs.chain_batch(n_inst=2, s=300, n_steps=150)
            sys_ = cho.cho_create_system(ctx, "chain", masses=cfg["masses"], springs=cfg["springs"])
        else:
            cfg = inputs.dense_group(s=40, n_inst=2, n_steps=150)
            sys_ = cho.cho_create_system(ctx, "dense", M=cfg["M"], K=cfg["K"])
        x0, v0, h = _device(cfg)
        ref = cho.cho_integrate_plain(ctx, sys_, x0, v0, h, cfg["n_steps"])
        # a different input on the first call leaves other data in the shared scratch
        other = cho.cho_integrate_plain_noalloc(ctx, sys_, x0.flip(0).contiguous(), v0, h, cfg["n_steps"])
        got = cho.cho_integrate_plain_noalloc(ctx, sys_, x0, v0, h, cfg["n_steps"])
        torch.cuda.synchronize()
        for key in ("x", "v"):
            r = ref[key].cpu().numpy()
            g = got[key].cpu().numpy()
            err = np.max(np.abs(g - r)) / np.max(np.abs(r))
            assert err <= TOL_FP64, (kind, key, err)
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
