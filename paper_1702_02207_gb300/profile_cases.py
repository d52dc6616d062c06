"""Small single-launch cases of each kernel family, for profiler captures.

    python -m paper_1702_02207_gb300.profile_cases <case> [<case> ...]

Cases (each one cho_integrate_batch call, a few MB of device memory):
  pair      65,536 two-DOF systems, 1e4 steps, fp32_kahan   (rk4_pair2_balanced, the benchmark launch)
  chain     512 chains of 1024 masses, 2000 steps, fp32_kahan (rk4_chain<8>)
  dense_tc  s = 128, 2048 instances, 500 steps, bf16x5       (rk4_dense_tc, one CTA per SM)
  dense_tc64 s = 64, 4096 instances, 500 steps, bf16x5      (rk4_dense_tc, two tiles stacked per CTA)
  dense_tc2 s = 256, 2048 instances, 200 steps, bf16x5       (rk4_dense_tc, 2-CTA clusters)
  dense_simt s = 256, 512 instances, 50 steps, fp32_simt     (rk4_dense_simt)
"""
from __future__ import annotations

import sys


def run(case: str) -> None:
    import torch

    from paper_1702_02207_gb300 import cho, inputs

    dev = torch.device("cuda:0")
    ctx = cho.cho_init(0)
    try:
        if case == "pair":
            cfg, prec, kind = inputs.two_dof_batch(), "fp32_kahan", "two_dof"
        elif case == "chain":
            cfg, prec, kind = inputs.chain_batch(n_inst=512, n_steps=2000), "fp32_kahan", "chain"
        elif case == "dense_tc":
            cfg, prec, kind = inputs.dense_group(s=128, n_inst=2048, n_steps=500), "bf16x5", "dense"
        elif case == "dense_tc64":
            cfg, prec, kind = inputs.dense_group(s=64, n_inst=4096, n_steps=500), "bf16x5", "dense"
        elif case == "dense_tc2":
            cfg, prec, kind = inputs.dense_group(s=256, n_inst=2048, n_steps=200), "bf16x5", "dense"
        elif case == "dense_simt":
            cfg, prec, kind = inputs.dense_group(s=256, n_inst=512, n_steps=50), "fp32_simt", "dense"
        else:
            raise SystemExit(f"unknown case {case}")
        if kind == "dense":
            sys_ = cho.cho_create_system(ctx, "dense", M=cfg["M"], K=cfg["K"])
        else:
            sys_ = cho.cho_create_system(ctx, kind, masses=cfg["masses"], springs=cfg["springs"])
        x0 = torch.as_tensor(cfg["x0"], device=dev)
        v0 = torch.as_tensor(cfg["v0"], device=dev)
        h = torch.as_tensor(cfg["h"], device=dev)
        cho.cho_integrate_batch(ctx, sys_, x0, v0, h, cfg["n_steps"], prec)
        torch.cuda.synchronize()
        cho.cho_destroy_system(sys_)
    finally:
        cho.cho_shutdown(ctx)
    print(f"{case}: ok")


if __name__ == "__main__":
    for c in sys.argv[1:] or ["pair"]:
        run(c)
