"""Small single-launch cases of each kernel family, for profiler captures.

    python -m paper_1702_02207_gb300.profile_cases <case> [<case> ...]

Cases (each one cho_integrate_batch call, a few MB of device memory):
  pair      65,536 two-DOF systems, 1e4 steps, fp32_kahan   (rk4_pair2_balanced, the benchmark launch)
  pair_dw   65,536 two-DOF systems, 2000 steps, fp32x2      (rk4_dw_small<2>, double-FP32)
  chain     512 chains of 1024 masses, 2000 steps, fp32_kahan (rk4_chain_pk<8>)
  chain_dw  512 chains of 1024 masses, 500 steps, fp32x2    (rk4_chain_dw<4>, double-FP32)
  dense_tc  s = 128, 2048 instances, 500 steps, bf16x5       (rk4_dense_tc, one CTA per SM)
  dense_tc64 s = 64, 4096 instances, 500 steps, bf16x5      (rk4_dense_tc, two tiles stacked per CTA)
  dense_tc2 s = 256, 2048 instances, 200 steps, bf16x5       (rk4_dense_tc, 2-CTA clusters)
  dense_tc_bal s = 128, 8192 instances, 200 steps, bf16x5   (rk4_dense_tc_pair on the balanced schedule:
            one CTA per SM, 256 tiles cut in step blocks)
  dense_tc2_bal s = 256, 8192 instances, 60 steps, bf16x5   (rk4_dense_tc, balanced over resident clusters)
  dense_simt s = 256, 512 instances, 50 steps, fp32_simt     (rk4_dense_simt)
  dense_own s = 64, 8192 instances with their own (M, K), 100 steps, fp32_kahan (rk4_dense_own, one per CTA)
  dense_split s = 512, 4 instances of one (M, K), 500 steps, fp32_kahan (rk4_dense_split, 8-CTA clusters)
  dense_split128 s = 128, 608 instances with their own (M, K), 200 steps, fp32_kahan (rk4_dense_split, 1 CTA)
  dense_poly s = 128, 2048 instances, 500 steps, fp32_kahan, k = 25 steps per update (rk4_dense_poly)
  chain_ext 512 damped and forced chains of 1024 masses, 2000 steps, fp32_kahan (rk4_chain_ext)
  small_poly 4096 chains of 17 masses, 2000 steps, fp32_kahan, k = 5 steps per update
            (small_poly_setup_kernel<32>, rk4_small_poly_kernel<32>)
  packed    the bench's uneven batches (chains of 33..63 x 400, 5..8 x 4000, 3..4 x 8000), 1000 steps,
            fp32_kahan, through cho_integrate_packed (one slot-form launch per size class)
"""
from __future__ import annotations

import sys


def run(case: str) -> None:
    import torch

    from paper_1702_02207_gb300 import cho, inputs

    dev = torch.device("cuda:0")
    ctx = cho.cho_init(0)
    poly = 0
    try:
        if case == "pair":
            cfg, prec, kind = inputs.two_dof_batch(), "fp32_kahan", "two_dof"
        elif case == "pair_dw":
            cfg, prec, kind = inputs.two_dof_batch(n_steps=2000), "fp32x2", "two_dof"
        elif case == "chain":
            cfg, prec, kind = inputs.chain_batch(n_inst=512, n_steps=2000), "fp32_kahan", "chain"
        elif case == "chain_dw":
            cfg, prec, kind = inputs.chain_batch(n_inst=512, n_steps=500), "fp32x2", "chain"
        elif case == "dense_tc":
            cfg, prec, kind = inputs.dense_group(s=128, n_inst=2048, n_steps=500), "bf16x5", "dense"
        elif case == "dense_tc64":
            cfg, prec, kind = inputs.dense_group(s=64, n_inst=4096, n_steps=500), "bf16x5", "dense"
        elif case == "dense_tc2":
            cfg, prec, kind = inputs.dense_group(s=256, n_inst=2048, n_steps=200), "bf16x5", "dense"
        elif case == "dense_tc_bal":
            cfg, prec, kind = inputs.dense_group(s=128, n_inst=8192, n_steps=200), "bf16x5", "dense"
        elif case == "dense_tc2_bal":
            cfg, prec, kind = inputs.dense_group(s=256, n_inst=8192, n_steps=60), "bf16x5", "dense"
        elif case == "dense_simt":
            cfg, prec, kind = inputs.dense_group(s=256, n_inst=512, n_steps=50), "fp32_simt", "dense"
        elif case == "dense_own":
            cfg, prec, kind = inputs.dense_own(s=64, n_inst=8192, n_steps=100), "fp32_kahan", "dense"
        elif case == "dense_split":
            cfg, prec, kind = inputs.dense_group(s=512, n_inst=4, n_steps=500), "fp32_kahan", "dense"
        elif case == "dense_split128":
            cfg, prec, kind = inputs.dense_own(s=128, n_inst=608, n_steps=200), "fp32_kahan", "dense"
        elif case == "dense_poly":
            cfg, prec, kind = inputs.dense_group(s=128, n_inst=2048, n_steps=500), "fp32_kahan", "dense"
            poly = 25
        elif case == "small_poly":
            cfg, prec, kind = inputs.chain_batch(n_inst=4096, s=17, n_steps=2000, seed=1717), "fp32_kahan", "chain"
            poly = 5
        elif case == "packed":
            cfgs = ([inputs.chain_batch(n_inst=400, s=sv, n_steps=1, seed=9000 + sv) for sv in (33, 40, 47, 55, 63)] +
                    [inputs.chain_batch(n_inst=4000, s=sv, n_steps=1, seed=9100 + sv) for sv in (5, 6, 7, 8)] +
                    [inputs.chain_batch(n_inst=8000, s=sv, n_steps=1, seed=9200 + sv) for sv in (3, 4)])
            systems, batches = [], []
            for c in cfgs:
                sy = cho.cho_create_system(ctx, "chain", masses=c["masses"], springs=c["springs"])
                systems.append(sy)
                batches.append({"system": sy, "x0": torch.as_tensor(c["x0"], device=dev),
                                "v0": torch.as_tensor(c["v0"], device=dev), "h": torch.as_tensor(c["h"], device=dev),
                                "n_steps": 1000, "prec": "fp32_kahan"})
            cho.cho_integrate_packed(ctx, batches)
            torch.cuda.synchronize()
            for sy in systems:
                cho.cho_destroy_system(sy)
            return
        elif case == "chain_ext":
            cfg, prec, kind = inputs.chain_batch(n_inst=512, n_steps=2000), "fp32_kahan", "chain"
        else:
            raise SystemExit(f"unknown case {case}")
        if kind == "dense":
            sys_ = cho.cho_create_system(ctx, "dense", M=cfg["M"], K=cfg["K"])
        else:
            sys_ = cho.cho_create_system(ctx, kind, masses=cfg["masses"], springs=cfg["springs"])
        if case == "chain_ext":
            import numpy as np

            rng = np.random.default_rng(inputs.SEED_BASE + 6)
            C, m = cfg["springs"], cfg["masses"]
            cho.cho_system_set_damping(sys_, 0.04 * np.sqrt(C * m) * rng.uniform(0.5, 2.0, C.shape))
            cho.cho_system_set_forcing(sys_, C * rng.normal(0.0, 0.01, C.shape),
                                       cfg["omega_max"] * rng.uniform(0.05, 0.5, C.shape[0]),
                                       rng.uniform(-np.pi, np.pi, C.shape[0]))
        x0 = torch.as_tensor(cfg["x0"], device=dev)
        v0 = torch.as_tensor(cfg["v0"], device=dev)
        h = torch.as_tensor(cfg["h"], device=dev)
        cho.cho_integrate_batch(ctx, sys_, x0, v0, h, cfg["n_steps"], prec, poly_jump=poly)
        torch.cuda.synchronize()
        cho.cho_destroy_system(sys_)
    finally:
        cho.cho_shutdown(ctx)
    print(f"{case}: ok")


if __name__ == "__main__":
    for c in sys.argv[1:] or ["pair"]:
        run(c)
