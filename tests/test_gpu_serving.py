"""Serving: continuous batching through cho_submit / cho_poll.

Checks that a request's result is the same alone and inside a mixed stream,
the same for any chunk length, equal to the batch API and to the oracle within
tolerance; that admission follows the fixed priorities and the memory budget;
and that bad requests get clean status codes (faults are made on the host).
"""
import math
import time

import numpy as np
import pytest

from paper_1702_02207_gb300 import cho, inputs
from parity_util import TOL_FP32, TOL_FP64, oracle_run

pytestmark = pytest.mark.gpu


def wait_all(ctx, tickets, sizes, timeout=120.0):
    out = {}
    t0 = time.time()
    pending = dict(zip(tickets, sizes))
    while pending:
        for t in list(pending):
            try:
                st, res = cho.cho_poll(ctx, t, pending[t])
            except cho.ChoError as e:
                out[t] = e.status
                del pending[t]
                continue
            if st == cho.CHO_OK:
                out[t] = res
                del pending[t]
        if time.time() - t0 > timeout:
            raise TimeoutError(f"{len(pending)} requests still pending")
        time.sleep(0.002)
    return out


class Mix:
    """A few systems of each kernel family and a seeded list of requests on them."""

    def __init__(self, ctx, seed=0):
        self.ctx = ctx
        rng = np.random.default_rng(seed)
        self.systems = []
        two = inputs.two_dof_batch(n_inst=64, n_steps=1)
        self.systems.append(("two_dof", cho.cho_create_system(ctx, "two_dof", masses=two["masses"], springs=two["springs"]),
                             two, 2))
        for s in (5, 40, 300):
            ch = inputs.chain_batch(n_inst=16, s=s, n_steps=1, seed=70 + s)
            self.systems.append(("chain", cho.cho_create_system(ctx, "chain", masses=ch["masses"], springs=ch["springs"]),
                                 ch, s))
        for s in (12, 64):
            dn = inputs.dense_group(s=s, n_inst=1, n_steps=1)
            self.systems.append(("dense", cho.cho_create_system(ctx, "dense", M=dn["M"], K=dn["K"]), dn, s))
        self.rng = rng

    def request(self, k, n_steps=None, prec="fp32_kahan"):
        kind, sys_, cfg, s = self.systems[k % len(self.systems)]
        n_sys = cfg["masses"].shape[0] if kind != "dense" else 1
        idx = int(self.rng.integers(n_sys))
        x0 = self.rng.uniform(-1, 1, s)
        h = float(cfg["h"][idx if kind != "dense" else 0])
        n = int(self.rng.integers(500, 4000)) if n_steps is None else n_steps
        return dict(kind=kind, sys=sys_, cfg=cfg, s=s, idx=idx, x0=x0, v0=np.zeros(s), h=h, n=n, prec=prec)

    def submit(self, r, priority=2):
        return cho.cho_submit(self.ctx, r["sys"], r["x0"], r["v0"], r["h"], r["n"], r["prec"], priority, r["idx"])

    def close(self):
        for _, s, _, _ in self.systems:
            cho.cho_destroy_system(s)


def reference(r):
    """Oracle result of one request."""
    cfg = r["cfg"]
    if r["kind"] == "dense":
        c = dict(kind="dense", M=cfg["M"], K=cfg["K"], x0=r["x0"][None], v0=r["v0"][None], h=np.array([r["h"]]))
    else:
        i = r["idx"]
        c = dict(kind="chain", masses=cfg["masses"][i:i + 1], springs=cfg["springs"][i:i + 1], x0=r["x0"][None],
                 v0=r["v0"][None], h=np.array([r["h"]]))
    return oracle_run(c, n_steps=r["n"])


def batch_result(ctx, r):
    """The same instance through cho_integrate_batch (same kernel family and precision)."""
    cfg = r["cfg"]
    if r["kind"] == "dense":
        sys_ = r["sys"]
        out = cho.cho_integrate_batch(ctx, sys_, r["x0"][None], r["v0"][None], [r["h"]], r["n"], r["prec"])
        return out
    i = r["idx"]
    sys_ = cho.cho_create_system(ctx, r["kind"], masses=cfg["masses"][i:i + 1], springs=cfg["springs"][i:i + 1])
    try:
        return cho.cho_integrate_batch(ctx, sys_, r["x0"][None], r["v0"][None], [r["h"]], r["n"], r["prec"])
    finally:
        cho.cho_destroy_system(sys_)


def relerr(a, b):
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)


@pytest.mark.parametrize("prec,tol", [("fp32_kahan", TOL_FP32), ("fp64", TOL_FP64)])
def test_alone_matches_batch_and_oracle(prec, tol):
    ctx = cho.cho_init(0, chunk_steps=700)
    mix = Mix(ctx, seed=1)
    try:
        for k in range(len(mix.systems)):
            r = mix.request(k, prec=prec)
            t = mix.submit(r)
            res = wait_all(ctx, [t], [r["s"]])[t]
            b = batch_result(ctx, r)
            assert np.array_equal(res["x"], b["x"][0]) and np.array_equal(res["v"], b["v"][0]), r["kind"]
            ref = reference(r)
            assert relerr(res["x"], ref["x"][0]) < 50 * tol
            assert res["t_submit"] <= res["t_admit"] <= res["t_done"]
    finally:
        mix.close()
        cho.cho_shutdown(ctx)


def test_same_result_alone_and_in_the_mix_and_any_chunk():
    ctx = cho.cho_init(0, chunk_steps=512)
    mix = Mix(ctx, seed=2)
    try:
        probes = [mix.request(k) for k in range(len(mix.systems))]
        alone = {}
        for k, r in enumerate(probes):
            t = mix.submit(r)
            alone[k] = wait_all(ctx, [t], [r["s"]])[t]
        # the same requests inside a stream of 300 others of all kinds and priorities
        others = [mix.request(k) for k in range(300)]
        tickets, sizes, which = [], [], []
        for j, r in enumerate(others):
            tickets.append(mix.submit(r, priority=j % 3))
            sizes.append(r["s"])
            which.append(None)
            if j % 50 == 25:
                k = (j // 50) % len(probes)
                tickets.append(mix.submit(probes[k], priority=(j // 50) % 3))
                sizes.append(probes[k]["s"])
                which.append(k)
        res = wait_all(ctx, tickets, sizes)
        seen = 0
        for t, k in zip(tickets, which):
            if k is not None:
                assert np.array_equal(res[t]["x"], alone[k]["x"]) and np.array_equal(res[t]["v"], alone[k]["v"])
                seen += 1
        assert seen == 6
    finally:
        mix.close()
        cho.cho_shutdown(ctx)
    # chunk length does not change results (state stays in kernel precision between chunks)
    for chunk in (97, 100000):
        ctx = cho.cho_init(0, chunk_steps=chunk)
        mix2 = Mix(ctx, seed=2)
        try:
            for k, r in enumerate(probes):
                r2 = dict(r, sys=mix2.systems[k][1])
                t = mix2.submit(r2)
                got = wait_all(ctx, [t], [r["s"]])[t]
                assert np.array_equal(got["x"], alone[k]["x"]), (chunk, k)
        finally:
            mix2.close()
            cho.cho_shutdown(ctx)


def test_tuned_chunk_length_keeps_results():
    """With chunk_us set, each kernel group retunes its chunk length from the measured
    device time of its launches; results stay those of the batch API, bit for bit."""
    ctx = cho.cho_init(0, chunk_steps=64, chunk_us=300)
    mix = Mix(ctx, seed=4)
    try:
        reqs = [mix.request(k, n_steps=3000) for k in range(len(mix.systems))]
        tickets = [mix.submit(r, priority=k % 3) for k, r in enumerate(reqs)]
        res = wait_all(ctx, tickets, [r["s"] for r in reqs])
        for t, r in zip(tickets, reqs):
            b = batch_result(ctx, r)
            assert np.array_equal(res[t]["x"], b["x"][0]) and np.array_equal(res[t]["v"], b["v"][0]), r["kind"]
    finally:
        mix.close()
        cho.cho_shutdown(ctx)


def test_mixed_stream_against_oracle():
    ctx = cho.cho_init(0, chunk_steps=1000)
    mix = Mix(ctx, seed=3)
    try:
        reqs = [mix.request(k) for k in range(120)]
        tickets = [mix.submit(r, priority=k % 3) for k, r in enumerate(reqs)]
        res = wait_all(ctx, tickets, [r["s"] for r in reqs])
        for t, r in zip(tickets, reqs):
            ref = reference(r)
            assert relerr(res[t]["x"], ref["x"][0]) < 1e-4, (r["kind"], r["s"])
        st = cho.cho_serve_stats(ctx)
        assert st["queued"] == 0 and st["resident"] == 0 and st["completed"] >= 120
    finally:
        mix.close()
        cho.cho_shutdown(ctx)


def test_fixed_priority_admission_and_budget():
    # two slots at a time: admission order is decided by priority class, FIFO inside a class
    ctx = cho.cho_init(0, chunk_steps=200, max_slots=2)
    mix = Mix(ctx, seed=4)
    try:
        low = [mix.request(0, n_steps=2000) for _ in range(8)]
        high = [mix.request(0, n_steps=2000) for _ in range(8)]
        tl = [mix.submit(r, priority=2) for r in low]
        th = [mix.submit(r, priority=0) for r in high]
        peak = 0
        t0 = time.time()
        while time.time() - t0 < 60:
            st = cho.cho_serve_stats(ctx)
            peak = max(peak, st["resident"])
            if st["queued"] == 0 and st["resident"] == 0:
                break
            time.sleep(0.001)
        res = wait_all(ctx, tl + th, [2] * 16)
        assert peak <= 2
        adm_low = sorted(res[t]["t_admit"] for t in tl)
        adm_high = [res[t]["t_admit"] for t in th]
        # at most the two low-priority requests admitted before the high ones arrived run first
        assert sum(a < max(adm_high) for a in adm_low) <= 2
        # FIFO inside the high class
        assert adm_high == sorted(adm_high)
    finally:
        mix.close()
        cho.cho_shutdown(ctx)
    # a byte budget of one FP32 state block of s = 300 (4.8 KB -> 8 KB class) serialises chain requests
    ctx = cho.cho_init(0, chunk_steps=300, budget_bytes=8192)
    mix = Mix(ctx, seed=5)
    try:
        reqs = [mix.request(3, n_steps=900) for _ in range(4)]
        ts = [mix.submit(r) for r in reqs]
        peak_bytes = 0
        t0 = time.time()
        while time.time() - t0 < 60:
            st = cho.cho_serve_stats(ctx)
            peak_bytes = max(peak_bytes, st["resident_bytes"])
            if st["queued"] == 0 and st["resident"] == 0:
                break
        wait_all(ctx, ts, [300] * 4)
        assert 0 < peak_bytes <= 8192
        # a chain of 2000 masses in FP64 needs a 32 KiB block: it can never fit, so submit refuses it
        big = inputs.chain_batch(n_inst=1, s=2000, n_steps=1)
        sb = cho.cho_create_system(ctx, "chain", masses=big["masses"], springs=big["springs"])
        try:
            with pytest.raises(cho.ChoError) as ei:
                cho.cho_submit(ctx, sb, np.zeros(2000), np.zeros(2000), float(big["h"][0]), 10, "fp64")
            assert ei.value.status == cho.CHO_EBUDGET
        finally:
            cho.cho_destroy_system(sb)
    finally:
        mix.close()
        cho.cho_shutdown(ctx)


def test_request_errors_and_cancel():
    ctx = cho.cho_init(0, chunk_steps=100, max_slots=1)
    mix = Mix(ctx, seed=6)
    try:
        r = mix.request(0)
        with pytest.raises(cho.ChoError) as ei:
            cho.cho_submit(ctx, r["sys"], r["x0"], r["v0"], 10.0, 10, "fp32_kahan", 0, r["idx"])
        assert ei.value.status == cho.CHO_EUNSTABLE
        with pytest.raises(cho.ChoError) as ei:
            cho.cho_submit(ctx, r["sys"], [np.nan, 0.0], r["v0"], r["h"], 10, "fp32_kahan", 0, r["idx"])
        assert ei.value.status == cho.CHO_ENONFINITE
        with pytest.raises(cho.ChoError) as ei:
            cho.cho_submit(ctx, r["sys"], r["x0"], r["v0"], r["h"], 10, "fp32_kahan", 3, r["idx"])
        assert ei.value.status == cho.CHO_EINVAL
        with pytest.raises(cho.ChoError) as ei:
            cho.cho_submit(ctx, r["sys"], r["x0"], r["v0"], r["h"], 10, "fp32_kahan", 0, 10_000)
        assert ei.value.status == cho.CHO_EINVAL
        with pytest.raises(cho.ChoError) as ei:
            cho.cho_poll(ctx, 987654321, 2)
        assert ei.value.status == cho.CHO_ENOTFOUND
        # cancel a long request while it runs, and one still queued behind it
        t1 = cho.cho_submit(ctx, r["sys"], r["x0"], r["v0"], r["h"], 10_000_000, "fp32_kahan", 0, r["idx"])
        t2 = cho.cho_submit(ctx, r["sys"], r["x0"], r["v0"], r["h"], 10_000_000, "fp32_kahan", 2, r["idx"])
        time.sleep(0.05)
        cho.cho_cancel(ctx, t1)
        cho.cho_cancel(ctx, t2)
        out = wait_all(ctx, [t1, t2], [2, 2], timeout=60)
        assert out[t1] == cho.CHO_ECANCELLED and out[t2] == cho.CHO_ECANCELLED
        # a finite start that overflows FP32 in flight is reported at a chunk boundary,
        # without disturbing a healthy request served beside it
        ok = mix.request(0, n_steps=300)
        t3 = cho.cho_submit(ctx, r["sys"], [3e38, -3e38], [3e38, 3e38], r["h"], 500, "fp32_kahan", 0, r["idx"])
        t4 = mix.submit(ok, priority=0)
        out = wait_all(ctx, [t3, t4], [2, 2])
        assert out[t3] == cho.CHO_ENONFINITE
        assert np.array_equal(out[t4]["x"], batch_result(ctx, ok)["x"][0])
    finally:
        mix.close()
        cho.cho_shutdown(ctx)


def test_dense_requests_on_tensor_cores():
    """Dense requests in a BF16 mode run on the tensor-core kernel in slot form: same bits as the
    batch call, within the bf16x5 tolerance of the oracle, and the same alone and in a mix."""
    ctx = cho.cho_init(0, chunk_steps=300)
    try:
        systems = []
        for s in (64, 200):
            dn = inputs.dense_group(s=s, n_inst=1, n_steps=1)
            systems.append((cho.cho_create_system(ctx, "dense", M=dn["M"], K=dn["K"]), dn, s))
        rng = np.random.default_rng(9)
        reqs = []
        for k in range(40):
            sys_, dn, s = systems[k % 2]
            reqs.append(dict(kind="dense", sys=sys_, cfg=dn, s=s, idx=0, x0=rng.uniform(-1, 1, s), v0=np.zeros(s),
                             h=float(dn["h"][0]), n=int(rng.integers(200, 1500)), prec="bf16x5"))
        tickets = [cho.cho_submit(ctx, r["sys"], r["x0"], r["v0"], r["h"], r["n"], "bf16x5", k % 3) for k, r in enumerate(reqs)]
        res = wait_all(ctx, tickets, [r["s"] for r in reqs])
        for t, r in list(zip(tickets, reqs))[:6]:
            b = batch_result(ctx, r)
            assert np.array_equal(res[t]["x"], b["x"][0])
            ref = reference(r)
            assert relerr(res[t]["x"], ref["x"][0]) < 5 * TOL_FP32
        # alone
        r = reqs[3]
        t = cho.cho_submit(ctx, r["sys"], r["x0"], r["v0"], r["h"], r["n"], "bf16x5", 0)
        alone = wait_all(ctx, [t], [r["s"]])[t]
        assert np.array_equal(alone["x"], res[tickets[3]]["x"])
        for sys_, _, _ in systems:
            cho.cho_destroy_system(sys_)
    finally:
        cho.cho_shutdown(ctx)


# ---- fixed-priority periodic mode (the paper's real-time framing) ----------------------------

def _periodic_tasks(ctx):
    from paper_1702_02207_gb300 import periodic

    two = inputs.two_dof_batch(n_inst=1, n_steps=1)
    ch = inputs.chain_batch(n_inst=1, s=64, n_steps=1, seed=91)
    dn = inputs.dense_group(s=64, n_inst=1, n_steps=1)
    s2 = cho.cho_create_system(ctx, "two_dof", masses=two["masses"], springs=two["springs"])
    sc = cho.cho_create_system(ctx, "chain", masses=ch["masses"], springs=ch["springs"])
    sd = cho.cho_create_system(ctx, "dense", M=dn["M"], K=dn["K"])
    tasks = [
        periodic.PeriodicTask(s2, two["x0"][0], two["v0"][0], float(two["h"][0]), 2000, 0.05, name="two_dof"),
        periodic.PeriodicTask(sc, ch["x0"][0], ch["v0"][0], float(ch["h"][0]), 2000, 0.1, name="chain64"),
        periodic.PeriodicTask(sd, dn["x0"][0], dn["v0"][0], float(dn["h"][0]), 1000, 0.2, prec="bf16x5",
                              name="dense64"),
    ]
    return tasks, (s2, sc, sd)


def test_periodic_mode_meets_light_deadlines():
    """Three periodic tasks (50, 100, 200 ms) with jobs of a few ms: rate-monotonic classes,
    every job on time, results equal to the batch API."""
    from paper_1702_02207_gb300 import periodic

    ctx = cho.cho_init(0, chunk_steps=1000)
    try:
        tasks, systems = _periodic_tasks(ctx)
        warm = [cho.cho_submit(ctx, t.system, t.x0, t.v0, t.h, t.n_steps, t.prec, 0) for t in tasks]
        got = wait_all(ctx, warm, [2, 64, 64])
        ref = cho.cho_integrate_batch(ctx, tasks[0].system, tasks[0].x0[None], tasks[0].v0[None], tasks[0].h,
                                      2000, "fp32_kahan")
        assert np.array_equal(got[warm[0]]["x"], ref["x"][0])
        res = periodic.run_periodic(ctx, tasks, 1.5)
        by = {t["name"]: t for t in res["tasks"]}
        assert [by[n]["priority"] for n in ("two_dof", "chain64", "dense64")] == [0, 1, 2]
        assert by["two_dof"]["jobs"] == 30 and by["chain64"]["jobs"] == 15 and by["dense64"]["jobs"] == 8
        assert res["misses"] == 0, res
        for s in systems:
            cho.cho_destroy_system(s)
    finally:
        cho.cho_shutdown(ctx)


def test_periodic_mode_reports_overload():
    """A task whose job (a 1024-mass chain for 1e5 steps) outlasts its 10 ms period misses every
    deadline and the count says so."""
    from paper_1702_02207_gb300 import periodic

    ctx = cho.cho_init(0, chunk_steps=5000)
    try:
        ch = inputs.chain_batch(n_inst=1, s=1024, n_steps=1, seed=92)
        sc = cho.cho_create_system(ctx, "chain", masses=ch["masses"], springs=ch["springs"])
        task = periodic.PeriodicTask(sc, ch["x0"][0], ch["v0"][0], float(ch["h"][0]), 100000, 0.01, name="heavy")
        res = periodic.run_periodic(ctx, [task], 0.05)
        t = res["tasks"][0]
        assert t["jobs"] == 5 and t["misses"] == 5 and t["response_p50_s"] > 0.01
        cho.cho_destroy_system(sc)
    finally:
        cho.cho_shutdown(ctx)


def test_dense_requests_with_their_own_k():
    """Dense requests on a system with one (M, K) per parameter set: each request runs on its
    set's B, with the bits of the batch API and within tolerance of the oracle."""
    ctx = cho.cho_init(0, chunk_steps=250)
    try:
        cfg = inputs.dense_own(s=70, n_inst=5, n_steps=600)
        sys_ = cho.cho_create_system(ctx, "dense", M=cfg["M"], K=cfg["K"])
        tickets = [cho.cho_submit(ctx, sys_, cfg["x0"][i], cfg["v0"][i], float(cfg["h"][i]), 600, "fp32_kahan",
                                  i % 3, sys_index=i) for i in range(5)]
        got = wait_all(ctx, tickets, [70] * 5)
        b = cho.cho_integrate_batch(ctx, sys_, cfg["x0"], cfg["v0"], cfg["h"], 600, "fp32_kahan")
        ref = oracle_run(cfg)
        for i, t in enumerate(tickets):
            assert np.array_equal(got[t]["x"], b["x"][i]) and np.array_equal(got[t]["v"], b["v"][i])
            assert np.max(np.abs(got[t]["x"] - ref["x"][i])) / np.max(np.abs(ref["x"][i])) < TOL_FP32
        with pytest.raises(cho.ChoError) as ei:
            cho.cho_submit(ctx, sys_, cfg["x0"][0], cfg["v0"][0], float(cfg["h"][0]), 10, "bf16x5", 0)
        assert ei.value.status == cho.CHO_EINVAL
        cho.cho_destroy_system(sys_)
    finally:
        cho.cho_shutdown(ctx)


# ---- persistent serving -------------------------------------------------------------------

def test_persistent_mode_gives_the_bits_of_the_relaunch_mode():
    """The same requests served by resident kernels (small and chain groups: doorbell per
    chunk, completion ring, mapped slot table) and by per-chunk launches: bitwise equal results,
    alone and inside a mixed stream of 300 others, and equal to the batch API."""
    ref_ctx = cho.cho_init(0, chunk_steps=512)
    ref_mix = Mix(ref_ctx, seed=5)
    probes = [ref_mix.request(k) for k in range(len(ref_mix.systems))]
    others = [ref_mix.request(k) for k in range(300)]
    try:
        t = [ref_mix.submit(r, priority=k % 3) for k, r in enumerate(probes + others)]
        ref = wait_all(ref_ctx, t, [r["s"] for r in probes + others])
        ref = [ref[x] for x in t]
        for r, got in zip(probes, ref[:len(probes)]):
            b = batch_result(ref_ctx, r)
            assert np.array_equal(got["x"], b["x"][0]) and np.array_equal(got["v"], b["v"][0]), r["kind"]
    finally:
        ref_mix.close()
        cho.cho_shutdown(ref_ctx)
    for chunk in (512, 97):
        ctx = cho.cho_init(0, chunk_steps=chunk, persistent=1)
        mix = Mix(ctx, seed=5)
        try:
            reqs = [dict(r, sys=mix.systems[k % len(mix.systems)][1]) for k, r in enumerate(probes)]
            reqs += [dict(r, sys=mix.systems[k % len(mix.systems)][1]) for k, r in enumerate(others)]
            t = [mix.submit(r, priority=k % 3) for k, r in enumerate(reqs)]
            got = wait_all(ctx, t, [r["s"] for r in reqs])
            for x, want in zip(t, ref):
                assert not isinstance(got[x], int), got[x]
                assert np.array_equal(got[x]["x"], want["x"]) and np.array_equal(got[x]["v"], want["v"]), chunk
            # the resident kernels leave when their groups empty; a later request starts them again
            r2 = reqs[0]
            t2 = mix.submit(r2)
            again = wait_all(ctx, [t2], [r2["s"]])[t2]
            assert np.array_equal(again["x"], ref[0]["x"])
        finally:
            mix.close()
            cho.cho_shutdown(ctx)


def test_persistent_mode_doorbell_wait_runs_out_cleanly():
    """Test hook: the serving thread never rings the resident kernels' doorbell, so their
    bounded waits run out (about a second): the requests end with CHO_ETIMEOUT and nothing
    hangs; a new context without the hook serves normally."""
    import os

    os.environ["CHO_TEST_WITHHOLD_DOORBELL"] = "1"
    try:
        ctx = cho.cho_init(0, chunk_steps=256, persistent=1)
        mix = Mix(ctx, seed=6)
        try:
            reqs = [mix.request(0, n_steps=300), mix.request(2, n_steps=300)]     # 2-DOF and a 40-mass chain
            t = [mix.submit(r) for r in reqs]
            t0 = time.time()
            got = wait_all(ctx, t, [r["s"] for r in reqs], timeout=30.0)
            assert all(got[x] == cho.CHO_ETIMEOUT for x in t), got
            assert time.time() - t0 < 20.0
        finally:
            mix.close()
            cho.cho_shutdown(ctx)
    finally:
        del os.environ["CHO_TEST_WITHHOLD_DOORBELL"]
    ctx = cho.cho_init(0, chunk_steps=256, persistent=1)
    mix = Mix(ctx, seed=6)
    try:
        r = mix.request(0, n_steps=300)
        t = mix.submit(r)
        got = wait_all(ctx, [t], [r["s"]])[t]
        b = batch_result(ctx, r)
        assert np.array_equal(got["x"], b["x"][0])
    finally:
        mix.close()
        cho.cho_shutdown(ctx)


def test_poll_any_returns_every_finished_request_once():
    """cho_poll_any hands out finished requests of any ticket, each once, with the timings
    cho_poll gives; tickets collected by cho_poll are skipped."""
    ctx = cho.cho_init(0, chunk_steps=300)
    mix = Mix(ctx, seed=7)
    try:
        reqs = [mix.request(k, n_steps=600) for k in range(24)]
        tickets = [mix.submit(r, priority=k % 3) for k, r in enumerate(reqs)]
        got = {}
        by_poll = wait_all(ctx, tickets[:4], [r["s"] for r in reqs[:4]])      # four through cho_poll
        t0 = time.time()
        while len(got) < len(tickets) - 4 and time.time() - t0 < 60:
            code, t, tm = cho.cho_poll_any(ctx)
            if code == cho.CHO_PENDING:
                time.sleep(0.002)
                continue
            assert code == cho.CHO_OK and t not in got and t not in by_poll
            assert tm["t_submit"] <= tm["t_admit"] <= tm["t_done"]
            got[t] = tm
        assert sorted(got) == sorted(tickets[4:])
        assert cho.cho_poll_any(ctx)[0] == cho.CHO_PENDING
    finally:
        mix.close()
        cho.cho_shutdown(ctx)


@pytest.mark.parametrize("persistent", [0, 1])
def test_active_set_preempts_lower_classes(persistent):
    """Active set capped at 1 % of one wave of the device: of twelve class-2 chains of 2048
    masses only a few run at a time and the others stay resident, waiting at their chunk
    boundary; a class-0 request submitted right after them takes the place of a running
    class-2 request at its next chunk boundary and finishes before the class-2 requests that
    waited.  Every result is bitwise that of a context without the cap."""
    rng = np.random.default_rng(9)
    ch = inputs.chain_batch(n_inst=2, s=2048, n_steps=1, seed=2048)
    x0s = [rng.uniform(-1, 1, 2048) for _ in range(13)]
    prios = [2] * 12 + [0]

    def run(ctx):
        sys_ = cho.cho_create_system(ctx, "chain", masses=ch["masses"], springs=ch["springs"])
        try:
            tickets = [cho.cho_submit(ctx, sys_, x0s[k], np.zeros(2048), float(ch["h"][k % 2]), 20000,
                                      "fp32_kahan", prios[k], k % 2) for k in range(13)]
            res = wait_all(ctx, tickets, [2048] * 13)
            return [res[tk] for tk in tickets]
        finally:
            cho.cho_destroy_system(sys_)

    ctx = cho.cho_init(0, chunk_steps=500, active_pct=1, persistent=persistent)
    try:
        got = run(ctx)
    finally:
        cho.cho_shutdown(ctx)
    later = sum(got[k]["t_done"] > got[12]["t_done"] for k in range(12))
    assert later >= 8, later
    ctx = cho.cho_init(0, chunk_steps=500, active_pct=-1)
    try:
        ref = run(ctx)
    finally:
        cho.cho_shutdown(ctx)
    for k in range(13):
        assert np.array_equal(got[k]["x"], ref[k]["x"]) and np.array_equal(got[k]["v"], ref[k]["v"]), k


@pytest.mark.parametrize("persistent", [0, 1])
def test_serve_traffic_counts_chunk_boundary_state(persistent):
    """cho_serve_traffic: with a fixed chunk length L every chain request of s masses and n steps
    is advanced in ceil(n / L) chunks, each reading and writing back its FP32 state block
    (x, v and both compensations: 16 s bytes) once, and advances s n DOF-steps in all."""
    L = 300
    ctx = cho.cho_init(0, chunk_steps=L, persistent=persistent)
    mix = Mix(ctx, seed=10)
    try:
        reqs = [mix.request(k, n_steps=n) for k, n in zip((2, 3, 2, 3, 2), (900, 1000, 301, 299, 1))]
        t = [mix.submit(r) for r in reqs]
        got = wait_all(ctx, t, [r["s"] for r in reqs])
        assert all(not isinstance(got[x], int) for x in t)
        tr = cho.cho_serve_traffic(ctx)
        assert tr["dof_steps"] == sum(r["s"] * r["n"] for r in reqs)
        assert tr["state_bytes"] == sum(2 * 16 * r["s"] * -(-r["n"] // L) for r in reqs)
    finally:
        mix.close()
        cho.cho_shutdown(ctx)


def test_cancel_ends_a_paused_request_at_once():
    """A cancelled request that waits resident outside the active set (cap at 1 % of a wave:
    three of eight chains of 2048 masses run) ends with CHO_ECANCELLED at the engine's next
    scheduling point, while the requests that run are still running."""
    rng = np.random.default_rng(11)
    ch = inputs.chain_batch(n_inst=2, s=2048, n_steps=1, seed=2049)
    ctx = cho.cho_init(0, chunk_steps=500, active_pct=1)
    sys_ = cho.cho_create_system(ctx, "chain", masses=ch["masses"], springs=ch["springs"])
    try:
        tickets = [cho.cho_submit(ctx, sys_, rng.uniform(-1, 1, 2048), np.zeros(2048), float(ch["h"][0]), 60000,
                                  "fp32_kahan", 2, 0) for _ in range(8)]
        time.sleep(0.02)
        cho.cho_cancel(ctx, tickets[-1])
        t0 = time.time()
        while True:
            try:
                st, _ = cho.cho_poll(ctx, tickets[-1], 2048)
            except cho.ChoError as e:
                assert e.status == cho.CHO_ECANCELLED
                break
            assert st == cho.CHO_PENDING
            assert time.time() - t0 < 5.0
            time.sleep(0.001)
        first, _ = cho.cho_poll(ctx, tickets[0], 2048)
        assert first == cho.CHO_PENDING              # the running requests are not through yet
        wait_all(ctx, tickets[:-1], [2048] * 7)
    finally:
        cho.cho_destroy_system(sys_)
        cho.cho_shutdown(ctx)
