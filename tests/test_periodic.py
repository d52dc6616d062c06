"""Host logic of the fixed-priority periodic mode, against a fake engine and a fake clock."""
import numpy as np
import pytest

from paper_1702_02207_gb300 import periodic


def test_release_times():
    assert periodic.release_times(0.25, 1.0) == [0.0, 0.25, 0.5, 0.75]
    assert periodic.release_times(0.3, 1.0, phase=0.1) == pytest.approx([0.1, 0.4, 0.7])
    assert periodic.release_times(2.0, 1.0) == [0.0]
    assert periodic.release_times(0.5, 0.0) == []
    with pytest.raises(ValueError):
        periodic.release_times(0.0, 1.0)


def _task(period, prio=None, name=""):
    return periodic.PeriodicTask(system=None, x0=np.zeros(2), v0=np.zeros(2), h=1e-4, n_steps=10,
                                 period=period, priority=prio, name=name)


def test_rate_monotonic_classes():
    ts = periodic.rate_monotonic([_task(0.1), _task(0.01), _task(0.05)])
    assert [t.priority for t in ts] == [2, 0, 1]
    many = periodic.rate_monotonic([_task(p) for p in (0.9, 0.1, 0.5, 0.2, 0.3, 0.7)])
    by_period = sorted(many, key=lambda t: t.period)
    assert [t.priority for t in by_period] == [0, 0, 1, 1, 2, 2]
    fixed = periodic.rate_monotonic([_task(0.5, prio=0), _task(0.1)])
    assert fixed[0].priority == 0 and fixed[1].priority == 0


class FakeEngine:
    """Each job completes a fixed service time after its submission (no contention)."""

    def __init__(self, service):
        self.t = 0.0
        self.service = service
        self.jobs = {}
        self.cancelled = []

    def clock(self):
        return self.t

    def sleep(self, dt):
        self.t += max(dt, 1e-4)

    def submit(self, task):
        tk = len(self.jobs) + 1
        self.jobs[tk] = self.t + self.service[task.name]
        return tk

    def poll(self, tk, s):
        if self.jobs[tk] is None:
            return 1, None
        if self.t >= self.jobs[tk]:
            return 0, {"t_done": self.jobs[tk]}
        return 1, None

    def cancel(self, tk):
        self.cancelled.append(tk)


def test_run_periodic_counts_responses_and_misses():
    eng = FakeEngine({"fast": 0.002, "late": 0.07})
    tasks = [_task(0.01, name="fast"), _task(0.05, name="late")]
    res = periodic.run_periodic(None, tasks, 0.2, submit=eng.submit, poll=eng.poll, cancel=eng.cancel,
                                clock=eng.clock, sleep=eng.sleep)
    fast, late = res["tasks"]
    assert fast["priority"] == 0 and late["priority"] == 1
    assert fast["jobs"] == 20 and fast["misses"] == 0
    assert fast["response_max_s"] < 0.01 and fast["response_p50_s"] >= 0.002
    assert late["jobs"] == 4 and late["misses"] == 4 and late["miss_rate"] == 1.0
    assert late["response_p50_s"] >= 0.07
    assert res["jobs"] == 24 and res["misses"] == 4


def test_run_periodic_cancels_what_never_finishes():
    eng = FakeEngine({"stuck": 1e9})
    res = periodic.run_periodic(None, [_task(0.05, name="stuck")], 0.1, submit=eng.submit, poll=eng.poll,
                                cancel=eng.cancel, clock=eng.clock, sleep=eng.sleep, drain=0.5)
    t = res["tasks"][0]
    assert t["jobs"] == 2 and t["misses"] == 2
    assert sorted(eng.cancelled) == [1, 2]
