"""Fixed-priority periodic real-time mode on top of the serving engine.

The paper's motivation (Section 5) is real-time simulation under fixed-priority
scheduling: tasks release jobs periodically and each job must finish before
its deadline.  Here a periodic task is one instance of a system that is
integrated for ``n_steps`` RK4 steps per job; it releases a job every
``period`` seconds and the deadline of a job is its next release (implicit
deadlines).  Jobs are submitted to the serving engine (``cho_submit``) with the
task's priority class, so the engine's strict fixed-priority admission is the
scheduler; this module releases the jobs on time, collects their completion
times and reports response times and deadline misses per task.

``rate_monotonic`` assigns the three priority classes by period (shorter
period, higher priority).  ``run_periodic`` takes the submit/poll functions and
the clock as arguments so that its release and accounting logic can be tested
without a GPU.
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field

import numpy as np


@dataclass
class PeriodicTask:
    """One periodic task: a single instance of ``system`` (parameter set ``sys_index``)."""

    system: object
    x0: np.ndarray
    v0: np.ndarray
    h: float
    n_steps: int
    period: float                 # seconds between releases; also the relative deadline
    priority: int | None = None   # 0 (highest) .. 2; None: set by rate_monotonic
    sys_index: int = 0
    prec: str = "fp32_kahan"
    phase: float = 0.0            # first release, seconds after the start
    name: str = ""
    s: int = field(default=0)     # degrees of freedom (for result buffers)


def rate_monotonic(tasks):
    """Priority classes by period: the shortest third of the periods gets class 0, the next
    third class 1, the rest class 2 (with three or fewer tasks: rank order).  Tasks whose
    priority is already set keep it.  Returns the tasks."""
    free = [t for t in tasks if t.priority is None]
    order = sorted(free, key=lambda t: t.period)
    n = len(order)
    for rank, t in enumerate(order):
        t.priority = min(2, rank) if n <= 3 else min(2, (3 * rank) // n)
    return tasks


def release_times(period, duration, phase=0.0):
    """Release instants phase + j * period that fall in [0, duration)."""
    if period <= 0:
        raise ValueError("period must be > 0")
    n = int(np.ceil((duration - phase) / period)) if duration > phase else 0
    return [phase + j * period for j in range(n) if phase + j * period < duration]


def run_periodic(ctx, tasks, duration, submit=None, poll=None, cancel=None, clock=time.monotonic,
                 sleep=time.sleep, drain=None, poll_interval=5e-4):
    """Release the tasks' jobs for ``duration`` seconds, wait for the outstanding ones (up to
    ``drain`` seconds, default 10 s plus twice the longest period), and return per-task
    statistics: jobs, misses, miss_rate and response-time percentiles (seconds, from release
    to the result being available).  A job still running when the drain ends is cancelled and
    counted as a miss.  ``submit(task) -> ticket``, ``poll(ticket, s) -> (status, result)``,
    ``cancel(ticket)`` default to the serving engine of ``ctx``."""
    if submit is None or poll is None or cancel is None:
        from paper_1702_02207_gb300 import cho

        submit = submit or (lambda t: cho.cho_submit(ctx, t.system, t.x0, t.v0, t.h, t.n_steps, t.prec,
                                                     t.priority, t.sys_index))
        poll = poll or (lambda tk, s: cho.cho_poll(ctx, tk, s))
        cancel = cancel or (lambda tk: cho.cho_cancel(ctx, tk))
    if any(t.priority is None for t in tasks):
        rate_monotonic(tasks)
    for t in tasks:
        if not t.s:
            t.s = int(np.asarray(t.x0).size)
    schedule = sorted((r, i) for i, t in enumerate(tasks) for r in release_times(t.period, duration, t.phase))
    if drain is None:
        drain = 10.0 + 2.0 * max((t.period for t in tasks), default=0.0)
    jobs = []                      # [task, nominal release (s after start), release clock, ticket, done clock]
    pending = {}
    t0 = clock()
    nxt = 0
    while nxt < len(schedule) or pending:
        now = clock() - t0
        while nxt < len(schedule) and schedule[nxt][0] <= now:
            rel, i = schedule[nxt]
            nxt += 1
            job = [i, rel, clock(), submit(tasks[i]), None]
            jobs.append(job)
            pending[job[3]] = job
        for tk in list(pending):
            job = pending[tk]
            try:
                st, res = poll(tk, tasks[job[0]].s)
            except Exception as e:                  # the request failed (its status is in the error)
                st, res = getattr(e, "status", -1), None
            if res is not None or st != 1:          # CHO_PENDING == 1
                # completion on the engine's clock when it reports one (the same monotonic
                # clock as time.monotonic), else when this loop saw it
                job[4] = res["t_done"] if res and "t_done" in res else clock()
                job.append(st)
                del pending[tk]
        if nxt >= len(schedule) and pending and clock() - t0 > duration + drain:
            for tk, job in list(pending.items()):
                cancel(tk)
                job[4] = None
                job.append("unfinished")
                del pending[tk]
            break
        wait = poll_interval
        if nxt < len(schedule):
            wait = min(wait, max(0.0, schedule[nxt][0] - (clock() - t0)))
        if wait > 0:
            sleep(wait)
    out = []
    total_jobs = total_miss = 0
    for i, t in enumerate(tasks):
        mine = [j for j in jobs if j[0] == i]
        resp = []
        miss = 0
        for j in mine:
            if j[4] is None or j[5] != 0:
                miss += 1
                continue
            r = j[4] - (t0 + j[1])               # from the nominal release to completion
            resp.append(r)
            if r > t.period:
                miss += 1
        total_jobs += len(mine)
        total_miss += miss
        rs = np.asarray(resp) if resp else np.zeros(1)
        out.append({"name": t.name or f"task{i}", "period_s": t.period, "priority": t.priority,
                    "n_steps": t.n_steps, "jobs": len(mine), "misses": miss,
                    "miss_rate": miss / len(mine) if mine else 0.0,
                    "response_p50_s": float(np.percentile(rs, 50)), "response_p99_s": float(np.percentile(rs, 99)),
                    "response_max_s": float(rs.max())})
    return {"tasks": out, "jobs": total_jobs, "misses": total_miss,
            "miss_rate": total_miss / total_jobs if total_jobs else 0.0, "duration_s": duration}
