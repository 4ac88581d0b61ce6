"""The serving leg's request driver in bench.py (no GPU): against a stand-in server that finishes
each request after a fixed number of ticks, every request is submitted, ticked to completion and
timed, whether the requests arrive spread out or all at once (the saturation pass)."""
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


class _Spec:
    def __init__(self, k):
        self.method, self.nx, self.ny, self.h, self.dt, self.c, self.steps = 0, 16, 16, 1.0, 0.1, None, 10
        self.source = type("S", (), {"as_tuple": lambda self_: (1, 1, 1.0, 1.0, 0.0)})()


class _Req:
    def __init__(self, k):
        self.spec = _Spec(k)


class _FakeServer:
    """Admits up to two requests at a time; a running request finishes after three ticks."""

    instances = []

    def __init__(self, budget, precision=0, quantum=100, max_active=64):
        self.t0 = time.perf_counter()
        self.reqs = {}   # ticket -> [submit, start, done, ticks left]
        self.queue = []
        _FakeServer.instances.append(self)

    def now(self):
        return time.perf_counter() - self.t0

    def submit(self, *a, **k):
        t = len(self.reqs)
        self.reqs[t] = [self.now(), -1.0, -1.0, 3]
        self.queue.append(t)
        return t

    def tick(self):
        running = [t for t, r in self.reqs.items() if r[1] >= 0 and r[2] < 0]
        while self.queue and len(running) < 2:
            t = self.queue.pop(0)
            self.reqs[t][1] = self.now()
            running.append(t)
        for t in running:
            r = self.reqs[t]
            r[3] -= 1
            if r[3] == 0:
                r[2] = self.now()
        running = [t for t in running if self.reqs[t][2] < 0]
        return len(running), len(self.queue)

    def status(self, t):
        r = self.reqs[t]
        return (2 if r[2] >= 0 else 1), r[0], r[1], r[2]

    def close(self):
        pass


class _FakeAdi:
    ADI_FP32 = 0
    Server = _FakeServer


def test_all_requests_at_once_are_run_to_completion():
    reqs = [_Req(k) for k in range(7)]
    wall, lat = bench._run_server(_FakeAdi, reqs, [0.0] * len(reqs))
    srv = _FakeServer.instances[-1]
    assert len(srv.reqs) == 7 and all(r[2] >= 0 for r in srv.reqs.values())
    assert len(lat) == 7 and all(x >= 0 for x in lat) and wall > 0


def test_spread_arrivals_are_run_to_completion():
    reqs = [_Req(k) for k in range(5)]
    arrivals = [0.0, 0.01, 0.02, 0.05, 0.05]
    wall, lat = bench._run_server(_FakeAdi, reqs, arrivals)
    srv = _FakeServer.instances[-1]
    assert all(r[2] >= 0 for r in srv.reqs.values())
    assert len(lat) == 5 and all(x >= 0 for x in lat) and wall >= 0.05
