"""CPU checks of the serving loop's host logic with a stand-in solver (whose
polled solves take 10 ms): slots, a member's Newton steps in order and never
concurrent, admission under the HBM budget with least-recently-used eviction
of idle members, values-only updates for an unchanged pattern, and errors
raised to the caller.  The CUDA path of the same loop is tested on the GPU
(tests/test_gpu_serve.py)."""
import threading
import time
from types import SimpleNamespace

import numpy as np
import pytest

from paper_2201_01970_b300 import serve


class FakeSolver:
    """Records what the server asks of a handle; solve sleeps a little."""

    log = []
    active = 0
    peak = 0
    lock = threading.Lock()

    def __init__(self, A, member, fail_at=None):
        self.member, self.fail_at, self.updates = member, fail_at, 0
        FakeSolver.log.append(("open", member))

    def update(self, A):
        self.updates += 1

    def update_values(self, val):
        self.updates += 1

    def solve_start(self, b, x, rtol):
        with FakeSolver.lock:
            FakeSolver.active += 1
            FakeSolver.peak = max(FakeSolver.peak, FakeSolver.active)
        self.x, self.t_end = x, time.perf_counter() + 0.01   # the "device" takes 10 ms

    def poll(self):
        if time.perf_counter() < self.t_end:
            return None
        with FakeSolver.lock:
            FakeSolver.active -= 1
        if self.fail_at is not None and self.updates == self.fail_at:
            raise RuntimeError("solve failed")
        return self.x, {"iters": 3, "setup_called": int(self.updates == 0)}

    def close(self):
        FakeSolver.log.append(("close", self.member))


class FakeServer(serve.Server):
    def __init__(self, *a, fail=None, **kw):
        super().__init__(*a, **kw)
        self.fail = fail or {}

    def _open(self, A):
        return FakeSolver(A, A.member, self.fail.get(A.member))


def requests(members, steps, nb=100, nnzb=500, gap=0.0):
    out, t = [], 0.0
    for k in range(steps):
        for m in range(members):
            A = SimpleNamespace(nb=nb, col=np.zeros(nnzb, np.int32), val=np.zeros(9 * nnzb), member=m)
            out.append(serve.Request(m, k, A, np.zeros(3 * nb), t))
            t += gap
    return out


@pytest.fixture(autouse=True)
def reset():
    FakeSolver.log, FakeSolver.active, FakeSolver.peak = [], 0, 0


def test_slots_and_member_order():
    reqs = requests(members=6, steps=4)
    srv = FakeServer(slots=3, hbm_budget=1 << 40)
    res = srv.run(reqs, realtime=False)
    assert res["requests"] == 24 and FakeSolver.peak <= 3 and FakeSolver.peak >= 2
    for m in range(6):
        mine = sorted((r for r in reqs if r.member == m), key=lambda r: r.step)
        for a, b in zip(mine, mine[1:]):
            assert a.end <= b.start          # a member's steps run one after another, in order
    assert res["setups"] == 6 and res["evictions"] == 0
    assert [e for e in FakeSolver.log if e[0] == "open"] == [("open", m) for m in range(6)]
    srv.close()


def test_budget_evicts_least_recently_used_idle_members():
    fp = serve.footprint_bytes(100, 500)
    reqs = requests(members=3, steps=3, gap=1e-3)   # arrivals step by step: m0, m1, m2, m0, ...
    srv = FakeServer(slots=1, hbm_budget=2 * fp)
    res = srv.run(reqs, realtime=False)
    assert res["peak_resident_bytes"] <= 2 * fp
    assert res["evictions"] > 0
    opens = [m for e, m in FakeSolver.log if e == "open"]
    closes = [m for e, m in FakeSolver.log if e == "close"]
    # one slot, room for two: member 2 evicts member 0 (least recently used),
    # member 0 then evicts member 1, and so on round the ring
    assert closes[:3] == [0, 1, 2] and opens[:5] == [0, 1, 2, 0, 1]
    assert res["setups"] == len(opens)
    srv.close()


def test_a_failed_solve_is_raised():
    reqs = requests(members=2, steps=3)
    srv = FakeServer(slots=2, hbm_budget=1 << 40, fail={1: 1})
    with pytest.raises(RuntimeError, match="solve failed"):
        srv.run(reqs, realtime=False)
    srv.close()


def test_a_request_larger_than_the_budget_is_rejected():
    """Admission by HBM footprint: a member whose handle could not fit even on
    an empty device is rejected with a reason, and the other requests are
    served as usual (the loop does not wait for room that never comes)."""
    small = requests(members=2, steps=2)
    big = serve.Request(9, 0, SimpleNamespace(nb=10 ** 6, col=np.zeros(7 * 10 ** 6, np.int32), member=9),
                        np.zeros(3), 0.0)
    budget = 4 * serve.footprint_bytes(100, 500)
    assert serve.footprint_bytes(10 ** 6, 7 * 10 ** 6) > budget
    srv = FakeServer(slots=2, hbm_budget=budget)
    res = srv.run(small + [big], realtime=False)
    assert res["rejected"] == 1 and res["requests"] == 4
    assert big.error and "exceeds the HBM budget" in big.error and big.x is None
    assert all(r.error is None and r.stats for r in small)
    assert ("open", 9) not in FakeSolver.log
    srv.close()


def test_same_pattern_requests_update_values_only():
    """A member's later Newton steps that keep the block pattern go through the
    values-only update; the others (and the first, a setup) do not."""
    reqs = requests(members=2, steps=3)
    for r in reqs:
        r.same_pattern = r.step > 0
    calls = []

    class Recording(FakeSolver):
        def update(self, A):
            calls.append(("update", self.member))
            super().update(A)

        def update_values(self, val):
            calls.append(("values", self.member))
            super().update_values(val)

    class Srv(FakeServer):
        def _open(self, A):
            return Recording(A, A.member)

    srv = Srv(slots=2, hbm_budget=1 << 40)
    res = srv.run(reqs, realtime=False)
    assert res["requests"] == 6
    assert sorted(calls) == [("values", 0), ("values", 0), ("values", 1), ("values", 1)]
    srv.close()
