"""Serving loop: continuous batching of CPR-FGMRES solve requests.

Requests (member, Newton step k, A^(k), b^(k)) arrive over time from an
ensemble of simulation runs.  Each member keeps its hierarchy resident in a
handle of its own (own CUDA stream), so Alg. 3's adaptive rule applies per
member across its Newton steps.  A fixed number of slots run requests
concurrently: a request is admitted as soon as a slot is free, its member has
no request in flight (a member's steps run in order), and the member's
footprint fits the HBM budget -- least-recently-used idle members are evicted
(their handles destroyed) to make room.  A request whose member could not fit
even on an empty device is rejected at once (its `error` says why) instead of
waiting for room that never comes.  One host thread starts and polls every
running solve at Arnoldi-step granularity, so work of different members
overlaps on the device; every kernel is deterministic, so a request's result
does not depend on what else runs beside it.
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field

import numpy as np

from . import Solver


def footprint_bytes(nb: int, nnzb: int, restart: int = 30, fp32: bool = True) -> int:
    """Device bytes a member's handle holds (estimate): the outer A (values,
    pattern), the frozen column-0 copy, BILU(0) factors, the pressure hierarchy
    (natural and color-ordered copies), and the Krylov workspace V, Z."""
    s = 4 if fp32 else 8
    per_block = 76 + (3 * s + 4) + 2 * 9 * s + 9 * s + 64
    per_row = 3 * 8 * (2 * restart + 1) + 3 * 8 * 6 + 300
    return int(1.15 * (nnzb * per_block + nb * per_row)) + (8 << 20)


@dataclass
class Request:
    member: int
    step: int
    A: object            # has nb, rowptr, col, val (host numpy arrays or device tensors)
    b: np.ndarray
    arrival: float       # seconds after the start of the replay
    x: np.ndarray | None = None
    start: float = 0.0
    end: float = 0.0
    stats: dict = field(default_factory=dict)
    error: str | None = None   # set when the request was rejected, not served
    same_pattern: bool = False  # A has the block pattern of the member's previous request
    update_s: float = 0.0      # time of the member handle's setup or update for this request

    @property
    def latency_ms(self) -> float:
        return 1000.0 * (self.end - self.arrival)


class Server:
    """Run a stream of requests with `slots` concurrent solves under `hbm_budget` bytes.

    One scheduler thread drives every admitted request: it starts a solve
    (cpr_solve_start) as soon as the request is admitted and its member's
    handle is ready, and polls all running solves (cpr_solve_poll), each of
    which issues its member's next Arnoldi steps on the member's own stream,
    so the solves of different members run side by side on the device while
    one host thread feeds them.  Only a member's first setup (and an update
    that changes the block pattern) runs on a small pool of helper threads,
    since a setup waits on the device while it builds the hierarchy."""

    def __init__(self, slots: int = 4, hbm_budget: int = 64 << 30, rtol: float = 1e-6,
                 setup_workers: int = 4, **opts):
        self.slots = slots
        self.budget = hbm_budget
        self.rtol = rtol
        self.setup_workers = setup_workers
        self.opts = dict(opts)
        self.handles: dict[int, Solver] = {}
        self.bytes: dict[int, int] = {}
        self.last_used: dict[int, float] = {}
        self.evictions = 0
        self.rejected = 0
        self.peak_bytes = 0

    def _resident(self) -> int:
        return sum(self.bytes.values())

    def _open(self, A):
        """A new handle for a member, on a CUDA stream of its own (non-blocking:
        members never wait on each other)."""
        import torch
        st = torch.cuda.Stream()
        opts = dict(self.opts)
        opts["stream"] = st.cuda_stream
        h = Solver(A, **opts)
        h._serve_stream = st
        return h

    def _admit(self, req, busy, now):
        """Whether req can start now; evicts least-recently-used idle members
        to make room under the budget.  Returns 'ok', 'wait' or 'reject'."""
        need = 0 if req.member in self.handles else footprint_bytes(
            req.A.nb, int(req.A.col.shape[0]), self.opts.get("restart", 30),
            bool(self.opts.get("precond_fp32", 1)))
        if need > self.budget:
            return "reject", need
        if self._resident() + need > self.budget:
            idle = sorted((m for m in self.handles if m not in busy),
                          key=lambda m: self.last_used.get(m, 0.0))
            while idle and self._resident() + need > self.budget:
                m = idle.pop(0)
                self.handles.pop(m).close()
                self.bytes.pop(m, None)
                self.evictions += 1
            if self._resident() + need > self.budget:
                return "wait", need
        return "ok", need

    def run(self, requests: list[Request], realtime: bool = True) -> dict:
        """Replay the requests (arrival times honoured when `realtime`); returns metrics."""
        from concurrent.futures import ThreadPoolExecutor
        pending = sorted(requests, key=lambda r: (r.arrival, r.member, r.step))
        active = {}          # member -> [request, phase, future or None, x]
        t0 = time.perf_counter()

        def now():
            return time.perf_counter() - t0

        def start_solve(req, h):
            x = np.zeros(3 * req.A.nb)
            h.solve_start(req.b, x, rtol=self.rtol)
            return x

        pool = ThreadPoolExecutor(max_workers=self.setup_workers)
        try:
            while pending or active:
                progressed = False
                t = now()
                # admission: free slots take the earliest arrived requests whose
                # member is idle and fits the budget
                k = 0
                while len(active) < self.slots and k < len(pending):
                    req = pending[k]
                    if realtime and req.arrival > t:
                        break
                    if req.member in active:
                        k += 1
                        continue
                    verdict, need = self._admit(req, active, t)
                    if verdict == "reject":
                        req.error = (f"footprint {need} bytes exceeds the HBM budget of "
                                     f"{self.budget} bytes")
                        req.start = req.end = now()
                        self.rejected += 1
                        pending.pop(k)
                        progressed = True
                        continue
                    if verdict == "wait":
                        k += 1
                        continue
                    pending.pop(k)
                    req.start = now()
                    progressed = True
                    if req.member not in self.handles:
                        self.bytes[req.member] = need
                        self.peak_bytes = max(self.peak_bytes, self._resident())
                        active[req.member] = [req, "setup", pool.submit(self._open, req.A), None]
                    else:
                        h = self.handles[req.member]
                        if req.same_pattern:   # a Newton step of the same simulation: values only
                            h.update_values(req.A.val)
                            req.update_s = now() - req.start
                            active[req.member] = [req, "solve", None, start_solve(req, h)]
                        else:
                            active[req.member] = [req, "setup", pool.submit(h.update, req.A), None]
                # progress of every admitted request
                for m in list(active):
                    req, phase, fut, x = active[m]
                    if phase == "setup":
                        if not fut.done():
                            continue
                        res = fut.result()     # raises a failed setup or update
                        if m not in self.handles:
                            self.handles[m] = res
                        req.update_s = now() - req.start
                        active[m] = [req, "solve", None, start_solve(req, self.handles[m])]
                        progressed = True
                        continue
                    out = self.handles[m].poll()
                    if out is None:
                        continue
                    req.x, req.stats = out
                    req.end = now()
                    self.last_used[m] = req.end
                    del active[m]
                    progressed = True
                if not progressed:
                    if pending and realtime and not active:
                        time.sleep(max(0.0, min(0.002, pending[0].arrival - now())))
                    else:
                        time.sleep(20e-6)
        finally:
            pool.shutdown(wait=True)
        served = [r for r in requests if r.error is None]
        makespan = max(r.end for r in served) if served else 0.0
        lat = np.array([r.latency_ms for r in served]) if served else np.zeros(1)
        waits = [r.start - r.arrival for r in served]
        firsts = [r.latency_ms for r in served if r.stats.get("setup_called") and r.step == 0]
        later = [r.latency_ms for r in served if not (r.stats.get("setup_called") and r.step == 0)]

        def pct(v, q):
            return float(np.percentile(v, q)) if v else 0.0

        return {"requests": len(served), "rejected": self.rejected, "makespan_s": makespan,
                "first_setup_p50_ms": pct(firsts, 50), "first_setup_p99_ms": pct(firsts, 99),
                "later_p50_ms": pct(later, 50), "later_p99_ms": pct(later, 99),
                "wait_ms_mean": 1000 * float(np.mean(waits or [0])),
                "update_ms_mean": 1000 * float(np.mean([r.update_s for r in served] or [0])),
                "service_ms_mean": 1000 * float(np.mean([r.end - r.start for r in served] or [0])),
                "device_solve_ms_sum": float(sum(r.stats.get("solve_ms", 0.0) for r in served)),
                "value": len(served) / makespan if makespan else 0.0, "unit": "solves/s",
                "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                "mean_iters": float(np.mean([r.stats.get("iters", 0) for r in served] or [0])),
                "setups": int(sum(r.stats.get("setup_called", 0) for r in served)),
                "evictions": self.evictions, "peak_resident_bytes": self.peak_bytes,
                "slots": self.slots}

    def close(self):
        for h in self.handles.values():
            h.close()
        self.handles.clear()
        self.bytes.clear()


def pin_request(req: Request) -> None:
    """Move a request's host arrays (A's pattern and values, b) into page-locked
    memory, as a server's receive buffers would be, so that its copies to the
    device run asynchronously at full link speed instead of through the
    driver's staging of pageable memory."""
    import torch
    import blackoil_synth as bs

    def pinned(a):
        t = torch.empty(a.shape, dtype=torch.from_numpy(a[:1]).dtype, pin_memory=True)
        t.numpy()[...] = a
        return t.numpy()

    A = req.A
    req.A = bs.Jacobian(A.nb, pinned(A.rowptr), pinned(A.col), pinned(A.val), pinned(A.b))
    req.b = req.A.b


def poisson_requests(members: list, steps: int, rate: float, seed: int = 0, drift: float = 0.05,
                     workers: int = 8):
    """Requests of `steps` drifting Jacobians per member, arrivals a Poisson
    process of `rate` per second (seeded exponential gaps); a member's steps
    arrive in order."""
    import blackoil_synth as bs
    from concurrent.futures import ThreadPoolExecutor
    rng = np.random.Generator(np.random.PCG64([seed, 7]))
    # members are generated independently (each from its own seed), on threads
    with ThreadPoolExecutor(max_workers=workers) as ex:
        lists = list(ex.map(lambda g: list(bs.jacobian_sequence(g, steps, drift)), members))
    seqs = dict(enumerate(lists))
    order = [(m, k) for k in range(steps) for m in range(len(members))]
    rng.shuffle(order)
    # keep each member's steps in order
    nxt = {m: 0 for m in range(len(members))}
    seq = []
    for m, _ in order:
        seq.append((m, nxt[m]))
        nxt[m] += 1
    t, reqs = 0.0, []
    for m, k in seq:
        t += rng.exponential(1.0 / rate)
        J = seqs[m][k]
        reqs.append(Request(m, k, J, J.b, t, same_pattern=k > 0))
    return reqs
