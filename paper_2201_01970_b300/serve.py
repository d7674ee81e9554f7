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
waiting for room that never comes.  Work of different members overlaps on
the device; every kernel is deterministic, so a request's result does not
depend on what else runs beside it.
"""
from __future__ import annotations

import threading
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

    @property
    def latency_ms(self) -> float:
        return 1000.0 * (self.end - self.arrival)


class Server:
    """Run a stream of requests with `slots` concurrent solves under `hbm_budget` bytes."""

    def __init__(self, slots: int = 4, hbm_budget: int = 64 << 30, rtol: float = 1e-6, **opts):
        self.slots = slots
        self.budget = hbm_budget
        self.rtol = rtol
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

    def run(self, requests: list[Request], realtime: bool = True) -> dict:
        """Replay the requests (arrival times honoured when `realtime`); returns metrics."""
        pending = sorted(requests, key=lambda r: (r.arrival, r.member, r.step))
        busy_members: set[int] = set()
        lock = threading.Lock()
        cond = threading.Condition(lock)
        running = 0
        errors: list[BaseException] = []
        t0 = time.perf_counter()

        def now():
            return time.perf_counter() - t0

        def worker(req: Request, fresh: bool):
            nonlocal running
            try:
                req.start = now()
                if fresh:
                    h = self._open(req.A)
                    with lock:
                        self.handles[req.member] = h
                else:
                    h = self.handles[req.member]
                    h.update(req.A)
                x = np.zeros(3 * req.A.nb)
                x, st = h.solve(req.b, x, rtol=self.rtol)
                req.x, req.stats = x, st
                req.end = now()
            except BaseException as e:   # noqa: BLE001
                errors.append(e)
            finally:
                with cond:
                    busy_members.discard(req.member)
                    self.last_used[req.member] = now()
                    running -= 1
                    cond.notify_all()

        threads = []
        with cond:
            while pending or running:
                if errors:
                    break
                t = now()
                launched = False
                if running < self.slots:
                    for k, req in enumerate(pending):
                        if realtime and req.arrival > t:
                            break
                        if req.member in busy_members:
                            continue
                        need = 0 if req.member in self.handles else footprint_bytes(
                            req.A.nb, int(req.A.col.shape[0]), self.opts.get("restart", 30),
                            bool(self.opts.get("precond_fp32", 1)))
                        if need > self.budget:
                            # no eviction can make room: reject rather than wait forever
                            req.error = (f"footprint {need} bytes exceeds the HBM budget of "
                                         f"{self.budget} bytes")
                            req.start = req.end = now()
                            self.rejected += 1
                            pending.pop(k)
                            launched = True
                            break
                        if self._resident() + need > self.budget:
                            idle = sorted((m for m in self.handles if m not in busy_members),
                                          key=lambda m: self.last_used.get(m, 0.0))
                            while idle and self._resident() + need > self.budget:
                                m = idle.pop(0)
                                self.handles.pop(m).close()
                                self.bytes.pop(m, None)
                                self.evictions += 1
                            if self._resident() + need > self.budget:
                                continue
                        fresh = req.member not in self.handles
                        if fresh:
                            self.bytes[req.member] = need
                        self.peak_bytes = max(self.peak_bytes, self._resident())
                        busy_members.add(req.member)
                        running += 1
                        pending.pop(k)
                        th = threading.Thread(target=worker, args=(req, fresh), daemon=True)
                        threads.append(th)
                        th.start()
                        launched = True
                        break
                if launched:
                    continue
                wait = 0.05
                if pending and realtime:
                    wait = max(0.0, min(wait, pending[0].arrival - now()))
                cond.wait(timeout=wait if wait > 0 else 0.0005)
        for th in threads:
            th.join()
        if errors:
            raise errors[0]
        served = [r for r in requests if r.error is None]
        makespan = max(r.end for r in served) if served else 0.0
        lat = np.array([r.latency_ms for r in served]) if served else np.zeros(1)
        return {"requests": len(served), "rejected": self.rejected, "makespan_s": makespan,
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
        reqs.append(Request(m, k, J, J.b, t))
    return reqs
