"""GPU tests of the serving loop: continuous batching over resident per-member
hierarchies; every result is the same alone and in the mix."""
import numpy as np
import pytest

import blackoil_synth as bs
import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def serve():
    import torch
    from paper_2201_01970_b300 import build
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    build.build()
    from paper_2201_01970_b300 import serve as sv
    return sv


def _members():
    return [bs.GridSpec(nx, ny, nz, 0.0, 1.0, 1.0, None, "corners", seed=300 + k)
            for k, (nx, ny, nz) in enumerate([(8, 8, 4), (12, 10, 4), (16, 16, 4), (10, 6, 3), (20, 12, 5)])]


def test_results_identical_alone_and_in_the_mix(serve):
    reqs1 = serve.poisson_requests(_members(), steps=3, rate=2000.0, seed=1)
    reqs4 = serve.poisson_requests(_members(), steps=3, rate=2000.0, seed=1)
    s1 = serve.Server(slots=1, mu=30)
    m1 = s1.run(reqs1, realtime=False)
    s1.close()
    s4 = serve.Server(slots=4, mu=30)
    m4 = s4.run(reqs4, realtime=True)
    s4.close()
    assert m1["requests"] == m4["requests"] == 15
    by1 = {(r.member, r.step): r for r in reqs1}
    for r in reqs4:
        a = by1[(r.member, r.step)]
        assert r.stats["converged"] and a.stats["converged"]
        # deterministic kernels and per-member state: identical bits
        assert np.array_equal(r.x, a.x), (r.member, r.step)
        assert r.stats["iters"] == a.stats["iters"]
        res = np.linalg.norm(r.A.b - oracle.bsr3_spmv(r.A, r.x)) / np.linalg.norm(r.A.b)
        assert res < 1e-6
    assert m4["p99_ms"] >= m4["p50_ms"] > 0


def test_admission_by_hbm_budget_evicts_and_stays_correct(serve):
    members = _members()
    need = max(serve.footprint_bytes(bs.jacobian(g).nb, bs.jacobian(g).nnzb) for g in members)
    reqs = serve.poisson_requests(members, steps=2, rate=5000.0, seed=2)
    s = serve.Server(slots=3, hbm_budget=2 * need + 1, mu=30)
    m = s.run(reqs, realtime=False)
    s.close()
    assert m["evictions"] > 0 and m["peak_resident_bytes"] <= 2 * need + 1
    for r in reqs:
        assert r.stats["converged"]
        res = np.linalg.norm(r.A.b - oracle.bsr3_spmv(r.A, r.x)) / np.linalg.norm(r.A.b)
        assert res < 1e-6


def test_served_results_match_the_oracle(serve):
    """Each served request (FP64 preconditioner) against the oracle solving the
    same member's Newton sequence in order under Alg. 3 with the same mu: the
    same setup decisions while the iteration counts agree, iterations within
    one, and x within 1e-8 when the counts are equal."""
    from parity_helpers import SOLVE_TOL, rel
    members = _members()[:3]
    reqs = serve.poisson_requests(members, steps=3, rate=2000.0, seed=3)
    s = serve.Server(slots=3, precond_fp32=0, mu=8)
    s.run(reqs, realtime=True)
    s.close()
    for m in range(len(members)):
        mine = sorted((r for r in reqs if r.member == m), key=lambda r: r.step)
        o = oracle.Solver(mine[0].A, mu=8)
        prev_equal = True
        for k, r in enumerate(mine):
            if k:
                o.update(r.A)
            xo, so = o.solve(r.A.b, rtol=1e-6)
            if prev_equal:
                assert r.stats["setup_called"] == so["setup_called"], (m, k)
            assert r.stats["converged"] and so["converged"]
            assert abs(r.stats["iters"] - so["iters"]) <= 1, (m, k, r.stats, so)
            prev_equal = r.stats["iters"] == so["iters"]
            if prev_equal:
                assert rel(r.x, xo) < SOLVE_TOL, (m, k)
        o.close()
