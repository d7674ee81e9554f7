"""GPU tests of the batched solve (many systems, one block-diagonal
preconditioner, per-system FGMRES in lockstep)."""
import numpy as np
import pytest

import blackoil_synth as bs
import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    import paper_2201_01970_b300 as cpr
    from paper_2201_01970_b300 import build
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    build.build()
    return torch, cpr


def _dev(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


class _DJ:
    def __init__(self, torch, J):
        self.nb = J.nb
        self.rowptr, self.col, self.val = _dev(torch, J.rowptr), _dev(torch, J.col), _dev(torch, J.val)


def _systems():
    specs = [(4, 4, 2, 1), (7, 5, 3, 2), (20, 20, 5, 0), (13, 9, 6, 3), (16, 16, 4, 4)]
    return [bs.jacobian(bs.GridSpec(nx, ny, nz, 0.0, 1.5, 1.0, None, "corners", seed=sd))
            for nx, ny, nz, sd in specs]


def _true_rel(J, x):
    return np.linalg.norm(J.b - oracle.bsr3_spmv(J, x)) / np.linalg.norm(J.b)


@pytest.mark.parametrize("fp32", [0, 1])
def test_batch_converges_per_system_and_is_deterministic(env, fp32):
    torch, cpr = env
    Js = _systems()
    bt = cpr.BatchSolver([_DJ(torch, J) for J in Js], precond_fp32=fp32)
    xs, sts = bt.solve([_dev(torch, J.b) for J in Js], rtol=1e-6)
    for J, x, st in zip(Js, xs, sts):
        assert st["converged"], st
        assert _true_rel(J, x.cpu().numpy()) < 1e-6
    # the smallest system against the direct solution
    ref = np.linalg.solve(Js[0].to_dense(), Js[0].b)
    xs2, _ = bt.solve([_dev(torch, J.b) for J in Js], rtol=1e-10)
    assert np.linalg.norm(xs2[0].cpu().numpy() - ref) <= 1e-6 * np.linalg.norm(ref)
    # two solves give identical results
    xs3, _ = bt.solve([_dev(torch, J.b) for J in Js], rtol=1e-10)
    for a, b in zip(xs2, xs3):
        assert torch.equal(a, b)
    # host buffers give the same answer
    xh, sth = bt.solve([J.b for J in Js], rtol=1e-10)
    for a, b in zip(xh, xs3):
        assert np.array_equal(a, b.cpu().numpy())
    bt.close()


def test_batch_of_one_matches_single_solve(env):
    torch, cpr = env
    J = bs.jacobian("20x20x5")
    bt = cpr.BatchSolver([_DJ(torch, J)])
    g = cpr.Solver(_DJ(torch, J))
    xb, sb = bt.solve([_dev(torch, J.b)], rtol=1e-6)
    xg, sg = g.solve(_dev(torch, J.b), rtol=1e-6)
    assert abs(sb[0]["iters"] - sg["iters"]) <= 1
    a, b = xb[0].cpu().numpy(), xg.cpu().numpy()
    if sb[0]["iters"] == sg["iters"]:
        assert np.linalg.norm(a - b) <= 1e-8 * np.linalg.norm(b)
    bt.close()
    g.close()


def test_batch_update_and_zero_rhs(env):
    torch, cpr = env
    g1 = bs.GridSpec(6, 5, 3, 0.0, 1.0, 1.0, None, "corners", seed=1)
    g2 = bs.GridSpec(9, 4, 2, 0.0, 1.0, 1.0, None, "corners", seed=2)
    s1, s2 = list(bs.jacobian_sequence(g1, 2)), list(bs.jacobian_sequence(g2, 2))
    bt = cpr.BatchSolver([s1[0], s2[0]], mu=0)
    xs, sts = bt.solve([np.zeros(s1[0].n), s2[0].b.copy()])
    assert sts[0]["iters"] == 0 and sts[0]["converged"] and not xs[0].any()
    assert sts[1]["converged"]
    bt.update([s1[1], s2[1]])
    xs, sts = bt.solve([s1[1].b, s2[1].b])
    assert all(st["converged"] and st["setup_called"] for st in sts)
    for J, x in zip((s1[1], s2[1]), xs):
        assert _true_rel(J, x) < 1e-6
    with pytest.raises(cpr.CprError):
        bt.update([s1[1]])      # the batch's sizes cannot change
    bt.close()


def test_batch_matches_oracle(env):
    """A batch handle is the setup on the block-diagonal concatenation of its
    systems, so the oracle builds the same B from the same concatenation: the
    hierarchy, colors, C/F splits, P and BILU(0) equal the oracle's bit for
    bit; B applied to the concatenated vector matches element by element; and
    each system's lockstep FGMRES matches the oracle's FGMRES on that system's
    rows with the shared B restricted to them (iterations within one, x within
    1e-8 when the counts agree)."""
    from parity_helpers import SOLVE_TOL, assert_apply_close, block_diag, compare_hierarchy, rel
    torch, cpr = env
    Js = _systems()
    C = block_diag(Js)
    bt = cpr.BatchSolver([_DJ(torch, J) for J in Js])
    o = oracle.Solver(C)
    compare_hierarchy(o, bt)
    v = np.random.default_rng(4).standard_normal(C.n)
    z = torch.zeros(C.n, dtype=torch.float64, device="cuda")
    bt.apply(_dev(torch, v), z)
    assert_apply_close(z.cpu().numpy(), o.cpr_apply(v), what="batched B v")
    xs, sts = bt.solve([_dev(torch, J.b) for J in Js], rtol=1e-6)
    off = np.cumsum([0] + [J.nb for J in Js])
    for s, J in enumerate(Js):
        xo, so = o.solve_rows(int(off[s]), int(off[s + 1]), J.b, rtol=1e-6)
        assert so["converged"] and sts[s]["converged"]
        assert abs(sts[s]["iters"] - so["iters"]) <= 1, (s, sts[s], so)
        if sts[s]["iters"] == so["iters"]:
            assert rel(xs[s].cpu().numpy(), xo) < SOLVE_TOL, s
    bt.close()
    o.close()
