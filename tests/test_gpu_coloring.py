"""GPU parity of the paper's own coloring (Alg. 4-5, VerticesSplitting /
VerticesGrouping; coloring = 1) against the oracle: on every smoothed level
of at most coloring_rows rows the groups equal the oracle's bit for bit (JP,
bit-exact too, on the larger levels); solves match within one iteration."""
import numpy as np
import pytest

import blackoil_synth as bs
import oracle
from parity_helpers import SOLVE_TOL, assert_apply_close, compare_hierarchy, rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    import paper_2201_01970_b300 as cpr
    from paper_2201_01970_b300 import build
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    build.build()
    return torch, cpr


def dev(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


class DevJ:
    def __init__(self, torch, J):
        self.nb = J.nb
        self.rowptr, self.col, self.val = dev(torch, J.rowptr), dev(torch, J.col), dev(torch, J.val)


CASES = {
    "tiny": lambda: bs.tiny(),
    "20x20x5": lambda: bs.jacobian("20x20x5"),
    "37x23x9": lambda: bs.jacobian(bs.GridSpec(37, 23, 9, 0.0, 1.5, 0.3, None, "five_spot", seed=5)),
    "tall_well": lambda: bs.jacobian(bs.GridSpec(4, 4, 600, wells="corners", seed=3)),
}


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("theta", [0.0, 0.05, 0.1, 0.3])
def test_grouping_matches_oracle(env, case, theta):
    torch, cpr = env
    J = CASES[case]()
    kw = dict(coloring=1, coloring_rows=16384, theta_color=theta, coarse_max=16 if case == "tiny" else 256)
    o = oracle.Solver(J, **kw)
    g = cpr.Solver(DevJ(torch, J), **kw)
    compare_hierarchy(o, g)
    v = np.random.default_rng(2).standard_normal(J.n)
    z = torch.zeros(J.n, dtype=torch.float64, device="cuda")
    g.apply(dev(torch, v), z)
    assert_apply_close(z.cpu().numpy(), o.cpr_apply(v), what="B v with Alg. 4-5 colors")
    xo, so = o.solve(J.b, rtol=1e-6)
    xg, sg = g.solve(dev(torch, J.b), rtol=1e-6)
    assert sg["converged"] and so["converged"]
    assert abs(sg["iters"] - so["iters"]) <= 1, (sg, so)
    if sg["iters"] == so["iters"]:
        assert rel(xg.cpu().numpy(), xo) < SOLVE_TOL
    g.close()
    o.close()


def test_grouping_on_the_small_levels_of_128x128x32(env):
    """The default row limit (4096): levels 4 and 5 of the benchmark's
    hierarchy take Alg. 4-5, the larger ones JP; every coloring equals the
    oracle's under the same rule."""
    torch, cpr = env
    J = bs.jacobian("128x128x32")
    o = oracle.Solver(J, coloring=1)
    g = cpr.Solver(DevJ(torch, J), coloring=1)
    compare_hierarchy(o, g)
    small = [l for l in range(g.nlev - 1) if g.level(l)["n"] <= 4096]
    assert small
    j = cpr.Solver(DevJ(torch, J))
    print("colors, Alg. 4-5 on levels", small, [g.level(l)["ncolors"] for l in range(g.nlev - 1)],
          "JP", [j.level(l)["ncolors"] for l in range(j.nlev - 1)])
    g.close()
    j.close()
    o.close()
