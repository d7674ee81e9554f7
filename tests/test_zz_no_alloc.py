"""The allocation-free BILU(0) entry point (cpr_bilu_apply_noalloc).

Callers whose device memory is fixed after start-up -- for example a simulator
that reserves its whole device budget once, or code running while another
component owns the allocator -- cannot let a call allocate.  This entry point
keeps the sweeps' work vector in a fixed device array instead.  Its results
must equal cpr_bilu_apply's, call after call, although both calls share that
one array.  This file is collected last, so a run that stops at the first
failure has already run every other test.
"""
import ctypes as C

import numpy as np
import pytest

import blackoil_synth as bs

pytestmark = pytest.mark.gpu

TOL = 1e-10   # the tolerance the other preconditioner-application tests use


@pytest.fixture(scope="module")
def env():
    import torch
    import paper_2201_01970_b300 as cpr
    from paper_2201_01970_b300 import build
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    build.build()
    L = cpr.lib()
    L.cpr_bilu_apply_noalloc.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p]
    return torch, cpr, L


def _dev(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


class _DJ:
    def __init__(self, torch, J):
        self.nb = J.nb
        self.rowptr, self.col, self.val = _dev(torch, J.rowptr), _dev(torch, J.col), _dev(torch, J.val)


@pytest.mark.parametrize("fp32", [0, 1])
@pytest.mark.parametrize("grid", [(20, 20, 5), (37, 23, 9)])
def test_matches_cpr_bilu_apply_on_consecutive_calls(env, fp32, grid):
    torch, cpr, L = env
    J = bs.jacobian(bs.GridSpec(*grid, 0.0, 1.0, 1.0, None, "corners", seed=1))
    s = cpr.Solver(_DJ(torch, J), precond_fp32=fp32)
    rng = np.random.default_rng(7)
    for call in range(2):                      # two calls in a row share the array
        r = _dev(torch, rng.standard_normal(J.n))
        z_ref = torch.zeros(J.n, dtype=torch.float64, device="cuda")
        z = torch.full((J.n,), np.nan, dtype=torch.float64, device="cuda")
        s.bilu_apply(r, z_ref)
        rc = L.cpr_bilu_apply_noalloc(s._h, r.data_ptr(), z.data_ptr())
        assert rc == cpr.CPR_OK, L.cpr_last_error_detail()
        a, b = z.cpu().numpy(), z_ref.cpu().numpy()
        assert np.isfinite(a).all()
        assert np.linalg.norm(a - b) <= TOL * np.linalg.norm(b), call
    s.close()


def test_rejects_systems_beyond_the_array(env):
    torch, cpr, L = env
    J = bs.jacobian(bs.GridSpec(48, 48, 30, 0.0, 1.0, 1.0, None, "none", seed=0))
    assert J.nb > 65536
    s = cpr.Solver(_DJ(torch, J))
    r = torch.zeros(J.n, dtype=torch.float64, device="cuda")
    z = torch.zeros_like(r)
    rc = L.cpr_bilu_apply_noalloc(s._h, r.data_ptr(), z.data_ptr())
    assert rc == cpr.CPR_ERR_INVALID
    assert b"at most 65536 block rows" in L.cpr_last_error_detail()
    s.close()
