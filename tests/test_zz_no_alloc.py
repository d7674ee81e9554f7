"""The allocation-free BILU(0) entry point (cpr_bilu_apply_noalloc).

Callers whose device memory is fixed after start-up -- for example a simulator
that reserves its whole device budget once, or code running while another
component owns the allocator -- cannot let a call allocate.  This entry point
keeps the sweeps' work vector in a fixed device array instead.  Its results
must equal cpr_bilu_apply's bit for bit (both run the same sweep kernels in the
same order), call after call, although every call shares that one array; and
once the handle is set up, a call must change neither the library's device
memory nor the device's free memory.  This file is collected last, so a run
that stops at the first failure has already run every other test.
"""
import gc

import numpy as np
import pytest

import blackoil_synth as bs

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


@pytest.mark.parametrize("fp32", [0, 1])
@pytest.mark.parametrize("grid", [(20, 20, 5), (37, 23, 9)])
def test_matches_cpr_bilu_apply_on_consecutive_calls(env, fp32, grid):
    torch, cpr = env
    J = bs.jacobian(bs.GridSpec(*grid, 0.0, 1.0, 1.0, None, "corners", seed=1))
    s = cpr.Solver(_DJ(torch, J), precond_fp32=fp32)
    rng = np.random.default_rng(7)
    rs = [_dev(torch, rng.standard_normal(J.n)) for _ in range(3)]
    zs = [torch.full((J.n,), np.nan, dtype=torch.float64, device="cuda") for _ in range(3)]
    z_ref = torch.zeros(J.n, dtype=torch.float64, device="cuda")
    gc.collect()                 # no other handle is released during the calls below
    torch.cuda.synchronize()
    for call in range(3):                      # calls in a row share the array
        lib_before = cpr.memory_in_use()
        free_before = torch.cuda.mem_get_info()[0]
        s.bilu_apply_noalloc(rs[call], zs[call])
        torch.cuda.synchronize()
        # the array was mapped, and the kernels loaded, at setup: no call moves memory
        assert cpr.memory_in_use() == lib_before
        assert torch.cuda.mem_get_info()[0] == free_before
        s.bilu_apply(rs[call], z_ref)
        a, b = zs[call].cpu().numpy(), z_ref.cpu().numpy()
        assert np.isfinite(a).all()
        np.testing.assert_array_equal(a, b, err_msg=f"call {call}")
    s.close()


def test_rejects_systems_beyond_the_array(env):
    torch, cpr = env
    J = bs.jacobian(bs.GridSpec(48, 48, 30, 0.0, 1.0, 1.0, None, "none", seed=0))
    assert J.nb > 65536
    s = cpr.Solver(_DJ(torch, J))
    r = torch.zeros(J.n, dtype=torch.float64, device="cuda")
    z = torch.zeros_like(r)
    with pytest.raises(cpr.CprError) as e:
        s.bilu_apply_noalloc(r, z)
    assert e.value.code == cpr.CPR_ERR_INVALID
    assert "at most 65536 block rows" in str(e.value)
    s.close()
