"""GPU tests of failure handling that needs no GPU fault: a device-memory cap
makes allocations fail on the host side (CPR_ERR_OOM) and the library
recovers; every call leaves the caller's current device as it was."""
import gc

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


def test_memory_cap_gives_oom_and_the_library_recovers(env):
    torch, cpr = env
    J = bs.jacobian("20x20x5")
    gc.collect()                 # handles other tests left behind are released now, not mid-test
    base = cpr.memory_in_use()
    try:
        cpr.set_memory_limit(base + (1 << 20))          # 1 MiB more: the setup needs far more
        with pytest.raises(cpr.CprError) as e:
            cpr.Solver(J)
        assert e.value.code == cpr.CPR_ERR_OOM
        assert "memory limit" in str(e.value)
        assert cpr.memory_in_use() == base             # the failed setup released what it took
        cpr.set_memory_limit(0)
        s = cpr.Solver(J)
        held = cpr.memory_in_use()
        assert held > base
        # an update that needs a rebuild fails cleanly under a cap at the current use
        cpr.set_memory_limit(held)
        J2 = bs.jacobian("20x20x5", step=1)
        with pytest.raises(cpr.CprError) as e:
            s.update(J2)
        assert e.value.code == cpr.CPR_ERR_OOM
        s.close()
        assert cpr.memory_in_use() == base
        cpr.set_memory_limit(0)
        s = cpr.Solver(J)
        x, st = s.solve(J.b, rtol=1e-6)
        assert st["converged"]
        s.close()
    finally:
        cpr.set_memory_limit(0)


def test_calls_leave_the_current_device(env):
    torch, cpr = env
    J = bs.tiny()
    dev = torch.cuda.current_device()
    s = cpr.Solver(J)
    s.solve(J.b)
    s.close()
    assert torch.cuda.current_device() == dev
