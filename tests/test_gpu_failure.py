"""Failure detection without a GPU fault: a device-side wait that can never
be satisfied runs out after its limit, the kernel records the timeout and
returns, the library reports DNGD_ERR_TIMEOUT, and the context is still
usable (a full step afterwards matches a fresh context bit for bit)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2505_21404_gb300 import workloads  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module")
def dngd():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2505_21404_gb300 import dngd as mod
    return mod


def _t(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device=DEV)


@pytest.mark.parametrize("prec", ["MIXED_OZ", "MIXED_BF16", "FP64"])
def test_bounded_wait_expires_and_context_survives(dngd, prec):
    wl = workloads.poisson_sine(2, [2, 32, 32, 1], 200, 56, k=2, seed=9, lam=1e-5)
    desc = dngd.make_desc(wl, precision=getattr(dngd, prec), refine_tol=1e-8, refine_max_it=200)
    ctx = dngd.Context(desc)
    status = ctx.check_wait_expiry(5.0)
    assert dngd.STATUS[status] == "DNGD_ERR_TIMEOUT", status
    d1 = torch.zeros(ctx.n, dtype=torch.float64, device=DEV)
    ctx.step(_t(wl["theta"]), _t(wl["X"]), _t(wl["target"]), d1)
    fresh = dngd.Context(desc)
    d2 = torch.zeros(ctx.n, dtype=torch.float64, device=DEV)
    fresh.step(_t(wl["theta"]), _t(wl["X"]), _t(wl["target"]), d2)
    torch.cuda.synchronize()
    assert torch.equal(d1, d2)
