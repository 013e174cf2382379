"""The native optimizer loop (dngd_train, Alg. D-NGD Workflow with the damping
rule of App. A.3, resampled collocation points, wall-clock budget) against the
same loop written by hand over dngd_step / dngd_line_search_async."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import linesearch as olin  # noqa: E402
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


def _points(it):
    # a fresh draw of the 2-D benchmark's collocation points (same counts)
    wl = workloads.poisson_sine(2, [2, 32, 32, 1], 400, 100, k=1, seed=100 + it, lam=1e-8)
    return wl["X"], wl["target"]


def _manual(dngd, ctx, wl, n_iters, resample_every=0):
    th, X, tg = _t(wl["theta"]), _t(wl["X"]), _t(wl["target"])
    d = torch.zeros_like(th)
    etas = olin.grid()
    losses = []
    for it in range(n_iters):
        if it > 0 and resample_every and it % resample_every == 0:
            Xn, tn = _points(it)
            X.copy_(_t(Xn))
            tg.copy_(_t(tn))
        info = ctx.step(th, X, tg, d)
        losses.append(info["loss"])
        ctx.line_search_async(th, X, tg, d, etas)
    torch.cuda.synchronize()
    return th.cpu().numpy(), np.array(losses)


@pytest.mark.parametrize("prec,cap", [("FP64", 0.0), ("MIXED_OZ64", 1e-5)])
def test_train_equals_manual_loop(dngd, prec, cap):
    wl = workloads.poisson2d_fp64()
    desc = dngd.make_desc(wl, precision=getattr(dngd, prec), lambda_cap=cap, refine_tol=1e-10, refine_max_it=400)
    ref_th, ref_loss = _manual(dngd, dngd.Context(desc), wl, 6)
    ctx = dngd.Context(desc)
    th, X, tg = _t(wl["theta"]), _t(wl["X"]), _t(wl["target"])
    res, hist = ctx.train(th, X, tg, 6)
    torch.cuda.synchronize()
    assert res["iters"] == 6 and res["stop"] == "iters", res
    assert np.array_equal(th.cpu().numpy(), ref_th)
    assert np.array_equal(hist, ref_loss)
    assert res["loss"] < ref_loss[0]


def test_train_resampling(dngd):
    wl = workloads.poisson2d_fp64()
    desc = dngd.make_desc(wl, precision=dngd.FP64)
    ref_th, ref_loss = _manual(dngd, dngd.Context(desc), wl, 6, resample_every=2)
    ctx = dngd.Context(desc)
    th, X, tg = _t(wl["theta"]), _t(wl["X"]), _t(wl["target"])
    calls = []

    def resample(it):
        calls.append(it)
        Xn, tn = _points(it)
        X.copy_(_t(Xn))
        tg.copy_(_t(tn))
        torch.cuda.synchronize()

    res, hist = ctx.train(th, X, tg, 6, resample_every=2, resample=resample)
    torch.cuda.synchronize()
    assert calls == [2, 4]
    assert res["iters"] == 6
    assert np.array_equal(th.cpu().numpy(), ref_th)
    assert np.array_equal(hist, ref_loss)


def test_train_stops_on_budget_and_loss_target(dngd):
    wl = workloads.poisson2d_fp64()
    desc = dngd.make_desc(wl, precision=dngd.FP64)
    ctx = dngd.Context(desc)
    th, X, tg = _t(wl["theta"]), _t(wl["X"]), _t(wl["target"])
    th0 = th.clone()
    res, hist = ctx.train(th, X, tg, 50, time_budget_s=1e-9)
    assert res["stop"] == "budget" and res["iters"] == 0 and len(hist) == 0
    assert torch.equal(th, th0)
    res, hist = ctx.train(th, X, tg, 50, loss_target=1e30)
    assert res["stop"] == "loss" and res["iters"] == 0 and len(hist) == 1
    assert torch.equal(th, th0)
    # a budget that lets a few iterations through stops between iterations
    res, hist = ctx.train(th, X, tg, 10000, time_budget_s=0.5)
    assert res["stop"] == "budget" and 0 < res["iters"] < 10000
    assert res["elapsed_s"] >= 0.5
    assert np.all(np.diff(hist[:5]) < 0) or res["loss"] < hist[0]
