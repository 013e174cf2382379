"""Serving loop: PINN solve jobs submitted to a dngd_server.

A job's result must not depend on what else the server runs: each job has its
own context, stream and device-resident state, so a job run in a mix is
bitwise the job run alone.  A failing job (non-finite data) fails alone, a
job larger than the HBM budget is rejected, and a cancelled job stops without
touching the others."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import linesearch as olin, residual as ores, step as ostep  # noqa: E402
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


def _jobs():
    out = []
    for b, (d, w, m, k) in enumerate([(2, 32, 256, 1), (5, 64, 400, 3), (2, 128, 300, 5), (5, 32, 700, 8),
                                      (2, 64, 260, 2), (5, 128, 520, 4)]):
        nb = round(0.2 * m)
        out.append(workloads.poisson_sine(d, [d, w, w, 1], m - nb, nb, k=k, seed=2000 + b, lam=1e-5))
    return out


def _desc(dngd, wl, prec=None):
    return dngd.make_desc(wl, precision=dngd.MIXED_BF16 if prec is None else prec, refine_tol=1e-8,
                          refine_max_it=120)


def _run_alone(dngd, wl, n_steps, prec=None):
    srv = dngd.Server(max_slots=1)
    jid = srv.submit(_desc(dngd, wl, prec), wl["theta"], wl["X"], wl["target"], n_steps)
    srv.drain(300)
    info, theta = srv.result(jid)
    srv.close()
    assert info["state"] == "done", info
    return theta


def test_server_job_equals_manual_async_loop(dngd):
    wl = _jobs()[1]
    n_steps = 4
    theta_srv = _run_alone(dngd, wl, n_steps)
    ctx = dngd.Context(_desc(dngd, wl))
    th, X, tg = _t(wl["theta"]), _t(wl["X"]), _t(wl["target"])
    d = torch.zeros(ctx.n, dtype=torch.float64, device=DEV)
    etas = olin.grid()
    done = 0
    while done < n_steps:
        # as the server does: a failed factorisation leaves theta unchanged
        # and the iteration is re-run with the synchronous shift search
        ctx.step_async(th, X, tg, d)
        ctx.line_search_async(th, X, tg, d, etas)
        try:
            ctx.step_wait()
            done += 1
        except dngd.DngdError as e:
            assert "NOT_SPD" in str(e)
    torch.cuda.synchronize()
    assert np.array_equal(theta_srv, th.cpu().numpy())


def test_server_fp64_trajectory_matches_oracle(dngd):
    wl = _jobs()[0]
    theta = _run_alone(dngd, wl, 2, prec=dngd.FP64)
    prob = ores.problem_from_spec(wl)
    th = wl["theta"].copy()
    for _ in range(2):
        st = ostep.dense_step(th, prob, wl["X"], wl["target"], wl["lam"])
        eta, _ = olin.line_search(th, prob, wl["X"], wl["target"], st["delta"])
        th = th + eta * st["delta"]
    err = np.linalg.norm(theta - th) / np.linalg.norm(th - wl["theta"])
    assert err <= 1e-8, err


def test_mix_equals_alone(dngd):
    wls = _jobs()
    steps = [3, 5, 2, 4, 3, 2]
    alone = [_run_alone(dngd, wl, s) for wl, s in zip(wls, steps)]
    srv = dngd.Server(max_slots=3)
    ids = [srv.submit(_desc(dngd, wl), wl["theta"], wl["X"], wl["target"], s) for wl, s in zip(wls, steps)]
    srv.drain(300)
    for i, jid in enumerate(ids):
        info, theta = srv.result(jid)
        assert info["state"] == "done" and info["steps_done"] == steps[i], (i, info)
        assert np.array_equal(theta, alone[i]), i
    st = srv.stats()
    assert st["steps_total"] == sum(steps)
    assert st["admitted"] == len(wls) and st["done"] == len(wls) and st["failed"] == 0
    assert 0 < st["p50_ms"] <= st["p99_ms"]
    assert st["running"] == 0 and st["queued"] == 0 and st["hbm_used_bytes"] == 0
    srv.close()


def test_failing_job_is_isolated(dngd):
    wls = _jobs()[:3]
    ref = _run_alone(dngd, wls[2], 3)
    bad = dict(wls[1])
    bad["target"] = wls[1]["target"].copy()
    bad["target"][7] = np.nan
    srv = dngd.Server(max_slots=3)
    j0 = srv.submit(_desc(dngd, wls[0]), wls[0]["theta"], wls[0]["X"], wls[0]["target"], 3)
    jb = srv.submit(_desc(dngd, bad), bad["theta"], bad["X"], bad["target"], 3)
    j2 = srv.submit(_desc(dngd, wls[2]), wls[2]["theta"], wls[2]["X"], wls[2]["target"], 3)
    srv.drain(300)
    ib, _ = srv.result(jb)
    assert ib["state"] == "failed" and ib["status"] != 0, ib
    i0, _ = srv.result(j0)
    i2, th2 = srv.result(j2)
    assert i0["state"] == "done" and i2["state"] == "done"
    assert np.array_equal(th2, ref)
    assert srv.stats()["failed"] == 1
    srv.close()


def test_budget_rejects_oversized_job(dngd):
    small, big = _jobs()[0], _jobs()[5]
    ws_small = dngd.dngd_workspace_bytes(_desc(dngd, small))
    ws_big = dngd.dngd_workspace_bytes(_desc(dngd, big))
    assert ws_big > 2 * ws_small
    srv = dngd.Server(hbm_budget_bytes=ws_small + (16 << 20), max_slots=4)
    jb = srv.submit(_desc(dngd, big), big["theta"], big["X"], big["target"], 2)
    js = srv.submit(_desc(dngd, small), small["theta"], small["X"], small["target"], 2)
    srv.drain(300)
    ib, _ = srv.result(jb)
    assert ib["state"] == "failed" and dngd.STATUS[ib["status"]] == "DNGD_ERR_BUDGET", ib
    assert srv.result(js)[0]["state"] == "done"
    st = srv.stats()
    assert st["rejected"] == 1 and st["done"] == 1
    srv.close()


def test_cancel(dngd):
    wls = _jobs()[:2]
    ref = _run_alone(dngd, wls[0], 2)
    srv = dngd.Server(max_slots=2)
    j0 = srv.submit(_desc(dngd, wls[0]), wls[0]["theta"], wls[0]["X"], wls[0]["target"], 2)
    jl = srv.submit(_desc(dngd, wls[1]), wls[1]["theta"], wls[1]["X"], wls[1]["target"], 100000)
    srv.cancel(jl)
    srv.drain(300)
    il, th = srv.result(jl)
    assert il["state"] == "cancelled" and th is None
    i0, th0 = srv.result(j0)
    assert i0["state"] == "done" and np.array_equal(th0, ref)
    srv.close()


def test_job_setup_ordered_on_its_stream_while_legacy_stream_busy(dngd):
    """Jobs run on non-blocking streams, which are not ordered after work on
    the legacy default stream.  A job admitted while that stream is still
    busy (one spinning block queued there first) must still see its zeroed
    buffers, tile lists and inputs: its set-up is issued on its own stream,
    so it ends exactly as when it runs alone on an idle device."""
    wls = _jobs()
    ref = [_run_alone(dngd, wls[i], 3) for i in (3, 5)]
    srv = dngd.Server(max_slots=2)
    torch.cuda.synchronize()
    torch.cuda._sleep(int(3e9))   # ~1.5 s of one block on the legacy stream
    ids = [srv.submit(_desc(dngd, wls[i]), wls[i]["theta"], wls[i]["X"], wls[i]["target"], 3) for i in (3, 5)]
    srv.drain(300)
    for jid, r in zip(ids, ref):
        info, theta = srv.result(jid)
        assert info["state"] == "done", info
        assert np.array_equal(theta, r)
    srv.close()
    torch.cuda.synchronize()
