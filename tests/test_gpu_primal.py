"""GPU parity of the primal (parameter-space) Gauss-Newton step.

Prop. 3.1: (J^T J + lambda I) v = -J^T r, and Prop. 3.2: (J^T J + lambda I) a
= -J^T f_vv, solved with the n x n FP64 Cholesky factor; the step then takes
the same geodesic-acceleration test as the dual path.  The references are the
oracle's primal solve (``oracle.step.primal_step``, FP64) on the oracle's own
J, r and f_vv, and the oracle's dual step, which the push-through identity
(Thm. 3.1) makes the same vector: the two oracles agree to 2e-11-7e-11 on
these cases (cond(J^T J + lambda I) up to 4e6), so the bound 1e-9 leaves
rounding room for a different summation order and no room for a wrong term.

Cases: n = 337 and 241 (several 64-column factor blocks and a ragged tail),
n = 64 and 65 (one full block; a block plus a single column), n = 4 (one
partial block, GA accepted).  Plus the automatic space choice (primal exactly
when n < m), dngd_solve in the primal space, the n x n stages and the dual
stages' absence.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import residual as ores, step as ostep  # noqa: E402
from paper_2505_21404_gb300 import workloads  # noqa: E402

from _parity import check, layer_blocks, rel  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda:0"

CASES = {
    "p2d_n337": lambda: workloads.poisson_sine(2, [2, 16, 16, 1], 480, 120, k=2, seed=11, lam=1e-5),
    "p5d_n241": lambda: workloads.poisson_sine(5, [5, 12, 12, 1], 400, 100, k=1, seed=12, lam=1e-5),
    "n65": lambda: workloads.poisson_sine(2, [2, 16, 1], 160, 40, k=1, seed=13, lam=1e-5),
    "n64": lambda: workloads.poisson_sine(2, [2, 1, 20, 1], 160, 40, k=1, seed=14, lam=1e-5),
    "n4": lambda: workloads.poisson_sine(3, [3, 1], 9, 5, k=1, seed=5, lam=1e-3),
}


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


def _step(dngd, wl, space, keep_gram=False):
    ctx = dngd.Context(dngd.make_desc(wl, precision=dngd.FP64, keep_gram=keep_gram, solve_space=space))
    delta = torch.zeros(ctx.n, dtype=torch.float64, device=DEV)
    info = ctx.step(_t(wl["theta"]), _t(wl["X"]), _t(wl["target"]), delta)
    return ctx, delta, info


@pytest.mark.parametrize("case", list(CASES))
def test_primal_step_matches_oracle(dngd, case):
    wl = CASES[case]()
    lam = wl["lam"]
    ref = ostep.dense_step(wl["theta"], ores.problem_from_spec(wl), wl["X"], wl["target"], lam, use_ga=True)
    J = ref["J"]
    m, n = J.shape
    assert n < m
    vp = ostep.primal_step(J, ref["r"], lam)
    ap = ostep.primal_step(J, ref["fvv"], lam)
    ctx, delta, info = _step(dngd, wl, dngd.SPACE_PRIMAL, keep_gram=True)
    assert ctx.solve_space == dngd.SPACE_PRIMAL
    st = {}
    for name, size in (("r", m), ("v", n), ("fvv", m), ("a", n)):
        st[name] = torch.zeros(size, dtype=torch.float64, device=DEV)
        ctx.get_stage(name, st[name])
    G = torch.zeros(n, n, dtype=torch.float64, device=DEV)
    ctx.get_stage("gram", G)
    L = torch.zeros(n, n, dtype=torch.float64, device=DEV)
    ctx.get_stage("chol", L)
    torch.cuda.synchronize()
    spans = layer_blocks(wl["widths"])
    assert rel(st["r"], ref["r"]) <= 1e-12
    assert rel(st["fvv"], ref["fvv"]) <= 1e-9
    # the primal system J^T J + lambda I (lower) and its factor's backward error
    Gref = J.T @ J + lam * np.eye(n)
    assert rel(G, np.tril(Gref)) <= 1e-12
    Lh = L.cpu().numpy()
    assert np.allclose(Lh, np.tril(Lh))
    assert np.linalg.norm(Lh @ Lh.T - Gref) <= 1e-13 * np.linalg.norm(Gref)
    # v and a against the oracle's primal solves, delta against the dual oracle
    check("v", st["v"], vp, 1e-9, spans)
    check("a", st["a"], ap, 1e-9, spans)
    check("delta", delta, ref["delta"], 1e-9, spans)
    assert info["ga_accepted"] == ref["accepted"]
    assert abs(info["loss"] - 0.5 * float(ref["r"] @ ref["r"])) <= 1e-12 * (1 + info["loss"])


def test_auto_space_takes_the_smaller_system(dngd):
    """SPACE_AUTO is primal when n < m (bitwise the primal context's step) and
    dual when n > m (bitwise the dual context's step)."""
    tall = CASES["p2d_n337"]()
    wide = workloads.poisson_sine(2, [2, 20, 20, 1], 70, 26, k=2, seed=3, lam=1e-5)   # n = 501 > m = 96
    for wl, want in ((tall, dngd.SPACE_PRIMAL), (wide, dngd.SPACE_DUAL)):
        ca, da, _ = _step(dngd, wl, dngd.SPACE_AUTO)
        cw, dw, _ = _step(dngd, wl, want)
        assert ca.solve_space == want
        torch.cuda.synchronize()
        assert torch.equal(da, dw)
    # both spaces on the wide problem: the same step (push-through)
    _, dp, _ = _step(dngd, wide, dngd.SPACE_PRIMAL)
    _, dd, _ = _step(dngd, wide, dngd.SPACE_DUAL)
    torch.cuda.synchronize()
    assert rel(dp, dd.cpu().numpy()) <= 1e-8


def test_primal_solve_and_stages(dngd):
    """dngd_solve in the primal space solves (J^T J + lambda I) x = b with the
    step's factor (n-vectors); the dual vectors alpha and beta do not exist."""
    wl = CASES["p5d_n241"]()
    lam = wl["lam"]
    _, J = ores.residual_and_jacobian(wl["theta"], ores.problem_from_spec(wl), wl["X"], wl["target"])
    ctx, _, _ = _step(dngd, wl, dngd.SPACE_PRIMAL)
    n = ctx.n
    b = np.random.default_rng(7).standard_normal(n)
    x = torch.zeros(n, dtype=torch.float64, device=DEV)
    ctx.solve(_t(b), x)
    torch.cuda.synchronize()
    xref = np.linalg.solve(J.T @ J + lam * np.eye(n), b)
    assert rel(x, xref) <= 1e-9
    for name in ("alpha", "beta"):
        with pytest.raises(dngd.DngdError) as e:
            ctx.get_stage(name, torch.zeros(ctx.m, dtype=torch.float64, device=DEV))
        assert e.value.status == -8   # DNGD_ERR_STATE


def test_primal_async_and_training(dngd):
    """The primal space through the captured asynchronous step (replays equal
    the synchronous step bit for bit) and through dngd_train (equal to the
    hand-written loop bit for bit, the loss decreasing).  After six D-NGD
    iterations the primal and dual parameters agree within 1e-6: once the
    first step is taken, cond(J^T J + lambda I) is 4e8-8e8 on this problem, so
    each step of either space carries ~cond * 2^-53 ~ 1e-7 of rounding, and
    the oracle's own primal and dual trajectories (FP64, the same line-search
    choices) differ by 4.7e-8 after six iterations."""
    from oracle import linesearch as olin
    wl = CASES["p2d_n337"]()
    th, X, tg = _t(wl["theta"]), _t(wl["X"]), _t(wl["target"])
    ctx, d_sync, _ = _step(dngd, wl, dngd.SPACE_PRIMAL)
    d = torch.zeros_like(d_sync)
    for _ in range(3):      # the first asynchronous step runs synchronously, then graph replays
        ctx.step_async(th, X, tg, d)
        ctx.step_wait()
        torch.cuda.synchronize()
        assert torch.equal(d, d_sync)
    etas = olin.grid()
    thetas, losses = {}, {}
    for name, space in (("primal", dngd.SPACE_PRIMAL), ("dual", dngd.SPACE_DUAL)):
        desc = dngd.make_desc(wl, precision=dngd.FP64, solve_space=space)
        # the loop by hand
        c = dngd.Context(desc)
        t_h = _t(wl["theta"])
        dd = torch.zeros_like(t_h)
        hand = []
        for _ in range(6):
            hand.append(c.step(t_h, X, tg, dd)["loss"])
            c.line_search_async(t_h, X, tg, dd, etas)
        torch.cuda.synchronize()
        # the native loop
        t_n = _t(wl["theta"])
        res, hist = dngd.Context(desc).train(t_n, X, tg, 6)
        torch.cuda.synchronize()
        assert res["iters"] == 6
        assert np.array_equal(hist, np.array(hand))
        assert torch.equal(t_n, t_h)
        thetas[name], losses[name] = t_n.cpu().numpy(), hist
    assert losses["primal"][-1] < losses["primal"][0]
    assert rel(thetas["primal"], thetas["dual"]) <= 1e-6


@pytest.mark.parametrize("m,w", [(6300, 51), (3300, 51), (1800, 15)])
def test_primal_dual_agree_at_regime_map_sizes(dngd, m, w):
    """At the regime map's sizes (m = 6,300 and 3,300 with n = 2,857;
    m = 1,800 with n = 301), where the oracle is too slow for a test, the two
    spaces' steps agree within 1e-8 (push-through identity; cond(J^T J +
    lambda I) at theta_0 is ~1e6 on these problems) and the primal step's
    normal-equation residual ||(J^T J + lambda I) v + J^T r|| / ||J^T r|| is
    at rounding level, with J and r read back from the context."""
    ni = (4 * m) // 5
    wl = workloads.poisson_sine(2, [2, w, w, 1], ni, m - ni, k=2, seed=m + w, lam=1e-5)
    _, dp, _ = _step(dngd, wl, dngd.SPACE_PRIMAL)
    cd, dd, _ = _step(dngd, wl, dngd.SPACE_DUAL)
    n = cd.n
    r = torch.zeros(m, dtype=torch.float64, device=DEV)
    J = torch.zeros(m, n, dtype=torch.float64, device=DEV)
    cd.residual_jacobian(_t(wl["theta"]), _t(wl["X"]), _t(wl["target"]), r, J)
    cp, _, _ = _step(dngd, wl, dngd.SPACE_PRIMAL)
    v = torch.zeros(n, dtype=torch.float64, device=DEV)
    cp.get_stage("v", v)
    torch.cuda.synchronize()
    assert rel(dp, dd.cpu().numpy()) <= 1e-8
    g = J.T @ r
    res = J.T @ (J @ v) + wl["lam"] * v + g
    assert float(torch.linalg.norm(res) / torch.linalg.norm(g)) <= 1e-7
