"""GPU parity of the D-NGD step on the cases the basic parity tests leave out.

* The geodesic-acceleration branch taken: delta = v + a/2 (Alg.
  DenseDualSolve), on inputs where the oracle accepts (2||a||/||v|| <= 0.5),
  and with the threshold raised so that a case that rejects is accepted.
* The exact-Gram (MIXED_OZ) step at m = 2,000, n = 33,921 (5-128^3-1 net, 16
  row tiles and a 1,060-stage K extent) and at the 5-D benchmark size
  (m = 4,000, n = 133,377): the Gram against the FP64 product of the
  context's own FP32 Jacobian, entry by entry within the slicing bound, and
  alpha, v, a, delta against the FP64 oracle.
* dngd_solve against the oracle's triangular solves with the factor of the
  same step.
* An indefinite K + lambda I (FP64, lambda < 0, a residual class whose
  operator is zero so its Jacobian rows vanish): DNGD_ERR_NOT_SPD at the
  oracle's failing column.
* The 2-D benchmark at lambda = 1e-8 entry by entry.

Every call goes through the C ABI on cuda:0.  Errors are normwise, entrywise
(relative to the entry plus the RMS of the reference) and per block (each
layer's W and b; each residual class), see tests/_parity.py.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import residual as ores, step as ostep  # noqa: E402
from paper_2505_21404_gb300 import workloads  # noqa: E402

from _parity import check, class_blocks, layer_blocks, rel  # noqa: E402

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


def _stages(ctx, names):
    out = {}
    for name in names:
        size = ctx.n if name in ("v", "a") else ctx.m
        buf = torch.zeros(size, dtype=torch.float64, device=DEV)
        ctx.get_stage(name, buf)
        out[name] = buf
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in out.items()}


# (workload, GA threshold): the oracle accepts the GA correction on each
GA_CASES = {
    # heat, lambda = 0.1: ratio 0.35
    "heat_lam0.1": (lambda: workloads.heat_1d([2, 24, 24, 1], 40, 12, 12, kappa=0.1, seed=0, lam=0.1), 0.5),
    # 2-D Poisson, lambda = 10: ratio 0.14
    "poisson2d_lam10": (lambda: workloads.poisson_sine(2, [2, 20, 20, 1], 70, 26, k=2, seed=3, lam=10.0), 0.5),
    # 5-D Poisson, lambda = 1e-5: ratio ~300, accepted with the threshold raised
    "poisson5d_forced": (lambda: workloads.poisson_sine(5, [5, 33, 17, 9, 1], 61, 19, k=1, seed=4, lam=1e-5),
                         1e9),
}


@pytest.mark.parametrize("prec,tol", [("FP64", 1e-10), ("MIXED_OZ", 1e-4), ("MIXED_BF16", 1e-4)])
@pytest.mark.parametrize("case", list(GA_CASES))
def test_ga_accepted_step(dngd, case, prec, tol):
    make, ratio_max = GA_CASES[case]
    wl = make()
    prob = ores.problem_from_spec(wl)
    ref = ostep.dense_step(wl["theta"], prob, wl["X"], wl["target"], wl["lam"], use_ga=True, ratio_max=ratio_max)
    assert ref["accepted"], ref["ratio"]
    ctx = dngd.Context(dngd.make_desc(wl, precision=getattr(dngd, prec), ga_ratio_max=ratio_max, refine_tol=1e-12,
                                      refine_max_it=300))
    delta = torch.zeros(ctx.n, dtype=torch.float64, device=DEV)
    info = ctx.step(_t(wl["theta"]), _t(wl["X"]), _t(wl["target"]), delta)
    st = _stages(ctx, ["v", "a", "alpha", "beta"])
    d = delta.cpu().numpy()
    assert info["ga_accepted"], info
    assert abs(info["ga_ratio"] - ref["ratio"]) <= 1e-3 * ref["ratio"] + (1e-8 if prec == "FP64" else 1e-4)
    # the accepted step is exactly v + a/2 of the step's own v and a
    assert np.array_equal(d, st["v"] + 0.5 * st["a"])
    lb = layer_blocks(wl["widths"])
    cb = class_blocks(wl["classes"])
    check("delta", d, ref["delta"], tol, lb)
    check("v", st["v"], ref["v"], tol, lb)
    # alpha and a go through (K + lambda I)^{-1} without the map-back's
    # smoothing: 1e-9 on the FP64 path (as the all-stages FP64 test)
    check("a", st["a"], ref["a"], max(tol, 1e-9), lb)
    check("alpha", st["alpha"], ref["alpha"], max(tol, 1e-9), cb)
    ctx.close()


def _oz_gram_bound(J, ns=4):
    """Entry bound of the exact Gram of J from ns 8-bit slices per entry (rows
    scaled by 2^E_i, E_i = exponent of the row's largest |J| plus one): each
    entry of J is kept to 2^(E_i - 8 ns - 1), so
      |K_ij - (J J^T)_ij| <= 2^-(8 ns + 1) (||J_i||_1 2^E_j + ||J_j||_1 2^E_i)
                              + n 2^(E_i + E_j) t_ns
    where t covers the dropped slice products and the rounded trailing levels:
    t_4 = 2^-38 (the dropped levels s + t >= 5, 2^-40, and the rounded
    trailing levels, 2^-39; keeping level 5 only lowers the first)."""
    amax = np.abs(J).max(axis=1)
    E = np.where(amax > 0, np.frexp(amax)[1] + 1, 0).astype(np.float64)
    s = 2.0 ** E
    l1 = np.abs(J).sum(axis=1)
    n = J.shape[1]
    t = {4: 2.0 ** -38, 5: 2.0 ** -44}[ns]
    return 2.0 ** -(8 * ns + 1) * (np.outer(l1, s) + np.outer(s, l1)) + n * t * np.outer(s, s)


def _oz_case(dngd, wl, sample=None, seed=0, prec="MIXED_OZ", step_tol=1e-4, factor_update=0):
    ns = 4                       # slices per entry (both modes)
    prob = ores.problem_from_spec(wl)
    ref = ostep.dense_step(wl["theta"], prob, wl["X"], wl["target"], wl["lam"], use_ga=True)
    ctx = dngd.Context(dngd.make_desc(wl, precision=getattr(dngd, prec), refine_tol=1e-10, refine_max_it=400,
                                      factor_update=factor_update))
    delta = torch.zeros(ctx.n, dtype=torch.float64, device=DEV)
    info = ctx.step(_t(wl["theta"]), _t(wl["X"]), _t(wl["target"]), delta)
    st = _stages(ctx, ["v", "a", "alpha", "beta"])
    m, n = ctx.m, ctx.n
    K = torch.zeros(m, m, dtype=torch.float64, device=DEV)
    ctx.get_stage("gram64", K)
    L = torch.zeros(m, m, dtype=torch.float64, device=DEV)
    ctx.get_stage("chol64", L)
    J32 = torch.zeros(m, n, dtype=torch.float64, device=DEV)
    ctx.residual_jacobian(_t(wl["theta"]), _t(wl["X"]), _t(wl["target"]),
                          torch.zeros(m, dtype=torch.float64, device=DEV), J32)
    torch.cuda.synchronize()
    Kh = K.cpu().numpy()
    assert np.array_equal(Kh, Kh.T)
    # the context's own Jacobian: FP32 (MIXED_OZ) or FP64 (MIXED_OZ64).  An
    # FP32 entry within 2^8 of its row's largest is represented exactly by
    # the four slices, so the FP32 Gram is well inside 2^-33 normwise; an FP64
    # entry keeps 2^-33 of the row scale, which two rows' product doubles
    # (the FP64 jets' layer GEMMs run on slice products: each kept to 2^-33
    # of its rows' scales, so J to ~1e-10)
    j_tol = 1e-5 if prec == "MIXED_OZ" else 1e-9
    g_tol = 2.0 ** -(8 * ns + 1) if prec == "MIXED_OZ" else 2.0 ** -(8 * ns - 1)
    if sample is None:
        J = J32.cpu().numpy()
        Kx = J @ J.T
        assert rel(Kh, Kx) <= g_tol
        B = _oz_gram_bound(J, ns)
        assert np.all(np.abs(Kh - Kx) <= B), float(np.max(np.abs(Kh - Kx) / B))
        assert rel(J, ref["J"]) <= j_tol
    else:
        # sampled rows: the exact Gram's rows against FP64 products of the
        # context's rows with its whole Jacobian
        rows = np.sort(np.random.default_rng(seed).choice(m, size=sample, replace=False))
        Jr = J32[rows].cpu().numpy()
        Kx = (J32[rows] @ J32.T).cpu().numpy()
        Jall = J32.cpu().numpy()
        B = _oz_gram_bound(Jall, ns)[rows]
        assert np.all(np.abs(Kh[rows] - Kx) <= B), float(np.max(np.abs(Kh[rows] - Kx) / B))
        assert rel(Kh[rows], Kx) <= g_tol
        assert rel(Jr, ref["J"][rows]) <= j_tol
        del Jall
    assert max(info["solve_relres"]) <= 1e-10, info
    # the factor (double-float diagonal blocks and panels, sliced trailing
    # updates; read with the Gram, before the Jacobian call ends the step's
    # state): L L^T against the matrix it factors, K + (lambda + mu) I,
    # normwise on all rows or on the sampled ones (a backward error, so it
    # does not depend on K's condition number)
    Lh = L.cpu().numpy()
    assert np.all(np.triu(Lh, 1) == 0) and np.all(np.diag(Lh) > 0)
    sh = wl["lam"] + info["shift_used"]
    rows_f = np.arange(m) if sample is None else np.sort(np.random.default_rng(seed + 1).choice(m, 64, False))
    LLt = Lh[rows_f] @ Lh.T
    Ks = Kh[rows_f] + sh * np.eye(m)[rows_f]
    assert rel(LLt, Ks) <= 1e-11, rel(LLt, Ks)
    lb = layer_blocks(wl["widths"])
    cb = class_blocks(wl["classes"])
    check("delta", delta, ref["delta"], step_tol, lb)
    check("v", st["v"], ref["v"], step_tol, lb)
    check("alpha", st["alpha"], ref["alpha"], step_tol, cb)
    check("a", st["a"], ref["a"], step_tol, lb)
    assert info["ga_accepted"] == ref["accepted"]
    ctx.close()
    return info


OZ64_CASES = {
    "poisson2d": lambda: workloads.poisson_sine(2, [2, 20, 20, 1], 70, 26, k=2, seed=3, lam=1e-5),
    "poisson5d": lambda: workloads.poisson_sine(5, [5, 33, 17, 9, 1], 61, 19, k=1, seed=4, lam=1e-5),
    "heat": lambda: workloads.heat_1d([2, 24, 24, 1], 40, 12, 12, kappa=0.1, seed=0, lam=1e-5),
    # m = 601: five 128-row tiles and eight 80-column tiles with ragged tails
    "poisson5d_tiles": lambda: workloads.poisson_sine(5, [5, 64, 64, 64, 1], 481, 120, k=1, seed=6, lam=1e-5),
}


@pytest.mark.parametrize("case", list(OZ64_CASES))
def test_dense_step_oz64(dngd, case):
    """Exact Gram of the FP64 Jacobian from four 8-bit slices with the
    products of levels <= 5: the Gram within the slicing bound entry by entry,
    and the step within 1e-5 of the oracle (a CPU emulation of this Gram gave
    3e-6 at a trained theta with lambda = 1e-5 and 2e-8 at theta_0)."""
    _oz_case(dngd, OZ64_CASES[case](), prec="MIXED_OZ64", step_tol=1e-5)


@pytest.mark.parametrize("prec,factor", [("MIXED_OZ", "FACTOR_SLICED"), ("MIXED_OZ64", "FACTOR_SLICED"),
                                         ("MIXED_OZ64", "FACTOR_DF")])
def test_dense_step_oz_m2000(dngd, prec, factor):
    """5-D Poisson, MLP 5-128-128-128-1 (n = 33,921), 1,500 + 500 points;
    both forms of the factor's trailing updates (sliced tensor-core products
    with look-ahead, or double-float as in batches)."""
    wl = workloads.poisson_sine(5, [5, 128, 128, 128, 1], 1500, 500, k=1, seed=8, lam=1e-5)
    _oz_case(dngd, wl, prec=prec, step_tol=1e-4 if prec == "MIXED_OZ" else 1e-5,
             factor_update=getattr(dngd, factor))


@pytest.mark.parametrize("prec", ["MIXED_OZ", "MIXED_OZ64"])
def test_dense_step_oz_benchmark_size(dngd, prec):
    """The 5-D benchmark workload itself (m = 4,000, n = 133,377, lambda =
    1e-5, theta_0), in the launch configuration the benchmark times: Gram rows
    sampled, every stage against a full oracle step."""
    wl = workloads.poisson5d_dense(seed=0, lam=1e-5)
    _oz_case(dngd, wl, sample=48, seed=1, prec=prec, step_tol=1e-4 if prec == "MIXED_OZ" else 1e-5)


def test_trained_theta_paper_damping(dngd):
    """At parameters the oracle reaches after 12 D-NGD iterations of a 5-D
    Poisson problem (MLP 5-48-48-48-1, 360 + 120 points; loss ~1e-7), with the
    paper's rule lambda = min(loss, 1e-5): the FP64-Jacobian exact-Gram step
    within 1e-4 of the oracle, and the FP64 path within 50x the oracle's own
    one-ulp sensitivity.  (With an FP32 Jacobian the residuals themselves are
    off by ~1e-3 here, so MIXED_OZ is not held to the bound at such theta.)"""
    from oracle import linesearch as olin
    wl = workloads.poisson_sine(5, [5, 48, 48, 48, 1], 360, 120, k=1, seed=2, lam=1e-5)
    prob = ores.problem_from_spec(wl)
    X, tg = wl["X"], wl["target"]
    th = wl["theta"].copy()
    for _ in range(12):
        r = ores.residual(th, prob, X, tg)
        out = ostep.dense_step(th, prob, X, tg, min(0.5 * float(r @ r), 1e-5), use_ga=True)
        eta, _ = olin.line_search(th, prob, X, tg, out["delta"])
        th = th + eta * out["delta"]
    r = ores.residual(th, prob, X, tg)
    loss = 0.5 * float(r @ r)
    lam = min(loss, 1e-5)
    ref = ostep.dense_step(th, prob, X, tg, lam, use_ga=True)
    J, v = ref["J"], ref["v"]
    Jp = J * (1.0 + 2.0 ** -53 * np.random.default_rng(0).choice([-1.0, 1.0], size=J.shape))
    vp = -(Jp.T @ np.linalg.solve(Jp @ Jp.T + lam * np.eye(J.shape[0]), ref["r"]))
    spread = rel(vp, v)
    errs = {}
    for prec in ("FP64", "MIXED_OZ64", "MIXED_OZ"):
        ctx = dngd.Context(dngd.make_desc(wl, precision=getattr(dngd, prec), refine_tol=1e-10, refine_max_it=600,
                                          lambda_cap=1e-5))
        d = torch.zeros(ctx.n, dtype=torch.float64, device=DEV)
        info = ctx.step(_t(th), _t(X), _t(tg), d)
        torch.cuda.synchronize()
        errs[prec] = (rel(d, ref["delta"]), info["lambda_used"], info["solve_iters"])
        ctx.close()
    assert loss <= 1e-4, loss
    assert abs(errs["FP64"][1] - lam) <= 1e-10 * lam, errs
    assert errs["FP64"][0] <= max(1e-10, 50 * spread), (errs, spread)
    assert errs["MIXED_OZ64"][0] <= 1e-4, (errs, spread)
    # the exact-Gram mode's residuals come from jets whose layer GEMMs keep
    # 2^-33 of their rows' scales: the loss (hence lambda) to ~1e-5 here
    assert abs(errs["MIXED_OZ64"][1] - lam) <= 1e-4 * lam, errs


@pytest.mark.parametrize("prec,tol", [("FP64", 1e-10), ("MIXED_OZ", 1e-6), ("MIXED_BF16", 1e-6)])
def test_dngd_solve_matches_triangular_solves(dngd, prec, tol):
    """dngd_solve reuses the last step's factor (FP64) or preconditioned
    refinement (mixed) for a new right-hand side: against the oracle's two
    triangular solves with the Cholesky factor of the same K + lambda I (for
    the mixed paths, the Gram of the context's own FP32 Jacobian)."""
    wl = workloads.poisson_sine(2, [2, 20, 20, 1], 70, 26, k=2, seed=3, lam=1e-3)
    ctx = dngd.Context(dngd.make_desc(wl, precision=getattr(dngd, prec), refine_tol=1e-13, refine_max_it=400))
    m, n = ctx.m, ctx.n
    delta = torch.zeros(n, dtype=torch.float64, device=DEV)
    with pytest.raises(dngd.DngdError) as e:
        ctx.solve(_t(np.ones(m)), torch.zeros(m, dtype=torch.float64, device=DEV))
    assert e.value.status == -8   # DNGD_ERR_STATE before any step
    ctx.step(_t(wl["theta"]), _t(wl["X"]), _t(wl["target"]), delta)
    rng = np.random.default_rng(3)
    bs = [rng.normal(size=m) for _ in range(2)]
    xs = []
    for b in bs:
        x = torch.zeros(m, dtype=torch.float64, device=DEV)
        ctx.solve(_t(b), x)
        xs.append(x)
    # the step's own Jacobian (FP32 on the mixed paths), read after the solves
    # (a new Jacobian evaluation ends the step's state)
    J = torch.zeros(m, n, dtype=torch.float64, device=DEV)
    ctx.residual_jacobian(_t(wl["theta"]), _t(wl["X"]), _t(wl["target"]),
                          torch.zeros(m, dtype=torch.float64, device=DEV), J)
    torch.cuda.synchronize()
    L = ostep.cholesky(ostep.gram(J.cpu().numpy(), wl["lam"]))
    for k, (b, x) in enumerate(zip(bs, xs)):
        check(f"x{k}", x, ostep.chol_solve(L, b), tol, class_blocks(wl["classes"]))
    ctx.close()


def test_not_spd_reports_oracle_column(dngd):
    """FP64, lambda = -1e-12, classes: six boundary value points, then three
    points whose operator is zero (their Jacobian rows are zero, so their
    pivots are lambda < 0).  The oracle's Cholesky fails at column 6; the
    step must return DNGD_ERR_NOT_SPD with the same column."""
    wl = workloads.poisson_sine(2, [2, 8, 8, 1], 3, 6, k=1, seed=11, lam=-1e-12)
    wl["classes"] = [dict(count=6, c_val=1.0, c_grad=[0.0, 0.0], c_lap=0.0, lap_mask=[0, 0]),
                     dict(count=3, c_val=0.0, c_grad=[0.0, 0.0], c_lap=0.0, lap_mask=[0, 0])]
    wl["X"] = np.ascontiguousarray(np.concatenate([wl["X"][3:], wl["X"][:3]]))
    prob = ores.problem_from_spec(wl)
    r, J = ores.residual_and_jacobian(wl["theta"], prob, wl["X"], wl["target"])
    with pytest.raises(ostep.NotSPD) as e:
        ostep.cholesky(ostep.gram(J, wl["lam"]))
    col = e.value.column
    assert col == 6
    # a mixed-precision context refuses lambda <= 0
    with pytest.raises(dngd.DngdError):
        dngd.Context(dngd.make_desc(wl, precision=dngd.MIXED_OZ))
    ctx = dngd.Context(dngd.make_desc(wl, precision=dngd.FP64, keep_gram=True))
    # with lambda = 1e-3 the same context forms the oracle's K + lambda I and factor
    ctx.set_lambda(1e-3)
    d0 = torch.zeros(ctx.n, dtype=torch.float64, device=DEV)
    ctx.step(_t(wl["theta"]), _t(wl["X"]), _t(wl["target"]), d0)
    Kg = torch.zeros(ctx.m, ctx.m, dtype=torch.float64, device=DEV)
    Lg = torch.zeros(ctx.m, ctx.m, dtype=torch.float64, device=DEV)
    ctx.get_stage("gram", Kg)
    ctx.get_stage("chol", Lg)
    torch.cuda.synchronize()
    Kref = np.tril(J @ J.T + 1e-3 * np.eye(ctx.m))
    assert rel(Kg, Kref) <= 1e-12, (Kg.cpu().numpy(), Kref)
    assert rel(Lg, ostep.cholesky(J @ J.T + 1e-3 * np.eye(ctx.m))) <= 1e-10, Lg.cpu().numpy()
    ctx.set_lambda(wl["lam"])
    # the context's Jacobian is the oracle's (the zero-operator rows included)
    Jg = torch.zeros(ctx.m, ctx.n, dtype=torch.float64, device=DEV)
    rg = torch.zeros(ctx.m, dtype=torch.float64, device=DEV)
    ctx.residual_jacobian(_t(wl["theta"]), _t(wl["X"]), _t(wl["target"]), rg, Jg)
    torch.cuda.synchronize()
    assert rel(Jg, J) <= 1e-12 and not np.any(Jg.cpu().numpy()[6:]), (Jg.cpu().numpy(), J)
    assert rel(rg, r) <= 1e-12
    info = dngd.StepInfo()
    d = torch.zeros(ctx.n, dtype=torch.float64, device=DEV)
    # the input tensors are held for the call (a temporary's memory may be
    # handed to the next one before the kernels read it)
    th_d, X_d, tg_d = _t(wl["theta"]), _t(wl["X"]), _t(wl["target"])
    s = dngd.lib.dngd_step(ctx._h, dngd._ptr(th_d), dngd._ptr(X_d), dngd._ptr(tg_d), dngd._ptr(d),
                           dngd.C.byref(info))
    torch.cuda.synchronize()
    assert dngd.STATUS[s] == "DNGD_ERR_NOT_SPD"
    assert info.not_spd_column == col
    # the same context steps normally once lambda is positive again
    ctx.set_lambda(1e-3)
    ref = ostep.dense_step(wl["theta"], prob, wl["X"], wl["target"], 1e-3, use_ga=True)
    ctx.step(_t(wl["theta"]), _t(wl["X"]), _t(wl["target"]), d)
    torch.cuda.synchronize()
    check("delta", d, ref["delta"], 1e-10)
    ctx.close()


def test_poisson2d_benchmark_entrywise(dngd):
    """The 2-D benchmark (m = 500, n = 1,185, lambda = 1e-8, FP64) entry by
    entry and per block.  The bound 1e-7 on v and delta is ~50x the oracle's
    own FP64 rounding spread at this lambda (about 2e-9 on v against an
    extended-precision solve of the same J; test_oracle_step.py pins it)."""
    wl = workloads.poisson2d_fp64()
    prob = ores.problem_from_spec(wl)
    ref = ostep.dense_step(wl["theta"], prob, wl["X"], wl["target"], wl["lam"], use_ga=True)
    ctx = dngd.Context(dngd.make_desc(wl, precision=dngd.FP64))
    delta = torch.zeros(ctx.n, dtype=torch.float64, device=DEV)
    info = ctx.step(_t(wl["theta"]), _t(wl["X"]), _t(wl["target"]), delta)
    st = _stages(ctx, ["v", "a", "alpha"])
    lb = layer_blocks(wl["widths"])
    check("delta", delta, ref["delta"], 1e-7, lb)
    check("v", st["v"], ref["v"], 1e-7, lb)
    check("alpha", st["alpha"], ref["alpha"], 1e-6, class_blocks(wl["classes"]))
    check("a", st["a"], ref["a"], 1e-6, lb)
    assert info["ga_accepted"] == ref["accepted"]
    ctx.close()
