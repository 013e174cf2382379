"""GPU parity of the CUDA D-NGD path against the FP64 CPU oracle.

Every test calls the library through its C ABI (ctypes binding) on cuda:0 and
compares element by element with the oracle on the same seeded inputs.

Tolerances (relative 2-norm errors):
* FP64 path, jets and Jacobian: 1e-12 (only rounding order differs).
* FP64 path, step at lambda = 1e-5: 1e-10 on v / delta.  At lambda = 1e-8
  the problem itself amplifies rounding: perturbing J by one ulp moves the
  oracle's own v by ~3e-9 and alpha by ~4e-8 on the 2-D benchmark, so the
  bound there is 1e-7 on v / delta and 1e-6 on alpha.
* Mixed paths after refinement: 1e-4 on delta (the stated mixed tolerance).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import linesearch as olin, residual as ores, step as ostep  # noqa: E402
from paper_2505_21404_gb300 import workloads  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dngd():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2505_21404_gb300 import dngd as mod
    return mod


DEV = "cuda:0"


def _t(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device=DEV)


def _rel(a, b):
    a = a.detach().cpu().numpy() if hasattr(a, "detach") else np.asarray(a)
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))


def _heat_small(seed=0):
    return workloads.heat_1d([2, 24, 24, 1], 40, 12, 12, kappa=0.1, seed=seed, lam=1e-5)


CASES = {
    "poisson2d": lambda: workloads.poisson_sine(2, [2, 20, 20, 1], 70, 26, k=2, seed=3, lam=1e-5),
    "poisson5d": lambda: workloads.poisson_sine(5, [5, 33, 17, 9, 1], 61, 19, k=1, seed=4, lam=1e-5),
    "heat": _heat_small,
    "nohidden": lambda: workloads.poisson_sine(3, [3, 1], 9, 5, k=1, seed=5, lam=1e-3),
}


@pytest.mark.parametrize("case", list(CASES))
def test_residual_and_jacobian_fp64(dngd, case):
    wl = CASES[case]()
    prob = ores.problem_from_spec(wl)
    r_ref, J_ref = ores.residual_and_jacobian(wl["theta"], prob, wl["X"], wl["target"])
    ctx = dngd.Context(dngd.make_desc(wl, precision=dngd.FP64))
    r = torch.zeros(ctx.m, dtype=torch.float64, device=DEV)
    J = torch.zeros(ctx.m, ctx.n, dtype=torch.float64, device=DEV)
    ctx.residual_jacobian(_t(wl["theta"]), _t(wl["X"]), _t(wl["target"]), r, J)
    torch.cuda.synchronize()
    assert _rel(r, r_ref) <= 1e-12
    assert _rel(J, J_ref) <= 1e-12
    # element-wise on every row as well (no row may be off)
    Jh = J.cpu().numpy()
    row_err = np.linalg.norm(Jh - J_ref, axis=1) / np.maximum(np.linalg.norm(J_ref, axis=1), 1e-300)
    assert row_err.max() <= 1e-11


@pytest.mark.parametrize("case", ["poisson2d", "poisson5d", "heat"])
def test_fvv_fp64(dngd, case):
    wl = CASES[case]()
    prob = ores.problem_from_spec(wl)
    v = np.random.default_rng(7).normal(size=ores.mlp.n_params(wl["widths"])) * 0.2
    ref = ores.second_directional(wl["theta"], prob, wl["X"], wl["target"], v)
    ctx = dngd.Context(dngd.make_desc(wl, precision=dngd.FP64))
    out = torch.zeros(ctx.m, dtype=torch.float64, device=DEV)
    ctx.fvv(_t(wl["theta"]), _t(wl["X"]), _t(wl["target"]), _t(v), out)
    torch.cuda.synchronize()
    assert _rel(out, ref) <= 1e-11


@pytest.mark.parametrize("case", ["poisson2d", "poisson5d", "heat"])
def test_dense_step_fp64_all_stages(dngd, case):
    wl = CASES[case]()
    prob = ores.problem_from_spec(wl)
    lam = wl["lam"]
    ref = ostep.dense_step(wl["theta"], prob, wl["X"], wl["target"], lam, use_ga=True)
    ctx = dngd.Context(dngd.make_desc(wl, precision=dngd.FP64, keep_gram=True))
    delta = torch.zeros(ctx.n, dtype=torch.float64, device=DEV)
    info = ctx.step(_t(wl["theta"]), _t(wl["X"]), _t(wl["target"]), delta)
    m, n = ctx.m, ctx.n
    stage = {}
    for name, size in (("r", m), ("alpha", m), ("v", n), ("fvv", m), ("beta", m), ("a", n)):
        buf = torch.zeros(size, dtype=torch.float64, device=DEV)
        ctx.get_stage(name, buf)
        stage[name] = buf
    K = torch.zeros(m, m, dtype=torch.float64, device=DEV)
    ctx.get_stage("gram", K)
    Lf = torch.zeros(m, m, dtype=torch.float64, device=DEV)
    ctx.get_stage("chol", Lf)
    torch.cuda.synchronize()
    Kref = np.tril(ref["J"] @ ref["J"].T + lam * np.eye(m))
    assert _rel(K, Kref) <= 1e-12
    assert _rel(Lf, ref["L"]) <= 1e-9
    assert _rel(stage["r"], ref["r"]) <= 1e-12
    assert _rel(stage["alpha"], ref["alpha"]) <= 1e-9
    assert _rel(stage["v"], ref["v"]) <= 1e-10
    assert _rel(stage["fvv"], ref["fvv"]) <= 1e-9
    assert _rel(stage["beta"], ref["beta"]) <= 1e-8
    assert _rel(stage["a"], ref["a"]) <= 1e-9
    assert _rel(delta, ref["delta"]) <= 1e-10
    assert info["ga_accepted"] == ref["accepted"]
    assert abs(info["loss"] - 0.5 * float(ref["r"] @ ref["r"])) <= 1e-12 * (1 + info["loss"])


def test_poisson2d_benchmark_step_fp64(dngd):
    """The 2-D benchmark (m = 500, n = 1,185, lambda = 1e-8) at full size."""
    wl = workloads.poisson2d_fp64()
    prob = ores.problem_from_spec(wl)
    ref = ostep.dense_step(wl["theta"], prob, wl["X"], wl["target"], wl["lam"], use_ga=True)
    ctx = dngd.Context(dngd.make_desc(wl, precision=dngd.FP64))
    delta = torch.zeros(ctx.n, dtype=torch.float64, device=DEV)
    info = ctx.step(_t(wl["theta"]), _t(wl["X"]), _t(wl["target"]), delta)
    alpha = torch.zeros(ctx.m, dtype=torch.float64, device=DEV)
    ctx.get_stage("alpha", alpha)
    a = torch.zeros(ctx.n, dtype=torch.float64, device=DEV)
    ctx.get_stage("a", a)
    torch.cuda.synchronize()
    assert _rel(delta, ref["delta"]) <= 1e-7
    assert _rel(alpha, ref["alpha"]) <= 1e-6
    assert _rel(a, ref["a"]) <= 1e-6
    assert info["ga_accepted"] == ref["accepted"]


@pytest.mark.parametrize("prec", ["MIXED_BF16", "MIXED_TF32"])
@pytest.mark.parametrize("case", ["poisson2d", "poisson5d", "heat"])
def test_dense_step_mixed(dngd, case, prec):
    wl = CASES[case]()
    prob = ores.problem_from_spec(wl)
    ref = ostep.dense_step(wl["theta"], prob, wl["X"], wl["target"], wl["lam"], use_ga=True)
    ctx = dngd.Context(dngd.make_desc(wl, precision=getattr(dngd, prec), refine_tol=1e-12, refine_max_it=300,
                                      keep_gram=True))
    delta = torch.zeros(ctx.n, dtype=torch.float64, device=DEV)
    info = ctx.step(_t(wl["theta"]), _t(wl["X"]), _t(wl["target"]), delta)
    K = torch.zeros(ctx.m, ctx.m, dtype=torch.float64, device=DEV)
    ctx.get_stage("gram", K)
    torch.cuda.synchronize()
    # tensor-core Gram vs the oracle's Gram of the rounded operands
    J = ref["J"].astype(np.float32)
    if prec == "MIXED_BF16":
        Jl = torch.tensor(J).to(torch.bfloat16).double().numpy()
    else:
        Jl = J.astype(np.float64)
    Kref = np.tril(Jl @ Jl.T + wl["lam"] * np.eye(ctx.m))
    kerr = _rel(K, Kref)
    assert kerr <= (1e-5 if prec == "MIXED_BF16" else 2e-3), kerr
    err = _rel(delta, ref["delta"])
    assert err <= 1e-4, (err, info)


@pytest.mark.parametrize("case", ["poisson2d", "poisson5d", "heat", "poisson5d_tiles"])
def test_dense_step_mixed_oz(dngd, case):
    """Exact Gram of the FP32 Jacobian from 8-bit integer slices on the BF16
    tensor cores: it equals the FP64 product of the context's own FP32
    Jacobian to the slicing bound, and the refinement on that exact operator
    converges to the oracle's step."""
    # poisson5d_tiles: m = 601 spans five 128-row tiles with a ragged tail
    wl = CASES[case]() if case in CASES else workloads.poisson_sine(5, [5, 64, 64, 64, 1], 481, 120, k=1, seed=6,
                                                                     lam=1e-5)
    prob = ores.problem_from_spec(wl)
    ref = ostep.dense_step(wl["theta"], prob, wl["X"], wl["target"], wl["lam"], use_ga=True)
    ctx = dngd.Context(dngd.make_desc(wl, precision=dngd.MIXED_OZ, refine_tol=1e-10, refine_max_it=300))
    delta = torch.zeros(ctx.n, dtype=torch.float64, device=DEV)
    info = ctx.step(_t(wl["theta"]), _t(wl["X"]), _t(wl["target"]), delta)
    K = torch.zeros(ctx.m, ctx.m, dtype=torch.float64, device=DEV)
    ctx.get_stage("gram64", K)
    # the context's own FP32 Jacobian (its jets round differently from the
    # oracle's FP64 ones, at the 1e-7 level)
    J32 = torch.zeros(ctx.m, ctx.n, dtype=torch.float64, device=DEV)
    ctx.residual_jacobian(_t(wl["theta"]), _t(wl["X"]), _t(wl["target"]),
                          torch.zeros(ctx.m, dtype=torch.float64, device=DEV), J32)
    torch.cuda.synchronize()
    J = J32.cpu().numpy()
    Kh = K.cpu().numpy()
    assert np.array_equal(Kh, Kh.T)
    # four 8-bit slices keep 32 bits below each row's largest entry (entry
    # error <= 2^-33 of it) and the dropped products s + t >= 5 are 2^-40 of
    # the row scales: ~1e-11 relative on these cases, bounded here by 2^-33
    kerr = _rel(Kh, J @ J.T)
    assert kerr <= 2.0 ** -33, kerr
    assert _rel(J, ref["J"]) <= 1e-5
    # the step's floor is the FP32 jets (as on the MIXED_BF16 path)
    err = _rel(delta, ref["delta"])
    assert err <= 1e-4, (err, info)
    assert max(info["solve_relres"]) <= 1e-10, info


@pytest.mark.parametrize("prec", ["MIXED_OZ", "MIXED_BF16"])
def test_line_search_losses_mixed(dngd, prec):
    """Trial losses of the line search (their hidden layers run on the TF32
    tensor cores with hi/lo splits, ~2^-21 per product) against the oracle's
    FP64 losses, on a case whose stream matrix spans several 128-row tiles."""
    wl = workloads.poisson_sine(5, [5, 64, 64, 64, 1], 481, 120, k=1, seed=6, lam=1e-5)
    prob = ores.problem_from_spec(wl)
    ctx = dngd.Context(dngd.make_desc(wl, precision=getattr(dngd, prec), refine_tol=1e-8, refine_max_it=300))
    delta = torch.zeros(ctx.n, dtype=torch.float64, device=DEV)
    ctx.step(_t(wl["theta"]), _t(wl["X"]), _t(wl["target"]), delta)
    d = delta.cpu().numpy()
    etas = olin.grid()
    got = ctx.loss(_t(wl["theta"]), _t(wl["X"]), _t(wl["target"]), delta, etas)
    ref = np.array([ores.loss(wl["theta"] + e * d, prob, wl["X"], wl["target"]) for e in etas])
    rel = np.abs(got - ref) / ref
    near = ref <= 10 * ref.min()
    # near the minimum (where the choice is made) the losses agree to FP32
    # level; far out (eta ~ 1 here: loss 1e10, saturated units) the FP32 jets
    # lose a few more digits
    assert np.max(rel[near]) <= 1e-6, rel
    assert np.max(rel) <= 2e-4, rel
    assert int(np.argmin(got)) == int(np.argmin(ref))
