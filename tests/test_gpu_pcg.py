"""GPU parity of the matrix-free Nystrom-PCG path (Sec. 3.3, Alg. PCGStep)
against the FP64 oracle, through the C ABI.

The GPU operator is FP32 (factor-form GEMMs over the cached stream
activations and adjoints), so operator-level tolerances are FP32-sized
(1e-5 relative); the converged step is held to the mixed-path bound 1e-4.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import nystrom as onys, residual as ores, step as ostep  # noqa: E402
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


def _rel(a, b):
    a = a.detach().cpu().numpy() if hasattr(a, "detach") else np.asarray(a)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _heat(seed=0, lam=1e-3):
    return workloads.heat_1d([2, 24, 24, 24, 1], 48, 8, 8, kappa=0.1, seed=seed, lam=lam)


def _poisson(seed=1, lam=1e-3):
    return workloads.poisson_sine(3, [3, 20, 20, 1], 40, 16, k=1, seed=seed, lam=lam)


@pytest.fixture(scope="module", params=["heat", "poisson3d"])
def case(request, dngd):
    wl = _heat() if request.param == "heat" else _poisson()
    prob = ores.problem_from_spec(wl)
    r, J = ores.residual_and_jacobian(wl["theta"], prob, wl["X"], wl["target"])
    m = J.shape[0]
    ell = 16
    lm = workloads.landmarks(m, ell, seed=3)
    ctx = dngd.Context(dngd.make_desc(wl, precision=dngd.MIXED_BF16, solver=dngd.PCG, pcg_rank=ell,
                                      pcg_tol=1e-9, pcg_max_it=400))
    ctx.set_landmarks(lm)
    delta = torch.zeros(ctx.n, dtype=torch.float64, device=DEV)
    info = ctx.step(_t(wl["theta"]), _t(wl["X"]), _t(wl["target"]), delta)
    return dict(wl=wl, prob=prob, r=r, J=J, lm=lm, ctx=ctx, delta=delta, info=info)


def test_kernel_vector_product(dngd, case):
    J, lam, ctx = case["J"], case["wl"]["lam"], case["ctx"]
    v = np.random.default_rng(5).normal(size=J.shape[0])
    w = torch.zeros(J.shape[0], dtype=torch.float64, device=DEV)
    ctx.kvp(_t(v), w)
    torch.cuda.synchronize()
    assert _rel(w, onys.kvp(J, lam, v)) <= 1e-5


def test_landmark_columns(dngd, case):
    J, lm, ctx = case["J"], case["lm"], case["ctx"]
    K = torch.zeros(J.shape[0], len(lm), dtype=torch.float64, device=DEV)
    ctx.get_stage("kci", K)
    torch.cuda.synchronize()
    assert _rel(K, J @ J[lm].T) <= 1e-5


def test_nystrom_preconditioner(dngd, case):
    J, lm, lam, ctx = case["J"], case["lm"], case["wl"]["lam"], case["ctx"]
    U, lh = onys.nystrom(J, lm)
    x = np.random.default_rng(6).normal(size=J.shape[0])
    z = torch.zeros(J.shape[0], dtype=torch.float64, device=DEV)
    ctx.precond_apply(_t(x), z)
    torch.cuda.synchronize()
    assert case["info"]["shift_used"] == 0.0
    assert _rel(z, onys.precond_apply(U, lh, lam, x)) <= 1e-3


def test_pcg_step_matches_oracle(dngd, case):
    wl, prob, lm = case["wl"], case["prob"], case["lm"]
    ref = onys.pcg_step(wl["theta"], prob, wl["X"], wl["target"], wl["lam"], lm, tol=1e-12, max_it=400)
    dense = ostep.dense_step(wl["theta"], prob, wl["X"], wl["target"], wl["lam"])
    info = case["info"]
    assert all(ref["converged"])
    assert info["solve_relres"][0] <= 1e-9
    assert _rel(case["delta"], ref["delta"]) <= 1e-4
    assert _rel(case["delta"], dense["delta"]) <= 1e-4
    assert info["ga_accepted"] == ref["accepted"]
    alpha = torch.zeros(len(ref["alpha"]), dtype=torch.float64, device=DEV)
    case["ctx"].get_stage("alpha", alpha)
    torch.cuda.synchronize()
    assert _rel(alpha, ref["alpha"]) <= 1e-3


def test_all_landmarks_converge_in_one_iteration(dngd):
    """With ell = m the Nystrom approximation is exact, so P^{-1} = (K + lam I)^{-1}
    and PCG stops after one iteration (Sec. 3.3.1)."""
    wl = workloads.heat_1d([2, 16, 16, 1], 20, 6, 6, kappa=0.1, seed=4, lam=1e-2)
    m = 32
    ctx = dngd.Context(dngd.make_desc(wl, precision=dngd.MIXED_BF16, solver=dngd.PCG, pcg_rank=m, pcg_tol=1e-5,
                                      pcg_max_it=50))
    ctx.set_landmarks(np.arange(m))
    delta = torch.zeros(ctx.n, dtype=torch.float64, device=DEV)
    info = ctx.step(_t(wl["theta"]), _t(wl["X"]), _t(wl["target"]), delta)
    assert info["solve_iters"][0] <= 2, info
    prob = ores.problem_from_spec(wl)
    dense = ostep.dense_step(wl["theta"], prob, wl["X"], wl["target"], wl["lam"])
    assert _rel(delta, dense["delta"]) <= 1e-3


@pytest.mark.parametrize("op", ["tc3", "compensated"])
def test_operator_and_step_several_row_chunks(dngd, op):
    """The matrix-free J^T v reduces over the point-stream rows: here
    R = 4 * 400 + 64 + 64 = 1,728 rows (14 TMEM chunks of 128 on the tensor
    cores) and width 256.  K v against (J J^T + lambda I) v from the FP64
    Jacobian of a dense context at the same theta (both operators carry the
    FP32 jets' ~2e-6), and the converged PCG step against that context's
    FP64 step within the mixed path's 1e-4 (measured on GB300: 2.9e-5 with
    the 3xTF32 operator, 1.7e-5 with the compensated one)."""
    wl = workloads.heat_1d([2, 256, 256, 256, 1], 400, 64, 64, kappa=0.1, seed=2, lam=1e-3)
    th, X, tg = _t(wl["theta"]), _t(wl["X"]), _t(wl["target"])
    dense = dngd.Context(dngd.make_desc(wl, precision=dngd.FP64))
    m = dense.m
    r = torch.zeros(m, dtype=torch.float64, device=DEV)
    J = torch.zeros(m, dense.n, dtype=torch.float64, device=DEV)
    dense.residual_jacobian(th, X, tg, r, J)
    d64 = torch.zeros(dense.n, dtype=torch.float64, device=DEV)
    dense.step(th, X, tg, d64)
    opc = dngd.PCG_OP_TC3 if op == "tc3" else dngd.PCG_OP_COMPENSATED
    ctx = dngd.Context(dngd.make_desc(wl, precision=dngd.MIXED_BF16, solver=dngd.PCG, pcg_rank=64, pcg_tol=1e-8,
                                      pcg_max_it=400, pcg_operator=opc))
    ctx.set_landmarks(workloads.landmarks(m, 64, seed=3))
    delta = torch.zeros(ctx.n, dtype=torch.float64, device=DEV)
    info = ctx.step(th, X, tg, delta)
    lam = wl["lam"]
    v = torch.tensor(np.random.default_rng(7).normal(size=m), device=DEV)
    w = torch.zeros_like(v)
    ctx.kvp(v, w)
    ref = J @ (J.T @ v) + lam * v
    torch.cuda.synchronize()
    assert _rel(w, ref.cpu().numpy()) <= 1e-5
    assert info["solve_relres"][0] <= 1e-8, info
    assert _rel(delta, d64.cpu().numpy()) <= 1e-4
    dense.close()
    ctx.close()
