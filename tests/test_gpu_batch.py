"""Asynchronous (graph-captured) steps and batches of independent instances.

Each instance of a batch must give the same result as the instance stepped
alone: the batch only overlaps independent work on the device, it never
changes what an instance computes (no batch-dependent split or reduction
order).  Exact-Gram instances are factored together by the batch, with
double-float trailing updates (FACTOR_DF); the same instance stepped alone
with that factor setting must agree bit for bit."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import residual as ores, step as ostep  # noqa: E402
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


def _instances():
    out = []
    for b, (w, m, k) in enumerate([(32, 256, 1), (64, 400, 3), (128, 300, 5), (32, 700, 8), (64, 260, 2),
                                   (128, 520, 4)]):
        nb = round(0.2 * m)
        out.append(workloads.poisson_sine(2, [2, w, w, 1], m - nb, nb, k=k, seed=1000 + b, lam=1e-5))
    return out


def test_async_step_equals_sync_step(dngd):
    wl = _instances()[1]
    desc = dngd.make_desc(wl, precision=dngd.MIXED_BF16, refine_tol=1e-8, refine_max_it=120)
    a = dngd.Context(desc)
    b = dngd.Context(desc)
    th, X, tg = _t(wl["theta"]), _t(wl["X"]), _t(wl["target"])
    da = torch.zeros(a.n, dtype=torch.float64, device=DEV)
    db = torch.zeros(b.n, dtype=torch.float64, device=DEV)
    for _ in range(3):
        ia = a.step(th, X, tg, da)
        b.step_async(th, X, tg, db)
        ib = b.step_wait()
        torch.cuda.synchronize()
        assert torch.equal(da, db)
        assert ia["solve_iters"] == ib["solve_iters"]


def test_batch_equals_each_instance_alone(dngd):
    wls = _instances()
    descs = [dngd.make_desc(wl, precision=dngd.MIXED_BF16, refine_tol=1e-8, refine_max_it=120) for wl in wls]
    batch = dngd.Batch(descs)
    alone = [dngd.Context(d) for d in descs]
    ths = [_t(wl["theta"]) for wl in wls]
    Xs = [_t(wl["X"]) for wl in wls]
    tgs = [_t(wl["target"]) for wl in wls]
    db = [torch.zeros(c.n, dtype=torch.float64, device=DEV) for c in alone]
    da = [torch.zeros(c.n, dtype=torch.float64, device=DEV) for c in alone]
    for it in range(3):
        infos = batch.step(ths, Xs, tgs, db)
        for i, c in enumerate(alone):
            info = c.step(ths[i], Xs[i], tgs[i], da[i])
            assert info["solve_iters"] == infos[i]["solve_iters"], (it, i)
        torch.cuda.synchronize()
        for i in range(len(wls)):
            assert torch.equal(da[i], db[i]), (it, i)


def test_batch_instance_matches_oracle(dngd):
    wls = _instances()[:3]
    descs = [dngd.make_desc(wl, precision=dngd.MIXED_BF16, refine_tol=1e-10, refine_max_it=200) for wl in wls]
    batch = dngd.Batch(descs)
    ths = [_t(wl["theta"]) for wl in wls]
    Xs = [_t(wl["X"]) for wl in wls]
    tgs = [_t(wl["target"]) for wl in wls]
    ds = [torch.zeros(len(wl["theta"]), dtype=torch.float64, device=DEV) for wl in wls]
    for _ in range(2):      # second call runs the captured graph
        batch.step(ths, Xs, tgs, ds)
    torch.cuda.synchronize()
    for wl, d in zip(wls, ds):
        ref = ostep.dense_step(wl["theta"], ores.problem_from_spec(wl), wl["X"], wl["target"], wl["lam"])
        err = float(np.linalg.norm(d.cpu().numpy() - ref["delta"]) / np.linalg.norm(ref["delta"]))
        assert err <= 1e-4, err


def test_crowded_batch_equals_alone(dngd):
    """Many larger instances at once, so that the CTAs of one instance's
    kernels start at different times on a busy device: every instance of the
    captured batch step still equals the same instance stepped alone, bit for
    bit, and no factorisation fails (a failed one would be redone
    synchronously and recaptured)."""
    rng = np.random.default_rng(77)
    wls = []
    for b in range(24):
        m = int(rng.integers(1000, 2001))
        w = int(rng.choice([32, 64]))
        nb = round(0.2 * m)
        wls.append(workloads.poisson_sine(2, [2, w, w, 1], m - nb, nb, k=int(rng.integers(1, 9)), seed=2000 + b,
                                          lam=1e-5))
    descs = [dngd.make_desc(wl, precision=dngd.MIXED_OZ, refine_tol=1e-8, refine_max_it=60) for wl in wls]
    batch = dngd.Batch(descs)
    ths = [_t(wl["theta"]) for wl in wls]
    Xs = [_t(wl["X"]) for wl in wls]
    tgs = [_t(wl["target"]) for wl in wls]
    db = [torch.zeros(len(wl["theta"]), dtype=torch.float64, device=DEV) for wl in wls]
    for _ in range(3):      # synchronous first step, then the captured graph twice
        batch.step(ths, Xs, tgs, db)
    torch.cuda.synchronize()
    alone = [dngd.Context(dngd.make_desc(wl, precision=dngd.MIXED_OZ, refine_tol=1e-8, refine_max_it=60,
                                         factor_update=dngd.FACTOR_DF)) for wl in wls]
    da = [torch.zeros_like(d) for d in db]
    for i, c in enumerate(alone):
        for _ in range(2):      # the first call is synchronous and fixes the shift, as in the batch
            c.step_async(ths[i], Xs[i], tgs[i], da[i])
            c.step_wait()
    torch.cuda.synchronize()
    for i in range(len(wls)):
        assert torch.equal(da[i], db[i]), i


@pytest.mark.parametrize("prec", ["MIXED_OZ", "MIXED_OZ64"])
def test_exact_gram_batch_matches_oracle(dngd, prec):
    """A batch of uneven exact-Gram instances (the batched factorisation of
    every instance in one launch per kernel and 64-column step): each
    instance's captured step against the FP64 oracle, and its factor L against
    the matrix it factors, K + (lambda + mu) I (a backward error)."""
    wls = _instances()
    descs = [dngd.make_desc(wl, precision=getattr(dngd, prec), refine_tol=1e-10, refine_max_it=200) for wl in wls]
    batch = dngd.Batch(descs)
    ths = [_t(wl["theta"]) for wl in wls]
    Xs = [_t(wl["X"]) for wl in wls]
    tgs = [_t(wl["target"]) for wl in wls]
    ds = [torch.zeros(len(wl["theta"]), dtype=torch.float64, device=DEV) for wl in wls]
    for _ in range(3):      # synchronous first step, then the captured graph twice
        infos = batch.step(ths, Xs, tgs, ds)
    torch.cuda.synchronize()
    for i, (wl, d) in enumerate(zip(wls, ds)):
        ref = ostep.dense_step(wl["theta"], ores.problem_from_spec(wl), wl["X"], wl["target"], wl["lam"])
        err = float(np.linalg.norm(d.cpu().numpy() - ref["delta"]) / np.linalg.norm(ref["delta"]))
        assert err <= 1e-4, (i, err)
        c = batch.context(i)
        m = c.m
        K = torch.zeros(m, m, dtype=torch.float64, device=DEV)
        L = torch.zeros(m, m, dtype=torch.float64, device=DEV)
        c.get_stage("gram64", K)
        c.get_stage("chol64", L)
        torch.cuda.synchronize()
        Kh, Lh = K.cpu().numpy(), L.cpu().numpy()
        assert np.all(np.triu(Lh, 1) == 0) and np.all(np.diag(Lh) > 0)
        Ks = Kh + (wl["lam"] + infos[i]["shift_used"]) * np.eye(m)
        assert np.linalg.norm(Lh @ Lh.T - Ks) <= 1e-11 * np.linalg.norm(Ks), i


def test_exact_gram_batch_block_edges(dngd):
    """Instances at the 64-column step boundaries (m = 40, 64, 65, 129: a
    diagonal block alone, one full block, a one-row panel, a trailing block of
    one row) in one batched factorisation: each step against the oracle and
    each factor against the matrix it factors."""
    wls = [workloads.poisson_sine(2, [2, 16, 16, 1], m - round(0.2 * m), round(0.2 * m), k=2, seed=3000 + m,
                                  lam=1e-5) for m in (40, 64, 65, 129)]
    descs = [dngd.make_desc(wl, precision=dngd.MIXED_OZ64, refine_tol=1e-10, refine_max_it=200) for wl in wls]
    batch = dngd.Batch(descs)
    ths = [_t(wl["theta"]) for wl in wls]
    Xs = [_t(wl["X"]) for wl in wls]
    tgs = [_t(wl["target"]) for wl in wls]
    ds = [torch.zeros(len(wl["theta"]), dtype=torch.float64, device=DEV) for wl in wls]
    for _ in range(2):      # synchronous first step, then the captured graph
        infos = batch.step(ths, Xs, tgs, ds)
    torch.cuda.synchronize()
    for i, (wl, d) in enumerate(zip(wls, ds)):
        ref = ostep.dense_step(wl["theta"], ores.problem_from_spec(wl), wl["X"], wl["target"], wl["lam"])
        err = float(np.linalg.norm(d.cpu().numpy() - ref["delta"]) / np.linalg.norm(ref["delta"]))
        assert err <= 1e-6, (i, err)
        c = batch.context(i)
        K = torch.zeros(c.m, c.m, dtype=torch.float64, device=DEV)
        L = torch.zeros(c.m, c.m, dtype=torch.float64, device=DEV)
        c.get_stage("gram64", K)
        c.get_stage("chol64", L)
        torch.cuda.synchronize()
        Kh, Lh = K.cpu().numpy(), L.cpu().numpy()
        Ks = Kh + (wl["lam"] + infos[i]["shift_used"]) * np.eye(c.m)
        assert np.linalg.norm(Lh @ Lh.T - Ks) <= 1e-11 * np.linalg.norm(Ks), i
