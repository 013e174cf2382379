"""The allocation-free Gram entry point (dngd_gram_bf16_noalloc) against the
Gram that a mixed-precision step computes through the regular context, and
against the FP64 product of the same BF16 operand computed on the host.

The no-alloc call exists for callers that cannot allocate device memory when
they need the Gram (their framework owns all device memory, or an allocation
would disturb surrounding work).  Its scratch is a fixed static device array,
so this test also checks that a second call in a row, which finds the first
call's leftovers in that array, is just as correct.  The file is named to be
collected last.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dngd():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2505_21404_gb300 import dngd as mod
    return mod


def test_gram_noalloc_matches_context_gram_twice(dngd):
    from paper_2505_21404_gb300 import workloads
    dev = "cuda:0"
    wl = workloads.poisson_sine(5, [5, 48, 40, 1], 300, 100, k=1, seed=2, lam=1e-5)
    ctx = dngd.Context(dngd.make_desc(wl, precision=dngd.MIXED_BF16, keep_gram=True, refine_tol=1e-10))
    m, n = ctx.m, ctx.n
    th = torch.tensor(wl["theta"], device=dev)
    X = torch.tensor(wl["X"], device=dev)
    tg = torch.tensor(wl["target"], device=dev)
    # the step's own Gram (context workspace) ...
    delta = torch.zeros(n, dtype=torch.float64, device=dev)
    info = ctx.step(th, X, tg, delta)
    K_ref = torch.zeros(m, m, dtype=torch.float64, device=dev)
    ctx.get_stage("gram", K_ref)
    shift = wl["lam"] + info["shift_used"]
    # ... and the same BF16 operand the step used (bf16 of the FP32 Jacobian)
    r = torch.zeros(m, dtype=torch.float64, device=dev)
    J = torch.zeros(m, n, dtype=torch.float64, device=dev)
    ctx.residual_jacobian(th, X, tg, r, J)
    ld = ((n + 7) // 8) * 8
    Jb = torch.zeros(m, ld, dtype=torch.bfloat16, device=dev)
    Jb[:, :n] = J.to(torch.bfloat16)
    K = torch.empty(m, m, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream().cuda_stream
    Kd = K_ref.cpu().numpy()
    # the FP64 product of the BF16 operand, on the host
    Jh = Jb[:, :n].double().cpu().numpy()
    K64 = np.tril(Jh @ Jh.T + shift * np.eye(m))
    for call in range(2):
        K.fill_(float("nan"))
        st = dngd.dngd_gram_bf16_noalloc(Jb, m, n, ld, K, m, shift, stream)
        assert st == 0, dngd.STATUS.get(st, st)
        torch.cuda.synchronize()
        Kh = K.double().cpu().numpy()
        assert np.all(np.isfinite(Kh)), call
        assert np.allclose(np.triu(Kh, 1), 0.0), call
        err = np.linalg.norm(Kh - Kd) / np.linalg.norm(Kd)
        assert err <= 1e-5, (call, err)
        err64 = np.linalg.norm(Kh - K64) / np.linalg.norm(K64)
        assert err64 <= 1e-5, (call, err64)
    ctx.close()


def test_gram_noalloc_largest_size_and_one_beyond(dngd):
    """m = 2000 (the stated maximum) is accepted and agrees with the host FP64
    product of its BF16 operand on two calls in a row; m = 2001 is rejected."""
    dev = "cuda:0"
    m, n = 2000, 1000
    g = torch.Generator(device="cpu").manual_seed(5)
    Jb = (torch.randn(m, n, generator=g, dtype=torch.float64) / 32.0).to(torch.bfloat16).to(dev)
    Jh = Jb.double().cpu().numpy()
    K64 = np.tril(Jh @ Jh.T + 0.25 * np.eye(m))
    K = torch.empty(m, m, dtype=torch.float32, device=dev)
    for call in range(2):
        K.fill_(float("nan"))
        st = dngd.dngd_gram_bf16_noalloc(Jb, m, n, n, K, m, 0.25, None)
        assert st == 0, dngd.STATUS.get(st, st)
        torch.cuda.synchronize()
        Kh = K.double().cpu().numpy()
        assert np.all(np.isfinite(Kh)), call
        err = np.linalg.norm(Kh - K64) / np.linalg.norm(K64)
        assert err <= 1e-5, (call, err)
    Jb1 = torch.zeros(m + 1, n, dtype=torch.bfloat16, device=dev)
    K1 = torch.zeros(1, dtype=torch.float32, device=dev)
    st = dngd.dngd_gram_bf16_noalloc(Jb1, m + 1, n, n, K1, m + 1, 0.0, None)
    assert dngd.STATUS[st] == "DNGD_ERR_INVALID_ARG"
