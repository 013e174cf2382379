"""Nystrom spectral preconditioner and PCG on the dual system (Sec. 3.3, App. A.2).

* ``nystrom``: Alg. "Nystrom construction of U, Lambda_hat" (Sec. 3.3.1,
  App. A.2).  Landmarks I are scalar residual indices, C the rest; K_II and
  K_CI are Gramian blocks; K_II = Q Lambda_Q Q^T keeping the r positive
  eigenpairs; U~_I = Q, U~_C = K_CI Q Lambda_Q^{-1}; M = U~ Lambda_Q^{1/2};
  SVD M = V Sigma W^T; U = V, Lambda_hat = Sigma^2.
* ``precond_apply``: P^{-1} = U (Lambda_hat + lambda I)^{-1} U^T
  + (1/lambda)(I - U U^T) (Eq. spec_precond_nystrom_main_final).
* ``pcg``: Alg. PCGStep with the kernel-vector product of Def. 3.3
  (w = J (J^T p) + lambda p).

Readings adopted (the paper is silent or garbled here):
* the landmark index set is an input (drawn by the caller from a seeded
  permutation);
* "positive" eigenvalues are those above ell * eps64 * max eigenvalue;
* the system solved is the push-through one, (K + lambda I) alpha = rhs,
  and the stop test is ||res|| <= tol * ||rhs||;
* breakdown: stop when <p, Ap> <= 1e-300 or the new rho is exactly 0.
"""
import numpy as np


def nystrom(J, landmarks):
    """Return (U [m, r], lam_hat [r]) from the landmark columns of K = J J^T."""
    m = J.shape[0]
    I = np.asarray(landmarks, dtype=np.int64)
    mask = np.ones(m, dtype=bool)
    mask[I] = False
    C = np.nonzero(mask)[0]
    JI = J[I]
    K_II = JI @ JI.T
    K_CI = J[C] @ JI.T
    w, Q = np.linalg.eigh(K_II)
    thresh = len(I) * np.finfo(np.float64).eps * max(float(w.max()), 0.0)
    keep = w > thresh
    w, Q = w[keep], Q[:, keep]
    Ut = np.zeros((m, w.size))
    Ut[I] = Q
    Ut[C] = K_CI @ Q / w[None, :]
    M = Ut * np.sqrt(w)[None, :]
    V, S, _ = np.linalg.svd(M, full_matrices=False)
    return V, S * S


def precond_apply(U, lam_hat, lam, x):
    """P^{-1} x (Eq. spec_precond_nystrom_main_final)."""
    c = U.T @ x
    return U @ (c / (lam_hat + lam)) + (x - U @ c) / lam


def kvp(J, lam, p):
    """Kernel-vector product w = J (J^T p) + lambda p (Def. 3.3)."""
    return J @ (J.T @ p) + lam * p


def pcg(J, lam, rhs, U, lam_hat, tol, max_it, apply_A=None):
    """Solve (K + lambda I) y = rhs by left-preconditioned CG (Alg. PCGStep).
    Returns (y, iterations, converged, final residual norm)."""
    if apply_A is None:
        def apply_A(p):
            return kvp(J, lam, p)
    m = rhs.shape[0]
    y = np.zeros(m)
    r = rhs.copy()
    bnorm = float(np.linalg.norm(rhs))
    if bnorm == 0.0:
        return y, 0, True, 0.0
    z = precond_apply(U, lam_hat, lam, r)
    p = z.copy()
    rho = float(r @ z)
    it = 0
    converged = False
    for j in range(max_it):
        Ap = apply_A(p)
        pAp = float(p @ Ap)
        if not pAp > 1e-300:
            break
        alpha = rho / pAp
        y = y + alpha * p
        r = r - alpha * Ap
        it = j + 1
        if float(np.linalg.norm(r)) <= tol * bnorm:
            converged = True
            break
        z = precond_apply(U, lam_hat, lam, r)
        rho_new = float(r @ z)
        if rho_new == 0.0:
            break
        beta = rho_new / rho
        p = z + beta * p
        rho = rho_new
    return y, it, converged, float(np.linalg.norm(r))


def pcg_step(theta, problem, X, target, lam, landmarks, tol, max_it, use_ga=True,
             eps_norm=0.0, ratio_max=0.5):
    """D-NGD step with the iterative dual solver (Alg. PCGStep), push-through
    recovery v = -J^T y, and the GA correction re-solved with the same
    preconditioner (Remark 3.1)."""
    from . import residual as res
    from .step import ga_accept
    r, J = res.residual_and_jacobian(theta, problem, X, target)
    U, lh = nystrom(J, landmarks)
    alpha, it1, ok1, _ = pcg(J, lam, r, U, lh, tol, max_it)
    v = -(J.T @ alpha)
    out = dict(r=r, J=J, U=U, lam_hat=lh, alpha=alpha, v=v, iters=[it1], converged=[ok1])
    if use_ga:
        fvv = res.second_directional(theta, problem, X, target, v)
        beta, it2, ok2, _ = pcg(J, lam, fvv, U, lh, tol, max_it)
        a = -(J.T @ beta)
        delta, ratio, acc = ga_accept(v, a, eps_norm, ratio_max)
        out.update(fvv=fvv, beta=beta, a=a, ratio=ratio, accepted=acc, delta=delta)
        out["iters"].append(it2)
        out["converged"].append(ok2)
    else:
        out.update(delta=v.copy(), ratio=float("nan"), accepted=False)
    return out
