"""Damped Gauss-Newton step in residual space with geodesic acceleration.

Follows Sec. 3 of the paper:
* Levenberg-Marquardt subproblem F_lambda (Sec. 3, Prop. 3.1): the step
  minimises 1/2 ||r + J dtheta||^2 + lambda/2 ||dtheta||^2.
* Residual Gramian K = J J^T (Def. 3.1) and the dual normal equations
  (K + lambda I) y = -J grad L with recovery
  dtheta = -(1/lambda)(J^T y + grad L) (Thm. 3.1, Eq. dual-system / dual-recovery).
* Geodesic acceleration (Sec. 3.2, Def. 3.2, Prop. 3.2): a minimises
  1/2 ||J a + f_vv||^2 + lambda/2 ||a||^2.
* The DenseDualSolve algorithm (App. A.2): one Cholesky factor of
  K + lambda I, two triangular solves for v, two more for a, acceptance test
  2 ||a|| / ||v|| <= 0.5 guarded by ||v|| > eps_norm.

Reading adopted for the recovery: the push-through form
v = -J^T (K + lambda I)^{-1} r, a = -J^T (K + lambda I)^{-1} f_vv, which is
algebraically identical to the paper's recovery (substitute y = -(K+lambda)^{-1} K r)
and does not divide by lambda.  ``dense_step_literal`` keeps the paper's form
for the equivalence check.
"""
import numpy as np

from . import residual as res


class NotSPD(ArithmeticError):
    def __init__(self, column):
        super().__init__(f"matrix not positive definite at column {column}")
        self.column = column


def cholesky(A):
    """Textbook column-by-column Cholesky A = L L^T (lower).  Raises NotSPD
    with the failing column when a pivot is not positive."""
    A = np.asarray(A, dtype=np.float64)
    m = A.shape[0]
    L = np.zeros_like(A)
    for j in range(m):
        piv = A[j, j] - L[j, :j] @ L[j, :j]
        if not piv > 0.0:
            raise NotSPD(j)
        L[j, j] = np.sqrt(piv)
        if j + 1 < m:
            L[j + 1:, j] = (A[j + 1:, j] - L[j + 1:, :j] @ L[j, :j]) / L[j, j]
    return L


def forward_subst(L, b):
    """Solve L y = b (L lower triangular), row by row."""
    m = L.shape[0]
    y = np.zeros(m)
    for i in range(m):
        y[i] = (b[i] - L[i, :i] @ y[:i]) / L[i, i]
    return y


def back_subst_t(L, y):
    """Solve L^T x = y, row by row from the bottom."""
    m = L.shape[0]
    x = np.zeros(m)
    for i in range(m - 1, -1, -1):
        x[i] = (y[i] - L[i + 1:, i] @ x[i + 1:]) / L[i, i]
    return x


def chol_solve(L, b):
    """x = (L L^T)^{-1} b by the two triangular solves of App. A.2."""
    return back_subst_t(L, forward_subst(L, b))


def gram(J, lam):
    """Regularised residual Gramian K + lambda I = J J^T + lambda I (Def. 3.1)."""
    return J @ J.T + lam * np.eye(J.shape[0])


def ga_accept(v, a, eps_norm=0.0, ratio_max=0.5):
    """Acceptance rule of DenseDualSolve (App. A.2): keep v + a/2 when
    ||v|| > eps_norm and 2 ||a|| / ||v|| <= ratio_max, else v.
    Returns (delta, ratio, accepted)."""
    nv = float(np.linalg.norm(v))
    if not nv > eps_norm:
        return v.copy(), float("nan"), False
    ratio = 2.0 * float(np.linalg.norm(a)) / nv
    if ratio <= ratio_max:
        return v + 0.5 * a, ratio, True
    return v.copy(), ratio, False


def dense_step(theta, problem, X, target, lam, use_ga=True, eps_norm=0.0, ratio_max=0.5):
    """One D-NGD step with the dense dual solver (App. A.2, DenseDualSolve),
    push-through recovery.  Returns a dict with r, J, alpha, v, fvv, beta, a,
    ratio, accepted, delta (the step to ADD to theta)."""
    r, J = res.residual_and_jacobian(theta, problem, X, target)
    L = cholesky(gram(J, lam))
    alpha = chol_solve(L, r)
    v = -(J.T @ alpha)
    out = dict(r=r, J=J, L=L, alpha=alpha, v=v)
    if use_ga:
        fvv = res.second_directional(theta, problem, X, target, v)
        beta = chol_solve(L, fvv)
        a = -(J.T @ beta)
        delta, ratio, acc = ga_accept(v, a, eps_norm, ratio_max)
        out.update(fvv=fvv, beta=beta, a=a, ratio=ratio, accepted=acc, delta=delta)
    else:
        out.update(delta=v.copy(), ratio=float("nan"), accepted=False)
    return out


def dense_step_literal(J, r, lam, fvv=None):
    """The paper's literal recovery (Thm. 3.1; Prop. 3.2 dual form):
    y = (K+lambda I)^{-1}(-J g), v = -(J^T y + g)/lambda with g = J^T r;
    y_a = (K+lambda I)^{-1}(-K f_vv), a = -J^T (y_a + f_vv)/lambda.
    Divides by lambda, so it loses accuracy as lambda -> 0."""
    K = J @ J.T
    L = cholesky(K + lam * np.eye(K.shape[0]))
    g = J.T @ r
    y = chol_solve(L, -(J @ g))
    v = -(J.T @ y + g) / lam
    if fvv is None:
        return v, None
    ya = chol_solve(L, -(K @ fvv))
    a = -(J.T @ (ya + fvv)) / lam
    return v, a


def primal_step(J, r, lam):
    """Primal normal equations (J^T J + lambda I) dtheta = -J^T r (Prop. 3.1)."""
    n = J.shape[1]
    return np.linalg.solve(J.T @ J + lam * np.eye(n), -(J.T @ r))
