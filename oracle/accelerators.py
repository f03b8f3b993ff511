"""Plain FP64 CPU oracle of the paper's own outer accelerators (test infrastructure only).

  * flexible GCR(m) (Sec. "Generalized Conjugate Residual Method", Algorithm gcr): each step
    preconditions the current residual, maps the direction through A, orthogonalises the image
    against the earlier images by modified Gram-Schmidt (the same coefficients update the
    directions), normalises, and moves x and r along the new pair; restarts after m steps;
  * Anderson acceleration AA(m) with mixing beta (Sec. "Anderson Acceleration", Algorithm
    anderson) of the fixed-point map G(x) = x + M^-1 (b - A x): the newest m+1 fixed-point
    residuals f_i = G(x_i) - x_i are combined with weights that sum to one and minimise the norm
    of the combination, and x_{k+1} = sum a_i ((1 - beta) x_i + beta G(x_i)).

Readings (listed with the design notes):
  * inner product: both take an optional positive weight vector W and use <u, v> = sum W u v.
    GCR with W = the energy weights (diag(-L)^-1 on velocities, eta/(2/dx^2+2/dy^2) on pressure)
    minimises the relative energy residual the solver stops on, as FGMRES does; Anderson's
    least-squares norm is the plain 2-norm of the paper unless a weight is given;
  * the stopping test of both is the relative energy residual of the current iterate;
  * GCR's restart keeps x and the recursively updated residual r (Algorithm gcr) unless
    `true_residual_at_restart`, which recomputes r = b - A x there.
"""
import numpy as np


def _dot(W, u, v):
    return float(np.dot(u * W, v)) if W is not None else float(np.dot(u, v))


def gcr(A, b, precond, x0=None, m=30, tol=1e-10, maxit=1000, W=None, stop_norm=None,
        true_residual_at_restart=False, history=None):
    """Flexible GCR(m) for A x = b. `A` is a callable or matrix, `precond(r)` returns M_k^-1 r.
    Stops when stop_norm(r) <= tol * stop_norm(b) (default: the W-norm). Returns (x, iters)."""
    Aop = A if callable(A) else (lambda v: A @ v)
    nrm = stop_norm if stop_norm is not None else (lambda v: np.sqrt(_dot(W, v, v)))
    x = np.zeros_like(b) if x0 is None else x0.copy()
    r = b - Aop(x)
    nb = nrm(b)
    its = 0
    if nb == 0.0:
        return x, 0
    while nrm(r) > tol * nb and its < maxit:
        Ws, Zs = [], []
        for i in range(m):
            z = precond(r)                       # z^{k+i} = M^-1 r^{k+i}
            w = Aop(z)                           # w^{k+i} = A z^{k+i}
            for wj, zj in zip(Ws, Zs):           # modified Gram-Schmidt; w_j are normalised
                g = _dot(W, w, wj)
                w = w - g * wj
                z = z - g * zj
            nu = np.sqrt(_dot(W, w, w))
            w = w / nu
            z = z / nu
            a = _dot(W, r, w)
            x = x + a * z
            r = r - a * w
            Ws.append(w); Zs.append(z)
            its += 1
            if history is not None:
                history.append(x.copy())
            if nrm(r) <= tol * nb or its >= maxit:
                break
        if true_residual_at_restart:
            r = b - Aop(x)
    return x, its


def anderson(A, b, precond, x0=None, m=5, beta=1.0, tol=1e-10, maxit=1000, W=None, stop_norm=None,
             history=None):
    """Anderson acceleration AA(m) with mixing beta of G(x) = x + M^-1 (b - A x).
    Returns (x, iterations); one iteration = one application of G."""
    Aop = A if callable(A) else (lambda v: A @ v)
    nrm = stop_norm if stop_norm is not None else (lambda v: np.sqrt(_dot(W, v, v)))

    def G(x):
        return x + precond(b - Aop(x))

    x = np.zeros_like(b) if x0 is None else x0.copy()
    nb = nrm(b)
    if nb == 0.0:
        return x, 0
    X, GX = [x], [G(x)]                           # x^0 and G(x^0)
    x = GX[0]                                     # x^1 := G(x^0)
    its = 1
    if history is not None:
        history.append(x.copy())
    while its < maxit:
        if nrm(b - Aop(x)) <= tol * nb:
            break
        X.append(x)
        GX.append(G(x))
        X, GX = X[-(m + 1):], GX[-(m + 1):]        # the newest m_k + 1 = min(m, k) + 1 pairs
        F = np.column_stack([gx - xx for xx, gx in zip(X, GX)])
        if W is not None:
            F = F * np.sqrt(W)[:, None]
        a = _constrained_lsq(F)
        x = sum(ai * ((1.0 - beta) * xx + beta * gx) for ai, xx, gx in zip(a, X, GX))
        its += 1
        if history is not None:
            history.append(x.copy())
    return x, its


def _constrained_lsq(F):
    """argmin ||F a||_2 subject to sum(a) = 1, by eliminating the constraint:
    a = e_last + D c with D the differences basis, c from an ordinary least-squares solve."""
    n = F.shape[1]
    if n == 1:
        return np.array([1.0])
    # a_i = c_i for i < n-1, a_{n-1} = 1 - sum c  =>  F a = f_last + (F[:, :-1] - f_last) c
    fl = F[:, -1]
    Dm = F[:, :-1] - fl[:, None]
    c, *_ = np.linalg.lstsq(Dm, -fl, rcond=None)
    return np.concatenate([c, [1.0 - c.sum()]])
