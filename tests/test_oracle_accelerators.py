"""Pins of the accelerator oracle (flexible GCR(m), Anderson AA(m, beta)) against facts that do not
come from the oracle itself: finite termination, brute-force residual minimisation over the
Krylov space, the Walker-Ni equivalence of undamped Anderson with GMRES, and the closed form of
depth-0 mixing (damped Richardson)."""
import numpy as np
import pytest

from oracle import accelerators as AC
from oracle import stokes as S
from oracle import multigrid as M


def _nonsym(n, seed):
    rng = np.random.default_rng(seed)
    return np.eye(n) * 4 + 0.6 * rng.standard_normal((n, n)) / np.sqrt(n), rng.standard_normal(n)


def _krylov_basis(op, v, k):
    Q = []
    u = v.copy()
    for _ in range(k):
        for q in Q:
            u = u - (q @ u) * q
        for q in Q:
            u = u - (q @ u) * q
        Q.append(u / np.linalg.norm(u))
        u = op(Q[-1])
    return np.column_stack(Q)


def test_gcr_finite_termination_identity_preconditioner():
    A, b = _nonsym(20, 1)
    x, its = AC.gcr(A, b, lambda r: r, m=25, tol=1e-13, maxit=25)
    assert its <= 20
    assert np.linalg.norm(b - A @ x) <= 1e-12 * np.linalg.norm(b)


@pytest.mark.parametrize("weighted", [False, True])
def test_gcr_iterates_minimise_residual_over_krylov_space(weighted):
    n = 30
    A, b = _nonsym(n, 2)
    rng = np.random.default_rng(3)
    Mi = np.eye(n) + 0.2 * rng.standard_normal((n, n)) / np.sqrt(n)      # fixed preconditioner
    W = rng.uniform(0.5, 2.0, n) if weighted else None
    hist = []
    AC.gcr(A, b, lambda r: Mi @ r, m=50, tol=1e-14, maxit=8, W=W, history=hist)
    Wv = W if W is not None else np.ones(n)
    for k, xk in enumerate(hist, start=1):
        K = _krylov_basis(lambda v: Mi @ (A @ v), Mi @ b, k)       # span{M r0, (M A) M r0, ...}
        AK = A @ K
        c, *_ = np.linalg.lstsq(np.sqrt(Wv)[:, None] * AK, np.sqrt(Wv) * b, rcond=None)
        assert np.linalg.norm(xk - K @ c) <= 1e-9 * np.linalg.norm(K @ c)


def test_gcr_residual_is_monotone_and_solves_stokes_with_uzawa_preconditioner():
    g = S.Grid(16, 12, 1.0, 0.75)
    rng = np.random.default_rng(4)
    en = 10.0 ** rng.uniform(-1, 1, (14, 18)); ec = 10.0 ** rng.uniform(-1, 1, (14, 18))
    rho = 1.0 + 0.1 * rng.standard_normal((14, 18))
    sysm = S.assemble(g, en, ec, rho, (0.0, 1.0))
    h = M.Hierarchy(g, en, ec, coarsest_min=2)
    pre = lambda r: M.uzawa_precond(h, r, ec, alpha=1.0)
    W = np.concatenate([1.0 / -sysm.A.diagonal()[:g.n_v], S.pressure_weights(g, ec)])
    hist = []
    x, its = AC.gcr(sysm.A, sysm.b, pre, m=30, tol=1e-12, maxit=400, W=W, history=hist)
    res = [np.sqrt(np.sum(W * (sysm.b - sysm.A @ xk) ** 2)) for xk in hist[:40]]
    assert all(r1 <= r0 * (1 + 1e-10) for r0, r1 in zip(res, res[1:]))
    xd = S.remove_pressure_mean(g, S.solve_direct(sysm))
    assert np.linalg.norm(S.remove_pressure_mean(g, x) - xd) <= 1e-9 * np.linalg.norm(xd)


def test_constrained_least_squares_satisfies_kkt():
    rng = np.random.default_rng(5)
    F = rng.standard_normal((40, 6))
    a = AC._constrained_lsq(F)
    assert abs(a.sum() - 1) <= 1e-13
    g = F.T @ (F @ a)                      # KKT: F^T F a = lambda 1
    assert np.ptp(g) <= 1e-10 * np.abs(g).max()
    for _ in range(20):
        d = rng.standard_normal(6); d -= d.mean()
        assert np.linalg.norm(F @ (a + 0.1 * d)) >= np.linalg.norm(F @ a) - 1e-12


def test_anderson_undamped_is_gmres_followed_by_one_fixed_point_step():
    """Walker & Ni (SIAM J. Numer. Anal. 49, 2011): for a linear map G and no truncation, AA with
    beta = 1 satisfies x_{k+1} = G(x_k^GMRES), GMRES on M^-1 A x = M^-1 b in the 2-norm."""
    n = 25
    A, b = _nonsym(n, 6)
    rng = np.random.default_rng(7)
    Mi = np.eye(n) / 4 + 0.05 * rng.standard_normal((n, n)) / np.sqrt(n)
    G = lambda x: x + Mi @ (b - A @ x)
    hist = []
    AC.anderson(A, b, lambda r: Mi @ r, m=50, beta=1.0, tol=1e-15, maxit=7, history=hist)
    f0 = Mi @ b
    for k in range(1, len(hist)):
        K = _krylov_basis(lambda v: Mi @ (A @ v), f0, k)
        c, *_ = np.linalg.lstsq(Mi @ A @ K, f0, rcond=None)
        xg = K @ c
        assert np.linalg.norm(hist[k] - G(xg)) <= 1e-8 * np.linalg.norm(G(xg))


@pytest.mark.parametrize("beta", [0.5, 0.8])
def test_anderson_depth_zero_is_damped_richardson(beta):
    n = 12
    A, b = _nonsym(n, 8)
    Mi = np.eye(n) / 4
    hist = []
    AC.anderson(A, b, lambda r: Mi @ r, m=0, beta=beta, tol=1e-16, maxit=6, history=hist)
    x = Mi @ b                                  # x^1 = G(x^0), x^0 = 0
    assert np.allclose(hist[0], x, rtol=1e-14, atol=1e-15)
    for k in range(1, len(hist)):
        x = (1 - beta) * x + beta * (x + Mi @ (b - A @ x))
        assert np.allclose(hist[k], x, rtol=1e-12, atol=1e-14)
