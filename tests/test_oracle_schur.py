"""Pins of the oracle's weighted BFBt Schur-complement surrogate and its smoothed-aggregation
pressure multigrid (CPU only). Neither is in the paper; both are pinned by properties the
mathematics fixes, not by re-typing their formulas:
  * the multigrid: Galerkin coarse operators keep symmetry and the constant null space, the
    smoothed prolongator reproduces constants, the coarse stencils stay inside a 5 x 5 box, the
    two-grid correction is the K-orthogonal projection onto the range of P, and the cycle contracts
    a plain Poisson problem at a textbook multigrid rate;
  * the surrogate: it is symmetric positive semi-definite like the Schur complement it replaces, it
    is spectrally equivalent to it at constant viscosity, and on a high-contrast inclusion it is far
    better conditioned than the paper's diagonal viscosity surrogate.
"""
import numpy as np
import scipy.sparse as sp
import pytest

from oracle import stokes as S
from oracle import multigrid as M
from synth import sinker


def _random_K(nx, ny, seed, decades=3):
    rng = np.random.default_rng(seed)
    cx = 10.0 ** rng.uniform(-decades, 0, (ny, nx - 1))
    cy = 10.0 ** rng.uniform(-decades, 0, (ny - 1, nx))
    idx = np.arange(nx * ny).reshape(ny, nx)
    rows, cols, vals = [], [], []
    for a, b, c in ((idx[:, :-1], idx[:, 1:], cx), (idx[:-1, :], idx[1:, :], cy)):
        a, b, c = a.ravel(), b.ravel(), c.ravel()
        rows += [a, b, a, b]; cols += [a, b, b, a]; vals += [c, c, -c, -c]
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(nx * ny,) * 2)


def test_pressure_amg_coarse_operators_keep_symmetry_null_space_and_a_5x5_stencil():
    nx, ny = 37, 23
    amg = M.PressureAMG(_random_K(nx, ny, 1), nx, ny, max_coarse=16)
    assert amg.nlev >= 4
    for l, K in enumerate(amg.K):
        assert abs(K - K.T).max() <= 1e-13 * abs(K).max()
        assert np.abs(K @ np.ones(K.shape[0])).max() <= 1e-12 * abs(K).max()
        lnx = amg.shape[l][0]
        C = K.tocoo()
        assert np.all(np.abs(C.row // lnx - C.col // lnx) <= 2) and np.all(np.abs(C.row % lnx - C.col % lnx) <= 2)
    for P in amg.P:
        assert np.allclose(P @ np.ones(P.shape[1]), 1.0, atol=1e-13)
    assert amg.shape[-1][0] * amg.shape[-1][1] <= 16


def test_two_grid_correction_is_the_K_orthogonal_projection():
    nx, ny = 12, 10
    K = _random_K(nx, ny, 2)
    amg = M.PressureAMG(K, nx, ny, nu=0, max_coarse=30)      # exactly two levels, no smoothing
    assert amg.nlev == 2
    f = np.random.default_rng(3).standard_normal(nx * ny)
    f -= f.mean()
    x = amg.vcycle(f)
    P = amg.P[0]
    assert np.abs(P.T @ (f - K @ x)).max() <= 1e-10 * np.abs(f).max()


def test_pressure_amg_cycle_contracts_poisson_at_a_multigrid_rate():
    n = 64
    idx = np.arange(n * n).reshape(n, n)
    K = _random_K(n, n, 4, decades=0)                       # unit conductances: the 5-point Laplacian
    amg = M.PressureAMG(K, n, n)
    x = np.random.default_rng(5).standard_normal(n * n)
    x -= x.mean()
    norms = []
    for _ in range(12):
        r = -K @ x
        norms.append(np.linalg.norm(r))
        x = x + amg.vcycle(r)
        x -= x.mean()
    rate = (norms[-1] / norms[-6]) ** 0.2
    assert rate <= 0.2, rate


def _dense_blocks(sysm):
    g = sysm.grid
    A = sysm.A.toarray()
    nv = g.n_v
    return A[:nv, :nv], A[:nv, nv:], A[nv:, :nv]


def _surrogate_matrix(B, npr):
    return np.column_stack([B.apply(e) for e in np.eye(npr)])


def test_weighted_bfbt_is_symmetric_positive_semidefinite_and_equivalent_at_constant_viscosity():
    n = 12
    g = S.Grid(n, n, 1.0, 1.0)
    eta = 3.0 * np.ones((n + 2, n + 2))
    sysm = S.assemble(g, eta, eta)
    L, G, D = _dense_blocks(sysm)
    Sch = -D @ np.linalg.solve(L, G)
    B = M.WeightedBFBt(sysm, exact=True)
    St = _surrogate_matrix(B, g.n_p)
    assert np.abs(St - St.T).max() <= 1e-10 * np.abs(St).max()
    Q = np.linalg.qr(np.column_stack([np.ones(g.n_p), np.eye(g.n_p)[:, :-1]]))[0][:, 1:]  # mean-zero basis
    assert np.linalg.eigvalsh(Q.T @ St @ Q).min() > 0
    ev = np.linalg.eigvals(Q.T @ St @ Sch @ Q).real
    assert ev.min() >= 0.5 and ev.max() <= 2.0, (ev.min(), ev.max())


def test_weighted_bfbt_cuts_krylov_iterations_on_the_lid_and_inclusions_field():
    """With exact velocity solves the pressure block alone decides the FGMRES iteration count. On the
    lid + inclusions field (viscosity 1e-3 .. 1e6) the weighted BFBt block, with its multigrid K^-1,
    needs less than half the iterations of the paper's diagonal viscosity surrogate (measured: 62 vs
    263 at 48 x 48, 49 with exact K^-1)."""
    import scipy.sparse.linalg as spla
    from oracle import iterative as I
    from synth import layered_config
    n = 48
    f = layered_config(n, n, seed=3)
    g = S.Grid(n, n)
    sysm = S.assemble(g, f.eta_n, f.eta_c, f.rho, (0.0, 1.0))
    nv = g.n_v
    A = sysm.A.tocsr()
    lu = spla.splu(A[:nv, :nv].tocsc())
    D = A[nv:, :nv]
    ec = g.eta_c_at(f.eta_c, g.p_i, g.p_j)
    its = {}
    for name, sch in (("eta", None), ("bfbt", M.WeightedBFBt(sysm))):
        def prec(r, sch=sch):
            zv = lu.solve(r[:nv])
            y = r[nv:] - D @ zv
            zp = ec * y if sch is None else sch.apply(y)
            return np.concatenate([zv, zp - zp.mean()])
        res = I.fgmres(sysm, f.eta_c, prec, tol=1e-10, m=400, max_iter=400)
        assert res.rel_energy <= 1e-10
        its[name] = res.iterations
    assert 2 * its["bfbt"] <= its["eta"], its
