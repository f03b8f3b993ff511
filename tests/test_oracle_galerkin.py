"""Pins of the oracle's Galerkin coarse velocity operators (CPU only; not in the paper).

L_c = R L P with the cycle's own transfer operators. Pinned by what that product must satisfy:
  * a uniform velocity field has no strain, so L annihilates it away from the walls, P reproduces it
    there and R averages: the interior rows of each coarse level sum to zero within a field;
  * R is P^T / 4 at interior points (factor 2), so L_c is symmetric on rows away from the walls,
    like L itself;
  * the stencil stays within the 31 offsets the GPU stores (vx-vx 5 x 3, vx-vy 4 x 4, mirrored);
  * only levels reached by a chain of halvings are replaced;
  * with damped-Jacobi smoothing on those levels the cycle contracts a constant-viscosity problem at
    a multigrid rate.
"""
import numpy as np
import pytest

from oracle import stokes as S
from oracle import multigrid as M
from synth import layered_config


def _rows(c, r):
    if r < c.n_vx:
        return 0, c.vx_i[r], c.vx_j[r]
    return 1, c.vy_i[r - c.n_vx], c.vy_j[r - c.n_vx]


def test_galerkin_rows_annihilate_uniform_fields_and_are_symmetric_inside():
    n = 32
    f = layered_config(n, n, seed=3)
    h = M.Hierarchy(S.Grid(n, n), f.eta_n, f.eta_c, coarsest_min=4, galerkin=True)
    assert h.gal[1:] == [True] * (h.nlev - 1)
    for l in range(1, h.nlev - 1):
        c = h.grids[l]
        A = h.L[l].tocsr()
        ones_x = np.concatenate([np.ones(c.n_vx), np.zeros(c.n_vy)])
        ones_y = np.concatenate([np.zeros(c.n_vx), np.ones(c.n_vy)])
        for r in range(A.shape[0]):
            fld, i, j = _rows(c, r)
            if not (3 <= i <= c.ny - 2 and 3 <= j <= c.nx - 2):
                continue
            scale = abs(A[r, r])
            assert abs(A[r] @ (ones_x if fld == 0 else ones_y)) <= 1e-10 * scale
            cols = A.indices[A.indptr[r]:A.indptr[r + 1]]
            for col in cols:
                f2, i2, j2 = _rows(c, col)
                if 3 <= i2 <= c.ny - 2 and 3 <= j2 <= c.nx - 2:
                    assert abs(A[r, col] - A[col, r]) <= 1e-10 * scale


def test_galerkin_stencil_fits_the_stored_offsets():
    n = 32
    f = layered_config(n, n, seed=4)
    h = M.Hierarchy(S.Grid(n, n), f.eta_n, f.eta_c, coarsest_min=4, galerkin=True)
    allowed = {(0, 0): (range(-2, 3), range(-1, 2)), (0, 1): (range(-2, 2), range(-1, 3)),
               (1, 1): (range(-1, 2), range(-2, 3)), (1, 0): (range(-1, 3), range(-2, 2))}
    for l in range(1, h.nlev):
        c = h.grids[l]
        A = h.L[l].tocoo()
        for r, col, v in zip(A.row, A.col, A.data):
            if v == 0:
                continue
            f1, i1, j1 = _rows(c, r)
            f2, i2, j2 = _rows(c, col)
            di_ok, dj_ok = allowed[(f1, f2)]
            assert (i2 - i1) in di_ok and (j2 - j1) in dj_ok


def test_only_levels_reached_by_halving_are_galerkin():
    f = layered_config(120, 90, seed=5, Lx=1.2, Ly=0.9)
    h = M.Hierarchy(S.Grid(120, 90, 1.2, 0.9), f.eta_n, f.eta_c, coarsest_min=2, galerkin=True)
    sizes = [(g.nx, g.ny) for g in h.grids]
    assert sizes[:2] == [(120, 90), (60, 45)] and h.gal[1] and not any(h.gal[2:])


def test_galerkin_cycle_contracts_a_constant_viscosity_problem():
    n = 64
    g = S.Grid(n, n)
    eta = np.ones((n + 2, n + 2))
    h = M.Hierarchy(g, eta, eta, coarsest_min=4, galerkin=True)
    L = h.L[0]
    x = np.random.default_rng(0).standard_normal(L.shape[0])
    norms = []
    for _ in range(12):
        r = -L @ x
        norms.append(np.linalg.norm(r))
        x = x + M.vcycle(h, r, 2, 2, 1.0)
    rate = (norms[-1] / norms[-6]) ** 0.2
    assert rate <= 0.3, rate
