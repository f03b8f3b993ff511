"""Pins of the oracle's iterative reference solve (CPU only).

The iterative reference (restarted flexible GMRES with an exact-velocity block preconditioner,
oracle/iterative.py) exists to reach sizes the direct solve cannot. It is pinned to something other
than itself: on grids the direct sparse LU of the bordered system still solves in seconds, the two
must give the same solution (the discrete system has one solution up to the pressure constant,
which both remove), and the residual it reports must be the true residual recomputed from the
assembled matrix (Sec. "Global Relative Energy Residual").
"""
import numpy as np
import pytest

from oracle import stokes as S
from oracle import iterative as I
from synth import grf_config, sinker


def _case(name):
    if name == "grf64":
        f = grf_config(64, 64, seed=2)
        return f, S.Grid(64, 64)
    if name == "sinker64":
        f = sinker(64, 64)
        return f, S.Grid(64, 64)
    if name == "grf48x32_mixed_bc":
        f = grf_config(48, 32, seed=5, Lx=1.5, Ly=1.0)
        bc = S.BC((S.NO_SLIP, S.FREE_SLIP, S.VELOCITY, S.NO_SLIP), (0, 0, 0.3, 0))
        return f, S.Grid(48, 32, 1.5, 1.0, bc)
    raise KeyError(name)


@pytest.mark.parametrize("name", ["grf64", "sinker64", "grf48x32_mixed_bc"])
def test_iterative_reference_equals_direct_solve(name):
    f, g = _case(name)
    sysm = S.assemble(g, f.eta_n, f.eta_c, f.rho, (0.0, 1.0))
    res = I.solve_reference(sysm, f.eta_c, tol=1e-13)
    assert res.rel_energy <= 1e-13
    xd = S.remove_pressure_mean(g, S.solve_direct(sysm))
    nv = g.n_v
    dv = np.linalg.norm(res.x[:nv] - xd[:nv]) / np.linalg.norm(xd[:nv])
    dp = np.linalg.norm(res.x[nv:] - xd[nv:]) / np.linalg.norm(xd[nv:])
    assert dv <= 1e-10 and dp <= 1e-10, (dv, dp)


def test_reported_residual_is_the_true_residual_and_pressure_has_zero_mean():
    f, g = _case("grf64")
    sysm = S.assemble(g, f.eta_n, f.eta_c, f.rho, (0.0, 1.0))
    res = I.solve_reference(sysm, f.eta_c, tol=1e-9)
    e, l2 = S.energy_residual(sysm, f.eta_c, res.x)
    assert res.rel_energy == e and res.rel_l2 == l2
    assert e <= 1e-9
    assert abs(res.x[g.n_v:].mean()) <= 1e-14 * np.abs(res.x[g.n_v:]).max()
    # the history is made of true residuals, and it ends with the returned one
    assert res.history[-1][1] == pytest.approx(e, rel=1e-6)


def test_energy_weights_follow_the_paper_norm():
    # W reproduces the relative energy residual of the oracle's own norm for any vector
    f, g = _case("sinker64")
    sysm = S.assemble(g, f.eta_n, f.eta_c, f.rho, (0.0, 1.0))
    W = I.energy_weights(sysm, f.eta_c)
    x = np.random.default_rng(3).standard_normal(g.n)
    r = sysm.b - sysm.A @ x
    den = np.sum(W[:g.n_v] * sysm.b[:g.n_v] ** 2)
    assert np.sqrt(np.sum(W * r * r) / den) == pytest.approx(S.energy_residual(sysm, f.eta_c, x)[0], rel=1e-12)



def test_bfbt_preconditioned_reference_equals_direct_solve_on_the_layered_field():
    """The reference form used for the layered workload (exact velocity LU, weighted BFBt pressure
    block) reaches the direct solution of a lid + inclusions field with viscosity from 1e-3 to 1e6."""
    from oracle import multigrid as M
    from synth import layered_config
    n = 64
    f = layered_config(n, n, seed=3)
    g = S.Grid(n, n)
    sysm = S.assemble(g, f.eta_n, f.eta_c, f.rho, (0.0, 1.0))
    res = I.solve_reference(sysm, f.eta_c, tol=1e-13, m=200, schur=M.WeightedBFBt(sysm))
    assert res.rel_energy <= 1e-13
    xd = S.remove_pressure_mean(g, S.solve_direct(sysm))
    nv = g.n_v
    dv = np.linalg.norm(res.x[:nv] - xd[:nv]) / np.linalg.norm(xd[:nv])
    dp = np.linalg.norm(res.x[nv:] - xd[nv:]) / np.linalg.norm(xd[nv:])
    assert dv <= 1e-9 and dp <= 1e-9, (dv, dp)
