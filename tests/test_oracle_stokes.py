"""Pins of the FP64 oracle against what the paper and the mathematics fix (CPU only)."""
import os
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import stokes as S
from synth import sinker

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")

BCS = {
    "free_slip": S.BC(),
    "no_slip": S.BC(kind=(S.NO_SLIP,) * 4),
    "mixed": S.BC(kind=(S.NO_SLIP, S.FREE_SLIP, S.VELOCITY, S.NO_SLIP), vt=(0, 0, 0.7, 0)),
    "periodic": S.BC(kind=(S.PERIODIC, S.PERIODIC, S.VELOCITY, S.NO_SLIP), vt=(0, 0, 1.0, 0)),
}


def rand_eta(nx, ny, seed, lo=-2, hi=2):
    rng = np.random.default_rng(seed)
    return 10.0 ** rng.uniform(lo, hi, (ny + 2, nx + 2)), 10.0 ** rng.uniform(lo, hi, (ny + 2, nx + 2))


def test_listing_coefficients():
    """Every entry of an interior x-momentum row equals the paper's point listing (golden values)."""
    g = S.Grid(4, 4, Lx=2.0, Ly=1.0)
    assert g.dx == 0.5 and g.dy == 0.25
    eta_n = np.ones((6, 6)); eta_c = np.ones((6, 6))
    i, j = 2, 2
    eta_c[i, j] = 2.0; eta_c[i, j + 1] = 3.0; eta_n[i - 1, j] = 5.0; eta_n[i, j] = 7.0
    A = S.assemble(g, eta_n, eta_c).A.tocsr()
    row = g.idx_vx[i, j]
    idx = {"vx": g.idx_vx, "vy": g.idx_vy, "p": g.idx_p}
    seen = 0
    for line in open(os.path.join(GOLDEN, "listing_vx_coefficients.txt")):
        if line.startswith("#") or not line.strip():
            continue
        name, di, dj, fld, val = line.split()
        col = idx[fld][i + int(di), j + int(dj)]
        assert A[row, col] == pytest.approx(float(val), rel=1e-15), name
        seen += 1
    assert seen == 11 and A[row].nnz == 11


@pytest.mark.parametrize("bc", list(BCS))
def test_symmetry(bc):
    """<Ax, y> = <x, Ay>: D = G^T and the ghost elimination only touches diagonals."""
    g = S.Grid(12, 10, 1.3, 0.9, BCS[bc])
    en, ec = rand_eta(12, 10, 1)
    A = S.assemble(g, en, ec).A
    rng = np.random.default_rng(2)
    x, y = rng.standard_normal(g.n), rng.standard_normal(g.n)
    lhs, rhs = (A @ x) @ y, x @ (A @ y)
    assert abs(lhs - rhs) <= 1e-13 * abs(A).sum() * 1e-2
    assert abs(A - A.T).max() <= 1e-14 * abs(A).max()


@pytest.mark.parametrize("bc", list(BCS))
def test_L_negative_definite(bc):
    g = S.Grid(8, 6, 1.0, 1.0, BCS[bc])
    en, ec = rand_eta(8, 6, 3)
    L = S.assemble(g, en, ec, velocity_only=True).A.toarray()
    np.linalg.cholesky(-L)
    assert np.linalg.eigvalsh(-L).min() > 0


@pytest.mark.parametrize("bc", ["free_slip", "no_slip", "mixed"])
def test_direct_equals_dense_lu(bc):
    g = S.Grid(10, 12, 1.0, 1.2, BCS[bc])
    en, ec = rand_eta(10, 12, 4)
    rho = np.random.default_rng(5).uniform(0.9, 1.1, (14, 12))
    sysm = S.assemble(g, en, ec, rho, (0.3, 1.0))
    x = S.solve_direct(sysm)
    K = S.bordered(sysm).toarray()
    xd = np.linalg.solve(K, np.concatenate([sysm.b, [0.0]]))[:-1]
    assert np.linalg.norm(x - xd) <= 1e-12 * np.linalg.norm(xd)


def test_hydrostatic():
    """Uniform density, any viscosity: v = 0 and p = rho g_y (y - mean y) exactly."""
    nx, ny = 16, 12
    en, ec = rand_eta(nx, ny, 6)
    rho = np.full((ny + 2, nx + 2), 1.7)
    sol = S.solve_fields(nx, ny, 1.0, 1.5, en, ec, rho, (0.0, 2.0))
    g = S.Grid(nx, ny, 1.0, 1.5)
    y = (np.arange(ny + 2) - 0.5) * g.dy
    pex = 1.7 * 2.0 * (y - y[1:ny + 1].mean())
    assert np.abs(sol.vx).max() < 1e-12 and np.abs(sol.vy).max() < 1e-12
    assert np.abs(sol.p[1:ny + 1, 1:nx + 1] - pex[1:ny + 1, None]).max() < 1e-11


def test_couette():
    """Periodic x, top moving at U, bottom no slip: vx = U (1 - y / Ly) to rounding."""
    nx, ny, U = 8, 16, 1.3
    bc = S.BC(kind=(S.PERIODIC, S.PERIODIC, S.VELOCITY, S.NO_SLIP), vt=(0, 0, U, 0))
    one = np.ones((ny + 2, nx + 2))
    sol = S.solve_fields(nx, ny, 2.0, 1.0, 3.0 * one, 3.0 * one, one, (0.0, 0.0), bc)
    y = (np.arange(1, ny + 1) - 0.5) / ny
    assert np.abs(sol.vx[1:ny + 1, :nx] - (U * (1 - y))[:, None]).max() < 1e-13
    assert np.abs(sol.vy).max() < 1e-13 and np.abs(sol.p).max() < 1e-11


def test_poiseuille():
    """Periodic x, no-slip top/bottom, body force rho g_x: discrete solution is the parabola plus
    the constant dy^2/4 forced by the mirror ghost (exact for quadratics)."""
    nx, ny, eta, gx = 6, 20, 2.5, 0.8
    bc = S.BC(kind=(S.PERIODIC, S.PERIODIC, S.NO_SLIP, S.NO_SLIP))
    one = np.ones((ny + 2, nx + 2))
    sol = S.solve_fields(nx, ny, 1.0, 1.0, eta * one, eta * one, one, (gx, 0.0), bc)
    dy = 1.0 / ny
    y = (np.arange(1, ny + 1) - 0.5) * dy
    ex = gx / (2 * eta) * (y * (1 - y) + dy * dy / 4)
    assert np.abs(sol.vx[1:ny + 1, :nx] - ex[:, None]).max() < 1e-13
    # the continuous parabola alone is off by exactly gx dy^2 / (8 eta)
    assert np.abs(sol.vx[1:ny + 1, 0] - gx / (2 * eta) * y * (1 - y)).min() == pytest.approx(gx * dy * dy / (8 * eta), rel=1e-9)


def _manufactured(n):
    import sympy as sy
    x, y = sy.symbols("x y")
    psi = sy.sin(sy.pi * x) * sy.sin(sy.pi * y)
    vx, vy = sy.diff(psi, y), -sy.diff(psi, x)
    p = sy.cos(sy.pi * x) * sy.cos(sy.pi * y)
    eta = sy.exp(x * y)
    sxx = 2 * eta * sy.diff(vx, x); syy = 2 * eta * sy.diff(vy, y)
    sxy = eta * (sy.diff(vx, y) + sy.diff(vy, x))
    fx = sy.diff(sxx, x) + sy.diff(sxy, y) - sy.diff(p, x)
    fy = sy.diff(sxy, x) + sy.diff(syy, y) - sy.diff(p, y)
    F = {k: sy.lambdify((x, y), v, "numpy") for k, v in
         dict(vx=vx, vy=vy, p=p, eta=eta, fx=fx, fy=fy).items()}
    g = S.Grid(n, n)
    h = 1.0 / n
    jn, in_ = np.meshgrid(np.arange(n + 2) * h, np.arange(n + 2) * h)
    en = F["eta"](jn, in_)
    ec = F["eta"](jn - h / 2, in_ - h / 2)
    sysm = S.assemble(g, en, ec)
    b = sysm.b.copy()
    b[:g.n_vx] = F["fx"](g.vx_j * h, (g.vx_i - 0.5) * h)
    b[g.n_vx:g.n_v] = F["fy"]((g.vy_j - 0.5) * h, g.vy_i * h)
    sysm.b = b
    xs = S.solve_direct(sysm)
    ex_v = np.concatenate([F["vx"](g.vx_j * h, (g.vx_i - 0.5) * h), F["vy"]((g.vy_j - 0.5) * h, g.vy_i * h)])
    ex_p = F["p"]((g.p_j - 0.5) * h, (g.p_i - 0.5) * h)
    ex_p -= ex_p.mean()
    ev = np.sqrt(np.mean((xs[:g.n_v] - ex_v) ** 2))
    ep = np.sqrt(np.mean((xs[g.n_v:] - ex_p) ** 2))
    return ev, ep


def test_manufactured_second_order():
    errs = [_manufactured(n) for n in (16, 32, 64, 128)]
    for (ev0, ep0), (ev1, ep1) in zip(errs[:-1], errs[1:]):
        assert 1.8 <= np.log2(ev0 / ev1) <= 2.2
        assert 1.8 <= np.log2(ep0 / ep1) <= 2.2


def test_sinker_divergence_and_symmetry():
    f = sinker(64, 64)
    sol = S.solve_fields(64, 64, 1.0, 1.0, f.eta_n, f.eta_c, f.rho, (0.0, 1.0))
    h = 1.0 / 64
    div = (sol.vx[1:65, 1:65] - sol.vx[1:65, 0:64]) / h + (sol.vy[1:65, 1:65] - sol.vy[0:64, 1:65]) / h
    vmax = max(np.abs(sol.vx).max(), np.abs(sol.vy).max())
    assert np.abs(div).max() <= 1e-10 * vmax / h
    # two symmetric counter-rotating cells: vx odd, vy even about x = 1/2
    vx = sol.vx[1:65, 0:65]; vy = sol.vy[0:65, 1:65]
    assert np.abs(vx + vx[:, ::-1]).max() <= 1e-9 * vmax
    assert np.abs(vy - vy[:, ::-1]).max() <= 1e-9 * vmax
    # the dense inclusion sinks: vy > 0 (toward larger row index) at the centre
    assert vy[32, 32] > 0
    assert sol.rel_energy < 1e-12


def test_energy_residual_special_values():
    f = sinker(16, 16)
    g = S.Grid(16, 16)
    sysm = S.assemble(g, f.eta_n, f.eta_c, f.rho, (0.0, 1.0))
    e0, l0 = S.energy_residual(sysm, f.eta_c, np.zeros(g.n))
    assert e0 == pytest.approx(1.0, rel=1e-15) and l0 == pytest.approx(1.0, rel=1e-15)
    x = S.solve_direct(sysm)
    assert S.energy_residual(sysm, f.eta_c, x)[0] < 1e-13
    # a residual living only in one pressure cell: sqrt(r^2 eta/(2/dx^2+2/dy^2) / |f|^2_W)
    r = np.zeros(g.n); r[g.n_v + 5] = 3.0
    dL = -sysm.A.diagonal()[:g.n_v]
    fw = np.sum(sysm.b[:g.n_v] ** 2 / dL)
    wp = f.eta_c[g.p_i[5], g.p_j[5]] / (2 * 16**2 + 2 * 16**2)
    rr = S.System(g, sysm.A, sysm.b + r)
    e1, _ = S.energy_residual(rr, f.eta_c, x)
    assert e1 == pytest.approx(np.sqrt(9.0 * wp / fw), rel=1e-6)


def test_lithostatic_pressure_balances_horizontally_layered_density():
    """For rho varying with depth only (any viscosity, any horizontal gravity-free column), the
    lithostatic pressure with v = 0 is the exact discrete solution: the oracle's assembled
    residual vanishes."""
    nx, ny = 12, 16
    en, ec = rand_eta(nx, ny, 8)
    rho = np.repeat(1.0 + 0.3 * np.sin(np.arange(ny + 2) * 0.7)[:, None], nx + 2, axis=1)
    g = S.Grid(nx, ny, 1.0, 1.4)
    p = S.lithostatic_pressure(g, rho, (0.0, 2.5))
    sysm = S.assemble(g, en, ec, rho, (0.0, 2.5))
    x = S.fields_to_vector(g, np.zeros_like(p), np.zeros_like(p), p)
    r = sysm.b - sysm.A @ x
    assert np.abs(r).max() <= 1e-12 * np.abs(sysm.b).max()
    sol = S.solve_fields(nx, ny, 1.0, 1.4, en, ec, rho, (0.0, 2.5))
    assert np.abs(sol.p[1:ny + 1, 1:nx + 1] - p[1:ny + 1, 1:nx + 1]).max() <= 1e-10 * np.abs(p).max()


def test_viscosity_blend_end_points_and_contrast():
    nx, ny = 10, 8
    en, ec = rand_eta(nx, ny, 9)
    emin = min(en[:ny + 1, :nx + 1].min(), ec[1:ny + 1, 1:nx + 1].min())
    a_n, a_c = S.blend_viscosity(en, ec, 0.0, nx, ny)
    assert np.all(a_n[:ny + 1, :nx + 1] == emin) and np.all(a_c[1:ny + 1, 1:nx + 1] == emin)
    b_n, b_c = S.blend_viscosity(en, ec, 1.0, nx, ny)
    assert np.array_equal(b_n, en) and np.array_equal(b_c, ec)
    h_n, h_c = S.blend_viscosity(en, ec, 0.5, nx, ny)
    emax = max(en[:ny + 1, :nx + 1].max(), ec[1:ny + 1, 1:nx + 1].max())
    # the contrast of the blend is (emin + emax) / (2 emin), monotone in theta
    assert np.isclose(max(h_n[:ny + 1, :nx + 1].max(), h_c[1:ny + 1, 1:nx + 1].max()) / emin, (emin + emax) / (2 * emin))
