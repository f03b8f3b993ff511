"""Pins of the oracle's adjoint gradient (CPU only).

J = 1/2 sum_j (vx(1, j) - vx_obs(j))^2 (surface-velocity misfit). The oracle gradient comes from
the linearity of the assembly in eta; it is pinned here against central finite differences in
log(eta) and, independently, against the strain-rate-product closed form derived by discrete
summation by parts (the form the fused GPU kernel evaluates).
"""
import numpy as np
import pytest

from oracle import stokes as S
from synth import random_field_log10, sample_lattice_to_fields


def _setup(n, seed, bc):
    l10 = random_field_log10(n, n, seed, corr_len=0.2)
    rho_s = 1.0 + 0.1 * random_field_log10(n, n, seed + 7, corr_len=0.2)
    f = sample_lattice_to_fields(10.0 ** l10, rho_s, n, n)
    g = S.Grid(n, n, bc=bc)
    rng = np.random.default_rng(seed)
    vx_obs = rng.standard_normal(n + 2) * 1e-3
    return f, g, vx_obs


def _J_and_dJdx(g, x, vx_obs):
    vx, _, _ = S.vector_to_fields(g, x, fill_ghosts=False)
    js = np.arange(1, g.nx)
    mis = vx[1, js] - vx_obs[js]
    dJ = np.zeros(g.n)
    dJ[g.idx_vx[1, js]] = mis
    return 0.5 * np.sum(mis ** 2), dJ


def _solve(g, en, ec, rho):
    sysm = S.assemble(g, en, ec, rho, (0.0, 1.0))
    return sysm, S.solve_direct(sysm)


def _adjoint(g, sysm, dJ):
    # A is symmetric: the adjoint system is A lam = dJ/dx with the same zero-mean gauge
    adj = S.System(g, sysm.A, dJ)
    return S.solve_direct(adj)


@pytest.mark.parametrize("bc", [S.BC(), S.BC(kind=(S.NO_SLIP,) * 4)])
def test_linearity_gradient_matches_central_fd(bc):
    n = 16
    f, g, vx_obs = _setup(n, 11, bc)
    sysm, x = _solve(g, f.eta_n, f.eta_c, f.rho)
    _, dJ = _J_and_dJdx(g, x, vx_obs)
    lam = _adjoint(g, sysm, dJ)
    g_n, g_c = S.eta_gradient_by_linearity(g, f.eta_n, f.eta_c, x, lam)
    h = 1e-5
    errs, scale = [], np.nanmax(np.abs(np.concatenate([(g_c * f.eta_c).ravel(), (g_n * f.eta_n).ravel()])))
    for which, arr, grad in (("c", f.eta_c, g_c), ("n", f.eta_n, g_n)):
        rng_i = range(1, n + 1) if which == "c" else range(0, n + 1)
        for i in rng_i:
            for j in rng_i:
                Jpm = []
                for sgn in (1, -1):
                    a = arr.copy(); a[i, j] *= np.exp(sgn * h)
                    en, ec = (f.eta_n, a) if which == "c" else (a, f.eta_c)
                    _, xs = _solve(g, en, ec, f.rho)
                    Jpm.append(_J_and_dJdx(g, xs, vx_obs)[0])
                fd = (Jpm[0] - Jpm[1]) / (2 * h)
                errs.append(abs(fd - grad[i, j] * arr[i, j]))
    assert max(errs) <= 1e-6 * scale


def _strain_rate_product(g, vx, vy, lx, ly, bc):
    """Closed form: dJ/deta_c = 2 (exx(v) exx(l) + eyy(v) eyy(l)); dJ/deta_n = w_n gam(v) gam(l)
    with w_n = 1 inside, 1/2 on no-slip walls, 0 at corners (unused nodes)."""
    nx, ny, dx, dy = g.nx, g.ny, g.dx, g.dy
    gc = np.zeros((ny + 2, nx + 2)); gn = np.zeros((ny + 2, nx + 2))
    exx = lambda u: (u[1:ny + 1, 1:nx + 1] - u[1:ny + 1, 0:nx]) / dx
    eyy = lambda w: (w[1:ny + 1, 1:nx + 1] - w[0:ny, 1:nx + 1]) / dy
    gc[1:ny + 1, 1:nx + 1] = 2 * (exx(vx) * exx(lx) + eyy(vy) * eyy(ly))
    gam = lambda u, w: (u[1:ny + 2, 0:nx + 1] - u[0:ny + 1, 0:nx + 1]) / dy + (w[0:ny + 1, 1:nx + 2] - w[0:ny + 1, 0:nx + 1]) / dx
    wn = np.ones((ny + 1, nx + 1))
    wn[0, :] *= 0.5; wn[ny, :] *= 0.5; wn[:, 0] *= 0.5; wn[:, nx] *= 0.5
    wn[0, 0] = wn[0, nx] = wn[ny, 0] = wn[ny, nx] = 0.0
    gn[0:ny + 1, 0:nx + 1] = wn * gam(vx, vy) * gam(lx, ly)
    return gn, gc


@pytest.mark.parametrize("bc", [S.BC(), S.BC(kind=(S.NO_SLIP,) * 4),
                                S.BC(kind=(S.FREE_SLIP, S.NO_SLIP, S.NO_SLIP, S.FREE_SLIP))])
def test_strain_rate_product_equals_linearity(bc):
    n = 12
    f, g, vx_obs = _setup(n, 5, bc)
    sysm, x = _solve(g, f.eta_n, f.eta_c, f.rho)
    _, dJ = _J_and_dJdx(g, x, vx_obs)
    lam = _adjoint(g, sysm, dJ)
    g_n, g_c = S.eta_gradient_by_linearity(g, f.eta_n, f.eta_c, x, lam)
    vx, vy, _ = S.vector_to_fields(g, x)
    lx, ly, _ = S.vector_to_fields(g, lam)
    S.fill_boundary(g, lx, ly, homogeneous=True)
    fn, fc = _strain_rate_product(g, vx, vy, lx, ly, bc)
    sc = np.abs(g_c[1:n + 1, 1:n + 1]).max()
    assert np.abs(fc[1:n + 1, 1:n + 1] - g_c[1:n + 1, 1:n + 1]).max() <= 1e-10 * sc
    assert np.abs(fn[:n + 1, :n + 1] - g_n[:n + 1, :n + 1]).max() <= 1e-10 * sc


def test_rho_gradient_matches_fd():
    n = 8
    f, g, vx_obs = _setup(n, 3, S.BC())
    sysm, x = _solve(g, f.eta_n, f.eta_c, f.rho)
    _, dJ = _J_and_dJdx(g, x, vx_obs)
    lam = _adjoint(g, sysm, dJ)
    gr = S.rho_gradient_by_linearity(g, (0.0, 1.0), lam)
    h = 1e-6
    for (i, j) in [(0, 0), (3, 4), (8, 8), (5, 0), (2, 7)]:
        Jpm = []
        for sgn in (1, -1):
            r = f.rho.copy(); r[i, j] += sgn * h
            _, xs = _solve(g, f.eta_n, f.eta_c, r)
            Jpm.append(_J_and_dJdx(g, xs, vx_obs)[0])
        assert (Jpm[0] - Jpm[1]) / (2 * h) == pytest.approx(gr[i, j], rel=1e-5, abs=1e-12)
