"""Pins of the marker oracle. Interpolation (Sec. "Marker-to-grid interpolation", "Grid-to-marker
interpolation"): partition of unity, exactness of the bilinear gather on bilinear fields, and the
equal-weight average of symmetric markers. Advection (Sec. "Advection of Lagrangian Markers"): the
closed-form amplification of each scheme in a rigid rotation, the convergence orders against the
exact trajectory of a bilinear velocity field, the third-order term of the Taylor update,
uniform translation with the wall clamp, and the CFL step."""
import numpy as np
import pytest

from oracle import markers as MK

NX, NY, LX, LY = 12, 9, 1.5, 1.0


def _nodes(kind):
    dx, dy = LX / NX, LY / NY
    x0, y0, *_ = MK.lattice(NX, NY, LX, LY, kind)
    jj, ii = np.meshgrid(np.arange(NX + 2), np.arange(NY + 2))
    return x0 + jj * dx, y0 + ii * dy


@pytest.mark.parametrize("kind", [MK.BASIC_NODES, MK.CELL_CENTRES])
def test_constant_field_is_reproduced_where_markers_reach(kind):
    rng = np.random.default_rng(1)
    xm, ym = rng.uniform(0, LX, 2000), rng.uniform(0, LY, 2000)
    g, w = MK.markers_to_grid(NX, NY, LX, LY, kind, xm, ym, np.full(2000, 3.25), np.zeros((NY + 2, NX + 2)))
    assert np.all(w >= 0) and np.count_nonzero(w) > 0
    assert np.allclose(g[w > 0], 3.25, rtol=0, atol=1e-14)
    assert np.all(g[w == 0] == 0)


@pytest.mark.parametrize("kind", [MK.BASIC_NODES, MK.CELL_CENTRES, MK.VX_POINTS, MK.VY_POINTS])
def test_grid_to_markers_is_exact_on_bilinear_fields(kind):
    X, Y = _nodes(kind)
    f = lambda x, y: 0.3 - 1.2 * x + 0.7 * y + 2.1 * x * y
    rng = np.random.default_rng(2)
    x0, y0, ilo, ihi, jlo, jhi = MK.lattice(NX, NY, LX, LY, kind)
    dx, dy = LX / NX, LY / NY
    xm = rng.uniform(x0 + jlo * dx, x0 + jhi * dx, 500)
    ym = rng.uniform(y0 + ilo * dy, y0 + ihi * dy, 500)
    got = MK.grid_to_markers(NX, NY, LX, LY, kind, xm, ym, f(X, Y))
    assert np.allclose(got, f(xm, ym), rtol=0, atol=1e-13)


def test_symmetric_markers_average_linear_field_exactly():
    """One marker at the centre of every basic-node cell: each interior node gets the mean of its
    four surrounding markers with equal weights 1/4, which is exact for a linear field."""
    dx, dy = LX / NX, LY / NY
    xc, yc = np.meshgrid((np.arange(NX) + 0.5) * dx, (np.arange(NY) + 0.5) * dy)
    f = lambda x, y: 1.0 + 2.0 * x - 3.0 * y
    g, w = MK.markers_to_grid(NX, NY, LX, LY, MK.BASIC_NODES, xc.ravel(), yc.ravel(), f(xc, yc).ravel(),
                              np.zeros((NY + 2, NX + 2)))
    X, Y = _nodes(MK.BASIC_NODES)
    inner = (slice(1, NY), slice(1, NX))
    assert np.allclose(w[inner], 1.0, atol=1e-14)
    assert np.allclose(g[inner], f(X, Y)[inner], atol=1e-13)


# ---- advection ----------------------------------------------------------------------------------
def _staggered(fu, fv):
    """vx and vy arrays sampling u(x, y) on the vx lattice and v(x, y) on the vy lattice."""
    Xu, Yu = _nodes(MK.VX_POINTS)
    Xv, Yv = _nodes(MK.VY_POINTS)
    return fu(Xu, Yu), fv(Xv, Yv)


# per-step amplification of z = (x - xc) + i (y - yc) in the rotation dz/dt = i w z (theta = w h)
_AMPLIFICATION = {
    MK.EULER: lambda t: 1 + 1j * t,
    MK.HEUN: lambda t: 1 + 1j * t - t * t / 2,
    MK.RK4: lambda t: 1 + 1j * t - t * t / 2 - 1j * t ** 3 / 6 + t ** 4 / 24,
    MK.TAYLOR: lambda t: 1 + 1j * t - t * t / 2,   # J v0 = A^2 z, H = 0 for a linear field
}


@pytest.mark.parametrize("scheme", [MK.EULER, MK.HEUN, MK.RK4, MK.TAYLOR])
def test_rigid_rotation_has_the_closed_form_amplification_of_each_scheme(scheme):
    """u = -w (y - yc), v = w (x - xc) is linear, so the bilinear interpolation is exact and each
    step multiplies z by the scheme's stability polynomial at i w h."""
    w, xc, yc = 0.8, 0.75, 0.5
    vx, vy = _staggered(lambda x, y: -w * (y - yc), lambda x, y: w * (x - xc))
    rng = np.random.default_rng(5)
    r = rng.uniform(0.05, 0.2, 40); a = rng.uniform(0, 2 * np.pi, 40)
    xm, ym = xc + r * np.cos(a), yc + r * np.sin(a)
    h, k = 0.05, 7
    x, y = MK.advect(NX, NY, LX, LY, vx, vy, xm, ym, h * k, scheme, substeps=k)
    z = ((xm - xc) + 1j * (ym - yc)) * _AMPLIFICATION[scheme](w * h) ** k
    assert np.allclose(x - xc, z.real, rtol=0, atol=1e-13) and np.allclose(y - yc, z.imag, rtol=0, atol=1e-13)


def _bilinear_flow():
    """u = d x y, v = e (both reproduced exactly by bilinear interpolation): y(t) = y0 + e t,
    x(t) = x0 exp(d (y0 t + e t^2 / 2))."""
    d, e = 0.9, 0.4
    vx, vy = _staggered(lambda x, y: d * x * y, lambda x, y: e + 0 * x)
    exact = lambda x0, y0, t: (x0 * np.exp(d * (y0 * t + 0.5 * e * t * t)), y0 + e * t)
    return d, e, vx, vy, exact


@pytest.mark.parametrize("scheme,order", [(MK.EULER, 1), (MK.HEUN, 2), (MK.RK4, 4), (MK.TAYLOR, 2)])
def test_convergence_order_against_the_exact_trajectory(scheme, order):
    d, e, vx, vy, exact = _bilinear_flow()
    xm, ym = np.array([0.4, 0.7, 0.55]), np.array([0.2, 0.3, 0.25])
    T = 0.5
    xe, ye = exact(xm, ym, T)
    errs = []
    for k in (8, 16, 32):
        x, y = MK.advect(NX, NY, LX, LY, vx, vy, xm, ym, T, scheme, substeps=k)
        errs.append(np.max(np.hypot(x - xe, y - ye)))
    for a, b in zip(errs, errs[1:]):
        assert 2 ** order * 0.8 < a / b < 2 ** order * 1.25, (errs, order)


def test_taylor_update_carries_the_curvature_term():
    """One Taylor step misses only the (J J v0) h^3/6 part of the exact third-order term: the
    H : v0 v0 part (here 2 d u e, from the interpolant's d2/dxdy) must be present."""
    d, e, vx, vy, exact = _bilinear_flow()
    x0, y0 = np.array([0.6]), np.array([0.3])
    u = d * x0 * y0
    jjv = d * y0 * (d * y0 * u + d * x0 * e)          # (J J v0)_x with J = [[d y, d x], [0, 0]]
    for h in (1e-2, 5e-3):
        x, _ = MK.advect(NX, NY, LX, LY, vx, vy, x0, y0, h, MK.TAYLOR)
        xe, _ = exact(x0, y0, h)
        lim = (x - xe) / h ** 3
        assert abs(lim[0] + jjv[0] / 6) < 0.05 * abs(jjv[0] / 6) + 2e-3
    # dropping the curvature term would change that limit by 2 d u e / 6
    assert 2 * d * u[0] * e / 6 > 0.3 * abs(jjv[0] / 6)


@pytest.mark.parametrize("scheme", [MK.EULER, MK.HEUN, MK.RK4, MK.TAYLOR])
def test_uniform_translation_and_wall_clamp(scheme):
    U, V = 0.3, -0.2
    vx, vy = _staggered(lambda x, y: U + 0 * x, lambda x, y: V + 0 * x)
    xm, ym = np.array([0.2, 1.4, 0.7]), np.array([0.5, 0.9, 0.05])
    x, y = MK.advect(NX, NY, LX, LY, vx, vy, xm, ym, 0.5, scheme, substeps=2)
    assert np.allclose(x, np.clip(xm + 0.5 * U, 0, LX), atol=1e-15)
    assert np.allclose(y, np.clip(ym + 0.5 * V, 0, LY), atol=1e-15)
    assert x[1] == LX and y[2] == 0.0


def test_cfl_step():
    vx = np.zeros((NY + 2, NX + 2)); vy = np.zeros((NY + 2, NX + 2))
    assert MK.max_dt(NX, NY, LX, LY, vx, vy, 0.5) == np.inf
    vx[3, 4] = -2.0; vy[5, 6] = 0.5
    dx, dy = LX / NX, LY / NY
    assert MK.max_dt(NX, NY, LX, LY, vx, vy, 0.5) == pytest.approx(0.5 * min(dx / 2.0, dy / 0.5), rel=1e-15)
