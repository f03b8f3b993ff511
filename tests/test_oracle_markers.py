"""Pins of the marker <-> grid interpolation oracle (Sec. "Marker-to-grid interpolation",
"Grid-to-marker interpolation"): partition of unity, exactness of the bilinear gather on bilinear
fields, and the equal-weight average of symmetric markers."""
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


@pytest.mark.parametrize("kind", [MK.BASIC_NODES, MK.CELL_CENTRES])
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
