"""Marker <-> grid interpolation on the GPU against the oracle (Sec. "Marker-to-grid
interpolation", "Grid-to-marker interpolation"): random markers including ones on walls and
beyond the lattice, both lattices, a grid with empty cells, determinism, and the full-size
case of 16 markers per cell on 1024 x 1024."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import markers as MK
from gpu_util import dev, host

import paper_2603_14040_b300 as P


def _markers(n, Lx, Ly, seed, edge=True):
    rng = np.random.default_rng(seed)
    xm = rng.uniform(0, Lx, n); ym = rng.uniform(0, Ly, n)
    if edge:   # some on the walls and corners, a few just beyond
        xm[:8] = [0.0, Lx, 0.0, Lx, -1e-3, Lx + 1e-3, 0.5 * Lx, 0.5 * Lx]
        ym[:8] = [0.0, 0.0, Ly, Ly, 0.5 * Ly, 0.5 * Ly, -1e-3, Ly + 1e-3]
    return xm, ym, rng.standard_normal(n)


@pytest.mark.parametrize("kind", [P.LATTICE_NODES, P.LATTICE_CELLS])
@pytest.mark.parametrize("nx,ny,Lx,Ly,per_cell", [(16, 12, 1.0, 0.75, 10), (64, 48, 2.0, 1.0, 8), (40, 30, 1.0, 1.0, 0.3)])
def test_markers_to_grid_and_back_match_oracle(kind, nx, ny, Lx, Ly, per_cell):
    n = int(per_cell * nx * ny)
    xm, ym, ph = _markers(n, Lx, Ly, nx + ny)
    g0 = np.random.default_rng(3).standard_normal((ny + 2, nx + 2))       # kept where no marker reaches
    ref, wref = MK.markers_to_grid(nx, ny, Lx, Ly, kind, xm, ym, ph, g0)
    mk = P.Markers(nx, ny, Lx, Ly, max_markers=n)
    grid, w = dev(g0), torch.zeros((ny + 2, nx + 2), dtype=torch.float64, device="cuda")
    mk.to_grid(kind, dev(xm), dev(ym), dev(ph), grid, w)
    g, wg = host(grid), host(w)
    # the marker's cell fraction (x - x0)/dx is formed by a multiply with 1/dx on the GPU, a division
    # in the oracle: a few ulp of the cell count apart (about 1e-14), hence 1e-12 below
    assert np.allclose(wg, wref, rtol=1e-12, atol=1e-12)
    assert np.allclose(g, ref, rtol=1e-12, atol=1e-12)
    if per_cell < 1:
        assert np.any(wref == 0) and np.array_equal(g[wref == 0], g0[wref == 0])
    # grid -> markers on an arbitrary field
    field = np.random.default_rng(4).standard_normal((ny + 2, nx + 2))
    out = torch.zeros(n, dtype=torch.float64, device="cuda")
    mk.to_markers(kind, dev(xm), dev(ym), dev(field), out)
    torch.cuda.synchronize()
    assert np.allclose(host(out), MK.grid_to_markers(nx, ny, Lx, Ly, kind, xm, ym, field), rtol=1e-12, atol=1e-12)
    mk.close()


def test_markers_to_grid_is_deterministic_and_full_size():
    nx = ny = 1024
    n = 16 * nx * ny
    xm, ym, ph = _markers(n, 1.0, 1.0, 7, edge=False)
    mk = P.Markers(nx, ny, 1.0, 1.0, max_markers=n)
    outs = []
    for _ in range(2):
        grid = torch.zeros((ny + 2, nx + 2), dtype=torch.float64, device="cuda")
        mk.to_grid(P.LATTICE_NODES, dev(xm), dev(ym), dev(ph), grid)
        outs.append(host(grid))
    assert np.array_equal(outs[0], outs[1])
    ref, _ = MK.markers_to_grid(nx, ny, 1.0, 1.0, MK.BASIC_NODES, xm, ym, ph, np.zeros((ny + 2, nx + 2)))
    assert np.allclose(outs[0], ref, rtol=1e-11, atol=1e-12)
    mk.close()


def test_nonfinite_position_is_rejected():
    mk = P.Markers(8, 8, max_markers=4)
    xm = dev(np.array([0.1, np.nan, 0.3, 0.4])); ym = dev(np.array([0.1, 0.2, 0.3, 0.4]))
    grid = torch.zeros((10, 10), dtype=torch.float64, device="cuda")
    with pytest.raises(P.PyroError):
        mk.to_grid(P.LATTICE_NODES, xm, ym, dev(np.ones(4)), grid)
    mk.close()
