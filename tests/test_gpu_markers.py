"""Marker steps on the GPU against the oracle. Interpolation (Sec. "Marker-to-grid interpolation",
"Grid-to-marker interpolation"): random markers including ones on walls and beyond the lattice,
all four lattices, a grid with empty cells, determinism, and the full-size case of 16 markers per
cell on 1024 x 1024. Advection (Sec. "Advection of Lagrangian Markers"): every scheme with
substeps in random and solved velocity fields, the CFL step, and invalid arguments."""
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


@pytest.mark.parametrize("kind", [P.LATTICE_NODES, P.LATTICE_CELLS, P.LATTICE_VX, P.LATTICE_VY])
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


# ---- advection ----------------------------------------------------------------------------------
def _inner_markers(n, Lx, Ly, seed):
    """Random markers strictly inside the box (no marker on a lattice line, where the Taylor
    update's derivative has two one-sided values), plus a few within 1e-3 of the walls."""
    rng = np.random.default_rng(seed)
    xm = rng.uniform(0, Lx, n); ym = rng.uniform(0, Ly, n)
    xm[:4] = [1e-3 * Lx, Lx * (1 - 1e-3), 0.3 * Lx + 1e-7, 0.61 * Lx]
    ym[:4] = [0.41 * Ly, 0.27 * Ly, 1e-3 * Ly, Ly * (1 - 1e-3)]
    return xm, ym


@pytest.mark.parametrize("scheme", [P.ADVECT_EULER, P.ADVECT_HEUN, P.ADVECT_RK4, P.ADVECT_TAYLOR])
@pytest.mark.parametrize("nx,ny,Lx,Ly,substeps", [(16, 12, 1.0, 0.75, 1), (40, 30, 1.0, 1.0, 3), (64, 48, 2.0, 1.0, 2)])
def test_advection_matches_oracle(scheme, nx, ny, Lx, Ly, substeps):
    rng = np.random.default_rng(nx + 7 * substeps)
    vx = rng.standard_normal((ny + 2, nx + 2)); vy = rng.standard_normal((ny + 2, nx + 2))
    n = 20 * nx * ny
    xm, ym = _inner_markers(n, Lx, Ly, nx + ny)
    mk = P.Markers(nx, ny, Lx, Ly, max_markers=1)
    dt = mk.max_dt(dev(vx), dev(vy), cfl=2.0)
    assert dt == pytest.approx(MK.max_dt(nx, ny, Lx, Ly, vx, vy, 2.0), rel=1e-15)
    X, Y = dev(xm), dev(ym)
    mk.advect(X, Y, dev(vx), dev(vy), dt, scheme=scheme, substeps=substeps)
    torch.cuda.synchronize()
    rx, ry = MK.advect(nx, ny, Lx, Ly, vx, vy, xm, ym, dt, scheme, substeps)
    # cell fractions by a multiply with 1/dx on the GPU, a division in the oracle: a few ulp apart
    assert np.allclose(host(X), rx, rtol=0, atol=1e-12 * Lx)
    assert np.allclose(host(Y), ry, rtol=0, atol=1e-12 * Ly)
    assert host(X).min() >= 0 and host(X).max() <= Lx and host(Y).min() >= 0 and host(Y).max() <= Ly
    mk.close()


@pytest.mark.parametrize("scheme", [P.ADVECT_RK4, P.ADVECT_TAYLOR])
def test_advection_in_the_solved_sinker_velocity_matches_oracle(scheme):
    """End to end: solve the sinker with the library, advect markers in its velocity on the GPU and
    with the oracle from the same velocity arrays."""
    from synth import sinker
    n = 48
    f = sinker(n, n)
    h = P.Stokes(n, n, prec=P.PREC_FP64)
    outs = [torch.zeros((n + 2, n + 2), dtype=torch.float64, device="cuda") for _ in range(3)]
    h.solve(dev(f.eta_n), dev(f.eta_c), dev(f.rho), (0.0, 1.0), 1e-10, *outs)
    vx, vy = host(outs[0]), host(outs[1])
    xm, ym = _inner_markers(4000, 1.0, 1.0, 11)
    mk = P.Markers(n, n, 1.0, 1.0)
    dt = mk.max_dt(outs[0], outs[1], cfl=0.5)
    X, Y = dev(xm), dev(ym)
    mk.advect(X, Y, outs[0], outs[1], 8 * dt, scheme=scheme, substeps=8)
    torch.cuda.synchronize()
    rx, ry = MK.advect(n, n, 1.0, 1.0, vx, vy, xm, ym, 8 * dt, scheme, 8)
    assert np.allclose(host(X), rx, rtol=0, atol=1e-12) and np.allclose(host(Y), ry, rtol=0, atol=1e-12)
    moved = np.hypot(host(X) - xm, host(Y) - ym)
    assert moved.max() > 1.0 / n          # the markers did move by more than a cell
    mk.close(); h.close()


def test_advection_invalid_arguments_and_empty_input():
    mk = P.Markers(8, 8)
    v = torch.zeros((10, 10), dtype=torch.float64, device="cuda")
    x = torch.zeros(3, dtype=torch.float64, device="cuda")
    for kw in (dict(scheme=7), dict(substeps=0)):
        with pytest.raises(P.PyroError):
            mk.advect(x, x.clone(), v, v, 0.1, **kw)
    with pytest.raises(P.PyroError):
        mk.advect(x, x.clone(), v, v, float("nan"))
    with pytest.raises(P.PyroError):
        mk.advect(np.zeros(3), np.zeros(3), v, v, 0.1)            # host positions
    e = torch.zeros(0, dtype=torch.float64, device="cuda")
    assert mk.advect(e, e.clone(), v, v, 0.1) == P.PYRO_OK
    assert mk.max_dt(v, v, 0.5) == float("inf")
    bad = v.clone(); bad[3, 3] = float("nan")
    with pytest.raises(P.PyroError):
        mk.max_dt(bad, v, 0.5)
    mk.close()
