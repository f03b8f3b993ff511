"""The window residual (test infrastructure for full-size parity) equals the rows of the oracle's
whole-grid residual, for every boundary kind and window placement (corner, edges, interior)."""
import numpy as np
import pytest

from oracle import stokes as S
from synth import random_vectors, random_field_log10, sample_lattice_to_fields
from window_residual import window_residual, global_positions

KINDS = {
    "free": ((S.FREE_SLIP,) * 4, (0.0,) * 4),
    "noslip": ((S.NO_SLIP,) * 4, (0.0,) * 4),
    "lid": ((S.FREE_SLIP, S.NO_SLIP, S.VELOCITY, S.NO_SLIP), (0.0, 0.0, 0.7, 0.0)),
}


@pytest.mark.parametrize("bc", list(KINDS))
def test_window_rows_equal_whole_grid_rows(bc):
    nx, ny, Lx, Ly = 40, 28, 1.3, 0.9
    kind, vt = KINDS[bc]
    g = S.Grid(nx, ny, Lx, Ly, S.BC(kind, vt))
    l10 = random_field_log10(nx, ny, 3, corr_len=0.2)
    f = sample_lattice_to_fields(10.0 ** (2 * l10), 1.0 + 0.05 * l10, nx, ny, Lx, Ly)
    gvec = (0.3, 1.0)
    vx, vy, p = random_vectors(nx, ny, 9)
    x = S.fields_to_vector(g, vx, vy, p)
    sysm = S.assemble(g, f.eta_n, f.eta_c, f.rho, gvec)
    xf = S.vector_to_fields(g, x, fill_ghosts=False)
    for product in (False, True):
        r = sysm.A @ x if product else sysm.b - sysm.A @ x
        Rx, Ry, Rp = S.vector_to_fields(g, r, fill_ghosts=False)
        checked = 0
        for rows, cols in [((1, 6), (1, 7)), ((23, 28), (34, 40)), ((1, 5), (15, 22)), ((10, 17), (1, 4)),
                           ((11, 19), (12, 25)), ((24, 28), (1, 40))]:
            wx, wy, wp, *_, lo = window_residual(nx, ny, Lx, Ly, g.bc, f.eta_n, f.eta_c, f.rho, gvec, *xf, rows,
                                                 cols, product=product)
            for win, ref in ((wx, Rx), (wy, Ry), (wp, Rp)):
                gi, gj, li, lj = global_positions(win, lo)
                assert len(gi) > 0
                assert np.abs(win[li, lj] - ref[gi, gj]).max() <= 1e-12 * np.abs(ref).max()
                checked += len(gi)
        assert checked > 500
