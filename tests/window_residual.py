"""Residual rows of the oracle's system at a window of a large grid (test infrastructure).

A row of r = b - A x (eqs. xmom/ymom/mass after boundary elimination) involves only the unknowns
next to it, the viscosities and densities around it and, at the domain boundary, the boundary
rule. So the rows of the unknowns inside a block of cells can be had from the oracle's own
assembly of a small grid that covers the block plus a margin: sides of the window that lie on the
domain boundary keep the domain's boundary condition; rows within the margin of an artificial
side are discarded. This gives the oracle's residual at sampled places of grids whose whole
assembly would not fit (4096 x 4096 and up).
"""
import numpy as np

from oracle import stokes as S

MARGIN = 2


def window_residual(nx, ny, Lx, Ly, bc, eta_n, eta_c, rho, gvec, vx, vy, p, rows, cols, product=False):
    """Oracle residual of the unknowns whose cells lie in rows [rows[0], rows[1]] and columns
    [cols[0], cols[1]] (1-based cell indices, inclusive) of an nx x ny grid.

    Returns (r_vx, r_vy, r_p, scale_vx, scale_vy, scale_p, (i_lo, j_lo)): padded arrays of the
    window (NaN outside the requested block), each row's magnitude |b| + |A| |x| as scale, and the
    global index of the window array's [0, 0] entry. With product=True the rows of A x are returned
    instead of b - A x."""
    if bc.kind[S.WEST] == S.PERIODIC:
        raise ValueError("windows of periodic grids are not supported")
    a = max(1, rows[0] - MARGIN)
    b = min(ny, rows[1] + MARGIN)
    c = max(1, cols[0] - MARGIN)
    d = min(nx, cols[1] + MARGIN)
    nyw, nxw = b - a + 1, d - c + 1
    dx, dy = Lx / nx, Ly / ny
    kind = list(bc.kind)
    vt = list(bc.vt)
    # artificial sides: any rule (their rows are discarded); keep free slip there
    if c > 1:
        kind[S.WEST], vt[S.WEST] = S.FREE_SLIP, 0.0
    if d < nx:
        kind[S.EAST], vt[S.EAST] = S.FREE_SLIP, 0.0
    if a > 1:
        kind[S.NORTH], vt[S.NORTH] = S.FREE_SLIP, 0.0
    if b < ny:
        kind[S.SOUTH], vt[S.SOUTH] = S.FREE_SLIP, 0.0
    gw = S.Grid(nxw, nyw, nxw * dx, nyw * dy, S.BC(tuple(kind), tuple(vt)))
    sl = (slice(a - 1, b + 2), slice(c - 1, d + 2))
    sysm = S.assemble(gw, eta_n[sl], eta_c[sl], rho[sl], gvec)
    x = S.fields_to_vector(gw, vx[sl], vy[sl], p[sl])
    r = sysm.A @ x if product else sysm.b - sysm.A @ x
    mag = np.abs(sysm.b) + abs(sysm.A) @ np.abs(x)
    rx, ry, rp = S.vector_to_fields(gw, r, fill_ghosts=False)
    mx, my, mp = S.vector_to_fields(gw, mag, fill_ghosts=False)
    # keep the requested block only (window-local cell indices)
    keep = np.zeros((nyw + 2, nxw + 2), dtype=bool)
    keep[rows[0] - a + 1:rows[1] - a + 2, cols[0] - c + 1:cols[1] - c + 2] = True
    out = []
    for arr, idx in ((rx, gw.idx_vx), (ry, gw.idx_vy), (rp, gw.idx_p)):
        o = np.where(keep & (idx >= 0), arr, np.nan)
        out.append(o)
    for arr in (mx, my, mp):
        out.append(arr)
    out.append((a - 1, c - 1))
    return tuple(out)


def global_positions(win, lo):
    """(i, j) global indices of the non-NaN entries of a window array returned above."""
    ii, jj = np.nonzero(~np.isnan(win))
    return ii + lo[0], jj + lo[1], ii, jj
