"""Plain FP64 CPU oracle of the marker <-> grid interpolation of the marker-in-cell loop (Sec.
"Marker-to-grid interpolation" and "Grid-to-marker interpolation"). Test infrastructure only.

Lattices: basic nodes (x_j = j dx, y_i = i dy, i in [0, ny], j in [0, nx]) or cell centres
(x_j = (j - 1/2) dx, y_i = (i - 1/2) dy, i in [1, ny], j in [1, nx]), stored in the padded
(ny+2) x (nx+2) layout. Row index i goes with y, column j with x.

Readings (listed with the design notes):
  * the reference node of a marker is the lattice node at the top-left corner of the lattice cell
    that contains it, r_x = x_m - x_j, r_y = y_m - y_i; the node to its right (j+1) takes the
    weight (r_x/dx)(1 - r_y/dy), the one below (i+1) takes (1 - r_x/dx)(r_y/dy) (the printed
    equations attach r_x to the first index; the weights follow the geometry);
  * markers outside the lattice's span are clamped into its outermost lattice cell (a marker on
    the far wall belongs to the last cell);
  * a node that no marker reaches (sum of weights 0) keeps the value it had on input.
"""
import numpy as np

BASIC_NODES, CELL_CENTRES = 0, 1


def lattice(nx, ny, Lx, Ly, kind):
    """(x0, y0, i_lo, i_hi, j_lo, j_hi): origin of the lattice and its index range (inclusive)."""
    dx, dy = Lx / nx, Ly / ny
    if kind == BASIC_NODES:
        return 0.0, 0.0, 0, ny, 0, nx
    return -0.5 * dx, -0.5 * dy, 1, ny, 1, nx


def _cell_and_fractions(nx, ny, Lx, Ly, kind, xm, ym):
    dx, dy = Lx / nx, Ly / ny
    x0, y0, ilo, ihi, jlo, jhi = lattice(nx, ny, Lx, Ly, kind)
    # position in lattice units relative to node (0, 0) of the padded indexing
    u = (xm - x0) / dx
    v = (ym - y0) / dy
    j = np.clip(np.floor(u).astype(np.int64), jlo, jhi - 1)
    i = np.clip(np.floor(v).astype(np.int64), ilo, ihi - 1)
    fx = np.clip(u - j, 0.0, 1.0)          # r_x / dx
    fy = np.clip(v - i, 0.0, 1.0)          # r_y / dy
    return i, j, fx, fy


def markers_to_grid(nx, ny, Lx, Ly, kind, xm, ym, phim, grid_in):
    """Weighted average of the marker values at each lattice node (eqs. of Sec. "Marker-to-grid
    interpolation"): phi = sum_m w_m phi_m / sum_m w_m with bilinear weights. Returns (phi, wsum)."""
    i, j, fx, fy = _cell_and_fractions(nx, ny, Lx, Ly, kind, xm, ym)
    num = np.zeros((ny + 2, nx + 2))
    den = np.zeros((ny + 2, nx + 2))
    for di, dj, w in ((0, 0, (1 - fx) * (1 - fy)), (0, 1, fx * (1 - fy)), (1, 0, (1 - fx) * fy), (1, 1, fx * fy)):
        np.add.at(num, (i + di, j + dj), w * phim)
        np.add.at(den, (i + di, j + dj), w)
    out = grid_in.copy()
    m = den > 0
    out[m] = num[m] / den[m]
    return out, den


def grid_to_markers(nx, ny, Lx, Ly, kind, xm, ym, grid):
    """Bilinear interpolation of a lattice field to the markers (Sec. "Grid-to-marker
    interpolation"): phi_m = sum over the four corners of w phi."""
    i, j, fx, fy = _cell_and_fractions(nx, ny, Lx, Ly, kind, xm, ym)
    return ((1 - fx) * (1 - fy) * grid[i, j] + fx * (1 - fy) * grid[i, j + 1] + (1 - fx) * fy * grid[i + 1, j]
            + fx * fy * grid[i + 1, j + 1])
