"""Plain FP64 CPU oracle of the marker steps of the marker-in-cell loop: marker <-> grid
interpolation (Sec. "Marker-to-grid interpolation" and "Grid-to-marker interpolation") and the
advection of the markers in the Stokes velocity (Sec. "Advection of Lagrangian Markers": forward
Euler, Heun, classical RK4 and the locally polynomial (Taylor) update). Test infrastructure only.

Lattices: basic nodes (x_j = j dx, y_i = i dy, i in [0, ny], j in [0, nx]) or cell centres
(x_j = (j - 1/2) dx, y_i = (i - 1/2) dy, i in [1, ny], j in [1, nx]), and the two staggered
velocity lattices, vx points (x_j = j dx, y_i = (i - 1/2) dy, i in [1, ny], j in [0, nx]) and vy
points (x_j = (j - 1/2) dx, y_i = i dy, i in [0, ny], j in [1, nx]), all stored in the padded
(ny+2) x (nx+2) layout. Row index i goes with y, column j with x.

Readings (listed with the design notes):
  * the reference node of a marker is the lattice node at the top-left corner of the lattice cell
    that contains it, r_x = x_m - x_j, r_y = y_m - y_i; the node to its right (j+1) takes the
    weight (r_x/dx)(1 - r_y/dy), the one below (i+1) takes (1 - r_x/dx)(r_y/dy) (the printed
    equations attach r_x to the first index; the weights follow the geometry);
  * markers outside the lattice's span are clamped into its outermost lattice cell (a marker on
    the far wall belongs to the last cell);
  * a node that no marker reaches (sum of weights 0) keeps the value it had on input;
  * the velocity at a marker is each component interpolated bilinearly from its own staggered
    lattice (the "trilinear" interpolation of the text, in 2D), with the same clamping;
  * the Taylor update takes J and H from that bilinear interpolant at the marker: its first
    derivatives, and its only non-zero second derivative d2/dxdy (zero in a direction in which the
    marker lies beyond the lattice, where the clamped interpolant is constant);
  * after each (sub)step the position is clamped into the box [0, Lx] x [0, Ly].
"""
import numpy as np

BASIC_NODES, CELL_CENTRES, VX_POINTS, VY_POINTS = 0, 1, 2, 3
EULER, HEUN, RK4, TAYLOR = 0, 1, 2, 3


def lattice(nx, ny, Lx, Ly, kind):
    """(x0, y0, i_lo, i_hi, j_lo, j_hi): origin of the lattice and its index range (inclusive)."""
    dx, dy = Lx / nx, Ly / ny
    if kind == BASIC_NODES:
        return 0.0, 0.0, 0, ny, 0, nx
    if kind == VX_POINTS:
        return 0.0, -0.5 * dy, 1, ny, 0, nx
    if kind == VY_POINTS:
        return -0.5 * dx, 0.0, 0, ny, 1, nx
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


def _interp_with_derivatives(nx, ny, Lx, Ly, kind, xm, ym, grid):
    """Bilinear interpolant of a lattice field at the markers: value, d/dx, d/dy, d2/dxdy (the
    derivatives of the clamped interpolant: zero across a direction in which the marker lies
    beyond the lattice)."""
    dx, dy = Lx / nx, Ly / ny
    x0, y0, ilo, ihi, jlo, jhi = lattice(nx, ny, Lx, Ly, kind)
    u = (xm - x0) / dx
    v = (ym - y0) / dy
    i, j, fx, fy = _cell_and_fractions(nx, ny, Lx, Ly, kind, xm, ym)
    a00, a01 = grid[i, j], grid[i, j + 1]
    a10, a11 = grid[i + 1, j], grid[i + 1, j + 1]
    val = (1 - fx) * (1 - fy) * a00 + fx * (1 - fy) * a01 + (1 - fx) * fy * a10 + fx * fy * a11
    inx = (u >= jlo) & (u <= jhi)
    iny = (v >= ilo) & (v <= ihi)
    ddx = np.where(inx, ((a01 - a00) * (1 - fy) + (a11 - a10) * fy) / dx, 0.0)
    ddy = np.where(iny, ((a10 - a00) * (1 - fx) + (a11 - a01) * fx) / dy, 0.0)
    dxy = np.where(inx & iny, (a11 - a10 - a01 + a00) / (dx * dy), 0.0)
    return val, ddx, ddy, dxy


def velocity_at(nx, ny, Lx, Ly, vx, vy, xm, ym):
    """Velocity at the markers: vx from the vx lattice, vy from the vy lattice (bilinear)."""
    return (grid_to_markers(nx, ny, Lx, Ly, VX_POINTS, xm, ym, vx),
            grid_to_markers(nx, ny, Lx, Ly, VY_POINTS, xm, ym, vy))


def advect(nx, ny, Lx, Ly, vx, vy, xm, ym, dt, scheme, substeps=1):
    """Marker positions after a time dt in the (frozen) grid velocity, in `substeps` equal steps of
    the chosen scheme (Sec. "Advection of Lagrangian Markers"):
      EULER  eq. euler_advection: x + h v(x);
      HEUN   eq. heun_method: x* = x + h v(x), x + h/2 (v(x) + v(x*));
      RK4    eq. rk4_method: the classical four-stage Runge-Kutta step;
      TAYLOR eq. lpi_update: x + h v0 + h^2/2 J v0 + h^3/6 (H : v0 v0), J and H of the bilinear
             velocity interpolant at the marker.
    Each step's result is clamped into [0, Lx] x [0, Ly]."""
    x = np.array(xm, dtype=np.float64)
    y = np.array(ym, dtype=np.float64)
    h = dt / substeps
    vel = lambda a, b: velocity_at(nx, ny, Lx, Ly, vx, vy, a, b)
    for _ in range(substeps):
        if scheme == EULER:
            u, v = vel(x, y)
            xn, yn = x + h * u, y + h * v
        elif scheme == HEUN:
            u1, v1 = vel(x, y)
            u2, v2 = vel(x + h * u1, y + h * v1)
            xn, yn = x + 0.5 * h * (u1 + u2), y + 0.5 * h * (v1 + v2)
        elif scheme == RK4:
            u1, v1 = vel(x, y)
            u2, v2 = vel(x + 0.5 * h * u1, y + 0.5 * h * v1)
            u3, v3 = vel(x + 0.5 * h * u2, y + 0.5 * h * v2)
            u4, v4 = vel(x + h * u3, y + h * v3)
            xn = x + h / 6.0 * (u1 + 2.0 * u2 + 2.0 * u3 + u4)
            yn = y + h / 6.0 * (v1 + 2.0 * v2 + 2.0 * v3 + v4)
        elif scheme == TAYLOR:
            u, ux, uy, uxy = _interp_with_derivatives(nx, ny, Lx, Ly, VX_POINTS, x, y, vx)
            v, vx_, vy_, vxy = _interp_with_derivatives(nx, ny, Lx, Ly, VY_POINTS, x, y, vy)
            xn = x + h * u + 0.5 * h * h * (ux * u + uy * v) + h ** 3 / 6.0 * (2.0 * uxy * u * v)
            yn = y + h * v + 0.5 * h * h * (vx_ * u + vy_ * v) + h ** 3 / 6.0 * (2.0 * vxy * u * v)
        else:
            raise ValueError("unknown scheme")
        x = np.clip(xn, 0.0, Lx)
        y = np.clip(yn, 0.0, Ly)
    return x, y


def max_dt(nx, ny, Lx, Ly, vx, vy, cfl):
    """Largest step that moves no marker more than cfl cells per step (the CFL-like limit of Sec.
    "Advection of Lagrangian Markers"): cfl * min(dx / max|vx|, dy / max|vy|) over the arrays
    (+inf when the velocity is zero everywhere)."""
    dx, dy = Lx / nx, Ly / ny
    mx, my = float(np.max(np.abs(vx))), float(np.max(np.abs(vy)))
    tx = dx / mx if mx > 0 else np.inf
    ty = dy / my if my > 0 else np.inf
    return cfl * min(tx, ty)
