"""Plain FP64 CPU oracle of the discrete staggered-grid Stokes system.

TEST INFRASTRUCTURE ONLY: nothing on the product path imports this module. Only the tests,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` use it.

What it computes is the plain definition of what the GPU solver converges to: the exact solution
of the assembled sparse saddle-point system [[L, G], [D, 0]] [v; p] = [f; 0] (Eq. stokes_saddle),
with the zero-mean pressure gauge (Eq. pressure_normalization) imposed as a bordering row. It does
not replay any iteration.

Discretisation (Sec. "Stress-Conservative Finite Differences", eqs. xmom/ymom/mass, and the
x-momentum point listing of Sec. "Backend / kernels"):
  x-momentum at vx(i,j):
     (sxx(i,j+1) - sxx(i,j))/dx + (sxy(i,j) - sxy(i-1,j))/dy - (p(i,j+1) - p(i,j))/dx = f_x(i,j)
  y-momentum at vy(i,j):
     (syy(i+1,j) - syy(i,j))/dy + (sxy(i,j) - sxy(i,j-1))/dx - (p(i+1,j) - p(i,j))/dy = f_y(i,j)
  continuity at p(i,j):
     (vx(i,j) - vx(i,j-1))/dx + (vy(i,j) - vy(i-1,j))/dy = 0
  with sxx(i,j) = 2 eta_c(i,j) (vx(i,j)-vx(i,j-1))/dx,  syy(i,j) = 2 eta_c(i,j) (vy(i,j)-vy(i-1,j))/dy,
       sxy(i,j) = eta_n(i,j) ((vx(i+1,j)-vx(i,j))/dy + (vy(i,j+1)-vy(i,j))/dx).

Readings of points the paper leaves open (all listed with the design notes):
  * gravity: momentum is div(sigma') - grad p + rho g = 0 in the grid frame with y (and the row
    index) pointing down, so f = -rho g; g = (0, 1) pulls dense material toward the last row.
  * rho lives on basic nodes; a velocity node takes the mean of its two adjacent basic nodes.
  * nx, ny count cells; arrays are (ny+2) x (nx+2) (the paper's (n_y+1) x (n_x+1) in node counts).
  * boundary ghosts are eliminated: a tangential ghost equals s * (adjacent interior) + c with
    s=+1, c=0 (free slip), s=-1, c=0 (no slip, the paper's mirror rule) or s=-1, c=2U
    (prescribed tangential velocity U); normal velocities on walls are zero. Periodic x wraps
    indices (node column nx and cell column 0 alias column 0 and nx respectively).

Index ranges of the unknowns (the x-momentum loop bounds of the paper's listing):
  vx: i in [1, ny], j in [1, nx-1] (periodic: j in [0, nx-1]);
  vy: i in [1, ny-1], j in [1, nx];
  p : i in [1, ny], j in [1, nx].
"""
from dataclasses import dataclass, field
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

FREE_SLIP, NO_SLIP, PERIODIC, VELOCITY = 0, 1, 2, 3
WEST, EAST, NORTH, SOUTH = 0, 1, 2, 3


@dataclass
class BC:
    """Boundary condition per side (W, E, N = top row i=0, S = bottom), Sec. "Boundary Conditions"."""
    kind: tuple = (FREE_SLIP, FREE_SLIP, FREE_SLIP, FREE_SLIP)
    vt: tuple = (0.0, 0.0, 0.0, 0.0)

    def ghost_rule(self, side):
        """(s, c) such that ghost = s * interior + c for the tangential component on `side`."""
        k = self.kind[side]
        if k == FREE_SLIP:
            return 1.0, 0.0
        if k == NO_SLIP:
            return -1.0, 0.0
        if k == VELOCITY:
            return -1.0, 2.0 * self.vt[side]
        raise ValueError("no ghost rule for periodic side")


class Grid:
    """Index bookkeeping of one staggered grid (cells nx x ny, box Lx x Ly)."""

    def __init__(self, nx, ny, Lx=1.0, Ly=1.0, bc=None):
        self.nx, self.ny = int(nx), int(ny)
        self.Lx, self.Ly = float(Lx), float(Ly)
        self.dx, self.dy = self.Lx / self.nx, self.Ly / self.ny
        self.bc = bc if bc is not None else BC()
        k = self.bc.kind
        if (k[WEST] == PERIODIC) != (k[EAST] == PERIODIC):
            raise ValueError("periodic must be set on both W and E")
        if k[NORTH] == PERIODIC or k[SOUTH] == PERIODIC:
            raise ValueError("periodic in y is not supported")
        self.periodic = k[WEST] == PERIODIC
        nx, ny = self.nx, self.ny
        shp = (ny + 2, nx + 2)
        self.idx_vx = -np.ones(shp, dtype=np.int64)
        self.idx_vy = -np.ones(shp, dtype=np.int64)
        self.idx_p = -np.ones(shp, dtype=np.int64)
        jr = np.arange(0, nx) if self.periodic else np.arange(1, nx)
        ii, jj = np.meshgrid(np.arange(1, ny + 1), jr, indexing="ij")
        self.vx_i, self.vx_j = ii.ravel(), jj.ravel()
        ii, jj = np.meshgrid(np.arange(1, ny), np.arange(1, nx + 1), indexing="ij")
        self.vy_i, self.vy_j = ii.ravel(), jj.ravel()
        ii, jj = np.meshgrid(np.arange(1, ny + 1), np.arange(1, nx + 1), indexing="ij")
        self.p_i, self.p_j = ii.ravel(), jj.ravel()
        self.n_vx, self.n_vy, self.n_p = len(self.vx_i), len(self.vy_i), len(self.p_i)
        self.idx_vx[self.vx_i, self.vx_j] = np.arange(self.n_vx)
        self.idx_vy[self.vy_i, self.vy_j] = self.n_vx + np.arange(self.n_vy)
        self.idx_p[self.p_i, self.p_j] = self.n_vx + self.n_vy + np.arange(self.n_p)
        self.n_v = self.n_vx + self.n_vy
        self.n = self.n_v + self.n_p

    # ---- periodic-aware accessors of material fields -------------------------------------------
    def eta_c_at(self, eta_c, i, j):
        if self.periodic:
            j = np.where(j == 0, self.nx, np.where(j == self.nx + 1, 1, j))
        return eta_c[i, j]

    def node_at(self, a, i, j):
        if self.periodic:
            j = np.mod(j, self.nx)
        return a[i, j]

    # ---- resolving a reference to a field value into (column, coefficient) or a constant --------
    def _resolve_vx(self, i, j, coef):
        i, j, coef = i.copy(), j.copy(), coef.copy()
        const = np.zeros_like(coef)
        keep = np.ones(len(i), dtype=bool)
        if self.periodic:
            j = np.mod(j, self.nx)
        else:
            keep &= (j != 0) & (j != self.nx)          # normal velocity on W/E walls is zero
        for row, side, inner in ((0, NORTH, 1), (self.ny + 1, SOUTH, self.ny)):
            m = i == row
            if m.any():
                s, c = self.bc.ghost_rule(side)
                const[m] += c * coef[m]
                coef[m] *= s
                i[m] = inner
        col = self.idx_vx[i, j]
        assert np.all(col[keep] >= 0), "vx reference outside unknowns"
        return col, coef, const, keep

    def _resolve_vy(self, i, j, coef):
        i, j, coef = i.copy(), j.copy(), coef.copy()
        const = np.zeros_like(coef)
        keep = (i != 0) & (i != self.ny)                # normal velocity on N/S walls is zero
        if self.periodic:
            j = np.where(j == 0, self.nx, np.where(j == self.nx + 1, 1, j))
        else:
            for colg, side, inner in ((0, WEST, 1), (self.nx + 1, EAST, self.nx)):
                m = j == colg
                if m.any():
                    s, c = self.bc.ghost_rule(side)
                    const[m] += c * coef[m]
                    coef[m] *= s
                    j[m] = inner
        col = self.idx_vy[i, j]
        assert np.all(col[keep] >= 0), "vy reference outside unknowns"
        return col, coef, const, keep

    def _resolve_p(self, i, j, coef):
        if self.periodic:
            j = np.where(j == 0, self.nx, np.where(j == self.nx + 1, 1, j))
        col = self.idx_p[i, j]
        assert np.all(col >= 0), "p reference outside unknowns"
        return col, coef, np.zeros_like(coef), np.ones(len(i), dtype=bool)


@dataclass
class System:
    grid: Grid
    A: sp.csr_matrix          # full saddle-point matrix, unknowns ordered [vx, vy, p]
    b: np.ndarray             # RHS with body force and the eliminated boundary constants
    f_body: np.ndarray = field(default=None)


def _add(rows, cols, vals, rhs, grid, fld, row, i, j, coef):
    res = {"vx": grid._resolve_vx, "vy": grid._resolve_vy, "p": grid._resolve_p}[fld]
    col, c, const, keep = res(np.asarray(i), np.asarray(j), np.asarray(coef, dtype=np.float64))
    rows.append(row[keep]); cols.append(col[keep]); vals.append(c[keep])
    np.add.at(rhs, row[keep], -const[keep])


def assemble(grid, eta_n, eta_c, rho=None, g=(0.0, 0.0), velocity_only=False):
    """Assemble A and b of the discrete Stokes system (or only the velocity block L and f)."""
    dx, dy = grid.dx, grid.dy
    n = grid.n_v if velocity_only else grid.n
    rows, cols, vals = [], [], []
    rhs = np.zeros(n)
    A_ = lambda fld, row, i, j, c: _add(rows, cols, vals, rhs, grid, fld, row, i, j, c)

    # x-momentum rows
    i, j = grid.vx_i, grid.vx_j
    row = grid.idx_vx[i, j]
    eA = grid.eta_c_at(eta_c, i, j)          # sxx at the cell west of vx(i,j)
    eB = grid.eta_c_at(eta_c, i, j + 1)      # sxx at the cell east of vx(i,j)
    e1 = grid.node_at(eta_n, i - 1, j)       # sxy at the node above
    e2 = grid.node_at(eta_n, i, j)           # sxy at the node below
    # (sxx(i,j+1) - sxx(i,j)) / dx
    A_("vx", row, i, j + 1, 2 * eB / dx**2); A_("vx", row, i, j, -2 * eB / dx**2)
    A_("vx", row, i, j, -2 * eA / dx**2);    A_("vx", row, i, j - 1, 2 * eA / dx**2)
    # (sxy(i,j) - sxy(i-1,j)) / dy
    A_("vx", row, i + 1, j, e2 / dy**2);     A_("vx", row, i, j, -e2 / dy**2)
    A_("vy", row, i, j + 1, e2 / (dx * dy)); A_("vy", row, i, j, -e2 / (dx * dy))
    A_("vx", row, i, j, -e1 / dy**2);        A_("vx", row, i - 1, j, e1 / dy**2)
    A_("vy", row, i - 1, j + 1, -e1 / (dx * dy)); A_("vy", row, i - 1, j, e1 / (dx * dy))
    if not velocity_only:
        # -(p(i,j+1) - p(i,j)) / dx
        A_("p", row, i, j + 1, -np.ones(len(i)) / dx); A_("p", row, i, j, np.ones(len(i)) / dx)
    if rho is not None:
        rbar = 0.5 * (grid.node_at(rho, i - 1, j) + grid.node_at(rho, i, j))
        np.add.at(rhs, row, -g[0] * rbar)

    # y-momentum rows
    i, j = grid.vy_i, grid.vy_j
    row = grid.idx_vy[i, j]
    eA = grid.eta_c_at(eta_c, i, j)          # syy at the cell above vy(i,j)
    eB = grid.eta_c_at(eta_c, i + 1, j)      # syy at the cell below
    e1 = grid.node_at(eta_n, i, j - 1)       # sxy at the node to the west
    e2 = grid.node_at(eta_n, i, j)           # sxy at the node to the east
    # (syy(i+1,j) - syy(i,j)) / dy
    A_("vy", row, i + 1, j, 2 * eB / dy**2); A_("vy", row, i, j, -2 * eB / dy**2)
    A_("vy", row, i, j, -2 * eA / dy**2);    A_("vy", row, i - 1, j, 2 * eA / dy**2)
    # (sxy(i,j) - sxy(i,j-1)) / dx
    A_("vx", row, i + 1, j, e2 / (dx * dy)); A_("vx", row, i, j, -e2 / (dx * dy))
    A_("vy", row, i, j + 1, e2 / dx**2);     A_("vy", row, i, j, -e2 / dx**2)
    A_("vx", row, i + 1, j - 1, -e1 / (dx * dy)); A_("vx", row, i, j - 1, e1 / (dx * dy))
    A_("vy", row, i, j, -e1 / dx**2);        A_("vy", row, i, j - 1, e1 / dx**2)
    if not velocity_only:
        # -(p(i+1,j) - p(i,j)) / dy
        A_("p", row, i + 1, j, -np.ones(len(i)) / dy); A_("p", row, i, j, np.ones(len(i)) / dy)
    if rho is not None:
        rbar = 0.5 * (grid.node_at(rho, i, j - 1) + grid.node_at(rho, i, j))
        np.add.at(rhs, row, -g[1] * rbar)

    if not velocity_only:
        # continuity rows: (vx(i,j) - vx(i,j-1))/dx + (vy(i,j) - vy(i-1,j))/dy
        i, j = grid.p_i, grid.p_j
        row = grid.idx_p[i, j]
        one = np.ones(len(i))
        A_("vx", row, i, j, one / dx); A_("vx", row, i, j - 1, -one / dx)
        A_("vy", row, i, j, one / dy); A_("vy", row, i - 1, j, -one / dy)

    A = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(n, n))
    A.sum_duplicates()
    return System(grid, A, rhs)


# ---- packing between padded fields and unknown vectors ---------------------------------------
def fields_to_vector(grid, vx, vy, p=None):
    parts = [vx[grid.vx_i, grid.vx_j], vy[grid.vy_i, grid.vy_j]]
    if p is not None:
        parts.append(p[grid.p_i, grid.p_j])
    return np.concatenate(parts)


def vector_to_fields(grid, x, fill_ghosts=True):
    """Unknown vector -> padded (vx, vy, p); ghosts/walls filled by the boundary rule."""
    nx, ny = grid.nx, grid.ny
    vx = np.zeros((ny + 2, nx + 2)); vy = np.zeros((ny + 2, nx + 2)); p = np.zeros((ny + 2, nx + 2))
    vx[grid.vx_i, grid.vx_j] = x[:grid.n_vx]
    vy[grid.vy_i, grid.vy_j] = x[grid.n_vx:grid.n_v]
    if len(x) > grid.n_v:
        p[grid.p_i, grid.p_j] = x[grid.n_v:]
    if fill_ghosts:
        fill_boundary(grid, vx, vy, p)
    return vx, vy, p


def fill_boundary(grid, vx, vy, p=None, homogeneous=False):
    nx, ny = grid.nx, grid.ny
    if grid.periodic:
        vx[1:ny + 1, nx] = vx[1:ny + 1, 0]
        vy[:, 0] = vy[:, nx]; vy[:, nx + 1] = vy[:, 1]
        if p is not None:
            p[:, 0] = p[:, nx]; p[:, nx + 1] = p[:, 1]
    else:
        vx[:, 0] = 0.0; vx[:, nx] = 0.0
        for colg, side, inner in ((0, WEST, 1), (nx + 1, EAST, nx)):
            s, c = grid.bc.ghost_rule(side)
            vy[1:ny, colg] = s * vy[1:ny, inner] + (0.0 if homogeneous else c)
    vy[0, :] = 0.0; vy[ny, :] = 0.0
    for rowg, side, inner in ((0, NORTH, 1), (ny + 1, SOUTH, ny)):
        s, c = grid.bc.ghost_rule(side)
        vx[rowg, :] = s * vx[inner, :] + (0.0 if homogeneous else c)
    if not grid.periodic:
        vx[:, 0] = 0.0; vx[:, nx] = 0.0
    vx[:, nx + 1] = 0.0
    vy[ny + 1, :] = 0.0


# ---- matrix-vector product and residual norms ----------------------------------------------
def apply_operator(grid, eta_n, eta_c, vx, vy, p):
    """y = A x with homogeneous boundary rules (no boundary constants), returned as padded fields
    holding values only at unknown locations."""
    sysm = assemble(grid, eta_n, eta_c)
    y = sysm.A @ fields_to_vector(grid, vx, vy, p)
    return vector_to_fields(grid, y, fill_ghosts=False)


def pressure_weights(grid, eta_c):
    """Diagonal Schur surrogate eta / (2/dx^2 + 2/dy^2) (Sec. "Residual Norms", pressure part)."""
    return grid.eta_c_at(eta_c, grid.p_i, grid.p_j) / (2.0 / grid.dx**2 + 2.0 / grid.dy**2)


def energy_residual(sysm, eta_c, x):
    """Relative energy residual of Sec. "Global Relative Energy Residual":
    sqrt((|r_v|^2_{diag(-L)^-1} + |r_p|^2_{S~^-1}) / |f|^2_{diag(-L)^-1}); diag(-L) is taken
    after boundary elimination. Also returns the plain l2 relative residual."""
    g = sysm.grid
    r = sysm.b - sysm.A @ x
    dL = -sysm.A.diagonal()[:g.n_v]
    wp = pressure_weights(g, eta_c)
    num = np.sum(r[:g.n_v] ** 2 / dL) + np.sum(r[g.n_v:] ** 2 * wp)
    den = np.sum(sysm.b[:g.n_v] ** 2 / dL)
    l2 = np.linalg.norm(r) / max(np.linalg.norm(sysm.b), 1e-300)
    return float(np.sqrt(num / den)) if den > 0 else float(np.sqrt(num)), float(l2)


# ---- direct solve ----------------------------------------------------------------------------
def bordered(sysm):
    """[[A, c], [c^T, 0]] with c the cell volumes of the pressure unknowns (zero-mean gauge)."""
    g = sysm.grid
    c = np.zeros(g.n)
    c[g.n_v:] = g.dx * g.dy
    K = sp.bmat([[sysm.A, sp.csr_matrix(c[:, None])], [sp.csr_matrix(c[None, :]), None]], format="csc")
    return K


def solve_direct(sysm, refine=2, permc_spec="COLAMD"):
    """Exact solution of A x = b with zero-mean pressure: sparse LU of the bordered matrix plus
    `refine` steps of FP64 iterative refinement on the bordered residual."""
    K = bordered(sysm)
    rhs = np.concatenate([sysm.b, [0.0]])
    lu = spla.splu(K, permc_spec=permc_spec)
    y = lu.solve(rhs)
    for _ in range(refine):
        y = y + lu.solve(rhs - K @ y)
    return y[:-1]


def remove_pressure_mean(grid, x):
    x = x.copy()
    x[grid.n_v:] -= x[grid.n_v:].mean()
    return x


@dataclass
class Solution:
    vx: np.ndarray
    vy: np.ndarray
    p: np.ndarray
    x: np.ndarray
    rel_energy: float
    rel_l2: float


def solve_fields(nx, ny, Lx, Ly, eta_n, eta_c, rho, g, bc=None):
    grid = Grid(nx, ny, Lx, Ly, bc)
    sysm = assemble(grid, eta_n, eta_c, rho, g)
    x = solve_direct(sysm)
    e, l2 = energy_residual(sysm, eta_c, x)
    vx, vy, p = vector_to_fields(grid, x)
    return Solution(vx, vy, p, x, e, l2)


# ---- adjoint by linearity of the assembly in eta -----------------------------------------------
def blend_viscosity(eta_n, eta_c, theta, nx, ny):
    """Viscosity-contrast continuation (Sec. "Viscosity Rescaling and Initial Guess"):
    eta_comp = (1 - theta) eta_min + theta eta, eta_min the smallest viscosity of the real nodes
    (i in [0, ny], j in [0, nx]) and cells (i, j in [1, n]). Padding entries are left as given."""
    emin = min(eta_n[:ny + 1, :nx + 1].min(), eta_c[1:ny + 1, 1:nx + 1].min())
    en = eta_n.copy(); ec = eta_c.copy()
    en[:ny + 1, :nx + 1] = (1 - theta) * emin + theta * eta_n[:ny + 1, :nx + 1]
    ec[1:ny + 1, 1:nx + 1] = (1 - theta) * emin + theta * eta_c[1:ny + 1, 1:nx + 1]
    return en, ec


def lithostatic_pressure(grid, rho, g):
    """Lithostatic initial pressure p = int_0^y rho g_y dy' (Sec. "Viscosity Rescaling and Initial
    Guess"), in this discretisation: going down a column, consecutive cell pressures differ by
    dy g_y rho_vy with rho_vy the density of the vy node between them (the mean of its two basic
    nodes, as in the y-momentum right-hand side); zero volume-weighted mean. Returns the padded
    (ny+2) x (nx+2) pressure array (cells only)."""
    nx, ny, dy = grid.nx, grid.ny, grid.dy
    p = np.zeros((ny + 2, nx + 2))
    for j in range(1, nx + 1):
        for i in range(1, ny):
            rho_vy = 0.5 * (rho[i, j - 1] + rho[i, j])
            p[i + 1, j] = p[i, j] + dy * g[1] * rho_vy
    p[1:ny + 1, 1:nx + 1] -= p[1:ny + 1, 1:nx + 1].mean()
    return p


def eta_gradient_by_linearity(grid, eta_n, eta_c, x, lam, cells=None, nodes=None):
    """dJ/d eta_k = -lam^T A_k x with A_k = A(e_k) - A(0), both from this module's assembler.

    Exact because the assembly is linear in eta (every viscous coefficient is eta times a mesh
    factor). `cells`/`nodes` optionally restrict the evaluation to lists of (i, j) indices.
    Returns (g_n, g_c) padded arrays (NaN where not evaluated)."""
    nx, ny = grid.nx, grid.ny
    zero = np.zeros((ny + 2, nx + 2))
    A0 = assemble(grid, zero, zero).A
    g_n = np.full((ny + 2, nx + 2), np.nan)
    g_c = np.full((ny + 2, nx + 2), np.nan)
    if cells is None:
        cells = [(i, j) for i in range(1, ny + 1) for j in range(1, nx + 1)]
    if nodes is None:
        nodes = [(i, j) for i in range(0, ny + 1) for j in range(0, nx + 1)]
    for (i, j) in cells:
        e = zero.copy(); e[i, j] = 1.0
        Ak = assemble(grid, zero, e).A - A0
        g_c[i, j] = -lam @ (Ak @ x)
    for (i, j) in nodes:
        if grid.periodic and j == nx:
            continue
        e = zero.copy(); e[i, j] = 1.0
        Ak = assemble(grid, e, zero).A - A0
        g_n[i, j] = -lam @ (Ak @ x)
    return g_n, g_c


def rho_gradient_by_linearity(grid, g, lam):
    """dJ/d rho_k = lam^T (b(e_k) - b(0)): the body force is linear in rho."""
    nx, ny = grid.nx, grid.ny
    zero = np.zeros((ny + 2, nx + 2))
    ones = np.ones((ny + 2, nx + 2))
    b0 = assemble(grid, ones, ones, zero, g).b
    out = np.zeros((ny + 2, nx + 2))
    for i in range(ny + 1):
        for j in range(nx + 1):
            e = zero.copy(); e[i, j] = 1.0
            out[i, j] = lam @ (assemble(grid, ones, ones, e, g).b - b0)
    return out
