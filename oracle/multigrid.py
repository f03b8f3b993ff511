"""Plain FP64 CPU oracle of the geometric-multigrid pieces (test infrastructure only).

Nothing on the product path imports this module. It states, as plainly as possible, what each
step of the V-cycle preconditioner computes, so that the GPU kernels can be compared with it one
step at a time:

  * coarse grids by re-discretisation with each material field transferred on its own
    (Sec. "Geometric vs Algebraic Multigrid");
  * restriction = normalised bilinear-weighted accumulation (Sec. "Restriction and Prolongation
    Operators", the normalised-sum equation), built here by brute force from the staggered
    positions; prolongation = bilinear interpolation from the four surrounding coarse points;
  * damped red-black Gauss-Seidel (Sec. "Smoothers", eq. sor_update) on the velocity block, or
    damped Jacobi (eq. damped_jacobi), or the RAS-type temporally blocked Jacobi smoother
    (Algorithm ras_temporal), or the "Mixed" configuration of the robustness study (Sec.
    "Numerical Stability and Solver Robustness": Jacobi on the finest level, RAS-type Jacobi on
    every coarser level);
  * the V-cycle of eq. multigrid_levels with a direct coarsest solve;
  * one Uzawa sweep as the preconditioner M^-1 (Sec. "Uzawa Iteration as a Fixed Point Method").

Readings (the paper is silent or inconsistent; each is listed with the design notes):
  * only fine locations that are unknowns (velocity) or real nodes / cells (viscosity) enter a
    restriction sum, and the normalisation compensates for the truncated support at walls;
  * coarse ghost values used by the prolongation follow the homogeneous boundary rule;
  * viscosity is coarsened with the same normalised bilinear weights, arithmetically or on
    log(eta) (geometric mean);
  * RBGS colour order: vx-red, vx-black, vy-red, vy-black with colour (i + j) mod 2;
  * RAS-type Jacobi: a tile owns the unknowns of its cells, its outer boundary is held at the
    pass-start values, ceil(nu / T_inner) passes (no rounding to an even count: the evenness in
    the paper's algorithm only returns the result to the first of two global buffers), tiles
    clipped at the domain edge, shifts from SplitMix64 of (level, pre/post, pass);
  * pressure sign of M^-1: the paper's splitting puts -(alpha eta)^-1 in the pressure block, but
    with L negative definite (as the paper states) D L^-1 G is negative semi-definite and that
    sign makes the stationary Uzawa iteration diverge. We take z_p = alpha eta_c (r_p - D z_v),
    i.e. the surrogate carries the sign of the operator it stands for; the test suite pins this by
    showing the stationary iteration converges with it and diverges with the literal sign.
"""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .stokes import Grid, assemble

ETA_ARITH, ETA_GEOM = 0, 1
MAX_COARSE = 1024
GAL_OMEGA = 0.6   # damped-Jacobi smoothing on Galerkin levels


def coarsen_grid(g, nxc=None, nyc=None):
    """The next level: halved by default, or nxc x nyc cells on the same box (general ratio)."""
    if nxc is None:
        if g.nx % 2 or g.ny % 2:
            raise ValueError("factor-2 coarsening needs even cell counts")
        nxc, nyc = g.nx // 2, g.ny // 2
    return Grid(nxc, nyc, g.Lx, g.Ly, g.bc)


def velocity_unknowns(nx, ny):
    return ny * (nx - 1) + (ny - 1) * nx


def level_sizes(nx, ny, coarsest_min, ratio=2.0, general=True):
    """Cell counts of every level. Halve while the ratio is 2, both counts are even and the short
    side stays >= coarsest_min; then, while the coarsest level is too large for the direct solve
    (more than MAX_COARSE velocity unknowns), coarsen by the ratio: n_c = ceil(n / ratio) (the
    paper's arbitrary coarsening ratio, Algorithms find_lower_index / restriction_checkerboard)."""
    sizes = [(nx, ny)]
    while True:
        nx, ny = sizes[-1]
        if ratio == 2.0 and nx % 2 == 0 and ny % 2 == 0 and min(nx, ny) // 2 >= coarsest_min:
            sizes.append((nx // 2, ny // 2))
            continue
        if general and velocity_unknowns(nx, ny) > MAX_COARSE:
            cx, cy = int(np.ceil(nx / ratio - 1e-9)), int(np.ceil(ny / ratio - 1e-9))
            if min(cx, cy) >= 2 and (cx, cy) != (nx, ny):
                sizes.append((cx, cy))
                continue
        return sizes


def n_levels(nx, ny, coarsest_min, ratio=2.0, general=True):
    return len(level_sizes(nx, ny, coarsest_min, ratio, general))


def _candidates(c, r, centred, lo, hi):
    """Fine indices whose position may lie within one coarse spacing of coarse index c (r = coarse
    spacing / fine spacing; positions c * h for nodes/faces, (c - 1/2) h for centred families)."""
    off = 0.5 if centred else 0.0
    a = np.floor((c - off - 1) * r + off).astype(np.int64) - 1
    b = np.ceil((c - off + 1) * r + off).astype(np.int64) + 1
    return np.maximum(a, lo), np.minimum(b, hi)


# ---- staggered positions --------------------------------------------------------------------
def positions(g, fld):
    if fld == "vx":
        return g.vx_j * g.dx, (g.vx_i - 0.5) * g.dy
    if fld == "vy":
        return (g.vy_j - 0.5) * g.dx, g.vy_i * g.dy
    raise ValueError(fld)


def _unknown_lookup(g, fld):
    return g.idx_vx if fld == "vx" else g.idx_vy


def restriction_matrix(fine, coarse, fld):
    """R with (R r)_K = sum_k w_Kk r_k / sum_k w_Kk, w = (1-|dx|/Hx)(1-|dy|/Hy) over fine unknowns."""
    Xc, Yc = positions(coarse, fld)
    Xf, Yf = positions(fine, fld)
    idx = _unknown_lookup(fine, fld)
    base = 0 if fld == "vx" else fine.n_vx
    # candidate fine indices: every fine unknown whose position is within one coarse spacing
    ci = coarse.vx_i if fld == "vx" else coarse.vy_i
    cj = coarse.vx_j if fld == "vx" else coarse.vy_j
    rx, ry = coarse.dx / fine.dx, coarse.dy / fine.dy
    ilo, ihi = _candidates(ci, ry, fld == "vx", 0, fine.ny + 1)    # vx rows are cell-centred
    jlo, jhi = _candidates(cj, rx, fld == "vy", 0, fine.nx + 1)    # vy columns are cell-centred
    span_i, span_j = int((ihi - ilo).max()) + 1, int((jhi - jlo).max()) + 1
    rows, cols, vals = [], [], []
    for di in range(span_i):
        for dj in range(span_j):
            fi = ilo + di
            fj = jlo + dj
            ok = (fi <= ihi) & (fj <= jhi) & (fi >= 0) & (fi < fine.ny + 2) & (fj >= 0) & (fj < fine.nx + 2)
            fi_ = np.where(ok, fi, 0); fj_ = np.where(ok, fj, 0)
            col = idx[fi_, fj_]
            ok &= col >= 0
            col = col - base
            xf = np.where(ok, Xf[np.maximum(col, 0)], 0.0)
            yf = np.where(ok, Yf[np.maximum(col, 0)], 0.0)
            wx = 1 - np.abs(xf - Xc) / coarse.dx
            wy = 1 - np.abs(yf - Yc) / coarse.dy
            ok &= (wx > 1e-9) & (wy > 1e-9)          # inside the bilinear support
            w = wx * wy
            k = np.nonzero(ok)[0]
            rows.append(k); cols.append(col[k]); vals.append(w[k])
    nC = len(Xc); nF = len(Xf)
    R = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(nC, nF))
    R.sum_duplicates()
    s = np.asarray(R.sum(axis=1)).ravel()
    return sp.diags(1.0 / s) @ R


def prolongation_matrix(fine, coarse, fld):
    """P: bilinear interpolation of a coarse correction at every fine unknown from the four
    surrounding coarse points of the same staggered family (ghosts by the homogeneous rule)."""
    Xf, Yf = positions(fine, fld)
    H, K = coarse.dx, coarse.dy
    if fld == "vx":
        fx, fy = Xf / H, Yf / K + 0.5          # coarse vx at X = J*H, Y = (I - 1/2)*K
    else:
        fx, fy = Xf / H + 0.5, Yf / K          # coarse vy at X = (J - 1/2)*H, Y = I*K
    J0 = np.floor(fx + 1e-12).astype(np.int64); I0 = np.floor(fy + 1e-12).astype(np.int64)
    tx = fx - J0; ty = fy - I0
    rows, cols, vals = [], [], []
    nF = len(Xf)
    for di, wy in ((0, 1 - ty), (1, ty)):
        for dj, wx in ((0, 1 - tx), (1, tx)):
            w = wy * wx
            I = I0 + di; J = J0 + dj
            m = w > 1e-14
            if fld == "vx":
                col, c, _, keep = coarse._resolve_vx(I[m], J[m], w[m])
            else:
                col, c, _, keep = coarse._resolve_vy(I[m], J[m], w[m])
                col = col - coarse.n_vx
            r = np.nonzero(m)[0]
            rows.append(r[keep]); cols.append(col[keep]); vals.append(c[keep])
    nC = coarse.n_vx if fld == "vx" else coarse.n_vy
    P = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(nF, nC))
    P.sum_duplicates()
    return P


def _material_restrict(fine, coarse, a, centred):
    """Normalised bilinear restriction of a material field (cells if centred, else nodes)."""
    nx, ny = coarse.nx, coarse.ny
    out = np.zeros((ny + 2, nx + 2))
    if centred:
        I, J = np.meshgrid(np.arange(1, ny + 1), np.arange(1, nx + 1), indexing="ij")
        Xc, Yc = (J - 0.5) * coarse.dx, (I - 0.5) * coarse.dy
        lo_i, hi_i, lo_j, hi_j = 1, fine.ny, 1, fine.nx
        posf = lambda i, j: ((j - 0.5) * fine.dx, (i - 0.5) * fine.dy)
    else:
        I, J = np.meshgrid(np.arange(0, ny + 1), np.arange(0, nx + 1), indexing="ij")
        Xc, Yc = J * coarse.dx, I * coarse.dy
        lo_i, hi_i, lo_j, hi_j = 0, fine.ny, 0, fine.nx
        posf = lambda i, j: (j * fine.dx, i * fine.dy)
    acc = np.zeros(I.shape); wsum = np.zeros(I.shape)
    rx, ry = coarse.dx / fine.dx, coarse.dy / fine.dy
    ilo, ihi = _candidates(I, ry, centred, lo_i, hi_i)
    jlo, jhi = _candidates(J, rx, centred, lo_j, hi_j)
    span_i, span_j = int((ihi - ilo).max()) + 1, int((jhi - jlo).max()) + 1
    for di in range(span_i):
        for dj in range(span_j):
            fi = ilo + di; fj = jlo + dj
            ok = (fi <= ihi) & (fj <= jhi) & (fi >= lo_i) & (fi <= hi_i) & (fj >= lo_j) & (fj <= hi_j)
            xf, yf = posf(fi, fj)
            wx = 1 - np.abs(xf - Xc) / coarse.dx
            wy = 1 - np.abs(yf - Yc) / coarse.dy
            ok &= (wx > 1e-9) & (wy > 1e-9)          # inside the bilinear support
            w = wx * wy
            vals = a[np.where(ok, fi, lo_i), np.where(ok, fj, lo_j)]
            acc += np.where(ok, w * vals, 0.0); wsum += np.where(ok, w, 0.0)
    out[I, J] = acc / wsum
    return out


def coarsen_eta(fine, coarse, eta_n, eta_c, mode=ETA_ARITH):
    if mode == ETA_GEOM:
        en = np.exp(_material_restrict(fine, coarse, np.log(np.where(eta_n > 0, eta_n, 1.0)), False))
        ec = np.exp(_material_restrict(fine, coarse, np.log(np.where(eta_c > 0, eta_c, 1.0)), True))
        en[coarse.ny + 1, :] = 0; en[:, coarse.nx + 1] = 0
        ec[0, :] = 0; ec[:, 0] = 0; ec[coarse.ny + 1, :] = 0; ec[:, coarse.nx + 1] = 0
        return en, ec
    return (_material_restrict(fine, coarse, eta_n, False),
            _material_restrict(fine, coarse, eta_c, True))


# ---- smoother --------------------------------------------------------------------------------
def colour_sets(g):
    """Row index sets of the four half-sweeps in order vx-red, vx-black, vy-red, vy-black."""
    vx_red = np.nonzero((g.vx_i + g.vx_j) % 2 == 0)[0]
    vx_blk = np.nonzero((g.vx_i + g.vx_j) % 2 == 1)[0]
    vy_red = g.n_vx + np.nonzero((g.vy_i + g.vy_j) % 2 == 0)[0]
    vy_blk = g.n_vx + np.nonzero((g.vy_i + g.vy_j) % 2 == 1)[0]
    return [vx_red, vx_blk, vy_red, vy_blk]


def rbgs_sweep(L, f, x, sets, omega):
    """One damped red-black Gauss-Seidel sweep: for each colour set S in order,
    x_S += omega * (f_S - (L x)_S) / diag(L)_S (points of one set do not couple)."""
    x = x.copy()
    d = L.diagonal()
    for S in sets:
        r = f[S] - L[S] @ x
        x[S] += omega * r / d[S]
    return x


def jacobi_sweep(L, f, x, omega):
    """One damped Jacobi sweep over every unknown of L x = f (eq. damped_jacobi):
    x + omega (f - L x) / diag(L), all from the old iterate."""
    return x + omega * (f - L @ x) / L.diagonal()


def splitmix64(z):
    """SplitMix64 (Steele, Lea & Flood, OOPSLA 2014), on Python integers modulo 2^64."""
    m = (1 << 64) - 1
    z = (z + 0x9E3779B97F4A7C15) & m
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & m
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & m
    return z ^ (z >> 31)


RAS_SEED = 0x5EED


def ras_shift(level, phase, t, TI, TJ):
    """Tiling shift (s_i, s_j) of pass t of the pre (phase 0) / post (phase 1) smoothing on a level:
    the random shift of Algorithm ras_temporal, drawn from SplitMix64 of a counter so that the
    smoother is the same operator at every application."""
    v = splitmix64(RAS_SEED + (((level * 2 + phase) << 16) + t))
    return (v & 0xFFFFFFFF) % TI, (v >> 32) % TJ


def ras_pass(g, L, f, x, omega, inner, TI, TJ, si, sj):
    """One pass of the RAS-type temporally blocked Jacobi smoother (Algorithm ras_temporal).
    The cells are tiled TI x TJ, tile k covering rows [k_i TI - si, (k_i + 1) TI - si) and the
    same for columns; a tile owns the unknowns of its cells (vx(i, j) and vy(i, j) belong to cell
    (i, j)); each tile runs `inner` damped Jacobi iterations on its own unknowns with every other
    unknown held at its value from the start of the pass (the tile's outer boundary is fixed), and
    the owned results make up the new iterate."""
    vi = np.concatenate([g.vx_i, g.vy_i]); vj = np.concatenate([g.vx_j, g.vy_j])
    tile = ((vi + si) // TI) * 1_000_003 + (vj + sj) // TJ
    C = L.tocoo()
    same = tile[C.row] == tile[C.col]
    Ls = sp.csr_matrix((C.data[same], (C.row[same], C.col[same])), shape=L.shape)
    Lo = sp.csr_matrix((C.data[~same], (C.row[~same], C.col[~same])), shape=L.shape)
    d = L.diagonal()
    rhs = f - Lo @ x                      # other tiles' unknowns at their pass-start values
    y = x.copy()
    for _ in range(inner):
        y = y + omega * (rhs - Ls @ y) / d
    return y


def level_smoother(smoother, level):
    """The smoother used on `level`: the hierarchy's own, except that "mixed" means damped Jacobi
    on the finest level and the RAS-type Jacobi smoother on the coarser ones."""
    if smoother == "mixed":
        return "jacobi" if level == 0 else "ras"
    return smoother


def smooth(h, level, f, x, nu, omega, phase):
    """nu smoothing steps on `level` with the level's smoother: damped RBGS sweeps (default),
    damped Jacobi sweeps, or ceil(nu / inner) RAS passes of `inner` local Jacobi iterations; a
    Galerkin level is always smoothed by damped Jacobi with GAL_OMEGA."""
    L = h.L[level]
    if h.gal[level]:
        for _ in range(nu):
            x = jacobi_sweep(L, f, x, GAL_OMEGA)
        return x
    kind = level_smoother(h.smoother, level)
    if kind == "rbgs":
        for _ in range(nu):
            x = rbgs_sweep(L, f, x, h.sets[level], omega)
        return x
    if kind == "jacobi":
        for _ in range(nu):
            x = jacobi_sweep(L, f, x, omega)
        return x
    npass = -(-nu // h.ras_inner)
    for t in range(npass):
        si, sj = ras_shift(level, phase, t, h.ras_tile, h.ras_tile)
        x = ras_pass(h.grids[level], L, f, x, omega, h.ras_inner, h.ras_tile, h.ras_tile, si, sj)
    return x


# ---- hierarchy and V-cycle ---------------------------------------------------------------------
class Hierarchy:
    def __init__(self, grid, eta_n, eta_c, coarsest_min=4, eta_mode=ETA_ARITH, n_lev=None, smoother="rbgs",
                 ras_inner=4, ras_tile=32, coarse_sweeps=40, coarsen_ratio=2.0, coarsen_general=True,
                 galerkin=False):
        self.smoother, self.ras_inner, self.ras_tile = smoother, ras_inner, ras_tile
        self.coarse_sweeps = coarse_sweeps
        sizes = level_sizes(grid.nx, grid.ny, coarsest_min, coarsen_ratio, coarsen_general)
        if n_lev is not None:
            sizes = sizes[:n_lev]
        self.grids = [grid]; self.eta = [(eta_n, eta_c)]
        for (cx, cy) in sizes[1:]:
            c = coarsen_grid(self.grids[-1], cx, cy)
            en, ec = coarsen_eta(self.grids[-1], c, *self.eta[-1], mode=eta_mode)
            self.grids.append(c); self.eta.append((en, ec))
        self.L = [assemble(g, en, ec, velocity_only=True).A.tocsr() for g, (en, ec) in zip(self.grids, self.eta)]
        self.sets = [colour_sets(g) for g in self.grids]
        self.R = []; self.P = []
        for f, c in zip(self.grids[:-1], self.grids[1:]):
            self.R.append(sp.block_diag([restriction_matrix(f, c, "vx"), restriction_matrix(f, c, "vy")]).tocsr())
            self.P.append(sp.block_diag([prolongation_matrix(f, c, "vx"), prolongation_matrix(f, c, "vy")]).tocsr())
        # Galerkin coarse operators (not in the paper): a level reached by halving from a chain of
        # halvings takes L_l = R_{l-1} L_{l-1} P_{l-1} with the cycle's own transfer operators
        self.gal = [False] * len(self.grids)
        if galerkin:
            for l in range(1, len(self.grids)):
                f, c = self.grids[l - 1], self.grids[l]
                if not (c.nx * 2 == f.nx and c.ny * 2 == f.ny and (l == 1 or self.gal[l - 1])):
                    break
                self.L[l] = (self.R[l - 1] @ self.L[l - 1] @ self.P[l - 1]).tocsr()
                self.gal[l] = True
        # the coarsest level is solved directly when it is small (<= MAX_COARSE velocity unknowns),
        # else by coarse_sweeps smoothing steps from zero (Sec. "Multigrid Cycles": a direct
        # method or a few smoothing iterations on the coarsest level)
        self.coarse_direct = self.L[-1].shape[0] <= MAX_COARSE
        self.coarse_lu = spla.splu(self.L[-1].tocsc()) if self.coarse_direct else None

    @property
    def nlev(self):
        return len(self.grids)


def vcycle(h, f, nu1=2, nu2=2, omega=1.0, level=0, kcycle=0):
    """One V-cycle for L x = f at `level` from x = 0 (eq. multigrid_levels, steps (1)-(6)).

    With kcycle > 0, on levels l < kcycle whose next level is not the coarsest, step (4) is
    replaced by the recursive Krylov cycle of Notay & Vassilevski (Numer. Linear Algebra Appl.
    15, 2008): two flexible conjugate-gradient steps on the next level's correction equation,
    each preconditioned by one cycle of that level (not part of the paper)."""
    if level == h.nlev - 1:
        if h.coarse_direct:
            return h.coarse_lu.solve(f)
        return smooth(h, level, f, np.zeros_like(f), h.coarse_sweeps, omega, 2)
    L = h.L[level]
    x = np.zeros_like(f)
    x = smooth(h, level, f, x, nu1, omega, 0)                     # (1) pre-smoothing
    r = f - L @ x                                                 # (2) residual
    fc = h.R[level] @ r                                           # (3) restriction
    if level < kcycle and level + 1 < h.nlev - 1:                 # (4) by two flexible-CG steps
        dc = kcycle_correction(h, fc, nu1, nu2, omega, level + 1, kcycle)
    else:                                                         # (4) coarse solve / recursion
        dc = vcycle(h, fc, nu1, nu2, omega, level + 1, kcycle)
    x = x + h.P[level] @ dc                                       # (5) prolongation + correction
    x = smooth(h, level, f, x, nu2, omega, 1)                     # (6) post-smoothing
    return x


def kcycle_correction(h, f, nu1, nu2, omega, level, kcycle):
    """Two flexible-CG steps for L e = f on `level` from e = 0, preconditioner = one cycle.
    L is negative definite; the step lengths are the usual CG ones written for L itself."""
    L = h.L[level]
    rc = f.copy()
    z1 = vcycle(h, rc, nu1, nu2, omega, level, kcycle)
    d1 = z1
    q1 = L @ d1
    a1 = (rc @ d1) / (d1 @ q1) if (d1 @ q1) != 0 else 0.0
    e = a1 * d1
    rc = rc - a1 * q1
    z2 = vcycle(h, rc, nu1, nu2, omega, level, kcycle)
    beta = (z2 @ q1) / (d1 @ q1) if (d1 @ q1) != 0 else 0.0
    d2 = z2 - beta * d1                      # L-conjugate to d1 (flexible CG)
    q2 = L @ d2
    a2 = (rc @ d2) / (d2 @ q2) if (d2 @ q2) != 0 else 0.0
    return e + a2 * d2


def divergence(grid, zv):
    """D z_v at every pressure unknown (continuity rows of the assembled system, velocity part)."""
    from .stokes import vector_to_fields
    vx, vy, _ = vector_to_fields(grid, np.concatenate([zv, np.zeros(grid.n_p)]), fill_ghosts=True)
    i, j = grid.p_i, grid.p_j
    jm = j - 1
    if grid.periodic:
        jm = np.where(jm == 0, grid.nx, jm)
        vx = vx.copy(); vx[:, grid.nx] = vx[:, 0]
    return (vx[i, j] - vx[i, jm]) / grid.dx + (vy[i, j] - vy[i - 1, j]) / grid.dy


def velocity_fcg(h, f, steps, nu1=2, nu2=2, omega=1.0, kcycle=0):
    """`steps` steps of flexible conjugate gradients on L x = f from x = 0, each preconditioned by
    one V-cycle, with the one-term flexible recurrence (each direction L-conjugate to the previous
    one; Notay, SIAM J. Sci. Comput. 22 (2000)). Not part of the paper, whose Uzawa sweep applies a
    single V-cycle to the velocity block."""
    L = h.L[0]
    x = np.zeros_like(f)
    r = f.copy()
    d = q = None
    for _ in range(steps):
        z = vcycle(h, r, nu1, nu2, omega, kcycle=kcycle)
        w = L @ z
        if d is not None:
            beta = (z @ q) / (d @ q)
            z = z - beta * d
            w = w - beta * q
        alpha = (r @ z) / (z @ w)
        x = x + alpha * z
        r = r - alpha * w
        d, q = z, w
    return x


def uzawa_precond(h, r, eta_c, alpha=0.6, nu1=2, nu2=2, omega=1.0, literal_sign=False, kcycle=0, schur=None,
                  inner_cg=0):
    """z = M^-1 r for one Uzawa sweep: z_v = V-cycle(L, r_v) (or `inner_cg` flexible-CG steps with that
    cycle as preconditioner), z_p = alpha S~^-1 (r_p - D z_v), then
    the mean of z_p is removed (Eq. pressure_normalization). S~^-1 is eta_c (the paper's diagonal
    viscosity surrogate) unless `schur` (a WeightedBFBt) is given. `literal_sign` flips to the
    paper's printed sign alpha eta_c (D z_v - r_p) (used only to demonstrate the reading)."""
    g = h.grids[0]
    if inner_cg > 0:
        zv = velocity_fcg(h, r[:g.n_v], inner_cg, nu1, nu2, omega, kcycle=kcycle)
    else:
        zv = vcycle(h, r[:g.n_v], nu1, nu2, omega, kcycle=kcycle)
    dz = divergence(g, zv)
    if schur is not None:
        zp = alpha * schur.apply(r[g.n_v:] - dz)
    else:
        e = g.eta_c_at(eta_c, g.p_i, g.p_j)
        zp = alpha * e * ((dz - r[g.n_v:]) if literal_sign else (r[g.n_v:] - dz))
    zp -= zp.mean()
    return np.concatenate([zv, zp])


# ---- weighted BFBt Schur-complement surrogate (not in the paper) ------------------------------
# The paper's pressure block uses the diagonal viscosity surrogate eta_c. Where the viscosity jumps
# by many orders of magnitude over short distances (a stiff lid over a weak mantle with weak and
# strong inclusions) that surrogate misses whole families of pressure modes and the outer Krylov
# method stalls. The weighted BFBt approximation of the Schur complement S = D (-L)^-1 G (Elman,
# SIAM J. Sci. Comput. 20 (1999) 1299-1316; the square-root-diagonal weighting of Rudi, Stadler and
# Ghattas, SIAM J. Sci. Comput. 39 (2017) S272-S297) is
#     S~^-1 = K^-1 (D W^-1 (-L) W^-1 G) K^-1,   K = D W^-1 G,   W = diag(-L)^(1/2),
# with both Poisson-type solves K^-1 replaced by one V-cycle of a smoothed-aggregation multigrid
# (PressureAMG below), so the surrogate is a fixed linear operator.
def aggregation_matrix(nx, ny):
    """P0: cell (i, j) of an nx x ny cell grid (compact row-major) -> aggregate (i // 2, j // 2) of the
    ceil(ny / 2) x ceil(nx / 2) coarse grid (2 x 2 aggregates, 1-wide ones at odd edges)."""
    nxc, nyc = (nx + 1) // 2, (ny + 1) // 2
    k = np.arange(nx * ny)
    i, j = np.divmod(k, nx)
    return sp.csr_matrix((np.ones(nx * ny), (k, (i // 2) * nxc + j // 2)), shape=(nx * ny, nxc * nyc))


def near_part(K, nx):
    """The part of K that couples cells at most one apart in both directions (a 3 x 3 box), with
    every dropped entry added to its row's diagonal, so row sums (and the constant null space) are
    unchanged."""
    C = K.tocoo()
    ri, rj = np.divmod(C.row, nx)
    ci, cj = np.divmod(C.col, nx)
    near = (np.abs(ri - ci) <= 1) & (np.abs(rj - cj) <= 1)
    lump = np.bincount(C.row[~near], weights=C.data[~near], minlength=K.shape[0])
    Kn = sp.csr_matrix((C.data[near], (C.row[near], C.col[near])), shape=K.shape)
    return (Kn + sp.diags(lump.astype(np.float64))).tocsr()


class PressureAMG:
    """Smoothed-aggregation multigrid for a symmetric cell-centred operator K with the constant null
    space (here K = D W^-1 G with the walls' zero-flux condition), on structured 2 x 2 aggregates.

    Level l -> l + 1: P = (I - omega_p diag(K)^-1 K_near) P0 with P0 the aggregation matrix and K_near
    the 3 x 3-box part of K (dropped couplings lumped on the diagonal), R = P^T, K_{l+1} = P^T K P
    (Galerkin). Smoothing the tentative prolongator with only the near part keeps every coarse
    operator within a 5 x 5 box stencil. Coarsening stops when a level has <= max_coarse cells; the
    coarsest level is solved exactly with the zero-mean gauge. The cycle: nu damped Jacobi sweeps
    x += omega_s (f - K x) / diag(K), residual, restriction, recursion from zero, prolongation,
    nu damped Jacobi sweeps."""

    def __init__(self, K, nx, ny, omega_p=2.0 / 3.0, omega_s=0.8, nu=2, max_coarse=256):
        self.omega_s, self.nu = omega_s, nu
        self.K, self.P, self.shape = [K.tocsr()], [], [(nx, ny)]
        while nx * ny > max_coarse:
            P0 = aggregation_matrix(nx, ny)
            Kl = self.K[-1]
            Kn = near_part(Kl, nx)
            P = (P0 - omega_p * (sp.diags(1.0 / Kl.diagonal()) @ (Kn @ P0))).tocsr()
            self.P.append(P)
            self.K.append((P.T @ Kl @ P).tocsr())
            nx, ny = (nx + 1) // 2, (ny + 1) // 2
            self.shape.append((nx, ny))
        Kc = self.K[-1]
        one = np.ones(Kc.shape[0])
        self.coarse_lu = spla.splu(sp.bmat([[Kc, sp.csr_matrix(one[:, None])],
                                            [sp.csr_matrix(one[None, :]), None]], format="csc"))

    @property
    def nlev(self):
        return len(self.K)

    def vcycle(self, f, level=0):
        if level == self.nlev - 1:
            return self.coarse_lu.solve(np.concatenate([f - f.mean(), [0.0]]))[:-1]
        K = self.K[level]
        d = K.diagonal()
        x = np.zeros_like(f)
        for _ in range(self.nu):
            x = x + self.omega_s * (f - K @ x) / d
        ec = self.vcycle(self.P[level].T @ (f - K @ x), level + 1)
        x = x + self.P[level] @ ec
        for _ in range(self.nu):
            x = x + self.omega_s * (f - K @ x) / d
        return x


class WeightedBFBt:
    """S~^-1 y = K^-1 (D W^-1 (-L) W^-1 G) K^-1 y on the pressure unknowns of the finest grid, with
    W = diag(-L)^(1/2) and each K^-1 one PressureAMG V-cycle (exact=True: sparse LU instead, used by
    the tests to separate the surrogate from its multigrid)."""

    def __init__(self, sysm, weight_exp=0.5, exact=False, **amg):
        g = sysm.grid
        A = sysm.A.tocsr()
        nv = g.n_v
        self.L = A[:nv, :nv].tocsr()
        self.G = A[:nv, nv:].tocsr()
        self.D = A[nv:, :nv].tocsr()
        self.W = (-self.L.diagonal()) ** weight_exp
        self.Kmat = (self.D @ sp.diags(1.0 / self.W) @ self.G).tocsr()
        if exact:
            one = np.ones(g.n_p)
            lu = spla.splu(sp.bmat([[self.Kmat, sp.csr_matrix(one[:, None])],
                                    [sp.csr_matrix(one[None, :]), None]], format="csc"))
            self.Kinv = lambda y: lu.solve(np.concatenate([y - y.mean(), [0.0]]))[:-1]
        else:
            self.amg = PressureAMG(self.Kmat, g.nx, g.ny, **amg)
            self.Kinv = self.amg.vcycle

    def apply(self, y):
        t1 = self.Kinv(y)
        t2 = self.D @ ((-(self.L @ ((self.G @ t1) / self.W))) / self.W)
        return self.Kinv(t2)
