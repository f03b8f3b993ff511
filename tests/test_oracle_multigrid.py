"""Pins of the oracle's multigrid pieces (CPU only)."""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from oracle import stokes as S
from oracle import multigrid as M
from synth import sinker


def rand_eta(nx, ny, seed, lo=-1, hi=1):
    rng = np.random.default_rng(seed)
    return 10.0 ** rng.uniform(lo, hi, (ny + 2, nx + 2)), 10.0 ** rng.uniform(lo, hi, (ny + 2, nx + 2))


@pytest.mark.parametrize("fld", ["vx", "vy"])
def test_restriction_preserves_constants_and_is_scaled_transpose(fld):
    fine, coarse = S.Grid(16, 12), S.Grid(8, 6)
    R = M.restriction_matrix(fine, coarse, fld)
    P = M.prolongation_matrix(fine, coarse, fld)
    assert np.allclose(R @ np.ones(R.shape[1]), 1.0, atol=1e-15)
    # interior: weights [1,2,1]/4 (node direction) x [1,3,3,1]/8 (cell direction) = P^T / 4
    Xc, Yc = M.positions(coarse, fld)
    inner = np.nonzero((Xc > 2 * coarse.dx) & (Xc < coarse.Lx - 2 * coarse.dx) &
                       (Yc > 2 * coarse.dy) & (Yc < coarse.Ly - 2 * coarse.dy))[0]
    assert len(inner) > 4
    Rd, Pd = R.toarray(), P.toarray()
    assert np.allclose(Rd[inner], Pd.T[inner] / 4.0, atol=1e-15)
    row = Rd[inner[0]]
    assert sorted(np.round(row[row > 0] * 32).astype(int).tolist()) == sorted([1, 3, 3, 1, 2, 6, 6, 2, 1, 3, 3, 1])


@pytest.mark.parametrize("fld", ["vx", "vy"])
def test_prolongation_exact_on_bilinear(fld):
    fine, coarse = S.Grid(16, 12, 2.0, 1.5), S.Grid(8, 6, 2.0, 1.5)
    P = M.prolongation_matrix(fine, coarse, fld)
    Xc, Yc = M.positions(coarse, fld)
    Xf, Yf = M.positions(fine, fld)
    fn = lambda x, y: 0.3 + 1.7 * x - 0.9 * y + 0.4 * x * y
    pf = P @ fn(Xc, Yc)
    # points whose four coarse neighbours are all unknowns
    ok = (Xf > coarse.dx) & (Xf < coarse.Lx - coarse.dx) & (Yf > coarse.dy) & (Yf < coarse.Ly - coarse.dy)
    assert ok.sum() > 10
    assert np.allclose(pf[ok], fn(Xf, Yf)[ok], atol=1e-13)
    # each row's weights sum to one away from walls (constants are reproduced)
    assert np.allclose((P @ np.ones(P.shape[1]))[ok], 1.0)


def test_prolongation_boundary_rule():
    """At the first fine row under a free-slip (no-slip) wall the mirrored coarse ghost gives
    weight 3/4 + 1/4 (3/4 - 1/4) on the first coarse row."""
    for kind, expect in ((S.FREE_SLIP, 1.0), (S.NO_SLIP, 0.5)):
        bc = S.BC(kind=(kind,) * 4)
        fine, coarse = S.Grid(8, 8, bc=bc), S.Grid(4, 4, bc=bc)
        P = M.prolongation_matrix(fine, coarse, "vx").toarray()
        r = fine.idx_vx[1, 2]
        c = coarse.idx_vx[1, 1]
        assert P[r, c] == pytest.approx(expect)


def test_eta_coarsening():
    fine, coarse = S.Grid(16, 8, 2.0, 1.0), S.Grid(8, 4, 2.0, 1.0)
    c = np.full((10, 18), 3.5)
    en, ec = M.coarsen_eta(fine, coarse, c, c)
    assert np.allclose(en[:5, :9], 3.5) and np.allclose(ec[1:5, 1:9], 3.5)
    en_g, ec_g = M.coarsen_eta(fine, coarse, c, c, M.ETA_GEOM)
    assert np.allclose(en_g[:5, :9], 3.5) and np.allclose(ec_g[1:5, 1:9], 3.5)
    # geometric = exp(arithmetic of log)
    a, b = rand_eta(16, 8, 7)
    ga = M.coarsen_eta(fine, coarse, a, b, M.ETA_GEOM)
    la = M.coarsen_eta(fine, coarse, np.log(a), np.log(b))
    assert np.allclose(ga[0][:5, :9], np.exp(la[0][:5, :9]))
    assert np.allclose(ga[1][1:5, 1:9], np.exp(la[1][1:5, 1:9]))
    # interior node: [1,2,1]/4 x [1,2,1]/4 weights
    I, J = 2, 3
    w = np.array([1, 2, 1]) / 4
    ex = sum(w[di] * w[dj] * a[2 * I - 1 + di, 2 * J - 1 + dj] for di in range(3) for dj in range(3))
    assert la[0] is not None and M.coarsen_eta(fine, coarse, a, b)[0][I, J] == pytest.approx(ex)


@pytest.mark.parametrize("omega", [1.0, 0.7])
def test_rbgs_is_textbook_sor_in_colour_order(omega):
    """One red-black sweep = one SOR sweep (D + w L_low) x' = w f - (w U + (w - 1) D) x in the
    permuted order vx-red, vx-black, vy-red, vy-black."""
    g = S.Grid(10, 8, bc=S.BC(kind=(S.NO_SLIP, S.FREE_SLIP, S.FREE_SLIP, S.NO_SLIP)))
    en, ec = rand_eta(10, 8, 9)
    L = S.assemble(g, en, ec, velocity_only=True).A.tocsr()
    rng = np.random.default_rng(3)
    f, x0 = rng.standard_normal(g.n_v), rng.standard_normal(g.n_v)
    sets = M.colour_sets(g)
    x1 = M.rbgs_sweep(L, f, x0, sets, omega)
    perm = np.concatenate(sets)
    Lp = L[perm][:, perm]
    D = sp.diags(Lp.diagonal())
    Llow, U = sp.tril(Lp, -1), sp.triu(Lp, 1)
    rhs = omega * f[perm] - (omega * U + (omega - 1) * D) @ x0[perm]
    xp = spla.spsolve_triangular((D + omega * Llow).tocsr(), rhs, lower=True)
    x_text = np.empty_like(xp); x_text[perm] = xp
    assert np.allclose(x1, x_text, rtol=1e-12, atol=1e-12)


def test_colours_decouple():
    g = S.Grid(12, 10)
    en, ec = rand_eta(12, 10, 2)
    L = S.assemble(g, en, ec, velocity_only=True).A.tocsr()
    for s in M.colour_sets(g):
        sub = L[s][:, s]
        assert (sub - sp.diags(sub.diagonal())).count_nonzero() == 0


def test_single_level_vcycle_is_exact():
    g = S.Grid(8, 8)
    en, ec = rand_eta(8, 8, 1)
    h = M.Hierarchy(g, en, ec, n_lev=1)
    f = np.random.default_rng(0).standard_normal(g.n_v)
    x = M.vcycle(h, f)
    assert np.allclose(h.L[0] @ x, f, atol=1e-10)


@pytest.mark.parametrize("n", [32, 64])
def test_vcycle_textbook_convergence(n):
    """Constant viscosity: the V(2,2) cycle as a stationary iteration contracts the error by a
    grid-independent factor well below 1 (multigrid's defining property)."""
    g = S.Grid(n, n)
    one = np.ones((n + 2, n + 2))
    h = M.Hierarchy(g, one, one, coarsest_min=2)
    assert h.nlev >= 4
    rng = np.random.default_rng(1)
    f = rng.standard_normal(g.n_v)
    L = h.L[0]
    x = np.zeros_like(f)
    res = [np.linalg.norm(f)]
    for _ in range(6):
        x = x + M.vcycle(h, f - L @ x)
        res.append(np.linalg.norm(f - L @ x))
    rate = (res[-1] / res[1]) ** (1 / 5)
    assert rate < 0.2


def test_uzawa_sign_reading():
    """Exact velocity solve: the stationary iteration x += M^-1 (b - A x) converges with the sign
    reading and diverges with the literal printed sign (the reason for the reading)."""
    f = sinker(16, 16, eta_inc=10.0)
    g = S.Grid(16, 16)
    sysm = S.assemble(g, f.eta_n, f.eta_c, f.rho, (0.0, 1.0))
    h = M.Hierarchy(g, f.eta_n, f.eta_c, n_lev=1)
    for literal, expect_conv in ((False, True), (True, False)):
        x = np.zeros(g.n)
        e0 = S.energy_residual(sysm, f.eta_c, x)[0]
        for _ in range(60):
            x = x + M.uzawa_precond(h, sysm.b - sysm.A @ x, f.eta_c, alpha=0.6, literal_sign=literal)
        e1 = S.energy_residual(sysm, f.eta_c, x)[0]
        if expect_conv:
            assert e1 < 1e-3 * e0
        else:
            assert e1 > e0


def test_preconditioner_pressure_mean_zero_and_linear():
    f = sinker(16, 16)
    g = S.Grid(16, 16)
    h = M.Hierarchy(g, f.eta_n, f.eta_c, coarsest_min=4)
    rng = np.random.default_rng(5)
    r1, r2 = rng.standard_normal(g.n), rng.standard_normal(g.n)
    z1, z2 = M.uzawa_precond(h, r1, f.eta_c), M.uzawa_precond(h, r2, f.eta_c)
    z12 = M.uzawa_precond(h, 2 * r1 - 3 * r2, f.eta_c)
    assert abs(z1[g.n_v:].mean()) < 1e-14
    assert np.allclose(z12, 2 * z1 - 3 * z2, atol=1e-10)


def test_kcycle_pins():
    """K-cycle: (a) with only one level below, no K step applies and it is the V-cycle; (b) the
    first CG direction satisfies Galerkin orthogonality d_1 . (f - L e) = 0 after both steps;
    (c) it contracts far better than the V-cycle on a rough random viscosity (its purpose)."""
    from synth import grf_config
    f = grf_config(64, 64, seed=2)
    g = S.Grid(64, 64)
    # (a) three levels: the K-cycle at level 0 uses level-1 cycles whose coarse solve is exact
    h2 = M.Hierarchy(g, f.eta_n, f.eta_c, n_lev=2)
    rv = np.random.default_rng(4).standard_normal(g.n_v)
    assert np.allclose(M.vcycle(h2, rv, kcycle=1), M.vcycle(h2, rv), atol=1e-12)
    # (b) Galerkin orthogonality on level 1 of a deeper hierarchy
    h = M.Hierarchy(g, f.eta_n, f.eta_c, coarsest_min=2)
    fc = np.random.default_rng(5).standard_normal(h.L[1].shape[0])
    e = M.kcycle_correction(h, fc, 2, 2, 1.0, 1, 99)
    L1 = h.L[1]
    z1 = M.vcycle(h, fc, level=1, kcycle=99)
    res = fc - L1 @ e
    assert abs(z1 @ res) <= 1e-10 * np.linalg.norm(z1) * np.linalg.norm(fc)
    # (c) contraction factor of the stationary iteration x += C(f - L x)
    L = h.L[0]
    def rate(k):
        x = np.zeros_like(rv); r0 = None
        for it in range(8):
            x = x + M.vcycle(h, rv - L @ x, kcycle=k)
            if it == 2:
                r0 = np.linalg.norm(rv - L @ x)
        return (np.linalg.norm(rv - L @ x) / r0) ** (1 / 5)
    assert rate(99) < 0.7 * rate(0)


# ---- the paper's other smoothers (damped Jacobi, RAS-type temporally blocked Jacobi) -------------
def _small_velocity_system(nx=12, ny=10, seed=41):
    g = S.Grid(nx, ny, 1.0, 0.8)
    rng = np.random.default_rng(seed)
    en = 10.0 ** rng.uniform(-1, 1, (ny + 2, nx + 2))
    ec = 10.0 ** rng.uniform(-1, 1, (ny + 2, nx + 2))
    L = S.assemble(g, en, ec, velocity_only=True).A.tocsr()
    f = rng.standard_normal(g.n_v)
    x0 = rng.standard_normal(g.n_v)
    return g, L, f, x0


def test_splitmix64_matches_published_reference_outputs():
    """First five outputs of the public-domain reference implementation (splitmix64.c, S. Vigna;
    generator of Steele, Lea & Flood, OOPSLA 2014) for seed 1234567."""
    ref = [6457827717110365317, 3203168211198807973, 9817491932198370423, 4593380528125082431,
           16408922859458223821]
    z = 1234567
    for r in ref:
        assert M.splitmix64(z) == r
        z = (z + 0x9E3779B97F4A7C15) % (1 << 64)


def test_damped_jacobi_converges_to_the_direct_solution():
    g, L, f, x0 = _small_velocity_system()
    x = x0.copy()
    for _ in range(6000):
        x = M.jacobi_sweep(L, f, x, 0.5)
    xs = spla.spsolve(L.tocsc(), f)
    assert np.linalg.norm(x - xs) <= 1e-8 * np.linalg.norm(xs)


@pytest.mark.parametrize("si,sj,T", [(0, 0, 4), (3, 1, 4), (2, 5, 6)])
def test_ras_with_one_inner_iteration_is_one_jacobi_sweep(si, sj, T):
    g, L, f, x0 = _small_velocity_system()
    a = M.ras_pass(g, L, f, x0, 0.7, 1, T, T, si, sj)
    b = M.jacobi_sweep(L, f, x0, 0.7)
    assert np.allclose(a, b, rtol=1e-13, atol=1e-13)


def test_ras_with_one_tile_is_plain_jacobi():
    g, L, f, x0 = _small_velocity_system()
    a = M.ras_pass(g, L, f, x0, 0.6, 5, 1000, 1000, 0, 0)
    b = x0
    for _ in range(5):
        b = M.jacobi_sweep(L, f, b, 0.6)
    assert np.allclose(a, b, rtol=1e-12, atol=1e-12)


def test_ras_with_single_cell_tiles_converges_to_block_jacobi():
    """Tiles of one cell own vx(i, j) and vy(i, j); many local iterations solve each cell's 1x1 or
    2x2 block exactly with everything else held: block Jacobi, computed here by direct solves."""
    g, L, f, x0 = _small_velocity_system()
    a = M.ras_pass(g, L, f, x0, 1.0, 200, 1, 1, 0, 0)
    vi = np.concatenate([g.vx_i, g.vy_i]); vj = np.concatenate([g.vx_j, g.vy_j])
    Ld = L.toarray()
    b = x0.copy()
    for key in set(zip(vi, vj)):
        S_ = np.nonzero((vi == key[0]) & (vj == key[1]))[0]
        O_ = np.setdiff1d(np.arange(len(x0)), S_)
        rhs = f[S_] - Ld[np.ix_(S_, O_)] @ x0[O_]
        b[S_] = np.linalg.solve(Ld[np.ix_(S_, S_)], rhs)
    assert np.allclose(a, b, rtol=1e-10, atol=1e-10)


def _mixed_case(nx=24, ny=16, n_lev=None, smoother="mixed", seed=53):
    g = S.Grid(nx, ny, 1.0, ny / nx)
    rng = np.random.default_rng(seed)
    en = 10.0 ** rng.uniform(-0.5, 0.5, (ny + 2, nx + 2)); ec = 10.0 ** rng.uniform(-0.5, 0.5, (ny + 2, nx + 2))
    return M.Hierarchy(g, en, ec, coarsest_min=2, n_lev=n_lev, smoother=smoother, ras_inner=2, ras_tile=4), rng


def test_mixed_smoother_is_damped_jacobi_on_the_finest_level():
    """Two levels with a direct coarsest solve: only the finest level is smoothed, so the "Mixed"
    configuration must give exactly the damped-Jacobi cycle (and differ from the RAS one)."""
    hm, rng = _mixed_case(n_lev=2)
    hj, _ = _mixed_case(n_lev=2, smoother="jacobi")
    hr, _ = _mixed_case(n_lev=2, smoother="ras")
    f = rng.standard_normal(hm.L[0].shape[0])
    a = M.vcycle(hm, f, 2, 2, 0.6)
    assert np.array_equal(a, M.vcycle(hj, f, 2, 2, 0.6))
    assert not np.allclose(a, M.vcycle(hr, f, 2, 2, 0.6), rtol=1e-6, atol=0)


def test_mixed_smoother_is_ras_below_the_finest_level():
    """A cycle started on level 1 never touches the finest level, so there the "Mixed"
    configuration must give exactly the RAS-type cycle (and differ from the Jacobi one)."""
    hm, rng = _mixed_case(n_lev=3)
    hj, _ = _mixed_case(n_lev=3, smoother="jacobi")
    hr, _ = _mixed_case(n_lev=3, smoother="ras")
    f1 = rng.standard_normal(hm.L[1].shape[0])
    a = M.vcycle(hm, f1, 2, 2, 0.6, level=1)
    assert np.array_equal(a, M.vcycle(hr, f1, 2, 2, 0.6, level=1))
    assert not np.allclose(a, M.vcycle(hj, f1, 2, 2, 0.6, level=1), rtol=1e-6, atol=0)


@pytest.mark.parametrize("smoother", ["jacobi", "ras", "mixed"])
def test_vcycle_with_jacobi_smoothers_contracts(smoother):
    g = S.Grid(32, 32)
    rng = np.random.default_rng(43)
    en = 10.0 ** rng.uniform(-0.5, 0.5, (34, 34)); ec = 10.0 ** rng.uniform(-0.5, 0.5, (34, 34))
    h = M.Hierarchy(g, en, ec, coarsest_min=4, smoother=smoother, ras_inner=2, ras_tile=8)
    L = h.L[0]
    e = rng.standard_normal(L.shape[0])
    for _ in range(6):
        e_new = e - M.vcycle(h, L @ e, 2, 2, 0.6)
        rate = np.linalg.norm(e_new) / np.linalg.norm(e)
        e = e_new
    assert rate < 0.8


def test_large_coarsest_level_is_smoothed_and_the_cycle_still_contracts():
    """90 x 66 halves once to 45 x 33 (2892 velocity unknowns, above the direct-solve limit): the
    coarsest level gets smoothing sweeps from zero; the cycle must still contract."""
    g = S.Grid(90, 66, 1.0, 66 / 90)
    rng = np.random.default_rng(47)
    en = 10.0 ** rng.uniform(-0.5, 0.5, (68, 92)); ec = 10.0 ** rng.uniform(-0.5, 0.5, (68, 92))
    h = M.Hierarchy(g, en, ec, coarsest_min=4, coarse_sweeps=40, coarsen_general=False)
    assert h.nlev == 2 and not h.coarse_direct
    L = h.L[0]
    e = rng.standard_normal(L.shape[0])
    for _ in range(5):
        e_new = e - M.vcycle(h, L @ e, 2, 2, 1.0)
        rate = np.linalg.norm(e_new) / np.linalg.norm(e)
        e = e_new
    assert rate < 0.9



# ---- arbitrary coarsening ratio ------------------------------------------------------------------
@pytest.mark.parametrize("ratio", [2.0, 2.5, 3.0])
def test_level_sizes_rule(ratio):
    sizes = M.level_sizes(500, 600, 4, ratio)
    assert sizes[0] == (500, 600)
    assert M.velocity_unknowns(*sizes[-1]) <= M.MAX_COARSE
    for (a, b), (c, d) in zip(sizes, sizes[1:]):
        if ratio == 2.0 and a % 2 == 0 and b % 2 == 0 and min(a, b) // 2 >= 4:
            assert (c, d) == (a // 2, b // 2)
        else:
            assert (c, d) == (int(np.ceil(a / ratio - 1e-9)), int(np.ceil(b / ratio - 1e-9)))
    assert M.level_sizes(45, 33, 4) == [(45, 33), (23, 17)]


@pytest.mark.parametrize("nf,nc", [((45, 33), (23, 17)), ((100, 80), (40, 32)), ((37, 29), (13, 10))])
def test_general_transfer_operators(nf, nc):
    """Any ratio: the normalised restriction maps constants to constants; bilinear prolongation
    reproduces a bilinear function at every fine unknown whose interpolation stencil avoids the
    wall ghosts; R and P have the supports of one coarse spacing."""
    fine = S.Grid(nf[0], nf[1], 1.3, 0.9)
    coarse = M.coarsen_grid(fine, *nc)
    for fld in ("vx", "vy"):
        R = M.restriction_matrix(fine, coarse, fld)
        P = M.prolongation_matrix(fine, coarse, fld)
        nF = R.shape[1]
        assert np.allclose(R @ np.ones(nF), 1.0, atol=1e-13)
        Xc, Yc = M.positions(coarse, fld)
        Xf, Yf = M.positions(fine, fld)
        f = lambda x, y: 0.4 + 1.1 * x - 0.7 * y + 0.9 * x * y
        pf = P @ f(Xc, Yc)
        H, K = coarse.dx, coarse.dy
        if fld == "vx":
            inner = (Xf > H) & (Xf < fine.Lx - H) & (Yf > K / 2) & (Yf < fine.Ly - K / 2)
        else:
            inner = (Xf > H / 2) & (Xf < fine.Lx - H / 2) & (Yf > K) & (Yf < fine.Ly - K)
        assert inner.sum() > 10
        assert np.allclose(pf[inner], f(Xf, Yf)[inner], atol=1e-12)
        C = R.tocoo()
        assert np.all(np.abs(Xf[C.col] - Xc[C.row]) < H) and np.all(np.abs(Yf[C.col] - Yc[C.row]) < K)
    en, ec = M.coarsen_eta(fine, coarse, np.full((nf[1] + 2, nf[0] + 2), 2.5), np.full((nf[1] + 2, nf[0] + 2), 2.5))
    assert np.allclose(en[:nc[1] + 1, :nc[0] + 1], 2.5) and np.allclose(ec[1:nc[1] + 1, 1:nc[0] + 1], 2.5)


@pytest.mark.parametrize("ratio", [2.0, 2.5])
def test_vcycle_with_general_levels_contracts(ratio):
    g = S.Grid(90, 66, 1.0, 66 / 90)
    rng = np.random.default_rng(53)
    en = 10.0 ** rng.uniform(-0.5, 0.5, (68, 92)); ec = 10.0 ** rng.uniform(-0.5, 0.5, (68, 92))
    h = M.Hierarchy(g, en, ec, coarsest_min=4, coarsen_ratio=ratio)
    assert h.coarse_direct and h.nlev >= 2
    L = h.L[0]
    e = rng.standard_normal(L.shape[0])
    for _ in range(6):
        e_new = e - M.vcycle(h, L @ e, 2, 2, 1.0)
        rate = np.linalg.norm(e_new) / np.linalg.norm(e)
        e = e_new
    assert rate < 0.6
