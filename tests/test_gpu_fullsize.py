"""Parity at the full sizes of the benchmark workloads, in the launch configuration bench.py times.

The oracle's direct solve does not reach these sizes. Two kinds of check replace it:
  * element by element against the oracle's iterative FP64 reference solutions stored under
    tests/golden/ (written by tests/golden/make_reference.py, which calls only oracle/; each is
    certified by the true residual of the assembled system at a relative energy residual <= 1e-13,
    and the iterative reference is pinned to the direct solve in tests/test_oracle_iterative.py):
    the 1024 x 1024 random-viscosity workload (FP64 and mixed, at tol 1e-10 and 1e-12; with the
    paper's pressure block and with the benchmark's weighted BFBt block), the 1024 x 1024 layered
    workload (its BFBt + inner-CG recipe) and the 512 x 512 adjoint member; relative L2 errors in u
    and in p (pressure mean removed on both sides) are printed and must be <= 1e-8 at tol 1e-12
    (with the BFBt block also at tol 1e-10). At tol 1e-10 the forward error is the residual
    times the conditioning of the system: with viscosity over four decades a 1e-10 energy residual
    leaves about 6e-8 in u (measured on a B300), so there the bound checked is 1e-6 and the 1e-8
    comparison is the tol 1e-12 one;
  * properties that hold at any size, computed by the oracle from the GPU's answer:
      - 1024 x 1024 random viscosity: the oracle assembles the whole system and recomputes the
        relative energy residual of the GPU solution (Sec. "Global Relative Energy Residual"),
        which must meet the tolerance and agree with the value the library reports; zero-mean
        pressure, zero normal velocity on the walls;
      - 4096 x 4096 layered lid + inclusions (mixed): at sampled windows (corners, edges, the lid
        interface, the interior) every row of the library's FP64 operator applied to an iterate
        equals the oracle's own row, assembled on the window (a check of the operator at full
        size, not of a converged solve);
      - 512 x 512 adjoint member: dJ/dlog(eta) from the adjoint equals central finite differences
        of J along random directions (each side a full solve).
"""
import json
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import stokes as S
from synth import grf_config, layered_config, adjoint_member
from gpu_util import dev, host, zeros, rel
from window_residual import window_residual, global_positions

import paper_2603_14040_b300 as P
from paper_2603_14040_b300.autograd import stokes_solve, surface_misfit, node_from_cell

G = (0.0, 1.0)
# the adjoint workload's solver options: the paper's eta_c pressure block, or the weighted BFBt block
# of the mixed headline (FGMRES(60), block scaled by 0.8, 16 x 16 coarsest velocity level)
ADJ_OPTS = {"paper": {}, "bfbt": {"schur": 1, "restart_m": 60, "alpha_p": 0.8, "coarsest_min": 16}}
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _reference(name):
    d = np.load(os.path.join(GOLDEN, f"reference_{name}.npz"))
    return d["x"], float(d["rel_energy"])


def _errors(g, x, xref):
    """relative L2 errors in u (both velocity components) and in p (means removed)"""
    nv = g.n_v
    pa = x[nv:] - x[nv:].mean()
    pb = xref[nv:] - xref[nv:].mean()
    return rel(x[:nv], xref[:nv]), rel(pa, pb)


def _record(key, value):
    # optional log of the achieved errors (the tests assert the bound either way)
    out = os.environ.get("PYRO_PARITY_OUT")
    print(f"{key}: {value}")
    if out:
        d = json.load(open(out)) if os.path.exists(out) else {}
        d[key] = value
        json.dump(d, open(out, "w"), indent=1)


def _solve(f, n, tol, **opts):
    h = P.Stokes(n, n, **opts)
    out = [zeros(n, n) for _ in range(3)]
    st = h.solve(dev(f.eta_n), dev(f.eta_c), dev(f.rho), G, tol, *out)
    torch.cuda.synchronize()
    h.close()
    return out, st


def test_random_viscosity_1024_fp64_and_mixed_meet_tolerance_by_oracle():
    n, tol = 1024, 1e-10
    f = grf_config(n, n, seed=2)
    g = S.Grid(n, n)
    sysm = S.assemble(g, f.eta_n, f.eta_c, f.rho, G)
    sols = {}
    for prec in (P.PREC_FP64, P.PREC_MIXED):
        out, st = _solve(f, n, tol, prec=prec, max_iter=3000)
        assert st.status == P.PYRO_OK, st.as_dict()
        vx, vy, p = (host(a) for a in out)
        x = S.fields_to_vector(g, vx, vy, p)
        e_or, l2_or = S.energy_residual(sysm, f.eta_c, x)
        assert e_or <= 1.01 * tol, (prec, e_or, st.as_dict())
        assert abs(e_or - st.rel_energy_res) <= 1e-3 * e_or
        assert abs(l2_or - st.rel_l2_res) <= 1e-3 * l2_or + 1e-16
        assert abs(p[1:n + 1, 1:n + 1].mean()) <= 1e-12 * np.abs(p).max()
        assert np.all(vx[:, 0] == 0) and np.all(vx[:, n] == 0)
        assert np.all(vy[0, :] == 0) and np.all(vy[n, :] == 0)
        sols[prec] = x
    a, b = sols[P.PREC_FP64], sols[P.PREC_MIXED]
    assert rel(b[:g.n_v], a[:g.n_v]) <= 1e-8 and rel(b[g.n_v:], a[g.n_v:]) <= 1e-8


def test_layered_4096_mixed_operator_rows_only_match_oracle_windows():
    n, tol = 4096, 1e-10
    f = layered_config(n, n, seed=3)
    h = P.Stokes(n, n, prec=P.PREC_MIXED, max_iter=600)
    out = [zeros(n, n) for _ in range(3)]
    en, ec, rho = dev(f.eta_n), dev(f.eta_c), dev(f.rho)
    st = h.solve(en, ec, rho, G, tol, *out)
    assert st.status in (P.PYRO_OK, P.PYRO_W_NOT_CONVERGED), st.as_dict()
    assert 0.0 < st.rel_energy_res < 1e-2, st.as_dict()
    r = [zeros(n, n) for _ in range(3)]
    h.apply(en, ec, *out, *r)
    torch.cuda.synchronize()
    h.close()
    vx, vy, p = (host(a) for a in out)
    R = [host(a) for a in r]
    lid = int(0.1 * n)
    blocks = [((1, 12), (1, 12)), ((n - 11, n), (n - 11, n)), ((1, 10), (2000, 2020)),
              ((lid - 6, lid + 6), (1000, 1016)), ((lid - 6, lid + 6), (n - 9, n)),
              ((2048, 2064), (2048, 2064)), ((3000, 3010), (1, 9))]
    rng = np.random.default_rng(7)
    for _ in range(5):
        i0, j0 = rng.integers(1, n - 16, size=2)
        blocks.append(((int(i0), int(i0) + 15), (int(j0), int(j0) + 15)))
    checked = 0
    for rows, cols in blocks:
        wx, wy, wp, sx, sy, sp, lo = window_residual(n, n, 1.0, 1.0, S.BC(), f.eta_n, f.eta_c, f.rho, G,
                                                     vx, vy, p, rows, cols, product=True)
        for win, sc, ref in ((wx, sx, R[0]), (wy, sy, R[1]), (wp, sp, R[2])):
            gi, gj, li, lj = global_positions(win, lo)
            err = np.abs(win[li, lj] - ref[gi, gj])
            assert np.all(err <= 1e-12 * sc[li, lj] + 1e-300), (rows, cols, err.max())
            checked += len(gi)
    assert checked > 2000


@pytest.mark.parametrize("block", ["paper", "bfbt"])
def test_adjoint_512_directional_derivatives_match_central_differences(block):
    n = 512
    base, pert = adjoint_member(0, n, n)
    h = P.Stokes(n, n, prec=P.PREC_MIXED, max_iter=3000, **ADJ_OPTS[block])
    rho = dev(base.rho)
    obs_out = [zeros(n, n) for _ in range(3)]
    st = h.solve(dev(pert.eta_n), dev(pert.eta_c), rho, G, 1e-12, *obs_out)
    assert st.status == P.PYRO_OK
    obs = obs_out[0][1, :].clone()
    log_ec = dev(np.log(np.where(base.eta_c > 0, base.eta_c, 1.0))).requires_grad_(True)

    def J_of(lec):
        ec = torch.zeros_like(lec)
        ec[1:n + 1, 1:n + 1] = torch.exp(lec[1:n + 1, 1:n + 1])
        en = node_from_cell(ec)
        vx, vy, p = stokes_solve(en, ec, rho, h, G, 1e-12)
        return surface_misfit(vx, obs)

    J = J_of(log_ec)
    J.backward()
    grad = log_ec.grad.detach().clone()
    assert torch.isfinite(grad).all()
    rng = np.random.default_rng(11)
    eps = 1e-4
    for k in range(2):
        d = np.zeros((n + 2, n + 2))
        d[1:n + 1, 1:n + 1] = rng.standard_normal((n, n))
        dd = dev(d)
        with torch.no_grad():
            jp = J_of(log_ec.detach() + eps * dd).item()
            jm = J_of(log_ec.detach() - eps * dd).item()
        fd = (jp - jm) / (2 * eps)
        an = float((grad * dd).sum())
        assert abs(fd - an) <= 1e-4 * abs(an) + 1e-14, (k, fd, an)
    h.close()


@pytest.mark.parametrize("tol", [1e-10, 1e-12])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_random_viscosity_1024_matches_iterative_reference_elementwise(prec, tol):
    n = 1024
    f = grf_config(n, n, seed=2)
    g = S.Grid(n, n)
    xref, eref = _reference("grf1024")
    assert eref <= 1e-13
    out, st = _solve(f, n, tol, prec=P.PREC_FP64 if prec == "fp64" else P.PREC_MIXED, max_iter=3000)
    assert st.status == P.PYRO_OK, st.as_dict()
    x = S.fields_to_vector(g, *(host(a) for a in out))
    du, dp = _errors(g, x, xref)
    _record(f"grf1024_{prec}_tol{tol:g}", {"du": du, "dp": dp, "iters": st.iters, "rel_energy": st.rel_energy_res})
    bound = 1e-8 if tol <= 1e-12 else 1e-6
    assert du <= bound and dp <= bound, (du, dp)


@pytest.mark.parametrize("tol", [1e-10, 1e-12])
@pytest.mark.parametrize("prec,restart,alpha,coarsest", [("fp64", 80, 1.0, 4), ("mixed", 60, 1.0, 4),
                                                         ("fp64", 80, 0.8, 16), ("mixed", 60, 0.8, 16)])
def test_random_viscosity_1024_bfbt_matches_iterative_reference_elementwise(prec, restart, alpha, coarsest, tol):
    """The benchmark's own configuration (weighted BFBt pressure block scaled by 0.8, a 16 x 16
    coarsest velocity level, FGMRES(80) in FP64 and FGMRES(60) mixed) and the same block unscaled
    on the default hierarchy: with the stronger pressure block the forward error at tol 1e-10 is
    already below 1e-8, so the 1e-8 bar is asserted at both tolerances."""
    n = 1024
    f = grf_config(n, n, seed=2)
    g = S.Grid(n, n)
    xref, eref = _reference("grf1024")
    assert eref <= 1e-13
    out, st = _solve(f, n, tol, prec=P.PREC_FP64 if prec == "fp64" else P.PREC_MIXED, max_iter=3000, schur=1,
                     restart_m=restart, alpha_p=alpha, coarsest_min=coarsest)
    assert st.status == P.PYRO_OK, st.as_dict()
    x = S.fields_to_vector(g, *(host(a) for a in out))
    du, dp = _errors(g, x, xref)
    _record(f"grf1024_bfbt_{prec}_m{restart}_a{alpha:g}_c{coarsest}_tol{tol:g}",
            {"du": du, "dp": dp, "iters": st.iters, "rel_energy": st.rel_energy_res})
    assert du <= 1e-8 and dp <= 1e-8, (du, dp)


@pytest.mark.parametrize("block", ["paper", "bfbt"])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_adjoint_member_512_forward_matches_iterative_reference_elementwise(prec, block):
    n = 512
    base, _ = adjoint_member(0, n, n)
    g = S.Grid(n, n)
    xref, eref = _reference("adjoint512")
    assert eref <= 1e-13
    out, st = _solve(base, n, 1e-12, prec=P.PREC_FP64 if prec == "fp64" else P.PREC_MIXED, max_iter=3000,
                     **ADJ_OPTS[block])
    assert st.status == P.PYRO_OK, st.as_dict()
    x = S.fields_to_vector(g, *(host(a) for a in out))
    du, dp = _errors(g, x, xref)
    _record(f"adjoint512_{prec}_{block}_tol1e-12", {"du": du, "dp": dp, "iters": st.iters})
    assert du <= 1e-8 and dp <= 1e-8, (du, dp)


@pytest.mark.parametrize("prec,tol,schur,res64", [("mixed", 1e-10, 1, 0), ("mixed", 1e-10, 2, 1), ("fp64", 1e-10, 1, 0),
                                                   ("fp64", 1e-12, 1, 0)])
def test_layered_1024_matches_iterative_reference_elementwise(prec, tol, schur, res64):
    """The layered workload's recipe (lid 1e6, inclusions 10^U[-3,3]) at 1024^2, solved with the
    weighted BFBt block and 5 inner flexible-CG steps, against the oracle's reference (exact velocity
    LU, BFBt pressure block, true residual <= 1e-13). At this contrast the residual is amplified into
    the error: the oracle's own solve of the same recipe at 96^2 leaves du = 1.7e-8, dp = 1.1e-7 at
    a residual of 1.7e-11 (about 1e3 in u and 6e3 in p), so the bounds are 10x that amplification
    times the tolerance. In mixed precision the block runs in FP32 (schur 1) or in FP64 after the
    FP32 V-cycle with the finest V-cycle residual in FP64 (schur 2, res64: the form that also
    converges at 4096^2)."""
    n = 1024
    f = layered_config(n, n, seed=3)
    g = S.Grid(n, n)
    xref, eref = _reference("layered1024")
    assert eref <= 1e-13
    out, st = _solve(f, n, tol, prec=P.PREC_FP64 if prec == "fp64" else P.PREC_MIXED, schur=schur, res64=res64, inner_cg=5,
                     restart_m=200, nu1=4, nu2=4, max_iter=3000)
    assert st.status == P.PYRO_OK, st.as_dict()
    x = S.fields_to_vector(g, *(host(a) for a in out))
    du, dp = _errors(g, x, xref)
    _record(f"layered1024_{prec}_schur{schur}_res64{res64}_tol{tol:g}",
            {"du": du, "dp": dp, "iters": st.iters, "rel_energy": st.rel_energy_res})
    assert du <= 1e4 * tol and dp <= 6e4 * tol, (du, dp)
