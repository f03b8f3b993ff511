"""Adjoint gradients on the GPU vs the oracle (assembly linearity) and finite differences."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import stokes as S
from synth import random_field_log10, sample_lattice_to_fields
from gpu_util import dev, host, zeros, rel

import paper_2603_14040_b300 as P
from paper_2603_14040_b300.autograd import stokes_solve, surface_misfit, node_from_cell


def _case(n, seed, corr=0.2):
    l10 = random_field_log10(n, n, seed, corr_len=corr)
    rho_s = 1.0 + 0.1 * random_field_log10(n, n, seed + 7, corr_len=corr)
    f = sample_lattice_to_fields(10.0 ** l10, rho_s, n, n)
    vx_obs = np.random.default_rng(seed).standard_normal(n + 2) * 1e-3
    return f, vx_obs


@pytest.mark.parametrize("block", ["paper", "bfbt"])
@pytest.mark.parametrize("bc", ["free", "noslip"])
@pytest.mark.parametrize("prec", [P.PREC_FP64, P.PREC_MIXED])
def test_adjoint_matches_oracle_linearity(bc, prec, block):
    """The adjoint solve (the same symmetric operator and preconditioner as the forward solve) and
    the strain-rate products against the oracle's gradient by assembly linearity, with the paper's
    eta_c pressure block and with the weighted BFBt block."""
    n = 16
    kind = (S.FREE_SLIP,) * 4 if bc == "free" else (S.NO_SLIP,) * 4
    f, vx_obs = _case(n, 11)
    g = S.Grid(n, n, bc=S.BC(kind))
    sysm = S.assemble(g, f.eta_n, f.eta_c, f.rho, (0.0, 1.0))
    x = S.solve_direct(sysm)
    vx, _, _ = S.vector_to_fields(g, x, fill_ghosts=False)
    dJ = np.zeros(g.n)
    js = np.arange(1, n)
    dJ[g.idx_vx[1, js]] = vx[1, js] - vx_obs[js]
    lam = S.solve_direct(S.System(g, sysm.A, dJ))
    gn_o, gc_o = S.eta_gradient_by_linearity(g, f.eta_n, f.eta_c, x, lam)
    gr_o = S.rho_gradient_by_linearity(g, (0.0, 1.0), lam)

    opts = {} if block == "paper" else {"schur": 1, "alpha_p": 0.8}
    h = P.Stokes(n, n, bc=P.make_bc(kind), prec=prec, **opts)
    out = [zeros(n, n) for _ in range(3)]
    h.solve(dev(f.eta_n), dev(f.eta_c), dev(f.rho), (0.0, 1.0), 1e-13, *out)
    dvx = np.zeros((n + 2, n + 2))
    dvx[1, js] = host(out[0])[1, js] - vx_obs[js]
    gn, gc, gr = zeros(n, n), zeros(n, n), zeros(n, n)
    h.adjoint(dev(dvx), zeros(n, n), zeros(n, n), 1e-13, gn, gc, gr)
    torch.cuda.synchronize()
    sc = np.abs(gc_o[1:n + 1, 1:n + 1]).max()
    assert np.abs(host(gc)[1:n + 1, 1:n + 1] - gc_o[1:n + 1, 1:n + 1]).max() <= 1e-7 * sc
    assert np.abs(host(gn)[:n + 1, :n + 1] - gn_o[:n + 1, :n + 1]).max() <= 1e-7 * sc
    assert np.abs(host(gr)[:n + 1, :n + 1] - gr_o[:n + 1, :n + 1]).max() <= 1e-7 * np.abs(gr_o).max()


def test_autograd_log_eta_matches_central_fd():
    """dJ/dlog(eta_c) through torch autograd (eta_n = mean of adjacent cells) vs central finite
    differences of the GPU solve itself in log(eta_c), 16 x 16, all 256 cells."""
    n = 16
    f, vx_obs = _case(n, 5)
    h = P.Stokes(n, n, prec=P.PREC_FP64)
    obs = dev(vx_obs)
    rho = dev(f.rho)
    log_ec = dev(np.log(np.where(f.eta_c > 0, f.eta_c, 1.0))).requires_grad_(True)

    def J_of(lec):
        ec = torch.zeros_like(lec)
        ec[1:n + 1, 1:n + 1] = torch.exp(lec[1:n + 1, 1:n + 1])
        en = node_from_cell(ec)
        vx, vy, p = stokes_solve(en, ec, rho, h, (0.0, 1.0), 1e-13)
        return surface_misfit(vx, obs)

    J = J_of(log_ec)
    J.backward()
    grad = host(log_ec.grad)
    hstep = 1e-5
    base = log_ec.detach().clone()
    errs = []
    scale = np.abs(grad).max()
    for i in range(1, n + 1):
        for j in range(1, n + 1):
            vals = []
            for sgn in (1, -1):
                t = base.clone(); t[i, j] += sgn * hstep
                with torch.no_grad():
                    vals.append(float(J_of(t)))
            fd = (vals[0] - vals[1]) / (2 * hstep)
            errs.append(abs(fd - grad[i, j]))
    assert max(errs) <= 1e-6 * scale
