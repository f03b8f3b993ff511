"""The paper's own outer accelerators on the GPU (flexible GCR(m), Algorithm gcr; Anderson
AA(m, beta), Algorithm anderson) against the oracle: iterate by iterate with the same FP64
Uzawa/multigrid preconditioner, and converged solutions against the direct solve."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import stokes as S
from oracle import multigrid as M
from oracle import accelerators as AC
from synth import sinker
from gpu_util import dev, host, zeros, rel

import paper_2603_14040_b300 as P
from test_gpu_parity import rand_eta, _solve_gpu, _check_against_direct

G = (0.0, 1.0)


def _problem(nx, ny, seed):
    g = S.Grid(nx, ny, 1.0, ny / nx)
    en, ec = rand_eta(nx, ny, seed, -1, 1)
    rho = 1.0 + 0.1 * np.random.default_rng(seed + 5).standard_normal((ny + 2, nx + 2))
    sysm = S.assemble(g, en, ec, rho, G)
    h_or = M.Hierarchy(g, en, ec, coarsest_min=2)
    pre = lambda r: M.uzawa_precond(h_or, r, ec, alpha=1.0)
    W = np.concatenate([1.0 / -sysm.A.diagonal()[:g.n_v], S.pressure_weights(g, ec)])
    return g, en, ec, rho, sysm, pre, W


def _gpu_iterate(g, en, ec, rho, k, **opts):
    h = P.Stokes(g.nx, g.ny, g.Lx, g.Ly, prec=P.PREC_FP64, coarsest_min=2, max_iter=k, **opts)
    out = [zeros(g.ny, g.nx) for _ in range(3)]
    st = h.solve(dev(en), dev(ec), dev(rho), G, 1e-30, *out)
    torch.cuda.synchronize()
    h.close()
    return S.fields_to_vector(g, *(host(a) for a in out)), st


@pytest.mark.parametrize("k", [1, 3, 7])
def test_gcr_iterates_match_oracle(k):
    g, en, ec, rho, sysm, pre, W = _problem(32, 24, 31)
    hist = []
    AC.gcr(sysm.A, sysm.b, pre, m=30, tol=1e-30, maxit=k, W=W, true_residual_at_restart=True, history=hist)
    x, st = _gpu_iterate(g, en, ec, rho, k, accel=P.ACCEL_GCR)
    assert st.iters == k
    ref = S.remove_pressure_mean(g, hist[-1])
    assert rel(x, ref) <= 1e-9, rel(x, ref)


@pytest.mark.parametrize("k,m,beta", [(1, 5, 0.8), (2, 5, 0.8), (6, 5, 0.8), (9, 3, 0.5), (6, 10, 1.0)])
def test_anderson_iterates_match_oracle(k, m, beta):
    g, en, ec, rho, sysm, pre, W = _problem(32, 24, 37)
    hist = []
    AC.anderson(sysm.A, sysm.b, pre, m=m, beta=beta, tol=1e-30, maxit=k + 1, history=hist)
    x, st = _gpu_iterate(g, en, ec, rho, k, accel=P.ACCEL_ANDERSON, restart_m=m, aa_beta=beta)
    assert st.iters == k
    ref = S.remove_pressure_mean(g, hist[k - 1])
    assert rel(x, ref) <= 1e-8, rel(x, ref)


@pytest.mark.parametrize("accel,m", [(P.ACCEL_GCR, 30), (P.ACCEL_ANDERSON, 10)])
@pytest.mark.parametrize("prec", [P.PREC_FP64, P.PREC_MIXED])
def test_accelerated_sinker_matches_direct_oracle(accel, m, prec):
    f = sinker(64, 64)
    out, st = _solve_gpu(f, G, 1e-12, prec, accel=accel, restart_m=m, max_iter=2000)
    _check_against_direct(f, out, st, tol=1e-12, tol_err=1e-8)
