"""Continuous batching on the GPU: each request's result is the same alone and in the mix."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from synth import serving_request
from paper_2603_14040_b300.serving import SolveServer, Request, PyroBackend, latency_stats


def _requests(ids):
    out = []
    for k in ids:
        f, contrast = serving_request(k, sizes=(32, 64), aspects=(1, 2), n_inc=4)
        dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
        out.append(Request(rid=k, nx=f.nx, ny=f.ny, Lx=f.Lx, Ly=f.Ly, eta_n=dev(f.eta_n), eta_c=dev(f.eta_c),
                           rho=dev(f.rho), g=(0.0, 1.0), tol=1e-8))
    return out


def test_same_result_alone_and_in_the_mix():
    ids = list(range(12))
    be = PyroBackend(opts_kw={"max_iter": 600})
    # alone: one slot, one request at a time
    alone = {}
    srv = SolveServer(be, max_slots=1)
    for r in _requests(ids):
        srv.submit(r)
        srv.drain(timeout=300)
        alone[r.rid] = [t.cpu().numpy() for t in r.result]
    srv.close()
    # in the mix: four slots, all submitted at once, handles shared between shapes
    srv = SolveServer(be, max_slots=4)
    mix = _requests(ids)
    for r in mix:
        srv.submit(r)
    done = srv.drain(timeout=300)
    srv.close()
    assert len(done) == len(ids) and all(r.error is None for r in done)
    assert srv.max_concurrent >= 2
    for r in mix:
        for a, b in zip(alone[r.rid], [t.cpu().numpy() for t in r.result]):
            assert np.array_equal(a, b), r.rid
    st = latency_stats(done)
    assert st["n"] == len(ids) and st["p99_ms"] >= st["p50_ms"] > 0


def test_served_results_match_the_direct_oracle():
    """Eight sharp-inclusion requests (contrast 10^U[2,6], 64 x 64 and 128 x 64) served three at a
    time: every result's energy residual, recomputed by the oracle from the assembled system, meets
    the tolerance, and the result matches the oracle's direct solve. The bound follows the
    conditioning: the oracle's own FGMRES at tol 1e-10 leaves up to du = 6.5e-7, dp = 2.9e-5 on these
    requests (contrast 3e5), so at tol 1e-11 du <= 1e-6 and dp <= 1e-5 are checked."""
    from oracle import stokes as S
    tol = 1e-11
    reqs, fields = [], {}
    for k in range(8):
        f, contrast = serving_request(k, sizes=(64,), aspects=(1, 2))
        fields[k] = f
        dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
        reqs.append(Request(rid=k, nx=f.nx, ny=f.ny, Lx=f.Lx, Ly=f.Ly, eta_n=dev(f.eta_n), eta_c=dev(f.eta_c),
                            rho=dev(f.rho), g=(0.0, 1.0), tol=tol))
    be = PyroBackend(opts_kw={"max_iter": 4000}, restart_choices=(200,))
    srv = SolveServer(be, max_slots=3)
    for r in reqs:
        srv.submit(r)
    done = srv.drain(timeout=600)
    srv.close()
    assert len(done) == 8 and all(r.error is None and r.status == 0 for r in done), [(r.rid, r.status) for r in done]
    for r in reqs:
        f = fields[r.rid]
        g = S.Grid(f.nx, f.ny, f.Lx, f.Ly)
        sysm = S.assemble(g, f.eta_n, f.eta_c, f.rho, (0.0, 1.0))
        x = S.fields_to_vector(g, *(t.cpu().numpy() for t in r.result))
        e, _ = S.energy_residual(sysm, f.eta_c, x)
        assert e <= 1.01 * tol, (r.rid, e)
        xd = S.remove_pressure_mean(g, S.solve_direct(sysm))
        nv = g.n_v
        du = np.linalg.norm(x[:nv] - xd[:nv]) / np.linalg.norm(xd[:nv])
        dp = np.linalg.norm(x[nv:] - xd[nv:]) / np.linalg.norm(xd[nv:])
        assert du <= 1e-6 and dp <= 1e-5, (r.rid, du, dp)
