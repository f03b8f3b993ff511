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
