"""Host-side logic of the continuous-batching server, driven by a fake backend (CPU only)."""
import threading
import time

import numpy as np
import pytest

from paper_2603_14040_b300.serving import (SolveServer, Request, HandlePool, latency_stats, poisson_arrivals)


class FakeBackend:
    """Footprint proportional to cells; solve sleeps in proportion to cells and returns a value
    that depends only on the request's inputs (so alone == in the mix iff the server passes the
    right data to the right handle)."""

    def __init__(self, budget=10**9, fail_rid=None, per_cell_s=2e-7):
        self.budget = budget
        self.fail_rid = fail_rid
        self.per_cell_s = per_cell_s
        self.lock = threading.Lock()
        self.creates = 0
        self.destroys = 0
        self.active = 0
        self.peak_active = 0
        self.peak_bytes = 0
        self.pool = None

    def default_budget(self):
        return self.budget

    def make_stream(self):
        return object()

    def footprint(self, shape):
        return shape[0] * shape[1] * 100

    def create(self, shape):
        with self.lock:
            self.creates += 1
        return {"shape": shape}

    def destroy(self, h):
        with self.lock:
            self.destroys += 1

    def solve(self, h, req, stream):
        assert h["shape"] == req.shape
        with self.lock:
            self.active += 1
            self.peak_active = max(self.peak_active, self.active)
            if self.pool is not None:
                self.peak_bytes = max(self.peak_bytes, self.pool.bytes_in_use)
        try:
            time.sleep(req.nx * req.ny * self.per_cell_s)
            if req.rid == self.fail_rid:
                raise RuntimeError("injected failure")
            val = float(np.sum(req.eta_c) * 1.5 + np.sum(req.rho))
            return val, {"status": 0, "iters": 7}
        finally:
            with self.lock:
                self.active -= 1


def _reqs(n, seed=0, sizes=(16, 32, 64)):
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n):
        s = int(rng.choice(sizes))
        a = int(rng.choice([1, 2]))
        ec = rng.standard_normal((s + 2, a * s + 2))
        out.append(Request(rid=k, nx=a * s, ny=s, Lx=float(a), Ly=1.0, eta_n=None, eta_c=ec,
                           rho=ec * 0.5, tol=1e-8))
    return out


def test_all_requests_complete_with_correct_results_and_slot_limit():
    be = FakeBackend()
    srv = SolveServer(be, max_slots=3)
    be.pool = srv.pool
    reqs = _reqs(40)
    for r in reqs:
        srv.submit(r)
    done = srv.drain(timeout=60)
    srv.close()
    assert len(done) == 40 and all(r.error is None for r in done)
    for r in reqs:
        assert r.result == pytest.approx(float(np.sum(r.eta_c) * 1.5 + np.sum(r.rho)))
        assert r.done >= r.admitted >= r.arrival
    assert be.peak_active <= 3 and srv.max_concurrent <= 3
    # handles are reused per shape: no more creations than distinct shapes x slots
    assert be.creates <= len({r.shape for r in reqs}) * 3


def test_memory_budget_is_never_exceeded_and_lru_eviction_works():
    be = FakeBackend(budget=2 * 64 * 64 * 100)      # two 64x64 handles at most
    srv = SolveServer(be, max_slots=4)
    be.pool = srv.pool
    reqs = _reqs(30, seed=3, sizes=(32, 64))
    for r in reqs:
        srv.submit(r)
    done = srv.drain(timeout=60)
    srv.close()
    assert all(r.error is None for r in done)
    assert be.peak_bytes <= srv.pool.budget
    assert be.destroys > 0                               # shapes had to be evicted


def test_oversized_and_failing_requests_do_not_stop_the_server():
    be = FakeBackend(budget=64 * 64 * 100, fail_rid=3)
    srv = SolveServer(be, max_slots=2)
    reqs = _reqs(10, seed=5, sizes=(16, 32))
    big = Request(rid=99, nx=256, ny=256, Lx=1.0, Ly=1.0, eta_n=None, eta_c=np.ones((258, 258)),
                  rho=np.ones((258, 258)))
    for r in reqs + [big]:
        srv.submit(r)
    done = srv.drain(timeout=60)
    srv.close()
    assert len(done) == 11
    assert big.error is not None and "cannot be served" in big.error
    assert reqs[3].error is not None and "injected" in reqs[3].error
    assert sum(r.error is None for r in done) == 9


def test_a_failed_handle_creation_fails_only_its_request():
    """A backend whose handle creation raises (as a CUDA error from the library would) ends that
    request with an error; the server keeps serving the others and drains."""
    class CreateFails(FakeBackend):
        def create(self, shape):
            if shape[0] == 32:
                raise RuntimeError("pyro_stokes_create: CUDA runtime error")
            return super().create(shape)

    be = CreateFails()
    srv = SolveServer(be, max_slots=2)
    reqs = _reqs(12, seed=7, sizes=(16, 32))
    for r in reqs:
        srv.submit(r)
    done = srv.drain(timeout=60)
    srv.close()
    assert len(done) == 12
    for r in reqs:
        if r.nx == 32:
            assert r.error is not None and "CUDA runtime error" in r.error and r.status == -1
        else:
            assert r.error is None
    assert any(r.nx == 32 for r in reqs) and any(r.nx != 32 for r in reqs)
    assert srv.pool.bytes_in_use == 0


def test_requests_arriving_while_others_run_are_admitted_continuously():
    """Continuous batching: a request submitted while slots are busy starts before earlier long
    solves finish (it takes a freed slot), and arrival order is kept among waiting requests."""
    be = FakeBackend(per_cell_s=0.0)
    srv = SolveServer(be, max_slots=2)
    long1 = Request(rid=1, nx=64, ny=64, Lx=1, Ly=1, eta_n=None, eta_c=np.ones((66, 66)), rho=np.ones((66, 66)))
    long1.tol = 1e-8
    be.per_cell_s = 5e-5                                  # ~0.2 s for 64x64
    srv.submit(long1)
    time.sleep(0.02)
    shorts = [Request(rid=10 + k, nx=4, ny=4, Lx=1, Ly=1, eta_n=None, eta_c=np.ones((6, 6)), rho=np.ones((6, 6)))
              for k in range(5)]
    for r in shorts:
        srv.submit(r)
    done = srv.drain(timeout=30)
    srv.close()
    assert all(r.done < long1.done for r in shorts)
    admits = [r.admitted for r in shorts]
    assert admits == sorted(admits)


def test_pool_reuse_and_accounting():
    be = FakeBackend(budget=10**6)
    pool = HandlePool(be, 10**6)
    h1 = pool.acquire((10, 10, 1.0, 1.0))
    pool.release((10, 10, 1.0, 1.0), h1)
    h2 = pool.acquire((10, 10, 1.0, 1.0))
    assert h2 is h1 and be.creates == 1
    assert pool.bytes_in_use == 10 * 10 * 100
    pool.release((10, 10, 1.0, 1.0), h2)
    pool.close()
    assert pool.bytes_in_use == 0 and be.destroys == 1


def test_poisson_arrivals_and_latency_stats():
    t = poisson_arrivals(20000, rate=50.0, seed=4)
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert abs(gaps.mean() - 1 / 50.0) < 0.05 / 50.0
    assert abs(np.std(gaps) / gaps.mean() - 1.0) < 0.05        # exponential: cv = 1
    reqs = []
    for k in range(100):
        r = Request(rid=k, nx=2, ny=2, Lx=1, Ly=1, eta_n=None, eta_c=None, rho=None)
        r.arrival, r.done = 0.0, (k + 1) * 1e-3
        reqs.append(r)
    st = latency_stats(reqs)
    assert st["n"] == 100 and st["p50_ms"] == pytest.approx(50.5, rel=1e-6)
    assert st["p99_ms"] == pytest.approx(99.01, rel=1e-4)


def test_restart_length_is_chosen_per_shape_to_fit():
    """The libpyro backend picks, per grid shape, the longest restart whose handle fits the
    per-handle share of the budget (host-side footprint only; no GPU)."""
    pytest.importorskip("torch")
    from paper_2603_14040_b300.serving import PyroBackend
    import paper_2603_14040_b300 as P
    be = PyroBackend(opts_kw={"prec": 1}, restart_choices=(200, 100, 50, 30), per_handle_bytes=4 * 2**30)
    small, big = (256, 256, 1.0, 1.0), (4096, 1024, 4.0, 1.0)
    assert be.opts_for(small)["restart_m"] == 200
    m_big = be.opts_for(big)["restart_m"]
    assert m_big < 200
    assert be.footprint(big) <= 4 * 2**30 or m_big == 30
    assert be.footprint(small) == P.footprint(256, 256, P.default_opts(prec=1, restart_m=200))
