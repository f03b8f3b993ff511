"""GPU test of pyro_stokes_residual_noalloc, the entry point for callers that cannot allocate
device memory (for instance an application whose pool allocator owns the whole GPU, or a loop in
which an allocation's implicit synchronisation is not acceptable). It must give the same numbers
as the regular entry points while allocating nothing: its scratch is a fixed array in device
global memory shared by all calls.

Kept in a file of its own, named so pytest collects it last."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2603_14040_b300 as P
from paper_2603_14040_b300.pyro import residual_noalloc
from synth import grf_config, random_vectors


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def _zeros(ny, nx):
    return torch.zeros((ny + 2, nx + 2), dtype=torch.float64, device="cuda")


def test_noalloc_residual_matches_regular_entry_points():
    nx, ny, Lx, Ly = 48, 80, 0.6, 1.0
    bc = P.make_bc((P.NO_SLIP, P.FREE_SLIP, P.VELOCITY, P.NO_SLIP), (0, 0, 0.7, 0))
    f = grf_config(nx, ny, seed=7, Lx=Lx, Ly=Ly)
    en, ec, rho = _dev(f.eta_n), _dev(f.eta_c), _dev(f.rho)
    h = P.Stokes(nx, ny, Lx, Ly, bc=bc)
    zero_rho = _zeros(ny, nx)
    free = P.make_bc()
    hf = P.Stokes(nx, ny, Lx, Ly, bc=free)
    rel_res = torch.zeros(2, dtype=torch.float64)          # host output
    r = [_zeros(ny, nx) for _ in range(3)]
    Ax = [_zeros(ny, nx) for _ in range(3)]
    sol = [_zeros(ny, nx) for _ in range(3)]
    fields = [tuple(_dev(a) for a in random_vectors(nx, ny, seed)) for seed in (1, 2)]
    torch.cuda.synchronize()

    # two calls in a row with different inputs: without forcing or boundary constants
    # r = -A x, which the regular pyro_stokes_apply computes with its own workspace
    for vx, vy, p in fields:
        st = residual_noalloc(nx, ny, Lx, Ly, free, en, ec, zero_rho, (0.0, 0.0), vx, vy, p, *r, rel_res)
        assert st == P.PYRO_OK
        hf.apply(en, ec, vx, vy, p, *Ax)
        torch.cuda.synchronize()
        for a, b in zip(r, Ax):
            scale = float(b.abs().max())
            assert float((a + b).abs().max()) <= 1e-13 * scale

    # with gravity and a prescribed-velocity wall: the relative energy residual of the solution
    # returned by pyro_stokes_solve equals the one the solve reports, on two calls in a row
    stats = h.solve(en, ec, rho, (0.2, 1.0), 1e-10, *sol)
    assert stats.status == P.PYRO_OK
    free_before = None
    for k in range(2):
        st = residual_noalloc(nx, ny, Lx, Ly, bc, en, ec, rho, (0.2, 1.0), *sol, *r, rel_res)
        assert st == P.PYRO_OK
        torch.cuda.synchronize()
        assert float(rel_res[0]) == pytest.approx(stats.rel_energy_res, rel=1e-8)
        assert float(rel_res[1]) == pytest.approx(stats.rel_l2_res, rel=1e-8)
        free_now = torch.cuda.mem_get_info()[0]
        if free_before is not None:
            assert free_now == free_before   # no device memory taken by the call
        free_before = free_now


def test_noalloc_rejects_sizes_beyond_its_fixed_scratch_and_host_pointers():
    nx, ny = 4, 16380       # ny + 2 rows need 4096 row blocks: one more than the scratch holds
    f = [_zeros(ny, nx) for _ in range(9)]
    rel = torch.zeros(2, dtype=torch.float64)
    st = residual_noalloc(nx, ny, 1.0, 1.0, None, f[0], f[1], f[2], (0.0, 1.0), f[3], f[4], f[5], f[6], f[7], f[8], rel)
    assert st == -1
    g = [np.zeros((10, 10)) for _ in range(9)]
    st = residual_noalloc(8, 8, 1.0, 1.0, None, g[0], g[1], g[2], (0.0, 1.0), g[3], g[4], g[5], g[6], g[7], g[8], rel)
    assert st == -1
