"""Writes the stored FP64 reference solutions of the benchmark-size workloads.

Calls only oracle/ (and the seeded input generators of synth/): each solution is the oracle's
iterative reference (oracle/iterative.py: flexible GMRES with an exact sparse-LU velocity block,
certified by the true residual of the assembled system) at a relative energy residual <= 1e-13,
with the pressure mean removed. Files are compressed .npz with the unknown vector `x` (ordered
[vx, vy, p] as oracle.stokes.Grid numbers them), the achieved residuals and the workload recipe.

    python tests/golden/make_reference.py grf1024      # 1024 x 1024 random viscosity, seed 2
    python tests/golden/make_reference.py adjoint512   # 512 x 512 adjoint member 0 (forward solve)
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from oracle import stokes as S          # noqa: E402
from oracle import iterative as I       # noqa: E402
from synth import grf_config, adjoint_member, layered_config   # noqa: E402
from oracle import multigrid as M   # noqa: E402

G = (0.0, 1.0)
TOL = 1e-13

WORKLOADS = {
    "grf1024": ("1024 x 1024 cells, unit box, free slip, g = (0, 1); log10 eta = clipped Gaussian random field "
                "(corr 0.05, [-2, 2]), seed 2; rho = 1 + 32 density inclusions", lambda: grf_config(1024, 1024, seed=2)),
    "adjoint512": ("512 x 512 cells, unit box, free slip, g = (0, 1); adjoint member 0 (log10 eta random field seed 500, "
                   "rho as the random-field workload)", lambda: adjoint_member(0, 512, 512)[0]),
    "layered1024": ("1024 x 1024 cells, unit box, free slip, g = (0, 1); the layered workload's recipe (lid 1e6 over the "
                    "top 10 %, mantle 1 +- 50 %, 64 inclusions eta 10^U[-3,3]), seed 3; pressure block of the reference "
                    "solve: weighted BFBt", lambda: layered_config(1024, 1024, seed=3)),
}
SCHUR = {"layered1024": True}


def path_of(name):
    return os.path.join(HERE, f"reference_{name}.npz")


def make(name):
    recipe, gen = WORKLOADS[name]
    f = gen()
    g = S.Grid(f.nx, f.ny, f.Lx, f.Ly)
    sysm = S.assemble(g, f.eta_n, f.eta_c, f.rho, G)
    t = time.time()
    schur = M.WeightedBFBt(sysm) if SCHUR.get(name) else None
    res = I.solve_reference(sysm, f.eta_c, tol=TOL, verbose=True, schur=schur, m=200 if schur is not None else 100)
    print(f"{name}: {res.iterations} iterations, rel energy {res.rel_energy:.3e}, l2 {res.rel_l2:.3e}, "
          f"{time.time() - t:.0f} s", flush=True)
    assert res.rel_energy <= TOL
    np.savez_compressed(path_of(name), x=res.x, rel_energy=res.rel_energy, rel_l2=res.rel_l2,
                        iterations=res.iterations, nx=f.nx, ny=f.ny, recipe=recipe)


if __name__ == "__main__":
    for name in sys.argv[1:] or list(WORKLOADS):
        make(name)
