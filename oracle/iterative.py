"""Plain FP64 CPU iterative reference solve of the discrete Stokes system.

TEST INFRASTRUCTURE ONLY: nothing on the product path imports this module. Only the tests, the
script that writes the stored reference solutions (``tests/golden/make_reference.py``) and the
CPU-baseline leg of ``bench.py`` use it.

Why it exists: the direct solve of ``oracle.stokes`` (SuperLU on the bordered saddle-point matrix)
does not reach the benchmark sizes in practical time (512 x 512 takes about 13 minutes, and the
factorisation grows faster than the unknown count). This module reaches the same answer — the
exact solution of the assembled system [[L, G], [D, 0]] [v; p] = [f; 0] with zero-mean pressure
(Eq. stokes_saddle, Eq. pressure_normalization) — by iteration, and certifies it by the true
residual recomputed from the assembled CSR matrix at every restart, never by a recursively updated
quantity. Its agreement with the direct solve is pinned in ``tests/test_oracle_iterative.py``.

Method (standard pieces, written plainly):
  * Krylov: restarted flexible GMRES (Saad, "A flexible inner-outer preconditioned GMRES
    algorithm", SIAM J. Sci. Comput. 14 (1993) 461-469), right-preconditioned, in the inner product
    weighted by the energy-norm weights of Sec. "Global Relative Energy Residual" (so each cycle
    minimises the residual the paper stops on); Arnoldi by modified Gram-Schmidt applied twice; the
    small (j+1) x j least-squares problem by numpy.linalg.lstsq.
  * Preconditioner: the block lower-triangular form z_v = L^-1 r_v with an EXACT sparse LU of the
    velocity block (SuperLU, minimum-degree ordering on L + L^T; no multigrid), then
    z_p = eta_c (r_p - D z_v) (the diagonal viscosity Schur surrogate of Sec. "Residual Norms") with
    its mean removed, or for the layered workload the oracle's weighted BFBt surrogate. It shares
    nothing with the GPU path; its answer is certified by the true residual either way.
"""
from dataclasses import dataclass, field

import numpy as np
import scipy.sparse.linalg as spla

from .stokes import energy_residual, pressure_weights


@dataclass
class IterativeResult:
    x: np.ndarray                 # unknown vector [vx, vy, p], pressure mean removed
    rel_energy: float             # true relative energy residual of x (oracle.stokes.energy_residual)
    rel_l2: float                 # true relative l2 residual of x
    iterations: int               # preconditioner applications
    history: list = field(default_factory=list)   # (iterations, true relative energy residual) per restart


def energy_weights(sysm, eta_c):
    """W of the energy inner product: 1 / diag(-L) on velocity rows (after boundary elimination),
    eta_c / (2/dx^2 + 2/dy^2) on continuity rows (Sec. "Global Relative Energy Residual")."""
    g = sysm.grid
    dL = -sysm.A.diagonal()[:g.n_v]
    return np.concatenate([1.0 / dL, pressure_weights(g, eta_c)])


def block_triangular_lu(sysm, eta_c, alpha=1.0, schur=None):
    """z = M^-1 r with z_v = L^-1 r_v (exact sparse LU), z_p = alpha eta_c (r_p - D z_v), mean removed;
    with `schur` (an object with .apply, e.g. multigrid.WeightedBFBt) z_p = alpha schur.apply(r_p - D z_v)."""
    g = sysm.grid
    nv = g.n_v
    A = sysm.A.tocsr()
    L = A[:nv, :nv].tocsc()
    D = A[nv:, :nv].tocsr()
    lu = spla.splu(L, permc_spec="MMD_AT_PLUS_A")
    ec = g.eta_c_at(eta_c, g.p_i, g.p_j)

    def apply(r):
        zv = lu.solve(r[:nv])
        y = r[nv:] - D @ zv
        zp = alpha * (schur.apply(y) if schur is not None else ec * y)
        zp -= zp.mean()
        return np.concatenate([zv, zp])
    return apply


def fgmres(sysm, eta_c, precond, tol=1e-13, m=100, max_iter=3000, x0=None, verbose=False):
    """Restarted right-preconditioned flexible GMRES(m) on A x = b in the energy inner product.

    Stops when the TRUE relative energy residual (recomputed from the CSR matrix at a restart)
    is <= tol, or after max_iter preconditioner applications. Within a cycle the Givens-free
    least-squares residual decides when to restart early (at tol / 4), so the final check is always
    a true residual."""
    A = sysm.A.tocsr()
    b = sysm.b
    g = sysm.grid
    W = energy_weights(sysm, eta_c)
    den = np.sqrt(np.sum(W[:g.n_v] * b[:g.n_v] ** 2))
    ip = lambda u, v: float(np.dot(W * u, v))
    x = np.zeros_like(b) if x0 is None else x0.copy()
    its, hist = 0, []
    while True:
        r = b - A @ x
        beta = np.sqrt(ip(r, r))
        hist.append((its, beta / den))
        if verbose:
            print(f"  fgmres restart at {its}: true rel energy residual {beta / den:.3e}", flush=True)
        if beta / den <= tol or its >= max_iter:
            break
        V = [r / beta]
        Z = []
        H = np.zeros((m + 1, m))
        y = np.zeros(0)
        for j in range(m):
            z = precond(V[j])
            Z.append(z)
            w = A @ z
            for _ in range(2):                      # modified Gram-Schmidt, applied twice
                for i in range(j + 1):
                    hij = ip(w, V[i])
                    H[i, j] += hij
                    w = w - hij * V[i]
            H[j + 1, j] = np.sqrt(ip(w, w))
            V.append(w / H[j + 1, j] if H[j + 1, j] > 0 else w)
            its += 1
            e1 = np.zeros(j + 2)
            e1[0] = beta
            y, *_ = np.linalg.lstsq(H[:j + 2, :j + 1], e1, rcond=None)
            est = np.linalg.norm(H[:j + 2, :j + 1] @ y - e1) / den
            if est <= 0.25 * tol or its >= max_iter or H[j + 1, j] == 0:
                break
        x = x + np.column_stack(Z[:len(y)]) @ y
    x = x.copy()
    x[g.n_v:] -= x[g.n_v:].mean()
    e, l2 = energy_residual(sysm, eta_c, x)
    return IterativeResult(x, e, l2, its, hist)


def solve_reference(sysm, eta_c, tol=1e-13, m=100, max_iter=3000, verbose=False, schur=None):
    """The iterative reference solution: FGMRES(m) preconditioned by the exact-velocity block
    lower-triangular preconditioner, to a true relative energy residual <= tol. `schur` replaces the
    diagonal viscosity surrogate of the pressure block (for viscosity contrasts of 1e9, where the
    surrogate needs thousands of iterations)."""
    return fgmres(sysm, eta_c, block_triangular_lu(sysm, eta_c, schur=schur), tol=tol, m=m, max_iter=max_iter,
                  verbose=verbose)
