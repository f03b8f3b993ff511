"""Seeded synthetic material fields on the fully staggered grid.

Layout (the paper's uniform padded staggered arrays, Sec. "Staggered Grid Layout"): with nx, ny
CELL counts every field is a row-major (ny+2) x (nx+2) float64 array. Basic nodes (eta_n, rho)
hold meaningful values at i in [0, ny], j in [0, nx]; cell centres (eta_c, p) at i in [1, ny],
j in [1, nx]. Row 0 is the top of the box (y = 0) and y grows with the row index.

Every continuous material field is point-sampled on a half-spacing lattice of (2ny+1) x (2nx+1)
points: lattice point (a, b) sits at (x, y) = (b*hx/2, a*hy/2). Basic node (i, j) is lattice
point (2i, 2j); the centre of cell (i, j) is lattice point (2i-1, 2j-1). So eta_n and eta_c
are samples of one and the same continuous field.
"""
from dataclasses import dataclass
import numpy as np


@dataclass
class Fields:
    nx: int
    ny: int
    Lx: float
    Ly: float
    eta_n: np.ndarray
    eta_c: np.ndarray
    rho: np.ndarray


def _lattice_xy(nx, ny, Lx, Ly):
    x = np.arange(2 * nx + 1) * (Lx / nx / 2.0)
    y = np.arange(2 * ny + 1) * (Ly / ny / 2.0)
    return x, y


def sample_lattice_to_fields(eta_s, rho_s, nx, ny, Lx=1.0, Ly=1.0):
    """Split half-spacing lattice samples into the padded node / cell arrays."""
    eta_n = np.zeros((ny + 2, nx + 2))
    eta_c = np.zeros((ny + 2, nx + 2))
    rho = np.zeros((ny + 2, nx + 2))
    eta_n[:ny + 1, :nx + 1] = eta_s[0::2, 0::2]
    rho[:ny + 1, :nx + 1] = rho_s[0::2, 0::2]
    eta_c[1:ny + 1, 1:nx + 1] = eta_s[1::2, 1::2]
    return Fields(nx, ny, Lx, Ly, eta_n, eta_c, rho)


def _paint_disc(arr, x, y, cx, cy, r, value):
    """Set arr to value where |(x, y) - (cx, cy)| <= r (later calls overwrite earlier ones)."""
    j0 = max(int(np.searchsorted(x, cx - r)) - 1, 0)
    j1 = min(int(np.searchsorted(x, cx + r)) + 1, len(x))
    i0 = max(int(np.searchsorted(y, cy - r)) - 1, 0)
    i1 = min(int(np.searchsorted(y, cy + r)) + 1, len(y))
    if j1 <= j0 or i1 <= i0:
        return
    xx = x[None, j0:j1]
    yy = y[i0:i1, None]
    inside = (xx - cx) ** 2 + (yy - cy) ** 2 <= r * r
    sub = arr[i0:i1, j0:j1]
    if callable(value):
        sub[inside] = value(sub[inside])
    else:
        sub[inside] = value


def sinker(nx=64, ny=64, Lx=1.0, Ly=1.0, eta_bg=1.0, rho_bg=1.0, eta_inc=1e3, rho_inc=1.1,
           r=0.1, cx=None, cy=None):
    """One centred circular inclusion in a uniform matrix (the sinker benchmark, scaled down)."""
    x, y = _lattice_xy(nx, ny, Lx, Ly)
    eta_s = np.full((2 * ny + 1, 2 * nx + 1), eta_bg)
    rho_s = np.full((2 * ny + 1, 2 * nx + 1), rho_bg)
    cx = 0.5 * Lx if cx is None else cx
    cy = 0.5 * Ly if cy is None else cy
    _paint_disc(eta_s, x, y, cx, cy, r, eta_inc)
    _paint_disc(rho_s, x, y, cx, cy, r, rho_inc)
    return sample_lattice_to_fields(eta_s, rho_s, nx, ny, Lx, Ly)


def random_field_log10(nx, ny, seed, corr_len=0.05, Lx=1.0, Ly=1.0, clip=2.0):
    """Gaussian random field on the half-spacing lattice: white noise filtered in Fourier space by
    exp(-(k*corr_len)^2 / 8), i.e. a Gaussian covariance exp(-r^2 / corr_len^2) (up to the
    periodic wrap of the FFT box), normalised to zero mean / unit std and clipped to [-clip, clip]."""
    rng = np.random.default_rng(seed)
    shape = (2 * ny + 1, 2 * nx + 1)
    noise = rng.standard_normal(shape)
    ky = 2 * np.pi * np.fft.fftfreq(shape[0], d=Ly / ny / 2.0)
    kx = 2 * np.pi * np.fft.rfftfreq(shape[1], d=Lx / nx / 2.0)
    k2 = ky[:, None] ** 2 + kx[None, :] ** 2
    filt = np.exp(-k2 * corr_len ** 2 / 8.0)
    f = np.fft.irfft2(np.fft.rfft2(noise) * filt, s=shape)
    f -= f.mean()
    std = f.std()
    if std > 0:
        f /= std
    return np.clip(f, -clip, clip)


def random_inclusions_density(rho_s, x, y, rng, count, rmin, rmax, rho_lo, rho_hi, Lx=1.0, Ly=1.0):
    for _ in range(count):
        r = rng.uniform(rmin, rmax)
        cx = rng.uniform(r, Lx - r)
        cy = rng.uniform(r, Ly - r)
        val = rng.uniform(rho_lo, rho_hi)
        _paint_disc(rho_s, x, y, cx, cy, r, val)


def grf_config(nx=1024, ny=1024, seed=2, n_inc=32, Lx=1.0, Ly=1.0):
    """Random-field viscosity (log10 eta a clipped Gaussian random field, correlation length 0.05)
    with a unit background density and n_inc density-only inclusions r~U[0.01,0.05], rho~U[0.9,1.1]."""
    x, y = _lattice_xy(nx, ny, Lx, Ly)
    eta_s = 10.0 ** random_field_log10(nx, ny, seed, Lx=Lx, Ly=Ly)
    rho_s = np.ones_like(eta_s)
    rng = np.random.default_rng(seed + 1_000_003)
    random_inclusions_density(rho_s, x, y, rng, n_inc, 0.01, 0.05, 0.9, 1.1, Lx, Ly)
    return sample_lattice_to_fields(eta_s, rho_s, nx, ny, Lx, Ly)


def layered_config(nx=4096, ny=4096, seed=3, n_inc=64, Lx=1.0, Ly=1.0):
    """Stiff lid (eta=1e6 for y<0.1*Ly) over a mantle eta=1+0.5u, u~U[-1,1] i.i.d. per lattice point,
    plus n_inc inclusions with eta=10^U[-3,3], rho=1+U[-0.05,0.05], r~U[0.01,0.05]."""
    rng = np.random.default_rng(seed)
    x, y = _lattice_xy(nx, ny, Lx, Ly)
    eta_s = 1.0 + 0.5 * rng.uniform(-1.0, 1.0, size=(2 * ny + 1, 2 * nx + 1))
    eta_s[y < 0.1 * Ly, :] = 1e6
    rho_s = np.ones_like(eta_s)
    for _ in range(n_inc):
        r = rng.uniform(0.01, 0.05)
        cx = rng.uniform(r, Lx - r)
        cy = rng.uniform(r, Ly - r)
        e = 10.0 ** rng.uniform(-3.0, 3.0)
        d = 1.0 + rng.uniform(-0.05, 0.05)
        _paint_disc(eta_s, x, y, cx, cy, r, e)
        _paint_disc(rho_s, x, y, cx, cy, r, d)
    return sample_lattice_to_fields(eta_s, rho_s, nx, ny, Lx, Ly)


def serving_request(req_id, base_seed=4, sizes=(128, 256, 512, 1024, 2048), aspects=(1, 2, 4),
                    n_inc=16, force_n=None, force_a=None):
    """One serving request: ny=n, nx=a*n (square cells, Lx=a, Ly=1), background eta=rho=1 and
    n_inc inclusions (r~U[0.02,0.08]) of viscosity C=10^U[2,6] and density 1.05."""
    rng = np.random.default_rng(base_seed * 1_000_000 + req_id)
    n = int(rng.choice(sizes)) if force_n is None else force_n
    a = int(rng.choice(aspects)) if force_a is None else force_a
    contrast = 10.0 ** rng.uniform(2.0, 6.0)
    nx, ny, Lx, Ly = a * n, n, float(a), 1.0
    x, y = _lattice_xy(nx, ny, Lx, Ly)
    eta_s = np.ones((2 * ny + 1, 2 * nx + 1))
    rho_s = np.ones_like(eta_s)
    for _ in range(n_inc):
        r = rng.uniform(0.02, 0.08)
        cx = rng.uniform(r, Lx - r)
        cy = rng.uniform(r, Ly - r)
        _paint_disc(eta_s, x, y, cx, cy, r, contrast)
        _paint_disc(rho_s, x, y, cx, cy, r, 1.05)
    f = sample_lattice_to_fields(eta_s, rho_s, nx, ny, Lx, Ly)
    return f, contrast


def adjoint_member(b, nx=512, ny=512, seed0=500, pert_seed0=600):
    """Member b of the adjoint batch: log10 eta a clipped random field (seed seed0+b), density as in
    the random-field workload, and the perturbed field eta*10^(0.1*xi) whose surface velocity is
    the observation (xi an independent random field, seed pert_seed0+b)."""
    x, y = _lattice_xy(nx, ny, 1.0, 1.0)
    l10 = random_field_log10(nx, ny, seed0 + b)
    rho_s = np.ones_like(l10)
    rng = np.random.default_rng(seed0 + b + 1_000_003)
    random_inclusions_density(rho_s, x, y, rng, 32, 0.01, 0.05, 0.9, 1.1)
    xi = random_field_log10(nx, ny, pert_seed0 + b)
    base = sample_lattice_to_fields(10.0 ** l10, rho_s, nx, ny)
    pert = sample_lattice_to_fields(10.0 ** (l10 + 0.1 * xi), rho_s, nx, ny)
    return base, pert


def random_vectors(nx, ny, seed, scale=1.0):
    """Random (vx, vy, p) padded arrays (all entries, ghosts included) for operator tests."""
    rng = np.random.default_rng(seed)
    return tuple(scale * rng.standard_normal((ny + 2, nx + 2)) for _ in range(3))
