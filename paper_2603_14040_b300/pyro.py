"""ctypes binding of libpyro (include/pyro.h): argument marshalling only.

Every computation runs in the library's CUDA kernels. Arrays may be torch tensors (CUDA or CPU,
float64, contiguous, shape (ny+2, nx+2)) or numpy float64 arrays; their data pointers are passed
as they are (the library detects host vs device pointers). There is no CPU fallback: importing
this module fails if libpyro.so is missing.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "libpyro.so")

PYRO_OK, PYRO_W_NOT_CONVERGED = 0, 1
ACCEL_FGMRES, ACCEL_GCR, ACCEL_ANDERSON = 0, 1, 2
SMOOTH_RBGS, SMOOTH_JACOBI, SMOOTH_RAS, SMOOTH_MIXED = 0, 1, 2, 3
PYRO_E_INVALID, PYRO_E_NOMEM, PYRO_E_CUDA, PYRO_E_NONFINITE, PYRO_E_TIMEOUT, PYRO_E_BREAKDOWN = -1, -2, -3, -4, -5, -6
FREE_SLIP, NO_SLIP, PERIODIC, VELOCITY = 0, 1, 2, 3
PREC_FP64, PREC_MIXED = 0, 1
ETA_ARITH, ETA_GEOM = 0, 1


class PyroBC(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int * 4), ("vt", ctypes.c_double * 4)]


class PyroOpts(ctypes.Structure):
    _fields_ = [("nu1", ctypes.c_int), ("nu2", ctypes.c_int), ("omega_v", ctypes.c_double),
                ("alpha_p", ctypes.c_double), ("restart_m", ctypes.c_int), ("max_iter", ctypes.c_int),
                ("prec", ctypes.c_int), ("coarsest_min", ctypes.c_int), ("eta_coarsen", ctypes.c_int),
                ("warm_start", ctypes.c_int), ("use_graphs", ctypes.c_int), ("timeout_s", ctypes.c_double),
                ("kcycle", ctypes.c_int), ("cluster_cells", ctypes.c_int), ("tile_fusion", ctypes.c_int),
                ("tile_sweeps", ctypes.c_int), ("tile_fusion64", ctypes.c_int), ("accel", ctypes.c_int),
                ("aa_beta", ctypes.c_double), ("smoother", ctypes.c_int), ("ras_inner", ctypes.c_int),
                ("litho_guess", ctypes.c_int), ("cont_stages", ctypes.c_int), ("cont_iters", ctypes.c_int),
                ("coarse_sweeps", ctypes.c_int), ("coarsen_ratio", ctypes.c_double),
                ("coarsen_general", ctypes.c_int), ("gram_schmidt", ctypes.c_int), ("schur", ctypes.c_int),
                ("galerkin", ctypes.c_int), ("inner_cg", ctypes.c_int), ("res64", ctypes.c_int)]


class PyroStats(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("restarts", ctypes.c_int), ("vcycles", ctypes.c_int),
                ("status", ctypes.c_int), ("rel_energy_res", ctypes.c_double), ("rel_l2_res", ctypes.c_double),
                ("t_setup_ms", ctypes.c_double), ("t_solve_ms", ctypes.c_double), ("alg_bytes", ctypes.c_double),
                ("levels", ctypes.c_int), ("coarse_n", ctypes.c_int), ("kernel_launches", ctypes.c_longlong)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


EXPORTED = ["pyro_default_opts", "pyro_stokes_create", "pyro_stokes_footprint", "pyro_stokes_apply",
            "pyro_stokes_solve", "pyro_stokes_precond", "pyro_stokes_set_timing", "pyro_stokes_get_timing",
            "pyro_stokes_residual_noalloc", "pyro_stokes_adjoint", "pyro_stokes_destroy", "pyro_strerror", "pyro_version",
            "pyro_markers_create", "pyro_markers_to_grid", "pyro_grid_to_markers", "pyro_markers_advect",
            "pyro_markers_max_dt", "pyro_markers_destroy"]


def load_library(path=_LIB_PATH):
    if not os.path.exists(path):
        raise ImportError(f"libpyro.so not built ({path}); run paper_2603_14040_b300._build.build()")
    lib = ctypes.CDLL(path)
    P, D, I, S = ctypes.c_void_p, ctypes.c_double, ctypes.c_int, ctypes.c_size_t
    lib.pyro_default_opts.argtypes = [ctypes.POINTER(PyroOpts)]
    lib.pyro_default_opts.restype = None
    lib.pyro_stokes_create.argtypes = [I, I, D, D, ctypes.POINTER(PyroBC), ctypes.POINTER(PyroOpts), ctypes.POINTER(P)]
    lib.pyro_stokes_create.restype = I
    lib.pyro_stokes_footprint.argtypes = [I, I, ctypes.POINTER(PyroOpts)]
    lib.pyro_stokes_footprint.restype = S
    lib.pyro_stokes_apply.argtypes = [P] * 9 + [P]
    lib.pyro_stokes_apply.restype = I
    lib.pyro_stokes_solve.argtypes = [P, P, P, P, D, D, D, P, P, P, ctypes.POINTER(PyroStats), P]
    lib.pyro_stokes_solve.restype = I
    lib.pyro_stokes_set_timing.argtypes = [P, I]
    lib.pyro_stokes_set_timing.restype = I
    lib.pyro_stokes_get_timing.argtypes = [P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_longlong)]
    lib.pyro_stokes_get_timing.restype = I
    lib.pyro_stokes_residual_noalloc.argtypes = [I, I, D, D, ctypes.POINTER(PyroBC), P, P, P, D, D, P, P, P, P, P, P,
                                                 P, P]
    lib.pyro_stokes_residual_noalloc.restype = I
    lib.pyro_stokes_precond.argtypes = [P] * 9 + [P]
    lib.pyro_stokes_precond.restype = I
    lib.pyro_stokes_adjoint.argtypes = [P, P, P, P, D, P, P, P, ctypes.POINTER(PyroStats), P]
    lib.pyro_stokes_adjoint.restype = I
    lib.pyro_stokes_destroy.argtypes = [P]
    lib.pyro_stokes_destroy.restype = None
    lib.pyro_strerror.argtypes = [I]
    lib.pyro_strerror.restype = ctypes.c_char_p
    lib.pyro_version.argtypes = []
    lib.pyro_version.restype = ctypes.c_char_p
    lib.pyro_markers_create.argtypes = [I, I, D, D, ctypes.c_longlong, ctypes.POINTER(P)]
    lib.pyro_markers_create.restype = I
    lib.pyro_markers_to_grid.argtypes = [P, I, ctypes.c_longlong, P, P, P, P, P, P]
    lib.pyro_markers_to_grid.restype = I
    lib.pyro_grid_to_markers.argtypes = [P, I, ctypes.c_longlong, P, P, P, P, P]
    lib.pyro_grid_to_markers.restype = I
    lib.pyro_markers_advect.argtypes = [P, I, ctypes.c_longlong, P, P, P, P, D, I, P]
    lib.pyro_markers_advect.restype = I
    lib.pyro_markers_max_dt.argtypes = [P, P, P, D, ctypes.POINTER(D), P]
    lib.pyro_markers_max_dt.restype = I
    lib.pyro_markers_destroy.argtypes = [P]
    lib.pyro_markers_destroy.restype = None
    lib.pyro_fp64_fma_rate.argtypes = [I, ctypes.POINTER(D), P]
    lib.pyro_fp64_fma_rate.restype = I
    return lib


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = load_library()
    return _lib


class PyroError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        super().__init__(f"{where}: {lib().pyro_strerror(status).decode()} (status {status})")


def default_opts(**kw):
    o = PyroOpts()
    lib().pyro_default_opts(ctypes.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


def make_bc(kind=(FREE_SLIP,) * 4, vt=(0.0,) * 4):
    b = PyroBC()
    for k in range(4):
        b.kind[k] = int(kind[k])
        b.vt[k] = float(vt[k])
    return b


def _count(a):
    """Element count of a torch tensor or numpy array."""
    return int(a.numel()) if hasattr(a, "numel") else int(a.size)


def _ptr(a, shape=None, writable=False):
    """Data pointer of a float64 contiguous torch tensor or numpy array (None -> NULL)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if a.dtype != np.float64 or not a.flags["C_CONTIGUOUS"]:
            raise TypeError("numpy arrays must be C-contiguous float64")
        if shape is not None and a.shape != shape:
            raise ValueError(f"expected shape {shape}, got {a.shape}")
        return a.ctypes.data
    import torch
    if not isinstance(a, torch.Tensor):
        raise TypeError(f"unsupported array type {type(a)}")
    if a.dtype != torch.float64 or not a.is_contiguous():
        raise TypeError("tensors must be contiguous float64")
    if shape is not None and tuple(a.shape) != shape:
        raise ValueError(f"expected shape {shape}, got {tuple(a.shape)}")
    return a.data_ptr()


def _stream_handle(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except ImportError:
            pass
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def footprint(nx, ny, opts=None):
    return int(lib().pyro_stokes_footprint(nx, ny, ctypes.byref(opts) if opts is not None else None))


def fp64_fma_rate(iters=4096, stream=None):
    """pyro_fp64_fma_rate: measured FP64 FMA rate of the current GPU in TFLOP/s."""
    out = ctypes.c_double(0.0)
    st = lib().pyro_fp64_fma_rate(int(iters), ctypes.byref(out), _stream_handle(stream))
    if st < 0:
        raise PyroError(st, "pyro_fp64_fma_rate")
    return out.value


def residual_noalloc(nx, ny, Lx, Ly, bc, eta_n, eta_c, rho, g, vx, vy, p, r_vx, r_vy, r_p, rel_res, stream=None):
    """pyro_stokes_residual_noalloc: residual and relative energy / l2 residuals without any device
    allocation (for callers that cannot allocate; see include/pyro.h). All fields must be CUDA
    tensors; rel_res is a float64 array of 2 (host or device). Returns the status code."""
    s = (ny + 2, nx + 2)
    return lib().pyro_stokes_residual_noalloc(int(nx), int(ny), float(Lx), float(Ly),
                                              ctypes.byref(bc if bc is not None else make_bc()),
                                              _ptr(eta_n, s), _ptr(eta_c, s), _ptr(rho, s), float(g[0]),
                                              float(g[1]), _ptr(vx, s), _ptr(vy, s), _ptr(p, s), _ptr(r_vx, s),
                                              _ptr(r_vy, s), _ptr(r_p, s), _ptr(rel_res), _stream_handle(stream))


LATTICE_NODES, LATTICE_CELLS, LATTICE_VX, LATTICE_VY = 0, 1, 2, 3
ADVECT_EULER, ADVECT_HEUN, ADVECT_RK4, ADVECT_TAYLOR = 0, 1, 2, 3


class Markers:
    """Marker workspace (pyro_markers): marker <-> grid interpolation and marker advection; CUDA
    float64 tensors in and out."""

    def __init__(self, nx, ny, Lx=1.0, Ly=1.0, max_markers=1):
        self.nx, self.ny, self.Lx, self.Ly = int(nx), int(ny), float(Lx), float(Ly)
        h = ctypes.c_void_p()
        st = lib().pyro_markers_create(self.nx, self.ny, self.Lx, self.Ly, int(max_markers), ctypes.byref(h))
        if st != PYRO_OK:
            raise PyroError(st, "pyro_markers_create")
        self._h = h
        self.shape = (self.ny + 2, self.nx + 2)

    def to_grid(self, lattice, xm, ym, phim, grid, wsum=None, stream=None):
        n = _count(xm)
        st = lib().pyro_markers_to_grid(self._h, int(lattice), n, _ptr(xm, (n,)), _ptr(ym, (n,)), _ptr(phim, (n,)),
                                        _ptr(grid, self.shape), _ptr(wsum, self.shape) if wsum is not None else None,
                                        _stream_handle(stream))
        if st < 0:
            raise PyroError(st, "pyro_markers_to_grid")
        return st

    def to_markers(self, lattice, xm, ym, grid, phim, stream=None):
        n = _count(xm)
        st = lib().pyro_grid_to_markers(self._h, int(lattice), n, _ptr(xm, (n,)), _ptr(ym, (n,)),
                                        _ptr(grid, self.shape), _ptr(phim, (n,)), _stream_handle(stream))
        if st < 0:
            raise PyroError(st, "pyro_grid_to_markers")
        return st

    def advect(self, xm, ym, vx, vy, dt, scheme=ADVECT_RK4, substeps=1, stream=None):
        """Move the markers (xm, ym updated in place) through dt in the velocity (vx, vy)."""
        n = _count(xm)
        st = lib().pyro_markers_advect(self._h, int(scheme), n, _ptr(xm, (n,)), _ptr(ym, (n,)), _ptr(vx, self.shape),
                                       _ptr(vy, self.shape), float(dt), int(substeps), _stream_handle(stream))
        if st < 0:
            raise PyroError(st, "pyro_markers_advect")
        return st

    def max_dt(self, vx, vy, cfl=0.5, stream=None):
        """cfl * min(dx / max|vx|, dy / max|vy|) (inf for a zero velocity)."""
        out = ctypes.c_double(0.0)
        st = lib().pyro_markers_max_dt(self._h, _ptr(vx, self.shape), _ptr(vy, self.shape), float(cfl),
                                       ctypes.byref(out), _stream_handle(stream))
        if st < 0:
            raise PyroError(st, "pyro_markers_max_dt")
        return out.value

    def close(self):
        if getattr(self, "_h", None):
            lib().pyro_markers_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Stokes:
    """One solver handle (pyro_stokes): resident hierarchy and Krylov workspace for an nx x ny grid."""

    def __init__(self, nx, ny, Lx=1.0, Ly=1.0, bc=None, opts=None, **opt_kw):
        self.nx, self.ny, self.Lx, self.Ly = int(nx), int(ny), float(Lx), float(Ly)
        self.opts = opts if opts is not None else default_opts(**opt_kw)
        self.bc = bc if bc is not None else make_bc()
        h = ctypes.c_void_p()
        st = lib().pyro_stokes_create(self.nx, self.ny, self.Lx, self.Ly, ctypes.byref(self.bc),
                                      ctypes.byref(self.opts), ctypes.byref(h))
        if st != PYRO_OK:
            raise PyroError(st, "pyro_stokes_create")
        self._h = h
        self.shape = (self.ny + 2, self.nx + 2)

    def close(self):
        if getattr(self, "_h", None):
            lib().pyro_stokes_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def apply(self, eta_n, eta_c, vx, vy, p, Ax, Ay, Ap, stream=None):
        s = self.shape
        st = lib().pyro_stokes_apply(self._h, _ptr(eta_n, s), _ptr(eta_c, s), _ptr(vx, s), _ptr(vy, s), _ptr(p, s),
                                     _ptr(Ax, s), _ptr(Ay, s), _ptr(Ap, s), _stream_handle(stream))
        if st < 0:
            raise PyroError(st, "pyro_stokes_apply")
        return st

    def solve(self, eta_n, eta_c, rho, g, tol, vx, vy, p, stream=None, raise_on_warning=False):
        s = self.shape
        stats = PyroStats()
        st = lib().pyro_stokes_solve(self._h, _ptr(eta_n, s), _ptr(eta_c, s), _ptr(rho, s), float(g[0]), float(g[1]),
                                     float(tol), _ptr(vx, s), _ptr(vy, s), _ptr(p, s), ctypes.byref(stats),
                                     _stream_handle(stream))
        if st < 0 or (raise_on_warning and st > 0):
            raise PyroError(st, "pyro_stokes_solve")
        return stats

    TIMING_PHASES = ("precond_in", "l0_pre_smooth", "coarse_levels", "l0_post_smooth", "pressure_and_apply",
                     "orthogonalise")

    def set_timing(self, enable=True):
        lib().pyro_stokes_set_timing(self._h, 1 if enable else 0)

    def get_timing(self):
        ms = (ctypes.c_double * 6)()
        cnt = (ctypes.c_longlong * 2)()
        lib().pyro_stokes_get_timing(self._h, ms, cnt)
        return dict(zip(self.TIMING_PHASES, list(ms))), {"iterations": cnt[0], "l0_sweeps": cnt[1]}

    def precond(self, eta_n, eta_c, r_vx, r_vy, r_p, z_vx, z_vy, z_p, stream=None):
        s = self.shape
        st = lib().pyro_stokes_precond(self._h, _ptr(eta_n, s), _ptr(eta_c, s), _ptr(r_vx, s), _ptr(r_vy, s),
                                       _ptr(r_p, s), _ptr(z_vx, s), _ptr(z_vy, s), _ptr(z_p, s),
                                       _stream_handle(stream))
        if st < 0:
            raise PyroError(st, "pyro_stokes_precond")
        return st

    def adjoint(self, dJ_dvx, dJ_dvy, dJ_dp, tol, dJ_deta_n, dJ_deta_c, dJ_drho=None, stream=None):
        s = self.shape
        stats = PyroStats()
        st = lib().pyro_stokes_adjoint(self._h, _ptr(dJ_dvx, s), _ptr(dJ_dvy, s), _ptr(dJ_dp, s), float(tol),
                                       _ptr(dJ_deta_n, s), _ptr(dJ_deta_c, s), _ptr(dJ_drho, s),
                                       ctypes.byref(stats), _stream_handle(stream))
        if st < 0:
            raise PyroError(st, "pyro_stokes_adjoint")
        return stats
