/*
 * pyro.h — C ABI of libpyro: matrix-free staggered-grid 2D variable-viscosity Stokes solver for
 * one NVIDIA B300 (sm_103a).
 *
 * The operator is the stress-conservative finite-difference discretisation of the incompressible
 * Stokes equations on a fully staggered grid (paper: Sec. "Conservation of Mass and Momentum",
 * eqs. xmom/ymom/mass; Sec. "Staggered Grid Layout"; Sec. "Stress-Conservative Finite
 * Differences"). The solve is flexible GMRES (Sec. "Comparison with FGMRES") preconditioned by one
 * Uzawa sweep (Sec. "Uzawa Iteration as a Fixed Point Method", eq. uzawa_split_system) whose
 * velocity block is one geometric-multigrid V-cycle (Sec. "Multigrid Cycles", eq.
 * multigrid_levels) with damped red-black Gauss-Seidel smoothing (Sec. "Smoothers", eq.
 * sor_update). Convergence is measured by the relative energy residual of Sec. "Global Relative
 * Energy Residual".
 *
 * ---------------------------------------------------------------------------------------------
 * GRID AND ARRAY LAYOUT (every field argument)
 *   nx, ny are CELL counts; hx = Lx/nx, hy = Ly/ny. Every field is a row-major array of
 *   (ny+2) x (nx+2) doubles (the paper's (n_y+1) x (n_x+1) in node counts); element (i, j) is at
 *   offset i*(nx+2) + j. Row 0 is the top (y = 0); y and the row index grow downward. Each
 *   staggered quantity carries the index of the basic node at its lower-right (paper's rule):
 *     vx(i,j) at (j*hx, (i-1/2)*hy)      meaningful i in [1,ny], j in [0,nx]; unknowns j in [1,nx-1]
 *     vy(i,j) at ((j-1/2)*hx, i*hy)      meaningful i in [0,ny], j in [1,nx]; unknowns i in [1,ny-1]
 *     p(i,j), eta_c(i,j) at cell centres meaningful i in [1,ny], j in [1,nx]
 *     eta_n(i,j), rho(i,j) at basic nodes meaningful i in [0,ny], j in [0,nx]
 *   Entries outside the meaningful ranges are ignored on input. On output, velocity ghosts and
 *   walls are written with the boundary values; other non-meaningful entries are written as 0.
 *
 * POINTERS
 *   Field pointers may be device pointers or host pointers (pageable or pinned); the library
 *   detects which with cudaPointerGetAttributes. Host buffers are staged through the handle's own
 *   device workspace with copies ordered on `cuda_stream`. A device pointer must belong to the
 *   handle's device (the current device for calls without a handle) or be managed memory; memory
 *   of another GPU is rejected with PYRO_E_INVALID. The caller owns every buffer.
 *   `cuda_stream` is a cudaStream_t (NULL = legacy default stream).
 *
 * STATUS CODES: 0 = success; > 0 warning with a valid best-effort result; < 0 error (outputs
 *   undefined). No C++ exception crosses this interface. A handle is not thread-safe; distinct
 *   handles are independent and may be used from different host threads and streams.
 *
 * SYNCHRONISATION: pyro_stokes_solve and pyro_stokes_adjoint drive the Krylov loop from the host
 *   and return when the result is complete on `cuda_stream` (they synchronise that stream).
 *   pyro_stokes_apply and pyro_stokes_precond also return after completion (they read an error flag).
 * ---------------------------------------------------------------------------------------------
 */
#ifndef PYRO_H
#define PYRO_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PYRO_OK 0
#define PYRO_W_NOT_CONVERGED 1   /* max_iter reached; best iterate returned */
#define PYRO_E_INVALID (-1)      /* bad argument, unsupported size or boundary combination */
#define PYRO_E_NOMEM (-2)        /* device allocation failed (or the handle's memory budget) */
#define PYRO_E_CUDA (-3)         /* a CUDA runtime call failed */
#define PYRO_E_NONFINITE (-4)    /* an input field holds NaN/Inf, or the iteration produced one */
#define PYRO_E_TIMEOUT (-5)      /* wall-clock limit of the solve exceeded */
#define PYRO_E_BREAKDOWN (-6)    /* Krylov breakdown that a restart could not cure */

/* Boundary kinds per side (paper Sec. "Boundary Conditions", eqs. free_slip_bc, no_slip_bc).
 * The normal velocity is zero on every wall. The tangential ghost is eliminated with
 * ghost = s * interior + c: free slip s=+1, c=0; no slip s=-1, c=0 (the paper's mirror rule);
 * prescribed tangential velocity U: s=-1, c=2U. PYRO_BC_PERIODIC is accepted by the oracle only;
 * the library rejects it with PYRO_E_INVALID. */
typedef enum { PYRO_BC_FREE_SLIP = 0, PYRO_BC_NO_SLIP = 1, PYRO_BC_PERIODIC = 2, PYRO_BC_VELOCITY = 3 } pyro_bc_kind;

/* Sides are ordered W, E, N (top, row 0), S (bottom). vt = tangential velocity for VELOCITY. */
typedef struct {
  int kind[4];
  double vt[4];
} pyro_bc;

typedef enum { PYRO_PREC_FP64 = 0, PYRO_PREC_MIXED = 1 } pyro_precision;

/* Outer accelerator around the Uzawa/multigrid preconditioner M^-1 (every one stops on the
 * relative energy residual and recomputes the true FP64 residual before it stops):
 *   FGMRES   restarted flexible GMRES(m) in the energy inner product (Sec. "Comparison with
 *            FGMRES"; Arnoldi by classical Gram-Schmidt with one re-orthogonalisation);
 *   GCR      restarted flexible GCR(m) (Sec. "Generalized Conjugate Residual Method", Algorithm
 *            gcr) in the energy inner product; the paper's modified Gram-Schmidt is done as
 *            classical Gram-Schmidt with one re-orthogonalisation (equal in exact arithmetic);
 *   ANDERSON Anderson acceleration AA(m, aa_beta) of G(x) = x + M^-1 (b - A x) (Sec. "Anderson
 *            Acceleration", Algorithm anderson), least squares in the 2-norm, depth m =
 *            restart_m, x^1 = G(x^0). */
typedef enum { PYRO_ACCEL_FGMRES = 0, PYRO_ACCEL_GCR = 1, PYRO_ACCEL_ANDERSON = 2 } pyro_accel;

/* Velocity smoother of the V-cycle (Sec. "Smoothers"), damping omega_v for all three:
 *   RBGS    red-black Gauss-Seidel (eq. sor_update), colour order vx-red, vx-black, vy-red, vy-black;
 *   JACOBI  damped Jacobi sweeps of the coupled velocity block (eq. damped_jacobi); needs
 *           omega_v well below 1 (0.5-0.7) to smooth;
 *   RAS     RAS-type temporally blocked Jacobi (Algorithm ras_temporal): ceil(nu / ras_inner)
 *           passes over 32 x 32-cell tiles, each tile running ras_inner local damped Jacobi
 *           iterations in shared memory with its one-cell ring held at the pass-start values; the
 *           tiling shift of each pass comes from SplitMix64 of (level, pre/post, pass), so the
 *           V-cycle is the same linear operator at every application;
 *   MIXED   the "Mixed" configuration of the robustness study (Sec. "Numerical Stability and
 *           Solver Robustness"): JACOBI on the finest level, RAS on every coarser level. */
typedef enum { PYRO_SMOOTH_RBGS = 0, PYRO_SMOOTH_JACOBI = 1, PYRO_SMOOTH_RAS = 2, PYRO_SMOOTH_MIXED = 3 } pyro_smoother;
typedef enum { PYRO_ETA_ARITH = 0, PYRO_ETA_GEOM = 1 } pyro_eta_coarsening;

/* Solver options. pyro_default_opts() fills the defaults given in brackets. pyro_stokes_create
 * returns PYRO_E_INVALID (and pyro_stokes_footprint 0) when an option lies outside the range given
 * here; nothing is clamped or replaced. */
typedef struct {
  int nu1, nu2;          /* pre/post smoothing sweeps per level, >= 0 with nu1 + nu2 >= 1 [2, 2] */
  double omega_v;        /* velocity smoother damping (eq. sor_update), in (0, 2) [1.0] */
  double alpha_p;        /* Uzawa pressure relaxation alpha (eq. uzawa_iteration), > 0 [1.0] */
  int restart_m;         /* FGMRES / GCR restart length, Anderson depth; 1..256 [30] */
  int max_iter;          /* total outer iterations before PYRO_W_NOT_CONVERGED, >= 1 [500] */
  int prec;              /* pyro_precision [PYRO_PREC_MIXED] */
  int coarsest_min;      /* halve while the short side stays >= this many cells, >= 1 [4] */
  int eta_coarsen;       /* pyro_eta_coarsening [PYRO_ETA_ARITH] */
  int warm_start;        /* 1: vx, vy, p passed to solve hold the initial guess [0] */
  int use_graphs;        /* 1: capture the FGMRES iteration into a CUDA graph [1] */
  double timeout_s;      /* wall-clock limit of one solve, <= 0 for none [0] */
  int kcycle;            /* K-cycle depth 0..16: on levels l < kcycle the coarse correction is two
                            flexible-CG steps preconditioned by the next level's cycle (recursive
                            Krylov cycle, not in the paper; 0 = the paper's plain V-cycle) [0] */
  int cluster_cells;     /* reserved, must be <= 0: a sub-cycle running the small levels inside one
                            thread-block-cluster launch was measured to save nothing against the
                            graph-launched per-level kernels and was removed [0] */
  int tile_fusion;       /* 1: smoothing sweeps (with the prolongation) and residual+restriction run
                            as shared-memory tile kernels, one launch each per level visit (FP32
                            levels; FP64 levels see tile_fusion64); 4: as 1 with the 64 x 32
                            colour-split tiles on large levels instead of the warp-per-row tiles; 0:
                            one kernel per colour and step; 0, 1 or 4 [1] (a row-streaming wavefront
                            variant measured no faster than the tiles and was removed) */
  int tile_sweeps;       /* FP32 tile kernels: sweeps fused per launch, 1 (halo 4, one HBM pass per
                            sweep) or 2 (halo 8, one pass per two sweeps) [2] */
  int tile_fusion64;     /* 1: FP64 levels of up to 65536 cells also smooth and restrict with the
                            tile kernels; 0: every FP64 level runs one kernel per colour and step on
                            precomputed viscosity coefficients (B300's FP64 rate per SM is so low
                            that one CTA per tile becomes the critical path); 0 or 1 [0] */
  int accel;             /* pyro_accel: outer accelerator [PYRO_ACCEL_FGMRES] */
  double aa_beta;        /* Anderson mixing beta in (0, 1] (the paper suggests 0.5-0.8) [1.0] */
  int smoother;          /* pyro_smoother [PYRO_SMOOTH_RBGS] */
  int ras_inner;         /* RAS smoother: local Jacobi iterations per tile pass (T_inner), >= 1 [4] */
  int litho_guess;       /* 1: start the pressure from the lithostatic column integral of rho g_y
                            (Sec. "Viscosity Rescaling and Initial Guess"; cell pressures going down
                            differ by dy g_y times the vy-node density) when not warm-starting [0] */
  int cont_stages;       /* viscosity-contrast continuation (same section): > 0 runs cont_stages
                            stages with eta_comp = (1 - theta) eta_min + theta eta, theta = k /
                            cont_stages, each cont_iters outer iterations from the previous stage's
                            iterate, then the full-contrast solve; 0 = off; >= 0 [0] */
  int cont_iters;        /* outer iterations per continuation stage (the paper: 25), >= 1 [25] */
  int coarse_sweeps;     /* when the coarsest level has more than 1024 velocity unknowns (grids that
                            do not halve down far, e.g. odd sizes), this many smoothing sweeps from
                            zero stand in for its direct solve (Sec. "Multigrid Cycles": direct
                            method or a few smoothing iterations); >= 1 [40] */
  double coarsen_ratio;  /* 2: halve while possible; any other value in [1.5, 8] coarsens every level
                            by that ratio, n_c = ceil(n / ratio) (the paper's arbitrary ratio, e.g.
                            2.5) [2.0] */
  int coarsen_general;   /* 1: when halving stops with more than 1024 coarsest velocity unknowns
                            (odd sizes, few factors of 2), keep coarsening by coarsen_ratio with the
                            general transfer operators (normalised bilinear restriction, bilinear
                            prolongation at any ratio); 0: stop there [1] */
  int gram_schmidt;      /* FGMRES orthogonalisation in the W inner product: 0 classical Gram-Schmidt
                            with one full re-orthogonalisation (CGS2: two fused multi-dot /
                            multi-axpy passes over the basis); 1 modified Gram-Schmidt on the basis
                            stored scaled by W^(1/2) (one fused subtract-and-dot step per basis
                            vector, half the FP64 arithmetic of CGS2, j + 2 dependent steps for
                            column j); 2 modified when nx ny >= 2^19 cells, else classical (the
                            faster of the two on B300 either side); 0..2 [2] */
  int schur;             /* pressure block of the Uzawa preconditioner: 0 the paper's diagonal viscosity
                            surrogate, z_p = alpha_p eta_c (r_p - D z_v); 1 the weighted BFBt
                            approximation of the Schur complement (not in the paper; for viscosity
                            that jumps by many orders of magnitude), z_p = alpha_p K^-1 (D W^-1 (-L)
                            W^-1 G) K^-1 (r_p - D z_v) with K = D W^-1 G, W = diag(-L)^(1/2), each K^-1
                            one V-cycle of a smoothed-aggregation multigrid on the cell grid (2 x 2
                            aggregates, Galerkin coarse operators in a 5 x 5-box stencil, damped Jacobi
                            smoothing, dense coarsest inverse); 2 the same block computed in FP64 also
                            when the V-cycle is FP32 (mixed precision; in FP64 mode the same as 1);
                            0..2 [0] */
  int galerkin;          /* 1: every coarse level reached by halving takes the Galerkin operator R L P of
                            the level above it (the V-cycle's own restriction and prolongation; a
                            31-point stencil per velocity unknown) instead of the re-discretised
                            operator of the transferred viscosity, and is smoothed by damped Jacobi
                            (omega 0.6; red-black ordering does not decouple that stencil); the
                            finest level keeps its smoother. Not in the paper: for viscosity that
                            jumps by orders of magnitude within a coarse cell. Requires kcycle = 0
                            and cluster_cells <= 0; 0 or 1 [0] */
  int inner_cg;          /* velocity block of the preconditioner: 0 one V-cycle (the paper); k >= 1: k
                            steps of flexible conjugate gradients on L z_v = r_v from zero, each
                            preconditioned by one V-cycle (one-term flexible recurrence; the recurrence,
                            the operator and the dot products in FP64 in both precision modes, only the
                            V-cycle in FP32 in mixed mode; reduced on the device). Not in the paper: on
                            viscosity that jumps by orders
                            of magnitude a single cycle leaves most of the velocity error, and each
                            outer Krylov iteration saved also saves its orthogonalisation; 0..16 [0] */
  int res64;             /* mixed precision: 1 forms the finest level's V-cycle residual (the one the
                            restriction passes down) in FP64, from the FP32 iterate and right-hand side
                            with the FP64 outer operator, and rounds it to FP32 once; smoothing stays
                            FP32. Not in the paper: where viscosity jumps by many orders of magnitude
                            the FP32 residual cancels terms of eta / h^2. Takes effect when the first
                            coarsening halves the grid (otherwise the FP32 residual is kept); ignored
                            in FP64 mode; 0 or 1 [0] */
} pyro_opts;

typedef struct {
  int iters;             /* FGMRES iterations (= preconditioner applications) */
  int restarts;          /* completed restart cycles */
  int vcycles;           /* V-cycles applied */
  int status;            /* return status of the call */
  double rel_energy_res; /* true relative energy residual of the returned iterate */
  double rel_l2_res;     /* true ||b - A x||_2 / ||b||_2 of the returned iterate */
  double t_setup_ms;     /* hierarchy set-up time (device) */
  double t_solve_ms;     /* Krylov loop time (device) */
  double alg_bytes;      /* algorithmic HBM bytes of the call (model, see the design notes) */
  int levels;            /* multigrid levels */
  int coarse_n;          /* velocity unknowns of the coarsest level (direct solve if <= 1024) */
  long long kernel_launches; /* CUDA kernels this call launched (graph kernel nodes included) */
} pyro_stats;

typedef struct pyro_stokes_s* pyro_stokes;

/* Default options (see pyro_opts). */
void pyro_default_opts(pyro_opts* opts);

/* Create a solver for an nx x ny cell grid on an Lx x Ly box with boundary `bc` (NULL = free slip
 * on all sides) and options `opts` (NULL = defaults). Allocates the whole multigrid hierarchy, the
 * Krylov bases and all workspaces on the current CUDA device; they stay resident until destroy,
 * so repeated solves of one shape reuse them. nx, ny >= 2 (any parity): levels halve while both
 * counts are even and the short side stays >= coarsest_min, then coarsen by coarsen_ratio while
 * the coarsest level has more than 1024 velocity unknowns (coarsen_general); a coarsest level of
 * at most 1024 velocity unknowns is solved by a dense FP64 inverse, a larger one by coarse_sweeps
 * smoothing sweeps.
 * Returns PYRO_OK and *out, or an error (then *out = NULL). */
int pyro_stokes_create(int nx, int ny, double Lx, double Ly, const pyro_bc* bc,
                       const pyro_opts* opts, pyro_stokes* out);

/* Bytes of device memory pyro_stokes_create(nx, ny, ..., opts) allocates (used for admission
 * control by callers that share the GPU). 0 if the size is invalid. */
size_t pyro_stokes_footprint(int nx, int ny, const pyro_opts* opts);

/* y = A x for the saddle-point operator [[L, G], [D, 0]] (eq. stokes_saddle) with homogeneous
 * boundary rules (no boundary constants; those belong to the right-hand side). Inputs eta_n,
 * eta_c, vx, vy, p; outputs Ax (x-momentum rows), Ay (y-momentum rows), Ap (continuity rows),
 * each written at its unknown locations and 0 elsewhere. Computed in FP64. */
int pyro_stokes_apply(pyro_stokes h, const double* eta_n, const double* eta_c,
                      const double* vx, const double* vy, const double* p,
                      double* Ax, double* Ay, double* Ap, void* cuda_stream);

/* Solve A [v; p] = [f; 0] with f = -rho g (gravity g = (gx, gy) in the grid frame, y down; the
 * paper's Sec. "Viscosity Rescaling and Initial Guess" lithostatic convention) plus the boundary
 * constants, to relative energy residual <= tol. Output pressure has zero mean (eq.
 * pressure_normalization). vx, vy, p: initial guess on input if opts.warm_start, solution on
 * output. stats (host pointer) may be NULL. Returns PYRO_OK, PYRO_W_NOT_CONVERGED, or an error. */
int pyro_stokes_solve(pyro_stokes h, const double* eta_n, const double* eta_c, const double* rho,
                      double gx, double gy, double tol, double* vx, double* vy, double* p,
                      pyro_stats* stats, void* cuda_stream);

/* Adjoint of the last successful solve on h: solves A lambda = [dJ_dvx; dJ_dvy; dJ_dp] (A is
 * symmetric) to tol and forms
 *   dJ_deta_c(cell) = 2 (exx(v) exx(lambda) + eyy(v) eyy(lambda)),
 *   dJ_deta_n(node) = w_n gamma(v) gamma(lambda)   (w_n = 1 inside, 1/2 on walls, 0 at corners),
 *   dJ_drho(node)   = lambda . d f / d rho          (may be NULL),
 * with exx = d vx/dx, eyy = d vy/dy at cells and gamma = d vx/dy + d vy/dx at nodes (boundary
 * ghosts filled homogeneously for lambda). Not in the paper: this is the discrete adjoint of its
 * operator. Rejects prescribed-velocity boundaries (PYRO_E_INVALID). */
int pyro_stokes_adjoint(pyro_stokes h, const double* dJ_dvx, const double* dJ_dvy,
                        const double* dJ_dp, double tol, double* dJ_deta_n, double* dJ_deta_c,
                        double* dJ_drho, pyro_stats* stats, void* cuda_stream);

/* One application of the preconditioner z = M^-1 r (diagnostic / test entry point): sets up the
 * hierarchy from eta_n, eta_c exactly as pyro_stokes_solve does, then applies one Uzawa sweep
 * (paper Sec. "Uzawa Iteration as a Fixed Point Method"): z_v = one multigrid V-cycle on L z_v = r_v
 * from zero (eq. multigrid_levels), z_p = alpha_p eta_c (r_p - D z_v) with its mean removed. In
 * PYRO_PREC_MIXED the V-cycle runs in FP32 (z_v holds its FP32 values) and z_p is FP64.
 * Inputs r_vx, r_vy, r_p are read at their unknown locations; outputs are written there and 0
 * elsewhere. Returns after completion on cuda_stream. */
int pyro_stokes_precond(pyro_stokes h, const double* eta_n, const double* eta_c, const double* r_vx,
                        const double* r_vy, const double* r_p, double* z_vx, double* z_vy, double* z_p,
                        void* cuda_stream);

/* Device-time breakdown of the FGMRES iterations (diagnostic). When enabled (takes effect at the
 * next solve, accumulators reset), CUDA events are recorded around the phases of every iteration
 * and read back at the iteration's existing host synchronisation. ms[6] receives accumulated
 * milliseconds of: [0] preconditioner input cast, [1] finest-level pre-smoothing sweeps,
 * [2] all coarser-level work (residual, restriction, coarse levels, prolongation), [3] finest-level
 * post-smoothing sweeps, [4] pressure block + FP64 operator A z, [5] orthogonalisation;
 * counts[2] receives [0] timed iterations, [1] finest-level smoothing sweeps (each sweep =
 * vx-red, vx-black, vy-red, vy-black launches). Returns PYRO_E_INVALID on a NULL handle. */
int pyro_stokes_set_timing(pyro_stokes h, int enable);
int pyro_stokes_get_timing(pyro_stokes h, double* ms, long long* counts);

/* Allocation-free residual (no counterpart in the paper: an interface addition of this library).
 * For callers that cannot call cudaMalloc — e.g. an application whose own pool allocator owns all
 * device memory, or a latency-critical loop where an allocation's implicit synchronisation is
 * not acceptable. Needs no handle and allocates nothing: computes r = b - A x with
 * b = -rho g plus the boundary constants (exactly the residual of pyro_stokes_solve) for the
 * fields vx, vy, p, writes r_vx, r_vy, r_p (residual at unknowns, 0 elsewhere) and
 * rel_res[0] = relative energy residual, rel_res[1] = relative l2 residual (rel_res may be a
 * host or device pointer; every field pointer must be a device pointer of the current device). Its
 * only scratch is a fixed 128 KiB array in device global memory (16384 doubles: one 4-value
 * partial per block of 4 grid rows), held by every GPU that loads the library until the process
 * exits; hence ny + 2 must not exceed 16380 rows (else PYRO_E_INVALID, as for host pointers, other
 * GPUs' memory or a periodic boundary). Every call looks up the array's device address in the
 * current device's context (a lookup allocates nothing); the first lookup in a context may load the
 * library's device code, so make the first call on a device before any stream capture. All calls
 * share the array and it keeps
 * the last call's contents (every slot read is written first in the same call, so nothing needs to
 * start at zero); calls that overlap on the GPU, on any streams, race on it. Returns after
 * completion on cuda_stream. */
int pyro_stokes_residual_noalloc(int nx, int ny, double Lx, double Ly, const pyro_bc* bc,
                                 const double* eta_n, const double* eta_c, const double* rho,
                                 double gx, double gy, const double* vx, const double* vy,
                                 const double* p, double* r_vx, double* r_vy, double* r_p,
                                 double* rel_res, void* cuda_stream);

/* Release every device allocation of h (NULL is a no-op). */
void pyro_stokes_destroy(pyro_stokes h);

/* Diagnostic (no counterpart in the paper): the FP64 fused multiply-add rate of the current GPU in
 * TFLOP/s (2 flop per FMA), timed with CUDA events on one launch of independent FMA chains
 * (8 chains x iters FMAs per thread, 8 blocks of 256 threads per SM) after one warm-up launch.
 * The library's FP64 stencils and Krylov passes are bound by this rate on B300, so it is the
 * denominator of their roofline. Allocates and frees one double. Synchronises cuda_stream.
 * PYRO_E_INVALID for iters < 1 or a null tflops. */
int pyro_fp64_fma_rate(int iters, double* tflops, void* cuda_stream);

/* Static description of a status code. */
const char* pyro_strerror(int status);

/* Library version string. */
const char* pyro_version(void);

/* ---- marker steps of the marker-in-cell loop: marker <-> grid interpolation (the step that feeds
 * eta and rho to the solve: Sec. "Marker-to-grid interpolation" and "Grid-to-marker
 * interpolation") and marker advection in the solved velocity (Sec. "Advection of Lagrangian
 * Markers") ---------------------------------------------------------------------------------
 * Lattices in the padded (ny+2) x (nx+2) layout, row i with y:
 *   PYRO_LATTICE_NODES  basic nodes  x_j = j dx,         y_i = i dy,         i in [0,ny], j in [0,nx]
 *   PYRO_LATTICE_CELLS  cell centres x_j = (j - 1/2) dx, y_i = (i - 1/2) dy, i in [1,ny], j in [1,nx]
 *   PYRO_LATTICE_VX     vx points    x_j = j dx,         y_i = (i - 1/2) dy, i in [1,ny], j in [0,nx]
 *   PYRO_LATTICE_VY     vy points    x_j = (j - 1/2) dx, y_i = i dy,         i in [0,ny], j in [1,nx]
 * A marker belongs to the lattice cell whose top-left node lies at or left/above it (clamped into
 * the outermost cell when it lies beyond the lattice). Bilinear weights: that node (1-fx)(1-fy),
 * its right neighbour fx(1-fy), the node below (1-fx)fy, the diagonal fx fy, with fx = r_x/dx,
 * fy = r_y/dy the offsets from the top-left node. */
typedef enum { PYRO_LATTICE_NODES = 0, PYRO_LATTICE_CELLS = 1, PYRO_LATTICE_VX = 2, PYRO_LATTICE_VY = 3 } pyro_lattice;
/* Advection schemes (Sec. "Advection of Lagrangian Markers"), per (sub)step of size h:
 *   EULER   x + h v(x)                                          (eq. euler_advection)
 *   HEUN    x* = x + h v(x); x + h/2 (v(x) + v(x*))              (eq. heun_method)
 *   RK4     the classical four-stage Runge-Kutta step            (eq. rk4_method)
 *   TAYLOR  x + h v0 + h^2/2 J v0 + h^3/6 (H : v0 v0)            (eq. lpi_update)
 * v(x) is vx interpolated bilinearly on PYRO_LATTICE_VX and vy on PYRO_LATTICE_VY; for TAYLOR, J
 * and H are the first derivatives and the d2/dxdy term of those interpolants at the marker (zero
 * across a direction in which the marker lies beyond the lattice). */
typedef enum { PYRO_ADVECT_EULER = 0, PYRO_ADVECT_HEUN = 1, PYRO_ADVECT_RK4 = 2, PYRO_ADVECT_TAYLOR = 3 } pyro_advect_scheme;
typedef struct pyro_markers_s* pyro_markers;  /* opaque; owns the bucketing workspace */

/* Workspace for an nx x ny grid of size Lx x Ly and up to max_markers markers (about
 * 24 B x max_markers + 76 B x cells of device memory). PYRO_E_INVALID on bad sizes,
 * PYRO_E_NOMEM if allocation fails. */
int pyro_markers_create(int nx, int ny, double Lx, double Ly, long long max_markers, pyro_markers* out);

/* Marker -> grid weighted average: grid(i,j) = sum_m w_m(i,j) phi_m / sum_m w_m(i,j) over the
 * markers of the four lattice cells around the node; nodes no marker reaches keep their input
 * value; wsum (optional) receives the weight sums (0 where no marker reaches). Deterministic: the
 * markers are bucketed by cell with integer atomics, each bucket sorted by marker index and summed
 * in that order into per-cell corner sums, and each node adds its four cells' sums in a fixed
 * order. xm, ym, phim: n device doubles; grid, wsum: device
 * (ny+2) x (nx+2) arrays. Synchronises cuda_stream before it returns. PYRO_E_INVALID for host
 * pointers, n > max_markers or an unknown lattice; PYRO_E_NONFINITE if a position is not finite. */
int pyro_markers_to_grid(pyro_markers h, int lattice, long long n, const double* xm, const double* ym,
                         const double* phim, double* grid, double* wsum, void* cuda_stream);

/* Grid -> marker bilinear interpolation phi_m = sum over the four corners of w grid (the weights
 * sum to one). Device pointers; stream-ordered, returns after enqueueing. */
int pyro_grid_to_markers(pyro_markers h, int lattice, long long n, const double* xm, const double* ym,
                         const double* grid, double* phim, void* cuda_stream);

/* Advect n markers in place through a time dt in the frozen velocity (vx, vy: device (ny+2) x
 * (nx+2) arrays as returned by pyro_stokes_solve), in `substeps` equal steps of `scheme`, each
 * step's result clamped into [0, Lx] x [0, Ly]. xm, ym: n device doubles (updated). One thread per
 * marker in FP64; stream-ordered, returns after enqueueing. PYRO_E_INVALID for a null handle,
 * n < 0, an unknown scheme, substeps < 1, non-finite dt or host pointers. Non-finite positions
 * stay non-finite. */
int pyro_markers_advect(pyro_markers h, int scheme, long long n, double* xm, double* ym, const double* vx,
                        const double* vy, double dt, int substeps, void* cuda_stream);

/* CFL-limited step (the grid-based step limit of Sec. "Advection of Lagrangian Markers"):
 * *dt_out = cfl * min(dx / max|vx|, dy / max|vy|), maxima over the whole padded arrays, +infinity
 * (HUGE_VAL) when both are zero everywhere. Synchronises cuda_stream. PYRO_E_INVALID for cfl <= 0,
 * a null dt_out or host pointers; PYRO_E_NONFINITE if an entry is not finite. */
int pyro_markers_max_dt(pyro_markers h, const double* vx, const double* vy, double cfl, double* dt_out,
                        void* cuda_stream);

/* Release the workspace (NULL is a no-op). */
void pyro_markers_destroy(pyro_markers h);

#ifdef __cplusplus
}
#endif

#endif /* PYRO_H */
