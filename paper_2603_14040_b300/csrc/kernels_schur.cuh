// Weighted BFBt approximation of the Schur complement for the pressure block of the Uzawa
// preconditioner, with its smoothed-aggregation pressure multigrid. Not in the paper: the paper's
// pressure block is the diagonal viscosity surrogate eta_c (Sec. "Uzawa Iteration as a Fixed Point
// Method"), which stalls the outer Krylov method when the viscosity jumps by many orders of
// magnitude (a stiff lid over weak and strong inclusions). The surrogate here is
//     S~^-1 = K^-1 (D W^-1 (-L) W^-1 G) K^-1,   K = D W^-1 G,   W = diag(-L)^(1/2)
// (Elman 1999; square-root-diagonal weighting after Rudi, Stadler and Ghattas 2017), each K^-1 one
// V-cycle of a smoothed-aggregation multigrid on 2 x 2 aggregates:
//   * K on the finest pressure grid is the 5-point cell operator with face conductances
//     c_f = 1 / (h_f^2 W_f) (walls carry no flux): (K p)_c = sum_f c_f (p_c - p_nb);
//   * prolongator P = (I - omega_p diag(K)^-1 K_near) P0, P0 the aggregation, K_near the 3 x 3-box
//     part of K with the dropped couplings lumped on the diagonal; R = P^T; K_{l+1} = P^T K_l P,
//     which stays inside a 5 x 5 box stencil on every coarse level;
//   * damped Jacobi smoothing, a dense inverse of K_c + s 1 1^T on the coarsest level.
// Pressure arrays are compact row-major (cell (i, j), 1-based in the padded layout, is entry
// (i-1) nx + (j-1)); a coarse level holds 25 coefficient planes, plane (di+2)*5 + (dj+2) for the
// coupling of cell k with cell k + di nx + dj.
#pragma once
#include "common.cuh"

namespace pyro {

constexpr int kSchurBox = 25;
constexpr int kSchurMaxCoarse = 256;   // cells of the coarsest pressure level (dense inverse)

// -diag(L) at an unknown vx(i, j) / vy(i, j) (the boundary-eliminated diagonal of the point operators)
template <typename T, typename SE>
__device__ inline T negdiag_vx(const GeomT<T>& g, int i, int j, const SE* en, const SE* ec) {
  const size_t c = (size_t)i * g.ld + j;
  T d = T(2) * ((T)ec[c] + (T)ec[c + 1]) * g.idx2 + ((T)en[c - g.ld] + (T)en[c]) * g.idy2;
  if (i == 1) d -= g.sN * (T)en[c - g.ld] * g.idy2;
  if (i == g.ny) d -= g.sS * (T)en[c] * g.idy2;
  return d;
}
template <typename T, typename SE>
__device__ inline T negdiag_vy(const GeomT<T>& g, int i, int j, const SE* en, const SE* ec) {
  const size_t c = (size_t)i * g.ld + j;
  T d = T(2) * ((T)ec[c] + (T)ec[c + g.ld]) * g.idy2 + ((T)en[c - 1] + (T)en[c]) * g.idx2;
  if (j == 1) d -= g.sW * (T)en[c - 1] * g.idx2;
  if (j == g.nx) d -= g.sE * (T)en[c] * g.idx2;
  return d;
}

// W^-1 = diag(-L)^(-1/2) at the velocity unknowns (padded layout, 0 elsewhere) and, per cell of the
// finest pressure grid, the conductances of its east face cx and south face cy (0 on walls), the
// diagonal of K (sum of the four face conductances) and omega / diagonal (omega the damping of the
// pressure cycle's Jacobi sweeps).
template <typename T, typename SE>
__global__ void k_schur_weights(GeomT<T> g, const SE* __restrict__ en, const SE* __restrict__ ec, T* __restrict__ wix,
                                T* __restrict__ wiy, T* __restrict__ cx, T* __restrict__ cy, T* __restrict__ diag,
                                T* __restrict__ widg, T omega) {
  const int i = blockIdx.y * blockDim.y + threadIdx.y;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (i > g.ny + 1 || j > g.nx + 1) return;
  const size_t c = (size_t)i * g.ld + j;
  const T one = T(1);
  wix[c] = is_vx(g.nx, g.ny, i, j) ? one / sqrt(negdiag_vx<T>(g, i, j, en, ec)) : T(0);
  wiy[c] = is_vy(g.nx, g.ny, i, j) ? one / sqrt(negdiag_vy<T>(g, i, j, en, ec)) : T(0);
  if (!is_p(g.nx, g.ny, i, j)) return;
  const size_t k = (size_t)(i - 1) * g.nx + (j - 1);
  const T ce = (j <= g.nx - 1) ? g.idx2 / sqrt(negdiag_vx<T>(g, i, j, en, ec)) : T(0);
  const T cw = (j - 1 >= 1) ? g.idx2 / sqrt(negdiag_vx<T>(g, i, j - 1, en, ec)) : T(0);
  const T cs = (i <= g.ny - 1) ? g.idy2 / sqrt(negdiag_vy<T>(g, i, j, en, ec)) : T(0);
  const T cn = (i - 1 >= 1) ? g.idy2 / sqrt(negdiag_vy<T>(g, i - 1, j, en, ec)) : T(0);
  cx[k] = ce;
  cy[k] = cs;
  const T d = ce + cw + cs + cn;
  diag[k] = d;
  widg[k] = d > T(0) ? omega / d : T(0);
}

// One level of the pressure hierarchy as seen by the kernels.
template <typename T>
struct PLev {
  int nx, ny;
  const T* cx;    // finest level: east-face conductances (else null)
  const T* cy;    // finest level: south-face conductances
  const T* box;   // coarse levels: 25 planes of nx*ny coefficients (else null)
  const T* diag;  // diagonal of K
  const T* widg;  // omega / diagonal (0 where the diagonal is 0)
};

// K(k, k + di nx + dj) for |di|, |dj| <= 2 (0 outside the stencil or the grid)
template <typename T>
__device__ inline T pcoef(const PLev<T>& L, int i, int j, int di, int dj) {
  const int ii = i + di, jj = j + dj;
  if (ii < 0 || ii >= L.ny || jj < 0 || jj >= L.nx) return T(0);
  const size_t k = (size_t)i * L.nx + j;
  const size_t n = (size_t)L.nx * L.ny;
  if (L.box) return L.box[(size_t)((di + 2) * 5 + (dj + 2)) * n + k];
  if (di == 0 && dj == 0) return L.diag[k];
  if (di == 0 && dj == 1) return -L.cx[k];
  if (di == 0 && dj == -1) return -L.cx[k - 1];
  if (di == 1 && dj == 0) return -L.cy[k];
  if (di == -1 && dj == 0) return -L.cy[k - L.nx];
  return T(0);
}

// (K x)_k, without branches around the loads so that all of them are in flight at once: the
// coefficient of every coupling that leaves the grid is 0 (walls carry no conductance, and the
// Galerkin boxes hold 0 there), so the neighbour index is only clamped into the array and the
// product adds an exact 0; the finest level's west / north couplings of the first column / row,
// whose stored conductance belongs to another cell, are masked. Same terms in the same order as
// the plain sum over the couplings inside the grid.
template <typename T>
__device__ inline T papply(const PLev<T>& L, int i, int j, const T* __restrict__ x) {
  const int n = L.nx * L.ny;
  const int k = i * L.nx + j;
  if (!L.box) {
    const T cE = L.cx[k], cS = L.cy[k];
    const T cWr = L.cx[max(k - 1, 0)], cNr = L.cy[max(k - L.nx, 0)];
    const T cW = j >= 1 ? cWr : T(0), cN = i >= 1 ? cNr : T(0);
    const T xE = x[min(k + 1, n - 1)], xW = x[max(k - 1, 0)];
    const T xS = x[min(k + L.nx, n - 1)], xN = x[max(k - L.nx, 0)];
    T s = L.diag[k] * x[k];
    s -= cE * xE;
    s -= cW * xW;
    s -= cS * xS;
    s -= cN * xN;
    return s;
  }
  T s = T(0);
#pragma unroll
  for (int di = -2; di <= 2; ++di) {
#pragma unroll
    for (int dj = -2; dj <= 2; ++dj) {
      const int kk = min(max(k + di * L.nx + dj, 0), n - 1);
      s += L.box[(size_t)((di + 2) * 5 + (dj + 2)) * n + k] * x[kk];
    }
  }
  return s;
}

// f_k minus the off-diagonal part of (K x)_k: with it a damped Jacobi update is
// (1 - omega) x_k + (omega / K_kk) poff, which on the FP64 path (bound by the FP64 rate) takes 6
// operations per finest-level cell instead of 9. Loads as in papply.
template <typename T>
__device__ inline T poff(const PLev<T>& L, int i, int j, T fk, const T* __restrict__ x) {
  const int n = L.nx * L.ny;
  const int k = i * L.nx + j;
  if (!L.box) {
    const T cE = L.cx[k], cS = L.cy[k];
    const T cWr = L.cx[max(k - 1, 0)], cNr = L.cy[max(k - L.nx, 0)];
    const T cW = j >= 1 ? cWr : T(0), cN = i >= 1 ? cNr : T(0);
    T s = fk;
    s += cE * x[min(k + 1, n - 1)];
    s += cW * x[max(k - 1, 0)];
    s += cS * x[min(k + L.nx, n - 1)];
    s += cN * x[max(k - L.nx, 0)];
    return s;
  }
  T s = fk;
#pragma unroll
  for (int di = -2; di <= 2; ++di) {
#pragma unroll
    for (int dj = -2; dj <= 2; ++dj) {
      if (di == 0 && dj == 0) continue;
      const int kk = min(max(k + di * L.nx + dj, 0), n - 1);
      s -= L.box[(size_t)((di + 2) * 5 + (dj + 2)) * n + k] * x[kk];
    }
  }
  return s;
}

// first coarse row / column of the 2 x 2 window of aggregates that the 3 x 3 neighbourhood of fine
// index a touches: floor((a - 1) / 2)
__device__ inline int pwin(int a) { return a >= 1 ? (a - 1) / 2 : -1; }

// Rows of the smoothed prolongator: pw[s * n + k] = P(k, J_s) for the window slots s = 2 a + b,
// J_s = (pwin(i) + a, pwin(j) + b): [agg(k) = J] - omega_p / K_kk * sum over the 3 x 3 neighbours c
// of k in aggregate J of K_near(k, c) (K_near(k, k) = K_kk + the couplings outside the 3 x 3 box).
template <typename T>
__global__ void k_schur_prow(PLev<T> L, int nxc, int nyc, T omega_p, T* __restrict__ pw) {
  const int k0 = blockIdx.x * blockDim.x + threadIdx.x;
  const int n = L.nx * L.ny;
  if (k0 >= n) return;
  const int i = k0 / L.nx, j = k0 % L.nx;
  const T kd = pcoef<T>(L, i, j, 0, 0);
  T far = T(0);
  if (L.box) {
    for (int di = -2; di <= 2; ++di)
      for (int dj = -2; dj <= 2; ++dj)
        if (di == -2 || di == 2 || dj == -2 || dj == 2) far += pcoef<T>(L, i, j, di, dj);
  }
  const int oi = pwin(i), oj = pwin(j);
  T w[4] = {T(0), T(0), T(0), T(0)};
  for (int di = -1; di <= 1; ++di)
    for (int dj = -1; dj <= 1; ++dj) {
      const int ci = i + di, cj = j + dj;
      if (ci < 0 || ci >= L.ny || cj < 0 || cj >= L.nx) continue;
      T kk = pcoef<T>(L, i, j, di, dj);
      if (di == 0 && dj == 0) kk += far;
      const int s = ((ci >> 1) - oi) * 2 + ((cj >> 1) - oj);
      w[s] += kk;
    }
  const int si = ((i >> 1) - oi) * 2 + ((j >> 1) - oj);
  const T f = omega_p / kd;
  for (int s = 0; s < 4; ++s) {
    const int Ji = oi + (s >> 1), Jj = oj + (s & 1);
    const bool ok = Ji >= 0 && Ji < nyc && Jj >= 0 && Jj < nxc;
    pw[(size_t)s * n + k0] = ok ? ((s == si ? T(1) : T(0)) - f * w[s]) : T(0);
  }
}

// Galerkin coarse operator K_c = P^T K P into 25 planes (+ the diagonal and omega / diagonal).
// Sixteen threads per coarse cell, one per fine cell of its 4 x 4 window, each summing that fine
// cell's contributions P(a, K) K(a, b) P(b, J) into its own 25 slots in shared memory (a register
// array indexed by the coupling would live in local memory); then each of the sixteen sums slots
// sub and sub + 16 over the sixteen partials, in a fixed order. One thread per coarse cell left the
// small levels of the set-up latency-bound on a few SMs. Launched with kSchurRapThreads threads and
// kSchurRapThreads * 25 * sizeof(T) bytes of dynamic shared memory.
constexpr int kSchurRapThreads = 128;
template <typename T>
__global__ void __launch_bounds__(kSchurRapThreads) k_schur_rap(PLev<T> L, const T* __restrict__ pw, int nxc,
                                                                int nyc, T* __restrict__ box, T* __restrict__ cdiag,
                                                                T* __restrict__ cwidg, T omega) {
  extern __shared__ __align__(16) unsigned char rap_raw[];
  T* sacc = reinterpret_cast<T*>(rap_raw);
  T* acc = sacc + (size_t)threadIdx.x * kSchurBox;
  const int gt = blockIdx.x * blockDim.x + threadIdx.x;
  const int K0 = gt >> 4, sub = gt & 15;
  const int nc = nxc * nyc;
  const bool active = K0 < nc;
  const int I = active ? K0 / nxc : 0, J = active ? K0 % nxc : 0;
  const int n = L.nx * L.ny;
  for (int q = 0; q < kSchurBox; ++q) acc[q] = T(0);
  const int ai = 2 * I - 1 + (sub >> 2), aj = 2 * J - 1 + (sub & 3);
  if (active && ai >= 0 && ai < L.ny && aj >= 0 && aj < L.nx) {
    const int sa_i = I - pwin(ai), sa_j = J - pwin(aj);
    const T pa = (sa_i >= 0 && sa_i <= 1 && sa_j >= 0 && sa_j <= 1)
                     ? pw[(size_t)(sa_i * 2 + sa_j) * n + (size_t)ai * L.nx + aj] : T(0);
    if (pa != T(0)) {
      const int r = L.box ? 2 : 1;
      for (int di = -r; di <= r; ++di)
        for (int dj = -r; dj <= r; ++dj) {
          const T kab = pcoef<T>(L, ai, aj, di, dj);
          if (kab == T(0)) continue;
          const int bi = ai + di, bj = aj + dj;
          const int obi = pwin(bi), obj = pwin(bj);
          const size_t b = (size_t)bi * L.nx + bj;
          for (int s = 0; s < 4; ++s) {
            const int Ji = obi + (s >> 1), Jj = obj + (s & 1);
            if (Ji < 0 || Ji >= nyc || Jj < 0 || Jj >= nxc) continue;
            const T wb = pw[(size_t)s * n + b];
            acc[(Ji - I + 2) * 5 + (Jj - J + 2)] += pa * kab * wb;
          }
        }
    }
  }
  __syncthreads();
  if (!active) return;
  const T* cell = sacc + (size_t)(threadIdx.x - sub) * kSchurBox;   // the cell's first thread's slots
  for (int q = sub; q < kSchurBox; q += 16) {
    T t = T(0);
    for (int u = 0; u < 16; ++u) t += cell[u * kSchurBox + q];
    box[(size_t)q * nc + K0] = t;
    if (q == 12) {
      cdiag[K0] = t;
      cwidg[K0] = t > T(0) ? omega / t : T(0);
    }
  }
}

// One damped Jacobi sweep x_out = x_in + omega (f - K x_in) / diag, formed as
// (1 - omega) x_in + (omega / diag) poff (the sweep from zero, omega f / diag, is formed by whoever
// writes f)
template <typename T>
__global__ void k_schur_jacobi(PLev<T> L, const T* __restrict__ x_in, T* __restrict__ x_out, const T* __restrict__ f,
                               T om1) {
  const int k0 = blockIdx.x * blockDim.x + threadIdx.x;
  if (k0 >= L.nx * L.ny) return;
  const int i = k0 / L.nx, j = k0 - i * L.nx;
  x_out[k0] = om1 * x_in[k0] + L.widg[k0] * poff<T>(L, i, j, f[k0], x_in);
}

// ---- fused steps of the pressure cycle (same arithmetic, fewer dependent launches) ----------
constexpr int kSchurTS = 16;   // fine cells per tile side of k_schur_prolong_jacobi

// Residual and restriction in one launch: a block computes r = f - K x on the fine cells its
// CT x CT coarse cells restrict from (a (2 CT + 2)^2 region, kept in shared memory; cells outside
// the grid hold 0), then f_c = P^T r for each coarse cell exactly as a separate restriction would
// sum it. With xc given (the coarse level is not the coarsest) the coarse level's first Jacobi
// sweep from zero is written too: xc = (omega / diag_c) f_c.
// CT is 16, 8 or 4 by level size (schur_tile_ct) so that small levels still spread their residuals
// over many SMs, one or two per thread: a single block doing a whole small level serially is
// latency- (and in FP64 arithmetic-) bound.
template <int CT>
constexpr int schur_rr_threads() { return CT == 16 ? 256 : (CT == 8 ? 352 : 128); }
inline int schur_tile_ct(long long coarse_cells) {
  return coarse_cells >= 148LL * 256 ? 16 : (coarse_cells >= 148LL * 64 ? 8 : 4);
}
template <typename T, int CT>
__global__ void __launch_bounds__(512) k_schur_resrestrict(PLev<T> L, const T* __restrict__ x,
                                                           const T* __restrict__ f, const T* __restrict__ pw,
                                                           int nxc, int nyc, T* __restrict__ fc,
                                                           const T* __restrict__ widgc, T* __restrict__ xc) {
  constexpr int RW = 2 * CT + 2;
  __shared__ T rs[RW * RW];
  const int I0 = blockIdx.y * CT, J0 = blockIdx.x * CT;
  const int fi0 = 2 * I0 - 1, fj0 = 2 * J0 - 1;
  for (int t = threadIdx.x; t < RW * RW; t += blockDim.x) {
    const int ai = fi0 + t / RW, aj = fj0 + t % RW;
    T v = T(0);
    if (ai >= 0 && ai < L.ny && aj >= 0 && aj < L.nx) {
      const int k = ai * L.nx + aj;
      v = f[k] - papply<T>(L, ai, aj, x);
    }
    rs[t] = v;
  }
  __syncthreads();
  const int I = I0 + (int)threadIdx.x / CT, J = J0 + (int)threadIdx.x % CT;
  if (threadIdx.x >= CT * CT || I >= nyc || J >= nxc) return;
  const size_t n = (size_t)L.nx * L.ny;
  const int li = 2 * (I - I0), lj = 2 * (J - J0);   // local origin of the cell's 4 x 4 window
  T s = T(0);
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int ai = 2 * I - 1 + a;
    const bool okr = ai >= 0 && ai < L.ny;
    const size_t row = (size_t)min(max(ai, 0), L.ny - 1) * L.nx;
    const int si = a < 2 ? 1 : 0;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int aj = 2 * J - 1 + b;
      const bool ok = okr && aj >= 0 && aj < L.nx;
      const size_t idx = row + min(max(aj, 0), L.nx - 1);
      const int sj = b < 2 ? 1 : 0;
      const T w = pw[(size_t)(si * 2 + sj) * n + idx];
      const T rv = rs[(li + a) * RW + (lj + b)];
      s += (ok ? w : T(0)) * rv;   // the weight masked, so that the product and the sum fuse
    }
  }
  const int K0 = I * nxc + J;
  fc[K0] = s;
  if (xc) xc[K0] = s * widgc[K0];
}

// Prolongation and the first post-smoothing Jacobi sweep in one launch: a block forms
// x + P e_c on its 16 x 16 fine cells and a halo of H (2 for the 5 x 5 boxes, 1 for the finest
// level's 5-point operator; shared memory, 0 outside the grid), then
// the damped Jacobi sweep on its own cells, in the form k_schur_jacobi uses.
template <typename T, int H>
__global__ void __launch_bounds__(256) k_schur_prolong_jacobi(PLev<T> L, const T* __restrict__ x,
                                                              const T* __restrict__ pw, const T* __restrict__ ec,
                                                              int nxc, int nyc, const T* __restrict__ f, T om1,
                                                              T* __restrict__ x_out) {
  constexpr int RW = kSchurTS + 2 * H;
  __shared__ T xs[RW * RW];
  const int i0 = blockIdx.y * kSchurTS - H, j0 = blockIdx.x * kSchurTS - H;
  const size_t n = (size_t)L.nx * L.ny;
  for (int t = threadIdx.x; t < RW * RW; t += blockDim.x) {
    const int i = i0 + t / RW, j = j0 + t % RW;
    T v = T(0);
    if (i >= 0 && i < L.ny && j >= 0 && j < L.nx) {
      const size_t k = (size_t)i * L.nx + j;
      const int oi = pwin(i), oj = pwin(j);
      T sp = T(0);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int Ji = oi + (q >> 1), Jj = oj + (q & 1);
        if (Ji < 0 || Ji >= nyc || Jj < 0 || Jj >= nxc) continue;
        sp += pw[(size_t)q * n + k] * ec[(size_t)Ji * nxc + Jj];
      }
      v = x[k] + sp;
    }
    xs[t] = v;
  }
  __syncthreads();
  const int li = H + (int)threadIdx.x / kSchurTS, lj = H + (int)threadIdx.x % kSchurTS;
  const int i = i0 + li, j = j0 + lj;
  if (threadIdx.x >= kSchurTS * kSchurTS || i >= L.ny || j >= L.nx) return;
  const int k = i * L.nx + j;
  const T xc = xs[li * RW + lj];
  T so = f[k];   // f minus the off-diagonal part of K x_p, as poff forms it
  if (!L.box) {
    const T cE = L.cx[k], cS = L.cy[k];
    const T cWr = L.cx[max(k - 1, 0)], cNr = L.cy[max(k - L.nx, 0)];
    const T cW = j >= 1 ? cWr : T(0), cN = i >= 1 ? cNr : T(0);
    so += cE * xs[li * RW + lj + 1];
    so += cW * xs[li * RW + lj - 1];
    so += cS * xs[(li + 1) * RW + lj];
    so += cN * xs[(li - 1) * RW + lj];
  } else if constexpr (H >= 2) {
#pragma unroll
    for (int di = -2; di <= 2; ++di) {
#pragma unroll
      for (int dj = -2; dj <= 2; ++dj) {
        if (di == 0 && dj == 0) continue;
        so -= L.box[(size_t)((di + 2) * 5 + (dj + 2)) * n + k] * xs[(li + di) * RW + (lj + dj)];
      }
    }
  }
  x_out[k] = om1 * xc + L.widg[k] * so;
}

// Dense coarsest matrix K_c + s 1 1^T with s = trace(K_c) / nc^2 (symmetric positive definite for
// the connected coarse grid; for a zero-sum right-hand side its solution is the zero-mean solution
// of K_c x = f). One block.
template <typename T>
__global__ void k_schur_coarse_assemble(PLev<T> L, double* __restrict__ A) {
  __shared__ double sh[32];
  const int nc = L.nx * L.ny;
  double t = 0.0;
  for (int k = threadIdx.x; k < nc; k += blockDim.x) t += (double)L.diag[k];
  for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = t;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = threadIdx.x < (blockDim.x + 31) / 32 ? sh[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (threadIdx.x == 0) sh[0] = v;
  }
  __syncthreads();
  const double s = sh[0] / ((double)nc * (double)nc);
  for (int e = threadIdx.x; e < nc * nc; e += blockDim.x) {
    const int r = e / nc, c = e % nc;
    const int di = c / L.nx - r / L.nx, dj = c % L.nx - r % L.nx;
    double v = s;
    if (di >= -2 && di <= 2 && dj >= -2 && dj <= 2) v += (double)pcoef<T>(L, r / L.nx, r % L.nx, di, dj);
    A[e] = v;
  }
}

// x = (K_c + s 1 1^T)^-1 (f - mean f), FP64 arithmetic, one warp per row of the inverse (coalesced
// row reads, spread over (nc + 7) / 8 blocks of 256 threads: FP64 work on a single SM is slow on this
// part). Every block forms the mean itself, in the same fixed order.
template <typename T>
__global__ void k_schur_coarse_solve(const double* __restrict__ Ainv, int nc, const T* __restrict__ f,
                                     T* __restrict__ x) {
  __shared__ double fv[kSchurMaxCoarse];
  __shared__ double sh[32];
  double t = 0.0;
  for (int k = threadIdx.x; k < nc; k += blockDim.x) {
    const double v = (double)f[k];
    fv[k] = v;
    t += v;
  }
  for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) sh[warp] = t;
  __syncthreads();
  double tot = 0.0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += sh[w];
  const double mean = tot / nc;
  const int r = blockIdx.x * (int)(blockDim.x >> 5) + warp;
  if (r >= nc) return;
  const double* a = Ainv + (size_t)r * nc;
  double s = 0.0;
  for (int c = lane; c < nc; c += 32) s += a[c] * (fv[c] - mean);
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) x[r] = (T)s;
}

// ---- the BFBt pieces around the two pressure cycles (finest grid) ---------------------------
// u = W^-1 G t (velocity unknowns, padded layout, 0 elsewhere); t compact. (G t) at vx(i, j) is
// (t(i,j) - t(i,j+1)) / dx, at vy(i, j) (t(i,j) - t(i+1,j)) / dy.
template <typename T>
__global__ void k_schur_grad(GeomT<T> g, const T* __restrict__ t, const T* __restrict__ wix, const T* __restrict__ wiy,
                             T* __restrict__ ux, T* __restrict__ uy) {
  const int i = blockIdx.y * blockDim.y + threadIdx.y;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (i > g.ny + 1 || j > g.nx + 1) return;
  const size_t c = (size_t)i * g.ld + j;
  T ox = T(0), oy = T(0);
  if (is_vx(g.nx, g.ny, i, j)) {
    const size_t k = (size_t)(i - 1) * g.nx + (j - 1);
    ox = wix[c] * (t[k] - t[k + 1]) * g.idx;
  }
  if (is_vy(g.nx, g.ny, i, j)) {
    const size_t k = (size_t)(i - 1) * g.nx + (j - 1);
    oy = wiy[c] * (t[k] - t[k + g.nx]) * g.idy;
  }
  ux[c] = ox;
  uy[c] = oy;
}

// w = W^-1 (-L u) at the velocity unknowns (homogeneous boundary rules), 0 elsewhere. With the
// finest velocity level's precomputed coefficient planes (kc, the FP64 path) L u is formed from
// them: about half the FP64 operations of the form from the viscosity, on a path bound by the FP64
// rate.
template <typename T, typename SE>
__global__ void k_schur_lw(GeomT<T> g, const T* __restrict__ ux, const T* __restrict__ uy, const SE* __restrict__ en,
                           const SE* __restrict__ ec, const T* __restrict__ wix, const T* __restrict__ wiy,
                           T* __restrict__ wx, T* __restrict__ wy, Coef<T> kc) {
  const int i = blockIdx.y * blockDim.y + threadIdx.y;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (i > g.ny + 1 || j > g.nx + 1) return;
  const size_t c = (size_t)i * g.ld + j;
  T ox = T(0), oy = T(0), d;
  if (is_vx(g.nx, g.ny, i, j))
    ox = -(kc.cxx ? lx_coef<T>(g, i, j, ux, uy, kc) : lx_point<T>(g, i, j, ux, uy, en, ec, d)) * wix[c];
  if (is_vy(g.nx, g.ny, i, j))
    oy = -(kc.cxx ? ly_coef<T>(g, i, j, ux, uy, kc) : ly_point<T>(g, i, j, ux, uy, en, ec, d)) * wiy[c];
  wx[c] = ox;
  wy[c] = oy;
}

// t = D w (compact), walls 0; x0 = (omega / diag_0) t, the pressure cycle's first Jacobi sweep from zero
template <typename T>
__global__ void k_schur_div(GeomT<T> g, const T* __restrict__ wx, const T* __restrict__ wy, T* __restrict__ t,
                            const T* __restrict__ widg0, T* __restrict__ x0) {
  const int k0 = blockIdx.x * blockDim.x + threadIdx.x;
  if (k0 >= g.nx * g.ny) return;
  const int i = k0 / g.nx + 1, j = k0 % g.nx + 1;
  const size_t c = (size_t)i * g.ld + j;
  const T e = (j <= g.nx - 1) ? wx[c] : T(0);
  const T w = (j - 1 >= 1) ? wx[c - 1] : T(0);
  const T s = (i <= g.ny - 1) ? wy[c] : T(0);
  const T nn = (i - 1 >= 1) ? wy[c - g.ld] : T(0);
  const T v = (e - w) * g.idx + (s - nn) * g.idy;
  t[k0] = v;
  x0[k0] = v * widg0[k0];
}

}  // namespace pyro

namespace pyro {

// As k_precond_out for the velocity planes of Z_j; instead of the diagonal surrogate, y = r_p - D z_v
// goes to the finest pressure grid (compact) for the Schur surrogate, with the pressure cycle's first
// Jacobi sweep from zero x0 = (omega / diag_0) y, and Z_j's pressure plane is left for k_schur_out.
template <typename T, typename TZ, typename TS = T>
__global__ void k_precond_out_schur(GeomT<double> g, const T* __restrict__ vx, const T* __restrict__ vy,
                                    const double* __restrict__ V, size_t vstride, TZ* __restrict__ Z, size_t stride,
                                    const int* __restrict__ d_j, TS* __restrict__ y, const double* __restrict__ isw,
                                    const TS* __restrict__ widg0, TS* __restrict__ x0) {
  const size_t P = (size_t)(g.ny + 2) * g.ld;
  const double* v = V + (size_t)(*d_j) * vstride;
  TZ* z = Z + (size_t)(*d_j) * stride;
  const int cols = g.nx + 2;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < P; e += (size_t)gridDim.x * blockDim.x) {
    int i, j;
    row_col(e, cols, i, j);
    const TZ zx = is_vx(g.nx, g.ny, i, j) ? (TZ)vx[e] : TZ(0);
    const TZ zy = is_vy(g.nx, g.ny, i, j) ? (TZ)vy[e] : TZ(0);
    z[e] = zx;
    z[P + e] = zy;
    if (is_p(g.nx, g.ny, i, j)) {
      const double ux = (double)zx;
      const double uxw = (j - 1 >= 1) ? (double)(TZ)vx[e - 1] : 0.0;
      const double uy = (double)zy;
      const double uyn = (i - 1 >= 1) ? (double)(TZ)vy[e - g.ld] : 0.0;
      const double div = (ux - uxw) * g.idx + (uy - uyn) * g.idy;
      const double rp = isw ? v[2 * P + e] * isw[2 * P + e] : v[2 * P + e];
      const size_t k = (size_t)(i - 1) * g.nx + (j - 1);
      const TS yk = (TS)(rp - div);
      y[k] = yk;
      x0[k] = yk * widg0[k];
    }
  }
}

// Z_j pressure plane <- alpha t (t compact on the finest pressure grid); per-block partial sums for
// the mean removal (k_sub_mean)
template <typename T, typename TZ>
__global__ void k_schur_out(GeomT<double> g, const T* __restrict__ t, double alpha, TZ* __restrict__ Z, size_t stride,
                            const int* __restrict__ d_j, double* __restrict__ part) {
  __shared__ double sh[32];
  const size_t P = (size_t)(g.ny + 2) * g.ld;
  TZ* zp = Z + (size_t)(*d_j) * stride + 2 * P;
  const int cols = g.nx + 2;
  double acc = 0.0;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < P; e += (size_t)gridDim.x * blockDim.x) {
    int i, j;
    row_col(e, cols, i, j);
    double v = 0.0;
    if (is_p(g.nx, g.ny, i, j)) {
      v = (double)(TZ)(alpha * (double)t[(size_t)(i - 1) * g.nx + (j - 1)]);
      acc += v;
    }
    zp[e] = (TZ)v;
  }
  const double s = block_sum(acc, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

}  // namespace pyro
