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
// finest pressure grid, the conductances of its east face cx and south face cy (0 on walls) and the
// diagonal of K (sum of the four face conductances).
template <typename T, typename SE>
__global__ void k_schur_weights(GeomT<T> g, const SE* __restrict__ en, const SE* __restrict__ ec, T* __restrict__ wix,
                                T* __restrict__ wiy, T* __restrict__ cx, T* __restrict__ cy, T* __restrict__ diag) {
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
  diag[k] = ce + cw + cs + cn;
}

// One level of the pressure hierarchy as seen by the kernels.
template <typename T>
struct PLev {
  int nx, ny;
  const T* cx;    // finest level: east-face conductances (else null)
  const T* cy;    // finest level: south-face conductances
  const T* box;   // coarse levels: 25 planes of nx*ny coefficients (else null)
  const T* diag;  // diagonal of K
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

// (K x)_k
template <typename T>
__device__ inline T papply(const PLev<T>& L, int i, int j, const T* __restrict__ x) {
  const size_t k = (size_t)i * L.nx + j;
  if (!L.box) {
    T s = L.diag[k] * x[k];
    if (j + 1 < L.nx) s -= L.cx[k] * x[k + 1];
    if (j >= 1) s -= L.cx[k - 1] * x[k - 1];
    if (i + 1 < L.ny) s -= L.cy[k] * x[k + L.nx];
    if (i >= 1) s -= L.cy[k - L.nx] * x[k - L.nx];
    return s;
  }
  const size_t n = (size_t)L.nx * L.ny;
  T s = T(0);
#pragma unroll
  for (int di = -2; di <= 2; ++di) {
    const int ii = i + di;
    if (ii < 0 || ii >= L.ny) continue;
#pragma unroll
    for (int dj = -2; dj <= 2; ++dj) {
      const int jj = j + dj;
      if (jj < 0 || jj >= L.nx) continue;
      s += L.box[(size_t)((di + 2) * 5 + (dj + 2)) * n + k] * x[(size_t)ii * L.nx + jj];
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

// Galerkin coarse operator K_c = P^T K P, one coarse cell per thread, into 25 planes (+ diagonal)
template <typename T>
__global__ void k_schur_rap(PLev<T> L, const T* __restrict__ pw, int nxc, int nyc, T* __restrict__ box,
                            T* __restrict__ cdiag) {
  const int K0 = blockIdx.x * blockDim.x + threadIdx.x;
  const int nc = nxc * nyc;
  if (K0 >= nc) return;
  const int I = K0 / nxc, J = K0 % nxc;
  const int n = L.nx * L.ny;
  T acc[kSchurBox];
#pragma unroll
  for (int q = 0; q < kSchurBox; ++q) acc[q] = T(0);
  for (int ai = 2 * I - 1; ai <= 2 * I + 2; ++ai) {
    if (ai < 0 || ai >= L.ny) continue;
    for (int aj = 2 * J - 1; aj <= 2 * J + 2; ++aj) {
      if (aj < 0 || aj >= L.nx) continue;
      const int sa_i = I - pwin(ai), sa_j = J - pwin(aj);
      if (sa_i < 0 || sa_i > 1 || sa_j < 0 || sa_j > 1) continue;
      const T pa = pw[(size_t)(sa_i * 2 + sa_j) * n + (size_t)ai * L.nx + aj];
      if (pa == T(0)) continue;
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
#pragma unroll
  for (int q = 0; q < kSchurBox; ++q) box[(size_t)q * nc + K0] = acc[q];
  cdiag[K0] = acc[12];
}

// One damped Jacobi sweep x_out = x_in + omega (f - K x_in) / diag (x_in null: from zero)
template <typename T>
__global__ void k_schur_jacobi(PLev<T> L, const T* __restrict__ x_in, T* __restrict__ x_out, const T* __restrict__ f,
                               T omega) {
  const int k0 = blockIdx.x * blockDim.x + threadIdx.x;
  if (k0 >= L.nx * L.ny) return;
  const int i = k0 / L.nx, j = k0 % L.nx;
  if (!x_in) { x_out[k0] = omega * f[k0] / L.diag[k0]; return; }
  x_out[k0] = x_in[k0] + omega * (f[k0] - papply<T>(L, i, j, x_in)) / L.diag[k0];
}

// r = f - K x
template <typename T>
__global__ void k_schur_resid(PLev<T> L, const T* __restrict__ x, const T* __restrict__ f, T* __restrict__ r) {
  const int k0 = blockIdx.x * blockDim.x + threadIdx.x;
  if (k0 >= L.nx * L.ny) return;
  r[k0] = f[k0] - papply<T>(L, k0 / L.nx, k0 % L.nx, x);
}

// f_c = P^T r
template <typename T>
__global__ void k_schur_restrict(int nx, int ny, const T* __restrict__ pw, const T* __restrict__ r, int nxc, int nyc,
                                 T* __restrict__ fc) {
  const int K0 = blockIdx.x * blockDim.x + threadIdx.x;
  if (K0 >= nxc * nyc) return;
  const int I = K0 / nxc, J = K0 % nxc;
  const size_t n = (size_t)nx * ny;
  T s = T(0);
  for (int ai = 2 * I - 1; ai <= 2 * I + 2; ++ai) {
    if (ai < 0 || ai >= ny) continue;
    const int si = I - pwin(ai);
    if (si < 0 || si > 1) continue;
    for (int aj = 2 * J - 1; aj <= 2 * J + 2; ++aj) {
      if (aj < 0 || aj >= nx) continue;
      const int sj = J - pwin(aj);
      if (sj < 0 || sj > 1) continue;
      const size_t a = (size_t)ai * nx + aj;
      s += pw[(size_t)(si * 2 + sj) * n + a] * r[a];
    }
  }
  fc[K0] = s;
}

// x += P e_c
template <typename T>
__global__ void k_schur_prolong(int nx, int ny, const T* __restrict__ pw, const T* __restrict__ ec, int nxc, int nyc,
                                T* __restrict__ x) {
  const int k0 = blockIdx.x * blockDim.x + threadIdx.x;
  const size_t n = (size_t)nx * ny;
  if (k0 >= (int)n) return;
  const int i = k0 / nx, j = k0 % nx;
  const int oi = pwin(i), oj = pwin(j);
  T s = T(0);
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int Ji = oi + (q >> 1), Jj = oj + (q & 1);
    if (Ji < 0 || Ji >= nyc || Jj < 0 || Jj >= nxc) continue;
    s += pw[(size_t)q * n + k0] * ec[(size_t)Ji * nxc + Jj];
  }
  x[k0] += s;
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

// x = (K_c + s 1 1^T)^-1 (f - mean f), one block, FP64 arithmetic
template <typename T>
__global__ void k_schur_coarse_solve(const double* __restrict__ Ainv, int nc, const T* __restrict__ f,
                                     T* __restrict__ x) {
  __shared__ double fv[kSchurMaxCoarse];
  __shared__ double mean;
  for (int k = threadIdx.x; k < nc; k += blockDim.x) fv[k] = (double)f[k];
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int k = 0; k < nc; ++k) s += fv[k];
    mean = s / nc;
  }
  __syncthreads();
  for (int k = threadIdx.x; k < nc; k += blockDim.x) fv[k] -= mean;
  __syncthreads();
  for (int r = threadIdx.x; r < nc; r += blockDim.x) {
    double s = 0.0;
    const double* a = Ainv + (size_t)r * nc;
    for (int c = 0; c < nc; ++c) s += a[c] * fv[c];
    x[r] = (T)s;
  }
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

// w = W^-1 (-L u) at the velocity unknowns (homogeneous boundary rules), 0 elsewhere
template <typename T, typename SE>
__global__ void k_schur_lw(GeomT<T> g, const T* __restrict__ ux, const T* __restrict__ uy, const SE* __restrict__ en,
                           const SE* __restrict__ ec, const T* __restrict__ wix, const T* __restrict__ wiy,
                           T* __restrict__ wx, T* __restrict__ wy) {
  const int i = blockIdx.y * blockDim.y + threadIdx.y;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (i > g.ny + 1 || j > g.nx + 1) return;
  const size_t c = (size_t)i * g.ld + j;
  T ox = T(0), oy = T(0), d;
  if (is_vx(g.nx, g.ny, i, j)) ox = -lx_point<T>(g, i, j, ux, uy, en, ec, d) * wix[c];
  if (is_vy(g.nx, g.ny, i, j)) oy = -ly_point<T>(g, i, j, ux, uy, en, ec, d) * wiy[c];
  wx[c] = ox;
  wy[c] = oy;
}

// t = D w (compact), walls 0
template <typename T>
__global__ void k_schur_div(GeomT<T> g, const T* __restrict__ wx, const T* __restrict__ wy, T* __restrict__ t) {
  const int k0 = blockIdx.x * blockDim.x + threadIdx.x;
  if (k0 >= g.nx * g.ny) return;
  const int i = k0 / g.nx + 1, j = k0 % g.nx + 1;
  const size_t c = (size_t)i * g.ld + j;
  const T e = (j <= g.nx - 1) ? wx[c] : T(0);
  const T w = (j - 1 >= 1) ? wx[c - 1] : T(0);
  const T s = (i <= g.ny - 1) ? wy[c] : T(0);
  const T nn = (i - 1 >= 1) ? wy[c - g.ld] : T(0);
  t[k0] = (e - w) * g.idx + (s - nn) * g.idy;
}

}  // namespace pyro

namespace pyro {

// As k_precond_out for the velocity planes of Z_j; instead of the diagonal surrogate, y = r_p - D z_v
// goes to the finest pressure grid (compact) for the Schur surrogate, and Z_j's pressure plane is
// left for k_schur_out.
template <typename T, typename TZ>
__global__ void k_precond_out_schur(GeomT<double> g, const T* __restrict__ vx, const T* __restrict__ vy,
                                    const double* __restrict__ V, size_t vstride, TZ* __restrict__ Z, size_t stride,
                                    const int* __restrict__ d_j, T* __restrict__ y, const double* __restrict__ isw) {
  const size_t P = (size_t)(g.ny + 2) * g.ld;
  const double* v = V + (size_t)(*d_j) * vstride;
  TZ* z = Z + (size_t)(*d_j) * stride;
  const int cols = g.nx + 2;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < P; e += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / cols), j = (int)(e % cols);
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
      y[(size_t)(i - 1) * g.nx + (j - 1)] = (T)(rp - div);
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
    const int i = (int)(e / cols), j = (int)(e % cols);
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
