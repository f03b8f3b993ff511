// Inner flexible conjugate gradients on the finest velocity level (option inner_cg; not in the
// paper, whose Uzawa preconditioner applies one V-cycle to the velocity block). k steps of
//   z = V(r);  beta = (z . q) / (d . q);  d <- z - beta d;  q <- L z - beta q;
//   alpha = (r . d) / (d . q);  x += alpha d;  r -= alpha q
// from x = 0, r = f (flexible CG with the one-term recurrence: every direction is made L-conjugate
// to the previous one, which keeps the method exact for a fixed symmetric preconditioner and
// tolerates a varying one). L is the finest level's re-discretised operator. The recurrence runs in
// FP64 whatever the cycle's precision (vectors, the operator with the FP64 viscosity, the dot
// products): in FP32 the residual recurrence drifts at viscosity contrasts of 1e9 and the method
// breaks down. Only the V-cycle sees FP32 (mixed mode): r is rounded into the cycle's right-hand
// side each step, and the result x is rounded back once at the end. Every dot product is reduced on
// the device in a fixed order, so the steps stay inside a captured graph.
#pragma once
#include "common.cuh"

namespace pyro {

// fixed-order block sum of a double (one value per block into part[blockIdx.x])
__device__ inline void fcg_block_sum(double v, double* sh, double* part) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    double s = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
  }
}

// w = L z at the velocity unknowns (0 elsewhere; FP64 operator and viscosity) and block partials of
// z . q (previous q)
template <typename TZ>
__global__ void k_fcg_apply(GeomT<double> g, const TZ* __restrict__ zx, const TZ* __restrict__ zy,
                            const double* __restrict__ en, const double* __restrict__ ec, const double* __restrict__ qx,
                            const double* __restrict__ qy, double* __restrict__ wx, double* __restrict__ wy, int first,
                            double* __restrict__ part) {
  __shared__ double sh[32];
  const size_t P = (size_t)(g.ny + 2) * g.ld;
  const int cols = g.nx + 2;
  double acc = 0.0;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < P; e += (size_t)gridDim.x * blockDim.x) {
    int i, j;
    row_col(e, cols, i, j);
    double ox = 0.0, oy = 0.0, d;
    if (is_vx(g.nx, g.ny, i, j)) {
      ox = lx_point<double>(g, i, j, zx, zy, en, ec, d);
      if (!first) acc += (double)zx[e] * qx[e];
    }
    if (is_vy(g.nx, g.ny, i, j)) {
      oy = ly_point<double>(g, i, j, zx, zy, en, ec, d);
      if (!first) acc += (double)zy[e] * qy[e];
    }
    wx[e] = ox;
    wy[e] = oy;
  }
  fcg_block_sum(acc, sh, part);
}

// scal[0] = beta = (z . q) / (d . q) (0 on the first step), d . q of the previous step in scal[2]
__global__ void k_fcg_beta(const double* __restrict__ part, int nblk, int first, double* __restrict__ scal) {
  __shared__ double sh[32];
  double s = 0.0;
  for (int b = threadIdx.x; b < nblk; b += blockDim.x) s += part[b];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
    scal[0] = (first || scal[2] == 0.0) ? 0.0 : t / scal[2];
  }
}

// d <- z - beta d, q <- w - beta q at the unknowns (0 elsewhere; on the first step d = z, q = w),
// partials of r . d and d . q into part[b] and part[nblk + b]
template <typename TZ>
__global__ void k_fcg_orth(GeomT<double> g, const TZ* __restrict__ zx, const TZ* __restrict__ zy,
                           const double* __restrict__ wx, const double* __restrict__ wy, const double* __restrict__ rx,
                           const double* __restrict__ ry, double* __restrict__ dx, double* __restrict__ dy,
                           double* __restrict__ qx, double* __restrict__ qy, const double* __restrict__ scal, int first,
                           double* __restrict__ part) {
  __shared__ double sh[32];
  const size_t P = (size_t)(g.ny + 2) * g.ld;
  const int cols = g.nx + 2;
  const double beta = first ? 0.0 : scal[0];
  double a1 = 0.0, a2 = 0.0;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < P; e += (size_t)gridDim.x * blockDim.x) {
    int i, j;
    row_col(e, cols, i, j);
    double nx_ = 0.0, ny_ = 0.0, mx = 0.0, my = 0.0;
    if (is_vx(g.nx, g.ny, i, j)) {
      nx_ = first ? (double)zx[e] : (double)zx[e] - beta * dx[e];
      mx = first ? wx[e] : wx[e] - beta * qx[e];
    }
    if (is_vy(g.nx, g.ny, i, j)) {
      ny_ = first ? (double)zy[e] : (double)zy[e] - beta * dy[e];
      my = first ? wy[e] : wy[e] - beta * qy[e];
    }
    dx[e] = nx_; dy[e] = ny_; qx[e] = mx; qy[e] = my;
    a1 += rx[e] * nx_ + ry[e] * ny_;
    a2 += nx_ * mx + ny_ * my;
  }
  fcg_block_sum(a1, sh, part);
  __syncthreads();
  fcg_block_sum(a2, sh, part + gridDim.x);
}

// scal[1] = alpha = (r . d) / (d . q), scal[2] = d . q
__global__ void k_fcg_alpha(const double* __restrict__ part, int nblk, double* __restrict__ scal) {
  __shared__ double sh[2][32];
  double s1 = 0.0, s2 = 0.0;
  for (int b = threadIdx.x; b < nblk; b += blockDim.x) { s1 += part[b]; s2 += part[nblk + b]; }
  for (int o = 16; o > 0; o >>= 1) {
    s1 += __shfl_xor_sync(0xffffffffu, s1, o);
    s2 += __shfl_xor_sync(0xffffffffu, s2, o);
  }
  if ((threadIdx.x & 31) == 0) { sh[0][threadIdx.x >> 5] = s1; sh[1][threadIdx.x >> 5] = s2; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double t1 = 0.0, t2 = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { t1 += sh[0][w]; t2 += sh[1][w]; }
    scal[1] = t2 != 0.0 ? t1 / t2 : 0.0;
    scal[2] = t2;
  }
}

// x += alpha d, r -= alpha q (x zeroed first on step 0)
__global__ void k_fcg_update(size_t P, const double* __restrict__ dx, const double* __restrict__ dy,
                             const double* __restrict__ qx, const double* __restrict__ qy, double* __restrict__ xx,
                             double* __restrict__ xy, double* __restrict__ rx, double* __restrict__ ry,
                             const double* __restrict__ scal, int first) {
  const double alpha = scal[1];
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < P; e += (size_t)gridDim.x * blockDim.x) {
    xx[e] = (first ? 0.0 : xx[e]) + alpha * dx[e];
    xy[e] = (first ? 0.0 : xy[e]) + alpha * dy[e];
    rx[e] -= alpha * qx[e];
    ry[e] -= alpha * qy[e];
  }
}

// r = the velocity part of the preconditioner's input (v = V + (*d_j) stride, unscaled by isw when
// the basis is stored scaled)
__global__ void k_fcg_init(size_t P, const double* __restrict__ V, size_t stride, const int* __restrict__ d_j,
                           const double* __restrict__ isw, double* __restrict__ rx, double* __restrict__ ry) {
  const double* v = V + (size_t)(*d_j) * stride;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < P; e += (size_t)gridDim.x * blockDim.x) {
    rx[e] = isw ? v[e] * isw[e] : v[e];
    ry[e] = isw ? v[P + e] * isw[P + e] : v[P + e];
  }
}

// the cycle's right-hand side <- r (rounded to the cycle's precision) and its first iterate buffer
// zeroed, before each V-cycle
template <typename T>
__global__ void k_fcg_load(size_t P, const double* __restrict__ rx, const double* __restrict__ ry, T* __restrict__ fx,
                           T* __restrict__ fy, T* __restrict__ vx, T* __restrict__ vy) {
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < P; e += (size_t)gridDim.x * blockDim.x) {
    fx[e] = (T)rx[e];
    fy[e] = (T)ry[e];
    vx[e] = T(0);
    vy[e] = T(0);
  }
}

// the result x rounded to the cycle's precision into the level's first iterate buffer
template <typename T>
__global__ void k_fcg_store(size_t P, const double* __restrict__ xx, const double* __restrict__ xy, T* __restrict__ vx,
                            T* __restrict__ vy) {
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < P; e += (size_t)gridDim.x * blockDim.x) {
    vx[e] = (T)xx[e];
    vy[e] = (T)xy[e];
  }
}

}  // namespace pyro
