// Multigrid kernels of the velocity block L (Sec. "The Multigrid Method"), templated on the
// arithmetic type T (float for the mixed-precision V-cycle, double for the plain FP64 one).
//
//  * k_rbgs: one colour of one field of damped red-black Gauss-Seidel (eq. sor_update); the
//    sweep order is vx-red, vx-black, vy-red, vy-black with colour (i + j) mod 2.
//  * k_vresidual: r = f - L x on one level (eq. mg_residual).
//  * k_restrict: normalised bilinear-weighted restriction (Sec. "Restriction"): for factor-2
//    coarsening the bilinear weights are [1,2,1]/4 across node-centred directions and
//    [1,3,3,1]/8 across cell-centred ones; locations that are not unknowns drop out and the
//    normalisation divides by the weights that remain. Each coarse point gathers its own fine
//    support, so no colouring and no atomics are needed.
//  * k_prolong_add: x_fine += P x_coarse, bilinear from the four surrounding coarse points
//    (Sec. "Prolongation"); coarse ghosts follow the homogeneous boundary rule.
//  * k_coarsen_eta: eta_n / eta_c of the next level with the same normalised bilinear weights,
//    arithmetic or on log(eta) (each field transferred on its own, Sec. "Geometric vs Algebraic").
//  * k_coarse_assemble / k_coarse_invert / k_coarse_solve: FP64 direct solve on the coarsest
//    level (Sec. "Multigrid Cycles", coarsest level solved directly): dense -L is assembled,
//    inverted once per set-up by Gauss-Jordan (it is SPD, no pivoting) and applied as a matvec.
#pragma once
#include "common.cuh"

namespace pyro {

// Division of the smoother update: FP32 levels use the fast approximate division (the smoother is
// only a preconditioner; every FP32 path uses this same form), FP64 levels divide exactly.
__device__ inline float sdiv(float a, float b) { return __fdividef(a, b); }
__device__ inline double sdiv(double a, double b) { return a / b; }

// idg (optional): precomputed 1/diag per field (used on FP64 levels, where a division costs far
// more than a load); without it the diagonal is divided inline.
template <typename T>
__device__ inline void rbgs_point(const GeomT<T>& g, int i, int j, int field, T omega, T* vx, T* vy, const T* fx,
                                  const T* fy, const T* en, const T* ec, const T* idgx, const T* idgy,
                                  const Coef<T>& kc = Coef<T>{}) {
  const size_t c = (size_t)i * g.ld + j;
  T diag;
  if (field == 0) {
    if (!is_vx(g.nx, g.ny, i, j)) return;
    if (kc.cxx && idgx) {
      const T t = idgx[c] * (fx[c] - lx_off<T>(g, i, j, vx, vy, kc));
      vx[c] = omega == T(1) ? t : (T(1) - omega) * vx[c] + omega * t;
      return;
    }
    const T Lv = lx_point<T>(g, i, j, vx, vy, en, ec, diag);
    if (idgx) vx[c] += omega * (fx[c] - Lv) * idgx[c];
    else vx[c] += omega * sdiv(fx[c] - Lv, diag);
  } else {
    if (!is_vy(g.nx, g.ny, i, j)) return;
    if (kc.cxx && idgy) {
      const T t = idgy[c] * (fy[c] - ly_off<T>(g, i, j, vx, vy, kc));
      vy[c] = omega == T(1) ? t : (T(1) - omega) * vy[c] + omega * t;
      return;
    }
    const T Lv = ly_point<T>(g, i, j, vx, vy, en, ec, diag);
    if (idgy) vy[c] += omega * (fy[c] - Lv) * idgy[c];
    else vy[c] += omega * sdiv(fy[c] - Lv, diag);
  }
}

template <typename T>
__global__ void k_invdiag(GeomT<T> g, const T* __restrict__ en, const T* __restrict__ ec, T* __restrict__ idgx,
                          T* __restrict__ idgy) {
  const int i = blockIdx.y * blockDim.y + threadIdx.y;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (i > g.ny + 1 || j > g.nx + 1) return;
  const size_t c = (size_t)i * g.ld + j;
  T ox = T(0), oy = T(0);
  if (is_vx(g.nx, g.ny, i, j)) {
    T d = -T(2) * (ec[c] + ec[c + 1]) * g.idx2 - (en[c - g.ld] + en[c]) * g.idy2;
    if (i == 1) d += g.sN * en[c - g.ld] * g.idy2;
    if (i == g.ny) d += g.sS * en[c] * g.idy2;
    ox = T(1) / d;
  }
  if (is_vy(g.nx, g.ny, i, j)) {
    T d = -T(2) * (ec[c] + ec[c + g.ld]) * g.idy2 - (en[c - 1] + en[c]) * g.idx2;
    if (j == 1) d += g.sW * en[c - 1] * g.idx2;
    if (j == g.nx) d += g.sE * en[c] * g.idx2;
    oy = T(1) / d;
  }
  idgx[c] = ox;
  idgy[c] = oy;
}

// Coefficient-form update of rbgs_point with the undamped case (omega = 1) fixed at compile time,
// so the damped form's extra multiplies and the read of the old value are not computed there.
template <typename T, bool UNDAMPED>
__device__ inline void rbgs_coef_point(const GeomT<T>& g, int i, int j, int field, T omega, T* vx, T* vy,
                                       const T* fx, const T* fy, const T* idgx, const T* idgy, const Coef<T>& kc) {
  const size_t c = (size_t)i * g.ld + j;
  if (field == 0) {
    if (!is_vx(g.nx, g.ny, i, j)) return;
    const T t = idgx[c] * (fx[c] - lx_off<T>(g, i, j, vx, vy, kc));
    vx[c] = UNDAMPED ? t : (T(1) - omega) * vx[c] + omega * t;
  } else {
    if (!is_vy(g.nx, g.ny, i, j)) return;
    const T t = idgy[c] * (fy[c] - ly_off<T>(g, i, j, vx, vy, kc));
    vy[c] = UNDAMPED ? t : (T(1) - omega) * vy[c] + omega * t;
  }
}

template <typename T>
__global__ void k_rbgs(GeomT<T> g, T* __restrict__ vx, T* __restrict__ vy, const T* __restrict__ fx,
                       const T* __restrict__ fy, const T* __restrict__ en, const T* __restrict__ ec,
                       int field, int colour, T omega, const T* __restrict__ idgx, const T* __restrict__ idgy,
                       Coef<T> kc) {
  const int i = blockIdx.y * blockDim.y + threadIdx.y;
  const int jh = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = 2 * jh + ((i + colour) & 1);
  if (i > g.ny + 1 || j > g.nx + 1) return;
  if (kc.cxx && idgx) {   // launch-uniform branches
    if (omega == T(1)) rbgs_coef_point<T, true>(g, i, j, field, omega, vx, vy, fx, fy, idgx, idgy, kc);
    else rbgs_coef_point<T, false>(g, i, j, field, omega, vx, vy, fx, fy, idgx, idgy, kc);
    return;
  }
  rbgs_point<T>(g, i, j, field, omega, vx, vy, fx, fy, en, ec, idgx, idgy, kc);
}

// coefficient arrays of one level (see Coef)
template <typename T>
__global__ void k_coefs(GeomT<T> g, const T* __restrict__ en, const T* __restrict__ ec, T* __restrict__ cxx,
                        T* __restrict__ cyy, T* __restrict__ nxx, T* __restrict__ nyy, T* __restrict__ nxy) {
  const int i = blockIdx.y * blockDim.y + threadIdx.y;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (i > g.ny + 1 || j > g.nx + 1) return;
  const size_t c = (size_t)i * g.ld + j;
  const T e = ec[c], n = en[c];
  cxx[c] = T(2) * e * g.idx2;
  cyy[c] = T(2) * e * g.idy2;
  nxx[c] = n * g.idx2;
  nyy[c] = n * g.idy2;
  nxy[c] = n * g.idxdy;
}

template <typename T>
__device__ inline void vresid_point(const GeomT<T>& g, int i, int j, const T* vx, const T* vy, const T* fx,
                                    const T* fy, const T* en, const T* ec, T* rx, T* ry,
                                    const Coef<T>& kc = Coef<T>{}) {
  const size_t c = (size_t)i * g.ld + j;
  T d, ox = T(0), oy = T(0);
  if (is_vx(g.nx, g.ny, i, j))
    ox = fx[c] - (kc.cxx ? lx_coef<T>(g, i, j, vx, vy, kc) : lx_point<T>(g, i, j, vx, vy, en, ec, d));
  if (is_vy(g.nx, g.ny, i, j))
    oy = fy[c] - (kc.cxx ? ly_coef<T>(g, i, j, vx, vy, kc) : ly_point<T>(g, i, j, vx, vy, en, ec, d));
  rx[c] = ox;
  ry[c] = oy;
}

template <typename T>
__global__ void k_vresidual(GeomT<T> g, const T* __restrict__ vx, const T* __restrict__ vy,
                            const T* __restrict__ fx, const T* __restrict__ fy, const T* __restrict__ en,
                            const T* __restrict__ ec, T* __restrict__ rx, T* __restrict__ ry, Coef<T> kc) {
  const int i = blockIdx.y * blockDim.y + threadIdx.y;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (i > g.ny + 1 || j > g.nx + 1) return;
  if (kc.cxx) vresid_point<T>(g, i, j, vx, vy, fx, fy, en, ec, rx, ry, kc);   // launch-uniform
  else vresid_point<T>(g, i, j, vx, vy, fx, fy, en, ec, rx, ry, Coef<T>{});
}

// r = f - L x on the finest level of an FP32 cycle with the products and sums formed in FP64: x
// and f are read in their storage type, L is the FP64 outer operator (its precomputed coefficient
// planes), and r is rounded to the storage type once. Where viscosity jumps by many orders of
// magnitude the FP32 form cancels terms of eta / h^2 against each other; this form keeps the
// residual of the stored iterate exact to FP64 before the restriction.
template <typename T>
__global__ void k_vresidual64(GeomT<double> g, const T* __restrict__ vx, const T* __restrict__ vy,
                              const T* __restrict__ fx, const T* __restrict__ fy, Coef<double> kc,
                              T* __restrict__ rx, T* __restrict__ ry) {
  const int i = blockIdx.y * blockDim.y + threadIdx.y;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (i > g.ny + 1 || j > g.nx + 1) return;
  const size_t c = (size_t)i * g.ld + j;
  double ox = 0.0, oy = 0.0;
  if (is_vx(g.nx, g.ny, i, j)) ox = (double)fx[c] - lx_coef<double>(g, i, j, vx, vy, kc);
  if (is_vy(g.nx, g.ny, i, j)) oy = (double)fy[c] - ly_coef<double>(g, i, j, vx, vy, kc);
  rx[c] = (T)ox;
  ry[c] = (T)oy;
}

template <typename T>
__device__ inline void restrict_point(const GeomT<T>& gf, const GeomT<T>& gc, int I, int J, const T* rx,
                                      const T* ry, T* fxc, T* fyc) {
  const size_t C = (size_t)I * gc.ld + J;
  const T w4[4] = {T(1), T(3), T(3), T(1)};
  const T w3[3] = {T(1), T(2), T(1)};
  T ox = T(0), oy = T(0);
  // FP64 levels: away from the walls all twelve taps are present and the weights sum to 32, so
  // the same sum in the same order is scaled by 1/32 (exact, equal to the division by the summed
  // weights) without the weight sum and the FP64 division (B300's FP64 rate is low).
  if (is_vx(gc.nx, gc.ny, I, J)) {
    // rows 2I-2 .. 2I+1 (cell-centred direction), columns 2J-1 .. 2J+1 (node direction)
    T s = T(0);
    if (sizeof(T) == 8 && 2 * I - 2 >= 1 && 2 * I + 1 <= gf.ny) {
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) s += w4[a] * w3[b] * rx[(size_t)(2 * I - 2 + a) * gf.ld + 2 * J - 1 + b];
      ox = s * T(0.03125);
    } else {
      T ws = T(0);
      for (int a = 0; a < 4; ++a) {
        const int i = 2 * I - 2 + a;
        if (i < 1 || i > gf.ny) continue;
        for (int b = 0; b < 3; ++b) {
          const int j = 2 * J - 1 + b;
          const T w = w4[a] * w3[b];
          s += w * rx[(size_t)i * gf.ld + j];
          ws += w;
        }
      }
      ox = s / ws;
    }
  }
  if (is_vy(gc.nx, gc.ny, I, J)) {
    T s = T(0);
    if (sizeof(T) == 8 && 2 * J - 2 >= 1 && 2 * J + 1 <= gf.nx) {
#pragma unroll
      for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) s += w3[a] * w4[b] * ry[(size_t)(2 * I - 1 + a) * gf.ld + 2 * J - 2 + b];
      oy = s * T(0.03125);
    } else {
      T ws = T(0);
      for (int a = 0; a < 3; ++a) {
        const int i = 2 * I - 1 + a;
        for (int b = 0; b < 4; ++b) {
          const int j = 2 * J - 2 + b;
          if (j < 1 || j > gf.nx) continue;
          const T w = w3[a] * w4[b];
          s += w * ry[(size_t)i * gf.ld + j];
          ws += w;
        }
      }
      oy = s / ws;
    }
  }
  fxc[C] = ox;
  fyc[C] = oy;
}


template <typename T>
// with vxc / vyc given, the coarse iterate is zeroed in the same pass (the cycle starts from 0)
__global__ void k_restrict(GeomT<T> gf, GeomT<T> gc, const T* __restrict__ rx, const T* __restrict__ ry,
                           T* __restrict__ fxc, T* __restrict__ fyc, T* __restrict__ vxc, T* __restrict__ vyc) {
  const int I = blockIdx.y * blockDim.y + threadIdx.y;
  const int J = blockIdx.x * blockDim.x + threadIdx.x;
  if (I > gc.ny + 1 || J > gc.nx + 1) return;
  restrict_point<T>(gf, gc, I, J, rx, ry, fxc, fyc);
  if (vxc) {
    const size_t C = (size_t)I * gc.ld + J;
    vxc[C] = T(0);
    vyc[C] = T(0);
  }
}

template <typename T>
__device__ inline T coarse_vx(const GeomT<T>& gc, const T* vxc, int I, int J) {
  if (J <= 0 || J >= gc.nx) return T(0);
  if (I == 0) return gc.sN * vxc[(size_t)1 * gc.ld + J];
  if (I == gc.ny + 1) return gc.sS * vxc[(size_t)gc.ny * gc.ld + J];
  return vxc[(size_t)I * gc.ld + J];
}
template <typename T>
__device__ inline T coarse_vy(const GeomT<T>& gc, const T* vyc, int I, int J) {
  if (I <= 0 || I >= gc.ny) return T(0);
  if (J == 0) return gc.sW * vyc[(size_t)I * gc.ld + 1];
  if (J == gc.nx + 1) return gc.sE * vyc[(size_t)I * gc.ld + gc.nx];
  return vyc[(size_t)I * gc.ld + J];
}

// bilinear coarse-to-fine increments at a fine vx / vy unknown (rows and columns follow the
// node-centred or cell-centred direction of each component). Branch-free in the node-centred
// direction: a fine node between two coarse nodes takes the mean of the two coarse blends, one
// on a coarse node takes the mean of that blend with itself (exactly the blend), so a warp does
// not run both forms (B300's FP64 pipe makes such divergence expensive).
template <typename T>
__device__ inline T prolong_vx_inc(const GeomT<T>& gc, int i, int j, const T* vxc) {
  const int I0 = i >> 1;                         // (i - 1) / 2 for odd i, i / 2 for even i
  const T wy0 = (i & 1) ? T(0.25) : T(0.75);
  const T wy1 = T(1) - wy0;
  const int Ja = j >> 1, Jb = Ja + (j & 1);
  const T a = wy0 * coarse_vx(gc, vxc, I0, Ja) + wy1 * coarse_vx(gc, vxc, I0 + 1, Ja);
  const T b = wy0 * coarse_vx(gc, vxc, I0, Jb) + wy1 * coarse_vx(gc, vxc, I0 + 1, Jb);
  return T(0.5) * (a + b);
}

template <typename T>
__device__ inline T prolong_vy_inc(const GeomT<T>& gc, int i, int j, const T* vyc) {
  const int J0 = j >> 1;
  const T wx0 = (j & 1) ? T(0.25) : T(0.75);
  const T wx1 = T(1) - wx0;
  const int Ia = i >> 1, Ib = Ia + (i & 1);
  const T a = wx0 * coarse_vy(gc, vyc, Ia, J0) + wx1 * coarse_vy(gc, vyc, Ia, J0 + 1);
  const T b = wx0 * coarse_vy(gc, vyc, Ib, J0) + wx1 * coarse_vy(gc, vyc, Ib, J0 + 1);
  return T(0.5) * (a + b);
}

template <typename T>
__device__ inline void prolong_point(const GeomT<T>& gf, const GeomT<T>& gc, int i, int j, T* vxf, T* vyf,
                                     const T* vxc, const T* vyc) {
  const size_t c = (size_t)i * gf.ld + j;
  if (is_vx(gf.nx, gf.ny, i, j)) vxf[c] += prolong_vx_inc(gc, i, j, vxc);
  if (is_vy(gf.nx, gf.ny, i, j)) vyf[c] += prolong_vy_inc(gc, i, j, vyc);
}

template <typename T>
__global__ void k_prolong_add(GeomT<T> gf, GeomT<T> gc, T* __restrict__ vxf, T* __restrict__ vyf,
                              const T* __restrict__ vxc, const T* __restrict__ vyc) {
  const int i = blockIdx.y * blockDim.y + threadIdx.y;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (i > gf.ny + 1 || j > gf.nx + 1) return;
  prolong_point<T>(gf, gc, i, j, vxf, vyf, vxc, vyc);
}

template <typename T>
__global__ void k_coarsen_eta(GeomT<T> gf, GeomT<T> gc, const T* __restrict__ enf, const T* __restrict__ ecf,
                              T* __restrict__ enc, T* __restrict__ ecc, int geometric) {
  const int I = blockIdx.y * blockDim.y + threadIdx.y;
  const int J = blockIdx.x * blockDim.x + threadIdx.x;
  if (I > gc.ny + 1 || J > gc.nx + 1) return;
  const size_t C = (size_t)I * gc.ld + J;
  const T w4[4] = {T(1), T(3), T(3), T(1)};
  const T w3[3] = {T(1), T(2), T(1)};
  T on = T(0), oc = T(0);
  if (I <= gc.ny && J <= gc.nx) {
    T s = T(0), ws = T(0);
    for (int a = 0; a < 3; ++a) {
      const int i = 2 * I - 1 + a;
      if (i < 0 || i > gf.ny) continue;
      for (int b = 0; b < 3; ++b) {
        const int j = 2 * J - 1 + b;
        if (j < 0 || j > gf.nx) continue;
        const T w = w3[a] * w3[b];
        const T e = enf[(size_t)i * gf.ld + j];
        s += w * (geometric ? log(e) : e);
        ws += w;
      }
    }
    on = geometric ? exp(s / ws) : s / ws;
  }
  if (I >= 1 && I <= gc.ny && J >= 1 && J <= gc.nx) {
    T s = T(0), ws = T(0);
    for (int a = 0; a < 4; ++a) {
      const int i = 2 * I - 2 + a;
      if (i < 1 || i > gf.ny) continue;
      for (int b = 0; b < 4; ++b) {
        const int j = 2 * J - 2 + b;
        if (j < 1 || j > gf.nx) continue;
        const T w = w4[a] * w4[b];
        const T e = ecf[(size_t)i * gf.ld + j];
        s += w * (geometric ? log(e) : e);
        ws += w;
      }
    }
    oc = geometric ? exp(s / ws) : s / ws;
  }
  enc[C] = on;
  ecc[C] = oc;
}

// ---- K-cycle (recursive Krylov cycle): the coarse correction of level l is obtained by two
// flexible-CG steps on level l+1 preconditioned by the level-(l+1) cycle. All vectors live on
// level l+1. The residual of the CG iteration is kept in f (the cycle's right-hand side).
// Dot products accumulate in double with one partial per block (fixed block count, fixed order).

template <typename T>
__device__ inline double kc_block_sum(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s += sh[k];
  return s;
}

// step 1: d1 = z1 (= x), q1 = L d1; partials [rc.d1, d1.q1] -> part[2*blk + {0,1}]
template <typename T>
__global__ void k_kc_step1(GeomT<T> g, const T* __restrict__ xx, const T* __restrict__ xy,
                           const T* __restrict__ fx, const T* __restrict__ fy, const T* __restrict__ en,
                           const T* __restrict__ ec, T* __restrict__ d1x, T* __restrict__ d1y,
                           T* __restrict__ q1x, T* __restrict__ q1y, double* __restrict__ part) {
  __shared__ double sh[32];
  const size_t P = (size_t)(g.ny + 2) * g.ld;
  const int cols = g.nx + 2;
  double a = 0.0, b = 0.0;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < P; e += (size_t)gridDim.x * blockDim.x) {
    int i, j;
    row_col(e, cols, i, j);
    T d, qx = T(0), qy = T(0), zx = T(0), zy = T(0);
    if (is_vx(g.nx, g.ny, i, j)) { zx = xx[e]; qx = lx_point<T>(g, i, j, xx, xy, en, ec, d); }
    if (is_vy(g.nx, g.ny, i, j)) { zy = xy[e]; qy = ly_point<T>(g, i, j, xx, xy, en, ec, d); }
    d1x[e] = zx; d1y[e] = zy; q1x[e] = qx; q1y[e] = qy;
    a += (double)fx[e] * zx + (double)fy[e] * zy;
    b += (double)zx * qx + (double)zy * qy;
  }
  a = kc_block_sum<T>(a, sh);
  b = kc_block_sum<T>(b, sh);
  if (threadIdx.x == 0) { part[2 * blockIdx.x] = a; part[2 * blockIdx.x + 1] = b; }
}

// out[k] = sum_b part[nval*b + k], one block, fixed order
__global__ void k_kc_reduce(const double* __restrict__ part, int nblk, int nval, double* __restrict__ out) {
  __shared__ double sh[32];
  for (int k = 0; k < nval; ++k) {
    double s = 0.0;
    for (int b = threadIdx.x; b < nblk; b += blockDim.x) s += part[nval * b + k];
    s = kc_block_sum<double>(s, sh);
    if (threadIdx.x == 0) out[k] = s;
  }
}

// alpha1 = (rc.d1)/(d1.q1); e = alpha1 d1; rc -= alpha1 q1 (in f); x = 0
template <typename T>
__global__ void k_kc_update1(size_t P, const double* __restrict__ s1, const T* __restrict__ d1x,
                             const T* __restrict__ d1y, const T* __restrict__ q1x, const T* __restrict__ q1y,
                             T* __restrict__ ex, T* __restrict__ ey, T* __restrict__ fx, T* __restrict__ fy,
                             T* __restrict__ xx, T* __restrict__ xy) {
  const double den = s1[1];
  const T a1 = (den != 0.0 && isfinite(den)) ? (T)(s1[0] / den) : T(0);
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < P; e += (size_t)gridDim.x * blockDim.x) {
    ex[e] = a1 * d1x[e];
    ey[e] = a1 * d1y[e];
    fx[e] -= a1 * q1x[e];
    fy[e] -= a1 * q1y[e];
    xx[e] = T(0);
    xy[e] = T(0);
  }
}

// step 2 (z2 = x): partials [z2.q1, z2.L z2, rc.z2] -> part[3*blk + {0,1,2}]
template <typename T>
__global__ void k_kc_step2(GeomT<T> g, const T* __restrict__ xx, const T* __restrict__ xy,
                           const T* __restrict__ fx, const T* __restrict__ fy, const T* __restrict__ en,
                           const T* __restrict__ ec, const T* __restrict__ q1x, const T* __restrict__ q1y,
                           double* __restrict__ part) {
  __shared__ double sh[32];
  const size_t P = (size_t)(g.ny + 2) * g.ld;
  const int cols = g.nx + 2;
  double a = 0.0, b = 0.0, c = 0.0;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < P; e += (size_t)gridDim.x * blockDim.x) {
    int i, j;
    row_col(e, cols, i, j);
    T d;
    if (is_vx(g.nx, g.ny, i, j)) {
      const T z = xx[e], Lz = lx_point<T>(g, i, j, xx, xy, en, ec, d);
      a += (double)z * q1x[e]; b += (double)z * Lz; c += (double)fx[e] * z;
    }
    if (is_vy(g.nx, g.ny, i, j)) {
      const T z = xy[e], Lz = ly_point<T>(g, i, j, xx, xy, en, ec, d);
      a += (double)z * q1y[e]; b += (double)z * Lz; c += (double)fy[e] * z;
    }
  }
  a = kc_block_sum<T>(a, sh);
  b = kc_block_sum<T>(b, sh);
  c = kc_block_sum<T>(c, sh);
  if (threadIdx.x == 0) { part[3 * blockIdx.x] = a; part[3 * blockIdx.x + 1] = b; part[3 * blockIdx.x + 2] = c; }
}

// d2 = z2 - beta d1 with beta = (z2.q1)/(d1.q1); since rc.d1 = 0 after step 1 and L = L^T,
// rc.d2 = rc.z2 and d2.L d2 = z2.L z2 - 2 beta z2.q1 + beta^2 d1.q1; x = e + alpha2 d2.
template <typename T>
__global__ void k_kc_final(size_t P, const double* __restrict__ s1, const double* __restrict__ s2,
                           const T* __restrict__ d1x, const T* __restrict__ d1y, const T* __restrict__ ex,
                           const T* __restrict__ ey, T* __restrict__ xx, T* __restrict__ xy) {
  const double dq = s1[1];
  const double beta = (dq != 0.0 && isfinite(dq)) ? s2[0] / dq : 0.0;
  const double den = s2[1] - 2.0 * beta * s2[0] + beta * beta * dq;
  const double a2 = (den != 0.0 && isfinite(den)) ? s2[2] / den : 0.0;
  const T A2 = (T)a2, B = (T)beta;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < P; e += (size_t)gridDim.x * blockDim.x) {
    xx[e] = ex[e] + A2 * (xx[e] - B * d1x[e]);
    xy[e] = ey[e] + A2 * (xy[e] - B * d1y[e]);
  }
}

// ---- coarsest level: unknown numbering vx (row-major over i in [1,ny], j in [1,nx-1]) then vy
__host__ __device__ inline int coarse_n(int nx, int ny) { return ny * (nx - 1) + (ny - 1) * nx; }

template <typename T>
__global__ void k_coarse_assemble(Geom g, const T* __restrict__ en, const T* __restrict__ ec,
                                  double* __restrict__ A, int n) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const int nx = g.nx, ny = g.ny, ld = g.ld;
  const int nvx = ny * (nx - 1);
  const double idx2 = 1.0 / (g.dx * g.dx), idy2 = 1.0 / (g.dy * g.dy), ixy = 1.0 / (g.dx * g.dy);
  auto VX = [&](int i, int j) { return (i - 1) * (nx - 1) + (j - 1); };
  auto VY = [&](int i, int j) { return nvx + (i - 1) * nx + (j - 1); };
  double* row = A + (size_t)k * n;
  // row entries are those of -L
  if (k < nvx) {
    const int i = k / (nx - 1) + 1, j = k % (nx - 1) + 1;
    const size_t c = (size_t)i * ld + j;
    const double eA = ec[c], eB = ec[c + 1], e1 = en[c - ld], e2 = en[c];
    double d = -2.0 * (eA + eB) * idx2 - (e1 + e2) * idy2;
    if (i == 1) d += g.sN * e1 * idy2;
    if (i == ny) d += g.sS * e2 * idy2;
    row[k] = -d;
    if (j - 1 >= 1) row[VX(i, j - 1)] = -2.0 * eA * idx2;
    if (j + 1 <= nx - 1) row[VX(i, j + 1)] = -2.0 * eB * idx2;
    if (i >= 2) row[VX(i - 1, j)] = -e1 * idy2;
    if (i <= ny - 1) row[VX(i + 1, j)] = -e2 * idy2;
    if (i - 1 >= 1) { row[VY(i - 1, j)] = -e1 * ixy; row[VY(i - 1, j + 1)] = e1 * ixy; }
    if (i <= ny - 1) { row[VY(i, j)] = e2 * ixy; row[VY(i, j + 1)] = -e2 * ixy; }
  } else {
    const int kk = k - nvx;
    const int i = kk / nx + 1, j = kk % nx + 1;
    const size_t c = (size_t)i * ld + j;
    const double eA = ec[c], eB = ec[c + ld], e1 = en[c - 1], e2 = en[c];
    double d = -2.0 * (eA + eB) * idy2 - (e1 + e2) * idx2;
    if (j == 1) d += g.sW * e1 * idx2;
    if (j == nx) d += g.sE * e2 * idx2;
    row[k] = -d;
    if (i - 1 >= 1) row[VY(i - 1, j)] = -2.0 * eA * idy2;
    if (i + 1 <= ny - 1) row[VY(i + 1, j)] = -2.0 * eB * idy2;
    if (j >= 2) row[VY(i, j - 1)] = -e1 * idx2;
    if (j <= nx - 1) row[VY(i, j + 1)] = -e2 * idx2;
    if (j <= nx - 1) { row[VX(i + 1, j)] = -e2 * ixy; row[VX(i, j)] = e2 * ixy; }
    if (j - 1 >= 1) { row[VX(i + 1, j - 1)] = e1 * ixy; row[VX(i, j - 1)] = -e1 * ixy; }
  }
}

// In-place Gauss-Jordan inversion of the SPD matrix A (n x n) by one thread block.
__global__ void k_coarse_invert(double* __restrict__ A, int n, int* __restrict__ flag) {
  extern __shared__ double col[];
  for (int k = 0; k < n; ++k) {
    for (int i = threadIdx.x; i < n; i += blockDim.x) col[i] = A[(size_t)i * n + k];
    __syncthreads();
    const double piv = col[k];
    if (!(piv > 0.0)) {  // not SPD or non-finite: report and leave
      if (threadIdx.x == 0) atomicOr(flag, FLAG_BREAKDOWN);
      return;
    }
    const double ip = 1.0 / piv;
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
      double* a = A + (size_t)k * n + j;
      *a = (j == k) ? ip : (*a) * ip;
    }
    __syncthreads();
    const size_t total = (size_t)n * n;
    for (size_t e = threadIdx.x; e < total; e += blockDim.x) {
      const int i = (int)(e / n), j = (int)(e % n);
      if (i == k) continue;
      const double f = col[i];
      if (j == k) A[e] = -f * ip;
      else A[e] -= f * A[(size_t)k * n + j];
    }
    __syncthreads();
  }
}

// Sixteen Gauss-Jordan pivots of the same inversion at once, spread over the whole GPU, out of
// place (B from A) so that no element is read after another CTA has rewritten it. With K the pivot
// set k0 .. k0 + nb - 1 (nb = min(16, n - k0)) and P = A[K, K]:
//   pivot rows:    B[K, c] = P^-1 A[K, c] for c outside K,          B[K, K] = P^-1
//   other rows i:  B[i, c] = A[i, c] - A[i, K] B[K, c] for c outside K,   B[i, K] = -A[i, K] P^-1
// which in exact arithmetic is nb successive single-pivot steps of k_coarse_invert (block
// Gauss-Jordan). Each CTA owns a 32 x 32 output tile; it inverts P itself (single-pivot steps on
// 16 x 16 in shared memory) and forms the pivot rows of its own 32 columns. One launch per pivot
// (n launches, each a few microseconds of launch latency) made the set-up of a 480-unknown
// coarsest level take about 4 ms; sixteen per launch take n / 16 launches. A pivot <= 0 (the
// matrix is not SPD, or non-finite) raises FLAG_BREAKDOWN and every CTA copies its tile.
constexpr int kGJB = 16;   // pivots per launch
constexpr int kGJT = 32;   // output tile side
__global__ void __launch_bounds__(256) k_coarse_invert_block(const double* __restrict__ A, double* __restrict__ B,
                                                             int n, int k0, int* __restrict__ flag) {
  __shared__ double P0[kGJB][kGJB + 1], P1[kGJB][kGJB + 1];
  __shared__ double Kr[kGJB][kGJT];       // pivot rows after the step, this CTA's columns
  __shared__ double Ai[kGJT][kGJB + 1];   // A[i, K] of this CTA's rows
  const int nb = min(kGJB, n - k0);
  const int c0 = blockIdx.x * kGJT, r0 = blockIdx.y * kGJT;
  const int tid = threadIdx.x;
  for (int e = tid; e < kGJB * kGJB; e += blockDim.x) {
    const int a = e / kGJB, b = e % kGJB;
    P0[a][b] = (a < nb && b < nb) ? A[(size_t)(k0 + a) * n + k0 + b] : 0.0;
  }
  for (int e = tid; e < kGJT * kGJB; e += blockDim.x) {
    const int r = e / kGJB, t = e % kGJB, i = r0 + r;
    Ai[r][t] = (i < n && t < nb) ? A[(size_t)i * n + k0 + t] : 0.0;
  }
  __syncthreads();
  // P^-1 by nb single-pivot steps; every thread reads the same pivot, so the exit is uniform
  double(*S)[kGJB + 1] = P0;
  double(*D)[kGJB + 1] = P1;
  bool ok = true;
  for (int t = 0; t < nb; ++t) {
    const double piv = S[t][t];
    if (!(piv > 0.0)) { ok = false; break; }
    const double ip = 1.0 / piv;
    for (int e = tid; e < nb * nb; e += blockDim.x) {
      const int a = e / nb, b = e % nb;
      const double stb = (b == t) ? ip : S[t][b] * ip;
      D[a][b] = (a == t) ? stb : ((b == t) ? -S[a][t] * ip : S[a][b] - S[a][t] * stb);
    }
    __syncthreads();
    double(*X)[kGJB + 1] = S;
    S = D;
    D = X;
  }
  if (!ok) {
    if (tid == 0 && blockIdx.x == 0 && blockIdx.y == 0) atomicOr(flag, FLAG_BREAKDOWN);
    for (int e = tid; e < kGJT * kGJT; e += blockDim.x) {
      const int i = r0 + e / kGJT, c = c0 + e % kGJT;
      if (i < n && c < n) B[(size_t)i * n + c] = A[(size_t)i * n + c];
    }
    return;
  }
  for (int e = tid; e < kGJB * kGJT; e += blockDim.x) {
    const int a = e / kGJT, cc = e % kGJT, c = c0 + cc;
    double v = 0.0;
    if (a < nb && c < n) {
      if (c >= k0 && c < k0 + nb) {
        v = S[a][c - k0];
      } else {
        for (int t = 0; t < nb; ++t) v += S[a][t] * A[(size_t)(k0 + t) * n + c];
      }
    }
    Kr[a][cc] = v;
  }
  __syncthreads();
  for (int e = tid; e < kGJT * kGJT; e += blockDim.x) {
    const int r = e / kGJT, cc = e % kGJT, i = r0 + r, c = c0 + cc;
    if (i >= n || c >= n) continue;
    double v;
    if (i >= k0 && i < k0 + nb) {
      v = Kr[i - k0][cc];
    } else if (c >= k0 && c < k0 + nb) {
      v = 0.0;
      for (int t = 0; t < nb; ++t) v -= Ai[r][t] * S[t][c - k0];
    } else {
      v = A[(size_t)i * n + c];
      for (int t = 0; t < nb; ++t) v -= Ai[r][t] * Kr[t][cc];
    }
    B[(size_t)i * n + c] = v;
  }
}

// x = L^-1 f = -(-L)^-1 f on the coarsest level (FP64 whatever T is). One warp per row of the
// inverse (coalesced row reads, fixed-order shuffle reduction), kCoarseRows rows per CTA, so the
// matvec spreads over ceil(n / kCoarseRows) SMs (one SM's FP64 rate would make it the critical path).
constexpr int kCoarseRows = 8;
template <typename T>
__global__ void __launch_bounds__(32 * kCoarseRows)
    k_coarse_solve(Geom g, const double* __restrict__ Ainv, int n, const T* __restrict__ fx,
                   const T* __restrict__ fy, T* __restrict__ vx, T* __restrict__ vy) {
  extern __shared__ double fv[];
  const int nx = g.nx, ny = g.ny, ld = g.ld, nvx = ny * (nx - 1);
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    if (k < nvx) { const int i = k / (nx - 1) + 1, j = k % (nx - 1) + 1; fv[k] = (double)fx[(size_t)i * ld + j]; }
    else { const int kk = k - nvx; const int i = kk / nx + 1, j = kk % nx + 1; fv[k] = (double)fy[(size_t)i * ld + j]; }
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int k = blockIdx.x * kCoarseRows + (threadIdx.x >> 5);
  if (k >= n) return;
  const double* a = Ainv + (size_t)k * n;
  double s = 0.0;
  for (int l = lane; l < n; l += 32) s += a[l] * fv[l];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane != 0) return;
  if (k < nvx) { const int i = k / (nx - 1) + 1, j = k % (nx - 1) + 1; vx[(size_t)i * ld + j] = (T)(-s); }
  else { const int kk = k - nvx; const int i = kk / nx + 1, j = kk % nx + 1; vy[(size_t)i * ld + j] = (T)(-s); }
}

// ---- transfers between levels of any size ratio ---------------------------------------------
// (the paper's arbitrary coarsening ratio; factor-2 levels use the kernels above). Positions and
// weights are formed in double from the box and the cell counts of both levels: vx at (j dx,
// (i - 1/2) dy), vy at ((j - 1/2) dx, i dy), basic nodes at (j dx, i dy), cells at ((j - 1/2) dx,
// (i - 1/2) dy). The bilinear weight of a fine point for a coarse point is (1 - |x - X|/DX)
// (1 - |y - Y|/DY) where both factors exceed 1e-9 (inside the support), else 0.

// first and last fine index whose position can lie within one coarse spacing of coarse index c
// (r = coarse spacing / fine spacing; off = 1/2 for a cell-centred direction)
__device__ inline void gen_candidates(int c, double r, double off, int lo, int hi, int& a, int& b) {
  a = max((int)floor((c - off - 1.0) * r + off) - 1, lo);
  b = min((int)ceil((c - off + 1.0) * r + off) + 1, hi);
}

__device__ inline double gen_w(double xf, double xc, double H) { return 1.0 - fabs(xf - xc) / H; }

// normalised bilinear restriction of the level residual to every coarse unknown; with vxc / vyc
// given the coarse iterate is zeroed in the same pass
template <typename T>
__global__ void k_restrict_gen(Geom fd, Geom cd, GeomT<T> gf, const T* __restrict__ rx, const T* __restrict__ ry,
                               T* __restrict__ fxc, T* __restrict__ fyc, T* __restrict__ vxc, T* __restrict__ vyc) {
  const int I = blockIdx.y * blockDim.y + threadIdx.y;
  const int J = blockIdx.x * blockDim.x + threadIdx.x;
  if (I > cd.ny + 1 || J > cd.nx + 1) return;
  const size_t C = (size_t)I * cd.ld + J;
  const double rxr = cd.dx / fd.dx, ryr = cd.dy / fd.dy;
  T ox = T(0), oy = T(0);
  if (is_vx(cd.nx, cd.ny, I, J)) {
    const double X = J * cd.dx, Y = (I - 0.5) * cd.dy;
    int i0, i1, j0, j1;
    gen_candidates(I, ryr, 0.5, 0, fd.ny + 1, i0, i1);
    gen_candidates(J, rxr, 0.0, 0, fd.nx + 1, j0, j1);
    double s = 0.0, ws = 0.0;
    for (int i = i0; i <= i1; ++i) {
      const double wy = gen_w((i - 0.5) * fd.dy, Y, cd.dy);
      if (!(wy > 1e-9)) continue;
      for (int j = j0; j <= j1; ++j) {
        if (!is_vx(fd.nx, fd.ny, i, j)) continue;
        const double wx = gen_w(j * fd.dx, X, cd.dx);
        if (!(wx > 1e-9)) continue;
        s += wx * wy * (double)rx[(size_t)i * fd.ld + j];
        ws += wx * wy;
      }
    }
    ox = (T)(s / ws);
  }
  if (is_vy(cd.nx, cd.ny, I, J)) {
    const double X = (J - 0.5) * cd.dx, Y = I * cd.dy;
    int i0, i1, j0, j1;
    gen_candidates(I, ryr, 0.0, 0, fd.ny + 1, i0, i1);
    gen_candidates(J, rxr, 0.5, 0, fd.nx + 1, j0, j1);
    double s = 0.0, ws = 0.0;
    for (int i = i0; i <= i1; ++i) {
      const double wy = gen_w(i * fd.dy, Y, cd.dy);
      if (!(wy > 1e-9)) continue;
      for (int j = j0; j <= j1; ++j) {
        if (!is_vy(fd.nx, fd.ny, i, j)) continue;
        const double wx = gen_w((j - 0.5) * fd.dx, X, cd.dx);
        if (!(wx > 1e-9)) continue;
        s += wx * wy * (double)ry[(size_t)i * fd.ld + j];
        ws += wx * wy;
      }
    }
    oy = (T)(s / ws);
  }
  fxc[C] = ox;
  fyc[C] = oy;
  if (vxc) { vxc[C] = T(0); vyc[C] = T(0); }
}

// x_fine += P x_coarse: bilinear interpolation from the four surrounding coarse points of the
// same family, coarse ghosts by the homogeneous boundary rule (coarse_vx / coarse_vy)
template <typename T>
__global__ void k_prolong_gen(Geom fd, Geom cd, GeomT<T> gc, T* __restrict__ vx, T* __restrict__ vy,
                              const T* __restrict__ cvx, const T* __restrict__ cvy) {
  const int i = blockIdx.y * blockDim.y + threadIdx.y;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (i > fd.ny + 1 || j > fd.nx + 1) return;
  const size_t c = (size_t)i * fd.ld + j;
  for (int fld = 0; fld < 2; ++fld) {
    if (fld == 0 ? !is_vx(fd.nx, fd.ny, i, j) : !is_vy(fd.nx, fd.ny, i, j)) continue;
    const double fx = fld == 0 ? (j * fd.dx) / cd.dx : ((j - 0.5) * fd.dx) / cd.dx + 0.5;
    const double fy = fld == 0 ? ((i - 0.5) * fd.dy) / cd.dy + 0.5 : (i * fd.dy) / cd.dy;
    const int J0 = (int)floor(fx + 1e-12), I0 = (int)floor(fy + 1e-12);
    const double tx = fx - J0, ty = fy - I0;
    double v = 0.0;
    for (int a = 0; a < 2; ++a)
      for (int b = 0; b < 2; ++b) {
        const double w = (a ? ty : 1.0 - ty) * (b ? tx : 1.0 - tx);
        if (!(w > 1e-14)) continue;
        const T cv = fld == 0 ? coarse_vx(gc, cvx, I0 + a, J0 + b) : coarse_vy(gc, cvy, I0 + a, J0 + b);
        v += w * (double)cv;
      }
    if (fld == 0) vx[c] += (T)v;
    else vy[c] += (T)v;
  }
}

// eta on the next level of any ratio: normalised bilinear weights over the real fine nodes /
// cells, arithmetic or on log(eta)
template <typename T>
__global__ void k_coarsen_eta_gen(Geom fd, Geom cd, const T* __restrict__ enf, const T* __restrict__ ecf,
                                  T* __restrict__ enc, T* __restrict__ ecc, int geometric) {
  const int I = blockIdx.y * blockDim.y + threadIdx.y;
  const int J = blockIdx.x * blockDim.x + threadIdx.x;
  if (I > cd.ny + 1 || J > cd.nx + 1) return;
  const size_t C = (size_t)I * cd.ld + J;
  const double rxr = cd.dx / fd.dx, ryr = cd.dy / fd.dy;
  T on = T(0), oc = T(0);
  if (I <= cd.ny && J <= cd.nx) {
    int i0, i1, j0, j1;
    gen_candidates(I, ryr, 0.0, 0, fd.ny, i0, i1);
    gen_candidates(J, rxr, 0.0, 0, fd.nx, j0, j1);
    double s = 0.0, ws = 0.0;
    for (int i = i0; i <= i1; ++i) {
      const double wy = gen_w(i * fd.dy, I * cd.dy, cd.dy);
      if (!(wy > 1e-9)) continue;
      for (int j = j0; j <= j1; ++j) {
        const double wx = gen_w(j * fd.dx, J * cd.dx, cd.dx);
        if (!(wx > 1e-9)) continue;
        const double e = (double)enf[(size_t)i * fd.ld + j];
        s += wx * wy * (geometric ? log(e) : e);
        ws += wx * wy;
      }
    }
    on = (T)(geometric ? exp(s / ws) : s / ws);
  }
  if (I >= 1 && I <= cd.ny && J >= 1 && J <= cd.nx) {
    int i0, i1, j0, j1;
    gen_candidates(I, ryr, 0.5, 1, fd.ny, i0, i1);
    gen_candidates(J, rxr, 0.5, 1, fd.nx, j0, j1);
    double s = 0.0, ws = 0.0;
    for (int i = i0; i <= i1; ++i) {
      const double wy = gen_w((i - 0.5) * fd.dy, (I - 0.5) * cd.dy, cd.dy);
      if (!(wy > 1e-9)) continue;
      for (int j = j0; j <= j1; ++j) {
        const double wx = gen_w((j - 0.5) * fd.dx, (J - 0.5) * cd.dx, cd.dx);
        if (!(wx > 1e-9)) continue;
        const double e = (double)ecf[(size_t)i * fd.ld + j];
        s += wx * wy * (geometric ? log(e) : e);
        ws += wx * wy;
      }
    }
    oc = (T)(geometric ? exp(s / ws) : s / ws);
  }
  enc[C] = on;
  ecc[C] = oc;
}

// ---- explicit instantiations ---------------------------------------------------------------
#define PYRO_INST(T)                                                                                         \
  template __global__ void k_rbgs<T>(GeomT<T>, T*, T*, const T*, const T*, const T*, const T*, int, int, T, \
                                     const T*, const T*, Coef<T>);                                         \
  template __global__ void k_vresidual<T>(GeomT<T>, const T*, const T*, const T*, const T*, const T*,      \
                                          const T*, T*, T*, Coef<T>);                                       \
  template __global__ void k_restrict<T>(GeomT<T>, GeomT<T>, const T*, const T*, T*, T*, T*, T*);          \
  template __global__ void k_restrict_gen<T>(Geom, Geom, GeomT<T>, const T*, const T*, T*, T*, T*, T*);   \
  template __global__ void k_prolong_gen<T>(Geom, Geom, GeomT<T>, T*, T*, const T*, const T*);            \
  template __global__ void k_coarsen_eta_gen<T>(Geom, Geom, const T*, const T*, T*, T*, int);             \
  template __global__ void k_prolong_add<T>(GeomT<T>, GeomT<T>, T*, T*, const T*, const T*);               \
  template __global__ void k_coarsen_eta<T>(GeomT<T>, GeomT<T>, const T*, const T*, T*, T*, int);          \
  template __global__ void k_coarse_assemble<T>(Geom, const T*, const T*, double*, int);                   \
  template __global__ void k_coarse_solve<T>(Geom, const double*, int, const T*, const T*, T*, T*);       \
  template __global__ void k_kc_step1<T>(GeomT<T>, const T*, const T*, const T*, const T*, const T*,      \
                                         const T*, T*, T*, T*, T*, double*);                              \
  template __global__ void k_kc_update1<T>(size_t, const double*, const T*, const T*, const T*, const T*, \
                                           T*, T*, T*, T*, T*, T*);                                        \
  template __global__ void k_kc_step2<T>(GeomT<T>, const T*, const T*, const T*, const T*, const T*,      \
                                         const T*, const T*, const T*, double*);                          \
  template __global__ void k_kc_final<T>(size_t, const double*, const double*, const T*, const T*,        \
                                         const T*, const T*, T*, T*);
PYRO_INST(float)
PYRO_INST(double)
#undef PYRO_INST

}  // namespace pyro
