// Galerkin coarse velocity operators (option galerkin; not in the paper, whose coarse operators are
// re-discretised from transferred viscosity, Sec. "Geometric vs Algebraic Multigrid"). On a factor-2
// level l + 1 the operator is L_{l+1} = R L_l P with the V-cycle's own normalised bilinear
// restriction R and bilinear prolongation P (homogeneous ghosts), so the coarse problem sees the fine
// viscosity exactly instead of an average of it; where the viscosity jumps by many orders of
// magnitude within a coarse cell this keeps the coarse correction consistent with the fine operator.
//
// Stencil of a Galerkin row (offsets in the level's own padded (i, j) indices):
//   vx row: vx at di in [-2, 2], dj in [-1, 1]  (15, slot (di+2)*3 + (dj+1))
//           vy at di in [-2, 1], dj in [-1, 2]  (16, slot 15 + (di+2)*4 + (dj+1))
//   vy row: vy at di in [-1, 1], dj in [-2, 2]  (15, slot (di+1)*5 + (dj+2))
//           vx at di in [-1, 2], dj in [-2, 1]  (16, slot 15 + (di+1)*4 + (dj+2))
// Level storage: 2 * kGalSlots planes of the padded size, plane q for the vx rows and kGalSlots + q
// for the vy rows; entries at non-unknown rows and at slots whose target is not an unknown are 0.
#pragma once
#include "common.cuh"

namespace pyro {

constexpr int kGalSlots = 31;
constexpr int kGalDiag = 7;          // slot of (0, 0) in both the vx and the vy rows
constexpr double kGalOmega = 0.6;    // damped-Jacobi smoothing on Galerkin levels

// slot of a same-field / cross-field coupling, -1 outside the stencil
__host__ __device__ inline int gal_slot(int row_field, int col_field, int di, int dj) {
  if (row_field == 0) {
    if (col_field == 0) return (di >= -2 && di <= 2 && dj >= -1 && dj <= 1) ? (di + 2) * 3 + (dj + 1) : -1;
    return (di >= -2 && di <= 1 && dj >= -1 && dj <= 2) ? 15 + (di + 2) * 4 + (dj + 1) : -1;
  }
  if (col_field == 1) return (di >= -1 && di <= 1 && dj >= -2 && dj <= 2) ? (di + 1) * 5 + (dj + 2) : -1;
  return (di >= -1 && di <= 2 && dj >= -2 && dj <= 1) ? 15 + (di + 1) * 4 + (dj + 2) : -1;
}

// inverse of gal_slot: the (field, di, dj) of slot q of a row of field row_field
__host__ __device__ inline void gal_offset(int row_field, int q, int& col_field, int& di, int& dj) {
  if (row_field == 0) {
    if (q < 15) { col_field = 0; di = q / 3 - 2; dj = q % 3 - 1; }
    else { col_field = 1; di = (q - 15) / 4 - 2; dj = (q - 15) % 4 - 1; }
  } else {
    if (q < 15) { col_field = 1; di = q / 5 - 1; dj = q % 5 - 2; }
    else { col_field = 0; di = (q - 15) / 4 - 1; dj = (q - 15) % 4 - 2; }
  }
}

__host__ __device__ inline bool is_unknown(int field, int nx, int ny, int i, int j) {
  return field == 0 ? is_vx(nx, ny, i, j) : is_vy(nx, ny, i, j);
}

// The entries of one row of the re-discretised operator L (level 0, from the viscosity), with the
// boundary ghosts eliminated as in the point operators: up to 9 (field, i, j, coefficient).
template <typename T, typename SE>
__device__ inline int eta_row(const GeomT<T>& g, int field, int i, int j, const SE* en, const SE* ec, int* cf,
                              int* ci, int* cj, T* cv) {
  const size_t c = (size_t)i * g.ld + j;
  int n = 0;
  auto put = [&](int f, int a, int b, T v) {
    if (!is_unknown(f, g.nx, g.ny, a, b)) return;
    cf[n] = f; ci[n] = a; cj[n] = b; cv[n] = v; ++n;
  };
  if (field == 0) {
    const T eA = (T)ec[c], eB = (T)ec[c + 1], e1 = (T)en[c - g.ld], e2 = (T)en[c];
    T d = -T(2) * (eA + eB) * g.idx2 - (e1 + e2) * g.idy2;
    if (i == 1) d += g.sN * e1 * g.idy2;
    if (i == g.ny) d += g.sS * e2 * g.idy2;
    put(0, i, j, d);
    put(0, i, j + 1, T(2) * eB * g.idx2);
    put(0, i, j - 1, T(2) * eA * g.idx2);
    if (i < g.ny) put(0, i + 1, j, e2 * g.idy2);
    if (i > 1) put(0, i - 1, j, e1 * g.idy2);
    put(1, i, j + 1, e2 * g.idxdy);
    put(1, i, j, -e2 * g.idxdy);
    put(1, i - 1, j + 1, -e1 * g.idxdy);
    put(1, i - 1, j, e1 * g.idxdy);
  } else {
    const T eA = (T)ec[c], eB = (T)ec[c + g.ld], e1 = (T)en[c - 1], e2 = (T)en[c];
    T d = -T(2) * (eA + eB) * g.idy2 - (e1 + e2) * g.idx2;
    if (j == 1) d += g.sW * e1 * g.idx2;
    if (j == g.nx) d += g.sE * e2 * g.idx2;
    put(1, i, j, d);
    put(1, i + 1, j, T(2) * eB * g.idy2);
    put(1, i - 1, j, T(2) * eA * g.idy2);
    if (j < g.nx) put(1, i, j + 1, e2 * g.idx2);
    if (j > 1) put(1, i, j - 1, e1 * g.idx2);
    put(0, i + 1, j, e2 * g.idxdy);
    put(0, i, j, -e2 * g.idxdy);
    put(0, i + 1, j - 1, -e1 * g.idxdy);
    put(0, i, j - 1, e1 * g.idxdy);
  }
  return n;
}

// The factor-2 bilinear prolongation of a fine unknown (field, i, j): up to 4 (coarse i, j, weight)
// of the same field, coarse ghosts folded onto the adjacent interior point with the boundary factor,
// walls dropped (the reading of the oracle's prolongation).
template <typename T>
__device__ inline int prolong_row(const GeomT<T>& gc, int field, int i, int j, int* pi, int* pj, T* pw) {
  int n = 0;
  int I0, J0;
  T ty, tx;
  if (field == 0) {            // fine vx(i, j): coarse x = j / 2, coarse row position (2 i + 1) / 4
    J0 = j >> 1; tx = (j & 1) ? T(0.5) : T(0);
    if (i & 1) { I0 = (i - 1) >> 1; ty = T(0.75); } else { I0 = i >> 1; ty = T(0.25); }
  } else {                     // fine vy(i, j): coarse y = i / 2, coarse column position (2 j + 1) / 4
    I0 = i >> 1; ty = (i & 1) ? T(0.5) : T(0);
    if (j & 1) { J0 = (j - 1) >> 1; tx = T(0.75); } else { J0 = j >> 1; tx = T(0.25); }
  }
  for (int a = 0; a < 2; ++a) {
    const T wy = a ? ty : T(1) - ty;
    if (wy == T(0)) continue;
    for (int b = 0; b < 2; ++b) {
      const T wx = b ? tx : T(1) - tx;
      if (wx == T(0)) continue;
      int I = I0 + a, J = J0 + b;
      T w = wy * wx;
      if (field == 0) {
        if (J <= 0 || J >= gc.nx) continue;                    // wall column: normal velocity 0
        if (I == 0) { I = 1; w *= gc.sN; } else if (I == gc.ny + 1) { I = gc.ny; w *= gc.sS; }
      } else {
        if (I <= 0 || I >= gc.ny) continue;                    // wall row
        if (J == 0) { J = 1; w *= gc.sW; } else if (J == gc.nx + 1) { J = gc.nx; w *= gc.sE; }
      }
      pi[n] = I; pj[n] = J; pw[n] = w; ++n;
    }
  }
  return n;
}

}  // namespace pyro

namespace pyro {

// Row source of a level: the re-discretised operator of the viscosity (level 0 of the Galerkin chain)
// or a stored Galerkin stencil.
template <typename T>
struct GalSrc {
  GeomT<T> g;
  const T* en;    // viscosity (eta source), else null
  const T* ec;
  const T* gal;   // Galerkin planes (stencil source), else null
  size_t P;
};

template <typename T>
__device__ inline int src_row(const GalSrc<T>& S, int field, int i, int j, int* cf, int* ci, int* cj, T* cv) {
  if (!S.gal) return eta_row<T, T>(S.g, field, i, j, S.en, S.ec, cf, ci, cj, cv);
  const size_t c = (size_t)i * S.g.ld + j;
  const T* base = S.gal + (size_t)(field ? kGalSlots : 0) * S.P;
  int n = 0;
  for (int q = 0; q < kGalSlots; ++q) {
    const T v = base[(size_t)q * S.P + c];
    if (v == T(0)) continue;
    int f, di, dj;
    gal_offset(field, q, f, di, dj);
    cf[n] = f; ci[n] = i + di; cj[n] = j + dj; cv[n] = v; ++n;
  }
  return n;
}

// Galerkin coarse rows R L P, one coarse padded point per thread (its vx row and its vy row).
// R: normalised [1,3,3,1] x [1,2,1] weights over fine unknowns (the V-cycle's restriction), P: the
// factor-2 bilinear prolongation. A coupling outside the stencil table (impossible for factor 2)
// raises FLAG_BREAKDOWN instead of being written.
template <typename T>
__global__ void k_gal_rap(GalSrc<T> F, GeomT<T> gc, T* __restrict__ gal, size_t Pc, int* __restrict__ flag) {
  const int I = blockIdx.y * blockDim.y + threadIdx.y;
  const int J = blockIdx.x * blockDim.x + threadIdx.x;
  if (I > gc.ny + 1 || J > gc.nx + 1) return;
  const size_t C = (size_t)I * gc.ld + J;
  const T w4[4] = {T(1), T(3), T(3), T(1)};
  const T w3[3] = {T(1), T(2), T(1)};
  for (int field = 0; field < 2; ++field) {
    T* out = gal + (size_t)(field ? kGalSlots : 0) * Pc;
    T acc[kGalSlots];
#pragma unroll
    for (int q = 0; q < kGalSlots; ++q) acc[q] = T(0);
    if (is_unknown(field, gc.nx, gc.ny, I, J)) {
      // restriction support and its normalisation
      const int na = field == 0 ? 4 : 3, nb = field == 0 ? 3 : 4;
      const int i0 = field == 0 ? 2 * I - 2 : 2 * I - 1, j0 = field == 0 ? 2 * J - 1 : 2 * J - 2;
      T ws = T(0);
      for (int a = 0; a < na; ++a)
        for (int b = 0; b < nb; ++b)
          if (is_unknown(field, F.g.nx, F.g.ny, i0 + a, j0 + b)) ws += (field == 0 ? w4[a] * w3[b] : w3[a] * w4[b]);
      for (int a = 0; a < na; ++a)
        for (int b = 0; b < nb; ++b) {
          const int fi = i0 + a, fj = j0 + b;
          if (!is_unknown(field, F.g.nx, F.g.ny, fi, fj)) continue;
          const T ra = (field == 0 ? w4[a] * w3[b] : w3[a] * w4[b]) / ws;
          int cf[kGalSlots], ci[kGalSlots], cj[kGalSlots];
          T cv[kGalSlots];
          const int nr = src_row<T>(F, field, fi, fj, cf, ci, cj, cv);
          for (int e = 0; e < nr; ++e) {
            int pi[4], pj[4];
            T pw[4];
            const int np = prolong_row<T>(gc, cf[e], ci[e], cj[e], pi, pj, pw);
            for (int k = 0; k < np; ++k) {
              const int q = gal_slot(field, cf[e], pi[k] - I, pj[k] - J);
              if (q < 0) { atomicOr(flag, FLAG_BREAKDOWN); continue; }
              acc[q] += ra * cv[e] * pw[k];
            }
          }
        }
    }
#pragma unroll
    for (int q = 0; q < kGalSlots; ++q) out[(size_t)q * Pc + C] = acc[q];
  }
}

// (L x) of a Galerkin row; targets outside the unknowns carry 0 coefficients and are not read
template <typename T>
__device__ inline T gal_apply(const GeomT<T>& g, const T* __restrict__ gal, size_t P, int field, int i, int j,
                              const T* __restrict__ vx, const T* __restrict__ vy) {
  const size_t c = (size_t)i * g.ld + j;
  const T* base = gal + (size_t)(field ? kGalSlots : 0) * P;
  T s = T(0);
#pragma unroll
  for (int q = 0; q < kGalSlots; ++q) {
    int f, di, dj;
    gal_offset(field, q, f, di, dj);
    const int a = i + di, b = j + dj;
    if (!is_unknown(f, g.nx, g.ny, a, b)) continue;
    s += base[(size_t)q * P + c] * (f ? vy : vx)[(size_t)a * g.ld + b];
  }
  return s;
}

// one damped Jacobi sweep of both fields on a Galerkin level, old iterate in, other buffer out
// (x_in null: from zero)
template <typename T>
__global__ void k_gal_jacobi(GeomT<T> g, const T* __restrict__ gal, size_t P, const T* __restrict__ vx,
                             const T* __restrict__ vy, T* __restrict__ ox, T* __restrict__ oy, const T* __restrict__ fx,
                             const T* __restrict__ fy, T omega) {
  const int i = blockIdx.y * blockDim.y + threadIdx.y;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (i > g.ny + 1 || j > g.nx + 1) return;
  const size_t c = (size_t)i * g.ld + j;
  T rx = T(0), ry = T(0);
  if (is_vx(g.nx, g.ny, i, j)) {
    const T d = gal[(size_t)kGalDiag * P + c];
    const T old = vx ? vx[c] : T(0);
    rx = old + omega * (fx[c] - (vx ? gal_apply<T>(g, gal, P, 0, i, j, vx, vy) : T(0))) / d;
  }
  if (is_vy(g.nx, g.ny, i, j)) {
    const T d = gal[(size_t)(kGalSlots + kGalDiag) * P + c];
    const T old = vy ? vy[c] : T(0);
    ry = old + omega * (fy[c] - (vy ? gal_apply<T>(g, gal, P, 1, i, j, vx, vy) : T(0))) / d;
  }
  ox[c] = rx;
  oy[c] = ry;
}

// r = f - L x on a Galerkin level (0 at non-unknowns)
template <typename T>
__global__ void k_gal_resid(GeomT<T> g, const T* __restrict__ gal, size_t P, const T* __restrict__ vx,
                            const T* __restrict__ vy, const T* __restrict__ fx, const T* __restrict__ fy,
                            T* __restrict__ rx, T* __restrict__ ry) {
  const int i = blockIdx.y * blockDim.y + threadIdx.y;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (i > g.ny + 1 || j > g.nx + 1) return;
  const size_t c = (size_t)i * g.ld + j;
  rx[c] = is_vx(g.nx, g.ny, i, j) ? fx[c] - gal_apply<T>(g, gal, P, 0, i, j, vx, vy) : T(0);
  ry[c] = is_vy(g.nx, g.ny, i, j) ? fy[c] - gal_apply<T>(g, gal, P, 1, i, j, vx, vy) : T(0);
}

// dense -L of a Galerkin coarsest level in the numbering of k_coarse_solve (vx unknowns row-major,
// then vy unknowns), FP64
template <typename T>
__global__ void k_gal_coarse_assemble(GeomT<T> g, const T* __restrict__ gal, size_t P, double* __restrict__ A, int n) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const int nx = g.nx, ny = g.ny, nvx = ny * (nx - 1);
  int field, i, j;
  if (k < nvx) { field = 0; i = k / (nx - 1) + 1; j = k % (nx - 1) + 1; }
  else { field = 1; const int kk = k - nvx; i = kk / nx + 1; j = kk % nx + 1; }
  const size_t c = (size_t)i * g.ld + j;
  const T* base = gal + (size_t)(field ? kGalSlots : 0) * P;
  double* row = A + (size_t)k * n;
  for (int q = 0; q < kGalSlots; ++q) {
    int f, di, dj;
    gal_offset(field, q, f, di, dj);
    const int a = i + di, b = j + dj;
    if (!is_unknown(f, nx, ny, a, b)) continue;
    const int col = f == 0 ? (a - 1) * (nx - 1) + (b - 1) : nvx + (a - 1) * nx + (b - 1);
    row[col] = -(double)base[(size_t)q * P + c];
  }
}

}  // namespace pyro
