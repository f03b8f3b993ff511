// The paper's other two velocity smoothers (Sec. "Smoothers"):
//  * k_jacobi: one damped Jacobi sweep (eq. damped_jacobi) of the coupled velocity block: every
//    vx and vy unknown moves by omega (f - L x)_i / a_ii computed from the old iterate only; the
//    new iterate goes to the level's other buffer.
//  * k_ras_tile: one pass of the RAS-type temporally blocked Jacobi smoother (Algorithm
//    ras_temporal): the cells are tiled TI x TJ with the tiling shifted by (si, sj); each CTA copies
//    its tile plus a one-cell ring into shared memory and runs `inner` local damped Jacobi
//    iterations on the unknowns it owns, the ring held at the values the pass started from (the
//    restricted-additive-Schwarz reading of "outer boundaries as fixed"), then writes the owned
//    unknowns to the other buffer. Every unknown has exactly one writer and all reads of other
//    tiles' cells come from the unchanged input buffer, so the result is deterministic.
// The tiling shifts come from SplitMix64 (Steele, Lea & Flood, OOPSLA 2014) of a counter made of
// the level, the pre/post phase and the pass number, so the smoother, and with it the V-cycle, is
// the same linear operator at every application.
#pragma once
#include "common.cuh"

namespace pyro {

__host__ __device__ inline unsigned long long splitmix64(unsigned long long z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

constexpr unsigned long long kRasSeed = 0x5EEDull;

// tiling shift of pass t of the pre (phase 0) or post (phase 1) smoothing on level l
inline void ras_shift(int level, int phase, int t, int TI, int TJ, int& si, int& sj) {
  const unsigned long long v =
      splitmix64(kRasSeed + (((unsigned long long)level * 2 + (unsigned long long)phase) << 16) + (unsigned long long)t);
  si = (int)((v & 0xffffffffull) % (unsigned long long)TI);
  sj = (int)((v >> 32) % (unsigned long long)TJ);
}

template <typename T>
__device__ inline T jacobi_value(const GeomT<T>& g, int i, int j, int field, size_t c, int ld, const T* vx,
                                 const T* vy, const T* f, const T* en, const T* ec, T omega) {
  T diag;
  const T Lv = field == 0 ? lx_point_at<T>(g, i, j, c, ld, vx, vy, en, ec, diag)
                          : ly_point_at<T>(g, i, j, c, ld, vx, vy, en, ec, diag);
  const T v = field == 0 ? vx[c] : vy[c];
  return v + omega * sdiv(f[c] - Lv, diag);
}

// Both velocity updates at an interior point (2 <= i <= ny-2, 2 <= j <= nx-2), where no wall,
// ghost or boundary term applies: lx_point_at / ly_point_at without their masks, same arithmetic.
template <typename T>
__device__ inline void jacobi_interior(const GeomT<T>& g, size_t c, int ld, const T* __restrict__ vx,
                                       const T* __restrict__ vy, const T* __restrict__ fx, const T* __restrict__ fy,
                                       const T* __restrict__ en, const T* __restrict__ ec, T omega, T& ox, T& oy) {
  {
    const T eA = ec[c], eB = ec[c + 1], e1 = en[c - ld], e2 = en[c];
    const T vc = vx[c], vw = vx[c - 1], ve = vx[c + 1], vn = vx[c - ld], vs = vx[c + ld];
    const T yA = vy[c - ld], yB = vy[c - ld + 1], yC = vy[c], yD = vy[c + 1];
    const T sxxE = T(2) * eB * (ve - vc);
    const T sxxW = T(2) * eA * (vc - vw);
    const T sxyS = e2 * ((vs - vc) * g.idy2 + (yD - yC) * g.idxdy);
    const T sxyN = e1 * ((vc - vn) * g.idy2 + (yB - yA) * g.idxdy);
    const T diag = -T(2) * (eA + eB) * g.idx2 - (e1 + e2) * g.idy2;
    const T Lv = (sxxE - sxxW) * g.idx2 + sxyS - sxyN;
    ox = vc + omega * sdiv(fx[c] - Lv, diag);
  }
  {
    const T eA = ec[c], eB = ec[c + ld], e1 = en[c - 1], e2 = en[c];
    const T vc = vy[c], vn = vy[c - ld], vs = vy[c + ld], vw = vy[c - 1], ve = vy[c + 1];
    const T xA = vx[c - 1], xB = vx[c + ld - 1], xC = vx[c], xD = vx[c + ld];
    const T syyS = T(2) * eB * (vs - vc);
    const T syyN = T(2) * eA * (vc - vn);
    const T sxyE = e2 * ((ve - vc) * g.idx2 + (xD - xC) * g.idxdy);
    const T sxyW = e1 * ((vc - vw) * g.idx2 + (xB - xA) * g.idxdy);
    const T diag = -T(2) * (eA + eB) * g.idy2 - (e1 + e2) * g.idx2;
    const T Lv = (syyS - syyN) * g.idy2 + sxyE - sxyW;
    oy = vc + omega * sdiv(fy[c] - Lv, diag);
  }
}

// Block (32, 4); each thread takes kJacobiCols cells of its row, 32 apart (coalesced, and the
// independent updates give the loads of one thread something to overlap with: 8 columns reached
// 3.8 TB/s of algorithmic traffic at 4096^2 in FP32, against 3.3 TB/s with one column).
constexpr int kJacobiCols = 8;
inline dim3 jacobi_block() { return dim3(32, 4); }
inline dim3 jacobi_grid(int nx, int ny) {
  return dim3((nx + 2 + 32 * kJacobiCols - 1) / (32 * kJacobiCols), (ny + 2 + 3) / 4);
}

template <typename T>
__global__ void k_jacobi(GeomT<T> g, const T* __restrict__ vx, const T* __restrict__ vy, T* __restrict__ ox,
                         T* __restrict__ oy, const T* __restrict__ fx, const T* __restrict__ fy,
                         const T* __restrict__ en, const T* __restrict__ ec, T omega) {
  const int i = blockIdx.y * blockDim.y + threadIdx.y;
  if (i > g.ny + 1) return;
  const int j0 = blockIdx.x * blockDim.x * kJacobiCols + threadIdx.x;
  const bool row_in = i >= 2 && i <= g.ny - 2;
#pragma unroll
  for (int q = 0; q < kJacobiCols; ++q) {
    const int j = j0 + q * (int)blockDim.x;
    if (j > g.nx + 1) return;
    const size_t c = (size_t)i * g.ld + j;
    const int jw = j - (int)threadIdx.x;   // first column of this warp's 32 (blockDim.x == 32)
    if (row_in && jw >= 2 && jw + 31 <= g.nx - 2) {   // warp-uniform: every point interior
      T a, b;
      jacobi_interior<T>(g, c, g.ld, vx, vy, fx, fy, en, ec, omega, a, b);
      ox[c] = a;
      oy[c] = b;
      continue;
    }
    ox[c] = is_vx(g.nx, g.ny, i, j) ? jacobi_value<T>(g, i, j, 0, c, g.ld, vx, vy, fx, en, ec, omega) : vx[c];
    oy[c] = is_vy(g.nx, g.ny, i, j) ? jacobi_value<T>(g, i, j, 1, c, g.ld, vx, vy, fy, en, ec, omega) : vy[c];
  }
}

template <int TI, int TJ>
struct RasTile {
  static constexpr int RH = TI + 2, RW = TJ + 2, N = RH * RW;
  template <typename T>
  static constexpr size_t smem_bytes() { return (size_t)8 * N * sizeof(T); }
};

// Grid: ceil((ny + 2 + si) / TI) x ceil((nx + 2 + sj) / TJ) tiles; tile (by, bx) owns cells
// [by TI - si, (by + 1) TI - si) x [bx TJ - sj, (bx + 1) TJ - sj) clipped to the padded grid.
template <typename T, int TI, int TJ>
__global__ void __launch_bounds__(256)
    k_ras_tile(GeomT<T> g, const T* __restrict__ vx, const T* __restrict__ vy, T* __restrict__ ox,
               T* __restrict__ oy, const T* __restrict__ fx, const T* __restrict__ fy, const T* __restrict__ en,
               const T* __restrict__ ec, T omega, int si, int sj, int inner) {
  using Tl = RasTile<TI, TJ>;
  constexpr int RW = Tl::RW, N = Tl::N;
  extern __shared__ __align__(16) unsigned char ras_smem[];
  T* sm = reinterpret_cast<T*>(ras_smem);
  // iterate buffers: vx in sm + k N, vy in sm + (2 + k) N, k = 0, 1 (local ping-pong)
  T* FX = sm + 4 * N;
  T* FY = sm + 5 * N;
  T* EN = sm + 6 * N;
  T* EC = sm + 7 * N;
  const int i0 = blockIdx.y * TI - si, j0 = blockIdx.x * TJ - sj;   // first owned cell
  // region rows i0-1 .. i0+TI, columns j0-1 .. j0+TJ; local (a, b) <-> global (i0-1+a, j0-1+b)
  for (int t = threadIdx.x; t < N; t += blockDim.x) {
    const int a = t / RW, b = t - a * RW;
    const int gi = i0 - 1 + a, gj = j0 - 1 + b;
    const bool in = gi >= 0 && gi <= g.ny + 1 && gj >= 0 && gj <= g.nx + 1;
    const size_t o = in ? (size_t)gi * g.ld + gj : 0;
    const T xv = in ? vx[o] : T(0), yv = in ? vy[o] : T(0);
    sm[t] = xv; sm[N + t] = xv;
    sm[2 * N + t] = yv; sm[3 * N + t] = yv;
    FX[t] = in ? fx[o] : T(0);
    FY[t] = in ? fy[o] : T(0);
    EN[t] = in ? en[o] : T(0);
    EC[t] = in ? ec[o] : T(0);
  }
  __syncthreads();
  // every owned cell interior (2 <= i <= ny-2, 2 <= j <= nx-2): no masks needed (block-uniform)
  const bool interior = i0 >= 2 && i0 + TI - 1 <= g.ny - 2 && j0 >= 2 && j0 + TJ - 1 <= g.nx - 2;
  int cur = 0;
  for (int it = 0; it < inner; ++it) {
    const T* xs = sm + cur * N;
    const T* ys = sm + (2 + cur) * N;
    T* xd = sm + (cur ^ 1) * N;
    T* yd = sm + (2 + (cur ^ 1)) * N;
    if (interior) {
      for (int t = threadIdx.x; t < TI * TJ; t += blockDim.x) {
        const size_t c = (size_t)(1 + t / TJ) * RW + 1 + t % TJ;
        T a, b;
        jacobi_interior<T>(g, c, RW, xs, ys, FX, FY, EN, EC, omega, a, b);
        xd[c] = a;
        yd[c] = b;
      }
      __syncthreads();
      cur ^= 1;
      continue;
    }
    for (int t = threadIdx.x; t < TI * TJ; t += blockDim.x) {
      const int a = 1 + t / TJ, b = 1 + t % TJ;
      const int gi = i0 - 1 + a, gj = j0 - 1 + b;
      const size_t c = (size_t)a * RW + b;
      if (is_vx(g.nx, g.ny, gi, gj)) xd[c] = jacobi_value<T>(g, gi, gj, 0, c, RW, xs, ys, FX, EN, EC, omega);
      if (is_vy(g.nx, g.ny, gi, gj)) yd[c] = jacobi_value<T>(g, gi, gj, 1, c, RW, xs, ys, FY, EN, EC, omega);
    }
    __syncthreads();
    cur ^= 1;
  }
  for (int t = threadIdx.x; t < TI * TJ; t += blockDim.x) {
    const int a = 1 + t / TJ, b = 1 + t % TJ;
    const int gi = i0 - 1 + a, gj = j0 - 1 + b;
    if (gi < 0 || gi > g.ny + 1 || gj < 0 || gj > g.nx + 1) continue;
    const size_t o = (size_t)gi * g.ld + gj, c = (size_t)a * RW + b;
    if (is_vx(g.nx, g.ny, gi, gj)) ox[o] = sm[cur * N + c];
    if (is_vy(g.nx, g.ny, gi, gj)) oy[o] = sm[(2 + cur) * N + c];
  }
}

}  // namespace pyro
