// Tile-fused multigrid kernels: one launch per smoothing block and one per residual+restriction.
//
// k_rbgs_tile: NS full red-black Gauss-Seidel sweeps (each = vx-red, vx-black, vy-red, vy-black,
// eq. sor_update) of one output tile in shared memory. Every point update reads neighbours at
// Chebyshev distance <= 1, so after h half-sweeps the values are exact in the loaded region
// shrunk by h; loading a halo of 4*NS points and updating the shrinking region makes the output
// tile exactly (bitwise) what NS sweeps of the one-kernel-per-colour path produce. Tiles read the
// iterate from one buffer and write their output tile to another (ping-pong), so no tile can see
// a neighbour's already-updated values in its halo. The halo work
// is redundant arithmetic, not extra DRAM traffic: each array is read once per tile (the halo
// overlap is served from L2) and the tile is written once, so NS sweeps cost one pass over HBM.
// With a coarse correction given (cvx != null), the bilinear prolongation is added while the
// tile is loaded (eq. multigrid_levels step (5) fused into the first post-smoothing pass).
//
// k_resrestrict_tile: residual r = f - L x on the fine points a tile of coarse points needs,
// kept in shared memory, then the normalised bilinear restriction to the coarse right-hand side
// and the zeroing of the coarse iterate (steps (2)-(3) and the start of (4)). The fine residual
// never goes to global memory.
//
// The point functions are the same as in the unfused kernels; shared-memory arrays are addressed
// with the global (i, j) through base pointers shifted by the tile origin, so the boundary logic
// (walls, ghost elimination) is untouched.
#pragma once
#include "kernels_mg.cuh"

namespace pyro {

constexpr int kTileThreads = 512;

template <typename T, int NS, int TX, int TY>
struct SweepTile {
  static constexpr int M = 4 * NS;
  static constexpr int RX = TX + 2 * M, RY = TY + 2 * M, NPT = RX * RY;
  static size_t smem_bytes(bool with_idg) { return (size_t)NPT * (with_idg ? 8 : 6) * sizeof(T); }
};

template <typename T, int NS, int TX, int TY>
__global__ void __launch_bounds__(kTileThreads)
    k_rbgs_tile(GeomT<T> g, const T* __restrict__ vx, const T* __restrict__ vy, T* __restrict__ ox,
                T* __restrict__ oy, const T* __restrict__ fx, const T* __restrict__ fy, const T* __restrict__ en,
                const T* __restrict__ ec, const T* __restrict__ idgx, const T* __restrict__ idgy, T omega,
                GeomT<T> gc, const T* __restrict__ cvx, const T* __restrict__ cvy) {
  using Tl = SweepTile<T, NS, TX, TY>;
  constexpr int M = Tl::M, RX = Tl::RX, RY = Tl::RY, NPT = Tl::NPT;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* s_vx = reinterpret_cast<T*>(smem_raw);
  T* s_vy = s_vx + NPT;
  T* s_fx = s_vy + NPT;
  T* s_fy = s_fx + NPT;
  T* s_en = s_fy + NPT;
  T* s_ec = s_en + NPT;
  const bool has_idg = idgx != nullptr;
  T* s_ix = has_idg ? s_ec + NPT : nullptr;
  T* s_iy = has_idg ? s_ix + NPT : nullptr;
  const int i0 = blockIdx.y * TY - M, j0 = blockIdx.x * TX - M;
  // part of the region inside the padded domain (local coordinates); nothing outside is read
  const int rlo = max(0, -i0), rhi = min(RY, g.ny + 2 - i0);
  const int clo = max(0, -j0), chi = min(RX, g.nx + 2 - j0);
  const int rw = chi - clo;

  for (int t = threadIdx.x; t < (rhi - rlo) * rw; t += blockDim.x) {
    const int ri = rlo + t / rw, rj = clo + t % rw;
    const int gi = i0 + ri, gj = j0 + rj;
    const int st = ri * RX + rj;
    const size_t o = (size_t)gi * g.ld + gj;
    T a = vx[o], b = vy[o];
    if (cvx) {
      if (is_vx(g.nx, g.ny, gi, gj)) a += prolong_vx_inc(gc, gi, gj, cvx);
      if (is_vy(g.nx, g.ny, gi, gj)) b += prolong_vy_inc(gc, gi, gj, cvy);
    }
    s_vx[st] = a; s_vy[st] = b; s_fx[st] = fx[o]; s_fy[st] = fy[o]; s_en[st] = en[o]; s_ec[st] = ec[o];
    if (has_idg) { s_ix[st] = idgx[o]; s_iy[st] = idgy[o]; }
  }
  __syncthreads();

  GeomT<T> gs = g;
  gs.ld = RX;
  const ptrdiff_t off = (ptrdiff_t)i0 * RX + j0;
  T* pvx = s_vx - off;
  T* pvy = s_vy - off;
  const T* pfx = s_fx - off;
  const T* pfy = s_fy - off;
  const T* pen = s_en - off;
  const T* pec = s_ec - off;
  const T* pix = has_idg ? s_ix - off : nullptr;
  const T* piy = has_idg ? s_iy - off : nullptr;
  int h = 0;
  for (int sw = 0; sw < NS; ++sw)
    for (int fld = 0; fld < 2; ++fld)
      for (int col = 0; col < 2; ++col, ++h) {
        const int m = h + 1;                       // exact region after this half-sweep
        const int r0 = max(m, rlo), r1 = min(RY - m, rhi);
        const int c0 = max(m, clo), c1 = min(RX - m, chi);
        const int hw = (c1 - c0) / 2 + 1;
        for (int t = threadIdx.x; t < (r1 - r0) * hw; t += blockDim.x) {
          const int ri = r0 + t / hw;
          const int gi = i0 + ri;
          const int par = ((col - gi - j0 - c0) % 2 + 2) % 2;  // first local column of this colour
          const int rj = c0 + par + 2 * (t % hw);
          if (rj >= c1) continue;
          rbgs_point<T>(gs, gi, j0 + rj, fld, omega, pvx, pvy, pfx, pfy, pen, pec, pix, piy);
        }
        __syncthreads();
      }

  for (int t = threadIdx.x; t < TX * TY; t += blockDim.x) {
    const int ri = M + t / TX, rj = M + t % TX;
    const int gi = i0 + ri, gj = j0 + rj;
    if (gi > g.ny + 1 || gj > g.nx + 1) continue;
    const size_t o = (size_t)gi * g.ld + gj;
    const int st = ri * RX + rj;
    if (is_vx(g.nx, g.ny, gi, gj)) ox[o] = s_vx[st];
    if (is_vy(g.nx, g.ny, gi, gj)) oy[o] = s_vy[st];
  }
}

template <typename T, int CTX, int CTY>
struct ResTile {
  static constexpr int LRX = 2 * CTX + 4, LRY = 2 * CTY + 4, NPT = LRX * LRY;
  static size_t smem_bytes() { return (size_t)NPT * 8 * sizeof(T); }
};

template <typename T, int CTX, int CTY>
__global__ void __launch_bounds__(kTileThreads)
    k_resrestrict_tile(GeomT<T> g, GeomT<T> gc, const T* __restrict__ vx, const T* __restrict__ vy,
                       const T* __restrict__ fx, const T* __restrict__ fy, const T* __restrict__ en,
                       const T* __restrict__ ec, T* __restrict__ fxc, T* __restrict__ fyc, T* __restrict__ cvx,
                       T* __restrict__ cvy) {
  using Tl = ResTile<T, CTX, CTY>;
  constexpr int LRX = Tl::LRX, LRY = Tl::LRY, NPT = Tl::NPT;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* s_vx = reinterpret_cast<T*>(smem_raw);
  T* s_vy = s_vx + NPT;
  T* s_fx = s_vy + NPT;
  T* s_fy = s_fx + NPT;
  T* s_en = s_fy + NPT;
  T* s_ec = s_en + NPT;
  T* s_rx = s_ec + NPT;
  T* s_ry = s_rx + NPT;
  const int I0 = blockIdx.y * CTY, J0 = blockIdx.x * CTX;
  const int i0 = 2 * I0 - 3, j0 = 2 * J0 - 3;  // loaded fine region origin
  const int rlo = max(0, -i0), rhi = min(LRY, g.ny + 2 - i0);
  const int clo = max(0, -j0), chi = min(LRX, g.nx + 2 - j0);
  const int rw = chi - clo;

  for (int t = threadIdx.x; t < (rhi - rlo) * rw; t += blockDim.x) {
    const int ri = rlo + t / rw, rj = clo + t % rw;
    const size_t o = (size_t)(i0 + ri) * g.ld + (j0 + rj);
    const int st = ri * LRX + rj;
    s_vx[st] = vx[o]; s_vy[st] = vy[o]; s_fx[st] = fx[o]; s_fy[st] = fy[o]; s_en[st] = en[o]; s_ec[st] = ec[o];
  }
  __syncthreads();

  GeomT<T> gs = g;
  gs.ld = LRX;
  const ptrdiff_t off = (ptrdiff_t)i0 * LRX + j0;
  // residual on the fine region the coarse tile restricts from (loaded region shrunk by 1)
  const int r0 = max(1, rlo), r1 = min(LRY - 1, rhi), c0 = max(1, clo), c1 = min(LRX - 1, chi);
  for (int t = threadIdx.x; t < (r1 - r0) * (c1 - c0); t += blockDim.x) {
    const int gi = i0 + r0 + t / (c1 - c0), gj = j0 + c0 + t % (c1 - c0);
    vresid_point<T>(gs, gi, gj, s_vx - off, s_vy - off, s_fx - off, s_fy - off, s_en - off, s_ec - off,
                    s_rx - off, s_ry - off);
  }
  __syncthreads();

  for (int t = threadIdx.x; t < CTX * CTY; t += blockDim.x) {
    const int I = I0 + t / CTX, J = J0 + t % CTX;
    if (I > gc.ny + 1 || J > gc.nx + 1) continue;
    restrict_point<T>(gs, gc, I, J, s_rx - off, s_ry - off, fxc, fyc);
    const size_t o = (size_t)I * gc.ld + J;
    cvx[o] = T(0);
    cvy[o] = T(0);
  }
}

}  // namespace pyro
