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

namespace pyro {

// ---------------------------------------------------------------------------------------------
// FP32 tile sweep on colour-split shared-memory planes.
//
// Each array of the tile region is stored as two planes, one per colour (i + j) mod 2, with
// element (ri, rj) at plane c, column rj >> 1 (the region's first column is even in global
// terms, so the two points of a column pair always have different colours). A half-sweep then
// touches 32 consecutive entries of each plane per warp: every shared-memory access of the update
// is conflict-free, and neighbour positions are fixed per-row offsets instead of index
// arithmetic. The boundary rules (ghost elimination, zero normal velocity on walls) are applied
// with selects on the global indices, so one code path serves interior and boundary tiles. The
// update arithmetic is the same expression as rbgs_point<float>.
// ---------------------------------------------------------------------------------------------
template <int NS, int TX, int TY>
struct SweepTileCS {
  static constexpr int M = 4 * NS;
  static constexpr int RX = TX + 2 * M, RY = TY + 2 * M, HX = RX / 2;
  static constexpr int PLANE = RY * HX;                 // one colour plane of one array
  // staged coarse block for the fused prolongation: rows/columns (origin / 2) - 1 ... covering
  // the region, plus one on each side
  static constexpr int CY = RY / 2 + 2, CX = RX / 2 + 2, CPL = CY * CX;
  static constexpr size_t smem_bytes() { return ((size_t)PLANE * 2 * 6 + 2 * CPL) * sizeof(float); }
  static_assert(RX % 2 == 0 && M % 2 == 0, "region must start on an even global column");
};

// One colour of one field over rows [r0, r1) and columns [c0, c1) of a colour-split tile. Threads
// take consecutive (row, slot) pairs, so a warp covers 32 consecutive same-colour points. With
// INTERIOR the boundary rules are provably inactive for every point and are not evaluated.
template <bool INTERIOR, typename Tl>
__device__ __forceinline__ void cs_halfsweep(const GeomT<float>& g, float* smf, int fld, int col, float omega,
                                             int i0, int j0, int r0, int r1, int c0, int c1) {
  constexpr int HX = Tl::HX, PL = Tl::PLANE;
  const float* Xo = smf + (0 + (col ^ 1)) * PL;
  const float* Xs = smf + (0 + col) * PL;
  const float* Yo = smf + (2 + (col ^ 1)) * PL;
  const float* Ys = smf + (2 + col) * PL;
  const float* No = smf + (8 + (col ^ 1)) * PL;
  const float* Ns = smf + (8 + col) * PL;
  const float* Eo = smf + (10 + (col ^ 1)) * PL;
  const float* Es = smf + (10 + col) * PL;
  float* U = smf + (2 * fld + col) * PL;
  const float* F = smf + (4 + 2 * fld + col) * PL;
  const int nrow = r1 - r0;
  for (int t = threadIdx.x; t < nrow * HX; t += blockDim.x) {
    const int ri = r0 + t / HX;
    const int k = t - (ri - r0) * HX;
    const int gi = i0 + ri;
    const int p = (col - gi - j0) & 1;
    const int rj = 2 * k + p;
    if (rj < c0 || rj >= c1) continue;
    const int gj = j0 + rj;
    const int s = ri * HX + k;
    const int kw = s - 1 + p, ke = s + p;
    if (fld == 0) {
      if (!INTERIOR && !is_vx(g.nx, g.ny, gi, gj)) continue;
      const float vc = Xs[s];
      const float eA = Es[s], eB = Eo[ke];
      const float e1 = No[s - HX], e2 = Ns[s];
      float vw = Xo[kw], ve = Xo[ke], vn = Xo[s - HX], vs = Xo[s + HX];
      float yA = Yo[s - HX], yB = Ys[s - HX + p], yC = Ys[s], yD = Yo[ke];
      if (!INTERIOR) {
        if (gj - 1 < 1) vw = 0.f;
        if (gj + 1 > g.nx - 1) ve = 0.f;
        if (gi == 1) vn = g.sN * vc;
        if (gi == g.ny) vs = g.sS * vc;
        if (gi - 1 < 1) { yA = 0.f; yB = 0.f; }
        if (gi > g.ny - 1) { yC = 0.f; yD = 0.f; }
      }
      const float sxxE = 2.f * eB * (ve - vc);
      const float sxxW = 2.f * eA * (vc - vw);
      const float sxyS = e2 * ((vs - vc) * g.idy2 + (yD - yC) * g.idxdy);
      const float sxyN = e1 * ((vc - vn) * g.idy2 + (yB - yA) * g.idxdy);
      float diag = -2.f * (eA + eB) * g.idx2 - (e1 + e2) * g.idy2;
      if (!INTERIOR) {
        if (gi == 1) diag += g.sN * e1 * g.idy2;
        if (gi == g.ny) diag += g.sS * e2 * g.idy2;
      }
      const float Lv = (sxxE - sxxW) * g.idx2 + sxyS - sxyN;
      U[s] = vc + omega * __fdividef(F[s] - Lv, diag);
    } else {
      if (!INTERIOR && !is_vy(g.nx, g.ny, gi, gj)) continue;
      const float vc = Ys[s];
      const float eA = Es[s], eB = Eo[s + HX];
      const float e1 = No[kw], e2 = Ns[s];
      float vn = Yo[s - HX], vs = Yo[s + HX], vw = Yo[kw], ve = Yo[ke];
      float xA = Xo[kw], xB = Xs[s + HX - 1 + p], xC = Xs[s], xD = Xo[s + HX];
      if (!INTERIOR) {
        if (gi - 1 < 1) vn = 0.f;
        if (gi + 1 > g.ny - 1) vs = 0.f;
        if (gj == 1) vw = g.sW * vc;
        if (gj == g.nx) ve = g.sE * vc;
        if (gj - 1 < 1) { xA = 0.f; xB = 0.f; }
        if (gj > g.nx - 1) { xC = 0.f; xD = 0.f; }
      }
      const float syyS = 2.f * eB * (vs - vc);
      const float syyN = 2.f * eA * (vc - vn);
      const float sxyE = e2 * ((ve - vc) * g.idx2 + (xD - xC) * g.idxdy);
      const float sxyW = e1 * ((vc - vw) * g.idx2 + (xB - xA) * g.idxdy);
      float diag = -2.f * (eA + eB) * g.idy2 - (e1 + e2) * g.idx2;
      if (!INTERIOR) {
        if (gj == 1) diag += g.sW * e1 * g.idx2;
        if (gj == g.nx) diag += g.sE * e2 * g.idx2;
      }
      const float Lv = (syyS - syyN) * g.idy2 + sxyE - sxyW;
      U[s] = vc + omega * __fdividef(F[s] - Lv, diag);
    }
  }
}

template <int NS, int TX, int TY>
__global__ void __launch_bounds__(kTileThreads)
    k_rbgs_tile_cs(GeomT<float> g, const float* __restrict__ vx, const float* __restrict__ vy,
                   float* __restrict__ ox, float* __restrict__ oy, const float* __restrict__ fx,
                   const float* __restrict__ fy, const float* __restrict__ en, const float* __restrict__ ec,
                   float omega, GeomT<float> gc, const float* __restrict__ cvx, const float* __restrict__ cvy) {
  using Tl = SweepTileCS<NS, TX, TY>;
  constexpr int M = Tl::M, RX = Tl::RX, RY = Tl::RY, HX = Tl::HX, PL = Tl::PLANE;
  extern __shared__ __align__(16) float smf[];
  // plane (array a, colour c) starts at smf + (2 a + c) * PL; arrays: 0 vx, 1 vy, 2 fx, 3 fy, 4 en, 5 ec
  auto plane = [&](int a, int c) { return smf + (2 * a + c) * PL; };
  (void)HX;
  const int i0 = blockIdx.y * TY - M, j0 = blockIdx.x * TX - M;
  const int rlo = max(0, -i0), rhi = min(RY, g.ny + 2 - i0);
  const int clo = max(0, -j0), chi = min(RX, g.nx + 2 - j0);

  // coarse correction (post-smoothing): stage the coarse block this region interpolates from,
  // with the coarse boundary rule already applied, in shared memory behind the planes
  float* cbx = smf + 12 * PL;
  float* cby = cbx + Tl::CPL;
  const int I0 = (i0 >> 1) - 1, J0 = (j0 >> 1) - 1;   // floor division (i0, j0 may be negative)
  if (cvx) {
    for (int t = threadIdx.x; t < Tl::CY * Tl::CX; t += blockDim.x) {
      const int I = I0 + t / Tl::CX, J = J0 + t % Tl::CX;
      const bool in = I >= 0 && I <= gc.ny + 1 && J >= 0 && J <= gc.nx + 1;
      cbx[t] = in ? coarse_vx(gc, cvx, I, J) : 0.f;
      cby[t] = in ? coarse_vy(gc, cvy, I, J) : 0.f;
    }
    __syncthreads();
  }
  auto cvxs = [&](int I, int J) { return cbx[(I - I0) * Tl::CX + (J - J0)]; };
  auto cvys = [&](int I, int J) { return cby[(I - I0) * Tl::CX + (J - J0)]; };

  // load the part of the region inside the domain, splitting colours
#pragma unroll 2
  for (int t = threadIdx.x; t < (rhi - rlo) * RX; t += blockDim.x) {
    const int ri = rlo + t / RX, rj = t % RX;
    if (rj < clo || rj >= chi) continue;
    const int gi = i0 + ri, gj = j0 + rj;
    const size_t o = (size_t)gi * g.ld + gj;
    const int c = (gi + gj) & 1;
    const int s = ri * HX + (rj >> 1);
    float a = vx[o], b = vy[o];
    const float f0 = fx[o], f1 = fy[o], e0 = en[o], e1 = ec[o];
    if (cvx) {
      if (is_vx(g.nx, g.ny, gi, gj)) {
        // same weights as prolong_vx_inc, coarse values from the staged block
        const int Ia = (gi & 1) ? (gi - 1) / 2 : gi / 2;
        const float wy0 = (gi & 1) ? 0.25f : 0.75f, wy1 = 1.f - wy0;
        if (gj & 1) {
          const int Ja = (gj - 1) / 2;
          a += 0.5f * (wy0 * cvxs(Ia, Ja) + wy1 * cvxs(Ia + 1, Ja) + wy0 * cvxs(Ia, Ja + 1) + wy1 * cvxs(Ia + 1, Ja + 1));
        } else {
          const int Jc = gj / 2;
          a += wy0 * cvxs(Ia, Jc) + wy1 * cvxs(Ia + 1, Jc);
        }
      }
      if (is_vy(g.nx, g.ny, gi, gj)) {
        const int Ja = (gj & 1) ? (gj - 1) / 2 : gj / 2;
        const float wx0 = (gj & 1) ? 0.25f : 0.75f, wx1 = 1.f - wx0;
        if (gi & 1) {
          const int Ia = (gi - 1) / 2;
          b += 0.5f * (wx0 * cvys(Ia, Ja) + wx1 * cvys(Ia, Ja + 1) + wx0 * cvys(Ia + 1, Ja) + wx1 * cvys(Ia + 1, Ja + 1));
        } else {
          const int Ic = gi / 2;
          b += wx0 * cvys(Ic, Ja) + wx1 * cvys(Ic, Ja + 1);
        }
      }
    }
    plane(0, c)[s] = a;
    plane(1, c)[s] = b;
    plane(2, c)[s] = f0;
    plane(3, c)[s] = f1;
    plane(4, c)[s] = e0;
    plane(5, c)[s] = e1;
  }
  __syncthreads();

  // a tile whose whole region lies in rows/columns [2, n-2] needs no boundary rule anywhere
  const bool interior = i0 >= 2 && i0 + RY - 1 <= g.ny - 2 && j0 >= 2 && j0 + RX - 1 <= g.nx - 2;
  int h = 0;
  for (int sw = 0; sw < NS; ++sw)
    for (int fld = 0; fld < 2; ++fld)
      for (int col = 0; col < 2; ++col, ++h) {
        const int m = h + 1;
        const int r0 = max(m, rlo), r1 = min(RY - m, rhi);
        const int c0 = max(m, clo), c1 = min(RX - m, chi);
        if (interior) cs_halfsweep<true, Tl>(g, smf, fld, col, omega, i0, j0, r0, r1, c0, c1);
        else cs_halfsweep<false, Tl>(g, smf, fld, col, omega, i0, j0, r0, r1, c0, c1);
        __syncthreads();
      }

  for (int t = threadIdx.x; t < TX * TY; t += blockDim.x) {
    const int ri = M + t / TX, rj = M + t % TX;
    const int gi = i0 + ri, gj = j0 + rj;
    if (gi > g.ny + 1 || gj > g.nx + 1) continue;
    const size_t o = (size_t)gi * g.ld + gj;
    const int c = (gi + gj) & 1;
    const int s = ri * HX + (rj >> 1);
    if (is_vx(g.nx, g.ny, gi, gj)) ox[o] = plane(0, c)[s];
    if (is_vy(g.nx, g.ny, gi, gj)) oy[o] = plane(1, c)[s];
  }
}

// ---------------------------------------------------------------------------------------------
// FP32 tile sweep, warp-per-row form. The region is 64 columns wide (a tile of TX = 64 - 8 NS
// owned columns plus the 4 NS halo on each side), so each colour plane row has exactly 32 slots:
// lane k of a warp owns slot k of a row, warps stride over rows. No per-point division or
// modulo, and the region loads and the final stores move column pairs (one 8-byte access for
// the two colours of a pair when the row stride is even). Same point arithmetic as
// cs_halfsweep.
// ---------------------------------------------------------------------------------------------
template <int NS, int TY>
struct SweepTileW {
  static constexpr int M = 4 * NS;
  static constexpr int RX = 64, TX = RX - 2 * M, RY = TY + 2 * M, HX = 32;
  static constexpr int PLANE = RY * HX;
  static constexpr int CY = RY / 2 + 2, CX = RX / 2 + 2, CPL = CY * CX;
  static constexpr size_t smem_bytes() { return ((size_t)PLANE * 2 * 6 + 2 * CPL) * sizeof(float); }
};

template <bool INTERIOR, typename Tl>
__device__ __forceinline__ void w_halfsweep(const GeomT<float>& g, float* smf, int fld, int col, float omega,
                                            int i0, int j0, int r0, int r1, int c0, int c1) {
  constexpr int HX = Tl::HX, PL = Tl::PLANE;
  const float* Xo = smf + (0 + (col ^ 1)) * PL;
  const float* Xs = smf + (0 + col) * PL;
  const float* Yo = smf + (2 + (col ^ 1)) * PL;
  const float* Ys = smf + (2 + col) * PL;
  const float* No = smf + (8 + (col ^ 1)) * PL;
  const float* Ns = smf + (8 + col) * PL;
  const float* Eo = smf + (10 + (col ^ 1)) * PL;
  const float* Es = smf + (10 + col) * PL;
  float* U = smf + (2 * fld + col) * PL;
  const float* F = smf + (4 + 2 * fld + col) * PL;
  const int k = threadIdx.x & 31;
  for (int ri = r0 + (int)(threadIdx.x >> 5); ri < r1; ri += (int)(blockDim.x >> 5)) {
    const int gi = i0 + ri;
    const int p = (col + gi) & 1;          // j0 is even
    const int rj = 2 * k + p;
    if (rj < c0 || rj >= c1) continue;
    const int gj = j0 + rj;
    const int s = ri * HX + k;
    const int kw = s - 1 + p, ke = s + p;
    if (fld == 0) {
      if (!INTERIOR && !is_vx(g.nx, g.ny, gi, gj)) continue;
      const float vc = Xs[s];
      const float eA = Es[s], eB = Eo[ke];
      const float e1 = No[s - HX], e2 = Ns[s];
      float vw = Xo[kw], ve = Xo[ke], vn = Xo[s - HX], vs = Xo[s + HX];
      float yA = Yo[s - HX], yB = Ys[s - HX + p], yC = Ys[s], yD = Yo[ke];
      if (!INTERIOR) {
        if (gj - 1 < 1) vw = 0.f;
        if (gj + 1 > g.nx - 1) ve = 0.f;
        if (gi == 1) vn = g.sN * vc;
        if (gi == g.ny) vs = g.sS * vc;
        if (gi - 1 < 1) { yA = 0.f; yB = 0.f; }
        if (gi > g.ny - 1) { yC = 0.f; yD = 0.f; }
      }
      const float sxxE = 2.f * eB * (ve - vc);
      const float sxxW = 2.f * eA * (vc - vw);
      const float sxyS = e2 * ((vs - vc) * g.idy2 + (yD - yC) * g.idxdy);
      const float sxyN = e1 * ((vc - vn) * g.idy2 + (yB - yA) * g.idxdy);
      float diag = -2.f * (eA + eB) * g.idx2 - (e1 + e2) * g.idy2;
      if (!INTERIOR) {
        if (gi == 1) diag += g.sN * e1 * g.idy2;
        if (gi == g.ny) diag += g.sS * e2 * g.idy2;
      }
      const float Lv = (sxxE - sxxW) * g.idx2 + sxyS - sxyN;
      U[s] = vc + omega * __fdividef(F[s] - Lv, diag);
    } else {
      if (!INTERIOR && !is_vy(g.nx, g.ny, gi, gj)) continue;
      const float vc = Ys[s];
      const float eA = Es[s], eB = Eo[s + HX];
      const float e1 = No[kw], e2 = Ns[s];
      float vn = Yo[s - HX], vs = Yo[s + HX], vw = Yo[kw], ve = Yo[ke];
      float xA = Xo[kw], xB = Xs[s + HX - 1 + p], xC = Xs[s], xD = Xo[s + HX];
      if (!INTERIOR) {
        if (gi - 1 < 1) vn = 0.f;
        if (gi + 1 > g.ny - 1) vs = 0.f;
        if (gj == 1) vw = g.sW * vc;
        if (gj == g.nx) ve = g.sE * vc;
        if (gj - 1 < 1) { xA = 0.f; xB = 0.f; }
        if (gj > g.nx - 1) { xC = 0.f; xD = 0.f; }
      }
      const float syyS = 2.f * eB * (vs - vc);
      const float syyN = 2.f * eA * (vc - vn);
      const float sxyE = e2 * ((ve - vc) * g.idx2 + (xD - xC) * g.idxdy);
      const float sxyW = e1 * ((vc - vw) * g.idx2 + (xB - xA) * g.idxdy);
      float diag = -2.f * (eA + eB) * g.idy2 - (e1 + e2) * g.idx2;
      if (!INTERIOR) {
        if (gj == 1) diag += g.sW * e1 * g.idx2;
        if (gj == g.nx) diag += g.sE * e2 * g.idx2;
      }
      const float Lv = (syyS - syyN) * g.idy2 + sxyE - sxyW;
      U[s] = vc + omega * __fdividef(F[s] - Lv, diag);
    }
  }
}

template <int NS, int TY>
__global__ void __launch_bounds__(kTileThreads)
    k_rbgs_tile_w(GeomT<float> g, const float* __restrict__ vx, const float* __restrict__ vy,
                  float* __restrict__ ox, float* __restrict__ oy, const float* __restrict__ fx,
                  const float* __restrict__ fy, const float* __restrict__ en, const float* __restrict__ ec,
                  float omega, GeomT<float> gc, const float* __restrict__ cvx, const float* __restrict__ cvy) {
  using Tl = SweepTileW<NS, TY>;
  constexpr int M = Tl::M, RX = Tl::RX, RY = Tl::RY, HX = Tl::HX, PL = Tl::PLANE, TX = Tl::TX;
  extern __shared__ __align__(16) float smf[];
  const int i0 = blockIdx.y * TY - M, j0 = blockIdx.x * TX - M;   // j0 even (TX, M even)
  const int rlo = max(0, -i0), rhi = min(RY, g.ny + 2 - i0);
  const int clo = max(0, -j0), chi = min(RX, g.nx + 2 - j0);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;

  float* cbx = smf + 12 * PL;
  float* cby = cbx + Tl::CPL;
  const int I0 = (i0 >> 1) - 1, J0 = (j0 >> 1) - 1;
  if (cvx) {
    for (int t = threadIdx.x; t < Tl::CY * Tl::CX; t += blockDim.x) {
      const int I = I0 + t / Tl::CX, J = J0 + t % Tl::CX;
      const bool in = I >= 0 && I <= gc.ny + 1 && J >= 0 && J <= gc.nx + 1;
      cbx[t] = in ? coarse_vx(gc, cvx, I, J) : 0.f;
      cby[t] = in ? coarse_vy(gc, cvy, I, J) : 0.f;
    }
    __syncthreads();
  }
  auto cvxs = [&](int I, int J) { return cbx[(I - I0) * Tl::CX + (J - J0)]; };
  auto cvys = [&](int I, int J) { return cby[(I - I0) * Tl::CX + (J - J0)]; };
  auto prolong = [&](int gi, int gj, float& a, float& b) {
    if (is_vx(g.nx, g.ny, gi, gj)) {
      const int Ia = (gi & 1) ? (gi - 1) / 2 : gi / 2;
      const float wy0 = (gi & 1) ? 0.25f : 0.75f, wy1 = 1.f - wy0;
      if (gj & 1) {
        const int Ja = (gj - 1) / 2;
        a += 0.5f * (wy0 * cvxs(Ia, Ja) + wy1 * cvxs(Ia + 1, Ja) + wy0 * cvxs(Ia, Ja + 1) + wy1 * cvxs(Ia + 1, Ja + 1));
      } else {
        const int Jc = gj / 2;
        a += wy0 * cvxs(Ia, Jc) + wy1 * cvxs(Ia + 1, Jc);
      }
    }
    if (is_vy(g.nx, g.ny, gi, gj)) {
      const int Ja = (gj & 1) ? (gj - 1) / 2 : gj / 2;
      const float wx0 = (gj & 1) ? 0.25f : 0.75f, wx1 = 1.f - wx0;
      if (gi & 1) {
        const int Ia = (gi - 1) / 2;
        b += 0.5f * (wx0 * cvys(Ia, Ja) + wx1 * cvys(Ia, Ja + 1) + wx0 * cvys(Ia + 1, Ja) + wx1 * cvys(Ia + 1, Ja + 1));
      } else {
        const int Ic = gi / 2;
        b += wx0 * cvys(Ic, Ja) + wx1 * cvys(Ic, Ja + 1);
      }
    }
  };

  // load: lane takes the column pair (2 lane, 2 lane + 1); element (ri, 2k + h) goes to the plane
  // of its colour at slot k
  const bool even_ld = (g.ld & 1) == 0;
  for (int ri = rlo + warp; ri < rhi; ri += nw) {
    const int gi = i0 + ri;
    const int c = gi & 1;                    // colour of the pair's even column (j0 even)
    const int s = ri * HX + lane;
    const int rj = 2 * lane, gj = j0 + rj;
    float a[2] = {0.f, 0.f}, b[2] = {0.f, 0.f}, f0[2] = {0.f, 0.f}, f1[2] = {0.f, 0.f}, e0[2] = {0.f, 0.f},
          e1[2] = {0.f, 0.f};
    const size_t o = (size_t)gi * g.ld + gj;
    if (even_ld && rj >= clo && rj + 1 < chi) {
      const float2 va = *reinterpret_cast<const float2*>(vx + o), vb = *reinterpret_cast<const float2*>(vy + o);
      const float2 vf0 = *reinterpret_cast<const float2*>(fx + o), vf1 = *reinterpret_cast<const float2*>(fy + o);
      const float2 ve0 = *reinterpret_cast<const float2*>(en + o), ve1 = *reinterpret_cast<const float2*>(ec + o);
      a[0] = va.x; a[1] = va.y; b[0] = vb.x; b[1] = vb.y; f0[0] = vf0.x; f0[1] = vf0.y;
      f1[0] = vf1.x; f1[1] = vf1.y; e0[0] = ve0.x; e0[1] = ve0.y; e1[0] = ve1.x; e1[1] = ve1.y;
    } else {
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        if (rj + h < clo || rj + h >= chi) continue;
        a[h] = vx[o + h]; b[h] = vy[o + h]; f0[h] = fx[o + h]; f1[h] = fy[o + h]; e0[h] = en[o + h]; e1[h] = ec[o + h];
      }
    }
    if (cvx) {
#pragma unroll
      for (int h = 0; h < 2; ++h)
        if (rj + h >= clo && rj + h < chi) prolong(gi, gj + h, a[h], b[h]);
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int pc = c ^ h;
      smf[(0 + pc) * PL + s] = a[h];
      smf[(2 + pc) * PL + s] = b[h];
      smf[(4 + pc) * PL + s] = f0[h];
      smf[(6 + pc) * PL + s] = f1[h];
      smf[(8 + pc) * PL + s] = e0[h];
      smf[(10 + pc) * PL + s] = e1[h];
    }
  }
  __syncthreads();

  const bool interior = i0 >= 2 && i0 + RY - 1 <= g.ny - 2 && j0 >= 2 && j0 + RX - 1 <= g.nx - 2;
  int hs = 0;
  for (int sw = 0; sw < NS; ++sw)
    for (int fld = 0; fld < 2; ++fld)
      for (int col = 0; col < 2; ++col, ++hs) {
        const int m = hs + 1;
        const int r0 = max(m, rlo), r1 = min(RY - m, rhi);
        const int c0 = max(m, clo), c1 = min(RX - m, chi);
        if (interior) w_halfsweep<true, Tl>(g, smf, fld, col, omega, i0, j0, r0, r1, c0, c1);
        else w_halfsweep<false, Tl>(g, smf, fld, col, omega, i0, j0, r0, r1, c0, c1);
        __syncthreads();
      }

  // store the owned columns [M, M + TX) of rows [M, M + TY) at the unknowns
  for (int ri = M + warp; ri < M + TY; ri += nw) {
    const int gi = i0 + ri;
    if (gi > g.ny + 1) break;
    const int c = gi & 1;
    const int rj = 2 * lane, gj = j0 + rj;
    if (rj < M || rj >= M + TX) continue;   // M even: a pair is wholly owned or not
    const int s = ri * HX + lane;
    const size_t o = (size_t)gi * g.ld + gj;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      if (gj + h > g.nx + 1) continue;
      const int pc = c ^ h;
      if (is_vx(g.nx, g.ny, gi, gj + h)) ox[o + h] = smf[(0 + pc) * PL + s];
      if (is_vy(g.nx, g.ny, gi, gj + h)) oy[o + h] = smf[(2 + pc) * PL + s];
    }
  }
}

}  // namespace pyro
