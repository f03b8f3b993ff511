// Host side of libpyro (single translation unit: the kernel headers are included here): solver handle, multigrid hierarchy, V-cycle driver, flexible GMRES with
// the Uzawa/multigrid preconditioner, adjoint, and the extern "C" entry points of pyro.h.
#include <cuda_runtime.h>
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <initializer_list>
#include <new>
#include <utility>
#include <vector>

#include "../../include/pyro.h"
#include "common.cuh"

#include "kernels_mg.cuh"
#include "kernels_krylov.cuh"
#include "kernels_tile.cuh"
#include "kernels_jacobi.cuh"
#include "kernels_schur.cuh"
#include "kernels_galerkin.cuh"
#include "kernels_fcg.cuh"

using namespace pyro;

namespace {

constexpr int kMaxCoarse = 1024;
constexpr int kCoarseInvertMulti = 80;    // larger coarsest systems invert over the whole GPU, sixteen
                                          // pivots per launch (one CTA: about n^3 / 2 clocks of one
                                          // SM plus a barrier per pivot)
constexpr int kRasTile = 32;        // RAS-type Jacobi tile edge (cells), the paper's 32 x 32
constexpr long long kSmallTileCells = 65536;  // FP32 levels up to 256^2 smooth with 32 x 16 tiles
constexpr int kWTileY2 = 48;        // owned rows of the two-sweep warp-per-row tile (2 CTAs per SM)
constexpr int kWTileY1 = 48;        // owned rows of the one-sweep warp-per-row tile

struct CudaError {
  cudaError_t e;
};
#define CK(call)                                   \
  do {                                             \
    cudaError_t _e = (call);                       \
    if (_e != cudaSuccess) throw CudaError{_e};    \
  } while (0)

inline dim3 grid2(int nx, int ny, dim3 b) { return dim3((nx + 2 + b.x - 1) / b.x, (ny + 2 + b.y - 1) / b.y); }
inline dim3 grid_rb(int nx, int ny, dim3 b) { return dim3(((nx + 2) / 2 + 1 + b.x - 1) / b.x, (ny + 2 + b.y - 1) / b.y); }
const dim3 kBlk2(32, 8);

// In-place inverse of the SPD matrix A (n x n, row-major, device) by block Gauss-Jordan steps of
// sixteen pivots over the whole GPU, through the second buffer tmp; returns the launches made.
long long invert_spd_blocked(double* A, double* tmp, int n, cudaStream_t s, int* flag) {
  double *a = A, *b = tmp;
  const dim3 gg((n + kGJT - 1) / kGJT, (n + kGJT - 1) / kGJT);
  long long cnt = 0;
  for (int k0 = 0; k0 < n; k0 += kGJB, ++cnt) {
    k_coarse_invert_block<<<gg, 256, 0, s>>>(a, b, n, k0, flag);
    std::swap(a, b);
  }
  if (a != A) CK(cudaMemcpyAsync(A, a, (size_t)n * n * sizeof(double), cudaMemcpyDeviceToDevice, s));
  return cnt;
}

// true for memory the current device reads in place; host pointers are staged. Entry points reject
// other GPUs' memory up front (places_ok), so everything that is not PTR_HERE here is host memory.
bool is_device_ptr(const void* p) { return ptr_place(p) == PTR_HERE; }

// every non-null caller pointer is host memory or memory of the handle's device
bool places_ok(std::initializer_list<const void*> ptrs) {
  for (const void* p : ptrs)
    if (p && ptr_place(p) == PTR_OTHER) return false;
  return true;
}

struct DevAlloc {
  std::vector<void*> ptrs;
  size_t bytes = 0;
  template <typename T>
  T* get(size_t n) {
    void* p = nullptr;
    if (n == 0) n = 1;
    if (cudaMalloc(&p, n * sizeof(T)) != cudaSuccess) {
      cudaGetLastError();
      throw std::bad_alloc();
    }
    ptrs.push_back(p);
    bytes += n * sizeof(T);
    return (T*)p;
  }
  void release() {
    for (void* p : ptrs) cudaFree(p);
    ptrs.clear();
  }
};

Geom make_geom(int nx, int ny, double Lx, double Ly, const pyro_bc& bc) {
  Geom g;
  g.nx = nx; g.ny = ny; g.ld = nx + 2;
  g.dx = Lx / nx; g.dy = Ly / ny;
  auto s = [&](int side) { return bc.kind[side] == PYRO_BC_FREE_SLIP ? 1.0 : -1.0; };
  g.sW = s(0); g.sE = s(1); g.sN = s(2); g.sS = s(3);
  return g;
}

inline long long velocity_unknowns(int nx, int ny) { return (long long)ny * (nx - 1) + (long long)(ny - 1) * nx; }

// Cell counts of every level: halve while the ratio is 2, both counts are even and the short side
// stays >= cmin; then, while the coarsest level is too large for the dense inverse, coarsen by
// the ratio, n_c = ceil(n / ratio) (the paper's arbitrary coarsening ratio).
std::vector<std::pair<int, int>> level_sizes(int nx, int ny, int cmin, double ratio, bool general) {
  std::vector<std::pair<int, int>> sz{{nx, ny}};
  for (;;) {
    const int a = sz.back().first, b = sz.back().second;
    if (ratio == 2.0 && a % 2 == 0 && b % 2 == 0 && std::min(a, b) / 2 >= cmin) {
      sz.push_back({a / 2, b / 2});
      continue;
    }
    if (general && velocity_unknowns(a, b) > kMaxCoarse) {
      const int cx = (int)std::ceil(a / ratio - 1e-9), cy = (int)std::ceil(b / ratio - 1e-9);
      if (std::min(cx, cy) >= 2 && (cx != a || cy != b)) {
        sz.push_back({cx, cy});
        continue;
      }
    }
    return sz;
  }
}

// ---- multigrid hierarchy on one arithmetic type --------------------------------------------
template <typename T>
struct Level {
  Geom g;
  GeomT<T> gt;
  size_t P;
  T *vx, *vy, *fx, *fy, *rx, *ry, *en, *ec;
  // K-cycle vectors (allocated on levels whose coarse correction is Krylov-accelerated from above)
  T *d1x = nullptr, *d1y = nullptr, *q1x = nullptr, *q1y = nullptr, *ex = nullptr, *ey = nullptr;
  T *idgx = nullptr, *idgy = nullptr;  // precomputed 1/diag (FP64 levels)
  T *vx2 = nullptr, *vy2 = nullptr;    // second iterate buffer for the tile sweeps (ping-pong)
  Coef<T> kc{};                        // precomputed coefficients (FP64 levels smoothed per colour)
  bool own_kc = false;
  int cur = 0;                         // which buffer holds the iterate (set while launching)
  T* X() const { return cur ? vx2 : vx; }
  T* Y() const { return cur ? vy2 : vy; }
  double *kpart = nullptr, *ks = nullptr;
  int kblocks = 0;
  T* gal = nullptr;                    // Galerkin coarse operator R L P (2 x kGalSlots planes), else null
};

template <typename T>
struct MG {
  std::vector<Level<T>> lv;
  std::vector<char> f2;    // f2[l]: level l+1 is level l halved (factor-2 kernels), else any ratio
  double* Ainv = nullptr;  // coarsest (-L)^-1, dense FP64 (when coarse_direct)
  double* Atmp = nullptr;  // second buffer of the multi-launch inversion (nc > kCoarseInvertMulti)
  bool coarse_direct = true;  // coarsest level solved by the dense inverse, else by smoothing
  int coarse_sweeps = 40;     // smoothing sweeps on a coarsest level too large for the inverse
  int nc = 0;              // coarse unknowns
  int nu1 = 2, nu2 = 2, eta_mode = 0;
  int kcycle = 0;  // levels l < kcycle get their coarse correction from two flexible-CG steps
  bool tiles = true;                        // tile-fused smoothing / residual+restriction
  int tile_form = 0;                        // FP32 large levels: 0 warp-per-row tiles, 1 64 x 32 colour-split
  bool res64 = false;                       // FP32 cycles: finest residual formed in FP64 (option res64)
  GeomT<double> r64_g{};                    // ... with the FP64 outer operator's geometry and coefficients
  Coef<double> r64_kc{};
  int smoother = PYRO_SMOOTH_RBGS;          // velocity smoother (MIXED: Jacobi on level 0, RAS below)
  int ras_inner = 4;                        // RAS-type Jacobi: local iterations per tile pass
  int tile_sweeps = 2;                      // FP32: sweeps fused per tile launch
  int galerkin = 0;                         // 1: factor-2 coarse levels take R L P (damped-Jacobi smoothed)
  static constexpr long long kFuse64Cells = 65536;
  T omega = T(1);
  const cudaEvent_t* hooks = nullptr;  // level-0 phase events (timing mode), else null
  long long* nlaunch = nullptr;        // kernel-launch counter of the owning handle
  void count(long long k) const { if (nlaunch) *nlaunch += k; }
  // FP64 levels of up to 65536 cells: blocks of 64 threads, so even a tiny level spreads over many
  // SMs (one SM's FP64 pipe, about 2 FMA per clock, would otherwise serialise the whole level)
  static dim3 blk(const Level<T>& L) {
    return (sizeof(T) == 8 && (long long)L.g.nx * L.g.ny <= 65536) ? dim3(32, 2) : kBlk2;
  }

  static bool kc_level(int l, int nlev, int kcycle) { return l >= 1 && l - 1 < kcycle && l < nlev - 1; }

  // level l takes a Galerkin operator when every level above it halves its predecessor
  static bool gal_level(const std::vector<std::pair<int, int>>& sz, int l, int galerkin) {
    if (!galerkin || l < 1) return false;
    for (int k = 1; k <= l; ++k)
      if (sz[k].first * 2 != sz[k - 1].first || sz[k].second * 2 != sz[k - 1].second) return false;
    return true;
  }

  static size_t bytes(const std::vector<std::pair<int, int>>& sz, int kcycle = 0, int galerkin = 0) {
    size_t b = 0;
    const int nlev = (int)sz.size();
    for (int l = 0; l < nlev; ++l) {
      const size_t P = (size_t)(sz[l].second + 2) * (sz[l].first + 2);
      b += (size_t)(sizeof(T) == 8 ? 17 : 10) * P * sizeof(T);
      if (gal_level(sz, l, galerkin)) b += (size_t)2 * kGalSlots * P * sizeof(T) + 256;
      if (kc_level(l, nlev, kcycle)) b += (size_t)6 * P * sizeof(T) + 5 * 296 * 8 + 64;
    }
    const size_t nc = (size_t)velocity_unknowns(sz.back().first, sz.back().second);
    if (nc > (size_t)kMaxCoarse) return b;
    return b + (nc > (size_t)kCoarseInvertMulti ? 2 : 1) * nc * nc * sizeof(double);
  }

  void alloc(DevAlloc& A, const Geom& g0, double Lx, double Ly, const std::vector<std::pair<int, int>>& sz,
             bool alias_eta0) {
    Geom g = g0;
    const int nlev = (int)sz.size();
    for (int l = 0; l < nlev; ++l) {
      g.nx = sz[l].first; g.ny = sz[l].second; g.ld = g.nx + 2;
      g.dx = Lx / g.nx; g.dy = Ly / g.ny;
      f2.push_back(l + 1 < nlev && sz[l + 1].first * 2 == g.nx && sz[l + 1].second * 2 == g.ny);
      Level<T> L;
      L.g = g;
      L.gt = geomT<T>(g);
      L.P = (size_t)(g.ny + 2) * g.ld;
      L.vx = A.get<T>(L.P); L.vy = A.get<T>(L.P); L.fx = A.get<T>(L.P); L.fy = A.get<T>(L.P);
      L.rx = A.get<T>(L.P); L.ry = A.get<T>(L.P);
      if (l == 0 && alias_eta0) { L.en = nullptr; L.ec = nullptr; }
      else { L.en = A.get<T>(L.P); L.ec = A.get<T>(L.P); }
      if (sizeof(T) == 8) { L.idgx = A.get<T>(L.P); L.idgy = A.get<T>(L.P); }
      if (sizeof(T) == 8 && (!tiles || (long long)g.nx * g.ny > kFuse64Cells) && !(l == 0 && alias_eta0)) {
        T* k5 = A.get<T>(5 * L.P);
        L.kc = Coef<T>{k5, k5 + L.P, k5 + 2 * L.P, k5 + 3 * L.P, k5 + 4 * L.P};
        L.own_kc = true;
      }
      if (gal_level(sz, l, galerkin)) L.gal = A.get<T>((size_t)2 * kGalSlots * L.P);
      if (tiles || smoother != PYRO_SMOOTH_RBGS || L.gal) {
        L.vx2 = A.get<T>(L.P); L.vy2 = A.get<T>(L.P);
        CK(cudaMemset(L.vx2, 0, L.P * sizeof(T)));
        CK(cudaMemset(L.vy2, 0, L.P * sizeof(T)));
      }
      if (kc_level(l, nlev, kcycle)) {
        L.d1x = A.get<T>(L.P); L.d1y = A.get<T>(L.P); L.q1x = A.get<T>(L.P); L.q1y = A.get<T>(L.P);
        L.ex = A.get<T>(L.P); L.ey = A.get<T>(L.P);
        L.kblocks = (int)std::min<size_t>(296, (L.P + 255) / 256);
        L.kpart = A.get<double>((size_t)5 * 296);
        L.ks = A.get<double>(8);
      }
      lv.push_back(L);
    }
    const Geom& gc = lv.back().g;
    nc = gc.ny * (gc.nx - 1) + (gc.ny - 1) * gc.nx;
    coarse_direct = nc <= kMaxCoarse;
    if (coarse_direct) Ainv = A.get<double>((size_t)nc * nc);
    if (coarse_direct && nc > kCoarseInvertMulti) Atmp = A.get<double>((size_t)nc * nc);
  }

  // viscosity on every level + coarse inverse (eta of level 0 must already be in place)
  void setup(cudaStream_t s, int* flag) {
    for (size_t l = 1; l < lv.size(); ++l) {
      const Level<T>& F = lv[l - 1];
      Level<T>& C = lv[l];
      if (f2[l - 1])
        k_coarsen_eta<T><<<grid2(C.g.nx, C.g.ny, kBlk2), kBlk2, 0, s>>>(F.gt, C.gt, F.en, F.ec, C.en, C.ec, eta_mode);
      else
        k_coarsen_eta_gen<T><<<grid2(C.g.nx, C.g.ny, kBlk2), kBlk2, 0, s>>>(F.g, C.g, F.en, F.ec, C.en, C.ec,
                                                                             eta_mode);
    }
    for (size_t l = 0; l < lv.size(); ++l)
      if (lv[l].own_kc) {
        const Level<T>& L = lv[l];
        k_coefs<T><<<grid2(L.g.nx, L.g.ny, kBlk2), kBlk2, 0, s>>>(L.gt, L.en, L.ec, (T*)L.kc.cxx, (T*)L.kc.cyy,
                                                                   (T*)L.kc.nxx, (T*)L.kc.nyy, (T*)L.kc.nxy);
        count(1);
      }
    for (size_t l = 0; l < lv.size(); ++l)
      if (lv[l].idgx) {
        const Level<T>& L = lv[l];
        k_invdiag<T><<<grid2(L.g.nx, L.g.ny, kBlk2), kBlk2, 0, s>>>(L.gt, L.en, L.ec, L.idgx, L.idgy);
        count(1);
      }
    for (size_t l = 1; l < lv.size(); ++l)
      if (lv[l].gal) {
        const Level<T>& F = lv[l - 1];
        Level<T>& G = lv[l];
        const GalSrc<T> src{F.gt, F.gal ? nullptr : F.en, F.gal ? nullptr : F.ec, F.gal, F.P};
        k_gal_rap<T><<<grid2(G.g.nx, G.g.ny, kBlk2), kBlk2, 0, s>>>(src, G.gt, G.gal, G.P, flag);
        count(1);
      }
    const Level<T>& C = lv.back();
    if (!coarse_direct) return;
    CK(cudaMemsetAsync(Ainv, 0, (size_t)nc * nc * sizeof(double), s));
    if (C.gal)
      k_gal_coarse_assemble<T><<<(nc + 127) / 128, 128, 0, s>>>(C.gt, C.gal, C.P, Ainv, nc);
    else
      k_coarse_assemble<T><<<(nc + 127) / 128, 128, 0, s>>>(C.g, C.en, C.ec, Ainv, nc);
    if (nc > kCoarseInvertMulti) {
      count((long long)lv.size() - 1 + 1 + invert_spd_blocked(Ainv, Atmp, nc, s, flag));
    } else {
      k_coarse_invert<<<1, 1024, nc * sizeof(double), s>>>(Ainv, nc, flag);
      count((long long)lv.size() - 1 + 2);
    }
  }

  bool fused(int l) const {
    if (lv[l].gal) return false;
    return tiles && (sizeof(T) == 4 || (long long)lv[l].g.nx * lv[l].g.ny <= kFuse64Cells);
  }

  // nsweeps RBGS sweeps on level l with tile kernels; with C given, the prolongation of C's
  // iterate is added when the first tile is loaded
  void smooth_tiles(int l, int nsweeps, const Level<T>* C, cudaStream_t s) {
    Level<T>& L = lv[l];
    const GeomT<T> gc = C ? C->gt : L.gt;
    const T* cvx = C ? C->X() : nullptr;
    const T* cvy = C ? C->Y() : nullptr;
    if (nsweeps == 0 && C) {
      k_prolong_add<T><<<grid2(L.g.nx, L.g.ny, blk(L)), blk(L), 0, s>>>(L.gt, C->gt, L.X(), L.Y(), C->X(), C->Y());
      count(1);
      return;
    }
    while (nsweeps > 0) {
      if constexpr (sizeof(T) == 4) {
        float* ox = L.cur ? L.vx : L.vx2;
        float* oy = L.cur ? L.vy : L.vy2;
        const int ns = (nsweeps >= 2 && tile_sweeps >= 2) ? 2 : 1;
        if ((long long)L.g.nx * L.g.ny > kSmallTileCells && tile_form == 0) {
          // large levels: warp-per-row tiles (64-column regions, 32-slot colour rows)
          if (ns == 2) {
            using Tl = SweepTileW<2, kWTileY2>;
            const dim3 gr((L.g.nx + 2 + Tl::TX - 1) / Tl::TX, (L.g.ny + 2 + kWTileY2 - 1) / kWTileY2);
            k_rbgs_tile_w<2, kWTileY2><<<gr, kTileThreads, Tl::smem_bytes(), s>>>(
                L.gt, L.X(), L.Y(), ox, oy, L.fx, L.fy, L.en, L.ec, omega, gc, cvx, cvy);
          } else {
            using Tl = SweepTileW<1, kWTileY1>;
            const dim3 gr((L.g.nx + 2 + Tl::TX - 1) / Tl::TX, (L.g.ny + 2 + kWTileY1 - 1) / kWTileY1);
            k_rbgs_tile_w<1, kWTileY1><<<gr, kTileThreads, Tl::smem_bytes(), s>>>(
                L.gt, L.X(), L.Y(), ox, oy, L.fx, L.fy, L.en, L.ec, omega, gc, cvx, cvy);
          }
        } else if ((long long)L.g.nx * L.g.ny > kSmallTileCells) {
          constexpr int TX = 64, TY = 32;   // large levels: the least halo recomputation
          const dim3 gr((L.g.nx + 2 + TX - 1) / TX, (L.g.ny + 2 + TY - 1) / TY);
          if (ns == 2)
            k_rbgs_tile_cs<2, TX, TY><<<gr, kTileThreads, SweepTileCS<2, TX, TY>::smem_bytes(), s>>>(
                L.gt, L.X(), L.Y(), ox, oy, L.fx, L.fy, L.en, L.ec, omega, gc, cvx, cvy);
          else
            k_rbgs_tile_cs<1, TX, TY><<<gr, kTileThreads, SweepTileCS<1, TX, TY>::smem_bytes(), s>>>(
                L.gt, L.X(), L.Y(), ox, oy, L.fx, L.fy, L.en, L.ec, omega, gc, cvx, cvy);
        } else {
          constexpr int TX = 32, TY = 16;   // small levels: more, shorter CTAs (one CTA's chain of
                                            // half-sweeps is the critical path there)
          const dim3 gr((L.g.nx + 2 + TX - 1) / TX, (L.g.ny + 2 + TY - 1) / TY);
          if (ns == 2)
            k_rbgs_tile_cs<2, TX, TY><<<gr, kTileThreads, SweepTileCS<2, TX, TY>::smem_bytes(), s>>>(
                L.gt, L.X(), L.Y(), ox, oy, L.fx, L.fy, L.en, L.ec, omega, gc, cvx, cvy);
          else
            k_rbgs_tile_cs<1, TX, TY><<<gr, kTileThreads, SweepTileCS<1, TX, TY>::smem_bytes(), s>>>(
                L.gt, L.X(), L.Y(), ox, oy, L.fx, L.fy, L.en, L.ec, omega, gc, cvx, cvy);
        }
        nsweeps -= ns;
      } else {
        constexpr int TX = 64, TY = 16;
        const dim3 gr((L.g.nx + 2 + TX - 1) / TX, (L.g.ny + 2 + TY - 1) / TY);
        k_rbgs_tile<T, 1, TX, TY><<<gr, kTileThreads, SweepTile<T, 1, TX, TY>::smem_bytes(L.idgx != nullptr), s>>>(
            L.gt, L.X(), L.Y(), L.cur ? L.vx : L.vx2, L.cur ? L.vy : L.vy2, L.fx, L.fy, L.en, L.ec, L.idgx,
            L.idgy, omega, gc, cvx, cvy);
        nsweeps -= 1;
      }
      count(1);
      L.cur ^= 1;
      cvx = nullptr;
      cvy = nullptr;
    }
  }


  void resrestrict_tiles(int l, cudaStream_t s) {
    Level<T>& L = lv[l];
    Level<T>& C = lv[l + 1];
    constexpr int CTX = 32, CTY = sizeof(T) == 4 ? 16 : 8;
    const dim3 gr((C.g.nx + 2 + CTX - 1) / CTX, (C.g.ny + 2 + CTY - 1) / CTY);
    k_resrestrict_tile<T, CTX, CTY><<<gr, kTileThreads, ResTile<T, CTX, CTY>::smem_bytes(), s>>>(
        L.gt, C.gt, L.X(), L.Y(), L.fx, L.fy, L.en, L.ec, C.fx, C.fy, C.vx, C.vy);
    C.cur = 0;  // the coarse iterate starts from zero in its first buffer
    count(1);
  }

  // raise the dynamic shared-memory limit of the tile kernels (once per handle)
  static void enable_tiles() {
    if constexpr (sizeof(T) == 4) {
      CK(cudaFuncSetAttribute(k_rbgs_tile_cs<2, 64, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)SweepTileCS<2, 64, 32>::smem_bytes()));
      CK(cudaFuncSetAttribute(k_rbgs_tile_cs<1, 64, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)SweepTileCS<1, 64, 32>::smem_bytes()));
      CK(cudaFuncSetAttribute(k_rbgs_tile_w<2, kWTileY2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)SweepTileW<2, kWTileY2>::smem_bytes()));
      CK(cudaFuncSetAttribute(k_rbgs_tile_w<1, kWTileY1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)SweepTileW<1, kWTileY1>::smem_bytes()));
      CK(cudaFuncSetAttribute(k_rbgs_tile_cs<2, 32, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)SweepTileCS<2, 32, 16>::smem_bytes()));
      CK(cudaFuncSetAttribute(k_rbgs_tile_cs<1, 32, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)SweepTileCS<1, 32, 16>::smem_bytes()));
      CK(cudaFuncSetAttribute(k_resrestrict_tile<T, 32, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)ResTile<T, 32, 16>::smem_bytes()));
    } else {
      CK(cudaFuncSetAttribute(k_rbgs_tile<T, 1, 64, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)SweepTile<T, 1, 64, 16>::smem_bytes(true)));
      CK(cudaFuncSetAttribute(k_resrestrict_tile<T, 32, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)ResTile<T, 32, 8>::smem_bytes()));
    }
  }

  // the smoother of level l: the configured one, or for MIXED Jacobi on the finest level and the
  // RAS-type Jacobi smoother on the coarser ones
  int level_smoother(int l) const {
    if (smoother == PYRO_SMOOTH_MIXED) return l == 0 ? PYRO_SMOOTH_JACOBI : PYRO_SMOOTH_RAS;
    return smoother;
  }

  // nsweeps smoothing steps on level l with the level's smoother; with C given, the coarse
  // correction (prolongation of C's iterate) is added first. phase: 0 pre, 1 post (RAS shifts).
  void smooth(int l, int nsweeps, const Level<T>* C, int phase, cudaStream_t s) {
    Level<T>& L = lv[l];
    const int sm = level_smoother(l);
    if (sm == PYRO_SMOOTH_RBGS && fused(l)) {
      smooth_tiles(l, nsweeps, C, s);
      return;
    }
    if (C) {
      k_prolong_add<T><<<grid2(L.g.nx, L.g.ny, blk(L)), blk(L), 0, s>>>(L.gt, C->gt, L.X(), L.Y(), C->X(), C->Y());
      count(1);
    }
    if (L.gal) {
      // Galerkin level: damped Jacobi on the stored stencil (red-black ordering is not a Gauss-Seidel
      // ordering of its couplings)
      for (int k = 0; k < nsweeps; ++k) {
        k_gal_jacobi<T><<<grid2(L.g.nx, L.g.ny, blk(L)), blk(L), 0, s>>>(L.gt, L.gal, L.P, L.X(), L.Y(),
                                                                         L.cur ? L.vx : L.vx2, L.cur ? L.vy : L.vy2,
                                                                         L.fx, L.fy, T(kGalOmega));
        L.cur ^= 1;
      }
      count(nsweeps);
      return;
    }
    if (sm == PYRO_SMOOTH_RBGS) {
      for (int k = 0; k < nsweeps; ++k) sweep(l, s);
      return;
    }
    if (sm == PYRO_SMOOTH_JACOBI) {
      for (int k = 0; k < nsweeps; ++k) {
        k_jacobi<T><<<jacobi_grid(L.g.nx, L.g.ny), jacobi_block(), 0, s>>>(L.gt, L.X(), L.Y(), L.cur ? L.vx : L.vx2,
                                                                     L.cur ? L.vy : L.vy2, L.fx, L.fy, L.en, L.ec,
                                                                     omega);
        L.cur ^= 1;
      }
      count(nsweeps);
      return;
    }
    const int npass = (nsweeps + ras_inner - 1) / ras_inner;
    for (int t = 0; t < npass; ++t) {
      int si = 0, sj = 0;
      ras_shift(l, phase, t, kRasTile, kRasTile, si, sj);
      const dim3 gr((L.g.nx + 2 + sj + kRasTile - 1) / kRasTile, (L.g.ny + 2 + si + kRasTile - 1) / kRasTile);
      k_ras_tile<T, kRasTile, kRasTile><<<gr, 256, RasTile<kRasTile, kRasTile>::template smem_bytes<T>(), s>>>(
          L.gt, L.X(), L.Y(), L.cur ? L.vx : L.vx2, L.cur ? L.vy : L.vy2, L.fx, L.fy, L.en, L.ec, omega, si, sj,
          ras_inner);
      L.cur ^= 1;
    }
    count(npass);
  }

  static void enable_ras() {
    CK(cudaFuncSetAttribute(k_ras_tile<T, kRasTile, kRasTile>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                            (int)RasTile<kRasTile, kRasTile>::template smem_bytes<T>()));
  }

  void sweep(int l, cudaStream_t s) {
    Level<T>& L = lv[l];
    const dim3 b = blk(L), g = grid_rb(L.g.nx, L.g.ny, b);
    for (int f = 0; f < 2; ++f)
      for (int c = 0; c < 2; ++c)
        k_rbgs<T><<<g, b, 0, s>>>(L.gt, L.X(), L.Y(), L.fx, L.fy, L.en, L.ec, f, c, omega, L.idgx, L.idgy, L.kc);
    count(4);
  }

  // one V-cycle at level l for L x = f from x = 0 (x_l must be zero on entry)
  void cycle(int l, cudaStream_t s) {
    Level<T>& L = lv[l];
    // entry: the iterate is zero in the first buffer
    L.cur = 0;
    if (l == (int)lv.size() - 1) {
      if (coarse_direct) {
        k_coarse_solve<T><<<(nc + kCoarseRows - 1) / kCoarseRows, 32 * kCoarseRows, nc * sizeof(double), s>>>(
            L.g, Ainv, nc, L.fx, L.fy, L.vx, L.vy);
        count(1);
      } else {
        // too many coarsest unknowns for the dense inverse: smoothing sweeps from zero stand in for
        // the coarsest solve (the paper's "direct method or a few smoothing iterations")
        smooth(l, coarse_sweeps, nullptr, 2, s);
      }
      return;
    }
    Level<T>& C = lv[l + 1];
    const bool fz = fused(l);
    smooth(l, nu1, nullptr, 0, s);
    if (l == 0 && hooks) CK(cudaEventRecordWithFlags(hooks[2], s, cudaEventRecordExternal));
    bool restricted = false;
    if constexpr (sizeof(T) == 4) {
      if (l == 0 && res64 && f2[0] && !L.gal) {
        // finest residual of the FP32 cycle formed in FP64 (option res64), then the restriction
        k_vresidual64<T><<<grid2(L.g.nx, L.g.ny, blk(L)), blk(L), 0, s>>>(r64_g, L.X(), L.Y(), L.fx, L.fy, r64_kc,
                                                                           L.rx, L.ry);
        k_restrict<T><<<grid2(C.g.nx, C.g.ny, blk(C)), blk(C), 0, s>>>(L.gt, C.gt, L.rx, L.ry, C.fx, C.fy, C.vx,
                                                                         C.vy);   // also zeroes the coarse iterate
        count(2);
        C.cur = 0;
        restricted = true;
      }
    }
    if (restricted) {
    } else if (fz && f2[l]) {
      resrestrict_tiles(l, s);  // also zeroes the coarse iterate
    } else if (!f2[l]) {
      if (L.gal)
        k_gal_resid<T><<<grid2(L.g.nx, L.g.ny, blk(L)), blk(L), 0, s>>>(L.gt, L.gal, L.P, L.X(), L.Y(), L.fx, L.fy,
                                                                         L.rx, L.ry);
      else
        k_vresidual<T><<<grid2(L.g.nx, L.g.ny, blk(L)), blk(L), 0, s>>>(L.gt, L.X(), L.Y(), L.fx, L.fy, L.en, L.ec,
                                                                         L.rx, L.ry, L.kc);
      k_restrict_gen<T><<<grid2(C.g.nx, C.g.ny, blk(C)), blk(C), 0, s>>>(L.g, C.g, L.gt, L.rx, L.ry, C.fx, C.fy, C.vx,
                                                                          C.vy);
      count(2);
      C.cur = 0;
    } else {
      if (L.gal)
        k_gal_resid<T><<<grid2(L.g.nx, L.g.ny, blk(L)), blk(L), 0, s>>>(L.gt, L.gal, L.P, L.X(), L.Y(), L.fx, L.fy,
                                                                         L.rx, L.ry);
      else
        k_vresidual<T><<<grid2(L.g.nx, L.g.ny, blk(L)), blk(L), 0, s>>>(L.gt, L.X(), L.Y(), L.fx, L.fy, L.en, L.ec,
                                                                         L.rx, L.ry, L.kc);
      k_restrict<T><<<grid2(C.g.nx, C.g.ny, blk(C)), blk(C), 0, s>>>(L.gt, C.gt, L.rx, L.ry, C.fx, C.fy, C.vx,
                                                                       C.vy);   // also zeroes the coarse iterate
      count(2);
      C.cur = 0;
    }
    if (kc_level(l + 1, (int)lv.size(), kcycle)) {
      // K-cycle: two flexible-CG steps on level l+1, each preconditioned by one level-(l+1) cycle
      const int nb = C.kblocks;
      cycle(l + 1, s);
      k_kc_step1<T><<<nb, 256, 0, s>>>(C.gt, C.X(), C.Y(), C.fx, C.fy, C.en, C.ec, C.d1x, C.d1y, C.q1x, C.q1y, C.kpart);
      k_kc_reduce<<<1, 256, 0, s>>>(C.kpart, nb, 2, C.ks);
      // zero the first iterate buffer for the second inner cycle
      k_kc_update1<T><<<nb, 256, 0, s>>>(C.P, C.ks, C.d1x, C.d1y, C.q1x, C.q1y, C.ex, C.ey, C.fx, C.fy, C.vx, C.vy);
      cycle(l + 1, s);
      k_kc_step2<T><<<nb, 256, 0, s>>>(C.gt, C.X(), C.Y(), C.fx, C.fy, C.en, C.ec, C.q1x, C.q1y, C.kpart);
      k_kc_reduce<<<1, 256, 0, s>>>(C.kpart, nb, 3, C.ks + 2);
      k_kc_final<T><<<nb, 256, 0, s>>>(C.P, C.ks, C.ks + 2, C.d1x, C.d1y, C.ex, C.ey, C.X(), C.Y());
      count(6);
    } else {
      cycle(l + 1, s);
    }
    // prolongation + correction (fused into the first post-smoothing pass of the RBGS tiles)
    const bool fused_post = level_smoother(l) == PYRO_SMOOTH_RBGS && fz && f2[l];
    if (!fused_post) {
      if (f2[l])
        k_prolong_add<T><<<grid2(L.g.nx, L.g.ny, blk(L)), blk(L), 0, s>>>(L.gt, C.gt, L.X(), L.Y(), C.X(), C.Y());
      else
        k_prolong_gen<T><<<grid2(L.g.nx, L.g.ny, blk(L)), blk(L), 0, s>>>(L.g, C.g, C.gt, L.X(), L.Y(), C.X(), C.Y());
      count(1);
    }
    if (l == 0 && hooks) CK(cudaEventRecordWithFlags(hooks[3], s, cudaEventRecordExternal));
    smooth(l, nu2, fused_post ? &C : nullptr, 1, s);
    if (l == 0 && hooks) CK(cudaEventRecordWithFlags(hooks[4], s, cudaEventRecordExternal));
  }
};

}  // namespace

// ---- pressure multigrid of the weighted BFBt Schur surrogate ----------------------------------
// Levels of the pressure grid (compact nx * ny cells): level 0 holds the face conductances, each
// coarser level (ceil halves, 2 x 2 aggregates) a 5 x 5-box Galerkin stencil; the coarsest level
// (<= kSchurMaxCoarse cells) a dense inverse. One V-cycle: nu damped Jacobi sweeps from zero,
// residual, restriction P^T r, the coarse cycle, x += P e, nu damped Jacobi sweeps.
template <typename T>
struct SchurMG {
  struct Lv {
    int nx = 0, ny = 0;
    size_t n = 0;
    T *cx = nullptr, *cy = nullptr, *box = nullptr, *diag = nullptr, *widg = nullptr;
    T *x = nullptr, *x2 = nullptr, *f = nullptr, *pw = nullptr;
    int cur = 0;
    T* X() const { return cur ? x2 : x; }
    T* Xo() const { return cur ? x : x2; }
  };
  std::vector<Lv> lv;
  T *wix = nullptr, *wiy = nullptr;  // W^-1 at the velocity unknowns of the finest grid (padded)
  double* Ainv = nullptr;
  double* Atmp = nullptr;            // second buffer of the one-launch-per-pivot inversion (nc > 80)
  int nc = 0;
  int nu = 2;
  T omega_s = T(0.8), omega_p = T(2.0 / 3.0);
  long long* nlaunch = nullptr;
  void count(long long k) const { if (nlaunch) *nlaunch += k; }

  static std::vector<std::pair<int, int>> sizes(int nx, int ny) {
    std::vector<std::pair<int, int>> v{{nx, ny}};
    while ((long long)nx * ny > kSchurMaxCoarse) {
      nx = (nx + 1) / 2;
      ny = (ny + 1) / 2;
      v.push_back({nx, ny});
    }
    return v;
  }
  static size_t bytes(int nx, int ny, size_t P) {
    const auto sz = sizes(nx, ny);
    size_t b = 2 * P * sizeof(T);
    for (size_t l = 0; l < sz.size(); ++l) {
      const size_t n = (size_t)sz[l].first * sz[l].second;
      b += (3 + 2) * n * sizeof(T);                                    // x, x2, f, diag, omega/diag
      b += (l == 0 ? 2 : kSchurBox) * n * sizeof(T);                   // conductances / box stencil
      if (l + 1 < sz.size()) b += 4 * n * sizeof(T);                   // prolongator rows
      b += 5 * 256;                                                    // allocation rounding
    }
    const size_t ncl = (size_t)sz.back().first * sz.back().second;
    return b + (ncl > (size_t)kCoarseInvertMulti ? 2 : 1) * ncl * ncl * sizeof(double);
  }
  void alloc(DevAlloc& A, int nx, int ny, size_t P) {
    const auto sz = sizes(nx, ny);
    wix = A.get<T>(P);
    wiy = A.get<T>(P);
    for (size_t l = 0; l < sz.size(); ++l) {
      Lv L;
      L.nx = sz[l].first; L.ny = sz[l].second;
      L.n = (size_t)L.nx * L.ny;
      if (l == 0) { L.cx = A.get<T>(L.n); L.cy = A.get<T>(L.n); }
      else L.box = A.get<T>((size_t)kSchurBox * L.n);
      L.diag = A.get<T>(L.n);
      L.widg = A.get<T>(L.n);
      L.x = A.get<T>(L.n); L.x2 = A.get<T>(L.n); L.f = A.get<T>(L.n);
      if (l + 1 < sz.size()) L.pw = A.get<T>(4 * L.n);
      lv.push_back(L);
    }
    nc = (int)lv.back().n;
    Ainv = A.get<double>((size_t)nc * nc);
    if (nc > kCoarseInvertMulti) Atmp = A.get<double>((size_t)nc * nc);
  }
  PLev<T> plev(int l) const {
    const Lv& L = lv[l];
    return PLev<T>{L.nx, L.ny, L.cx, L.cy, L.box, L.diag, L.widg};
  }
  static unsigned nb(size_t n) { return (unsigned)((n + 255) / 256); }

  // conductances from the finest level's viscosity, prolongators and Galerkin coarse operators,
  // dense coarsest inverse
  void setup(const GeomT<T>& g, const T* en, const T* ec, cudaStream_t s, int* flag) {
    k_schur_weights<T, T><<<grid2(g.nx, g.ny, kBlk2), kBlk2, 0, s>>>(g, en, ec, wix, wiy, lv[0].cx, lv[0].cy,
                                                                     lv[0].diag, lv[0].widg, omega_s);
    for (size_t l = 0; l + 1 < lv.size(); ++l) {
      const Lv& F = lv[l];
      Lv& C = lv[l + 1];
      k_schur_prow<T><<<nb(F.n), 256, 0, s>>>(plev((int)l), C.nx, C.ny, omega_p, F.pw);
      k_schur_rap<T><<<(unsigned)((16 * C.n + kSchurRapThreads - 1) / kSchurRapThreads), kSchurRapThreads,
                       kSchurRapThreads * kSchurBox * sizeof(T), s>>>(plev((int)l), F.pw, C.nx, C.ny, C.box, C.diag,
                                                                      C.widg, omega_s);
    }
    k_schur_coarse_assemble<T><<<1, 1024, 0, s>>>(plev((int)lv.size() - 1), Ainv);
    if (nc > kCoarseInvertMulti) {
      // sixteen Gauss-Jordan pivots per launch over the whole GPU (a single CTA would take milliseconds)
      count(1 + 2 * ((long long)lv.size() - 1) + 1 + invert_spd_blocked(Ainv, Atmp, nc, s, flag));
    } else {
      k_coarse_invert<<<1, 1024, nc * sizeof(double), s>>>(Ainv, nc, flag);
      count(1 + 2 * ((long long)lv.size() - 1) + 2);
    }
  }

  // residual of level l restricted to level l + 1 (and, if smoothed, its first sweep from zero)
  template <int CT>
  void resrestrict_ct(int l, bool coarse_smoothed, cudaStream_t s) {
    Lv& L = lv[l];
    Lv& C = lv[l + 1];
    const dim3 gr((C.nx + CT - 1) / CT, (C.ny + CT - 1) / CT);
    k_schur_resrestrict<T, CT><<<gr, schur_rr_threads<CT>(), 0, s>>>(plev(l), L.X(), L.f, L.pw, C.nx, C.ny, C.f,
                                                                     C.widg, coarse_smoothed ? C.x : nullptr);
    count(1);
  }
  void resrestrict(int l, bool coarse_smoothed, cudaStream_t s) {
    const int ct = schur_tile_ct((long long)lv[l + 1].n);
    if (ct == 16) resrestrict_ct<16>(l, coarse_smoothed, s);
    else if (ct == 8) resrestrict_ct<8>(l, coarse_smoothed, s);
    else resrestrict_ct<4>(l, coarse_smoothed, s);
  }

  // one damped Jacobi sweep X() -> Xo()
  void jacobi(int l, cudaStream_t s) {
    Lv& L = lv[l];
    k_schur_jacobi<T><<<nb(L.n), 256, 0, s>>>(plev(l), L.X(), L.Xo(), L.f, T(1) - omega_s);
    L.cur ^= 1;
    count(1);
  }

  // one V-cycle on level l for K x = lv[l].f from zero; the result is lv[l].X(). On entry lv[l].x
  // already holds the first Jacobi sweep from zero (omega f / diag): whoever writes a level's
  // right-hand side writes it too (k_precond_out_schur and k_schur_div on the finest level, the
  // fused residual-restriction below), which saves one launch per level and visit. The residual
  // and the restriction run as one tile kernel, and so do the prolongation and the first
  // post-smoothing sweep: 4 launches per level and visit instead of 7, same arithmetic.
  void cycle(int l, cudaStream_t s) {
    Lv& L = lv[l];
    const int last = (int)lv.size() - 1;
    if (l == last) {
      k_schur_coarse_solve<T><<<(nc + 7) / 8, 256, 0, s>>>(Ainv, nc, L.f, L.x);
      L.cur = 0;
      count(1);
      return;
    }
    Lv& C = lv[l + 1];
    L.cur = 0;
    for (int k = 1; k < nu; ++k) jacobi(l, s);
    resrestrict(l, l + 1 < last, s);
    cycle(l + 1, s);
    const dim3 gp((L.nx + kSchurTS - 1) / kSchurTS, (L.ny + kSchurTS - 1) / kSchurTS);
    if (l == 0)
      k_schur_prolong_jacobi<T, 1><<<gp, 256, 0, s>>>(plev(l), L.X(), L.pw, C.X(), C.nx, C.ny, L.f, T(1) - omega_s, L.Xo());
    else
      k_schur_prolong_jacobi<T, 2><<<gp, 256, 0, s>>>(plev(l), L.X(), L.pw, C.X(), C.nx, C.ny, L.f, T(1) - omega_s, L.Xo());
    L.cur ^= 1;
    count(1);
    for (int k = 1; k < nu; ++k) jacobi(l, s);
  }
};

// ---- inner flexible CG on the finest velocity level (option inner_cg): FP64 recurrence -------
struct InnerCG {
  double *xx = nullptr, *xy = nullptr, *wx = nullptr, *wy = nullptr, *dx = nullptr, *dy = nullptr, *qx = nullptr,
         *qy = nullptr, *rx = nullptr, *ry = nullptr;
  double *part = nullptr, *scal = nullptr;
  static size_t bytes(size_t P) { return 10 * P * sizeof(double) + (2 * kReduceBlocks + 3) * sizeof(double) + 12 * 256; }
  void alloc(DevAlloc& A, size_t P) {
    double** arr[10] = {&xx, &xy, &wx, &wy, &dx, &dy, &qx, &qy, &rx, &ry};
    for (double** a : arr) {
      *a = A.get<double>(P);
      CK(cudaMemset(*a, 0, P * sizeof(double)));
    }
    part = A.get<double>(2 * kReduceBlocks);
    scal = A.get<double>(3);
    CK(cudaMemset(scal, 0, 3 * sizeof(double)));
  }
};

// ---- the handle -----------------------------------------------------------------------------
struct pyro_stokes_s {
  int dev = 0;
  int nx = 0, ny = 0;
  double Lx = 1, Ly = 1;
  pyro_bc bc{};
  pyro_opts o{};
  Geom g{};
  GeomT<double> g64{};
  size_t P = 0, n3 = 0;
  int nlev = 1;
  bool mixed = true;
  DevAlloc mem;
  // FP64 state
  Coef<double> okc{};  // coefficients of the FP64 outer operator (shared with FP64 level 0)
  double *en = nullptr, *ec = nullptr, *rho = nullptr, *b = nullptr, *x = nullptr, *r = nullptr, *w = nullptr,
         *W = nullptr, *stage = nullptr, *xf = nullptr, *V = nullptr;
  void* Z = nullptr;
  double *h1 = nullptr, *h2 = nullptr, *partial = nullptr, *part2 = nullptr, *hcol = nullptr, *inv = nullptr,
         *ydev = nullptr;
  int *d_j = nullptr, *flag = nullptr;
  double *sw = nullptr, *isw = nullptr;    // W^(1/2), W^(-1/2) (modified Gram-Schmidt basis scaling)
  double* zc = nullptr;                    // GCR / Anderson: the current preconditioned residual
  double *en_full = nullptr, *ec_full = nullptr;  // continuation: the full-contrast viscosity
  int *d_slot = nullptr, *d_cnt = nullptr;  // Anderson: history slot of this step, pairs stored
  // pinned host scratch
  double* hbuf = nullptr;
  int* hflag = nullptr;
  MG<float> mgf;
  MG<double> mgd;
  SchurMG<float> smf;                        // weighted BFBt pressure block (option schur = 1, mixed)
  SchurMG<double> smd;                       // the same block in FP64 (FP64 mode, or schur = 2)
  double* sc64 = nullptr;                    // schur = 2 in mixed mode: FP64 middle-product planes (4 P)
  InnerCG ic;                                 // inner flexible CG on the finest velocity level
  std::vector<cudaGraphExec_t> graphs;       // captured iteration graphs (per Krylov column with MGS)
  std::vector<long long> graph_kernel_counts;
  int cur_j = 0;                              // Krylov column of the step being launched or captured
  cudaEvent_t ev[4]{};
  bool have_solution = false;
  double last_gx = 0, last_gy = 0;
  int m = 30;
  size_t dot_grid_y = 1;
  // timing mode
  bool timing = false, graph_timing = false;
  cudaEvent_t tev[7]{};
  double tacc[6]{};
  long long tcount[2]{};
  long long launches = 0;       // kernels launched by the current call
  long long graph_kernels = 0;  // kernel nodes of the captured iteration graph
};

namespace {

inline void mark(pyro_stokes_s* h, int k, cudaStream_t s) {
  if (h->timing) CK(cudaEventRecordWithFlags(h->tev[k], s, cudaEventRecordExternal));
}

// partial[k * nblk + b] = block b's share of sum_e (W[e]) w[e] V_k[e], k < *d_cnt + 1 + off: the
// one-pass register kernel while the basis fits (m + 1 <= kDotRegs), else groups of 8 vectors.
// Returns nblk, the number of partials per vector (for k_reduce).
template <bool WEIGHTED>
int multidot(pyro_stokes_s* h, cudaStream_t s, const double* V, const int* d_cnt, const double* w, int off) {
  if (h->m + 1 <= kDotRegs) {
    k_multidot_r<WEIGHTED><<<kDotBlocks, kThreads, 0, s>>>(V, h->n3, d_cnt, w, h->W, h->n3, h->partial, off);
    return kDotBlocks;
  }
  k_multidot<WEIGHTED><<<dim3(kReduceBlocks, (unsigned)h->dot_grid_y), kThreads, 0, s>>>(
      V, h->n3, d_cnt, 0, w, h->W, h->n3, h->partial, off);
  return kReduceBlocks;
}

template <typename T>
SchurMG<T>& schur_of(pyro_stokes_s* h);
template <>
SchurMG<float>& schur_of<float>(pyro_stokes_s* h) { return h->smf; }
template <>
SchurMG<double>& schur_of<double>(pyro_stokes_s* h) { return h->smd; }

// z = M^-1 v with v = in + (*d_idx) in_stride and z = out + (*d_idx) out_stride (device index), and
// optionally w = A z.
template <typename T, typename TZ>
void precond_body(pyro_stokes_s* h, MG<T>& mg, cudaStream_t s, const double* in, size_t in_stride, TZ* out,
                  size_t out_stride, const int* d_idx, bool with_apply, const double* isw) {
  Level<T>& L0 = mg.lv[0];
  mark(h, 0, s);
  k_precond_in<T><<<kReduceBlocks, kThreads, 0, s>>>(h->P, in, in_stride, d_idx, L0.fx, L0.fy, L0.vx, L0.vy, isw);
  mark(h, 1, s);
  mg.hooks = h->timing ? h->tev : nullptr;
  mg.nlaunch = &h->launches;
  const T* zvx = nullptr;
  const T* zvy = nullptr;
  if (h->o.inner_cg > 0) {
    // inner flexible CG on L z_v = r_v (the residual lives in the level-0 right-hand side), each step
    // preconditioned by one V-cycle; the phase events time the first cycle only
    InnerCG& ic = h->ic;
    k_fcg_init<<<kReduceBlocks, kThreads, 0, s>>>(h->P, in, in_stride, d_idx, isw, ic.rx, ic.ry);
    for (int k = 0; k < h->o.inner_cg; ++k) {
      const int first = k == 0;
      // step 0's right-hand side and zero iterate were set by k_precond_in
      if (!first) k_fcg_load<T><<<kReduceBlocks, kThreads, 0, s>>>(L0.P, ic.rx, ic.ry, L0.fx, L0.fy, L0.vx, L0.vy);
      mg.cycle(0, s);
      mg.hooks = nullptr;
      k_fcg_apply<T><<<kReduceBlocks, kThreads, 0, s>>>(h->g64, L0.X(), L0.Y(), h->en, h->ec, ic.qx, ic.qy, ic.wx,
                                                        ic.wy, first, ic.part);
      k_fcg_beta<<<1, kThreads, 0, s>>>(ic.part, kReduceBlocks, first, ic.scal);
      k_fcg_orth<T><<<kReduceBlocks, kThreads, 0, s>>>(h->g64, L0.X(), L0.Y(), ic.wx, ic.wy, ic.rx, ic.ry, ic.dx,
                                                       ic.dy, ic.qx, ic.qy, ic.scal, first, ic.part);
      k_fcg_alpha<<<1, kThreads, 0, s>>>(ic.part, kReduceBlocks, ic.scal);
      k_fcg_update<<<kReduceBlocks, kThreads, 0, s>>>(h->P, ic.dx, ic.dy, ic.qx, ic.qy, ic.xx, ic.xy, ic.rx, ic.ry,
                                                      ic.scal, first);
      h->launches += first ? 5 : 6;
    }
    k_fcg_store<T><<<kReduceBlocks, kThreads, 0, s>>>(L0.P, ic.xx, ic.xy, L0.vx, L0.vy);
    L0.cur = 0;
    h->launches += 2;
    zvx = L0.vx;
    zvy = L0.vy;
  } else {
    mg.cycle(0, s);
    zvx = L0.X();
    zvy = L0.Y();
  }
  mg.hooks = nullptr;
  h->launches += 3;
  bool schur_done = false;
  if constexpr (sizeof(T) == 4) {
    if (h->o.schur == 2) {
      // the weighted BFBt block in FP64 after the FP32 V-cycle: the same steps as below on the FP64
      // pressure hierarchy, the middle product on the FP64 viscosity and outer coefficient planes
      SchurMG<double>& sm = h->smd;
      auto& F0 = sm.lv[0];
      sm.nlaunch = &h->launches;
      double* ux = h->sc64;
      double* uy = ux + h->P;
      double* wx = uy + h->P;
      double* wy = wx + h->P;
      k_precond_out_schur<T, TZ, double><<<kReduceBlocks, kThreads, 0, s>>>(h->g64, zvx, zvy, in, in_stride, out,
                                                                            out_stride, d_idx, F0.f, isw, F0.widg,
                                                                            F0.x);
      sm.cycle(0, s);
      const dim3 g2 = grid2(h->nx, h->ny, kBlk2);
      k_schur_grad<double><<<g2, kBlk2, 0, s>>>(h->g64, F0.X(), sm.wix, sm.wiy, ux, uy);
      k_schur_lw<double, double><<<g2, kBlk2, 0, s>>>(h->g64, ux, uy, h->en, h->ec, sm.wix, sm.wiy, wx, wy, h->okc);
      k_schur_div<double><<<SchurMG<double>::nb(F0.n), 256, 0, s>>>(h->g64, wx, wy, F0.f, F0.widg, F0.x);
      sm.cycle(0, s);
      k_schur_out<double, TZ><<<kReduceBlocks, kThreads, 0, s>>>(h->g64, F0.X(), h->o.alpha_p, out, out_stride,
                                                                  d_idx, h->part2);
      h->launches += 4;
      schur_done = true;
    }
  }
  if (schur_done) {
  } else if (h->o.schur) {
    // weighted BFBt pressure block: z_p = alpha K^-1 (D W^-1 (-L) W^-1 G) K^-1 (r_p - D z_v)
    SchurMG<T>& sm = schur_of<T>(h);
    auto& F0 = sm.lv[0];
    sm.nlaunch = &h->launches;
    k_precond_out_schur<T, TZ><<<kReduceBlocks, kThreads, 0, s>>>(h->g64, zvx, zvy, in, in_stride, out,
                                                                   out_stride, d_idx, F0.f, isw, F0.widg, F0.x);
    sm.cycle(0, s);
    const dim3 g2 = grid2(h->nx, h->ny, kBlk2);
    k_schur_grad<T><<<g2, kBlk2, 0, s>>>(L0.gt, F0.X(), sm.wix, sm.wiy, L0.rx, L0.ry);
    k_schur_lw<T, T><<<g2, kBlk2, 0, s>>>(L0.gt, L0.rx, L0.ry, L0.en, L0.ec, sm.wix, sm.wiy, L0.fx, L0.fy, L0.kc);
    k_schur_div<T><<<SchurMG<T>::nb(F0.n), 256, 0, s>>>(L0.gt, L0.fx, L0.fy, F0.f, F0.widg, F0.x);
    sm.cycle(0, s);
    k_schur_out<T, TZ><<<kReduceBlocks, kThreads, 0, s>>>(h->g64, F0.X(), h->o.alpha_p, out, out_stride, d_idx,
                                                           h->part2);
    h->launches += 4;
  } else {
    k_precond_out<T, TZ><<<kReduceBlocks, kThreads, 0, s>>>(h->g64, zvx, zvy, in, in_stride, out, out_stride,
                                                             d_idx, h->ec, h->o.alpha_p, h->part2, isw);
  }
  k_sub_mean<TZ><<<kReduceBlocks, kThreads, 0, s>>>(h->g64, out + 2 * h->P, out_stride, d_idx, h->part2, kReduceBlocks);
  if (with_apply) {
    k_apply<TZ><<<grid2(h->nx, h->ny, kBlk2), kBlk2, 0, s>>>(h->g64, h->en, h->ec, (const TZ*)out, out_stride, d_idx,
                                                              h->w, h->okc);
    h->launches += 1;
  }
  mark(h, 5, s);
}

// isw (optional): the input is stored scaled by W^(1/2) and is unscaled on the way in
void precond_any(pyro_stokes_s* h, cudaStream_t s, const double* in, size_t in_stride, double* out,
                 size_t out_stride, const int* d_idx, bool with_apply, const double* isw = nullptr) {
  if (h->mixed) precond_body<float, double>(h, h->mgf, s, in, in_stride, out, out_stride, d_idx, with_apply, isw);
  else precond_body<double, double>(h, h->mgd, s, in, in_stride, out, out_stride, d_idx, with_apply, isw);
}

// one Arnoldi step j (j read on the device): z_j = M^-1 v_j, w = A z_j, CGS2 against v_0..v_j,
// v_{j+1} = w / ||w||_W, Hessenberg column j into hcol, j += 1.
void fgmres_body(pyro_stokes_s* h, cudaStream_t s) {
  precond_any(h, s, h->V, h->n3, (double*)h->Z, h->n3, h->d_j, true);
  // classical Gram-Schmidt with one re-orthogonalisation (CGS2) in the W inner product
  int nb = multidot<true>(h, s, h->V, h->d_j, h->w, 0);
  k_reduce<<<h->m + 1, kThreads, 0, s>>>(h->partial, nb, h->d_j, 0, h->h1);
  k_multiaxpy<<<kReduceBlocks * 2, kThreads, 0, s>>>(h->w, h->V, h->n3, h->d_j, h->h1, h->n3, nullptr, nullptr);
  nb = multidot<true>(h, s, h->V, h->d_j, h->w, 0);
  k_reduce<<<h->m + 1, kThreads, 0, s>>>(h->partial, nb, h->d_j, 0, h->h2);
  k_multiaxpy<<<kReduceBlocks * 2, kThreads, 0, s>>>(h->w, h->V, h->n3, h->d_j, h->h2, h->n3, h->W, h->part2);
  k_arnoldi_finish<<<1, kThreads, 0, s>>>(h->d_j, h->h1, h->h2, h->part2, 2 * kReduceBlocks, h->hcol, h->inv,
                                          h->flag);
  k_scale_next<<<kReduceBlocks * 2, kThreads, 0, s>>>(h->V, h->n3, h->d_j, h->w, h->inv, h->n3);
  k_inc<<<1, 1, 0, s>>>(h->d_j);
  h->launches += 9;
  mark(h, 6, s);
}

constexpr int kMgsBlocks = 592;   // blocks of one modified Gram-Schmidt step (4 per SM)

// One Arnoldi step j with modified Gram-Schmidt (option gram_schmidt = 1), the basis stored scaled
// by W^(1/2) so that the W inner product is a plain dot product: z_j = M^-1 (W^(-1/2) v_j),
// w = A z_j, then the m + 1 fused steps of k_mgs_step (those beyond column j's j + 2 return at
// once), each subtracting the previous basis vector's component and forming the next inner
// product, then the column's norm.
void fgmres_body_mgs(pyro_stokes_s* h, cudaStream_t s) {
  precond_any(h, s, h->V, h->n3, (double*)h->Z, h->n3, h->d_j, true, h->isw);
  double* pb = h->partial;   // two alternating partial buffers of kReduceBlocks
  const int nsteps = std::min(h->cur_j + 2, h->m + 1);   // steps 0 .. j + 1 of column j
  for (int k = 0; k < nsteps; ++k)
    k_mgs_step<<<kMgsBlocks, kThreads, 0, s>>>(h->V, h->n3, h->d_j, k, h->w, h->sw, h->n3,
                                               pb + (size_t)((k + 1) & 1) * kMgsBlocks,
                                               pb + (size_t)(k & 1) * kMgsBlocks, h->h1);
  k_mgs_finish<<<1, kThreads, 0, s>>>(h->d_j, h->h1, pb, kMgsBlocks, h->hcol, h->inv, h->flag);
  k_scale_next<<<kReduceBlocks * 2, kThreads, 0, s>>>(h->V, h->n3, h->d_j, h->w, h->inv, h->n3);
  k_inc<<<1, 1, 0, s>>>(h->d_j);
  h->launches += nsteps + 3;
  mark(h, 6, s);
}

// one flexible GCR step j (Algorithm gcr; j on the device): z = M^-1 r, w = A z, CGS2 of w against
// the normalised images w_0..w_{j-1} (V) with the same coefficients applied to z against
// z_0..z_{j-1} (Z), normalisation, then x += alpha z_j, r -= alpha w_j with alpha = <r, w_j>_W
// (the W inner product: the method minimises the energy residual, as FGMRES does here).
void gcr_body(pyro_stokes_s* h, cudaStream_t s) {
  precond_any(h, s, h->r, 0, h->zc, 0, h->d_j, true);
  double* Zb = (double*)h->Z;
  for (int pass = 0; pass < 2; ++pass) {
    double* hc = pass == 0 ? h->h1 : h->h2;
    const int nb = multidot<true>(h, s, h->V, h->d_j, h->w, -1);
    k_reduce<<<h->m + 1, kThreads, 0, s>>>(h->partial, nb, h->d_j, 0, hc, -1);
    k_multiaxpy<<<kReduceBlocks, kThreads, 0, s>>>(h->w, h->V, h->n3, h->d_j, hc, h->n3, pass ? h->W : nullptr,
                                                   pass ? h->part2 : nullptr, -1);
    k_multiaxpy<<<kReduceBlocks * 2, kThreads, 0, s>>>(h->zc, Zb, h->n3, h->d_j, hc, h->n3, nullptr, nullptr, -1);
  }
  // ||w||_W: the second pass left its per-block partials in part2 (also when j = 0 and no vector is
  // subtracted); the Hessenberg column it also writes is not used by GCR
  k_arnoldi_finish<<<1, kThreads, 0, s>>>(h->d_j, h->h1, h->h2, h->part2, kReduceBlocks, h->hcol, h->inv, h->flag);
  k_gcr_scale<<<kReduceBlocks, kThreads, 0, s>>>(h->V, Zb, h->n3, h->d_j, h->w, h->zc, h->inv, h->r, h->W, h->n3,
                                                 h->partial);
  k_reduce<<<1, kThreads, 0, s>>>(h->partial, kReduceBlocks, nullptr, 1, h->ydev);
  k_gcr_update<<<kReduceBlocks, kThreads, 0, s>>>(h->x, h->r, h->V, Zb, h->n3, h->d_j, h->ydev, h->W, h->n3,
                                                  h->part2);
  k_reduce<<<1, kThreads, 0, s>>>(h->part2, kReduceBlocks, nullptr, 1, h->ydev + 1);
  k_inc<<<1, 1, 0, s>>>(h->d_j);
  h->launches += 15;
  mark(h, 6, s);
}

// one Anderson step (Algorithm anderson, the fixed-point map G(x) = x + M^-1 (b - A x)):
// r = b - A x with its energy / l2 norms, z = M^-1 r, history slot d_slot <- (x, z), and the dots
// <z, z_i> (2-norm) with the d_cnt stored residuals; the host then solves the constrained
// least-squares problem and combines (k_aa_combine).
void aa_body(pyro_stokes_s* h, cudaStream_t s) {
  k_residual<<<kReduceBlocks, kThreads, 0, s>>>(h->g64, h->en, h->ec, h->b, h->x, h->r, h->W, h->partial, h->okc);
  k_sum_pairs<<<1, kThreads, 0, s>>>(h->partial, kReduceBlocks, h->ydev);
  precond_any(h, s, h->r, 0, h->zc, 0, h->d_j, false);
  k_aa_store<<<kReduceBlocks * 2, kThreads, 0, s>>>(h->V, (double*)h->Z, h->n3, h->d_slot, h->x, h->zc, h->n3);
  const int nb = multidot<false>(h, s, (double*)h->Z, h->d_cnt, h->zc, -1);
  k_reduce<<<h->m + 1, kThreads, 0, s>>>(h->partial, nb, h->d_cnt, 0, h->h1, -1);
  h->launches += 6;
  mark(h, 6, s);
}

void iteration_body(pyro_stokes_s* h, cudaStream_t s) {
  if (h->o.accel == PYRO_ACCEL_GCR) gcr_body(h, s);
  else if (h->o.accel == PYRO_ACCEL_ANDERSON) aa_body(h, s);
  else if (h->sw) fgmres_body_mgs(h, s);
  else fgmres_body(h, s);
}

// after the iteration's sync: accumulate the phase times
void collect_timing(pyro_stokes_s* h) {
  if (!h->timing) return;
  float t[6];
  const int pairs[6][2] = {{0, 1}, {1, 2}, {2, 3}, {3, 4}, {4, 5}, {5, 6}};
  for (int k = 0; k < 6; ++k) {
    t[k] = 0.f;
    if (cudaEventElapsedTime(&t[k], h->tev[pairs[k][0]], h->tev[pairs[k][1]]) != cudaSuccess) {
      cudaGetLastError();
      t[k] = 0.f;
    }
    h->tacc[k] += t[k];
  }
  h->tcount[0] += 1;
  h->tcount[1] += h->o.nu1 + h->o.nu2;
}

// j: the Krylov column of this step (host side); the modified Gram-Schmidt iteration captures one
// graph per column (exactly j + 2 orthogonalisation steps), every other iteration one graph
void launch_iteration(pyro_stokes_s* h, cudaStream_t s, int j = 0) {
  if (h->o.use_graphs) {
    const size_t slot = h->sw ? (size_t)j : 0;
    if (h->graphs.size() <= slot) h->graphs.resize(slot + 1, nullptr);
    if (h->graph_timing != h->timing) {
      for (auto& g : h->graphs)
        if (g) { cudaGraphExecDestroy(g); g = nullptr; }
    }
    cudaGraphExec_t& graph = h->graphs[slot];
    h->cur_j = j;
    if (!graph) {
      std::lock_guard<std::recursive_mutex> lk(device_sync_lock());
      const long long saved = h->launches;  // capture records kernels, it does not launch them
      h->graph_timing = h->timing;
      cudaStream_t cs;
      CK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
      cudaGraph_t gr;
      CK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
      iteration_body(h, cs);
      cudaError_t e = cudaStreamEndCapture(cs, &gr);
      cudaStreamDestroy(cs);
      CK(e);
      size_t nn = 0;
      h->graph_kernels = 0;
      if (cudaGraphGetNodes(gr, nullptr, &nn) == cudaSuccess && nn > 0) {
        std::vector<cudaGraphNode_t> nodes(nn);
        cudaGraphGetNodes(gr, nodes.data(), &nn);
        for (auto nd : nodes) {
          cudaGraphNodeType t;
          if (cudaGraphNodeGetType(nd, &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++h->graph_kernels;
        }
      }
      e = cudaGraphInstantiate(&graph, gr, 0);
      cudaGraphDestroy(gr);
      h->launches = saved;
      CK(e);
      if (h->graph_kernel_counts.size() <= slot) h->graph_kernel_counts.resize(slot + 1, 0);
      h->graph_kernel_counts[slot] = h->graph_kernels;
    }
    CK(cudaGraphLaunch(graph, s));
    h->launches += h->graph_kernel_counts[slot];
  } else {
    h->cur_j = j;
    iteration_body(h, s);
  }
}

// host-side sum of the per-block partials (fixed order)
std::pair<double, double> residual_norms(pyro_stokes_s* h, const double* b, const double* x, double* r, cudaStream_t s) {
  k_residual<<<kReduceBlocks, kThreads, 0, s>>>(h->g64, h->en, h->ec, b, x, r, h->W, h->partial, h->okc);
  h->launches += 1;
  CK(cudaMemcpyAsync(h->hbuf, h->partial, 2 * kReduceBlocks * sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  double a = 0, c = 0;
  for (int k = 0; k < kReduceBlocks; ++k) { a += h->hbuf[2 * k]; c += h->hbuf[2 * k + 1]; }
  return {a, c};
}

double weighted_norm2(pyro_stokes_s* h, const double* v, cudaStream_t s) {
  k_multidot<true><<<dim3(kReduceBlocks, 1), kThreads, 0, s>>>(v, 0, nullptr, 1, v, h->W, h->n3, h->partial);
  h->launches += 1;
  CK(cudaMemcpyAsync(h->hbuf, h->partial, kReduceBlocks * sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  double a = 0;
  for (int k = 0; k < kReduceBlocks; ++k) a += h->hbuf[k];
  return a;
}

double l2_norm2(pyro_stokes_s* h, const double* v, cudaStream_t s) {
  k_sumsq<<<kReduceBlocks, kThreads, 0, s>>>(v, h->n3, h->partial);
  h->launches += 1;
  CK(cudaMemcpyAsync(h->hbuf, h->partial, kReduceBlocks * sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  double c = 0;
  for (int k = 0; k < kReduceBlocks; ++k) c += h->hbuf[k];
  return c;
}

void ingest(pyro_stokes_s* h, const double* src, double* dst, int kind, cudaStream_t s) {
  const double* from = src;
  if (!is_device_ptr(src)) {
    CK(cudaMemcpyAsync(h->stage, src, h->P * sizeof(double), cudaMemcpyHostToDevice, s));
    from = h->stage;
  }
  k_ingest<<<grid2(h->nx, h->ny, kBlk2), kBlk2, 0, s>>>(h->nx, h->ny, h->g.ld, from, dst, kind, h->flag);
  h->launches += 1;
}

// write x (3 planes) to caller arrays (host or device), ghosts by the boundary rule
void emit(pyro_stokes_s* h, const double* x, double* vx, double* vy, double* p, bool with_bc_consts, cudaStream_t s) {
  const double cN = with_bc_consts && h->bc.kind[2] == PYRO_BC_VELOCITY ? 2 * h->bc.vt[2] : 0.0;
  const double cS = with_bc_consts && h->bc.kind[3] == PYRO_BC_VELOCITY ? 2 * h->bc.vt[3] : 0.0;
  const double cW = with_bc_consts && h->bc.kind[0] == PYRO_BC_VELOCITY ? 2 * h->bc.vt[0] : 0.0;
  const double cE = with_bc_consts && h->bc.kind[1] == PYRO_BC_VELOCITY ? 2 * h->bc.vt[1] : 0.0;
  double* outs[3] = {vx, vy, p};
  bool dev[3];
  for (int k = 0; k < 3; ++k) dev[k] = outs[k] && is_device_ptr(outs[k]);
  double* d[3];
  for (int k = 0; k < 3; ++k) d[k] = outs[k] ? (dev[k] ? outs[k] : h->stage + k * h->P) : nullptr;
  k_output<<<grid2(h->nx, h->ny, kBlk2), kBlk2, 0, s>>>(h->g64, x, d[0], d[1], d[2], cN, cS, cW, cE);
  h->launches += 1;
  for (int k = 0; k < 3; ++k)
    if (outs[k] && !dev[k]) CK(cudaMemcpyAsync(outs[k], d[k], h->P * sizeof(double), cudaMemcpyDeviceToHost, s));
}

void outer_coefs(pyro_stokes_s* h, cudaStream_t s) {
  k_coefs<double><<<grid2(h->nx, h->ny, kBlk2), kBlk2, 0, s>>>(h->g64, h->en, h->ec, (double*)h->okc.cxx,
                                                               (double*)h->okc.cyy, (double*)h->okc.nxx,
                                                               (double*)h->okc.nyy, (double*)h->okc.nxy);
  h->launches += 1;
}

void setup_eta(pyro_stokes_s* h, cudaStream_t s) {
  outer_coefs(h, s);
  // level-0 viscosity of the V-cycle: FP32 copies (mixed) or the FP64 arrays themselves
  if (h->mixed) {
    Level<float>& L0 = h->mgf.lv[0];
    k_to_float<<<kReduceBlocks, kThreads, 0, s>>>(h->en, L0.en, h->P);
    k_to_float<<<kReduceBlocks, kThreads, 0, s>>>(h->ec, L0.ec, h->P);
    h->launches += 2;
    h->mgf.nlaunch = &h->launches;
    h->mgf.setup(s, h->flag);
    if (h->o.schur == 1) {
      h->smf.nlaunch = &h->launches;
      h->smf.setup(L0.gt, L0.en, L0.ec, s, h->flag);
    } else if (h->o.schur == 2) {
      h->smd.nlaunch = &h->launches;
      h->smd.setup(h->g64, h->en, h->ec, s, h->flag);
    }
  } else {
    h->mgd.nlaunch = &h->launches;
    h->mgd.setup(s, h->flag);
    if (h->o.schur) {
      const Level<double>& D0 = h->mgd.lv[0];
      h->smd.nlaunch = &h->launches;
      h->smd.setup(D0.gt, D0.en, D0.ec, s, h->flag);
    }
  }
  k_weights<<<grid2(h->nx, h->ny, kBlk2), kBlk2, 0, s>>>(h->g64, h->en, h->ec, h->W);
  if (h->sw) {
    k_sqrt_weights<<<kReduceBlocks, kThreads, 0, s>>>(h->W, h->sw, h->isw, h->n3);
    h->launches += 1;
  }
  h->launches += 1;
}

// Givens-rotation least squares of FGMRES on the host
struct Givens {
  std::vector<double> H, cs, sn, gv;
  int m;
  explicit Givens(int m_) : H((size_t)(m_ + 1) * m_), cs(m_), sn(m_), gv(m_ + 1), m(m_) {}
  double& at(int i, int j) { return H[(size_t)j * (m + 1) + i]; }
  void start(double beta) { std::fill(gv.begin(), gv.end(), 0.0); gv[0] = beta; }
  // returns |residual estimate|
  double add_column(int j, const double* col) {
    for (int i = 0; i <= j + 1; ++i) at(i, j) = col[i];
    for (int k = 0; k < j; ++k) {
      const double t = cs[k] * at(k, j) + sn[k] * at(k + 1, j);
      at(k + 1, j) = -sn[k] * at(k, j) + cs[k] * at(k + 1, j);
      at(k, j) = t;
    }
    const double a = at(j, j), bb = at(j + 1, j);
    const double d = std::hypot(a, bb);
    cs[j] = d > 0 ? a / d : 1.0;
    sn[j] = d > 0 ? bb / d : 0.0;
    at(j, j) = d;
    at(j + 1, j) = 0.0;
    gv[j + 1] = -sn[j] * gv[j];
    gv[j] = cs[j] * gv[j];
    return std::fabs(gv[j + 1]);
  }
  void solve(int k, double* y) {
    for (int i = k - 1; i >= 0; --i) {
      double t = gv[i];
      for (int l = i + 1; l < k; ++l) t -= at(i, l) * y[l];
      y[i] = at(i, i) != 0.0 ? t / at(i, i) : 0.0;
    }
  }
};

// FGMRES(m) on A x = b (h->b, h->x), preconditioned by one Uzawa/multigrid sweep, minimising the
// W-weighted (energy) residual; restarts recompute the true FP64 residual (refinement step).
int fgmres(pyro_stokes_s* h, double tol, pyro_stats* st, cudaStream_t s) {
  const auto t0 = std::chrono::steady_clock::now();
  CK(cudaEventRecord(h->ev[2], s));
  const double nb2 = weighted_norm2(h, h->b, s);
  const double nb = std::sqrt(nb2);
  Givens gv(h->m);
  std::vector<double> y(h->m);
  int total = 0, restarts = 0, status = PYRO_OK;
  double rel_e = 1.0;
  if (nb == 0.0) {
    CK(cudaMemsetAsync(h->x, 0, h->n3 * sizeof(double), s));
    rel_e = 0.0;
  }
  while (nb > 0.0) {
    auto rn = residual_norms(h, h->b, h->x, h->r, s);
    const double beta = std::sqrt(rn.first);
    rel_e = beta / nb;
    if (!std::isfinite(beta)) { status = PYRO_E_NONFINITE; break; }
    if (rel_e <= tol) break;
    if (total >= h->o.max_iter) { status = PYRO_W_NOT_CONVERGED; break; }
    if (h->o.timeout_s > 0) {
      const double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
      if (el > h->o.timeout_s) { status = PYRO_E_TIMEOUT; break; }
    }
    if (h->sw)
      k_scale_sw<<<kReduceBlocks * 2, kThreads, 0, s>>>(h->V, h->r, h->sw, 1.0 / beta, h->n3);
    else
      k_scale<<<kReduceBlocks * 2, kThreads, 0, s>>>(h->V, h->r, 1.0 / beta, h->n3);
    h->launches += 1;
    CK(cudaMemsetAsync(h->d_j, 0, sizeof(int), s));
    gv.start(beta);
    int k = 0;
    bool stop_inner = false;
    for (int j = 0; j < h->m; ++j) {
      launch_iteration(h, s, j);
      CK(cudaMemcpyAsync(h->hbuf, h->hcol + (size_t)j * kHcolStride, (j + 2) * sizeof(double), cudaMemcpyDeviceToHost, s));
      CK(cudaMemcpyAsync(h->hflag, h->flag, sizeof(int), cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      collect_timing(h);
      ++total;
      k = j + 1;
      if (*h->hflag & FLAG_NONFINITE) { status = PYRO_E_NONFINITE; stop_inner = true; break; }
      const double est = gv.add_column(j, h->hbuf);
      const double hnext = h->hbuf[j + 1];
      if (!std::isfinite(est)) { status = PYRO_E_NONFINITE; stop_inner = true; break; }
      // stop the cycle a little below tol so the true residual check at restart passes
      if (est <= 0.5 * tol * nb || hnext <= 1e-300) break;
      if (total >= h->o.max_iter) break;
      if (h->o.timeout_s > 0) {
        const double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        if (el > h->o.timeout_s) break;
      }
    }
    if (stop_inner && status != PYRO_OK) break;
    gv.solve(k, y.data());
    std::memcpy(h->hbuf, y.data(), k * sizeof(double));
    CK(cudaMemcpyAsync(h->ydev, h->hbuf, k * sizeof(double), cudaMemcpyHostToDevice, s));
    k_update_x<double><<<kReduceBlocks * 2, kThreads, 0, s>>>(h->x, (const double*)h->Z, h->n3, k, h->ydev, h->n3);
    h->launches += 1;
    ++restarts;
  }
  // zero-mean pressure (eq. pressure_normalization), then the final true residuals
  k_psum<<<kReduceBlocks, kThreads, 0, s>>>(h->g64, h->x + 2 * h->P, h->part2);
  k_sub_mean<double><<<kReduceBlocks, kThreads, 0, s>>>(h->g64, h->x + 2 * h->P, 0, nullptr, h->part2, kReduceBlocks);
  h->launches += 2;
  auto rn = residual_norms(h, h->b, h->x, h->r, s);
  CK(cudaEventRecord(h->ev[3], s));
  CK(cudaStreamSynchronize(s));
  if (st) {
    st->iters += total;
    st->restarts += restarts;
    st->vcycles += total;
    st->rel_energy_res = nb > 0 ? std::sqrt(rn.first) / nb : 0.0;
    float ms = 0;
    cudaEventElapsedTime(&ms, h->ev[2], h->ev[3]);
    st->t_solve_ms += ms;
    // algorithmic bytes: per iteration one V-cycle, the FP64 operator, and CGS2 over j+1 vectors
    const double cells = (double)h->nx * h->ny;
    const double tb = h->mixed ? 4.0 : 8.0;
    const double vcycle = (h->o.nu1 + h->o.nu2) * 8.0 * tb * 4.0 / 3.0 + 10.0 * tb;
    const double per_it = vcycle + 64.0 + 2 * 24.0 + 24.0 * 4.0 * (h->m / 4.0 + 1);
    st->alg_bytes += cells * per_it * total;
  }
  if (status == PYRO_OK && !(rel_e <= tol) && nb > 0) {
    const double fin = std::sqrt(rn.first) / nb;
    if (!(fin <= tol)) status = PYRO_W_NOT_CONVERGED;
  }
  if (st) {
    const double l2b = l2_norm2(h, h->b, s);
    st->rel_l2_res = l2b > 0 ? std::sqrt(rn.second / l2b) : 0.0;
  }
  return status;
}

// common end of an outer solve: zero-mean pressure, final true residuals, statistics
int finish_solve(pyro_stokes_s* h, double tol, pyro_stats* st, cudaStream_t s, int status, int total, int restarts,
                 double nb, double rel_e, double per_it_vectors) {
  k_psum<<<kReduceBlocks, kThreads, 0, s>>>(h->g64, h->x + 2 * h->P, h->part2);
  k_sub_mean<double><<<kReduceBlocks, kThreads, 0, s>>>(h->g64, h->x + 2 * h->P, 0, nullptr, h->part2, kReduceBlocks);
  h->launches += 2;
  auto rn = residual_norms(h, h->b, h->x, h->r, s);
  CK(cudaEventRecord(h->ev[3], s));
  CK(cudaStreamSynchronize(s));
  if (st) {
    st->iters += total;
    st->restarts += restarts;
    st->vcycles += total;
    st->rel_energy_res = nb > 0 ? std::sqrt(rn.first) / nb : 0.0;
    float ms = 0;
    cudaEventElapsedTime(&ms, h->ev[2], h->ev[3]);
    st->t_solve_ms += ms;
    const double cells = (double)h->nx * h->ny;
    const double tb = h->mixed ? 4.0 : 8.0;
    const double vcycle = (h->o.nu1 + h->o.nu2) * 8.0 * tb * 4.0 / 3.0 + 10.0 * tb;
    st->alg_bytes += cells * (vcycle + 64.0 + 24.0 * per_it_vectors) * total;
  }
  if (status == PYRO_OK && !(rel_e <= tol) && nb > 0) {
    const double fin = std::sqrt(rn.first) / nb;
    if (!(fin <= tol)) status = PYRO_W_NOT_CONVERGED;
  }
  if (st) {
    const double l2b = l2_norm2(h, h->b, s);
    st->rel_l2_res = l2b > 0 ? std::sqrt(rn.second / l2b) : 0.0;
  }
  return status;
}

bool out_of_time(const pyro_stokes_s* h, std::chrono::steady_clock::time_point t0) {
  if (h->o.timeout_s <= 0) return false;
  return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count() > h->o.timeout_s;
}

// Flexible GCR(m) (Algorithm gcr) in the W inner product; every restart recomputes the true FP64
// residual (refinement step), within a cycle the residual is updated recursively.
int gcr(pyro_stokes_s* h, double tol, pyro_stats* st, cudaStream_t s) {
  const auto t0 = std::chrono::steady_clock::now();
  CK(cudaEventRecord(h->ev[2], s));
  const double nb = std::sqrt(weighted_norm2(h, h->b, s));
  int total = 0, restarts = 0, status = PYRO_OK;
  double rel_e = 1.0;
  if (nb == 0.0) {
    CK(cudaMemsetAsync(h->x, 0, h->n3 * sizeof(double), s));
    rel_e = 0.0;
  }
  while (nb > 0.0) {
    auto rn = residual_norms(h, h->b, h->x, h->r, s);
    rel_e = std::sqrt(rn.first) / nb;
    if (!std::isfinite(rel_e)) { status = PYRO_E_NONFINITE; break; }
    if (rel_e <= tol) break;
    if (total >= h->o.max_iter) { status = PYRO_W_NOT_CONVERGED; break; }
    if (out_of_time(h, t0)) { status = PYRO_E_TIMEOUT; break; }
    CK(cudaMemsetAsync(h->d_j, 0, sizeof(int), s));
    bool stop = false;
    for (int j = 0; j < h->m; ++j) {
      launch_iteration(h, s);
      CK(cudaMemcpyAsync(h->hbuf, h->ydev, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
      CK(cudaMemcpyAsync(h->hflag, h->flag, sizeof(int), cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      collect_timing(h);
      ++total;
      const double est = std::sqrt(std::fabs(h->hbuf[1])) / nb;
      if ((*h->hflag & FLAG_NONFINITE) || !std::isfinite(est)) { status = PYRO_E_NONFINITE; stop = true; break; }
      if (est <= 0.5 * tol || total >= h->o.max_iter || out_of_time(h, t0)) break;
    }
    if (stop) break;
    ++restarts;
  }
  return finish_solve(h, tol, st, s, status, total, restarts, nb, rel_e, 6.0 * (h->m / 4.0 + 1) + 4.0);
}

// Anderson acceleration AA(m, beta) of the Uzawa fixed-point map (Algorithm anderson). The
// constrained least-squares problem min ||F a||_2, sum a = 1 over the newest cnt = min(m, k) + 1
// fixed-point residuals is solved on the host from their Gram matrix: a = G^-1 1 / (1^T G^-1 1),
// with G regularised by 1e-13 of its largest diagonal entry; the first step is x^1 = G(x^0).
int anderson(pyro_stokes_s* h, double tol, pyro_stats* st, cudaStream_t s) {
  const auto t0 = std::chrono::steady_clock::now();
  CK(cudaEventRecord(h->ev[2], s));
  const double nb = std::sqrt(weighted_norm2(h, h->b, s));
  const int depth = h->m;                 // AA depth m: up to m + 1 stored pairs
  const int nslot = depth + 1;
  std::vector<double> Gm((size_t)nslot * nslot, 0.0), a(nslot);
  int total = 0, status = PYRO_OK;
  double rel_e = nb > 0 ? 1.0 : 0.0;
  if (nb == 0.0) CK(cudaMemsetAsync(h->x, 0, h->n3 * sizeof(double), s));
  for (int k = 0; nb > 0.0; ++k) {
    const int slot = k % nslot, cnt = std::min(k + 1, nslot);
    int idx[2] = {slot, cnt};
    CK(cudaMemcpyAsync(h->d_slot, &idx[0], sizeof(int), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(h->d_cnt, &idx[1], sizeof(int), cudaMemcpyHostToDevice, s));
    launch_iteration(h, s);
    CK(cudaMemcpyAsync(h->hbuf, h->ydev, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(h->hbuf + 2, h->h1, cnt * sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(h->hflag, h->flag, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    collect_timing(h);
    rel_e = std::sqrt(h->hbuf[0]) / nb;       // energy residual of the current iterate x^k
    if ((*h->hflag & FLAG_NONFINITE) || !std::isfinite(rel_e)) { status = PYRO_E_NONFINITE; break; }
    if (rel_e <= tol) break;
    if (total >= h->o.max_iter) { status = PYRO_W_NOT_CONVERGED; break; }
    if (out_of_time(h, t0)) { status = PYRO_E_TIMEOUT; break; }
    ++total;
    for (int i = 0; i < cnt; ++i) { Gm[(size_t)slot * nslot + i] = h->hbuf[2 + i]; Gm[(size_t)i * nslot + slot] = h->hbuf[2 + i]; }
    // solve (G + eps I) y = 1 on the cnt stored slots by Gaussian elimination with partial pivoting
    std::vector<long double> M((size_t)cnt * (cnt + 1));
    double dmax = 0.0;
    for (int i = 0; i < cnt; ++i) dmax = std::max(dmax, Gm[(size_t)i * nslot + i]);
    for (int i = 0; i < cnt; ++i) {
      for (int j = 0; j < cnt; ++j) M[(size_t)i * (cnt + 1) + j] = Gm[(size_t)i * nslot + j];
      M[(size_t)i * (cnt + 1) + i] += 1e-13L * dmax;
      M[(size_t)i * (cnt + 1) + cnt] = 1.0L;
    }
    for (int c = 0; c < cnt; ++c) {
      int piv = c;
      for (int i = c + 1; i < cnt; ++i)
        if (std::fabs((double)M[(size_t)i * (cnt + 1) + c]) > std::fabs((double)M[(size_t)piv * (cnt + 1) + c])) piv = i;
      if (piv != c)
        for (int j = 0; j <= cnt; ++j) std::swap(M[(size_t)c * (cnt + 1) + j], M[(size_t)piv * (cnt + 1) + j]);
      const long double d = M[(size_t)c * (cnt + 1) + c];
      if (d == 0.0L) continue;
      for (int i = c + 1; i < cnt; ++i) {
        const long double f = M[(size_t)i * (cnt + 1) + c] / d;
        for (int j = c; j <= cnt; ++j) M[(size_t)i * (cnt + 1) + j] -= f * M[(size_t)c * (cnt + 1) + j];
      }
    }
    std::vector<long double> y(cnt, 0.0L);
    for (int i = cnt - 1; i >= 0; --i) {
      long double t = M[(size_t)i * (cnt + 1) + cnt];
      for (int j = i + 1; j < cnt; ++j) t -= M[(size_t)i * (cnt + 1) + j] * y[j];
      const long double d = M[(size_t)i * (cnt + 1) + i];
      y[i] = d != 0.0L ? t / d : 0.0L;
    }
    long double sy = 0.0L;
    for (int i = 0; i < cnt; ++i) sy += y[i];
    for (int i = 0; i < cnt; ++i) a[i] = (sy != 0.0L) ? (double)(y[i] / sy) : (i == slot ? 1.0 : 0.0);
    std::memcpy(h->hbuf, a.data(), cnt * sizeof(double));
    CK(cudaMemcpyAsync(h->ydev + 2, h->hbuf, cnt * sizeof(double), cudaMemcpyHostToDevice, s));
    const double beta = k == 0 ? 1.0 : h->o.aa_beta;     // x^1 = G(x^0)
    k_aa_combine<<<kReduceBlocks * 2, kThreads, 0, s>>>(h->x, h->V, (double*)h->Z, h->n3, cnt, h->ydev + 2, beta,
                                                        h->n3);
    h->launches += 1;
  }
  return finish_solve(h, tol, st, s, status, total, 0, nb, rel_e, 3.0 * (h->m + 1) + 4.0);
}

int outer_solve(pyro_stokes_s* h, double tol, pyro_stats* st, cudaStream_t s) {
  if (h->o.accel == PYRO_ACCEL_GCR) return gcr(h, tol, st, s);
  if (h->o.accel == PYRO_ACCEL_ANDERSON) return anderson(h, tol, st, s);
  return fgmres(h, tol, st, s);
}

// Viscosity-contrast continuation: cont_stages stages with theta = k / cont_stages (k = 0 ..
// cont_stages - 1), each cont_iters iterations of the outer solver on eta_comp = (1 - theta)
// eta_min + theta eta from the previous stage's iterate, then the full-contrast solve to tol.
int continuation_solve(pyro_stokes_s* h, double tol, pyro_stats* st, cudaStream_t s) {
  CK(cudaMemcpyAsync(h->en_full, h->en, h->P * sizeof(double), cudaMemcpyDeviceToDevice, s));
  CK(cudaMemcpyAsync(h->ec_full, h->ec, h->P * sizeof(double), cudaMemcpyDeviceToDevice, s));
  k_eta_min<<<kReduceBlocks, kThreads, 0, s>>>(h->g64, h->en, h->ec, h->partial);
  h->launches += 1;
  CK(cudaMemcpyAsync(h->hbuf, h->partial, kReduceBlocks * sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  double emin = h->hbuf[0];
  for (int b = 1; b < kReduceBlocks; ++b) emin = std::min(emin, h->hbuf[b]);
  const int max_iter = h->o.max_iter;
  int status = PYRO_OK;
  for (int k = 0; k < h->o.cont_stages; ++k) {
    const double theta = (double)k / h->o.cont_stages;
    k_eta_blend<<<kReduceBlocks, kThreads, 0, s>>>(h->g64, h->en_full, h->ec_full, h->en, h->ec, theta, emin);
    h->launches += 1;
    setup_eta(h, s);
    h->o.max_iter = h->o.cont_iters;
    status = outer_solve(h, tol, st, s);
    h->o.max_iter = max_iter;
    if (status < 0) return status;
  }
  CK(cudaMemcpyAsync(h->en, h->en_full, h->P * sizeof(double), cudaMemcpyDeviceToDevice, s));
  CK(cudaMemcpyAsync(h->ec, h->ec_full, h->P * sizeof(double), cudaMemcpyDeviceToDevice, s));
  setup_eta(h, s);
  return outer_solve(h, tol, st, s);
}

// FGMRES orthogonalisation: modified Gram-Schmidt when asked, or (gram_schmidt 2) when the grid is
// large enough that each step's FP64 arithmetic outweighs its launch: with FGMRES(30) the measured
// crossover lies between 512^2, where CGS2 is 1-2% faster, and 1024^2, where MGS is 10-17% faster;
// with the serving handles' FGMRES(200), 1024 x 512 and 2048 x 512 requests solve 18-27% faster
// (6-18% on the first solve, which also captures the per-column graphs), 1024 x 256 ones at par
constexpr long long kMgsMinCells = 1LL << 19;
bool use_mgs(const pyro_opts& o, int nx, int ny) {
  if (o.accel != PYRO_ACCEL_FGMRES) return false;
  if (o.gram_schmidt == 1) return true;
  return o.gram_schmidt == 2 && (long long)nx * ny >= kMgsMinCells;
}

// true when every option lies in the range pyro.h documents (nothing is clamped or replaced)
bool opts_valid(const pyro_opts& o) {
  return o.nu1 >= 0 && o.nu2 >= 0 && o.nu1 + o.nu2 >= 1 && o.omega_v > 0.0 && o.omega_v < 2.0 &&
         o.alpha_p > 0.0 && std::isfinite(o.alpha_p) && o.restart_m >= 1 && o.restart_m <= kMaxRestart &&
         o.max_iter >= 1 && (o.prec == PYRO_PREC_FP64 || o.prec == PYRO_PREC_MIXED) && o.coarsest_min >= 1 &&
         (o.eta_coarsen == PYRO_ETA_ARITH || o.eta_coarsen == PYRO_ETA_GEOM) && o.kcycle >= 0 && o.kcycle <= 16 &&
         (o.tile_fusion == 0 || o.tile_fusion == 1 || o.tile_fusion == 4) && o.cluster_cells <= 0 &&
         (o.tile_sweeps == 1 || o.tile_sweeps == 2) &&
         (o.tile_fusion64 == 0 || o.tile_fusion64 == 1) && o.accel >= PYRO_ACCEL_FGMRES &&
         o.accel <= PYRO_ACCEL_ANDERSON && o.aa_beta > 0.0 && o.aa_beta <= 1.0 && o.smoother >= PYRO_SMOOTH_RBGS &&
         o.smoother <= PYRO_SMOOTH_MIXED && o.ras_inner >= 1 && o.cont_stages >= 0 && o.cont_iters >= 1 &&
         o.coarse_sweeps >= 1 && o.coarsen_ratio >= 1.5 && o.coarsen_ratio <= 8.0 &&
         o.gram_schmidt >= 0 && o.gram_schmidt <= 2 && o.schur >= 0 && o.schur <= 2 &&
         (o.galerkin == 0 || (o.galerkin == 1 && o.kcycle == 0 && o.cluster_cells <= 0)) && o.inner_cg >= 0 &&
         o.inner_cg <= 16 && (o.res64 == 0 || o.res64 == 1);
}

std::vector<std::pair<int, int>> sizes_of(int nx, int ny, const pyro_opts& o) {
  return level_sizes(nx, ny, o.coarsest_min, o.coarsen_ratio, o.coarsen_general != 0);
}

int check_size(int nx, int ny, const pyro_opts& o) {
  if (nx < 2 || ny < 2 || (long long)(nx + 2) * (ny + 2) > (1LL << 31)) return PYRO_E_INVALID;
  return (int)sizes_of(nx, ny, o).size();
}


size_t footprint_bytes(int nx, int ny, const pyro_opts& o, int L) {
  const size_t P = (size_t)(ny + 2) * (nx + 2);
  const size_t n3 = 3 * P;
  const bool mixed = o.prec == PYRO_PREC_MIXED;
  const size_t m = (size_t)o.restart_m;
  size_t b = 0;
  b += 3 * P * 8;                  // en, ec, rho
  b += 5 * P * 8;                  // outer operator coefficients
  b += 6 * n3 * 8;                 // b, x, r, w, W, xf
  b += n3 * 8;                     // stage
  b += (m + 1) * n3 * 8;           // V
  b += (m + 1) * n3 * 8;           // Z (preconditioned vectors; FP32-valued velocities in mixed mode)
  b += n3 * 8 + 16;                // GCR / Anderson current direction, Anderson slot indices
  if (use_mgs(o, nx, ny)) b += 2 * n3 * 8;   // W^(1/2), W^(-1/2)
  if (o.cont_stages > 0) b += 2 * P * 8;   // full-contrast viscosity kept during continuation
  (void)L;
  const auto sz = sizes_of(nx, ny, o);
  b += mixed ? MG<float>::bytes(sz, o.kcycle, o.galerkin) : MG<double>::bytes(sz, o.kcycle, o.galerkin) - 2 * P * 8;
  if (o.schur) b += (mixed && o.schur == 1) ? SchurMG<float>::bytes(nx, ny, P) : SchurMG<double>::bytes(nx, ny, P);
  if (mixed && o.schur == 2) b += 4 * P * 8;   // FP64 middle-product planes
  if (o.inner_cg) b += InnerCG::bytes(P);
  b += 2 * (kMaxRestart + 2) * 8 + 2 * (size_t)kReduceBlocks * (kMaxRestart + 1) * 8 + 4 * kReduceBlocks * 8 +
       (size_t)kMaxRestart * kHcolStride * 8 + 64;
  return b;
}

}  // namespace

// ---- C ABI --------------------------------------------------------------------------------------
extern "C" {

void pyro_default_opts(pyro_opts* o) {
  if (!o) return;
  o->nu1 = 2; o->nu2 = 2;
  o->omega_v = 1.0;
  o->alpha_p = 1.0;
  o->restart_m = 30;
  o->max_iter = 500;
  o->prec = PYRO_PREC_MIXED;
  o->coarsest_min = 4;
  o->eta_coarsen = PYRO_ETA_ARITH;
  o->warm_start = 0;
  o->use_graphs = 1;
  o->timeout_s = 0.0;
  o->kcycle = 0;
  o->cluster_cells = 0;
  o->tile_fusion = 1;
  o->tile_sweeps = 2;
  o->tile_fusion64 = 0;
  o->accel = PYRO_ACCEL_FGMRES;
  o->aa_beta = 1.0;
  o->smoother = PYRO_SMOOTH_RBGS;
  o->ras_inner = 4;
  o->litho_guess = 0;
  o->cont_stages = 0;
  o->cont_iters = 25;
  o->coarse_sweeps = 40;
  o->coarsen_ratio = 2.0;
  o->coarsen_general = 1;
  o->gram_schmidt = 2;
  o->schur = 0;
  o->galerkin = 0;
  o->inner_cg = 0;
  o->res64 = 0;
}

const char* pyro_version(void) { return "pyro-b300 0.1 (sm_103a)"; }

const char* pyro_strerror(int s) {
  switch (s) {
    case PYRO_OK: return "ok";
    case PYRO_W_NOT_CONVERGED: return "not converged within max_iter (best iterate returned)";
    case PYRO_E_INVALID: return "invalid argument or unsupported grid / boundary";
    case PYRO_E_NOMEM: return "device allocation failed";
    case PYRO_E_CUDA: return "CUDA runtime error";
    case PYRO_E_NONFINITE: return "non-finite input or iterate";
    case PYRO_E_TIMEOUT: return "wall-clock limit exceeded";
    case PYRO_E_BREAKDOWN: return "Krylov or coarse-solve breakdown";
    default: return "unknown status";
  }
}

size_t pyro_stokes_footprint(int nx, int ny, const pyro_opts* opts) {
  pyro_opts o;
  pyro_default_opts(&o);
  if (opts) o = *opts;
  if (!opts_valid(o)) return 0;
  const int L = check_size(nx, ny, o);
  if (L < 1) return 0;
  return footprint_bytes(nx, ny, o, L);
}

int pyro_stokes_create(int nx, int ny, double Lx, double Ly, const pyro_bc* bc, const pyro_opts* opts,
                       pyro_stokes* out) {
  if (!out) return PYRO_E_INVALID;
  *out = nullptr;
  if (!(Lx > 0) || !(Ly > 0)) return PYRO_E_INVALID;
  std::lock_guard<std::recursive_mutex> lk(device_sync_lock());
  pyro_opts o;
  pyro_default_opts(&o);
  if (opts) o = *opts;
  if (!opts_valid(o)) return PYRO_E_INVALID;
  pyro_bc b{};
  for (int k = 0; k < 4; ++k) { b.kind[k] = PYRO_BC_FREE_SLIP; b.vt[k] = 0.0; }
  if (bc) b = *bc;
  for (int k = 0; k < 4; ++k) {
    if (b.kind[k] != PYRO_BC_FREE_SLIP && b.kind[k] != PYRO_BC_NO_SLIP && b.kind[k] != PYRO_BC_VELOCITY)
      return PYRO_E_INVALID;  // periodic: oracle only
    if (!std::isfinite(b.vt[k])) return PYRO_E_INVALID;
  }
  const int L = check_size(nx, ny, o);
  if (L < 1) return PYRO_E_INVALID;
  pyro_stokes_s* h = new (std::nothrow) pyro_stokes_s();
  if (!h) return PYRO_E_NOMEM;
  try {
    CK(cudaGetDevice(&h->dev));
    h->nx = nx; h->ny = ny; h->Lx = Lx; h->Ly = Ly; h->bc = b; h->o = o;
    h->g = make_geom(nx, ny, Lx, Ly, b);
    h->g64 = geomT<double>(h->g);
    h->P = (size_t)(ny + 2) * (nx + 2);
    h->n3 = 3 * h->P;
    h->nlev = L;
    h->mixed = o.prec == PYRO_PREC_MIXED;
    h->m = o.restart_m;
    h->dot_grid_y = (h->m + 1 + 7) / 8;
    DevAlloc& A = h->mem;
    h->en = A.get<double>(h->P); h->ec = A.get<double>(h->P); h->rho = A.get<double>(h->P);
    h->b = A.get<double>(h->n3); h->x = A.get<double>(h->n3); h->r = A.get<double>(h->n3);
    h->w = A.get<double>(h->n3); h->W = A.get<double>(h->n3); h->xf = A.get<double>(h->n3);
    h->stage = A.get<double>(h->n3);
    {
      double* k5 = A.get<double>(5 * h->P);
      h->okc = Coef<double>{k5, k5 + h->P, k5 + 2 * h->P, k5 + 3 * h->P, k5 + 4 * h->P};
    }
    h->V = A.get<double>((size_t)(h->m + 1) * h->n3);
    h->Z = A.get<double>((size_t)(h->m + 1) * h->n3);   // m for FGMRES / GCR, m + 1 for Anderson
    h->zc = A.get<double>(h->n3);
    if (o.cont_stages > 0) { h->en_full = A.get<double>(h->P); h->ec_full = A.get<double>(h->P); }
    h->d_slot = A.get<int>(2);
    h->d_cnt = h->d_slot + 1;
    h->h1 = A.get<double>(kMaxRestart + 2); h->h2 = A.get<double>(kMaxRestart + 2);
    h->partial = A.get<double>((size_t)kReduceBlocks * (kMaxRestart + 1) * 2);
    h->part2 = A.get<double>(4 * kReduceBlocks);
    h->hcol = A.get<double>((size_t)kMaxRestart * kHcolStride);
    h->inv = A.get<double>(1);
    h->ydev = A.get<double>(kMaxRestart + 2);
    h->d_j = A.get<int>(1);
    h->flag = A.get<int>(1);
    if (use_mgs(o, nx, ny)) {
      h->sw = A.get<double>(h->n3);
      h->isw = A.get<double>(h->n3);
    }
    if (h->mixed) {
      h->mgf.nu1 = o.nu1; h->mgf.nu2 = o.nu2; h->mgf.omega = (float)o.omega_v; h->mgf.eta_mode = o.eta_coarsen;
      h->mgf.coarse_sweeps = o.coarse_sweeps;
      h->mgf.kcycle = o.kcycle;
      h->mgf.smoother = o.smoother;
      h->mgf.ras_inner = o.ras_inner;
      if (o.smoother == PYRO_SMOOTH_RAS || o.smoother == PYRO_SMOOTH_MIXED) MG<float>::enable_ras();
      h->mgf.tiles = o.tile_fusion != 0;
      h->mgf.tile_form = o.tile_fusion == 4 ? 1 : 0;
      h->mgf.tile_sweeps = o.tile_sweeps;
      h->mgf.galerkin = o.galerkin;
      if (h->mgf.tiles) MG<float>::enable_tiles();
      CK(cudaDeviceSynchronize());
      h->mgf.alloc(A, h->g, Lx, Ly, sizes_of(nx, ny, o), false);
      h->mgf.res64 = o.res64 != 0;
      h->mgf.r64_g = h->g64;
      h->mgf.r64_kc = h->okc;
      if (o.schur == 1) h->smf.alloc(A, nx, ny, h->P);
      if (o.schur == 2) {
        h->smd.alloc(A, nx, ny, h->P);
        h->sc64 = A.get<double>(4 * h->P);
      }
      if (o.inner_cg) h->ic.alloc(A, h->P);
    } else {
      h->mgd.nu1 = o.nu1; h->mgd.nu2 = o.nu2; h->mgd.omega = o.omega_v; h->mgd.eta_mode = o.eta_coarsen;
      h->mgd.coarse_sweeps = o.coarse_sweeps;
      h->mgd.kcycle = o.kcycle;
      h->mgd.smoother = o.smoother;
      h->mgd.ras_inner = o.ras_inner;
      if (o.smoother == PYRO_SMOOTH_RAS || o.smoother == PYRO_SMOOTH_MIXED) MG<double>::enable_ras();
      h->mgd.tiles = o.tile_fusion64 != 0;
      h->mgd.galerkin = o.galerkin;
      if (h->mgd.tiles) MG<double>::enable_tiles();
      h->mgd.alloc(A, h->g, Lx, Ly, sizes_of(nx, ny, o), true);
      h->mgd.lv[0].en = h->en;
      h->mgd.lv[0].ec = h->ec;
      if (!h->mgd.fused(0)) h->mgd.lv[0].kc = h->okc;  // FP64 level 0 shares the outer coefficients
      if (o.schur) h->smd.alloc(A, nx, ny, h->P);
      if (o.inner_cg) h->ic.alloc(A, h->P);
    }
    CK(cudaMallocHost(&h->hbuf, 4 * kReduceBlocks * sizeof(double) + 1024));
    CK(cudaMallocHost(&h->hflag, sizeof(int)));
    for (int k = 0; k < 4; ++k) CK(cudaEventCreate(&h->ev[k]));
    for (int k = 0; k < 7; ++k) CK(cudaEventCreate(&h->tev[k]));
    CK(cudaMemset(h->x, 0, h->n3 * sizeof(double)));
    CK(cudaMemset(h->xf, 0, h->n3 * sizeof(double)));
    CK(cudaMemset(h->flag, 0, sizeof(int)));
    CK(cudaDeviceSynchronize());
  } catch (const std::bad_alloc&) {
    pyro_stokes_destroy(h);
    return PYRO_E_NOMEM;
  } catch (const CudaError&) {
    pyro_stokes_destroy(h);
    return PYRO_E_CUDA;
  }
  *out = h;
  return PYRO_OK;
}

int pyro_stokes_precond(pyro_stokes h, const double* eta_n, const double* eta_c, const double* r_vx,
                        const double* r_vy, const double* r_p, double* z_vx, double* z_vy, double* z_p,
                        void* cuda_stream) {
  if (!h || !eta_n || !eta_c || !r_vx || !r_vy || !r_p || !z_vx || !z_vy || !z_p) return PYRO_E_INVALID;
  if (cudaSetDevice(h->dev) != cudaSuccess) return PYRO_E_CUDA;
  if (!places_ok({eta_n, eta_c, r_vx, r_vy, r_p, z_vx, z_vy, z_p})) return PYRO_E_INVALID;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  try {
    CK(cudaSetDevice(h->dev));
    h->have_solution = false;
    CK(cudaMemsetAsync(h->flag, 0, sizeof(int), s));
    ingest(h, eta_n, h->en, 3, s);
    ingest(h, eta_c, h->ec, 2, s);
    ingest(h, r_vx, h->V, 4, s);
    ingest(h, r_vy, h->V + h->P, 5, s);
    ingest(h, r_p, h->V + 2 * h->P, 2, s);
    setup_eta(h, s);
    CK(cudaMemsetAsync(h->d_j, 0, sizeof(int), s));
    // the same preconditioner body the Krylov iteration runs (V-cycle, pressure block, mean removal)
    precond_any(h, s, h->V, h->n3, (double*)h->Z, h->n3, h->d_j, false);
    CK(cudaMemcpyAsync(h->w, h->Z, h->n3 * sizeof(double), cudaMemcpyDeviceToDevice, s));
    double* outs[3] = {z_vx, z_vy, z_p};
    for (int k = 0; k < 3; ++k)
      CK(cudaMemcpyAsync(outs[k], h->w + k * h->P, h->P * sizeof(double),
                         is_device_ptr(outs[k]) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(h->hflag, h->flag, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (*h->hflag & FLAG_NONFINITE) return PYRO_E_NONFINITE;
    if (*h->hflag & FLAG_BREAKDOWN) return PYRO_E_BREAKDOWN;
  } catch (const CudaError&) {
    return PYRO_E_CUDA;
  }
  return PYRO_OK;
}

int pyro_stokes_set_timing(pyro_stokes h, int enable) {
  if (!h) return PYRO_E_INVALID;
  h->timing = enable != 0;
  for (int k = 0; k < 6; ++k) h->tacc[k] = 0.0;
  h->tcount[0] = h->tcount[1] = 0;
  return PYRO_OK;
}

int pyro_stokes_get_timing(pyro_stokes h, double* ms, long long* counts) {
  if (!h) return PYRO_E_INVALID;
  if (ms)
    for (int k = 0; k < 6; ++k) ms[k] = h->tacc[k];
  if (counts) { counts[0] = h->tcount[0]; counts[1] = h->tcount[1]; }
  return PYRO_OK;
}

void pyro_stokes_destroy(pyro_stokes h) {
  if (!h) return;
  std::lock_guard<std::recursive_mutex> lk(device_sync_lock());
  cudaSetDevice(h->dev);
  for (auto g : h->graphs)
    if (g) cudaGraphExecDestroy(g);
  for (int k = 0; k < 4; ++k)
    if (h->ev[k]) cudaEventDestroy(h->ev[k]);
  for (int k = 0; k < 7; ++k)
    if (h->tev[k]) cudaEventDestroy(h->tev[k]);
  if (h->hbuf) cudaFreeHost(h->hbuf);
  if (h->hflag) cudaFreeHost(h->hflag);
  h->mem.release();
  delete h;
}

int pyro_stokes_apply(pyro_stokes h, const double* eta_n, const double* eta_c, const double* vx, const double* vy,
                      const double* p, double* Ax, double* Ay, double* Ap, void* cuda_stream) {
  if (!h || !eta_n || !eta_c || !vx || !vy || !p || !Ax || !Ay || !Ap) return PYRO_E_INVALID;
  if (cudaSetDevice(h->dev) != cudaSuccess) return PYRO_E_CUDA;
  if (!places_ok({eta_n, eta_c, vx, vy, p, Ax, Ay, Ap})) return PYRO_E_INVALID;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  try {
    CK(cudaSetDevice(h->dev));
    CK(cudaMemsetAsync(h->flag, 0, sizeof(int), s));
    ingest(h, eta_n, h->en, 3, s);
    ingest(h, eta_c, h->ec, 2, s);
    ingest(h, vx, h->r, 4, s);
    ingest(h, vy, h->r + h->P, 5, s);
    ingest(h, p, h->r + 2 * h->P, 2, s);
    outer_coefs(h, s);
    k_apply<double><<<grid2(h->nx, h->ny, kBlk2), kBlk2, 0, s>>>(h->g64, h->en, h->ec, h->r, 0, nullptr, h->w, h->okc);
    double* outs[3] = {Ax, Ay, Ap};
    for (int k = 0; k < 3; ++k) {
      if (is_device_ptr(outs[k])) CK(cudaMemcpyAsync(outs[k], h->w + k * h->P, h->P * sizeof(double), cudaMemcpyDeviceToDevice, s));
      else CK(cudaMemcpyAsync(outs[k], h->w + k * h->P, h->P * sizeof(double), cudaMemcpyDeviceToHost, s));
    }
    CK(cudaMemcpyAsync(h->hflag, h->flag, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (*h->hflag & FLAG_NONFINITE) return PYRO_E_NONFINITE;
  } catch (const CudaError&) {
    return PYRO_E_CUDA;
  }
  return PYRO_OK;
}

int pyro_stokes_solve(pyro_stokes h, const double* eta_n, const double* eta_c, const double* rho, double gx, double gy,
                      double tol, double* vx, double* vy, double* p, pyro_stats* stats, void* cuda_stream) {
  if (!h || !eta_n || !eta_c || !rho || !vx || !vy || !p) return PYRO_E_INVALID;
  if (!(tol > 0) || !std::isfinite(gx) || !std::isfinite(gy)) return PYRO_E_INVALID;
  if (cudaSetDevice(h->dev) != cudaSuccess) return PYRO_E_CUDA;
  if (!places_ok({eta_n, eta_c, rho, vx, vy, p})) return PYRO_E_INVALID;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  pyro_stats st{};
  st.levels = h->nlev;
  st.coarse_n = h->mixed ? h->mgf.nc : h->mgd.nc;
  int status = PYRO_OK;
  h->launches = 0;
  try {
    CK(cudaSetDevice(h->dev));
    h->have_solution = false;
    CK(cudaEventRecord(h->ev[0], s));
    CK(cudaMemsetAsync(h->flag, 0, sizeof(int), s));
    ingest(h, eta_n, h->en, 3, s);
    ingest(h, eta_c, h->ec, 2, s);
    ingest(h, rho, h->rho, 3, s);
    if (h->o.warm_start) {
      ingest(h, vx, h->x, 4, s);
      ingest(h, vy, h->x + h->P, 5, s);
      ingest(h, p, h->x + 2 * h->P, 2, s);
    } else {
      CK(cudaMemsetAsync(h->x, 0, h->n3 * sizeof(double), s));
    }
    CK(cudaMemcpyAsync(h->hflag, h->flag, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (*h->hflag & FLAG_NONFINITE) { status = PYRO_E_NONFINITE; }
    else {
      const pyro_bc& b = h->bc;
      auto cst = [&](int side) { return b.kind[side] == PYRO_BC_VELOCITY ? 2.0 * b.vt[side] : 0.0; };
      k_rhs<<<grid2(h->nx, h->ny, kBlk2), kBlk2, 0, s>>>(h->g64, h->en, h->rho, gx, gy, cst(2), cst(3), cst(0), cst(1), h->b);
      h->launches += 1;
      setup_eta(h, s);
      CK(cudaMemcpyAsync(h->hflag, h->flag, sizeof(int), cudaMemcpyDeviceToHost, s));
      CK(cudaEventRecord(h->ev[1], s));
      CK(cudaStreamSynchronize(s));
      float ms = 0;
      cudaEventElapsedTime(&ms, h->ev[0], h->ev[1]);
      st.t_setup_ms = ms;
      if (*h->hflag & FLAG_BREAKDOWN) status = PYRO_E_BREAKDOWN;
      else {
        if (h->o.litho_guess && !h->o.warm_start) {
          k_litho<<<(h->nx + 127) / 128, 128, 0, s>>>(h->g64, h->rho, gy, h->g.dy, h->x + 2 * h->P);
          k_psum<<<kReduceBlocks, kThreads, 0, s>>>(h->g64, h->x + 2 * h->P, h->part2);
          k_sub_mean<double><<<kReduceBlocks, kThreads, 0, s>>>(h->g64, h->x + 2 * h->P, 0, nullptr, h->part2,
                                                                kReduceBlocks);
          h->launches += 3;
        }
        status = h->o.cont_stages > 0 ? continuation_solve(h, tol, &st, s) : outer_solve(h, tol, &st, s);
      }
    }
    if (status >= 0) {
      CK(cudaMemcpyAsync(h->xf, h->x, h->n3 * sizeof(double), cudaMemcpyDeviceToDevice, s));
      emit(h, h->x, vx, vy, p, true, s);
      CK(cudaStreamSynchronize(s));
      h->have_solution = true;
      h->last_gx = gx; h->last_gy = gy;
    }
  } catch (const CudaError&) {
    status = PYRO_E_CUDA;
  }
  st.status = status;
  st.kernel_launches = h->launches;
  if (stats) *stats = st;
  return status;
}

int pyro_stokes_adjoint(pyro_stokes h, const double* dJ_dvx, const double* dJ_dvy, const double* dJ_dp, double tol,
                        double* dJ_deta_n, double* dJ_deta_c, double* dJ_drho, pyro_stats* stats, void* cuda_stream) {
  if (!h || !dJ_dvx || !dJ_dvy || !dJ_dp || !dJ_deta_n || !dJ_deta_c || !(tol > 0)) return PYRO_E_INVALID;
  if (!h->have_solution) return PYRO_E_INVALID;
  if (cudaSetDevice(h->dev) != cudaSuccess) return PYRO_E_CUDA;
  if (!places_ok({dJ_dvx, dJ_dvy, dJ_dp, dJ_deta_n, dJ_deta_c, dJ_drho})) return PYRO_E_INVALID;
  for (int k = 0; k < 4; ++k)
    if (h->bc.kind[k] == PYRO_BC_VELOCITY) return PYRO_E_INVALID;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  pyro_stats st{};
  st.levels = h->nlev;
  st.coarse_n = h->mixed ? h->mgf.nc : h->mgd.nc;
  int status = PYRO_OK;
  h->launches = 0;
  try {
    CK(cudaSetDevice(h->dev));
    CK(cudaMemsetAsync(h->flag, 0, sizeof(int), s));
    ingest(h, dJ_dvx, h->b, 4, s);
    ingest(h, dJ_dvy, h->b + h->P, 5, s);
    ingest(h, dJ_dp, h->b + 2 * h->P, 2, s);
    // the constant-pressure null space: only the zero-mean part of dJ/dp is solvable
    k_psum<<<kReduceBlocks, kThreads, 0, s>>>(h->g64, h->b + 2 * h->P, h->part2);
    k_sub_mean<double><<<kReduceBlocks, kThreads, 0, s>>>(h->g64, h->b + 2 * h->P, 0, nullptr, h->part2, kReduceBlocks);
    CK(cudaMemsetAsync(h->x, 0, h->n3 * sizeof(double), s));
    CK(cudaMemcpyAsync(h->hflag, h->flag, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (*h->hflag & FLAG_NONFINITE) status = PYRO_E_NONFINITE;
    else status = outer_solve(h, tol, &st, s);   // eta and the hierarchy of the last solve are still in place
    if (status >= 0) {
      // lambda is in h->x, the forward solution in h->xf
      double* on = dJ_deta_n; double* oc = dJ_deta_c; double* orh = dJ_drho;
      const bool dn = is_device_ptr(on), dc = is_device_ptr(oc), dr = orh && is_device_ptr(orh);
      double* tn = dn ? on : h->stage;
      double* tc = dc ? oc : h->stage + h->P;
      double* tr = orh ? (dr ? orh : h->stage + 2 * h->P) : nullptr;
      k_strain_product<<<grid2(h->nx, h->ny, kBlk2), kBlk2, 0, s>>>(h->g64, h->xf, h->x, tn, tc);
      if (tr) k_rho_grad<<<grid2(h->nx, h->ny, kBlk2), kBlk2, 0, s>>>(h->g64, h->x, h->last_gx, h->last_gy, tr);
      h->launches += tr ? 2 : 1;
      if (!dn) CK(cudaMemcpyAsync(on, tn, h->P * sizeof(double), cudaMemcpyDeviceToHost, s));
      if (!dc) CK(cudaMemcpyAsync(oc, tc, h->P * sizeof(double), cudaMemcpyDeviceToHost, s));
      if (tr && !dr) CK(cudaMemcpyAsync(orh, tr, h->P * sizeof(double), cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
    }
    // restore the forward solution as the handle's current iterate
    CK(cudaMemcpyAsync(h->x, h->xf, h->n3 * sizeof(double), cudaMemcpyDeviceToDevice, s));
    CK(cudaStreamSynchronize(s));
  } catch (const CudaError&) {
    status = PYRO_E_CUDA;
  }
  st.status = status;
  st.kernel_launches = h->launches;
  if (stats) *stats = st;
  return status;
}

}  // extern "C"
