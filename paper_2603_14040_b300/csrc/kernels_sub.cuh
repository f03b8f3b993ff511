// Small-level sub-cycle in one thread-block cluster.
//
// Below a size threshold the multigrid levels are too small to fill the GPU, and launching one
// kernel per step (sweep colour, residual, restriction, prolongation, K-cycle dot products) makes
// the cycle latency-bound. Here the whole cycle from level `ls` down to the coarsest — including
// the recursive Krylov (K-cycle) corrections and the FP64 coarse direct solve — runs inside ONE
// launch of one thread-block cluster (16 CTAs where the GPU can schedule a cluster that large,
// else 8; the size is read at run time). Steps are separated by cluster barriers (release/acquire
// at cluster scope, so global-memory writes of one CTA are visible to the others after the
// barrier). Levels with at most SubArgs::solo_points padded points are finished by CTA 0 alone
// with block barriers while the other CTAs wait at the next cluster barrier (FP32 arithmetic is
// cheap enough on one SM for 64^2 cells; FP64, at about 2 FMA per clock per SM, only for the
// tiniest levels).
//
// The arithmetic is the same per-point code as the one-kernel-per-step path (rbgs_point and
// vresid_point with the level's precomputed coefficients and inverse diagonal where it has them,
// restrict_point, prolong_point, lx_point/ly_point), and the coarse matvec sums in the same
// lane order as k_coarse_solve, so both paths produce bitwise-identical results for the same level
// sequence; only the dot-product partials of the K-cycle are grouped differently (fixed order in
// both).
#pragma once
#include <cooperative_groups.h>

#include "kernels_mg.cuh"

namespace pyro {

namespace cg = cooperative_groups;

constexpr int kSubClusterMax = 16;  // largest cluster tried (non-portable size); 8 is the fallback
constexpr int kSubThreads = 1024;
constexpr int kSubMaxLevels = 16;

template <typename T>
struct SubLevel {
  GeomT<T> gt;
  T *vx, *vy, *fx, *fy, *rx, *ry, *en, *ec;
  T *d1x, *d1y, *q1x, *q1y, *ex, *ey;
  T *idgx, *idgy;
  Coef<T> kc;
};

template <typename T>
struct SubArgs {
  SubLevel<T> L[kSubMaxLevels];
  int nlev, nu1, nu2, kcycle;
  T omega;
  Geom gc;            // coarsest geometry (unknown numbering of the direct solve)
  const double* Ainv;  // (-L_coarsest)^-1
  int nc;
  double* red;        // cross-CTA reduction slots: 2 banks x kSubClusterMax x 4
  int solo_points;    // levels with at most this many padded points run on CTA 0 alone
};

template <typename T>
struct SubCtx {
  const SubArgs<T>* a;
  int tid, nthr, rank, bank, ncta;
  bool solo;
  double* sh;   // 32 doubles of shared memory
  double* shv;  // broadcast slots (4 doubles)
  double* fv;   // shared copy of the coarse right-hand side (nc doubles)
};

__device__ inline double sub_block_sum(double v, double* sh) {
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

// Cluster-wide thread index: consecutive warps of work go to different CTAs (warp w of CTA r is
// global warp w * ncta + r), so a small level's points spread over every SM of the cluster
// instead of filling the first CTAs, while each warp still touches 32 consecutive points.
__device__ inline int sub_tid(int rank, int ncta) {
  return ((int)(threadIdx.x >> 5) * ncta + rank) * 32 + (int)(threadIdx.x & 31);
}

template <typename T>
__device__ inline void sub_sync(SubCtx<T>& c) {
  if (c.solo) __syncthreads();
  else cg::this_cluster().sync();
}

// fixed-order reduction of NV values over the cluster (or the block in solo mode); every thread
// receives the totals
template <typename T, int NV>
__device__ inline void sub_reduce(SubCtx<T>& c, double (&v)[NV]) {
  for (int k = 0; k < NV; ++k) v[k] = sub_block_sum(v[k], c.sh);
  if (c.solo) {
    if (threadIdx.x == 0)
      for (int k = 0; k < NV; ++k) c.shv[k] = v[k];
    __syncthreads();
    for (int k = 0; k < NV; ++k) v[k] = c.shv[k];
    __syncthreads();
    return;
  }
  double* slot = c.a->red + ((size_t)c.bank * kSubClusterMax) * 4;
  if (threadIdx.x == 0)
    for (int k = 0; k < NV; ++k) slot[c.rank * 4 + k] = v[k];
  cg::this_cluster().sync();
  for (int k = 0; k < NV; ++k) {
    double s = 0.0;
    for (int r = 0; r < c.ncta; ++r) s += ((volatile double*)slot)[r * 4 + k];
    v[k] = s;
  }
  c.bank ^= 1;
}

template <typename T>
__device__ void sub_sweep(SubCtx<T>& c, const SubLevel<T>& L, T omega) {
  const GeomT<T>& g = L.gt;
  const int hw = (g.nx + 2) / 2 + 1;
  const int total = (g.ny + 2) * hw;
  for (int f = 0; f < 2; ++f)
    for (int col = 0; col < 2; ++col) {
      for (int e = c.tid; e < total; e += c.nthr) {
        const int i = e / hw, jh = e % hw;
        const int j = 2 * jh + ((i + col) & 1);
        if (j <= g.nx + 1)
          rbgs_point<T>(g, i, j, f, omega, L.vx, L.vy, L.fx, L.fy, L.en, L.ec, L.idgx, L.idgy, L.kc);
      }
      sub_sync(c);
    }
}

template <typename T>
__device__ void sub_coarse_solve(SubCtx<T>& c) {
  const SubArgs<T>& a = *c.a;
  const SubLevel<T>& L = a.L[a.nlev - 1];
  const int nx = a.gc.nx, ny = a.gc.ny, ld = a.gc.ld, nvx = ny * (nx - 1), n = a.nc;
  for (int k = threadIdx.x; k < n; k += blockDim.x) {  // every CTA gathers the whole RHS
    if (k < nvx) { const int i = k / (nx - 1) + 1, j = k % (nx - 1) + 1; c.fv[k] = (double)L.fx[(size_t)i * ld + j]; }
    else { const int kk = k - nvx; const int i = kk / nx + 1, j = kk % nx + 1; c.fv[k] = (double)L.fy[(size_t)i * ld + j]; }
  }
  __syncthreads();
  // one warp per row, lane-strided products and the xor-shuffle tree of k_coarse_solve
  const int lane = threadIdx.x & 31;
  for (int k = c.tid >> 5; k < n; k += c.nthr >> 5) {
    double s = 0.0;
    const double* row = a.Ainv + (size_t)k * n;
    for (int l = lane; l < n; l += 32) s += row[l] * c.fv[l];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane != 0) continue;
    if (k < nvx) { const int i = k / (nx - 1) + 1, j = k % (nx - 1) + 1; L.vx[(size_t)i * ld + j] = (T)(-s); }
    else { const int kk = k - nvx; const int i = kk / nx + 1, j = kk % nx + 1; L.vy[(size_t)i * ld + j] = (T)(-s); }
  }
  sub_sync(c);
}

// K-cycle step 1 on level m after the first inner cycle (z1 in x): d1 = z1, q1 = L d1,
// s1 = [rc.d1, d1.q1], then e = a1 d1, rc -= a1 q1 (rc lives in f), x = 0.
template <typename T>
__device__ void sub_kstep1(SubCtx<T>& c, int m, double* s1out) {
  const SubLevel<T>& C = c.a->L[m];
  const GeomT<T>& g = C.gt;
  const int P = (g.ny + 2) * g.ld, cols = g.nx + 2;
  double s1[2] = {0.0, 0.0};
  for (int e = c.tid; e < P; e += c.nthr) {
    const int i = e / cols, j = e % cols;
    T d, qx = T(0), qy = T(0), zx = T(0), zy = T(0);
    if (is_vx(g.nx, g.ny, i, j)) { zx = C.vx[e]; qx = lx_point<T>(g, i, j, C.vx, C.vy, C.en, C.ec, d); }
    if (is_vy(g.nx, g.ny, i, j)) { zy = C.vy[e]; qy = ly_point<T>(g, i, j, C.vx, C.vy, C.en, C.ec, d); }
    C.d1x[e] = zx; C.d1y[e] = zy; C.q1x[e] = qx; C.q1y[e] = qy;
    s1[0] += (double)C.fx[e] * zx + (double)C.fy[e] * zy;
    s1[1] += (double)zx * qx + (double)zy * qy;
  }
  sub_reduce(c, s1);  // its barrier also orders the writes above before the update below
  const T a1 = (s1[1] != 0.0 && isfinite(s1[1])) ? (T)(s1[0] / s1[1]) : T(0);
  for (int e = c.tid; e < P; e += c.nthr) {
    C.ex[e] = a1 * C.d1x[e];
    C.ey[e] = a1 * C.d1y[e];
    C.fx[e] -= a1 * C.q1x[e];
    C.fy[e] -= a1 * C.q1y[e];
    C.vx[e] = T(0);
    C.vy[e] = T(0);
  }
  sub_sync(c);
  s1out[0] = s1[0];
  s1out[1] = s1[1];
}

// K-cycle step 2 on level m after the second inner cycle (z2 in x): x = e + a2 (z2 - beta d1)
template <typename T>
__device__ void sub_kstep2(SubCtx<T>& c, int m, double dq) {
  const SubLevel<T>& C = c.a->L[m];
  const GeomT<T>& g = C.gt;
  const int P = (g.ny + 2) * g.ld, cols = g.nx + 2;
  double s2[3] = {0.0, 0.0, 0.0};
  for (int e = c.tid; e < P; e += c.nthr) {
    const int i = e / cols, j = e % cols;
    T d;
    if (is_vx(g.nx, g.ny, i, j)) {
      const T z = C.vx[e], Lz = lx_point<T>(g, i, j, C.vx, C.vy, C.en, C.ec, d);
      s2[0] += (double)z * C.q1x[e]; s2[1] += (double)z * Lz; s2[2] += (double)C.fx[e] * z;
    }
    if (is_vy(g.nx, g.ny, i, j)) {
      const T z = C.vy[e], Lz = ly_point<T>(g, i, j, C.vx, C.vy, C.en, C.ec, d);
      s2[0] += (double)z * C.q1y[e]; s2[1] += (double)z * Lz; s2[2] += (double)C.fy[e] * z;
    }
  }
  sub_reduce(c, s2);
  const double beta = (dq != 0.0 && isfinite(dq)) ? s2[0] / dq : 0.0;
  const double den = s2[1] - 2.0 * beta * s2[0] + beta * beta * dq;
  const double a2 = (den != 0.0 && isfinite(den)) ? s2[2] / den : 0.0;
  const T A2 = (T)a2, B = (T)beta;
  for (int e = c.tid; e < P; e += c.nthr) {
    C.vx[e] = C.ex[e] + A2 * (C.vx[e] - B * C.d1x[e]);
    C.vy[e] = C.ey[e] + A2 * (C.vy[e] - B * C.d1y[e]);
  }
  sub_sync(c);
}

// pre-smoothing, residual and restriction (with the coarse iterate zeroed) on level l
template <typename T>
__device__ void sub_down(SubCtx<T>& c, int l) {
  const SubArgs<T>& a = *c.a;
  const SubLevel<T>& L = a.L[l];
  const SubLevel<T>& C = a.L[l + 1];
  for (int k = 0; k < a.nu1; ++k) sub_sweep(c, L, a.omega);
  const GeomT<T>& g = L.gt;
  const int total = (g.ny + 2) * (g.nx + 2);
  for (int e = c.tid; e < total; e += c.nthr)
    vresid_point<T>(g, e / (g.nx + 2), e % (g.nx + 2), L.vx, L.vy, L.fx, L.fy, L.en, L.ec, L.rx, L.ry, L.kc);
  sub_sync(c);
  const GeomT<T>& gc = C.gt;
  const int tc = (gc.ny + 2) * (gc.nx + 2);
  for (int e = c.tid; e < tc; e += c.nthr) {
    restrict_point<T>(g, gc, e / (gc.nx + 2), e % (gc.nx + 2), L.rx, L.ry, C.fx, C.fy);
    C.vx[e] = T(0);
    C.vy[e] = T(0);
  }
  sub_sync(c);
}

// prolongation + correction and post-smoothing on level l
template <typename T>
__device__ void sub_up(SubCtx<T>& c, int l) {
  const SubArgs<T>& a = *c.a;
  const SubLevel<T>& L = a.L[l];
  const SubLevel<T>& C = a.L[l + 1];
  const GeomT<T>& g = L.gt;
  const int total = (g.ny + 2) * (g.nx + 2);
  for (int e = c.tid; e < total; e += c.nthr)
    prolong_point<T>(g, C.gt, e / (g.nx + 2), e % (g.nx + 2), L.vx, L.vy, C.vx, C.vy);
  sub_sync(c);
  for (int k = 0; k < a.nu2; ++k) sub_sweep(c, L, a.omega);
}

// The cycle from level ls as an explicit-stack state machine (no device recursion, so the
// stack use is fixed). Frames: CYCLE(l) {ENTER, POST} and KCORR(m) {START, MID, END}; every
// thread of the cluster walks the same sequence of frames.
enum : int { F_CYCLE = 0, F_KCORR = 1 };
enum : int { S_ENTER = 0, S_POST = 1, S_START = 0, S_MID = 1, S_END = 2 };

template <typename T>
__device__ void sub_run(SubCtx<T>& c, int ls) {
  const SubArgs<T>& a = *c.a;
  int lev[2 * kSubMaxLevels + 2], kind[2 * kSubMaxLevels + 2], st[2 * kSubMaxLevels + 2];
  double dq[2 * kSubMaxLevels + 2];
  int sp = 0, solo_sp = -1;
  lev[0] = ls; kind[0] = F_CYCLE; st[0] = S_ENTER; sp = 1;
  while (sp > 0) {
    const int t = sp - 1;
    const int l = lev[t];
    bool pop = false;
    if (kind[t] == F_CYCLE) {
      if (st[t] == S_ENTER) {
        if (l == a.nlev - 1) {
          sub_coarse_solve(c);
          pop = true;
        } else if (!c.solo && (a.L[l].gt.ny + 2) * a.L[l].gt.ld <= a.solo_points) {
          // tiny level: CTA 0 finishes this subtree alone, the others wait for it
          if (c.rank == 0) {
            c.solo = true;
            c.tid = threadIdx.x;
            c.nthr = blockDim.x;
            solo_sp = t;
            sub_down(c, l);
            st[t] = S_POST;
            if (l < a.kcycle && l + 1 < a.nlev - 1) { lev[sp] = l + 1; kind[sp] = F_KCORR; st[sp] = S_START; }
            else { lev[sp] = l + 1; kind[sp] = F_CYCLE; st[sp] = S_ENTER; }
            ++sp;
          } else {
            cg::this_cluster().sync();
            pop = true;
          }
        } else {
          sub_down(c, l);
          st[t] = S_POST;
          if (l < a.kcycle && l + 1 < a.nlev - 1) { lev[sp] = l + 1; kind[sp] = F_KCORR; st[sp] = S_START; }
          else { lev[sp] = l + 1; kind[sp] = F_CYCLE; st[sp] = S_ENTER; }
          ++sp;
        }
      } else {
        sub_up(c, l);
        pop = true;
      }
    } else {  // F_KCORR on level l: two inner cycles of level l with CG steps between
      if (st[t] == S_START) {
        st[t] = S_MID;
        lev[sp] = l; kind[sp] = F_CYCLE; st[sp] = S_ENTER; ++sp;
      } else if (st[t] == S_MID) {
        double s1[2];
        sub_kstep1(c, l, s1);
        dq[t] = s1[1];
        st[t] = S_END;
        lev[sp] = l; kind[sp] = F_CYCLE; st[sp] = S_ENTER; ++sp;
      } else {
        sub_kstep2(c, l, dq[t]);
        pop = true;
      }
    }
    if (pop) {
      --sp;
      if (c.solo && sp == solo_sp) {  // subtree run by CTA 0 alone is complete: rejoin
        c.solo = false;
        c.tid = sub_tid(c.rank, c.ncta);
        c.nthr = c.ncta * blockDim.x;
        solo_sp = -1;
        cg::this_cluster().sync();
      }
    }
  }
}

// The cycle from level ls (x_ls must be zero, f_ls set) down to the coarsest, in one cluster.
// Launch: one cluster of gridDim.x CTAs (cluster dimension = grid dimension, at most
// kSubClusterMax) of kSubThreads threads.
template <typename T>
__global__ void __launch_bounds__(kSubThreads, 1) k_subcycle(const __grid_constant__ SubArgs<T> a, int ls) {
  __shared__ double sh[32];
  __shared__ double shv[4];
  __shared__ double fv[1024];
  SubCtx<T> c;
  c.a = &a;
  c.rank = (int)cg::this_cluster().block_rank();
  c.ncta = (int)cg::this_cluster().num_blocks();
  c.tid = sub_tid(c.rank, c.ncta);
  c.nthr = c.ncta * blockDim.x;
  c.bank = 0;
  c.solo = false;
  c.sh = sh;
  c.shv = shv;
  c.fv = fv;
  sub_run(c, ls);
}

}  // namespace pyro
