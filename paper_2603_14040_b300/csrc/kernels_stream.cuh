// FP32 row-streaming red-black Gauss-Seidel: NS damped sweeps of the velocity block (Sec.
// "Smoothers", eq. sor_update; colour order vx-red, vx-black, vy-red, vy-black) in ONE pass over
// HBM, as a wavefront pipeline down the rows.
//
// The S = 4 NS half-sweeps are pipeline stages. Stage s works on row R0 + t - 2 s at step t, so it
// trails the stage before it by two rows. A half-sweep at row r reads rows r-1..r+1 only, which
// makes every read see exactly the values the per-colour kernels would see at that point:
//   * rows r-1..r+1 of the previous stage's field are final (that stage passed r+1 a step ago);
//   * the next stage is still at row r-2 or above, so nothing a stage reads is overwritten early.
// The stages of one step touch disjoint rows, so one barrier per step is enough.
//
// A CTA owns C = 64 NW columns (its strip of W = C - 2 S columns plus one halo column per stage on
// each side) and H rows (plus S halo rows above and below). Halo points are computed redundantly
// from the CTA's own copy; values outside the dependence cone of the owned points are never
// written back. The output goes to the other buffer of the level's iterate (ping-pong), so CTAs
// never read a neighbour's new values.
//
// Shared memory holds a ring of D rows of the six arrays (vx, vy, fx, fy, eta_n, eta_c), each row
// split into its even and odd columns: a half-sweep touches one column of every pair, so a warp
// reads 32 consecutive words (conflict-free), and column neighbours are fixed offsets. Rows are
// prefetched PF steps ahead with 4-byte cp.async into the split layout (a row of a padded
// (ny+2) x (nx+2) array starts on any 8-byte boundary, which excludes 16-byte and bulk/TMA
// copies; the split layout excludes multi-word copies anyway).
//
// HBM per pass: read 6 arrays, write 2 (32 B per cell in FP32) plus the halo re-reads.
#pragma once
#include "common.cuh"

namespace pyro {

constexpr int kStreamRing = 32;   // rows of the shared-memory ring (power of two)
constexpr int kStreamAhead = 8;   // rows prefetched ahead of the first stage

template <int NS, int NW>
struct StreamCfg {
  static constexpr int S = 4 * NS;             // half-sweep stages
  static constexpr int C = 64 * NW;            // columns held per row (strip + halo)
  static constexpr int HC = C / 2;             // one parity half of a row
  static constexpr int W = C - 2 * S;          // columns written back per strip
  static constexpr int THREADS = S * 32 * NW;  // one thread per column pair per stage
  static constexpr int D = kStreamRing, PF = kStreamAhead;
  // the slot a step loads must be free at that step and the one before it
  static_assert(D > PF + 2 * S, "ring too short for the pipeline");
  static_assert(W > 0 && W % 2 == 0, "strip width must be positive and even");
  static constexpr size_t smem_bytes() { return (size_t)6 * D * C * sizeof(float); }
};

__device__ __forceinline__ void cp_async4(float* dst, const float* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// Grid: x = strips of W columns, y = chunks of H rows. Block: StreamCfg::THREADS threads.
// Shared-memory word (array a, ring slot, parity half h, pair k) = a*D*C + slot*C + h*HC + k.
template <int NS, int NW>
__global__ void __launch_bounds__(StreamCfg<NS, NW>::THREADS, 2)
    k_rbgs_stream(GeomT<float> g, const float* __restrict__ vx, const float* __restrict__ vy,
                  float* __restrict__ ox, float* __restrict__ oy, const float* __restrict__ fx,
                  const float* __restrict__ fy, const float* __restrict__ en, const float* __restrict__ ec,
                  float omega, int H) {
  using K = StreamCfg<NS, NW>;
  constexpr int S = K::S, C = K::C, HC = K::HC, D = K::D, PF = K::PF, T = K::THREADS;
  constexpr int A = D * C;                            // words per array ring
  constexpr int NLD = (6 * C + T - 1) / T;            // row elements each thread copies
  extern __shared__ __align__(16) float sm[];

  const int tid = threadIdx.x;
  const int jl = blockIdx.x * K::W - S;              // global column of local column 0 (even)
  const int i0 = blockIdx.y * H;
  const int iend = min(i0 + H, g.ny + 2);             // owned rows [i0, iend)
  const int R0 = i0 - S, Rend = iend + S;             // streamed rows [R0, Rend)
  const int nsteps = (Rend - R0) + S - 1;

  // fixed copy assignments: element e = tid + k T of a row (array e / C, column e % C)
  const float* lsrc[NLD];
  int ldst[NLD];
  bool lok[NLD], lcol[NLD];
#pragma unroll
  for (int k = 0; k < NLD; ++k) {
    const int e = tid + k * T;
    const int a = e / C, c = e % C;
    const int gj = jl + c;
    lok[k] = e < 6 * C;
    lcol[k] = gj >= 0 && gj <= g.nx + 1;
    const float* base = a == 0 ? vx : a == 1 ? vy : a == 2 ? fx : a == 3 ? fy : a == 4 ? en : ec;
    lsrc[k] = base + (lcol[k] ? gj : 0);
    ldst[k] = a * A + (c & 1) * HC + (c >> 1);
  }
  auto load_row = [&](int q) {
    if (q >= Rend) return;
    const bool rin = q >= 0 && q <= g.ny + 1;
    const size_t roff = rin ? (size_t)q * g.ld : 0;
    const int so = ((q - R0) & (D - 1)) * C;
#pragma unroll
    for (int k = 0; k < NLD; ++k) {
      if (!lok[k]) continue;
      float* dst = sm + ldst[k] + so;
      if (rin && lcol[k]) cp_async4(dst, lsrc[k] + roff);
      else *dst = 0.f;
    }
  };

  const int s = tid / (32 * NW);          // stage of this thread
  const int q = tid - s * 32 * NW;        // column pair (2q, 2q+1)
  const int fld = (s >> 1) & 1, col = s & 1;
  const bool strip_int = jl >= 2 && jl + C - 1 <= g.nx - 2;
  float* const out = s == 0 ? ox : oy;

#pragma unroll 1
  for (int k = 0; k < PF; ++k) {
    load_row(R0 + k);
    cp_async_commit();
  }
#pragma unroll 1
  for (int t = 0; t < nsteps; ++t) {
    load_row(R0 + t + PF);
    cp_async_commit();
    cp_async_wait<PF - 1>();   // rows up to R0 + t + 1 have landed (this thread's copies)
    __syncthreads();           // ... and everybody's; the previous step is complete

    // write back the row the last stage finished in the previous step (owned columns, unknowns)
    if (s < 2) {
      const int k = R0 + t - 2 * (S - 1) - 1;
      if (k >= i0 && k < iend) {
        const int so = ((k - R0) & (D - 1)) * C + s * A;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int c = 2 * q + h;
          const int gj = jl + c;
          if (c < S || c >= S + K::W || gj > g.nx + 1) continue;
          const bool unk = s == 0 ? is_vx(g.nx, g.ny, k, gj) : is_vy(g.nx, g.ny, k, gj);
          if (unk) out[(size_t)k * g.ld + gj] = sm[so + h * HC + q];
        }
      }
    }

    const int r = R0 + t - 2 * s;
    if (r < R0 + 1 || r > Rend - 2 || r < 1 || r > g.ny) continue;
    const int p = (col + r) & 1;          // column parity of this colour on row r
    const int c = 2 * q + p;
    if (c < 1 || c > C - 2) continue;
    const int gi = r, gj = jl + c;
    const bool interior = strip_int && gi >= 2 && gi <= g.ny - 2;
    // word offsets of rows r-1, r, r+1 and of columns c (half p), c-1 and c+1 (half 1-p)
    const int bm = ((r - 1 - R0) & (D - 1)) * C, b0 = ((r - R0) & (D - 1)) * C, bp = ((r + 1 - R0) & (D - 1)) * C;
    const int ip = p * HC + q, iw = (1 - p) * HC + q - 1 + p, ie = (1 - p) * HC + q + p;
    const float* Xs = sm;
    const float* Ys = sm + A;
    const float* Ns = sm + 4 * A;
    const float* Es = sm + 5 * A;
    if (fld == 0) {
      if (!interior && !is_vx(g.nx, g.ny, gi, gj)) continue;
      const float vc = Xs[b0 + ip];
      const float eA = Es[b0 + ip], eB = Es[b0 + ie];
      const float e1 = Ns[bm + ip], e2 = Ns[b0 + ip];
      float vw = Xs[b0 + iw], ve = Xs[b0 + ie], vn = Xs[bm + ip], vs = Xs[bp + ip];
      float yA = Ys[bm + ip], yB = Ys[bm + ie], yC = Ys[b0 + ip], yD = Ys[b0 + ie];
      if (!interior) {
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
      if (!interior) {
        if (gi == 1) diag += g.sN * e1 * g.idy2;
        if (gi == g.ny) diag += g.sS * e2 * g.idy2;
      }
      const float Lv = (sxxE - sxxW) * g.idx2 + sxyS - sxyN;
      sm[b0 + ip] = vc + omega * __fdividef(sm[2 * A + b0 + ip] - Lv, diag);
    } else {
      if (!interior && !is_vy(g.nx, g.ny, gi, gj)) continue;
      const float vc = Ys[b0 + ip];
      const float eA = Es[b0 + ip], eB = Es[bp + ip];
      const float e1 = Ns[b0 + iw], e2 = Ns[b0 + ip];
      float vn = Ys[bm + ip], vs = Ys[bp + ip], vw = Ys[b0 + iw], ve = Ys[b0 + ie];
      float xA = Xs[b0 + iw], xB = Xs[bp + iw], xC = Xs[b0 + ip], xD = Xs[bp + ip];
      if (!interior) {
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
      if (!interior) {
        if (gj == 1) diag += g.sW * e1 * g.idx2;
        if (gj == g.nx) diag += g.sE * e2 * g.idx2;
      }
      const float Lv = (syyS - syyN) * g.idy2 + sxyE - sxyW;
      sm[A + b0 + ip] = vc + omega * __fdividef(sm[3 * A + b0 + ip] - Lv, diag);
    }
  }
  cp_async_wait<0>();
}

}  // namespace pyro
