// FP64 kernels of the outer solve: the fused Stokes operator (eq. stokes_saddle), its residual
// with the energy-norm partial sums (Sec. "Global Relative Energy Residual"), the right-hand
// side, the Krylov building blocks (deterministic multi-dot / multi-axpy for classical
// Gram-Schmidt with one re-orthogonalisation), the Uzawa pressure block of the preconditioner
// (Sec. "Uzawa Iteration as a Fixed Point Method") and the adjoint strain-rate product.
//
// Vectors of the full system are flat arrays of 3 padded planes [vx | vy | p], each
// (ny+2) x (nx+2); entries that are not unknowns are kept at zero so that flat dot products over
// the whole array (weighted by W, which is zero there too) equal sums over unknowns.
//
// Every reduction writes one partial per block and is finished by a fixed-order sum over a fixed
// number of blocks, so results are bitwise reproducible run to run.
#pragma once
#include "common.cuh"

namespace pyro {

__device__ inline double block_sum(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s += sh[k];
  return s;  // valid in thread 0
}

// Stokes rows at padded point (i, j); x planes may be float (stored preconditioned vectors).
template <typename TV>
__device__ inline void stokes_point(const GeomT<double>& g, int i, int j, const double* en, const double* ec,
                                    const TV* xv, const TV* yv, const TV* pv, double& ox, double& oy,
                                    double& op, const Coef<double>& kc = Coef<double>{}) {
  const size_t c = (size_t)i * g.ld + j;
  double d;
  ox = oy = op = 0.0;
  if (is_vx(g.nx, g.ny, i, j))
    ox = (kc.cxx ? lx_coef<double>(g, i, j, xv, yv, kc) : lx_point<double>(g, i, j, xv, yv, en, ec, d)) -
         ((double)pv[c + 1] - (double)pv[c]) * g.idx;
  if (is_vy(g.nx, g.ny, i, j))
    oy = (kc.cxx ? ly_coef<double>(g, i, j, xv, yv, kc) : ly_point<double>(g, i, j, xv, yv, en, ec, d)) -
         ((double)pv[c + g.ld] - (double)pv[c]) * g.idy;
  if (is_p(g.nx, g.ny, i, j))
    op = (ldvx<double>(xv, g.ld, g.nx, i, j) - ldvx<double>(xv, g.ld, g.nx, i, j - 1)) * g.idx +
         (ldvy<double>(yv, g.ld, g.ny, i, j) - ldvy<double>(yv, g.ld, g.ny, i - 1, j)) * g.idy;
}

// The three Stokes rows at an interior point (2 <= i <= ny-2, 2 <= j <= nx-2) with precomputed
// coefficients: every neighbour is an unknown, so the masks of lx_coef / ly_coef / the
// divergence drop out (same arithmetic as stokes_point).
template <typename TV>
__device__ inline void stokes_point_interior(const GeomT<double>& g, size_t c, const TV* xv, const TV* yv,
                                             const TV* pv, const Coef<double>& k, double& ox, double& oy,
                                             double& op) {
  const int ld = g.ld;
  {
    const double vc = xv[c], vw = xv[c - 1], ve = xv[c + 1], vn = xv[c - ld], vs = xv[c + ld];
    const double yA = yv[c - ld], yB = yv[c - ld + 1], yC = yv[c], yD = yv[c + 1];
    ox = (k.cxx[c + 1] * (ve - vc) - k.cxx[c] * (vc - vw) + k.nyy[c] * (vs - vc) + k.nxy[c] * (yD - yC) -
          k.nyy[c - ld] * (vc - vn) - k.nxy[c - ld] * (yB - yA)) -
         ((double)pv[c + 1] - (double)pv[c]) * g.idx;
  }
  {
    const double vc = yv[c], vn = yv[c - ld], vs = yv[c + ld], vw = yv[c - 1], ve = yv[c + 1];
    const double xA = xv[c - 1], xB = xv[c + ld - 1], xC = xv[c], xD = xv[c + ld];
    oy = (k.cyy[c + ld] * (vs - vc) - k.cyy[c] * (vc - vn) + k.nxx[c] * (ve - vc) + k.nxy[c] * (xD - xC) -
          k.nxx[c - 1] * (vc - vw) - k.nxy[c - 1] * (xB - xA)) -
         ((double)pv[c + ld] - (double)pv[c]) * g.idy;
  }
  op = ((double)xv[c] - (double)xv[c - 1]) * g.idx + ((double)yv[c] - (double)yv[c - ld]) * g.idy;
}

// y = A x_k, x_k = X + (*d_k) * stride (d_k may be null: k = 0)
template <typename TV>
__global__ void k_apply(GeomT<double> g, const double* __restrict__ en, const double* __restrict__ ec,
                        const TV* __restrict__ X, size_t stride, const int* __restrict__ d_k,
                        double* __restrict__ y, Coef<double> kc) {
  const int i = blockIdx.y * blockDim.y + threadIdx.y;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (i > g.ny + 1 || j > g.nx + 1) return;
  const size_t P = (size_t)(g.ny + 2) * g.ld;
  const TV* x = X + (d_k ? (size_t)(*d_k) * stride : 0);
  double ox, oy, op;
  const size_t c = (size_t)i * g.ld + j;
  if (kc.cxx && i >= 2 && i <= g.ny - 2 && j >= 2 && j <= g.nx - 2)
    stokes_point_interior<TV>(g, c, x, x + P, x + 2 * P, kc, ox, oy, op);
  else
    stokes_point<TV>(g, i, j, en, ec, x, x + P, x + 2 * P, ox, oy, op, kc);
  y[c] = ox;
  y[P + c] = oy;
  y[2 * P + c] = op;
}

// r = b - A x; per-block partial sums of sum(W r^2) and sum(r^2) into part[2*blockId + {0,1}]
__global__ void k_residual(GeomT<double> g, const double* __restrict__ en, const double* __restrict__ ec,
                           const double* __restrict__ b, const double* __restrict__ x,
                           double* __restrict__ r, const double* __restrict__ W, double* __restrict__ part,
                           Coef<double> kc) {
  __shared__ double sh[32];
  const size_t P = (size_t)(g.ny + 2) * g.ld;
  const int rows = g.ny + 2, cols = g.nx + 2;
  double sw = 0.0, s2 = 0.0;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < P; e += (size_t)gridDim.x * blockDim.x) {
    int i, j;
    row_col(e, cols, i, j);
    if (i >= rows) break;
    double ox, oy, op;
    stokes_point<double>(g, i, j, en, ec, x, x + P, x + 2 * P, ox, oy, op, kc);
    const double rx = is_vx(g.nx, g.ny, i, j) ? b[e] - ox : 0.0;
    const double ry = is_vy(g.nx, g.ny, i, j) ? b[P + e] - oy : 0.0;
    const double rp = is_p(g.nx, g.ny, i, j) ? b[2 * P + e] - op : 0.0;
    r[e] = rx; r[P + e] = ry; r[2 * P + e] = rp;
    sw += W[e] * rx * rx + W[P + e] * ry * ry + W[2 * P + e] * rp * rp;
    s2 += rx * rx + ry * ry + rp * rp;
  }
  const double a = block_sum(sw, sh);
  const double c2 = block_sum(s2, sh);
  if (threadIdx.x == 0) { part[2 * blockIdx.x] = a; part[2 * blockIdx.x + 1] = c2; }
}

// Energy weights: W = 1/diag(-L) at velocity unknowns, eta_c/(2/dx^2+2/dy^2) at cells, else 0.
__global__ void k_weights(GeomT<double> g, const double* __restrict__ en, const double* __restrict__ ec,
                          double* __restrict__ W) {
  const int i = blockIdx.y * blockDim.y + threadIdx.y;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (i > g.ny + 1 || j > g.nx + 1) return;
  const size_t P = (size_t)(g.ny + 2) * g.ld, c = (size_t)i * g.ld + j;
  double wx = 0.0, wy = 0.0, wp = 0.0;
  if (is_vx(g.nx, g.ny, i, j)) {
    double d = -2.0 * (ec[c] + ec[c + 1]) * g.idx2 - (en[c - g.ld] + en[c]) * g.idy2;
    if (i == 1) d += g.sN * en[c - g.ld] * g.idy2;
    if (i == g.ny) d += g.sS * en[c] * g.idy2;
    wx = -1.0 / d;
  }
  if (is_vy(g.nx, g.ny, i, j)) {
    double d = -2.0 * (ec[c] + ec[c + g.ld]) * g.idy2 - (en[c - 1] + en[c]) * g.idx2;
    if (j == 1) d += g.sW * en[c - 1] * g.idx2;
    if (j == g.nx) d += g.sE * en[c] * g.idx2;
    wy = -1.0 / d;
  }
  if (is_p(g.nx, g.ny, i, j)) wp = ec[c] / (2.0 * g.idx2 + 2.0 * g.idy2);
  W[c] = wx; W[P + c] = wy; W[2 * P + c] = wp;
}

// Right-hand side: f = -rho g averaged onto velocity nodes, plus the constants of eliminated
// prescribed-velocity ghosts (ghost = -interior + 2U moves -coef * 2U to the RHS).
__global__ void k_rhs(GeomT<double> g, const double* __restrict__ en, const double* __restrict__ rho,
                      double gx, double gy, double cN, double cS, double cW, double cE, double* __restrict__ b) {
  const int i = blockIdx.y * blockDim.y + threadIdx.y;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (i > g.ny + 1 || j > g.nx + 1) return;
  const size_t P = (size_t)(g.ny + 2) * g.ld, c = (size_t)i * g.ld + j;
  double bx = 0.0, by = 0.0;
  if (is_vx(g.nx, g.ny, i, j)) {
    bx = -gx * 0.5 * (rho[c - g.ld] + rho[c]);
    if (i == 1) bx -= en[c - g.ld] * g.idy2 * cN;
    if (i == g.ny) bx -= en[c] * g.idy2 * cS;
  }
  if (is_vy(g.nx, g.ny, i, j)) {
    by = -gy * 0.5 * (rho[c - 1] + rho[c]);
    if (j == 1) by -= en[c - 1] * g.idx2 * cW;
    if (j == g.nx) by -= en[c] * g.idx2 * cE;
  }
  b[c] = bx; b[P + c] = by; b[2 * P + c] = 0.0;
}

// Copy a caller field into internal storage keeping only its meaningful entries (kind: 0 vx,
// 1 vy, 2 cell (p / eta_c), 3 node (eta_n / rho), 4 vx unknowns, 5 vy unknowns); others are
// zeroed. Non-finite meaningful entries raise FLAG_NONFINITE.
__global__ void k_ingest(int nx, int ny, int ld, const double* __restrict__ src, double* __restrict__ dst,
                         int kind, int* __restrict__ flag) {
  const int i = blockIdx.y * blockDim.y + threadIdx.y;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (i > ny + 1 || j > nx + 1) return;
  bool m;
  switch (kind) {
    case 0: m = i >= 1 && i <= ny && j <= nx; break;
    case 1: m = i <= ny && j >= 1 && j <= nx; break;
    case 2: m = is_p(nx, ny, i, j); break;
    case 3: m = i <= ny && j <= nx; break;
    case 4: m = is_vx(nx, ny, i, j); break;
    default: m = is_vy(nx, ny, i, j); break;
  }
  const size_t c = (size_t)i * ld + j;
  double v = m ? src[c] : 0.0;
  if (m && !isfinite(v)) { atomicOr(flag, FLAG_NONFINITE); v = 0.0; }
  dst[c] = v;
}

// per-block partial sums of v^2 (plain l2 norm)
__global__ void k_sumsq(const double* __restrict__ v, size_t n, double* __restrict__ part) {
  __shared__ double sh[32];
  double acc = 0.0;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
    acc += v[e] * v[e];
  const double s = block_sum(acc, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

__global__ void k_to_double(const float* __restrict__ a, double* __restrict__ b, size_t n) {
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
    b[e] = (double)a[e];
}

__global__ void k_to_float(const double* __restrict__ a, float* __restrict__ b, size_t n) {
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
    b[e] = (float)a[e];
}

// ---- Krylov building blocks -------------------------------------------------------------------
// partial[k * gridDim.x + blockIdx.x] = sum_e W[e] w[e] V_k[e] for k in [k0, k0+8) and k < nvec,
// nvec = *d_j + 1 (or nfix when d_j is null). blockIdx.y selects the group of 8 vectors.
template <bool WEIGHTED>
__global__ void k_multidot(const double* __restrict__ V, size_t stride, const int* __restrict__ d_j, int nfix,
                           const double* __restrict__ w, const double* __restrict__ W, size_t n,
                           double* __restrict__ partial, int off = 0) {
  __shared__ double sh[32];
  const int nvec = d_j ? (*d_j + 1 + off) : nfix;
  const int k0 = blockIdx.y * 8;
  if (k0 >= nvec) return;
  const int kn = min(8, nvec - k0);
  double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    const double t = WEIGHTED ? W[e] * w[e] : w[e];
#pragma unroll
    for (int q = 0; q < 8; ++q)
      if (q < kn) acc[q] += t * V[(size_t)(k0 + q) * stride + e];
  }
  for (int q = 0; q < kn; ++q) {
    const double s = block_sum(acc[q], sh);
    if (threadIdx.x == 0) partial[(size_t)(k0 + q) * gridDim.x + blockIdx.x] = s;
  }
}

// The same partial sums as k_multidot<WEIGHTED> for nvec <= kDotRegs, in a single pass over w and
// W: each thread keeps one accumulator per vector in registers. The code path is chosen from nvec
// in steps of 4 (the FP64 pipe, not memory, bounds these passes, so a path sized to the vector
// count avoids issuing FMAs for absent vectors). Launch kDotBlocks blocks of kThreads threads:
// two resident blocks per SM (up to 128 registers a thread) make one full wave on 148 SMs; block b
// writes partial[k * gridDim.x + b].
constexpr int kDotRegs = 32;
constexpr int kDotBlocks = 2 * 148;

template <int G, bool WEIGHTED>
__device__ __forceinline__ void multidot_regs(const double* __restrict__ V, size_t stride, int nvec,
                                              const double* __restrict__ w, const double* __restrict__ W, size_t n,
                                              double* __restrict__ partial, double (*red)[kThreads / 32]) {
  double acc[G];
#pragma unroll
  for (int q = 0; q < G; ++q) acc[q] = 0.0;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    const double t = WEIGHTED ? W[e] * w[e] : w[e];
#pragma unroll
    for (int q = 0; q < G; ++q)
      if (q < G - 4 || q < nvec) acc[q] += t * V[(size_t)q * stride + e];
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < G; ++q) {
    if (q >= G - 4 && q >= nvec) continue;
    double v = acc[q];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) red[q][wid] = v;
  }
  __syncthreads();
  if ((int)threadIdx.x < nvec) {
    double s = 0.0;
    for (int k = 0; k < kThreads / 32; ++k) s += red[threadIdx.x][k];
    partial[(size_t)threadIdx.x * gridDim.x + blockIdx.x] = s;
  }
}

template <bool WEIGHTED>
__global__ void __launch_bounds__(kThreads, 2) k_multidot_r(const double* __restrict__ V, size_t stride,
                                                         const int* __restrict__ d_j, const double* __restrict__ w,
                                                         const double* __restrict__ W, size_t n,
                                                         double* __restrict__ partial, int off) {
  __shared__ double red[kDotRegs][kThreads / 32];
  const int nvec = *d_j + 1 + off;
  if (nvec <= 0 || nvec > kDotRegs) return;
  switch ((nvec + 3) >> 2) {
    case 1: multidot_regs<4, WEIGHTED>(V, stride, nvec, w, W, n, partial, red); break;
    case 2: multidot_regs<8, WEIGHTED>(V, stride, nvec, w, W, n, partial, red); break;
    case 3: multidot_regs<12, WEIGHTED>(V, stride, nvec, w, W, n, partial, red); break;
    case 4: multidot_regs<16, WEIGHTED>(V, stride, nvec, w, W, n, partial, red); break;
    case 5: multidot_regs<20, WEIGHTED>(V, stride, nvec, w, W, n, partial, red); break;
    case 6: multidot_regs<24, WEIGHTED>(V, stride, nvec, w, W, n, partial, red); break;
    case 7: multidot_regs<28, WEIGHTED>(V, stride, nvec, w, W, n, partial, red); break;
    default: multidot_regs<32, WEIGHTED>(V, stride, nvec, w, W, n, partial, red); break;
  }
}

// out[k] = sum_b partial[k * nblk + b] for k < nvec (one block per k, fixed order)
__global__ void k_reduce(const double* __restrict__ partial, int nblk, const int* __restrict__ d_j, int nfix,
                         double* __restrict__ out, int off = 0) {
  __shared__ double sh[32];
  const int nvec = d_j ? (*d_j + 1 + off) : nfix;
  const int k = blockIdx.x;
  if (k >= nvec) return;
  double s = 0.0;
  for (int b = threadIdx.x; b < nblk; b += blockDim.x) s += partial[(size_t)k * nblk + b];
  s = block_sum(s, sh);
  if (threadIdx.x == 0) out[k] = s;
}

// w -= sum_{k<nvec} h[k] V_k; if part != null also per-block sum(W w^2) into part[blockIdx.x]
__global__ void k_multiaxpy(double* __restrict__ w, const double* __restrict__ V, size_t stride,
                            const int* __restrict__ d_j, const double* __restrict__ h, size_t n,
                            const double* __restrict__ W, double* __restrict__ part, int off = 0) {
  __shared__ double sh[32];
  __shared__ double hs[kMaxRestart + 2];
  const int nvec = *d_j + 1 + off;
  for (int k = threadIdx.x; k < nvec; k += blockDim.x) hs[k] = h[k];
  __syncthreads();
  double acc = 0.0;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    double v = w[e];
    for (int k = 0; k < nvec; ++k) v -= hs[k] * V[(size_t)k * stride + e];
    w[e] = v;
    if (part) acc += W[e] * v * v;
  }
  if (part) {
    const double s = block_sum(acc, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
  }
}

// Finish one Arnoldi step (one block; thread 0 writes): column j of the Hessenberg matrix
// hcol[k] = h1[k] + h2[k] (k <= j), hcol[j+1] = ||w||_W; inv = 1/||w||_W.
__global__ void k_arnoldi_finish(const int* __restrict__ d_j, const double* __restrict__ h1,
                                 const double* __restrict__ h2, const double* __restrict__ part, int nblk,
                                 double* __restrict__ hcol, double* __restrict__ inv, int* __restrict__ flag) {
  __shared__ double sh[32];
  double s = 0.0;
  for (int b = threadIdx.x; b < nblk; b += blockDim.x) s += part[b];
  s = block_sum(s, sh);
  if (threadIdx.x != 0) return;
  const int j = *d_j;
  double* col = hcol + (size_t)j * kHcolStride;
  for (int k = 0; k <= j; ++k) col[k] = h1[k] + h2[k];
  const double nrm = sqrt(s);
  col[j + 1] = nrm;
  if (!isfinite(nrm)) atomicOr(flag, FLAG_NONFINITE);
  *inv = (nrm > 0.0 && isfinite(nrm)) ? 1.0 / nrm : 0.0;
}

// V_{j+1} = w * inv, then j += 1
__global__ void k_scale_next(double* __restrict__ V, size_t stride, const int* __restrict__ d_j,
                             const double* __restrict__ w, const double* __restrict__ inv, size_t n) {
  const double a = *inv;
  double* dst = V + (size_t)(*d_j + 1) * stride;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
    dst[e] = w[e] * a;
}
__global__ void k_inc(int* d_j) { *d_j += 1; }

// ---- modified Gram-Schmidt in the W inner product, one fused step per basis vector ----------
// The basis is stored scaled by W^(1/2) (sw), so <u, v>_W is the plain dot product of the scaled
// vectors and each step costs two FP64 operations per element. Step k of column j (nvec = *d_j + 1
// basis vectors): step 0 scales w by sw; with k >= 1, h_{k-1} = sum of the previous step's
// per-block partials (fixed order, every block forms the same value; block 0 stores it in
// h[k-1]) and w -= h_{k-1} v_{k-1}; then the per-block partial of v_k . w (k < nvec) or of w . w
// (k == nvec) goes to part_out. Steps k > nvec return at once, so one captured chain of m + 1
// steps serves every j. part_in / part_out alternate between two buffers from step to step.
__global__ void k_mgs_step(const double* __restrict__ V, size_t stride, const int* __restrict__ d_j, int k,
                           double* __restrict__ w, const double* __restrict__ sw, size_t n,
                           const double* __restrict__ part_in, double* __restrict__ part_out,
                           double* __restrict__ h) {
  __shared__ double sh[32];
  __shared__ double hprev_s;
  const int nvec = *d_j + 1;
  if (k > nvec) return;
  double hp = 0.0;
  if (k >= 1) {
    double s = 0.0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) s += part_in[b];
    s = block_sum(s, sh);
    if (threadIdx.x == 0) {
      hprev_s = s;
      if (blockIdx.x == 0) h[k - 1] = s;
    }
    __syncthreads();
    hp = hprev_s;
  }
  const double* vp = V + (size_t)(k >= 1 ? k - 1 : 0) * stride;
  const double* vk = V + (size_t)(k < nvec ? k : 0) * stride;
  double acc = 0.0;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    double x;
    if (k == 0) {
      x = w[e] * sw[e];
      w[e] = x;
    } else {
      x = w[e] - hp * vp[e];
      w[e] = x;
    }
    acc += x * (k < nvec ? vk[e] : x);
  }
  const double s = block_sum(acc, sh);
  if (threadIdx.x == 0) part_out[blockIdx.x] = s;
}

// sw = W^(1/2), isw = W^(-1/2) (0 where W = 0: entries that are not unknowns)
__global__ void k_sqrt_weights(const double* __restrict__ W, double* __restrict__ sw, double* __restrict__ isw,
                               size_t n) {
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    const double r = sqrt(W[e]);
    sw[e] = r;
    isw[e] = r > 0.0 ? 1.0 / r : 0.0;
  }
}

// dst = src * sw * a (the first basis vector in the scaled space)
__global__ void k_scale_sw(double* __restrict__ dst, const double* __restrict__ src, const double* __restrict__ sw,
                           double a, size_t n) {
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
    dst[e] = src[e] * sw[e] * a;
}

// end of a modified Gram-Schmidt column j: ||w||_W from the last step's partials (buffer
// (nvec % 2)), Hessenberg column j = h[0..j] with ||w||_W below the diagonal, inv = 1/||w||_W
__global__ void k_mgs_finish(const int* __restrict__ d_j, const double* __restrict__ h,
                             const double* __restrict__ part2buf, int nblk, double* __restrict__ hcol,
                             double* __restrict__ inv, int* __restrict__ flag) {
  __shared__ double sh[32];
  const int j = *d_j, nvec = j + 1;
  const double* part = part2buf + (size_t)(nvec & 1) * nblk;
  double s = 0.0;
  for (int b = threadIdx.x; b < nblk; b += blockDim.x) s += part[b];
  s = block_sum(s, sh);
  if (threadIdx.x != 0) return;
  double* col = hcol + (size_t)j * kHcolStride;
  for (int q = 0; q <= j; ++q) col[q] = h[q];
  const double nrm = sqrt(s);
  col[j + 1] = nrm;
  if (!isfinite(nrm)) atomicOr(flag, FLAG_NONFINITE);
  *inv = (nrm > 0.0 && isfinite(nrm)) ? 1.0 / nrm : 0.0;
}

// dst = src * a (host scalar)
__global__ void k_scale(double* __restrict__ dst, const double* __restrict__ src, double a, size_t n) {
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
    dst[e] = src[e] * a;
}

// x += sum_{l<k} y[l] Z_l
template <typename TZ>
__global__ void k_update_x(double* __restrict__ x, const TZ* __restrict__ Z, size_t stride, int k,
                           const double* __restrict__ y, size_t n) {
  __shared__ double ys[kMaxRestart + 2];
  for (int l = threadIdx.x; l < k; l += blockDim.x) ys[l] = y[l];
  __syncthreads();
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    double v = x[e];
    for (int l = 0; l < k; ++l) v += ys[l] * (double)Z[(size_t)l * stride + e];
    x[e] = v;
  }
}

// ---- preconditioner input / output ---------------------------------------------------------
// fx, fy (level 0, type T) <- velocity planes of V_j (times isw, when given: the basis is stored
// scaled by W^(1/2)); level-0 iterate zeroed.
template <typename T>
__global__ void k_precond_in(size_t P, const double* __restrict__ V, size_t stride, const int* __restrict__ d_j,
                             T* __restrict__ fx, T* __restrict__ fy, T* __restrict__ vx, T* __restrict__ vy,
                             const double* __restrict__ isw) {
  const double* v = V + (size_t)(*d_j) * stride;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < P; e += (size_t)gridDim.x * blockDim.x) {
    fx[e] = (T)(isw ? v[e] * isw[e] : v[e]);
    fy[e] = (T)(isw ? v[P + e] * isw[P + e] : v[P + e]);
    vx[e] = T(0);
    vy[e] = T(0);
  }
}

// Z_j velocity planes <- level-0 V-cycle result; Z_j pressure <- alpha eta_c (r_p - D z_v)
// (Uzawa pressure block with the sign reading); per-block partial sums of z_p for its mean.
template <typename T, typename TZ>
__global__ void k_precond_out(GeomT<double> g, const T* __restrict__ vx, const T* __restrict__ vy,
                              const double* __restrict__ V, size_t vstride, TZ* __restrict__ Z, size_t stride,
                              const int* __restrict__ d_j, const double* __restrict__ ec, double alpha,
                              double* __restrict__ part, const double* __restrict__ isw) {
  __shared__ double sh[32];
  const size_t P = (size_t)(g.ny + 2) * g.ld;
  const double* v = V + (size_t)(*d_j) * vstride;
  TZ* z = Z + (size_t)(*d_j) * stride;
  const int cols = g.nx + 2;
  double acc = 0.0;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < P; e += (size_t)gridDim.x * blockDim.x) {
    int i, j;
    row_col(e, cols, i, j);
    const TZ zx = is_vx(g.nx, g.ny, i, j) ? (TZ)vx[e] : TZ(0);
    const TZ zy = is_vy(g.nx, g.ny, i, j) ? (TZ)vy[e] : TZ(0);
    z[e] = zx;
    z[P + e] = zy;
    double zp = 0.0;
    if (is_p(g.nx, g.ny, i, j)) {
      // D z_v from the stored (rounded) velocity values, walls masked; at a cell the east and
      // south faces are the point's own vx and vy, already in zx and zy (0 on the walls j = nx
      // and i = ny, where they are not unknowns)
      const double ux = (double)zx;
      const double uxw = (j - 1 >= 1) ? (double)(TZ)vx[e - 1] : 0.0;
      const double uy = (double)zy;
      const double uyn = (i - 1 >= 1) ? (double)(TZ)vy[e - g.ld] : 0.0;
      const double div = (ux - uxw) * g.idx + (uy - uyn) * g.idy;
      const double rp = isw ? v[2 * P + e] * isw[2 * P + e] : v[2 * P + e];
      zp = (double)(TZ)(alpha * ec[e] * (rp - div));
      acc += zp;
    }
    z[2 * P + e] = (TZ)zp;
  }
  const double s = block_sum(acc, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// subtract mean over cells of a pressure plane: every block re-reduces the partials in the same
// fixed order, then subtracts from its share of the cells
template <typename TZ>
__global__ void k_sub_mean(GeomT<double> g, TZ* __restrict__ Zp0, size_t stride, const int* __restrict__ d_j,
                           const double* __restrict__ part, int nblk) {
  __shared__ double sh[32];
  __shared__ double mean;
  double s = 0.0;
  for (int b = threadIdx.x; b < nblk; b += blockDim.x) s += part[b];
  s = block_sum(s, sh);
  if (threadIdx.x == 0) mean = s / ((double)g.nx * (double)g.ny);
  __syncthreads();
  TZ* zp = Zp0 + (d_j ? (size_t)(*d_j) * stride : 0);
  const size_t P = (size_t)(g.ny + 2) * g.ld;
  const int cols = g.nx + 2;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < P; e += (size_t)gridDim.x * blockDim.x) {
    int i, j;
    row_col(e, cols, i, j);
    if (is_p(g.nx, g.ny, i, j)) zp[e] = (TZ)((double)zp[e] - mean);
  }
}

// per-block partial sums of a pressure plane (for the final mean removal of the solution)
__global__ void k_psum(GeomT<double> g, const double* __restrict__ p, double* __restrict__ part) {
  __shared__ double sh[32];
  const size_t P = (size_t)(g.ny + 2) * g.ld;
  const int cols = g.nx + 2;
  double acc = 0.0;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < P; e += (size_t)gridDim.x * blockDim.x) {
    int i, j;
    row_col(e, cols, i, j);
    if (is_p(g.nx, g.ny, i, j)) acc += p[e];
  }
  const double s = block_sum(acc, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// Output: unknowns copied, walls zero, tangential ghosts = s * interior + c, the rest zero.
__global__ void k_output(GeomT<double> g, const double* __restrict__ x, double* __restrict__ vx,
                         double* __restrict__ vy, double* __restrict__ p, double cN, double cS, double cW,
                         double cE) {
  const int i = blockIdx.y * blockDim.y + threadIdx.y;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (i > g.ny + 1 || j > g.nx + 1) return;
  const size_t P = (size_t)(g.ny + 2) * g.ld, c = (size_t)i * g.ld + j;
  const int nx = g.nx, ny = g.ny, ld = g.ld;
  double ox = 0.0, oy = 0.0;
  if (is_vx(nx, ny, i, j)) ox = x[c];
  else if (j >= 1 && j <= nx - 1 && i == 0) ox = g.sN * x[(size_t)1 * ld + j] + cN;
  else if (j >= 1 && j <= nx - 1 && i == ny + 1) ox = g.sS * x[(size_t)ny * ld + j] + cS;
  if (is_vy(nx, ny, i, j)) oy = x[P + c];
  else if (i >= 1 && i <= ny - 1 && j == 0) oy = g.sW * x[P + (size_t)i * ld + 1] + cW;
  else if (i >= 1 && i <= ny - 1 && j == nx + 1) oy = g.sE * x[P + (size_t)i * ld + nx] + cE;
  if (vx) vx[c] = ox;
  if (vy) vy[c] = oy;
  if (p) p[c] = is_p(nx, ny, i, j) ? x[2 * P + c] : 0.0;
}

// ---- adjoint -------------------------------------------------------------------------------
// velocity with the homogeneous (lam) or full (v) boundary rule, for the strain-rate product
__device__ inline double vx_bc(const GeomT<double>& g, const double* x, int i, int j, double cN, double cS) {
  if (j <= 0 || j >= g.nx) return 0.0;
  if (i == 0) return g.sN * x[(size_t)g.ld + j] + cN;
  if (i == g.ny + 1) return g.sS * x[(size_t)g.ny * g.ld + j] + cS;
  return x[(size_t)i * g.ld + j];
}
__device__ inline double vy_bc(const GeomT<double>& g, const double* y, int i, int j, double cW, double cE) {
  if (i <= 0 || i >= g.ny) return 0.0;
  if (j == 0) return g.sW * y[(size_t)i * g.ld + 1] + cW;
  if (j == g.nx + 1) return g.sE * y[(size_t)i * g.ld + g.nx] + cE;
  return y[(size_t)i * g.ld + j];
}

// dJ/deta_c = 2 (exx(v) exx(l) + eyy(v) eyy(l)) at cells; dJ/deta_n = w_n gam(v) gam(l) at nodes
// (w_n = 1 inside, 1/2 on walls, 0 at the four corners); derived by discrete summation by parts
// of the x/y-momentum rows.
__global__ void k_strain_product(GeomT<double> g, const double* __restrict__ x, const double* __restrict__ lam,
                                 double* __restrict__ gn, double* __restrict__ gc) {
  const int i = blockIdx.y * blockDim.y + threadIdx.y;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (i > g.ny + 1 || j > g.nx + 1) return;
  const size_t P = (size_t)(g.ny + 2) * g.ld, c = (size_t)i * g.ld + j;
  const double *vx = x, *vy = x + P, *lx = lam, *ly = lam + P;
  double oc = 0.0, on = 0.0;
  if (is_p(g.nx, g.ny, i, j)) {
    const double exv = (vx_bc(g, vx, i, j, 0, 0) - vx_bc(g, vx, i, j - 1, 0, 0)) * g.idx;
    const double exl = (vx_bc(g, lx, i, j, 0, 0) - vx_bc(g, lx, i, j - 1, 0, 0)) * g.idx;
    const double eyv = (vy_bc(g, vy, i, j, 0, 0) - vy_bc(g, vy, i - 1, j, 0, 0)) * g.idy;
    const double eyl = (vy_bc(g, ly, i, j, 0, 0) - vy_bc(g, ly, i - 1, j, 0, 0)) * g.idy;
    oc = 2.0 * (exv * exl + eyv * eyl);
  }
  if (i <= g.ny && j <= g.nx) {
    const bool wi = (i == 0 || i == g.ny), wj = (j == 0 || j == g.nx);
    const double w = (wi && wj) ? 0.0 : ((wi || wj) ? 0.5 : 1.0);
    if (w > 0.0) {
      const double gv = (vx_bc(g, vx, i + 1, j, 0, 0) - vx_bc(g, vx, i, j, 0, 0)) * g.idy +
                        (vy_bc(g, vy, i, j + 1, 0, 0) - vy_bc(g, vy, i, j, 0, 0)) * g.idx;
      const double gl = (vx_bc(g, lx, i + 1, j, 0, 0) - vx_bc(g, lx, i, j, 0, 0)) * g.idy +
                        (vy_bc(g, ly, i, j + 1, 0, 0) - vy_bc(g, ly, i, j, 0, 0)) * g.idx;
      on = w * gv * gl;
    }
  }
  gc[c] = oc;
  gn[c] = on;
}

// dJ/drho(node) = lam . df/drho with f_x = -gx (rho(i-1,j)+rho(i,j))/2, f_y = -gy (rho(i,j-1)+rho(i,j))/2
__global__ void k_rho_grad(GeomT<double> g, const double* __restrict__ lam, double gx, double gy,
                           double* __restrict__ gr) {
  const int i = blockIdx.y * blockDim.y + threadIdx.y;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (i > g.ny + 1 || j > g.nx + 1) return;
  const size_t P = (size_t)(g.ny + 2) * g.ld, c = (size_t)i * g.ld + j;
  double s = 0.0;
  if (i <= g.ny && j <= g.nx) {
    if (is_vx(g.nx, g.ny, i, j)) s += -0.5 * gx * lam[c];
    if (is_vx(g.nx, g.ny, i + 1, j)) s += -0.5 * gx * lam[c + g.ld];
    if (is_vy(g.nx, g.ny, i, j)) s += -0.5 * gy * lam[P + c];
    if (is_vy(g.nx, g.ny, i, j + 1)) s += -0.5 * gy * lam[P + c + 1];
  }
  gr[c] = s;
}

// ---- viscosity-contrast continuation and lithostatic initial guess (Sec. "Viscosity Rescaling
// and Initial Guess") ---------------------------------------------------------------------------
// per-block minimum of the real nodes (i in [0, ny], j in [0, nx]) and cells of eta
__global__ void k_eta_min(GeomT<double> g, const double* __restrict__ en, const double* __restrict__ ec,
                          double* __restrict__ part) {
  __shared__ double sh[32];
  const size_t P = (size_t)(g.ny + 2) * g.ld;
  const int cols = g.nx + 2;
  double m = INFINITY;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < P; e += (size_t)gridDim.x * blockDim.x) {
    int i, j;
    row_col(e, cols, i, j);
    if (i <= g.ny && j <= g.nx) m = fmin(m, en[e]);
    if (is_p(g.nx, g.ny, i, j)) m = fmin(m, ec[e]);
  }
  for (int o = 16; o > 0; o >>= 1) m = fmin(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    double r = sh[0];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) r = fmin(r, sh[w]);
    part[blockIdx.x] = r;
  }
}

// eta_comp = (1 - theta) eta_min + theta eta on the real nodes and cells, padding copied
__global__ void k_eta_blend(GeomT<double> g, const double* __restrict__ en_full, const double* __restrict__ ec_full,
                            double* __restrict__ en, double* __restrict__ ec, double theta, double emin) {
  const size_t P = (size_t)(g.ny + 2) * g.ld;
  const int cols = g.nx + 2;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < P; e += (size_t)gridDim.x * blockDim.x) {
    int i, j;
    row_col(e, cols, i, j);
    en[e] = (i <= g.ny && j <= g.nx) ? (1.0 - theta) * emin + theta * en_full[e] : en_full[e];
    ec[e] = is_p(g.nx, g.ny, i, j) ? (1.0 - theta) * emin + theta * ec_full[e] : ec_full[e];
  }
}

// lithostatic pressure down each column: p(1, j) = 0, p(i+1, j) = p(i, j) + dy g_y rho_vy(i, j),
// rho_vy the mean of the two basic nodes of the vy node between the cells (one thread per column;
// the mean is removed afterwards)
__global__ void k_litho(GeomT<double> g, const double* __restrict__ rho, double gy, double dy, double* __restrict__ p) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x + 1;
  if (j > g.nx) return;
  double acc = 0.0;
  p[(size_t)1 * g.ld + j] = 0.0;
  for (int i = 1; i < g.ny; ++i) {
    const size_t c = (size_t)i * g.ld + j;
    acc += dy * gy * (0.5 * (rho[c - 1] + rho[c]));
    p[c + g.ld] = acc;
  }
}

// ---- flexible GCR(m) (Sec. "Generalized Conjugate Residual Method", Algorithm gcr) -----------------
// After the Gram-Schmidt passes: w_j = w / nu and z_j = z / nu go to slot j of the two bases,
// with per-block partials of <r, w_j>_W (alpha = that, since ||w_j||_W = 1).
__global__ void k_gcr_scale(double* __restrict__ Wb, double* __restrict__ Zb, size_t stride, const int* __restrict__ d_j,
                            const double* __restrict__ w, const double* __restrict__ zc, const double* __restrict__ inv,
                            const double* __restrict__ r, const double* __restrict__ W, size_t n,
                            double* __restrict__ part) {
  __shared__ double sh[32];
  const double a = *inv;
  double* wd = Wb + (size_t)(*d_j) * stride;
  double* zd = Zb + (size_t)(*d_j) * stride;
  double acc = 0.0;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    const double we = w[e] * a;
    wd[e] = we;
    zd[e] = zc[e] * a;
    acc += W[e] * r[e] * we;
  }
  const double s = block_sum(acc, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// x += alpha z_j, r -= alpha w_j; per-block partials of ||r||_W^2 (alpha reduced on the device)
__global__ void k_gcr_update(double* __restrict__ x, double* __restrict__ r, const double* __restrict__ Wb,
                             const double* __restrict__ Zb, size_t stride, const int* __restrict__ d_j,
                             const double* __restrict__ alpha, const double* __restrict__ W, size_t n,
                             double* __restrict__ part) {
  __shared__ double sh[32];
  const double a = *alpha;
  const double* wj = Wb + (size_t)(*d_j) * stride;
  const double* zj = Zb + (size_t)(*d_j) * stride;
  double acc = 0.0;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    x[e] += a * zj[e];
    const double re = r[e] - a * wj[e];
    r[e] = re;
    acc += W[e] * re * re;
  }
  const double s = block_sum(acc, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// ---- Anderson acceleration AA(m, beta) (Sec. "Anderson Acceleration", Algorithm anderson) -------
// out[q] = sum_b part[2 b + q], q = 0, 1 (the energy / l2 partials of k_residual), fixed order
__global__ void k_sum_pairs(const double* __restrict__ part, int nblk, double* __restrict__ out) {
  __shared__ double sh[32];
  for (int q = 0; q < 2; ++q) {
    double s = 0.0;
    for (int b = threadIdx.x; b < nblk; b += blockDim.x) s += part[2 * b + q];
    s = block_sum(s, sh);
    if (threadIdx.x == 0) out[q] = s;
    __syncthreads();
  }
}

// history slot d_slot <- (x, z): the iterate and its fixed-point residual G(x) - x = M^-1 (b - A x)
__global__ void k_aa_store(double* __restrict__ Xh, double* __restrict__ Zh, size_t stride, const int* __restrict__ d_slot,
                           const double* __restrict__ x, const double* __restrict__ zc, size_t n) {
  double* xd = Xh + (size_t)(*d_slot) * stride;
  double* zd = Zh + (size_t)(*d_slot) * stride;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    xd[e] = x[e];
    zd[e] = zc[e];
  }
}

// x = sum_i a_i ((1 - beta) x_i + beta G(x_i)) = sum_i a_i (x_i + beta z_i) over the cnt stored slots
__global__ void k_aa_combine(double* __restrict__ x, const double* __restrict__ Xh, const double* __restrict__ Zh,
                             size_t stride, int cnt, const double* __restrict__ a, double beta, size_t n) {
  __shared__ double as[kMaxRestart + 2];
  for (int k = threadIdx.x; k < cnt; k += blockDim.x) as[k] = a[k];
  __syncthreads();
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    double v = 0.0;
    for (int k = 0; k < cnt; ++k) v += as[k] * (Xh[(size_t)k * stride + e] + beta * Zh[(size_t)k * stride + e]);
    x[e] = v;
  }
}

template __global__ void k_apply<double>(GeomT<double>, const double*, const double*, const double*, size_t,
                                         const int*, double*, Coef<double>);
template __global__ void k_update_x<double>(double*, const double*, size_t, int, const double*, size_t);
template __global__ void k_update_x<float>(double*, const float*, size_t, int, const double*, size_t);
template __global__ void k_precond_in<float>(size_t, const double*, size_t, const int*, float*, float*, float*, float*,
                                             const double*);
template __global__ void k_precond_in<double>(size_t, const double*, size_t, const int*, double*, double*, double*,
                                              double*, const double*);
template __global__ void k_precond_out<float, double>(GeomT<double>, const float*, const float*, const double*,
                                                      size_t, double*, size_t, const int*, const double*, double,
                                                      double*, const double*);
template __global__ void k_precond_out<double, double>(GeomT<double>, const double*, const double*, const double*,
                                                       size_t, double*, size_t, const int*, const double*, double,
                                                       double*, const double*);
template __global__ void k_sub_mean<float>(GeomT<double>, float*, size_t, const int*, const double*, int);
template __global__ void k_sub_mean<double>(GeomT<double>, double*, size_t, const int*, const double*, int);

}  // namespace pyro
