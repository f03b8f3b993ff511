// Allocation-free variant of the fused Stokes residual + energy-norm kernel.
//
// Who needs this: some callers cannot call cudaMalloc at all — for example an application that
// has handed the whole device to its own pool allocator (a cudaMalloc would fail or fragment it),
// or a latency-critical loop in which an allocation's implicit device synchronisation is not
// acceptable. The regular entry points allocate their workspace in pyro_stokes_create; this one
// needs no handle and no allocation: its only scratch (the per-block partial sums of the
// reductions) lives in a fixed-size array in device global memory that exists from the moment the
// library is loaded until the process exits, on every GPU that loads the library.
//
// The computation is the same as the residual step of the solve: r = b - A x with
// b = -rho g on the velocity nodes plus the constants of prescribed-velocity boundaries, followed
// by the relative energy residual and the relative l2 residual.
#include <cuda_runtime.h>

#include <cmath>

#include "../../include/pyro.h"
#include "common.cuh"

namespace {

using namespace pyro;

// Scratch: one slot of 4 partial sums per block of rows, plus 4 result slots.
constexpr int kNoAllocRowsPerBlock = 4;
constexpr int kNoAllocMaxBlocks = 4095;
constexpr int kNoAllocSlots = 4 * kNoAllocMaxBlocks + 4;  // 16384 doubles = 128 KiB
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocSlots];

__device__ inline double nb_block_sum(double v, double* sh) {
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

__device__ inline double in_vx(const GeomT<double>& g, const double* a, int i, int j) {
  return is_vx(g.nx, g.ny, i, j) ? a[(size_t)i * g.ld + j] : 0.0;
}
__device__ inline double in_vy(const GeomT<double>& g, const double* a, int i, int j) {
  return is_vy(g.nx, g.ny, i, j) ? a[(size_t)i * g.ld + j] : 0.0;
}
__device__ inline double in_p(const GeomT<double>& g, const double* a, int i, int j) {
  return is_p(g.nx, g.ny, i, j) ? a[(size_t)i * g.ld + j] : 0.0;
}

// Velocity reads mask everything that is not an unknown (caller arrays may hold anything in
// ghosts and walls), then apply the same point operators as the solve.
__device__ inline double lx_masked(const GeomT<double>& g, int i, int j, const double* vx, const double* vy,
                                   const double* en, const double* ec) {
  const double eA = ec[(size_t)i * g.ld + j], eB = ec[(size_t)i * g.ld + j + 1];
  const double e1 = en[(size_t)(i - 1) * g.ld + j], e2 = en[(size_t)i * g.ld + j];
  const double vc = in_vx(g, vx, i, j);
  const double vw = in_vx(g, vx, i, j - 1), ve = in_vx(g, vx, i, j + 1);
  const double vn = (i == 1) ? g.sN * vc : in_vx(g, vx, i - 1, j);
  const double vs = (i == g.ny) ? g.sS * vc : in_vx(g, vx, i + 1, j);
  const double yA = in_vy(g, vy, i - 1, j), yB = in_vy(g, vy, i - 1, j + 1);
  const double yC = in_vy(g, vy, i, j), yD = in_vy(g, vy, i, j + 1);
  const double sxxE = 2.0 * eB * (ve - vc), sxxW = 2.0 * eA * (vc - vw);
  const double sxyS = e2 * ((vs - vc) * g.idy2 + (yD - yC) * g.idxdy);
  const double sxyN = e1 * ((vc - vn) * g.idy2 + (yB - yA) * g.idxdy);
  return (sxxE - sxxW) * g.idx2 + sxyS - sxyN;
}

__device__ inline double ly_masked(const GeomT<double>& g, int i, int j, const double* vx, const double* vy,
                                   const double* en, const double* ec) {
  const double eA = ec[(size_t)i * g.ld + j], eB = ec[(size_t)(i + 1) * g.ld + j];
  const double e1 = en[(size_t)i * g.ld + j - 1], e2 = en[(size_t)i * g.ld + j];
  const double vc = in_vy(g, vy, i, j);
  const double vn = in_vy(g, vy, i - 1, j), vs = in_vy(g, vy, i + 1, j);
  const double vw = (j == 1) ? g.sW * vc : in_vy(g, vy, i, j - 1);
  const double ve = (j == g.nx) ? g.sE * vc : in_vy(g, vy, i, j + 1);
  const double xA = in_vx(g, vx, i, j - 1), xB = in_vx(g, vx, i + 1, j - 1);
  const double xC = in_vx(g, vx, i, j), xD = in_vx(g, vx, i + 1, j);
  const double syyS = 2.0 * eB * (vs - vc), syyN = 2.0 * eA * (vc - vn);
  const double sxyE = e2 * ((ve - vc) * g.idx2 + (xD - xC) * g.idxdy);
  const double sxyW = e1 * ((vc - vw) * g.idx2 + (xB - xA) * g.idxdy);
  return (syyS - syyN) * g.idy2 + sxyE - sxyW;
}

__device__ inline double diag_x(const GeomT<double>& g, const double* en, const double* ec, int i, int j) {
  const size_t c = (size_t)i * g.ld + j;
  double d = -2.0 * (ec[c] + ec[c + 1]) * g.idx2 - (en[c - g.ld] + en[c]) * g.idy2;
  if (i == 1) d += g.sN * en[c - g.ld] * g.idy2;
  if (i == g.ny) d += g.sS * en[c] * g.idy2;
  return d;
}
__device__ inline double diag_y(const GeomT<double>& g, const double* en, const double* ec, int i, int j) {
  const size_t c = (size_t)i * g.ld + j;
  double d = -2.0 * (ec[c] + ec[c + g.ld]) * g.idy2 - (en[c - 1] + en[c]) * g.idx2;
  if (j == 1) d += g.sW * en[c - 1] * g.idx2;
  if (j == g.nx) d += g.sE * en[c] * g.idx2;
  return d;
}

// One block per kNoAllocRowsPerBlock padded rows. Writes r (all padded entries: unknowns get the
// residual, everything else 0) and the block's partials [sum W r^2, sum r^2, sum W b_v^2, sum b^2]
// into scratch[4 * blockIdx.x + 0..3]. Every slot read later is written here first.
__global__ void k_residual_noalloc(GeomT<double> g, const double* __restrict__ en, const double* __restrict__ ec,
                                   const double* __restrict__ rho, double gx, double gy, double cN, double cS,
                                   double cW, double cE, const double* __restrict__ vx,
                                   const double* __restrict__ vy, const double* __restrict__ p,
                                   double* __restrict__ rx, double* __restrict__ ry, double* __restrict__ rp,
                                   double* __restrict__ scratch) {
  __shared__ double sh[32];
  const int cols = g.nx + 2;
  const int i0 = blockIdx.x * kNoAllocRowsPerBlock;
  const int i1 = min(i0 + kNoAllocRowsPerBlock, g.ny + 2);
  double swr = 0.0, sr = 0.0, swb = 0.0, sb = 0.0;
  for (int e = threadIdx.x; e < (i1 - i0) * cols; e += blockDim.x) {
    const int i = i0 + e / cols, j = e % cols;
    const size_t c = (size_t)i * g.ld + j;
    double ox = 0.0, oy = 0.0, op = 0.0;
    if (is_vx(g.nx, g.ny, i, j)) {
      double b = -gx * 0.5 * (rho[c - g.ld] + rho[c]);
      if (i == 1) b -= en[c - g.ld] * g.idy2 * cN;
      if (i == g.ny) b -= en[c] * g.idy2 * cS;
      const double Ax = lx_masked(g, i, j, vx, vy, en, ec) - (in_p(g, p, i, j + 1) - in_p(g, p, i, j)) * g.idx;
      ox = b - Ax;
      const double w = -1.0 / diag_x(g, en, ec, i, j);
      swr += w * ox * ox; sr += ox * ox; swb += w * b * b; sb += b * b;
    }
    if (is_vy(g.nx, g.ny, i, j)) {
      double b = -gy * 0.5 * (rho[c - 1] + rho[c]);
      if (j == 1) b -= en[c - 1] * g.idx2 * cW;
      if (j == g.nx) b -= en[c] * g.idx2 * cE;
      const double Ay = ly_masked(g, i, j, vx, vy, en, ec) - (in_p(g, p, i + 1, j) - in_p(g, p, i, j)) * g.idy;
      oy = b - Ay;
      const double w = -1.0 / diag_y(g, en, ec, i, j);
      swr += w * oy * oy; sr += oy * oy; swb += w * b * b; sb += b * b;
    }
    if (is_p(g.nx, g.ny, i, j)) {
      const double div = (in_vx(g, vx, i, j) - in_vx(g, vx, i, j - 1)) * g.idx +
                         (in_vy(g, vy, i, j) - in_vy(g, vy, i - 1, j)) * g.idy;
      op = -div;
      const double w = ec[c] / (2.0 * g.idx2 + 2.0 * g.idy2);
      swr += w * op * op; sr += op * op;
    }
    rx[c] = ox; ry[c] = oy; rp[c] = op;
  }
  const double a0 = nb_block_sum(swr, sh), a1 = nb_block_sum(sr, sh);
  const double a2 = nb_block_sum(swb, sh), a3 = nb_block_sum(sb, sh);
  if (threadIdx.x == 0) {
    double* slot = scratch + 4 * blockIdx.x;
    slot[0] = a0; slot[1] = a1; slot[2] = a2; slot[3] = a3;
  }
}

// Fixed-order sum of the nblk slots into the 4 result slots behind them, then the two relative
// residuals into result slots 0 and 1.
__global__ void k_finish_noalloc(double* __restrict__ scratch, int nblk) {
  __shared__ double sh[32];
  double acc[4];
  for (int q = 0; q < 4; ++q) {
    double s = 0.0;
    for (int b = threadIdx.x; b < nblk; b += blockDim.x) s += scratch[4 * b + q];
    acc[q] = nb_block_sum(s, sh);
  }
  if (threadIdx.x == 0) {
    double* res = scratch + 4 * kNoAllocMaxBlocks;
    res[0] = acc[2] > 0.0 ? sqrt(acc[0] / acc[2]) : sqrt(acc[0]);
    res[1] = acc[3] > 0.0 ? sqrt(acc[1] / acc[3]) : sqrt(acc[1]);
    res[2] = acc[0];
    res[3] = acc[2];
  }
}

// Device address of g_noalloc_scratch in the current device's context. Looked up on every call:
// the lookup allocates nothing, and an address kept from an earlier call would be stale after the
// context that held it was destroyed (cudaDeviceReset, or a primary context released and made
// again). The first lookup in a context may load the library's device code, which is why the first
// call on a device should come before any stream capture.
int scratch_address(double** out) {
  void* ptr = nullptr;
  if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) {
    cudaGetLastError();
    return PYRO_E_CUDA;
  }
  *out = (double*)ptr;
  return PYRO_OK;
}

// device memory of the current device (or managed memory); host pointers and other GPUs' memory
// are rejected
bool on_device(const void* p) { return ptr_place(p) == PTR_HERE; }

}  // namespace

extern "C" int pyro_stokes_residual_noalloc(int nx, int ny, double Lx, double Ly, const pyro_bc* bc,
                                            const double* eta_n, const double* eta_c, const double* rho,
                                            double gx, double gy, const double* vx, const double* vy,
                                            const double* p, double* r_vx, double* r_vy, double* r_p,
                                            double* rel_res, void* cuda_stream) {
  if (nx < 2 || ny < 2 || !(Lx > 0) || !(Ly > 0) || !rel_res) return PYRO_E_INVALID;
  const int nblk = (ny + 2 + kNoAllocRowsPerBlock - 1) / kNoAllocRowsPerBlock;
  if (nblk > kNoAllocMaxBlocks) return PYRO_E_INVALID;  // ny + 2 > 16380: beyond the fixed scratch
  const double* ins[6] = {eta_n, eta_c, rho, vx, vy, p};
  double* outs[3] = {r_vx, r_vy, r_p};
  for (const double* a : ins)
    if (!on_device(a)) return PYRO_E_INVALID;
  for (double* a : outs)
    if (!on_device(a)) return PYRO_E_INVALID;
  const PtrPlace res_place = ptr_place(rel_res);
  if (res_place == PTR_OTHER) return PYRO_E_INVALID;
  pyro_bc b{};
  for (int k = 0; k < 4; ++k) { b.kind[k] = PYRO_BC_FREE_SLIP; b.vt[k] = 0.0; }
  if (bc) b = *bc;
  for (int k = 0; k < 4; ++k)
    if (b.kind[k] != PYRO_BC_FREE_SLIP && b.kind[k] != PYRO_BC_NO_SLIP && b.kind[k] != PYRO_BC_VELOCITY)
      return PYRO_E_INVALID;
  double* scratch = nullptr;
  const int st = scratch_address(&scratch);
  if (st != PYRO_OK) return st;
  Geom g0;
  g0.nx = nx; g0.ny = ny; g0.ld = nx + 2; g0.dx = Lx / nx; g0.dy = Ly / ny;
  auto s_of = [&](int side) { return b.kind[side] == PYRO_BC_FREE_SLIP ? 1.0 : -1.0; };
  auto c_of = [&](int side) { return b.kind[side] == PYRO_BC_VELOCITY ? 2.0 * b.vt[side] : 0.0; };
  g0.sW = s_of(0); g0.sE = s_of(1); g0.sN = s_of(2); g0.sS = s_of(3);
  const GeomT<double> g = geomT<double>(g0);
  cudaStream_t s = (cudaStream_t)cuda_stream;
  k_residual_noalloc<<<nblk, 256, 0, s>>>(g, eta_n, eta_c, rho, gx, gy, c_of(2), c_of(3), c_of(0), c_of(1), vx, vy,
                                          p, r_vx, r_vy, r_p, scratch);
  k_finish_noalloc<<<1, 256, 0, s>>>(scratch, nblk);
  const bool dev_out = res_place == PTR_HERE;
  if (cudaMemcpyAsync(rel_res, scratch + 4 * kNoAllocMaxBlocks, 2 * sizeof(double),
                      dev_out ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s) != cudaSuccess) {
    cudaGetLastError();
    return PYRO_E_CUDA;
  }
  if (cudaStreamSynchronize(s) != cudaSuccess) return PYRO_E_CUDA;
  return PYRO_OK;
}
