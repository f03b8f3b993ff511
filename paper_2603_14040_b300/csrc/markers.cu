// Marker steps of the marker-in-cell loop: marker <-> grid interpolation (Sec. "Marker-to-grid
// interpolation" and "Grid-to-marker interpolation"), the step that feeds eta and rho to the
// Stokes solve, and the advection of the markers in the solved velocity (Sec. "Advection of
// Lagrangian Markers": forward Euler, Heun, classical RK4, the locally polynomial Taylor update).
//
// Marker -> grid is a weighted average over the markers around each lattice node with bilinear
// weights. The paper accumulates with atomics; floating-point atomics make the result depend on
// the arrival order, so here the markers are bucketed by lattice cell (integer atomics only: the
// counts and slots), each bucket is sorted by marker index, and every node gathers from the four
// cells around it in a fixed order. The result is deterministic and independent of the launch.
//
// Lattices: basic nodes (x_j = j dx, y_i = i dy, i in [0, ny], j in [0, nx]), cell centres
// (x_j = (j - 1/2) dx, y_i = (i - 1/2) dy, i, j in [1, n]), vx points (x_j = j dx,
// y_i = (i - 1/2) dy, i in [1, ny], j in [0, nx]) and vy points (x_j = (j - 1/2) dx, y_i = i dy,
// i in [0, ny], j in [1, nx]) in the padded (ny+2) x (nx+2) layout; row i goes with y. A marker belongs to the lattice cell whose top-left node is at or left/above
// it (clamped into the outermost cell when it lies beyond the lattice); that node takes the weight
// (1 - fx)(1 - fy), its right neighbour fx (1 - fy), the one below (1 - fx) fy, the diagonal fx fy.
#include <cuda_runtime.h>
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <new>

#include "../../include/pyro.h"
#include "common.cuh"

struct pyro_markers_s {
  int dev = 0;
  int nx = 0, ny = 0;
  double Lx = 1, Ly = 1;
  long long cap = 0;       // marker capacity
  int* count = nullptr;    // per lattice cell (largest lattice: (ny + 1) x (nx + 1) cells)
  int* offset = nullptr;   // exclusive prefix of count (+1 entry)
  int* fill = nullptr;     // slots handed out per cell
  int* bsum = nullptr;     // per-block sums of the scan
  int* idx = nullptr;      // marker indices bucketed by cell
  int* cell = nullptr;     // cell of each marker
  double* frac = nullptr;  // (fx, fy) of each marker
  double* csum = nullptr;  // per-cell corner sums: 4 planes of sum w phi, 4 of sum w (TL, TR, BL, BR)
  int* flag = nullptr;
  double* red = nullptr;   // per-block maxima of the CFL reduction (2 x kRedBlocks)
};

namespace {

using namespace pyro;
constexpr int kMkThreads = 256;
constexpr int kScanBlock = 1024;
constexpr int kRedBlocks = 296;

struct Lat {
  double x0, y0, idx, idy;
  double ox, oy;           // -x0 idx, -y0 idy: lattice coordinate u = x idx + ox
  int ilo, ihi, jlo, jhi;  // lattice index range (inclusive)
  int ncx, ncy;            // lattice cells per row / column
};

Lat make_lat(const pyro_markers_s* h, int kind) {
  Lat L;
  const double dx = h->Lx / h->nx, dy = h->Ly / h->ny;
  L.idx = 1.0 / dx;
  L.idy = 1.0 / dy;
  if (kind == PYRO_LATTICE_CELLS) {
    L.x0 = -0.5 * dx; L.y0 = -0.5 * dy; L.ilo = 1; L.ihi = h->ny; L.jlo = 1; L.jhi = h->nx;
  } else if (kind == PYRO_LATTICE_VX) {
    L.x0 = 0.0; L.y0 = -0.5 * dy; L.ilo = 1; L.ihi = h->ny; L.jlo = 0; L.jhi = h->nx;
  } else if (kind == PYRO_LATTICE_VY) {
    L.x0 = -0.5 * dx; L.y0 = 0.0; L.ilo = 0; L.ihi = h->ny; L.jlo = 1; L.jhi = h->nx;
  } else {
    L.x0 = 0.0; L.y0 = 0.0; L.ilo = 0; L.ihi = h->ny; L.jlo = 0; L.jhi = h->nx;
  }
  L.ncx = L.jhi - L.jlo;
  L.ncy = L.ihi - L.ilo;
  L.ox = -L.x0 * L.idx;
  L.oy = -L.y0 * L.idy;
  return L;
}

// lattice cell (i, j) and fractions of (x, y); a coordinate beyond the lattice (or not finite)
// lands in the outermost cell (NaN: the first) with its fraction clamped to [0, 1]
__device__ inline void locate(const Lat& L, double x, double y, int& i, int& j, double& fx, double& fy) {
  const double u = fma(x, L.idx, L.ox), v = fma(y, L.idy, L.oy);
  const double fu = floor(u), fv = floor(v);
  j = !(fu >= L.jlo) ? L.jlo : (fu >= L.jhi - 1 ? L.jhi - 1 : (int)fu);
  i = !(fv >= L.ilo) ? L.ilo : (fv >= L.ihi - 1 ? L.ihi - 1 : (int)fv);
  fx = fmin(fmax(u - j, 0.0), 1.0);
  fy = fmin(fmax(v - i, 0.0), 1.0);
}

__global__ void k_mk_count(Lat L, long long n, const double* __restrict__ xm, const double* __restrict__ ym,
                           int* __restrict__ cell, double* __restrict__ frac, int* __restrict__ count,
                           int* __restrict__ flag) {
  for (long long m = (long long)blockIdx.x * blockDim.x + threadIdx.x; m < n; m += (long long)gridDim.x * blockDim.x) {
    const double x = xm[m], y = ym[m];
    if (!isfinite(x) || !isfinite(y)) { atomicOr(flag, FLAG_NONFINITE); cell[m] = -1; continue; }
    int i, j;
    double fx, fy;
    locate(L, x, y, i, j, fx, fy);
    const int c = (i - L.ilo) * L.ncx + (j - L.jlo);
    cell[m] = c;
    frac[2 * m] = fx;
    frac[2 * m + 1] = fy;
    atomicAdd(&count[c], 1);
  }
}

// exclusive scan of count[0..n) into offset[0..n]: per-block scans, then the block sums
__global__ void k_scan_blocks(const int* __restrict__ in, int* __restrict__ out, int n, int* __restrict__ bsum) {
  __shared__ int s[kScanBlock];
  const int g = blockIdx.x * kScanBlock + threadIdx.x;
  s[threadIdx.x] = g < n ? in[g] : 0;
  __syncthreads();
  for (int d = 1; d < kScanBlock; d <<= 1) {     // Hillis-Steele inclusive scan
    const int t = threadIdx.x >= d ? s[threadIdx.x - d] : 0;
    __syncthreads();
    s[threadIdx.x] += t;
    __syncthreads();
  }
  if (g < n) out[g] = s[threadIdx.x] - (g < n ? in[g] : 0);
  if (threadIdx.x == kScanBlock - 1) bsum[blockIdx.x] = s[threadIdx.x];
}

__global__ void k_scan_sums(int* __restrict__ bsum, int nb) {   // one thread, nb small
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  int acc = 0;
  for (int b = 0; b < nb; ++b) { const int t = bsum[b]; bsum[b] = acc; acc += t; }
  bsum[nb] = acc;
}

__global__ void k_scan_add(int* __restrict__ out, int n, const int* __restrict__ bsum) {
  const int g = blockIdx.x * kScanBlock + threadIdx.x;
  if (g < n) out[g] += bsum[blockIdx.x];
  if (g == 0) out[n] = bsum[gridDim.x];
}

__global__ void k_mk_scatter(long long n, const int* __restrict__ cell, const int* __restrict__ offset,
                             int* __restrict__ fill, int* __restrict__ idx) {
  for (long long m = (long long)blockIdx.x * blockDim.x + threadIdx.x; m < n; m += (long long)gridDim.x * blockDim.x) {
    const int c = cell[m];
    if (c < 0) continue;
    idx[offset[c] + atomicAdd(&fill[c], 1)] = (int)m;
  }
}

// insertion sort of each cell's bucket by marker index (buckets hold a few to a few tens)
__global__ void k_mk_sort(int ncell, const int* __restrict__ offset, int* __restrict__ idx) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncell) return;
  const int a = offset[c], b = offset[c + 1];
  for (int k = a + 1; k < b; ++k) {
    const int v = idx[k];
    int q = k - 1;
    while (q >= a && idx[q] > v) { idx[q + 1] = idx[q]; --q; }
    idx[q + 1] = v;
  }
}

// Per-cell corner sums: for the markers of lattice cell c in index order, sum w phi and sum w for
// each corner node of the cell (top-left, top-right, bottom-left, bottom-right), w the bilinear
// weight of the marker at that corner. Each marker is read once (the node pass below adds up
// four cells' sums instead of re-reading their markers).
__global__ void k_mk_cell_sums(int ncell, const int* __restrict__ offset, const int* __restrict__ idx,
                               const double* __restrict__ frac, const double* __restrict__ phim,
                               double* __restrict__ cs) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncell) return;
  double n0 = 0.0, n1 = 0.0, n2 = 0.0, n3 = 0.0, d0 = 0.0, d1 = 0.0, d2 = 0.0, d3 = 0.0;
  for (int k = offset[c]; k < offset[c + 1]; ++k) {
    const int m = idx[k];
    const double fx = frac[2 * m], fy = frac[2 * m + 1], p = phim[m];
    const double w0 = (1.0 - fx) * (1.0 - fy), w1 = fx * (1.0 - fy), w2 = (1.0 - fx) * fy, w3 = fx * fy;
    n0 += w0 * p; n1 += w1 * p; n2 += w2 * p; n3 += w3 * p;
    d0 += w0; d1 += w1; d2 += w2; d3 += w3;
  }
  cs[c] = n0; cs[(size_t)ncell + c] = n1; cs[2 * (size_t)ncell + c] = n2; cs[3 * (size_t)ncell + c] = n3;
  cs[4 * (size_t)ncell + c] = d0; cs[5 * (size_t)ncell + c] = d1; cs[6 * (size_t)ncell + c] = d2;
  cs[7 * (size_t)ncell + c] = d3;
}

// phi(i, j) = sum w phi_m / sum w over the markers of the four cells around node (i, j): the cells'
// corner sums for this node, cells in the order (i-1, j-1), (i-1, j), (i, j-1), (i, j)
__global__ void k_mk_node_sums(Lat L, int ld, const double* __restrict__ cs, int ncell,
                               double* __restrict__ grid, double* __restrict__ wsum) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x + L.jlo;
  const int i = blockIdx.y * blockDim.y + threadIdx.y + L.ilo;
  if (i > L.ihi || j > L.jhi) return;
  double num = 0.0, den = 0.0;
  for (int q = 0; q < 4; ++q) {
    const int ci = i - 1 + (q >> 1), cj = j - 1 + (q & 1);     // cell with top-left node (ci, cj)
    if (ci < L.ilo || ci > L.ihi - 1 || cj < L.jlo || cj > L.jhi - 1) continue;
    const int c = (ci - L.ilo) * L.ncx + (cj - L.jlo);
    const int corner = (ci < i ? 2 : 0) + (cj < j ? 1 : 0);     // this node is the cell's corner
    num += cs[(size_t)corner * ncell + c];
    den += cs[(size_t)(4 + corner) * ncell + c];
  }
  const size_t o = (size_t)i * ld + j;
  if (den > 0.0) grid[o] = num / den;
  if (wsum) wsum[o] = den;
}

__global__ void k_mk_to_markers(Lat L, int ld, long long n, const double* __restrict__ xm, const double* __restrict__ ym,
                                const double* __restrict__ grid, double* __restrict__ phim) {
  for (long long m = (long long)blockIdx.x * blockDim.x + threadIdx.x; m < n; m += (long long)gridDim.x * blockDim.x) {
    int i, j;
    double fx, fy;
    locate(L, xm[m], ym[m], i, j, fx, fy);
    const size_t o = (size_t)i * ld + j;
    phim[m] = (1.0 - fx) * (1.0 - fy) * grid[o] + fx * (1.0 - fy) * grid[o + 1] + (1.0 - fx) * fy * grid[o + ld] +
              fx * fy * grid[o + ld + 1];
  }
}

// ---- advection --------------------------------------------------------------------------------
// bilinear value of a lattice field at (x, y), the same arithmetic as k_mk_to_markers
__device__ inline double interp(const Lat& L, int ld, const double* __restrict__ g, double x, double y) {
  int i, j;
  double fx, fy;
  locate(L, x, y, i, j, fx, fy);
  const size_t o = (size_t)i * ld + j;
  return (1.0 - fx) * (1.0 - fy) * g[o] + fx * (1.0 - fy) * g[o + 1] + (1.0 - fx) * fy * g[o + ld] +
         fx * fy * g[o + ld + 1];
}

// value, d/dx, d/dy and d2/dxdy of the bilinear interpolant at (x, y); a derivative across a
// direction in which the point lies beyond the lattice is zero (the clamped interpolant is flat)
__device__ inline void interp_d(const Lat& L, int ld, const double* __restrict__ g, double x, double y, double& val,
                                double& ddx, double& ddy, double& dxy) {
  int i, j;
  double fx, fy;
  locate(L, x, y, i, j, fx, fy);
  const double u = fma(x, L.idx, L.ox), v = fma(y, L.idy, L.oy);
  const bool inx = u >= L.jlo && u <= L.jhi, iny = v >= L.ilo && v <= L.ihi;
  const size_t o = (size_t)i * ld + j;
  const double a00 = g[o], a01 = g[o + 1], a10 = g[o + ld], a11 = g[o + ld + 1];
  val = (1.0 - fx) * (1.0 - fy) * a00 + fx * (1.0 - fy) * a01 + (1.0 - fx) * fy * a10 + fx * fy * a11;
  ddx = inx ? ((a01 - a00) * (1.0 - fy) + (a11 - a10) * fy) * L.idx : 0.0;
  ddy = iny ? ((a10 - a00) * (1.0 - fx) + (a11 - a01) * fx) * L.idy : 0.0;
  dxy = (inx && iny) ? (a11 - a10 - a01 + a00) * (L.idx * L.idy) : 0.0;
}

struct VelField {
  Lat lu, lv;  // vx and vy lattices
  int ld;
  const double* vx;
  const double* vy;
  __device__ inline void at(double x, double y, double& u, double& v) const {
    u = interp(lu, ld, vx, x, y);
    v = interp(lv, ld, vy, x, y);
  }
};

// substeps steps of size h of the scheme (Sec. "Advection of Lagrangian Markers"), each result
// clamped into [0, Lx] x [0, Ly]; one thread per marker, FP64 throughout
template <int SCHEME>
__global__ void k_mk_advect(VelField F, long long n, double* __restrict__ xm, double* __restrict__ ym, double h,
                            int substeps, double Lx, double Ly) {
  for (long long m = (long long)blockIdx.x * blockDim.x + threadIdx.x; m < n; m += (long long)gridDim.x * blockDim.x) {
    double x = xm[m], y = ym[m];
    for (int k = 0; k < substeps; ++k) {
      double xn, yn;
      if (SCHEME == PYRO_ADVECT_EULER) {            // eq. euler_advection
        double u, v;
        F.at(x, y, u, v);
        xn = x + h * u;
        yn = y + h * v;
      } else if (SCHEME == PYRO_ADVECT_HEUN) {      // eq. heun_method
        double u1, v1, u2, v2;
        F.at(x, y, u1, v1);
        F.at(x + h * u1, y + h * v1, u2, v2);
        xn = x + 0.5 * h * (u1 + u2);
        yn = y + 0.5 * h * (v1 + v2);
      } else if (SCHEME == PYRO_ADVECT_RK4) {       // eq. rk4_method
        double u1, v1, u2, v2, u3, v3, u4, v4;
        F.at(x, y, u1, v1);
        F.at(x + 0.5 * h * u1, y + 0.5 * h * v1, u2, v2);
        F.at(x + 0.5 * h * u2, y + 0.5 * h * v2, u3, v3);
        F.at(x + h * u3, y + h * v3, u4, v4);
        xn = x + h / 6.0 * (u1 + 2.0 * u2 + 2.0 * u3 + u4);
        yn = y + h / 6.0 * (v1 + 2.0 * v2 + 2.0 * v3 + v4);
      } else {                                       // eq. lpi_update: x + h v0 + h^2/2 J v0 + h^3/6 H:v0 v0
        double u, ux, uy, uxy, v, vx_, vy_, vxy;
        interp_d(F.lu, F.ld, F.vx, x, y, u, ux, uy, uxy);
        interp_d(F.lv, F.ld, F.vy, x, y, v, vx_, vy_, vxy);
        const double h2 = 0.5 * h * h, h3 = h * h * h / 6.0;
        xn = x + h * u + h2 * (ux * u + uy * v) + h3 * (2.0 * uxy * u * v);
        yn = y + h * v + h2 * (vx_ * u + vy_ * v) + h3 * (2.0 * vxy * u * v);
      }
      x = fmin(fmax(xn, 0.0), Lx);
      y = fmin(fmax(yn, 0.0), Ly);
    }
    xm[m] = x;
    ym[m] = y;
  }
}

// per-block max |a| and max |b| over n entries (NaN propagates); red[blockIdx.x], red[gridDim.x + blockIdx.x]
__global__ void k_absmax2(const double* __restrict__ a, const double* __restrict__ b, size_t n, double* __restrict__ red) {
  __shared__ double sa[kMkThreads / 32], sb[kMkThreads / 32];
  double ma = 0.0, mb = 0.0;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    const double x = fabs(a[e]), y = fabs(b[e]);
    ma = (x > ma || isnan(x)) ? x : ma;
    mb = (y > mb || isnan(y)) ? y : mb;
  }
  for (int o = 16; o > 0; o >>= 1) {
    const double x = __shfl_xor_sync(0xffffffffu, ma, o), y = __shfl_xor_sync(0xffffffffu, mb, o);
    ma = (x > ma || isnan(x)) ? x : ma;
    mb = (y > mb || isnan(y)) ? y : mb;
  }
  if ((threadIdx.x & 31) == 0) { sa[threadIdx.x >> 5] = ma; sb[threadIdx.x >> 5] = mb; }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int k = 1; k < kMkThreads / 32; ++k) {
      ma = (sa[k] > ma || isnan(sa[k])) ? sa[k] : ma;
      mb = (sb[k] > mb || isnan(sb[k])) ? sb[k] : mb;
    }
    red[blockIdx.x] = ma;
    red[gridDim.x + blockIdx.x] = mb;
  }
}

// device memory of the current device (or managed memory); host pointers and other GPUs' memory
// are rejected by the callers
bool on_device(const void* p) { return pyro::ptr_place(p) == pyro::PTR_HERE; }

int grid_blocks(long long n) { return (int)((n + kMkThreads - 1) / kMkThreads < 4 * 148 * 8 ? (n + kMkThreads - 1) / kMkThreads : 4 * 148 * 8); }

}  // namespace

extern "C" {

int pyro_markers_create(int nx, int ny, double Lx, double Ly, long long max_markers, pyro_markers* out) {
  if (!out || nx < 2 || ny < 2 || !(Lx > 0) || !(Ly > 0) || max_markers < 1 || max_markers > 2000000000LL)
    return PYRO_E_INVALID;
  *out = nullptr;
  std::lock_guard<std::recursive_mutex> lk(pyro::device_sync_lock());
  pyro_markers_s* h = new (std::nothrow) pyro_markers_s;
  if (!h) return PYRO_E_NOMEM;
  h->nx = nx; h->ny = ny; h->Lx = Lx; h->Ly = Ly; h->cap = max_markers;
  cudaGetDevice(&h->dev);
  const size_t ncell = (size_t)(nx + 1) * (ny + 1);
  const size_t nb = (ncell + kScanBlock - 1) / kScanBlock + 1;
  bool ok = cudaMalloc(&h->count, ncell * sizeof(int)) == cudaSuccess &&
            cudaMalloc(&h->offset, (ncell + 1) * sizeof(int)) == cudaSuccess &&
            cudaMalloc(&h->fill, ncell * sizeof(int)) == cudaSuccess &&
            cudaMalloc(&h->bsum, nb * sizeof(int)) == cudaSuccess &&
            cudaMalloc(&h->idx, (size_t)max_markers * sizeof(int)) == cudaSuccess &&
            cudaMalloc(&h->cell, (size_t)max_markers * sizeof(int)) == cudaSuccess &&
            cudaMalloc(&h->frac, (size_t)max_markers * 2 * sizeof(double)) == cudaSuccess &&
            cudaMalloc(&h->csum, 8 * ncell * sizeof(double)) == cudaSuccess &&
            cudaMalloc(&h->flag, sizeof(int)) == cudaSuccess &&
            cudaMalloc(&h->red, 2 * kRedBlocks * sizeof(double)) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    pyro_markers_destroy(h);
    return PYRO_E_NOMEM;
  }
  *out = h;
  return PYRO_OK;
}

int pyro_markers_to_grid(pyro_markers h, int lattice, long long n, const double* xm, const double* ym,
                         const double* phim, double* grid, double* wsum, void* cuda_stream) {
  if (!h || n < 0 || n > h->cap || lattice < PYRO_LATTICE_NODES || lattice > PYRO_LATTICE_VY) return PYRO_E_INVALID;
  if (!grid || !on_device(grid) || (wsum && !on_device(wsum))) return PYRO_E_INVALID;
  if (n > 0 && (!on_device(xm) || !on_device(ym) || !on_device(phim))) return PYRO_E_INVALID;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  const Lat L = make_lat(h, lattice);
  const int ncell = L.ncx * L.ncy;
  const int nb = (ncell + kScanBlock - 1) / kScanBlock;
  cudaSetDevice(h->dev);
  cudaMemsetAsync(h->count, 0, (size_t)ncell * sizeof(int), s);
  cudaMemsetAsync(h->fill, 0, (size_t)ncell * sizeof(int), s);
  cudaMemsetAsync(h->flag, 0, sizeof(int), s);
  if (n > 0) k_mk_count<<<grid_blocks(n), kMkThreads, 0, s>>>(L, n, xm, ym, h->cell, h->frac, h->count, h->flag);
  k_scan_blocks<<<nb, kScanBlock, 0, s>>>(h->count, h->offset, ncell, h->bsum);
  k_scan_sums<<<1, 32, 0, s>>>(h->bsum, nb);
  k_scan_add<<<nb, kScanBlock, 0, s>>>(h->offset, ncell, h->bsum);
  if (n > 0) k_mk_scatter<<<grid_blocks(n), kMkThreads, 0, s>>>(n, h->cell, h->offset, h->fill, h->idx);
  k_mk_sort<<<(ncell + kMkThreads - 1) / kMkThreads, kMkThreads, 0, s>>>(ncell, h->offset, h->idx);
  // with n = 0 every cell is empty and phim is never read
  k_mk_cell_sums<<<(ncell + kMkThreads - 1) / kMkThreads, kMkThreads, 0, s>>>(ncell, h->offset, h->idx, h->frac,
                                                                              phim, h->csum);
  const dim3 b(32, 8), gr((L.jhi - L.jlo + 1 + 31) / 32, (L.ihi - L.ilo + 1 + 7) / 8);
  k_mk_node_sums<<<gr, b, 0, s>>>(L, h->nx + 2, h->csum, ncell, grid, wsum);
  int flag = 0;
  if (cudaMemcpyAsync(&flag, h->flag, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return PYRO_E_CUDA;
  if (cudaGetLastError() != cudaSuccess) return PYRO_E_CUDA;
  return (flag & FLAG_NONFINITE) ? PYRO_E_NONFINITE : PYRO_OK;
}

int pyro_grid_to_markers(pyro_markers h, int lattice, long long n, const double* xm, const double* ym,
                         const double* grid, double* phim, void* cuda_stream) {
  if (!h || n < 0 || lattice < PYRO_LATTICE_NODES || lattice > PYRO_LATTICE_VY) return PYRO_E_INVALID;
  if (n == 0) return PYRO_OK;
  if (!on_device(grid) || !on_device(xm) || !on_device(ym) || !on_device(phim)) return PYRO_E_INVALID;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  cudaSetDevice(h->dev);
  const Lat L = make_lat(h, lattice);
  k_mk_to_markers<<<grid_blocks(n), kMkThreads, 0, s>>>(L, h->nx + 2, n, xm, ym, grid, phim);
  if (cudaGetLastError() != cudaSuccess) return PYRO_E_CUDA;
  return PYRO_OK;
}

int pyro_markers_advect(pyro_markers h, int scheme, long long n, double* xm, double* ym, const double* vx,
                        const double* vy, double dt, int substeps, void* cuda_stream) {
  if (!h || n < 0 || scheme < PYRO_ADVECT_EULER || scheme > PYRO_ADVECT_TAYLOR || substeps < 1 || !isfinite(dt))
    return PYRO_E_INVALID;
  if (n == 0) return PYRO_OK;
  if (!on_device(xm) || !on_device(ym) || !on_device(vx) || !on_device(vy)) return PYRO_E_INVALID;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  cudaSetDevice(h->dev);
  const VelField F{make_lat(h, PYRO_LATTICE_VX), make_lat(h, PYRO_LATTICE_VY), h->nx + 2, vx, vy};
  const double step = dt / substeps;
  const int nb = grid_blocks(n);
  switch (scheme) {
    case PYRO_ADVECT_EULER:
      k_mk_advect<PYRO_ADVECT_EULER><<<nb, kMkThreads, 0, s>>>(F, n, xm, ym, step, substeps, h->Lx, h->Ly);
      break;
    case PYRO_ADVECT_HEUN:
      k_mk_advect<PYRO_ADVECT_HEUN><<<nb, kMkThreads, 0, s>>>(F, n, xm, ym, step, substeps, h->Lx, h->Ly);
      break;
    case PYRO_ADVECT_RK4:
      k_mk_advect<PYRO_ADVECT_RK4><<<nb, kMkThreads, 0, s>>>(F, n, xm, ym, step, substeps, h->Lx, h->Ly);
      break;
    default:
      k_mk_advect<PYRO_ADVECT_TAYLOR><<<nb, kMkThreads, 0, s>>>(F, n, xm, ym, step, substeps, h->Lx, h->Ly);
      break;
  }
  if (cudaGetLastError() != cudaSuccess) return PYRO_E_CUDA;
  return PYRO_OK;
}

int pyro_markers_max_dt(pyro_markers h, const double* vx, const double* vy, double cfl, double* dt_out,
                        void* cuda_stream) {
  if (!h || !dt_out || !(cfl > 0) || !isfinite(cfl) || !on_device(vx) || !on_device(vy)) return PYRO_E_INVALID;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  cudaSetDevice(h->dev);
  const size_t P = (size_t)(h->ny + 2) * (h->nx + 2);
  k_absmax2<<<kRedBlocks, kMkThreads, 0, s>>>(vx, vy, P, h->red);
  double r[2 * kRedBlocks];
  if (cudaMemcpyAsync(r, h->red, sizeof(r), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess || cudaGetLastError() != cudaSuccess)
    return PYRO_E_CUDA;
  double mx = 0.0, my = 0.0;
  for (int b = 0; b < kRedBlocks; ++b) {
    if (std::isnan(r[b]) || std::isnan(r[kRedBlocks + b])) return PYRO_E_NONFINITE;
    mx = std::max(mx, r[b]);
    my = std::max(my, r[kRedBlocks + b]);
  }
  if (!std::isfinite(mx) || !std::isfinite(my)) return PYRO_E_NONFINITE;
  const double tx = mx > 0.0 ? (h->Lx / h->nx) / mx : HUGE_VAL;
  const double ty = my > 0.0 ? (h->Ly / h->ny) / my : HUGE_VAL;
  *dt_out = cfl * std::min(tx, ty);
  return PYRO_OK;
}

void pyro_markers_destroy(pyro_markers h) {
  if (!h) return;
  std::lock_guard<std::recursive_mutex> lk(pyro::device_sync_lock());
  cudaFree(h->count); cudaFree(h->offset); cudaFree(h->fill); cudaFree(h->bsum);
  cudaFree(h->idx); cudaFree(h->cell); cudaFree(h->frac); cudaFree(h->csum); cudaFree(h->flag); cudaFree(h->red);
  delete h;
}

}  // extern "C"
