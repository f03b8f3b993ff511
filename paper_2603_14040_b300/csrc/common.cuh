// Shared device-side definitions of libpyro: grid geometry, staggered-field accessors and the
// point operators of the stress-conservative staggered discretisation.
//
// Layout: every field is a row-major (ny+2) x (nx+2) array with row stride ld = nx+2 (the
// paper's uniform padded staggered arrays, Sec. "Staggered Grid Layout"). Unknowns:
//   vx: i in [1,ny], j in [1,nx-1];  vy: i in [1,ny-1], j in [1,nx];  p: i in [1,ny], j in [1,nx].
// Walls (vx columns 0 and nx, vy rows 0 and ny) hold zero normal velocity. Tangential ghosts
// (vx rows 0 and ny+1, vy columns 0 and nx+1) are never read: the point operators substitute
// s * (adjacent interior value), which eliminates them exactly (free slip s=+1, no slip and
// prescribed velocity s=-1; the constant part of a prescribed velocity lives in the RHS).
#pragma once
#include <cuda_runtime.h>
#include <cstdint>
#include <mutex>

namespace pyro {

// Host side. A device-wide synchronisation (cudaDeviceSynchronize, cudaFree) issued while any
// stream of the device is being captured into a graph is invalid and ends that capture, so the
// calls that do either, and may run on different host threads, serialise on this lock: handle
// creation and destruction, and the one-time capture of the iteration graph.
inline std::recursive_mutex& device_sync_lock() {
  static std::recursive_mutex m;
  return m;
}

// Host side. Where a caller's pointer lives, seen from the current device:
//   PTR_HOST   host memory (pageable or pinned): staged through device buffers;
//   PTR_HERE   device memory of the current device, or managed memory: read / written in place;
//   PTR_OTHER  device memory of another GPU, or a null / unreadable pointer: rejected
//              (PYRO_E_INVALID), since a kernel here would read peer memory or fault.
enum PtrPlace { PTR_OTHER = -1, PTR_HOST = 0, PTR_HERE = 1 };
inline PtrPlace ptr_place(const void* p) {
  if (!p) return PTR_OTHER;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return PTR_OTHER;
  }
  if (a.type == cudaMemoryTypeManaged) return PTR_HERE;
  if (a.type == cudaMemoryTypeDevice) {
    int cur = -1;
    if (cudaGetDevice(&cur) != cudaSuccess) {
      cudaGetLastError();
      return PTR_OTHER;
    }
    return a.device == cur ? PTR_HERE : PTR_OTHER;
  }
  return PTR_HOST;
}

struct Geom {
  int nx, ny;      // cell counts
  int ld;          // row stride (nx + 2)
  double dx, dy;   // cell sizes
  double sN, sS, sW, sE;  // tangential ghost factors
};

template <typename T>
struct GeomT {
  int nx, ny, ld;
  T idx2, idy2, idxdy;  // 1/dx^2, 1/dy^2, 1/(dx dy)
  T idx, idy;           // 1/dx, 1/dy
  T sN, sS, sW, sE;
};

template <typename T>
__host__ __device__ inline GeomT<T> geomT(const Geom& g) {
  GeomT<T> t;
  t.nx = g.nx; t.ny = g.ny; t.ld = g.ld;
  t.idx2 = (T)(1.0 / (g.dx * g.dx));
  t.idy2 = (T)(1.0 / (g.dy * g.dy));
  t.idxdy = (T)(1.0 / (g.dx * g.dy));
  t.idx = (T)(1.0 / g.dx);
  t.idy = (T)(1.0 / g.dy);
  t.sN = (T)g.sN; t.sS = (T)g.sS; t.sW = (T)g.sW; t.sE = (T)g.sE;
  return t;
}

__host__ __device__ inline bool is_vx(int nx, int ny, int i, int j) { return i >= 1 && i <= ny && j >= 1 && j <= nx - 1; }
__host__ __device__ inline bool is_vy(int nx, int ny, int i, int j) { return i >= 1 && i <= ny - 1 && j >= 1 && j <= nx; }
__host__ __device__ inline bool is_p(int nx, int ny, int i, int j) { return i >= 1 && i <= ny && j >= 1 && j <= nx; }

// Row and column of entry e of a row-major array with `cols` columns. A 32-bit division when e fits
// in 32 bits (every grid a device can hold), instead of the much longer 64-bit division sequence.
__device__ __forceinline__ void row_col(size_t e, int cols, int& i, int& j) {
  if (e <= 0xffffffffull) {
    const unsigned u = (unsigned)e, c = (unsigned)cols, q = u / c;
    i = (int)q;
    j = (int)(u - q * c);
  } else {
    i = (int)(e / (size_t)cols);
    j = (int)(e % (size_t)cols);
  }
}

// vx value with walls masked (used where a reference may land on a wall column)
template <typename T, typename S>
__device__ inline T ldvx(const S* vx, int ld, int nx, int i, int j) {
  return (j <= 0 || j >= nx) ? T(0) : (T)vx[(size_t)i * ld + j];
}
template <typename T, typename S>
__device__ inline T ldvy(const S* vy, int ld, int ny, int i, int j) {
  return (i <= 0 || i >= ny) ? T(0) : (T)vy[(size_t)i * ld + j];
}

// x-momentum velocity part at the vx unknown (i, j):
//   (sxx(i,j+1) - sxx(i,j))/dx + (sxy(i,j) - sxy(i-1,j))/dy
// with sxx = 2 eta_c d vx/dx at cells and sxy = eta_n (d vx/dy + d vy/dx) at basic nodes.
// Returns the value and the diagonal coefficient (boundary elimination included).
// The _at form reads every array at c + offset with row stride ld (a copy of part of the grid,
// e.g. a shared-memory tile); (i, j) stay global indices for the boundary rules.
template <typename T, typename SV, typename SE>
__device__ inline T lx_point_at(const GeomT<T>& g, int i, int j, size_t c, int ld, const SV* vx, const SV* vy,
                                const SE* en, const SE* ec, T& diag) {
  const T eA = (T)ec[c], eB = (T)ec[c + 1];       // cells west / east of vx(i,j)
  const T e1 = (T)en[c - ld], e2 = (T)en[c];       // nodes above / below
  const T vc = (T)vx[c];
  const T vw = (j - 1 <= 0) ? T(0) : (T)vx[c - 1];
  const T ve = (j + 1 >= g.nx) ? T(0) : (T)vx[c + 1];
  const T vn = (i == 1) ? g.sN * vc : (T)vx[c - ld];
  const T vs = (i == g.ny) ? g.sS * vc : (T)vx[c + ld];
  const bool rn = i - 1 <= 0 || i - 1 >= g.ny, r0 = i <= 0 || i >= g.ny;
  const T yA = rn ? T(0) : (T)vy[c - ld], yB = rn ? T(0) : (T)vy[c - ld + 1];
  const T yC = r0 ? T(0) : (T)vy[c], yD = r0 ? T(0) : (T)vy[c + 1];
  const T sxxE = T(2) * eB * (ve - vc);
  const T sxxW = T(2) * eA * (vc - vw);
  const T sxyS = e2 * ((vs - vc) * g.idy2 + (yD - yC) * g.idxdy);
  const T sxyN = e1 * ((vc - vn) * g.idy2 + (yB - yA) * g.idxdy);
  diag = -T(2) * (eA + eB) * g.idx2 - (e1 + e2) * g.idy2;
  if (i == 1) diag += g.sN * e1 * g.idy2;
  if (i == g.ny) diag += g.sS * e2 * g.idy2;
  return (sxxE - sxxW) * g.idx2 + sxyS - sxyN;
}
template <typename T, typename SV, typename SE>
__device__ inline T lx_point(const GeomT<T>& g, int i, int j, const SV* vx, const SV* vy,
                             const SE* en, const SE* ec, T& diag) {
  return lx_point_at<T>(g, i, j, (size_t)i * g.ld + j, g.ld, vx, vy, en, ec, diag);
}

// y-momentum velocity part at the vy unknown (i, j):
//   (syy(i+1,j) - syy(i,j))/dy + (sxy(i,j) - sxy(i,j-1))/dx
template <typename T, typename SV, typename SE>
__device__ inline T ly_point_at(const GeomT<T>& g, int i, int j, size_t c, int ld, const SV* vx, const SV* vy,
                                const SE* en, const SE* ec, T& diag) {
  const T eA = (T)ec[c], eB = (T)ec[c + ld];      // cells above / below vy(i,j)
  const T e1 = (T)en[c - 1], e2 = (T)en[c];        // nodes west / east
  const T vc = (T)vy[c];
  const T vn = (i - 1 <= 0) ? T(0) : (T)vy[c - ld];
  const T vs = (i + 1 >= g.ny) ? T(0) : (T)vy[c + ld];
  const T vw = (j == 1) ? g.sW * vc : (T)vy[c - 1];
  const T ve = (j == g.nx) ? g.sE * vc : (T)vy[c + 1];
  const bool cw = j - 1 <= 0 || j - 1 >= g.nx, c0 = j <= 0 || j >= g.nx;
  const T xA = cw ? T(0) : (T)vx[c - 1], xB = cw ? T(0) : (T)vx[c + ld - 1];
  const T xC = c0 ? T(0) : (T)vx[c], xD = c0 ? T(0) : (T)vx[c + ld];
  const T syyS = T(2) * eB * (vs - vc);
  const T syyN = T(2) * eA * (vc - vn);
  const T sxyE = e2 * ((ve - vc) * g.idx2 + (xD - xC) * g.idxdy);
  const T sxyW = e1 * ((vc - vw) * g.idx2 + (xB - xA) * g.idxdy);
  diag = -T(2) * (eA + eB) * g.idy2 - (e1 + e2) * g.idx2;
  if (j == 1) diag += g.sW * e1 * g.idx2;
  if (j == g.nx) diag += g.sE * e2 * g.idx2;
  return (syyS - syyN) * g.idy2 + sxyE - sxyW;
}
template <typename T, typename SV, typename SE>
__device__ inline T ly_point(const GeomT<T>& g, int i, int j, const SV* vx, const SV* vy,
                             const SE* en, const SE* ec, T& diag) {
  return ly_point_at<T>(g, i, j, (size_t)i * g.ld + j, g.ld, vx, vy, en, ec, diag);
}

// Precomputed viscosity coefficients of one level (FP64 levels whose smoothing is ALU-bound):
// cxx = 2 eta_c/dx^2, cyy = 2 eta_c/dy^2 at cells; nxx = eta_n/dx^2, nyy = eta_n/dy^2,
// nxy = eta_n/(dx dy) at basic nodes. A null cxx means "use eta directly".
template <typename T>
struct Coef {
  const T *cxx, *cyy, *nxx, *nyy, *nxy;
};

// lx_point with precomputed coefficients: the same stress differences, about half the multiplies.
template <typename T, typename SV>
__device__ inline T lx_coef(const GeomT<T>& g, int i, int j, const SV* vx, const SV* vy, const Coef<T>& k) {
  const int ld = g.ld;
  const size_t c = (size_t)i * ld + j;
  const T vc = (T)vx[c];
  const T vw = ldvx<T>(vx, ld, g.nx, i, j - 1);
  const T ve = ldvx<T>(vx, ld, g.nx, i, j + 1);
  const T vn = (i == 1) ? g.sN * vc : (T)vx[c - ld];
  const T vs = (i == g.ny) ? g.sS * vc : (T)vx[c + ld];
  const T yA = ldvy<T>(vy, ld, g.ny, i - 1, j), yB = ldvy<T>(vy, ld, g.ny, i - 1, j + 1);
  const T yC = ldvy<T>(vy, ld, g.ny, i, j), yD = ldvy<T>(vy, ld, g.ny, i, j + 1);
  return k.cxx[c + 1] * (ve - vc) - k.cxx[c] * (vc - vw) + k.nyy[c] * (vs - vc) + k.nxy[c] * (yD - yC) -
         k.nyy[c - ld] * (vc - vn) - k.nxy[c - ld] * (yB - yA);
}

template <typename T, typename SV>
__device__ inline T ly_coef(const GeomT<T>& g, int i, int j, const SV* vx, const SV* vy, const Coef<T>& k) {
  const int ld = g.ld;
  const size_t c = (size_t)i * ld + j;
  const T vc = (T)vy[c];
  const T vn = ldvy<T>(vy, ld, g.ny, i - 1, j);
  const T vs = ldvy<T>(vy, ld, g.ny, i + 1, j);
  const T vw = (j == 1) ? g.sW * vc : (T)vy[c - 1];
  const T ve = (j == g.nx) ? g.sE * vc : (T)vy[c + 1];
  const T xA = ldvx<T>(vx, ld, g.nx, i, j - 1), xB = ldvx<T>(vx, ld, g.nx, i + 1, j - 1);
  const T xC = ldvx<T>(vx, ld, g.nx, i, j), xD = ldvx<T>(vx, ld, g.nx, i + 1, j);
  return k.cyy[c + ld] * (vs - vc) - k.cyy[c] * (vc - vn) + k.nxx[c] * (ve - vc) + k.nxy[c] * (xD - xC) -
         k.nxx[c - 1] * (vc - vw) - k.nxy[c - 1] * (xB - xA);
}

// Off-diagonal part of the velocity rows with precomputed coefficients: L v = off + diag v_c,
// where the ghost-eliminated neighbour (vn at i = 1, vs at i = ny for vx; vw at j = 1, ve at
// j = nx for vy) belongs to the diagonal and is left out here. With 1/diag the damped
// Gauss-Seidel update is v <- (1 - omega) v + omega (f - off) / diag: about a third fewer FP64
// operations than forming L v in full.
template <typename T, typename SV>
__device__ inline T lx_off(const GeomT<T>& g, int i, int j, const SV* vx, const SV* vy, const Coef<T>& k) {
  const int ld = g.ld;
  const size_t c = (size_t)i * ld + j;
  const T vw = ldvx<T>(vx, ld, g.nx, i, j - 1);
  const T ve = ldvx<T>(vx, ld, g.nx, i, j + 1);
  const T yA = ldvy<T>(vy, ld, g.ny, i - 1, j), yB = ldvy<T>(vy, ld, g.ny, i - 1, j + 1);
  const T yC = ldvy<T>(vy, ld, g.ny, i, j), yD = ldvy<T>(vy, ld, g.ny, i, j + 1);
  T s = k.cxx[c + 1] * ve + k.cxx[c] * vw + k.nxy[c] * (yD - yC) - k.nxy[c - ld] * (yB - yA);
  if (i != 1) s += k.nyy[c - ld] * (T)vx[c - ld];
  if (i != g.ny) s += k.nyy[c] * (T)vx[c + ld];
  return s;
}

template <typename T, typename SV>
__device__ inline T ly_off(const GeomT<T>& g, int i, int j, const SV* vx, const SV* vy, const Coef<T>& k) {
  const int ld = g.ld;
  const size_t c = (size_t)i * ld + j;
  const T vn = ldvy<T>(vy, ld, g.ny, i - 1, j);
  const T vs = ldvy<T>(vy, ld, g.ny, i + 1, j);
  const T xA = ldvx<T>(vx, ld, g.nx, i, j - 1), xB = ldvx<T>(vx, ld, g.nx, i + 1, j - 1);
  const T xC = ldvx<T>(vx, ld, g.nx, i, j), xD = ldvx<T>(vx, ld, g.nx, i + 1, j);
  T s = k.cyy[c + ld] * vs + k.cyy[c] * vn + k.nxy[c] * (xD - xC) - k.nxy[c - 1] * (xB - xA);
  if (j != 1) s += k.nxx[c - 1] * (T)vy[c - 1];
  if (j != g.nx) s += k.nxx[c] * (T)vy[c + 1];
  return s;
}

// Error flags written by kernels (host reads them after a sync).
enum : int { FLAG_NONFINITE = 1, FLAG_BREAKDOWN = 2 };

constexpr int kReduceBlocks = 592;  // 4 x 148 SMs: fixed so reductions are deterministic
constexpr int kThreads = 256;
constexpr int kMaxRestart = 256;               // longest FGMRES cycle (Krylov basis length)
constexpr int kHcolStride = kMaxRestart + 2;   // stride of the Hessenberg columns on the device

}  // namespace pyro
