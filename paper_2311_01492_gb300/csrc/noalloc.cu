// Column density of one source with no device allocation at all.
//
// Some callers cannot allocate device memory when they call into the library:
// code that runs while a CUDA graph is being captured by someone else, host
// frameworks that reserve all device memory up front and forbid cudaMalloc
// later, or a real-time loop where an allocation's implicit synchronisation is
// not acceptable.  For them rt_coldens_single_noalloc computes the same column
// densities as rt_raytrace_source_coldens (bit for bit) using only the buffers
// the caller passes plus one fixed scratch array that lives in this file as a
// static __device__ array.  The paper has no counterpart of this entry point.
//
// The scratch is one cube of (2*RT_NOALLOC_MAX_HALF+1)^3 doubles (4.25 MB); the
// driver reserves it on every GPU that loads the library, until the process
// exits.  Every call shares it, so two calls that overlap on the GPU (different
// streams, or host threads racing) overwrite each other's scratch: serialise
// them.  Host code must not use the array's name as a device address (there it
// names a host-side shadow); the device address comes from
// cudaGetSymbolAddress, looked up once per device on the first call made with
// that device current.  Make that first call before any stream capture.
#include <cmath>
#include <mutex>

#include "asora_internal.cuh"

namespace asora {

#define RT_NOALLOC_MAX_HALF 40
#define RT_NOALLOC_SIDE (2 * RT_NOALLOC_MAX_HALF + 1)

static __device__ __align__(256) double g_noalloc_cube[(size_t)RT_NOALLOC_SIDE * RT_NOALLOC_SIDE *
                                                       RT_NOALLOC_SIDE];

__device__ __forceinline__ int na_sgn(int x) { return (x > 0) - (x < 0); }

__global__ void k_noalloc_zero(double* __restrict__ out, int64_t n) {
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < n;
       c += (int64_t)gridDim.x * blockDim.x)
    out[c] = 0.0;
}

// One CTA walks the octahedral shells S_q of the source (Sec. 3.3) exactly as
// the plain schedule does, with dtau, the weights and ds evaluated in place by
// the same correctly rounded expressions that build the library's tables.
__global__ void __launch_bounds__(256) k_noalloc_coldens(
    int n, int wlo, int whi, double sig_cell, double sigma0, const double* __restrict__ nH,
    const double* __restrict__ xHI, int si, int sj, int sk, int r2, int E,
    double* __restrict__ cube, double* __restrict__ out) {
  const int side = 2 * E + 1;
  auto cidx = [&](int x, int y, int z) {
    return ((size_t)(x + E) * side + (size_t)(y + E)) * side + (size_t)(z + E);
  };
  auto wrap = [&](int x) {
    x = x < 0 ? x + n : x;
    return x >= n ? x - n : x;
  };
  auto dtau_at = [&](int64_t c) { return (sig_cell * nH[c]) * xHI[c]; };
  const int64_t scell = ((int64_t)si * n + sj) * n + sk;
  const double dts = dtau_at(scell);
  int rr = (int)sqrtf((float)(3 * r2));
  while (rr * rr > 3 * r2) --rr;
  while ((rr + 1) * (rr + 1) <= 3 * r2) ++rr;
  const int Q = min(3 * E, rr);
  for (int q = 0; q <= Q; ++q) {
    const int cnt = q == 0 ? 1 : 4 * q * q + 2;
    for (int t = threadIdx.x; t < cnt; t += blockDim.x) {
      // cell t of S_q: top diamond (Dk >= 0) of radius q, then bottom diamond of radius q-1
      const int top = 2 * q * q + 2 * q + 1;
      int r, u;
      bool up;
      if (t < top) { r = q; u = t; up = true; } else { r = q - 1; u = t - top; up = false; }
      int a, b;
      if (u < (r + 1) * (r + 1)) {
        const int A = u / (r + 1);
        a = -r + 2 * A;
        b = -r + 2 * (u - A * (r + 1));
      } else {
        u -= (r + 1) * (r + 1);
        const int A = u / r;
        a = -r + 1 + 2 * A;
        b = -r + 1 + 2 * (u - A * r);
      }
      const int di = (a + b) / 2, dj = (a - b) / 2;
      const int h = q - abs(di) - abs(dj);
      const int dk = up ? h : -h;
      if (di < wlo || di > whi || dj < wlo || dj > whi || dk < wlo || dk > whi) continue;
      if (di * di + dj * dj + dk * dk > r2) continue;
      const int64_t cell = ((int64_t)wrap(si + di) * n + wrap(sj + dj)) * n + wrap(sk + dk);
      if (q == 0) {
        const double tout = 0.5 * dts;
        cube[cidx(0, 0, 0)] = tout;
        out[cell] = tout / sigma0;
        continue;
      }
      const int D[3] = {di, dj, dk};
      const int m = max(abs(di), max(abs(dj), abs(dk)));
      int ax, x1, x2;
      if (abs(dk) == m) { ax = 2; x1 = 0; x2 = 1; }
      else if (abs(dj) == m) { ax = 1; x1 = 0; x2 = 2; }
      else { ax = 0; x1 = 1; x2 = 2; }
      const int p1 = D[x1], p2 = D[x2];
      const double wa_ = (double)abs(p1) / (double)m;
      const double wb_ = (double)abs(p2) / (double)m;
      const double w1 = (1.0 - wa_) * (1.0 - wb_);
      const double w2 = wa_ * (1.0 - wb_);
      const double w3 = (1.0 - wa_) * wb_;
      const double w4 = wa_ * wb_;
      const double ds = sqrt(1.0 + (double)(p1 * p1 + p2 * p2) / (double)(m * m));
      double tin;
      if (m == 1) {
        tin = (0.5 * dts) * ds;
      } else {
        int e1[3] = {di, dj, dk};
        e1[ax] -= na_sgn(D[ax]);
        int e2[3] = {e1[0], e1[1], e1[2]};
        e2[x1] -= na_sgn(p1);
        int e3[3] = {e1[0], e1[1], e1[2]};
        e3[x2] -= na_sgn(p2);
        int e4[3] = {e2[0], e2[1], e2[2]};
        e4[x2] -= na_sgn(p2);
        const double c1 = cube[cidx(e1[0], e1[1], e1[2])];
        const double c2 = cube[cidx(e2[0], e2[1], e2[2])];
        const double c3 = cube[cidx(e3[0], e3[1], e3[2])];
        const double c4 = cube[cidx(e4[0], e4[1], e4[2])];
        tin = fma(w4, c4, fma(w3, c3, fma(w2, c2, w1 * c1)));
      }
      const double tout = fma(dtau_at(cell), ds, tin);
      cube[cidx(di, dj, dk)] = tout;
      out[cell] = tout / sigma0;
    }
    __syncthreads();  // shell q complete before shell q+1 reads it
  }
}

// Device address of the scratch, looked up once per device.
static std::mutex g_noalloc_mu;
static double* g_noalloc_addr[256];

static rt_status noalloc_scratch(double** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "rt_coldens_single_noalloc: cudaGetDevice");
  if (dev < 0 || dev >= 256) return fail(RT_ERR_INVALID, "rt_coldens_single_noalloc: device id");
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_cube);
    if (e != cudaSuccess)
      return cuda_fail(e, "rt_coldens_single_noalloc: cudaGetSymbolAddress");
    g_noalloc_addr[dev] = static_cast<double*>(p);
  }
  *out = g_noalloc_addr[dev];
  return RT_OK;
}

}  // namespace asora

using namespace asora;

extern "C" rt_status rt_coldens_single_noalloc(int n, double cell_cm, double sigma0_cm2,
                                               const double* d_nH, const double* d_xHI, int i,
                                               int j, int k, double radius, double* d_coldens,
                                               rt_stream_t s) {
  if (n < 1 || n > 4096 || !(cell_cm > 0) || !std::isfinite(cell_cm) || !(sigma0_cm2 > 0) ||
      !std::isfinite(sigma0_cm2))
    return fail(RT_ERR_INVALID, "rt_coldens_single_noalloc: need 1 <= n <= 4096, cell > 0, sigma0 > 0");
  if (!d_nH || !d_xHI || !d_coldens)
    return fail(RT_ERR_INVALID, "rt_coldens_single_noalloc: null pointer");
  if (i < 0 || i >= n || j < 0 || j >= n || k < 0 || k >= n)
    return fail(RT_ERR_INVALID, "rt_coldens_single_noalloc: source outside the box");
  if (!(radius > 0) || !std::isfinite(radius))
    return fail(RT_ERR_INVALID, "rt_coldens_single_noalloc: radius must be > 0");
  const int wlo = -(n / 2), whi = (n % 2 == 0) ? n / 2 - 1 : n / 2;
  const double cap = 3.0 * (double)(n / 2) * (double)(n / 2) + 1.0;
  const int r2 = (int)std::fmin(std::floor(radius * radius), cap);
  int rmax = (int)std::sqrt((double)r2);
  while ((int64_t)rmax * rmax > r2) --rmax;
  while ((int64_t)(rmax + 1) * (rmax + 1) <= r2) ++rmax;
  const int E = std::max(1, std::min(rmax, std::max(-wlo, whi)));
  if (E > RT_NOALLOC_MAX_HALF)
    return fail(RT_ERR_INVALID,
                "rt_coldens_single_noalloc: traced half-extent min(floor(R), n/2) = " +
                    std::to_string(E) + " exceeds the fixed scratch limit of " +
                    std::to_string(RT_NOALLOC_MAX_HALF) + " cells");
  double* cube = nullptr;
  rt_status st = noalloc_scratch(&cube);
  if (st != RT_OK) return st;
  cudaStream_t cs = (cudaStream_t)s;
  const int64_t ncell = (int64_t)n * n * n;
  k_noalloc_zero<<<(int)std::min<int64_t>((ncell + 255) / 256, 2048), 256, 0, cs>>>(d_coldens, ncell);
  count_launch();
  k_noalloc_coldens<<<1, 256, 0, cs>>>(n, wlo, whi, sigma0_cm2 * cell_cm, sigma0_cm2, d_nH, d_xHI,
                                       i, j, k, r2, E, cube, d_coldens);
  count_launch();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "rt_coldens_single_noalloc: launch");
  return RT_OK;
}
