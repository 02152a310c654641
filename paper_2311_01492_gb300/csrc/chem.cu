// Chemistry step (arXiv 2311.01492, Sec. 2.1, Eq. time_avrg_sol) and the small
// kernels of the ray-tracing <-> chemistry iteration (Fig. 1).
//
// Per cell, with Gamma, n_e, C_H, alpha_H held constant over dt, the analytic
// solution of Eq. chemistry is x(t) = x_eq + (x0 - x_eq) exp(-t/t_i) with
//   1/t_i = Gamma + n_e (C_H + alpha_H),  x_eq = (Gamma + n_e C_H) t_i,
// and its time average over dt is x_eq + (x0 - x_eq)(1 - exp(-dt/t_i)) t_i/dt.
// n_e = n_H <x_HII> is iterated to convergence; n_H is the proper density (the
// given one times inv_a3 = a^-3 in an expanding background, an exact no-op for
// a = 1).  Built with --fmad=false so the expressions round exactly as written.
#include "asora_internal.cuh"

namespace asora {

__global__ void k_chemistry(int64_t n, const double* __restrict__ nH, double inv_a3,
                            const double* __restrict__ gamma, const double* __restrict__ x0,
                            const double* __restrict__ xavg_in, double dt, double alpha_H,
                            double C_H, double tol, int maxit, double conv_tol,
                            double* __restrict__ xavg_out, double* __restrict__ xnew_out,
                            unsigned long long* __restrict__ unconv, const int* __restrict__ skip) {
  if (skip && *skip) return;
  unsigned cnt = 0;
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < n;
       c += (int64_t)gridDim.x * blockDim.x) {
    const double G = gamma[c];
    const double xs = x0[c];
    const double nh = nH[c] * inv_a3;
    const double xin = xavg_in[c];
    double xa = xin;
    // x(t + dt) of the last pass only: its equilibrium value and y (rate <= 0: x0)
    double xeq_last = xs, y_last = 0.0;
    bool decays = false;
    for (int it = 0; it < maxit; ++it) {
      const double ne = nh * xa;
      const double rate = G + ne * (C_H + alpha_H);
      double xa_new;
      decays = rate > 0.0;
      if (decays) {
        const double xeq = (G + ne * C_H) / rate;
        const double y = dt * rate;
        xa_new = xeq + (xs - xeq) * (-expm1(-y) / y);
        xeq_last = xeq;
        y_last = y;
      } else {
        xa_new = xs;
      }
      const bool done = fabs(xa_new - xa) <= tol * xa_new;
      xa = xa_new;
      if (done) break;
    }
    const double xnew = decays ? xeq_last + (xs - xeq_last) * exp(-y_last) : xs;
    xavg_out[c] = xa;
    xnew_out[c] = xnew;
    const double xhi_old = 1.0 - xin, xhi_new = 1.0 - xa;
    if (fabs(xhi_new - xhi_old) > conv_tol * xhi_new) ++cnt;
  }
  // warp-aggregated count
  for (int o = 16; o > 0; o >>= 1) cnt += __shfl_down_sync(0xffffffffu, cnt, o);
  if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(unconv, (unsigned long long)cnt);
}

cudaError_t launch_chemistry(Grid& g, const double* gamma, const double* x0, const double* xavg_in,
                             double dt, double alpha_H, double C_H, double tol, int maxit,
                             double conv_tol, double* xavg_out, double* xnew_out, int64_t* unconv,
                             const int* skip_flag) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t want = (g.ncell + 255) / 256;
  const int grid = (int)std::min<int64_t>(want, (int64_t)sms * 8);
  k_chemistry<<<grid, 256, 0, g.stream>>>(g.ncell, g.nH, g.inv_a3, gamma, x0, xavg_in, dt, alpha_H, C_H, tol,
                                          maxit, conv_tol, xavg_out, xnew_out,
                                          reinterpret_cast<unsigned long long*>(unconv), skip_flag);
  count_launch();
  return cudaGetLastError();
}

__global__ void k_one_minus(const double* __restrict__ x, double* __restrict__ y, int64_t n,
                            const int* __restrict__ skip) {
  if (skip && *skip) return;
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < n;
       c += (int64_t)gridDim.x * blockDim.x)
    y[c] = 1.0 - x[c];
}

cudaError_t launch_one_minus(const double* x, double* y, int64_t n, const int* skip_flag,
                             cudaStream_t s) {
  const int grid = (int)std::min<int64_t>((n + 255) / 256, 152 * 8);
  k_one_minus<<<grid, 256, 0, s>>>(x, y, n, skip_flag);
  count_launch();
  return cudaGetLastError();
}

// flags[0]: converged, flags[1]: iterations run.
__global__ void k_conv_check(const int64_t* __restrict__ unconv, int64_t limit,
                             int* __restrict__ flags) {
  if (flags[0]) return;
  flags[1] += 1;
  if (unconv[0] < limit) flags[0] = 1;
}

cudaError_t launch_conv_check(const int64_t* unconv, int64_t limit, int* flags, cudaStream_t s) {
  k_conv_check<<<1, 1, 0, s>>>(unconv, limit, flags);
  count_launch();
  return cudaGetLastError();
}

}  // namespace asora
