// Host-side construction of the frequency-integrated transmission tables
// (arXiv 2311.01492, Eq. tables normalised by Eq. ngammalnu; Sec. 4.1.3 for
// the power-law cross section).  With x = nu/nu_th and theta = h nu_th/(k T):
//
//   g(tau) = int_1^inf B(x) exp(-tau x^-beta) dx / int_1^inf B(x) dx
//   h(tau) = int_1^inf B(x) x^-beta exp(-tau x^-beta) dx / int_1^inf B(x) dx
//   B(x)   = x^2 / (exp(theta x) - 1)   (blackbody photon number spectrum)
//
// Quadrature: double-exponential (tanh-sinh) rule on unit panels of x over
// [1, 1 + 740/theta]; the integrand beyond is below 1e-320 of its peak.
#include <cmath>
#include <thread>
#include <vector>

#include "../../include/asora.h"

namespace {

const double kPi = 3.14159265358979323846;

int nknots(int E0, int E1, int B) { return (E0 + E1) * (1 << B) + 2; }

double knot_tau(int idx, int E0, int E1, int B) {
  const int K = nknots(E0, E1, B);
  if (idx == 0) return 0.0;
  if (idx == K - 1) return std::ldexp(1.0, E1);
  const int t = idx - 1;
  return std::ldexp(1.0 + (double)(t & ((1 << B) - 1)) / (double)(1 << B), (t >> B) - E0);
}

}  // namespace

extern "C" int rt_table_nknots(int E0, int E1, int bits) {
  if (E0 < 1 || E1 < 1 || bits < 0 || bits > 12 || E0 + E1 > 2000) return -1;
  return nknots(E0, E1, bits);
}

extern "C" rt_status rt_table_blackbody(double T_bb, double beta, int E0, int E1, int bits,
                                        double* h_g, double* h_h) {
  if (!(T_bb > 0) || !std::isfinite(T_bb) || !(beta >= 0) || !std::isfinite(beta) || !h_g ||
      !h_h || rt_table_nknots(E0, E1, bits) < 0)
    return RT_ERR_INVALID;
  const double ev = 1.602176634e-12, kB = 1.380649e-16;
  const double theta = 13.6 * ev / (kB * T_bb);
  const double xmax = 1.0 + 740.0 / theta;
  const int npan = (int)std::ceil(xmax - 1.0);
  // tanh-sinh nodes on [-1, 1]: u = tanh(pi/2 sinh t), w = pi/2 cosh t / cosh^2(pi/2 sinh t)
  const double step = 1.0 / 64.0;
  const int kmax = (int)(4.0 / step);
  std::vector<double> xs, ws;
  xs.reserve((size_t)npan * (2 * kmax + 1));
  ws.reserve(xs.capacity());
  for (int p = 0; p < npan; ++p) {
    const double c = 1.0 + p + 0.5, hw = 0.5;
    for (int k = -kmax; k <= kmax; ++k) {
      const double t = k * step;
      const double sh = 0.5 * kPi * std::sinh(t);
      const double ch = std::cosh(sh);
      const double u = std::tanh(sh);
      const double w = step * 0.5 * kPi * std::cosh(t) / (ch * ch);
      if (w < 1e-300) continue;
      xs.push_back(c + hw * u);
      ws.push_back(hw * w);
    }
  }
  const size_t nn = xs.size();
  std::vector<double> sp(nn), bw(nn);
  double norm = 0.0;
  for (size_t i = 0; i < nn; ++i) {
    const double x = xs[i];
    const double y = theta * x;
    bw[i] = ws[i] * x * x * std::exp(-y) / -std::expm1(-y);
    sp[i] = std::pow(x, -beta);
    norm += bw[i];
  }
  const int K = nknots(E0, E1, bits);
  unsigned nth = std::thread::hardware_concurrency();
  nth = nth == 0 ? 1 : (nth > 16 ? 16 : nth);
  std::vector<std::thread> th;
  for (unsigned w = 0; w < nth; ++w) {
    th.emplace_back([&, w]() {
      for (int k = (int)w; k < K; k += (int)nth) {
        const double tau = knot_tau(k, E0, E1, bits);
        double sg = 0.0, sh = 0.0;
        for (size_t i = 0; i < nn; ++i) {
          const double e = std::exp(-tau * sp[i]);
          sg += bw[i] * e;
          sh += bw[i] * sp[i] * e;
        }
        h_g[k] = sg / norm;
        h_h[k] = sh / norm;
      }
    });
  }
  for (auto& t : th) t.join();
  return RT_OK;
}
