// ---------------------------------------------------------------------------
// ASORA / pyC2Ray hot path -- plain, slow, FP64 CPU ORACLE.
//
// THIS FILE IS TEST INFRASTRUCTURE.  Only tests/, the smoke check in
// __graft_entry__.py and the CPU-baseline leg of bench.py may load it.  The
// CUDA library never links, includes or calls it, and it shares no code with
// the CUDA library (each side writes out the same definitions independently).
//
// What it computes, step by step, in the paper's order and notation
// (arXiv 2311.01492, "pyC2Ray"):
//
//  * Per-cell optical depth at the H I threshold  dtau = sigma0 * alpha * n_HI,
//    n_HI = n_H * x_HI   (Sec. 3.1: Delta N_HI = n_HI alpha ds, tau = sigma N).
//    Evaluated as ((sigma0*alpha)*n_H)*x_HI, left to right.
//  * Short characteristics (Sec. 3.1, Eqs. raga/interp): for a voxel p with
//    offset Delta = p - s from the source, the dominant axis d is the one with
//    the largest |Delta| (ties: k before j before i).  The two other axes, in
//    increasing axis order, are p1 and p2; a = |Delta_p1|/|Delta_d|,
//    b = |Delta_p2|/|Delta_d|.  The four interpolants lie in the entry plane
//    (one step towards the source along d):
//       e1 = p - sd*e_d,  e2 = e1 - s1*e_p1,  e3 = e1 - s2*e_p2,
//       e4 = e1 - s1*e_p1 - s2*e_p2,     s = sign(), sign(0) = 0
//    with bilinear weights w1=(1-a)(1-b), w2=a(1-b), w3=(1-a)b, w4=ab, which
//    make the scheme exact on axes and grid diagonals (Sec. 3.1, last
//    paragraph).  tau_in = fma(w4,c4, fma(w3,c3, fma(w2,c2, w1*c1))).
//    Path length ds = sqrt(1 + (Delta_p1^2 + Delta_p2^2)/Delta_d^2)  (Sec. 3.1).
//    Optional optical-depth-modulated weights (interp_mode 1; the C2Ray paper's
//    App. A, which Sec. 3.1 cites for the weighting but does not print): each
//    weight is multiplied by m_n = 1/max(tau_n, tau_w0), tau_n the optical depth
//    at threshold out of interpolant n, and the sum is normalised:
//    w'_n = w_n*m_n, S = ((w'_1+w'_2)+w'_3)+w'_4,
//    tau_in = fma(w'4,c4, fma(w'3,c3, fma(w'2,c2, w'1*c1))) / S.  The default
//    (interp_mode 0) is the paper's geometric weighting.
//    tau_out = fma(dtau(p), ds, tau_in).
//    Source voxel (q = 0, "treated directly", Sec. 3.3): tau_in = 0,
//    tau_out = dtau(s)/2.  Voxels with max|Delta| = 1 (their only non-zero
//    weight interpolant is the source) take tau_in = (dtau(s)/2)*ds, the
//    column from the source centre to their entry face.
//  * ASORA traversal (Sec. 3.3, Fig. octa): octahedral shells
//    S_q = {|Di|+|Dj|+|Dk| = q}, q = 0..Q, processed in order; cells of one
//    shell are independent.  Q = ceil(sqrt(3) R) and cells with
//    |Delta|^2 > floor(R^2) are skipped (radius cut, Sec. 3.3).
//    Periodic window (App. A): Delta in [-N/2, N/2-1] for even N,
//    [-(N-1)/2, (N-1)/2] for odd N, so no two kept cells alias.
//  * Photo-ionisation rate (Sec. 2.2, Eqs. gamma, tables, sugg):
//      thick:  dG = Ndot [g(tau_in) - g(tau_out)] / (n_HI V),
//              V = 4 pi r^2 alpha ds  (r = alpha |Delta|),  V = alpha^3 at q = 0
//      thin (dtau*ds <= tau_lim, the Delta tau -> 0 limit, Eq. gammalocal):
//              dG = Ndot sigma0 h(tau_in) / (4 pi r^2),
//              source cell: Ndot sigma0 h(0) / (2 alpha^2)
//    g(tau) = gamma(N_HI)/Ndot is the frequency-integrated transmitted photon
//    fraction, h = -dg/dtau.  Rates add over sources (Sec. 2.2, last para).
//  * Tables (Eq. tables): knot values are evaluated by quadrature at
//    tau = 0, 2^e (1 + m/2^B) for e = -E0..E1-1, m = 0..2^B-1, and 2^E1.
//    Segment index from the IEEE bits of tau (exponent e, top B mantissa
//    bits m): 1 + (e+E0) 2^B + m; tau < 2^-E0 uses segment 0 = [0, 2^-E0];
//    tau >= 2^E1 gives 0.  Within a segment the value is the chord
//    c0 + c1 tau with c1 = (g_hi-g_lo)/(tau_hi-tau_lo),
//    c0 = fma(-c1, tau_lo, g_lo), evaluated as fma(c1, tau, c0).
//  * Chemistry (Sec. 2.1, Eq. time_avrg_sol): time-averaged analytic
//    solution with n_e = n_H <x_HII> iterated until converged.
//
// Build: g++ -O2 -ffp-contract=off -fopenmp -shared -fPIC (oracle/build.py).
// Contraction is off so that every fma is the explicit one written here.
// ---------------------------------------------------------------------------
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdint>
#include <cstring>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

typedef std::complex<double> cplx;

inline double re(double x) { return x; }
inline double re(const cplx& x) { return x.real(); }
inline double fmaT(double a, double b, double c) { return std::fma(a, b, c); }
inline cplx fmaT(double a, const cplx& b, const cplx& c) { return a * b + c; }
inline cplx fmaT(const cplx& a, const cplx& b, const cplx& c) { return a * b + c; }
inline double expT(double x) { return std::exp(x); }
inline cplx expT(const cplx& x) { return std::exp(x); }

const double kPi = 3.14159265358979323846;

inline int sgn(int x) { return (x > 0) - (x < 0); }

// ----------------------------------------------------------------- tables
struct Table {
  int kind = 0;  // 0: chords from knots, 1: analytic grey g = h = exp(-tau)
  int E0 = 0, E1 = 0, B = 0;
  double tau_min = 0, tau_max = 0;
  std::vector<double> gc0, gc1, hc0, hc1;
};

inline int n_knots(int E0, int E1, int B) { return (E0 + E1) * (1 << B) + 2; }

// tau of knot idx, idx in [0, n_knots)
double knot_tau(int idx, int E0, int E1, int B) {
  const int K = n_knots(E0, E1, B);
  if (idx == 0) return 0.0;
  if (idx == K - 1) return std::ldexp(1.0, E1);
  const int t = idx - 1;
  const int e = (t >> B) - E0;
  const int m = t & ((1 << B) - 1);
  return std::ldexp(1.0 + (double)m / (double)(1 << B), e);
}

void chords(const double* knots, int E0, int E1, int B, std::vector<double>& c0,
            std::vector<double>& c1) {
  const int S = n_knots(E0, E1, B) - 1;
  c0.resize(S);
  c1.resize(S);
  for (int s = 0; s < S; ++s) {
    const double tl = knot_tau(s, E0, E1, B), th = knot_tau(s + 1, E0, E1, B);
    c1[s] = (knots[s + 1] - knots[s]) / (th - tl);
    c0[s] = std::fma(-c1[s], tl, knots[s]);
  }
}

template <class T>
T tab_eval(const Table& t, const std::vector<double>& c0, const std::vector<double>& c1,
           const T& tau) {
  if (t.kind == 1) return expT(-tau);
  const double x = re(tau);
  if (!(x < t.tau_max)) return T(0.0);
  int seg;
  if (x < t.tau_min) {
    seg = 0;
  } else {
    uint64_t bits;
    std::memcpy(&bits, &x, 8);
    const int e = (int)((bits >> 52) & 0x7FF) - 1023;
    const int m = (int)((bits >> (52 - t.B)) & (uint64_t)((1 << t.B) - 1));
    seg = 1 + (e + t.E0) * (1 << t.B) + m;
  }
  return fmaT(c1[seg], tau, T(c0[seg]));
}

// -------------------------------------------------------------- parameters
struct Params {
  int n;
  double cell_cm;
  double sigma0;
  double tau_lim;
  int interp = 0;        // 0: geometric weights; 1: optical-depth-modulated weights
  double tau_w0 = 0.6;   // floor of tau_n in the modulation 1/max(tau_n, tau_w0)
};

inline int wrap(int x, int n) {
  x %= n;
  return x < 0 ? x + n : x;
}

// Enumerate the octahedral shell S_q in a fixed order: Di ascending, Dj
// ascending, Dk = +r then -r.  |S_q| = 4q^2 + 2 for q > 0 (Sec. 3.3).
template <class F>
void for_each_in_shell(int q, F&& f) {
  for (int di = -q; di <= q; ++di) {
    const int rem = q - std::abs(di);
    for (int dj = -rem; dj <= rem; ++dj) {
      const int r = rem - std::abs(dj);
      f(di, dj, r);
      if (r != 0) f(di, dj, -r);
    }
  }
}

// Field accessors: dtau and n_HI of cell g, optionally with a complex-step
// perturbation (log n_HI of one cell shifted by i*h).
template <class T>
struct Fields {
  const double* dtau;
  const double* nhi;
  int64_t pert_cell = -1;
  double h = 0.0;
  T dt(int64_t g) const;
  T nh(int64_t g) const;
};
template <>
double Fields<double>::dt(int64_t g) const { return dtau[g]; }
template <>
double Fields<double>::nh(int64_t g) const { return nhi[g]; }
template <>
cplx Fields<cplx>::dt(int64_t g) const {
  return g == pert_cell ? cplx(dtau[g], dtau[g] * h) : cplx(dtau[g], 0.0);
}
template <>
cplx Fields<cplx>::nh(int64_t g) const {
  return g == pert_cell ? cplx(nhi[g], nhi[g] * h) : cplx(nhi[g], 0.0);
}

struct Out {
  // any of these may be null
  void* gamma = nullptr;          // T[N^3], accumulated
  double* coldens = nullptr;      // double[N^3], column density out of each cell (cm^-2)
  double* tau_in = nullptr;       // double[N^3], tau up to each cell
  const double* wloss = nullptr;  // double[N^3], loss weights
  void* loss = nullptr;           // T*, accumulated sum_p w_p dG_p
  bool debug = false;             // NaN-fill the scratch to detect acausal reads
  int err = 0;                    // set to 1 if an interpolant was not yet computed
};

// One source: octahedral shells q = 0..Q in order (Sec. 3.3).
template <class T>
void trace_one(const Params& P, const Table& tab, const Fields<T>& F, int is, int js, int ks,
               T ndot, double R, Out& o) {
  const int N = P.n;
  const int wlo = -(N / 2);
  const int whi = (N % 2 == 0) ? N / 2 - 1 : N / 2;
  const int64_t R2 = (int64_t)std::floor(R * R);
  const int E = std::min((int)std::floor(R), N / 2);
  const int side = 2 * E + 1;
  std::vector<T> tout((size_t)side * side * side, o.debug ? T(NAN) : T(0.0));
  auto cidx = [&](int a, int b, int c) {
    return ((size_t)(a + E) * side + (size_t)(b + E)) * side + (size_t)(c + E);
  };
  auto gidx = [&](int a, int b, int c) {
    return ((int64_t)wrap(is + a, N) * N + wrap(js + b, N)) * N + wrap(ks + c, N);
  };
  T* gamma = (T*)o.gamma;
  T* loss = (T*)o.loss;
  const double alpha = P.cell_cm;
  const double sigma0 = P.sigma0;
  const int Q = (int)std::ceil(std::sqrt(3.0) * R);
  const int64_t gs = gidx(0, 0, 0);
  const T dts = F.dt(gs);

  auto deposit = [&](int64_t g, const T& dG) {
    if (gamma) gamma[g] += dG;
    if (loss && o.wloss) *loss += o.wloss[g] * dG;
  };

  for (int q = 0; q <= Q; ++q) {
    for_each_in_shell(q, [&](int di, int dj, int dk) {
      if (di < wlo || di > whi || dj < wlo || dj > whi || dk < wlo || dk > whi) return;
      const int64_t d2 = (int64_t)di * di + (int64_t)dj * dj + (int64_t)dk * dk;
      if (d2 > R2) return;
      const int64_t g = gidx(di, dj, dk);
      if (q == 0) {
        // source cell: no interpolation
        const T t_out = 0.5 * dts;
        tout[cidx(0, 0, 0)] = t_out;
        if (o.coldens) o.coldens[g] = re(t_out) / sigma0;
        if (o.tau_in) o.tau_in[g] = 0.0;
        T dG;
        if (re(t_out) <= P.tau_lim) {
          dG = ndot * sigma0 * tab_eval(tab, tab.hc0, tab.hc1, T(0.0)) / (2.0 * alpha * alpha);
        } else {
          dG = ndot * (tab_eval(tab, tab.gc0, tab.gc1, T(0.0)) - tab_eval(tab, tab.gc0, tab.gc1, t_out)) /
               (F.nh(g) * (alpha * alpha * alpha));
        }
        deposit(g, dG);
        return;
      }
      const int adi = std::abs(di), adj = std::abs(dj), adk = std::abs(dk);
      const int m = std::max(adi, std::max(adj, adk));
      int D[3] = {di, dj, dk};
      int ax, x1, x2;  // dominant axis and the two others in increasing order
      if (adk == m) {
        ax = 2; x1 = 0; x2 = 1;
      } else if (adj == m) {
        ax = 1; x1 = 0; x2 = 2;
      } else {
        ax = 0; x1 = 1; x2 = 2;
      }
      const int p1 = D[x1], p2 = D[x2];
      const double a = (double)std::abs(p1) / (double)m;
      const double b = (double)std::abs(p2) / (double)m;
      const double w1 = (1.0 - a) * (1.0 - b);
      const double w2 = a * (1.0 - b);
      const double w3 = (1.0 - a) * b;
      const double w4 = a * b;
      const double ds =
          std::sqrt(1.0 + (double)((int64_t)p1 * p1 + (int64_t)p2 * p2) / (double)((int64_t)m * m));
      T tin;
      if (m == 1) {
        tin = (0.5 * dts) * ds;
      } else {
        int e1[3] = {di, dj, dk};
        e1[ax] -= sgn(D[ax]);
        int e2[3] = {e1[0], e1[1], e1[2]};
        e2[x1] -= sgn(p1);
        int e3[3] = {e1[0], e1[1], e1[2]};
        e3[x2] -= sgn(p2);
        int e4[3] = {e2[0], e2[1], e2[2]};
        e4[x2] -= sgn(p2);
        const T c1 = tout[cidx(e1[0], e1[1], e1[2])];
        const T c2 = tout[cidx(e2[0], e2[1], e2[2])];
        const T c3 = tout[cidx(e3[0], e3[1], e3[2])];
        const T c4 = tout[cidx(e4[0], e4[1], e4[2])];
        if (o.debug && (std::isnan(re(c1)) || std::isnan(re(c2)) || std::isnan(re(c3)) ||
                        std::isnan(re(c4))))
          o.err = 1;
        if (P.interp == 1) {
          // optical-depth-modulated weights, normalised (branches on the real part)
          auto mod = [&](const T& c) { return re(c) > P.tau_w0 ? T(1.0) / c : T(1.0 / P.tau_w0); };
          const T v1 = w1 * mod(c1), v2 = w2 * mod(c2), v3 = w3 * mod(c3), v4 = w4 * mod(c4);
          const T S = ((v1 + v2) + v3) + v4;
          tin = fmaT(v4, c4, fmaT(v3, c3, fmaT(v2, c2, v1 * c1))) / S;
        } else {
          tin = fmaT(w4, c4, fmaT(w3, c3, fmaT(w2, c2, w1 * c1)));
        }
      }
      const T dtp = F.dt(g);
      const T t_out = fmaT(ds, dtp, tin);
      tout[cidx(di, dj, dk)] = t_out;
      if (o.coldens) o.coldens[g] = re(t_out) / sigma0;
      if (o.tau_in) o.tau_in[g] = re(tin);
      const T dcell = dtp * ds;
      const double r2 = alpha * alpha * (double)d2;
      T dG;
      if (re(dcell) <= P.tau_lim) {
        dG = ndot * sigma0 * tab_eval(tab, tab.hc0, tab.hc1, tin) / (4.0 * kPi * r2);
      } else {
        dG = ndot * (tab_eval(tab, tab.gc0, tab.gc1, tin) - tab_eval(tab, tab.gc0, tab.gc1, t_out)) /
             (F.nh(g) * (4.0 * kPi * r2 * alpha * ds));
      }
      deposit(g, dG);
    });
  }
}

bool make_table(int kind, int E0, int E1, int B, const double* gk, const double* hk, Table& t) {
  if (kind != 0 && kind != 1) return false;
  if (E0 < 1 || E0 > 1000 || E1 < 1 || E1 > 1000 || B < 0 || B > 12) return false;
  t.kind = kind;
  t.E0 = E0;
  t.E1 = E1;
  t.B = B;
  t.tau_min = std::ldexp(1.0, -E0);
  t.tau_max = std::ldexp(1.0, E1);
  if (kind == 0) {
    if (!gk || !hk) return false;
    chords(gk, E0, E1, B, t.gc0, t.gc1);
    chords(hk, E0, E1, B, t.hc0, t.hc1);
  }
  return true;
}

void per_cell(const Params& P, int64_t ncell, const double* nH, const double* xHI,
              std::vector<double>& dtau, std::vector<double>& nhi) {
  dtau.resize(ncell);
  nhi.resize(ncell);
  const double sa = P.sigma0 * P.cell_cm;
  for (int64_t c = 0; c < ncell; ++c) {
    dtau[c] = (sa * nH[c]) * xHI[c];
    nhi[c] = nH[c] * xHI[c];
  }
}

// ------------------------------------------------------------- quadrature
// Gauss-Legendre nodes/weights on [-1, 1] by Newton iteration on P_n.
void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
  x.resize(n);
  w.resize(n);
  for (int i = 0; i < n; ++i) {
    double z = std::cos(kPi * (i + 0.75) / (n + 0.5));
    double pp = 0;
    for (int it = 0; it < 100; ++it) {
      double p1 = 1.0, p2 = 0.0;
      for (int j = 1; j <= n; ++j) {
        const double p3 = p2;
        p2 = p1;
        p1 = ((2.0 * j - 1.0) * z * p2 - (j - 1.0) * p3) / j;
      }
      pp = n * (z * p1 - p2) / (z * z - 1.0);
      const double z1 = z;
      z = z1 - p1 / pp;
      if (std::fabs(z - z1) < 1e-16) break;
    }
    x[i] = z;
    w[i] = 2.0 / ((1.0 - z * z) * pp * pp);
  }
}

}  // namespace

extern "C" {

int or_version(void) { return 1; }

// Number of table knots for (E0, E1, B).
int or_table_nknots(int E0, int E1, int B) { return n_knots(E0, E1, B); }

// tau values of all knots.
void or_table_knot_taus(int E0, int E1, int B, double* out) {
  const int K = n_knots(E0, E1, B);
  for (int i = 0; i < K; ++i) out[i] = knot_tau(i, E0, E1, B);
}

// Table lookup (for tests): kind 0 chords / 1 analytic grey; which 0 = g, 1 = h.
int or_table_eval(int kind, int E0, int E1, int B, const double* gk, const double* hk, int which,
                  int n, const double* tau, double* out) {
  Table t;
  if (!make_table(kind, E0, E1, B, gk, hk, t)) return 1;
  for (int i = 0; i < n; ++i)
    out[i] = which == 0 ? tab_eval(t, t.gc0, t.gc1, tau[i]) : tab_eval(t, t.hc0, t.hc1, tau[i]);
  return 0;
}

// Knot values of g(tau) and h(tau) (Eq. tables, normalised by Ndot, Eq. ngammalnu).
// kind 0: grey (sigma_nu = sigma0): g = h = exp(-tau).
// kind 1: blackbody L_nu ~ nu^3/(exp(h nu/kT)-1) with sigma_nu = sigma0 (nu/nu_th)^-beta.
// With x = nu/nu_th and theta = h nu_th/(k T):
//   g(tau) = int_1^inf x^2/(e^{theta x}-1) exp(-tau x^-beta) dx / int_1^inf x^2/(e^{theta x}-1) dx
//   h(tau) = int_1^inf x^2/(e^{theta x}-1) x^-beta exp(-tau x^-beta) dx / (same norm)
// Composite 20-point Gauss-Legendre on panels of width 0.05 over [1, 1 + 740/theta].
int or_table_knots(int kind, double T_bb, double beta, int E0, int E1, int B, double* g_out,
                   double* h_out) {
  const int K = n_knots(E0, E1, B);
  if (kind == 0) {
    for (int i = 0; i < K; ++i) {
      g_out[i] = std::exp(-knot_tau(i, E0, E1, B));
      h_out[i] = g_out[i];
    }
    return 0;
  }
  if (kind != 1 || !(T_bb > 0)) return 1;
  const double h_planck = 6.62607015e-27;  // erg s
  const double k_boltz = 1.380649e-16;     // erg/K
  const double ev = 1.602176634e-12;       // erg
  const double theta = (13.6 * ev) / (k_boltz * T_bb);
  (void)h_planck;
  const double xmax = 1.0 + 740.0 / theta;
  const double width = 0.05;
  const int npan = (int)std::ceil((xmax - 1.0) / width);
  std::vector<double> gx, gw;
  gauss_legendre(20, gx, gw);
  const size_t nn = (size_t)npan * gx.size();
  std::vector<double> wt(nn), sx(nn);
  double norm = 0.0;
  for (int p = 0; p < npan; ++p) {
    const double lo = 1.0 + p * width, hi = lo + width;
    const double c = 0.5 * (lo + hi), hw = 0.5 * (hi - lo);
    for (size_t i = 0; i < gx.size(); ++i) {
      const double x = c + hw * gx[i];
      const double f = x * x / std::expm1(theta * x);
      wt[p * gx.size() + i] = hw * gw[i] * f;
      sx[p * gx.size() + i] = std::pow(x, -beta);
      norm += hw * gw[i] * f;
    }
  }
#pragma omp parallel for schedule(dynamic, 16)
  for (int k = 0; k < K; ++k) {
    const double tau = knot_tau(k, E0, E1, B);
    double sg = 0.0, sh = 0.0;
    for (size_t i = 0; i < nn; ++i) {
      const double e = std::exp(-tau * sx[i]);
      sg += wt[i] * e;
      sh += wt[i] * sx[i] * e;
    }
    g_out[k] = sg / norm;
    h_out[k] = sh / norm;
  }
  return 0;
}

// Shell S_q in the oracle's enumeration order; returns the count, writes
// (Di,Dj,Dk) triples if out != null.
int or_shell_list(int q, int* out) {
  int n = 0;
  for_each_in_shell(q, [&](int a, int b, int c) {
    if (out) {
      out[3 * n] = a;
      out[3 * n + 1] = b;
      out[3 * n + 2] = c;
    }
    ++n;
  });
  return n;
}

// Ray trace a single periodic box.
//   n, cell_cm, sigma0, tau_lim : grid and physics parameters
//   kind/E0/E1/B/gk/hk          : rate table (knot values) or analytic grey
//   nH, xHI                     : double[n^3], C order (i*n+j)*n+k
//   nsrc, pos (int[nsrc][3]), ndot, radius (cells)
//   gamma                       : double[n^3], rates are ADDED (may be null)
//   cd_src, coldens, tau_in     : if cd_src >= 0, the column density (cm^-2) out of
//                                 each cell and tau up to each cell for source
//                                 cd_src are written (others untouched)
//   wloss, loss                 : if both given, *loss += sum_p wloss_p dGamma_p
//   nthreads                    : >1 splits sources in contiguous chunks, each with
//                                 a private rate field, summed in chunk order
//   debug                       : NaN-fill scratch, return 2 on an acausal read
// Returns 0 on success, 1 on invalid arguments, 2 on a causality violation.
//   interp_mode, tau_w0          : weights (or_raytrace2 only): 0 geometric, 1
//                                 optical-depth-modulated with floor tau_w0
int or_raytrace2(int n, double cell_cm, double sigma0, double tau_lim, int kind, int E0, int E1,
                 int B, const double* gk, const double* hk, const double* nH, const double* xHI,
                 int nsrc, const int* pos, const double* ndot, const double* radius,
                 double* gamma, int cd_src, double* coldens, double* tau_in,
                 const double* wloss, double* loss, int nthreads, int debug, int interp_mode,
                 double tau_w0) {
  if (n < 1 || nsrc < 0) return 1;
  if (interp_mode != 0 && interp_mode != 1) return 1;
  if (!(tau_w0 > 0.0) || !std::isfinite(tau_w0)) return 1;
  Params P{n, cell_cm, sigma0, tau_lim};
  P.interp = interp_mode;
  P.tau_w0 = tau_w0;
  Table tab;
  if (!make_table(kind, E0, E1, B, gk, hk, tab)) return 1;
  const int64_t nc = (int64_t)n * n * n;
  std::vector<double> dtau, nhi;
  per_cell(P, nc, nH, xHI, dtau, nhi);
  Fields<double> F{dtau.data(), nhi.data()};
  for (int s = 0; s < nsrc; ++s)
    for (int a = 0; a < 3; ++a)
      if (pos[3 * s + a] < 0 || pos[3 * s + a] >= n) return 1;
  int err = 0;
  if (nthreads <= 1 || nsrc < 2) {
    for (int s = 0; s < nsrc; ++s) {
      Out o;
      o.gamma = gamma;
      o.debug = debug != 0;
      o.wloss = wloss;
      o.loss = loss;
      if (s == cd_src) {
        o.coldens = coldens;
        o.tau_in = tau_in;
      }
      trace_one<double>(P, tab, F, pos[3 * s], pos[3 * s + 1], pos[3 * s + 2], ndot[s], radius[s], o);
      err |= o.err;
    }
  } else {
    const int nt = std::min(nthreads, nsrc);
    std::vector<std::vector<double>> priv(nt);
    std::vector<double> ploss(nt, 0.0);
    std::vector<int> perr(nt, 0);
#ifdef _OPENMP
#pragma omp parallel for num_threads(nt) schedule(static, 1)
#endif
    for (int t = 0; t < nt; ++t) {
      const int s0 = (int)((int64_t)nsrc * t / nt), s1 = (int)((int64_t)nsrc * (t + 1) / nt);
      if (gamma) priv[t].assign(nc, 0.0);
      for (int s = s0; s < s1; ++s) {
        Out o;
        o.gamma = gamma ? priv[t].data() : nullptr;
        o.debug = debug != 0;
        o.wloss = wloss;
        o.loss = loss ? &ploss[t] : nullptr;
        if (s == cd_src) {
          o.coldens = coldens;
          o.tau_in = tau_in;
        }
        trace_one<double>(P, tab, F, pos[3 * s], pos[3 * s + 1], pos[3 * s + 2], ndot[s], radius[s], o);
        perr[t] |= o.err;
      }
    }
    for (int t = 0; t < nt; ++t) {
      if (gamma)
        for (int64_t c = 0; c < nc; ++c) gamma[c] += priv[t][c];
      if (loss) *loss += ploss[t];
      err |= perr[t];
    }
  }
  return err ? 2 : 0;
}

int or_raytrace(int n, double cell_cm, double sigma0, double tau_lim, int kind, int E0, int E1,
                int B, const double* gk, const double* hk, const double* nH, const double* xHI,
                int nsrc, const int* pos, const double* ndot, const double* radius,
                double* gamma, int cd_src, double* coldens, double* tau_in,
                const double* wloss, double* loss, int nthreads, int debug) {
  return or_raytrace2(n, cell_cm, sigma0, tau_lim, kind, E0, E1, B, gk, hk, nH, xHI, nsrc, pos,
                      ndot, radius, gamma, cd_src, coldens, tau_in, wloss, loss, nthreads, debug, 0,
                      0.6);
}

// Complex-step derivatives of L = sum_p w_p Gamma_p:
//   dL/dlog n_HI(c) for each cell c in cells[0..ncells), and
//   dL/dlog Ndot(s) for each source s in srcs[0..nsrcs).
// log n_HI(c) -> log n_HI(c) + i h changes dtau(c) and n_HI(c) by the factor (1 + i h);
// only sources whose traced region contains c contribute.
int or_loss_grad_cs(int n, double cell_cm, double sigma0, double tau_lim, int kind, int E0,
                    int E1, int B, const double* gk, const double* hk, const double* nH,
                    const double* xHI, int nsrc, const int* pos, const double* ndot,
                    const double* radius, const double* wloss, int ncells, const int64_t* cells,
                    double* dL_dlogn, int nsrcs, const int* srcs, double* dL_dlogndot, double h,
                    int nthreads) {
  Params P{n, cell_cm, sigma0, tau_lim};
  Table tab;
  if (!make_table(kind, E0, E1, B, gk, hk, tab)) return 1;
  const int64_t nc = (int64_t)n * n * n;
  std::vector<double> dtau, nhi;
  per_cell(P, nc, nH, xHI, dtau, nhi);
  const int wlo = -(n / 2), whi = (n % 2 == 0) ? n / 2 - 1 : n / 2;
  auto offs = [&](int c, int s) {
    int d = c - s;
    d = wrap(d - wlo, n) + wlo;  // representative in [wlo, wlo+n)
    return d;
  };
#ifdef _OPENMP
#pragma omp parallel for num_threads(std::max(1, nthreads)) schedule(dynamic, 1)
#endif
  for (int t = 0; t < ncells; ++t) {
    const int64_t c = cells[t];
    const int ci = (int)(c / ((int64_t)n * n)), cj = (int)((c / n) % n), ck = (int)(c % n);
    Fields<cplx> F{dtau.data(), nhi.data(), c, h};
    cplx L(0.0, 0.0);
    for (int s = 0; s < nsrc; ++s) {
      const int di = offs(ci, pos[3 * s]), dj = offs(cj, pos[3 * s + 1]), dk = offs(ck, pos[3 * s + 2]);
      if (di > whi || dj > whi || dk > whi) continue;
      const int64_t R2 = (int64_t)std::floor(radius[s] * radius[s]);
      if ((int64_t)di * di + (int64_t)dj * dj + (int64_t)dk * dk > R2) continue;
      Out o;
      o.wloss = wloss;
      o.loss = &L;
      trace_one<cplx>(P, tab, F, pos[3 * s], pos[3 * s + 1], pos[3 * s + 2], cplx(ndot[s], 0.0),
                      radius[s], o);
    }
    dL_dlogn[t] = L.imag() / h;
  }
#ifdef _OPENMP
#pragma omp parallel for num_threads(std::max(1, nthreads)) schedule(dynamic, 1)
#endif
  for (int t = 0; t < nsrcs; ++t) {
    const int s = srcs[t];
    Fields<cplx> F{dtau.data(), nhi.data(), -1, 0.0};
    cplx L(0.0, 0.0);
    Out o;
    o.wloss = wloss;
    o.loss = &L;
    trace_one<cplx>(P, tab, F, pos[3 * s], pos[3 * s + 1], pos[3 * s + 2],
                    cplx(ndot[s], ndot[s] * h), radius[s], o);
    dL_dlogndot[t] = L.imag() / h;
  }
  return 0;
}

// Long characteristics (Sec. 3, first paragraph), for tests only: for every
// cell of the traced region of one source, the optical depth from the source
// centre to the point where the straight ray towards the cell centre leaves
// the cell, summed exactly over the cells it crosses (3-D DDA).
int or_lc_tau(int n, double cell_cm, double sigma0, const double* nH, const double* xHI, int is,
              int js, int ks, double R, double* tau_out) {
  Params P{n, cell_cm, sigma0, 0.0};
  const int64_t nc = (int64_t)n * n * n;
  std::vector<double> dtau, nhi;
  per_cell(P, nc, nH, xHI, dtau, nhi);
  const int wlo = -(n / 2), whi = (n % 2 == 0) ? n / 2 - 1 : n / 2;
  const int64_t R2 = (int64_t)std::floor(R * R);
  for (int di = wlo; di <= whi; ++di)
    for (int dj = wlo; dj <= whi; ++dj)
      for (int dk = wlo; dk <= whi; ++dk) {
        const int64_t d2 = (int64_t)di * di + (int64_t)dj * dj + (int64_t)dk * dk;
        if (d2 > R2) continue;
        const int64_t g = ((int64_t)wrap(is + di, n) * n + wrap(js + dj, n)) * n + wrap(ks + dk, n);
        const int D[3] = {di, dj, dk};
        const int m = std::max(std::abs(di), std::max(std::abs(dj), std::abs(dk)));
        const double len = std::sqrt((double)d2);  // |Delta| in cells; ray r(t) = t Delta
        if (m == 0) {
          tau_out[g] = 0.5 * dtau[g];
          continue;
        }
        const double t_end = (m + 0.5) / m;
        // crossing parameters t = (c + 0.5)/|D_a| for c = 0,1,.. (each axis)
        std::vector<double> ts;
        for (int a = 0; a < 3; ++a) {
          const int ad = std::abs(D[a]);
          for (int c = 0; c < ad + 1; ++c) {
            const double t = (c + 0.5) / ad;
            if (t < t_end) ts.push_back(t);
          }
        }
        ts.push_back(t_end);
        std::sort(ts.begin(), ts.end());
        double tau = 0.0, t0 = 0.0;
        for (double t1 : ts) {
          if (t1 > t0) {
            const double tm = 0.5 * (t0 + t1);
            const int ci = (int)std::floor(tm * di + 0.5);
            const int cj = (int)std::floor(tm * dj + 0.5);
            const int ck = (int)std::floor(tm * dk + 0.5);
            const int64_t gc = ((int64_t)wrap(is + ci, n) * n + wrap(js + cj, n)) * n + wrap(ks + ck, n);
            tau += dtau[gc] * (t1 - t0) * len;
          }
          t0 = t1;
        }
        tau_out[g] = tau;
      }
  return 0;
}

// Chemistry step (Sec. 2.1, Eq. time_avrg_sol), per cell, isothermal hydrogen.
//   x0       : ionised fraction x_HII at the start of the step
//   xavg_in  : time-averaged x_HII used by the preceding ray trace
//   gamma    : photo-ionisation rate (s^-1)
// Iterates n_e = n_H <x>  (starting from <x> = xavg_in) until
// |<x>_new - <x>_old| <= tol <x>_new or maxit iterations.  Writes <x_HII> and
// x_HII(t+dt).  *nunconv = number of cells whose neutral fraction 1-<x> changed
// by more than conv_tol (relative) w.r.t. 1 - xavg_in.
int or_chemistry(int64_t ncell, const double* nH, const double* x0, const double* xavg_in,
                 const double* gamma, double dt, double alpha_H, double C_H, double tol, int maxit,
                 double conv_tol, double* xavg_out, double* xnew_out, int64_t* nunconv) {
  int64_t cnt = 0;
  for (int64_t c = 0; c < ncell; ++c) {
    const double G = gamma[c];
    double xa = xavg_in[c];
    double xnew = x0[c];
    for (int it = 0; it < maxit; ++it) {
      const double ne = nH[c] * xa;
      const double rate = G + ne * (C_H + alpha_H);  // 1/t_i
      double xa_new;
      if (rate > 0.0) {
        const double xeq = (G + ne * C_H) / rate;
        const double y = dt * rate;                  // dt/t_i
        xa_new = xeq + (x0[c] - xeq) * (-std::expm1(-y) / y);
        xnew = xeq + (x0[c] - xeq) * std::exp(-y);
      } else {  // no ionisation, no recombination: x stays x0
        xa_new = x0[c];
        xnew = x0[c];
      }
      const bool done = std::fabs(xa_new - xa) <= tol * xa_new;
      xa = xa_new;
      if (done) break;
    }
    xavg_out[c] = xa;
    xnew_out[c] = xnew;
    const double xhi_old = 1.0 - xavg_in[c], xhi_new = 1.0 - xa;
    if (std::fabs(xhi_new - xhi_old) > conv_tol * xhi_new) ++cnt;
  }
  *nunconv = cnt;
  return 0;
}

}  // extern "C"
