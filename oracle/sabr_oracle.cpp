// ORACLE -- test infrastructure only.
//
// A plain, slow, FP64 CPU restatement of the calibration objective and of the parallel
// simulated-annealing search of Ferreiro, Garcia, Lopez-Salas and Vazquez, "SABR/LIBOR market
// models: pricing and calibration for some interest rate derivatives" (arXiv 2408.01470).
// Only the test-suite, the smoke check and the CPU-baseline leg of the benchmark load it.  It
// shares no code, header, table or helper with the CUDA library; the two meet only through the
// seeded synthetic inputs.
//
// Every numeric routine is templated on its scalar so that the same definitions, instantiated
// with forward-mode dual numbers, give the gradient and the Jacobian (an independent route from
// the library's hand-written adjoint).
//
// What each part follows, and what pins it (tests/test_oracle_*.py):
//   normal_cdf / black / vega ...... Black's formula for caplets and swaptions (Section 1, the
//                                    cost functions of Section 3).  Pins: closed-form points,
//                                    put-call parity, the zero-vol and zero-strike limits.
//   sabr_hagan2002 ................. Hagan et al.'s lognormal expansion with the z/x(z) factor,
//                                    the formula Section 2.1 refers to by Hagan's name.  Pins:
//                                    beta=1,nu=0 gives alpha; ATM limit; mirror symmetry; a
//                                    50-digit evaluation of the textbook form.
//   sabr_paper ..................... Eq. (sigmaHagan) as printed.  Pin: the paper's calibrated
//                                    parameters (Table tab:paramsHaganVolas) reproduce its model
//                                    vols (Table tab:haganVolas).
//   rebonato_caplet ................ Eq. (haganForRebonato), the integrals by composite
//                                    Gauss-Legendre.  Pins: closed form of int g^2, 50-digit
//                                    adaptive quadrature of both integrals.
//   swap_params .................... the approximate swaption volatility (a quadratic form of
//                                    time-integrated forward-rate vols over the correlation
//                                    matrices of Eqs. rhoij, thetaij, phiij).  The paper names it
//                                    but does not print it; this is the reading fixed for this
//                                    project.  Pins: one-period swap == caplet; rho=1 with equal
//                                    vols gives the caplet vol; V1 >= 0.
//   mm_alpha ....................... Eq. (haganForMercurio), the Mercurio & Morini mapping: the
//                                    drift integral interval by interval between fixing dates.
//                                    Pins: the closed form -sigma sum_j c_j T_j of that integral;
//                                    sigma = 0 gives the smile formula at alpha_i; the paper's
//                                    calibrated parameters (Table tab:paramsMercurioVolas) against
//                                    its model vols (Table tab:mercurioVolas) and the descent from
//                                    them to its published MRE.
//   objective ...................... f_c and f_s of Section 3 in price space with vega weights.
//                                    Pin: zero at the generating point on noise-free quotes.
//   philox4x64_10 .................. Salmon, Moraes, Dror, Shaw (SC'11).  Pins: numpy's Philox
//                                    bit generator and the all-zero known-answer vector.
//   nm ............................. the Nelder-Mead local search of the hybrid scheme (Section
//                                    3), standard coefficients.  Pins: a separable quadratic bowl
//                                    in closed form, monotone best value, recovery on noise-free
//                                    quotes.
//   philox4x32_10, mc_normals4 ..... the 32-bit Philox and the Box-Muller normals of the Monte
//                                    Carlo pricer.  Pins: Random123's known-answer vectors; the
//                                    moments of the normals.
//   mc_price ....................... the Monte Carlo pricer of Section 3 (Table tab:haganMCpricer):
//                                    the Hagan SABR/LIBOR dynamics under the spot measure, log-Euler.
//                                    Pins: a zero-strike caplet is worth P(0,T_i) - P(0,T_{i+1})
//                                    and a zero-strike swaption P(0,T_a) - P(0,T_b) under any
//                                    arbitrage-free dynamics; with sigma = 0, beta = 1 every caplet
//                                    is Black's at vol alpha_i (the lognormal LIBOR market model).
//   mc_price, model 2 .............. the Mercurio & Morini dynamics (Section 2.2) under the spot
//                                    measure, one vol process.  Pins: the zero-strike floating legs;
//                                    sigma = 0, beta = 1 gives Black at alpha_i; the vol of vol
//                                    lifts far out-of-the-money caplets above Black.
//   mc_objective, orc_mc_anneal .... the swaption calibration of Section 3 over the Monte Carlo
//                                    objective (common random numbers), by the same annealing
//                                    loop.  Pins: f_s = 0 at the generating correlation parameters
//                                    on quotes made by the pricer itself; the search gets back to
//                                    them from the box centre.
//   anneal ......................... the SA loop of Section 3 and its one-GPU parallel form
//                                    (chains per level, min-reduction, broadcast).  Pins: the
//                                    evaluation-count identity C(LN+1); recovery on tiny sets.
//   lm ............................. Levenberg-Marquardt polish (replaces the Nelder-Mead of the
//                                    hybrid scheme in Section 3).  Pin: recovery of the
//                                    generating point on noise-free quotes.
//
// Readings of places where the paper is silent are listed at each function.

#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>
#include <map>
#include <utility>
#include <algorithm>
#include <limits>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace orc {

// ------------------------------------------------------------------ dual numbers (forward mode)
constexpr int ND = 12;

struct Dual {
  double v;
  double d[ND];
  Dual() : v(0.0) { for (int i = 0; i < ND; ++i) d[i] = 0.0; }
  Dual(double x) : v(x) { for (int i = 0; i < ND; ++i) d[i] = 0.0; }
};

inline double val(double x) { return x; }
inline double val(const Dual& x) { return x.v; }

inline Dual operator+(const Dual& a, const Dual& b) { Dual r(a.v + b.v); for (int i = 0; i < ND; ++i) r.d[i] = a.d[i] + b.d[i]; return r; }
inline Dual operator-(const Dual& a, const Dual& b) { Dual r(a.v - b.v); for (int i = 0; i < ND; ++i) r.d[i] = a.d[i] - b.d[i]; return r; }
inline Dual operator*(const Dual& a, const Dual& b) { Dual r(a.v * b.v); for (int i = 0; i < ND; ++i) r.d[i] = a.d[i] * b.v + a.v * b.d[i]; return r; }
inline Dual operator/(const Dual& a, const Dual& b) { Dual r(a.v / b.v); for (int i = 0; i < ND; ++i) r.d[i] = (a.d[i] * b.v - a.v * b.d[i]) / (b.v * b.v); return r; }
inline Dual operator-(const Dual& a) { Dual r(-a.v); for (int i = 0; i < ND; ++i) r.d[i] = -a.d[i]; return r; }
inline Dual operator+(const Dual& a, double b) { Dual r = a; r.v += b; return r; }
inline Dual operator+(double a, const Dual& b) { return b + a; }
inline Dual operator-(const Dual& a, double b) { Dual r = a; r.v -= b; return r; }
inline Dual operator-(double a, const Dual& b) { return -b + a; }
inline Dual operator*(const Dual& a, double b) { Dual r(a.v * b); for (int i = 0; i < ND; ++i) r.d[i] = a.d[i] * b; return r; }
inline Dual operator*(double a, const Dual& b) { return b * a; }
inline Dual operator/(const Dual& a, double b) { Dual r(a.v / b); for (int i = 0; i < ND; ++i) r.d[i] = a.d[i] / b; return r; }
inline Dual operator/(double a, const Dual& b) { Dual r(a / b.v); for (int i = 0; i < ND; ++i) r.d[i] = -a * b.d[i] / (b.v * b.v); return r; }
inline Dual& operator+=(Dual& a, const Dual& b) { a = a + b; return a; }
inline Dual& operator-=(Dual& a, const Dual& b) { a = a - b; return a; }
inline Dual& operator*=(Dual& a, const Dual& b) { a = a * b; return a; }

// chain rule: f(a) with f'(a) = dv
inline Dual chain(const Dual& a, double fv, double dv) { Dual r(fv); for (int i = 0; i < ND; ++i) r.d[i] = dv * a.d[i]; return r; }
inline Dual exp(const Dual& a) { double e = std::exp(a.v); return chain(a, e, e); }
inline Dual log(const Dual& a) { return chain(a, std::log(a.v), 1.0 / a.v); }
inline Dual log1p(const Dual& a) { return chain(a, std::log1p(a.v), 1.0 / (1.0 + a.v)); }
inline Dual sqrt(const Dual& a) { double s = std::sqrt(a.v); return chain(a, s, 0.5 / s); }
inline Dual erfc(const Dual& a) { return chain(a, std::erfc(a.v), -2.0 / std::sqrt(M_PI) * std::exp(-a.v * a.v)); }

using std::exp; using std::log; using std::log1p; using std::sqrt; using std::erfc;

// ------------------------------------------------------------------ Gauss-Legendre nodes
// Roots of the Legendre polynomial P_n by Newton's method on the three-term recurrence,
// in long double; weights 2 / ((1 - x^2) P_n'(x)^2).  Nodes ascending.
static void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
  x.assign(n, 0.0); w.assign(n, 0.0);
  const long double pi = 3.141592653589793238462643383279502884L;
  for (int i = 0; i < n; ++i) {
    long double z = std::cos(pi * (i + 0.75L) / (n + 0.5L));
    long double dp = 0.0L;
    for (int it = 0; it < 100; ++it) {
      long double p0 = 1.0L, p1 = z;
      for (int k = 2; k <= n; ++k) {
        long double p2 = ((2.0L * k - 1.0L) * z * p1 - (k - 1.0L) * p0) / k;
        p0 = p1; p1 = p2;
      }
      dp = n * (z * p1 - p0) / (z * z - 1.0L);
      long double dz = p1 / dp;
      z -= dz;
      if (std::fabs((double)dz) < 1e-19) break;
    }
    // recompute the derivative at the converged root
    long double p0 = 1.0L, p1 = z;
    for (int k = 2; k <= n; ++k) {
      long double p2 = ((2.0L * k - 1.0L) * z * p1 - (k - 1.0L) * p0) / k;
      p0 = p1; p1 = p2;
    }
    dp = n * (z * p1 - p0) / (z * z - 1.0L);
    x[n - 1 - i] = (double)z;
    w[n - 1 - i] = (double)(2.0L / ((1.0L - z * z) * dp * dp));
  }
  // i-th root from the top is descending in z; reversed above -> ascending
}

// ------------------------------------------------------------------ Black's formula
// Phi(x) = erfc(-x / sqrt 2) / 2.
template <class S> S normal_cdf(const S& x) { return 0.5 * erfc(-x / std::sqrt(2.0)); }

// Black's formula for an option on a forward F struck at K, expiry T, Black vol sigma, discount
// D (tau P(0,T_{k+1}) for a caplet, the annuity for a swaption).
template <class S> S black_call(double F, double K, double T, const S& sigma, double D) {
  S v = sigma * std::sqrt(T);
  S d1 = std::log(F / K) / v + 0.5 * v;
  S d2 = d1 - v;
  return D * (F * normal_cdf(d1) - K * normal_cdf(d2));
}
template <class S> S black_put(double F, double K, double T, const S& sigma, double D) {
  S v = sigma * std::sqrt(T);
  S d1 = std::log(F / K) / v + 0.5 * v;
  S d2 = d1 - v;
  return D * (K * normal_cdf(-d2) - F * normal_cdf(-d1));
}
// Reading: every quote is priced as its out-of-the-money option (a put below the forward, a call
// at or above it); put-call parity makes the two sides equivalent.
template <class S> S black_otm(double F, double K, double T, const S& sigma, double D) {
  return (K < F) ? black_put(F, K, T, sigma, D) : black_call(F, K, T, sigma, D);
}
// dPrice/dsigma, identical for calls and puts.
static double black_vega(double F, double K, double T, double sigma, double D) {
  double v = sigma * std::sqrt(T);
  double d1 = std::log(F / K) / v + 0.5 * v;
  return D * F * std::exp(-0.5 * d1 * d1) / std::sqrt(2.0 * M_PI) * std::sqrt(T);
}

// ------------------------------------------------------------------ SABR implied vol
// x(z) = log((sqrt(1 - 2 rho z + z^2) + z - rho) / (1 - rho)), written as log1p of
// ((s - 1) + z) / (1 - rho) with s - 1 = (z^2 - 2 rho z) / (s + 1) for z >= 0, and through the
// exact mirror x(z; rho) = -x(-z; -rho) for z < 0 (both rewrites are algebraic identities).
template <class S> S x_of_z(const S& z, const S& rho) {
  if (val(z) < 0.0) return -x_of_z(-z, -rho);
  S s = sqrt(1.0 - 2.0 * rho * z + z * z);
  return log1p(((z * z - 2.0 * rho * z) / (s + 1.0) + z) / (1.0 - rho));
}
// z / x(z), with its Taylor series 1 - rho z / 2 + (2 - 3 rho^2) z^2 / 12 for |z| < 1e-6.
template <class S> S z_over_x(const S& z, const S& rho) {
  if (std::fabs(val(z)) < 1e-6) return 1.0 - 0.5 * rho * z + (2.0 - 3.0 * rho * rho) * z * z / 12.0;
  return z / x_of_z(z, rho);
}

// Hagan, Kumar, Lesniewski, Woodward (2002), lognormal expansion:
//   sigma = alpha / ((FK)^{(1-b)/2} [1 + (1-b)^2 l^2/24 + (1-b)^4 l^4/1920]) * z/x(z)
//           * {1 + [(1-b)^2 alpha^2 / (24 (FK)^{1-b}) + rho b nu alpha / (4 (FK)^{(1-b)/2})
//                  + (2 - 3 rho^2) nu^2 / 24] T},
//   l = log(F/K), z = (nu/alpha) (FK)^{(1-b)/2} l.
template <class S>
S sabr_hagan2002(double F, double K, double T, const S& alpha, double beta, const S& rho, const S& nu) {
  double omb = 1.0 - beta;
  double fk = std::pow(F * K, 0.5 * omb);
  double l = std::log(F / K);
  S z = nu / alpha * fk * l;
  S zx = z_over_x(z, rho);
  double den = fk * (1.0 + omb * omb * l * l / 24.0 + omb * omb * omb * omb * l * l * l * l / 1920.0);
  S corr = 1.0 + (omb * omb * alpha * alpha / (24.0 * fk * fk) + rho * beta * nu * alpha / (4.0 * fk)
                  + (2.0 - 3.0 * rho * rho) * nu * nu / 24.0) * T;
  return alpha / den * zx * corr;
}

// Eq. (sigmaHagan) verbatim, with phi_ii -> rho, sigma_i -> nu, omega = F^{1-b} / alpha,
// m = log(K/F).  No expiry dependence.
template <class S>
S sabr_paper(double F, double K, const S& alpha, double beta, const S& rho, const S& nu) {
  double omb = 1.0 - beta;
  double fo = std::pow(F, omb);
  S omega = fo / alpha;
  double m = std::log(K / F);
  S rno = rho * nu * omega;
  return alpha / fo * (1.0 - 0.5 * (omb - rno) * m
                       + (omb * omb + (2.0 - 3.0 * rho * rho) * nu * nu * omega * omega + 3.0 * (omb - rno)) * (m * m) / 12.0);
}

// ------------------------------------------------------------------ market
struct Desc {  // mirrors the ctypes structure in oracle/__init__.py
  int32_t model, formula;
  double beta;
  int32_t n_fwd;
  const double* T;
  const double* P;
  int32_t n_cap;
  const int32_t* cap_fwd;
  const double* cap_K;
  const double* cap_vol;
  const double* cap_w;  // may be null -> 1/vega^2
  int32_t n_swp;
  const int32_t* swp_start;
  const int32_t* swp_end;
  const double* swp_K;
  const double* swp_vol;
  const double* swp_w;
  int32_t n_param;
  const double* lo;
  const double* hi;
  const uint8_t* free_mask;
  double panel;
  int32_t quad_nodes;
};

struct Market {
  int model, formula, n_param, Q;
  double beta, panel;
  std::vector<double> T, P, F, tau;
  // caplets
  std::vector<int> cfwd;
  std::vector<double> cK, cvol, cw, cpm;
  // swaptions, with the distinct underlying swaps
  std::vector<int> sstart, send, sswap;
  std::vector<double> sK, svol, sw, spm;
  std::vector<std::pair<int, int>> swaps;
  std::vector<double> swapA, swapS;           // annuity, swap rate
  std::vector<std::vector<double>> swapW;     // W_i = w_i F_i^b / S^b over the window
  std::vector<double> lo, hi;
  std::vector<uint8_t> freem;
  std::vector<double> xi, wi;                 // Gauss-Legendre on [-1, 1]
  int n_instr() const { return (int)cK.size() + (int)sK.size(); }
};

static int n_panels(double t, double panel) { return (int)std::lround(t / panel); }

static Market* build_market(const Desc* d) {
  Market* m = new Market();
  m->model = d->model; m->formula = d->formula; m->beta = d->beta; m->n_param = d->n_param;
  m->panel = d->panel; m->Q = d->quad_nodes;
  int n = d->n_fwd;
  m->T.assign(d->T, d->T + n + 1);
  m->P.assign(d->P, d->P + n + 1);
  m->F.resize(n); m->tau.resize(n);
  for (int k = 0; k < n; ++k) {
    m->tau[k] = m->T[k + 1] - m->T[k];
    m->F[k] = (m->P[k] / m->P[k + 1] - 1.0) / m->tau[k];   // simply-compounded forward
  }
  gauss_legendre(m->Q, m->xi, m->wi);
  m->lo.assign(d->lo, d->lo + d->n_param);
  m->hi.assign(d->hi, d->hi + d->n_param);
  m->freem.assign(d->free_mask, d->free_mask + d->n_param);
  for (int k = 0; k < d->n_cap; ++k) {
    int i = d->cap_fwd[k];
    double F = m->F[i], K = d->cap_K[k], T = m->T[i], D = m->tau[i] * m->P[i + 1];
    double vol = d->cap_vol ? d->cap_vol[k] : 0.2;
    m->cfwd.push_back(i); m->cK.push_back(K); m->cvol.push_back(vol);
    m->cpm.push_back(black_otm(F, K, T, vol, D));
    double vg = black_vega(F, K, T, vol, D);
    m->cw.push_back(d->cap_w ? d->cap_w[k] : 1.0 / (vg * vg));
  }
  std::map<std::pair<int, int>, int> index;
  for (int s = 0; s < d->n_swp; ++s) {
    int a = d->swp_start[s], b = d->swp_end[s];
    auto key = std::make_pair(a, b);
    if (!index.count(key)) {
      int id = (int)m->swaps.size();
      index[key] = id;
      m->swaps.push_back(key);
      double A = 0.0;
      for (int k = a; k < b; ++k) A += m->tau[k] * m->P[k + 1];
      double S = 0.0;
      for (int k = a; k < b; ++k) S += m->tau[k] * m->P[k + 1] / A * m->F[k];
      std::vector<double> W;
      for (int k = a; k < b; ++k)
        W.push_back(m->tau[k] * m->P[k + 1] / A * std::pow(m->F[k], m->beta) / std::pow(S, m->beta));
      m->swapA.push_back(A); m->swapS.push_back(S); m->swapW.push_back(W);
    }
    int id = index[key];
    double K = d->swp_K[s], T = m->T[a], A = m->swapA[id], S = m->swapS[id];
    double vol = d->swp_vol ? d->swp_vol[s] : 0.2;
    m->sstart.push_back(a); m->send.push_back(b); m->sswap.push_back(id);
    m->sK.push_back(K); m->svol.push_back(vol);
    m->spm.push_back(black_otm(S, K, T, vol, A));
    double vg = black_vega(S, K, T, vol, A);
    m->sw.push_back(d->swp_w ? d->swp_w[s] : 1.0 / (vg * vg));
  }
  return m;
}

// ------------------------------------------------------------------ Rebonato model
// g(u) and h(u) at time-to-fixing u = T_i - t (Section 2.3).
template <class S> S g_of(const S* th, double u) { return (th[0] + th[1] * u) * exp(-th[2] * u) + th[3]; }
template <class S> S h_of(const S* th, double u) { return (th[4] + th[5] * u) * exp(-th[6] * u) + th[7]; }

// Eq. (haganForRebonato) with kappa = 1, the caplet's SABR alpha and nu:
//   G = int_0^Ti g(Ti - t)^2 dt,   X = int_0^Ti g(Ti - t)^2 H(t) dt,   H(t) = int_0^t h(Ti - s)^2 ds
//   (t hhat(t)^2 = H(t) removes the 1/t of the printed form),
//   alpha = sqrt(G / Ti),   nu = sqrt(2 X) / (alpha Ti).
// Reading (the quadrature is the definition): composite Gauss-Legendre with Q nodes on every
// panel [p D, (p+1) D] of [0, Ti]; H at a node t of panel p is the sum of the full panels below
// plus a Q-node Gauss-Legendre rule on [p D, t].
template <class S>
void rebonato_caplet(const Market& m, const S* th, double Ti, S& alpha, S& nu, S* Gout = nullptr, S* Xout = nullptr) {
  const int n = n_panels(Ti, m.panel), Q = m.Q;
  const double D = m.panel;
  S G = 0.0, X = 0.0, Hcum = 0.0;
  for (int p = 0; p < n; ++p) {
    double t0 = p * D;
    for (int q = 0; q < Q; ++q) {
      double t = t0 + 0.5 * D * (1.0 + m.xi[q]);
      double wq = 0.5 * D * m.wi[q];
      S gv = g_of(th, Ti - t);
      double half = 0.5 * (t - t0);
      S part = 0.0;
      for (int r = 0; r < Q; ++r) {
        double s = t0 + half * (1.0 + m.xi[r]);
        S hv = h_of(th, Ti - s);
        part += half * m.wi[r] * hv * hv;
      }
      G += wq * gv * gv;
      X += wq * gv * gv * (Hcum + part);
    }
    for (int q = 0; q < Q; ++q) {
      double t = t0 + 0.5 * D * (1.0 + m.xi[q]);
      S hv = h_of(th, Ti - t);
      Hcum += 0.5 * D * m.wi[q] * hv * hv;
    }
  }
  alpha = sqrt(G / Ti);
  nu = sqrt(2.0 * X) / (alpha * Ti);
  if (Gout) *Gout = G;
  if (Xout) *Xout = X;
}

// The approximate swaption volatility (reading; the paper names Rebonato's approximation but
// prints no formula).  For the swap over forwards [a, b) with expiry T = T_a, frozen weights
// W_i = w_i F_i^b / S^b and
//   G_ij = int_0^T g_i g_j dt,   X_ij = theta_ij int_0^T g_i g_j (int_0^t h_i h_j ds) dt,
//   V1 = sum W_i W_j rho_ij G_ij,  V2 = sum W_i W_j rho_ij X_ij,  V3 = sum W_i W_j phi_ij G_ij,
//   alpha_S = sqrt(V1 / T),  nu_S = sqrt(2 V2) / (alpha_S T),  rho_S = clamp(V3 / V1, +-0.999),
// with rho_ij, theta_ij, phi_ij from Eqs. (rhoij), (thetaij), (phiij) at eta1 = eta2 = 0 and
// phi_ii = phi for every forward, and the quadrature of rebonato_caplet.  For a one-period swap
// this is exactly the caplet mapping.
template <class S>
void swap_params(const Market& m, const S* th, int id, S& alpha, S& nu, S& rho, S* V = nullptr) {
  const int a = m.swaps[id].first, b = m.swaps[id].second, Q = m.Q;
  const double TE = m.T[a], D = m.panel;
  const int n = n_panels(TE, D);
  const std::vector<double>& W = m.swapW[id];
  S V1 = 0.0, V2 = 0.0, V3 = 0.0;
  for (int i = a; i < b; ++i) {
    for (int j = a; j < b; ++j) {
      double Ti = m.T[i], Tj = m.T[j], dT = std::fabs(Ti - Tj);
      S rho_ij = exp(-th[9] * dT);
      S theta_ij = exp(-th[10] * dT);
      S phi_ij = th[8] * exp(-th[11] * dT);
      S Gij = 0.0, Xij = 0.0, Hcum = 0.0;
      for (int p = 0; p < n; ++p) {
        double t0 = p * D;
        for (int q = 0; q < Q; ++q) {
          double t = t0 + 0.5 * D * (1.0 + m.xi[q]);
          double wq = 0.5 * D * m.wi[q];
          S gg = g_of(th, Ti - t) * g_of(th, Tj - t);
          double half = 0.5 * (t - t0);
          S part = 0.0;
          for (int r = 0; r < Q; ++r) {
            double s = t0 + half * (1.0 + m.xi[r]);
            part += half * m.wi[r] * h_of(th, Ti - s) * h_of(th, Tj - s);
          }
          Gij += wq * gg;
          Xij += wq * gg * (Hcum + part);
        }
        for (int q = 0; q < Q; ++q) {
          double t = t0 + 0.5 * D * (1.0 + m.xi[q]);
          Hcum += 0.5 * D * m.wi[q] * h_of(th, Ti - t) * h_of(th, Tj - t);
        }
      }
      Xij = theta_ij * Xij;
      double WW = W[i - a] * W[j - a];
      V1 += WW * rho_ij * Gij;
      V2 += WW * rho_ij * Xij;
      V3 += WW * phi_ij * Gij;
    }
  }
  alpha = sqrt(V1 / TE);
  nu = sqrt(2.0 * V2) / (alpha * TE);
  S r = V3 / V1;
  if (val(r) > 0.999) r = S(0.999);
  if (val(r) < -0.999) r = S(-0.999);
  rho = r;
  if (V) { V[0] = V1; V[1] = V2; V[2] = V3; }
}

// ------------------------------------------------------------------ model vols, objective
// ------------------------------------------------------------------ Mercurio & Morini model
// Eq. (haganForMercurio): forward i's SABR alpha is alpha_i exp(int_0^{T_i} M_i(s) ds) with
//   M_i(t) = -sigma sum_{j = h(t)}^{i} tau_j phi_j alpha_j F_j(0)^b / (1 + tau_j F_j(0)),
// h(t) the first forward not yet fixed at t (Eq. h_t: forward j fixes at T_j, so h(t) = k on
// [T_{k-1}, T_k), with T_{-1} = 0).  M_i is constant on each of those intervals, so the integral
// is, interval by interval, its length times the value of M_i there.  The smile of forward i is
// Eq. (sigmaHagan) with beta_i = beta, phi_ii = phi_i, sigma_i = sigma.
// Parameter slots: [phi_0 .. phi_{M-1}, sigma, alpha_0 .. alpha_{M-1}] (M forwards).
template <class S>
S mm_alpha(const Market& m, const S* th, int i) {
  const int M = (int)m.F.size();
  const S& sigma = th[M];
  S integral = 0.0;
  for (int k = 0; k <= i; ++k) {
    const double len = m.T[k] - (k == 0 ? 0.0 : m.T[k - 1]);
    S Mi = 0.0;
    for (int j = k; j <= i; ++j)
      Mi += m.tau[j] * th[j] * th[M + 1 + j] * std::pow(m.F[j], m.beta) / (1.0 + m.tau[j] * m.F[j]);
    integral += len * (-sigma * Mi);
  }
  return th[M + 1 + i] * exp(integral);
}

template <class S>
S model_vol(const Market& m, double F, double K, double T, const S& alpha, const S& rho, const S& nu) {
  if (m.formula == 1) return sabr_paper(F, K, alpha, m.beta, rho, nu);
  return sabr_hagan2002(F, K, T, alpha, m.beta, rho, nu);
}

// Model vols of every instrument (caplets first, then swaptions), per-forward and per-swap SABR
// parameters computed once each.
template <class S>
void all_vols(const Market& m, const S* th, std::vector<S>& vols) {
  const int nc = (int)m.cK.size(), ns = (int)m.sK.size();
  vols.assign(nc + ns, S(0.0));
  std::map<int, std::pair<S, S>> fwd_par;
  for (int k = 0; k < nc; ++k) {
    int i = m.cfwd[k];
    double F = m.F[i], K = m.cK[k], T = m.T[i];
    if (m.model == 0) {
      vols[k] = model_vol(m, F, K, T, th[0], th[1], th[2]);
    } else if (m.model == 2) {
      const int M = (int)m.F.size();
      vols[k] = model_vol(m, F, K, T, mm_alpha(m, th, i), th[i], th[M]);
    } else {
      auto it = fwd_par.find(i);
      if (it == fwd_par.end()) {
        S al, nu;
        rebonato_caplet(m, th, T, al, nu);
        it = fwd_par.emplace(i, std::make_pair(al, nu)).first;
      }
      vols[k] = model_vol(m, F, K, T, it->second.first, th[8], it->second.second);
    }
  }
  std::vector<int> done(m.swaps.size(), 0);
  std::vector<S> sa(m.swaps.size()), sn(m.swaps.size()), sr(m.swaps.size());
  for (int s = 0; s < ns; ++s) {
    int id = m.sswap[s];
    if (!done[id]) { swap_params(m, th, id, sa[id], sn[id], sr[id]); done[id] = 1; }
    vols[nc + s] = model_vol(m, m.swapS[id], m.sK[s], m.T[m.sstart[s]], sa[id], sr[id], sn[id]);
  }
}

// Residuals r_k = sqrt(w_k) (P_k(theta) - P_k^mkt); returns false if any model vol is not a
// finite positive number (the point is infeasible: f = +inf).
template <class S>
bool residuals(const Market& m, const S* th, std::vector<S>& r) {
  std::vector<S> vols;
  all_vols(m, th, vols);
  const int nc = (int)m.cK.size(), ns = (int)m.sK.size();
  r.assign(nc + ns, S(0.0));
  for (int k = 0; k < nc + ns; ++k) {
    double v = val(vols[k]);
    if (!(v > 0.0) || !std::isfinite(v)) return false;
  }
  for (int k = 0; k < nc; ++k) {
    int i = m.cfwd[k];
    S p = black_otm(m.F[i], m.cK[k], m.T[i], vols[k], m.tau[i] * m.P[i + 1]);
    r[k] = std::sqrt(m.cw[k]) * (p - m.cpm[k]);
  }
  for (int s = 0; s < ns; ++s) {
    int id = m.sswap[s];
    S p = black_otm(m.swapS[id], m.sK[s], m.T[m.sstart[s]], vols[nc + s], m.swapA[id]);
    r[nc + s] = std::sqrt(m.sw[s]) * (p - m.spm[s]);
  }
  return true;
}

// f(theta) = sum_k w_k (P_k(theta) - P_k^mkt)^2, summed in instrument order; +inf if infeasible.
// Reading: f_c of Section 3 is a sum of squared vol errors; pricing in price space with
// w_k = 1 / vega_k(sigma_k^mkt)^2 keeps it equal to f_c to first order.
template <class S>
S objective_t(const Market& m, const S* th) {
  std::vector<S> vols;
  all_vols(m, th, vols);
  const int nc = (int)m.cK.size(), ns = (int)m.sK.size();
  S f = 0.0;
  for (int k = 0; k < nc + ns; ++k) {
    double v = val(vols[k]);
    if (!(v > 0.0) || !std::isfinite(v)) return S(std::numeric_limits<double>::infinity());
  }
  for (int k = 0; k < nc; ++k) {
    int i = m.cfwd[k];
    S p = black_otm(m.F[i], m.cK[k], m.T[i], vols[k], m.tau[i] * m.P[i + 1]);
    S e = p - m.cpm[k];
    f += m.cw[k] * e * e;
  }
  for (int s = 0; s < ns; ++s) {
    int id = m.sswap[s];
    S p = black_otm(m.swapS[id], m.sK[s], m.T[m.sstart[s]], vols[nc + s], m.swapA[id]);
    S e = p - m.spm[s];
    f += m.sw[s] * e * e;
  }
  if (!std::isfinite(val(f))) return S(std::numeric_limits<double>::infinity());
  return f;
}

static double objective(const Market& m, const double* th) { return objective_t<double>(m, th); }

// RMSE of model vols against market vols, in vol points.
static double rmse_volpt(const Market& m, const double* th) {
  std::vector<double> vols;
  all_vols(m, th, vols);
  const int nc = (int)m.cK.size();
  double s = 0.0;
  for (size_t k = 0; k < vols.size(); ++k) {
    double mk = k < (size_t)nc ? m.cvol[k] : m.svol[k - nc];
    double e = vols[k] - mk;
    s += e * e;
  }
  return 100.0 * std::sqrt(s / (double)vols.size());
}

static void seed_duals(const Market& m, const double* th, std::vector<Dual>& x) {
  x.assign(m.n_param, Dual(0.0));
  for (int k = 0; k < m.n_param; ++k) { x[k] = Dual(th[k]); x[k].d[k] = 1.0; }
}

// ------------------------------------------------------------------ Philox4x64-10
// Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3" (SC'11): ten rounds
// of two 64x64->128 multiplications with the Weyl key schedule.
static void philox4x64_10(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4]) {
  const uint64_t M0 = 0xD2E7470EE14C6C93ULL, M1 = 0xCA5A826395121157ULL;
  const uint64_t W0 = 0x9E3779B97F4A7C15ULL, W1 = 0xBB67AE8584CAA73BULL;
  uint64_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3], k0 = key[0], k1 = key[1];
  for (int r = 0; r < 10; ++r) {
    unsigned __int128 p0 = (unsigned __int128)M0 * c0;
    unsigned __int128 p1 = (unsigned __int128)M1 * c2;
    uint64_t hi0 = (uint64_t)(p0 >> 64), lo0 = (uint64_t)p0;
    uint64_t hi1 = (uint64_t)(p1 >> 64), lo1 = (uint64_t)p1;
    uint64_t n0 = hi1 ^ c1 ^ k0, n1 = lo1, n2 = hi0 ^ c3 ^ k1, n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    k0 += W0; k1 += W1;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

// The uniforms of one annealing step: block b of step s, level l, chain c (market index in the
// upper half of the chain word) under key (seed, 0); word j of the step is uniform j,
// u = (x >> 11) 2^-53 in [0, 1).
static void step_uniforms(uint64_t seed, uint64_t chain_word, int level, int step, int count, double* u) {
  uint64_t key[2] = {seed, 0};
  for (int b = 0; b * 4 < count; ++b) {
    uint64_t ctr[4] = {(uint64_t)b, (uint64_t)step, (uint64_t)level, chain_word};
    uint64_t o[4];
    philox4x64_10(ctr, key, o);
    for (int w = 0; w < 4 && 4 * b + w < count; ++w) u[4 * b + w] = (double)(o[w] >> 11) * 0x1.0p-53;
  }
}

// ------------------------------------------------------------------ Philox4x32-10
// The 32-bit member of the same family (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two
// 32x32->64 multiplications with the Weyl key schedule.  It feeds the Monte Carlo pricer.
static void philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u, W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3], k0 = key[0], k1 = key[1];
  for (int r = 0; r < 10; ++r) {
    const uint64_t p0 = (uint64_t)M0 * c0, p1 = (uint64_t)M1 * c2;
    const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0, hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    c0 = hi1 ^ c1 ^ k0; c1 = lo1; c2 = hi0 ^ c3 ^ k1; c3 = lo0;
    k0 += W0; k1 += W1;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

// Normals r = 4b .. 4b + 3 of time step `step` of path `path`: Philox4x32-10 at counter
// (b, step, path, 0) under key (seed low word, seed high word); uniforms u = (x + 1/2) 2^-32 in
// (0, 1); Box-Muller on the pairs (u0, u1) and (u2, u3): sqrt(-2 ln u_even) (cos, sin)(2 pi u_odd).
static void mc_normals4(uint64_t seed, uint64_t path, int step, int b, double* z) {
  const uint32_t ctr[4] = {(uint32_t)b, (uint32_t)step, (uint32_t)path, (uint32_t)(path >> 32)};
  const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  uint32_t o[4];
  philox4x32_10(ctr, key, o);
  for (int q = 0; q < 2; ++q) {
    const double u0 = ((double)o[2 * q] + 0.5) * 0x1.0p-32, u1 = ((double)o[2 * q + 1] + 0.5) * 0x1.0p-32;
    const double r = std::sqrt(-2.0 * std::log(u0));
    z[2 * q] = r * std::cos(2.0 * M_PI * u1);
    z[2 * q + 1] = r * std::sin(2.0 * M_PI * u1);
  }
}

// ------------------------------------------------------------------ Monte Carlo pricer
// The Hagan SABR/LIBOR model (Section 2.1, Eqs. dinamicasHagan1-2) under the spot measure:
//   dF_i = mu^F_i dt + V_i F_i^b dW_i,   dV_i = mu^V_i dt + sigma_i V_i dZ_i,
//   mu^F_i = V_i F_i^b sum_{j = h(t)}^{i} tau_j rho_ij V_j F_j^b / (1 + tau_j F_j),
//   mu^V_i = sigma_i V_i sum_{j = h(t)}^{i} tau_j phi_ij V_j F_j^b / (1 + tau_j F_j),
// V_i(0) = alpha_i, correlations rho_ij, theta_ij, phi_ij of Eqs. (rhoij), (thetaij), (phiij)
// (phi_ij from the phi_ii), h(t) the first forward not yet fixed (Eq. h_t, forward j fixing at T_j).
// phi_ij is the correlation of W_i with Z_j (the block of Section 2.1); the vol drift takes it with
// the indices as printed.
// Readings (the paper prints no scheme): Euler steps in F, absorbed at zero (for b < 1 the CEV
// forward reaches zero; its drift and diffusion both carry F^b, so it stays there), log-Euler steps
// in ln V, the drifts frozen over a step; a path whose state (F or ln V) is not finite at a fixing
// date pays nothing from there on and is counted (n_bad); the simulation ends at the last fixing
// an instrument needs; every interval [T_{k-1}, T_k] (T_{-1} = 0) is cut into ceil(len / dt) equal steps,
// so the fixings fall on the grid; the Brownian increments of a step are L xi with xi standard
// normals (mc_normals4, numbered r = 0, 1, ... within the step) and L the Cholesky factor of the
// correlation matrix of (W, Z) ordered by forward, last forward first, W before Z (row 2(M-1-i)
// is W_i, row 2(M-1-i) + 1 is Z_i): the forwards still alive are then the leading rows.  The spot
// numeraire rolls over at the fixings, B(T_{i+1}) = prod_{k <= i} (1 + tau_k F_k(T_k)) / P(0, T_0).
//   caplet on forward i, strike K: tau_i (F_i(T_i) - K)^+ paid at T_{i+1};
//   swaption on the swap over [a, b), strike K: A(T_a) (S(T_a) - K)^+ at T_a, the annuity
//   A = sum_k tau_k P(T_a, T_{k+1}) and S = (1 - P(T_a, T_b)) / A from the forwards at T_a.
// price[k] = mean over all paths of the deflated payoff; sq[k] = mean of its square.
struct McModel {
  int M;                       // forwards simulated
  int model = 0;               // 0: Hagan (Section 2.1); 2: Mercurio & Morini (Section 2.2)
  double beta, eta1, lambda1, eta2, lambda2, lambda3;
  std::vector<double> alpha, sigma, phi;   // per forward: V_i(0), vol of vol, phi_ii (Hagan);
                                           // alpha_i, the common sigma (sigma[0]), phi_i (MM)
};

// The Mercurio & Morini dynamics (Section 2.2, Eqs. dinamicasMercurio1-2) under the spot measure:
//   dF_i = mu^F_i dt + alpha_i V F_i^b dW_i,  dV = sigma V dZ,  V(0) = 1,
//   mu^F_i = alpha_i V F_i^b sum_{j = h(t)}^{i} tau_j rho_ij alpha_j V F_j^b / (1 + tau_j F_j),
// corr(W_i, W_j) = rho_ij of Eq. (rhoij), corr(W_i, Z) = phi_i; V has no drift (as printed).  The
// increments are L xi with L the Cholesky factor of the correlation matrix ordered Z first, then
// the forwards last first (row 0 is Z, row 1 + (M - 1 - i) is W_i): the alive forwards again lead.

static bool mc_cholesky(const Market& m, const McModel& md, std::vector<double>& L, std::vector<double>& C) {
  const bool mm = md.model == 2;
  const int n = mm ? md.M + 1 : 2 * md.M;
  C.assign((size_t)n * n, 0.0);
  auto fwd = [&](int r) { return md.M - 1 - r / 2; };
  if (mm) {
    for (int r = 0; r < n; ++r)
      for (int c = 0; c < n; ++c) {
        double v;
        if (r == 0 && c == 0) v = 1.0;
        else if (r == 0 || c == 0) v = md.phi[md.M - 1 - (r + c - 1)];      // corr(W_i, Z) = phi_i
        else {
          const int i = md.M - r, j = md.M - c;                               // row 1 + (M - 1 - i)
          v = md.eta1 + (1.0 - md.eta1) * std::exp(-md.lambda1 * std::fabs(m.T[i] - m.T[j]));
        }
        C[(size_t)r * n + c] = v;
      }
  }
  for (int r = 0; r < n && !mm; ++r)
    for (int c = 0; c < n; ++c) {
      const int i = fwd(r), j = fwd(c);
      const bool wi = (r % 2) == 0, wj = (c % 2) == 0;
      const double dT = std::fabs(m.T[i] - m.T[j]);
      double v;
      if (wi && wj) v = md.eta1 + (1.0 - md.eta1) * std::exp(-md.lambda1 * dT);          // rho_ij
      else if (!wi && !wj) v = md.eta2 + (1.0 - md.eta2) * std::exp(-md.lambda2 * dT);   // theta_ij
      else {                                                                             // phi_ij (W_i with Z_j)
        const int a = wi ? i : j, b = wi ? j : i;
        const double pa = md.phi[a], pb = md.phi[b];
        v = (pa < 0 ? -1.0 : 1.0) * std::sqrt(std::fabs(pa * pb)) * std::exp(-md.lambda3 * std::fabs(m.T[a] - m.T[b]));
      }
      C[(size_t)r * n + c] = v;
    }
  // Reading: with phi_ii of both signs Eq. (phiij) can make the matrix indefinite (the paper's own
  // calibrated Hagan parameters do); it is then replaced by the nearest correlation matrix in the
  // spectral sense (Rebonato and Jaeckel): eigenvalues below zero set to zero, B = S Lambda^(1/2)
  // with every row scaled to unit length, C = B B^T.  Eigen-decomposition by cyclic Jacobi rotations.
  // The repaired matrix replaces the printed one everywhere (increments and drifts), so that the
  // discretised model stays free of arbitrage.
  {
    std::vector<double> A = C, S((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i) S[(size_t)i * n + i] = 1.0;
    for (int sweep = 0; sweep < 100; ++sweep) {
      double off = 0.0;
      for (int i = 0; i < n; ++i)
        for (int j = i + 1; j < n; ++j) off += A[(size_t)i * n + j] * A[(size_t)i * n + j];
      if (off < 1e-30) break;
      for (int p = 0; p < n; ++p)
        for (int q = p + 1; q < n; ++q) {
          const double apq = A[(size_t)p * n + q];
          if (std::fabs(apq) < 1e-300) continue;
          const double th = (A[(size_t)q * n + q] - A[(size_t)p * n + p]) / (2.0 * apq);
          const double t = (th >= 0 ? 1.0 : -1.0) / (std::fabs(th) + std::sqrt(th * th + 1.0));
          const double c = 1.0 / std::sqrt(t * t + 1.0), sn = t * c;
          for (int k = 0; k < n; ++k) {   // A <- A J (columns p, q)
            const double akp = A[(size_t)k * n + p], akq = A[(size_t)k * n + q];
            A[(size_t)k * n + p] = c * akp - sn * akq;
            A[(size_t)k * n + q] = sn * akp + c * akq;
          }
          for (int k = 0; k < n; ++k) {   // A <- J^T A (rows p, q)
            const double apk = A[(size_t)p * n + k], aqk = A[(size_t)q * n + k];
            A[(size_t)p * n + k] = c * apk - sn * aqk;
            A[(size_t)q * n + k] = sn * apk + c * aqk;
          }
          for (int k = 0; k < n; ++k) {   // S <- S J
            const double skp = S[(size_t)k * n + p], skq = S[(size_t)k * n + q];
            S[(size_t)k * n + p] = c * skp - sn * skq;
            S[(size_t)k * n + q] = sn * skp + c * skq;
          }
        }
    }
    bool neg = false;
    for (int i = 0; i < n; ++i) neg = neg || A[(size_t)i * n + i] < 0.0;
    if (neg) {
      std::vector<double> B((size_t)n * n);
      for (int i = 0; i < n; ++i) {
        double nrm = 0.0;
        for (int k = 0; k < n; ++k) {
          const double v = S[(size_t)i * n + k] * std::sqrt(std::max(A[(size_t)k * n + k], 0.0));
          B[(size_t)i * n + k] = v;
          nrm += v * v;
        }
        for (int k = 0; k < n; ++k) B[(size_t)i * n + k] /= std::sqrt(nrm);
      }
      for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
          double v = 0.0;
          for (int k = 0; k < n; ++k) v += B[(size_t)i * n + k] * B[(size_t)j * n + k];
          C[(size_t)i * n + j] = v;
        }
    }
  }
  // Cholesky factor, semi-definite: a pivot at or below 1e-12 ends its column (no new noise there)
  L.assign((size_t)n * n, 0.0);
  for (int j = 0; j < n; ++j) {
    double d = C[(size_t)j * n + j];
    for (int k = 0; k < j; ++k) d -= L[(size_t)j * n + k] * L[(size_t)j * n + k];
    if (!(d > 1e-12)) continue;
    d = std::sqrt(d);
    L[(size_t)j * n + j] = d;
    for (int i = j + 1; i < n; ++i) {
      double t = C[(size_t)i * n + j];
      for (int k = 0; k < j; ++k) t -= L[(size_t)i * n + k] * L[(size_t)j * n + k];
      L[(size_t)i * n + j] = t / d;
    }
  }
  return true;
}

static int mc_price(const Market& m, const McModel& md, int n_cap, const int* cap_fwd, const double* cap_K,
                    int n_swp, const int* swp_a, const int* swp_b, const double* swp_K, int64_t n_paths, double dt,
                    uint64_t seed, int n_threads, double* price, double* sq, int64_t* n_bad) {
  const bool mm = md.model == 2;
  const int M = md.M, n = mm ? M + 1 : 2 * M, ni = n_cap + n_swp;
  std::vector<double> L, Cr;
  if (!mc_cholesky(m, md, L, Cr)) return 1;
  // the correlations the drifts use: those of the (repaired) matrix the increments are drawn from
  auto rho = [&](int i, int j) {
    return mm ? Cr[(size_t)(M - i) * n + (M - j)] : Cr[(size_t)(2 * (M - 1 - i)) * n + 2 * (M - 1 - j)];
  };
  auto phi = [&](int i, int j) { return Cr[(size_t)(2 * (M - 1 - i)) * n + 2 * (M - 1 - j) + 1]; };
  // the time grid: interval k ends at T_k
  std::vector<int> nsteps(M);
  for (int k = 0; k < M; ++k) {
    const double len = m.T[k] - (k == 0 ? 0.0 : m.T[k - 1]);
    nsteps[k] = std::max(1, (int)std::ceil(len / dt - 1e-9));
  }
  // the simulation ends at the last fixing an instrument needs
  int K_end = 1;
  for (int c = 0; c < n_cap; ++c) K_end = std::max(K_end, cap_fwd[c] + 1);
  for (int c = 0; c < n_swp; ++c) K_end = std::max(K_end, swp_a[c] + 1);
  std::vector<double> sum(ni, 0.0), sum2(ni, 0.0);
  int64_t bad = 0;
#pragma omp parallel num_threads(n_threads > 0 ? n_threads : 1)
  {
    std::vector<double> ls(ni, 0.0), ls2(ni, 0.0);
    int64_t lbad = 0;
    std::vector<double> lnV(M), F(M), V(M), x(M), DF(M), DV(M), xi(n + 4), Z(n), fix(M), numer(M + 1);
    std::vector<std::vector<double>> snap(M, std::vector<double>(M, 0.0));   // forwards at each fixing date
    std::vector<char> good(M);
#pragma omp for schedule(static)
    for (int64_t p = 0; p < n_paths; ++p) {
      for (int i = 0; i < M; ++i) { F[i] = m.F[i]; lnV[i] = mm ? 0.0 : std::log(md.alpha[i]); }
      int step = 0;
      for (int k = 0; k < K_end; ++k) {      // interval k: forwards k .. M-1 alive (h(t) = k)
        const double h = (m.T[k] - (k == 0 ? 0.0 : m.T[k - 1])) / nsteps[k];
        const int na = mm ? 1 + (M - k) : 2 * (M - k);   // alive rows of L
        for (int s = 0; s < nsteps[k]; ++s, ++step) {
          for (int b = 0; 4 * b < na; ++b) mc_normals4(seed, (uint64_t)p, step, b, &xi[4 * b]);
          for (int r = 0; r < na; ++r) {
            double z = 0.0;
            for (int c = 0; c <= r; ++c) z += L[(size_t)r * n + c] * xi[c];
            Z[r] = z;
          }
          if (mm) {   // the Mercurio & Morini step: one vol process for every forward
            const double Vc = std::exp(lnV[0]);
            for (int i = k; i < M; ++i)
              x[i] = m.tau[i] * md.alpha[i] * std::pow(F[i], md.beta) / (1.0 + m.tau[i] * F[i]);
            for (int i = k; i < M; ++i) {
              double dF = 0.0;
              for (int j = k; j <= i; ++j) dF += rho(i, j) * x[j];
              DF[i] = dF;
            }
            for (int i = k; i < M; ++i) {
              const double vf = md.alpha[i] * Vc * std::pow(F[i], md.beta);   // alpha_i V F_i^b
              const double fn = F[i] + vf * Vc * DF[i] * h + vf * std::sqrt(h) * Z[M - i];
              F[i] = fn > 0.0 ? fn : 0.0;
            }
            lnV[0] += -0.5 * md.sigma[0] * md.sigma[0] * h + md.sigma[0] * std::sqrt(h) * Z[0];
            continue;
          }
          for (int i = k; i < M; ++i) V[i] = std::exp(lnV[i]);
          for (int i = k; i < M; ++i)
            x[i] = m.tau[i] * V[i] * std::pow(F[i], md.beta) / (1.0 + m.tau[i] * F[i]);
          for (int i = k; i < M; ++i) {
            double dF = 0.0, dV = 0.0;
            for (int j = k; j <= i; ++j) {
              dF += rho(i, j) * x[j];
              dV += phi(i, j) * x[j];
            }
            DF[i] = dF;
            DV[i] = dV;
          }
          for (int i = k; i < M; ++i) {
            const double vf = V[i] * std::pow(F[i], md.beta);          // V_i F_i^b
            const int rw = 2 * (M - 1 - i);
            const double fn = F[i] + vf * DF[i] * h + vf * std::sqrt(h) * Z[rw];
            F[i] = fn > 0.0 ? fn : 0.0;
            lnV[i] += (md.sigma[i] * DV[i] - 0.5 * md.sigma[i] * md.sigma[i]) * h + md.sigma[i] * std::sqrt(h) * Z[rw + 1];
          }
        }
        bool fin = true;
        for (int i = k; i < M; ++i) {
          snap[k][i] = F[i];   // the forwards at T_k
          fin = fin && std::isfinite(F[i]) && std::isfinite(lnV[mm ? 0 : i]);
        }
        good[k] = fin && (k == 0 || good[k - 1]);
        fix[k] = snap[k][k];
      }
      // a path whose state leaves the finite numbers at a fixing date (the vol process can explode:
      // its spot-measure drift grows with the vols) is stopped there: it pays nothing from that date
      // on, and it is counted
      if (!good[K_end - 1]) ++lbad;
      // deflators: 1 / B(T_{i+1}) = P(0, T_0) / prod_{k <= i} (1 + tau_k F_k(T_k)); numer[i] = 1 / B(T_i)
      numer[0] = m.P[0];
      for (int k = 0; k < K_end; ++k) numer[k + 1] = numer[k] / (1.0 + m.tau[k] * fix[k]);
      for (int c = 0; c < n_cap; ++c) {
        const int i = cap_fwd[c];
        if (!good[i]) continue;
        const double pay = m.tau[i] * std::max(fix[i] - cap_K[c], 0.0) * numer[i + 1];
        ls[c] += pay;
        ls2[c] += pay * pay;
      }
      for (int c = 0; c < n_swp; ++c) {
        const int a = swp_a[c], b = swp_b[c];
        if (!good[a]) continue;
        double disc = 1.0, A = 0.0;
        for (int j = a; j < b; ++j) {
          disc /= 1.0 + m.tau[j] * snap[a][j];
          A += m.tau[j] * disc;
        }
        const double S = (1.0 - disc) / A;
        const double pay = A * std::max(S - swp_K[c], 0.0) * numer[a];
        ls[n_cap + c] += pay;
        ls2[n_cap + c] += pay * pay;
      }
    }
#pragma omp critical
    {
      for (int c = 0; c < ni; ++c) { sum[c] += ls[c]; sum2[c] += ls2[c]; }
      bad += lbad;
    }
  }
  for (int c = 0; c < ni; ++c) { price[c] = sum[c] / (double)n_paths; sq[c] = sum2[c] / (double)n_paths; }
  if (n_bad) *n_bad = bad;
  return 0;
}

// ------------------------------------------------------------------ simulated annealing
struct SAOpts {  // mirrors oracle/__init__.py
  int32_t n_chains, n_levels, steps;
  double T0, cooling, step_frac, step_floor;
  uint64_t seed;
  uint64_t market_index;
  const double* x0;
  int32_t n_threads;
};

// Neighbour (reading; the paper leaves ComputeNeighbour open): every free slot moves by
// sf (hi - lo) (2u - 1), is reflected once at the bound it crossed and then clamped.
// The search box of an annealing run: P slots, bounds and the slots that move.
struct Box {
  int P;
  const double* lo;
  const double* hi;
  const uint8_t* freem;
};

static void neighbour(const Box& bx, const double* x, const double* u, double sf, double* y) {
  for (int k = 0; k < bx.P; ++k) {
    if (!bx.freem[k]) { y[k] = x[k]; continue; }
    double v = x[k] + sf * (bx.hi[k] - bx.lo[k]) * (2.0 * u[k] - 1.0);
    if (v < bx.lo[k]) v = 2.0 * bx.lo[k] - v;
    if (v > bx.hi[k]) v = 2.0 * bx.hi[k] - v;
    if (v < bx.lo[k]) v = bx.lo[k];
    if (v > bx.hi[k]) v = bx.hi[k];
    y[k] = v;
  }
}

// The annealing loop of Section 3 in its one-GPU parallel form: at each temperature every chain
// runs `steps` Metropolis steps from the shared start point; the start point of the next level
// is the chain end point with the lowest f (ties to the lowest chain index).  T_{l+1} = cooling T_l.
// Readings: T0 <= 0 means T0 = f(x0); the step fraction of level l is
// max(step_frac sqrt(T_l / T0), step_floor); every chain evaluates f(x0) once, so the count of
// objective evaluations is C (L N + 1); the best point ever accepted is kept apart and returned.
// (The loop is written once for any objective f over a box: the calibration objective of a
// market, or the Monte Carlo objective of mc_anneal.)
template <class Obj>
static int anneal_box(const Box& bx, Obj objective_of, const SAOpts& o, double* x_best, double* f_best,
                      double* chain_xb, double* chain_fb, double* trace_f, double* trace_x,
                      uint8_t* bits, int64_t* n_evals, double* T0_used) {
  const int P = bx.P, C = o.n_chains, L = o.n_levels, N = o.steps;
  std::vector<double> x0(P);
  for (int k = 0; k < P; ++k) x0[k] = o.x0 ? o.x0[k] : 0.5 * (bx.lo[k] + bx.hi[k]);
  double f0 = objective_of(x0.data());
  double T0 = o.T0 > 0.0 ? o.T0 : ((std::isfinite(f0) && f0 > 0.0) ? f0 : 1.0);
  std::vector<double> xs = x0, xb((size_t)C * P), fb(C, f0), xe((size_t)C * P), fe(C);
  for (int c = 0; c < C; ++c) std::copy(x0.begin(), x0.end(), xb.begin() + (size_t)c * P);
  double fs = f0;
  double T = T0;
  for (int l = 0; l < L; ++l) {
    double sf = std::max(o.step_frac * std::sqrt(T / T0), o.step_floor);
#pragma omp parallel for schedule(dynamic, 1) num_threads(o.n_threads > 0 ? o.n_threads : 1)
    for (int c = 0; c < C; ++c) {
      std::vector<double> x(xs), y(P), u(P + 1);
      double f = fs;
      uint64_t cw = (uint64_t)c | (o.market_index << 32);
      for (int s = 0; s < N; ++s) {
        step_uniforms(o.seed, cw, l, s, P + 1, u.data());
        neighbour(bx, x.data(), u.data(), sf, y.data());
        double fy = objective_of(y.data());
        if (!(fy == fy)) fy = std::numeric_limits<double>::infinity();
        bool acc = (fy < f) || (u[P] < std::exp(-(fy - f) / T));
        if (bits) bits[((size_t)c * L + l) * N + s] = acc ? 1 : 0;
        if (acc) {
          x = y; f = fy;
          if (f < fb[c]) { fb[c] = f; std::copy(x.begin(), x.end(), xb.begin() + (size_t)c * P); }
        }
      }
      std::copy(x.begin(), x.end(), xe.begin() + (size_t)c * P);
      fe[c] = f;
    }
    int best = 0;
    for (int c = 1; c < C; ++c) if (fe[c] < fe[best]) best = c;
    std::copy(xe.begin() + (size_t)best * P, xe.begin() + (size_t)(best + 1) * P, xs.begin());
    fs = fe[best];
    if (trace_f) trace_f[l] = fs;
    if (trace_x) std::copy(xs.begin(), xs.end(), trace_x + (size_t)l * P);
    T = T * o.cooling;
  }
  int best = 0;
  for (int c = 1; c < C; ++c) if (fb[c] < fb[best]) best = c;
  std::copy(xb.begin() + (size_t)best * P, xb.begin() + (size_t)(best + 1) * P, x_best);
  *f_best = fb[best];
  if (chain_xb) std::copy(xb.begin(), xb.end(), chain_xb);
  if (chain_fb) std::copy(fb.begin(), fb.end(), chain_fb);
  if (n_evals) *n_evals = (int64_t)C * ((int64_t)L * N + 1);
  if (T0_used) *T0_used = T0;
  return 0;
}

static int anneal(const Market& m, const SAOpts& o, double* x_best, double* f_best,
                  double* chain_xb, double* chain_fb, double* trace_f, double* trace_x,
                  uint8_t* bits, int64_t* n_evals, double* T0_used) {
  const Box bx{m.n_param, m.lo.data(), m.hi.data(), m.freem.data()};
  return anneal_box(bx, [&](const double* y) { return objective(m, y); }, o, x_best, f_best, chain_xb, chain_fb,
                    trace_f, trace_x, bits, n_evals, T0_used);
}

// ------------------------------------------------------------------ SA over the Monte Carlo objective
// The swaption calibration of Section 3: the correlation parameters y = (eta1, lambda1, eta2,
// lambda2, lambda3) minimise f_s(y) = sum_k (P_k^Black - P_k^MC(y))^2 over the instruments, with the
// caplet-calibrated alpha_i, sigma_i, phi_ii fixed.  Every evaluation prices with the same paths
// (one Monte Carlo seed: common random numbers, so f_s is a deterministic function of y), and the
// annealing loop above searches the box.  The market prices: Black's formula at the quoted vols
// (payer swaption: annuity A = sum_{k in [a, b)} tau_k P(0, T_{k+1}), swap rate (P(0, T_a) - P(0, T_b)) / A,
// expiry T_a; caplet: discount tau_i P(0, T_{i+1}), forward F_i(0), expiry T_i).  A y whose Monte
// Carlo cannot run (a non-finite price) has f_s = +inf.
struct McTarget {
  int n_cap, n_swp;
  const int *cap_fwd, *swp_a, *swp_b;
  const double *cap_K, *swp_K;
  std::vector<double> price;   // market prices, caplets then swaptions
};

static McTarget mc_target(const Market& m, int n_cap, const int* cap_fwd, const double* cap_K, int n_swp,
                          const int* swp_a, const int* swp_b, const double* swp_K, const double* quote_vol) {
  McTarget t{n_cap, n_swp, cap_fwd, swp_a, swp_b, cap_K, swp_K, {}};
  for (int c = 0; c < n_cap; ++c) {
    const int i = cap_fwd[c];
    t.price.push_back(black_call(m.F[i], cap_K[c], m.T[i], quote_vol[c], m.tau[i] * m.P[i + 1]));
  }
  for (int c = 0; c < n_swp; ++c) {
    const int a = swp_a[c], b = swp_b[c];
    double A = 0.0;
    for (int k = a; k < b; ++k) A += m.tau[k] * m.P[k + 1];
    const double S = (m.P[a] - m.P[b]) / A;
    t.price.push_back(black_call(S, swp_K[c], m.T[a], quote_vol[n_cap + c], A));
  }
  return t;
}

static double mc_objective(const Market& m, McModel md, const McTarget& t, const double* y, int64_t n_paths,
                           double dt, uint64_t mc_seed, int n_threads) {
  md.eta1 = y[0]; md.lambda1 = y[1]; md.eta2 = y[2]; md.lambda2 = y[3]; md.lambda3 = y[4];
  const int ni = t.n_cap + t.n_swp;
  std::vector<double> price(ni), sq(ni);
  int64_t bad = 0;
  if (mc_price(m, md, t.n_cap, t.cap_fwd, t.cap_K, t.n_swp, t.swp_a, t.swp_b, t.swp_K, n_paths, dt, mc_seed,
               n_threads, price.data(), sq.data(), &bad) != 0)
    return std::numeric_limits<double>::infinity();
  double f = 0.0;
  for (int k = 0; k < ni; ++k) {
    const double e = price[k] - t.price[k];
    f += e * e;
  }
  return std::isfinite(f) ? f : std::numeric_limits<double>::infinity();
}

// ------------------------------------------------------------------ Levenberg-Marquardt
// Classic LM with Marquardt's diagonal scaling: solve (J^T J + mu diag(J^T J)) d = -J^T r over
// the free slots by Cholesky, project theta + d on the box, accept if f drops (mu /= 10), else
// mu *= 10.  Stops at the target RMSE (vol points), after max_iter accepted or rejected trials,
// or when mu exceeds 1e16.  Reading: a zero diagonal entry is floored at 1e-12 of the largest.
static bool cholesky_solve(std::vector<double> A, std::vector<double> b, int n, std::vector<double>& x) {
  for (int j = 0; j < n; ++j) {
    double s = A[j * n + j];
    for (int k = 0; k < j; ++k) s -= A[j * n + k] * A[j * n + k];
    if (!(s > 0.0)) return false;
    double d = std::sqrt(s);
    A[j * n + j] = d;
    for (int i = j + 1; i < n; ++i) {
      double t = A[i * n + j];
      for (int k = 0; k < j; ++k) t -= A[i * n + k] * A[j * n + k];
      A[i * n + j] = t / d;
    }
  }
  for (int i = 0; i < n; ++i) {
    double t = b[i];
    for (int k = 0; k < i; ++k) t -= A[i * n + k] * b[k];
    b[i] = t / A[i * n + i];
  }
  for (int i = n - 1; i >= 0; --i) {
    double t = b[i];
    for (int k = i + 1; k < n; ++k) t -= A[k * n + i] * b[k];
    b[i] = t / A[i * n + i];
  }
  x = b;
  return true;
}

static int lm(const Market& m, const double* theta0, int max_iter, double target_rmse, double mu0,
              double* theta_out, double* f_out, double* rmse_out, int* iters_out) {
  const int P = m.n_param;
  std::vector<int> fi;
  for (int k = 0; k < P; ++k) if (m.freem[k]) fi.push_back(k);
  const int nf = (int)fi.size();
  std::vector<double> th(theta0, theta0 + P);
  double f = objective(m, th.data());
  double mu = mu0;
  int it = 0;
  for (; it < max_iter; ++it) {
    if (rmse_volpt(m, th.data()) <= target_rmse) break;
    std::vector<Dual> xd;
    seed_duals(m, th.data(), xd);
    std::vector<Dual> r;
    if (!residuals(m, xd.data(), r)) break;
    std::vector<double> A((size_t)nf * nf, 0.0), g(nf, 0.0);
    for (const Dual& rk : r) {
      for (int a = 0; a < nf; ++a) {
        g[a] += rk.d[fi[a]] * rk.v;
        for (int b = 0; b < nf; ++b) A[a * nf + b] += rk.d[fi[a]] * rk.d[fi[b]];
      }
    }
    double dmax = 0.0;
    for (int a = 0; a < nf; ++a) dmax = std::max(dmax, A[a * nf + a]);
    bool improved = false;
    while (mu < 1e16) {
      std::vector<double> M = A, rhs(nf), d;
      for (int a = 0; a < nf; ++a) {
        M[a * nf + a] += mu * std::max(A[a * nf + a], 1e-12 * dmax);
        rhs[a] = -g[a];
      }
      if (cholesky_solve(M, rhs, nf, d)) {
        std::vector<double> tn = th;
        for (int a = 0; a < nf; ++a) {
          int k = fi[a];
          tn[k] = std::min(std::max(th[k] + d[a], m.lo[k]), m.hi[k]);
        }
        double fn = objective(m, tn.data());
        if (fn < f) { th = tn; f = fn; mu = std::max(mu / 10.0, 1e-12); improved = true; break; }
      }
      mu *= 10.0;
    }
    if (!improved) break;
  }
  std::copy(th.begin(), th.end(), theta_out);
  *f_out = f;
  *rmse_out = rmse_volpt(m, th.data());
  *iters_out = it;
  return 0;
}

// Nelder-Mead simplex descent on the free slots: the local search that follows the annealing in the
// paper's hybrid scheme (Section 3), with the standard coefficients (reflection 1, expansion 2,
// contraction 1/2, shrink 1/2) of Lagarias, Reeds, Wright and Wright (1998).  Every trial point is
// projected onto the box.  Initial simplex: x0 and, per free slot k, x0 + step (hi_k - lo_k) e_k
// (the step taken downwards where it would leave the box).  Vertices are ordered by f with a stable
// insertion sort of the previous order.  Stops after max_iter iterations, or once
// f_worst - f_best <= ftol |f_best|.
static int nm(const Market& m, const double* theta0, int max_iter, double step, double ftol,
              double* theta_out, double* f_out, int* iters_out, int* evals_out) {
  const int P = m.n_param;
  std::vector<int> fi;
  for (int k = 0; k < P; ++k) if (m.freem[k]) fi.push_back(k);
  const int nf = (int)fi.size();
  auto project = [&](std::vector<double>& x) {
    for (int s : fi) x[s] = std::min(std::max(x[s], m.lo[s]), m.hi[s]);
  };
  std::vector<std::vector<double>> V(nf + 1, std::vector<double>(theta0, theta0 + P));
  std::vector<double> F(nf + 1);
  int evals = 0;
  auto eval = [&](const std::vector<double>& x) { ++evals; return objective(m, x.data()); };
  for (int k = 1; k <= nf; ++k) {
    const int s = fi[k - 1];
    const double d = step * (m.hi[s] - m.lo[s]);
    double v = theta0[s] + d;
    if (v > m.hi[s]) v = theta0[s] - d;
    V[k][s] = v;
    project(V[k]);
  }
  for (int k = 0; k <= nf; ++k) F[k] = eval(V[k]);
  std::vector<int> idx(nf + 1);
  for (int k = 0; k <= nf; ++k) idx[k] = k;
  int it = 0;
  std::vector<double> c(P), xr(P), xt(P);
  for (;; ++it) {
    for (int i = 1; i <= nf; ++i)
      for (int j = i; j > 0 && F[idx[j - 1]] > F[idx[j]]; --j) std::swap(idx[j - 1], idx[j]);
    const int b = idx[0], w = idx[nf], sw = idx[nf > 0 ? nf - 1 : 0];
    if (it >= max_iter || nf == 0 || !std::isfinite(F[b]) || F[w] - F[b] <= ftol * std::fabs(F[b])) break;
    c = V[b];
    for (int s : fi) {
      double t = 0.0;
      for (int j = 0; j < nf; ++j) t += V[idx[j]][s];
      c[s] = t / nf;
    }
    xr = c;
    for (int s : fi) xr[s] = c[s] + (c[s] - V[w][s]);
    project(xr);
    const double fr = eval(xr);
    if (F[b] <= fr && fr < F[sw]) {
      V[w] = xr; F[w] = fr;
      continue;
    }
    if (fr < F[b]) {
      xt = c;
      for (int s : fi) xt[s] = c[s] + 2.0 * (xr[s] - c[s]);
      project(xt);
      const double fe = eval(xt);
      if (fe < fr) { V[w] = xt; F[w] = fe; } else { V[w] = xr; F[w] = fr; }
      continue;
    }
    xt = c;
    bool accept;
    double ft;
    if (fr < F[w]) {   // outside contraction
      for (int s : fi) xt[s] = c[s] + 0.5 * (xr[s] - c[s]);
      project(xt);
      ft = eval(xt);
      accept = ft <= fr;
    } else {           // inside contraction
      for (int s : fi) xt[s] = c[s] + 0.5 * (V[w][s] - c[s]);
      project(xt);
      ft = eval(xt);
      accept = ft < F[w];
    }
    if (accept) { V[w] = xt; F[w] = ft; continue; }
    for (int j = 1; j <= nf; ++j) {   // shrink towards the best vertex
      const int v = idx[j];
      for (int s : fi) V[v][s] = V[b][s] + 0.5 * (V[v][s] - V[b][s]);
      project(V[v]);
      F[v] = eval(V[v]);
    }
  }
  const int b = idx[0];
  std::copy(V[b].begin(), V[b].end(), theta_out);
  *f_out = F[b];
  *iters_out = it;
  *evals_out = evals;
  return 0;
}

}  // namespace orc

// ====================================================================== C interface (ctypes)
extern "C" {

void* orc_market_new(const orc::Desc* d) { return orc::build_market(d); }
void orc_market_free(void* m) { delete (orc::Market*)m; }

void orc_gl_nodes(int n, double* x, double* w) {
  std::vector<double> xs, ws;
  orc::gauss_legendre(n, xs, ws);
  std::copy(xs.begin(), xs.end(), x);
  std::copy(ws.begin(), ws.end(), w);
}

double orc_normal_cdf(double x) { return orc::normal_cdf(x); }
double orc_black_call(double F, double K, double T, double s, double D) { return orc::black_call(F, K, T, s, D); }
double orc_black_put(double F, double K, double T, double s, double D) { return orc::black_put(F, K, T, s, D); }
double orc_black_otm(double F, double K, double T, double s, double D) { return orc::black_otm(F, K, T, s, D); }
double orc_black_vega(double F, double K, double T, double s, double D) { return orc::black_vega(F, K, T, s, D); }
double orc_z_over_x(double z, double rho) { return orc::z_over_x(z, rho); }
double orc_sabr_hagan2002(double F, double K, double T, double a, double b, double r, double n) {
  return orc::sabr_hagan2002(F, K, T, a, b, r, n);
}
double orc_sabr_paper(double F, double K, double a, double b, double r, double n) {
  return orc::sabr_paper(F, K, a, b, r, n);
}

// Forward levels and market prices/weights as the oracle sees them.
void orc_market_info(const void* mp, double* F, double* cap_pm, double* cap_w, double* swp_pm,
                     double* swp_w, double* swp_S, double* swp_A) {
  const orc::Market& m = *(const orc::Market*)mp;
  if (F) std::copy(m.F.begin(), m.F.end(), F);
  if (cap_pm) std::copy(m.cpm.begin(), m.cpm.end(), cap_pm);
  if (cap_w) std::copy(m.cw.begin(), m.cw.end(), cap_w);
  if (swp_pm) std::copy(m.spm.begin(), m.spm.end(), swp_pm);
  if (swp_w) std::copy(m.sw.begin(), m.sw.end(), swp_w);
  for (size_t s = 0; s < m.sK.size(); ++s) {
    if (swp_S) swp_S[s] = m.swapS[m.sswap[s]];
    if (swp_A) swp_A[s] = m.swapA[m.sswap[s]];
  }
}

void orc_rebonato_caplet(const void* mp, const double* th, double Ti, double* out4) {
  double a, n, G, X;
  orc::rebonato_caplet(*(const orc::Market*)mp, th, Ti, a, n, &G, &X);
  out4[0] = G; out4[1] = X; out4[2] = a; out4[3] = n;
}

// SABR parameters of the swap underlying swaption s: out6 = (V1, V2, V3, alpha, nu, rho).
void orc_swap_params(const void* mp, const double* th, int s, double* out6) {
  const orc::Market& m = *(const orc::Market*)mp;
  double a, n, r, V[3];
  orc::swap_params(m, th, m.sswap[s], a, n, r, V);
  out6[0] = V[0]; out6[1] = V[1]; out6[2] = V[2]; out6[3] = a; out6[4] = n; out6[5] = r;
}

void orc_model_vols(const void* mp, const double* th, double* vols) {
  std::vector<double> v;
  orc::all_vols(*(const orc::Market*)mp, th, v);
  std::copy(v.begin(), v.end(), vols);
}

double orc_objective(const void* mp, const double* th) { return orc::objective(*(const orc::Market*)mp, th); }

void orc_objective_batch(const void* mp, const double* X, int64_t n, double* f, int n_threads) {
  const orc::Market& m = *(const orc::Market*)mp;
#pragma omp parallel for schedule(dynamic, 1) num_threads(n_threads > 0 ? n_threads : 1)
  for (int64_t i = 0; i < n; ++i) f[i] = orc::objective(m, X + i * m.n_param);
}

double orc_rmse_volpt(const void* mp, const double* th) { return orc::rmse_volpt(*(const orc::Market*)mp, th); }

// f and df/dtheta (all slots, free or not) by forward-mode dual numbers.
double orc_objective_grad(const void* mp, const double* th, double* grad) {
  const orc::Market& m = *(const orc::Market*)mp;
  if (m.n_param > orc::ND) return std::numeric_limits<double>::quiet_NaN();   // more slots than duals
  std::vector<orc::Dual> x;
  orc::seed_duals(m, th, x);
  orc::Dual f = orc::objective_t<orc::Dual>(m, x.data());
  for (int k = 0; k < m.n_param; ++k) grad[k] = f.d[k];
  return f.v;
}

// Residuals r_k and their Jacobian J[k, p] (row-major, n_instr x n_param); returns 0 if feasible.
int orc_residuals_jac(const void* mp, const double* th, double* r, double* J) {
  const orc::Market& m = *(const orc::Market*)mp;
  if (!J) {   // residuals alone, in plain FP64
    std::vector<double> rr;
    if (!orc::residuals(m, th, rr)) return 1;
    std::copy(rr.begin(), rr.end(), r);
    return 0;
  }
  if (m.n_param > orc::ND) return 2;   // more slots than dual components
  std::vector<orc::Dual> x, rr;
  orc::seed_duals(m, th, x);
  if (!orc::residuals(m, x.data(), rr)) return 1;
  for (size_t k = 0; k < rr.size(); ++k) {
    r[k] = rr[k].v;
    if (J) for (int p = 0; p < m.n_param; ++p) J[k * m.n_param + p] = rr[k].d[p];
  }
  return 0;
}

void orc_philox4x64_10(const uint64_t* ctr, const uint64_t* key, uint64_t* out) { orc::philox4x64_10(ctr, key, out); }
void orc_philox4x32_10(const uint32_t* ctr, const uint32_t* key, uint32_t* out) { orc::philox4x32_10(ctr, key, out); }
void orc_mc_normals4(uint64_t seed, uint64_t path, int step, int b, double* z) { orc::mc_normals4(seed, path, step, b, z); }

// Monte Carlo prices of caplets and swaptions on market mp's tenor structure (its first M forwards)
// under the Hagan SABR/LIBOR model; params = [beta, eta1, lambda1, eta2, lambda2, lambda3] and the
// per-forward alpha, sigma, phi_ii.  Returns 1 if the correlation matrix is not positive definite.
int orc_mc_price(const void* mp, int M, int model, const double* params, const double* alpha, const double* sigma,
                 const double* phi, int n_cap, const int* cap_fwd, const double* cap_K, int n_swp, const int* swp_a,
                 const int* swp_b, const double* swp_K, int64_t n_paths, double dt, uint64_t seed, int n_threads,
                 double* price, double* sq, int64_t* n_bad) {
  orc::McModel md;
  md.M = M; md.model = model; md.beta = params[0]; md.eta1 = params[1]; md.lambda1 = params[2]; md.eta2 = params[3];
  md.lambda2 = params[4]; md.lambda3 = params[5];
  md.alpha.assign(alpha, alpha + M); md.sigma.assign(sigma, sigma + M); md.phi.assign(phi, phi + M);
  return orc::mc_price(*(const orc::Market*)mp, md, n_cap, cap_fwd, cap_K, n_swp, swp_a, swp_b, swp_K, n_paths, dt,
                       seed, n_threads, price, sq, n_bad);
}

void orc_step_uniforms(uint64_t seed, uint64_t chain_word, int level, int step, int count, double* u) {
  orc::step_uniforms(seed, chain_word, level, step, count, u);
}

int orc_anneal(const void* mp, const orc::SAOpts* o, double* x_best, double* f_best, double* chain_xb,
               double* chain_fb, double* trace_f, double* trace_x, uint8_t* bits, int64_t* n_evals,
               double* T0_used) {
  return orc::anneal(*(const orc::Market*)mp, *o, x_best, f_best, chain_xb, chain_fb, trace_f, trace_x,
                     bits, n_evals, T0_used);
}

// f_s at the correlation parameters y[5] (see mc_objective); quote_vol [n_cap + n_swp].
double orc_mc_objective(const void* mp, int M, int model, const double* params, const double* alpha, const double* sigma,
                        const double* phi, int n_cap, const int* cap_fwd, const double* cap_K, int n_swp,
                        const int* swp_a, const int* swp_b, const double* swp_K, const double* quote_vol,
                        int64_t n_paths, double dt, uint64_t mc_seed, const double* y, int n_threads) {
  const orc::Market& m = *(const orc::Market*)mp;
  orc::McModel md;
  md.M = M; md.model = model; md.beta = params[0];
  md.alpha.assign(alpha, alpha + M); md.sigma.assign(sigma, sigma + M); md.phi.assign(phi, phi + M);
  const orc::McTarget t = orc::mc_target(m, n_cap, cap_fwd, cap_K, n_swp, swp_a, swp_b, swp_K, quote_vol);
  return orc::mc_objective(m, md, t, y, n_paths, dt, mc_seed, n_threads);
}

// The annealing search of f_s over the box lo/hi/free_mask [5] (SAOpts as for orc_anneal; the
// Monte Carlo of each evaluation single-threaded, the chains in parallel).
int orc_mc_anneal(const void* mp, int M, int model, const double* params, const double* alpha, const double* sigma,
                  const double* phi, int n_cap, const int* cap_fwd, const double* cap_K, int n_swp, const int* swp_a,
                  const int* swp_b, const double* swp_K, const double* quote_vol, int64_t n_paths, double dt,
                  uint64_t mc_seed, const double* lo, const double* hi, const uint8_t* freem, const orc::SAOpts* o,
                  double* y_best, double* f_best, double* trace_f, double* trace_x, double* T0_used) {
  const orc::Market& m = *(const orc::Market*)mp;
  orc::McModel md;
  md.M = M; md.model = model; md.beta = params[0];
  md.alpha.assign(alpha, alpha + M); md.sigma.assign(sigma, sigma + M); md.phi.assign(phi, phi + M);
  const orc::McTarget t = orc::mc_target(m, n_cap, cap_fwd, cap_K, n_swp, swp_a, swp_b, swp_K, quote_vol);
  const orc::Box bx{5, lo, hi, freem};
  return orc::anneal_box(bx, [&](const double* y) { return orc::mc_objective(m, md, t, y, n_paths, dt, mc_seed, 1); },
                         *o, y_best, f_best, nullptr, nullptr, trace_f, trace_x, nullptr, nullptr, T0_used);
}

int orc_nm(const void* mp, const double* theta0, int max_iter, double step, double ftol, double* theta_out,
           double* f_out, int* iters_out, int* evals_out) {
  return orc::nm(*(const orc::Market*)mp, theta0, max_iter, step, ftol, theta_out, f_out, iters_out, evals_out);
}

int orc_lm(const void* mp, const double* theta0, int max_iter, double target_rmse, double mu0,
           double* theta_out, double* f_out, double* rmse_out, int* iters_out) {
  if (((const orc::Market*)mp)->n_param > orc::ND) return 2;   // the Jacobian's duals hold 12 slots
  return orc::lm(*(const orc::Market*)mp, theta0, max_iter, target_rmse, mu0, theta_out, f_out, rmse_out, iters_out);
}

}  // extern "C"
