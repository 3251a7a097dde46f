// Hand-written reverse-mode (adjoint) sweep of the caplet objective, one warp per parameter point.
//
// Forward sweep: the Rebonato mapping (S2, per-panel tables kept in the warp's scratch) and the
// caplet prices.  Reverse sweep, in the opposite order:
//   f = sum r_k^2, r_k = sqrt(w_k)(P_k - P_k^mkt)          r_bar = 2 r_k, P_bar = 2 r_k sqrt(w_k)
//   P_k = Black(sigma_k)                                      sigma_bar = P_bar * vega_k (closed form)
//   sigma_k = SABR(alpha_i, nu_i, rho)                        (alpha, nu, rho)_bar from the partials
//   alpha_i = sqrt(G_i / T_i), nu_i = sqrt(2 X_i)/(alpha_i T_i)   G_bar_i, X_bar_i
//   G_i, X_i = panel sums (prefix structure of S2)           Gp_bar, Hp_bar, Ap_bar per panel
//   Gp, Hp, Ap = node sums of g^2, h^2, g^2 R(h^2)            g_bar, h_bar at every node
//   g(u) = (a + b u) e^{-cu} + d, h(u) likewise              parameter adjoints.
// Per-forward adjoints are accumulated in shared memory with FP64 atomics; the parameter adjoints
// are summed per lane in the pricing precision and reduced across lanes in FP64.
#pragma once
#include "objective.cuh"

namespace sabr {

// z/x(z) and its partial derivatives in z and rho (same algebra as z_over_x_fast).  With
// zz = |z|, r = sign(z) rho, s = sqrt(1 - 2 r zz + zz^2), N = zz Q / (s + 1), x = log1p(N/(1-r)):
//   d(zz/x)/d zz = (x - zz/s) / x^2,
//   d(zz/x)/d r  = -zz x_r / x^2,
//   x_r = zz^2 (r (2r - zz)/(s + 1) + zz + s - 2r) / ((s + 1)(1 - r) s ((1 - r) + N)),
// and d/dz = sign(z) d/dzz, d/drho = sign(z) d/dr.  Near z = 0 the series and its derivatives.
template <class R>
__device__ __forceinline__ void z_over_x_grad(R z, const RhoConsts<R>& rc, R& zx, R& dz, R& drho) {
  typedef Num<R> M;
  const R zz = M::abs_(z);
  const R rho = rc.rho;
  if (zz < M::zx_series) {
    zx = R(1) - R(0.5) * rho * z + (R(2) - R(3) * rho * rho) * z * z * R(1.0 / 12.0);
    dz = -R(0.5) * rho + (R(2) - R(3) * rho * rho) * z * R(1.0 / 6.0);
    drho = -R(0.5) * z - R(0.5) * rho * z * z;
    return;
  }
  const bool neg = z < R(0);
  const R sg = neg ? R(-1) : R(1);
  const R r = neg ? -rho : rho;
  const R omr = neg ? rc.omr_m : rc.omr_p;
  const R iomr = neg ? rc.iomr_m : rc.iomr_p;
  const R zq = zz * (zz - R(2) * r);
  const R s = fsqrt<R>(R(1) + zq);
  const R smr = fdiv<R>(rc.omr2 + zq, s + r);
  const R Q = (r > R(0)) ? (smr + omr + zz) : (zz - R(2) * r + s + R(1));
  const R N = fdiv<R>(zz * Q, s + R(1));
  const R x = M::log1p_(N * iomr);
  zx = fdiv<R>(zz, x);
  const R ix2 = fdiv<R>(R(1), x * x);
  const R dzz = (x - fdiv<R>(zz, s)) * ix2;
  const R br = fdiv<R>(r * (R(2) * r - zz), s + R(1)) + zz + s - R(2) * r;
  const R xr = fdiv<R>(zz * zz * br, (s + R(1)) * omr * s * (omr + N));
  const R dr = -zz * xr * ix2;
  dz = sg * dzz;
  drho = sg * dr;
}

template <class R> struct AdjScratch {
  double* abar;   // [NFc] per-forward adjoints of alpha
  double* nbar;   // [NFc] of nu
  R* Gbar;        // [NFc] of G_i
  R* Xbar;        // [NFc] of X_i
  R* SH;          // [NPc + 4] prefix sums of Hp
  R* PG;          // [NPc + 4] prefix sums of Gp
};

__host__ __device__ inline int adj_scratch_bytes(int NP, int n_fwd, int rbytes) {
  const int NFc = round_up(n_fwd, 4), NPc = round_up(NP > 0 ? NP : 1, 4);
  return 2 * NFc * 8 + (2 * NFc + 2 * (NPc + 4)) * rbytes;
}

template <class R>
__device__ __forceinline__ AdjScratch<R> adj_scratch(unsigned char* base, int NP, int n_fwd) {
  AdjScratch<R> s;
  const int NFc = round_up(n_fwd, 4), NPc = round_up(NP > 0 ? NP : 1, 4);
  s.abar = (double*)base;
  s.nbar = s.abar + NFc;
  R* p = (R*)(s.nbar + NFc);
  s.Gbar = p; p += NFc;
  s.Xbar = p; p += NFc;
  s.SH = p; p += NPc + 4;
  s.PG = p;
  return s;
}

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  return v;
}

// Accumulate the adjoints of g or h at a node u with e = e^{-k u} (k = c or gamma_h), the value
// gv = g(u) and the linear part lin = a + b u: slots (a, b, c, d) of the function.
template <class R>
__device__ __forceinline__ void abcd_bar(R bar, R u, R e, R lin, R* acc4) {
  acc4[0] += bar * e;
  acc4[1] += bar * u * e;
  acc4[2] -= bar * u * lin * e;
  acc4[3] += bar;
}

// SABR vol and its partials in (alpha, nu, rho) for one instrument with per-forward (or per-swap)
// factors fw = {alpha, nu/alpha, alpha^2, rho nu alpha}, A3 = (2 - 3 rho^2) nu^2, and its constants
// g0 = {l, fk, inv_den, c1}, g1 = {c2, c3, sqrt T, D F}.
template <class R, int FORMULA>
__device__ __forceinline__ R sabr_vol_grad(const Q4<R>& fw, R A3, const RhoConsts<R>& rc, const Q4<R>& g0,
                                           const Q4<R>& g1, R omb, R& s_al, R& s_nu, R& s_rho) {
  const R al = fw.a, nu = fw.b * fw.a, rho = rc.rho;
  R sig;
  if (FORMULA == 0) {
    const R z = fw.b * g0.b;
    R zx, dzx, dzr;
    z_over_x_grad<R>(z, rc, zx, dzx, dzr);
    const R corr = R(1) + g0.d * fw.c + g1.a * fw.d + g1.b * A3;
    const R pre = al * g0.c;                          // alpha * inv_den
    sig = pre * zx * corr;
    s_al = g0.c * zx * corr + pre * dzx * (-z / al) * corr + pre * zx * (R(2) * g0.d * al + g1.a * rho * nu);
    s_nu = pre * (dzx * (g0.b / al) * corr + zx * (g1.a * rho * al + R(2) * g1.b * (R(2) - R(3) * rho * rho) * nu));
    s_rho = pre * (dzr * corr + zx * (g1.a * nu * al - R(6) * g1.b * rho * nu * nu));
  } else {
    // Eq. (sigmaHagan): sigma = alpha/fo (1 - (omb - rho nu w) m/2 + (omb^2 + (2-3rho^2) nu^2 w^2 + 3(omb - rho nu w)) m^2/12),
    // w = fo/alpha, m = -l
    const R fo = g0.b, mm = -g0.a, w = fo / al;
    const R rnw = rho * nu * w;
    const R br = R(1) - R(0.5) * (omb - rnw) * mm + (omb * omb + (R(2) - R(3) * rho * rho) * nu * nu * w * w + R(3) * (omb - rnw)) * mm * mm * R(1.0 / 12.0);
    sig = al / fo * br;
    // partials of the bracket in (nu w) and rho at fixed alpha, then w = fo/alpha
    const R d_rnw = R(0.5) * mm - R(3) * mm * mm * R(1.0 / 12.0);              // d br / d(rho nu w)
    const R d_nw2 = (R(2) - R(3) * rho * rho) * mm * mm * R(1.0 / 12.0);       // d br / d(nu^2 w^2)
    const R dbr_dw = d_rnw * rho * nu + d_nw2 * R(2) * nu * nu * w;
    const R dbr_dnu = d_rnw * rho * w + d_nw2 * R(2) * nu * w * w;
    const R dbr_drho = d_rnw * nu * w - R(6) * rho * nu * nu * w * w * mm * mm * R(1.0 / 12.0);
    s_al = br / fo + al / fo * dbr_dw * (-w / al);
    s_nu = al / fo * dbr_dnu;
    s_rho = al / fo * dbr_drho;
  }
  return sig;
}

// The weighted residual r = sqrt(w) (P - P_mkt) of an instrument at vol sig and the adjoint of the
// vol from f's term r^2: sigma_bar = 2 r sqrt(w) vega(sig).  g2 = {K/F, sgn, P_mkt, sqrt(w)}.
template <class R>
__device__ __forceinline__ R black_residual_grad(R sig, const Q4<R>& g0, const Q4<R>& g1, const Q4<R>& g2, R& sbar) {
  typedef Num<R> M;
  const R v = sig * g1.c;
  const R d1 = fdiv<R>(g0.a, v) + R(0.5) * v;
  const R sg = g2.b;
  const R p = sg * g1.d * (ncdf<R>(sg * d1) - g2.a * ncdf<R>(sg * (d1 - v)));
  const R r = g2.d * (p - g2.c);
  const R vega = g1.d * M::exp_(R(-0.5) * d1 * d1) * R(0.39894228040143267794) * g1.c;
  sbar = R(2) * r * g2.d * vega;
  return r;
}

// Caplet pricing with the local reverse sweep, lane-strided over every caplet (k0, k0 + stride, ...):
// adds r^2 to facc, the per-forward adjoints of alpha_i and nu_i to as.abar / as.nbar (FP64 atomics)
// and the adjoint of the common rho to rho_bar; clears ok on an infeasible vol.
template <class R, int FORMULA>
__device__ void caplet_price_reverse(const DevMarket& m, const InstrView<R>& capB, const WarpScratch<R>& ws,
                                     const AdjScratch<R>& as, const RhoConsts<R>& rc, int k0, int stride, bool& ok,
                                     R& facc, double& rho_bar) {
  typedef Num<R> M;
  const R omb = (R)(1.0 - m.beta);
  for (int k = k0; k < m.n_cap; k += stride) {
    const int i = capB.idx[k];
    const Q4<R> g0 = capB.g0[k], g1 = capB.g1[k], g2 = capB.g2[k];
    R s_al, s_nu, s_rho;
    const R sig = sabr_vol_grad<R, FORMULA>(ws.F4[i], ws.fA3[i], rc, g0, g1, omb, s_al, s_nu, s_rho);
    const bool good = (sig > R(0)) && M::finite_(sig);
    ok = ok && good;
    if (!good) continue;
    R sbar;
    const R r = black_residual_grad<R>(sig, g0, g1, g2, sbar);
    facc += r * r;
    atomicAdd(as.abar + i, (double)(sbar * s_al));
    atomicAdd(as.nbar + i, (double)(sbar * s_nu));
    rho_bar += (double)(sbar * s_rho);
  }
}

// Reverse of the Rebonato caplet mapping (alpha_i, nu_i of every caplet forward from the panel sums
// of S2) down to the parameters a, b, c, d, alpha_h, beta_h, gamma_h, delta_h: this lane's share in
// gacc[0..7] (the caller reduces across the warp).  Reads as.abar / as.nbar and the forward sweep's
// tables in ws (inclusive prefix sums in Gp, Hp).
template <class R>
__device__ void caplet_mapping_reverse(const DevMarket& m, const QuadTab<R>& qt, const WarpScratch<R>& ws,
                                       const AdjScratch<R>& as, int lane, double* gacc) {
  const int NP = m.NP;
  // the forward pass leaves inclusive prefix sums over panels in Hp and Gp
  for (int p = lane; p <= NP; p += 32) {
    as.SH[p] = p > 0 ? ws.Hp[p - 1] : R(0);
    as.PG[p] = p > 0 ? ws.Gp[p - 1] : R(0);
  }
  for (int j = lane; j < m.n_capfwd; j += 32) {
    const int i = m.capfwd_list[j];
    const Q4<R> fw = ws.F4[i];
    const R al = fw.a, nu = fw.b * fw.a, Ti = (R)m.T[i];
    // X_i from nu_i: nu = sqrt(2X)/(alpha T)  ->  X = (nu alpha T)^2 / 2
    const R X = R(0.5) * (nu * al * Ti) * (nu * al * Ti);
    const R ab = (R)as.abar[i], nb = (R)as.nbar[i];
    as.Gbar[i] = (ab - nb * nu / al) / (R(2) * al * Ti);
    as.Xbar[i] = X > R(0) ? nb * nu / (R(2) * X) : R(0);
  }
  __syncwarp();
  // ---------------- reverse of the panel sums and of the node tables
  const R a = ws.xs[0], b = ws.xs[1], c = ws.xs[2], d = ws.xs[3];
  const R ah = ws.xs[4], bh = ws.xs[5], gh = ws.xs[6], dh = ws.xs[7];
  const R D = (R)m.panel;
  const int q = lane & 7, pg = lane >> 3;
  const R wq = qt.w[q];
  const Q4<R> tq = ws.Tq[q];
  R acc[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) acc[k] = 0;
  // e^{-gamma_h o2} of this lane's inner nodes: the same for every panel
  R eo2[kQ];
#pragma unroll
  for (int r = 0; r < kQ; ++r) eo2[r] = Num<R>::exp_(-gh * qt.o2[q * kQ + r]);
  const int NPc = round_up(NP, 4);
  for (int p = pg; p < NPc; p += 4) {
    if (p >= NP) continue;
    R Gpb = 0, Apb = 0, Hpb = 0;
    for (int j = 0; j < m.n_capfwd; ++j) {
      const int i = m.capfwd_list[j];
      const int n = m.fwd_np[i];
      if (n > p) {
        const R xb = as.Xbar[i];
        Gpb += as.Gbar[i] + xb * (as.SH[n] - as.SH[p + 1]);
        Apb += xb;
        Hpb += xb * as.PG[p];
      }
    }
    const R base = D * (R)p;
    Q2<R> E;
    E.a = Num<R>::exp_(-c * base);
    E.b = Num<R>::exp_(-gh * base);
    const R u = base + qt.o[q];
    const R eg = E.a * tq.a, eh = E.b * tq.c;      // e^{-c u}, e^{-gamma_h u}
    const R lin_g = a + b * u, lin_h = ah + bh * u;
    const R g = lin_g * eg + d;
    const R h = lin_h * eh + dh;
    const R Rbar = Apb * wq * g * g;
    R Rin = 0;
#pragma unroll
    for (int r = 0; r < kQ; ++r) {
      // inner node v = base + o2: R = sum w2 h(v)^2, so h(v)_bar = 2 Rbar w2 h(v)
      const R o2 = qt.o2[q * kQ + r];
      const R sw2 = qt.sw2[q * kQ + r];
      const R v = base + o2;
      const R ev = E.b * eo2[r];                   // e^{-gamma_h v}
      const R lin = ah + bh * v;
      const R hv = lin * ev + dh;
      Rin += sw2 * sw2 * hv * hv;
      const R hvbar = R(2) * Rbar * sw2 * sw2 * hv;
      abcd_bar<R>(hvbar, v, ev, lin, acc + 4);
    }
    const R gbar = R(2) * wq * g * (Gpb + Apb * Rin);
    const R hbar = R(2) * wq * h * Hpb;
    abcd_bar<R>(gbar, u, eg, lin_g, acc);
    abcd_bar<R>(hbar, u, eh, lin_h, acc + 4);
  }
#pragma unroll
  for (int k = 0; k < 8; ++k) gacc[k] += (double)acc[k];
}

// f and df/dtheta of the point in ws.xs (all 32 lanes call).  g_out (12 doubles) and f_out are
// written by lane 0.
template <class R, int MODEL, int FORMULA>
__device__ void warp_objective_grad(const DevMarket& m, const InstrView<R>& capB, const QuadTab<R>& qt,
                                    const WarpScratch<R>& ws, const AdjScratch<R>& as, int lane, double* f_out,
                                    double* g_out) {
  // ---------------- forward sweep
  RhoConsts<R> rc;
  if (MODEL == 0) {
    const R al = ws.xs[0], rho = ws.xs[1], nu = ws.xs[2];
    for (int j = lane; j < m.n_capfwd; j += 32) put_forward<R>(ws, m.capfwd_list[j], al, nu, rho);
    rc.init(rho);
  } else {
    rebonato_forward_params<R>(m, qt, ws, lane);
    rc.init(ws.xs[8]);
  }
  for (int j = lane; j < m.n_capfwd; j += 32) {
    const int i = m.capfwd_list[j];
    as.abar[i] = 0.0;
    as.nbar[i] = 0.0;
  }
  __syncwarp();
  // ---------------- pricing with the local reverse sweep
  bool ok = true;
  R facc = 0;
  double rho_bar = 0.0;
  caplet_price_reverse<R, FORMULA>(m, capB, ws, as, rc, lane, 32, ok, facc, rho_bar);
  const bool bad = __any_sync(0xffffffffu, !ok);
  const double f = warp_sum_d((double)facc);
  rho_bar = warp_sum_d(rho_bar);
  __syncwarp();
  double gacc[kMaxGradParam];
#pragma unroll
  for (int k = 0; k < kMaxGradParam; ++k) gacc[k] = 0.0;
  if (MODEL == 0) {
    double sa = 0.0, sn = 0.0;
    for (int j = lane; j < m.n_capfwd; j += 32) {
      const int i = m.capfwd_list[j];
      sa += as.abar[i];
      sn += as.nbar[i];
    }
    gacc[0] = sa;
    gacc[2] = sn;
  } else {
    caplet_mapping_reverse<R>(m, qt, ws, as, lane, gacc);
  }
#pragma unroll
  for (int k = 0; k < kMaxGradParam; ++k) gacc[k] = warp_sum_d(gacc[k]);
  if (MODEL == 0) gacc[1] = rho_bar;
  else gacc[8] = rho_bar;
  if (lane == 0) {
    const double inf = __longlong_as_double(0x7ff0000000000000LL);
    *f_out = (bad || !isfinite(f)) ? inf : f;
    for (int k = 0; k < m.n_param; ++k) g_out[k] = (bad || !isfinite(f)) ? 0.0 : gacc[k];
  }
  __syncwarp();
}

}  // namespace sabr
