// Warp-cooperative evaluation of the calibration objective for one parameter point.
//
// One warp owns one parameter point (one annealing chain).  The market's instrument blocks sit
// in shared memory (staged once per CTA by a bulk copy); each warp has a private scratch region
// for the per-panel integrals and the per-forward SABR parameters of its point.
//
//   S2  rebonato_forward_params : Eq. (haganForRebonato) for every caplet forward, by the
//       composite Gauss-Legendre rule written in time-to-fixing u.  Time homogeneity makes one
//       table of panel integrals serve every maturity: panel p of [0, T_i] in u is the same
//       interval [pD, (p+1)D] for every i, so
//         G_i = sum_{p < n_i} Gp[p],   X_i = sum_{p < n_i} (Ap[p] + Gp[p] sum_{p < p' < n_i} Hp[p'])
//       with Gp = int g^2, Hp = int h^2 over panel p and Ap = int g(u)^2 R(u) over panel p,
//       R(u) the inner rule on [u, panel top].  (The same discrete sums as a direct rule in
//       calendar time, reordered.)  Lanes split (panel, node); exponentials factor as
//       e^{-c(pD + o)} = e^{-c pD} e^{-c o}.
//   S4  price_caplets : per caplet, SABR vol -> OTM Black price -> vega-weighted residual.
//   S7  the squared residuals summed per lane in the pricing precision, across lanes in FP64.
#pragma once
#include "device_math.cuh"
#include "market.cuh"

namespace sabr {

template <class R> struct WarpScratch {
  R* xs;   // [16] parameter point in the pricing precision
  R* Gp;   // [NPc] per-panel integrals
  R* Hp;
  R* Ap;
  R* af;   // [n_fwd] per-forward SABR alpha
  R* nf;   // [n_fwd] per-forward SABR nu
};

__host__ __device__ inline int round_up(int x, int m) { return (x + m - 1) / m * m; }

// Elements (of R) of one warp's scratch; a multiple of 4 so that every region stays 16B-aligned.
__host__ __device__ inline int warp_scratch_elems(int NP, int n_fwd) {
  return round_up(16 + 3 * round_up(NP > 0 ? NP : 1, 4) + 2 * round_up(n_fwd, 4), 4);
}

template <class R>
__device__ __forceinline__ WarpScratch<R> warp_scratch(R* base, int NP, int n_fwd) {
  WarpScratch<R> s;
  const int NPc = round_up(NP > 0 ? NP : 1, 4);
  s.xs = base;
  s.Gp = base + 16;
  s.Hp = s.Gp + NPc;
  s.Ap = s.Hp + NPc;
  s.af = s.Ap + NPc;
  s.nf = s.af + round_up(n_fwd, 4);
  return s;
}

template <class R> __device__ __forceinline__ const QuadTab<R>* quad_of(const DevMarket& m);
template <> __device__ __forceinline__ const QuadTab<double>* quad_of<double>(const DevMarket& m) { return m.q64; }
template <> __device__ __forceinline__ const QuadTab<float>* quad_of<float>(const DevMarket& m) { return m.q32; }

// S2: alpha_i, nu_i of every caplet forward (Rebonato mapping, kappa = 1).
template <class R>
__device__ void rebonato_forward_params(const DevMarket& m, const R* th, const WarpScratch<R>& ws, int lane) {
  typedef Num<R> M;
  const QuadTab<R>& qt = *quad_of<R>(m);
  const R a = th[0], b = th[1], c = th[2], d = th[3];
  const R ah = th[4], bh = th[5], gh = th[6], dh = th[7];
  const R D = (R)m.panel;
  const int q = lane & 7, pg = lane >> 3;
  const R oq = qt.o[q], wq = qt.w[q];
  const R eg = M::exp_(-c * oq), eh = M::exp_(-gh * oq);
  R o2[kQ], w2[kQ], ehs[kQ];
#pragma unroll
  for (int r = 0; r < kQ; ++r) {
    o2[r] = qt.o2[q * kQ + r];
    w2[r] = qt.w2[q * kQ + r];
    ehs[r] = M::exp_(-gh * o2[r]);
  }
  const int NP = m.NP, NPc = round_up(NP, 4);
  for (int p = pg; p < NPc; p += 4) {
    R G = 0, H = 0, A = 0;
    if (p < NP) {
      const R base = D * (R)p;
      const R Eg = M::exp_(-c * base), Eh = M::exp_(-gh * base);
      const R u = base + oq;
      const R g = (a + b * u) * (Eg * eg) + d;
      const R h = (ah + bh * u) * (Eh * eh) + dh;
      R Rin = 0;
#pragma unroll
      for (int r = 0; r < kQ; ++r) {
        const R v = base + o2[r];
        const R hr = (ah + bh * v) * (Eh * ehs[r]) + dh;
        Rin += w2[r] * hr * hr;
      }
      const R gw = wq * g * g;
      G = gw;
      H = wq * h * h;
      A = gw * Rin;
    }
#pragma unroll
    for (int off = 1; off < 8; off <<= 1) {
      G += __shfl_xor_sync(0xffffffffu, G, off);
      H += __shfl_xor_sync(0xffffffffu, H, off);
      A += __shfl_xor_sync(0xffffffffu, A, off);
    }
    if (q == 0 && p < NP) { ws.Gp[p] = G; ws.Hp[p] = H; ws.Ap[p] = A; }
  }
  __syncwarp();
  for (int j = lane; j < m.n_capfwd; j += 32) {
    const int i = m.capfwd_list[j];
    const int n = m.fwd_np[i];
    const R Ti = (R)m.T[i];
    R G = 0, X = 0, S = 0;
    for (int p = n - 1; p >= 0; --p) {
      X += ws.Ap[p] + ws.Gp[p] * S;
      G += ws.Gp[p];
      S += ws.Hp[p];
    }
    const R al = M::sqrt_(G / Ti);
    ws.af[i] = al;
    ws.nf[i] = M::sqrt_(R(2) * X) / (al * Ti);
  }
  __syncwarp();
}

// S4 + S7 (caplets): lane-strided pricing; returns this lane's partial sum of squared
// residuals in the pricing precision and clears `ok` on an infeasible vol.  With vols != null
// the model vols are written instead (NaN where infeasible).
template <class R, int FORMULA>
__device__ __forceinline__ R price_caplets(const InstrView<R>& B, int n, const R* af, const R* nf, R rho,
                                           R omb, int lane, bool& ok, double* vols) {
  typedef Num<R> M;
  R acc = 0;
  for (int k = lane; k < n; k += 32) {
    const int i = B.idx[k];
    const R al = af[i], nu = nf[i];
    const R l = B.l[k];
    R sig;
    if (FORMULA == 0) sig = sabr_hagan<R>(al, rho, nu, l, B.fk[k], B.inv_den[k], B.c1[k], B.c2[k], B.c3[k]);
    else sig = sabr_paper<R>(al, rho, nu, l, B.fk[k], omb);
    const bool good = (sig > R(0)) && M::finite_(sig);
    if (vols) { vols[k] = good ? (double)sig : __longlong_as_double(0x7ff8000000000000LL); continue; }
    ok = ok && good;
    const R p = black_otm<R>(sig, B.sqrtT[k], l, B.DF[k], B.KF[k], B.sgn[k]);
    const R r = B.sw[k] * (p - B.pm[k]);
    acc += r * r;
  }
  return acc;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  return v;
}

// Objective of the point held in ws.xs (all 32 lanes call; all return the same value).
// MODEL 0: SABR smile [alpha, rho, nu];  MODEL 1: Rebonato caplets.
template <class R, int MODEL, int FORMULA>
__device__ double warp_objective(const DevMarket& m, const InstrView<R>& capB, const WarpScratch<R>& ws,
                                 int lane, double* vols) {
  R th[kMaxParam];
#pragma unroll
  for (int k = 0; k < kMaxParam; ++k) th[k] = ws.xs[k];
  R rho;
  if (MODEL == 0) {
    for (int j = lane; j < m.n_capfwd; j += 32) {
      const int i = m.capfwd_list[j];
      ws.af[i] = th[0];
      ws.nf[i] = th[2];
    }
    __syncwarp();
    rho = th[1];
  } else {
    rebonato_forward_params<R>(m, th, ws, lane);
    rho = th[8];
  }
  bool ok = true;
  const R part = price_caplets<R, FORMULA>(capB, m.n_cap, ws.af, ws.nf, rho, (R)(1.0 - m.beta), lane, ok, vols);
  __syncwarp();
  if (vols) return 0.0;
  const double f = warp_sum((double)part);
  const bool bad = __any_sync(0xffffffffu, !ok);
  if (bad || !isfinite(f)) return __longlong_as_double(0x7ff0000000000000LL);  // +inf
  return f;
}

}  // namespace sabr
