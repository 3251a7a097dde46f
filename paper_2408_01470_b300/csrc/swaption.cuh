// CTA-cooperative evaluation of the objective for markets with swaptions: one CTA owns one
// parameter point (one chain); its warps split the swap-rate integrals, the quadratic forms and the
// instruments.
//
// S3  Pair integrals.  Every forward's vol and vol-of-vol are g(T_i - t), h(T_i - t) (time
//     homogeneity), so on the uniform panel grid the integrand of G_ij(T_E) and X_ij(T_E) at a
//     quadrature node depends only on the absolute panels A = p + delta_i, B = p + delta_j the
//     node falls in for forwards i and j (p the panel of time-to-expiry, delta_i = (T_i - T_E)/D).
//     With the per-chain matrix Y[A][k] (k < 8: sqrt(w_q) g at the outer nodes; 8 <= k < 16:
//     sqrt(w_q) h there; 16 <= k < 80: sqrt(w_q) g times sqrt(w_qr) h at the inner nodes) the
//     panel-pair sums are Gram sums
//       Gd(A,B) = sum_{k<8} Y_A Y_B,  Hd(A,B) = sum_{8<=k<16} Y_A Y_B,  Ad(A,B) = sum_{k>=16} Y_A Y_B,
//     and along each diagonal e = B - A the prefix sums PG, PA, SH and PGS (of Gd * inclusive SH)
//     give, for a swap expiring after nE panels and the pair (i, j) with e = delta_j - delta_i,
//       G_ij = PG(hi) - PG(lo),  X_ij / theta_ij = PA(hi) - PA(lo) + SH(hi)(PG(hi) - PG(lo)) - (PGS(hi) - PGS(lo))
//     (lo = delta_i, hi = lo + nE): the composite rule of the oracle, calendar time reversed.
// S5  Quadratic forms per swap: V = sum_{i<=j} (2 - [i=j]) W_i W_j B_ij, B = (rho G, rho X, phi G).
//     The frozen weights factor as W_i = u_i / (A S^b) with u_i = tau_i P(0, T_{i+1}) F_i^b, and the
//     swaps of an expiry group (sharing their first forward) are leading blocks of the group's
//     window, so one pass over each group's pair triangle, prefix-summed over its columns, gives the
//     forms of all its swaps: V(swap) = (A S^b)^-2 Q(g, L_swap).
// S6  alpha_S = sqrt(V1/T), nu_S = sqrt(2 V2)/(alpha_S T), rho_S = clamp(V3/V1, +-0.999), then
//     SABR and Black per swaption, with the caplets priced alongside.
#pragma once
#include "objective.cuh"
#include "tcgen05_gram.cuh"

namespace sabr {

template <class R> struct CtaScratch {
  R* xs;            // [kMaxParam]
  WarpScratch<R> cap;  // caplet mapping (warp 0); its xs is a private copy
  Q2<R>* Ep;        // [NAc] {e^{-c A D}, e^{-gamma_h A D}}
  Q4<R>* Tq;        // [8]
  Q4<R>* T2;        // [8 x 9]
  Q4<R>* Sq;        // [8 x 2] per outer node q the inner-rule sums {Saa, Sab, Sbb, Sac}, {Sbc, Scc, 0, 0}
  R* Y;             // [NA x 84]
  R* PQ;            // [kPQ x ND x PL] the prefix tables along each diagonal (PairTables below)
  Q4<R>* crq;       // [ND]: {rho_e, rho_e theta_e, phi_e, 0} per diagonal e
  Q4<R>* F4s;       // [n_swap] {alpha, nu/alpha, alpha^2, rho nu alpha}
  R* A3s;           // [n_swap] (2 - 3 rho^2) nu^2
  Q4<R>* RCs;       // [n_swap] {rho, 1/(1 - rho), 1/(1 + rho), 1 - rho^2}
  R* Qs;            // [3 x n_seg] segment partials of the quadratic forms (in the Y region, dead
                    //   after the Grams, unless qf_own)
};

// Y row pitch: 16-byte rows, conflict-free 4-vector loads.  The tensor-core form fills all 80 values
// of a row (g, h and the 64 inner-node products); the ALU form only the first 16 (g and h), the rest
// of the region serving phase 5's partials.
__host__ __device__ inline int cta_y_stride() { return 84; }
// Row pitch of the prefix tables: at least NA + 1, and even, so that the pairs of a window column
// (address stride 1 - pitch along a column) fall on distinct banks.
__host__ __device__ inline int cta_pq_len(int NA) { return (NA + 2) & ~1; }

// Prefix tables per diagonal: 4 (FP64), 6 (FP32: float-float PG and PGS).
template <class R> __host__ __device__ constexpr int cta_pq_tables() { return sizeof(R) == 4 ? 6 : 4; }

// Layout of the pair tables [ND x PL] per table.  FP64: four tables PG, PA, SH, PGS.  FP32: three
// tables of float2, {PG hi, PG lo}, {PGS hi, PGS lo}, {PA, SH}, so that a window integral reads
// six words instead of eleven.  Before phase 4 the tables hold each cell's raw G, A and H: FP64 in
// PG, PA, SH; FP32 in PG.hi, PA and SH.
template <class R> struct PairTables {
  R* PQ;
  int ND, PL;
  __device__ __forceinline__ R& G(int e, int A) const {
    if constexpr (sizeof(R) == 4) return ((float2*)PQ)[e * PL + A].x;
    else return PQ[e * PL + A];
  }
  __device__ __forceinline__ R& Ac(int e, int A) const {
    if constexpr (sizeof(R) == 4) return ((float2*)PQ + 2 * ND * PL)[e * PL + A].x;
    else return PQ[(ND + e) * PL + A];
  }
  __device__ __forceinline__ R& H(int e, int A) const {
    if constexpr (sizeof(R) == 4) return ((float2*)PQ + 2 * ND * PL)[e * PL + A].y;
    else return PQ[(2 * ND + e) * PL + A];
  }
  // raw cell slot q: 0 G, 1 A, 2 H (the tensor-core form's order)
  __device__ __forceinline__ R& raw(int q, int e, int A) const { return q == 0 ? G(e, A) : (q == 1 ? Ac(e, A) : H(e, A)); }
};

template <class R>
__host__ __device__ inline int cta_scratch_elems(const DevMarket& m) {
  const int NAc = round_up(m.NA, 4);
  return round_up(kMaxParam + warp_scratch_elems(m.NP, m.n_fwd) + 2 * NAc + 32 + 4 * 72 + 4 * 16 + round_up(m.NA * cta_y_stride(), 4) +
                      round_up(cta_pq_tables<R>() * m.ND * cta_pq_len(m.NA), 4) + 4 * m.ND + 4 * m.n_swap +
                      round_up(m.n_swap, 4) + 4 * m.n_swap + (m.qf_own ? round_up(3 * m.n_seg, 4) : 0),
                  4);
}

template <class R>
__device__ __forceinline__ CtaScratch<R> cta_scratch(R* base, const DevMarket& m) {
  CtaScratch<R> s;
  const int NAc = round_up(m.NA, 4);
  R* p = base;
  s.xs = p; p += kMaxParam;
  s.cap = warp_scratch<R>(p, m.NP, m.n_fwd); p += warp_scratch_elems(m.NP, m.n_fwd);
  s.Ep = (Q2<R>*)p; p += 2 * NAc;
  s.Tq = (Q4<R>*)p; p += 32;
  s.T2 = (Q4<R>*)p; p += 4 * 72;
  s.Sq = (Q4<R>*)p; p += 4 * 16;
  s.Y = p; p += round_up(m.NA * cta_y_stride(), 4);
  s.PQ = p; p += round_up(cta_pq_tables<R>() * m.ND * cta_pq_len(m.NA), 4);
  s.crq = (Q4<R>*)p; p += 4 * m.ND;
  s.F4s = (Q4<R>*)p; p += 4 * m.n_swap;
  s.A3s = p; p += round_up(m.n_swap, 4);
  s.RCs = (Q4<R>*)p; p += 4 * m.n_swap;
  s.Qs = m.qf_own ? p : s.Y;
  return s;
}

template <class R> __device__ __forceinline__ const R* grp_u_of(const DevMarket& m);
template <> __device__ __forceinline__ const double* grp_u_of<double>(const DevMarket& m) { return m.grp_u64; }
template <> __device__ __forceinline__ const float* grp_u_of<float>(const DevMarket& m) { return m.grp_u32; }
template <class R> __device__ __forceinline__ const Q4<R>* seg_w_of(const DevMarket& m);
template <> __device__ __forceinline__ const Q4<double>* seg_w_of<double>(const DevMarket& m) {
  return (const Q4<double>*)m.seg_w64;
}
template <> __device__ __forceinline__ const Q4<float>* seg_w_of<float>(const DevMarket& m) {
  return (const Q4<float>*)m.seg_w32;
}
template <class R> __device__ __forceinline__ const R* swap_scale_of(const DevMarket& m);
template <> __device__ __forceinline__ const double* swap_scale_of<double>(const DevMarket& m) { return m.swap_scale64; }
template <> __device__ __forceinline__ const float* swap_scale_of<float>(const DevMarket& m) { return m.swap_scale32; }


// Inclusive warp scan (lanes in order).
template <class R>
__device__ __forceinline__ R warp_inclusive_scan(R v, int lane) {
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const R o = __shfl_up_sync(0xffffffffu, v, off);
    if (lane >= off) v += o;
  }
  return v;
}

// Swaption pricing of instrument k of the swaption block (S6 + S4 Black); returns the squared
// weighted residual, or writes the model vol when vols != null; with res != null it also writes the
// weighted residual sqrt(w) (P - P_mkt) (NaN where the vol is infeasible).
template <class R, int FORMULA>
__device__ __forceinline__ R price_swaption(const InstrView<R>& B, int k, const CtaScratch<R>& cs, R omb, bool& ok,
                                            double* vols, double* res = nullptr) {
  typedef Num<R> M;
  const int s = B.idx[k];
  const Q4<R> fw = cs.F4s[s];
  const Q4<R> rq = cs.RCs[s];
  RhoConsts<R> rc;
  rc.rho = rq.a;
  rc.omr_p = R(1) - rq.a;
  rc.omr_m = R(1) + rq.a;
  rc.iomr_p = rq.b;
  rc.iomr_m = rq.c;
  rc.omr2 = rq.d;
  const Q4<R> g0 = B.g0[k];
  const Q4<R> g1 = B.g1[k];
  R sig;
  if (FORMULA == 0) {
    const R z = fw.b * g0.b;
    const R zx = z_over_x_fast<R>(z, rc);
    const R corr = R(1) + g0.d * fw.c + g1.a * fw.d + g1.b * cs.A3s[s];
    sig = fw.a * g0.c * zx * corr;
  } else {
    sig = sabr_paper<R>(fw.a, rc.rho, fw.b * fw.a, g0.a, g0.b, omb);
  }
  const bool good = (sig > R(0)) && M::finite_(sig);
  if (vols) { vols[k] = good ? (double)sig : __longlong_as_double(0x7ff8000000000000LL); return R(0); }
  ok = ok && good;
  const Q4<R> g2 = B.g2[k];
  const R v = sig * g1.c;
  const R d1 = fdiv<R>(g0.a, v) + R(0.5) * v;
  const R sg = g2.b;
  const R p = sg * g1.d * (ncdf<R>(sg * d1) - g2.a * ncdf<R>(sg * (d1 - v)));
  const R r = g2.d * (p - g2.c);
  if (res) res[k] = good ? (double)r : __longlong_as_double(0x7ff8000000000000LL);
  return r * r;
}

template <class R, int FORMULA>
__device__ __forceinline__ R price_one_caplet(const InstrView<R>& B, int k, const WarpScratch<R>& ws,
                                              const RhoConsts<R>& rc, R omb, bool& ok, double* vols,
                                              double* res = nullptr) {
  typedef Num<R> M;
  const int i = B.idx[k];
  const Q4<R> fw = ws.F4[i];
  const Q4<R> g0 = B.g0[k];
  const Q4<R> g1 = B.g1[k];
  R sig;
  if (FORMULA == 0) {
    const R z = fw.b * g0.b;
    const R zx = z_over_x_fast<R>(z, rc);
    const R corr = R(1) + g0.d * fw.c + g1.a * fw.d + g1.b * ws.fA3[i];
    sig = fw.a * g0.c * zx * corr;
  } else {
    sig = sabr_paper<R>(fw.a, rc.rho, fw.b * fw.a, g0.a, g0.b, omb);
  }
  const bool good = (sig > R(0)) && M::finite_(sig);
  if (vols) { vols[k] = good ? (double)sig : __longlong_as_double(0x7ff8000000000000LL); return R(0); }
  ok = ok && good;
  const Q4<R> g2 = B.g2[k];
  const R v = sig * g1.c;
  const R d1 = fdiv<R>(g0.a, v) + R(0.5) * v;
  const R sg = g2.b;
  const R p = sg * g1.d * (ncdf<R>(sg * d1) - g2.a * ncdf<R>(sg * (d1 - v)));
  const R r = g2.d * (p - g2.c);
  if (res) res[k] = good ? (double)r : __longlong_as_double(0x7ff8000000000000LL);
  return r * r;
}

// The window integrals of a pair on diagonal e over the absolute panels [lo, hi), from the prefix
// tables of phase 4: G = PG(hi) - PG(lo) and X / theta = PA(hi) - PA(lo) + SH(hi) G - (PGS(hi) -
// PGS(lo)).  FP32: PG and PGS are float-float, so G is formed to a few ulp of itself, SH(hi) G is
// split exactly by an fma into hi + lo, and SH(hi) G - (PGS(hi) - PGS(lo)) cancels between
// operands within a factor 2 of each other (an exact subtraction), leaving an error ~ (window
// offset / window) ulp of X rather than its square.
template <class R>
__device__ __forceinline__ void window_integrals(const R* PQ, int e, int ND, int PL, int lo, int hi, R& G, R& X) {
  if constexpr (sizeof(R) == 4) {
    const float2* PG2 = (const float2*)PQ + e * PL;
    const float2* PGS2 = (const float2*)PQ + (ND + e) * PL;
    const float2* PASH = (const float2*)PQ + (2 * ND + e) * PL;
    const float2 gh = PG2[hi], gl = PG2[lo], sh2 = PGS2[hi], sl2 = PGS2[lo], ash = PASH[hi];
    const float alo = PASH[lo].x;
    G = (gh.x - gl.x) + (gh.y - gl.y);
    const R p = ash.y * G;
    const R pe = fmaf(ash.y, G, -p);
    const R dh = sh2.x - sl2.x, dl = sh2.y - sl2.y;
    X = (ash.x - alo) + ((p - dh) + (pe - dl));
  } else {
    const R* PG = PQ + e * PL;
    const R* PA = PG + ND * PL;
    const R* SH = PA + ND * PL;
    const R* PGS = SH + ND * PL;
    G = PG[hi] - PG[lo];
    X = (PA[hi] - PA[lo]) + SH[hi] * G - (PGS[hi] - PGS[lo]);
  }
}

// Objective of the point in cs.xs (every thread of the CTA calls; all return the same value).
// `red` is shared scratch of 32 objective values.
// TC: the pair Grams of phase 3 on the tensor cores (tcgen05_gram.cuh; FP32 pricing only).
// res != null: the weighted residuals of every instrument (caplets first) are written as well, by
// the pricer the search uses.
template <class R, int FORMULA, bool TC = false>
__device__ typename ObjOf<R>::T cta_objective(const DevMarket& m, const InstrView<R>& capB, const InstrView<R>& swpB,
                                              const QuadTab<R>& qt, const CtaScratch<R>& cs,
                                              typename ObjOf<R>::T* red, double* vols, TcState* tc = nullptr,
                                              double* res = nullptr) {
  typedef typename ObjOf<R>::T O;
  typedef Num<R> M;
  const int tid = threadIdx.x, nth = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = nth >> 5;
  const R a = cs.xs[0], b = cs.xs[1], c = cs.xs[2], d = cs.xs[3];
  const R ah = cs.xs[4], bh = cs.xs[5], gh = cs.xs[6], dh = cs.xs[7];
  const R phi = cs.xs[8], l1 = cs.xs[9], l2 = cs.xs[10], l3 = cs.xs[11];
  const R D = (R)m.panel;
  const int NA = m.NA, ND = m.ND, YS = cta_y_stride(), PL = cta_pq_len(NA);

  // ---- phase 1: per-chain exponential tables (every warp).  The caplet forwards' SABR parameters
  //      need no mapping of their own: a caplet on forward i is the window [0, n_i) of diagonal 0 of
  //      the pair tables (phase 5).
  {
    for (int j = tid; j < kQ * kQ; j += nth) {
      const R o2 = qt.o2[j], sw = qt.sw2[j];
      const R e = M::exp_(-gh * o2);
      Q4<R> t;
      t.a = sw * e;
      t.b = sw * bh * o2 * e;
      t.c = sw * dh;
      t.d = R(0);
      cs.T2[(j >> 3) * 9 + (j & 7)] = t;
    }
    for (int j = tid; j < kQ; j += nth) {
      const R o = qt.o[j];
      const R eg = M::exp_(-c * o), eh = M::exp_(-gh * o);
      Q4<R> t;
      t.a = eg;
      t.b = b * o * eg;
      t.c = eh;
      t.d = bh * o * eh;
      cs.Tq[j] = t;
    }
    for (int A = tid; A < NA; A += nth) {
      const R base = D * (R)A;
      Q2<R> e;
      e.a = M::exp_(-c * base);
      e.b = M::exp_(-gh * base);
      cs.Ep[A] = e;
    }
    for (int e = tid; e < ND; e += nth) {
      const R dt = D * (R)e;
      Q4<R> q;
      q.a = M::exp_(-l1 * dt);
      q.b = q.a * M::exp_(-l2 * dt);
      q.c = phi * M::exp_(-l3 * dt);
      q.d = R(0);
      cs.crq[e] = q;
    }
  }
  __syncthreads();
  const int ptid = tid, pnth = nth;

  // ---- phase 2: Y rows, one thread per (panel A, outer node q): g and h at the node once; the
  //      tensor-core form also the 8 inner-node products.  The ALU form keeps the inner rule in
  //      closed form instead: with hin(A, q, r) = alpha_A a_qr + beta_A b_qr + c_qr (alpha_A =
  //      E_h(A) a'(A), beta_A = E_h(A), {a, b, c}_qr the T2 table), the pair sum over r of
  //      hin(A) hin(B) is a bilinear form in (alpha, beta, 1) with the six per-node sums
  //      S_xy(q) = sum_r x_qr y_qr, formed here once per evaluation.
  if (!TC && ptid < 6 * kQ) {
    const int q = ptid / 6, kd = ptid - 6 * q;   // kd: aa, ab, bb, ac, bc, cc
    R acc = 0;
#pragma unroll
    for (int r = 0; r < kQ; ++r) {
      const Q4<R> t = cs.T2[q * 9 + r];
      const R x = (kd == 0 || kd == 1 || kd == 3) ? t.a : (kd == 5 ? t.c : t.b);
      const R y = kd == 0 ? t.a : ((kd == 1 || kd == 2) ? t.b : t.c);
      acc += x * y;
    }
    ((R*)cs.Sq)[q * 8 + kd] = acc;
  }
  for (int it = ptid; it < NA * kQ; it += pnth) {
    const int A = it >> 3, q = it & 7;
    const R base = D * (R)A;
    const Q2<R> E = cs.Ep[A];
    const Q4<R> t = cs.Tq[q];
    const R ahp = ah + bh * base;
    const R swq = qt.sw[q];
    const R g = E.a * ((a + b * base) * t.a + t.b) + d;
    const R vg = swq * g;
    const R vh = swq * (E.b * (ahp * t.c + t.d) + dh);
    if (TC) {
      tc_put(*tc, A, q, (float)vg);
      tc_put(*tc, A, 8 + q, (float)vh);
#pragma unroll
      for (int r = 0; r < kQ; ++r) {
        const Q4<R> t2 = cs.T2[q * 9 + r];
        tc_put(*tc, A, 16 + q * kQ + r, (float)(vg * (E.b * (ahp * t2.a + t2.b) + t2.c)));
      }
    } else {
      R* y = cs.Y + A * YS;
      y[q] = vg;
      y[8 + q] = vh;
    }
  }
  __syncthreads();

  // ---- phase 3: pair sums along the diagonals (raw, then prefix-summed in phase 4)
  const PairTables<R> pt{cs.PQ, ND, PL};
  if (TC) {
    const int N = round_up(NA, 16);
    tc_gram(*tc, N);
    // warps 0-3 hold TMEM lanes 0-127: rows 0..63 hi (hi+lo)^T, rows 64..127 lo (hi+lo)^T.
    // The upper rows go to the raw pair tables, the lower ones to a band buffer (the Y region).
    R* Tb = cs.Y;
    if (warp < 4) {
      const int row = warp * 32 + lane;
      const bool top = row < 64;
      const int A = top ? row : row - 64;
      for (int g = 0; g < 3; ++g) {
        const int q = g == 0 ? 0 : (g == 1 ? 2 : 1);   // PQ slots: 0 = G, 1 = A-part, 2 = H
        for (int c0 = 0; c0 < N; c0 += 16) {
          float v[16];
          tc_ld16(tc->tmem + (uint32_t)(g * N + c0) + ((uint32_t)(warp * 32) << 16), v);
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const int e = c0 + j - A;
            if (A < NA && e >= 0 && e < ND && c0 + j < NA) {
              if (top) pt.raw(q, e, A) = (R)v[j];
              else Tb[(q * ND + e) * NA + A] = (R)v[j];
            }
          }
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    }
    __syncthreads();
    for (int it = tid; it < 3 * ND * NA; it += nth) {
      const int q = it / (ND * NA), r = it - q * ND * NA, e = r / NA, A = r - e * NA;
      if (A + e < NA) pt.raw(q, e, A) += Tb[(q * ND + e) * NA + A];
    }
  } else {
    // one thread per (panel A, block of 4 diagonals): the Y row of A is loaded once per 4 pairs
    const int NEB = (ND + 3) >> 2;
    for (int it = ptid; it < NEB * NA; it += pnth) {
      const int eb = it / NA, A = it - eb * NA, e0 = 4 * eb;
      const R* ya = cs.Y + A * YS;
      const R* yb[4];
      bool in[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        in[u] = e0 + u < ND && A + e0 + u < NA;
        yb[u] = cs.Y + (in[u] ? A + e0 + u : A) * YS;
      }
      if constexpr (sizeof(R) == 4) {
        // FP32: the four diagonals as two packed pairs (u = 0, 1 and 2, 3), one .f32x2 instruction
        // per pair of products, sums and fmas
        const float bA = cs.Ep[A].b, aA = bA * (ah + bh * (D * (float)A));
        float2 cp[2], cq[2], cr[2], cu[2], cv[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          float a2[2], b2[2];
#pragma unroll
          for (int t = 0; t < 2; ++t) {
            const int u = 2 * h + t;
            const int B = in[u] ? A + e0 + u : A;
            b2[t] = cs.Ep[B].b;
            a2[t] = b2[t] * (ah + bh * (D * (float)B));
          }
          const float2 aB = make_float2(a2[0], a2[1]), bB = make_float2(b2[0], b2[1]);
          cp[h] = mul2(bc2(aA), aB);
          cq[h] = fma2(bc2(aA), bB, mul2(bc2(bA), aB));
          cr[h] = mul2(bc2(bA), bB);
          cu[h] = add2(bc2(aA), aB);
          cv[h] = add2(bc2(bA), bB);
        }
        float2 G2[2] = {bc2(0.f), bc2(0.f)}, H2[2] = {bc2(0.f), bc2(0.f)}, A2[2] = {bc2(0.f), bc2(0.f)};
#pragma unroll
        for (int k = 0; k < 8; k += 4) {
          const float4 x = *(const float4*)(ya + k);
          float4 y[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) y[u] = *(const float4*)(yb[u] + k);
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const float4 s0 = *(const float4*)&cs.Sq[2 * (k + j)];
            const float4 s1 = *(const float4*)&cs.Sq[2 * (k + j) + 1];
            const float xa = j == 0 ? x.x : (j == 1 ? x.y : (j == 2 ? x.z : x.w));
#pragma unroll
            for (int h = 0; h < 2; ++h) {
              const float4& p = y[2 * h];
              const float4& q = y[2 * h + 1];
              const float2 yy = j == 0 ? make_float2(p.x, q.x)
                                       : (j == 1 ? make_float2(p.y, q.y) : (j == 2 ? make_float2(p.z, q.z) : make_float2(p.w, q.w)));
              const float2 pr = mul2(bc2(xa), yy);
              G2[h] = add2(G2[h], pr);
              float2 form = fma2(cv[h], bc2(s1.x), bc2(s1.y));
              form = fma2(cu[h], bc2(s0.w), form);
              form = fma2(cr[h], bc2(s0.z), form);
              form = fma2(cq[h], bc2(s0.y), form);
              form = fma2(cp[h], bc2(s0.x), form);
              A2[h] = fma2(pr, form, A2[h]);
            }
          }
        }
#pragma unroll
        for (int k = 8; k < 16; k += 4) {
          const float4 x = *(const float4*)(ya + k);
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const float4 p = *(const float4*)(yb[2 * h] + k);
            const float4 q = *(const float4*)(yb[2 * h + 1] + k);
            H2[h] = fma2(bc2(x.x), make_float2(p.x, q.x), H2[h]);
            H2[h] = fma2(bc2(x.y), make_float2(p.y, q.y), H2[h]);
            H2[h] = fma2(bc2(x.z), make_float2(p.z, q.z), H2[h]);
            H2[h] = fma2(bc2(x.w), make_float2(p.w, q.w), H2[h]);
          }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
          if (in[u]) {
            const int e = e0 + u, h = u >> 1;
            const float g = (u & 1) ? G2[h].y : G2[h].x;
            const float ad = (u & 1) ? A2[h].y : A2[h].x;
            const float hh = (u & 1) ? H2[h].y : H2[h].x;
            pt.G(e, A) = g;
            ((float2*)cs.PQ + 2 * ND * PL)[e * PL + A] = make_float2(ad, hh);
          }
      } else {
      R G[4], H[4], Ad[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) { G[u] = 0; H[u] = 0; Ad[u] = 0; }
      // (alpha, beta) of panel A and of the 4 partner panels: the pair coefficients of the form
      const R bA = cs.Ep[A].b, aA = bA * (ah + bh * (D * (R)A));
      R cp[4], cq[4], cr[4], cu[4], cv[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int B = in[u] ? A + e0 + u : A;
        const R bB = cs.Ep[B].b, aB = bB * (ah + bh * (D * (R)B));
        cp[u] = aA * aB;
        cq[u] = aA * bB + bA * aB;
        cr[u] = bA * bB;
        cu[u] = aA + aB;
        cv[u] = bA + bB;
      }
#pragma unroll
      for (int k = 0; k < 8; k += 4) {
        const Q4<R> x = *(const Q4<R>*)(ya + k);
        Q4<R> y[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) y[u] = *(const Q4<R>*)(yb[u] + k);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const Q4<R> s0 = cs.Sq[2 * (k + j)], s1 = cs.Sq[2 * (k + j) + 1];
          const R xa = j == 0 ? x.a : (j == 1 ? x.b : (j == 2 ? x.c : x.d));
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const R ya_ = j == 0 ? y[u].a : (j == 1 ? y[u].b : (j == 2 ? y[u].c : y[u].d));
            G[u] += xa * ya_;
            const R form = cp[u] * s0.a + cq[u] * s0.b + cr[u] * s0.c + cu[u] * s0.d + cv[u] * s1.a + s1.b;
            Ad[u] += (xa * ya_) * form;
          }
        }
      }
#pragma unroll
      for (int k = 8; k < 16; k += 4) {
        const Q4<R> x = *(const Q4<R>*)(ya + k);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const Q4<R> y = *(const Q4<R>*)(yb[u] + k);
          H[u] += x.a * y.a;
          H[u] += x.b * y.b;
          H[u] += x.c * y.c;
          H[u] += x.d * y.d;
        }
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (in[u]) {
          const int e = e0 + u;
          if constexpr (sizeof(R) == 4) {
            pt.G(e, A) = G[u];
            ((float2*)cs.PQ + 2 * ND * PL)[e * PL + A] = make_float2(Ad[u], H[u]);
          } else {
            pt.G(e, A) = G[u];
            pt.Ac(e, A) = Ad[u];
            pt.H(e, A) = H[u];
          }
        }
      }
    }
  }
  __syncthreads();

  // ---- phase 4: exclusive prefix sums along each diagonal, one diagonal per 8-lane group (five
  //      panels per lane and chunk of 40): four diagonals per warp at a time.  In FP32 the prefix
  //      sums of G and of G x (inclusive H prefix) are float-float (hi in PG / PGS, lo in PGl /
  //      PGSl): the window integrals are their differences, which would otherwise lose a factor
  //      (offset + window) / window of G's bits, and its square in X.
  {
    constexpr bool kFF = sizeof(R) == 4;
    constexpr int kL = 8, kE = 5, kC = kL * kE;   // lanes per diagonal, panels per lane, per chunk
    const int hw = lane >> 3, l8 = lane & 7;
    auto scan8 = [l8](R v) {   // inclusive scan within each 8-lane group
#pragma unroll
      for (int off = 1; off < kL; off <<= 1) {
        const R o = __shfl_up_sync(0xffffffffu, v, off, kL);
        if (l8 >= off) v += o;
      }
      return v;
    };
    auto scan8_ff = [l8](FF v) {   // inclusive float-float scan within each 8-lane group
#pragma unroll
      for (int off = 1; off < kL; off <<= 1) {
        FF o;
        o.hi = __shfl_up_sync(0xffffffffu, v.hi, off, kL);
        o.lo = __shfl_up_sync(0xffffffffu, v.lo, off, kL);
        if (l8 >= off) v = ff_add(v, o);
      }
      return v;
    };
    for (int eb = 4 * warp; eb < ND; eb += 4 * nw) {
      const int e = eb + hw;
      const int n = e < ND ? NA - e : 0;   // a group without a diagonal reads and writes nothing
      const int nmax = NA - eb;            // the first group's diagonal is the longest
      const int ee = e < ND ? e : eb;
      R cg = 0, ca = 0, chh = 0, cgs = 0;
      FF cgf = {0.f, 0.f}, cgsf = {0.f, 0.f};
      for (int c0 = 0; c0 < nmax; c0 += kC) {
        const int A0 = c0 + kE * l8;
        R g[kE], a[kE], h[kE];
#pragma unroll
        for (int j = 0; j < kE; ++j) {
          const bool in = A0 + j < n;
          g[j] = in ? pt.G(ee, A0 + j) : R(0);
          a[j] = in ? pt.Ac(ee, A0 + j) : R(0);
          h[j] = in ? pt.H(ee, A0 + j) : R(0);
        }
        R sa = 0, sh = 0;
#pragma unroll
        for (int j = 0; j < kE; ++j) { sa += a[j]; sh += h[j]; }
        const R ia = scan8(sa), ih = scan8(sh);
        const R hx = chh + ih - sh;   // exclusive prefix of H before A0
        R gs[kE];
        {
          R hin = hx;
#pragma unroll
          for (int j = 0; j < kE; ++j) {   // G(A) times the inclusive H prefix at A
            hin += h[j];
            gs[j] = g[j] * hin;
          }
        }
        if constexpr (kFF) {
          FF lg = ff_of(g[0]), lgs = ff_of(gs[0]);
#pragma unroll
          for (int j = 1; j < kE; ++j) {
            lg = ff_add_f(lg, g[j]);
            lgs = ff_add_f(lgs, gs[j]);
          }
          const FF ig = scan8_ff(lg), igs = scan8_ff(lgs);
          FF xg, xgs;   // exclusive prefixes at A0 within the chunk
          xg.hi = __shfl_up_sync(0xffffffffu, ig.hi, 1, kL);
          xg.lo = __shfl_up_sync(0xffffffffu, ig.lo, 1, kL);
          xgs.hi = __shfl_up_sync(0xffffffffu, igs.hi, 1, kL);
          xgs.lo = __shfl_up_sync(0xffffffffu, igs.lo, 1, kL);
          if (l8 == 0) { xg = ff_of(0.f); xgs = ff_of(0.f); }
          __syncwarp();
          FF pg = ff_add(cgf, xg), pgs = ff_add(cgsf, xgs);
          R pa = ca + ia - sa, ph = hx;
#pragma unroll
          for (int j = 0; j < kE; ++j) {
            if (A0 + j < n) {
              float2* T2p = (float2*)cs.PQ + ee * PL + A0 + j;
              T2p[0] = make_float2(pg.hi, pg.lo);
              T2p[ND * PL] = make_float2(pgs.hi, pgs.lo);
              T2p[2 * ND * PL] = make_float2(pa, ph);
            }
            pg = ff_add_f(pg, g[j]);
            pa += a[j];
            ph += h[j];
            pgs = ff_add_f(pgs, gs[j]);
          }
          FF tg, tgs;
          tg.hi = __shfl_sync(0xffffffffu, ig.hi, kL - 1, kL);
          tg.lo = __shfl_sync(0xffffffffu, ig.lo, kL - 1, kL);
          tgs.hi = __shfl_sync(0xffffffffu, igs.hi, kL - 1, kL);
          tgs.lo = __shfl_sync(0xffffffffu, igs.lo, kL - 1, kL);
          cgf = ff_add(cgf, tg);
          cgsf = ff_add(cgsf, tgs);
        } else {
          R sg = 0, sgs = 0;
#pragma unroll
          for (int j = 0; j < kE; ++j) { sg += g[j]; sgs += gs[j]; }
          const R ig = scan8(sg);
          const R igs = scan8(sgs);
          __syncwarp();
          R pg = cg + ig - sg, pa = ca + ia - sa, ph = hx, pgs = cgs + igs - sgs;
#pragma unroll
          for (int j = 0; j < kE; ++j) {
            if (A0 + j < n) {
              R* P = cs.PQ + ee * PL + A0 + j;
              P[0] = pg;
              P[ND * PL] = pa;
              P[2 * ND * PL] = ph;
              P[3 * ND * PL] = pgs;
            }
            pg += g[j];
            pa += a[j];
            ph += h[j];
            pgs += gs[j];
          }
          cg += __shfl_sync(0xffffffffu, ig, kL - 1, kL);
          cgs += __shfl_sync(0xffffffffu, igs, kL - 1, kL);
        }
        ca += __shfl_sync(0xffffffffu, ia, kL - 1, kL);
        chh += __shfl_sync(0xffffffffu, ih, kL - 1, kL);
        __syncwarp();
      }
      if (e < ND && l8 == 0) {
        if constexpr (kFF) {
          float2* T2p = (float2*)cs.PQ + e * PL + n;
          T2p[0] = make_float2(cgf.hi, cgf.lo);
          T2p[ND * PL] = make_float2(cgsf.hi, cgsf.lo);
          T2p[2 * ND * PL] = make_float2(ca, chh);
        } else {
          R* P = cs.PQ + e * PL + n;
          P[0] = cg;
          P[ND * PL] = ca;
          P[2 * ND * PL] = chh;
          P[3 * ND * PL] = cgs;
        }
      }
    }
  }
  __syncthreads();

  // ---- phase 5: the quadratic forms by expiry group.  The frozen weights of a swap are W_i = u_i /
  //      (A S^b) with u_i = tau_i P(0, T_{i+1}) F_i^b independent of the swap, and the swaps of a
  //      group share their first forward, so each is a leading block of the group's window:
  //        V_k(swap) = sum_{i <= j < L} (2 - [i = j]) W_i W_j B_k[i, j] = scale(swap) Q_k(g, L),
  //        Q_k(g, L) = sum_{j < L} u_j sum_{i <= j} (2 - [i = j]) u_i B_k[i, j],
  //      B = (rho G, rho theta X, phi G) of the pair, its window integrals from the prefix tables.
  //      (a) segments of <= kSeg pairs of one column, one thread each (segment s of S takes the
  //      pairs s + S r: consecutive lanes read consecutive diagonals), weights (2 - [i = j]) u_i u_j;
  //      (b) per swap, the sum of the segments of its group's first L columns (a contiguous range),
  //      V = scale Q, and the swap-rate SABR factors; per caplet forward i, alpha_i and nu_i from the
  //      window [0, n_i) of diagonal 0 (theta_ii = 1), the caplet's own Rebonato mapping.
  {
    R* Ps = cs.Qs;                  // [3 x n_seg]
    const int ns = m.n_seg;
    for (int q = tid; q < ns; q += nth) {
      const int4 d = m.seg_dsc[q];
      const Q4<R> w = seg_w_of<R>(m)[q];
      const R wr[4] = {w.a, w.b, w.c, w.d};
      R s1 = 0, s2 = 0, s3 = 0;
      // all kSeg slots evaluated (an empty slot repeats pair (j, j) with weight 0), so that the
      // loads of the pairs are independent and issue together
#pragma unroll
      for (int r = 0; r < kSeg; ++r) {
        const int lo = (d.x >> (8 * r)) & 255, e = (d.y >> (8 * r)) & 255;
        R G, X;
        window_integrals<R>(cs.PQ, e, ND, PL, lo, lo + d.z, G, X);
        const Q4<R> cr = cs.crq[e];
        s1 += wr[r] * (cr.a * G);
        s2 += wr[r] * (cr.b * X);
        s3 += wr[r] * (cr.c * G);
      }
      Ps[q] = s1;
      Ps[ns + q] = s2;
      Ps[2 * ns + q] = s3;
    }
    __syncthreads();
    const R* SC = swap_scale_of<R>(m);
    for (int s = tid; s < m.n_swap + m.n_capfwd; s += nth) {
      if (s >= m.n_swap) {   // a caplet forward: diagonal 0, window [0, n_i)
        const int i = m.capfwd_list[s - m.n_swap];
        const R Ti = (R)m.T[i];
        R G, X;
        window_integrals<R>(cs.PQ, 0, ND, PL, 0, m.fwd_np[i], G, X);
        const R al = fsqrt<R>(fdiv<R>(G, Ti));
        const R X2 = R(2) * X;
        put_forward<R>(cs.cap, i, al, X2 > R(0) ? fdiv<R>(fsqrt<R>(X2), al * Ti) : R(0), phi);
        continue;
      }
      // the segments of the group's first L columns (their weights carry u_i u_j)
      const int2 sr = m.swap_segs[s];
      R q1 = 0, q2 = 0, q3 = 0;
      for (int q = sr.x; q < sr.y; ++q) {
        q1 += Ps[q];
        q2 += Ps[ns + q];
        q3 += Ps[2 * ns + q];
      }
      const R sc = SC[s];
      const R v1 = sc * q1, v2 = sc * q2, v3 = sc * q3;
      // (FP32: the hardware reciprocal and reciprocal square root, as in the caplet mapping; FP64
      // exact.  nu = 0 stays 0.)
      const R TE = (R)m.swap_TE[s];
      const R al = fsqrt<R>(fdiv<R>(v1, TE));
      const R v2x = R(2) * v2;
      const R nu = v2x > R(0) ? fdiv<R>(fsqrt<R>(v2x), al * TE) : R(0);
      R rho = fdiv<R>(v3, v1);
      rho = rho > R(0.999) ? R(0.999) : (rho < R(-0.999) ? R(-0.999) : rho);
      Q4<R> f;
      f.a = al;
      f.b = fdiv<R>(nu, al);
      f.c = al * al;
      f.d = rho * nu * al;
      cs.F4s[s] = f;
      cs.A3s[s] = (R(2) - R(3) * rho * rho) * nu * nu;
      Q4<R> q;
      q.a = rho;
      q.b = fdiv<R>(R(1), R(1) - rho);
      q.c = fdiv<R>(R(1), R(1) + rho);
      q.d = (R(1) - rho) * (R(1) + rho);
      cs.RCs[s] = q;
    }
    __syncthreads();
  }

  // ---- phase 6: price every caplet and swaption, reduce
  RhoConsts<R> rc;
  rc.init(phi);
  const R omb = (R)(1.0 - m.beta);
  bool ok = true;
  R part = 0;
  const int ntot = m.n_cap + m.n_swp;
  if constexpr (std::is_same<R, float>::value && FORMULA == 0) {
    if (vols == nullptr) {
      // FP32, Hagan (2002): instruments k and k + nth as a packed pair (either kind)
      float2 acc = bc2(0.0f);
      for (int k = tid; k < ntot; k += 2 * nth) {
        const bool has2 = k + nth < ntot;
        Q4<float> F[2], g0[2], g1[2], g2[2];
        float a3[2], rh[2];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
          const int kk = (u == 1 && has2) ? k + nth : k;
          if (kk < m.n_cap) {
            const int i = capB.idx[kk];
            F[u] = cs.cap.F4[i];
            a3[u] = cs.cap.fA3[i];
            rh[u] = phi;
            g0[u] = capB.g0[kk]; g1[u] = capB.g1[kk]; g2[u] = capB.g2[kk];
          } else {
            const int j = kk - m.n_cap, sw = swpB.idx[j];
            F[u] = cs.F4s[sw];
            a3[u] = cs.A3s[sw];
            rh[u] = cs.RCs[sw].a;
            g0[u] = swpB.g0[j]; g1[u] = swpB.g1[j]; g2[u] = swpB.g2[j];
          }
        }
        bool oka = true, okb = true;
        float2 r = price_pair_x2(F[0], F[1], a3[0], a3[1], rh[0], rh[1], g0[0], g0[1], g1[0], g1[1], g2[0], g2[1],
                                 oka, okb);
        r.y = has2 ? r.y : 0.0f;
        ok = ok && oka && (okb || !has2);
        if (res) {
          const double qnan = __longlong_as_double(0x7ff8000000000000LL);
          res[k] = oka ? (double)r.x : qnan;
          if (has2) res[k + nth] = okb ? (double)r.y : qnan;
        }
        acc = fma2(r, r, acc);
      }
      part = acc.x + acc.y;
    } else {
      for (int k = tid; k < ntot; k += nth) {
        if (k < m.n_cap) part += price_one_caplet<R, FORMULA>(capB, k, cs.cap, rc, omb, ok, vols);
        else part += price_swaption<R, FORMULA>(swpB, k - m.n_cap, cs, omb, ok, vols + m.n_cap);
      }
    }
  } else {
    for (int k = tid; k < ntot; k += nth) {
      if (k < m.n_cap) part += price_one_caplet<R, FORMULA>(capB, k, cs.cap, rc, omb, ok, vols, res);
      else part += price_swaption<R, FORMULA>(swpB, k - m.n_cap, cs, omb, ok, vols ? vols + m.n_cap : nullptr,
                                              res ? res + m.n_cap : nullptr);
    }
  }
  const int bad = __syncthreads_or(!ok);
  if (vols) return obj_inf(O());
  O wsum;
  if constexpr (std::is_same<R, float>::value) wsum = warp_sum_lanes_f32(part);
  else wsum = warp_sum_lanes(part);
  if (lane == 0) red[warp] = wsum;
  __syncthreads();
  O f = red[0];
  for (int w = 1; w < nw; ++w) f = obj_add(f, red[w]);
  __syncthreads();   // red is reused by the next evaluation
  if (bad || !obj_finite(f)) return obj_inf(O());
  return f;
}

}  // namespace sabr
