// Hand-written reverse-mode (adjoint) sweep of the objective of markets with swaptions, one CTA per
// parameter point, FP64.
//
// Forward sweep: cta_objective (swaption.cuh) with the quadratic forms' partials in a region of
// their own, so that every table the reverse sweep reads is still in shared memory afterwards: the
// per-chain exponential tables (Ep, Tq, T2, Sq, crq), the Y rows, the prefix tables along the
// diagonals, the column sums of the group forms, the swap-rate SABR factors and the caplet
// forwards' factors.  Reverse sweep, in the opposite order:
//   f = sum r_k^2, r = sqrt(w)(P - P_mkt), P = Black(sigma)       sigma_bar = 2 r sqrt(w) vega
//   sigma = SABR(alpha, nu, rho) per caplet forward / per swap      (alpha, nu, rho)_bar
//   alpha_S = sqrt(V1/T), nu_S = sqrt(2 V2)/(alpha_S T),
//   rho_S = clamp(V3/V1)                                             V_bar (per swap)
//   V_k = scale Q_k(g, L), Q the sum of a group's first L columns    Q_bar, then column sums' bars
//   column sum = u_j sum_i (2 - [i=j]) u_i B_k[i, j]                 B_bar per pair
//   caplet forward i: alpha_i, nu_i from its window [0, n_i) of diagonal 0  G_bar, X_bar of that window
//   B = (rho_e G, rho_e theta_e X, phi_e G)                          G_bar, X_bar, (rho, rho theta, phi)_bar per diagonal
//   G = PG(hi) - PG(lo), X = PA(hi) - PA(lo) + SH(hi) G - (PGS(hi) - PGS(lo))
//                                                                    adjoints of the prefix tables (atomics)
//   PG, PA, SH, PGS exclusive prefix sums of G, A, H, G SH_incl      cell adjoints (suffix sums)
//   G, H, A cells = Gram sums of the Y rows, A with the inner rule's
//   bilinear form in (alpha_A, beta_A, alpha_B, beta_B; Sq)          Y_bar (gather), panel and Sq adjoints
//   Y rows = sqrt(w_q) g(u), sqrt(w_q) h(u)                          parameter adjoints (a .. delta_h)
//   Sq = sums over the inner nodes of T2 products, T2 = f(gamma_h, beta_h, delta_h)
//   rho_e = e^{-l1 dt}, theta_e = e^{-l2 dt}, phi_e = phi e^{-l3 dt}  (lambda1..3, phi)_bar
// The caplets' prices go through caplet_price_reverse (adjoint.cuh); their forwards' parameters are
// windows of diagonal 0 and join the swaptions' reverse sweep there.
#pragma once
#include "adjoint.cuh"
#include "swaption.cuh"

namespace sabr {

// Adjoint scratch of one CTA (FP64), after the forward scratch.
struct GradScratchS {
  double* PQb;    // [4 x ND x PL] adjoints of PG, PA, SH, PGS; then the cells' G, A, H adjoints
  double* Yb;     // [NA x 16]
  double* swb;    // [3 x n_swap] alpha, nu, rho adjoints of each swap's SABR parameters
  double* Vb;     // [6 x n_col] adjoints of the column prefix sums Q, then of the column sums
  double* crqb;   // [3 x ND] rho_e, rho_e theta_e, phi_e adjoints
  double* panb;   // [2 x NA] alpha_A, beta_A adjoints (the inner-rule form's panel coefficients)
  double* Sqb;    // [64] adjoints of the inner-rule sums Sq (8 nodes x 8 slots)
  double* red;    // [32 x 16] reduction of the parameter adjoints
  AdjScratch<double> cap;   // the caplet mapping's adjoints (warp 0)
};

__host__ __device__ inline uint32_t grad_scratch_bytes_cta(const DevMarket& m) {
  const int PL = cta_pq_len(m.NA);
  size_t n = (size_t)4 * m.ND * PL + 16 * m.NA + 3 * m.n_swap + 6 * m.n_col + 3 * m.ND + 2 * m.NA + 64 + 32 * 16;
  return (uint32_t)(n * 8 + 64 + adj_scratch_bytes(m.NP, m.n_fwd, 8));
}

__device__ __forceinline__ GradScratchS grad_scratch_cta(unsigned char* base, const DevMarket& m) {
  GradScratchS g;
  const int PL = cta_pq_len(m.NA);
  double* p = (double*)base;
  g.PQb = p; p += (size_t)4 * m.ND * PL;
  g.Yb = p; p += 16 * m.NA;
  g.swb = p; p += 3 * m.n_swap;
  g.Vb = p; p += 6 * m.n_col;
  g.crqb = p; p += 3 * m.ND;
  g.panb = p; p += 2 * m.NA;
  g.Sqb = p; p += 64;
  g.red = p; p += 32 * 16;
  g.cap = adj_scratch<double>((unsigned char*)(((uintptr_t)p + 63) & ~(uintptr_t)63), m.NP, m.n_fwd);
  return g;
}

// f and df/dtheta (12 slots) of the point in cs.xs; every thread of the CTA calls; thread 0 writes
// f_out and g_out.  The market record m must carry qf_own = 1 (the forward sweep keeps the Y rows).
template <int FORMULA>
__device__ void cta_objective_grad(const DevMarket& m, const InstrView<double>& capB, const InstrView<double>& swpB,
                                   const QuadTab<double>& qt, const CtaScratch<double>& cs, double* red_fwd,
                                   const GradScratchS& gs, double* f_out, double* g_out) {
  typedef double R;
  const int tid = threadIdx.x, nth = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = nth >> 5;
  const int NA = m.NA, ND = m.ND, PL = cta_pq_len(NA), YS = cta_y_stride();
  const int ns = m.n_swap, nc = m.n_col;
  const R D = m.panel;
  // ---------------- forward sweep (leaves its tables in shared memory)
  const double f_fwd = cta_objective<R, FORMULA, false>(m, capB, swpB, qt, cs, red_fwd, nullptr);
  const R a = cs.xs[0], b = cs.xs[1], c = cs.xs[2];   // d enters g additively: its adjoint is g's
  const R ah = cs.xs[4], bh = cs.xs[5], gh = cs.xs[6], dh = cs.xs[7];
  const R phi = cs.xs[8], l1 = cs.xs[9], l2 = cs.xs[10], l3 = cs.xs[11];
  if (!isfinite(f_fwd)) {
    if (tid == 0) {
      *f_out = __longlong_as_double(0x7ff0000000000000LL);
      for (int k = 0; k < m.n_param; ++k) g_out[k] = 0.0;
    }
    __syncthreads();
    return;
  }
  // ---------------- R0: zero the accumulators
  for (int i = tid; i < 4 * ND * PL; i += nth) gs.PQb[i] = 0.0;
  for (int i = tid; i < 3 * ns; i += nth) gs.swb[i] = 0.0;
  for (int i = tid; i < 6 * nc; i += nth) gs.Vb[i] = 0.0;
  for (int i = tid; i < 3 * ND; i += nth) gs.crqb[i] = 0.0;
  for (int i = tid; i < 2 * NA; i += nth) gs.panb[i] = 0.0;
  for (int i = tid; i < 64; i += nth) gs.Sqb[i] = 0.0;
  for (int j = tid; j < m.n_capfwd; j += nth) {
    const int i = m.capfwd_list[j];
    gs.cap.abar[i] = 0.0;
    gs.cap.nbar[i] = 0.0;
  }
  __syncthreads();
  double gacc[kMaxGradParam];
#pragma unroll
  for (int k = 0; k < kMaxGradParam; ++k) gacc[k] = 0.0;
  // ---------------- R1: pricing with the local reverse sweep (caplets, then swaptions)
  bool ok = true;
  R facc = 0.0;
  double rho_bar = 0.0;
  {
    RhoConsts<R> rc;
    rc.init(phi);
    caplet_price_reverse<R, FORMULA>(m, capB, cs.cap, gs.cap, rc, tid, nth, ok, facc, rho_bar);
  }
  const R omb = 1.0 - m.beta;
  for (int k = tid; k < m.n_swp; k += nth) {
    const int s = swpB.idx[k];
    const Q4<R> rq = cs.RCs[s];
    RhoConsts<R> rc;
    rc.rho = rq.a;
    rc.omr_p = 1.0 - rq.a;
    rc.omr_m = 1.0 + rq.a;
    rc.iomr_p = rq.b;
    rc.iomr_m = rq.c;
    rc.omr2 = rq.d;
    const Q4<R> g0 = swpB.g0[k], g1 = swpB.g1[k], g2 = swpB.g2[k];
    R s_al, s_nu, s_rho;
    const R sig = sabr_vol_grad<R, FORMULA>(cs.F4s[s], cs.A3s[s], rc, g0, g1, omb, s_al, s_nu, s_rho);
    const bool good = (sig > 0.0) && isfinite(sig);
    ok = ok && good;
    if (!good) continue;
    R sbar;
    const R r = black_residual_grad<R>(sig, g0, g1, g2, sbar);
    facc += r * r;
    atomicAdd(gs.swb + s, sbar * s_al);
    atomicAdd(gs.swb + ns + s, sbar * s_nu);
    atomicAdd(gs.swb + 2 * ns + s, sbar * s_rho);
  }
  gacc[8] += rho_bar;
  const int bad = __syncthreads_or(!ok);
  // ---------------- R2: the swap-rate SABR parameters -> the forms -> the column sums; the caplet
  //      forwards' (alpha_i, nu_i) -> their window [0, n_i) on diagonal 0 -> the prefix tables
  const R* SC = m.swap_scale64;
  const R* Ps = cs.Qs;   // segment partials (forward), weights (2 - [i = j]) u_i u_j
  const int nseg = m.n_seg;
  for (int s = tid; s < ns + m.n_capfwd; s += nth) {
    if (s >= ns) {
      const int i = m.capfwd_list[s - ns];
      const int hi = m.fwd_np[i];
      const R Ti = m.T[i];
      R G, X;
      window_integrals<R>(cs.PQ, 0, ND, PL, 0, hi, G, X);
      const R al = sqrt(G / Ti);
      const R nu = 2.0 * X > 0.0 ? sqrt(2.0 * X) / (al * Ti) : 0.0;
      const R ab = gs.cap.abar[i], nb = gs.cap.nbar[i];
      const R Gb = (ab - nb * nu / al) / (2.0 * al * Ti);
      const R Xb = X > 0.0 ? nb * nu / (2.0 * X) : 0.0;
      const R* SH = cs.PQ + 2 * ND * PL;
      const R Gt = Gb + Xb * SH[hi];
      double* PGb = gs.PQb;
      atomicAdd(PGb + hi, Gt);
      atomicAdd(PGb, -Gt);
      atomicAdd(PGb + ND * PL + hi, Xb);
      atomicAdd(PGb + ND * PL, -Xb);
      atomicAdd(PGb + 2 * ND * PL + hi, Xb * G);
      atomicAdd(PGb + 3 * ND * PL + hi, -Xb);
      atomicAdd(PGb + 3 * ND * PL, Xb);
      continue;
    }
    const int col = m.grp_col0[m.swap_grp[s]] + m.swap_L[s] - 1;
    const int2 sr = m.swap_segs[s];
    R q1 = 0.0, q2 = 0.0, q3 = 0.0;
    for (int q = sr.x; q < sr.y; ++q) {
      q1 += Ps[q];
      q2 += Ps[nseg + q];
      q3 += Ps[2 * nseg + q];
    }
    const R sc = SC[s];
    const R V1 = sc * q1, V2 = sc * q2, V3 = sc * q3;
    const R TE = m.swap_TE[s];
    const R al = sqrt(V1 / TE);
    const R nu = 2.0 * V2 > 0.0 ? sqrt(2.0 * V2) / (al * TE) : 0.0;
    const R rr = V3 / V1;
    const R ab = gs.swb[s], nb = gs.swb[ns + s], rb = gs.swb[2 * ns + s];
    const R abt = ab - nb * nu / al;                 // nu = sqrt(2 V2) / (alpha T) depends on alpha
    R V1b = abt * al / (2.0 * V1);
    R V2b = V2 > 0.0 ? nb * nu / (2.0 * V2) : 0.0;
    R V3b = 0.0;
    if (rr < 0.999 && rr > -0.999) {                 // rho = V3 / V1 unclamped
      V1b -= rb * rr / V1;
      V3b = rb / V1;
    }
    gs.Vb[col] = sc * V1b;
    gs.Vb[nc + col] = sc * V2b;
    gs.Vb[2 * nc + col] = sc * V3b;
  }
  __syncthreads();
  // ---------------- R3: reverse of the sum over a swap's leading columns (suffix sums within the group)
  for (int col = tid; col < nc; col += nth) {
    int g = 0;
    while (m.grp_col0[g + 1] <= col) ++g;
    const int c1 = m.grp_col0[g + 1];
    R v1 = 0.0, v2 = 0.0, v3 = 0.0;
    for (int cc = col; cc < c1; ++cc) {
      v1 += gs.Vb[cc];
      v2 += gs.Vb[nc + cc];
      v3 += gs.Vb[2 * nc + cc];
    }
    const R uj = m.grp_u64[m.col_u[col]];
    gs.Vb[3 * nc + col] = uj * v1;
    gs.Vb[4 * nc + col] = uj * v2;
    gs.Vb[5 * nc + col] = uj * v3;
  }
  __syncthreads();
  // ---------------- R4: per pair, the B adjoints -> window integrals -> prefix-table adjoints
  {
    double* PGb = gs.PQb;
    double* PAb = PGb + ND * PL;
    double* SHb = PAb + ND * PL;
    double* PGSb = SHb + ND * PL;
    const int W = m.max_gwin;
    for (int q = tid; q < m.n_seg; q += nth) {
      const int w = m.seg[q];
      const int g = w & 255, j = (w >> 8) & 255, i0 = (w >> 16) & 255, ni = w >> 24;
      const int col = m.grp_col0[g] + j;
      const R cb1 = gs.Vb[3 * nc + col], cb2 = gs.Vb[4 * nc + col], cb3 = gs.Vb[5 * nc + col];
      const int* dl = m.grp_delta + g * W;
      const R* u = m.grp_u64 + g * W;
      const int nE = m.grp_nE[g], dj = dl[j];
      for (int i = i0; i < i0 + ni; ++i) {
        const int lo = dl[i], e = dj - lo, hi = lo + nE;
        R G, X;
        window_integrals<R>(cs.PQ, e, ND, PL, lo, hi, G, X);
        const Q4<R> cr = cs.crq[e];
        const R cij = (i == j ? 1.0 : 2.0) * u[i];
        const R B1b = cij * cb1, B2b = cij * cb2, B3b = cij * cb3;
        const R Gb = cr.a * B1b + cr.c * B3b, Xb = cr.b * B2b;
        atomicAdd(gs.crqb + e, G * B1b);
        atomicAdd(gs.crqb + ND + e, X * B2b);
        atomicAdd(gs.crqb + 2 * ND + e, G * B3b);
        const R* SH = cs.PQ + (2 * ND + e) * PL;
        const R Gt = Gb + Xb * SH[hi];
        atomicAdd(PGb + e * PL + hi, Gt);
        atomicAdd(PGb + e * PL + lo, -Gt);
        atomicAdd(PAb + e * PL + hi, Xb);
        atomicAdd(PAb + e * PL + lo, -Xb);
        atomicAdd(SHb + e * PL + hi, Xb * G);
        atomicAdd(PGSb + e * PL + hi, -Xb);
        atomicAdd(PGSb + e * PL + lo, Xb);
      }
    }
  }
  __syncthreads();
  // ---------------- R5: reverse of the exclusive prefix sums along each diagonal -> cell adjoints
  //      (in place: tables 0, 1, 2 become the adjoints of the cells' G, A, H)
  for (int e = tid; e < ND; e += nth) {
    const int n = NA - e;
    double* Gb = gs.PQb + e * PL;
    double* Ab = gs.PQb + (ND + e) * PL;
    double* Hb = gs.PQb + (2 * ND + e) * PL;
    double* GSb = gs.PQb + (3 * ND + e) * PL;
    const R* PG = cs.PQ + e * PL;
    const R* SH = cs.PQ + (2 * ND + e) * PL;
    R sG = 0.0, sA = 0.0, sH = 0.0, sGS = 0.0, tSHi = 0.0;
    R cG = Gb[n], cA = Ab[n], cH = Hb[n], cGS = GSb[n];   // adjoints at index A + 1
    for (int A = n - 1; A >= 0; --A) {
      const R nG = Gb[A], nA = Ab[A], nH = Hb[A], nGS = GSb[A];
      sG += cG;
      sA += cA;
      sH += cH;
      sGS += cGS;
      const R Gd = PG[A + 1] - PG[A];
      const R SHi = SH[A + 1];
      tSHi += Gd * sGS;
      Gb[A] = sG + SHi * sGS;
      Ab[A] = sA;
      Hb[A] = sH + tSHi;
      cG = nG;
      cA = nA;
      cH = nH;
      cGS = nGS;
    }
  }
  __syncthreads();
  // ---------------- R6a: Y row adjoints by gathering over the cells that use each row
  {
    const double* CG = gs.PQb;
    const double* CA = gs.PQb + ND * PL;
    const double* CH = gs.PQb + 2 * ND * PL;
    for (int it = tid; it < NA * 16; it += nth) {
      const int A = it >> 4, k = it & 15;
      R acc = 0.0;
      if (k < 8) {
        const int q = k;
        const Q4<R> s0 = cs.Sq[2 * q], s1 = cs.Sq[2 * q + 1];
        const R bA = cs.Ep[A].b, aA = bA * (ah + bh * (D * (R)A));
        for (int e = 0; e < ND; ++e) {
          if (A + e < NA) {        // cell (A, e): the partner panel B = A + e
            const int B = A + e;
            const R bB = cs.Ep[B].b, aB = bB * (ah + bh * (D * (R)B));
            const R form = aA * aB * s0.a + (aA * bB + bA * aB) * s0.b + bA * bB * s0.c + (aA + aB) * s0.d +
                           (bA + bB) * s1.a + s1.b;
            acc += (CG[e * PL + A] + CA[e * PL + A] * form) * cs.Y[B * YS + q];
          }
          if (A - e >= 0) {        // cell (A - e, e): this panel is the partner
            const int B = A - e;
            const R bB = cs.Ep[B].b, aB = bB * (ah + bh * (D * (R)B));
            const R form = aA * aB * s0.a + (aA * bB + bA * aB) * s0.b + bA * bB * s0.c + (aA + aB) * s0.d +
                           (bA + bB) * s1.a + s1.b;
            acc += (CG[e * PL + B] + CA[e * PL + B] * form) * cs.Y[B * YS + q];
          }
        }
      } else {
        const int q = k - 8;
        for (int e = 0; e < ND; ++e) {
          if (A + e < NA) acc += CH[e * PL + A] * cs.Y[(A + e) * YS + 8 + q];
          if (A - e >= 0) acc += CH[e * PL + A - e] * cs.Y[(A - e) * YS + 8 + q];
        }
      }
      gs.Yb[A * 16 + k] = acc;
    }
  }
  // ---------------- R6b: the inner-rule form's adjoints per cell: panel coefficients and Sq
  {
    const double* CA = gs.PQb + ND * PL;
    const int q = tid & 7;
    const Q4<R> s0 = cs.Sq[2 * q], s1 = cs.Sq[2 * q + 1];
    R sb[6] = {0, 0, 0, 0, 0, 0};
    int ncell = 0;
    for (int e = 0; e < ND; ++e) ncell += NA - e;
    // cells in diagonal-major order; 8 threads (the 8 nodes) per cell, nth / 8 cells at a time
    const int ng = nth >> 3;
    for (int base = 0; base < ncell; base += ng) {
      const int ci = base + (tid >> 3);
      R gA = 0.0, gB = 0.0, hA = 0.0, hB = 0.0;
      int A = 0, B = 0;
      if (ci < ncell) {
        int e = 0, r = ci;
        while (r >= NA - e) { r -= NA - e; ++e; }
        A = r;
        B = A + e;
        const R fb = CA[e * PL + A] * cs.Y[A * YS + q] * cs.Y[B * YS + q];
        const R bA = cs.Ep[A].b, aA = bA * (ah + bh * (D * (R)A));
        const R bB = cs.Ep[B].b, aB = bB * (ah + bh * (D * (R)B));
        gA = fb * (aB * s0.a + bB * s0.b + s0.d);   // d form / d alpha_A
        hA = fb * (aB * s0.b + bB * s0.c + s1.a);   // d form / d beta_A
        gB = fb * (aA * s0.a + bA * s0.b + s0.d);
        hB = fb * (aA * s0.b + bA * s0.c + s1.a);
        sb[0] += fb * aA * aB;
        sb[1] += fb * (aA * bB + bA * aB);
        sb[2] += fb * bA * bB;
        sb[3] += fb * (aA + aB);
        sb[4] += fb * (bA + bB);
        sb[5] += fb;
      }
#pragma unroll
      for (int off = 1; off < 8; off <<= 1) {       // the cell's 8 nodes: sum, then one atomic each
        gA += __shfl_xor_sync(0xffffffffu, gA, off);
        hA += __shfl_xor_sync(0xffffffffu, hA, off);
        gB += __shfl_xor_sync(0xffffffffu, gB, off);
        hB += __shfl_xor_sync(0xffffffffu, hB, off);
      }
      if (q == 0 && ci < ncell) {
        atomicAdd(gs.panb + A, gA);
        atomicAdd(gs.panb + NA + A, hA);
        atomicAdd(gs.panb + B, gB);
        atomicAdd(gs.panb + NA + B, hB);
      }
    }
    // Sq slots: s0 = {aa, ab, bb, ac}, s1 = {bc, cc}: the form's coefficients of those slots are
    // {cp, cq, cr, cu} and {cv, 1}
#pragma unroll
    for (int k = 0; k < 6; ++k) atomicAdd(gs.Sqb + q * 8 + k, sb[k]);
  }
  __syncthreads();
  // ---------------- R7: down to the parameters
  // Y rows: Y[A][q] = sqrt(w_q) g(u), Y[A][8 + q] = sqrt(w_q) h(u), u = D A + o_q
  for (int it = tid; it < NA * kQ; it += nth) {
    const int A = it >> 3, q = it & 7;
    const R u = D * (R)A + qt.o[q];
    const R swq = qt.sw[q];
    const R eg = exp(-c * u), eh = exp(-gh * u);
    abcd_bar<R>(gs.Yb[A * 16 + q] * swq, u, eg, a + b * u, gacc);
    abcd_bar<R>(gs.Yb[A * 16 + 8 + q] * swq, u, eh, ah + bh * u, gacc + 4);
  }
  // panel coefficients: alpha_A = beta_A (alpha_h + beta_h D A), beta_A = e^{-gamma_h D A}
  for (int A = tid; A < NA; A += nth) {
    const R t = D * (R)A;
    const R bA = exp(-gh * t), aA = bA * (ah + bh * t);
    const R ab = gs.panb[A], bb = gs.panb[NA + A];
    gacc[4] += ab * bA;
    gacc[5] += ab * bA * t;
    gacc[6] += -t * (ab * aA + bb * bA);
  }
  // Sq = sums over the inner nodes of products of T2 = {sw2 e^{-gamma_h o2}, sw2 beta_h o2
  // e^{-gamma_h o2}, sw2 delta_h}
  for (int it = tid; it < kQ * kQ; it += nth) {
    const int q = it >> 3;
    const R o2 = qt.o2[it], sw2 = qt.sw2[it];
    const R ta = sw2 * exp(-gh * o2), tb = ta * bh * o2, tc = sw2 * dh;
    const double* S = gs.Sqb + q * 8;   // aa, ab, bb, ac, bc, cc
    const R tab = 2.0 * S[0] * ta + S[1] * tb + S[3] * tc;
    const R tbb = S[1] * ta + 2.0 * S[2] * tb + S[4] * tc;
    const R tcb = S[3] * ta + S[4] * tb + 2.0 * S[5] * tc;
    gacc[6] += -o2 * (tab * ta + tbb * tb);
    gacc[5] += tbb * o2 * ta;
    gacc[7] += tcb * sw2;
  }
  // per-diagonal correlations: rho_e = e^{-l1 dt}, rho_e theta_e = e^{-(l1 + l2) dt}, phi_e = phi e^{-l3 dt}
  for (int e = tid; e < ND; e += nth) {
    const R dt = D * (R)e;
    const R r1 = exp(-l1 * dt), r2 = r1 * exp(-l2 * dt), e3 = exp(-l3 * dt);
    const R b1 = gs.crqb[e], b2 = gs.crqb[ND + e], b3 = gs.crqb[2 * ND + e];
    gacc[9] += -dt * (b1 * r1 + b2 * r2);
    gacc[10] += -dt * b2 * r2;
    gacc[11] += -dt * b3 * phi * e3;
    gacc[8] += b3 * e3;
  }
  // ---------------- R8: reduce f and the parameter adjoints over the CTA
  R fsum = facc;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) fsum += __shfl_xor_sync(0xffffffffu, fsum, off);
#pragma unroll
  for (int k = 0; k < kMaxGradParam; ++k) gacc[k] = warp_sum_d(gacc[k]);
  if (lane == 0) {
    gs.red[warp * 16 + 12] = fsum;
#pragma unroll
    for (int k = 0; k < kMaxGradParam; ++k) gs.red[warp * 16 + k] = gacc[k];
  }
  __syncthreads();
  if (tid == 0) {
    double f = 0.0, g[kMaxGradParam];
    for (int k = 0; k < kMaxGradParam; ++k) g[k] = 0.0;
    for (int w = 0; w < nw; ++w) {
      f += gs.red[w * 16 + 12];
      for (int k = 0; k < kMaxGradParam; ++k) g[k] += gs.red[w * 16 + k];
    }
    const bool fin = !bad && isfinite(f);
    *f_out = fin ? f : __longlong_as_double(0x7ff0000000000000LL);
    for (int k = 0; k < m.n_param; ++k) g_out[k] = fin ? g[k] : 0.0;
  }
  __syncthreads();
}

}  // namespace sabr
