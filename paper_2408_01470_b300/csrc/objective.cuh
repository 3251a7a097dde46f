// Warp-cooperative evaluation of the calibration objective for one parameter point.
//
// One warp owns one parameter point (one annealing chain).  The market's instrument blocks and
// the quadrature table sit in shared memory (staged once per CTA by a bulk copy); each warp has
// a private scratch region for the per-panel integrals and the per-forward SABR factors of its
// point.
//
//   S2  rebonato_forward_params : Eq. (haganForRebonato) for every caplet forward, by the
//       composite Gauss-Legendre rule written in time-to-fixing u.  Time homogeneity makes one
//       table of panel integrals serve every maturity: panel p of [0, T_i] in u is the same
//       interval [pD, (p+1)D] for every i, so
//         G_i = sum_{p < n_i} Gp[p],   X_i = sum_{p < n_i} (Ap[p] + Gp[p] sum_{p < p' < n_i} Hp[p'])
//       with Gp = int g^2, Hp = int h^2 over panel p and Ap = int g(u)^2 R(u) over panel p,
//       R(u) the inner rule on [u, panel top].  (The same discrete sums as a direct rule in
//       calendar time, reordered.)  Lanes split (panel, node).  With base = pD and a node at
//       base + o, the exponentials factor as e^{-c(base + o)} = e^{-c base} e^{-c o}, so
//         g(base + o) = E_g(p) ((a + b base) e_g(o) + b o e_g(o)) + d
//       and likewise h; the per-node factors e(o), o e(o) and, for the inner rule, six weighted
//       sums per outer node (the square of h expanded in E_h(p)) are tabulated once per
//       evaluation in the warp's scratch, and the sums over panels are warp prefix scans.
//   S4  price_caplets : per caplet, SABR vol -> OTM Black price -> vega-weighted residual.
//   S7  squared residuals summed per lane in the pricing precision; across lanes in FP64 (FP64
//       path) or in float-float, a 48-bit significand on the FP32 pipes (FP32 path).
#pragma once
#include <type_traits>
#include "device_math.cuh"
#include "market.cuh"

namespace sabr {

// Division and square root of the pricing precision: IEEE in FP64, the hardware approximations
// in FP32.
template <class R> __device__ __forceinline__ R fdiv(R a, R b);
template <> __device__ __forceinline__ double fdiv<double>(double a, double b) { return a / b; }
template <> __device__ __forceinline__ float fdiv<float>(float a, float b) { return a * rcp_approx(b); }
template <class R> __device__ __forceinline__ R fsqrt(R a);
template <> __device__ __forceinline__ double fsqrt<double>(double a) { return sqrt(a); }
template <> __device__ __forceinline__ float fsqrt<float>(float a) { return a * rsqrt_approx(a); }   // a > 0 here
// log1p on the non-negative argument of x(z)
template <class R> __device__ __forceinline__ R log1p_zx(R y);
template <> __device__ __forceinline__ double log1p_zx<double>(double y) { return log1p(y); }
template <> __device__ __forceinline__ float log1p_zx<float>(float y) { return log1p_pos(y); }

template <class R> struct Q2 { R a, b; };

// Per-forward SABR factors consumed by the pricer:
//   F4 = {alpha, nu / alpha, alpha^2, rho nu alpha},  fA3 = (2 - 3 rho^2) nu^2.
template <class R> struct WarpScratch {
  R* xs;        // [kMaxParam] parameter point in the pricing precision
  R* Gp;        // [NPc] per-panel integrals
  R* Hp;
  R* Ap;
  Q4<R>* F4;    // [NFc]
  R* fA3;       // [NFc]
  Q2<R>* Ep;    // [NPc] {e^{-c pD}, e^{-gamma_h pD}}
  Q4<R>* Tq;    // [8]   {e_g(o_q), b o_q e_g(o_q), e_h(o_q), beta_h o_q e_h(o_q)}
  Q4<R>* T2;    // [8 x 2]: per outer node, the inner-rule sums {S1..S4}, {S5, S6, -, -}
};

__host__ __device__ inline int round_up(int x, int m) { return (x + m - 1) / m * m; }

// Elements (of R) of one warp's scratch; a multiple of 4 so that every region stays aligned to
// 4 elements (the alignment of Q4<R>).
__host__ __device__ inline int warp_scratch_elems(int NP, int n_fwd) {
  const int NPc = round_up(NP > 0 ? NP : 1, 4), NFc = round_up(n_fwd, 4);
  return kMaxParam + 3 * NPc + 4 * NFc + NFc + 2 * NPc + 4 * 8 + 4 * 16;
}

template <class R>
__device__ __forceinline__ WarpScratch<R> warp_scratch(R* base, int NP, int n_fwd) {
  WarpScratch<R> s;
  const int NPc = round_up(NP > 0 ? NP : 1, 4), NFc = round_up(n_fwd, 4);
  s.xs = base;
  s.Gp = base + kMaxParam;
  s.Hp = s.Gp + NPc;
  s.Ap = s.Hp + NPc;
  s.F4 = (Q4<R>*)(s.Ap + NPc);
  s.fA3 = (R*)(s.F4 + NFc);
  s.Ep = (Q2<R>*)(s.fA3 + NFc);
  s.Tq = (Q4<R>*)(s.Ep + NPc);
  s.T2 = s.Tq + 8;
  return s;
}

// Per-forward factors from (alpha, nu) and the chain's rho.
template <class R>
__device__ __forceinline__ void put_forward(const WarpScratch<R>& ws, int i, R al, R nu, R rho) {
  Q4<R> v;
  v.a = al;
  v.b = fdiv<R>(nu, al);
  v.c = al * al;
  v.d = rho * nu * al;
  ws.F4[i] = v;
  ws.fA3[i] = (R(2) - R(3) * rho * rho) * nu * nu;
}

template <class R> __device__ __forceinline__ const R* mm_k(const DevMarket& m);
template <> __device__ __forceinline__ const double* mm_k<double>(const DevMarket& m) { return m.mm_k64; }
template <> __device__ __forceinline__ const float* mm_k<float>(const DevMarket& m) { return m.mm_k32; }
template <class R> __device__ __forceinline__ R exp_mm(R x);
template <> __device__ __forceinline__ double exp_mm<double>(double x) { return exp(x); }
template <> __device__ __forceinline__ float exp_mm<float>(float x) { return exp_approx(x); }

// S2 for the Mercurio & Morini model (Eq. haganForMercurio): forward i's SABR alpha is
// alpha_i exp(-sigma S_i) with S_i = sum_{j <= i} k_j phi_j alpha_j, where the market constant
// k_j = tau_j F_j^b T_j / (1 + tau_j F_j) carries the drift integral's interval lengths (the
// piecewise-constant M_i integrates to -sigma sum_{j <= i} c_j T_j).  Lane i holds forward i
// (n_fwd <= 15): one warp scan.  Slots [phi_0..phi_{M-1}, sigma, alpha_0..alpha_{M-1}].  The
// forward's rho phi_i sits in fA3 (the pricer forms (2 - 3 rho^2) nu^2 itself for this model).
template <class R>
__device__ __forceinline__ void mm_forward_params(const DevMarket& m, const WarpScratch<R>& ws, int lane) {
  const int M = m.n_fwd;
  const bool in = lane < M;
  const R phi = in ? ws.xs[lane] : R(0), al = in ? ws.xs[M + 1 + lane] : R(0);
  const R kj = in ? mm_k<R>(m)[lane] : R(0);
  R c = kj * phi * al;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const R o = __shfl_up_sync(0xffffffffu, c, off);
    if (lane >= off) c += o;
  }
  const R sig = ws.xs[M];
  if (in) {
    const R aS = al * exp_mm<R>(-sig * c);
    Q4<R> v;
    v.a = aS;
    v.b = fdiv<R>(sig, aS);
    v.c = aS * aS;
    v.d = phi * sig * aS;
    ws.F4[lane] = v;
    ws.fA3[lane] = phi;
  }
  __syncwarp();
}

// Inclusive prefix scans over the panel integrals, in place (Gp -> SG, Ap -> SA, Hp -> SH, and
// SGH in Ep's slot), then alpha_i and nu_i of every caplet forward.
template <class R>
__device__ __forceinline__ void prefix_and_forwards(const DevMarket& m, const WarpScratch<R>& ws, int lane, R rho) {
  const int NP = m.NP;
  R cg = 0, ca = 0, chh = 0, cgs = 0;
  for (int c0 = 0; c0 < NP; c0 += 32) {
    const int p = c0 + lane;
    const bool in = p < NP;
    const R g = in ? ws.Gp[p] : R(0), ap = in ? ws.Ap[p] : R(0), hh = in ? ws.Hp[p] : R(0);
    R ig = g, ia = ap, ih = hh;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const R og = __shfl_up_sync(0xffffffffu, ig, off);
      const R oa = __shfl_up_sync(0xffffffffu, ia, off);
      const R oh = __shfl_up_sync(0xffffffffu, ih, off);
      if (lane >= off) { ig += og; ia += oa; ih += oh; }
    }
    ih += chh;
    R igs = g * ih;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const R o2 = __shfl_up_sync(0xffffffffu, igs, off);
      if (lane >= off) igs += o2;
    }
    __syncwarp();
    if (in) {
      ws.Gp[p] = cg + ig;
      ws.Ap[p] = ca + ia;
      ws.Hp[p] = ih;
      ((R*)ws.Ep)[p] = cgs + igs;
    }
    cg += __shfl_sync(0xffffffffu, ig, 31);
    ca += __shfl_sync(0xffffffffu, ia, 31);
    chh = __shfl_sync(0xffffffffu, ih, 31);
    cgs += __shfl_sync(0xffffffffu, igs, 31);
  }
  __syncwarp();
  for (int j = lane; j < m.n_capfwd; j += 32) {
    const int i = m.capfwd_list[j];
    const int n = m.fwd_np[i];
    const R Ti = (R)m.T[i];
    const R G = ws.Gp[n - 1];
    const R X = ws.Ap[n - 1] + ws.Hp[n - 1] * G - ((const R*)ws.Ep)[n - 1];
    const R al = fsqrt<R>(fdiv<R>(G, Ti));
    const R X2 = R(2) * X;
    put_forward<R>(ws, i, al, X2 > R(0) ? fdiv<R>(fsqrt<R>(X2), al * Ti) : R(0), rho);
  }
  __syncwarp();
}

// S2: alpha_i, nu_i of every caplet forward (Rebonato mapping, kappa = 1).
// The inner rule at outer node q of panel p is R(p, q) = sum_r w_qr h(base + o2_qr)^2 with
// h(base + o2) = E (a' e_r + b_r) + d_h, E = e^{-gamma_h base}, a' = alpha_h + beta_h base,
// e_r = e^{-gamma_h o2_qr}, b_r = beta_h o2_qr e_r; expanding the square,
//   R = E^2 (a'^2 S1 + 2 a' S2 + S3) + 2 E d_h (a' S4 + S5) + d_h^2 S6
// with the per-node sums S1 = sum w e^2, S2 = sum w e b, S3 = sum w b^2, S4 = sum w e, S5 = sum w b,
// S6 = sum w, formed once per evaluation.  The per-forward sums over panels come from warp prefix
// scans: G_i = SG(n_i), X_i = SA(n_i) + SH(n_i) SG(n_i) - SGH(n_i), SGH(n) = sum_{p<n} Gp[p] SH(p+1).
template <class R>
__device__ void rebonato_forward_params(const DevMarket& m, const QuadTab<R>& qt, const WarpScratch<R>& ws, int lane) {
  typedef Num<R> M;
  const R a = ws.xs[0], b = ws.xs[1], c = ws.xs[2], d = ws.xs[3];
  const R ah = ws.xs[4], bh = ws.xs[5], gh = ws.xs[6], dh = ws.xs[7];
  const R rho = ws.xs[8];
  const R D = (R)m.panel;
  const int NP = m.NP, NPc = round_up(NP, 4);
  // inner-rule sums: lane -> node q = lane / 4, inner nodes r = lane % 4 and lane % 4 + 4
  {
    const int q = lane >> 2, r0 = lane & 3;
    R s1 = 0, s2 = 0, s3 = 0, s4 = 0, s5 = 0, s6 = 0;
#pragma unroll
    for (int h2 = 0; h2 < 2; ++h2) {
      const int j = q * kQ + r0 + 4 * h2;
      const R o2 = qt.o2[j], sw = qt.sw2[j];
      const R w = sw * sw;
      const R e = M::exp_(-gh * o2);
      const R bb = bh * o2 * e;
      s1 += w * e * e;
      s2 += w * e * bb;
      s3 += w * bb * bb;
      s4 += w * e;
      s5 += w * bb;
      s6 += w;
    }
#pragma unroll
    for (int off = 1; off < 4; off <<= 1) {
      s1 += __shfl_xor_sync(0xffffffffu, s1, off);
      s2 += __shfl_xor_sync(0xffffffffu, s2, off);
      s3 += __shfl_xor_sync(0xffffffffu, s3, off);
      s4 += __shfl_xor_sync(0xffffffffu, s4, off);
      s5 += __shfl_xor_sync(0xffffffffu, s5, off);
      s6 += __shfl_xor_sync(0xffffffffu, s6, off);
    }
    if (r0 == 0) {
      Q4<R> t;
      t.a = s1; t.b = s2; t.c = s3; t.d = s4;
      ws.T2[2 * q] = t;
      t.a = s5; t.b = s6; t.c = R(0); t.d = R(0);
      ws.T2[2 * q + 1] = t;
    }
  }
  if (lane < kQ) {
    const R o = qt.o[lane];
    const R eg = M::exp_(-c * o), eh = M::exp_(-gh * o);
    Q4<R> t;
    t.a = eg;
    t.b = b * o * eg;
    t.c = eh;
    t.d = bh * o * eh;
    ws.Tq[lane] = t;
  }
  for (int p = lane; p < NP; p += 32) {
    const R base = D * (R)p;
    Q2<R> e;
    e.a = M::exp_(-c * base);
    e.b = M::exp_(-gh * base);
    ws.Ep[p] = e;
  }
  __syncwarp();
  const int q = lane & 7, pg = lane >> 3;
  const R wq = qt.w[q];
  const Q4<R> tq = ws.Tq[q];
  const Q4<R> S14 = ws.T2[2 * q], S56 = ws.T2[2 * q + 1];
  for (int p = pg; p < NPc; p += 4) {
    R G = 0, H = 0, A = 0;
    if (p < NP) {
      const R base = D * (R)p;
      const Q2<R> E = ws.Ep[p];
      const R g = E.a * ((a + b * base) * tq.a + tq.b) + d;
      const R ahp = ah + bh * base;
      const R h = E.b * (ahp * tq.c + tq.d) + dh;
      const R Rin = E.b * E.b * (ahp * (ahp * S14.a + R(2) * S14.b) + S14.c) +
                    R(2) * E.b * dh * (ahp * S14.d + S56.a) + dh * dh * S56.b;
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
  prefix_and_forwards<R>(m, ws, lane, rho);
}

// S2 in FP32 on the packed pair instructions.  Same sums as rebonato_forward_params, laid out for
// pairs of outer nodes (q, q + 1): the per-evaluation tables are pair-major floats
//   Tq: [4 pairs][e_g, b o e_g, e_h, beta_h o e_h][2]      (32 floats)
//   T2: [4 pairs][S1, 2 S2, S3, S4, S5, S6][2]             (48 floats)
// so that one lane owns one panel and walks the 8 nodes as 4 pairs with no shuffles; the
// exponentials are e^x = 2^(x log2 e) with the rounding of x log2 e carried as a first-order
// correction.
__device__ __forceinline__ float exp_fast(float x) {
  const float L = 1.44269504088896341f, Llo = 1.92596299112661746e-8f;   // log2 e = L + Llo
  const float hi = x * L;
  const float lo = fmaf(x, L, -hi) + x * Llo;
  return ex2_approx(hi) * fmaf(lo, 0.693147180559945309f, 1.0f);
}

__device__ void rebonato_forward_params_f32(const DevMarket& m, const QuadTab<float>& qt,
                                            const WarpScratch<float>& ws, int lane) {
  const float a = ws.xs[0], b = ws.xs[1], c = ws.xs[2], d = ws.xs[3];
  const float ah = ws.xs[4], bh = ws.xs[5], gh = ws.xs[6], dh = ws.xs[7];
  const float rho = ws.xs[8];
  const float D = (float)m.panel;
  const int NP = m.NP;
  float* tq = (float*)ws.Tq;
  float* t2 = (float*)ws.T2;
  {
    // inner-rule sums: lane -> outer node q = lane / 4, inner nodes r0 = lane % 4 and r0 + 4
    const int q = lane >> 2, r0 = lane & 3;
    const float2 o2 = make_float2(qt.o2[q * kQ + r0], qt.o2[q * kQ + r0 + 4]);
    const float2 sw = make_float2(qt.sw2[q * kQ + r0], qt.sw2[q * kQ + r0 + 4]);
    const float2 w = mul2(sw, sw);
    const float2 e = make_float2(exp_fast(-gh * o2.x), exp_fast(-gh * o2.y));
    const float2 bb = mul2(mul2(bc2(bh), o2), e);
    const float2 we = mul2(w, e), wb = mul2(w, bb);
    const float2 p1 = mul2(we, e), p2 = mul2(we, bb), p3 = mul2(wb, bb);
    float S[6] = {p1.x + p1.y, p2.x + p2.y, p3.x + p3.y, we.x + we.y, wb.x + wb.y, w.x + w.y};
#pragma unroll
    for (int off = 1; off < 4; off <<= 1)
#pragma unroll
      for (int j = 0; j < 6; ++j) S[j] += __shfl_xor_sync(0xffffffffu, S[j], off);
    if (r0 == 0) {
      float* t = t2 + (q >> 1) * 12 + (q & 1);
      t[0] = S[0];
      t[2] = 2.0f * S[1];
      t[4] = S[2];
      t[6] = S[3];
      t[8] = S[4];
      t[10] = S[5];
    }
  }
  if (lane < kQ) {
    const float o = qt.o[lane];
    const float eg = exp_fast(-c * o), eh = exp_fast(-gh * o);
    float* t = tq + (lane >> 1) * 8 + (lane & 1);
    t[0] = eg;
    t[2] = b * o * eg;
    t[4] = eh;
    t[6] = bh * o * eh;
  }
  __syncwarp();
  const float2* tq2 = (const float2*)tq;
  const float2* t22 = (const float2*)t2;
  const float2* w2 = (const float2*)qt.w;
  for (int p = lane; p < NP; p += 32) {
    const float base = D * (float)p;
    const float Eg = exp_fast(-c * base), Eh = exp_fast(-gh * base);
    const float2 agp = bc2(a + b * base), ahp = bc2(ah + bh * base);
    const float2 E2 = bc2(Eh * Eh), c2e = bc2(2.0f * Eh * dh), dh2 = bc2(dh * dh);
    float2 G = bc2(0.0f), H = bc2(0.0f), A = bc2(0.0f);
#pragma unroll
    for (int qp = 0; qp < 4; ++qp) {
      const float2 wq = w2[qp];
      const float2* T = tq2 + qp * 4;
      const float2* S = t22 + qp * 6;
      const float2 g = fma2(bc2(Eg), fma2(agp, T[0], T[1]), bc2(d));
      const float2 h = fma2(bc2(Eh), fma2(ahp, T[2], T[3]), bc2(dh));
      float2 t1 = fma2(ahp, S[0], S[1]);
      t1 = fma2(ahp, t1, S[2]);
      const float2 t2v = fma2(ahp, S[3], S[4]);
      float2 Rin = mul2(E2, t1);
      Rin = fma2(c2e, t2v, Rin);
      Rin = fma2(dh2, S[5], Rin);
      const float2 gw = mul2(mul2(wq, g), g);
      G = add2(G, gw);
      H = fma2(mul2(wq, h), h, H);
      A = fma2(gw, Rin, A);
    }
    ws.Gp[p] = G.x + G.y;
    ws.Hp[p] = H.x + H.y;
    ws.Ap[p] = A.x + A.y;
  }
  __syncwarp();
  prefix_and_forwards<float>(m, ws, lane, rho);
}

// S2 dispatch for the objective: the packed FP32 form, or the plain form in FP64.  (The adjoint
// keeps the plain form, whose node tables it reads back.)
template <class R>
__device__ __forceinline__ void forward_params(const DevMarket& m, const QuadTab<R>& qt, const WarpScratch<R>& ws,
                                               int lane) {
  if constexpr (std::is_same<R, float>::value) rebonato_forward_params_f32(m, qt, ws, lane);
  else rebonato_forward_params<R>(m, qt, ws, lane);
}

// z / x(z) with per-chain constants of rho: omr = 1 - r, inv_omr = 1 / (1 - r), omr2 = 1 - r^2
// for r = rho (z >= 0) and r = -rho (z < 0) (x(z; rho) = -x(-z; -rho)).  With zz = |z| and
// s = sqrt(1 - 2 r zz + zz^2):  x = log1p(zz Q / ((s + 1)(1 - r))),  Q = s + 1 - 2r + zz,
// where Q is formed as (s - r) + (1 - r) + zz with s - r = (1 - r^2 + zz (zz - 2r)) / (s + r)
// when r > 0 (no cancellation of s against r as r -> 1), and directly when r <= 0 (every term
// non-negative).  Near z = 0 the series 1 - rho z / 2 + (2 - 3 rho^2) z^2 / 12.
template <class R>
struct RhoConsts {
  R rho, omr_p, omr_m, iomr_p, iomr_m, omr2;
  __device__ __forceinline__ void init(R r) {
    rho = r;
    omr_p = R(1) - r;
    omr_m = R(1) + r;
    iomr_p = R(1) / omr_p;
    iomr_m = R(1) / omr_m;
    omr2 = omr_p * omr_m;
  }
};

template <class R>
__device__ __forceinline__ R z_over_x_fast(R z, const RhoConsts<R>& rc) {
  typedef Num<R> M;
  const R zz = M::abs_(z);
  const bool neg = z < R(0);
  const R r = neg ? -rc.rho : rc.rho;
  const R omr = neg ? rc.omr_m : rc.omr_p;
  const R iomr = neg ? rc.iomr_m : rc.iomr_p;
  const R zq = zz * (zz - R(2) * r);
  const R s = fsqrt<R>(R(1) + zq);
  const R smr = fdiv<R>(rc.omr2 + zq, s + r);
  const R Q = (r > R(0)) ? (smr + omr + zz) : (zz - R(2) * r + s + R(1));
  const R x = log1p_zx<R>(fdiv<R>(zz * Q, s + R(1)) * iomr);
  const R series = R(1) - R(0.5) * rc.rho * z + (R(2) - R(3) * rc.rho * rc.rho) * z * z * R(1.0 / 12.0);
  return (zz < M::zx_series) ? series : fdiv<R>(zz, x);
}

// S4 + S7 (caplets): lane-strided pricing; returns this lane's partial sum of squared
// residuals in the pricing precision and clears `ok` on an infeasible vol.  With vols != null
// the model vols are written instead (NaN where infeasible); with res != null the weighted
// residuals sqrt(w_k) (P_k - P_k^mkt) are written as well (NaN where infeasible).
// PFR: rho per forward (Mercurio & Morini: phi_i in fA3) instead of the chain's rho.
template <class R, int FORMULA, bool PFR = false>
__device__ __forceinline__ R price_caplets(const InstrView<R>& B, int n, const WarpScratch<R>& ws, const RhoConsts<R>& rc,
                                           R omb, int lane, bool& ok, double* vols, double* res = nullptr) {
  typedef Num<R> M;
  R acc = 0;
  for (int k = lane; k < n; k += 32) {
    const int i = B.idx[k];
    const Q4<R> fw = ws.F4[i];
    const Q4<R> g0 = B.g0[k];   // l, fk, inv_den, c1
    const Q4<R> g1 = B.g1[k];   // c2, c3, sqrt(T), D F
    R sig;
    if (FORMULA == 0) {
      const R z = fw.b * g0.b;
      R zx, a3;
      if (PFR) {
        RhoConsts<R> ri;
        const R rho = ws.fA3[i], nu = fw.b * fw.a;
        ri.init(rho);
        zx = z_over_x_fast<R>(z, ri);
        a3 = (R(2) - R(3) * rho * rho) * nu * nu;
      } else {
        zx = z_over_x_fast<R>(z, rc);
        a3 = ws.fA3[i];
      }
      const R corr = R(1) + g0.d * fw.c + g1.a * fw.d + g1.b * a3;
      sig = fw.a * g0.c * zx * corr;
    } else {
      sig = sabr_paper<R>(fw.a, PFR ? ws.fA3[i] : rc.rho, fw.b * fw.a, g0.a, g0.b, omb);
    }
    const bool good = (sig > R(0)) && M::finite_(sig);
    if (vols) { vols[k] = good ? (double)sig : __longlong_as_double(0x7ff8000000000000LL); continue; }
    ok = ok && good;
    const Q4<R> g2 = B.g2[k];   // K/F, sgn, P_mkt, sqrt(w)
    const R v = sig * g1.c;
    const R d1 = fdiv<R>(g0.a, v) + R(0.5) * v;
    const R sg = g2.b;
    const R p = sg * g1.d * (ncdf<R>(sg * d1) - g2.a * ncdf<R>(sg * (d1 - v)));
    const R r = g2.d * (p - g2.c);
    if (res) res[k] = good ? (double)r : __longlong_as_double(0x7ff8000000000000LL);
    acc += r * r;
  }
  return acc;
}

// z_over_x_fast on a pair (FP32).  Per element: rho, omr2 = 1 - rho^2 and the series
// coefficients c1 = -rho / 2, c2 = (2 - 3 rho^2) / 12.  The sign of z is the sign of fk
// (nu / alpha > 0), so r = +-rho comes from the sign bit of the instrument constant, and
// 1 / ((s + 1)(1 - r)) is one reciprocal.
__device__ __forceinline__ float2 z_over_x2(float2 z, float fkx, float fky, float rhox, float rhoy, float2 omr2,
                                            float2 c1, float2 c2) {
  const float2 zz = abs2(z);
  const float2 r = make_float2(__uint_as_float(__float_as_uint(rhox) ^ (__float_as_uint(fkx) & 0x80000000u)),
                               __uint_as_float(__float_as_uint(rhoy) ^ (__float_as_uint(fky) & 0x80000000u)));
  const float2 zm2r = fma2(r, bc2(-2.0f), zz);
  const float2 zq = mul2(zz, zm2r);
  const float2 s2 = add2(bc2(1.0f), zq);
  const float2 s = mul2(s2, rsqrt2(s2));
  const float2 smr = mul2(add2(omr2, zq), rcp2(add2(s, r)));
  const float2 sp1 = add2(s, bc2(1.0f));
  const float2 omr = sub2(bc2(1.0f), r);
  const float2 qa = add2(add2(smr, omr), zz);
  const float2 qb = add2(zm2r, sp1);
  const float2 Q = sel2(r.x > 0.0f, r.y > 0.0f, qa, qb);
  const float2 x = log1p_pos2(mul2(mul2(zz, Q), rcp2(mul2(sp1, omr))));
  const float2 ser = fma2(fma2(c2, z, c1), z, bc2(1.0f));
  const float2 zx = mul2(zz, rcp2(x));
  return sel2(zz.x < Num<float>::zx_series, zz.y < Num<float>::zx_series, ser, zx);
}

// The weighted residuals r = sqrt(w) (P - P_mkt) of a pair of instruments (caplets or swaptions
// alike) on the packed instructions: per element its SABR factors F = {alpha, nu/alpha, alpha^2,
// rho nu alpha}, A3 = (2 - 3 rho^2) nu^2, rho, and its three constant vectors g0 = {l, fk, inv_den,
// c1}, g1 = {c2, c3, sqrt T, D F}, g2 = {K/F, sgn, P_mkt, sqrt w}.  Clears oka / okb on an
// infeasible vol of the first / second element.
__device__ __forceinline__ float2 price_pair_x2(const Q4<float>& fa, const Q4<float>& fb, float a3a, float a3b,
                                                float rhoa, float rhob, const Q4<float>& g0a, const Q4<float>& g0b,
                                                const Q4<float>& g1a, const Q4<float>& g1b, const Q4<float>& g2a,
                                                const Q4<float>& g2b, bool& oka, bool& okb) {
  const float2 rho = make_float2(rhoa, rhob);
  const float2 omr2 = mul2(sub2(bc2(1.0f), rho), add2(bc2(1.0f), rho));
  const float2 c1 = mul2(bc2(-0.5f), rho);
  const float2 c2 = mul2(fma2(mul2(bc2(-3.0f), rho), rho, bc2(2.0f)), bc2(1.0f / 12.0f));
  const float2 fk = make_float2(g0a.b, g0b.b);
  const float2 z = mul2(make_float2(fa.b, fb.b), fk);
  const float2 zx = z_over_x2(z, fk.x, fk.y, rhoa, rhob, omr2, c1, c2);
  float2 corr = fma2(make_float2(g0a.d, g0b.d), make_float2(fa.c, fb.c), bc2(1.0f));
  corr = fma2(make_float2(g1a.a, g1b.a), make_float2(fa.d, fb.d), corr);
  corr = fma2(make_float2(g1a.b, g1b.b), make_float2(a3a, a3b), corr);
  const float2 sig = mul2(mul2(mul2(make_float2(fa.a, fb.a), make_float2(g0a.c, g0b.c)), zx), corr);
  oka = (sig.x > 0.0f) && (sig.x < INFINITY);
  okb = (sig.y > 0.0f) && (sig.y < INFINITY);
  const float2 v = mul2(sig, make_float2(g1a.c, g1b.c));
  const float2 d1 = fma2(make_float2(g0a.a, g0b.a), rcp2(v), mul2(bc2(0.5f), v));
  const float2 sg = make_float2(g2a.b, g2b.b);
  const float2 n1 = ncdf2(mul2(sg, d1));
  const float2 n2 = ncdf2(mul2(sg, sub2(d1, v)));
  const float2 nkf = mul2(make_float2(g2a.a, g2b.a), bc2(-1.0f));
  const float2 p = mul2(mul2(sg, make_float2(g1a.d, g1b.d)), fma2(nkf, n2, n1));
  return mul2(make_float2(g2a.d, g2b.d), sub2(p, make_float2(g2a.c, g2b.c)));
}

// price_caplets for FP32 and the Hagan (2002) form on the packed instructions: lane l takes the
// caplet pair P = 32 i + l of the pair-major block (caplets 64 i + l and 64 i + l + 32), so every
// 16-byte load gives two ready operand pairs.  A missing second caplet carries sqrt(w) = 0.
// RES: also write each caplet's weighted residual sqrt(w) (P - P_mkt) to res (NaN where the vol
// is infeasible), from the same arithmetic the search runs.
template <bool RES = false>
__device__ __forceinline__ float price_caplets_x2(const void* blk, int npairs, int n, const WarpScratch<float>& ws,
                                                  const RhoConsts<float>& rc, int lane, bool& ok,
                                                  double* res = nullptr) {
  const PairView B = pair_view(blk, npairs);
  const float c1 = -0.5f * rc.rho, c2 = (2.0f - 3.0f * rc.rho * rc.rho) * (1.0f / 12.0f);
  float2 acc = bc2(0.0f);
  for (int it = 0; 64 * it + lane < n; ++it) {
    const int P = 32 * it + lane;
    const int2 ix = B.idx[P];
    const Q4<float> fa = ws.F4[ix.x], fb = ws.F4[ix.y];
    const float4 v0 = B.v[P], v1 = B.v[npairs + P], v2 = B.v[2 * npairs + P];
    const float2 l = make_float2(v0.x, v0.y), fk = make_float2(v0.z, v0.w);
    const float2 z = mul2(make_float2(fa.b, fb.b), fk);
    const float2 zx = z_over_x2(z, fk.x, fk.y, rc.rho, rc.rho, bc2(rc.omr2), bc2(c1), bc2(c2));
    // inv_den (1 + c1 alpha^2 + c2 rho nu alpha + c3 A3), inv_den folded into the constants
    float2 corr = fma2(make_float2(v1.z, v1.w), make_float2(fa.c, fb.c), make_float2(v1.x, v1.y));
    corr = fma2(make_float2(v2.x, v2.y), make_float2(fa.d, fb.d), corr);
    corr = fma2(make_float2(v2.z, v2.w), make_float2(ws.fA3[ix.x], ws.fA3[ix.y]), corr);
    const float2 sig = mul2(mul2(make_float2(fa.a, fb.a), zx), corr);
    ok = ok && (sig.x > 0.0f) && (sig.x < INFINITY) && (sig.y > 0.0f) && (sig.y < INFINITY);
    const float4 v3 = B.v[3 * npairs + P], v4 = B.v[4 * npairs + P];
    const float2 v5 = *(const float2*)(B.v + 5 * npairs + P);
    // xf = -|l| / v + v / 2 and xs = xf - v <= 0 (v = sigma sqrtT, v / 2 = (sqrtT / 2) sigma)
    const float2 v = mul2(sig, make_float2(v3.x, v3.y));
    const float2 hv = mul2(make_float2(v4.z, v4.w), sig);
    const float2 xf = fma2(l, rcp2(v), hv);
    const float2 xs = fma2(hv, bc2(-2.0f), xf);
    const float2 nf = ncdf2(xf);
    const float2 ns = ncdf2_nonpos(xs);
    // Phi(xf) + B Phi(xs) in one rounding (the two nearly cancel far out of the money), and the
    // weighted residual C (Phi(xf) + B Phi(xs)) - sqrt(w) P_mkt in one more
    const float2 nn = fma2(make_float2(v4.x, v4.y), ns, nf);
    const float2 r = fma2(make_float2(v3.z, v3.w), nn, v5);
    if constexpr (RES) {
      const int a = 64 * it + lane, b = a + 32;
      const double qnan = __longlong_as_double(0x7ff8000000000000LL);
      const bool ga = (sig.x > 0.0f) && (sig.x < INFINITY), gb = (sig.y > 0.0f) && (sig.y < INFINITY);
      res[a] = ga ? (double)r.x : qnan;
      if (b < n) res[b] = gb ? (double)r.y : qnan;
    }
    acc = fma2(r, r, acc);
  }
  return acc.x + acc.y;
}

// ------------------------------------------------------------------ objective values
// FP64 path: a double.  FP32 path: a float-float pair (hi + lo, |lo| <= ulp(hi)/2).
struct FF { float hi, lo; };

__device__ __forceinline__ FF ff_add(FF a, FF b) {
  // Knuth's two-sum on the high parts, low parts added with the rounding error
  const float s = a.hi + b.hi;
  const float bp = s - a.hi;
  const float e = (a.hi - (s - bp)) + (b.hi - bp);
  const float lo = e + a.lo + b.lo;
  FF r;
  r.hi = s + lo;
  r.lo = lo - (r.hi - s);
  return r;
}

__device__ __forceinline__ FF ff_of(float a) {
  FF r;
  r.hi = a;
  r.lo = 0.0f;
  return r;
}

// float-float plus float (two-sum, then the low parts added and renormalised)
__device__ __forceinline__ FF ff_add_f(FF a, float b) {
  const float s = a.hi + b;
  const float bp = s - a.hi;
  const float e = (a.hi - (s - bp)) + (b - bp);
  const float lo = e + a.lo;
  FF r;
  r.hi = s + lo;
  r.lo = lo - (r.hi - s);
  return r;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  return v;
}

__device__ __forceinline__ double warp_sum_lanes(double p) { return warp_sum(p); }

// The per-lane FP32 partials of one warp summed by an FP32 butterfly (the same value in every lane:
// each level adds the same two operands in both lanes).  Relative error <= 5 u, below the
// per-lane accumulation's; no FP64 instruction.
__device__ __forceinline__ FF warp_sum_lanes_f32(float p) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) p += __shfl_xor_sync(0xffffffffu, p, off);
  FF r;
  r.hi = p;
  r.lo = 0.0f;
  return r;
}


template <class R> struct ObjOf { typedef double T; };
template <> struct ObjOf<float> { typedef FF T; };

__device__ __forceinline__ double obj_add(double a, double b) { return a + b; }
__device__ __forceinline__ FF obj_add(FF a, FF b) { return ff_add(a, b); }
__device__ __forceinline__ double obj_inf(double) { return __longlong_as_double(0x7ff0000000000000LL); }
__device__ __forceinline__ FF obj_inf(FF) { FF r; r.hi = __int_as_float(0x7f800000); r.lo = 0.f; return r; }
__device__ __forceinline__ bool obj_finite(double v) { return isfinite(v); }
__device__ __forceinline__ bool obj_finite(FF v) { return isfinite(v.hi); }
__device__ __forceinline__ double obj_to_double(double v) { return v; }
__device__ __forceinline__ double obj_to_double(FF v) { return (double)v.hi + (double)v.lo; }
__device__ __forceinline__ bool obj_less(double a, double b) { return a < b; }
__device__ __forceinline__ bool obj_less(FF a, FF b) { return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }
__device__ __forceinline__ void obj_from_double(double v, double& o) { o = v; }
__device__ __forceinline__ void obj_from_double(double v, FF& o) {
  o.hi = (float)v;
  o.lo = isfinite(v) ? (float)(v - (double)o.hi) : 0.f;
}

// Objective of the point held in ws.xs (all 32 lanes call; all return the same value).
// MODEL 0: SABR smile [alpha, rho, nu];  MODEL 1: Rebonato caplets;  MODEL 2: Mercurio & Morini
// caplets (scalar pricer with a rho per forward).
// vols != null: the model vols are written instead.  res != null: the weighted residuals are
// written as well, by the pricer the search uses (the packed one in FP32 with the Hagan form).
template <class R, int MODEL, int FORMULA>
__device__ typename ObjOf<R>::T warp_objective(const DevMarket& m, const InstrView<R>& capB, const QuadTab<R>& qt,
                                               const WarpScratch<R>& ws, int lane, double* vols,
                                               double* res = nullptr) {
  typedef typename ObjOf<R>::T O;
  RhoConsts<R> rc;
  if (MODEL == 0) {
    const R al = ws.xs[0], rho = ws.xs[1], nu = ws.xs[2];
    for (int j = lane; j < m.n_capfwd; j += 32) put_forward<R>(ws, m.capfwd_list[j], al, nu, rho);
    __syncwarp();
    rc.init(rho);
  } else if (MODEL == 2) {
    mm_forward_params<R>(m, ws, lane);
    rc.init(R(0));
  } else {
    forward_params<R>(m, qt, ws, lane);
    rc.init(ws.xs[8]);
  }
  bool ok = true;
  R part;
  if constexpr (MODEL == 2) {
    part = price_caplets<R, FORMULA, true>(capB, m.n_cap, ws, rc, (R)(1.0 - m.beta), lane, ok, vols, res);
  } else if constexpr (std::is_same<R, float>::value && FORMULA == 0) {
    // (with no vols requested the caller staged the pair-major block; its base is capB.g0)
    if (vols != nullptr)
      part = price_caplets<R, FORMULA>(capB, m.n_cap, ws, rc, (R)(1.0 - m.beta), lane, ok, vols);
    else if (res != nullptr)
      part = price_caplets_x2<true>(capB.g0, m.n_cap_pairs, m.n_cap, ws, rc, lane, ok, res);
    else
      part = price_caplets_x2<false>(capB.g0, m.n_cap_pairs, m.n_cap, ws, rc, lane, ok);
  } else {
    part = price_caplets<R, FORMULA>(capB, m.n_cap, ws, rc, (R)(1.0 - m.beta), lane, ok, vols, res);
  }
  __syncwarp();
  if (vols) return obj_inf(O());
  O f;
  if constexpr (std::is_same<R, float>::value) f = warp_sum_lanes_f32(part);
  else f = warp_sum_lanes(part);
  const bool bad = __any_sync(0xffffffffu, !ok);
  if (bad || !obj_finite(f)) return obj_inf(O());
  return f;
}

}  // namespace sabr
