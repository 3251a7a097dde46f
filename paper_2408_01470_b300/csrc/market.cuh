// Device layout of a loaded market.
//
// One device arena per sabr_lmm_load_market call holds, per market: the raw description (tenor
// grid, discounts, strikes, quotes, box), integer bookkeeping built on the host (distinct caplet
// forwards, distinct underlying swaps), and the market-only constants computed by
// setup_market_kernel in FP64 (forwards, discounts, annuities, swap rates, frozen weights,
// market prices, vega weights, log-moneyness, SABR constants).  The pricing constants of the
// caplets and of the swaptions are stored twice, as FP64 and FP32 "instrument blocks": a block
// is a contiguous, 16-byte aligned run of structure-of-arrays, so a CTA stages it into shared
// memory with one bulk copy.
#pragma once
#include <cstdint>

namespace sabr {

constexpr int kQ = 8;               // Gauss-Legendre nodes per panel
constexpr int kMaxParam = 32;       // parameter slots (Mercurio & Morini: 2 n_fwd + 1 <= 31)
constexpr int kMaxGradParam = 12;   // slots of the adjoint, Levenberg-Marquardt and no-alloc paths
constexpr int kBlkArrays = 12;      // R values per instrument in a block (+ one int)
constexpr int kSeg = 4;             // pairs per segment of a group's pair triangle (quadratic forms)

// Quadrature table per precision, offsets relative to the start of a panel of width D:
//   o[q] = (D/2)(1 + xi_q), w[q] = (D/2) w_q, sw[q] = sqrt(w[q])   (outer rule on the panel)
//   o2[q*8+r] = o[q] + h_q (1 + xi_r), sw2[q*8+r] = sqrt(h_q w_r), h_q = (D - o[q]) / 2
//                                                         (inner rule on [u_q, panel top])
template <class R> struct QuadTab { R o[kQ]; R w[kQ]; R sw[kQ]; R o2[kQ * kQ]; R sw2[kQ * kQ]; };

template <class R> struct alignas(4 * sizeof(R)) Q4 { R a, b, c, d; };

// An instrument block of n (padded) instruments: three structure-of-arrays groups of 4-vectors
// (one vector load each per instrument) and the index array.
//   g0 = {l = log(F/K), fk, inv_den, c1},  g1 = {c2, c3, sqrt(T), D F},  g2 = {K/F, sgn, P_mkt, sqrt(w)}
// fk is (FK)^{(1-b)/2} l for the Hagan formula and F^{1-b} for Eq. (sigmaHagan).
template <class R> struct InstrView {
  const Q4<R>* g0;
  const Q4<R>* g1;
  const Q4<R>* g2;
  const int* idx;
};

template <class R> __host__ __device__ inline uint32_t instr_block_bytes(int npad) {
  const uint32_t raw = (uint32_t)npad * (uint32_t)(3 * sizeof(Q4<R>) + sizeof(int));
  return (raw + 63u) & ~63u;
}

template <class R> __host__ __device__ inline InstrView<R> instr_view(const void* base, int npad) {
  const Q4<R>* p = (const Q4<R>*)base;
  InstrView<R> v;
  v.g0 = p;
  v.g1 = p + npad;
  v.g2 = p + 2 * npad;
  v.idx = (const int*)(p + 3 * npad);
  return v;
}

// The FP32 caplet block again, pair-major for the packed pricer: caplets a = 64 i + l and
// b = a + 32 (l = 0..31) form pair P = 32 i + l, and each 16-byte vector holds two fields of both,
// with the constants that the pricer multiplies together folded in advance:
//   v0 = {-|l|_a, -|l|_b, fk_a, fk_b}            v1 = {e_a, e_b, e c1_a, e c1_b}
//   v2 = {e c2_a, e c2_b, e c3_a, e c3_b}        v3 = {sqrtT_a, sqrtT_b, C_a, C_b}
//   v4 = {B_a, B_b, sqrtT_a / 2, sqrtT_b / 2}    v5 = {-sqrtw P_mkt_a, -sqrtw P_mkt_b, 0, 0}
// with e = inv_den (so that sigma = alpha (z / x) (e + e c1 alpha^2 + ...)).  An out-of-the-money
// option has sgn l = -|l|, so of its two Black arguments sgn d1, sgn d2 the one on the far side,
// xs = -|l| / v - v / 2, is never positive and the other is xf = -|l| / v + v / 2 (xf = sgn d1 for
// a call, sgn d2 for a put).  The weighted residual is C (Phi(xf) + B Phi(xs)) - sqrt(w) P_mkt with
// C = DF sqrt(w), B = -KF for a call and C = KF DF sqrt(w), B = -1 / KF for a put.  Then the
// forward indices {idx_a, idx_b}.  A missing b (b >= n) repeats a with sqrt(w) = 0.
__host__ __device__ inline int cap_pairs(int n) { return 32 * ((n + 63) / 64); }
__host__ __device__ inline uint32_t pair_block_bytes(int npairs) {
  const uint32_t raw = (uint32_t)npairs * (uint32_t)(6 * 16 + 8);
  return (raw + 63u) & ~63u;
}
struct PairView {
  const float4* v;   // [6 x npairs]
  const int2* idx;   // [npairs]
  int np;
};
__host__ __device__ inline PairView pair_view(const void* base, int npairs) {
  PairView w;
  w.v = (const float4*)base;
  w.idx = (const int2*)(w.v + 6 * npairs);
  w.np = npairs;
  return w;
}

struct DevMarket {
  int model, formula, n_param, n_fwd;
  int n_cap, n_swp, n_swap;        // caplets, swaptions, distinct underlying swaps
  int n_cap_pad, n_swp_pad;        // multiples of 4
  int n_capfwd;                    // distinct caplet forwards
  int NP;                          // panels the caplet mapping needs (max over caplet forwards)
  int max_win;                     // longest swap window
  // swaption geometry (time-homogeneous tables over absolute panels)
  int n_grp;                       // expiry groups: distinct first forwards of the swaps
  int NA;                          // absolute panels the swap integrals touch (max n_E + delta)
  int ND;                          // diagonals of the pair tables (max delta spread + 1)
  int max_gwin;                    // longest group window
  const int* grp_a;                // [n_grp] first forward of the group's swaps
  const int* grp_nE;               // [n_grp] panels to the group's expiry
  const int* grp_L;                // [n_grp] forwards spanned by the group's longest swap
  const int* grp_delta;            // [n_grp x max_gwin] (T_i - T_a) / panel for the group's forwards
  const int* grp_swap0;            // [n_grp + 1] swaps sorted by group: first swap of each group
  const int* swap_grp;             // [n_swap]
  const int* swap_L;               // [n_swap] forwards in the swap
  // quadratic forms by expiry group: with the frozen weights W_i = u_i / (A S^b) of a swap (u_i =
  // tau_i P(0, T_{i+1}) F_i^b, A the annuity, S the swap rate), every swap of a group is a leading
  // block of the group's window, so V_k(swap) = scale(swap) Q_k(g, L) with Q_k(g, L) = the sum of
  // (2 - [i = j]) u_i u_j B_k[i, j] over i <= j < L: one pass over the group's pair triangle serves
  // all its swaps.  The triangle is cut into segments of at most kSeg pairs of one column j.
  int n_seg;                       // segments over every group's triangle
  const int* seg;                  // [n_seg] g | j << 8 | i0 << 16 | (pairs) << 24, column by column
  int n_col;                       // columns over every group (sum of the group windows)
  const int* col_seg0;             // [n_col + 1] first segment of each column
  // The forward sweep's segments: the same count per column, but segment s of a column with S
  // segments takes the pairs i = s, s + S, s + 2S, s + 3S (i <= j), so that the lanes of a warp,
  // which hold consecutive segments of a column, read consecutive diagonals at consecutive panel
  // offsets (prefix-table addresses on distinct banks).  One 16-byte descriptor per segment and its
  // four weights (2 - [i = j]) u_i (0 on an empty slot, whose offsets repeat pair (j, j)).
  // The weights carry u_j as well, (2 - [i = j]) u_i u_j, so a segment's sums are already terms of
  // Q_k(g, L), and a swap's forms are the sums over the segments of its group's first L columns, a
  // contiguous range.
  const int4* seg_dsc;             // [n_seg] x: lo_r << 8r, y: e_r << 8r (r = 0..3), z: the window nE,
                                   //   w: g * max_gwin + j (the index of u_j)
  const int4* seg_uix;             // [n_seg] per slot r: g * max_gwin + i | (i == j) << 20 | valid << 21
  const double* seg_w64;           // [n_seg x 4] the slot weights (FP64)
  const float* seg_w32;            //   the same in FP32
  const int2* swap_segs;           // [n_swap] the segments [x, y) of the swap's group's first L columns
  const int* col_u;                // [n_col] index g * max_gwin + j of the column's u_j
  const int* grp_col0;             // [n_grp + 1] first column of each group
  const double* grp_u64;           // [n_grp x max_gwin] u_{a + i} (FP64)
  const float* grp_u32;            //   the same in FP32
  const double* swap_scale64;      // [n_swap] 1 / (A S^b)^2
  const float* swap_scale32;       //   the same in FP32
  int qf_own;                      // 1: the segment and column partials have their own region
                                   //   (else they live in the Y region, dead after the Grams)
  double beta, panel;
  // raw description
  const double *T, *P, *cap_K, *cap_vol, *cap_wu, *swp_K, *swp_vol, *swp_wu;
  const int *cap_fwd, *swp_start, *swp_end, *swp_swap;
  const int *swap_a, *swap_b;      // [n_swap]
  const int* capfwd_list;          // [n_capfwd]
  const int* fwd_np;               // [n_fwd] panels to T_k (valid for REBONATO)
  const double *lo, *hi;
  const unsigned char* freem;
  // derived by setup_market_kernel
  double *F, *tau;                 // [n_fwd]
  double *swap_A, *swap_S, *swap_TE;  // [n_swap]
  double* swap_W;                  // [n_swap x max_win] frozen weights W_i = w_i F_i^b / S^b
  int* swap_np;                    // [n_swap] panels to the expiry
  double *cap_pm, *cap_w, *swp_pm, *swp_w;  // market prices and weights (FP64)
  void *cblk64, *cblk32, *sblk64, *sblk32;  // instrument blocks
  void* cpair32;                   // the FP32 caplet block, pair-major (PairView)
  int n_cap_pairs;                 // cap_pairs(n_cap)
  const QuadTab<double>* q64;
  const QuadTab<float>* q32;
  int* err;                        // device error word (nonzero: a bounded wait gave up)
  // Mercurio & Morini markets: per forward k_i = tau_i F_i^b T_i / (1 + tau_i F_i) (null otherwise)
  const double* mm_k64;
  const float* mm_k32;
};

}  // namespace sabr
