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
constexpr int kMaxParam = 12;       // parameter slots
constexpr int kBlkArrays = 12;      // R arrays per instrument in a block (+ one int array)

// Quadrature table per precision, offsets relative to the start of a panel of width D:
//   o[q] = (D/2)(1 + xi_q), w[q] = (D/2) w_q             (outer rule on the panel)
//   o2[q*8+r] = o[q] + h_q (1 + xi_r), w2[q*8+r] = h_q w_r, h_q = (D - o[q]) / 2
//                                                         (inner rule on [u_q, panel top])
template <class R> struct QuadTab { R o[kQ]; R w[kQ]; R o2[kQ * kQ]; R w2[kQ * kQ]; };

// Pointers into an instrument block of n (padded) instruments.
template <class R> struct InstrView {
  const R *l, *fk, *inv_den, *c1, *c2, *c3, *sqrtT, *DF, *KF, *sgn, *pm, *sw;
  const int* idx;
};

template <class R> __host__ __device__ inline uint32_t instr_block_bytes(int npad) {
  return (uint32_t)npad * (uint32_t)(kBlkArrays * sizeof(R) + sizeof(int));
}

template <class R> __host__ __device__ inline InstrView<R> instr_view(const void* base, int npad) {
  const R* p = (const R*)base;
  InstrView<R> v;
  v.l = p; v.fk = p + npad; v.inv_den = p + 2 * npad; v.c1 = p + 3 * npad; v.c2 = p + 4 * npad;
  v.c3 = p + 5 * npad; v.sqrtT = p + 6 * npad; v.DF = p + 7 * npad; v.KF = p + 8 * npad;
  v.sgn = p + 9 * npad; v.pm = p + 10 * npad; v.sw = p + 11 * npad;
  v.idx = (const int*)(p + 12 * npad);
  return v;
}

struct DevMarket {
  int model, formula, n_param, n_fwd;
  int n_cap, n_swp, n_swap;        // caplets, swaptions, distinct underlying swaps
  int n_cap_pad, n_swp_pad;        // multiples of 4
  int n_capfwd;                    // distinct caplet forwards
  int NP;                          // panels the model mapping needs (max over forwards/expiries)
  int max_win;                     // longest swap window
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
  const QuadTab<double>* q64;
  const QuadTab<float>* q32;
  int* err;                        // device error word (nonzero: a bounded wait gave up)
};

}  // namespace sabr
