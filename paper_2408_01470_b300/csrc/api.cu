// C-ABI of the library (include/sabr_lmm.h): validation, the device arena of a market, kernel
// dispatch by (precision, model, formula), and the annealing plan (optionally replayed as a CUDA
// graph).  Host code only schedules: every number of the hot path is computed in the kernels.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <functional>
#include <map>
#include <mutex>
#include <tuple>
#include <string>
#include <vector>
#include <thread>
#include <condition_variable>
#include <atomic>
#include <chrono>

#include "../../include/sabr_lmm.h"
#include "kernels.cuh"
#include "lm.cuh"

using namespace sabr;

namespace {

thread_local std::string g_err;

sabr_lmm_status fail(sabr_lmm_status st, const std::string& msg) {
  g_err = msg;
  return st;
}

#define CUDA_TRY(expr)                                                                      \
  do {                                                                                      \
    cudaError_t e_ = (expr);                                                                \
    if (e_ != cudaSuccess) return fail(SABR_LMM_ECUDA, std::string(#expr) + ": " + cudaGetErrorString(e_)); \
  } while (0)

// Gauss-Legendre, 8 nodes on [-1, 1] (tabulated values of the Legendre roots and weights).
const double kGLx[8] = {-0.96028985649753623168, -0.79666647741362673959, -0.52553240991632898582,
                        -0.18343464249564980494, 0.18343464249564980494, 0.52553240991632898582,
                        0.79666647741362673959, 0.96028985649753623168};
const double kGLw[8] = {0.10122853629037625915, 0.22238103445337447054, 0.31370664587788728734,
                        0.36268378337836198297, 0.36268378337836198297, 0.31370664587788728734,
                        0.22238103445337447054, 0.10122853629037625915};

// Layout builder for one device arena: 256-byte aligned regions.
struct Arena {
  size_t size = 0;
  size_t take(size_t bytes) {
    size_t off = (size + 255) & ~size_t(255);
    size = off + std::max<size_t>(bytes, 16);
    return off;
  }
};

struct HostMarket {
  int model, formula, n_param, n_fwd, n_cap, n_swp;
  double beta;
  std::vector<double> lo, hi, cap_vol, swp_vol;
  std::vector<uint8_t> freem;
};

}  // namespace

struct sabr_lmm_market {
  void* arena = nullptr;
  std::vector<DevMarket> dm;
  std::vector<HostMarket> hm;
  int device = 0;
};

struct sabr_lmm_anneal_plan {
  const sabr_lmm_market* mk = nullptr;
  sabr_lmm_anneal_opts opts{};
  int W = 4;
  int grid = 0;
  int cta_warps = 8;              // warps per CTA of the kernels of markets with swaptions
  void* state = nullptr;          // device chain state for every market
  std::vector<SAState> st;        // per market
  std::vector<SAParams> sp;
  std::vector<double> x0;         // host copy
  double* x0_dev = nullptr;
  double* vols_dev = nullptr;     // scratch for the RMSE of the best point
  double* rmse_dev = nullptr;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  cudaGraphExec_t gexec = nullptr;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr, ev2 = nullptr;
  void* lm_buf = nullptr;         // polish buffers (top-k points, selection, LM work) per market
  std::vector<size_t> lm_off;
  // batch mode: per temperature level one persistent launch per shared-memory bucket (markets
  // grouped by the CTAs per SM their shared memory allows), each over its markets' chains
  bool batch = false;
  void* batch_buf = nullptr;
  BatchArgs ba{};                 // every market (start and final kernels)
  uint32_t bsmem = 0;             // the largest market's shared memory
  struct Bucket {
    BatchArgs ba;                 // the bucket's markets (order, count, work counters)
    uint32_t smem = 0;
    int per_sm = 1, threads = 256, grid = 148;
    std::vector<int> markets;     // host copy of the bucket's order
  };
  std::vector<Bucket> bk;
};

namespace {

std::string validate(const sabr_lmm_market_desc& d, int idx) {
  char buf[256];
  auto bad = [&](const char* what) {
    snprintf(buf, sizeof buf, "market %d: %s", idx, what);
    return std::string(buf);
  };
  if (d.model != SABR_LMM_MODEL_SMILE && d.model != SABR_LMM_MODEL_REBONATO && d.model != SABR_LMM_MODEL_MERCURIO_MORINI)
    return bad("model must be 0, 1 or 2");
  if (d.formula != SABR_LMM_HAGAN2002 && d.formula != SABR_LMM_PAPER) return bad("formula must be 0 or 1");
  if (!(d.beta >= 0.0 && d.beta <= 1.0)) return bad("beta must be in [0, 1]");
  if (d.n_fwd < 1 || d.n_fwd > 120) return bad("n_fwd must be in [1, 120]");
  if (!d.T || !d.P) return bad("T and P are required");
  for (int k = 0; k <= d.n_fwd; ++k) {
    if (!(d.T[k] > 0.0) || !std::isfinite(d.T[k])) return bad("T must be finite and > 0");
    if (k > 0 && !(d.T[k] > d.T[k - 1])) return bad("T must be strictly increasing");
    if (!(d.P[k] > 0.0) || !std::isfinite(d.P[k])) return bad("P must be finite and > 0");
  }
  if (d.n_cap < 0 || d.n_swp < 0 || d.n_cap + d.n_swp < 1) return bad("need at least one instrument");
  if (d.n_cap > 0 && (!d.cap_fwd || !d.cap_K || !d.cap_vol)) return bad("caplet arrays are required");
  if (d.n_swp > 0 && (!d.swp_start || !d.swp_end || !d.swp_K || !d.swp_vol)) return bad("swaption arrays are required");
  for (int k = 0; k < d.n_cap; ++k) {
    if (d.cap_fwd[k] < 0 || d.cap_fwd[k] >= d.n_fwd) return bad("cap_fwd out of range");
    if (!(d.cap_K[k] > 0.0) || !std::isfinite(d.cap_K[k])) return bad("cap_K must be finite and > 0");
    if (!(d.cap_vol[k] > 0.0) || !std::isfinite(d.cap_vol[k])) return bad("cap_vol must be finite and > 0");
    if (d.cap_w && !(d.cap_w[k] >= 0.0 && std::isfinite(d.cap_w[k]))) return bad("cap_w must be finite and >= 0");
  }
  for (int k = 0; k < d.n_swp; ++k) {
    if (d.swp_start[k] < 0 || d.swp_end[k] <= d.swp_start[k] || d.swp_end[k] > d.n_fwd)
      return bad("swaption window out of range");
    if (d.swp_end[k] - d.swp_start[k] > 64) return bad("swap windows longer than 64 forwards are not supported");
    if (!(d.swp_K[k] > 0.0) || !std::isfinite(d.swp_K[k])) return bad("swp_K must be finite and > 0");
    if (!(d.swp_vol[k] > 0.0) || !std::isfinite(d.swp_vol[k])) return bad("swp_vol must be finite and > 0");
    if (d.swp_w && !(d.swp_w[k] >= 0.0 && std::isfinite(d.swp_w[k]))) return bad("swp_w must be finite and >= 0");
  }
  if (d.model == SABR_LMM_MODEL_SMILE) {
    if (d.n_param != 3) return bad("the smile model has 3 parameters [alpha, rho, nu]");
    if (d.n_swp != 0) return bad("the smile model prices caplets only");
  } else if (d.model == SABR_LMM_MODEL_MERCURIO_MORINI) {
    if (d.n_fwd > 15) return bad("the Mercurio & Morini model takes at most 15 forwards (2 n_fwd + 1 <= 31 slots)");
    if (d.n_param != 2 * d.n_fwd + 1) return bad("the Mercurio & Morini model has 2 n_fwd + 1 slots [phi_i, sigma, alpha_i]");
    if (d.n_swp != 0) return bad("the Mercurio & Morini model prices caplets only");
  } else {
    if (d.n_param != 12) return bad("the Rebonato model has 12 parameter slots");
    if (!(d.panel > 0.0)) return bad("panel must be > 0");
    for (int k = 0; k <= d.n_fwd; ++k) {
      double r = d.T[k] / d.panel;
      if (std::fabs(r - std::round(r)) > 1e-9 * std::max(1.0, r)) return bad("every T[k] must be a multiple of panel");
    }
    if (std::round(d.T[d.n_fwd] / d.panel) > 240) return bad("more than 240 panels");
  }
  if (!d.lo || !d.hi || !d.free_mask) return bad("lo, hi and free_mask are required");
  for (int k = 0; k < d.n_param; ++k)
    if (!(d.lo[k] <= d.hi[k]) || !std::isfinite(d.lo[k]) || !std::isfinite(d.hi[k])) return bad("box must satisfy lo <= hi");
  return std::string();
}

int n_panels(double t, double panel) { return (int)std::lround(t / panel); }

bool valid_prec(int p) { return p == SABR_LMM_FP64 || p == SABR_LMM_FP32 || p == SABR_LMM_FP32_BF16X3; }

}  // namespace

// ====================================================================== load / free
extern "C" sabr_lmm_status sabr_lmm_load_market(const sabr_lmm_market_desc* descs, int32_t n_markets, void* stream,
                                                sabr_lmm_market** out) {
  if (!descs || !out || n_markets < 1) return fail(SABR_LMM_EINVAL, "descs, out and n_markets >= 1 are required");
  *out = nullptr;
  for (int j = 0; j < n_markets; ++j) {
    if (descs[j].quad_nodes != 8 && descs[j].model == SABR_LMM_MODEL_REBONATO)
      return fail(SABR_LMM_ENOTSUP, "quad_nodes must be 8");
    std::string e = validate(descs[j], j);
    if (!e.empty()) return fail(SABR_LMM_EINVAL, e);
  }
  cudaStream_t s = (cudaStream_t)stream;
  Arena A;
  struct Off {
    size_t T, P, cap_K, cap_vol, cap_wu, swp_K, swp_vol, swp_wu, cap_fwd, swp_start, swp_end, swp_swap, swap_a, swap_b,
        capfwd_list, fwd_np, lo, hi, freem, F, tau, swap_A, swap_S, swap_TE, swap_W, swap_np, cap_pm, cap_w, swp_pm,
        swp_w, cblk64, cblk32, cpair32, sblk64, sblk32, q64, q32, err, grp_a, grp_nE, grp_L, grp_delta, grp_swap0,
        swap_grp, swap_L, seg, col_seg0, col_u, grp_col0, grp_u64, grp_u32, swap_scale64, swap_scale32, seg_dsc,
        seg_uix, seg_w64, seg_w32, swap_segs, mm_k64, mm_k32;
  };
  std::vector<Off> off(n_markets);
  std::vector<DevMarket> dm(n_markets);
  std::vector<HostMarket> hm(n_markets);
  // host-side integer bookkeeping
  std::vector<std::vector<int>> capfwd(n_markets), fwdnp(n_markets), swp_swap(n_markets), swap_a(n_markets),
      swap_b(n_markets), swap_np(n_markets), grp_a(n_markets), grp_nE(n_markets), grp_L(n_markets),
      grp_delta(n_markets), grp_swap0(n_markets), swap_grp(n_markets), swap_L(n_markets), seg(n_markets),
      col_seg0(n_markets), col_u(n_markets), grp_col0(n_markets), sdsc(n_markets), suix(n_markets), sseg(n_markets);
  for (int j = 0; j < n_markets; ++j) {
    const sabr_lmm_market_desc& d = descs[j];
    DevMarket& m = dm[j];
    std::memset(&m, 0, sizeof m);
    m.model = d.model; m.formula = d.formula; m.n_param = d.n_param; m.n_fwd = d.n_fwd;
    m.n_cap = d.n_cap; m.n_swp = d.n_swp; m.beta = d.beta;
    m.panel = d.model == SABR_LMM_MODEL_REBONATO ? d.panel : 0.5;
    m.n_cap_pad = (d.n_cap + 3) / 4 * 4;
    m.n_swp_pad = (d.n_swp + 3) / 4 * 4;
    std::vector<int> seen(d.n_fwd, 0);
    for (int k = 0; k < d.n_cap; ++k)
      if (!seen[d.cap_fwd[k]]) { seen[d.cap_fwd[k]] = 1; capfwd[j].push_back(d.cap_fwd[k]); }
    m.n_capfwd = (int)capfwd[j].size();
    fwdnp[j].assign(d.n_fwd, 0);
    int NP = 0;
    for (int i = 0; i < d.n_fwd; ++i) {
      fwdnp[j][i] = d.model == SABR_LMM_MODEL_REBONATO ? n_panels(d.T[i], m.panel) : 0;
      if (seen[i]) NP = std::max(NP, fwdnp[j][i]);
    }
    // distinct underlying swaps, numbered in (first forward, last forward) order so that the swaps
    // of one expiry group are contiguous
    std::map<std::pair<int, int>, int> idx;
    for (int k = 0; k < d.n_swp; ++k) idx[std::make_pair(d.swp_start[k], d.swp_end[k])] = 0;
    int max_win = 1, nid = 0;
    for (auto& kv : idx) {
      kv.second = nid++;
      swap_a[j].push_back(kv.first.first);
      swap_b[j].push_back(kv.first.second);
      swap_np[j].push_back(n_panels(d.T[kv.first.first], m.panel));
      max_win = std::max(max_win, kv.first.second - kv.first.first);
    }
    for (int k = 0; k < d.n_swp; ++k) swp_swap[j].push_back(idx[std::make_pair(d.swp_start[k], d.swp_end[k])]);
    // expiry groups: swaps sharing their first forward share every pair integral G_ij(T_E), X_ij(T_E)
    int NA = 1, ND = 1, max_gwin = 1;
    for (int sidx = 0; sidx < (int)swap_a[j].size(); ++sidx) {
      const int a = swap_a[j][sidx];
      if (grp_a[j].empty() || grp_a[j].back() != a) {
        grp_a[j].push_back(a);
        grp_nE[j].push_back(n_panels(d.T[a], m.panel));
        grp_L[j].push_back(0);
        grp_swap0[j].push_back(sidx);
      }
      const int g = (int)grp_a[j].size() - 1;
      swap_grp[j].push_back(g);
      swap_L[j].push_back(swap_b[j][sidx] - a);
      grp_L[j][g] = std::max(grp_L[j][g], swap_b[j][sidx] - a);
    }
    grp_swap0[j].push_back((int)swap_a[j].size());
    for (size_t g = 0; g < grp_a[j].size(); ++g) max_gwin = std::max(max_gwin, grp_L[j][g]);
    for (size_t g = 0; g < grp_a[j].size(); ++g) {
      const int a = grp_a[j][g];
      for (int i = 0; i < max_gwin; ++i) {
        const int dl = i < grp_L[j][g] ? n_panels(d.T[a + i] - d.T[a], m.panel) : 0;
        grp_delta[j].push_back(dl);
      }
      const int dmax = grp_delta[j][g * max_gwin + grp_L[j][g] - 1];
      NA = std::max(NA, grp_nE[j][g] + dmax);
      ND = std::max(ND, dmax + 1);
    }
    m.n_grp = (int)grp_a[j].size();
    // on the CTA path a caplet on forward i is the window [0, n_i) of diagonal 0 of the pair
    // tables: the tables reach every caplet forward's fixing (a caplet-only market takes that path
    // inside a batch with swaption markets)
    m.NA = d.n_cap > 0 ? std::max(NA, NP) : NA;
    m.ND = ND;
    m.max_gwin = max_gwin;
    // quadratic forms by expiry group: every group's pair triangle (columns j < L_g, rows i <= j)
    // cut into segments of <= kSeg pairs of one column, column by column, group by group
    if (ND > 255) return fail(SABR_LMM_ENOTSUP, "market " + std::to_string(j) + ": a swap window spans more than 255 panels");
    for (size_t g = 0; g < grp_a[j].size(); ++g) {
      grp_col0[j].push_back((int)col_seg0[j].size());
      for (int jj = 0; jj < grp_L[j][g]; ++jj) {
        col_seg0[j].push_back((int)seg[j].size());
        col_u[j].push_back((int)g * max_gwin + jj);
        for (int i0 = 0; i0 <= jj; i0 += kSeg) {
          const int n = std::min(kSeg, jj + 1 - i0);
          seg[j].push_back((int)g | (jj << 8) | (i0 << 16) | (n << 24));
        }
      }
    }
    grp_col0[j].push_back((int)col_seg0[j].size());
    m.n_col = (int)col_seg0[j].size();
    col_seg0[j].push_back((int)seg[j].size());
    m.n_seg = (int)seg[j].size();
    for (size_t sidx = 0; sidx < swap_a[j].size(); ++sidx) {
      const int c0 = grp_col0[j][swap_grp[j][sidx]];
      sseg[j].push_back(col_seg0[j][c0]);
      sseg[j].push_back(col_seg0[j][c0 + swap_L[j][sidx]]);
    }
    // the forward sweep's segment descriptors: segment s of S in column jj takes the pairs
    // i = s + S r (r = 0..3, i <= jj); an empty slot repeats pair (jj, jj) with weight 0
    {
      std::vector<int>& dv = sdsc[j];
      std::vector<int>& uv = suix[j];
      dv.assign((size_t)m.n_seg * 4, 0);
      uv.assign((size_t)m.n_seg * 4, 0);
      int q = 0;
      for (size_t g = 0; g < grp_a[j].size(); ++g) {
        const int nE = grp_nE[j][g];
        const int* dl = grp_delta[j].data() + g * max_gwin;
        for (int jj = 0; jj < grp_L[j][g]; ++jj) {
          const int S = (jj + 1 + kSeg - 1) / kSeg;
          for (int sg = 0; sg < S; ++sg, ++q) {
            for (int r = 0; r < kSeg; ++r) {
              const int i = sg + S * r;
              const bool valid = i <= jj;
              const int ii = valid ? i : jj;
              const int lo = dl[ii], e = dl[jj] - lo;
              if (lo + nE > 255) return fail(SABR_LMM_ENOTSUP, "market " + std::to_string(j) + ": a swap window ends beyond panel 255");
              dv[(size_t)q * 4 + 0] |= lo << (8 * r);
              dv[(size_t)q * 4 + 1] |= e << (8 * r);
              uv[(size_t)q * 4 + r] = ((int)g * max_gwin + ii) | ((ii == jj ? 1 : 0) << 20) | ((valid ? 1 : 0) << 21);
            }
            dv[(size_t)q * 4 + 2] = nE;
            dv[(size_t)q * 4 + 3] = (int)g * max_gwin + jj;
          }
        }
      }
    }
    m.n_swap = (int)swap_a[j].size();
    m.max_win = max_win;
    m.NP = std::max(NP, 1);
    // the segment partials (3 x n_seg) in the Y region when they fit there
    m.qf_own = 3 * m.n_seg > m.NA * cta_y_stride() ? 1 : 0;
    HostMarket& h = hm[j];
    h.model = d.model; h.formula = d.formula; h.n_param = d.n_param; h.n_fwd = d.n_fwd;
    h.n_cap = d.n_cap; h.n_swp = d.n_swp; h.beta = d.beta;
    h.lo.assign(d.lo, d.lo + d.n_param);
    h.hi.assign(d.hi, d.hi + d.n_param);
    h.freem.assign(d.free_mask, d.free_mask + d.n_param);
    h.cap_vol.assign(d.cap_vol ? d.cap_vol : d.cap_K, (d.cap_vol ? d.cap_vol : d.cap_K) + d.n_cap);
    h.swp_vol.assign(d.swp_vol ? d.swp_vol : d.swp_K, (d.swp_vol ? d.swp_vol : d.swp_K) + d.n_swp);
    Off& o = off[j];
    const int nf1 = d.n_fwd + 1;
    o.T = A.take(nf1 * 8); o.P = A.take(nf1 * 8);
    o.cap_K = A.take(d.n_cap * 8); o.cap_vol = A.take(d.n_cap * 8); o.cap_wu = A.take(d.n_cap * 8);
    o.swp_K = A.take(d.n_swp * 8); o.swp_vol = A.take(d.n_swp * 8); o.swp_wu = A.take(d.n_swp * 8);
    o.cap_fwd = A.take(d.n_cap * 4); o.swp_start = A.take(d.n_swp * 4); o.swp_end = A.take(d.n_swp * 4);
    o.swp_swap = A.take(d.n_swp * 4); o.swap_a = A.take(m.n_swap * 4); o.swap_b = A.take(m.n_swap * 4);
    o.capfwd_list = A.take(m.n_capfwd * 4); o.fwd_np = A.take(d.n_fwd * 4);
    o.lo = A.take(d.n_param * 8); o.hi = A.take(d.n_param * 8); o.freem = A.take(d.n_param);
    o.F = A.take(d.n_fwd * 8); o.tau = A.take(d.n_fwd * 8);
    o.swap_A = A.take(m.n_swap * 8); o.swap_S = A.take(m.n_swap * 8); o.swap_TE = A.take(m.n_swap * 8);
    o.swap_W = A.take((size_t)m.n_swap * max_win * 8); o.swap_np = A.take(m.n_swap * 4);
    o.cap_pm = A.take(d.n_cap * 8); o.cap_w = A.take(d.n_cap * 8);
    o.swp_pm = A.take(d.n_swp * 8); o.swp_w = A.take(d.n_swp * 8);
    o.cblk64 = A.take(instr_block_bytes<double>(m.n_cap_pad)); o.cblk32 = A.take(instr_block_bytes<float>(m.n_cap_pad));
    o.cpair32 = A.take(pair_block_bytes(cap_pairs(d.n_cap)));
    o.sblk64 = A.take(instr_block_bytes<double>(m.n_swp_pad)); o.sblk32 = A.take(instr_block_bytes<float>(m.n_swp_pad));
    o.q64 = A.take(sizeof(QuadTab<double>)); o.q32 = A.take(sizeof(QuadTab<float>));
    o.err = A.take(16);
    const int ng = m.n_grp;
    o.grp_a = A.take(ng * 4); o.grp_nE = A.take(ng * 4); o.grp_L = A.take(ng * 4);
    o.grp_delta = A.take((size_t)ng * m.max_gwin * 4); o.grp_swap0 = A.take((ng + 1) * 4);
    o.swap_grp = A.take(m.n_swap * 4); o.swap_L = A.take(m.n_swap * 4);
    o.seg = A.take((size_t)m.n_seg * 4);
    o.col_seg0 = A.take((size_t)(m.n_col + 1) * 4);
    o.seg_dsc = A.take((size_t)m.n_seg * 16);
    o.seg_uix = A.take((size_t)m.n_seg * 16);
    o.seg_w64 = A.take((size_t)m.n_seg * 32);
    o.seg_w32 = A.take((size_t)m.n_seg * 16);
    o.swap_segs = A.take((size_t)m.n_swap * 8);
    o.col_u = A.take((size_t)m.n_col * 4);
    o.grp_col0 = A.take((size_t)(ng + 1) * 4);
    o.grp_u64 = A.take((size_t)ng * m.max_gwin * 8);
    o.grp_u32 = A.take((size_t)ng * m.max_gwin * 4);
    o.swap_scale64 = A.take((size_t)m.n_swap * 8);
    o.swap_scale32 = A.take((size_t)m.n_swap * 4);
    const bool mm = d.model == SABR_LMM_MODEL_MERCURIO_MORINI;
    o.mm_k64 = A.take(mm ? d.n_fwd * 8 : 0);
    o.mm_k32 = A.take(mm ? d.n_fwd * 4 : 0);
  }
  std::vector<unsigned char> host(A.size, 0);
  auto put = [&](size_t o, const void* src, size_t bytes) { if (src && bytes) std::memcpy(host.data() + o, src, bytes); };
  // quadrature table (same for every market of a given panel width)
  for (int j = 0; j < n_markets; ++j) {
    const sabr_lmm_market_desc& d = descs[j];
    const Off& o = off[j];
    const DevMarket& m = dm[j];
    put(o.T, d.T, (d.n_fwd + 1) * 8); put(o.P, d.P, (d.n_fwd + 1) * 8);
    put(o.cap_K, d.cap_K, d.n_cap * 8); put(o.cap_vol, d.cap_vol, d.n_cap * 8); put(o.cap_wu, d.cap_w, d.cap_w ? d.n_cap * 8 : 0);
    put(o.swp_K, d.swp_K, d.n_swp * 8); put(o.swp_vol, d.swp_vol, d.n_swp * 8); put(o.swp_wu, d.swp_w, d.swp_w ? d.n_swp * 8 : 0);
    put(o.cap_fwd, d.cap_fwd, d.n_cap * 4); put(o.swp_start, d.swp_start, d.n_swp * 4); put(o.swp_end, d.swp_end, d.n_swp * 4);
    put(o.swp_swap, swp_swap[j].data(), d.n_swp * 4);
    put(o.swap_a, swap_a[j].data(), m.n_swap * 4); put(o.swap_b, swap_b[j].data(), m.n_swap * 4);
    put(o.swap_np, swap_np[j].data(), m.n_swap * 4);
    put(o.capfwd_list, capfwd[j].data(), m.n_capfwd * 4); put(o.fwd_np, fwdnp[j].data(), d.n_fwd * 4);
    put(o.lo, d.lo, d.n_param * 8); put(o.hi, d.hi, d.n_param * 8); put(o.freem, d.free_mask, d.n_param);
    put(o.grp_a, grp_a[j].data(), m.n_grp * 4); put(o.grp_nE, grp_nE[j].data(), m.n_grp * 4);
    put(o.grp_L, grp_L[j].data(), m.n_grp * 4);
    put(o.grp_delta, grp_delta[j].data(), (size_t)m.n_grp * m.max_gwin * 4);
    put(o.grp_swap0, grp_swap0[j].data(), (m.n_grp + 1) * 4);
    put(o.swap_grp, swap_grp[j].data(), m.n_swap * 4); put(o.swap_L, swap_L[j].data(), m.n_swap * 4);
    put(o.seg, seg[j].data(), (size_t)m.n_seg * 4);
    put(o.col_seg0, col_seg0[j].data(), col_seg0[j].size() * 4);
    put(o.seg_dsc, sdsc[j].data(), sdsc[j].size() * 4);
    put(o.seg_uix, suix[j].data(), suix[j].size() * 4);
    put(o.swap_segs, sseg[j].data(), sseg[j].size() * 4);
    put(o.col_u, col_u[j].data(), col_u[j].size() * 4);
    put(o.grp_col0, grp_col0[j].data(), grp_col0[j].size() * 4);
    QuadTab<double> q64;
    QuadTab<float> q32;
    const double D = m.panel;
    for (int q = 0; q < kQ; ++q) {
      const double oq = 0.5 * D * (1.0 + kGLx[q]);
      const double hq = 0.5 * (D - oq);
      q64.o[q] = oq; q64.w[q] = 0.5 * D * kGLw[q]; q64.sw[q] = std::sqrt(0.5 * D * kGLw[q]);
      for (int r = 0; r < kQ; ++r) {
        q64.o2[q * kQ + r] = oq + hq * (1.0 + kGLx[r]);
        q64.sw2[q * kQ + r] = std::sqrt(hq * kGLw[r]);
      }
    }
    for (int i = 0; i < kQ; ++i) { q32.o[i] = (float)q64.o[i]; q32.w[i] = (float)q64.w[i]; q32.sw[i] = (float)q64.sw[i]; }
    for (int i = 0; i < kQ * kQ; ++i) { q32.o2[i] = (float)q64.o2[i]; q32.sw2[i] = (float)q64.sw2[i]; }
    put(o.q64, &q64, sizeof q64);
    put(o.q32, &q32, sizeof q32);
  }
  sabr_lmm_market* mk = new sabr_lmm_market();
  cudaGetDevice(&mk->device);
  cudaError_t e = cudaMalloc(&mk->arena, A.size);
  if (e != cudaSuccess) { delete mk; return fail(SABR_LMM_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e)); }
  e = cudaMemcpyAsync(mk->arena, host.data(), A.size, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) { cudaFree(mk->arena); delete mk; return fail(SABR_LMM_ECUDA, cudaGetErrorString(e)); }
  char* base = (char*)mk->arena;
  for (int j = 0; j < n_markets; ++j) {
    DevMarket& m = dm[j];
    const Off& o = off[j];
    m.T = (const double*)(base + o.T); m.P = (const double*)(base + o.P);
    m.cap_K = (const double*)(base + o.cap_K); m.cap_vol = (const double*)(base + o.cap_vol);
    m.cap_wu = descs[j].cap_w ? (const double*)(base + o.cap_wu) : nullptr;
    m.swp_K = (const double*)(base + o.swp_K); m.swp_vol = (const double*)(base + o.swp_vol);
    m.swp_wu = descs[j].swp_w ? (const double*)(base + o.swp_wu) : nullptr;
    m.cap_fwd = (const int*)(base + o.cap_fwd); m.swp_start = (const int*)(base + o.swp_start);
    m.swp_end = (const int*)(base + o.swp_end); m.swp_swap = (const int*)(base + o.swp_swap);
    m.swap_a = (const int*)(base + o.swap_a); m.swap_b = (const int*)(base + o.swap_b);
    m.capfwd_list = (const int*)(base + o.capfwd_list); m.fwd_np = (const int*)(base + o.fwd_np);
    m.lo = (const double*)(base + o.lo); m.hi = (const double*)(base + o.hi);
    m.freem = (const unsigned char*)(base + o.freem);
    m.F = (double*)(base + o.F); m.tau = (double*)(base + o.tau);
    m.swap_A = (double*)(base + o.swap_A); m.swap_S = (double*)(base + o.swap_S); m.swap_TE = (double*)(base + o.swap_TE);
    m.swap_W = (double*)(base + o.swap_W); m.swap_np = (int*)(base + o.swap_np);
    m.cap_pm = (double*)(base + o.cap_pm); m.cap_w = (double*)(base + o.cap_w);
    m.swp_pm = (double*)(base + o.swp_pm); m.swp_w = (double*)(base + o.swp_w);
    m.cblk64 = base + o.cblk64; m.cblk32 = base + o.cblk32; m.sblk64 = base + o.sblk64; m.sblk32 = base + o.sblk32;
    m.cpair32 = base + o.cpair32; m.n_cap_pairs = cap_pairs(m.n_cap);
    m.q64 = (const QuadTab<double>*)(base + o.q64); m.q32 = (const QuadTab<float>*)(base + o.q32);
    m.err = (int*)(base + o.err);
    m.grp_a = (const int*)(base + o.grp_a); m.grp_nE = (const int*)(base + o.grp_nE);
    m.grp_L = (const int*)(base + o.grp_L); m.grp_delta = (const int*)(base + o.grp_delta);
    m.grp_swap0 = (const int*)(base + o.grp_swap0); m.swap_grp = (const int*)(base + o.swap_grp);
    m.swap_L = (const int*)(base + o.swap_L);
    m.seg = (const int*)(base + o.seg); m.col_seg0 = (const int*)(base + o.col_seg0);
    m.seg_dsc = (const int4*)(base + o.seg_dsc); m.seg_uix = (const int4*)(base + o.seg_uix);
    m.seg_w64 = (const double*)(base + o.seg_w64); m.seg_w32 = (const float*)(base + o.seg_w32);
    m.swap_segs = (const int2*)(base + o.swap_segs);
    m.col_u = (const int*)(base + o.col_u); m.grp_col0 = (const int*)(base + o.grp_col0);
    m.grp_u64 = (const double*)(base + o.grp_u64); m.grp_u32 = (const float*)(base + o.grp_u32);
    m.swap_scale64 = (const double*)(base + o.swap_scale64); m.swap_scale32 = (const float*)(base + o.swap_scale32);
    const bool mm = m.model == SABR_LMM_MODEL_MERCURIO_MORINI;
    m.mm_k64 = mm ? (const double*)(base + o.mm_k64) : nullptr;
    m.mm_k32 = mm ? (const float*)(base + o.mm_k32) : nullptr;
    setup_forwards_kernel<<<(m.n_fwd + 127) / 128, 128, 0, s>>>(m);
    if (m.n_swap > 0) {
      setup_swaps_kernel<<<(m.n_swap + 127) / 128, 128, 0, s>>>(m);
      setup_group_u_kernel<<<(m.n_grp * m.max_gwin + 127) / 128, 128, 0, s>>>(m);
      setup_seg_weights_kernel<<<(m.n_seg + 127) / 128, 128, 0, s>>>(m);
    }
    const int ni = m.n_cap + m.n_swp;
    setup_instruments_kernel<<<(ni + 127) / 128, 128, 0, s>>>(m);
    if (m.n_cap > 0) setup_pairs_kernel<<<(m.n_cap_pairs + 127) / 128, 128, 0, s>>>(m);
  }
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) { cudaFree(mk->arena); delete mk; return fail(SABR_LMM_ECUDA, cudaGetErrorString(e)); }
  mk->dm = dm;
  mk->hm = hm;
  *out = mk;
  return SABR_LMM_OK;
}

extern "C" void sabr_lmm_free_market(sabr_lmm_market* m) {
  if (!m) return;
  if (m->arena) cudaFree(m->arena);
  delete m;
}

// ====================================================================== dispatch
namespace {

// Raise, never lower, a kernel's dynamic shared-memory limit on the current device.  Plans of
// different markets configure the same kernel functions, and a launch (or a graph captured at a
// plan's first launch) needs the largest size any of them asked for.
template <class K>
cudaError_t raise_smem_limit(K kern, uint32_t bytes) {
  static std::mutex mu;
  static std::map<std::pair<int, const void*>, uint32_t> lim;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lk(mu);
  uint32_t& cur = lim[std::make_pair(dev, (const void*)kern)];
  if (bytes <= cur) return cudaSuccess;
  e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess) cur = bytes;
  return e;
}

template <class R, int MODEL, int FORMULA>
cudaError_t launch_objective(const DevMarket& m, const double* X, long long n, double* f, double* vols, double* res,
                             cudaStream_t s) {
  // a few sets (a polish's trial points and stencils): one set per CTA spreads them over the SMs
  const int W = n <= 148 * 8 ? 1 : 4;
  const uint32_t sm = smem_bytes<R>(m, W);
  auto kern = objective_kernel<R, MODEL, FORMULA>;
  cudaError_t e = raise_smem_limit(kern, sm);
  if (e != cudaSuccess) return e;
  long long blocks = (n + W - 1) / W;
  if (blocks > 148 * 64) blocks = 148 * 64;
  if (blocks < 1) blocks = 1;
  kern<<<(unsigned)blocks, W * 32, sm, s>>>(m, X, n, f, vols, res);
  return cudaGetLastError();
}

template <class R>
cudaError_t launch_objective_r(const DevMarket& m, const double* X, long long n, double* f, double* vols, double* res,
                               cudaStream_t s) {
  if (m.model == 0) return m.formula == 0 ? launch_objective<R, 0, 0>(m, X, n, f, vols, res, s) : launch_objective<R, 0, 1>(m, X, n, f, vols, res, s);
  if (m.model == 2) return m.formula == 0 ? launch_objective<R, 2, 0>(m, X, n, f, vols, res, s) : launch_objective<R, 2, 1>(m, X, n, f, vols, res, s);
  return m.formula == 0 ? launch_objective<R, 1, 0>(m, X, n, f, vols, res, s) : launch_objective<R, 1, 1>(m, X, n, f, vols, res, s);
}

// The tensor-core contraction of the pair Grams applies when the panel tables fit one MMA tile.
bool tc_eligible(const DevMarket& m) { return m.n_swp > 0 && m.NA <= 64 && m.ND <= 27; }
bool use_tc(const DevMarket& m, int prec) { return prec == SABR_LMM_FP32_BF16X3 && tc_eligible(m); }

template <class R, int FORMULA, bool TC>
cudaError_t launch_objective_cta(const DevMarket& m, const double* X, long long n, double* f, double* vols, double* res,
                                 cudaStream_t s) {
  const uint32_t sm = smem_bytes_cta<R>(m, TC);
  auto kern = objective_cta_kernel<R, FORMULA, TC>;
  cudaError_t e = raise_smem_limit(kern, sm);
  if (e != cudaSuccess) return e;
  long long blocks = n < 148 * 16 ? n : 148 * 16;
  if (blocks < 1) blocks = 1;
  kern<<<(unsigned)blocks, 256, sm, s>>>(m, X, n, f, vols, res);
  return cudaGetLastError();
}

cudaError_t launch_objective_any(const DevMarket& m, int prec, const double* X, long long n, double* f, double* vols,
                                 cudaStream_t s, double* res = nullptr) {
  if (m.n_swp > 0) {
    if (prec == SABR_LMM_FP64)
      return m.formula == 0 ? launch_objective_cta<double, 0, false>(m, X, n, f, vols, res, s) : launch_objective_cta<double, 1, false>(m, X, n, f, vols, res, s);
    if (use_tc(m, prec))
      return m.formula == 0 ? launch_objective_cta<float, 0, true>(m, X, n, f, vols, res, s) : launch_objective_cta<float, 1, true>(m, X, n, f, vols, res, s);
    return m.formula == 0 ? launch_objective_cta<float, 0, false>(m, X, n, f, vols, res, s) : launch_objective_cta<float, 1, false>(m, X, n, f, vols, res, s);
  }
  return prec == SABR_LMM_FP64 ? launch_objective_r<double>(m, X, n, f, vols, res, s)
                               : launch_objective_r<float>(m, X, n, f, vols, res, s);
}

// Shared memory a market needs per CTA in the given precision (the caller checks it against the
// device's opt-in limit).
uint32_t market_smem(const DevMarket& m, int prec) {
  if (m.n_swp > 0) return prec == SABR_LMM_FP64 ? smem_bytes_cta<double>(m) : smem_bytes_cta<float>(m, use_tc(m, prec));
  return prec == SABR_LMM_FP64 ? smem_bytes<double>(m, 4) : smem_bytes<float>(m, 4);
}

sabr_lmm_status check_call(const sabr_lmm_market* m, int32_t idx, int64_t n, int32_t prec) {
  if (!m) return fail(SABR_LMM_EINVAL, "market is NULL");
  if (idx < 0 || idx >= (int)m->dm.size()) return fail(SABR_LMM_EINVAL, "market_idx out of range");
  if (n < 0) return fail(SABR_LMM_EINVAL, "n must be >= 0");
  if (!valid_prec(prec)) return fail(SABR_LMM_EINVAL, "unknown precision");
  if (market_smem(m->dm[idx], prec) > 227 * 1024)
    return fail(SABR_LMM_ENOTSUP, "the market does not fit in one CTA's shared memory at this precision");
  if (m->dm[idx].n_swp > 0 && prec == SABR_LMM_FP32_BF16X3 && !tc_eligible(m->dm[idx]))
    return fail(SABR_LMM_ENOTSUP, "the market's panel tables exceed one tensor-core tile (NA <= 64, ND <= 27)");
  return SABR_LMM_OK;
}

}  // namespace

extern "C" sabr_lmm_status sabr_lmm_objective(const sabr_lmm_market* m, int32_t idx, const double* X, int64_t n,
                                              int32_t prec, double* f, void* stream) {
  sabr_lmm_status st = check_call(m, idx, n, prec);
  if (st != SABR_LMM_OK) return st;
  if (n == 0) return SABR_LMM_OK;
  if (!X || !f) return fail(SABR_LMM_EINVAL, "X and f are required");
  CUDA_TRY(launch_objective_any(m->dm[idx], prec, X, n, f, nullptr, (cudaStream_t)stream));
  return SABR_LMM_OK;
}

extern "C" sabr_lmm_status sabr_lmm_residuals(const sabr_lmm_market* m, int32_t idx, const double* X, int64_t n,
                                              int32_t prec, double* f, double* res, void* stream) {
  sabr_lmm_status st = check_call(m, idx, n, prec);
  if (st != SABR_LMM_OK) return st;
  if (n == 0) return SABR_LMM_OK;
  if (!X || !res) return fail(SABR_LMM_EINVAL, "X and res are required");
  CUDA_TRY(launch_objective_any(m->dm[idx], prec, X, n, f, nullptr, (cudaStream_t)stream, res));
  return SABR_LMM_OK;
}

extern "C" sabr_lmm_status sabr_lmm_model_vols(const sabr_lmm_market* m, int32_t idx, const double* X, int64_t n,
                                               int32_t prec, double* vols, void* stream) {
  sabr_lmm_status st = check_call(m, idx, n, prec);
  if (st != SABR_LMM_OK) return st;
  if (n == 0) return SABR_LMM_OK;
  if (!X || !vols) return fail(SABR_LMM_EINVAL, "X and vols are required");
  CUDA_TRY(launch_objective_any(m->dm[idx], prec, X, n, nullptr, vols, (cudaStream_t)stream));
  return SABR_LMM_OK;
}

namespace {
template <class R, int MODEL, int FORMULA>
cudaError_t launch_grad(const DevMarket& m, const double* X, long long n, double* f, double* G, cudaStream_t s) {
  const int W = n <= 148 * 8 ? 1 : 4;   // a few sets: one per CTA
  const uint32_t sm = smem_bytes_grad<R>(m, W);
  auto kern = grad_kernel<R, MODEL, FORMULA>;
  cudaError_t e = raise_smem_limit(kern, sm);
  if (e != cudaSuccess) return e;
  long long blocks = (n + W - 1) / W;
  if (blocks > 148 * 32) blocks = 148 * 32;
  if (blocks < 1) blocks = 1;
  kern<<<(unsigned)blocks, W * 32, sm, s>>>(m, X, n, f, G);
  return cudaGetLastError();
}

template <class R>
cudaError_t launch_grad_r(const DevMarket& m, const double* X, long long n, double* f, double* G, cudaStream_t s) {
  if (m.model == 0) return m.formula == 0 ? launch_grad<R, 0, 0>(m, X, n, f, G, s) : launch_grad<R, 0, 1>(m, X, n, f, G, s);
  return m.formula == 0 ? launch_grad<R, 1, 0>(m, X, n, f, G, s) : launch_grad<R, 1, 1>(m, X, n, f, G, s);
}
}  // namespace

namespace {
// Markets with swaptions: one CTA per point (FP64), the forms' partials in their own region.
template <int FORMULA>
cudaError_t launch_grad_cta(DevMarket m, const double* X, long long n, double* f, double* G, cudaStream_t s) {
  m.qf_own = 1;
  const uint32_t sm = smem_bytes_grad_cta(m);
  auto kern = grad_cta_kernel<FORMULA>;
  cudaError_t e = raise_smem_limit(kern, sm);
  if (e != cudaSuccess) return e;
  long long blocks = n < 148 * 4 ? n : 148 * 4;
  if (blocks < 1) blocks = 1;
  kern<<<(unsigned)blocks, 256, sm, s>>>(m, X, n, f, G);
  return cudaGetLastError();
}

// The reverse sweep of any market: caplet markets at `prec`, markets with swaptions in FP64.
cudaError_t launch_grad_any(const DevMarket& m, int prec, const double* X, long long n, double* f, double* G,
                            cudaStream_t s) {
  if (m.n_swp > 0) return m.formula == 0 ? launch_grad_cta<0>(m, X, n, f, G, s) : launch_grad_cta<1>(m, X, n, f, G, s);
  return prec == SABR_LMM_FP64 ? launch_grad_r<double>(m, X, n, f, G, s) : launch_grad_r<float>(m, X, n, f, G, s);
}

// Whether the reverse sweep of market m fits one CTA's shared memory.
bool grad_fits(const DevMarket& m) {
  if (m.n_swp == 0) return true;
  DevMarket m1 = m;
  m1.qf_own = 1;
  return smem_bytes_grad_cta(m1) <= 227u * 1024u;
}
}  // namespace

extern "C" sabr_lmm_status sabr_lmm_objective_grad(const sabr_lmm_market* m, int32_t idx, const double* X, int64_t n,
                                                   int32_t prec, double* f, double* G, void* stream) {
  sabr_lmm_status st = check_call(m, idx, n, prec);
  if (st != SABR_LMM_OK) return st;
  if (m->dm[idx].n_param > kMaxGradParam || m->dm[idx].model == SABR_LMM_MODEL_MERCURIO_MORINI)
    return fail(SABR_LMM_ENOTSUP, "the reverse sweep covers the smile and Rebonato models (at most 12 parameter slots)");
  if (!grad_fits(m->dm[idx]))
    return fail(SABR_LMM_ENOTSUP, "the reverse sweep of this market does not fit one CTA's shared memory");
  if (n == 0) return SABR_LMM_OK;
  if (!X || !f || !G) return fail(SABR_LMM_EINVAL, "X, f and G are required");
  CUDA_TRY(launch_grad_any(m->dm[idx], prec, X, n, f, G, (cudaStream_t)stream));
  return SABR_LMM_OK;
}

namespace {
// Nelder-Mead from n points (FP64): one warp per point on caplet markets, one CTA per point on markets
// with swaptions.
template <int MODEL, int FORMULA>
cudaError_t launch_nm_t(const DevMarket& m, double* X, long long n, int max_iter, double step, double ftol, double* f,
                        int* evals, cudaStream_t s) {
  const uint32_t sm = ((smem_bytes<double>(m, 1) + 15u) & ~15u) + nm_team_bytes();
  auto kern = nm_kernel<MODEL, FORMULA>;
  cudaError_t e = raise_smem_limit(kern, sm);
  if (e != cudaSuccess) return e;
  const long long blocks = n < 148 * 16 ? n : 148 * 16;
  kern<<<(unsigned)blocks, 32, sm, s>>>(m, X, n, max_iter, step, ftol, f, evals);
  return cudaGetLastError();
}

template <int FORMULA>
cudaError_t launch_nm_cta_t(const DevMarket& m, double* X, long long n, int max_iter, double step, double ftol,
                            double* f, int* evals, cudaStream_t s) {
  const uint32_t sm = ((smem_bytes_cta<double>(m) + 15u) & ~15u) + nm_team_bytes();
  auto kern = nm_cta_kernel<FORMULA>;
  cudaError_t e = raise_smem_limit(kern, sm);
  if (e != cudaSuccess) return e;
  const long long blocks = n < 148 * 2 ? n : 148 * 2;
  kern<<<(unsigned)blocks, 256, sm, s>>>(m, X, n, max_iter, step, ftol, f, evals);
  return cudaGetLastError();
}

cudaError_t launch_nm(const DevMarket& m, double* X, long long n, int max_iter, double step, double ftol, double* f,
                      int* evals, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  if (m.n_swp > 0)
    return m.formula == 0 ? launch_nm_cta_t<0>(m, X, n, max_iter, step, ftol, f, evals, s)
                          : launch_nm_cta_t<1>(m, X, n, max_iter, step, ftol, f, evals, s);
  if (m.model == 0)
    return m.formula == 0 ? launch_nm_t<0, 0>(m, X, n, max_iter, step, ftol, f, evals, s)
                          : launch_nm_t<0, 1>(m, X, n, max_iter, step, ftol, f, evals, s);
  if (m.model == 2)
    return m.formula == 0 ? launch_nm_t<2, 0>(m, X, n, max_iter, step, ftol, f, evals, s)
                          : launch_nm_t<2, 1>(m, X, n, max_iter, step, ftol, f, evals, s);
  return m.formula == 0 ? launch_nm_t<1, 0>(m, X, n, max_iter, step, ftol, f, evals, s)
                        : launch_nm_t<1, 1>(m, X, n, max_iter, step, ftol, f, evals, s);
}

uint32_t nm_smem(const DevMarket& m) {
  return (m.n_swp > 0 ? ((smem_bytes_cta<double>(m) + 15u) & ~15u) : ((smem_bytes<double>(m, 1) + 15u) & ~15u)) +
         nm_team_bytes();
}
}  // namespace

extern "C" sabr_lmm_status sabr_lmm_nm_polish(const sabr_lmm_market* m, int32_t idx, double* X, int64_t n,
                                              int32_t max_iter, double step, double ftol, double* f, int32_t* evals,
                                              void* stream) {
  sabr_lmm_status st = check_call(m, idx, n, SABR_LMM_FP64);
  if (st != SABR_LMM_OK) return st;
  if (max_iter < 0 || !(step > 0.0 && step <= 1.0) || !(ftol >= 0.0))
    return fail(SABR_LMM_EINVAL, "max_iter >= 0, 0 < step <= 1 and ftol >= 0 required");
  if (nm_smem(m->dm[idx]) > 227u * 1024u) return fail(SABR_LMM_ENOTSUP, "the market and the simplex do not fit one CTA");
  if (n == 0) return SABR_LMM_OK;
  if (!X || !f) return fail(SABR_LMM_EINVAL, "X and f are required");
  CUDA_TRY(launch_nm(m->dm[idx], X, n, max_iter, step, ftol, f, evals, (cudaStream_t)stream));
  return SABR_LMM_OK;
}

namespace {

// Device buffers of a polish of n points (allocated by the caller of lm_enqueue).
struct LmWork {
  double *Xp, *vols, *res, *grad, *gf, *mu, *f, *ft, *rmse, *rmse_t, *Xt;
  int* done;
  int* any;     // set once any point has reached the target
};

size_t lm_work_bytes(const DevMarket& m, int n) {
  const size_t P = m.n_param, ni = m.n_cap + m.n_swp, S = kLmStencil;
  return 8 * ((size_t)n * S * P + 2 * (size_t)n * S * ni + 6 * (size_t)n + 2 * (size_t)n * P) + 4 * ((size_t)n + 1) + 16;
}

LmWork lm_carve(void* base, const DevMarket& m, int n) {
  const size_t P = m.n_param, ni = m.n_cap + m.n_swp, S = kLmStencil;
  double* p = (double*)base;
  LmWork w;
  w.Xp = p; p += (size_t)n * S * P;
  w.vols = p; p += (size_t)n * S * ni;
  w.res = p; p += (size_t)n * S * ni;
  w.grad = p; p += (size_t)n * P;
  w.gf = p; p += n;
  w.mu = p; p += n;
  w.f = p; p += n;
  w.ft = p; p += n;
  w.rmse = p; p += n;
  w.rmse_t = p; p += n;
  w.Xt = p; p += (size_t)n * P;
  w.done = (int*)p;
  w.any = w.done + n;
  return w;
}

__global__ void lm_init_kernel(int n, double* mu, int* done, int* any) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) { mu[i] = 1e-3; done[i] = 0; }
  if (i == 0) *any = 0;
}

// A non-blocking side stream and a fork/join event pair per device, made on first use: the
// reverse sweep of a polish runs there beside the stencil evaluation.
struct LmSide {
  cudaStream_t s2 = nullptr;
  cudaEvent_t fork = nullptr, join = nullptr;
};
std::mutex g_side_mu;

cudaError_t lm_side(LmSide& out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  static std::map<int, LmSide> sides;
  std::lock_guard<std::mutex> lk(g_side_mu);
  auto it = sides.find(dev);
  if (it == sides.end()) {
    LmSide sd;
    if ((e = cudaStreamCreateWithFlags(&sd.s2, cudaStreamNonBlocking)) != cudaSuccess) return e;
    if ((e = cudaEventCreateWithFlags(&sd.fork, cudaEventDisableTiming)) != cudaSuccess) return e;
    if ((e = cudaEventCreateWithFlags(&sd.join, cudaEventDisableTiming)) != cudaSuccess) return e;
    it = sides.emplace(dev, sd).first;
  }
  out = it->second;
  return cudaSuccess;
}

// Enqueue max_iter LM iterations on the n points X (device, updated in place); f and rmse end as
// those of the final points.  Per iteration: the stencil's model vols (1 + n_free points per point)
// and, on caplet markets, the reverse sweep beside them on a side stream; residuals, the step, the
// trial points' model vols with their f and RMSE, accept.  The first iteration's stencil row 0 gives
// the starting f and RMSE.  With stop_at_first (host-driven, never under stream capture) the
// iterations end as soon as any point has reached the target RMSE: the host reads one flag after
// the start and after each iteration.  Calls sharing a device share the side stream, so polishes
// on different streams of one device serialise their reverse sweeps.
cudaError_t lm_enqueue(const DevMarket& m, int n_free, double* X, int n, int max_iter, double target, const LmWork& w,
                       cudaStream_t s, bool stop_at_first = false) {
  const int S = 1 + n_free;   // stencil: the point and one forward step per free slot
  const bool have_adjoint = grad_fits(m);
  cudaError_t e;
  LmSide side;
  if (have_adjoint && max_iter > 0 && (e = lm_side(side)) != cudaSuccess) return e;
  lm_init_kernel<<<(n + 127) / 128, 128, 0, s>>>(n, w.mu, w.done, w.any);
  if (max_iter == 0) {
    if ((e = launch_objective_any(m, SABR_LMM_FP64, X, n, nullptr, w.vols, s)) != cudaSuccess) return e;
    lm_eval_kernel<<<n, 256, 0, s>>>(m, n, 1, w.vols, target, w.f, w.rmse, w.done, w.any);
    return cudaGetLastError();
  }
  auto reached = [&]() {
    if (!stop_at_first || !(target > 0.0)) return false;
    int h = 0;
    if (cudaMemcpyAsync(&h, w.any, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess) return false;
    return cudaStreamSynchronize(s) == cudaSuccess && h != 0;
  };
  for (int it = 0; it < max_iter; ++it) {
    if (have_adjoint) {   // fork: the reverse sweep at X on the side stream, beside the stencil
      if ((e = cudaEventRecord(side.fork, s)) != cudaSuccess) return e;
      if ((e = cudaStreamWaitEvent(side.s2, side.fork, 0)) != cudaSuccess) return e;
      e = launch_grad_any(m, SABR_LMM_FP64, X, n, w.gf, w.grad, side.s2);
      const cudaError_t e2 = cudaEventRecord(side.join, side.s2);
      if (e != cudaSuccess) return e;
      if (e2 != cudaSuccess) return e2;
    }
    // join before anything that reads the gradient, and before leaving (the caller may free w)
    auto join = [&]() { return have_adjoint ? cudaStreamWaitEvent(s, side.join, 0) : cudaSuccess; };
    lm_perturb_kernel<<<n, 32, 0, s>>>(n, m.n_param, S, m.freem, X, w.Xp);
    if ((e = launch_objective_any(m, SABR_LMM_FP64, w.Xp, (long long)n * S, nullptr, w.vols, s)) != cudaSuccess) {
      join();
      return e;
    }
    if (it == 0) {
      lm_eval_kernel<<<n, 256, 0, s>>>(m, n, S, w.vols, target, w.f, w.rmse, w.done, w.any);
      if (reached()) {
        if ((e = join()) != cudaSuccess) return e;
        break;
      }
    }
    residuals_from_vols_kernel<<<148 * 4, 256, 0, s>>>(m, (long long)n * S, w.vols, w.res);
    if ((e = join()) != cudaSuccess) return e;
    lm_step_kernel<<<n, 256, 0, s>>>(m, n, S, w.res, have_adjoint ? w.grad : nullptr, w.mu, w.done, X, w.Xt);
    if ((e = launch_objective_any(m, SABR_LMM_FP64, w.Xt, n, nullptr, w.vols, s)) != cudaSuccess) return e;
    lm_eval_kernel<<<n, 256, 0, s>>>(m, n, 1, w.vols, target, w.ft, w.rmse_t, nullptr, nullptr);
    lm_accept_kernel<<<(n + 127) / 128, 128, 0, s>>>(n, m.n_param, X, w.Xt, w.f, w.ft, w.rmse, w.rmse_t, target, w.mu,
                                                     w.done, w.any);
    if (reached()) break;
  }
  return cudaGetLastError();
}

}  // namespace

extern "C" sabr_lmm_status sabr_lmm_lm_polish(const sabr_lmm_market* m, int32_t idx, double* X, int64_t n,
                                              int32_t max_iter, double target, double* f, double* rmse, void* stream) {
  sabr_lmm_status st = check_call(m, idx, n, SABR_LMM_FP64);
  if (st != SABR_LMM_OK) return st;
  if (n == 0) return SABR_LMM_OK;
  if (!X) return fail(SABR_LMM_EINVAL, "X is required");
  if (max_iter < 0 || n > (1 << 20)) return fail(SABR_LMM_EINVAL, "max_iter >= 0 and n <= 2^20 required");
  if (m->dm[idx].n_param > kMaxGradParam || m->dm[idx].model == SABR_LMM_MODEL_MERCURIO_MORINI)
    return fail(SABR_LMM_ENOTSUP, "the Levenberg-Marquardt polish covers the smile and Rebonato models (at most 12 "
                                  "parameter slots)");
  const DevMarket& dm = m->dm[idx];
  cudaStream_t s = (cudaStream_t)stream;
  void* buf = nullptr;
  if (cudaMalloc(&buf, lm_work_bytes(dm, (int)n)) != cudaSuccess) return fail(SABR_LMM_ENOMEM, "cudaMalloc of the polish buffers failed");
  const LmWork w = lm_carve(buf, dm, (int)n);
  int n_free = 0;
  for (unsigned char f : m->hm[idx].freem) n_free += f != 0;
  cudaError_t e = lm_enqueue(dm, n_free, X, (int)n, max_iter, target, w, s);
  if (e == cudaSuccess && f) e = cudaMemcpyAsync(f, w.f, n * sizeof(double), cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess && rmse) e = cudaMemcpyAsync(rmse, w.rmse, n * sizeof(double), cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(buf);
  if (e != cudaSuccess) return fail(SABR_LMM_ECUDA, std::string("lm_polish: ") + cudaGetErrorString(e));
  return SABR_LMM_OK;
}

// ====================================================================== annealing
namespace {

// Kernel attributes are set before any launch (outside stream capture); enqueue only launches.
template <class R, int MODEL, int FORMULA>
cudaError_t enqueue_anneal_t(const DevMarket& m, const SAState& st, const SAParams& sp, int W, int grid, cudaStream_t s,
                             bool configure_only) {
  const uint32_t sm1 = smem_bytes<R>(m, 1), smW = smem_bytes<R>(m, W);
  auto k0 = sa_start_kernel<R, MODEL, FORMULA>;
  // more than 4 chains per CTA (FP32): the form with one CTA of up to 28 chains per SM
  auto k1 = (sizeof(R) == 4 && W > 4) ? sa_level_kernel<R, MODEL, FORMULA, true> : sa_level_kernel<R, MODEL, FORMULA, false>;
  if (configure_only) {
    cudaError_t e = raise_smem_limit(k0, sm1);
    if (e == cudaSuccess) e = raise_smem_limit(k1, smW);
    return e;
  }
  k0<<<1, 32, sm1, s>>>(m, st, sp);
  for (int l = 0; l < sp.L; ++l) k1<<<grid, W * 32, smW, s>>>(m, st, sp, l);
  sa_final_kernel<<<1, 1024, 0, s>>>(st, sp.C, sp.P);
  return cudaGetLastError();
}

// Markets with swaptions: one CTA of `threads` (256, or 128 without the tensor-core Grams) per chain.
template <class R, int FORMULA, bool TC>
cudaError_t enqueue_anneal_cta_t(const DevMarket& m, const SAState& st, const SAParams& sp, cudaStream_t s,
                                 bool configure_only, int threads) {
  const uint32_t sm = smem_bytes_cta<R>(m, TC);
  auto k0 = sa_start_cta_kernel<R, FORMULA, TC>;
  auto k1 = sa_level_cta_kernel<R, FORMULA, TC>;
  if (configure_only) {
    cudaError_t e = raise_smem_limit(k0, sm);
    if (e == cudaSuccess) e = raise_smem_limit(k1, sm);
    return e;
  }
  const int nt = TC ? 256 : threads;
  k0<<<1, nt, sm, s>>>(m, st, sp);
  for (int l = 0; l < sp.L; ++l) k1<<<sp.C, nt, sm, s>>>(m, st, sp, l);
  sa_final_kernel<<<1, 1024, 0, s>>>(st, sp.C, sp.P);
  return cudaGetLastError();
}

// Warps per CTA of the kernels of markets with swaptions: 4 (the default, 18 % faster per level than
// 8 on the 40-forward joint market: four CTAs per SM instead of two hide each other's barriers), or
// 8 when asked (warps_per_block >= 5).
int cta_warps_of(const sabr_lmm_anneal_opts* o) { return o->warps_per_block <= 4 ? 4 : 8; }

// cta_warps: warps per CTA of the kernels of markets with swaptions (4 or 8).
cudaError_t enqueue_anneal(const DevMarket& m, int prec, const SAState& st, const SAParams& sp, int W, int grid,
                           cudaStream_t s, bool configure_only = false, int cta_warps = 8) {
  const bool f64 = prec == SABR_LMM_FP64;
  if (m.n_swp > 0) {
    const int nt = 32 * cta_warps;
    if (f64) return m.formula == 0 ? enqueue_anneal_cta_t<double, 0, false>(m, st, sp, s, configure_only, nt)
                                   : enqueue_anneal_cta_t<double, 1, false>(m, st, sp, s, configure_only, nt);
    if (use_tc(m, prec))
      return m.formula == 0 ? enqueue_anneal_cta_t<float, 0, true>(m, st, sp, s, configure_only, nt)
                            : enqueue_anneal_cta_t<float, 1, true>(m, st, sp, s, configure_only, nt);
    return m.formula == 0 ? enqueue_anneal_cta_t<float, 0, false>(m, st, sp, s, configure_only, nt)
                          : enqueue_anneal_cta_t<float, 1, false>(m, st, sp, s, configure_only, nt);
  }
#define DISPATCH(R)                                                                                           \
  if (m.model == 0) return m.formula == 0 ? enqueue_anneal_t<R, 0, 0>(m, st, sp, W, grid, s, configure_only)  \
                                          : enqueue_anneal_t<R, 0, 1>(m, st, sp, W, grid, s, configure_only); \
  if (m.model == 2) return m.formula == 0 ? enqueue_anneal_t<R, 2, 0>(m, st, sp, W, grid, s, configure_only)  \
                                          : enqueue_anneal_t<R, 2, 1>(m, st, sp, W, grid, s, configure_only); \
  return m.formula == 0 ? enqueue_anneal_t<R, 1, 0>(m, st, sp, W, grid, s, configure_only)                   \
                        : enqueue_anneal_t<R, 1, 1>(m, st, sp, W, grid, s, configure_only);
  if (f64) { DISPATCH(double) } else { DISPATCH(float) }
#undef DISPATCH
}

template <class R, int FORMULA>
cudaError_t enqueue_batch_t(const sabr_lmm_anneal_plan* p, cudaStream_t s, int levels, bool configure_only, int only) {
  auto k0 = sa_start_batch_kernel<R, FORMULA>;
  auto k1 = sa_level_batch_kernel<R, FORMULA>;
  if (configure_only) {
    cudaError_t e = raise_smem_limit(k0, p->bsmem);
    if (e == cudaSuccess) e = raise_smem_limit(k1, p->bsmem);
    return e;
  }
  // every bucket's counters are one contiguous run after the first bucket's
  cudaError_t e = cudaMemsetAsync(p->bk[0].ba.item_ctr, 0,
                                  p->bk.size() * (size_t)p->opts.n_levels * sizeof(unsigned int), s);
  if (e != cudaSuccess) return e;
  k0<<<p->ba.n_markets, 256, p->bsmem, s>>>(p->ba);
  for (int l = 0; l < levels; ++l)
    for (int i = 0; i < (int)p->bk.size(); ++i) {
      if (only >= 0 && i != only) continue;
      const auto& b = p->bk[i];
      k1<<<b.grid, b.threads, b.smem, s>>>(b.ba, l);
    }
  sa_final_batch_kernel<<<p->ba.n_markets, 1024, 0, s>>>(p->ba);
  return cudaGetLastError();
}

// The batch search: start, levels x (one launch per bucket, or only bucket `only`), final.
cudaError_t enqueue_batch(const sabr_lmm_anneal_plan* p, cudaStream_t s, int levels, bool configure_only = false,
                          int only = -1) {
  const bool f64 = p->opts.prec == SABR_LMM_FP64;
  const int formula = p->mk->dm[0].formula;
  if (f64) return formula == 0 ? enqueue_batch_t<double, 0>(p, s, levels, configure_only, only)
                               : enqueue_batch_t<double, 1>(p, s, levels, configure_only, only);
  return formula == 0 ? enqueue_batch_t<float, 0>(p, s, levels, configure_only, only)
                      : enqueue_batch_t<float, 1>(p, s, levels, configure_only, only);
}

// CTAs of a kernel per SM at this CTA size and dynamic shared memory (0 if one does not fit).
// The occupancy query counts no CTA whose request exceeds the kernel's opt-in limit, so the
// limit is raised first to the device maximum less the kernel's static shared memory.
template <class K>
int blocks_per_sm(K kern, int threads, uint32_t smem) {
  int dev = 0, optin = 0, per_sm = 0;
  cudaFuncAttributes fa;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess ||
      cudaFuncGetAttributes(&fa, kern) != cudaSuccess)
    return 0;
  const int dyn_max = optin - (int)fa.sharedSizeBytes;
  if ((int)smem > dyn_max) return 0;
  if (raise_smem_limit(kern, (uint32_t)dyn_max) != cudaSuccess) return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem) != cudaSuccess) return 0;
  return per_sm;
}

int batch_blocks_per_sm(int prec, int threads, uint32_t smem) {
  return prec == SABR_LMM_FP64 ? blocks_per_sm(sa_level_batch_kernel<double, 0>, threads, smem)
                               : blocks_per_sm(sa_level_batch_kernel<float, 0>, threads, smem);
}

// Autotuner of the batch launches: per shared-memory bucket, CTA size x persistent grid, chosen by
// timing that bucket's launch on one level of a short probe (4 steps per chain) per candidate;
// cached per (precision, formula, instrument bucket, market-count bucket, CTAs/SM).
std::mutex g_tune_mu;
std::map<std::tuple<int, int, int, int, int>, std::pair<int, int>> g_tune_cache;

sabr_lmm_status tune_batch(sabr_lmm_anneal_plan* p, cudaStream_t s) {
  int dev = 0, nsm = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  std::vector<SAParams> probe(p->sp);
  for (auto& q : probe) q.N = std::min(q.N, 4);
  bool probing = false;
  cudaEvent_t a = nullptr, b = nullptr;
  for (int bi = 0; bi < (int)p->bk.size(); ++bi) {
    auto& bk = p->bk[bi];
    int max_instr = 0;
    for (int j : bk.markets) max_instr = std::max(max_instr, p->mk->dm[j].n_cap + p->mk->dm[j].n_swp);
    const auto key = std::make_tuple(p->opts.prec, p->mk->dm[0].formula, (max_instr + 255) / 256,
                                     (bk.ba.n_markets + 63) / 64, bk.per_sm);
    {
      std::lock_guard<std::mutex> lk(g_tune_mu);
      auto it = g_tune_cache.find(key);
      if (it != g_tune_cache.end()) { bk.threads = it->second.first; bk.grid = it->second.second; continue; }
    }
    std::vector<std::pair<int, int>> cand;
    for (int threads : {128, 256}) {
      const int per_sm = batch_blocks_per_sm(p->opts.prec, threads, bk.smem);
      if (per_sm < 1) continue;
      cand.push_back({threads, nsm * per_sm});
      cand.push_back({threads, 2 * nsm * per_sm});
    }
    if (cand.empty()) return fail(SABR_LMM_ENOTSUP, "a batch market does not fit in one CTA's shared memory");
    if (!probing) {
      CUDA_TRY(cudaMemcpyAsync((void*)p->ba.sp, probe.data(), probe.size() * sizeof(SAParams), cudaMemcpyHostToDevice, s));
      cudaEventCreate(&a);
      cudaEventCreate(&b);
      probing = true;
    }
    float best_ms = 1e30f;
    std::pair<int, int> best = cand[0];
    for (const auto& c : cand) {
      bk.threads = c.first;
      bk.grid = c.second;
      CUDA_TRY(enqueue_batch(p, s, 1, false, bi));   // warm-up
      CUDA_TRY(cudaEventRecord(a, s));
      CUDA_TRY(enqueue_batch(p, s, 1, false, bi));
      CUDA_TRY(cudaEventRecord(b, s));
      CUDA_TRY(cudaEventSynchronize(b));
      float ms = 0.f;
      cudaEventElapsedTime(&ms, a, b);
      if (ms < best_ms) { best_ms = ms; best = c; }
    }
    bk.threads = best.first;
    bk.grid = best.second;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune_cache[key] = best;
  }
  if (probing) {
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    CUDA_TRY(cudaMemcpyAsync((void*)p->ba.sp, p->sp.data(), p->sp.size() * sizeof(SAParams), cudaMemcpyHostToDevice, s));
    CUDA_TRY(cudaStreamSynchronize(s));
  }
  return SABR_LMM_OK;
}

// Autotuner of the caplet level kernel's tile: chains (warps) per CTA, for a single caplet market in
// FP32.  Every CTA size runs the same search bit for bit (a chain is one warp either way), so the
// choice changes the time only.  Candidates: the one-wave heuristic, 28, 16, 14, 8, 7 and 4 chains
// (those whose shared memory fits); each is timed on one level of the plan's own length (at most
// 100 steps), best of three after one untimed run; the heuristic stays unless another is 2 %
// faster; cached per (caplet pairs, panels, forwards, chains).  (Markets with swaptions get no such
// tuner: there the CTA size changes the order of the partial sums, and a timing-dependent choice
// would make a search differ in its last bits from one process to the next.)
std::map<std::tuple<int, int, int, int>, int> g_tune_w_cache;

sabr_lmm_status tune_caplet_w(sabr_lmm_anneal_plan* p, cudaStream_t s) {
  const DevMarket& m = p->mk->dm[0];
  const int C = p->opts.n_chains;
  const auto key = std::make_tuple(m.n_cap_pairs, m.NP, m.n_fwd, C);
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune_w_cache.find(key);
    if (it != g_tune_w_cache.end()) {
      p->W = it->second;
      p->grid = (C + p->W - 1) / p->W;
      CUDA_TRY(enqueue_anneal(m, p->opts.prec, p->st[0], p->sp[0], p->W, p->grid, s, true));
      return SABR_LMM_OK;
    }
  }
  std::vector<int> cand = {p->W, 28, 16, 14, 8, 7, 4};
  std::vector<int> uniq;
  for (int w : cand)
    if (w >= 4 && w <= 28 && smem_bytes<float>(m, w) <= 227u * 1024u &&
        std::find(uniq.begin(), uniq.end(), w) == uniq.end())
      uniq.push_back(w);
  // one level of the search's own length (at most 100 steps) per probe; a level of the benchmark's
  // 300-caplet market is ~0.7 ms.  Probes of 8 steps favoured CTA sizes that lose over the search.
  SAParams probe = p->sp[0];
  probe.L = 1;
  probe.N = std::min(probe.N, 100);
  cudaEvent_t a = nullptr, b = nullptr;
  CUDA_TRY(cudaEventCreate(&a));
  CUDA_TRY(cudaEventCreate(&b));
  float best_ms = 1e30f, first_ms = 0.f;
  int best = p->W;
  for (int w : uniq) {
    const int grid = (C + w - 1) / w;
    cudaError_t e = enqueue_anneal(m, p->opts.prec, p->st[0], probe, w, grid, s, true);
    float ms = 1e30f;
    for (int rep = 0; e == cudaSuccess && rep < 4; ++rep) {   // a warm-up, then the best of three
      if (e == cudaSuccess) e = cudaEventRecord(a, s);
      if (e == cudaSuccess) e = enqueue_anneal(m, p->opts.prec, p->st[0], probe, w, grid, s);
      if (e == cudaSuccess) e = cudaEventRecord(b, s);
      if (e == cudaSuccess) e = cudaEventSynchronize(b);
      float t = 0.f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&t, a, b);
      if (rep > 0 && t < ms) ms = t;
    }
    if (e != cudaSuccess) {
      cudaEventDestroy(a);
      cudaEventDestroy(b);
      return fail(SABR_LMM_ECUDA, std::string("tile autotuner: ") + cudaGetErrorString(e));
    }
    if (w == uniq[0]) first_ms = ms;
    if (ms < best_ms) { best_ms = ms; best = w; }
  }
  // the heuristic's choice (the first candidate) stays unless another is faster beyond timing noise
  if (best_ms > 0.98f * first_ms) best = uniq[0];
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  p->W = best;
  p->grid = (C + best - 1) / best;
  // the chosen kernel's attributes for the real launches
  CUDA_TRY(enqueue_anneal(m, p->opts.prec, p->st[0], p->sp[0], p->W, p->grid, s, true));
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune_w_cache[key] = best;
  return SABR_LMM_OK;
}

sabr_lmm_status enqueue_plan(sabr_lmm_anneal_plan* p, cudaStream_t s) {
  if (p->batch) {
    cudaError_t e = enqueue_batch(p, s, p->opts.n_levels);
    if (e != cudaSuccess) return fail(SABR_LMM_ECUDA, std::string("batch launch: ") + cudaGetErrorString(e));
    return SABR_LMM_OK;
  }
  const int nm = (int)p->mk->dm.size();
  for (int j = 0; j < nm; ++j) {
    cudaError_t e = enqueue_anneal(p->mk->dm[j], p->opts.prec, p->st[j], p->sp[j], p->W, p->grid, s, false,
                                   p->cta_warps);
    if (e != cudaSuccess) return fail(SABR_LMM_ECUDA, std::string("anneal launch: ") + cudaGetErrorString(e));
  }
  return SABR_LMM_OK;
}

// One market's start point (host, n_param values): finite, and inside the box on the free slots
// (fixed slots keep their given values).
sabr_lmm_status check_x0(const HostMarket& h, const double* x0) {
  for (int k = 0; k < h.n_param; ++k) {
    const double v = x0[k];
    if (!std::isfinite(v)) return fail(SABR_LMM_EINVAL, "x0 must be finite");
    if (h.freem[k] && (v < h.lo[k] || v > h.hi[k])) return fail(SABR_LMM_EINVAL, "x0 must lie in the box on the free slots");
  }
  return SABR_LMM_OK;
}

}  // namespace

extern "C" sabr_lmm_status sabr_lmm_anneal_prepare(const sabr_lmm_market* mk, const sabr_lmm_anneal_opts* o,
                                                   void* stream, sabr_lmm_anneal_plan** out) {
  if (!mk || !o || !out) return fail(SABR_LMM_EINVAL, "market, opts and out are required");
  *out = nullptr;
  if (o->n_chains < 1 || o->n_levels < 1 || o->steps_per_level < 1) return fail(SABR_LMM_EINVAL, "n_chains, n_levels, steps_per_level must be >= 1");
  if (!(o->cooling > 0.0 && o->cooling <= 1.0)) return fail(SABR_LMM_EINVAL, "cooling must be in (0, 1]");
  if (!(o->step_frac > 0.0) || !(o->step_floor >= 0.0)) return fail(SABR_LMM_EINVAL, "step_frac > 0 and step_floor >= 0 required");
  if (!valid_prec(o->prec)) return fail(SABR_LMM_EINVAL, "unknown precision");
  if (o->warps_per_block < 0 || o->warps_per_block > 28) return fail(SABR_LMM_EINVAL, "warps_per_block must be in [0, 28]");
  if (o->lm_top_k < 0 || o->lm_top_k > o->n_chains || o->lm_top_k > 1024) return fail(SABR_LMM_EINVAL, "lm_top_k must be in [0, min(n_chains, 1024)]");
  if (o->lm_top_k > 0 && o->lm_max_iter < 0) return fail(SABR_LMM_EINVAL, "lm_max_iter must be >= 0");
  if (o->polish_nm != 0 && o->polish_nm != 1) return fail(SABR_LMM_EINVAL, "polish_nm must be 0 or 1");
  for (const DevMarket& m : mk->dm) {
    if (o->lm_top_k > 0 && o->polish_nm && nm_smem(m) > 227u * 1024u)
      return fail(SABR_LMM_ENOTSUP, "a market and the Nelder-Mead simplex do not fit one CTA");
    if (o->lm_top_k > 0 && !o->polish_nm && (m.n_param > kMaxGradParam || m.model == SABR_LMM_MODEL_MERCURIO_MORINI))
      return fail(SABR_LMM_ENOTSUP, "the Levenberg-Marquardt polish covers the smile and Rebonato models, at most 12 "
                                    "parameter slots (polish_nm = 1 runs Nelder-Mead instead)");
  }
  for (size_t j = 0; o->x0 && j < mk->dm.size(); ++j)
    if (sabr_lmm_status st = check_x0(mk->hm[j], o->x0 + j * (size_t)mk->hm[j].n_param); st != SABR_LMM_OK) return st;
  for (const DevMarket& m : mk->dm) {
    if (market_smem(m, o->prec) > 227 * 1024)
      return fail(SABR_LMM_ENOTSUP, "a market does not fit in one CTA's shared memory at this precision");
    if (m.n_swp > 0 && o->prec == SABR_LMM_FP32_BF16X3 && (!tc_eligible(m) || mk->dm.size() > 1))
      return fail(SABR_LMM_ENOTSUP, "the tensor-core contraction needs a single market whose panel tables fit one tile");
  }
  sabr_lmm_anneal_plan* p = new sabr_lmm_anneal_plan();
  p->mk = mk;
  p->opts = *o;
  p->opts.x0 = nullptr;
  // chains (warps) per CTA: FP32 one CTA per SM with up to 28 chains, as many as spread the chains
  // over the SMs in one wave; FP64 (128 registers a thread) 4 chains per CTA
  int nsm = 148;
  {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  }
  p->W = o->warps_per_block > 0 ? o->warps_per_block
                                : (o->prec == SABR_LMM_FP64 ? 4 : std::min(28, std::max(1, (o->n_chains + nsm - 1) / nsm)));
  if (o->prec == SABR_LMM_FP64 && p->W > 4) p->W = 4;
  // fewer chains per CTA if a caplet market's shared memory would not fit (the 4-chain form is
  // what the load-time check admits)
  for (const DevMarket& m : mk->dm)
    if (m.n_swp == 0 && o->prec != SABR_LMM_FP64)
      while (p->W > 4 && smem_bytes<float>(m, p->W) > 227u * 1024u) --p->W;
  p->grid = (o->n_chains + p->W - 1) / p->W;
  p->cta_warps = cta_warps_of(o);
  const int nm = (int)mk->dm.size();
  const int P = mk->dm[0].n_param;
  const size_t C = o->n_chains, L = o->n_levels, N = o->steps_per_level;
  // per market: xs[P] fs T0 xe[CP] fe[C] xb[CP] fb[C] part_f[grid] part_c[grid] counter trace[L] best_x[P] best_f x0[P]
  Arena A;
  struct Off { size_t xs, fs, T0, lvl, xe, fe, xb, fb, pf, pc, cnt, tr, trx, trt, bx, bf, x0, bits, vols, rmse; };
  std::vector<Off> off(nm);
  for (int j = 0; j < nm; ++j) {
    const int Pj = mk->dm[j].n_param;
    Off& q = off[j];
    q.xs = A.take(Pj * 8); q.fs = A.take(8); q.T0 = A.take(8); q.lvl = A.take(3 * 8);
    q.xe = A.take(C * Pj * 8); q.fe = A.take(C * 8); q.xb = A.take(C * Pj * 8); q.fb = A.take(C * 8);
    const size_t nparts = std::max<size_t>((size_t)p->grid, C);   // CTA minima (one CTA per chain with swaptions)
    q.pf = A.take(nparts * 8); q.pc = A.take(nparts * 4); q.cnt = A.take(16);
    q.tr = A.take(L * 8); q.trx = A.take(L * Pj * 8); q.trt = A.take((L + 1) * 8);
    q.bx = A.take(Pj * 8); q.bf = A.take(8); q.x0 = A.take(Pj * 8);
    q.bits = (j == 0 && o->record_accepts) ? A.take(C * L * N) : 0;
    size_t max_ni = 1;   // the RMSE of every market's best point reuses market 0's buffer
    for (const DevMarket& mm : mk->dm) max_ni = std::max<size_t>(max_ni, (size_t)(mm.n_cap + mm.n_swp));
    q.vols = A.take(max_ni * 8);
    q.rmse = A.take(8);
  }
  if (cudaMalloc(&p->state, A.size) != cudaSuccess) { delete p; return fail(SABR_LMM_ENOMEM, "cudaMalloc of the chain state failed"); }
  char* b = (char*)p->state;
  p->x0.resize((size_t)nm * P);
  for (int j = 0; j < nm; ++j) {
    const DevMarket& m = mk->dm[j];
    const HostMarket& h = mk->hm[j];
    const Off& q = off[j];
    SAState s{};
    s.xs = (double*)(b + q.xs); s.fs = (double*)(b + q.fs); s.T0 = (double*)(b + q.T0); s.lvl = (double*)(b + q.lvl);
    s.xe = (double*)(b + q.xe); s.fe = (double*)(b + q.fe); s.xb = (double*)(b + q.xb); s.fb = (double*)(b + q.fb);
    s.part_f = (double*)(b + q.pf); s.part_c = (int*)(b + q.pc); s.counter = (unsigned int*)(b + q.cnt);
    s.trace_f = (double*)(b + q.tr); s.best_x = (double*)(b + q.bx); s.best_f = (double*)(b + q.bf);
    s.trace_x = (double*)(b + q.trx); s.trace_t = (unsigned long long*)(b + q.trt);
    s.bits = (j == 0 && o->record_accepts) ? (uint8_t*)(b + q.bits) : nullptr;
    p->st.push_back(s);
    SAParams sp{};
    sp.C = o->n_chains; sp.L = o->n_levels; sp.N = o->steps_per_level; sp.P = m.n_param;
    sp.cooling = o->cooling; sp.step_frac = o->step_frac; sp.step_floor = o->step_floor; sp.T0_opt = o->T0;
    sp.seed = o->seed; sp.market_index = (unsigned long long)j;
    sp.x0 = (const double*)(b + q.x0);
    p->sp.push_back(sp);
    for (int k = 0; k < m.n_param; ++k)
      p->x0[(size_t)j * P + k] = o->x0 ? o->x0[(size_t)j * m.n_param + k] : 0.5 * (h.lo[k] + h.hi[k]);
  }
  p->vols_dev = (double*)(b + off[0].vols);
  p->rmse_dev = (double*)(b + off[0].rmse);
  p->stream = (cudaStream_t)stream;
  if (!p->stream && o->use_graph) {
    cudaStreamCreateWithFlags(&p->stream, cudaStreamNonBlocking);
    p->own_stream = true;
  }
  cudaEventCreate(&p->ev0);
  cudaEventCreate(&p->ev1);
  cudaEventCreate(&p->ev2);
  // batch mode: several Rebonato markets of one formula, one persistent launch per level
  bool batchable = nm > 1;
  for (const DevMarket& m : mk->dm)
    batchable = batchable && m.model == SABR_LMM_MODEL_REBONATO && m.formula == mk->dm[0].formula;
  if (batchable) {
    p->batch = true;
    uint32_t smax = 0;
    // buckets by the CTAs per SM each market's shared memory allows; LPT order inside a bucket
    std::map<int, std::vector<std::pair<long long, int>>, std::greater<int>> buckets;
    std::map<int, uint32_t> bsm;
    for (int j = 0; j < nm; ++j) {
      const DevMarket& m = mk->dm[j];
      const uint32_t sm = o->prec == SABR_LMM_FP64 ? smem_bytes_cta<double>(m) : smem_bytes_cta<float>(m);
      if (sm > 227 * 1024) { sabr_lmm_anneal_plan_free(p); return fail(SABR_LMM_ENOTSUP, "a batch market does not fit in one CTA's shared memory at this precision"); }
      smax = std::max(smax, sm);
      // keyed at 128 threads (1-4 CTAs per SM; at 256 the registers cap every market at 2)
      const int per_sm = batch_blocks_per_sm(o->prec, 128, sm);
      if (per_sm < 1) { sabr_lmm_anneal_plan_free(p); return fail(SABR_LMM_ENOTSUP, "a batch market does not fit in one CTA's shared memory at this precision"); }
      buckets[per_sm].push_back({-(long long)(m.n_cap + 4 * m.n_swp + 60 * m.n_swap), j});
      bsm[per_sm] = std::max(bsm[per_sm], sm);
    }
    p->bsmem = smax;
    std::vector<int> order;
    for (auto& kv : buckets) {
      std::sort(kv.second.begin(), kv.second.end());
      sabr_lmm_anneal_plan::Bucket b;
      b.per_sm = kv.first;
      b.smem = bsm[kv.first];
      b.ba.n_markets = (int)kv.second.size();
      for (auto& c : kv.second) { order.push_back(c.second); b.markets.push_back(c.second); }
      p->bk.push_back(b);
    }
    const int nb = (int)p->bk.size();
    Arena B;
    const size_t o_mk = B.take(nm * sizeof(DevMarket)), o_st = B.take(nm * sizeof(SAState)),
                 o_sp = B.take(nm * sizeof(SAParams)), o_or = B.take(nm * sizeof(int)),
                 o_ct = B.take((size_t)nb * o->n_levels * sizeof(unsigned int));
    if (cudaMalloc(&p->batch_buf, B.size) != cudaSuccess) { sabr_lmm_anneal_plan_free(p); return fail(SABR_LMM_ENOMEM, "cudaMalloc of the batch tables failed"); }
    char* bb = (char*)p->batch_buf;
    p->ba.mk = (const DevMarket*)(bb + o_mk);
    p->ba.st = (const SAState*)(bb + o_st);
    p->ba.sp = (const SAParams*)(bb + o_sp);
    p->ba.order = (const int*)(bb + o_or);
    p->ba.item_ctr = (unsigned int*)(bb + o_ct);
    p->ba.n_markets = nm;
    p->ba.C = o->n_chains;
    int first = 0;
    for (int i = 0; i < nb; ++i) {
      BatchArgs& a = p->bk[i].ba;
      const int n = a.n_markets;
      a = p->ba;
      a.n_markets = n;
      a.order = p->ba.order + first;
      a.item_ctr = p->ba.item_ctr + (size_t)i * o->n_levels;
      first += n;
    }
    cudaMemcpyAsync(bb + o_mk, mk->dm.data(), nm * sizeof(DevMarket), cudaMemcpyHostToDevice, p->stream);
    cudaMemcpyAsync(bb + o_st, p->st.data(), nm * sizeof(SAState), cudaMemcpyHostToDevice, p->stream);
    cudaMemcpyAsync(bb + o_sp, p->sp.data(), nm * sizeof(SAParams), cudaMemcpyHostToDevice, p->stream);
    cudaMemcpyAsync(bb + o_or, order.data(), nm * sizeof(int), cudaMemcpyHostToDevice, p->stream);
  }
  if (o->lm_top_k > 0) {
    Arena B;
    for (int j = 0; j < nm; ++j) {
      const int k = o->lm_top_k, Pj = mk->dm[j].n_param;
      p->lm_off.push_back(B.take((size_t)k * Pj * 8));          // points
      p->lm_off.push_back(B.take((size_t)k * 4));               // selected chains
      p->lm_off.push_back(B.take(lm_work_bytes(mk->dm[j], k)));  // LM work
    }
    if (cudaMalloc(&p->lm_buf, B.size) != cudaSuccess) { sabr_lmm_anneal_plan_free(p); return fail(SABR_LMM_ENOMEM, "cudaMalloc of the polish buffers failed"); }
    LmSide side;   // the polish's side stream, made here rather than inside a timed launch
    if (cudaError_t e = lm_side(side); e != cudaSuccess) {
      sabr_lmm_anneal_plan_free(p);
      return fail(SABR_LMM_ECUDA, std::string("polish side stream: ") + cudaGetErrorString(e));
    }
  }
  for (int j = 0; j < nm && !p->batch; ++j) {
    cudaError_t e = enqueue_anneal(mk->dm[j], o->prec, p->st[j], p->sp[j], p->W, p->grid, p->stream, true,
                                   p->cta_warps);
    if (e != cudaSuccess) { sabr_lmm_anneal_plan_free(p); return fail(SABR_LMM_ECUDA, std::string("configure: ") + cudaGetErrorString(e)); }
  }
  if (p->batch) {
    cudaError_t e = enqueue_batch(p, p->stream, 0, true);
    if (e != cudaSuccess) { sabr_lmm_anneal_plan_free(p); return fail(SABR_LMM_ECUDA, std::string("configure: ") + cudaGetErrorString(e)); }
  }
  for (int j = 0; j < nm; ++j) {
    cudaError_t e = cudaMemcpyAsync((void*)p->sp[j].x0, p->x0.data() + (size_t)j * P, mk->dm[j].n_param * 8,
                                    cudaMemcpyHostToDevice, p->stream);
    if (e != cudaSuccess) { sabr_lmm_anneal_plan_free(p); return fail(SABR_LMM_ECUDA, cudaGetErrorString(e)); }
  }
  cudaError_t e = cudaStreamSynchronize(p->stream);
  if (e != cudaSuccess) { sabr_lmm_anneal_plan_free(p); return fail(SABR_LMM_ECUDA, cudaGetErrorString(e)); }
  if (p->batch) {
    if (o->warps_per_block > 0) {
      int dev = 0, nsm = 148;
      cudaGetDevice(&dev);
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
      for (auto& b : p->bk) {
        b.threads = o->warps_per_block >= 8 ? 256 : 128;
        b.grid = nsm * std::max(batch_blocks_per_sm(o->prec, b.threads, b.smem), 1);
      }
    } else {
      sabr_lmm_status st = tune_batch(p, p->stream);
      if (st != SABR_LMM_OK) { sabr_lmm_anneal_plan_free(p); return st; }
    }
  } else if (nm == 1 && mk->dm[0].n_swp == 0 && o->prec == SABR_LMM_FP32 && o->warps_per_block == 0) {
    sabr_lmm_status st = tune_caplet_w(p, p->stream);
    if (st != SABR_LMM_OK) { sabr_lmm_anneal_plan_free(p); return st; }
  }
  *out = p;
  return SABR_LMM_OK;
}

namespace {
// The polish of the lm_top_k lowest best-ever chain points of every market, after the search.
sabr_lmm_status enqueue_polish(sabr_lmm_anneal_plan* p, cudaStream_t s) {
  const int k = p->opts.lm_top_k;
  char* b = (char*)p->lm_buf;
  for (size_t j = 0; j < p->mk->dm.size(); ++j) {
    const DevMarket& m = p->mk->dm[j];
    double* X = (double*)(b + p->lm_off[3 * j]);
    int* sel = (int*)(b + p->lm_off[3 * j + 1]);
    const LmWork w = lm_carve(b + p->lm_off[3 * j + 2], m, k);
    select_lowest_kernel<<<1, 1024, 0, s>>>(p->st[j].fb, p->opts.n_chains, k, sel);
    gather_points_kernel<<<k, 32, 0, s>>>(p->st[j].xb, sel, k, m.n_param, X);
    int n_free = 0;
    for (unsigned char f : p->mk->hm[j].freem) n_free += f != 0;
    cudaError_t e = p->opts.polish_nm ? launch_nm(m, X, k, p->opts.lm_max_iter, 0.02, 1e-12, w.f, nullptr, s)
                                      : lm_enqueue(m, n_free, X, k, p->opts.lm_max_iter, p->opts.target_rmse_volpt, w, s, true);
    if (e != cudaSuccess) return fail(SABR_LMM_ECUDA, std::string("polish launch: ") + cudaGetErrorString(e));
    take_best_kernel<<<1, 32, 0, s>>>(X, w.f, k, m.n_param, p->st[j].best_x, p->st[j].best_f);
  }
  CUDA_TRY(cudaGetLastError());
  return SABR_LMM_OK;
}
}  // namespace

extern "C" sabr_lmm_status sabr_lmm_anneal_launch(sabr_lmm_anneal_plan* p, void* stream) {
  if (!p) return fail(SABR_LMM_EINVAL, "plan is NULL");
  cudaStream_t s = stream ? (cudaStream_t)stream : p->stream;
  if (p->opts.use_graph) {
    if (!s) return fail(SABR_LMM_EINVAL, "graph replay needs a non-default stream");
    if (!p->gexec) {
      cudaGraph_t g = nullptr;
      CUDA_TRY(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
      sabr_lmm_status st = enqueue_plan(p, s);
      cudaError_t e = cudaStreamEndCapture(s, &g);
      if (st != SABR_LMM_OK) { if (g) cudaGraphDestroy(g); return st; }
      if (e != cudaSuccess) return fail(SABR_LMM_ECUDA, std::string("capture: ") + cudaGetErrorString(e));
      e = cudaGraphInstantiate(&p->gexec, g, 0);
      cudaGraphDestroy(g);
      if (e != cudaSuccess) return fail(SABR_LMM_ECUDA, std::string("instantiate: ") + cudaGetErrorString(e));
    }
    CUDA_TRY(cudaEventRecord(p->ev0, s));
    CUDA_TRY(cudaGraphLaunch(p->gexec, s));
    CUDA_TRY(cudaEventRecord(p->ev1, s));
  } else {
    CUDA_TRY(cudaEventRecord(p->ev0, s));
    sabr_lmm_status st = enqueue_plan(p, s);
    if (st != SABR_LMM_OK) return st;
    CUDA_TRY(cudaEventRecord(p->ev1, s));
  }
  if (p->opts.lm_top_k > 0) {
    sabr_lmm_status st = enqueue_polish(p, s);
    if (st != SABR_LMM_OK) return st;
  }
  CUDA_TRY(cudaEventRecord(p->ev2, s));
  p->stream = s;
  return SABR_LMM_OK;
}

namespace {
// Read and clear the error word of every market of mk after `s` has been synchronised: a raised
// word (a bounded device-side wait gave up since the last read) is reported once, as ETIMEOUT.
sabr_lmm_status take_error_words(const sabr_lmm_market* mk, cudaStream_t s) {
  int err = 0;
  for (const DevMarket& m : mk->dm) {
    int e = 0;
    CUDA_TRY(cudaMemcpyAsync(&e, m.err, sizeof(int), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    if (e) CUDA_TRY(cudaMemsetAsync(m.err, 0, sizeof(int), s));
    err |= e;
  }
  CUDA_TRY(cudaStreamSynchronize(s));
  if (err) return fail(SABR_LMM_ETIMEOUT, "a bounded device-side wait gave up (outputs of the affected calls are NaN)");
  return SABR_LMM_OK;
}
}  // namespace

extern "C" sabr_lmm_status sabr_lmm_sync(const sabr_lmm_market* m, void* stream) {
  if (!m) return fail(SABR_LMM_EINVAL, "market is NULL");
  CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
  return take_error_words(m, (cudaStream_t)stream);
}

extern "C" sabr_lmm_status sabr_lmm_test_raise_error(const sabr_lmm_market* m, int32_t idx, void* stream) {
  if (!m) return fail(SABR_LMM_EINVAL, "market is NULL");
  if (idx < 0 || idx >= (int)m->dm.size()) return fail(SABR_LMM_EINVAL, "market_idx out of range");
  CUDA_TRY(cudaMemsetAsync(m->dm[idx].err, 0x01, 1, (cudaStream_t)stream));
  return SABR_LMM_OK;
}

extern "C" sabr_lmm_status sabr_lmm_anneal_fetch(sabr_lmm_anneal_plan* p, sabr_lmm_result* out) {
  if (!p || !out) return fail(SABR_LMM_EINVAL, "plan and out are required");
  cudaStream_t s = p->stream;
  CUDA_TRY(cudaStreamSynchronize(s));
  const sabr_lmm_market* mk = p->mk;
  const int nm = (int)mk->dm.size();
  if (sabr_lmm_status st = take_error_words(mk, s); st != SABR_LMM_OK) return st;
  float ms = 0.f;
  cudaEventElapsedTime(&ms, p->ev0, p->ev1);
  out->seconds = ms * 1e-3;
  float ms2 = 0.f;
  cudaEventElapsedTime(&ms2, p->ev1, p->ev2);
  out->lm_seconds = p->opts.lm_top_k > 0 ? ms2 * 1e-3 : 0.0;
  out->n_evals = (int64_t)p->opts.n_chains * ((int64_t)p->opts.n_levels * p->opts.steps_per_level + 1);
  for (int j = 0; j < nm; ++j) {
    const DevMarket& m = mk->dm[j];
    const int Pj = m.n_param;
    if (out->x_best) CUDA_TRY(cudaMemcpy(out->x_best + (size_t)j * Pj, p->st[j].best_x, Pj * 8, cudaMemcpyDeviceToHost));
    if (out->f_best) CUDA_TRY(cudaMemcpy(out->f_best + j, p->st[j].best_f, 8, cudaMemcpyDeviceToHost));
    const size_t L = p->opts.n_levels;
    if (out->trace_f)
      CUDA_TRY(cudaMemcpy(out->trace_f + (size_t)j * L, p->st[j].trace_f, L * 8, cudaMemcpyDeviceToHost));
    if (out->trace_x)
      CUDA_TRY(cudaMemcpy(out->trace_x + (size_t)j * L * Pj, p->st[j].trace_x, L * Pj * 8, cudaMemcpyDeviceToHost));
    if (out->trace_seconds) {
      std::vector<unsigned long long> t(L + 1);
      CUDA_TRY(cudaMemcpy(t.data(), p->st[j].trace_t, (L + 1) * 8, cudaMemcpyDeviceToHost));
      for (size_t l = 0; l < L; ++l) out->trace_seconds[(size_t)j * L + l] = (double)(t[l + 1] - t[0]) * 1e-9;
    }
    if (j == 0) CUDA_TRY(cudaMemcpy(&out->T0_used, p->st[0].T0, 8, cudaMemcpyDeviceToHost));
    if (out->rmse_volpt) {
      CUDA_TRY(launch_objective_any(m, SABR_LMM_FP64, p->st[j].best_x, 1, nullptr, p->vols_dev, s));
      rmse_from_vols_kernel<<<1, 256, 0, s>>>(p->vols_dev, m.cap_vol, m.swp_vol, m.n_cap, m.n_swp, p->rmse_dev);
      CUDA_TRY(cudaGetLastError());
      CUDA_TRY(cudaMemcpyAsync(out->rmse_volpt + j, p->rmse_dev, 8, cudaMemcpyDeviceToHost, s));
      CUDA_TRY(cudaStreamSynchronize(s));
    }
  }
  if (out->accept_bits && p->st[0].bits)
    CUDA_TRY(cudaMemcpy(out->accept_bits, p->st[0].bits,
                        (size_t)p->opts.n_chains * p->opts.n_levels * p->opts.steps_per_level, cudaMemcpyDeviceToHost));
  return SABR_LMM_OK;
}

extern "C" sabr_lmm_status sabr_lmm_anneal_plan_config(const sabr_lmm_anneal_plan* p, sabr_lmm_plan_config* out) {
  if (!p || !out) return fail(SABR_LMM_EINVAL, "plan and out are required");
  std::memset(out, 0, sizeof *out);
  out->chains_per_cta = p->W;
  out->grid = p->grid;
  out->cta_threads_swaptions = 32 * p->cta_warps;
  out->n_buckets = p->batch ? (int)std::min<size_t>(p->bk.size(), 16) : 0;
  for (int i = 0; i < out->n_buckets; ++i) {
    out->bucket_markets[i] = p->bk[i].ba.n_markets;
    out->bucket_threads[i] = p->bk[i].threads;
    out->bucket_grid[i] = p->bk[i].grid;
    out->bucket_ctas_per_sm[i] = p->bk[i].per_sm;
  }
  return SABR_LMM_OK;
}

extern "C" void sabr_lmm_anneal_plan_free(sabr_lmm_anneal_plan* p) {
  if (!p) return;
  if (p->gexec) cudaGraphExecDestroy(p->gexec);
  if (p->ev0) cudaEventDestroy(p->ev0);
  if (p->ev1) cudaEventDestroy(p->ev1);
  if (p->ev2) cudaEventDestroy(p->ev2);
  if (p->lm_buf) cudaFree(p->lm_buf);
  if (p->batch_buf) cudaFree(p->batch_buf);
  if (p->own_stream && p->stream) cudaStreamDestroy(p->stream);
  if (p->state) cudaFree(p->state);
  delete p;
}

extern "C" sabr_lmm_status sabr_lmm_anneal(const sabr_lmm_market* mk, const sabr_lmm_anneal_opts* o, sabr_lmm_result* out) {
  if (!out) return fail(SABR_LMM_EINVAL, "out is required");
  sabr_lmm_anneal_plan* p = nullptr;
  sabr_lmm_status st = sabr_lmm_anneal_prepare(mk, o, nullptr, &p);
  if (st != SABR_LMM_OK) return st;
  st = sabr_lmm_anneal_launch(p, nullptr);
  if (st == SABR_LMM_OK) st = sabr_lmm_anneal_fetch(p, out);
  sabr_lmm_anneal_plan_free(p);
  return st;
}

extern "C" sabr_lmm_status sabr_lmm_market_info(const sabr_lmm_market* m, int32_t idx, sabr_lmm_market_info_t* out) {
  if (!m || !out) return fail(SABR_LMM_EINVAL, "market and out are required");
  if (idx < 0 || idx >= (int)m->dm.size()) return fail(SABR_LMM_EINVAL, "market_idx out of range");
  const DevMarket& d = m->dm[idx];
  out->n_fwd = d.n_fwd;
  out->n_cap = d.n_cap;
  out->n_swp = d.n_swp;
  out->n_swap = d.n_swap;
  out->n_panels = d.NA;
  out->n_diag = d.ND;
  out->max_window = d.max_gwin;
  out->smem_fp64 = market_smem(d, SABR_LMM_FP64);
  out->smem_fp32 = market_smem(d, SABR_LMM_FP32);
  auto per_sm = [&](int prec, uint32_t sm) {
    if (d.model != SABR_LMM_MODEL_REBONATO || sm > 227u * 1024u) return 0;
    return std::max(0, batch_blocks_per_sm(prec, 256, prec == SABR_LMM_FP64 ? smem_bytes_cta<double>(d)
                                                                              : smem_bytes_cta<float>(d)));
  };
  out->batch_ctas_per_sm_fp64 = per_sm(SABR_LMM_FP64, out->smem_fp64);
  out->batch_ctas_per_sm_fp32 = per_sm(SABR_LMM_FP32, out->smem_fp32);
  CUDA_TRY(cudaGetLastError());
  return SABR_LMM_OK;
}

extern "C" sabr_lmm_status sabr_lmm_selftest_wait(int64_t polls, void* stream) {
  if (polls < 1 || polls > kWaitLimit) return fail(SABR_LMM_EINVAL, "polls must be in [1, 2^24]");
  int* err = nullptr;
  CUDA_TRY(cudaMalloc(&err, sizeof(int)));
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaMemsetAsync(err, 0, sizeof(int), s);
  if (e == cudaSuccess) {
    wait_selftest_kernel<<<1, 64, 0, s>>>(err, (long long)polls);
    e = cudaGetLastError();
  }
  int h = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(err);
  if (e != cudaSuccess) return fail(SABR_LMM_ECUDA, std::string("selftest_wait: ") + cudaGetErrorString(e));
  if (h) return fail(SABR_LMM_ETIMEOUT, "a bounded device-side wait gave up (the self-test's expected outcome)");
  return SABR_LMM_OK;
}

extern "C" sabr_lmm_status sabr_lmm_quadrature_rule(int32_t q, double* x, double* w) {
  if (q != 8 || !x || !w) return fail(SABR_LMM_EINVAL, "q must be 8 and x, w non-NULL");
  for (int i = 0; i < 8; ++i) { x[i] = kGLx[i]; w[i] = kGLw[i]; }
  return SABR_LMM_OK;
}

extern "C" const char* sabr_lmm_last_error(void) { return g_err.c_str(); }
extern "C" const char* sabr_lmm_version(void) { return "sabr_lmm 0.1 (sm_103a)"; }

// ====================================================================== annealing without allocation
// sabr_lmm_anneal_noalloc runs the same kernels as sabr_lmm_anneal, but keeps every byte of the
// search's working state in one fixed-size array that lives in the library's own device image
// (allocated when the library's module is loaded on a device, held until the process exits).  It
// never calls cudaMalloc or cudaFree, so a caller that must not allocate can still anneal.
namespace {

constexpr int kNoAllocMaxChains = 16384;
constexpr int kNoAllocMaxLevels = 4096;
constexpr int kNoAllocMaxParam = kMaxGradParam;
constexpr int kNoAllocW = 4;  // warps (chains) per CTA: the 4-chain form of the caplet level kernel
// level-minimum slots: one per CTA of the caplet kernel, one per chain for markets with swaptions
constexpr int kNoAllocMaxParts = kNoAllocMaxChains;

// Byte offsets of the regions in the array (each 256-byte aligned).
constexpr size_t kNaHead = 0;  // xs[12] fs T0 x0[12] best_x[12] best_f counter lvl[3]
constexpr size_t kNaXe = 512;
constexpr size_t kNaFe = kNaXe + (size_t)kNoAllocMaxChains * kNoAllocMaxParam * 8;
constexpr size_t kNaXb = kNaFe + (size_t)kNoAllocMaxChains * 8;
constexpr size_t kNaFb = kNaXb + (size_t)kNoAllocMaxChains * kNoAllocMaxParam * 8;
constexpr size_t kNaPf = kNaFb + (size_t)kNoAllocMaxChains * 8;
constexpr size_t kNaPc = kNaPf + (size_t)kNoAllocMaxParts * 8;
constexpr size_t kNaTr = kNaPc + (size_t)kNoAllocMaxParts * 4;
constexpr size_t kNaBytes = kNaTr + (size_t)kNoAllocMaxLevels * 8;   // 3,637,760 B (3.64 MB)
static_assert(kNaBytes == 3637760, "the size quoted in sabr_lmm.h");

// The start point travels as a kernel argument (no host copy is enqueued).
struct NoAllocX0 { double v[kNoAllocMaxParam]; };
__global__ void noalloc_put_x0_kernel(double* dst, NoAllocX0 x0, int P) {
  if ((int)threadIdx.x < P) dst[threadIdx.x] = x0.v[threadIdx.x];
}

__device__ __align__(256) unsigned char g_noalloc_scratch[kNaBytes];

std::mutex g_noalloc_mu;
std::map<int, unsigned char*> g_noalloc_addr;   // device ordinal -> device address of the array

// The device address of the array on the current device, looked up once per device.  In host
// code `g_noalloc_scratch` is only a stand-in symbol; a kernel must be given this address.
sabr_lmm_status noalloc_scratch(unsigned char** out) {
  int dev = 0;
  CUDA_TRY(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  auto it = g_noalloc_addr.find(dev);
  if (it == g_noalloc_addr.end()) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr)
      return fail(SABR_LMM_ECUDA, std::string("cudaGetSymbolAddress of the static scratch: ") + cudaGetErrorString(e));
    it = g_noalloc_addr.emplace(dev, (unsigned char*)p).first;
  }
  *out = it->second;
  return SABR_LMM_OK;
}

}  // namespace

extern "C" sabr_lmm_status sabr_lmm_anneal_noalloc(const sabr_lmm_market* mk, int32_t market_idx,
                                                   const sabr_lmm_anneal_opts* o, double* x_best, double* f_best,
                                                   double* trace_f, void* stream) {
  if (!mk || !o || !x_best || !f_best) return fail(SABR_LMM_EINVAL, "market, opts, x_best and f_best are required");
  if (market_idx < 0 || market_idx >= (int)mk->dm.size()) return fail(SABR_LMM_EINVAL, "market_idx out of range");
  if (o->n_chains < 1 || o->n_levels < 1 || o->steps_per_level < 1)
    return fail(SABR_LMM_EINVAL, "n_chains, n_levels, steps_per_level must be >= 1");
  if (o->n_chains > kNoAllocMaxChains || o->n_levels > kNoAllocMaxLevels) {
    char buf[200];
    snprintf(buf, sizeof buf, "anneal_noalloc: %d chains x %d levels exceeds the static scratch limit of %d chains x %d levels",
             o->n_chains, o->n_levels, kNoAllocMaxChains, kNoAllocMaxLevels);
    return fail(SABR_LMM_EINVAL, buf);
  }
  if (!(o->cooling > 0.0 && o->cooling <= 1.0)) return fail(SABR_LMM_EINVAL, "cooling must be in (0, 1]");
  if (!(o->step_frac > 0.0) || !(o->step_floor >= 0.0)) return fail(SABR_LMM_EINVAL, "step_frac > 0 and step_floor >= 0 required");
  if (!valid_prec(o->prec)) return fail(SABR_LMM_EINVAL, "unknown precision");
  if (o->lm_top_k > 0 || o->record_accepts) return fail(SABR_LMM_EINVAL, "anneal_noalloc supports neither the polish nor accept records");
  if (sabr_lmm_status st = check_call(mk, market_idx, 0, o->prec); st != SABR_LMM_OK) return st;
  const DevMarket& m = mk->dm[market_idx];
  const HostMarket& h = mk->hm[market_idx];
  if (m.n_param > kNoAllocMaxParam)
    return fail(SABR_LMM_ENOTSUP, "anneal_noalloc takes markets of at most 12 parameter slots");
  if (o->x0)
    if (sabr_lmm_status st = check_x0(h, o->x0); st != SABR_LMM_OK) return st;
  const int P = m.n_param;
  unsigned char* base = nullptr;
  sabr_lmm_status st0 = noalloc_scratch(&base);
  if (st0 != SABR_LMM_OK) return st0;
  cudaStream_t s = (cudaStream_t)stream;
  double* head = (double*)(base + kNaHead);
  SAState st{};
  st.xs = head;
  st.fs = head + 12;
  st.T0 = head + 13;
  double* x0 = head + 14;
  st.best_x = head + 26;
  st.best_f = head + 38;
  st.counter = (unsigned int*)(head + 39);
  st.lvl = head + 40;
  st.xe = (double*)(base + kNaXe);
  st.fe = (double*)(base + kNaFe);
  st.xb = (double*)(base + kNaXb);
  st.fb = (double*)(base + kNaFb);
  st.part_f = (double*)(base + kNaPf);
  st.part_c = (int*)(base + kNaPc);
  st.trace_f = (double*)(base + kNaTr);
  st.bits = nullptr;
  SAParams sp{};
  sp.C = o->n_chains; sp.L = o->n_levels; sp.N = o->steps_per_level; sp.P = P;
  sp.cooling = o->cooling; sp.step_frac = o->step_frac; sp.step_floor = o->step_floor; sp.T0_opt = o->T0;
  sp.seed = o->seed; sp.market_index = (unsigned long long)market_idx;
  sp.x0 = x0;
  NoAllocX0 hx0{};
  for (int k = 0; k < P; ++k) hx0.v[k] = o->x0 ? o->x0[k] : 0.5 * (h.lo[k] + h.hi[k]);
  // every value the kernels read before writing is set here or by the start kernel (f(x0), T0,
  // the first start point and the level counter), so the previous call's contents do not leak in
  noalloc_put_x0_kernel<<<1, 32, 0, s>>>(x0, hx0, P);
  CUDA_TRY(cudaGetLastError());
  const int grid = (o->n_chains + kNoAllocW - 1) / kNoAllocW;
  CUDA_TRY(enqueue_anneal(m, o->prec, st, sp, kNoAllocW, grid, s, true, cta_warps_of(o)));
  CUDA_TRY(enqueue_anneal(m, o->prec, st, sp, kNoAllocW, grid, s, false, cta_warps_of(o)));
  CUDA_TRY(cudaMemcpyAsync(x_best, st.best_x, P * sizeof(double), cudaMemcpyDeviceToDevice, s));
  CUDA_TRY(cudaMemcpyAsync(f_best, st.best_f, sizeof(double), cudaMemcpyDeviceToDevice, s));
  if (trace_f) CUDA_TRY(cudaMemcpyAsync(trace_f, st.trace_f, o->n_levels * sizeof(double), cudaMemcpyDeviceToDevice, s));
  return SABR_LMM_OK;
}

#include "mc_api.cuh"
