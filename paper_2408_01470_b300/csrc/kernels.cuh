// Kernels of the hot path and of market set-up.
//
//   setup_*_kernel ......... market-only constants in FP64 (once per load), the FP32 pair-major
//                            caplet block and the swaptions' coefficient rows.
//   objective_kernel ....... f (or the model vols) for n parameter sets, one warp per set
//                            (grid-stride); caplet markets.
//   sa_start_kernel ........ f(x0), T0, the first start point.
//   sa_level_kernel ........ one temperature level: every chain (one warp) runs N Metropolis
//                            steps (S1 proposal, S2-S7 objective, S8 acceptance), then the
//                            minimum over the chains' end points is taken by the last CTA to
//                            finish (no grid-wide wait) and becomes the next start point.  CTAs
//                            of 4 chains, or (FP32) one CTA of up to 28 chains per SM.
//   sa_final_kernel ........ the best point ever accepted over all chains.
//   *_cta_kernel ........... the same for markets with swaptions, one CTA (256 threads) per
//                            chain or per point (cta_objective in swaption.cuh).
//   *_batch_kernel ......... many markets: per level a persistent grid over (market, chain)
//                            items in LPT order.
//   grad_kernel ............ f and df/dtheta by the reverse sweep (adjoint.cuh), caplet markets.
//   grad_cta_kernel ........ the same for markets with swaptions, one CTA per point, FP64
//                            (adjoint_swaption.cuh).
//   nm_kernel, nm_cta_kernel  Nelder-Mead from n points (nelder_mead.cuh), one warp / CTA each.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>
#include "device_math.cuh"
#include "market.cuh"
#include "objective.cuh"
#include "swaption.cuh"
#include "adjoint.cuh"
#include "adjoint_swaption.cuh"
#include "nelder_mead.cuh"

namespace sabr {

// ------------------------------------------------------------------ market set-up (FP64)
__global__ void setup_forwards_kernel(DevMarket m) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < m.n_fwd) {
    const double tau = m.T[i + 1] - m.T[i];
    const double F = (m.P[i] / m.P[i + 1] - 1.0) / tau;
    m.tau[i] = tau;
    m.F[i] = F;
    if (m.mm_k64) {   // Mercurio & Morini: the drift integral's constant of forward i
      const double k = tau * pow(F, m.beta) * m.T[i] / (1.0 + tau * F);
      ((double*)m.mm_k64)[i] = k;
      ((float*)m.mm_k32)[i] = (float)k;
    }
  }
}

__global__ void setup_swaps_kernel(DevMarket m) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= m.n_swap) return;
  const int a = m.swap_a[s], b = m.swap_b[s];
  double A = 0.0;
  for (int k = a; k < b; ++k) A += m.tau[k] * m.P[k + 1];
  double S = 0.0;
  for (int k = a; k < b; ++k) S += m.tau[k] * m.P[k + 1] / A * m.F[k];
  for (int k = a; k < b; ++k) {
    const double W = m.tau[k] * m.P[k + 1] / A * pow(m.F[k], m.beta) / pow(S, m.beta);
    m.swap_W[(size_t)s * m.max_win + (k - a)] = W;
  }
  m.swap_A[s] = A;
  m.swap_S[s] = S;
  m.swap_TE[s] = m.T[a];
  // W_i = u_i / (A S^b): the swap's quadratic forms are scale x the group's forms in u
  const double as = A * pow(S, m.beta);
  const double sc = 1.0 / (as * as);
  ((double*)m.swap_scale64)[s] = sc;
  ((float*)m.swap_scale32)[s] = (float)sc;
}

// u_{a+i} = tau_{a+i} P(0, T_{a+i+1}) F_{a+i}^b over every group's window (zero past its end), in
// FP64 and FP32: the swap-independent factor of the frozen weights.
__global__ void setup_group_u_kernel(DevMarket m) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= m.n_grp * m.max_gwin) return;
  const int g = t / m.max_gwin, i = t - g * m.max_gwin;
  double u = 0.0;
  if (i < m.grp_L[g]) {
    const int k = m.grp_a[g] + i;
    u = m.tau[k] * m.P[k + 1] * pow(m.F[k], m.beta);
  }
  ((double*)m.grp_u64)[t] = u;
  ((float*)m.grp_u32)[t] = (float)u;
}

// The four slot weights (2 - [i = j]) u_i u_j of every segment of the forward sweep (0 on an empty
// slot).
__global__ void setup_seg_weights_kernel(DevMarket m) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= m.n_seg) return;
  const int4 x = m.seg_uix[q];
  const double uj = m.grp_u64[m.seg_dsc[q].w];
  const int v[4] = {x.x, x.y, x.z, x.w};
  for (int r = 0; r < 4; ++r) {
    const int ix = v[r] & 0xfffff;
    const double w = (v[r] >> 21) & 1 ? (((v[r] >> 20) & 1) ? 1.0 : 2.0) * m.grp_u64[ix] * uj : 0.0;
    ((double*)m.seg_w64)[4 * q + r] = w;
    ((float*)m.seg_w32)[4 * q + r] = (float)w;
  }
}

// Pricing constants of one instrument, into the three 4-vector groups of its block.
template <class R>
__device__ void put_instr(void* blk, int npad, int k, double l, double fk, double inv_den, double c1, double c2,
                          double c3, double sqrtT, double DF, double KF, double sgn, double pm, double sw, int idx) {
  Q4<R>* p = (Q4<R>*)blk;
  Q4<R> v0, v1, v2;
  v0.a = (R)l; v0.b = (R)fk; v0.c = (R)inv_den; v0.d = (R)c1;
  v1.a = (R)c2; v1.b = (R)c3; v1.c = (R)sqrtT; v1.d = (R)DF;
  v2.a = (R)KF; v2.b = (R)sgn; v2.c = (R)pm; v2.d = (R)sw;
  p[k] = v0;
  p[npad + k] = v1;
  p[2 * npad + k] = v2;
  ((int*)(p + 3 * npad))[k] = idx;
}

__device__ void instr_constants(const DevMarket& m, double F, double K, double T, double D, double vol, const double* wu,
                                int k, double* pm_out, double* w_out, void* b64, void* b32, int npad, int idx) {
  const double omb = 1.0 - m.beta;
  const double l = log(F / K);
  const double fkh = pow(F * K, 0.5 * omb);
  const double fk = (m.formula == 0) ? fkh * l : pow(F, omb);   // Hagan: (FK)^{(1-b)/2} l; paper: F^{1-b}
  const double den = fkh * (1.0 + omb * omb * l * l / 24.0 + omb * omb * omb * omb * l * l * l * l / 1920.0);
  const double c1 = omb * omb * T / (24.0 * fkh * fkh);
  const double c2 = m.beta * T / (4.0 * fkh);
  const double c3 = T / 24.0;
  const double sqrtT = sqrt(T);
  const double sgn = (K < F) ? -1.0 : 1.0;
  const double pm = black_otm<double>(vol, sqrtT, l, D * F, K / F, sgn);
  const double v = vol * sqrtT;
  const double d1 = l / v + 0.5 * v;
  const double vega = D * F * exp(-0.5 * d1 * d1) * 0.39894228040143267794 * sqrtT;
  const double w = wu ? wu[k] : 1.0 / (vega * vega);
  pm_out[k] = pm;
  w_out[k] = w;
  const double sw = sqrt(w);
  put_instr<double>(b64, npad, k, l, fk, 1.0 / den, c1, c2, c3, sqrtT, D * F, K / F, sgn, pm, sw, idx);
  put_instr<float>(b32, npad, k, l, fk, 1.0 / den, c1, c2, c3, sqrtT, D * F, K / F, sgn, pm, sw, idx);
}

__global__ void setup_instruments_kernel(DevMarket m) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < m.n_cap) {
    const int i = m.cap_fwd[k];
    instr_constants(m, m.F[i], m.cap_K[k], m.T[i], m.tau[i] * m.P[i + 1], m.cap_vol[k], m.cap_wu, k, m.cap_pm,
                    m.cap_w, m.cblk64, m.cblk32, m.n_cap_pad, i);
  } else if (k < m.n_cap + m.n_swp) {
    const int s = k - m.n_cap;
    const int id = m.swp_swap[s];
    instr_constants(m, m.swap_S[id], m.swp_K[s], m.swap_TE[id], m.swap_A[id], m.swp_vol[s], m.swp_wu, s, m.swp_pm,
                    m.swp_w, m.sblk64, m.sblk32, m.n_swp_pad, id);
  }
}

// The pair-major copy of the FP32 caplet block (PairView), from the scalar FP32 block.
__global__ void setup_pairs_kernel(DevMarket m) {
  const int P = blockIdx.x * blockDim.x + threadIdx.x;
  if (P >= m.n_cap_pairs) return;
  const int np = m.n_cap_pairs;
  const int a = 64 * (P >> 5) + (P & 31), b = a + 32;
  float4* V = (float4*)m.cpair32;
  int2* idx = (int2*)(V + 6 * np);
  if (a >= m.n_cap) {
    for (int j = 0; j < 6; ++j) V[j * np + P] = make_float4(0.f, 0.f, 0.f, 0.f);
    idx[P] = make_int2(0, 0);
    return;
  }
  const InstrView<float> S = instr_view<float>(m.cblk32, m.n_cap_pad);
  const bool hb = b < m.n_cap;
  const int bb = hb ? b : a;
  const Q4<float> g0a = S.g0[a], g0b = S.g0[bb], g1a = S.g1[a], g1b = S.g1[bb], g2a = S.g2[a], g2b = S.g2[bb];
  const float swa = g2a.d, swb = hb ? g2b.d : 0.0f;
  // call (sgn = +1): r = DF sw (Phi(xf) - KF Phi(xs)) - sw P_mkt;
  // put (sgn = -1):  r = KF DF sw (Phi(xf) - Phi(xs) / KF) - sw P_mkt
  const bool ca = g2a.b > 0.0f, cb = g2b.b > 0.0f;
  const float Ca = ca ? g1a.d * swa : g2a.a * g1a.d * swa, Cb = cb ? g1b.d * swb : g2b.a * g1b.d * swb;
  const float Ba = ca ? -g2a.a : -1.0f / g2a.a, Bb = cb ? -g2b.a : -1.0f / g2b.a;
  V[0 * np + P] = make_float4(-fabsf(g0a.a), -fabsf(g0b.a), g0a.b, g0b.b);
  V[1 * np + P] = make_float4(g0a.c, g0b.c, g0a.c * g0a.d, g0b.c * g0b.d);
  V[2 * np + P] = make_float4(g0a.c * g1a.a, g0b.c * g1b.a, g0a.c * g1a.b, g0b.c * g1b.b);
  V[3 * np + P] = make_float4(g1a.c, g1b.c, Ca, Cb);
  V[4 * np + P] = make_float4(Ba, Bb, 0.5f * g1a.c, 0.5f * g1b.c);
  V[5 * np + P] = make_float4(-swa * g2a.c, -swb * g2b.c, 0.0f, 0.0f);
  idx[P] = make_int2(S.idx[a], S.idx[bb]);
}

// ------------------------------------------------------------------ bulk staging into SMEM
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

constexpr long long kWaitLimit = 1LL << 24;

// Stage two regions (sizes multiples of 16, 16-byte aligned both sides) from global memory into
// shared memory with the bulk-copy engine, completion tracked by one mbarrier.  Called by every
// thread of the CTA.  Returns false (and raises the error word) if the bounded wait gave up.
__device__ __forceinline__ void bulk_g2s(void* sdst, const void* gsrc, uint32_t bytes, uint32_t bar) {
  const uint32_t chunk = 32768;
  for (uint32_t off = 0; off < bytes; off += chunk) {
    const uint32_t nb = (bytes - off < chunk) ? (bytes - off) : chunk;
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(smem_u32((char*)sdst + off)), "l"((const char*)gsrc + off), "r"(nb), "r"(bar)
                 : "memory");
  }
}

// The bounded wait on phase 0 of an mbarrier, called by every thread of the CTA: true once the
// phase has completed; after `limit` polls without completion the error word is raised, the
// copies in flight get a second bounded chance to land, and false is returned (the same value in
// every thread).
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, int* err, long long limit = kWaitLimit) {
  uint32_t done = 0;
  long long it = 0;
  while (!done) {
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
                 : "=r"(done) : "r"(bar), "r"(0u) : "memory");
    if (!done && ++it > limit) break;
  }
  const int timed_out = __syncthreads_or(!done);
  if (timed_out) {
    if (threadIdx.x == 0) atomicOr(err, 1);
    it = 0;
    while (!done && ++it < limit) {
      asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
                   : "=r"(done) : "r"(bar), "r"(0u) : "memory");
    }
    __syncthreads();
    return false;
  }
  return true;
}

// Check of the bounded wait itself: one CTA arms an mbarrier for 16 bytes that are never sent (no
// copy is issued, so nothing can land after the CTA retires); the wait gives up after `limit`
// polls and raises *err.
__global__ void wait_selftest_kernel(int* err, long long limit) {
  __shared__ __align__(8) uint64_t mbar;
  const uint32_t bar = smem_u32(&mbar);
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0) asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], 16;" ::"r"(bar) : "memory");
  mbar_wait_bounded(bar, err, limit);
}

__device__ bool stage_to_smem2(void* sdst, const void* gsrc, uint32_t bytes, void* sdst2, const void* gsrc2,
                               uint32_t bytes2, uint64_t* mbar, int* err) {
  if (bytes + bytes2 == 0) return true;
  const uint32_t bar = smem_u32(mbar);
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes + bytes2) : "memory");
    bulk_g2s(sdst, gsrc, bytes, bar);
    bulk_g2s(sdst2, gsrc2, bytes2, bar);
  }
  if (!mbar_wait_bounded(bar, err)) return false;
  // every thread has seen the phase complete: the barrier may be re-initialised by a later stage
  if (threadIdx.x == 0) asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(bar) : "memory");
  return true;
}

template <class R> __device__ __forceinline__ const void* cap_block(const DevMarket& m);
template <> __device__ __forceinline__ const void* cap_block<double>(const DevMarket& m) { return m.cblk64; }
template <> __device__ __forceinline__ const void* cap_block<float>(const DevMarket& m) { return m.cblk32; }

template <class R> __device__ __forceinline__ const void* quad_block(const DevMarket& m);
template <> __device__ __forceinline__ const void* quad_block<double>(const DevMarket& m) { return m.q64; }
template <> __device__ __forceinline__ const void* quad_block<float>(const DevMarket& m) { return m.q32; }

// Shared-memory plan: [caplet block][quadrature table][warp scratch x W][mbarrier (16 B),
// 32 doubles, 32 ints].  Every region starts on a 16-byte boundary.
constexpr uint32_t kRngBytesPerWarp = 32 * 4 * sizeof(uint64_t);

// Shared-memory room for the caplet block: the scalar block, or in FP32 the pair-major block
// (whichever is larger).
template <class R>
__host__ __device__ inline uint32_t cap_region_bytes(const DevMarket& m) {
  const uint32_t a = instr_block_bytes<R>(m.n_cap_pad);
  if (sizeof(R) != 4) return a;
  const uint32_t b = pair_block_bytes(m.n_cap_pairs);
  return a > b ? a : b;
}

template <class R>
__host__ __device__ inline uint32_t smem_bytes(const DevMarket& m, int W) {
  return cap_region_bytes<R>(m) + (uint32_t)sizeof(QuadTab<R>) +
         (uint32_t)W * warp_scratch_elems(m.NP, m.n_fwd) * sizeof(R) + 512 + (uint32_t)W * kRngBytesPerWarp;
}

template <class R>
struct CtaSmem {
  void* cap;
  QuadTab<R>* quad;
  unsigned char* scratch;
  uint64_t* mbar;
  double* red_f;
  int* red_c;
  uint64_t* rng;    // [W x 32 x 4] Philox words of the next 8 steps, per warp
};

template <class R>
__device__ __forceinline__ CtaSmem<R> carve(unsigned char* smem, const DevMarket& m, int W) {
  CtaSmem<R> s;
  s.cap = smem;
  s.quad = (QuadTab<R>*)(smem + cap_region_bytes<R>(m));
  s.scratch = (unsigned char*)s.quad + sizeof(QuadTab<R>);
  unsigned char* tail = s.scratch + (size_t)W * warp_scratch_elems(m.NP, m.n_fwd) * sizeof(R);
  s.mbar = (uint64_t*)tail;
  s.red_f = (double*)(tail + 16);
  s.red_c = (int*)(tail + 16 + 32 * sizeof(double));
  s.rng = (uint64_t*)(tail + 512);
  return s;
}

// Stage the caplet block (pair-major with `pairs`, for the packed FP32 pricer) and the quadrature
// table.
template <class R>
__device__ __forceinline__ bool stage_market(const CtaSmem<R>& cs, const DevMarket& m, bool pairs) {
  if (pairs)
    return stage_to_smem2(cs.cap, m.cpair32, pair_block_bytes(m.n_cap_pairs), cs.quad, quad_block<R>(m),
                          (uint32_t)sizeof(QuadTab<R>), cs.mbar, m.err);
  return stage_to_smem2(cs.cap, cap_block<R>(m), instr_block_bytes<R>(m.n_cap_pad), cs.quad, quad_block<R>(m),
                        (uint32_t)sizeof(QuadTab<R>), cs.mbar, m.err);
}

// Whether warp_objective prices the caplets with the packed FP32 pricer (and so reads the
// pair-major block): FP32, the Hagan (2002) form, no model vols requested; not the Mercurio &
// Morini model (a rho per forward: the scalar pricer).
template <class R, int MODEL, int FORMULA>
__host__ __device__ constexpr bool packed_pricer() { return sizeof(R) == 4 && FORMULA == 0 && MODEL != 2; }

// ------------------------------------------------------------------ objective and vols
// When a CTA's staging gave up (the error word is raised), its points' outputs are set to NaN
// rather than left unwritten: point i of the grid-stride loop starting at i0 with stride `step`,
// thread t of nt per point.
__device__ __forceinline__ void nan_outputs(long long i0, long long step, long long n, int t, int nt, double* f,
                                            double* v1, int w1, double* v2, int w2) {
  const double qnan = __longlong_as_double(0x7ff8000000000000LL);
  for (long long i = i0; i < n; i += step) {
    if (f && t == 0) f[i] = qnan;
    if (v1) for (int k = t; k < w1; k += nt) v1[i * w1 + k] = qnan;
    if (v2) for (int k = t; k < w2; k += nt) v2[i * w2 + k] = qnan;
  }
}

// f, the model vols (vols != null) or the weighted residuals (res != null) of n points; one warp
// per point, grid-stride.
template <class R, int MODEL, int FORMULA>
__global__ void objective_kernel(DevMarket m, const double* __restrict__ X, long long n, double* __restrict__ f,
                                 double* __restrict__ vols, double* __restrict__ res) {
  extern __shared__ __align__(128) unsigned char smem[];
  const int W = blockDim.x >> 5, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  CtaSmem<R> cs = carve<R>(smem, m, W);
  const int n_instr = m.n_cap + m.n_swp;
  if (!stage_market<R>(cs, m, packed_pricer<R, MODEL, FORMULA>() && vols == nullptr)) {
    nan_outputs((long long)blockIdx.x * W + warp, (long long)gridDim.x * W, n, lane, 32, f, vols, n_instr, res, n_instr);
    return;
  }
  const InstrView<R> capB = instr_view<R>(cs.cap, m.n_cap_pad);
  WarpScratch<R> ws = warp_scratch<R>((R*)cs.scratch + (size_t)warp * warp_scratch_elems(m.NP, m.n_fwd), m.NP, m.n_fwd);
  for (long long i = (long long)blockIdx.x * W + warp; i < n; i += (long long)gridDim.x * W) {
    if (lane < kMaxParam) ws.xs[lane] = lane < m.n_param ? (R)X[i * m.n_param + lane] : R(0);
    __syncwarp();
    const auto fi = warp_objective<R, MODEL, FORMULA>(m, capB, *cs.quad, ws, lane, vols ? vols + i * n_instr : nullptr,
                                                      res ? res + i * n_instr : nullptr);
    if (f && lane == 0) f[i] = obj_to_double(fi);
    __syncwarp();
  }
}

// ------------------------------------------------------------------ simulated annealing
struct SAState {
  double* xs;        // [P]  level start point
  double* fs;        // [1]
  double* T0;        // [1]
  double* xe;        // [C x P] chain end points of the current level
  double* fe;        // [C]
  double* xb;        // [C x P] chain best-ever points
  double* fb;        // [C]
  double* part_f;    // [gridDim] CTA minima
  int* part_c;
  unsigned int* counter;
  double* trace_f;   // [L]
  double* trace_x;   // [L x P] the start point after each level (the best end point), or null
  unsigned long long* trace_t;   // [L + 1] global timer (ns) at the start and at each level's end, or null
  uint8_t* bits;     // [C x L x N] or null
  double* best_x;    // [P]
  double* best_f;    // [1]
  double* lvl;       // [3] of the level about to run: T_l, its step scale, 1 / T_l
};

struct SAParams {
  int C, L, N, P;
  double cooling, step_frac, step_floor, T0_opt;
  unsigned long long seed, market_index;
  const double* x0;  // device [P]
};

// The search's start (f(x0), T0, the first start point, the level counter).  If the staging gave up
// (error word raised) f(x0) is taken as +inf, so that the level kernels still run to completion and
// the caller reads SABR_LMM_ETIMEOUT.
__device__ __forceinline__ unsigned long long global_timer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// The constants of a level: T_l = T0 cooling^l as repeated products (each level's last CTA
// multiplies the previous T once, so no thread runs the product chain), the step scale
// max(step_frac sqrt(T_l / T0), step_floor) and 1 / T_l.  One thread writes them.
__device__ __forceinline__ void level_consts_write(const SAState& st, const SAParams& sp, double T, double T0) {
  st.lvl[0] = T;
  st.lvl[1] = fmax(sp.step_frac * sqrt(T / T0), sp.step_floor);
  st.lvl[2] = 1.0 / T;
}

__device__ __forceinline__ void sa_start_write(const SAState& st, const SAParams& sp, int t, double x0, double f0) {
  if (t < sp.P) st.xs[t] = x0;
  if (t == 0) {
    st.fs[0] = f0;
    const double T0 = sp.T0_opt > 0.0 ? sp.T0_opt : ((isfinite(f0) && f0 > 0.0) ? f0 : 1.0);
    st.T0[0] = T0;
    level_consts_write(st, sp, T0, T0);
    st.counter[0] = 0u;
    if (st.trace_t) st.trace_t[0] = global_timer_ns();
  }
}

// The level's trace after its minimum is known: the next start point (read back from the best end
// point) and the time the level ended.  Called by the threads of the last CTA of the level.
__device__ __forceinline__ void level_trace_write(const SAState& st, int P, int level, int t, double x) {
  if (st.trace_x && t < P) st.trace_x[(size_t)level * P + t] = x;
  if (st.trace_t && t == 0) st.trace_t[level + 1] = global_timer_ns();
}

template <class R, int MODEL, int FORMULA>
__global__ void sa_start_kernel(DevMarket m, SAState st, SAParams sp) {
  extern __shared__ __align__(128) unsigned char smem[];
  const int lane = threadIdx.x & 31;
  CtaSmem<R> cs = carve<R>(smem, m, 1);
  // the start point in the chain-state precision (FP32 chains start from the rounded point)
  const double x0 = lane < sp.P ? (double)(R)sp.x0[lane] : 0.0;
  if (!stage_market<R>(cs, m, packed_pricer<R, MODEL, FORMULA>())) {
    sa_start_write(st, sp, lane, x0, __longlong_as_double(0x7ff0000000000000LL));
    return;
  }
  const InstrView<R> capB = instr_view<R>(cs.cap, m.n_cap_pad);
  WarpScratch<R> ws = warp_scratch<R>((R*)cs.scratch, m.NP, m.n_fwd);
  if (lane < kMaxParam) ws.xs[lane] = (R)x0;
  __syncwarp();
  const double f0 = obj_to_double(warp_objective<R, MODEL, FORMULA>(m, capB, *cs.quad, ws, lane, nullptr));
  sa_start_write(st, sp, lane, x0, f0);
}

__device__ __forceinline__ bool lex_less(double fa, int ca, double fb, int cb) {
  return fa < fb || (fa == fb && ca < cb);
}

// S1: the neighbour of slot k (lane k) from its uniform, in the chain-state precision.
//   FP64: x + sf (hi - lo)(2u - 1) with no contraction (the rounding of the plain sequence of
//         products and sums), u = (word >> 11) 2^-53, reflected once, clamped.
//   FP32: the same in FP32 with u = (word >> 40) 2^-24.
__device__ __forceinline__ double neighbour(double x, double lo, double hi, double sf, uint64_t word) {
  const double u = u53(word);
  double v = __dadd_rn(x, __dmul_rn(__dmul_rn(sf, __dsub_rn(hi, lo)), __dsub_rn(__dmul_rn(2.0, u), 1.0)));
  if (v < lo) v = __dsub_rn(__dmul_rn(2.0, lo), v);
  if (v > hi) v = __dsub_rn(__dmul_rn(2.0, hi), v);
  return fmin(fmax(v, lo), hi);
}
__device__ __forceinline__ float neighbour(float x, float lo, float hi, float sf, uint64_t word) {
  const float u = (float)(uint32_t)(word >> 40) * 0x1.0p-24f;
  float v = x + sf * (hi - lo) * (2.0f * u - 1.0f);
  if (v < lo) v = 2.0f * lo - v;
  if (v > hi) v = 2.0f * hi - v;
  return fminf(fmaxf(v, lo), hi);
}

// S8: Metropolis test, identical on every lane.
//   FP64: accept iff fy < f or u < exp(-(fy - f) / T).
//   FP32: dE from the float-float values; the test runs in FP32 (e = exp(-dE/T)) and is redone in
//         FP64 whenever u lies within the FP32 error band of e, so the decision equals the FP64
//         decision on the same objective values.
__device__ __forceinline__ bool metropolis(double fy, double f, uint64_t word, double T, float) {
  return (fy < f) || (u53(word) < exp(-(fy - f) / T));
}
__device__ __forceinline__ bool metropolis(FF fy, FF f, uint64_t word, double T, float invT) {
  const float dE = (fy.hi - f.hi) + (fy.lo - f.lo);
  if (dE < 0.f) return true;
  const float t = dE * invT;
  const float e = exp_approx(-t);
  const float uf = (float)(uint32_t)(word >> 40) * 0x1.0p-24f;   // uf <= u < uf + 2^-24
  const float band = 0x1.0p-24f + e * (1e-6f + 4e-7f * fabsf(t));
  if (fabsf(uf - e) > band) return uf < e;
  const double dEd = ((double)fy.hi - (double)f.hi) + ((double)fy.lo - (double)f.lo);
  return u53(word) < exp(-dEd / T);
}

template <class R>
__device__ __forceinline__ R box_lo(const DevMarket& m, int k) { return (R)m.lo[k]; }
template <class R>
__device__ __forceinline__ R box_hi(const DevMarket& m, int k) { return (R)m.hi[k]; }

// BIG: one CTA of up to 28 chains (the whole SM at 72 registers) instead of 4-chain CTAs, so the
// market is staged once per SM rather than once per 4 chains.
template <class R, int MODEL, int FORMULA, bool BIG = false>
__global__ void __launch_bounds__(BIG ? 896 : 128, BIG ? 1 : (sizeof(R) == 4 ? 7 : 4))
sa_level_kernel(DevMarket m, SAState st, SAParams sp, int level) {
  typedef typename ObjOf<R>::T O;
  extern __shared__ __align__(128) unsigned char smem[];
  const int W = blockDim.x >> 5, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  CtaSmem<R> cs = carve<R>(smem, m, W);
  // a CTA whose staging gave up (error word raised) runs no step: its chains end the level at the
  // start point with f = +inf, and it still takes its level ticket, so the level-end minimum over
  // the other CTAs completes
  const bool staged = stage_market<R>(cs, m, packed_pricer<R, MODEL, FORMULA>());
  const InstrView<R> capB = instr_view<R>(cs.cap, m.n_cap_pad);
  WarpScratch<R> ws = warp_scratch<R>((R*)cs.scratch + (size_t)warp * warp_scratch_elems(m.NP, m.n_fwd), m.NP, m.n_fwd);

  const int c = blockIdx.x * W + warp;
  const bool active = staged && c < sp.C;
  if (!staged && c < sp.C) {
    if (lane < sp.P) {
      st.xe[(size_t)c * sp.P + lane] = st.xs[lane];
      if (level == 0) st.xb[(size_t)c * sp.P + lane] = st.xs[lane];
    }
    if (lane == 0) {
      st.fe[c] = __longlong_as_double(0x7ff0000000000000LL);
      if (level == 0) st.fb[c] = __longlong_as_double(0x7ff0000000000000LL);
    }
  }
  const int P = sp.P;
  const double T = st.lvl[0], sf = st.lvl[1];
  const float invT = (float)st.lvl[2];

  O f;
  obj_from_double(st.fs[0], f);
  R x = 0, lo = 0, hi = 0, xbk = 0;
  bool freek = false;
  if (lane < P) {
    x = (R)st.xs[lane];
    lo = box_lo<R>(m, lane);
    hi = box_hi<R>(m, lane);
    freek = m.freem[lane] != 0;
  }
  O fbest = f;
  if (active) {
    if (level > 0) {
      obj_from_double(st.fb[c], fbest);
      if (lane < P) xbk = (R)st.xb[(size_t)c * P + lane];
    } else {
      xbk = x;
    }
  }
  const unsigned long long cw = (unsigned long long)c | (sp.market_index << 32);
  // Philox block (lane & 3) of step s0 + (lane >> 2), 8 steps at a time, parked in shared memory;
  // with 16 or more slots (Mercurio & Morini) block (lane & 7) of step s0 + (lane >> 3), 4 steps at
  // a time (up to 32 words a step)
  constexpr bool WIDE = MODEL == 2;
  constexpr int BPS = WIDE ? 8 : 4, SPR = 32 / BPS;   // blocks per step, steps per refill
  uint64_t* rng = cs.rng + (size_t)warp * 128;
  for (int s = 0; s < sp.N; ++s) {
    if (active) {
      // S1: the step's uniforms; lane k needs word (k & 3) of block (k >> 2) of this step
      if ((s & (SPR - 1)) == 0) {
        const U4 o = philox4x64_10((uint64_t)(lane & (BPS - 1)), (uint64_t)(s + lane / BPS), (uint64_t)level, cw,
                                   sp.seed, 0ull);
        __syncwarp();
#pragma unroll
        for (int j = 0; j < 4; ++j) rng[lane * 4 + j] = o.v[j];
        __syncwarp();
      }
      const int row = (s & (SPR - 1)) * BPS;
      const uint64_t word = rng[(row | ((lane >> 2) & (BPS - 1))) * 4 + (lane & 3)];
      const uint64_t wacc = rng[(row | (P >> 2)) * 4 + (P & 3)];
      R y = x;
      if (lane < P && freek) y = neighbour(x, lo, hi, (R)sf, word);
      if (lane < kMaxParam) ws.xs[lane] = lane < P ? y : R(0);
      __syncwarp();
      const O fy = warp_objective<R, MODEL, FORMULA>(m, capB, *cs.quad, ws, lane, nullptr);
      const bool acc = metropolis(fy, f, wacc, T, invT);
      if (acc) {
        x = y;
        f = fy;
        if (obj_less(f, fbest)) { fbest = f; xbk = x; }
      }
      if (st.bits && lane == 0) st.bits[((size_t)c * sp.L + level) * sp.N + s] = acc ? 1 : 0;
    }
  }
  if (active) {
    if (lane < P) {
      st.xe[(size_t)c * P + lane] = (double)x;
      st.xb[(size_t)c * P + lane] = (double)xbk;
    }
    if (lane == 0) {
      st.fe[c] = obj_to_double(f);
      st.fb[c] = obj_to_double(fbest);
    }
    __threadfence();
  }
  const double fend = active ? obj_to_double(f) : __longlong_as_double(0x7ff0000000000000LL);
  // CTA minimum over its chains' end points, lexicographic in (f, chain)
  if (lane == 0) {
    cs.red_f[warp] = fend;
    cs.red_c[warp] = active ? c : 0x7fffffff;
  }
  __syncthreads();
  __shared__ bool last;
  if (threadIdx.x == 0) {
    double bf = cs.red_f[0];
    int bc = cs.red_c[0];
    for (int w = 1; w < W; ++w)
      if (lex_less(cs.red_f[w], cs.red_c[w], bf, bc)) { bf = cs.red_f[w]; bc = cs.red_c[w]; }
    st.part_f[blockIdx.x] = bf;
    st.part_c[blockIdx.x] = bc;
    __threadfence();
    const unsigned int ticket = atomicAdd(st.counter, 1u);
    last = (ticket == gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return;
  // the last CTA to finish: minimum over all CTAs, the next start point, the level trace
  double bf = __longlong_as_double(0x7ff0000000000000LL);
  int bc = 0x7fffffff;
  for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) {
    const double pf = __ldcg(st.part_f + b);
    const int pc = __ldcg(st.part_c + b);
    if (lex_less(pf, pc, bf, bc)) { bf = pf; bc = pc; }
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const double of = __shfl_xor_sync(0xffffffffu, bf, off);
    const int oc = __shfl_xor_sync(0xffffffffu, bc, off);
    if (lex_less(of, oc, bf, bc)) { bf = of; bc = oc; }
  }
  __syncthreads();
  if (lane == 0) { cs.red_f[warp] = bf; cs.red_c[warp] = bc; }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < W; ++w)
      if (lex_less(cs.red_f[w], cs.red_c[w], cs.red_f[0], cs.red_c[0])) { cs.red_f[0] = cs.red_f[w]; cs.red_c[0] = cs.red_c[w]; }
    st.fs[0] = cs.red_f[0];
    st.trace_f[level] = cs.red_f[0];
    level_consts_write(st, sp, T * sp.cooling, st.T0[0]);
  }
  __syncthreads();
  const int cbest = cs.red_c[0];
  if (threadIdx.x < P) {
    const double xn = __ldcg(st.xe + (size_t)cbest * P + threadIdx.x);
    st.xs[threadIdx.x] = xn;
    level_trace_write(st, P, level, threadIdx.x, xn);
  } else {
    level_trace_write(st, P, level, threadIdx.x, 0.0);
  }
  if (threadIdx.x == 0) st.counter[0] = 0u;
}

// The best point ever accepted, over all chains (ties to the lowest chain index).
__global__ void sa_final_kernel(SAState st, int C, int P) {
  __shared__ double sf[32];
  __shared__ int sc[32];
  double bf = __longlong_as_double(0x7ff0000000000000LL);
  int bc = 0x7fffffff;
  for (int c = threadIdx.x; c < C; c += blockDim.x)
    if (lex_less(st.fb[c], c, bf, bc)) { bf = st.fb[c]; bc = c; }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const double of = __shfl_xor_sync(0xffffffffu, bf, off);
    const int oc = __shfl_xor_sync(0xffffffffu, bc, off);
    if (lex_less(of, oc, bf, bc)) { bf = of; bc = oc; }
  }
  if (lane == 0) { sf[warp] = bf; sc[warp] = bc; }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
      if (lex_less(sf[w], sc[w], sf[0], sc[0])) { sf[0] = sf[w]; sc[0] = sc[w]; }
    st.best_f[0] = sf[0];
  }
  __syncthreads();
  if (threadIdx.x < P) st.best_x[threadIdx.x] = st.xb[(size_t)sc[0] * P + threadIdx.x];
}

// RMSE (vol points) of model vols against market vols for one point per market.
__global__ void rmse_from_vols_kernel(const double* vols, const double* cap_vol, const double* swp_vol, int n_cap,
                                      int n_swp, double* out) {
  __shared__ double part[32];
  double s = 0.0;
  const int n = n_cap + n_swp;
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    const double mk = k < n_cap ? cap_vol[k] : swp_vol[k - n_cap];
    const double e = vols[k] - mk;
    s += e * e;
  }
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += part[w];
    out[0] = 100.0 * sqrt(t / (double)n);
  }
}



// ====================================================================== markets with swaptions
// One CTA per parameter point (chain).  Shared-memory plan: [caplet block][swaption block]
// [quadrature table][chain scratch][32 objective values][mbarrier, 32 doubles, 32 ints].

template <class R> __device__ __forceinline__ const void* swp_block(const DevMarket& m);
template <> __device__ __forceinline__ const void* swp_block<double>(const DevMarket& m) { return m.sblk64; }
template <> __device__ __forceinline__ const void* swp_block<float>(const DevMarket& m) { return m.sblk32; }

// With tc, the tensor-core operand (kTcBytes), its barrier and the TMEM address slot follow, and the
// request is at least 80 KB so that at most two CTAs (2 x 256 TMEM columns) share an SM.
template <class R>
__host__ __device__ inline uint32_t smem_bytes_cta(const DevMarket& m, bool tc = false) {
  uint32_t b = (uint32_t)sizeof(QuadTab<R>) +
               (uint32_t)cta_scratch_elems<R>(m) * sizeof(R) + 32 * 16 + 512;
  if (tc) {
    b += kTcBytes + 32;
    if (b < 80u * 1024u) b = 80u * 1024u;
  }
  return b;
}

template <class R>
struct CtaSmemS {
  void* cap;
  void* swp;
  QuadTab<R>* quad;
  R* scratch;
  void* red;
  uint64_t* mbar;
  double* red_f;
  int* red_c;
  unsigned char* tcU;    // tensor-core operand (TC kernels)
  uint64_t* tc_mbar;
  uint32_t* tc_slot;
};

template <class R>
__device__ __forceinline__ CtaSmemS<R> carve_cta(unsigned char* smem, const DevMarket& m) {
  CtaSmemS<R> s;
  unsigned char* p = smem;
  // the instrument blocks are read in place from global memory (read once per evaluation, by the
  // pricing phase): the shared memory they would take is worth more as L1 and occupancy
  s.cap = const_cast<void*>(cap_block<R>(m));
  s.swp = const_cast<void*>(swp_block<R>(m));
  s.quad = (QuadTab<R>*)p; p += sizeof(QuadTab<R>);
  s.scratch = (R*)p; p += (size_t)cta_scratch_elems<R>(m) * sizeof(R);
  s.red = p; p += 32 * 16;
  s.mbar = (uint64_t*)p;
  s.red_f = (double*)(p + 16);
  s.red_c = (int*)(p + 16 + 32 * sizeof(double));
  s.tcU = p + 512;
  s.tc_mbar = (uint64_t*)(s.tcU + kTcBytes);
  s.tc_slot = (uint32_t*)(s.tcU + kTcBytes + 16);
  return s;
}

// Set up the tensor-core state of a CTA (after staging): completion barrier, TMEM columns, a
// zeroed operand (its padding rows and columns stay zero).  Every thread calls.
template <class R>
__device__ __forceinline__ TcState tc_setup(const CtaSmemS<R>& cs, int* err) {
  if (threadIdx.x == 0) {
    const uint32_t bar = (uint32_t)__cvta_generic_to_shared(cs.tc_mbar);
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tc_alloc(cs.tc_slot);
  for (uint32_t i = threadIdx.x; i < kTcBytes / 16; i += blockDim.x) ((uint4*)cs.tcU)[i] = make_uint4(0, 0, 0, 0);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  TcState tc;
  tc.U = cs.tcU;
  tc.tmem = *cs.tc_slot;
  tc.mbar = cs.tc_mbar;
  tc.phase = 0;
  tc.err = err;
  return tc;
}

__device__ __forceinline__ void tc_teardown(const TcState& tc) {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  tc_dealloc(tc.tmem);
}

__device__ bool stage_to_smem3(void* d0, const void* g0, uint32_t b0, void* d1, const void* g1, uint32_t b1, void* d2,
                               const void* g2, uint32_t b2, uint64_t* mbar, int* err) {
  const uint32_t bar = smem_u32(mbar);
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    // earlier generic-proxy reads of the destination (a previous market) precede the async writes
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(b0 + b1 + b2) : "memory");
    bulk_g2s(d0, g0, b0, bar);
    bulk_g2s(d1, g1, b1, bar);
    bulk_g2s(d2, g2, b2, bar);
  }
  if (!mbar_wait_bounded(bar, err)) return false;
  // every thread has seen the phase complete: the barrier may be re-initialised by a later stage
  if (threadIdx.x == 0) asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(bar) : "memory");
  return true;
}

template <class R>
__device__ __forceinline__ bool stage_market_cta(const CtaSmemS<R>& cs, const DevMarket& m) {
  if (!stage_to_smem2(cs.quad, quad_block<R>(m), (uint32_t)sizeof(QuadTab<R>), nullptr, nullptr, 0u, cs.mbar, m.err))
    return false;
  return true;
}

template <class R, int FORMULA, bool TC>
__global__ void __launch_bounds__(256, 2) objective_cta_kernel(DevMarket m, const double* __restrict__ X, long long n,
                                                            double* __restrict__ f, double* __restrict__ vols,
                                                            double* __restrict__ res) {
  typedef typename ObjOf<R>::T O;
  extern __shared__ __align__(128) unsigned char smem[];
  CtaSmemS<R> cs = carve_cta<R>(smem, m);
  const int n_instr = m.n_cap + m.n_swp;
  if (!stage_market_cta<R>(cs, m)) {
    nan_outputs(blockIdx.x, gridDim.x, n, threadIdx.x, blockDim.x, f, vols, n_instr, res, n_instr);
    return;
  }
  TcState tc{};
  if (TC) tc = tc_setup<R>(cs, m.err);
  const InstrView<R> capB = instr_view<R>(cs.cap, m.n_cap_pad);
  const InstrView<R> swpB = instr_view<R>(cs.swp, m.n_swp_pad);
  CtaScratch<R> sc = cta_scratch<R>(cs.scratch, m);
  for (long long i = blockIdx.x; i < n; i += gridDim.x) {
    if (threadIdx.x < kMaxParam) sc.xs[threadIdx.x] = threadIdx.x < m.n_param ? (R)X[i * m.n_param + threadIdx.x] : R(0);
    __syncthreads();
    const O fi = cta_objective<R, FORMULA, TC>(m, capB, swpB, *cs.quad, sc, (O*)cs.red,
                                               vols ? vols + i * n_instr : nullptr, &tc,
                                               res ? res + i * n_instr : nullptr);
    if (f && threadIdx.x == 0) f[i] = obj_to_double(fi);
    __syncthreads();
  }
  if (TC) tc_teardown(tc);
}

template <class R, int FORMULA, bool TC>
__global__ void __launch_bounds__(256, 2) sa_start_cta_kernel(DevMarket m, SAState st, SAParams sp) {
  typedef typename ObjOf<R>::T O;
  extern __shared__ __align__(128) unsigned char smem[];
  CtaSmemS<R> cs = carve_cta<R>(smem, m);
  const double x0 = threadIdx.x < (unsigned)sp.P ? (double)(R)sp.x0[threadIdx.x] : 0.0;
  if (!stage_market_cta<R>(cs, m)) {
    sa_start_write(st, sp, threadIdx.x, x0, __longlong_as_double(0x7ff0000000000000LL));
    return;
  }
  TcState tc{};
  if (TC) tc = tc_setup<R>(cs, m.err);
  const InstrView<R> capB = instr_view<R>(cs.cap, m.n_cap_pad);
  const InstrView<R> swpB = instr_view<R>(cs.swp, m.n_swp_pad);
  CtaScratch<R> sc = cta_scratch<R>(cs.scratch, m);
  if (threadIdx.x < kMaxParam) sc.xs[threadIdx.x] = (R)x0;
  __syncthreads();
  const double f0 = obj_to_double(cta_objective<R, FORMULA, TC>(m, capB, swpB, *cs.quad, sc, (O*)cs.red, nullptr, &tc));
  sa_start_write(st, sp, threadIdx.x, x0, f0);
  if (TC) tc_teardown(tc);
}

// One chain of one market at one temperature level, run by the whole CTA (markets with swaptions
// and the batch).  The chain's end state is written; the CTA that finishes the market's last chain
// (counted on st.counter, n_chains arrivals) takes the minimum over the market's chains and sets
// the next start point and the level trace.
// With staged == false (the CTA's staging gave up and raised the error word) the chain runs no
// step: it ends the level at the start point with f = +inf, and the ticket is still taken so that
// the market's level-end minimum completes.
template <class R, int FORMULA, bool TC = false>
__device__ void cta_chain_level(const DevMarket& m, const SAState& st, const SAParams& sp, int c, int level,
                                const CtaSmemS<R>& cs, const InstrView<R>& capB, const InstrView<R>& swpB,
                                const CtaScratch<R>& sc, unsigned long long* s_wacc, bool* s_last,
                                TcState* tc = nullptr, bool staged = true) {
  typedef typename ObjOf<R>::T O;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int P = sp.P;
  const double T = st.lvl[0], sf = st.lvl[1];
  const float invT = (float)st.lvl[2];

  O f;
  obj_from_double(st.fs[0], f);
  R x = 0, lo = 0, hi = 0, xbk = 0;
  bool freek = false;
  if (warp == 0 && lane < P) {
    x = (R)st.xs[lane];
    lo = box_lo<R>(m, lane);
    hi = box_hi<R>(m, lane);
    freek = m.freem[lane] != 0;
    xbk = level > 0 ? (R)st.xb[(size_t)c * P + lane] : x;
  }
  O fbest = f;
  if (level > 0) obj_from_double(st.fb[c], fbest);
  if (!staged) {
    f = obj_inf(O());
    if (level == 0) fbest = f;
  }
  const unsigned long long cw = (unsigned long long)c | (sp.market_index << 32);
  U4 o;
  R y = x;
  for (int s = 0; s < (staged ? sp.N : 0); ++s) {
    if (warp == 0) {
      if ((s & 7) == 0) o = philox4x64_10((uint64_t)(lane & 3), (uint64_t)(s + (lane >> 2)), (uint64_t)level, cw, sp.seed, 0ull);
      const int src = ((s & 7) << 2) | ((lane >> 2) & 3), wsel = lane & 3;
      const uint64_t w0 = __shfl_sync(0xffffffffu, o.v[0], src);
      const uint64_t w1 = __shfl_sync(0xffffffffu, o.v[1], src);
      const uint64_t w2 = __shfl_sync(0xffffffffu, o.v[2], src);
      const uint64_t w3 = __shfl_sync(0xffffffffu, o.v[3], src);
      const uint64_t word = wsel == 0 ? w0 : (wsel == 1 ? w1 : (wsel == 2 ? w2 : w3));
      y = x;
      if (lane < P && freek) y = neighbour(x, lo, hi, (R)sf, word);
      if (lane < kMaxParam) sc.xs[lane] = lane < P ? y : R(0);
      const uint64_t wacc = __shfl_sync(0xffffffffu, word, P);
      if (lane == 0) *s_wacc = wacc;
    }
    __syncthreads();
    const O fy = cta_objective<R, FORMULA, TC>(m, capB, swpB, *cs.quad, sc, (O*)cs.red, nullptr, tc);
    const bool acc = metropolis(fy, f, (uint64_t)*s_wacc, T, invT);
    if (acc) {
      x = y;
      f = fy;
      if (obj_less(f, fbest)) { fbest = f; xbk = x; }
    }
    if (st.bits && threadIdx.x == 0) st.bits[((size_t)c * sp.L + level) * sp.N + s] = acc ? 1 : 0;
    __syncthreads();   // s_wacc and the point are rewritten by the next step
  }
  if (warp == 0 && lane < P) {
    st.xe[(size_t)c * P + lane] = (double)x;
    st.xb[(size_t)c * P + lane] = (double)xbk;
  }
  if (threadIdx.x == 0) {
    st.fe[c] = obj_to_double(f);
    st.fb[c] = obj_to_double(fbest);
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    st.part_f[c] = obj_to_double(f);
    st.part_c[c] = c;
    __threadfence();
    const unsigned int ticket = atomicAdd(st.counter, 1u);
    *s_last = (ticket == (unsigned)sp.C - 1);
  }
  __syncthreads();
  if (!*s_last) return;
  double bf = __longlong_as_double(0x7ff0000000000000LL);
  int bc = 0x7fffffff;
  for (int b = threadIdx.x; b < sp.C; b += blockDim.x) {
    const double pf = __ldcg(st.part_f + b);
    const int pc = __ldcg(st.part_c + b);
    if (lex_less(pf, pc, bf, bc)) { bf = pf; bc = pc; }
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const double of = __shfl_xor_sync(0xffffffffu, bf, off);
    const int oc = __shfl_xor_sync(0xffffffffu, bc, off);
    if (lex_less(of, oc, bf, bc)) { bf = of; bc = oc; }
  }
  if (lane == 0) { cs.red_f[warp] = bf; cs.red_c[warp] = bc; }
  __syncthreads();
  if (threadIdx.x == 0) {
    const int W = blockDim.x >> 5;
    for (int w = 1; w < W; ++w)
      if (lex_less(cs.red_f[w], cs.red_c[w], cs.red_f[0], cs.red_c[0])) { cs.red_f[0] = cs.red_f[w]; cs.red_c[0] = cs.red_c[w]; }
    st.fs[0] = cs.red_f[0];
    st.trace_f[level] = cs.red_f[0];
    level_consts_write(st, sp, T * sp.cooling, st.T0[0]);
  }
  __syncthreads();
  const int cbest = cs.red_c[0];
  if (threadIdx.x < (unsigned)P) {
    const double xn = __ldcg(st.xe + (size_t)cbest * P + threadIdx.x);
    st.xs[threadIdx.x] = xn;
    level_trace_write(st, P, level, threadIdx.x, xn);
  } else {
    level_trace_write(st, P, level, threadIdx.x, 0.0);
  }
  if (threadIdx.x == 0) st.counter[0] = 0u;
  __syncthreads();
}

template <class R, int FORMULA, bool TC>
__global__ void __launch_bounds__(256, 2) sa_level_cta_kernel(DevMarket m, SAState st, SAParams sp, int level) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ unsigned long long s_wacc;
  __shared__ bool s_last;
  CtaSmemS<R> cs = carve_cta<R>(smem, m);
  const bool staged = stage_market_cta<R>(cs, m);
  TcState tc{};
  if (TC && staged) tc = tc_setup<R>(cs, m.err);
  const InstrView<R> capB = instr_view<R>(cs.cap, m.n_cap_pad);
  const InstrView<R> swpB = instr_view<R>(cs.swp, m.n_swp_pad);
  CtaScratch<R> sc = cta_scratch<R>(cs.scratch, m);
  cta_chain_level<R, FORMULA, TC>(m, st, sp, blockIdx.x, level, cs, capB, swpB, sc, &s_wacc, &s_last, &tc, staged);
  if (TC && staged) tc_teardown(tc);
}

// ====================================================================== batch of markets
// A persistent launch per temperature level over every (market, chain) work item of a batch.  CTAs
// take items from an atomic counter, markets in the given order (largest first); a CTA re-stages
// the market's blocks only when its next item belongs to another market.  Each market keeps its
// own chain state and its own best-chain reduction (cta_chain_level).
struct BatchArgs {
  const DevMarket* mk;      // [n_markets]
  const SAState* st;        // [n_markets]
  const SAParams* sp;       // [n_markets]
  const int* order;         // [n_markets] processing order
  int n_markets;
  int C;                    // chains per market (the same for every market)
  unsigned int* item_ctr;   // [n_levels] work counters, zero at the start of the search
};

template <class R, int FORMULA>
__global__ void __launch_bounds__(256, 2) sa_level_batch_kernel(BatchArgs ba, int level) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ DevMarket sm_m;
  __shared__ SAState sm_st;
  __shared__ SAParams sm_sp;
  __shared__ unsigned long long s_wacc;
  __shared__ bool s_last;
  __shared__ int s_item;
  int cur = -1;
  bool staged = true;   // whether the current market's staging completed (else its items run no step)
  const long long total = (long long)ba.n_markets * ba.C;
  for (;;) {
    if (threadIdx.x == 0) s_item = (int)atomicAdd(ba.item_ctr + level, 1u);
    __syncthreads();
    const int item = s_item;
    if (item >= total) break;
    const int j = ba.order[item / ba.C], c = item % ba.C;
    if (j != cur) {
      if (threadIdx.x == 0) { sm_m = ba.mk[j]; sm_st = ba.st[j]; sm_sp = ba.sp[j]; }
      __syncthreads();
      CtaSmemS<R> cs0 = carve_cta<R>(smem, sm_m);
      staged = stage_market_cta<R>(cs0, sm_m);
      cur = j;
    }
    const DevMarket& m = sm_m;
    CtaSmemS<R> cs = carve_cta<R>(smem, m);
    const InstrView<R> capB = instr_view<R>(cs.cap, m.n_cap_pad);
    const InstrView<R> swpB = instr_view<R>(cs.swp, m.n_swp_pad);
    CtaScratch<R> sc = cta_scratch<R>(cs.scratch, m);
    cta_chain_level<R, FORMULA, false>(m, sm_st, sm_sp, c, level, cs, capB, swpB, sc, &s_wacc, &s_last, nullptr,
                                       staged);
  }
}

// f(x0), T0 and the first start point of every market of the batch (one CTA per market).
template <class R, int FORMULA>
__global__ void __launch_bounds__(256, 2) sa_start_batch_kernel(BatchArgs ba) {
  typedef typename ObjOf<R>::T O;
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ DevMarket sm_m;
  const int j = blockIdx.x;
  if (threadIdx.x == 0) sm_m = ba.mk[j];
  __syncthreads();
  const DevMarket& m = sm_m;
  const SAState st = ba.st[j];
  const SAParams sp = ba.sp[j];
  CtaSmemS<R> cs = carve_cta<R>(smem, m);
  const double x0 = threadIdx.x < (unsigned)sp.P ? (double)(R)sp.x0[threadIdx.x] : 0.0;
  if (!stage_market_cta<R>(cs, m)) {
    sa_start_write(st, sp, threadIdx.x, x0, __longlong_as_double(0x7ff0000000000000LL));
    return;
  }
  const InstrView<R> capB = instr_view<R>(cs.cap, m.n_cap_pad);
  const InstrView<R> swpB = instr_view<R>(cs.swp, m.n_swp_pad);
  CtaScratch<R> sc = cta_scratch<R>(cs.scratch, m);
  if (threadIdx.x < kMaxParam) sc.xs[threadIdx.x] = (R)x0;
  __syncthreads();
  const double f0 = obj_to_double(cta_objective<R, FORMULA>(m, capB, swpB, *cs.quad, sc, (O*)cs.red, nullptr));
  sa_start_write(st, sp, threadIdx.x, x0, f0);
}

// The best point ever accepted in each market of the batch (one CTA per market).
__global__ void sa_final_batch_kernel(BatchArgs ba) {
  const SAState st = ba.st[blockIdx.x];
  const SAParams sp = ba.sp[blockIdx.x];
  __shared__ double sf[32];
  __shared__ int sc[32];
  double bf = __longlong_as_double(0x7ff0000000000000LL);
  int bc = 0x7fffffff;
  for (int c = threadIdx.x; c < sp.C; c += blockDim.x)
    if (lex_less(st.fb[c], c, bf, bc)) { bf = st.fb[c]; bc = c; }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const double of = __shfl_xor_sync(0xffffffffu, bf, off);
    const int oc = __shfl_xor_sync(0xffffffffu, bc, off);
    if (lex_less(of, oc, bf, bc)) { bf = of; bc = oc; }
  }
  if (lane == 0) { sf[warp] = bf; sc[warp] = bc; }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
      if (lex_less(sf[w], sc[w], sf[0], sc[0])) { sf[0] = sf[w]; sc[0] = sc[w]; }
    st.best_f[0] = sf[0];
  }
  __syncthreads();
  if (threadIdx.x < (unsigned)sp.P) st.best_x[threadIdx.x] = st.xb[(size_t)sc[0] * sp.P + threadIdx.x];
}

// ====================================================================== adjoint (caplet markets)
// One warp per point; shared-memory plan: [caplet block][quadrature table]
// [W x (warp scratch, adjoint scratch)][tail].
template <class R>
__host__ __device__ inline uint32_t grad_warp_bytes(const DevMarket& m) {
  const uint32_t a = (uint32_t)warp_scratch_elems(m.NP, m.n_fwd) * sizeof(R);
  const uint32_t b = (uint32_t)adj_scratch_bytes(m.NP, m.n_fwd, sizeof(R));
  return ((a + 31u) & ~31u) + ((b + 31u) & ~31u);
}

template <class R>
__host__ __device__ inline uint32_t smem_bytes_grad(const DevMarket& m, int W) {
  return instr_block_bytes<R>(m.n_cap_pad) + (uint32_t)sizeof(QuadTab<R>) + (uint32_t)W * grad_warp_bytes<R>(m) + 512;
}

template <class R, int MODEL, int FORMULA>
__global__ void grad_kernel(DevMarket m, const double* __restrict__ X, long long n, double* __restrict__ f,
                            double* __restrict__ G) {
  extern __shared__ __align__(128) unsigned char smem[];
  const int W = blockDim.x >> 5, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  void* cap = smem;
  QuadTab<R>* quad = (QuadTab<R>*)(smem + instr_block_bytes<R>(m.n_cap_pad));
  unsigned char* wbase = (unsigned char*)quad + sizeof(QuadTab<R>) + (size_t)warp * grad_warp_bytes<R>(m);
  uint64_t* mbar = (uint64_t*)((unsigned char*)quad + sizeof(QuadTab<R>) + (size_t)W * grad_warp_bytes<R>(m));
  if (!stage_to_smem2(cap, cap_block<R>(m), instr_block_bytes<R>(m.n_cap_pad), quad, quad_block<R>(m),
                      (uint32_t)sizeof(QuadTab<R>), mbar, m.err)) {
    nan_outputs((long long)blockIdx.x * W + warp, (long long)gridDim.x * W, n, lane, 32, f, G, m.n_param, nullptr, 0);
    return;
  }
  const InstrView<R> capB = instr_view<R>(cap, m.n_cap_pad);
  WarpScratch<R> ws = warp_scratch<R>((R*)wbase, m.NP, m.n_fwd);
  const uint32_t wbytes = ((uint32_t)warp_scratch_elems(m.NP, m.n_fwd) * sizeof(R) + 31u) & ~31u;
  AdjScratch<R> as = adj_scratch<R>(wbase + wbytes, m.NP, m.n_fwd);
  for (long long i = (long long)blockIdx.x * W + warp; i < n; i += (long long)gridDim.x * W) {
    if (lane < kMaxParam) ws.xs[lane] = lane < m.n_param ? (R)X[i * m.n_param + lane] : R(0);
    __syncwarp();
    warp_objective_grad<R, MODEL, FORMULA>(m, capB, *quad, ws, as, lane, f + i, G + i * m.n_param);
  }
}

// ====================================================================== adjoint (markets with swaptions)
// One CTA (256 threads) per point, grid-stride, FP64.  Shared memory: the forward CTA plan with the
// forms' partials in their own region (m.qf_own = 1, set by the launcher), then the adjoint scratch.
__host__ __device__ inline uint32_t smem_bytes_grad_cta(const DevMarket& m) {
  return ((smem_bytes_cta<double>(m) + 63u) & ~63u) + grad_scratch_bytes_cta(m);
}

template <int FORMULA>
__global__ void __launch_bounds__(256, 1) grad_cta_kernel(DevMarket m, const double* __restrict__ X, long long n,
                                                       double* __restrict__ f, double* __restrict__ G) {
  extern __shared__ __align__(128) unsigned char smem[];
  CtaSmemS<double> cs = carve_cta<double>(smem, m);
  if (!stage_market_cta<double>(cs, m)) {
    nan_outputs(blockIdx.x, gridDim.x, n, threadIdx.x, blockDim.x, f, G, m.n_param, nullptr, 0);
    return;
  }
  const GradScratchS gs = grad_scratch_cta(smem + ((smem_bytes_cta<double>(m) + 63u) & ~63u), m);
  const InstrView<double> capB = instr_view<double>(cs.cap, m.n_cap_pad);
  const InstrView<double> swpB = instr_view<double>(cs.swp, m.n_swp_pad);
  CtaScratch<double> sc = cta_scratch<double>(cs.scratch, m);
  for (long long i = blockIdx.x; i < n; i += gridDim.x) {
    if (threadIdx.x < kMaxParam)
      sc.xs[threadIdx.x] = threadIdx.x < (unsigned)m.n_param ? X[i * m.n_param + threadIdx.x] : 0.0;
    __syncthreads();
    cta_objective_grad<FORMULA>(m, capB, swpB, *cs.quad, sc, (double*)cs.red, gs, f + i, G + i * m.n_param);
  }
}

// ====================================================================== Nelder-Mead polish
// Caplet markets: one warp (CTA of 32 threads) per start point, grid-stride; shared memory: the
// market staged as for the FP64 objective, then the simplex.  X is updated in place.
template <int MODEL, int FORMULA>
__global__ void nm_kernel(DevMarket m, double* X, long long n, int max_iter, double step, double ftol, double* f,
                          int* evals) {
  extern __shared__ __align__(128) unsigned char smem[];
  const int lane = threadIdx.x & 31;
  CtaSmem<double> cs = carve<double>(smem, m, 1);
  if (!stage_market<double>(cs, m, false)) {
    nan_outputs(blockIdx.x, gridDim.x, n, lane, 32, f, X, m.n_param, nullptr, 0);
    return;
  }
  const InstrView<double> capB = instr_view<double>(cs.cap, m.n_cap_pad);
  WarpScratch<double> ws = warp_scratch<double>((double*)cs.scratch, m.NP, m.n_fwd);
  const NmTeam team = nm_team((double*)(smem + ((smem_bytes<double>(m, 1) + 15u) & ~15u)));
  const int P = m.n_param;
  auto eval = [&](const double* x) {
    if (lane < kMaxParam) ws.xs[lane] = lane < P ? x[lane] : 0.0;
    __syncwarp();
    const double v = obj_to_double(warp_objective<double, MODEL, FORMULA>(m, capB, *cs.quad, ws, lane, nullptr));
    __syncwarp();
    return v;
  };
  auto sync = []() { __syncwarp(); };
  for (long long i = blockIdx.x; i < n; i += gridDim.x)
    nelder_mead(m, team, X + i * P, max_iter, step, ftol, lane, eval, sync, X + i * P, f + i,
                evals ? evals + i : nullptr);
}

// Markets with swaptions: one CTA (256 threads) per start point.
template <int FORMULA>
__global__ void __launch_bounds__(256, 1) nm_cta_kernel(DevMarket m, double* X, long long n, int max_iter,
                                                     double step, double ftol, double* f, int* evals) {
  extern __shared__ __align__(128) unsigned char smem[];
  CtaSmemS<double> cs = carve_cta<double>(smem, m);
  if (!stage_market_cta<double>(cs, m)) {
    nan_outputs(blockIdx.x, gridDim.x, n, threadIdx.x, blockDim.x, f, X, m.n_param, nullptr, 0);
    return;
  }
  const InstrView<double> capB = instr_view<double>(cs.cap, m.n_cap_pad);
  const InstrView<double> swpB = instr_view<double>(cs.swp, m.n_swp_pad);
  CtaScratch<double> sc = cta_scratch<double>(cs.scratch, m);
  const NmTeam team = nm_team((double*)(smem + ((smem_bytes_cta<double>(m) + 15u) & ~15u)));
  const int P = m.n_param, t = threadIdx.x;
  auto eval = [&](const double* x) {
    if (t < kMaxParam) sc.xs[t] = t < P ? x[t] : 0.0;
    __syncthreads();
    return obj_to_double(cta_objective<double, FORMULA, false>(m, capB, swpB, *cs.quad, sc, (double*)cs.red, nullptr));
  };
  auto sync = []() { __syncthreads(); };
  for (long long i = blockIdx.x; i < n; i += gridDim.x)
    nelder_mead(m, team, X + i * P, max_iter, step, ftol, t, eval, sync, X + i * P, f + i,
                evals ? evals + i : nullptr);
}

}  // namespace sabr
