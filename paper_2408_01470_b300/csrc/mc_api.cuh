// C-ABI of the Monte Carlo pricer (include/sabr_lmm.h: sabr_lmm_mc_*), included by api.cu.
// Preparation (once per plan, host C++ in FP64): the time grid (every interval between fixings cut
// into ceil(len / dt) equal steps), the instruments sorted by fixing, and the model constants:
// the correlation matrix of (W, Z) from Eqs. (rhoij), (thetaij), (phiij), repaired to the nearest
// correlation matrix in the spectral sense when it is indefinite (negative eigenvalues set to
// zero, rows of S Lambda^(1/2) scaled to unit length; eigenvectors by cyclic Jacobi rotations), and
// its semi-definite Cholesky factor (a pivot at or below 1e-12 ends its column).  Launch: the path
// kernel (every step of every path) and the reduction kernel, stream-ordered.  Mercurio & Morini:
// the (M + 1) x (M + 1) matrix of (Z, W) with corr(W_i, Z) = phi_i, treated the same way.
#pragma once
#include "mc.cuh"

struct sabr_lmm_mc_plan {
  int device = 0;
  int prec = SABR_LMM_FP32;
  int grid = 0;
  int threads = 128;            // paths per CTA
  int n_cap = 0, n_swp = 0;
  McArgs args{};
  McConsts<double> c64{};
  McConsts<float> c32{};
  void* buf = nullptr;          // device: time grid, instruments, partial sums
  double* out = nullptr;        // device: price [ni], stderr [ni]
  long long* nbad = nullptr;    // device
  // host copies for re-deriving constants at other correlation parameters (the annealer)
  int M = 0;
  std::vector<double> tau;
  std::vector<int> cap_order, swp_order;   // sorted position -> the caller's index
};

namespace {

// Spectral repair of a symmetric n x n matrix C (row-major) into a correlation matrix, in place,
// when it has a negative eigenvalue.  Returns whether it was repaired.
bool mc_repair(std::vector<double>& C, int n) {
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
        // the rotation that zeroes A[p][q]: t = tan(angle) from cot(2 angle) = (A_qq - A_pp) / (2 A_pq)
        const double cot2 = (A[(size_t)q * n + q] - A[(size_t)p * n + p]) / (2.0 * apq);
        const double t = (cot2 >= 0.0 ? 1.0 : -1.0) / (std::fabs(cot2) + std::sqrt(cot2 * cot2 + 1.0));
        const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < n; ++k) {
          const double x = A[(size_t)k * n + p], y = A[(size_t)k * n + q];
          A[(size_t)k * n + p] = c * x - s * y;
          A[(size_t)k * n + q] = s * x + c * y;
        }
        for (int k = 0; k < n; ++k) {
          const double x = A[(size_t)p * n + k], y = A[(size_t)q * n + k];
          A[(size_t)p * n + k] = c * x - s * y;
          A[(size_t)q * n + k] = s * x + c * y;
        }
        for (int k = 0; k < n; ++k) {
          const double x = S[(size_t)k * n + p], y = S[(size_t)k * n + q];
          S[(size_t)k * n + p] = c * x - s * y;
          S[(size_t)k * n + q] = s * x + c * y;
        }
      }
  }
  bool neg = false;
  for (int i = 0; i < n; ++i) neg = neg || A[(size_t)i * n + i] < 0.0;
  if (!neg) return false;
  std::vector<double> B((size_t)n * n);
  for (int i = 0; i < n; ++i) {
    double nrm = 0.0;
    for (int k = 0; k < n; ++k) {
      const double v = S[(size_t)i * n + k] * std::sqrt(std::max(A[(size_t)k * n + k], 0.0));
      B[(size_t)i * n + k] = v;
      nrm += v * v;
    }
    const double inv = 1.0 / std::sqrt(nrm);
    for (int k = 0; k < n; ++k) B[(size_t)i * n + k] *= inv;
  }
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      double v = 0.0;
      for (int k = 0; k < n; ++k) v += B[(size_t)i * n + k] * B[(size_t)j * n + k];
      C[(size_t)i * n + j] = v;
    }
  return true;
}

// The model constants of one parameter point: the correlation matrix in u-order (u = M - 1 - i;
// row 2u is W_i, row 2u + 1 is Z_i) from eta1, lambda1, eta2, lambda2, lambda3 (y[0..4] when y is
// given, else the description's), repaired when indefinite, its Cholesky factor, and the
// per-forward constants; in FP64 and FP32.
void mc_build_consts(const sabr_lmm_mc_desc* d, int M, const double* tau, const double* y, McConsts<double>& c64,
                     McConsts<float>& c32) {
  const double eta1 = y ? y[0] : d->eta1, lambda1 = y ? y[1] : d->lambda1, eta2 = y ? y[2] : d->eta2;
  const double lambda2 = y ? y[3] : d->lambda2, lambda3 = y ? y[4] : d->lambda3;
  const bool mm = d->model == SABR_LMM_MODEL_MERCURIO_MORINI;
  // Mercurio & Morini: row 0 is Z, row 1 + u is W of forward M - 1 - u; corr(W_i, Z) = phi_i
  const int n = mm ? M + 1 : 2 * M;
  std::vector<double> Cm((size_t)n * n);
  for (int r = 0; r < n && mm; ++r)
    for (int c = 0; c < n; ++c) {
      double v;
      if (r == 0 && c == 0) v = 1.0;
      else if (r == 0 || c == 0) v = d->phi[M - (r + c)];
      else v = eta1 + (1.0 - eta1) * std::exp(-lambda1 * std::fabs(d->T[M - r] - d->T[M - c]));
      Cm[(size_t)r * n + c] = v;
    }
  for (int r = 0; r < n && !mm; ++r)
    for (int c = 0; c < n; ++c) {
      const int i = M - 1 - r / 2, j = M - 1 - c / 2;
      const bool wr = (r & 1) == 0, wc = (c & 1) == 0;
      const double dT = std::fabs(d->T[i] - d->T[j]);
      double v;
      if (wr && wc) v = eta1 + (1.0 - eta1) * std::exp(-lambda1 * dT);
      else if (!wr && !wc) v = eta2 + (1.0 - eta2) * std::exp(-lambda2 * dT);
      else {   // corr(W_a, Z_b) = sign(phi_aa) sqrt(|phi_aa phi_bb|) e^{-lambda3 |T_a - T_b|}
        const int fa = wr ? i : j, fb = wr ? j : i;
        v = (d->phi[fa] < 0.0 ? -1.0 : 1.0) * std::sqrt(std::fabs(d->phi[fa] * d->phi[fb])) * std::exp(-lambda3 * dT);
      }
      Cm[(size_t)r * n + c] = v;
    }
  mc_repair(Cm, n);
  std::vector<double> L((size_t)n * n, 0.0);
  for (int j = 0; j < n; ++j) {
    double dd = Cm[(size_t)j * n + j];
    for (int k = 0; k < j; ++k) dd -= L[(size_t)j * n + k] * L[(size_t)j * n + k];
    if (!(dd > 1e-12)) continue;
    dd = std::sqrt(dd);
    L[(size_t)j * n + j] = dd;
    for (int i = j + 1; i < n; ++i) {
      double t = Cm[(size_t)i * n + j];
      for (int k = 0; k < j; ++k) t -= L[(size_t)i * n + k] * L[(size_t)j * n + k];
      L[(size_t)i * n + j] = t / dd;
    }
  }
  c64 = McConsts<double>{};
  for (int r = 0; r < n; ++r)
    for (int c = 0; c < n; ++c) c64.L[r * kMcRows + c] = L[(size_t)r * n + c];
  for (int u = 0; u < M; ++u) {
    const int i = M - 1 - u;
    for (int v = 0; v < M; ++v) {
      c64.rho[u * kMcMaxFwd + v] = mm ? Cm[(size_t)(1 + u) * n + 1 + v] : Cm[(size_t)(2 * u) * n + 2 * v];
      c64.phi[u * kMcMaxFwd + v] = mm ? 0.0 : Cm[(size_t)(2 * u) * n + 2 * v + 1];
    }
    c64.tau[u] = tau[i];
    c64.sig[u] = mm ? d->sigma[0] : d->sigma[i];
    c64.hs2[u] = 0.5 * c64.sig[u] * c64.sig[u];
    c64.F0[u] = (d->P[i] / d->P[i + 1] - 1.0) / tau[i];
    c64.lnV0[u] = mm ? 0.0 : std::log(d->alpha[i]);
    c64.alpha[u] = d->alpha[i];
  }
  const double* src = (const double*)&c64;
  float* dst = (float*)&c32;
  static_assert(sizeof(McConsts<double>) == 2 * sizeof(McConsts<float>), "the two layouts must match element by element");
  for (size_t k = 0; k < sizeof(McConsts<double>) / sizeof(double); ++k) dst[k] = (float)src[k];
}

std::string mc_validate(const sabr_lmm_mc_desc* d, const sabr_lmm_mc_opts* o) {
  if (!d || !o) return "desc and opts are required";
  if (d->n_fwd < 1 || d->n_fwd > 120) return "n_fwd must be in [1, 120]";
  if (!d->T || !d->P || !d->alpha || !d->sigma || !d->phi) return "T, P, alpha, sigma and phi are required";
  for (int k = 0; k <= d->n_fwd; ++k) {
    if (!(d->T[k] > 0.0) || !std::isfinite(d->T[k]) || (k > 0 && !(d->T[k] > d->T[k - 1])))
      return "T must be finite, > 0 and strictly increasing";
    if (!(d->P[k] > 0.0) || !std::isfinite(d->P[k])) return "P must be finite and > 0";
  }
  if (!(d->beta >= 0.0 && d->beta <= 1.0)) return "beta must be in [0, 1]";
  if (d->model != SABR_LMM_MODEL_SMILE && d->model != SABR_LMM_MODEL_MERCURIO_MORINI)
    return "model must be 0 (Hagan) or 2 (Mercurio & Morini)";
  for (int i = 0; i < d->n_fwd; ++i) {
    if (!(d->alpha[i] > 0.0) || !std::isfinite(d->alpha[i])) return "alpha must be finite and > 0";
    if (!(d->sigma[i] >= 0.0) || !std::isfinite(d->sigma[i])) return "sigma must be finite and >= 0";
    if (!(std::fabs(d->phi[i]) <= 1.0)) return "phi must be in [-1, 1]";
  }
  if (!(d->eta1 >= 0.0 && d->eta1 <= 1.0 && d->eta2 >= 0.0 && d->eta2 <= 1.0)) return "eta1, eta2 must be in [0, 1]";
  if (!(d->lambda1 >= 0.0 && d->lambda2 >= 0.0 && d->lambda3 >= 0.0) || !std::isfinite(d->lambda1 + d->lambda2 + d->lambda3))
    return "lambda1..3 must be finite and >= 0";
  if (d->n_cap < 0 || d->n_swp < 0 || d->n_cap + d->n_swp < 1) return "need at least one instrument";
  if (d->n_cap + d->n_swp > 4096) return "at most 4096 instruments";
  if (d->n_cap > 0 && (!d->cap_fwd || !d->cap_K)) return "cap_fwd and cap_K are required";
  if (d->n_swp > 0 && (!d->swp_start || !d->swp_end || !d->swp_K)) return "swp_start, swp_end and swp_K are required";
  for (int c = 0; c < d->n_cap; ++c) {
    if (d->cap_fwd[c] < 0 || d->cap_fwd[c] >= d->n_fwd) return "cap_fwd out of range";
    if (!(d->cap_K[c] >= 0.0) || !std::isfinite(d->cap_K[c])) return "cap_K must be finite and >= 0";
  }
  for (int c = 0; c < d->n_swp; ++c) {
    if (d->swp_start[c] < 0 || d->swp_end[c] <= d->swp_start[c] || d->swp_end[c] > d->n_fwd)
      return "swaption window out of range";
    if (!(d->swp_K[c] >= 0.0) || !std::isfinite(d->swp_K[c])) return "swp_K must be finite and >= 0";
  }
  if (o->n_paths < 1 || o->n_paths > (1ll << 40)) return "n_paths must be in [1, 2^40]";
  if (!(o->dt > 0.0) || !std::isfinite(o->dt)) return "dt must be finite and > 0";
  if (o->prec != SABR_LMM_FP64 && o->prec != SABR_LMM_FP32) return "prec must be FP64 or FP32";
  if (o->grid < 0) return "grid must be >= 0";
  return std::string();
}

}  // namespace

namespace {
// shrink: CTAs smaller than the largest when the paths do not fill one per SM (a pricing alone on the
// GPU); the annealer's many concurrent launches keep the largest, so that an SM runs one CTA.
sabr_lmm_status mc_prepare(const sabr_lmm_mc_desc* d, const sabr_lmm_mc_opts* o, void* stream, sabr_lmm_mc_plan** out,
                           bool shrink) {
  if (!out) return fail(SABR_LMM_EINVAL, "out is required");
  *out = nullptr;
  const std::string e0 = mc_validate(d, o);
  if (!e0.empty()) return fail(SABR_LMM_EINVAL, "mc: " + e0);
  // forwards simulated: every forward an instrument fixes or reads
  int M = 0;
  for (int c = 0; c < d->n_cap; ++c) M = std::max(M, d->cap_fwd[c] + 1);
  for (int c = 0; c < d->n_swp; ++c) M = std::max(M, d->swp_end[c]);
  if (M > kMcMaxFwd) return fail(SABR_LMM_ENOTSUP, "mc: the instruments reach more than 16 forwards");
  std::vector<int> nsteps(M);
  std::vector<double> h(M), tau(M);
  long long total = 0;
  for (int k = 0; k < M; ++k) {
    const double len = d->T[k] - (k == 0 ? 0.0 : d->T[k - 1]);
    nsteps[k] = std::max(1, (int)std::ceil(len / o->dt - 1e-9));
    h[k] = len / nsteps[k];
    tau[k] = d->T[k + 1] - d->T[k];
    total += nsteps[k];
  }
  if (total > (1 << 30)) return fail(SABR_LMM_EINVAL, "mc: too many time steps");
  sabr_lmm_mc_plan* p = new sabr_lmm_mc_plan();
  cudaGetDevice(&p->device);
  p->prec = o->prec;
  p->n_cap = d->n_cap;
  p->n_swp = d->n_swp;
  p->M = M;
  p->tau = tau;
  mc_build_consts(d, M, tau.data(), nullptr, p->c64, p->c32);
  // instruments sorted by fixing (stable), with their output slots
  std::vector<int> ci(d->n_cap), si(d->n_swp);
  for (int c = 0; c < d->n_cap; ++c) ci[c] = c;
  for (int c = 0; c < d->n_swp; ++c) si[c] = c;
  std::stable_sort(ci.begin(), ci.end(), [&](int x, int y) { return d->cap_fwd[x] < d->cap_fwd[y]; });
  // swaptions by expiry, then by swap end: at a fixing one running discount product serves them all
  std::stable_sort(si.begin(), si.end(), [&](int x, int y) {
    return d->swp_start[x] != d->swp_start[y] ? d->swp_start[x] < d->swp_start[y] : d->swp_end[x] < d->swp_end[y];
  });
  std::vector<int> cap_lo(M + 1, 0), swp_lo(M + 1, 0), cap_out(d->n_cap), swp_out(d->n_swp), swp_b(d->n_swp);
  std::vector<double> cap_K(d->n_cap), swp_K(d->n_swp);
  std::vector<float> cap_K32(d->n_cap), swp_K32(d->n_swp), tau32(M);
  for (int c = 0; c < d->n_cap; ++c) {
    cap_out[c] = ci[c];
    cap_K[c] = d->cap_K[ci[c]];
    cap_K32[c] = (float)cap_K[c];
    cap_lo[d->cap_fwd[ci[c]] + 1]++;
  }
  for (int c = 0; c < d->n_swp; ++c) {
    swp_out[c] = si[c];
    swp_K[c] = d->swp_K[si[c]];
    swp_K32[c] = (float)swp_K[c];
    swp_b[c] = d->swp_end[si[c]];
    swp_lo[d->swp_start[si[c]] + 1]++;
  }
  for (int k = 0; k < M; ++k) { cap_lo[k + 1] += cap_lo[k]; swp_lo[k + 1] += swp_lo[k]; }
  p->cap_order = ci;
  p->swp_order = si;
  const int ni = d->n_cap + d->n_swp;
  // CTA size: the largest (up to 512 paths in FP32, 128 in FP64) whose per-warp sums fit in a
  // CTA's shared memory.  Grid: enough CTAs for every path, at most one wave of 512 paths per SM in
  // FP32 (8 CTAs per SM in FP64), persistent beyond.
  const bool f64 = o->prec == SABR_LMM_FP64;
  const int tmax = f64 ? mc_max_threads<double>() : mc_max_threads<float>();
  int nsm = 148;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, p->device);
  // a pricing alone on the GPU: the paths split evenly over the rounds of one CTA per SM, in whole
  // warps (the rounds a largest CTA would need, each of fewer paths: the last round is not mostly
  // empty, and fewer paths than one largest CTA per SM spread over all SMs)
  p->threads = tmax;
  if (shrink) {
    const long long per_round = (long long)nsm * tmax;
    const long long rounds = (o->n_paths + per_round - 1) / per_round;
    const long long per_cta = (o->n_paths + nsm * rounds - 1) / (nsm * rounds);
    p->threads = (int)std::min<long long>(tmax, std::max<long long>(32, (per_cta + 31) / 32 * 32));
  }
  const int t_req = p->threads;
  // (the annealer's batch kernel also stages one set's constants in shared memory)
  const size_t extra = shrink ? 0 : ((f64 ? sizeof(McConsts<double>) : sizeof(McConsts<float>)) + 127) & ~(size_t)127;
  while (p->threads > 32 && mc_smem_bytes(ni, p->threads) + extra > kMcSmemMax)
    p->threads = std::max(32, p->threads / 64 * 32);
  const long long need = (o->n_paths + p->threads - 1) / p->threads;
  // FP32: one CTA per SM, looping over its rounds (as many CTAs per SM as the shared-memory limit
  // took from the CTA size); FP64: up to 8 CTAs per SM
  const long long cap = (long long)nsm * (f64 ? 8 : std::max(1, t_req / p->threads));
  p->grid = (int)std::min<long long>(need, o->grid > 0 ? o->grid : cap);
  for (int k = 0; k < M; ++k) tau32[k] = (float)tau[k];
  // device buffer: nsteps, h, tau, cap_lo, swp_lo, cap_out, swp_out, swp_b, cap_K, swp_K, their FP32
  // copies, part, bad, out, nbad
  Arena A;
  const size_t o_ns = A.take(M * 4), o_h = A.take(M * 8), o_tau = A.take(M * 8), o_clo = A.take((M + 1) * 4),
               o_slo = A.take((M + 1) * 4), o_cout = A.take(d->n_cap * 4), o_sout = A.take(d->n_swp * 4),
               o_sb = A.take(d->n_swp * 4), o_cK = A.take(d->n_cap * 8), o_sK = A.take(d->n_swp * 8),
               o_cK32 = A.take(d->n_cap * 4), o_sK32 = A.take(d->n_swp * 4), o_tau32 = A.take(M * 4),
               o_part = A.take((size_t)p->grid * ni * 16), o_bad = A.take((size_t)p->grid * 8),
               o_out = A.take((size_t)ni * 16), o_nbad = A.take(8);
  std::vector<unsigned char> host(A.size, 0);
  auto put = [&](size_t off, const void* src, size_t bytes) { if (bytes) std::memcpy(host.data() + off, src, bytes); };
  put(o_ns, nsteps.data(), M * 4); put(o_h, h.data(), M * 8); put(o_tau, tau.data(), M * 8);
  put(o_clo, cap_lo.data(), (M + 1) * 4); put(o_slo, swp_lo.data(), (M + 1) * 4);
  put(o_cout, cap_out.data(), d->n_cap * 4); put(o_sout, swp_out.data(), d->n_swp * 4);
  put(o_sb, swp_b.data(), d->n_swp * 4); put(o_cK, cap_K.data(), d->n_cap * 8); put(o_sK, swp_K.data(), d->n_swp * 8);
  put(o_cK32, cap_K32.data(), d->n_cap * 4); put(o_sK32, swp_K32.data(), d->n_swp * 4); put(o_tau32, tau32.data(), M * 4);
  if (cudaMalloc(&p->buf, A.size) != cudaSuccess) {
    delete p;
    return fail(SABR_LMM_ENOMEM, "mc: cudaMalloc of the plan's buffers failed");
  }
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaMemcpyAsync(p->buf, host.data(), A.size, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    cudaFree(p->buf);
    delete p;
    return fail(SABR_LMM_ECUDA, std::string("mc: ") + cudaGetErrorString(e));
  }
  char* b = (char*)p->buf;
  McArgs& a = p->args;
  a.M = M; a.n_cap = d->n_cap; a.n_swp = d->n_swp; a.beta = d->beta; a.P0 = d->P[0];
  a.model = d->model;
  a.n_int = 1;   // the simulation ends at the last fixing an instrument needs
  for (int c = 0; c < d->n_cap; ++c) a.n_int = std::max(a.n_int, d->cap_fwd[c] + 1);
  for (int c = 0; c < d->n_swp; ++c) a.n_int = std::max(a.n_int, d->swp_start[c] + 1);
  a.nsteps = (const int*)(b + o_ns); a.h = (const double*)(b + o_h); a.tau64 = (const double*)(b + o_tau);
  a.cap_lo = (const int*)(b + o_clo); a.swp_lo = (const int*)(b + o_slo);
  a.cap_out = (const int*)(b + o_cout); a.swp_out = (const int*)(b + o_sout); a.swp_b = (const int*)(b + o_sb);
  a.cap_K = (const double*)(b + o_cK); a.swp_K = (const double*)(b + o_sK);
  a.cap_K32 = (const float*)(b + o_cK32); a.swp_K32 = (const float*)(b + o_sK32); a.tau32 = (const float*)(b + o_tau32);
  a.seed = o->seed; a.n_paths = o->n_paths;
  a.part = (double*)(b + o_part); a.bad = (unsigned long long*)(b + o_bad);
  p->out = (double*)(b + o_out);
  p->nbad = (long long*)(b + o_nbad);
  const size_t sm = mc_smem_bytes(ni, p->threads);
  const bool mm = d->model == SABR_LMM_MODEL_MERCURIO_MORINI;
  e = o->prec == SABR_LMM_FP64 ? (mm ? raise_smem_limit(mc_path_kernel<double, true>, (uint32_t)sm)
                                     : raise_smem_limit(mc_path_kernel<double, false>, (uint32_t)sm))
                               : (mm ? raise_smem_limit(mc_path_kernel<float, true>, (uint32_t)sm)
                                     : raise_smem_limit(mc_path_kernel<float, false>, (uint32_t)sm));
  if (e != cudaSuccess) {
    cudaFree(p->buf);
    delete p;
    return fail(SABR_LMM_ECUDA, std::string("mc: ") + cudaGetErrorString(e));
  }
  *out = p;
  return SABR_LMM_OK;
}
}  // namespace

extern "C" sabr_lmm_status sabr_lmm_mc_prepare(const sabr_lmm_mc_desc* d, const sabr_lmm_mc_opts* o, void* stream,
                                               sabr_lmm_mc_plan** out) {
  return mc_prepare(d, o, stream, out, true);
}

extern "C" sabr_lmm_status sabr_lmm_mc_launch(sabr_lmm_mc_plan* p, double* price, double* stderr_out,
                                              long long* n_bad, void* stream) {
  if (!p) return fail(SABR_LMM_EINVAL, "plan is required");
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev != p->device) return fail(SABR_LMM_EINVAL, "mc: the plan belongs to another device");
  cudaStream_t s = (cudaStream_t)stream;
  const int ni = p->n_cap + p->n_swp;
  const size_t sm = mc_smem_bytes(ni, p->threads);
  const bool mm = p->args.model == SABR_LMM_MODEL_MERCURIO_MORINI;
  if (p->prec == SABR_LMM_FP64) {
    if (mm) mc_path_kernel<double, true><<<p->grid, p->threads, sm, s>>>(p->args, p->c64);
    else mc_path_kernel<double, false><<<p->grid, p->threads, sm, s>>>(p->args, p->c64);
  } else {
    if (mm) mc_path_kernel<float, true><<<p->grid, p->threads, sm, s>>>(p->args, p->c32);
    else mc_path_kernel<float, false><<<p->grid, p->threads, sm, s>>>(p->args, p->c32);
  }
  mc_reduce_kernel<<<(ni + 127) / 128, 128, 0, s>>>(p->args, p->grid, price ? price : p->out,
                                                      price ? stderr_out : p->out + ni, n_bad ? n_bad : p->nbad);
  CUDA_TRY(cudaGetLastError());
  return SABR_LMM_OK;
}

extern "C" void sabr_lmm_mc_plan_free(sabr_lmm_mc_plan* p) {
  if (!p) return;
  if (p->buf) cudaFree(p->buf);
  delete p;
}

extern "C" sabr_lmm_status sabr_lmm_mc_price(const sabr_lmm_mc_desc* d, const sabr_lmm_mc_opts* o, double* price,
                                             double* stderr_out, int64_t* n_bad, void* stream) {
  if (!price) return fail(SABR_LMM_EINVAL, "price is required");
  sabr_lmm_mc_plan* p = nullptr;
  sabr_lmm_status st = sabr_lmm_mc_prepare(d, o, stream, &p);
  if (st != SABR_LMM_OK) return st;
  const int ni = p->n_cap + p->n_swp;
  cudaStream_t s = (cudaStream_t)stream;
  st = sabr_lmm_mc_launch(p, nullptr, nullptr, nullptr, stream);
  std::vector<double> hout((size_t)2 * ni);
  long long hb = 0;
  cudaError_t e = cudaSuccess;
  if (st == SABR_LMM_OK) {
    e = cudaMemcpyAsync(hout.data(), p->out, (size_t)2 * ni * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hb, p->nbad, sizeof(long long), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  }
  sabr_lmm_mc_plan_free(p);
  if (st != SABR_LMM_OK) return st;
  if (e != cudaSuccess) return fail(SABR_LMM_ECUDA, std::string("mc: ") + cudaGetErrorString(e));
  std::memcpy(price, hout.data(), ni * sizeof(double));
  if (stderr_out) std::memcpy(stderr_out, hout.data() + ni, ni * sizeof(double));
  if (n_bad) *n_bad = hb;
  return SABR_LMM_OK;
}

// ====================================================================== SA over the Monte Carlo objective
namespace {

// Philox4x64-10 on the host (the counter-based generator of the annealer's uniforms, Salmon et al.
// SC'11), and the uniforms of one annealing step: word w of block b at counter (b, step, level,
// chain) under key (seed, 0), u = (x >> 11) 2^-53.
void philox4x64_10_host(const uint64_t ctr[4], uint64_t k0, uint64_t k1, uint64_t out[4]) {
  const uint64_t M0 = 0xD2E7470EE14C6C93ULL, M1 = 0xCA5A826395121157ULL;
  const uint64_t W0 = 0x9E3779B97F4A7C15ULL, W1 = 0xBB67AE8584CAA73BULL;
  uint64_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  for (int r = 0; r < 10; ++r) {
    const unsigned __int128 p0 = (unsigned __int128)M0 * c0, p1 = (unsigned __int128)M1 * c2;
    const uint64_t n0 = (uint64_t)(p1 >> 64) ^ c1 ^ k0, n2 = (uint64_t)(p0 >> 64) ^ c3 ^ k1;
    c0 = n0; c1 = (uint64_t)p1; c2 = n2; c3 = (uint64_t)p0;
    k0 += W0; k1 += W1;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

void sa_step_uniforms(uint64_t seed, uint64_t chain, int level, int step, int count, double* u) {
  for (int b = 0; 4 * b < count; ++b) {
    const uint64_t ctr[4] = {(uint64_t)b, (uint64_t)step, (uint64_t)level, chain};
    uint64_t o[4];
    philox4x64_10_host(ctr, seed, 0, o);
    for (int w = 0; w < 4 && 4 * b + w < count; ++w) u[4 * b + w] = (double)(o[w] >> 11) * 0x1.0p-53;
  }
}

}  // namespace

namespace {
// Worker threads that live for one search: run(n, fn) calls fn(i) for i in [0, n) spread over the
// workers and the caller, and returns when all are done.  Between calls a worker spins for a while
// (about a millisecond) before it sleeps, so that the next annealing step finds it awake: on a
// loaded host, waking sleeping threads took longer than the constants they were to build.
class McPool {
 public:
  explicit McPool(unsigned n_workers) {
    for (unsigned t = 0; t < n_workers; ++t) th_.emplace_back([this] { loop(); });
  }
  ~McPool() {
    {
      std::lock_guard<std::mutex> lk(mu_);
      stop_.store(true);
    }
    cv_.notify_all();
    for (auto& t : th_) t.join();
  }
  void run(int n, const std::function<void(int)>& fn) {
    fn_ = &fn;
    n_ = n;
    next_.store(0);
    busy_.store((int)th_.size());
    {
      std::lock_guard<std::mutex> lk(mu_);
      gen_.fetch_add(1, std::memory_order_release);
    }
    cv_.notify_all();
    drain();
    for (int k = 0; k < kSpin && busy_.load(std::memory_order_acquire) != 0; ++k) std::this_thread::yield();
    std::unique_lock<std::mutex> lk(mu_);
    done_.wait(lk, [this] { return busy_.load() == 0; });
  }

 private:
  static constexpr int kSpin = 20000;
  void drain() {
    for (int i = next_.fetch_add(1); i < n_; i = next_.fetch_add(1)) (*fn_)(i);
  }
  void loop() {
    unsigned long long seen = 0;
    for (;;) {
      for (int k = 0; k < kSpin && !stop_.load() && gen_.load(std::memory_order_acquire) == seen; ++k)
        std::this_thread::yield();
      {
        std::unique_lock<std::mutex> lk(mu_);
        cv_.wait(lk, [&] { return stop_.load() || gen_.load() != seen; });
        if (stop_.load()) return;
        seen = gen_.load();
      }
      drain();
      if (busy_.fetch_sub(1) == 1) {
        std::lock_guard<std::mutex> lk(mu_);
        done_.notify_one();
      }
    }
  }
  std::vector<std::thread> th_;
  std::mutex mu_;
  std::condition_variable cv_, done_;
  const std::function<void(int)>* fn_ = nullptr;
  int n_ = 0;
  std::atomic<int> next_{0}, busy_{0};
  std::atomic<unsigned long long> gen_{0};
  std::atomic<bool> stop_{false};
};
}  // namespace

extern "C" sabr_lmm_status sabr_lmm_mc_anneal(const sabr_lmm_mc_desc* d, const double* quote_vol,
                                              const sabr_lmm_mc_opts* mo, const sabr_lmm_mc_anneal_opts* o,
                                              sabr_lmm_mc_anneal_result* out, void* stream) {
  if (!quote_vol || !o || !out) return fail(SABR_LMM_EINVAL, "mc_anneal: quote_vol, opts and out are required");
  if (o->n_chains < 1 || o->n_chains > 4096 || o->n_levels < 1 || o->steps_per_level < 1)
    return fail(SABR_LMM_EINVAL, "mc_anneal: n_chains in [1, 4096], n_levels and steps_per_level >= 1 required");
  if (!(o->cooling > 0.0 && o->cooling <= 1.0) || !(o->step_frac > 0.0) || !(o->step_floor >= 0.0))
    return fail(SABR_LMM_EINVAL, "mc_anneal: cooling in (0, 1], step_frac > 0, step_floor >= 0 required");
  if (!o->lo || !o->hi || !o->free_mask) return fail(SABR_LMM_EINVAL, "mc_anneal: lo, hi and free_mask are required");
  for (int k = 0; k < 5; ++k) {
    const double ub = (k == 0 || k == 2) ? 1.0 : 1e6;
    if (!(o->lo[k] >= 0.0 && o->lo[k] <= o->hi[k] && o->hi[k] <= ub))
      return fail(SABR_LMM_EINVAL, "mc_anneal: the box must satisfy 0 <= lo <= hi (eta1, eta2 <= 1)");
    if (o->y0 && !(o->y0[k] >= o->lo[k] && o->y0[k] <= o->hi[k])) return fail(SABR_LMM_EINVAL, "mc_anneal: y0 outside the box");
  }
  const int ni = d ? d->n_cap + d->n_swp : 0;
  for (int k = 0; k < ni; ++k)
    if (!(quote_vol[k] > 0.0) || !std::isfinite(quote_vol[k])) return fail(SABR_LMM_EINVAL, "mc_anneal: quote_vol must be finite and > 0");
  sabr_lmm_mc_plan* p = nullptr;
  sabr_lmm_status st = mc_prepare(d, mo, stream, &p, false);
  if (st != SABR_LMM_OK) return st;
  const int C = o->n_chains, L = o->n_levels, N = o->steps_per_level, P = 5, M = p->M, G = p->grid;
  const bool f64 = p->prec == SABR_LMM_FP64;
  const size_t csz = f64 ? sizeof(McConsts<double>) : sizeof(McConsts<float>);
  cudaStream_t s = (cudaStream_t)stream;
  // device: the constants of C sets, their CTA sums and stopped paths, f, the market prices, and the
  // sorted instruments' quotes with the tenor grid; host (pinned): the constants and f
  Arena A;
  const size_t o_cs = A.take((size_t)C * csz), o_part = A.take((size_t)C * G * ni * 16), o_bad = A.take((size_t)C * G * 8),
               o_f = A.take((size_t)C * 8), o_mkt = A.take((size_t)ni * 8), o_vol = A.take((size_t)ni * 8),
               o_cf = A.take((size_t)p->n_cap * 4), o_sa = A.take((size_t)p->n_swp * 4),
               o_T = A.take((size_t)(d->n_fwd + 1) * 8), o_P = A.take((size_t)(d->n_fwd + 1) * 8);
  void* dbuf = nullptr;
  unsigned char* hcs = nullptr;
  double* hf = nullptr;
  const bool ok = cudaMalloc(&dbuf, A.size) == cudaSuccess &&
                  cudaMallocHost((void**)&hcs, (size_t)C * csz) == cudaSuccess &&
                  cudaMallocHost((void**)&hf, (size_t)C * 8) == cudaSuccess;
  char* b = (char*)dbuf;
  auto cleanup = [&]() {
    if (dbuf) cudaFree(dbuf);
    if (hcs) cudaFreeHost(hcs);
    if (hf) cudaFreeHost(hf);
    sabr_lmm_mc_plan_free(p);
  };
  if (!ok) {
    cleanup();
    return fail(SABR_LMM_ENOMEM, "mc_anneal: allocation of the search buffers failed");
  }
  std::vector<double> vol_sorted(ni);
  std::vector<int> cf_sorted(p->n_cap), sa_sorted(p->n_swp);
  for (int c = 0; c < p->n_cap; ++c) {
    vol_sorted[c] = quote_vol[p->cap_order[c]];
    cf_sorted[c] = d->cap_fwd[p->cap_order[c]];
  }
  for (int c = 0; c < p->n_swp; ++c) {
    vol_sorted[p->n_cap + c] = quote_vol[p->n_cap + p->swp_order[c]];
    sa_sorted[c] = d->swp_start[p->swp_order[c]];
  }
  cudaError_t e = cudaSuccess;
  auto put = [&](size_t off, const void* src, size_t bytes) {
    if (e == cudaSuccess && bytes) e = cudaMemcpyAsync(b + off, src, bytes, cudaMemcpyHostToDevice, s);
  };
  put(o_vol, vol_sorted.data(), ni * 8);
  put(o_cf, cf_sorted.data(), p->n_cap * 4);
  put(o_sa, sa_sorted.data(), p->n_swp * 4);
  put(o_T, d->T, (d->n_fwd + 1) * 8);
  put(o_P, d->P, (d->n_fwd + 1) * 8);
  McArgs ab = p->args;
  ab.part = (double*)(b + o_part);
  ab.bad = (unsigned long long*)(b + o_bad);
  if (e == cudaSuccess) {
    mc_market_kernel<<<(ni + 127) / 128, 128, 0, s>>>(ab, (const double*)(b + o_T), (const double*)(b + o_P),
                                                      (const int*)(b + o_cf), (const int*)(b + o_sa),
                                                      (const double*)(b + o_vol), (double*)(b + o_mkt));
    e = cudaGetLastError();
  }
  const size_t smb = f64 ? mc_batch_smem_bytes<double>(ni, p->threads) : mc_batch_smem_bytes<float>(ni, p->threads);
  const bool mmb = p->args.model == SABR_LMM_MODEL_MERCURIO_MORINI;
  if (e == cudaSuccess && smb > kMcSmemMax) e = cudaErrorInvalidValue;
  if (e == cudaSuccess)
    e = f64 ? (mmb ? raise_smem_limit(mc_path_batch_kernel<double, true>, (uint32_t)smb)
                   : raise_smem_limit(mc_path_batch_kernel<double, false>, (uint32_t)smb))
            : (mmb ? raise_smem_limit(mc_path_batch_kernel<float, true>, (uint32_t)smb)
                   : raise_smem_limit(mc_path_batch_kernel<float, false>, (uint32_t)smb));
  if (e != cudaSuccess) {
    cleanup();
    return fail(SABR_LMM_ECUDA, std::string("mc_anneal: ") + cudaGetErrorString(e));
  }
  // f_s of n points Y [n x 5]: constants on the host (threads), one batched launch (a CTA grid per
  // point, its constants staged in shared memory), f back
  const unsigned nthr = std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
  McPool pool(std::min<unsigned>(nthr - 1, (unsigned)std::max(0, C - 1)));
  auto evaluate = [&](const std::vector<double>& Y, int n, double* f) -> cudaError_t {
    const std::function<void(int)> work = [&](int i) {
      McConsts<double> c64;
      McConsts<float> c32;
      mc_build_consts(d, M, p->tau.data(), &Y[(size_t)i * P], c64, c32);
      if (f64) std::memcpy(hcs + (size_t)i * csz, &c64, csz);
      else std::memcpy(hcs + (size_t)i * csz, &c32, csz);
    };
    pool.run(n, work);
    cudaError_t ee = cudaMemcpyAsync(b + o_cs, hcs, (size_t)n * csz, cudaMemcpyHostToDevice, s);
    if (ee != cudaSuccess) return ee;
    const dim3 grid(G, n);
    const McConsts<double>* c64 = (const McConsts<double>*)(b + o_cs);
    const McConsts<float>* c32 = (const McConsts<float>*)(b + o_cs);
    if (f64) {
      if (mmb) mc_path_batch_kernel<double, true><<<grid, p->threads, smb, s>>>(ab, c64);
      else mc_path_batch_kernel<double, false><<<grid, p->threads, smb, s>>>(ab, c64);
    } else {
      if (mmb) mc_path_batch_kernel<float, true><<<grid, p->threads, smb, s>>>(ab, c32);
      else mc_path_batch_kernel<float, false><<<grid, p->threads, smb, s>>>(ab, c32);
    }
    mc_objective_kernel<<<(n + 3) / 4, 128, 0, s>>>(ab, G, n, (const double*)(b + o_mkt), (double*)(b + o_f));
    if ((ee = cudaGetLastError()) != cudaSuccess) return ee;
    if ((ee = cudaMemcpyAsync(hf, b + o_f, (size_t)n * 8, cudaMemcpyDeviceToHost, s)) != cudaSuccess) return ee;
    if ((ee = cudaStreamSynchronize(s)) != cudaSuccess) return ee;
    for (int i = 0; i < n; ++i) f[i] = (hf[i] == hf[i]) ? hf[i] : HUGE_VAL;
    return cudaSuccess;
  };
  const auto t_start = std::chrono::steady_clock::now();
  // the annealing loop of Section 3 (as in the closed-form search): chains from a shared start
  // point, the best end point starts the next level, the best point ever accepted is returned
  std::vector<double> x0(P);
  for (int k = 0; k < P; ++k) x0[k] = o->y0 ? o->y0[k] : 0.5 * (o->lo[k] + o->hi[k]);
  double f0 = 0.0;
  if ((e = evaluate(x0, 1, &f0)) != cudaSuccess) {
    cleanup();
    return fail(SABR_LMM_ECUDA, std::string("mc_anneal: ") + cudaGetErrorString(e));
  }
  const double T0 = o->T0 > 0.0 ? o->T0 : ((std::isfinite(f0) && f0 > 0.0) ? f0 : 1.0);
  std::vector<double> xs = x0, X((size_t)C * P), Y((size_t)C * P), xb((size_t)C * P), fx(C), fy(C), fb(C, f0);
  for (int c = 0; c < C; ++c) std::copy(x0.begin(), x0.end(), xb.begin() + (size_t)c * P);
  double fs = f0, T = T0;
  std::vector<double> u(P + 1);
  for (int l = 0; l < L; ++l) {
    const double sf = std::max(o->step_frac * std::sqrt(T / T0), o->step_floor);
    for (int c = 0; c < C; ++c) {
      std::copy(xs.begin(), xs.end(), X.begin() + (size_t)c * P);
      fx[c] = fs;
    }
    for (int st2 = 0; st2 < N; ++st2) {
      std::vector<double> uacc(C);
      for (int c = 0; c < C; ++c) {
        sa_step_uniforms(o->seed, (uint64_t)c, l, st2, P + 1, u.data());
        for (int k = 0; k < P; ++k) {
          const double xk = X[(size_t)c * P + k];
          double v = xk;
          if (o->free_mask[k]) {
            v = xk + sf * (o->hi[k] - o->lo[k]) * (2.0 * u[k] - 1.0);
            if (v < o->lo[k]) v = 2.0 * o->lo[k] - v;
            if (v > o->hi[k]) v = 2.0 * o->hi[k] - v;
            v = std::min(std::max(v, o->lo[k]), o->hi[k]);
          }
          Y[(size_t)c * P + k] = v;
        }
        uacc[c] = u[P];
      }
      if ((e = evaluate(Y, C, fy.data())) != cudaSuccess) {
        cleanup();
        return fail(SABR_LMM_ECUDA, std::string("mc_anneal: ") + cudaGetErrorString(e));
      }
      for (int c = 0; c < C; ++c) {
        const bool acc = (fy[c] < fx[c]) || (uacc[c] < std::exp(-(fy[c] - fx[c]) / T));
        if (!acc) continue;
        std::copy(Y.begin() + (size_t)c * P, Y.begin() + (size_t)(c + 1) * P, X.begin() + (size_t)c * P);
        fx[c] = fy[c];
        if (fx[c] < fb[c]) {
          fb[c] = fx[c];
          std::copy(X.begin() + (size_t)c * P, X.begin() + (size_t)(c + 1) * P, xb.begin() + (size_t)c * P);
        }
      }
    }
    int best = 0;
    for (int c = 1; c < C; ++c)
      if (fx[c] < fx[best]) best = c;
    std::copy(X.begin() + (size_t)best * P, X.begin() + (size_t)(best + 1) * P, xs.begin());
    fs = fx[best];
    if (out->trace_f) out->trace_f[l] = fs;
    if (out->trace_y) std::copy(xs.begin(), xs.end(), out->trace_y + (size_t)l * P);
    T *= o->cooling;
  }
  int best = 0;
  for (int c = 1; c < C; ++c)
    if (fb[c] < fb[best]) best = c;
  for (int k = 0; k < P; ++k) out->y_best[k] = xb[(size_t)best * P + k];
  out->f_best = fb[best];
  out->T0_used = T0;
  out->n_evals = (int64_t)C * ((int64_t)L * N) + 1;
  out->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
  cleanup();
  return SABR_LMM_OK;
}
