// C-ABI of the Monte Carlo pricer (include/sabr_lmm.h: sabr_lmm_mc_*), included by api.cu.
// Preparation (once per plan, host C++ in FP64): the time grid (every interval between fixings cut
// into ceil(len / dt) equal steps), the instruments sorted by fixing, and the model constants:
// the correlation matrix of (W, Z) from Eqs. (rhoij), (thetaij), (phiij), repaired to the nearest
// correlation matrix in the spectral sense when it is indefinite (negative eigenvalues set to
// zero, rows of S Lambda^(1/2) scaled to unit length; eigenvectors by cyclic Jacobi rotations), and
// its semi-definite Cholesky factor (a pivot at or below 1e-12 ends its column).  Launch: the path
// kernel (every step of every path) and the reduction kernel, stream-ordered.
#pragma once
#include "mc.cuh"

struct sabr_lmm_mc_plan {
  int device = 0;
  int prec = SABR_LMM_FP32;
  int grid = 0;
  int n_cap = 0, n_swp = 0;
  McArgs args{};
  McConsts<double> c64{};
  McConsts<float> c32{};
  void* buf = nullptr;          // device: time grid, instruments, partial sums
  double* out = nullptr;        // device: price [ni], stderr [ni]
  long long* nbad = nullptr;    // device
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

extern "C" sabr_lmm_status sabr_lmm_mc_prepare(const sabr_lmm_mc_desc* d, const sabr_lmm_mc_opts* o, void* stream,
                                               sabr_lmm_mc_plan** out) {
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
  // the correlation matrix in u-order (u = M - 1 - i; row 2u is W_i, row 2u + 1 is Z_i)
  const int n = 2 * M;
  std::vector<double> Cm((size_t)n * n);
  for (int r = 0; r < n; ++r)
    for (int c = 0; c < n; ++c) {
      const int i = M - 1 - r / 2, j = M - 1 - c / 2;
      const bool wr = (r & 1) == 0, wc = (c & 1) == 0;
      const double dT = std::fabs(d->T[i] - d->T[j]);
      double v;
      if (wr && wc) v = d->eta1 + (1.0 - d->eta1) * std::exp(-d->lambda1 * dT);
      else if (!wr && !wc) v = d->eta2 + (1.0 - d->eta2) * std::exp(-d->lambda2 * dT);
      else {   // corr(W_a, Z_b) = sign(phi_aa) sqrt(|phi_aa phi_bb|) e^{-lambda3 |T_a - T_b|}
        const int fa = wr ? i : j, fb = wr ? j : i;
        v = (d->phi[fa] < 0.0 ? -1.0 : 1.0) * std::sqrt(std::fabs(d->phi[fa] * d->phi[fb])) * std::exp(-d->lambda3 * dT);
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
  sabr_lmm_mc_plan* p = new sabr_lmm_mc_plan();
  cudaGetDevice(&p->device);
  p->prec = o->prec;
  p->n_cap = d->n_cap;
  p->n_swp = d->n_swp;
  for (int r = 0; r < n; ++r)
    for (int c = 0; c < n; ++c) p->c64.L[r * kMcRows + c] = L[(size_t)r * n + c];
  for (int u = 0; u < M; ++u) {
    const int i = M - 1 - u;
    for (int v = 0; v < M; ++v) {
      p->c64.rho[u * kMcMaxFwd + v] = Cm[(size_t)(2 * u) * n + 2 * v];
      p->c64.phi[u * kMcMaxFwd + v] = Cm[(size_t)(2 * u) * n + 2 * v + 1];
    }
    p->c64.tau[u] = tau[i];
    p->c64.sig[u] = d->sigma[i];
    p->c64.hs2[u] = 0.5 * d->sigma[i] * d->sigma[i];
    p->c64.F0[u] = (d->P[i] / d->P[i + 1] - 1.0) / tau[i];
    p->c64.lnV0[u] = std::log(d->alpha[i]);
  }
  {
    const double* s = (const double*)&p->c64;
    float* t = (float*)&p->c32;
    for (size_t k = 0; k < sizeof(McConsts<double>) / sizeof(double); ++k) t[k] = (float)s[k];
  }
  // instruments sorted by fixing (stable), with their output slots
  std::vector<int> ci(d->n_cap), si(d->n_swp);
  for (int c = 0; c < d->n_cap; ++c) ci[c] = c;
  for (int c = 0; c < d->n_swp; ++c) si[c] = c;
  std::stable_sort(ci.begin(), ci.end(), [&](int x, int y) { return d->cap_fwd[x] < d->cap_fwd[y]; });
  std::stable_sort(si.begin(), si.end(), [&](int x, int y) { return d->swp_start[x] < d->swp_start[y]; });
  std::vector<int> cap_lo(M + 1, 0), swp_lo(M + 1, 0), cap_out(d->n_cap), swp_out(d->n_swp), swp_b(d->n_swp);
  std::vector<double> cap_K(d->n_cap), swp_K(d->n_swp);
  for (int c = 0; c < d->n_cap; ++c) {
    cap_out[c] = ci[c];
    cap_K[c] = d->cap_K[ci[c]];
    cap_lo[d->cap_fwd[ci[c]] + 1]++;
  }
  for (int c = 0; c < d->n_swp; ++c) {
    swp_out[c] = si[c];
    swp_K[c] = d->swp_K[si[c]];
    swp_b[c] = d->swp_end[si[c]];
    swp_lo[d->swp_start[si[c]] + 1]++;
  }
  for (int k = 0; k < M; ++k) { cap_lo[k + 1] += cap_lo[k]; swp_lo[k + 1] += swp_lo[k]; }
  // grid: enough CTAs for every path, at most 8 per SM (persistent beyond that)
  int nsm = 148;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, p->device);
  const long long need = (o->n_paths + kMcThreads - 1) / kMcThreads;
  p->grid = (int)std::min<long long>(need, o->grid > 0 ? o->grid : (long long)nsm * 8);
  const int ni = d->n_cap + d->n_swp;
  // device buffer: nsteps, h, tau, cap_lo, swp_lo, cap_out, swp_out, swp_b, cap_K, swp_K, part, bad, out, nbad
  Arena A;
  const size_t o_ns = A.take(M * 4), o_h = A.take(M * 8), o_tau = A.take(M * 8), o_clo = A.take((M + 1) * 4),
               o_slo = A.take((M + 1) * 4), o_cout = A.take(d->n_cap * 4), o_sout = A.take(d->n_swp * 4),
               o_sb = A.take(d->n_swp * 4), o_cK = A.take(d->n_cap * 8), o_sK = A.take(d->n_swp * 8),
               o_part = A.take((size_t)p->grid * ni * 16), o_bad = A.take((size_t)p->grid * 8),
               o_out = A.take((size_t)ni * 16), o_nbad = A.take(8);
  std::vector<unsigned char> host(A.size, 0);
  auto put = [&](size_t off, const void* src, size_t bytes) { if (bytes) std::memcpy(host.data() + off, src, bytes); };
  put(o_ns, nsteps.data(), M * 4); put(o_h, h.data(), M * 8); put(o_tau, tau.data(), M * 8);
  put(o_clo, cap_lo.data(), (M + 1) * 4); put(o_slo, swp_lo.data(), (M + 1) * 4);
  put(o_cout, cap_out.data(), d->n_cap * 4); put(o_sout, swp_out.data(), d->n_swp * 4);
  put(o_sb, swp_b.data(), d->n_swp * 4); put(o_cK, cap_K.data(), d->n_cap * 8); put(o_sK, swp_K.data(), d->n_swp * 8);
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
  a.nsteps = (const int*)(b + o_ns); a.h = (const double*)(b + o_h); a.tau64 = (const double*)(b + o_tau);
  a.cap_lo = (const int*)(b + o_clo); a.swp_lo = (const int*)(b + o_slo);
  a.cap_out = (const int*)(b + o_cout); a.swp_out = (const int*)(b + o_sout); a.swp_b = (const int*)(b + o_sb);
  a.cap_K = (const double*)(b + o_cK); a.swp_K = (const double*)(b + o_sK);
  a.seed = o->seed; a.n_paths = o->n_paths;
  a.part = (double*)(b + o_part); a.bad = (unsigned long long*)(b + o_bad);
  p->out = (double*)(b + o_out);
  p->nbad = (long long*)(b + o_nbad);
  const size_t sm = mc_smem_bytes(ni);
  e = o->prec == SABR_LMM_FP64 ? raise_smem_limit(mc_path_kernel<double>, (uint32_t)sm)
                               : raise_smem_limit(mc_path_kernel<float>, (uint32_t)sm);
  if (e != cudaSuccess) {
    cudaFree(p->buf);
    delete p;
    return fail(SABR_LMM_ECUDA, std::string("mc: ") + cudaGetErrorString(e));
  }
  *out = p;
  return SABR_LMM_OK;
}

extern "C" sabr_lmm_status sabr_lmm_mc_launch(sabr_lmm_mc_plan* p, double* price, double* stderr_out,
                                              long long* n_bad, void* stream) {
  if (!p) return fail(SABR_LMM_EINVAL, "plan is required");
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev != p->device) return fail(SABR_LMM_EINVAL, "mc: the plan belongs to another device");
  cudaStream_t s = (cudaStream_t)stream;
  const int ni = p->n_cap + p->n_swp;
  const size_t sm = mc_smem_bytes(ni);
  if (p->prec == SABR_LMM_FP64) mc_path_kernel<double><<<p->grid, kMcThreads, sm, s>>>(p->args, p->c64);
  else mc_path_kernel<float><<<p->grid, kMcThreads, sm, s>>>(p->args, p->c32);
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
