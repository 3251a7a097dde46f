// Levenberg-Marquardt polish of annealed points (replaces the Nelder-Mead polish of the hybrid
// scheme, Section 3).  Per point and iteration:
//   r      residuals sqrt(w_k)(P_k - P_k^mkt) at theta (FP64, from the model vols);
//   J      columns by forward differences (r(theta + h e_p) - r(theta)) / h, h = 1e-7 max(|theta_p|, 1),
//          over the free slots only (1 + n_free evaluations per point and iteration);
//   g      J^T r, taken from the hand-written adjoint (g = grad f / 2) when the market has one,
//          else from the difference Jacobian;
//   step   (J^T J + mu diag(J^T J)) d = -g by Cholesky over the free slots (a zero diagonal is
//          floored at 1e-12 of the largest), theta' = clamp(theta + d) on the box;
//   accept if f(theta') < f(theta): theta = theta', mu = max(mu / 10, 1e-12); else mu *= 10.
// A point stops when its vol RMSE reaches the target or mu exceeds 1e16.
#pragma once
#include "kernels.cuh"

namespace sabr {

constexpr int kLmStencil = 1 + kMaxParam;   // most points per stencil: theta and theta + h e_p

__device__ __forceinline__ double lm_h(double x) { return 1e-7 * fmax(fabs(x), 1.0); }

// Slot of the a-th free parameter.
__device__ __forceinline__ int lm_free_slot(const unsigned char* freem, int P, int a) {
  for (int k = 0; k < P; ++k)
    if (freem[k] && a-- == 0) return k;
  return -1;
}

// Xp[(i * S + j) * P + k], S = 1 + n_free: j = 0 the point, j = 1 + a the point + h e_(a-th free slot).
__global__ void lm_perturb_kernel(int n, int P, int S, const unsigned char* freem, const double* X, double* Xp) {
  const int i = blockIdx.x, j = threadIdx.x;
  if (i >= n || j >= S) return;
  const int slot = j > 0 ? lm_free_slot(freem, P, j - 1) : -1;
  double* out = Xp + ((size_t)i * S + j) * P;
  for (int k = 0; k < P; ++k) {
    double v = X[(size_t)i * P + k];
    if (k == slot) v += lm_h(v);
    out[k] = v;
  }
}

// Residuals from model vols with the FP64 instrument blocks (Black, out-of-the-money option).
__global__ void residuals_from_vols_kernel(DevMarket m, long long npts, const double* vols, double* res) {
  const int ni = m.n_cap + m.n_swp;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < npts * ni; t += (long long)gridDim.x * blockDim.x) {
    const int k = (int)(t % ni);
    const bool cap = k < m.n_cap;
    const InstrView<double> B = instr_view<double>(cap ? m.cblk64 : m.sblk64, cap ? m.n_cap_pad : m.n_swp_pad);
    const int kk = cap ? k : k - m.n_cap;
    const double sig = vols[t];
    const Q4<double> g0 = B.g0[kk], g1 = B.g1[kk], g2 = B.g2[kk];
    const double p = black_otm<double>(sig, g1.c, g0.a, g1.d, g2.a, g2.b);
    res[t] = g2.d * (p - g2.c);
  }
}

// Normal equations and the damped step, one CTA per point.
__global__ void lm_step_kernel(DevMarket m, int n, int S, const double* res, const double* grad, const double* mu,
                               const int* done, const double* X, double* Xt) {
  const int i = blockIdx.x;
  if (i >= n) return;
  const int P = m.n_param, ni = m.n_cap + m.n_swp;
  __shared__ int fi[kMaxParam];
  __shared__ int nf;
  __shared__ double A[kMaxParam * kMaxParam], g[kMaxParam], hs[kMaxParam];
  if (threadIdx.x == 0) {
    int c = 0;
    for (int k = 0; k < P; ++k)
      if (m.freem[k]) fi[c++] = k;
    nf = c;
  }
  __syncthreads();
  const double* r0 = res + (size_t)i * S * ni;
  const double* x = X + (size_t)i * P;
  if (threadIdx.x < nf) hs[threadIdx.x] = lm_h(x[fi[threadIdx.x]]);
  __syncthreads();
  // J[k][a] = (r(theta + h_a e_fa) - r(theta))[k] / h_a, the stencil's row 1 + a
  for (int t = threadIdx.x; t < nf * nf + nf; t += blockDim.x) {
    if (t < nf * nf) {
      const int a = t / nf, b = t - a * nf;
      if (b < a) continue;
      const double* pa = r0 + (size_t)(1 + a) * ni;
      const double* pb = r0 + (size_t)(1 + b) * ni;
      double s = 0.0;
      for (int k = 0; k < ni; ++k) s += (pa[k] - r0[k]) * (pb[k] - r0[k]);
      s /= hs[a] * hs[b];
      A[a * nf + b] = s;
      A[b * nf + a] = s;
    } else {
      const int a = t - nf * nf;
      if (grad) {
        g[a] = 0.5 * grad[(size_t)i * P + fi[a]];
      } else {
        const double* pa = r0 + (size_t)(1 + a) * ni;
        double s = 0.0;
        for (int k = 0; k < ni; ++k) s += (pa[k] - r0[k]) * r0[k];
        g[a] = s / hs[a];
      }
    }
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  double* xt = Xt + (size_t)i * P;
  for (int k = 0; k < P; ++k) xt[k] = x[k];
  if (done[i]) return;
  const int n_ = nf;
  double L[kMaxParam * kMaxParam], y[kMaxParam];
  double dmax = 0.0;
  for (int a = 0; a < n_; ++a) dmax = fmax(dmax, A[a * n_ + a]);
  for (int a = 0; a < n_; ++a)
    for (int b = 0; b < n_; ++b) L[a * n_ + b] = A[a * n_ + b] + (a == b ? mu[i] * fmax(A[a * n_ + a], 1e-12 * dmax) : 0.0);
  for (int j = 0; j < n_; ++j) {
    double s = L[j * n_ + j];
    for (int k = 0; k < j; ++k) s -= L[j * n_ + k] * L[j * n_ + k];
    if (!(s > 0.0)) return;   // not positive definite: no move (the accept step raises mu)
    const double dj = sqrt(s);
    L[j * n_ + j] = dj;
    for (int r = j + 1; r < n_; ++r) {
      double t = L[r * n_ + j];
      for (int k = 0; k < j; ++k) t -= L[r * n_ + k] * L[j * n_ + k];
      L[r * n_ + j] = t / dj;
    }
  }
  for (int a = 0; a < n_; ++a) {
    double t = -g[a];
    for (int k = 0; k < a; ++k) t -= L[a * n_ + k] * y[k];
    y[a] = t / L[a * n_ + a];
  }
  for (int a = n_ - 1; a >= 0; --a) {
    double t = y[a];
    for (int k = a + 1; k < n_; ++k) t -= L[k * n_ + a] * y[k];
    y[a] = t / L[a * n_ + a];
  }
  for (int a = 0; a < n_; ++a) {
    const int k = fi[a];
    xt[k] = fmin(fmax(x[k] + y[a], m.lo[k]), m.hi[k]);
  }
}

__global__ void lm_accept_kernel(int n, int P, double* X, const double* Xt, double* f, const double* ft, double* mu,
                                 int* done) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n || done[i]) return;
  if (ft[i] < f[i]) {
    for (int k = 0; k < P; ++k) X[(size_t)i * P + k] = Xt[(size_t)i * P + k];
    f[i] = ft[i];
    mu[i] = fmax(mu[i] / 10.0, 1e-12);
  } else {
    mu[i] *= 10.0;
    if (mu[i] > 1e16) done[i] = 1;
  }
}

// RMSE in vol points of each point's model vols; marks points at or below the target as done.
__global__ void lm_rmse_kernel(DevMarket m, int n, const double* vols, double target, double* rmse, int* done,
                               int* any) {
  const int i = blockIdx.x;
  const int ni = m.n_cap + m.n_swp;
  __shared__ double part[32];
  double s = 0.0;
  for (int k = threadIdx.x; k < ni; k += blockDim.x) {
    const double mk = k < m.n_cap ? m.cap_vol[k] : m.swp_vol[k - m.n_cap];
    const double e = vols[(size_t)i * ni + k] - mk;
    s += e * e;
  }
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += part[w];
    const double r = 100.0 * sqrt(t / (double)ni);
    if (rmse) rmse[i] = r;
    if (r <= target) {
      done[i] = 1;
      *any = 1;
    }
  }
}

// Indices of the k lowest f (ties to the lower index) among C chains: k rounds of a block argmin
// with the chosen entries masked.  One CTA of 1024 threads.
__global__ void select_lowest_kernel(const double* fb, int C, int k, int* sel) {
  __shared__ double sf[32];
  __shared__ int sc[32];
  __shared__ int chosen;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int r = 0; r < k; ++r) {
    double bf = __longlong_as_double(0x7ff0000000000000LL);
    int bc = 0x7fffffff;
    for (int c = threadIdx.x; c < C; c += blockDim.x) {
      bool taken = false;
      for (int q = 0; q < r; ++q) taken = taken || (sel[q] == c);
      if (!taken && lex_less(fb[c], c, bf, bc)) { bf = fb[c]; bc = c; }
    }
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
      chosen = sc[0];
      sel[r] = chosen;
    }
    __syncthreads();
  }
}

__global__ void gather_points_kernel(const double* xb, const int* sel, int k, int P, double* X) {
  const int i = blockIdx.x, j = threadIdx.x;
  if (i < k && j < P) X[(size_t)i * P + j] = xb[(size_t)sel[i] * P + j];
}

// The best polished point replaces the annealer's best point if it is better.
__global__ void take_best_kernel(const double* X, const double* f, int k, int P, double* best_x, double* best_f) {
  if (threadIdx.x != 0) return;
  int b = 0;
  for (int i = 1; i < k; ++i) if (f[i] < f[b]) b = i;
  if (f[b] < best_f[0] || !(best_f[0] == best_f[0])) {
    best_f[0] = f[b];
    for (int j = 0; j < P; ++j) best_x[j] = X[(size_t)b * P + j];
  }
}

}  // namespace sabr
