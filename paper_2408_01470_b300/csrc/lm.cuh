// Levenberg-Marquardt polish of annealed points (replaces the Nelder-Mead polish of the hybrid
// scheme, Section 3).  Per point and iteration:
//   r      residuals sqrt(w_k)(P_k - P_k^mkt) at theta (FP64, from the model vols);
//   J      columns by forward differences (r(theta + h e_p) - r(theta)) / h, h = 1e-7 max(|theta_p|, 1),
//          over the free slots only (1 + n_free evaluations per point and iteration);
//   g      half the gradient from the reverse sweep where the market has one (caplet markets; it
//          runs on a side stream beside the stencil), else J^T r from the same J;
//   step   (J^T J + mu diag(J^T J)) d = -g by Cholesky over the free slots (a zero diagonal is
//          floored at 1e-12 of the largest), theta' = clamp(theta + d) on the box;
//   accept if f(theta') < f(theta): theta = theta', mu = max(mu / 10, 1e-12); else mu *= 10.
// A point stops when its vol RMSE reaches the target or mu exceeds 1e16.  f and the RMSE of the
// trial point come from its model vols, so an accepted trial needs no second evaluation.
#pragma once
#include "kernels.cuh"

namespace sabr {

constexpr int kLmStencil = 1 + kMaxGradParam;   // most points per stencil: theta and theta + h e_p

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

// Normal equations and the damped step, one CTA (256 threads) per point.  The residual rows of the
// stencil pass through shared memory in tiles of kLmTile instruments; thread t < n_free (n_free + 1) / 2
// accumulates one entry (a, b >= a) of J^T J, the next n_free threads one entry of J^T r (replaced
// by grad / 2 when grad is given).  Warp 0 factors the damped matrix in shared memory.
constexpr int kLmTile = 64;

__global__ void __launch_bounds__(256) lm_step_kernel(DevMarket m, int n, int S, const double* res, const double* grad,
                                                      const double* mu, const int* done, const double* X, double* Xt) {
  const int i = blockIdx.x;
  if (i >= n) return;
  const int P = m.n_param, ni = m.n_cap + m.n_swp;
  __shared__ int fi[kMaxGradParam];
  __shared__ int nf_s;
  __shared__ double A[kMaxGradParam * kMaxGradParam], g[kMaxGradParam], ih[kMaxGradParam], y[kMaxGradParam], id[kMaxGradParam];
  __shared__ double D[kMaxGradParam + 1][kLmTile];   // row 0: r(theta); row 1 + a: (r(theta + h_a e_fa) - r(theta)) / h_a
  const double* x = X + (size_t)i * P;
  double* xt = Xt + (size_t)i * P;
  if ((int)threadIdx.x < P) xt[threadIdx.x] = x[threadIdx.x];   // no move unless a step is taken
  if (done[i]) return;
  if (threadIdx.x == 0) {
    int c = 0;
    for (int k = 0; k < P; ++k)
      if (m.freem[k]) fi[c++] = k;
    nf_s = c;
  }
  __syncthreads();
  const int nf = nf_s, npair = nf * (nf + 1) / 2;
  if ((int)threadIdx.x < nf) ih[threadIdx.x] = 1.0 / lm_h(x[fi[threadIdx.x]]);
  int ra = -1, rb = -1;   // this thread's entry: A[ra][rb] (rb >= ra), or g[ra] when rb < 0
  if ((int)threadIdx.x < npair) {
    int t = threadIdx.x;
    ra = 0;
    while (t >= nf - ra) { t -= nf - ra; ++ra; }
    rb = ra + t;
  } else if ((int)threadIdx.x < npair + nf) {
    ra = threadIdx.x - npair;
  }
  const double* r0 = res + (size_t)i * S * ni;
  double acc = 0.0;
  for (int k0 = 0; k0 < ni; k0 += kLmTile) {
    const int kn = min(kLmTile, ni - k0);
    __syncthreads();   // the previous tile is consumed (and ih is written)
    for (int e = threadIdx.x; e < (nf + 1) * kLmTile; e += blockDim.x) {
      const int row = e / kLmTile, k = e - row * kLmTile;
      double v = 0.0;
      if (k < kn) {
        const double base = r0[k0 + k];
        v = row == 0 ? base : (r0[(size_t)row * ni + k0 + k] - base) * ih[row - 1];
      }
      D[row][k] = v;
    }
    __syncthreads();
    if (ra >= 0) {
      const double* u = D[1 + ra];
      const double* v = rb >= 0 ? D[1 + rb] : D[0];
      for (int k = 0; k < kn; ++k) acc = fma(u[k], v[k], acc);
    }
  }
  if (ra >= 0) {
    if (rb >= 0) {
      A[ra * nf + rb] = acc;
      A[rb * nf + ra] = acc;
    } else {
      g[ra] = grad ? 0.5 * grad[(size_t)i * P + fi[ra]] : acc;
    }
  }
  __syncthreads();
  if (threadIdx.x >= 32) return;
  const int lane = threadIdx.x;
  double dmax = 0.0;
  for (int a = 0; a < nf; ++a) dmax = fmax(dmax, A[a * nf + a]);
  if (lane < nf) A[lane * nf + lane] += mu[i] * fmax(A[lane * nf + lane], 1e-12 * dmax);
  __syncwarp();
  // right-looking Cholesky: the lower triangle of A becomes L, lane r owns row r; id = 1 / diag L
  for (int j = 0; j < nf; ++j) {
    const double djj = A[j * nf + j];
    if (!(djj > 0.0)) return;   // not positive definite (the same value in every lane): no move
    const double d = sqrt(djj), rd = 1.0 / d;
    __syncwarp();
    if (lane == j) {
      A[j * nf + j] = d;
      id[j] = rd;
    }
    if (lane > j && lane < nf) A[lane * nf + j] *= rd;
    __syncwarp();
    if (lane > j && lane < nf)
      for (int c = j + 1; c <= lane; ++c) A[lane * nf + c] -= A[lane * nf + j] * A[c * nf + j];
    __syncwarp();
  }
  if (lane != 0) return;
  for (int a = 0; a < nf; ++a) {
    double t = -g[a];
    for (int k = 0; k < a; ++k) t -= A[a * nf + k] * y[k];
    y[a] = t * id[a];
  }
  for (int a = nf - 1; a >= 0; --a) {
    double t = y[a];
    for (int k = a + 1; k < nf; ++k) t -= A[k * nf + a] * y[k];
    y[a] = t * id[a];
  }
  for (int a = 0; a < nf; ++a) {
    const int k = fi[a];
    xt[k] = fmin(fmax(x[k] + y[a], m.lo[k]), m.hi[k]);
  }
}

// Accept or reject each point's trial; an accepted trial brings its f and RMSE along and, at or
// below the target, marks the point done.
__global__ void lm_accept_kernel(int n, int P, double* X, const double* Xt, double* f, const double* ft, double* rmse,
                                 const double* rmse_t, double target, double* mu, int* done, int* any) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n || done[i]) return;
  if (ft[i] < f[i]) {
    for (int k = 0; k < P; ++k) X[(size_t)i * P + k] = Xt[(size_t)i * P + k];
    f[i] = ft[i];
    rmse[i] = rmse_t[i];
    mu[i] = fmax(mu[i] / 10.0, 1e-12);
    if (rmse_t[i] <= target) {
      done[i] = 1;
      *any = 1;
    }
  } else {
    mu[i] *= 10.0;
    if (mu[i] > 1e16) done[i] = 1;
  }
}

// f (the sum of squared residuals) and the RMSE in vol points of the model vols in row i * stride
// of vols, one CTA per point; with done, a point at or below the target is marked done and any set.
__global__ void lm_eval_kernel(DevMarket m, int n, int stride, const double* vols, double target, double* f,
                               double* rmse, int* done, int* any) {
  const int i = blockIdx.x;
  if (i >= n) return;
  const int ni = m.n_cap + m.n_swp;
  __shared__ double part[2][32];
  const double* v = vols + (size_t)i * stride * ni;
  double se = 0.0, sf = 0.0;
  for (int k = threadIdx.x; k < ni; k += blockDim.x) {
    const bool cap = k < m.n_cap;
    const int kk = cap ? k : k - m.n_cap;
    const double sig = v[k];
    const double e = sig - (cap ? m.cap_vol[kk] : m.swp_vol[kk]);
    se += e * e;
    const InstrView<double> B = instr_view<double>(cap ? m.cblk64 : m.sblk64, cap ? m.n_cap_pad : m.n_swp_pad);
    const Q4<double> g0 = B.g0[kk], g1 = B.g1[kk], g2 = B.g2[kk];
    const double r = g2.d * (black_otm<double>(sig, g1.c, g0.a, g1.d, g2.a, g2.b) - g2.c);
    sf += r * r;
  }
  se = warp_sum(se);
  sf = warp_sum(sf);
  if ((threadIdx.x & 31) == 0) {
    part[0][threadIdx.x >> 5] = se;
    part[1][threadIdx.x >> 5] = sf;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double te = 0.0, tf = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      te += part[0][w];
      tf += part[1][w];
    }
    const double r = 100.0 * sqrt(te / (double)ni);
    f[i] = tf;
    if (rmse) rmse[i] = r;
    if (done && r <= target) {
      done[i] = 1;
      *any = 1;
    }
  }
}

// Key whose unsigned order is the order of f: -0 as +0, NaN above +inf.
__device__ __forceinline__ unsigned long long order_key(double f) {
  if (f != f) return ~0ull;
  if (f == 0.0) return 0x8000000000000000ull;
  const unsigned long long b = (unsigned long long)__double_as_longlong(f);
  return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}

// Indices of the k lowest f among C chains (1 <= k <= C; of equal f the lower indices), written in
// index order.  One CTA of 1024 threads: a radix select of the k-th smallest key, 8 bits per pass
// from the top, then one ordered compaction of the keys below it and the first equal ones.
__global__ void __launch_bounds__(1024) select_lowest_kernel(const double* fb, int C, int k, int* sel) {
  __shared__ unsigned int hist[256];
  __shared__ unsigned long long s_prefix;
  __shared__ int s_kr;
  __shared__ int wsum[32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  if (k <= 0 || k > C) return;
  unsigned long long prefix = 0, mask = 0;
  int kr = k;   // rank (from 1) of the wanted key among the keys that share the prefix
  for (int shift = 56; shift >= 0; shift -= 8) {
    for (int b = tid; b < 256; b += blockDim.x) hist[b] = 0;
    __syncthreads();
    for (int c = tid; c < C; c += blockDim.x) {
      const unsigned long long key = order_key(fb[c]);
      if ((key & mask) == prefix) atomicAdd(&hist[(key >> shift) & 255], 1u);
    }
    __syncthreads();
    if (warp == 0) {
      unsigned int h[8], cnt = 0;
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        h[q] = hist[lane * 8 + q];
        cnt += h[q];
      }
      unsigned int incl = cnt;
#pragma unroll
      for (int off = 1; off < 32; off <<= 1) {
        const unsigned int o = __shfl_up_sync(0xffffffffu, incl, off);
        if (lane >= off) incl += o;
      }
      unsigned int run = incl - cnt;
      if (run < (unsigned)kr && (unsigned)kr <= incl) {
        int d = lane * 8 + 7;
        for (int q = 0; q < 8; ++q) {
          if ((unsigned)kr <= run + h[q]) { d = lane * 8 + q; break; }
          run += h[q];
        }
        s_prefix = prefix | ((unsigned long long)d << shift);
        s_kr = kr - (int)run;
      }
    }
    __syncthreads();
    prefix = s_prefix;
    kr = s_kr;
    mask |= 255ull << shift;
  }
  // prefix is the k-th smallest key: take every key below it and the first kr keys equal to it
  const unsigned int below = (1u << lane) - 1u;
  int taken = 0, eq_seen = 0;
  for (int base = 0; base < C; base += blockDim.x) {
    const int c = base + tid;
    const unsigned long long key = c < C ? order_key(fb[c]) : ~0ull;
    const bool lt = c < C && key < prefix, eq = c < C && key == prefix;
    const unsigned int be = __ballot_sync(0xffffffffu, eq);
    __syncthreads();
    if (lane == 0) wsum[warp] = __popc(be);
    __syncthreads();
    int eq_before = eq_seen + __popc(be & below), eq_tile = 0;
    for (int w = 0; w < nw; ++w) {
      eq_before += w < warp ? wsum[w] : 0;
      eq_tile += wsum[w];
    }
    const bool take = lt || (eq && eq_before < kr);
    const unsigned int bt = __ballot_sync(0xffffffffu, take);
    __syncthreads();
    if (lane == 0) wsum[warp] = __popc(bt);
    __syncthreads();
    int pos = taken + __popc(bt & below), t_tile = 0;
    for (int w = 0; w < nw; ++w) {
      pos += w < warp ? wsum[w] : 0;
      t_tile += wsum[w];
    }
    if (take) sel[pos] = c;
    taken += t_tile;
    eq_seen += eq_tile;
  }
}

__global__ void gather_points_kernel(const double* xb, const int* sel, int k, int P, double* X) {
  const int i = blockIdx.x, j = threadIdx.x;
  if (i < k && j < P) X[(size_t)i * P + j] = xb[(size_t)sel[i] * P + j];
}

// The best polished point becomes the search's result.  The polish starts from the k lowest chain
// bests, the search's best point among them, and never raises a value, so its best FP64 value is at
// most the FP64 objective of the search's best point; an FP32 search's own best value is an FP32
// evaluation and is not compared with it.  A polish without a finite value keeps the search's.
__global__ void take_best_kernel(const double* X, const double* f, int k, int P, double* best_x, double* best_f) {
  if (threadIdx.x != 0) return;
  int b = 0;
  for (int i = 1; i < k; ++i) if (f[i] < f[b]) b = i;
  if (f[b] == f[b] && f[b] < __longlong_as_double(0x7ff0000000000000LL)) {
    best_f[0] = f[b];
    for (int j = 0; j < P; ++j) best_x[j] = X[(size_t)b * P + j];
  }
}

}  // namespace sabr
