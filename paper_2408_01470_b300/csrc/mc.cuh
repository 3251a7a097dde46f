// Monte Carlo pricer of the Hagan SABR/LIBOR model (Section 2.1, Eqs. dinamicasHagan1-2) and of
// the Mercurio & Morini one (Section 2.2, one volatility process; the MM branch below) under the
// spot measure: the Monte Carlo pricing of caplets and swaptions of Section 3 (Table
// tab:haganMCpricer).  One thread per path; the paths of a warp run in lockstep (every path has
// the same time grid), so the per-instrument sums are warp reductions at the fixing dates, and the
// warps of a CTA meet at every fixing date.
//
// Per step of the interval [T_{k-1}, T_k] (h(t) = k, forwards k .. M-1 alive):
//   xi    : 2a standard normals (a = M - k alive forwards), Philox4x32-10 at counter
//           (b, step, path low word, path high word), key (seed low, seed high), uniforms
//           (x + 1/2) 2^-32 (FP64) or (x >> 8 + 1/2) 2^-24 (FP32), Box-Muller on pairs;
//   Z     : L xi with L the Cholesky factor of the (W, Z) correlation matrix ordered last forward
//           first (u = M - 1 - i: row 2u is W_i, row 2u + 1 is Z_i), so the alive forwards are the
//           leading 2a rows and need only the first 2a normals;
//   x_i   = tau_i V_i F_i^b / (1 + tau_i F_i),
//   F_i  <- max(F_i + V_i F_i^b (h sum_{j=k}^{i} rho_ij x_j + sqrt(h) Z_{W_i}), 0)   (Euler, absorbed at 0),
//   ln V_i <- ln V_i + h (sigma_i sum_{j=k}^{i} phi_ij x_j - sigma_i^2 / 2) + sigma_i sqrt(h) Z_{Z_i};
// at T_k forward k fixes: its caplets pay tau_k (F_k - K)^+ at T_{k+1}, deflated by
// 1 / B(T_{k+1}) = P(0, T_0) / prod_{j <= k} (1 + tau_j F_j(T_j)); the swaptions expiring at T_k
// pay A (S - K)^+ deflated by 1 / B(T_k), with the annuity and swap rate from the forwards at T_k.
// A path whose F or ln V is not finite at a fixing date pays nothing from there on (counted).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace sabr {

constexpr int kMcMaxFwd = 16;            // forwards a pricer simulates
constexpr int kMcRows = 2 * kMcMaxFwd;   // rows of the correlation factor
// Paths per CTA (one thread each): at most 512 in FP32 (one CTA of 16 warps per SM at 128
// registers, so that every warp of an SM runs the same interval's code), 128 in FP64; fewer when
// the per-warp sums of many instruments would not fit in shared memory.
template <class R> __host__ __device__ constexpr int mc_max_threads() { return sizeof(R) == 4 ? 512 : 128; }
constexpr int kMcMaxWarps = 16;
constexpr size_t kMcSmemMax = 227 * 1024;   // dynamic shared memory a CTA may take

// Model constants, in u-order (u = M - 1 - i), one copy per precision.
// (16-byte aligned rows, so that reads of consecutive coefficients from shared memory combine into
// 16-byte loads)
template <class R> struct McConsts {
  alignas(16) R L[kMcRows * kMcRows];          // Cholesky factor, row-major
  alignas(16) R rho[kMcMaxFwd * kMcMaxFwd];    // rho(u, v): correlation of W_(M-1-u) with W_(M-1-v)
  alignas(16) R phi[kMcMaxFwd * kMcMaxFwd];    // phi(u, v): correlation of W_(M-1-u) with Z_(M-1-v)
  alignas(16) R tau[kMcMaxFwd];
  alignas(16) R sig[kMcMaxFwd];
  alignas(16) R hs2[kMcMaxFwd];
  alignas(16) R F0[kMcMaxFwd];
  alignas(16) R lnV0[kMcMaxFwd];
  alignas(16) R alpha[kMcMaxFwd];              // Mercurio & Morini: alpha_i (the Hagan model's alpha is V_i(0))
};

struct McArgs {
  int M;                         // forwards simulated (the largest forward any instrument needs + 1)
  int model;                     // 0: Hagan; 2: Mercurio & Morini (one vol process, row 0 of L is Z)
  int n_int;                     // intervals simulated: the last fixing any instrument needs + 1
  int n_cap, n_swp;
  double beta, P0;               // P0 = P(0, T_0)
  const int* nsteps;             // [M] steps of interval k
  const double* h;               // [M] step length of interval k
  // caplets sorted by forward, swaptions by expiry; per interval k the ranges [lo[k], lo[k+1])
  const int* cap_lo;             // [M + 1]
  const int* swp_lo;             // [M + 1]
  const int* cap_out;            // [n_cap] output slot of sorted caplet c
  const int* swp_out;            // [n_swp]
  const double* cap_K;           // [n_cap] sorted
  const double* swp_K;           // [n_swp] sorted
  const int* swp_b;              // [n_swp] one past the swap's last forward (sorted)
  const double* tau64;           // [M] accruals (for the FP64 payoffs)
  const float* cap_K32;          // [n_cap] cap_K in FP32 (the FP32 payoffs)
  const float* swp_K32;          // [n_swp]
  const float* tau32;            // [M]
  unsigned long long seed;
  long long n_paths;
  double* part;                  // [grid x (n_cap + n_swp) x 2] per-CTA sums of payoff, payoff^2
  unsigned long long* bad;       // [grid] stopped paths per CTA
};

__device__ __forceinline__ void philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0,
                                              uint32_t k1, uint32_t o[4]) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u, W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    // one 32 x 32 -> 64 multiply-wide each (hi and lo words of the product from one instruction)
    const uint64_t p0 = (uint64_t)M0 * c0, p1 = (uint64_t)M1 * c2;
    const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0, hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
    k0 += W0; k1 += W1;
  }
  o[0] = c0; o[1] = c1; o[2] = c2; o[3] = c3;
}

// Box-Muller on two 32-bit words.
__device__ __forceinline__ void box_muller(uint32_t a, uint32_t b, double& z0, double& z1) {
  const double u0 = ((double)a + 0.5) * 0x1.0p-32, u1 = ((double)b + 0.5) * 0x1.0p-32;
  const double r = sqrt(-2.0 * log(u0));
  double s, c;
  sincospi(2.0 * u1, &s, &c);
  z0 = r * c;
  z1 = r * s;
}
// FP32: ln u0 from the MUFU log2 below u0 = 3/4 (relative error ~1e-7 there) and above it, where
// ln u0 is small and the MUFU form's absolute error would dominate, from the atanh series
// ln u = 2 (s + s^3/3 + s^5/5 + s^7/7 + s^9/9), s = (u - 1) / (u + 1), |s| < 1/7 (truncation
// below 1e-9 of ln u); (cos, sin)(2 pi u1) = -(cos, sin)(2 pi (u1 - 1/2)) on the MUFU with the
// argument in (-pi, pi).
__device__ __forceinline__ void box_muller(uint32_t a, uint32_t b, float& z0, float& z1) {
  const float u0 = ((float)(a >> 8) + 0.5f) * 0x1.0p-24f, u1 = ((float)(b >> 8) + 0.5f) * 0x1.0p-24f;
  const float sa = __fdividef(u0 - 1.0f, u0 + 1.0f), s2 = sa * sa;
  const float ser = 2.0f * sa * fmaf(s2, fmaf(s2, fmaf(s2, fmaf(s2, 1.0f / 9.0f, 1.0f / 7.0f), 0.2f), 1.0f / 3.0f), 1.0f);
  const float lu = u0 > 0.75f ? ser : __logf(u0);
  float r;   // the MUFU square root (the argument is > 0: u0 < 1)
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(-2.0f * lu));
  float s, c;
  __sincosf(6.28318530717958647692f * (u1 - 0.5f), &s, &c);
  z0 = -r * c;
  z1 = -r * s;
}

template <class R> __device__ __forceinline__ R mc_exp(R x);
template <> __device__ __forceinline__ double mc_exp<double>(double x) { return exp(x); }
template <> __device__ __forceinline__ float mc_exp<float>(float x) { return __expf(x); }
template <class R> __device__ __forceinline__ R mc_log(R x);
template <> __device__ __forceinline__ double mc_log<double>(double x) { return log(x); }
template <> __device__ __forceinline__ float mc_log<float>(float x) { return __logf(x); }
template <class R> __device__ __forceinline__ R mc_rcp(R x);
template <> __device__ __forceinline__ double mc_rcp<double>(double x) { return 1.0 / x; }
template <> __device__ __forceinline__ float mc_rcp<float>(float x) {   // the MUFU reciprocal (x >= 1 here)
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// Payoff inputs in the path precision: FP32 copies of the strikes and accruals for the FP32 paths.
template <class R> __device__ __forceinline__ R mc_tau(const McArgs& a, int j) {
  if constexpr (sizeof(R) == 4) return a.tau32[j];
  else return a.tau64[j];
}
template <class R> __device__ __forceinline__ R mc_cap_K(const McArgs& a, int c) {
  if constexpr (sizeof(R) == 4) return a.cap_K32[c];
  else return a.cap_K[c];
}
template <class R> __device__ __forceinline__ R mc_swp_K(const McArgs& a, int c) {
  if constexpr (sizeof(R) == 4) return a.swp_K32[c];
  else return a.swp_K[c];
}
// Sum over the warp (butterfly), in the path precision: the 32 payoffs of a warp in FP32 for FP32
// paths (relative rounding ~1e-7 of the sum), every warp's sum then accumulated in FP64.
template <class R> __device__ __forceinline__ R warp_sum_r(R v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  return v;
}

__device__ __forceinline__ double warp_sum_mc(double v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  return v;
}

// Dynamic shared memory of the path kernel: the per-warp sums.
__host__ __device__ inline size_t mc_smem_bytes(int n_instr, int threads) {
  return (size_t)(threads / 32) * n_instr * 2 * sizeof(double);
}

// The steps of one interval with NA alive forwards (u = 0 .. NA - 1), NA a compile-time constant:
// every guard on the alive count folds away, and only the normals, rows and drift terms the
// interval needs are generated.  The arithmetic and its order are those of every NA.
template <class R, bool MM, bool SMEM, int NA>
__device__ __forceinline__ void mc_interval(const McConsts<R>& C, R (&F)[kMcMaxFwd], R (&lnV)[kMcMaxFwd], const int ns,
                                            const R h, const R sh, int& step, const long long p, const uint32_t k0,
                                            const uint32_t k1, const R beta) {
  constexpr int na = NA;
  for (int s = 0; s < ns; ++s, ++step) {
    // SMEM (constants in shared memory): read where they are used, every step; held in registers
    // across the steps they would take more than a thread has
    if constexpr (SMEM) asm volatile("" ::: "memory");
    R xi[kMcRows];
#pragma unroll
    for (int b = 0; b < kMcRows / 4; ++b) {
      if (4 * b < (MM ? na + 1 : 2 * na)) {
        uint32_t o[4];
        philox4x32_10((uint32_t)b, (uint32_t)step, (uint32_t)p, (uint32_t)((unsigned long long)p >> 32), k0, k1, o);
        box_muller(o[0], o[1], xi[4 * b], xi[4 * b + 1]);
        box_muller(o[2], o[3], xi[4 * b + 2], xi[4 * b + 3]);
      } else {
        xi[4 * b] = xi[4 * b + 1] = xi[4 * b + 2] = xi[4 * b + 3] = R(0);
      }
    }
    if constexpr (MM) {
      const R Vc = mc_exp<R>(lnV[0]);
      R x[kMcMaxFwd], vf[kMcMaxFwd];
#pragma unroll
      for (int u = 0; u < kMcMaxFwd; ++u) {
        if (u < na) {
          const R fb = F[u] > R(0) ? mc_exp<R>(beta * mc_log<R>(F[u])) : R(0);
          vf[u] = C.alpha[u] * Vc * fb;
          x[u] = C.tau[u] * C.alpha[u] * fb * mc_rcp<R>(R(1) + C.tau[u] * F[u]);
        } else {
          vf[u] = x[u] = R(0);
        }
      }
      const R zz = C.L[0] * xi[0];
#pragma unroll
      for (int u = 0; u < kMcMaxFwd; ++u) {
        if (u < na) {
          R dF0 = 0, dF1 = 0;
#pragma unroll
          for (int v = u; v < kMcMaxFwd; ++v)
            if (v < na) {
              if ((v - u) & 1) dF1 += C.rho[u * kMcMaxFwd + v] * x[v];
              else dF0 += C.rho[u * kMcMaxFwd + v] * x[v];
            }
          R zw0 = 0, zw1 = 0;
#pragma unroll
          for (int c = 0; c <= u + 1; ++c) {
            if (c & 1) zw1 += C.L[(u + 1) * kMcRows + c] * xi[c];
            else zw0 += C.L[(u + 1) * kMcRows + c] * xi[c];
          }
          const R fn = F[u] + vf[u] * (h * Vc * (dF0 + dF1) + sh * (zw0 + zw1));
          F[u] = fn > R(0) ? fn : R(0);
        }
      }
      lnV[0] += h * (-C.hs2[0]) + C.sig[0] * sh * zz;
    } else {
    R x[kMcMaxFwd], vf[kMcMaxFwd], V[kMcMaxFwd];
#pragma unroll
    for (int u = 0; u < kMcMaxFwd; ++u) {
      if (u < na) {
        V[u] = mc_exp<R>(lnV[u]);
        const R fb = F[u] > R(0) ? mc_exp<R>(beta * mc_log<R>(F[u])) : R(0);
        vf[u] = V[u] * fb;
        x[u] = C.tau[u] * vf[u] * mc_rcp<R>(R(1) + C.tau[u] * F[u]);
      } else {
        V[u] = vf[u] = x[u] = R(0);
      }
    }
#pragma unroll
    for (int u = 0; u < kMcMaxFwd; ++u) {
      if (u < na) {
        // drifts: forwards j = k .. i, i.e. v = u .. na - 1
        // (two partial sums per dot product: half the length of each dependent FMA chain)
        R dF0 = 0, dV0 = 0, dF1 = 0, dV1 = 0;
#pragma unroll
        for (int v = u; v < kMcMaxFwd; ++v)
          if (v < na) {
            if ((v - u) & 1) {
              dF1 += C.rho[u * kMcMaxFwd + v] * x[v];
              dV1 += C.phi[u * kMcMaxFwd + v] * x[v];
            } else {
              dF0 += C.rho[u * kMcMaxFwd + v] * x[v];
              dV0 += C.phi[u * kMcMaxFwd + v] * x[v];
            }
          }
        const R dF = dF0 + dF1, dV = dV0 + dV1;
        R zw0 = 0, zw1 = 0, zz0 = 0, zz1 = 0;
#pragma unroll
        for (int c = 0; c <= 2 * u; ++c) {
          if (c & 1) zw1 += C.L[(2 * u) * kMcRows + c] * xi[c];
          else zw0 += C.L[(2 * u) * kMcRows + c] * xi[c];
        }
#pragma unroll
        for (int c = 0; c <= 2 * u + 1; ++c) {
          if (c & 1) zz1 += C.L[(2 * u + 1) * kMcRows + c] * xi[c];
          else zz0 += C.L[(2 * u + 1) * kMcRows + c] * xi[c];
        }
        const R zw = zw0 + zw1, zz = zz0 + zz1;
        const R fn = F[u] + vf[u] * (h * dF + sh * zw);
        F[u] = fn > R(0) ? fn : R(0);
        lnV[u] += h * (C.sig[u] * dV - C.hs2[u]) + C.sig[u] * sh * zz;
      }
    }
    }
  }
}

// The paths of CTA blockIdx.x (grid-stride over gridDim.x CTAs): their per-warp sums in acc
// (shared, [warps][n_instr][2]), the CTA's sums to part_out [n_instr x 2] and its stopped paths to
// bad_out.  C is read with compile-time indices after unrolling.
// MM: the Mercurio & Morini dynamics (Section 2.2): dF_i = mu_i dt + alpha_i V F_i^b dW_i with
// mu_i = alpha_i V F_i^b V sum_{j=k}^{i} rho_ij tau_j alpha_j F_j^b / (1 + tau_j F_j), dV = sigma V dZ,
// V(0) = 1; the factor's row 0 is Z and row 1 + u is W of forward M - 1 - u, so a step draws 1 + a
// normals; ln V is lnV[0].
template <class R, bool MM, bool SMEM>
__device__ __forceinline__ void mc_paths(const McArgs& a, const McConsts<R>& C, double* acc, double* part_out,
                                         unsigned long long* bad_out) {
  const int n_instr = a.n_cap + a.n_swp, n_warps = blockDim.x >> 5;
  for (int t = threadIdx.x; t < n_warps * n_instr * 2; t += blockDim.x) acc[t] = 0.0;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double* wacc = acc + (size_t)warp * n_instr * 2;
  const int M = a.M;
  const R beta = (R)a.beta;
  const uint32_t k0 = (uint32_t)a.seed, k1 = (uint32_t)(a.seed >> 32);
  unsigned long long nbad = 0;
  // The CTA's batches of blockDim.x paths: every warp takes the same number of batches and meets the
  // barrier at the end of every interval (a warp past the last path only meets the barriers), so
  // the warps of the CTA run the same interval's code at the same time.
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long cbase = (long long)blockIdx.x * blockDim.x; cbase < a.n_paths; cbase += stride) {
    const long long base = cbase + warp * 32;
    const bool warp_live = base < a.n_paths;
    const long long p = base + lane;
    const bool live = p < a.n_paths;
    R F[kMcMaxFwd], lnV[kMcMaxFwd];
#pragma unroll
    for (int u = 0; u < kMcMaxFwd; ++u) { F[u] = C.F0[u]; lnV[u] = C.lnV0[u]; }
    bool good = live;
    R numer = (R)a.P0;     // 1 / B(T_k) at the start of interval k
    int step = 0;
    for (int k = 0; k < a.n_int; ++k) {
      if (warp_live) {
        const int na = M - k;   // alive forwards: u = 0 .. na - 1
        const int ns = a.nsteps[k];
        const R h = (R)a.h[k], sh = (R)sqrt(a.h[k]);
        switch (na) {
#define SABR_MC_CASE(n) \
    case n: mc_interval<R, MM, SMEM, n>(C, F, lnV, ns, h, sh, step, p, k0, k1, beta); break;
          SABR_MC_CASE(1) SABR_MC_CASE(2) SABR_MC_CASE(3) SABR_MC_CASE(4) SABR_MC_CASE(5) SABR_MC_CASE(6)
          SABR_MC_CASE(7) SABR_MC_CASE(8) SABR_MC_CASE(9) SABR_MC_CASE(10) SABR_MC_CASE(11) SABR_MC_CASE(12)
          SABR_MC_CASE(13) SABR_MC_CASE(14) SABR_MC_CASE(15) SABR_MC_CASE(16)
#undef SABR_MC_CASE
          default: break;
        }
        // T_k: forward k (u = na - 1) fixes
        bool fin = true;
        R Fs[kMcMaxFwd];
#pragma unroll
        for (int u = 0; u < kMcMaxFwd; ++u) {
          Fs[u] = F[u];
          if (u < na) fin = fin && isfinite(F[u]) && isfinite(lnV[MM ? 0 : u]);
        }
        if (good && !fin) ++nbad;
        good = good && fin;
        const R fix = Fs[na - 1];
        // swaptions expiring at T_k (sorted by swap end), deflated by 1 / B(T_k): one running product
        // disc_j = prod_{l=k..j} 1 / (1 + tau_l F_l) serves them all, with the annuity A = sum tau_j
        // disc_j; the swap rate is (1 - disc) / A, in FP32 (sum tau_j F_j disc_j) / A, the same
        // number as a sum of positive terms (1 - disc_j telescopes into it), free of cancellation
        {
          R disc = 1, A = 0, fl = 0;
          int j = k;
          for (int c = a.swp_lo[k]; c < a.swp_lo[k + 1]; ++c) {
            R pay = 0;
            if (good) {
              for (const int b = a.swp_b[c]; j < b; ++j) {
                const R tj = mc_tau<R>(a, j), Fj = Fs[M - 1 - j];
                disc = disc / (R(1) + tj * Fj);
                A += tj * disc;
                if constexpr (sizeof(R) == 4) fl += tj * Fj * disc;
              }
              R S;
              if constexpr (sizeof(R) == 4) S = fl / A;
              else S = (R(1) - disc) / A;
              const R dS = S - mc_swp_K<R>(a, c);
              pay = dS > R(0) ? A * dS * numer : R(0);
            }
            const R s1 = warp_sum_r(pay), s2 = warp_sum_r(pay * pay);
            if (lane == 0) { wacc[2 * (a.n_cap + c)] += (double)s1; wacc[2 * (a.n_cap + c) + 1] += (double)s2; }
          }
        }
        const R tk = mc_tau<R>(a, k);
        numer = good ? numer / (R(1) + tk * fix) : R(0);
        // caplets on forward k, paid at T_{k+1}
        for (int c = a.cap_lo[k]; c < a.cap_lo[k + 1]; ++c) {
          const R dK = fix - mc_cap_K<R>(a, c);
          const R pay = good && dK > R(0) ? tk * dK * numer : R(0);
          const R s1 = warp_sum_r(pay), s2 = warp_sum_r(pay * pay);
          if (lane == 0) { wacc[2 * c] += (double)s1; wacc[2 * c + 1] += (double)s2; }
        }
      }
      __syncthreads();
    }
  }
  __syncthreads();
  // the CTA's sums, warp by warp in order
  double* out = part_out;
  for (int t = threadIdx.x; t < n_instr * 2; t += blockDim.x) {
    double v = 0.0;
    for (int w = 0; w < n_warps; ++w) v += acc[(size_t)w * n_instr * 2 + t];
    out[t] = v;
  }
  __shared__ unsigned long long sbad[kMcMaxWarps];
  nbad = (unsigned long long)__reduce_add_sync(0xffffffffu, (unsigned)nbad);
  if (lane == 0) sbad[warp] = nbad;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long t = 0;
    for (int w = 0; w < n_warps; ++w) t += sbad[w];
    *bad_out = t;
  }
}

// The model constants travel as a kernel parameter (constant bank): after unrolling, every index
// into them is a compile-time constant, so the FMAs of the correlation product and the drifts read
// their coefficient straight from the constant bank, with no shared-memory load.
template <class R, bool MM>
__global__ void __launch_bounds__(mc_max_threads<R>(), 1) mc_path_kernel(const __grid_constant__ McArgs a,
                                                                    const __grid_constant__ McConsts<R> C) {
  extern __shared__ __align__(128) unsigned char smem[];
  const int n_instr = a.n_cap + a.n_swp;
  mc_paths<R, MM, false>(a, C, (double*)smem, a.part + (size_t)blockIdx.x * n_instr * 2, a.bad + blockIdx.x);
}

// Many parameter sets in one launch (the annealer's proposals): set blockIdx.y has its constants
// Cs[set], staged into shared memory ahead of the per-warp sums, and its own CTA sums,
// part[(set x gridDim.x + CTA) x n_instr x 2], bad[set x gridDim.x + CTA].
template <class R>
__host__ __device__ inline size_t mc_batch_smem_bytes(int n_instr, int threads) {
  return ((sizeof(McConsts<R>) + 127) & ~(size_t)127) + mc_smem_bytes(n_instr, threads);
}

template <class R, bool MM>
__global__ void __launch_bounds__(mc_max_threads<R>(), 1) mc_path_batch_kernel(const __grid_constant__ McArgs a,
                                                                          const McConsts<R>* __restrict__ Cs) {
  extern __shared__ __align__(128) unsigned char smem[];
  McConsts<R>& C = *(McConsts<R>*)smem;
  const int set = blockIdx.y, n_instr = a.n_cap + a.n_swp;
  {
    const uint4* src = (const uint4*)(Cs + set);
    uint4* dst = (uint4*)smem;
    for (int t = threadIdx.x; t < (int)(sizeof(McConsts<R>) / 16); t += blockDim.x) dst[t] = src[t];
  }
  // (mc_paths synchronises the CTA before it reads C)
  double* acc = (double*)(smem + ((sizeof(McConsts<R>) + 127) & ~(size_t)127));
  const size_t cta = (size_t)set * gridDim.x + blockIdx.x;
  mc_paths<R, MM, true>(a, C, acc, a.part + cta * n_instr * 2, a.bad + cta);
}

// f_s of every set: the Monte Carlo prices from its CTA sums (CTA by CTA in order) against the
// market prices mkt [n_instr] (sorted order), f[set] = sum_k (price_k - mkt_k)^2 (+inf if any
// price is not finite); one warp per set.
__global__ void mc_objective_kernel(McArgs a, int grid, int n_sets, const double* mkt, double* f) {
  const int set = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (set >= n_sets) return;
  const int n_instr = a.n_cap + a.n_swp;
  double acc = 0.0;
  for (int t = lane; t < n_instr; t += 32) {
    double s1 = 0.0;
    for (int g = 0; g < grid; ++g) s1 += a.part[(((size_t)set * grid + g) * n_instr + t) * 2];
    const double e = s1 / (double)a.n_paths - mkt[t];
    acc += e * e;
  }
  acc = warp_sum_mc(acc);
  if (lane == 0) f[set] = isfinite(acc) ? acc : __longlong_as_double(0x7ff0000000000000LL);
}

// Market prices of the sorted instruments from their quoted Black vols: caplet on forward i,
// discount tau_i P(0, T_{i+1}), forward F_i(0), expiry T_i; payer swaption over [a, b), annuity
// A = sum tau_k P(0, T_{k+1}), swap rate (P(0, T_a) - P(0, T_b)) / A, expiry T_a.  One thread each.
__device__ __forceinline__ double mc_black_call(double F, double K, double T, double v, double D) {
  const double s = v * sqrt(T);
  const double d1 = log(F / K) / s + 0.5 * s;
  return D * (F * normcdf(d1) - K * normcdf(d1 - s));
}
__global__ void mc_market_kernel(McArgs a, const double* T, const double* P, const int* cap_fwd_sorted,
                                 const int* swp_a_sorted, const double* vol_sorted, double* mkt) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < a.n_cap) {
    const int i = cap_fwd_sorted[t];
    const double tau = T[i + 1] - T[i];
    const double F = (P[i] / P[i + 1] - 1.0) / tau;
    mkt[t] = mc_black_call(F, a.cap_K[t], T[i], vol_sorted[t], tau * P[i + 1]);
  } else if (t < a.n_cap + a.n_swp) {
    const int c = t - a.n_cap, s0 = swp_a_sorted[c], b = a.swp_b[c];
    double A = 0.0;
    for (int k = s0; k < b; ++k) A += (T[k + 1] - T[k]) * P[k + 1];
    mkt[t] = mc_black_call((P[s0] - P[b]) / A, a.swp_K[c], T[s0], vol_sorted[t], A);
  }
}

// Prices and standard errors from the per-CTA sums, CTA by CTA in order; out slot by the
// instruments' original order.  One thread per instrument.
__global__ void mc_reduce_kernel(McArgs a, int grid, double* price, double* stderr_out, long long* n_bad) {
  const int n_instr = a.n_cap + a.n_swp;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n_instr) {
    double s1 = 0.0, s2 = 0.0;
    for (int g = 0; g < grid; ++g) {
      s1 += a.part[((size_t)g * n_instr + t) * 2];
      s2 += a.part[((size_t)g * n_instr + t) * 2 + 1];
    }
    const double n = (double)a.n_paths;
    const double m = s1 / n;
    const double var = fmax(s2 / n - m * m, 0.0);
    const int o = t < a.n_cap ? a.cap_out[t] : a.n_cap + a.swp_out[t - a.n_cap];
    price[o] = m;
    if (stderr_out) stderr_out[o] = n > 1.0 ? sqrt(var / (n - 1.0)) : 0.0;
  }
  if (t == 0 && n_bad) {
    long long b = 0;
    for (int g = 0; g < grid; ++g) b += (long long)a.bad[g];
    *n_bad = b;
  }
}

}  // namespace sabr
