// Device arithmetic of the hot path, templated on the pricing precision R (double or float).
//
//   philox4x64_10 ... counter-based uniforms (Salmon et al., SC'11): ten rounds of two
//                     64x64->128 products with the Weyl key schedule.
//   z_over_x ........ z / x(z) of Hagan et al. (2002), x(z) = log((sqrt(1-2rz+z^2)+z-r)/(1-r)),
//                     in a cancellation-free form (see below) with its Taylor series near z = 0.
//   sabr_* .......... the Hagan (2002) lognormal expansion and Eq. (sigmaHagan) of the paper.
//   black_otm ....... Black's formula for the out-of-the-money option on a forward or swap rate.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace sabr {

// ------------------------------------------------------------------ precision traits
template <class R> struct Num;
template <> struct Num<double> {
  static __device__ __forceinline__ double exp_(double x) { return exp(x); }
  static __device__ __forceinline__ double log1p_(double x) { return log1p(x); }
  static __device__ __forceinline__ double sqrt_(double x) { return sqrt(x); }
  static __device__ __forceinline__ double erfc_(double x) { return erfc(x); }
  static __device__ __forceinline__ double abs_(double x) { return fabs(x); }
  static __device__ __forceinline__ bool finite_(double x) { return isfinite(x); }
  static constexpr double zx_series = 1e-6;  // |z| below which z/x(z) uses its series
};
template <> struct Num<float> {
  static __device__ __forceinline__ float exp_(float x) { return expf(x); }
  static __device__ __forceinline__ float log1p_(float x) { return log1pf(x); }
  static __device__ __forceinline__ float sqrt_(float x) { return sqrtf(x); }
  static __device__ __forceinline__ float erfc_(float x) { return erfcf(x); }
  static __device__ __forceinline__ float abs_(float x) { return fabsf(x); }
  static __device__ __forceinline__ bool finite_(float x) { return isfinite(x); }
  static constexpr float zx_series = 1e-3f;  // series error O(z^3) < 2^-24 there
};

// ------------------------------------------------------------------ FP32 approximations
// The FP32 path uses the hardware approximations of PTX (rcp, rsqrt, ex2 .approx.ftz: about 1-2
// ulp, denormal inputs and results flushed to zero) where its error budget allows.
__device__ __forceinline__ float rcp_approx(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float rsqrt_approx(float x) {
  float r;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float ex2_approx(float x) {
  float r;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
// log2 x on the MUFU (PTX lg2.approx; flushes subnormals).
__device__ __forceinline__ float lg2_approx(float x) {
  float r;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
// e^x = 2^(x log2 e); the rounding of x log2 e adds |x| 2^-24 to the relative error.
__device__ __forceinline__ float exp_approx(float x) { return ex2_approx(x * 1.44269504088896341f); }

// log1p of a non-negative argument (the argument of x(z)).  y < 1/2: the atanh series
// 2 s (1 + s^2/3 + ... + s^8/9) in s = y / (2 + y) (|s| <= 1/5, truncation below 1e-8 relative);
// y >= 1/2: log2(1 + y) ln 2 on the MUFU (PTX lg2.approx), where 1 + y carries no cancellation
// (a few 1e-7 relative).  An infinite or NaN argument takes the second form and stays so.
__device__ __forceinline__ float log1p_pos(float y) {
  if (y < 0.5f) {
    // the series' factor 2 rides on the coefficients (a power-of-two scaling: same roundings)
    const float s = y * rcp_approx(2.0f + y);
    const float s2 = s * s;
    float p = fmaf(s2, 2.0f / 9.0f, 2.0f / 7.0f);
    p = fmaf(s2, p, 2.0f / 5.0f);
    p = fmaf(s2, p, 2.0f / 3.0f);
    p = fmaf(s2, p, 2.0f);
    return s * p;
  }
  return lg2_approx(1.0f + y) * 0.693147180559945309f;
}

// ------------------------------------------------------------------ Philox4x64-10
struct U4 { uint64_t v[4]; };

__device__ __forceinline__ U4 philox4x64_10(uint64_t c0, uint64_t c1, uint64_t c2, uint64_t c3,
                                            uint64_t k0, uint64_t k1) {
  const uint64_t M0 = 0xD2E7470EE14C6C93ULL, M1 = 0xCA5A826395121157ULL;
  const uint64_t W0 = 0x9E3779B97F4A7C15ULL, W1 = 0xBB67AE8584CAA73BULL;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint64_t hi0 = __umul64hi(M0, c0), lo0 = M0 * c0;
    const uint64_t hi1 = __umul64hi(M1, c2), lo1 = M1 * c2;
    const uint64_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
    k0 += W0; k1 += W1;
  }
  U4 o; o.v[0] = c0; o.v[1] = c1; o.v[2] = c2; o.v[3] = c3;
  return o;
}

__device__ __forceinline__ double u53(uint64_t w) { return (double)(w >> 11) * 0x1.0p-53; }

// ------------------------------------------------------------------ SABR
// z / x(z).  With zz = |z| and r = sign(z) rho (x(z; rho) = -x(-z; -rho)), and s = sqrt(1 - 2 r zz
// + zz^2):  x = log1p(N / (1 - r)),  N = ((s - 1) + zz) = zz (s + 1 - 2r + zz) / (s + 1).
// For r > 0 the factor s + 1 - 2r + zz = (s - r) + (1 - r) + zz is formed from
// s - r = ((1 - r)(1 + r) + zz (zz - 2r)) / (s + r), which avoids the cancellation of s against r
// when r approaches 1; for r <= 0 every term of (zz^2 - 2 r zz)/(s+1) + zz is non-negative.
template <class R>
__device__ __forceinline__ R z_over_x(R z, R rho) {
  typedef Num<R> M;
  const R zz = M::abs_(z);
  if (zz < M::zx_series) return R(1) - R(0.5) * rho * z + (R(2) - R(3) * rho * rho) * z * z / R(12);
  const R r = z < R(0) ? -rho : rho;
  const R s = M::sqrt_(R(1) - R(2) * r * zz + zz * zz);
  R num;
  if (r > R(0)) {
    const R omr = R(1) - r;
    const R smr = (omr * (R(1) + r) + zz * (zz - R(2) * r)) / (s + r);
    num = zz * (smr + omr + zz) / (s + R(1));
  } else {
    num = (zz * zz - R(2) * r * zz) / (s + R(1)) + zz;
  }
  return zz / M::log1p_(num / (R(1) - r));
}

// Hagan et al. (2002): sigma = alpha * inv_den * z/x(z) * (1 + c1 alpha^2 + c2 rho nu alpha
// + c3 (2 - 3 rho^2) nu^2), with z = (nu/alpha) fk l and the market-only constants
// fk = (FK)^{(1-b)/2}, l = log(F/K), inv_den = 1/(fk (1 + (1-b)^2 l^2/24 + (1-b)^4 l^4/1920)),
// c1 = (1-b)^2 T / (24 fk^2), c2 = b T / (4 fk), c3 = T / 24.
template <class R>
__device__ __forceinline__ R sabr_hagan(R alpha, R rho, R nu, R l, R fk, R inv_den, R c1, R c2, R c3) {
  const R z = nu / alpha * fk * l;
  const R zx = z_over_x(z, rho);
  const R corr = R(1) + c1 * alpha * alpha + c2 * rho * nu * alpha + c3 * (R(2) - R(3) * rho * rho) * nu * nu;
  return alpha * inv_den * zx * corr;
}

// Eq. (sigmaHagan): sigma = alpha/fo {1 - (1/2)(omb - rho nu w) m + (1/12)[omb^2 + (2 - 3 rho^2)
// nu^2 w^2 + 3 (omb - rho nu w)] m^2}, w = fo / alpha, fo = F^{1-b}, m = log(K/F) = -l.
template <class R>
__device__ __forceinline__ R sabr_paper(R alpha, R rho, R nu, R l, R fo, R omb) {
  const R w = fo / alpha;
  const R rnw = rho * nu * w;
  const R m = -l;
  return alpha / fo * (R(1) - R(0.5) * (omb - rnw) * m
                       + (omb * omb + (R(2) - R(3) * rho * rho) * nu * nu * w * w + R(3) * (omb - rnw)) * (m * m) / R(12));
}

// ------------------------------------------------------------------ Black
// Phi(x) = erfc(-x / sqrt 2) / 2.  FP64: the library erfc.  FP32: erfc(y) for y = |x|/sqrt 2 in
// the Chebyshev-exponent form t exp(-y^2 + P(t)), t = 1 / (1 + y/2), of Press et al. (Numerical
// Recipes, 2nd ed., Section 6.2), with our own coefficients fitted against 40-digit values
// (csrc/gen_erfc_fit.py; relative error of erfc <= 5.5e-8 on [0, 12] before FP32 rounding).
template <class R> __device__ __forceinline__ R ncdf(R x);
template <> __device__ __forceinline__ double ncdf<double>(double x) {
  return 0.5 * erfc(-x * 0.70710678118654752440);
}
// Coefficient of t^j in the fitted exponent P(t) (csrc/gen_erfc_fit.py).
__host__ __device__ constexpr float erfc_fit(int j) {
  return j == 0 ? -1.265476212e+00f : j == 1 ? +9.992080434e-01f : j == 2 ? +3.816971254e-01f :
         j == 3 ? +5.818804080e-02f : j == 4 ? -6.786663929e-02f : j == 5 ? +4.935479974e-02f :
         j == 6 ? -8.523480751e-01f : j == 7 ? +1.273531464e+00f : j == 8 ? -7.302618493e-01f :
                  +1.539733566e-01f;
}
template <> __device__ __forceinline__ float ncdf<float>(float x) {
  const float y = fabsf(x) * 0.70710678f;
  const float t = rcp_approx(fmaf(0.5f, y, 1.0f));
  float p = erfc_fit(9);
#pragma unroll
  for (int j = 8; j >= 0; --j) p = fmaf(p, t, erfc_fit(j));
  const float half_erfc = 0.5f * t * exp_approx(fmaf(-y, y, p));
  return x < 0.0f ? half_erfc : 1.0f - half_erfc;
}

// ------------------------------------------------------------------ packed FP32 pairs
// Blackwell issues add, mul and fma on a pair of FP32 values in a register pair (.f32x2) as one
// instruction.  The FP32 pricer carries two instruments per lane through these; the hardware
// approximations (rcp, rsqrt, ex2) and the selects act on each half.
__device__ __forceinline__ float2 bc2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.0f, -1.0f), a); }
__device__ __forceinline__ float2 abs2(float2 a) { return make_float2(fabsf(a.x), fabsf(a.y)); }
__device__ __forceinline__ float2 rcp2(float2 a) { return make_float2(rcp_approx(a.x), rcp_approx(a.y)); }
__device__ __forceinline__ float2 rsqrt2(float2 a) { return make_float2(rsqrt_approx(a.x), rsqrt_approx(a.y)); }
__device__ __forceinline__ float2 ex2_2(float2 a) { return make_float2(ex2_approx(a.x), ex2_approx(a.y)); }
__device__ __forceinline__ float2 sel2(bool cx, bool cy, float2 a, float2 b) {
  return make_float2(cx ? a.x : b.x, cy ? a.y : b.y);
}

// log1p on a pair of non-negative arguments.  y < 1/2: the atanh series 2 s (1 + s^2/3 + ... + s^8/9)
// in s = y / (2 + y) (|s| <= 1/5, truncation below 1e-8 relative); y >= 1/2: log2(1 + y) ln 2 on
// the MUFU, where 1 + y carries no cancellation (relative error a few 1e-7).  Both are formed and
// one is selected, so the pair needs no bit-level argument reduction.  An infinite or NaN argument
// takes the second form and comes back infinite or NaN.
__device__ __forceinline__ float2 log1p_pos2(float2 y) {
  const float2 s = mul2(y, rcp2(add2(bc2(2.0f), y)));
  const float2 s2 = mul2(s, s);
  float2 p = fma2(s2, bc2(2.0f / 9.0f), bc2(2.0f / 7.0f));
  p = fma2(s2, p, bc2(2.0f / 5.0f));
  p = fma2(s2, p, bc2(2.0f / 3.0f));
  p = fma2(s2, p, bc2(2.0f));
  const float2 ser = mul2(s, p);
  const float2 u = add2(bc2(1.0f), y);
  const float2 big = mul2(make_float2(lg2_approx(u.x), lg2_approx(u.y)), bc2(0.693147180559945309f));
  return sel2(y.x < 0.5f, y.y < 0.5f, ser, big);
}

// ncdf<float> on a pair, rearranged to save packed instructions: with u = t / 2 = 1 / (2 + y),
// P(t) = sum_j (2^j c_j) u^j, and the exponent goes to the MUFU in base 2, so the coefficients
// are taken as 2^j c_j log2 e (one rounding each) and -y^2 log2 e = (-|x| log2 e / 2) |x|;
// u 2^(...) is then erfc(y) / 2 directly.
__host__ __device__ constexpr float erfc_fit_u2(int j) {
  return (float)((double)erfc_fit(j) * (double)(1 << j) * 1.44269504088896341);
}
__device__ __forceinline__ float2 ncdf2(float2 x) {
  const float2 ax = abs2(x);
  const float2 u = rcp2(fma2(ax, bc2(0.70710678f), bc2(2.0f)));
  float2 p = bc2(erfc_fit_u2(9));
#pragma unroll
  for (int j = 8; j >= 0; --j) p = fma2(p, u, bc2(erfc_fit_u2(j)));
  const float2 m = mul2(ax, bc2(-0.721347520444481703f));   // -|x| log2(e) / 2
  const float2 h = mul2(u, ex2_2(fma2(m, ax, p)));          // erfc(|x| / sqrt 2) / 2
  return sel2(x.x < 0.0f, x.y < 0.0f, h, sub2(bc2(1.0f), h));
}
// ncdf2 for arguments known not to be positive (the far-side Black argument): erfc(-x / sqrt 2) / 2
// with |x| = -x, no select.
__device__ __forceinline__ float2 ncdf2_nonpos(float2 x) {
  const float2 u = rcp2(fma2(x, bc2(-0.70710678f), bc2(2.0f)));
  float2 p = bc2(erfc_fit_u2(9));
#pragma unroll
  for (int j = 8; j >= 0; --j) p = fma2(p, u, bc2(erfc_fit_u2(j)));
  const float2 m = mul2(x, bc2(-0.721347520444481703f));   // -x log2(e) / 2
  return mul2(u, ex2_2(fma2(m, x, p)));
}

// Out-of-the-money Black price with sgn = +1 (call, K >= F) or -1 (put, K < F):
//   P = sgn * DF * (Phi(sgn d1) - KF Phi(sgn d2)),  DF = D F,  KF = K / F,
//   d1 = l / v + v / 2, d2 = d1 - v, v = sigma sqrt(T), l = log(F/K).
template <class R>
__device__ __forceinline__ R black_otm(R sigma, R sqrtT, R l, R DF, R KF, R sgn) {
  const R v = sigma * sqrtT;
  const R d1 = l / v + R(0.5) * v;
  const R d2 = d1 - v;
  return sgn * DF * (ncdf(sgn * d1) - KF * ncdf(sgn * d2));
}

}  // namespace sabr
