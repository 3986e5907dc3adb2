// qk_device.cuh -- per-cell and per-face arithmetic of the update, device side.
// Formulas follow the paper's statement (arXiv:2110.01792, Sec. 2.2); each
// function notes the passage.  T is the stencil type (double for QK_FP64,
// float for QK_FP32_MIXED).
#pragma once

#include "qk_internal.cuh"

namespace qk {

// FP64 reciprocal: the hardware's approximate reciprocal r (PTX
// rcp.approx.ftz.f64, about 20 correct bits, r = (1 - eps)/b) and one
// third-order correction: with e = 1 - b r = eps (one FMA, exact to rounding),
// r (1 + e + e^2) = (1 - eps^3)/b, so the relative error drops to ~2^-60 and
// the result is within an ulp of 1/b after the single rounding of the last FMA
// (normal b with a normal reciprocal; b = 0 or an infinite b give NaN).
// Three FP64 slots against the ~7.5 of an IEEE division on this part.
__device__ __forceinline__ double frcp(double b) {
  double r;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(b));
  const double e = fma(-b, r, 1.0);
  return fma(r, fma(e, e, e), r);
}
__device__ __forceinline__ double qdiv(double a, double b) { return a * frcp(b); }
__device__ __forceinline__ float qdiv(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double qrcp(double b) { return frcp(b); }
// Division that must be exact in FP64 (the HLLC ratio of a stationary contact
// has to come out as exactly 1).
__device__ __forceinline__ double xdiv(double a, double b) { return a / b; }
__device__ __forceinline__ float xdiv(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ float qrcp(float b) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(b));
  return r;
}
__device__ __forceinline__ double qsqrt(double x) { return sqrt(x); }
// Square root of a positive normal double (no infinity): the hardware's
// approximate reciprocal square root y (PTX rsqrt.approx.ftz.f64, about 20
// correct bits) gives s = x y; with e = 1 - s y (one FMA) the exact root is
// s / sqrt(1 - e) up to the rounding of s, and the binomial series
// (1 - e)^(-1/2) = 1 + e/2 + 3e^2/8 + O(e^3) truncated after e^2 leaves a
// relative error ~(5/16) e^3 ~ 2^-58: within an ulp of sqrt(x).  A zero
// argument returns itself (the series would give 0 * inf).  Five FP64 slots
// against 7.6 for the IEEE square root on this part.
__device__ __forceinline__ double psqrt(double x) {
  double y;
  asm("rsqrt.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
  const double s = x * y;
  const double e = fma(-s, y, 1.0);
  const double r = fma(s, e * fma(e, 0.375, 0.5), s);
  return (__double_as_longlong(x) << 1) == 0 ? x : r;
}
__device__ __forceinline__ float qsqrt(float x) {
  float r;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float psqrt(float x) { return qsqrt(x); }
// sqrt(n / d) for a positive normal d and n >= 0 with a normal product n d:
// y ~ 1/sqrt(n d) (rsqrt.approx.ftz.f64) gives s = n y ~ sqrt(n/d), and the
// series of psqrt on e = 1 - (n d) y^2 corrects it to within about an ulp
// (the rounding of n d adds at most 2^-54).  Seven FP64 slots against the
// nine of a reciprocal, a product and psqrt.  A zero n returns zero.
__device__ __forceinline__ double psqrt_div(double n, double d) {
  const double P = n * d;
  double y;
  asm("rsqrt.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(P));
  const double s = n * y;
  const double e = fma(-(P * y), y, 1.0);
  const double r = fma(s, e * fma(e, 0.375, 0.5), s);
  return (__double_as_longlong(n) << 1) == 0 ? n : r;
}
__device__ __forceinline__ float psqrt_div(float n, float d) { return qsqrt(__fdividef(n, d)); }

// float <-> double conversions on the integer pipe.  On GB300 every F2F
// conversion occupies a slot of the 1/64-rate FP64 pipe; these do the same
// with integer operations on the bit patterns.
// f2d: exact widening (normal, subnormal, zero, infinite and NaN floats).
__device__ __forceinline__ double f2d(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned sign = u & 0x80000000u;
  unsigned e = (u >> 23) & 0xffu, m = u & 0x7fffffu;
  if (e == 0u) {
    if (m == 0u) return __hiloint2double((int)sign, 0);
    const int sh = __clz(m) - 8;  // normalise the subnormal: leading 1 to bit 23
    m = (m << sh) & 0x7fffffu;
    e = 1u - (unsigned)sh;        // wraps; the rebias below brings it back in range
  }
  const unsigned ed = e == 0xffu ? 0x7ffu : e + 896u;  // rebias 127 -> 1023
  return __hiloint2double((int)(sign | (ed << 20) | (m >> 3)), (int)(m << 29));
}
// d2f_trunc: narrowing by truncation of the mantissa (within one FP32 ulp,
// toward zero); magnitudes below the normal FP32 range give a signed zero,
// above it the largest finite float (infinities and NaNs map to infinities
// and NaNs).
__device__ __forceinline__ float d2f_trunc(double x) {
  const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
  const unsigned sign = hi & 0x80000000u;
  const int e = (int)((hi >> 20) & 0x7ffu);
  const unsigned m = ((hi & 0xfffffu) << 3) | (lo >> 29);
  if (e == 0x7ff) return __uint_as_float(sign | 0x7f800000u | (m ? 0x400000u : 0u));
  const int fe = e - 896;
  if (fe <= 0) return __uint_as_float(sign);
  if (fe >= 255) return __uint_as_float(sign | 0x7f7fffffu);
  return __uint_as_float(sign | ((unsigned)fe << 23) | m);
}

// Conserved -> primitive (Sec. 2.2.1): v = m / rho, E_g = E - rho v^2 / 2,
// P = (gamma - 1) E_g, with gm1 = gamma - 1 given in the stencil precision
// (formed once per kernel: a conversion per cell would occupy the FP64 pipe).  In mixed precision the internal energy is recovered
// with ~48-bit error-free arithmetic (cancellation of E against the kinetic
// energy), the rest in FP32.
template <typename T>
__device__ __forceinline__ void con2prim(const T u[5], T gm1, T w[5]);

template <>
__device__ __forceinline__ void con2prim<double>(const double u[5], double gm1, double w[5]) {
  double rho = u[0];
  const double inv = frcp(rho);
  double vx = u[1] * inv, vy = u[2] * inv, vz = u[3] * inv;
  double v2 = (vx * vx + vy * vy) + vz * vz;
  double Eg = u[4] - 0.5 * rho * v2;
  w[0] = rho;
  w[1] = vx;
  w[2] = vy;
  w[3] = vz;
  w[4] = gm1 * Eg;
}

// Error-free transformations (Knuth's TwoSum, FMA TwoProduct) for the FP32
// path: a value carried as hi + lo holds about 48 significant bits.
// The operations are the round-to-nearest intrinsics, which the compiler never
// fuses into an FMA with a neighbouring product (a fused operand would break
// the identity s + e = a + b that the transform relies on).
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// Mixed precision: the internal energy E_g = E - |m|^2/(2 rho) is recovered
// with error-free transformations on the FP32 pipe (|m|^2 by FMA TwoProduct
// and TwoSum, the division and the subtraction in hi + lo form), which is as
// accurate as an FP64 recovery relative to the FP32-stored E and costs no FP64
// instruction (one FP64 instruction occupies ~64 FP32 issue slots on GB300).
// Double-float (hi + lo FP32 pair) accumulation for the compensated FP32
// state: (h, l) += x with the rounding error of h + x kept in l by TwoSum.
__device__ __forceinline__ void df_add(float &h, float &l, float x) {
  float s, t;
  two_sum(h, x, s, t);
  h = s;
  l = __fadd_rn(l, t);
}
// Renormalise (h, l) so that h is the FP32 rounding of h + l.
__device__ __forceinline__ void df_norm(float &h, float &l) {
  float s, t;
  two_sum(h, l, s, t);
  h = s;
  l = t;
}

// Per-thread asynchronous copy of one 4- or 8-byte element from global to
// shared memory (cp.async, the L1-allocating form); the copies of a thread are
// committed as a group and waited for by the same thread, which is the only
// reader of what it staged (no barrier needed).
template <typename T>
__device__ __forceinline__ void cp_async_elem(T *dst_smem, const T *src) {
  static_assert(sizeof(T) == 4 || sizeof(T) == 8, "4- or 8-byte elements");
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst_smem);
  if constexpr (sizeof(T) == 4)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}
// Wait until at most N of this thread's most recent groups are pending.
template <int N>
__device__ __forceinline__ void cp_async_wait_group() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Binary exponent and mantissa of a positive normal float (x = fmant(x)
// 2^fexpo(x), fmant in [1, 2)), 2^ex for |ex| <= 126, and m 2^ex for a
// positive normal m (0 below the normal range, infinity above it), on the
// integer pipe.
__device__ __forceinline__ int fexpo(float x) {
  return (int)((__float_as_uint(x) >> 23) & 0xffu) - 127;
}
__device__ __forceinline__ float fmant(float x) {
  return __uint_as_float((__float_as_uint(x) & 0x007fffffu) | 0x3f800000u);
}
__device__ __forceinline__ float pow2f(int ex) { return __uint_as_float((unsigned)(ex + 127) << 23); }
__device__ __forceinline__ float fscale(float m, int ex) {
  const unsigned u = __float_as_uint(m);
  const int be = (int)((u >> 23) & 0xffu) + ex;
  if (be <= 0) return 0.0f;
  if (be >= 255) return __uint_as_float(0x7f800000u);
  return __uint_as_float((u & 0x807fffffu) | ((unsigned)be << 23));
}

// Storage of the low parts of a compensated FP32 state (hi + lo per conserved
// value).  CP = 1: lo as an FP32 value (8 bytes per value in all).  CP = 2: lo
// in 16 bits as the integer k = rint(lo 2^(38 - E)), E the binary exponent of
// hi: after renormalisation |lo| <= ulp(hi)/2 = 2^(E - 24), so |k| <= 2^14, and
// lo is kept to 2^-15 ulp(hi): a 39-bit significand in 6 bytes per value.  A
// CP = 2 array travels as float* and is read and written as int16.  lo is
// dropped (k = 0) where it is zero or below the normal FP32 range (|hi| below
// ~2^-100), and decodes to zero below 2^(E - 38) = 2^-126.
template <int CP>
__device__ __forceinline__ float lo_get(const float *p, long long e, float hi) {
  if constexpr (CP == 2) {
    const int k = reinterpret_cast<const short *>(p)[e];
    if (k == 0) return 0.0f;
    const int E = (int)((__float_as_uint(hi) >> 23) & 0xffu) - 127;
    return fscale((float)k, E - 38);
  } else {
    return p[e];
  }
}
template <int CP>
__device__ __forceinline__ void lo_put(float *p, long long e, float hi, float lo) {
  if constexpr (CP == 2) {
    int k = 0;
    if ((__float_as_uint(lo) & 0x7f800000u) != 0u) {
      const int E = (int)((__float_as_uint(hi) >> 23) & 0xffu) - 127;
      k = min(max(__float2int_rn(fscale(lo, 38 - E)), -32767), 32767);
    }
    reinterpret_cast<short *>(p)[e] = (short)k;
  } else {
    p[e] = lo;
  }
}

// Double-float values (h + l, |l| <= ulp(h)/2, ~48 significant bits) for
// arithmetic that needs more than FP32 without the FP64 pipe (Dekker 1971;
// Knuth's TwoSum; FMA TwoProduct), on round-to-nearest intrinsics so that no
// product is fused into the transforms.  Sums and products end with the fast
// renormalisation (Dekker's FastTwoSum), whose error under cancellation is
// bounded in absolute terms (~2^-48 of the operands), the measure the
// callers need.
struct DF {
  float h, l;
};
__device__ __forceinline__ DF df_fast(float a, float b) {  // |a| >= |b| or a == 0
  const float s = __fadd_rn(a, b);
  return DF{s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ DF df_of(float a, float b) {  // any a, b
  float s, e;
  two_sum(a, b, s, e);
  return DF{s, e};
}
__device__ __forceinline__ DF df_add(DF x, DF y) {
  float s, e;
  two_sum(x.h, y.h, s, e);
  return df_fast(s, __fadd_rn(e, __fadd_rn(x.l, y.l)));
}
__device__ __forceinline__ DF df_neg(DF x) { return DF{-x.h, -x.l}; }
__device__ __forceinline__ DF df_sub(DF x, DF y) { return df_add(x, df_neg(y)); }
__device__ __forceinline__ DF df_add_f(DF x, float b) {
  float s, e;
  two_sum(x.h, b, s, e);
  return df_fast(s, __fadd_rn(e, x.l));
}
__device__ __forceinline__ DF df_mul(DF x, DF y) {
  const float p = __fmul_rn(x.h, y.h);
  const float e = fmaf(x.h, y.h, -p);
  return df_fast(p, __fadd_rn(e, __fadd_rn(__fmul_rn(x.h, y.l), __fmul_rn(x.l, y.h))));
}
__device__ __forceinline__ DF df_mul_f(DF x, float b) {
  const float p = __fmul_rn(x.h, b);
  const float e = fmaf(x.h, b, -p);
  return df_fast(p, __fadd_rn(e, __fmul_rn(x.l, b)));
}

// Internal energy E_g = E - |m|^2/(2 rho) of an FP32 state as an unevaluated
// sum hi + lo (about 48 significant bits), from the velocity reciprocal `inv`
// (~1 ulp of 1/rho).
__device__ __forceinline__ void internal_energy_f32(const float u[5], float rho, float inv,
                                                    float &hi, float &lo) {
  const float px = __fmul_rn(u[1], u[1]), py = __fmul_rn(u[2], u[2]), pz = __fmul_rn(u[3], u[3]);
  float ex = fmaf(u[1], u[1], -px), ey = fmaf(u[2], u[2], -py), ez = fmaf(u[3], u[3], -pz);
  float s1, t1, s2, t2;
  two_sum(px, py, s1, t1);
  two_sum(s1, pz, s2, t2);
  const float l2 = ((t1 + t2) + (ex + ey)) + ez;
  // q = (s2 + l2) / rho as qh + ql
  const float qh = __fmul_rn(s2, inv);
  const float r = fmaf(-qh, rho, s2) + l2;
  const float ql = r * inv;
  // E_g = E - (qh + ql)/2
  float d, dl;
  two_sum(u[4], __fmul_rn(-0.5f, qh), d, dl);
  hi = d;
  lo = dl - 0.5f * ql;
}

template <>
__device__ __forceinline__ void con2prim<float>(const float u[5], float gm1, float w[5]) {
  const float rho = u[0];
  float inv = qrcp(rho);
  inv = inv * fmaf(-rho, inv, 2.0f);  // one Newton step: ~1 ulp
  w[0] = rho;
  w[1] = u[1] * inv;
  w[2] = u[2] * inv;
  w[3] = u[3] * inv;
  float hi, lo;
  internal_energy_f32(u, rho, inv, hi, lo);
  w[4] = gm1 * (hi + lo);
}

// PPM reconstruction of one cell from the stencil s0..s4 = q_{i-2..i+2}
// (Sec. 2.2.1): interface values (7/12)(q_j + q_{j+1}) - (1/12)(q_{j-1} +
// q_{j+2}) grouped symmetrically; clamp to the min/max of the cell and its
// neighbours; at an extremum ((qR - q)(q - qL) <= 0) linear reconstruction
// with the monotonized-central slope; otherwise the CW84 overshoot reset.
template <typename T>
__device__ __forceinline__ void ppm(T s0, T s1, T s2, T s3, T s4, T &qL, T &qR) {
  const T c7 = T(7.0 / 12.0), c1 = T(1.0 / 12.0);
  T fL = c7 * (s1 + s2) - c1 * (s0 + s3);
  T fR = c7 * (s2 + s3) - c1 * (s1 + s4);
  T lo = min(s1, min(s2, s3));
  T hi = max(s1, max(s2, s3));
  T l = min(max(fL, lo), hi);
  T r = min(max(fR, lo), hi);
  if ((r - s2) * (s2 - l) <= T(0)) {
    T dm = s2 - s1, dp = s3 - s2, slope = T(0);
    if (dm * dp > T(0)) {
      T m = min(T(2) * fabs(dm), min(T(2) * fabs(dp), T(0.5) * fabs(dm + dp)));
      slope = dp > T(0) ? m : -m;
    }
    l = s2 - T(0.5) * slope;
    r = s2 + T(0.5) * slope;
  } else {
    T d = r - l;
    T q6 = T(6) * (s2 - T(0.5) * (l + r));
    if (d * q6 > d * d) {
      l = T(3) * s2 - T(2) * r;
    } else if (-(d * d) > d * q6) {
      r = T(3) * s2 - T(2) * l;
    }
  }
  qL = l;
  qR = r;
}

// Exact comparisons of finite doubles on the integer pipe.  On GB300 every
// FP64 instruction, min/max and compare included, occupies a slot of the
// 1/64-rate FP64 pipe; the map key(x) = bits(x) ^ ((bits(x) >> 63) & 0x7ff..f)
// is strictly increasing in x (with -0 < +0) and its own inverse, so min, max
// and order tests of doubles become 64-bit integer operations.
__device__ __forceinline__ long long dkey(double x) {
  const long long b = __double_as_longlong(x);
  return b ^ ((b >> 63) & 0x7fffffffffffffffLL);
}
__device__ __forceinline__ double dunkey(long long k) {
  return __longlong_as_double(k ^ ((k >> 63) & 0x7fffffffffffffffLL));
}
__device__ __forceinline__ bool dle0(double x) { return __double_as_longlong(x) <= 0; }
__device__ __forceinline__ bool dgt0(double x) { return __double_as_longlong(x) > 0; }

// Order of non-negative values (+0 included): doubles compare as their bit
// patterns on the integer pipe; floats use the FP32 comparisons.
__device__ __forceinline__ bool nn_gt(double a, double b) {
  return __double_as_longlong(a) > __double_as_longlong(b);
}
__device__ __forceinline__ bool nn_gt(float a, float b) { return a > b; }
__device__ __forceinline__ double nn_max(double a, double b) { return nn_gt(a, b) ? a : b; }
__device__ __forceinline__ float nn_max(float a, float b) { return fmaxf(a, b); }
__device__ __forceinline__ double nn_min(double a, double b) { return nn_gt(a, b) ? b : a; }
__device__ __forceinline__ float nn_min(float a, float b) { return fminf(a, b); }

// Sign tests and max(0, x) of doubles on the integer pipe (x >= 0 and x <= 0
// hold for both zeros, as IEEE comparisons do); floats use FP32 operations.
__device__ __forceinline__ bool is_ge0(double x) {
  const long long b = __double_as_longlong(x);
  return b >= 0 || (b << 1) == 0;
}
__device__ __forceinline__ bool is_le0(double x) { return __double_as_longlong(x) <= 0; }
__device__ __forceinline__ double pos_part(double x) { return __double_as_longlong(x) > 0 ? x : 0.0; }
__device__ __forceinline__ bool is_ge0(float x) { return x >= 0.0f; }
__device__ __forceinline__ bool is_le0(float x) { return x <= 0.0f; }
__device__ __forceinline__ float pos_part(float x) { return fmaxf(x, 0.0f); }
// The same number (bit patterns for doubles; an FP32 compare for floats).
__device__ __forceinline__ bool same_value(double a, double b) {
  return __double_as_longlong(a) == __double_as_longlong(b);
}
__device__ __forceinline__ bool same_value(float a, float b) { return a == b; }

// Signs of differences of finite doubles from their keys: kzero identifies the
// two zeros (dkey(-0) = -1, dkey(+0) = 0), after which a - b > 0, = 0, < 0
// exactly when kzero(dkey(a)) >, =, < kzero(dkey(b)) (the difference of two
// doubles rounds to zero only when they are equal).  kdiff_same: a - b and
// c - d are nonzero with the same sign, i.e. (a - b)(c - d) > 0.
__device__ __forceinline__ long long kzero(long long k) { return k == -1 ? 0 : k; }
__device__ __forceinline__ bool kdiff_same(long long za, long long zb, long long zc,
                                           long long zd) {
  return (za > zb && zc > zd) || (za < zb && zc < zd);
}

// Product sign tests of finite doubles on the integer pipe: a b > 0 exactly
// when both are nonzero with equal sign bits (a product that underflows to
// zero, |a b| < 2^-1074, counts here as positive).
__device__ __forceinline__ bool dsame_nz(double a, double b) {
  const long long x = __double_as_longlong(a), y = __double_as_longlong(b);
  return (x ^ y) >= 0 && (x << 1) != 0 && (y << 1) != 0;
}

// FP64 PPM interface value between q_j = b and q_{j+1} = c (a = q_{j-1},
// d = q_{j+2}): (7/12)(b + c) - (1/12)(a + d), with the FMA written out so that
// every caller (the stage kernels' shared interface pass, the flux registers
// of mesh refinement) rounds it the same way.
__device__ __forceinline__ double ppm_face(double a, double b, double c, double d) {
  return fma(7.0 / 12.0, b + c, -((1.0 / 12.0) * (a + d)));
}

// The limiter of FP64 PPM for one cell from its two raw interface values fL,
// fR and the cell averages s1, s2, s3 = q_{i-1}, q_i, q_{i+1}, with the
// min/max and every order test on the integer pipe, and the tests rewritten
// to need fewer FP64 operations:
// - extremum, (qR - q)(q - qL) <= 0: a sign test of the two differences;
// - MC slope: half of sign * min(2|dm|, 2|dp|, |dm + dp|/2) is
//   sign * min(|dm|, |dp|, |dm + dp|/4) exactly (scaling by 2 is exact);
// - CW84 overshoot, with d = qR - qL and q6 = 6 (q - (qL + qR)/2):
//   d q6 > d^2  <=>  d (l' - qL) > 0  with l' = 3 q - 2 qR, and
//   -d^2 > d q6 <=>  d (qR - r') > 0  with r' = 3 q - 2 qL
//   (expand d q6 -+ d^2); at the tie l' = qL (r' = qR), so a decision that
//   rounding flips moves the result only by rounding.
// The sign tests compare integer keys instead of forming the differences.
// The values equal the direct evaluation bit for bit except at such ties.
__device__ __forceinline__ void ppm_limit(double fL, double fR, double s1, double s2, double s3,
                                          double &qL, double &qR) {
  const long long k1 = dkey(s1), k2 = dkey(s2), k3 = dkey(s3);
  const long long klo = min(k1, min(k2, k3)), khi = max(k1, max(k2, k3));
  const long long kl = min(max(dkey(fL), klo), khi), kr = min(max(dkey(fR), klo), khi);
  double l = dunkey(kl);
  double r = dunkey(kr);
  // the signs of the differences from the keys (no FP64 subtraction)
  const long long zl = kzero(kl), zr = kzero(kr), z2 = kzero(k2);
  if (!kdiff_same(zr, z2, z2, zl)) {  // (r - q)(q - l) <= 0
    const double dm = s2 - s1, dp = s3 - s2;
    double h = 0.0;  // half the MC slope
    if (dsame_nz(dm, dp)) {
      // positive doubles order like their bit patterns
      const long long a = __double_as_longlong(fabs(dm));
      const long long b = __double_as_longlong(fabs(dp));
      const long long c = __double_as_longlong(0.25 * fabs(dm + dp));
      const long long m = min(a, min(b, c));
      const long long sign = __double_as_longlong(dp) & (long long)0x8000000000000000ULL;
      h = __longlong_as_double(m | sign);
    }
    l = s2 - h;
    r = s2 + h;
  } else {
    // d = r - l has the sign of zr - zl (nonzero: r > q > l or r < q < l)
    const double t3 = 3.0 * s2;
    const double ln = fma(-2.0, r, t3);
    if (kdiff_same(zr, zl, kzero(dkey(ln)), zl)) {  // d (l' - l) > 0
      l = ln;
    } else {
      const double rn = fma(-2.0, l, t3);
      if (kdiff_same(zr, zl, zr, kzero(dkey(rn)))) r = rn;  // d (r - r') > 0
    }
  }
  qL = l;
  qR = r;
}

// FP64 PPM of one cell from its stencil s0..s4 (interface values, then the
// limiter); the stage kernels compute the interface values once per face
// instead and call ppm_limit.
template <>
__device__ __forceinline__ void ppm<double>(double s0, double s1, double s2, double s3,
                                            double s4, double &qL, double &qR) {
  ppm_limit(ppm_face(s0, s1, s2, s3), ppm_face(s1, s2, s3, s4), s1, s2, s3, qL, qR);
}

// FP64 PPM with shared interface values, first pass of one direction D: the
// interface value at the left face of every cell -1 .. v[D]+1 of every line
// along D of the tile (NIFP per line, indexed like the line positions with
// item_index<D>(.., NIFP)), from the cross-slot primitives prim[q], into
// iface[q].  Position p of a line (cell p-1) then reads its raw face values
// at p and p+1: each interface value is computed once instead of twice.
template <int D, int NT, int NV>
__device__ __forceinline__ void ppm_faces_pass(const double (*prim)[NCROSS],
                                               double (*iface)[NIF], const int v[3]) {
  constexpr int A = (D + 1) % 3, B = (D + 2) % 3;
  for (int it = threadIdx.x; it < NIF; it += NT) {
    int k, cc[3];
    item_cell<D>(it, NIFP, k, cc[0], cc[1], cc[2]);
    if (cc[A] >= v[A] || cc[B] >= v[B] || cc[D] > v[D] + 1) continue;
    int s[4];
#pragma unroll
    for (int o = 0; o < 4; ++o) {
      int x[3] = {cc[0], cc[1], cc[2]};
      x[D] += o - 2;
      s[o] = cross_slot(x[0], x[1], x[2]);
    }
#pragma unroll
    for (int q = 0; q < NV; ++q)
      iface[q][it] = ppm_face(prim[q][s[0]], prim[q][s[1]], prim[q][s[2]], prim[q][s[3]]);
  }
}

// PLM with the monotonized-central limiter (van Leer 1977), the paper's
// alternative reconstruction (Sec. 2.2.1): zero slope at an extremum of the
// cell averages, else sign(dq+) min(2|dq-|, 2|dq+|, |dq- + dq+|/2).
template <typename T>
__device__ __forceinline__ void plm(T s1, T s2, T s3, T &qL, T &qR) {
  const T dm = s2 - s1, dp = s3 - s2;
  T slope = T(0);
  if (dm * dp > T(0)) {
    const T m = min(T(2) * fabs(dm), min(T(2) * fabs(dp), T(0.5) * fabs(dm + dp)));
    slope = dp > T(0) ? m : -m;
  }
  qL = s2 - T(0.5) * slope;
  qR = s2 + T(0.5) * slope;
}

template <typename T>
__device__ __forceinline__ void recon(int kind, T s0, T s1, T s2, T s3, T s4, T &qL, T &qR) {
  if (kind == QK_RECON_PLM)
    plm<T>(s1, s2, s3, qL, qR);
  else
    ppm<T>(s0, s1, s2, s3, s4, qL, qR);
}

// HLLC flux normal to axis D (Sec. 2.2.1; Toro 2009, ch. 10) from primitive
// states wL, wR = (rho, vx, vy, vz, P): PVRS pressure estimate for the
// wavespeeds S_L, S_R, contact speed S*, and the HLLC star state written with
// the ratio (S_K - u_K)/(S_K - S*) first so that a stationary contact keeps
// U*_K = U_K exactly (the ratio is taken as exactly 1 when numerator and
// denominator are the same number).  Only one side K enters the flux: the
// supersonic side (S_L >= 0: left, else S_R <= 0: right), else the upwind
// side of the star region (tie S* = 0 -> left); its total energy alone is
// formed.  The transverse momentum fluxes are the mass flux times the
// transverse velocity of K (for the star state,
// m_K a_K + S_K (rho*_K a_K - rho_K a_K) = a_K F_rho).  The region is chosen
// by selects, not branches; in FP64 the sign and order tests run on the
// integer pipe.  sqrt(gamma p / rho) and sqrt(1 + g1 (p*/p_K - 1)) =
// sqrt((p_K + g1 (p* - p_K)) / p_K) are square roots of quotients
// (psqrt_div: one approximate reciprocal square root, no division).
template <typename T, int D>
__device__ __forceinline__ void hllc(const T wL[5], const T wR[5], T gamma, T gm1inv, T g1,
                                     T F[5]) {
  constexpr int A = (D + 1) % 3, B = (D + 2) % 3;
  const T rL = wL[0], uL = wL[1 + D], pL = wL[4];
  const T rR = wR[0], uR = wR[1 + D], pR = wR[4];
  const T cL = psqrt_div(gamma * pL, rL), cR = psqrt_div(gamma * pR, rR);
  // p_pvrs = (pL + pR)/2 - (uR - uL) rbar abar / 2, rbar abar = (rL + rR)(cL + cR)/4
  const T ppvrs =
      T(0.5) * fma(T(-0.25) * (uR - uL), (rL + rR) * (cL + cR), pL + pR);
  const T ps = pos_part(ppvrs);
  // shock branch (the argument exceeds 1): one square root for the first
  // shocked side (left if both), the second only where both sides are
  const bool shL = nn_gt(ps, pL), shR = nn_gt(ps, pR);
  const T p1 = shL ? pL : pR;
  const T q1 = psqrt_div(fma(g1, ps - p1, p1), p1);
  const T qL = shL ? q1 : T(1);
  T qR = shR ? q1 : T(1);
  if (shL && shR) qR = psqrt_div(fma(g1, ps - pR, pR), pR);
  const T SL = uL - cL * qL, SR = uR + cR * qR;
  const T mL = rL * (SL - uL), mR = rR * (SR - uR);
  const T Ss = qdiv(pR - pL + uL * mL - uR * mR, mL - mR);
  const bool supL = is_ge0(SL), supR = !supL && is_le0(SR);
  const bool left = supL || (!supR && is_ge0(Ss));
  const T rK = left ? rL : rR, uK = left ? uL : uR, pK = left ? pL : pR;
  const T aK = left ? wL[1 + A] : wR[1 + A], bK = left ? wL[1 + B] : wR[1 + B];
  const T SK = left ? SL : SR;
  const T EK = pK * gm1inv + T(0.5) * rK * (uK * uK + (aK * aK + bK * bK));
  // physical fluxes of K
  const T mK = rK * uK;
  const T FKn = mK * uK + pK, FKe = uK * (EK + pK);
  // star-state fluxes of K
  const T num = SK - uK, den = SK - Ss;
  const T ratio = same_value(num, den) ? T(1) : qdiv(num, den);
  const T fac = rK * ratio;
  // E*_K = ratio (E_K + (S* - u_K)(rho_K S* + p_K / (S_K - u_K)))
  const T Ue = ratio * fma(Ss - uK, fma(rK, Ss, qdiv(pK, num)), EK);
  const T Fs0 = mK + SK * (fac - rK);
  const T Fsn = FKn + SK * (fac * Ss - mK);
  const T Fse = FKe + SK * (Ue - EK);
  const bool sup = supL || supR;
  const T F0 = sup ? mK : Fs0;
  F[0] = F0;
  F[1 + D] = sup ? FKn : Fsn;
  F[1 + A] = aK * F0;
  F[1 + B] = bK * F0;
  F[4] = sup ? FKe : Fse;
}

// Levermore (1984) closure coefficients of T = a I + b f f (so that the
// n n = f f / |f|^2 term needs no |f|): with s = sqrt(4 - 3 fc^2) and
// (5 + 2 s)(5 - 2 s) = 3 (3 + 4 fc^2), chi = (3 + 4 fc^2)/(5 + 2 s) = (5 - 2 s)/3,
// hence
//   a = (1 - chi)/2 = (s - 1)/3,
//   b = (3 chi - 1)/(2 |f|^2) = (2 - s)/|f|^2 = 3/(2 + s) = 1/(a + 1)   for |f| <= 1
// (2 - s = 3 |f|^2/(2 + s)), and a = 0, b = 1/|f|^2 beyond (fc = 1, chi = 1).
// One square root and one reciprocal, free of cancellation at small |f|.
template <typename T>
__device__ __forceinline__ void levermore_ab_f2(T f2, T &a, T &b) {
  if (nn_gt(f2, T(1))) {
    a = T(0);
    b = qrcp(f2);
    return;
  }
  const T s = psqrt(T(4) - T(3) * f2);  // argument in [1, 4]
  a = fma(s, T(1.0 / 3.0), T(-1.0 / 3.0));
  b = qrcp(a + T(1));                    // 3/(2 + s) = 1/(a + 1)
}

// The same coefficients for every closure of Sec. 2.2.2, selected at compile
// time (CL = QK_CLOSURE_*):
//   Minerbo, chi = 1/3 + (2/15) g, g = 3 fc^2 - fc^3 + 3 fc^4 = fc^2 (3 - fc + 3 fc^2):
//     a = 1/3 - g/15,  b = (3 chi - 1)/(2 |f|^2) = g / (5 |f|^2) = (3 - fc + 3 fc^2)/5
//     for |f| <= 1 (fc^2 = |f|^2); chi = 1 beyond: a = 0, b = 1/|f|^2;
//   Eddington, chi = 1/3: a = 1/3, b = 0 (T = I/3 for every flux).
template <typename T, int CL>
__device__ __forceinline__ void closure_ab_f2(T f2, T &a, T &b) {
  if constexpr (CL == QK_CLOSURE_EDDINGTON) {
    a = T(1) / T(3);
    b = T(0);
  } else if constexpr (CL == QK_CLOSURE_MINERBO) {
    if (nn_gt(f2, T(1))) {
      a = T(0);
      b = qrcp(f2);
    } else {
      const T fc = qsqrt(f2);
      const T h = (T(3) - fc) + T(3) * f2;
      a = T(1) / T(3) - (f2 * h) * (T(1) / T(15));
      b = h * T(0.2);
    }
  } else {
    levermore_ab_f2<T>(f2, a, b);
  }
}

template <typename T, int CL>
__device__ __forceinline__ void closure_ab(T fx, T fy, T fz, T &a, T &b) {
  closure_ab_f2<T, CL>((fx * fx + fy * fy) + fz * fz, a, b);
}

// Column D of the Eddington tensor.
template <typename T, int D, int CL>
__device__ __forceinline__ void eddington_col(T fx, T fy, T fz, T &Tx, T &Ty, T &Tz) {
  T a, b;
  closure_ab<T, CL>(fx, fy, fz, a, b);
  const T fD = D == 0 ? fx : (D == 1 ? fy : fz);
  Tx = b * fx * fD + (D == 0 ? a : T(0));
  Ty = b * fy * fD + (D == 1 ? a : T(0));
  Tz = b * fz * fD + (D == 2 ? a : T(0));
}

// Diagonal element T_DD only (for the HLL wavespeed).
template <typename T, int D, int CL>
__device__ __forceinline__ T eddington_diag(T fx, T fy, T fz) {
  T Tx, Ty, Tz;
  eddington_col<T, D, CL>(fx, fy, fz, Tx, Ty, Tz);
  return D == 0 ? Tx : (D == 1 ? Ty : Tz);
}

}  // namespace qk
