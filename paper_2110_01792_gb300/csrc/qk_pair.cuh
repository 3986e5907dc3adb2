// qk_pair.cuh -- the FP32 reconstruction and HLLC flux of Sec. 2.2.1 on two
// independent lanes at once, with Blackwell's packed FP32 arithmetic
// (add/mul/fma.rn.f32x2: one instruction issues both lanes).  The column
// kernels pair an x item with a y item of the same plane (two reconstruction
// positions, or two faces), so that every add, multiply and FMA of the
// formulas issues once for both; minima, maxima, comparisons, selections and
// the special-function approximations (reciprocal, square root) stay per lane.
// The formulas are those of ppm / plm / hllc in qk_device.cuh, lane by lane.
#pragma once
#include "qk_device.cuh"

namespace qk {

typedef float2 f2;

__device__ __forceinline__ f2 p2(float a) { return make_float2(a, a); }
__device__ __forceinline__ f2 add2(f2 a, f2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ f2 mul2(f2 a, f2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c) { return __ffma2_rn(a, b, c); }
// a - b as fma(b, -1, a): one packed instruction, exact like a subtraction
__device__ __forceinline__ f2 sub2(f2 a, f2 b) { return __ffma2_rn(b, p2(-1.0f), a); }
// three-input FP32 minimum / maximum (one instruction on sm_100 and later)
__device__ __forceinline__ float fmin3f(float a, float b, float c) {
  float d;
  asm("min.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
  return d;
}
__device__ __forceinline__ float fmax3f(float a, float b, float c) {
  float d;
  asm("max.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
  return d;
}
__device__ __forceinline__ f2 min2(f2 a, f2 b) { return make_float2(fminf(a.x, b.x), fminf(a.y, b.y)); }
__device__ __forceinline__ f2 max2(f2 a, f2 b) { return make_float2(fmaxf(a.x, b.x), fmaxf(a.y, b.y)); }
__device__ __forceinline__ f2 rcp2(f2 a) { return make_float2(qrcp(a.x), qrcp(a.y)); }
__device__ __forceinline__ f2 sqrt2(f2 a) { return make_float2(qsqrt(a.x), qsqrt(a.y)); }
__device__ __forceinline__ f2 sel2(bool cx, bool cy, f2 a, f2 b) {
  return make_float2(cx ? a.x : b.x, cy ? a.y : b.y);
}

// PPM of one cell per lane from the stencil s0..s4 (ppm in qk_device.cuh):
// interface values, clamp to the neighbours' range, linear MC reconstruction
// at an extremum ((qR - q)(q - qL) <= 0), else the CW84 overshoot resets.
// The MC half slope is sign(dp) min(|dm|, |dp|, |dm + dp|/4) (half of the
// slope min(2|dm|, 2|dp|, |dm + dp|/2), scaling by 2 being exact), and the
// CW84 tests d q6 > d^2 and -d^2 > d q6 are d (l' - qL) > 0 and
// d (qR - r') > 0 with l' = 3q - 2qR, r' = 3q - 2qL (expand d q6 -+ d^2).
__device__ __forceinline__ void ppm2(f2 s0, f2 s1, f2 s2, f2 s3, f2 s4, f2 &qL, f2 &qR) {
  const f2 fL = fma2(p2(7.0f / 12.0f), add2(s1, s2), mul2(p2(-1.0f / 12.0f), add2(s0, s3)));
  const f2 fR = fma2(p2(7.0f / 12.0f), add2(s2, s3), mul2(p2(-1.0f / 12.0f), add2(s1, s4)));
  const f2 lo = make_float2(fmin3f(s1.x, s2.x, s3.x), fmin3f(s1.y, s2.y, s3.y));
  const f2 hi = make_float2(fmax3f(s1.x, s2.x, s3.x), fmax3f(s1.y, s2.y, s3.y));
  const f2 l = min2(max2(fL, lo), hi), r = min2(max2(fR, lo), hi);
  const f2 dm = sub2(s2, s1), dp = sub2(s3, s2);
  const f2 pr = mul2(dm, dp);
  const f2 q4 = mul2(p2(0.25f), add2(dm, dp));
  f2 h;
  h.x = pr.x > 0.0f ? copysignf(fmin3f(fabsf(dm.x), fabsf(dp.x), fabsf(q4.x)), dp.x) : 0.0f;
  h.y = pr.y > 0.0f ? copysignf(fmin3f(fabsf(dm.y), fabsf(dp.y), fabsf(q4.y)), dp.y) : 0.0f;
  const f2 t3 = mul2(p2(3.0f), s2);
  const f2 ln = fma2(p2(-2.0f), r, t3), rn = fma2(p2(-2.0f), l, t3);
  const f2 d = sub2(r, l);
  const f2 a1 = mul2(d, sub2(ln, l)), a2 = mul2(d, sub2(r, rn));
  const f2 ex = mul2(sub2(r, s2), sub2(s2, l));
  const f2 lh = sub2(s2, h), rh = add2(s2, h);
  const bool ex_x = ex.x <= 0.0f, ex_y = ex.y <= 0.0f;
  const bool c1x = a1.x > 0.0f, c1y = a1.y > 0.0f;
  const bool c2x = !c1x && a2.x > 0.0f, c2y = !c1y && a2.y > 0.0f;
  qL = sel2(ex_x, ex_y, lh, sel2(c1x, c1y, ln, l));
  qR = sel2(ex_x, ex_y, rh, sel2(c2x, c2y, rn, r));
}

// PLM with the MC limiter per lane (plm in qk_device.cuh).
__device__ __forceinline__ void plm2(f2 s1, f2 s2, f2 s3, f2 &qL, f2 &qR) {
  const f2 dm = sub2(s2, s1), dp = sub2(s3, s2);
  const f2 pr = mul2(dm, dp);
  const f2 q4 = mul2(p2(0.25f), add2(dm, dp));
  f2 h;
  h.x = pr.x > 0.0f ? copysignf(fmin3f(fabsf(dm.x), fabsf(dp.x), fabsf(q4.x)), dp.x) : 0.0f;
  h.y = pr.y > 0.0f ? copysignf(fmin3f(fabsf(dm.y), fabsf(dp.y), fabsf(q4.y)), dp.y) : 0.0f;
  qL = sub2(s2, h);
  qR = add2(s2, h);
}

__device__ __forceinline__ void recon2(int kind, f2 s0, f2 s1, f2 s2, f2 s3, f2 s4, f2 &qL,
                                       f2 &qR) {
  if (kind == QK_RECON_PLM)
    plm2(s1, s2, s3, qL, qR);
  else
    ppm2(s0, s1, s2, s3, s4, qL, qR);
}

// One-lane forms of the packed helpers (float), so that the radiation
// closure and face flux below can run on one face as well as on a pair: the
// same IEEE operations in the same order, lane by lane, hence the same bits
// as the lane of a pair.
__device__ __forceinline__ float add2(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float mul2(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float fma2(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ float sub2(float a, float b) { return __fmaf_rn(b, -1.0f, a); }
__device__ __forceinline__ float rcp2(float a) { return qrcp(a); }
__device__ __forceinline__ float sqrt2(float a) { return qsqrt(a); }
__device__ __forceinline__ float max2(float a, float b) { return fmaxf(a, b); }
__device__ __forceinline__ f2 abs2(f2 a) { return make_float2(fabsf(a.x), fabsf(a.y)); }
__device__ __forceinline__ float abs2(float a) { return fabsf(a); }
template <class V> __device__ __forceinline__ V splat(float a);
template <> __device__ __forceinline__ f2 splat<f2>(float a) { return p2(a); }
template <> __device__ __forceinline__ float splat<float>(float a) { return a; }
// per-lane conditions: a pair of flags (two lanes) or one flag (one lane)
struct M2 {
  bool x, y;
};
__device__ __forceinline__ M2 gt(f2 a, f2 b) { return M2{a.x > b.x, a.y > b.y}; }
__device__ __forceinline__ bool gt(float a, float b) { return a > b; }
__device__ __forceinline__ M2 m_or(M2 a, M2 b) { return M2{a.x || b.x, a.y || b.y}; }
__device__ __forceinline__ bool m_or(bool a, bool b) { return a || b; }
__device__ __forceinline__ M2 m_and(M2 a, M2 b) { return M2{a.x && b.x, a.y && b.y}; }
__device__ __forceinline__ bool m_and(bool a, bool b) { return a && b; }
__device__ __forceinline__ M2 m_not(M2 a) { return M2{!a.x, !a.y}; }
__device__ __forceinline__ bool m_not(bool a) { return !a; }
__device__ __forceinline__ M2 ge(f2 a, f2 b) { return M2{a.x >= b.x, a.y >= b.y}; }
__device__ __forceinline__ bool ge(float a, float b) { return a >= b; }
__device__ __forceinline__ M2 eq(f2 a, f2 b) { return M2{a.x == b.x, a.y == b.y}; }
__device__ __forceinline__ bool eq(float a, float b) { return a == b; }
__device__ __forceinline__ bool any(M2 m) { return m.x || m.y; }
__device__ __forceinline__ bool any(bool m) { return m; }
__device__ __forceinline__ f2 sel(M2 m, f2 a, f2 b) { return sel2(m.x, m.y, a, b); }
__device__ __forceinline__ float sel(bool m, float a, float b) { return m ? a : b; }

// HLLC flux per lane (hllc in qk_device.cuh) from face states given in the
// face's own frame: w = (rho, u_n, u_t1, u_t2, P), u_n the velocity normal to
// the face; F = (mass, normal momentum, t1 momentum, t2 momentum, energy)
// fluxes; V = f2 (two faces) or float (one).  Each lane may be a face of
// another direction; the caller maps the components.  PVRS pressure, shock
// factors (the second square root only where both sides are shocked), S*,
// and the flux of the side K that the face's region selects; the star ratio
// (S_K - u_K)/(S_K - S*) is exactly 1 when numerator and denominator are the
// same number.
template <class V>
__device__ __forceinline__ void hllc2(const V wL[5], const V wR[5], float gamma, float gm1inv,
                                      float g1, V F[5]) {
  const V rL = wL[0], uL = wL[1], pL = wL[4];
  const V rR = wR[0], uR = wR[1], pR = wR[4];
  const V zero = splat<V>(0.0f), one = splat<V>(1.0f);
  // c = sqrt(gamma p / rho)
  const V cL = sqrt2(mul2(mul2(splat<V>(gamma), pL), rcp2(rL)));
  const V cR = sqrt2(mul2(mul2(splat<V>(gamma), pR), rcp2(rR)));
  // p_pvrs = (pL + pR)/2 - (uR - uL)(rL + rR)(cL + cR)/8
  const V ppv = mul2(splat<V>(0.5f), fma2(mul2(splat<V>(-0.25f), sub2(uR, uL)),
                                          mul2(add2(rL, rR), add2(cL, cR)), add2(pL, pR)));
  const V ps = max2(ppv, zero);
  const auto shL = gt(ps, pL), shR = gt(ps, pR);
  // shock factor sqrt((p_K + g1 (p* - p_K)) / p_K) for the first shocked side
  // (left if both), and for the right side where both are shocked
  const V p1 = sel(shL, pL, pR);
  const V q1 = sqrt2(mul2(fma2(splat<V>(g1), sub2(ps, p1), p1), rcp2(p1)));
  V qL = sel(shL, q1, one);
  V qR = sel(shR, q1, one);
  const auto both = m_and(shL, shR);
  if (any(both)) {
    const V q2 = sqrt2(mul2(fma2(splat<V>(g1), sub2(ps, pR), pR), rcp2(pR)));
    qR = sel(both, q2, qR);
  }
  const V SL = sub2(uL, mul2(cL, qL)), SR = fma2(cR, qR, uR);
  const V mL = mul2(rL, sub2(SL, uL)), mR = mul2(rR, sub2(SR, uR));
  // S* = (pR - pL + uL mL - uR mR) / (mL - mR)
  const V nS = sub2(fma2(uL, mL, sub2(pR, pL)), mul2(uR, mR));
  const V Ss = mul2(nS, rcp2(sub2(mL, mR)));
  const auto supL = ge(SL, zero);
  const auto supR = m_and(m_not(supL), ge(zero, SR));
  const auto lft = m_or(supL, m_and(m_not(supR), ge(Ss, zero)));
  const V rK = sel(lft, rL, rR), uK = sel(lft, uL, uR), pK = sel(lft, pL, pR);
  const V aK = sel(lft, wL[2], wR[2]), bK = sel(lft, wL[3], wR[3]);
  const V SK = sel(lft, SL, SR);
  // E_K = p_K/(gamma - 1) + rho_K (u_K^2 + (a_K^2 + b_K^2)) / 2
  const V v2 = fma2(uK, uK, fma2(aK, aK, mul2(bK, bK)));
  const V EK = fma2(pK, splat<V>(gm1inv), mul2(mul2(splat<V>(0.5f), rK), v2));
  const V mK = mul2(rK, uK);
  const V FKn = fma2(mK, uK, pK), FKe = mul2(uK, add2(EK, pK));
  const V num = sub2(SK, uK), den = sub2(SK, Ss);
  const V rq = mul2(num, rcp2(den));
  const V ratio = sel(eq(num, den), one, rq);
  const V fac = mul2(rK, ratio);
  // E*_K = ratio (E_K + (S* - u_K)(rho_K S* + p_K / (S_K - u_K)))
  const V Ue = mul2(ratio, fma2(sub2(Ss, uK), fma2(rK, Ss, mul2(pK, rcp2(num))), EK));
  const V Fs0 = fma2(SK, sub2(fac, rK), mK);
  const V Fsn = fma2(SK, sub2(mul2(fac, Ss), mK), FKn);
  const V Fse = fma2(SK, sub2(Ue, EK), FKe);
  const auto sup = m_or(supL, supR);
  const V F0 = sel(sup, mK, Fs0);
  F[0] = F0;
  F[1] = sel(sup, FKn, Fsn);
  F[2] = mul2(aK, F0);
  F[3] = mul2(bK, F0);
  F[4] = sel(sup, FKe, Fse);
}

// Closure coefficients of T = a I + b f f per lane from |f|^2 (closure_ab_f2
// in qk_device.cuh, closure CL); V = f2 (two lanes) or float (one).
template <int CL, class V>
__device__ __forceinline__ void closure_ab2(V fsq, V &a, V &b) {
  if constexpr (CL == QK_CLOSURE_EDDINGTON) {
    a = splat<V>(1.0f / 3.0f);
    b = splat<V>(0.0f);
  } else {
    const auto sup = gt(fsq, splat<V>(1.0f));
    if constexpr (CL == QK_CLOSURE_MINERBO) {
      const V fc = sqrt2(fsq);
      const V h = fma2(splat<V>(3.0f), fsq, sub2(splat<V>(3.0f), fc));
      a = sub2(splat<V>(1.0f / 3.0f), mul2(mul2(fsq, h), splat<V>(1.0f / 15.0f)));
      b = mul2(h, splat<V>(0.2f));
    } else {
      // Levermore: s = sqrt(4 - 3 |f|^2), a = (s - 1)/3, b = 1/(a + 1)
      const V sq = sqrt2(fma2(splat<V>(-3.0f), fsq, splat<V>(4.0f)));
      a = fma2(sq, splat<V>(1.0f / 3.0f), splat<V>(-1.0f / 3.0f));
      b = rcp2(add2(a, splat<V>(1.0f)));
    }
    // |f| > 1: chi = 1, a = 0, b = 1/|f|^2
    if (any(sup)) {
      const V ib = rcp2(fsq);
      a = sel(sup, splat<V>(0.0f), a);
      b = sel(sup, ib, b);
    }
  }
}

// The radiation HLL face flux per lane (rad_face_hll in qk_rad.cuh), each
// lane in its face's own frame: w = (E_r, f_n, f_t1, f_t2), out = (energy
// flux, F_n flux, F_t1 flux, F_t2 flux); V = f2 (two faces) or float (one).
// averages(avL, avR) supplies the two cell averages in the same frame
// (called only when some lane needs them): they replace the lane's face
// states where either of them has |f| > 1; S the lane's wavespeed, rka / rkb
// the cells' rho kappa_R.
template <int CL, class V, class Averages>
__device__ __forceinline__ void rad_face_hll2(V wL[4], V wR[4], Averages averages, V S, V rka,
                                              V rkb, V dx, float c, float chat, float hchat_c,
                                              float hccc, int tau_corr, V out[4]) {
  const V one = splat<V>(1.0f);
  V fL2 = fma2(wL[3], wL[3], fma2(wL[1], wL[1], mul2(wL[2], wL[2])));
  V fR2 = fma2(wR[3], wR[3], fma2(wR[1], wR[1], mul2(wR[2], wR[2])));
  const auto fb = m_or(gt(fL2, one), gt(fR2, one));
  if (any(fb)) {
    V avL[4], avR[4];
    averages(avL, avR);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      wL[q] = sel(fb, avL[q], wL[q]);
      wR[q] = sel(fb, avR[q], wR[q]);
    }
    fL2 = fma2(wL[3], wL[3], fma2(wL[1], wL[1], mul2(wL[2], wL[2])));
    fR2 = fma2(wR[3], wR[3], fma2(wR[1], wR[1], mul2(wR[2], wR[2])));
  }
  V aL, bL, aR, bR;
  closure_ab2<CL>(fL2, aL, bL);
  closure_ab2<CL>(fR2, aR, bR);
  const V EL = wL[0], ER = wR[0], fLD = wL[1], fRD = wR[1];
  V eps = one;
  if (tau_corr) {
    const V tau = mul2(mul2(dx, splat<V>(0.5f)), add2(rka, rkb));
    const auto thick = gt(tau, one);
    if (any(thick)) eps = sel(thick, rcp2(tau), eps);
  }
  const V hS = mul2(splat<V>(0.5f), S);
  V hSe = mul2(hS, eps);
  const V FE = mul2(splat<V>(hchat_c * c), fma2(EL, fLD, mul2(ER, fRD)));
  const V dE = sub2(ER, EL);
  V o0 = sub2(FE, mul2(hSe, dE));
  // the correction is dropped where the energy flux would exceed chat max(E_L, E_R)
  const auto keep = m_and(gt(one, eps), gt(abs2(o0), mul2(splat<V>(chat), max2(EL, ER))));
  if (any(keep)) {
    hSe = sel(keep, hS, hSe);
    o0 = sub2(FE, mul2(hSe, dE));
  }
  out[0] = o0;
  const V hSec = mul2(hSe, splat<V>(c));
  const V cEbL = mul2(splat<V>(hccc), EL), cEbR = mul2(splat<V>(hccc), ER);
  const V alL = fma2(mul2(cEbL, bL), fLD, mul2(hSec, EL));
  const V alR = sub2(mul2(mul2(cEbR, bR), fRD), mul2(hSec, ER));
  out[2] = fma2(alL, wL[2], mul2(alR, wR[2]));
  out[3] = fma2(alL, wL[3], mul2(alR, wR[3]));
  out[1] = fma2(alL, fLD, fma2(alR, fRD, fma2(cEbL, aL, mul2(cEbR, aR))));
}

}  // namespace qk
