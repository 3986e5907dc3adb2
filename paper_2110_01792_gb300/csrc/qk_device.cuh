// qk_device.cuh -- per-cell and per-face arithmetic of the update, device side.
// Formulas follow the paper's statement (arXiv:2110.01792, Sec. 2.2); each
// function notes the passage.  T is the stencil type (double for QK_FP64,
// float for QK_FP32_MIXED).
#pragma once

#include "qk_internal.cuh"

namespace qk {

// Conserved -> primitive (Sec. 2.2.1): v = m / rho, E_g = E - rho v^2 / 2,
// P = (gamma - 1) E_g.  In mixed precision the internal energy is recovered in
// FP64 (cancellation of E against the kinetic energy), the rest in FP32.
template <typename T>
__device__ __forceinline__ void con2prim(const T u[5], double gamma, T w[5]);

template <>
__device__ __forceinline__ void con2prim<double>(const double u[5], double gamma, double w[5]) {
  double rho = u[0];
  double vx = u[1] / rho, vy = u[2] / rho, vz = u[3] / rho;
  double v2 = (vx * vx + vy * vy) + vz * vz;
  double Eg = u[4] - 0.5 * rho * v2;
  w[0] = rho;
  w[1] = vx;
  w[2] = vy;
  w[3] = vz;
  w[4] = (gamma - 1.0) * Eg;
}

template <>
__device__ __forceinline__ void con2prim<float>(const float u[5], double gamma, float w[5]) {
  float rho = u[0];
  float inv = 1.0f / rho;
  w[0] = rho;
  w[1] = u[1] * inv;
  w[2] = u[2] * inv;
  w[3] = u[3] * inv;
  double m2 = ((double)u[1] * (double)u[1] + (double)u[2] * (double)u[2]) +
              (double)u[3] * (double)u[3];
  double Eg = (double)u[4] - 0.5 * m2 / (double)rho;
  w[4] = (float)((gamma - 1.0) * Eg);
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

// HLLC flux normal to axis D (Sec. 2.2.1; Toro 2009, ch. 10) from primitive
// states wL, wR = (rho, vx, vy, vz, P): PVRS pressure estimate for the
// wavespeeds S_L, S_R, contact speed S*, and the HLLC star state written with
// the ratio (S_K - u_K)/(S_K - S*) first so that a stationary contact keeps
// U*_K = U_K exactly.  The region is chosen by selects, not branches.
template <typename T, int D>
__device__ __forceinline__ void hllc(const T wL[5], const T wR[5], T gamma, T gm1inv, T g1,
                                     T F[5]) {
  constexpr int A = (D + 1) % 3, B = (D + 2) % 3;
  const T rL = wL[0], uL = wL[1 + D], aL_ = wL[1 + A], bL = wL[1 + B], pL = wL[4];
  const T rR = wR[0], uR = wR[1 + D], aR_ = wR[1 + A], bR = wR[1 + B], pR = wR[4];
  const T EL = pL * gm1inv + T(0.5) * rL * (uL * uL + (aL_ * aL_ + bL * bL));
  const T ER = pR * gm1inv + T(0.5) * rR * (uR * uR + (aR_ * aR_ + bR * bR));
  const T cL = sqrt(gamma * pL / rL), cR = sqrt(gamma * pR / rR);
  const T abar = T(0.5) * (cL + cR), rbar = T(0.5) * (rL + rR);
  const T ppvrs = T(0.5) * (pL + pR) - T(0.5) * (uR - uL) * rbar * abar;
  const T ps = max(T(0), ppvrs);
  const T qL = ps <= pL ? T(1) : sqrt(T(1) + g1 * (ps / pL - T(1)));
  const T qR = ps <= pR ? T(1) : sqrt(T(1) + g1 * (ps / pR - T(1)));
  const T SL = uL - cL * qL, SR = uR + cR * qR;
  const T mL = rL * (SL - uL), mR = rR * (SR - uR);
  const T Ss = (pR - pL + uL * mL - uR * mR) / (mL - mR);
  // upwind side K of the star region (tie S* = 0 -> left)
  const bool left = Ss >= T(0);
  const T rK = left ? rL : rR, uK = left ? uL : uR, aK = left ? aL_ : aR_;
  const T bK = left ? bL : bR, pK = left ? pL : pR, EK = left ? EL : ER;
  const T SK = left ? SL : SR;
  const T mK = rK * uK;
  // physical fluxes of K
  const T FK0 = mK, FKn = mK * uK + pK, FKa = mK * aK, FKb = mK * bK, FKe = uK * (EK + pK);
  const T ratio = (SK - uK) / (SK - Ss);
  const T fac = rK * ratio;
  const T Ue = ratio * (EK + rK * (Ss - uK) * (Ss + pK / (rK * (SK - uK))));
  T Fs0 = FK0 + SK * (fac - rK);
  T Fsn = FKn + SK * (fac * Ss - mK);
  T Fsa = FKa + SK * (fac * aK - rK * aK);
  T Fsb = FKb + SK * (fac * bK - rK * bK);
  T Fse = FKe + SK * (Ue - EK);
  // supersonic cases take the upwind physical flux
  if (SL >= T(0)) {
    const T m = rL * uL;
    Fs0 = m; Fsn = m * uL + pL; Fsa = m * aL_; Fsb = m * bL; Fse = uL * (EL + pL);
  } else if (SR <= T(0)) {
    const T m = rR * uR;
    Fs0 = m; Fsn = m * uR + pR; Fsa = m * aR_; Fsb = m * bR; Fse = uR * (ER + pR);
  }
  F[0] = Fs0;
  F[1 + D] = Fsn;
  F[1 + A] = Fsa;
  F[1 + B] = Fsb;
  F[4] = Fse;
}

// Levermore closure (eq. M1_closure): column D of the Eddington tensor
// T = P_r / E_r for the reduced flux f, with |f| rescaled to 1 for the closure
// when |f| > 1 and the n n term dropped when f = 0 (Sec. 2.2.2).  Written with
// n_i n_D = f_i f_D / |f|^2, so the rescaling never needs |f| itself:
//   T_iD = (1 - chi)/2 delta_iD + (3 chi - 1)/2 f_i f_D / |f|^2,
//   chi = (3 + 4 fc^2) / (5 + 2 sqrt(4 - 3 fc^2)),  fc^2 = min(|f|^2, 1).
template <typename T, int D>
__device__ __forceinline__ void eddington_col(T fx, T fy, T fz, T &Tx, T &Ty, T &Tz) {
  const T f2 = (fx * fx + fy * fy) + fz * fz;
  const T fc2 = min(f2, T(1));
  const T chi = (T(3) + T(4) * fc2) / (T(5) + T(2) * sqrt(T(4) - T(3) * fc2));
  const T a = T(0.5) * (T(1) - chi);
  const T bc = f2 > T(0) ? T(0.5) * (T(3) * chi - T(1)) / f2 : T(0);
  const T fD = D == 0 ? fx : (D == 1 ? fy : fz);
  Tx = bc * fx * fD + (D == 0 ? a : T(0));
  Ty = bc * fy * fD + (D == 1 ? a : T(0));
  Tz = bc * fz * fD + (D == 2 ? a : T(0));
}

// Diagonal element T_DD only (for the HLL wavespeed).
template <typename T, int D>
__device__ __forceinline__ T eddington_diag(T fx, T fy, T fz) {
  T Tx, Ty, Tz;
  eddington_col<T, D>(fx, fy, fz, Tx, Ty, Tz);
  return D == 0 ? Tx : (D == 1 ? Ty : Tz);
}

}  // namespace qk
