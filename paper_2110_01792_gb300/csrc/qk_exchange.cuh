// qk_exchange.cuh -- the implicit matter-radiation exchange of one cell
// (Sec. 2.2.3 of arXiv:2110.01792), shared by the exchange kernels and the
// epilogue of the radiation stage 2 that fuses it (the exchange is pointwise
// and follows the transport of every substep).
#pragma once
#include "qk_device.cuh"

namespace qk {

template <typename T>
__device__ __forceinline__ double load_d(const T *p, long long e) { return (double)p[e]; }

// |x| < t for a finite positive threshold t: doubles compare as bit
// patterns on the integer pipe (NaN fails); floats use the FP32 compare.
__device__ __forceinline__ bool abs_below(double x, double t) {
  return (__double_as_longlong(x) & 0x7fffffffffffffffLL) < __double_as_longlong(t);
}
__device__ __forceinline__ bool abs_below(float x, float t) { return fabsf(x) < t; }
// x > 0 and finite, on the integer pipe; floats by FP32 compares.
__device__ __forceinline__ bool pos_finite(double x) {
  const long long b = __double_as_longlong(x);
  return b > 0 && b < 0x7ff0000000000000LL;
}
__device__ __forceinline__ bool pos_finite(float x) { return x > 0.0f && x <= 3.402823466e38f; }
// a positive normal float
__device__ __forceinline__ bool pos_normal(float x) {
  return x >= 1.175494351e-38f && x <= 3.402823466e38f;
}

// Newton-Raphson on (E_g, E_r) for one cell (Sec. 2.2.3, eqs. delta_er and
// delta_eg).  R = dt rho kappa_P chat (a_r T^4 - E_r) (the '4 pi B' of the
// paper read as chat a_r T^4), F_G = (E_g - E_g0) + (c/chat) R,
// F_R = (E_r - E_r0) - R; with a radiation source S the callers pass
// E_r0 + S for E_r0 (F_R = (E_r - E_r0) - (R + S); the Jacobian does not
// change).  Convergence |F_G/E_tot| < eps and |(c/chat) F_R / E_tot| < eps,
// E_tot = E_g0 + (c/chat)(E_r0 + S), tested as |F_G| < thr_g = eps E_tot and
// |F_R| < thr_r = thr_g chat/c; the update of the iterate that passes is
// applied, then the loop stops.  With k = dt rho kappa_P chat and
// T = E_g/(rho c_v), R = A E_g^4 - k E_r with A = k a_r/(rho c_v)^4 (for the
// alpha T^3 heat capacity, T^4 = 4 E_g/alpha: R = A E_g - k E_r with
// A = 4 k a_r/alpha; `alpha_eos`).  The 2x2 elimination of eqs.
// delta_er / delta_eg is evaluated with one division: with G = dF_G/dE_g,
//   dE_r = -(F_R G + R' F_G) / D1,  D1 = (dF_R/dE_r) G + R' (dF_G/dE_r),
//   dE_g = -(F_G + dE_r dF_G/dE_r) / G,
// and 1/D1, 1/G taken from the single reciprocal of D1 G.  Starts from
// (Eg, Er) (the cell state, or a warm start); returns the iteration count,
// or -1 after max_iter iterations.
template <typename R_>
__device__ __forceinline__ int newton_exchange(bool alpha_eos, R_ A, R_ k, R_ cr, R_ Eg0, R_ Er0,
                                               R_ thr_g, R_ thr_r, int max_iter, R_ &Eg,
                                               R_ &Er) {
  const R_ dFG_dEr = -cr * k;     // -c dt rho kappa_P
  const R_ dFR_dEr = R_(1) + k;
  const R_ A4 = R_(4) * A;
  bool conv = false;
  int it = 0;
  for (it = 0; it < max_iter; ++it) {
    R_ Rr, dRdEg;
    if (alpha_eos) {
      Rr = fma(A, Eg, -(k * Er));
      dRdEg = A;
    } else {
      const R_ E2 = Eg * Eg;
      Rr = fma(A, E2 * E2, -(k * Er));
      dRdEg = A4 * E2 * Eg;
    }
    const R_ FG = (Eg - Eg0) + cr * Rr;
    const R_ FR = (Er - Er0) - Rr;
    conv = abs_below(FG, thr_g) && abs_below(FR, thr_r);
    const R_ G = R_(1) + cr * dRdEg;
    const R_ D1 = dFR_dEr * G + dRdEg * dFG_dEr;
    const R_ inv = qrcp(D1 * G);
    const R_ dEr = -(FR * G + dRdEg * FG) * (G * inv);
    const R_ dEg = -(FG + dEr * dFG_dEr) * (D1 * inv);
    Er += dEr;
    Eg += dEg;
    if (conv) break;
  }
  return conv ? it + 1 : -1;
}

// Warp-aggregated status update of the exchange kernels.
__device__ __forceinline__ void exchange_status(Status *st, int my_max, unsigned my_flags,
                                                unsigned long long my_bad) {
  const unsigned full = 0xffffffffu;
  int wmax = __reduce_max_sync(full, my_max);
  unsigned wflags = __reduce_or_sync(full, my_flags);
  unsigned long long wbad = my_bad;
  for (int o = 16; o > 0; o >>= 1) wbad = min(wbad, __shfl_xor_sync(full, wbad, o));
  if ((threadIdx.x & 31) == 0) {
    atomicMax(&st->max_iter, wmax);
    if (wflags) {
      atomicOr(&st->flags, wflags);
      atomicMin(&st->first_bad, wbad);
    }
  }
}

// Mixed-precision Newton for one cell: the residuals F_G, F_R are evaluated
// in FP64 at the FP64 iterate (R = A E_g^4 - k E_r as in newton_exchange,
// with the coefficients A, k given to FP32 accuracy), the convergence test on
// their FP32 roundings against the FP32 thresholds, and the 2x2 correction
// (the same elimination as newton_exchange) is solved in FP32 (iterative
// refinement: each iteration gains ~7 digits, so two iterations from an FP32
// warm start reach the 1e-10 tolerance).  Returns the iteration count or -1.
__device__ __forceinline__ int newton_refine(bool alpha_eos, int max_iter, double A, double k,
                                             double cr, double Eg0, double Er0, float Af,
                                             float kf, float crf, float thr_g, float thr_r,
                                             double &Eg, double &Er) {
  const float dFG_dEr = -crf * kf, dFR_dEr = 1.0f + kf;
  const float A4 = 4.0f * Af;
  bool conv = false;
  int it = 0;
  for (it = 0; it < max_iter; ++it) {
    double Rr;
    float dRdEg;
    if (alpha_eos) {
      Rr = fma(A, Eg, -(k * Er));
      dRdEg = Af;
    } else {
      const double E2 = Eg * Eg;
      Rr = fma(A, E2 * E2, -(k * Er));
      const float Ef = d2f_trunc(Eg);
      dRdEg = A4 * Ef * Ef * Ef;
    }
    // the FP32 correction needs the residuals to FP32 accuracy only: narrowed
    // on the integer pipe
    const float fg = d2f_trunc((Eg - Eg0) + cr * Rr);
    const float fr = d2f_trunc((Er - Er0) - Rr);
    conv = fabsf(fg) < thr_g && fabsf(fr) < thr_r;
    const float G = 1.0f + crf * dRdEg;
    const float D1 = dFR_dEr * G + dRdEg * dFG_dEr;
    const float inv = qrcp(D1 * G);
    const float dEr = -(fr * G + dRdEg * fg) * (G * inv);
    const float dEg = -(fg + dEr * dFG_dEr) * (D1 * inv);
    Er += f2d(dEr);
    Eg += f2d(dEg);
    if (conv) break;
  }
  return conv ? it + 1 : -1;
}

// The same refinement with double-float residuals and iterates (~48
// significant bits, on the FP32 pipes): the residual of a cell is evaluated
// to ~2^-46 k (c/chat) E_tot, well inside the 1e-10 tolerance while
// k (c/chat) <= 1e3 (the callers use newton_refine beyond).  A, k are FP32
// numbers (the coefficients of the equations being solved), cr = c/chat is a
// double-float constant.
__device__ __forceinline__ int newton_refine_df(bool alpha_eos, int max_iter, float Af, float kf,
                                                DF cr, float crf, DF Eg0, DF Er0, float thr_g,
                                                float thr_r, DF &Eg, DF &Er) {
  const float dFG_dEr = -crf * kf, dFR_dEr = 1.0f + kf;
  const float A4 = 4.0f * Af;
  bool conv = false;
  int it = 0;
  for (it = 0; it < max_iter; ++it) {
    DF Rr;
    float dRdEg;
    if (alpha_eos) {
      Rr = df_sub(df_mul_f(Eg, Af), df_mul_f(Er, kf));
      dRdEg = Af;
    } else {
      const DF E2 = df_mul(Eg, Eg);
      Rr = df_sub(df_mul_f(df_mul(E2, E2), Af), df_mul_f(Er, kf));
      dRdEg = A4 * Eg.h * Eg.h * Eg.h;
    }
    const DF FG = df_add(df_sub(Eg, Eg0), df_mul(cr, Rr));
    const DF FR = df_sub(df_sub(Er, Er0), Rr);
    const float fg = FG.h, fr = FR.h;
    conv = fabsf(fg) < thr_g && fabsf(fr) < thr_r;
    const float G = 1.0f + crf * dRdEg;
    const float D1 = dFR_dEr * G + dRdEg * dFG_dEr;
    const float inv = qrcp(D1 * G);
    const float dEr = -(fr * G + dRdEg * fg) * (G * inv);
    const float dEg = -(fg + dEr * dFG_dEr) * (D1 * inv);
    Er = df_add_f(Er, dEr);
    Eg = df_add_f(Eg, dEg);
    if (conv) break;
  }
  return conv ? it + 1 : -1;
}

// Constants of the exchange (host or device; the substep dt is passed apart,
// since inside a captured step it is read from device memory).
struct ExK {
  double cr, icc_d, rc_d, inv_cv;
  double a_e;             // a_r, or 4 a_r/alpha for the alpha T^3 heat capacity
  float icc, rc, icc_lo;  // FP32 forms; icc_lo: 1/(c chat) - icc
  float crf, a_ef, inv_cvf, kchat;  // kchat: kappa_P chat (or kappa0 chat)
  float kRf, chatf, epsf;          // kappa_R (or kappa0), chat, the Newton tolerance
  DF cr_df, rc_df;                 // c/chat and chat/c as double-float
  float a_m, cv_m;                 // a_e = a_m 2^a_e2, 1/c_v = cv_m 2^cv_e, mantissas in [1, 2)
  int a_e2, cv_e;
};
__host__ __device__ __forceinline__ ExK make_exk(const qk_params &p) {
  ExK K;
  K.cr = p.c / p.chat;
  K.icc_d = 1.0 / (p.chat * p.c);
  K.rc_d = p.chat / p.c;
  K.inv_cv = p.eos == QK_EOS_ALPHA_T3 ? 0.0 : 1.0 / p.c_v;
  K.a_e = p.eos == QK_EOS_ALPHA_T3 ? 4.0 * p.a_r / p.alpha_eos : p.a_r;
  K.icc = (float)K.icc_d;
  K.rc = (float)K.rc_d;
  K.icc_lo = (float)(K.icc_d - (double)K.icc);
  K.crf = (float)K.cr;
  K.a_ef = (float)K.a_e;
  K.inv_cvf = (float)K.inv_cv;
  K.kchat = (float)(p.kappa_P * p.chat);
  K.kRf = (float)p.kappa_R;
  K.chatf = (float)p.chat;
  K.epsf = (float)p.eps_newton;
  K.cr_df.h = (float)K.cr;
  K.cr_df.l = (float)(K.cr - (double)K.cr_df.h);
  K.rc_df.h = (float)K.rc_d;
  K.rc_df.l = (float)(K.rc_d - (double)K.rc_df.h);
  int ex = 0;
  double m = frexp(K.a_e, &ex);  // m in [0.5, 1)
  K.a_m = (float)(2.0 * m);
  K.a_e2 = ex - 1;
  m = frexp(K.inv_cv, &ex);
  K.cv_m = (float)(2.0 * m);
  K.cv_e = ex - 1;
  return K;
}

// Per-thread status of the exchange cells it processed.
struct ExStat {
  int max = 0;
  unsigned flags = 0;
  unsigned long long bad = ~0ull;
};

// FP64 exchange of cell e: (er, fr) is the radiation state after the
// transport (read from R by the exchange kernel, or the stage-2 result in
// registers); reads the gas state from U, writes U and R.
template <typename T>
__device__ __forceinline__ void exchange_cell(const qk_params &p, const ExK &K, double dt, F5<T> U,
                                              F4<T> R, const T *src, long long e, double er,
                                              const double fr[3], ExStat &xs) {
  const double rho = load_d(U.f[0], e);
  double m[3] = {load_d(U.f[1], e), load_d(U.f[2], e), load_d(U.f[3], e)};
  const double E = load_d(U.f[4], e);
  const double Er0 = er;
  const double kP = p.kappa_mode == QK_KAPPA_RHO ? p.kappa_P * rho : p.kappa_P;
  const double kF = p.kappa_mode == QK_KAPPA_RHO ? p.kappa_R * rho : p.kappa_R;
  const double m2 = (m[0] * m[0] + m[1] * m[1]) + m[2] * m[2];
  // one reciprocal serves 1/rho and the flux damping 1/(1 + rho kF chat dt)
  const double Dm = 1.0 + rho * kF * p.chat * dt;
  const double inv_rho_Dm = frcp(rho * Dm);
  const double inv_rho = Dm * inv_rho_Dm;
  const double damp = rho * inv_rho_Dm;
  const double Ekin0 = 0.5 * m2 * inv_rho;
  const double Eg0 = E - Ekin0;
  // radiation source S = dt (chat/c) j, carried in the residual's E_r0
  const double Er0S = src ? Er0 + dt * K.rc_d * load_d(src, e) : Er0;
  // tolerance against E_tot = E_g0 + (c/chat)(E_r0 + S)
  const double thr_g = p.eps_newton * (Eg0 + K.cr * Er0S);
  const double thr_r = thr_g * K.rc_d;
  const double k = dt * rho * kP * p.chat;
  double A = k * K.a_e;
  if (p.eos != QK_EOS_ALPHA_T3) {
    const double i2 = (inv_rho * K.inv_cv) * (inv_rho * K.inv_cv);
    A *= i2 * i2;
  }
  // Start the FP64 iteration from an FP32 Newton solve to 1e-6 (the same
  // equations on FP32 pipes, inputs narrowed on the integer pipe): the FP64
  // iteration then needs about two steps, one correction and one confirming
  // the tolerance, instead of ~4 from the cell state.  It converges to the
  // same root (the last correction is applied, so the result is accurate far
  // below the tolerance whichever start is taken); a failed FP32 solve leaves
  // the start at the cell state.
  // Where the FP32 solve succeeded and its coefficients and the thresholds
  // are normal floats, the FP64 iteration is newton_refine: FP64 residuals
  // and convergence test (the same equations and tolerance), the 2x2
  // correction from the FP32 Jacobian (a Jacobian accurate to ~1e-7 still
  // gains ~7 digits per step, so the two steps from the warm start remain);
  // otherwise, or if that does not converge, the full FP64 Newton iteration.
  const bool alpha_eos = p.eos == QK_EOS_ALPHA_T3;
  double Eg = Eg0, Er = Er0;
  int it = -1;
  {
    const float Ef0 = d2f_trunc(Eg0), Rf0 = d2f_trunc(Er0S);
    const float Af = d2f_trunc(A), kf = d2f_trunc(k), tf = d2f_trunc(thr_g);
    float Egf = Ef0, Erf = Rf0;
    const int itf = newton_exchange<float>(alpha_eos, Af, kf, K.crf, Ef0, Rf0, 1e4f * tf,
                                           1e4f * tf * K.rc, 12, Egf, Erf);
    const bool warm = itf > 0 && pos_finite(Egf) && pos_finite(Erf);
    if (warm) {
      Eg = f2d(Egf);
      Er = f2d(Erf);
    }
    const float trf = d2f_trunc(thr_r);
    if (warm && pos_normal(Af) && pos_normal(kf) && pos_normal(tf) && pos_normal(trf))
      it = newton_refine(alpha_eos, p.max_iter, A, k, K.cr, Eg0, Er0S, Af, kf, K.crf, tf, trf,
                         Eg, Er);
  }
  if (it < 0) {
    Eg = Eg0;
    Er = Er0;
    it = newton_exchange<double>(alpha_eos, A, k, K.cr, Eg0, Er0S, thr_g, thr_r, p.max_iter, Eg,
                                 Er);
  }
  if (it < 0) {
    xs.flags |= 1u << QK_ENOCONV;
    xs.bad = min(xs.bad, (unsigned long long)e);
  } else {
    xs.max = max(xs.max, it);
  }
  // flux source (backward Euler) and the equal and opposite momentum change
  double mn[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const double F0 = fr[a];
    const double Fn = F0 * damp;
    mn[a] = m[a] - (Fn - F0) * K.icc_d;
    R.f[1 + a][e] = (T)Fn;
    U.f[1 + a][e] = (T)mn[a];
  }
  // work of the radiation force through the kinetic-energy change
  const double Ekin1 = 0.5 * ((mn[0] * mn[0] + mn[1] * mn[1]) + mn[2] * mn[2]) * inv_rho;
  const double dEkin = Ekin1 - Ekin0;
  U.f[4][e] = (T)(Eg + (Ekin0 + dEkin));
  const double Er_new = Er - K.rc_d * dEkin;
  R.f[0][e] = (T)Er_new;
  if (!pos_finite(Eg) || !pos_finite(Er_new)) {
    xs.flags |= 1u << QK_ENEGATIVE;
    xs.bad = min(xs.bad, (unsigned long long)e);
  }
}

// FP32-mixed exchange of cell e (see exchange_kernel_mixed): (er, fr) the
// radiation state after the transport, (er_lo, fr_lo) its low parts (CP);
// dt the substep and dtf its FP32 rounding (formed once by the caller);
// u_pre: the gas state of the cell already staged by the caller (field q at
// u_pre[q u_stride]), else it is read from U.
// FP32 state; the internal energy recovered with the error-free FP32
// transforms of con2prim; the Newton solve on the FP32 coefficients A, k with
// ~48-bit residuals: an FP32 warm start, then newton_refine_df in
// double-float where its rounding (~2^-43 (1 + k c/chat) E_tot) stays below
// the tolerance eps E_tot, else newton_refine in FP64, both on the energies
// scaled by a power of two to O(1); the flux source and
// the momentum and kinetic-energy work in FP32, the new total energy and
// radiation energy formed in double-float before the final rounding.
// CP: compensated state (every conserved field hi + lo; UL, RL the lo
// arrays): E, E_r, m and F are read as hi + lo, the new E and E_r are formed
// from the invariant E + (c/chat) E_r (the kinetic-energy change taken from
// the double-float difference of the same two values) and stored hi + lo,
// and the momentum exchange m + F/(c chat) = const is carried in double-float
// with a double-float 1/(c chat), so that both invariants hold to ~2^-47.
__device__ __forceinline__ DF df_of_double(double x) {
  const float h = (float)x;
  return DF{h, (float)(x - (double)h)};
}

template <int CP>
__device__ __forceinline__ void exchange_cell_mixed(const qk_params &p, const ExK &K, double dt,
                                                    float dtf, F5<float> U, F4<float> R,
                                                    F5<float> UL, F4<float> RL, const float *src,
                                                    long long e, float er, float er_lo,
                                                    const float fr[3], const float fr_lo[3],
                                                    ExStat &xs, const float *u_pre = nullptr,
                                                    int u_stride = 0) {
  float u[5];
#pragma unroll
  for (int q = 0; q < 5; ++q) u[q] = u_pre ? u_pre[q * u_stride] : U.f[q][e];
  const float rho = u[0];
  float rinv = qrcp(rho);
  rinv = rinv * fmaf(-rho, rinv, 2.0f);  // one Newton step: ~1 ulp
  float eg_hi, eg_lo;
  internal_energy_f32(u, rho, rinv, eg_hi, eg_lo);  // ~48-bit E_g, no EOS round trip
  DF Eg0 = df_of(eg_hi, eg_lo);
  DF Er0{er, 0.0f};
  float E_lo = 0.0f;
  if constexpr (CP) {
    E_lo = lo_get<CP>(UL.f[4], e, u[4]);
    Eg0 = df_add_f(Eg0, E_lo);
    Er0 = df_of(er, er_lo);
  }
  // The solve runs on the energies divided by 2^eE (exact), eE the binary
  // exponent of E_tot = E_g0 + (c/chat)(E_r0 + S), so that its FP32 and
  // double-float numbers are O(1) in any units (in cgs E_g^4 would overflow
  // FP32): with E = E' 2^eE the equations keep their form with k unchanged and
  // A' = A 2^(3 eE) (A for the alpha T^3 heat capacity, where R is linear in
  // E_g).  Coefficients in FP32: k = dt rho kappa_P chat and
  // A' = k a_r (rho c_v)^-4 2^(3 eE) as a product of mantissas and a sum of
  // exponents (the factors alone may leave the FP32 range); the thresholds
  // eps E_tot', eps E_tot' chat/c.  (Scaling every cell, rather than only
  // those outside the FP32 range, measured faster: no divergent branch.)
  const bool alpha_eos = p.eos == QK_EOS_ALPHA_T3;
  const float kf = dtf * K.kchat * (p.kappa_mode == QK_KAPPA_RHO ? rho * rho : rho);
  // radiation source S = dt (chat/c) j, carried in the residual's E_r0
  const float S_u = src ? (dtf * K.rc) * src[e] : 0.0f;
  const float Etot_u = Eg0.h + K.crf * (Er0.h + S_u);
  const int eE = pos_normal(Etot_u) ? min(max(fexpo(Etot_u), -100), 100) : 0;
  const float sc = pow2f(-eE), isc = pow2f(eE);
  float Af;
  if (alpha_eos) {
    Af = kf * K.a_ef;
  } else {
    const float mq = fmant(rinv) * K.cv_m, mq2 = mq * mq;  // (rho c_v)^-1 = mq 2^eq
    const int eq = fexpo(rinv) + K.cv_e;
    Af = fscale(kf * K.a_m * (mq2 * mq2), K.a_e2 + 4 * eq + 3 * eE);
  }
  const DF Eg0s{Eg0.h * sc, Eg0.l * sc};
  const DF Er0s{Er0.h * sc, Er0.l * sc};
  const float Etotf = Etot_u * sc;
  const float thr_g = K.epsf * Etotf, thr_r = thr_g * K.rc;
  const DF Er0S = src ? df_add_f(Er0s, S_u * sc) : Er0s;
  // FP32 warm start to 1e-6
  float Egf = Eg0s.h, Erf = Er0S.h;
  const int itf = newton_exchange<float>(alpha_eos, Af, kf, K.crf, Eg0s.h, Erf, 1e-6f * Etotf,
                                         1e-6f * Etotf * K.rc, 12, Egf, Erf);
  DF Eg = Eg0s, Er = Er0S;
  if (itf > 0 && pos_finite(Egf) && pos_finite(Erf)) {
    Eg = DF{Egf, 0.0f};
    Er = DF{Erf, 0.0f};
  }
  int it;
  if ((1.0f + kf * K.crf) * 0x1p-43f < K.epsf) {  // false for a NaN k
    it = newton_refine_df(alpha_eos, p.max_iter, Af, kf, K.cr_df, K.crf, Eg0s, Er0S, thr_g, thr_r,
                          Eg, Er);
  } else {
    double Egd = f2d(Eg.h), Erd = f2d(Er.h);
    it = newton_refine(alpha_eos, p.max_iter, f2d(Af), f2d(kf), K.cr, f2d(Eg0s.h) + f2d(Eg0s.l),
                       f2d(Er0S.h) + f2d(Er0S.l), Af, kf, K.crf, thr_g, thr_r, Egd, Erd);
    Eg = df_of_double(Egd);
    Er = df_of_double(Erd);
  }
  Eg = DF{Eg.h * isc, Eg.l * isc};
  Er = DF{Er.h * isc, Er.l * isc};
  if (it < 0) {
    xs.flags |= 1u << QK_ENOCONV;
    xs.bad = min(xs.bad, (unsigned long long)e);
  } else {
    xs.max = max(xs.max, it);
  }
  const float kF = p.kappa_mode == QK_KAPPA_RHO ? K.kRf * rho : K.kRf;
  const float damp = qrcp(1.0f + rho * kF * (K.chatf * dtf));
  float mn[3];
  float ke0 = 0.0f, ke1 = 0.0f;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const float F0 = fr[a];
    if constexpr (CP) {
      // dF = F0 (damp - 1); F += dF and m -= dF/(c chat), both in double-float
      float Fl = fr_lo[a];
      const float dF = (F0 + Fl) * (damp - 1.0f);
      float Fh = F0;
      df_add(Fh, Fl, dF);
      df_norm(Fh, Fl);
      R.f[1 + a][e] = Fh;
      lo_put<CP>(RL.f[1 + a], e, Fh, Fl);
      const float p1 = __fmul_rn(dF, K.icc);
      const float e1 = fmaf(dF, K.icc, -p1) + dF * K.icc_lo;
      float mh = u[1 + a], ml = lo_get<CP>(UL.f[1 + a], e, u[1 + a]);
      df_add(mh, ml, -p1);
      ml = __fsub_rn(ml, e1);
      df_norm(mh, ml);
      U.f[1 + a][e] = mh;
      lo_put<CP>(UL.f[1 + a], e, mh, ml);
      mn[a] = mh;
    } else {
      const float Fn = F0 * damp;
      mn[a] = u[1 + a] - (Fn - F0) * K.icc;
      R.f[1 + a][e] = Fn;
      U.f[1 + a][e] = mn[a];
    }
    ke0 = fmaf(u[1 + a], u[1 + a], ke0);
    ke1 = fmaf(mn[a], mn[a], ke1);
  }
  const float Ekin1 = 0.5f * ke1 * rinv;
  const DF Enew = df_add_f(Eg, Ekin1);
  DF Er_new;
  if constexpr (CP) {
    // E_new = E_g + E_kin,1; E_r,new = E_r - (chat/c)(E_kin,1 - E_kin,0) with
    // E_kin,0 = E - E_g0 (the same double-float values)
    const DF Ekin0 = df_sub(df_of(u[4], E_lo), Eg0);
    Er_new = df_sub(Er, df_mul(K.rc_df, df_add_f(df_neg(Ekin0), Ekin1)));
    U.f[4][e] = Enew.h;
    lo_put<CP>(UL.f[4], e, Enew.h, Enew.l);
    R.f[0][e] = Er_new.h;
    lo_put<CP>(RL.f[0], e, Er_new.h, Er_new.l);
  } else {
    const float dEkin = 0.5f * (ke1 - ke0) * rinv;
    Er_new = df_add_f(Er, -K.rc * dEkin);
    U.f[4][e] = Enew.h;
    R.f[0][e] = Er_new.h;
  }
  if (!pos_finite(Eg.h) || !pos_finite(Er_new.h)) {
    xs.flags |= 1u << QK_ENEGATIVE;
    xs.bad = min(xs.bad, (unsigned long long)e);
  }
}

}  // namespace qk
