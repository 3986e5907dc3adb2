// qk_cell.cu -- per-cell kernels of the update (arXiv:2110.01792) for sm_103a:
// the implicit matter-radiation exchange (Sec. 2.2.3), the CFL reduction and
// timestep (Sec. 2.2.1, Sec. 2.2.4), the batched ghost fill, and the
// compensated conservation sums.
#include <algorithm>

#include "qk_device.cuh"

namespace qk {

// ----------------------------------------------------------- cell lookup ---
// Map a flat interior-cell index to (patch, element) with a binary search over
// the per-patch prefix of interior cells.
__device__ __forceinline__ long long cell_to_elem(const Geometry &g, long long c) {
  int lo = 0, hi = g.nbox - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (g.box_cell0[mid] <= c) lo = mid; else hi = mid - 1;
  }
  const DevBox &b = g.boxes[lo];
  long long r = c - g.box_cell0[lo];
  int nx = b.n[0], ny = b.n[1];
  int i = (int)(r % nx);
  long long q = r / nx;
  int j = (int)(q % ny);
  int k = (int)(q / ny);
  return cell_elem(b, g.ng, i, j, k);
}

// -------------------------------------------------------------- exchange ---
template <typename T>
__device__ __forceinline__ double load_d(const T *p, long long e) { return (double)p[e]; }

// Newton-Raphson on (E_g, E_r) for one cell (Sec. 2.2.3, eqs. delta_er and
// delta_eg).  R = dt rho kappa_P chat (a_r T^4 - E_r) (the '4 pi B' of the
// paper read as chat a_r T^4), F_G = (E_g - E_g0) + (c/chat) R,
// F_R = (E_r - E_r0) - R; with a radiation source S the callers pass
// E_r0 + S for E_r0 (F_R = (E_r - E_r0) - (R + S); the Jacobian does not
// change); convergence |F_G/E_tot| < eps and
// |(c/chat) F_R / E_tot| < eps, E_tot = E_g0 + (c/chat) E_r0; the update of
// the iterate that passes is applied, then the loop stops.  The 2x2
// elimination of eqs. delta_er / delta_eg is evaluated with one division:
// with G = dF_G/dE_g, eta = (dR/dE_g)/G,
//   dE_r = -(F_R G + R' F_G) / D1,  D1 = (dF_R/dE_r) G + R' (dF_G/dE_r),
//   dE_g = -(F_G + dE_r dF_G/dE_r) / G,
// and 1/D1, 1/G taken from the single reciprocal of D1 G.  Starts from
// (Eg, Er) (the cell state, or a warm start); returns the iteration count,
// or -1 after max_iter iterations.
template <typename R_>
__device__ __forceinline__ int newton_exchange(const qk_params &p, R_ Eg0, R_ Er0, R_ k, R_ cr,
                                               R_ inv_Etot, R_ inv_rcv, R_ eps, int max_iter,
                                               R_ &Eg, R_ &Er) {
  const R_ a_r = (R_)p.a_r;
  const R_ dFG_dEr = -cr * k;     // -c dt rho kappa_P
  const R_ dFR_dEr = R_(1) + k;
  const bool alpha_eos = p.eos == QK_EOS_ALPHA_T3;
  const R_ dT4_alpha = alpha_eos ? (R_)(4.0 / p.alpha_eos) : R_(0);
  bool conv = false;
  int it = 0;
  for (it = 0; it < max_iter; ++it) {
    R_ T4, dT4;
    if (alpha_eos) {
      T4 = dT4_alpha * Eg;
      dT4 = dT4_alpha;
    } else {
      const R_ Tg = Eg * inv_rcv;
      const R_ T2 = Tg * Tg;
      T4 = T2 * T2;
      dT4 = R_(4) * T2 * Tg * inv_rcv;
    }
    const R_ Rr = k * (a_r * T4 - Er);
    const R_ FG = (Eg - Eg0) + cr * Rr;
    const R_ FR = (Er - Er0) - Rr;
    conv = fabs(FG * inv_Etot) < eps && fabs(cr * FR * inv_Etot) < eps;
    const R_ dRdEg = k * a_r * dT4;
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

// Mixed-precision Newton for one cell: the residuals F_G, F_R and the
// convergence test of Sec. 2.2.3 are evaluated in FP64 at the FP64 iterate,
// the 2x2 correction (the same elimination as newton_exchange) is solved in
// FP32 (iterative refinement: each iteration gains ~7 digits, so two
// iterations from an FP32 warm start reach the 1e-10 tolerance).  Returns
// the iteration count or -1.
__device__ __forceinline__ int newton_refine(const qk_params &p, double Eg0, double Er0,
                                             double k, double cr, double inv_Etot,
                                             double inv_rcv, double &Eg, double &Er) {
  const double a_r = p.a_r;
  const float kf = (float)k, crf = (float)cr, arf = (float)p.a_r;
  const float dFG_dEr = -crf * kf, dFR_dEr = 1.0f + kf;
  const bool alpha_eos = p.eos == QK_EOS_ALPHA_T3;
  const double dT4_alpha = alpha_eos ? 4.0 / p.alpha_eos : 0.0;
  bool conv = false;
  int it = 0;
  for (it = 0; it < p.max_iter; ++it) {
    double T4;
    float dT4;
    if (alpha_eos) {
      T4 = dT4_alpha * Eg;
      dT4 = (float)dT4_alpha;
    } else {
      const double Tg = Eg * inv_rcv;
      const double T2 = Tg * Tg;
      T4 = T2 * T2;
      const float Tf = (float)Tg;
      dT4 = 4.0f * Tf * Tf * Tf * (float)inv_rcv;
    }
    const double Rr = k * (a_r * T4 - Er);
    const double FG = (Eg - Eg0) + cr * Rr;
    const double FR = (Er - Er0) - Rr;
    conv = fabs(FG * inv_Etot) < p.eps_newton && fabs(cr * FR * inv_Etot) < p.eps_newton;
    const float fg = (float)FG, fr = (float)FR;
    const float dRdEg = kf * arf * dT4;
    const float G = 1.0f + crf * dRdEg;
    const float D1 = dFR_dEr * G + dRdEg * dFG_dEr;
    const float inv = qrcp(D1 * G);
    const float dEr = -(fr * G + dRdEg * fg) * (G * inv);
    const float dEg = -(fg + dEr * dFG_dEr) * (D1 * inv);
    Er += (double)dEr;
    Eg += (double)dEg;
    if (conv) break;
  }
  return conv ? it + 1 : -1;
}

// FP32-mixed exchange: FP32 state; the internal energy recovered with the
// error-free FP32 transforms of con2prim; the Newton solve with FP64 residuals
// and convergence test (FP32 warm start, then newton_refine); the flux
// source, momentum and kinetic-energy work in FP32, the new total energy
// accumulated in FP64 before the final rounding.
// CP: compensated state (every conserved field hi + lo; UL, RL the lo
// arrays): E, E_r, m and F are read as hi + lo, the new E and E_r are formed
// in FP64 from the invariant E + (c/chat) E_r (the kinetic-energy change
// taken from the FP64 difference of the same two values), and the momentum
// exchange m + F/(c chat) = const is carried in double-float with a
// double-float 1/(c chat), so that both invariants hold to ~2^-48.
template <bool CP>
__global__ void __launch_bounds__(256) exchange_kernel_mixed(Geometry g, qk_params p,
                                                              F5<float> U, F4<float> R,
                                                              const float *src, DtSrc dts,
                                                              Status *st, F5<float> UL,
                                                              F4<float> RL) {
  if (skip_substep(dts)) return;
  const double dt = dt_of(dts);
  const double cr = p.c / p.chat;
  const float icc = (float)(1.0 / (p.chat * p.c)), rc = (float)(p.chat / p.c);
  const float icc_lo = (float)(1.0 / (p.chat * p.c) - (double)icc);
  const double inv_cv = p.eos == QK_EOS_ALPHA_T3 ? 0.0 : 1.0 / p.c_v;
  int my_max = 0;
  unsigned my_flags = 0;
  unsigned long long my_bad = ~0ull;
  for (long long cidx = (long long)blockIdx.x * blockDim.x + threadIdx.x; cidx < g.ncells;
       cidx += (long long)gridDim.x * blockDim.x) {
    const long long e = cell_to_elem(g, cidx);
    float u[5];
#pragma unroll
    for (int q = 0; q < 5; ++q) u[q] = U.f[q][e];
    const float rho = u[0];
    float rinv = qrcp(rho);
    rinv = rinv * fmaf(-rho, rinv, 2.0f);  // one Newton step: ~1 ulp
    float eg_hi, eg_lo;
    internal_energy_f32(u, rho, rinv, eg_hi, eg_lo);  // ~48-bit E_g, no EOS round trip
    const float Er0f = R.f[0][e];
    const double rho_d = (double)rho;
    double Eg0 = (double)eg_hi + (double)eg_lo;
    double Er0 = (double)Er0f;
    float E_lo = 0.0f;
    if constexpr (CP) {
      E_lo = UL.f[4][e];
      Eg0 += (double)E_lo;
      Er0 += (double)RL.f[0][e];
    }
    const double kP = p.kappa_mode == QK_KAPPA_RHO ? p.kappa_P * rho_d : p.kappa_P;
    const double k = dt * rho_d * kP * p.chat;
    const double inv_rcv = (double)(rinv * (float)inv_cv);
    const double inv_Etot = (double)qrcp((float)(Eg0 + cr * Er0));
    // radiation source S = dt (chat/c) j, carried in the residual's E_r0
    const double Er0S = src ? Er0 + dt * (p.chat / p.c) * (double)src[e] : Er0;
    // FP32 warm start
    float Egf = (float)Eg0, Erf = (float)Er0S;
    const int itf = newton_exchange<float>(p, (float)Eg0, (float)Er0S, (float)k, (float)cr,
                                           (float)inv_Etot, (float)inv_rcv, 1e-6f, 12, Egf, Erf);
    double Eg = Eg0, Er = Er0;
    if (itf > 0 && Egf > 0.0f && Erf > 0.0f && isfinite(Egf) && isfinite(Erf)) {
      Eg = Egf;
      Er = Erf;
    }
    const int it = newton_refine(p, Eg0, Er0S, k, cr, inv_Etot, inv_rcv, Eg, Er);
    if (it < 0) {
      my_flags |= 1u << QK_ENOCONV;
      my_bad = min(my_bad, (unsigned long long)e);
    } else {
      my_max = max(my_max, it);
    }
    const float kF = p.kappa_mode == QK_KAPPA_RHO ? (float)p.kappa_R * rho : (float)p.kappa_R;
    const float damp = qrcp(1.0f + rho * kF * (float)(p.chat * dt));
    float mn[3];
    float ke0 = 0.0f, ke1 = 0.0f;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const float F0 = R.f[1 + a][e];
      if constexpr (CP) {
        // dF = F0 (damp - 1); F += dF and m -= dF/(c chat), both in double-float
        float Fl = RL.f[1 + a][e];
        const float dF = (F0 + Fl) * (damp - 1.0f);
        float Fh = F0;
        df_add(Fh, Fl, dF);
        df_norm(Fh, Fl);
        R.f[1 + a][e] = Fh;
        RL.f[1 + a][e] = Fl;
        const float p1 = __fmul_rn(dF, icc);
        const float e1 = fmaf(dF, icc, -p1) + dF * icc_lo;
        float mh = u[1 + a], ml = UL.f[1 + a][e];
        df_add(mh, ml, -p1);
        ml = __fsub_rn(ml, e1);
        df_norm(mh, ml);
        U.f[1 + a][e] = mh;
        UL.f[1 + a][e] = ml;
        mn[a] = mh;
      } else {
        const float Fn = F0 * damp;
        mn[a] = u[1 + a] - (Fn - F0) * icc;
        R.f[1 + a][e] = Fn;
        U.f[1 + a][e] = mn[a];
      }
      ke0 = fmaf(u[1 + a], u[1 + a], ke0);
      ke1 = fmaf(mn[a], mn[a], ke1);
    }
    const float Ekin1 = 0.5f * ke1 * rinv;
    double Er_new;
    if constexpr (CP) {
      // E_new = E_g + E_kin,1; E_r,new = E_r - (chat/c)(E_kin,1 - E_kin,0) with
      // E_kin,0 = E - E_g0 (the same FP64 values), split into hi + lo
      const double Ekin0 = ((double)u[4] + (double)E_lo) - Eg0;
      const double Enew = Eg + (double)Ekin1;
      Er_new = Er - (p.chat / p.c) * ((double)Ekin1 - Ekin0);
      const float Eh = (float)Enew, Rh = (float)Er_new;
      U.f[4][e] = Eh;
      UL.f[4][e] = (float)(Enew - (double)Eh);
      R.f[0][e] = Rh;
      RL.f[0][e] = (float)(Er_new - (double)Rh);
    } else {
      const float dEkin = 0.5f * (ke1 - ke0) * rinv;
      U.f[4][e] = (float)(Eg + (double)Ekin1);
      Er_new = Er - (double)(rc * dEkin);
      R.f[0][e] = (float)Er_new;
    }
    if (!(Eg > 0.0) || !(Er_new > 0.0)) {
      my_flags |= 1u << QK_ENEGATIVE;
      my_bad = min(my_bad, (unsigned long long)e);
    }
  }
  exchange_status(st, my_max, my_flags, my_bad);
}

template <typename T>
__global__ void __launch_bounds__(256) exchange_kernel(Geometry g, qk_params p, F5<T> U, F4<T> R,
                                                        const T *src, DtSrc dts, Status *st) {
  if (skip_substep(dts)) return;
  const double dt = dt_of(dts);
  const double chat = p.chat, c = p.c;
  const double cr = c / chat, icc = 1.0 / (chat * c), rc = chat / c;
  const double inv_cv = p.eos == QK_EOS_ALPHA_T3 ? 0.0 : 1.0 / p.c_v;
  int my_max = 0;
  unsigned my_flags = 0;
  unsigned long long my_bad = ~0ull;
  for (long long cidx = (long long)blockIdx.x * blockDim.x + threadIdx.x; cidx < g.ncells;
       cidx += (long long)gridDim.x * blockDim.x) {
    const long long e = cell_to_elem(g, cidx);
    const double rho = load_d(U.f[0], e);
    double m[3] = {load_d(U.f[1], e), load_d(U.f[2], e), load_d(U.f[3], e)};
    const double E = load_d(U.f[4], e);
    const double Er0 = load_d(R.f[0], e);
    const double kP = p.kappa_mode == QK_KAPPA_RHO ? p.kappa_P * rho : p.kappa_P;
    const double kF = p.kappa_mode == QK_KAPPA_RHO ? p.kappa_R * rho : p.kappa_R;
    const double m2 = (m[0] * m[0] + m[1] * m[1]) + m[2] * m[2];
    // one reciprocal serves 1/rho and the flux damping 1/(1 + rho kF chat dt)
    const double Dm = 1.0 + rho * kF * chat * dt;
    const double inv_rho_Dm = frcp(rho * Dm);
    const double inv_rho = Dm * inv_rho_Dm;
    const double damp = rho * inv_rho_Dm;
    const double Ekin0 = 0.5 * m2 * inv_rho;
    const double Eg0 = E - Ekin0;
    const double inv_Etot = frcp(Eg0 + cr * Er0);
    const double k = dt * rho * kP * chat;
    const double inv_rcv = inv_rho * inv_cv;
    // radiation source S = dt (chat/c) j, carried in the residual's E_r0
    const double Er0S = src ? Er0 + dt * rc * load_d(src, e) : Er0;
    double Eg = Eg0, Er = Er0;
    int it;
    it = newton_exchange<double>(p, Eg0, Er0S, k, cr, inv_Etot, inv_rcv, p.eps_newton,
                                 p.max_iter, Eg, Er);
    if (it < 0) {
      my_flags |= 1u << QK_ENOCONV;
      my_bad = min(my_bad, (unsigned long long)e);
    } else {
      my_max = max(my_max, it);
    }
    // flux source (backward Euler) and the equal and opposite momentum change
    double mn[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const double F0 = load_d(R.f[1 + a], e);
      const double Fn = F0 * damp;
      mn[a] = m[a] - (Fn - F0) * icc;
      R.f[1 + a][e] = (T)Fn;
      U.f[1 + a][e] = (T)mn[a];
    }
    // work of the radiation force through the kinetic-energy change
    const double Ekin1 = 0.5 * ((mn[0] * mn[0] + mn[1] * mn[1]) + mn[2] * mn[2]) * inv_rho;
    const double dEkin = Ekin1 - Ekin0;
    U.f[4][e] = (T)(Eg + (Ekin0 + dEkin));
    const double Er_new = Er - rc * dEkin;
    R.f[0][e] = (T)Er_new;
    if (!(Eg > 0.0) || !(Er_new > 0.0)) {
      my_flags |= 1u << QK_ENEGATIVE;
      my_bad = min(my_bad, (unsigned long long)e);
    }
  }
  exchange_status(st, my_max, my_flags, my_bad);
}

cudaError_t launch_exchange(int fp32, const Geometry &g, const qk_params &p, void *const *U,
                            void *const *R, const void *src, DtSrc dt, Status *st,
                            cudaStream_t s, void *const *Ulo, void *const *Rlo) {
  int nsm = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  long long want = (g.ncells + 255) / 256;
  int grid = (int)std::min<long long>(want, (long long)nsm * 8);
  if (grid < 1) return cudaSuccess;
  if (fp32) {
    F5<float> u, ul{}; F4<float> r, rl{};
    for (int q = 0; q < 5; ++q) u.f[q] = (float *)U[q];
    for (int q = 0; q < 4; ++q) r.f[q] = (float *)R[q];
    if (Ulo) {
      for (int q = 0; q < 5; ++q) ul.f[q] = (float *)Ulo[q];
      for (int q = 0; q < 4; ++q) rl.f[q] = (float *)Rlo[q];
      exchange_kernel_mixed<true><<<grid, 256, 0, s>>>(g, p, u, r, (const float *)src, dt, st,
                                                       ul, rl);
    } else {
      exchange_kernel_mixed<false><<<grid, 256, 0, s>>>(g, p, u, r, (const float *)src, dt, st,
                                                        ul, rl);
    }
  } else {
    F5<double> u; F4<double> r;
    for (int q = 0; q < 5; ++q) u.f[q] = (double *)U[q];
    for (int q = 0; q < 4; ++q) r.f[q] = (double *)R[q];
    exchange_kernel<double><<<grid, 256, 0, s>>>(g, p, u, r, (const double *)src, dt, st);
  }
  return cudaGetLastError();
}

// -------------------------------------------------- signal speed, dt -----
// max(|v| + c_s) over the interior cells (Sec. 2.2.1, eq. signal), with
// |v| = sqrt((vx^2 + vy^2) + vz^2) and c_s = sqrt(gamma P / rho); FP32 state
// uses the FP32 con2prim (error-free internal-energy recovery).
template <typename T>
__device__ __forceinline__ double cell_speed(const F5<T> &U, long long e, double gamma);
template <>
__device__ __forceinline__ double cell_speed<double>(const F5<double> &U, long long e,
                                                     double gamma) {
  const double rho = U.f[0][e];
  const double inv = 1.0 / rho;
  const double vx = U.f[1][e] * inv, vy = U.f[2][e] * inv, vz = U.f[3][e] * inv;
  const double v2 = (vx * vx + vy * vy) + vz * vz;
  const double P = (gamma - 1.0) * (U.f[4][e] - 0.5 * rho * v2);
  return sqrt(v2) + sqrt(gamma * P * inv);
}
template <>
__device__ __forceinline__ double cell_speed<float>(const F5<float> &U, long long e,
                                                    double gamma) {
  float u[5], w[5];
#pragma unroll
  for (int q = 0; q < 5; ++q) u[q] = U.f[q][e];
  con2prim<float>(u, gamma, w);
  const float v2 = (w[1] * w[1] + w[2] * w[2]) + w[3] * w[3];
  return (double)(qsqrt(v2) + qsqrt((float)gamma * w[4] * qrcp(w[0])));
}

template <typename T>
__global__ void __launch_bounds__(256) max_speed_kernel(Geometry g, double gamma, F5<T> U,
                                                        StepInfo *si) {
  double best = 0.0;
  for (long long cidx = (long long)blockIdx.x * blockDim.x + threadIdx.x; cidx < g.ncells;
       cidx += (long long)gridDim.x * blockDim.x) {
    best = fmax(best, cell_speed<T>(U, cell_to_elem(g, cidx), gamma));
  }
  for (int o = 16; o > 0; o >>= 1) best = fmax(best, __shfl_xor_sync(0xffffffffu, best, o));
  __shared__ double wbest[8];
  if ((threadIdx.x & 31) == 0) wbest[threadIdx.x >> 5] = best;
  __syncthreads();
  if (threadIdx.x == 0) {
    double b = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) b = fmax(b, wbest[w]);
    atomic_max_pos(&si->smax_bits, b);
  }
}

cudaError_t launch_max_speed(int fp32, const Geometry &g, const qk_params &p, void *const *U,
                             StepInfo *si, cudaStream_t s) {
  int nsm = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  long long want = (g.ncells + 255) / 256;
  int grid = (int)std::min<long long>(want, (long long)nsm * 8);
  if (grid < 1) grid = 1;
  if (fp32) {
    F5<float> u;
    for (int q = 0; q < 5; ++q) u.f[q] = (float *)U[q];
    max_speed_kernel<float><<<grid, 256, 0, s>>>(g, p.gamma, u, si);
  } else {
    F5<double> u;
    for (int q = 0; q < 5; ++q) u.f[q] = (double *)U[q];
    max_speed_kernel<double><<<grid, 256, 0, s>>>(g, p.gamma, u, si);
  }
  return cudaGetLastError();
}

// dt = CFL dx_min / smax; with radiation at most N_sub,max substeps of
// CFL dx_min / chat (Sec. 2.2.4): if dt > N_sub,max dt_r then N_sub = N_sub,max
// and dt = N_sub,max dt_r, else N_sub = max(1, ceil(dt / dt_r)); dt_rad =
// dt / N_sub.  Resets the running maximum for the next step.
__global__ void timestep_kernel(qk_params p, StepInfo *si) {
  const double smax = __longlong_as_double((long long)si->smax_bits);
  const double dxm = fmin(p.dx[0], fmin(p.dx[1], p.dx[2]));
  double dt = __ddiv_rn(__dmul_rn(p.cfl, dxm), smax);
  double nsub = 0.0, dtrad = 0.0;
  if (!p.hydro_only) {
    const double dtr = __ddiv_rn(__dmul_rn(p.cfl, dxm), p.chat);
    const double cap = __dmul_rn((double)p.nsub_max, dtr);
    if (dt > cap) {
      nsub = (double)p.nsub_max;
      dt = cap;
    } else {
      nsub = fmax(1.0, ceil(__ddiv_rn(dt, dtr)));
    }
    dtrad = __ddiv_rn(dt, nsub);
  }
  si->dt = dt;
  si->nsub = nsub;
  si->dtrad = dtrad;
  si->smax = smax;
  si->smax_bits = 0ull;
  si->nsub_total += nsub;
  si->nsteps += 1.0;
}

cudaError_t launch_timestep(const qk_params &p, StepInfo *si, cudaStream_t s) {
  timestep_kernel<<<1, 1, 0, s>>>(p, si);
  return cudaGetLastError();
}

// ------------------------------------------------------------ ghost fill ---
// Every ghost cell of every patch receives the value of the cell
// its copy descriptor names (periodic image, mirror image or nearest interior
// cell), with the vector components along reflecting axes negated.  One CTA
// per chunk of at most CHUNK_CELLS destination cells of one descriptor; the
// same source addresses serve all fields.  Fields are the state fields
// first .. first+nf-1 (their identity decides the sign flips).
template <typename T>
__device__ __forceinline__ T *field_ptr(const F5<T> &fa, const F4<T> &fb, int f) {
  return f < 5 ? fa.f[f] : fb.f[f - 5];
}

template <typename T>
__global__ void __launch_bounds__(256) ghost_fill_kernel(const Copy *copies, const Chunk *chunks,
                                                         F5<T> fa, F4<T> fb, int nf, int first,
                                                         DtSrc pred) {
  if (skip_substep(pred)) return;
  const Chunk ch = chunks[blockIdx.x];
  const Copy cp = copies[ch.copy];
  const int ncell = cp.ex * cp.ey * cp.ez;
  const int end = min(ncell, ch.start + CHUNK_CELLS);
  for (int l = ch.start + threadIdx.x; l < end; l += blockDim.x) {
    const int x = l % cp.ex;
    const int r = l / cp.ex;
    const int y = r % cp.ey;
    const int z = r / cp.ey;
    const long long d = cp.dst + ((long long)z * cp.dsy + y) * cp.dsx + x;
    const long long s = cp.src + z * cp.sz + y * cp.sy + x * cp.sx;
#pragma unroll
    for (int f = 0; f < 9; ++f) {
      if (f >= nf) break;
      T *fld = field_ptr(fa, fb, f);
      const int ax = field_axis(first + f);
      const T v = fld[s];
      fld[d] = (ax >= 0 && ((cp.flip >> ax) & 1)) ? -v : v;
    }
  }
}

cudaError_t launch_ghost_fill(int fp32, const Copy *copies, const Chunk *chunks, int nchunks,
                              void *const *fields, int nf, int first, DtSrc pred, cudaStream_t s) {
  if (nchunks < 1 || nf < 1) return cudaSuccess;
  if (fp32) {
    F5<float> a{}; F4<float> b{};
    for (int q = 0; q < nf && q < 5; ++q) a.f[q] = (float *)fields[q];
    for (int q = 5; q < nf; ++q) b.f[q - 5] = (float *)fields[q];
    ghost_fill_kernel<float><<<nchunks, 256, 0, s>>>(copies, chunks, a, b, nf, first, pred);
  } else {
    F5<double> a{}; F4<double> b{};
    for (int q = 0; q < nf && q < 5; ++q) a.f[q] = (double *)fields[q];
    for (int q = 5; q < nf; ++q) b.f[q - 5] = (double *)fields[q];
    ghost_fill_kernel<double><<<nchunks, 256, 0, s>>>(copies, chunks, a, b, nf, first, pred);
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------- halo pack ---
// Cross-rank part of the ghost fill, and the Dirichlet boundary store.  The
// packing side gathers, for each region, the source cells (the descriptor's
// strided source, sign flips applied) into a contiguous buffer (x fastest,
// regions in the agreed order, one block of `nbuf` cells per field); the
// unpacking side scatters the same buffer into the destination regions.  A
// descriptor's other side is its position in the buffer (`dst` when packing,
// `src` when unpacking).
template <typename T, bool PACK>
__global__ void __launch_bounds__(256) halo_kernel(const Copy *copies, const Chunk *chunks,
                                                   F5<T> fa, F4<T> fb, int nf, int first, T *buf,
                                                   long long nbuf, DtSrc pred) {
  if (skip_substep(pred)) return;
  const Chunk ch = chunks[blockIdx.x];
  const Copy cp = copies[ch.copy];
  const int ncell = cp.ex * cp.ey * cp.ez;
  const int end = min(ncell, ch.start + CHUNK_CELLS);
  for (int l = ch.start + threadIdx.x; l < end; l += blockDim.x) {
    const int x = l % cp.ex;
    const int r = l / cp.ex;
    const int y = r % cp.ey;
    const int z = r / cp.ey;
    long long e, q;  // field element, buffer position
    if (PACK) {
      e = cp.src + z * cp.sz + y * cp.sy + x * cp.sx;
      q = cp.dst + l;
    } else {
      e = cp.dst + ((long long)z * cp.dsy + y) * cp.dsx + x;
      q = cp.src + l;
    }
#pragma unroll
    for (int f = 0; f < 9; ++f) {
      if (f >= nf) break;
      T *fld = field_ptr(fa, fb, f);
      if (PACK) {
        const int ax = field_axis(first + f);
        const T v = fld[e];
        buf[f * nbuf + q] = (ax >= 0 && ((cp.flip >> ax) & 1)) ? -v : v;
      } else {
        fld[e] = buf[f * nbuf + q];
      }
    }
  }
}

cudaError_t launch_halo(int fp32, int pack, const Copy *copies, const Chunk *chunks, int nchunks,
                        void *const *fields, int nf, int first, void *buf, long long nbuf,
                        DtSrc pred, cudaStream_t s) {
  if (nchunks < 1 || nf < 1) return cudaSuccess;
  if (fp32) {
    F5<float> a{}; F4<float> b{};
    for (int q = 0; q < nf && q < 5; ++q) a.f[q] = (float *)fields[q];
    for (int q = 5; q < nf; ++q) b.f[q - 5] = (float *)fields[q];
    if (pack)
      halo_kernel<float, true><<<nchunks, 256, 0, s>>>(copies, chunks, a, b, nf, first, (float *)buf, nbuf, pred);
    else
      halo_kernel<float, false><<<nchunks, 256, 0, s>>>(copies, chunks, a, b, nf, first, (float *)buf, nbuf, pred);
  } else {
    F5<double> a{}; F4<double> b{};
    for (int q = 0; q < nf && q < 5; ++q) a.f[q] = (double *)fields[q];
    for (int q = 5; q < nf; ++q) b.f[q - 5] = (double *)fields[q];
    if (pack)
      halo_kernel<double, true><<<nchunks, 256, 0, s>>>(copies, chunks, a, b, nf, first, (double *)buf, nbuf, pred);
    else
      halo_kernel<double, false><<<nchunks, 256, 0, s>>>(copies, chunks, a, b, nf, first, (double *)buf, nbuf, pred);
  }
  return cudaGetLastError();
}

// ------------------------------------------------------ conservation sums ---
// Double-double accumulation (Knuth's TwoSum) with a fixed assignment of cells
// to threads and a fixed reduction tree: the result is bitwise reproducible.
struct DD { double hi, lo; };
__device__ __forceinline__ DD dd_add(DD a, double b) {
  double s = a.hi + b;
  double bb = s - a.hi;
  double err = (a.hi - (s - bb)) + (b - bb);
  return DD{s, a.lo + err};
}
__device__ __forceinline__ DD dd_add(DD a, DD b) {
  DD s = dd_add(a, b.hi);
  s.lo += b.lo;
  double hi = s.hi + s.lo;
  double lo = s.lo - (hi - s.hi);
  return DD{hi, lo};
}

constexpr int SUM_NT = 256;

template <typename T>
__global__ void __launch_bounds__(SUM_NT) sums_kernel(Geometry g, double cr, double icc, F5<T> U,
                                                      F4<T> R, int has_rad, double *partials,
                                                      F5<T> UL, F4<T> RL) {
  DD acc[QK_NSUMS];
#pragma unroll
  for (int q = 0; q < QK_NSUMS; ++q) acc[q] = DD{0.0, 0.0};
  for (long long cidx = (long long)blockIdx.x * SUM_NT + threadIdx.x; cidx < g.ncells;
       cidx += (long long)gridDim.x * SUM_NT) {
    const long long e = cell_to_elem(g, cidx);
    double x[QK_NSUMS];
#pragma unroll
    for (int q = 0; q < 5; ++q) x[q] = (double)U.f[q][e];
#pragma unroll
    for (int q = 0; q < 4; ++q) x[5 + q] = has_rad ? (double)R.f[q][e] : 0.0;
    // compensated FP32 state: the value is hi + lo (exact in double)
    if (UL.f[0]) {
#pragma unroll
      for (int q = 0; q < 5; ++q) x[q] += (double)UL.f[q][e];
      if (has_rad) {
#pragma unroll
        for (int q = 0; q < 4; ++q) x[5 + q] += (double)RL.f[q][e];
      }
    }
    x[9] = x[4] + cr * x[5];
#pragma unroll
    for (int a = 0; a < 3; ++a) x[10 + a] = x[1 + a] + x[6 + a] * icc;
#pragma unroll
    for (int q = 0; q < QK_NSUMS; ++q) acc[q] = dd_add(acc[q], x[q]);
  }
  __shared__ DD sh[SUM_NT];
  for (int q = 0; q < QK_NSUMS; ++q) {
    sh[threadIdx.x] = acc[q];
    __syncthreads();
    for (int w = SUM_NT / 2; w > 0; w >>= 1) {
      if (threadIdx.x < w) sh[threadIdx.x] = dd_add(sh[threadIdx.x], sh[threadIdx.x + w]);
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      partials[(blockIdx.x * QK_NSUMS + q) * 2 + 0] = sh[0].hi;
      partials[(blockIdx.x * QK_NSUMS + q) * 2 + 1] = sh[0].lo;
    }
    __syncthreads();
  }
}

__global__ void sums_final_kernel(const double *partials, int nblocks, double vol, double *out) {
  const int q = threadIdx.x;
  if (q >= QK_NSUMS) return;
  DD a{0.0, 0.0};
  for (int b = 0; b < nblocks; ++b)
    a = dd_add(a, DD{partials[(b * QK_NSUMS + q) * 2], partials[(b * QK_NSUMS + q) * 2 + 1]});
  out[q] = (a.hi + a.lo) * vol;
}

cudaError_t launch_sums(int fp32, const Geometry &g, const qk_params &p, void *const *U,
                        void *const *R, double *partials, int nblocks, double *out,
                        cudaStream_t s, void *const *Ulo, void *const *Rlo) {
  const double cr = p.c / p.chat, icc = 1.0 / (p.c * p.chat);
  const double vol = p.dx[0] * p.dx[1] * p.dx[2];
  const int has_rad = R != nullptr;
  if (fp32) {
    F5<float> u, ul{}; F4<float> r{}, rl{};
    for (int q = 0; q < 5; ++q) u.f[q] = (float *)U[q];
    if (has_rad) for (int q = 0; q < 4; ++q) r.f[q] = (float *)R[q];
    if (Ulo) {
      for (int q = 0; q < 5; ++q) ul.f[q] = (float *)Ulo[q];
      if (has_rad) for (int q = 0; q < 4; ++q) rl.f[q] = (float *)Rlo[q];
    }
    sums_kernel<float><<<nblocks, SUM_NT, 0, s>>>(g, cr, icc, u, r, has_rad, partials, ul, rl);
  } else {
    F5<double> u, ul{}; F4<double> r{}, rl{};
    for (int q = 0; q < 5; ++q) u.f[q] = (double *)U[q];
    if (has_rad) for (int q = 0; q < 4; ++q) r.f[q] = (double *)R[q];
    sums_kernel<double><<<nblocks, SUM_NT, 0, s>>>(g, cr, icc, u, r, has_rad, partials, ul, rl);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  sums_final_kernel<<<1, 32, 0, s>>>(partials, nblocks, vol, out);
  return cudaGetLastError();
}

// ------------------------------------------------------ arithmetic check ---
// The FP64 reciprocal and square root that the stage kernels use, applied
// element-wise, so that callers and tests can compare them with the IEEE
// operations.
__global__ void eval_math_kernel(const double *x, long long n, double *rcp, double *sq) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const double v = x[i];
    if (rcp) rcp[i] = frcp(v);
    if (sq) sq[i] = psqrt(v);
  }
}

}  // namespace qk

extern "C" int qk_eval_math(const double *x, int64_t n, double *rcp, double *sqrt_out,
                            void *stream) {
  if (n < 0 || (n > 0 && !x)) return QK_EINVAL;
  if (n == 0) return QK_OK;
  const long long blocks = std::min<long long>((n + 255) / 256, 152LL * 16);
  qk::eval_math_kernel<<<(int)blocks, 256, 0, (cudaStream_t)stream>>>(x, n, rcp, sqrt_out);
  return cudaGetLastError() == cudaSuccess ? QK_OK : QK_ECUDA;
}

