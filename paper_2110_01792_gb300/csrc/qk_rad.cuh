// qk_rad.cuh -- fused radiation RK2-SSP stage (Sec. 2.2.2 of arXiv:2110.01792)
// for sm_103a: PPM reconstruction of E_r and f = F/(c E_r), first-order
// fallback at faces where a state has |f| > 1, the M1 closure
// (eq. M1_closure; Levermore, Minerbo or Eddington, a template parameter), HLL flux with wavespeeds from the cell-average Eddington
// factors, optical-depth correction, RSLA fluxes (eqs. rad_energy, rad_flux),
// divergence and RK combination.  Same tile scheme as the hydro stage.
#pragma once
#include "qk_exchange.cuh"

namespace qk {

// FP64 keeps the cell-average closure coefficients (a, b) of every slot next
// to a face (computed once per cell, shared by the three directions); FP32
// recomputes sqrt(T_DD) per line position instead, which is cheap on the FP32
// pipe and keeps three CTAs per SM.
template <typename T> struct RadSmem {
  static constexpr bool kAB = sizeof(T) == 8;
  T prim[4][NCROSS];               // E_r, f_x, f_y, f_z of the tile and its cross halo
  T rk[NCROSS];                    // rho kappa_R of the cell
  T ab[2][kAB ? NCROSS : 1];       // FP64: Levermore a, b of the cell-average state
  T rec[8][NREC];                  // qL, qR of each reconstructed variable
  T iface[kAB ? 4 : 1][kAB ? NIF : 1];  // FP64 PPM: interface values, once per face
  T sq[kAB ? 1 : NREC];            // FP32: sqrt(T_DD) of the cell average per position
  T flux[4][NFLUX];
};

// The matter-radiation exchange fused into the epilogue of stage 2 (qk_step):
// the gas fields U (and their low parts UL for a compensated state), the
// emissivity field or NULL, and the status word.  on = 0: plain stage.
template <typename T> struct ExFuse {
  F5<T> U, UL;
  const T *src;
  Status *st;
  ExK K;
  int on;
};

template <typename T> __device__ __forceinline__ T kappa_of(const qk_params &p, double k, T rho) {
  return p.kappa_mode == QK_KAPPA_RHO ? (T)k * rho : (T)k;
}
// rho kappa_R of a cell from the host-formed constant (no conversion)
template <typename T> __device__ __forceinline__ T rho_kappa(const SC<T> &K, T rho) {
  return rho * (K.kmode == QK_KAPPA_RHO ? K.kR * rho : K.kR);
}

// Stage one cross slot: E_r, f = F / (c E_r) (one reciprocal), rho kappa_R,
// and in FP64 the closure coefficients of the cell average when the slot is
// adjacent to a face of the tile (within one cell of the valid region).
template <typename T, int CL>
__device__ __forceinline__ void load_slot(RadSmem<T> &sm, int s, const T u[4], T c, T r,
                                          const SC<T> &K, int i, int j, int k,
                                          const int v[3]) {
  const T inv = qrcp(c * u[0]);
  const T fx = u[1] * inv, fy = u[2] * inv, fz = u[3] * inv;
  sm.prim[0][s] = u[0];
  sm.prim[1][s] = fx;
  sm.prim[2][s] = fy;
  sm.prim[3][s] = fz;
  sm.rk[s] = rho_kappa<T>(K, r);
  if constexpr (RadSmem<T>::kAB) {
    const bool near = i >= -1 && j >= -1 && k >= -1 && i <= v[0] && j <= v[1] && k <= v[2];
    if (near) {
      T a, b;
      closure_ab<T, CL>(fx, fy, fz, a, b);
      sm.ab[0][s] = a;
      sm.ab[1][s] = b;
    }
  }
}

// HLL wavespeed from the diagonal Eddington-tensor elements T_DD of the two
// cell averages (Sec. 2.2.2): S = chat sqrt(max(Ta, Tb)), equal to chat
// max(sqrt(Ta), sqrt(Tb)) since the square root is monotone (within an ulp:
// psqrt).  T_DD lies in [0, 1]; it is 0 only for a superluminal state with no
// flux along D.
template <typename T>
__device__ __forceinline__ T rad_speed(T Ta, T Tb, T chat) {
  const T Tm = nn_max(Ta, Tb);
  return nn_gt(Tm, T(0)) ? chat * psqrt(Tm) : T(0);
}

// The radiation flux through one face (Sec. 2.2.2): the face states wL, wR
// (reconstructed E_r and f; `fallback` replaces both by the two cell
// averages when either has |f| > 1), the wavespeed S, the cells' rho kappa_R
// for the optical-depth correction, HLL with S_L = -S, S_R = S, and the
// correction switched off where it would make the energy flux exceed
// chat max(E_L, E_R).  Shared by the stage kernel and the flux registers of
// mesh refinement, so both use the same arithmetic.
//
// With flux_D = ((chat/c) F_D, c chat E T_qD) (eqs. rad_energy, rad_flux),
// F = c E f and T = a I + b f f (closure CL), the HLL flux
// (flux_L + flux_R)/2 - (S eps/2)(U_R - U_L) is evaluated as
//   energy: (chat/2)(E_L f_L,D + E_R f_R,D) - (S eps/2)(E_R - E_L),
//   F_q:    al_L f_L,q + al_R f_R,q (+ (c chat/2)(E_L a_L + E_R a_R) for q = D),
// al_L = (c chat/2) E_L b_L f_L,D + (S eps c/2) E_L and
// al_R = (c chat/2) E_R b_R f_R,D - (S eps c/2) E_R: the terms of each side
// that multiply the same f_q are gathered before the product.
template <typename T, int D, int CL, class Fallback>
__device__ __forceinline__ void rad_face_hll(T wL[4], T wR[4], Fallback fallback, T S, T rka,
                                             T rkb, T dx, T c, T chat, T hchat_c, T hccc,
                                             int tau_corr, T out[4]) {
  constexpr int A = (D + 1) % 3, B = (D + 2) % 3;
  T fL2 = (wL[1] * wL[1] + wL[2] * wL[2]) + wL[3] * wL[3];
  T fR2 = (wR[1] * wR[1] + wR[2] * wR[2]) + wR[3] * wR[3];
  if (nn_gt(fL2, T(1)) || nn_gt(fR2, T(1))) {
    fallback(wL, wR);
    fL2 = (wL[1] * wL[1] + wL[2] * wL[2]) + wL[3] * wL[3];
    fR2 = (wR[1] * wR[1] + wR[2] * wR[2]) + wR[3] * wR[3];
  }
  T aL, bL, aR, bR;
  closure_ab_f2<T, CL>(fL2, aL, bL);
  closure_ab_f2<T, CL>(fR2, aR, bR);
  const T EL = wL[0], ER = wR[0], fLD = wL[1 + D], fRD = wR[1 + D];
  T eps = T(1);
  if (tau_corr) {
    const T tau = dx * T(0.5) * (rka + rkb);
    if (nn_gt(tau, T(1))) eps = qrcp(tau);
  }
  const T hS = T(0.5) * S;
  T hSe = hS * eps;
  const T FE = (hchat_c * c) * fma(EL, fLD, ER * fRD);
  const T dE = ER - EL;
  T o0 = fma(-hSe, dE, FE);
  if (nn_gt(T(1), eps) && nn_gt(fabs(o0), chat * nn_max(EL, ER))) {
    hSe = hS;
    o0 = fma(-hSe, dE, FE);
  }
  out[0] = o0;
  const T hSec = hSe * c;
  const T cEbL = hccc * EL, cEbR = hccc * ER;
  const T alL = fma(cEbL * bL, fLD, hSec * EL);
  const T alR = fma(cEbR * bR, fRD, -(hSec * ER));
  out[1 + A] = fma(alL, wL[1 + A], alR * wR[1 + A]);
  out[1 + B] = fma(alL, wL[1 + B], alR * wR[1 + B]);
  out[1 + D] = fma(alL, fLD, fma(alR, fRD, fma(cEbL, aL, cEbR * aR)));
}

template <typename T, int D, int NT, int NOWN, int CL, int CP>
__device__ __forceinline__ void rad_dir(RadSmem<T> &sm, const int v[3], T inv_dx, T dx, T c,
                                        T chat, int tau_corr, int rk, T (&acc)[NOWN][4],
                                        T (&accl)[NOWN][4], T cdt) {
  constexpr int A = (D + 1) % 3, B = (D + 2) % 3;
  const T hccc = T(0.5) * c * chat;
  const T hchat_c = T(0.5) * chat / c;
  // FP64 PPM: the interface values first, once per face
  bool shared_faces = false;
  if constexpr (RadSmem<T>::kAB) {
    if (rk != QK_RECON_PLM) {
      ppm_faces_pass<D, NT, 4>(sm.prim, sm.iface, v);
      shared_faces = true;
      __syncthreads();
    }
  }
  for (int it = threadIdx.x; it < NREC; it += NT) {
    int pos, cc[3];
    item_cell<D>(it, NPOS, pos, cc[0], cc[1], cc[2]);
    if (cc[A] >= v[A] || cc[B] >= v[B] || cc[D] > v[D]) continue;
    int s[5];
#pragma unroll
    for (int o = 0; o < 5; ++o) {
      int x[3] = {cc[0], cc[1], cc[2]};
      x[D] += o - 2;
      s[o] = cross_slot(x[0], x[1], x[2]);
    }
    if constexpr (RadSmem<T>::kAB) {
      if (shared_faces) {
        const int fl = item_index<D>(pos, cc[0], cc[1], cc[2], NIFP);
        const int fr = item_index<D>(pos + 1, cc[0], cc[1], cc[2], NIFP);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          T qL, qR;
          ppm_limit(sm.iface[q][fl], sm.iface[q][fr], sm.prim[q][s[1]], sm.prim[q][s[2]],
                    sm.prim[q][s[3]], qL, qR);
          sm.rec[2 * q][it] = qL;
          sm.rec[2 * q + 1][it] = qR;
        }
        continue;
      }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      T qL, qR;
      recon<T>(rk, sm.prim[q][s[0]], sm.prim[q][s[1]], sm.prim[q][s[2]], sm.prim[q][s[3]],
               sm.prim[q][s[4]], qL, qR);
      sm.rec[2 * q][it] = qL;
      sm.rec[2 * q + 1][it] = qR;
    }
    if constexpr (!RadSmem<T>::kAB)
      sm.sq[it] = qsqrt(eddington_diag<T, D, CL>(sm.prim[1][s[2]], sm.prim[2][s[2]], sm.prim[3][s[2]]));
  }
  __syncthreads();
  for (int it = threadIdx.x; it < NFLUX; it += NT) {
    int f, cc[3];
    item_cell<D>(it, NFACE, f, cc[0], cc[1], cc[2]);
    if (cc[A] >= v[A] || cc[B] >= v[B] || f > v[D]) continue;
    const int il = item_index<D>(f, cc[0], cc[1], cc[2], NPOS);
    const int ir = item_index<D>(f + 1, cc[0], cc[1], cc[2], NPOS);
    T wL[4], wR[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      wL[q] = sm.rec[2 * q + 1][il];
      wR[q] = sm.rec[2 * q][ir];
    }
    int xa[3] = {cc[0], cc[1], cc[2]}, xb[3] = {cc[0], cc[1], cc[2]};
    xa[D] = f - 1;
    xb[D] = f;
    const int sa = cross_slot(xa[0], xa[1], xa[2]);
    const int sb = cross_slot(xb[0], xb[1], xb[2]);
    T S;
    if constexpr (RadSmem<T>::kAB) {
      const T fa = sm.prim[1 + D][sa], fb = sm.prim[1 + D][sb];
      S = rad_speed<T>(sm.ab[0][sa] + sm.ab[1][sa] * fa * fa, sm.ab[0][sb] + sm.ab[1][sb] * fb * fb,
                       chat);
    } else {
      S = chat * max(sm.sq[il], sm.sq[ir]);
    }
    T out[4];
    rad_face_hll<T, D, CL>(
        wL, wR,
        [&](T *l, T *r) {
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            l[q] = sm.prim[q][sa];
            r[q] = sm.prim[q][sb];
          }
        },
        S, sm.rk[sa], sm.rk[sb], dx, c, chat, hchat_c, hccc, tau_corr, out);
#pragma unroll
    for (int q = 0; q < 4; ++q) sm.flux[q][it] = out[q];
  }
  __syncthreads();
#pragma unroll
  for (int m = 0; m < NOWN; ++m) {
    int s = threadIdx.x + m * NT;
    int cc[3] = {s % TS, (s / TS) % TS, s / (TS * TS)};
    if (cc[0] >= v[0] || cc[1] >= v[1] || cc[2] >= v[2]) continue;
    int lo = item_index<D>(cc[D], cc[0], cc[1], cc[2], NFACE);
    int hi = item_index<D>(cc[D] + 1, cc[0], cc[1], cc[2], NFACE);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      if constexpr (CP) {
        // compensated state: face terms dt F / dx rounded once per face
        df_add(acc[m][q], accl[m][q], -__fmul_rn(cdt, sm.flux[q][hi]));
        df_add(acc[m][q], accl[m][q], __fmul_rn(cdt, sm.flux[q][lo]));
      } else {
        T dv = (sm.flux[q][hi] - sm.flux[q][lo]) * inv_dx;
        acc[m][q] = (D == 0) ? dv : acc[m][q] + dv;
      }
    }
  }
}

// CP (FP32 only): compensated state hi + lo (L0, L1, Lo the lo arrays of R0,
// R1, Ro), as in the hydro stage.  EX (stage 2 only): the matter-radiation
// exchange of every owned cell after its update (xf: the gas fields, the
// emissivity and the status word).
// FP32 kernels with the fused exchange are held to the registers of three
// CTAs per SM (as many as their shared memory allows), the exchange's FP64
// temporaries spilling to L1 rather than halving the resident warps.
template <typename T, int NT, bool EX> struct RadMinBlocks {
  static constexpr int value = (EX && sizeof(T) == 4) ? (NT == 128 ? 6 : (NT == 256 ? 3 : 1)) : 1;
};

template <typename T, int STAGE, int NT, int CL, int CP, bool EX>
__device__ __forceinline__ void rad_stage_body(const Geometry &g, const qk_params &p,
                                               const SC<T> &K, F4<T> R0, F4<T> R1, F4<T> Ro,
                                               const T *rho, DtSrc dts, int sched, F4<T> L0,
                                               F4<T> L1, F4<T> Lo, const ExFuse<T> &xf) {
  if (skip_substep(dts)) return;
  ExStat xs;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  RadSmem<T> &sm = *reinterpret_cast<RadSmem<T> *>(smem_raw);
  constexpr int NOWN = NCORE / NT;
  // the timestep, converted once per CTA
  __shared__ T s_dt;
  if (threadIdx.x == 0) s_dt = (T)dt_of(dts);
  __syncthreads();
  const T dt = s_dt;
  const T c = K.c, chat = K.chat;
  const T *inv_dx = K.inv_dx, *dx = K.dx;
  const F4<T> src = STAGE == 1 ? R0 : R1;

  // tile schedule: strided over the grid (0) or one contiguous run of tiles
  // per CTA (1, neighbouring tiles in sequence on one SM)
  int t0 = blockIdx.x, t1 = g.ntiles, tstep = gridDim.x;
  if (sched) {
    const int per = (g.ntiles + gridDim.x - 1) / gridDim.x;
    t0 = blockIdx.x * per;
    t1 = min(g.ntiles, t0 + per);
    tstep = 1;
  }
  for (int t = t0; t < t1; t += tstep) {
    const Tile tl = g.tiles[t];
    const DevBox b = g.boxes[tl.box];
    const int v[3] = {min(TS, b.n[0] - tl.x0), min(TS, b.n[1] - tl.y0), min(TS, b.n[2] - tl.z0)};
    T own[NOWN][4], ownl[NOWN][4];
#pragma unroll
    for (int m = 0; m < NOWN; ++m) {
      int s = threadIdx.x + m * NT;
      int i = s % TS, j = (s / TS) % TS, k = s / (TS * TS);
      if (!slot_needed(i, j, k, v)) continue;
      long long e = cell_elem(b, g.ng, tl.x0 + i, tl.y0 + j, tl.z0 + k);
      T u[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) u[q] = src.f[q][e];
      load_slot<T, CL>(sm, s, u, c, rho[e], K, i, j, k, v);
#pragma unroll
      for (int q = 0; q < 4; ++q) own[m][q] = u[q];
      if constexpr (CP) {
        if (i < v[0] && j < v[1] && k < v[2]) {
#pragma unroll
          for (int q = 0; q < 4; ++q)
            ownl[m][q] = lo_get<CP>((STAGE == 1 ? L0 : L1).f[q], e, own[m][q]);
        }
      }
    }
    for (int s = NCORE + threadIdx.x; s < NCROSS; s += NT) {
      int i, j, k;
      slot_cell(s, i, j, k);
      if (!slot_needed(i, j, k, v)) continue;
      long long e = cell_elem(b, g.ng, tl.x0 + i, tl.y0 + j, tl.z0 + k);
      T u[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) u[q] = src.f[q][e];
      load_slot<T, CL>(sm, s, u, c, rho[e], K, i, j, k, v);
    }
    __syncthreads();
    T acc[NOWN][4], accl[NOWN][4];
    if constexpr (CP) {
#pragma unroll
      for (int m = 0; m < NOWN; ++m)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          acc[m][q] = own[m][q];
          accl[m][q] = ownl[m][q];
        }
    }
    rad_dir<T, 0, NT, NOWN, CL, CP>(sm, v, inv_dx[0], dx[0], c, chat, p.tau_correction, p.recon,
                                    acc, accl, dt * inv_dx[0]);
    rad_dir<T, 1, NT, NOWN, CL, CP>(sm, v, inv_dx[1], dx[1], c, chat, p.tau_correction, p.recon,
                                    acc, accl, dt * inv_dx[1]);
    rad_dir<T, 2, NT, NOWN, CL, CP>(sm, v, inv_dx[2], dx[2], c, chat, p.tau_correction, p.recon,
                                    acc, accl, dt * inv_dx[2]);
#pragma unroll
    for (int m = 0; m < NOWN; ++m) {
      int s = threadIdx.x + m * NT;
      int i = s % TS, j = (s / TS) % TS, k = s / (TS * TS);
      if (i >= v[0] || j >= v[1] || k >= v[2]) continue;
      long long e = cell_elem(b, g.ng, tl.x0 + i, tl.y0 + j, tl.z0 + k);
      T rv[4], rl[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        if constexpr (CP) {
          T h = acc[m][q], l = accl[m][q];
          if (STAGE == 2) {
            const T r0h = R0.f[q][e];
            df_add(h, l, r0h);
            l = __fadd_rn(l, lo_get<CP>(L0.f[q], e, r0h));
          }
          df_norm(h, l);
          if (STAGE == 2) {
            h *= T(0.5);
            l *= T(0.5);
          }
          rv[q] = h;
          rl[q] = l;
        } else {
          T L = -acc[m][q];
          if (STAGE == 1) {
            rv[q] = own[m][q] + dt * L;
          } else {
            T u0 = R0.f[q][e];
            rv[q] = T(0.5) * u0 + T(0.5) * (own[m][q] + dt * L);
          }
          rl[q] = T(0);
        }
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        Ro.f[q][e] = rv[q];
        if constexpr (CP) lo_put<CP>(Lo.f[q], e, rv[q], rl[q]);
      }
    }
    if constexpr (EX) {
      // the exchange of the owned cells on the state just stored (read back
      // by the same thread, from L1/L2); one cell at a time keeps the
      // exchange's registers apart from the sweeps'
#pragma unroll 1
      for (int m = 0; m < NOWN; ++m) {
        int s = threadIdx.x + m * NT;
        int i = s % TS, j = (s / TS) % TS, k = s / (TS * TS);
        if (i >= v[0] || j >= v[1] || k >= v[2]) continue;
        long long e = cell_elem(b, g.ng, tl.x0 + i, tl.y0 + j, tl.z0 + k);
        if constexpr (sizeof(T) == 8) {
          const double fr[3] = {(double)Ro.f[1][e], (double)Ro.f[2][e], (double)Ro.f[3][e]};
          exchange_cell<T>(p, xf.K, dt_of(dts), xf.U, Ro, xf.src, e, (double)Ro.f[0][e], fr,
                           xs);
        } else {
          const float fr[3] = {Ro.f[1][e], Ro.f[2][e], Ro.f[3][e]};
          float fl[3] = {0.0f, 0.0f, 0.0f}, el = 0.0f;
          const float er = Ro.f[0][e];
          if constexpr (CP) {
            el = lo_get<CP>(Lo.f[0], e, er);
            fl[0] = lo_get<CP>(Lo.f[1], e, fr[0]);
            fl[1] = lo_get<CP>(Lo.f[2], e, fr[1]);
            fl[2] = lo_get<CP>(Lo.f[3], e, fr[2]);
          }
          exchange_cell_mixed<CP>(p, xf.K, dt_of(dts), dt, xf.U, Ro, xf.UL, Lo, xf.src, e, er,
                                  el, fr, fl, xs);
        }
      }
    }
  }
  if constexpr (EX) exchange_status(xf.st, xs.max, xs.flags, xs.bad);
}

template <typename T, int STAGE, int NT, int CL, int CP>
__global__ void __launch_bounds__(NT) rad_stage_kernel(Geometry g, qk_params p, SC<T> K,
                                                       F4<T> R0, F4<T> R1, F4<T> Ro, const T *rho,
                                                       DtSrc dts, int sched, F4<T> L0, F4<T> L1,
                                                       F4<T> Lo, ExFuse<T> xf) {
  rad_stage_body<T, STAGE, NT, CL, CP, false>(g, p, K, R0, R1, Ro, rho, dts, sched, L0, L1, Lo,
                                              xf);
}

template <typename T, int NT, int CL, int CP>
__global__ void __launch_bounds__(NT, (RadMinBlocks<T, NT, true>::value))
    rad_stage_ex_kernel(Geometry g, qk_params p, SC<T> K, F4<T> R0, F4<T> R1, F4<T> Ro,
                        const T *rho, DtSrc dts, int sched, F4<T> L0, F4<T> L1, F4<T> Lo,
                        ExFuse<T> xf) {
  rad_stage_body<T, 2, NT, CL, CP, true>(g, p, K, R0, R1, Ro, rho, dts, sched, L0, L1, Lo, xf);
}

template <typename T, int STAGE, int NT, int CL, int CP>
static cudaError_t launch_one(const Geometry &g, const qk_params &p, void *const *R0,
                              void *const *R1, void *const *Ro, const void *rho, DtSrc dt,
                              int grid, int sched, const LoPtrs &lo, const FuseArgs *fx,
                              cudaStream_t s) {
  F4<T> a, b, c, l0{}, l1{}, lo_{};
  for (int q = 0; q < 4; ++q) {
    a.f[q] = (T *)R0[q];
    b.f[q] = R1 ? (T *)R1[q] : nullptr;
    c.f[q] = (T *)Ro[q];
    if (CP) {
      l0.f[q] = (T *)lo.l0[q];
      l1.f[q] = lo.l1 ? (T *)lo.l1[q] : nullptr;
      lo_.f[q] = (T *)lo.lo[q];
    }
  }
  ExFuse<T> xf{};
  if (fx && STAGE == 2) {
    for (int q = 0; q < 5; ++q) {
      xf.U.f[q] = (T *)fx->U[q];
      xf.UL.f[q] = fx->Ulo ? (T *)fx->Ulo[q] : nullptr;
    }
    xf.src = (const T *)fx->src;
    xf.st = fx->st;
    xf.K = make_exk(p);
    xf.on = 1;
  }
  int smem = (int)sizeof(RadSmem<T>);
  auto kern = rad_stage_kernel<T, STAGE, NT, CL, CP>;
  if constexpr (STAGE == 2)
    if (xf.on) kern = rad_stage_ex_kernel<T, NT, CL, CP>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  if (grid <= 0) {
    int per_sm = 0, nsm = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT, smem);
    grid = nsm * (per_sm > 0 ? per_sm : 1);
  }
  if (grid > g.ntiles) grid = g.ntiles;
  if (grid < 1) return cudaSuccess;
  kern<<<grid, NT, smem, s>>>(g, p, make_sc<T>(p), a, b, c, (const T *)rho, dt, sched, l0, l1,
                              lo_, xf);
  return cudaGetLastError();
}

template <typename T, int STAGE, int CL, int CP>
static cudaError_t launch_nt(const Geometry &g, const qk_params &p, void *const *R0,
                             void *const *R1, void *const *Ro, const void *rho, DtSrc dt,
                             int grid, int cfg, const LoPtrs &lo, const FuseArgs *fx,
                             cudaStream_t s) {
  const int sched = cfg_sched(cfg);
  // the 16-bit compensated form exists for 256 threads per tile only
  if constexpr (CP == 2) {
    return launch_one<T, STAGE, 256, CL, CP>(g, p, R0, R1, Ro, rho, dt, grid, sched, lo, fx, s);
  } else {
    switch (cfg_threads(cfg)) {
      case 128:
        return launch_one<T, STAGE, 128, CL, CP>(g, p, R0, R1, Ro, rho, dt, grid, sched, lo, fx,
                                                 s);
      case 512:
        return launch_one<T, STAGE, 512, CL, CP>(g, p, R0, R1, Ro, rho, dt, grid, sched, lo, fx,
                                                 s);
      default:
        return launch_one<T, STAGE, 256, CL, CP>(g, p, R0, R1, Ro, rho, dt, grid, sched, lo, fx,
                                                 s);
    }
  }
}

// All stage kernels of one closure (instantiated in qk_rad.cu and
// qk_rad_closures.cu, which nvcc compiles in parallel).  `lo` non-null selects
// the compensated FP32 kernels; `fx` non-null fuses the exchange into stage 2.
template <int CL>
cudaError_t launch_rad_closure(int fp32, int stage, const Geometry &g, const qk_params &p,
                               void *const *R0, void *const *R1, void *const *Rout,
                               const void *rho, DtSrc dt, int grid, int cfg, cudaStream_t s,
                               const LoPtrs *lo, const FuseArgs *fx) {
  if (fp32 && lo && lo->fmt == 2)
    return stage == 1
               ? launch_nt<float, 1, CL, 2>(g, p, R0, R1, Rout, rho, dt, grid, cfg, *lo, fx, s)
               : launch_nt<float, 2, CL, 2>(g, p, R0, R1, Rout, rho, dt, grid, cfg, *lo, fx, s);
  if (fp32 && lo)
    return stage == 1
               ? launch_nt<float, 1, CL, 1>(g, p, R0, R1, Rout, rho, dt, grid, cfg, *lo, fx, s)
               : launch_nt<float, 2, CL, 1>(g, p, R0, R1, Rout, rho, dt, grid, cfg, *lo, fx, s);
  const LoPtrs none{};
  if (fp32)
    return stage == 1
               ? launch_nt<float, 1, CL, 0>(g, p, R0, R1, Rout, rho, dt, grid, cfg, none, fx, s)
               : launch_nt<float, 2, CL, 0>(g, p, R0, R1, Rout, rho, dt, grid, cfg, none, fx, s);
  return stage == 1
             ? launch_nt<double, 1, CL, 0>(g, p, R0, R1, Rout, rho, dt, grid, cfg, none, fx, s)
             : launch_nt<double, 2, CL, 0>(g, p, R0, R1, Rout, rho, dt, grid, cfg, none, fx, s);
}

}  // namespace qk
