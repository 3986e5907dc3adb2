// qk_hydro.cu -- fused hydro RK2-SSP stage (Sec. 2.2.1 of arXiv:2110.01792)
// for sm_103a: conserved -> primitive, PPM reconstruction, HLLC flux, flux
// divergence and the RK combination in one kernel per stage.  Each CTA owns
// one TS^3 tile at a time (grid-stride over a tile work list spanning every
// patch), stages the primitives of the tile and its cross halo in shared
// memory once, then sweeps x, y, z: reconstruct -> face fluxes -> divergence,
// with face states and fluxes kept in shared memory.
#include "qk_device.cuh"

namespace qk {

template <typename T> struct HydroSmem {
  static constexpr bool kF = sizeof(T) == 8;
  T prim[5][NCROSS];   // rho, vx, vy, vz, P of the tile and its cross halo
  T rec[10][NREC];     // per line position: qL, qR of each primitive
  T flux[5][NFLUX];    // per face: mass, momentum x/y/z, energy
  T iface[kF ? 5 : 1][kF ? NIF : 1];  // FP64 PPM: interface values, once per face
};

template <typename T, int D, int NT, int NOWN, int CP>
__device__ __forceinline__ void hydro_dir(HydroSmem<T> &sm, const int v[3], T inv_dx, T gamma,
                                          T gm1inv, T g1, int rk, const T *chi,
                                          const DevBox &bx, int ng, int x0, int y0, int z0,
                                          T (&acc)[NOWN][5], T (&accl)[NOWN][5], T cdt) {
  constexpr int A = (D + 1) % 3, B = (D + 2) % 3;
  // FP64 PPM: the interface values first, once per face
  bool shared_faces = false;
  if constexpr (HydroSmem<T>::kF) {
    if (rk != QK_RECON_PLM) {
      ppm_faces_pass<D, NT, 5>(sm.prim, sm.iface, v);
      shared_faces = true;
      __syncthreads();
    }
  }
  // Phase A: reconstruction of every needed position of every line along D.
  for (int it = threadIdx.x; it < NREC; it += NT) {
    int pos, c[3];
    item_cell<D>(it, NPOS, pos, c[0], c[1], c[2]);
    if (c[A] >= v[A] || c[B] >= v[B] || c[D] > v[D]) continue;
    int s[5];
#pragma unroll
    for (int o = 0; o < 5; ++o) {
      int cc[3] = {c[0], c[1], c[2]};
      cc[D] += o - 2;
      s[o] = cross_slot(cc[0], cc[1], cc[2]);
    }
    // shock flattening: blend the face states with the cell average,
    // q <- chi q + (1 - chi) q_cell (chi from the flattening pre-pass)
    const T ch = chi ? chi[cell_elem(bx, ng, x0 + c[0], y0 + c[1], z0 + c[2])] : T(1);
    int fl = 0, fr = 0;
    if (shared_faces) {
      fl = item_index<D>(pos, c[0], c[1], c[2], NIFP);
      fr = item_index<D>(pos + 1, c[0], c[1], c[2], NIFP);
    }
#pragma unroll
    for (int q = 0; q < 5; ++q) {
      T qL, qR;
      if constexpr (HydroSmem<T>::kF) {
        if (shared_faces)
          ppm_limit(sm.iface[q][fl], sm.iface[q][fr], sm.prim[q][s[1]], sm.prim[q][s[2]],
                    sm.prim[q][s[3]], qL, qR);
        else
          recon<T>(rk, sm.prim[q][s[0]], sm.prim[q][s[1]], sm.prim[q][s[2]], sm.prim[q][s[3]],
                   sm.prim[q][s[4]], qL, qR);
      } else {
        recon<T>(rk, sm.prim[q][s[0]], sm.prim[q][s[1]], sm.prim[q][s[2]], sm.prim[q][s[3]],
                 sm.prim[q][s[4]], qL, qR);
      }
      if (chi) {
        const T qc = sm.prim[q][s[2]];
        qL = ch * qL + (T(1) - ch) * qc;
        qR = ch * qR + (T(1) - ch) * qc;
      }
      sm.rec[2 * q][it] = qL;
      sm.rec[2 * q + 1][it] = qR;
    }
  }
  __syncthreads();
  // Phase B: HLLC flux at every needed face (between positions f and f+1).
  for (int it = threadIdx.x; it < NFLUX; it += NT) {
    int f, c[3];
    item_cell<D>(it, NFACE, f, c[0], c[1], c[2]);
    if (c[A] >= v[A] || c[B] >= v[B] || f > v[D]) continue;
    int il = item_index<D>(f, c[0], c[1], c[2], NPOS);
    int ir = item_index<D>(f + 1, c[0], c[1], c[2], NPOS);
    T wL[5], wR[5], F[5];
#pragma unroll
    for (int q = 0; q < 5; ++q) {
      wL[q] = sm.rec[2 * q + 1][il];
      wR[q] = sm.rec[2 * q][ir];
    }
    hllc<T, D>(wL, wR, gamma, gm1inv, g1, F);
#pragma unroll
    for (int q = 0; q < 5; ++q) sm.flux[q][it] = F[q];
  }
  __syncthreads();
  // Phase C: accumulate the divergence of the owned cells, ((x + y) + z).
#pragma unroll
  for (int m = 0; m < NOWN; ++m) {
    int s = threadIdx.x + m * NT;
    int c[3] = {s % TS, (s / TS) % TS, s / (TS * TS)};
    if (c[0] >= v[0] || c[1] >= v[1] || c[2] >= v[2]) continue;
    int lo = item_index<D>(c[D] + 0, c[0], c[1], c[2], NFACE);
    int hi = item_index<D>(c[D] + 1, c[0], c[1], c[2], NFACE);
    // item_index for faces takes the face number as the position
#pragma unroll
    for (int q = 0; q < 5; ++q) {
      if constexpr (CP) {
        // compensated state: (acc, accl) -= dt (F_hi - F_lo) / dx exactly,
        // each face term dt F / dx rounded once, identically in both cells
        // that share the face, so that the face terms cancel in the sum
        df_add(acc[m][q], accl[m][q], -__fmul_rn(cdt, sm.flux[q][hi]));
        df_add(acc[m][q], accl[m][q], __fmul_rn(cdt, sm.flux[q][lo]));
      } else {
        T dv = (sm.flux[q][hi] - sm.flux[q][lo]) * inv_dx;
        acc[m][q] = (D == 0) ? dv : acc[m][q] + dv;
      }
    }
  }
}

// CP (FP32 only): compensated state, every conserved field held as hi + lo
// (L0, L1, Lo the lo arrays of U0, U1, Uo, stored as lo_get / lo_put read and
// write them: CP = 1 FP32, CP = 2 16 bits); the stencil reads hi only, the
// update is accumulated in double-float so that the face terms telescope.
template <typename T, int STAGE, int NT, int CP>
__global__ void __launch_bounds__(NT) hydro_stage_kernel(Geometry g, qk_params p, SC<T> K,
                                                         F5<T> U0, F5<T> U1, F5<T> Uo, DtSrc dts,
                                                         int sched, const T *chi, F5<T> L0,
                                                         F5<T> L1, F5<T> Lo) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  HydroSmem<T> &sm = *reinterpret_cast<HydroSmem<T> *>(smem_raw);
  constexpr int NOWN = NCORE / NT;
  // the timestep, converted once per CTA
  __shared__ T s_dt;
  if (threadIdx.x == 0) s_dt = (T)dt_of(dts);
  __syncthreads();
  const T dt = s_dt;
  const T gm1 = K.gm1, gamma = K.gamma, gm1inv = K.gm1inv, g1 = K.g1;
  const T *inv_dx = K.inv_dx;
  const F5<T> src = STAGE == 1 ? U0 : U1;

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
    // ---- load: conserved -> primitive into shared memory ----
    T own[NOWN][5], ownl[NOWN][5];
#pragma unroll
    for (int m = 0; m < NOWN; ++m) {
      int s = threadIdx.x + m * NT;
      int i = s % TS, j = (s / TS) % TS, k = s / (TS * TS);
      if (!slot_needed(i, j, k, v)) continue;
      long long e = cell_elem(b, g.ng, tl.x0 + i, tl.y0 + j, tl.z0 + k);
      T u[5], w[5];
#pragma unroll
      for (int q = 0; q < 5; ++q) u[q] = src.f[q][e];
      con2prim<T>(u, gm1, w);
#pragma unroll
      for (int q = 0; q < 5; ++q) {
        own[m][q] = u[q];
        sm.prim[q][s] = w[q];
      }
      if constexpr (CP) {
        if (i < v[0] && j < v[1] && k < v[2]) {
#pragma unroll
          for (int q = 0; q < 5; ++q)
            ownl[m][q] = lo_get<CP>((STAGE == 1 ? L0 : L1).f[q], e, own[m][q]);
        }
      }
    }
    for (int s = NCORE + threadIdx.x; s < NCROSS; s += NT) {
      int i, j, k;
      slot_cell(s, i, j, k);
      if (!slot_needed(i, j, k, v)) continue;
      long long e = cell_elem(b, g.ng, tl.x0 + i, tl.y0 + j, tl.z0 + k);
      T u[5], w[5];
#pragma unroll
      for (int q = 0; q < 5; ++q) u[q] = src.f[q][e];
      con2prim<T>(u, gm1, w);
#pragma unroll
      for (int q = 0; q < 5; ++q) sm.prim[q][s] = w[q];
    }
    __syncthreads();
    T acc[NOWN][5], accl[NOWN][5];
    if constexpr (CP) {
#pragma unroll
      for (int m = 0; m < NOWN; ++m)
#pragma unroll
        for (int q = 0; q < 5; ++q) {
          acc[m][q] = own[m][q];
          accl[m][q] = ownl[m][q];
        }
    }
    hydro_dir<T, 0, NT, NOWN, CP>(sm, v, inv_dx[0], gamma, gm1inv, g1, p.recon, chi, b, g.ng,
                                  tl.x0, tl.y0, tl.z0, acc, accl, dt * inv_dx[0]);
    hydro_dir<T, 1, NT, NOWN, CP>(sm, v, inv_dx[1], gamma, gm1inv, g1, p.recon, chi, b, g.ng,
                                  tl.x0, tl.y0, tl.z0, acc, accl, dt * inv_dx[1]);
    hydro_dir<T, 2, NT, NOWN, CP>(sm, v, inv_dx[2], gamma, gm1inv, g1, p.recon, chi, b, g.ng,
                                  tl.x0, tl.y0, tl.z0, acc, accl, dt * inv_dx[2]);
    // ---- RK2-SSP combination for the owned cells ----
#pragma unroll
    for (int m = 0; m < NOWN; ++m) {
      int s = threadIdx.x + m * NT;
      int i = s % TS, j = (s / TS) % TS, k = s / (TS * TS);
      if (i >= v[0] || j >= v[1] || k >= v[2]) continue;
      long long e = cell_elem(b, g.ng, tl.x0 + i, tl.y0 + j, tl.z0 + k);
#pragma unroll
      for (int q = 0; q < 5; ++q) {
        if constexpr (CP) {
          // (acc, accl) = U^s - dt div F; stage 2 averages it with U^0
          T h = acc[m][q], l = accl[m][q];
          if (STAGE == 2) {
            const T u0h = U0.f[q][e];
            df_add(h, l, u0h);
            l = __fadd_rn(l, lo_get<CP>(L0.f[q], e, u0h));
          }
          df_norm(h, l);
          if (STAGE == 2) {
            h *= T(0.5);
            l *= T(0.5);
          }
          Uo.f[q][e] = h;
          lo_put<CP>(Lo.f[q], e, h, l);
        } else {
          T L = -acc[m][q];
          if (STAGE == 1) {
            Uo.f[q][e] = own[m][q] + dt * L;
          } else {
            T u0 = U0.f[q][e];
            Uo.f[q][e] = T(0.5) * u0 + T(0.5) * (own[m][q] + dt * L);
          }
        }
      }
    }
    // the next tile's load overwrites prim, last read before the syncs of z
  }
}

template <typename T, int STAGE, int NT, int CP>
static cudaError_t launch_one(const Geometry &g, const qk_params &p, void *const *U0,
                              void *const *U1, void *const *Uo, DtSrc dt, int grid, int sched,
                              const void *chi, const LoPtrs &lo, cudaStream_t s) {
  F5<T> a, b, c, l0{}, l1{}, lo_{};
  for (int q = 0; q < 5; ++q) {
    a.f[q] = (T *)U0[q];
    b.f[q] = U1 ? (T *)U1[q] : nullptr;
    c.f[q] = (T *)Uo[q];
    if (CP) {
      l0.f[q] = (T *)lo.l0[q];
      l1.f[q] = lo.l1 ? (T *)lo.l1[q] : nullptr;
      lo_.f[q] = (T *)lo.lo[q];
    }
  }
  int smem = (int)sizeof(HydroSmem<T>);
  auto kern = hydro_stage_kernel<T, STAGE, NT, CP>;
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
  kern<<<grid, NT, smem, s>>>(g, p, make_sc<T>(p), a, b, c, dt, sched, (const T *)chi, l0, l1,
                              lo_);
  return cudaGetLastError();
}

template <typename T, int STAGE, int CP>
static cudaError_t launch_nt(const Geometry &g, const qk_params &p, void *const *U0,
                             void *const *U1, void *const *Uo, DtSrc dt, int grid, int cfg,
                             const void *chi, const LoPtrs &lo, cudaStream_t s) {
  const int sched = cfg_sched(cfg);
  // the 16-bit compensated form exists for 256 threads per tile only
  if constexpr (CP == 2) {
    return launch_one<T, STAGE, 256, CP>(g, p, U0, U1, Uo, dt, grid, sched, chi, lo, s);
  } else {
    switch (cfg_threads(cfg)) {
      case 128:
        return launch_one<T, STAGE, 128, CP>(g, p, U0, U1, Uo, dt, grid, sched, chi, lo, s);
      case 512:
        return launch_one<T, STAGE, 512, CP>(g, p, U0, U1, Uo, dt, grid, sched, chi, lo, s);
      default:
        return launch_one<T, STAGE, 256, CP>(g, p, U0, U1, Uo, dt, grid, sched, chi, lo, s);
    }
  }
}

cudaError_t launch_hydro_stage(int fp32, int stage, const Geometry &g, const qk_params &p,
                               void *const *U0, void *const *U1, void *const *Uout, DtSrc dt,
                               int grid, int cfg, const void *chi, cudaStream_t s,
                               const LoPtrs *lo) {
  // columns (shape 1) when the geometry has them; compensated states use tiles
  if (cfg_shape(cfg) == 1 && g.cols && g.ncols > 0 && !lo)
    return launch_hydro_column(fp32, stage, g, p, U0, U1, Uout, dt, chi, s, cfg);
  if (fp32 && lo && lo->fmt == 2)
    return stage == 1 ? launch_nt<float, 1, 2>(g, p, U0, U1, Uout, dt, grid, cfg, chi, *lo, s)
                      : launch_nt<float, 2, 2>(g, p, U0, U1, Uout, dt, grid, cfg, chi, *lo, s);
  if (fp32 && lo)
    return stage == 1 ? launch_nt<float, 1, 1>(g, p, U0, U1, Uout, dt, grid, cfg, chi, *lo, s)
                      : launch_nt<float, 2, 1>(g, p, U0, U1, Uout, dt, grid, cfg, chi, *lo, s);
  const LoPtrs none{};
  if (fp32)
    return stage == 1 ? launch_nt<float, 1, 0>(g, p, U0, U1, Uout, dt, grid, cfg, chi, none, s)
                      : launch_nt<float, 2, 0>(g, p, U0, U1, Uout, dt, grid, cfg, chi, none, s);
  return stage == 1 ? launch_nt<double, 1, 0>(g, p, U0, U1, Uout, dt, grid, cfg, chi, none, s)
                    : launch_nt<double, 2, 0>(g, p, U0, U1, Uout, dt, grid, cfg, chi, none, s);
}

// ------------------------------------------------------------- flattening ---
// Shock flattening coefficient chi (Sec. 2.2.1; Colella & Woodward 1984,
// appendix, and its multidimensional form by Miller & Colella 2002) of every
// cell within one cell of a patch interior, written into `chi` (same layout as
// the fields).  Per direction d: ftilde = min(1, max(0, 10 (|dp1|/|dp2| -
// 0.75))) in a compressive jump (u_{c-1} > u_{c+1}, |dp1| > 0.33 min(p_{c+1},
// p_{c-1})), else 0, with dp1 = p_{c+1} - p_{c-1}, dp2 = p_{c+2} - p_{c-2};
// f_d = max(ftilde(c), ftilde(c - sign(dp1))); chi = min_d (1 - f_d).
template <typename T>
__device__ __forceinline__ void flat_prim(const F5<T> &U, long long e, T gm1, int d,
                                          T &pr, T &un) {
  T u[5], w[5];
#pragma unroll
  for (int q = 0; q < 5; ++q) u[q] = U.f[q][e];
  con2prim<T>(u, gm1, w);
  pr = w[4];
  un = w[1 + d];
}

template <typename T>
__device__ __forceinline__ T flat_ftilde(const T pr[7], const T un[7], int c) {
  // c indexes the 7-point window -3..3 (c in 2..4)
  const T dp1 = pr[c + 1] - pr[c - 1], dp2 = pr[c + 2] - pr[c - 2];
  const bool shock = fabs(dp1) > T(0.33) * min(pr[c + 1], pr[c - 1]) && un[c - 1] - un[c + 1] > T(0);
  if (!shock) return T(0);
  if (!(fabs(dp2) > T(0))) return T(1);
  return min(T(1), max(T(0), T(10) * (qdiv(fabs(dp1), fabs(dp2)) - T(0.75))));
}

template <typename T>
__global__ void __launch_bounds__(512) flatten_kernel(Geometry g, double gamma, F5<T> U, T *chi) {
  const T gm1 = (T)(gamma - 1.0);
  for (int t = blockIdx.x; t < g.ntiles; t += gridDim.x) {
    const Tile tl = g.tiles[t];
    const DevBox b = g.boxes[tl.box];
    const int v[3] = {min(TS, b.n[0] - tl.x0), min(TS, b.n[1] - tl.y0), min(TS, b.n[2] - tl.z0)};
    // the tile extended by one cell on every side: (v+2)^3 cells
    const int ex = v[0] + 2, ey = v[1] + 2, ez = v[2] + 2;
    for (int l = threadIdx.x; l < ex * ey * ez; l += blockDim.x) {
      const int c[3] = {l % ex - 1, (l / ex) % ey - 1, l / (ex * ey) - 1};
      T x = T(1);
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        T pr[7], un[7];
#pragma unroll
        for (int o = -3; o <= 3; ++o) {
          int cc[3] = {tl.x0 + c[0], tl.y0 + c[1], tl.z0 + c[2]};
          cc[d] += o;
          flat_prim<T>(U, cell_elem(b, g.ng, cc[0], cc[1], cc[2]), gm1, d, pr[o + 3], un[o + 3]);
        }
        T f = flat_ftilde<T>(pr, un, 3);
        const T dp1 = pr[4] - pr[2];
        if (dp1 > T(0)) f = max(f, flat_ftilde<T>(pr, un, 2));
        else if (dp1 < T(0)) f = max(f, flat_ftilde<T>(pr, un, 4));
        x = min(x, T(1) - f);
      }
      chi[cell_elem(b, g.ng, tl.x0 + c[0], tl.y0 + c[1], tl.z0 + c[2])] = x;
    }
  }
}

cudaError_t launch_flatten(int fp32, const Geometry &g, const qk_params &p, void *const *U,
                           void *chi, cudaStream_t s) {
  int nsm = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const int grid = g.ntiles < nsm * 4 ? g.ntiles : nsm * 4;
  if (grid < 1) return cudaSuccess;
  if (fp32) {
    F5<float> u;
    for (int q = 0; q < 5; ++q) u.f[q] = (float *)U[q];
    flatten_kernel<float><<<grid, 512, 0, s>>>(g, p.gamma, u, (float *)chi);
  } else {
    F5<double> u;
    for (int q = 0; q < 5; ++q) u.f[q] = (double *)U[q];
    flatten_kernel<double><<<grid, 512, 0, s>>>(g, p.gamma, u, (double *)chi);
  }
  return cudaGetLastError();
}

int hydro_smem_bytes(int fp32) {
  return fp32 ? (int)sizeof(HydroSmem<float>) : (int)sizeof(HydroSmem<double>);
}

}  // namespace qk
