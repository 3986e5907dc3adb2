// qk_column.cu -- plane-marching form of the fused hydro RK2-SSP stage
// (Sec. 2.2.1 of arXiv:2110.01792) for sm_103a: the same arithmetic per cell
// and per face as qk_hydro.cu (con2prim, PPM/PLM with flattening, HLLC, the
// divergence summed ((x + y) + z), the RK combination), organised for fewer
// instructions per cell.  A CTA of CW x CW threads owns a CW x CW footprint of
// one patch and walks its planes along z:
//   - z: every thread keeps the primitives of planes z-1 .. z+3 of its own
//     cell in registers, reconstructs cell z+1 and computes the flux through
//     face z+1/2 once; the flux through z-1/2 is carried from the previous
//     plane, so each z face is solved once per column;
//   - x and y: the plane z with a HALO-deep ring sits in shared memory;
//     reconstruction (CW+2 positions per row) and faces (CW+1 per row) of both
//     directions are computed in one pass each;
//   - the item -> shared-memory index maps are fixed for the whole column.
// Two barriers per plane.  Used through launch configurations of shape 1
// (cfg_shape); results equal the TS^3 tile kernels' up to the rounding of
// the identical formulas (the same device functions).
#include "qk_pair.cuh"

namespace qk {

template <typename T> struct ColSmem {
  T prim[5][CNPL];                 // rho, vx, vy, vz, P of plane z and its ring
  T rec[2][10][CXPOS * CW];        // x and y: qL, qR of each primitive per position
  T flux[2][5][CXFACE * CW];       // x and y face fluxes
  // FP32: the own cell's U_src (5) and U_0 (5, stage 2) read by the epilogue,
  // staged one phase ahead (cp.async)
  static constexpr bool kPre = sizeof(T) == 4;
  T pre[kPre ? 10 : 1][kPre ? CNT : 1];
  // FP32: the conserved values of the next plane to enter (own cells, then
  // ring cells), staged one plane ahead (cp.async)
  T nxt[kPre ? 5 : 1][kPre ? CNT + CNRING : 1];
};

__device__ __forceinline__ int pslot(int i, int j) { return (j + HALO) * CPW + (i + HALO); }

// HLLC along axis D from the face states, as the tile kernel's phase B.
template <typename T, int D>
__device__ __forceinline__ void col_face(const T wL[5], const T wR[5], T gamma, T gm1inv, T g1,
                                         T F[5]) {
  hllc<T, D>(wL, wR, gamma, gm1inv, g1, F);
}

template <typename T>
__device__ __forceinline__ void load_prim(const F5<T> &U, long long e, T gm1, T w[5]) {
  T u[5];
#pragma unroll
  for (int q = 0; q < 5; ++q) u[q] = U.f[q][e];
  con2prim<T>(u, gm1, w);
}

// Threads per CTA: CNT (one per footprint cell), or CNT + 32: a ninth warp
// without an own cell, so that the x and y items of a plane (CW (CW + 2)
// reconstruction positions and CW (CW + 1) faces per direction; FP32: as
// x/y pairs) come to one pair per thread (FP32) or at most two items per
// thread (FP64) -- the phases between barriers end together.  MINB:
// resident CTAs per SM the registers are held to.
template <typename T, int STAGE, int NT, int MINB>
__global__ void __launch_bounds__(NT, MINB) hydro_column_kernel(Geometry g, qk_params p, SC<T> K,
                                                          F5<T> U0, F5<T> U1, F5<T> Uo, DtSrc dts,
                                                          const T *chi) {
  static_assert(NT >= CNT && NT >= CNRING, "one own cell per thread, ring cells on the last");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  ColSmem<T> &sm = *reinterpret_cast<ColSmem<T> *>(smem_raw);
  // the timestep, converted once per CTA
  __shared__ T s_dt;
  if (threadIdx.x == 0) s_dt = (T)dt_of(dts);
  __syncthreads();
  const T dt = s_dt;
  const T gm1 = K.gm1, gamma = K.gamma, gm1inv = K.gm1inv, g1 = K.g1;
  const T *inv_dx = K.inv_dx;
  const F5<T> src = STAGE == 1 ? U0 : U1;
  const int rk = p.recon;
  const int t = threadIdx.x;
  const bool has_own = t < CNT;        // threads CNT.. (the ninth warp) own no cell
  const int ti = t % CW, tj = t / CW;  // own cell in the footprint
  const int rt = t - (NT - CNRING);    // ring cells go to the last CNRING threads

  for (int w = blockIdx.x; w < g.ncols; w += gridDim.x) {
    const Column col = g.cols[w];
    const DevBox b = g.boxes[col.box];
    const int vx = min(CW, b.n[0] - col.x0), vy = min(CW, b.n[1] - col.y0);
    const long long plane = (long long)b.sx * b.sy;
    // own cell: its primitives feed the ring of valid neighbours up to HALO
    // cells beyond the valid footprint (the patch's ghost cells)
    const bool own_load = has_own && ti < vx + HALO && tj < vy + HALO;
    const bool own_valid = has_own && ti < vx && tj < vy;
    const long long own0 = has_own ? cell_elem(b, g.ng, col.x0 + ti, col.y0 + tj, 0) : 0;
    // ring cell of this thread (x sides first, then y sides), if any
    int ri = 0, rj = 0;
    bool ring = false;
    if (rt >= 0) {
      const int side = rt / (HALO * CW), r = rt % (HALO * CW);
      const int h = r % HALO, along = r / HALO;
      if (side == 0) { ri = h - HALO; rj = along; }
      else if (side == 1) { ri = CW + h; rj = along; }
      else if (side == 2) { ri = along; rj = h - HALO; }
      else { ri = along; rj = CW + h; }
      // needed where a valid stencil reaches it: rows (columns) of the valid
      // footprint, and on the far sides only the cells within HALO of the
      // valid extent (the rest lies beyond the patch ghosts; for a partial
      // footprint the own cells past the valid extent supply the near ones)
      ring = (side == 0 && rj < vy) || (side == 1 && ri < vx + HALO && rj < vy) ||
             (side == 2 && ri < vx) || (side == 3 && rj < vy + HALO && ri < vx);
    }
    const long long ring0 = ring ? cell_elem(b, g.ng, col.x0 + ri, col.y0 + rj, 0) : 0;

    // z window: primitives of planes z-1 .. z+3 of the own cell
    T win[5][5];
    auto load_plane = [&](int z, T out[5]) {
      if (own_load) {
        load_prim<T>(src, own0 + (long long)z * plane, gm1, out);
      } else {
#pragma unroll
        for (int q = 0; q < 5; ++q) out[q] = (q == 0 || q == 4) ? T(1) : T(0);
      }
    };
    auto chi_at = [&](int z) -> T {
      return (chi && own_load) ? chi[own0 + (long long)z * plane] : T(1);
    };
    // reconstruct the own cell at plane z from the five planes st[0..4]
    // (FP32: the primitives in pairs (rho, v_x), (v_y, v_z) as the lanes of
    // packed arithmetic, P alone)
    auto recon_z = [&](const T st[5][5], T ch, T qL[5], T qR[5]) {
      constexpr int q0 = sizeof(T) == 4 ? 4 : 0;
      if constexpr (sizeof(T) == 4) {
#pragma unroll
        for (int q = 0; q < 4; q += 2) {
          f2 s2[5];
#pragma unroll
          for (int o = 0; o < 5; ++o) s2[o] = make_float2(st[o][q], st[o][q + 1]);
          f2 l2, r2;
          recon2(rk, s2[0], s2[1], s2[2], s2[3], s2[4], l2, r2);
          qL[q] = l2.x;
          qL[q + 1] = l2.y;
          qR[q] = r2.x;
          qR[q + 1] = r2.y;
        }
      }
#pragma unroll
      for (int q = q0; q < 5; ++q)
        recon<T>(rk, st[0][q], st[1][q], st[2][q], st[3][q], st[4][q], qL[q], qR[q]);
      if (chi) {
#pragma unroll
        for (int q = 0; q < 5; ++q) {
          qL[q] = ch * qL[q] + (T(1) - ch) * st[2][q];
          qR[q] = ch * qR[q] + (T(1) - ch) * st[2][q];
        }
      }
    };
    // start-up: face z0 - 1/2 from the reconstructions of cells z0-1 and z0
    T carryR[5], Fz[5];
    if (has_own) {
      T st[5][5];
#pragma unroll
      for (int o = 0; o < 5; ++o) load_plane(col.z0 - 3 + o, st[o]);
      T qL[5], qR[5];
      recon_z(st, chi_at(col.z0 - 1), qL, qR);
#pragma unroll
      for (int q = 0; q < 5; ++q) carryR[q] = qR[q];
#pragma unroll
      for (int o = 0; o < 4; ++o)
#pragma unroll
        for (int q = 0; q < 5; ++q) st[o][q] = st[o + 1][q];
      load_plane(col.z0 + 2, st[4]);
      recon_z(st, chi_at(col.z0), qL, qR);
      col_face<T, 2>(carryR, qL, gamma, gm1inv, g1, Fz);
#pragma unroll
      for (int q = 0; q < 5; ++q) carryR[q] = qR[q];
#pragma unroll
      for (int o = 0; o < 4; ++o)
#pragma unroll
        for (int q = 0; q < 5; ++q) win[o][q] = st[o + 1][q];  // planes z0-1 .. z0+2
    }

    // the conserved values of the next plane to enter (own: z+3, ring: z),
    // loaded one plane ahead so that their latency overlaps the work on the
    // current plane: FP32 into shared memory by per-thread cp.async (each
    // thread reads back only what it staged, after its own wait; no register
    // is held across the plane), FP64 into registers
    constexpr bool kStage = ColSmem<T>::kPre;
    T nown[5], nring[5];
    // (FP32: every call commits one group, empty past the column's last
    // plane, so that the waits below can count groups)
    auto fetch = [&](int z) {
      const bool any = z < col.z1;
      if constexpr (kStage) {
        if (any && own_load) {
#pragma unroll
          for (int q = 0; q < 5; ++q)
            cp_async_elem(&sm.nxt[q][t], src.f[q] + own0 + (long long)(z + 3) * plane);
        }
        if (any && ring) {
#pragma unroll
          for (int q = 0; q < 5; ++q)
            cp_async_elem(&sm.nxt[q][CNT + rt], src.f[q] + ring0 + (long long)z * plane);
        }
        cp_async_commit();
      } else if (any) {
#pragma unroll
        for (int q = 0; q < 5; ++q) {
          nown[q] = own_load ? src.f[q][own0 + (long long)(z + 3) * plane] : T(1);
          nring[q] = ring ? src.f[q][ring0 + (long long)z * plane] : T(1);
        }
      }
    };
    // plane zp enters: zp+3 into the own window (which holds zp-1 .. zp+2),
    // plane zp of the own cell and of the ring cells into smem (FP32: from the
    // staged values, after the thread's own wait)
    auto enter = [&](int zp) {
      if constexpr (kStage) {
#pragma unroll
        for (int q = 0; q < 5; ++q) {
          nown[q] = own_load ? sm.nxt[q][t] : T(1);
          nring[q] = ring ? sm.nxt[q][CNT + (ring ? rt : 0)] : T(1);
        }
      }
      if (own_load) {
        con2prim<T>(nown, gm1, win[4]);
#pragma unroll
        for (int q = 0; q < 5; ++q) sm.prim[q][pslot(ti, tj)] = win[1][q];
      } else if (has_own) {
#pragma unroll
        for (int q = 0; q < 5; ++q) win[4][q] = (q == 0 || q == 4) ? T(1) : T(0);
      }
      if (ring) {
        T wr[5];
        con2prim<T>(nring, gm1, wr);
#pragma unroll
        for (int q = 0; q < 5; ++q) sm.prim[q][pslot(ri, rj)] = wr[q];
      }
    };
    // Two barriers per plane: the x/y reconstruction and the z face of
    // plane z; then the x/y faces of plane z with plane z+1 entering the
    // primitives (no face reads them); then the epilogue of plane z.
    fetch(col.z0);
    if constexpr (kStage) cp_async_wait_all();
    enter(col.z0);
    fetch(col.z0 + 1);
    __syncthreads();
    for (int z = col.z0; z < col.z1; ++z) {
      if constexpr (ColSmem<T>::kPre) {
        // the epilogue's own-cell inputs, in flight during the two phases
        if (own_valid) {
          const long long e = own0 + (long long)z * plane;
#pragma unroll
          for (int q = 0; q < 5; ++q) cp_async_elem(&sm.pre[q][t], src.f[q] + e);
          if constexpr (STAGE == 2) {
#pragma unroll
            for (int q = 0; q < 5; ++q) cp_async_elem(&sm.pre[5 + q][t], U0.f[q] + e);
          }
        }
        cp_async_commit();
      }
      // ---- x and y reconstruction (items t, t + NT, ...), and z in registers
      if constexpr (sizeof(T) == 4) {
        // FP32: position r of the x rows and position r of the y columns as
        // the two lanes of packed arithmetic (qk_pair.cuh); both lanes' reads
        // lie in the plane for every r < CXPOS CW, and a lane whose position
        // is not needed writes a slot that no face reads.  Each thread takes
        // position t with all five primitives; the positions past NT (32 of
        // them at NT = CNT) go one primitive per warp to the first five warps,
        // so that no warp reconstructs two whole positions while the others
        // wait at the barrier.
        constexpr int NREC = CXPOS * CW;
        constexpr int NXR = NREC > NT ? NREC - NT : 0;
        static_assert(NXR <= 32, "the extra positions fit one warp per primitive");
        // primitive q of pair item r (ch: the flattening coefficients of its
        // two cells)
        auto item_ok = [&](int r, bool &okx, bool &oky) {
          const int cjx = r / CXPOS, cix = r % CXPOS - 1;
          const int ciy = r % CW, cjy = r / CW - 1;
          okx = cjx < vy && cix <= vx;
          oky = ciy < vx && cjy <= vy;
          return okx || oky;
        };
        auto item_chi = [&](int r, bool okx, bool oky) {
          f2 ch = p2(1.0f);
          if (chi) {
            const int cjx = r / CXPOS, cix = r % CXPOS - 1;
            const int ciy = r % CW, cjy = r / CW - 1;
            if (okx) ch.x = chi[cell_elem(b, g.ng, col.x0 + cix, col.y0 + cjx, z)];
            if (oky) ch.y = chi[cell_elem(b, g.ng, col.x0 + ciy, col.y0 + cjy, z)];
          }
          return ch;
        };
        auto recon_xy = [&](int r, int q, f2 ch) {
          const int cjx = r / CXPOS, cix = r % CXPOS - 1;
          const int ciy = r % CW, cjy = r / CW - 1;
          const int bx = pslot(cix - 2, cjx), by = pslot(ciy, cjy - 2);
          const float *pq = sm.prim[q];
          f2 st[5];
#pragma unroll
          for (int o = 0; o < 5; ++o) st[o] = make_float2(pq[bx + o], pq[by + o * CPW]);
          f2 qL, qR;
          recon2(rk, st[0], st[1], st[2], st[3], st[4], qL, qR);
          if (chi) {
            const f2 oc = sub2(p2(1.0f), ch);
            qL = fma2(ch, qL, mul2(oc, st[2]));
            qR = fma2(ch, qR, mul2(oc, st[2]));
          }
          sm.rec[0][2 * q][r] = qL.x;
          sm.rec[0][2 * q + 1][r] = qR.x;
          sm.rec[1][2 * q][r] = qL.y;
          sm.rec[1][2 * q + 1][r] = qR.y;
        };
        {
          bool okx, oky;
          if (t < NREC && item_ok(t, okx, oky)) {
            const f2 ch = item_chi(t, okx, oky);
#pragma unroll
            for (int q = 0; q < 5; ++q) recon_xy(t, q, ch);
          }
        }
        if constexpr (NXR > 0) {
          const int lane = t & 31, q = t >> 5;
          bool okx, oky;
          if (q < 5 && lane < NXR && item_ok(NT + lane, okx, oky))
            recon_xy(NT + lane, q, item_chi(NT + lane, okx, oky));
        }
      } else {
        for (int it = t; it < 2 * CXPOS * CW; it += NT) {
          const int dir = it >= CXPOS * CW;
          const int r = it - dir * CXPOS * CW;
          int ci, cj, base, stride;
          if (!dir) {
            const int pos = r % CXPOS;
            cj = r / CXPOS;
            ci = pos - 1;
            if (cj >= vy || ci > vx) continue;
            base = pslot(ci - 2, cj);
            stride = 1;
          } else {
            ci = r % CW;
            const int pos = r / CW;
            cj = pos - 1;
            if (ci >= vx || cj > vy) continue;
            base = pslot(ci, cj - 2);
            stride = CPW;
          }
          const T ch = chi ? chi[cell_elem(b, g.ng, col.x0 + ci, col.y0 + cj, z)] : T(1);
#pragma unroll
          for (int q = 0; q < 5; ++q) {
            const T *pq = sm.prim[q] + base;
            T qL, qR;
            recon<T>(rk, pq[0], pq[stride], pq[2 * stride], pq[3 * stride], pq[4 * stride], qL,
                     qR);
            if (chi) {
              const T qc = pq[2 * stride];
              qL = ch * qL + (T(1) - ch) * qc;
              qR = ch * qR + (T(1) - ch) * qc;
            }
            sm.rec[dir][2 * q][r] = qL;
            sm.rec[dir][2 * q + 1][r] = qR;
          }
        }
      }
      T Fzn[5];
      if (has_own) {
        T qL[5], qR[5];
        recon_z(win, chi_at(z + 1), qL, qR);
        col_face<T, 2>(carryR, qL, gamma, gm1inv, g1, Fzn);
#pragma unroll
        for (int q = 0; q < 5; ++q) carryR[q] = qR[q];
      }
      __syncthreads();
      // ---- x and y faces
      if constexpr (sizeof(T) == 4) {
        // FP32: face r of the x rows and face r of the y columns as the two
        // lanes of hllc2, each in its own frame (rho, u_n, u_t1, u_t2, P):
        // x (rho, vx, vy, vz, P), y (rho, vy, vz, vx, P).  Each thread takes
        // pair t; the pairs past NT (16 of them at NT = CNT) go as single
        // faces, x and y on separate lanes, to the first warp (which enters
        // no ring cell below), so that its extra round costs one face per
        // lane rather than a pair.
        constexpr int NFP = CXFACE * CW;
        constexpr int NXF = NFP > NT ? NFP - NT : 0;
        static_assert(2 * NXF <= 32, "the extra faces fit one warp");
        constexpr int qy[5] = {0, 2, 3, 1, 4};
        if (t < NFP) {
          const int r = t;
          const int fx = r % CXFACE, cjx = r / CXFACE;
          const int ciy = r % CW, fy = r / CW;
          const bool okx = cjx < vy && fx <= vx, oky = ciy < vx && fy <= vy;
          if (okx || oky) {
            const int ilx = cjx * CXPOS + fx, ily = fy * CW + ciy;
            f2 wL[5], wR[5], F[5];
#pragma unroll
            for (int k = 0; k < 5; ++k) {
              wL[k] = make_float2(sm.rec[0][2 * k + 1][ilx], sm.rec[1][2 * qy[k] + 1][ily]);
              wR[k] = make_float2(sm.rec[0][2 * k][ilx + 1], sm.rec[1][2 * qy[k]][ily + CW]);
            }
            hllc2(wL, wR, gamma, gm1inv, g1, F);
#pragma unroll
            for (int k = 0; k < 5; ++k) {
              sm.flux[0][k][r] = F[k].x;
              sm.flux[1][qy[k]][r] = F[k].y;
            }
          }
        }
        if constexpr (NXF > 0) {
          if (t < 2 * NXF) {
            const int dir = t / NXF, r = NT + t % NXF;
            int il, step;
            bool ok;
            if (dir == 0) {
              const int fx = r % CXFACE, cjx = r / CXFACE;
              ok = cjx < vy && fx <= vx;
              il = cjx * CXPOS + fx;
              step = 1;
            } else {
              const int ciy = r % CW, fy = r / CW;
              ok = ciy < vx && fy <= vy;
              il = fy * CW + ciy;
              step = CW;
            }
            if (ok) {
              float wL[5], wR[5], F[5];
#pragma unroll
              for (int k = 0; k < 5; ++k) {
                const int qk = dir ? qy[k] : k;
                wL[k] = sm.rec[dir][2 * qk + 1][il];
                wR[k] = sm.rec[dir][2 * qk][il + step];
              }
              hllc2(wL, wR, gamma, gm1inv, g1, F);
#pragma unroll
              for (int k = 0; k < 5; ++k) sm.flux[dir][dir ? qy[k] : k][r] = F[k];
            }
          }
        }
      } else {
        for (int it = t; it < 2 * CXFACE * CW; it += NT) {
          const int dir = it >= CXFACE * CW;
          const int r = it - dir * CXFACE * CW;
          int il, ir;
          if (!dir) {
            const int f = r % CXFACE, cj = r / CXFACE;
            if (cj >= vy || f > vx) continue;
            il = cj * CXPOS + f;
            ir = il + 1;
          } else {
            const int ci = r % CW, f = r / CW;
            if (ci >= vx || f > vy) continue;
            il = f * CW + ci;
            ir = il + CW;
          }
          T wL[5], wR[5], F[5];
#pragma unroll
          for (int q = 0; q < 5; ++q) {
            wL[q] = sm.rec[dir][2 * q + 1][il];
            wR[q] = sm.rec[dir][2 * q][ir];
          }
          if (!dir)
            col_face<T, 0>(wL, wR, gamma, gm1inv, g1, F);
          else
            col_face<T, 1>(wL, wR, gamma, gm1inv, g1, F);
#pragma unroll
          for (int q = 0; q < 5; ++q) sm.flux[dir][q][r] = F[q];
        }
      }
      // ---- plane z+1 enters (the window first moves on to planes z .. z+3)
      if (has_own) {
#pragma unroll
        for (int o = 0; o < 4; ++o)
#pragma unroll
          for (int q = 0; q < 5; ++q) win[o][q] = win[o + 1][q];
      }
      if (z + 1 < col.z1) {
        // its staged values: the group before the most recent one
        if constexpr (kStage) cp_async_wait_group<1>();
        enter(z + 1);
      }
      fetch(z + 2);
      __syncthreads();
      // ---- divergence ((x + y) + z) and the RK combination of the own cell
      if (own_valid) {
        const long long e = own0 + (long long)z * plane;
        const int fx = tj * CXFACE + ti, fy = tj * CW + ti;
        constexpr bool kPre = ColSmem<T>::kPre;
        // its own-cell inputs: the group before the most recent one
        if constexpr (kPre) cp_async_wait_group<1>();
#pragma unroll
        for (int q = 0; q < 5; ++q) {
          T acc = (sm.flux[0][q][fx + 1] - sm.flux[0][q][fx]) * inv_dx[0];
          acc = acc + (sm.flux[1][q][fy + CW] - sm.flux[1][q][fy]) * inv_dx[1];
          acc = acc + (Fzn[q] - Fz[q]) * inv_dx[2];
          const T L = -acc;
          const T own = kPre ? sm.pre[kPre ? q : 0][kPre ? t : 0] : src.f[q][e];
          if (STAGE == 1) {
            Uo.f[q][e] = own + dt * L;
          } else {
            const T u0 = kPre ? sm.pre[kPre ? 5 + q : 0][kPre ? t : 0] : U0.f[q][e];
            Uo.f[q][e] = T(0.5) * u0 + T(0.5) * (own + dt * L);
          }
        }
      }
      if (has_own) {
#pragma unroll
        for (int q = 0; q < 5; ++q) Fz[q] = Fzn[q];
      }
      // the next plane's reconstruction rewrites rec (last read before the
      // barrier above); its faces rewrite flux after the next barrier
    }
    if constexpr (kStage) cp_async_wait_all();
    __syncthreads();
  }
}

template <typename T, int STAGE, int NT, int MINB>
static cudaError_t launch_col(const Geometry &g, const qk_params &p, void *const *U0,
                              void *const *U1, void *const *Uo, DtSrc dt, const void *chi,
                              cudaStream_t s) {
  F5<T> a, b, c;
  for (int q = 0; q < 5; ++q) {
    a.f[q] = (T *)U0[q];
    b.f[q] = U1 ? (T *)U1[q] : nullptr;
    c.f[q] = (T *)Uo[q];
  }
  const int smem = (int)sizeof(ColSmem<T>);
  auto kern = hydro_column_kernel<T, STAGE, NT, MINB>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0, nsm = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT, smem);
  int grid = nsm * (per_sm > 0 ? per_sm : 1);
  if (grid > g.ncols) grid = g.ncols;
  if (grid < 1) return cudaSuccess;
  kern<<<grid, NT, smem, s>>>(g, p, make_sc<T>(p), a, b, c, dt, (const T *)chi);
  return cudaGetLastError();
}

template <int STAGE>
static cudaError_t launch_col_f32(int cfg, const Geometry &g, const qk_params &p, void *const *U0,
                                  void *const *U1, void *const *Uo, DtSrc dt, const void *chi,
                                  cudaStream_t s) {
  // the column configurations: CNT threads at COL_CTAS_FP32 per SM, or
  // CNT + 32 threads at 3 (schedule 0) or 2 (schedule 1) per SM
  if (cfg_threads(cfg) == CNT + 32)
    return cfg_sched(cfg) ? launch_col<float, STAGE, CNT + 32, 2>(g, p, U0, U1, Uo, dt, chi, s)
                          : launch_col<float, STAGE, CNT + 32, 3>(g, p, U0, U1, Uo, dt, chi, s);
  return launch_col<float, STAGE, CNT, COL_CTAS_FP32>(g, p, U0, U1, Uo, dt, chi, s);
}

cudaError_t launch_hydro_column(int fp32, int stage, const Geometry &g, const qk_params &p,
                                void *const *U0, void *const *U1, void *const *Uout, DtSrc dt,
                                const void *chi, cudaStream_t s, int cfg) {
  if (fp32)
    return stage == 1 ? launch_col_f32<1>(cfg, g, p, U0, U1, Uout, dt, chi, s)
                      : launch_col_f32<2>(cfg, g, p, U0, U1, Uout, dt, chi, s);
  // FP64: one configuration (CNT threads, COL_CTAS_FP64 per SM)
  return stage == 1 ? launch_col<double, 1, CNT, COL_CTAS_FP64>(g, p, U0, U1, Uout, dt, chi, s)
                    : launch_col<double, 2, CNT, COL_CTAS_FP64>(g, p, U0, U1, Uout, dt, chi, s);
}

}  // namespace qk
