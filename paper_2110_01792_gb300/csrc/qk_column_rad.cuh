// qk_column_rad.cuh -- plane-marching form of the fused radiation RK2-SSP stage
// (Sec. 2.2.2 of arXiv:2110.01792), with the matter-radiation exchange
// optionally fused per cell (Sec. 2.2.3, stage 2): the same per-cell and
// per-face arithmetic as qk_rad.cuh (f = F/(c E_r), the closure, PPM/PLM, the
// |f| > 1 fallback, the HLL wavespeed from the cell-average Eddington factors,
// the optical-depth correction, the divergence ((x + y) + z), the RK
// combination), organised as the hydro column kernel (qk_column.cu): a CTA of
// CW x CW threads walks the planes of a CW x CW footprint along z, the z
// stencil in a per-thread register window, x and y on one shared-memory plane
// with a HALO-deep ring.
#pragma once
#include "qk_rad.cuh"
#include "qk_pair.cuh"

namespace qk {

template <typename T> struct ColRadSmem {
  static constexpr bool kAB = sizeof(T) == 8;
  T prim[4][CNPL];                   // E_r, f_x, f_y, f_z of plane z and its ring
  T rk[CNPL];                        // rho kappa_R
  T ab[2][kAB ? CNPL : 1];           // FP64: closure a, b of the cell average
  T rec[2][8][CXPOS * CW];           // x and y: qL, qR per position
  T sq[2][kAB ? 1 : CXPOS * CW];     // FP32: sqrt(T_DD) of the cell average per position
  T flux[2][4][CXFACE * CW];
  // FP32: the own cell's values read by the epilogue, staged one phase ahead
  // (cp.async): R_src (4), R_0 (4, stage 2), the gas state U (5, exchange)
  static constexpr int kPre = kAB ? 1 : 13;
  T pre[kPre][kAB ? 1 : CNT];
  // FP32: E_r, F and rho of the next plane to enter (own cells, then ring
  // cells), staged one plane ahead (cp.async)
  T nxt[kAB ? 1 : 5][kAB ? 1 : CNT + CNRING];
};

__device__ __forceinline__ int cslot(int i, int j) { return (j + HALO) * CPW + (i + HALO); }

// E_r, f = F/(c E_r) and rho kappa_R of one cell from its conserved values.
template <typename T>
__device__ __forceinline__ void rad_prim(const T u[4], T c, T r, const SC<T> &K, T w[4], T &rk) {
  const T inv = qrcp(c * u[0]);
  w[0] = u[0];
  w[1] = u[1] * inv;
  w[2] = u[2] * inv;
  w[3] = u[3] * inv;
  rk = rho_kappa<T>(K, r);
}

template <typename T> struct ColMinBlocksRad {
  static constexpr int value = sizeof(T) == 4 ? COL_CTAS_FP32 : COL_CTAS_FP64;
};

// NT threads per CTA: CNT (one per footprint cell) or, FP32, CNT + 32 (a
// ninth warp without an own cell, so that a plane's x/y pairs come to one per
// thread), registers held to MINB CTAs per SM.
template <typename T, int STAGE, int CL, bool EX, int NT = CNT,
          int MINB = ColMinBlocksRad<T>::value>
__global__ void __launch_bounds__(NT, MINB)
    rad_column_kernel(Geometry g, qk_params p, SC<T> K, F4<T> R0, F4<T> R1, F4<T> Ro,
                      const T *rho, DtSrc dts, ExFuse<T> xf) {
  static_assert(NT >= CNT && NT >= CNRING, "one own cell per thread, ring cells on the last");
  if (skip_substep(dts)) return;
  constexpr bool kAB = ColRadSmem<T>::kAB;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  ColRadSmem<T> &sm = *reinterpret_cast<ColRadSmem<T> *>(smem_raw);
  // the timestep, converted once per CTA
  __shared__ T s_dt;
  if (threadIdx.x == 0) s_dt = (T)dt_of(dts);
  __syncthreads();
  const T dt = s_dt;
  const T c = K.c, chat = K.chat;
  const T *inv_dx = K.inv_dx, *dx = K.dx;
  const T hccc = T(0.5) * c * chat;
  const T hchat_c = T(0.5) * chat / c;
  const F4<T> src = STAGE == 1 ? R0 : R1;
  const int rk = p.recon;
  const int t = threadIdx.x;
  const bool has_own = t < CNT;  // threads CNT.. (a ninth warp) own no cell
  const int ti = t % CW, tj = t / CW;
  ExStat xs;

  for (int w = blockIdx.x; w < g.ncols; w += gridDim.x) {
    const Column col = g.cols[w];
    const DevBox b = g.boxes[col.box];
    const int vx = min(CW, b.n[0] - col.x0), vy = min(CW, b.n[1] - col.y0);
    const long long plane = (long long)b.sx * b.sy;
    const bool own_load = has_own && ti < vx + HALO && tj < vy + HALO;
    const bool own_valid = has_own && ti < vx && tj < vy;
    // the cell-average closure of the own cell is read by faces of valid cells
    const bool own_near = has_own && ti <= vx && tj <= vy;
    const long long own0 = has_own ? cell_elem(b, g.ng, col.x0 + ti, col.y0 + tj, 0) : 0;
    int ri = 0, rj = 0, rside = 0;
    bool ring = false;
    // ring cells go to the last CNRING threads
    const int rt = t - (NT - CNRING);
    if (rt >= 0) {
      rside = rt / (HALO * CW);
      const int r = rt % (HALO * CW), h = r % HALO, along = r / HALO;
      if (rside == 0) { ri = h - HALO; rj = along; }
      else if (rside == 1) { ri = CW + h; rj = along; }
      else if (rside == 2) { ri = along; rj = h - HALO; }
      else { ri = along; rj = CW + h; }
      ring = (rside == 0 && rj < vy) || (rside == 1 && ri < vx + HALO && rj < vy) ||
             (rside == 2 && ri < vx) || (rside == 3 && rj < vy + HALO && ri < vx);
    }
    // ring cells adjacent to the footprint need the cell-average closure
    const bool ring_near = ring && (ri == -1 || rj == -1 || ri == vx || rj == vy);
    const long long ring0 = ring ? cell_elem(b, g.ng, col.x0 + ri, col.y0 + rj, 0) : 0;

    // z window: E_r, f and rho kappa_R of planes z-1 .. z+3 (own cell)
    T win[5][4], rkw[5];
    T az0 = T(0), bz0 = T(0);     // FP64: closure of plane z (carried)
    T sqz0 = T(0);                // FP32: sqrt(T_zz) of plane z (carried)
    auto load_plane = [&](int z, T out[4], T &rko) {
      if (own_load) {
        const long long e = own0 + (long long)z * plane;
        T u[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) u[q] = src.f[q][e];
        rad_prim<T>(u, c, rho[e], K, out, rko);
      } else {
        out[0] = T(1);
        out[1] = out[2] = out[3] = T(0);
        rko = T(0);
      }
    };
    // the z-face quantities of the cell in window slot s: closure (FP64) or
    // sqrt(T_zz) (FP32)
    auto zclosure = [&](const T wq[4], T &a, T &bb, T &sq) {
      if constexpr (kAB) {
        closure_ab<T, CL>(wq[1], wq[2], wq[3], a, bb);
      } else {
        sq = qsqrt(eddington_diag<T, 2, CL>(wq[1], wq[2], wq[3]));
      }
    };
    auto zface = [&](const T wL[4], const T wR[4], const T cL[4], const T cR[4], T aL, T bL,
                     T sqL, T aR, T bR, T sqR, T rka, T rkb, T out[4]) {
      T S;
      if constexpr (kAB) {
        S = rad_speed<T>(aL + bL * cL[3] * cL[3], aR + bR * cR[3] * cR[3], chat);
      } else {
        S = chat * max(sqL, sqR);
      }
      T l[4], r[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        l[q] = wL[q];
        r[q] = wR[q];
      }
      rad_face_hll<T, 2, CL>(
          l, r,
          [&](T *ll, T *rr) {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              ll[q] = cL[q];
              rr[q] = cR[q];
            }
          },
          S, rka, rkb, dx[2], c, chat, hchat_c, hccc, p.tau_correction, out);
    };
    // (FP32: the fields in pairs (E_r, f_x), (f_y, f_z) as the lanes of packed
    // arithmetic)
    auto recon_z = [&](const T st[5][4], T qL[4], T qR[4]) {
      if constexpr (!kAB) {
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
      } else {
#pragma unroll
        for (int q = 0; q < 4; ++q)
          recon<T>(rk, st[0][q], st[1][q], st[2][q], st[3][q], st[4][q], qL[q], qR[q]);
      }
    };

    // start-up: face z0 - 1/2 from cells z0-1 and z0
    T carryR[4], Fz[4];
    if (has_own) {
      T st[5][4], rks[5];
#pragma unroll
      for (int o = 0; o < 5; ++o) load_plane(col.z0 - 3 + o, st[o], rks[o]);
      T qL[4], qR[4];
      recon_z(st, qL, qR);  // cell z0-1
#pragma unroll
      for (int q = 0; q < 4; ++q) carryR[q] = qR[q];
      T am = T(0), bm = T(0), sqm = T(0);
      zclosure(st[2], am, bm, sqm);  // cell z0-1
#pragma unroll
      for (int o = 0; o < 4; ++o) {
        rks[o] = rks[o + 1];
#pragma unroll
        for (int q = 0; q < 4; ++q) st[o][q] = st[o + 1][q];
      }
      load_plane(col.z0 + 2, st[4], rks[4]);
      recon_z(st, qL, qR);  // cell z0
      zclosure(st[2], az0, bz0, sqz0);
      zface(carryR, qL, st[1], st[2], am, bm, sqm, az0, bz0, sqz0, rks[1], rks[2], Fz);
#pragma unroll
      for (int q = 0; q < 4; ++q) carryR[q] = qR[q];
#pragma unroll
      for (int o = 0; o < 4; ++o) {
        rkw[o] = rks[o + 1];
#pragma unroll
        for (int q = 0; q < 4; ++q) win[o][q] = st[o + 1][q];  // planes z0-1 .. z0+2
      }
    }

    // next plane's inputs, fetched one plane ahead: FP32 into shared memory
    // by per-thread cp.async (read back by the same thread after its own
    // wait), FP64 into registers
    const int rslot = CNT + (rt >= 0 ? rt : 0);
    T nown[4], nring[4], nrho_own = T(1), nrho_ring = T(1);
    auto fetch = [&](int z) {
      const long long eo = own0 + (long long)(z + 3) * plane;
      const long long er = ring0 + (long long)z * plane;
      if constexpr (!kAB) {
        if (own_load) {
#pragma unroll
          for (int q = 0; q < 4; ++q) cp_async_elem(&sm.nxt[q][t], src.f[q] + eo);
          cp_async_elem(&sm.nxt[4][t], rho + eo);
        }
        if (ring) {
#pragma unroll
          for (int q = 0; q < 4; ++q) cp_async_elem(&sm.nxt[q][rslot], src.f[q] + er);
          cp_async_elem(&sm.nxt[4][rslot], rho + er);
        }
        cp_async_commit();
      } else {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          nown[q] = own_load ? src.f[q][eo] : T(1);
          nring[q] = ring ? src.f[q][er] : T(1);
        }
        nrho_own = own_load ? rho[eo] : T(1);
        nrho_ring = ring ? rho[er] : T(1);
      }
    };
    fetch(col.z0);
    for (int z = col.z0; z < col.z1; ++z) {
      if constexpr (!kAB) {
        cp_async_wait_all();
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          nown[q] = own_load ? sm.nxt[q][t] : T(1);
          nring[q] = ring ? sm.nxt[q][rslot] : T(1);
        }
        nrho_own = own_load ? sm.nxt[4][t] : T(1);
        nrho_ring = ring ? sm.nxt[4][rslot] : T(1);
      }
      // ---- plane z+3 into the window; plane z (own + ring) into smem
      if (own_load) {
        rad_prim<T>(nown, c, nrho_own, K, win[4], rkw[4]);
        const int s = cslot(ti, tj);
#pragma unroll
        for (int q = 0; q < 4; ++q) sm.prim[q][s] = win[1][q];
        sm.rk[s] = rkw[1];
        if constexpr (kAB) {
          if (own_near) {
            sm.ab[0][s] = az0;
            sm.ab[1][s] = bz0;
          }
        }
      } else if (has_own) {
        win[4][0] = T(1);
        win[4][1] = win[4][2] = win[4][3] = T(0);
        rkw[4] = T(0);
      }
      if (ring) {
        T wr[4], rkr;
        rad_prim<T>(nring, c, nrho_ring, K, wr, rkr);
        const int s = cslot(ri, rj);
#pragma unroll
        for (int q = 0; q < 4; ++q) sm.prim[q][s] = wr[q];
        sm.rk[s] = rkr;
        if constexpr (kAB) {
          if (ring_near) {
            T a, bb;
            closure_ab<T, CL>(wr[1], wr[2], wr[3], a, bb);
            sm.ab[0][s] = a;
            sm.ab[1][s] = bb;
          }
        }
      }
      if (z + 1 < col.z1) fetch(z + 1);
      __syncthreads();
      if constexpr (!kAB) {
        // the epilogue's own-cell inputs, in flight during the two phases
        if (own_valid) {
          const long long e = own0 + (long long)z * plane;
#pragma unroll
          for (int q = 0; q < 4; ++q) cp_async_elem(&sm.pre[q][t], src.f[q] + e);
          if constexpr (STAGE == 2) {
#pragma unroll
            for (int q = 0; q < 4; ++q) cp_async_elem(&sm.pre[4 + q][t], R0.f[q] + e);
          }
          if constexpr (EX) {
#pragma unroll
            for (int q = 0; q < 5; ++q) cp_async_elem(&sm.pre[8 + q][t], xf.U.f[q] + e);
          }
        }
        cp_async_commit();
      }
      // ---- x and y reconstruction; z in registers
      if constexpr (!kAB) {
        // FP32: position r of the x rows and position r of the y columns as
        // the two lanes of packed arithmetic (qk_pair.cuh), with sqrt(T_DD) of
        // each position's cell average (x: T_xx, y: T_yy); every read lies in
        // the plane for r < CXPOS CW, and a lane whose position is not needed
        // writes a slot that no face reads.  Each thread takes position t
        // (four fields and sqrt(T_DD)); the positions past NT (32 of them at
        // NT = CNT) go one field per warp to the first four warps and their
        // sqrt(T_DD) to the fifth, so that no warp takes two whole positions
        // while the others wait at the barrier.
        constexpr int NREC = CXPOS * CW;
        constexpr int NXR = NREC > NT ? NREC - NT : 0;
        static_assert(NXR <= 32, "the extra positions fit one warp per field");
        auto item_ok = [&](int r) {
          const int cjx = r / CXPOS, cix = r % CXPOS - 1;
          const int ciy = r % CW, cjy = r / CW - 1;
          return (cjx < vy && cix <= vx) || (ciy < vx && cjy <= vy);
        };
        auto item_base = [&](int r, int &bx, int &by) {
          const int cjx = r / CXPOS, cix = r % CXPOS - 1;
          const int ciy = r % CW, cjy = r / CW - 1;
          bx = cslot(cix - 2, cjx);
          by = cslot(ciy, cjy - 2);
        };
        // field q of pair item r; returns its cell-average values
        auto recon_xy = [&](int r, int q) -> f2 {
          int bx, by;
          item_base(r, bx, by);
          const float *pq = sm.prim[q];
          f2 st[5];
#pragma unroll
          for (int o = 0; o < 5; ++o) st[o] = make_float2(pq[bx + o], pq[by + o * CPW]);
          f2 qL, qR;
          recon2(rk, st[0], st[1], st[2], st[3], st[4], qL, qR);
          sm.rec[0][2 * q][r] = qL.x;
          sm.rec[0][2 * q + 1][r] = qR.x;
          sm.rec[1][2 * q][r] = qL.y;
          sm.rec[1][2 * q + 1][r] = qR.y;
          return st[2];
        };
        // T_DD = a + b f_D^2 of the cell average of item r, D = x (lane x),
        // y (lane y), from its four fields mid
        auto sq_xy = [&](int r, const f2 mid[4]) {
          const f2 fsq = fma2(mid[3], mid[3], fma2(mid[1], mid[1], mul2(mid[2], mid[2])));
          f2 a, bb;
          closure_ab2<CL>(fsq, a, bb);
          const f2 fD = make_float2(mid[1].x, mid[2].y);
          const f2 Tdd = fma2(mul2(bb, fD), fD, a);
          sm.sq[0][r] = qsqrt(Tdd.x);
          sm.sq[1][r] = qsqrt(Tdd.y);
        };
        if (t < NREC && item_ok(t)) {
          f2 mid[4];
#pragma unroll
          for (int q = 0; q < 4; ++q) mid[q] = recon_xy(t, q);
          sq_xy(t, mid);
        }
        if constexpr (NXR > 0) {
          const int lane = t & 31, q = t >> 5, r = NT + lane;
          if (q < 5 && lane < NXR && item_ok(r)) {
            if (q < 4) {
              recon_xy(r, q);
            } else {
              int bx, by;
              item_base(r, bx, by);
              f2 mid[4];
#pragma unroll
              for (int k = 0; k < 4; ++k)
                mid[k] = make_float2(sm.prim[k][bx + 2], sm.prim[k][by + 2 * CPW]);
              sq_xy(r, mid);
            }
          }
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
            base = cslot(ci - 2, cj);
            stride = 1;
          } else {
            ci = r % CW;
            const int pos = r / CW;
            cj = pos - 1;
            if (ci >= vx || cj > vy) continue;
            base = cslot(ci, cj - 2);
            stride = CPW;
          }
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const T *pq = sm.prim[q] + base;
            T qL, qR;
            recon<T>(rk, pq[0], pq[stride], pq[2 * stride], pq[3 * stride], pq[4 * stride], qL,
                     qR);
            sm.rec[dir][2 * q][r] = qL;
            sm.rec[dir][2 * q + 1][r] = qR;
          }
        }
      }
      T Fzn[4];
      T az1 = T(0), bz1 = T(0), sqz1 = T(0);
      if (has_own) {
        T qL[4], qR[4];
        recon_z(win, qL, qR);  // cell z+1
        zclosure(win[2], az1, bz1, sqz1);
        zface(carryR, qL, win[1], win[2], az0, bz0, sqz0, az1, bz1, sqz1, rkw[1], rkw[2], Fzn);
#pragma unroll
        for (int q = 0; q < 4; ++q) carryR[q] = qR[q];
      }
      __syncthreads();
      // ---- x and y faces
      if constexpr (!kAB) {
        // FP32: face r of the x rows and face r of the y columns as the two
        // lanes of rad_face_hll2, each in its own frame (E_r, f_n, f_t1,
        // f_t2): x (E_r, f_x, f_y, f_z), y (E_r, f_y, f_z, f_x).  Each thread
        // takes pair t; the pairs past NT (16 of them at NT = CNT) go as
        // single faces, x and y on separate lanes, to the last warp, so that
        // its extra round costs one face per lane rather than a pair.
        constexpr int NFP = CXFACE * CW;
        constexpr int NXF = NFP > NT ? NFP - NT : 0;
        static_assert(2 * NXF <= 32, "the extra faces fit one warp");
        constexpr int qy[4] = {0, 2, 3, 1};
        if (t < NFP) {
          const int r = t;
          const int fx = r % CXFACE, cjx = r / CXFACE;
          const int ciy = r % CW, fy = r / CW;
          const bool okx = cjx < vy && fx <= vx, oky = ciy < vx && fy <= vy;
          if (okx || oky) {
            const int ilx = cjx * CXPOS + fx, ily = fy * CW + ciy;
            const int sax = cslot(fx - 1, cjx), say = cslot(ciy, fy - 1);
            f2 wL[4], wR[4], out[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
              wL[k] = make_float2(sm.rec[0][2 * k + 1][ilx], sm.rec[1][2 * qy[k] + 1][ily]);
              wR[k] = make_float2(sm.rec[0][2 * k][ilx + 1], sm.rec[1][2 * qy[k]][ily + CW]);
            }
            auto averages = [&](f2 *avL, f2 *avR) {
#pragma unroll
              for (int k = 0; k < 4; ++k) {
                avL[k] = make_float2(sm.prim[k][sax], sm.prim[qy[k]][say]);
                avR[k] = make_float2(sm.prim[k][sax + 1], sm.prim[qy[k]][say + CPW]);
              }
            };
            const f2 S = mul2(p2(chat), make_float2(fmaxf(sm.sq[0][ilx], sm.sq[0][ilx + 1]),
                                                    fmaxf(sm.sq[1][ily], sm.sq[1][ily + CW])));
            const f2 rka = make_float2(sm.rk[sax], sm.rk[say]);
            const f2 rkb = make_float2(sm.rk[sax + 1], sm.rk[say + CPW]);
            rad_face_hll2<CL>(wL, wR, averages, S, rka, rkb, make_float2(dx[0], dx[1]), c, chat,
                              hchat_c, hccc, p.tau_correction, out);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
              sm.flux[0][k][r] = out[k].x;
              sm.flux[1][qy[k]][r] = out[k].y;
            }
          }
        }
        if constexpr (NXF > 0) {
          const int lane = t - (NT - 32);
          if (lane >= 0 && lane < 2 * NXF) {
            const int dir = lane / NXF, r = NT + lane % NXF;
            int il, step, sa, sstep;
            bool ok;
            if (dir == 0) {
              const int fx = r % CXFACE, cjx = r / CXFACE;
              ok = cjx < vy && fx <= vx;
              il = cjx * CXPOS + fx;
              step = 1;
              sa = cslot(fx - 1, cjx);
              sstep = 1;
            } else {
              const int ciy = r % CW, fy = r / CW;
              ok = ciy < vx && fy <= vy;
              il = fy * CW + ciy;
              step = CW;
              sa = cslot(ciy, fy - 1);
              sstep = CPW;
            }
            if (ok) {
              float wL[4], wR[4], out[4];
#pragma unroll
              for (int k = 0; k < 4; ++k) {
                const int qk = dir ? qy[k] : k;
                wL[k] = sm.rec[dir][2 * qk + 1][il];
                wR[k] = sm.rec[dir][2 * qk][il + step];
              }
              auto averages = [&](float *avL, float *avR) {
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                  const int qk = dir ? qy[k] : k;
                  avL[k] = sm.prim[qk][sa];
                  avR[k] = sm.prim[qk][sa + sstep];
                }
              };
              const float S = __fmul_rn(chat, fmaxf(sm.sq[dir][il], sm.sq[dir][il + step]));
              rad_face_hll2<CL>(wL, wR, averages, S, sm.rk[sa], sm.rk[sa + sstep],
                                dir ? dx[1] : dx[0], c, chat, hchat_c, hccc, p.tau_correction,
                                out);
#pragma unroll
              for (int k = 0; k < 4; ++k) sm.flux[dir][dir ? qy[k] : k][r] = out[k];
            }
          }
        }
      } else {
        for (int it = t; it < 2 * CXFACE * CW; it += NT) {
          const int dir = it >= CXFACE * CW;
          const int r = it - dir * CXFACE * CW;
          int il, ir, sa, sb;
          if (!dir) {
            const int f = r % CXFACE, cj = r / CXFACE;
            if (cj >= vy || f > vx) continue;
            il = cj * CXPOS + f;
            ir = il + 1;
            sa = cslot(f - 1, cj);
            sb = sa + 1;
          } else {
            const int ci = r % CW, f = r / CW;
            if (ci >= vx || f > vy) continue;
            il = f * CW + ci;
            ir = il + CW;
            sa = cslot(ci, f - 1);
            sb = sa + CPW;
          }
          T wL[4], wR[4], out[4];
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            wL[q] = sm.rec[dir][2 * q + 1][il];
            wR[q] = sm.rec[dir][2 * q][ir];
          }
          auto fallback = [&](T *l, T *r2) {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              l[q] = sm.prim[q][sa];
              r2[q] = sm.prim[q][sb];
            }
          };
          const T fa = sm.prim[1 + dir][sa], fb = sm.prim[1 + dir][sb];
          const T S = rad_speed<T>(sm.ab[0][sa] + sm.ab[1][sa] * fa * fa,
                                   sm.ab[0][sb] + sm.ab[1][sb] * fb * fb, chat);
          if (!dir)
            rad_face_hll<T, 0, CL>(wL, wR, fallback, S, sm.rk[sa], sm.rk[sb], dx[0], c, chat,
                                   hchat_c, hccc, p.tau_correction, out);
          else
            rad_face_hll<T, 1, CL>(wL, wR, fallback, S, sm.rk[sa], sm.rk[sb], dx[1], c, chat,
                                   hchat_c, hccc, p.tau_correction, out);
#pragma unroll
          for (int q = 0; q < 4; ++q) sm.flux[dir][q][r] = out[q];
        }
      }
      __syncthreads();
      // ---- divergence ((x + y) + z), RK combination, optional exchange
      if (own_valid) {
        const long long e = own0 + (long long)z * plane;
        const int fx = tj * CXFACE + ti, fy = tj * CW + ti;
        if constexpr (!kAB) cp_async_wait_all();
        T rv[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          T acc = (sm.flux[0][q][fx + 1] - sm.flux[0][q][fx]) * inv_dx[0];
          acc = acc + (sm.flux[1][q][fy + CW] - sm.flux[1][q][fy]) * inv_dx[1];
          acc = acc + (Fzn[q] - Fz[q]) * inv_dx[2];
          const T L = -acc;
          const T own = kAB ? src.f[q][e] : sm.pre[kAB ? 0 : q][kAB ? 0 : t];
          if (STAGE == 1) {
            rv[q] = own + dt * L;
          } else {
            const T u0 = kAB ? R0.f[q][e] : sm.pre[kAB ? 0 : 4 + q][kAB ? 0 : t];
            rv[q] = T(0.5) * u0 + T(0.5) * (own + dt * L);
          }
          Ro.f[q][e] = rv[q];
        }
        if constexpr (EX) {
          if constexpr (kAB) {
            const double fr[3] = {(double)rv[1], (double)rv[2], (double)rv[3]};
            exchange_cell<T>(p, xf.K, dt_of(dts), xf.U, Ro, xf.src, e, (double)rv[0], fr, xs);
          } else {
            const float fl[3] = {0.0f, 0.0f, 0.0f};
            F4<float> none{};
            exchange_cell_mixed<0>(p, xf.K, dt_of(dts), dt, xf.U, Ro, xf.UL, none, xf.src, e,
                                       rv[0], 0.0f, rv + 1, fl, xs, &sm.pre[8][t], CNT);
          }
        }
      }
      if (has_own) {
#pragma unroll
        for (int q = 0; q < 4; ++q) Fz[q] = Fzn[q];
#pragma unroll
        for (int o = 0; o < 4; ++o) {
          rkw[o] = rkw[o + 1];
#pragma unroll
          for (int q = 0; q < 4; ++q) win[o][q] = win[o + 1][q];
        }
        az0 = az1;
        bz0 = bz1;
        sqz0 = sqz1;
      }
    }
    __syncthreads();
  }
  if constexpr (EX) exchange_status(xf.st, xs.max, xs.flags, xs.bad);
}

template <typename T, int STAGE, int CL, bool EX, int NT = CNT,
          int MINB = ColMinBlocksRad<T>::value>
static cudaError_t launch_rad_col_one(const Geometry &g, const qk_params &p, void *const *R0,
                                      void *const *R1, void *const *Ro, const void *rho,
                                      DtSrc dt, const FuseArgs *fx, cudaStream_t s) {
  F4<T> a, b, c;
  for (int q = 0; q < 4; ++q) {
    a.f[q] = (T *)R0[q];
    b.f[q] = R1 ? (T *)R1[q] : nullptr;
    c.f[q] = (T *)Ro[q];
  }
  ExFuse<T> xf{};
  if (EX) {
    for (int q = 0; q < 5; ++q) xf.U.f[q] = (T *)fx->U[q];
    xf.src = (const T *)fx->src;
    xf.st = fx->st;
    xf.K = make_exk(p);
    xf.on = 1;
  }
  const int smem = (int)sizeof(ColRadSmem<T>);
  auto kern = rad_column_kernel<T, STAGE, CL, EX, NT, MINB>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0, nsm = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT, smem);
  int grid = nsm * (per_sm > 0 ? per_sm : 1);
  if (grid > g.ncols) grid = g.ncols;
  if (grid < 1) return cudaSuccess;
  kern<<<grid, NT, smem, s>>>(g, p, make_sc<T>(p), a, b, c, (const T *)rho, dt, xf);
  return cudaGetLastError();
}

// FP32 column launches of one stage form (STAGE, EX) in launch configuration
// `cfg`: CNT threads, or (Levermore closure, the default) CNT + 32 threads at
// 3 (schedule 0) or 2 (schedule 1) CTAs per SM; other closures run the
// CNT-thread kernel for every column configuration.
template <int STAGE, int CL, bool EX>
static cudaError_t launch_rad_col_f32(int cfg, const Geometry &g, const qk_params &p,
                                      void *const *R0, void *const *R1, void *const *Ro,
                                      const void *rho, DtSrc dt, const FuseArgs *fx,
                                      cudaStream_t s) {
  if constexpr (CL == QK_CLOSURE_LEVERMORE) {
    if (cfg_threads(cfg) == CNT + 32)
      return cfg_sched(cfg)
                 ? launch_rad_col_one<float, STAGE, CL, EX, CNT + 32, 2>(g, p, R0, R1, Ro, rho,
                                                                          dt, fx, s)
                 : launch_rad_col_one<float, STAGE, CL, EX, CNT + 32, 3>(g, p, R0, R1, Ro, rho,
                                                                          dt, fx, s);
  }
  return launch_rad_col_one<float, STAGE, CL, EX>(g, p, R0, R1, Ro, rho, dt, fx, s);
}

// Column launches of one closure (instantiated per closure in
// qk_column_rad.cu); fx non-null fuses the exchange into stage 2.
template <int CL>
cudaError_t launch_rad_column_closure(int fp32, int stage, const Geometry &g, const qk_params &p,
                                      void *const *R0, void *const *R1, void *const *Ro,
                                      const void *rho, DtSrc dt, const FuseArgs *fx,
                                      cudaStream_t s, int cfg) {
  if (fp32) {
    if (stage == 1) return launch_rad_col_f32<1, CL, false>(cfg, g, p, R0, R1, Ro, rho, dt, fx, s);
    if (fx) return launch_rad_col_f32<2, CL, true>(cfg, g, p, R0, R1, Ro, rho, dt, fx, s);
    return launch_rad_col_f32<2, CL, false>(cfg, g, p, R0, R1, Ro, rho, dt, fx, s);
  }
  if (stage == 1) return launch_rad_col_one<double, 1, CL, false>(g, p, R0, R1, Ro, rho, dt, fx, s);
  if (fx) return launch_rad_col_one<double, 2, CL, true>(g, p, R0, R1, Ro, rho, dt, fx, s);
  return launch_rad_col_one<double, 2, CL, false>(g, p, R0, R1, Ro, rho, dt, fx, s);
}

}  // namespace qk
