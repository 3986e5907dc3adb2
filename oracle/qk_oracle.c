/*
 * qk_oracle.c -- plain, slow, FP64 CPU oracle for the per-cell uniform-patch
 * radiation-hydrodynamics update of Wibking & Krumholz, "QUOKKA: a code for
 * two-moment AMR radiation hydrodynamics on GPUs" (arXiv:2110.01792).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the parity reference that the CUDA
 * path is checked against, and the timed CPU baseline.  Only the tests, the
 * smoke check and the benchmark's CPU-baseline leg may load it.  It shares no
 * code, header or constant with the CUDA library, and the CUDA library never
 * calls it.
 *
 * Every step follows the paper's text in the paper's order, one cell and one
 * face at a time, with no blocking, fusion or reordering:
 *   - conserved -> primitive            Sec. 2.2.1 (cell average = cell centre)
 *   - PPM interface value + limiting    Sec. 2.2.1 (interface stencil equation,
 *                                        min/max clamp, CW84 extremum/overshoot)
 *   - HLLC flux with PVRS wavespeeds    Sec. 2.2.1 (Toro 2013, ch. 10)
 *   - RK2-SSP method-of-lines stage     Sec. 2.2.1 (Shu & Osher 1988)
 *   - CFL timestep                      Sec. 2.2.1 (eq. signal and the dt formula)
 *   - radiation reconstruction, Levermore closure, HLL flux, RSLA
 *                                        Sec. 2.2.2 (eq. M1_closure, eqs. rad_energy,
 *                                        rad_flux)
 *   - implicit matter-radiation exchange Sec. 2.2.3 (eqs. delta_er, delta_eg and the
 *                                        convergence test; flux backward Euler;
 *                                        momentum and kinetic-energy work terms)
 *   - radiation substep count            Sec. 2.2.4 (N_sub,max)
 *
 * Readings of passages that are ambiguous or garbled in the paper are listed in
 * the design notes and repeated at the point of use below.
 *
 * Layout: every field is one contiguous array over all patches; patch b starts
 * at element off[b] and holds (n+2g)^3 cells, x fastest.  The oracle reads only
 * interior cells: a stencil neighbour outside its patch is fetched from the
 * patch that owns the periodic image of that cell (an owner map over the
 * periodic domain), so the oracle needs no ghost fill of its own.  Across a
 * non-periodic domain face the neighbour is resolved by the boundary
 * condition of that face (mirror image with the normal vector components
 * negated, nearest interior cell, or a stored boundary state).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_OK 0
#define OR_EINVAL 1
#define OR_ENOCONV 3
#define OR_ENEGATIVE 4

#define NHYD 5 /* rho, mx, my, mz, E */
#define NRAD 4 /* Er, Fx, Fy, Fz */
#define NSUMS 13

typedef struct {
  double gamma;      /* adiabatic index of the gamma-law gas                    */
  double cfl;        /* CFL number, C0/D in Sec. 2.2.1                          */
  double a_r;        /* radiation constant                                      */
  double c;          /* speed of light                                          */
  double chat;       /* reduced speed of light                                  */
  double c_v;        /* specific heat at constant volume: T = E_g/(rho c_v)     */
  double kappa_P;    /* Planck mean opacity (or kappa0 when kappa_mode = 1)     */
  double kappa_R;    /* Rosseland mean opacity (or kappa0 when kappa_mode = 1)  */
  double alpha_eos;  /* alpha of the C_v = alpha T^3 test EOS (eq. heat_capacity) */
  double eps_newton; /* Newton relative tolerance epsilon                       */
  double dx[3];      /* cell spacing                                            */
  int32_t kappa_mode;     /* 0: constant kappa; 1: kappa = kappa0 * rho            */
  int32_t eos;            /* 0: gamma-law; 1: E_g = alpha T^4 / 4                  */
  int32_t max_iter;       /* Newton iteration limit (400 in the paper)             */
  int32_t nsub_max;       /* N_sub,max (10 in the paper)                           */
  int32_t tau_correction; /* 1: optical-depth correction of the radiation flux     */
  int32_t hydro_only;     /* 1: skip radiation substeps                            */
  int32_t recon;          /* 0: PPM; 1: PLM with the MC limiter (Sec. 2.2.1)       */
  int32_t flattening;     /* 1: multidimensional shock flattening (Sec. 2.2.1)     */
  int32_t closure;        /* 0: Levermore; 1: Minerbo; 2: Eddington (Sec. 2.2.2)   */
  int32_t bc_lo[3];       /* boundary of the low / high domain face per axis:      */
  int32_t bc_hi[3];       /* 0 periodic, 1 reflecting, 2 outflow, 3 Dirichlet      */
} or_params;

#define OR_BC_PERIODIC 0
#define OR_BC_REFLECT 1
#define OR_BC_OUTFLOW 2
#define OR_BC_DIRICHLET 3
#define NFIELD 9 /* rho, mx, my, mz, E, Er, Fx, Fy, Fz: field ids of the boundary code */

typedef struct {
  int32_t nbox, ng;
  int32_t dom_n[3];
  int32_t *lo, *n; /* 3*nbox */
  int64_t *off;    /* nbox   */
  int32_t *owner;  /* dom_n[0]*dom_n[1]*dom_n[2] -> box id */
  /* Dirichlet boundary states: NFIELD values per cell of the domain extended
   * by ng cells on every side (only cells outside a Dirichlet face are used) */
  double *dstore;
  unsigned char *dset;
} or_grid;

/* ------------------------------------------------------------------------ */
/* grid and cell access                                                      */
/* ------------------------------------------------------------------------ */

static int64_t wrap(int64_t a, int64_t n) {
  int64_t r = a % n;
  return r < 0 ? r + n : r;
}

or_grid *or_grid_create(int32_t nbox, const int32_t *lo, const int32_t *n,
                        const int64_t *off, const int32_t *dom_n, int32_t ng) {
  or_grid *g = (or_grid *)calloc(1, sizeof(or_grid));
  g->nbox = nbox;
  g->ng = ng;
  memcpy(g->dom_n, dom_n, 3 * sizeof(int32_t));
  g->lo = (int32_t *)malloc(3 * sizeof(int32_t) * nbox);
  g->n = (int32_t *)malloc(3 * sizeof(int32_t) * nbox);
  g->off = (int64_t *)malloc(sizeof(int64_t) * nbox);
  memcpy(g->lo, lo, 3 * sizeof(int32_t) * nbox);
  memcpy(g->n, n, 3 * sizeof(int32_t) * nbox);
  memcpy(g->off, off, sizeof(int64_t) * nbox);
  int64_t ncell = (int64_t)dom_n[0] * dom_n[1] * dom_n[2];
  g->owner = (int32_t *)malloc(sizeof(int32_t) * ncell);
  for (int64_t c = 0; c < ncell; ++c) g->owner[c] = -1;
  for (int b = 0; b < nbox; ++b)
    for (int k = 0; k < n[3 * b + 2]; ++k)
      for (int j = 0; j < n[3 * b + 1]; ++j)
        for (int i = 0; i < n[3 * b + 0]; ++i) {
          int64_t x = wrap(lo[3 * b] + i, dom_n[0]);
          int64_t y = wrap(lo[3 * b + 1] + j, dom_n[1]);
          int64_t z = wrap(lo[3 * b + 2] + k, dom_n[2]);
          g->owner[(z * dom_n[1] + y) * dom_n[0] + x] = b;
        }
  return g;
}

void or_grid_destroy(or_grid *g) {
  if (!g) return;
  free(g->lo);
  free(g->n);
  free(g->off);
  free(g->owner);
  free(g->dstore);
  free(g->dset);
  free(g);
}

/* element index of local cell (i,j,k) of patch b, (i,j,k) in [-ng, n+ng) */
static int64_t cell_index(const or_grid *g, int b, int i, int j, int k) {
  int64_t sx = g->n[3 * b] + 2 * g->ng, sy = g->n[3 * b + 1] + 2 * g->ng;
  return g->off[b] + ((int64_t)(k + g->ng) * sy + (j + g->ng)) * sx + (i + g->ng);
}

/* element index of the interior cell holding the value of patch b's local
 * (i,j,k), which may lie outside the patch: periodic image, then its owner. */
static int64_t owner_index(const or_grid *g, int b, int i, int j, int k) {
  const int32_t *n = g->n + 3 * b;
  if (i >= 0 && j >= 0 && k >= 0 && i < n[0] && j < n[1] && k < n[2])
    return cell_index(g, b, i, j, k);
  int64_t x = wrap((int64_t)g->lo[3 * b] + i, g->dom_n[0]);
  int64_t y = wrap((int64_t)g->lo[3 * b + 1] + j, g->dom_n[1]);
  int64_t z = wrap((int64_t)g->lo[3 * b + 2] + k, g->dom_n[2]);
  int q = g->owner[(z * g->dom_n[1] + y) * g->dom_n[0] + x];
  const int32_t *lq = g->lo + 3 * q;
  /* local coordinates of the global cell in patch q (unwrapped into q's range) */
  int64_t li = wrap(x - lq[0], g->dom_n[0]);
  int64_t lj = wrap(y - lq[1], g->dom_n[1]);
  int64_t lk = wrap(z - lq[2], g->dom_n[2]);
  return cell_index(g, q, (int)li, (int)lj, (int)lk);
}

/* Where the value of patch b's local cell c comes from, under the domain
 * boundary conditions.  Each axis is resolved on its own: inside the domain
 * the coordinate stays; across a periodic face it wraps; across a reflecting
 * face it is mirrored (x -> -1-x below, 2N-1-x above) and the vector
 * components along that axis change sign; across an outflow face it is
 * clamped to the nearest interior cell (zero gradient); across a Dirichlet
 * face the cell takes the stored boundary state (whatever the other axes do).
 * Result: the element index of the interior cell (e >= 0) with the axes to
 * negate, or e = -1 and the index of the cell in the Dirichlet store. */
typedef struct {
  int64_t e;
  int flip;      /* bit d: negate the d-components of vectors */
  int64_t key;   /* Dirichlet store index (e = -1) */
  int outside;   /* 1: outside a non-periodic face on some axis */
} or_src;

static int64_t ext_index(const or_grid *g, const int64_t x[3]) {
  int64_t ex = g->dom_n[0] + 2 * g->ng, ey = g->dom_n[1] + 2 * g->ng;
  return ((x[2] + g->ng) * ey + (x[1] + g->ng)) * ex + (x[0] + g->ng);
}

static or_src resolve(const or_grid *g, const or_params *p, int b, const int c[3]) {
  or_src r = {-1, 0, -1, 0};
  int64_t x[3], raw[3];
  int dir = 0;
  for (int d = 0; d < 3; ++d) {
    int64_t D = g->dom_n[d];
    int64_t v = (int64_t)g->lo[3 * b + d] + c[d];
    raw[d] = v;
    if (v < 0 || v >= D) {
      int bc = v < 0 ? p->bc_lo[d] : p->bc_hi[d];
      if (bc == OR_BC_PERIODIC) {
        v = wrap(v, D);
        raw[d] = v;
      } else {
        r.outside = 1;
        if (bc == OR_BC_REFLECT) {
          v = v < 0 ? -1 - v : 2 * D - 1 - v;
          r.flip |= 1 << d;
        } else if (bc == OR_BC_OUTFLOW) {
          v = v < 0 ? 0 : D - 1;
        } else {
          dir = 1;
        }
      }
    }
    x[d] = v;
  }
  if (dir) {
    r.key = ext_index(g, raw);
    r.flip = 0;
    return r;
  }
  int q = g->owner[(x[2] * g->dom_n[1] + x[1]) * g->dom_n[0] + x[0]];
  if (q < 0) {
    /* a refined level that does not cover this cell: the value is the one
     * patch b's own ghost cell holds (interpolated from the coarser level) */
    r.e = cell_index(g, b, c[0], c[1], c[2]);
    r.outside = 1;
    return r;
  }
  r.e = cell_index(g, q, (int)(x[0] - g->lo[3 * q]), (int)(x[1] - g->lo[3 * q + 1]),
                   (int)(x[2] - g->lo[3 * q + 2]));
  return r;
}

/* vector axis of a field id (momentum or radiation flux component), or -1 */
static int field_axis(int fid) {
  if (fid >= 1 && fid <= 3) return fid - 1;
  if (fid >= 6 && fid <= 8) return fid - 6;
  return -1;
}

/* value of field `fid` (array f) at a resolved cell */
static double src_value(const or_grid *g, const double *f, int fid, const or_src *r) {
  if (r->e < 0) return g->dstore[r->key * NFIELD + fid];
  int ax = field_axis(fid);
  double v = f[r->e];
  return (ax >= 0 && ((r->flip >> ax) & 1)) ? -v : v;
}

/* value of field fid (array f) at patch b's local cell c */
static double cell_value(const or_grid *g, const or_params *p, const double *f, int fid, int b,
                         const int c[3]) {
  or_src r = resolve(g, p, b, c);
  return src_value(g, f, fid, &r);
}

/* Record the Dirichlet boundary states: the values that the caller's arrays
 * (all NFIELD fields, hydro then radiation) hold in the ghost cells beyond
 * the Dirichlet faces.  Every ghost cell that maps to the same boundary
 * position must hold the same values (else OR_EINVAL). */
int or_set_dirichlet(or_grid *g, const or_params *p, double *const *fields) {
  int64_t ne = 1;
  for (int d = 0; d < 3; ++d) ne *= g->dom_n[d] + 2 * g->ng;
  free(g->dstore);
  free(g->dset);
  g->dstore = (double *)calloc((size_t)(ne * NFIELD), sizeof(double));
  g->dset = (unsigned char *)calloc((size_t)ne, 1);
  int ng = g->ng;
  for (int b = 0; b < g->nbox; ++b) {
    const int32_t *n = g->n + 3 * b;
    for (int k = -ng; k < n[2] + ng; ++k)
      for (int j = -ng; j < n[1] + ng; ++j)
        for (int i = -ng; i < n[0] + ng; ++i) {
          int c[3] = {i, j, k};
          or_src r = resolve(g, p, b, c);
          if (r.e >= 0) continue;
          int64_t e = cell_index(g, b, i, j, k);
          for (int f = 0; f < NFIELD; ++f) {
            double v = fields[f][e];
            if (g->dset[r.key] && g->dstore[r.key * NFIELD + f] != v) return OR_EINVAL;
            g->dstore[r.key * NFIELD + f] = v;
          }
          g->dset[r.key] = 1;
        }
  }
  return OR_OK;
}

/* Fill every ghost cell of nf fields (field ids fid0 .. fid0+nf-1) under the
 * boundary conditions: the value a stencil read of that cell sees. */
/* ------------------------------------------------------------------------ */
/* host threads                                                              */
/* ------------------------------------------------------------------------ */

/* Cell loops run over z-planes (patch b, index k), distributed over host
 * threads with OpenMP when the oracle is compiled with it.  Every cell is
 * computed by the same code from the same inputs whichever thread takes its
 * plane, and every reduction whose result depends on the order (the exchange
 * status, the conservation sums) is combined in the serial plane order, so
 * the results are bit-identical to one thread. */
static int or_nthreads = 1;

/* Set the number of host threads of the cell loops; returns the number in
 * effect (1 when the oracle was compiled without OpenMP). */
int or_set_threads(int n) {
#ifdef _OPENMP
  or_nthreads = n < 1 ? 1 : n;
#else
  (void)n;
  or_nthreads = 1;
#endif
  return or_nthreads;
}

typedef struct {
  int b, k;
} or_plane;

/* the z-planes k in [k0, n_z + k1) of every patch, in serial order
 * (interior planes: k0 = k1 = 0; with ghost layers: k0 = -ng, k1 = ng) */
static or_plane *grid_planes(const or_grid *g, int k0, int k1, int64_t *np) {
  int64_t n = 0;
  for (int b = 0; b < g->nbox; ++b) n += g->n[3 * b + 2] + k1 - k0;
  or_plane *pl = (or_plane *)malloc((size_t)(n > 0 ? n : 1) * sizeof(or_plane));
  int64_t t = 0;
  for (int b = 0; b < g->nbox; ++b)
    for (int k = k0; k < g->n[3 * b + 2] + k1; ++k) {
      pl[t].b = b;
      pl[t].k = k;
      ++t;
    }
  *np = n;
  return pl;
}

int or_fill_ghosts_bc(const or_grid *g, const or_params *p, double *const *f, int nf, int fid0) {
  int ng = g->ng;
  int bad = 0;
  int64_t np;
  or_plane *pl = grid_planes(g, -ng, ng, &np);
  /* ghost cells are written from interior cells (or the boundary store)
   * only, so the planes are independent */
#pragma omp parallel for schedule(dynamic, 1) num_threads(or_nthreads) if (or_nthreads > 1)
  for (int64_t t = 0; t < np; ++t) {
    const int b = pl[t].b, k = pl[t].k;
    const int32_t *n = g->n + 3 * b;
    for (int j = -ng; j < n[1] + ng; ++j)
      for (int i = -ng; i < n[0] + ng; ++i) {
        int inside = i >= 0 && j >= 0 && k >= 0 && i < n[0] && j < n[1] && k < n[2];
        if (inside) continue;
        int c[3] = {i, j, k};
        or_src r = resolve(g, p, b, c);
        if (r.e < 0 && !g->dstore) {
#pragma omp atomic write
          bad = 1;
          continue;
        }
        for (int v = 0; v < nf; ++v) f[v][cell_index(g, b, i, j, k)] = src_value(g, f[v], fid0 + v, &r);
      }
  }
  free(pl);
  return bad ? OR_EINVAL : OR_OK;
}

/* fill every ghost cell of every patch from the owner of its periodic image */
void or_fill_ghosts(const or_grid *g, double *f) {
  int ng = g->ng;
  int64_t np;
  or_plane *pl = grid_planes(g, -ng, ng, &np);
#pragma omp parallel for schedule(dynamic, 1) num_threads(or_nthreads) if (or_nthreads > 1)
  for (int64_t t = 0; t < np; ++t) {
    const int b = pl[t].b, k = pl[t].k;
    const int32_t *n = g->n + 3 * b;
    for (int j = -ng; j < n[1] + ng; ++j)
      for (int i = -ng; i < n[0] + ng; ++i) {
        int inside = i >= 0 && j >= 0 && k >= 0 && i < n[0] && j < n[1] && k < n[2];
        if (inside) continue;
        f[cell_index(g, b, i, j, k)] = f[owner_index(g, b, i, j, k)];
      }
  }
  free(pl);
}

/* ------------------------------------------------------------------------ */
/* hydrodynamics (Sec. 2.2.1)                                                */
/* ------------------------------------------------------------------------ */

/* Conserved -> primitive, assuming cell average = cell centre value.
 * E_g = E - rho v^2 / 2 (Sec. 2.2.3), P = (gamma - 1) E_g.
 * |v|^2 is summed as (vx^2 + vy^2) + vz^2 so that an x<->y transposition of
 * the data transposes the result exactly. */
static void con2prim(const double U[NHYD], double gamma, double q[NHYD]) {
  double rho = U[0];
  double vx = U[1] / rho, vy = U[2] / rho, vz = U[3] / rho;
  double v2 = (vx * vx + vy * vy) + vz * vz;
  double Eg = U[4] - 0.5 * rho * v2;
  q[0] = rho;
  q[1] = vx;
  q[2] = vy;
  q[3] = vz;
  q[4] = (gamma - 1.0) * Eg;
}

static double dmin(double a, double b) { return a < b ? a : b; }
static double dmax(double a, double b) { return a > b ? a : b; }

/* PPM reconstruction of one cell i from the stencil s[0..4] = q_{i-2..i+2}
 * (Sec. 2.2.1).  Returns the left-face state qL (at i-1/2) and the
 * right-face state qR (at i+1/2).  Steps, in the paper's order:
 *  1. interface values from the 4-point stencil, grouped symmetrically:
 *     q_{j+1/2} = (7/12)(q_j + q_{j+1}) - (1/12)(q_{j-1} + q_{j+2});
 *  2. clamp both face values to [min, max] of the cell and its two neighbours;
 *  3. extremum ((qR - q)(q - qL) <= 0): linear reconstruction in the cell,
 *     reading: with the monotonized-central slope, the paper's PLM limiter;
 *  4. otherwise the CW84 overshoot correction, reading: CW84's own formulas
 *     qL = 3q - 2qR or qR = 3q - 2qL on the side of the overshoot.
 * Flattening and contact steepening are not applied (plain method). */
void or_ppm_cell(const double s[5], double *qL_out, double *qR_out) {
  const double c7 = 7.0 / 12.0, c1 = 1.0 / 12.0;
  double qm = s[1], q0 = s[2], qp = s[3];
  /* step 1 */
  double fL = c7 * (s[1] + s[2]) - c1 * (s[0] + s[3]); /* q_{i-1/2} */
  double fR = c7 * (s[2] + s[3]) - c1 * (s[1] + s[4]); /* q_{i+1/2} */
  /* step 2 */
  double lo = dmin(qm, dmin(q0, qp));
  double hi = dmax(qm, dmax(q0, qp));
  double qL = dmin(dmax(fL, lo), hi);
  double qR = dmin(dmax(fR, lo), hi);
  if ((qR - q0) * (q0 - qL) <= 0.0) {
    /* step 3: extremum -> linear reconstruction with the MC slope */
    double dm = q0 - qm, dp = qp - q0, slope = 0.0;
    if (dm * dp > 0.0) {
      double a = fabs(dm), b = fabs(dp), cc = fabs(dm + dp);
      double m = dmin(2.0 * a, dmin(2.0 * b, 0.5 * cc));
      slope = dp > 0.0 ? m : -m;
    }
    qL = q0 - 0.5 * slope;
    qR = q0 + 0.5 * slope;
  } else {
    /* step 4: CW84 overshoot test on the parabola through qL, q0, qR */
    double d = qR - qL;
    double q6 = 6.0 * (q0 - 0.5 * (qL + qR));
    if (d * q6 > d * d) {
      qL = 3.0 * q0 - 2.0 * qR;
    } else if (-(d * d) > d * q6) {
      qR = 3.0 * q0 - 2.0 * qL;
    }
  }
  *qL_out = qL;
  *qR_out = qR;
}

/* PLM reconstruction of one cell with the monotonized-central limiter
 * (van Leer 1977), the paper's compile-time alternative to PPM (Sec. 2.2.1):
 * slope = 0 at a local extremum of the cell averages, else
 * sign(dq+) min(2|dq-|, 2|dq+|, |dq- + dq+|/2); qL,R = q -/+ slope/2. */
void or_plm_cell(const double s[5], double *qL_out, double *qR_out) {
  double qm = s[1], q0 = s[2], qp = s[3];
  double dm = q0 - qm, dp = qp - q0, slope = 0.0;
  if (dm * dp > 0.0) {
    double a = fabs(dm), b = fabs(dp), cc = fabs(dm + dp);
    double m = dmin(2.0 * a, dmin(2.0 * b, 0.5 * cc));
    slope = dp > 0.0 ? m : -m;
  }
  *qL_out = q0 - 0.5 * slope;
  *qR_out = q0 + 0.5 * slope;
}

static void recon_cell(const or_params *p, const double s[5], double *qL, double *qR) {
  if (p->recon == 1)
    or_plm_cell(s, qL, qR);
  else
    or_ppm_cell(s, qL, qR);
}

/* Euler flux normal to direction d of primitive state w = (rho, vx, vy, vz, P)
 * and the matching conserved state.  The kinetic energy is summed as
 * un^2 + (ut1^2 + ut2^2), symmetric in the two transverse components. */
static void euler_state(const double w[NHYD], int d, double gamma, double U[NHYD],
                        double F[NHYD]) {
  int t1 = (d + 1) % 3, t2 = (d + 2) % 3;
  double rho = w[0], un = w[1 + d], u1 = w[1 + t1], u2 = w[1 + t2], p = w[4];
  double E = p / (gamma - 1.0) + 0.5 * rho * (un * un + (u1 * u1 + u2 * u2));
  U[0] = rho;
  U[1 + d] = rho * un;
  U[1 + t1] = rho * u1;
  U[1 + t2] = rho * u2;
  U[4] = E;
  F[0] = rho * un;
  F[1 + d] = rho * un * un + p;
  F[1 + t1] = rho * un * u1;
  F[1 + t2] = rho * un * u2;
  F[4] = un * (E + p);
}

/* HLLC flux across a face normal to d with left state wL and right state wR
 * (primitive), with the 'primitive variable Riemann solver' pressure estimate
 * (Toro 2013, ch. 9-10) used for the wavespeeds (Sec. 2.2.1):
 *   p_pvrs = (pL+pR)/2 - (uR-uL) rhobar abar / 2,  p_s = max(0, p_pvrs)
 *   q_K = 1 if p_s <= p_K else sqrt(1 + (gamma+1)/(2 gamma) (p_s/p_K - 1))
 *   S_L = uL - aL qL,  S_R = uR + aR qR,  S* from Toro eq. 10.37
 * and the standard HLLC star states (Toro eq. 10.39). */
void or_hllc(const double wL[NHYD], const double wR[NHYD], int d, double gamma,
             double F[NHYD]) {
  double UL[NHYD], UR[NHYD], FL[NHYD], FR[NHYD];
  euler_state(wL, d, gamma, UL, FL);
  euler_state(wR, d, gamma, UR, FR);
  double rL = wL[0], rR = wR[0], uL = wL[1 + d], uR = wR[1 + d], pL = wL[4], pR = wR[4];
  double aL = sqrt(gamma * pL / rL), aR = sqrt(gamma * pR / rR);
  double abar = 0.5 * (aL + aR), rbar = 0.5 * (rL + rR);
  double ppvrs = 0.5 * (pL + pR) - 0.5 * (uR - uL) * rbar * abar;
  double ps = dmax(0.0, ppvrs);
  double g1 = (gamma + 1.0) / (2.0 * gamma);
  double qL = ps <= pL ? 1.0 : sqrt(1.0 + g1 * (ps / pL - 1.0));
  double qR = ps <= pR ? 1.0 : sqrt(1.0 + g1 * (ps / pR - 1.0));
  double SL = uL - aL * qL, SR = uR + aR * qR;
  double Ss = (pR - pL + rL * uL * (SL - uL) - rR * uR * (SR - uR)) /
              (rL * (SL - uL) - rR * (SR - uR));
  if (0.0 <= SL) {
    memcpy(F, FL, sizeof(FL));
    return;
  }
  if (SR <= 0.0) {
    memcpy(F, FR, sizeof(FR));
    return;
  }
  /* star region: the tie S* = 0 goes to the left star state */
  const double *w = Ss >= 0.0 ? wL : wR;
  const double *U = Ss >= 0.0 ? UL : UR;
  const double *FK = Ss >= 0.0 ? FL : FR;
  double SK = Ss >= 0.0 ? SL : SR;
  double rK = w[0], uK = w[1 + d], pK = w[4];
  int t1 = (d + 1) % 3, t2 = (d + 2) % 3;
  /* Toro eq. 10.39, U*_K = rho_K (S_K - u_K)/(S_K - S*) [1, S*, v, w,
   * E_K/rho_K + (S* - u_K)(S* + p_K/(rho_K (S_K - u_K)))], written with the
   * ratio (S_K - u_K)/(S_K - S*) taken first and E_K kept whole, so that a
   * stationary contact (u = S* = 0, equal p) gives U*_K = U_K bit for bit and
   * the exactly-zero contact error of Sec. 3.1.2 holds in floating point. */
  double ratio = (SK - uK) / (SK - Ss);
  double fac = rK * ratio;
  double Us[NHYD];
  Us[0] = fac;
  Us[1 + d] = fac * Ss;
  Us[1 + t1] = fac * w[1 + t1];
  Us[1 + t2] = fac * w[1 + t2];
  Us[4] = ratio * (U[4] + rK * (Ss - uK) * (Ss + pK / (rK * (SK - uK))));
  for (int v = 0; v < NHYD; ++v) F[v] = FK[v] + SK * (Us[v] - U[v]);
}

/* gather the primitive variables of cells i0..i0+5 along d around (b,i,j,k) */
static void gather_prims(const or_grid *g, const or_params *p, double *const *U, int b,
                         const int c[3], int d, int first, double w[NHYD][6]) {
  for (int s = 0; s < 6; ++s) {
    int cc[3] = {c[0], c[1], c[2]};
    cc[d] += first + s;
    or_src r = resolve(g, p, b, cc);
    double Uc[NHYD], q[NHYD];
    for (int v = 0; v < NHYD; ++v) Uc[v] = src_value(g, U[v], v, &r);
    con2prim(Uc, p->gamma, q);
    for (int v = 0; v < NHYD; ++v) w[v][s] = q[v];
  }
}

/* Shock flattening (Sec. 2.2.1): the one-dimensional coefficient of Colella &
 * Woodward (1984, appendix) along direction d at cell c,
 *   ftilde = min(1, max(0, w2 (|p_{c+1} - p_{c-1}| / |p_{c+2} - p_{c-2}| - w1)))
 * where the cell sits in a compressive jump (u_{c-1} > u_{c+1} along d and
 * |p_{c+1} - p_{c-1}| > eps min(p_{c+1}, p_{c-1})), else 0; CW84's constants
 * eps = 0.33, w1 = 0.75, w2 = 10. */
static double flat_ftilde(const or_grid *g, const or_params *p, double *const *U, int b,
                          const int c[3], int d) {
  double pr[5], un[5];
  for (int o = -2; o <= 2; ++o) {
    int cc[3] = {c[0], c[1], c[2]};
    cc[d] += o;
    or_src r = resolve(g, p, b, cc);
    double Uc[NHYD], q[NHYD];
    for (int v = 0; v < NHYD; ++v) Uc[v] = src_value(g, U[v], v, &r);
    con2prim(Uc, p->gamma, q);
    pr[o + 2] = q[4];
    un[o + 2] = q[1 + d];
  }
  double dp1 = pr[3] - pr[1], dp2 = pr[4] - pr[0];
  int shock = fabs(dp1) > 0.33 * dmin(pr[3], pr[1]) && un[1] - un[3] > 0.0;
  if (!shock) return 0.0;
  if (!(fabs(dp2) > 0.0)) return 1.0;
  return dmin(1.0, dmax(0.0, 10.0 * (fabs(dp1) / fabs(dp2) - 0.75)));
}

/* Multidimensional flattening coefficient of Miller & Colella (2002) at cell c:
 * chi = min over directions of (1 - f_d), with f_d = max(ftilde_d(c),
 * ftilde_d(c - sign(p_{c+1} - p_{c-1}))) (CW84's extension by one cell on the
 * low-pressure side).  chi = 1 leaves the reconstruction unchanged. */
static double flat_chi(const or_grid *g, const or_params *p, double *const *U, int b,
                       const int c[3]) {
  double chi = 1.0;
  for (int d = 0; d < 3; ++d) {
    double f = flat_ftilde(g, p, U, b, c, d);
    double pr[2];
    for (int s = 0; s < 2; ++s) {
      int cc[3] = {c[0], c[1], c[2]};
      cc[d] += s == 0 ? -1 : 1;
      or_src r = resolve(g, p, b, cc);
      double Uc[NHYD], q[NHYD];
      for (int v = 0; v < NHYD; ++v) Uc[v] = src_value(g, U[v], v, &r);
      con2prim(Uc, p->gamma, q);
      pr[s] = q[4];
    }
    double dp1 = pr[1] - pr[0];
    if (dp1 != 0.0) {
      int cc[3] = {c[0], c[1], c[2]};
      cc[d] += dp1 > 0.0 ? -1 : 1;
      f = dmax(f, flat_ftilde(g, p, U, b, cc, d));
    }
    chi = dmin(chi, 1.0 - f);
  }
  return chi;
}

/* Flattening coefficient of patch b's local cell c: the stored value of the
 * interior cell it maps to, or, for a cell outside a non-periodic domain
 * face, the coefficient computed at that position from the boundary values
 * around it (what a ghost cell holding those values yields). */
static double chi_at(const or_grid *g, const or_params *p, double *const *U, const double *chi,
                     int b, const int c[3]) {
  or_src r = resolve(g, p, b, c);
  if (r.outside) return flat_chi(g, p, U, b, c);
  return chi[r.e];
}

/* hydro flux at the face between cell c+first+2 and c+first+3 along d,
 * computed from the six cells c+first .. c+first+5 */
static void hydro_face_flux(const or_grid *g, const or_params *p, double *const *U,
                            const double *chi, int b, const int c[3], int d, int first,
                            double F[NHYD]) {
  double w[NHYD][6], wL[NHYD], wR[NHYD], dummy;
  gather_prims(g, p, U, b, c, d, first, w);
  for (int v = 0; v < NHYD; ++v) {
    recon_cell(p, &w[v][0], &dummy, &wL[v]); /* right face of the left cell  */
    recon_cell(p, &w[v][1], &wR[v], &dummy); /* left face of the right cell  */
  }
  if (p->flattening) {
    /* reading: the face states are blended with the cell average after the
     * limiter, q <- chi q + (1 - chi) q_cell; the coefficients come from the
     * stage's table, or are computed here when there is none */
    int cA[3] = {c[0], c[1], c[2]}, cB[3] = {c[0], c[1], c[2]};
    cA[d] += first + 2;
    cB[d] += first + 3;
    double chiA = chi ? chi_at(g, p, U, chi, b, cA) : flat_chi(g, p, U, b, cA);
    double chiB = chi ? chi_at(g, p, U, chi, b, cB) : flat_chi(g, p, U, b, cB);
    for (int v = 0; v < NHYD; ++v) {
      wL[v] = chiA * wL[v] + (1.0 - chiA) * w[v][2];
      wR[v] = chiB * wR[v] + (1.0 - chiB) * w[v][3];
    }
  }
  or_hllc(wL, wR, d, p->gamma, F);
}

/* The hydro flux through the low face of patch b's cell c along d (between
 * c - e_d and c), from the state U: the flux the stage uses at that face.
 * For the flux registers of mesh refinement (Berger & Colella 1989). */
void or_hydro_face_flux(const or_grid *g, const or_params *p, double *const *U, int32_t b,
                        const int32_t c[3], int32_t d, double F[NHYD]) {
  const int cc[3] = {c[0], c[1], c[2]};
  hydro_face_flux(g, p, U, NULL, b, cc, d, -3, F);
}

/* L(U) at interior cell (b,i,j,k): minus the divergence of the face fluxes,
 * summed as ((x + y) + z) (Sec. 2.2.1, exact x<->y symmetry, Sec. 3.1). */
static void hydro_rhs_cell(const or_grid *g, const or_params *p, double *const *U,
                           const double *chi, int b, const int c[3], double L[NHYD]) {
  double div[3][NHYD];
  for (int d = 0; d < 3; ++d) {
    double Flo[NHYD], Fhi[NHYD];
    hydro_face_flux(g, p, U, chi, b, c, d, -3, Flo); /* face c-1/2 */
    hydro_face_flux(g, p, U, chi, b, c, d, -2, Fhi); /* face c+1/2 */
    for (int v = 0; v < NHYD; ++v) div[d][v] = (Fhi[v] - Flo[v]) / p->dx[d];
  }
  for (int v = 0; v < NHYD; ++v) L[v] = -((div[0][v] + div[1][v]) + div[2][v]);
}

/* iterate over a list of interior cells (b,i,j,k quadruples) or, when
 * cells == NULL, over every interior cell of every patch (z-planes over the
 * host threads; fn writes only its own cell of its outputs and reads no
 * output of another cell, as every stage here does) */
typedef void (*cell_fn)(const or_grid *g, const or_params *p, int b, const int c[3],
                        void *ctx);
static void for_plane(const or_grid *g, const or_params *p, int b, int k, cell_fn fn,
                      void *ctx) {
  const int32_t *n = g->n + 3 * b;
  for (int j = 0; j < n[1]; ++j)
    for (int i = 0; i < n[0]; ++i) {
      int c[3] = {i, j, k};
      fn(g, p, b, c, ctx);
    }
}

static void for_cells(const or_grid *g, const or_params *p, int64_t ncell,
                      const int32_t *cells, cell_fn fn, void *ctx) {
  if (cells) {
    for (int64_t t = 0; t < ncell; ++t) {
      int c[3] = {cells[4 * t + 1], cells[4 * t + 2], cells[4 * t + 3]};
      fn(g, p, cells[4 * t], c, ctx);
    }
    return;
  }
  int64_t np;
  or_plane *pl = grid_planes(g, 0, 0, &np);
#pragma omp parallel for schedule(dynamic, 1) num_threads(or_nthreads) if (or_nthreads > 1)
  for (int64_t t = 0; t < np; ++t) for_plane(g, p, pl[t].b, pl[t].k, fn, ctx);
  free(pl);
}

typedef struct {
  int stage;
  double *const *U0;
  double *const *U1;
  double *const *Uout;
  double dt;
  const double *rho; /* radiation stages only */
  int nvar;
  const double *chi; /* flattening coefficient per cell (hydro, or NULL) */
} stage_ctx;

/* RK2-SSP (Shu & Osher 1988), Sec. 2.2.1:
 *   stage 1: U1 = U0 + dt L(U0)
 *   stage 2: U2 = U0/2 + (U1 + dt L(U1))/2 */
static void hydro_stage_cell(const or_grid *g, const or_params *p, int b, const int c[3],
                             void *vctx) {
  stage_ctx *s = (stage_ctx *)vctx;
  double L[NHYD];
  int64_t e = cell_index(g, b, c[0], c[1], c[2]);
  if (s->stage == 1) {
    hydro_rhs_cell(g, p, s->U0, s->chi, b, c, L);
    for (int v = 0; v < NHYD; ++v) s->Uout[v][e] = s->U0[v][e] + s->dt * L[v];
  } else {
    hydro_rhs_cell(g, p, s->U1, s->chi, b, c, L);
    for (int v = 0; v < NHYD; ++v)
      s->Uout[v][e] = 0.5 * s->U0[v][e] + 0.5 * (s->U1[v][e] + s->dt * L[v]);
  }
}

/* One hydro RK stage.  Uout may alias U0 only when every listed cell is
 * written after all its reads, which holds cell by cell because a stage-2
 * update reads U0 only at its own cell (and the stencil from U1).  Stage 1
 * must not alias U0 with Uout. */
int or_hydro_stage(const or_grid *g, const or_params *p, int stage, double *const *U0,
                   double *const *U1, double *const *Uout, double dt, int64_t ncell,
                   const int32_t *cells) {
  stage_ctx s = {stage, U0, U1, Uout, dt, NULL, NHYD, NULL};
  double *chi = NULL;
  if (p->flattening) {
    /* the flattening coefficient of every interior cell of the stencil source,
     * computed once per stage (neighbours outside a patch read their owner's) */
    double *const *src = stage == 1 ? U0 : U1;
    int64_t len = 0;
    for (int b = 0; b < g->nbox; ++b) {
      int64_t end = cell_index(g, b, g->n[3 * b] + g->ng - 1, g->n[3 * b + 1] + g->ng - 1,
                               g->n[3 * b + 2] + g->ng - 1) + 1;
      if (end > len) len = end;
    }
    chi = (double *)calloc((size_t)len, sizeof(double));
    int64_t np;
    or_plane *pl = grid_planes(g, 0, 0, &np);
#pragma omp parallel for schedule(dynamic, 1) num_threads(or_nthreads) if (or_nthreads > 1)
    for (int64_t t = 0; t < np; ++t) {
      const int b = pl[t].b, k = pl[t].k;
      const int32_t *n = g->n + 3 * b;
      for (int j = 0; j < n[1]; ++j)
        for (int i = 0; i < n[0]; ++i) {
          int c[3] = {i, j, k};
          chi[cell_index(g, b, i, j, k)] = flat_chi(g, p, src, b, c);
        }
    }
    free(pl);
    s.chi = chi;
  }
  for_cells(g, p, ncell, cells, hydro_stage_cell, &s);
  free(chi);
  return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* timestep (Sec. 2.2.1 and Sec. 2.2.4)                                      */
/* ------------------------------------------------------------------------ */

/* max(|v| + c_s) over all interior cells, |v| = sqrt((vx^2+vy^2)+vz^2) */
double or_max_signal_speed(const or_grid *g, const or_params *p, double *const *U) {
  int64_t np;
  or_plane *pl = grid_planes(g, 0, 0, &np);
  double *pmax = (double *)malloc((size_t)(np > 0 ? np : 1) * sizeof(double));
#pragma omp parallel for schedule(dynamic, 1) num_threads(or_nthreads) if (or_nthreads > 1)
  for (int64_t t = 0; t < np; ++t) {
    const int b = pl[t].b, k = pl[t].k;
    const int32_t *n = g->n + 3 * b;
    double m = 0.0;
    for (int j = 0; j < n[1]; ++j)
      for (int i = 0; i < n[0]; ++i) {
        int64_t e = cell_index(g, b, i, j, k);
        double Uc[NHYD], q[NHYD];
        for (int v = 0; v < NHYD; ++v) Uc[v] = U[v][e];
        con2prim(Uc, p->gamma, q);
        double vmag = sqrt((q[1] * q[1] + q[2] * q[2]) + q[3] * q[3]);
        double cs = sqrt(p->gamma * q[4] / q[0]);
        m = dmax(m, vmag + cs);
      }
    pmax[t] = m;
  }
  /* the maximum of the plane maxima (exact in any order) */
  double smax = 0.0;
  for (int64_t t = 0; t < np; ++t) smax = dmax(smax, pmax[t]);
  free(pmax);
  free(pl);
  return smax;
}

/* dt = CFL dx_min / max(|v| + c_s); radiation: dt_rad,CFL = CFL dx_min / chat.
 * Reading of Sec. 2.2.4: the hydro step is capped at N_sub,max radiation CFL
 * steps; N_sub = ceil(dt / dt_rad,CFL) otherwise, decided as
 *   if dt > N_sub,max dt_rad,CFL: N_sub = N_sub,max, dt = N_sub,max dt_rad,CFL
 *   else N_sub = max(1, ceil(dt / dt_rad,CFL)),
 * and dt_rad = dt / N_sub. */
void or_timestep_from_speed(const or_params *p, double smax, double out[3]) {
  double dxm = dmin(p->dx[0], dmin(p->dx[1], p->dx[2]));
  double dt = p->cfl * dxm / smax;
  double nsub = 0.0, dtrad = 0.0;
  if (!p->hydro_only) {
    double dtr = p->cfl * dxm / p->chat;
    if (dt > p->nsub_max * dtr) {
      nsub = p->nsub_max;
      dt = p->nsub_max * dtr;
    } else {
      nsub = dmax(1.0, ceil(dt / dtr));
    }
    dtrad = dt / nsub;
  }
  out[0] = dt;
  out[1] = nsub;
  out[2] = dtrad;
}

void or_timestep(const or_grid *g, const or_params *p, double *const *U, double out[3]) {
  or_timestep_from_speed(p, or_max_signal_speed(g, p, U), out);
}

/* ------------------------------------------------------------------------ */
/* radiation transport (Sec. 2.2.2)                                          */
/* ------------------------------------------------------------------------ */

/* Eddington factor chi(f), 0 <= f <= 1, of the local closures (Sec. 2.2.2):
 *   Levermore (1984):  chi = (3 + 4 f^2) / (5 + 2 sqrt(4 - 3 f^2))
 *   Minerbo (1978):    the maximum-entropy closure in its polynomial form,
 *                      chi = 1/3 + (2/15) (3 f^2 - f^3 + 3 f^4)
 *   Eddington:         chi = 1/3 (isotropic pressure P_r = E_r I / 3). */
double or_eddington_factor(int closure, double f) {
  if (closure == 2) return 1.0 / 3.0;
  if (closure == 1) return 1.0 / 3.0 + (2.0 / 15.0) * (3.0 * f * f - f * f * f + 3.0 * f * f * f * f);
  return (3.0 + 4.0 * f * f) / (5.0 + 2.0 * sqrt(4.0 - 3.0 * f * f));
}

/* M1 closure, eq. M1_closure:
 *   P_r = [ (1-chi)/2 I + (3 chi - 1)/2 n n ] E_r,  n = F / |F|,
 * with f = |F| / (c E_r) and chi from the selected closure.  When |f| > 1 the
 * flux is rescaled to |F| = c E_r for the closure only (Sec. 2.2.2); when
 * F = 0 the n n term is dropped.  The Eddington closure gives T = I/3
 * exactly.  Returns the Eddington tensor T = P_r / E_r (row-major 3x3). */
void or_eddington_tensor(int closure, const double f[3], double T[9]) {
  double f2 = (f[0] * f[0] + f[1] * f[1]) + f[2] * f[2];
  double fmag = sqrt(f2);
  double fc = dmin(fmag, 1.0);
  double chi = or_eddington_factor(closure, fc);
  double a = 0.5 * (1.0 - chi), bcoef = 0.5 * (3.0 * chi - 1.0);
  if (closure == 2) {
    a = 1.0 / 3.0;
    bcoef = 0.0;
  }
  double nh[3] = {0.0, 0.0, 0.0};
  if (fmag > 0.0)
    for (int i = 0; i < 3; ++i) nh[i] = f[i] / fmag;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double t = (i == j ? a : 0.0);
      if (fmag > 0.0) t += bcoef * nh[i] * nh[j];
      T[3 * i + j] = t;
    }
}

static double kappa_of(const or_params *p, double kappa, double rho) {
  return p->kappa_mode == 1 ? kappa * rho : kappa;
}

/* radiation state of the six cells along d: E_r and f = F/(c E_r) */
static void gather_rad(const or_grid *g, const or_params *p, double *const *R, int b,
                       const int c[3], int d, int first, double w[NRAD][6]) {
  for (int s = 0; s < 6; ++s) {
    int cc[3] = {c[0], c[1], c[2]};
    cc[d] += first + s;
    or_src r = resolve(g, p, b, cc);
    double Er = src_value(g, R[0], NHYD, &r);
    w[0][s] = Er;
    for (int v = 1; v < NRAD; ++v) w[v][s] = src_value(g, R[v], NHYD + v, &r) / (p->c * Er);
  }
}

/* conserved state (E, F) and flux along d of a radiation state (E_r, f):
 *   flux_d = ( (chat/c) F_d,  c chat P_{x d},  c chat P_{y d},  c chat P_{z d} )
 * from eq. rad_energy and eq. rad_flux. */
static void rad_state(const or_params *p, const double w[NRAD], int d, double U[NRAD],
                      double F[NRAD]) {
  double T[9];
  double f[3] = {w[1], w[2], w[3]};
  or_eddington_tensor(p->closure, f, T);
  double E = w[0];
  U[0] = E;
  for (int i = 0; i < 3; ++i) U[1 + i] = p->c * E * f[i];
  F[0] = (p->chat / p->c) * U[1 + d];
  for (int i = 0; i < 3; ++i) F[1 + i] = p->c * p->chat * (E * T[3 * i + d]);
}

/* radiation flux at the face between cells c+first+2 and c+first+3 along d
 * (Sec. 2.2.2).  Readings:
 *  - PPM of E_r and f with the hydro limiter steps, no flattening;
 *  - if either face state has |f| > 1, both states fall back to the two cell
 *    averages (first order) at that face;
 *  - HLL with S_L = -S, S_R = S, S = chat max(sqrt(T_dd(i)), sqrt(T_dd(i+1)))
 *    from the cell-average states at the start of the stage (Eddington
 *    factors frozen, Balsara 1999);
 *  - optical-depth correction eps = min(1, 1/tau), tau = dx (rho_i kR_i +
 *    rho_{i+1} kR_{i+1}) / 2, multiplying the dissipation term, switched off
 *    (eps = 1) where the corrected energy flux would exceed chat max(E_L, E_R). */
static void rad_face_flux(const or_grid *g, const or_params *p, double *const *R,
                          const double *rho, int b, const int c[3], int d, int first,
                          double Fout[NRAD]) {
  double w[NRAD][6], wL[NRAD], wR[NRAD], dummy;
  gather_rad(g, p, R, b, c, d, first, w);
  for (int v = 0; v < NRAD; ++v) {
    recon_cell(p, &w[v][0], &dummy, &wL[v]);
    recon_cell(p, &w[v][1], &wR[v], &dummy);
  }
  double fL2 = (wL[1] * wL[1] + wL[2] * wL[2]) + wL[3] * wL[3];
  double fR2 = (wR[1] * wR[1] + wR[2] * wR[2]) + wR[3] * wR[3];
  if (fL2 > 1.0 || fR2 > 1.0) {
    for (int v = 0; v < NRAD; ++v) {
      wL[v] = w[v][2];
      wR[v] = w[v][3];
    }
  }
  double UL[NRAD], UR[NRAD], FL[NRAD], FR[NRAD];
  rad_state(p, wL, d, UL, FL);
  rad_state(p, wR, d, UR, FR);
  /* wavespeed from the cell-average Eddington factors */
  double TA[9], TB[9];
  double fA[3] = {w[1][2], w[2][2], w[3][2]}, fB[3] = {w[1][3], w[2][3], w[3][3]};
  or_eddington_tensor(p->closure, fA, TA);
  or_eddington_tensor(p->closure, fB, TB);
  double S = p->chat * dmax(sqrt(TA[4 * d]), sqrt(TB[4 * d]));
  double eps = 1.0;
  if (p->tau_correction) {
    int cA[3] = {c[0], c[1], c[2]}, cB[3] = {c[0], c[1], c[2]};
    cA[d] += first + 2;
    cB[d] += first + 3;
    double rA = cell_value(g, p, rho, 0, b, cA);
    double rB = cell_value(g, p, rho, 0, b, cB);
    double tau = p->dx[d] * 0.5 * (rA * kappa_of(p, p->kappa_R, rA) + rB * kappa_of(p, p->kappa_R, rB));
    if (tau > 1.0) eps = 1.0 / tau;
  }
  for (int v = 0; v < NRAD; ++v) Fout[v] = 0.5 * (FL[v] + FR[v]) - 0.5 * S * eps * (UR[v] - UL[v]);
  if (eps < 1.0 && fabs(Fout[0]) > p->chat * dmax(UL[0], UR[0])) {
    for (int v = 0; v < NRAD; ++v) Fout[v] = 0.5 * (FL[v] + FR[v]) - 0.5 * S * (UR[v] - UL[v]);
  }
}

/* The radiation flux through the low face of patch b's cell c along d. */
static void rad_face_flux(const or_grid *g, const or_params *p, double *const *R,
                          const double *rho, int b, const int c[3], int d, int first,
                          double Fout[NRAD]);
void or_rad_face_flux(const or_grid *g, const or_params *p, double *const *R, const double *rho,
                      int32_t b, const int32_t c[3], int32_t d, double F[NRAD]) {
  const int cc[3] = {c[0], c[1], c[2]};
  rad_face_flux(g, p, R, rho, b, cc, d, -3, F);
}

static void rad_rhs_cell(const or_grid *g, const or_params *p, double *const *R,
                         const double *rho, int b, const int c[3], double L[NRAD]) {
  double div[3][NRAD];
  for (int d = 0; d < 3; ++d) {
    double Flo[NRAD], Fhi[NRAD];
    rad_face_flux(g, p, R, rho, b, c, d, -3, Flo);
    rad_face_flux(g, p, R, rho, b, c, d, -2, Fhi);
    for (int v = 0; v < NRAD; ++v) div[d][v] = (Fhi[v] - Flo[v]) / p->dx[d];
  }
  for (int v = 0; v < NRAD; ++v) L[v] = -((div[0][v] + div[1][v]) + div[2][v]);
}

static void rad_stage_cell(const or_grid *g, const or_params *p, int b, const int c[3],
                           void *vctx) {
  stage_ctx *s = (stage_ctx *)vctx;
  double L[NRAD];
  int64_t e = cell_index(g, b, c[0], c[1], c[2]);
  if (s->stage == 1) {
    rad_rhs_cell(g, p, s->U0, s->rho, b, c, L);
    for (int v = 0; v < NRAD; ++v) s->Uout[v][e] = s->U0[v][e] + s->dt * L[v];
  } else {
    rad_rhs_cell(g, p, s->U1, s->rho, b, c, L);
    for (int v = 0; v < NRAD; ++v)
      s->Uout[v][e] = 0.5 * s->U0[v][e] + 0.5 * (s->U1[v][e] + s->dt * L[v]);
  }
}

/* One radiation RK2-SSP stage (Sec. 2.2.2, same integrator as the hydro). */
int or_rad_stage(const or_grid *g, const or_params *p, int stage, double *const *R0,
                 double *const *R1, double *const *Rout, const double *rho, double dt,
                 int64_t ncell, const int32_t *cells) {
  stage_ctx s = {stage, R0, R1, Rout, dt, rho, NRAD, NULL};
  for_cells(g, p, ncell, cells, rad_stage_cell, &s);
  return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* matter-radiation exchange (Sec. 2.2.3)                                    */
/* ------------------------------------------------------------------------ */

/* gas temperature and d(T^4)/dE_g for the two equations of state */
static void eos_T4(const or_params *p, double rho, double Eg, double *T4, double *dT4dEg) {
  if (p->eos == 1) {
    /* E_g = alpha T^4 / 4 (eq. heat_capacity) */
    *T4 = 4.0 * Eg / p->alpha_eos;
    *dT4dEg = 4.0 / p->alpha_eos;
  } else {
    /* gamma-law: T = E_g / (rho c_v) */
    double T = Eg / (rho * p->c_v);
    *T4 = T * T * T * T;
    *dT4dEg = 4.0 * T * T * T / (rho * p->c_v);
  }
}

/* Implicit energy exchange of one cell (Howell & Greenough 2003 extended to
 * the RSLA, Sec. 2.2.3).  Residuals
 *   F_G = (E_g - E_g0) + (c/chat) R,   F_R = (E_r - E_r0) - R,
 *   R   = dt rho kappa_P (chat a_r T^4 - chat E_r)
 * Reading: the garbled '4 pi B' of the paper's R is chat a_r T^4, the only
 * reading that agrees with eq. rad_energy and with the closed form
 * eq. rsla_temperature.  Jacobian entries and the update follow
 * eqs. delta_er and delta_eg with eta = -(dF_R/dE_g)/(dF_G/dE_g); kappa does
 * not depend on T here, so dkappa/dT = 0.  The convergence test
 * |F_G/E_tot| < eps and |(c/chat) F_R/E_tot| < eps with E_tot = E_g0 +
 * (c/chat)(E_r0 + S) is made on the residuals of each iterate; reading: the Newton
 * update computed from the iterate whose residuals pass is still applied,
 * and the iteration then stops.  S is the optional source of the radiation
 * energy residual, F_R = (E_r - E_r0) - (R + S); it does not depend on the
 * iterate, so the Jacobian is unchanged.  Returns the number of iterations,
 * or -1 after max_iter iterations without convergence. */
int or_exchange_energy_src(const or_params *p, double rho, double Eg0, double Er0, double dt,
                           double S, double *Eg_out, double *Er_out) {
  double kP = kappa_of(p, p->kappa_P, rho);
  double cr = p->c / p->chat;
  /* E_tot = E_g^(t) + (c/chat)(E_r^(t) + S), the paper's definition */
  double Etot = Eg0 + cr * (Er0 + S);
  double Eg = Eg0, Er = Er0;
  int it = 0, converged = 0;
  for (it = 0; it < p->max_iter; ++it) {
    double T4, dT4;
    eos_T4(p, rho, Eg, &T4, &dT4);
    double R = dt * rho * kP * (p->chat * p->a_r * T4 - p->chat * Er);
    double FG = (Eg - Eg0) + cr * R;
    double RS = R;
    if (S != 0.0) RS = R + S; /* the source, when there is one */
    double FR = (Er - Er0) - RS;
    converged = fabs(FG / Etot) < p->eps_newton && fabs(cr * FR / Etot) < p->eps_newton;
    double dRdEg = dt * rho * kP * p->chat * p->a_r * dT4;
    double dFG_dEg = 1.0 + cr * dRdEg;
    double dFG_dEr = -p->c * dt * rho * kP;
    double dFR_dEg = -dRdEg;
    double dFR_dEr = 1.0 + p->chat * dt * rho * kP;
    double eta = -dFR_dEg / dFG_dEg;
    double dEr = -(FR + eta * FG) / (dFR_dEr + eta * dFG_dEr);
    double dEg = -(FG + dEr * dFG_dEr) / dFG_dEg;
    Er += dEr;
    Eg += dEg;
    if (converged) break;
  }
  *Eg_out = Eg;
  *Er_out = Er;
  return converged ? it + 1 : -1;
}

int or_exchange_energy(const or_params *p, double rho, double Eg0, double Er0, double dt,
                       double *Eg_out, double *Er_out) {
  return or_exchange_energy_src(p, rho, Eg0, Er0, dt, 0.0, Eg_out, Er_out);
}

typedef struct {
  double *const *U;
  double *const *R;
  double dt;
  const double *src; /* emissivity j per cell, or NULL */
  int status;
  int64_t first_bad;
  int max_it;
  int64_t total_it;
} exch_ctx;

/* Exchange of one cell: energy (Newton), then the flux source by backward
 * Euler F <- F / (1 + rho kappa_F chat dt) with kappa_F = kappa_R at the new
 * temperature, the equal and opposite momentum change (rho v) -= dF/(chat c),
 * and the work term through the kinetic energy change (Sec. 2.2.3). */
static void exchange_cell(const or_grid *g, const or_params *p, int b, const int c[3],
                          void *vctx) {
  exch_ctx *x = (exch_ctx *)vctx;
  int64_t e = cell_index(g, b, c[0], c[1], c[2]);
  double rho = x->U[0][e];
  double m[3] = {x->U[1][e], x->U[2][e], x->U[3][e]};
  double E = x->U[4][e];
  double Ekin0 = 0.5 * ((m[0] * m[0] + m[1] * m[1]) + m[2] * m[2]) / rho;
  double Eg0 = E - Ekin0;
  double Er0 = x->R[0][e];
  double Eg, Er;
  /* reading: the source is an emissivity j (energy per volume per time, in
   * the physical energy equation); in the reduced-speed system it enters the
   * radiation energy as S = dt (chat/c) j, like the emission part of R */
  double S = x->src ? x->dt * (p->chat / p->c) * x->src[e] : 0.0;
  int it = or_exchange_energy_src(p, rho, Eg0, Er0, x->dt, S, &Eg, &Er);
  if (it < 0) {
    x->status |= 1 << OR_ENOCONV;
    if (x->first_bad < 0) x->first_bad = e;
  } else {
    x->total_it += it;
    if (it > x->max_it) x->max_it = it;
  }
  double kF = kappa_of(p, p->kappa_R, rho);
  double F0[3] = {x->R[1][e], x->R[2][e], x->R[3][e]};
  double mn[3];
  for (int i = 0; i < 3; ++i) {
    double Fn = F0[i] / (1.0 + rho * kF * p->chat * x->dt);
    double dF = Fn - F0[i];
    mn[i] = m[i] - dF / (p->chat * p->c);
    x->R[1 + i][e] = Fn;
    x->U[1 + i][e] = mn[i];
  }
  double Ekin1 = 0.5 * ((mn[0] * mn[0] + mn[1] * mn[1]) + mn[2] * mn[2]) / rho;
  double dEkin = Ekin1 - Ekin0;
  x->U[4][e] = Eg + (Ekin0 + dEkin);
  x->R[0][e] = Er - (p->chat / p->c) * dEkin;
  if (!(Eg > 0.0) || !(x->R[0][e] > 0.0)) {
    x->status |= 1 << OR_ENEGATIVE;
    if (x->first_bad < 0) x->first_bad = e;
  }
}

/* out_info[0] = status bits, [1] = first bad element, [2] = max iterations,
 * [3] = total iterations */
int or_exchange(const or_grid *g, const or_params *p, double *const *U, double *const *R,
                double dt, int64_t ncell, const int32_t *cells, const double *src,
                int64_t out_info[4]) {
  exch_ctx x = {U, R, dt, src, 0, -1, 0, 0};
  if (cells) {
    for_cells(g, p, ncell, cells, exchange_cell, &x);
  } else {
    /* one status record per z-plane, combined in the serial plane order (the
     * first failing element is the one a serial sweep meets first) */
    int64_t np;
    or_plane *pl = grid_planes(g, 0, 0, &np);
    exch_ctx *px = (exch_ctx *)malloc((size_t)(np > 0 ? np : 1) * sizeof(exch_ctx));
#pragma omp parallel for schedule(dynamic, 1) num_threads(or_nthreads) if (or_nthreads > 1)
    for (int64_t t = 0; t < np; ++t) {
      px[t] = x;
      for_plane(g, p, pl[t].b, pl[t].k, exchange_cell, &px[t]);
    }
    for (int64_t t = 0; t < np; ++t) {
      x.status |= px[t].status;
      if (x.first_bad < 0) x.first_bad = px[t].first_bad;
      if (px[t].max_it > x.max_it) x.max_it = px[t].max_it;
      x.total_it += px[t].total_it;
    }
    free(px);
    free(pl);
  }
  if (out_info) {
    out_info[0] = x.status;
    out_info[1] = x.first_bad;
    out_info[2] = x.max_it;
    out_info[3] = x.total_it;
  }
  return (x.status & (1 << OR_ENOCONV)) ? OR_ENOCONV
         : (x.status & (1 << OR_ENEGATIVE)) ? OR_ENEGATIVE
                                            : OR_OK;
}

/* Closed-system relaxation of one uniform cell (no transport): apply the
 * exchange nsteps times with a constant dt, as in the radiation-matter
 * exchange test of Sec. 3.2.3, recording E_g after every step. */
int or_relax_cell(const or_params *p, double rho, double Eg, double Er, double dt,
                  int64_t nsteps, double *Eg_hist, double *Er_hist) {
  for (int64_t n = 0; n < nsteps; ++n) {
    double Egn, Ern;
    if (or_exchange_energy(p, rho, Eg, Er, dt, &Egn, &Ern) < 0) return OR_ENOCONV;
    Eg = Egn;
    Er = Ern;
    if (Eg_hist) Eg_hist[n] = Eg;
    if (Er_hist) Er_hist[n] = Er;
  }
  return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* whole step and conservation sums                                          */
/* ------------------------------------------------------------------------ */

/* ghost cells as a stencil read sees them (the stages themselves read
 * through the boundary resolver and do not need this) */
static void fill_all(const or_grid *g, const or_params *p, double *const *f, int nf, int fid0) {
  or_fill_ghosts_bc(g, p, f, nf, fid0);
}

/* One hydro step, then N_sub radiation substeps, each ending with the local
 * exchange (operator split, Sec. 2.2 and Sec. 2.2.3).  R == NULL or
 * hydro_only runs the hydro step alone.  scratch must hold 9 arrays of the
 * field length.  out[0..2] = dt, N_sub, dt_rad; info as or_exchange. */
int or_step(const or_grid *g, const or_params *p, double *const *U, double *const *R,
            double *const *scratch, const double *src, double out[3], int64_t info[4]) {
  double ts[3];
  or_timestep(g, p, U, ts);
  double dt = ts[0];
  double *const *U1 = scratch;
  fill_all(g, p, U, NHYD, 0);
  or_hydro_stage(g, p, 1, U, NULL, U1, dt, 0, NULL);
  fill_all(g, p, U1, NHYD, 0);
  or_hydro_stage(g, p, 2, U, U1, U, dt, 0, NULL);
  int rc = OR_OK;
  int64_t tot[4] = {0, -1, 0, 0};
  if (R && !p->hydro_only) {
    double *const *R1 = scratch + NHYD;
    fill_all(g, p, U, NHYD, 0);
    int nsub = (int)ts[1];
    for (int s = 0; s < nsub; ++s) {
      fill_all(g, p, R, NRAD, NHYD);
      or_rad_stage(g, p, 1, R, NULL, R1, U[0], ts[2], 0, NULL);
      fill_all(g, p, R1, NRAD, NHYD);
      or_rad_stage(g, p, 2, R, R1, R, U[0], ts[2], 0, NULL);
      int64_t inf[4];
      int r = or_exchange(g, p, U, R, ts[2], 0, NULL, src, inf);
      if (r != OR_OK && rc == OR_OK) rc = r;
      tot[0] |= inf[0];
      if (tot[1] < 0) tot[1] = inf[1];
      if (inf[2] > tot[2]) tot[2] = inf[2];
      tot[3] += inf[3];
    }
  }
  if (out) memcpy(out, ts, sizeof(ts));
  if (info) memcpy(info, tot, sizeof(tot));
  return rc;
}

/* Neumaier-compensated sums over interior cells, times the cell volume:
 *  [0] rho, [1..3] m, [4] E, [5] E_r, [6..8] F, [9] E + (c/chat) E_r,
 *  [10..12] m + F/(c chat).  R may be NULL (radiation sums are then 0). */
void or_conserved_sums(const or_grid *g, const or_params *p, double *const *U,
                       double *const *R, double out[NSUMS]) {
  double s[NSUMS], comp[NSUMS];
  memset(s, 0, sizeof(s));
  memset(comp, 0, sizeof(comp));
  double vol = p->dx[0] * p->dx[1] * p->dx[2];
  for (int b = 0; b < g->nbox; ++b) {
    const int32_t *n = g->n + 3 * b;
    for (int k = 0; k < n[2]; ++k)
      for (int j = 0; j < n[1]; ++j)
        for (int i = 0; i < n[0]; ++i) {
          int64_t e = cell_index(g, b, i, j, k);
          double x[NSUMS];
          for (int v = 0; v < NHYD; ++v) x[v] = U[v][e];
          for (int v = 0; v < NRAD; ++v) x[NHYD + v] = R ? R[v][e] : 0.0;
          x[9] = x[4] + (p->c / p->chat) * x[5];
          for (int a = 0; a < 3; ++a) x[10 + a] = x[1 + a] + x[6 + a] / (p->c * p->chat);
          for (int v = 0; v < NSUMS; ++v) {
            double t = s[v] + x[v];
            if (fabs(s[v]) >= fabs(x[v]))
              comp[v] += (s[v] - t) + x[v];
            else
              comp[v] += (x[v] - t) + s[v];
            s[v] = t;
          }
        }
  }
  for (int v = 0; v < NSUMS; ++v) out[v] = (s[v] + comp[v]) * vol;
}
