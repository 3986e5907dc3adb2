// qk_amr.cu -- two-level mesh refinement over two libqk contexts (Berger &
// Colella 1989, as Sec. 2.2 of arXiv:2110.01792 and its level
// synchronisation apply it): the fine level's ghost cells outside the fine
// region from conservative linear interpolation of the coarse state (in
// space and time), the flux registers at the coarse-fine faces, the reflux
// of their mismatch into the adjacent coarse cells, and the average of the
// fine cells down onto the coarse cells they cover.  The stage kernels of
// each level are the ordinary ones; this file adds the operations between
// levels, each one launch over precomputed per-cell or per-face lists (one
// thread per destination, fixed summation order: deterministic, no atomics).
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "qk_ctx.cuh"
#include "qk_rad.cuh"

namespace qk {

struct CfGhost {
  long long fe, ce;  // fine ghost element, coarse parent element
  long long cs[3];   // coarse element steps along x, y, z
  int oct;           // bit d: the fine cell is the upper child of its parent along d
};
struct RegFace {
  long long e[4];  // element of the high-side cell of each face (1 coarse or 4 fine)
  long long step;  // element step along d in that patch
  int d;
};
struct RefluxCell {
  long long ce;  // uncovered coarse cell next to the fine region
  int f0, nf;    // its faces: ids rf[f0 .. f0+nf)
};
struct AvgCell {
  long long ce, fe;  // coarse cell; its fine child (0, 0, 0)
  long long fs[3];   // fine element steps along x, y, z
};

template <typename T> struct F9 { T *f[9]; };

// Monotonized-central slope of two one-sided differences (the paper's PLM
// limiter): 0 unless they share a sign, else sign * min(2|a|, 2|b|, |a+b|/2).
template <typename T> __device__ __forceinline__ T mc_slope(T a, T b) {
  if (!(a * b > T(0))) return T(0);
  const T m = min(min(T(2) * fabs(a), T(2) * fabs(b)), T(0.5) * fabs(a + b));
  return (a + b) > T(0) ? m : -m;
}

// Fine ghost cells outside the fine region: the coarse state at
// (1 - alpha) old + alpha new, interpolated linearly with MC-limited slopes
// toward the fine cell (a quarter slope per axis; conservative: the eight
// children's offsets cancel).
template <typename T>
__global__ void __launch_bounds__(256) cf_interp_kernel(const CfGhost *g, long long n,
                                                        F9<const T> oldv, F9<const T> newv,
                                                        T alpha, F9<T> fine, int first, int nf) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const CfGhost h = g[i];
    for (int k = 0; k < nf; ++k) {
      const T *o = oldv.f[first + k], *w = newv.f[first + k];
      const T u = (T(1) - alpha) * o[h.ce] + alpha * w[h.ce];
      T v = u;
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        const T up = (T(1) - alpha) * o[h.ce + h.cs[d]] + alpha * w[h.ce + h.cs[d]];
        const T um = (T(1) - alpha) * o[h.ce - h.cs[d]] + alpha * w[h.ce - h.cs[d]];
        v = v + (((h.oct >> d) & 1) ? T(0.25) : T(-0.25)) * mc_slope<T>(up - u, u - um);
      }
      fine.f[k][h.fe] = v;
    }
  }
}

// Hydro flux through the low face (along d) of the cell at element e, with
// the stage's arithmetic: primitives of the six cells e-3s .. e+2s, the
// reconstruction of the two face states, the flattening blend (coefficients
// of the stage just run), HLLC.
template <typename T, int D>
__device__ __forceinline__ void hydro_face_at(const F5<const T> &U, const T *chi,
                                              const qk_params &p, long long e, long long s,
                                              T F[5]) {
  T q[6][5];
#pragma unroll
  for (int o = 0; o < 6; ++o) {
    const long long c = e + (o - 3) * s;
    T u[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) u[v] = U.f[v][c];
    con2prim<T>(u, (T)(p.gamma - 1.0), q[o]);
  }
  T wL[5], wR[5], dummy;
#pragma unroll
  for (int v = 0; v < 5; ++v) {
    recon<T>(p.recon, q[0][v], q[1][v], q[2][v], q[3][v], q[4][v], dummy, wL[v]);
    recon<T>(p.recon, q[1][v], q[2][v], q[3][v], q[4][v], q[5][v], wR[v], dummy);
  }
  if (chi) {
    const T ca = chi[e - s], cb = chi[e];
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      wL[v] = ca * wL[v] + (T(1) - ca) * q[2][v];
      wR[v] = cb * wR[v] + (T(1) - cb) * q[3][v];
    }
  }
  const T gamma = (T)p.gamma;
  const T gm1inv = (T)(1.0 / (p.gamma - 1.0));
  const T g1 = (T)((p.gamma + 1.0) / (2.0 * p.gamma));
  hllc<T, D>(wL, wR, gamma, gm1inv, g1, F);
}

// Radiation flux through the low face of the cell at element e: E_r and
// f = F/(c E_r) of the six cells, reconstruction, the wavespeed from the two
// cell averages, rho kappa_R of the two cells, and the stage's face function.
template <typename T, int D, int CL>
__device__ __forceinline__ void rad_face_at(const F4<const T> &R, const T *rho,
                                            const qk_params &p, long long e, long long s,
                                            T out[4]) {
  const T c = (T)p.c, chat = (T)p.chat;
  T pr[6][4];
#pragma unroll
  for (int o = 0; o < 6; ++o) {
    const long long x = e + (o - 3) * s;
    const T E = R.f[0][x];
    const T inv = qrcp(c * E);
    pr[o][0] = E;
    pr[o][1] = R.f[1][x] * inv;
    pr[o][2] = R.f[2][x] * inv;
    pr[o][3] = R.f[3][x] * inv;
  }
  T wL[4], wR[4], dummy;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    recon<T>(p.recon, pr[0][q], pr[1][q], pr[2][q], pr[3][q], pr[4][q], dummy, wL[q]);
    recon<T>(p.recon, pr[1][q], pr[2][q], pr[3][q], pr[4][q], pr[5][q], wR[q], dummy);
  }
  T S;
  if constexpr (sizeof(T) == 8) {
    T aa, ba, ab, bb;
    closure_ab<T, CL>(pr[2][1], pr[2][2], pr[2][3], aa, ba);
    closure_ab<T, CL>(pr[3][1], pr[3][2], pr[3][3], ab, bb);
    const T fa = pr[2][1 + D], fb = pr[3][1 + D];
    S = rad_speed<T>(aa + ba * fa * fa, ab + bb * fb * fb, chat);
  } else {
    S = chat * max(qsqrt(eddington_diag<T, D, CL>(pr[2][1], pr[2][2], pr[2][3])),
                   qsqrt(eddington_diag<T, D, CL>(pr[3][1], pr[3][2], pr[3][3])));
  }
  const T ra = rho[e - s], rb = rho[e];
  const T rka = ra * kappa_of<T>(p, p.kappa_R, ra), rkb = rb * kappa_of<T>(p, p.kappa_R, rb);
  rad_face_hll<T, D, CL>(
      wL, wR,
      [&](T *l, T *r) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          l[q] = pr[2][q];
          r[q] = pr[3][q];
        }
      },
      S, rka, rkb, (T)p.dx[D], c, chat, T(0.5) * chat / c, T(0.5) * c * chat, p.tau_correction,
      out);
}

// Flux register accumulation: for every coarse-fine face (one thread each),
// reg += w * (flux through the coarse face), or for the fine level
// reg += (w / 4) * (flux through each of the four fine faces in turn).
template <typename T>
__global__ void __launch_bounds__(256) reg_hydro_kernel(const RegFace *faces, int n, int nsub,
                                                        F5<const T> U, const T *chi, qk_params p,
                                                        double w, double *reg) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const RegFace fc = faces[i];
    double acc[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) acc[v] = reg[9 * i + v];
    for (int k = 0; k < nsub; ++k) {
      T F[5];
      if (fc.d == 0) hydro_face_at<T, 0>(U, chi, p, fc.e[k], fc.step, F);
      else if (fc.d == 1) hydro_face_at<T, 1>(U, chi, p, fc.e[k], fc.step, F);
      else hydro_face_at<T, 2>(U, chi, p, fc.e[k], fc.step, F);
#pragma unroll
      for (int v = 0; v < 5; ++v) acc[v] += w * (double)F[v];
    }
#pragma unroll
    for (int v = 0; v < 5; ++v) reg[9 * i + v] = acc[v];
  }
}

template <typename T, int CL>
__global__ void __launch_bounds__(256) reg_rad_kernel(const RegFace *faces, int n, int nsub,
                                                      F4<const T> R, const T *rho, qk_params p,
                                                      double w, double *reg) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const RegFace fc = faces[i];
    double acc[4];
#pragma unroll
    for (int v = 0; v < 4; ++v) acc[v] = reg[9 * i + 5 + v];
    for (int k = 0; k < nsub; ++k) {
      T F[4];
      if (fc.d == 0) rad_face_at<T, 0, CL>(R, rho, p, fc.e[k], fc.step, F);
      else if (fc.d == 1) rad_face_at<T, 1, CL>(R, rho, p, fc.e[k], fc.step, F);
      else rad_face_at<T, 2, CL>(R, rho, p, fc.e[k], fc.step, F);
#pragma unroll
      for (int v = 0; v < 4; ++v) acc[v] += w * (double)F[v];
    }
#pragma unroll
    for (int v = 0; v < 4; ++v) reg[9 * i + 5 + v] = acc[v];
  }
}

// Reflux: each uncovered coarse cell next to the fine region gets, face by
// face in id order, -side (fine - coarse flux integral) / dx_d.
template <typename T>
__global__ void __launch_bounds__(256) reflux_kernel(const RefluxCell *cells, int n,
                                                     const int *rf, const int *fd,
                                                     const double *fside, const double *reg_c,
                                                     const double *reg_f, F9<T> U, int nf,
                                                     double idx0, double idx1, double idx2) {
  const double idx[3] = {idx0, idx1, idx2};
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const RefluxCell rc = cells[i];
    for (int v = 0; v < nf; ++v) {
      double u = (double)U.f[v][rc.ce];
      for (int j = 0; j < rc.nf; ++j) {
        const int f = rf[rc.f0 + j];
        u += -fside[f] * (reg_f[9 * f + v] - reg_c[9 * f + v]) * idx[fd[f]];
      }
      U.f[v][rc.ce] = (T)u;
    }
  }
}

// Average down: every covered coarse cell becomes the mean of its 8 fine
// cells, summed ((000 + 100) + (010 + 110)) + ((001 + 101) + (011 + 111)).
template <typename T>
__global__ void __launch_bounds__(256) avg_down_kernel(const AvgCell *cells, long long n,
                                                       F9<const T> fine, F9<T> coarse, int nf) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const AvgCell a = cells[i];
    const long long sx = a.fs[0], sy = a.fs[1], sz = a.fs[2];
    for (int v = 0; v < nf; ++v) {
      const T *f = fine.f[v];
      const long long e = a.fe;
      const double s = (((double)f[e] + (double)f[e + sx]) + ((double)f[e + sy] + (double)f[e + sy + sx])) +
                       (((double)f[e + sz] + (double)f[e + sz + sx]) +
                        ((double)f[e + sz + sy] + (double)f[e + sz + sy + sx]));
      coarse.f[v][a.ce] = (T)(0.125 * s);
    }
  }
}

static int grid_for(long long n) {
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  long long want = (n + 255) / 256;
  return (int)std::max<long long>(1, std::min<long long>(want, (long long)nsm * 8));
}

}  // namespace qk

struct qk_amr {
  qk_ctx *c = nullptr, *f = nullptr;
  CfGhost *d_cf = nullptr;
  long long ncf = 0;
  RegFace *d_cface = nullptr, *d_fface = nullptr;
  int nfaces = 0;
  RefluxCell *d_rcell = nullptr;
  int nrcell = 0;
  int *d_rf = nullptr, *d_fd = nullptr;
  double *d_fside = nullptr;
  AvgCell *d_avg = nullptr;
  long long navg = 0;
  double *d_reg_c = nullptr, *d_reg_f = nullptr;
  std::string err;
};

static thread_local std::string g_amr_err = "qk_amr: null handle";

static int afail(qk_amr *a, int code, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  if (a) a->err = buf;
  else g_amr_err = buf;
  return code;
}

template <typename T> static int aupload(qk_amr *a, T **dst, const std::vector<T> &v) {
  size_t n = std::max<size_t>(v.size(), 1) * sizeof(T);
  cudaError_t e = cudaMalloc((void **)dst, n);
  if (e == cudaSuccess && !v.empty())
    e = cudaMemcpy(*dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return afail(a, QK_ECUDA, "upload: %s", cudaGetErrorString(e));
  return QK_OK;
}

static void arelease(qk_amr *a) {
  cudaFree(a->d_cf);
  cudaFree(a->d_cface);
  cudaFree(a->d_fface);
  cudaFree(a->d_rcell);
  cudaFree(a->d_rf);
  cudaFree(a->d_fd);
  cudaFree(a->d_fside);
  cudaFree(a->d_avg);
  cudaFree(a->d_reg_c);
  cudaFree(a->d_reg_f);
}

// element of local cell (x, y, z) (interior coordinates, ghosts negative) of patch b
static long long elem_of(const qk_ctx *c, int b, int x, int y, int z) {
  const qk_box &q = c->boxes[b];
  const long long sx = q.n[0] + 2 * c->ng, sy = q.n[1] + 2 * c->ng;
  return q.offset + ((long long)(z + c->ng) * sy + (y + c->ng)) * sx + (x + c->ng);
}

static long long step_of(const qk_ctx *c, int b, int d) {
  const qk_box &q = c->boxes[b];
  const long long sx = q.n[0] + 2 * c->ng, sy = q.n[1] + 2 * c->ng;
  return d == 0 ? 1 : (d == 1 ? sx : sx * sy);
}

static int wrapi(int a, int n) {
  int r = a % n;
  return r < 0 ? r + n : r;
}

template <typename T>
static void launch_reg(qk_amr *a, int level, int kind, void *const *fields, const void *rho,
                       double w, cudaStream_t s) {
  qk_ctx *L = level ? a->f : a->c;
  const RegFace *faces = level ? a->d_fface : a->d_cface;
  double *reg = level ? a->d_reg_f : a->d_reg_c;
  const int nsub = level ? 4 : 1;
  const double wk = level ? 0.25 * w : w;
  const int grid = grid_for(a->nfaces);
  if (kind == 0) {
    F5<const T> U{};
    for (int q = 0; q < 5; ++q) U.f[q] = (const T *)fields[q];
    const T *chi = L->p.flattening ? (const T *)L->chi : nullptr;
    reg_hydro_kernel<T><<<grid, 256, 0, s>>>(faces, a->nfaces, nsub, U, chi, L->p, wk, reg);
  } else {
    F4<const T> R{};
    for (int q = 0; q < 4; ++q) R.f[q] = (const T *)fields[q];
    if (L->p.closure == QK_CLOSURE_MINERBO)
      reg_rad_kernel<T, QK_CLOSURE_MINERBO><<<grid, 256, 0, s>>>(faces, a->nfaces, nsub, R,
                                                                 (const T *)rho, L->p, wk, reg);
    else if (L->p.closure == QK_CLOSURE_EDDINGTON)
      reg_rad_kernel<T, QK_CLOSURE_EDDINGTON><<<grid, 256, 0, s>>>(faces, a->nfaces, nsub, R,
                                                                   (const T *)rho, L->p, wk, reg);
    else
      reg_rad_kernel<T, QK_CLOSURE_LEVERMORE><<<grid, 256, 0, s>>>(faces, a->nfaces, nsub, R,
                                                                   (const T *)rho, L->p, wk, reg);
  }
}

template <typename T>
static void launch_sync(qk_amr *a, void *const cU[5], void *const cR[4], void *const fU[5],
                        void *const fR[4], cudaStream_t s) {
  F9<T> cf{};
  F9<const T> ff{};
  const int nf = cR ? 9 : 5;
  for (int q = 0; q < 5; ++q) {
    cf.f[q] = (T *)cU[q];
    ff.f[q] = (const T *)fU[q];
  }
  for (int q = 0; cR && q < 4; ++q) {
    cf.f[5 + q] = (T *)cR[q];
    ff.f[5 + q] = (const T *)fR[q];
  }
  const double *dx = a->c->p.dx;
  if (a->nrcell > 0)
    reflux_kernel<T><<<grid_for(a->nrcell), 256, 0, s>>>(a->d_rcell, a->nrcell, a->d_rf, a->d_fd,
                                                         a->d_fside, a->d_reg_c, a->d_reg_f, cf,
                                                         nf, 1.0 / dx[0], 1.0 / dx[1], 1.0 / dx[2]);
  if (a->navg > 0) {
    F9<const T> ffc = ff;
    avg_down_kernel<T><<<grid_for(a->navg), 256, 0, s>>>(a->d_avg, a->navg, ffc, cf, nf);
  }
}

extern "C" {

int qk_amr_init(qk_amr **out, qk_ctx *c, qk_ctx *f) {
  if (!out) return QK_EINVAL;
  *out = nullptr;
  if (!c || !f) return afail(nullptr, QK_EINVAL, "qk_amr_init: NULL context");
  if (c->fp32 != f->fp32) return afail(nullptr, QK_EINVAL, "levels differ in precision");
  if (!c->owner.empty() || !f->owner.empty())
    return afail(nullptr, QK_EINVAL, "refinement levels cannot be sharded contexts");
  if (c->ng != f->ng) return afail(nullptr, QK_EINVAL, "levels differ in ghost width");
  for (int d = 0; d < 3; ++d) {
    if (f->dom[d] != 2 * c->dom[d])
      return afail(nullptr, QK_EINVAL, "axis %d: the fine domain must be twice the coarse", d);
    if (std::fabs(f->p.dx[d] * 2.0 - c->p.dx[d]) > 1e-12 * c->p.dx[d])
      return afail(nullptr, QK_EINVAL, "axis %d: the fine dx must be half the coarse dx", d);
    if (c->p.bc_lo[d] != QK_BC_PERIODIC || c->p.bc_hi[d] != QK_BC_PERIODIC ||
        f->p.bc_lo[d] != QK_BC_PERIODIC || f->p.bc_hi[d] != QK_BC_PERIODIC)
      return afail(nullptr, QK_EINVAL, "refined hierarchies are periodic");
  }
  if (c->partial) return afail(nullptr, QK_EINVAL, "the coarse level must cover the domain");
  for (const qk_box &q : f->boxes)
    for (int d = 0; d < 3; ++d)
      if ((q.lo[d] | q.n[d]) & 1)
        return afail(nullptr, QK_EINVAL, "fine patches must be aligned to coarse cells");
  const int ng = c->ng;
  const int *Dc = c->dom, *Df = f->dom;
  // owner maps: coarse cell -> coarse patch, fine cell -> fine patch (or -1)
  std::vector<int> cown((size_t)Dc[0] * Dc[1] * Dc[2], -1), fown((size_t)Df[0] * Df[1] * Df[2], -1);
  for (int b = 0; b < c->nbox; ++b) {
    const qk_box &q = c->boxes[b];
    for (int z = 0; z < q.n[2]; ++z)
      for (int y = 0; y < q.n[1]; ++y)
        for (int x = 0; x < q.n[0]; ++x)
          cown[((size_t)(q.lo[2] + z) * Dc[1] + (q.lo[1] + y)) * Dc[0] + (q.lo[0] + x)] = b;
  }
  for (int b = 0; b < f->nbox; ++b) {
    const qk_box &q = f->boxes[b];
    for (int z = 0; z < q.n[2]; ++z)
      for (int y = 0; y < q.n[1]; ++y)
        for (int x = 0; x < q.n[0]; ++x)
          fown[((size_t)(q.lo[2] + z) * Df[1] + (q.lo[1] + y)) * Df[0] + (q.lo[0] + x)] = b;
  }
  auto fcov = [&](int x, int y, int z) {
    return fown[((size_t)wrapi(z, Df[2]) * Df[1] + wrapi(y, Df[1])) * Df[0] + wrapi(x, Df[0])] >= 0;
  };
  auto celem = [&](int X, int Y, int Z) {
    X = wrapi(X, Dc[0]);
    Y = wrapi(Y, Dc[1]);
    Z = wrapi(Z, Dc[2]);
    const int q = cown[((size_t)Z * Dc[1] + Y) * Dc[0] + X];
    const qk_box &B = c->boxes[q];
    return std::make_pair(q, elem_of(c, q, X - B.lo[0], Y - B.lo[1], Z - B.lo[2]));
  };
  qk_amr *a = new qk_amr();
  a->c = c;
  a->f = f;
  auto bail = [&](int rc) {
    g_amr_err = a->err.empty() ? std::string("qk_amr_init failed") : a->err;
    arelease(a);
    delete a;
    return rc;
  };
  // fine ghost cells outside the fine region
  std::vector<CfGhost> cf;
  for (int b = 0; b < f->nbox; ++b) {
    const qk_box &q = f->boxes[b];
    for (int z = -ng; z < q.n[2] + ng; ++z)
      for (int y = -ng; y < q.n[1] + ng; ++y)
        for (int x = -ng; x < q.n[0] + ng; ++x) {
          const bool inside = x >= 0 && y >= 0 && z >= 0 && x < q.n[0] && y < q.n[1] && z < q.n[2];
          if (inside) continue;
          const int gx = wrapi(q.lo[0] + x, Df[0]), gy = wrapi(q.lo[1] + y, Df[1]),
                    gz = wrapi(q.lo[2] + z, Df[2]);
          if (fcov(gx, gy, gz)) continue;
          CfGhost h;
          auto pe = celem(gx / 2, gy / 2, gz / 2);
          h.fe = elem_of(f, b, x, y, z);
          h.ce = pe.second;
          for (int d = 0; d < 3; ++d) h.cs[d] = step_of(c, pe.first, d);
          h.oct = (gx & 1) | ((gy & 1) << 1) | ((gz & 1) << 2);
          cf.push_back(h);
        }
  }
  // coarse-fine faces, keyed (d, coarse cell on the high side), in the order
  // of first appearance over fine patches, axes, sides and boundary cells
  std::map<std::pair<int, long long>, int> key;
  std::vector<RegFace> cfaces, ffaces;
  std::vector<int> fcount, fd;
  std::vector<double> fside;
  std::vector<long long> outcell;
  for (int b = 0; b < f->nbox; ++b) {
    const qk_box &q = f->boxes[b];
    for (int d = 0; d < 3; ++d)
      for (int hs = 0; hs < 2; ++hs) {
        int lo3[3] = {0, 0, 0}, hi3[3] = {q.n[0], q.n[1], q.n[2]};
        lo3[d] = hs ? q.n[d] - 1 : 0;
        hi3[d] = lo3[d] + 1;
        for (int z = lo3[2]; z < hi3[2]; ++z)
          for (int y = lo3[1]; y < hi3[1]; ++y)
            for (int x = lo3[0]; x < hi3[0]; ++x) {
              int cl[3] = {x, y, z}, nb[3] = {x, y, z};
              nb[d] += hs ? 1 : -1;
              if (fcov(q.lo[0] + nb[0], q.lo[1] + nb[1], q.lo[2] + nb[2])) continue;
              const int *hc = hs ? nb : cl;
              const int gh[3] = {wrapi(q.lo[0] + hc[0], Df[0]), wrapi(q.lo[1] + hc[1], Df[1]),
                                 wrapi(q.lo[2] + hc[2], Df[2])};
              const int ch[3] = {gh[0] / 2, gh[1] / 2, gh[2] / 2};
              const long long lin = ((long long)ch[2] * Dc[1] + ch[1]) * Dc[0] + ch[0];
              auto it = key.find({d, lin});
              int id;
              if (it == key.end()) {
                id = (int)cfaces.size();
                key[{d, lin}] = id;
                auto pe = celem(ch[0], ch[1], ch[2]);
                RegFace cface{};
                cface.e[0] = pe.second;
                cface.step = step_of(c, pe.first, d);
                cface.d = d;
                cfaces.push_back(cface);
                RegFace fface{};
                fface.step = step_of(f, b, d);
                fface.d = d;
                ffaces.push_back(fface);
                fcount.push_back(0);
                fd.push_back(d);
                int oc[3] = {ch[0], ch[1], ch[2]};
                if (!hs) oc[d] -= 1;  // the uncovered cell is on the face's low side
                fside.push_back(hs ? -1.0 : 1.0);
                outcell.push_back(celem(oc[0], oc[1], oc[2]).second);
              } else {
                id = it->second;
              }
              if (fcount[id] >= 4 || step_of(f, b, d) != ffaces[id].step) {
                a->err = "fine patches must be aligned to coarse cells";
                return bail(QK_EINVAL);
              }
              ffaces[id].e[fcount[id]++] = elem_of(f, b, hc[0], hc[1], hc[2]);
            }
      }
  }
  for (int id = 0; id < (int)fcount.size(); ++id)
    if (fcount[id] != 4) {
      a->err = "a coarse-fine face without its four fine faces";
      return bail(QK_EINVAL);
    }
  // reflux lists: faces grouped by the uncovered coarse cell they correct
  std::vector<RefluxCell> rcells;
  std::vector<int> rf;
  {
    std::map<long long, std::vector<int>> by;
    std::vector<long long> order;
    for (int id = 0; id < (int)outcell.size(); ++id) {
      auto &v = by[outcell[id]];
      if (v.empty()) order.push_back(outcell[id]);
      v.push_back(id);
    }
    for (long long ce : order) {
      const auto &v = by[ce];
      rcells.push_back(RefluxCell{ce, (int)rf.size(), (int)v.size()});
      rf.insert(rf.end(), v.begin(), v.end());
    }
  }
  // average down: every coarse cell under a fine patch
  std::vector<AvgCell> avg;
  for (int b = 0; b < f->nbox; ++b) {
    const qk_box &q = f->boxes[b];
    for (int z = 0; z < q.n[2]; z += 2)
      for (int y = 0; y < q.n[1]; y += 2)
        for (int x = 0; x < q.n[0]; x += 2) {
          AvgCell av;
          av.ce = celem((q.lo[0] + x) / 2, (q.lo[1] + y) / 2, (q.lo[2] + z) / 2).second;
          av.fe = elem_of(f, b, x, y, z);
          for (int d = 0; d < 3; ++d) av.fs[d] = step_of(f, b, d);
          avg.push_back(av);
        }
  }
  a->ncf = (long long)cf.size();
  a->nfaces = (int)cfaces.size();
  a->nrcell = (int)rcells.size();
  a->navg = (long long)avg.size();
  int rc;
  if ((rc = aupload(a, &a->d_cf, cf))) return bail(rc);
  if ((rc = aupload(a, &a->d_cface, cfaces))) return bail(rc);
  if ((rc = aupload(a, &a->d_fface, ffaces))) return bail(rc);
  if ((rc = aupload(a, &a->d_rcell, rcells))) return bail(rc);
  if ((rc = aupload(a, &a->d_rf, rf))) return bail(rc);
  if ((rc = aupload(a, &a->d_fd, fd))) return bail(rc);
  if ((rc = aupload(a, &a->d_fside, fside))) return bail(rc);
  if ((rc = aupload(a, &a->d_avg, avg))) return bail(rc);
  std::vector<double> zeros((size_t)std::max(1, a->nfaces) * 9, 0.0);
  if ((rc = aupload(a, &a->d_reg_c, zeros))) return bail(rc);
  if ((rc = aupload(a, &a->d_reg_f, zeros))) return bail(rc);
  *out = a;
  return QK_OK;
}

void qk_amr_destroy(qk_amr *a) {
  if (!a) return;
  arelease(a);
  delete a;
}

const char *qk_amr_last_error(const qk_amr *a) { return a ? a->err.c_str() : g_amr_err.c_str(); }

int qk_amr_info(const qk_amr *a, int64_t *n_cf_ghosts, int64_t *n_faces, int64_t *n_covered) {
  if (!a) return QK_EINVAL;
  if (n_cf_ghosts) *n_cf_ghosts = a->ncf;
  if (n_faces) *n_faces = a->nfaces;
  if (n_covered) *n_covered = a->navg;
  return QK_OK;
}

static bool fields_ok(void *const *f, int first, int n) {
  if (!f) return false;
  for (int i = 0; i < n; ++i)
    if (!f[first + i]) return false;
  return true;
}

int qk_amr_interp(qk_amr *a, void *const c_old[9], void *const c_new[9], double alpha,
                  void *const *fine_fields, int32_t first, int32_t nfields, void *stream) {
  if (!a) return QK_EINVAL;
  if (first < 0 || nfields < 1 || first + nfields > 9)
    return afail(a, QK_EINVAL, "fields first .. first+nfields-1 must lie in [0, 9)");
  if (!fields_ok(c_old, first, nfields) || !fields_ok(c_new, first, nfields) ||
      !fields_ok(fine_fields, 0, nfields))
    return afail(a, QK_EINVAL, "a field pointer is NULL");
  if (a->ncf == 0) return QK_OK;
  cudaStream_t s = (cudaStream_t)stream;
  if (a->c->fp32) {
    F9<const float> o{}, w{};
    F9<float> fi{};
    for (int i = 0; i < 9; ++i) {
      o.f[i] = (const float *)c_old[i];
      w.f[i] = (const float *)c_new[i];
    }
    for (int i = 0; i < nfields; ++i) fi.f[i] = (float *)fine_fields[i];
    cf_interp_kernel<float><<<grid_for(a->ncf), 256, 0, s>>>(a->d_cf, a->ncf, o, w, (float)alpha, fi,
                                                             first, nfields);
  } else {
    F9<const double> o{}, w{};
    F9<double> fi{};
    for (int i = 0; i < 9; ++i) {
      o.f[i] = (const double *)c_old[i];
      w.f[i] = (const double *)c_new[i];
    }
    for (int i = 0; i < nfields; ++i) fi.f[i] = (double *)fine_fields[i];
    cf_interp_kernel<double><<<grid_for(a->ncf), 256, 0, s>>>(a->d_cf, a->ncf, o, w, alpha, fi,
                                                              first, nfields);
  }
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? QK_OK : afail(a, QK_ECUDA, "interp: %s", cudaGetErrorString(e));
}

int qk_amr_register(qk_amr *a, int32_t level, int32_t kind, void *const *fields, const void *rho,
                    double weight, void *stream) {
  if (!a) return QK_EINVAL;
  if (level != 0 && level != 1) return afail(a, QK_EINVAL, "level must be 0 (coarse) or 1 (fine)");
  if (kind != 0 && kind != 1) return afail(a, QK_EINVAL, "kind must be 0 (hydro) or 1 (radiation)");
  if (!fields_ok(fields, 0, kind ? 4 : 5)) return afail(a, QK_EINVAL, "a field pointer is NULL");
  if (kind == 1 && !rho) return afail(a, QK_EINVAL, "rho is NULL");
  if (a->nfaces == 0) return QK_OK;
  cudaStream_t s = (cudaStream_t)stream;
  if (a->c->fp32) launch_reg<float>(a, level, kind, fields, rho, weight, s);
  else launch_reg<double>(a, level, kind, fields, rho, weight, s);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? QK_OK : afail(a, QK_ECUDA, "register: %s", cudaGetErrorString(e));
}

int qk_amr_sync(qk_amr *a, void *const cU[5], void *const cR[4], void *const fU[5],
                void *const fR[4], void *stream) {
  if (!a) return QK_EINVAL;
  if (!fields_ok(cU, 0, 5) || !fields_ok(fU, 0, 5)) return afail(a, QK_EINVAL, "a hydro field is NULL");
  if ((cR == nullptr) != (fR == nullptr)) return afail(a, QK_EINVAL, "give radiation on both levels or none");
  if (cR && (!fields_ok(cR, 0, 4) || !fields_ok(fR, 0, 4)))
    return afail(a, QK_EINVAL, "a radiation field is NULL");
  cudaStream_t s = (cudaStream_t)stream;
  if (a->c->fp32) launch_sync<float>(a, cU, cR, fU, fR, s);
  else launch_sync<double>(a, cU, cR, fU, fR, s);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess && a->nfaces > 0) {
    e = cudaMemsetAsync(a->d_reg_c, 0, sizeof(double) * 9 * a->nfaces, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(a->d_reg_f, 0, sizeof(double) * 9 * a->nfaces, s);
  }
  return e == cudaSuccess ? QK_OK : afail(a, QK_ECUDA, "sync: %s", cudaGetErrorString(e));
}

}  // extern "C"
