// qk_cell.cu -- per-cell kernels of the update (arXiv:2110.01792) for sm_103a:
// the implicit matter-radiation exchange (Sec. 2.2.3), the CFL reduction and
// timestep (Sec. 2.2.1, Sec. 2.2.4), the batched ghost fill, and the
// compensated conservation sums.
#include <algorithm>

#include "qk_copy.cuh"
#include "qk_exchange.cuh"

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
// One thread per interior cell (grid-stride over the flat cell index); the
// per-cell arithmetic is in qk_exchange.cuh.
template <int CP>
__global__ void __launch_bounds__(256) exchange_kernel_mixed(Geometry g, qk_params p,
                                                              F5<float> U, F4<float> R,
                                                              const float *src, DtSrc dts,
                                                              Status *st, F5<float> UL,
                                                              F4<float> RL) {
  if (skip_substep(dts)) return;
  const ExK K = make_exk(p);
  const double dt = dt_of(dts);
  const float dtf = (float)dt;
  ExStat xs;
  for (long long cidx = (long long)blockIdx.x * blockDim.x + threadIdx.x; cidx < g.ncells;
       cidx += (long long)gridDim.x * blockDim.x) {
    const long long e = cell_to_elem(g, cidx);
    const float fr[3] = {R.f[1][e], R.f[2][e], R.f[3][e]};
    float fl[3] = {0.0f, 0.0f, 0.0f}, el = 0.0f;
    const float er = R.f[0][e];
    if constexpr (CP) {
      el = lo_get<CP>(RL.f[0], e, er);
      fl[0] = lo_get<CP>(RL.f[1], e, fr[0]);
      fl[1] = lo_get<CP>(RL.f[2], e, fr[1]);
      fl[2] = lo_get<CP>(RL.f[3], e, fr[2]);
    }
    exchange_cell_mixed<CP>(p, K, dt, dtf, U, R, UL, RL, src, e, er, el, fr, fl, xs);
  }
  exchange_status(st, xs.max, xs.flags, xs.bad);
}

template <typename T>
__global__ void __launch_bounds__(256) exchange_kernel(Geometry g, qk_params p, F5<T> U, F4<T> R,
                                                        const T *src, DtSrc dts, Status *st) {
  if (skip_substep(dts)) return;
  const ExK K = make_exk(p);
  const double dt = dt_of(dts);
  ExStat xs;
  for (long long cidx = (long long)blockIdx.x * blockDim.x + threadIdx.x; cidx < g.ncells;
       cidx += (long long)gridDim.x * blockDim.x) {
    const long long e = cell_to_elem(g, cidx);
    const double fr[3] = {load_d(R.f[1], e), load_d(R.f[2], e), load_d(R.f[3], e)};
    exchange_cell<T>(p, K, dt, U, R, src, e, load_d(R.f[0], e), fr, xs);
  }
  exchange_status(st, xs.max, xs.flags, xs.bad);
}

cudaError_t launch_exchange(int fp32, const Geometry &g, const qk_params &p, void *const *U,
                            void *const *R, const void *src, DtSrc dt, Status *st,
                            cudaStream_t s, void *const *Ulo, void *const *Rlo, int lofmt) {
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
      if (lofmt == 2)
        exchange_kernel_mixed<2><<<grid, 256, 0, s>>>(g, p, u, r, (const float *)src, dt, st,
                                                      ul, rl);
      else
        exchange_kernel_mixed<1><<<grid, 256, 0, s>>>(g, p, u, r, (const float *)src, dt, st,
                                                      ul, rl);
    } else {
      exchange_kernel_mixed<0><<<grid, 256, 0, s>>>(g, p, u, r, (const float *)src, dt, st,
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
  con2prim<float>(u, (float)(gamma - 1.0), w);
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

// 16-byte vector of the field type (4 floats or 2 doubles) and its negation.
template <typename T> struct Vec16;
template <> struct Vec16<float> {
  typedef float4 type;
  static constexpr int n = 4;
  __device__ static float4 neg(float4 v) { return make_float4(-v.x, -v.y, -v.z, -v.w); }
};
template <> struct Vec16<double> {
  typedef double2 type;
  static constexpr int n = 2;
  __device__ static double2 neg(double2 v) { return make_double2(-v.x, -v.y); }
};

template <typename T>
__global__ void __launch_bounds__(256) ghost_fill_kernel(const Copy *copies, const Chunk *chunks,
                                                         F5<T> fa, F4<T> fb, int nf, int first,
                                                         DtSrc pred, int vec_ok) {
  if (skip_substep(pred)) return;
  const Chunk ch = chunks[blockIdx.x];
  const Copy cp = copies[ch.copy];
  const int ncell = cp.ex * cp.ey * cp.ez;
  const int end = min(ncell, ch.start + CHUNK_CELLS);
  if (vec_ok && cp.vec) {
    // rows of 4-element multiples, every row start on a 16-byte boundary (the
    // field pointers are 16-byte aligned): 16-byte loads and stores; the
    // chunk starts on a multiple of 4 cells, so no vector crosses a row
    typedef typename Vec16<T>::type VT;
    constexpr int V = Vec16<T>::n;
    for (int l = ch.start + threadIdx.x * V; l < end; l += blockDim.x * V) {
      const int x = l % cp.ex;
      const int r = l / cp.ex;
      const int y = r % cp.ey;
      const int z = r / cp.ey;
      const long long d = cp.dst + ((long long)z * cp.dsy + y) * cp.dsx + x;
      const long long s = cp.src + z * cp.sz + y * cp.sy + x;
#pragma unroll
      for (int f = 0; f < 9; ++f) {
        if (f >= nf) break;
        T *fld = field_ptr(fa, fb, f);
        const int ax = field_axis(first + f);
        const VT v = *reinterpret_cast<const VT *>(fld + s);
        *reinterpret_cast<VT *>(fld + d) =
            (ax >= 0 && ((cp.flip >> ax) & 1)) ? Vec16<T>::neg(v) : v;
      }
    }
    return;
  }
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
  // the vector path needs every field pointer on a 16-byte boundary
  int vec_ok = 1;
  for (int q = 0; q < nf; ++q)
    if (reinterpret_cast<uintptr_t>(fields[q]) % 16 != 0) vec_ok = 0;
  if (fp32) {
    F5<float> a{}; F4<float> b{};
    for (int q = 0; q < nf && q < 5; ++q) a.f[q] = (float *)fields[q];
    for (int q = 5; q < nf; ++q) b.f[q - 5] = (float *)fields[q];
    ghost_fill_kernel<float><<<nchunks, 256, 0, s>>>(copies, chunks, a, b, nf, first, pred,
                                                     vec_ok);
  } else {
    F5<double> a{}; F4<double> b{};
    for (int q = 0; q < nf && q < 5; ++q) a.f[q] = (double *)fields[q];
    for (int q = 5; q < nf; ++q) b.f[q - 5] = (double *)fields[q];
    ghost_fill_kernel<double><<<nchunks, 256, 0, s>>>(copies, chunks, a, b, nf, first, pred,
                                                      vec_ok);
  }
  return cudaGetLastError();
}

// ------------------------------------------------------- field copies ---
// Host <-> device copies of whole fields by the SMs (loads or stores through
// the host mapping of pinned memory cross the CPU-GPU link in parallel from
// every SM): blockIdx.y is the field, 16-byte words grid-strided over x, the
// tail (bytes mod 16) by the first threads.
__global__ void __launch_bounds__(256) field_copy_kernel(FieldCopies fc, long long n16,
                                                         int tail) {
  const uint4 *src = (const uint4 *)fc.src[blockIdx.y];
  uint4 *dst = (uint4 *)fc.dst[blockIdx.y];
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n16;
       i += (long long)gridDim.x * blockDim.x)
    dst[i] = src[i];
  if (blockIdx.x == 0 && threadIdx.x < tail)
    ((unsigned char *)(dst + n16))[threadIdx.x] = ((const unsigned char *)(src + n16))[threadIdx.x];
}

cudaError_t launch_field_copies(const FieldCopies &fc, int nf, size_t bytes, cudaStream_t s) {
  if (nf < 1 || nf > 9 || bytes == 0) return cudaSuccess;
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const long long n16 = (long long)(bytes / 16);
  const int tail = (int)(bytes % 16);
  long long bx = (n16 + 255) / 256;
  const long long cap = (long long)std::max(nsm, 1) * 8 / nf + 1;  // ~8 CTAs per SM in all
  if (bx > cap) bx = cap;
  if (bx < 1) bx = 1;
  field_copy_kernel<<<dim3((unsigned)bx, (unsigned)nf), 256, 0, s>>>(fc, n16, tail);
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

template <typename T, int CP>
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
    if constexpr (CP != 0) {
#pragma unroll
      for (int q = 0; q < 5; ++q) x[q] += (double)lo_get<CP>(UL.f[q], e, U.f[q][e]);
      if (has_rad) {
#pragma unroll
        for (int q = 0; q < 4; ++q) x[5 + q] += (double)lo_get<CP>(RL.f[q], e, R.f[q][e]);
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
                        cudaStream_t s, void *const *Ulo, void *const *Rlo, int lofmt) {
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
    if (!Ulo)
      sums_kernel<float, 0><<<nblocks, SUM_NT, 0, s>>>(g, cr, icc, u, r, has_rad, partials, ul,
                                                       rl);
    else if (lofmt == 2)
      sums_kernel<float, 2><<<nblocks, SUM_NT, 0, s>>>(g, cr, icc, u, r, has_rad, partials, ul,
                                                       rl);
    else
      sums_kernel<float, 1><<<nblocks, SUM_NT, 0, s>>>(g, cr, icc, u, r, has_rad, partials, ul,
                                                       rl);
  } else {
    F5<double> u, ul{}; F4<double> r{}, rl{};
    for (int q = 0; q < 5; ++q) u.f[q] = (double *)U[q];
    if (has_rad) for (int q = 0; q < 4; ++q) r.f[q] = (double *)R[q];
    sums_kernel<double, 0><<<nblocks, SUM_NT, 0, s>>>(g, cr, icc, u, r, has_rad, partials, ul,
                                                      rl);
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

__global__ void eval_convert_kernel(const float *fi, double *dout, const double *di, float *fout,
                                    long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    if (fi && dout) dout[i] = f2d(fi[i]);
    if (di && fout) fout[i] = d2f_trunc(di[i]);
  }
}

// -------------------------------------------------------- ALU probe ---
// FMA throughput probe: every thread runs QK_FMA_CHAINS independent chains
// a <- a m + c for `iters` steps (2 flops per step and chain) and stores the
// sum of its chains, so that nothing is dead code.  With m = 1 - 2^-20 and
// c = 2^-10 the chains approach c / (1 - m) = 1024 from their start values
// and stay finite and normal.
constexpr int QK_FMA_CHAINS = 8;
template <typename T>
__global__ void __launch_bounds__(256) fma_probe_kernel(long long iters, T *sink) {
  const T m = T(1) - T(1.0 / 1048576.0), c = T(1.0 / 1024.0);
  T a[QK_FMA_CHAINS];
#pragma unroll
  for (int i = 0; i < QK_FMA_CHAINS; ++i) a[i] = T(threadIdx.x % 32 + i);
  for (long long k = 0; k < iters; ++k) {
#pragma unroll
    for (int i = 0; i < QK_FMA_CHAINS; ++i) a[i] = fma(a[i], m, c);
  }
  T sum = T(0);
#pragma unroll
  for (int i = 0; i < QK_FMA_CHAINS; ++i) sum += a[i];
  sink[(long long)blockIdx.x * blockDim.x + threadIdx.x] = sum;
}

}  // namespace qk

extern "C" int qk_fma_probe(int32_t fp64, int64_t iters, void *sink, int64_t sink_len,
                            double *flops, void *stream) {
  if (iters < 1 || !sink || sink_len < 1) return QK_EINVAL;
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return QK_ECUDA;
  // 8 blocks of 256 threads per SM (64 warps), fewer if the sink is smaller
  long long blocks = std::min<long long>(8LL * nsm, sink_len / 256);
  if (blocks < 1) return QK_EINVAL;
  if (fp64)
    qk::fma_probe_kernel<double><<<(int)blocks, 256, 0, (cudaStream_t)stream>>>(iters, (double *)sink);
  else
    qk::fma_probe_kernel<float><<<(int)blocks, 256, 0, (cudaStream_t)stream>>>(iters, (float *)sink);
  if (cudaGetLastError() != cudaSuccess) return QK_ECUDA;
  if (flops) *flops = 2.0 * qk::QK_FMA_CHAINS * (double)iters * (double)(blocks * 256);
  return QK_OK;
}

extern "C" int qk_eval_convert(const float *f_in, double *d_out, const double *d_in, float *f_out,
                               int64_t n, void *stream) {
  if (n < 0) return QK_EINVAL;
  if (n == 0) return QK_OK;
  const long long blocks = std::min<long long>((n + 255) / 256, 152LL * 16);
  qk::eval_convert_kernel<<<(int)blocks, 256, 0, (cudaStream_t)stream>>>(f_in, d_out, d_in, f_out, n);
  return cudaGetLastError() == cudaSuccess ? QK_OK : QK_ECUDA;
}

extern "C" int qk_eval_math(const double *x, int64_t n, double *rcp, double *sqrt_out,
                            void *stream) {
  if (n < 0 || (n > 0 && !x)) return QK_EINVAL;
  if (n == 0) return QK_OK;
  const long long blocks = std::min<long long>((n + 255) / 256, 152LL * 16);
  qk::eval_math_kernel<<<(int)blocks, 256, 0, (cudaStream_t)stream>>>(x, n, rcp, sqrt_out);
  return cudaGetLastError() == cudaSuccess ? QK_OK : QK_ECUDA;
}

