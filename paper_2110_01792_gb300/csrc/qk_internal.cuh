// qk_internal.cuh -- device-side data structures, tile geometry and launch
// declarations shared by the translation units of libqk (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "qk.h"

namespace qk {

// ---------------------------------------------------------------------------
// Tile geometry.  A stage kernel processes one TS^3 block of interior cells of
// one patch at a time (a partial block at a patch edge is masked).  The
// primitive variables of the block and of a HALO-deep "cross" around it (the
// cells a 1-D PPM stencil along x, y or z reaches, never the corners) are
// staged in shared memory once per tile:
//   core      TS^3 slots                 (i, j, k) in [0, TS)^3
//   x-halo    2*HALO*TS*TS slots         i in [-HALO, 0) U [TS, TS+HALO)
//   y-halo, z-halo likewise.
// Reconstruction runs on TS+2 positions per line (-1 .. TS) and the Riemann
// solver on TS+1 faces per line; fluxes stay in shared memory.
// ---------------------------------------------------------------------------
constexpr int TS = 8;
constexpr int HALO = 3;
constexpr int NCORE = TS * TS * TS;
constexpr int NHD = 2 * HALO * TS * TS;
constexpr int NCROSS = NCORE + 3 * NHD;
constexpr int NPOS = TS + 2;
constexpr int NFACE = TS + 1;
constexpr int NREC = NPOS * TS * TS;
constexpr int NIFP = TS + 3;            // PPM interface values per line (FP64)
constexpr int NIF = NIFP * TS * TS;
constexpr int NFLUX = NFACE * TS * TS;

// Column geometry (the plane-marching stage kernels).  A CTA of CW x CW
// threads owns a CW x CW footprint of one patch and marches along z through
// planes [z0, z1): the z stencil lives in a per-thread register window, the
// x and y stencils of the current plane in shared memory (the plane and a
// HALO-deep ring, corners unused).
constexpr int CW = 16;
constexpr int CPW = CW + 2 * HALO;     // plane row length with the ring
constexpr int CNPL = CPW * CPW;        // plane slots
constexpr int CXPOS = CW + 2;          // reconstruction positions per row (cells -1..CW)
constexpr int CXFACE = CW + 1;         // faces per row
constexpr int CNT = CW * CW;           // threads per column CTA
// resident column CTAs per SM the kernels' registers are held to (FP32:
// three, as many as fit beside each other's shared memory; FP64: two), also
// the slots of the host's z-chunk cost model
constexpr int COL_CTAS_FP32 = 3, COL_CTAS_FP64 = 2;
constexpr int CNRING = 4 * HALO * CW;  // ring cells of a plane (x and y sides)

struct Column {
  int box;
  int x0, y0, z0, z1;
};

struct DevBox {
  int lo[3];
  int n[3];
  int sx, sy;          // padded row length and rows per plane (n + 2g)
  long long off;       // element offset of the patch's first cell
  long long cell0;     // number of interior cells in the patches before this one
};

struct Tile {
  int box;
  int x0, y0, z0;      // tile origin in the patch's interior coordinates
};

// One rectangular ghost region copied from an interior region (possibly of
// another patch, possibly a periodic image).  Element offsets are absolute.
struct Copy {
  long long dst, src;  // first destination / source element
  int ex, ey, ez;      // extents
  int dsx, dsy;        // destination row / plane strides (elements / rows)
  int flip;            // bit d: negate the d-components of vectors (reflecting face)
  int vec;             // 1: rows move as 16-byte vectors (x step +1; extent, offsets and
                       // row / plane strides multiples of 4 elements)
  long long sx, sy, sz;  // source element step per x, y, z step: +-1 / +-row / +-plane,
                         // negative across a reflecting face, 0 across an outflow face
};

// Vector axis of state field `fid` (0-4 rho, m_x, m_y, m_z, E; 5-8 E_r, F_x,
// F_y, F_z), -1 for scalars.
__host__ __device__ __forceinline__ int field_axis(int fid) {
  return (fid >= 1 && fid <= 3) ? fid - 1 : ((fid >= 6 && fid <= 8) ? fid - 6 : -1);
}

struct Chunk {
  int copy;            // index into the copy list
  int start;           // first cell (linear in the copy region) of this chunk
};
constexpr int CHUNK_CELLS = 1024;

// Step quantities produced on the device by the timestep kernel.
struct StepInfo {
  double dt;           // hydro timestep
  double nsub;         // number of radiation substeps
  double dtrad;        // radiation substep
  double smax;         // max(|v| + c_s)
  unsigned long long smax_bits;  // running max (bit pattern of a positive double)
  double nsub_total;   // radiation substeps summed over all steps so far
  double nsteps;       // timesteps computed so far
};

struct Status {
  unsigned int flags;          // 1 << QK_ENOCONV | 1 << QK_ENEGATIVE
  int max_iter;
  unsigned long long first_bad;  // smallest failing element index (~0 if none)
  unsigned long long total_iter;
};

// Constants of a stage kernel in its stencil precision, formed on the host:
// device-side conversions and divisions of the FP64 parameters occupy the
// FP64 pipe, and a register-bound kernel may repeat them at every use.
template <typename T> struct SC {
  T gamma, gm1, gm1inv, g1;  // gamma, gamma - 1, 1/(gamma - 1), (gamma + 1)/(2 gamma)
  T inv_dx[3], dx[3];
  T c, chat, kR;             // speed of light, reduced speed, kappa_R (or kappa0)
  int kmode;                 // QK_KAPPA_*
};
template <typename T> inline SC<T> make_sc(const qk_params &p) {
  SC<T> k;
  k.gamma = (T)p.gamma;
  k.gm1 = (T)(p.gamma - 1.0);
  k.gm1inv = (T)(1.0 / (p.gamma - 1.0));
  k.g1 = (T)((p.gamma + 1.0) / (2.0 * p.gamma));
  for (int d = 0; d < 3; ++d) {
    k.inv_dx[d] = (T)(1.0 / p.dx[d]);
    k.dx[d] = (T)p.dx[d];
  }
  k.c = (T)p.c;
  k.chat = (T)p.chat;
  k.kR = (T)p.kappa_R;
  k.kmode = p.kappa_mode;
  return k;
}

// Where a stage takes its timestep: a device StepInfo field when `p` is set,
// else the host value `v`.  `nsub`/`sub` predicate radiation substeps.
struct DtSrc {
  const StepInfo *p;
  double v;
  int which;           // 0: dt, 2: dtrad
  int sub;             // substep index (-1: always run)
};

__device__ __forceinline__ double dt_of(const DtSrc &s) {
  if (!s.p) return s.v;
  return s.which == 0 ? s.p->dt : s.p->dtrad;
}
__device__ __forceinline__ bool skip_substep(const DtSrc &s) {
  return s.p && s.sub >= 0 && (double)s.sub >= s.p->nsub;
}

template <typename T> struct F5 { T *f[5]; };
template <typename T> struct F4 { T *f[4]; };

// Shared-memory slot of tile-local cell (i,j,k); at most one coordinate may lie
// outside [0, TS).
__device__ __forceinline__ int cross_slot(int i, int j, int k) {
  if ((unsigned)i >= (unsigned)TS) {
    int h = i < 0 ? i + HALO : i - TS + HALO;
    return NCORE + (k * TS + j) * (2 * HALO) + h;
  }
  if ((unsigned)j >= (unsigned)TS) {
    int h = j < 0 ? j + HALO : j - TS + HALO;
    return NCORE + NHD + (k * (2 * HALO) + h) * TS + i;
  }
  if ((unsigned)k >= (unsigned)TS) {
    int h = k < 0 ? k + HALO : k - TS + HALO;
    return NCORE + 2 * NHD + (h * TS + j) * TS + i;
  }
  return (k * TS + j) * TS + i;
}

// Inverse of cross_slot.
__device__ __forceinline__ void slot_cell(int s, int &i, int &j, int &k) {
  if (s < NCORE) {
    i = s % TS; j = (s / TS) % TS; k = s / (TS * TS);
    return;
  }
  s -= NCORE;
  int part = s / NHD;
  s -= part * NHD;
  if (part == 0) {
    int h = s % (2 * HALO); int r = s / (2 * HALO);
    j = r % TS; k = r / TS;
    i = h < HALO ? h - HALO : TS + h - HALO;
  } else if (part == 1) {
    i = s % TS; int r = s / TS; int h = r % (2 * HALO); k = r / (2 * HALO);
    j = h < HALO ? h - HALO : TS + h - HALO;
  } else {
    i = s % TS; j = (s / TS) % TS; int h = s / (TS * TS);
    k = h < HALO ? h - HALO : TS + h - HALO;
  }
}

// Whether a cross slot is read by some stencil of a tile with valid extents v.
__device__ __forceinline__ bool slot_needed(int i, int j, int k, const int v[3]) {
  int c[3] = {i, j, k};
  int out = 0;
  bool ok = true;
  for (int d = 0; d < 3; ++d) {
    if (c[d] < 0 || c[d] >= v[d]) {
      ++out;
      ok = ok && c[d] >= -HALO && c[d] < v[d] + HALO;
    }
  }
  return out <= 1 && ok;
}

// Line item <-> cell for direction D: position p in [0, NPOS) (cell p-1) or
// face f in [0, NFACE) along D, and the two transverse coordinates, ordered so
// that consecutive threads touch consecutive x where possible.
template <int D> __device__ __forceinline__ void item_cell(int item, int npos, int &pos,
                                                           int &i, int &j, int &k) {
  if (D == 0) {
    pos = item % npos; int r = item / npos; j = r % TS; k = r / TS; i = pos - 1;
  } else if (D == 1) {
    i = item % TS; int r = item / TS; k = r % TS; pos = r / TS; j = pos - 1;
  } else {
    i = item % TS; int r = item / TS; j = r % TS; pos = r / TS; k = pos - 1;
  }
}
template <int D> __device__ __forceinline__ int item_index(int pos, int i, int j, int k,
                                                           int npos) {
  if (D == 0) return (k * TS + j) * npos + pos;
  if (D == 1) return (pos * TS + k) * TS + i;
  return (pos * TS + j) * TS + i;
}

__device__ __forceinline__ long long cell_elem(const DevBox &b, int g, int x, int y, int z) {
  return b.off + ((long long)(z + g) * b.sy + (y + g)) * b.sx + (x + g);
}

// atomic max of a positive double through its bit pattern
__device__ __forceinline__ void atomic_max_pos(unsigned long long *a, double v) {
  atomicMax(a, (unsigned long long)__double_as_longlong(v));
}

// ---------------------------------------------------------------------------
// Launchers (defined in the stage translation units).  Each returns a
// cudaError_t from the launch.
// ---------------------------------------------------------------------------
struct Geometry {
  const DevBox *boxes;
  const Tile *tiles;
  int ntiles;
  const Column *cols;  // column work list (plane-marching kernels)
  int ncols;
  int nbox;
  int ng;
  long long ncells;
  const long long *box_cell0;  // nbox+1 prefix of interior cells
};

// Launch configuration of a stage kernel: threads per CTA (128, 256 or 512 on
// the same shared-memory tile) and the tile schedule (0: strided over the
// grid, 1: one contiguous run of tiles per CTA), packed as threads | sched<<16.
constexpr int cfg_make(int threads, int sched, int shape = 0) {
  return threads | (sched << 16) | (shape << 17);
}
constexpr int cfg_threads(int cfg) { return cfg & 0xffff; }
constexpr int cfg_sched(int cfg) { return (cfg >> 16) & 1; }
// tile shape: 0 = TS^3 cross tiles, 1 = CW x CW columns marching along z
constexpr int cfg_shape(int cfg) { return (cfg >> 17) & 1; }
constexpr int kDefaultCfg = cfg_make(256, 0);

// Low parts of a compensated FP32 state (hi + lo per conserved field): those
// of the stage input U0 (R0), of the stage-1 result U1 (R1, stage 2 only) and
// of the output.  A null LoPtrs* selects the plain kernels.
struct LoPtrs {
  void *const *l0;
  void *const *l1;
  void *const *lo;
  int fmt = 1;  // storage of the low parts: 1 FP32, 2 16-bit (see lo_get / lo_put)
};

cudaError_t launch_hydro_stage(int fp32, int stage, const Geometry &g, const qk_params &p,
                               void *const *U0, void *const *U1, void *const *Uout, DtSrc dt,
                               int grid, int cfg, const void *chi, cudaStream_t s,
                               const LoPtrs *lo = nullptr);
cudaError_t launch_hydro_column(int fp32, int stage, const Geometry &g, const qk_params &p,
                                void *const *U0, void *const *U1, void *const *Uout, DtSrc dt,
                                const void *chi, cudaStream_t s, int cfg);
cudaError_t launch_flatten(int fp32, const Geometry &g, const qk_params &p, void *const *U,
                           void *chi, cudaStream_t s);
// The exchange fused into radiation stage 2: gas fields (and their low parts
// for a compensated state, else NULL), emissivity field or NULL, status word.
struct FuseArgs {
  void *const *U;
  void *const *Ulo;
  const void *src;
  Status *st;
};

cudaError_t launch_rad_column(int fp32, int stage, const Geometry &g, const qk_params &p,
                              void *const *R0, void *const *R1, void *const *Rout,
                              const void *rho, DtSrc dt, const FuseArgs *fx, cudaStream_t s,
                              int cfg);
cudaError_t launch_rad_stage(int fp32, int stage, const Geometry &g, const qk_params &p,
                             void *const *R0, void *const *R1, void *const *Rout,
                             const void *rho, DtSrc dt, int grid, int cfg, cudaStream_t s,
                             const LoPtrs *lo = nullptr, const FuseArgs *fx = nullptr);
cudaError_t launch_exchange(int fp32, const Geometry &g, const qk_params &p, void *const *U,
                            void *const *R, const void *src, DtSrc dt, Status *st,
                            cudaStream_t s, void *const *Ulo = nullptr,
                            void *const *Rlo = nullptr, int lofmt = 1);
cudaError_t launch_max_speed(int fp32, const Geometry &g, const qk_params &p,
                             void *const *U, StepInfo *si, cudaStream_t s);
cudaError_t launch_halo(int fp32, int pack, const Copy *copies, const Chunk *chunks, int nchunks,
                        void *const *fields, int nf, int first, void *buf, long long nbuf,
                        DtSrc pred, cudaStream_t s);
cudaError_t launch_timestep(const qk_params &p, StepInfo *si, cudaStream_t s);
cudaError_t launch_ghost_fill(int fp32, const Copy *copies, const Chunk *chunks, int nchunks,
                              void *const *fields, int nf, int first, DtSrc pred, cudaStream_t s);
cudaError_t launch_sums(int fp32, const Geometry &g, const qk_params &p, void *const *U,
                        void *const *R, double *partials, int nblocks, double *out,
                        cudaStream_t s, void *const *Ulo = nullptr, void *const *Rlo = nullptr,
                        int lofmt = 1);
int hydro_smem_bytes(int fp32);
int rad_smem_bytes(int fp32);
cudaError_t stage_kernel_setup(int fp32);

}  // namespace qk
