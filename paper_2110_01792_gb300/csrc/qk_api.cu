// qk_api.cu -- host side of libqk: the C ABI of include/qk.h.  Validates the
// patch set, builds the tile work list and the ghost-copy descriptors (with
// periodic images), owns the scratch for qk_step and its CUDA graph, and
// launches the stage kernels.
#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "qk_copy.cuh"
#include "qk_ctx.cuh"

using namespace qk;


static thread_local std::string g_init_err = "qk: null context";

static int fail(qk_ctx *c, int code, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  if (c) c->err = buf;
  return code;
}

static int cuda_fail(qk_ctx *c, cudaError_t e, const char *what) {
  return fail(c, QK_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define QK_CUDA(ctx, call)                                  \
  do {                                                      \
    cudaError_t e_ = (call);                                \
    if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call); \
  } while (0)

static Geometry geom(const qk_ctx *c) {
  Geometry g;
  g.boxes = c->d_boxes;
  g.tiles = c->d_tiles;
  g.ntiles = c->ntiles;
  if (c->part == QK_PART_INTERIOR) {
    g.tiles = c->d_tiles_ib;
    g.ntiles = c->n_interior;
  } else if (c->part == QK_PART_BOUNDARY) {
    g.tiles = c->d_tiles_ib + c->n_interior;
    g.ntiles = c->ntiles - c->n_interior;
  }
  // columns cover every owned cell: only for the whole tile set
  g.cols = c->part == QK_PART_ALL ? c->d_cols : nullptr;
  g.ncols = c->part == QK_PART_ALL ? c->ncols : 0;
  g.nbox = c->nbox_dev;
  g.ng = c->ng;
  g.ncells = c->ncells;
  g.box_cell0 = c->d_cell0;
  return g;
}

// The column list a launch configuration runs on: the one chunked for two
// CTAs per SM for the column configurations held to two (any list covers
// every cell, so this choice changes only the load balance).
static bool two_cta_cols(const qk_ctx *c, int cfg) {
  return c->d_cols2 && cfg_shape(cfg) == 1 && cfg_threads(cfg) == CNT + 32 && cfg_sched(cfg) == 1;
}
static Geometry geom_cfg(const qk_ctx *c, int cfg) {
  Geometry g = geom(c);
  if (g.cols && two_cta_cols(c, cfg)) {
    g.cols = c->d_cols2;
    g.ncols = c->ncols2;
  }
  return g;
}


static int check_params(qk_ctx *c, const qk_params *p) {
  if (!p) return fail(c, QK_EINVAL, "params is NULL");
  if (p->closure < QK_CLOSURE_LEVERMORE || p->closure > QK_CLOSURE_EDDINGTON)
    return fail(c, QK_EINVAL, "unknown closure %d", p->closure);
  for (int d = 0; d < 3; ++d) {
    if (p->bc_lo[d] < QK_BC_PERIODIC || p->bc_lo[d] > QK_BC_DIRICHLET || p->bc_hi[d] < QK_BC_PERIODIC ||
        p->bc_hi[d] > QK_BC_DIRICHLET)
      return fail(c, QK_EINVAL, "unknown boundary type on axis %d", d);
    if ((p->bc_lo[d] == QK_BC_PERIODIC) != (p->bc_hi[d] == QK_BC_PERIODIC))
      return fail(c, QK_EINVAL, "axis %d: a periodic boundary needs both faces periodic", d);
  }
  if (!(p->gamma > 1.0)) return fail(c, QK_EINVAL, "gamma must exceed 1");
  if (!(p->cfl > 0.0)) return fail(c, QK_EINVAL, "cfl must be positive");
  for (int d = 0; d < 3; ++d)
    if (!(p->dx[d] > 0.0)) return fail(c, QK_EINVAL, "dx must be positive");
  if (!p->hydro_only) {
    if (!(p->c > 0.0) || !(p->chat > 0.0)) return fail(c, QK_EINVAL, "c and chat must be positive");
    if (p->max_iter < 1) return fail(c, QK_EINVAL, "max_iter must be >= 1");
    if (p->nsub_max < 1) return fail(c, QK_EINVAL, "nsub_max must be >= 1");
    if (p->eos == QK_EOS_ALPHA_T3 && !(p->alpha_eos > 0.0))
      return fail(c, QK_EINVAL, "alpha_eos must be positive");
    if (p->eos == QK_EOS_GAMMA && !(p->c_v > 0.0)) return fail(c, QK_EINVAL, "c_v must be positive");
  }
  if (p->kappa_mode != QK_KAPPA_CONST && p->kappa_mode != QK_KAPPA_RHO)
    return fail(c, QK_EINVAL, "unknown kappa_mode %d", p->kappa_mode);
  if (p->eos != QK_EOS_GAMMA && p->eos != QK_EOS_ALPHA_T3)
    return fail(c, QK_EINVAL, "unknown eos %d", p->eos);
  if (p->recon != QK_RECON_PPM && p->recon != QK_RECON_PLM)
    return fail(c, QK_EINVAL, "unknown recon %d", p->recon);
  if (p->flattening != 0 && p->flattening != 1)
    return fail(c, QK_EINVAL, "flattening must be 0 or 1");
  if (p->flattening && c && c->ng && c->ng < 4)
    return fail(c, QK_EINVAL, "flattening needs nghost >= 4 (its stencil reaches 4 cells)");
  return QK_OK;
}

static int64_t padded_vol(const qk_box &b, int ng) {
  return (int64_t)(b.n[0] + 2 * ng) * (b.n[1] + 2 * ng) * (b.n[2] + 2 * ng);
}

// One axis of a ghost sub-region: destination cells [a0, a1) in global
// (unwrapped) coordinates and the rule that gives their source coordinate.
struct Piece {
  int a0, a1;
  int kind;   // 0: x - shift (inside, or a periodic image); 1: mirror, m - x;
              // 2: clamp to c (outflow); 3: Dirichlet store
  int shift, m, c;
};

static int fdiv(int a, int m) { return a >= 0 ? a / m : -((-a + m - 1) / m); }

// Split [r0, r1) on one axis of length D by the domain faces and their
// boundary types.
static void axis_pieces(int r0, int r1, int D, int bclo, int bchi, std::vector<Piece> &out) {
  out.clear();
  if (bclo == QK_BC_PERIODIC) {
    for (int k = fdiv(r0, D); k <= fdiv(r1 - 1, D); ++k) {
      const int a0 = std::max(r0, k * D), a1 = std::min(r1, (k + 1) * D);
      if (a0 < a1) out.push_back(Piece{a0, a1, 0, k * D, 0, 0});
    }
    return;
  }
  auto outside = [&](int a0, int a1, int bc, bool low) {
    if (a0 >= a1) return;
    if (bc == QK_BC_REFLECT) out.push_back(Piece{a0, a1, 1, 0, low ? -1 : 2 * D - 1, 0});
    else if (bc == QK_BC_OUTFLOW) out.push_back(Piece{a0, a1, 2, 0, 0, low ? 0 : D - 1});
    else out.push_back(Piece{a0, a1, 3, 0, 0, 0});
  };
  outside(r0, std::min(r1, 0), bclo, true);
  if (std::max(r0, 0) < std::min(r1, D)) out.push_back(Piece{std::max(r0, 0), std::min(r1, D), 0, 0, 0, 0});
  outside(std::max(r0, D), r1, bchi, false);
}

// Ghost-copy descriptors: for each patch, the 26 ghost sub-boxes around its
// interior, split per axis by the domain faces (periodic images, mirror
// images, clamped cells, Dirichlet cells), and each copyable piece
// intersected with every patch's interior that supplies its sources.  A
// binned index of the patches keeps this linear.  Dirichlet pieces become
// store regions (destination boxes in patch-local coordinates).  In a
// sharded context, copies with both ends owned go to `out`, the others to the
// per-peer send / receive lists; Dirichlet regions of owned patches only.
struct DirRegion {
  long long dst;      // first element
  int ex, ey, ez, dsx, dsy;
};

static int build_copies(qk_ctx *c, std::vector<Copy> &out,
                        std::vector<std::vector<Copy>> *send,
                        std::vector<std::vector<Copy>> *recv, std::vector<DirRegion> *dir) {
  const int ng = c->ng;
  const int *D = c->dom;
  const int BIN = 16;
  int nb[3];
  for (int d = 0; d < 3; ++d) nb[d] = (D[d] + BIN - 1) / BIN;
  std::vector<std::vector<int>> bins((size_t)nb[0] * nb[1] * nb[2]);
  for (int b = 0; b < c->nbox; ++b) {
    const qk_box &q = c->boxes[b];
    int lo[3], hi[3];
    for (int d = 0; d < 3; ++d) {
      lo[d] = q.lo[d] / BIN;
      hi[d] = (q.lo[d] + q.n[d] - 1) / BIN;
    }
    for (int z = lo[2]; z <= hi[2]; ++z)
      for (int y = lo[1]; y <= hi[1]; ++y)
        for (int x = lo[0]; x <= hi[0]; ++x) bins[((size_t)z * nb[1] + y) * nb[0] + x].push_back(b);
  }
  std::vector<int> stamp(c->nbox, -1);
  int stamp_id = 0;
  const bool sharded = !c->owner.empty();
  std::vector<Piece> pc[3];
  for (int b = 0; b < c->nbox; ++b) {
    const qk_box &B = c->boxes[b];
    const int sx = B.n[0] + 2 * ng, sy = B.n[1] + 2 * ng;
    const bool own_b = !sharded || c->owner[b] == c->rank;
    // a sharded rank visits every destination patch: remote destinations
    // can still need this rank's patches as sources (send lists)
    for (int rz = 0; rz < 3; ++rz)
      for (int ry = 0; ry < 3; ++ry)
        for (int rx = 0; rx < 3; ++rx) {
          if (rx == 1 && ry == 1 && rz == 1) continue;
          const int rs[3] = {rx, ry, rz};
          for (int d = 0; d < 3; ++d) {
            int r0, r1;  // region in global (unwrapped) coordinates
            if (rs[d] == 0) { r0 = B.lo[d] - ng; r1 = B.lo[d]; }
            else if (rs[d] == 1) { r0 = B.lo[d]; r1 = B.lo[d] + B.n[d]; }
            else { r0 = B.lo[d] + B.n[d]; r1 = B.lo[d] + B.n[d] + ng; }
            axis_pieces(r0, r1, D[d], c->p.bc_lo[d], c->p.bc_hi[d], pc[d]);
          }
          for (const Piece &pz : pc[2])
            for (const Piece &py : pc[1])
              for (const Piece &px : pc[0]) {
                const Piece *P[3] = {&px, &py, &pz};
                long long dl0[3];
                for (int d = 0; d < 3; ++d) dl0[d] = (long long)P[d]->a0 - B.lo[d] + ng;
                if (px.kind == 3 || py.kind == 3 || pz.kind == 3) {
                  if (own_b && dir)
                    dir->push_back(DirRegion{B.offset + (dl0[2] * sy + dl0[1]) * sx + dl0[0],
                                             px.a1 - px.a0, py.a1 - py.a0, pz.a1 - pz.a0, sx, sy});
                  continue;
                }
                int s0[3], s1[3];  // source range in the domain
                for (int d = 0; d < 3; ++d) {
                  const Piece &q = *P[d];
                  if (q.kind == 0) { s0[d] = q.a0 - q.shift; s1[d] = q.a1 - q.shift; }
                  else if (q.kind == 1) { s0[d] = q.m - q.a1 + 1; s1[d] = q.m - q.a0 + 1; }
                  else { s0[d] = q.c; s1[d] = q.c + 1; }
                }
                ++stamp_id;
                for (int z = s0[2] / BIN; z <= (s1[2] - 1) / BIN; ++z)
                  for (int y = s0[1] / BIN; y <= (s1[1] - 1) / BIN; ++y)
                    for (int x = s0[0] / BIN; x <= (s1[0] - 1) / BIN; ++x)
                      for (int qb : bins[((size_t)z * nb[1] + y) * nb[0] + x]) {
                        if (stamp[qb] == stamp_id) continue;
                        stamp[qb] = stamp_id;
                        const qk_box &Q = c->boxes[qb];
                        int i0[3], i1[3];
                        bool none = false;
                        for (int d = 0; d < 3; ++d) {
                          i0[d] = std::max(s0[d], Q.lo[d]);
                          i1[d] = std::min(s1[d], Q.lo[d] + Q.n[d]);
                          if (i0[d] >= i1[d]) none = true;
                        }
                        if (none) continue;
                        // destination range and the source of its first cell, per axis
                        int e0[3], ext[3], sfirst[3], step[3], flip = 0;
                        for (int d = 0; d < 3; ++d) {
                          const Piece &q = *P[d];
                          if (q.kind == 0) {
                            e0[d] = i0[d] + q.shift;
                            ext[d] = i1[d] - i0[d];
                            sfirst[d] = i0[d];
                            step[d] = 1;
                          } else if (q.kind == 1) {
                            e0[d] = q.m - i1[d] + 1;
                            ext[d] = i1[d] - i0[d];
                            sfirst[d] = i1[d] - 1;
                            step[d] = -1;
                            flip |= 1 << d;
                          } else {
                            e0[d] = q.a0;
                            ext[d] = q.a1 - q.a0;
                            sfirst[d] = q.c;
                            step[d] = 0;
                          }
                        }
                        const long long qsx = Q.n[0] + 2 * ng, qsy = Q.n[1] + 2 * ng;
                        long long dl[3], sl[3];
                        for (int d = 0; d < 3; ++d) {
                          dl[d] = (long long)e0[d] - B.lo[d] + ng;
                          sl[d] = (long long)sfirst[d] - Q.lo[d] + ng;
                        }
                        Copy cp;
                        cp.dst = B.offset + (dl[2] * sy + dl[1]) * sx + dl[0];
                        cp.src = Q.offset + (sl[2] * qsy + sl[1]) * qsx + sl[0];
                        cp.ex = ext[0];
                        cp.ey = ext[1];
                        cp.ez = ext[2];
                        cp.dsx = sx;
                        cp.dsy = sy;
                        cp.flip = flip;
                        cp.sx = step[0];
                        cp.sy = step[1] * qsx;
                        cp.sz = step[2] * qsx * qsy;
                        // 16-byte rows (4 floats or 2 doubles) when every row of the
                        // region starts on a multiple of 4 elements on both sides
                        cp.vec = cp.sx == 1 && cp.ex % 4 == 0 && cp.dst % 4 == 0 &&
                                 cp.src % 4 == 0 && cp.dsx % 4 == 0 && cp.sy % 4 == 0 &&
                                 cp.sz % 4 == 0;
                        if (!sharded) {
                          out.push_back(cp);
                        } else {
                          const int rb = c->owner[b], rq = c->owner[qb];
                          if (rb == c->rank && rq == c->rank) out.push_back(cp);
                          else if (rb == c->rank) (*recv)[rq].push_back(cp);
                          else if (rq == c->rank) (*send)[rb].push_back(cp);
                        }
                      }
              }
        }
  }
  return QK_OK;
}

static int validate_boxes(qk_ctx *c) {
  const int ng = c->ng;
  int64_t dvol = (int64_t)c->dom[0] * c->dom[1] * c->dom[2];
  int64_t tot = 0;
  for (int b = 0; b < c->nbox; ++b) {
    const qk_box &q = c->boxes[b];
    for (int d = 0; d < 3; ++d) {
      if (q.n[d] < 1) return fail(c, QK_EINVAL, "box %d: empty extent", b);
      if (q.lo[d] < 0 || q.lo[d] + q.n[d] > c->dom[d])
        return fail(c, QK_EINVAL, "box %d lies outside the domain", b);
    }
    if (q.offset < 0) return fail(c, QK_EINVAL, "box %d: negative offset", b);
    tot += (int64_t)q.n[0] * q.n[1] * q.n[2];
  }
  if (!c->partial && tot != dvol)
    return fail(c, QK_EINVAL, "boxes cover %lld cells, the domain has %lld", (long long)tot,
                (long long)dvol);
  // pairwise overlap (sweep on x)
  std::vector<int> order(c->nbox);
  for (int b = 0; b < c->nbox; ++b) order[b] = b;
  std::sort(order.begin(), order.end(),
            [&](int a, int b) { return c->boxes[a].lo[0] < c->boxes[b].lo[0]; });
  for (size_t a = 0; a < order.size(); ++a) {
    const qk_box &A = c->boxes[order[a]];
    for (size_t b = a + 1; b < order.size(); ++b) {
      const qk_box &B = c->boxes[order[b]];
      if (B.lo[0] >= A.lo[0] + A.n[0]) break;
      bool ov = true;
      for (int d = 0; d < 3; ++d)
        if (B.lo[d] >= A.lo[d] + A.n[d] || A.lo[d] >= B.lo[d] + B.n[d]) ov = false;
      if (ov) return fail(c, QK_EINVAL, "boxes %d and %d overlap", order[a], order[b]);
    }
  }
  // disjoint field ranges (of the owned patches in a sharded context)
  std::vector<int> byoff;
  for (int b = 0; b < c->nbox; ++b)
    if (c->owner.empty() || c->owner[b] == c->rank) byoff.push_back(b);
  std::sort(byoff.begin(), byoff.end(),
            [&](int a, int b) { return c->boxes[a].offset < c->boxes[b].offset; });
  int64_t end = 0;
  for (int b : byoff) {
    const qk_box &q = c->boxes[b];
    if (q.offset < end) return fail(c, QK_EINVAL, "box %d: field range overlaps another box", b);
    end = q.offset + padded_vol(q, ng);
  }
  c->field_len = end;
  c->ncells = 0;
  for (int b : byoff) c->ncells += (int64_t)c->boxes[b].n[0] * c->boxes[b].n[1] * c->boxes[b].n[2];
  return QK_OK;
}

template <typename T> static int upload(qk_ctx *c, T **dst, const std::vector<T> &v) {
  size_t n = std::max<size_t>(v.size(), 1) * sizeof(T);
  QK_CUDA(c, cudaMalloc((void **)dst, n));
  if (!v.empty()) QK_CUDA(c, cudaMemcpy(*dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
  return QK_OK;
}

static void release(qk_ctx *c) {
  if (c->gexec) cudaGraphExecDestroy(c->gexec);
  if (c->gexec_c) cudaGraphExecDestroy(c->gexec_c);
  for (void *s : c->scratch_lo) cudaFree(s);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  cudaFree(c->d_boxes);
  cudaFree(c->d_tiles);
  cudaFree(c->d_tiles_ib);
  cudaFree(c->d_cols);
  cudaFree(c->d_cols2);
  cudaFree(c->d_cell0);
  cudaFree(c->d_copies);
  cudaFree(c->d_chunks);
  cudaFree(c->d_send);
  cudaFree(c->d_recv);
  cudaFree(c->d_send_chunks);
  cudaFree(c->d_recv_chunks);
  cudaFree(c->d_dpack);
  cudaFree(c->d_dunpack);
  cudaFree(c->d_dchunks);
  cudaFree(c->dstore);
  cudaFree(c->d_si);
  cudaFree(c->d_status);
  cudaFree(c->d_partials);
  cudaFree(c->d_sums);
  for (void *s : c->scratch) cudaFree(s);
  cudaFree(c->chi);
  if (c->h_buf) cudaFreeHost(c->h_buf);
  for (void *h : c->hstate) cudaFree(h);
  for (cudaStream_t h : c->hcopy)
    if (h) cudaStreamDestroy(h);
  for (cudaEvent_t e : c->hcopy_ev)
    if (e) cudaEventDestroy(e);
}

// Forget the captured step graphs (parameters, launch configurations or
// modes changed).
static void drop_graphs(qk_ctx *c) {
  if (c->gexec) cudaGraphExecDestroy(c->gexec);
  if (c->gexec_c) cudaGraphExecDestroy(c->gexec_c);
  c->gexec = nullptr;
  c->gexec_c = nullptr;
}

extern "C" {

static int init_common(qk_ctx **out, const qk_params *p, const qk_box *boxes, int32_t nbox,
                       const int32_t domain_n[3], int32_t nghost, int32_t precision,
                       const int32_t *owner, int32_t nranks, int32_t rank, int partial = 0) {
  if (!out) return QK_EINVAL;
  *out = nullptr;
  qk_ctx *c = new qk_ctx();
  c->partial = partial;
  auto bail = [&](int rc) {
    g_init_err = c->err.empty() ? std::string("qk_init_patches failed") : c->err;
    release(c);
    delete c;
    return rc;
  };
  int rc = check_params(c, p);
  if (rc) return bail(rc);
  if (!boxes || nbox < 1 || !domain_n) return bail(fail(c, QK_EINVAL, "no boxes"));
  if (nghost < HALO || nghost > 16) return bail(fail(c, QK_EINVAL, "nghost must be in [3, 16]"));
  if (p->flattening && nghost < 4)
    return bail(fail(c, QK_EINVAL, "flattening needs nghost >= 4 (its stencil reaches 4 cells)"));
  if (precision != QK_FP64 && precision != QK_FP32_MIXED)
    return bail(fail(c, QK_EINVAL, "unknown precision"));
  for (int d = 0; d < 3; ++d)
    if (domain_n[d] < 1) return bail(fail(c, QK_EINVAL, "empty domain"));
  c->p = *p;
  c->fp32 = precision == QK_FP32_MIXED;
  c->elem = c->fp32 ? 4 : 8;
  c->ng = nghost;
  c->nbox = nbox;
  for (int d = 0; d < 3; ++d) c->dom[d] = domain_n[d];
  for (int d = 0; d < 3; ++d)
    if ((p->bc_lo[d] == QK_BC_REFLECT || p->bc_hi[d] == QK_BC_REFLECT) && domain_n[d] < nghost)
      return bail(fail(c, QK_EINVAL, "axis %d: a reflecting boundary needs at least nghost cells", d));
  c->boxes.assign(boxes, boxes + nbox);
  if (owner) {
    if (nranks < 1 || rank < 0 || rank >= nranks)
      return bail(fail(c, QK_EINVAL, "rank %d of %d ranks", rank, nranks));
    c->owner.assign(owner, owner + nbox);
    for (int b = 0; b < nbox; ++b)
      if (owner[b] < 0 || owner[b] >= nranks)
        return bail(fail(c, QK_EINVAL, "patch %d: owner %d outside [0, %d)", b, owner[b], nranks));
    c->rank = rank;
    c->nranks = nranks;
  }
  if ((rc = validate_boxes(c))) return bail(rc);
  for (int b = 0; b < nbox; ++b)
    if (c->owner.empty() || c->owner[b] == c->rank) c->own.push_back(b);
  if (c->own.empty()) return bail(fail(c, QK_EINVAL, "rank %d owns no patch", rank));

  // device table of the owned patches and their interior-cell prefix
  const int nown = (int)c->own.size();
  std::vector<DevBox> db(nown);
  std::vector<long long> cell0(nown + 1, 0);
  for (int l = 0; l < nown; ++l) {
    const qk_box &q = boxes[c->own[l]];
    for (int d = 0; d < 3; ++d) {
      db[l].lo[d] = q.lo[d];
      db[l].n[d] = q.n[d];
    }
    db[l].sx = q.n[0] + 2 * nghost;
    db[l].sy = q.n[1] + 2 * nghost;
    db[l].off = q.offset;
    db[l].cell0 = cell0[l];
    cell0[l + 1] = cell0[l] + (long long)q.n[0] * q.n[1] * q.n[2];
  }
  std::vector<Tile> tiles;
  c->tile_start.assign(nown + 1, 0);
  for (int l = 0; l < nown; ++l) {
    const qk_box &q = boxes[c->own[l]];
    c->tile_start[l] = (int)tiles.size();
    for (int z = 0; z < q.n[2]; z += TS)
      for (int y = 0; y < q.n[1]; y += TS)
        for (int x = 0; x < q.n[0]; x += TS) tiles.push_back(Tile{l, x, y, z});
  }
  c->tile_start[nown] = (int)tiles.size();
  c->ntiles = (int)tiles.size();
  // column work list: CW x CW footprints, z split into chunks of cz planes.
  // A column costs ~ (cz + 2.5) plane times (the start-up reconstructs two
  // planes ahead); the persistent grid holds `slots` columns at once, so cz
  // minimises waves x (cz + 2.5), waves = ceil(columns / slots).  Two lists:
  // for the column kernels' usual residency (COL_CTAS_* per SM) and, FP32,
  // for the configurations held to two CTAs per SM.
  std::vector<Column> cols, cols2;
  {
    int nsm = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    int max_nz = 1;
    for (int l = 0; l < nown; ++l) max_nz = std::max(max_nz, (int)boxes[c->own[l]].n[2]);
    auto build = [&](long long slots, std::vector<Column> &out, std::vector<int> &start) {
      int best_cz = max_nz;
      double best_cost = 1e300;
      for (int cz = std::min(8, max_nz); cz <= max_nz; ++cz) {
        long long items = 0;
        for (int l = 0; l < nown; ++l) {
          const qk_box &q = boxes[c->own[l]];
          items += (long long)((q.n[0] + CW - 1) / CW) * ((q.n[1] + CW - 1) / CW) *
                   ((q.n[2] + cz - 1) / cz);
        }
        const double cost = (double)((items + slots - 1) / slots) * (std::min(cz, max_nz) + 2.5);
        if (cost < best_cost) {
          best_cost = cost;
          best_cz = cz;
        }
      }
      start.assign(nown + 1, 0);
      for (int l = 0; l < nown; ++l) {
        const qk_box &q = boxes[c->own[l]];
        start[l] = (int)out.size();
        for (int y = 0; y < q.n[1]; y += CW)
          for (int x = 0; x < q.n[0]; x += CW)
            for (int z = 0; z < q.n[2]; z += best_cz)
              out.push_back(Column{l, x, y, z, std::min(z + best_cz, (int)q.n[2])});
      }
      start[nown] = (int)out.size();
    };
    const long long sm = std::max(nsm, 1);
    build(sm * (c->fp32 ? COL_CTAS_FP32 : COL_CTAS_FP64), cols, c->col_start);
    if (c->fp32) build(sm * 2, cols2, c->col_start2);
  }
  c->ncols = (int)cols.size();
  c->ncols2 = (int)cols2.size();
  std::vector<Copy> copies;
  std::vector<std::vector<Copy>> send(c->nranks), recv(c->nranks);
  std::vector<DirRegion> dir;
  build_copies(c, copies, &send, &recv, &dir);
  // Dirichlet store descriptors: packing reads the region (strided) into the
  // store, unpacking writes it back; store positions in region order
  {
    std::vector<Copy> dp, du;
    std::vector<Chunk> dch;
    long long pos = 0;
    for (const DirRegion &r : dir) {
      Copy cp{};
      cp.ex = r.ex;
      cp.ey = r.ey;
      cp.ez = r.ez;
      cp.dsx = r.dsx;
      cp.dsy = r.dsy;
      cp.sx = 1;
      cp.sy = r.dsx;
      cp.sz = (long long)r.dsx * r.dsy;
      Copy pk = cp, up = cp;
      pk.src = r.dst;
      pk.dst = pos;
      up.dst = r.dst;
      up.src = pos;
      dp.push_back(pk);
      du.push_back(up);
      const int n = r.ex * r.ey * r.ez;
      for (int s0 = 0; s0 < n; s0 += CHUNK_CELLS) dch.push_back(Chunk{(int)dp.size() - 1, s0});
      pos += n;
    }
    c->ndir = pos;
    c->ndchunks = (int)dch.size();
    if ((rc = upload(c, &c->d_dpack, dp))) return bail(rc);
    if ((rc = upload(c, &c->d_dunpack, du))) return bail(rc);
    if ((rc = upload(c, &c->d_dchunks, dch))) return bail(rc);
    if (pos > 0) {
      cudaError_t e2 = cudaMalloc(&c->dstore, (size_t)(9 * pos) * c->elem);
      if (e2 == cudaSuccess) e2 = cudaMemset(c->dstore, 0, (size_t)(9 * pos) * c->elem);
      if (e2 != cudaSuccess) return bail(cuda_fail(c, e2, "cudaMalloc(Dirichlet store)"));
    }
  }
  // halo descriptors: the send side packs each region contiguously (x fastest)
  // into the peer's buffer; the receive side unpacks in the same order
  std::vector<Copy> sd, rv;
  std::vector<Chunk> sch, rch;
  c->send_chunk0.assign(c->nranks + 1, 0);
  c->recv_chunk0.assign(c->nranks + 1, 0);
  c->send_cells.assign(c->nranks, 0);
  c->recv_cells.assign(c->nranks, 0);
  for (int pr = 0; pr < c->nranks; ++pr) {
    c->send_chunk0[pr] = (int)sch.size();
    for (Copy cp : send[pr]) {
      cp.dst = c->send_cells[pr];  // position in the peer's buffer
      sd.push_back(cp);
      const int n = cp.ex * cp.ey * cp.ez;
      for (int s0 = 0; s0 < n; s0 += CHUNK_CELLS) sch.push_back(Chunk{(int)sd.size() - 1, s0});
      c->send_cells[pr] += n;
    }
    c->recv_chunk0[pr] = (int)rch.size();
    for (Copy cp : recv[pr]) {
      cp.src = c->recv_cells[pr];
      rv.push_back(cp);
      const int n = cp.ex * cp.ey * cp.ez;
      for (int s0 = 0; s0 < n; s0 += CHUNK_CELLS) rch.push_back(Chunk{(int)rv.size() - 1, s0});
      c->recv_cells[pr] += n;
    }
  }
  c->send_chunk0[c->nranks] = (int)sch.size();
  c->recv_chunk0[c->nranks] = (int)rch.size();
  if ((rc = upload(c, &c->d_send, sd))) return bail(rc);
  if ((rc = upload(c, &c->d_recv, rv))) return bail(rc);
  if ((rc = upload(c, &c->d_send_chunks, sch))) return bail(rc);
  if ((rc = upload(c, &c->d_recv_chunks, rch))) return bail(rc);
  c->nbox_dev = nown;
  std::vector<Chunk> chunks;
  for (int i = 0; i < (int)copies.size(); ++i) {
    int n = copies[i].ex * copies[i].ey * copies[i].ez;
    for (int s = 0; s < n; s += CHUNK_CELLS) chunks.push_back(Chunk{i, s});
  }
  c->ncopies = (int)copies.size();
  c->nchunks = (int)chunks.size();

  if ((rc = upload(c, &c->d_boxes, db))) return bail(rc);
  if ((rc = upload(c, &c->d_tiles, tiles))) return bail(rc);
  if ((rc = upload(c, &c->d_cols, cols))) return bail(rc);
  if (!cols2.empty() && (rc = upload(c, &c->d_cols2, cols2))) return bail(rc);
  {
    // Interior / boundary split of the tiles.  A tile is a boundary tile when
    // a ghost cell that another rank fills lies within STENCIL_REACH cells of
    // it (the stage stencils reach 3 cells, the flattening coefficient of the
    // ring around a tile 4).  Remote ghost cells are marked per owned patch
    // from the receive descriptors and counted with a summed-volume table.
    const int R = 4;
    std::vector<int> order(nown);
    for (int l = 0; l < nown; ++l) order[l] = l;
    std::sort(order.begin(), order.end(),
              [&](int x, int y) { return boxes[c->own[x]].offset < boxes[c->own[y]].offset; });
    std::vector<std::vector<int>> sat(nown);
    for (const Copy &cp : rv) {
      // owning patch of the destination by offset
      int lo = 0, hi = nown - 1;
      while (lo < hi) {
        int mid = (lo + hi + 1) / 2;
        if (boxes[c->own[order[mid]]].offset <= cp.dst) lo = mid; else hi = mid - 1;
      }
      const int l = order[lo];
      const qk_box &q = boxes[c->own[l]];
      const int sx = q.n[0] + 2 * nghost, sy = q.n[1] + 2 * nghost, sz = q.n[2] + 2 * nghost;
      std::vector<int> &m = sat[l];
      if (m.empty()) m.assign((size_t)(sx + 1) * (sy + 1) * (sz + 1), 0);
      const long long r0 = cp.dst - q.offset;
      const int x0 = (int)(r0 % sx), y0 = (int)((r0 / sx) % sy), z0 = (int)(r0 / ((long long)sx * sy));
      for (int z = 0; z < cp.ez; ++z)
        for (int y = 0; y < cp.ey; ++y)
          for (int x = 0; x < cp.ex; ++x)
            m[((size_t)(z0 + z + 1) * (sy + 1) + (y0 + y + 1)) * (sx + 1) + (x0 + x + 1)] = 1;
    }
    for (int l = 0; l < nown; ++l) {
      std::vector<int> &m = sat[l];
      if (m.empty()) continue;
      const qk_box &q = boxes[c->own[l]];
      const int sx = q.n[0] + 2 * nghost + 1, sy = q.n[1] + 2 * nghost + 1, sz = q.n[2] + 2 * nghost + 1;
      for (int z = 1; z < sz; ++z)
        for (int y = 1; y < sy; ++y)
          for (int x = 1; x < sx; ++x) {
            auto at = [&](int zz, int yy, int xx) { return m[((size_t)zz * sy + yy) * sx + xx]; };
            m[((size_t)z * sy + y) * sx + x] += at(z - 1, y, x) + at(z, y - 1, x) + at(z, y, x - 1) -
                                                at(z - 1, y - 1, x) - at(z - 1, y, x - 1) -
                                                at(z, y - 1, x - 1) + at(z - 1, y - 1, x - 1);
          }
    }
    std::vector<Tile> inner, outer;
    for (const Tile &t : tiles) {
      const std::vector<int> &m = sat[t.box];
      bool remote = false;
      if (!m.empty()) {
        const qk_box &q = boxes[c->own[t.box]];
        const int full[3] = {q.n[0] + 2 * nghost, q.n[1] + 2 * nghost, q.n[2] + 2 * nghost};
        const int t0[3] = {t.x0, t.y0, t.z0};
        int lo3[3], hi3[3];
        for (int d = 0; d < 3; ++d) {
          lo3[d] = std::max(0, t0[d] + nghost - R);
          hi3[d] = std::min(full[d], t0[d] + nghost + std::min(TS, q.n[d] - t0[d]) + R);
        }
        const int sx = full[0] + 1, sy = full[1] + 1;
        auto at = [&](int zz, int yy, int xx) { return m[((size_t)zz * sy + yy) * sx + xx]; };
        const int cnt = at(hi3[2], hi3[1], hi3[0]) - at(lo3[2], hi3[1], hi3[0]) -
                        at(hi3[2], lo3[1], hi3[0]) - at(hi3[2], hi3[1], lo3[0]) +
                        at(lo3[2], lo3[1], hi3[0]) + at(lo3[2], hi3[1], lo3[0]) +
                        at(hi3[2], lo3[1], lo3[0]) - at(lo3[2], lo3[1], lo3[0]);
        remote = cnt > 0;
      }
      (remote ? outer : inner).push_back(t);
    }
    c->n_interior = (int)inner.size();
    inner.insert(inner.end(), outer.begin(), outer.end());
    if ((rc = upload(c, &c->d_tiles_ib, inner))) return bail(rc);
  }
  if ((rc = upload(c, &c->d_cell0, cell0))) return bail(rc);
  if ((rc = upload(c, &c->d_copies, copies))) return bail(rc);
  if ((rc = upload(c, &c->d_chunks, chunks))) return bail(rc);
  cudaError_t e;
  if ((e = cudaMalloc((void **)&c->d_si, sizeof(StepInfo))) != cudaSuccess)
    return bail(cuda_fail(c, e, "cudaMalloc(step info)"));
  if ((e = cudaMemset(c->d_si, 0, sizeof(StepInfo))) != cudaSuccess)
    return bail(cuda_fail(c, e, "cudaMemset"));
  if ((e = cudaMalloc((void **)&c->d_status, sizeof(Status))) != cudaSuccess)
    return bail(cuda_fail(c, e, "cudaMalloc(status)"));
  Status st0{0u, 0, ~0ull, 0ull};
  if ((e = cudaMemcpy(c->d_status, &st0, sizeof(st0), cudaMemcpyHostToDevice)) != cudaSuccess)
    return bail(cuda_fail(c, e, "cudaMemcpy(status)"));
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  c->sum_blocks = std::max(1, nsm * 2);
  if ((e = cudaMalloc((void **)&c->d_partials, sizeof(double) * 2 * QK_NSUMS * c->sum_blocks)) !=
      cudaSuccess)
    return bail(cuda_fail(c, e, "cudaMalloc(partials)"));
  if ((e = cudaMalloc((void **)&c->d_sums, sizeof(double) * QK_NSUMS)) != cudaSuccess)
    return bail(cuda_fail(c, e, "cudaMalloc(sums)"));
  for (int f = 0; f < 9; ++f)
    if ((e = cudaMalloc(&c->scratch[f], (size_t)c->field_len * c->elem)) != cudaSuccess)
      return bail(cuda_fail(c, e, "cudaMalloc(scratch field)"));
  if ((e = cudaMalloc(&c->chi, (size_t)c->field_len * c->elem)) != cudaSuccess)
    return bail(cuda_fail(c, e, "cudaMalloc(flattening field)"));
  if ((e = cudaMallocHost((void **)&c->h_buf, 64 * sizeof(double))) != cudaSuccess)
    return bail(cuda_fail(c, e, "cudaMallocHost"));
  if ((e = cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking)) != cudaSuccess)
    return bail(cuda_fail(c, e, "cudaStreamCreate"));
  *out = c;
  return QK_OK;
}

int qk_fill_plan(const qk_params *p, const qk_box *boxes, int32_t nbox,
                 const int32_t domain_n[3], int32_t nghost, int64_t *out, int64_t cap,
                 int64_t *ncopies, int64_t *ndirichlet) {
  qk_ctx c;
  int rc = check_params(&c, p);
  if (!rc && (!boxes || nbox < 1 || !domain_n)) rc = fail(&c, QK_EINVAL, "no boxes");
  if (!rc && (nghost < HALO || nghost > 16)) rc = fail(&c, QK_EINVAL, "nghost must be in [3, 16]");
  if (rc) {
    g_init_err = c.err;
    return rc;
  }
  c.p = *p;
  c.ng = nghost;
  c.nbox = nbox;
  for (int d = 0; d < 3; ++d) c.dom[d] = domain_n[d];
  for (int d = 0; d < 3; ++d)
    if ((p->bc_lo[d] == QK_BC_REFLECT || p->bc_hi[d] == QK_BC_REFLECT) && domain_n[d] < nghost) {
      g_init_err = "a reflecting boundary needs at least nghost cells";
      return QK_EINVAL;
    }
  c.boxes.assign(boxes, boxes + nbox);
  if ((rc = validate_boxes(&c))) {
    g_init_err = c.err;
    return rc;
  }
  std::vector<Copy> copies;
  std::vector<DirRegion> dir;
  build_copies(&c, copies, nullptr, nullptr, &dir);
  if (ncopies) *ncopies = (int64_t)copies.size();
  if (ndirichlet) *ndirichlet = (int64_t)dir.size();
  int64_t k = 0;
  for (const Copy &cp : copies) {
    if (k >= cap) break;
    int64_t *o = out + 12 * k++;
    const int64_t v[12] = {cp.dst, cp.src, cp.ex, cp.ey, cp.ez, cp.dsx, cp.dsy, cp.flip,
                           cp.sx, cp.sy, cp.sz, 0};
    memcpy(o, v, sizeof(v));
  }
  for (const DirRegion &r : dir) {
    if (k >= cap) break;
    int64_t *o = out + 12 * k++;
    const int64_t v[12] = {r.dst, 0, r.ex, r.ey, r.ez, r.dsx, r.dsy, 0, 0, 0, 0, 1};
    memcpy(o, v, sizeof(v));
  }
  return QK_OK;
}

int qk_init_patches(qk_ctx **out, const qk_params *p, const qk_box *boxes, int32_t nbox,
                    const int32_t domain_n[3], int32_t nghost, int32_t precision) {
  return init_common(out, p, boxes, nbox, domain_n, nghost, precision, nullptr, 1, 0);
}

int qk_init_level(qk_ctx **out, const qk_params *p, const qk_box *boxes, int32_t nbox,
                  const int32_t domain_n[3], int32_t nghost, int32_t precision) {
  for (int d = 0; d < 3; ++d)
    if (p && (p->bc_lo[d] != QK_BC_PERIODIC || p->bc_hi[d] != QK_BC_PERIODIC)) {
      g_init_err = "qk_init_level: refinement levels are periodic";
      return QK_EINVAL;
    }
  return init_common(out, p, boxes, nbox, domain_n, nghost, precision, nullptr, 1, 0, 1);
}

int qk_init_shard(qk_ctx **out, const qk_params *p, const qk_box *boxes, int32_t nbox,
                  const int32_t domain_n[3], int32_t nghost, int32_t precision,
                  const int32_t *owner, int32_t nranks, int32_t rank) {
  if (!owner) {
    g_init_err = "qk_init_shard: owner is NULL";
    return QK_EINVAL;
  }
  return init_common(out, p, boxes, nbox, domain_n, nghost, precision, owner, nranks, rank);
}

void qk_destroy(qk_ctx *c) {
  if (!c) return;
  release(c);
  delete c;
}

const char *qk_last_error(const qk_ctx *c) {
  if (!c) return g_init_err.c_str();
  return c->err.c_str();
}

int64_t qk_field_len(const qk_ctx *c) { return c ? c->field_len : -1; }
int64_t qk_num_cells(const qk_ctx *c) { return c ? c->ncells : -1; }

int qk_set_params(qk_ctx *c, const qk_params *p) {
  if (!c) return QK_EINVAL;
  int rc = check_params(c, p);
  if (rc) return rc;
  if (memcmp(p->bc_lo, c->p.bc_lo, sizeof(p->bc_lo)) != 0 ||
      memcmp(p->bc_hi, c->p.bc_hi, sizeof(p->bc_hi)) != 0)
    return fail(c, QK_EINVAL, "boundary types are fixed when the context is created");
  c->p = *p;
  drop_graphs(c);
  return QK_OK;
}

static int check_fields(qk_ctx *c, void *const *f, int n, const char *what);

// Full ghost fill of nf fields holding state fields first .. first+nf-1:
// descriptor copies (periodic, mirror, clamped), then the Dirichlet states.
static cudaError_t fill(qk_ctx *c, void *const *fields, int nf, int first, DtSrc pred,
                        cudaStream_t s) {
  cudaError_t e =
      launch_ghost_fill(c->fp32, c->d_copies, c->d_chunks, c->nchunks, fields, nf, first, pred, s);
  if (e == cudaSuccess && c->ndir > 0)
    e = launch_halo(c->fp32, 0, c->d_dunpack, c->d_dchunks, c->ndchunks, fields, nf, first,
                    (char *)c->dstore + (size_t)first * c->ndir * c->elem, c->ndir, pred, s);
  return e;
}

static int need_dirichlet(qk_ctx *c) {
  if (c->ndir > 0 && !c->dir_set)
    return fail(c, QK_EINVAL, "Dirichlet faces: record the boundary states with qk_set_dirichlet first");
  return QK_OK;
}

// Autotuner: time every candidate launch configuration of each stage kernel
// (threads per CTA x tile schedule) on the caller's state and keep the
// fastest.  Timing launches write only library scratch (stage outputs go to
// scratch buffers); the ghost cells of `hydro` and `rad` are refilled.
int qk_autotune(qk_ctx *c, void *const hydro[5], void *const rad[4], int32_t out_cfg[4],
                void *stream) {
  if (!c) return QK_EINVAL;
  int rc = check_fields(c, hydro, 5, "hydro");
  if (rc) return rc;
  if (rad && (rc = check_fields(c, rad, 4, "rad"))) return rc;
  if ((rc = need_dirichlet(c))) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  const Geometry g = geom(c);
  const int threads[3] = {128, 256, 512};
  // scratch: five fields for the stage outputs and, when qk_step fuses the
  // exchange into radiation stage 2, a copy of the gas state for the
  // exchange to update, and a status word of its own
  const bool fused = rad && c->fuse_exchange;
  void *tmp[10] = {};
  Status *tst = nullptr;
  auto release = [&]() {
    for (void *t : tmp) cudaFree(t);
    cudaFree(tst);
  };
  for (int q = 0; q < (fused ? 10 : 5); ++q) {
    cudaError_t e = cudaMalloc(&tmp[q], (size_t)c->field_len * c->elem);
    if (e != cudaSuccess) {
      release();
      return cuda_fail(c, e, "cudaMalloc(autotune scratch)");
    }
  }
  if (fused) {
    cudaError_t e = cudaMalloc((void **)&tst, sizeof(Status));
    if (e != cudaSuccess) {
      release();
      return cuda_fail(c, e, "cudaMalloc(autotune status)");
    }
  }
  void *Uc[5];
  for (int q = 0; q < 5; ++q) Uc[q] = tmp[5 + q];
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  void *U1[5], *R1[4], *Rt[4];
  for (int q = 0; q < 5; ++q) U1[q] = c->scratch[q];
  for (int q = 0; q < 4; ++q) {
    R1[q] = c->scratch[5 + q];
    Rt[q] = tmp[q];
  }
  // timestep for realistic dt values; it does not change the state
  cudaError_t err = launch_max_speed(c->fp32, g, c->p, hydro, c->d_si, s);
  if (err == cudaSuccess) err = launch_timestep(c->p, c->d_si, s);
  if (err == cudaSuccess) err = fill(c, hydro, 5, 0, DtSrc{nullptr, 0.0, 0, -1}, s);
  if (err == cudaSuccess && rad) err = fill(c, rad, 4, 5, DtSrc{nullptr, 0.0, 0, -1}, s);
  if (err == cudaSuccess && c->p.flattening) err = launch_flatten(c->fp32, g, c->p, hydro, c->chi, s);
  const DtSrc dth{c->d_si, 0.0, 0, -1}, dtr{c->d_si, 0.0, 2, -1};
  const FuseArgs fx{Uc, nullptr, c->src, tst};
  for (int which = 0; which < 4 && err == cudaSuccess; ++which) {
    const bool is_rad = which >= 2;
    if (is_rad && !rad) continue;
    const int stage = which % 2 + 1;
    float best = 1e30f;
    int best_cfg = c->cfg[which];
    // stage 2 reads the stage-1 result with its ghosts filled
    if (which == 1) err = fill(c, U1, 5, 0, DtSrc{nullptr, 0.0, 0, -1}, s);
    if (which == 3) err = fill(c, R1, 4, 5, DtSrc{nullptr, 0.0, 0, -1}, s);
    // candidates: threads x schedule on TS^3 tiles, and the columns (FP32
    // hydro, and radiation with the Levermore closure: also CNT + 32 threads
    // at 3 or 2 CTAs per SM)
    const bool wide = c->fp32 && (!is_rad || c->p.closure == QK_CLOSURE_LEVERMORE);
    const int ncand = wide ? 9 : 7;
    for (int ci = 0; ci < ncand && err == cudaSuccess; ++ci) {
        const int cfg = ci < 6    ? cfg_make(threads[ci / 2], ci % 2)
                        : ci == 6 ? cfg_make(CNT, 0, 1)
                                  : cfg_make(CNT + 32, ci - 7, 1);
        // radiation stage 2 is timed as qk_step runs it: with the exchange
        // fused when it is, on a fresh copy of the gas state
        if (which == 3 && fused)
          for (int q = 0; q < 5 && err == cudaSuccess; ++q)
            err = cudaMemcpyAsync(Uc[q], hydro[q], (size_t)c->field_len * c->elem,
                                  cudaMemcpyDeviceToDevice, s);
        if (err != cudaSuccess) break;
        const Geometry gc = geom_cfg(c, cfg);
        auto launch = [&]() {
          if (!is_rad)
            return launch_hydro_stage(c->fp32, stage, gc, c->p, hydro, stage == 2 ? U1 : nullptr,
                                      stage == 1 ? U1 : tmp, dth, 0, cfg,
                                      c->p.flattening ? c->chi : nullptr, s);
          return launch_rad_stage(c->fp32, stage, gc, c->p, rad, stage == 2 ? R1 : nullptr,
                                  stage == 1 ? R1 : Rt, hydro[0], dtr, 0, cfg, s, nullptr,
                                  which == 3 && fused ? &fx : nullptr);
        };
        err = launch();
        if (err != cudaSuccess) break;
        cudaEventRecord(e0, s);
        for (int r = 0; r < 3 && err == cudaSuccess; ++r) err = launch();
        cudaEventRecord(e1, s);
        if (err == cudaSuccess) err = cudaEventSynchronize(e1);
        float ms = 0.0f;
        if (err == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
        if (err == cudaSuccess && ms < best) {
          best = ms;
          best_cfg = cfg;
        }
      }
    c->cfg[which] = best_cfg;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (err == cudaSuccess) err = cudaStreamSynchronize(s);
  release();
  if (err != cudaSuccess) return cuda_fail(c, err, "autotune launch");
  drop_graphs(c);
  if (out_cfg)
    for (int w = 0; w < 4; ++w) out_cfg[w] = c->cfg[w];
  return QK_OK;
}

int qk_set_launch_config(qk_ctx *c, const int32_t cfg[4]) {
  if (!c) return QK_EINVAL;
  if (!cfg) return fail(c, QK_EINVAL, "cfg is NULL");
  for (int w = 0; w < 4; ++w) {
    const int v = cfg[w], th = cfg_threads(v), shape = cfg_shape(v);
    const bool ok = (v >> 18) == 0 &&
                    (shape == 0 ? (th == 128 || th == 256 || th == 512)
                                : ((th == CNT && cfg_sched(v) == 0) || th == CNT + 32));
    if (!ok) return fail(c, QK_EINVAL, "invalid launch configuration %d for stage kernel %d", v, w);
  }
  for (int w = 0; w < 4; ++w) c->cfg[w] = cfg[w];
  drop_graphs(c);
  return QK_OK;
}

int qk_set_launch_mode(qk_ctx *c, int32_t mode) {
  if (!c) return QK_EINVAL;
  if (mode != QK_LAUNCH_BATCHED && mode != QK_LAUNCH_PER_PATCH)
    return fail(c, QK_EINVAL, "unknown launch mode %d", mode);
  c->launch_mode = mode;
  drop_graphs(c);
  return QK_OK;
}

int qk_set_source(qk_ctx *c, const void *j) {
  if (!c) return QK_EINVAL;
  c->src = j;
  drop_graphs(c);
  return QK_OK;
}

int qk_set_tile_part(qk_ctx *c, int32_t part) {
  if (!c) return QK_EINVAL;
  if (part != QK_PART_ALL && part != QK_PART_INTERIOR && part != QK_PART_BOUNDARY)
    return fail(c, QK_EINVAL, "unknown tile part %d", part);
  c->part = part;
  return QK_OK;
}

int qk_tile_counts(const qk_ctx *c, int32_t *n_interior, int32_t *n_boundary) {
  if (!c) return QK_EINVAL;
  if (n_interior) *n_interior = c->n_interior;
  if (n_boundary) *n_boundary = c->ntiles - c->n_interior;
  return QK_OK;
}

int qk_set_fused_exchange(qk_ctx *c, int32_t enable) {
  if (!c) return QK_EINVAL;
  c->fuse_exchange = enable ? 1 : 0;
  drop_graphs(c);
  return QK_OK;
}

int qk_set_graph(qk_ctx *c, int32_t enable) {
  if (!c) return QK_EINVAL;
  c->use_graph = enable ? 1 : 0;
  return QK_OK;
}

static int check_fields(qk_ctx *c, void *const *f, int n, const char *what) {
  if (!f) return fail(c, QK_EINVAL, "%s is NULL", what);
  for (int i = 0; i < n; ++i)
    if (!f[i]) return fail(c, QK_EINVAL, "%s[%d] is NULL", what, i);
  return QK_OK;
}

int qk_fill_ghosts_range(qk_ctx *c, void *const *fields, int32_t first, int32_t nfields,
                         void *stream) {
  if (!c) return QK_EINVAL;
  if (first < 0 || nfields < 0 || first + nfields > 9)
    return fail(c, QK_EINVAL, "fields first .. first+nfields-1 must lie in [0, 9)");
  int rc = check_fields(c, fields, nfields, "fields");
  if (rc) return rc;
  if ((rc = need_dirichlet(c))) return rc;
  DtSrc pred{nullptr, 0.0, 0, -1};
  QK_CUDA(c, fill(c, fields, nfields, first, pred, (cudaStream_t)stream));
  return QK_OK;
}

int qk_fill_ghosts(qk_ctx *c, void *const *fields, int32_t nfields, void *stream) {
  return qk_fill_ghosts_range(c, fields, 0, nfields, stream);
}

int qk_set_dirichlet(qk_ctx *c, void *const hydro[5], void *const rad[4], void *stream) {
  if (!c) return QK_EINVAL;
  int rc = check_fields(c, hydro, 5, "hydro");
  if (rc) return rc;
  if (rad && (rc = check_fields(c, rad, 4, "rad"))) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  if (c->ndir > 0) {
    const DtSrc none{nullptr, 0.0, 0, -1};
    QK_CUDA(c, launch_halo(c->fp32, 1, c->d_dpack, c->d_dchunks, c->ndchunks, hydro, 5, 0,
                           c->dstore, c->ndir, none, s));
    char *rbuf = (char *)c->dstore + (size_t)5 * c->ndir * c->elem;
    if (rad)
      QK_CUDA(c, launch_halo(c->fp32, 1, c->d_dpack, c->d_dchunks, c->ndchunks, rad, 4, 5, rbuf,
                             c->ndir, none, s));
    else
      QK_CUDA(c, cudaMemsetAsync(rbuf, 0, (size_t)4 * c->ndir * c->elem, s));
  }
  c->dir_set = 1;
  return QK_OK;
}

int qk_hydro_stage(qk_ctx *c, int32_t stage, void *const U0[5], void *const U1[5],
                   void *const Uout[5], double dt, void *stream) {
  if (!c) return QK_EINVAL;
  if (stage != 1 && stage != 2) return fail(c, QK_EINVAL, "stage must be 1 or 2");
  int rc = check_fields(c, U0, 5, "U0");
  if (!rc && stage == 2) rc = check_fields(c, U1, 5, "U1");
  if (!rc) rc = check_fields(c, Uout, 5, "Uout");
  if (rc) return rc;
  if (stage == 1)
    for (int q = 0; q < 5; ++q)
      if (Uout[q] == U0[q]) return fail(c, QK_EINVAL, "stage 1 cannot update in place");
  if (stage == 2)
    for (int q = 0; q < 5; ++q)
      if (Uout[q] == U1[q]) return fail(c, QK_EINVAL, "Uout must not alias U1");
  DtSrc d{nullptr, dt, 0, -1};
  if (c->p.flattening)
    QK_CUDA(c, launch_flatten(c->fp32, geom(c), c->p, stage == 1 ? U0 : U1, c->chi,
                              (cudaStream_t)stream));
  QK_CUDA(c, launch_hydro_stage(c->fp32, stage, geom_cfg(c, c->cfg[stage - 1]), c->p, U0,
                                stage == 2 ? U1 : nullptr,
                                Uout, d, 0, c->cfg[stage - 1], c->p.flattening ? c->chi : nullptr,
                                (cudaStream_t)stream));
  return QK_OK;
}

int qk_rad_stage(qk_ctx *c, int32_t stage, void *const R0[4], void *const R1[4],
                 void *const Rout[4], const void *rho, double dt_rad, void *stream) {
  if (!c) return QK_EINVAL;
  if (stage != 1 && stage != 2) return fail(c, QK_EINVAL, "stage must be 1 or 2");
  int rc = check_fields(c, R0, 4, "R0");
  if (!rc && stage == 2) rc = check_fields(c, R1, 4, "R1");
  if (!rc) rc = check_fields(c, Rout, 4, "Rout");
  if (rc) return rc;
  if (!rho) return fail(c, QK_EINVAL, "rho is NULL");
  if (stage == 1)
    for (int q = 0; q < 4; ++q)
      if (Rout[q] == R0[q]) return fail(c, QK_EINVAL, "stage 1 cannot update in place");
  if (stage == 2)
    for (int q = 0; q < 4; ++q)
      if (Rout[q] == R1[q]) return fail(c, QK_EINVAL, "Rout must not alias R1");
  DtSrc d{nullptr, dt_rad, 2, -1};
  QK_CUDA(c, launch_rad_stage(c->fp32, stage, geom_cfg(c, c->cfg[1 + stage]), c->p, R0,
                              stage == 2 ? R1 : nullptr, Rout,
                              rho, d, 0, c->cfg[2 + stage - 1], (cudaStream_t)stream));
  return QK_OK;
}

int qk_rad_stage2_exchange(qk_ctx *c, void *const R0[4], void *const R1[4], void *const Rout[4],
                           void *const hydro[5], double dt_rad, void *stream) {
  if (!c) return QK_EINVAL;
  int rc = check_fields(c, R0, 4, "R0");
  if (!rc) rc = check_fields(c, R1, 4, "R1");
  if (!rc) rc = check_fields(c, Rout, 4, "Rout");
  if (!rc) rc = check_fields(c, hydro, 5, "hydro");
  if (rc) return rc;
  for (int q = 0; q < 4; ++q)
    if (Rout[q] == R1[q]) return fail(c, QK_EINVAL, "Rout must not alias R1");
  DtSrc d{nullptr, dt_rad, 2, -1};
  const FuseArgs fx{hydro, nullptr, c->src, c->d_status};
  QK_CUDA(c, launch_rad_stage(c->fp32, 2, geom_cfg(c, c->cfg[3]), c->p, R0, R1, Rout, hydro[0], d,
                              0, c->cfg[3],
                              (cudaStream_t)stream, nullptr, &fx));
  return QK_OK;
}

int qk_rad_matter_exchange(qk_ctx *c, void *const hydro[5], void *const rad[4], double dt_rad,
                           void *stream) {
  if (!c) return QK_EINVAL;
  int rc = check_fields(c, hydro, 5, "hydro");
  if (!rc) rc = check_fields(c, rad, 4, "rad");
  if (rc) return rc;
  DtSrc d{nullptr, dt_rad, 2, -1};
  QK_CUDA(c, launch_exchange(c->fp32, geom(c), c->p, hydro, rad, c->src, d, c->d_status,
                             (cudaStream_t)stream));
  return QK_OK;
}

int qk_timestep(qk_ctx *c, void *const hydro[5], double out[4], void *stream) {
  if (!c) return QK_EINVAL;
  int rc = check_fields(c, hydro, 5, "hydro");
  if (rc) return rc;
  if (!out) return fail(c, QK_EINVAL, "out is NULL");
  if (c->nranks > 1)
    return fail(c, QK_EINVAL, "sharded context: use qk_signal_speed and qk_set_timestep");
  cudaStream_t s = (cudaStream_t)stream;
  QK_CUDA(c, launch_max_speed(c->fp32, geom(c), c->p, hydro, c->d_si, s));
  QK_CUDA(c, launch_timestep(c->p, c->d_si, s));
  QK_CUDA(c, cudaMemcpyAsync(c->h_buf, c->d_si, 4 * sizeof(double), cudaMemcpyDeviceToHost, s));
  QK_CUDA(c, cudaStreamSynchronize(s));
  out[0] = c->h_buf[0];
  out[1] = c->h_buf[1];
  out[2] = c->h_buf[2];
  out[3] = c->h_buf[3];
  return QK_OK;
}

// The work lists of patch b alone (tiles and columns are grouped by patch).
static Geometry patch_geom(const qk_ctx *c, Geometry g, int b, int cfg = 0) {
  g.tiles = c->d_tiles + c->tile_start[b];
  g.ntiles = c->tile_start[b + 1] - c->tile_start[b];
  if (g.cols && two_cta_cols(c, cfg)) {
    g.cols = c->d_cols2 + c->col_start2[b];
    g.ncols = c->col_start2[b + 1] - c->col_start2[b];
  } else if (g.cols) {
    g.cols = c->d_cols + c->col_start[b];
    g.ncols = c->col_start[b + 1] - c->col_start[b];
  }
  return g;
}

// Stage launches: one persistent launch over the tiles of every patch
// (QK_LAUNCH_BATCHED), or one launch per patch over its own tiles
// (QK_LAUNCH_PER_PATCH, kept for comparison).
static cudaError_t hydro_launches(qk_ctx *c, int stage, void *const *U0, void *const *U1,
                                  void *const *Uo, DtSrc dt, cudaStream_t s,
                                  const LoPtrs *lo = nullptr) {
  const Geometry g = geom_cfg(c, c->cfg[stage - 1]);
  const void *chi = c->p.flattening ? c->chi : nullptr;
  if (chi) {
    cudaError_t e = launch_flatten(c->fp32, g, c->p, stage == 1 ? U0 : U1, c->chi, s);
    if (e != cudaSuccess) return e;
  }
  if (c->launch_mode == QK_LAUNCH_BATCHED || c->part != QK_PART_ALL)
    return launch_hydro_stage(c->fp32, stage, g, c->p, U0, U1, Uo, dt, 0, c->cfg[stage - 1], chi,
                              s, lo);
  for (int b = 0; b < c->nbox_dev; ++b) {
    const Geometry gb = patch_geom(c, g, b, c->cfg[stage - 1]);
    cudaError_t e = launch_hydro_stage(c->fp32, stage, gb, c->p, U0, U1, Uo, dt, 0,
                                       c->cfg[stage - 1], chi, s, lo);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

static cudaError_t rad_launches(qk_ctx *c, int stage, void *const *R0, void *const *R1,
                                void *const *Ro, const void *rho, DtSrc dt, cudaStream_t s,
                                const LoPtrs *lo = nullptr, const FuseArgs *fx = nullptr) {
  const Geometry g = geom_cfg(c, c->cfg[1 + stage]);
  if (c->launch_mode == QK_LAUNCH_BATCHED || c->part != QK_PART_ALL)
    return launch_rad_stage(c->fp32, stage, g, c->p, R0, R1, Ro, rho, dt, 0, c->cfg[1 + stage], s,
                            lo, fx);
  for (int b = 0; b < c->nbox_dev; ++b) {
    const Geometry gb = patch_geom(c, g, b, c->cfg[1 + stage]);
    cudaError_t e = launch_rad_stage(c->fp32, stage, gb, c->p, R0, R1, Ro, rho, dt, 0,
                                     c->cfg[1 + stage], s, lo, fx);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// The launch sequence of one full update (Sec. 2.2 operator split).  With
// hlo (and rlo) the state is compensated: hi + lo per conserved field, the
// stage-1 results keeping their low parts in the library's scratch_lo.
static int enqueue_step(qk_ctx *c, void *const hydro[5], void *const rad[4], cudaStream_t s,
                        void *const *hlo = nullptr, void *const *rlo = nullptr) {
  const Geometry g = geom(c);
  void *U1[5], *R1[4], *U1l[5], *R1l[4];
  for (int q = 0; q < 5; ++q) U1[q] = c->scratch[q];
  for (int q = 0; q < 4; ++q) R1[q] = c->scratch[5 + q];
  for (int q = 0; q < 5; ++q) U1l[q] = c->scratch_lo[q];
  for (int q = 0; q < 4; ++q) R1l[q] = c->scratch_lo[5 + q];
  const LoPtrs h1{hlo, nullptr, U1l, c->lo_fmt}, h2{hlo, U1l, hlo, c->lo_fmt};
  const LoPtrs r1{rlo, nullptr, R1l, c->lo_fmt}, r2{rlo, R1l, rlo, c->lo_fmt};
  const DtSrc dth{c->d_si, 0.0, 0, -1};
  const DtSrc none{nullptr, 0.0, 0, -1};
  QK_CUDA(c, launch_max_speed(c->fp32, g, c->p, hydro, c->d_si, s));
  QK_CUDA(c, launch_timestep(c->p, c->d_si, s));
  QK_CUDA(c, fill(c, hydro, 5, 0, none, s));
  QK_CUDA(c, hydro_launches(c, 1, hydro, nullptr, U1, dth, s, hlo ? &h1 : nullptr));
  QK_CUDA(c, fill(c, U1, 5, 0, none, s));
  QK_CUDA(c, hydro_launches(c, 2, hydro, U1, hydro, dth, s, hlo ? &h2 : nullptr));
  if (rad && !c->p.hydro_only) {
    QK_CUDA(c, fill(c, hydro, 1, 0, none, s));
    for (int sub = 0; sub < c->p.nsub_max; ++sub) {
      const DtSrc dr{c->d_si, 0.0, 2, sub};
      QK_CUDA(c, fill(c, rad, 4, 5, dr, s));
      QK_CUDA(c, rad_launches(c, 1, rad, nullptr, R1, hydro[0], dr, s, rlo ? &r1 : nullptr));
      QK_CUDA(c, fill(c, R1, 4, 5, dr, s));
      if (c->fuse_exchange) {
        // stage 2 with the exchange of every cell in its epilogue
        const FuseArgs fx{hydro, hlo, c->src, c->d_status};
        QK_CUDA(c, rad_launches(c, 2, rad, R1, rad, hydro[0], dr, s, rlo ? &r2 : nullptr, &fx));
      } else {
        QK_CUDA(c, rad_launches(c, 2, rad, R1, rad, hydro[0], dr, s, rlo ? &r2 : nullptr));
        QK_CUDA(c, launch_exchange(c->fp32, g, c->p, hydro, rad, c->src, dr, c->d_status, s, hlo,
                                   rlo, c->lo_fmt));
      }
    }
  }
  return QK_OK;
}

int qk_step(qk_ctx *c, void *const hydro[5], void *const rad[4], double *dt_out, int32_t *nsub_out,
            void *stream) {
  if (!c) return QK_EINVAL;
  int rc = check_fields(c, hydro, 5, "hydro");
  if (rc) return rc;
  if (rad && (rc = check_fields(c, rad, 4, "rad"))) return rc;
  if (c->nranks > 1)
    return fail(c, QK_EINVAL, "sharded context: compose the step from the stage entry points");
  if ((rc = need_dirichlet(c))) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  if (c->use_graph) {
    void *key[10];
    for (int q = 0; q < 5; ++q) key[q] = hydro[q];
    for (int q = 0; q < 4; ++q) key[5 + q] = rad ? rad[q] : nullptr;
    key[9] = (void *)(intptr_t)(rad ? 1 : 0);
    if (!c->gexec || memcmp(key, c->gkey, sizeof(key)) != 0) {
      if (c->gexec) {
        cudaGraphExecDestroy(c->gexec);
        c->gexec = nullptr;
      }
      // kernels see the caller's stream order through the graph launch; the
      // capture itself runs on a private stream
      QK_CUDA(c, cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
      rc = enqueue_step(c, hydro, rad, c->cap_stream);
      cudaGraph_t graph = nullptr;
      cudaError_t e = cudaStreamEndCapture(c->cap_stream, &graph);
      if (rc) {
        if (graph) cudaGraphDestroy(graph);
        return rc;
      }
      if (e != cudaSuccess) return cuda_fail(c, e, "cudaStreamEndCapture");
      e = cudaGraphInstantiate(&c->gexec, graph, 0);
      cudaGraphDestroy(graph);
      if (e != cudaSuccess) return cuda_fail(c, e, "cudaGraphInstantiate");
      memcpy(c->gkey, key, sizeof(key));
    }
    QK_CUDA(c, cudaGraphLaunch(c->gexec, s));
  } else {
    if ((rc = enqueue_step(c, hydro, rad, s))) return rc;
  }
  if (dt_out) QK_CUDA(c, cudaMemcpyAsync(dt_out, &c->d_si->dt, sizeof(double), cudaMemcpyDeviceToHost, s));
  if (nsub_out) {
    // N_sub is stored as a double on the device; convert on the host side
    // through the pinned buffer only when asked, synchronously
    QK_CUDA(c, cudaMemcpyAsync(c->h_buf + 8, &c->d_si->nsub, sizeof(double), cudaMemcpyDeviceToHost, s));
    QK_CUDA(c, cudaStreamSynchronize(s));
    *nsub_out = (int32_t)c->h_buf[8];
  }
  return QK_OK;
}

// Copies of `nf` whole fields between the caller's arrays and the context's
// device copies.  Pinned, 16-byte aligned host arrays (all of them) are copied
// by the SMs through their device mapping, on `s`, in one launch per
// direction; otherwise one cudaMemcpyAsync per field, spread over the copy
// streams (field q on stream q mod 3) and ordered after the work already on
// `s`, which waits for all of them.
static int host_copies(qk_ctx *c, void *const *host, int nf, bool to_device, cudaStream_t s) {
  const size_t bytes = (size_t)c->field_len * c->elem;
  FieldCopies fc{};
  bool mapped = true;
  for (int q = 0; q < nf && mapped; ++q) {
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, host[q]) != cudaSuccess) {
      cudaGetLastError();  // clear: an unknown pointer is pageable memory
      mapped = false;
      break;
    }
    void *dp = a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
    if (!dp || ((uintptr_t)dp & 15) != 0) {
      mapped = false;
      break;
    }
    fc.src[q] = to_device ? (const void *)dp : (const void *)c->hstate[q];
    fc.dst[q] = to_device ? c->hstate[q] : dp;
  }
  if (mapped) {
    QK_CUDA(c, launch_field_copies(fc, nf, bytes, s));
    return QK_OK;
  }
  QK_CUDA(c, cudaEventRecord(c->hcopy_ev[3], s));
  for (int i = 0; i < 3; ++i) QK_CUDA(c, cudaStreamWaitEvent(c->hcopy[i], c->hcopy_ev[3], 0));
  for (int q = 0; q < nf; ++q) {
    void *dst = to_device ? c->hstate[q] : host[q];
    const void *src = to_device ? (const void *)host[q] : (const void *)c->hstate[q];
    QK_CUDA(c, cudaMemcpyAsync(dst, src, bytes,
                               to_device ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToHost,
                               c->hcopy[q % 3]));
  }
  for (int i = 0; i < 3; ++i) {
    QK_CUDA(c, cudaEventRecord(c->hcopy_ev[i], c->hcopy[i]));
    QK_CUDA(c, cudaStreamWaitEvent(s, c->hcopy_ev[i], 0));
  }
  return QK_OK;
}

int qk_step_host(qk_ctx *c, void *const hydro[5], void *const rad[4], double *dt_out,
                 int32_t *nsub_out, void *stream) {
  if (!c) return QK_EINVAL;
  if (!hydro) return fail(c, QK_EINVAL, "hydro fields missing");
  for (int q = 0; q < 5; ++q)
    if (!hydro[q]) return fail(c, QK_EINVAL, "hydro field %d is NULL", q);
  if (rad)
    for (int q = 0; q < 4; ++q)
      if (!rad[q]) return fail(c, QK_EINVAL, "rad field %d is NULL", q);
  const int nf = rad ? 9 : 5;
  const size_t bytes = (size_t)c->field_len * c->elem;
  for (int q = 0; q < nf; ++q)
    if (!c->hstate[q]) QK_CUDA(c, cudaMalloc(&c->hstate[q], bytes));
  if (!c->hcopy[0]) {
    for (int i = 0; i < 3; ++i)
      QK_CUDA(c, cudaStreamCreateWithFlags(&c->hcopy[i], cudaStreamNonBlocking));
    for (int i = 0; i < 4; ++i)
      QK_CUDA(c, cudaEventCreateWithFlags(&c->hcopy_ev[i], cudaEventDisableTiming));
  }
  void *host[9];
  for (int q = 0; q < 5; ++q) host[q] = hydro[q];
  for (int q = 5; q < nf; ++q) host[q] = rad[q - 5];
  cudaStream_t s = (cudaStream_t)stream;
  int rc = host_copies(c, host, nf, true, s);
  if (rc) return rc;
  void *const *dev = c->hstate;
  if ((rc = qk_step(c, dev, rad ? dev + 5 : nullptr, dt_out, nullptr, stream))) return rc;
  if ((rc = host_copies(c, host, nf, false, s))) return rc;
  if (nsub_out)
    QK_CUDA(c, cudaMemcpyAsync(c->h_buf + 8, &c->d_si->nsub, sizeof(double),
                               cudaMemcpyDeviceToHost, s));
  QK_CUDA(c, cudaStreamSynchronize(s));
  if (nsub_out) *nsub_out = (int32_t)c->h_buf[8];
  return QK_OK;
}

int qk_step_compensated(qk_ctx *c, void *const hydro[5], void *const rad[4],
                        void *const hydro_lo[5], void *const rad_lo[4], double *dt_out,
                        int32_t *nsub_out, void *stream) {
  if (!c) return QK_EINVAL;
  if (!c->fp32) return fail(c, QK_EINVAL, "compensated steps need a QK_FP32_MIXED context");
  int rc = check_fields(c, hydro, 5, "hydro");
  if (rc) return rc;
  if ((rc = check_fields(c, hydro_lo, 5, "hydro_lo"))) return rc;
  if (rad && (rc = check_fields(c, rad, 4, "rad"))) return rc;
  if (rad && (rc = check_fields(c, rad_lo, 4, "rad_lo"))) return rc;
  if (c->nranks > 1)
    return fail(c, QK_EINVAL, "sharded context: compose the step from the stage entry points");
  if ((rc = need_dirichlet(c))) return rc;
  for (int f = 0; f < 9; ++f)
    if (!c->scratch_lo[f]) {
      const size_t lo_elem = c->lo_fmt == QK_LO_I16 ? 2 : 4;
      cudaError_t e = cudaMalloc(&c->scratch_lo[f], (size_t)c->field_len * lo_elem);
      if (e != cudaSuccess) return cuda_fail(c, e, "cudaMalloc(compensation scratch)");
    }
  cudaStream_t s = (cudaStream_t)stream;
  if (c->use_graph) {
    void *key[19];
    for (int q = 0; q < 5; ++q) key[q] = hydro[q];
    for (int q = 0; q < 4; ++q) key[5 + q] = rad ? rad[q] : nullptr;
    for (int q = 0; q < 5; ++q) key[9 + q] = hydro_lo[q];
    for (int q = 0; q < 4; ++q) key[14 + q] = rad ? rad_lo[q] : nullptr;
    key[18] = (void *)(intptr_t)(rad ? 1 : 0);
    if (!c->gexec_c || memcmp(key, c->gkey_c, sizeof(key)) != 0) {
      if (c->gexec_c) {
        cudaGraphExecDestroy(c->gexec_c);
        c->gexec_c = nullptr;
      }
      QK_CUDA(c, cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
      rc = enqueue_step(c, hydro, rad, c->cap_stream, hydro_lo, rad ? rad_lo : nullptr);
      cudaGraph_t graph = nullptr;
      cudaError_t e = cudaStreamEndCapture(c->cap_stream, &graph);
      if (rc) {
        if (graph) cudaGraphDestroy(graph);
        return rc;
      }
      if (e != cudaSuccess) return cuda_fail(c, e, "cudaStreamEndCapture");
      e = cudaGraphInstantiate(&c->gexec_c, graph, 0);
      cudaGraphDestroy(graph);
      if (e != cudaSuccess) return cuda_fail(c, e, "cudaGraphInstantiate");
      memcpy(c->gkey_c, key, sizeof(key));
    }
    QK_CUDA(c, cudaGraphLaunch(c->gexec_c, s));
  } else {
    if ((rc = enqueue_step(c, hydro, rad, s, hydro_lo, rad ? rad_lo : nullptr))) return rc;
  }
  if (dt_out) QK_CUDA(c, cudaMemcpyAsync(dt_out, &c->d_si->dt, sizeof(double), cudaMemcpyDeviceToHost, s));
  if (nsub_out) {
    QK_CUDA(c, cudaMemcpyAsync(c->h_buf + 8, &c->d_si->nsub, sizeof(double), cudaMemcpyDeviceToHost, s));
    QK_CUDA(c, cudaStreamSynchronize(s));
    *nsub_out = (int32_t)c->h_buf[8];
  }
  return QK_OK;
}

int qk_conserved_sums_compensated(qk_ctx *c, void *const hydro[5], void *const rad[4],
                                  void *const hydro_lo[5], void *const rad_lo[4],
                                  double out[QK_NSUMS], void *stream) {
  if (!c) return QK_EINVAL;
  if (!c->fp32) return fail(c, QK_EINVAL, "compensated sums need a QK_FP32_MIXED context");
  int rc = check_fields(c, hydro, 5, "hydro");
  if (rc) return rc;
  if ((rc = check_fields(c, hydro_lo, 5, "hydro_lo"))) return rc;
  if (rad && (rc = check_fields(c, rad, 4, "rad"))) return rc;
  if (rad && (rc = check_fields(c, rad_lo, 4, "rad_lo"))) return rc;
  if (!out) return fail(c, QK_EINVAL, "out is NULL");
  cudaStream_t s = (cudaStream_t)stream;
  QK_CUDA(c, launch_sums(c->fp32, geom(c), c->p, hydro, rad, c->d_partials, c->sum_blocks,
                         c->d_sums, s, hydro_lo, rad ? rad_lo : nullptr, c->lo_fmt));
  QK_CUDA(c, cudaMemcpyAsync(c->h_buf, c->d_sums, QK_NSUMS * sizeof(double), cudaMemcpyDeviceToHost, s));
  QK_CUDA(c, cudaStreamSynchronize(s));
  memcpy(out, c->h_buf, QK_NSUMS * sizeof(double));
  return QK_OK;
}

int qk_set_lo_format(qk_ctx *c, int32_t fmt) {
  if (!c) return QK_EINVAL;
  if (fmt != QK_LO_F32 && fmt != QK_LO_I16)
    return fail(c, QK_EINVAL, "unknown low-part format %d", fmt);
  if (fmt == c->lo_fmt) return QK_OK;
  // the stage-1 low parts and the captured step change with the format
  for (void *&p : c->scratch_lo) {
    cudaFree(p);
    p = nullptr;
  }
  if (c->gexec_c) {
    cudaGraphExecDestroy(c->gexec_c);
    c->gexec_c = nullptr;
  }
  c->lo_fmt = fmt;
  return QK_OK;
}

int qk_step_info(qk_ctx *c, double out[6], void *stream) {
  if (!c) return QK_EINVAL;
  if (!out) return fail(c, QK_EINVAL, "out is NULL");
  cudaStream_t s = (cudaStream_t)stream;
  QK_CUDA(c, cudaMemcpyAsync(c->h_buf + 24, c->d_si, sizeof(StepInfo), cudaMemcpyDeviceToHost, s));
  QK_CUDA(c, cudaStreamSynchronize(s));
  const StepInfo *h = (const StepInfo *)(c->h_buf + 24);
  out[0] = h->dt;
  out[1] = h->nsub;
  out[2] = h->dtrad;
  out[3] = h->smax;
  out[4] = h->nsub_total;
  out[5] = h->nsteps;
  return QK_OK;
}

int qk_conserved_sums(qk_ctx *c, void *const hydro[5], void *const rad[4], double out[QK_NSUMS],
                      void *stream) {
  if (!c) return QK_EINVAL;
  int rc = check_fields(c, hydro, 5, "hydro");
  if (rc) return rc;
  if (rad && (rc = check_fields(c, rad, 4, "rad"))) return rc;
  if (!out) return fail(c, QK_EINVAL, "out is NULL");
  cudaStream_t s = (cudaStream_t)stream;
  QK_CUDA(c, launch_sums(c->fp32, geom(c), c->p, hydro, rad, c->d_partials, c->sum_blocks,
                         c->d_sums, s));
  QK_CUDA(c, cudaMemcpyAsync(c->h_buf, c->d_sums, QK_NSUMS * sizeof(double), cudaMemcpyDeviceToHost, s));
  QK_CUDA(c, cudaStreamSynchronize(s));
  memcpy(out, c->h_buf, QK_NSUMS * sizeof(double));
  return QK_OK;
}

int qk_halo_info(const qk_ctx *c, int32_t peer, int64_t *send_cells, int64_t *recv_cells,
                 int32_t *owned_boxes) {
  if (!c) return QK_EINVAL;
  if (peer < 0 || peer >= c->nranks) return QK_EINVAL;
  if (send_cells) *send_cells = c->send_cells[peer];
  if (recv_cells) *recv_cells = c->recv_cells[peer];
  if (owned_boxes) *owned_boxes = (int32_t)c->own.size();
  return QK_OK;
}

static int halo(qk_ctx *c, int pack, int32_t peer, void *const *fields, int32_t first,
                int32_t nfields, void *buf, void *stream) {
  if (!c) return QK_EINVAL;
  if (peer < 0 || peer >= c->nranks) return fail(c, QK_EINVAL, "peer %d outside [0, %d)", peer, c->nranks);
  if (peer == c->rank) return fail(c, QK_EINVAL, "peer %d is this rank", peer);
  if (first < 0 || nfields < 1 || first + nfields > 9)
    return fail(c, QK_EINVAL, "fields first .. first+nfields-1 must lie in [0, 9)");
  int rc = check_fields(c, fields, nfields, "fields");
  if (rc) return rc;
  const int *ch0 = pack ? c->send_chunk0.data() : c->recv_chunk0.data();
  const long long n = pack ? c->send_cells[peer] : c->recv_cells[peer];
  if (n == 0) return QK_OK;
  if (!buf) return fail(c, QK_EINVAL, "buf is NULL");
  QK_CUDA(c, launch_halo(c->fp32, pack, pack ? c->d_send : c->d_recv,
                         (pack ? c->d_send_chunks : c->d_recv_chunks) + ch0[peer],
                         ch0[peer + 1] - ch0[peer], fields, nfields, first, buf, n,
                         DtSrc{nullptr, 0.0, 0, -1}, (cudaStream_t)stream));
  return QK_OK;
}

int qk_halo_pack(qk_ctx *c, int32_t peer, void *const *fields, int32_t first, int32_t nfields,
                 void *buf, void *stream) {
  return halo(c, 1, peer, fields, first, nfields, buf, stream);
}

int qk_halo_unpack(qk_ctx *c, int32_t peer, void *const *fields, int32_t first, int32_t nfields,
                   const void *buf, void *stream) {
  return halo(c, 0, peer, fields, first, nfields, const_cast<void *>(buf), stream);
}

int qk_signal_speed(qk_ctx *c, void *const hydro[5], double *smax, void *stream) {
  if (!c) return QK_EINVAL;
  int rc = check_fields(c, hydro, 5, "hydro");
  if (rc) return rc;
  if (!smax) return fail(c, QK_EINVAL, "smax is NULL");
  cudaStream_t s = (cudaStream_t)stream;
  QK_CUDA(c, launch_max_speed(c->fp32, geom(c), c->p, hydro, c->d_si, s));
  unsigned long long *hb = (unsigned long long *)(c->h_buf + 40);
  QK_CUDA(c, cudaMemcpyAsync(hb, &c->d_si->smax_bits, sizeof(*hb), cudaMemcpyDeviceToHost, s));
  // the running maximum starts from zero at every step
  QK_CUDA(c, cudaMemsetAsync(&c->d_si->smax_bits, 0, sizeof(*hb), s));
  QK_CUDA(c, cudaStreamSynchronize(s));
  memcpy(smax, hb, sizeof(double));
  return QK_OK;
}

int qk_set_timestep(qk_ctx *c, double smax, double out[4], void *stream) {
  if (!c) return QK_EINVAL;
  if (!(smax > 0.0) || smax != smax || smax > 1.7976931348623157e308)
    return fail(c, QK_EINVAL, "smax must be positive and finite");
  cudaStream_t s = (cudaStream_t)stream;
  double *hv = c->h_buf + 41;
  *hv = smax;
  QK_CUDA(c, cudaMemcpyAsync(&c->d_si->smax_bits, hv, sizeof(double), cudaMemcpyHostToDevice, s));
  QK_CUDA(c, launch_timestep(c->p, c->d_si, s));
  QK_CUDA(c, cudaMemcpyAsync(c->h_buf + 42, c->d_si, 4 * sizeof(double), cudaMemcpyDeviceToHost, s));
  QK_CUDA(c, cudaStreamSynchronize(s));
  if (out) memcpy(out, c->h_buf + 42, 4 * sizeof(double));
  return QK_OK;
}

int qk_status(qk_ctx *c, uint32_t *flags, int64_t *first_bad, int32_t *max_iter, int32_t reset,
              void *stream) {
  if (!c) return QK_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  Status *h = (Status *)(c->h_buf + 16);
  QK_CUDA(c, cudaMemcpyAsync(h, c->d_status, sizeof(Status), cudaMemcpyDeviceToHost, s));
  QK_CUDA(c, cudaStreamSynchronize(s));
  Status st = *h;
  if (flags) *flags = st.flags;
  if (first_bad) *first_bad = st.first_bad == ~0ull ? -1 : (int64_t)st.first_bad;
  if (max_iter) *max_iter = st.max_iter;
  if (reset) {
    Status st0{0u, 0, ~0ull, 0ull};
    *h = st0;
    QK_CUDA(c, cudaMemcpyAsync(c->d_status, h, sizeof(Status), cudaMemcpyHostToDevice, s));
    QK_CUDA(c, cudaStreamSynchronize(s));
  }
  if (st.flags & (1u << QK_ENOCONV)) return fail(c, QK_ENOCONV, "Newton exchange did not converge");
  if (st.flags & (1u << QK_ENEGATIVE)) return fail(c, QK_ENEGATIVE, "non-positive E_g or E_r");
  return QK_OK;
}

}  // extern "C"
