// qk_ctx.cuh -- the context of include/qk.h's opaque qk_ctx, shared by the
// host-side translation units of libqk (qk_api.cu builds and drives it;
// qk_amr.cu reads the geometry of two refinement levels).
#pragma once

#include <string>
#include <vector>

#include "qk_internal.cuh"

using namespace qk;

struct qk_ctx {
  qk_params p{};
  int fp32 = 0;
  int ng = 0;
  int nbox = 0;
  int partial = 0;      // a refinement level: the patches need not cover the domain
  int dom[3] = {0, 0, 0};
  std::vector<qk_box> boxes;
  int64_t field_len = 0;
  int64_t ncells = 0;
  // device tables
  DevBox *d_boxes = nullptr;
  Tile *d_tiles = nullptr;
  long long *d_cell0 = nullptr;
  int ntiles = 0;
  int nbox_dev = 0;            // patches in the device table (the owned ones)
  std::vector<int> tile_start;  // first tile of each owned patch (tiles grouped by patch)
  // sharded contexts: the same tiles reordered, interior tiles (no ghost cell
  // filled from another rank within their stencil reach) first, then the
  // boundary tiles; `part` selects which ones the stage launches process
  Tile *d_tiles_ib = nullptr;
  Column *d_cols = nullptr;    // column work list of the plane-marching kernels
  int ncols = 0;
  std::vector<int> col_start;  // first column of each owned patch (grouped by patch)
  Column *d_cols2 = nullptr;   // FP32: the list chunked for two column CTAs per SM
  int ncols2 = 0;
  std::vector<int> col_start2;
  int n_interior = 0;
  int part = QK_PART_ALL;
  // sharded contexts: owner rank of every patch, this rank, and the halo
  // descriptors exchanged with each peer (send: owned source -> buffer;
  // recv: buffer -> owned ghost region), in one global order on every rank
  std::vector<int> owner;
  int rank = 0, nranks = 1;
  std::vector<int> own;          // owned patch indices (global numbering)
  Copy *d_send = nullptr, *d_recv = nullptr;
  Chunk *d_send_chunks = nullptr, *d_recv_chunks = nullptr;
  std::vector<int> send_chunk0, recv_chunk0;  // per peer: chunk range [p], [p+1)
  std::vector<long long> send_cells, recv_cells;
  int launch_mode = QK_LAUNCH_BATCHED;
  int fuse_exchange = 1;  // qk_step: exchange in the epilogue of radiation stage 2
  int cfg[4] = {kDefaultCfg, kDefaultCfg, kDefaultCfg, kDefaultCfg};  // hydro1/2, rad1/2
  Copy *d_copies = nullptr;
  Chunk *d_chunks = nullptr;
  int ncopies = 0, nchunks = 0;
  // Dirichlet boundary store: 9 fields x ndir cells, recorded by
  // qk_set_dirichlet from the caller's ghost cells, restored by every fill
  Copy *d_dpack = nullptr, *d_dunpack = nullptr;
  Chunk *d_dchunks = nullptr;
  int ndchunks = 0;
  long long ndir = 0;
  void *dstore = nullptr;
  int dir_set = 0;
  StepInfo *d_si = nullptr;
  Status *d_status = nullptr;
  double *d_partials = nullptr;
  double *d_sums = nullptr;
  int sum_blocks = 0;
  void *scratch[9] = {};
  void *scratch_lo[9] = {};  // low parts of the stage-1 results (compensated steps)
  int lo_fmt = QK_LO_F32;    // storage of the low parts (QK_LO_F32 or QK_LO_I16)
  void *chi = nullptr;   // shock-flattening coefficient (one field)
  const void *src = nullptr;  // caller's emissivity field j of the exchange, or none
  size_t elem = 8;
  // pinned host staging
  double *h_buf = nullptr;
  // qk_step_host: device copy of a host-resident state, and the streams and
  // events that spread its copies over the copy engines
  void *hstate[9] = {};
  cudaStream_t hcopy[3] = {};
  cudaEvent_t hcopy_ev[4] = {};
  // step graph
  int use_graph = 1;
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t gexec = nullptr;
  void *gkey[10] = {};
  cudaGraphExec_t gexec_c = nullptr;  // compensated step graph
  void *gkey_c[19] = {};
  std::string err;
};
