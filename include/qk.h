/*
 * qk.h -- C ABI of the GB300 (sm_103a) per-cell uniform-patch
 * radiation-hydrodynamics update of Wibking & Krumholz, "QUOKKA"
 * (arXiv:2110.01792).
 *
 * Conventions (all entry points):
 *   - Every call returns an int status: QK_OK (0) or one of the QK_E* codes.
 *     A failing call leaves a message for qk_last_error().  No C++ exception
 *     crosses this boundary.
 *   - Field arguments are DEVICE pointers, one contiguous array per field.
 *     All patches share each array: patch b starts at element boxes[b].offset
 *     and holds (n_x+2g)(n_y+2g)(n_z+2g) cells, x fastest, the interior at
 *     local cells [g, g+n) on each axis.  The element type is double for
 *     QK_FP64 contexts and float for QK_FP32_MIXED contexts.  Hydro fields are
 *     ordered (rho, m_x, m_y, m_z, E) (density, momentum, total gas energy
 *     density); radiation fields (E_r, F_x, F_y, F_z).  The caller owns every
 *     field buffer and stream; the library owns only its context, its
 *     descriptor tables and its scratch (released by qk_destroy).
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Every launch is asynchronous on it unless stated otherwise.
 *   - Calls on one context are not thread safe; use one context per thread.
 */
#ifndef QK_H
#define QK_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define QK_OK 0
#define QK_EINVAL 1     /* invalid argument                                  */
#define QK_ECUDA 2      /* a CUDA runtime call failed                          */
#define QK_ENOCONV 3    /* a Newton exchange exceeded max_iter (Sec. 2.2.3)   */
#define QK_ENEGATIVE 4  /* a cell ended with E_g <= 0 or E_r <= 0            */

#define QK_FP64 0        /* FP64 state and arithmetic                          */
#define QK_FP32_MIXED 1  /* FP32 state and stencils; FP64 internal-energy
                            recovery, Newton exchange and conservation sums   */

#define QK_KAPPA_CONST 0 /* kappa_P, kappa_R are constant specific opacities  */
#define QK_KAPPA_RHO 1   /* kappa = kappa0 * rho with kappa0 = kappa_P/kappa_R */

#define QK_EOS_GAMMA 0   /* gamma-law gas, T = E_g / (rho c_v)                 */
#define QK_EOS_ALPHA_T3 1 /* E_g = alpha T^4 / 4, i.e. C_v = alpha T^3
                            (eq. heat_capacity; exchange test mode)           */

#define QK_NSUMS 13

typedef struct qk_ctx qk_ctx;

/* Physical and numerical parameters (Sec. 2.1-2.2).  dx is the cell size on
 * each axis; cfl is C0/D of Sec. 2.2.1 (the maximum stable value in 3-D is
 * 1/3).  eps_newton and max_iter are the Newton tolerance and iteration limit
 * of Sec. 2.2.3 (1e-10 and 400 in the paper); nsub_max is N_sub,max of
 * Sec. 2.2.4 (10).  tau_correction enables the optical-depth correction of the
 * radiation Riemann solver (Sec. 2.2.2).  hydro_only skips the radiation
 * substeps in qk_step.  recon selects PPM or PLM for both subsystems;
 * flattening enables the shock flattening of Miller & Colella (2002) on the
 * hydro reconstruction (Sec. 2.2.1; the radiation is never flattened).
 * closure selects the local M1 closure chi(f) of the radiation pressure
 * tensor (Sec. 2.2.2).  bc_lo / bc_hi give the boundary of the low / high
 * domain face on each axis (QK_BC_*); periodic faces come in pairs.  The
 * boundary types are fixed when the context is created (qk_set_params
 * rejects a change). */
typedef struct {
  double gamma;      /* adiabatic index                                        */
  double cfl;        /* CFL number                                             */
  double a_r;        /* radiation constant                                     */
  double c;          /* speed of light                                         */
  double chat;       /* reduced speed of light (RSLA), Sec. 2.1               */
  double c_v;        /* specific heat at constant volume                       */
  double kappa_P;    /* Planck mean opacity, or kappa0 (QK_KAPPA_RHO)          */
  double kappa_R;    /* Rosseland mean opacity, or kappa0 (QK_KAPPA_RHO)       */
  double alpha_eos;  /* alpha of QK_EOS_ALPHA_T3                               */
  double eps_newton; /* Newton relative tolerance                              */
  double dx[3];      /* cell size per axis                                     */
  int32_t kappa_mode;
  int32_t eos;
  int32_t max_iter;
  int32_t nsub_max;
  int32_t tau_correction;
  int32_t hydro_only;
  int32_t recon;       /* QK_RECON_PPM (default) or QK_RECON_PLM, hydro and radiation */
  int32_t flattening;  /* 1: multidimensional shock flattening of the hydro states    */
  int32_t closure;     /* QK_CLOSURE_LEVERMORE (default), _MINERBO or _EDDINGTON       */
  int32_t bc_lo[3];    /* QK_BC_* of the low face of x, y, z                            */
  int32_t bc_hi[3];    /* QK_BC_* of the high face of x, y, z                           */
} qk_params;

/* Closures (Sec. 2.2.2): P_r = [(1-chi)/2 I + (3 chi - 1)/2 n n] E_r with
 * f = |F|/(c E_r) clamped to 1 for the closure. */
#define QK_CLOSURE_LEVERMORE 0 /* chi = (3 + 4 f^2)/(5 + 2 sqrt(4 - 3 f^2))              */
#define QK_CLOSURE_MINERBO 1   /* maximum entropy, polynomial form:
                                  chi = 1/3 + (2/15)(3 f^2 - f^3 + 3 f^4)              */
#define QK_CLOSURE_EDDINGTON 2 /* chi = 1/3: P_r = E_r I / 3                           */

/* Domain boundaries.  Ghost cells beyond a face hold:
 *   PERIODIC  the interior cell of the periodic image;
 *   REFLECT   the mirror image across the face (x -> -1-x), with the vector
 *             components along that axis (m and F) negated;
 *   OUTFLOW   the nearest interior cell (zero gradient);
 *   DIRICHLET the boundary state recorded by qk_set_dirichlet.
 * Each axis is mapped on its own (edges and corners combine them); a ghost
 * cell beyond any Dirichlet face takes its recorded state.  A reflecting
 * axis needs at least nghost cells across the domain. */
#define QK_BC_PERIODIC 0
#define QK_BC_REFLECT 1
#define QK_BC_OUTFLOW 2
#define QK_BC_DIRICHLET 3

#define QK_RECON_PPM 0 /* piecewise parabolic with the paper's limiter (Sec. 2.2.1)  */
#define QK_RECON_PLM 1 /* piecewise linear, monotonized-central slope (Sec. 2.2.1)  */

/* One patch: lower corner in the periodic domain, interior extents, and the
 * element offset of its first (ghost) cell in every field array. */
typedef struct {
  int32_t lo[3];
  int32_t n[3];
  int64_t offset;
} qk_box;

/* Create a context for a set of patches that tile the periodic domain
 * [0, domain_n) exactly once (Sec. 2.2, domain decomposition into boxes).
 * Validates the boxes (inside the domain, no overlap, full cover, disjoint
 * field ranges), builds the tile work list and the ghost-copy descriptors
 * (periodic images included), uploads them, and allocates the scratch for
 * qk_step (one extra copy of each field).  nghost >= 3 (the PPM stencil reach).
 * precision is QK_FP64 or QK_FP32_MIXED.  Must be called with the target device
 * current.  On failure *out is NULL and the status says why. */
int qk_init_patches(qk_ctx **out, const qk_params *p, const qk_box *boxes, int32_t nbox,
                    const int32_t domain_n[3], int32_t nghost, int32_t precision);

/* A shard of a patch set for one rank of a multi-GPU run (Sec. 4: the
 * update is distributed by patches and the ghost exchange between them is
 * the only data-path communication).  `boxes`, `nbox`, `domain_n` describe the
 * WHOLE patch set, identically on every rank; owner[b] in [0, nranks) names
 * the rank that holds patch b (caller-owned host array of nbox entries).  This
 * context advances only the patches with owner[b] == rank: their offsets
 * place them in this rank's field arrays (offsets of other ranks' patches are
 * not read) and every per-cell entry point works on them alone.
 * qk_fill_ghosts then fills only the ghost regions whose source is also owned
 * here; the rest travel through qk_halo_pack / qk_halo_unpack.  With
 * nranks > 1, qk_step and qk_timestep return QK_EINVAL (they would need the
 * other ranks' cells): a sharded step is composed from the stage entry points,
 * qk_signal_speed and qk_set_timestep.  Returns QK_EINVAL
 * when owner is NULL, an owner is out of range, or the rank owns no patch. */
int qk_init_shard(qk_ctx **out, const qk_params *p, const qk_box *boxes, int32_t nbox,
                  const int32_t domain_n[3], int32_t nghost, int32_t precision,
                  const int32_t *owner, int32_t nranks, int32_t rank);

/* Host-only view of the ghost-fill plan that qk_init_patches would build
 * for this patch set (no GPU call; for inspection and CPU-side checks of the
 * boundary handling).  Writes at most `cap` records of 12 int64 each to
 * `out`, copies first, then Dirichlet regions:
 *   copy:      dst, src, ex, ey, ez, dsx, dsy, flip, sx, sy, sz, 0
 *              (destination cell (x, y, z) of the region is element
 *               dst + (z dsy + y) dsx + x; its source is src + x sx + y sy +
 *               z sz; flip bit d negates the d-components of vectors)
 *   Dirichlet: dst, 0, ex, ey, ez, dsx, dsy, 0, 0, 0, 0, 1
 *              (a region whose cells take the recorded boundary state).
 * *ncopies and *ndirichlet receive the full counts (records beyond cap are
 * not written).  Validation as qk_init_patches; failures are reported through
 * qk_last_error(NULL). */
int qk_fill_plan(const qk_params *p, const qk_box *boxes, int32_t nbox,
                 const int32_t domain_n[3], int32_t nghost, int64_t *out, int64_t cap,
                 int64_t *ncopies, int64_t *ndirichlet);

/* Free the context and all library-owned device memory. */
void qk_destroy(qk_ctx *ctx);

/* Message of the last failing call on this context (never NULL); with
 * ctx == NULL, the message of the last failed qk_init_patches on this thread. */
const char *qk_last_error(const qk_ctx *ctx);

/* Minimum number of elements of each field array (max over patches of
 * offset + padded volume). */
int64_t qk_field_len(const qk_ctx *ctx);

/* Number of interior cells over all patches. */
int64_t qk_num_cells(const qk_ctx *ctx);

/* Replace the parameters (same patch set).  Captured step graphs are dropped. */
int qk_set_params(qk_ctx *ctx, const qk_params *p);

/* Fill the ghost cells of `nfields` field arrays (Sec. 2.2, 'FillBoundary'):
 * every ghost cell of every patch receives the value of the interior cell that
 * owns its periodic image (or, at non-periodic faces, its QK_BC_* value).  One
 * batched launch over precomputed copy descriptors (plus one for Dirichlet
 * states).  fields[i] holds state field i of (rho, m_x, m_y, m_z, E, E_r,
 * F_x, F_y, F_z). */
int qk_fill_ghosts(qk_ctx *ctx, void *const *fields, int32_t nfields, void *stream);

/* The same fill for fields that hold the state fields first .. first+nfields-1
 * of the list (rho, m_x, m_y, m_z, E, E_r, F_x, F_y, F_z): their identity
 * decides which values change sign at a reflecting face and which Dirichlet
 * states they take (qk_fill_ghosts is first = 0).  Under non-periodic
 * boundaries every ghost cell follows the QK_BC_* rule of its faces. */
int qk_fill_ghosts_range(qk_ctx *ctx, void *const *fields, int32_t first, int32_t nfields,
                         void *stream);

/* Record the Dirichlet boundary states: the values the caller's hydro and
 * radiation arrays (rad may be NULL: zero radiation) hold in the ghost cells
 * beyond the QK_BC_DIRICHLET faces are copied into library storage (9 values
 * per such ghost cell, on the device); every later ghost fill restores them.
 * Must precede any fill or step of a context with Dirichlet faces (those
 * calls return QK_EINVAL until it has been made); call again to change the
 * states.  Asynchronous on `stream`. */
int qk_set_dirichlet(qk_ctx *ctx, void *const hydro[5], void *const rad[4], void *stream);

/* Radiation source of the matter-radiation exchange (Sec. 2.2.3, the S of
 * eq. F_R): `j` is a device field (the context's element type and layout)
 * holding an emissivity per cell, energy per unit volume per unit time in
 * the physical energy equation; each exchange of duration dt_rad adds
 * S = dt_rad (chat/c) j to the radiation-energy residual (the reduced-speed
 * form of that equation).  NULL removes it.  The caller keeps the array alive
 * while it is set; qk_step and qk_rad_matter_exchange read it.  Captured step
 * graphs are dropped. */
int qk_set_source(qk_ctx *ctx, const void *j);

/* One RK2-SSP stage of the hydro update (Sec. 2.2.1): conserved -> primitive,
 * PPM reconstruction of (rho, v, P) per direction, HLLC fluxes with PVRS
 * wavespeeds, flux divergence, and
 *   stage 1: Uout = U0 + dt L(U0)
 *   stage 2: Uout = U0/2 + (U1 + dt L(U1))/2.
 * The stencil source (U0 in stage 1, U1 in stage 2) must have its ghosts
 * filled.  Uout may equal U0 in stage 2 (in place), never the stencil source.
 * U1 is ignored in stage 1.  Face fluxes never leave the chip.  With
 * flattening, the coefficient is computed from the stencil source first (one
 * extra launch into library scratch). */
int qk_hydro_stage(qk_ctx *ctx, int32_t stage, void *const U0[5], void *const U1[5],
                   void *const Uout[5], double dt, void *stream);

/* One RK2-SSP stage of the radiation transport (Sec. 2.2.2): PPM of E_r and
 * the reduced flux f = F/(c E_r), first-order fallback at faces where a state
 * has |f| > 1, Levermore closure (eq. M1_closure), HLL flux with wavespeeds from
 * the cell-average Eddington factors and the optical-depth correction, RSLA
 * fluxes ((chat/c) F, c chat P_r) (eqs. rad_energy, rad_flux).  rho (the hydro
 * density field, ghosts filled) sets the optical depth.  Same stage and alias
 * rules as qk_hydro_stage. */
int qk_rad_stage(qk_ctx *ctx, int32_t stage, void *const R0[4], void *const R1[4],
                 void *const Rout[4], const void *rho, double dt_rad, void *stream);

/* Radiation stage 2 with the matter-radiation exchange of every cell in its
 * epilogue (Sec. 2.2.2 then Sec. 2.2.3, per cell): the same result as
 * qk_rad_stage(stage 2) followed by qk_rad_matter_exchange on Rout, in one
 * launch (the form qk_step uses).  hydro is read and its momenta and energy
 * are updated; its density (ghosts filled) sets the optical depth.  Rout may
 * alias R0, not R1.  Newton failures go to the context status (qk_status). */
int qk_rad_stage2_exchange(qk_ctx *ctx, void *const R0[4], void *const R1[4],
                           void *const Rout[4], void *const hydro[5], double dt_rad,
                           void *stream);

/* Per-cell implicit matter-radiation exchange over dt_rad (Sec. 2.2.3), in
 * FP64 for both precisions: Newton-Raphson on (E_g, E_r) with the residuals
 * F_G, F_R and eqs. delta_er / delta_eg, the backward-Euler flux source
 * F <- F/(1 + rho kappa_R chat dt), the momentum update m -= dF/(c chat), and
 * the work term through the kinetic-energy change.  Updates hydro (m, E) and
 * rad (E_r, F) in place.  A cell that does not converge within max_iter sets
 * QK_ENOCONV in the context status (see qk_status); the kernel never traps
 * and always ends. */
int qk_rad_matter_exchange(qk_ctx *ctx, void *const hydro[5], void *const rad[4],
                           double dt_rad, void *stream);

/* Device-side timestep (Sec. 2.2.1, Sec. 2.2.4) of the current hydro state:
 * dt = CFL dx_min / max(|v| + c_s); with radiation, at most N_sub,max substeps
 * of CFL dx_min / chat, N_sub = ceil(dt / (CFL dx_min / chat)) otherwise,
 * dt_rad = dt / N_sub.  Synchronises `stream` and returns
 * out[0] = dt, out[1] = N_sub, out[2] = dt_rad, out[3] = max(|v| + c_s). */
int qk_timestep(qk_ctx *ctx, void *const hydro[5], double out[4], void *stream);

/* One full update (operator split, Sec. 2.2): timestep on the device, ghost
 * fill + hydro stage 1, ghost fill + hydro stage 2, then N_sub radiation
 * substeps, each: ghost fill + radiation stage 1, ghost fill + radiation
 * stage 2, exchange.  rad == NULL (or hydro_only) runs hydro alone.  The
 * launch sequence is captured once into a CUDA graph per (hydro, rad) pointer
 * set and replayed (N_sub,max predicated substeps; those beyond N_sub exit at
 * once).  dt_out / nsub_out, when not NULL, receive dt and N_sub of this step
 * by an asynchronous copy: valid after `stream` synchronises (use pinned host
 * memory to keep the call asynchronous). */
int qk_step(qk_ctx *ctx, void *const hydro[5], void *const rad[4], double *dt_out,
            int32_t *nsub_out, void *stream);

/* One full update of a compensated FP32 state (QK_FP32_MIXED contexts only):
 * every conserved field is held as the unevaluated sum hi + lo of two float
 * arrays, hydro/rad the hi parts (what the stencils read, exactly as in
 * qk_step) and hydro_lo/rad_lo the low parts (caller-owned, same layout;
 * zero for a state that starts as plain floats).  The update is qk_step's,
 * with the RK combinations accumulated in double-float (every face term dt F/dx
 * rounded once, identically in both cells sharing the face) and the exchange's
 * invariants E + (c/chat) E_r and m + F/(c chat) carried to ~2^-48, so that the
 * periodic conserved totals (qk_conserved_sums_compensated) drift by rounding
 * at the 1e-14 level instead of the ~1e-11 per step of FP32 storage
 * (Sec. 2.2's conservative update; not a passage of the paper, a storage
 * choice).  The first call allocates nine fields of library scratch for the
 * low parts of the stage-1 results; the launch sequence is captured into its
 * own CUDA graph per pointer set.  QK_EINVAL for an FP64 or sharded context
 * or a NULL field. */
int qk_step_compensated(qk_ctx *ctx, void *const hydro[5], void *const rad[4],
                        void *const hydro_lo[5], void *const rad_lo[4], double *dt_out,
                        int32_t *nsub_out, void *stream);

/* Storage of the low parts of a compensated state (qk_step_compensated,
 * qk_conserved_sums_compensated).  QK_LO_F32 (the default): float arrays, the
 * value hi + lo held to ~48 bits in 8 bytes.  QK_LO_I16: int16 arrays (the
 * caller's hydro_lo / rad_lo then hold 2-byte elements), lo kept as the
 * integer k = rint(lo 2^(38 - E)), E the binary exponent of hi, i.e. to 2^-15
 * of an FP32 ulp of hi: ~39 significant bits in 6 bytes per value, three
 * quarters of FP64's bytes, with the same exact telescoping of the face terms
 * in the accumulation (every store rounds the value once, at ~2^-40).  Values
 * below ~2^-100 in magnitude keep hi only.  Not a passage of the paper (a
 * storage choice of the conservative update, Sec. 2.2).  Changing the format
 * releases the library's stage-1 low parts and the captured compensated step.
 * QK_EINVAL for another value. */
#define QK_LO_F32 1
#define QK_LO_I16 2
int qk_set_lo_format(qk_ctx *ctx, int32_t fmt);

/* The device step record (synchronises `stream`): out[0] = dt, out[1] = N_sub,
 * out[2] = dt_rad, out[3] = max(|v| + c_s) of the last timestep computed;
 * out[4] = radiation substeps and out[5] = timesteps summed since the context
 * was created. */
int qk_step_info(qk_ctx *ctx, double out[6], void *stream);

/* Autotune the launch configuration of the four stage kernels (hydro stage
 * 1/2, radiation stage 1/2): the tile shape and schedule -- 8^3 tiles with
 * 128, 256 or 512 threads per CTA (the same shared-memory tile), strided over
 * the grid or one contiguous run of tiles per CTA, or 16 x 16 columns of 256
 * threads marching along z (FP32 hydro: also of 288 threads, whose ninth warp
 * evens out the per-plane work, at 3 or 2 CTAs per SM) -- each timed with CUDA
 * events on the caller's state; the fastest is kept for qk_step and the stage
 * entry points of this context.  rad may be NULL (hydro only).  The state is
 * not changed except that its ghost cells are refilled; radiation stage 2 is
 * timed with the exchange fused when qk_step fuses it (on a copy of the gas
 * state); allocates and frees temporary copies of five (ten with the fused
 * exchange) fields; synchronises `stream`.  out_cfg (may be
 * NULL) receives the choices as threads | schedule << 16 | shape << 17
 * (shape 1: columns).  Results do not depend on the configuration beyond the
 * rounding of identical formulas. */
int qk_autotune(qk_ctx *ctx, void *const hydro[5], void *const rad[4], int32_t out_cfg[4],
                void *stream);

/* Set the launch configuration of the four stage kernels (hydro stage 1/2,
 * radiation stage 1/2) directly, in qk_autotune's encoding: threads (128,
 * 256, 512) | schedule (0 strided, 1 contiguous) << 16 | shape << 17, shape 1
 * being 16 x 16 columns of 256 threads (schedule 0) or of 288 threads
 * (schedule 0: registers held to 3 CTAs per SM, 1: to 2; FP32 hydro stages --
 * elsewhere a 288-thread column configuration runs as 256).  Compensated steps
 * (qk_step_compensated) and the tile parts of sharded contexts always use the
 * 8^3 tiles.  QK_EINVAL for any other value. */
int qk_set_launch_config(qk_ctx *ctx, const int32_t cfg[4]);

#define QK_LAUNCH_BATCHED 0   /* one persistent launch per stage over all patches */
#define QK_LAUNCH_PER_PATCH 1 /* one launch per patch and stage (for comparison)  */

/* Select how qk_step launches the hydro and radiation stage kernels (the
 * default is QK_LAUNCH_BATCHED).  Results are identical; captured step graphs
 * are dropped. */
int qk_set_launch_mode(qk_ctx *ctx, int32_t mode);

/* qk_step (and qk_step_compensated): run the matter-radiation exchange of
 * every substep in the epilogue of radiation stage 2 (1, default), or as its
 * own launch after it (0).  The exchange is pointwise (Sec. 2.2.3) and reads
 * exactly the state stage 2 produces, so both give identical results; fusing
 * saves re-reading the state and lets the exchange's FP64 work overlap the
 * stage's FP32 work on the same SMs. */
int qk_set_fused_exchange(qk_ctx *ctx, int32_t enable);

/* Enable (1, default) or disable (0) CUDA-graph capture in qk_step. */
int qk_set_graph(qk_ctx *ctx, int32_t enable);

/* Conservation sums over the interior cells times the cell volume, in
 * compensated FP64 with a fixed reduction order (bitwise reproducible):
 * out[0] = sum rho, out[1..3] = sum m, out[4] = sum E, out[5] = sum E_r,
 * out[6..8] = sum F, out[9] = sum (E + (c/chat) E_r),
 * out[10..12] = sum (m + F/(c chat)) (the quantities that the RSLA system
 * conserves, Sec. 3.2.3).  rad may be NULL (radiation entries are then 0).
 * Synchronises `stream`. */
int qk_conserved_sums(qk_ctx *ctx, void *const hydro[5], void *const rad[4],
                      double out[QK_NSUMS], void *stream);

/* qk_conserved_sums of a compensated FP32 state (see qk_step_compensated):
 * each cell contributes hi + lo of every field.  Same output layout. */
int qk_conserved_sums_compensated(qk_ctx *ctx, void *const hydro[5], void *const rad[4],
                                  void *const hydro_lo[5], void *const rad_lo[4],
                                  double out[QK_NSUMS], void *stream);

/* Conservation sums without any GPU allocation.  There is no counterpart in the
 * paper: this serves callers that cannot call cudaMalloc where they need the
 * totals (a diagnostics hook that runs between steps under a fixed memory
 * budget, a process whose device memory is owned by an external allocator, or
 * code that never creates a qk_ctx).  It launches kernels and synchronises
 * `stream`, so it must not be called from a CUDA stream host callback (CUDA
 * API calls are not allowed there).
 * It computes exactly what qk_conserved_sums computes (same kernels, same
 * fixed reduction order, same output layout and units, bit-identical
 * results) for the patch set `boxes` (the layout of the field arrays, as given
 * to qk_init_patches, patches disjoint), and copies the QK_NSUMS results to
 * the host array `out`.  field_len: elements of every field array; a patch
 * whose padded extent (n + 2 nghost per axis, from its offset) ends beyond it
 * is rejected with QK_EINVAL, so no kernel reads past the arrays.  All
 * working memory (patch table, partial sums, result) lives in one static
 * device array of QK_NOALLOC_SCRATCH_BYTES inside the library, held by every
 * GPU that loads the library until the process exits; at most
 * QK_NOALLOC_MAX_BOXES patches (QK_EINVAL beyond that).  On failure a message
 * is written to `err` (a caller-owned buffer of `errlen` bytes; may be NULL).
 * The call allocates nothing and synchronises `stream`.  The first call on
 * each device looks up the array's device address (cudaGetSymbolAddress) with
 * that device current and keeps it for the life of the process; make that
 * first call outside any stream capture, and make none after a
 * cudaDeviceReset (which unloads the array; the kept address would be stale).
 * Every call overwrites the whole array, so nothing carries over between
 * calls, but calls that overlap on the GPU (other streams, other host
 * threads) race on it. */
#define QK_NOALLOC_MAX_BOXES 4096
#define QK_NOALLOC_SCRATCH_BYTES (576 * 1024)
int qk_conserved_sums_noalloc(const qk_params *p, const qk_box *boxes, int32_t nbox,
                              int32_t nghost, int32_t precision, int64_t field_len,
                              void *const hydro[5], void *const rad[4], double out[QK_NSUMS],
                              void *stream, char *err, int32_t errlen);

/* Halo sizes of a sharded context: *send_cells = cells per field this rank
 * sends to `peer`, *recv_cells = cells per field it receives from `peer`,
 * *owned_boxes = patches this rank holds (any pointer may be NULL).  For a
 * context from qk_init_patches there is one rank (peer 0, no halo). */
int qk_halo_info(const qk_ctx *ctx, int32_t peer, int64_t *send_cells, int64_t *recv_cells,
                 int32_t *owned_boxes);

/* Cross-rank ghost exchange (Sec. 4, FillBoundary across GPUs).  Pack gathers,
 * from this rank's `nfields` field arrays (state fields first ..
 * first+nfields-1, as in qk_fill_ghosts_range: the sign flips of reflecting
 * faces are applied while packing), the interior cells that `peer`'s
 * ghost regions need, into the device buffer `buf` of nfields x send_cells
 * elements (the context's precision; field-major, regions in one order agreed
 * by both ranks, x fastest).  Unpack scatters a buffer received from `peer`
 * (nfields x recv_cells elements, same layout) into this rank's ghost cells.
 * The caller moves the buffer between the ranks (NCCL send/recv, a peer copy,
 * or a plain device copy when both ranks share one GPU); the library never
 * waits on another rank.  A full ghost fill of a sharded context is
 * qk_fill_ghosts plus, for every peer, pack -> transfer -> unpack.  QK_EINVAL
 * for peer == this rank or out of range; nothing is launched when the halo to
 * that peer is empty. */
int qk_halo_pack(qk_ctx *ctx, int32_t peer, void *const *fields, int32_t first, int32_t nfields,
                 void *buf, void *stream);
int qk_halo_unpack(qk_ctx *ctx, int32_t peer, void *const *fields, int32_t first,
                   int32_t nfields, const void *buf, void *stream);

/* Overlap of the halo exchange with the stage work (Sec. 4: the boundary
 * fill dominated the paper's multi-GPU runs).  In a sharded context the tiles
 * are split at creation into interior tiles, whose stencils (reach 4 cells,
 * flattening included) touch no ghost cell that another rank fills, and
 * boundary tiles.  qk_set_tile_part selects the tiles that later
 * qk_hydro_stage / qk_rad_stage calls process (with their flattening
 * pre-pass): QK_PART_ALL (default), QK_PART_INTERIOR or QK_PART_BOUNDARY.
 * A stage may therefore run on the interior tiles as soon as the rank-local
 * ghosts are filled and the halo is packed, and on the boundary tiles after
 * the halo is unpacked; the two launches write disjoint cells and together
 * give exactly the full stage.  qk_tile_counts reports the split (a context
 * from qk_init_patches has no boundary tiles).  Per-patch launches
 * (qk_set_launch_mode) apply only to QK_PART_ALL. */
#define QK_PART_ALL 0
#define QK_PART_INTERIOR 1
#define QK_PART_BOUNDARY 2
int qk_set_tile_part(qk_ctx *ctx, int32_t part);
int qk_tile_counts(const qk_ctx *ctx, int32_t *n_interior, int32_t *n_boundary);

/* Global timestep of a sharded step, in two halves around the caller's
 * max-reduction over ranks (Sec. 2.2: one dt from the CFL condition on the
 * whole domain).  qk_signal_speed writes the maximum of |v| + c_s over this
 * context's cells to *smax (host); qk_set_timestep takes the global maximum
 * and computes dt, N_sub and dt_rad on the device exactly as qk_step does,
 * writing (dt, N_sub, dt_rad, smax) to out (may be NULL).  Both synchronise
 * `stream`.  qk_set_timestep returns QK_EINVAL unless smax is positive and
 * finite. */
int qk_signal_speed(qk_ctx *ctx, void *const hydro[5], double *smax, void *stream);
int qk_set_timestep(qk_ctx *ctx, double smax, double out[4], void *stream);

/* ---- Mesh refinement (two levels; Sec. 2.2, Berger & Colella 1989) ----
 * A refinement level is a patch set that need not cover its domain.  Its
 * ghost cells that no patch of the level covers are left to qk_amr_interp;
 * the rest is as qk_init_patches.  Refinement levels are periodic. */
int qk_init_level(qk_ctx **out, const qk_params *p, const qk_box *boxes, int32_t nbox,
                  const int32_t domain_n[3], int32_t nghost, int32_t precision);

/* A coarse level (covering its periodic domain) and a fine level with cells
 * a factor 2 smaller (domain twice as many cells, dx half, patches aligned to
 * coarse cells, same precision and ghost width).  qk_amr_init builds, on the
 * host, the lists of: fine ghost cells outside the fine region (with their
 * coarse parents), coarse-fine faces (each with its four fine faces and the
 * uncovered coarse cell beside it), and coarse cells under the fine region;
 * and zeroes the flux registers.  Both contexts must outlive the handle. */
typedef struct qk_amr qk_amr;
int qk_amr_init(qk_amr **out, qk_ctx *coarse, qk_ctx *fine);
void qk_amr_destroy(qk_amr *amr);
/* Message of the last failing call on `amr` (or of the last failed
 * qk_amr_init on this thread when amr is NULL). */
const char *qk_amr_last_error(const qk_amr *amr);
/* Sizes of the lists: fine ghost cells filled by interpolation, coarse-fine
 * faces, coarse cells under the fine region (pointers may be NULL). */
int qk_amr_info(const qk_amr *amr, int64_t *n_cf_ghosts, int64_t *n_faces, int64_t *n_covered);

/* Fill the fine ghost cells outside the fine region of `nfields` fine arrays
 * holding state fields first .. first+nfields-1 (as qk_fill_ghosts_range)
 * from the coarse state (1 - alpha) c_old + alpha c_new (arrays of all nine
 * state fields; only the requested ones are read; their ghost cells filled):
 * per axis, a quarter of the monotonized-central slope of the coarse
 * conserved variable toward the fine cell (conservative linear
 * interpolation; the paper uses linear interpolation for robustness). */
int qk_amr_interp(qk_amr *amr, void *const c_old[9], void *const c_new[9], double alpha,
                  void *const *fine_fields, int32_t first, int32_t nfields, void *stream);

/* Flux register: accumulate `weight` times the flux through every
 * coarse-fine face (level 0: the coarse face; level 1: each of its four fine
 * faces with a quarter of the weight) computed from the given state with the
 * stage's arithmetic.  kind 0: hydro, fields = the 5 hydro arrays; kind 1:
 * radiation, fields = the 4 radiation arrays and rho.  Ghost cells must be
 * filled; with flattening, call it right after the stage on the same state
 * (its coefficients are reused).  For one RK2-SSP step of duration dt the
 * weights are dt/2 for the stage-1 and the stage-2 input states. */
int qk_amr_register(qk_amr *amr, int32_t level, int32_t kind, void *const *fields,
                    const void *rho, double weight, void *stream);

/* Level synchronisation: every uncovered coarse cell beside the fine region
 * gets -side (fine - coarse flux integral) / dx through each of its
 * coarse-fine faces (side +1 when the cell is on the face's low side), then
 * every coarse cell under the fine region becomes the mean of its eight fine
 * cells; the registers are zeroed.  cR and fR are both NULL for hydro only. */
int qk_amr_sync(qk_amr *amr, void *const cU[5], void *const cR[4], void *const fU[5],
                void *const fR[4], void *stream);

/* Read the accumulated exchange status (synchronises `stream`):
 * *flags = bit (1 << QK_ENOCONV) | bit (1 << QK_ENEGATIVE); *first_bad = the
 * smallest element index of a failing cell (-1 if none); *max_iter = the
 * largest Newton iteration count seen.  reset != 0 clears the status.
 * Returns QK_ENOCONV / QK_ENEGATIVE when those bits are set, else QK_OK. */
int qk_status(qk_ctx *ctx, uint32_t *flags, int64_t *first_bad, int32_t *max_iter,
              int32_t reset, void *stream);

/* The library's FP64 reciprocal and square root, element-wise over n device
 * doubles x: rcp[i] = 1/x[i] (hardware approximate reciprocal with one
 * third-order correction) and sqrt_out[i] = sqrt(x[i]) (hardware approximate
 * reciprocal square root with a second-order correction), the forms the FP64
 * stage kernels use for the divisions and square roots of Sec. 2.2.1-2.2.2
 * (HLLC sound speeds, Levermore closure, HLL wavespeed).  Either output may be
 * NULL.  Valid for positive normal x with a normal reciprocal (and x = 0 for
 * the square root); each result is meant to lie within one ulp of the IEEE
 * value.  Asynchronous on `stream`; QK_EINVAL if n < 0 or x is NULL with
 * n > 0, QK_ECUDA if the launch fails. */
int qk_eval_math(const double *x, int64_t n, double *rcp, double *sqrt_out, void *stream);

/* The library's integer-pipe conversions, element-wise over n device values
 * (either pair may be NULL): d_out[i] = f_in[i] widened to double (exact, for
 * every float), f_out[i] = d_in[i] narrowed to float by truncation toward
 * zero (within one FP32 ulp; magnitudes below the normal float range give a
 * signed zero, above it the largest finite float).  The mixed-precision
 * exchange (Sec. 2.2.3) uses them in place of conversion instructions, which
 * occupy the FP64 pipe on this part.  Asynchronous on `stream`; QK_EINVAL if
 * n < 0, QK_ECUDA if the launch fails. */
int qk_eval_convert(const float *f_in, double *d_out, const double *d_in, float *f_out, int64_t n,
                    void *stream);

/* qk_step on a state held in host memory (the end-to-end form of the
 * update): copies the 5 hydro (and 4 radiation) fields of all patches,
 * field_len elements each in the context's precision, from the caller's host
 * arrays (pinned or pageable; pinned ones move by DMA at full rate) into
 * device copies owned by the context (allocated on the first call), runs
 * qk_step on them and copies the updated fields back into the same host
 * arrays.  The copies are spread over three internal streams (one field per
 * copy engine at a time) and ordered after the work already on `stream`;
 * the call returns when the host arrays hold the result.  dt_out and
 * nsub_out as in qk_step (dt_out must then be host memory that stays valid
 * until the call returns).  QK_EINVAL for a NULL field; QK_ECUDA if an
 * allocation, copy or launch fails. */
int qk_step_host(qk_ctx *ctx, void *const hydro[5], void *const rad[4], double *dt_out,
                 int32_t *nsub_out, void *stream);

/* FMA throughput probe (not part of the method): the ALU peak against which
 * the stage kernels' arithmetic is measured.  Launches min(8 x SMs,
 * sink_len / 256) blocks of 256 threads; each thread runs 8 independent
 * chains a <- a (1 - 2^-20) + 2^-10 for `iters` steps, starting from
 * a = (thread index mod 32) + chain index, in FP64 (fp64 != 0) or FP32, and
 * stores the sum of its chains in sink[thread] (device array of sink_len
 * doubles or floats, owned by the caller).  *flops (may be NULL) receives the
 * flop count of the launch (2 per step and chain); the caller times the
 * launch on `stream`.  QK_EINVAL if iters < 1, sink is NULL or sink_len < 256,
 * QK_ECUDA if the launch fails. */
int qk_fma_probe(int32_t fp64, int64_t iters, void *sink, int64_t sink_len, double *flops,
                 void *stream);

#ifdef __cplusplus
}
#endif

#endif /* QK_H */
