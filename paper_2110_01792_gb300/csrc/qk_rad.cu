// qk_rad.cu -- radiation stage launchers: the Levermore instantiation of the
// fused radiation stage (qk_rad.cuh) and the dispatch on the closure (the
// other closures are instantiated in qk_rad_closures.cu).
#include "qk_rad.cuh"

namespace qk {

extern template cudaError_t launch_rad_closure<QK_CLOSURE_MINERBO>(
    int, int, const Geometry &, const qk_params &, void *const *, void *const *, void *const *,
    const void *, DtSrc, int, int, cudaStream_t, const LoPtrs *, const FuseArgs *);
extern template cudaError_t launch_rad_closure<QK_CLOSURE_EDDINGTON>(
    int, int, const Geometry &, const qk_params &, void *const *, void *const *, void *const *,
    const void *, DtSrc, int, int, cudaStream_t, const LoPtrs *, const FuseArgs *);

template cudaError_t launch_rad_closure<QK_CLOSURE_LEVERMORE>(
    int, int, const Geometry &, const qk_params &, void *const *, void *const *, void *const *,
    const void *, DtSrc, int, int, cudaStream_t, const LoPtrs *, const FuseArgs *);

cudaError_t launch_rad_stage(int fp32, int stage, const Geometry &g, const qk_params &p,
                             void *const *R0, void *const *R1, void *const *Rout,
                             const void *rho, DtSrc dt, int grid, int cfg, cudaStream_t s,
                             const LoPtrs *lo, const FuseArgs *fx) {
  // columns (shape 1) when the geometry has them; compensated states use tiles
  if (cfg_shape(cfg) == 1 && g.cols && g.ncols > 0 && !lo)
    return launch_rad_column(fp32, stage, g, p, R0, R1, Rout, rho, dt, fx, s, cfg);
  switch (p.closure) {
    case QK_CLOSURE_MINERBO:
      return launch_rad_closure<QK_CLOSURE_MINERBO>(fp32, stage, g, p, R0, R1, Rout, rho, dt, grid,
                                                    cfg, s, lo, fx);
    case QK_CLOSURE_EDDINGTON:
      return launch_rad_closure<QK_CLOSURE_EDDINGTON>(fp32, stage, g, p, R0, R1, Rout, rho, dt,
                                                      grid, cfg, s, lo, fx);
    default:
      return launch_rad_closure<QK_CLOSURE_LEVERMORE>(fp32, stage, g, p, R0, R1, Rout, rho, dt,
                                                      grid, cfg, s, lo, fx);
  }
}

int rad_smem_bytes(int fp32) {
  return fp32 ? (int)sizeof(RadSmem<float>) : (int)sizeof(RadSmem<double>);
}

}  // namespace qk
