// qk_column_rad.cu -- instantiations of the plane-marching radiation stage
// (qk_column_rad.cuh) for the three closures, and its dispatch.
#include "qk_column_rad.cuh"

namespace qk {

cudaError_t launch_rad_column(int fp32, int stage, const Geometry &g, const qk_params &p,
                              void *const *R0, void *const *R1, void *const *Rout,
                              const void *rho, DtSrc dt, const FuseArgs *fx, cudaStream_t s,
                              int cfg) {
  switch (p.closure) {
    case QK_CLOSURE_MINERBO:
      return launch_rad_column_closure<QK_CLOSURE_MINERBO>(fp32, stage, g, p, R0, R1, Rout, rho,
                                                           dt, fx, s, cfg);
    case QK_CLOSURE_EDDINGTON:
      return launch_rad_column_closure<QK_CLOSURE_EDDINGTON>(fp32, stage, g, p, R0, R1, Rout, rho,
                                                             dt, fx, s, cfg);
    default:
      return launch_rad_column_closure<QK_CLOSURE_LEVERMORE>(fp32, stage, g, p, R0, R1, Rout, rho,
                                                             dt, fx, s, cfg);
  }
}

}  // namespace qk
