// qk_rad_closures.cu -- the Minerbo and Eddington instantiations of the
// fused radiation stage (qk_rad.cuh), compiled beside qk_rad.cu.
#include "qk_rad.cuh"

namespace qk {

template cudaError_t launch_rad_closure<QK_CLOSURE_MINERBO>(
    int, int, const Geometry &, const qk_params &, void *const *, void *const *, void *const *,
    const void *, DtSrc, int, int, cudaStream_t, const LoPtrs *, const FuseArgs *);
template cudaError_t launch_rad_closure<QK_CLOSURE_EDDINGTON>(
    int, int, const Geometry &, const qk_params &, void *const *, void *const *, void *const *,
    const void *, DtSrc, int, int, cudaStream_t, const LoPtrs *, const FuseArgs *);

}  // namespace qk
