// qk_copy.cuh -- whole-field copies by the SMs between device arrays and
// pinned host arrays mapped into the device address space (qk_step_host).
#pragma once
#include <cuda_runtime.h>

namespace qk {

// up to 9 fields, 16-byte aligned, `bytes` each, in one launch
struct FieldCopies {
  const void *src[9];
  void *dst[9];
};
cudaError_t launch_field_copies(const FieldCopies &fc, int nf, size_t bytes, cudaStream_t s);

}  // namespace qk
