// Gaussian deformation field, BF16 tensor-core path (placeholder until the
// tcgen05 kernel lands).
#include "fs4d_internal.cuh"

namespace fs4d {

bool deform_bf16_supported(int feat_dim, int n_levels) {
  (void)feat_dim;
  (void)n_levels;
  return false;
}

cudaError_t launch_deform_bf16(const DeformArgs& a, cudaStream_t s) {
  (void)a;
  (void)s;
  return cudaErrorNotSupported;
}

}  // namespace fs4d
