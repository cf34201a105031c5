// Multi-right-hand-side dslash instantiations for __nv_bfloat16 storage.
#include "dslash_mrhs.cuh"

namespace lqcd {
template <>
cudaError_t launch_dslash_mrhs<__nv_bfloat16>(const DslashParams &P, int recon, int mode, int g, cudaStream_t st) {
  if (recon == 12) return launch_mrhs_mode<__nv_bfloat16, 12>(P, mode, g, st);
  return cudaErrorInvalidValue;
}
}  // namespace lqcd
