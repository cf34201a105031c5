// Multi-right-hand-side dslash instantiations for __half storage.
#include "dslash_mrhs.cuh"

namespace lqcd {
template <>
cudaError_t launch_dslash_mrhs<__half>(const DslashParams &P, int recon, int mode, int g, cudaStream_t st) {
  if (recon == 12) return launch_mrhs_mode<__half, 12>(P, mode, g, st);
  return cudaErrorInvalidValue;
}
}  // namespace lqcd
