// Multi-right-hand-side dslash instantiations for float storage.
#include "dslash_mrhs.cuh"

namespace lqcd {
template <>
cudaError_t launch_dslash_mrhs<float>(const DslashParams &P, int recon, int mode, int g, cudaStream_t st) {
  if (recon == 12) return launch_mrhs_mode<float, 12>(P, mode, g, st);
  if (recon == 18) return launch_mrhs_mode<float, 18>(P, mode, g, st);
  return cudaErrorInvalidValue;
}
}  // namespace lqcd
