// dslash kernel instantiations for __half storage.
#include "dslash_inst.cuh"

namespace lqcd {
template <>
cudaError_t launch_dslash<__half>(const DslashParams &P, int recon, int mode, int nr, cudaStream_t st) {
  return launch_dslash_impl<__half, false, true, true>(P, recon, mode, nr, st);
}
}  // namespace lqcd
