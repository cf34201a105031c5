// dslash kernel instantiations for float storage.
#include "dslash_inst.cuh"

namespace lqcd {
template <>
cudaError_t launch_dslash<float>(const DslashParams &P, int recon, int mode, int nr, cudaStream_t st) {
  return launch_dslash_impl<float, true, true, true>(P, recon, mode, nr, st);
}
}  // namespace lqcd
