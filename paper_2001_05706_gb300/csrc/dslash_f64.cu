// dslash kernel instantiations for double storage.
#include "dslash_inst.cuh"

namespace lqcd {
template <>
cudaError_t launch_dslash<double>(const DslashParams &P, int recon, int mode, int nr, cudaStream_t st) {
  return launch_dslash_impl<double, true>(P, recon, mode, nr, st);
}
}  // namespace lqcd
