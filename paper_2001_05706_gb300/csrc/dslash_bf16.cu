// dslash kernel instantiations for __nv_bfloat16 storage.
#include "dslash_inst.cuh"

namespace lqcd {
template <>
cudaError_t launch_dslash<__nv_bfloat16>(const DslashParams &P, int recon, int mode, int nr, cudaStream_t st) {
  return launch_dslash_impl<__nv_bfloat16, false>(P, recon, mode, nr, st);
}
}  // namespace lqcd
