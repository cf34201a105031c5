// dslash kernel instantiations for double-float (DF64) storage: 18-real
// links only (the kernel is bound by its FP32 instruction count, and the
// 12-real form would trade bytes it does not need for arithmetic it does).
// The modes with a local term are instantiated in dslash_df64_local.cu so the
// two halves compile in parallel.
#include "dslash_inst.cuh"

namespace lqcd {
cudaError_t launch_df64_local(const DslashParams &P, int mode, int nr, cudaStream_t st);

template <>
cudaError_t launch_dslash<df>(const DslashParams &P, int recon, int mode, int nr, cudaStream_t st) {
  if (recon != 18 || P.nrhs % nr != 0) return cudaErrorInvalidValue;
  switch (mode) {
    case MODE_HOP: return launch_nr<df, 18, MODE_HOP>(P, nr, st);
    case MODE_HOP_AINV: return launch_nr<df, 18, MODE_HOP_AINV>(P, nr, st);
    case MODE_FOLDED_AINV: return launch_nr<df, 18, MODE_FOLDED_AINV>(P, nr, st);
    default: return launch_df64_local(P, mode, nr, st);
  }
}
}  // namespace lqcd
