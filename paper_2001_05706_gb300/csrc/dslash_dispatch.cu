// Precision dispatch of the dslash launcher.
#include "internal.h"

namespace lqcd {
cudaError_t launch_dslash_prec(lqcd_prec prec, const DslashParams &P, int recon, int mode, int nr, cudaStream_t st) {
  switch (prec) {
    case LQCD_F64: return launch_dslash<double>(P, recon, mode, nr, st);
    case LQCD_F32: return launch_dslash<float>(P, recon, mode, nr, st);
    case LQCD_F16: return launch_dslash<__half>(P, recon, mode, nr, st);
    case LQCD_BF16: return launch_dslash<__nv_bfloat16>(P, recon, mode, nr, st);
    case LQCD_DF64: return launch_dslash<df>(P, recon, mode, nr, st);
  }
  return cudaErrorInvalidValue;
}
}  // namespace lqcd
