// Precision dispatch of the dslash launcher.
#include "dslash_mrhs.cuh"
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

cudaError_t launch_dslash_mrhs_prec(lqcd_prec prec, const DslashParams &P, int recon, int mode, int g, cudaStream_t st) {
  switch (prec) {
    case LQCD_F32: return launch_dslash_mrhs<float>(P, recon, mode, g, st);
    case LQCD_F16: return launch_dslash_mrhs<__half>(P, recon, mode, g, st);
    case LQCD_BF16: return launch_dslash_mrhs<__nv_bfloat16>(P, recon, mode, g, st);
    default: break;
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_dslash_variant(lqcd_prec prec, const DslashParams &P, int recon, int mode, int variant,
                                  cudaStream_t st) {
  if (variant > kMrhsVariant) return launch_dslash_mrhs_prec(prec, P, recon, mode, variant - kMrhsVariant, st);
  return launch_dslash_prec(prec, P, recon, mode, variant, st);
}
}  // namespace lqcd
