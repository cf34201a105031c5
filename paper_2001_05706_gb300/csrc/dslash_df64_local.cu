// dslash kernel instantiations for double-float (DF64) storage, the modes
// with a local term (K2b, the full-lattice M and H_W, the Chebyshev step).
#include "dslash_inst.cuh"

namespace lqcd {
cudaError_t launch_df64_local(const DslashParams &P, int mode, int nr, cudaStream_t st) {
  switch (mode) {
    case MODE_LOCAL_IDENT: return launch_nr<df, 18, MODE_LOCAL_IDENT>(P, nr, st);
    case MODE_LOCAL_A: return launch_nr<df, 18, MODE_LOCAL_A>(P, nr, st);
    case MODE_CHEB: return launch_nr<df, 18, MODE_CHEB>(P, nr, st);
  }
  return cudaErrorInvalidValue;
}
}  // namespace lqcd
