// Launch-shape selection for the dslash kernel; included once per storage
// type by dslash_f64.cu, dslash_f32.cu, dslash_f16.cu and dslash_bf16.cu so
// the instantiations compile in parallel.
#pragma once
#include <type_traits>

#include "dslash.cuh"

namespace lqcd {

template <typename S, int R, int MODE, int NR>
static cudaError_t launch_one(const DslashParams &P, cudaStream_t st) {
  constexpr int T = LaunchCfg<S, NR, MODE>::threads;
  dim3 grid((unsigned)((P.h1 - P.h0 + T - 1) / T), (unsigned)(P.nrhs / NR));
  dslash_kernel<S, R, MODE, NR><<<grid, T, 0, st>>>(P);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || !P.norm_partials) return e;
  return finish_reduce(P.norm_partials, (int)grid.x, P.nrhs, P.norm_result, P.norm_stride, st);
}

template <typename S, int R, int MODE>
static cudaError_t launch_nr(const DslashParams &P, int nr, cudaStream_t st) {
  if (nr == 1) return launch_one<S, R, MODE, 1>(P, st);
  if constexpr (R == 8) return cudaErrorInvalidValue;  // the 8-real form: one right-hand side per thread
  if constexpr (R != 8 && MODE != MODE_FOLDED_AINV) {
    if (nr == 2) return launch_one<S, R, MODE, 2>(P, st);
    // double-float accumulators for four right-hand sides exceed the register file
    if constexpr (!std::is_same<S, df>::value)
      if (nr == 4) return launch_one<S, R, MODE, 4>(P, st);
  }
  return cudaErrorInvalidValue;
}

template <typename S, int R>
static cudaError_t launch_mode(const DslashParams &P, int mode, int nr, cudaStream_t st) {
  switch (mode) {
    case MODE_HOP: return launch_nr<S, R, MODE_HOP>(P, nr, st);
    case MODE_HOP_AINV: return launch_nr<S, R, MODE_HOP_AINV>(P, nr, st);
    case MODE_LOCAL_IDENT: return launch_nr<S, R, MODE_LOCAL_IDENT>(P, nr, st);
    case MODE_LOCAL_A: return launch_nr<S, R, MODE_LOCAL_A>(P, nr, st);
    case MODE_FOLDED_AINV: return launch_nr<S, R, MODE_FOLDED_AINV>(P, nr, st);
    case MODE_CHEB:
      // the Chebyshev step runs in the overlap's FP64, DF64 and FP32 sign functions only
      if constexpr (std::is_same<S, double>::value || std::is_same<S, float>::value || std::is_same<S, df>::value)
        return launch_nr<S, R, MODE_CHEB>(P, nr, st);
      break;
  }
  return cudaErrorInvalidValue;
}

template <typename S, bool WITH18, bool WITH12 = true, bool WITH8 = false>
static cudaError_t launch_dslash_impl(const DslashParams &P, int recon, int mode, int nr, cudaStream_t st) {
  if (P.nrhs % nr != 0) return cudaErrorInvalidValue;
  if constexpr (WITH8) {
    if (recon == 8) return launch_mode<S, 8>(P, mode, nr, st);
  }
  if constexpr (WITH12) {
    if (recon == 12) return launch_mode<S, 12>(P, mode, nr, st);
  }
  if constexpr (WITH18) {
    if (recon == 18) return launch_mode<S, 18>(P, mode, nr, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace lqcd
