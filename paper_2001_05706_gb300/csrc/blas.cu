// Fused BLAS-1 kernels of the CG solvers with deterministic FP64 norms.
//
// The paper's QUDA port passes the multi-blas coefficients and kernel
// arguments through device memory (Sec. 2, items 3.4 and 3.5) and notes
// that Thrust reductions in double can be slow (Sec. 3); here the scalar
// state of every right-hand side (gamma, ||q||^2, ...) lives in device
// memory (SolverScalars) and each kernel derives its coefficient from it, so
// a CG iteration needs no host round trip, and every norm is a fixed-order
// tree reduction fused into the kernel that produces the vector.
#include "internal.h"

namespace lqcd {

constexpr int kBlasThreads = 256;

// CG step: alpha = gamma[cur] / qq;  x += alpha p;  r -= alpha q;  rr = ||r||^2
template <typename SX, typename SV>
__global__ void __launch_bounds__(kBlasThreads) cg_xr_kernel(long Vh, MutField x, FieldRef p, MutField r,
                                                             FieldRef q, SolverScalars *sc, int cur, double *partials,
                                                             int nrhs) {
  using TV = typename Math<SV>::T;
  using TX = typename Math<SX>::T;
  const long h = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const int k = blockIdx.y;
  typename RedVal<TV>::type nrm[1] = {0};
  const SolverScalars s = sc[k];
  const bool on = s.active != 0.0 && s.qq > 0.0;
  const double alpha = on ? s.gamma[cur] / s.qq : 0.0;
  if (h < Vh && on) {
    cx<TV> pv[4][3], qv[4][3], rv[4][3];
    cx<TX> xv[4][3];
    load_spinor<SV>(p, Vh, k, h, pv);
    load_spinor<SV>(q, Vh, k, h, qv);
    load_spinor<SV>(r.ref(), Vh, k, h, rv);
    load_spinor<SX>(x.ref(), Vh, k, h, xv);
    const TV a = (TV)alpha;
    const TX ax = (TX)alpha;
#pragma unroll
    for (int sp = 0; sp < 4; sp++)
#pragma unroll
      for (int c = 0; c < 3; c++) {
        xv[sp][c] = mk<TX>(fma(ax, (TX)pv[sp][c].r, xv[sp][c].r), fma(ax, (TX)pv[sp][c].i, xv[sp][c].i));
        rv[sp][c] = mk<TV>(fma(-a, qv[sp][c].r, rv[sp][c].r), fma(-a, qv[sp][c].i, rv[sp][c].i));
      }
    store_spinor<SX>(x.data, x.scale, x.rhs_words, Vh, k, h, xv);
    store_spinor<SV>(r.data, r.scale, r.rhs_words, Vh, k, h, rv);
    nrm[0] = typename RedVal<TV>::type(site_norm2_t<TV>(rv));
  }
  // an inactive right-hand side reduces zeros: its rr reads 0 from then on
  block_partials<1>(nrm, partials, k);
}

// p = s + beta p with beta = gamma[1-cur] / gamma[cur]
template <typename SV>
__global__ void __launch_bounds__(kBlasThreads) cg_p_kernel(long Vh, MutField p, FieldRef sv, SolverScalars *sc,
                                                            int cur) {
  using TV = typename Math<SV>::T;
  const long h = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const int k = blockIdx.y;
  const SolverScalars s = sc[k];
  if (h >= Vh || s.active == 0.0) return;
  const TV beta = s.gamma[cur] > 0.0 ? (TV)(s.gamma[1 - cur] / s.gamma[cur]) : (TV)0;
  cx<TV> pv[4][3], ss[4][3];
  load_spinor<SV>(p.ref(), Vh, k, h, pv);
  load_spinor<SV>(sv, Vh, k, h, ss);
#pragma unroll
  for (int sp = 0; sp < 4; sp++)
#pragma unroll
    for (int c = 0; c < 3; c++) pv[sp][c] = mk<TV>(fma(beta, pv[sp][c].r, ss[sp][c].r), fma(beta, pv[sp][c].i, ss[sp][c].i));
  store_spinor<SV>(p.data, p.scale, p.rhs_words, Vh, k, h, pv);
}

// ||v||^2 per right-hand side into result[k * stride]
template <typename S>
__global__ void __launch_bounds__(kBlasThreads) norm2_kernel(long Vh, FieldRef v, double *partials, int nrhs) {
  using T = typename Math<S>::T;
  const long h = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const int k = blockIdx.y;
  typename RedVal<T>::type nrm[1] = {0};
  if (h < Vh) {
    cx<T> a[4][3];
    load_spinor<S>(v, Vh, k, h, a);
    nrm[0] = typename RedVal<T>::type(site_norm2_t<T>(a));
  }
  block_partials<1>(nrm, partials, k);
}

// y += f_k x  (per right-hand side factor f[k]; arithmetic in the wider of
// the two types: FP32 unless y or x is FP64 or DF64)
template <typename SY, typename SX>
__global__ void __launch_bounds__(kBlasThreads) axpy_kernel(long Vh, MutField y, FieldRef x, const double *f) {
  using TY = typename Math<SY>::T;
  using TX = typename Math<SX>::T;
  using W = typename Wide<TY, TX>::type;
  const long h = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const int k = blockIdx.y;
  if (h >= Vh) return;
  const double a = f[k];
  if (a == 0.0) return;
  const W aw = (W)a;
  cx<TY> yv[4][3];
  cx<TX> xv[4][3];
  load_spinor<SY>(y.ref(), Vh, k, h, yv);
  load_spinor<SX>(x, Vh, k, h, xv);
#pragma unroll
  for (int sp = 0; sp < 4; sp++)
#pragma unroll
    for (int c = 0; c < 3; c++)
      yv[sp][c] = mk<TY>((TY)fma(aw, (W)xv[sp][c].r, (W)yv[sp][c].r), (TY)fma(aw, (W)xv[sp][c].i, (W)yv[sp][c].i));
  store_spinor<SY>(y.data, y.scale, y.rhs_words, Vh, k, h, yv);
}

// y = f_k x with per-RHS factors (precision conversion included; arithmetic
// in the wider of the two types)
template <typename SY, typename SX>
__global__ void __launch_bounds__(kBlasThreads) scale_kernel(long Vh, MutField y, FieldRef x, const double *f) {
  using TY = typename Math<SY>::T;
  using TX = typename Math<SX>::T;
  using W = typename Wide<TY, TX>::type;
  const long h = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const int k = blockIdx.y;
  if (h >= Vh) return;
  const double a = f[k];
  cx<TX> xv[4][3];
  cx<TY> yv[4][3];
  load_spinor<SX>(x, Vh, k, h, xv);
#pragma unroll
  for (int sp = 0; sp < 4; sp++)
#pragma unroll
    for (int c = 0; c < 3; c++) yv[sp][c] = mk<TY>((TY)((W)a * (W)xv[sp][c].r), (TY)((W)a * (W)xv[sp][c].i));
  store_spinor<SY>(y.data, y.scale, y.rhs_words, Vh, k, h, yv);
}

static dim3 bgrid(long Vh, int nrhs) { return dim3((unsigned)((Vh + kBlasThreads - 1) / kBlasThreads), (unsigned)nrhs); }

// one block per quantity: thread t adds partials t, t + 256, ... into eight
// accumulators (independent loads in flight), then the fixed tree
constexpr int kFinishThreads = 256;
__global__ void __launch_bounds__(kFinishThreads) finish_reduce_kernel(const double *partials, int nblk,
                                                                        double *result, int rstride) {
  const int k = blockIdx.x, t = threadIdx.x;
  const double *p = partials + (long)k * nblk;
  double a[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  int b = t;
  for (; b + 7 * kFinishThreads < nblk; b += 8 * kFinishThreads) {
#pragma unroll
    for (int u = 0; u < 8; u++) a[u] += __ldcg(p + b + u * kFinishThreads);
  }
#pragma unroll
  for (int u = 0; u < 8; u++)
    if (b + u * kFinishThreads < nblk) a[u] += __ldcg(p + b + u * kFinishThreads);
  double v[1] = {((a[0] + a[1]) + (a[2] + a[3])) + ((a[4] + a[5]) + (a[6] + a[7]))};
  __shared__ double sh[kFinishThreads / 32];
  v[0] = warp_sum(v[0]);
  if ((t & 31) == 0) sh[t >> 5] = v[0];
  __syncthreads();
  if (t == 0) {
    double s = 0.0;
#pragma unroll
    for (int w = 0; w < kFinishThreads / 32; w++) s += sh[w];
    result[(long)k * rstride] = s;
  }
}

cudaError_t finish_reduce(const double *partials, int nblk, int nk, double *result, int rstride, cudaStream_t st) {
  finish_reduce_kernel<<<nk, kFinishThreads, 0, st>>>(partials, nblk, result, rstride);
  return cudaGetLastError();
}

long blas_blocks(long Vh) { return (Vh + kBlasThreads - 1) / kBlasThreads; }

#define LQ_DISPATCH_V(prec, CALL)                                  \
  switch (prec) {                                                  \
    case LQCD_F64: { using SV = double; CALL; } break;             \
    case LQCD_F32: { using SV = float; CALL; } break;              \
    case LQCD_F16: { using SV = __half; CALL; } break;             \
    case LQCD_BF16: { using SV = __nv_bfloat16; CALL; } break;     \
    case LQCD_DF64: { using SV = df; CALL; } break;                \
  }

cudaError_t blas_cg_xr(lqcd_prec px, lqcd_prec pv, long Vh, int nrhs, MutField x, FieldRef p, MutField r, FieldRef q,
                       SolverScalars *sc, int cur, double *partials, cudaStream_t st) {
  dim3 g = bgrid(Vh, nrhs);
  if (px == LQCD_F64 && pv == LQCD_F64) {
    cg_xr_kernel<double, double><<<g, kBlasThreads, 0, st>>>(Vh, x, p, r, q, sc, cur, partials, nrhs);
  } else if (px == LQCD_DF64 && pv == LQCD_DF64) {
    cg_xr_kernel<df, df><<<g, kBlasThreads, 0, st>>>(Vh, x, p, r, q, sc, cur, partials, nrhs);
  } else if (px == LQCD_F32) {
    LQ_DISPATCH_V(pv, (cg_xr_kernel<float, SV><<<g, kBlasThreads, 0, st>>>(Vh, x, p, r, q, sc, cur, partials, nrhs)));
  } else {
    return cudaErrorInvalidValue;
  }
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return finish_reduce(partials, (int)g.x, nrhs, &sc[0].rr, (int)(sizeof(SolverScalars) / 8), st);
}

cudaError_t blas_cg_p(lqcd_prec pv, long Vh, int nrhs, MutField p, FieldRef s, SolverScalars *sc, int cur,
                      cudaStream_t st) {
  dim3 g = bgrid(Vh, nrhs);
  LQ_DISPATCH_V(pv, (cg_p_kernel<SV><<<g, kBlasThreads, 0, st>>>(Vh, p, s, sc, cur)));
  return cudaGetLastError();
}

cudaError_t blas_norm2(lqcd_prec pv, long Vh, int nrhs, FieldRef v, double *partials, double *result, int stride,
                       cudaStream_t st) {
  dim3 g = bgrid(Vh, nrhs);
  LQ_DISPATCH_V(pv, (norm2_kernel<SV><<<g, kBlasThreads, 0, st>>>(Vh, v, partials, nrhs)));
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return finish_reduce(partials, (int)g.x, nrhs, result, stride, st);
}

cudaError_t blas_axpy(lqcd_prec py, lqcd_prec px, long Vh, int nrhs, MutField y, FieldRef x, const double *f,
                      cudaStream_t st) {
  dim3 g = bgrid(Vh, nrhs);
  if (py == LQCD_F64) {
    LQ_DISPATCH_V(px, (axpy_kernel<double, SV><<<g, kBlasThreads, 0, st>>>(Vh, y, x, f)));
  } else if (py == LQCD_DF64) {
    LQ_DISPATCH_V(px, (axpy_kernel<df, SV><<<g, kBlasThreads, 0, st>>>(Vh, y, x, f)));
  } else if (py == LQCD_F32) {
    LQ_DISPATCH_V(px, (axpy_kernel<float, SV><<<g, kBlasThreads, 0, st>>>(Vh, y, x, f)));
  } else if (py == LQCD_F16 && px == LQCD_F16) {
    axpy_kernel<__half, __half><<<g, kBlasThreads, 0, st>>>(Vh, y, x, f);
  } else if (py == LQCD_BF16 && px == LQCD_BF16) {
    axpy_kernel<__nv_bfloat16, __nv_bfloat16><<<g, kBlasThreads, 0, st>>>(Vh, y, x, f);
  } else {
    return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t blas_scale(lqcd_prec py, lqcd_prec px, long Vh, int nrhs, MutField y, FieldRef x, const double *f,
                       cudaStream_t st) {
  dim3 g = bgrid(Vh, nrhs);
  switch (py) {
    case LQCD_F64: LQ_DISPATCH_V(px, (scale_kernel<double, SV><<<g, kBlasThreads, 0, st>>>(Vh, y, x, f))); break;
    case LQCD_F32: LQ_DISPATCH_V(px, (scale_kernel<float, SV><<<g, kBlasThreads, 0, st>>>(Vh, y, x, f))); break;
    case LQCD_F16: LQ_DISPATCH_V(px, (scale_kernel<__half, SV><<<g, kBlasThreads, 0, st>>>(Vh, y, x, f))); break;
    case LQCD_BF16:
      LQ_DISPATCH_V(px, (scale_kernel<__nv_bfloat16, SV><<<g, kBlasThreads, 0, st>>>(Vh, y, x, f)));
      break;
    case LQCD_DF64: LQ_DISPATCH_V(px, (scale_kernel<df, SV><<<g, kBlasThreads, 0, st>>>(Vh, y, x, f))); break;
  }
  return cudaGetLastError();
}

}  // namespace lqcd
