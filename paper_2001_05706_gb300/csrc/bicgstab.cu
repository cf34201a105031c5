// Building blocks of BiCGStab (van der Vorst, SIAM J. Sci. Stat. Comput. 13,
// 631 (1992)) on the even-odd operator Mhat, one independent recursion per
// right-hand side:
//   rho = (rhat, r); beta = (rho / rho_old)(alpha / omega); p = r + beta (p - omega v)
//   v = Mhat p; alpha = rho / (rhat, v); s = r - alpha v
//   t = Mhat s; omega = (t, s) / (t, t); x += alpha p + omega s; r = s - omega t
// The complex scalars of every right-hand side live in device memory
// (BiScalars) and are advanced by one-thread-per-RHS kernels between the
// vector kernels, so an iteration needs no host round trip; the inner
// products are deterministic fixed-tree reductions fused into the kernels
// that read the vectors.  Vector arithmetic is in the storage's arithmetic
// type (FP32 for FP32/FP16/BF16, double-float for DF64, FP64 for FP64).
#include "internal.h"

namespace lqcd {

namespace {

constexpr int kBiThreads = 256;

__device__ __forceinline__ double2 zmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 zdiv(double2 a, double2 b) {
  const double d = b.x * b.x + b.y * b.y;
  return make_double2((a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d);
}
template <typename T> __device__ __forceinline__ cx<T> zc(double2 z) { return mk<T>((T)z.x, (T)z.y); }

// conj(a) . b and |a|^2 of one site in the arithmetic type, returned as
// reduction values (double for FP64, double-float otherwise)
template <typename T>
__device__ __forceinline__ void site_dot3(const cx<T> (&a)[4][3], const cx<T> (&b)[4][3],
                                          typename RedVal<T>::type (&o)[3]) {
  using RT = typename RedVal<T>::type;
  T re = (T)0, im = (T)0, nn = (T)0;
#pragma unroll
  for (int sp = 0; sp < 4; sp++)
#pragma unroll
    for (int c = 0; c < 3; c++) {
      re = fma(a[sp][c].r, b[sp][c].r, fma(a[sp][c].i, b[sp][c].i, re));
      im = fma(a[sp][c].r, b[sp][c].i, fma(-a[sp][c].i, b[sp][c].r, im));
      nn = fma(a[sp][c].r, a[sp][c].r, fma(a[sp][c].i, a[sp][c].i, nn));
    }
  o[0] = RT(re);
  o[1] = RT(im);
  o[2] = RT(nn);
}

__global__ void bi_scalar_kernel(int which, BiScalars *s, const double *red, int n) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n || s[k].active == 0.0) return;
  BiScalars q = s[k];
  const double *r = red + 3 * k;
  if (which == BI_BETA) {  // red: (rhat, r), |r|^2 of the last update of r
    q.rho = make_double2(r[0], r[1]);
    q.rr = r[2];
    q.beta = zmul(zdiv(q.rho, q.rho_old), zdiv(q.alpha, q.omega));
    q.rho_old = q.rho;
  } else if (which == BI_ALPHA) {  // red: (rhat, v)
    q.alpha = zdiv(q.rho, make_double2(r[0], r[1]));
  } else {  // red: (t, s), |t|^2
    q.omega = r[2] > 0.0 ? make_double2(r[0] / r[2], r[1] / r[2]) : make_double2(0.0, 0.0);
  }
  s[k] = q;
}

// p = r + beta (p - omega v)
template <typename S>
__global__ void __launch_bounds__(kBiThreads) bi_p_kernel(long Vh, MutField p, FieldRef r, FieldRef v,
                                                          const BiScalars *s) {
  using T = typename Math<S>::T;
  const long h = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const int k = blockIdx.y;
  if (h >= Vh || s[k].active == 0.0) return;
  const cx<T> beta = zc<T>(s[k].beta), om = zc<T>(s[k].omega);
  const cx<T> mom = mk<T>(-om.r, -om.i);
  cx<T> pv[4][3], rv[4][3], vv[4][3];
  load_spinor<S>(p.ref(), Vh, k, h, pv);
  load_spinor<S>(r, Vh, k, h, rv);
  load_spinor<S>(v, Vh, k, h, vv);
#pragma unroll
  for (int sp = 0; sp < 4; sp++)
#pragma unroll
    for (int c = 0; c < 3; c++) pv[sp][c] = cmadd(beta, cmadd(mom, vv[sp][c], pv[sp][c]), rv[sp][c]);
  store_spinor<S>(p.data, p.scale, p.rhs_words, Vh, k, h, pv);
}

// s = r - alpha v
template <typename S>
__global__ void __launch_bounds__(kBiThreads) bi_s_kernel(long Vh, MutField sv, FieldRef r, FieldRef v,
                                                          const BiScalars *s) {
  using T = typename Math<S>::T;
  const long h = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const int k = blockIdx.y;
  if (h >= Vh || s[k].active == 0.0) return;
  const cx<T> al = zc<T>(s[k].alpha);
  const cx<T> mal = mk<T>(-al.r, -al.i);
  cx<T> rv[4][3], vv[4][3];
  load_spinor<S>(r, Vh, k, h, rv);
  load_spinor<S>(v, Vh, k, h, vv);
#pragma unroll
  for (int sp = 0; sp < 4; sp++)
#pragma unroll
    for (int c = 0; c < 3; c++) rv[sp][c] = cmadd(mal, vv[sp][c], rv[sp][c]);
  store_spinor<S>(sv.data, sv.scale, sv.rhs_words, Vh, k, h, rv);
}

// red[3k..] = (a, b), |a|^2 over the sites of RHS k
template <typename S>
__global__ void __launch_bounds__(kBiThreads) bi_dot3_kernel(long Vh, FieldRef a, FieldRef b, double *partials) {
  using T = typename Math<S>::T;
  const long h = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const int k = blockIdx.y;
  using RT = typename RedVal<T>::type;
  RT o[3] = {RT(0), RT(0), RT(0)};
  if (h < Vh) {
    cx<T> av[4][3], bv[4][3];
    load_spinor<S>(a, Vh, k, h, av);
    load_spinor<S>(b, Vh, k, h, bv);
    site_dot3<T>(av, bv, o);
  }
  block_partials<3>(o, partials, 3 * k);
}

// x += alpha p + omega s; r = s - omega t; red = (rhat, r) and |r|^2
template <typename SX, typename S>
__global__ void __launch_bounds__(kBiThreads) bi_xr_kernel(long Vh, MutField x, FieldRef p, FieldRef sv, FieldRef t,
                                                           MutField r, FieldRef rhat, const BiScalars *s,
                                                           double *partials) {
  using T = typename Math<S>::T;
  using TX = typename Math<SX>::T;
  const long h = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const int k = blockIdx.y;
  using RT = typename RedVal<T>::type;
  RT o[3] = {RT(0), RT(0), RT(0)};
  if (h < Vh && s[k].active != 0.0) {
    const cx<TX> al = zc<TX>(s[k].alpha), om = zc<TX>(s[k].omega);
    const cx<T> omt = zc<T>(s[k].omega);
    const cx<T> mom = mk<T>(-omt.r, -omt.i);
    cx<T> pv[4][3], ss[4][3], tv[4][3], rh[4][3];
    cx<TX> xv[4][3];
    load_spinor<SX>(x.ref(), Vh, k, h, xv);
    load_spinor<S>(p, Vh, k, h, pv);
    load_spinor<S>(sv, Vh, k, h, ss);
#pragma unroll
    for (int sp = 0; sp < 4; sp++)
#pragma unroll
      for (int c = 0; c < 3; c++) {
        const cx<TX> pw = mk<TX>((TX)pv[sp][c].r, (TX)pv[sp][c].i);
        const cx<TX> sw = mk<TX>((TX)ss[sp][c].r, (TX)ss[sp][c].i);
        xv[sp][c] = cmadd(om, sw, cmadd(al, pw, xv[sp][c]));
      }
    store_spinor<SX>(x.data, x.scale, x.rhs_words, Vh, k, h, xv);
    load_spinor<S>(t, Vh, k, h, tv);
#pragma unroll
    for (int sp = 0; sp < 4; sp++)
#pragma unroll
      for (int c = 0; c < 3; c++) ss[sp][c] = cmadd(mom, tv[sp][c], ss[sp][c]);
    store_spinor<S>(r.data, r.scale, r.rhs_words, Vh, k, h, ss);
    // (rhat, r) and |r|^2 from the values in registers: r must not be read back
    // through the read-only path in the kernel that writes it
    load_spinor<S>(rhat, Vh, k, h, rh);
    RT d[3], n2[3];
    site_dot3<T>(rh, ss, d);
    site_dot3<T>(ss, ss, n2);
    o[0] = d[0];
    o[1] = d[1];
    o[2] = n2[2];
  }
  block_partials<3>(o, partials, 3 * k);
}

dim3 bgrid(long Vh, int nrhs) { return dim3((unsigned)((Vh + kBiThreads - 1) / kBiThreads), (unsigned)nrhs); }

#define LQ_BI_DISPATCH(prec, CALL)                                 \
  switch (prec) {                                                  \
    case LQCD_F64: { using SV = double; CALL; } break;             \
    case LQCD_F32: { using SV = float; CALL; } break;              \
    case LQCD_F16: { using SV = __half; CALL; } break;             \
    case LQCD_BF16: { using SV = __nv_bfloat16; CALL; } break;     \
    case LQCD_DF64: { using SV = df; CALL; } break;                \
  }

}  // namespace

cudaError_t bi_scalar(int which, BiScalars *s, const double *red, int nrhs, cudaStream_t st) {
  bi_scalar_kernel<<<1, 64, 0, st>>>(which, s, red, nrhs);
  return cudaGetLastError();
}

cudaError_t bi_p(lqcd_prec pv, long Vh, int nrhs, MutField p, FieldRef r, FieldRef v, const BiScalars *s,
                 cudaStream_t st) {
  LQ_BI_DISPATCH(pv, (bi_p_kernel<SV><<<bgrid(Vh, nrhs), kBiThreads, 0, st>>>(Vh, p, r, v, s)));
  return cudaGetLastError();
}

cudaError_t bi_s(lqcd_prec pv, long Vh, int nrhs, MutField sv, FieldRef r, FieldRef v, const BiScalars *s,
                 cudaStream_t st) {
  LQ_BI_DISPATCH(pv, (bi_s_kernel<SV><<<bgrid(Vh, nrhs), kBiThreads, 0, st>>>(Vh, sv, r, v, s)));
  return cudaGetLastError();
}

// GCR: y_k += c_k x_k with a complex coefficient per right-hand side (c_k =
// 0: right-hand side k untouched); y may be a wider type than x
template <typename SY, typename SX>
__global__ void __launch_bounds__(kBiThreads) gcr_caxpy_kernel(long Vh, MutField y, FieldRef x, const double2 *cf) {
  using T = typename Math<SY>::T;
  using TX = typename Math<SX>::T;
  const long h = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const int k = blockIdx.y;
  if (h >= Vh || (cf[k].x == 0.0 && cf[k].y == 0.0)) return;
  const cx<T> a = zc<T>(cf[k]);
  cx<T> yv[4][3];
  cx<TX> xv[4][3];
  const FieldRef yr{y.data, y.scale, y.rhs_words};
  load_spinor<SY>(yr, Vh, k, h, yv);
  load_spinor<SX>(x, Vh, k, h, xv);
#pragma unroll
  for (int sp = 0; sp < 4; sp++)
#pragma unroll
    for (int c = 0; c < 3; c++) yv[sp][c] = cmadd(a, mk<T>((T)xv[sp][c].r, (T)xv[sp][c].i), yv[sp][c]);
  store_spinor<SY>(y.data, y.scale, y.rhs_words, Vh, k, h, yv);
}

cudaError_t gcr_caxpy(lqcd_prec py, lqcd_prec px, long Vh, int nrhs, MutField y, FieldRef x, const double2 *cf,
                      cudaStream_t st) {
  const dim3 g = bgrid(Vh, nrhs);
  if (py == px) {
    LQ_BI_DISPATCH(py, (gcr_caxpy_kernel<SV, SV><<<g, kBiThreads, 0, st>>>(Vh, y, x, cf)));
  } else if (py == LQCD_F32 && (px == LQCD_F16 || px == LQCD_BF16)) {
    if (px == LQCD_F16)
      gcr_caxpy_kernel<float, __half><<<g, kBiThreads, 0, st>>>(Vh, y, x, cf);
    else
      gcr_caxpy_kernel<float, __nv_bfloat16><<<g, kBiThreads, 0, st>>>(Vh, y, x, cf);
  } else {
    return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t bi_dot3(lqcd_prec pv, long Vh, int nrhs, FieldRef a, FieldRef b, double *partials, double *red,
                    cudaStream_t st) {
  const dim3 g = bgrid(Vh, nrhs);
  LQ_BI_DISPATCH(pv, (bi_dot3_kernel<SV><<<g, kBiThreads, 0, st>>>(Vh, a, b, partials)));
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return finish_reduce(partials, (int)g.x, 3 * nrhs, red, 1, st);
}

cudaError_t bi_xr(lqcd_prec px, lqcd_prec pv, long Vh, int nrhs, MutField x, FieldRef p, FieldRef sv, FieldRef t,
                  MutField r, FieldRef rhat, const BiScalars *s, double *partials, double *red, cudaStream_t st) {
  const dim3 g = bgrid(Vh, nrhs);
  if (px == pv && (pv == LQCD_F64 || pv == LQCD_DF64)) {
    if (pv == LQCD_F64)
      bi_xr_kernel<double, double><<<g, kBiThreads, 0, st>>>(Vh, x, p, sv, t, r, rhat, s, partials);
    else
      bi_xr_kernel<df, df><<<g, kBiThreads, 0, st>>>(Vh, x, p, sv, t, r, rhat, s, partials);
  } else if (px == LQCD_F32 && pv != LQCD_F64 && pv != LQCD_DF64) {
    switch (pv) {
      case LQCD_F32:
        bi_xr_kernel<float, float><<<g, kBiThreads, 0, st>>>(Vh, x, p, sv, t, r, rhat, s, partials);
        break;
      case LQCD_F16:
        bi_xr_kernel<float, __half><<<g, kBiThreads, 0, st>>>(Vh, x, p, sv, t, r, rhat, s, partials);
        break;
      default:
        bi_xr_kernel<float, __nv_bfloat16><<<g, kBiThreads, 0, st>>>(Vh, x, p, sv, t, r, rhat, s, partials);
        break;
    }
  } else {
    return cudaErrorInvalidValue;
  }
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return finish_reduce(partials, (int)g.x, 3 * nrhs, red, 1, st);
}

}  // namespace lqcd
