#include <cstring>
#include <algorithm>
// Field layout conversions: canonical FP64 arrays <-> site-blocked
// word-major fields of one parity in FP64/FP32/FP16/BF16, link packing into
// the 18- and 12-real forms, clover packing, precision conversion, and the
// unitarity check of loaded links.
#include "internal.h"

namespace lqcd {

// lexicographic index of the site with half index h in parity p
__device__ __forceinline__ long lex_of(const Geom &g, long h, int p) {
  Coords c = site_coords(g, h, p);
  return c.x[0] + (long)g.L[0] * (c.x[1] + (long)g.L[1] * (c.x[2] + (long)g.L[2] * c.x[3]));
}

// ---------------------------------------------------------------------------
// spinors
// ---------------------------------------------------------------------------
template <typename S>
__global__ void pack_spinor_kernel(Geom g, int p, const double *__restrict__ canon, long V, void *out, float *scale,
                                   long rhs_words, long h0, long h1) {
  const long h = h0 + (long)blockIdx.x * blockDim.x + threadIdx.x;
  const int r = blockIdx.y;
  if (h >= h1) return;
  const long s = lex_of(g, h, p);
  const double2 *src = reinterpret_cast<const double2 *>(canon + ((long)r * V + s) * 24);
  using T = typename Math<S>::T;
  cx<T> psi[4][3];
#pragma unroll
  for (int k = 0; k < 12; k++) {
    double2 v = src[k];
    psi[k / 3][k % 3] = mk<T>((T)v.x, (T)v.y);
  }
  store_spinor<S>(out, scale, rhs_words, g.Vh, r, h, psi);
}

template <typename S>
__global__ void unpack_spinor_kernel(Geom g, int p, const void *in, const float *scale, long rhs_words,
                                     double *__restrict__ canon, long V, long h0, long h1) {
  const long h = h0 + (long)blockIdx.x * blockDim.x + threadIdx.x;
  const int r = blockIdx.y;
  if (h >= h1) return;
  const long s = lex_of(g, h, p);
  FieldRef f{in, scale, rhs_words};
  using T = typename Math<S>::T;
  cx<T> psi[4][3];
  load_spinor<S>(f, g.Vh, r, h, psi);
  double2 *dst = reinterpret_cast<double2 *>(canon + ((long)r * V + s) * 24);
#pragma unroll
  for (int k = 0; k < 12; k++) dst[k] = make_double2((double)psi[k / 3][k % 3].r, (double)psi[k / 3][k % 3].i);
}

// zero the sites of parity p in a canonical array (nrhs fields)
__global__ void zero_parity_kernel(Geom g, int p, double *canon, long V, long h0, long h1) {
  const long h = h0 + (long)blockIdx.x * blockDim.x + threadIdx.x;
  const int r = blockIdx.y;
  if (h >= h1) return;
  const long s = lex_of(g, h, p);
  double2 *dst = reinterpret_cast<double2 *>(canon + ((long)r * V + s) * 24);
#pragma unroll
  for (int k = 0; k < 12; k++) dst[k] = make_double2(0.0, 0.0);
}

template <typename SI, typename SO>
__global__ void convert_spinor_kernel(long Vh, const void *in, const float *in_scale, long in_rhs_words, void *out,
                                      float *out_scale, long out_rhs_words, double factor) {
  const long h = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const int r = blockIdx.y;
  if (h >= Vh) return;
  FieldRef f{in, in_scale, in_rhs_words};
  using TI = typename Math<SI>::T;
  using TO = typename Math<SO>::T;
  cx<TI> a[4][3];
  load_spinor<SI>(f, Vh, r, h, a);
  cx<TO> b[4][3];
#pragma unroll
  for (int s = 0; s < 4; s++)
#pragma unroll
    for (int c = 0; c < 3; c++) b[s][c] = mk<TO>((TO)(factor * (double)a[s][c].r), (TO)(factor * (double)a[s][c].i));
  store_spinor<SO>(out, out_scale, out_rhs_words, Vh, r, h, b);
}

static dim3 grid2(long n, int y, int t) { return dim3((unsigned)((n + t - 1) / t), (unsigned)y); }

template <typename S>
static cudaError_t pack_spinor_t(const Geom &g, int p, const double *canon, int nrhs, void *out, float *scale,
                                 long rhs_words, cudaStream_t st, long h0, long h1) {
  long V = 2 * g.Vh;
  pack_spinor_kernel<S><<<grid2(h1 - h0, nrhs, 128), 128, 0, st>>>(g, p, canon, V, out, scale, rhs_words, h0, h1);
  return cudaGetLastError();
}
template <typename S>
static cudaError_t unpack_spinor_t(const Geom &g, int p, const void *in, const float *scale, long rhs_words,
                                   int nrhs, double *canon, cudaStream_t st, long h0, long h1) {
  long V = 2 * g.Vh;
  unpack_spinor_kernel<S><<<grid2(h1 - h0, nrhs, 128), 128, 0, st>>>(g, p, in, scale, rhs_words, canon, V, h0, h1);
  return cudaGetLastError();
}

static bool bad_range(const Geom &g, long &h0, long &h1) {
  if (h1 < 0) h1 = g.Vh;
  return h0 < 0 || h1 > g.Vh || h0 >= h1;
}

cudaError_t pack_spinor(lqcd_prec prec, const Geom &g, int p, const double *canon, int nrhs, void *out, float *scale,
                        long rhs_words, cudaStream_t st, long h0, long h1) {
  if (bad_range(g, h0, h1)) return cudaErrorInvalidValue;
  switch (prec) {
    case LQCD_F64: return pack_spinor_t<double>(g, p, canon, nrhs, out, scale, rhs_words, st, h0, h1);
    case LQCD_F32: return pack_spinor_t<float>(g, p, canon, nrhs, out, scale, rhs_words, st, h0, h1);
    case LQCD_F16: return pack_spinor_t<__half>(g, p, canon, nrhs, out, scale, rhs_words, st, h0, h1);
    case LQCD_BF16: return pack_spinor_t<__nv_bfloat16>(g, p, canon, nrhs, out, scale, rhs_words, st, h0, h1);
    case LQCD_DF64: return pack_spinor_t<df>(g, p, canon, nrhs, out, scale, rhs_words, st, h0, h1);
  }
  return cudaErrorInvalidValue;
}

cudaError_t unpack_spinor(lqcd_prec prec, const Geom &g, int p, const void *in, const float *scale, long rhs_words,
                          int nrhs, double *canon, cudaStream_t st, long h0, long h1) {
  if (bad_range(g, h0, h1)) return cudaErrorInvalidValue;
  switch (prec) {
    case LQCD_F64: return unpack_spinor_t<double>(g, p, in, scale, rhs_words, nrhs, canon, st, h0, h1);
    case LQCD_F32: return unpack_spinor_t<float>(g, p, in, scale, rhs_words, nrhs, canon, st, h0, h1);
    case LQCD_F16: return unpack_spinor_t<__half>(g, p, in, scale, rhs_words, nrhs, canon, st, h0, h1);
    case LQCD_BF16: return unpack_spinor_t<__nv_bfloat16>(g, p, in, scale, rhs_words, nrhs, canon, st, h0, h1);
    case LQCD_DF64: return unpack_spinor_t<df>(g, p, in, scale, rhs_words, nrhs, canon, st, h0, h1);
  }
  return cudaErrorInvalidValue;
}

cudaError_t zero_parity(const Geom &g, int p, double *canon, int nrhs, cudaStream_t st, long h0, long h1) {
  if (bad_range(g, h0, h1)) return cudaErrorInvalidValue;
  zero_parity_kernel<<<grid2(h1 - h0, nrhs, 128), 128, 0, st>>>(g, p, canon, 2 * g.Vh, h0, h1);
  return cudaGetLastError();
}

template <typename SI>
static cudaError_t convert_from(lqcd_prec po, long Vh, int nrhs, const void *in, const float *is, long irw, void *out,
                                float *os, long orw, double f, cudaStream_t st) {
  dim3 gr = grid2(Vh, nrhs, 128);
  switch (po) {
    case LQCD_F64: convert_spinor_kernel<SI, double><<<gr, 128, 0, st>>>(Vh, in, is, irw, out, os, orw, f); break;
    case LQCD_F32: convert_spinor_kernel<SI, float><<<gr, 128, 0, st>>>(Vh, in, is, irw, out, os, orw, f); break;
    case LQCD_F16: convert_spinor_kernel<SI, __half><<<gr, 128, 0, st>>>(Vh, in, is, irw, out, os, orw, f); break;
    case LQCD_BF16:
      convert_spinor_kernel<SI, __nv_bfloat16><<<gr, 128, 0, st>>>(Vh, in, is, irw, out, os, orw, f);
      break;
    case LQCD_DF64: convert_spinor_kernel<SI, df><<<gr, 128, 0, st>>>(Vh, in, is, irw, out, os, orw, f); break;
  }
  return cudaGetLastError();
}

cudaError_t convert_spinor(lqcd_prec pi, lqcd_prec po, long Vh, int nrhs, const void *in, const float *is, long irw,
                           void *out, float *os, long orw, double factor, cudaStream_t st) {
  switch (pi) {
    case LQCD_F64: return convert_from<double>(po, Vh, nrhs, in, is, irw, out, os, orw, factor, st);
    case LQCD_F32: return convert_from<float>(po, Vh, nrhs, in, is, irw, out, os, orw, factor, st);
    case LQCD_F16: return convert_from<__half>(po, Vh, nrhs, in, is, irw, out, os, orw, factor, st);
    case LQCD_BF16: return convert_from<__nv_bfloat16>(po, Vh, nrhs, in, is, irw, out, os, orw, factor, st);
    case LQCD_DF64: return convert_from<df>(po, Vh, nrhs, in, is, irw, out, os, orw, factor, st);
  }
  return cudaErrorInvalidValue;
}

// ---------------------------------------------------------------------------
// links
// ---------------------------------------------------------------------------
template <typename S, int R>
__global__ void pack_links_kernel(Geom g, const double *__restrict__ U, void *out) {
  const long h = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const int mu = blockIdx.y & 3, p = blockIdx.y >> 2;
  if (h >= g.Vh) return;
  const long s = lex_of(g, h, p);
  const double *u = U + (s * 4 + mu) * 18;
  S raw[R];
  if constexpr (R == 8) {  // (arg U00, arg U20, U01, U02, U10)
    const double p8[8] = {atan2(u[1], u[0]), atan2(u[13], u[12]), u[2], u[3], u[4], u[5], u[6], u[7]};
#pragma unroll
    for (int k = 0; k < 8; k++) raw[k] = from_d<S>(p8[k]);
  } else {
#pragma unroll
    for (int k = 0; k < R; k++) raw[k] = from_d<S>(u[k]);
  }
  using Wd = Words<S, R>;
  char *base = reinterpret_cast<char *>(out) + (long)(mu * 2 + p) * Wd::NW * g.Vh * Wd::W;
  store_reals<S, R>(base, g.Vh, h, raw);
}

size_t link_bytes(lqcd_prec prec, int recon, long Vh) {
  return (size_t)8 * Vh * recon * prec_bytes(prec);
}

template <typename S>
static cudaError_t pack_links_t(const Geom &g, const double *U, int recon, void *out, cudaStream_t st) {
  dim3 gr = grid2(g.Vh, 8, 128);
  if (recon == 12)
    pack_links_kernel<S, 12><<<gr, 128, 0, st>>>(g, U, out);
  else if (recon == 8)
    pack_links_kernel<S, 8><<<gr, 128, 0, st>>>(g, U, out);
  else
    pack_links_kernel<S, 18><<<gr, 128, 0, st>>>(g, U, out);
  return cudaGetLastError();
}

// min over links of |U01|^2 + |U02|^2 = 1 - |U00|^2, the determinant the
// 8-real rebuild divides by, as a min of IEEE bit patterns of non-negative
// doubles (order-independent); *out starts at all ones
__global__ void recon8_det_kernel(const double *__restrict__ U, long nlinks, unsigned long long *out) {
  for (long l = (long)blockIdx.x * blockDim.x + threadIdx.x; l < nlinks; l += (long)gridDim.x * blockDim.x) {
    const double *u = U + l * 18;
    const double d = u[2] * u[2] + u[3] * u[3] + u[4] * u[4] + u[5] * u[5];
    atomicMin(out, (unsigned long long)__double_as_longlong(d));
  }
}

cudaError_t recon8_min_det(const double *U, long nlinks, unsigned long long *dev_word, double *out, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(dev_word, 0xff, sizeof(unsigned long long), st);
  if (e != cudaSuccess) return e;
  recon8_det_kernel<<<(unsigned)std::min<long>((nlinks + 255) / 256, 4096), 256, 0, st>>>(U, nlinks, dev_word);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  unsigned long long w = 0;
  e = cudaMemcpyAsync(&w, dev_word, sizeof(w), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  std::memcpy(out, &w, sizeof(w));  // the bit pattern of a non-negative double
  return e;
}

cudaError_t pack_links(lqcd_prec prec, const Geom &g, const double *U, int recon, void *out, cudaStream_t st) {
  switch (prec) {
    case LQCD_F64: return pack_links_t<double>(g, U, recon, out, st);
    case LQCD_F32: return pack_links_t<float>(g, U, recon, out, st);
    case LQCD_F16: return pack_links_t<__half>(g, U, recon, out, st);
    case LQCD_BF16: return pack_links_t<__nv_bfloat16>(g, U, recon, out, st);
    case LQCD_DF64: return pack_links_t<df>(g, U, recon, out, st);
  }
  return cudaErrorInvalidValue;
}

// pointer of U_mu of parity p inside a packed allocation
const void *link_ptr(const void *base, lqcd_prec prec, int recon, long Vh, int mu, int p) {
  size_t per = link_bytes(prec, recon, Vh) / 8;
  return reinterpret_cast<const char *>(base) + per * (size_t)(mu * 2 + p);
}

// max over links of max(|U U^dag - 1|_max, |det U - 1|), as a max of the
// IEEE bit patterns of non-negative doubles (order-independent)
__global__ void su3_check_kernel(const double *__restrict__ U, long nlinks, unsigned long long *worst) {
  const long k = (long)blockIdx.x * blockDim.x + threadIdx.x;
  double e = 0.0;
  if (k < nlinks) {
    const double *u = U + 18 * k;
    cx<double> m[3][3];
#pragma unroll
    for (int i = 0; i < 9; i++) m[i / 3][i % 3] = mk<double>(u[2 * i], u[2 * i + 1]);
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
      for (int j = 0; j < 3; j++) {
        cx<double> t = mk<double>(i == j ? -1.0 : 0.0, 0.0);
#pragma unroll
        for (int c = 0; c < 3; c++) t = cjmadd(m[j][c], m[i][c], t);  // sum_c m_ic conj(m_jc)
        const double d = fmax(fabs(t.r), fabs(t.i));
        if (!(d <= e)) e = d;  // keeps a NaN (fmax would drop it)
      }
    cx<double> det = m[0][0] * (m[1][1] * m[2][2] - m[1][2] * m[2][1]) -
                     m[0][1] * (m[1][0] * m[2][2] - m[1][2] * m[2][0]) +
                     m[0][2] * (m[1][0] * m[2][1] - m[1][1] * m[2][0]);
    const double dd = fmax(fabs(det.r - 1.0), fabs(det.i));
    if (!(dd <= e)) e = dd;
    for (int i = 0; i < 18; i++)
      if (!(u[i] == u[i]) || fabs(u[i]) > 1e300) e = 1e300;  // NaN or Inf entries count as failure
    if (!(e == e)) e = 1e300;
  }
  for (int o = 16; o > 0; o >>= 1) e = fmax(e, __shfl_xor_sync(0xffffffffu, e, o));
  if ((threadIdx.x & 31) == 0) atomicMax(worst, (unsigned long long)__double_as_longlong(e));
}

cudaError_t su3_check(const double *U, long nlinks, unsigned long long *worst, cudaStream_t st) {
  su3_check_kernel<<<(unsigned)((nlinks + 255) / 256), 256, 0, st>>>(U, nlinks, worst);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// clover: FP64 master [blk][words][Vh] -> storage type S
// ---------------------------------------------------------------------------
template <typename S>
__global__ void pack_clover_kernel(long Vh, const double *__restrict__ in, void *out, float *scale) {
  const long h = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (h >= Vh) return;
  using W64 = Words<double, 36>;
  using WS = Words<S, 36>;
  double v[2][36];
#pragma unroll
  for (int blk = 0; blk < 2; blk++) {
    double raw[36];
    load_reals<double, 36>(reinterpret_cast<const char *>(in) + (long)blk * W64::NW * Vh * W64::W, Vh, h, raw);
#pragma unroll
    for (int k = 0; k < 36; k++) v[blk][k] = raw[k];
  }
  double sc = 1.0;
  if (IsHalf<S>::value) {
    double m = 0.0;
#pragma unroll
    for (int blk = 0; blk < 2; blk++)
#pragma unroll
      for (int k = 0; k < 36; k++) m = fmax(m, fabs(v[blk][k]));
    scale[h] = (float)m;
    sc = m > 0.0 ? 1.0 / m : 0.0;
  }
#pragma unroll
  for (int blk = 0; blk < 2; blk++) {
    S raw[36];
#pragma unroll
    for (int k = 0; k < 36; k++) raw[k] = from_d<S>(v[blk][k] * sc);
    store_reals<S, 36>(reinterpret_cast<char *>(out) + (long)blk * WS::NW * Vh * WS::W, Vh, h, raw);
  }
}

size_t clover_bytes(lqcd_prec prec, long Vh) {
  return (size_t)72 * prec_bytes(prec) * Vh;
}

cudaError_t pack_clover(lqcd_prec prec, long Vh, const double *in, void *out, float *scale, cudaStream_t st) {
  unsigned gr = (unsigned)((Vh + 127) / 128);
  switch (prec) {
    case LQCD_F64: return cudaMemcpyAsync(out, in, clover_bytes(prec, Vh), cudaMemcpyDeviceToDevice, st);
    case LQCD_F32: pack_clover_kernel<float><<<gr, 128, 0, st>>>(Vh, in, out, scale); break;
    case LQCD_F16: pack_clover_kernel<__half><<<gr, 128, 0, st>>>(Vh, in, out, scale); break;
    case LQCD_BF16: pack_clover_kernel<__nv_bfloat16><<<gr, 128, 0, st>>>(Vh, in, out, scale); break;
    case LQCD_DF64: pack_clover_kernel<df><<<gr, 128, 0, st>>>(Vh, in, out, scale); break;
  }
  return cudaGetLastError();
}

}  // namespace lqcd
