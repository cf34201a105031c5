// Building blocks of a domain-decomposed operator along t: time-slice
// packing of a field into contiguous halo buffers, the two kernels of the
// Schur complement on a range of time slices, and per-right-hand-side BLAS
// for the driver that runs the Krylov recursion across domains.
//
// A domain holds its time slices plus `halo` ghost slices on either side as
// an ordinary (extended) lattice context.  Because t is the slowest index of
// the site numbering and L0 is even, the sites of one parity on time slices
// [t0, t1) are the contiguous range h in [t0 S, t1 S) with S = Vh / L3, in
// the same order as on the full lattice: a slice of one domain is a slice of
// the global field, word for word.  The exchange between domains (NCCL,
// gloo, or copies between domains held by one process) is the caller's.
#include <cstring>

#include "internal.h"

namespace lqcd {
namespace {

constexpr int kDomT = 256;

// buf[(r NW + w) n + i] <-> field word w of RHS r at site h0 + i, times factor
template <typename W>
__global__ void __launch_bounds__(kDomT) slices_kernel(char *field, long rhs_bytes, long word_stride_bytes, long h0,
                                                       long n, int nw, int nrhs, W *buf, int to_field, double factor) {
  const long total = (long)nrhs * nw * n;
  for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (long)gridDim.x * blockDim.x) {
    const long i = e % n;
    const int w = (int)((e / n) % nw);
    const int r = (int)(e / ((long)n * nw));
    W *fw = reinterpret_cast<W *>(field + (long)r * rhs_bytes + (long)w * word_stride_bytes) + h0 + i;
    if (to_field) {
      *fw = buf[e];
    } else {
      buf[e] = *fw;
    }
  }
}

// the same with a sign factor on the reals of an FP64 or FP32 field (exact: +-1)
template <typename T>
__global__ void __launch_bounds__(kDomT) slices_sign_kernel(char *field, long rhs_bytes, long word_stride_bytes,
                                                            long h0, long n, int nw, int nrhs, uint4 *buf,
                                                            int to_field, T factor) {
  constexpr int per = 16 / sizeof(T);
  const long total = (long)nrhs * nw * n;
  for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (long)gridDim.x * blockDim.x) {
    const long i = e % n;
    const int w = (int)((e / n) % nw);
    const int r = (int)(e / ((long)n * nw));
    uint4 *fw = reinterpret_cast<uint4 *>(field + (long)r * rhs_bytes + (long)w * word_stride_bytes) + h0 + i;
    uint4 v = to_field ? buf[e] : *fw;
    T *t = reinterpret_cast<T *>(&v);
#pragma unroll
    for (int k = 0; k < per; k++) t[k] = factor * t[k];
    if (to_field)
      *fw = v;
    else
      buf[e] = v;
  }
}

// y = a_k x + b_k y on every complex number of right-hand side k (FP64 or FP32
// fields, arithmetic in the storage type; a, b per RHS on the device)
template <typename T>
__global__ void __launch_bounds__(kDomT) axpby_kernel(T *y, const T *x, long n_per_rhs, int nrhs, const double *a,
                                                      const double *b) {
  const long total = (long)nrhs * n_per_rhs;
  for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (long)gridDim.x * blockDim.x) {
    const int k = (int)(e / n_per_rhs);
    y[e] = fma((T)a[k], x[e], (T)b[k] * y[e]);
  }
}

unsigned dom_blocks(long total) {
  long b = (total + kDomT - 1) / kDomT;
  return (unsigned)(b < 1 ? 1 : (b > 8L * 152 * 8 ? 8L * 152 * 8 : b));
}

lqcd_status slice_range(lqcd_ctx *c, int t0, int t1, long *h0, long *h1) {
  if (t0 < 0 || t1 > c->dims[3] || t0 >= t1)
    return set_error(LQCD_ERR_ARG, "time slices [%d, %d) outside 0..%d", t0, t1, c->dims[3]);
  const long S = c->Vh / c->dims[3];
  *h0 = (long)t0 * S;
  *h1 = (long)t1 * S;
  return LQCD_OK;
}

lqcd_status check_pair(lqcd_ctx *c, const lqcd_field *f) {
  if (!c) return set_error(LQCD_ERR_ARG, "NULL context");
  if (!f || f->ctx != c) return set_error(LQCD_ERR_ARG, "field missing or of another context");
  return LQCD_OK;
}

}  // namespace
}  // namespace lqcd

using namespace lqcd;

extern "C" {

lqcd_status lqcd_field_slices(lqcd_ctx *c, lqcd_field *f, int parity, int t0, int t1, void *buf, int to_field,
                              double factor) {
  LQ_TRY(check_pair(c, f));
  if (!buf) return set_error(LQCD_ERR_ARG, "buf is NULL");
  if (parity != 0 && parity != 1) return set_error(LQCD_ERR_ARG, "parity must be 0 or 1");
  if (!f->has(parity)) return set_error(LQCD_ERR_ARG, "the field holds no sites of parity %d", parity);
  if (factor != 1.0 && factor != -1.0) return set_error(LQCD_ERR_ARG, "factor must be +1 or -1");
  // FP16/BF16 fields keep a per-site scale outside the 16-byte words
  if (prec_half(f->prec)) return set_error(LQCD_ERR_ARG, "FP16/BF16 fields are not sliced (their scales live apart)");
  cudaPointerAttributes pa;
  if (cudaPointerGetAttributes(&pa, buf) != cudaSuccess ||
      (pa.type != cudaMemoryTypeDevice && pa.type != cudaMemoryTypeManaged)) {
    cudaGetLastError();
    return set_error(LQCD_ERR_ARG, "buf must be device memory");
  }
  long h0, h1;
  LQ_TRY(slice_range(c, t0, t1, &h0, &h1));
  const long n = h1 - h0;
  const int nw = (int)spinor_words(f->prec);  // 16-byte words per site
  const long word_stride = 16L * f->Vh;
  const long rhs_bytes = 16L * f->rhs_words();
  char *base = reinterpret_cast<char *>(f->data[parity]);
  const long total = (long)f->nrhs * nw * n;
  if (factor == 1.0) {
    slices_kernel<uint4><<<dom_blocks(total), kDomT, 0, c->stream>>>(base, rhs_bytes, word_stride, h0, n, nw, f->nrhs,
                                                                     (uint4 *)buf, to_field, 1.0);
  } else if (f->prec == LQCD_F64) {  // DF64 (hi, lo floats) and FP32 flip float by float below
    slices_sign_kernel<double><<<dom_blocks(total), kDomT, 0, c->stream>>>(base, rhs_bytes, word_stride, h0, n, nw,
                                                                           f->nrhs, (uint4 *)buf, to_field, -1.0);
  } else {
    slices_sign_kernel<float><<<dom_blocks(total), kDomT, 0, c->stream>>>(base, rhs_bytes, word_stride, h0, n, nw,
                                                                          f->nrhs, (uint4 *)buf, to_field, -1.0f);
  }
  LQ_CU(cudaGetLastError());
  return LQCD_OK;
}

lqcd_status lqcd_k2a_slices(lqcd_ctx *c, lqcd_recon recon, int dagger, lqcd_field *y_even, const lqcd_field *x_odd,
                            int t0, int t1) {
  LQ_TRY(check_pair(c, y_even));
  LQ_TRY(check_pair(c, x_odd));
  if (!y_even->has(0) || !x_odd->has(1)) return set_error(LQCD_ERR_ARG, "needs even y and odd x");
  if (y_even->prec != x_odd->prec || y_even->nrhs != x_odd->nrhs)
    return set_error(LQCD_ERR_ARG, "fields must share precision and nrhs");
  long h0, h1;
  LQ_TRY(slice_range(c, t0, t1, &h0, &h1));
  return op_k2a(c, y_even->prec, (int)recon, dagger ? 1 : 0, y_even->nrhs, y_even->mut(0), x_odd->ref(1), h0, h1);
}

lqcd_status lqcd_k2b_slices(lqcd_ctx *c, lqcd_recon recon, int dagger, lqcd_field *z_odd, const lqcd_field *x_odd,
                            const lqcd_field *y_even, int t0, int t1, double *norm2) {
  LQ_TRY(check_pair(c, z_odd));
  LQ_TRY(check_pair(c, x_odd));
  LQ_TRY(check_pair(c, y_even));
  if (!z_odd->has(1) || !x_odd->has(1) || !y_even->has(0))
    return set_error(LQCD_ERR_ARG, "needs odd output, odd x and even y");
  if (z_odd->prec != x_odd->prec || z_odd->prec != y_even->prec || z_odd->nrhs != x_odd->nrhs ||
      z_odd->nrhs != y_even->nrhs)
    return set_error(LQCD_ERR_ARG, "fields must share precision and nrhs");
  if (z_odd == x_odd) return set_error(LQCD_ERR_ARG, "z and x must be different fields");
  if (norm2 && z_odd->nrhs > 256) return set_error(LQCD_ERR_ARG, "norms of up to 256 right-hand sides");
  long h0, h1;
  LQ_TRY(slice_range(c, t0, t1, &h0, &h1));
  const FieldRef none{nullptr, nullptr, 0};
  LQ_TRY(op_k2b(c, z_odd->prec, (int)recon, dagger ? 1 : 0, z_odd->nrhs, z_odd->mut(1), x_odd->ref(1),
                y_even->ref(0), none, 0.0, norm2 ? c->results : nullptr, 1, h0, h1));
  if (norm2) {
    LQ_CU(cudaMemcpyAsync(c->h_results, c->results, sizeof(double) * z_odd->nrhs, cudaMemcpyDeviceToHost, c->stream));
    LQ_CU(cudaStreamSynchronize(c->stream));
    for (int k = 0; k < z_odd->nrhs; k++) norm2[k] = c->h_results[k];
  }
  return LQCD_OK;
}

lqcd_status lqcd_field_axpby(lqcd_ctx *c, lqcd_field *y, const double *a, const double *b, const lqcd_field *x) {
  LQ_TRY(check_pair(c, y));
  LQ_TRY(check_pair(c, x));
  if (!a || !b) return set_error(LQCD_ERR_ARG, "coefficients are NULL");
  if (y->prec != x->prec || y->nrhs != x->nrhs || y->subset != x->subset)
    return set_error(LQCD_ERR_ARG, "x and y must share precision, subset and nrhs");
  if (y->prec != LQCD_F64 && y->prec != LQCD_F32) return set_error(LQCD_ERR_ARG, "axpby takes FP64 or FP32 fields");
  if (y->nrhs > 128) return set_error(LQCD_ERR_ARG, "axpby takes up to 128 right-hand sides");
  // the coefficients go to the context's small device array ([256, 512) is theirs)
  double *dc = c->results + 256;
  std::memcpy(c->h_results + 256, a, sizeof(double) * y->nrhs);
  std::memcpy(c->h_results + 256 + y->nrhs, b, sizeof(double) * y->nrhs);
  LQ_CU(cudaMemcpyAsync(dc, c->h_results + 256, sizeof(double) * 2 * y->nrhs, cudaMemcpyHostToDevice, c->stream));
  const long n = 24L * y->Vh;  // reals of one RHS of one parity
  for (int p = 0; p < 2; p++) {
    if (!y->has(p)) continue;
    if (y->prec == LQCD_F64)
      axpby_kernel<double><<<dom_blocks((long)y->nrhs * n), kDomT, 0, c->stream>>>(
          (double *)y->data[p], (const double *)x->data[p], n, y->nrhs, dc, dc + y->nrhs);
    else
      axpby_kernel<float><<<dom_blocks((long)y->nrhs * n), kDomT, 0, c->stream>>>(
          (float *)y->data[p], (const float *)x->data[p], n, y->nrhs, dc, dc + y->nrhs);
    LQ_CU(cudaGetLastError());
  }
  // the host staging of the coefficients is reused by the next call
  LQ_CU(cudaStreamSynchronize(c->stream));
  return LQCD_OK;
}

lqcd_status lqcd_field_norm2s(lqcd_ctx *c, const lqcd_field *f, double *out) {
  LQ_TRY(check_pair(c, f));
  if (!out) return set_error(LQCD_ERR_ARG, "out is NULL");
  if (f->nrhs > 256) return set_error(LQCD_ERR_ARG, "norms of up to 256 right-hand sides");
  LQ_TRY(ensure_partials(c, f->nrhs));
  for (int k = 0; k < f->nrhs; k++) out[k] = 0.0;
  for (int p = 0; p < 2; p++) {
    if (!f->has(p)) continue;
    LQ_CU(blas_norm2(f->prec, c->Vh, f->nrhs, f->ref(p), c->partials, c->results, 1, c->stream));
    LQ_CU(cudaMemcpyAsync(c->h_results, c->results, sizeof(double) * f->nrhs, cudaMemcpyDeviceToHost, c->stream));
    LQ_CU(cudaStreamSynchronize(c->stream));
    for (int k = 0; k < f->nrhs; k++) out[k] += c->h_results[k];
  }
  return LQCD_OK;
}

}  // extern "C"
