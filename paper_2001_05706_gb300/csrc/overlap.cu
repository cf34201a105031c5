// Overlap operator: low modes of H_W, the polynomial sign function and the
// overlap operator and its CG inverse (GWU-code's overlap inverter, abstract
// and Secs. 3-4 of the paper; standard definitions, see include/lqcd.h).
//
//  * Low modes: block subspace iteration on H_W^2 in FP64.  Each sweep
//    applies a Chebyshev filter of H_W^2 that damps the interval
//    [mu_max, b] (mu_max the largest Ritz value of H_W^2 in the block),
//    orthonormalises the block by Cholesky QR (twice), and does a
//    Rayleigh-Ritz step with H_W^2; once the wanted vectors have converged,
//    a Rayleigh-Ritz step with H_W in their span fixes the signs of the
//    eigenvalues.  The block inner products (Gram matrices) and rotations are
//    own tiled kernels accumulating in double-float on the FP32 pipes (GB300
//    runs FP64 multiply-adds at 1/64 of its FP32 rate); the m x m Hermitian
//    eigenproblem (m <= 96) is solved on the host by cyclic Jacobi rotations.
//  * Sign function: exact low modes plus H_W P(H_W^2) on their complement,
//    P the Chebyshev interpolant of 1/sqrt(y) on [a, b], evaluated by the
//    Clenshaw recurrence b_k = c_k w + 2 T b_{k+1} - b_{k+2},
//    T = (2 H_W^2 - a - b)/(b - a); each step is two H_W applications (the
//    dslash kernel, all right-hand sides per launch), the second of which
//    adds the three-term update in its epilogue (MODE_CHEB).
//  * D_ov(m) = f (1 + g5 eps) + m with f = (1 - m/(2 rho)) rho, and CG on its
//    normal equations for the inverse.

#include <algorithm>
#include <functional>
#include <chrono>
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "internal.h"

namespace lqcd {

using zc = std::complex<double>;

struct OverlapState {
  bool ready = false;
  lqcd_overlap_params prm{};
  int nlow = 0;
  std::vector<double> lam;
  lqcd_field *vecs = nullptr;    // FULL FP64, nrhs = nlow
  lqcd_field *vecs32 = nullptr;  // the same in FP32 (inner solves)
  std::vector<double> coef;    // sign function to sign_tol (FP64 / DF64)
  std::vector<double> coef32;  // the FP32 one inside the mixed CG: to max(sign_tol, 1e-6)
  double a = 0, b = 0;
  int degree = 0, degree32 = 0;
  bool df = false;            // FP64 parts computed in double-float (prm.high == LQCD_DF64)
  double2 *dsmall = nullptr;  // device scratch for small matrices
  size_t dsmall_n = 0;
  double *gpart = nullptr;  // per-chunk partials of the Gram kernel
  size_t gpart_n = 0;
  // eigensystem of D_ov(0)^dag D_ov(0) (lqcd_overlap_eigen): ev_n vectors of
  // chirality ev_sector, then ev_np partners of the other chirality (FULL FP64)
  lqcd_field *ev = nullptr;
  int ev_n = 0, ev_np = 0, ev_sector = 0;
  std::vector<double> ev_mu;    // eigenvalue of each column of ev
  std::vector<double> ev_c;     // <chi_i, eps chi_i> of each sector vector
  std::vector<double> ev_pn;    // |P_-s eps chi_i| (0: no partner)
  std::vector<int> ev_partner;  // column of chi_i's partner in ev, or -1
};

void overlap_free(lqcd_ctx *c) {
  OverlapState *s = c->ov;
  if (!s) return;
  if (s->vecs) lqcd_field_destroy(s->vecs);
  if (s->vecs32) lqcd_field_destroy(s->vecs32);
  if (s->ev) lqcd_field_destroy(s->ev);
  if (s->gpart) cudaFree(s->gpart);
  if (s->dsmall) cudaFree(s->dsmall);
  delete s;
  c->ov = nullptr;
}

namespace {

constexpr int kT = 256;
// accuracy of the FP32 sign function of the mixed overlap CG (its rounding level)
constexpr double kInnerSignTol = 1e-6;
// widest low-mode block (the rotation kernel holds this many rows of its matrix)
constexpr int kOvMaxBlock = 96;
// Low-mode block size m = max(want + 16, LQCD_OV_BLOCK_MULT * want), capped at
// 96.  Measured on 16^3x32 (20 modes, |lambda| 0.509-0.510 clustered, DF64
// sweeps): m = 40: 214 sweeps, 84 s; m = 60: 191 sweeps, 114 s; m = 96: 143
// sweeps, 163 s -- a wider block widens the damped gap, but not by enough to
// pay for its cost per sweep.
// Lanczos basis size (thick restart keeps the block size m of vectors)
#ifndef LQCD_OV_LANCZOS_MMAX
#define LQCD_OV_LANCZOS_MMAX 256
#endif
#ifndef LQCD_OV_BLOCK_MULT
#define LQCD_OV_BLOCK_MULT 2
#endif
#ifndef LQCD_OV_FP32_RULE
#define LQCD_OV_FP32_RULE 1
#endif
// LQCD_OVERLAP_TRACE=1 prints one line per low-mode sweep to stderr
const bool kOvTrace = std::getenv("LQCD_OVERLAP_TRACE") != nullptr;

// ---- kernels on FULL FP64 fields: grid (blocks over words*Vh, nrhs, parity) --

// out = cw w + t (s2 hh + s0 b1) - b2   (w, b2 may be null: zero), element-wise
// on the complex numbers of FULL fields (FP64: double2, FP32: float2 view);
// coefficients in FP64, arithmetic in the storage precision's math type
template <typename C2>
__global__ void clenshaw_kernel(long n, C2 *o0, C2 *o1, const C2 *w0, const C2 *w1, const C2 *h0, const C2 *h1,
                                const C2 *a0, const C2 *a1, const C2 *c0, const C2 *c1, double cw_, double t_,
                                double s2_, double s0_) {
  using R = decltype(C2{}.x);
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const long off = (long)blockIdx.y * n + i;
  if (i >= n) return;
  const int p = blockIdx.z;
  const R cw = (R)cw_, t = (R)t_, s2 = (R)s2_, s0 = (R)s0_;
  C2 *o = p ? o1 : o0;
  const C2 *w = p ? w1 : w0, *h = p ? h1 : h0, *b1 = p ? a1 : a0, *b2 = p ? c1 : c0;
  const C2 hv = h[off], bv = b1[off];
  C2 r;
  r.x = t * (s2 * hv.x + s0 * bv.x);
  r.y = t * (s2 * hv.y + s0 * bv.y);
  if (w) {
    const C2 wv = w[off];
    r.x += cw * wv.x;
    r.y += cw * wv.y;
  }
  if (b2) {
    const C2 cv = b2[off];
    r.x -= cv.x;
    r.y -= cv.y;
  }
  o[off] = r;
}

// out = a in + b (g5 e or e), element-wise on complex numbers.  Element e of
// one RHS of one parity holds spin: FP64 (one complex per 16-byte word w,
// e = w Vh + i) spin = w / 3; FP32 (two complex per word, e = 2 (w Vh + i) + j)
// spin = (2 w + j) / 3.
template <typename C2>
__global__ void ov_combine_kernel(long Vh, long n, C2 *o0, C2 *o1, const C2 *i0, const C2 *i1, const C2 *e0,
                                  const C2 *e1, double a_, double b_, int g5) {
  using R = decltype(C2{}.x);
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const long off = (long)blockIdx.y * n + i;
  const int p = blockIdx.z;
  const C2 x = (p ? i1 : i0)[off], e = (p ? e1 : e0)[off];
  int spin;
  if (sizeof(R) == 8)
    spin = (int)(i / Vh) / 3;
  else
    spin = (int)(2 * ((i >> 1) / Vh) + (i & 1)) / 3;
  const R a = (R)a_, b = (g5 && spin >= 2) ? (R)-b_ : (R)b_;
  C2 r;
  r.x = a * x.x + b * e.x;
  r.y = a * x.y + b * e.y;
  (p ? o1 : o0)[off] = r;
}

// Gaussian fill of raw doubles: SplitMix64 (Steele et al. 2014) counters + Box-Muller
__device__ __forceinline__ unsigned long long sm64(unsigned long long x) {
  unsigned long long z = x + 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}
__global__ void gauss_fill_kernel(double *x, long n, unsigned long long seed) {
  const long k = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (2 * k >= n) return;
  const unsigned long long s = sm64(seed);
  const double u1 = ((double)((sm64(s ^ (2 * k + 1) * 0xD1B54A32D192ED03ULL) >> 11) + 1)) * 0x1.0p-53;
  const double u2 = ((double)((sm64(s ^ (2 * k + 2) * 0xD1B54A32D192ED03ULL) >> 11) + 1)) * 0x1.0p-53;
  const double r = sqrt(-2.0 * log(u1));
  double sn, cs;
  sincospi(2.0 * u2, &sn, &cs);
  x[2 * k] = r * cs;
  if (2 * k + 1 < n) x[2 * k + 1] = r * sn;
}

// per-RHS ||x_k + c_k y_k||^2 over both parities (c on the device)
__global__ void axpy_norm_kernel(long n, const double2 *x0, const double2 *x1, const double2 *y0, const double2 *y1,
                                 const double *c, double *partials, unsigned *counter, double *result, int nrhs) {
  const int k = blockIdx.y;
  const double ck = c[k];
  double v[1] = {0.0};
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < 2 * n; i += (long)gridDim.x * blockDim.x) {
    const int p = i >= n;
    const long off = (long)k * n + (p ? i - n : i);
    const double2 a = (p ? x1 : x0)[off], b = (p ? y1 : y0)[off];
    const double re = a.x + ck * b.x, im = a.y + ck * b.y;
    v[0] += re * re + im * im;
  }
  grid_reduce<1>(v, partials, counter, result, k, nrhs, 1);
}

template <typename C2>
__global__ void scale_rows_kernel(C2 *m, int rows, int cols, const double *s) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= rows * cols) return;
  const double f = s[i % rows];
  m[i].x *= f;
  m[i].y *= f;
}

// ---- host helpers ------------------------------------------------------------

lqcd_status ensure_state(lqcd_ctx *c) {
  if (!c->ov) c->ov = new OverlapState();
  return LQCD_OK;
}

lqcd_status small_scratch(lqcd_ctx *c, size_t n, double2 **p) {
  OverlapState &s = *c->ov;
  if (s.dsmall_n < n) {
    if (s.dsmall) {
      LQ_CU(cudaStreamSynchronize(c->stream));
      cudaFree(s.dsmall);
      s.dsmall = nullptr;
    }
    LQ_CU(dev_malloc((void **)&s.dsmall, n * sizeof(double2)));
    s.dsmall_n = n;
  }
  *p = s.dsmall;
  return LQCD_OK;
}

long cwords(const lqcd_field *f) { return 12L * f->Vh; }  // complex numbers per RHS per parity
size_t celem(const lqcd_field *f) { return 2 * (size_t)prec_bytes(f->prec); }  // bytes per complex number

void *col(const lqcd_field *f, int p, int k) {
  return reinterpret_cast<char *>(f->data[p]) + (size_t)k * cwords(f) * celem(f);
}

// ---- block inner products and rotations ---------------------------------------
// Own kernels for the two dense products of the low-mode solver and of the
// sign function's projection: C = X^H Y (Gram) and Z = alpha X M + beta Z
// (rotation), X, Y, Z columns of FULL fields (both parities; complex numbers
// as double2 for FP64, float2 for FP32 fields).  Products accumulate in
// double-float (compensated, ~2^-44 relative) on the FP32 pipes: an FP64
// inner product would run at GB300's 1/64 FP64 rate.  Every input is
// converted to double-float once per shared-memory tile or per rotation
// column tile, not per product.
struct cdf {
  df re, im;
};
__device__ __forceinline__ cdf to_cdf(double2 v) { return cdf{df(v.x), df(v.y)}; }
__device__ __forceinline__ cdf to_cdf(float2 v) { return cdf{df(v.x), df(v.y)}; }
__device__ __forceinline__ void from_cdf(double2 &o, cdf a) { o = make_double2((double)a.re, (double)a.im); }
__device__ __forceinline__ void from_cdf(float2 &o, cdf a) {
  o = make_float2(__fadd_rn(a.re.hi, a.re.lo), __fadd_rn(a.im.hi, a.im.lo));
}

constexpr int kGT = 16;    // edge of the C tile of one Gram block
constexpr int kGE = 32;    // elements per shared-memory step
constexpr int kRQ = 16;    // Z columns per rotation thread
constexpr int kRMaxP = 96; // rows of M a rotation block holds

// partials of C = X^H Y: block (tile, chunk) sums elements [chunk * per, ...)
// of both parities (e < n parity 0, e - n parity 1) for a kGT x kGT tile of C
template <typename E>
__global__ void __launch_bounds__(kGT * kGT) ov_gram_kernel(const E *X0, const E *X1, const E *Y0, const E *Y1, long ld,
                                                             long n, int p, int q, int tiles_i, long per,
                                                             double *part) {
  __shared__ cdf sx[kGE][kGT], sy[kGE][kGT];
  const int nch = gridDim.y, chunk = blockIdx.y;
  const int i0 = (blockIdx.x % tiles_i) * kGT, j0 = (blockIdx.x / tiles_i) * kGT;
  const int ti = threadIdx.x % kGT, tj = threadIdx.x / kGT;
  const long e_beg = (long)chunk * per, e_end = min(2 * n, e_beg + per);
  dfacc re{0.0f, 0.0f}, im{0.0f, 0.0f};
  const cdf zero{df(0.0f, 0.0f), df(0.0f, 0.0f)};
  for (long e0 = e_beg; e0 < e_end; e0 += kGE) {
    for (int l = threadIdx.x; l < kGE * kGT; l += kGT * kGT) {
      const int ee = l % kGE, cc = l / kGE;
      const long e = e0 + ee;
      cdf vx = zero, vy = zero;
      if (e < e_end) {
        const long off = e < n ? e : e - n;
        if (i0 + cc < p) vx = to_cdf((e < n ? X0 : X1)[(long)(i0 + cc) * ld + off]);
        if (j0 + cc < q) vy = to_cdf((e < n ? Y0 : Y1)[(long)(j0 + cc) * ld + off]);
      }
      sx[ee][cc] = vx;
      sy[ee][cc] = vy;
    }
    __syncthreads();
#pragma unroll 4
    for (int ee = 0; ee < kGE; ee++) {
      const cdf x = sx[ee][ti], y = sy[ee][tj];
      dfacc_madd(re, x.re, y.re);  // conj(x) y
      dfacc_madd(re, x.im, y.im);
      dfacc_madd(im, x.re, y.im);
      dfacc_madd(im, -x.im, y.re);
    }
    __syncthreads();
  }
  const int i = i0 + ti, j = j0 + tj;
  if (i < p && j < q) {
    const long k = (long)i + (long)p * j;
    part[(2 * k) * nch + chunk] = (double)dfacc_value(re);
    part[(2 * k + 1) * nch + chunk] = (double)dfacc_value(im);
  }
}

// C[k] = the sum of its chunk partials, in chunk order (deterministic)
template <typename CE> __global__ void ov_gram_finish_kernel(const double *part, int nch, int pq, CE *C) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= pq) return;
  double re = 0.0, im = 0.0;
  for (int ch = 0; ch < nch; ch++) {
    re += part[(2L * k) * nch + ch];
    im += part[(2L * k + 1) * nch + ch];
  }
  if constexpr (std::is_same<CE, double2>::value)
    C[k] = make_double2(re, im);
  else
    C[k] = make_float2((float)re, (float)im);
}

// Z[:, q0 + c] = alpha sum_l X[:, l] M[l, q0 + c] + beta Z[:, q0 + c] for kRQ columns
// per block row; grid (element chunks, column tiles), grid-stride over elements
template <typename E>
__global__ void __launch_bounds__(128) ov_rotate_kernel(const E *X0, const E *X1, long ld, long n, int p, const E *M,
                                                         int q, E *Z0, E *Z1, double alpha, double beta) {
  __shared__ cdf ms[kRMaxP][kRQ];
  const int q0 = blockIdx.y * kRQ;
  const cdf zero{df(0.0f, 0.0f), df(0.0f, 0.0f)};
  for (int l = threadIdx.x; l < p * kRQ; l += blockDim.x) {
    const int r = l / kRQ, cc = l % kRQ;
    ms[r][cc] = q0 + cc < q ? to_cdf(M[r + (long)p * (q0 + cc)]) : zero;
  }
  __syncthreads();
  const df al((float)alpha), be((float)beta);
  const int nq = min(kRQ, q - q0);
  for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < 2 * n; e += (long)gridDim.x * blockDim.x) {
    const E *Xp = e < n ? X0 : X1;
    E *Zp = e < n ? Z0 : Z1;
    const long off = e < n ? e : e - n;
    dfacc re[kRQ], im[kRQ];
#pragma unroll
    for (int cc = 0; cc < kRQ; cc++) re[cc] = im[cc] = dfacc{0.0f, 0.0f};
    for (int l = 0; l < p; l++) {
      const cdf x = to_cdf(Xp[(long)l * ld + off]);
#pragma unroll
      for (int cc = 0; cc < kRQ; cc++) {
        const cdf m = ms[l][cc];
        dfacc_madd(re[cc], x.re, m.re);
        dfacc_madd(re[cc], -x.im, m.im);
        dfacc_madd(im[cc], x.re, m.im);
        dfacc_madd(im[cc], x.im, m.re);
      }
    }
#pragma unroll
    for (int cc = 0; cc < kRQ; cc++) {
      if (cc >= nq) break;
      E &z = Zp[(long)(q0 + cc) * ld + off];
      cdf v{al * dfacc_value(re[cc]), al * dfacc_value(im[cc])};
      if (beta != 0.0) {
        const cdf zo = to_cdf(z);
        v.re = fma(be, zo.re, v.re);
        v.im = fma(be, zo.im, v.im);
      }
      from_cdf(z, v);
    }
  }
}

lqcd_status gram_partials(lqcd_ctx *c, size_t n, double **p) {
  OverlapState &s = *c->ov;
  if (s.gpart_n < n) {
    if (s.gpart) {
      LQ_CU(cudaStreamSynchronize(c->stream));
      cudaFree(s.gpart);
      s.gpart = nullptr;
    }
    LQ_CU(dev_malloc((void **)&s.gpart, n * sizeof(double)));
    s.gpart_n = n;
  }
  *p = s.gpart;
  return LQCD_OK;
}

// C(p x q) = X^H Y over both parities (X: first p RHS of fx, Y: first q RHS of
// fy, same precision), C on the device as double2 (FP64) or float2 (FP32)
lqcd_status gram(lqcd_ctx *c, const lqcd_field *fx, int p, const lqcd_field *fy, int q, void *C) {
  if (fx->prec != fy->prec || (fx->prec != LQCD_F64 && fx->prec != LQCD_F32))
    return set_error(LQCD_ERR_ARG, "Gram of fields of precisions %d, %d", (int)fx->prec, (int)fy->prec);
  const long n = cwords(fx);
  const int ti = (p + kGT - 1) / kGT, tq = (q + kGT - 1) / kGT;
  // about four blocks per SM over all tiles, chunks of whole shared-memory steps
  const int nch = (int)std::max<long>(1, std::min<long>(64, (4 * 152 + ti * tq - 1) / (ti * tq)));
  const long per = ((2 * n + nch - 1) / nch + kGE - 1) / kGE * kGE;
  double *part;
  LQ_TRY(gram_partials(c, 2 * (size_t)p * q * nch, &part));
  const dim3 grid((unsigned)(ti * tq), (unsigned)nch);
  if (fx->prec == LQCD_F64) {
    ov_gram_kernel<double2><<<grid, kGT * kGT, 0, c->stream>>>(
        (const double2 *)fx->data[0], (const double2 *)fx->data[1], (const double2 *)fy->data[0],
        (const double2 *)fy->data[1], n, n, p, q, ti, per, part);
    LQ_CU(cudaGetLastError());
    ov_gram_finish_kernel<double2><<<(p * q + 127) / 128, 128, 0, c->stream>>>(part, nch, p * q, (double2 *)C);
  } else {
    ov_gram_kernel<float2><<<grid, kGT * kGT, 0, c->stream>>>(
        (const float2 *)fx->data[0], (const float2 *)fx->data[1], (const float2 *)fy->data[0],
        (const float2 *)fy->data[1], n, n, p, q, ti, per, part);
    LQ_CU(cudaGetLastError());
    ov_gram_finish_kernel<float2><<<(p * q + 127) / 128, 128, 0, c->stream>>>(part, nch, p * q, (float2 *)C);
  }
  LQ_CU(cudaGetLastError());
  return LQCD_OK;
}

// Z = alpha X M + beta Z (X: N x p block of fx, M: p x q on the device, Z: N x q block of fz;
// alpha, beta real, fz not overlapping fx)
lqcd_status rotate(lqcd_ctx *c, const lqcd_field *fx, int p, const void *M, int q, lqcd_field *fz, double alpha,
                   double beta) {
  if (fx->prec != fz->prec || (fx->prec != LQCD_F64 && fx->prec != LQCD_F32))
    return set_error(LQCD_ERR_ARG, "rotation of fields of precisions %d, %d", (int)fx->prec, (int)fz->prec);
  if (p > kRMaxP) return set_error(LQCD_ERR_ARG, "rotation of %d > %d columns", p, kRMaxP);
  const long n = cwords(fx);
  const int tq = (q + kRQ - 1) / kRQ;
  const long chunks = std::max<long>(1, std::min<long>((2 * n + 127) / 128, (8L * 152 + tq - 1) / tq));
  const dim3 grid((unsigned)chunks, (unsigned)tq);
  if (fx->prec == LQCD_F64)
    ov_rotate_kernel<double2><<<grid, 128, 0, c->stream>>>(
        (const double2 *)fx->data[0], (const double2 *)fx->data[1], n, n, p, (const double2 *)M, q,
        (double2 *)fz->data[0], (double2 *)fz->data[1], alpha, beta);
  else
    ov_rotate_kernel<float2><<<grid, 128, 0, c->stream>>>((const float2 *)fx->data[0], (const float2 *)fx->data[1], n,
                                                          n, p, (const float2 *)M, q, (float2 *)fz->data[0],
                                                          (float2 *)fz->data[1], alpha, beta);
  LQ_CU(cudaGetLastError());
  return LQCD_OK;
}

// Cyclic Jacobi eigensolver for a Hermitian m x m matrix (column-major).
// On return A is diagonal (eigenvalues on the diagonal) and V holds the
// eigenvectors as columns: A_in = V diag V^H.
void jacobi_eigh(int m, std::vector<zc> &A, std::vector<zc> &V, std::vector<double> &w) {
  auto at = [&](int i, int j) -> zc & { return A[i + (size_t)m * j]; };
  V.assign((size_t)m * m, zc(0, 0));
  for (int i = 0; i < m; i++) V[i + (size_t)m * i] = 1.0;
  for (int sweep = 0; sweep < 100; sweep++) {
    double off = 0, dia = 0;
    for (int j = 0; j < m; j++)
      for (int i = 0; i < m; i++) (i == j ? dia : off) += std::norm(at(i, j));
    if (off <= 1e-30 * dia || off == 0.0) break;
    for (int p = 0; p < m - 1; p++)
      for (int q = p + 1; q < m; q++) {
        const zc apq = at(p, q);
        const double g = std::abs(apq);
        if (g < 1e-300) continue;
        const zc e = apq / g;  // phase: D = diag(1 at p, conj(e) at q) makes a_pq real
        const double app = at(p, p).real(), aqq = at(q, q).real();
        const double tau = (aqq - app) / (2 * g);
        const double t = (tau >= 0 ? 1.0 : -1.0) / (std::fabs(tau) + std::sqrt(1 + tau * tau));
        const double cs = 1 / std::sqrt(1 + t * t), sn = t * cs;
        // unitary U on columns (p, q): U = D R, R = [[cs, sn], [-sn, cs]]
        const zc u_pp = cs, u_pq = sn, u_qp = -sn * std::conj(e), u_qq = cs * std::conj(e);
        for (int k = 0; k < m; k++) {  // A <- A U
          const zc akp = at(k, p), akq = at(k, q);
          at(k, p) = akp * u_pp + akq * u_qp;
          at(k, q) = akp * u_pq + akq * u_qq;
        }
        for (int k = 0; k < m; k++) {  // A <- U^H A
          const zc apk = at(p, k), aqk = at(q, k);
          at(p, k) = std::conj(u_pp) * apk + std::conj(u_qp) * aqk;
          at(q, k) = std::conj(u_pq) * apk + std::conj(u_qq) * aqk;
        }
        for (int k = 0; k < m; k++) {  // V <- V U
          const zc vkp = V[k + (size_t)m * p], vkq = V[k + (size_t)m * q];
          V[k + (size_t)m * p] = vkp * u_pp + vkq * u_qp;
          V[k + (size_t)m * q] = vkp * u_pq + vkq * u_qq;
        }
        at(p, q) = at(q, p) = 0.0;
      }
  }
  w.resize(m);
  for (int i = 0; i < m; i++) w[i] = at(i, i).real();
}

// Hermitian eigendecomposition for larger projected matrices (the Lanczos
// Rayleigh-Ritz step, where the cyclic Jacobi method's O(m^3) per sweep,
// times ten sweeps, dominated a 511-column restart):
// Householder reduction to Hermitian tridiagonal form, a diagonal phase
// transformation to a real symmetric tridiagonal, and the implicit QL method
// with Wilkinson shifts (Givens rotations accumulated into the eigenvectors).
// A (column-major, destroyed), V the eigenvectors as columns, w the
// eigenvalues (unsorted, as the Jacobi routine).  False if QL stalls.
bool tridiag_eigh(int m, std::vector<zc> &A, std::vector<zc> &V, std::vector<double> &w) {
  auto at = [&](int i, int j) -> zc & { return A[i + (size_t)m * j]; };
  std::vector<zc> Q((size_t)m * m, zc(0, 0)), off(m, zc(0, 0)), v(m), p(m), q(m);
  for (int i = 0; i < m; i++) Q[i + (size_t)m * i] = 1.0;
  std::vector<double> d(m), e(m, 0.0);
  // 1. A = Q T Q^H: for column k, H = I - 2 u u^H maps A[k+1:, k] to alpha e_1
  for (int k = 0; k + 2 < m; k++) {
    const int n = m - k - 1;  // length of the trailing block
    double xn = 0;
    for (int i = 0; i < n; i++) xn += std::norm(at(k + 1 + i, k));
    xn = std::sqrt(xn);
    if (xn == 0.0) continue;
    const zc x0 = at(k + 1, k);
    const zc ph = std::abs(x0) > 0 ? x0 / std::abs(x0) : zc(1, 0);
    const zc alpha = -ph * xn;
    for (int i = 0; i < n; i++) v[i] = at(k + 1 + i, k);
    v[0] -= alpha;
    double vn = 0;
    for (int i = 0; i < n; i++) vn += std::norm(v[i]);
    vn = std::sqrt(vn);
    if (vn == 0.0) continue;
    for (int i = 0; i < n; i++) v[i] /= vn;
    // trailing block B <- H B H = B - 2 (v w^H + w v^H), w = B v - (v^H B v) v
    for (int i = 0; i < n; i++) {
      zc s = 0;
      for (int j = 0; j < n; j++) s += at(k + 1 + i, k + 1 + j) * v[j];
      p[i] = s;
    }
    zc vp = 0;
    for (int i = 0; i < n; i++) vp += std::conj(v[i]) * p[i];
    for (int i = 0; i < n; i++) q[i] = p[i] - vp.real() * v[i];
    for (int j = 0; j < n; j++)
      for (int i = 0; i < n; i++)
        at(k + 1 + i, k + 1 + j) -= 2.0 * (v[i] * std::conj(q[j]) + q[i] * std::conj(v[j]));
    // the column and row k: alpha below the diagonal, zeros under it
    at(k + 1, k) = alpha;
    at(k, k + 1) = std::conj(alpha);
    for (int i = 1; i < n; i++) at(k + 1 + i, k) = at(k, k + 1 + i) = 0.0;
    // Q <- Q H on columns k + 1 ..
    for (int r = 0; r < m; r++) {
      zc s = 0;
      for (int j = 0; j < n; j++) s += Q[r + (size_t)m * (k + 1 + j)] * v[j];
      for (int j = 0; j < n; j++) Q[r + (size_t)m * (k + 1 + j)] -= 2.0 * s * std::conj(v[j]);
    }
  }
  // 2. T = D S D^H with S real: D_0 = 1, D_{k+1} = D_k t_k / |t_k| for the
  //    subdiagonal t_k = T[k+1][k]; S has |t_k| below the diagonal
  std::vector<zc> ph(m, zc(1, 0));
  for (int k = 0; k < m; k++) d[k] = at(k, k).real();
  for (int k = 0; k + 1 < m; k++) {
    const zc t = at(k + 1, k);
    e[k] = std::abs(t);
    ph[k + 1] = e[k] > 0 ? ph[k] * (t / e[k]) : ph[k];
  }
  // 3. implicit QL on (d, e): Z accumulates the rotations, S = Z diag(d) Z^T
  std::vector<double> Z((size_t)m * m, 0.0);
  for (int i = 0; i < m; i++) Z[i + (size_t)m * i] = 1.0;
  for (int l = 0; l < m; l++) {
    for (int iter = 0;; iter++) {
      int mm = l;
      for (; mm + 1 < m; mm++) {  // first negligible subdiagonal entry at or after l
        const double dd = std::fabs(d[mm]) + std::fabs(d[mm + 1]);
        if (std::fabs(e[mm]) <= 1e-16 * dd) break;
      }
      if (mm == l) break;
      if (iter == 100) return false;
      // Wilkinson shift from the leading 2 x 2 block of the unreduced part
      double g = (d[l + 1] - d[l]) / (2.0 * e[l]);
      double r = std::hypot(g, 1.0);
      g = d[mm] - d[l] + e[l] / (g + (g >= 0 ? r : -r));
      double s = 1.0, c = 1.0, pp = 0.0;
      int i = mm - 1;
      bool split = false;
      for (; i >= l; i--) {  // chase the bulge from the bottom of the block up to l
        const double f = s * e[i], b = c * e[i];
        r = std::hypot(f, g);
        e[i + 1] = r;
        if (r == 0.0) {  // the block split: deflate and restart on it
          d[i + 1] -= pp;
          e[mm] = 0.0;
          split = true;
          break;
        }
        s = f / r;
        c = g / r;
        g = d[i + 1] - pp;
        r = (d[i] - g) * s + 2.0 * c * b;
        pp = s * r;
        d[i + 1] = g + pp;
        g = c * r - b;
        for (int k = 0; k < m; k++) {
          const double z1 = Z[k + (size_t)m * (i + 1)], z0 = Z[k + (size_t)m * i];
          Z[k + (size_t)m * (i + 1)] = s * z0 + c * z1;
          Z[k + (size_t)m * i] = c * z0 - s * z1;
        }
      }
      if (split) continue;
      d[l] -= pp;
      e[l] = g;
      e[mm] = 0.0;
    }
  }
  // 4. eigenvectors of A: Q D Z
  V.assign((size_t)m * m, zc(0, 0));
  for (int j = 0; j < m; j++)
    for (int k = 0; k < m; k++) {
      const zc f = ph[k] * Z[k + (size_t)m * j];
      if (f == zc(0, 0)) continue;
      for (int r = 0; r < m; r++) V[r + (size_t)m * j] += Q[r + (size_t)m * k] * f;
    }
  w = d;
  return true;
}

// the Hermitian eigensolver of the Lanczos Rayleigh-Ritz steps: cyclic Jacobi
// up to 32 columns, Householder + QL beyond (x86 host: 0.013 s against 0.5 s at
// 129 columns, 1.0 s against 40 s at 511; eigenvalues agree to ~1e-14 |A|)
void herm_eigh(int m, std::vector<zc> &A, std::vector<zc> &V, std::vector<double> &w) {
  if (m > 32) {
    std::vector<zc> B = A;
    if (tridiag_eigh(m, B, V, w)) return;
  }
  jacobi_eigh(m, A, V, w);
}

// Cholesky G = R^H R of a Hermitian positive definite m x m matrix and the
// inverse of the upper-triangular R (column-major); false if not positive.
bool chol_inv(int m, const std::vector<zc> &G, std::vector<zc> &Rinv) {
  std::vector<zc> R((size_t)m * m, 0.0);
  auto g = [&](int i, int j) { return G[i + (size_t)m * j]; };
  auto r = [&](int i, int j) -> zc & { return R[i + (size_t)m * j]; };
  for (int j = 0; j < m; j++) {
    double d = g(j, j).real();
    for (int k = 0; k < j; k++) d -= std::norm(r(k, j));
    if (!(d > 0)) return false;
    r(j, j) = std::sqrt(d);
    for (int i = j + 1; i < m; i++) {
      zc t = g(j, i);
      for (int k = 0; k < j; k++) t -= std::conj(r(k, j)) * r(k, i);
      r(j, i) = t / r(j, j).real();
    }
  }
  Rinv.assign((size_t)m * m, 0.0);
  for (int j = 0; j < m; j++) {  // solve R x = e_j by back substitution
    for (int i = j; i >= 0; i--) {
      zc t = (i == j) ? zc(1.0) : zc(0.0);
      for (int k = i + 1; k <= j; k++) t -= R[i + (size_t)m * k] * Rinv[k + (size_t)m * j];
      Rinv[i + (size_t)m * j] = t / R[i + (size_t)m * i].real();
    }
  }
  return true;
}

lqcd_status to_host(lqcd_ctx *c, const double2 *d, size_t n, std::vector<zc> &h) {
  h.resize(n);
  LQ_CU(cudaMemcpyAsync(h.data(), d, n * sizeof(double2), cudaMemcpyDeviceToHost, c->stream));
  LQ_CU(cudaStreamSynchronize(c->stream));
  return LQCD_OK;
}

lqcd_status to_dev(lqcd_ctx *c, const std::vector<zc> &h, double2 *d) {
  LQ_CU(cudaMemcpyAsync(d, h.data(), h.size() * sizeof(double2), cudaMemcpyHostToDevice, c->stream));
  LQ_CU(cudaStreamSynchronize(c->stream));
  return LQCD_OK;
}

lqcd_status new_full(lqcd_ctx *c, int nrhs, lqcd_field **f) { return lqcd_field_create(c, LQCD_F64, LQCD_FULL, nrhs, f); }
lqcd_status new_prec(lqcd_ctx *c, lqcd_prec prec, int nrhs, lqcd_field **f) {
  return lqcd_field_create(c, prec, LQCD_FULL, nrhs, f);
}

lqcd_status new_like(lqcd_ctx *c, const lqcd_field *ref, int nrhs, lqcd_field **f) {
  return lqcd_field_create(c, ref->prec, LQCD_FULL, nrhs, f);
}

struct FieldGuard {
  std::vector<lqcd_field *> f;
  ~FieldGuard() {
    for (auto *x : f)
      if (x) lqcd_field_destroy(x);
  }
};

// links of the H_W kernel: all 18 reals for FP64 and DF64, 12 for FP32
int hw_recon(lqcd_prec p) { return (p == LQCD_F64 || p == LQCD_DF64) ? 18 : 12; }

lqcd_status hw(lqcd_ctx *c, int nrhs, lqcd_field *out, const lqcd_field *in) {
  MutField o[2] = {out->mut(0), out->mut(1)};
  FieldRef x[2] = {in->ref(0), in->ref(1)};
  return op_hw(c, out->prec, hw_recon(out->prec), nrhs, o, x, nullptr, 0);
}

// out = t H_W in + c1 z1 + c2 z2 + c3 z3 (a null z drops its term), FULL fields
lqcd_status hw_cheb(lqcd_ctx *c, int nrhs, lqcd_field *out, const lqcd_field *in, double t, const lqcd_field *z1,
                    double c1, const lqcd_field *z2, double c2, const lqcd_field *z3, double c3) {
  MutField o[2] = {out->mut(0), out->mut(1)};
  FieldRef x[2] = {in->ref(0), in->ref(1)};
  const FieldRef none{nullptr, nullptr, 0};
  const lqcd_field *zs[3] = {z1, z2, z3};
  FieldRef z[3][2];
  for (int k = 0; k < 3; k++)
    for (int p = 0; p < 2; p++) z[k][p] = zs[k] ? zs[k]->ref(p) : none;
  const double cz[3] = {z1 ? c1 : 0.0, z2 ? c2 : 0.0, z3 ? c3 : 0.0};
  return op_hw_cheb(c, out->prec, hw_recon(out->prec), nrhs, o, x, t, z, cz);
}

// dst = factor * src converted between precisions (FULL fields, first nrhs RHS)
lqcd_status convert_full(lqcd_ctx *c, lqcd_field *dst, const lqcd_field *src, int nrhs, double factor = 1.0) {
  for (int p = 0; p < 2; p++)
    LQ_CU(convert_spinor(src->prec, dst->prec, c->Vh, nrhs, src->data[p], src->scale[p], src->rhs_words(),
                         dst->data[p], dst->scale[p], dst->rhs_words(), factor, c->stream));
  return LQCD_OK;
}

dim3 fgrid(long n, int nrhs) { return dim3((unsigned)((n + kT - 1) / kT), (unsigned)nrhs, 2); }

lqcd_status clenshaw(lqcd_ctx *c, int nrhs, lqcd_field *o, const lqcd_field *w, const lqcd_field *hh,
                     const lqcd_field *b1, const lqcd_field *b2, double cw, double t, double s2, double s0) {
  const long n = cwords(o);
  if (o->prec == LQCD_F64) {
    auto P = [](const lqcd_field *f, int p) { return f ? (const double2 *)f->data[p] : (const double2 *)nullptr; };
    clenshaw_kernel<double2><<<fgrid(n, nrhs), kT, 0, c->stream>>>(
        n, (double2 *)o->data[0], (double2 *)o->data[1], P(w, 0), P(w, 1), P(hh, 0), P(hh, 1), P(b1, 0), P(b1, 1),
        P(b2, 0), P(b2, 1), cw, t, s2, s0);
  } else if (o->prec == LQCD_F32) {
    auto P = [](const lqcd_field *f, int p) { return f ? (const float2 *)f->data[p] : (const float2 *)nullptr; };
    clenshaw_kernel<float2><<<fgrid(n, nrhs), kT, 0, c->stream>>>(
        n, (float2 *)o->data[0], (float2 *)o->data[1], P(w, 0), P(w, 1), P(hh, 0), P(hh, 1), P(b1, 0), P(b1, 1),
        P(b2, 0), P(b2, 1), cw, t, s2, s0);
  } else {
    return set_error(LQCD_ERR_ARG, "three-term kernel needs FP64 or FP32 fields");
  }
  LQ_CU(cudaGetLastError());
  return LQCD_OK;
}

lqcd_status copy_field(lqcd_ctx *c, lqcd_field *dst, const lqcd_field *src, int nrhs) {
  const size_t bytes = (size_t)cwords(src) * celem(src) * nrhs;
  for (int p = 0; p < 2; p++)
    LQ_CU(cudaMemcpyAsync(dst->data[p], src->data[p], bytes, cudaMemcpyDeviceToDevice, c->stream));
  return LQCD_OK;
}

// per-RHS ||x + c y||^2 (c on the host) into out
lqcd_status axpy_norms(lqcd_ctx *c, const lqcd_field *x, const lqcd_field *y, const std::vector<double> &cf, int nrhs,
                       std::vector<double> &out) {
  if (nrhs > 256) return set_error(LQCD_ERR_ARG, "at most 256 vectors per norm batch");
  LQ_TRY(ensure_partials(c, nrhs));
  double *dc = c->results + 256;
  LQ_CU(cudaMemcpyAsync(dc, cf.data(), sizeof(double) * nrhs, cudaMemcpyHostToDevice, c->stream));
  const long n = cwords(x);
  // grid-stride: at most as many blocks per RHS as the partials hold
  const long gx = std::min<long>(std::min<long>(1024, (2 * n + kT - 1) / kT), (c->Vh + 127) / 128 + 1);
  dim3 g((unsigned)gx, (unsigned)nrhs);
  axpy_norm_kernel<<<g, kT, 0, c->stream>>>(n, (const double2 *)x->data[0], (const double2 *)x->data[1],
                                            (const double2 *)y->data[0], (const double2 *)y->data[1], dc, c->partials,
                                            c->counter, c->results, nrhs);
  LQ_CU(cudaGetLastError());
  out.resize(nrhs);
  LQ_CU(cudaMemcpyAsync(c->h_results, c->results, sizeof(double) * nrhs, cudaMemcpyDeviceToHost, c->stream));
  LQ_CU(cudaStreamSynchronize(c->stream));
  std::memcpy(out.data(), c->h_results, sizeof(double) * nrhs);
  return LQCD_OK;
}

// orthonormalise the first m RHS of X (Cholesky QR), result in X (T scratch)
lqcd_status orthonormalise(lqcd_ctx *c, lqcd_field *&X, lqcd_field *&T, int m) {
  double2 *d;
  LQ_TRY(small_scratch(c, (size_t)m * m, &d));
  std::vector<zc> G, Rinv;
  for (int pass = 0; pass < 2; pass++) {
    LQ_TRY(gram(c, X, m, X, m, d));
    LQ_TRY(to_host(c, d, (size_t)m * m, G));
    if (!chol_inv(m, G, Rinv)) return set_error(LQCD_ERR_NOCONV, "low-mode block lost rank");
    LQ_TRY(to_dev(c, Rinv, d));
    LQ_TRY(rotate(c, X, m, d, m, T, 1.0, 0.0));
    std::swap(X, T);
  }
  return LQCD_OK;
}

// Chebyshev coefficients of 1/sqrt(y) on [a, b], degree n (c[0] halved)
void cheb_coeffs(double a, double b, int n, std::vector<double> &c) {
  const int N = n + 1;
  c.assign(N, 0.0);
  std::vector<double> f(N), th(N);
  for (int j = 0; j < N; j++) {
    th[j] = M_PI * (j + 0.5) / N;
    f[j] = 1.0 / std::sqrt(0.5 * ((b - a) * std::cos(th[j]) + a + b));
  }
  for (int k = 0; k < N; k++) {
    double s = 0;
    for (int j = 0; j < N; j++) s += f[j] * std::cos(k * th[j]);
    c[k] = 2.0 * s / N;
  }
  c[0] *= 0.5;
}

double cheb_eval(double a, double b, const std::vector<double> &c, double y) {
  const double t = (2 * y - a - b) / (b - a);
  double b1 = 0, b2 = 0;
  for (int k = (int)c.size() - 1; k >= 1; k--) {
    const double b0 = c[k] + 2 * t * b1 - b2;
    b2 = b1;
    b1 = b0;
  }
  return c[0] + t * b1 - b2;
}

// sup over x in [sqrt a, sqrt b] of |x P(x^2) - 1|: a fine grid in x plus the nodes
double sign_error(double a, double b, const std::vector<double> &c) {
  const int npts = 50000;
  double worst = 0;
  const double lo = std::sqrt(a), hi = std::sqrt(b);
  for (int i = 0; i < npts; i++) {
    const double x = lo + (hi - lo) * i / (npts - 1);
    worst = std::max(worst, std::fabs(x * cheb_eval(a, b, c, x * x) - 1));
  }
  const int N = (int)c.size();
  for (int j = 0; j < N; j++) {
    const double y = 0.5 * ((b - a) * std::cos(M_PI * (j + 0.5) / N) + a + b);
    worst = std::max(worst, std::fabs(std::sqrt(y) * cheb_eval(a, b, c, y) - 1));
  }
  return worst;
}

// smallest degree <= nmax meeting tol (bisection around the Bernstein estimate)
int cheb_degree(double a, double b, double tol, int nmax, std::vector<double> &c) {
  auto ok = [&](int n) {
    std::vector<double> cc;
    cheb_coeffs(a, b, n, cc);
    return sign_error(a, b, cc) <= tol;
  };
  int hi = std::max(4, (int)(std::log(2.0 / tol) * std::sqrt(b / a) / 2.0 * 1.2));
  while (hi <= nmax && !ok(hi)) hi = (int)(hi * 1.5) + 1;
  if (hi > nmax) {
    if (!ok(nmax)) return -1;
    hi = nmax;
  }
  int lo = 1;
  while (lo < hi) {
    const int mid = (lo + hi) / 2;
    if (ok(mid))
      hi = mid;
    else
      lo = mid + 1;
  }
  cheb_coeffs(a, b, hi, c);
  return hi;
}

// eps(H_W) in -> out (nrhs RHS), FULL fields of one precision (FP64 or FP32)
lqcd_status sign_apply(lqcd_ctx *c, int nrhs, const lqcd_field *in, lqcd_field *out) {
  NvtxRange nv("lqcd sign function");
  OverlapState &S = *c->ov;
  const bool f64 = in->prec == LQCD_F64;
  // the recurrence of an FP64 sign function runs in double-float on request
  const lqcd_prec rp = (f64 && S.df) ? LQCD_DF64 : in->prec;
  FieldGuard g;
  lqcd_field *w, *wr, *b1, *b2, *h, *hh;
  LQ_TRY(new_like(c, in, nrhs, &w));
  g.f.push_back(w);
  for (lqcd_field **q : {&b1, &b2, &h, &hh}) {
    LQ_TRY(new_prec(c, rp, nrhs, q));
    g.f.push_back(*q);
  }
  LQ_TRY(copy_field(c, w, in, nrhs));
  void *proj = nullptr;
  const int nl = S.nlow;
  const lqcd_field *V = f64 ? S.vecs : S.vecs32;
  if (nl > 0) {
    double2 *d;
    LQ_TRY(small_scratch(c, (size_t)nl * nrhs, &d));
    proj = d;
    LQ_TRY(gram(c, V, nl, in, nrhs, proj));             // P = V^H in
    LQ_TRY(rotate(c, V, nl, proj, nrhs, w, -1.0, 1.0));  // w = in - V P
  }
  const double a = S.a, b = S.b;
  const double s2 = 2.0 / (b - a), s0 = -(a + b) / (b - a);
  // an FP32 sign function carries ~1e-6 rounding anyway: its polynomial stops there
  const bool lowdeg = in->prec == LQCD_F32;
  const int n = lowdeg ? S.degree32 : S.degree;
  const std::vector<double> &coef = lowdeg ? S.coef32 : S.coef;
  // b_n = c_n w  (and w in the recurrence's precision)
  if (rp != in->prec) {
    LQ_TRY(new_prec(c, rp, nrhs, &wr));
    g.f.push_back(wr);
    LQ_TRY(convert_full(c, wr, w, nrhs));
    LQ_TRY(convert_full(c, b1, w, nrhs, coef[n]));
  } else {
    wr = w;
    LQ_TRY(clenshaw(c, nrhs, b1, w, w, w, nullptr, coef[n], 0.0, 0.0, 0.0));
  }
  // b_k = c_k w + 2 T b_{k+1} - b_{k+2} (k = n-1 .. 1), then P w = c_0 w + T b_1 - b_2
  // (n = 0: P w = c_0 w = b_0),
  // T = s2 H^2 + s0: the second H_W of each step carries the three-term update
  // in its epilogue; three buffers rotate so no launch writes what it reads
  bool b2_zero = true;
  for (int k = n - 1; k >= 0; k--) {
    const double t = k > 0 ? 2.0 : 1.0;
    LQ_TRY(hw(c, nrhs, h, b1));
    LQ_TRY(hw_cheb(c, nrhs, hh, h, t * s2, wr, coef[k], b1, t * s0, b2_zero ? nullptr : b2, -1.0));
    b2_zero = false;
    lqcd_field *o = hh;
    hh = b2;
    b2 = b1;
    b1 = o;
  }
  if (rp != in->prec) {  // H P(H^2) w, back to FP64
    LQ_TRY(hw(c, nrhs, h, b1));
    LQ_TRY(convert_full(c, out, h, nrhs));
  } else {
    LQ_TRY(hw(c, nrhs, out, b1));  // H P(H^2) w
  }
  if (nl > 0) {
    double *dsg = c->results + 512;
    std::vector<double> sg(nl);
    for (int i = 0; i < nl; i++) sg[i] = S.lam[i] > 0 ? 1.0 : -1.0;
    LQ_CU(cudaMemcpyAsync(dsg, sg.data(), sizeof(double) * nl, cudaMemcpyHostToDevice, c->stream));
    if (f64)
      scale_rows_kernel<double2><<<(nl * nrhs + 255) / 256, 256, 0, c->stream>>>((double2 *)proj, nl, nrhs, dsg);
    else
      scale_rows_kernel<float2><<<(nl * nrhs + 255) / 256, 256, 0, c->stream>>>((float2 *)proj, nl, nrhs, dsg);
    LQ_CU(cudaGetLastError());
    LQ_TRY(rotate(c, V, nl, proj, nrhs, out, 1.0, 1.0));  // += V sign(lam) P
    LQ_CU(cudaStreamSynchronize(c->stream));  // dsg and proj are reused by the next call
  }
  return LQCD_OK;
}

// out = a in + b (g5 e or e) on FULL fields of one precision
lqcd_status combine(lqcd_ctx *c, int nrhs, lqcd_field *out, const lqcd_field *in, const lqcd_field *e, double a,
                    double b, int g5) {
  const long n = cwords(in);
  if (in->prec == LQCD_F64)
    ov_combine_kernel<double2><<<fgrid(n, nrhs), kT, 0, c->stream>>>(
        in->Vh, n, (double2 *)out->data[0], (double2 *)out->data[1], (const double2 *)in->data[0],
        (const double2 *)in->data[1], (const double2 *)e->data[0], (const double2 *)e->data[1], a, b, g5);
  else
    ov_combine_kernel<float2><<<fgrid(n, nrhs), kT, 0, c->stream>>>(
        in->Vh, n, (float2 *)out->data[0], (float2 *)out->data[1], (const float2 *)in->data[0],
        (const float2 *)in->data[1], (const float2 *)e->data[0], (const float2 *)e->data[1], a, b, g5);
  LQ_CU(cudaGetLastError());
  return LQCD_OK;
}

// out = D_ov in = f (in + g5 eps in) + m in, or
// out = D_ov^dag in = f (in + eps g5 in) + m in   (eps Hermitian)
lqcd_status dov_apply(lqcd_ctx *c, int nrhs, const lqcd_field *in, lqcd_field *out, int dagger) {
  OverlapState &S = *c->ov;
  const double rho = S.prm.rho, m = S.prm.mass;
  const double f = (1.0 - m / (2.0 * rho)) * rho;
  FieldGuard g;
  lqcd_field *e;
  LQ_TRY(new_like(c, in, nrhs, &e));
  g.f.push_back(e);
  if (!dagger) {
    LQ_TRY(sign_apply(c, nrhs, in, e));
    LQ_TRY(combine(c, nrhs, out, in, e, f + m, f, 1));
  } else {
    lqcd_field *g5in;
    LQ_TRY(new_like(c, in, nrhs, &g5in));
    g.f.push_back(g5in);
    LQ_TRY(combine(c, nrhs, g5in, in, in, 0.0, 1.0, 1));  // g5 in
    LQ_TRY(sign_apply(c, nrhs, g5in, e));
    LQ_TRY(combine(c, nrhs, out, in, e, f + m, f, 0));
  }
  LQ_CU(cudaStreamSynchronize(c->stream));
  return LQCD_OK;
}

// per-RHS ||v||^2 of a FULL field (any precision), both parities
lqcd_status field_norms(lqcd_ctx *c, const lqcd_field *v, int nrhs, std::vector<double> &out) {
  if (nrhs > 128) return set_error(LQCD_ERR_ARG, "at most 128 vectors per norm batch");
  LQ_TRY(ensure_partials(c, nrhs));
  for (int p = 0; p < 2; p++)
    LQ_CU(blas_norm2(v->prec, c->Vh, nrhs, v->ref(p), c->partials, c->results + 128 * p, 1, c->stream));
  LQ_CU(cudaMemcpyAsync(c->h_results, c->results, sizeof(double) * 256, cudaMemcpyDeviceToHost, c->stream));
  LQ_CU(cudaStreamSynchronize(c->stream));
  out.resize(nrhs);
  for (int k = 0; k < nrhs; k++) out[k] = c->h_results[k] + c->h_results[128 + k];
  return LQCD_OK;
}

// y += f_k x (per-RHS factors on the host), FULL fields, y precision >= x precision
lqcd_status axpy_full(lqcd_ctx *c, lqcd_field *y, const lqcd_field *x, const std::vector<double> &f, int nrhs) {
  double *dfac = c->results + 768;
  LQ_CU(cudaMemcpyAsync(dfac, f.data(), sizeof(double) * nrhs, cudaMemcpyHostToDevice, c->stream));
  for (int par = 0; par < 2; par++)
    LQ_CU(blas_axpy(y->prec, x->prec, c->Vh, nrhs, y->mut(par), x->ref(par), dfac, c->stream));
  LQ_CU(cudaStreamSynchronize(c->stream));
  return LQCD_OK;
}

// y = f_k x (precision conversion included), FULL fields
lqcd_status scale_full(lqcd_ctx *c, lqcd_field *y, const lqcd_field *x, const std::vector<double> &f, int nrhs) {
  double *dfac = c->results + 768;
  LQ_CU(cudaMemcpyAsync(dfac, f.data(), sizeof(double) * nrhs, cudaMemcpyHostToDevice, c->stream));
  for (int par = 0; par < 2; par++)
    LQ_CU(blas_scale(y->prec, x->prec, c->Vh, nrhs, y->mut(par), x->ref(par), dfac, c->stream));
  LQ_CU(cudaStreamSynchronize(c->stream));
  return LQCD_OK;
}

// CG on the normal equations of D_ov x = b, FP64 throughout (x0 = 0)
lqcd_status ov_cgls_fp64(lqcd_ctx *c, int nrhs, const lqcd_field *b, lqcd_field *x, const lqcd_solve_params *cg,
                         lqcd_solve_info *inf, const std::vector<double> &bn2) {
  FieldGuard g;
  lqcd_field *r, *s, *p, *q;
  for (lqcd_field **f : {&r, &s, &p, &q}) {
    LQ_TRY(new_full(c, nrhs, f));
    g.f.push_back(*f);
  }
  const size_t bytes = (size_t)cwords(b) * 16 * nrhs;
  for (int par = 0; par < 2; par++) LQ_CU(cudaMemsetAsync(x->data[par], 0, bytes, c->stream));
  LQ_TRY(copy_field(c, r, b, nrhs));
  std::vector<double> gam, qq, rr;
  LQ_TRY(dov_apply(c, nrhs, r, s, 1));
  LQ_TRY(copy_field(c, p, s, nrhs));
  LQ_TRY(field_norms(c, s, nrhs, gam));
  std::vector<char> active(nrhs, 1);
  int it = 0;
  for (; it < cg->max_iter; it++) {
    LQ_TRY(dov_apply(c, nrhs, p, q, 0));
    LQ_TRY(field_norms(c, q, nrhs, qq));
    std::vector<double> al(nrhs), nal(nrhs);
    for (int k = 0; k < nrhs; k++) {
      al[k] = active[k] && qq[k] > 0 ? gam[k] / qq[k] : 0.0;
      nal[k] = -al[k];
    }
    LQ_TRY(axpy_full(c, x, p, al, nrhs));
    LQ_TRY(axpy_full(c, r, q, nal, nrhs));
    LQ_TRY(field_norms(c, r, nrhs, rr));
    bool all = true;
    for (int k = 0; k < nrhs; k++) {
      if (!(rr[k] == rr[k])) return set_error(LQCD_ERR_NOCONV, "overlap CG residual is NaN");
      if (active[k] && rr[k] <= std::pow(0.5 * cg->tol, 2) * bn2[k]) active[k] = 0;
      all &= !active[k];
    }
    if (all) {
      it++;
      break;
    }
    LQ_TRY(dov_apply(c, nrhs, r, s, 1));
    std::vector<double> gn, be(nrhs), one(nrhs);
    LQ_TRY(field_norms(c, s, nrhs, gn));
    for (int k = 0; k < nrhs; k++) {
      be[k] = active[k] && gam[k] > 0 ? gn[k] / gam[k] : 1.0;
      one[k] = active[k] ? 1.0 : 0.0;
      if (active[k]) gam[k] = gn[k];
    }
    LQ_TRY(scale_full(c, p, p, be, nrhs));
    LQ_TRY(axpy_full(c, p, s, one, nrhs));
  }
  inf->iters = it;
  inf->mhat_applies += 2.0 * it + 1;
  return LQCD_OK;
}

// Mixed precision: CG on the normal equations of D_ov with FP32 storage and
// arithmetic (FP32 sign function) on the residual normalised to 1; the FP64
// solution absorbs the inner one and the residual is recomputed with the FP64
// operator when every active inner residual fell below delta or reached its
// target (a right-hand side that reached it is parked: it stops updating
// until the FP64 check), or one stagnated (no 4x drop of |r|^2 in
// kOvStallIters iterations) or grew 20 % past its best.  The update is accepted only if it lowers the FP64
// residual; the search direction is kept across accepted updates, rescaled,
// and CG restarts from p = s after a rejected, grown or stagnated one (the
// same policy as the Wilson-clover mixed solver).
constexpr int kOvStallIters = 48;

lqcd_status copy_rhs(lqcd_ctx *c, lqcd_field *dst, const lqcd_field *src, int k) {
  const size_t bytes = (size_t)cwords(src) * celem(src);
  for (int p = 0; p < 2; p++)
    LQ_CU(cudaMemcpyAsync(static_cast<char *>(dst->data[p]) + bytes * k,
                          static_cast<const char *>(src->data[p]) + bytes * k, bytes, cudaMemcpyDeviceToDevice,
                          c->stream));
  return LQCD_OK;
}

lqcd_status deflate(lqcd_ctx *c, int nrhs, lqcd_field *r, lqcd_field *x, bool x_zero, const std::vector<char> &mask);

// deflate: with the context's eigensystem, each accepted reliable update also
// adds the exact low-mode part of the correction for the new FP64 residual
// (no operator application; the inner FP32 iteration restarts from that
// residual, whose low modes its rounding and FP32 sign function would
// otherwise bring back); the next update's FP64 residual checks it
lqcd_status ov_cgls_mixed(lqcd_ctx *c, int nrhs, const lqcd_field *b, lqcd_field *x, const lqcd_solve_params *cg,
                          lqcd_solve_info *inf, const std::vector<double> &bn2, bool deflated = false) {
  FieldGuard g;
  lqcd_field *r64, *t64, *xtry, *xlo, *r, *s, *p, *q;
  for (lqcd_field **f : {&r64, &t64, &xtry}) {
    LQ_TRY(new_full(c, nrhs, f));
    g.f.push_back(*f);
  }
  for (lqcd_field **f : {&xlo, &r, &s, &p, &q}) {
    LQ_TRY(lqcd_field_create(c, LQCD_F32, LQCD_FULL, nrhs, f));
    g.f.push_back(*f);
  }
  const double delta = (cg->delta > 0 && cg->delta < 1) ? cg->delta : 0.1;
  const size_t bytes64 = (size_t)cwords(b) * 16 * nrhs, bytes32 = (size_t)cwords(b) * 8 * nrhs;
  for (int par = 0; par < 2; par++) {
    LQ_CU(cudaMemsetAsync(x->data[par], 0, bytes64, c->stream));
    LQ_CU(cudaMemsetAsync(xlo->data[par], 0, bytes32, c->stream));
  }
  std::vector<double> target(nrhs), sigma(nrhs), inv(nrhs), gam, qq, rr, best(nrhs, 1.0), ref(nrhs, 1.0);
  std::vector<int> stall(nrhs, 0);
  std::vector<char> active(nrhs, 1), grown(nrhs, 0), parked(nrhs, 0);
  for (int k = 0; k < nrhs; k++) {
    target[k] = 0.5 * cg->tol * std::sqrt(bn2[k]);
    sigma[k] = std::sqrt(bn2[k]);
    inv[k] = 1.0 / sigma[k];
  }
  LQ_TRY(copy_field(c, r64, b, nrhs));
  LQ_TRY(scale_full(c, r, r64, inv, nrhs));
  LQ_TRY(dov_apply(c, nrhs, r, s, 1));
  LQ_TRY(copy_field(c, p, s, nrhs));
  LQ_TRY(field_norms(c, s, nrhs, gam));
  int it = 0;
  bool done = false;
  while (!done && it < cg->max_iter) {
    LQ_TRY(dov_apply(c, nrhs, p, q, 0));
    LQ_TRY(field_norms(c, q, nrhs, qq));
    std::vector<double> al(nrhs), nal(nrhs);
    for (int k = 0; k < nrhs; k++) {
      al[k] = active[k] && !parked[k] && qq[k] > 0 ? gam[k] / qq[k] : 0.0;
      nal[k] = -al[k];
    }
    LQ_TRY(axpy_full(c, xlo, p, al, nrhs));
    LQ_TRY(axpy_full(c, r, q, nal, nrhs));
    LQ_TRY(field_norms(c, r, nrhs, rr));
    it++;
    bool all_dropped = true, trigger = false;
    for (int k = 0; k < nrhs; k++) {
      if (!active[k] || parked[k]) continue;
      if (!(rr[k] == rr[k])) return set_error(LQCD_ERR_NOCONV, "overlap inner residual is NaN");
      if (sigma[k] * std::sqrt(rr[k]) <= target[k]) {
        parked[k] = 1;  // waits, unchanged, for the next FP64 update to confirm it
        continue;
      }
      if (rr[k] < best[k]) best[k] = rr[k];
      if (rr[k] < 0.25 * ref[k]) {
        ref[k] = rr[k];
        stall[k] = 0;
      } else if (++stall[k] >= kOvStallIters) {
        trigger = true;
      }
      if (rr[k] > 1.44 * best[k]) {
        grown[k] = 1;
        trigger = true;
      }
      if (!(best[k] <= delta * delta)) all_dropped = false;
    }
    if (all_dropped || trigger || it >= cg->max_iter) {
      // reliable update in FP64: x_try = x + sigma x_lo, r_try = b - D_ov x_try
      std::vector<double> fx(nrhs), r2;
      for (int k = 0; k < nrhs; k++) fx[k] = active[k] ? sigma[k] : 0.0;
      LQ_TRY(copy_field(c, xtry, x, nrhs));
      LQ_TRY(axpy_full(c, xtry, xlo, fx, nrhs));
      for (int par = 0; par < 2; par++) LQ_CU(cudaMemsetAsync(xlo->data[par], 0, bytes32, c->stream));
      LQ_TRY(dov_apply(c, nrhs, xtry, t64, 0));
      LQ_TRY(combine(c, nrhs, t64, b, t64, 1.0, -1.0, 0));  // element-wise, in place
      LQ_TRY(field_norms(c, t64, nrhs, r2));
      inf->reliable_updates++;
      inf->mhat_applies += 1;
      done = true;
      std::vector<double> fp(nrhs, 0.0), fr(nrhs, 0.0), fs(nrhs, 0.0);
      for (int k = 0; k < nrhs; k++) {
        if (!active[k]) continue;
        const double snew = std::sqrt(r2[k]);
        if (!(snew == snew) || std::isinf(snew)) return set_error(LQCD_ERR_NOCONV, "overlap FP64 residual is not finite");
        const bool accept = snew < sigma[k];
        if (accept) {
          LQ_TRY(copy_rhs(c, x, xtry, k));
          LQ_TRY(copy_rhs(c, r64, t64, k));
          if (snew <= target[k]) {
            active[k] = 0;
            continue;
          }
        }
        done = false;
        const bool restart = !accept || grown[k] || parked[k] || stall[k] >= kOvStallIters;
        const double snext = accept ? snew : sigma[k];
        fp[k] = restart ? 0.0 : sigma[k] / snext;
        fs[k] = restart ? 1.0 : 0.0;
        fr[k] = 1.0 / snext;
        sigma[k] = snext;
        best[k] = ref[k] = 1.0;
        stall[k] = 0;
        grown[k] = 0;
        parked[k] = 0;
      }
      if (done) break;
      if (deflated) {
        std::vector<char> mask(nrhs, 0);
        for (int k = 0; k < nrhs; k++) mask[k] = active[k] && fr[k] > 0;
        LQ_TRY(deflate(c, nrhs, r64, x, false, mask));
      }
      LQ_TRY(scale_full(c, p, p, fp, nrhs));
      LQ_TRY(scale_full(c, r, r64, fr, nrhs));
      LQ_TRY(dov_apply(c, nrhs, r, s, 1));
      std::vector<double> gn;
      LQ_TRY(field_norms(c, s, nrhs, gn));
      for (int k = 0; k < nrhs; k++)
        if (active[k]) gam[k] = gn[k];
      LQ_TRY(axpy_full(c, p, s, fs, nrhs));
      continue;
    }
    LQ_TRY(dov_apply(c, nrhs, r, s, 1));
    std::vector<double> gn, be(nrhs), one(nrhs);
    LQ_TRY(field_norms(c, s, nrhs, gn));
    for (int k = 0; k < nrhs; k++) {
      const bool on = active[k] && !parked[k];
      be[k] = on && gam[k] > 0 ? gn[k] / gam[k] : 1.0;
      one[k] = on ? 1.0 : 0.0;
      if (on) gam[k] = gn[k];
    }
    LQ_TRY(scale_full(c, p, p, be, nrhs));
    LQ_TRY(axpy_full(c, p, s, one, nrhs));
  }
  inf->iters = it;
  return LQCD_OK;
}

}  // namespace

}  // namespace lqcd

using namespace lqcd;

namespace lqcd {
namespace {

// ---- thick-restart Lanczos on H_W^2 -------------------------------------------
// The smallest eigenpairs of H_W^2 by the thick-restart Lanczos method (Wu and
// Simon, SIAM J. Matrix Anal. Appl. 22 (2000) 602).  A Lanczos basis V of up
// to mmax vectors is built one vector at a time, each new H_W^2 v_j made
// orthogonal to all of V by two passes of classical Gram-Schmidt (so the
// projected matrix is the Gram coefficients, tridiagonal up to rounding).
// At a restart the kkeep smallest Ritz vectors and the last Lanczos vector
// v_m are kept: H_W^2 V_k = V_k diag(theta) + beta_m v_m e_m^T Y_k, so the
// new projected matrix is diag(theta) bordered by beta_m Y_{m-1,i} (an
// arrowhead) and the recursion continues from v_m.  The residual of Ritz
// pair i is beta_m |Y_{m-1,i}|.  Against block subspace iteration with a
// fixed Chebyshev filter this adapts its polynomial to the spectrum and
// applies H_W^2 to one vector per step instead of a whole block per filter
// degree.  H_W^2 runs in FP64 or double-float; the basis, the Gram
// coefficients and the rotations are FP64 (the library's own Gram and rotation kernels).
struct LanczosResult {
  int kneed = 0, cycles = 0;
  long applies = 0;
  bool converged = false;
};

// dst columns kd .. kd + n - 1 = src columns ks .. (same precision)
lqcd_status copy_col_range(lqcd_ctx *c, lqcd_field *dst, int kd, const lqcd_field *src, int ks, int n) {
  const size_t bytes = (size_t)cwords(src) * celem(src);
  for (int p = 0; p < 2; p++)
    LQ_CU(cudaMemcpyAsync(static_cast<char *>(dst->data[p]) + bytes * kd,
                          static_cast<const char *>(src->data[p]) + bytes * ks, bytes * n, cudaMemcpyDeviceToDevice,
                          c->stream));
  return LQCD_OK;
}

// dst column kd = src column ks (same precision)
lqcd_status copy_col(lqcd_ctx *c, lqcd_field *dst, int kd, const lqcd_field *src, int ks) {
  const size_t bytes = (size_t)cwords(src) * celem(src);
  for (int p = 0; p < 2; p++)
    LQ_CU(cudaMemcpyAsync(static_cast<char *>(dst->data[p]) + bytes * kd,
                          static_cast<const char *>(src->data[p]) + bytes * ks, bytes, cudaMemcpyDeviceToDevice,
                          c->stream));
  return LQCD_OK;
}

// ---- double-float kernels of the Lanczos Gram-Schmidt ------------------------
// The basis is a DF64 field: each complex number one float4 {re.hi, re.lo,
// im.hi, im.lo}, columns of cwords complex numbers per parity.  GB300 runs
// FP64 multiply-adds at 1/64 of its FP32 rate, which made FP64 projections
// against the basis (ZGEMV) ~5 ms per Lanczos step; in double-float on the
// FP32 pipes they are bound by the basis' bytes.  Elements are indexed over
// both parities: e < n is parity 0, e - n parity 1.
constexpr int kLzT = 256;
constexpr int kLzMaxP = 512;  // basis columns a kernel can take (mmax + 1 <= 512)

struct dfc {
  df re, im;
};
__device__ __forceinline__ dfc lz_load(const float4 *p0, const float4 *p1, long n, long cs, int k, long e) {
  const float4 v = e < n ? p0[(long)k * cs + e] : p1[(long)k * cs + e - n];
  return dfc{df(v.x, v.y), df(v.z, v.w)};
}
__device__ __forceinline__ void lz_store(float4 *p0, float4 *p1, long n, long cs, int k, long e, dfc a) {
  const float4 v = make_float4(a.re.hi, a.re.lo, a.im.hi, a.im.lo);
  if (e < n)
    p0[(long)k * cs + e] = v;
  else
    p1[(long)k * cs + e - n] = v;
}

// partials of <V_k, w> = sum conj(V_k) w: grid (gx, p), quantities 2k (re), 2k+1 (im)
__global__ void __launch_bounds__(kLzT) lz_dots_kernel(long n, long cs, const float4 *V0, const float4 *V1,
                                                        const float4 *w0, const float4 *w1, double *partials) {
  const int k = blockIdx.y;
  dfacc re{0.0f, 0.0f}, im{0.0f, 0.0f};
  for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < 2 * n; e += (long)gridDim.x * blockDim.x) {
    const dfc v = lz_load(V0, V1, n, cs, k, e), w = lz_load(w0, w1, n, 0, 0, e);
    dfacc_madd(re, v.re, w.re);
    dfacc_madd(re, v.im, w.im);
    dfacc_madd(im, v.re, w.im);
    dfacc_madd(im, -v.im, w.re);
  }
  const df vals[2] = {dfacc_value(re), dfacc_value(im)};
  block_partials<2>(vals, partials, 2 * k);
}

// w -= sum_{k < p} V_k h_k (h: p complex doubles on the device)
__global__ void __launch_bounds__(kLzT) lz_sub_kernel(long n, long cs, int p, const float4 *V0, const float4 *V1,
                                                       const double2 *h, float4 *w0, float4 *w1) {
  __shared__ dfc hs[kLzMaxP];
  for (int k = threadIdx.x; k < p; k += blockDim.x) hs[k] = dfc{df(h[k].x), df(h[k].y)};
  __syncthreads();
  for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < 2 * n; e += (long)gridDim.x * blockDim.x) {
    dfc a = lz_load(w0, w1, n, 0, 0, e);
    for (int k = 0; k < p; k++) {
      const dfc v = lz_load(V0, V1, n, cs, k, e);
      a.re = fma(-v.re, hs[k].re, a.re);
      a.re = fma(v.im, hs[k].im, a.re);
      a.im = fma(-v.re, hs[k].im, a.im);
      a.im = fma(-v.im, hs[k].re, a.im);
    }
    lz_store(w0, w1, n, 0, 0, e, a);
  }
}

// Z_q = sum_{l < p} V_l M_{l q} for q < nq (M: p x nq complex doubles, column-major, on the
// device); grid (nq, element chunks, grid-stride) so the blocks of one chunk share its basis
// rows in L2
__global__ void __launch_bounds__(kLzT) lz_rotate_kernel(long n, long cs, int p, const float4 *V0, const float4 *V1,
                                                          const double2 *M, float4 *Z0, float4 *Z1) {
  __shared__ dfc ms[kLzMaxP];
  const int q = blockIdx.x;
  for (int l = threadIdx.x; l < p; l += blockDim.x) ms[l] = dfc{df(M[l + (long)p * q].x), df(M[l + (long)p * q].y)};
  __syncthreads();
  for (long e = (long)blockIdx.y * blockDim.x + threadIdx.x; e < 2 * n; e += (long)gridDim.y * blockDim.x) {
    dfacc re{0.0f, 0.0f}, im{0.0f, 0.0f};
    for (int l = 0; l < p; l++) {
      const dfc v = lz_load(V0, V1, n, cs, l, e);
      dfacc_madd(re, v.re, ms[l].re);
      dfacc_madd(re, -v.im, ms[l].im);
      dfacc_madd(im, v.re, ms[l].im);
      dfacc_madd(im, v.im, ms[l].re);
    }
    lz_store(Z0, Z1, n, cs, q, e, dfc{dfacc_value(re), dfacc_value(im)});
  }
}

// w *= 1 / sqrt(n2[0]) (n2[0] = |w|^2 from the dots kernel)
__global__ void __launch_bounds__(kLzT) lz_normalise_kernel(long n, const double *n2, float4 *w0, float4 *w1) {
  const df f(1.0 / sqrt(n2[0]));
  for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < 2 * n; e += (long)gridDim.x * blockDim.x) {
    dfc a = lz_load(w0, w1, n, 0, 0, e);
    a.re = a.re * f;
    a.im = a.im * f;
    lz_store(w0, w1, n, 0, 0, e, a);
  }
}

struct LzOps {
  lqcd_ctx *c;
  long n;   // complex numbers per column and parity
  long gx;  // blocks of the grid-stride kernels (the partials of the dots kernel)
  const float4 *cp(const lqcd_field *f, int par) const { return reinterpret_cast<const float4 *>(f->data[par]); }
  float4 *mp(lqcd_field *f, int par) const { return reinterpret_cast<float4 *>(f->data[par]); }
  // out[2k], out[2k+1] = <V_k, w> for k < p (device doubles)
  lqcd_status dots(const lqcd_field *V, int p, const lqcd_field *w, double *out) const {
    lz_dots_kernel<<<dim3((unsigned)gx, (unsigned)p), kLzT, 0, c->stream>>>(n, n, cp(V, 0), cp(V, 1), cp(w, 0), cp(w, 1),
                                                                             c->partials);
    LQ_CU(cudaGetLastError());
    LQ_CU(finish_reduce(c->partials, (int)gx, 2 * p, out, 1, c->stream));
    return LQCD_OK;
  }
  lqcd_status sub(const lqcd_field *V, int p, const double *h, lqcd_field *w) const {
    lz_sub_kernel<<<(unsigned)gx, kLzT, 0, c->stream>>>(n, n, p, cp(V, 0), cp(V, 1), (const double2 *)h, mp(w, 0),
                                                         mp(w, 1));
    LQ_CU(cudaGetLastError());
    return LQCD_OK;
  }
  lqcd_status rotate(const lqcd_field *V, int p, const double2 *M, int nq, lqcd_field *Z) const {
    const long chunks = std::min<long>((2 * n + kLzT - 1) / kLzT, 65535);
    lz_rotate_kernel<<<dim3((unsigned)nq, (unsigned)chunks), kLzT, 0, c->stream>>>(
        n, n, p, cp(V, 0), cp(V, 1), M, mp(Z, 0), mp(Z, 1));
    LQ_CU(cudaGetLastError());
    return LQCD_OK;
  }
  lqcd_status normalise(const double *n2, lqcd_field *w) const {
    lz_normalise_kernel<<<(unsigned)gx, kLzT, 0, c->stream>>>(n, n2, mp(w, 0), mp(w, 1));
    LQ_CU(cudaGetLastError());
    return LQCD_OK;
  }
};

// A Hermitian operator for the thick-restart Lanczos: w = A x on single
// double-float columns, `per_call` operator applications counted per call;
// `start` (may be empty) maps the FP64 random start vector into the subspace
// A acts on (a chirality sector, say) before it is normalised.
struct LzSpec {
  std::function<lqcd_status(lqcd_field *x, lqcd_field *w)> apply;
  int per_call = 1;
  std::function<lqcd_status(lqcd_field *x64)> start;
  double tol = 1e-10;    // Ritz residual estimate beta_m |q_{m,i}| of each wanted pair
  int max_cycles = 100;  // restart cycles
  unsigned long long seed = 1;
};

// Thick-restart Lanczos for the lowest eigenpairs of a Hermitian operator:
// X (FP64 FULL, >= kkeep columns) receives the kneed lowest Ritz vectors
// (kneed >= want: a cluster straddling the want-th value is kept whole) and
// ritz (may be NULL) their Ritz values.
lqcd_status lanczos_lowest(lqcd_ctx *c, const LzSpec &sp, int want, int kkeep, int mmax, lqcd_field *X, FieldGuard &g,
                           LanczosResult &out, std::vector<double> *ritz) {
  if (mmax + 1 > kLzMaxP) return set_error(LQCD_ERR_ARG, "Lanczos basis of %d vectors too large", mmax + 1);
  // the basis and the vector the operator acts on in double-float
  lqcd_field *V, *V2, *xd, *wd, *x64 = nullptr;
  for (lqcd_field **f : {&V, &V2}) {
    LQ_TRY(lqcd_field_create(c, LQCD_DF64, LQCD_FULL, mmax + 1, f));
    g.f.push_back(*f);
  }
  for (lqcd_field **f : {&xd, &wd}) {
    LQ_TRY(lqcd_field_create(c, LQCD_DF64, LQCD_FULL, 1, f));
    g.f.push_back(*f);
  }
  LQ_TRY(new_full(c, 1, &x64));
  g.f.push_back(x64);
  const long n = cwords(V);
  const long gx = std::min<long>((2 * n + kLzT - 1) / kLzT, (c->Vh + 31) / 32);
  LQ_TRY(ensure_partials(c, 2 * (mmax + 1)));
  const LzOps ops{c, n, gx};
  // random unit start vector (FP64 Gaussian, converted)
  {
    const long nd = 2L * n;
    for (int p = 0; p < 2; p++) {
      gauss_fill_kernel<<<(unsigned)((nd / 2 + kT - 1) / kT), kT, 0, c->stream>>>((double *)x64->data[p], nd,
                                                                                   sp.seed * 2 + p + 1);
      LQ_CU(cudaGetLastError());
    }
    if (sp.start) LQ_TRY(sp.start(x64));
    std::vector<double> n2;
    LQ_TRY(field_norms(c, x64, 1, n2));
    LQ_TRY(convert_full(c, wd, x64, 1, 1.0 / std::sqrt(n2[0])));
    LQ_TRY(copy_col(c, V, 0, wd, 0));
  }
  const int ld = mmax + 1;
  std::vector<zc> Hm((size_t)ld * mmax, zc(0, 0));
  double2 *d;
  LQ_TRY(small_scratch(c, (size_t)(mmax + 1) * mmax + 2 * (size_t)(mmax + 1) + 1, &d));
  double2 *dh1 = d + (size_t)(mmax + 1) * mmax, *dh2 = dh1 + (mmax + 1), *dn = dh2 + (mmax + 1);
  // pinned host copies of one step's coefficients and norm: one sync per step
  struct Pinned {
    double2 *h = nullptr;
    ~Pinned() {
      if (h) cudaFreeHost(h);
    }
  } hp;
  if (cudaMallocHost(&hp.h, sizeof(double2) * (2 * (size_t)(mmax + 1) + 1)) != cudaSuccess) {
    cudaGetLastError();
    return set_error(LQCD_ERR_OOM, "cannot allocate Lanczos host scratch");
  }
  int j0 = 0;
  for (;;) {
    for (int j = j0; j < mmax; j++) {
      // w = A v_j
      LQ_TRY(copy_col(c, xd, 0, V, j));
      LQ_TRY(sp.apply(xd, wd));
      out.applies += sp.per_call;
      // two passes of classical Gram-Schmidt against v_0 .. v_j, then
      // v_{j+1} = w / |w|, all on the stream; the host reads the
      // coefficients and |w|^2 once
      LQ_TRY(ops.dots(V, j + 1, wd, (double *)dh1));
      LQ_TRY(ops.sub(V, j + 1, (const double *)dh1, wd));
      LQ_TRY(ops.dots(V, j + 1, wd, (double *)dh2));
      LQ_TRY(ops.sub(V, j + 1, (const double *)dh2, wd));
      LQ_TRY(ops.dots(wd, 1, wd, (double *)dn));
      LQ_TRY(ops.normalise((const double *)dn, wd));
      LQ_TRY(copy_col(c, V, j + 1, wd, 0));
      LQ_CU(cudaMemcpyAsync(hp.h, dh1, sizeof(double2) * (2 * (size_t)(mmax + 1) + 1), cudaMemcpyDeviceToHost,
                            c->stream));
      LQ_CU(cudaStreamSynchronize(c->stream));
      const double beta = std::sqrt(hp.h[2 * (size_t)(mmax + 1)].x);
      if (!(beta > 1e-13)) return set_error(LQCD_ERR_NOCONV, "Lanczos breakdown at step %d (beta %.3e)", j, beta);
      for (int i = 0; i <= j; i++)
        Hm[i + (size_t)ld * j] = zc(hp.h[i].x + hp.h[mmax + 1 + i].x, hp.h[i].y + hp.h[mmax + 1 + i].y);
      Hm[j + 1 + (size_t)ld * j] = beta;
    }
    out.cycles++;
    // Ritz pairs of the (Hermitian part of the) mmax x mmax projected matrix
    const int m = mmax;
    std::vector<zc> W((size_t)m * m), Q;
    for (int jj = 0; jj < m; jj++)
      for (int i = 0; i < m; i++) W[i + (size_t)m * jj] = Hm[i + (size_t)ld * jj];
    for (int jj = 0; jj < m; jj++)
      for (int i = 0; i < jj; i++) {
        const zc avg = 0.5 * (W[i + (size_t)m * jj] + std::conj(W[jj + (size_t)m * i]));
        W[i + (size_t)m * jj] = avg;
        W[jj + (size_t)m * i] = std::conj(avg);
      }
    std::vector<double> mu;
    herm_eigh(m, W, Q, mu);
    std::vector<int> order(m);
    for (int i = 0; i < m; i++) order[i] = i;
    std::sort(order.begin(), order.end(), [&](int x, int y) { return mu[x] < mu[y]; });
    std::vector<zc> Qs((size_t)m * m);
    std::vector<double> mus(m);
    for (int jj = 0; jj < m; jj++) {
      mus[jj] = mu[order[jj]];
      for (int i = 0; i < m; i++) Qs[i + (size_t)m * jj] = Q[i + (size_t)m * order[jj]];
    }
    const double beta_m = Hm[m + (size_t)ld * (m - 1)].real();
    int kneed = want;
    while (kneed < kkeep - 4 && mus[kneed] <= 1.01 * mus[want - 1]) kneed++;
    bool conv = true;
    double worst = 0;
    for (int i = 0; i < kneed; i++) {
      const double r = beta_m * std::abs(Qs[m - 1 + (size_t)m * i]);
      worst = std::max(worst, r);
      conv &= r <= sp.tol;
    }
    if (kOvTrace)
      std::fprintf(stderr, "lqcd overlap: Lanczos cycle %d worst %.3e kneed %d mu[kneed-1] %.6f mu[kkeep-1] %.6f\n",
                   out.cycles, worst, kneed, mus[kneed - 1], mus[kkeep - 1]);
    LQ_TRY(to_dev(c, Qs, d));
    if (conv || out.cycles >= sp.max_cycles) {
      LQ_TRY(ops.rotate(V, m, d, kneed, V2));
      LQ_TRY(convert_full(c, X, V2, kneed));
      out.kneed = kneed;
      out.converged = conv;
      if (ritz) ritz->assign(mus.begin(), mus.begin() + kneed);
      return LQCD_OK;
    }
    // thick restart: V2 = [V Q_k, v_m]; projected matrix diag(theta) bordered by beta_m Q_{m-1,i}
    LQ_TRY(ops.rotate(V, m, d, kkeep, V2));
    LQ_TRY(copy_col(c, V2, kkeep, V, m));
    std::swap(V, V2);
    std::fill(Hm.begin(), Hm.end(), zc(0, 0));
    for (int i = 0; i < kkeep; i++) {
      Hm[i + (size_t)ld * i] = mus[i];
      Hm[kkeep + (size_t)ld * i] = beta_m * Qs[m - 1 + (size_t)m * i];
    }
    j0 = kkeep;
  }
}

// X (FP64 FULL, >= kkeep columns) receives the kneed lowest Ritz vectors of H_W^2
lqcd_status lowmodes_lanczos(lqcd_ctx *c, const lqcd_overlap_params *prm, int want, int kkeep, int mmax,
                             lqcd_field *X, FieldGuard &g, LanczosResult &out) {
  OverlapState &S = *c->ov;
  lqcd_field *td, *x64, *t64;
  LQ_TRY(lqcd_field_create(c, LQCD_DF64, LQCD_FULL, 1, &td));
  g.f.push_back(td);
  LQ_TRY(new_full(c, 1, &x64));
  g.f.push_back(x64);
  LQ_TRY(new_full(c, 1, &t64));
  g.f.push_back(t64);
  LzSpec sp;
  sp.per_call = 2;
  sp.tol = prm->eig_tol;
  sp.max_cycles = prm->max_filter;
  sp.seed = prm->seed;
  sp.apply = [&](lqcd_field *xd, lqcd_field *wd) -> lqcd_status {
    if (S.df) {  // H_W in double-float
      LQ_TRY(hw(c, 1, td, xd));
      return hw(c, 1, wd, td);
    }
    LQ_TRY(convert_full(c, x64, xd, 1));
    LQ_TRY(hw(c, 1, t64, x64));
    LQ_TRY(hw(c, 1, x64, t64));
    return convert_full(c, wd, x64, 1);
  };
  return lanczos_lowest(c, sp, want, kkeep, mmax, X, g, out, nullptr);
}


// ---- the overlap eigensystem and the deflated overlap CG -------------------

// columns [k0, k0 + n) of a FULL field as a field of its own (no ownership)
lqcd_field col_view(const lqcd_field *f, int k0, int n) {
  lqcd_field v = *f;
  for (int p = 0; p < 2; p++) v.data[p] = col(f, p, k0);
  for (int p = 0; p < 2; p++) v.scale[p] = nullptr;
  v.nrhs = n;
  v.alloc = nullptr;
  v.scale_alloc = nullptr;
  return v;
}

// keep chirality sector s (g5 = diag(1, 1, -1, -1): s = +1 spins 0, 1, s = -1
// spins 2, 3) of the first nrhs columns of a FULL FP64 or double-float field:
// a column's spins 0, 1 are its complex words 0-5, spins 2, 3 words 6-11
lqcd_status chiral_project(lqcd_ctx *c, lqcd_field *f, int nrhs, int sector) {
  if (celem(f) != 16) return set_error(LQCD_ERR_ARG, "chiral projection of a field of precision %d", (int)f->prec);
  const size_t half = 6 * (size_t)f->Vh * 16, colb = (size_t)cwords(f) * 16;
  for (int p = 0; p < 2; p++)
    LQ_CU(cudaMemset2DAsync(static_cast<char *>(f->data[p]) + (sector > 0 ? half : 0), colb, 0, half, nrhs,
                            c->stream));
  return LQCD_OK;
}

// Deflation with the kept eigensystem.  D_ov(0) maps each pair span{chi, eta}
// into itself: with eps chi = c chi + n eta (c = <chi, eps chi>, n = |P_-s eps
// chi|), g5 = s on chi's sector and -s on eta's,
//   D_ov(0) chi = rho ((1 + s c) chi - s n eta),  D_ov(0) eta = rho (s n chi + (1 + s c) eta),
// so D(m) = a D_ov(0) + m (a = 1 - m / (2 rho)) is the real 2 x 2 matrix
// M = [[A, B], [-B, A]], A = a rho (1 + s c) + m, B = a rho s n, on it (1 x 1,
// A, for an unpaired chi) and M^T M = mu' = A^2 + B^2.  For a residual r the
// least-squares correction in the span is x_W = W M^T (W^H r) / mu' and
// D(m) x_W = W (W^H r): x += x_W and r -= W (W^H r) need one Gram product and
// two rotations, no operator application.  Columns k with mask[k] = 0 are left
// alone; a massless zero mode (mu' = 0) is not deflated.
lqcd_status deflate(lqcd_ctx *c, int nrhs, lqcd_field *r, lqcd_field *x, bool x_zero, const std::vector<char> &mask) {
  OverlapState &S = *c->ov;
  const int nw = S.ev_n + S.ev_np, sg = S.ev_sector;
  const double rho = S.prm.rho, m = S.prm.mass, a = 1.0 - m / (2.0 * rho);
  double2 *d;
  LQ_TRY(small_scratch(c, (size_t)nw * nrhs, &d));
  LQ_TRY(gram(c, S.ev, nw, r, nrhs, d));  // G = W^H r, nw x nrhs
  std::vector<zc> G, Z((size_t)nw * nrhs, zc(0, 0));
  LQ_TRY(to_host(c, d, (size_t)nw * nrhs, G));
  for (int k = 0; k < nrhs; k++) {
    zc *g = &G[(size_t)nw * k], *z = &Z[(size_t)nw * k];
    if (!mask[k]) {
      for (int w = 0; w < nw; w++) g[w] = 0;
      continue;
    }
    for (int i = 0; i < S.ev_n; i++) {
      const int j = S.ev_partner[i];
      const double A = a * rho * (1.0 + sg * S.ev_c[i]) + m, B = j >= 0 ? a * rho * sg * S.ev_pn[i] : 0.0;
      const double mu = A * A + B * B;
      if (!(mu > 1e-14)) {  // a massless zero mode
        g[i] = 0;
        if (j >= 0) g[j] = 0;
        continue;
      }
      if (j < 0) {
        z[i] = g[i] * (A / mu);
      } else {
        z[i] = (A * g[i] - B * g[j]) / mu;
        z[j] = (B * g[i] + A * g[j]) / mu;
      }
    }
  }
  // x (+)= W Z, r -= W G, in chunks of the rotation kernel's width
  for (int pass = 0; pass < 2; pass++) {
    const std::vector<zc> &C = pass == 0 ? Z : G;
    lqcd_field *t = pass == 0 ? x : r;
    for (int k0 = 0; k0 < nw; k0 += kRMaxP) {
      const int pc = std::min(kRMaxP, nw - k0);
      std::vector<zc> M((size_t)pc * nrhs);
      for (int k = 0; k < nrhs; k++)
        for (int w = 0; w < pc; w++) M[w + (size_t)pc * k] = C[k0 + w + (size_t)nw * k];
      LQ_TRY(to_dev(c, M, d));
      const lqcd_field Wv = col_view(S.ev, k0, pc);
      const double beta = (pass == 0 && x_zero && k0 == 0) ? 0.0 : 1.0;
      LQ_TRY(rotate(c, &Wv, pc, d, nrhs, t, pass == 0 ? 1.0 : -1.0, beta));
    }
  }
  return LQCD_OK;
}

// the deflated start of the overlap CG: x0 = x_W of b, and r0 = b - D(m) x0
// recomputed with the operator (so the CG's right-hand side is exact)
lqcd_status deflation_guess(lqcd_ctx *c, int nrhs, const lqcd_field *b, lqcd_field *x0, lqcd_field *r0) {
  LQ_TRY(copy_field(c, r0, b, nrhs));
  LQ_TRY(deflate(c, nrhs, r0, x0, true, std::vector<char>(nrhs, 1)));
  LQ_TRY(dov_apply(c, nrhs, x0, r0, 0));
  return combine(c, nrhs, r0, b, r0, 1.0, -1.0, 0);
}

}  // namespace
}  // namespace lqcd

extern "C" lqcd_status lqcd_overlap_setup(lqcd_ctx *c, const lqcd_overlap_params *prm, lqcd_overlap_info *info) {
  NvtxRange nv("lqcd overlap set-up");
  if (!c || !prm) return set_error(LQCD_ERR_ARG, "NULL argument");
  if (!c->have_gauge) return set_error(LQCD_ERR_STATE, "no gauge field loaded");
  if (!(prm->rho > 0 && prm->rho < 2)) return set_error(LQCD_ERR_ARG, "rho must be in (0, 2)");
  if (prm->n_low < 0 || prm->n_low > 64) return set_error(LQCD_ERR_ARG, "n_low must be in 0..64");
  if (!(prm->sign_tol > 0) || !(prm->eig_tol > 0)) return set_error(LQCD_ERR_ARG, "tolerances must be > 0");
  if (prm->max_degree < 1 || prm->max_filter < 1) return set_error(LQCD_ERR_ARG, "max_degree, max_filter >= 1");
  if (prm->high != LQCD_F64 && prm->high != LQCD_DF64) return set_error(LQCD_ERR_ARG, "high must be LQCD_F64 or LQCD_DF64");
  if (prm->eig_method != LQCD_EIG_SUBSPACE && prm->eig_method != LQCD_EIG_LANCZOS)
    return set_error(LQCD_ERR_ARG, "bad eig_method %d", prm->eig_method);
  const auto t0 = std::chrono::steady_clock::now();
  lqcd_overlap_info local{};
  lqcd_overlap_info *inf = info ? info : &local;
  std::memset(inf, 0, sizeof(*inf));
  overlap_free(c);
  LQ_TRY(ensure_state(c));
  OverlapState &S = *c->ov;
  S.prm = *prm;
  S.df = prm->high == LQCD_DF64;
  LQ_TRY(lqcd_set_rho(c, prm->rho));
  const long N = 12L * c->V;
  const int want = std::max(1, prm->n_low);
  // the block holds the wanted modes plus a margin wide enough to contain a
  // near-degenerate cluster at the edge (smooth fields keep the free field's
  // 12-fold momentum multiplets almost degenerate)
  int m = std::min<long>(std::max(want + 16, LQCD_OV_BLOCK_MULT * want), kOvMaxBlock);
  if (m > N) m = (int)N;
  if (want >= m) return set_error(LQCD_ERR_ARG, "lattice too small for %d low modes", want);
  FieldGuard g;
  lqcd_field *X, *T, *HX, *Y, *Z;
  LQ_TRY(new_full(c, m, &X));
  g.f.push_back(X);
  LQ_TRY(new_full(c, m, &T));
  g.f.push_back(T);
  LQ_TRY(new_full(c, m, &HX));
  g.f.push_back(HX);
  LQ_TRY(new_full(c, m, &Y));
  g.f.push_back(Y);
  LQ_TRY(new_full(c, m, &Z));
  g.f.push_back(Z);
  const double bmax = std::pow(4.0 - prm->rho + 4.0, 2);
  std::vector<double> theta, resid;
  std::vector<int> order;
  double2 *d;
  int sweep = 0, kneed = want;
  long applies = 0;  // H_W applications, one per right-hand side
  bool converged = false;
  bool fp32_phase = true;
  int fp32_stall = 0;
  double prev_worst = 1e300;
  lqcd_field *Bs[4] = {nullptr, nullptr, nullptr, nullptr};  // FP32 filter block
  lqcd_field *Bd[4] = {nullptr, nullptr, nullptr, nullptr};  // double-float filter block
  // Block subspace sweeps on X (m orthonormal columns) until the kneed wanted
  // (and edge-degenerate) vectors have H_W^2 residuals <= tol2, or the sweep
  // budget is spent.  `cut` reports a near-degenerate cluster at the edge of
  // the wanted set that fills the block up to its margin (and so may extend
  // beyond it): the block must grow before the H_W Rayleigh-Ritz step, which
  // is exact only on a union of whole clusters (an incomplete one is not
  // H_W-invariant and gives spurious interior Ritz values).
  bool cut = false;
  bool refining = false;  // the refinement filters in FP64 (below double-float's noise floor)
  auto sweeps = [&](double tol2) -> lqcd_status {
    cut = false;
    for (;; sweep++) {
      // Rayleigh-Ritz with H_W^2 (the wanted eigenvalues are its smallest, an
      // extremal problem; Rayleigh-Ritz with H_W itself would be an interior one
      // and produce spurious Ritz values near zero)
      LQ_TRY(hw(c, m, HX, X));
      LQ_TRY(small_scratch(c, (size_t)m * m, &d));
      LQ_TRY(gram(c, HX, m, HX, m, d));
      std::vector<zc> W, Q;
      LQ_TRY(to_host(c, d, (size_t)m * m, W));
      for (int j = 0; j < m; j++)  // symmetrise
        for (int i = 0; i < j; i++) {
          const zc avg = 0.5 * (W[i + (size_t)m * j] + std::conj(W[j + (size_t)m * i]));
          W[i + (size_t)m * j] = avg;
          W[j + (size_t)m * i] = std::conj(avg);
        }
      std::vector<double> mu;
      jacobi_eigh(m, W, Q, mu);
      // ascending order of mu
      order.resize(m);
      for (int i = 0; i < m; i++) order[i] = i;
      std::sort(order.begin(), order.end(), [&](int x, int y) { return mu[x] < mu[y]; });
      std::vector<zc> Qs((size_t)m * m);
      std::vector<double> mus(m);
      for (int jj = 0; jj < m; jj++) {
        mus[jj] = mu[order[jj]];
        for (int i = 0; i < m; i++) Qs[i + (size_t)m * jj] = Q[i + (size_t)m * order[jj]];
      }
      LQ_TRY(to_dev(c, Qs, d));
      LQ_TRY(rotate(c, X, m, d, m, T, 1.0, 0.0));
      LQ_TRY(rotate(c, HX, m, d, m, Y, 1.0, 0.0));
      std::swap(X, T);
      std::swap(HX, Y);
      // residuals of H_W^2: || H_W (H_W x) - mu x ||
      LQ_TRY(hw(c, m, Z, HX));
      std::vector<double> neg(m), r2;
      for (int i = 0; i < m; i++) neg[i] = -mus[i];
      LQ_TRY(axpy_norms(c, Z, X, neg, m, r2));
      applies += 2L * m;
      // converge the wanted vectors and every vector nearly degenerate with the
      // edge of the wanted set (a near-degenerate +-lambda partner left outside
      // would stay mixed into a wanted vector)
      kneed = want;
      while (kneed < m - 4 && mus[kneed] <= 1.01 * mus[want - 1]) kneed++;
      bool done = true;
      for (int i = 0; i < kneed; i++) done &= std::sqrt(r2[i]) <= tol2;
      theta = mus;
      double worst = 0;
      for (int i = 0; i < kneed; i++) worst = std::max(worst, std::sqrt(r2[i]));
      // once the Ritz values mean something, a cluster reaching the margin
      // asks for a wider block
      if (m < kOvMaxBlock && kneed == m - 4 && mus[kneed] <= 1.01 * mus[want - 1] && worst < 1e-2) {
        cut = true;
        sweep++;
        return LQCD_OK;
      }
      if (done || sweep + 1 >= prm->max_filter) {
        sweep++;
        return LQCD_OK;
      }
      // Chebyshev filter of H_W^2 damping [mu_max, bmax], in FP32 while the
      // residuals are far above the FP32 noise floor, in FP64 afterwards
      // FP32 filtering injects ~1e-7 relative noise: use it only while the
      // residuals are large and still falling, FP64 from then on
#if LQCD_OV_FP32_RULE == 0
      if (fp32_phase && (worst < 1e-4 || worst > 0.5 * prev_worst)) fp32_phase = false;
#else
      // FP32 filtering injects ~1e-7 relative noise (a floor of ~1e-5 on the
      // H_W^2 residuals, |H_W^2| ~ 42): keep it while the residuals are above
      // 1e-4 and not stuck on that floor (three sweeps in a row without a 1 %
      // drop end it; slow progress while an edge eigenvalue settles does not)
      fp32_stall = worst > 0.99 * prev_worst ? fp32_stall + 1 : 0;
      if (fp32_phase && (worst < 1e-4 || fp32_stall >= 3)) fp32_phase = false;
#endif
      if (kOvTrace)
        std::fprintf(stderr, "lqcd overlap: sweep %d worst %.3e kneed %d mu[kneed-1] %.6f mu[m-1] %.6f %s\n", sweep,
                     worst, kneed, mus[kneed - 1], mus[m - 1], fp32_phase ? "fp32" : (S.df ? "df64" : "fp64"));
      prev_worst = worst;
      const bool low = fp32_phase;
      const double lo = std::min(std::max(mus[m - 1], 1.02 * mus[kneed - 1]), 0.9 * bmax), hi = bmax;
      const double s2 = 2.0 / (hi - lo), s0 = -(hi + lo) / (hi - lo);
      const int deg = 16;
      // the filter runs on a copy of X in FP32 (early sweeps) or double-float
      // (on request), in place in FP64 otherwise
      const lqcd_prec fp = low ? LQCD_F32 : (S.df && !refining) ? LQCD_DF64 : LQCD_F64;
      lqcd_field *fX = X, *fY = Y, *fH = HX, *fT = T;
      if (fp != LQCD_F64) {
        lqcd_field **blk = fp == LQCD_F32 ? Bs : Bd;
        if (!blk[0]) {
          for (int q = 0; q < 4; q++) {
            LQ_TRY(lqcd_field_create(c, fp, LQCD_FULL, m, &blk[q]));
            g.f.push_back(blk[q]);
          }
        }
        LQ_TRY(convert_full(c, blk[0], X, m));
        fX = blk[0], fY = blk[1], fH = blk[2], fT = blk[3];
      }
      // Y0 = X, Y1 = T(X), Y_{k+1} = 2 T(Y_k) - Y_{k-1} with T = s2 H^2 + s0: the
      // second H_W of each step carries the update in its epilogue
      LQ_TRY(hw(c, m, fT, fX));
      LQ_TRY(hw_cheb(c, m, fY, fT, s2, fX, s0, nullptr, 0.0, nullptr, 0.0));
      lqcd_field *prev = fX, *cur = fY, *nxt = fH;
      for (int k = 1; k < deg; k++) {
        LQ_TRY(hw(c, m, fT, cur));
        LQ_TRY(hw_cheb(c, m, nxt, fT, 2.0 * s2, cur, 2.0 * s0, prev, -1.0, nullptr, 0.0));
        lqcd_field *t = prev;
        prev = cur;
        cur = nxt;
        nxt = t;
      }
      applies += 2L * deg * m;
      if (fp != LQCD_F64) {
        LQ_TRY(convert_full(c, X, cur, m));
      } else if (cur != X) {  // the filtered block becomes X; the other two are scratch
        lqcd_field *others[3] = {X, Y, HX};
        lqcd_field *rest[2];
        int r = 0;
        for (auto *o : others)
          if (o != cur) rest[r++] = o;
        X = cur;
        Y = rest[0];
        HX = rest[1];
      }
      LQ_TRY(orthonormalise(c, X, T, m));
    }
  };
  // Rayleigh-Ritz with H_W in the span of the kneed converged vectors of
  // H_W^2 (an invariant subspace of H_W): signed eigenvalues and vectors and
  // their H_W residuals ||H_W v - lambda v||; returns the largest residual of
  // the `want` of smallest |lambda|
  auto final_rr = [&](double &worst_wanted) -> lqcd_status {
    const int k = kneed;
    LQ_TRY(hw(c, k, HX, X));
    applies += k;
    LQ_TRY(small_scratch(c, (size_t)k * k, &d));
    LQ_TRY(gram(c, X, k, HX, k, d));
    std::vector<zc> W, Q;
    LQ_TRY(to_host(c, d, (size_t)k * k, W));
    for (int j = 0; j < k; j++)
      for (int i = 0; i < j; i++) {
        const zc avg = 0.5 * (W[i + (size_t)k * j] + std::conj(W[j + (size_t)k * i]));
        W[i + (size_t)k * j] = avg;
        W[j + (size_t)k * i] = std::conj(avg);
      }
    jacobi_eigh(k, W, Q, theta);
    LQ_TRY(to_dev(c, Q, d));
    LQ_TRY(rotate(c, X, k, d, k, T, 1.0, 0.0));
    LQ_TRY(rotate(c, HX, k, d, k, Y, 1.0, 0.0));
    // the rotated Ritz vectors go back into the first k columns of X (the
    // rest of the block is untouched, so X stays an orthonormal block)
    for (int p = 0; p < 2; p++) {
      LQ_CU(cudaMemcpyAsync(col(X, p, 0), col(T, p, 0), (size_t)k * cwords(X) * 16, cudaMemcpyDeviceToDevice,
                            c->stream));
      LQ_CU(cudaMemcpyAsync(col(HX, p, 0), col(Y, p, 0), (size_t)k * cwords(X) * 16, cudaMemcpyDeviceToDevice,
                            c->stream));
    }
    std::vector<double> neg(k), r2;
    for (int i = 0; i < k; i++) neg[i] = -theta[i];
    LQ_TRY(axpy_norms(c, HX, X, neg, k, r2));
    resid.resize(k);
    for (int i = 0; i < k; i++) resid[i] = std::sqrt(r2[i]);
    order.resize(k);
    for (int i = 0; i < k; i++) order[i] = i;
    std::sort(order.begin(), order.end(), [&](int x, int y) { return std::fabs(theta[x]) < std::fabs(theta[y]); });
    worst_wanted = 0;
    for (int i = 0; i < want; i++) worst_wanted = std::max(worst_wanted, resid[order[i]]);
    return LQCD_OK;
  };
  auto random_columns = [&](int from) -> lqcd_status {
    if (from >= m) return LQCD_OK;
    const long nd = 2L * cwords(X) * (m - from);  // doubles per parity
    for (int p = 0; p < 2; p++) {
      gauss_fill_kernel<<<(unsigned)((nd / 2 + kT - 1) / kT), kT, 0, c->stream>>>(
          (double *)col(X, p, from), nd, prm->seed * 2 + p + 1 + 1000003ULL * (unsigned long long)sweep);
      LQ_CU(cudaGetLastError());
    }
    return LQCD_OK;
  };
  // widen the block to m2 columns: the current ones are kept, the new ones
  // random, then the block is orthonormalised (Cholesky QR keeps the span of
  // the leading columns)
  auto grow = [&](int m2) -> lqcd_status {
    lqcd_field *nf[5];
    for (auto &f : nf) {
      LQ_TRY(new_full(c, m2, &f));
      g.f.push_back(f);
    }
    for (int p = 0; p < 2; p++)
      LQ_CU(cudaMemcpyAsync(col(nf[0], p, 0), col(X, p, 0), (size_t)m * cwords(X) * 16, cudaMemcpyDeviceToDevice,
                            c->stream));
    X = nf[0], T = nf[1], HX = nf[2], Y = nf[3], Z = nf[4];
    for (int q = 0; q < 4; q++) Bs[q] = Bd[q] = nullptr;  // the filter blocks follow the new width
    const int old = m;
    m = m2;
    if (kOvTrace) std::fprintf(stderr, "lqcd overlap: edge cluster fills the block, widening it %d -> %d\n", old, m);
    LQ_TRY(random_columns(old));
    return orthonormalise(c, X, T, m);
  };
  auto run_sweeps = [&](double tol2) -> lqcd_status {
    for (;;) {
      LQ_TRY(sweeps(tol2));
      if (!cut || sweep >= prm->max_filter) return LQCD_OK;
      LQ_TRY(grow((int)std::min<long>(std::min<long>(kOvMaxBlock, N), std::max(2 * m, m + 16))));
    }
  };
  double tol2 = prm->eig_tol;
  if (prm->eig_method == LQCD_EIG_LANCZOS) {
    // restart size m (the block of the subspace method), basis of max(2m, m + 104): on a
    // dense low spectrum (24^3 x 64, eps 0.1) a basis of 2m = 80 for 20 modes stalled for
    // 1000 restarts; the thick restart needs room beyond the kept block
    const int mmax = std::min<long>(std::min(std::max(2 * m, m + 104), LQCD_OV_LANCZOS_MMAX), N - 1);
    if (mmax < m + 8) return set_error(LQCD_ERR_ARG, "lattice too small for a Lanczos basis of %d vectors", m + 8);
    // the H_W residual of the result is about |lambda| / gap times its H_W^2
    // residual: the Krylov method is asked for 1 % of eig_tol on H_W^2, cheap
    // once it has converged
    lqcd_overlap_params lprm = *prm;
    lprm.eig_tol = std::max(1e-2 * prm->eig_tol, 1e-13);
    LanczosResult lr;
    LQ_TRY(lowmodes_lanczos(c, &lprm, want, m, mmax, X, g, lr));
    kneed = lr.kneed;
    sweep = lr.cycles;
    applies = lr.applies;
    converged = lr.converged;
    fp32_phase = false;
  } else {
    LQ_TRY(random_columns(0));
    LQ_TRY(orthonormalise(c, X, T, m));
    LQ_TRY(run_sweeps(tol2));
  }
  // The contract is on H_W itself: ||H_W v - lambda v|| <= eig_tol for every
  // returned mode.  An H_W^2 residual of eig_tol leaves an eigenvector error
  // of about eig_tol / gap, gap the distance of the cluster's H_W^2 eigenvalue
  // to the rest of the spectrum, so on a clustered spectrum the H_W residual
  // can exceed eig_tol by the ratio |lambda| / gap.  The set-up therefore
  // checks the H_W residuals after the final Rayleigh-Ritz step and, while
  // they exceed eig_tol, tightens the H_W^2 target in proportion and sweeps
  // on (the first time after the Lanczos method, on its Ritz vectors padded
  // with random columns to a full block).
  bool padded = prm->eig_method != LQCD_EIG_LANCZOS;
  if (!padded && kneed >= m - 4) {  // Lanczos kept a cluster as wide as its restart block
    LQ_TRY(random_columns(kneed));
    LQ_TRY(orthonormalise(c, X, T, m));
    padded = true;
    LQ_TRY(run_sweeps(tol2));
  }
  double worst = 0;
  LQ_TRY(final_rr(worst));
  // the H_W^2 residual the refinement can still resolve: its filter runs in
  // FP64 (double-float filtering leaves ~3e-12 of noise); two rounds at the
  // floor without meeting eig_tol end it (LQCD_ERR_NOCONV)
  const double floor2 = 5e-14;
  int at_floor = 0;
  refining = true;
  while (worst > prm->eig_tol && sweep < prm->max_filter && at_floor < 2) {
    tol2 = std::max(floor2, tol2 * std::min(0.5, std::max(0.1, 0.5 * prm->eig_tol / worst)));
    if (tol2 <= floor2) at_floor++;
    if (!padded) {
      LQ_TRY(random_columns(kneed));
      LQ_TRY(orthonormalise(c, X, T, m));
      padded = true;
    }
    if (kOvTrace)
      std::fprintf(stderr, "lqcd overlap: H_W residual %.3e > eig_tol, refining to H_W^2 residual %.3e\n", worst,
                   tol2);
    LQ_TRY(run_sweeps(tol2));
    LQ_TRY(final_rr(worst));
  }
  converged = worst <= prm->eig_tol;
  sweep--;  // inf->sweeps below counts sweep + 1
  inf->sweeps = sweep + 1;
  inf->hw_applies = (double)applies;
  // keep the `want` lowest (by |theta|), sorted
  S.nlow = prm->n_low;
  S.lam.assign(S.nlow, 0.0);
  if (S.nlow > 0) {
    LQ_TRY(lqcd_field_create(c, LQCD_F64, LQCD_FULL, S.nlow, &S.vecs));
    const size_t bytes = (size_t)cwords(X) * 16;
    for (int i = 0; i < S.nlow; i++) {
      S.lam[i] = theta[order[i]];
      for (int p = 0; p < 2; p++)
        LQ_CU(cudaMemcpyAsync(col(S.vecs, p, i), col(X, p, order[i]), bytes, cudaMemcpyDeviceToDevice, c->stream));
    }
  }
  inf->n_low = S.nlow;
  for (int i = 0; i < std::min(64, want); i++) {
    if (i < S.nlow) inf->lambda[i] = theta[order[i]];
    inf->resid[i] = resid[order[i]];
  }
  // interval of the polynomial: every unprojected |lambda| >= |lambda_{n_low}|
  const double lam_edge = std::fabs(theta[order[want - 1]]);
  const double lam_a = prm->n_low > 0 ? lam_edge : lam_edge - resid[order[0]];
  S.a = std::max(lam_a * lam_a, 1e-8);
  S.b = bmax;
  S.degree = cheb_degree(S.a, S.b, prm->sign_tol, prm->max_degree, S.coef);
  if (S.degree < 0) return set_error(LQCD_ERR_NOCONV, "no Chebyshev degree <= %d reaches %.3g", prm->max_degree, prm->sign_tol);
  inf->a = S.a;
  inf->b = S.b;
  inf->degree = S.degree;
  S.degree32 = cheb_degree(S.a, S.b, std::max(prm->sign_tol, kInnerSignTol), prm->max_degree, S.coef32);
  if (S.degree32 < 0) {
    S.degree32 = S.degree;
    S.coef32 = S.coef;
  }
  inf->degree_inner = S.degree32;
  inf->sign_error = sign_error(S.a, S.b, S.coef);
  LQ_CU(cudaStreamSynchronize(c->stream));
  inf->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  // an unconverged set-up leaves the state unusable: the sign function would
  // project with inexact eigenvectors
  if (!converged)
    return set_error(LQCD_ERR_NOCONV, "low modes not converged to ||H_W v - lambda v|| <= %.3g in %d sweeps",
                     prm->eig_tol, prm->max_filter);
  S.ready = true;
  return LQCD_OK;
}

extern "C" lqcd_status lqcd_overlap_lowmodes(lqcd_ctx *c, double *vecs, int on_device) {
  if (!c || !vecs) return set_error(LQCD_ERR_ARG, "NULL argument");
  if (!c->ov || !c->ov->ready) return set_error(LQCD_ERR_STATE, "overlap not set up");
  if (c->ov->nlow == 0) return LQCD_OK;
  return lqcd_field_export(c, c->ov->vecs, vecs, on_device);
}

extern "C" lqcd_status lqcd_overlap(lqcd_ctx *c, double *out, const double *in, int nrhs, int on_device,
                                    lqcd_overlap_op op, const lqcd_solve_params *cg, lqcd_solve_info *info) {
  if (!c || !out || !in) return set_error(LQCD_ERR_ARG, "NULL argument");
  if (!c->ov || !c->ov->ready) return set_error(LQCD_ERR_STATE, "overlap not set up (lqcd_overlap_setup)");
  if (nrhs < 1 || nrhs > 64) return set_error(LQCD_ERR_ARG, "nrhs must be in 1..64");
  if ((int)op < 0 || (int)op > 4) return set_error(LQCD_ERR_ARG, "bad overlap op");
  const bool solve = op == LQCD_OV_SOLVE || op == LQCD_OV_SOLVE_DEFLATED;
  if (solve && (!cg || !(cg->tol > 0) || cg->max_iter < 1))
    return set_error(LQCD_ERR_ARG, "solve needs cg with tol > 0 and max_iter >= 1");
  if (op == LQCD_OV_SOLVE_DEFLATED && !c->ov->ev)
    return set_error(LQCD_ERR_STATE, "no overlap eigensystem to deflate with (lqcd_overlap_eigen)");
  LQ_TRY(ensure_state(c));
  const auto t0 = std::chrono::steady_clock::now();
  FieldGuard g;
  lqcd_field *fin, *fout;
  LQ_TRY(new_full(c, nrhs, &fin));
  g.f.push_back(fin);
  LQ_TRY(new_full(c, nrhs, &fout));
  g.f.push_back(fout);
  LQ_TRY(lqcd_field_import(c, fin, in, on_device));
  lqcd_solve_info local{};
  lqcd_solve_info *inf = info ? info : &local;
  std::memset(inf, 0, sizeof(*inf));
  inf->nrhs = nrhs;
  lqcd_status result = LQCD_OK;
  if (op == LQCD_OV_SIGN) {
    LQ_TRY(sign_apply(c, nrhs, fin, fout));
  } else if (op == LQCD_OV_APPLY || op == LQCD_OV_APPLY_DAG) {
    LQ_TRY(dov_apply(c, nrhs, fin, fout, op == LQCD_OV_APPLY_DAG));
  } else {
    std::vector<double> bn2;
    LQ_TRY(field_norms(c, fin, nrhs, bn2));
    for (int k = 0; k < nrhs; k++)
      if (!(bn2[k] > 0) || !std::isfinite(bn2[k]))
        return set_error(LQCD_ERR_ARG, "right-hand side %d is zero or not finite", k);
    // deflated: the CG solves D e = r0 = b - D x0 from the eigensystem's
    // exact low-mode part x0, to the same target |b - D x| <= tol |b|
    lqcd_field *x0 = nullptr, *rhs = fin;
    if (op == LQCD_OV_SOLVE_DEFLATED) {
      LQ_TRY(new_full(c, nrhs, &x0));
      g.f.push_back(x0);
      LQ_TRY(new_full(c, nrhs, &rhs));
      g.f.push_back(rhs);
      LQ_TRY(deflation_guess(c, nrhs, fin, x0, rhs));
    }
    if (cg->inner == LQCD_F64) {
      LQ_TRY(ov_cgls_fp64(c, nrhs, rhs, fout, cg, inf, bn2));
    } else {
      if (cg->inner != LQCD_F32) return set_error(LQCD_ERR_ARG, "overlap inner precision must be F64 or F32");
      if (c->ov->nlow > 0 && !c->ov->vecs32) {
        LQ_TRY(lqcd_field_create(c, LQCD_F32, LQCD_FULL, c->ov->nlow, &c->ov->vecs32));
        LQ_TRY(convert_full(c, c->ov->vecs32, c->ov->vecs, c->ov->nlow));
      }
      LQ_TRY(ov_cgls_mixed(c, nrhs, rhs, fout, cg, inf, bn2, op == LQCD_OV_SOLVE_DEFLATED));
    }
    if (x0) LQ_TRY(axpy_full(c, fout, x0, std::vector<double>(nrhs, 1.0), nrhs));
    int it = inf->iters;
    lqcd_field *q;
    LQ_TRY(new_full(c, nrhs, &q));
    g.f.push_back(q);
    // true residual b - D_ov x, FP64
    LQ_TRY(dov_apply(c, nrhs, fout, q, 0));
    std::vector<double> mone(nrhs, -1.0), res;
    LQ_TRY(axpy_norms(c, fin, q, mone, nrhs, res));
    bool ok = true;
    for (int k = 0; k < nrhs; k++) {
      inf->true_resid[k] = std::sqrt(res[k] / bn2[k]);
      ok &= inf->true_resid[k] <= cg->tol;
    }
    if (!ok) result = set_error(LQCD_ERR_NOCONV, "overlap CG: true residual above tol after %d iterations", it);
  }
  LQ_TRY(lqcd_field_export(c, fout, out, on_device));
  LQ_CU(cudaStreamSynchronize(c->stream));
  inf->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  return result;
}

// The low eigenpairs of D_ov(0)^dag D_ov(0) in one chirality sector (Sec. 4's
// overlap eigensystem).  On sector s, D_ov(0)^dag D_ov(0) = H_s = 2 rho^2 P_s
// (1 + s eps) P_s: thick-restart Lanczos on H_s, one sign-function application
// per Krylov vector; then, in batches, eps chi_i gives both the residual
// ||H_s chi_i - mu_i chi_i|| = 2 rho^2 ||P_s eps chi_i - c_i chi_i|| (c_i =
// <chi_i, eps chi_i>, mu_i = 2 rho^2 (1 + s c_i)) and the partner eta_i =
// P_-s eps chi_i / |.| of the other sector with the same eigenvalue.
extern "C" lqcd_status lqcd_overlap_eigen(lqcd_ctx *c, const lqcd_overlap_eigen_params *ep,
                                          lqcd_overlap_eigen_info *info) {
  using namespace lqcd;
  NvtxRange nv("lqcd overlap eigensystem");
  if (!c || !ep) return set_error(LQCD_ERR_ARG, "NULL argument");
  if (!c->ov || !c->ov->ready) return set_error(LQCD_ERR_STATE, "overlap not set up (lqcd_overlap_setup)");
  if (ep->n_ev < 1 || ep->n_ev > LQCD_OV_MAX_EV) return set_error(LQCD_ERR_ARG, "n_ev must be in 1..%d", LQCD_OV_MAX_EV);
  if (ep->sector != 1 && ep->sector != -1) return set_error(LQCD_ERR_ARG, "sector must be +1 or -1");
  if (!(ep->tol > 0) || ep->max_restarts < 1) return set_error(LQCD_ERR_ARG, "need tol > 0 and max_restarts >= 1");
  const int n_ev = ep->n_ev, s = ep->sector;
  const long N = 6L * c->V;  // dimension of a chirality sector
  // a basis of ~3 n_ev: thick restarts then converge in a few tens of cycles
  // (16^3 x 32, 100 pairs: 40 cycles with 2 n_ev, 153 for 50 pairs)
  int mmax = ep->basis > 0 ? ep->basis : std::min(std::max(3 * n_ev, n_ev + 48), kLzMaxP - 1);
  if (mmax > kLzMaxP - 1 || mmax < n_ev + 16)
    return set_error(LQCD_ERR_ARG, "Lanczos basis must be in n_ev + 16 .. %d", kLzMaxP - 1);
  if (mmax >= N) return set_error(LQCD_ERR_ARG, "lattice too small for a Lanczos basis of %d vectors", mmax);
  const int kkeep = std::min(mmax - 8, std::max(n_ev + 8, (n_ev + mmax) / 2));
  const auto t0 = std::chrono::steady_clock::now();
  lqcd_overlap_eigen_info local{};
  lqcd_overlap_eigen_info *inf = info ? info : &local;
  std::memset(inf, 0, sizeof(*inf));
  OverlapState &S = *c->ov;
  if (S.ev) {
    lqcd_field_destroy(S.ev);
    S.ev = nullptr;
  }
  S.ev_n = S.ev_np = 0;
  S.ev_mu.clear();
  const double rho = S.prm.rho, r2 = 2.0 * rho * rho;
  FieldGuard g;
  lqcd_field *X;
  LQ_TRY(new_full(c, kkeep, &X));
  g.f.push_back(X);
  LanczosResult lr;
  {
    FieldGuard gl;  // the Lanczos basis is released before the vectors are post-processed
    lqcd_field *x64, *e64;
    LQ_TRY(new_full(c, 1, &x64));
    gl.f.push_back(x64);
    LQ_TRY(new_full(c, 1, &e64));
    gl.f.push_back(e64);
    LzSpec sp;
    sp.per_call = 1;
    sp.tol = 0.5 * ep->tol;
    sp.max_cycles = ep->max_restarts;
    sp.seed = ep->seed;
    sp.start = [&](lqcd_field *x) { return chiral_project(c, x, 1, s); };
    sp.apply = [&](lqcd_field *xd, lqcd_field *wd) -> lqcd_status {
      LQ_TRY(convert_full(c, x64, xd, 1));
      LQ_TRY(sign_apply(c, 1, x64, e64));
      LQ_TRY(chiral_project(c, e64, 1, s));
      LQ_TRY(combine(c, 1, e64, x64, e64, r2, r2 * s, 0));  // 2 rho^2 (x + s P_s eps x)
      return convert_full(c, wd, e64, 1);
    };
    LQ_TRY(lanczos_lowest(c, sp, n_ev, kkeep, mmax, X, gl, lr, nullptr));
  }
  inf->restarts = lr.cycles;
  inf->sign_applies = (double)lr.applies;
  if (!lr.converged) {
    inf->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    return set_error(LQCD_ERR_NOCONV, "overlap eigensystem: Lanczos did not converge in %d restarts", lr.cycles);
  }
  // residuals, Rayleigh quotients and partners, 16 vectors at a time
  lqcd_field *ev;
  LQ_TRY(new_full(c, 2 * n_ev, &ev));
  g.f.push_back(ev);
  constexpr int kB = 16;
  lqcd_field *E, *P;
  LQ_TRY(new_full(c, kB, &E));
  g.f.push_back(E);
  LQ_TRY(new_full(c, kB, &P));
  g.f.push_back(P);
  std::vector<double> mu(n_ev), res(n_ev), pmu, cvec(n_ev), pnv(n_ev, 0.0);
  std::vector<int> pidx, pcol(n_ev, -1);
  double2 *d;
  bool ok = true;
  for (int k0 = 0; k0 < n_ev; k0 += kB) {
    const int nb = std::min(kB, n_ev - k0);
    const lqcd_field Xv = col_view(X, k0, nb);
    LQ_TRY(sign_apply(c, nb, &Xv, E));
    LQ_TRY(small_scratch(c, (size_t)nb * nb, &d));
    LQ_TRY(gram(c, &Xv, nb, E, nb, d));
    std::vector<zc> G;
    LQ_TRY(to_host(c, d, (size_t)nb * nb, G));
    std::vector<double> cc(nb), mc(nb), r2v, pn;
    for (int i = 0; i < nb; i++) {
      cc[i] = G[i + (size_t)nb * i].real();
      mc[i] = -cc[i];
      mu[k0 + i] = r2 * (1.0 + s * cc[i]);
      cvec[k0 + i] = cc[i];
    }
    LQ_TRY(copy_field(c, P, E, nb));
    LQ_TRY(chiral_project(c, P, nb, s));
    LQ_TRY(axpy_norms(c, P, &Xv, mc, nb, r2v));  // |P_s eps chi - c chi|^2
    for (int i = 0; i < nb; i++) {
      res[k0 + i] = r2 * std::sqrt(std::max(r2v[i], 0.0));
      ok &= res[k0 + i] <= ep->tol;
    }
    LQ_TRY(copy_col_range(c, ev, k0, X, k0, nb));
    LQ_TRY(chiral_project(c, E, nb, -s));  // P_-s eps chi
    LQ_TRY(field_norms(c, E, nb, pn));
    for (int i = 0; i < nb; i++) {
      if (!(pn[i] > 1e-10)) continue;  // a chiral zero mode, or mu = 4 rho^2: no partner
      pidx.push_back(k0 + i);
      pmu.push_back(mu[k0 + i]);
      pcol[k0 + i] = n_ev + (int)pidx.size() - 1;
      pnv[k0 + i] = std::sqrt(pn[i]);
      // partners follow the n_ev sector vectors, in the order found
      std::vector<double> f(1, 1.0 / std::sqrt(pn[i]));
      const lqcd_field Ei = col_view(E, i, 1);
      lqcd_field Ev = col_view(ev, n_ev + (int)pidx.size() - 1, 1);
      LQ_TRY(scale_full(c, &Ev, &Ei, f, 1));
    }
  }
  inf->sign_applies += n_ev;
  inf->n_ev = n_ev;
  inf->n_partners = (int)pidx.size();
  for (int i = 0; i < n_ev; i++) {
    inf->mu[i] = mu[i];
    inf->resid[i] = res[i];
    const double re = mu[i] / (2.0 * rho);
    inf->lambda_re[i] = re;
    inf->lambda_im[i] = std::sqrt(std::max(mu[i] - re * re, 0.0));
  }
  inf->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  if (!ok) return set_error(LQCD_ERR_NOCONV, "overlap eigensystem: a residual is above tol");
  S.ev = ev;
  g.f.erase(std::find(g.f.begin(), g.f.end(), ev));
  S.ev_n = n_ev;
  S.ev_np = (int)pidx.size();
  S.ev_sector = s;
  S.ev_mu = mu;
  S.ev_mu.insert(S.ev_mu.end(), pmu.begin(), pmu.end());
  S.ev_c = cvec;
  S.ev_pn = pnv;
  S.ev_partner = pcol;
  return LQCD_OK;
}

extern "C" lqcd_status lqcd_overlap_eigvecs(lqcd_ctx *c, double *vecs, int partners, int on_device) {
  using namespace lqcd;
  if (!c || !vecs) return set_error(LQCD_ERR_ARG, "NULL argument");
  if (!c->ov || !c->ov->ev) return set_error(LQCD_ERR_STATE, "no overlap eigensystem (lqcd_overlap_eigen)");
  OverlapState &S = *c->ov;
  const int k0 = partners ? S.ev_n : 0, n = partners ? S.ev_np : S.ev_n;
  if (n == 0) return LQCD_OK;
  const lqcd_field v = col_view(S.ev, k0, n);
  return lqcd_field_export(c, &v, vecs, on_device);
}
