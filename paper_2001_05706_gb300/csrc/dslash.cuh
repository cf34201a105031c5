// The even-odd Wilson-clover hopping kernel and its fused epilogues.
//
// One thread owns one output site of one parity (and NR right-hand sides).
// For each of the 8 directions it loads the neighbour spinor, projects it
// onto a half-spinor with (1 -+ g_mu) (DeGrand-Rossi basis: g_mu =
// [[0, B_mu], [B_mu^dag, 0]], so (1 + s g_mu) psi = (h, s B_mu^dag h) with
// h = u + s B_mu l for psi = (u, l)), multiplies the two colour vectors by
// U_mu(x) or U_mu(x-mu)^dag (the 12-real form rebuilt in registers), and
// accumulates the reconstructed spinor.  The epilogue then applies, per
// MODE, the inverse clover block (K2a: y = A^-1 D x), the local clover term
// and an xpay (K2b: z = A x - kappa^2 D y), the folded reconstruction
// A^-1 (b + kappa D x), gamma5 and an optional "z + c * result", and
// accumulates ||result||^2 into a deterministic grid reduction.
//
// Link times spinor is a 3x3 complex matrix-vector product: no dense
// contraction, so this runs on the CUDA cores; it is HBM-bound for FP32 and
// half storage and FP64-ALU-bound for FP64 on GB300.
#pragma once
#include <type_traits>

#include "common.cuh"
#include "reduce.cuh"

namespace lqcd {

enum DslashMode {
  MODE_HOP = 0,          // out = beta * hop
  MODE_HOP_AINV = 1,     // out = Ainv (beta * hop)
  MODE_LOCAL_IDENT = 2,  // out = alpha * x + beta * hop
  MODE_LOCAL_A = 3,      // out = alpha * A x + beta * hop
  MODE_FOLDED_AINV = 4,  // out = Ainv (alpha * x + beta * hop)
  MODE_CHEB = 5          // out = (g5) (alpha * x + beta * hop) + sum_k cz[k] zc[k]  (Chebyshev step)
};

struct FieldRef {
  const void *data;  // [rhs][words][Vh]
  const float *scale;  // [rhs][Vh] for FP16/BF16, else nullptr
  long rhs_words;      // words of one RHS of one parity (stride between RHS, in words of that field)
};

struct DslashParams {
  Geom g;
  long h0, h1;  // output sites [h0, h1) of the parity (a whole parity: 0, Vh)
  int out_parity;
  int nrhs;
  void *out;
  float *out_scale;
  FieldRef in;    // hop input (other parity); data == nullptr or beta == 0: no hop
  FieldRef xloc;  // local term input (output parity)
  FieldRef z;     // optional xpay input (output parity)
  FieldRef zc[3];  // MODE_CHEB: extra terms of the output parity (data == nullptr: absent)
  double cz[3];
  const void *links[4][2];  // [mu][parity]
  const void *cmat;         // A^-1 of the output parity (packed blocks)
  const float *cmat_scale;
  const void *lmat;         // A of the output parity
  const float *lmat_scale;
  double alpha, beta, gz;
  int g5_in, g5_hop, g5_total;
  double *norm_partials;  // nullptr: no norm (else per-block partials, summed by finish_reduce)
  double *norm_result;    // result of RHS r at norm_result[r * norm_stride]
  int norm_stride;
  unsigned int *dbg;      // builds with LQCD_DEBUG_BOUNDS: set to 1 on an out-of-range index
};

// Debug builds (-DLQCD_DEBUG_BOUNDS=1) check every gathered index against the
// parity's site range; a bad one is recorded in *P.dbg (the host turns it into
// an error after the launch) and replaced by 0 so no access leaves the field.
#ifndef LQCD_DEBUG_BOUNDS
#define LQCD_DEBUG_BOUNDS 0
#endif
#if LQCD_DEBUG_BOUNDS
#define LQCD_CHECK_INDEX(P, i)            \
  do {                                    \
    if ((i) < 0 || (i) >= (P).g.Vh) {     \
      atomicOr((P).dbg, 1u);              \
      (i) = 0;                            \
    }                                     \
  } while (0)
#else
#define LQCD_CHECK_INDEX(P, i) \
  do {                         \
  } while (0)
#endif

// ---------------------------------------------------------------------------
// field access
// ---------------------------------------------------------------------------
template <typename S> __device__ __forceinline__ const void *rhs_base(const void *base, long rhs_words, int r) {
  using Wd = Words<S, 24>;
  return reinterpret_cast<const char *>(base) + (long)r * rhs_words * Wd::W;
}

// FP16/BF16 (re, im) pairs as one 32-bit word: unpacked and packed two
// values per instruction (exact on the way in; round to nearest on the way
// out, as the scalar conversions)
template <typename S> struct PackedPair;
template <> struct PackedPair<__half> {
  using type = __half2;
  static __device__ __forceinline__ type from(unsigned u) { return *reinterpret_cast<const type *>(&u); }
  static __device__ __forceinline__ type make(float a, float b) { return __floats2half2_rn(a, b); }
  static __device__ __forceinline__ float2 f2(type v) { return __half22float2(v); }
};
template <> struct PackedPair<__nv_bfloat16> {
  using type = __nv_bfloat162;
  static __device__ __forceinline__ type from(unsigned u) { return *reinterpret_cast<const type *>(&u); }
  static __device__ __forceinline__ type make(float a, float b) { return __floats2bfloat162_rn(a, b); }
  // a BF16 value is the upper half of an FP32: one shift or mask per value
  static __device__ __forceinline__ float2 f2(type v) {
    const unsigned u = *reinterpret_cast<const unsigned *>(&v);
    return make_float2(__uint_as_float(u << 16), __uint_as_float(u & 0xffff0000u));
  }
};
template <typename S> __device__ __forceinline__ unsigned pack_pair(float a, float b) {
  const auto v = PackedPair<S>::make(a, b);
  return *reinterpret_cast<const unsigned *>(&v);
}
template <typename S> __device__ __forceinline__ float2 unpack_pair(unsigned u) {
  return PackedPair<S>::f2(PackedPair<S>::from(u));
}

// the twelve (re, im) pairs of one FP16/BF16 spinor (three 16-byte words)
template <typename S, bool STREAM = false>
__device__ __forceinline__ void load_pairs(const FieldRef &f, long Vh, int r, long i, unsigned (&u)[12]) {
  static_assert(Words<S, 24>::W == 16, "FP16/BF16 spinors are three 16-byte words");
  const uint4 *p = reinterpret_cast<const uint4 *>(rhs_base<S>(f.data, f.rhs_words, r));
#pragma unroll
  for (int w = 0; w < 3; w++) {
    const uint4 v = STREAM ? ldcs_word(p + (long)w * Vh + i) : ldg_word(p + (long)w * Vh + i);
    u[4 * w] = v.x;
    u[4 * w + 1] = v.y;
    u[4 * w + 2] = v.z;
    u[4 * w + 3] = v.w;
  }
}

template <typename S, bool STREAM = false>
__device__ __forceinline__ void load_spinor(const FieldRef &f, long Vh, int r, long i,
                                            cx<typename Math<S>::T> (&psi)[4][3]) {
  using T = typename Math<S>::T;
  if constexpr (IsHalf<S>::value) {
    unsigned u[12];
    load_pairs<S, STREAM>(f, Vh, r, i, u);
    const T sc = (T)__ldg(f.scale + (long)r * Vh + i);
#pragma unroll
    for (int a = 0; a < 4; a++)
#pragma unroll
      for (int c = 0; c < 3; c++) {
        const float2 v = unpack_pair<S>(u[3 * a + c]);
        psi[a][c] = mk<T>(sc * v.x, sc * v.y);
      }
  } else {
    S raw[24];
    load_reals<S, 24, STREAM>(rhs_base<S>(f.data, f.rhs_words, r), Vh, i, raw);
#pragma unroll
    for (int a = 0; a < 4; a++)
#pragma unroll
      for (int c = 0; c < 3; c++) psi[a][c] = mk<T>((T)to_f(raw[6 * a + 2 * c]), (T)to_f(raw[6 * a + 2 * c + 1]));
  }
}

// The same load without applying the FP16/BF16 scale: returns it instead, so
// callers can fold it into an FMA they do anyway.
template <typename S>
__device__ __forceinline__ typename Math<S>::T load_spinor_raw(const FieldRef &f, long Vh, int r, long i,
                                                               cx<typename Math<S>::T> (&psi)[4][3]) {
  using T = typename Math<S>::T;
  T sc = (T)1;
  if constexpr (IsHalf<S>::value) {
    unsigned u[12];
    load_pairs<S>(f, Vh, r, i, u);
    sc = (T)__ldg(f.scale + (long)r * Vh + i);
#pragma unroll
    for (int a = 0; a < 4; a++)
#pragma unroll
      for (int c = 0; c < 3; c++) {
        const float2 v = unpack_pair<S>(u[3 * a + c]);
        psi[a][c] = mk<T>(v.x, v.y);
      }
  } else {
    S raw[24];
    load_reals<S, 24>(rhs_base<S>(f.data, f.rhs_words, r), Vh, i, raw);
#pragma unroll
    for (int a = 0; a < 4; a++)
#pragma unroll
      for (int c = 0; c < 3; c++) psi[a][c] = mk<T>((T)to_f(raw[6 * a + 2 * c]), (T)to_f(raw[6 * a + 2 * c + 1]));
  }
  return sc;
}

template <typename S>
__device__ __forceinline__ void store_spinor(void *base, float *scale, long rhs_words, long Vh, int r, long i,
                                             const cx<typename Math<S>::T> (&psi)[4][3]) {
  using T = typename Math<S>::T;
  S raw[24];
  T inv = (T)1;
  if constexpr (IsHalf<S>::value) {
    T m = (T)0;
#pragma unroll
    for (int a = 0; a < 4; a++)
#pragma unroll
      for (int c = 0; c < 3; c++) m = fmax(m, fmax(fabs(psi[a][c].r), fabs(psi[a][c].i)));
    scale[(long)r * Vh + i] = (float)m;
    inv = m > (T)0 ? (T)1 / m : (T)0;
    unsigned u[12];
#pragma unroll
    for (int a = 0; a < 4; a++)
#pragma unroll
      for (int c = 0; c < 3; c++) u[3 * a + c] = pack_pair<S>(psi[a][c].r * inv, psi[a][c].i * inv);
    uint4 *p = reinterpret_cast<uint4 *>(reinterpret_cast<char *>(base) + (long)r * rhs_words * 16);
#pragma unroll
    for (int w = 0; w < 3; w++) p[(long)w * Vh + i] = make_uint4(u[4 * w], u[4 * w + 1], u[4 * w + 2], u[4 * w + 3]);
    return;
  }
#pragma unroll
  for (int a = 0; a < 4; a++)
#pragma unroll
    for (int c = 0; c < 3; c++) {
      raw[6 * a + 2 * c] = from_f<S>(psi[a][c].r * inv);
      raw[6 * a + 2 * c + 1] = from_f<S>(psi[a][c].i * inv);
    }
  void *b = reinterpret_cast<char *>(base) + (long)r * rhs_words * Words<S, 24>::W;
  store_reals<S, 24>(b, Vh, i, raw);
}

template <> __device__ __forceinline__ void store_spinor<double>(void *base, float *, long rhs_words, long Vh, int r,
                                                                 long i, const cx<double> (&psi)[4][3]) {
  double raw[24];
#pragma unroll
  for (int a = 0; a < 4; a++)
#pragma unroll
    for (int c = 0; c < 3; c++) {
      raw[6 * a + 2 * c] = psi[a][c].r;
      raw[6 * a + 2 * c + 1] = psi[a][c].i;
    }
  void *b = reinterpret_cast<char *>(base) + (long)r * rhs_words * Words<double, 24>::W;
  store_reals<double, 24>(b, Vh, i, raw);
}

template <> __device__ __forceinline__ void store_spinor<df>(void *base, float *, long rhs_words, long Vh, int r, long i,
                                                             const cx<df> (&psi)[4][3]) {
  df raw[24];
#pragma unroll
  for (int a = 0; a < 4; a++)
#pragma unroll
    for (int c = 0; c < 3; c++) {
      raw[6 * a + 2 * c] = psi[a][c].r;
      raw[6 * a + 2 * c + 1] = psi[a][c].i;
    }
  void *b = reinterpret_cast<char *>(base) + (long)r * rhs_words * Words<df, 24>::W;
  store_reals<df, 24>(b, Vh, i, raw);
}

// The 8-real form (FP32/FP16 storage): v = (arg U00, arg U20, U01, U02,
// U10) as (re, im) pairs.  |U00|^2 = 1 - |U01|^2 - |U02|^2 (row 0 is a unit
// vector), |U20|^2 = 1 - |U00|^2 - |U10|^2 (so is column 0); U11 and U12 solve
// the two linear conditions row 1 . conj(row 0) = 0 and conj(U20) = U01 U12 -
// U02 U11 (row 2 = conj(row 0 x row 1) for det U = 1), whose determinant is
// |U01|^2 + |U02|^2 = 1 - |U00|^2; row 2 is then that cross product.  The
// library refuses the form for fields with a link where this determinant
// nearly vanishes (U00 of modulus one, e.g. unit links).
// sin and cos of a stored angle (|x| <= pi): the FP32 intrinsic, whose
// absolute error there is below the angle's own FP32 rounding
__device__ __forceinline__ void sincos_angle(float x, float *s, float *c) { __sincosf(x, s, c); }
__device__ __forceinline__ void sincos_angle(double x, double *s, double *c) { sincos(x, s, c); }

template <typename T> __device__ __forceinline__ void rebuild_link8(const T (&v)[8], cx<T> (&U)[3][3]) {
  const cx<T> u01 = mk<T>(v[2], v[3]), u02 = mk<T>(v[4], v[5]), u10 = mk<T>(v[6], v[7]);
  const T d = u01.r * u01.r + u01.i * u01.i + u02.r * u02.r + u02.i * u02.i;  // 1 - |U00|^2
  const T a00 = sqrt(fmax((T)1 - d, (T)0));
  T s0, c0, s2, c2;
  sincos_angle(v[0], &s0, &c0);
  sincos_angle(v[1], &s2, &c2);
  const cx<T> u00 = mk<T>(a00 * c0, a00 * s0);
  const T a20 = sqrt(fmax(d - (u10.r * u10.r + u10.i * u10.i), (T)0));
  const cx<T> u20 = mk<T>(a20 * c2, a20 * s2);
  const T id = (T)1 / d;
  const cx<T> e = (T)-1 * (u10 * conjg(u00));  // right-hand side of the orthogonality condition
  const cx<T> f = conjg(u20);
  // [[conj u01, conj u02], [-u02, u01]] (u11, u12) = (e, f)
  const cx<T> u11 = id * (e * u01 - conjg(u02) * f);
  const cx<T> u12 = id * (conjg(u01) * f + u02 * e);
  U[0][0] = u00;
  U[0][1] = u01;
  U[0][2] = u02;
  U[1][0] = u10;
  U[1][1] = u11;
  U[1][2] = u12;
  U[2][0] = u20;
  U[2][1] = conjg(u02 * u10 - u00 * u12);
  U[2][2] = conjg(u00 * u11 - u01 * u10);
}

// Link U_mu at site i of one parity; 12-real form rebuilds row 2 = conj(row0 x row1).
#ifndef LQCD_LINK_STREAM
#define LQCD_LINK_STREAM true
#endif
template <typename S, int R>
__device__ __forceinline__ void load_link(const void *base, long Vh, long i, cx<typename Math<S>::T> (&U)[3][3]) {
  using T = typename Math<S>::T;
  S raw[R];
  load_reals<S, R, LQCD_LINK_STREAM>(base, Vh, i, raw);
  if constexpr (R == 8) {
    T v[8];
#pragma unroll
    for (int k = 0; k < 8; k++) v[k] = (T)to_f(raw[k]);
    rebuild_link8<T>(v, U);
    return;
  }
#pragma unroll
  for (int k = 0; k < R / 6; k++)
#pragma unroll
    for (int c = 0; c < 3; c++) U[k][c] = mk<T>((T)to_f(raw[6 * k + 2 * c]), (T)to_f(raw[6 * k + 2 * c + 1]));
  if (R == 12) {
#pragma unroll
    for (int j = 0; j < 3; j++) {
      const int a = (j + 1) % 3, b = (j + 2) % 3;
      cx<T> t = U[0][a] * U[1][b] - U[0][b] * U[1][a];
      U[2][j] = conjg(t);
    }
  }
}

// Packed Hermitian 6x6 block: 6 real diagonal entries, then the 15 complex
// entries below the diagonal in row order (1,0),(2,0),(2,1),(3,0),...,(5,4).
template <typename T>
__device__ __forceinline__ void herm6_mul(const T (&m)[36], const cx<T> (&v)[6], cx<T> (&o)[6]) {
#pragma unroll
  for (int i = 0; i < 6; i++) o[i] = m[i] * v[i];
#pragma unroll
  for (int i = 1; i < 6; i++)
#pragma unroll
    for (int j = 0; j < i; j++) {
      const int k = 6 + 2 * (i * (i - 1) / 2 + j);
      cx<T> l = mk<T>(m[k], m[k + 1]);
      o[i] = cmadd(l, v[j], o[i]);   // L_ij v_j
      o[j] = cjmadd(l, v[i], o[j]);  // conj(L_ij) v_i
    }
}

// The same product in double-float, with compensated accumulators for the
// six outputs (each a sum of eleven real products per component).
__device__ __forceinline__ void herm6_mul(const df (&m)[36], const cx<df> (&v)[6], cx<df> (&o)[6]) {
  dfacc re[6], im[6];
#pragma unroll
  for (int i = 0; i < 6; i++) {
    re[i] = dfacc{0.0f, 0.0f};
    im[i] = dfacc{0.0f, 0.0f};
    dfacc_madd(re[i], m[i], v[i].r);
    dfacc_madd(im[i], m[i], v[i].i);
  }
#pragma unroll
  for (int i = 1; i < 6; i++)
#pragma unroll
    for (int j = 0; j < i; j++) {
      const int k = 6 + 2 * (i * (i - 1) / 2 + j);
      const df lr = m[k], li = m[k + 1];
      dfacc_madd(re[i], lr, v[j].r);  // L_ij v_j
      dfacc_madd(re[i], -li, v[j].i);
      dfacc_madd(im[i], lr, v[j].i);
      dfacc_madd(im[i], li, v[j].r);
      dfacc_madd(re[j], lr, v[i].r);  // conj(L_ij) v_i
      dfacc_madd(re[j], li, v[i].i);
      dfacc_madd(im[j], lr, v[i].i);
      dfacc_madd(im[j], -li, v[i].r);
    }
#pragma unroll
  for (int i = 0; i < 6; i++) o[i] = mk<df>(dfacc_value(re[i]), dfacc_value(im[i]));
}

// Clover storage of one parity: two blocks of 36 reals, block-major,
// [blk][words][Vh], plus one FP32 scale per site for FP16/BF16.
template <typename S>
__device__ __forceinline__ typename Math<S>::T load_clover_block(const void *base, const float *scale, long Vh,
                                                                 long i, int blk, typename Math<S>::T (&m)[36]) {
  using T = typename Math<S>::T;
  using Wd = Words<S, 36>;
  const void *b = reinterpret_cast<const char *>(base) + (long)blk * Wd::NW * Vh * Wd::W;
  T sc = (T)1;
  if constexpr (IsHalf<S>::value) {
    static_assert(Wd::W == 8 && Wd::NW == 9, "FP16/BF16 clover blocks are nine 8-byte words");
    const uint2 *p = reinterpret_cast<const uint2 *>(b);
#pragma unroll
    for (int w = 0; w < 9; w++) {
      const uint2 v = ldcs_word(p + (long)w * Vh + i);
      const float2 x = unpack_pair<S>(v.x), y = unpack_pair<S>(v.y);
      m[4 * w] = x.x;
      m[4 * w + 1] = x.y;
      m[4 * w + 2] = y.x;
      m[4 * w + 3] = y.y;
    }
    sc = (T)__ldg(scale + i);
  } else {
    S raw[36];
    load_reals<S, 36, true>(b, Vh, i, raw);
#pragma unroll
    for (int k = 0; k < 36; k++) m[k] = (T)to_f(raw[k]);
  }
  return sc;  // the FP16/BF16 scale, applied to the products by the caller
}

// out = M psi with M = diag(block+, block-) acting on (spins 0,1) and (2,3);
// the storage scale multiplies the 6 outputs of each block, not its 36 entries
template <typename S, int NR>
__device__ __forceinline__ void clover_apply(const void *base, const float *scale, long Vh, long i,
                                             cx<typename Math<S>::T> (&psi)[NR][4][3]) {
  using T = typename Math<S>::T;
#pragma unroll
  for (int blk = 0; blk < 2; blk++) {
    T m[36];
    const T sc = load_clover_block<S>(base, scale, Vh, i, blk, m);
#pragma unroll
    for (int r = 0; r < NR; r++) {
      cx<T> v[6], o[6];
#pragma unroll
      for (int k = 0; k < 6; k++) v[k] = psi[r][2 * blk + k / 3][k % 3];
      herm6_mul(m, v, o);
#pragma unroll
      for (int k = 0; k < 6; k++) psi[r][2 * blk + k / 3][k % 3] = IsHalf<S>::value ? sc * o[k] : o[k];
    }
  }
}

// ---------------------------------------------------------------------------
// spin projection and reconstruction, (1 + s g_mu), s = +-1
// ---------------------------------------------------------------------------
// s * a for the sign s = +-1 (double-float: two exact multiplications)
template <typename T> __device__ __forceinline__ T sgn_mul(T s, T a) { return s * a; }
template <typename T> __device__ __forceinline__ cx<T> sgn_mul(T s, cx<T> a) { return {sgn_mul(s, a.r), sgn_mul(s, a.i)}; }

template <typename T>
__device__ __forceinline__ void project(int mu, T s, const cx<T> (&p)[4][3], cx<T> (&h)[2][3]) {
#pragma unroll
  for (int c = 0; c < 3; c++) {
    switch (mu) {
      case 0:  // B = [[0, i], [i, 0]]
        h[0][c] = p[0][c] + sgn_mul(s, times_i(p[3][c]));
        h[1][c] = p[1][c] + sgn_mul(s, times_i(p[2][c]));
        break;
      case 1:  // B = [[0, -1], [1, 0]]
        h[0][c] = p[0][c] - sgn_mul(s, p[3][c]);
        h[1][c] = p[1][c] + sgn_mul(s, p[2][c]);
        break;
      case 2:  // B = [[i, 0], [0, -i]]
        h[0][c] = p[0][c] + sgn_mul(s, times_i(p[2][c]));
        h[1][c] = p[1][c] - sgn_mul(s, times_i(p[3][c]));
        break;
      default:  // B = 1
        h[0][c] = p[0][c] + sgn_mul(s, p[2][c]);
        h[1][c] = p[1][c] + sgn_mul(s, p[3][c]);
        break;
    }
  }
}

// The projection of FP16/BF16 spinors on their stored (normalised) pairs:
// h = u + c l with c in {+-1, +-i} is one packed multiply-add per colour and
// spin (the products by +-1 are exact, so each component is rounded once, at
// the storage precision), and only the six projected colour components are
// converted to FP32 instead of all twelve.  u[3 a + c] holds (re, im) of
// psi[a][c]; s is the projection sign (with g5 on the input folded in).
template <typename S>
__device__ __forceinline__ void project_packed(int mu, float s, const unsigned (&u)[12], cx<float> (&h)[2][3]) {
  using PP = PackedPair<S>;
  using T2 = typename PP::type;
  const T2 sp = PP::make(s, s), sm = PP::make(-s, -s);
  const T2 ip = PP::make(-s, s), im = PP::make(s, -s);  // s i z = (-s z.im, s z.re)
#pragma unroll
  for (int c = 0; c < 3; c++) {
    const T2 p0 = PP::from(u[c]), p1 = PP::from(u[3 + c]), p2 = PP::from(u[6 + c]), p3 = PP::from(u[9 + c]);
    T2 r0, r1;
    switch (mu) {
      case 0:  // h0 = p0 + s i p3, h1 = p1 + s i p2
        r0 = __hfma2(__lowhigh2highlow(p3), ip, p0);
        r1 = __hfma2(__lowhigh2highlow(p2), ip, p1);
        break;
      case 1:  // h0 = p0 - s p3, h1 = p1 + s p2
        r0 = __hfma2(p3, sm, p0);
        r1 = __hfma2(p2, sp, p1);
        break;
      case 2:  // h0 = p0 + s i p2, h1 = p1 - s i p3
        r0 = __hfma2(__lowhigh2highlow(p2), ip, p0);
        r1 = __hfma2(__lowhigh2highlow(p3), im, p1);
        break;
      default:  // h0 = p0 + s p2, h1 = p1 + s p3
        r0 = __hfma2(p2, sp, p0);
        r1 = __hfma2(p3, sp, p1);
        break;
    }
    const float2 a = PP::f2(r0), b = PP::f2(r1);
    h[0][c] = mk<float>(a.x, a.y);
    h[1][c] = mk<float>(b.x, b.y);
  }
}

// FP16/BF16 hop in packed FP32x2 arithmetic (sm_100+ __ffma2_rn): the two
// projected half-spinors h0, h1 sit in the two lanes of each float2 (real
// parts together, imaginary parts together), so U h0 and U h1 take one
// instruction per link-entry product (the entry broadcast to both lanes), and
// the accumulators pair spins (0, 1) and (2, 3): f (U h) adds to the upper
// pair as is, and to the lower pair as is (mu = 3) or lane-signed and
// re/im-exchanged (mu = 2); mu = 0, 1 exchange the two spins, which packed
// operands cannot, and stay scalar.  Each product sums the real-part terms
// and the imaginary-part terms apart (A - B, C + D) where the scalar
// link_mul interleaves them: the same products, another rounding order.
__device__ __forceinline__ float2 pr_bc(float v) { return make_float2(v, v); }
__device__ __forceinline__ void hop_pair_accumulate(int mu, bool dag, float s, float f, const cx<float> (&U)[3][3],
                                                    const cx<float> (&h)[2][3], float2 (&aur)[3], float2 (&aui)[3],
                                                    float2 (&alr)[3], float2 (&ali)[3]) {
  float2 hr[3], hi[3];
#pragma unroll
  for (int c = 0; c < 3; c++) {
    hr[c] = make_float2(h[0][c].r, h[1][c].r);
    hi[c] = make_float2(h[0][c].i, h[1][c].i);
  }
  const float2 ff = pr_bc(f);
  const float fs = f * s;
#pragma unroll
  for (int r = 0; r < 3; r++) {
    float2 A = pr_bc(0.0f), B = pr_bc(0.0f), C = pr_bc(0.0f), D = pr_bc(0.0f);
#pragma unroll
    for (int c = 0; c < 3; c++) {
      const cx<float> u = dag ? U[c][r] : U[r][c];
      const float2 ur = pr_bc(u.r), ui = pr_bc(u.i);
      A = __ffma2_rn(ur, hr[c], A);
      B = __ffma2_rn(ui, hi[c], B);
      C = __ffma2_rn(ur, hi[c], C);
      D = __ffma2_rn(ui, hr[c], D);
    }
    // U h: (A - B, C + D); U^dag h (entries conj(U[c][r])): (A + B, C - D)
    const float2 nB = make_float2(-B.x, -B.y), nD = make_float2(-D.x, -D.y);
    const float2 tr = __fadd2_rn(A, dag ? B : nB), ti = __fadd2_rn(C, dag ? nD : D);
    aur[r] = __ffma2_rn(ff, tr, aur[r]);
    aui[r] = __ffma2_rn(ff, ti, aui[r]);
    switch (mu) {
      case 0:  // spin 2 += -i fs t1, spin 3 += -i fs t0
        alr[r].x = fmaf(fs, ti.y, alr[r].x);
        ali[r].x = fmaf(-fs, tr.y, ali[r].x);
        alr[r].y = fmaf(fs, ti.x, alr[r].y);
        ali[r].y = fmaf(-fs, tr.x, ali[r].y);
        break;
      case 1:  // spin 2 += fs t1, spin 3 -= fs t0
        alr[r].x = fmaf(fs, tr.y, alr[r].x);
        ali[r].x = fmaf(fs, ti.y, ali[r].x);
        alr[r].y = fmaf(-fs, tr.x, alr[r].y);
        ali[r].y = fmaf(-fs, ti.x, ali[r].y);
        break;
      case 2:  // spin 2 += -i fs t0, spin 3 += i fs t1
        alr[r] = __ffma2_rn(make_float2(fs, -fs), ti, alr[r]);
        ali[r] = __ffma2_rn(make_float2(-fs, fs), tr, ali[r]);
        break;
      default:  // spin 2 += fs t0, spin 3 += fs t1
        alr[r] = __ffma2_rn(pr_bc(fs), tr, alr[r]);
        ali[r] = __ffma2_rn(pr_bc(fs), ti, ali[r]);
        break;
    }
  }
}

// acc += f * reconstruct(h): f folds the storage scale of the neighbour and
// the boundary sign into the FMAs of the accumulation
template <typename T>
__device__ __forceinline__ void reconstruct(int mu, T s, T f, const cx<T> (&h)[2][3], cx<T> (&acc)[4][3]) {
  const T fs = f * s;
#pragma unroll
  for (int c = 0; c < 3; c++) {
    acc[0][c] = mk<T>(fma(f, h[0][c].r, acc[0][c].r), fma(f, h[0][c].i, acc[0][c].i));
    acc[1][c] = mk<T>(fma(f, h[1][c].r, acc[1][c].r), fma(f, h[1][c].i, acc[1][c].i));
    switch (mu) {
      case 0:  // s B^dag h, B^dag = [[0, -i], [-i, 0]]: lower0 -= s i h1, lower1 -= s i h0
        acc[2][c] = mk<T>(fma(fs, h[1][c].i, acc[2][c].r), fma(-fs, h[1][c].r, acc[2][c].i));
        acc[3][c] = mk<T>(fma(fs, h[0][c].i, acc[3][c].r), fma(-fs, h[0][c].r, acc[3][c].i));
        break;
      case 1:  // B^dag = [[0, 1], [-1, 0]]: lower0 += s h1, lower1 -= s h0
        acc[2][c] = mk<T>(fma(fs, h[1][c].r, acc[2][c].r), fma(fs, h[1][c].i, acc[2][c].i));
        acc[3][c] = mk<T>(fma(-fs, h[0][c].r, acc[3][c].r), fma(-fs, h[0][c].i, acc[3][c].i));
        break;
      case 2:  // B^dag = [[-i, 0], [0, i]]: lower0 -= s i h0, lower1 += s i h1
        acc[2][c] = mk<T>(fma(fs, h[0][c].i, acc[2][c].r), fma(-fs, h[0][c].r, acc[2][c].i));
        acc[3][c] = mk<T>(fma(-fs, h[1][c].i, acc[3][c].r), fma(fs, h[1][c].r, acc[3][c].i));
        break;
      default:  // B^dag = 1
        acc[2][c] = mk<T>(fma(fs, h[0][c].r, acc[2][c].r), fma(fs, h[0][c].i, acc[2][c].i));
        acc[3][c] = mk<T>(fma(fs, h[1][c].r, acc[3][c].r), fma(fs, h[1][c].i, acc[3][c].i));
        break;
    }
  }
}

// The same in double-float for f = +-1 (df storage carries no scale): sign
// flips are exact, and the sixteen additions into each accumulator over the
// eight directions take the lazy TwoSum form (8 FP32 operations, not 15)
__device__ __forceinline__ void reconstruct(int mu, df s, df f, const cx<df> (&h)[2][3], cx<df> (&acc)[4][3]) {
  const df fs = sgn_mul(f, s);
  auto add = [](cx<df> &a, df xr, df xi) { a = mk<df>(df_lazy_add(a.r, xr), df_lazy_add(a.i, xi)); };
#pragma unroll
  for (int c = 0; c < 3; c++) {
    add(acc[0][c], sgn_mul(f, h[0][c].r), sgn_mul(f, h[0][c].i));
    add(acc[1][c], sgn_mul(f, h[1][c].r), sgn_mul(f, h[1][c].i));
    switch (mu) {
      case 0:
        add(acc[2][c], sgn_mul(fs, h[1][c].i), -sgn_mul(fs, h[1][c].r));
        add(acc[3][c], sgn_mul(fs, h[0][c].i), -sgn_mul(fs, h[0][c].r));
        break;
      case 1:
        add(acc[2][c], sgn_mul(fs, h[1][c].r), sgn_mul(fs, h[1][c].i));
        add(acc[3][c], -sgn_mul(fs, h[0][c].r), -sgn_mul(fs, h[0][c].i));
        break;
      case 2:
        add(acc[2][c], sgn_mul(fs, h[0][c].i), -sgn_mul(fs, h[0][c].r));
        add(acc[3][c], -sgn_mul(fs, h[1][c].i), sgn_mul(fs, h[1][c].r));
        break;
      default:
        add(acc[2][c], sgn_mul(fs, h[0][c].r), sgn_mul(fs, h[0][c].i));
        add(acc[3][c], sgn_mul(fs, h[1][c].r), sgn_mul(fs, h[1][c].i));
        break;
    }
  }
}

template <typename T>
__device__ __forceinline__ void link_mul(const cx<T> (&U)[3][3], bool dag, const cx<T> (&h)[2][3],
                                         cx<T> (&o)[2][3]) {
#pragma unroll
  for (int a = 0; a < 2; a++)
#pragma unroll
    for (int r = 0; r < 3; r++) {
      cx<T> t = mk<T>(0, 0);
#pragma unroll
      for (int c = 0; c < 3; c++) t = dag ? cjmadd(U[c][r], h[a][c], t) : cmadd(U[r][c], h[a][c], t);
      o[a][r] = t;
    }
}

// The same product in double-float with compensated accumulators.
__device__ __forceinline__ void link_mul(const cx<df> (&U)[3][3], bool dag, const cx<df> (&h)[2][3],
                                         cx<df> (&o)[2][3]) {
#pragma unroll
  for (int a = 0; a < 2; a++)
#pragma unroll
    for (int r = 0; r < 3; r++) {
      dfacc re{0.0f, 0.0f}, im{0.0f, 0.0f};
#pragma unroll
      for (int c = 0; c < 3; c++) {
        const cx<df> u = dag ? U[c][r] : U[r][c];
        const cx<df> v = h[a][c];
        dfacc_madd(re, u.r, v.r);
        dfacc_madd(re, dag ? u.i : -u.i, v.i);
        dfacc_madd(im, u.r, v.i);
        dfacc_madd(im, dag ? -u.i : u.i, v.r);
      }
      o[a][r] = mk<df>(dfacc_value(re), dfacc_value(im));
    }
}

// ---------------------------------------------------------------------------
// Software-pipelined neighbour gathers (LQCD_PIPE): the link and neighbour
// spinor of direction k + 2 are copied global -> shared by cp.async (LDGSTS)
// while direction k is computed, so the loads in flight hold no registers.
// Every thread owns its staging slots; no block barrier is involved.
// ---------------------------------------------------------------------------
#ifndef LQCD_PIPE
#define LQCD_PIPE 1
#endif
#ifndef LQCD_PIPE_UNROLL
#define LQCD_PIPE_UNROLL 8
#endif
constexpr int kPipeUnroll = LQCD_PIPE_UNROLL;  // pragma arguments are not macro-expanded

// global -> shared copy of B bytes; `dep` is an unused operand that makes the
// copy wait for a value combined from every word of the slot's previous
// contents, so the reads of that slot are complete before it is overwritten
template <int B>
__device__ __forceinline__ void cp_async_after(void *smem, const void *gmem, unsigned dep) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(sa), "l"(gmem), "n"(B), "r"(dep) : "memory");
}
template <typename W> __device__ __forceinline__ unsigned first_bits(const W &v) {
  return *reinterpret_cast<const unsigned *>(&v);
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

template <typename S, int R, int TB> struct HopStage {
  using WS = Words<S, 24>;
  using WL = Words<S, R>;
  typename WordT<WS::W>::type sp[2][WS::NW][TB];
  typename WordT<WL::W>::type ln[2][WL::NW][TB];
  float sc[2][TB];
};

// the hop sum of one right-hand side (NR = 1) with a two-deep cp.async pipeline
template <typename S, int R, int TB>
__device__ __forceinline__ void hop_pipelined(const DslashParams &P, long h, int p, int rg, const Coords &xc,
                                              cx<typename Math<S>::T> (&acc)[4][3]) {
  using T = typename Math<S>::T;
  using St = HopStage<S, R, TB>;
  using WS = typename St::WS;
  using WL = typename St::WL;
  __shared__ St st;
  const int tid = threadIdx.x;
  const long Vh = P.g.Vh;
  const char *spb = reinterpret_cast<const char *>(rhs_base<S>(P.in.data, P.in.rhs_words, rg));
  const float *scb = IsHalf<S>::value ? P.in.scale + (long)rg * Vh : nullptr;
  auto issue = [&](int k, unsigned dep) {
    const int mu = k >> 1, b = k & 1;
    long n = neighbour(P.g, xc, h, mu, (k & 1) ? -1 : +1);
    LQCD_CHECK_INDEX(P, n);
#pragma unroll
    for (int w = 0; w < WS::NW; w++) cp_async_after<WS::W>(&st.sp[b][w][tid], spb + ((long)w * Vh + n) * WS::W, dep);
    if constexpr (IsHalf<S>::value) cp_async_after<4>(&st.sc[b][tid], scb + n, dep);
    const char *lb = reinterpret_cast<const char *>((k & 1) ? P.links[mu][1 - p] : P.links[mu][p]);
    const long li = (k & 1) ? n : h;
#pragma unroll
    for (int w = 0; w < WL::NW; w++) cp_async_after<WL::W>(&st.ln[b][w][tid], lb + ((long)w * Vh + li) * WL::W, dep);
    cp_async_commit();
  };
  issue(0, 0u);
  issue(1, 0u);
  // FP16/BF16: the accumulators paired over spins (0, 1) and (2, 3), see hop_pair_accumulate
  float2 aur[3], aui[3], alr[3], ali[3];
  if constexpr (IsHalf<S>::value) {
#pragma unroll
    for (int c = 0; c < 3; c++) {
      aur[c] = make_float2((float)acc[0][c].r, (float)acc[1][c].r);
      aui[c] = make_float2((float)acc[0][c].i, (float)acc[1][c].i);
      alr[c] = make_float2((float)acc[2][c].r, (float)acc[3][c].r);
      ali[c] = make_float2((float)acc[2][c].i, (float)acc[3][c].i);
    }
  }
#pragma unroll kPipeUnroll
  for (int k = 0; k < 8; k++) {
    const int mu = k >> 1, dir = (k & 1) ? -1 : +1, b = k & 1;
    if (k < 7)
      cp_async_wait<1>();
    else
      cp_async_wait<0>();
    S raw[24];
    unsigned uw[12];  // FP16/BF16: the spinor as its twelve stored (re, im) pairs
    unsigned dep = 0;
#pragma unroll
    for (int w = 0; w < WS::NW; w++) {
      const auto v = st.sp[b][w][tid];
      dep |= first_bits(v);
      if constexpr (IsHalf<S>::value) {
        static_assert(WS::W == 16, "FP16/BF16 spinors are three 16-byte words");
        const unsigned *q = reinterpret_cast<const unsigned *>(&v);
#pragma unroll
        for (int j = 0; j < 4; j++) uw[w * 4 + j] = q[j];
      } else {
        const S *q = reinterpret_cast<const S *>(&v);
#pragma unroll
        for (int j = 0; j < WS::PER; j++) raw[w * WS::PER + j] = q[j];
      }
    }
    S lraw[R];
    unsigned lw[R / 2];  // FP16/BF16: the link's (re, im) pairs
#pragma unroll
    for (int w = 0; w < WL::NW; w++) {
      const auto v = st.ln[b][w][tid];
      dep |= first_bits(v);
      if constexpr (IsHalf<S>::value) {
        const unsigned *q = reinterpret_cast<const unsigned *>(&v);
#pragma unroll
        for (int j = 0; j < WL::PER / 2; j++) lw[w * (WL::PER / 2) + j] = q[j];
      } else {
        const S *q = reinterpret_cast<const S *>(&v);
#pragma unroll
        for (int j = 0; j < WL::PER; j++) lraw[w * WL::PER + j] = q[j];
      }
    }
    T f = (T)1;
    if constexpr (IsHalf<S>::value) {
      f = (T)st.sc[b][tid];
      dep |= __float_as_uint(f);
    }
    cx<T> U[3][3];
    if constexpr (R == 8) {
      T v8[8];
#pragma unroll
      for (int k = 0; k < 4; k++) {
        if constexpr (IsHalf<S>::value) {
          const float2 e = unpack_pair<S>(lw[k]);
          v8[2 * k] = e.x;
          v8[2 * k + 1] = e.y;
        } else {
          v8[2 * k] = (T)to_f(lraw[2 * k]);
          v8[2 * k + 1] = (T)to_f(lraw[2 * k + 1]);
        }
      }
      rebuild_link8<T>(v8, U);
    } else {
#pragma unroll
      for (int r = 0; r < R / 6; r++)
#pragma unroll
        for (int c = 0; c < 3; c++) {
          if constexpr (IsHalf<S>::value) {
            const float2 e = unpack_pair<S>(lw[3 * r + c]);
            U[r][c] = mk<T>(e.x, e.y);
          } else {
            U[r][c] = mk<T>((T)to_f(lraw[6 * r + 2 * c]), (T)to_f(lraw[6 * r + 2 * c + 1]));
          }
        }
    }
    if (R == 12) {
#pragma unroll
      for (int j = 0; j < 3; j++) {
        const int a = (j + 1) % 3, bb = (j + 2) % 3;
        cx<T> t = U[0][a] * U[1][bb] - U[0][bb] * U[1][a];
        U[2][j] = conjg(t);
      }
    }
    // the slot is free once its values are in registers: the next copy into it
    // depends on all of its words
    if (k + 2 < 8) issue(k + 2, dep);
    const bool wrap = (mu == 3) && P.g.tbc && (dir > 0 ? xc.x[3] == P.g.L[3] - 1 : xc.x[3] == 0);
    if (wrap) f = -f;
    const T s = dir > 0 ? (T)-1 : (T)1;
    cx<T> hh[2][3], uh[2][3];
    if constexpr (IsHalf<S>::value) {
      // g5 on the input negates the lower spins: the projection sign flips
      project_packed<S>(mu, P.g5_in ? -s : s, uw, hh);
    } else {
      cx<T> psi[4][3];
#pragma unroll
      for (int a = 0; a < 4; a++)
#pragma unroll
        for (int c = 0; c < 3; c++) psi[a][c] = mk<T>((T)to_f(raw[6 * a + 2 * c]), (T)to_f(raw[6 * a + 2 * c + 1]));
      if (P.g5_in) {
#pragma unroll
        for (int c = 0; c < 3; c++) {
          psi[2][c] = (T)-1 * psi[2][c];
          psi[3][c] = (T)-1 * psi[3][c];
        }
      }
      project<T>(mu, s, psi, hh);
    }
    if constexpr (IsHalf<S>::value) {
      hop_pair_accumulate(mu, dir < 0, s, f, U, hh, aur, aui, alr, ali);
    } else {
      link_mul(U, dir < 0, hh, uh);
      reconstruct(mu, s, f, uh, acc);
    }
  }
  if constexpr (IsHalf<S>::value) {
#pragma unroll
    for (int c = 0; c < 3; c++) {
      acc[0][c] = mk<T>(aur[c].x, aui[c].x);
      acc[1][c] = mk<T>(aur[c].y, aui[c].y);
      acc[2][c] = mk<T>(alr[c].x, ali[c].x);
      acc[3][c] = mk<T>(alr[c].y, ali[c].y);
    }
  }
}

// The hop sum with the eight directions in a rolled loop: the double-float
// kernel is ~15 k instructions per site when unrolled, and ncu shows it
// stalled on instruction fetch ("no_instruction") more than on anything else;
// one direction's code stays resident in the instruction cache.
template <typename S, int R, int NR>
__device__ __forceinline__ void hop_rolled(const DslashParams &P, long h, int p, int rg, const Coords &xc,
                                           cx<typename Math<S>::T> (&acc)[NR][4][3]) {
  using T = typename Math<S>::T;
#pragma unroll 1
  for (int k = 0; k < 8; k++) {
    const int mu = k >> 1, dir = (k & 1) ? -1 : +1;
    long n = neighbour(P.g, xc, h, mu, dir);
    LQCD_CHECK_INDEX(P, n);
    const bool wrap = (mu == 3) && P.g.tbc && (dir > 0 ? xc.x[3] == P.g.L[3] - 1 : xc.x[3] == 0);
    const T s = dir > 0 ? (T)-1 : (T)1;
    cx<T> U[3][3];
    if (dir > 0)
      load_link<S, R>(P.links[mu][p], P.g.Vh, h, U);
    else
      load_link<S, R>(P.links[mu][1 - p], P.g.Vh, n, U);
#pragma unroll
    for (int r = 0; r < NR; r++) {
      cx<T> psi[4][3];
      T f = load_spinor_raw<S>(P.in, P.g.Vh, rg * NR + r, n, psi);
      if (wrap) f = -f;
      if (P.g5_in) {
#pragma unroll
        for (int c = 0; c < 3; c++) {
          psi[2][c] = (T)-1 * psi[2][c];
          psi[3][c] = (T)-1 * psi[3][c];
        }
      }
      cx<T> hh[2][3], uh[2][3];
      project<T>(mu, s, psi, hh);
      link_mul(U, dir < 0, hh, uh);
      reconstruct(mu, s, f, uh, acc[r]);
    }
  }
}

// ---------------------------------------------------------------------------
// the kernel
// ---------------------------------------------------------------------------
// Launch shape per storage type: threads per block and the minimum number
// of resident blocks per SM promised to the register allocator.  Without the
// cp.async pipeline the kernel was latency-bound (long-scoreboard stalls) and
// ran best with many small register-capped blocks (FP32: ten 64-thread blocks
// per SM, K2a/K2b 0.147/0.162 ms at 32^3x64; FP16: sixteen, 0.117/0.128).
// With the gathers staged through shared memory the loads in flight cost no
// registers, and a looser cap pays: FP32 eight blocks (128 registers)
// 0.137/0.150, FP16 ten (102 registers) 0.105/0.113, BF16 0.116/0.122.
#ifndef LQCD_T64
#define LQCD_T64 128
#endif
#ifndef LQCD_M64
#define LQCD_M64 1
#endif
#ifndef LQCD_T32
#define LQCD_T32 64
#endif
#ifndef LQCD_M32
#define LQCD_M32 8
#endif
#ifndef LQCD_T16
#define LQCD_T16 64
#endif
#ifndef LQCD_M16
#define LQCD_M16 10
#endif
// Kernels carrying several right-hand sides per thread need their registers:
// they keep 128 threads and no cap.
template <typename S, int NR, int MODE> struct LaunchCfg {
  static constexpr int threads = NR > 1 ? 128 : LQCD_T16, min_blocks = NR > 1 ? 1 : LQCD_M16;
};
template <int NR, int MODE> struct LaunchCfg<float, NR, MODE> {
  static constexpr int threads = NR > 1 ? 128 : LQCD_T32, min_blocks = NR > 1 ? 1 : LQCD_M32;
};
template <int NR, int MODE> struct LaunchCfg<double, NR, MODE> {
  static constexpr int threads = NR > 1 ? 128 : LQCD_T64, min_blocks = NR > 1 ? 1 : LQCD_M64;
};
// Double-float keeps ~200 live FP32 registers per site; measured at 32^3x64
// (K2a / K2b ms): 255 registers, 8 warps per SM: 1.89 / 1.92; 168 registers
// (three 128-thread blocks): 1.31 / 1.40; 128 registers (four 128-thread
// blocks): 1.20 / 1.61, the hop-only kernel tolerating its ~400 B of spills
// while the clover-and-local kernel's 650 B cost more than the extra warps
// gain; 204 registers (five 64-thread blocks): 1.30 / 1.39.  With the
// compensated accumulators and the rolled direction loop (far fewer live
// values) the balance moved: 128 registers 0.86 / 0.93, 204 registers 0.72 /
// 0.74, 170 registers (six 64-thread blocks) 0.71 / 0.74, the choice for both.
#ifndef LQCD_TDF_HOP
#define LQCD_TDF_HOP 64
#endif
#ifndef LQCD_MDF_HOP
#define LQCD_MDF_HOP 6
#endif
#ifndef LQCD_TDF_LOC
#define LQCD_TDF_LOC 64
#endif
#ifndef LQCD_MDF_LOC
#define LQCD_MDF_LOC 6
#endif
template <int NR, int MODE> struct LaunchCfg<df, NR, MODE> {
  static constexpr bool hop_only = MODE == MODE_HOP || MODE == MODE_HOP_AINV;
  static constexpr int threads = NR > 1 ? 128 : (hop_only ? LQCD_TDF_HOP : LQCD_TDF_LOC);
  static constexpr int min_blocks = NR > 1 ? 1 : (hop_only ? LQCD_MDF_HOP : LQCD_MDF_LOC);
};

template <typename S, int R, int MODE, int NR>
__global__ void __launch_bounds__(LaunchCfg<S, NR, MODE>::threads, LaunchCfg<S, NR, MODE>::min_blocks) dslash_kernel(const __grid_constant__ DslashParams P) {
  using T = typename Math<S>::T;
  const long h = P.h0 + (long)blockIdx.x * blockDim.x + threadIdx.x;
  const int rg = blockIdx.y;  // right-hand-side group
  const bool valid = h < P.h1;
  const int p = P.out_parity;
  using RT = typename RedVal<T>::type;
  RT nrm[NR];
#pragma unroll
  for (int r = 0; r < NR; r++) nrm[r] = RT(0);

  if (valid) {
    cx<T> acc[NR][4][3];
#pragma unroll
    for (int r = 0; r < NR; r++)
#pragma unroll
      for (int a = 0; a < 4; a++)
#pragma unroll
        for (int c = 0; c < 3; c++) acc[r][a][c] = mk<T>(0, 0);

    const bool hop = P.in.data != nullptr && P.beta != 0.0;
    constexpr bool kPipe = LQCD_PIPE && NR == 1 && (std::is_same<S, float>::value || IsHalf<S>::value);
    if (hop && kPipe) {
      const Coords xc = site_coords(P.g, h, p);
      hop_pipelined<S, R, LaunchCfg<S, NR, MODE>::threads>(P, h, p, rg, xc, acc[0]);
    } else if (hop && std::is_same<S, df>::value) {
      const Coords xc = site_coords(P.g, h, p);
      hop_rolled<S, R, NR>(P, h, p, rg, xc, acc);
    } else if (hop) {
      const Coords xc = site_coords(P.g, h, p);
#pragma unroll
      for (int mu = 0; mu < 4; mu++) {
#pragma unroll
        for (int d = 0; d < 2; d++) {
          const int dir = d == 0 ? +1 : -1;
          long n = neighbour(P.g, xc, h, mu, dir);
          LQCD_CHECK_INDEX(P, n);
          const bool wrap = (mu == 3) && P.g.tbc && (dir > 0 ? xc.x[3] == P.g.L[3] - 1 : xc.x[3] == 0);
          const T s = dir > 0 ? (T)-1 : (T)1;  // forward (1 - g_mu), backward (1 + g_mu)
          cx<T> U[3][3];
          if (dir > 0)
            load_link<S, R>(P.links[mu][p], P.g.Vh, h, U);
          else
            load_link<S, R>(P.links[mu][1 - p], P.g.Vh, n, U);
#pragma unroll
          for (int r = 0; r < NR; r++) {
            cx<T> psi[4][3];
            T f = load_spinor_raw<S>(P.in, P.g.Vh, rg * NR + r, n, psi);
            if (wrap) f = -f;
            if (P.g5_in) {
#pragma unroll
              for (int c = 0; c < 3; c++) {
                psi[2][c] = (T)-1 * psi[2][c];
                psi[3][c] = (T)-1 * psi[3][c];
              }
            }
            cx<T> hh[2][3], uh[2][3];
            project<T>(mu, s, psi, hh);
            link_mul(U, dir < 0, hh, uh);
            reconstruct(mu, s, f, uh, acc[r]);
          }
        }
      }
    }
    if (hop) {
      const T beta = (T)P.beta;
#pragma unroll
      for (int r = 0; r < NR; r++)
#pragma unroll
        for (int a = 0; a < 4; a++)
#pragma unroll
          for (int c = 0; c < 3; c++) {
            const T sg = (P.g5_hop && a >= 2) ? -beta : beta;
            acc[r][a][c] = sg * acc[r][a][c];
          }
    }

    // ---- epilogue -------------------------------------------------------
    if (MODE == MODE_LOCAL_IDENT || MODE == MODE_FOLDED_AINV || MODE == MODE_LOCAL_A || MODE == MODE_CHEB) {
      const T alpha = (T)P.alpha;
      cx<T> x[NR][4][3];
#pragma unroll
      for (int r = 0; r < NR; r++) load_spinor<S>(P.xloc, P.g.Vh, rg * NR + r, h, x[r]);
      if (MODE == MODE_LOCAL_A) clover_apply<S, NR>(P.lmat, P.lmat_scale, P.g.Vh, h, x);
#pragma unroll
      for (int r = 0; r < NR; r++)
#pragma unroll
        for (int a = 0; a < 4; a++)
#pragma unroll
          for (int c = 0; c < 3; c++) acc[r][a][c] = acc[r][a][c] + alpha * x[r][a][c];
    }
    if (MODE == MODE_HOP_AINV || MODE == MODE_FOLDED_AINV) clover_apply<S, NR>(P.cmat, P.cmat_scale, P.g.Vh, h, acc);
    if (P.g5_total) {
#pragma unroll
      for (int r = 0; r < NR; r++)
#pragma unroll
        for (int c = 0; c < 3; c++) {
          acc[r][2][c] = (T)-1 * acc[r][2][c];
          acc[r][3][c] = (T)-1 * acc[r][3][c];
        }
    }
    if (MODE == MODE_CHEB) {
#pragma unroll
      for (int k = 0; k < 3; k++) {
        if (P.zc[k].data == nullptr) continue;
        const T ck = (T)P.cz[k];
#pragma unroll
        for (int r = 0; r < NR; r++) {
          cx<T> zz[4][3];
          load_spinor<S>(P.zc[k], P.g.Vh, rg * NR + r, h, zz);
#pragma unroll
          for (int a = 0; a < 4; a++)
#pragma unroll
            for (int c = 0; c < 3; c++) acc[r][a][c] = acc[r][a][c] + ck * zz[a][c];
        }
      }
    }
    if (MODE != MODE_CHEB && P.z.data != nullptr) {
      const T gz = (T)P.gz;
#pragma unroll
      for (int r = 0; r < NR; r++) {
        cx<T> zz[4][3];
        load_spinor<S>(P.z, P.g.Vh, rg * NR + r, h, zz);
#pragma unroll
        for (int a = 0; a < 4; a++)
#pragma unroll
          for (int c = 0; c < 3; c++) acc[r][a][c] = zz[a][c] + gz * acc[r][a][c];
      }
    }
    const long out_words = Words<S, 24>::NW * P.g.Vh;
#pragma unroll
    for (int r = 0; r < NR; r++) {
      store_spinor<S>(P.out, P.out_scale, out_words, P.g.Vh, rg * NR + r, h, acc[r]);
      if (P.norm_partials) nrm[r] = RT(site_norm2_t<T>(acc[r]));
    }
  }
  if (P.norm_partials) block_partials<NR>(nrm, P.norm_partials, rg * NR);
}

// Host-side launcher, instantiated per storage type in dslash_<type>.cu.
template <typename S>
cudaError_t launch_dslash(const DslashParams &P, int recon, int mode, int nr, cudaStream_t st);

}  // namespace lqcd
