// Shared device-side definitions of the GB300 Wilson-clover library:
// storage types, the 16/8/4-byte word layout of site-blocked fields,
// complex arithmetic, the DeGrand-Rossi spin structure and the lattice
// geometry of one parity.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/lqcd.h"
#include "df64.cuh"

namespace lqcd {

// ---------------------------------------------------------------------------
// Storage precisions.  Arithmetic is FP64 for FP64 storage, double-float for
// DF64 storage (df, two FP32 numbers per real) and FP32 for the three others;
// FP16 and BF16 spinors and clover terms carry one FP32 scale per site (the
// largest |component|), links are stored unscaled (|U_ij|<=1).
// ---------------------------------------------------------------------------
template <typename S> struct Math { using T = float; };
template <> struct Math<double> { using T = double; };
template <> struct Math<df> { using T = df; };

template <typename S> struct IsHalf { static constexpr bool value = false; };
template <> struct IsHalf<__half> { static constexpr bool value = true; };
template <> struct IsHalf<__nv_bfloat16> { static constexpr bool value = true; };

__device__ __forceinline__ float to_f(float v) { return v; }
__device__ __forceinline__ double to_f(double v) { return v; }
__device__ __forceinline__ float to_f(__half v) { return __half2float(v); }
__device__ __forceinline__ float to_f(__nv_bfloat16 v) { return __bfloat162float(v); }

template <typename S> __device__ __forceinline__ S from_f(float v);
template <> __device__ __forceinline__ float from_f<float>(float v) { return v; }
template <> __device__ __forceinline__ __half from_f<__half>(float v) { return __float2half_rn(v); }
template <> __device__ __forceinline__ __nv_bfloat16 from_f<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }
template <typename S> __device__ __forceinline__ S from_d(double v);
template <> __device__ __forceinline__ double from_d<double>(double v) { return v; }
template <> __device__ __forceinline__ float from_d<float>(double v) { return (float)v; }
template <> __device__ __forceinline__ __half from_d<__half>(double v) { return __double2half(v); }
template <> __device__ __forceinline__ __nv_bfloat16 from_d<__nv_bfloat16>(double v) {
  return __float2bfloat16_rn((float)v);
}
template <> __device__ __forceinline__ df from_d<df>(double v) { return df(v); }

// ---------------------------------------------------------------------------
// Word layout.  A field of N reals of type S per site is stored as NW words
// of W bytes, word-major: word w of site i lives at byte
//   (w * Vs + i) * W
// so a warp reading word w of 32 consecutive sites issues one fully
// coalesced 128-bit (or 64/32-bit) access.  W is the largest of 16, 8, 4
// dividing N * sizeof(S).
// ---------------------------------------------------------------------------
template <typename S, int N> struct Words {
  static constexpr int bytes = N * (int)sizeof(S);
  static constexpr int W = (bytes % 16 == 0) ? 16 : (bytes % 8 == 0) ? 8 : 4;
  static constexpr int NW = bytes / W;
  static constexpr int PER = W / (int)sizeof(S);  // reals per word
};

template <int W> struct WordT;
template <> struct WordT<16> { using type = uint4; };
template <> struct WordT<8> { using type = uint2; };
template <> struct WordT<4> { using type = unsigned int; };

// Read-only (non-coherent) and streaming loads; plain and streaming stores.
__device__ __forceinline__ uint4 ldg_word(const uint4 *p) { return __ldg(p); }
__device__ __forceinline__ uint2 ldg_word(const uint2 *p) { return __ldg(p); }
__device__ __forceinline__ unsigned int ldg_word(const unsigned int *p) { return __ldg(p); }
__device__ __forceinline__ uint4 ldcs_word(const uint4 *p) { return __ldcs(p); }
__device__ __forceinline__ uint2 ldcs_word(const uint2 *p) { return __ldcs(p); }
__device__ __forceinline__ unsigned int ldcs_word(const unsigned int *p) { return __ldcs(p); }

template <typename S, int N, bool STREAM = false>
__device__ __forceinline__ void load_reals(const void *base, long Vs, long i, S (&out)[N]) {
  using Wd = Words<S, N>;
  using WT = typename WordT<Wd::W>::type;
  const WT *p = reinterpret_cast<const WT *>(base);
#pragma unroll
  for (int w = 0; w < Wd::NW; w++) {
    WT v = STREAM ? ldcs_word(p + (long)w * Vs + i) : ldg_word(p + (long)w * Vs + i);
    const S *s = reinterpret_cast<const S *>(&v);
#pragma unroll
    for (int k = 0; k < Wd::PER; k++) out[w * Wd::PER + k] = s[k];
  }
}

template <typename S, int N>
__device__ __forceinline__ void store_reals(void *base, long Vs, long i, const S (&in)[N]) {
  using Wd = Words<S, N>;
  using WT = typename WordT<Wd::W>::type;
  WT *p = reinterpret_cast<WT *>(base);
#pragma unroll
  for (int w = 0; w < Wd::NW; w++) {
    WT v;
    S *s = reinterpret_cast<S *>(&v);
#pragma unroll
    for (int k = 0; k < Wd::PER; k++) s[k] = in[w * Wd::PER + k];
    p[(long)w * Vs + i] = v;
  }
}

// ---------------------------------------------------------------------------
// Complex arithmetic on (re, im) pairs held in registers.
// ---------------------------------------------------------------------------
template <typename T> struct cx {
  T r, i;
};
template <typename T> __device__ __forceinline__ cx<T> mk(T r, T i) { return {r, i}; }
template <typename T> __device__ __forceinline__ cx<T> operator+(cx<T> a, cx<T> b) { return {a.r + b.r, a.i + b.i}; }
template <typename T> __device__ __forceinline__ cx<T> operator-(cx<T> a, cx<T> b) { return {a.r - b.r, a.i - b.i}; }
template <typename T> __device__ __forceinline__ cx<T> operator*(cx<T> a, cx<T> b) {
  return {a.r * b.r - a.i * b.i, a.r * b.i + a.i * b.r};
}
template <typename T> __device__ __forceinline__ cx<T> operator*(T s, cx<T> a) { return {s * a.r, s * a.i}; }
template <typename T> __device__ __forceinline__ cx<T> conjg(cx<T> a) { return {a.r, -a.i}; }
// a * b + c, and conj(a) * b + c
template <typename T> __device__ __forceinline__ cx<T> cmadd(cx<T> a, cx<T> b, cx<T> c) {
  return {fma(a.r, b.r, fma(-a.i, b.i, c.r)), fma(a.r, b.i, fma(a.i, b.r, c.i))};
}
template <typename T> __device__ __forceinline__ cx<T> cjmadd(cx<T> a, cx<T> b, cx<T> c) {
  return {fma(a.r, b.r, fma(a.i, b.i, c.r)), fma(a.r, b.i, fma(-a.i, b.r, c.i))};
}
// multiply by i * s for s = +-1
template <typename T> __device__ __forceinline__ cx<T> times_i(cx<T> a) { return {-a.i, a.r}; }

// |psi|^2 of one site, accumulated in the arithmetic type of the data (FP64,
// double-float, or FP32 for FP32 and FP16/BF16 data) and returned as a
// double; sums over sites are FP64.  GB300 executes FP64 at 1/64 of its FP32
// rate, so a per-site FP64 sum would make the norms fused into the FP32 and
// half-precision kernels FP64-bound.
template <typename T> __device__ __forceinline__ T site_norm2_t(const cx<T> (&a)[4][3]) {
  T s = (T)0;
#pragma unroll
  for (int sp = 0; sp < 4; sp++)
#pragma unroll
    for (int c = 0; c < 3; c++) {
      s = fma(a[sp][c].r, a[sp][c].r, s);
      s = fma(a[sp][c].i, a[sp][c].i, s);
    }
  return s;
}
template <typename T> __device__ __forceinline__ double site_norm2(const cx<T> (&a)[4][3]) {
  return (double)site_norm2_t<T>(a);
}

// arithmetic type of a binary operation between fields of compute types A, B:
// double-float if either is, else FP64 if either is, else FP32
template <typename A, typename B> struct Wide { using type = float; };
template <typename A> struct Wide<A, double> { using type = double; };
template <typename B> struct Wide<double, B> { using type = double; };
template <> struct Wide<double, double> { using type = double; };
template <typename A> struct Wide<A, df> { using type = df; };
template <typename B> struct Wide<df, B> { using type = df; };
template <> struct Wide<df, df> { using type = df; };
template <> struct Wide<df, double> { using type = df; };
template <> struct Wide<double, df> { using type = df; };

// ---------------------------------------------------------------------------
// Geometry of one parity.  Sites are numbered lexicographically,
// s = x0 + L0 (x1 + L1 (x2 + L2 x3)), parity (x0+x1+x2+x3) & 1, and the
// sites of one parity by h = s / 2 (L0 even).  Hops in mu = 1, 2, 3 move h
// by a fixed stride; hops in mu = 0 change x0 and hence h by 0 or +-1.
// ---------------------------------------------------------------------------
struct Geom {
  int L[4];
  int L0h;         // L0 / 2
  long Vh;         // sites per parity
  long stride[4];  // h-stride of a unit step in mu (mu >= 1)
  int tbc;         // 1: antiperiodic in t
};

struct Coords {
  int x[4];
};

__device__ __forceinline__ Coords site_coords(const Geom &g, long h, int parity) {
  Coords c;
  int xh = (int)(h % g.L0h);
  long r = h / g.L0h;
  c.x[1] = (int)(r % g.L[1]);
  r /= g.L[1];
  c.x[2] = (int)(r % g.L[2]);
  c.x[3] = (int)(r / g.L[2]);
  c.x[0] = 2 * xh + ((parity + c.x[1] + c.x[2] + c.x[3]) & 1);
  return c;
}

// Index (in the other parity) of the neighbour x + dir * mu.
__device__ __forceinline__ long neighbour(const Geom &g, const Coords &c, long h, int mu, int dir) {
  if (mu == 0) {
    int x0 = c.x[0] + dir;
    x0 = (x0 == g.L[0]) ? 0 : (x0 < 0 ? g.L[0] - 1 : x0);
    return (h - (c.x[0] >> 1)) + (x0 >> 1);
  }
  int xm = c.x[mu] + dir;
  if (xm == g.L[mu]) return h - (long)(g.L[mu] - 1) * g.stride[mu];
  if (xm < 0) return h + (long)(g.L[mu] - 1) * g.stride[mu];
  return h + dir * g.stride[mu];
}

// ---------------------------------------------------------------------------
// Scalar state of the Krylov solvers, one record per right-hand side, kept
// in device memory so no iteration needs a host round trip.
// ---------------------------------------------------------------------------
struct SolverScalars {
  double gamma[2];  // ||s||^2 of the current / next iteration (ping-pong)
  double qq;        // ||q||^2 = ||Mhat p||^2
  double rr;        // ||r||^2
  double aux;       // spare reduction slot
  double active;    // 1.0 while this right-hand side iterates, 0.0 once done
  double pad[2];
};

}  // namespace lqcd
