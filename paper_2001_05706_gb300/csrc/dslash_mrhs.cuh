// The even-odd Wilson-clover hopping kernel for many right-hand sides.
//
// A block owns a tile of 32 consecutive output sites of one parity and up to
// 2G right-hand sides (G warps, each warp two right-hand sides).  The tile's
// eight links per site (rebuilt to 18 reals in FP32) and its clover block pair
// are read from HBM once, converted once and staged in shared memory, where
// every warp of the block reads them: for 12 right-hand sides a site's links
// and clover cost 1/12 of their bytes per right-hand side (the 132 B per site
// and right-hand side of an FP16 A^-1 D application instead of 444 B).
//
// Each thread carries its site for two right-hand sides a, b in packed FP32
// pairs (float2 = (a, b)) and does all its arithmetic with the packed
// FP32x2 instructions of sm_100+ (__ffma2_rn, __fadd2_rn, __fmul2_rn): one
// instruction issues the multiply-adds of both right-hand sides, halving the
// instruction stream of the FP32 arithmetic (the single right-hand-side
// kernels in FP16 storage are issue-bound, not HBM-bound).  Spin projection,
// the SU(3) products, reconstruction, the epilogues and the fused norms are
// the same operations, in the same order per right-hand side, as in
// dslash.cuh's kernel (the DeGrand-Rossi spin structure documented there).
//
// Storage types: FP32, FP16 and BF16 (FP32 arithmetic).  FP64 and
// double-float right-hand sides stay on dslash_kernel: they are bound by
// their arithmetic, not by the link bytes this kernel saves.
#pragma once
#include "dslash.cuh"

namespace lqcd {

constexpr int kMrhsTile = 32;  // output sites per block (one per lane)

__device__ __forceinline__ float2 bc2(float v) { return make_float2(v, v); }
#ifndef LQCD_MRHS_SCALAR
#define LQCD_MRHS_SCALAR 0
#endif
#if LQCD_MRHS_SCALAR
// the same pair arithmetic as two scalar FP32 operations
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) {
  return make_float2(__fmaf_rn(a.x, b.x, c.x), __fmaf_rn(a.y, b.y, c.y));
}
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return make_float2(__fmul_rn(a.x, b.x), __fmul_rn(a.y, b.y)); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return make_float2(__fadd_rn(a.x, b.x), __fadd_rn(a.y, b.y)); }
#else
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
#endif
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }

// a complex number of two right-hand sides: r = (re_a, re_b), i = (im_a, im_b)
struct c2 {
  float2 r, i;
};

// Tile storage of the links and the clover pair.  LQCD_MRHS_DUP stores every
// value twice, (v, v), so an FP32x2 multiply-add takes it straight from a
// shared-memory load instead of building the pair in registers.
#ifndef LQCD_MRHS_DUP
#define LQCD_MRHS_DUP 0
#endif
struct MrhsSmem {
#if LQCD_MRHS_DUP
  float4 lk[8][9][kMrhsTile];  // link entry (r, c) of direction k: (re, re, im, im)
  float2 cm[2][36][kMrhsTile];  // clover block pair, each real twice
#else
  float4 lk4[8][4][kMrhsTile];  // link of direction k = 2 mu + (backward): entries (0,0)..(2,1)
  float2 lk2[8][kMrhsTile];     // entry (2,2)
  float4 cm[2][9][kMrhsTile];   // clover block pair (A or A^-1 per mode), 36 reals per block
#endif
  float cms[kMrhsTile];         // FP16/BF16 clover scale
};

// link entry (r, c) of direction k for this lane as broadcast pairs (re, re), (im, im)
__device__ __forceinline__ void link_entry(const MrhsSmem &sm, int k, int lane, int r, int c, float2 &ur,
                                           float2 &ui) {
#if LQCD_MRHS_DUP
  const float4 v = sm.lk[k][3 * r + c][lane];
  ur = make_float2(v.x, v.y);
  ui = make_float2(v.z, v.w);
#else
  const int e = 3 * r + c;  // entries 0..7 in lk4 (two per word), 8 in lk2
  float re, im;
  if (e == 8) {
    const float2 v = sm.lk2[k][lane];
    re = v.x;
    im = v.y;
  } else {
    const float4 v = sm.lk4[k][e >> 1][lane];
    re = (e & 1) ? v.z : v.x;
    im = (e & 1) ? v.w : v.y;
  }
  ur = make_float2(re, re);
  ui = make_float2(im, im);
#endif
}

__device__ __forceinline__ void store_link_tile(MrhsSmem &sm, int k, int s, const cx<float> (&U)[3][3]) {
#if LQCD_MRHS_DUP
#pragma unroll
  for (int r = 0; r < 3; r++)
#pragma unroll
    for (int c = 0; c < 3; c++) sm.lk[k][3 * r + c][s] = make_float4(U[r][c].r, U[r][c].r, U[r][c].i, U[r][c].i);
#else
  sm.lk4[k][0][s] = make_float4(U[0][0].r, U[0][0].i, U[0][1].r, U[0][1].i);
  sm.lk4[k][1][s] = make_float4(U[0][2].r, U[0][2].i, U[1][0].r, U[1][0].i);
  sm.lk4[k][2][s] = make_float4(U[1][1].r, U[1][1].i, U[1][2].r, U[1][2].i);
  sm.lk4[k][3][s] = make_float4(U[2][0].r, U[2][0].i, U[2][1].r, U[2][1].i);
  sm.lk2[k][s] = make_float2(U[2][2].r, U[2][2].i);
#endif
}

// clover word w (reals 4w .. 4w + 3) of block blk of site s
__device__ __forceinline__ void store_clover_tile(MrhsSmem &sm, int blk, int w, int s, float4 v) {
#if LQCD_MRHS_DUP
  sm.cm[blk][4 * w][s] = make_float2(v.x, v.x);
  sm.cm[blk][4 * w + 1][s] = make_float2(v.y, v.y);
  sm.cm[blk][4 * w + 2][s] = make_float2(v.z, v.z);
  sm.cm[blk][4 * w + 3][s] = make_float2(v.w, v.w);
#else
  sm.cm[blk][w][s] = v;
#endif
}

// ---------------------------------------------------------------------------
// packed spin projection, SU(3) product and reconstruction
// ---------------------------------------------------------------------------
// (1 + sp g_mu) psi -> half-spinor h; sp2 = (sp, sp), nsp2 = -sp2
template <int MU>
__device__ __forceinline__ void project2(const c2 (&p)[4][3], float2 sp2, float2 nsp2, c2 (&h)[2][3]) {
#pragma unroll
  for (int c = 0; c < 3; c++) {
    if (MU == 0) {  // h0 = p0 + sp i p3, h1 = p1 + sp i p2
      h[0][c] = {fma2(nsp2, p[3][c].i, p[0][c].r), fma2(sp2, p[3][c].r, p[0][c].i)};
      h[1][c] = {fma2(nsp2, p[2][c].i, p[1][c].r), fma2(sp2, p[2][c].r, p[1][c].i)};
    } else if (MU == 1) {  // h0 = p0 - sp p3, h1 = p1 + sp p2
      h[0][c] = {fma2(nsp2, p[3][c].r, p[0][c].r), fma2(nsp2, p[3][c].i, p[0][c].i)};
      h[1][c] = {fma2(sp2, p[2][c].r, p[1][c].r), fma2(sp2, p[2][c].i, p[1][c].i)};
    } else if (MU == 2) {  // h0 = p0 + sp i p2, h1 = p1 - sp i p3
      h[0][c] = {fma2(nsp2, p[2][c].i, p[0][c].r), fma2(sp2, p[2][c].r, p[0][c].i)};
      h[1][c] = {fma2(sp2, p[3][c].i, p[1][c].r), fma2(nsp2, p[3][c].r, p[1][c].i)};
    } else {  // h0 = p0 + sp p2, h1 = p1 + sp p3
      h[0][c] = {fma2(sp2, p[2][c].r, p[0][c].r), fma2(sp2, p[2][c].i, p[0][c].i)};
      h[1][c] = {fma2(sp2, p[3][c].r, p[1][c].r), fma2(sp2, p[3][c].i, p[1][c].i)};
    }
  }
}

// acc += reconstruction of U h (DAG: U^dag h), one colour row at a time: row r
// of both colour vectors (upper spins) is formed and accumulated before the
// next, so no full U h is ever held.  acc[0,1] += f (U h); acc[2,3] += flo
// B_mu^dag (U h) with flo = f s (and the g5 sign of the hop sum); nflo = -flo.
template <int MU, bool DAG>
__device__ __forceinline__ void link_recon2(const MrhsSmem &sm, int k, int lane, const c2 (&h)[2][3], float2 f,
                                            float2 flo, float2 nflo, c2 (&acc)[4][3]) {
#pragma unroll
  for (int r = 0; r < 3; r++) {
    float2 t0r = bc2(0.0f), t0i = bc2(0.0f), t1r = bc2(0.0f), t1i = bc2(0.0f);
#pragma unroll
    for (int c = 0; c < 3; c++) {
      float2 ur, ui;
      if (DAG)
        link_entry(sm, k, lane, c, r, ur, ui);  // conj(U[c][r])
      else
        link_entry(sm, k, lane, r, c, ur, ui);
      const float2 nui = neg2(ui);
      const float2 pim = DAG ? nui : ui;  // imaginary part of the factor
      const float2 nim = DAG ? ui : nui;
      t0r = fma2(ur, h[0][c].r, fma2(nim, h[0][c].i, t0r));
      t0i = fma2(ur, h[0][c].i, fma2(pim, h[0][c].r, t0i));
      t1r = fma2(ur, h[1][c].r, fma2(nim, h[1][c].i, t1r));
      t1i = fma2(ur, h[1][c].i, fma2(pim, h[1][c].r, t1i));
    }
    acc[0][r] = {fma2(f, t0r, acc[0][r].r), fma2(f, t0i, acc[0][r].i)};
    acc[1][r] = {fma2(f, t1r, acc[1][r].r), fma2(f, t1i, acc[1][r].i)};
    if (MU == 0) {  // lower0 -= s i h1, lower1 -= s i h0
      acc[2][r] = {fma2(flo, t1i, acc[2][r].r), fma2(nflo, t1r, acc[2][r].i)};
      acc[3][r] = {fma2(flo, t0i, acc[3][r].r), fma2(nflo, t0r, acc[3][r].i)};
    } else if (MU == 1) {  // lower0 += s h1, lower1 -= s h0
      acc[2][r] = {fma2(flo, t1r, acc[2][r].r), fma2(flo, t1i, acc[2][r].i)};
      acc[3][r] = {fma2(nflo, t0r, acc[3][r].r), fma2(nflo, t0i, acc[3][r].i)};
    } else if (MU == 2) {  // lower0 -= s i h0, lower1 += s i h1
      acc[2][r] = {fma2(flo, t0i, acc[2][r].r), fma2(nflo, t0r, acc[2][r].i)};
      acc[3][r] = {fma2(nflo, t1i, acc[3][r].r), fma2(flo, t1r, acc[3][r].i)};
    } else {  // lower0 += s h0, lower1 += s h1
      acc[2][r] = {fma2(flo, t0r, acc[2][r].r), fma2(flo, t0i, acc[2][r].i)};
      acc[3][r] = {fma2(flo, t1r, acc[3][r].r), fma2(flo, t1i, acc[3][r].i)};
    }
  }
}

// packed Hermitian 6x6 product (the storage of herm6_mul in dslash.cuh) with
// the block's 36 reals from the tile
__device__ __forceinline__ float2 clover_real(const MrhsSmem &sm, int blk, int k, int lane) {
#if LQCD_MRHS_DUP
  return sm.cm[blk][k][lane];
#else
  const float4 v = sm.cm[blk][k >> 2][lane];
  const float x = (k & 3) == 0 ? v.x : (k & 3) == 1 ? v.y : (k & 3) == 2 ? v.z : v.w;
  return make_float2(x, x);
#endif
}

__device__ __forceinline__ void herm6_mul2(const MrhsSmem &sm, int blk, int lane, const c2 (&v)[6], c2 (&o)[6]) {
#pragma unroll
  for (int i = 0; i < 6; i++) {
    const float2 d = clover_real(sm, blk, i, lane);
    o[i] = {mul2(d, v[i].r), mul2(d, v[i].i)};
  }
#pragma unroll
  for (int i = 1; i < 6; i++)
#pragma unroll
    for (int j = 0; j < i; j++) {
      const int k = 6 + 2 * (i * (i - 1) / 2 + j);
      const float2 lr = clover_real(sm, blk, k, lane), li = clover_real(sm, blk, k + 1, lane), nli = neg2(li);
      // o_i += L_ij v_j
      o[i].r = fma2(lr, v[j].r, fma2(nli, v[j].i, o[i].r));
      o[i].i = fma2(lr, v[j].i, fma2(li, v[j].r, o[i].i));
      // o_j += conj(L_ij) v_i
      o[j].r = fma2(lr, v[i].r, fma2(li, v[i].i, o[j].r));
      o[j].i = fma2(lr, v[i].i, fma2(nli, v[i].r, o[j].i));
    }
}

// psi = M psi with the tile's clover pair from shared memory; the FP16/BF16
// storage scale multiplies the six outputs of each block
template <typename S>
__device__ __forceinline__ void clover_apply2(const MrhsSmem &sm, int lane, c2 (&psi)[4][3]) {
#pragma unroll
  for (int blk = 0; blk < 2; blk++) {
    c2 v[6], o[6];
#pragma unroll
    for (int k = 0; k < 6; k++) v[k] = psi[2 * blk + k / 3][k % 3];
    herm6_mul2(sm, blk, lane, v, o);
    if constexpr (IsHalf<S>::value) {
      const float2 sc = bc2(sm.cms[lane]);
#pragma unroll
      for (int k = 0; k < 6; k++) o[k] = {mul2(sc, o[k].r), mul2(sc, o[k].i)};
    }
#pragma unroll
    for (int k = 0; k < 6; k++) psi[2 * blk + k / 3][k % 3] = o[k];
  }
}

// ---------------------------------------------------------------------------
// spinor access for a pair of right-hand sides
// ---------------------------------------------------------------------------
template <typename S>
__device__ __forceinline__ void load_pair(const FieldRef &f, long Vh, int ra, int rb, long i, c2 (&psi)[4][3]) {
  cx<float> a[4][3], b[4][3];
  load_spinor<S>(f, Vh, ra, i, a);
  load_spinor<S>(f, Vh, rb, i, b);
#pragma unroll
  for (int s = 0; s < 4; s++)
#pragma unroll
    for (int c = 0; c < 3; c++) psi[s][c] = {make_float2(a[s][c].r, b[s][c].r), make_float2(a[s][c].i, b[s][c].i)};
}

// Raw words of one tile's links and clover pair, copied global -> shared by
// cp.async while the block computes the previous tile, then converted
// (12-real links rebuilt) into MrhsSmem.
template <typename S, int R> struct MrhsRaw {
  using WL = Words<S, R>;
  using WC = Words<S, 36>;  // nine words of four reals per clover block
  typename WordT<WL::W>::type lk[8][WL::NW][kMrhsTile];
  typename WordT<WC::W>::type cm[18][kMrhsTile];
  float cms[kMrhsTile];
};

// Each thread's neighbour spinors of its two right-hand sides, D directions
// ahead: per-thread slots (no block barrier), filled by cp.async while the
// thread computes the directions before.  FP16/BF16 run two directions
// ahead, FP32 (twice the bytes per slot) one.
#ifndef LQCD_MRHS_D16
#define LQCD_MRHS_D16 2
#endif
#ifndef LQCD_MRHS_D32
#define LQCD_MRHS_D32 1
#endif
template <typename S> struct MrhsDepth { static constexpr int D = IsHalf<S>::value ? LQCD_MRHS_D16 : LQCD_MRHS_D32; };
template <typename S, int NT> struct MrhsSpin {
  static constexpr int D = MrhsDepth<S>::D;
  using WS = Words<S, 24>;
  typename WordT<WS::W>::type sp[D][2][WS::NW][NT];
  float sc[D][2][NT];
};

template <typename S, int R, int G>
constexpr size_t mrhs_smem_bytes() {
  return sizeof(MrhsSmem) + sizeof(MrhsRaw<S, R>) + sizeof(MrhsSpin<S, 32 * G>);
}

template <int B> __device__ __forceinline__ void cp_async_g2s(void *smem, const void *gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(sa), "l"(gmem), "n"(B) : "memory");
}

template <typename S, int R, int MODE, int NT>
__device__ __forceinline__ void mrhs_stage(const DslashParams &P, long t0, MrhsRaw<S, R> &rw, bool hop) {
  using WL = typename MrhsRaw<S, R>::WL;
  using WC = typename MrhsRaw<S, R>::WC;
  constexpr bool kMat = MODE == MODE_HOP_AINV || MODE == MODE_FOLDED_AINV || MODE == MODE_LOCAL_A;
  const int p = P.out_parity;
  const long Vh = P.g.Vh;
  if (hop) {
    for (int j = threadIdx.x; j < 8 * kMrhsTile; j += NT) {
      const int k = j / kMrhsTile, s = j % kMrhsTile;
      const long h = t0 + s;
      if (h >= P.h1) continue;
      const int mu = k >> 1;
      long li = h;
      const char *base = reinterpret_cast<const char *>(P.links[mu][p]);
      if (k & 1) {  // backward hop: U_mu(x - mu)^dag, stored at the neighbour of the other parity
        const Coords xc = site_coords(P.g, h, p);
        li = neighbour(P.g, xc, h, mu, -1);
        LQCD_CHECK_INDEX(P, li);
        base = reinterpret_cast<const char *>(P.links[mu][1 - p]);
      }
#pragma unroll
      for (int w = 0; w < WL::NW; w++) cp_async_g2s<WL::W>(&rw.lk[k][w][s], base + ((long)w * Vh + li) * WL::W);
    }
  }
  if constexpr (kMat) {
    const char *mat = reinterpret_cast<const char *>(MODE == MODE_LOCAL_A ? P.lmat : P.cmat);
    for (int j = threadIdx.x; j < 18 * kMrhsTile; j += NT) {
      const int bw = j / kMrhsTile, s = j % kMrhsTile;
      const long h = t0 + s;
      if (h < P.h1) cp_async_g2s<WC::W>(&rw.cm[bw][s], mat + ((long)bw * Vh + h) * WC::W);
    }
    if constexpr (IsHalf<S>::value) {
      const float *msc = MODE == MODE_LOCAL_A ? P.lmat_scale : P.cmat_scale;
      for (int s = threadIdx.x; s < kMrhsTile; s += NT)
        if (t0 + s < P.h1) cp_async_g2s<4>(&rw.cms[s], msc + t0 + s);
    }
  }
}

template <typename S, int R, int MODE, int NT>
__device__ __forceinline__ void mrhs_convert(const DslashParams &P, long t0, const MrhsRaw<S, R> &rw, MrhsSmem &sm,
                                             bool hop) {
  using WL = typename MrhsRaw<S, R>::WL;
  constexpr bool kMat = MODE == MODE_HOP_AINV || MODE == MODE_FOLDED_AINV || MODE == MODE_LOCAL_A;
  if (hop) {
    for (int j = threadIdx.x; j < 8 * kMrhsTile; j += NT) {
      const int k = j / kMrhsTile, s = j % kMrhsTile;
      if (t0 + s >= P.h1) continue;
      S raw[R];
#pragma unroll
      for (int w = 0; w < WL::NW; w++) {
        const auto v = rw.lk[k][w][s];
        const S *q = reinterpret_cast<const S *>(&v);
#pragma unroll
        for (int e = 0; e < WL::PER; e++) raw[w * WL::PER + e] = q[e];
      }
      cx<float> U[3][3];
#pragma unroll
      for (int r = 0; r < R / 6; r++)
#pragma unroll
        for (int c = 0; c < 3; c++) U[r][c] = {to_f(raw[6 * r + 2 * c]), to_f(raw[6 * r + 2 * c + 1])};
      if (R == 12) {
#pragma unroll
        for (int c = 0; c < 3; c++) {
          const int a = (c + 1) % 3, b = (c + 2) % 3;
          U[2][c] = conjg(U[0][a] * U[1][b] - U[0][b] * U[1][a]);
        }
      }
      store_link_tile(sm, k, s, U);
    }
  }
  if constexpr (kMat) {
    for (int j = threadIdx.x; j < 18 * kMrhsTile; j += NT) {
      const int bw = j / kMrhsTile, s = j % kMrhsTile;
      if (t0 + s >= P.h1) continue;
      const auto v = rw.cm[bw][s];
      const S *x = reinterpret_cast<const S *>(&v);
      store_clover_tile(sm, bw / 9, bw % 9, s, make_float4(to_f(x[0]), to_f(x[1]), to_f(x[2]), to_f(x[3])));
    }
    if constexpr (IsHalf<S>::value) {
      for (int s = threadIdx.x; s < kMrhsTile; s += NT)
        if (t0 + s < P.h1) sm.cms[s] = rw.cms[s];
    }
  }
}

// Per-thread view of the hop sum's gathers: the two right-hand sides' base
// addresses and the site of the current and of the next tile.
template <typename S> struct MrhsGather {
  const char *ia, *ib;    // spinor data of right-hand sides a and b
  const float *sa, *sb;   // their FP16/BF16 scales
  long h, hn;             // this lane's site in the current and the next tile
  bool ok, okn;           // ... and whether it exists
  Coords xc, xn;
};

// issue the cp.async copies of direction k of site (h, xc) into slot `slot`;
// `dep` orders them after the reads of that slot's previous contents
template <typename S, int NT>
__device__ __forceinline__ void mrhs_issue(const DslashParams &P, MrhsSpin<S, NT> &st, const MrhsGather<S> &g,
                                           int slot, int k, bool next, unsigned dep) {
  using WS = Words<S, 24>;
  const bool ok = next ? g.okn : g.ok;
  if (ok) {
    const long Vh = P.g.Vh;
    const int mu = k >> 1;
    long n = neighbour(P.g, next ? g.xn : g.xc, next ? g.hn : g.h, mu, (k & 1) ? -1 : +1);
    LQCD_CHECK_INDEX(P, n);
    const int tid = threadIdx.x;
#pragma unroll
    for (int w = 0; w < WS::NW; w++) {
      const long off = ((long)w * Vh + n) * WS::W;
      cp_async_after<WS::W>(&st.sp[slot][0][w][tid], g.ia + off, dep);
      cp_async_after<WS::W>(&st.sp[slot][1][w][tid], g.ib + off, dep);
    }
    if constexpr (IsHalf<S>::value) {
      cp_async_after<4>(&st.sc[slot][0][tid], g.sa + n, dep);
      cp_async_after<4>(&st.sc[slot][1][tid], g.sb + n, dep);
    }
  }
  cp_async_commit();  // one group per direction, empty where the site does not exist
}

// one direction K = 2 mu + (backward): read its slot, hand the slot to
// direction K + D (of this tile, or of the next one), compute
template <typename S, int NT, int K>
__device__ __forceinline__ void mrhs_dir(const DslashParams &P, const MrhsSmem &sm, MrhsSpin<S, NT> &st,
                                         const MrhsGather<S> &g, int lane, float sp, float fb, float g5h,
                                         c2 (&acc)[4][3]) {
  using WS = Words<S, 24>;
  constexpr int D = MrhsDepth<S>::D;
  constexpr int MU = K >> 1;
  constexpr int DIR = (K & 1) ? -1 : +1;
  constexpr float S_ = DIR > 0 ? -1.0f : 1.0f;  // forward (1 - g_mu), backward (1 + g_mu)
  constexpr int slot = K % D;
  // groups committed after direction K's: the other in-flight directions, plus
  // (K < D) the tile's link and clover words committed before direction D
  if constexpr (K < D)
    cp_async_wait<D>();
  else
    cp_async_wait<D - 1>();
  const int tid = threadIdx.x;
  S ra[24], rb[24];
  unsigned ua[12], ub[12];  // FP16/BF16: the stored (re, im) pairs
  unsigned dep = 0;
#pragma unroll
  for (int w = 0; w < WS::NW; w++) {
    const auto va = st.sp[slot][0][w][tid];
    const auto vb = st.sp[slot][1][w][tid];
    dep |= first_bits(va) ^ first_bits(vb);
    if constexpr (IsHalf<S>::value) {
      static_assert(WS::W == 16, "FP16/BF16 spinors are three 16-byte words");
      const unsigned *xa = reinterpret_cast<const unsigned *>(&va);
      const unsigned *xb = reinterpret_cast<const unsigned *>(&vb);
#pragma unroll
      for (int j = 0; j < 4; j++) {
        ua[w * 4 + j] = xa[j];
        ub[w * 4 + j] = xb[j];
      }
    } else {
      const S *xa = reinterpret_cast<const S *>(&va);
      const S *xb = reinterpret_cast<const S *>(&vb);
#pragma unroll
      for (int j = 0; j < WS::PER; j++) {
        ra[w * WS::PER + j] = xa[j];
        rb[w * WS::PER + j] = xb[j];
      }
    }
  }
  float sca = 1.0f, scb = 1.0f;
  if constexpr (IsHalf<S>::value) {
    sca = st.sc[slot][0][tid];
    scb = st.sc[slot][1][tid];
    dep |= __float_as_uint(sca) ^ __float_as_uint(scb);
  }
  // the slot's values are in registers: refill it with direction K + D
  if (K + D < 8)
    mrhs_issue<S, NT>(P, st, g, slot, K + D, false, dep);
  else
    mrhs_issue<S, NT>(P, st, g, slot, K + D - 8, true, dep);
  if (!g.ok) return;
  const bool wrap = (MU == 3) && P.g.tbc && (DIR > 0 ? g.xc.x[3] == P.g.L[3] - 1 : g.xc.x[3] == 0);
  const float fw = wrap ? -fb : fb;
  const float2 f = make_float2(fw * sca, fw * scb);
  const float2 flo = mul2(bc2(S_ * g5h), f);
  const float2 spp = bc2(S_ * sp);
  c2 h[2][3];
  if constexpr (IsHalf<S>::value) {
    // each right-hand side projected on its stored pairs (project_packed),
    // then the two packed into FP32 pairs
    cx<float> ha[2][3], hb[2][3];
    project_packed<S>(MU, S_ * sp, ua, ha);
    project_packed<S>(MU, S_ * sp, ub, hb);
#pragma unroll
    for (int a = 0; a < 2; a++)
#pragma unroll
      for (int c = 0; c < 3; c++) h[a][c] = {make_float2(ha[a][c].r, hb[a][c].r), make_float2(ha[a][c].i, hb[a][c].i)};
  } else {
    c2 psi[4][3];
#pragma unroll
    for (int s = 0; s < 4; s++)
#pragma unroll
      for (int c = 0; c < 3; c++)
        psi[s][c] = {make_float2(to_f(ra[6 * s + 2 * c]), to_f(rb[6 * s + 2 * c])),
                     make_float2(to_f(ra[6 * s + 2 * c + 1]), to_f(rb[6 * s + 2 * c + 1]))};
    project2<MU>(psi, spp, neg2(spp), h);
  }
  link_recon2<MU, (DIR < 0)>(sm, K, lane, h, f, flo, neg2(flo), acc);
}

// the epilogue of one tile's site for the warp's pair of right-hand sides
template <typename S, int MODE>
__device__ __forceinline__ void mrhs_epilogue(const DslashParams &P, const MrhsSmem &sm, long h, int lane, int ra,
                                              int rb, int rbb, bool hasb, c2 (&acc)[4][3], df &na, df &nb) {
  const long Vh = P.g.Vh;
  if (MODE == MODE_LOCAL_IDENT || MODE == MODE_FOLDED_AINV || MODE == MODE_LOCAL_A || MODE == MODE_CHEB) {
    const float2 al = bc2((float)P.alpha);
    c2 x[4][3];
    load_pair<S>(P.xloc, Vh, ra, rbb, h, x);
    if constexpr (MODE == MODE_LOCAL_A) clover_apply2<S>(sm, lane, x);
#pragma unroll
    for (int s = 0; s < 4; s++)
#pragma unroll
      for (int c = 0; c < 3; c++) acc[s][c] = {fma2(al, x[s][c].r, acc[s][c].r), fma2(al, x[s][c].i, acc[s][c].i)};
  }
  if constexpr (MODE == MODE_HOP_AINV || MODE == MODE_FOLDED_AINV) clover_apply2<S>(sm, lane, acc);
  if (P.g5_total) {
#pragma unroll
    for (int s = 2; s < 4; s++)
#pragma unroll
      for (int c = 0; c < 3; c++) acc[s][c] = {neg2(acc[s][c].r), neg2(acc[s][c].i)};
  }
  if constexpr (MODE == MODE_CHEB) {
#pragma unroll
    for (int k = 0; k < 3; k++) {
      if (P.zc[k].data == nullptr) continue;
      const float2 ck = bc2((float)P.cz[k]);
      c2 zz[4][3];
      load_pair<S>(P.zc[k], Vh, ra, rbb, h, zz);
#pragma unroll
      for (int s = 0; s < 4; s++)
#pragma unroll
        for (int c = 0; c < 3; c++)
          acc[s][c] = {fma2(ck, zz[s][c].r, acc[s][c].r), fma2(ck, zz[s][c].i, acc[s][c].i)};
    }
  }
  if (MODE != MODE_CHEB && P.z.data != nullptr) {
    const float2 gz = bc2((float)P.gz);
    c2 zz[4][3];
    load_pair<S>(P.z, Vh, ra, rbb, h, zz);
#pragma unroll
    for (int s = 0; s < 4; s++)
#pragma unroll
      for (int c = 0; c < 3; c++) acc[s][c] = {fma2(gz, acc[s][c].r, zz[s][c].r), fma2(gz, acc[s][c].i, zz[s][c].i)};
  }
  cx<float> oa[4][3], ob[4][3];
#pragma unroll
  for (int s = 0; s < 4; s++)
#pragma unroll
    for (int c = 0; c < 3; c++) {
      oa[s][c] = {acc[s][c].r.x, acc[s][c].i.x};
      ob[s][c] = {acc[s][c].r.y, acc[s][c].i.y};
    }
  const long out_words = Words<S, 24>::NW * Vh;
  store_spinor<S>(P.out, P.out_scale, out_words, Vh, ra, h, oa);
  if (hasb) store_spinor<S>(P.out, P.out_scale, out_words, Vh, rb, h, ob);
  if (P.norm_partials) {
    na = df(site_norm2_t<float>(oa));
    nb = df(site_norm2_t<float>(ob));
  }
}

// Persistent over the tiles of the parity: block (x, y) takes tiles x,
// x + gridDim.x, ... for the right-hand-side pairs of chunk y.  While its
// warps compute one tile, the raw link and clover words of the next tile are
// in flight (cp.async), and so are each thread's next neighbour spinors (D
// directions ahead, running on into the next tile's first directions);
// between tiles the block converts the staged words (two block barriers).
// LQCD_MRHS_WARPS: resident warps per SM the register allocator is held to
// (12: two blocks of six warps).
#ifndef LQCD_MRHS_WARPS
#define LQCD_MRHS_WARPS 12
#endif
template <typename S, int R, int MODE, int G>
__global__ void __launch_bounds__(32 * G, (LQCD_MRHS_WARPS + G - 1) / G) dslash_mrhs_kernel(const __grid_constant__ DslashParams P) {
  extern __shared__ __align__(16) unsigned char mrhs_smem[];
  constexpr int NT = 32 * G;
  constexpr int D = MrhsDepth<S>::D;
  MrhsSmem &sm = *reinterpret_cast<MrhsSmem *>(mrhs_smem);
  MrhsRaw<S, R> &rw = *reinterpret_cast<MrhsRaw<S, R> *>(mrhs_smem + sizeof(MrhsSmem));
  MrhsSpin<S, NT> &st = *reinterpret_cast<MrhsSpin<S, NT> *>(mrhs_smem + sizeof(MrhsSmem) + sizeof(MrhsRaw<S, R>));
  const int ntiles = (int)((P.h1 - P.h0 + kMrhsTile - 1) / kMrhsTile);
  const bool hop = P.in.data != nullptr && P.beta != 0.0;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int p = P.out_parity;
  const long Vh = P.g.Vh;
  const int pair = blockIdx.y * G + warp;
  const int ra = 2 * pair, rb = 2 * pair + 1;
  const bool busy = ra < P.nrhs;  // warps of a last, partial chunk may have no right-hand sides
  const bool hasb = rb < P.nrhs;
  const int rbb = hasb ? rb : ra;  // an odd count computes a's site twice and stores it once
  const bool gather = busy && hop;

  MrhsGather<S> g;
  g.ia = reinterpret_cast<const char *>(rhs_base<S>(P.in.data, P.in.rhs_words, busy ? ra : 0));
  g.ib = reinterpret_cast<const char *>(rhs_base<S>(P.in.data, P.in.rhs_words, busy ? rbb : 0));
  g.sa = IsHalf<S>::value ? P.in.scale + (long)(busy ? ra : 0) * Vh : nullptr;
  g.sb = IsHalf<S>::value ? P.in.scale + (long)(busy ? rbb : 0) * Vh : nullptr;
  const float sp = P.g5_in ? -1.0f : 1.0f;  // g5 on the input flips the lower spins' projection sign
  const float fb = (float)P.beta;
  const float g5h = P.g5_hop ? -1.0f : 1.0f;

  int tile = blockIdx.x;
  if (tile < ntiles) {
    const long t0 = P.h0 + (long)tile * kMrhsTile;
    mrhs_stage<S, R, MODE, NT>(P, t0, rw, hop);
    cp_async_commit();
    cp_async_wait<0>();
    __syncthreads();
    mrhs_convert<S, R, MODE, NT>(P, t0, rw, sm, hop);
    // the first tile's first D directions
    g.hn = t0 + lane;
    g.okn = gather && g.hn < P.h1;
    if (g.okn) g.xn = site_coords(P.g, g.hn, p);
    for (int k = 0; k < D; k++) mrhs_issue<S, NT>(P, st, g, k, k, true, 0u);
  }
  __syncthreads();
  for (; tile < ntiles; tile += gridDim.x) {
    const long t0 = P.h0 + (long)tile * kMrhsTile;
    const int next = tile + gridDim.x;
    g.h = g.hn;
    g.ok = g.okn;
    g.xc = g.xn;
    if (next < ntiles) mrhs_stage<S, R, MODE, NT>(P, P.h0 + (long)next * kMrhsTile, rw, hop);
    cp_async_commit();
    g.hn = P.h0 + (long)next * kMrhsTile + lane;
    g.okn = gather && next < ntiles && g.hn < P.h1;
    if (g.okn) g.xn = site_coords(P.g, g.hn, p);
    const bool valid = busy && g.h < P.h1;
    c2 acc[4][3];
#pragma unroll
    for (int s = 0; s < 4; s++)
#pragma unroll
      for (int c = 0; c < 3; c++) acc[s][c] = {bc2(0.0f), bc2(0.0f)};
    if (gather) {
      mrhs_dir<S, NT, 0>(P, sm, st, g, lane, sp, fb, g5h, acc);
      mrhs_dir<S, NT, 1>(P, sm, st, g, lane, sp, fb, g5h, acc);
      mrhs_dir<S, NT, 2>(P, sm, st, g, lane, sp, fb, g5h, acc);
      mrhs_dir<S, NT, 3>(P, sm, st, g, lane, sp, fb, g5h, acc);
      mrhs_dir<S, NT, 4>(P, sm, st, g, lane, sp, fb, g5h, acc);
      mrhs_dir<S, NT, 5>(P, sm, st, g, lane, sp, fb, g5h, acc);
      mrhs_dir<S, NT, 6>(P, sm, st, g, lane, sp, fb, g5h, acc);
      mrhs_dir<S, NT, 7>(P, sm, st, g, lane, sp, fb, g5h, acc);
    } else {
      cp_async_wait<0>();  // no gathers: only the tile's words are in flight
    }
    df na(0.0f, 0.0f), nb(0.0f, 0.0f);
    if (valid) mrhs_epilogue<S, MODE>(P, sm, g.h, lane, ra, rb, rbb, hasb, acc, na, nb);
    if (busy && P.norm_partials) {
      // each right-hand side lives in one warp of the block: its partial over
      // the tile is that warp's fixed shuffle tree (double-float), one per tile
      na = warp_sum(na);
      nb = warp_sum(nb);
      if (lane == 0) {
        P.norm_partials[(long)ra * ntiles + tile] = (double)na.hi + (double)na.lo;
        if (hasb) P.norm_partials[(long)rb * ntiles + tile] = (double)nb.hi + (double)nb.lo;
      }
    }
    __syncthreads();  // the next tile's words have landed; no warp reads this tile's any more
    if (next < ntiles) mrhs_convert<S, R, MODE, NT>(P, P.h0 + (long)next * kMrhsTile, rw, sm, hop);
    __syncthreads();
  }
  cp_async_wait<0>();
}

template <typename S, int R, int MODE, int G>
static cudaError_t launch_mrhs_one(const DslashParams &P, cudaStream_t st) {
  constexpr size_t kSmem = mrhs_smem_bytes<S, R, G>();
  // resident blocks per SM of this instantiation, found once (it also lifts
  // the dynamic shared-memory limit above 48 KB where the tile needs it)
  static const int occ = [] {
    int n = 0;
    if (cudaFuncSetAttribute(dslash_mrhs_kernel<S, R, MODE, G>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kSmem) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, dslash_mrhs_kernel<S, R, MODE, G>, 32 * G, kSmem) !=
            cudaSuccess)
      n = 0;
    cudaGetLastError();
    return n;
  }();
  if (occ < 1) return cudaErrorInvalidConfiguration;
  int dev = 0, nsm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const int pairs = (P.nrhs + 1) / 2;
  const long ntiles = (P.h1 - P.h0 + kMrhsTile - 1) / kMrhsTile;
  const int chunks = (pairs + G - 1) / G;
  // enough blocks to fill every SM over all chunks, none without a tile
  long nx = ((long)nsm * occ + chunks - 1) / chunks;
  if (nx > ntiles) nx = ntiles;
  if (nx < 1) nx = 1;
  dim3 grid((unsigned)nx, (unsigned)chunks);
  dslash_mrhs_kernel<S, R, MODE, G><<<grid, 32 * G, kSmem, st>>>(P);
  e = cudaGetLastError();
  if (e != cudaSuccess || !P.norm_partials) return e;
  return finish_reduce(P.norm_partials, (int)ntiles, P.nrhs, P.norm_result, P.norm_stride, st);
}

template <typename S, int R, int MODE>
static cudaError_t launch_mrhs_g(const DslashParams &P, int g, cudaStream_t st) {
  switch (g) {
    case 1: return launch_mrhs_one<S, R, MODE, 1>(P, st);
    case 2: return launch_mrhs_one<S, R, MODE, 2>(P, st);
    case 3: return launch_mrhs_one<S, R, MODE, 3>(P, st);
    case 6: return launch_mrhs_one<S, R, MODE, 6>(P, st);
  }
  return cudaErrorInvalidValue;
}

template <typename S, int R>
static cudaError_t launch_mrhs_mode(const DslashParams &P, int mode, int g, cudaStream_t st) {
  switch (mode) {
    case MODE_HOP: return launch_mrhs_g<S, R, MODE_HOP>(P, g, st);
    case MODE_HOP_AINV: return launch_mrhs_g<S, R, MODE_HOP_AINV>(P, g, st);
    case MODE_LOCAL_IDENT: return launch_mrhs_g<S, R, MODE_LOCAL_IDENT>(P, g, st);
    case MODE_LOCAL_A: return launch_mrhs_g<S, R, MODE_LOCAL_A>(P, g, st);
    case MODE_CHEB:
      if constexpr (std::is_same<S, float>::value) return launch_mrhs_g<S, R, MODE_CHEB>(P, g, st);
      break;
  }
  return cudaErrorInvalidValue;
}

// g: warps per block (right-hand-side pairs sharing one staged tile)
template <typename S>
cudaError_t launch_dslash_mrhs(const DslashParams &P, int recon, int mode, int g, cudaStream_t st);

}  // namespace lqcd
