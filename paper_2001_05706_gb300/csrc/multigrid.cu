// Adaptive aggregation multigrid for the Wilson-clover operator: the GPU
// building blocks of the 3-level multigrid inverter the paper runs with QUDA
// (Sec. 4: blocks (4,4,4,4) and (2,2,2,2); Table 1: every part a clover
// multigrid needs).  The paper prints none of the method's steps; these are
// the standard ones of adaptive aggregation multigrid (Babich et al. 2010,
// Clark et al. 2016):
//
//   every level is a nearest-neighbour stencil on a periodic 4-d lattice,
//     D v(x) = X(x) v(x) + sum_mu F_mu(x) v(x + mu) + B_mu(x) v(x - mu),
//   with n complex components per site, the first n/2 of chirality +1 and
//   the last n/2 of chirality -1 (gamma5 = diag(1, 1, -1, -1) in spin for
//   the fine level, index 3 spin + colour);
//   the prolongator P (V, n, 2 nv) holds, on each block of the lattice and
//   each chirality, the Gram-Schmidt orthonormalisation of nv near-null
//   vectors restricted there (coarse components [chirality +: nv, -: nv]);
//   the coarse operator is the Galerkin product P^H D P, again a stencil.
//
// All arrays are complex FP64, interleaved (re, im), 16-byte aligned, in
// lexicographic site order with x fastest: fields (V, n), X (V, n, n),
// F and B (4, V, n, n) row-major, P (V, n, nc).  The Krylov iteration and
// the cycle around these calls run on the host
// (paper_2001_05706_gb300/multigrid.py); every arithmetic step is here.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>

#include "internal.h"

namespace lqcd {
namespace {

constexpr int kMgT = 256;          // threads of the elementwise kernels
constexpr int kMgOrthT = 128;      // threads of one block orthonormalisation
constexpr int kMgCoarsenT = 256;   // threads of one coarse matrix
constexpr int kMgMaxN = 64;        // components per site of any level
constexpr int kMgMaxK = 64;        // vectors of one dots / axpys call
constexpr int kMgMaxEnt = (kMgMaxN * kMgMaxN + kMgCoarsenT - 1) / kMgCoarsenT;  // coarse entries per thread

using C = cx<double>;

struct MgDims {
  int L[4];
  long V;
};

struct MgCoefs {
  double2 c[kMgMaxK];
};

__device__ __forceinline__ C cxd(double r, double i) { return mk<double>(r, i); }
__device__ __forceinline__ C ld2(const double2 *p, long i) {
  const double2 v = p[i];
  return cxd(v.x, v.y);
}
__device__ __forceinline__ double2 st2(C v) { return make_double2(v.r, v.i); }

__device__ __forceinline__ void mg_coords(const MgDims &d, long s, int (&x)[4]) {
  long r = s;
#pragma unroll
  for (int mu = 0; mu < 4; mu++) {
    x[mu] = (int)(r % d.L[mu]);
    r /= d.L[mu];
  }
}
__device__ __forceinline__ long mg_index(const MgDims &d, const int (&x)[4]) {
  return x[0] + (long)d.L[0] * (x[1] + (long)d.L[1] * (x[2] + (long)d.L[2] * x[3]));
}
__device__ __forceinline__ long mg_shift(const MgDims &d, const int (&x)[4], int mu, int step) {
  int y[4] = {x[0], x[1], x[2], x[3]};
  y[mu] = (y[mu] + step + d.L[mu]) % d.L[mu];
  return mg_index(d, y);
}
// fine site number q (x fastest) of the block at coarse coordinates xc
__device__ __forceinline__ long mg_block_site(const MgDims &fd, const int4 &b, const int (&xc)[4], int q,
                                              int (&o)[4]) {
  o[0] = q % b.x;
  o[1] = (q / b.x) % b.y;
  o[2] = (q / (b.x * b.y)) % b.z;
  o[3] = q / (b.x * b.y * b.z);
  const int x[4] = {xc[0] * b.x + o[0], xc[1] * b.y + o[1], xc[2] * b.z + o[2], xc[3] * b.w + o[3]};
  return mg_index(fd, x);
}

// the 2x2 block B_mu of gamma_mu = [[0, B_mu], [B_mu^dag, 0]] (DeGrand-Rossi)
__device__ __forceinline__ C dr_block(int mu, int a, int b) {
  switch (mu) {
    case 0: return a != b ? cxd(0.0, 1.0) : cxd(0.0, 0.0);
    case 1: return a != b ? cxd(a == 0 ? -1.0 : 1.0, 0.0) : cxd(0.0, 0.0);
    case 2: return a == b ? cxd(0.0, a == 0 ? 1.0 : -1.0) : cxd(0.0, 0.0);
    default: return a == b ? cxd(1.0, 0.0) : cxd(0.0, 0.0);
  }
}
__device__ __forceinline__ C gamma_entry(int mu, int a, int b) {
  if (a < 2 && b >= 2) return dr_block(mu, a, b - 2);
  if (a >= 2 && b < 2) return conjg(dr_block(mu, b, a - 2));
  return cxd(0.0, 0.0);
}

// M = A - kappa D_W as a stencil: X = A (two 6x6 Hermitian blocks of the FP64
// clover term, or 1), F_mu = -kappa (1 - gamma_mu) U_mu(x), B_mu = -kappa
// (1 + gamma_mu) U_mu(x - mu)^dag, -1 on the hops across the t boundary when
// tbc is set.  One thread per site.
__global__ void __launch_bounds__(kMgT) mg_fine_kernel(MgDims d, int tbc, double kappa, const double *__restrict__ U,
                                                        const char *A0, const char *A1, long Vh, double2 *X,
                                                        double2 *F, double2 *B) {
  const long s = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= d.V) return;
  int x[4];
  mg_coords(d, s, x);
  double2 *Xs = X + s * 144;
  for (int e = 0; e < 144; e++) Xs[e] = make_double2(e / 12 == e % 12 ? 1.0 : 0.0, 0.0);
  if (A0) {
    const int p = (x[0] + x[1] + x[2] + x[3]) & 1;
    const char *base = p ? A1 : A0;
    const long h = s >> 1;
    using Wd = Words<double, 36>;
    for (int b = 0; b < 2; b++) {
      double raw[36];
      load_reals<double, 36>(base + (long)b * Wd::NW * Vh * Wd::W, Vh, h, raw);
      for (int i = 0; i < 6; i++)
        for (int j = 0; j < 6; j++) {
          C v;
          if (i == j) {
            v = cxd(raw[i], 0.0);
          } else if (i > j) {
            const int k = 6 + 2 * (i * (i - 1) / 2 + j);
            v = cxd(raw[k], raw[k + 1]);
          } else {
            const int k = 6 + 2 * (j * (j - 1) / 2 + i);
            v = cxd(raw[k], -raw[k + 1]);
          }
          Xs[(6 * b + i) * 12 + 6 * b + j] = st2(v);
        }
    }
  }
  for (int mu = 0; mu < 4; mu++) {
    const double sf = (mu == 3 && tbc && x[3] == d.L[3] - 1) ? -1.0 : 1.0;
    const double sb = (mu == 3 && tbc && x[3] == 0) ? -1.0 : 1.0;
    const long sbw = mg_shift(d, x, mu, -1);
    const double *Uf = U + (s * 4 + mu) * 18;
    const double *Ub = U + (sbw * 4 + mu) * 18;
    double2 *Fs = F + ((long)mu * d.V + s) * 144;
    double2 *Bs = B + ((long)mu * d.V + s) * 144;
    for (int a = 0; a < 4; a++)
      for (int bb = 0; bb < 4; bb++) {
        const C g = gamma_entry(mu, a, bb);
        const double one = a == bb ? 1.0 : 0.0;
        const C pm = cxd(one - g.r, -g.i);  // (1 - gamma_mu)[a][bb]
        const C pp = cxd(one + g.r, g.i);   // (1 + gamma_mu)[a][bb]
        for (int i = 0; i < 3; i++)
          for (int j = 0; j < 3; j++) {
            const C uf = cxd(Uf[2 * (3 * i + j)], Uf[2 * (3 * i + j) + 1]);
            const C ub = cxd(Ub[2 * (3 * j + i)], -Ub[2 * (3 * j + i) + 1]);  // (U^dag)[i][j]
            Fs[(3 * a + i) * 12 + 3 * bb + j] = st2((-kappa * sf) * (pm * uf));
            Bs[(3 * a + i) * 12 + 3 * bb + j] = st2((-kappa * sb) * (pp * ub));
          }
      }
  }
}

// out = D in; one thread per (site, row)
__global__ void __launch_bounds__(kMgT) mg_apply_kernel(MgDims d, int n, const double2 *__restrict__ X,
                                                         const double2 *__restrict__ F,
                                                         const double2 *__restrict__ B,
                                                         const double2 *__restrict__ in, double2 *out) {
  const long total = d.V * n;
  const long nn = (long)n * n;
  for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (long)gridDim.x * blockDim.x) {
    const long s = e / n;
    const int i = (int)(e % n);
    int x[4];
    mg_coords(d, s, x);
    C acc = cxd(0.0, 0.0);
    const double2 *row = X + s * nn + (long)i * n;
    const double2 *v = in + s * n;
    for (int j = 0; j < n; j++) acc = cmadd(ld2(row, j), ld2(v, j), acc);
    for (int mu = 0; mu < 4; mu++) {
      const double2 *rf = F + ((long)mu * d.V + s) * nn + (long)i * n;
      const double2 *vf = in + mg_shift(d, x, mu, 1) * n;
      for (int j = 0; j < n; j++) acc = cmadd(ld2(rf, j), ld2(vf, j), acc);
      const double2 *rb = B + ((long)mu * d.V + s) * nn + (long)i * n;
      const double2 *vb = in + mg_shift(d, x, mu, -1) * n;
      for (int j = 0; j < n; j++) acc = cmadd(ld2(rb, j), ld2(vb, j), acc);
    }
    out[e] = st2(acc);
  }
}

// block-wide sum of one complex value per thread (fixed tree); every thread
// gets the sum
__device__ __forceinline__ C block_sum(C v, double2 *red) {
  const int t = threadIdx.x;
  red[t] = st2(v);
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (t < w) red[t] = make_double2(red[t].x + red[t + w].x, red[t].y + red[t + w].y);
    __syncthreads();
  }
  const C r = ld2(red, 0);
  __syncthreads();
  return r;
}

// P on one block and one chirality (blockIdx.x = coarse site, blockIdx.y =
// chirality): the nv vectors restricted there, orthonormalised one after the
// other by classical Gram-Schmidt applied twice (each column made orthogonal
// to the earlier ones, then normalised: the QR factor with a real positive
// diagonal).  A column whose norm falls below 1e-12 of its norm before the
// projections sets *flag and is left zero.
__global__ void __launch_bounds__(kMgOrthT) mg_orth_kernel(MgDims fd, MgDims cd, int4 blk, int n, int nv,
                                                            const double2 *__restrict__ vecs, double2 *P, int *flag) {
  __shared__ double2 red[kMgOrthT];
  __shared__ double2 dots[kMgMaxN];
  const long xcs = blockIdx.x;
  const int c = blockIdx.y;
  const int nh = n / 2, nc = 2 * nv;
  int xc[4];
  mg_coords(cd, xcs, xc);
  const long len = (long)blk.x * blk.y * blk.z * blk.w * nh;
  // element e of a restricted vector: block site e / nh, component c nh + e % nh
  auto addr = [&](long e, int col) -> long {
    int o[4];
    const long s = mg_block_site(fd, blk, xc, (int)(e / nh), o);
    return (s * n + c * nh + e % nh) * nc + col;
  };
  for (int k = 0; k < nv; k++) {
    const int col = c * nv + k;
    C nrm0 = cxd(0.0, 0.0);
    for (long e = threadIdx.x; e < len; e += blockDim.x) {
      int o[4];
      const long s = mg_block_site(fd, blk, xc, (int)(e / nh), o);
      const C v = ld2(vecs, ((long)k * fd.V + s) * n + c * nh + e % nh);
      P[addr(e, col)] = st2(v);
      nrm0.r += v.r * v.r + v.i * v.i;
    }
    nrm0 = block_sum(nrm0, red);
    for (int pass = 0; pass < 2; pass++) {
      for (int j = 0; j < k; j++) {
        C acc = cxd(0.0, 0.0);
        for (long e = threadIdx.x; e < len; e += blockDim.x)
          acc = cmadd(conjg(ld2(P, addr(e, c * nv + j))), ld2(P, addr(e, col)), acc);
        acc = block_sum(acc, red);
        if (threadIdx.x == 0) dots[j] = st2(acc);
      }
      __syncthreads();
      for (long e = threadIdx.x; e < len; e += blockDim.x) {
        C v = ld2(P, addr(e, col));
        for (int j = 0; j < k; j++) v = v - ld2(dots, j) * ld2(P, addr(e, c * nv + j));
        P[addr(e, col)] = st2(v);
      }
      __syncthreads();
    }
    C nrm = cxd(0.0, 0.0);
    for (long e = threadIdx.x; e < len; e += blockDim.x) {
      const C v = ld2(P, addr(e, col));
      nrm.r += v.r * v.r + v.i * v.i;
    }
    nrm = block_sum(nrm, red);
    const bool ok = sqrt(nrm.r) > 1e-12 * sqrt(nrm0.r);
    if (!ok && threadIdx.x == 0) atomicOr(flag, 1);
    const double scale = ok ? 1.0 / sqrt(nrm.r) : 0.0;
    for (long e = threadIdx.x; e < len; e += blockDim.x) {
      const C v = ld2(P, addr(e, col));
      P[addr(e, col)] = st2(scale * v);
    }
    __syncthreads();
  }
}

// out(s) = P(s) w(block of s); one thread per (fine site, component)
__global__ void __launch_bounds__(kMgT) mg_prolong_kernel(MgDims fd, MgDims cd, int4 blk, int n, int nc,
                                                           const double2 *__restrict__ P,
                                                           const double2 *__restrict__ w, double2 *out) {
  const long total = fd.V * n;
  for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (long)gridDim.x * blockDim.x) {
    const long s = e / n;
    int x[4];
    mg_coords(fd, s, x);
    const int xc[4] = {x[0] / blk.x, x[1] / blk.y, x[2] / blk.z, x[3] / blk.w};
    const double2 *wc = w + mg_index(cd, xc) * nc;
    const double2 *row = P + e * nc;
    C acc = cxd(0.0, 0.0);
    for (int k = 0; k < nc; k++) acc = cmadd(ld2(row, k), ld2(wc, k), acc);
    out[e] = st2(acc);
  }
}

// out(xc) = sum over the block's sites s of P(s)^H v(s); one thread per
// (coarse site, coarse component), sites in block order
__global__ void __launch_bounds__(kMgT) mg_restrict_kernel(MgDims fd, MgDims cd, int4 blk, int n, int nc,
                                                            const double2 *__restrict__ P,
                                                            const double2 *__restrict__ v, double2 *out) {
  const long total = cd.V * nc;
  const int bsz = blk.x * blk.y * blk.z * blk.w;
  for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (long)gridDim.x * blockDim.x) {
    const long xcs = e / nc;
    const int k = (int)(e % nc);
    int xc[4];
    mg_coords(cd, xcs, xc);
    C acc = cxd(0.0, 0.0);
    for (int q = 0; q < bsz; q++) {
      int o[4];
      const long s = mg_block_site(fd, blk, xc, q, o);
      for (int i = 0; i < n; i++) acc = cmadd(conjg(ld2(P, (s * n + i) * nc + k)), ld2(v, s * n + i), acc);
    }
    out[e] = st2(acc);
  }
}

// one coarse matrix of P^H D P (blockIdx.x = coarse site, blockIdx.y = target:
// 0 = X_c, 1 + mu = F_c[mu], 5 + mu = B_c[mu]).  For each fine term
// P(s)^H T P(s') that lands there (the site term and the hops inside the
// block for X_c, the hops across the block's forward / backward face in mu
// for F_c / B_c), W = T P(s') is formed in shared memory and P(s)^H W added
// to the thread's entries; sites and terms in a fixed order.
__global__ void __launch_bounds__(kMgCoarsenT) mg_coarsen_kernel(MgDims fd, MgDims cd, int4 blk, int n, int nc,
                                                                  const double2 *__restrict__ X,
                                                                  const double2 *__restrict__ F,
                                                                  const double2 *__restrict__ B,
                                                                  const double2 *__restrict__ P, double2 *Xc,
                                                                  double2 *Fc, double2 *Bc) {
  extern __shared__ double2 W[];  // n x nc
  const long xcs = blockIdx.x;
  const int t = blockIdx.y;
  int xc[4];
  mg_coords(cd, xcs, xc);
  const int b[4] = {blk.x, blk.y, blk.z, blk.w};
  const int bsz = b[0] * b[1] * b[2] * b[3];
  const long nn = (long)n * n;
  const int nent = nc * nc;
  C acc[kMgMaxEnt];
  for (int r = 0; r < kMgMaxEnt; r++) acc[r] = cxd(0.0, 0.0);
  for (int q = 0; q < bsz; q++) {
    int o[4];
    const long s = mg_block_site(fd, blk, xc, q, o);
    int x[4];
    mg_coords(fd, s, x);
    // the terms of site s for this target: (matrix, neighbour site)
    for (int term = 0; term < 9; term++) {
      const double2 *T = nullptr;
      long s2 = s;
      if (term == 0) {
        if (t == 0) T = X + s * nn;
      } else {
        const int mu = (term - 1) % 4;
        const bool fwd = term <= 4;
        const bool cross = fwd ? (o[mu] == b[mu] - 1) : (o[mu] == 0);
        const bool want = t == 0 ? !cross : (cross && t == term);
        if (want) {
          T = (fwd ? F : B) + ((long)mu * fd.V + s) * nn;
          s2 = mg_shift(fd, x, mu, fwd ? 1 : -1);
        }
      }
      if (!T) continue;  // uniform across the block: every thread sees the same t, q, term
      __syncthreads();
      for (int e = threadIdx.x; e < n * nc; e += blockDim.x) {
        const int i = e / nc, l = e % nc;
        C w = cxd(0.0, 0.0);
        for (int j = 0; j < n; j++) w = cmadd(ld2(T, (long)i * n + j), ld2(P, (s2 * n + j) * nc + l), w);
        W[e] = st2(w);
      }
      __syncthreads();
      for (int r = 0; r < kMgMaxEnt; r++) {
        const int ent = threadIdx.x + r * blockDim.x;
        if (ent >= nent) break;
        const int k = ent / nc, l = ent % nc;
        C a = acc[r];
        for (int i = 0; i < n; i++) a = cmadd(conjg(ld2(P, (s * n + i) * nc + k)), ld2(W, (long)i * nc + l), a);
        acc[r] = a;
      }
    }
  }
  double2 *dst = t == 0 ? Xc + xcs * nent : (t <= 4 ? Fc + ((long)(t - 1) * cd.V + xcs) * nent
                                                     : Bc + ((long)(t - 5) * cd.V + xcs) * nent);
  for (int r = 0; r < kMgMaxEnt; r++) {
    const int ent = threadIdx.x + r * blockDim.x;
    if (ent >= nent) break;
    dst[ent] = st2(acc[r]);
  }
}

// partials[j nb + block] = this block's share of <X_j, y> = sum conj(X_j) y
__global__ void __launch_bounds__(kMgT) mg_dots_kernel(long len, int k, const double2 *__restrict__ Xv,
                                                        const double2 *__restrict__ y, double2 *partials) {
  __shared__ double2 red[kMgT];
  for (int j = 0; j < k; j++) {
    C acc = cxd(0.0, 0.0);
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < len; i += (long)gridDim.x * blockDim.x)
      acc = cmadd(conjg(ld2(Xv, (long)j * len + i)), ld2(y, i), acc);
    acc = block_sum(acc, red);
    if (threadIdx.x == 0) partials[(long)j * gridDim.x + blockIdx.x] = st2(acc);
  }
}

__global__ void mg_dots_finish_kernel(int k, int nb, const double2 *partials, double2 *out) {
  const int j = threadIdx.x;
  if (j >= k) return;
  C acc = cxd(0.0, 0.0);
  for (int b = 0; b < nb; b++) acc = acc + ld2(partials, (long)j * nb + b);
  out[j] = st2(acc);
}

// y += sum_j c_j X_j
__global__ void __launch_bounds__(kMgT) mg_axpys_kernel(long len, int k, MgCoefs cf, const double2 *__restrict__ Xv,
                                                         double2 *y) {
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < len; i += (long)gridDim.x * blockDim.x) {
    C acc = ld2(y, i);
    for (int j = 0; j < k; j++) acc = cmadd(cxd(cf.c[j].x, cf.c[j].y), ld2(Xv, (long)j * len + i), acc);
    y[i] = st2(acc);
  }
}

// y = a x + b y (x may be y)
__global__ void __launch_bounds__(kMgT) mg_axpby_kernel(long len, double2 a, const double2 *x, double2 b, double2 *y) {
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < len; i += (long)gridDim.x * blockDim.x) {
    const C xv = ld2(x, i), yv = ld2(y, i);
    y[i] = st2(cxd(a.x, a.y) * xv + cxd(b.x, b.y) * yv);
  }
}

}  // namespace
}  // namespace lqcd

namespace lqcd {
namespace {

lqcd_status mg_check_ptr(const void *p, const char *what) {
  if (!p) return set_error(LQCD_ERR_ARG, "%s is NULL", what);
  if (reinterpret_cast<uintptr_t>(p) % 16) return set_error(LQCD_ERR_ARG, "%s must be 16-byte aligned", what);
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return set_error(LQCD_ERR_ARG, "%s: not a CUDA pointer", what);
  }
  int dev = 0;
  LQ_CU(cudaGetDevice(&dev));
  if ((a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged) || a.device != dev)
    return set_error(LQCD_ERR_ARG, "%s must be device memory of the current device", what);
  return LQCD_OK;
}

lqcd_status mg_dims(const int dims[4], MgDims *d) {
  if (!dims) return set_error(LQCD_ERR_ARG, "dims is NULL");
  d->V = 1;
  for (int mu = 0; mu < 4; mu++) {
    if (dims[mu] < 1 || dims[mu] > 4096) return set_error(LQCD_ERR_ARG, "dims[%d] = %d outside 1..4096", mu, dims[mu]);
    d->L[mu] = dims[mu];
    d->V *= dims[mu];
  }
  if (d->V > (1L << 30)) return set_error(LQCD_ERR_ARG, "lattice of %ld sites is too large", d->V);
  return LQCD_OK;
}

lqcd_status mg_n(int n, const char *what) {
  if (n < 2 || n > kMgMaxN || n % 2) return set_error(LQCD_ERR_ARG, "%s = %d: even, 2..%d", what, n, kMgMaxN);
  return LQCD_OK;
}

// the coarse lattice of `block` on fd, and the coarse component count nc = 2 nv
lqcd_status mg_blocks(const MgDims &fd, const int block[4], MgDims *cd, int4 *b) {
  if (!block) return set_error(LQCD_ERR_ARG, "block is NULL");
  int c[4];
  for (int mu = 0; mu < 4; mu++) {
    if (block[mu] < 1 || fd.L[mu] % block[mu])
      return set_error(LQCD_ERR_ARG, "block[%d] = %d does not divide %d", mu, block[mu], fd.L[mu]);
    c[mu] = fd.L[mu] / block[mu];
  }
  LQ_TRY(mg_dims(c, cd));
  *b = make_int4(block[0], block[1], block[2], block[3]);
  return LQCD_OK;
}

unsigned mg_grid(long work) {
  const long b = (work + kMgT - 1) / kMgT;
  return (unsigned)(b < 1 ? 1 : (b > 152L * 16 ? 152L * 16 : b));
}

}  // namespace
}  // namespace lqcd

using namespace lqcd;

extern "C" {

lqcd_status lqcd_mg_fine_stencil(lqcd_ctx *c, void *X, void *F, void *B) {
  if (!c) return set_error(LQCD_ERR_ARG, "NULL context");
  if (!c->have_gauge) return set_error(LQCD_ERR_STATE, "no gauge field loaded");
  if (!c->have_kappa) return set_error(LQCD_ERR_STATE, "lqcd_clover (kappa, c_sw) not called");
  LQ_TRY(mg_check_ptr(X, "X"));
  LQ_TRY(mg_check_ptr(F, "F"));
  LQ_TRY(mg_check_ptr(B, "B"));
  MgDims d;
  LQ_TRY(mg_dims(c->dims, &d));
  const char *A0 = nullptr, *A1 = nullptr;
  if (c->clover_on) {
    A0 = static_cast<const char *>(c->clov[LQCD_F64].A[0]);
    A1 = static_cast<const char *>(c->clov[LQCD_F64].A[1]);
  }
  mg_fine_kernel<<<(unsigned)((d.V + kMgT - 1) / kMgT), kMgT, 0, c->stream>>>(
      d, c->tbc, c->kappa, c->U64, A0, A1, c->Vh, (double2 *)X, (double2 *)F, (double2 *)B);
  LQ_CU(cudaGetLastError());
  return LQCD_OK;
}

lqcd_status lqcd_mg_apply(lqcd_ctx *c, const int dims[4], int n, const void *X, const void *F, const void *B,
                          const void *in, void *out) {
  if (!c) return set_error(LQCD_ERR_ARG, "NULL context");
  MgDims d;
  LQ_TRY(mg_dims(dims, &d));
  LQ_TRY(mg_n(n, "n"));
  LQ_TRY(mg_check_ptr(X, "X"));
  LQ_TRY(mg_check_ptr(F, "F"));
  LQ_TRY(mg_check_ptr(B, "B"));
  LQ_TRY(mg_check_ptr(in, "in"));
  LQ_TRY(mg_check_ptr(out, "out"));
  if (in == out) return set_error(LQCD_ERR_ARG, "in and out must be different arrays");
  mg_apply_kernel<<<mg_grid(d.V * n), kMgT, 0, c->stream>>>(d, n, (const double2 *)X, (const double2 *)F,
                                                             (const double2 *)B, (const double2 *)in,
                                                             (double2 *)out);
  LQ_CU(cudaGetLastError());
  return LQCD_OK;
}

lqcd_status lqcd_mg_orthonormalize(lqcd_ctx *c, const int dims[4], int n, const int block[4], int nv,
                                   const void *vecs, void *P) {
  if (!c) return set_error(LQCD_ERR_ARG, "NULL context");
  MgDims fd, cd;
  int4 b;
  LQ_TRY(mg_dims(dims, &fd));
  LQ_TRY(mg_n(n, "n"));
  LQ_TRY(mg_blocks(fd, block, &cd, &b));
  const long rows = (long)b.x * b.y * b.z * b.w * (n / 2);
  if (nv < 1 || 2 * nv > kMgMaxN) return set_error(LQCD_ERR_ARG, "nv = %d outside 1..%d", nv, kMgMaxN / 2);
  if (nv > rows) return set_error(LQCD_ERR_ARG, "%d vectors exceed the %ld components of a block chirality", nv, rows);
  LQ_TRY(mg_check_ptr(vecs, "vecs"));
  LQ_TRY(mg_check_ptr(P, "P"));
  int *flag = reinterpret_cast<int *>(c->results);
  LQ_CU(cudaMemsetAsync(flag, 0, sizeof(int), c->stream));
  LQ_CU(cudaMemsetAsync(P, 0, (size_t)fd.V * n * 2 * nv * sizeof(double2), c->stream));
  mg_orth_kernel<<<dim3((unsigned)cd.V, 2), kMgOrthT, 0, c->stream>>>(fd, cd, b, n, nv, (const double2 *)vecs,
                                                                      (double2 *)P, flag);
  LQ_CU(cudaGetLastError());
  LQ_CU(cudaMemcpyAsync(c->h_results, c->results, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  LQ_CU(cudaStreamSynchronize(c->stream));
  int hflag = 0;
  std::memcpy(&hflag, c->h_results, sizeof(int));
  if (hflag) return set_error(LQCD_ERR_SINGULAR, "near-null vectors linearly dependent on a block");
  return LQCD_OK;
}

lqcd_status lqcd_mg_prolong(lqcd_ctx *c, const int dims[4], int n, const int block[4], int nc, const void *P,
                            const void *w, void *out) {
  if (!c) return set_error(LQCD_ERR_ARG, "NULL context");
  MgDims fd, cd;
  int4 b;
  LQ_TRY(mg_dims(dims, &fd));
  LQ_TRY(mg_n(n, "n"));
  LQ_TRY(mg_n(nc, "nc"));
  LQ_TRY(mg_blocks(fd, block, &cd, &b));
  LQ_TRY(mg_check_ptr(P, "P"));
  LQ_TRY(mg_check_ptr(w, "w"));
  LQ_TRY(mg_check_ptr(out, "out"));
  mg_prolong_kernel<<<mg_grid(fd.V * n), kMgT, 0, c->stream>>>(fd, cd, b, n, nc, (const double2 *)P,
                                                                (const double2 *)w, (double2 *)out);
  LQ_CU(cudaGetLastError());
  return LQCD_OK;
}

lqcd_status lqcd_mg_restrict(lqcd_ctx *c, const int dims[4], int n, const int block[4], int nc, const void *P,
                             const void *v, void *out) {
  if (!c) return set_error(LQCD_ERR_ARG, "NULL context");
  MgDims fd, cd;
  int4 b;
  LQ_TRY(mg_dims(dims, &fd));
  LQ_TRY(mg_n(n, "n"));
  LQ_TRY(mg_n(nc, "nc"));
  LQ_TRY(mg_blocks(fd, block, &cd, &b));
  LQ_TRY(mg_check_ptr(P, "P"));
  LQ_TRY(mg_check_ptr(v, "v"));
  LQ_TRY(mg_check_ptr(out, "out"));
  mg_restrict_kernel<<<mg_grid(cd.V * nc), kMgT, 0, c->stream>>>(fd, cd, b, n, nc, (const double2 *)P,
                                                                  (const double2 *)v, (double2 *)out);
  LQ_CU(cudaGetLastError());
  return LQCD_OK;
}

lqcd_status lqcd_mg_coarsen(lqcd_ctx *c, const int dims[4], int n, const int block[4], int nc, const void *X,
                            const void *F, const void *B, const void *P, void *Xc, void *Fc, void *Bc) {
  if (!c) return set_error(LQCD_ERR_ARG, "NULL context");
  MgDims fd, cd;
  int4 b;
  LQ_TRY(mg_dims(dims, &fd));
  LQ_TRY(mg_n(n, "n"));
  LQ_TRY(mg_n(nc, "nc"));
  LQ_TRY(mg_blocks(fd, block, &cd, &b));
  const void *ptrs[] = {X, F, B, P, Xc, Fc, Bc};
  const char *names[] = {"X", "F", "B", "P", "Xc", "Fc", "Bc"};
  for (int i = 0; i < 7; i++) LQ_TRY(mg_check_ptr(ptrs[i], names[i]));
  const size_t smem = (size_t)n * nc * sizeof(double2);
  if (smem > 48 * 1024)
    LQ_CU(cudaFuncSetAttribute(mg_coarsen_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  mg_coarsen_kernel<<<dim3((unsigned)cd.V, 9), kMgCoarsenT, smem, c->stream>>>(
      fd, cd, b, n, nc, (const double2 *)X, (const double2 *)F, (const double2 *)B, (const double2 *)P,
      (double2 *)Xc, (double2 *)Fc, (double2 *)Bc);
  LQ_CU(cudaGetLastError());
  return LQCD_OK;
}

lqcd_status lqcd_mg_dots(lqcd_ctx *c, long len, int k, const void *Xv, const void *y, double *out) {
  if (!c) return set_error(LQCD_ERR_ARG, "NULL context");
  if (len < 1) return set_error(LQCD_ERR_ARG, "len = %ld must be positive", len);
  if (k < 1 || k > kMgMaxK) return set_error(LQCD_ERR_ARG, "k = %d outside 1..%d", k, kMgMaxK);
  if (!out) return set_error(LQCD_ERR_ARG, "out is NULL");
  LQ_TRY(mg_check_ptr(Xv, "X"));
  LQ_TRY(mg_check_ptr(y, "y"));
  const int nb = (int)std::min<long>((len + kMgT - 1) / kMgT, 2 * 152);
  // partial sums: k x nb complex = 2 k nb doubles of the context's scratch
  const long per = (c->Vh + 31) / 32 + 1;
  LQ_TRY(ensure_partials(c, (int)((2L * k * nb + per - 1) / per)));
  mg_dots_kernel<<<nb, kMgT, 0, c->stream>>>(len, k, (const double2 *)Xv, (const double2 *)y,
                                             reinterpret_cast<double2 *>(c->partials));
  LQ_CU(cudaGetLastError());
  mg_dots_finish_kernel<<<1, kMgMaxK, 0, c->stream>>>(k, nb, reinterpret_cast<const double2 *>(c->partials),
                                                      reinterpret_cast<double2 *>(c->results));
  LQ_CU(cudaGetLastError());
  LQ_CU(cudaMemcpyAsync(c->h_results, c->results, 2 * k * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  LQ_CU(cudaStreamSynchronize(c->stream));
  std::memcpy(out, c->h_results, 2 * k * sizeof(double));
  return LQCD_OK;
}

lqcd_status lqcd_mg_axpys(lqcd_ctx *c, long len, int k, const double *coef, const void *Xv, void *y) {
  if (!c) return set_error(LQCD_ERR_ARG, "NULL context");
  if (len < 1) return set_error(LQCD_ERR_ARG, "len = %ld must be positive", len);
  if (k < 1 || k > kMgMaxK) return set_error(LQCD_ERR_ARG, "k = %d outside 1..%d", k, kMgMaxK);
  if (!coef) return set_error(LQCD_ERR_ARG, "coef is NULL");
  LQ_TRY(mg_check_ptr(Xv, "X"));
  LQ_TRY(mg_check_ptr(y, "y"));
  MgCoefs cf;
  for (int j = 0; j < kMgMaxK; j++) cf.c[j] = j < k ? make_double2(coef[2 * j], coef[2 * j + 1]) : make_double2(0, 0);
  mg_axpys_kernel<<<mg_grid(len), kMgT, 0, c->stream>>>(len, k, cf, (const double2 *)Xv, (double2 *)y);
  LQ_CU(cudaGetLastError());
  return LQCD_OK;
}

lqcd_status lqcd_mg_axpby(lqcd_ctx *c, long len, const double a[2], const void *x, const double b[2], void *y) {
  if (!c) return set_error(LQCD_ERR_ARG, "NULL context");
  if (len < 1) return set_error(LQCD_ERR_ARG, "len = %ld must be positive", len);
  if (!a || !b) return set_error(LQCD_ERR_ARG, "coefficients are NULL");
  LQ_TRY(mg_check_ptr(x, "x"));
  LQ_TRY(mg_check_ptr(y, "y"));
  mg_axpby_kernel<<<mg_grid(len), kMgT, 0, c->stream>>>(len, make_double2(a[0], a[1]), (const double2 *)x,
                                                        make_double2(b[0], b[1]), (double2 *)y);
  LQ_CU(cudaGetLastError());
  return LQCD_OK;
}

}  // extern "C"
