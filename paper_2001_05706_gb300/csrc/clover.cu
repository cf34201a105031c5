// Clover term construction on the GPU, in FP64 (set-up, once per gauge
// field and (kappa, c_sw)).
//
// Per site: the four plaquette leaves Q_munu(x) of each of the six planes,
// F_munu = (Q - Q^dag)/(8i) minus trace/3, and
//   A(x) = 1 - c_sw kappa sum_{mu<nu} sigma_munu (x) F_munu(x).
// In the DeGrand-Rossi chiral basis g_mu = [[0, B_mu], [B_mu^dag, 0]], so
// sigma_munu = (i/2)[g_mu, g_nu] is block diagonal with blocks
//   upper (spins 0,1): (i/2)(B_mu B_nu^dag - B_nu B_mu^dag)
//   lower (spins 2,3): (i/2)(B_mu^dag B_nu - B_nu^dag B_mu)
// and A = diag(A+, A-) with two 6x6 Hermitian blocks (index 3*spin + colour).
// Each block is factorised A = L D L^dag (unit lower L, real D) and
// inverted column by column.  Blocks are written packed (6 real diagonal
// entries, then the 15 complex entries below the diagonal in row order).
#include "internal.h"

namespace lqcd {

// B_mu as (row, column) of the single non-zero entry in each row and its value
__device__ __forceinline__ cx<double> Bmat(int mu, int a, int b) {
  // mu=0: [[0, i], [i, 0]]; mu=1: [[0,-1],[1,0]]; mu=2: [[i,0],[0,-i]]; mu=3: identity
  switch (mu) {
    case 0: return (a != b) ? mk<double>(0, 1) : mk<double>(0, 0);
    case 1: return (a != b) ? mk<double>(a == 0 ? -1.0 : 1.0, 0) : mk<double>(0, 0);
    case 2: return (a == b) ? mk<double>(0, a == 0 ? 1.0 : -1.0) : mk<double>(0, 0);
    default: return (a == b) ? mk<double>(1, 0) : mk<double>(0, 0);
  }
}

// sigma block (upper: lower=0, lower: lower=1) entry (a, b) for the plane (mu, nu)
__device__ __forceinline__ cx<double> sigma_block(int lower, int mu, int nu, int a, int b) {
  cx<double> s = mk<double>(0, 0);
  for (int k = 0; k < 2; k++) {
    if (!lower) {  // B_mu B_nu^dag - B_nu B_mu^dag
      s = s + Bmat(mu, a, k) * conjg(Bmat(nu, b, k)) - Bmat(nu, a, k) * conjg(Bmat(mu, b, k));
    } else {  // B_mu^dag B_nu - B_nu^dag B_mu
      s = s + conjg(Bmat(mu, k, a)) * Bmat(nu, k, b) - conjg(Bmat(nu, k, a)) * Bmat(mu, k, b);
    }
  }
  return mk<double>(-0.5 * s.i, 0.5 * s.r);  // (i/2) s
}

struct M3 {
  cx<double> m[3][3];
};

__device__ __forceinline__ M3 ld(const double *U, long s, int mu) {
  M3 r;
  const double *u = U + (s * 4 + mu) * 18;
  for (int i = 0; i < 9; i++) r.m[i / 3][i % 3] = mk<double>(u[2 * i], u[2 * i + 1]);
  return r;
}
__device__ __forceinline__ M3 mul(const M3 &a, const M3 &b) {
  M3 c;
  for (int i = 0; i < 3; i++)
    for (int j = 0; j < 3; j++) {
      cx<double> t = mk<double>(0, 0);
      for (int k = 0; k < 3; k++) t = cmadd(a.m[i][k], b.m[k][j], t);
      c.m[i][j] = t;
    }
  return c;
}
__device__ __forceinline__ M3 dag(const M3 &a) {
  M3 c;
  for (int i = 0; i < 3; i++)
    for (int j = 0; j < 3; j++) c.m[i][j] = conjg(a.m[j][i]);
  return c;
}

__device__ __forceinline__ long lex_shift(const int L[4], const int x[4], int mu, int dir, int nu = -1, int dir2 = 0) {
  int y[4] = {x[0], x[1], x[2], x[3]};
  y[mu] = (y[mu] + dir + L[mu]) % L[mu];
  if (nu >= 0) y[nu] = (y[nu] + dir2 + L[nu]) % L[nu];
  return y[0] + (long)L[0] * (y[1] + (long)L[1] * (y[2] + (long)L[2] * y[3]));
}

// F_munu at site x (traceless, Hermitian)
__device__ M3 field_strength(const int L[4], const double *U, const int x[4], int mu, int nu) {
  const long s = lex_shift(L, x, 0, 0);
  const long xpm = lex_shift(L, x, mu, 1), xpn = lex_shift(L, x, nu, 1);
  const long xmm = lex_shift(L, x, mu, -1), xmn = lex_shift(L, x, nu, -1);
  const long xmm_pn = lex_shift(L, x, mu, -1, nu, 1), xmm_mn = lex_shift(L, x, mu, -1, nu, -1);
  const long xmn_pm = lex_shift(L, x, nu, -1, mu, 1);
  M3 q1 = mul(mul(ld(U, s, mu), ld(U, xpm, nu)), mul(dag(ld(U, xpn, mu)), dag(ld(U, s, nu))));
  M3 q2 = mul(mul(ld(U, s, nu), dag(ld(U, xmm_pn, mu))), mul(dag(ld(U, xmm, nu)), ld(U, xmm, mu)));
  M3 q3 = mul(mul(dag(ld(U, xmm, mu)), dag(ld(U, xmm_mn, nu))), mul(ld(U, xmm_mn, mu), ld(U, xmn, nu)));
  M3 q4 = mul(mul(dag(ld(U, xmn, nu)), ld(U, xmn, mu)), mul(ld(U, xmn_pm, nu), dag(ld(U, s, mu))));
  M3 f;
  for (int i = 0; i < 3; i++)
    for (int j = 0; j < 3; j++) {
      cx<double> q = q1.m[i][j] + q2.m[i][j] + q3.m[i][j] + q4.m[i][j];
      cx<double> qt = conjg(q1.m[j][i] + q2.m[j][i] + q3.m[j][i] + q4.m[j][i]);
      cx<double> d = q - qt;  // (Q - Q^dag) / (8 i) = -i d / 8
      f.m[i][j] = mk<double>(d.i / 8.0, -d.r / 8.0);
    }
  cx<double> tr = f.m[0][0] + f.m[1][1] + f.m[2][2];
  for (int i = 0; i < 3; i++) f.m[i][i] = f.m[i][i] - (1.0 / 3.0) * tr;
  return f;
}

// A = L D L^dag, then A^-1; returns false on a zero pivot.
__device__ bool ldl_inverse6(const cx<double> (&A)[6][6], cx<double> (&Ai)[6][6]) {
  cx<double> Lm[6][6];
  double D[6];
  for (int j = 0; j < 6; j++) {
    double d = A[j][j].r;
    for (int k = 0; k < j; k++) d -= (Lm[j][k].r * Lm[j][k].r + Lm[j][k].i * Lm[j][k].i) * D[k];
    if (!(fabs(d) > 1e-300)) return false;
    D[j] = d;
    Lm[j][j] = mk<double>(1, 0);
    for (int i = j + 1; i < 6; i++) {
      cx<double> t = A[i][j];
      for (int k = 0; k < j; k++) t = t - D[k] * (Lm[i][k] * conjg(Lm[j][k]));
      Lm[i][j] = (1.0 / d) * t;
    }
  }
  for (int c = 0; c < 6; c++) {
    cx<double> y[6];
    for (int i = 0; i < 6; i++) {  // L y = e_c
      cx<double> t = mk<double>(i == c ? 1.0 : 0.0, 0);
      for (int k = 0; k < i; k++) t = t - Lm[i][k] * y[k];
      y[i] = t;
    }
    for (int i = 0; i < 6; i++) y[i] = (1.0 / D[i]) * y[i];
    for (int i = 5; i >= 0; i--) {  // L^dag x = y
      cx<double> t = y[i];
      for (int k = i + 1; k < 6; k++) t = t - conjg(Lm[k][i]) * Ai[k][c];
      Ai[i][c] = t;
    }
  }
  return true;
}

__device__ __forceinline__ void store_block(double *base, long Vh, long h, int blk, const cx<double> (&M)[6][6]) {
  double raw[36];
  for (int i = 0; i < 6; i++) raw[i] = M[i][i].r;
  for (int i = 1; i < 6; i++)
    for (int j = 0; j < i; j++) {
      const int k = 6 + 2 * (i * (i - 1) / 2 + j);
      raw[k] = M[i][j].r;
      raw[k + 1] = M[i][j].i;
    }
  using Wd = Words<double, 36>;
  store_reals<double, 36>(reinterpret_cast<char *>(base) + (long)blk * Wd::NW * Vh * Wd::W, Vh, h, raw);
}

__global__ void __launch_bounds__(64) clover_build_kernel(Geom g, const double *__restrict__ U, double kappa,
                                                           double csw, double *A0, double *A1, double *Ai0,
                                                           double *Ai1, int *singular,
                                                           unsigned long long *bound) {
  const long s = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const long V = 2 * g.Vh;
  if (s >= V) return;
  int x[4];
  long r = s;
  for (int mu = 0; mu < 4; mu++) {
    x[mu] = (int)(r % g.L[mu]);
    r /= g.L[mu];
  }
  const int p = (x[0] + x[1] + x[2] + x[3]) & 1;
  const long h = s >> 1;
  cx<double> Ab[2][6][6];
  for (int b = 0; b < 2; b++)
    for (int i = 0; i < 6; i++)
      for (int j = 0; j < 6; j++) Ab[b][i][j] = mk<double>(i == j ? 1.0 : 0.0, 0);
  const double c = -csw * kappa;
  for (int mu = 0; mu < 4; mu++)
    for (int nu = mu + 1; nu < 4; nu++) {
      M3 F = field_strength(g.L, U, x, mu, nu);
      for (int b = 0; b < 2; b++)
        for (int sa = 0; sa < 2; sa++)
          for (int sb = 0; sb < 2; sb++) {
            cx<double> sg = sigma_block(b, mu, nu, sa, sb);
            if (sg.r == 0.0 && sg.i == 0.0) continue;
            for (int i = 0; i < 3; i++)
              for (int j = 0; j < 3; j++) Ab[b][3 * sa + i][3 * sb + j] = Ab[b][3 * sa + i][3 * sb + j] + c * (sg * F.m[i][j]);
          }
    }
  double *A = p ? A1 : A0;
  double *Ai = p ? Ai1 : Ai0;
  // Gershgorin: every eigenvalue of a Hermitian block lies within
  // |a_ii| + sum_{j != i} |a_ij| of 0, so the largest row sum bounds ||A||
  double gb = 0.0;
  for (int b = 0; b < 2; b++)
    for (int i = 0; i < 6; i++) {
      double row = 0.0;
      for (int j = 0; j < 6; j++) row += hypot(Ab[b][i][j].r, Ab[b][i][j].i);
      gb = fmax(gb, row);
    }
  // non-negative doubles order like their bit patterns
  atomicMax(bound + p, (unsigned long long)__double_as_longlong(gb));
  for (int b = 0; b < 2; b++) {
    store_block(A, g.Vh, h, b, Ab[b]);
    cx<double> inv[6][6];
    if (!ldl_inverse6(Ab[b], inv)) {
      atomicOr(singular, 1);
      for (int i = 0; i < 6; i++)
        for (int j = 0; j < 6; j++) inv[i][j] = mk<double>(0, 0);
    }
    store_block(Ai, g.Vh, h, b, inv);
  }
}

cudaError_t clover_build(const Geom &g, const double *U, double kappa, double csw, double *A[2], double *Ainv[2],
                         int *singular, unsigned long long *bound, cudaStream_t st) {
  const long V = 2 * g.Vh;
  clover_build_kernel<<<(unsigned)((V + 63) / 64), 64, 0, st>>>(g, U, kappa, csw, A[0], A[1], Ainv[0], Ainv[1],
                                                                 singular, bound);
  return cudaGetLastError();
}

}  // namespace lqcd
