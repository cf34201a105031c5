/*
 * FP64 CPU oracle for the Wilson-clover / overlap fermion hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  The CUDA library
 * shares no code, header, table or helper with it.
 *
 * The paper (Bi et al., "Lattice QCD package GWU-code and QUDA with HIP",
 * Lattice 2019) names the operators it runs -- the Wilson and clover Dirac
 * operators (Table 1: QUDA_DIRAC_WILSON, QUDA_DIRAC_CLOVER), the D-slash
 * kernel (Sec. 3, Sec. 4, Table 2), the overlap inverter (abstract, Sec. 3,
 * Sec. 4) -- but prints no formula.  Every routine below is the standard
 * textbook definition of the operator it names, written out plainly:
 *   - full 4x4 spin matrices, no spin projection;
 *   - the full 12x12 clover matrix per site, inverted by Gauss-Jordan
 *     elimination with partial pivoting;
 *   - even-odd blocks taken by zeroing the other parity of a full-lattice
 *     vector;
 *   - sequential fixed-order reductions.
 * Site loops are parallel (OpenMP) only where sites are independent.
 *
 * Conventions (each a reading of the standard definitions, since the paper
 * fixes none):
 *   lattice  x = (x0,x1,x2,x3), x3 = t; s = x0 + L0(x1 + L1(x2 + L2 x3));
 *            parity (x0+x1+x2+x3) mod 2, even = 0.  Periodic in mu = 0,1,2;
 *            a hop across the t boundary carries a factor -1 when tbc = 1
 *            (applied as a sign, not folded into the links).
 *   gamma    DeGrand-Rossi chiral basis, gamma5 = g0 g1 g2 g3 = diag(1,1,-1,-1).
 *   hopping  (D psi)(x) = sum_mu (1 - g_mu) U_mu(x) psi(x+mu)
 *                              + (1 + g_mu) U_mu(x-mu)^dag psi(x-mu).
 *   clover   Q_munu = sum of the four plaquette leaves at x,
 *            F_munu = (Q - Q^dag)/(8i) minus its trace/3,
 *            A(x)   = 1 - c_sw kappa sum_{mu<nu} sigma_munu F_munu(x),
 *            sigma_munu = (i/2)[g_mu, g_nu].
 *   Wilson-clover  M = A - kappa D.
 *   Schur    Mhat = A_oo - kappa^2 D_oe A_ee^-1 D_eo on odd sites.
 *   overlap  D_W(m) = (4 + m) - D/2, H_W = g5 D_W(-rho),
 *            D_ov(m) = (1 - m/(2 rho)) rho (1 + g5 eps(H_W)) + m.
 *
 * Memory: complex numbers are C99 double complex; spinor fields are
 * [site][spin 4][colour 3], links [site][mu 4][row 3][col 3], clover
 * matrices [site][12][12] with index 3*spin + colour.
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

/* ------------------------------------------------------------------ */
/* Lattice geometry                                                    */
/* ------------------------------------------------------------------ */

static long volume_of(const int L[4]) { return (long)L[0] * L[1] * L[2] * L[3]; }

static void coords_of(const int L[4], long s, int x[4]) {
  for (int mu = 0; mu < 4; mu++) {
    x[mu] = (int)(s % L[mu]);
    s /= L[mu];
  }
}

static long index_of(const int L[4], const int x[4]) {
  return x[0] + (long)L[0] * (x[1] + (long)L[1] * (x[2] + (long)L[2] * x[3]));
}

static int parity_of(const int L[4], long s) {
  int x[4];
  coords_of(L, s, x);
  return (x[0] + x[1] + x[2] + x[3]) & 1;
}

/* Site x + dir*mu (dir = +1 or -1), with the boundary sign of the hop. */
static long hop_to(const int L[4], int tbc, long s, int mu, int dir, double *sign) {
  int x[4];
  coords_of(L, s, x);
  int y = x[mu] + dir;
  *sign = 1.0;
  if (y == L[mu]) {
    y = 0;
    if (mu == 3 && tbc) *sign = -1.0;
  } else if (y < 0) {
    y = L[mu] - 1;
    if (mu == 3 && tbc) *sign = -1.0;
  }
  x[mu] = y;
  return index_of(L, x);
}

/* Link (row r, column c) of U_mu at site s. */
static inline cplx link_elem(const cplx *U, long s, int mu, int r, int c) {
  return U[((s * 4 + mu) * 3 + r) * 3 + c];
}

/* ------------------------------------------------------------------ */
/* Gamma matrices (DeGrand-Rossi chiral basis)                         */
/* ------------------------------------------------------------------ */

static cplx G[5][4][4];
static int gamma_ready = 0;

static void init_gammas(void) {
  if (gamma_ready) return;
  memset(G, 0, sizeof(G));
  /* gamma_0 */
  G[0][0][3] = I;  G[0][1][2] = I;  G[0][2][1] = -I; G[0][3][0] = -I;
  /* gamma_1 */
  G[1][0][3] = -1; G[1][1][2] = 1;  G[1][2][1] = 1;  G[1][3][0] = -1;
  /* gamma_2 */
  G[2][0][2] = I;  G[2][1][3] = -I; G[2][2][0] = -I; G[2][3][1] = I;
  /* gamma_3 */
  G[3][0][2] = 1;  G[3][1][3] = 1;  G[3][2][0] = 1;  G[3][3][1] = 1;
  /* gamma_5 = g0 g1 g2 g3 */
  cplx t1[4][4], t2[4][4];
  for (int a = 0; a < 4; a++)
    for (int b = 0; b < 4; b++) {
      cplx s = 0;
      for (int k = 0; k < 4; k++) s += G[0][a][k] * G[1][k][b];
      t1[a][b] = s;
    }
  for (int a = 0; a < 4; a++)
    for (int b = 0; b < 4; b++) {
      cplx s = 0;
      for (int k = 0; k < 4; k++) s += t1[a][k] * G[2][k][b];
      t2[a][b] = s;
    }
  for (int a = 0; a < 4; a++)
    for (int b = 0; b < 4; b++) {
      cplx s = 0;
      for (int k = 0; k < 4; k++) s += t2[a][k] * G[3][k][b];
      G[4][a][b] = s;
    }
  gamma_ready = 1;
}

/* Export gamma_mu (mu = 0..3) or gamma_5 (mu = 4) as 16 complex numbers. */
void or_gamma(int mu, cplx *out16) {
  init_gammas();
  for (int a = 0; a < 4; a++)
    for (int b = 0; b < 4; b++) out16[4 * a + b] = G[mu][a][b];
}

/* ------------------------------------------------------------------ */
/* Hopping term                                                        */
/* ------------------------------------------------------------------ */

/* (D psi)(s), or its adjoint: D^dag is the same hop with (1 -/+ g_mu)
 * exchanged, since (D^dag)(x,y) = D(y,x)^dag and g_mu is Hermitian. */
static void hop_site(const int L[4], int tbc, const cplx *U, const cplx *in, long s, int dagger,
                     cplx out[4][3]) {
  memset(out, 0, sizeof(cplx) * 12);
  double fwd = dagger ? +1.0 : -1.0; /* forward projector 1 + fwd*g_mu */
  for (int mu = 0; mu < 4; mu++) {
    for (int dir = +1; dir >= -1; dir -= 2) {
      double sign;
      long n = hop_to(L, tbc, s, mu, dir, &sign);
      const cplx *psi = in + 12 * n;
      cplx upsi[4][3];
      for (int a = 0; a < 4; a++)
        for (int r = 0; r < 3; r++) {
          cplx acc = 0;
          for (int c = 0; c < 3; c++) {
            cplx u = (dir > 0) ? link_elem(U, s, mu, r, c) : conj(link_elem(U, n, mu, c, r));
            acc += u * psi[3 * a + c];
          }
          upsi[a][r] = acc;
        }
      double g = (dir > 0) ? fwd : -fwd;
      for (int a = 0; a < 4; a++)
        for (int r = 0; r < 3; r++) {
          cplx acc = upsi[a][r];
          for (int b = 0; b < 4; b++) acc += g * G[mu][a][b] * upsi[b][r];
          out[a][r] += sign * acc;
        }
    }
  }
}

void or_hop(const int L[4], int tbc, const cplx *U, const cplx *in, cplx *out, int dagger) {
  init_gammas();
  long V = volume_of(L);
#pragma omp parallel for schedule(static)
  for (long s = 0; s < V; s++) hop_site(L, tbc, U, in, s, dagger, (cplx(*)[3])(out + 12 * s));
}

/* D psi at the listed sites only: out[k] = (D psi)(sites[k]), 12 complex each. */
void or_hop_sites(const int L[4], int tbc, const cplx *U, const cplx *in, const long *sites, long n,
                  cplx *out, int dagger) {
  init_gammas();
#pragma omp parallel for schedule(static)
  for (long k = 0; k < n; k++) hop_site(L, tbc, U, in, sites[k], dagger, (cplx(*)[3])(out + 12 * k));
}

/* ------------------------------------------------------------------ */
/* Clover term                                                         */
/* ------------------------------------------------------------------ */

typedef struct { cplx m[3][3]; } mat3;

static mat3 getU(const cplx *U, long s, int mu) {
  mat3 r;
  for (int i = 0; i < 3; i++)
    for (int j = 0; j < 3; j++) r.m[i][j] = link_elem(U, s, mu, i, j);
  return r;
}

static mat3 mul3(mat3 a, mat3 b) {
  mat3 c;
  for (int i = 0; i < 3; i++)
    for (int j = 0; j < 3; j++) {
      cplx s = 0;
      for (int k = 0; k < 3; k++) s += a.m[i][k] * b.m[k][j];
      c.m[i][j] = s;
    }
  return c;
}

static mat3 dag3(mat3 a) {
  mat3 c;
  for (int i = 0; i < 3; i++)
    for (int j = 0; j < 3; j++) c.m[i][j] = conj(a.m[j][i]);
  return c;
}

static long shift(const int L[4], long s, int mu, int dir) {
  double sign;
  return hop_to(L, 0, s, mu, dir, &sign); /* plaquettes use bare periodic links */
}

/* Sum of the four plaquette leaves Q_munu(x) of the clover. */
static mat3 clover_leaf_sum(const int L[4], const cplx *U, long s, int mu, int nu) {
  long xpm = shift(L, s, mu, +1), xpn = shift(L, s, nu, +1);
  long xmm = shift(L, s, mu, -1), xmn = shift(L, s, nu, -1);
  long xmm_pn = shift(L, xmm, nu, +1);
  long xmm_mn = shift(L, xmm, nu, -1);
  long xmn_pm = shift(L, xmn, mu, +1);
  mat3 q1 = mul3(mul3(getU(U, s, mu), getU(U, xpm, nu)), mul3(dag3(getU(U, xpn, mu)), dag3(getU(U, s, nu))));
  mat3 q2 = mul3(mul3(getU(U, s, nu), dag3(getU(U, xmm_pn, mu))), mul3(dag3(getU(U, xmm, nu)), getU(U, xmm, mu)));
  mat3 q3 = mul3(mul3(dag3(getU(U, xmm, mu)), dag3(getU(U, xmm_mn, nu))), mul3(getU(U, xmm_mn, mu), getU(U, xmn, nu)));
  mat3 q4 = mul3(mul3(dag3(getU(U, xmn, nu)), getU(U, xmn, mu)), mul3(getU(U, xmn_pm, nu), dag3(getU(U, s, mu))));
  mat3 q;
  for (int i = 0; i < 3; i++)
    for (int j = 0; j < 3; j++) q.m[i][j] = q1.m[i][j] + q2.m[i][j] + q3.m[i][j] + q4.m[i][j];
  return q;
}

/* F_munu(x) = (Q - Q^dag)/(8i), traceless part; written as 9 complex. */
static mat3 field_strength(const int L[4], const cplx *U, long s, int mu, int nu) {
  mat3 q = clover_leaf_sum(L, U, s, mu, nu), f;
  for (int i = 0; i < 3; i++)
    for (int j = 0; j < 3; j++) f.m[i][j] = (q.m[i][j] - conj(q.m[j][i])) / (8.0 * I);
  cplx tr = (f.m[0][0] + f.m[1][1] + f.m[2][2]) / 3.0;
  for (int i = 0; i < 3; i++) f.m[i][i] -= tr;
  return f;
}

void or_field_strength(const int L[4], const cplx *U, long s, int mu, int nu, cplx *out9) {
  mat3 f = field_strength(L, U, s, mu, nu);
  for (int i = 0; i < 3; i++)
    for (int j = 0; j < 3; j++) out9[3 * i + j] = f.m[i][j];
}

/* The full 12x12 clover matrix A(x) = 1 - csw*kappa*sum_{mu<nu} sigma_munu (x) F_munu. */
static void clover_site(const int L[4], const cplx *U, double kappa, double csw, long s, cplx *A) {
  memset(A, 0, sizeof(cplx) * 144);
  for (int i = 0; i < 12; i++) A[13 * i] = 1.0;
  if (csw == 0.0) return;
  for (int mu = 0; mu < 4; mu++)
    for (int nu = mu + 1; nu < 4; nu++) {
      mat3 f = field_strength(L, U, s, mu, nu);
      cplx sig[4][4];
      for (int a = 0; a < 4; a++)
        for (int b = 0; b < 4; b++) {
          cplx comm = 0;
          for (int k = 0; k < 4; k++) comm += G[mu][a][k] * G[nu][k][b] - G[nu][a][k] * G[mu][k][b];
          sig[a][b] = 0.5 * I * comm;
        }
      for (int a = 0; a < 4; a++)
        for (int b = 0; b < 4; b++)
          for (int i = 0; i < 3; i++)
            for (int j = 0; j < 3; j++) A[(3 * a + i) * 12 + 3 * b + j] -= csw * kappa * sig[a][b] * f.m[i][j];
    }
}

void or_clover(const int L[4], const cplx *U, double kappa, double csw, cplx *A) {
  init_gammas();
  long V = volume_of(L);
#pragma omp parallel for schedule(static)
  for (long s = 0; s < V; s++) clover_site(L, U, kappa, csw, s, A + 144 * s);
}

void or_clover_sites(const int L[4], const cplx *U, double kappa, double csw, const long *sites, long n,
                     cplx *A) {
  init_gammas();
#pragma omp parallel for schedule(static)
  for (long k = 0; k < n; k++) clover_site(L, U, kappa, csw, sites[k], A + 144 * k);
}

/* Gauss-Jordan inverse of an n x n complex matrix with partial pivoting.
 * Returns 0 on success, -1 if a pivot is exactly zero. */
int or_inverse(int n, const cplx *M, cplx *Minv) {
  cplx *a = malloc(sizeof(cplx) * n * 2 * n);
  for (int i = 0; i < n; i++)
    for (int j = 0; j < 2 * n; j++) a[i * 2 * n + j] = (j < n) ? M[i * n + j] : (j - n == i ? 1.0 : 0.0);
  int rc = 0;
  for (int c = 0; c < n; c++) {
    int p = c;
    for (int r = c + 1; r < n; r++)
      if (cabs(a[r * 2 * n + c]) > cabs(a[p * 2 * n + c])) p = r;
    if (a[p * 2 * n + c] == 0) { rc = -1; break; }
    if (p != c)
      for (int j = 0; j < 2 * n; j++) {
        cplx t = a[c * 2 * n + j];
        a[c * 2 * n + j] = a[p * 2 * n + j];
        a[p * 2 * n + j] = t;
      }
    cplx piv = a[c * 2 * n + c];
    for (int j = 0; j < 2 * n; j++) a[c * 2 * n + j] /= piv;
    for (int r = 0; r < n; r++) {
      if (r == c) continue;
      cplx f = a[r * 2 * n + c];
      if (f == 0) continue;
      for (int j = 0; j < 2 * n; j++) a[r * 2 * n + j] -= f * a[c * 2 * n + j];
    }
  }
  for (int i = 0; i < n; i++)
    for (int j = 0; j < n; j++) Minv[i * n + j] = a[i * 2 * n + n + j];
  free(a);
  return rc;
}

int or_clover_inverse(long V, const cplx *A, cplx *Ainv) {
  int bad = 0;
#pragma omp parallel for schedule(static) reduction(| : bad)
  for (long s = 0; s < V; s++) bad |= (or_inverse(12, A + 144 * s, Ainv + 144 * s) != 0);
  return bad ? -1 : 0;
}

/* ------------------------------------------------------------------ */
/* Wilson-clover operator and its even-odd Schur complement            */
/* ------------------------------------------------------------------ */

static void site_matvec(const cplx *A, const cplx *in, cplx *out) {
  for (int i = 0; i < 12; i++) {
    cplx acc = 0;
    for (int j = 0; j < 12; j++) acc += A[12 * i + j] * in[j];
    out[i] = acc;
  }
}

/* out = Amat(x) in(x) at every site (Amat = NULL means identity). */
void or_site_mul(long V, const cplx *Amat, const cplx *in, cplx *out) {
#pragma omp parallel for schedule(static)
  for (long s = 0; s < V; s++) {
    if (Amat)
      site_matvec(Amat + 144 * s, in + 12 * s, out + 12 * s);
    else
      memcpy(out + 12 * s, in + 12 * s, sizeof(cplx) * 12);
  }
}

/* Zero every site whose parity is not p. */
void or_keep_parity(const int L[4], int p, cplx *v) {
  long V = volume_of(L);
#pragma omp parallel for schedule(static)
  for (long s = 0; s < V; s++)
    if (parity_of(L, s) != p) memset(v + 12 * s, 0, sizeof(cplx) * 12);
}

/* out = M in = A in - kappa D in (full lattice; A = NULL means c_sw = 0). */
void or_apply_M(const int L[4], int tbc, const cplx *U, const cplx *A, double kappa, const cplx *in, cplx *out,
                int dagger) {
  long V = volume_of(L);
  cplx *d = malloc(sizeof(cplx) * 12 * V);
  or_hop(L, tbc, U, in, d, dagger);
  or_site_mul(V, A, in, out);
  for (long i = 0; i < 12 * V; i++) out[i] -= kappa * d[i];
  free(d);
}

/* out_o = Mhat in_o = A_oo in_o - kappa^2 D_oe A_ee^-1 D_eo in_o, or its
 * adjoint A_oo in_o - kappa^2 D_eo^dag A_ee^-1 D_oe^dag in_o (A Hermitian).
 * in and out are full-lattice fields; in must be zero on even sites and out
 * is zero on even sites. */
void or_apply_Mhat(const int L[4], int tbc, const cplx *U, const cplx *A, const cplx *Ainv, double kappa,
                   const cplx *in, cplx *out, int dagger) {
  long V = volume_of(L);
  cplx *t = malloc(sizeof(cplx) * 12 * V);
  cplx *u = malloc(sizeof(cplx) * 12 * V);
  or_hop(L, tbc, U, in, t, dagger);
  or_keep_parity(L, 0, t);
  or_site_mul(V, Ainv, t, u);
  or_hop(L, tbc, U, u, t, dagger);
  or_keep_parity(L, 1, t);
  or_site_mul(V, A, in, out);
  for (long i = 0; i < 12 * V; i++) out[i] -= kappa * kappa * t[i];
  or_keep_parity(L, 1, out);
  free(t);
  free(u);
}

/* The symmetric even-odd Schur complement, defined as A_oo^-1 Mhat:
 * out_o = A_oo^-1 Mhat in_o (= in_o - kappa^2 A_oo^-1 D_oe A_ee^-1 D_eo in_o),
 * or its adjoint Mhat^dag A_oo^-1 in_o (A^-1 is Hermitian).  Same field
 * conventions as or_apply_Mhat. */
void or_apply_Mhat_sym(const int L[4], int tbc, const cplx *U, const cplx *A, const cplx *Ainv, double kappa,
                       const cplx *in, cplx *out, int dagger) {
  long V = volume_of(L);
  cplx *t = malloc(sizeof(cplx) * 12 * V);
  if (!dagger) {
    or_apply_Mhat(L, tbc, U, A, Ainv, kappa, in, t, 0);
    or_site_mul(V, Ainv, t, out);
  } else {
    or_site_mul(V, Ainv, in, t);
    or_keep_parity(L, 1, t);
    or_apply_Mhat(L, tbc, U, A, Ainv, kappa, t, out, 1);
  }
  or_keep_parity(L, 1, out);
  free(t);
}

/* Even-odd source: bhat_o = b_o + kappa D_oe A_ee^-1 b_e (odd sites of out). */
void or_prepare_source(const int L[4], int tbc, const cplx *U, const cplx *Ainv, double kappa, const cplx *b,
                       cplx *bhat) {
  long V = volume_of(L);
  cplx *be = malloc(sizeof(cplx) * 12 * V);
  cplx *t = malloc(sizeof(cplx) * 12 * V);
  memcpy(be, b, sizeof(cplx) * 12 * V);
  or_keep_parity(L, 0, be);
  or_site_mul(V, Ainv, be, t);
  or_hop(L, tbc, U, t, be, 0);
  for (long i = 0; i < 12 * V; i++) bhat[i] = b[i] + kappa * be[i];
  or_keep_parity(L, 1, bhat);
  free(be);
  free(t);
}

/* Even-odd reconstruction: x_e = A_ee^-1 (b_e + kappa D_eo x_o); x holds x_o
 * on odd sites on entry and the full solution on exit. */
void or_reconstruct(const int L[4], int tbc, const cplx *U, const cplx *Ainv, double kappa, const cplx *b,
                    cplx *x) {
  long V = volume_of(L);
  cplx *t = malloc(sizeof(cplx) * 12 * V);
  cplx *u = malloc(sizeof(cplx) * 12 * V);
  or_keep_parity(L, 1, x);
  or_hop(L, tbc, U, x, t, 0);
  for (long i = 0; i < 12 * V; i++) t[i] = b[i] + kappa * t[i];
  or_keep_parity(L, 0, t);
  or_site_mul(V, Ainv, t, u);
  for (long s = 0; s < V; s++)
    if (parity_of(L, s) == 0) memcpy(x + 12 * s, u + 12 * s, sizeof(cplx) * 12);
  free(t);
  free(u);
}

/* Mhat x at the odd sites with t0 <= t < t1 only (0 <= t0 < t1 <= L3),
 * written into out at those sites; other sites of out are left untouched.
 * The even-site intermediate y = A_ee^-1 D_eo x is formed only on the time
 * slices t0-1 .. t1 that those sites reach.  A, Ainv: [V][12][12]. */
void or_mhat_slab(const int L[4], int tbc, const cplx *U, const cplx *A, const cplx *Ainv, double kappa,
                  const cplx *x, int t0, int t1, cplx *out) {
  init_gammas();
  long V = volume_of(L), slice = (long)L[0] * L[1] * L[2];
  cplx *y = calloc(12 * V, sizeof(cplx));
  int nt = t1 - t0 + 2 > L[3] ? L[3] : t1 - t0 + 2;
  for (int k = 0; k < nt; k++) {
    int t = ((t0 - 1 + k) % L[3] + L[3]) % L[3];
#pragma omp parallel for schedule(static)
    for (long i = 0; i < slice; i++) {
      long s = t * slice + i;
      if (parity_of(L, s) != 0) continue;
      cplx d[4][3];
      hop_site(L, tbc, U, x, s, 0, d);
      if (Ainv)
        site_matvec(Ainv + 144 * s, &d[0][0], y + 12 * s);
      else
        memcpy(y + 12 * s, &d[0][0], sizeof(cplx) * 12);
    }
  }
  for (int t = t0; t < t1; t++) {
#pragma omp parallel for schedule(static)
    for (long i = 0; i < slice; i++) {
      long s = t * slice + i;
      if (parity_of(L, s) != 1) continue;
      cplx d[4][3], ax[12];
      hop_site(L, tbc, U, y, s, 0, d);
      if (A)
        site_matvec(A + 144 * s, x + 12 * s, ax);
      else
        memcpy(ax, x + 12 * s, sizeof(cplx) * 12);
      for (int j = 0; j < 12; j++) out[12 * s + j] = ax[j] - kappa * kappa * (&d[0][0])[j];
    }
  }
  free(y);
}

/* ------------------------------------------------------------------ */
/* Vector algebra (sequential, fixed order)                             */
/* ------------------------------------------------------------------ */

double or_norm2(long n, const cplx *v) {
  double s = 0;
  for (long i = 0; i < n; i++) s += creal(v[i]) * creal(v[i]) + cimag(v[i]) * cimag(v[i]);
  return s;
}

cplx or_dot(long n, const cplx *a, const cplx *b) {
  cplx s = 0;
  for (long i = 0; i < n; i++) s += conj(a[i]) * b[i];
  return s;
}

/* ||b - M x|| / ||b|| over the full lattice. */
double or_true_residual(const int L[4], int tbc, const cplx *U, const cplx *A, double kappa, const cplx *x,
                        const cplx *b) {
  long V = volume_of(L);
  cplx *mx = malloc(sizeof(cplx) * 12 * V);
  or_apply_M(L, tbc, U, A, kappa, x, mx, 0);
  for (long i = 0; i < 12 * V; i++) mx[i] = b[i] - mx[i];
  double r = sqrt(or_norm2(12 * V, mx) / or_norm2(12 * V, b));
  free(mx);
  return r;
}

/* ------------------------------------------------------------------ */
/* CG on the normal equations (CGLS form) for Mhat x = bhat             */
/* ------------------------------------------------------------------ */

/* Solves Mhat x_o = bhat_o; x holds the initial guess on entry.  Stops when
 * ||r|| <= tol ||bhat|| with r recomputed as bhat - Mhat x.  Returns the
 * iteration count, or -1 without convergence in max_iter. */
int or_cgls(const int L[4], int tbc, const cplx *U, const cplx *A, const cplx *Ainv, double kappa, const cplx *bhat,
            cplx *x, double tol, int max_iter, double *resid_out) {
  long V = volume_of(L), n = 12 * V;
  cplx *r = malloc(sizeof(cplx) * n), *s = malloc(sizeof(cplx) * n), *p = malloc(sizeof(cplx) * n),
       *q = malloc(sizeof(cplx) * n);
  double bnorm = sqrt(or_norm2(n, bhat));
  or_apply_Mhat(L, tbc, U, A, Ainv, kappa, x, q, 0);
  for (long i = 0; i < n; i++) r[i] = bhat[i] - q[i];
  or_apply_Mhat(L, tbc, U, A, Ainv, kappa, r, s, 1);
  memcpy(p, s, sizeof(cplx) * n);
  double gamma = or_norm2(n, s);
  int k, done = 0;
  double rn = sqrt(or_norm2(n, r));
  for (k = 0; k < max_iter && !done; k++) {
    if (rn <= tol * bnorm) { done = 1; break; }
    or_apply_Mhat(L, tbc, U, A, Ainv, kappa, p, q, 0);
    double alpha = gamma / or_norm2(n, q);
    for (long i = 0; i < n; i++) {
      x[i] += alpha * p[i];
      r[i] -= alpha * q[i];
    }
    rn = sqrt(or_norm2(n, r));
    if (rn <= tol * bnorm) {
      or_apply_Mhat(L, tbc, U, A, Ainv, kappa, x, q, 0);
      for (long i = 0; i < n; i++) r[i] = bhat[i] - q[i];
      rn = sqrt(or_norm2(n, r));
      if (rn <= tol * bnorm) { done = 1; k++; break; }
    }
    or_apply_Mhat(L, tbc, U, A, Ainv, kappa, r, s, 1);
    double gnew = or_norm2(n, s);
    double beta = gnew / gamma;
    for (long i = 0; i < n; i++) p[i] = s[i] + beta * p[i];
    gamma = gnew;
  }
  if (resid_out) *resid_out = rn / bnorm;
  free(r); free(s); free(p); free(q);
  return done ? k : -1;
}

/* Full Wilson-clover solve M x = b by the even-odd route: source
 * preparation, CGLS on Mhat, reconstruction.  Returns CGLS's count. */
int or_solve(const int L[4], int tbc, const cplx *U, const cplx *A, const cplx *Ainv, double kappa, const cplx *b,
             cplx *x, double tol, int max_iter, double *resid_out) {
  long V = volume_of(L);
  cplx *bhat = malloc(sizeof(cplx) * 12 * V);
  or_prepare_source(L, tbc, U, Ainv, kappa, b, bhat);
  memset(x, 0, sizeof(cplx) * 12 * V);
  int it = or_cgls(L, tbc, U, A, Ainv, kappa, bhat, x, tol, max_iter, resid_out);
  or_reconstruct(L, tbc, U, Ainv, kappa, b, x);
  free(bhat);
  return it;
}

/* ------------------------------------------------------------------ */
/* Overlap: Wilson kernel, Chebyshev sign function, overlap operator    */
/* ------------------------------------------------------------------ */

/* out = D_W(m) in = (4 + m) in - D in / 2 on the full lattice. */
void or_apply_DW(const int L[4], int tbc, const cplx *U, double m, const cplx *in, cplx *out) {
  long V = volume_of(L);
  or_hop(L, tbc, U, in, out, 0);
  for (long i = 0; i < 12 * V; i++) out[i] = (4.0 + m) * in[i] - 0.5 * out[i];
}

void or_apply_gamma5(long V, const cplx *in, cplx *out) {
  for (long s = 0; s < V; s++)
    for (int a = 0; a < 4; a++)
      for (int c = 0; c < 3; c++) out[12 * s + 3 * a + c] = (a < 2 ? 1.0 : -1.0) * in[12 * s + 3 * a + c];
}

/* out = H_W in = gamma5 D_W(-rho) in. */
void or_apply_HW(const int L[4], int tbc, const cplx *U, double rho, const cplx *in, cplx *out) {
  long V = volume_of(L);
  cplx *t = malloc(sizeof(cplx) * 12 * V);
  or_apply_DW(L, tbc, U, -rho, in, t);
  or_apply_gamma5(V, t, out);
  free(t);
}

/* Chebyshev interpolant of f(y) = 1/sqrt(y) on [a, b] of degree n:
 * P(y) = sum_{k=0}^{n} c[k] T_k(t), t = (2y - a - b)/(b - a), from the
 * n+1 Chebyshev-Gauss nodes; c[0] already carries its factor 1/2. */
void or_cheb_coeffs(double a, double b, int n, double *c) {
  int N = n + 1;
  for (int k = 0; k <= n; k++) {
    double s = 0;
    for (int j = 0; j < N; j++) {
      double th = M_PI * (j + 0.5) / N;
      double y = 0.5 * ((b - a) * cos(th) + a + b);
      s += cos(k * th) / sqrt(y);
    }
    c[k] = 2.0 * s / N;
  }
  c[0] *= 0.5;
}

/* Scalar evaluation of the series by the Clenshaw recurrence. */
double or_cheb_eval(double a, double b, int n, const double *c, double y) {
  double t = (2.0 * y - a - b) / (b - a), b1 = 0, b2 = 0;
  for (int k = n; k >= 1; k--) {
    double b0 = c[k] + 2.0 * t * b1 - b2;
    b2 = b1;
    b1 = b0;
  }
  return c[0] + t * b1 - b2;
}

/* max |x P(x^2) - sign(x)| over x in [sqrt(a), sqrt(b)]: npts uniform
 * points in x plus the interpolation nodes (sign is odd, so x > 0 suffices). */
double or_sign_error(double a, double b, int n, const double *c, int npts) {
  double worst = 0, lo = sqrt(a), hi = sqrt(b);
  for (int i = 0; i < npts; i++) {
    double x = lo + (hi - lo) * i / (npts - 1);
    double e = fabs(x * or_cheb_eval(a, b, n, c, x * x) - 1.0);
    if (e > worst) worst = e;
  }
  for (int j = 0; j <= n; j++) {
    double y = 0.5 * ((b - a) * cos(M_PI * (j + 0.5) / (n + 1)) + a + b);
    double e = fabs(sqrt(y) * or_cheb_eval(a, b, n, c, y) - 1.0);
    if (e > worst) worst = e;
  }
  return worst;
}

/* Smallest degree n <= nmax whose sign error is <= tol (coefficients in c,
 * which must hold nmax+1 values); -1 if none. */
int or_cheb_degree(double a, double b, double tol, int nmax, int npts, double *c) {
  for (int n = 1; n <= nmax; n++) {
    or_cheb_coeffs(a, b, n, c);
    if (or_sign_error(a, b, n, c, npts) <= tol) return n;
  }
  return -1;
}

/* eps(H_W) in, with the k listed eigenpairs (lam[i], vecs[i]) of H_W treated
 * exactly and the rest by H_W P(H_W^2):
 *   eps v = sum_i sign(lam_i) v_i <v_i, v> + H P(H^2) (v - sum_i v_i <v_i, v>). */
void or_apply_sign(const int L[4], int tbc, const cplx *U, double rho, int nlow, const double *lam,
                   const cplx *vecs, double a, double b, int n, const double *c, const cplx *in, cplx *out) {
  long V = volume_of(L), N = 12 * V;
  cplx *w = malloc(sizeof(cplx) * N), *b1 = calloc(N, sizeof(cplx)), *b2 = calloc(N, sizeof(cplx)),
       *b0 = malloc(sizeof(cplx) * N), *h = malloc(sizeof(cplx) * N), *hh = malloc(sizeof(cplx) * N);
  memcpy(w, in, sizeof(cplx) * N);
  cplx *proj = malloc(sizeof(cplx) * (nlow > 0 ? nlow : 1));
  for (int i = 0; i < nlow; i++) {
    proj[i] = or_dot(N, vecs + (long)i * N, in);
    for (long j = 0; j < N; j++) w[j] -= proj[i] * vecs[(long)i * N + j];
  }
  /* Clenshaw with T = (2 H^2 - (a+b)) / (b - a) */
  double s2 = 2.0 / (b - a), s0 = -(a + b) / (b - a);
  for (int k = n; k >= 1; k--) {
    or_apply_HW(L, tbc, U, rho, b1, h);
    or_apply_HW(L, tbc, U, rho, h, hh);
    for (long j = 0; j < N; j++) b0[j] = c[k] * w[j] + 2.0 * (s2 * hh[j] + s0 * b1[j]) - b2[j];
    cplx *t = b2; b2 = b1; b1 = b0; b0 = t;
  }
  or_apply_HW(L, tbc, U, rho, b1, h);
  or_apply_HW(L, tbc, U, rho, h, hh);
  for (long j = 0; j < N; j++) b0[j] = c[0] * w[j] + (s2 * hh[j] + s0 * b1[j]) - b2[j];
  or_apply_HW(L, tbc, U, rho, b0, out);
  for (int i = 0; i < nlow; i++) {
    double sg = lam[i] > 0 ? 1.0 : -1.0;
    for (long j = 0; j < N; j++) out[j] += sg * proj[i] * vecs[(long)i * N + j];
  }
  free(w); free(b1); free(b2); free(b0); free(h); free(hh); free(proj);
}

/* D_ov(m) in = (1 - m/(2 rho)) rho (in + g5 eps in) + m in. */
void or_apply_overlap(const int L[4], int tbc, const cplx *U, double rho, double m, int nlow, const double *lam,
                      const cplx *vecs, double a, double b, int n, const double *c, const cplx *in, cplx *out,
                      int dagger) {
  long V = volume_of(L), N = 12 * V;
  cplx *e = malloc(sizeof(cplx) * N), *g = malloc(sizeof(cplx) * N);
  double f = (1.0 - m / (2.0 * rho)) * rho;
  if (!dagger) {
    or_apply_sign(L, tbc, U, rho, nlow, lam, vecs, a, b, n, c, in, e);
    or_apply_gamma5(V, e, g);
    for (long j = 0; j < N; j++) out[j] = f * (in[j] + g[j]) + m * in[j];
  } else {
    /* D_ov^dag = f (1 + eps g5) + m, since eps is Hermitian */
    or_apply_gamma5(V, in, g);
    or_apply_sign(L, tbc, U, rho, nlow, lam, vecs, a, b, n, c, g, e);
    for (long j = 0; j < N; j++) out[j] = f * (in[j] + e[j]) + m * in[j];
  }
  free(e); free(g);
}
