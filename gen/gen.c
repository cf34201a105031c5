/*
 * Seeded synthetic inputs for the Wilson-clover / overlap hot path.
 *
 * This module holds input generation only (random numbers, SU(3) link
 * matrices, Gaussian spinors); none of the operator arithmetic lives here.
 * Both the FP64 oracle and the CUDA library consume the arrays it writes.
 *
 * Random numbers: counter-based, so every value depends only on (seed,
 * counter) and never on thread count or call order.  The mixer is SplitMix64
 * (Steele, Lea, Flood, "Fast splittable pseudorandom number generators",
 * OOPSLA 2014), uniform doubles take its top 53 bits, and normals come from
 * the Box-Muller transform.
 *
 * Links: U = exp(i eps A) with A = sum_a c_a lambda_a / 2, c_a ~ N(0,1) and
 * lambda_a the eight Gell-Mann matrices; exp by scaling and squaring of a
 * truncated Taylor series, then reunitarised (Gram-Schmidt of rows 0 and 1,
 * row 2 = conj(row0 x row1), which also fixes det U = 1).
 *
 * Canonical layouts (complex numbers as interleaved re, im doubles):
 *   links  [t][z][y][x][mu 0..3][row 3][col 3]
 *   spinor [t][z][y][x][spin 4][colour 3]
 */
#include <math.h>
#include <stdint.h>
#include <string.h>

static inline uint64_t splitmix64(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

/* Uniform double in (0, 1]: value number `ctr` of the stream keyed by `seed`. */
static inline double uniform01(uint64_t seed, uint64_t ctr) {
  uint64_t r = splitmix64(splitmix64(seed) ^ (ctr * 0xD1B54A32D192ED03ULL));
  return ((double)((r >> 11) + 1)) * (1.0 / 9007199254740992.0);
}

/* Two independent N(0,1) values from counters 2*k and 2*k+1 (Box-Muller). */
static inline void normal_pair(uint64_t seed, uint64_t k, double *g0, double *g1) {
  const double two_pi = 6.283185307179586476925286766559;
  double u1 = uniform01(seed, 2 * k);
  double u2 = uniform01(seed, 2 * k + 1);
  double rad = sqrt(-2.0 * log(u1));
  *g0 = rad * cos(two_pi * u2);
  *g1 = rad * sin(two_pi * u2);
}

void gen_uniform(long n, uint64_t seed, double *out) {
#pragma omp parallel for schedule(static)
  for (long i = 0; i < n; i++) out[i] = uniform01(seed, (uint64_t)i);
}

void gen_gaussian(long n, uint64_t seed, double *out) {
#pragma omp parallel for schedule(static)
  for (long k = 0; k < (n + 1) / 2; k++) {
    double g0, g1;
    normal_pair(seed, (uint64_t)k, &g0, &g1);
    out[2 * k] = g0;
    if (2 * k + 1 < n) out[2 * k + 1] = g1;
  }
}

/* 3x3 complex matrices as 18 doubles, row-major, (re, im) interleaved. */
typedef struct { double re[9], im[9]; } cm3;

static void cm3_mul(const cm3 *a, const cm3 *b, cm3 *c) {
  for (int i = 0; i < 3; i++)
    for (int j = 0; j < 3; j++) {
      double sr = 0, si = 0;
      for (int k = 0; k < 3; k++) {
        sr += a->re[3 * i + k] * b->re[3 * k + j] - a->im[3 * i + k] * b->im[3 * k + j];
        si += a->re[3 * i + k] * b->im[3 * k + j] + a->im[3 * i + k] * b->re[3 * k + j];
      }
      c->re[3 * i + j] = sr;
      c->im[3 * i + j] = si;
    }
}

/* H = sum_a c_a lambda_a / 2 (Hermitian, traceless), Gell-Mann basis. */
static void hermitian_from_coeffs(const double c[8], cm3 *h) {
  memset(h, 0, sizeof(*h));
  const double inv_sqrt3 = 0.57735026918962576451;
  /* lambda_1: (0,1),(1,0) = 1 */
  h->re[1] += c[0]; h->re[3] += c[0];
  /* lambda_2: (0,1) = -i, (1,0) = +i */
  h->im[1] -= c[1]; h->im[3] += c[1];
  /* lambda_3: diag(1,-1,0) */
  h->re[0] += c[2]; h->re[4] -= c[2];
  /* lambda_4: (0,2),(2,0) = 1 */
  h->re[2] += c[3]; h->re[6] += c[3];
  /* lambda_5: (0,2) = -i, (2,0) = +i */
  h->im[2] -= c[4]; h->im[6] += c[4];
  /* lambda_6: (1,2),(2,1) = 1 */
  h->re[5] += c[5]; h->re[7] += c[5];
  /* lambda_7: (1,2) = -i, (2,1) = +i */
  h->im[5] -= c[6]; h->im[7] += c[6];
  /* lambda_8: diag(1,1,-2)/sqrt(3) */
  h->re[0] += c[7] * inv_sqrt3; h->re[4] += c[7] * inv_sqrt3; h->re[8] -= 2.0 * c[7] * inv_sqrt3;
  for (int i = 0; i < 9; i++) { h->re[i] *= 0.5; h->im[i] *= 0.5; }
}

/* exp(i eps H) by scaling and squaring with a degree-12 Taylor polynomial. */
static void expi(const cm3 *h, double eps, cm3 *u) {
  cm3 x; /* x = i eps H */
  double nrm = 0;
  for (int i = 0; i < 9; i++) {
    x.re[i] = -eps * h->im[i];
    x.im[i] = eps * h->re[i];
    nrm += x.re[i] * x.re[i] + x.im[i] * x.im[i];
  }
  nrm = sqrt(nrm);
  int s = 0;
  while (nrm > 0.125) { nrm *= 0.5; s++; }
  double f = ldexp(1.0, -s);
  for (int i = 0; i < 9; i++) { x.re[i] *= f; x.im[i] *= f; }
  /* Horner: u = 1 + x(1 + x/2(1 + x/3(...))) */
  cm3 acc, tmp;
  memset(&acc, 0, sizeof(acc));
  for (int i = 0; i < 3; i++) acc.re[4 * i] = 1.0;
  for (int k = 12; k >= 1; k--) {
    cm3_mul(&x, &acc, &tmp);
    for (int i = 0; i < 9; i++) { acc.re[i] = tmp.re[i] / k; acc.im[i] = tmp.im[i] / k; }
    for (int i = 0; i < 3; i++) acc.re[4 * i] += 1.0;
  }
  for (int q = 0; q < s; q++) {
    cm3_mul(&acc, &acc, &tmp);
    acc = tmp;
  }
  *u = acc;
}

/* Gram-Schmidt on rows 0, 1; row 2 = conj(row0 x row1). */
static void reunitarise(cm3 *u) {
  double n0 = 0;
  for (int j = 0; j < 3; j++) n0 += u->re[j] * u->re[j] + u->im[j] * u->im[j];
  n0 = 1.0 / sqrt(n0);
  for (int j = 0; j < 3; j++) { u->re[j] *= n0; u->im[j] *= n0; }
  double pr = 0, pi = 0; /* <row0, row1> = sum conj(r0) r1 */
  for (int j = 0; j < 3; j++) {
    pr += u->re[j] * u->re[3 + j] + u->im[j] * u->im[3 + j];
    pi += u->re[j] * u->im[3 + j] - u->im[j] * u->re[3 + j];
  }
  for (int j = 0; j < 3; j++) {
    u->re[3 + j] -= pr * u->re[j] - pi * u->im[j];
    u->im[3 + j] -= pr * u->im[j] + pi * u->re[j];
  }
  double n1 = 0;
  for (int j = 0; j < 3; j++) n1 += u->re[3 + j] * u->re[3 + j] + u->im[3 + j] * u->im[3 + j];
  n1 = 1.0 / sqrt(n1);
  for (int j = 0; j < 3; j++) { u->re[3 + j] *= n1; u->im[3 + j] *= n1; }
  for (int j = 0; j < 3; j++) {
    int a = (j + 1) % 3, b = (j + 2) % 3;
    /* (r0 x r1)_j = r0_a r1_b - r0_b r1_a, then conjugate */
    double cr = u->re[a] * u->re[3 + b] - u->im[a] * u->im[3 + b] - (u->re[b] * u->re[3 + a] - u->im[b] * u->im[3 + a]);
    double ci = u->re[a] * u->im[3 + b] + u->im[a] * u->re[3 + b] - (u->re[b] * u->im[3 + a] + u->im[b] * u->re[3 + a]);
    u->re[6 + j] = cr;
    u->im[6 + j] = -ci;
  }
}

/* nmat SU(3) matrices exp(i eps A_k), A_k from 8 normals at counters 4k..4k+3. */
void gen_su3(long nmat, double eps, uint64_t seed, double *out) {
#pragma omp parallel for schedule(static)
  for (long k = 0; k < nmat; k++) {
    double c[8];
    for (int p = 0; p < 4; p++) normal_pair(seed, 4 * (uint64_t)k + p, &c[2 * p], &c[2 * p + 1]);
    cm3 h, u;
    hermitian_from_coeffs(c, &h);
    expi(&h, eps, &u);
    reunitarise(&u);
    double *o = out + 18 * k;
    for (int i = 0; i < 9; i++) { o[2 * i] = u.re[i]; o[2 * i + 1] = u.im[i]; }
  }
}

/* The traceless Hermitian generator matrix of link k (for tests of the map). */
void gen_su3_generator(long k, uint64_t seed, double *out18) {
  double c[8];
  for (int p = 0; p < 4; p++) normal_pair(seed, 4 * (uint64_t)k + p, &c[2 * p], &c[2 * p + 1]);
  cm3 h;
  hermitian_from_coeffs(c, &h);
  for (int i = 0; i < 9; i++) { out18[2 * i] = h.re[i]; out18[2 * i + 1] = h.im[i]; }
}

/* Gauge field on an L0 x L1 x L2 x L3 lattice: 4 links per site, canonical order. */
void gen_gauge(const int L[4], double eps, uint64_t seed, double *U) {
  long V = (long)L[0] * L[1] * L[2] * L[3];
  gen_su3(4 * V, eps, seed, U);
}
