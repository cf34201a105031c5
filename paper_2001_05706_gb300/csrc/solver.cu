// Solver driver: even-odd preconditioned CG on the normal equations (CGLS
// form) for M x = b, in FP64 or in mixed precision with reliable updates.
//
// The paper's inverters (abstract; Sec. 4: "the multigrid inverter works
// correctly") rest on Krylov solves of the Wilson-clover operator; QUDA's
// mixed-precision CG with reliable updates is its reference [Clark:2009wm]
// (Sec. 1).  Per right-hand side the recursion is
//   r = bhat - Mhat x;  s = Mhat^dag r;  p = s;  gamma = |s|^2
//   repeat: q = Mhat p; alpha = gamma/|q|^2; x += alpha p; r -= alpha q;
//           s = Mhat^dag r; gamma' = |s|^2; p = s + (gamma'/gamma) p
// with every scalar kept in device memory (no host round trip inside an
// iteration); the host reads the residual norms every `check_every`
// iterations.  Mixed precision: r, p, q, s in FP32/FP16/BF16 storage and
// FP32 arithmetic, x_lo in FP32, normalised so the inner residual starts at
// norm 1; when it has fallen below delta (or reaches the target) the FP64
// solution absorbs x_lo and the residual is recomputed with the FP64
// operator; the search direction p is kept, rescaled into the new
// normalisation, and gamma = |Mhat^dag r|^2 recomputed from the new residual;
// an update that fails to reduce the residual restarts CG from p = s.
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "internal.h"

namespace lqcd {

namespace {

struct SolveBufs {
  SolverScalars *sc = nullptr;  // device [nrhs]
  double *fac = nullptr;        // device [3 nrhs] per-RHS factors
  SolverScalars *h_sc = nullptr;  // pinned mirrors
  double *h_fac = nullptr;
  ~SolveBufs() {
    if (sc) cudaFree(sc);
    if (fac) cudaFree(fac);
    if (h_sc) cudaFreeHost(h_sc);
    if (h_fac) cudaFreeHost(h_fac);
  }
};

const FieldRef kNone{nullptr, nullptr, 0};
// LQCD_SOLVER_TRACE=1 prints one line per reliable update to stderr
const bool kTrace = std::getenv("LQCD_SOLVER_TRACE") != nullptr;
constexpr int kScStride = (int)(sizeof(SolverScalars) / sizeof(double));

lqcd_status read_scalars(lqcd_ctx *c, SolveBufs &B, int nrhs) {
  LQ_CU(cudaMemcpyAsync(B.h_sc, B.sc, sizeof(SolverScalars) * nrhs, cudaMemcpyDeviceToHost, c->stream));
  LQ_CU(cudaStreamSynchronize(c->stream));
  return LQCD_OK;
}

lqcd_status write_scalars(lqcd_ctx *c, SolveBufs &B, int nrhs) {
  LQ_CU(cudaMemcpyAsync(B.sc, B.h_sc, sizeof(SolverScalars) * nrhs, cudaMemcpyHostToDevice, c->stream));
  return LQCD_OK;
}

lqcd_status write_fac(lqcd_ctx *c, SolveBufs &B, int nrhs) {
  LQ_CU(cudaMemcpyAsync(B.fac, B.h_fac, sizeof(double) * nrhs, cudaMemcpyHostToDevice, c->stream));
  return LQCD_OK;
}

// norms of nrhs parity fields into host array out (FP64 reduction on GPU)
lqcd_status norms(lqcd_ctx *c, lqcd_prec prec, int nrhs, FieldRef f, double *out) {
  LQ_TRY(ensure_partials(c, nrhs));
  LQ_CU(blas_norm2(prec, c->Vh, nrhs, f, c->partials, c->counter, c->results, 1, c->stream));
  LQ_CU(cudaMemcpyAsync(c->h_results, c->results, sizeof(double) * nrhs, cudaMemcpyDeviceToHost, c->stream));
  LQ_CU(cudaStreamSynchronize(c->stream));
  std::memcpy(out, c->h_results, sizeof(double) * nrhs);
  return LQCD_OK;
}

struct Work {
  lqcd_ctx *c;
  int nrhs;
  int recon64, recon_lo;
  lqcd_prec lo;
  double tol, delta;
  int max_iter, check_every;
  std::vector<double> bnorm;  // ||b|| full lattice per RHS
  lqcd_field *bhat, *x64, *r64;  // FP64: bhat_o, x (full), r_o
  lqcd_solve_info *info;
};

// FP64 CGLS: iterate until every RHS has ||r|| <= target, where r is
// recomputed as bhat - Mhat x before a right-hand side is accepted.
lqcd_status cgls_fp64(Work &W, SolveBufs &B) {
  lqcd_ctx *c = W.c;
  const int n = W.nrhs;
  const lqcd_prec P = LQCD_F64;
  lqcd_field *s, *p, *q, *ye;
  LQ_TRY(temp_field(c, P, LQCD_ODD, n, 20, &s));
  LQ_TRY(temp_field(c, P, LQCD_ODD, n, 21, &p));
  LQ_TRY(temp_field(c, P, LQCD_ODD, n, 22, &q));
  LQ_TRY(temp_field(c, P, LQCD_EVEN, n, 23, &ye));
  LQ_TRY(ensure_partials(c, n));
  std::vector<double> target2(n);
  for (int k = 0; k < n; k++) target2[k] = std::pow(0.5 * W.tol * W.bnorm[k], 2);
  // r = bhat - Mhat x ; s = Mhat^dag r ; p = s
  LQ_TRY(op_mhat(c, P, W.recon64, 0, n, W.r64->mut(1), W.x64->ref(1), ye->mut(0), W.bhat->ref(1), -1.0, &B.sc[0].rr,
                 kScStride));
  int cur = 0;
  LQ_TRY(op_mhat(c, P, W.recon64, 1, n, s->mut(1), W.r64->ref(1), ye->mut(0), kNone, 0.0, &B.sc[0].gamma[cur],
                 kScStride));
  LQ_CU(cudaMemcpyAsync(p->data[1], s->data[1], (size_t)p->rhs_words() * 16 * n, cudaMemcpyDeviceToDevice, c->stream));
  W.info->mhat_applies += 2;
  int it = 0;
  bool all_done = false;
  // host-side check at the start (the guess may already solve it)
  LQ_TRY(read_scalars(c, B, n));
  while (true) {
    all_done = true;
    bool changed = false;
    for (int k = 0; k < n; k++) {
      if (B.h_sc[k].active == 0.0) continue;
      const double rr = B.h_sc[k].rr;
      if (!(rr == rr)) return set_error(LQCD_ERR_NOCONV, "residual of RHS %d is NaN at iteration %d", k, it);
      if (rr <= target2[k]) {
        B.h_sc[k].active = 0.0;
        changed = true;
      } else {
        all_done = false;
      }
    }
    if (changed) LQ_TRY(write_scalars(c, B, n));
    if (all_done || it >= W.max_iter) break;
    for (int j = 0; j < W.check_every && it < W.max_iter; j++, it++) {
      LQ_TRY(op_mhat(c, P, W.recon64, 0, n, q->mut(1), p->ref(1), ye->mut(0), kNone, 0.0, &B.sc[0].qq, kScStride));
      LQ_CU(blas_cg_xr(P, P, c->Vh, n, W.x64->mut(1), p->ref(1), W.r64->mut(1), q->ref(1), B.sc, cur, c->partials,
                       c->counter, c->stream));
      LQ_TRY(op_mhat(c, P, W.recon64, 1, n, s->mut(1), W.r64->ref(1), ye->mut(0), kNone, 0.0, &B.sc[0].gamma[1 - cur],
                     kScStride));
      LQ_CU(blas_cg_p(P, c->Vh, n, p->mut(1), s->ref(1), B.sc, cur, c->stream));
      cur ^= 1;
      W.info->mhat_applies += 2;
    }
    LQ_TRY(read_scalars(c, B, n));
    // residual below target: recompute r = bhat - Mhat x before accepting it
    bool any = false;
    for (int k = 0; k < n; k++) any |= (B.h_sc[k].active != 0.0 && B.h_sc[k].rr <= target2[k]);
    if (any) {
      LQ_TRY(op_mhat(c, P, W.recon64, 0, n, W.r64->mut(1), W.x64->ref(1), ye->mut(0), W.bhat->ref(1), -1.0,
                     &B.sc[0].aux, kScStride));
      W.info->mhat_applies += 1;
      W.info->reliable_updates += 1;
      LQ_TRY(read_scalars(c, B, n));
      for (int k = 0; k < n; k++)
        if (B.h_sc[k].active != 0.0) B.h_sc[k].rr = B.h_sc[k].aux;
    }
  }
  W.info->iters = it;
  return all_done ? LQCD_OK : set_error(LQCD_ERR_NOCONV, "CG did not converge in %d iterations", W.max_iter);
}

lqcd_status cgls_mixed(Work &W, SolveBufs &B) {
  lqcd_ctx *c = W.c;
  const int n = W.nrhs;
  const lqcd_prec L = W.lo;
  lqcd_field *s, *p, *q, *ye, *r, *xlo, *ye64;
  LQ_TRY(temp_field(c, L, LQCD_ODD, n, 30, &s));
  LQ_TRY(temp_field(c, L, LQCD_ODD, n, 31, &p));
  LQ_TRY(temp_field(c, L, LQCD_ODD, n, 32, &q));
  LQ_TRY(temp_field(c, L, LQCD_EVEN, n, 33, &ye));
  LQ_TRY(temp_field(c, L, LQCD_ODD, n, 34, &r));
  LQ_TRY(temp_field(c, LQCD_F32, LQCD_ODD, n, 35, &xlo));
  LQ_TRY(temp_field(c, LQCD_F64, LQCD_EVEN, n, 23, &ye64));
  LQ_TRY(ensure_partials(c, n));
  std::vector<double> target(n), sigma(n), best_rr(n, 1.0);
  std::vector<int> stall(n, 0);
  for (int k = 0; k < n; k++) target[k] = 0.5 * W.tol * W.bnorm[k];
  const double delta2 = W.delta * W.delta;
  // an inner residual that has not halved over kStallChecks checks is
  // stagnating at the precision floor of the storage type: force an update
  constexpr int kStallChecks = 3;
  const size_t xlo_bytes = (size_t)xlo->rhs_words() * 16 * n;

  // r64 = bhat - Mhat64 x64 -> sigma
  LQ_TRY(op_mhat(c, LQCD_F64, W.recon64, 0, n, W.r64->mut(1), W.x64->ref(1), ye64->mut(0), W.bhat->ref(1), -1.0,
                 &B.sc[0].aux, kScStride));
  W.info->mhat_applies += 1;
  LQ_TRY(read_scalars(c, B, n));
  int nactive = 0;
  for (int k = 0; k < n; k++) {
    sigma[k] = std::sqrt(B.h_sc[k].aux);
    B.h_sc[k].active = sigma[k] > target[k] ? 1.0 : 0.0;
    nactive += B.h_sc[k].active != 0.0;
    B.h_fac[k] = sigma[k] > 0 ? 1.0 / sigma[k] : 0.0;
    B.h_sc[k].rr = 1.0;
  }
  if (nactive == 0) {
    W.info->iters = 0;
    return LQCD_OK;
  }
  LQ_TRY(write_scalars(c, B, n));
  LQ_TRY(write_fac(c, B, n));
  // r_lo = r64 / sigma ; x_lo = 0 ; s = Mhat^dag r ; p = s
  LQ_CU(blas_scale(L, LQCD_F64, c->Vh, n, r->mut(1), W.r64->ref(1), B.fac, c->stream));
  LQ_CU(cudaMemsetAsync(xlo->data[1], 0, xlo_bytes, c->stream));
  int cur = 0;
  LQ_TRY(op_mhat(c, L, W.recon_lo, 1, n, s->mut(1), r->ref(1), ye->mut(0), kNone, 0.0, &B.sc[0].gamma[cur], kScStride));
  LQ_CU(cudaMemcpyAsync(p->data[1], s->data[1], (size_t)p->rhs_words() * 16 * n, cudaMemcpyDeviceToDevice, c->stream));
  if (p->scale[1])
    LQ_CU(cudaMemcpyAsync(p->scale[1], s->scale[1], sizeof(float) * c->Vh * n, cudaMemcpyDeviceToDevice, c->stream));
  W.info->mhat_applies += 1;

  int it = 0;
  bool done = false;
  while (!done) {
    if (it >= W.max_iter) break;
    for (int j = 0; j < W.check_every && it < W.max_iter; j++, it++) {
      LQ_TRY(op_mhat(c, L, W.recon_lo, 0, n, q->mut(1), p->ref(1), ye->mut(0), kNone, 0.0, &B.sc[0].qq, kScStride));
      LQ_CU(blas_cg_xr(LQCD_F32, L, c->Vh, n, xlo->mut(1), p->ref(1), r->mut(1), q->ref(1), B.sc, cur, c->partials,
                       c->counter, c->stream));
      LQ_TRY(op_mhat(c, L, W.recon_lo, 1, n, s->mut(1), r->ref(1), ye->mut(0), kNone, 0.0, &B.sc[0].gamma[1 - cur],
                     kScStride));
      LQ_CU(blas_cg_p(L, c->Vh, n, p->mut(1), s->ref(1), B.sc, cur, c->stream));
      cur ^= 1;
      W.info->mhat_applies += 2;
    }
    LQ_TRY(read_scalars(c, B, n));
    // trigger: every active RHS dropped by delta, or one reached its target,
    // or one stagnates
    bool all_dropped = true, any_target = false, any_stall = false;
    for (int k = 0; k < n; k++) {
      if (B.h_sc[k].active == 0.0) continue;
      const double rr = B.h_sc[k].rr;
      if (!(rr == rr)) return set_error(LQCD_ERR_NOCONV, "inner residual of RHS %d is NaN at iteration %d", k, it);
      if (rr > delta2) all_dropped = false;
      if (sigma[k] * std::sqrt(rr) <= target[k]) any_target = true;
      if (rr < 0.25 * best_rr[k]) {
        best_rr[k] = rr;
        stall[k] = 0;
      } else if (++stall[k] >= kStallChecks) {
        any_stall = true;
      }
    }
    if (!(all_dropped || any_target || any_stall || it >= W.max_iter)) continue;

    // ---- reliable update: x64 += sigma x_lo ; r64 = bhat - Mhat64 x64
    for (int k = 0; k < n; k++) B.h_fac[k] = B.h_sc[k].active != 0.0 ? sigma[k] : 0.0;
    LQ_TRY(write_fac(c, B, n));
    LQ_CU(blas_axpy(LQCD_F64, LQCD_F32, c->Vh, n, W.x64->mut(1), xlo->ref(1), B.fac, c->stream));
    LQ_CU(cudaMemsetAsync(xlo->data[1], 0, xlo_bytes, c->stream));
    LQ_TRY(op_mhat(c, LQCD_F64, W.recon64, 0, n, W.r64->mut(1), W.x64->ref(1), ye64->mut(0), W.bhat->ref(1), -1.0,
                   &B.sc[0].aux, kScStride));
    W.info->mhat_applies += 1;
    W.info->reliable_updates += 1;
    LQ_TRY(read_scalars(c, B, n));
    done = true;
    for (int k = 0; k < n; k++) {
      if (B.h_sc[k].active == 0.0) {
        B.h_fac[k] = 0.0;
        continue;
      }
      const double snew = std::sqrt(B.h_sc[k].aux);
      if (kTrace)
        std::fprintf(stderr, "lqcd: update %d it %d rhs %d inner |r| %.3e  FP64 |r| %.6e -> %.6e (target %.3e)\n",
                     W.info->reliable_updates, it, k, std::sqrt(B.h_sc[k].rr), sigma[k], snew, target[k]);
      if (!(snew == snew) || std::isinf(snew))
        return set_error(LQCD_ERR_NOCONV, "FP64 residual of RHS %d is not finite", k);
      if (snew <= target[k]) {
        B.h_sc[k].active = 0.0;
        B.h_fac[k] = 0.0;
        continue;
      }
      done = false;
      // p (the next search direction) is kept, rescaled into the new
      // normalisation r_lo = r64 / snew, unless this update failed to reduce
      // the residual: then CG restarts from p = s (low-precision noise has
      // spoilt the conjugacy of p)
      const bool restart = snew >= sigma[k] || stall[k] >= kStallChecks;
      stall[k] = 0;
      best_rr[k] = 1.0;
      B.h_fac[k] = restart ? 0.0 : sigma[k] / snew;
      B.h_fac[2 * n + k] = restart ? 1.0 : 0.0;
      B.h_sc[k].rr = 1.0;
      sigma[k] = snew;
    }
    if (done) break;
    // factors: p *= fac[0, n); r = r64 * fac[n, 2n); p += fac[2n, 3n) s
    for (int k = 0; k < n; k++) B.h_fac[n + k] = B.h_sc[k].active != 0.0 ? 1.0 / sigma[k] : 0.0;
    LQ_TRY(write_scalars(c, B, n));
    LQ_TRY(write_fac(c, B, 3 * n));
    LQ_CU(blas_scale(L, L, c->Vh, n, p->mut(1), p->ref(1), B.fac, c->stream));
    LQ_CU(blas_scale(L, LQCD_F64, c->Vh, n, r->mut(1), W.r64->ref(1), B.fac + n, c->stream));
    LQ_TRY(op_mhat(c, L, W.recon_lo, 1, n, s->mut(1), r->ref(1), ye->mut(0), kNone, 0.0, &B.sc[0].gamma[cur],
                   kScStride));
    LQ_CU(blas_axpy(L, L, c->Vh, n, p->mut(1), s->ref(1), B.fac + 2 * n, c->stream));
    W.info->mhat_applies += 1;
  }
  W.info->iters = it;
  return done ? LQCD_OK : set_error(LQCD_ERR_NOCONV, "mixed CG did not converge in %d iterations", W.max_iter);
}

}  // namespace

}  // namespace lqcd

using namespace lqcd;

extern "C" lqcd_status lqcd_solve(lqcd_ctx *c, double *x, const double *b, int on_device,
                                  const lqcd_solve_params *prm, lqcd_solve_info *info) {
  if (!c) return set_error(LQCD_ERR_ARG, "context is NULL");
  if (!x || !b || !prm) return set_error(LQCD_ERR_ARG, "NULL argument");
  if (!(prm->tol > 0.0)) return set_error(LQCD_ERR_ARG, "tol must be > 0");
  if (prm->max_iter < 1) return set_error(LQCD_ERR_ARG, "max_iter must be >= 1");
  if (prm->nrhs < 1 || prm->nrhs > 64) return set_error(LQCD_ERR_ARG, "nrhs must be in 1..64");
  if ((int)prm->inner < 0 || (int)prm->inner > 3) return set_error(LQCD_ERR_ARG, "bad inner precision");
  if (prm->inner != LQCD_F64 && !(prm->delta > 0.0 && prm->delta < 1.0))
    return set_error(LQCD_ERR_ARG, "delta must be in (0, 1)");
  if (!c->have_gauge) return set_error(LQCD_ERR_STATE, "no gauge field loaded");
  if (!c->have_kappa) return set_error(LQCD_ERR_STATE, "kappa not set (call lqcd_clover)");
  const int recon64 = prm->recon == 12 ? 12 : 18;
  const int recon_lo = prm->inner_recon == 18 ? 18 : 12;
  if (prec_half(prm->inner) && recon_lo != 12) {
    return set_error(LQCD_ERR_ARG, "FP16/BF16 inner solves need 12-real links");
  }
  const auto t0 = std::chrono::steady_clock::now();
  lqcd_solve_info local{};
  lqcd_solve_info *inf = info ? info : &local;
  std::memset(inf, 0, sizeof(*inf));
  const int n = prm->nrhs;
  inf->nrhs = n;
  const size_t nd = (size_t)n * c->V * 24;

  SolveBufs B;
  if (cudaMalloc(&B.sc, sizeof(SolverScalars) * n) != cudaSuccess ||
      cudaMalloc(&B.fac, sizeof(double) * 3 * n) != cudaSuccess ||
      cudaMallocHost(&B.h_sc, sizeof(SolverScalars) * n) != cudaSuccess ||
      cudaMallocHost(&B.h_fac, sizeof(double) * 3 * n) != cudaSuccess) {
    cudaGetLastError();
    return set_error(LQCD_ERR_OOM, "cannot allocate solver scalars");
  }
  for (int k = 0; k < n; k++) {
    std::memset(&B.h_sc[k], 0, sizeof(SolverScalars));
    B.h_sc[k].active = 1.0;
  }
  LQ_CU(cudaMemcpyAsync(B.sc, B.h_sc, sizeof(SolverScalars) * n, cudaMemcpyHostToDevice, c->stream));

  // stage b (and x0) on the device
  const double *db = b;
  const double *dx0 = x;
  double *dx = x;
  if (!on_device) {
    double *d0, *d1;
    LQ_TRY(staging(c, 0, nd, &d0));
    LQ_TRY(staging(c, 1, nd, &d1));
    LQ_CU(cudaMemcpyAsync(d0, b, nd * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    if (prm->use_x0) LQ_CU(cudaMemcpyAsync(d1, x, nd * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    db = d0;
    dx0 = d1;
    dx = d1;
  }
  lqcd_field *bf, *xf, *bhat, *r64, *tmpe;
  LQ_TRY(temp_field(c, LQCD_F64, LQCD_FULL, n, 10, &bf));
  LQ_TRY(temp_field(c, LQCD_F64, LQCD_FULL, n, 11, &xf));
  LQ_TRY(temp_field(c, LQCD_F64, LQCD_ODD, n, 12, &bhat));
  LQ_TRY(temp_field(c, LQCD_F64, LQCD_ODD, n, 13, &r64));
  LQ_TRY(temp_field(c, LQCD_F64, LQCD_EVEN, n, 14, &tmpe));
  for (int p = 0; p < 2; p++)
    LQ_CU(pack_spinor(LQCD_F64, c->geom, p, db, n, bf->data[p], nullptr, bf->rhs_words(), c->stream));
  if (prm->use_x0)
    LQ_CU(pack_spinor(LQCD_F64, c->geom, 1, dx0, n, xf->data[1], nullptr, xf->rhs_words(), c->stream));
  else
    LQ_CU(cudaMemsetAsync(xf->data[1], 0, (size_t)xf->rhs_words() * 16 * n, c->stream));

  Work W;
  W.c = c;
  W.nrhs = n;
  W.recon64 = recon64;
  W.recon_lo = recon_lo;
  W.lo = prm->inner;
  W.tol = prm->tol;
  W.delta = prm->delta;
  W.max_iter = prm->max_iter;
  W.check_every = prm->check_every > 0 ? prm->check_every : 8;
  W.info = inf;
  W.bnorm.assign(n, 0.0);
  {
    std::vector<double> e(n), o(n);
    LQ_TRY(norms(c, LQCD_F64, n, bf->ref(0), e.data()));
    LQ_TRY(norms(c, LQCD_F64, n, bf->ref(1), o.data()));
    for (int k = 0; k < n; k++) W.bnorm[k] = std::sqrt(e[k] + o[k]);
  }
  for (int k = 0; k < n; k++)
    if (!(W.bnorm[k] > 0.0)) return set_error(LQCD_ERR_ARG, "right-hand side %d is zero or not finite", k);
  LQ_TRY(op_prepare(c, LQCD_F64, recon64, n, bhat->mut(1), bf->ref(0), bf->ref(1), tmpe->mut(0)));
  W.bhat = bhat;
  W.x64 = xf;
  W.r64 = r64;

  lqcd_status st;
  if (prm->inner == LQCD_F64) {
    st = cgls_fp64(W, B);
  } else {
    st = cgls_mixed(W, B);
  }
  lqcd_status solve_status = st;
  // reconstruct x_e, then the FP64 full-lattice residual b - M x
  LQ_TRY(op_reconstruct(c, LQCD_F64, recon64, n, xf->mut(0), bf->ref(0), xf->ref(1)));
  {
    lqcd_field *rf;
    LQ_TRY(temp_field(c, LQCD_F64, LQCD_FULL, n, 15, &rf));
    MutField o[2] = {rf->mut(0), rf->mut(1)};
    FieldRef xr[2] = {xf->ref(0), xf->ref(1)};
    FieldRef zr[2] = {bf->ref(0), bf->ref(1)};
    LQ_TRY(op_M(c, LQCD_F64, recon64, 0, n, o, xr, zr, -1.0, nullptr, 0));
    std::vector<double> e(n), od(n);
    LQ_TRY(norms(c, LQCD_F64, n, rf->ref(0), e.data()));
    LQ_TRY(norms(c, LQCD_F64, n, rf->ref(1), od.data()));
    bool ok = true;
    for (int k = 0; k < n; k++) {
      const double rel = std::sqrt(e[k] + od[k]) / W.bnorm[k];
      if (k < 64) inf->true_resid[k] = rel;
      if (!(rel <= prm->tol)) ok = false;
    }
    if (solve_status == LQCD_OK && !ok)
      solve_status = set_error(LQCD_ERR_NOCONV, "true residual above tol after convergence of the iterated one");
  }
  for (int p = 0; p < 2; p++)
    LQ_CU(unpack_spinor(LQCD_F64, c->geom, p, xf->data[p], nullptr, xf->rhs_words(), n, dx, c->stream));
  if (!on_device) LQ_CU(cudaMemcpyAsync(x, dx, nd * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  LQ_CU(cudaStreamSynchronize(c->stream));
  inf->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  return solve_status;
}
