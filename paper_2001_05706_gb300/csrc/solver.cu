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
// iteration).  FP64 CG: the host reads the residual norms every `check_every`
// iterations.  Mixed precision: r, p, q, s in FP32/FP16/BF16 storage and
// FP32 arithmetic, x_lo in FP32, normalised so the inner residual starts at
// norm 1; the inner loop runs in a CUDA graph conditional WHILE node until a
// device-side control kernel finds an update due (the inner residual fell
// below delta, reached the target, stagnated or turned round); then the FP64
// solution absorbs x_lo and the residual is recomputed with the FP64
// operator, the update being kept only if it lowers that residual; the search
// direction p is kept, rescaled into the new normalisation, and
// gamma = |Mhat^dag r|^2 recomputed from the new residual, or CG restarts
// from p = s after a rejected update or a turn-round.  With the symmetric
// Schur form every Mhat above is A_oo^-1 Mhat and every residual
// A_oo^-1 (bhat - Mhat x) (op_eo, residual_eo), its targets divided by a
// bound of ||A_oo||; BiCGStab (below) works on the same operators.
#include <algorithm>
#include <chrono>
#include <functional>
#include <memory>
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
  LQ_CU(blas_norm2(prec, c->Vh, nrhs, f, c->partials, c->results, 1, c->stream));
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
  lqcd_prec hp;  // precision of the CG (plain) or of the reliable updates (mixed): FP64 or DF64
  double tol, delta;
  int max_iter, check_every;
  std::vector<double> bnorm;  // ||b|| full lattice per RHS
  lqcd_field *bhat, *x64, *r64;  // precision hp: bhat_o, x (odd part used), r_o
  lqcd_solve_info *info;
  int schur = LQCD_SCHUR_ASYM;
  // targets on the recursion's residual are 0.5 tol ||b|| / rscale: 1 for Mhat; a
  // bound of ||A_oo|| for A_oo^-1 Mhat, whose residual is A_oo^-1 times the true one
  double rscale = 1.0;
  lqcd_field *t_hp = nullptr, *t_lo = nullptr;  // odd scratch of the symmetric form (precision hp, lo)
};

// The recursion's operator: Mhat x_o, or A_oo^-1 Mhat x_o with the symmetric
// Schur form (or the adjoint), optional fused norm.
lqcd_status op_eo(const Work &W, lqcd_prec prec, int recon, int dagger, MutField out, FieldRef x, lqcd_field *ye,
                  double *norm, int stride) {
  if (W.schur == LQCD_SCHUR_SYM) {
    lqcd_field *t = prec == W.hp ? W.t_hp : W.t_lo;
    return op_mhat_sym(W.c, prec, recon, dagger, W.nrhs, out, x, ye->mut(0), t->mut(1), norm, stride);
  }
  return op_mhat(W.c, prec, recon, dagger, W.nrhs, out, x, ye->mut(0), kNone, 0.0, norm, stride);
}

// The recursion's residual in precision hp: bhat - Mhat x, or A_oo^-1 (bhat -
// Mhat x) = A_oo^-1 bhat - A_oo^-1 Mhat x for the symmetric form, with its norm.
lqcd_status residual_eo(const Work &W, MutField r, FieldRef x, lqcd_field *ye, double *norm, int stride) {
  if (W.schur == LQCD_SCHUR_SYM) {
    LQ_TRY(op_mhat(W.c, W.hp, W.recon64, 0, W.nrhs, W.t_hp->mut(1), x, ye->mut(0), W.bhat->ref(1), -1.0, nullptr,
                   0));
    return op_ainv_odd(W.c, W.hp, W.recon64, W.nrhs, r, W.t_hp->ref(1), norm, stride);
  }
  return op_mhat(W.c, W.hp, W.recon64, 0, W.nrhs, r, x, ye->mut(0), W.bhat->ref(1), -1.0, norm, stride);
}

// Plain CGLS in FP64 or DF64: iterate until every RHS has ||r|| <= target,
// where r is recomputed as bhat - Mhat x before a right-hand side is accepted.
lqcd_status cgls_plain(Work &W, SolveBufs &B) {
  NvtxRange nv("lqcd CGLS (plain)");
  lqcd_ctx *c = W.c;
  const int n = W.nrhs;
  const lqcd_prec P = W.hp;
  lqcd_field *s, *p, *q, *ye;
  LQ_TRY(temp_field(c, P, LQCD_ODD, n, 20, &s));
  LQ_TRY(temp_field(c, P, LQCD_ODD, n, 21, &p));
  LQ_TRY(temp_field(c, P, LQCD_ODD, n, 22, &q));
  LQ_TRY(temp_field(c, P, LQCD_EVEN, n, 23, &ye));
  LQ_TRY(ensure_partials(c, n));
  std::vector<double> target2(n);
  for (int k = 0; k < n; k++) target2[k] = std::pow(0.5 * W.tol * W.bnorm[k] / W.rscale, 2);
  // r = bhat - Mhat x ; s = Mhat^dag r ; p = s
  LQ_TRY(residual_eo(W, W.r64->mut(1), W.x64->ref(1), ye, &B.sc[0].rr, kScStride));
  int cur = 0;
  LQ_TRY(op_eo(W, P, W.recon64, 1, s->mut(1), W.r64->ref(1), ye, &B.sc[0].gamma[cur], kScStride));
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
      LQ_TRY(op_eo(W, P, W.recon64, 0, q->mut(1), p->ref(1), ye, &B.sc[0].qq, kScStride));
      LQ_CU(blas_cg_xr(P, P, c->Vh, n, W.x64->mut(1), p->ref(1), W.r64->mut(1), q->ref(1), B.sc, cur, c->partials,
                       c->stream));
      LQ_TRY(op_eo(W, P, W.recon64, 1, s->mut(1), W.r64->ref(1), ye, &B.sc[0].gamma[1 - cur], kScStride));
      LQ_CU(blas_cg_p(P, c->Vh, n, p->mut(1), s->ref(1), B.sc, cur, c->stream));
      cur ^= 1;
      W.info->mhat_applies += 2;
    }
    LQ_TRY(read_scalars(c, B, n));
    // residual below target: recompute r = bhat - Mhat x before accepting it
    bool any = false;
    for (int k = 0; k < n; k++) any |= (B.h_sc[k].active != 0.0 && B.h_sc[k].rr <= target2[k]);
    if (any) {
      LQ_TRY(residual_eo(W, W.r64->mut(1), W.x64->ref(1), ye, &B.sc[0].aux, kScStride));
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

// ---------------------------------------------------------------------------
// Device-side loop control of the mixed-precision inner CG.
//
// The inner iterations run inside a CUDA graph conditional WHILE node: its
// body is one CG iteration followed by cg_control_kernel, which reads the new
// iterated residuals, updates per-RHS trigger state (best and reference
// residual, stagnation count, growth) and sets the loop condition.  The loop
// stops when a reliable update is due -- every active RHS dropped by delta or
// reached its target (a right-hand side that reached it is parked: it stops
// updating until the FP64 check), or one stagnated for kStallIters iterations
// or grew 20 % past its best -- or when the iteration cap of this launch is
// reached, so it always terminates.  The control kernel also moves the new gamma into the
// slot the next iteration reads, which makes the body the same every time.
// ---------------------------------------------------------------------------
constexpr int kStallIters = 48;

struct CtrlRhs {
  double best, ref, sigma, target;
  int stall, grown, parked, pad;
};
struct CtrlGlobal {
  int it, cap, stop, pad;
  double delta2;
};

__global__ void cg_control_kernel(SolverScalars *sc, CtrlRhs *cr, CtrlGlobal *cg, int n,
                                  cudaGraphConditionalHandle h, int use_handle) {
  __shared__ int all_dropped, any_trigger, nactive;
  const int k = threadIdx.x;
  if (k == 0) {
    all_dropped = 1;
    any_trigger = 0;
    nactive = 0;
  }
  __syncthreads();
  if (k < n) {
    sc[k].gamma[0] = sc[k].gamma[1];
    if (sc[k].active != 0.0) {
      atomicAdd(&nactive, 1);
      const double rr = sc[k].rr;
      CtrlRhs c = cr[k];
      if (!(rr == rr)) {
        c.grown = 1;
        any_trigger = 1;
      } else {
        if (rr < c.best) c.best = rr;
        if (rr < 0.25 * c.ref) {
          c.ref = rr;
          c.stall = 0;
        } else if (++c.stall >= kStallIters) {
          any_trigger = 1;
        }
        if (rr > 1.44 * c.best) {
          c.grown = 1;
          any_trigger = 1;
        }
        // a right-hand side at its target is parked (it stops updating) until
        // the FP64 check of the next reliable update confirms it; the others
        // iterate on
        if (c.sigma * sqrt(rr) <= c.target) {
          c.parked = 1;
          sc[k].active = 0.0;
        }
      }
      if (!c.parked && !(c.best <= cg->delta2)) all_dropped = 0;
      cr[k] = c;
    }
  }
  __syncthreads();
  if (k == 0) {
    const int it = cg->it + 1;
    cg->it = it;
    const int stop = (nactive == 0) || any_trigger || all_dropped || it >= cg->cap;
    cg->stop = stop;
    if (use_handle) cudaGraphSetConditional(h, stop ? 0u : 1u);
  }
}

// Mixed-precision CGLS as a resumable state machine: init() once, then the
// inner loop runs on the device (a graph with a WHILE node, see run_graph),
// and update() performs the reliable update the loop stopped for.
struct MixedCG {
  Work &W;
  SolveBufs &B;
  lqcd_ctx *c;
  int n;
  lqcd_prec L;
  lqcd_field *s = nullptr, *p = nullptr, *q = nullptr, *ye = nullptr, *r = nullptr, *xlo = nullptr, *ye64 = nullptr;
  lqcd_field *xtry = nullptr, *rtry = nullptr;
  std::vector<double> target, sigma;
  double delta2 = 0;
  size_t xlo_bytes = 0, rhs_bytes64 = 0;
  int it = 0;
  bool done = false;
  CtrlRhs *dcr = nullptr, *hcr = nullptr;
  CtrlGlobal *dcg = nullptr, *hcg = nullptr;

  MixedCG(Work &w, SolveBufs &b) : W(w), B(b), c(w.c), n(w.nrhs), L(w.lo) {}
  ~MixedCG() {
    if (dcr) cudaFree(dcr);
    if (dcg) cudaFree(dcg);
    if (hcr) cudaFreeHost(hcr);
    if (hcg) cudaFreeHost(hcg);
  }

  lqcd_status upload_ctrl() {
    LQ_CU(cudaMemcpyAsync(dcr, hcr, sizeof(CtrlRhs) * n, cudaMemcpyHostToDevice, c->stream));
    LQ_CU(cudaMemcpyAsync(dcg, hcg, sizeof(CtrlGlobal), cudaMemcpyHostToDevice, c->stream));
    return LQCD_OK;
  }

  lqcd_status download_ctrl() {
    LQ_CU(cudaMemcpyAsync(hcr, dcr, sizeof(CtrlRhs) * n, cudaMemcpyDeviceToHost, c->stream));
    LQ_CU(cudaMemcpyAsync(hcg, dcg, sizeof(CtrlGlobal), cudaMemcpyDeviceToHost, c->stream));
    LQ_TRY(read_scalars(c, B, n));
    return LQCD_OK;
  }

  void reset_rhs(int k) {
    hcr[k].parked = 0;
    hcr[k].best = 1.0;
    hcr[k].ref = 1.0;
    hcr[k].stall = 0;
    hcr[k].grown = 0;
    hcr[k].sigma = sigma[k];
    hcr[k].target = target[k];
  }

  lqcd_status init() {
    LQ_TRY(temp_field(c, L, LQCD_ODD, n, 30, &s));
    LQ_TRY(temp_field(c, L, LQCD_ODD, n, 31, &p));
    LQ_TRY(temp_field(c, L, LQCD_ODD, n, 32, &q));
    LQ_TRY(temp_field(c, L, LQCD_EVEN, n, 33, &ye));
    LQ_TRY(temp_field(c, L, LQCD_ODD, n, 34, &r));
    LQ_TRY(temp_field(c, LQCD_F32, LQCD_ODD, n, 35, &xlo));
    LQ_TRY(temp_field(c, W.hp, LQCD_ODD, n, 37, &xtry));
    LQ_TRY(temp_field(c, W.hp, LQCD_ODD, n, 38, &rtry));
    LQ_TRY(temp_field(c, W.hp, LQCD_EVEN, n, 23, &ye64));
    LQ_TRY(ensure_partials(c, n));
    if (dev_malloc((void **)&dcr, sizeof(CtrlRhs) * n) != cudaSuccess ||
        dev_malloc((void **)&dcg, sizeof(CtrlGlobal)) != cudaSuccess ||
        cudaMallocHost(&hcr, sizeof(CtrlRhs) * n) != cudaSuccess ||
        cudaMallocHost(&hcg, sizeof(CtrlGlobal)) != cudaSuccess) {
      cudaGetLastError();
      return set_error(LQCD_ERR_OOM, "cannot allocate solver control state");
    }
    target.assign(n, 0.0);
    sigma.assign(n, 0.0);
    for (int k = 0; k < n; k++) target[k] = 0.5 * W.tol * W.bnorm[k] / W.rscale;
    delta2 = W.delta * W.delta;
    rhs_bytes64 = (size_t)xtry->rhs_words() * 16;
    xlo_bytes = (size_t)xlo->rhs_words() * 16 * n;
    // r64 = bhat - Mhat64 x64 -> sigma
    LQ_TRY(residual_eo(W, W.r64->mut(1), W.x64->ref(1), ye64, &B.sc[0].aux, kScStride));
    W.info->mhat_applies += 1;
    LQ_TRY(read_scalars(c, B, n));
    int nactive = 0;
    for (int k = 0; k < n; k++) {
      sigma[k] = std::sqrt(B.h_sc[k].aux);
      B.h_sc[k].active = sigma[k] > target[k] ? 1.0 : 0.0;
      nactive += B.h_sc[k].active != 0.0;
      B.h_fac[k] = sigma[k] > 0 ? 1.0 / sigma[k] : 0.0;
      B.h_sc[k].rr = 1.0;
      std::memset(&hcr[k], 0, sizeof(CtrlRhs));
      reset_rhs(k);
    }
    std::memset(hcg, 0, sizeof(CtrlGlobal));
    hcg->delta2 = delta2;
    if (nactive == 0) {
      done = true;
      return LQCD_OK;
    }
    LQ_TRY(write_scalars(c, B, n));
    LQ_TRY(write_fac(c, B, n));
    // r_lo = r64 / sigma ; x_lo = 0 ; s = Mhat^dag r -> gamma[0] ; p = s
    LQ_CU(blas_scale(L, W.hp, c->Vh, n, r->mut(1), W.r64->ref(1), B.fac, c->stream));
    LQ_CU(cudaMemsetAsync(xlo->data[1], 0, xlo_bytes, c->stream));
    LQ_TRY(op_eo(W, L, W.recon_lo, 1, s->mut(1), r->ref(1), ye, &B.sc[0].gamma[0], kScStride));
    LQ_CU(cudaMemcpyAsync(p->data[1], s->data[1], (size_t)p->rhs_words() * 16 * n, cudaMemcpyDeviceToDevice,
                          c->stream));
    if (p->scale[1])
      LQ_CU(cudaMemcpyAsync(p->scale[1], s->scale[1], sizeof(float) * c->Vh * n, cudaMemcpyDeviceToDevice, c->stream));
    W.info->mhat_applies += 1;
    LQ_TRY(upload_ctrl());
    // one plain iteration: packs the inner links/clover and fills the tuning
    // cache before any capture (its result is thrown away by resetting x_lo,
    // r, p below is not needed: it is a genuine first iteration, kept)
    LQ_TRY(enqueue_iteration(0, false));
    LQ_CU(cudaStreamSynchronize(c->stream));
    it = 1;
    W.info->mhat_applies += 2;
    return LQCD_OK;
  }

  // one CG iteration and the control kernel; the new gamma goes to slot 1 and
  // the control kernel moves it to slot 0
  lqcd_status enqueue_iteration(cudaGraphConditionalHandle h, bool use_handle) const {
    LQ_TRY(op_eo(W, L, W.recon_lo, 0, q->mut(1), p->ref(1), ye, &B.sc[0].qq, kScStride));
    LQ_CU(blas_cg_xr(LQCD_F32, L, c->Vh, n, xlo->mut(1), p->ref(1), r->mut(1), q->ref(1), B.sc, 0, c->partials,
                     c->stream));
    LQ_TRY(op_eo(W, L, W.recon_lo, 1, s->mut(1), r->ref(1), ye, &B.sc[0].gamma[1], kScStride));
    LQ_CU(blas_cg_p(L, c->Vh, n, p->mut(1), s->ref(1), B.sc, 0, c->stream));
    cg_control_kernel<<<1, 64, 0, c->stream>>>(B.sc, dcr, dcg, n, h, use_handle ? 1 : 0);
    LQ_CU(cudaGetLastError());
    return LQCD_OK;
  }

  // before a graph launch: this launch may run up to `cap` iterations
  lqcd_status arm() {
    hcg->it = 0;
    hcg->cap = std::max(1, W.max_iter - it);
    hcg->stop = 0;
    LQ_CU(cudaMemcpyAsync(dcg, hcg, sizeof(CtrlGlobal), cudaMemcpyHostToDevice, c->stream));
    LQ_CU(cudaStreamSynchronize(c->stream));
    return LQCD_OK;
  }

  // after a graph launch: book the iterations and do the reliable update
  lqcd_status finish_launch() {
    LQ_TRY(download_ctrl());
    it += hcg->it;
    W.info->mhat_applies += 2.0 * hcg->it;
    return update();
  }

  char *rhs_ptr(lqcd_field *f, int k, size_t bytes) const { return static_cast<char *>(f->data[1]) + bytes * k; }

  // reliable update, accepted only if it lowers the FP64 residual:
  // x_try = x64 + sigma x_lo, r_try = bhat - Mhat64 x_try
  // a right-hand side takes part in an update while it iterates or is parked
  bool takes_part(int k) const { return B.h_sc[k].active != 0.0 || hcr[k].parked; }

  lqcd_status update() {
    NvtxRange nv("lqcd reliable update");
    for (int k = 0; k < n; k++) {
      if (B.h_sc[k].active != 0.0 && !(B.h_sc[k].rr == B.h_sc[k].rr))
        return set_error(LQCD_ERR_NOCONV, "inner residual of RHS %d is NaN at iteration %d", k, it);
      B.h_fac[k] = takes_part(k) ? sigma[k] : 0.0;
    }
    LQ_TRY(write_fac(c, B, n));
    LQ_CU(cudaMemcpyAsync(xtry->data[1], W.x64->data[1], rhs_bytes64 * n, cudaMemcpyDeviceToDevice, c->stream));
    LQ_CU(blas_axpy(W.hp, LQCD_F32, c->Vh, n, xtry->mut(1), xlo->ref(1), B.fac, c->stream));
    LQ_TRY(residual_eo(W, rtry->mut(1), xtry->ref(1), ye64, &B.sc[0].aux, kScStride));
    W.info->mhat_applies += 1;
    W.info->reliable_updates += 1;
    LQ_TRY(read_scalars(c, B, n));
    done = true;
    for (int k = 0; k < n; k++) {
      B.h_fac[k] = B.h_fac[n + k] = B.h_fac[2 * n + k] = 0.0;
      if (!takes_part(k)) continue;
      const double snew = std::sqrt(B.h_sc[k].aux);
      if (kTrace)
        std::fprintf(stderr,
                     "lqcd: update %d it %d rhs %d inner |r| %.3e best %.3e  FP64 |r| %.6e -> %.6e (target %.3e)\n",
                     W.info->reliable_updates, it, k, std::sqrt(B.h_sc[k].rr), std::sqrt(hcr[k].best), sigma[k],
                     snew, target[k]);
      if (!(snew == snew) || std::isinf(snew))
        return set_error(LQCD_ERR_NOCONV, "FP64 residual of RHS %d is not finite", k);
      const bool accept = snew < sigma[k];
      if (accept) {
        LQ_CU(cudaMemcpyAsync(rhs_ptr(W.x64, k, rhs_bytes64), rhs_ptr(xtry, k, rhs_bytes64), rhs_bytes64,
                              cudaMemcpyDeviceToDevice, c->stream));
        LQ_CU(cudaMemcpyAsync(rhs_ptr(W.r64, k, rhs_bytes64), rhs_ptr(rtry, k, rhs_bytes64), rhs_bytes64,
                              cudaMemcpyDeviceToDevice, c->stream));
        if (snew <= target[k]) {
          B.h_sc[k].active = 0.0;
          hcr[k].parked = 0;
          continue;
        }
      }
      done = false;
      // p (the next search direction) is kept, rescaled into the new
      // normalisation r_lo = r64 / snew, unless the update was rejected or the
      // inner iteration was turning round (grown, stagnating): then CG
      // restarts from p = s
      const bool restart = !accept || hcr[k].grown || hcr[k].parked || hcr[k].stall >= kStallIters;
      B.h_sc[k].active = 1.0;  // a parked right-hand side that was not converged iterates again
      const double snext = accept ? snew : sigma[k];
      B.h_fac[k] = restart ? 0.0 : sigma[k] / snext;
      B.h_fac[n + k] = 1.0 / snext;
      B.h_fac[2 * n + k] = restart ? 1.0 : 0.0;
      B.h_sc[k].rr = 1.0;
      sigma[k] = snext;
      reset_rhs(k);
    }
    LQ_CU(cudaMemsetAsync(xlo->data[1], 0, xlo_bytes, c->stream));
    if (done) return LQCD_OK;
    // factors: p *= fac[0, n); r = r64 * fac[n, 2n); p += fac[2n, 3n) s
    LQ_TRY(write_scalars(c, B, n));
    LQ_TRY(write_fac(c, B, 3 * n));
    LQ_TRY(upload_ctrl());
    LQ_CU(blas_scale(L, L, c->Vh, n, p->mut(1), p->ref(1), B.fac, c->stream));
    LQ_CU(blas_scale(L, W.hp, c->Vh, n, r->mut(1), W.r64->ref(1), B.fac + n, c->stream));
    LQ_TRY(op_eo(W, L, W.recon_lo, 1, s->mut(1), r->ref(1), ye, &B.sc[0].gamma[0], kScStride));
    LQ_CU(blas_axpy(L, L, c->Vh, n, p->mut(1), s->ref(1), B.fac + 2 * n, c->stream));
    W.info->mhat_applies += 1;
    LQ_CU(cudaStreamSynchronize(c->stream));
    return LQCD_OK;
  }
};

// A graph with one conditional WHILE node per solver, each body captured on
// that solver's stream; the nodes are independent, so the lattices of a batch
// run concurrently.  Launched on `launch`.
struct LoopGraph {
  cudaGraphExec_t exec = nullptr;
  ~LoopGraph() {
    if (exec) cudaGraphExecDestroy(exec);
  }
  lqcd_status build(const std::vector<MixedCG *> &cgs) {
    if (exec) {
      cudaGraphExecDestroy(exec);
      exec = nullptr;
    }
    cudaGraph_t g = nullptr;
    LQ_CU(cudaGraphCreate(&g, 0));
    lqcd_status st = LQCD_OK;
    for (MixedCG *m : cgs) {
      cudaGraphConditionalHandle h;
      if (cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault) != cudaSuccess) {
        st = set_error(LQCD_ERR_CUDA, "cudaGraphConditionalHandleCreate failed");
        break;
      }
      cudaGraphNodeParams prm = {};
      prm.type = cudaGraphNodeTypeConditional;
      prm.conditional.handle = h;
      prm.conditional.type = cudaGraphCondTypeWhile;
      prm.conditional.size = 1;
      cudaGraphNode_t node;
      if (cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &prm) != cudaSuccess) {
        st = set_error(LQCD_ERR_CUDA, "adding the conditional WHILE node failed");
        break;
      }
      cudaGraph_t body = prm.conditional.phGraph_out[0];
      if (cudaStreamBeginCaptureToGraph(m->c->stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) !=
          cudaSuccess) {
        st = set_error(LQCD_ERR_CUDA, "capture into the loop body failed");
        break;
      }
      st = m->enqueue_iteration(h, true);
      cudaGraph_t out = nullptr;
      const cudaError_t e = cudaStreamEndCapture(m->c->stream, &out);
      if (st == LQCD_OK && e != cudaSuccess) st = set_error(LQCD_ERR_CUDA, "loop body capture: %s", cudaGetErrorString(e));
      if (st != LQCD_OK) break;
    }
    if (st == LQCD_OK) {
      const cudaError_t e = cudaGraphInstantiate(&exec, g, 0);
      if (e != cudaSuccess) st = set_error(LQCD_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(e));
    }
    cudaGraphDestroy(g);
    cudaGetLastError();
    return st;
  }
};

// Drive a set of mixed solvers to completion: arm, launch the loop graph,
// update, repeat; the graph is rebuilt when the set of unfinished solvers
// changes.
lqcd_status run_mixed(const std::vector<MixedCG *> &all, cudaStream_t launch, int max_iter) {
  LoopGraph graph;
  std::vector<MixedCG *> prev;
  while (true) {
    std::vector<MixedCG *> active;
    for (MixedCG *m : all)
      if (!m->done && m->it < max_iter) active.push_back(m);
    if (active.empty()) return LQCD_OK;
    if (active != prev || !graph.exec) {
      LQ_TRY(graph.build(active));
      prev = active;
    }
    for (MixedCG *m : active) LQ_TRY(m->arm());
    LQ_CU(cudaGraphLaunch(graph.exec, launch));
    LQ_CU(cudaStreamSynchronize(launch));
    for (MixedCG *m : active) LQ_TRY(m->finish_launch());
  }
}

lqcd_status cgls_mixed(Work &W, SolveBufs &B) {
  NvtxRange nv("lqcd CGLS (mixed)");
  MixedCG m(W, B);
  LQ_TRY(m.init());
  if (!m.done) LQ_TRY(run_mixed({&m}, W.c->stream, W.max_iter));
  W.info->iters = m.it;
  return m.done ? LQCD_OK : set_error(LQCD_ERR_NOCONV, "mixed CG did not converge in %d iterations", W.max_iter);
}

// ---------------------------------------------------------------------------
// BiCGStab on Mhat x = bhat (building blocks in bicgstab.cu), one recursion per
// right-hand side with its complex scalars in device memory.  Plain: vectors
// in FP64 or DF64, and when an iterated residual reaches its target the true
// residual bhat - Mhat x replaces r (converged right-hand sides stop).  Mixed:
// vectors in FP32/FP16/BF16 (FP32 arithmetic) on the residual normalised to 1,
// x_lo in FP32; when every active inner residual fell by delta or reached its
// target (a right-hand side that reached it is parked: it stops until the
// check), or one grew past 1e4, the high-precision solution absorbs sigma x_lo and
// the residual is recomputed in FP64/DF64 (a reliable update).  The shadow
// residual rhat is kept across updates; r takes the new residual, p and v are
// rescaled with it, rho_old too, and rho = (rhat, r) is recomputed, so the
// recursion continues where it was.  The host looks at the residuals every
// check_every iterations.
// ---------------------------------------------------------------------------
lqcd_status bicgstab(Work &W, bool mixed) {
  NvtxRange nv(mixed ? "lqcd BiCGStab (mixed)" : "lqcd BiCGStab (plain)");
  lqcd_ctx *c = W.c;
  const int n = W.nrhs;
  const lqcd_prec L = mixed ? W.lo : W.hp;
  const int rec = mixed ? W.recon_lo : W.recon64;
  lqcd_field *rhat, *r, *p, *v, *sv, *t, *ye, *ye64, *xlo = nullptr;
  LQ_TRY(temp_field(c, L, LQCD_ODD, n, 50, &rhat));
  LQ_TRY(temp_field(c, L, LQCD_ODD, n, 51, &r));
  LQ_TRY(temp_field(c, L, LQCD_ODD, n, 52, &p));
  LQ_TRY(temp_field(c, L, LQCD_ODD, n, 53, &v));
  LQ_TRY(temp_field(c, L, LQCD_ODD, n, 54, &sv));
  LQ_TRY(temp_field(c, L, LQCD_ODD, n, 55, &t));
  LQ_TRY(temp_field(c, L, LQCD_EVEN, n, 56, &ye));
  LQ_TRY(temp_field(c, W.hp, LQCD_EVEN, n, 58, &ye64));
  if (mixed) LQ_TRY(temp_field(c, LQCD_F32, LQCD_ODD, n, 57, &xlo));
  LQ_TRY(ensure_partials(c, 3 * n));
  struct Bufs {
    BiScalars *ds = nullptr, *hs = nullptr;
    double *red = nullptr, *hred = nullptr, *fac = nullptr, *hfac = nullptr;
    ~Bufs() {
      if (ds) cudaFree(ds);
      if (red) cudaFree(red);
      if (fac) cudaFree(fac);
      if (hs) cudaFreeHost(hs);
      if (hred) cudaFreeHost(hred);
      if (hfac) cudaFreeHost(hfac);
    }
  } b;
  if (dev_malloc((void **)&b.ds, sizeof(BiScalars) * n) != cudaSuccess ||
      dev_malloc((void **)&b.red, sizeof(double) * kBiRed * n) != cudaSuccess ||
      dev_malloc((void **)&b.fac, sizeof(double) * 2 * n) != cudaSuccess ||
      cudaMallocHost(&b.hs, sizeof(BiScalars) * n) != cudaSuccess ||
      cudaMallocHost(&b.hred, sizeof(double) * kBiRed * n) != cudaSuccess ||
      cudaMallocHost(&b.hfac, sizeof(double) * 2 * n) != cudaSuccess) {
    cudaGetLastError();
    return set_error(LQCD_ERR_OOM, "cannot allocate BiCGStab state");
  }
  double *red_rv = b.red, *red_ts = b.red + 3 * n, *red_xr = b.red + 6 * n;
  const size_t vbytes = (size_t)r->rhs_words() * 16 * n;
  const size_t sbytes = r->scale[1] ? sizeof(float) * c->Vh * n : 0;
  std::vector<double> target(n), sigma(n, 1.0), nrm(n);
  std::vector<char> active(n, 1), parked(n, 0);
  for (int k = 0; k < n; k++) target[k] = 0.5 * W.tol * W.bnorm[k] / W.rscale;
  // high-precision residual r64 = bhat - Mhat x64 (symmetric form: A_oo^-1 times it) and its norms
  auto true_residual = [&]() -> lqcd_status {
    LQ_TRY(residual_eo(W, W.r64->mut(1), W.x64->ref(1), ye64, c->results, 1));
    LQ_CU(cudaMemcpyAsync(c->h_results, c->results, sizeof(double) * n, cudaMemcpyDeviceToHost, c->stream));
    LQ_CU(cudaStreamSynchronize(c->stream));
    for (int k = 0; k < n; k++) nrm[k] = std::sqrt(c->h_results[k]);
    W.info->mhat_applies += 1;
    return LQCD_OK;
  };
  auto copy_vec = [&](lqcd_field *dst, const lqcd_field *src) -> lqcd_status {
    LQ_CU(cudaMemcpyAsync(dst->data[1], src->data[1], vbytes, cudaMemcpyDeviceToDevice, c->stream));
    if (sbytes) LQ_CU(cudaMemcpyAsync(dst->scale[1], src->scale[1], sbytes, cudaMemcpyDeviceToDevice, c->stream));
    return LQCD_OK;
  };
  // r from r64 (normalised when mixed), then rho = (rhat, r)
  auto load_r = [&]() -> lqcd_status {
    if (mixed) {
      for (int k = 0; k < n; k++) b.hfac[k] = active[k] ? 1.0 / sigma[k] : 0.0;
      LQ_CU(cudaMemcpyAsync(b.fac, b.hfac, sizeof(double) * n, cudaMemcpyHostToDevice, c->stream));
      LQ_CU(blas_scale(L, W.hp, c->Vh, n, r->mut(1), W.r64->ref(1), b.fac, c->stream));
    } else {
      LQ_TRY(copy_vec(r, W.r64));
    }
    return LQCD_OK;
  };
  LQ_TRY(true_residual());
  int nact = 0;
  for (int k = 0; k < n; k++) {
    active[k] = nrm[k] > target[k];
    nact += active[k];
    if (mixed) sigma[k] = nrm[k] > 0 ? nrm[k] : 1.0;
  }
  if (nact == 0) return LQCD_OK;
  LQ_TRY(load_r());
  LQ_TRY(copy_vec(rhat, r));
  for (lqcd_field *f : {p, v}) {
    LQ_CU(cudaMemsetAsync(f->data[1], 0, vbytes, c->stream));
    if (sbytes) LQ_CU(cudaMemsetAsync(f->scale[1], 0, sbytes, c->stream));
  }
  if (mixed) LQ_CU(cudaMemsetAsync(xlo->data[1], 0, (size_t)xlo->rhs_words() * 16 * n, c->stream));
  for (int k = 0; k < n; k++) {
    std::memset(&b.hs[k], 0, sizeof(BiScalars));
    b.hs[k].rho_old = b.hs[k].alpha = b.hs[k].omega = make_double2(1.0, 0.0);
    b.hs[k].active = active[k] ? 1.0 : 0.0;
  }
  LQ_CU(cudaMemcpyAsync(b.ds, b.hs, sizeof(BiScalars) * n, cudaMemcpyHostToDevice, c->stream));
  LQ_CU(bi_dot3(L, c->Vh, n, rhat->ref(1), r->ref(1), c->partials, red_xr, c->stream));
  lqcd_field *x = mixed ? xlo : W.x64;
  const lqcd_prec px = mixed ? LQCD_F32 : W.hp;
  const double delta2 = W.delta * W.delta;
  int it = 0;
  while (true) {
    for (int j = 0; j < W.check_every && it < W.max_iter; j++, it++) {
      LQ_CU(bi_scalar(BI_BETA, b.ds, red_xr, n, c->stream));
      LQ_CU(bi_p(L, c->Vh, n, p->mut(1), r->ref(1), v->ref(1), b.ds, c->stream));
      LQ_TRY(op_eo(W, L, rec, 0, v->mut(1), p->ref(1), ye, nullptr, 0));
      LQ_CU(bi_dot3(L, c->Vh, n, rhat->ref(1), v->ref(1), c->partials, red_rv, c->stream));
      LQ_CU(bi_scalar(BI_ALPHA, b.ds, red_rv, n, c->stream));
      LQ_CU(bi_s(L, c->Vh, n, sv->mut(1), r->ref(1), v->ref(1), b.ds, c->stream));
      LQ_TRY(op_eo(W, L, rec, 0, t->mut(1), sv->ref(1), ye, nullptr, 0));
      LQ_CU(bi_dot3(L, c->Vh, n, t->ref(1), sv->ref(1), c->partials, red_ts, c->stream));
      LQ_CU(bi_scalar(BI_OMEGA, b.ds, red_ts, n, c->stream));
      LQ_CU(bi_xr(px, L, c->Vh, n, x->mut(1), p->ref(1), sv->ref(1), t->ref(1), r->mut(1), rhat->ref(1), b.ds,
                  c->partials, red_xr, c->stream));
      W.info->mhat_applies += 2;
    }
    LQ_CU(cudaMemcpyAsync(b.hred, b.red, sizeof(double) * kBiRed * n, cudaMemcpyDeviceToHost, c->stream));
    LQ_CU(cudaStreamSynchronize(c->stream));
    // a right-hand side whose iterated residual reached its target is parked
    // (the kernels skip it) until the next true-residual check confirms it
    bool all_dropped = true, grown = false, newly_parked = false, any_left = false;
    for (int k = 0; k < n; k++) {
      if (!active[k] || parked[k]) continue;
      const double rr = b.hred[6 * n + 3 * k + 2];
      if (!std::isfinite(rr)) return set_error(LQCD_ERR_NOCONV, "BiCGStab breakdown on RHS %d at iteration %d", k, it);
      if (sigma[k] * std::sqrt(rr) <= target[k]) {
        parked[k] = 1;
        newly_parked = true;
        continue;
      }
      any_left = true;
      if (!(rr <= delta2)) all_dropped = false;
      if (rr > 1e8) grown = true;
    }
    const bool at_cap = it >= W.max_iter;
    if (!(!any_left || (mixed && (all_dropped || grown)) || at_cap)) {
      if (newly_parked) {
        LQ_CU(cudaMemcpyAsync(b.hs, b.ds, sizeof(BiScalars) * n, cudaMemcpyDeviceToHost, c->stream));
        LQ_CU(cudaStreamSynchronize(c->stream));
        for (int k = 0; k < n; k++)
          if (parked[k]) b.hs[k].active = 0.0;
        LQ_CU(cudaMemcpyAsync(b.ds, b.hs, sizeof(BiScalars) * n, cudaMemcpyHostToDevice, c->stream));
      }
      continue;
    }
    // reliable update (mixed) / true-residual replacement (plain)
    if (mixed) {
      for (int k = 0; k < n; k++) b.hfac[k] = active[k] ? sigma[k] : 0.0;
      LQ_CU(cudaMemcpyAsync(b.fac, b.hfac, sizeof(double) * n, cudaMemcpyHostToDevice, c->stream));
      LQ_CU(blas_axpy(W.hp, LQCD_F32, c->Vh, n, W.x64->mut(1), xlo->ref(1), b.fac, c->stream));
      LQ_CU(cudaMemsetAsync(xlo->data[1], 0, (size_t)xlo->rhs_words() * 16 * n, c->stream));
      W.info->reliable_updates += 1;
    }
    LQ_TRY(true_residual());
    LQ_CU(cudaMemcpyAsync(b.hs, b.ds, sizeof(BiScalars) * n, cudaMemcpyDeviceToHost, c->stream));
    LQ_CU(cudaStreamSynchronize(c->stream));
    nact = 0;
    for (int k = 0; k < n; k++) {
      b.hfac[k] = 0.0;
      if (!active[k]) continue;
      if (!std::isfinite(nrm[k])) return set_error(LQCD_ERR_NOCONV, "residual of RHS %d is not finite", k);
      if (nrm[k] <= target[k]) {
        active[k] = 0;
        parked[k] = 0;
        b.hs[k].active = 0.0;
        continue;
      }
      nact++;
      parked[k] = 0;
      b.hs[k].active = 1.0;  // a parked right-hand side that was not converged iterates again
      if (mixed) {  // p, v and rho_old follow r into the new normalisation
        const double f = sigma[k] / nrm[k];
        b.hfac[k] = f;
        b.hs[k].rho_old = make_double2(b.hs[k].rho_old.x * f, b.hs[k].rho_old.y * f);
        sigma[k] = nrm[k];
      }
    }
    if (nact == 0) break;
    if (at_cap) break;
    LQ_CU(cudaMemcpyAsync(b.ds, b.hs, sizeof(BiScalars) * n, cudaMemcpyHostToDevice, c->stream));
    if (mixed) {
      LQ_CU(cudaMemcpyAsync(b.fac, b.hfac, sizeof(double) * n, cudaMemcpyHostToDevice, c->stream));
      LQ_CU(blas_scale(L, L, c->Vh, n, p->mut(1), p->ref(1), b.fac, c->stream));
      LQ_CU(blas_scale(L, L, c->Vh, n, v->mut(1), v->ref(1), b.fac, c->stream));
    }
    LQ_TRY(load_r());
    LQ_CU(bi_dot3(L, c->Vh, n, rhat->ref(1), r->ref(1), c->partials, red_xr, c->stream));
  }
  W.info->iters = it;
  return nact == 0 ? LQCD_OK : set_error(LQCD_ERR_NOCONV, "BiCGStab did not converge in %d iterations", W.max_iter);
}

// Restarted GCR(m) on the recursion's operator (Mhat, or A_oo^-1 Mhat).  Per
// step: z = r, q = A z, q and z orthogonalised against the cycle's earlier
// q_i (one classical Gram-Schmidt pass, the same coefficients on z), both
// scaled to |q| = 1; then alpha = (q, r), x += alpha z, r -= alpha q, so |r|
// falls monotonically (GCR minimises it over the cycle's Krylov space).
// Plain: every step in precision hp, the cycle restarted from the true
// residual after m steps.  Mixed: a cycle runs in the inner precision on the
// residual normalised to 1 and ends after m steps, when every active |r|
// dropped below delta, or when a right-hand side reached its target; the
// FP64 (DF64) solution absorbs it and the true residual starts the next one.
lqcd_status gcr(Work &W, bool mixed, int m) {
  NvtxRange nv(mixed ? "lqcd GCR (mixed)" : "lqcd GCR (plain)");
  lqcd_ctx *c = W.c;
  const int n = W.nrhs;
  const lqcd_prec L = mixed ? W.lo : W.hp;
  const int rec = mixed ? W.recon_lo : W.recon64;
  const lqcd_prec px = mixed ? LQCD_F32 : W.hp;  // the cycle's solution accumulates in FP32 when mixed
  std::vector<lqcd_field *> z(m), q(m);
  lqcd_field *r, *ye, *ye64, *xlo = nullptr;
  for (int j = 0; j < m; j++) {
    LQ_TRY(temp_field(c, L, LQCD_ODD, n, 100 + j, &z[j]));
    LQ_TRY(temp_field(c, L, LQCD_ODD, n, 200 + j, &q[j]));
  }
  LQ_TRY(temp_field(c, L, LQCD_ODD, n, 60, &r));
  LQ_TRY(temp_field(c, L, LQCD_EVEN, n, 61, &ye));
  LQ_TRY(temp_field(c, W.hp, LQCD_EVEN, n, 62, &ye64));
  if (mixed) LQ_TRY(temp_field(c, LQCD_F32, LQCD_ODD, n, 63, &xlo));
  LQ_TRY(ensure_partials(c, 3 * n * m));
  struct Bufs {
    double *red = nullptr, *hred = nullptr, *fac = nullptr, *hfac = nullptr;
    double2 *cf = nullptr, *hcf = nullptr;
    ~Bufs() {
      if (red) cudaFree(red);
      if (fac) cudaFree(fac);
      if (cf) cudaFree(cf);
      if (hred) cudaFreeHost(hred);
      if (hfac) cudaFreeHost(hfac);
      if (hcf) cudaFreeHost(hcf);
    }
  } b;
  const size_t nred = 3 * (size_t)n * (m + 2);
  if (dev_malloc((void **)&b.red, sizeof(double) * nred) != cudaSuccess ||
      dev_malloc((void **)&b.fac, sizeof(double) * n) != cudaSuccess ||
      dev_malloc((void **)&b.cf, sizeof(double2) * n * (size_t)(m + 1)) != cudaSuccess ||
      cudaMallocHost(&b.hred, sizeof(double) * nred) != cudaSuccess ||
      cudaMallocHost(&b.hfac, sizeof(double) * n) != cudaSuccess ||
      cudaMallocHost(&b.hcf, sizeof(double2) * n * (size_t)(m + 1)) != cudaSuccess) {
    cudaGetLastError();
    return set_error(LQCD_ERR_OOM, "cannot allocate GCR state");
  }
  const size_t vbytes = (size_t)r->rhs_words() * 16 * n;
  const size_t sbytes = r->scale[1] ? sizeof(float) * c->Vh * n : 0;
  std::vector<double> target(n), sigma(n, 1.0), nrm(n), rr(n);
  std::vector<char> active(n, 1);
  for (int k = 0; k < n; k++) target[k] = 0.5 * W.tol * W.bnorm[k] / W.rscale;
  auto sync_red = [&]() -> lqcd_status {
    LQ_CU(cudaMemcpyAsync(b.hred, b.red, sizeof(double) * nred, cudaMemcpyDeviceToHost, c->stream));
    LQ_CU(cudaStreamSynchronize(c->stream));
    return LQCD_OK;
  };
  auto true_residual = [&]() -> lqcd_status {
    LQ_TRY(residual_eo(W, W.r64->mut(1), W.x64->ref(1), ye64, c->results, 1));
    LQ_CU(cudaMemcpyAsync(c->h_results, c->results, sizeof(double) * n, cudaMemcpyDeviceToHost, c->stream));
    LQ_CU(cudaStreamSynchronize(c->stream));
    for (int k = 0; k < n; k++) nrm[k] = std::sqrt(c->h_results[k]);
    W.info->mhat_applies += 1;
    return LQCD_OK;
  };
  auto copy_vec = [&](lqcd_field *dst, const lqcd_field *src) -> lqcd_status {
    LQ_CU(cudaMemcpyAsync(dst->data[1], src->data[1], vbytes, cudaMemcpyDeviceToDevice, c->stream));
    if (sbytes) LQ_CU(cudaMemcpyAsync(dst->scale[1], src->scale[1], sbytes, cudaMemcpyDeviceToDevice, c->stream));
    return LQCD_OK;
  };
  auto scale = [&](lqcd_field *f, const std::vector<double> &fv) -> lqcd_status {
    std::memcpy(b.hfac, fv.data(), sizeof(double) * n);
    LQ_CU(cudaMemcpyAsync(b.fac, b.hfac, sizeof(double) * n, cudaMemcpyHostToDevice, c->stream));
    LQ_CU(blas_scale(L, L, c->Vh, n, f->mut(1), f->ref(1), b.fac, c->stream));
    return LQCD_OK;
  };
  // the coefficient set `slot` of the cycle's device coefficient array
  auto put_cf = [&](int slot) -> double2 * {
    return b.cf + (size_t)n * slot;
  };
  auto upload_cf = [&](int slot) -> lqcd_status {
    LQ_CU(cudaMemcpyAsync(put_cf(slot), b.hcf + (size_t)n * slot, sizeof(double2) * n, cudaMemcpyHostToDevice,
                          c->stream));
    return LQCD_OK;
  };
  LQ_TRY(true_residual());
  int nact = 0;
  for (int k = 0; k < n; k++) {
    active[k] = nrm[k] > target[k];
    nact += active[k];
  }
  lqcd_field *x = mixed ? xlo : W.x64;
  int it = 0;
  while (nact > 0 && it < W.max_iter) {
    // the cycle's residual r: r64 (normalised when mixed)
    std::vector<double> f(n, 0.0);
    for (int k = 0; k < n; k++) {
      if (mixed) sigma[k] = nrm[k] > 0 ? nrm[k] : 1.0;
      f[k] = active[k] ? (mixed ? 1.0 / sigma[k] : 1.0) : 0.0;
      rr[k] = (active[k] ? nrm[k] * f[k] : 0.0);
      rr[k] *= rr[k];
    }
    std::memcpy(b.hfac, f.data(), sizeof(double) * n);
    LQ_CU(cudaMemcpyAsync(b.fac, b.hfac, sizeof(double) * n, cudaMemcpyHostToDevice, c->stream));
    LQ_CU(blas_scale(L, W.hp, c->Vh, n, r->mut(1), W.r64->ref(1), b.fac, c->stream));
    if (mixed) LQ_CU(cudaMemsetAsync(xlo->data[1], 0, (size_t)xlo->rhs_words() * 16 * n, c->stream));
    std::vector<char> on = active;  // right-hand sides this cycle still works on
    const std::vector<double> rr0 = rr;
    int j = 0;
    for (; j < m && it < W.max_iter; j++, it++) {
      LQ_TRY(copy_vec(z[j], r));
      LQ_TRY(op_eo(W, L, rec, 0, q[j]->mut(1), z[j]->ref(1), ye, nullptr, 0));
      W.info->mhat_applies += 1;
      // beta_i = (q_i, q), all i < j at once (classical Gram-Schmidt)
      for (int i = 0; i < j; i++)
        LQ_CU(bi_dot3(L, c->Vh, n, q[i]->ref(1), q[j]->ref(1), c->partials, b.red + 3 * (size_t)n * i, c->stream));
      if (j > 0) {
        LQ_TRY(sync_red());
        for (int i = 0; i < j; i++) {
          for (int k = 0; k < n; k++) {
            const double *d = b.hred + 3 * (size_t)n * i + 3 * k;
            b.hcf[(size_t)n * i + k] = on[k] ? make_double2(-d[0], -d[1]) : make_double2(0.0, 0.0);
          }
          LQ_TRY(upload_cf(i));
          LQ_CU(gcr_caxpy(L, L, c->Vh, n, q[j]->mut(1), q[i]->ref(1), put_cf(i), c->stream));
          LQ_CU(gcr_caxpy(L, L, c->Vh, n, z[j]->mut(1), z[i]->ref(1), put_cf(i), c->stream));
        }
      }
      // |q|, then q, z scaled to |q| = 1
      LQ_CU(bi_dot3(L, c->Vh, n, q[j]->ref(1), q[j]->ref(1), c->partials, b.red, c->stream));
      LQ_TRY(sync_red());
      std::vector<double> inv(n, 0.0);
      for (int k = 0; k < n; k++) {
        const double qq = b.hred[3 * k + 2];
        if (!std::isfinite(qq)) return set_error(LQCD_ERR_NOCONV, "GCR breakdown on RHS %d at iteration %d", k, it);
        if (on[k] && qq > 0) inv[k] = 1.0 / std::sqrt(qq);
        else on[k] = 0;
      }
      LQ_TRY(scale(q[j], inv));
      LQ_TRY(scale(z[j], inv));
      // alpha = (q, r): x += alpha z, r -= alpha q
      LQ_CU(bi_dot3(L, c->Vh, n, q[j]->ref(1), r->ref(1), c->partials, b.red, c->stream));
      LQ_TRY(sync_red());
      for (int k = 0; k < n; k++) {
        const double *d = b.hred + 3 * k;
        b.hcf[(size_t)n * m + k] = on[k] ? make_double2(d[0], d[1]) : make_double2(0.0, 0.0);
        if (on[k]) rr[k] = std::max(rr[k] - (d[0] * d[0] + d[1] * d[1]), 0.0);  // |r|^2 - |alpha|^2
      }
      LQ_TRY(upload_cf(m));
      LQ_CU(gcr_caxpy(px, L, c->Vh, n, x->mut(1), z[j]->ref(1), put_cf(m), c->stream));
      for (int k = 0; k < n; k++) b.hcf[(size_t)n * m + k] = make_double2(-b.hcf[(size_t)n * m + k].x,
                                                                          -b.hcf[(size_t)n * m + k].y);
      LQ_TRY(upload_cf(m));
      LQ_CU(gcr_caxpy(L, L, c->Vh, n, r->mut(1), q[j]->ref(1), put_cf(m), c->stream));
      // end the cycle early once every right-hand side reached its target, or
      // (mixed) once every active residual fell by delta or one reached it
      bool all_dropped = true, reached = false, all_reached = true;
      for (int k = 0; k < n; k++) {
        if (!on[k]) continue;
        const bool rk = sigma[k] * std::sqrt(rr[k]) <= target[k];
        reached |= rk;
        all_reached &= rk;
        if (rr[k] > W.delta * W.delta * rr0[k]) all_dropped = false;
      }
      if (all_reached || (mixed && (all_dropped || reached))) {
        j++;
        it++;
        break;
      }
    }
    if (mixed) {  // x64 += sigma x_lo
      for (int k = 0; k < n; k++) b.hfac[k] = active[k] ? sigma[k] : 0.0;
      LQ_CU(cudaMemcpyAsync(b.fac, b.hfac, sizeof(double) * n, cudaMemcpyHostToDevice, c->stream));
      LQ_CU(blas_axpy(W.hp, LQCD_F32, c->Vh, n, W.x64->mut(1), xlo->ref(1), b.fac, c->stream));
      W.info->reliable_updates += 1;
    }
    LQ_TRY(true_residual());
    nact = 0;
    for (int k = 0; k < n; k++) {
      if (!active[k]) continue;
      if (!std::isfinite(nrm[k])) return set_error(LQCD_ERR_NOCONV, "residual of RHS %d is not finite", k);
      if (nrm[k] <= target[k]) {
        active[k] = 0;
        continue;
      }
      nact++;
    }
  }
  W.info->iters = it;
  return nact == 0 ? LQCD_OK : set_error(LQCD_ERR_NOCONV, "GCR did not converge in %d iterations", W.max_iter);
}

// One solve: staging, even-odd source, the recursion, reconstruction and the
// FP64 true residual.  Split so that a batch of lattices can share the loop.
struct SolveJob {
  lqcd_ctx *c = nullptr;
  double *x = nullptr;
  const double *b = nullptr;
  int on_device = 0;
  lqcd_solve_params prm{};
  lqcd_solve_info *inf = nullptr;
  lqcd_solve_info local{};
  SolveBufs B;
  Work W;
  lqcd_field *bf = nullptr, *xf = nullptr, *bhat = nullptr, *r64 = nullptr, *tmpe = nullptr;
  double *dx = nullptr;
  size_t nd = 0;
  std::chrono::steady_clock::time_point t0;
};

// inner FP64 or DF64: the plain CG in that precision, no reliable updates
bool plain_cg(const lqcd_solve_params *prm) { return prm->inner == LQCD_F64 || prm->inner == LQCD_DF64; }

lqcd_status check_params(lqcd_ctx *c, const lqcd_solve_params *prm) {
  if (!c) return set_error(LQCD_ERR_ARG, "context is NULL");
  if (!prm) return set_error(LQCD_ERR_ARG, "NULL argument");
  if (!(prm->tol > 0.0)) return set_error(LQCD_ERR_ARG, "tol must be > 0");
  if (prm->max_iter < 1) return set_error(LQCD_ERR_ARG, "max_iter must be >= 1");
  if (prm->nrhs < 1 || prm->nrhs > 64) return set_error(LQCD_ERR_ARG, "nrhs must be in 1..64");
  if ((int)prm->inner < 0 || (int)prm->inner > 4) return set_error(LQCD_ERR_ARG, "bad inner precision");
  if (prm->solver != LQCD_SOLVER_CGLS && prm->solver != LQCD_SOLVER_BICGSTAB && prm->solver != LQCD_SOLVER_GCR)
    return set_error(LQCD_ERR_ARG, "bad solver %d", prm->solver);
  if (prm->solver == LQCD_SOLVER_GCR && (prm->gcr_nkrylov < 0 || prm->gcr_nkrylov > 64))
    return set_error(LQCD_ERR_ARG, "gcr_nkrylov must be in 0..64");
  if (prm->schur != LQCD_SCHUR_ASYM && prm->schur != LQCD_SCHUR_SYM)
    return set_error(LQCD_ERR_ARG, "bad schur %d", prm->schur);
  if (prm->outer != LQCD_F64 && prm->outer != LQCD_DF64)
    return set_error(LQCD_ERR_ARG, "outer precision must be LQCD_F64 or LQCD_DF64");
  if (!plain_cg(prm) && !(prm->delta > 0.0 && prm->delta < 1.0))
    return set_error(LQCD_ERR_ARG, "delta must be in (0, 1)");
  if (!c->have_gauge) return set_error(LQCD_ERR_STATE, "no gauge field loaded");
  if (!c->have_kappa) return set_error(LQCD_ERR_STATE, "kappa not set (call lqcd_clover)");
  const int recon_lo = (prm->inner_recon == 18 ? 18 : prm->inner_recon == 8 ? 8 : 12);
  if (prec_half(prm->inner) && recon_lo == 18)
    return set_error(LQCD_ERR_ARG, "FP16/BF16 inner solves need 12- or 8-real links");
  if (recon_lo == 8 && prm->inner != LQCD_F32 && prm->inner != LQCD_F16)
    return set_error(LQCD_ERR_ARG, "8-real inner links need an FP32 or FP16 inner solve");
  return LQCD_OK;
}

lqcd_status job_prepare(SolveJob &J) {
  NvtxRange nv("lqcd solve: stage and even-odd source");
  lqcd_ctx *c = J.c;
  const lqcd_solve_params *prm = &J.prm;
  J.t0 = std::chrono::steady_clock::now();
  J.inf = J.inf ? J.inf : &J.local;
  lqcd_solve_info *inf = J.inf;
  std::memset(inf, 0, sizeof(*inf));
  const int n = prm->nrhs;
  inf->nrhs = n;
  J.nd = (size_t)n * c->V * 24;
  SolveBufs &B = J.B;
  if (dev_malloc((void **)&B.sc, sizeof(SolverScalars) * n) != cudaSuccess ||
      dev_malloc((void **)&B.fac, sizeof(double) * 3 * n) != cudaSuccess ||
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
  const double *db = J.b;
  const double *dx0 = J.x;
  J.dx = J.x;
  if (!J.on_device) {
    double *d0, *d1;
    LQ_TRY(staging(c, 0, J.nd, &d0));
    LQ_TRY(staging(c, 1, J.nd, &d1));
    LQ_CU(cudaMemcpyAsync(d0, J.b, J.nd * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    if (prm->use_x0) LQ_CU(cudaMemcpyAsync(d1, J.x, J.nd * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    db = d0;
    dx0 = d1;
    J.dx = d1;
  }
  LQ_TRY(temp_field(c, LQCD_F64, LQCD_FULL, n, 10, &J.bf));
  LQ_TRY(temp_field(c, LQCD_F64, LQCD_FULL, n, 11, &J.xf));
  LQ_TRY(temp_field(c, LQCD_F64, LQCD_ODD, n, 12, &J.bhat));
  LQ_TRY(temp_field(c, LQCD_F64, LQCD_ODD, n, 13, &J.r64));
  LQ_TRY(temp_field(c, LQCD_F64, LQCD_EVEN, n, 14, &J.tmpe));
  for (int p = 0; p < 2; p++)
    LQ_CU(pack_spinor(LQCD_F64, c->geom, p, db, n, J.bf->data[p], nullptr, J.bf->rhs_words(), c->stream));
  if (prm->use_x0)
    LQ_CU(pack_spinor(LQCD_F64, c->geom, 1, dx0, n, J.xf->data[1], nullptr, J.xf->rhs_words(), c->stream));
  else
    LQ_CU(cudaMemsetAsync(J.xf->data[1], 0, (size_t)J.xf->rhs_words() * 16 * n, c->stream));
  Work &W = J.W;
  W.c = c;
  W.nrhs = n;
  W.recon64 = prm->recon == 12 ? 12 : 18;
  W.recon_lo = (prm->inner_recon == 18 ? 18 : prm->inner_recon == 8 ? 8 : 12);
  W.lo = prm->inner;
  W.hp = prm->inner == LQCD_F64 ? LQCD_F64 : prm->inner == LQCD_DF64 ? LQCD_DF64 : prm->outer;
  W.tol = prm->tol;
  W.delta = prm->delta;
  W.max_iter = prm->max_iter;
  // check often with 16-bit storage: its inner solves can turn round quickly
  W.check_every = prm->check_every > 0 ? prm->check_every : (prec_half(prm->inner) ? 4 : 8);
  W.info = inf;
  // the two Schur forms coincide without a clover term
  W.schur = c->clover_on ? prm->schur : LQCD_SCHUR_ASYM;
  W.rscale = W.schur == LQCD_SCHUR_SYM ? std::max(1.0, c->a_bound[1]) : 1.0;
  if (W.schur == LQCD_SCHUR_SYM) {
    LQ_TRY(temp_field(c, W.hp, LQCD_ODD, n, 40, &W.t_hp));
    if (W.lo != W.hp) LQ_TRY(temp_field(c, W.lo, LQCD_ODD, n, 41, &W.t_lo));
  }
  W.bnorm.assign(n, 0.0);
  {
    std::vector<double> e(n), o(n);
    LQ_TRY(norms(c, LQCD_F64, n, J.bf->ref(0), e.data()));
    LQ_TRY(norms(c, LQCD_F64, n, J.bf->ref(1), o.data()));
    for (int k = 0; k < n; k++) W.bnorm[k] = std::sqrt(e[k] + o[k]);
  }
  for (int k = 0; k < n; k++)
    if (!(W.bnorm[k] > 0.0) || !std::isfinite(W.bnorm[k]))
      return set_error(LQCD_ERR_ARG, "right-hand side %d is zero or not finite", k);
  LQ_TRY(op_prepare(c, LQCD_F64, W.recon64, n, J.bhat->mut(1), J.bf->ref(0), J.bf->ref(1), J.tmpe->mut(0)));
  W.bhat = J.bhat;
  W.x64 = J.xf;
  W.r64 = J.r64;
  if (W.hp == LQCD_DF64) {  // the recursion's own copies in double-float
    lqcd_field *bh, *xh, *rh;
    LQ_TRY(temp_field(c, LQCD_DF64, LQCD_ODD, n, 16, &bh));
    LQ_TRY(temp_field(c, LQCD_DF64, LQCD_ODD, n, 17, &xh));
    LQ_TRY(temp_field(c, LQCD_DF64, LQCD_ODD, n, 18, &rh));
    LQ_CU(convert_spinor(LQCD_F64, LQCD_DF64, c->Vh, n, J.bhat->data[1], nullptr, J.bhat->rhs_words(), bh->data[1],
                         nullptr, bh->rhs_words(), 1.0, c->stream));
    LQ_CU(convert_spinor(LQCD_F64, LQCD_DF64, c->Vh, n, J.xf->data[1], nullptr, J.xf->rhs_words(), xh->data[1],
                         nullptr, xh->rhs_words(), 1.0, c->stream));
    W.bhat = bh;
    W.x64 = xh;
    W.r64 = rh;
  }
  return LQCD_OK;
}

lqcd_status job_finish(SolveJob &J, lqcd_status solve_status) {
  NvtxRange nv("lqcd solve: reconstruct and FP64 residual");
  lqcd_ctx *c = J.c;
  const int n = J.prm.nrhs;
  lqcd_solve_info *inf = J.inf;
  const int recon64 = J.W.recon64;
  if (J.W.hp == LQCD_DF64)
    LQ_CU(convert_spinor(LQCD_DF64, LQCD_F64, c->Vh, n, J.W.x64->data[1], nullptr, J.W.x64->rhs_words(),
                         J.xf->data[1], nullptr, J.xf->rhs_words(), 1.0, c->stream));
  // reconstruct x_e, then the FP64 full-lattice residual b - M x
  LQ_TRY(op_reconstruct(c, LQCD_F64, recon64, n, J.xf->mut(0), J.bf->ref(0), J.xf->ref(1)));
  {
    lqcd_field *rf;
    LQ_TRY(temp_field(c, LQCD_F64, LQCD_FULL, n, 15, &rf));
    MutField o[2] = {rf->mut(0), rf->mut(1)};
    FieldRef xr[2] = {J.xf->ref(0), J.xf->ref(1)};
    FieldRef zr[2] = {J.bf->ref(0), J.bf->ref(1)};
    LQ_TRY(op_M(c, LQCD_F64, recon64, 0, n, o, xr, zr, -1.0, nullptr, 0));
    std::vector<double> e(n), od(n);
    LQ_TRY(norms(c, LQCD_F64, n, rf->ref(0), e.data()));
    LQ_TRY(norms(c, LQCD_F64, n, rf->ref(1), od.data()));
    bool ok = true;
    for (int k = 0; k < n; k++) {
      const double rel = std::sqrt(e[k] + od[k]) / J.W.bnorm[k];
      if (k < 64) inf->true_resid[k] = rel;
      if (!(rel <= J.prm.tol)) ok = false;
    }
    if (solve_status == LQCD_OK && !ok)
      solve_status = set_error(LQCD_ERR_NOCONV, "true residual above tol after convergence of the iterated one");
  }
  for (int p = 0; p < 2; p++)
    LQ_CU(unpack_spinor(LQCD_F64, c->geom, p, J.xf->data[p], nullptr, J.xf->rhs_words(), n, J.dx, c->stream));
  if (!J.on_device) LQ_CU(cudaMemcpyAsync(J.x, J.dx, J.nd * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  LQ_CU(cudaStreamSynchronize(c->stream));
  inf->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - J.t0).count();
  return solve_status;
}

}  // namespace

}  // namespace lqcd

using namespace lqcd;

extern "C" lqcd_status lqcd_solve(lqcd_ctx *c, double *x, const double *b, int on_device,
                                  const lqcd_solve_params *prm, lqcd_solve_info *info) {
  LQ_TRY(check_params(c, prm));
  if (!x || !b) return set_error(LQCD_ERR_ARG, "NULL argument");
  // the call blocks, so it runs on a private non-blocking stream (the legacy
  // default stream cannot be captured into the loop graph), after waiting for
  // the work queued on the context's stream
  struct PrivateStream {
    lqcd_ctx *c;
    cudaStream_t saved, own = nullptr;
    explicit PrivateStream(lqcd_ctx *ctx) : c(ctx), saved(ctx->stream) {}
    ~PrivateStream() {
      if (own) {
        cudaStreamSynchronize(own);
        c->stream = saved;
        cudaStreamDestroy(own);
      }
    }
  } ps(c);
  LQ_CU(cudaStreamSynchronize(c->stream));
  LQ_CU(cudaStreamCreateWithFlags(&ps.own, cudaStreamNonBlocking));
  c->stream = ps.own;
  SolveJob J;
  J.c = c;
  J.x = x;
  J.b = b;
  J.on_device = on_device;
  J.prm = *prm;
  J.inf = info;
  LQ_TRY(job_prepare(J));
  const lqcd_status st = prm->solver == LQCD_SOLVER_GCR
                             ? gcr(J.W, !plain_cg(prm), prm->gcr_nkrylov > 0 ? prm->gcr_nkrylov : 8)
                         : prm->solver == LQCD_SOLVER_BICGSTAB ? bicgstab(J.W, !plain_cg(prm))
                         : plain_cg(prm)                      ? cgls_plain(J.W, J.B)
                                                              : cgls_mixed(J.W, J.B);
  return job_finish(J, st);
}

// Several lattices at once: every lattice runs on its own stream, and the
// inner loops of all of them are one CUDA graph -- one conditional WHILE node
// per lattice, running on the GPU until that lattice needs a reliable update
// -- launched once per update cycle; the graph is rebuilt when a lattice has
// finished.
extern "C" lqcd_status lqcd_solve_batch(lqcd_ctx *const *ctxs, int nctx, double *const *x, const double *const *b,
                                        int on_device, const lqcd_solve_params *prm, lqcd_solve_info *infos) {
  if (!ctxs || !x || !b || !prm) return set_error(LQCD_ERR_ARG, "NULL argument");
  if (nctx < 1 || nctx > 256) return set_error(LQCD_ERR_ARG, "nctx must be in 1..256");
  if (plain_cg(prm)) return set_error(LQCD_ERR_ARG, "batched solves run the mixed-precision recursion");
  if (prm->solver != LQCD_SOLVER_CGLS) return set_error(LQCD_ERR_ARG, "batched solves run CGLS");
  for (int i = 0; i < nctx; i++) {
    LQ_TRY(check_params(ctxs[i], prm));
    if (!x[i] || !b[i]) return set_error(LQCD_ERR_ARG, "NULL buffer for lattice %d", i);
    for (int j = 0; j < i; j++)
      if (ctxs[j] == ctxs[i]) return set_error(LQCD_ERR_ARG, "lattice %d repeats a context", i);
  }
  // private non-blocking streams for the duration of the call
  std::vector<cudaStream_t> saved(nctx), own(nctx, nullptr);
  cudaStream_t root = nullptr;
  auto cleanup = [&]() {
    for (int i = 0; i < nctx; i++) {
      if (own[i]) {
        cudaStreamSynchronize(own[i]);
        ctxs[i]->stream = saved[i];
        cudaStreamDestroy(own[i]);
      }
    }
    if (root) cudaStreamDestroy(root);
  };
  struct Guard {
    std::function<void()> f;
    ~Guard() { f(); }
  } guard{cleanup};
  LQ_CU(cudaStreamCreateWithFlags(&root, cudaStreamNonBlocking));
  for (int i = 0; i < nctx; i++) {
    LQ_CU(cudaStreamSynchronize(ctxs[i]->stream));
    saved[i] = ctxs[i]->stream;
    LQ_CU(cudaStreamCreateWithFlags(&own[i], cudaStreamNonBlocking));
    ctxs[i]->stream = own[i];
  }
  std::vector<std::unique_ptr<SolveJob>> jobs(nctx);
  std::vector<std::unique_ptr<MixedCG>> cgs(nctx);
  for (int i = 0; i < nctx; i++) {
    jobs[i].reset(new SolveJob());
    SolveJob &J = *jobs[i];
    J.c = ctxs[i];
    J.x = x[i];
    J.b = b[i];
    J.on_device = on_device;
    J.prm = *prm;
    J.inf = infos ? &infos[i] : nullptr;
    LQ_TRY(job_prepare(J));
    cgs[i].reset(new MixedCG(J.W, J.B));
    LQ_TRY(cgs[i]->init());
  }
  std::vector<MixedCG *> all;
  for (auto &m : cgs) all.push_back(m.get());
  LQ_TRY(run_mixed(all, root, prm->max_iter));
  lqcd_status result = LQCD_OK;
  for (int i = 0; i < nctx; i++) {
    jobs[i]->inf->iters = cgs[i]->it;
    const lqcd_status st =
        cgs[i]->done ? LQCD_OK : set_error(LQCD_ERR_NOCONV, "lattice %d did not converge in %d iterations", i,
                                           prm->max_iter);
    const lqcd_status fs = job_finish(*jobs[i], st);
    if (fs != LQCD_OK && result == LQCD_OK) result = fs;
  }
  return result;
}
