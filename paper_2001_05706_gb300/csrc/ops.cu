// Operator layer: the even-odd Wilson-clover operators built from launches
// of the generic dslash kernel, and the lazily packed link and clover forms
// they read.
#include <cstdio>
#include <cstdlib>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "internal.h"

namespace lqcd {

lqcd_status get_links(lqcd_ctx *c, lqcd_prec prec, int recon, const void **base) {
  if (!c->have_gauge) return set_error(LQCD_ERR_STATE, "no gauge field loaded");
  if (recon != 12 && recon != 18 && recon != 8) return set_error(LQCD_ERR_ARG, "recon must be 8, 12 or 18");
  if (prec_half(prec) && recon == 18) return set_error(LQCD_ERR_ARG, "FP16/BF16 links are stored in 12- or 8-real form");
  // BF16's 8-bit mantissa would store the two angles only to ~6e-3 rad
  if (recon == 8 && prec != LQCD_F32 && prec != LQCD_F16)
    return set_error(LQCD_ERR_ARG, "the 8-real form is for FP32/FP16 links");
  const int key = 100 * (int)prec + recon;
  auto it = c->links.find(key);
  if (it != c->links.end()) {
    *base = it->second;
    return LQCD_OK;
  }
  if (recon == 8) {  // the rebuild divides by 1 - |U00|^2: refuse links where it vanishes (unit links)
    unsigned long long *w = nullptr;
    if (dev_malloc((void **)&w, sizeof(*w)) != cudaSuccess) {
      cudaGetLastError();
      return set_error(LQCD_ERR_OOM, "cannot allocate a reduction word");
    }
    double dmin = 0;
    const cudaError_t e = recon8_min_det(c->U64, 4L * c->V, w, &dmin, c->stream);
    cudaFree(w);
    LQ_CU(e);
    if (!(dmin > 1e-10))
      return set_error(LQCD_ERR_ARG, "8-real links need |U00| < 1 on every link (min 1 - |U00|^2 = %.3e)", dmin);
  }
  void *p = nullptr;
  if (dev_malloc(&p, link_bytes(prec, recon, c->Vh)) != cudaSuccess) {
    cudaGetLastError();
    return set_error(LQCD_ERR_OOM, "cannot allocate packed links");
  }
  LQ_CU(pack_links(prec, c->geom, c->U64, recon, p, c->stream));
  c->links[key] = p;
  *base = p;
  return LQCD_OK;
}

lqcd_status get_clover(lqcd_ctx *c, lqcd_prec prec, CloverStore **cs) {
  if (!c->clover_on) return set_error(LQCD_ERR_STATE, "no clover term (c_sw = 0 or lqcd_clover not called)");
  CloverStore &s = c->clov[prec];
  if (!s.alloc) {
    const size_t nb = clover_bytes(prec, c->Vh);
    const size_t ns = prec_half(prec) ? sizeof(float) * c->Vh : 0;
    char *p = nullptr;
    if (dev_malloc((void **)&p, 4 * (nb + ns)) != cudaSuccess) {
      cudaGetLastError();
      return set_error(LQCD_ERR_OOM, "cannot allocate clover storage");
    }
    s.alloc = p;
    for (int q = 0; q < 2; q++) {
      s.A[q] = p + (2 * q) * nb;
      s.Ainv[q] = p + (2 * q + 1) * nb;
      if (ns) {
        s.As[q] = reinterpret_cast<float *>(p + 4 * nb + (2 * q) * ns);
        s.Ais[q] = reinterpret_cast<float *>(p + 4 * nb + (2 * q + 1) * ns);
      }
    }
    const CloverStore &m = c->clov[LQCD_F64];
    for (int q = 0; q < 2; q++) {
      LQ_CU(pack_clover(prec, c->Vh, (const double *)m.A[q], s.A[q], s.As[q], c->stream));
      LQ_CU(pack_clover(prec, c->Vh, (const double *)m.Ainv[q], s.Ainv[q], s.Ais[q], c->stream));
    }
  }
  *cs = &s;
  return LQCD_OK;
}

lqcd_status ensure_partials(lqcd_ctx *c, int nrhs) {
  // one partial per block and quantity; blocks have at least 32 threads
  const size_t need = (size_t)((c->Vh + 31) / 32 + 1) * (size_t)(nrhs < 1 ? 1 : nrhs);
  if (need <= c->partials_n) return LQCD_OK;
  if (c->partials) {
    LQ_CU(cudaStreamSynchronize(c->stream));
    cudaFree(c->partials);
    c->partials = nullptr;
  }
  if (dev_malloc((void **)&c->partials, need * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    c->partials_n = 0;
    return set_error(LQCD_ERR_OOM, "cannot allocate reduction scratch");
  }
  c->partials_n = need;
  return LQCD_OK;
}

// ---------------------------------------------------------------------------
// Autotuner for the kernel variant of a dslash launch: dslash_kernel with 1,
// 2 or 4 right-hand sides per thread (links and clover loaded once for all of
// them), or, for FP32/FP16/BF16 with several right-hand sides,
// dslash_mrhs_kernel with g warps of two right-hand sides sharing one staged
// tile of links and clover (g = 1, 2, 3, 6).  On the first launch of a given
// (precision, link form, mode, nrhs, volume) every admissible variant is timed
// with CUDA events on the context's stream and the fastest is kept, in memory
// and, if LQCD_TUNE_CACHE names a file, in that file (one line per entry).
// Re-running a launch is harmless: the kernel never writes its inputs.
// LQCD_FORCE_VARIANT (read at every launch) forces a variant wherever it is
// admissible, so tests can compare each kernel with the oracle.
// ---------------------------------------------------------------------------
using TuneKey = std::tuple<int, int, int, int, long>;
static std::map<TuneKey, int> g_tune;
static std::mutex g_tune_mu;
static bool g_tune_loaded = false;

static void tune_load() {
  g_tune_loaded = true;
  const char *path = std::getenv("LQCD_TUNE_CACHE");
  if (!path) return;
  FILE *f = std::fopen(path, "r");
  if (!f) return;
  int a, b, m, n, nr;
  long v;
  while (std::fscanf(f, "%d %d %d %d %ld %d", &a, &b, &m, &n, &v, &nr) == 6) g_tune[TuneKey(a, b, m, n, v)] = nr;
  std::fclose(f);
}

static void tune_store(const TuneKey &k, int nr) {
  const char *path = std::getenv("LQCD_TUNE_CACHE");
  if (!path) return;
  FILE *f = std::fopen(path, "a");
  if (!f) return;
  std::fprintf(f, "%d %d %d %d %ld %d\n", std::get<0>(k), std::get<1>(k), std::get<2>(k), std::get<3>(k),
               std::get<4>(k), nr);
  std::fclose(f);
}

static bool mrhs_ok(lqcd_prec prec, int mode, int nrhs) {
  if (nrhs < 2) return false;
  if (prec != LQCD_F32 && prec != LQCD_F16 && prec != LQCD_BF16) return false;
  if (mode == MODE_FOLDED_AINV) return false;
  return mode != MODE_CHEB || prec == LQCD_F32;
}

// every variant that can run this launch
static std::vector<int> variants(lqcd_prec prec, int mode, int nrhs, int recon) {
  std::vector<int> v;
  if (recon == 8) return {1};  // the 8-real form: dslash_kernel with one right-hand side per thread
  for (int nr : {1, 2, 4}) {
    if (nrhs % nr != 0) continue;
    if (nr > 1 && mode == MODE_FOLDED_AINV) continue;
    if (nr == 4 && prec == LQCD_DF64) continue;
    v.push_back(nr);
  }
  if (mrhs_ok(prec, mode, nrhs)) {
    const int pairs = (nrhs + 1) / 2;
    for (int g : {1, 2, 3, 6})
      if (g <= pairs) v.push_back(kMrhsVariant + g);
  }
  return v;
}

static int default_variant(lqcd_prec prec, int mode, int nrhs) {
  if (mrhs_ok(prec, mode, nrhs)) {
    const int pairs = (nrhs + 1) / 2;
    for (int g : {6, 3, 2, 1})
      if (pairs % g == 0) return kMrhsVariant + g;
  }
  if (mode == MODE_FOLDED_AINV) return 1;
  if (prec == LQCD_F64 || prec == LQCD_DF64) return nrhs % 2 == 0 ? 2 : 1;
  if (nrhs % 4 == 0) return 4;
  if (nrhs % 2 == 0) return 2;
  return 1;
}

static int pick_variant(lqcd_ctx *c, const DslashParams &P, lqcd_prec prec, int recon, int mode, int nrhs) {
  const std::vector<int> cand = variants(prec, mode, nrhs, recon);
  if (const char *f = std::getenv("LQCD_FORCE_VARIANT")) {
    const int v = std::atoi(f);
    for (int x : cand)
      if (x == v) return v;
  }
  if (cand.size() == 1) return cand[0];
  // keyed on the launch's site count: a launch over part of the parity (the
  // host pipeline's chunks, a domain's slices) tunes apart from a whole one
  const TuneKey key((int)prec, recon, mode, nrhs, P.h1 - P.h0);
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    if (!g_tune_loaded) tune_load();
    auto it = g_tune.find(key);
    if (it != g_tune.end()) {
      for (int x : cand)  // a cached choice outside this launch's candidates is ignored
        if (x == it->second) return x;
    }
  }
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(c->stream, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
    cudaGetLastError();
    return default_variant(prec, mode, nrhs);
  }
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    cudaGetLastError();
    return default_variant(prec, mode, nrhs);
  }
  int best = default_variant(prec, mode, nrhs);
  float best_ms = 1e30f;
  for (int v : cand) {
    if (launch_dslash_variant(prec, P, recon, mode, v, c->stream) != cudaSuccess) {
      cudaGetLastError();
      continue;
    }
    cudaEventRecord(e0, c->stream);
    for (int r = 0; r < 3; r++) launch_dslash_variant(prec, P, recon, mode, v, c->stream);
    cudaEventRecord(e1, c->stream);
    float ms = 0;
    if (cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess && ms < best_ms) {
      best_ms = ms;
      best = v;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaGetLastError();
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune[key] = best;
  tune_store(key, best);
  return best;
}

lqcd_status run_dslash(lqcd_ctx *c, lqcd_prec prec, int recon, int mode, int out_p, int nrhs, MutField out, FieldRef in,
                       FieldRef xloc, FieldRef z, double alpha, double beta, double gz, int g5_in, int g5_hop,
                       int g5_total, double *norm_result, int norm_stride, const FieldRef *zc, const double *cz,
                       long h0, long h1) {
  if (prec == LQCD_DF64 && recon != 18) return set_error(LQCD_ERR_ARG, "DF64 operators use 18-real links");
  if (prec_half(prec) && recon == 18) return set_error(LQCD_ERR_ARG, "FP16/BF16 operators use 12- or 8-real links");
  DslashParams P{};
  P.g = c->geom;
  P.h0 = h0;
  P.h1 = h1 < 0 ? c->Vh : h1;
  if (P.h0 < 0 || P.h1 > c->Vh || P.h0 >= P.h1) return set_error(LQCD_ERR_ARG, "bad site range [%ld, %ld)", h0, h1);
  P.out_parity = out_p;
  P.nrhs = nrhs;
  P.out = out.data;
  P.out_scale = out.scale;
  P.in = in;
  P.xloc = xloc;
  P.z = z;
  const bool hop = in.data != nullptr && beta != 0.0;
  if (hop) {
    const void *base = nullptr;
    LQ_TRY(get_links(c, prec, recon, &base));
    for (int mu = 0; mu < 4; mu++)
      for (int q = 0; q < 2; q++) P.links[mu][q] = link_ptr(base, prec, recon, c->Vh, mu, q);
  }
  if (mode == MODE_HOP_AINV || mode == MODE_FOLDED_AINV || mode == MODE_LOCAL_A) {
    CloverStore *cs = nullptr;
    LQ_TRY(get_clover(c, prec, &cs));
    P.cmat = cs->Ainv[out_p];
    P.cmat_scale = cs->Ais[out_p];
    P.lmat = cs->A[out_p];
    P.lmat_scale = cs->As[out_p];
  }
  P.alpha = alpha;
  P.beta = beta;
  P.gz = gz;
  P.g5_in = g5_in;
  P.g5_hop = g5_hop;
  P.g5_total = g5_total;
  if (mode == MODE_CHEB) {
    if (!zc || !cz) return set_error(LQCD_ERR_ARG, "Chebyshev step without its terms");
    for (int k = 0; k < 3; k++) {
      P.zc[k] = zc[k];
      P.cz[k] = cz[k];
    }
  }
  if (norm_result) {
    LQ_TRY(ensure_partials(c, nrhs));
    P.norm_partials = c->partials;
    P.norm_result = norm_result;
    P.norm_stride = norm_stride;
  }
#if LQCD_DEBUG_BOUNDS
  P.dbg = c->counter + 63;  // spare reduction counter, zero between launches
#endif
  const int variant = pick_variant(c, P, prec, recon, mode, nrhs);
  LQ_CU(launch_dslash_variant(prec, P, recon, mode, variant, c->stream));
#if LQCD_DEBUG_BOUNDS
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  LQ_CU(cudaStreamIsCapturing(c->stream, &cap));
  if (cap == cudaStreamCaptureStatusNone) {
    unsigned flag = 0;
    LQ_CU(cudaMemcpyAsync(&flag, P.dbg, sizeof(flag), cudaMemcpyDeviceToHost, c->stream));
    LQ_CU(cudaStreamSynchronize(c->stream));
    if (flag) {
      LQ_CU(cudaMemsetAsync(P.dbg, 0, sizeof(flag), c->stream));
      return set_error(LQCD_ERR_CUDA, "dslash gathered an out-of-range site index (mode %d, parity %d)", mode,
                       out_p);
    }
  }
#endif
  return LQCD_OK;
}

static const FieldRef kNone{nullptr, nullptr, 0};

lqcd_status op_k2a(lqcd_ctx *c, lqcd_prec prec, int recon, int dagger, int nrhs, MutField y_e, FieldRef x_o, long h0,
                   long h1) {
  if (!c->have_kappa) return set_error(LQCD_ERR_STATE, "kappa not set (call lqcd_clover)");
  const int mode = c->clover_on ? MODE_HOP_AINV : MODE_HOP;
  return run_dslash(c, prec, recon, mode, 0, nrhs, y_e, x_o, kNone, kNone, 0.0, 1.0, 0.0, dagger, 0, 0, nullptr, 0,
                    nullptr, nullptr, h0, h1);
}

lqcd_status op_k2b(lqcd_ctx *c, lqcd_prec prec, int recon, int dagger, int nrhs, MutField out_o, FieldRef x_o,
                   FieldRef y_e, FieldRef zf, double gz, double *norm_result, int norm_stride, long h0, long h1) {
  if (!c->have_kappa) return set_error(LQCD_ERR_STATE, "kappa not set (call lqcd_clover)");
  const int mode = c->clover_on ? MODE_LOCAL_A : MODE_LOCAL_IDENT;
  return run_dslash(c, prec, recon, mode, 1, nrhs, out_o, y_e, x_o, zf, 1.0, -c->kappa * c->kappa, gz, 0, dagger, 0,
                    norm_result, norm_stride, nullptr, nullptr, h0, h1);
}

lqcd_status op_mhat(lqcd_ctx *c, lqcd_prec prec, int recon, int dagger, int nrhs, MutField out_o, FieldRef x_o,
                    MutField y_e, FieldRef zf, double gz, double *norm_result, int norm_stride) {
  LQ_TRY(op_k2a(c, prec, recon, dagger, nrhs, y_e, x_o));
  return op_k2b(c, prec, recon, dagger, nrhs, out_o, x_o, y_e.ref(), zf, gz, norm_result, norm_stride);
}

lqcd_status op_ainv_odd(lqcd_ctx *c, lqcd_prec prec, int recon, int nrhs, MutField out_o, FieldRef x_o,
                        double *norm_result, int norm_stride) {
  if (!c->have_kappa) return set_error(LQCD_ERR_STATE, "kappa not set (call lqcd_clover)");
  if (!c->clover_on) return set_error(LQCD_ERR_STATE, "no clover term");
  return run_dslash(c, prec, recon, MODE_FOLDED_AINV, 1, nrhs, out_o, kNone, x_o, kNone, 1.0, 0.0, 0.0, 0, 0, 0,
                    norm_result, norm_stride);
}

// Symmetric Schur complement Mhat_s = A_oo^-1 Mhat = 1 - kappa^2 A_oo^-1 D_oe A_ee^-1 D_eo.
// Forward: K2a, then the second hop with A_oo^-1 applied to the hop sum and x_o
// added in the epilogue (same bytes as K2b: A_oo^-1 replaces A_oo).  Adjoint,
// with A Hermitian, commuting with g5, and D_eo^dag = g5 D_oe g5:
//   Mhat_s^dag = 1 - kappa^2 g5 D_oe A_ee^-1 D_eo g5 A_oo^-1,
// i.e. a site-local A_oo^-1 pass, K2a with g5 on its input, and the second
// hop with g5 on the hop sum plus x_o.  c_sw = 0: A = 1 and Mhat_s = Mhat.
lqcd_status op_mhat_sym(lqcd_ctx *c, lqcd_prec prec, int recon, int dagger, int nrhs, MutField out_o, FieldRef x_o,
                        MutField y_e, MutField t_o, double *norm_result, int norm_stride) {
  if (!c->have_kappa) return set_error(LQCD_ERR_STATE, "kappa not set (call lqcd_clover)");
  if (!c->clover_on) return op_mhat(c, prec, recon, dagger, nrhs, out_o, x_o, y_e, kNone, 0.0, norm_result, norm_stride);
  const double k2 = c->kappa * c->kappa;
  if (!dagger) {
    LQ_TRY(op_k2a(c, prec, recon, 0, nrhs, y_e, x_o));
    return run_dslash(c, prec, recon, MODE_HOP_AINV, 1, nrhs, out_o, y_e.ref(), kNone, x_o, 0.0, -k2, 1.0, 0, 0, 0,
                      norm_result, norm_stride);
  }
  LQ_TRY(op_ainv_odd(c, prec, recon, nrhs, t_o, x_o, nullptr, 0));
  LQ_TRY(op_k2a(c, prec, recon, 1, nrhs, y_e, t_o.ref()));
  return run_dslash(c, prec, recon, MODE_LOCAL_IDENT, 1, nrhs, out_o, y_e.ref(), x_o, kNone, 1.0, -k2, 0.0, 0, 1, 0,
                    norm_result, norm_stride);
}

lqcd_status op_M(lqcd_ctx *c, lqcd_prec prec, int recon, int dagger, int nrhs, MutField out[2], FieldRef x[2],
                 FieldRef zf[2], double gz, double *norm_result, int norm_stride) {
  if (!c->have_kappa) return set_error(LQCD_ERR_STATE, "kappa not set (call lqcd_clover)");
  const int mode = c->clover_on ? MODE_LOCAL_A : MODE_LOCAL_IDENT;
  for (int p = 0; p < 2; p++) {
    // M^dag = g5 M g5 = A - kappa g5 D g5 (A commutes with g5)
    LQ_TRY(run_dslash(c, prec, recon, mode, p, nrhs, out[p], x[1 - p], x[p], zf[p], 1.0, -c->kappa, gz, dagger, dagger,
                      0, norm_result ? norm_result + p : nullptr, norm_stride));
  }
  return LQCD_OK;
}

lqcd_status op_prepare(lqcd_ctx *c, lqcd_prec prec, int recon, int nrhs, MutField bhat_o, FieldRef b_e, FieldRef b_o,
                       MutField tmp_e) {
  if (!c->have_kappa) return set_error(LQCD_ERR_STATE, "kappa not set (call lqcd_clover)");
  FieldRef src = b_e;
  if (c->clover_on) {  // tmp_e = A_ee^-1 b_e (site-local: no hop)
    LQ_TRY(run_dslash(c, prec, recon, MODE_FOLDED_AINV, 0, nrhs, tmp_e, kNone, b_e, kNone, 1.0, 0.0, 0.0, 0, 0, 0,
                      nullptr, 0));
    src = tmp_e.ref();
  }
  return run_dslash(c, prec, recon, MODE_HOP, 1, nrhs, bhat_o, src, kNone, b_o, 0.0, c->kappa, 1.0, 0, 0, 0, nullptr, 0);
}

lqcd_status op_reconstruct(lqcd_ctx *c, lqcd_prec prec, int recon, int nrhs, MutField x_e, FieldRef b_e,
                           FieldRef x_o) {
  if (!c->have_kappa) return set_error(LQCD_ERR_STATE, "kappa not set (call lqcd_clover)");
  const int mode = c->clover_on ? MODE_FOLDED_AINV : MODE_LOCAL_IDENT;
  return run_dslash(c, prec, recon, mode, 0, nrhs, x_e, x_o, b_e, kNone, 1.0, c->kappa, 0.0, 0, 0, 0, nullptr, 0);
}

lqcd_status op_hw(lqcd_ctx *c, lqcd_prec prec, int recon, int nrhs, MutField out[2], FieldRef x[2], double *norm_result,
                  int norm_stride) {
  if (!c->have_rho) return set_error(LQCD_ERR_STATE, "rho not set (call lqcd_set_rho)");
  for (int p = 0; p < 2; p++)
    LQ_TRY(run_dslash(c, prec, recon, MODE_LOCAL_IDENT, p, nrhs, out[p], x[1 - p], x[p], kNone, 4.0 - c->rho, -0.5, 0.0,
                      0, 0, 1, norm_result ? norm_result + p : nullptr, norm_stride));
  return LQCD_OK;
}

lqcd_status op_hw_cheb(lqcd_ctx *c, lqcd_prec prec, int recon, int nrhs, MutField out[2], FieldRef x[2], double t,
                       const FieldRef z[3][2], const double cz[3]) {
  if (!c->have_rho) return set_error(LQCD_ERR_STATE, "rho not set (call lqcd_set_rho)");
  if (prec != LQCD_F64 && prec != LQCD_F32 && prec != LQCD_DF64)
    return set_error(LQCD_ERR_ARG, "Chebyshev step needs FP64, DF64 or FP32");
  for (int p = 0; p < 2; p++) {
    const FieldRef zp[3] = {z[0][p], z[1][p], z[2][p]};
    LQ_TRY(run_dslash(c, prec, recon, MODE_CHEB, p, nrhs, out[p], x[1 - p], x[p], kNone, t * (4.0 - c->rho),
                      -0.5 * t, 0.0, 0, 0, 1, nullptr, 0, zp, cz));
  }
  return LQCD_OK;
}

}  // namespace lqcd
