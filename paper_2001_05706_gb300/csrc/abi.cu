// The C ABI: argument checking, context and field lifetime, gauge and
// clover set-up, and operator application on canonical arrays and on
// device-resident fields.  Declarations and their contracts: include/lqcd.h.
#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>

#include "internal.h"

namespace lqcd {

static thread_local char g_err[512] = "";

lqcd_status set_error(lqcd_status s, const char *fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return s;
}

// Every device allocation of the library goes through dev_malloc.  For
// failure-injection tests, LQCD_FAULT_ALLOC_AFTER=N makes every allocation
// after the N-th one (counted from the first use of this variable) fail as if
// the device were out of memory; nothing touches the GPU.
static long g_fault_after = -2;  // -2: not read yet, -1: no fault injection
static long g_alloc_count = 0;

cudaError_t dev_malloc(void **p, size_t bytes) {
  if (g_fault_after == -2) {
    const char *e = std::getenv("LQCD_FAULT_ALLOC_AFTER");
    g_fault_after = e ? std::atol(e) : -1;
  }
  if (g_fault_after >= 0 && ++g_alloc_count > g_fault_after) {
    *p = nullptr;
    return cudaErrorMemoryAllocation;
  }
  return cudaMalloc(p, bytes);
}

static lqcd_status alloc_dev(void **p, size_t bytes, const char *what) {
  if (dev_malloc(p, bytes) != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return set_error(LQCD_ERR_OOM, "cannot allocate %zu bytes for %s", bytes, what);
  }
  return LQCD_OK;
}

static void free_links(lqcd_ctx *c) {
  for (auto &kv : c->links) cudaFree(kv.second);
  c->links.clear();
}

static void free_clover(lqcd_ctx *c) {
  for (int p = 0; p < 5; p++) {
    if (c->clov[p].alloc) cudaFree(c->clov[p].alloc);
    c->clov[p] = CloverStore{};
  }
  c->clover_on = false;
}

static lqcd_status check_ctx(const lqcd_ctx *c) {
  if (!c) return set_error(LQCD_ERR_ARG, "context is NULL");
  return LQCD_OK;
}

// device staging buffer `slot` of at least n doubles
lqcd_status staging(lqcd_ctx *c, int slot, size_t n, double **out) {
  if (c->canon_n[slot] < n) {
    if (c->canon[slot]) {
      LQ_CU(cudaStreamSynchronize(c->stream));
      cudaFree(c->canon[slot]);
      c->canon[slot] = nullptr;
      c->canon_n[slot] = 0;
    }
    LQ_TRY(alloc_dev((void **)&c->canon[slot], n * sizeof(double), "canonical staging"));
    c->canon_n[slot] = n;
  }
  *out = c->canon[slot];
  return LQCD_OK;
}

// temporary field cached in the context: (prec, subset, nrhs, slot)
lqcd_status temp_field(lqcd_ctx *c, lqcd_prec prec, lqcd_subset subset, int nrhs, int slot, lqcd_field **out) {
  const long key = (((long)slot * 8 + (long)subset) * 8 + (long)prec) * 8192 + nrhs;
  auto it = c->temps.find(key);
  if (it != c->temps.end()) {
    *out = it->second;
    return LQCD_OK;
  }
  LQ_TRY(lqcd_field_create(c, prec, subset, nrhs, out));
  c->temps[key] = *out;
  return LQCD_OK;
}

}  // namespace lqcd

using namespace lqcd;

extern "C" {

const char *lqcd_last_error(void) { return g_err; }

lqcd_status lqcd_create(lqcd_ctx **ctx, const int dims[4], int t_antiperiodic, void *cuda_stream) {
  if (!ctx || !dims) return set_error(LQCD_ERR_ARG, "NULL argument");
  *ctx = nullptr;
  for (int mu = 0; mu < 4; mu++)
    if (dims[mu] < 2 || dims[mu] % 2 != 0 || dims[mu] > (1 << 20))
      return set_error(LQCD_ERR_ARG, "dims[%d] = %d: every extent must be even and >= 2", mu, dims[mu]);
  long V = (long)dims[0] * dims[1] * dims[2] * dims[3];
  if (V > (1L << 34)) return set_error(LQCD_ERR_ARG, "lattice too large");
  lqcd_ctx *c = new lqcd_ctx();
  for (int mu = 0; mu < 4; mu++) c->dims[mu] = dims[mu];
  c->tbc = t_antiperiodic ? 1 : 0;
  c->stream = (cudaStream_t)cuda_stream;
  c->V = V;
  c->Vh = V / 2;
  Geom &g = c->geom;
  for (int mu = 0; mu < 4; mu++) g.L[mu] = dims[mu];
  g.L0h = dims[0] / 2;
  g.Vh = c->Vh;
  g.stride[0] = 0;
  g.stride[1] = g.L0h;
  g.stride[2] = (long)g.L0h * dims[1];
  g.stride[3] = (long)g.L0h * dims[1] * dims[2];
  g.tbc = c->tbc;
  lqcd_status s = LQCD_OK;
  if ((s = alloc_dev((void **)&c->counter, 64 * sizeof(unsigned), "reduction counter")) != LQCD_OK ||
      (s = alloc_dev((void **)&c->results, 1024 * sizeof(double), "reduction results")) != LQCD_OK) {
    lqcd_destroy(c);
    return s;
  }
  if (cudaMemsetAsync(c->counter, 0, 64 * sizeof(unsigned), c->stream) != cudaSuccess ||
      cudaMallocHost(&c->h_results, 1024 * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    lqcd_destroy(c);
    return set_error(LQCD_ERR_CUDA, "context set-up failed");
  }
  if ((s = ensure_partials(c, 1)) != LQCD_OK) {
    lqcd_destroy(c);
    return s;
  }
  *ctx = c;
  return LQCD_OK;
}

lqcd_status lqcd_destroy(lqcd_ctx *c) {
  if (!c) return LQCD_OK;
  cudaStreamSynchronize(c->stream);
  free_links(c);
  free_clover(c);
  for (auto &kv : c->temps) {
    cudaFree(kv.second->alloc);
    if (kv.second->scale_alloc) cudaFree(kv.second->scale_alloc);
    delete kv.second;
  }
  overlap_free(c);
  if (c->U64) cudaFree(c->U64);
  if (c->partials) cudaFree(c->partials);
  if (c->counter) cudaFree(c->counter);
  if (c->results) cudaFree(c->results);
  if (c->h_results) cudaFreeHost(c->h_results);
  for (int k = 0; k < 2; k++)
    if (c->canon[k]) cudaFree(c->canon[k]);
  for (int k = 0; k < 2; k++) {
    if (c->copy_stream[k]) cudaStreamDestroy(c->copy_stream[k]);
    for (cudaEvent_t &e : c->chunk_event[k])
      if (e) cudaEventDestroy(e);
  }
  cudaGetLastError();
  delete c;
  return LQCD_OK;
}

lqcd_status lqcd_set_stream(lqcd_ctx *c, void *cuda_stream) {
  LQ_TRY(check_ctx(c));
  LQ_CU(cudaStreamSynchronize(c->stream));
  c->stream = (cudaStream_t)cuda_stream;
  return LQCD_OK;
}

lqcd_status lqcd_synchronize(lqcd_ctx *c) {
  LQ_TRY(check_ctx(c));
  LQ_CU(cudaStreamSynchronize(c->stream));
  return LQCD_OK;
}

lqcd_status lqcd_load_gauge(lqcd_ctx *c, const double *U, int on_device) {
  LQ_TRY(check_ctx(c));
  if (!U) return set_error(LQCD_ERR_ARG, "U is NULL");
  const size_t n = (size_t)c->V * 4 * 18;
  if (!c->U64) LQ_TRY(alloc_dev((void **)&c->U64, n * sizeof(double), "gauge field"));
  free_links(c);
  free_clover(c);
  overlap_free(c);
  c->have_gauge = false;
  LQ_CU(cudaMemcpyAsync(c->U64, U, n * sizeof(double), on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                        c->stream));
  unsigned long long *worst = reinterpret_cast<unsigned long long *>(c->results);
  LQ_CU(cudaMemsetAsync(worst, 0, sizeof(unsigned long long), c->stream));
  LQ_CU(su3_check(c->U64, c->V * 4, worst, c->stream));
  unsigned long long hw = 0;
  LQ_CU(cudaMemcpyAsync(c->h_results, worst, sizeof(hw), cudaMemcpyDeviceToHost, c->stream));
  LQ_CU(cudaStreamSynchronize(c->stream));
  std::memcpy(&hw, c->h_results, sizeof(hw));
  double w;
  std::memcpy(&w, &hw, sizeof(w));
  if (!(w <= 1e-10))
    return set_error(LQCD_ERR_NOT_SU3, "links are not SU(3): max deviation %.3e (|U U^dag - 1|, |det U - 1|)", w);
  c->have_gauge = true;
  return LQCD_OK;
}

lqcd_status lqcd_clover(lqcd_ctx *c, double kappa, double c_sw) {
  LQ_TRY(check_ctx(c));
  if (!c->have_gauge) return set_error(LQCD_ERR_STATE, "no gauge field loaded");
  if (!(kappa == kappa) || !(c_sw == c_sw)) return set_error(LQCD_ERR_ARG, "kappa or c_sw is NaN");
  free_clover(c);
  c->a_bound[0] = c->a_bound[1] = 1.0;
  c->kappa = kappa;
  c->csw = c_sw;
  c->have_kappa = true;
  if (c_sw == 0.0) return LQCD_OK;
  CloverStore &m = c->clov[LQCD_F64];
  const size_t nb = clover_bytes(LQCD_F64, c->Vh);
  char *p = nullptr;
  LQ_TRY(alloc_dev((void **)&p, 4 * nb, "clover term"));
  m.alloc = p;
  double *A[2], *Ai[2];
  for (int q = 0; q < 2; q++) {
    m.A[q] = p + (2 * q) * nb;
    m.Ainv[q] = p + (2 * q + 1) * nb;
    A[q] = (double *)m.A[q];
    Ai[q] = (double *)m.Ainv[q];
  }
  // results[0]: the singular flag; results[1], results[2]: the per-parity norm bounds
  int *sing = reinterpret_cast<int *>(c->results);
  unsigned long long *bound = reinterpret_cast<unsigned long long *>(c->results + 1);
  LQ_CU(cudaMemsetAsync(c->results, 0, 3 * sizeof(double), c->stream));
  LQ_CU(clover_build(c->geom, c->U64, kappa, c_sw, A, Ai, sing, bound, c->stream));
  LQ_CU(cudaMemcpyAsync(c->h_results, c->results, 3 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  LQ_CU(cudaStreamSynchronize(c->stream));
  int hs = 0;
  std::memcpy(&hs, c->h_results, sizeof(int));
  for (int q = 0; q < 2; q++) {
    unsigned long long bits;
    std::memcpy(&bits, c->h_results + 1 + q, sizeof(bits));
    std::memcpy(&c->a_bound[q], &bits, sizeof(double));
  }
  c->clover_on = true;
  if (hs) {
    free_clover(c);
    return set_error(LQCD_ERR_SINGULAR, "a clover block has a zero pivot");
  }
  return LQCD_OK;
}

lqcd_status lqcd_set_rho(lqcd_ctx *c, double rho) {
  LQ_TRY(check_ctx(c));
  if (!(rho == rho)) return set_error(LQCD_ERR_ARG, "rho is NaN");
  c->rho = rho;
  c->have_rho = true;
  return LQCD_OK;
}

// ---- fields -------------------------------------------------------------

lqcd_status lqcd_field_create(lqcd_ctx *c, lqcd_prec prec, lqcd_subset subset, int nrhs, lqcd_field **field) {
  LQ_TRY(check_ctx(c));
  if (!field) return set_error(LQCD_ERR_ARG, "field is NULL");
  *field = nullptr;
  if ((int)prec < 0 || (int)prec > 4) return set_error(LQCD_ERR_ARG, "bad precision %d", (int)prec);
  if ((int)subset < 0 || (int)subset > 2) return set_error(LQCD_ERR_ARG, "bad subset %d", (int)subset);
  if (nrhs < 1 || nrhs > 4096) return set_error(LQCD_ERR_ARG, "nrhs must be in 1..4096");
  lqcd_field *f = new lqcd_field();
  f->ctx = c;
  f->prec = prec;
  f->subset = subset;
  f->nrhs = nrhs;
  f->Vh = c->Vh;
  const int np = subset == LQCD_FULL ? 2 : 1;
  const size_t per = (size_t)f->rhs_words() * 16 * nrhs;
  lqcd_status s = alloc_dev(&f->alloc, per * np, "spinor field");
  if (s != LQCD_OK) {
    delete f;
    return s;
  }
  const size_t sper = prec_half(prec) ? sizeof(float) * c->Vh * nrhs : 0;
  if (sper) {
    s = alloc_dev((void **)&f->scale_alloc, sper * np, "spinor scales");
    if (s != LQCD_OK) {
      cudaFree(f->alloc);
      delete f;
      return s;
    }
  }
  int k = 0;
  for (int p = 0; p < 2; p++) {
    if (f->has(p)) {
      f->data[p] = (char *)f->alloc + per * k;
      f->scale[p] = sper ? (float *)((char *)f->scale_alloc + sper * k) : nullptr;
      k++;
    }
  }
  // zero-filled on the context's stream (ordered before any use on it)
  cudaError_t e = cudaMemsetAsync(f->alloc, 0, per * np, c->stream);
  if (e == cudaSuccess && sper) e = cudaMemsetAsync(f->scale_alloc, 0, sper * np, c->stream);
  if (e != cudaSuccess) {
    lqcd_field_destroy(f);
    return set_error(LQCD_ERR_CUDA, "zeroing a new field failed: %s", cudaGetErrorString(e));
  }
  *field = f;
  return LQCD_OK;
}

lqcd_status lqcd_field_destroy(lqcd_field *f) {
  if (!f) return LQCD_OK;
  cudaStreamSynchronize(f->ctx->stream);
  cudaFree(f->alloc);
  if (f->scale_alloc) cudaFree(f->scale_alloc);
  delete f;
  return LQCD_OK;
}

static lqcd_status check_field(lqcd_ctx *c, const lqcd_field *f) {
  if (!f) return set_error(LQCD_ERR_ARG, "field is NULL");
  if (f->ctx != c) return set_error(LQCD_ERR_ARG, "field belongs to another context");
  return LQCD_OK;
}

static lqcd_status import_canon(lqcd_ctx *c, lqcd_field *f, const double *dcanon) {
  for (int p = 0; p < 2; p++)
    if (f->has(p)) LQ_CU(pack_spinor(f->prec, c->geom, p, dcanon, f->nrhs, f->data[p], f->scale[p], f->rhs_words(), c->stream));
  return LQCD_OK;
}

static lqcd_status export_canon(lqcd_ctx *c, const lqcd_field *f, double *dcanon) {
  for (int p = 0; p < 2; p++)
    if (f->has(p))
      LQ_CU(unpack_spinor(f->prec, c->geom, p, f->data[p], f->scale[p], f->rhs_words(), f->nrhs, dcanon, c->stream));
  return LQCD_OK;
}

lqcd_status lqcd_field_import(lqcd_ctx *c, lqcd_field *f, const double *canon, int on_device) {
  LQ_TRY(check_ctx(c));
  LQ_TRY(check_field(c, f));
  if (!canon) return set_error(LQCD_ERR_ARG, "canon is NULL");
  const size_t n = (size_t)f->nrhs * c->V * 24;
  const double *src = canon;
  if (!on_device) {
    double *d;
    LQ_TRY(staging(c, 0, n, &d));
    LQ_CU(cudaMemcpyAsync(d, canon, n * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    src = d;
  }
  LQ_TRY(import_canon(c, f, src));
  if (!on_device) LQ_CU(cudaStreamSynchronize(c->stream));
  return LQCD_OK;
}

lqcd_status lqcd_field_export(lqcd_ctx *c, const lqcd_field *f, double *canon, int on_device) {
  LQ_TRY(check_ctx(c));
  LQ_TRY(check_field(c, f));
  if (!canon) return set_error(LQCD_ERR_ARG, "canon is NULL");
  const size_t n = (size_t)f->nrhs * c->V * 24;
  if (on_device) return export_canon(c, f, canon);
  double *d;
  LQ_TRY(staging(c, 1, n, &d));
  // unwritten sites keep the caller's values: stage them first
  LQ_CU(cudaMemcpyAsync(d, canon, n * sizeof(double), cudaMemcpyHostToDevice, c->stream));
  LQ_TRY(export_canon(c, f, d));
  LQ_CU(cudaMemcpyAsync(canon, d, n * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  LQ_CU(cudaStreamSynchronize(c->stream));
  return LQCD_OK;
}

static const FieldRef kNoField{nullptr, nullptr, 0};

static lqcd_status apply_fields(lqcd_ctx *c, lqcd_op op, int recon, lqcd_field *out, const lqcd_field *in) {
  const lqcd_prec prec = out->prec;
  const int nrhs = out->nrhs;
  auto need = [&](bool ok, const char *what) -> lqcd_status {
    return ok ? LQCD_OK : set_error(LQCD_ERR_ARG, "op %d: %s", (int)op, what);
  };
  switch (op) {
    case LQCD_OP_MHAT:
    case LQCD_OP_MHAT_DAG:
    case LQCD_OP_MHAT_NORMAL: {
      LQ_TRY(need(in->has(1) && out->has(1), "needs odd-parity input and output"));
      lqcd_field *y;
      LQ_TRY(temp_field(c, prec, LQCD_EVEN, nrhs, 0, &y));
      if (op == LQCD_OP_MHAT_NORMAL) {
        lqcd_field *t;
        LQ_TRY(temp_field(c, prec, LQCD_ODD, nrhs, 1, &t));
        LQ_TRY(op_mhat(c, prec, recon, 0, nrhs, t->mut(1), in->ref(1), y->mut(0), kNoField, 0.0, nullptr, 0));
        return op_mhat(c, prec, recon, 1, nrhs, out->mut(1), t->ref(1), y->mut(0), kNoField, 0.0, nullptr, 0);
      }
      return op_mhat(c, prec, recon, op == LQCD_OP_MHAT_DAG, nrhs, out->mut(1), in->ref(1), y->mut(0), kNoField, 0.0,
                     nullptr, 0);
    }
    case LQCD_OP_MHAT_SYM:
    case LQCD_OP_MHAT_SYM_DAG: {
      LQ_TRY(need(in->has(1) && out->has(1), "needs odd-parity input and output"));
      lqcd_field *y, *t;
      LQ_TRY(temp_field(c, prec, LQCD_EVEN, nrhs, 0, &y));
      LQ_TRY(temp_field(c, prec, LQCD_ODD, nrhs, 1, &t));
      return op_mhat_sym(c, prec, recon, op == LQCD_OP_MHAT_SYM_DAG, nrhs, out->mut(1), in->ref(1), y->mut(0),
                         t->mut(1), nullptr, 0);
    }
    case LQCD_OP_K2A:
      LQ_TRY(need(in->has(1) && out->has(0), "needs odd input and even output"));
      return op_k2a(c, prec, recon, 0, nrhs, out->mut(0), in->ref(1));
    case LQCD_OP_HOP_EO:
    case LQCD_OP_HOP_OE: {
      const int po = op == LQCD_OP_HOP_EO ? 0 : 1;
      LQ_TRY(need(in->has(1 - po) && out->has(po), "parity mismatch"));
      return run_dslash(c, prec, recon, MODE_HOP, po, nrhs, out->mut(po), in->ref(1 - po), kNoField, kNoField, 0.0,
                        1.0, 0.0, 0, 0, 0, nullptr, 0);
    }
    case LQCD_OP_M:
    case LQCD_OP_M_DAG: {
      LQ_TRY(need(in->subset == LQCD_FULL && out->subset == LQCD_FULL, "needs full-lattice fields"));
      MutField o[2] = {out->mut(0), out->mut(1)};
      FieldRef x[2] = {in->ref(0), in->ref(1)};
      FieldRef z[2] = {kNoField, kNoField};
      return op_M(c, prec, recon, op == LQCD_OP_M_DAG, nrhs, o, x, z, 0.0, nullptr, 0);
    }
    case LQCD_OP_HW: {
      LQ_TRY(need(in->subset == LQCD_FULL && out->subset == LQCD_FULL, "needs full-lattice fields"));
      MutField o[2] = {out->mut(0), out->mut(1)};
      FieldRef x[2] = {in->ref(0), in->ref(1)};
      return op_hw(c, prec, recon, nrhs, o, x, nullptr, 0);
    }
  }
  return set_error(LQCD_ERR_ARG, "unknown op %d", (int)op);
}

lqcd_status lqcd_apply(lqcd_ctx *c, lqcd_op op, lqcd_recon recon, lqcd_field *out, const lqcd_field *in) {
  LQ_TRY(check_ctx(c));
  LQ_TRY(check_field(c, out));
  LQ_TRY(check_field(c, in));
  if (out == in) return set_error(LQCD_ERR_ARG, "out and in must be different fields");
  if (out->prec != in->prec || out->nrhs != in->nrhs)
    return set_error(LQCD_ERR_ARG, "out and in must have the same precision and nrhs");
  return apply_fields(c, op, (int)recon, out, in);
}

lqcd_status lqcd_apply_schur(lqcd_ctx *c, lqcd_recon recon, int dagger, lqcd_field *out, const lqcd_field *x_odd,
                             const lqcd_field *y_even) {
  LQ_TRY(check_ctx(c));
  LQ_TRY(check_field(c, out));
  LQ_TRY(check_field(c, x_odd));
  LQ_TRY(check_field(c, y_even));
  if (!out->has(1) || !x_odd->has(1) || !y_even->has(0))
    return set_error(LQCD_ERR_ARG, "needs odd output, odd x and even y");
  if (out->prec != x_odd->prec || out->prec != y_even->prec || out->nrhs != x_odd->nrhs || out->nrhs != y_even->nrhs)
    return set_error(LQCD_ERR_ARG, "fields must share precision and nrhs");
  if (out == x_odd) return set_error(LQCD_ERR_ARG, "out and x must be different fields");
  return op_k2b(c, out->prec, (int)recon, dagger ? 1 : 0, out->nrhs, out->mut(1), x_odd->ref(1), y_even->ref(0),
                kNoField, 0.0, nullptr, 0);
}

lqcd_status lqcd_field_norm2(lqcd_ctx *c, const lqcd_field *f, double *result) {
  LQ_TRY(check_ctx(c));
  LQ_TRY(check_field(c, f));
  if (!result) return set_error(LQCD_ERR_ARG, "result is NULL");
  LQ_TRY(ensure_partials(c, f->nrhs));
  double total = 0.0;
  for (int p = 0; p < 2; p++) {
    if (!f->has(p)) continue;
    if (f->nrhs > 256) return set_error(LQCD_ERR_ARG, "norm2 supports up to 256 right-hand sides");
    LQ_CU(blas_norm2(f->prec, c->Vh, f->nrhs, f->ref(p), c->partials, c->results, 1, c->stream));
    LQ_CU(cudaMemcpyAsync(c->h_results, c->results, sizeof(double) * f->nrhs, cudaMemcpyDeviceToHost, c->stream));
    LQ_CU(cudaStreamSynchronize(c->stream));
    for (int k = 0; k < f->nrhs; k++) total += c->h_results[k];
  }
  *result = total;
  return LQCD_OK;
}

}  // extern "C"

namespace {

// Mhat on host canonical arrays, pipelined over chunks of whole time slices
// (contiguous in the canonical t-slowest order): chunk copies in on one copy
// stream, out on another, while the context's stream packs the odd sites of
// each arrived chunk, runs K2a on a chunk once its neighbour chunks are in,
// K2b once K2a has covered its neighbours, and unpacks it.  Chunks arrive in
// the order last, 0, 1, ..., so the periodic wrap is available early; the
// host link carries both directions at once.
lqcd_status mhat_host_pipelined(lqcd_ctx *c, double *out, const double *in, int nrhs, lqcd_prec prec, int recon,
                                int nch) {
  NvtxRange nv("lqcd Mhat on host buffers (pipelined)");
  const size_t n = (size_t)nrhs * c->V * 24;
  double *din, *dout;
  LQ_TRY(staging(c, 0, n, &din));
  LQ_TRY(staging(c, 1, n, &dout));
  lqcd_field *fin, *fy, *fout;
  LQ_TRY(temp_field(c, prec, LQCD_ODD, nrhs, 2, &fin));
  LQ_TRY(temp_field(c, prec, LQCD_EVEN, nrhs, 0, &fy));
  LQ_TRY(temp_field(c, prec, LQCD_ODD, nrhs, 3, &fout));
  for (int k = 0; k < 2; k++) {
    if (!c->copy_stream[k]) LQ_CU(cudaStreamCreateWithFlags(&c->copy_stream[k], cudaStreamNonBlocking));
    for (int j = 0; j < nch; j++)
      if (!c->chunk_event[k][j]) LQ_CU(cudaEventCreateWithFlags(&c->chunk_event[k][j], cudaEventDisableTiming));
  }
  cudaStream_t sin = c->copy_stream[0], sout = c->copy_stream[1];
  // whatever happens below, the call returns only once no copy touches the
  // caller's host buffers any more
  struct Drain {
    cudaStream_t a, b, d;
    ~Drain() {
      cudaStreamSynchronize(a);
      cudaStreamSynchronize(b);
      cudaStreamSynchronize(d);
    }
  } drain{sin, sout, c->stream};
  const long slab = c->V / nch;  // sites per chunk
  const long hs = slab / 2;      // sites per parity per chunk
  const size_t bytes = (size_t)slab * 24 * sizeof(double);
  // the copies may not start before earlier work on the context's stream is done with the staging buffers
  LQ_CU(cudaEventRecord(c->chunk_event[1][0], c->stream));
  LQ_CU(cudaStreamWaitEvent(sin, c->chunk_event[1][0], 0));
  LQ_CU(cudaStreamWaitEvent(sout, c->chunk_event[1][0], 0));
  auto order = [&](int i) { return i == 0 ? nch - 1 : i - 1; };
  for (int i = 0; i < nch; i++) {
    const int ch = order(i);
    for (int r = 0; r < nrhs; r++) {
      const size_t off = ((size_t)r * c->V + (size_t)ch * slab) * 24;
      LQ_CU(cudaMemcpyAsync(din + off, in + off, bytes, cudaMemcpyHostToDevice, sin));
    }
    LQ_CU(cudaEventRecord(c->chunk_event[0][ch], sin));
  }
  auto k2a = [&](int ch) {
    return op_k2a(c, prec, recon, 0, nrhs, fy->mut(0), fin->ref(1), ch * hs, (ch + 1) * hs);
  };
  auto k2b_out = [&](int ch) -> lqcd_status {
    const FieldRef none{nullptr, nullptr, 0};
    LQ_TRY(op_k2b(c, prec, recon, 0, nrhs, fout->mut(1), fin->ref(1), fy->ref(0), none, 0.0, nullptr, 0, ch * hs,
                  (ch + 1) * hs));
    LQ_CU(unpack_spinor(prec, c->geom, 1, fout->data[1], fout->scale[1], fout->rhs_words(), nrhs, dout, c->stream,
                        ch * hs, (ch + 1) * hs));
    LQ_CU(zero_parity(c->geom, 0, dout, nrhs, c->stream, ch * hs, (ch + 1) * hs));
    LQ_CU(cudaEventRecord(c->chunk_event[1][ch], c->stream));
    LQ_CU(cudaStreamWaitEvent(sout, c->chunk_event[1][ch], 0));
    for (int r = 0; r < nrhs; r++) {
      const size_t off = ((size_t)r * c->V + (size_t)ch * slab) * 24;
      LQ_CU(cudaMemcpyAsync(out + off, dout + off, bytes, cudaMemcpyDeviceToHost, sout));
    }
    return LQCD_OK;
  };
  // arrival i brings chunk i-1 (i >= 1): then K2a of chunk i-2 has both
  // neighbours, and K2b of chunk i-3 has K2a on both of its neighbours
  for (int i = 0; i < nch; i++) {
    const int ch = order(i);
    LQ_CU(cudaStreamWaitEvent(c->stream, c->chunk_event[0][ch], 0));
    LQ_CU(pack_spinor(prec, c->geom, 1, din, nrhs, fin->data[1], fin->scale[1], fin->rhs_words(), c->stream, ch * hs,
                      (ch + 1) * hs));
    if (i >= 2) LQ_TRY(k2a(i - 2));
    if (i >= 4) LQ_TRY(k2b_out(i - 3));
  }
  LQ_TRY(k2a(nch - 2));
  LQ_TRY(k2a(nch - 1));
  for (int ch = std::max(1, nch - 3); ch < nch; ch++) LQ_TRY(k2b_out(ch));
  LQ_TRY(k2b_out(0));
  LQ_CU(cudaStreamSynchronize(sout));
  LQ_CU(cudaStreamSynchronize(c->stream));
  return LQCD_OK;
}

}  // namespace

extern "C" {

lqcd_status lqcd_dslash(lqcd_ctx *c, double *out, const double *in, int nrhs, lqcd_op op, lqcd_prec prec,
                        lqcd_recon recon, int on_device) {
  LQ_TRY(check_ctx(c));
  if (!out || !in) return set_error(LQCD_ERR_ARG, "NULL buffer");
  if (out == in) return set_error(LQCD_ERR_ARG, "out and in must not alias");
  if (nrhs < 1 || nrhs > 4096) return set_error(LQCD_ERR_ARG, "nrhs must be in 1..4096");
  if ((int)prec < 0 || (int)prec > 4) return set_error(LQCD_ERR_ARG, "bad precision");
  if ((int)op < 0 || (int)op > 10) return set_error(LQCD_ERR_ARG, "bad op");
  if (!c->have_gauge) return set_error(LQCD_ERR_STATE, "no gauge field loaded");
  if (!on_device && op == LQCD_OP_MHAT && c->have_kappa && !std::getenv("LQCD_NO_PIPELINE")) {
    // chunks of whole time slices, at least 4 of them, at most LQCD_HOST_CHUNKS (default 32,
    // <= 64).  Measured at 32^3x64 (ms per call): 8 chunks 3.55, 16 3.17, 32 2.92, 64 3.08
    const char *env = std::getenv("LQCD_HOST_CHUNKS");
    int nch = env ? std::max(4, std::min(64, std::atoi(env))) : 32;
    while (nch >= 4 && c->dims[3] % nch != 0) nch--;
    if (nch >= 4) return mhat_host_pipelined(c, out, in, nrhs, prec, (int)recon, nch);
  }
  const size_t n = (size_t)nrhs * c->V * 24;
  const double *din = in;
  double *dout = out;
  if (!on_device) {
    double *d0, *d1;
    LQ_TRY(staging(c, 0, n, &d0));
    LQ_TRY(staging(c, 1, n, &d1));
    LQ_CU(cudaMemcpyAsync(d0, in, n * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    din = d0;
    dout = d1;
  }
  lqcd_field *fin, *fout;
  LQ_TRY(temp_field(c, prec, LQCD_FULL, nrhs, 2, &fin));
  LQ_TRY(temp_field(c, prec, LQCD_FULL, nrhs, 3, &fout));
  LQ_TRY(import_canon(c, fin, din));
  LQ_TRY(apply_fields(c, op, (int)recon, fout, fin));
  const bool full = op == LQCD_OP_M || op == LQCD_OP_M_DAG || op == LQCD_OP_HW;
  for (int p = 0; p < 2; p++) {
    const bool written = full || (p == 0 ? (op == LQCD_OP_HOP_EO || op == LQCD_OP_K2A)
                                         : (op == LQCD_OP_MHAT || op == LQCD_OP_MHAT_DAG ||
                                            op == LQCD_OP_MHAT_NORMAL || op == LQCD_OP_HOP_OE ||
                                            op == LQCD_OP_MHAT_SYM || op == LQCD_OP_MHAT_SYM_DAG));
    if (written)
      LQ_CU(unpack_spinor(prec, c->geom, p, fout->data[p], fout->scale[p], fout->rhs_words(), nrhs, dout, c->stream));
    else
      LQ_CU(zero_parity(c->geom, p, dout, nrhs, c->stream));
  }
  if (!on_device) {
    LQ_CU(cudaMemcpyAsync(out, dout, n * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    LQ_CU(cudaStreamSynchronize(c->stream));
  }
  return LQCD_OK;
}

}  // extern "C"
