// Library-internal declarations shared by the .cu files: the context and
// field objects behind the opaque C handles, and the host-side launchers.
#pragma once
#include <cstddef>
#include <map>
#include <string>

#include <nvtx3/nvToolsExt.h>

#include "common.cuh"
#include "dslash.cuh"

namespace lqcd {

// NVTX range over a scope: the solver phases show up by name in Nsight
// Systems and can filter ncu captures (no cost without an attached tool)
struct NvtxRange {
  explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange &) = delete;
  NvtxRange &operator=(const NvtxRange &) = delete;
};

struct MutField {
  void *data;
  float *scale;
  long rhs_words;
  __host__ __device__ FieldRef ref() const { return FieldRef{data, scale, rhs_words}; }
};

// ---- layout.cu
// [h0, h1): the sites of parity p converted (h1 < 0: to the end of the parity)
cudaError_t pack_spinor(lqcd_prec prec, const Geom &g, int p, const double *canon, int nrhs, void *out, float *scale,
                        long rhs_words, cudaStream_t st, long h0 = 0, long h1 = -1);
cudaError_t unpack_spinor(lqcd_prec prec, const Geom &g, int p, const void *in, const float *scale, long rhs_words,
                          int nrhs, double *canon, cudaStream_t st, long h0 = 0, long h1 = -1);
cudaError_t zero_parity(const Geom &g, int p, double *canon, int nrhs, cudaStream_t st, long h0 = 0, long h1 = -1);
cudaError_t convert_spinor(lqcd_prec pi, lqcd_prec po, long Vh, int nrhs, const void *in, const float *is, long irw,
                           void *out, float *os, long orw, double factor, cudaStream_t st);
size_t link_bytes(lqcd_prec prec, int recon, long Vh);
cudaError_t pack_links(lqcd_prec prec, const Geom &g, const double *U, int recon, void *out, cudaStream_t st);
// min over the canonical links of 1 - |U00|^2 (the 8-real form's determinant)
cudaError_t recon8_min_det(const double *U, long nlinks, unsigned long long *dev_word, double *out, cudaStream_t st);
const void *link_ptr(const void *base, lqcd_prec prec, int recon, long Vh, int mu, int p);
cudaError_t su3_check(const double *U, long nlinks, unsigned long long *worst, cudaStream_t st);
size_t clover_bytes(lqcd_prec prec, long Vh);
cudaError_t pack_clover(lqcd_prec prec, long Vh, const double *in, void *out, float *scale, cudaStream_t st);

// ---- clover.cu
// bound[p] (as the bits of a non-negative double, max-combined): a Gershgorin
// bound of ||A|| over the sites of parity p
cudaError_t clover_build(const Geom &g, const double *U, double kappa, double csw, double *A[2], double *Ainv[2],
                         int *singular, unsigned long long *bound, cudaStream_t st);

// ---- blas.cu
long blas_blocks(long Vh);
cudaError_t blas_cg_xr(lqcd_prec px, lqcd_prec pv, long Vh, int nrhs, MutField x, FieldRef p, MutField r, FieldRef q,
                       SolverScalars *sc, int cur, double *partials, cudaStream_t st);
cudaError_t blas_cg_p(lqcd_prec pv, long Vh, int nrhs, MutField p, FieldRef s, SolverScalars *sc, int cur,
                      cudaStream_t st);
cudaError_t blas_norm2(lqcd_prec pv, long Vh, int nrhs, FieldRef v, double *partials, double *result, int stride,
                       cudaStream_t st);
cudaError_t blas_axpy(lqcd_prec py, lqcd_prec px, long Vh, int nrhs, MutField y, FieldRef x, const double *f,
                      cudaStream_t st);
cudaError_t blas_scale(lqcd_prec py, lqcd_prec px, long Vh, int nrhs, MutField y, FieldRef x, const double *f,
                       cudaStream_t st);

// ---- bicgstab.cu: building blocks of BiCGStab (complex per-RHS scalars)
struct BiScalars {
  double2 rho, rho_old, alpha, omega, beta;
  double rr;      // ||r||^2 of the last iteration
  double active;  // 1.0 while this right-hand side iterates
  double pad[3];
};
// reduction buffer: three regions of 3 doubles per right-hand side, written by
// bi_dot3 / bi_xr as (complex dot re, im, squared norm): (rhat, v), (t, s) with
// |t|^2, and (rhat, r) with |r|^2
constexpr int kBiRed = 9;
enum { BI_BETA = 0, BI_ALPHA = 1, BI_OMEGA = 2 };
cudaError_t bi_scalar(int which, BiScalars *s, const double *red, int nrhs, cudaStream_t st);
cudaError_t bi_p(lqcd_prec pv, long Vh, int nrhs, MutField p, FieldRef r, FieldRef v, const BiScalars *s,
                 cudaStream_t st);
cudaError_t bi_s(lqcd_prec pv, long Vh, int nrhs, MutField sv, FieldRef r, FieldRef v, const BiScalars *s,
                 cudaStream_t st);
// red[3k..3k+2] = (a_k^H b_k) re, im, |a_k|^2  (red may be any of the slots)
cudaError_t bi_dot3(lqcd_prec pv, long Vh, int nrhs, FieldRef a, FieldRef b, double *partials, double *red,
                    cudaStream_t st);
// GCR: y_k += cf_k x_k, cf a complex coefficient per RHS on the device (0: skip);
// py == px, or FP32 y with FP16/BF16 x
cudaError_t gcr_caxpy(lqcd_prec py, lqcd_prec px, long Vh, int nrhs, MutField y, FieldRef x, const double2 *cf,
                      cudaStream_t st);
// x += alpha p + omega s; r = s - omega t; red = (rhat, r), |r|^2
cudaError_t bi_xr(lqcd_prec px, lqcd_prec pv, long Vh, int nrhs, MutField x, FieldRef p, FieldRef sv, FieldRef t,
                  MutField r, FieldRef rhat, const BiScalars *s, double *partials, double *red, cudaStream_t st);

// ---- dslash_<type>.cu
cudaError_t launch_dslash_prec(lqcd_prec prec, const DslashParams &P, int recon, int mode, int nr, cudaStream_t st);
// the tiled many-right-hand-side kernel (dslash_mrhs.cuh), g warps per block
cudaError_t launch_dslash_mrhs_prec(lqcd_prec prec, const DslashParams &P, int recon, int mode, int g, cudaStream_t st);
// Kernel variants of one dslash launch: 1, 2, 4 = dslash_kernel with that many
// right-hand sides per thread; kMrhsVariant + g = dslash_mrhs_kernel with g warps
// (2g right-hand sides) per block
constexpr int kMrhsVariant = 100;
cudaError_t launch_dslash_variant(lqcd_prec prec, const DslashParams &P, int recon, int mode, int variant,
                                  cudaStream_t st);

inline int prec_bytes(lqcd_prec p) { return (p == LQCD_F64 || p == LQCD_DF64) ? 8 : p == LQCD_F32 ? 4 : 2; }
inline bool prec_half(lqcd_prec p) { return p == LQCD_F16 || p == LQCD_BF16; }
// 16-byte words of one spinor site (24 reals) in precision p
inline long spinor_words(lqcd_prec p) { return 24L * prec_bytes(p) / 16; }

}  // namespace lqcd

// ---- the objects behind the opaque handles
struct lqcd_field {
  lqcd_ctx *ctx;
  lqcd_prec prec;
  lqcd_subset subset;
  int nrhs;
  long Vh;
  void *data[2];    // per parity: [rhs][words][Vh]
  float *scale[2];  // per parity: [rhs][Vh] (FP16/BF16), else nullptr
  void *alloc;
  float *scale_alloc;
  long rhs_words() const { return lqcd::spinor_words(prec) * Vh; }
  lqcd::FieldRef ref(int p) const { return lqcd::FieldRef{data[p], scale[p], rhs_words()}; }
  lqcd::MutField mut(int p) const { return lqcd::MutField{data[p], scale[p], rhs_words()}; }
  bool has(int p) const { return subset == LQCD_FULL || (int)subset == p; }
};

namespace lqcd {
struct OverlapState;
void overlap_free(lqcd_ctx *c);
}  // namespace lqcd

struct CloverStore {
  void *A[2] = {nullptr, nullptr};
  void *Ainv[2] = {nullptr, nullptr};
  float *As[2] = {nullptr, nullptr};
  float *Ais[2] = {nullptr, nullptr};
  void *alloc = nullptr;
};

struct lqcd_ctx {
  int dims[4];
  int tbc;
  cudaStream_t stream;
  lqcd::Geom geom;
  long V, Vh;
  double *U64 = nullptr;  // canonical FP64 links on the device
  bool have_gauge = false;
  std::map<int, void *> links;  // key 100*prec + recon
  double kappa = 0, csw = 0;
  bool have_kappa = false;
  bool clover_on = false;  // csw != 0 and built
  double a_bound[2] = {1.0, 1.0};  // per parity: Gershgorin bound of ||A|| (1 without clover)
  CloverStore clov[5];  // indexed by lqcd_prec
  double rho = 0;
  bool have_rho = false;
  // reduction scratch
  double *partials = nullptr;
  size_t partials_n = 0;
  unsigned *counter = nullptr;
  double *results = nullptr;  // 1024 doubles: [0,256) norms, [256,1024) small per-RHS coefficient arrays
  double *h_results = nullptr;  // pinned mirror
  // canonical staging for host <-> device transfers
  double *canon[2] = {nullptr, nullptr};
  size_t canon_n[2] = {0, 0};
  // copy streams and per-chunk events of the pipelined host-buffer dslash
  cudaStream_t copy_stream[2] = {nullptr, nullptr};
  cudaEvent_t chunk_event[2][64] = {};
  // cached intermediate fields (key: slot, subset, prec, nrhs; see temp_field)
  std::map<long, lqcd_field *> temps;
  // overlap operator state (low modes, Chebyshev coefficients), overlap.cu
  lqcd::OverlapState *ov = nullptr;
};

// ---- errors and allocation (abi.cu)
namespace lqcd {
lqcd_status set_error(lqcd_status s, const char *fmt, ...);
// cudaMalloc with the failure-injection hook (LQCD_FAULT_ALLOC_AFTER)
cudaError_t dev_malloc(void **p, size_t bytes);
}
#define LQ_CU(call)                                                                                      \
  do {                                                                                                   \
    cudaError_t e_ = (call);                                                                             \
    if (e_ != cudaSuccess)                                                                               \
      return ::lqcd::set_error(LQCD_ERR_CUDA, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, \
                               __LINE__);                                                                \
  } while (0)
#define LQ_TRY(call)                       \
  do {                                     \
    lqcd_status s_ = (call);               \
    if (s_ != LQCD_OK) return s_;          \
  } while (0)

// ---- operator layer (ops.cu)
namespace lqcd {
struct Term {  // an optional field operand of the dslash epilogue
  FieldRef f{nullptr, nullptr, 0};
};
lqcd_status get_links(lqcd_ctx *c, lqcd_prec prec, int recon, const void **base);
lqcd_status get_clover(lqcd_ctx *c, lqcd_prec prec, CloverStore **cs);
lqcd_status ensure_partials(lqcd_ctx *c, int nrhs);
// one launch of the generic dslash kernel on output parity out_p
lqcd_status run_dslash(lqcd_ctx *c, lqcd_prec prec, int recon, int mode, int out_p, int nrhs, MutField out, FieldRef in,
                       FieldRef xloc, FieldRef z, double alpha, double beta, double gz, int g5_in, int g5_hop,
                       int g5_total, double *norm_result, int norm_stride, const FieldRef *zc = nullptr,
                       const double *cz = nullptr, long h0 = 0, long h1 = -1);
// y_e = A_ee^-1 D_eo x_o (g5 on the input if dagger)
lqcd_status op_k2a(lqcd_ctx *c, lqcd_prec prec, int recon, int dagger, int nrhs, MutField y_e, FieldRef x_o,
                   long h0 = 0, long h1 = -1);
// z_o = [zf +gz*] (A_oo x_o - kappa^2 [g5] D_oe y_e), optional norm
lqcd_status op_k2b(lqcd_ctx *c, lqcd_prec prec, int recon, int dagger, int nrhs, MutField out_o, FieldRef x_o,
                   FieldRef y_e, FieldRef zf, double gz, double *norm_result, int norm_stride, long h0 = 0,
                   long h1 = -1);
// out_o = Mhat x_o or Mhat^dag x_o, y_e scratch
lqcd_status op_mhat(lqcd_ctx *c, lqcd_prec prec, int recon, int dagger, int nrhs, MutField out_o, FieldRef x_o,
                    MutField y_e, FieldRef zf, double gz, double *norm_result, int norm_stride);
// out_o = A_oo^-1 Mhat x_o (the symmetric Schur complement) or its adjoint;
// y_e and t_o scratch (t_o used by the adjoint only)
lqcd_status op_mhat_sym(lqcd_ctx *c, lqcd_prec prec, int recon, int dagger, int nrhs, MutField out_o, FieldRef x_o,
                        MutField y_e, MutField t_o, double *norm_result, int norm_stride);
// out_o = A_oo^-1 x_o (site-local), optional norm
lqcd_status op_ainv_odd(lqcd_ctx *c, lqcd_prec prec, int recon, int nrhs, MutField out_o, FieldRef x_o,
                        double *norm_result, int norm_stride);
// full-lattice out = [zf + gz*] M x (dagger: M^dag), per parity
lqcd_status op_M(lqcd_ctx *c, lqcd_prec prec, int recon, int dagger, int nrhs, MutField out[2], FieldRef x[2],
                 FieldRef zf[2], double gz, double *norm_result, int norm_stride);
// bhat_o = b_o + kappa D_oe A_ee^-1 b_e  (tmp_e scratch)
lqcd_status op_prepare(lqcd_ctx *c, lqcd_prec prec, int recon, int nrhs, MutField bhat_o, FieldRef b_e, FieldRef b_o,
                       MutField tmp_e);
// x_e = A_ee^-1 (b_e + kappa D_eo x_o)
lqcd_status op_reconstruct(lqcd_ctx *c, lqcd_prec prec, int recon, int nrhs, MutField x_e, FieldRef b_e,
                           FieldRef x_o);
// out_p = g5 [(4 - rho) x_p - D x_{1-p} / 2] on both parities
lqcd_status op_hw(lqcd_ctx *c, lqcd_prec prec, int recon, int nrhs, MutField out[2], FieldRef x[2], double *norm_result,
                  int norm_stride);
// one Chebyshev (Clenshaw) step fused into the second H_W application:
// out_p = t H_W x + sum_k cz[k] z[k]_p on both parities (z[k][p].data == nullptr: term absent)
lqcd_status op_hw_cheb(lqcd_ctx *c, lqcd_prec prec, int recon, int nrhs, MutField out[2], FieldRef x[2], double t,
                       const FieldRef z[3][2], const double cz[3]);
}  // namespace lqcd

namespace lqcd {
// context-cached temporary field for (prec, subset, nrhs, slot); owned by the context
lqcd_status temp_field(lqcd_ctx *c, lqcd_prec prec, lqcd_subset subset, int nrhs, int slot, lqcd_field **out);
// device staging buffer `slot` (0 or 1) of at least n doubles
lqcd_status staging(lqcd_ctx *c, int slot, size_t n, double **out);
}  // namespace lqcd
