// C ABI of the library (declared in include/gpcg.h): context management,
// argument validation, device buffers and the launch sequence of each call.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <type_traits>
#include <vector>

#include "../../include/gpcg.h"
#include "analysis.h"
#include "common.cuh"
#include "ctx_view.h"
#include "fdpf.h"

namespace gpcg {
// build.cu
void launch_branch_params(cudaStream_t, int, const double*, const double*, double*, double*,
                          double*, double*);
void launch_ybus_diag(cudaStream_t, int, const int32_t*, const int32_t*, const int32_t*,
                      const double*, const double*, const double*, const double*, double*,
                      double*);
void launch_laplacian_values(cudaStream_t, int, const int32_t*, const int32_t*, const int32_t*,
                             const int32_t*, const int32_t*, const double*, const int32_t*,
                             const double*, const int32_t*, const int32_t*, double*, int32_t*);
void launch_ic_level(cudaStream_t, int, int, const int32_t*, const int32_t*, const double*,
                     const int32_t*, const int32_t*, double*, int32_t*);
void launch_scatter(cudaStream_t, int, const int32_t*, const double*, double*);
void launch_to_float(cudaStream_t, int, const double*, float*);
void launch_gather_diag(cudaStream_t, int, const int32_t*, const double*, double*);
void launch_gather_int(cudaStream_t, int, const int32_t*, const int32_t*, int32_t*);
void launch_gather_val(cudaStream_t, int, const int32_t*, const double*, double*, float*);
void launch_scale_factor(cudaStream_t, int, const int32_t*, const int32_t*, const double*, double*,
                         double*, float*);
void launch_gather_half(cudaStream_t, int, const int32_t*, const double*, __half*);
void launch_inv_diag(cudaStream_t, int, const int32_t*, const double*, double*, float*);
void launch_tail_inverse(cudaStream_t, int, int, const int32_t*, const int32_t*, const double*,
                         const double*, double*, double*, float*, float*);
void launch_adj_values(cudaStream_t, int, const int32_t*, const double*, const double*,
                       const double*, double*, double*);
void launch_ext_rows(cudaStream_t, int, const int32_t*, const int32_t*, const int32_t*,
                     const int32_t*, const double*, const double*, const int32_t*, int32_t*,
                     double*, float*, double*, float*);
}  // namespace gpcg


using namespace gpcg;

// ------------------------------------------------------------------ errors
static thread_local std::string g_err;

static gpcg_status fail(gpcg_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return st;
}

#define CUDA_TRY(call)                                                                  \
  do {                                                                                  \
    cudaError_t ce_ = (call);                                                           \
    if (ce_ != cudaSuccess) {                                                           \
      if (ce_ == cudaErrorMemoryAllocation)                                             \
        return fail(GPCG_ERR_OOM, "%s: %s", #call, cudaGetErrorString(ce_));            \
      return fail(GPCG_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(ce_));             \
    }                                                                                   \
  } while (0)

// CUDA_TRY for the screen after its output staging exists: the staging is
// freed before the error returns (`cleanup` in scope).
#define CUDA_TRY_C(call)                                                                \
  do {                                                                                  \
    cudaError_t ce_ = (call);                                                           \
    if (ce_ != cudaSuccess) {                                                           \
      cleanup();                                                                        \
      if (ce_ == cudaErrorMemoryAllocation)                                             \
        return fail(GPCG_ERR_OOM, "%s: %s", #call, cudaGetErrorString(ce_));            \
      return fail(GPCG_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(ce_));             \
    }                                                                                   \
  } while (0)

// ------------------------------------------------------------------ context
// Padded rows (ELL) of one operator: integer structure built on the host,
// values gathered on the device from the CSR values through `src`.
struct EllDev {
  int K = 0;
  int32_t *col = nullptr, *src = nullptr;    // [n*K]; src = CSR position or -1
  int32_t *optr = nullptr, *ocol = nullptr, *osrc = nullptr;
  double* val = nullptr;
  float* val32 = nullptr;
  double* oval = nullptr;
  float* oval32 = nullptr;
  __half *valh = nullptr, *ovalh = nullptr;  // scaled factor values in FP16 (L, U only)
  int nslot = 0, nover = 0;
  template <typename VT>
  Ell<VT> view() const;
};
template <>
Ell<double> EllDev::view<double>() const { return Ell<double>{col, val, optr, ocol, oval}; }
template <>
Ell<float> EllDev::view<float>() const { return Ell<float>{col, val32, optr, ocol, oval32}; }

struct MatDev {
  MatrixPlan plan;
  int32_t *bus_of_row = nullptr, *row_of_bus = nullptr, *pre_of_row = nullptr, *visit = nullptr;
  int32_t *a_ptr = nullptr, *a_idx = nullptr, *a_diag = nullptr;
  int32_t *l_ptr = nullptr, *l_idx = nullptr, *l_diag = nullptr;
  int32_t *lev_ptr = nullptr, *blev_ptr = nullptr, *blev_rows = nullptr;
  int32_t *tblev_ptr = nullptr, *tblev_rows = nullptr;
  double *xc = nullptr, *xr = nullptr;  // inverse of the factor's tail block
  float *xc32 = nullptr, *xr32 = nullptr;
  float *xch = nullptr, *xrh = nullptr;  // the same for the FP16-stored factor
  double *a_val = nullptr, *l_val = nullptr, *diag = nullptr, *inv_diag = nullptr;
  float *diag32 = nullptr, *inv_diag32 = nullptr;
  double *lsc = nullptr, *inv_d2 = nullptr;  // scaled factor (FP64) and 1 / L_ii^2
  float* inv_d2_32 = nullptr;
  EllDev A, L, U;
  double* w = nullptr;  // per-branch weight
  double* c = nullptr;  // per-branch from-end factor (B'': 1 / turns ratio), null = 1
  // rows for buses without one (B'': tripped generators), see DevMatT
  const int32_t *xptr = nullptr, *xnb = nullptr, *xbr = nullptr;
  int32_t* xrow = nullptr;
  double *xval = nullptr, *xdiag = nullptr;
  float *xval32 = nullptr, *xdiag32 = nullptr;
  template <typename VT>
  DevMatT<VT> view(bool f16 = false) const;
};

template <>
DevMatT<double> MatDev::view<double>(bool) const {
  DevMatT<double> M;
  M.n = plan.n;
  M.bus_of_row = bus_of_row; M.row_of_bus = row_of_bus; M.pre_of_row = pre_of_row;
  M.visit = visit;
  M.A = A.view<double>(); M.L = L.view<double>(); M.U = U.view<double>();
  M.inv_diag = inv_diag;
  M.diag = diag;
  M.lev_ptr = lev_ptr; M.blev_ptr = blev_ptr; M.blev_rows = blev_rows;
  M.nlev = (int)plan.lev_ptr.size() - 1;
  M.nblev = (int)plan.blev_ptr.size() - 1;
  M.tail_lev = plan.tail_lev; M.tail_row0 = plan.tail_row0;
  M.tblev_ptr = tblev_ptr; M.tblev_rows = tblev_rows;
  M.ntblev = (int)plan.tblev_ptr.size() - 1;
  M.xc = xc; M.xr = xr;
  M.w = w;
  M.c = c;
  M.xptr = xptr; M.xrow = xrow; M.xval = xval; M.xdiag = xdiag; M.xnb = xnb; M.xbr = xbr;
  return M;
}
template <>
DevMatT<float> MatDev::view<float>(bool f16) const {
  DevMatT<float> M;
  M.n = plan.n;
  M.bus_of_row = bus_of_row; M.row_of_bus = row_of_bus; M.pre_of_row = pre_of_row;
  M.visit = visit;
  M.A = A.view<float>(); M.L = L.view<float>(); M.U = U.view<float>();
  M.inv_diag = inv_diag32;
  M.diag = diag32;
  if (f16) {
    M.Lh = L.valh; M.Loh = L.ovalh; M.Uh = U.valh; M.Uoh = U.ovalh;
    M.inv_d2 = inv_d2_32;
  }
  M.lev_ptr = lev_ptr; M.blev_ptr = blev_ptr; M.blev_rows = blev_rows;
  M.nlev = (int)plan.lev_ptr.size() - 1;
  M.nblev = (int)plan.blev_ptr.size() - 1;
  M.tail_lev = plan.tail_lev; M.tail_row0 = plan.tail_row0;
  M.tblev_ptr = tblev_ptr; M.tblev_rows = tblev_rows;
  M.ntblev = (int)plan.tblev_ptr.size() - 1;
  M.xc = f16 && xch ? xch : xc32;
  M.xr = f16 && xrh ? xrh : xr32;
  M.w = w;
  M.c = c;
  M.xptr = xptr; M.xrow = xrow; M.xval = xval32; M.xdiag = xdiag32; M.xnb = xnb; M.xbr = xbr;
  return M;
}

struct gpcg_ctx {
  int device = 0, num_sms = 0;
  gpcg_options opt{};
  int n = 0, m = 0, slack = -1, slack_user = -1;  // slack: internal numbering
  std::vector<int8_t> bus_type;                    // internal numbering
  std::vector<int32_t> user_of, intl;              // internal -> user, user -> internal
  // caller-numbered copies for the islanding kernel (labels are user indices)
  int32_t *u_f = nullptr, *u_t = nullptr, *u_pre = nullptr;
  int8_t* u_bus_type = nullptr;
  double *u_P_sched = nullptr, *u_P_gen = nullptr;
  std::vector<int32_t> f, t;
  BusGraph bg;
  std::vector<int32_t> pre, sub;
  std::vector<uint8_t> bridge;
  int n_bridges = 0;
  double pv_gen_total = 0.0;
  IslandPlan isl;              // per-grid islanding data (device)
  double *r0P = nullptr, *r0Q = nullptr;  // base-case mismatch per bus (after the base solve)
  double* d_prefP = nullptr;   // [n + 1] prefix sums of a caller's injections
  int n_adj_slots = 0, n_adj_over = 0;
  std::vector<int32_t> deg;
  int32_t *mis_order = nullptr, *misq_order = nullptr;
  int32_t* d_bus_of_user = nullptr;  // caller's bus -> internal bus
  unsigned long long* phase = nullptr;  // diagnostics: [8 + 2 phase_cap]
  size_t phase_cap = 0;
  bool phase_on = false;
  // each tile's z vector in shared memory where it fits (branch outages
  // without reactive limits, tiles of 2 or 4), asked for with GPCG_Z_SMEM=1:
  // it halves a scenario's latency but fits 2 CTAs per SM instead of 5, so a
  // full screen is slower
  bool zs_allowed = false;
  DevGrid G;
  double *wP = nullptr, *wQ = nullptr;
  MatDev MP, MQ;
  int planned_precond = -1;
  // base case
  double *th0 = nullptr, *V0 = nullptr, *flow0 = nullptr, *c0 = nullptr, *s0 = nullptr;
  int base_outer = -1;
  bool base_ok = false;
  // per-call buffers
  int32_t *d_outages = nullptr, *d_lo = nullptr, *d_cnt = nullptr, *d_nogen = nullptr,
          *d_order = nullptr, *d_genbus = nullptr;
  int32_t* d_porder = nullptr;  // the autotuner's probe: a strided subset of d_order
  std::vector<double> base_flow;  // |P_ij| of the base case: scheduling priority
  double* d_coef = nullptr;
  size_t sc_cap = 0;
  int32_t *d_counter = nullptr, *d_err = nullptr;
  void* work = nullptr;
  size_t work_bytes = 0;
  int tile = 0;
  // the autotuner's state: tiles per SM and dense-tail cap in use (0: not
  // chosen yet), how they were chosen (0 none, 1 probes, 2 cache) and the
  // power of two of the scenario count they were chosen for
  int per_sm = 0, per_sm_used = 0, tuned = 0, tuned_bucket = -1;
  int tail_rows_now = TAIL_ROWS;  // the cap the factors' tails are built with
  // the factors' dense-tail data of B' (0) and B'' (1): level schedule of the
  // rows before the tail and the tail block's inverse, rebuilt when the tail
  // cap changes
  std::vector<void*> tail_owned[2];
  // adjoint: B' with caller-given susceptances (structure of MP, own values)
  MatDev MA;
  bool ma_ready = false;
  std::vector<void*> adj_owned;
  double* adj_acc = nullptr;
  size_t adj_acc_bytes = 0;
  cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
  bool timed = false;
  // the plain FP64 path's work buffers (allocated on first use)
  PlainBuffers plainb;
  int plain_grid_size = 0;
  std::vector<void*> plain_owned;
  // the screen's launch sequence, captured once per argument set and replayed
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t graph = nullptr;
  std::vector<uintptr_t> graph_key;
  std::vector<void*> owned;  // freed at destroy (structures of the grid)
  std::vector<void*> mat_owned;  // freed when the matrices are rebuilt
};

template <typename X>
static cudaError_t dalloc(std::vector<void*>& own, X** p, size_t count) {
  *p = nullptr;
  if (count == 0) count = 1;
  cudaError_t ce = cudaMalloc((void**)p, count * sizeof(X));
  if (ce == cudaSuccess) own.push_back((void*)*p);
  return ce;
}

template <typename X>
static cudaError_t upload(std::vector<void*>& own, X** p, const X* src, size_t count) {
  cudaError_t ce = dalloc(own, p, count);
  if (ce != cudaSuccess || count == 0) return ce;
  return cudaMemcpy(*p, src, count * sizeof(X), cudaMemcpyHostToDevice);
}

static void free_list(std::vector<void*>& v) {
  for (void* p : v) cudaFree(p);
  v.clear();
}

// ------------------------------------------------------------------ options
extern "C" gpcg_status gpcg_default_options(gpcg_options* opt) {
  if (!opt) return fail(GPCG_ERR_INVALID_ARG, "gpcg_default_options: opt is NULL");
  opt->tol = 1e-4;
  opt->base_tol = 1e-10;
  opt->inner_rtol = 3e-3;  // the outer FP64 loop refines; tighter only adds inner iterations
  opt->max_outer = 50;
  opt->max_inner = 500;
  opt->precision = GPCG_BATCHED_FP32;
  opt->precond = GPCG_PRECOND_EXACT;
  opt->tile = 0;
  opt->ctas_per_sm = 0;
  opt->tail_rows = 0;
  opt->wait_limit = 0;
  g_err.clear();
  return GPCG_OK;
}

static gpcg_status check_options(const gpcg_options& o) {
  if (!(o.tol > 0) || !(o.base_tol > 0) || !(o.inner_rtol > 0) || !(o.inner_rtol < 1))
    return fail(GPCG_ERR_INVALID_ARG, "tolerances must be positive (inner_rtol < 1)");
  if (o.max_outer < 1 || o.max_inner < 1)
    return fail(GPCG_ERR_INVALID_ARG, "max_outer and max_inner must be >= 1");
  if (o.precision < 0 || o.precision > 3)
    return fail(GPCG_ERR_INVALID_ARG, "precision must be 0, 1, 2 or 3");
  if (o.precision == GPCG_BATCHED_FP32_F16 && o.precond == GPCG_PRECOND_JACOBI)
    return fail(GPCG_ERR_INVALID_ARG, "FP16 factors need a factor preconditioner (IC0 or EXACT)");
  if (o.precond < 0 || o.precond > 2)
    return fail(GPCG_ERR_INVALID_ARG, "precond must be 0, 1 or 2");
  if (!(o.tile == 0 || o.tile == 2 || o.tile == 4 || o.tile == 8 || o.tile == 16 || o.tile == 32))
    return fail(GPCG_ERR_INVALID_ARG, "tile must be 0, 2, 4, 8, 16 or 32");
  if (o.ctas_per_sm < 0 || o.ctas_per_sm > 64)
    return fail(GPCG_ERR_INVALID_ARG, "ctas_per_sm must be in [0, 64]");
  if (o.wait_limit < 0)
    return fail(GPCG_ERR_INVALID_ARG, "wait_limit must be >= 0");
  if (o.tail_rows < -1 || o.tail_rows > GPCG_MAX_TAIL_ROWS)
    return fail(GPCG_ERR_INVALID_ARG, "tail_rows must be -1, 0 or in [1, %d]", GPCG_MAX_TAIL_ROWS);
  return GPCG_OK;
}

// ------------------------------------------------------------------ build
// Host side of a padded-row operator: for each row the first K entries of
// `entries[row]` (pairs of column, source position) go to the slots, the
// rest to the overflow CSR; padding points at `pad_col` with source -1.
struct EllHost {
  int K = 0;
  std::vector<int32_t> col, src, optr, ocol, osrc;
};

static EllHost ell_from_rows(const std::vector<std::vector<std::pair<int, int>>>& rows, int K,
                             int pad_col) {
  EllHost E;
  E.K = K;
  const int n = (int)rows.size();
  E.col.assign((size_t)n * K, pad_col);
  E.src.assign((size_t)n * K, -1);
  E.optr.assign(n + 1, 0);
  for (int i = 0; i < n; ++i) {
    const auto& r = rows[i];
    for (size_t k = 0; k < r.size(); ++k) {
      if ((int)k < K) {
        E.col[(size_t)i * K + k] = r[k].first;
        E.src[(size_t)i * K + k] = r[k].second;
      } else {
        E.ocol.push_back(r[k].first);
        E.osrc.push_back(r[k].second);
      }
    }
    E.optr[i + 1] = (int32_t)E.ocol.size();
  }
  return E;
}

static cudaError_t ell_upload(std::vector<void*>& own, const EllHost& H, EllDev& D) {
  cudaError_t ce;
  D.K = H.K;
  D.nslot = (int)H.col.size();
  D.nover = (int)H.ocol.size();
  if ((ce = upload(own, &D.col, H.col.data(), H.col.size())) != cudaSuccess) return ce;
  if ((ce = upload(own, &D.src, H.src.data(), H.src.size())) != cudaSuccess) return ce;
  if ((ce = upload(own, &D.optr, H.optr.data(), H.optr.size())) != cudaSuccess) return ce;
  if ((ce = upload(own, &D.ocol, H.ocol.data(), H.ocol.size())) != cudaSuccess) return ce;
  if ((ce = upload(own, &D.osrc, H.osrc.data(), H.osrc.size())) != cudaSuccess) return ce;
  if ((ce = dalloc(own, &D.val, H.col.size())) != cudaSuccess) return ce;
  if ((ce = dalloc(own, &D.val32, H.col.size())) != cudaSuccess) return ce;
  if ((ce = dalloc(own, &D.oval, H.ocol.size())) != cudaSuccess) return ce;
  return dalloc(own, &D.oval32, H.ocol.size());
}

static void ell_fill(cudaStream_t st, EllDev& D, const double* csr_val) {
  launch_gather_val(st, D.nslot, D.src, csr_val, D.val, D.val32);
  launch_gather_val(st, D.nover, D.osrc, csr_val, D.oval, D.oval32);
}

// Values of a matrix whose structure is built: the weighted Laplacian
// (weights w per branch), its factor on the planned pattern, diagonals and
// padded-row values.  Synchronous.
// The dense tail of a factor: the last forward levels, together at most
// `cap` rows (0: none), solved with the inverse of their block; the rows
// before it get a backward level schedule of their own.  Allocates the
// schedule and the inverse's arrays (FP64, FP32, and for the FP16-stored
// factor) in the matrix's own tail list, replacing earlier ones.
static gpcg_status alloc_tail(gpcg_ctx* c, MatDev& M, int which, int cap) {
  auto& own = c->tail_owned[which];
  free_list(own);
  plan_tail(M.plan, cap);
  const MatrixPlan& P = M.plan;
  CUDA_TRY(upload(own, &M.tblev_ptr, P.tblev_ptr.data(), P.tblev_ptr.size()));
  M.tblev_rows = nullptr;
  if (!P.tblev_rows.empty())
    CUDA_TRY(upload(own, &M.tblev_rows, P.tblev_rows.data(), P.tblev_rows.size()));
  const size_t nt = (size_t)(P.n - P.tail_row0);
  CUDA_TRY(dalloc(own, &M.xc, nt * nt));
  CUDA_TRY(dalloc(own, &M.xr, nt * nt));
  CUDA_TRY(dalloc(own, &M.xc32, nt * nt));
  CUDA_TRY(dalloc(own, &M.xr32, nt * nt));
  CUDA_TRY(dalloc(own, &M.xch, nt * nt));
  CUDA_TRY(dalloc(own, &M.xrh, nt * nt));
  return GPCG_OK;
}

// The tail block's inverse from the factor's values: of the FP16-stored
// factor first (M.xc as FP64 scratch), then of the factor itself.
static void launch_tail_inverses(const MatDev& M, cudaStream_t st) {
  const MatrixPlan& P = M.plan;
  if (M.lsc && M.xch)
    launch_tail_inverse(st, P.tail_row0, P.n - P.tail_row0, M.l_ptr, M.l_idx, M.l_val, M.lsc,
                        M.xc, nullptr, M.xch, M.xrh);
  launch_tail_inverse(st, P.tail_row0, P.n - P.tail_row0, M.l_ptr, M.l_idx, M.l_val, nullptr,
                      M.xc, M.xr, M.xc32, M.xr32);
}

static gpcg_status fill_values(gpcg_ctx* c, MatDev& M, const double* w) {
  const MatrixPlan& P = M.plan;
  const int nl = P.L.nnz();
  (void)nl;
  cudaStream_t st = 0;
  CUDA_TRY(cudaMemset(c->d_err, 0, sizeof(int32_t)));
  launch_laplacian_values(st, P.n, M.bus_of_row, M.row_of_bus, c->G.adj_ptr, c->G.adj_idx,
                          c->G.adj_br, w, c->G.f, M.c, M.a_ptr, M.a_idx, M.a_val, c->d_err);
  for (size_t k = 0; k + 1 < P.lev_ptr.size(); ++k)
    launch_ic_level(st, P.lev_ptr[k], P.lev_ptr[k + 1], M.a_ptr, M.a_idx, M.a_val, M.l_ptr,
                    M.l_idx, M.l_val, c->d_err);
  launch_gather_diag(st, P.n, M.a_diag, M.a_val, M.diag);
  launch_to_float(st, P.n, M.diag, M.diag32);
  launch_inv_diag(st, P.n, M.l_diag, M.l_val, M.inv_diag, M.inv_diag32);
  ell_fill(st, M.A, M.a_val);
  ell_fill(st, M.L, M.l_val);
  ell_fill(st, M.U, M.l_val);
  if (M.lsc) {
    launch_scale_factor(st, P.n, M.l_ptr, M.l_idx, M.l_val, M.lsc, M.inv_d2, M.inv_d2_32);
    for (EllDev* E : {&M.L, &M.U}) {
      if (!E->valh) continue;
      launch_gather_half(st, E->nslot, E->src, M.lsc, E->valh);
      launch_gather_half(st, E->nover, E->osrc, M.lsc, E->ovalh);
    }
  }
  launch_tail_inverses(M, st);
  CUDA_TRY(cudaGetLastError());
  int32_t herr = 0;
  CUDA_TRY(cudaMemcpy(&herr, c->d_err, sizeof herr, cudaMemcpyDeviceToHost));
  if (herr == 1) return fail(GPCG_ERR_CUDA, "internal: CSR slot missing while building values");
  if (herr == 2)
    return fail(GPCG_ERR_INVALID_ARG,
                "base-case factorisation met a non-positive pivot (matrix not positive definite)");
  return GPCG_OK;
}

static gpcg_status build_matrix(gpcg_ctx* c, MatDev& M, int which,
                                const std::vector<uint8_t>& keep, double* w, double* cf,
                                bool fill) {
  M.plan = plan_matrix(c->n, c->bg, keep, fill);
  {
    gpcg_status st = alloc_tail(c, M, which, c->tail_rows_now);
    if (st != GPCG_OK) return st;
  }
  const MatrixPlan& P = M.plan;
  auto& own = c->mat_owned;
  std::vector<int32_t> pre_of_row(P.n);
  for (int i = 0; i < P.n; ++i) pre_of_row[i] = c->pre[P.bus_of_row[i]];
  CUDA_TRY(upload(own, &M.bus_of_row, P.bus_of_row.data(), P.n));
  CUDA_TRY(upload(own, &M.row_of_bus, P.row_of_bus.data(), c->n));
  CUDA_TRY(upload(own, &M.pre_of_row, pre_of_row.data(), P.n));
  {
    std::vector<int32_t> visit(P.n);
    for (int i = 0; i < P.n; ++i) visit[i] = i;
    std::sort(visit.begin(), visit.end(),
              [&](int a, int b) { return P.bus_of_row[a] < P.bus_of_row[b]; });
    CUDA_TRY(upload(own, &M.visit, visit.data(), P.n));
  }
  CUDA_TRY(upload(own, &M.a_ptr, P.A.ptr.data(), P.A.ptr.size()));
  CUDA_TRY(upload(own, &M.a_idx, P.A.idx.data(), P.A.idx.size()));
  CUDA_TRY(upload(own, &M.a_diag, P.a_diag.data(), P.n));
  CUDA_TRY(upload(own, &M.l_ptr, P.L.ptr.data(), P.L.ptr.size()));
  CUDA_TRY(upload(own, &M.l_idx, P.L.idx.data(), P.L.idx.size()));
  CUDA_TRY(upload(own, &M.lev_ptr, P.lev_ptr.data(), P.lev_ptr.size()));
  CUDA_TRY(upload(own, &M.blev_ptr, P.blev_ptr.data(), P.blev_ptr.size()));
  CUDA_TRY(upload(own, &M.blev_rows, P.blev_rows.data(), P.blev_rows.size()));
  std::vector<int32_t> ldiag(P.n);
  for (int i = 0; i < P.n; ++i) ldiag[i] = P.L.ptr[i + 1] - 1;
  CUDA_TRY(upload(own, &M.l_diag, ldiag.data(), P.n));
  const int nnz = P.A.nnz(), nl = P.L.nnz();
  CUDA_TRY(dalloc(own, &M.a_val, nnz));
  CUDA_TRY(dalloc(own, &M.l_val, nl));
  CUDA_TRY(dalloc(own, &M.diag, P.n));
  CUDA_TRY(dalloc(own, &M.diag32, P.n));
  CUDA_TRY(dalloc(own, &M.inv_diag, P.n));
  CUDA_TRY(dalloc(own, &M.inv_diag32, P.n));
  CUDA_TRY(dalloc(own, &M.lsc, nl));
  CUDA_TRY(dalloc(own, &M.inv_d2, P.n));
  CUDA_TRY(dalloc(own, &M.inv_d2_32, P.n));
  // padded rows: A (all entries), strictly lower L, strictly upper L^T
  {
    std::vector<std::vector<std::pair<int, int>>> ra(P.n), rl(P.n), ru(P.n);
    for (int i = 0; i < P.n; ++i) {
      for (int k = P.A.ptr[i]; k < P.A.ptr[i + 1]; ++k) ra[i].push_back({P.A.idx[k], k});
      for (int k = P.L.ptr[i]; k < P.L.ptr[i + 1] - 1; ++k) rl[i].push_back({P.L.idx[k], k});
    }
    std::vector<int32_t> u_to_l(nl);
    for (int k = 0; k < nl; ++k) u_to_l[P.l_to_u[k]] = k;
    for (int i = 0; i < P.n; ++i)
      for (int k = P.U.ptr[i] + 1; k < P.U.ptr[i + 1]; ++k) ru[i].push_back({P.U.idx[k], u_to_l[k]});
    CUDA_TRY(ell_upload(own, ell_from_rows(ra, KA, P.n), M.A));
    CUDA_TRY(ell_upload(own, ell_from_rows(rl, KL, P.n), M.L));
    CUDA_TRY(ell_upload(own, ell_from_rows(ru, KU, P.n), M.U));
    for (EllDev* E : {&M.L, &M.U}) {
      CUDA_TRY(dalloc(own, &E->valh, E->nslot));
      CUDA_TRY(dalloc(own, &E->ovalh, E->nover));
    }
  }
  M.w = w;
  M.c = cf;
  return fill_values(c, M, w);
}

static gpcg_status build_matrices(gpcg_ctx* c) {
  free_list(c->adj_owned);
  c->ma_ready = false;
  free_list(c->mat_owned);
  std::vector<uint8_t> keepP(c->n), keepQ(c->n);
  for (int b = 0; b < c->n; ++b) {
    keepP[b] = c->bus_type[b] != GPCG_SLACK;
    keepQ[b] = c->bus_type[b] == GPCG_PQ;
  }
  const bool fill = c->opt.precond == GPCG_PRECOND_EXACT;
  // B' leaves turns ratios out, B'' keeps them (the XB scheme)
  gpcg_status st = build_matrix(c, c->MP, 0, keepP, c->wP, nullptr, fill);
  if (st != GPCG_OK) return st;
  st = build_matrix(c, c->MQ, 1, keepQ, c->wQ, c->G.cf, fill);
  if (st != GPCG_OK) return st;
  {
    // B'' rows of PV buses, taken by a bus whose generator trips
    MatDev& M = c->MQ;
    auto& own = c->mat_owned;
    const size_t na = c->bg.adj.idx.size();
    CUDA_TRY(dalloc(own, &M.xrow, na));
    CUDA_TRY(dalloc(own, &M.xval, na));
    CUDA_TRY(dalloc(own, &M.xval32, na));
    CUDA_TRY(dalloc(own, &M.xdiag, c->n));
    CUDA_TRY(dalloc(own, &M.xdiag32, c->n));
    M.xptr = c->G.adj_ptr;
    M.xnb = c->G.adj_idx;
    M.xbr = c->G.adj_br;
    launch_ext_rows(0, c->n, c->G.adj_ptr, c->G.adj_idx, c->G.adj_br, c->G.f, c->G.cf, c->wQ,
                    M.row_of_bus, M.xrow, M.xval, M.xval32, M.xdiag, M.xdiag32);
    CUDA_TRY(cudaGetLastError());
    CUDA_TRY(cudaDeviceSynchronize());
  }
  {
    const MatrixPlan& Q = c->MQ.plan;
    std::vector<int32_t> order(Q.n);
    for (int k = 0; k < Q.n; ++k) order[k] = k;
    std::sort(order.begin(), order.end(),
              [&](int a, int b) { return Q.bus_of_row[a] < Q.bus_of_row[b]; });
    for (size_t w0 = 0; w0 < order.size(); w0 += 128)
      std::stable_sort(order.begin() + w0, order.begin() + std::min(order.size(), w0 + 128),
                       [&](int a, int b) {
                         return c->deg[Q.bus_of_row[a]] > c->deg[Q.bus_of_row[b]];
                       });
    CUDA_TRY(upload(c->mat_owned, &c->misq_order, order.data(), order.size()));
  }
  c->planned_precond = c->opt.precond;
  return GPCG_OK;
}

static void destroy(gpcg_ctx* c) {
  if (!c) return;
  free_list(c->plain_owned);
  free_list(c->adj_owned);
  if (c->adj_acc) cudaFree(c->adj_acc);
  free_list(c->mat_owned);
  for (auto& v : c->tail_owned) free_list(v);
  free_list(c->owned);
  if (c->work) cudaFree(c->work);
  for (auto& e : c->ev)
    if (e) cudaEventDestroy(e);
  if (c->graph) cudaGraphExecDestroy(c->graph);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  cudaFree(c->d_outages); cudaFree(c->d_lo); cudaFree(c->d_cnt); cudaFree(c->d_nogen);
  cudaFree(c->d_coef); cudaFree(c->d_order); cudaFree(c->d_genbus); cudaFree(c->d_porder);
  delete c;
}

extern "C" void gpcg_destroy(gpcg_ctx* c) { destroy(c); }

// Checks a grid; on success *slack_out is the slack bus.
static gpcg_status validate_grid(const gpcg_grid* g, int* slack_out) {
  const int n = g->n_bus, m = g->n_branch;
  if (n < 2 || m < 1) return fail(GPCG_ERR_INVALID_ARG, "need n_bus >= 2 and n_branch >= 1");
  if (!g->bus_type || !g->P_sched || !g->Q_sched || !g->P_gen || !g->V_set || !g->from ||
      !g->to || !g->r || !g->x || !g->b_sh || !g->rating)
    return fail(GPCG_ERR_INVALID_ARG, "a grid array is NULL");
  int slack = -1;
  for (int b = 0; b < n; ++b) {
    int bt = g->bus_type[b];
    if (bt < 0 || bt > 2) return fail(GPCG_ERR_INVALID_ARG, "bus %d: bad bus_type %d", b, bt);
    if (bt == GPCG_SLACK) {
      if (slack >= 0) return fail(GPCG_ERR_INVALID_ARG, "more than one slack bus (%d, %d)", slack, b);
      slack = b;
    }
    if (!std::isfinite(g->P_sched[b]) || !std::isfinite(g->Q_sched[b]) ||
        !std::isfinite(g->P_gen[b]) || !(g->V_set[b] > 0) || !std::isfinite(g->V_set[b]))
      return fail(GPCG_ERR_INVALID_ARG, "bus %d: non-finite injection or V_set <= 0", b);
  }
  if (slack < 0) return fail(GPCG_ERR_INVALID_ARG, "no slack bus");
  for (int e = 0; e < m; ++e) {
    int a = g->from[e], b = g->to[e];
    if (a < 0 || a >= n || b < 0 || b >= n || a == b)
      return fail(GPCG_ERR_INVALID_ARG, "branch %d: bad end buses (%d, %d)", e, a, b);
    if (!(g->x[e] > 0) || !std::isfinite(g->x[e]) || !(g->r[e] >= 0) ||
        !std::isfinite(g->r[e]) || !std::isfinite(g->b_sh[e]) || !(g->rating[e] > 0))
      return fail(GPCG_ERR_INVALID_ARG, "branch %d: needs x > 0, r >= 0, rating > 0", e);
    if (g->tap && !(g->tap[e] > 0 && std::isfinite(g->tap[e])))
      return fail(GPCG_ERR_INVALID_ARG, "branch %d: turns ratio %g is not positive and finite",
                  e, g->tap[e]);
  }
  if (!g->Q_min != !g->Q_max)
    return fail(GPCG_ERR_INVALID_ARG, "Q_min and Q_max come together (both or neither)");
  if (g->Q_max)
    for (int b = 0; b < n; ++b)
      if (g->bus_type[b] == GPCG_PV &&
          !(std::isfinite(g->Q_min[b]) && std::isfinite(g->Q_max[b]) && g->Q_min[b] <= g->Q_max[b]))
        return fail(GPCG_ERR_INVALID_ARG, "bus %d: reactive limits [%g, %g] are not an interval",
                    b, g->Q_min[b], g->Q_max[b]);
  *slack_out = slack;
  return GPCG_OK;
}

extern "C" gpcg_status gpcg_create(const gpcg_grid* g, const gpcg_options* opt, gpcg_ctx** out) {
  if (!out) return fail(GPCG_ERR_INVALID_ARG, "gpcg_create: out is NULL");
  *out = nullptr;
  if (!g) return fail(GPCG_ERR_INVALID_ARG, "gpcg_create: grid is NULL");
  const int n = g->n_bus, m = g->n_branch;
  gpcg_options o;
  gpcg_default_options(&o);
  if (opt) o = *opt;
  gpcg_status st = check_options(o);
  if (st != GPCG_OK) return st;
  int slack = -1;
  st = validate_grid(g, &slack);
  if (st != GPCG_OK) return st;
  gpcg_ctx* c = new gpcg_ctx();
  c->opt = o;
  c->tile = o.tile;  // 0: chosen on the first batched screen
  c->per_sm = o.ctas_per_sm;
  c->tail_rows_now = o.tail_rows > 0 ? o.tail_rows : (o.tail_rows < 0 ? 0 : TAIL_ROWS);
  c->n = n;
  c->m = m;
  c->slack_user = slack;
  // internal bus numbering: reverse Cuthill-McKee of the bus graph, so buses
  // adjacent in the grid sit close together in every per-bus array
  {
    BusGraph gu = build_bus_graph(n, m, g->from, g->to);
    c->user_of = rcm_order(n, gu);
  }
  c->intl.assign(n, 0);
  for (int k = 0; k < n; ++k) c->intl[c->user_of[k]] = k;
  const std::vector<int32_t>& U = c->user_of;
  const std::vector<int32_t>& I = c->intl;
  std::vector<int8_t> bt_i(n);
  std::vector<double> P_i(n), Q_i(n), Pg_i(n), V_i(n), qmin_i, qmax_i;
  for (int k = 0; k < n; ++k) {
    bt_i[k] = g->bus_type[U[k]];
    P_i[k] = g->P_sched[U[k]];
    Q_i[k] = g->Q_sched[U[k]];
    Pg_i[k] = g->P_gen[U[k]];
    V_i[k] = g->V_set[U[k]];
  }
  if (g->Q_max) {
    qmin_i.resize(n);
    qmax_i.resize(n);
    for (int k = 0; k < n; ++k) {
      qmin_i[k] = g->Q_min[U[k]];
      qmax_i[k] = g->Q_max[U[k]];
    }
  }
  std::vector<int32_t> f_i(m), t_i(m);
  for (int e = 0; e < m; ++e) {
    f_i[e] = I[g->from[e]];
    t_i[e] = I[g->to[e]];
  }
  c->slack = I[slack];
  c->bus_type = bt_i;
  c->f = f_i;
  c->t = t_i;
  cudaGetDevice(&c->device);
  cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device);
  c->bg = build_bus_graph(n, m, f_i.data(), t_i.data());
  if (!dfs_numbering(n, c->bg, c->slack, c->pre, c->sub, c->bridge, m)) {
    destroy(c);
    return fail(GPCG_ERR_BASE_ISLANDED, "the intact grid is not connected");
  }
  slack = c->slack;
  for (int e = 0; e < m; ++e) c->n_bridges += c->bridge[e];
  for (int b = 0; b < n; ++b)
    if (g->bus_type[b] == GPCG_PV && g->P_gen[b] > 0) c->pv_gen_total += g->P_gen[b];
  auto fail_cuda = [&](cudaError_t ce, const char* what) {
    destroy(c);
    return fail(ce == cudaErrorMemoryAllocation ? GPCG_ERR_OOM : GPCG_ERR_CUDA, "%s: %s", what,
                cudaGetErrorString(ce));
  };
  cudaError_t ce;
  auto& own = c->owned;
  DevGrid& G = c->G;
  G.n = n; G.m = m; G.slack = slack;
#define UP(dst, src, cnt)                                   \
  if ((ce = upload(own, &dst, src, cnt)) != cudaSuccess) return fail_cuda(ce, "upload " #dst)
#define AL(dst, cnt)                                        \
  if ((ce = dalloc(own, &dst, cnt)) != cudaSuccess) return fail_cuda(ce, "alloc " #dst)
  UP(G.bus_type, bt_i.data(), n);
  UP(G.P_sched, P_i.data(), n);
  UP(G.Q_sched, Q_i.data(), n);
  UP(G.P_gen, Pg_i.data(), n);
  UP(G.V_set, V_i.data(), n);
  if (g->Q_max) {
    UP(G.qmin, qmin_i.data(), n);
    UP(G.qmax, qmax_i.data(), n);
  }
  UP(G.f, f_i.data(), m);
  UP(G.t, t_i.data(), m);
  UP(G.user_of_bus, U.data(), n);
  UP(c->d_bus_of_user, I.data(), n);
  {
    std::vector<int32_t> pre_u(n);
    for (int b = 0; b < n; ++b) pre_u[b] = c->pre[I[b]];
    UP(c->u_pre, pre_u.data(), n);
    // islanding plan: bridge intervals, labels of both sides, preorder sums
    std::vector<int32_t> ord(n);
    for (int b = 0; b < n; ++b) ord[pre_u[b]] = b;
    std::vector<double> prefPs(n + 1, 0.0), prefG(n + 1, 0.0);
    std::vector<int32_t> prefGc(n + 1, 0);
    for (int k = 0; k < n; ++k) {
      const int b = ord[k];
      const bool gen = g->bus_type[b] == GPCG_PV && g->P_gen[b] > 0;
      prefPs[k + 1] = prefPs[k] + g->P_sched[b];
      prefG[k + 1] = prefG[k] + (gen ? g->P_gen[b] : 0.0);
      prefGc[k + 1] = prefGc[k] + (gen ? 1 : 0);
    }
    // range minimum of the caller's bus indices over preorder intervals
    std::vector<int32_t> pmin(n + 1, INT32_MAX), smin(n + 1, INT32_MAX);
    for (int k = 0; k < n; ++k) pmin[k + 1] = std::min(pmin[k], ord[k]);
    for (int k = n - 1; k >= 0; --k) smin[k] = std::min(smin[k + 1], ord[k]);
    int lg = 1;
    while ((1 << lg) <= n) ++lg;
    std::vector<std::vector<int32_t>> sp(lg, std::vector<int32_t>(n));
    sp[0] = ord;
    for (int j = 1; j < lg; ++j)
      for (int k = 0; k + (1 << j) <= n; ++k)
        sp[j][k] = std::min(sp[j - 1][k], sp[j - 1][k + (1 << (j - 1))]);
    auto range_min = [&](int a, int b) {  // [a, b), b > a
      int j = 31 - __builtin_clz((unsigned)(b - a));
      return std::min(sp[j][a], sp[j][b - (1 << j)]);
    };
    std::vector<int32_t> br_lo(m, 0), br_cnt(m, 0), lab_isl(m, 0), lab_main(m, 0);
    for (int e = 0; e < m; ++e) {
      if (!c->bridge[e]) continue;
      const int a = f_i[e], b = t_i[e];
      const int child = c->pre[a] > c->pre[b] ? a : b;  // the tree edge's lower end
      const int lo = c->pre[child], cnt = c->sub[child];
      br_lo[e] = lo;
      br_cnt[e] = cnt;
      lab_isl[e] = range_min(lo, lo + cnt);
      lab_main[e] = std::min(pmin[lo], smin[lo + cnt]);
    }
    int32_t *d_lo_, *d_cnt_, *d_li, *d_lm, *d_ord, *d_gc;
    double *d_ps, *d_pg;
    UP(d_lo_, br_lo.data(), m);
    UP(d_cnt_, br_cnt.data(), m);
    UP(d_li, lab_isl.data(), m);
    UP(d_lm, lab_main.data(), m);
    UP(d_ord, ord.data(), n);
    UP(d_ps, prefPs.data(), n + 1);
    UP(d_pg, prefG.data(), n + 1);
    UP(d_gc, prefGc.data(), n + 1);
    AL(c->d_prefP, n + 1);
    c->isl.br_lo = d_lo_; c->isl.br_cnt = d_cnt_;
    c->isl.lab_isl = d_li; c->isl.lab_main = d_lm;
    c->isl.u_pre = c->u_pre; c->isl.ord_u = d_ord;
    c->isl.prefPs = d_ps; c->isl.prefG = d_pg; c->isl.prefGc = d_gc;
  }
  UP(c->u_f, g->from, m);
  UP(c->u_t, g->to, m);
  UP(c->u_bus_type, g->bus_type, n);
  UP(c->u_P_sched, g->P_sched, n);
  UP(c->u_P_gen, g->P_gen, n);
  UP(G.r, g->r, m);
  UP(G.x, g->x, m);
  UP(G.b_sh, g->b_sh, m);
  UP(G.rating, g->rating, m);
  {
    std::vector<double> inv(m);
    for (int e = 0; e < m; ++e) inv[e] = 1.0 / g->rating[e];
    UP(G.inv_rating, inv.data(), m);
    for (int e = 0; e < m; ++e) inv[e] = g->tap ? 1.0 / g->tap[e] : 1.0;
    UP(G.cf, inv.data(), m);
  }
  UP(G.adj_ptr, c->bg.adj.ptr.data(), n + 1);
  UP(G.adj_idx, c->bg.adj.idx.data(), c->bg.adj.idx.size());
  UP(G.adj_br, c->bg.adj_branch.data(), c->bg.adj_branch.size());
  UP(G.pre, c->pre.data(), n);
  {
    // padded adjacency of the mismatch: padding repeats the bus itself with a
    // zero admittance and branch id -2
    std::vector<std::vector<std::pair<int, int>>> rows(n);
    for (int b = 0; b < n; ++b)
      for (int k = c->bg.adj.ptr[b]; k < c->bg.adj.ptr[b + 1]; ++k)
        rows[b].push_back({c->bg.adj.idx[k], c->bg.adj_branch[k]});
    EllHost E = ell_from_rows(rows, KG, 0);
    // slot-major: slot k of bus b at k * n + b
    std::vector<int32_t> pad_nbr(E.col.size()), brl(E.src.size());
    for (int b = 0; b < n; ++b)
      for (int k = 0; k < KG; ++k) {
        const size_t o = (size_t)b * KG + k, t = (size_t)k * n + b;
        const bool pad = E.src[o] < 0;
        pad_nbr[t] = pad ? b : E.col[o];
        brl[t] = pad ? -2 : E.src[o];
      }
    UP(G.adj_nbr, pad_nbr.data(), pad_nbr.size());
    UP(G.adj_brl, brl.data(), brl.size());
    UP(G.adj_optr, E.optr.data(), E.optr.size());
    UP(G.adj_onbr, E.ocol.data(), E.ocol.size());
    UP(G.adj_obr, E.osrc.data(), E.osrc.size());
    AL(G.adj_g, pad_nbr.size());
    AL(G.adj_b, pad_nbr.size());
    AL(G.adj_og, E.ocol.size());
    AL(G.adj_ob, E.ocol.size());
    c->n_adj_slots = (int)pad_nbr.size();
    c->n_adj_over = (int)E.ocol.size();
    std::vector<int32_t> deg(n), order;
    for (int b = 0; b < n; ++b) deg[b] = std::min(c->bg.adj.ptr[b + 1] - c->bg.adj.ptr[b], KG);
    for (int b = 0; b < n; ++b)
      if (b != slack) order.push_back(b);
    // bus order (neighbours close), degree-sorted inside windows of 128 rows
    // so the threads of a warp mostly run neighbour loops of equal length
    for (size_t w0 = 0; w0 < order.size(); w0 += 128)
      std::stable_sort(order.begin() + w0, order.begin() + std::min(order.size(), w0 + 128),
                       [&](int a, int b) { return deg[a] > deg[b]; });
    UP(G.adj_deg, deg.data(), n);
    UP(c->mis_order, order.data(), order.size());
    c->deg = deg;
  }
  UP(G.sub, c->sub.data(), n);
  AL(G.g, m);
  AL(G.by, m);
  AL(G.Gii, n);
  AL(G.Bii, n);
  AL(c->wP, m);
  AL(c->wQ, m);
  AL(c->th0, n);
  AL(c->V0, n);
  AL(c->flow0, m);
  AL(c->c0, n);
  AL(c->s0, n);
  AL(c->d_counter, 1);
  AL(c->d_err, 1);
  AL(c->r0P, n);
  AL(c->r0Q, n);
  for (auto& e : c->ev)
    if ((ce = cudaEventCreate(&e)) != cudaSuccess) return fail_cuda(ce, "event");
  AL(c->phase, 8 + 2 + 4);
  c->phase_cap = 1;
  if ((ce = cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking)) != cudaSuccess)
    return fail_cuda(ce, "stream");
  {
    const char* ev = std::getenv("GPCG_PHASE_TIMERS");
    c->phase_on = ev && ev[0] == '1';
    const char* zv = std::getenv("GPCG_Z_SMEM");
    c->zs_allowed = zv && zv[0] == '1';
  }
#undef UP
#undef AL
  launch_branch_params(0, m, G.r, G.x, G.g, G.by, c->wP, c->wQ);
  launch_ybus_diag(0, n, G.adj_ptr, G.adj_br, G.f, G.cf, G.g, G.by, G.b_sh, G.Gii, G.Bii);
  launch_adj_values(0, c->n_adj_slots, G.adj_brl, G.cf, G.g, G.by, G.adj_g, G.adj_b);
  launch_adj_values(0, c->n_adj_over, G.adj_obr, G.cf, G.g, G.by, G.adj_og, G.adj_ob);
  if ((ce = cudaGetLastError()) != cudaSuccess) return fail_cuda(ce, "build kernels");
  st = build_matrices(c);
  if (st != GPCG_OK) {
    std::string msg = g_err;
    destroy(c);
    g_err = msg;
    return st;
  }
  if ((ce = cudaDeviceSynchronize()) != cudaSuccess) return fail_cuda(ce, "create");
  *out = c;
  g_err.clear();
  return GPCG_OK;
}

static void drop_graph(gpcg_ctx* c) {
  if (c->graph) cudaGraphExecDestroy(c->graph);
  c->graph = nullptr;
  c->graph_key.clear();
}

// Both factors' dense tails rebuilt with at most `cap` rows (0: none).
static gpcg_status set_tail(gpcg_ctx* c, int cap) {
  if (cap == c->tail_rows_now) return GPCG_OK;
  CUDA_TRY(cudaDeviceSynchronize());  // launches in flight read the old tails
  c->tail_rows_now = cap;
  for (int k = 0; k < 2; ++k) {
    MatDev& M = k ? c->MQ : c->MP;
    gpcg_status s = alloc_tail(c, M, k, cap);
    if (s != GPCG_OK) return s;
    launch_tail_inverses(M, 0);
  }
  CUDA_TRY(cudaGetLastError());
  CUDA_TRY(cudaDeviceSynchronize());
  // the adjoint's copy of B' shares the tail's schedule: rebuilt on next use
  free_list(c->adj_owned);
  c->ma_ready = false;
  drop_graph(c);
  return GPCG_OK;
}

extern "C" gpcg_status gpcg_set_options(gpcg_ctx* c, const gpcg_options* opt) {
  if (!c || !opt) return fail(GPCG_ERR_INVALID_ARG, "gpcg_set_options: NULL argument");
  gpcg_status st = check_options(*opt);
  if (st != GPCG_OK) return st;
  const bool rebuild = opt->precond != c->planned_precond &&
                       ((opt->precond == GPCG_PRECOND_EXACT) !=
                        (c->planned_precond == GPCG_PRECOND_EXACT));
  // a knob, the precision or the preconditioner changed: tune again
  const bool retune = opt->tile != c->opt.tile || opt->ctas_per_sm != c->opt.ctas_per_sm ||
                      opt->tail_rows != c->opt.tail_rows || opt->precision != c->opt.precision ||
                      opt->precond != c->opt.precond;
  drop_graph(c);
  c->opt = *opt;
  if (retune) {
    c->tile = opt->tile;
    c->per_sm = opt->ctas_per_sm;
    c->tuned = 0;
    c->tuned_bucket = -1;
  }
  const int cap = opt->tail_rows > 0 ? opt->tail_rows
                                     : (opt->tail_rows < 0 ? 0 : c->tail_rows_now);
  if (rebuild) {
    c->tail_rows_now = cap;
    st = build_matrices(c);
  } else {
    st = set_tail(c, cap);
  }
  if (st != GPCG_OK) return st;
  c->planned_precond = opt->precond;
  g_err.clear();
  return GPCG_OK;
}

extern "C" gpcg_status gpcg_get_info(const gpcg_ctx* c, gpcg_info* info) {
  if (!c || !info) return fail(GPCG_ERR_INVALID_ARG, "gpcg_get_info: NULL argument");
  info->n_bus = c->n;
  info->n_branch = c->m;
  info->slack = c->slack_user;
  info->n_p = c->MP.plan.n;
  info->n_q = c->MQ.plan.n;
  info->nnz_p = c->MP.plan.A.nnz();
  info->nnz_q = c->MQ.plan.A.nnz();
  info->nnz_lp = c->MP.plan.L.nnz();
  info->nnz_lq = c->MQ.plan.L.nnz();
  info->levels_p = (int)c->MP.plan.lev_ptr.size() - 1;
  info->levels_q = (int)c->MQ.plan.lev_ptr.size() - 1;
  info->blevels_p = (int)c->MP.plan.blev_ptr.size() - 1;
  info->blevels_q = (int)c->MQ.plan.blev_ptr.size() - 1;
  info->n_bridges = c->n_bridges;
  info->tile = c->tile;
  info->num_sms = c->num_sms;
  info->base_outer = c->base_outer;
  info->ctas_per_sm = c->per_sm_used;
  info->tail_rows_p = c->MP.plan.n - c->MP.plan.tail_row0;
  info->tail_rows_q = c->MQ.plan.n - c->MQ.plan.tail_row0;
  info->tuned = c->tuned;
  g_err.clear();
  return GPCG_OK;
}

// ------------------------------------------------------------------ solves
static gpcg_status ensure_scen(gpcg_ctx* c, size_t S) {
  if (S <= c->sc_cap) return GPCG_OK;
  drop_graph(c);
  cudaFree(c->d_outages); cudaFree(c->d_lo); cudaFree(c->d_cnt); cudaFree(c->d_nogen);
  cudaFree(c->d_coef); cudaFree(c->d_order); cudaFree(c->d_genbus); cudaFree(c->d_porder);
  c->d_porder = nullptr;
  c->d_outages = c->d_lo = c->d_cnt = c->d_nogen = c->d_order = c->d_genbus = nullptr;
  c->d_coef = nullptr;
  c->sc_cap = 0;
  size_t cap = std::max<size_t>(S, 64);
  CUDA_TRY(cudaMalloc(&c->d_outages, cap * 4));
  CUDA_TRY(cudaMalloc(&c->d_lo, cap * 4));
  CUDA_TRY(cudaMalloc(&c->d_cnt, cap * 4));
  CUDA_TRY(cudaMalloc(&c->d_nogen, cap * 4));
  CUDA_TRY(cudaMalloc(&c->d_coef, cap * 8));
  CUDA_TRY(cudaMalloc(&c->d_order, cap * 4));
  CUDA_TRY(cudaMalloc(&c->d_genbus, cap * 4));
  CUDA_TRY(cudaMalloc(&c->d_porder, cap * 4));
  c->sc_cap = cap;
  return GPCG_OK;
}

static gpcg_status ensure_work(gpcg_ctx* c, size_t bytes) {
  if (bytes <= c->work_bytes) return GPCG_OK;
  drop_graph(c);
  if (c->work) cudaFree(c->work);
  c->work = nullptr;
  c->work_bytes = 0;
  CUDA_TRY(cudaMalloc(&c->work, bytes));
  c->work_bytes = bytes;
  return GPCG_OK;
}

struct Layout {
  int T = 32, slots = 1;
  size_t vstride = 0, sstride = 0, vec_bytes = 0, bytes = 0;
};

static Layout make_layout(const gpcg_ctx* c, int T, int slots, size_t vt_size, bool zs = false) {
  Layout L;
  L.T = T;
  L.slots = slots;
  // B' rows + its zero row; B'' rows + its zero row + the extension rows
  const size_t rows = (size_t)std::max(c->MP.plan.n + 1, c->MQ.plan.n + 1 + KX);
  L.vstride = rows * T;
  L.sstride = (size_t)c->n * T;
  L.vec_bytes = ((L.vstride * vt_size + 255) / 256) * 256;
  const size_t st_bytes = ((L.sstride * 8 + 255) / 256) * 256;
  L.bytes = (size_t)slots * ((zs ? 4 : 5) * L.vec_bytes + 4 * st_bytes);
  return L;
}

// zs: each tile's z vector in the kernel's dynamic shared memory (the
// vector's bytes of it) instead of the work buffer.
template <typename VT>
static gpcg_status run_fdpf(gpcg_ctx* c, cudaStream_t st, FdpfParams P, int T, int slots,
                            bool f16 = false, bool zs = false) {
  Layout Lo = make_layout(c, T, slots, sizeof(VT), zs);
  gpcg_status s = ensure_work(c, Lo.bytes);
  if (s != GPCG_OK) return s;
  char* base = (char*)c->work;
  const size_t vb = (size_t)slots * Lo.vec_bytes;
  const size_t sb = (size_t)slots * (((Lo.sstride * 8 + 255) / 256) * 256);
  const int nv = zs ? 4 : 5;
  P.wx = base; P.wr = base + vb; P.wp = base + 2 * vb; P.wq = base + 3 * vb;
  P.wz = zs ? nullptr : base + 4 * vb;
  P.vstride = Lo.vec_bytes / sizeof(VT);
  double* sbase = (double*)(base + nv * vb);
  const size_t ss = sb / slots / 8;
  P.wth = sbase; P.wV = sbase + slots * ss; P.we = sbase + 2 * slots * ss;
  P.wf = sbase + 3 * slots * ss;
  P.sstride = ss;
  P.tile_counter = c->d_counter;
  CUDA_TRY(cudaMemsetAsync(c->d_counter, 0, sizeof(int32_t), st));
  CUDA_TRY(launch_fdpf<VT>(st, T, slots, P, c->MP.view<VT>(f16), c->MQ.view<VT>(f16),
                           zs ? Lo.vec_bytes : 0));
  return GPCG_OK;
}

static FdpfParams base_params(gpcg_ctx* c) {
  FdpfParams P;
  P.G = c->G;
  P.mis_order = c->mis_order;
  P.misq_order = c->misq_order;
  P.phase_cycles = c->phase_on ? c->phase : nullptr;
  P.tol = c->opt.tol;
  P.inner_rtol = c->opt.inner_rtol;
  P.max_outer = c->opt.max_outer;
  P.max_inner = c->opt.max_inner;
  P.precond = c->opt.precond;
  if (c->base_ok) {  // warm starts from the base case
    P.r0P = c->r0P;
    P.r0Q = c->r0Q;
  }
  return P;
}

extern "C" gpcg_status gpcg_base_solve(gpcg_ctx* c, double* theta, double* vm, double* flow,
                                       int32_t* iters) {
  if (!c) return fail(GPCG_ERR_INVALID_ARG, "gpcg_base_solve: ctx is NULL");
  gpcg_status s = ensure_scen(c, 1);
  if (s != GPCG_OK) return s;
  cudaStream_t st = 0;
  const int32_t neg = -1, zero = 0;
  const double dz = 0.0;
  CUDA_TRY(cudaMemcpy(c->d_outages, &neg, 4, cudaMemcpyHostToDevice));
  CUDA_TRY(cudaMemcpy(c->d_lo, &zero, 4, cudaMemcpyHostToDevice));
  CUDA_TRY(cudaMemcpy(c->d_cnt, &zero, 4, cudaMemcpyHostToDevice));
  CUDA_TRY(cudaMemcpy(c->d_nogen, &zero, 4, cudaMemcpyHostToDevice));
  CUDA_TRY(cudaMemcpy(c->d_coef, &dz, 8, cudaMemcpyHostToDevice));
  FdpfParams P = base_params(c);
  P.S = 1;
  P.n_tiles = 1;
  P.sc = ScenInfo{c->d_outages, c->d_lo, c->d_cnt, c->d_coef, c->d_nogen};
  P.flat_start = 1;
  P.r0P = P.r0Q = nullptr;
  P.tol = c->opt.base_tol;
  P.max_outer = std::max(c->opt.max_outer, 100);
  P.out_theta = c->th0;
  P.out_vm = c->V0;
  P.out_flow = c->flow0;
  int32_t* d_stat = c->d_cnt;  // the scenario's own count slot doubles as its status
  int32_t* d_iters3 = nullptr;
  CUDA_TRY(cudaMalloc(&d_iters3, 3 * sizeof(int32_t)));
  P.out_iters = d_iters3;
  P.out_status = d_stat;
  s = run_fdpf<double>(c, st, P, 2, 1);
  int32_t hs = -1, hit[3] = {0, 0, 0};
  if (s == GPCG_OK) {
    cudaError_t ce = cudaDeviceSynchronize();
    if (ce == cudaSuccess) ce = cudaMemcpy(&hs, d_stat, 4, cudaMemcpyDeviceToHost);
    if (ce == cudaSuccess) ce = cudaMemcpy(hit, d_iters3, 12, cudaMemcpyDeviceToHost);
    if (ce != cudaSuccess) s = fail(GPCG_ERR_CUDA, "base solve: %s", cudaGetErrorString(ce));
  }
  cudaFree(d_iters3);
  if (s != GPCG_OK) return s;
  c->base_outer = hit[0];
  if (hs == GPCG_SCEN_QLIM_OVERFLOW) {
    c->base_ok = false;
    return fail(GPCG_ERR_BASE_NOT_CONVERGED,
                "the base case needs PV generators outside their reactive limits");
  }
  if (hs != GPCG_SCEN_OK) {
    c->base_ok = false;
    return fail(GPCG_ERR_BASE_NOT_CONVERGED,
                "base case did not converge (status %d after %d outer iterations)", hs, hit[0]);
  }
  CUDA_TRY(launch_base_trig(0, c->n, c->th0, c->c0, c->s0));
  CUDA_TRY(launch_base_residual(0, c->G, c->V0, c->c0, c->s0, c->r0P, c->r0Q));
  CUDA_TRY(cudaDeviceSynchronize());
  c->base_flow.resize(c->m);
  CUDA_TRY(cudaMemcpy(c->base_flow.data(), c->flow0, (size_t)c->m * 8, cudaMemcpyDeviceToHost));
  for (auto& v : c->base_flow) v = std::fabs(v);
  c->base_ok = true;
  if (theta || vm) {
    std::vector<double> h(c->n);
    if (theta) {
      CUDA_TRY(cudaMemcpy(h.data(), c->th0, (size_t)c->n * 8, cudaMemcpyDeviceToHost));
      for (int k = 0; k < c->n; ++k) theta[c->user_of[k]] = h[k];
    }
    if (vm) {
      CUDA_TRY(cudaMemcpy(h.data(), c->V0, (size_t)c->n * 8, cudaMemcpyDeviceToHost));
      for (int k = 0; k < c->n; ++k) vm[c->user_of[k]] = h[k];
    }
  }
  if (flow) CUDA_TRY(cudaMemcpy(flow, c->flow0, (size_t)c->m * 8, cudaMemcpyDeviceToHost));
  if (iters) { iters[0] = hit[0]; iters[1] = hit[1]; iters[2] = hit[2]; }
  g_err.clear();
  return GPCG_OK;
}

// Work buffers of the plain path for this context's grid.
static gpcg_status ensure_plain(gpcg_ctx* c) {
  if (c->plain_grid_size) return GPCG_OK;
  const int grid = plain_grid(c->num_sms);
  if (grid <= 0) return fail(GPCG_ERR_CUDA, "plain path: no cooperative launch configuration");
  PlainBuffers& B = c->plainb;
  auto& own = c->plain_owned;
  const size_t rows = (size_t)std::max(c->MP.plan.n, c->MQ.plan.n) + 1;
  CUDA_TRY(dalloc(own, &B.part, (size_t)2 * 4 * grid));
  CUDA_TRY(dalloc(own, &B.bar, 2));
  CUDA_TRY(dalloc(own, &B.err, 1));
  for (double** v : {&B.x, &B.r, &B.p, &B.q, &B.z, &B.t}) CUDA_TRY(dalloc(own, v, rows));
  CUDA_TRY(dalloc(own, &B.th, (size_t)c->n));
  CUDA_TRY(dalloc(own, &B.V, (size_t)c->n));
  CUDA_TRY(dalloc(own, &B.ef, (size_t)2 * c->n));
  c->plain_grid_size = grid;
  return GPCG_OK;
}

// The autotuner's choices, shared by the contexts of the process: keyed by
// the device, the grid's sizes, precision, preconditioner, kernel kind, the
// options that fix knobs, and the power of two of the scenario count.
struct TuneChoice {
  int tile, per_sm, tail;
};
static std::mutex g_tune_mu;
static std::map<std::vector<long long>, TuneChoice> g_tune_cache;

static_assert(KX == GPCG_MAX_EXT_ROWS, "extension rows of the kernel and of the C ABI");
static_assert(TAIL_ROWS >= GPCG_MAX_TAIL_ROWS, "the kernel's tail buffer holds the largest tail");

static std::vector<long long> tune_key(const gpcg_ctx* c, bool ext, int bucket) {
  int major = 0, minor = 0;
  cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, c->device);
  cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, c->device);
  return {c->num_sms, major, minor, c->n, c->m,
          c->MP.plan.A.nnz(), c->MP.plan.L.nnz(), c->MQ.plan.A.nnz(), c->MQ.plan.L.nnz(),
          c->opt.precision, c->opt.precond, ext, c->zs_allowed, bucket,
          c->opt.tile, c->opt.ctas_per_sm, c->opt.tail_rows};
}

template <typename X>
struct OutBuf {
  X* dev = nullptr;
  X* host = nullptr;
  size_t count = 0;
  bool owned = false;
};

// The N-1 screen of branch outages (gen = false: `outages` are branch
// indices) or of generator outages (gen = true: PV bus indices).
static gpcg_status n1_screen_impl(gpcg_ctx* c, const int32_t* outages, int32_t n_out,
                                  int32_t mem, void* stream, double* theta, double* vm,
                                  double* flow, int32_t* island_label, int32_t* iters,
                                  int32_t* status, double* max_loading, int32_t* n_overload,
                                  uint32_t* overload, bool gen) {
  if (!c) return fail(GPCG_ERR_INVALID_ARG, "gpcg_n1_screen: ctx is NULL");
  if (n_out < 0) return fail(GPCG_ERR_INVALID_ARG, "n_out < 0");
  if (mem != GPCG_MEM_HOST && mem != GPCG_MEM_DEVICE)
    return fail(GPCG_ERR_INVALID_ARG, "mem must be 0 (host) or 1 (device)");
  if (!c->base_ok) return fail(GPCG_ERR_NOT_READY, "gpcg_base_solve has not succeeded");
  if (n_out == 0) { g_err.clear(); return GPCG_OK; }
  if (!outages) return fail(GPCG_ERR_INVALID_ARG, "outages is NULL");
  cudaStream_t st = (cudaStream_t)stream;
  const size_t S = (size_t)n_out;
  // validate the outage list on the host
  std::vector<int32_t> hout(S);
  if (mem == GPCG_MEM_HOST) {
    std::memcpy(hout.data(), outages, S * 4);
  } else {
    CUDA_TRY(cudaMemcpyAsync(hout.data(), outages, S * 4, cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
  }
  if (gen) {
    for (size_t s = 0; s < S; ++s) {
      if (hout[s] < 0 || hout[s] >= c->n || c->bus_type[c->intl[hout[s]]] != GPCG_PV)
        return fail(GPCG_ERR_INVALID_ARG, "gen_buses[%zu] = %d is not a PV bus", s, hout[s]);
      hout[s] = c->intl[hout[s]];
    }
  } else {
    for (size_t s = 0; s < S; ++s)
      if (hout[s] < 0 || hout[s] >= c->m)
        return fail(GPCG_ERR_INVALID_ARG, "outages[%zu] = %d is not a branch index", s, hout[s]);
  }
  gpcg_status s_ = ensure_scen(c, S);
  if (s_ != GPCG_OK) return s_;
  CUDA_TRY(cudaMemcpyAsync(gen ? c->d_genbus : c->d_outages, hout.data(), S * 4,
                           cudaMemcpyHostToDevice, st));
  // scheduling order: heavily loaded branches first (their outages take the
  // most outer iterations), so the longest scenarios start earliest
  std::vector<int32_t> order(S);
  for (size_t s = 0; s < S; ++s) order[s] = (int32_t)s;
  if (!gen)
    std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) {
      return c->base_flow[hout[a]] > c->base_flow[hout[b]];
    });
  CUDA_TRY(cudaMemcpyAsync(c->d_order, order.data(), S * 4, cudaMemcpyHostToDevice, st));
  CUDA_TRY(cudaStreamSynchronize(st));  // the host vectors above go out of scope

  // outputs: device pointers directly; host pointers to page-locked memory
  // through their device-visible addresses (the kernels store into host
  // memory over the host link as scenarios retire, overlapped with the
  // solve); other host pointers through device staging, copied back after
  std::vector<void*> staging;
  auto stage = [&](auto* user, size_t count, auto** dev) -> cudaError_t {
    *dev = nullptr;
    if (!user) return cudaSuccess;
    if (mem == GPCG_MEM_DEVICE) { *dev = user; return cudaSuccess; }
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, user) == cudaSuccess && at.type == cudaMemoryTypeHost &&
        at.devicePointer) {
      *dev = static_cast<std::remove_reference_t<decltype(*dev)>>(at.devicePointer);
      return cudaSuccess;
    }
    cudaGetLastError();  // an unregistered pointer is not an error here
    cudaError_t ce = cudaMallocAsync((void**)dev, count * sizeof(**dev), st);
    if (ce == cudaSuccess) staging.push_back((void*)*dev);
    return ce;
  };
  double *d_theta, *d_vm, *d_flow, *d_ml;
  int32_t *d_lab, *d_iters, *d_stat, *d_nov;
  uint32_t* d_ovm;
  const size_t nw = (size_t)GPCG_MASK_WORDS(c->m);
  cudaError_t ce = cudaSuccess;
  if (ce == cudaSuccess) ce = stage(theta, S * c->n, &d_theta);
  if (ce == cudaSuccess) ce = stage(vm, S * c->n, &d_vm);
  if (ce == cudaSuccess) ce = stage(flow, S * c->m, &d_flow);
  if (ce == cudaSuccess) ce = stage(island_label, S * c->n, &d_lab);
  if (ce == cudaSuccess) ce = stage(iters, S * 3, &d_iters);
  if (ce == cudaSuccess) ce = stage(status, S, &d_stat);
  if (ce == cudaSuccess) ce = stage(max_loading, S, &d_ml);
  if (ce == cudaSuccess) ce = stage(n_overload, S, &d_nov);
  if (ce == cudaSuccess) ce = stage(overload, S * nw, &d_ovm);
  auto cleanup = [&]() { for (void* p : staging) cudaFreeAsync(p, st); };
  if (ce != cudaSuccess) {
    cleanup();
    return fail(ce == cudaErrorMemoryAllocation ? GPCG_ERR_OOM : GPCG_ERR_CUDA,
                "output staging: %s", cudaGetErrorString(ce));
  }
  if (c->phase_on && S > c->phase_cap) {
    // diagnostics: room for every scenario's start and finish times
    CUDA_TRY_C(cudaStreamSynchronize(st));
    cudaFree(c->phase);
    c->phase = nullptr;
    c->phase_cap = 0;
    CUDA_TRY_C(cudaMalloc(&c->phase, (8 + 2 * S + 4) * sizeof(unsigned long long)));
    c->phase_cap = S;
  }
  FdpfParams P = base_params(c);
  P.sc = ScenInfo{c->d_outages, c->d_lo, c->d_cnt, c->d_coef, c->d_nogen,
                  gen ? c->d_genbus : nullptr};
  P.th0 = c->th0;
  P.V0 = c->V0;
  P.c0 = c->c0;
  P.s0 = c->s0;
  P.out_theta = d_theta; P.out_vm = d_vm; P.out_flow = d_flow; P.out_maxload = d_ml;
  P.out_bus_map = c->d_bus_of_user;
  P.out_iters = d_iters; P.out_status = d_stat;
  P.out_nover = d_nov; P.out_ovmask = d_ovm;
  const bool plain = c->opt.precision == GPCG_PLAIN_FP64;
  // generator outages and reactive limits take the kernel with extension rows
  const bool ext = gen || c->G.qmax != nullptr;
  const bool f16 = c->opt.precision == GPCG_BATCHED_FP32_F16;
  const bool f32 = c->opt.precision == GPCG_BATCHED_FP32 || f16;
  // islanding for every outage (the autotuner's probes need it too)
  // (inside a stream capture the events become event-record nodes of the graph)
  auto record = [](cudaEvent_t ev, cudaStream_t s, bool cap) {
    return cap ? cudaEventRecordWithFlags(ev, s, cudaEventRecordExternal) : cudaEventRecord(ev, s);
  };
  auto enqueue_islands = [&](cudaStream_t s, bool cap = false) -> cudaError_t {
    cudaError_t e = record(c->ev[0], s, cap);
    if (e == cudaSuccess && gen)
      e = launch_gen_outages(s, (int)S, c->n, c->d_genbus, c->G.P_gen, c->isl, c->d_outages,
                             c->d_lo, c->d_cnt, c->d_coef, c->d_nogen, d_lab);
    else if (e == cudaSuccess)
      e = launch_islands(s, (int)S, c->n, c->d_outages, c->isl, nullptr, nullptr, c->d_lo,
                         c->d_cnt, c->d_coef, c->d_nogen, d_lab);
    if (e == cudaSuccess) e = record(c->ev[1], s, cap);
    return e;
  };
  gpcg_status rs = GPCG_OK;
  int T = 2, slots = 1;
  bool zs = false;
  // CTAs per SM of tile width t, with z in shared memory or not (0: does not fit)
  auto blocks = [&](int t, bool z) {
    const size_t zb = z ? make_layout(c, t, 1, f32 ? 4 : 8, true).vec_bytes : 0;
    return f32 ? fdpf_max_blocks_per_sm<float>(t, ext, zb)
               : fdpf_max_blocks_per_sm<double>(t, ext, zb);
  };
  auto use_zs = [&](int t) {
    return c->zs_allowed && !ext && (t == 2 || t == 4) && blocks(t, true) > 0;
  };
  if (!plain) {
    // tile width, tiles per SM and dense tail: fixed by the options, else
    // chosen by the autotuner for this power of two of the scenario count
    int bucket = 0;
    while (((size_t)1 << bucket) < S) ++bucket;
    const bool knobs = !c->opt.tile || !c->opt.ctas_per_sm || !c->opt.tail_rows;
    if (knobs && bucket != c->tuned_bucket) {
      const std::vector<long long> key = tune_key(c, ext, bucket);
      TuneChoice got{0, 0, 0};
      bool hit = false;
      {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) { got = it->second; hit = true; }
      }
      if (!hit) {
        auto max_ps = [&](int t) { return std::max(1, blocks(t, use_zs(t))); };
        std::vector<int> tiles = c->opt.tile ? std::vector<int>{c->opt.tile}
                                             : std::vector<int>{2, 4, 8};
        if (ext)
          for (int& t : tiles) t = std::min(t, 8);
        // the probe every candidate screens: the call's outages, or when
        // there are more than 16,384 of them (and more than eight times the
        // most scenarios a candidate keeps in flight) that many taken at an
        // even stride from the call's scheduling order, so that it mixes
        // light and heavy scenarios as the call does, every candidate does
        // the same work, and the drain at the end of a persistent launch
        // weighs as much as in the call (shorter probes favour fewer
        // scenarios in flight, which the full call does not)
        size_t lanes = 0;
        for (int t : tiles)
          lanes = std::max(lanes, (size_t)t * (c->opt.ctas_per_sm ? c->opt.ctas_per_sm
                                                                  : max_ps(t)) * c->num_sms);
        const int np = (int)std::min(S, std::max<size_t>(16384, 8 * lanes));
        std::vector<int32_t> po(np);
        for (int k = 0; k < np; ++k) po[k] = order[(size_t)k * S / np];
        {
          cudaError_t e = cudaMemcpyAsync(c->d_porder, po.data(), (size_t)np * 4,
                                          cudaMemcpyHostToDevice, st);
          if (e == cudaSuccess) e = enqueue_islands(st);
          if (e != cudaSuccess) {
            cleanup();
            return fail(GPCG_ERR_CUDA, "autotuner set-up: %s", cudaGetErrorString(e));
          }
        }
        auto rate = [&](int t, int ps, int cap, bool timed, double* out) -> gpcg_status {
          gpcg_status r = set_tail(c, cap);
          if (r != GPCG_OK) return r;
          FdpfParams Q = base_params(c);
          Q.sc = P.sc;
          Q.th0 = P.th0; Q.V0 = P.V0; Q.c0 = P.c0; Q.s0 = P.s0;
          // untimed: the first launch of a kernel variant, one tile of the
          // probe's lightest scenarios (the end of the scheduling order)
          const int nq = timed ? np : std::min(np, t);
          Q.S = nq;
          Q.n_tiles = (nq + t - 1) / t;
          Q.order = c->d_porder + (np - nq);
          const bool z = use_zs(t);
          const int sl = std::max(1, std::min(Q.n_tiles, c->num_sms * ps));
          CUDA_TRY(cudaEventRecord(c->ev[3], st));
          r = f32 ? run_fdpf<float>(c, st, Q, t, sl, f16, z)
                  : run_fdpf<double>(c, st, Q, t, sl, false, z);
          if (r != GPCG_OK) return r;
          CUDA_TRY(cudaEventRecord(c->ev[2], st));
          CUDA_TRY(cudaEventSynchronize(c->ev[2]));
          float ms = 0.f;
          CUDA_TRY(cudaEventElapsedTime(&ms, c->ev[3], c->ev[2]));
          *out = nq / std::max(ms, 1e-3f);  // scenarios per ms
          return GPCG_OK;
        };
        const int cap0 = c->opt.tail_rows > 0 ? c->opt.tail_rows
                         : (c->opt.tail_rows < 0 ? 0 : TAIL_ROWS);
        // a candidate replaces the one before it (narrower tiles, more tiles
        // per SM, the wider tail) only when it is 3 % faster: probes are
        // short, and their timing noise must not move the choice
        constexpr double MARGIN = 1.03;
        // (a) the tile width, at the most tiles per SM and the widest tail
        double best = -1.0;
        int bT = tiles[0], bP = 0, bC = cap0;
        for (int t : tiles) {
          const int ps = c->opt.ctas_per_sm ? c->opt.ctas_per_sm : max_ps(t);
          double v = 0.0;
          gpcg_status r = rate(t, ps, cap0, false, &v);  // first launch of the variant: untimed
          if (r == GPCG_OK) r = rate(t, ps, cap0, true, &v);
          if (r != GPCG_OK) { cleanup(); return r; }
          if (v > best * MARGIN) { best = v; bT = t; bP = ps; }
        }
        // (b) tiles per SM: the occupancy maximum and the two counts below it
        if (!c->opt.ctas_per_sm)
          for (int ps = max_ps(bT) - 1; ps >= std::max(1, max_ps(bT) - 2); --ps) {
            double v = 0.0;
            gpcg_status r = rate(bT, ps, cap0, true, &v);
            if (r != GPCG_OK) { cleanup(); return r; }
            if (v > best * MARGIN) { best = v; bP = ps; }
          }
        // (c) the dense tail: 248, 128, 64 rows or none
        if (!c->opt.tail_rows)
          for (int cap : {128, 64, 0}) {
            double v = 0.0;
            gpcg_status r = rate(bT, bP, cap, true, &v);
            if (r != GPCG_OK) { cleanup(); return r; }
            if (v > best * MARGIN) { best = v; bC = cap; }
          }
        got = TuneChoice{bT, bP, bC};
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune_cache[key] = got;
      }
      gpcg_status r = set_tail(c, got.tail);
      if (r != GPCG_OK) { cleanup(); return r; }
      c->tile = got.tile;
      c->per_sm = got.per_sm;
      c->tuned = hit ? 2 : 1;
      c->tuned_bucket = bucket;
    }
    T = c->opt.tile ? c->opt.tile : (c->tile ? c->tile : 2);
    if (ext) T = std::min(T, 8);  // the kernel with extension rows: tiles of 2, 4, 8
    zs = use_zs(T);
    const int n_tiles = (int)((S + T - 1) / T);
    int per_sm = c->opt.ctas_per_sm ? c->opt.ctas_per_sm : c->per_sm;
    if (!c->opt.ctas_per_sm && per_sm > blocks(T, zs)) per_sm = blocks(T, zs);
    if (per_sm == 0 || (zs && per_sm > blocks(T, true))) per_sm = blocks(T, zs);
    per_sm = std::max(per_sm, 1);
    c->per_sm_used = per_sm;
    slots = std::max(1, std::min(n_tiles, c->num_sms * per_sm));
    P.S = (int)S;
    P.n_tiles = n_tiles;
    P.order = c->d_order;
  }
  if (c->phase_on) CUDA_TRY_C(cudaMemsetAsync(c->phase, 0, (8 + 2 * S + 4) * sizeof(unsigned long long), st));
  if (plain && !ext) {
    // one scenario at a time, each spread over the whole GPU (cooperative
    // launches with grid-wide barriers): no batching across scenarios
    CUDA_TRY_C(enqueue_islands(st));
    rs = ensure_plain(c);
    if (rs != GPCG_OK) { cleanup(); return rs; }
    CUDA_TRY_C(cudaMemsetAsync(c->plainb.bar, 0, 2 * sizeof(unsigned int), st));
    CUDA_TRY_C(cudaMemsetAsync(c->plainb.err, 0, sizeof(int), st));
    c->plainb.wait_limit = c->opt.wait_limit > 0 ? (unsigned)c->opt.wait_limit : (1u << 25);
    P.S = (int)S;
    P.phase_cycles = nullptr;
    const DevMatT<double> MPd = c->MP.view<double>(), MQd = c->MQ.view<double>();
    for (size_t s = 0; s < S; ++s)
      CUDA_TRY_C(launch_plain(st, c->plain_grid_size, P, MPd, MQd, c->plainb, (int)s));
    int32_t herr = 0;
    CUDA_TRY_C(cudaMemcpyAsync(&herr, c->plainb.err, sizeof herr, cudaMemcpyDeviceToHost, st));
    CUDA_TRY_C(cudaStreamSynchronize(st));
    if (herr) {
      cleanup();
      return fail(GPCG_ERR_TIMEOUT, "plain path: a grid-wide barrier wait gave up");
    }
  } else if (plain) {
    CUDA_TRY_C(enqueue_islands(st));
    // one scenario at a time: no batching across scenarios (the kernel with
    // extension rows, one CTA per scenario)
    for (size_t s = 0; s < S && rs == GPCG_OK; ++s) {
      FdpfParams Q = P;
      Q.S = 1;
      Q.n_tiles = 1;
      Q.sc = ScenInfo{c->d_outages + s, c->d_lo + s, c->d_cnt + s, c->d_coef + s, c->d_nogen + s,
                      gen ? c->d_genbus + s : nullptr};
      Q.out_theta = d_theta ? d_theta + s * c->n : nullptr;
      Q.out_vm = d_vm ? d_vm + s * c->n : nullptr;
      Q.out_flow = d_flow ? d_flow + s * c->m : nullptr;
      Q.out_maxload = d_ml ? d_ml + s : nullptr;
      Q.out_iters = d_iters ? d_iters + 3 * s : nullptr;
      Q.out_status = d_stat ? d_stat + s : nullptr;
      Q.out_nover = d_nov ? d_nov + s : nullptr;
      Q.out_ovmask = d_ovm ? d_ovm + s * nw : nullptr;
      rs = run_fdpf<double>(c, st, Q, 2, 1);
    }
  } else if (mem == GPCG_MEM_DEVICE && !c->phase_on) {
    // device mode: islanding + solve as one CUDA graph, captured on the
    // context's own stream for this argument set and replayed on `st`
    Layout Lo = make_layout(c, T, slots, f32 ? 4 : 8, zs);
    s_ = ensure_work(c, Lo.bytes);
    if (s_ != GPCG_OK) { cleanup(); return s_; }
    std::vector<uintptr_t> key = {S, (uintptr_t)T, (uintptr_t)slots,
                                  (uintptr_t)c->opt.precision, (uintptr_t)c->opt.precond,
                                  (uintptr_t)c->work, (uintptr_t)d_theta, (uintptr_t)d_vm,
                                  (uintptr_t)d_flow, (uintptr_t)d_lab, (uintptr_t)d_iters,
                                  (uintptr_t)d_stat, (uintptr_t)d_ml, (uintptr_t)d_nov,
                                  (uintptr_t)d_ovm, (uintptr_t)c->d_outages,
                                  (uintptr_t)c->d_order, (uintptr_t)c->d_lo, (uintptr_t)gen,
                                  (uintptr_t)zs};
    {
      double opts[3] = {c->opt.tol, c->opt.inner_rtol, 0.0};
      uintptr_t bits[3];
      std::memcpy(bits, opts, sizeof bits);
      key.insert(key.end(), {bits[0], bits[1], (uintptr_t)c->opt.max_outer,
                             (uintptr_t)c->opt.max_inner});
    }
    if (!c->graph || key != c->graph_key) {
      if (c->graph) { cudaGraphExecDestroy(c->graph); c->graph = nullptr; }
      cudaGraph_t gr = nullptr;
      CUDA_TRY_C(cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
      cudaError_t e = enqueue_islands(c->cap_stream, true);
      if (e == cudaSuccess) {
        rs = f32 ? run_fdpf<float>(c, c->cap_stream, P, T, slots, f16, zs)
                 : run_fdpf<double>(c, c->cap_stream, P, T, slots, false, zs);
        if (rs == GPCG_OK) e = record(c->ev[2], c->cap_stream, true);
      }
      cudaError_t e2 = cudaStreamEndCapture(c->cap_stream, &gr);
      if (rs != GPCG_OK) { if (gr) cudaGraphDestroy(gr); cleanup(); return rs; }
      if (e == cudaSuccess) e = e2;
      if (e == cudaSuccess) e = cudaGraphInstantiate(&c->graph, gr, 0);
      if (gr) cudaGraphDestroy(gr);
      if (e != cudaSuccess) { c->graph = nullptr; cleanup(); return fail(GPCG_ERR_CUDA, "graph: %s", cudaGetErrorString(e)); }
      c->graph_key = key;
    }
    CUDA_TRY_C(cudaGraphLaunch(c->graph, st));
    c->timed = true;
    g_err.clear();
    return GPCG_OK;
  } else {
    CUDA_TRY_C(enqueue_islands(st));
    rs = f32 ? run_fdpf<float>(c, st, P, T, slots, f16, zs)
             : run_fdpf<double>(c, st, P, T, slots, false, zs);
  }
  if (rs != GPCG_OK) { cleanup(); return rs; }
  CUDA_TRY_C(cudaEventRecord(c->ev[2], st));
  c->timed = true;
  if (c->phase_on) {
    // diagnostics requested through GPCG_PHASE_TIMERS=1: SM cycles per phase,
    // summed over CTAs (thread 0 of each CTA)
    unsigned long long h[8];
    CUDA_TRY_C(cudaMemcpyAsync(h, c->phase, sizeof h, cudaMemcpyDeviceToHost, st));
    CUDA_TRY_C(cudaStreamSynchronize(st));
    static const char* names[8] = {"init", "mismatchP", "pcgP", "updateP", "mismatchQ",
                                   "pcgQ", "updateQ", "output"};
    double tot = 0;
    for (int k = 0; k < 8; ++k) tot += (double)h[k];
    std::fprintf(stderr, "gpcg phase cycles (sum over CTAs):");
    for (int k = 0; k < 8; ++k) std::fprintf(stderr, " %s=%.1f%%", names[k], 100.0 * h[k] / tot);
    std::fprintf(stderr, " total=%.3e\n", tot);
    if (!plain) {
      unsigned long long sub[3];
      CUDA_TRY_C(cudaMemcpy(sub, c->phase + 8 + 2 * S, sizeof sub, cudaMemcpyDeviceToHost));
      std::fprintf(stderr, "gpcg inner-solve cycles: spmv=%.1f%% fwd=%.1f%% bwd=%.1f%% of all\n",
                   100.0 * sub[0] / tot, 100.0 * sub[1] / tot, 100.0 * sub[2] / tot);
    }
  }
  if (c->phase_on && !plain) {
    // per-scenario start and finish times: completion profile and the
    // longest scenarios (the tail of the persistent launch)
    std::vector<unsigned long long> tt(2 * S);
    CUDA_TRY_C(cudaMemcpy(tt.data(), c->phase + 8, 2 * S * sizeof(unsigned long long),
                        cudaMemcpyDeviceToHost));
    unsigned long long t0 = ~0ull, t1 = 0;
    for (size_t k = 0; k < S; ++k) {
      t0 = std::min(t0, tt[2 * k]);
      t1 = std::max(t1, tt[2 * k + 1]);
    }
    std::vector<double> fin(S), dur(S);
    for (size_t k = 0; k < S; ++k) {
      fin[k] = 1e-6 * (double)(tt[2 * k + 1] - t0);
      dur[k] = 1e-6 * (double)(tt[2 * k + 1] - tt[2 * k]);
    }
    std::vector<double> fs = fin, ds = dur;
    std::sort(fs.begin(), fs.end());
    std::sort(ds.begin(), ds.end());
    auto q = [&](const std::vector<double>& v, double f) {
      return v[std::min(v.size() - 1, (size_t)(f * (double)(v.size() - 1)))];
    };
    std::fprintf(stderr,
                 "gpcg scenario finish (ms after the first start): 50%% %.2f, 90%% %.2f, "
                 "99%% %.2f, last %.2f; scenario durations: median %.2f, 99%% %.2f, max %.2f\n",
                 q(fs, 0.5), q(fs, 0.9), q(fs, 0.99), 1e-6 * (double)(t1 - t0), q(ds, 0.5),
                 q(ds, 0.99), ds.back());
    size_t kmax = 0;
    for (size_t k = 0; k < S; ++k)
      if (dur[k] > dur[kmax]) kmax = k;
    std::fprintf(stderr, "gpcg longest scenario: index %zu (outage %d), start %.2f ms, %.2f ms\n",
                 kmax, hout[kmax], 1e-6 * (double)(tt[2 * kmax] - t0), dur[kmax]);
  }
  if (mem == GPCG_MEM_HOST) {
    auto back = [&](auto* user, auto* dev, size_t count) -> cudaError_t {
      if (!user) return cudaSuccess;
      if (std::find(staging.begin(), staging.end(), (void*)dev) == staging.end())
        return cudaSuccess;  // written in place (page-locked host memory)
      return cudaMemcpyAsync(user, dev, count * sizeof(*user), cudaMemcpyDeviceToHost, st);
    };
    if (ce == cudaSuccess) ce = back(theta, d_theta, S * c->n);
    if (ce == cudaSuccess) ce = back(vm, d_vm, S * c->n);
    if (ce == cudaSuccess) ce = back(flow, d_flow, S * c->m);
    if (ce == cudaSuccess) ce = back(island_label, d_lab, S * c->n);
    if (ce == cudaSuccess) ce = back(iters, d_iters, S * 3);
    if (ce == cudaSuccess) ce = back(status, d_stat, S);
    if (ce == cudaSuccess) ce = back(max_loading, d_ml, S);
    if (ce == cudaSuccess) ce = back(n_overload, d_nov, S);
    if (ce == cudaSuccess) ce = back(overload, d_ovm, S * nw);
    cleanup();
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
    if (ce != cudaSuccess) return fail(GPCG_ERR_CUDA, "n1_screen: %s", cudaGetErrorString(ce));
  }
  g_err.clear();
  return GPCG_OK;
}

extern "C" gpcg_status gpcg_n1_screen(gpcg_ctx* c, const int32_t* outages, int32_t n_out,
                                      int32_t mem, void* stream, double* theta, double* vm,
                                      double* flow, int32_t* island_label, int32_t* iters,
                                      int32_t* status, double* max_loading, int32_t* n_overload,
                                      uint32_t* overload) {
  return n1_screen_impl(c, outages, n_out, mem, stream, theta, vm, flow, island_label, iters,
                        status, max_loading, n_overload, overload, false);
}

extern "C" gpcg_status gpcg_n1_gen_screen(gpcg_ctx* c, const int32_t* gen_buses, int32_t n_out,
                                          int32_t mem, void* stream, double* theta, double* vm,
                                          double* flow, int32_t* island_label, int32_t* iters,
                                          int32_t* status, double* max_loading,
                                          int32_t* n_overload, uint32_t* overload) {
  return n1_screen_impl(c, gen_buses, n_out, mem, stream, theta, vm, flow, island_label, iters,
                        status, max_loading, n_overload, overload, true);
}

// ------------------------------------------------------------------ adjoint
static gpcg_status ensure_adj_matrix(gpcg_ctx* c) {
  if (c->ma_ready) return GPCG_OK;
  MatDev& M = c->MA;
  M = c->MP;  // structure shared; values replaced below
  M.lsc = nullptr;  // the adjoint solves in FP64: no scaled FP16 factor
  M.xch = M.xrh = nullptr;
  M.L.valh = M.L.ovalh = M.U.valh = M.U.ovalh = nullptr;
  auto& own = c->adj_owned;
  const int n = M.plan.n, nnz = M.plan.A.nnz(), nl = M.plan.L.nnz();
  CUDA_TRY(dalloc(own, &M.a_val, nnz));
  CUDA_TRY(dalloc(own, &M.l_val, nl));
  CUDA_TRY(dalloc(own, &M.diag, n));
  CUDA_TRY(dalloc(own, &M.diag32, n));
  CUDA_TRY(dalloc(own, &M.inv_diag, n));
  CUDA_TRY(dalloc(own, &M.inv_diag32, n));
  {
    const size_t nt = (size_t)(n - M.plan.tail_row0);
    CUDA_TRY(dalloc(own, &M.xc, nt * nt));
    CUDA_TRY(dalloc(own, &M.xr, nt * nt));
    CUDA_TRY(dalloc(own, &M.xc32, nt * nt));
    CUDA_TRY(dalloc(own, &M.xr32, nt * nt));
  }
  for (EllDev* E : {&M.A, &M.L, &M.U}) {
    CUDA_TRY(dalloc(own, &E->val, E->nslot));
    CUDA_TRY(dalloc(own, &E->val32, E->nslot));
    CUDA_TRY(dalloc(own, &E->oval, E->nover));
    CUDA_TRY(dalloc(own, &E->oval32, E->nover));
  }
  c->ma_ready = true;
  return GPCG_OK;
}

extern "C" gpcg_status gpcg_n1_adjoint(gpcg_ctx* c, const int32_t* outages, int32_t n_out,
                                       int32_t mem, void* stream, const double* P_in,
                                       const double* b_in, double* loss, double* dL_dP,
                                       double* dL_db) {
  if (!c) return fail(GPCG_ERR_INVALID_ARG, "gpcg_n1_adjoint: ctx is NULL");
  if (n_out < 0 || !loss) return fail(GPCG_ERR_INVALID_ARG, "n_out < 0 or loss is NULL");
  if (mem != GPCG_MEM_HOST && mem != GPCG_MEM_DEVICE)
    return fail(GPCG_ERR_INVALID_ARG, "mem must be 0 (host) or 1 (device)");
  if (n_out > 0 && !outages) return fail(GPCG_ERR_INVALID_ARG, "outages is NULL");
  cudaStream_t st = (cudaStream_t)stream;
  const int n = c->n, m = c->m;
  const size_t S = (size_t)n_out;
  std::vector<int32_t> hout(S);
  if (S) {
    if (mem == GPCG_MEM_HOST) std::memcpy(hout.data(), outages, S * 4);
    else {
      CUDA_TRY(cudaMemcpyAsync(hout.data(), outages, S * 4, cudaMemcpyDeviceToHost, st));
      CUDA_TRY(cudaStreamSynchronize(st));
    }
  }
  for (size_t s = 0; s < S; ++s)
    if (hout[s] < 0 || hout[s] >= m)
      return fail(GPCG_ERR_INVALID_ARG, "outages[%zu] = %d is not a branch index", s, hout[s]);
  std::vector<double> hb;
  if (b_in) {
    hb.resize(m);
    if (mem == GPCG_MEM_HOST) std::memcpy(hb.data(), b_in, (size_t)m * 8);
    else {
      CUDA_TRY(cudaMemcpyAsync(hb.data(), b_in, (size_t)m * 8, cudaMemcpyDeviceToHost, st));
      CUDA_TRY(cudaStreamSynchronize(st));
    }
    for (int k = 0; k < m; ++k)
      if (!(hb[k] > 0) || !std::isfinite(hb[k]))
        return fail(GPCG_ERR_INVALID_ARG, "b[%d] = %g: susceptances must be positive", k, hb[k]);
  }
  gpcg_status s_ = ensure_scen(c, std::max<size_t>(S, 1));
  if (s_ != GPCG_OK) return s_;
  s_ = ensure_adj_matrix(c);
  if (s_ != GPCG_OK) return s_;
  // inputs on the device: P in the caller's and in the internal bus order, b
  double *dPu = nullptr, *dPi = nullptr, *db = nullptr;
  std::vector<void*> tmp;
  auto cleanup = [&]() { for (void* p : tmp) cudaFree(p); };
  auto alloc = [&](double** p, size_t cnt) -> cudaError_t {
    cudaError_t ce = cudaMalloc((void**)p, cnt * 8);
    if (ce == cudaSuccess) tmp.push_back(*p);
    return ce;
  };
  cudaError_t ce = alloc(&dPi, n);
  if (ce == cudaSuccess) {
    if (!P_in) dPu = c->u_P_sched;
    else if (mem == GPCG_MEM_DEVICE) dPu = const_cast<double*>(P_in);
    else if ((ce = alloc(&dPu, n)) == cudaSuccess)
      ce = cudaMemcpy(dPu, P_in, (size_t)n * 8, cudaMemcpyHostToDevice);
  }
  if (ce == cudaSuccess) {
    if (!b_in) db = c->wP;
    else if ((ce = alloc(&db, m)) == cudaSuccess)
      ce = cudaMemcpy(db, hb.data(), (size_t)m * 8, cudaMemcpyHostToDevice);
  }
  if (ce == cudaSuccess) ce = launch_gather_perm(st, n, c->G.user_of_bus, dPu, dPi);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
  if (ce != cudaSuccess) { cleanup(); return fail(GPCG_ERR_CUDA, "adjoint inputs: %s", cudaGetErrorString(ce)); }
  // base-case B' with the given susceptances, and its factor
  s_ = fill_values(c, c->MA, db);
  if (s_ != GPCG_OK) { cleanup(); return s_; }
  // outputs (device staging in host mode)
  double *oL = nullptr, *oP = nullptr, *ob = nullptr;
  if (mem == GPCG_MEM_DEVICE) { oL = loss; oP = dL_dP; ob = dL_db; }
  else {
    if ((ce = alloc(&oL, 1)) == cudaSuccess && dL_dP) ce = alloc(&oP, n);
    if (ce == cudaSuccess && dL_db) ce = alloc(&ob, m);
    if (ce != cudaSuccess) { cleanup(); return fail(GPCG_ERR_OOM, "adjoint outputs: %s", cudaGetErrorString(ce)); }
  }
  const int T = 2;
  const int n_tiles = (int)((S + T - 1) / T);
  const int per_sm = std::max(1, adjoint_max_blocks_per_sm());
  const int slots = std::max(1, std::min(n_tiles, c->num_sms * per_sm));
  const size_t acc_bytes = (size_t)slots * ((size_t)n + m + 1) * 8;
  if (acc_bytes > c->adj_acc_bytes) {
    if (c->adj_acc) cudaFree(c->adj_acc);
    c->adj_acc = nullptr;
    c->adj_acc_bytes = 0;
    ce = cudaMalloc(&c->adj_acc, acc_bytes);
    if (ce != cudaSuccess) { cleanup(); return fail(GPCG_ERR_OOM, "adjoint sums: %s", cudaGetErrorString(ce)); }
    c->adj_acc_bytes = acc_bytes;
  }
  double* accP = c->adj_acc;
  double* accb = accP + (size_t)slots * n;
  double* accL = accb + (size_t)slots * m;
  if (S) {
    CUDA_TRY_C(cudaMemcpyAsync(c->d_outages, hout.data(), S * 4, cudaMemcpyHostToDevice, st));
    ce = launch_islands(st, (int)S, n, c->d_outages, c->isl, P_in ? dPu : nullptr, c->d_prefP,
                        c->d_lo, c->d_cnt, c->d_coef, c->d_nogen, nullptr);
    if (ce != cudaSuccess) { cleanup(); return fail(GPCG_ERR_CUDA, "islands: %s", cudaGetErrorString(ce)); }
    FdpfParams P = base_params(c);
    P.phase_cycles = nullptr;  // the diagnostics cover the N-1 screens
    P.inner_rtol = 1e-12;  // gradients want converged solves (2-3 iterations with the exact factor)
    P.max_inner = std::max(c->opt.max_inner, 2000);
    P.S = (int)S;
    P.n_tiles = n_tiles;
    P.sc = ScenInfo{c->d_outages, c->d_lo, c->d_cnt, c->d_coef, c->d_nogen};
    Layout Lo = make_layout(c, T, slots, 8);
    s_ = ensure_work(c, Lo.bytes);
    if (s_ != GPCG_OK) { cleanup(); return s_; }
    char* base = (char*)c->work;
    const size_t vb = (size_t)slots * Lo.vec_bytes;
    const size_t ss = (((Lo.sstride * 8 + 255) / 256) * 256) / 8;
    P.wx = base; P.wr = base + vb; P.wp = base + 2 * vb; P.wq = base + 3 * vb; P.wz = base + 4 * vb;
    P.vstride = Lo.vec_bytes / 8;
    double* sbase = (double*)(base + 5 * vb);
    P.wth = sbase; P.wV = sbase + slots * ss; P.we = sbase + 2 * slots * ss;
    P.wf = sbase + 3 * slots * ss;
    P.sstride = ss;
    P.tile_counter = c->d_counter;
    CUDA_TRY(cudaMemsetAsync(c->d_counter, 0, sizeof(int32_t), st));
    AdjParamsView A{dPi, db, accP, accb, accL};
    ce = launch_adjoint(st, slots, P, A, c->MA.view<double>());
    if (ce == cudaSuccess) ce = launch_slot_sum(st, 1, slots, accL, nullptr, oL);
    if (ce == cudaSuccess && oP) ce = launch_slot_sum(st, n, slots, accP, c->G.user_of_bus, oP);
    if (ce == cudaSuccess && ob) ce = launch_slot_sum(st, m, slots, accb, nullptr, ob);
  } else {
    if (ce == cudaSuccess) ce = cudaMemsetAsync(oL, 0, 8, st);
    if (ce == cudaSuccess && oP) ce = cudaMemsetAsync(oP, 0, (size_t)n * 8, st);
    if (ce == cudaSuccess && ob) ce = cudaMemsetAsync(ob, 0, (size_t)m * 8, st);
  }
  if (ce != cudaSuccess) { cleanup(); return fail(GPCG_ERR_CUDA, "adjoint: %s", cudaGetErrorString(ce)); }
  if (mem == GPCG_MEM_HOST) {
    ce = cudaMemcpyAsync(loss, oL, 8, cudaMemcpyDeviceToHost, st);
    if (ce == cudaSuccess && dL_dP) ce = cudaMemcpyAsync(dL_dP, oP, (size_t)n * 8, cudaMemcpyDeviceToHost, st);
    if (ce == cudaSuccess && dL_db) ce = cudaMemcpyAsync(dL_db, ob, (size_t)m * 8, cudaMemcpyDeviceToHost, st);
  }
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);  // temporaries are freed below
  cleanup();
  if (ce != cudaSuccess) return fail(GPCG_ERR_CUDA, "adjoint: %s", cudaGetErrorString(ce));
  g_err.clear();
  return GPCG_OK;
}

// ---------------------------------------------------------- DC quick screen
extern "C" gpcg_status gpcg_n1_dc_screen(gpcg_ctx* c, const int32_t* outages, int32_t n_out,
                                         int32_t mem, void* stream, const double* P_in,
                                         double* theta, double* flow, int32_t* iters,
                                         int32_t* status, double* max_loading,
                                         int32_t* n_overload, uint32_t* overload) {
  if (!c) return fail(GPCG_ERR_INVALID_ARG, "gpcg_n1_dc_screen: ctx is NULL");
  if (n_out < 0) return fail(GPCG_ERR_INVALID_ARG, "n_out < 0");
  if (mem != GPCG_MEM_HOST && mem != GPCG_MEM_DEVICE)
    return fail(GPCG_ERR_INVALID_ARG, "mem must be 0 (host) or 1 (device)");
  if (n_out == 0) { g_err.clear(); return GPCG_OK; }
  if (!outages) return fail(GPCG_ERR_INVALID_ARG, "outages is NULL");
  if (c->opt.precision == GPCG_PLAIN_FP64)
    return fail(GPCG_ERR_INVALID_ARG, "gpcg_n1_dc_screen runs batched (precision 1, 2 or 3)");
  cudaStream_t st = (cudaStream_t)stream;
  const int n = c->n, m = c->m;
  const size_t S = (size_t)n_out;
  std::vector<int32_t> hout(S);
  if (mem == GPCG_MEM_HOST) std::memcpy(hout.data(), outages, S * 4);
  else {
    CUDA_TRY(cudaMemcpyAsync(hout.data(), outages, S * 4, cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
  }
  for (size_t s = 0; s < S; ++s)
    if (hout[s] < 0 || hout[s] >= m)
      return fail(GPCG_ERR_INVALID_ARG, "outages[%zu] = %d is not a branch index", s, hout[s]);
  gpcg_status s_ = ensure_scen(c, S);
  if (s_ != GPCG_OK) return s_;
  std::vector<void*> tmp;
  auto cleanup = [&]() { for (void* p : tmp) cudaFreeAsync(p, st); };
  auto alloc = [&](void** p, size_t bytes) -> cudaError_t {
    cudaError_t ce = cudaMallocAsync(p, bytes, st);
    if (ce == cudaSuccess) tmp.push_back(*p);
    return ce;
  };
  // injections: the caller's (host or device, caller's bus order) or P_sched
  double *dPu = c->u_P_sched, *dPi = nullptr;
  cudaError_t ce = alloc((void**)&dPi, (size_t)n * 8);
  if (ce == cudaSuccess && P_in) {
    if (mem == GPCG_MEM_DEVICE) dPu = const_cast<double*>(P_in);
    else if ((ce = alloc((void**)&dPu, (size_t)n * 8)) == cudaSuccess)
      ce = cudaMemcpyAsync(dPu, P_in, (size_t)n * 8, cudaMemcpyHostToDevice, st);
  }
  if (ce == cudaSuccess) ce = launch_gather_perm(st, n, c->G.user_of_bus, dPu, dPi);
  // outputs: device pointers directly, or device staging for host pointers
  auto stage = [&](auto* user, size_t count, auto** dev) -> cudaError_t {
    *dev = nullptr;
    if (!user) return cudaSuccess;
    if (mem == GPCG_MEM_DEVICE) { *dev = user; return cudaSuccess; }
    return alloc((void**)dev, count * sizeof(**dev));
  };
  double *d_th = nullptr, *d_fl = nullptr, *d_ml = nullptr;
  int32_t *d_it = nullptr, *d_st = nullptr, *d_nov = nullptr;
  uint32_t* d_ovm = nullptr;
  const size_t nw = (size_t)GPCG_MASK_WORDS(m);
  if (ce == cudaSuccess) ce = stage(n_overload, S, &d_nov);
  if (ce == cudaSuccess) ce = stage(overload, S * nw, &d_ovm);
  if (ce == cudaSuccess) ce = stage(theta, S * n, &d_th);
  if (ce == cudaSuccess) ce = stage(flow, S * m, &d_fl);
  if (ce == cudaSuccess) ce = stage(max_loading, S, &d_ml);
  if (ce == cudaSuccess) ce = stage(iters, S, &d_it);
  if (ce == cudaSuccess) ce = stage(status, S, &d_st);
  if (ce != cudaSuccess) {
    cleanup();
    return fail(ce == cudaErrorMemoryAllocation ? GPCG_ERR_OOM : GPCG_ERR_CUDA,
                "dc screen buffers: %s", cudaGetErrorString(ce));
  }
  CUDA_TRY_C(cudaMemcpyAsync(c->d_outages, hout.data(), S * 4, cudaMemcpyHostToDevice, st));
  ce = launch_islands(st, (int)S, n, c->d_outages, c->isl, P_in ? dPu : nullptr, c->d_prefP,
                      c->d_lo, c->d_cnt, c->d_coef, c->d_nogen, nullptr);
  if (ce != cudaSuccess) { cleanup(); return fail(GPCG_ERR_CUDA, "islands: %s", cudaGetErrorString(ce)); }
  const bool f16 = c->opt.precision == GPCG_BATCHED_FP32_F16;
  const bool f32 = c->opt.precision == GPCG_BATCHED_FP32 || f16;
  const int T = 2;
  const int n_tiles = (int)((S + T - 1) / T);
  const int per_sm = std::max(1, f32 ? dc_max_blocks_per_sm<float>() : dc_max_blocks_per_sm<double>());
  const int slots = std::max(1, std::min(n_tiles, c->num_sms * per_sm));
  FdpfParams P = base_params(c);
  P.phase_cycles = nullptr;  // the diagnostics cover the AC screens
  // converged solves (2-3 iterations with the exact factor); FP32 solves are
  // followed by one refinement step in the kernel
  P.inner_rtol = std::min(c->opt.inner_rtol, f32 ? 1e-6 : 1e-12);
  P.S = (int)S;
  P.n_tiles = n_tiles;
  P.sc = ScenInfo{c->d_outages, c->d_lo, c->d_cnt, c->d_coef, c->d_nogen};
  const size_t vt = f32 ? 4 : 8;
  Layout Lo = make_layout(c, T, slots, vt);
  s_ = ensure_work(c, Lo.bytes);
  if (s_ != GPCG_OK) { cleanup(); return s_; }
  char* base = (char*)c->work;
  const size_t vb = (size_t)slots * Lo.vec_bytes;
  const size_t ss = (((Lo.sstride * 8 + 255) / 256) * 256) / 8;
  P.wx = base; P.wr = base + vb; P.wp = base + 2 * vb; P.wq = base + 3 * vb; P.wz = base + 4 * vb;
  P.vstride = Lo.vec_bytes / vt;
  double* sbase = (double*)(base + 5 * vb);
  P.wth = sbase; P.wV = sbase + slots * ss; P.we = sbase + 2 * slots * ss;
  P.wf = sbase + 3 * slots * ss;
  P.sstride = ss;
  DcParamsView D{dPi, c->G.user_of_bus, d_th, d_fl, d_ml, d_it, d_st, d_nov, d_ovm};
  ce = f32 ? launch_dc<float>(st, slots, P, D, c->MP.view<float>(f16), c->MP.view<double>())
           : launch_dc<double>(st, slots, P, D, c->MP.view<double>(), c->MP.view<double>());
  if (ce != cudaSuccess) { cleanup(); return fail(GPCG_ERR_CUDA, "dc screen: %s", cudaGetErrorString(ce)); }
  if (mem == GPCG_MEM_HOST) {
    auto back = [&](auto* user, auto* dev, size_t count) -> cudaError_t {
      if (!user) return cudaSuccess;
      return cudaMemcpyAsync(user, dev, count * sizeof(*user), cudaMemcpyDeviceToHost, st);
    };
    if (ce == cudaSuccess) ce = back(theta, d_th, S * n);
    if (ce == cudaSuccess) ce = back(flow, d_fl, S * m);
    if (ce == cudaSuccess) ce = back(max_loading, d_ml, S);
    if (ce == cudaSuccess) ce = back(iters, d_it, S);
    if (ce == cudaSuccess) ce = back(status, d_st, S);
    if (ce == cudaSuccess) ce = back(n_overload, d_nov, S);
    if (ce == cudaSuccess) ce = back(overload, d_ovm, S * nw);
  }
  cleanup();  // stream-ordered frees: after the kernel and the copies
  if (mem == GPCG_MEM_HOST && ce == cudaSuccess) ce = cudaStreamSynchronize(st);
  if (ce != cudaSuccess) return fail(GPCG_ERR_CUDA, "dc screen: %s", cudaGetErrorString(ce));
  g_err.clear();
  return GPCG_OK;
}

extern "C" gpcg_status gpcg_apply(gpcg_ctx* c, int32_t which, int32_t op, const int32_t* outages,
                                  int32_t S, int32_t precision, const double* X, double* Y) {
  if (!c || !outages || !X || !Y || S < 0)
    return fail(GPCG_ERR_INVALID_ARG, "gpcg_apply: NULL argument or S < 0");
  if ((which != 0 && which != 1) || (op != 0 && op != 1))
    return fail(GPCG_ERR_INVALID_ARG, "gpcg_apply: which and op must be 0 or 1");
  if (precision != GPCG_BATCHED_FP32 && precision != GPCG_BATCHED_FP64 &&
      precision != GPCG_BATCHED_FP32_F16)
    return fail(GPCG_ERR_INVALID_ARG, "gpcg_apply: precision must be 1, 2 or 3");
  if (S == 0) { g_err.clear(); return GPCG_OK; }
  for (int s = 0; s < S; ++s)
    if (outages[s] < -1 || outages[s] >= c->m)
      return fail(GPCG_ERR_INVALID_ARG, "gpcg_apply: outage %d out of range", outages[s]);
  const MatDev& M = which ? c->MQ : c->MP;
  const int rows = M.plan.n;
  const size_t vt = precision == GPCG_BATCHED_FP64 ? 8 : 4;
  const int T = 32;
  const int grid = std::max(1, std::min((S + T - 1) / T, c->num_sms * 2));
  const size_t vstride = (size_t)(rows + 1) * T;
  int32_t* d_out = nullptr;
  double *dX = nullptr, *dY = nullptr;
  void* wbuf = nullptr;
  gpcg_status rs = GPCG_OK;
  cudaError_t ce = cudaMalloc(&d_out, (size_t)S * 4);
  if (ce == cudaSuccess) ce = cudaMalloc(&dX, (size_t)S * rows * 8 + 8);
  if (ce == cudaSuccess) ce = cudaMalloc(&dY, (size_t)S * rows * 8 + 8);
  if (ce == cudaSuccess) ce = cudaMalloc(&wbuf, (size_t)grid * 3 * vstride * vt + 16);
  if (ce == cudaSuccess) ce = cudaMemcpy(d_out, outages, (size_t)S * 4, cudaMemcpyHostToDevice);
  if (ce == cudaSuccess) ce = cudaMemcpy(dX, X, (size_t)S * rows * 8, cudaMemcpyHostToDevice);
  if (ce == cudaSuccess) {
    if (vt == 4)
      ce = launch_apply<float>(0, grid, M.view<float>(precision == GPCG_BATCHED_FP32_F16), op, S,
                               d_out, c->G.f, c->G.t, dX, dY,
                               (float*)wbuf, vstride, c->opt.precond);
    else
      ce = launch_apply<double>(0, grid, M.view<double>(), op, S, d_out, c->G.f, c->G.t, dX, dY,
                                (double*)wbuf, vstride, c->opt.precond);
  }
  if (ce == cudaSuccess) ce = cudaDeviceSynchronize();
  if (ce == cudaSuccess) ce = cudaMemcpy(Y, dY, (size_t)S * rows * 8, cudaMemcpyDeviceToHost);
  if (ce != cudaSuccess) rs = fail(GPCG_ERR_CUDA, "gpcg_apply: %s", cudaGetErrorString(ce));
  cudaFree(d_out); cudaFree(dX); cudaFree(dY); cudaFree(wbuf);
  if (rs == GPCG_OK) g_err.clear();
  return rs;
}

extern "C" gpcg_status gpcg_export_matrix(const gpcg_ctx* c, int32_t which, int32_t* bus_of_row,
                                          int32_t* rowptr, int32_t* col, double* val,
                                          int32_t* lrowptr, int32_t* lcol, double* lval,
                                          int32_t* level) {
  if (!c) return fail(GPCG_ERR_INVALID_ARG, "gpcg_export_matrix: ctx is NULL");
  if (which != 0 && which != 1) return fail(GPCG_ERR_INVALID_ARG, "which must be 0 or 1");
  const MatDev& M = which ? c->MQ : c->MP;
  const MatrixPlan& P = M.plan;
  if (bus_of_row)
    for (int i = 0; i < P.n; ++i) bus_of_row[i] = c->user_of[P.bus_of_row[i]];
  if (rowptr) std::memcpy(rowptr, P.A.ptr.data(), P.A.ptr.size() * 4);
  if (col) std::memcpy(col, P.A.idx.data(), P.A.idx.size() * 4);
  if (lrowptr) std::memcpy(lrowptr, P.L.ptr.data(), P.L.ptr.size() * 4);
  if (lcol) std::memcpy(lcol, P.L.idx.data(), P.L.idx.size() * 4);
  if (level) std::memcpy(level, P.level.data(), (size_t)P.n * 4);
  if (val) CUDA_TRY(cudaMemcpy(val, M.a_val, (size_t)P.A.nnz() * 8, cudaMemcpyDeviceToHost));
  if (lval) CUDA_TRY(cudaMemcpy(lval, M.l_val, (size_t)P.L.nnz() * 8, cudaMemcpyDeviceToHost));
  g_err.clear();
  return GPCG_OK;
}

extern "C" gpcg_status gpcg_last_timings(gpcg_ctx* c, float* ms) {
  if (!c || !ms) return fail(GPCG_ERR_INVALID_ARG, "gpcg_last_timings: NULL argument");
  if (!c->timed) return fail(GPCG_ERR_NOT_READY, "no N-1 screen has run");
  CUDA_TRY(cudaEventSynchronize(c->ev[2]));
  CUDA_TRY(cudaEventElapsedTime(&ms[0], c->ev[0], c->ev[1]));
  CUDA_TRY(cudaEventElapsedTime(&ms[1], c->ev[1], c->ev[2]));
  g_err.clear();
  return GPCG_OK;
}

extern "C" gpcg_status gpcg_analyze(const gpcg_grid* g, int32_t precond, int32_t which,
                                    gpcg_plan_info* info, int32_t* bus_order,
                                    int32_t* bus_of_row, int32_t* lrowptr, int32_t* lcol,
                                    int32_t* level, uint8_t* bridge) {
  if (!g || !info) return fail(GPCG_ERR_INVALID_ARG, "gpcg_analyze: NULL argument");
  if (precond < 0 || precond > 2) return fail(GPCG_ERR_INVALID_ARG, "precond must be 0, 1 or 2");
  if (which != 0 && which != 1) return fail(GPCG_ERR_INVALID_ARG, "which must be 0 or 1");
  int slack = -1;
  gpcg_status st = validate_grid(g, &slack);
  if (st != GPCG_OK) return st;
  const int n = g->n_bus, m = g->n_branch;
  // the same steps as gpcg_create: internal numbering, bus graph, depth-first
  // numbering, matrix plan
  const std::vector<int32_t> U = rcm_order(n, build_bus_graph(n, m, g->from, g->to));
  std::vector<int32_t> I(n);
  for (int k = 0; k < n; ++k) I[U[k]] = k;
  std::vector<int32_t> f_i(m), t_i(m);
  for (int e = 0; e < m; ++e) {
    f_i[e] = I[g->from[e]];
    t_i[e] = I[g->to[e]];
  }
  const BusGraph bg = build_bus_graph(n, m, f_i.data(), t_i.data());
  std::vector<int32_t> pre, sub;
  std::vector<uint8_t> br;
  if (!dfs_numbering(n, bg, I[slack], pre, sub, br, m))
    return fail(GPCG_ERR_BASE_ISLANDED, "the intact grid is not connected");
  std::vector<uint8_t> keep(n);
  for (int k = 0; k < n; ++k) {
    const int bt = g->bus_type[U[k]];
    keep[k] = which == 0 ? bt != GPCG_SLACK : bt == GPCG_PQ;
  }
  const MatrixPlan P = plan_matrix(n, bg, keep, precond == GPCG_PRECOND_EXACT);
  info->n_rows = P.n;
  info->nnz_a = P.A.nnz();
  info->nnz_l = P.L.nnz();
  info->levels = (int)P.lev_ptr.size() - 1;
  info->blevels = (int)P.blev_ptr.size() - 1;
  info->n_bridges = 0;
  for (int e = 0; e < m; ++e) info->n_bridges += br[e];
  if (bus_order) std::memcpy(bus_order, U.data(), (size_t)n * 4);
  if (bus_of_row)
    for (int i = 0; i < P.n; ++i) bus_of_row[i] = U[P.bus_of_row[i]];
  if (lrowptr) std::memcpy(lrowptr, P.L.ptr.data(), P.L.ptr.size() * 4);
  if (lcol) std::memcpy(lcol, P.L.idx.data(), P.L.idx.size() * 4);
  if (level) std::memcpy(level, P.level.data(), (size_t)P.n * 4);
  if (bridge) std::memcpy(bridge, br.data(), (size_t)m);
  g_err.clear();
  return GPCG_OK;
}

extern "C" const char* gpcg_last_error(void) { return g_err.c_str(); }

// ------------------------------------------------------------ internal view
// Read-only view of a context for other translation units of the library.
namespace gpcg {
bool ctx_view(const gpcg_ctx* c, CtxView* v) {
  if (!c || !v) return false;
  v->G = c->G;
  const bool f16 = c->opt.precision == GPCG_BATCHED_FP32_F16;
  v->MPf = c->MP.view<float>(f16);
  v->MQf = c->MQ.view<float>(f16);
  v->MPd = c->MP.view<double>();
  v->MQd = c->MQ.view<double>();
  v->th0 = c->th0;
  v->V0 = c->V0;
  v->c0 = c->c0;
  v->s0 = c->s0;
  v->mis_order = c->mis_order;
  v->bus_of_user = c->d_bus_of_user;
  v->misq_order = c->misq_order;
  v->opt = c->opt;
  v->num_sms = c->num_sms;
  v->n = c->n;
  v->m = c->m;
  v->slack = c->slack;
  v->rows = std::max(c->MP.plan.n, c->MQ.plan.n + KX);  // B'': + the extension rows
  v->slack_user = c->slack_user;
  v->u_f = c->u_f;
  v->u_t = c->u_t;
  v->u_pre = c->u_pre;
  v->isl = c->isl;
  v->r0P = c->r0P;
  v->r0Q = c->r0Q;
  v->u_bus_type = c->u_bus_type;
  v->u_P_sched = c->u_P_sched;
  v->u_P_gen = c->u_P_gen;
  v->tile = c->tile;
  v->per_sm = c->per_sm;
  v->base_ok = c->base_ok;
  return true;
}
}  // namespace gpcg

namespace gpcg {
// Record the calling thread's error message (read by gpcg_last_error).
void set_last_error(const char* msg) { g_err = msg ? msg : ""; }
}  // namespace gpcg
