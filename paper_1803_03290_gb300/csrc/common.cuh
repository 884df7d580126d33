// Shared device-side definitions of the GB300 N-1 screen.
#pragma once
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace gpcg {

// Slots per row of the padded row descriptors (ELL layout: row i's entries
// at [i*K, i*K+K), padding points at the zero row and carries value 0;
// entries beyond K live in a small per-matrix overflow CSR).
constexpr int KA = 6;   // B' / B'' rows, diagonal included
constexpr int KL = 4;   // strictly lower part of the factor
constexpr int KU = 4;   // strictly upper part (L^T)
constexpr int KG = 6;   // bus adjacency of the mismatch
// Tail of the forward level schedule solved with the dense inverse of its
// factor block: the last levels, together at most TAIL_ROWS rows.  Its
// right-hand side sits in shared memory (TAIL_ROWS x T values); 248 rows keep
// the persistent kernel's CTA (T = 2, FP32) at or under 9 KB of shared
// memory, so five resident CTAs fit the 50 KB carveout that leaves the L1
// cache its size.
#ifndef GPCG_TAIL_ROWS
#define GPCG_TAIL_ROWS 248
#endif
constexpr int TAIL_ROWS = GPCG_TAIL_ROWS;

// Grid arrays on the device.  Buses use the library's internal numbering (a
// bandwidth-reducing order of the bus graph); branches keep the caller's
// order, their end buses in internal numbers.
struct DevGrid {
  int n = 0, m = 0, slack = -1;
  int8_t* bus_type = nullptr;
  double *P_sched = nullptr, *Q_sched = nullptr, *P_gen = nullptr, *V_set = nullptr;
  int32_t *f = nullptr, *t = nullptr;
  double *r = nullptr, *x = nullptr, *b_sh = nullptr, *rating = nullptr;
  double* inv_rating = nullptr;              // 1 / rating
  double* cf = nullptr;                      // 1 / turns ratio at the from end (1: a line)
  double *qmin = nullptr, *qmax = nullptr;   // PV generators' reactive limits (null: none)
  double *g = nullptr, *by = nullptr;        // series admittance g + j b_y
  int32_t *adj_ptr = nullptr, *adj_idx = nullptr, *adj_br = nullptr;  // CSR adjacency
  double *Gii = nullptr, *Bii = nullptr;     // bus admittance diagonal
  int32_t *pre = nullptr, *sub = nullptr;    // depth-first preorder, subtree size
  int32_t* user_of_bus = nullptr;            // internal bus index -> caller's index
  // padded adjacency for the mismatch: neighbour, branch, -g, -b_y per slot,
  // slot-major (slot a of bus i at a * n + i: a warp taking consecutive buses
  // reads consecutive entries)
  int32_t *adj_nbr = nullptr, *adj_brl = nullptr, *adj_deg = nullptr;  // deg = used slots
  double *adj_g = nullptr, *adj_b = nullptr;
  int32_t *adj_optr = nullptr, *adj_onbr = nullptr, *adj_obr = nullptr;
  double *adj_og = nullptr, *adj_ob = nullptr;
};

// Padded rows plus overflow of one sparse operator.
template <typename VT>
struct Ell {
  const int32_t* col = nullptr;   // [n*K]
  const VT* val = nullptr;        // [n*K]
  const int32_t* optr = nullptr;  // [n+1] overflow CSR
  const int32_t* ocol = nullptr;
  const VT* oval = nullptr;
};

// One fast-decoupled matrix (B' or B'') with its base-case factor.  VT is
// the value type used by the solve kernels (float or double).  Vectors of
// this matrix have n+1 rows per scenario: row n is kept at zero and is what
// padding slots point at.
template <typename VT>
struct DevMatT {
  int n = 0;
  const int32_t *bus_of_row = nullptr, *row_of_bus = nullptr, *pre_of_row = nullptr;
  const int32_t* visit = nullptr;            // rows in bus order (SpMV, p update)
  Ell<VT> A, L, U;
  const VT* inv_diag = nullptr;              // 1 / L_ii
  // optional scaled FP16 factor: L = Ls D with D = diag(L), Ls unit lower;
  // when set, the substitutions use Ls (values here) and 1 / L_ii^2
  const __half *Lh = nullptr, *Loh = nullptr, *Uh = nullptr, *Uoh = nullptr;
  const VT* inv_d2 = nullptr;
  const VT* diag = nullptr;                  // A_ii (Jacobi)
  const int32_t *lev_ptr = nullptr;          // forward levels (contiguous rows)
  const int32_t *blev_ptr = nullptr, *blev_rows = nullptr;
  int nlev = 0, nblev = 0;
  // the tail: forward levels [tail_lev, nlev) = rows [tail_row0, n), solved
  // with X = inverse of the factor's tail block, stored column-major (xc)
  // and row-major (xr); and the backward levels of rows < tail_row0 with
  // the tail taken as solved
  int tail_lev = 0, tail_row0 = 0, ntblev = 0;
  const int32_t *tblev_ptr = nullptr, *tblev_rows = nullptr;
  const VT *xc = nullptr, *xr = nullptr;
  const double* w = nullptr;                 // per-branch weight of this matrix
  // per-branch factor of the from end (B'': 1 / turns ratio; null: 1): the
  // branch adds w v v^T with v = c e_from - e_to
  const double* c = nullptr;
  // the row a bus without one would have (B'': a PV bus whose generator
  // trips becomes PQ): per bus-adjacency entry k (the bus CSR adjacency,
  // xptr = its row pointer) the neighbour's row (-1: none) and the
  // off-diagonal value, and per bus the diagonal.  Null: not supported.
  const int32_t *xptr = nullptr, *xrow = nullptr;
  const int32_t* xnb = nullptr;  // the neighbour bus of each adjacency entry
  const int32_t* xbr = nullptr;  // the branch of each adjacency entry
  const VT *xval = nullptr, *xdiag = nullptr;
};

// Extension rows a lane may carry at once (see Ext in fdpf_ops.cuh): a
// tripped generator's bus and PV buses switched to PQ at a reactive limit
// (GPCG_MAX_EXT_ROWS of the C ABI).
constexpr int KX = 8;

// What the islanding pass leaves for each scenario.
struct ScenInfo {
  int32_t* outage = nullptr;   // branch index
  int32_t* isl_lo = nullptr;   // islanded buses: preorder in [lo, lo + cnt)
  int32_t* isl_cnt = nullptr;
  double* coef = nullptr;      // re-dispatch: P_gen multiplier
  int32_t* no_gen = nullptr;
  int32_t* gen_bus = nullptr;  // tripped generator's bus (-1: none); null: none in the call
};

__device__ __forceinline__ bool in_island(int32_t pre, int32_t lo, int32_t cnt) {
  return (uint32_t)(pre - lo) < (uint32_t)cnt;
}

// Per-grid islanding data (device arrays).  A single-branch outage islands
// buses only when the branch is a bridge; the island is then the subtree
// below it in the depth-first tree rooted at the slack, preorder interval
// [br_lo, br_lo + br_cnt) (br_cnt = 0: no island).  Preorder prefix sums
// (n + 1 entries) of P_sched and of the PV generation with P_gen > 0 give
// the island's injection and the main island's generation by difference.
struct IslandPlan {
  const int32_t *br_lo = nullptr, *br_cnt = nullptr;       // [n_branch]
  const int32_t *lab_isl = nullptr, *lab_main = nullptr;   // [n_branch] component labels
  const int32_t* u_pre = nullptr;     // [n_bus] preorder of each bus (caller's numbering)
  const int32_t* ord_u = nullptr;     // [n_bus] caller's bus at each preorder position
  const double* prefPs = nullptr;     // [n_bus + 1] prefix sums of P_sched
  const double* prefG = nullptr;      // [n_bus + 1] prefix sums of PV P_gen > 0
  const int32_t* prefGc = nullptr;    // [n_bus + 1] prefix counts of those generators
};

// Islanding of S outages: interval, re-dispatch coefficient, no-generator
// flag per scenario, and (when label_out is given) labels [S][n_bus].
// P_user: the caller's injections (caller's bus order) for the island sums,
// with prefP_scratch (n_bus + 1 doubles) to hold their prefix sums; null
// uses P_sched.
cudaError_t launch_islands(cudaStream_t st, int S, int n, const int32_t* outages,
                           const IslandPlan& I, const double* P_user, double* prefP_scratch,
                           int32_t* isl_lo, int32_t* isl_cnt, double* coef, int32_t* no_gen,
                           int32_t* label_out);
// Generator outages of S PV buses (internal indices): per-scenario data as
// launch_islands leaves it (no branch out, nothing islanded) and the
// re-dispatch of the tripped generation; labels all 0 when requested.
cudaError_t launch_gen_outages(cudaStream_t st, int S, int n, const int32_t* gen_bus,
                               const double* P_gen, const IslandPlan& I, int32_t* outage,
                               int32_t* isl_lo, int32_t* isl_cnt, double* coef, int32_t* no_gen,
                               int32_t* label_out);

}  // namespace gpcg
