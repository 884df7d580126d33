// Shared device-side definitions of the GB300 N-1 screen.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace gpcg {

// Grid arrays on the device (bus order and branch order of the caller).
struct DevGrid {
  int n = 0, m = 0, slack = -1;
  int8_t* bus_type = nullptr;
  double *P_sched = nullptr, *Q_sched = nullptr, *P_gen = nullptr, *V_set = nullptr;
  int32_t *f = nullptr, *t = nullptr;
  double *r = nullptr, *x = nullptr, *b_sh = nullptr, *rating = nullptr;
  double *g = nullptr, *by = nullptr;        // series admittance g + j b_y
  int32_t *adj_ptr = nullptr, *adj_idx = nullptr, *adj_br = nullptr;
  double *Gii = nullptr, *Bii = nullptr;     // bus admittance diagonal
  int32_t *pre = nullptr, *sub = nullptr;    // depth-first preorder, subtree size
};

// One fast-decoupled matrix (B' or B'') with its base-case factor.  VT is
// the value type used by the solve kernels (float or double).
template <typename VT>
struct DevMatT {
  int n = 0;
  const int32_t *bus_of_row = nullptr, *row_of_bus = nullptr, *pre_of_row = nullptr;
  const int32_t *a_ptr = nullptr, *a_idx = nullptr;
  const VT* a_val = nullptr;
  const int32_t *l_ptr = nullptr, *l_idx = nullptr;
  const VT* l_val = nullptr;
  const int32_t *u_ptr = nullptr, *u_idx = nullptr;
  const VT* u_val = nullptr;
  const VT* diag = nullptr;                  // diagonal of A (Jacobi)
  const int32_t *lev_ptr = nullptr;          // forward levels (contiguous rows)
  const int32_t *blev_ptr = nullptr, *blev_rows = nullptr;
  int nlev = 0, nblev = 0;
  const double* w = nullptr;                 // per-branch weight of this matrix
};

// What the islanding pass leaves for each scenario.
struct ScenInfo {
  int32_t* outage = nullptr;   // branch index
  int32_t* isl_lo = nullptr;   // islanded buses: preorder in [lo, lo + cnt)
  int32_t* isl_cnt = nullptr;
  double* coef = nullptr;      // re-dispatch: P_gen multiplier
  int32_t* no_gen = nullptr;
};

__device__ __forceinline__ bool in_island(int32_t pre, int32_t lo, int32_t cnt) {
  return (uint32_t)(pre - lo) < (uint32_t)cnt;
}

}  // namespace gpcg
