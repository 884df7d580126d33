// Kernels that build the base-case structures once per grid: branch
// admittances, the bus admittance diagonal, the B'/B'' values (Sec. III.B:
// the diagonal .BIJ on the vertex, the off-diagonal .BIJ on the edge) and the
// level-scheduled numeric factorisation of the base-case matrix that
// preconditions every scenario (Sec. IV.B, eq. (6)).
#include "common.cuh"

namespace gpcg {

// y = 1/(r + jx) = g + j b_y; weights of B' (1/x) and B'' (x/(r^2+x^2)).
__global__ void branch_params_kernel(int m, const double* __restrict__ r,
                                     const double* __restrict__ x, double* g, double* by,
                                     double* wP, double* wQ) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= m) return;
  double rr = r[e], xx = x[e];
  double d = rr * rr + xx * xx;
  g[e] = rr / d;
  by[e] = -xx / d;
  wP[e] = 1.0 / xx;
  wQ[e] = xx / d;
}

// Y_ii = sum over incident branches of (y + j b_sh/2), times c^2 at the
// from end of a transformer (c = 1 / turns ratio: the pi-model sees V_i c),
// summed in the fixed order of the bus adjacency lists.
__global__ void ybus_diag_kernel(int n, const int32_t* __restrict__ adj_ptr,
                                 const int32_t* __restrict__ adj_br,
                                 const int32_t* __restrict__ from, const double* __restrict__ cf,
                                 const double* __restrict__ g, const double* __restrict__ by,
                                 const double* __restrict__ b_sh, double* Gii, double* Bii) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double G = 0.0, B = 0.0;
  for (int k = adj_ptr[i]; k < adj_ptr[i + 1]; ++k) {
    int e = adj_br[k];
    const double c2 = from[e] == i ? cf[e] * cf[e] : 1.0;
    G += c2 * g[e];
    B += c2 * (by[e] + 0.5 * b_sh[e]);
  }
  Gii[i] = G;
  Bii[i] = B;
}

// Values of a grounded sum of branch terms w v v^T, v = c e_from - e_to
// (c = 1 for every branch when cf is null: a weighted Laplacian), on its CSR
// pattern: one thread per matrix row walks the bus's incident branches in a
// fixed order.  The diagonal collects every incident branch (also those to
// buses without a row), w c^2 at a from end and w at a to end; each
// neighbour with a row receives -w c in its slot.
__global__ void laplacian_values_kernel(int nrows, const int32_t* __restrict__ bus_of_row,
                                        const int32_t* __restrict__ row_of_bus,
                                        const int32_t* __restrict__ adj_ptr,
                                        const int32_t* __restrict__ adj_idx,
                                        const int32_t* __restrict__ adj_br,
                                        const double* __restrict__ w,
                                        const int32_t* __restrict__ from,
                                        const double* __restrict__ cf,
                                        const int32_t* __restrict__ a_ptr,
                                        const int32_t* __restrict__ a_idx, double* a_val,
                                        int32_t* err) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nrows) return;
  int b = bus_of_row[i];
  int s = a_ptr[i], e_ = a_ptr[i + 1];
  for (int k = s; k < e_; ++k) a_val[k] = 0.0;
  double diag = 0.0;
  for (int k = adj_ptr[b]; k < adj_ptr[b + 1]; ++k) {
    const int e = adj_br[k];
    double we = w[e];
    if (cf) {
      diag += from[e] == b ? we * cf[e] * cf[e] : we;
      we *= cf[e];
    } else {
      diag += we;
    }
    int c = row_of_bus[adj_idx[k]];
    if (c < 0) continue;
    int lo = s, hi = e_ - 1, pos = -1;
    while (lo <= hi) {
      int mid = (lo + hi) >> 1;
      int v = a_idx[mid];
      if (v == c) { pos = mid; break; }
      if (v < c) lo = mid + 1; else hi = mid - 1;
    }
    if (pos < 0) { atomicExch(err, 1); continue; }
    a_val[pos] -= we;
  }
  int lo = s, hi = e_ - 1, pos = -1;
  while (lo <= hi) {
    int mid = (lo + hi) >> 1;
    int v = a_idx[mid];
    if (v == i) { pos = mid; break; }
    if (v < i) lo = mid + 1; else hi = mid - 1;
  }
  if (pos < 0) { atomicExch(err, 1); return; }
  a_val[pos] += diag;
}

// The row a bus without one would have in a matrix of branch terms w v v^T
// (v = c e_from - e_to; cf null: c = 1), for every bus: per adjacency entry
// the neighbour's row (-1: none) and -w c, and per bus the diagonal, summed
// in the same order and form as laplacian_values_kernel.
__global__ void ext_rows_kernel(int n, const int32_t* __restrict__ adj_ptr,
                                const int32_t* __restrict__ adj_idx,
                                const int32_t* __restrict__ adj_br,
                                const int32_t* __restrict__ from, const double* __restrict__ cf,
                                const double* __restrict__ w,
                                const int32_t* __restrict__ row_of_bus, int32_t* xrow,
                                double* xval, float* xval32, double* xdiag, float* xdiag32) {
  int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= n) return;
  double diag = 0.0;
  for (int k = adj_ptr[b]; k < adj_ptr[b + 1]; ++k) {
    const int e = adj_br[k];
    double we = w[e];
    if (cf) {
      diag += from[e] == b ? we * cf[e] * cf[e] : we;
      we *= cf[e];
    } else {
      diag += we;
    }
    xrow[k] = row_of_bus[adj_idx[k]];
    xval[k] = -we;
    xval32[k] = (float)-we;
  }
  xdiag[b] = diag;
  xdiag32[b] = (float)diag;
}

void launch_ext_rows(cudaStream_t st, int n, const int32_t* adj_ptr, const int32_t* adj_idx,
                     const int32_t* adj_br, const int32_t* from, const double* cf,
                     const double* w, const int32_t* row_of_bus, int32_t* xrow, double* xval,
                     float* xval32, double* xdiag, float* xdiag32) {
  if (n > 0)
    ext_rows_kernel<<<(n + 255) / 256, 256, 0, st>>>(n, adj_ptr, adj_idx, adj_br, from, cf, w,
                                                     row_of_bus, xrow, xval, xval32, xdiag,
                                                     xdiag32);
}

__device__ __forceinline__ double csr_lookup(const int32_t* idx, const double* val, int s,
                                             int e, int col) {
  int lo = s, hi = e - 1;
  while (lo <= hi) {
    int mid = (lo + hi) >> 1;
    int v = idx[mid];
    if (v == col) return val[mid];
    if (v < col) lo = mid + 1; else hi = mid - 1;
  }
  return 0.0;
}

// Incomplete Cholesky on the pattern of L, rows of one level at a time (all
// rows a row depends on sit in lower levels):
//   L_ij = (A_ij - sum_{k<j} L_ik L_jk) / L_jj,   L_ii = sqrt(A_ii - sum L_ik^2),
// the sums running over the columns both rows hold.  With the complete
// symbolic pattern this is the exact Cholesky factor.
__global__ void ic_level_kernel(int row0, int row1, const int32_t* __restrict__ a_ptr,
                                const int32_t* __restrict__ a_idx,
                                const double* __restrict__ a_val,
                                const int32_t* __restrict__ l_ptr,
                                const int32_t* __restrict__ l_idx, double* l_val,
                                int32_t* err) {
  int i = row0 + blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= row1) return;
  int ls = l_ptr[i], le = l_ptr[i + 1];
  for (int k = ls; k < le; ++k) {
    int j = l_idx[k];
    double s = csr_lookup(a_idx, a_val, a_ptr[i], a_ptr[i + 1], j);
    // merge row i (entries before k) with row j (off-diagonal entries)
    int p = ls, q = l_ptr[j], qe = l_ptr[j + 1] - 1;
    while (p < k && q < qe) {
      int ci = l_idx[p], cj = l_idx[q];
      if (ci == cj) { s -= l_val[p] * l_val[q]; ++p; ++q; }
      else if (ci < cj) ++p;
      else ++q;
    }
    if (j < i) {
      l_val[k] = s / l_val[l_ptr[j + 1] - 1];
    } else {
      if (!(s > 0.0)) { atomicExch(err, 2); s = 1.0; }
      l_val[k] = sqrt(s);
    }
  }
}

__global__ void scatter_kernel(int nnz, const int32_t* __restrict__ map,
                               const double* __restrict__ src, double* dst) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < nnz) dst[map[k]] = src[k];
}

__global__ void to_float_kernel(int n, const double* __restrict__ src, float* dst) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n) dst[k] = (float)src[k];
}

__global__ void gather_diag_kernel(int n, const int32_t* __restrict__ pos,
                                   const double* __restrict__ a_val, double* d) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n) d[k] = a_val[pos[k]];
}

__global__ void gather_int_kernel(int n, const int32_t* __restrict__ idx,
                                  const int32_t* __restrict__ src, int32_t* dst) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n) dst[k] = src[idx[k]];
}

// ---------------------------------------------------------------- launchers
static inline int nblk(int n, int b) { return (n + b - 1) / b; }

void launch_branch_params(cudaStream_t st, int m, const double* r, const double* x, double* g,
                          double* by, double* wP, double* wQ) {
  if (m) branch_params_kernel<<<nblk(m, 256), 256, 0, st>>>(m, r, x, g, by, wP, wQ);
}
void launch_ybus_diag(cudaStream_t st, int n, const int32_t* adj_ptr, const int32_t* adj_br,
                      const int32_t* from, const double* cf, const double* g, const double* by,
                      const double* b_sh, double* Gii, double* Bii) {
  if (n)
    ybus_diag_kernel<<<nblk(n, 256), 256, 0, st>>>(n, adj_ptr, adj_br, from, cf, g, by, b_sh,
                                                   Gii, Bii);
}
void launch_laplacian_values(cudaStream_t st, int nrows, const int32_t* bus_of_row,
                             const int32_t* row_of_bus, const int32_t* adj_ptr,
                             const int32_t* adj_idx, const int32_t* adj_br, const double* w,
                             const int32_t* from, const double* cf, const int32_t* a_ptr,
                             const int32_t* a_idx, double* a_val, int32_t* err) {
  if (nrows)
    laplacian_values_kernel<<<nblk(nrows, 128), 128, 0, st>>>(
        nrows, bus_of_row, row_of_bus, adj_ptr, adj_idx, adj_br, w, from, cf, a_ptr, a_idx,
        a_val, err);
}
void launch_ic_level(cudaStream_t st, int row0, int row1, const int32_t* a_ptr,
                     const int32_t* a_idx, const double* a_val, const int32_t* l_ptr,
                     const int32_t* l_idx, double* l_val, int32_t* err) {
  int n = row1 - row0;
  if (n > 0)
    ic_level_kernel<<<nblk(n, 128), 128, 0, st>>>(row0, row1, a_ptr, a_idx, a_val, l_ptr,
                                                  l_idx, l_val, err);
}
void launch_scatter(cudaStream_t st, int nnz, const int32_t* map, const double* src,
                    double* dst) {
  if (nnz) scatter_kernel<<<nblk(nnz, 256), 256, 0, st>>>(nnz, map, src, dst);
}
void launch_to_float(cudaStream_t st, int n, const double* src, float* dst) {
  if (n) to_float_kernel<<<nblk(n, 256), 256, 0, st>>>(n, src, dst);
}
void launch_gather_diag(cudaStream_t st, int n, const int32_t* pos, const double* a_val,
                        double* d) {
  if (n) gather_diag_kernel<<<nblk(n, 256), 256, 0, st>>>(n, pos, a_val, d);
}
void launch_gather_int(cudaStream_t st, int n, const int32_t* idx, const int32_t* src,
                       int32_t* dst) {
  if (n) gather_int_kernel<<<nblk(n, 256), 256, 0, st>>>(n, idx, src, dst);
}

}  // namespace gpcg

namespace gpcg {

// dst[k] = csr[src[k]] (0 where src[k] < 0), in FP64 and FP32.
__global__ void gather_val_kernel(int n, const int32_t* __restrict__ src,
                                  const double* __restrict__ csr, double* dst, float* dst32) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const int s = src[k];
  const double v = s >= 0 ? csr[s] : 0.0;
  dst[k] = v;
  dst32[k] = (float)v;
}

__global__ void inv_diag_kernel(int n, const int32_t* __restrict__ pos,
                                const double* __restrict__ l_val, double* inv, float* inv32) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double d = 1.0 / l_val[pos[i]];
  inv[i] = d;
  inv32[i] = (float)d;
}

// Per-slot branch admittance of the mismatch adjacency (0 on padding).
__global__ void adj_values_kernel(int n, const int32_t* __restrict__ br,
                                  const double* __restrict__ cf,
                                  const double* __restrict__ g, const double* __restrict__ by,
                                  double* ag, double* ab) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const int e = br[k];
  // Y_ij = -c y for either end (c = 1 / turns ratio)
  ag[k] = e >= 0 ? cf[e] * g[e] : 0.0;
  ab[k] = e >= 0 ? cf[e] * by[e] : 0.0;
}

void launch_gather_val(cudaStream_t st, int n, const int32_t* src, const double* csr, double* dst,
                       float* dst32) {
  if (n > 0) gather_val_kernel<<<(n + 255) / 256, 256, 0, st>>>(n, src, csr, dst, dst32);
}
void launch_inv_diag(cudaStream_t st, int n, const int32_t* pos, const double* l_val, double* inv,
                     float* inv32) {
  if (n > 0) inv_diag_kernel<<<(n + 255) / 256, 256, 0, st>>>(n, pos, l_val, inv, inv32);
}
// X = inverse of the factor's tail block L_tt (rows and columns
// [t0, t0 + nt) of L, lower triangular): column c of X by forward
// substitution of L_tt x = e_c, one thread per column, in FP64.  Written
// column-major (xc[c nt + i] = X_ic) and row-major (xr[i nt + c] = X_ic),
// zeros above the diagonal, in FP64 (xr optional) and FP32.
// With lsc (the scaled factor Ls = L D^-1) the block inverted is the one
// the FP16 storage represents: L_ij = fp16(Ls_ij) L_jj.
__global__ void tail_inverse_kernel(int t0, int nt, const int32_t* __restrict__ l_ptr,
                                    const int32_t* __restrict__ l_idx,
                                    const double* __restrict__ l_val,
                                    const double* __restrict__ lsc, double* xc, double* xr,
                                    float* xc32, float* xr32) {
  for (int c = threadIdx.x; c < nt; c += blockDim.x) {
    // xc holds the column in FP64 while it is built (its earlier entries
    // are the unknowns solved before)
    for (int i = 0; i < nt; ++i) {
      double v = 0.0;
      if (i >= c) {
        const int R = t0 + i, e0 = l_ptr[R], e1 = l_ptr[R + 1] - 1;  // diagonal last
        double sum = (i == c) ? 1.0 : 0.0;
        for (int e = e0; e < e1; ++e) {
          const int jg = l_idx[e], j = jg - t0;
          if (j < c) continue;
          const double lij =
              lsc ? (double)__half2float(__double2half(lsc[e])) * l_val[l_ptr[jg + 1] - 1]
                  : l_val[e];
          sum -= lij * xc[(size_t)c * nt + j];
        }
        v = sum / l_val[e1];
      }
      xc[(size_t)c * nt + i] = v;
      if (xr) xr[(size_t)i * nt + c] = v;
      xc32[(size_t)c * nt + i] = (float)v;
      xr32[(size_t)i * nt + c] = (float)v;
    }
  }
}

void launch_tail_inverse(cudaStream_t st, int t0, int nt, const int32_t* l_ptr,
                         const int32_t* l_idx, const double* l_val, const double* lsc, double* xc,
                         double* xr, float* xc32, float* xr32) {
  if (nt > 0)
    tail_inverse_kernel<<<1, 128, 0, st>>>(t0, nt, l_ptr, l_idx, l_val, lsc, xc, xr, xc32, xr32);
}

void launch_adj_values(cudaStream_t st, int n, const int32_t* br, const double* cf,
                       const double* g, const double* by, double* ag, double* ab) {
  if (n > 0) adj_values_kernel<<<(n + 255) / 256, 256, 0, st>>>(n, br, cf, g, by, ag, ab);
}

}  // namespace gpcg

namespace gpcg {

// Scaled factor for FP16 storage: L = Ls D, D = diag(L); Ls_ij = L_ij / L_jj
// (unit diagonal), and 1 / L_ii^2 for the back substitution.
__global__ void scale_factor_kernel(int n, const int32_t* __restrict__ l_ptr,
                                    const int32_t* __restrict__ l_idx,
                                    const double* __restrict__ l_val, double* lsc, double* inv_d2,
                                    float* inv_d2_32) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  for (int k = l_ptr[i]; k < l_ptr[i + 1]; ++k) {
    const int j = l_idx[k];
    lsc[k] = l_val[k] / l_val[l_ptr[j + 1] - 1];
  }
  const double d = l_val[l_ptr[i + 1] - 1];
  inv_d2[i] = 1.0 / (d * d);
  inv_d2_32[i] = (float)(1.0 / (d * d));
}

__global__ void gather_half_kernel(int n, const int32_t* __restrict__ src,
                                   const double* __restrict__ v, __half* dst) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const int s = src[k];
  dst[k] = __double2half(s >= 0 ? v[s] : 0.0);
}

void launch_scale_factor(cudaStream_t st, int n, const int32_t* l_ptr, const int32_t* l_idx,
                         const double* l_val, double* lsc, double* inv_d2, float* inv_d2_32) {
  if (n > 0)
    scale_factor_kernel<<<(n + 255) / 256, 256, 0, st>>>(n, l_ptr, l_idx, l_val, lsc, inv_d2,
                                                         inv_d2_32);
}
void launch_gather_half(cudaStream_t st, int n, const int32_t* src, const double* v, __half* dst) {
  if (n > 0) gather_half_kernel<<<(n + 255) / 256, 256, 0, st>>>(n, src, v, dst);
}

}  // namespace gpcg
