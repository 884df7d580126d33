// The overload-penalty adjoint over N-1 scenarios (DC model of eq. (4)).
//
// For scenario s (outage l): theta_s = B'_s^{-1} R_s P with B'_s the base
// matrix (weights b) minus the outaged branch's four-element change
// (Sec. IV.B), islands removed and their injection re-dispatched
// (Sec. IV.C, weights frozen); flows f = b (theta_i - theta_j);
// L = sum softplus(|f|/rating - 1)^2.  With g = dL/df the adjoint is one more
// solve with the symmetric B'_s, lambda_s = B'_s^{-1} A^T diag(b_s) g_s, and
//   dL/dP   = sum_s R_s^T lambda_s,
//   dL/db_k = sum_s [ g_ks (A theta_s)_k - (A lambda_s)_k (A theta_s)_k ].
// Both solves are the batched base-preconditioned PCG of the N-1 screen.
// Tiles are dealt to CTAs statically; each CTA accumulates its scenarios'
// terms in its own slot and a second kernel sums the slots in a fixed order,
// so the gradients are bitwise reproducible.
#include "fdpf_ops.cuh"

namespace gpcg {

struct AdjParams {
  const double* P = nullptr;   // [n] injections, internal bus order
  const double* b = nullptr;   // [m] branch susceptances
  double* gP = nullptr;        // [slots][n] per-slot sums (internal order)
  double* gb = nullptr;        // [slots][m]
  double* loss = nullptr;      // [slots]
};

__device__ __forceinline__ double softplus_d(double u) {
  return u > 0.0 ? u + log1p(exp(-u)) : log1p(exp(u));
}
// penalty phi(F) = softplus(|F|/rating - 1)^2 and its derivative (odd in F)
__device__ __forceinline__ double penalty(double F, double rating) {
  const double s = softplus_d(fabs(F) / rating - 1.0);
  return s * s;
}
__device__ __forceinline__ double penalty_grad(double F, double rating) {
  const double u = fabs(F) / rating - 1.0;
  const double sig = 0.5 * (1.0 + tanh(0.5 * u));
  const double sg = F > 0.0 ? 1.0 : (F < 0.0 ? -1.0 : 0.0);
  return 2.0 * softplus_d(u) * sig * sg / rating;
}

template <int T, typename VT>
__global__ void __launch_bounds__(NTHREADS, FDPF_MIN_BLOCKS)
    adjoint_tiles_kernel(FdpfParams P, AdjParams A, DevMatT<VT> M) {
  static_assert(T == 2 && Geo<T>::LP == 2, "one thread per row, two lanes: the slot sums need no atomics");
  __shared__ LaneState<T> L;
  __shared__ double red[NTHREADS * 2];  // lane_reduce and the loss sum
  const Geo<T> g;
  const int tid = threadIdx.x;
  const DevGrid& G = P.G;
  VT* x = (VT*)P.wx + (size_t)blockIdx.x * P.vstride;
  VT* r = (VT*)P.wr + (size_t)blockIdx.x * P.vstride;
  VT* p = (VT*)P.wp + (size_t)blockIdx.x * P.vstride;
  VT* q = (VT*)P.wq + (size_t)blockIdx.x * P.vstride;
  VT* z = (VT*)P.wz + (size_t)blockIdx.x * P.vstride;
  const size_t so = (size_t)blockIdx.x * P.sstride;
  double* th = P.wth + so;   // theta by bus
  double* lm = P.wV + so;    // lambda by bus
  double* gP = A.gP + (size_t)blockIdx.x * G.n;
  double* gb = A.gb + (size_t)blockIdx.x * G.m;
  const int l0 = g.lane, l1 = g.lane + 1;
  for (int i = tid; i < G.n; i += NTHREADS) gP[i] = 0.0;
  for (int k = tid; k < G.m; k += NTHREADS) gb[k] = 0.0;
  double loss_acc = 0.0;
  __syncthreads();
  // tiles are dealt to CTAs statically (every scenario costs two solves), so
  // the per-slot sums, and hence the gradients, do not depend on timing
  for (int tile = blockIdx.x; tile < P.n_tiles; tile += gridDim.x) {
    if (tid < T) {
      const int ln = tid, s = tile * T + ln;
      const bool valid = s < P.S;
      const int l = valid ? P.sc.outage[s] : -1;
      L.scen[ln] = valid ? s : -1;
      L.l[ln] = l;
      L.lo[ln] = valid ? P.sc.isl_lo[s] : 0;
      L.cnt[ln] = valid ? P.sc.isl_cnt[s] : 0;
      L.coef[ln] = valid ? P.sc.coef[s] : 0.0;
      L.nogen[ln] = valid ? P.sc.no_gen[s] : 0;
      L.raP[ln] = l >= 0 ? M.row_of_bus[G.f[l]] : -1;
      L.rbP[ln] = l >= 0 ? M.row_of_bus[G.t[l]] : -1;
      L.wP[ln] = l >= 0 ? A.b[l] : 0.0;
      L.active[ln] = valid;
      L.inP[ln] = 0;
    }
    __syncthreads();
    const int lo0 = L.lo[l0], cnt0 = L.cnt[l0], lo1 = L.lo[l1], cnt1 = L.cnt[l1];
    const int br0 = L.l[l0], br1 = L.l[l1];
    const bool v0 = L.scen[l0] >= 0, v1 = L.scen[l1] >= 0;
    // right-hand side R_s P on the main island's non-slack rows
    for (int k = g.rs; k < M.n; k += Geo<T>::RPS) {
      const int i = M.bus_of_row[k], pr = M.pre_of_row[k];
      double pi = A.P[i];
      const double pg = G.bus_type[i] == 1 ? fmax(G.P_gen[i], 0.0) : 0.0;
      const double a = (v0 && !in_island(pr, lo0, cnt0)) ? pi + L.coef[l0] * pg : 0.0;
      const double b = (v1 && !in_island(pr, lo1, cnt1)) ? pi + L.coef[l1] * pg : 0.0;
      r[(size_t)k * T + g.lane] = (VT)a;
      r[(size_t)k * T + g.lane + 1] = (VT)b;
    }
    __syncthreads();
    pcg_solve<T, VT>(P, M, L, x, r, p, q, z, L.raP, L.rbP, L.wP, L.inP);
    for (int i = g.rs; i < G.n; i += Geo<T>::RPS) {
      const int k = M.row_of_bus[i];
      double a = 0.0, b = 0.0;
      if (k >= 0) {
        a = (double)x[(size_t)k * T + g.lane];
        b = (double)x[(size_t)k * T + g.lane + 1];
      }
      th[(size_t)i * T + g.lane] = a;
      th[(size_t)i * T + g.lane + 1] = b;
    }
    __syncthreads();
    // loss over branches, then y = A^T diag(b_s) g on the rows
    for (int k = g.rs; k < G.m; k += Geo<T>::RPS) {
      const int a = G.f[k], b = G.t[k];
      const int pa = G.pre[a], pb = G.pre[b];
      const double bk = A.b[k], rk = G.rating[k];
      if (v0 && k != br0 && !in_island(pa, lo0, cnt0) && !in_island(pb, lo0, cnt0))
        loss_acc += penalty(bk * (th[(size_t)a * T + l0] - th[(size_t)b * T + l0]), rk);
      if (v1 && k != br1 && !in_island(pa, lo1, cnt1) && !in_island(pb, lo1, cnt1))
        loss_acc += penalty(bk * (th[(size_t)a * T + l1] - th[(size_t)b * T + l1]), rk);
    }
    for (int k = g.rs; k < M.n; k += Geo<T>::RPS) {
      const int i = M.bus_of_row[k], pr = M.pre_of_row[k];
      const bool m0 = v0 && !in_island(pr, lo0, cnt0), m1 = v1 && !in_island(pr, lo1, cnt1);
      double y0 = 0.0, y1 = 0.0;
      for (int e = G.adj_ptr[i]; e < G.adj_ptr[i + 1]; ++e) {
        const int j = G.adj_idx[e], br = G.adj_br[e];
        const double bk = A.b[br], rk = G.rating[br];
        const int pj = G.pre[j];
        if (m0 && br != br0 && !in_island(pj, lo0, cnt0))
          y0 += bk * penalty_grad(bk * (th[(size_t)i * T + l0] - th[(size_t)j * T + l0]), rk);
        if (m1 && br != br1 && !in_island(pj, lo1, cnt1))
          y1 += bk * penalty_grad(bk * (th[(size_t)i * T + l1] - th[(size_t)j * T + l1]), rk);
      }
      r[(size_t)k * T + g.lane] = (VT)y0;
      r[(size_t)k * T + g.lane + 1] = (VT)y1;
    }
    __syncthreads();
    pcg_solve<T, VT>(P, M, L, x, r, p, q, z, L.raP, L.rbP, L.wP, L.inP);
    // lambda by bus; the re-dispatch transpose needs sum_k P_gen,k lambda_k
    // and sum_k P_gen,k over the main island's PV buses
    double wl0 = 0.0, wl1 = 0.0, dn0 = 0.0, dn1 = 0.0;
    for (int i = g.rs; i < G.n; i += Geo<T>::RPS) {
      const int k = M.row_of_bus[i];
      double a = 0.0, b = 0.0;
      if (k >= 0) {
        a = (double)x[(size_t)k * T + g.lane];
        b = (double)x[(size_t)k * T + g.lane + 1];
      }
      lm[(size_t)i * T + g.lane] = a;
      lm[(size_t)i * T + g.lane + 1] = b;
      if (G.bus_type[i] == 1 && G.P_gen[i] > 0.0) {
        const int pr = G.pre[i];
        const double pg = G.P_gen[i];
        if (!in_island(pr, lo0, cnt0)) { wl0 += pg * a; dn0 += pg; }
        if (!in_island(pr, lo1, cnt1)) { wl1 += pg * b; dn1 += pg; }
      }
    }
    const Pair<double> WL = lane_reduce<T, false>(red, wl0, wl1);
    const Pair<double> DN = lane_reduce<T, false>(red, dn0, dn1);
    const double W0 = (v0 && cnt0 > 0 && !L.nogen[l0] && DN.a > 0.0) ? WL.a / DN.a : 0.0;
    const double W1 = (v1 && cnt1 > 0 && !L.nogen[l1] && DN.b > 0.0) ? WL.b / DN.b : 0.0;
    for (int i = g.rs; i < G.n; i += Geo<T>::RPS) {
      const int pr = G.pre[i];
      double add = 0.0;
      if (v0) add += in_island(pr, lo0, cnt0) ? W0 : lm[(size_t)i * T + l0];
      if (v1) add += in_island(pr, lo1, cnt1) ? W1 : lm[(size_t)i * T + l1];
      gP[i] += add;
    }
    for (int k = g.rs; k < G.m; k += Geo<T>::RPS) {
      const int a = G.f[k], b = G.t[k];
      const int pa = G.pre[a], pb = G.pre[b];
      const double bk = A.b[k], rk = G.rating[k];
      double add = 0.0;
      if (v0 && k != br0 && !in_island(pa, lo0, cnt0) && !in_island(pb, lo0, cnt0)) {
        const double At = th[(size_t)a * T + l0] - th[(size_t)b * T + l0];
        const double Al = lm[(size_t)a * T + l0] - lm[(size_t)b * T + l0];
        add += penalty_grad(bk * At, rk) * At - Al * At;
      }
      if (v1 && k != br1 && !in_island(pa, lo1, cnt1) && !in_island(pb, lo1, cnt1)) {
        const double At = th[(size_t)a * T + l1] - th[(size_t)b * T + l1];
        const double Al = lm[(size_t)a * T + l1] - lm[(size_t)b * T + l1];
        add += penalty_grad(bk * At, rk) * At - Al * At;
      }
      gb[k] += add;
    }
    __syncthreads();
  }
  // the CTA's loss: sum over threads in a fixed order
  red[tid] = loss_acc;
  __syncthreads();
  if (tid == 0) {
    double s = 0.0;
    for (int k = 0; k < NTHREADS; ++k) s += red[k];
    A.loss[blockIdx.x] = s;
  }
}

// out[user_of[i]] = sum over slots of acc[slot][i] (slot order fixed).
__global__ void slot_sum_kernel(int n, int slots, const double* __restrict__ acc,
                                const int32_t* __restrict__ map, double* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double s = 0.0;
  for (int k = 0; k < slots; ++k) s += acc[(size_t)k * n + i];
  out[map ? map[i] : i] = s;
}

__global__ void gather_perm_kernel(int n, const int32_t* __restrict__ idx,
                                   const double* __restrict__ src, double* dst) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = src[idx[i]];
}

cudaError_t launch_adjoint(cudaStream_t st, int grid, const FdpfParams& P, const AdjParamsView& A,
                           const DevMatT<double>& M) {
  AdjParams a;
  a.P = A.P;
  a.b = A.b;
  a.gP = A.gP;
  a.gb = A.gb;
  a.loss = A.loss;
  adjoint_tiles_kernel<2, double><<<grid, NTHREADS, 0, st>>>(P, a, M);
  return cudaGetLastError();
}

int adjoint_max_blocks_per_sm() {
  int nb = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, adjoint_tiles_kernel<2, double>, NTHREADS, 0);
  return nb;
}

cudaError_t launch_slot_sum(cudaStream_t st, int n, int slots, const double* acc,
                            const int32_t* map, double* out) {
  if (n > 0) slot_sum_kernel<<<(n + 255) / 256, 256, 0, st>>>(n, slots, acc, map, out);
  return cudaGetLastError();
}

cudaError_t launch_gather_perm(cudaStream_t st, int n, const int32_t* idx, const double* src,
                               double* dst) {
  if (n > 0) gather_perm_kernel<<<(n + 255) / 256, 256, 0, st>>>(n, idx, src, dst);
  return cudaGetLastError();
}

}  // namespace gpcg
