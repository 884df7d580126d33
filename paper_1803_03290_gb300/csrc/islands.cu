// Islanding detection (Sec. IV.C) for a batch of single-branch outages, and
// the per-scenario data of the proportional re-dispatch.
//
// The grid is connected, so removing one branch islands buses only when the
// branch is a bridge, and then the islanded buses are exactly the subtree
// below the bridge in a depth-first tree rooted at the slack: one interval
// [lo, lo + cnt) of the depth-first preorder.  The bridges, their intervals
// and the canonical labels of both sides (the smallest bus index of each
// component) are found once per grid on the host (Tarjan's bridge search);
// per scenario the interval is looked up, and the island's net injection
// and the main island's PV generation come from prefix sums over the
// preorder.  The solve kernels then test island membership with one
// comparison per bus.
#include <algorithm>

#include "common.cuh"

namespace gpcg {

// One thread per scenario: island interval, re-dispatch coefficient (the
// island's net injection over the main island's PV generation with
// P_gen > 0) and the no-generator flag.
__global__ void islands_kernel(int S, const int32_t* __restrict__ outages,
                               const int32_t* __restrict__ br_lo,
                               const int32_t* __restrict__ br_cnt,
                               const double* __restrict__ prefP, const double* __restrict__ prefG,
                               const int32_t* __restrict__ prefGc, int n, int32_t* isl_lo,
                               int32_t* isl_cnt, double* coef, int32_t* no_gen) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= S) return;
  const int l = outages[s];
  const int lo = br_lo[l], cnt = br_cnt[l];
  isl_lo[s] = lo;
  isl_cnt[s] = cnt;
  if (cnt == 0) {
    coef[s] = 0.0;
    no_gen[s] = 0;
    return;
  }
  const int hi = lo + cnt;
  const double sumP = prefP[hi] - prefP[lo];
  const int gens_main = prefGc[n] - (prefGc[hi] - prefGc[lo]);
  const double gen_main = prefG[n] - (prefG[hi] - prefG[lo]);
  const int ng = gens_main == 0;
  no_gen[s] = ng;
  coef[s] = ng ? 0.0 : sumP / gen_main;
}

// Component labels per scenario and bus (the caller's numbering): the
// island's smallest bus index inside the interval, the main island's
// outside it (0 for every bus of a non-bridge outage).
__global__ void labels_kernel(int S, int n, const int32_t* __restrict__ outages,
                              const int32_t* __restrict__ pre, const int32_t* __restrict__ isl_lo,
                              const int32_t* __restrict__ isl_cnt,
                              const int32_t* __restrict__ lab_isl,
                              const int32_t* __restrict__ lab_main, int32_t* label_out) {
  const size_t total = (size_t)S * n;
  for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < total;
       k += (size_t)gridDim.x * blockDim.x) {
    const int s = (int)(k / n), b = (int)(k % n);
    const int l = outages[s];
    label_out[k] = in_island(pre[b], isl_lo[s], isl_cnt[s]) ? lab_isl[l] : lab_main[l];
  }
}

// prefP[k] = sum of P over the buses of preorder < k (ord[j]: the bus of
// preorder j), in a fixed order: each thread sums a contiguous chunk, one
// thread scans the chunk sums.
__global__ void __launch_bounds__(1024) preorder_prefix_kernel(int n,
                                                               const int32_t* __restrict__ ord,
                                                               const double* __restrict__ P,
                                                               double* prefP) {
  __shared__ double part[1024];
  const int t = threadIdx.x;
  const int chunk = (n + 1023) / 1024;
  const int a = min(n, t * chunk), b = min(n, a + chunk);
  double s = 0.0;
  for (int k = a; k < b; ++k) s += P[ord[k]];
  part[t] = s;
  __syncthreads();
  if (t == 0) {
    double run = 0.0;
    for (int k = 0; k < 1024; ++k) {
      const double v = part[k];
      part[k] = run;
      run += v;
    }
    prefP[n] = run;
  }
  __syncthreads();
  double run = part[t];
  for (int k = a; k < b; ++k) {
    prefP[k] = run;
    run += P[ord[k]];
  }
}

// Generator outages, one thread per scenario: no branch out (outage -1),
// nothing islanded, and the tripped bus's P_gen shared by the other PV
// generators with P_gen > 0 in proportion to theirs (coef = P_gen,k over
// their total; no_gen when there are none).  gen_bus: internal bus indices
// of PV buses (checked on the host).
__global__ void gen_outage_kernel(int S, int n, const int32_t* __restrict__ gen_bus,
                                  const double* __restrict__ P_gen,
                                  const double* __restrict__ prefG,
                                  const int32_t* __restrict__ prefGc, int32_t* outage,
                                  int32_t* isl_lo, int32_t* isl_cnt, double* coef,
                                  int32_t* no_gen) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= S) return;
  const int k = gen_bus[s];
  const double pg = P_gen[k];
  const bool in = pg > 0.0;  // k counts among the sharing generators
  const int others = prefGc[n] - (in ? 1 : 0);
  const double rest = prefG[n] - (in ? pg : 0.0);
  outage[s] = -1;
  isl_lo[s] = 0;
  isl_cnt[s] = 0;
  no_gen[s] = others == 0;
  coef[s] = others == 0 ? 0.0 : pg / rest;
}

cudaError_t launch_gen_outages(cudaStream_t st, int S, int n, const int32_t* gen_bus,
                               const double* P_gen, const IslandPlan& I, int32_t* outage,
                               int32_t* isl_lo, int32_t* isl_cnt, double* coef, int32_t* no_gen,
                               int32_t* label_out) {
  if (S == 0) return cudaSuccess;
  gen_outage_kernel<<<(S + 255) / 256, 256, 0, st>>>(S, n, gen_bus, P_gen, I.prefG, I.prefGc,
                                                      outage, isl_lo, isl_cnt, coef, no_gen);
  cudaError_t e = cudaGetLastError();
  // one component: every bus carries the smallest bus index, 0
  if (e == cudaSuccess && label_out)
    e = cudaMemsetAsync(label_out, 0, (size_t)S * n * sizeof(int32_t), st);
  return e;
}

cudaError_t launch_islands(cudaStream_t st, int S, int n, const int32_t* outages,
                           const IslandPlan& I, const double* P_user, double* prefP_scratch,
                           int32_t* isl_lo, int32_t* isl_cnt, double* coef, int32_t* no_gen,
                           int32_t* label_out) {
  if (S == 0) return cudaSuccess;
  const double* prefP = I.prefPs;
  if (P_user) {
    preorder_prefix_kernel<<<1, 1024, 0, st>>>(n, I.ord_u, P_user, prefP_scratch);
    prefP = prefP_scratch;
  }
  islands_kernel<<<(S + 255) / 256, 256, 0, st>>>(S, outages, I.br_lo, I.br_cnt, prefP, I.prefG,
                                                   I.prefGc, n, isl_lo, isl_cnt, coef, no_gen);
  if (label_out) {
    const size_t total = (size_t)S * n;
    const int grid = (int)std::min<size_t>((total + 255) / 256, 152 * 64);
    labels_kernel<<<grid, 256, 0, st>>>(S, n, outages, I.u_pre, isl_lo, isl_cnt, I.lab_isl,
                                        I.lab_main, label_out);
  }
  return cudaGetLastError();
}

}  // namespace gpcg
