// Islanding detection (Sec. IV.C) for a batch of outage scenarios, and the
// per-scenario data of the proportional re-dispatch.
//
// One CTA takes one scenario at a time: every bus's parent pointer lives in
// shared memory; the CTA unites the two ends of every in-service branch
// (the outaged branch is skipped), always hooking the larger root under the
// smaller one, so that each component's final root is its smallest bus
// index -- the canonical label.  The main island is the slack's component.
//
// For a single-branch outage of a connected grid the islanded buses are
// exactly one subtree of a depth-first tree rooted at the slack, hence one
// interval of the depth-first preorder.  The kernel records that interval
// (and checks that the island really fills it), so the solve kernels can
// test island membership with one comparison per bus.
#include "common.cuh"

namespace gpcg {

__device__ __forceinline__ int uf_find(volatile int32_t* p, int x) {
  int px = p[x];
  while (px != x) {
    int gp = p[px];
    p[x] = gp;  // path halving; parents only ever decrease
    x = px;
    px = gp;
  }
  return x;
}

__device__ __forceinline__ void uf_unite(int32_t* p, int a, int b) {
  volatile int32_t* vp = p;
  a = uf_find(vp, a);
  b = uf_find(vp, b);
  while (a != b) {
    if (a < b) { int t = a; a = b; b = t; }
    int old = atomicCAS(&p[a], a, b);
    if (old == a) return;
    a = uf_find(vp, old);
    b = uf_find(vp, b);
  }
}

template <int NT>
__global__ void __launch_bounds__(NT) islands_kernel(
    int n, int m, int slack, int S, const int32_t* __restrict__ outages,
    const int32_t* __restrict__ f, const int32_t* __restrict__ t,
    const int8_t* __restrict__ bus_type, const double* __restrict__ P_sched,
    const double* __restrict__ P_gen, const int32_t* __restrict__ pre,
    int32_t* isl_lo, int32_t* isl_cnt, double* coef, int32_t* no_gen, int32_t* label_out,
    int32_t* err) {
  extern __shared__ int32_t parent[];
  __shared__ double red_d[2][NT / 32];
  __shared__ int32_t red_i[3][NT / 32];
  const int tid = threadIdx.x, wid = tid >> 5, ln = tid & 31;
  for (int s = blockIdx.x; s < S; s += gridDim.x) {
    int l = outages[s];
    for (int i = tid; i < n; i += NT) parent[i] = i;
    __syncthreads();
    for (int e = tid; e < m; e += NT)
      if (e != l) uf_unite(parent, f[e], t[e]);
    __syncthreads();
    for (int i = tid; i < n; i += NT) parent[i] = uf_find(parent, i);
    __syncthreads();
    int main_lab = parent[slack];
    double sumP = 0.0, genM = 0.0;  // island net injection, main-island PV generation
    int cnt = 0, lo = 0x7fffffff, hi = -1;
    for (int i = tid; i < n; i += NT) {
      int lab = parent[i];
      if (label_out) label_out[(size_t)s * n + i] = lab;
      if (lab == main_lab) {
        if (bus_type[i] == 1 && P_gen[i] > 0.0) genM += P_gen[i];
      } else {
        ++cnt;
        sumP += P_sched[i];
        int pr = pre[i];
        lo = min(lo, pr);
        hi = max(hi, pr);
      }
    }
    for (int o = 16; o; o >>= 1) {
      sumP += __shfl_xor_sync(0xffffffffu, sumP, o);
      genM += __shfl_xor_sync(0xffffffffu, genM, o);
      cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
      lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
      hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    if (ln == 0) {
      red_d[0][wid] = sumP; red_d[1][wid] = genM;
      red_i[0][wid] = cnt; red_i[1][wid] = lo; red_i[2][wid] = hi;
    }
    __syncthreads();
    if (tid == 0) {
      double sp = 0.0, gi = 0.0;
      int c = 0, a = 0x7fffffff, b = -1;
      for (int w = 0; w < NT / 32; ++w) {  // fixed order: deterministic sums
        sp += red_d[0][w]; gi += red_d[1][w];
        c += red_i[0][w]; a = min(a, red_i[1][w]); b = max(b, red_i[2][w]);
      }
      if (c > 0 && b - a + 1 != c) atomicExch(err, 3);
      isl_lo[s] = c > 0 ? a : 0;
      isl_cnt[s] = c;
      const double den = gi;  // main-island PV generation
      int ng = (c > 0) && !(den > 0.0);
      no_gen[s] = ng;
      coef[s] = (c > 0 && !ng) ? sp / den : 0.0;
    }
    __syncthreads();
  }
}

size_t islands_smem(int n) { return (size_t)n * sizeof(int32_t); }

cudaError_t launch_islands(cudaStream_t st, int grid, int n, int m, int slack, int S,
                           const int32_t* outages, const int32_t* f, const int32_t* t,
                           const int8_t* bus_type, const double* P_sched, const double* P_gen,
                           const int32_t* pre, int32_t* isl_lo,
                           int32_t* isl_cnt, double* coef, int32_t* no_gen, int32_t* label_out,
                           int32_t* err) {
  if (S == 0) return cudaSuccess;
  size_t smem = islands_smem(n);
  cudaError_t ce = cudaFuncSetAttribute(islands_kernel<512>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (ce != cudaSuccess) return ce;
  islands_kernel<512><<<grid, 512, smem, st>>>(n, m, slack, S, outages, f, t, bus_type, P_sched,
                                               P_gen, pre, isl_lo, isl_cnt, coef,
                                               no_gen, label_out, err);
  return cudaGetLastError();
}

}  // namespace gpcg
