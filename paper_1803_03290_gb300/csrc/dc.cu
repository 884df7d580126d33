// The N-1 quick screen of the P-theta equation alone (Sec. IV.A): eq. (4)
// with |V| = 1, i.e. the DC power flow of every single-branch outage.
//
// For scenario s (outage l): B'_s theta_s = R_s P on the main island's
// non-slack buses, with B'_s the base matrix minus the outaged branch's
// four-element change (Sec. IV.B), islanded buses removed and their net
// injection re-dispatched over the main island's generators (Sec. IV.C).
// One batched PCG solve per scenario with the base-case preconditioner
// (eq. (6)) -- with FP32 vectors and factors, followed by one step of
// iterative refinement (FP64 residual with the FP64 matrix, FP32 solve,
// FP64 update) -- then branch flows f_k = (theta_i - theta_j) / x_k and the
// loading max_k |f_k| / rating_k.  Tiles of two scenarios are dealt to CTAs
// statically.
#include "fdpf_ops.cuh"

namespace gpcg {

template <typename VT>
__global__ void __launch_bounds__(NTHREADS, FDPF_MIN_BLOCKS)
    dc_tiles_kernel(FdpfParams P, DcParamsView D, DevMatT<VT> M, DevMatT<double> M64) {
  constexpr int T = 2;
  static_assert(Geo<T>::LP == 2, "one thread per row, two lanes");
  __shared__ LaneState<T> L;
  const Geo<T> g;
  const int tid = threadIdx.x;
  const DevGrid& G = P.G;
  VT* x = (VT*)P.wx + (size_t)blockIdx.x * P.vstride;
  VT* r = (VT*)P.wr + (size_t)blockIdx.x * P.vstride;
  VT* p = (VT*)P.wp + (size_t)blockIdx.x * P.vstride;
  VT* q = (VT*)P.wq + (size_t)blockIdx.x * P.vstride;
  VT* z = (VT*)P.wz + (size_t)blockIdx.x * P.vstride;
  double* th = P.wth + (size_t)blockIdx.x * P.sstride;  // theta by bus, [bus][lane]
  // FP64 work by row for the refinement step: solution, B_s x, right-hand side
  double* xd = P.wV + (size_t)blockIdx.x * P.sstride;
  double* qd = P.we + (size_t)blockIdx.x * P.sstride;
  double* bd = P.wf + (size_t)blockIdx.x * P.sstride;
  __shared__ Stamp<T, double> St64;
  const int l0 = g.lane, l1 = g.lane + 1;
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
      L.wP[ln] = l >= 0 ? M.w[l] : 0.0;
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
      const double pi = D.P[i];
      const double pg = G.bus_type[i] == 1 ? fmax(G.P_gen[i], 0.0) : 0.0;
      const double a = (v0 && !in_island(pr, lo0, cnt0)) ? fma(L.coef[l0], pg, pi) : 0.0;
      const double b = (v1 && !in_island(pr, lo1, cnt1)) ? fma(L.coef[l1], pg, pi) : 0.0;
      st2(r + (size_t)k * T + g.lane, Pair<VT>{(VT)a, (VT)b});
      st2(bd + (size_t)k * T + g.lane, Pair<double>{a, b});
    }
    __syncthreads();
    pcg_solve<T, VT>(P, M, L, x, r, p, q, z, L.raP, L.rbP, L.wP, L.inP);
    for (int k = g.rs; k < M.n; k += Geo<T>::RPS) {
      const Pair<VT> xv = ld2(x + (size_t)k * T + g.lane);
      st2(xd + (size_t)k * T + g.lane, Pair<double>{(double)xv.a, (double)xv.b});
    }
    if constexpr (sizeof(VT) < sizeof(double)) {
      // one step of iterative refinement: the FP64 residual b - B_s x (with
      // the FP64 matrix), its FP32 solve, and the FP64 update of x
      if (tid < T) {
        const bool on = L.active[tid];
        St64.ra[tid] = on ? L.raP[tid] : -1;
        St64.rb[tid] = on ? L.rbP[tid] : -1;
        St64.w[tid] = L.wP[tid];
        St64.c[tid] = 1.0;
      }
      if (g.rs == 0) st2(xd + (size_t)M.n * T + g.lane, Pair<double>{0.0, 0.0});
      __syncthreads();
      const unsigned long long filt = stamp_filter<T, double>(St64);
      spmv_pass<T, double, false>(M64, xd, nullptr, qd, St64, filt, vzero<double, 2>(), true,
                                  nullptr);
      __syncthreads();  // the SpMV writes rows in bus order, read below by slot
      for (int k = g.rs; k < M.n; k += Geo<T>::RPS) {
        const int pr = M.pre_of_row[k];
        const size_t o = (size_t)k * T + g.lane;
        const Pair<double> b_ = ld2(bd + o), q_ = ld2(qd + o);
        const double a = (v0 && !in_island(pr, lo0, cnt0)) ? b_.a - q_.a : 0.0;
        const double b = (v1 && !in_island(pr, lo1, cnt1)) ? b_.b - q_.b : 0.0;
        st2(r + o, Pair<VT>{(VT)a, (VT)b});
      }
      __syncthreads();
      pcg_solve<T, VT>(P, M, L, x, r, p, q, z, L.raP, L.rbP, L.wP, L.inP);
      for (int k = g.rs; k < M.n; k += Geo<T>::RPS) {
        const size_t o = (size_t)k * T + g.lane;
        const Pair<VT> dx = ld2(x + o);
        const Pair<double> x0 = ld2(xd + o);
        st2(xd + o, Pair<double>{x0.a + (double)dx.a, x0.b + (double)dx.b});
      }
    }
    __syncthreads();
    // theta by bus (slack and islanded buses 0: no row, or x kept at 0)
    for (int i = g.rs; i < G.n; i += Geo<T>::RPS) {
      const int k = M.row_of_bus[i];
      const Pair<double> t = k >= 0 ? ld2(xd + (size_t)k * T + g.lane) : Pair<double>{0.0, 0.0};
      st2(th + (size_t)i * T + g.lane, t);
      if (D.theta) {
        const int iu = D.user_of_bus[i];
        if (v0) D.theta[(size_t)L.scen[l0] * G.n + iu] = t.a;
        if (v1) D.theta[(size_t)L.scen[l1] * G.n + iu] = t.b;
      }
    }
    __syncthreads();
    // flows on the branches in service between main-island buses; loading,
    // and the branches loaded above their rating (count and bit mask)
    Vec<unsigned long long, 2> ml = vzero<unsigned long long, 2>();
    Vec<int, 2> nov = vzero<int, 2>();
    const int nw = (G.m + 31) >> 5;
    if (D.ovmask) {
      for (int w = g.rs; w < nw; w += Geo<T>::RPS) {
        if (v0) D.ovmask[(size_t)L.scen[l0] * nw + w] = 0u;
        if (v1) D.ovmask[(size_t)L.scen[l1] * nw + w] = 0u;
      }
      __syncthreads();  // the rows are cleared before any bit is set
    }
    for (int k = g.rs; k < G.m; k += Geo<T>::RPS) {
      const int a = G.f[k], b = G.t[k];
      const int pa = G.pre[a], pb = G.pre[b];
      const double bk = M.w[k], ir = G.inv_rating[k];
      const Pair<double> ta = ld2(th + (size_t)a * T + g.lane), tb = ld2(th + (size_t)b * T + g.lane);
      double f0 = 0.0, f1 = 0.0;
      if (v0 && k != br0 && !in_island(pa, lo0, cnt0) && !in_island(pb, lo0, cnt0)) {
        f0 = bk * (ta.a - tb.a);
        const double ld = f0 * ir;
        upd_max_bits(ml.v[0], ld);
        if (overloaded(ld)) {
          nov.v[0] += 1;
          if (D.ovmask) atomicOr(D.ovmask + (size_t)L.scen[l0] * nw + (k >> 5), 1u << (k & 31));
        }
      }
      if (v1 && k != br1 && !in_island(pa, lo1, cnt1) && !in_island(pb, lo1, cnt1)) {
        f1 = bk * (ta.b - tb.b);
        const double ld = f1 * ir;
        upd_max_bits(ml.v[1], ld);
        if (overloaded(ld)) {
          nov.v[1] += 1;
          if (D.ovmask) atomicOr(D.ovmask + (size_t)L.scen[l1] * nw + (k >> 5), 1u << (k & 31));
        }
      }
      if (D.flow) {
        if (v0) D.flow[(size_t)L.scen[l0] * G.m + k] = f0;
        if (v1) D.flow[(size_t)L.scen[l1] * G.m + k] = f1;
      }
    }
    const Vec<unsigned long long, 2> mlb = lane_max_bits<T, RS_LOAD>(L, ml);
    if (D.nover) nov = lane_sum<T, RS_BB>(L, nov);
    if (g.rs == 0) {
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        const int ln = g.lane + j, s = L.scen[ln];
        if (s < 0) continue;
        if (D.maxload) D.maxload[s] = from_bits(mlb.v[j]);
        if (D.nover) D.nover[s] = nov.v[j];
        if (D.iters) D.iters[s] = L.inP[ln];
        if (D.status) D.status[s] = (L.cnt[ln] > 0 && L.nogen[ln]) ? 3 : 0;
      }
    }
    __syncthreads();
  }
}

template <typename VT>
cudaError_t launch_dc(cudaStream_t st, int grid, const FdpfParams& P, const DcParamsView& D,
                      const DevMatT<VT>& M, const DevMatT<double>& M64) {
  dc_tiles_kernel<VT><<<grid, NTHREADS, 0, st>>>(P, D, M, M64);
  return cudaGetLastError();
}

template <typename VT>
int dc_max_blocks_per_sm() {
  int nb = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, dc_tiles_kernel<VT>, NTHREADS, 0);
  return nb;
}

template cudaError_t launch_dc<float>(cudaStream_t, int, const FdpfParams&, const DcParamsView&,
                                      const DevMatT<float>&, const DevMatT<double>&);
template cudaError_t launch_dc<double>(cudaStream_t, int, const FdpfParams&, const DcParamsView&,
                                       const DevMatT<double>&, const DevMatT<double>&);
template int dc_max_blocks_per_sm<float>();
template int dc_max_blocks_per_sm<double>();

}  // namespace gpcg
