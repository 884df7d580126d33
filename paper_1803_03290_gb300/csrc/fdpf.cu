// Instantiation of the persistent N-1 kernel (fdpf_kernel.cuh) for branch
// outages, the batched operator application used to verify the operators,
// and the base-case helpers.  The generator-outage kernel is built in
// fdpf_gen.cu.
#include "fdpf_kernel.cuh"

namespace gpcg {

// Batched operator application for verification (gpcg_apply): X and Y are
// [S][rows]; each CTA handles tiles of T scenarios.
template <int T, typename VT>
__global__ void __launch_bounds__(NTHREADS) apply_kernel(DevMatT<VT> M, int op, int S,
                                                         const int32_t* outages,
                                                         const int32_t* f_, const int32_t* t_,
                                                         const double* X, double* Y, VT* wbuf,
                                                         size_t vstride, int precond) {
  constexpr int LP = Geo<T>::LP;
  __shared__ __align__(16) VT zt[TAIL_ROWS * T];
  __shared__ Stamp<T, VT> St;
  const Geo<T> g;
  VT* a = wbuf + (size_t)blockIdx.x * 3 * vstride;
  VT* b = a + vstride;
  VT* c = b + vstride;
  const int ntiles = (S + T - 1) / T;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    if (threadIdx.x < T) {
      const int s = tile * T + threadIdx.x;
      const int l = s < S ? outages[s] : -1;
      St.ra[threadIdx.x] = l >= 0 ? M.row_of_bus[f_[l]] : -1;
      St.rb[threadIdx.x] = l >= 0 ? M.row_of_bus[t_[l]] : -1;
      St.w[threadIdx.x] = l >= 0 ? (VT)M.w[l] : (VT)0;
      St.c[threadIdx.x] = l >= 0 && M.c ? (VT)M.c[l] : (VT)1;
    }
    for (int i = g.rs; i <= M.n; i += Geo<T>::RPS) {
      Vec<VT, LP> v = vzero<VT, LP>();
      if (i < M.n)
#pragma unroll
        for (int j = 0; j < LP; ++j) {
          const int s = tile * T + g.lane + j;
          if (s < S) v.v[j] = (VT)X[(size_t)s * M.n + i];
        }
      stv<LP>(a + (size_t)i * T + g.lane, v);
      stv<LP>(b + (size_t)i * T + g.lane, vzero<VT, LP>());
    }
    __syncthreads();
    const unsigned long long filt = stamp_filter<T, VT>(St);
    const Vec<VT, LP> zero = vzero<VT, LP>();
    if (op == 0) {
      spmv_pass<T, VT, false>(M, a, nullptr, b, St, filt, zero, true, nullptr);
    } else if (precond == PREC_JACOBI) {
      Vec<VT, LP> rr = zero, rz = zero;
      jacobi_pass<T, VT, false>(M, c, a, nullptr, nullptr, b, zero, St, rr, rz);
    } else {
      Vec<VT, LP> rzt = zero;
      fwd_pass<T, VT, false>(M, c, a, nullptr, nullptr, b, zero, zt, rzt);
      bwd_pass<T, VT>(M, a, b, rzt);
    }
    __syncthreads();
    for (int i = g.rs; i < M.n; i += Geo<T>::RPS) {
      const Vec<VT, LP> v = ldv<LP>(b + (size_t)i * T + g.lane);
#pragma unroll
      for (int j = 0; j < LP; ++j) {
        const int s = tile * T + g.lane + j;
        if (s < S) Y[(size_t)s * M.n + i] = (double)v.v[j];
      }
    }
    __syncthreads();
  }
}

// Mismatch of the intact grid at the base-case state (eqs. (1)-(3)), per bus:
// r0P = P_sched - P(V0), r0Q = Q_sched - Q(V0), summed like mismatch_pass.
// At a scenario's warm start only the two ends of the outaged branch see a
// different network, so its first P half-step takes every other bus's
// mismatch from here (plus the re-dispatch).
__global__ void base_residual_kernel(DevGrid G, const double* __restrict__ V0,
                                     const double* __restrict__ c0,
                                     const double* __restrict__ s0, double* r0P, double* r0Q) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= G.n) return;
  const double ei = V0[i] * c0[i], fi = V0[i] * s0[i];
  double re = fma(G.Gii[i], ei, -G.Bii[i] * fi), im = fma(G.Gii[i], fi, G.Bii[i] * ei);
  const int deg = G.adj_deg[i];
  for (int a = 0; a < deg; ++a) {
    const int j = G.adj_nbr[(size_t)a * G.n + i];
    const double gv = G.adj_g[(size_t)a * G.n + i], bv = G.adj_b[(size_t)a * G.n + i];
    const double ej = V0[j] * c0[j], fj = V0[j] * s0[j];
    re = fma(-gv, ej, fma(bv, fj, re));
    im = fma(-gv, fj, fma(-bv, ej, im));
  }
  for (int e = G.adj_optr[i]; e < G.adj_optr[i + 1]; ++e) {
    const int j = G.adj_onbr[e];
    const double ej = V0[j] * c0[j], fj = V0[j] * s0[j];
    re = fma(-G.adj_og[e], ej, fma(G.adj_ob[e], fj, re));
    im = fma(-G.adj_og[e], fj, fma(-G.adj_ob[e], ej, im));
  }
  r0P[i] = fma(-ei, re, fma(-fi, im, G.P_sched[i]));
  r0Q[i] = fma(-fi, re, fma(ei, im, G.Q_sched[i]));
}

cudaError_t launch_base_residual(cudaStream_t st, const DevGrid& G, const double* V0,
                                 const double* c0, const double* s0, double* r0P, double* r0Q) {
  base_residual_kernel<<<(G.n + 255) / 256, 256, 0, st>>>(G, V0, c0, s0, r0P, r0Q);
  return cudaGetLastError();
}

// Base-case cos/sin per bus, shared by every scenario's warm start.
__global__ void base_trig_kernel(int n, const double* th, double* c, double* s) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) sincos(th[i], &s[i], &c[i]);
}

// ----------------------------------------------------------- launchers
template <typename VT>
cudaError_t launch_fdpf(cudaStream_t st, int T, int grid, const FdpfParams& P,
                        const DevMatT<VT>& MP, const DevMatT<VT>& MQ, size_t zbytes) {
  if (P.sc.gen_bus || P.G.qmax) {
    if (zbytes) return cudaErrorInvalidValue;
    return launch_fdpf_gen<VT>(st, T, grid, P, MP, MQ);
  }
  return launch_fdpf_g<false, VT>(st, T, grid, P, MP, MQ, zbytes);
}

template <typename VT>
int fdpf_max_blocks_per_sm(int T, bool gen, size_t zbytes) {
  if (gen) return zbytes ? 0 : fdpf_blocks_gen<VT>(T);
  return fdpf_blocks_g<false, VT>(T, zbytes);
}

template <typename VT>
cudaError_t launch_apply(cudaStream_t st, int grid, const DevMatT<VT>& M, int op, int S,
                         const int32_t* outages, const int32_t* f, const int32_t* t,
                         const double* X, double* Y, VT* wbuf, size_t vstride, int precond) {
  apply_kernel<32, VT><<<grid, NTHREADS, 0, st>>>(M, op, S, outages, f, t, X, Y, wbuf, vstride,
                                                  precond);
  return cudaGetLastError();
}

cudaError_t launch_base_trig(cudaStream_t st, int n, const double* th, double* c, double* s) {
  base_trig_kernel<<<(n + 255) / 256, 256, 0, st>>>(n, th, c, s);
  return cudaGetLastError();
}

template cudaError_t launch_fdpf<float>(cudaStream_t, int, int, const FdpfParams&,
                                        const DevMatT<float>&, const DevMatT<float>&, size_t);
template cudaError_t launch_fdpf<double>(cudaStream_t, int, int, const FdpfParams&,
                                         const DevMatT<double>&, const DevMatT<double>&, size_t);
template int fdpf_max_blocks_per_sm<float>(int, bool, size_t);
template int fdpf_max_blocks_per_sm<double>(int, bool, size_t);
template cudaError_t launch_apply<float>(cudaStream_t, int, const DevMatT<float>&, int, int,
                                         const int32_t*, const int32_t*, const int32_t*,
                                         const double*, double*, float*, size_t, int);
template cudaError_t launch_apply<double>(cudaStream_t, int, const DevMatT<double>&, int, int,
                                          const int32_t*, const int32_t*, const int32_t*,
                                          const double*, double*, double*, size_t, int);

}  // namespace gpcg
