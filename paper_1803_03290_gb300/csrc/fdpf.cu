// The persistent N-1 kernel: one CTA owns a tile of T scenarios and runs the
// whole fast-decoupled power flow of that tile (Sec. III.B eqs. (4)-(5),
// Sec. IV) without leaving the kernel, then takes the next tile from a
// device-side counter.  Vectors live in global memory as [row][T] per CTA
// slot, so every row access of a warp is one contiguous chunk across the
// tile's scenarios.  Tiles are independent: the only inter-CTA traffic is
// the atomic tile counter, and no CTA ever waits on another.
//
// Per outer iteration and scenario (Sec. III.B, eqs. (4)-(5)):
//   FP64 mismatch dP, dQ (eqs. (1)-(3)), convergence test;
//   PCG on B'_s dtheta = dP/V preconditioned by the base-case factor
//   (Sec. IV.B eq. (6)); theta += dtheta (FP64);
//   FP64 mismatch dQ; PCG on B''_s dV = dQ/V; V += dV (FP64).
// B'_s and B''_s are the base-case matrices with the outaged branch's
// four-element change (Sec. IV.B) applied on the fly inside the SpMV.
// Islanded buses (Sec. IV.C) are masked out of the right-hand side and of
// the search directions; their state stays zero.
#include <math.h>
#include "common.cuh"
#include "fdpf.h"

namespace gpcg {

// Inner iterations without progress after which a solve stops: the outer
// FP64 loop then refines the answer (iterative refinement).
constexpr int STALL_ITERS = 16;

// ------------------------------------------------------------ lane state
template <int T>
struct LaneState {
  int scen[T], l[T], fb[T], tb[T], lo[T], cnt[T];
  int raP[T], rbP[T], raQ[T], rbQ[T];
  double wP[T], wQ[T], coef[T], gl[T], bl[T], bshl[T];
  int active[T], outer[T], inP[T], inQ[T], status[T], nogen[T];
  double err[T];
  double rz[T], bb[T], alpha[T], beta[T], rrmin[T];
  int pdone[T], stall[T];
  double red[NTHREADS];
  int flag;
  int tile;
};

// Sum (or max) over the R row groups of each lane's partial value.
template <int T, bool MAX>
__device__ __forceinline__ double lane_reduce(LaneState<T>& L, double v) {
  constexpr int R = NTHREADS / T;
  const int tid = threadIdx.x;
  L.red[tid] = v;
  __syncthreads();
#pragma unroll
  for (int st = R / 2; st > 0; st >>= 1) {
    if (tid / T < st) {
      double a = L.red[tid], b = L.red[tid + st * T];
      L.red[tid] = MAX ? ((b > a || b != b) ? b : a) : a + b;
    }
    __syncthreads();
  }
  double out = L.red[tid % T];
  __syncthreads();
  return out;
}

// True when some lane has a nonzero entry in `flags` (block-uniform).
template <int T>
__device__ __forceinline__ bool any_lane_d(LaneState<T>& L, const double* flags) {
  __syncthreads();
  if (threadIdx.x == 0) {
    int any = 0;
    for (int s = 0; s < T; ++s) any |= (flags[s] != 0.0);
    L.flag = any;
  }
  __syncthreads();
  const bool r = L.flag != 0;
  __syncthreads();
  return r;
}

// True when some lane has a nonzero entry in `flags` (block-uniform).
template <int T>
__device__ __forceinline__ bool any_lane(LaneState<T>& L, const int* flags) {
  __syncthreads();
  if (threadIdx.x == 0) {
    int any = 0;
    for (int s = 0; s < T; ++s) any |= flags[s];
    L.flag = any;
  }
  __syncthreads();
  const bool r = L.flag != 0;
  __syncthreads();
  return r;
}

__device__ __forceinline__ void upd_max(double& m, double d) {
  double a = fabs(d);
  if (!(a <= m)) m = (a == a) ? a : INFINITY;
}

// ----------------------------------------------------- batched operators
// q = B_s p for the lane's scenario: base CSR times p, plus the outaged
// branch's four-element change (Sec. IV.B) -- off-diagonal +w, diagonal -w
// at both ends.  Returns the lane's partial p.q.
template <int T, typename VT>
__device__ __forceinline__ double spmv_pass(const DevMatT<VT>& M, const VT* p, VT* q, int ra,
                                            int rb, VT w) {
  constexpr int R = NTHREADS / T;
  const int lane = threadIdx.x % T, rg = threadIdx.x / T;
  double pq = 0.0;
  for (int i = rg; i < M.n; i += R) {
    const int oth = (i == ra) ? rb : ((i == rb) ? ra : -2);
    VT acc = 0, pi = 0;
    for (int k = M.a_ptr[i]; k < M.a_ptr[i + 1]; ++k) {
      const int c = M.a_idx[k];
      const VT pc = p[(size_t)c * T + lane];
      acc += M.a_val[k] * pc;
      if (c == oth) acc += w * pc;
      if (c == i) pi = pc;
    }
    if (oth != -2) acc -= w * pi;
    q[(size_t)i * T + lane] = acc;
    pq += (double)(pi * acc);
  }
  return pq;
}

// Forward substitution L y = r over the level schedule (rows of one level
// are independent).  With FUSED, first x += alpha p and r -= alpha q (the
// PCG update), accumulating r.r; without it, accumulates r.r of the input.
template <int T, typename VT, bool FUSED>
__device__ __forceinline__ double fwd_pass(const DevMatT<VT>& M, VT* x, VT* r, const VT* p,
                                           const VT* q, VT* z, VT alpha) {
  constexpr int R = NTHREADS / T;
  const int lane = threadIdx.x % T, rg = threadIdx.x / T;
  double rr = 0.0;
  for (int lev = 0; lev < M.nlev; ++lev) {
    const int r0 = M.lev_ptr[lev], r1 = M.lev_ptr[lev + 1];
    for (int i = r0 + rg; i < r1; i += R) {
      const size_t o = (size_t)i * T + lane;
      VT ri = r[o];
      if (FUSED) {
        const VT pi = p[o];
        x[o] += alpha * pi;
        ri -= alpha * q[o];
        r[o] = ri;
      } else {
        x[o] = 0;
      }
      rr += (double)(ri * ri);
      const int ks = M.l_ptr[i], ke = M.l_ptr[i + 1] - 1;
      VT acc = ri;
      for (int k = ks; k < ke; ++k) acc -= M.l_val[k] * z[(size_t)M.l_idx[k] * T + lane];
      z[o] = acc / M.l_val[ke];
    }
    __syncthreads();
  }
  return rr;
}

// Back substitution L^T z = y in place (z holds y on entry), over the
// backward level schedule; accumulates r.z.
template <int T, typename VT>
__device__ __forceinline__ double bwd_pass(const DevMatT<VT>& M, const VT* r, VT* z) {
  constexpr int R = NTHREADS / T;
  const int lane = threadIdx.x % T, rg = threadIdx.x / T;
  double rz = 0.0;
  for (int lev = 0; lev < M.nblev; ++lev) {
    const int r0 = M.blev_ptr[lev], r1 = M.blev_ptr[lev + 1];
    for (int k0 = r0 + rg; k0 < r1; k0 += R) {
      const int i = M.blev_rows[k0];
      const size_t o = (size_t)i * T + lane;
      const int ks = M.u_ptr[i], ke = M.u_ptr[i + 1];  // diagonal first
      VT acc = z[o];
      for (int k = ks + 1; k < ke; ++k) acc -= M.u_val[k] * z[(size_t)M.u_idx[k] * T + lane];
      const VT zi = acc / M.u_val[ks];
      z[o] = zi;
      rz += (double)(r[o] * zi);
    }
    __syncthreads();
  }
  return rz;
}

// Jacobi: z = r / diag(B_s) (the diagonal with the outage applied).
template <int T, typename VT, bool FUSED>
__device__ __forceinline__ void jacobi_pass(const DevMatT<VT>& M, VT* x, VT* r, const VT* p,
                                            const VT* q, VT* z, VT alpha, int ra, int rb, VT w,
                                            double& rr, double& rz) {
  constexpr int R = NTHREADS / T;
  const int lane = threadIdx.x % T, rg = threadIdx.x / T;
  for (int i = rg; i < M.n; i += R) {
    const size_t o = (size_t)i * T + lane;
    VT ri = r[o];
    if (FUSED) {
      x[o] += alpha * p[o];
      ri -= alpha * q[o];
      r[o] = ri;
    } else {
      x[o] = 0;
    }
    VT d = M.diag[i] - ((i == ra || i == rb) ? w : (VT)0);
    VT zi = ri / d;
    z[o] = zi;
    rr += (double)(ri * ri);
    rz += (double)(ri * zi);
  }
  __syncthreads();
}

// p = mask(z) + beta p: islanded rows keep a zero search direction.
template <int T, typename VT>
__device__ __forceinline__ void pupdate_pass(const DevMatT<VT>& M, const VT* z, VT* p, VT beta,
                                             int lo, int cnt, bool first) {
  constexpr int R = NTHREADS / T;
  const int lane = threadIdx.x % T, rg = threadIdx.x / T;
  for (int i = rg; i < M.n; i += R) {
    const size_t o = (size_t)i * T + lane;
    const bool isl = in_island(M.pre_of_row[i], lo, cnt);
    VT zi = isl ? (VT)0 : z[o];
    p[o] = first ? zi : zi + beta * p[o];
  }
  __syncthreads();
}

// ------------------------------------------------------------ the solve
// Batched PCG (Sec. III.A listing, read as textbook PCG) on B_s x = r for
// the lanes that are active; x starts at 0.  Returns nothing; adds the
// lane's iteration count to *iters.
template <int T, typename VT>
__device__ void pcg_solve(const FdpfParams& P, const DevMatT<VT>& M, LaneState<T>& L, VT* x,
                          VT* r, VT* p, VT* q, VT* z, const int* ra_, const int* rb_,
                          const double* w_, int* iters) {
  const int tid = threadIdx.x, lane = tid % T, rg = tid / T;
  const int ra = ra_[lane], rb = rb_[lane];
  const VT w = (VT)w_[lane];
  const int lo = L.lo[lane], cnt = L.cnt[lane];
  const bool jac = (P.precond == PREC_JACOBI);
  if (rg == 0) L.pdone[lane] = !L.active[lane];
  __syncthreads();
  double bbp = 0.0, rzp = 0.0;
  if (jac) {
    jacobi_pass<T, VT, false>(M, x, r, p, q, z, (VT)0, ra, rb, w, bbp, rzp);
  } else {
    bbp = fwd_pass<T, VT, false>(M, x, r, p, q, z, (VT)0);
    rzp = bwd_pass<T, VT>(M, r, z);
  }
  const double bb = lane_reduce<T, false>(L, bbp);
  const double rz0 = lane_reduce<T, false>(L, rzp);
  pupdate_pass<T, VT>(M, z, p, (VT)0, lo, cnt, true);
  if (rg == 0) {
    L.bb[lane] = bb;
    L.rz[lane] = rz0;
    L.rrmin[lane] = bb;
    L.stall[lane] = 0;
    if (!(bb > 0.0) || !(rz0 > 0.0)) L.pdone[lane] = 1;
  }
  const double tol2 = P.inner_rtol * P.inner_rtol;
  for (int it = 0; it < P.max_inner; ++it) {
    if (rg == 0) L.alpha[lane] = L.pdone[lane] ? 0.0 : 1.0;  // alpha doubles as "still running"
    if (!any_lane_d<T>(L, L.alpha)) break;
    const double pq = lane_reduce<T, false>(L, spmv_pass<T, VT>(M, p, q, ra, rb, w));
    if (rg == 0) {
      double a = 0.0;
      if (!L.pdone[lane]) {
        if (pq > 0.0 && isfinite(pq)) a = L.rz[lane] / pq;
        else L.pdone[lane] = 1;  // breakdown: keep the current iterate
      }
      L.alpha[lane] = a;
    }
    __syncthreads();
    const VT alpha = (VT)L.alpha[lane];
    double rrp = 0.0, rzn = 0.0;
    if (jac) {
      jacobi_pass<T, VT, true>(M, x, r, p, q, z, alpha, ra, rb, w, rrp, rzn);
    } else {
      rrp = fwd_pass<T, VT, true>(M, x, r, p, q, z, alpha);
    }
    const double rr = lane_reduce<T, false>(L, rrp);
    if (rg == 0 && !L.pdone[lane]) {
      iters[lane] += 1;
      // converged; or stagnated at the rounding floor of VT (no 0.1 % gain
      // in STALL_ITERS iterations); or growing away from the best residual
      if (rr < 0.999 * L.rrmin[lane]) { L.rrmin[lane] = rr; L.stall[lane] = 0; }
      else L.stall[lane] += 1;
      if (rr <= tol2 * L.bb[lane] || !isfinite(rr) || L.stall[lane] >= STALL_ITERS ||
          rr > 1e4 * L.rrmin[lane])
        L.pdone[lane] = 1;
    }
    __syncthreads();
    if (rg == 0) L.beta[lane] = L.pdone[lane] ? 0.0 : 1.0;
    if (!any_lane_d<T>(L, L.beta)) break;
    if (!jac) rzn = bwd_pass<T, VT>(M, r, z);
    const double rz = lane_reduce<T, false>(L, rzn);
    if (rg == 0) {
      L.beta[lane] = L.pdone[lane] ? 0.0 : rz / L.rz[lane];
      if (!L.pdone[lane]) L.rz[lane] = rz;
      if (!(rz > 0.0)) L.pdone[lane] = 1;
    }
    __syncthreads();
    pupdate_pass<T, VT>(M, z, p, (VT)L.beta[lane], lo, cnt, false);
  }
}

// ------------------------------------------------------------ mismatch
// dP_i, dQ_i of eqs. (1)-(3) from the rectangular voltages e + jf:
// I = Y V, P + jQ = V conj(I).  The outaged branch is left out of the
// neighbour sum and of the diagonal.  WITH_P: the P half-step (writes
// dP/V into the B' right-hand side and tracks max|dP| and max|dQ| for the
// convergence test); otherwise writes dQ/V into the B'' right-hand side.
template <int T, typename VT, bool WITH_P>
__device__ void mismatch_pass(const FdpfParams& P, const DevMatT<VT>& MP, const DevMatT<VT>& MQ,
                              LaneState<T>& L, const double* E, const double* F,
                              const double* V, VT* rhs, double& errP, double& errQ) {
  constexpr int R = NTHREADS / T;
  const int lane = threadIdx.x % T, rg = threadIdx.x / T;
  const DevGrid& G = P.G;
  const int l = L.l[lane], fb = L.fb[lane], tb = L.tb[lane];
  const int lo = L.lo[lane], cnt = L.cnt[lane];
  const bool act = L.active[lane];
  const double coef = L.coef[lane], gl = L.gl[lane], bl = L.bl[lane] + 0.5 * L.bshl[lane];
  const int nrows = WITH_P ? G.n : MQ.n;
  for (int k = rg; k < nrows; k += R) {
    const int i = WITH_P ? k : MQ.bus_of_row[k];
    const int bt = G.bus_type[i];
    if (WITH_P && bt == 2) continue;
    const bool isl = in_island(G.pre[i], lo, cnt);
    VT out = 0;
    if (act && !isl) {
      const size_t o = (size_t)i * T + lane;
      const double ei = E[o], fi = F[o];
      double Gd = G.Gii[i], Bd = G.Bii[i];
      if (i == fb || i == tb) { Gd -= gl; Bd -= bl; }
      double re = Gd * ei - Bd * fi, im = Gd * fi + Bd * ei;
      for (int a = G.adj_ptr[i]; a < G.adj_ptr[i + 1]; ++a) {
        const int e = G.adj_br[a];
        if (e == l) continue;
        const int j = G.adj_idx[a];
        const double ej = E[(size_t)j * T + lane], fj = F[(size_t)j * T + lane];
        const double g = G.g[e], b = G.by[e];
        re -= g * ej - b * fj;
        im -= g * fj + b * ej;
      }
      const double Vi = V[o];
      const double dQ = G.Q_sched[i] - (fi * re - ei * im);
      if (WITH_P) {
        double Ps = G.P_sched[i];
        if (bt == 1) Ps += coef * G.P_gen[i];
        const double dP = Ps - (ei * re + fi * im);
        upd_max(errP, dP);
        if (bt == 0) upd_max(errQ, dQ);
        out = (VT)(dP / Vi);
      } else {
        out = (VT)(dQ / Vi);
      }
    }
    if (WITH_P) rhs[(size_t)MP.row_of_bus[i] * T + lane] = out;
    else rhs[(size_t)k * T + lane] = out;
  }
}

// theta += dtheta (P half-step) or |V| += dV (Q half-step) on the matrix's
// rows, then refresh the rectangular voltages.
template <int T, typename VT, bool IS_P>
__device__ void update_pass(const DevMatT<VT>& M, LaneState<T>& L, const VT* x, double* th,
                            double* V, double* C, double* Sn, double* E, double* F) {
  constexpr int R = NTHREADS / T;
  const int lane = threadIdx.x % T, rg = threadIdx.x / T;
  const int lo = L.lo[lane], cnt = L.cnt[lane];
  if (!L.active[lane]) return;
  for (int k = rg; k < M.n; k += R) {
    if (in_island(M.pre_of_row[k], lo, cnt)) continue;
    const int i = M.bus_of_row[k];
    const size_t o = (size_t)i * T + lane;
    const double dx = (double)x[(size_t)k * T + lane];
    if (IS_P) {
      const double t = th[o] + dx;
      double sn, cs;
      sincos(t, &sn, &cs);
      const double v = V[o];
      th[o] = t;
      C[o] = cs;
      Sn[o] = sn;
      E[o] = v * cs;
      F[o] = v * sn;
    } else {
      const double v = V[o] + dx;
      V[o] = v;
      E[o] = v * C[o];
      F[o] = v * Sn[o];
    }
  }
}

// ------------------------------------------------------------ the kernel
template <int T, typename VT>
__global__ void __launch_bounds__(NTHREADS) fdpf_tiles_kernel(FdpfParams P, DevMatT<VT> MP,
                                                              DevMatT<VT> MQ) {
  constexpr int R = NTHREADS / T;
  __shared__ LaneState<T> L;
  const int tid = threadIdx.x, lane = tid % T, rg = tid / T;
  const DevGrid& G = P.G;
  VT* x = (VT*)P.wx + (size_t)blockIdx.x * P.vstride;
  VT* r = (VT*)P.wr + (size_t)blockIdx.x * P.vstride;
  VT* p = (VT*)P.wp + (size_t)blockIdx.x * P.vstride;
  VT* q = (VT*)P.wq + (size_t)blockIdx.x * P.vstride;
  VT* z = (VT*)P.wz + (size_t)blockIdx.x * P.vstride;
  const size_t so = (size_t)blockIdx.x * P.sstride;
  double *th = P.wth + so, *V = P.wV + so, *C = P.wc + so, *Sn = P.ws + so, *E = P.we + so,
         *F = P.wf + so;

  for (;;) {
    if (tid == 0) L.tile = atomicAdd(P.tile_counter, 1);
    __syncthreads();
    const int tile = L.tile;
    if (tile >= P.n_tiles) break;
    if (rg == 0) {
      const int s = tile * T + lane;
      const bool valid = s < P.S;
      const int l = valid ? P.sc.outage[s] : -1;
      L.scen[lane] = valid ? s : -1;
      L.l[lane] = l;
      L.fb[lane] = l >= 0 ? G.f[l] : -1;
      L.tb[lane] = l >= 0 ? G.t[l] : -1;
      L.lo[lane] = valid ? P.sc.isl_lo[s] : 0;
      L.cnt[lane] = valid ? P.sc.isl_cnt[s] : 0;
      L.coef[lane] = valid ? P.sc.coef[s] : 0.0;
      L.nogen[lane] = valid ? P.sc.no_gen[s] : 0;
      L.raP[lane] = l >= 0 ? MP.row_of_bus[G.f[l]] : -1;
      L.rbP[lane] = l >= 0 ? MP.row_of_bus[G.t[l]] : -1;
      L.raQ[lane] = l >= 0 ? MQ.row_of_bus[G.f[l]] : -1;
      L.rbQ[lane] = l >= 0 ? MQ.row_of_bus[G.t[l]] : -1;
      L.wP[lane] = l >= 0 ? MP.w[l] : 0.0;
      L.wQ[lane] = l >= 0 ? MQ.w[l] : 0.0;
      L.gl[lane] = l >= 0 ? G.g[l] : 0.0;
      L.bl[lane] = l >= 0 ? G.by[l] : 0.0;
      L.bshl[lane] = l >= 0 ? G.b_sh[l] : 0.0;
      L.active[lane] = valid;
      L.outer[lane] = 0;
      L.inP[lane] = 0;
      L.inQ[lane] = 0;
      L.status[lane] = 0;
      L.err[lane] = 0.0;
    }
    __syncthreads();
    // warm start from the base case (Sec. III.B); islanded buses at zero
    {
      const int lo = L.lo[lane], cnt = L.cnt[lane];
      for (int i = rg; i < G.n; i += R) {
        const size_t o = (size_t)i * T + lane;
        double t0, v0;
        if (P.flat_start) { t0 = 0.0; v0 = G.V_set[i]; }
        else { t0 = P.th0[i]; v0 = P.V0[i]; }
        if (in_island(G.pre[i], lo, cnt)) { t0 = 0.0; v0 = 0.0; }
        double sn, cs;
        sincos(t0, &sn, &cs);
        th[o] = t0; V[o] = v0; C[o] = cs; Sn[o] = sn; E[o] = v0 * cs; F[o] = v0 * sn;
      }
    }
    __syncthreads();
    for (;;) {
      // P half-step: mismatch + convergence test
      double eP = 0.0, eQ = 0.0;
      mismatch_pass<T, VT, true>(P, MP, MQ, L, E, F, V, r, eP, eQ);
      eP = lane_reduce<T, true>(L, eP);
      eQ = lane_reduce<T, true>(L, eQ);
      if (rg == 0 && L.active[lane]) {
        const double e2 = (eP != eP || eQ != eQ) ? INFINITY : fmax(eP, eQ);
        L.err[lane] = e2;
        if (!(e2 <= DIVERGE_LIMIT)) { L.status[lane] = 2; L.active[lane] = 0; }
        else if (e2 <= P.tol) { L.status[lane] = 0; L.active[lane] = 0; }
        else if (L.outer[lane] >= P.max_outer) { L.status[lane] = 1; L.active[lane] = 0; }
      }
      if (!any_lane<T>(L, L.active)) break;
      pcg_solve<T, VT>(P, MP, L, x, r, p, q, z, L.raP, L.rbP, L.wP, L.inP);
      update_pass<T, VT, true>(MP, L, x, th, V, C, Sn, E, F);
      __syncthreads();
      // Q half-step
      double d0 = 0.0, d1 = 0.0;
      mismatch_pass<T, VT, false>(P, MP, MQ, L, E, F, V, r, d0, d1);
      __syncthreads();
      pcg_solve<T, VT>(P, MQ, L, x, r, p, q, z, L.raQ, L.rbQ, L.wQ, L.inQ);
      update_pass<T, VT, false>(MQ, L, x, th, V, C, Sn, E, F);
      if (rg == 0 && L.active[lane]) L.outer[lane] += 1;
      __syncthreads();
    }
    // outputs: state, branch flows, loading (Sec. I: overload screening)
    const int s = L.scen[lane];
    if (s >= 0) {
      if (P.out_theta || P.out_vm) {
        for (int i = rg; i < G.n; i += R) {
          const size_t o = (size_t)i * T + lane;
          if (P.out_theta) P.out_theta[(size_t)s * G.n + i] = th[o];
          if (P.out_vm) P.out_vm[(size_t)s * G.n + i] = V[o];
        }
      }
    }
    double mload = 0.0;
    {
      const int l = L.l[lane], lo = L.lo[lane], cnt = L.cnt[lane];
      for (int k = rg; k < G.m; k += R) {
        const int a = G.f[k], b = G.t[k];
        double Pab = 0.0, Pba = 0.0;
        const bool off = (k == l) || in_island(G.pre[a], lo, cnt) || in_island(G.pre[b], lo, cnt);
        if (!off) {
          const double ea = E[(size_t)a * T + lane], fa = F[(size_t)a * T + lane];
          const double eb = E[(size_t)b * T + lane], fbv = F[(size_t)b * T + lane];
          const double g = G.g[k], by = G.by[k];
          const double cr = ea * eb + fa * fbv, sr = fa * eb - ea * fbv;
          Pab = g * (ea * ea + fa * fa) - g * cr - by * sr;
          Pba = g * (eb * eb + fbv * fbv) - g * cr + by * sr;
        }
        upd_max(mload, fmax(fabs(Pab), fabs(Pba)) / G.rating[k]);
        if (s >= 0 && P.out_flow) P.out_flow[(size_t)s * G.m + k] = Pab;
      }
    }
    mload = lane_reduce<T, true>(L, mload);
    if (rg == 0 && s >= 0) {
      int st = L.status[lane];
      if (st == 0 && L.nogen[lane]) st = 3;
      if (P.out_status) P.out_status[s] = st;
      if (P.out_iters) {
        P.out_iters[(size_t)s * 3 + 0] = L.outer[lane];
        P.out_iters[(size_t)s * 3 + 1] = L.inP[lane];
        P.out_iters[(size_t)s * 3 + 2] = L.inQ[lane];
      }
      if (P.out_maxload) P.out_maxload[s] = mload;
    }
    __syncthreads();
  }
}

// Batched operator application for verification (gpcg_apply): X and Y are
// [S][rows]; each CTA handles tiles of T scenarios.
template <int T, typename VT>
__global__ void __launch_bounds__(NTHREADS) apply_kernel(DevMatT<VT> M, int op, int S,
                                                         const int32_t* outages,
                                                         const int32_t* f_, const int32_t* t_,
                                                         const double* X, double* Y, VT* wbuf,
                                                         size_t vstride, int precond) {
  constexpr int R = NTHREADS / T;
  __shared__ LaneState<T> L;
  const int tid = threadIdx.x, lane = tid % T, rg = tid / T;
  VT* a = wbuf + (size_t)blockIdx.x * 4 * vstride;
  VT* b = a + vstride;
  VT* c = b + vstride;
  VT* d = c + vstride;
  const int ntiles = (S + T - 1) / T;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int s = tile * T + lane;
    const bool valid = s < S;
    const int l = valid ? outages[s] : -1;
    const int ra = l >= 0 ? M.row_of_bus[f_[l]] : -1;
    const int rb = l >= 0 ? M.row_of_bus[t_[l]] : -1;
    const VT w = l >= 0 ? (VT)M.w[l] : (VT)0;
    for (int i = rg; i < M.n; i += R) a[(size_t)i * T + lane] = valid ? (VT)X[(size_t)s * M.n + i] : (VT)0;
    __syncthreads();
    if (op == 0) {
      spmv_pass<T, VT>(M, a, b, ra, rb, w);
    } else if (precond == PREC_JACOBI) {
      double rr = 0.0, rz = 0.0;
      jacobi_pass<T, VT, false>(M, c, a, nullptr, nullptr, b, (VT)0, ra, rb, w, rr, rz);
    } else {
      fwd_pass<T, VT, false>(M, c, a, nullptr, nullptr, b, (VT)0);
      bwd_pass<T, VT>(M, a, b);
    }
    __syncthreads();
    for (int i = rg; i < M.n; i += R)
      if (valid) Y[(size_t)s * M.n + i] = (double)b[(size_t)i * T + lane];
    __syncthreads();
  }
  (void)d;
  (void)L;
}

// ----------------------------------------------------------- launchers
template <int T, typename VT>
cudaError_t launch_fdpf_t(cudaStream_t st, int grid, const FdpfParams& P, const DevMatT<VT>& MP,
                          const DevMatT<VT>& MQ) {
  fdpf_tiles_kernel<T, VT><<<grid, NTHREADS, 0, st>>>(P, MP, MQ);
  return cudaGetLastError();
}

template <typename VT>
cudaError_t launch_fdpf(cudaStream_t st, int T, int grid, const FdpfParams& P,
                        const DevMatT<VT>& MP, const DevMatT<VT>& MQ) {
  switch (T) {
    case 1: return launch_fdpf_t<1, VT>(st, grid, P, MP, MQ);
    case 8: return launch_fdpf_t<8, VT>(st, grid, P, MP, MQ);
    case 16: return launch_fdpf_t<16, VT>(st, grid, P, MP, MQ);
    case 32: return launch_fdpf_t<32, VT>(st, grid, P, MP, MQ);
    default: return cudaErrorInvalidValue;
  }
}

template <typename VT>
int fdpf_max_blocks_per_sm(int T) {
  int nb = 0;
  cudaError_t ce = cudaErrorInvalidValue;
  switch (T) {
    case 1: ce = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fdpf_tiles_kernel<1, VT>, NTHREADS, 0); break;
    case 8: ce = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fdpf_tiles_kernel<8, VT>, NTHREADS, 0); break;
    case 16: ce = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fdpf_tiles_kernel<16, VT>, NTHREADS, 0); break;
    case 32: ce = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fdpf_tiles_kernel<32, VT>, NTHREADS, 0); break;
  }
  return ce == cudaSuccess ? nb : 0;
}

template <typename VT>
cudaError_t launch_apply(cudaStream_t st, int grid, const DevMatT<VT>& M, int op, int S,
                         const int32_t* outages, const int32_t* f, const int32_t* t,
                         const double* X, double* Y, VT* wbuf, size_t vstride, int precond) {
  apply_kernel<32, VT><<<grid, NTHREADS, 0, st>>>(M, op, S, outages, f, t, X, Y, wbuf, vstride,
                                                  precond);
  return cudaGetLastError();
}

template cudaError_t launch_fdpf<float>(cudaStream_t, int, int, const FdpfParams&,
                                        const DevMatT<float>&, const DevMatT<float>&);
template cudaError_t launch_fdpf<double>(cudaStream_t, int, int, const FdpfParams&,
                                         const DevMatT<double>&, const DevMatT<double>&);
template int fdpf_max_blocks_per_sm<float>(int);
template int fdpf_max_blocks_per_sm<double>(int);
template cudaError_t launch_apply<float>(cudaStream_t, int, const DevMatT<float>&, int, int,
                                         const int32_t*, const int32_t*, const int32_t*,
                                         const double*, double*, float*, size_t, int);
template cudaError_t launch_apply<double>(cudaStream_t, int, const DevMatT<double>&, int, int,
                                          const int32_t*, const int32_t*, const int32_t*,
                                          const double*, double*, double*, size_t, int);

}  // namespace gpcg
