// The plain FP64 path: one N-1 scenario at a time, with the whole GPU working
// on it -- the vertex-parallel reading of the GPCG algorithm (Sec. III.B).
// Every pass over buses, branches or matrix rows is spread over all threads
// of a cooperative launch, and the steps that depend on one another (each
// level of the triangular substitutions, each dot product, the convergence
// test) are separated by grid-wide barriers: the supersteps of the paper's
// bulk-synchronous vertex programs.  No launch holds more than one scenario,
// so this is the unbatched comparison for the batched screen; everything is
// FP64.  The arithmetic is the batched kernel's (fdpf_kernel.cuh): the FP64
// mismatch of eqs. (1)-(3) with the outaged branch left out, base-case
// preconditioned CG on B'_s and B''_s (Sec. IV.B, eq. (6)) with the
// outage's four-element change applied in the SpMV, the exact rotation of
// the rectangular voltages, and the same stopping and divergence rules.
//
// Sums over the grid are deterministic: each CTA's partial goes to its slot
// of a global array and, after a barrier, every CTA adds the slots in the
// same order.  A barrier whose wait runs past its iteration limit sets an
// error flag, and the kernel returns at the next barrier (GPCG_ERR_TIMEOUT).
#include "fdpf_kernel.cuh"

namespace gpcg {

namespace {

constexpr int PT = 256;               // threads per CTA
constexpr int PW = PT / 32;           // warps per CTA

struct PlainState {
  double* part;          // [2][4 * grid] per-CTA partials (two alternating sets)
  unsigned int* bar;     // [2] arrival count, generation
  int* err;              // set when a barrier wait gave up
  unsigned limit;        // polls a barrier wait makes before it gives up
  double *x, *r, *p, *q, *z, *t;  // [rows + 1]; t: the tail's right-hand side
  double *th, *V, *ef;   // state by bus: theta, |V|, (e, f) interleaved
};

// Wait for every CTA of the grid (all resident: cooperative launch).
__device__ bool grid_barrier(const PlainState& W) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned int* gen = W.bar + 1;
    const unsigned int g = *gen;
    __threadfence();
    ok = 1;
    if (atomicAdd(W.bar, 1u) == gridDim.x - 1) {
      atomicExch(W.bar, 0u);
      __threadfence();
      atomicAdd(W.bar + 1, 1u);
    } else {
      // poll until the last CTA arrives; give up after W.limit polls, or as
      // soon as another CTA has given up (its flag is set)
      unsigned int spins = 0;
      while (*gen == g) {
        if (++spins > W.limit) {
          atomicExch(W.err, 1);
          break;
        }
        if (*(volatile int*)W.err) break;
        __nanosleep(64);
      }
    }
    __threadfence();
    if (*(volatile int*)W.err) ok = 0;
  }
  __syncthreads();
  return ok != 0;
}

// Grid-wide sums of K values (K <= 4) in a fixed order; `round` alternates
// the partial sets so a slow reader of one sum never sees the next one's
// partials.  Returns false when a barrier gave up.
template <int K>
__device__ bool grid_sums(const PlainState& W, int& round, double (&v)[K]) {
  __shared__ double ws[PW][4];
  __shared__ double tot[4];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    double a = v[k];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) a += __shfl_xor_sync(0xffffffffu, a, off);
    if (lane == 0) ws[w][k] = a;
  }
  __syncthreads();
  double* part = W.part + (size_t)(round & 1) * 4 * gridDim.x;
  round += 1;
  if (threadIdx.x == 0)
#pragma unroll
    for (int k = 0; k < K; ++k) {
      double a = 0.0;
      for (int j = 0; j < PW; ++j) a += ws[j][k];
      part[(size_t)blockIdx.x * 4 + k] = a;
    }
  if (!grid_barrier(W)) return false;
  if (threadIdx.x == 0)
#pragma unroll
    for (int k = 0; k < K; ++k) {
      double a = 0.0;
      for (unsigned b = 0; b < gridDim.x; ++b) a += part[(size_t)b * 4 + k];
      tot[k] = a;
    }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < K; ++k) v[k] = tot[k];
  __syncthreads();
  return true;
}

// Grid-wide maxima of K non-negative values held as abs_bits patterns (NaN
// sorts above infinity), through the same partial sets.
template <int K>
__device__ bool grid_maxes(const PlainState& W, int& round, unsigned long long (&v)[K]) {
  __shared__ unsigned long long ws[PW][4];
  __shared__ unsigned long long tot[4];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    unsigned long long a = v[k];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      const unsigned long long b = __shfl_xor_sync(0xffffffffu, a, off);
      a = b > a ? b : a;
    }
    if (lane == 0) ws[w][k] = a;
  }
  __syncthreads();
  unsigned long long* part =
      reinterpret_cast<unsigned long long*>(W.part + (size_t)(round & 1) * 4 * gridDim.x);
  round += 1;
  if (threadIdx.x == 0)
#pragma unroll
    for (int k = 0; k < K; ++k) {
      unsigned long long a = 0ull;
      for (int j = 0; j < PW; ++j) a = ws[j][k] > a ? ws[j][k] : a;
      part[(size_t)blockIdx.x * 4 + k] = a;
    }
  if (!grid_barrier(W)) return false;
  if (threadIdx.x == 0)
#pragma unroll
    for (int k = 0; k < K; ++k) {
      unsigned long long a = 0ull;
      for (unsigned b = 0; b < gridDim.x; ++b) {
        const unsigned long long u = part[(size_t)b * 4 + k];
        a = u > a ? u : a;
      }
      tot[k] = a;
    }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < K; ++k) v[k] = tot[k];
  __syncthreads();
  return true;
}

// The scenario: outaged branch l with ends fb, tb, its series admittance and
// charging (gl, bl) and from-end factor cl, the islanded preorder interval
// [lo, lo + cnt), and the re-dispatch coefficient.
struct Scen {
  int l, fb, tb, lo, cnt, nogen;
  double gl, bl, cl, coef;
};

// I_i = sum_j Y_ij V_j at bus i with the outaged branch left out (as the
// batched kernel's mismatch_pass sums it).
__device__ double2 current_at(const DevGrid& G, const Scen& c, const double2* __restrict__ EF,
                              int i) {
  double re = 0.0, im = 0.0;
  const int deg = __ldg(G.adj_deg + i);
  for (int a = 0; a < deg; ++a) {
    if (__ldg(G.adj_brl + (size_t)a * G.n + i) == c.l) continue;
    const int j = __ldg(G.adj_nbr + (size_t)a * G.n + i);
    const double gv = __ldg(G.adj_g + (size_t)a * G.n + i), bv = __ldg(G.adj_b + (size_t)a * G.n + i);
    const double2 u = EF[j];
    re = fma(-gv, u.x, fma(bv, u.y, re));
    im = fma(-gv, u.y, fma(-bv, u.x, im));
  }
  const int o1 = __ldg(G.adj_optr + i + 1);
  for (int e = __ldg(G.adj_optr + i); e < o1; ++e) {
    if (__ldg(G.adj_obr + e) == c.l) continue;
    const int j = __ldg(G.adj_onbr + e);
    const double gw = __ldg(G.adj_og + e), bw = __ldg(G.adj_ob + e);
    const double2 u = EF[j];
    re = fma(-gw, u.x, fma(bw, u.y, re));
    im = fma(-gw, u.y, fma(-bw, u.x, im));
  }
  const double2 v = EF[i];
  double Gd = __ldg(G.Gii + i), Bd = __ldg(G.Bii + i);
  if (i == c.fb || i == c.tb) {  // the outaged branch's share of the diagonal
    const double c2 = i == c.fb ? c.cl * c.cl : 1.0;
    Gd -= c2 * c.gl;
    Bd -= c2 * c.bl;
  }
  return make_double2(fma(Gd, v.x, fma(-Bd, v.y, re)), fma(Gd, v.y, fma(Bd, v.x, im)));
}

// Base-case preconditioned CG (Sec. III.A listing read as textbook PCG) on
// B_s x = b, b in W.r on entry, x in W.x on exit; the outage's change is the
// rank-one term w v v^T, v = c e_ra - e_rb (an end without a row: -1).
// Returns false when a barrier gave up.
__device__ bool plain_pcg(const FdpfParams& P, const DevMatT<double>& M, const Scen& c,
                          const PlainState& W, int& round, int ra, int rb, double w, double cf,
                          int& iters) {
  const int n = M.n;
  const int gt = blockIdx.x * PT + threadIdx.x, NT = gridDim.x * PT;
  const bool jac = P.precond == PREC_JACOBI;
  // row k is islanded: its search directions are kept at zero
  auto islanded = [&](int k) { return in_island(__ldg(M.pre_of_row + k), c.lo, c.cnt); };
  // z = M^-1 r: forward substitution over the level schedule, the tail by
  // its dense inverse, then the backward substitution
  auto precond = [&]() -> bool {
    if (jac) {
      for (int k = gt; k < n; k += NT) {
        const double d = __ldg(M.diag + k) - (k == ra ? w * cf * cf : k == rb ? w : 0.0);
        W.z[k] = d > 0.0 ? W.r[k] / d : 0.0;
      }
      return grid_barrier(W);
    }
    for (int lev = 0; lev < M.tail_lev; ++lev) {
      const int r0 = __ldg(M.lev_ptr + lev), r1 = __ldg(M.lev_ptr + lev + 1);
      for (int i = r0 + gt; i < r1; i += NT) {
        double a = W.r[i];
        for (int k = 0; k < KL; ++k)
          a -= __ldg(M.L.val + (size_t)i * KL + k) * W.z[__ldg(M.L.col + (size_t)i * KL + k)];
        for (int e = __ldg(M.L.optr + i); e < __ldg(M.L.optr + i + 1); ++e)
          a -= __ldg(M.L.oval + e) * W.z[__ldg(M.L.ocol + e)];
        W.z[i] = a * __ldg(M.inv_diag + i);
      }
      if (!grid_barrier(W)) return false;
    }
    const int t0 = M.tail_row0, nt = n - t0;
    if (nt > 0) {
      // right-hand side of the tail: its rows minus their parts on solved rows
      for (int k = gt; k < nt; k += NT) {
        const int i = t0 + k;
        double a = W.r[i];
        for (int s = 0; s < KL; ++s) {
          const int col = __ldg(M.L.col + (size_t)i * KL + s);
          if (col < t0) a -= __ldg(M.L.val + (size_t)i * KL + s) * W.z[col];
        }
        for (int e = __ldg(M.L.optr + i); e < __ldg(M.L.optr + i + 1); ++e) {
          const int col = __ldg(M.L.ocol + e);
          if (col < t0) a -= __ldg(M.L.oval + e) * W.z[col];
        }
        W.t[k] = a;
      }
      if (!grid_barrier(W)) return false;
      // y_t = X rhs (X_kj = xc[j nt + k]), held in z
      for (int k = gt; k < nt; k += NT) {
        double a = 0.0;
        for (int j = 0; j <= k; ++j) a += __ldg(M.xc + (size_t)j * nt + k) * W.t[j];
        W.z[t0 + k] = a;
      }
      if (!grid_barrier(W)) return false;
      // z_t = X^T y_t (X_ik = xr[i nt + k]), from the copy in t
      for (int k = gt; k < nt; k += NT) W.t[k] = W.z[t0 + k];
      if (!grid_barrier(W)) return false;
      for (int k = gt; k < nt; k += NT) {
        double a = 0.0;
        for (int i = k; i < nt; ++i) a += __ldg(M.xr + (size_t)i * nt + k) * W.t[i];
        W.z[t0 + k] = a;
      }
      if (!grid_barrier(W)) return false;
    }
    // back substitution of the rows before the tail
    for (int lev = 0; lev < M.ntblev; ++lev) {
      const int r0 = __ldg(M.tblev_ptr + lev), r1 = __ldg(M.tblev_ptr + lev + 1);
      for (int kk = r0 + gt; kk < r1; kk += NT) {
        const int i = __ldg(M.tblev_rows + kk);
        double a = W.z[i];
        for (int k = 0; k < KU; ++k)
          a -= __ldg(M.U.val + (size_t)i * KU + k) * W.z[__ldg(M.U.col + (size_t)i * KU + k)];
        for (int e = __ldg(M.U.optr + i); e < __ldg(M.U.optr + i + 1); ++e)
          a -= __ldg(M.U.oval + e) * W.z[__ldg(M.U.ocol + e)];
        W.z[i] = a * __ldg(M.inv_diag + i);
      }
      if (!grid_barrier(W)) return false;
    }
    return true;
  };
  // x = 0; ||b||^2
  double bb[1] = {0.0};
  for (int k = gt; k < n; k += NT) {
    W.x[k] = 0.0;
    bb[0] += W.r[k] * W.r[k];
  }
  if (gt == 0) { W.z[n] = 0.0; W.p[n] = 0.0; }
  if (!grid_sums<1>(W, round, bb)) return false;
  if (!(bb[0] > 0.0)) return true;
  if (!precond()) return false;
  double rz[1] = {0.0};
  for (int k = gt; k < n; k += NT) rz[0] += W.r[k] * W.z[k];
  if (!grid_sums<1>(W, round, rz)) return false;
  if (!(rz[0] > 0.0)) return true;
  const double tol2 = P.inner_rtol * P.inner_rtol;
  double rrmin = bb[0];
  int stall = 0;
  for (int it = 0; it < P.max_inner; ++it) {
    // p = mask(z) + beta p (beta = 0 first), then q = B_s p and p.q
    if (it == 0)
      for (int k = gt; k < n; k += NT) W.p[k] = islanded(k) ? 0.0 : W.z[k];
    if (!grid_barrier(W)) return false;
    double pq[1] = {0.0};
    for (int k = gt; k < n; k += NT) {
      double a = 0.0;
      for (int s = 0; s < KA; ++s)
        a += __ldg(M.A.val + (size_t)k * KA + s) * W.p[__ldg(M.A.col + (size_t)k * KA + s)];
      for (int e = __ldg(M.A.optr + k); e < __ldg(M.A.optr + k + 1); ++e)
        a += __ldg(M.A.oval + e) * W.p[__ldg(M.A.ocol + e)];
      if (k == ra || k == rb) {  // -w v (v.p), v = c e_ra - e_rb
        const double xa = ra >= 0 ? W.p[ra] : 0.0, xb = rb >= 0 ? W.p[rb] : 0.0;
        const double wt = w * (cf * xa - xb);
        a += k == ra ? -(cf * wt) : wt;
      }
      if (islanded(k)) a = 0.0;
      W.q[k] = a;
      pq[0] += W.p[k] * a;
    }
    if (!grid_sums<1>(W, round, pq)) return false;
    if (!(pq[0] > 0.0) || !isfinite(pq[0])) break;  // breakdown: keep the iterate
    const double alpha = rz[0] / pq[0];
    double rr[1] = {0.0};
    for (int k = gt; k < n; k += NT) {
      W.x[k] = fma(alpha, W.p[k], W.x[k]);
      const double rv = W.r[k] - alpha * W.q[k];
      W.r[k] = rv;
      rr[0] += rv * rv;
    }
    if (!grid_sums<1>(W, round, rr)) return false;
    iters += 1;
    // converged; stagnated (no 0.1 % gain in STALL_ITERS iterations); or
    // growing away from the best residual
    if (rr[0] < 0.999 * rrmin) { rrmin = rr[0]; stall = 0; }
    else stall += 1;
    if (rr[0] <= tol2 * bb[0] || !isfinite(rr[0]) || stall >= STALL_ITERS ||
        rr[0] > 1e4 * rrmin)
      break;
    if (!precond()) return false;
    double rzn[1] = {0.0};
    for (int k = gt; k < n; k += NT) rzn[0] += W.r[k] * W.z[k];
    if (!grid_sums<1>(W, round, rzn)) return false;
    if (!(rzn[0] > 0.0)) break;
    const double beta = rzn[0] / rz[0];
    rz[0] = rzn[0];
    for (int k = gt; k < n; k += NT) W.p[k] = (islanded(k) ? 0.0 : W.z[k]) + beta * W.p[k];
  }
  return grid_barrier(W);
}

}  // namespace

// One scenario (index s of the call) through the whole fast-decoupled power
// flow, retired into the call's outputs.
__global__ void __launch_bounds__(PT) plain_fdpf_kernel(FdpfParams P, DevMatT<double> MP,
                                                         DevMatT<double> MQ, PlainState W,
                                                         int s) {
  const DevGrid& G = P.G;
  const int gt = blockIdx.x * PT + threadIdx.x, NT = gridDim.x * PT;
  const int n = G.n;
  double2* EF = reinterpret_cast<double2*>(W.ef);
  Scen c;
  c.l = P.sc.outage[s];
  c.fb = c.l >= 0 ? G.f[c.l] : -1;
  c.tb = c.l >= 0 ? G.t[c.l] : -1;
  c.lo = P.sc.isl_lo[s];
  c.cnt = P.sc.isl_cnt[s];
  c.nogen = P.sc.no_gen[s];
  c.coef = P.sc.coef[s];
  c.gl = c.l >= 0 ? G.g[c.l] : 0.0;
  c.bl = c.l >= 0 ? G.by[c.l] + 0.5 * G.b_sh[c.l] : 0.0;
  c.cl = c.l >= 0 ? G.cf[c.l] : 1.0;
  const int raP = c.l >= 0 ? MP.row_of_bus[c.fb] : -1, rbP = c.l >= 0 ? MP.row_of_bus[c.tb] : -1;
  const int raQ = c.l >= 0 ? MQ.row_of_bus[c.fb] : -1, rbQ = c.l >= 0 ? MQ.row_of_bus[c.tb] : -1;
  const double wP = c.l >= 0 ? MP.w[c.l] : 0.0, wQ = c.l >= 0 ? MQ.w[c.l] : 0.0;
  const double cQ = (c.l >= 0 && MQ.c) ? MQ.c[c.l] : 1.0;
  int round = 0;
  // warm start from the base case (Sec. III.B), islanded buses at zero
  for (int i = gt; i < n; i += NT) {
    const bool isl = in_island(G.pre[i], c.lo, c.cnt);
    const double v0 = P.V0[i];
    W.th[i] = isl ? 0.0 : P.th0[i];
    W.V[i] = isl ? 0.0 : v0;
    EF[i] = isl ? make_double2(0.0, 0.0) : make_double2(v0 * P.c0[i], v0 * P.s0[i]);
  }
  if (!grid_barrier(W)) return;
  int outer = 0, inP = 0, inQ = 0, status = -1;
  double best = INFINITY;
  for (;;) {
    // P half-step: mismatch (eqs. (1)-(3)) and the convergence test
    unsigned long long mx[2] = {0ull, 0ull};
    for (int k = gt; k < MP.n; k += NT) {
      const int i = MP.bus_of_row[k];
      double rhs = 0.0;
      if (!in_island(G.pre[i], c.lo, c.cnt)) {
        const double2 I = current_at(G, c, EF, i);
        const double2 v = EF[i];
        const int bt = G.bus_type[i];
        const double pg = bt == 1 ? fmax(G.P_gen[i], 0.0) : 0.0;
        const double dP = fma(-v.x, I.x, fma(-v.y, I.y, fma(c.coef, pg, G.P_sched[i])));
        upd_max_bits(mx[0], dP);
        if (bt == 0) upd_max_bits(mx[1], fma(-v.y, I.x, fma(v.x, I.y, G.Q_sched[i])));
        rhs = dP / W.V[i];
      }
      W.r[k] = rhs;
    }
    if (!grid_maxes<2>(W, round, mx)) return;
    const double a = from_bits(mx[0]), b = from_bits(mx[1]);
    const double err = (a != a || b != b) ? INFINITY : fmax(a, b);
    if (!(err <= DIVERGE_LIMIT) || err > DIVERGE_GROWTH * best) status = 2;
    else if (err <= P.tol) status = 0;
    else if (outer >= P.max_outer) status = 1;
    best = fmin(best, err);
    if (status >= 0) break;
    // P half-step, unless the P mismatch is already within the tolerance
    if (!(a <= P.tol)) {
      if (!plain_pcg(P, MP, c, W, round, raP, rbP, wP, 1.0, inP)) return;
      // theta += dtheta, (e, f) rotated with it
      for (int k = gt; k < MP.n; k += NT) {
        const int i = MP.bus_of_row[k];
        if (in_island(G.pre[i], c.lo, c.cnt)) continue;
        const double d = W.x[k];
        W.th[i] += d;
        double2 u = EF[i];
        rotate_ef(d, u.x, u.y);
        EF[i] = u;
      }
      if (!grid_barrier(W)) return;
    }
    // Q half-step on the PQ buses, unless their mismatch is within the tolerance
    unsigned long long mq[1] = {0ull};
    for (int k = gt; k < MQ.n; k += NT) {
      const int i = MQ.bus_of_row[k];
      double rhs = 0.0;
      if (!in_island(G.pre[i], c.lo, c.cnt)) {
        const double2 I = current_at(G, c, EF, i);
        const double2 v = EF[i];
        const double dQ = fma(-v.y, I.x, fma(v.x, I.y, G.Q_sched[i]));
        upd_max_bits(mq[0], dQ);
        rhs = dQ / W.V[i];
      }
      W.r[k] = rhs;
    }
    if (!grid_maxes<1>(W, round, mq)) return;
    if (!(from_bits(mq[0]) <= P.tol)) {
      if (!plain_pcg(P, MQ, c, W, round, raQ, rbQ, wQ, cQ, inQ)) return;
      for (int k = gt; k < MQ.n; k += NT) {
        const int i = MQ.bus_of_row[k];
        if (in_island(G.pre[i], c.lo, c.cnt)) continue;
        const double r = W.x[k] / W.V[i];
        W.V[i] = fma(W.V[i], r, W.V[i]);
        const double2 u = EF[i];
        EF[i] = make_double2(fma(u.x, r, u.x), fma(u.y, r, u.y));
      }
      if (!grid_barrier(W)) return;
    }
    outer += 1;
  }
  // outputs (Sec. I): state, branch flows, loading and overloads
  const int nw = (G.m + 31) >> 5;
  for (int iu = gt; iu < n; iu += NT) {
    const int i = P.out_bus_map ? P.out_bus_map[iu] : iu;
    if (P.out_theta) P.out_theta[(size_t)s * n + iu] = W.th[i];
    if (P.out_vm) P.out_vm[(size_t)s * n + iu] = W.V[i];
  }
  if (P.out_ovmask) {
    for (int w = gt; w < nw; w += NT) P.out_ovmask[(size_t)s * nw + w] = 0u;
    if (!grid_barrier(W)) return;
  }
  unsigned long long ml[1] = {0ull};
  double nov[1] = {0.0};
  for (int k = gt; k < G.m; k += NT) {
    const int a = G.f[k], b = G.t[k];
    double Pab = 0.0;
    if (k != c.l && !in_island(G.pre[a], c.lo, c.cnt) && !in_island(G.pre[b], c.lo, c.cnt)) {
      const double2 va = EF[a], vb = EF[b];
      const double gk = G.g[k], bk = G.by[k], ck = G.cf[k];
      const double cr = ck * fma(va.x, vb.x, va.y * vb.y), sr = ck * fma(va.y, vb.x, -va.x * vb.y);
      const double gc = gk * cr;
      Pab = fma(gk * ck * ck, fma(va.x, va.x, va.y * va.y), -fma(bk, sr, gc));
      const double Pba = fma(gk, fma(vb.x, vb.x, vb.y * vb.y), fma(bk, sr, -gc));
      const unsigned long long u = abs_bits(Pab), v = abs_bits(Pba);
      const double ld = __longlong_as_double((long long)(u > v ? u : v)) * G.inv_rating[k];
      upd_max_bits(ml[0], ld);
      if (overloaded(ld)) {
        nov[0] += 1.0;
        if (P.out_ovmask) atomicOr(P.out_ovmask + (size_t)s * nw + (k >> 5), 1u << (k & 31));
      }
    }
    if (P.out_flow) P.out_flow[(size_t)s * G.m + k] = Pab;
  }
  if (!grid_maxes<1>(W, round, ml)) return;
  if (!grid_sums<1>(W, round, nov)) return;
  if (gt == 0) {
    int st = status;
    if (st == 0 && c.nogen) st = 3;
    if (P.out_status) P.out_status[s] = st;
    if (P.out_iters) {
      P.out_iters[(size_t)s * 3 + 0] = outer;
      P.out_iters[(size_t)s * 3 + 1] = inP;
      P.out_iters[(size_t)s * 3 + 2] = inQ;
    }
    if (P.out_maxload) P.out_maxload[s] = from_bits(ml[0]);
    if (P.out_nover) P.out_nover[s] = (int)nov[0];
  }
}

// Launch scenario s of the call on `grid` co-resident CTAs.  The work
// buffers (see PlainState) come from the caller.
cudaError_t launch_plain(cudaStream_t st, int grid, const FdpfParams& P,
                         const DevMatT<double>& MP, const DevMatT<double>& MQ,
                         const PlainBuffers& B, int s) {
  PlainState W;
  W.part = B.part; W.bar = B.bar; W.err = B.err;
  W.limit = B.wait_limit;
  W.x = B.x; W.r = B.r; W.p = B.p; W.q = B.q; W.z = B.z; W.t = B.t;
  W.th = B.th; W.V = B.V; W.ef = B.ef;
  FdpfParams Pc = P;
  DevMatT<double> MPc = MP, MQc = MQ;
  void* args[] = {&Pc, &MPc, &MQc, &W, &s};
  return cudaLaunchCooperativeKernel((const void*)plain_fdpf_kernel, dim3(grid), dim3(PT), args,
                                     0, st);
}

int plain_grid(int num_sms) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, plain_fdpf_kernel, PT, 0) !=
      cudaSuccess)
    return 0;
  return per_sm * num_sms;
}

}  // namespace gpcg
