// Batched operators and the batched PCG shared by the persistent kernels
// (fdpf.cu: the N-1 screen; adjoint.cu: the overload-penalty adjoint).
//
// A CTA owns T scenario lanes; vectors are [row][T]; each thread owns two
// adjacent lanes of a row.  Every sparse row is read through a padded
// descriptor (ELL) so a thread issues all of a row's gathers at once.
#pragma once
#include <math.h>
#include "common.cuh"
#include "fdpf.h"

namespace gpcg {


constexpr int LP = 2;  // scenario lanes per thread
#ifndef FDPF_UNROLL
#define FDPF_UNROLL 1
#endif
constexpr int UNR = FDPF_UNROLL;  // rows per thread in flight in the PCG passes
#ifndef FDPF_MIS_GROUP
#define FDPF_MIS_GROUP 1
#endif
constexpr int MIS_GROUP = FDPF_MIS_GROUP;  // neighbours loaded together in the mismatch
// Large passes are kept out of line by default (separate register
// allocation); -DGPCG_PASS_INLINE=__forceinline__ inlines them.
#ifndef GPCG_PASS_INLINE
#define GPCG_PASS_INLINE __noinline__
#endif
// The row loops of the inner solve: inlined into their caller by default;
// -DGPCG_LOOP_INLINE=__noinline__ gives each its own register allocation.
#ifndef GPCG_LOOP_INLINE
#define GPCG_LOOP_INLINE __forceinline__
#endif
#ifndef FDPF_MIN_BLOCKS
#define FDPF_MIN_BLOCKS 5  // resident CTAs per SM the register budget is cut for
#endif

// Inner iterations without progress after which a solve stops: the outer
// FP64 loop then refines the answer (iterative refinement).
constexpr int STALL_ITERS = 50;

// ------------------------------------------------------------ helpers
template <typename VT> struct Pair { VT a, b; };

__device__ __forceinline__ Pair<float> ld2(const float* p) {
  const float2 v = *reinterpret_cast<const float2*>(p);
  return {v.x, v.y};
}
__device__ __forceinline__ Pair<double> ld2(const double* p) {
  const double2 v = *reinterpret_cast<const double2*>(p);
  return {v.x, v.y};
}
__device__ __forceinline__ void st2(float* p, Pair<float> v) {
  *reinterpret_cast<float2*>(p) = make_float2(v.a, v.b);
}
__device__ __forceinline__ void st2(double* p, Pair<double> v) {
  *reinterpret_cast<double2*>(p) = make_double2(v.a, v.b);
}

template <int K>
__device__ __forceinline__ void ld_cols(const int32_t* p, int (&c)[K]) {
  static_assert(K % 2 == 0, "slots come in pairs");
#pragma unroll
  for (int k = 0; k < K; k += 2) {
    const int2 v = __ldg(reinterpret_cast<const int2*>(p + k));
    c[k] = v.x; c[k + 1] = v.y;
  }
}
template <int K>
__device__ __forceinline__ void ld_vals(const float* p, float (&v)[K]) {
#pragma unroll
  for (int k = 0; k < K; k += 2) {
    const float2 u = __ldg(reinterpret_cast<const float2*>(p + k));
    v[k] = u.x; v[k + 1] = u.y;
  }
}
template <int K>
__device__ __forceinline__ void ld_vals(const double* p, double (&v)[K]) {
#pragma unroll
  for (int k = 0; k < K; k += 2) {
    const double2 u = __ldg(reinterpret_cast<const double2*>(p + k));
    v[k] = u.x; v[k + 1] = u.y;
  }
}

template <int K>
__device__ __forceinline__ void ld_halfs(const __half* p, float (&v)[K]) {
#pragma unroll
  for (int k = 0; k < K; k += 2) {
    const __half2 h = __ldg(reinterpret_cast<const __half2*>(p + k));
    const float2 f = __half22float2(h);
    v[k] = f.x; v[k + 1] = f.y;
  }
}
template <int K>
__device__ __forceinline__ void ld_halfs(const __half* p, double (&v)[K]) {
  float f[K];
  ld_halfs<K>(p, f);
#pragma unroll
  for (int k = 0; k < K; ++k) v[k] = f[k];
}

// ------------------------------------------------------------ lane state
constexpr int NRED_SITES = 8;  // reduction sites with a buffer of their own
enum RedSite { RS_BB = 0, RS_RZ0, RS_PQ, RS_RR, RS_RZ, RS_ERRP, RS_ERRQ, RS_LOAD };

template <int T>
struct LaneState {
  int scen[T], l[T], fb[T], tb[T], lo[T], cnt[T];
  int raP[T], rbP[T], raQ[T], rbQ[T];
  double wP[T], wQ[T], coef[T], gl[T], bl[T];
  int active[T], outer[T], inP[T], inQ[T], status[T], nogen[T];
  double err[T], best[T];
  double rz[T], bb[T], alpha[T], beta[T], rrmin[T];
  unsigned long long tphase[8];
  int pdone[T], stall[T];
  int done[T], fresh[T];
  double red[NTHREADS * LP];
  // one small buffer per reduction site (see lane_sum): [site][warp][lane]
  double red2[NRED_SITES * (NTHREADS / 32) * T];
  int flag;
  int drained;
};

template <int T>
struct Geo {
  static constexpr int TPR = T / LP;             // threads per row
  static constexpr int RPS = NTHREADS / TPR;     // rows per step
  int rs, lane;                                  // row slot, first lane
  __device__ Geo() : rs(threadIdx.x / TPR), lane((threadIdx.x % TPR) * LP) {}
};

// Sum (or max) over the row slots of each lane's partial values.
template <int T, bool MAX>
__device__ __forceinline__ Pair<double> lane_reduce(LaneState<T>& L, double v0, double v1) {
  const Geo<T> g;
  constexpr int RPS = Geo<T>::RPS;
  L.red[g.rs * T + g.lane] = v0;
  L.red[g.rs * T + g.lane + 1] = v1;
  __syncthreads();
#pragma unroll
  for (int st = RPS / 2; st > 0; st >>= 1) {
    if (g.rs < st) {
#pragma unroll
      for (int j = 0; j < LP; ++j) {
        const int o = g.rs * T + g.lane + j;
        const double a = L.red[o], b = L.red[o + st * T];
        L.red[o] = MAX ? ((b > a || b != b) ? b : a) : a + b;
      }
    }
    __syncthreads();
  }
  const Pair<double> out{L.red[g.lane], L.red[g.lane + 1]};
  __syncthreads();
  return out;
}

// True when some lane has a nonzero flag (block-uniform).
template <int T, typename F>
__device__ __forceinline__ bool any_lane(LaneState<T>& L, const F* flags) {
  __syncthreads();
  if (threadIdx.x == 0) {
    int any = 0;
    for (int s = 0; s < T; ++s) any |= (flags[s] != 0);
    L.flag = any;
  }
  __syncthreads();
  const bool r = L.flag != 0;
  __syncthreads();
  return r;
}

__device__ __forceinline__ void upd_max(double& m, double d) {
  const double a = fabs(d);
  if (!(a <= m)) m = (a == a) ? a : INFINITY;
}

// |d| as an unsigned 64-bit pattern: for non-negative doubles the integer
// order is the numeric order (a NaN sorts above +inf), so running maxima of
// |d| take integer instructions and leave the FP64 pipe alone.
__device__ __forceinline__ unsigned long long abs_bits(double d) {
  return (unsigned long long)__double_as_longlong(d) & 0x7fffffffffffffffull;
}
__device__ __forceinline__ void upd_max_bits(unsigned long long& m, double d) {
  const unsigned long long a = abs_bits(d);
  m = a > m ? a : m;
}
__device__ __forceinline__ double from_bits(unsigned long long b) {
  const double v = __longlong_as_double((long long)b);
  return v == v ? v : INFINITY;
}

// Per-lane sum of the threads' partial values in a fixed order: a shuffle
// tree inside each warp over the threads that hold the same lanes, then the
// warps' partials through shared memory (buffer SITE) and one barrier.
// Every thread returns the totals of its own two lanes.  A site's buffer is
// read right after the barrier and rewritten only after a later barrier,
// so consecutive reductions at different sites need no barrier between.
template <int T, int SITE, typename X>
__device__ __forceinline__ Pair<X> lane_sum(LaneState<T>& L, X v0, X v1) {
  const Geo<T> g;
  constexpr int TPR = Geo<T>::TPR, NW = NTHREADS / 32;
#pragma unroll
  for (int off = 16; off >= TPR; off >>= 1) {
    v0 += __shfl_xor_sync(0xffffffffu, v0, off);
    v1 += __shfl_xor_sync(0xffffffffu, v1, off);
  }
  X* buf = reinterpret_cast<X*>(L.red2 + SITE * NW * T);
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) < TPR) {
    buf[w * T + g.lane] = v0;
    buf[w * T + g.lane + 1] = v1;
  }
  __syncthreads();
  X s0 = buf[g.lane], s1 = buf[g.lane + 1];
#pragma unroll
  for (int k = 1; k < NW; ++k) {
    s0 += buf[k * T + g.lane];
    s1 += buf[k * T + g.lane + 1];
  }
  return {s0, s1};
}

// The same for running maxima held as abs_bits patterns.
template <int T, int SITE>
__device__ __forceinline__ Pair<unsigned long long> lane_max_bits(LaneState<T>& L,
                                                                   unsigned long long v0,
                                                                   unsigned long long v1) {
  const Geo<T> g;
  constexpr int TPR = Geo<T>::TPR, NW = NTHREADS / 32;
#pragma unroll
  for (int off = 16; off >= TPR; off >>= 1) {
    const unsigned long long u0 = __shfl_xor_sync(0xffffffffu, v0, off);
    const unsigned long long u1 = __shfl_xor_sync(0xffffffffu, v1, off);
    v0 = u0 > v0 ? u0 : v0;
    v1 = u1 > v1 ? u1 : v1;
  }
  unsigned long long* buf = reinterpret_cast<unsigned long long*>(L.red2 + SITE * NW * T);
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) < TPR) {
    buf[w * T + g.lane] = v0;
    buf[w * T + g.lane + 1] = v1;
  }
  __syncthreads();
  unsigned long long s0 = buf[g.lane], s1 = buf[g.lane + 1];
#pragma unroll
  for (int k = 1; k < NW; ++k) {
    s0 = buf[k * T + g.lane] > s0 ? buf[k * T + g.lane] : s0;
    s1 = buf[k * T + g.lane + 1] > s1 ? buf[k * T + g.lane + 1] : s1;
  }
  return {s0, s1};
}

// ----------------------------------------------------- batched operators
// y = B_s v for the thread's two lanes: base row times v, plus the outaged
// branch's four-element change (Sec. IV.B) -- off-diagonal +w, diagonal -w
// at both ends.
//
// Plain (DIRECTION = false): q = B_s p, returns the lanes' partial p.q.
// DIRECTION = true, the PCG direction update folded in: with v = z,
//   p <- mask(z) + beta p,   q <- mask(B_s z) + beta q,
// which is q = B_s p for the new p because q held B_s p for the old one
// (first: p = mask(z), q = mask(B_s z)).  mask zeroes the rows of islanded
// buses: B_s couples no main-island row to an islanded one, so on the main
// island B_s z = B_s mask(z).  Returns the partial p.q of the new p, q.
template <int T, typename VT, bool DIRECTION>
__device__ GPCG_LOOP_INLINE Pair<VT> spmv_pass(const DevMatT<VT>& M, const VT* __restrict__ v_,
                                              VT* __restrict__ p, VT* __restrict__ q, int ra0,
                                              int rb0, VT w0, int ra1, int rb1, VT w1,
                                              VT be0 = 0, VT be1 = 0, bool first = true,
                                              int lo0 = 0, int cnt0 = 0, int lo1 = 0,
                                              int cnt1 = 0) {
  const Geo<T> g;
  constexpr int RPS = Geo<T>::RPS, STEP = RPS * UNR;
  VT pq0 = 0, pq1 = 0;
  // UNR rows per thread per step, and the column indices of the next step
  // loaded one step ahead: each step waits on one memory latency for
  // UNR rows' gathers
  // rows are visited in bus order (M.visit), so a row's neighbours were
  // visited just before it and their chunks of v are still in cache
  int cn[UNR][KA], vn[UNR];
#pragma unroll
  for (int u = 0; u < UNR; ++u)
    if (g.rs + u * RPS < M.n) {
      vn[u] = __ldg(M.visit + g.rs + u * RPS);
      ld_cols<KA>(M.A.col + (size_t)vn[u] * KA, cn[u]);
    }
  for (int i0 = g.rs; i0 < M.n; i0 += STEP) {
    int c[UNR][KA], ii[UNR];
    VT v[UNR][KA];
    Pair<VT> pc[UNR][KA], pi[UNR];
#pragma unroll
    for (int u = 0; u < UNR; ++u) {
      ii[u] = vn[u];
#pragma unroll
      for (int k = 0; k < KA; ++k) c[u][k] = cn[u][k];
      const int in = i0 + STEP + u * RPS;
      if (in < M.n) {
        vn[u] = __ldg(M.visit + in);
        ld_cols<KA>(M.A.col + (size_t)vn[u] * KA, cn[u]);
      }
    }
#pragma unroll
    for (int u = 0; u < UNR; ++u) {
      const int i = ii[u];
      if (i0 + u * RPS < M.n) {
        ld_vals<KA>(M.A.val + (size_t)i * KA, v[u]);
#pragma unroll
        for (int k = 0; k < KA; ++k) pc[u][k] = ld2(v_ + (size_t)c[u][k] * T + g.lane);
        pi[u] = ld2(v_ + (size_t)i * T + g.lane);
      }
    }
#pragma unroll
    for (int u = 0; u < UNR; ++u) {
      const int i = ii[u];
      if (i0 + u * RPS >= M.n) continue;
      VT a0 = 0, a1 = 0;
#pragma unroll
      for (int k = 0; k < KA; ++k) {
        a0 += v[u][k] * pc[u][k].a;
        a1 += v[u][k] * pc[u][k].b;
      }
      const int o0 = __ldg(M.A.optr + i), o1 = __ldg(M.A.optr + i + 1);
      for (int o = o0; o < o1; ++o) {
        const int cc = __ldg(M.A.ocol + o);
        const VT vv = __ldg(M.A.oval + o);
        const Pair<VT> pp = ld2(v_ + (size_t)cc * T + g.lane);
        a0 += vv * pp.a;
        a1 += vv * pp.b;
      }
      // the outage's change, on the two rows of the outaged branch only:
      // + w v_other (when the other end has a row) - w v_own
      if (i == ra0 || i == rb0) {
        const int oth = (i == ra0) ? rb0 : ra0;
        a0 += w0 * ((oth >= 0 ? v_[(size_t)oth * T + g.lane] : (VT)0) - pi[u].a);
      }
      if (i == ra1 || i == rb1) {
        const int oth = (i == ra1) ? rb1 : ra1;
        a1 += w1 * ((oth >= 0 ? v_[(size_t)oth * T + g.lane + 1] : (VT)0) - pi[u].b);
      }
      const size_t o = (size_t)i * T + g.lane;
      if (DIRECTION) {
        const int pr = __ldg(M.pre_of_row + i);
        const bool m0 = in_island(pr, lo0, cnt0), m1 = in_island(pr, lo1, cnt1);
        Pair<VT> pn{m0 ? (VT)0 : pi[u].a, m1 ? (VT)0 : pi[u].b};
        Pair<VT> qn{m0 ? (VT)0 : a0, m1 ? (VT)0 : a1};
        if (!first) {
          const Pair<VT> po = ld2(p + o), qo = ld2(q + o);
          pn.a += be0 * po.a;
          pn.b += be1 * po.b;
          qn.a += be0 * qo.a;
          qn.b += be1 * qo.b;
        }
        st2(p + o, pn);
        st2(q + o, qn);
        pq0 += pn.a * qn.a;
        pq1 += pn.b * qn.b;
      } else {
        st2(q + o, Pair<VT>{a0, a1});
        pq0 += pi[u].a * a0;
        pq1 += pi[u].b * a1;
      }
    }
  }
  return {pq0, pq1};
}

// The tail of the level schedule (rows [tail_row0, n): the last, narrow
// levels) is solved densely instead of level by level: with X = L_tt^-1 the
// inverse of the factor's tail block (computed once per factor),
//   forward:  y_t = X (r_t - L_t,s y_s)   (s: the rows solved before)
//   backward: z_t = X^T y_t               (tail rows depend on tail rows only)
// Each is one pass of all threads over X (stored both column- and row-major
// so both products read it coalesced) instead of one block barrier and one
// memory latency per narrow level.  s holds the tail's right-hand side,
// then y (TAIL_ROWS rows of T lanes).  Adds the tail rows' r.r to rr and
// their r.z to rzt; writes the tail's final z.
template <int T, typename VT, bool FUSED>
__device__ GPCG_LOOP_INLINE void tail_solve(const DevMatT<VT>& M, VT* __restrict__ x,
                                           VT* __restrict__ r, const VT* __restrict__ p,
                                           const VT* __restrict__ q, VT* __restrict__ z,
                                           VT al0, VT al1, VT* __restrict__ s, VT& rr0, VT& rr1,
                                           Pair<VT>& rzt) {
  const Geo<T> g;
  constexpr int RPS = Geo<T>::RPS, NPT = (TAIL_ROWS + RPS - 1) / RPS;
  const int t0 = M.tail_row0, nt = M.n - t0;
  // (a) right-hand side: the PCG update of the tail rows, minus the part of
  // their factor rows on the rows solved before the tail
  for (int k = g.rs; k < nt; k += RPS) {
    const int i = t0 + k;
    const size_t o = (size_t)i * T + g.lane;
    int c[KL];
    VT v[KL];
    ld_cols<KL>(M.L.col + (size_t)i * KL, c);
    if (M.Lh) ld_halfs<KL>(M.Lh + (size_t)i * KL, v);
    else ld_vals<KL>(M.L.val + (size_t)i * KL, v);
    Pair<VT> rv = ld2(r + o);
    if (FUSED) {
      const Pair<VT> pi = ld2(p + o), qi = ld2(q + o), xi = ld2(x + o);
      st2(x + o, Pair<VT>{xi.a + al0 * pi.a, xi.b + al1 * pi.b});
      rv.a -= al0 * qi.a;
      rv.b -= al1 * qi.b;
      st2(r + o, rv);
    } else {
      st2(x + o, Pair<VT>{(VT)0, (VT)0});
    }
    rr0 += rv.a * rv.a;
    rr1 += rv.b * rv.b;
    VT a0 = rv.a, a1 = rv.b;
#pragma unroll
    for (int k2 = 0; k2 < KL; ++k2) {
      if (c[k2] >= t0) continue;
      const Pair<VT> zz = ld2(z + (size_t)c[k2] * T + g.lane);
      a0 -= v[k2] * zz.a;
      a1 -= v[k2] * zz.b;
    }
    const int o0 = __ldg(M.L.optr + i), o1 = __ldg(M.L.optr + i + 1);
    for (int e = o0; e < o1; ++e) {
      const int cc = __ldg(M.L.ocol + e);
      if (cc >= t0) continue;
      const VT vv = M.Lh ? (VT)__half2float(M.Loh[e]) : __ldg(M.L.oval + e);
      const Pair<VT> zz = ld2(z + (size_t)cc * T + g.lane);
      a0 -= vv * zz.a;
      a1 -= vv * zz.b;
    }
    st2(s + (size_t)k * T + g.lane, Pair<VT>{a0, a1});
  }
  __syncthreads();
  // (b) y_t = X rhs: X_kj = xc[j nt + k], zero above the diagonal
  Pair<VT> y[NPT];
#pragma unroll
  for (int m = 0; m < NPT; ++m) {
    const int k = g.rs + m * RPS;
    VT a0 = 0, a1 = 0;
    if (k < nt) {
      const VT* col = M.xc + k;
#pragma unroll 4
      for (int j = 0; j < nt; ++j) {
        const VT xv = __ldg(col + (size_t)j * nt);
        const Pair<VT> sv = ld2(s + (size_t)j * T + g.lane);
        a0 += xv * sv.a;
        a1 += xv * sv.b;
      }
    }
    y[m] = Pair<VT>{a0, a1};
  }
  __syncthreads();
#pragma unroll
  for (int m = 0; m < NPT; ++m) {
    const int k = g.rs + m * RPS;
    if (k < nt) st2(s + (size_t)k * T + g.lane, y[m]);
  }
  __syncthreads();
  // (c) z_t = X^T y_t: X_ik = xr[i nt + k], zero for i < k
#pragma unroll
  for (int m = 0; m < NPT; ++m) {
    const int k = g.rs + m * RPS;
    if (k >= nt) continue;
    const VT* col = M.xr + k;
    VT a0 = 0, a1 = 0;
#pragma unroll 4
    for (int i = 0; i < nt; ++i) {
      const VT xv = __ldg(col + (size_t)i * nt);
      const Pair<VT> sv = ld2(s + (size_t)i * T + g.lane);
      a0 += xv * sv.a;
      a1 += xv * sv.b;
    }
    const size_t o = (size_t)(t0 + k) * T + g.lane;
    st2(z + o, Pair<VT>{a0, a1});
    const Pair<VT> ri = ld2(r + o);
    rzt.a += ri.a * a0;
    rzt.b += ri.b * a1;
  }
  __syncthreads();
}

// Forward substitution L y = r over the level schedule (rows of one level
// are independent).  With FUSED, first x += alpha p and r -= alpha q (the
// PCG update); without it, x = 0.  Accumulates r.r.  Each thread loads the
// column indices of its next row -- in this level or the next -- while it
// works on the current one, and the next level's bounds a level ahead, so
// after a level barrier only the gathers of the solved values are waited on.
template <int T, typename VT, bool FUSED>
__device__ GPCG_LOOP_INLINE Pair<VT> fwd_pass(const DevMatT<VT>& M, VT* __restrict__ x,
                                                 VT* __restrict__ r, const VT* __restrict__ p,
                                                 const VT* __restrict__ q, VT* __restrict__ z,
                                                 VT al0, VT al1, VT* zt, Pair<VT>& rzt) {
  const Geo<T> g;
  constexpr int RPS = Geo<T>::RPS;
  VT rr0 = 0, rr1 = 0;
  const int nl = M.tail_lev;
  int r0 = 0, r1 = 0, pf = -1, cn[KL];
  if (nl > 0) {
    r0 = __ldg(M.lev_ptr);
    r1 = __ldg(M.lev_ptr + 1);
    if (r0 + g.rs < r1) {
      pf = r0 + g.rs;
      ld_cols<KL>(M.L.col + (size_t)pf * KL, cn);
    }
  }
  for (int lev = 0; lev < nl; ++lev) {
    const int r2 = (lev + 1 < nl) ? __ldg(M.lev_ptr + lev + 2) : r1;  // end of the next level
    for (int i = r0 + g.rs; i < r1; i += RPS) {
      int c[KL];
      if (pf == i) {
#pragma unroll
        for (int k = 0; k < KL; ++k) c[k] = cn[k];
      } else {
        ld_cols<KL>(M.L.col + (size_t)i * KL, c);
      }
      const size_t o = (size_t)i * T + g.lane;
      VT v[KL];
      Pair<VT> zc[KL], ri, pi, qi, xi;
      if (M.Lh) ld_halfs<KL>(M.Lh + (size_t)i * KL, v);
      else ld_vals<KL>(M.L.val + (size_t)i * KL, v);
#pragma unroll
      for (int k = 0; k < KL; ++k) zc[k] = ld2(z + (size_t)c[k] * T + g.lane);
      ri = ld2(r + o);
      if (FUSED) {
        pi = ld2(p + o);
        qi = ld2(q + o);
        xi = ld2(x + o);
      }
      // the thread's next row: in this level, else the first of the next
      const int is = (i + RPS < r1) ? i + RPS : ((lev + 1 < nl && r1 + g.rs < r2) ? r1 + g.rs : -1);
      pf = is;
      if (is >= 0) ld_cols<KL>(M.L.col + (size_t)is * KL, cn);
      Pair<VT> rv = ri;
      if (FUSED) {
        st2(x + o, Pair<VT>{xi.a + al0 * pi.a, xi.b + al1 * pi.b});
        rv.a -= al0 * qi.a;
        rv.b -= al1 * qi.b;
        st2(r + o, rv);
      } else {
        st2(x + o, Pair<VT>{(VT)0, (VT)0});
      }
      rr0 += rv.a * rv.a;
      rr1 += rv.b * rv.b;
      VT a0 = rv.a, a1 = rv.b;
#pragma unroll
      for (int k = 0; k < KL; ++k) {
        a0 -= v[k] * zc[k].a;
        a1 -= v[k] * zc[k].b;
      }
      const int o0 = __ldg(M.L.optr + i), o1 = __ldg(M.L.optr + i + 1);
      for (int e = o0; e < o1; ++e) {
        const VT vv = M.Lh ? (VT)__half2float(M.Loh[e]) : __ldg(M.L.oval + e);
        const Pair<VT> zz = ld2(z + (size_t)__ldg(M.L.ocol + e) * T + g.lane);
        a0 -= vv * zz.a;
        a1 -= vv * zz.b;
      }
      // scaled factor: unit diagonal, w = D y is what is stored
      const VT id = M.Lh ? (VT)1 : __ldg(M.inv_diag + i);
      st2(z + o, Pair<VT>{a0 * id, a1 * id});
    }
    // no row in this level: load the next level's first row ahead anyway
    if (pf < 0 && lev + 1 < nl && r1 + g.rs < r2) {
      pf = r1 + g.rs;
      ld_cols<KL>(M.L.col + (size_t)pf * KL, cn);
    }
    __syncthreads();
    r0 = r1;
    r1 = r2;
  }
  if (M.tail_row0 < M.n) tail_solve<T, VT, FUSED>(M, x, r, p, q, z, al0, al1, zt, rr0, rr1, rzt);
  return {rr0, rr1};
}

// Back substitution L^T z = y in place (z holds y on entry), over the
// backward level schedule of the rows before the tail (the tail was solved
// in fwd_pass); accumulates r.z.  Rows and their column indices are loaded
// one row ahead across level barriers, as in fwd_pass.
template <int T, typename VT>
__device__ GPCG_LOOP_INLINE Pair<VT> bwd_pass(const DevMatT<VT>& M, const VT* __restrict__ r,
                                                 VT* __restrict__ z, Pair<VT> rzt) {
  const Geo<T> g;
  constexpr int RPS = Geo<T>::RPS;
  VT rz0 = rzt.a, rz1 = rzt.b;
  const int nb = M.ntblev;
  const int32_t* bptr = M.tblev_ptr;
  const int32_t* brows = M.tblev_rows;
  int r0 = 0, r1 = 0, pk = -1, pi_ = 0, cn[KU];
  if (nb > 0) {
    r0 = __ldg(bptr);
    r1 = __ldg(bptr + 1);
    if (r0 + g.rs < r1) {
      pk = r0 + g.rs;
      pi_ = __ldg(brows + pk);
      ld_cols<KU>(M.U.col + (size_t)pi_ * KU, cn);
    }
  }
  for (int lev = 0; lev < nb; ++lev) {
    const int r2 = (lev + 1 < nb) ? __ldg(bptr + lev + 2) : r1;
    for (int k = r0 + g.rs; k < r1; k += RPS) {
      int i, c[KU];
      if (pk == k) {
        i = pi_;
#pragma unroll
        for (int a = 0; a < KU; ++a) c[a] = cn[a];
      } else {
        i = __ldg(brows + k);
        ld_cols<KU>(M.U.col + (size_t)i * KU, c);
      }
      const size_t o = (size_t)i * T + g.lane;
      VT v[KU];
      Pair<VT> zc[KU];
      if (M.Uh) ld_halfs<KU>(M.Uh + (size_t)i * KU, v);
      else ld_vals<KU>(M.U.val + (size_t)i * KU, v);
#pragma unroll
      for (int a = 0; a < KU; ++a) zc[a] = ld2(z + (size_t)c[a] * T + g.lane);
      const Pair<VT> yi = ld2(z + o), ri = ld2(r + o);
      const int ks = (k + RPS < r1) ? k + RPS : ((lev + 1 < nb && r1 + g.rs < r2) ? r1 + g.rs : -1);
      pk = ks;
      if (ks >= 0) {
        pi_ = __ldg(brows + ks);
        ld_cols<KU>(M.U.col + (size_t)pi_ * KU, cn);
      }
      // scaled factor: L_s^T z = D^-2 w with a unit diagonal
      const VT pre = M.Uh ? __ldg(M.inv_d2 + i) : (VT)1;
      VT a0 = yi.a * pre, a1 = yi.b * pre;
#pragma unroll
      for (int a = 0; a < KU; ++a) {
        a0 -= v[a] * zc[a].a;
        a1 -= v[a] * zc[a].b;
      }
      const int o0 = __ldg(M.U.optr + i), o1 = __ldg(M.U.optr + i + 1);
      for (int e = o0; e < o1; ++e) {
        const VT vv = M.Uh ? (VT)__half2float(M.Uoh[e]) : __ldg(M.U.oval + e);
        const Pair<VT> zz = ld2(z + (size_t)__ldg(M.U.ocol + e) * T + g.lane);
        a0 -= vv * zz.a;
        a1 -= vv * zz.b;
      }
      const VT id = M.Uh ? (VT)1 : __ldg(M.inv_diag + i);
      a0 *= id;
      a1 *= id;
      st2(z + o, Pair<VT>{a0, a1});
      rz0 += ri.a * a0;
      rz1 += ri.b * a1;
    }
    if (pk < 0 && lev + 1 < nb && r1 + g.rs < r2) {
      pk = r1 + g.rs;
      pi_ = __ldg(brows + pk);
      ld_cols<KU>(M.U.col + (size_t)pi_ * KU, cn);
    }
    __syncthreads();
    r0 = r1;
    r1 = r2;
  }
  return {rz0, rz1};
}

// Jacobi: z = r / diag(B_s), the diagonal with the outage applied; a row
// whose diagonal vanishes (a bus the outage isolates) gets z = 0.
template <int T, typename VT, bool FUSED>
__device__ GPCG_LOOP_INLINE void jacobi_pass(const DevMatT<VT>& M, VT* __restrict__ x,
                                            VT* __restrict__ r, const VT* __restrict__ p,
                                            const VT* __restrict__ q, VT* __restrict__ z, VT al0,
                                            VT al1, int ra0, int rb0, VT w0, int ra1, int rb1,
                                            VT w1, Pair<VT>& rr, Pair<VT>& rz) {
  const Geo<T> g;
  for (int i = g.rs; i < M.n; i += Geo<T>::RPS) {
    const size_t o = (size_t)i * T + g.lane;
    Pair<VT> ri = ld2(r + o);
    if (FUSED) {
      const Pair<VT> pi = ld2(p + o), qi = ld2(q + o), xi = ld2(x + o);
      st2(x + o, Pair<VT>{xi.a + al0 * pi.a, xi.b + al1 * pi.b});
      ri.a -= al0 * qi.a;
      ri.b -= al1 * qi.b;
      st2(r + o, ri);
    } else {
      st2(x + o, Pair<VT>{(VT)0, (VT)0});
    }
    const VT dg = __ldg(M.diag + i);
    const VT d0 = dg - ((i == ra0 || i == rb0) ? w0 : (VT)0);
    const VT d1 = dg - ((i == ra1 || i == rb1) ? w1 : (VT)0);
    const VT z0 = d0 > (VT)0 ? ri.a / d0 : (VT)0;
    const VT z1 = d1 > (VT)0 ? ri.b / d1 : (VT)0;
    st2(z + o, Pair<VT>{z0, z1});
    rr.a += ri.a * ri.a;
    rr.b += ri.b * ri.b;
    rz.a += ri.a * z0;
    rz.b += ri.b * z1;
  }
  __syncthreads();
}

// ------------------------------------------------------------ the solve
// Per-lane scalars of the inner solve.  Each is written by the threads of
// row slot 0 in one phase of an iteration and read by every thread only
// after a later barrier; r.z alternates between two copies so the old value
// can be read while the new one is written.
template <int T, typename VT>
struct PcgLanes {
  VT rz[2][T];
  VT bb[T], rrmin[T];
  int stall[T];
  int pdone[T];  // stopped at the convergence test (written after r.r)
  int brk[T];    // p.Bp breakdown (written after p.Bp)
  int stop[T];   // r.z breakdown (written after r.z)
};

// Batched PCG (Sec. III.A listing, read as textbook PCG) on B_s x = r for
// the lanes that are active; x starts at 0.  Adds each lane's iteration
// count to iters[lane].  Every thread computes alpha and beta of its own
// lanes from the reduced sums, so an iteration has five barriers besides
// the substitution levels'.
template <int T, typename VT>
__device__ GPCG_PASS_INLINE void pcg_solve(const FdpfParams& P, const DevMatT<VT>& M, LaneState<T>& L, VT* x,
                          VT* r, VT* p, VT* q, VT* z, const int* ra_, const int* rb_,
                          const double* w_, int* iters) {
  __shared__ PcgLanes<T, VT> S;
  // right-hand side and y of the schedule's tail (lane pairs: 16-byte aligned)
  __shared__ __align__(16) VT zt[TAIL_ROWS * T];
  const Geo<T> g;
  const int l0 = g.lane, l1 = g.lane + 1;
  // the outage's rows (-1: none) of the lanes that run; the SpMV reads the
  // vector at the other end's row
  const bool on0 = L.active[l0], on1 = L.active[l1];
  const int ra0 = on0 ? ra_[l0] : -1, rb0 = on0 ? rb_[l0] : -1;
  const int ra1 = on1 ? ra_[l1] : -1, rb1 = on1 ? rb_[l1] : -1;
  const VT w0 = (VT)w_[l0], w1 = (VT)w_[l1];
  const int lo0 = L.lo[l0], cnt0 = L.cnt[l0], lo1 = L.lo[l1], cnt1 = L.cnt[l1];
  const bool jac = (P.precond == PREC_JACOBI);
  // the zero row that padding slots point at
  if (g.rs == 0) {
    st2(p + (size_t)M.n * T + g.lane, Pair<VT>{(VT)0, (VT)0});
    st2(z + (size_t)M.n * T + g.lane, Pair<VT>{(VT)0, (VT)0});
  }
  __syncthreads();
  Pair<VT> bbp{0, 0}, rzp{0, 0};
  if (jac) {
    jacobi_pass<T, VT, false>(M, x, r, p, q, z, (VT)0, (VT)0, ra0, rb0, w0, ra1, rb1, w1, bbp, rzp);
  } else {
    Pair<VT> rzt{0, 0};
    bbp = fwd_pass<T, VT, false>(M, x, r, p, q, z, (VT)0, (VT)0, zt, rzt);
    rzp = bwd_pass<T, VT>(M, r, z, rzt);
  }
  const Pair<VT> bb = lane_sum<T, RS_BB>(L, bbp.a, bbp.b);
  const Pair<VT> rz0 = lane_sum<T, RS_RZ0>(L, rzp.a, rzp.b);
  if (g.rs == 0) {
#pragma unroll
    for (int j = 0; j < LP; ++j) {
      const int ln = g.lane + j;
      const VT b_ = j ? bb.b : bb.a, r_ = j ? rz0.b : rz0.a;
      S.bb[ln] = b_;
      S.rz[0][ln] = r_;
      S.rrmin[ln] = b_;
      S.stall[ln] = 0;
      S.brk[ln] = 0;
      S.stop[ln] = 0;
      S.pdone[ln] = !L.active[ln] || !(b_ > (VT)0) || !(r_ > (VT)0);
    }
  }
  __syncthreads();  // publishes S and the first z
  const VT tol2 = (VT)(P.inner_rtol * P.inner_rtol);
  int par = 0;
  VT be0 = 0, be1 = 0;
  for (int it = 0; it < P.max_inner; ++it) {
    bool any = false;
#pragma unroll 1
    for (int k = 0; k < T; ++k) any |= !(S.pdone[k] | S.stop[k]);
    if (!any) break;
    const bool run0 = !(S.pdone[l0] | S.stop[l0]), run1 = !(S.pdone[l1] | S.stop[l1]);
    // new direction p = mask(z) + beta p and q = B_s p in one pass
    const Pair<VT> pqp = spmv_pass<T, VT, true>(M, z, p, q, ra0, rb0, w0, ra1, rb1, w1, be0,
                                                be1, it == 0, lo0, cnt0, lo1, cnt1);
    const Pair<VT> pq = lane_sum<T, RS_PQ>(L, pqp.a, pqp.b);
    VT al0 = 0, al1 = 0;
    bool bk0 = false, bk1 = false;
    if (run0) {
      if (pq.a > (VT)0 && isfinite(pq.a)) al0 = S.rz[par][l0] / pq.a;
      else bk0 = true;  // breakdown: keep the current iterate
    }
    if (run1) {
      if (pq.b > (VT)0 && isfinite(pq.b)) al1 = S.rz[par][l1] / pq.b;
      else bk1 = true;
    }
    if (g.rs == 0) {
      if (bk0) S.brk[l0] = 1;
      if (bk1) S.brk[l1] = 1;
    }
    Pair<VT> rrp{0, 0}, rzn{0, 0};
    if (jac) {
      jacobi_pass<T, VT, true>(M, x, r, p, q, z, al0, al1, ra0, rb0, w0, ra1, rb1, w1, rrp, rzn);
    } else {
      rrp = fwd_pass<T, VT, true>(M, x, r, p, q, z, al0, al1, zt, rzn);  // rzn: the tail's r.z
    }
    const Pair<VT> rr = lane_sum<T, RS_RR>(L, rrp.a, rrp.b);
    if (g.rs == 0) {
#pragma unroll
      for (int j = 0; j < LP; ++j) {
        const int ln = g.lane + j;
        const VT v = j ? rr.b : rr.a;
        if (S.pdone[ln] | S.stop[ln]) continue;
        if (S.brk[ln]) { S.pdone[ln] = 1; continue; }
        iters[ln] += 1;
        // converged; or stagnated at the rounding floor of VT (no 0.1 % gain
        // in STALL_ITERS iterations); or growing away from the best residual
        if (v < (VT)0.999 * S.rrmin[ln]) { S.rrmin[ln] = v; S.stall[ln] = 0; }
        else S.stall[ln] += 1;
        if (v <= tol2 * S.bb[ln] || !isfinite(v) || S.stall[ln] >= STALL_ITERS ||
            v > (VT)1e4 * S.rrmin[ln])
          S.pdone[ln] = 1;
      }
    }
    __syncthreads();
    // lanes still running, read before S.stop is next written (after r.z)
    const bool go0 = !(S.pdone[l0] | S.stop[l0]), go1 = !(S.pdone[l1] | S.stop[l1]);
    any = false;
#pragma unroll 1
    for (int k = 0; k < T; ++k) any |= !(S.pdone[k] | S.stop[k]);
    if (!any) break;
    if (!jac) rzn = bwd_pass<T, VT>(M, r, z, rzn);
    const Pair<VT> rz = lane_sum<T, RS_RZ>(L, rzn.a, rzn.b);
    be0 = go0 ? rz.a / S.rz[par][l0] : (VT)0;
    be1 = go1 ? rz.b / S.rz[par][l1] : (VT)0;
    if (g.rs == 0) {
#pragma unroll
      for (int j = 0; j < LP; ++j) {
        const int ln = g.lane + j;
        if (!(j ? go1 : go0)) continue;
        const VT v = j ? rz.b : rz.a;
        S.rz[par ^ 1][ln] = v;
        if (!(v > (VT)0)) S.stop[ln] = 1;
      }
    }
    __syncthreads();  // publishes S.rz, S.stop and z
    par ^= 1;
  }
  __syncthreads();
}


}  // namespace gpcg
