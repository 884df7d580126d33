// Batched operators and the batched PCG shared by the persistent kernels
// (fdpf.cu: the N-1 screen; adjoint.cu: the overload-penalty adjoint).
//
// A CTA owns T scenario lanes; vectors are [row][T]; each thread owns LP
// adjacent lanes of a row (Geo<T>::LP).  Every sparse row is read through a
// padded descriptor (ELL) so a thread issues all of a row's gathers at once.
#pragma once
#include <math.h>
#include "common.cuh"
#include "fdpf.h"

namespace gpcg {

#ifndef FDPF_LP
#define FDPF_LP 2
#endif
constexpr int LP_MAX = FDPF_LP;  // scenario lanes a thread holds, at most
#ifndef FDPF_UNROLL
#define FDPF_UNROLL 1
#endif
constexpr int UNR = FDPF_UNROLL;  // rows per thread in flight in the SpMV
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
template <typename X> struct Pair { X a, b; };
template <typename X, int N> struct Vec { X v[N]; };

// FP64 <-> FP32 conversions from the IEEE-754 binary64 / binary32 layouts,
// in integer operations: GB300 issues the conversion instructions on its
// FP64 pipe (2 operations per SM per cycle), integer operations run at the
// FP32 rate.  Both are exact or round to nearest (ties away from zero) for
// normal numbers; magnitudes below the FP32 normal range become a signed
// zero (the mixed-precision path never needs them: they are far below the
// FP32 rounding of any quantity they are added to); infinities and NaNs
// stay non-finite.
__device__ __forceinline__ float cvt_f32(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned hi = (unsigned)(b >> 32), lo = (unsigned)b;
  const unsigned sign = hi & 0x80000000u;
  const int e = (int)((hi >> 20) & 0x7ffu) - (1023 - 127);
  // 20 fraction bits from the high word, 3 from the low one, and the first
  // dropped bit added: a carry out of the fraction lands in the exponent
  const unsigned r = ((unsigned)e << 23) + (((hi & 0xfffffu) << 3) | (lo >> 29)) +
                     ((lo >> 28) & 1u);
  const unsigned out = e <= 0 ? sign : (e >= 255 || r >= 0x7f800000u) ? (sign | 0x7f800000u)
                                                                      : (sign | r);
  return __uint_as_float(out);
}
__device__ __forceinline__ double cvt_f64(float x) {
  const unsigned b = __float_as_uint(x);
  const unsigned sign = b & 0x80000000u, e = (b >> 23) & 0xffu, m = b & 0x7fffffu;
  const unsigned eo = e == 255u ? 0x7ffu : e + (1023u - 127u);
  const unsigned hi = e ? (sign | (eo << 20) | (m >> 3)) : sign;
  const unsigned lo = e ? (m << 29) : 0u;
  return __hiloint2double((int)hi, (int)lo);
}
template <typename VT> __device__ __forceinline__ VT to_vt(double x);
template <> __device__ __forceinline__ float to_vt<float>(double x) { return cvt_f32(x); }
template <> __device__ __forceinline__ double to_vt<double>(double x) { return x; }
__device__ __forceinline__ double to_f64(float x) { return cvt_f64(x); }
__device__ __forceinline__ float to_f32(double x) { return cvt_f32(x); }
__device__ __forceinline__ float to_f32(float x) { return x; }
__device__ __forceinline__ double to_f64(double x) { return x; }

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

// N consecutive lanes (N = 2 or 4), one vector access per 8 or 16 bytes.
template <int N>
__device__ __forceinline__ Vec<float, N> ldv(const float* p) {
  Vec<float, N> r;
  if constexpr (N == 2) {
    const float2 u = *reinterpret_cast<const float2*>(p);
    r.v[0] = u.x; r.v[1] = u.y;
  } else {
    static_assert(N == 4, "2 or 4 lanes");
    const float4 u = *reinterpret_cast<const float4*>(p);
    r.v[0] = u.x; r.v[1] = u.y; r.v[2] = u.z; r.v[3] = u.w;
  }
  return r;
}
template <int N>
__device__ __forceinline__ Vec<double, N> ldv(const double* p) {
  static_assert(N == 2 || N == 4, "2 or 4 lanes");
  Vec<double, N> r;
#pragma unroll
  for (int k = 0; k < N; k += 2) {
    const double2 u = reinterpret_cast<const double2*>(p)[k / 2];
    r.v[k] = u.x; r.v[k + 1] = u.y;
  }
  return r;
}
template <int N>
__device__ __forceinline__ void stv(float* p, const Vec<float, N>& r) {
  if constexpr (N == 2) {
    *reinterpret_cast<float2*>(p) = make_float2(r.v[0], r.v[1]);
  } else {
    static_assert(N == 4, "2 or 4 lanes");
    *reinterpret_cast<float4*>(p) = make_float4(r.v[0], r.v[1], r.v[2], r.v[3]);
  }
}
template <int N>
__device__ __forceinline__ void stv(double* p, const Vec<double, N>& r) {
  static_assert(N == 2 || N == 4, "2 or 4 lanes");
#pragma unroll
  for (int k = 0; k < N; k += 2)
    reinterpret_cast<double2*>(p)[k / 2] = make_double2(r.v[k], r.v[k + 1]);
}
template <typename X, int N>
__device__ __forceinline__ Vec<X, N> vzero() {
  Vec<X, N> r;
#pragma unroll
  for (int j = 0; j < N; ++j) r.v[j] = (X)0;
  return r;
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

// ------------------------------------------------------------ geometry
template <int T>
struct Geo {
  static constexpr int LP = T < LP_MAX ? T : LP_MAX;  // lanes per thread
  static constexpr int TPR = T / LP;                  // threads per row
  static constexpr int RPS = NTHREADS / TPR;          // rows per step
  int rs, lane;                                       // row slot, first lane
  __device__ Geo() : rs(threadIdx.x / TPR), lane((threadIdx.x % TPR) * LP) {}
};

// ------------------------------------------------------------ lane state
// Per-lane B'' extension rows (the kernel with extension rows keeps this
// in shared memory of its own): the tripped generator's bus and PV buses
// switched to PQ at a reactive limit, with the reactive injection each now
// holds and the limit it is held at (xs: +1 Q_max, -1 Q_min, 0 the tripped
// bus); the PV buses the last P mismatch found outside their limits (nc may
// exceed KX: only the first KX are kept), with their new injection and
// limit; the extension rows whose bus can hold its set point again (bk, a
// bit per row); and the lanes that sit out the rest of an outer iteration
// after a switch (skip), so that the next one starts from a fresh mismatch.
template <int T>
struct SwitchState {
  int nx[T], xb[T][KX], xs[T][KX];
  double xq[T][KX];
  int nc[T], cb[T][KX], cs[T][KX];
  double cq[T][KX];
  unsigned bk[T];
  int skip[T];
};

constexpr int NRED_SITES = 10;  // reduction sites with a buffer of their own
enum RedSite { RS_BB = 0, RS_RZ0, RS_PQ, RS_RR, RS_RZ, RS_ERRP, RS_ERRQ, RS_LOAD, RS_RQ, RS_QQ };

template <int T>
struct LaneState {
  int scen[T], l[T], fb[T], tb[T], lo[T], cnt[T];
  int raP[T], rbP[T], raQ[T], rbQ[T];
  double wP[T], wQ[T], coef[T], gl[T], bl[T];
  double cl[T];  // the outaged branch's 1 / turns ratio (1 for a line)
  // the outaged branch's off-diagonal admittance entries as the bus
  // adjacency holds them, at its from end [0] and its to end [1]
  double og[T][2], ob[T][2];
  int gb[T];     // bus of a tripped generator (-1: none)
  int active[T], outer[T], inP[T], inQ[T], status[T], nogen[T];
  double err[T], best[T];
  unsigned long long tphase[8];
  int done[T], fresh[T];
  // lanes that take no step in the current half-step: their own mismatch is
  // already within the tolerance
  int hold[T];
  double xalpha[T];          // a deferred last step x += alpha p of the inner solve
  // one small buffer per reduction site (see lane_sum): [site][warp][lane]
  double red2[NRED_SITES * (NTHREADS / 32) * T];
  int flag;
  int drained;
};

// Sum (or max) over the row slots of each lane's partial values, for
// layouts with two lanes per thread, through `red` (NTHREADS * 2 doubles of
// shared memory that the calling kernel provides).
template <int T, bool MAX>
__device__ __forceinline__ Pair<double> lane_reduce(double* red, double v0, double v1) {
  static_assert(Geo<T>::LP == 2, "two lanes per thread");
  const Geo<T> g;
  constexpr int RPS = Geo<T>::RPS;
  red[g.rs * T + g.lane] = v0;
  red[g.rs * T + g.lane + 1] = v1;
  __syncthreads();
#pragma unroll
  for (int st = RPS / 2; st > 0; st >>= 1) {
    if (g.rs < st) {
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        const int o = g.rs * T + g.lane + j;
        const double a = red[o], b = red[o + st * T];
        red[o] = MAX ? ((b > a || b != b) ? b : a) : a + b;
      }
    }
    __syncthreads();
  }
  const Pair<double> out{red[g.lane], red[g.lane + 1]};
  __syncthreads();
  return out;
}

// True when some active lane is not held (block-uniform).
template <int T>
__device__ __forceinline__ bool any_stepping(LaneState<T>& L) {
  __syncthreads();
  if (threadIdx.x == 0) {
    int any = 0;
    for (int s = 0; s < T; ++s) any |= (L.active[s] != 0 && L.hold[s] == 0);
    L.flag = any;
  }
  __syncthreads();
  const bool r = L.flag != 0;
  __syncthreads();
  return r;
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
// A loading (non-negative) above 1, infinity included and NaN not, decided on
// the bit pattern (the order of non-negative doubles is their integer order).
__device__ __forceinline__ bool overloaded(double ld) {
  const unsigned long long b = abs_bits(ld);
  return b > 0x3ff0000000000000ull && b <= 0x7ff0000000000000ull;
}
__device__ __forceinline__ double from_bits(unsigned long long b) {
  const double v = __longlong_as_double((long long)b);
  return v == v ? v : INFINITY;
}

// Per-lane sum of the threads' partial values in a fixed order: a shuffle
// tree inside each warp over the threads that hold the same lanes, then the
// warps' partials through shared memory (buffer SITE) and one barrier.
// Every thread returns the totals of its own lanes.  A site's buffer is
// read right after the barrier and rewritten only after a later barrier,
// so consecutive reductions at different sites need no barrier between.
template <int T, int SITE, typename X, int N>
__device__ __forceinline__ Vec<X, N> lane_sum(LaneState<T>& L, Vec<X, N> v) {
  static_assert(N == Geo<T>::LP, "a thread's lanes");
  const Geo<T> g;
  constexpr int TPR = Geo<T>::TPR, NW = NTHREADS / 32;
#pragma unroll
  for (int off = 16; off >= TPR; off >>= 1)
#pragma unroll
    for (int j = 0; j < N; ++j) v.v[j] += __shfl_xor_sync(0xffffffffu, v.v[j], off);
  X* buf = reinterpret_cast<X*>(L.red2 + SITE * NW * T);
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) < TPR)
#pragma unroll
    for (int j = 0; j < N; ++j) buf[w * T + g.lane + j] = v.v[j];
  __syncthreads();
  Vec<X, N> s;
#pragma unroll
  for (int j = 0; j < N; ++j) s.v[j] = buf[g.lane + j];
#pragma unroll
  for (int k = 1; k < NW; ++k)
#pragma unroll
    for (int j = 0; j < N; ++j) s.v[j] += buf[k * T + g.lane + j];
  return s;
}

// Three sums at three sites with one barrier (see lane_sum).
template <int T, int S1, int S2, int S3, typename X, int N>
__device__ __forceinline__ void lane_sum3(LaneState<T>& L, Vec<X, N>& a, Vec<X, N>& b,
                                          Vec<X, N>& c) {
  static_assert(N == Geo<T>::LP, "a thread's lanes");
  const Geo<T> g;
  constexpr int TPR = Geo<T>::TPR, NW = NTHREADS / 32;
#pragma unroll
  for (int off = 16; off >= TPR; off >>= 1)
#pragma unroll
    for (int j = 0; j < N; ++j) {
      a.v[j] += __shfl_xor_sync(0xffffffffu, a.v[j], off);
      b.v[j] += __shfl_xor_sync(0xffffffffu, b.v[j], off);
      c.v[j] += __shfl_xor_sync(0xffffffffu, c.v[j], off);
    }
  X* ba = reinterpret_cast<X*>(L.red2 + S1 * NW * T);
  X* bb = reinterpret_cast<X*>(L.red2 + S2 * NW * T);
  X* bc = reinterpret_cast<X*>(L.red2 + S3 * NW * T);
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) < TPR)
#pragma unroll
    for (int j = 0; j < N; ++j) {
      ba[w * T + g.lane + j] = a.v[j];
      bb[w * T + g.lane + j] = b.v[j];
      bc[w * T + g.lane + j] = c.v[j];
    }
  __syncthreads();
#pragma unroll
  for (int j = 0; j < N; ++j) {
    a.v[j] = ba[g.lane + j];
    b.v[j] = bb[g.lane + j];
    c.v[j] = bc[g.lane + j];
  }
#pragma unroll
  for (int k = 1; k < NW; ++k)
#pragma unroll
    for (int j = 0; j < N; ++j) {
      a.v[j] += ba[k * T + g.lane + j];
      b.v[j] += bb[k * T + g.lane + j];
      c.v[j] += bc[k * T + g.lane + j];
    }
}

// The same for running maxima held as abs_bits patterns.
template <int T, int SITE, int N>
__device__ __forceinline__ Vec<unsigned long long, N> lane_max_bits(
    LaneState<T>& L, Vec<unsigned long long, N> v) {
  static_assert(N == Geo<T>::LP, "a thread's lanes");
  const Geo<T> g;
  constexpr int TPR = Geo<T>::TPR, NW = NTHREADS / 32;
#pragma unroll
  for (int off = 16; off >= TPR; off >>= 1)
#pragma unroll
    for (int j = 0; j < N; ++j) {
      const unsigned long long u = __shfl_xor_sync(0xffffffffu, v.v[j], off);
      v.v[j] = u > v.v[j] ? u : v.v[j];
    }
  unsigned long long* buf = reinterpret_cast<unsigned long long*>(L.red2 + SITE * NW * T);
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) < TPR)
#pragma unroll
    for (int j = 0; j < N; ++j) buf[w * T + g.lane + j] = v.v[j];
  __syncthreads();
  Vec<unsigned long long, N> s;
#pragma unroll
  for (int j = 0; j < N; ++j) s.v[j] = buf[g.lane + j];
#pragma unroll
  for (int k = 1; k < NW; ++k)
#pragma unroll
    for (int j = 0; j < N; ++j) {
      const unsigned long long u = buf[k * T + g.lane + j];
      s.v[j] = u > s.v[j] ? u : s.v[j];
    }
  return s;
}

// ----------------------------------------------------- the outage's change
// Rows, weight and from-end factor of each lane's outaged branch in the
// matrix being solved (-1: that end has no row): the outage removes
// w v v^T, v = c e_ra - e_rb (c = 1 / turns ratio in B'', 1 in B').
// stamp_filter sets bit (row & 63) for every such row, so the SpMV tests one
// bit per row and looks at the lanes only on a hit.
template <int T, typename VT>
struct Stamp {
  int ra[T], rb[T];
  VT w[T], c[T];
};

// A PV bus that becomes PQ -- its generator tripped, or held at a reactive
// limit -- gets the B'' row it lacks: extension row s of a lane sits at
// vector row n + 1 + s (row n is the zero row), up to KX per lane; per lane
// their number, buses and diagonals.  The base-case factor preconditions
// the rows it has, the diagonals these (a block-diagonal preconditioner).
template <int T, typename VT, int K = KX>
struct Ext {
  int n[T];
  int lb[T];  // the lane's outaged branch (-1: none): not part of these rows
  int gb[T][K];
  VT gd[T][K];
};

template <int T, typename VT>
__device__ __forceinline__ unsigned long long stamp_filter(const Stamp<T, VT>& S) {
  unsigned long long f = 0ull;
#pragma unroll 1
  for (int j = 0; j < T; ++j) {
    if (S.ra[j] >= 0) f |= 1ull << (S.ra[j] & 63);
    if (S.rb[j] >= 0) f |= 1ull << (S.rb[j] & 63);
  }
  return f;
}

// ----------------------------------------------------- batched operators
// y = B_s v for the thread's lanes: base row times v, plus the outaged
// branch's four-element change (Sec. IV.B) -- off-diagonal +w c, diagonal
// -w c^2 at the from end and -w at the to end (c = 1 without a transformer).
//
// Plain (DIRECTION = false): q = B_s p, returns the lanes' partial p.q.
// DIRECTION = true, the PCG direction update folded in: with v = z,
//   p <- mask(z) + beta p,   q <- mask(B_s z) + beta q,
// which is q = B_s p for the new p because q held B_s p for the old one
// (first: p = mask(z), q = mask(B_s z)).  mask zeroes the rows of islanded
// buses (isl: the lanes' island intervals, null when no lane has one):
// B_s couples no main-island row to an islanded one, so on the main island
// B_s z = B_s mask(z).  Returns the partial p.q of the new p, q.
template <int T, typename VT, bool DIRECTION>
__device__ GPCG_LOOP_INLINE Vec<VT, Geo<T>::LP> spmv_pass(
    const DevMatT<VT>& M, const VT* __restrict__ v_, VT* __restrict__ p, VT* __restrict__ q,
    const Stamp<T, VT>& S, unsigned long long filt, Vec<VT, Geo<T>::LP> be, bool first,
    const LaneState<T>* isl, const VT* __restrict__ r = nullptr,
    Vec<VT, Geo<T>::LP>* rq = nullptr, Vec<VT, Geo<T>::LP>* qq = nullptr,
    const Ext<T, VT>* X = nullptr) {
  constexpr int LP = Geo<T>::LP;
  const Geo<T> g;
  constexpr int RPS = Geo<T>::RPS, STEP = RPS * UNR;
  Vec<VT, LP> pq = vzero<VT, LP>();
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
      if (i0 + u * RPS >= M.n) continue;
      VT v[KA];
      Vec<VT, LP> pc[KA];
      ld_vals<KA>(M.A.val + (size_t)i * KA, v);
#pragma unroll
      for (int k = 0; k < KA; ++k) pc[k] = ldv<LP>(v_ + (size_t)c[u][k] * T + g.lane);
      const size_t o = (size_t)i * T + g.lane;
      const Vec<VT, LP> pi = ldv<LP>(v_ + o);
      Vec<VT, LP> a = vzero<VT, LP>();
#pragma unroll
      for (int k = 0; k < KA; ++k)
#pragma unroll
        for (int j = 0; j < LP; ++j) a.v[j] += v[k] * pc[k].v[j];
      const int o0 = __ldg(M.A.optr + i), o1 = __ldg(M.A.optr + i + 1);
      for (int e = o0; e < o1; ++e) {
        const int cc = __ldg(M.A.ocol + e);
        const VT vv = __ldg(M.A.oval + e);
        const Vec<VT, LP> pp = ldv<LP>(v_ + (size_t)cc * T + g.lane);
#pragma unroll
        for (int j = 0; j < LP; ++j) a.v[j] += vv * pp.v[j];
      }
      // the outage's change, on the two rows of the outaged branch only:
      // -w v (v.x) with v = c e_ra - e_rb (an end without a row holds 0)
      if ((filt >> (i & 63)) & 1ull) {
#pragma unroll
        for (int j = 0; j < LP; ++j) {
          const int ln = g.lane + j, ra = S.ra[ln], rb = S.rb[ln];
          if (i == ra || i == rb) {
            const VT xa = i == ra ? pi.v[j] : (ra >= 0 ? v_[(size_t)ra * T + ln] : (VT)0);
            const VT xb = i == rb ? pi.v[j] : (rb >= 0 ? v_[(size_t)rb * T + ln] : (VT)0);
            const VT wt = S.w[ln] * (S.c[ln] * xa - xb);
            a.v[j] += i == ra ? -(S.c[ln] * wt) : wt;
          }
        }
        // a neighbour of an extension row's bus: its coupling to that row
        if (X) {
#pragma unroll
          for (int j = 0; j < LP; ++j) {
            const int ln = g.lane + j, ne = X->n[ln];
            for (int s = 0; s < ne; ++s) {
              const int b = X->gb[ln][s];
              const VT ve = v_[(size_t)(M.n + 1 + s) * T + ln];
              const int e1 = __ldg(M.xptr + b + 1);
              for (int e = __ldg(M.xptr + b); e < e1; ++e)
                if (__ldg(M.xrow + e) == i && __ldg(M.xbr + e) != X->lb[ln])
                  a.v[j] += __ldg(M.xval + e) * ve;
            }
          }
        }
      }
      if (DIRECTION) {
        Vec<VT, LP> pn = pi, qn = a;
        if (isl) {
          const int pr = __ldg(M.pre_of_row + i);
#pragma unroll
          for (int j = 0; j < LP; ++j)
            if (in_island(pr, isl->lo[g.lane + j], isl->cnt[g.lane + j])) {
              pn.v[j] = (VT)0;
              qn.v[j] = (VT)0;
            }
        }
        if (!first) {
          const Vec<VT, LP> po = ldv<LP>(p + o), qo = ldv<LP>(q + o);
#pragma unroll
          for (int j = 0; j < LP; ++j) {
            pn.v[j] += be.v[j] * po.v[j];
            qn.v[j] += be.v[j] * qo.v[j];
          }
        }
        stv<LP>(p + o, pn);
        stv<LP>(q + o, qn);
#pragma unroll
        for (int j = 0; j < LP; ++j) pq.v[j] += pn.v[j] * qn.v[j];
        if (r) {  // r.q and q.q: the residual after the step, before taking it
          const Vec<VT, LP> ro = ldv<LP>(r + o);
#pragma unroll
          for (int j = 0; j < LP; ++j) {
            rq->v[j] += ro.v[j] * qn.v[j];
            qq->v[j] += qn.v[j] * qn.v[j];
          }
        }
      } else {
        stv<LP>(q + o, a);
#pragma unroll
        for (int j = 0; j < LP; ++j) pq.v[j] += pi.v[j] * a.v[j];
      }
    }
  }
  // the extension rows: couplings to the matrix rows and to the lane's
  // other extension rows (two switched buses next to each other)
  if (DIRECTION && X && g.rs == 0) {
#pragma unroll
    for (int j = 0; j < LP; ++j)
    for (int s = 0; s < X->n[g.lane + j]; ++s) {
      const int ln = g.lane + j, ne = X->n[ln], b = X->gb[ln][s];
      const size_t o = (size_t)(M.n + 1 + s) * T + ln;
      const VT ve = v_[o];
      VT a = X->gd[ln][s] * ve;
      const int e1 = __ldg(M.xptr + b + 1);
      for (int e = __ldg(M.xptr + b); e < e1; ++e) {
        if (__ldg(M.xbr + e) == X->lb[ln]) continue;  // the outaged branch
        const int rw = __ldg(M.xrow + e);
        if (rw >= 0) {
          a += __ldg(M.xval + e) * v_[(size_t)rw * T + ln];
        } else {
          const int nb = __ldg(M.xnb + e);
          for (int t = 0; t < ne; ++t)
            if (t != s && X->gb[ln][t] == nb)
              a += __ldg(M.xval + e) * v_[(size_t)(M.n + 1 + t) * T + ln];
        }
      }
      VT pn = ve, qn = a;
      if (!first) {
        pn += be.v[j] * p[o];
        qn += be.v[j] * q[o];
      }
      p[o] = pn;
      q[o] = qn;
      pq.v[j] += pn * qn;
      if (r) {
        rq->v[j] += r[o] * qn;
        qq->v[j] += qn * qn;
      }
    }
  }
  return pq;
}

// The extension rows in the forward (or Jacobi) pass: the PCG update
// (FUSED) or x = 0, r.r, and z = r / diagonal with its r.z.
template <int T, typename VT, bool FUSED>
__device__ __forceinline__ void ext_update(const DevMatT<VT>& M, const Ext<T, VT>* X,
                                           VT* __restrict__ x, VT* __restrict__ r,
                                           const VT* __restrict__ p, const VT* __restrict__ q,
                                           VT* __restrict__ z, const Vec<VT, Geo<T>::LP>& al,
                                           Vec<VT, Geo<T>::LP>& rr, Vec<VT, Geo<T>::LP>& rz) {
  constexpr int LP = Geo<T>::LP;
  const Geo<T> g;
  if (!X || g.rs != 0) return;
#pragma unroll
  for (int j = 0; j < LP; ++j)
  for (int s = 0; s < X->n[g.lane + j]; ++s) {
    const int ln = g.lane + j;
    const size_t o = (size_t)(M.n + 1 + s) * T + ln;
    VT rv = r[o];
    if (FUSED) {
      x[o] = fma(al.v[j], p[o], x[o]);
      rv -= al.v[j] * q[o];
      r[o] = rv;
    } else {
      x[o] = (VT)0;
    }
    rr.v[j] += rv * rv;
    const VT d = X->gd[ln][s];
    const VT zv = d > (VT)0 ? rv / d : (VT)0;
    z[o] = zv;
    rz.v[j] += rv * zv;
  }
}

// The PCG update of one row in the forward pass: x += alpha p, r -= alpha q
// (FUSED), or x = 0; returns the row's residual and adds its r.r.
template <int T, typename VT, bool FUSED>
__device__ __forceinline__ Vec<VT, Geo<T>::LP> pcg_update_row(
    size_t o, VT* __restrict__ x, VT* __restrict__ r, const VT* __restrict__ p,
    const VT* __restrict__ q, const Vec<VT, Geo<T>::LP>& al, Vec<VT, Geo<T>::LP>& rr) {
  constexpr int LP = Geo<T>::LP;
  Vec<VT, LP> rv = ldv<LP>(r + o);
  if (FUSED) {
    const Vec<VT, LP> pi = ldv<LP>(p + o), qi = ldv<LP>(q + o);
    Vec<VT, LP> xi = ldv<LP>(x + o);
#pragma unroll
    for (int j = 0; j < LP; ++j) {
      xi.v[j] = fma(al.v[j], pi.v[j], xi.v[j]);  // as the deferred step takes it
      rv.v[j] -= al.v[j] * qi.v[j];
    }
    stv<LP>(x + o, xi);
    stv<LP>(r + o, rv);
  } else {
    stv<LP>(x + o, vzero<VT, LP>());
  }
#pragma unroll
  for (int j = 0; j < LP; ++j) rr.v[j] += rv.v[j] * rv.v[j];
  return rv;
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
                                           const Vec<VT, Geo<T>::LP>& al, VT* __restrict__ s,
                                           Vec<VT, Geo<T>::LP>& rr, Vec<VT, Geo<T>::LP>& rzt) {
  constexpr int LP = Geo<T>::LP;
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
    Vec<VT, LP> a = pcg_update_row<T, VT, FUSED>(o, x, r, p, q, al, rr);
#pragma unroll
    for (int k2 = 0; k2 < KL; ++k2) {
      if (c[k2] >= t0) continue;
      const Vec<VT, LP> zz = ldv<LP>(z + (size_t)c[k2] * T + g.lane);
#pragma unroll
      for (int j = 0; j < LP; ++j) a.v[j] -= v[k2] * zz.v[j];
    }
    const int o0 = __ldg(M.L.optr + i), o1 = __ldg(M.L.optr + i + 1);
    for (int e = o0; e < o1; ++e) {
      const int cc = __ldg(M.L.ocol + e);
      if (cc >= t0) continue;
      const VT vv = M.Lh ? (VT)__half2float(M.Loh[e]) : __ldg(M.L.oval + e);
      const Vec<VT, LP> zz = ldv<LP>(z + (size_t)cc * T + g.lane);
#pragma unroll
      for (int j = 0; j < LP; ++j) a.v[j] -= vv * zz.v[j];
    }
    stv<LP>(s + (size_t)k * T + g.lane, a);
  }
  __syncthreads();
  // (b) y_t = X rhs: X_kj = xc[j nt + k], zero above the diagonal; a warp's
  // rows k are consecutive, so it stops at the diagonal of its last row
  Vec<VT, LP> y[NPT];
#pragma unroll
  for (int m = 0; m < NPT; ++m) {
    const int k = g.rs + m * RPS;
    const int jend = min(nt, __shfl_sync(0xffffffffu, k, 31) + 1);  // every lane takes part
    y[m] = vzero<VT, LP>();
    if (k < nt) {
      const VT* col = M.xc + k;
#pragma unroll 4
      for (int j = 0; j < jend; ++j) {
        const VT xv = __ldg(col + (size_t)j * nt);
        const Vec<VT, LP> sv = ldv<LP>(s + (size_t)j * T + g.lane);
#pragma unroll
        for (int l = 0; l < LP; ++l) y[m].v[l] += xv * sv.v[l];
      }
    }
  }
  __syncthreads();
#pragma unroll
  for (int m = 0; m < NPT; ++m) {
    const int k = g.rs + m * RPS;
    if (k < nt) stv<LP>(s + (size_t)k * T + g.lane, y[m]);
  }
  __syncthreads();
  // (c) z_t = X^T y_t: X_ik = xr[i nt + k], zero for i < k; a warp starts at
  // the diagonal of its first row
#pragma unroll
  for (int m = 0; m < NPT; ++m) {
    const int k = g.rs + m * RPS;
    const int ibeg = __shfl_sync(0xffffffffu, k, 0);
    if (k >= nt) continue;
    const VT* col = M.xr + k;
    Vec<VT, LP> a = vzero<VT, LP>();
#pragma unroll 4
    for (int i = ibeg; i < nt; ++i) {
      const VT xv = __ldg(col + (size_t)i * nt);
      const Vec<VT, LP> sv = ldv<LP>(s + (size_t)i * T + g.lane);
#pragma unroll
      for (int l = 0; l < LP; ++l) a.v[l] += xv * sv.v[l];
    }
    const size_t o = (size_t)(t0 + k) * T + g.lane;
    stv<LP>(z + o, a);
    const Vec<VT, LP> ri = ldv<LP>(r + o);
#pragma unroll
    for (int l = 0; l < LP; ++l) rzt.v[l] += ri.v[l] * a.v[l];
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
__device__ GPCG_LOOP_INLINE Vec<VT, Geo<T>::LP> fwd_pass(
    const DevMatT<VT>& M, VT* __restrict__ x, VT* __restrict__ r, const VT* __restrict__ p,
    const VT* __restrict__ q, VT* __restrict__ z, const Vec<VT, Geo<T>::LP>& al, VT* zt,
    Vec<VT, Geo<T>::LP>& rzt, const Ext<T, VT>* X = nullptr) {
  constexpr int LP = Geo<T>::LP;
  const Geo<T> g;
  constexpr int RPS = Geo<T>::RPS;
  Vec<VT, LP> rr = vzero<VT, LP>();
  ext_update<T, VT, FUSED>(M, X, x, r, p, q, z, al, rr, rzt);
  const int nl = M.tail_lev;
  int r0 = 0, r1 = 0, pf = -1, cn[KL];
  if (nl > 0) {
    r0 = __ldg(M.lev_ptr);
    r1 = __ldg(M.lev_ptr + 1);
    // level 0: the rows without off-diagonal entries in L (a third of the
    // rows on these grids) take the update and the diagonal scaling only,
    // with nothing to gather; the next level's first row is loaded ahead
    const int r2 = nl > 1 ? __ldg(M.lev_ptr + 2) : r1;
    if (nl > 1 && r1 + g.rs < r2) {
      pf = r1 + g.rs;
      ld_cols<KL>(M.L.col + (size_t)pf * KL, cn);
    }
    for (int i = r0 + g.rs; i < r1; i += RPS) {
      const size_t o = (size_t)i * T + g.lane;
      Vec<VT, LP> a = pcg_update_row<T, VT, FUSED>(o, x, r, p, q, al, rr);
      const VT id = M.Lh ? (VT)1 : __ldg(M.inv_diag + i);
#pragma unroll
      for (int j = 0; j < LP; ++j) a.v[j] *= id;
      stv<LP>(z + o, a);
    }
    __syncthreads();
    r0 = r1;
    r1 = r2;
  }
  for (int lev = 1; lev < nl; ++lev) {
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
      Vec<VT, LP> zc[KL];
      if (M.Lh) ld_halfs<KL>(M.Lh + (size_t)i * KL, v);
      else ld_vals<KL>(M.L.val + (size_t)i * KL, v);
#pragma unroll
      for (int k = 0; k < KL; ++k) zc[k] = ldv<LP>(z + (size_t)c[k] * T + g.lane);
      // the thread's next row: in this level, else the first of the next
      const int is = (i + RPS < r1) ? i + RPS : ((lev + 1 < nl && r1 + g.rs < r2) ? r1 + g.rs : -1);
      pf = is;
      if (is >= 0) ld_cols<KL>(M.L.col + (size_t)is * KL, cn);
      Vec<VT, LP> a = pcg_update_row<T, VT, FUSED>(o, x, r, p, q, al, rr);
#pragma unroll
      for (int k = 0; k < KL; ++k)
#pragma unroll
        for (int j = 0; j < LP; ++j) a.v[j] -= v[k] * zc[k].v[j];
      const int o0 = __ldg(M.L.optr + i), o1 = __ldg(M.L.optr + i + 1);
      for (int e = o0; e < o1; ++e) {
        const VT vv = M.Lh ? (VT)__half2float(M.Loh[e]) : __ldg(M.L.oval + e);
        const Vec<VT, LP> zz = ldv<LP>(z + (size_t)__ldg(M.L.ocol + e) * T + g.lane);
#pragma unroll
        for (int j = 0; j < LP; ++j) a.v[j] -= vv * zz.v[j];
      }
      // scaled factor: unit diagonal, w = D y is what is stored
      const VT id = M.Lh ? (VT)1 : __ldg(M.inv_diag + i);
#pragma unroll
      for (int j = 0; j < LP; ++j) a.v[j] *= id;
      stv<LP>(z + o, a);
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
  if (M.tail_row0 < M.n) tail_solve<T, VT, FUSED>(M, x, r, p, q, z, al, zt, rr, rzt);
  return rr;
}

// Back substitution L^T z = y in place (z holds y on entry), over the
// backward level schedule of the rows before the tail (the tail was solved
// in fwd_pass); accumulates r.z on top of rz.  Rows and their column
// indices are loaded one row ahead across level barriers, as in fwd_pass.
template <int T, typename VT>
__device__ GPCG_LOOP_INLINE Vec<VT, Geo<T>::LP> bwd_pass(const DevMatT<VT>& M,
                                                        const VT* __restrict__ r,
                                                        VT* __restrict__ z,
                                                        Vec<VT, Geo<T>::LP> rz) {
  constexpr int LP = Geo<T>::LP;
  const Geo<T> g;
  constexpr int RPS = Geo<T>::RPS;
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
      Vec<VT, LP> zc[KU];
      if (M.Uh) ld_halfs<KU>(M.Uh + (size_t)i * KU, v);
      else ld_vals<KU>(M.U.val + (size_t)i * KU, v);
#pragma unroll
      for (int a = 0; a < KU; ++a) zc[a] = ldv<LP>(z + (size_t)c[a] * T + g.lane);
      const Vec<VT, LP> yi = ldv<LP>(z + o), ri = ldv<LP>(r + o);
      const int ks = (k + RPS < r1) ? k + RPS : ((lev + 1 < nb && r1 + g.rs < r2) ? r1 + g.rs : -1);
      pk = ks;
      if (ks >= 0) {
        pi_ = __ldg(brows + ks);
        ld_cols<KU>(M.U.col + (size_t)pi_ * KU, cn);
      }
      // scaled factor: L_s^T z = D^-2 w with a unit diagonal
      const VT pre = M.Uh ? __ldg(M.inv_d2 + i) : (VT)1;
      Vec<VT, LP> acc;
#pragma unroll
      for (int j = 0; j < LP; ++j) acc.v[j] = yi.v[j] * pre;
#pragma unroll
      for (int a = 0; a < KU; ++a)
#pragma unroll
        for (int j = 0; j < LP; ++j) acc.v[j] -= v[a] * zc[a].v[j];
      const int o0 = __ldg(M.U.optr + i), o1 = __ldg(M.U.optr + i + 1);
      for (int e = o0; e < o1; ++e) {
        const VT vv = M.Uh ? (VT)__half2float(M.Uoh[e]) : __ldg(M.U.oval + e);
        const Vec<VT, LP> zz = ldv<LP>(z + (size_t)__ldg(M.U.ocol + e) * T + g.lane);
#pragma unroll
        for (int j = 0; j < LP; ++j) acc.v[j] -= vv * zz.v[j];
      }
      const VT id = M.Uh ? (VT)1 : __ldg(M.inv_diag + i);
#pragma unroll
      for (int j = 0; j < LP; ++j) {
        acc.v[j] *= id;
        rz.v[j] += ri.v[j] * acc.v[j];
      }
      stv<LP>(z + o, acc);
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
  return rz;
}

// Jacobi: z = r / diag(B_s), the diagonal with the outage applied; a row
// whose diagonal vanishes (a bus the outage isolates) gets z = 0.
template <int T, typename VT, bool FUSED>
__device__ GPCG_LOOP_INLINE void jacobi_pass(const DevMatT<VT>& M, VT* __restrict__ x,
                                            VT* __restrict__ r, const VT* __restrict__ p,
                                            const VT* __restrict__ q, VT* __restrict__ z,
                                            const Vec<VT, Geo<T>::LP>& al,
                                            const Stamp<T, VT>& S,
                                            Vec<VT, Geo<T>::LP>& rr, Vec<VT, Geo<T>::LP>& rz,
                                            const Ext<T, VT>* X = nullptr) {
  constexpr int LP = Geo<T>::LP;
  const Geo<T> g;
  ext_update<T, VT, FUSED>(M, X, x, r, p, q, z, al, rr, rz);
  for (int i = g.rs; i < M.n; i += Geo<T>::RPS) {
    const size_t o = (size_t)i * T + g.lane;
    const Vec<VT, LP> ri = pcg_update_row<T, VT, FUSED>(o, x, r, p, q, al, rr);
    const VT dg = __ldg(M.diag + i);
    Vec<VT, LP> zi;
#pragma unroll
    for (int j = 0; j < LP; ++j) {
      const int ln = g.lane + j;
      const VT d = dg - (i == S.ra[ln] ? S.w[ln] * S.c[ln] * S.c[ln]
                                       : i == S.rb[ln] ? S.w[ln] : (VT)0);
      zi.v[j] = d > (VT)0 ? ri.v[j] / d : (VT)0;
      rz.v[j] += ri.v[j] * zi.v[j];
    }
    stv<LP>(z + o, zi);
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
  VT rrl[T];     // r.r of the last forward pass (written after r.r)
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
//
// DEFER: when, at some iteration, the residual after the step --
// ||r - alpha q||^2 = r.r - 2 alpha r.q + alpha^2 q.q, from dot products the
// SpMV pass accumulates -- meets the tolerance for every running lane, the
// solve ends there without the forward pass that would apply the step: the
// step is left in L.xalpha for the caller to apply as x + xalpha p.
template <int T, typename VT, bool DEFER = false, bool GEN = false>
__device__ GPCG_PASS_INLINE void pcg_solve(const FdpfParams& P, const DevMatT<VT>& M, LaneState<T>& L, VT* x,
                          VT* r, VT* p, VT* q, VT* z, const int* ra_, const int* rb_,
                          const double* w_, int* iters, const double* c_ = nullptr,
                          const SwitchState<T>* SW = nullptr, const int* hold = nullptr) {
  constexpr int LP = Geo<T>::LP;
  __shared__ PcgLanes<T, VT> S;
  __shared__ Stamp<T, VT> St;
  // the extension rows' block: in the kernel with extension rows only
  Ext<T, VT>* Xw = nullptr;
  if constexpr (GEN) {
    __shared__ Ext<T, VT> Xs;
    Xw = &Xs;
  }
  // right-hand side and y of the schedule's tail (lane groups: 16-byte aligned)
  __shared__ __align__(16) VT zt[TAIL_ROWS * T];
  const Geo<T> g;
  const int tid = threadIdx.x;
  const bool jac = (P.precond == PREC_JACOBI);
  // the outage's rows of the lanes that run (-1: none); the zero row that
  // padding slots point at
  if (tid < T) {
    const bool on = L.active[tid];
    St.ra[tid] = on ? ra_[tid] : -1;
    St.rb[tid] = on ? rb_[tid] : -1;
    St.w[tid] = (VT)w_[tid];
    St.c[tid] = c_ ? (VT)c_[tid] : (VT)1;
    L.xalpha[tid] = 0.0;
    if constexpr (GEN) {
      const int ne = (SW && M.xptr && on) ? SW->nx[tid] : 0;
      Xw->n[tid] = ne;
      Xw->lb[tid] = on ? L.l[tid] : -1;
      for (int s = 0; s < ne; ++s) {
        const int b = SW->xb[tid][s];
        Xw->gb[tid][s] = b;
        // the diagonal without the outaged branch's term (w c^2 at its from
        // end, w at its to end)
        VT d = M.xdiag[b];
        const VT c = c_ ? (VT)c_[tid] : (VT)1;
        if (b == L.fb[tid]) d -= (VT)w_[tid] * c * c;
        else if (b == L.tb[tid]) d -= (VT)w_[tid];
        Xw->gd[tid][s] = d;
      }
    }
  }
  if (g.rs == 0) {
    stv<LP>(p + (size_t)M.n * T + g.lane, vzero<VT, LP>());
    stv<LP>(z + (size_t)M.n * T + g.lane, vzero<VT, LP>());
  }
  __syncthreads();
  unsigned long long filt = stamp_filter<T, VT>(St);
  // lanes with extension rows: the rows coupled to them go in the filter
  bool ext = false;
  if constexpr (GEN) {
#pragma unroll 1
    for (int k = 0; k < T; ++k)
      for (int s = 0; s < Xw->n[k]; ++s) {
        const int b = Xw->gb[k][s];
        ext = true;
        const int e1 = __ldg(M.xptr + b + 1);
        for (int e = __ldg(M.xptr + b); e < e1; ++e) {
          const int rw = __ldg(M.xrow + e);
          if (rw >= 0) filt |= 1ull << (rw & 63);
        }
      }
  }
  const Ext<T, VT>* X = nullptr;
  if constexpr (GEN)
    if (ext) X = Xw;
  // islands in this tile: the SpMV then masks rows per lane
  bool islands = false;
#pragma unroll 1
  for (int k = 0; k < T; ++k) islands |= L.active[k] && L.cnt[k] > 0;
  const LaneState<T>* isl = islands ? &L : nullptr;
  Vec<VT, LP> bbp = vzero<VT, LP>(), rzp = vzero<VT, LP>(), al = vzero<VT, LP>();
  const bool tim0 = P.phase_cycles != nullptr && tid == 0;
  long long t0a = tim0 ? clock64() : 0, t0b = 0;
  if (jac) {
    jacobi_pass<T, VT, false>(M, x, r, p, q, z, al, St, bbp, rzp, X);
  } else {
    Vec<VT, LP> rzt = vzero<VT, LP>();
    bbp = fwd_pass<T, VT, false>(M, x, r, p, q, z, al, zt, rzt, X);
    if (tim0) t0b = clock64();
    rzp = bwd_pass<T, VT>(M, r, z, rzt);
  }
  if (tim0 && !jac) {
    atomicAdd(P.phase_cycles + 8 + 2 * (size_t)P.S + 1, (unsigned long long)(t0b - t0a));
    atomicAdd(P.phase_cycles + 8 + 2 * (size_t)P.S + 2, (unsigned long long)(clock64() - t0b));
  }
  const Vec<VT, LP> bb = lane_sum<T, RS_BB>(L, bbp);
  const Vec<VT, LP> rz0 = lane_sum<T, RS_RZ0>(L, rzp);
  if (g.rs == 0) {
#pragma unroll
    for (int j = 0; j < LP; ++j) {
      const int ln = g.lane + j;
      const VT b_ = bb.v[j], r_ = rz0.v[j];
      S.bb[ln] = b_;
      S.rrl[ln] = b_;  // r = b while x = 0
      S.rz[0][ln] = r_;
      S.rrmin[ln] = b_;
      S.stall[ln] = 0;
      S.brk[ln] = 0;
      S.stop[ln] = 0;
      // held lanes take no step: x stays 0
      S.pdone[ln] = !L.active[ln] || (hold && hold[ln]) || !(b_ > (VT)0) || !(r_ > (VT)0);
    }
  }
  __syncthreads();  // publishes S and the first z
  const VT tol2 = (VT)(P.inner_rtol * P.inner_rtol);
  // diagnostics (P.phase_cycles set): thread 0's SM cycles in the SpMV, the
  // forward and the backward passes of this solve, added to the three slots
  // after the per-scenario times
  const bool tim = P.phase_cycles != nullptr && tid == 0;
  unsigned long long tsub[3] = {0ull, 0ull, 0ull};
  long long tmark = 0;
#define GPCG_SUB_BEGIN() \
  if (tim) tmark = clock64();
#define GPCG_SUB_END(k) \
  if (tim) tsub[k] += (unsigned long long)(clock64() - tmark);
  int par = 0;
  Vec<VT, LP> be = vzero<VT, LP>();
  for (int it = 0; it < P.max_inner; ++it) {
    bool any = false;
#pragma unroll 1
    for (int k = 0; k < T; ++k) any |= !(S.pdone[k] | S.stop[k]);
    if (!any) break;
    // new direction p = mask(z) + beta p and q = B_s p in one pass
    Vec<VT, LP> rqp = vzero<VT, LP>(), qqp = vzero<VT, LP>();
    GPCG_SUB_BEGIN();
    const Vec<VT, LP> pqp = spmv_pass<T, VT, true>(
        M, z, p, q, St, filt, be, it == 0, isl, (DEFER && Geo<T>::TPR == 1) ? r : nullptr, &rqp,
        &qqp, X);
    GPCG_SUB_END(0);
    Vec<VT, LP> pq = pqp, rq = rqp, qq = qqp;
    if constexpr (DEFER && Geo<T>::TPR == 1) lane_sum3<T, RS_PQ, RS_RQ, RS_QQ>(L, pq, rq, qq);
    else pq = lane_sum<T, RS_PQ>(L, pqp);
    int bk = 0;   // lanes whose p.Bp broke down: keep the current iterate
    int pok = 0;  // lanes whose predicted residual after the step converged
#pragma unroll
    for (int j = 0; j < LP; ++j) {
      const int ln = g.lane + j;
      al.v[j] = (VT)0;
      if (!(S.pdone[ln] | S.stop[ln])) {
        if (pq.v[j] > (VT)0 && isfinite(pq.v[j])) al.v[j] = S.rz[par][ln] / pq.v[j];
        else bk |= 1 << j;
      }
    }
    if constexpr (DEFER && Geo<T>::TPR == 1) {
      // a thread holds every lane of the tile: when each running lane meets
      // the tolerance with this step, every thread sees it, and the solve
      // ends here with the step deferred to the caller
      // A lane converges on the predicted residual whether or not the
      // step is deferred, so that its iterates do not depend on the
      // scenarios it shares a tile with.
      bool fin = true, run = false;
#pragma unroll
      for (int j = 0; j < LP; ++j) {
        const int ln = g.lane + j;
        if (S.pdone[ln] | S.stop[ln]) continue;
        run = true;
        if ((bk >> j) & 1) { fin = false; continue; }
        const VT pred = S.rrl[ln] - al.v[j] * ((VT)2 * rq.v[j] - al.v[j] * qq.v[j]);
        if (pred <= tol2 * S.bb[ln]) pok |= 1 << j;
        else fin = false;
      }
      if (run && fin) {
        if (g.rs == 0)
#pragma unroll
          for (int j = 0; j < LP; ++j) {
            const int ln = g.lane + j;
            if (S.pdone[ln] | S.stop[ln]) continue;
            L.xalpha[ln] = (double)al.v[j];
            iters[ln] += 1;
          }
        break;  // the closing barrier publishes xalpha and the counts
      }
    }
    if (g.rs == 0)
#pragma unroll
      for (int j = 0; j < LP; ++j)
        if ((bk >> j) & 1) S.brk[g.lane + j] = 1;
    Vec<VT, LP> rrp = vzero<VT, LP>(), rzn = vzero<VT, LP>();
    GPCG_SUB_BEGIN();
    if (jac) {
      jacobi_pass<T, VT, true>(M, x, r, p, q, z, al, St, rrp, rzn, X);
    } else {
      rrp = fwd_pass<T, VT, true>(M, x, r, p, q, z, al, zt, rzn, X);  // rzn: the tail's r.z
    }
    GPCG_SUB_END(1);
    const Vec<VT, LP> rr = lane_sum<T, RS_RR>(L, rrp);
    if (g.rs == 0) {
#pragma unroll
      for (int j = 0; j < LP; ++j) {
        const int ln = g.lane + j;
        const VT v = rr.v[j];
        if (S.pdone[ln] | S.stop[ln]) continue;
        if (S.brk[ln]) { S.pdone[ln] = 1; continue; }
        iters[ln] += 1;
        S.rrl[ln] = v;
        // converged; or stagnated at the rounding floor of VT (no 0.1 % gain
        // in STALL_ITERS iterations); or growing away from the best residual
        if (v < (VT)0.999 * S.rrmin[ln]) { S.rrmin[ln] = v; S.stall[ln] = 0; }
        else S.stall[ln] += 1;
        if (((pok >> j) & 1) || v <= tol2 * S.bb[ln] || !isfinite(v) ||
            S.stall[ln] >= STALL_ITERS ||
            v > (VT)1e4 * S.rrmin[ln])
          S.pdone[ln] = 1;
      }
    }
    __syncthreads();
    // lanes still running, read before S.stop is next written (after r.z)
    int go = 0;
#pragma unroll
    for (int j = 0; j < LP; ++j) go |= (!(S.pdone[g.lane + j] | S.stop[g.lane + j])) << j;
    any = false;
#pragma unroll 1
    for (int k = 0; k < T; ++k) any |= !(S.pdone[k] | S.stop[k]);
    if (!any) break;
    GPCG_SUB_BEGIN();
    if (!jac) rzn = bwd_pass<T, VT>(M, r, z, rzn);
    GPCG_SUB_END(2);
    const Vec<VT, LP> rz = lane_sum<T, RS_RZ>(L, rzn);
#pragma unroll
    for (int j = 0; j < LP; ++j)
      be.v[j] = ((go >> j) & 1) ? rz.v[j] / S.rz[par][g.lane + j] : (VT)0;
    if (g.rs == 0) {
#pragma unroll
      for (int j = 0; j < LP; ++j) {
        const int ln = g.lane + j;
        if (!((go >> j) & 1)) continue;
        const VT v = rz.v[j];
        S.rz[par ^ 1][ln] = v;
        if (!(v > (VT)0)) S.stop[ln] = 1;
      }
    }
    __syncthreads();  // publishes S.rz, S.stop and z
    par ^= 1;
  }
  if (tim)
    for (int k = 0; k < 3; ++k) atomicAdd(P.phase_cycles + 8 + 2 * (size_t)P.S + k, tsub[k]);
#undef GPCG_SUB_BEGIN
#undef GPCG_SUB_END
  __syncthreads();
}


}  // namespace gpcg
