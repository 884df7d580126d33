// The persistent N-1 kernel: one CTA owns a tile of T scenarios and runs the
// whole fast-decoupled power flow of that tile (Sec. III.B eqs. (4)-(5),
// Sec. IV) without leaving the kernel, then takes the next tile from a
// device-side counter.  Vectors live in global memory as [row][T] per CTA
// slot, so a row touches one contiguous chunk across the tile's scenarios;
// each thread owns two adjacent scenario lanes of a row.  Tiles are
// independent: the only inter-CTA traffic is the atomic tile counter, and no
// CTA ever waits on another.
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
//
// Every sparse row is read through a padded descriptor (ELL): its column
// indices and values sit at fixed offsets, so a thread issues all of a row's
// gathers at once instead of walking a row pointer first.
//
// GEN: the kernel with B'' extension rows -- for generator outages (the
// tripped generator's bus) and for grids whose PV generators have reactive
// limits (buses switched to PQ at a limit); the kernel for branch outages
// without limits is built without that code.
#pragma once
#include <math.h>
#include "common.cuh"
#include "fdpf.h"
#include "fdpf_ops.cuh"

namespace gpcg {

// 1 / |V| of the rectangular voltage e + jf in the inner solve's precision.
// It only scales inner-solve quantities -- the right-hand sides dP/|V| and
// dQ/|V| and the relative step dV/|V| -- which the outer FP64 loop refines,
// so the FP32 form's few-ulp rounding moves no converged state.  The state
// keeps no |V| of its own: e + jf is the state.
template <typename VT>
__device__ __forceinline__ VT inv_vmag(double e, double f);
template <>
__device__ __forceinline__ float inv_vmag<float>(double e, double f) {
  const float a = to_f32(e), b = to_f32(f);
  return rsqrtf(fmaf(a, a, b * b));
}
template <>
__device__ __forceinline__ double inv_vmag<double>(double e, double f) {
  return 1.0 / sqrt(fma(e, e, f * f));
}

// ------------------------------------------------------------ mismatch
// The rectangular voltages e + jf of a slot are stored interleaved,
// [bus][lane][e, f], so one 16-byte load gives a lane's (e, f) and a thread's
// two lanes sit in 32 contiguous bytes.
template <int T>
__device__ __forceinline__ size_t ef_at(int bus, int lane) {
  return ((size_t)bus * T + lane) * 2;
}

// The neighbour slots of bus i (slot-major adjacency).
__device__ __forceinline__ void ld_nbrs(const DevGrid& G, int i, int (&nb)[KG]) {
#pragma unroll
  for (int a = 0; a < KG; ++a) nb[a] = __ldg(G.adj_nbr + (size_t)a * G.n + i);
}

// I_i = sum_j Y_ij V_j at bus i for lane ln, the lane's outaged branch left
// out (off the diagonal and its share of it), summed like mismatch_pass.
template <int T>
__device__ __forceinline__ double2 bus_current(const DevGrid& G, const LaneState<T>& L,
                                               const double* __restrict__ EF, int i, int ln) {
  double re = 0.0, im = 0.0;
  const int br = L.l[ln];
  const int deg = __ldg(G.adj_deg + i);
  for (int a = 0; a < deg; ++a) {
    if (__ldg(G.adj_brl + (size_t)a * G.n + i) == br) continue;
    const int j = __ldg(G.adj_nbr + (size_t)a * G.n + i);
    const double gv = __ldg(G.adj_g + (size_t)a * G.n + i), bv = __ldg(G.adj_b + (size_t)a * G.n + i);
    const double2 u = *reinterpret_cast<const double2*>(EF + ef_at<T>(j, ln));
    re = fma(-gv, u.x, fma(bv, u.y, re));
    im = fma(-gv, u.y, fma(-bv, u.x, im));
  }
  const int o1 = __ldg(G.adj_optr + i + 1);
  for (int e = __ldg(G.adj_optr + i); e < o1; ++e) {
    if (__ldg(G.adj_obr + e) == br) continue;
    const int j = __ldg(G.adj_onbr + e);
    const double gw = __ldg(G.adj_og + e), bw = __ldg(G.adj_ob + e);
    const double2 u = *reinterpret_cast<const double2*>(EF + ef_at<T>(j, ln));
    re = fma(-gw, u.x, fma(bw, u.y, re));
    im = fma(-gw, u.y, fma(-bw, u.x, im));
  }
  const double2 v = *reinterpret_cast<const double2*>(EF + ef_at<T>(i, ln));
  double Gii = __ldg(G.Gii + i), Bii = __ldg(G.Bii + i);
  if (i == L.fb[ln] || i == L.tb[ln]) {
    const double c2 = i == L.fb[ln] ? L.cl[ln] * L.cl[ln] : 1.0;
    Gii -= c2 * L.gl[ln];
    Bii -= c2 * L.bl[ln];
  }
  return make_double2(fma(Gii, v.x, fma(-Bii, v.y, re)), fma(Gii, v.y, fma(Bii, v.x, im)));
}

// dP_i, dQ_i of eqs. (1)-(3) from the rectangular voltages:
// I = Y V, P + jQ = V conj(I).  The outaged branch is left out of the
// neighbour sum and of the diagonal.  WITH_P: the P half-step (writes
// dP/V into the B' right-hand side and tracks max|dP| and max|dQ| for the
// convergence test); otherwise writes dQ/V into the B'' right-hand side.
// A thread takes a bus and its lanes two at a time: each neighbour's
// admittance and the pair's voltages are loaded once for the two lanes.
template <int T, typename VT, bool WITH_P, bool GEN>
__device__ GPCG_PASS_INLINE void mismatch_pass(const FdpfParams& P, const DevMatT<VT>& MP,
                                               const DevMatT<VT>& MQ, LaneState<T>& L,
                                               const double* __restrict__ EF,
                                               VT* __restrict__ rhs,
                                               Vec<unsigned long long, Geo<T>::LP>& errP_,
                                               Vec<unsigned long long, Geo<T>::LP>& errQ_,
                                               SwitchState<T>* SW = nullptr) {
  constexpr int LP = Geo<T>::LP;
  const Geo<T> g;
  const DevGrid& G = P.G;
  // the running maxima in registers through the row loop (the caller's
  // copies sit in its local memory)
  Vec<unsigned long long, LP> errP = errP_, errQ = errQ_;
  // rows are visited in order of bus degree, so the threads of a warp run
  // neighbour loops of equal length and no FP64 work is spent on padding
  const int nrows = WITH_P ? G.n - 1 : MQ.n;
  const int32_t* order = WITH_P ? P.mis_order : P.misq_order;
  int kn = 0, nbn[KG];
  if (g.rs < nrows) {
    kn = __ldg(order + g.rs);
    ld_nbrs(G, WITH_P ? kn : __ldg(MQ.bus_of_row + kn), nbn);
  }
  for (int kk = g.rs; kk < nrows; kk += Geo<T>::RPS) {
    const int k = kn;
    int nb[KG];
#pragma unroll
    for (int a = 0; a < KG; ++a) nb[a] = nbn[a];
    if (kk + Geo<T>::RPS < nrows) {
      kn = __ldg(order + kk + Geo<T>::RPS);
      ld_nbrs(G, WITH_P ? kn : __ldg(MQ.bus_of_row + kn), nbn);
    }
    const int i = WITH_P ? k : __ldg(MQ.bus_of_row + k);
    const int pr = __ldg(G.pre + i);
    const int deg = __ldg(G.adj_deg + i);
    Vec<VT, LP> out = vzero<VT, LP>();
#pragma unroll 1
    for (int jp = 0; jp < LP; jp += 2) {
      const int l0 = g.lane + jp, l1 = l0 + 1;
      const bool on0 = L.active[l0] && !in_island(pr, L.lo[l0], L.cnt[l0]);
      const bool on1 = L.active[l1] && !in_island(pr, L.lo[l1], L.cnt[l1]);
      if (!(on0 || on1)) continue;
      // a lane's first P half-step away from the ends of its outaged branch:
      // the base-case mismatch holds (the state is the base case there)
      bool w0 = false, w1 = false;
      if (WITH_P && P.r0P) {
        w0 = on0 && L.outer[l0] == 0 && i != L.fb[l0] && i != L.tb[l0];
        w1 = on1 && L.outer[l1] == 0 && i != L.fb[l1] && i != L.tb[l1];
      }
      const bool n0 = on0 && !w0, n1 = on1 && !w1;  // lanes that sum the neighbours
      // -sum over the neighbours of Y_ij V_j, both lanes of the pair
      double re0 = 0.0, im0 = 0.0, re1 = 0.0, im1 = 0.0;
      if (n0 || n1) {
#pragma unroll
      for (int a0 = 0; a0 < KG; a0 += MIS_GROUP) {
        double2 u0[MIS_GROUP], u1[MIS_GROUP];
        double gv[MIS_GROUP], bv[MIS_GROUP];
#pragma unroll
        for (int a = 0; a < MIS_GROUP; ++a)
          if (a0 + a < deg) {
            const double2* q2 = reinterpret_cast<const double2*>(EF + ef_at<T>(nb[a0 + a], l0));
            u0[a] = q2[0];
            u1[a] = q2[1];
            gv[a] = __ldg(G.adj_g + (size_t)(a0 + a) * G.n + i);
            bv[a] = __ldg(G.adj_b + (size_t)(a0 + a) * G.n + i);
          }
#pragma unroll
        for (int a = 0; a < MIS_GROUP; ++a)
          if (a0 + a < deg) {
            if (n0) {
              re0 = fma(-gv[a], u0[a].x, fma(bv[a], u0[a].y, re0));
              im0 = fma(-gv[a], u0[a].y, fma(-bv[a], u0[a].x, im0));
            }
            if (n1) {
              re1 = fma(-gv[a], u1[a].x, fma(bv[a], u1[a].y, re1));
              im1 = fma(-gv[a], u1[a].y, fma(-bv[a], u1[a].x, im1));
            }
          }
      }
      const int o0 = __ldg(G.adj_optr + i), o1 = __ldg(G.adj_optr + i + 1);
      for (int e = o0; e < o1; ++e) {
        const int jn = __ldg(G.adj_onbr + e);
        const double gw = __ldg(G.adj_og + e), bw = __ldg(G.adj_ob + e);
        const double2* q2 = reinterpret_cast<const double2*>(EF + ef_at<T>(jn, l0));
        const double2 v0 = q2[0], v1 = q2[1];
        if (n0) {
          re0 = fma(-gw, v0.x, fma(bw, v0.y, re0));
          im0 = fma(-gw, v0.y, fma(-bw, v0.x, im0));
        }
        if (n1) {
          re1 = fma(-gw, v1.x, fma(bw, v1.y, re1));
          im1 = fma(-gw, v1.y, fma(-bw, v1.x, im1));
        }
      }
      // the outaged branch's term back out at its two end buses
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        const int ln = j ? l1 : l0;
        if (!(j ? n1 : n0) || (i != L.fb[ln] && i != L.tb[ln])) continue;
        const int e = i == L.fb[ln] ? 0 : 1;
        const double2 v = *reinterpret_cast<const double2*>(
            EF + ef_at<T>(e ? L.fb[ln] : L.tb[ln], ln));
        const double go = L.og[ln][e], bo = L.ob[ln][e];
        double& re = j ? re1 : re0;
        double& im = j ? im1 : im0;
        re -= fma(-go, v.x, bo * v.y);
        im -= fma(-go, v.y, -bo * v.x);
      }
      }
      // own voltage, the diagonal term and the mismatch of each lane
      const double2* own = reinterpret_cast<const double2*>(EF + ef_at<T>(i, l0));
      const double2 ev0 = own[0], ev1 = own[1];
      const int bt = G.bus_type[i];
      const double Gii = __ldg(G.Gii + i), Bii = __ldg(G.Bii + i), qs = __ldg(G.Q_sched + i);
      double Ps = 0.0, pg = 0.0, Pgr = 0.0;
      if (WITH_P) {
        Ps = __ldg(G.P_sched + i);
        if (bt == 1) {
          Pgr = __ldg(G.P_gen + i);
          pg = fmax(Pgr, 0.0);  // generators with P_gen > 0 take it
        }
      }
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        if (!(j ? on1 : on0)) continue;
        const int ln = j ? l1 : l0;
        // a tripped generator's bus keeps only its load and takes no share
        // of the re-dispatch; a bus with an extension row (that one, or a PV
        // bus held at a reactive limit) is PQ with the injection qx
        const bool tr = GEN && WITH_P && i == L.gb[ln];
        const double pgl = tr ? 0.0 : pg;
        bool xe = false;
        double qx = qs;
        int xr = -1;  // the bus's extension row
        if (GEN && WITH_P)
          for (int s = 0; s < SW->nx[ln]; ++s)
            if (SW->xb[ln][s] == i) { xe = true; qx = SW->xq[ln][s]; xr = s; }
        if (j ? w1 : w0) {
          // the base-case state here: the base case is within the reactive limits
          const double dP = fma(L.coef[ln], pgl, __ldg(P.r0P + i)) - (tr ? Pgr : 0.0);
          upd_max_bits(errP.v[jp + j], dP);
          if (bt == 0 || xe) {
            const double q0 = __ldg(P.r0Q + i);
            upd_max_bits(errQ.v[jp + j], xe ? q0 + (qx - qs) : q0);
          }
          out.v[jp + j] = to_vt<VT>(dP) * (j ? inv_vmag<VT>(ev1.x, ev1.y)
                                             : inv_vmag<VT>(ev0.x, ev0.y));
          continue;
        }
        const double ei = j ? ev1.x : ev0.x, fi = j ? ev1.y : ev0.y;
        const VT iv = inv_vmag<VT>(ei, fi);
        double Gd = Gii, Bd = Bii;
        if (i == L.fb[ln] || i == L.tb[ln]) {  // the outaged branch's share
          const double c2 = i == L.fb[ln] ? L.cl[ln] * L.cl[ln] : 1.0;
          Gd -= c2 * L.gl[ln];
          Bd -= c2 * L.bl[ln];
        }
        // I_i = Y_ii V_i + sum_j Y_ij V_j
        const double re = fma(Gd, ei, fma(-Bd, fi, j ? re1 : re0));
        const double im = fma(Gd, fi, fma(Bd, ei, j ? im1 : im0));
        // dQ = Q_sched - Im(V_i conj(I_i)); dP = P_sched + re-dispatch - Re(...)
        VT res;
        if (WITH_P) {
          const double dP =
              fma(-ei, re, fma(-fi, im, fma(L.coef[ln], pgl, tr ? Ps - Pgr : Ps)));
          upd_max_bits(errP.v[jp + j], dP);
          if (bt == 0 || xe) upd_max_bits(errQ.v[jp + j], fma(-fi, re, fma(ei, im, qx)));
          if (GEN && bt == 1 && !xe && G.qmax) {
            // a PV generator's output Q(V) - Q_sched = -dQ against its limits:
            // a violation is a candidate for the switch to PQ at that limit
            const double qg = -fma(-fi, re, fma(ei, im, qs));
            const double hi = __ldg(G.qmax + i), lo = __ldg(G.qmin + i);
            if (qg > hi || qg < lo) {
              const int at = atomicAdd(&SW->nc[ln], 1);
              if (at < KX) {
                SW->cb[ln][at] = i;
                SW->cq[ln][at] = qs + (qg > hi ? hi : lo);
                SW->cs[ln][at] = qg > hi ? 1 : -1;
              }
            }
          }
          if (GEN && xe && SW->xs[ln][xr] != 0) {
            // a generator held at Q_max whose |V| is above its set point (at
            // Q_min, below) can hold the set point again: back to PV
            const double vm = sqrt(fma(ei, ei, fi * fi)), vs = __ldg(G.V_set + i);
            const int side = SW->xs[ln][xr];
            if ((side > 0 && vm > vs) || (side < 0 && vm < vs))
              atomicOr(&SW->bk[ln], 1u << xr);
          }
          res = to_vt<VT>(dP) * iv;
        } else {
          const double dQ = fma(-fi, re, fma(ei, im, qs));
          upd_max_bits(errQ.v[jp + j], dQ);  // decides whether the Q step is taken
          res = to_vt<VT>(dQ) * iv;
        }
        out.v[jp + j] = res;
      }
    }
    if (WITH_P) stv<LP>(rhs + (size_t)__ldg(MP.row_of_bus + i) * T + g.lane, out);
    else stv<LP>(rhs + (size_t)k * T + g.lane, out);
  }
  // the B'' extension rows: dQ/V at their buses, with the reactive
  // injection each holds
  if (GEN && !WITH_P && MQ.xptr && g.rs == 0)
#pragma unroll
    for (int j = 0; j < LP; ++j) {
      const int ln = g.lane + j;
      if (!L.active[ln]) continue;
      for (int s = 0; s < SW->nx[ln]; ++s) {
        const int b = SW->xb[ln][s];
        const double2 I = bus_current<T>(G, L, EF, b, ln);
        const double2 v = *reinterpret_cast<const double2*>(EF + ef_at<T>(b, ln));
        const double dQ = fma(-v.y, I.x, fma(v.x, I.y, SW->xq[ln][s]));
        upd_max_bits(errQ.v[j], dQ);
        rhs[(size_t)(MQ.n + 1 + s) * T + ln] = to_vt<VT>(dQ) * inv_vmag<VT>(v.x, v.y);
      }
    }
  errP_ = errP;
  errQ_ = errQ;
}

// (e, f) rotated through the angle d, in FP64:
//   e' = e cos d - f sin d = e - (e a + f b),  f' = f - (f a - e b),
// with a = 1 - cos d and b = sin d.  For |d| <= 0.02 both come from their
// Taylor series in u = d^2 (a = u/2 - u^2/24 + u^3/720, b = d - d^3/6 +
// d^5/120; the first dropped terms are below 3e-16 there), larger steps call
// sincos.  The rotation is exact to FP64 rounding, so the state (e, f) stays
// at the angle theta and modulus |V| that the kernel reports: the state whose
// mismatch the convergence test evaluated is the state that is returned.
__device__ __forceinline__ void rotate_ef(double d, double& e, double& f) {
  double a, b;
  if (fabs(d) <= 0.02) {
    const double u = d * d;
    a = u * fma(u, fma(u, 1.0 / 720.0, -1.0 / 24.0), 0.5);
    b = fma(d * u, fma(u, 1.0 / 120.0, -1.0 / 6.0), d);
  } else {
    double c;
    sincos(d, &b, &c);
    a = 1.0 - c;
  }
  const double e0 = e;
  e = fma(-e0, a, fma(-f, b, e0));
  f = fma(-f, a, fma(e0, b, f));
}

// The relative step r = dV / |V| of a |V| update at the voltage e + jf:
// FP32 vectors take it in FP32 (the step is an inner-solve iterate that the
// outer FP64 loop refines; r is then exact as an FP64 number), FP64 vectors
// in FP64.
template <typename VT>
__device__ __forceinline__ double v_ratio(VT dv, double e, double f) {
  return to_f64(dv * inv_vmag<VT>(e, f));
}

// theta += dtheta (P half-step) or |V| += dV (Q half-step) on the matrix's
// rows, as moves of the rectangular voltage: (e, f) rotated through dtheta
// (theta kept beside it), or e and f both scaled by 1 + dV/|V|, so that
// e + jf = |V| exp(j theta) holds to FP64 rounding; lanes two at a time.
template <int T, typename VT, bool IS_P, bool GEN>
__device__ GPCG_LOOP_INLINE void update_pass(const DevMatT<VT>& M, LaneState<T>& L,
                                             const VT* __restrict__ x,
                                             const VT* __restrict__ p, double* th,
                                             double* EF, const SwitchState<T>* SW = nullptr) {
  constexpr int LP = Geo<T>::LP;
  const Geo<T> g;
  bool any = false;
#pragma unroll
  for (int j = 0; j < LP; ++j) any |= L.active[g.lane + j] != 0;
  if (!any) return;
  for (int k = g.rs; k < M.n; k += Geo<T>::RPS) {
    const int pr = __ldg(M.pre_of_row + k);
    const int i = __ldg(M.bus_of_row + k);
#pragma unroll 1
    for (int jp = 0; jp < LP; jp += 2) {
      const int l0 = g.lane + jp, l1 = l0 + 1;
      const bool on0 = L.active[l0] && !in_island(pr, L.lo[l0], L.cnt[l0]);
      const bool on1 = L.active[l1] && !in_island(pr, L.lo[l1], L.cnt[l1]);
      if (!on0 && !on1) continue;
      const size_t o = (size_t)i * T + l0;
      Pair<VT> dx = ld2(x + (size_t)k * T + l0);
      // the inner solve's deferred last step, x += alpha p
      const VT xa0 = (VT)L.xalpha[l0], xa1 = (VT)L.xalpha[l1];
      if (xa0 != (VT)0 || xa1 != (VT)0) {
        const Pair<VT> pv = ld2(p + (size_t)k * T + l0);
        dx.a = fma(xa0, pv.a, dx.a);  // as the solve's own step would take it
        dx.b = fma(xa1, pv.b, dx.b);
      }
      double2* ef = reinterpret_cast<double2*>(EF + ef_at<T>(i, l0));
      double2 u0 = ef[0], u1 = ef[1];
      if (IS_P) {
        Pair<double> t = ld2(th + o);
        if (on0) {
          const double d = to_f64(dx.a);
          t.a += d;
          rotate_ef(d, u0.x, u0.y);
        }
        if (on1) {
          const double d = to_f64(dx.b);
          t.b += d;
          rotate_ef(d, u1.x, u1.y);
        }
        st2(th + o, t);
      } else {
        if (on0) {
          const double r = v_ratio<VT>(dx.a, u0.x, u0.y);
          u0 = make_double2(fma(u0.x, r, u0.x), fma(u0.y, r, u0.y));
        }
        if (on1) {
          const double r = v_ratio<VT>(dx.b, u1.x, u1.y);
          u1 = make_double2(fma(u1.x, r, u1.x), fma(u1.y, r, u1.y));
        }
      }
      ef[0] = u0;
      ef[1] = u1;
    }
  }
  // |V| of the extension rows' buses
  if (GEN && !IS_P && M.xptr && g.rs == 0)
#pragma unroll
    for (int j = 0; j < LP; ++j)
    for (int s = 0; s < SW->nx[g.lane + j]; ++s) {
      const int ln = g.lane + j;
      if (!L.active[ln]) continue;
      const int b = SW->xb[ln][s];
      const size_t oe = (size_t)(M.n + 1 + s) * T + ln;
      VT dx = x[oe];
      const VT xa = (VT)L.xalpha[ln];
      if (xa != (VT)0) dx = fma(xa, p[oe], dx);
      double2* ef = reinterpret_cast<double2*>(EF + ef_at<T>(b, ln));
      const double2 u = ef[0];
      const double r = v_ratio<VT>(dx, u.x, u.y);
      ef[0] = make_double2(fma(u.x, r, u.x), fma(u.y, r, u.y));
    }
}

// ------------------------------------------------------------ the kernel
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Scenario info of a lane taking scenario s (thread `ln`, one per lane).
template <int T, typename VT>
__device__ __forceinline__ void setup_lane(const FdpfParams& P, const DevMatT<VT>& MP,
                                           const DevMatT<VT>& MQ, LaneState<T>& L, int ln,
                                           SwitchState<T>* SW) {
  const DevGrid& G = P.G;
  const int s = L.scen[ln];
  const int l = P.sc.outage[s];
  L.l[ln] = l;
  L.fb[ln] = l >= 0 ? G.f[l] : -1;
  L.tb[ln] = l >= 0 ? G.t[l] : -1;
  L.lo[ln] = P.sc.isl_lo[s];
  L.cnt[ln] = P.sc.isl_cnt[s];
  L.coef[ln] = P.sc.coef[s];
  L.nogen[ln] = P.sc.no_gen[s];
  L.raP[ln] = l >= 0 ? MP.row_of_bus[G.f[l]] : -1;
  L.rbP[ln] = l >= 0 ? MP.row_of_bus[G.t[l]] : -1;
  L.raQ[ln] = l >= 0 ? MQ.row_of_bus[G.f[l]] : -1;
  L.rbQ[ln] = l >= 0 ? MQ.row_of_bus[G.t[l]] : -1;
  L.wP[ln] = l >= 0 ? MP.w[l] : 0.0;
  L.wQ[ln] = l >= 0 ? MQ.w[l] : 0.0;
  L.gl[ln] = l >= 0 ? G.g[l] : 0.0;
  L.bl[ln] = l >= 0 ? G.by[l] + 0.5 * G.b_sh[l] : 0.0;
  L.cl[ln] = l >= 0 ? G.cf[l] : 1.0;
  // the adjacency entries of the outaged branch at its two ends: the
  // mismatch sums every neighbour and takes these back out
  for (int e = 0; e < 2; ++e) {
    L.og[ln][e] = 0.0;
    L.ob[ln][e] = 0.0;
    const int x = e ? L.tb[ln] : L.fb[ln];
    if (x < 0) continue;
    bool hit = false;
    const int dg = G.adj_deg[x];
    for (int a = 0; a < dg && !hit; ++a)
      if (G.adj_brl[(size_t)a * G.n + x] == l) {
        L.og[ln][e] = G.adj_g[(size_t)a * G.n + x];
        L.ob[ln][e] = G.adj_b[(size_t)a * G.n + x];
        hit = true;
      }
    for (int k = G.adj_optr[x]; k < G.adj_optr[x + 1] && !hit; ++k)
      if (G.adj_obr[k] == l) {
        L.og[ln][e] = G.adj_og[k];
        L.ob[ln][e] = G.adj_ob[k];
        hit = true;
      }
  }
  L.gb[ln] = P.sc.gen_bus ? P.sc.gen_bus[s] : -1;
  // the tripped generator's bus is the lane's first extension row, with its
  // load's reactive injection
  if (SW) {
    SW->nx[ln] = L.gb[ln] >= 0 ? 1 : 0;
    if (L.gb[ln] >= 0) {
      SW->xb[ln][0] = L.gb[ln];
      SW->xq[ln][0] = G.Q_sched[L.gb[ln]];
      SW->xs[ln][0] = 0;
    }
    SW->nc[ln] = 0;
    SW->bk[ln] = 0u;
    SW->skip[ln] = 0;
  }
  L.active[ln] = 1;
  L.outer[ln] = 0;
  L.inP[ln] = 0;
  L.inQ[ln] = 0;
  L.status[ln] = 0;
  L.err[ln] = 0.0;
  L.best[ln] = INFINITY;
}

// Warm start (Sec. III.B) of the lanes flagged `fresh`: the base-case state,
// zero on islanded buses.  Other lanes keep their state.
template <int T>
__device__ GPCG_PASS_INLINE void init_pass(const FdpfParams& P, LaneState<T>& L, double* th,
                                           double* EF) {
  constexpr int LP = Geo<T>::LP;
  const Geo<T> g;
  const DevGrid& G = P.G;
  int fresh = 0;
#pragma unroll
  for (int j = 0; j < LP; ++j) fresh |= (L.fresh[g.lane + j] != 0) << j;
  if (!fresh) return;
  for (int i = g.rs; i < G.n; i += Geo<T>::RPS) {
    double t0, v0, c0, s0;
    if (P.flat_start) { t0 = 0.0; v0 = G.V_set[i]; c0 = 1.0; s0 = 0.0; }
    else { t0 = P.th0[i]; v0 = P.V0[i]; c0 = P.c0[i]; s0 = P.s0[i]; }
    const int pr = G.pre[i];
#pragma unroll
    for (int j = 0; j < LP; ++j) {
      if (!((fresh >> j) & 1)) continue;
      const int ln = g.lane + j;
      const size_t o = (size_t)i * T + ln;
      const bool isl = in_island(pr, L.lo[ln], L.cnt[ln]);
      th[o] = isl ? 0.0 : t0;
      reinterpret_cast<double2*>(EF + ef_at<T>(i, ln))[0] =
          isl ? make_double2(0.0, 0.0) : make_double2(v0 * c0, v0 * s0);
    }
  }
}

// Outputs of the lanes flagged `done`: state, branch flows and loading
// (Sec. I: overload screening), status and iteration counts.
template <int T>
__device__ GPCG_PASS_INLINE void retire_pass(const FdpfParams& P, LaneState<T>& L,
                                             const double* th, const double* EF) {
  constexpr int LP = Geo<T>::LP;
  const Geo<T> g;
  const DevGrid& G = P.G;
  int dn = 0;
#pragma unroll
  for (int j = 0; j < LP; ++j) dn |= (L.done[g.lane + j] != 0) << j;
  if ((P.out_theta || P.out_vm) && dn) {
    for (int iu = g.rs; iu < G.n; iu += Geo<T>::RPS) {
      const int i = P.out_bus_map ? __ldg(P.out_bus_map + iu) : iu;
#pragma unroll
      for (int j = 0; j < LP; ++j) {
        if (!((dn >> j) & 1)) continue;
        const int ln = g.lane + j, s = L.scen[ln];
        const size_t o = (size_t)i * T + ln;
        if (P.out_theta) P.out_theta[(size_t)s * G.n + iu] = th[o];
        if (P.out_vm) {  // |V| of the state e + jf (0 on islanded buses)
          const double2 u = *reinterpret_cast<const double2*>(EF + ef_at<T>(i, ln));
          P.out_vm[(size_t)s * G.n + iu] = sqrt(fma(u.x, u.x, u.y * u.y));
        }
      }
    }
  }
  Vec<unsigned long long, LP> ml = vzero<unsigned long long, LP>();  // abs_bits patterns
  Vec<int, LP> nov = vzero<int, LP>();  // branches loaded above their rating
  const int nw = (G.m + 31) >> 5;       // words of a scenario's overload mask
  if (P.out_ovmask && dn) {
    for (int w = g.rs; w < nw; w += Geo<T>::RPS)
#pragma unroll
      for (int j = 0; j < LP; ++j)
        if ((dn >> j) & 1) P.out_ovmask[(size_t)L.scen[g.lane + j] * nw + w] = 0u;
    __syncthreads();  // the rows are cleared before any bit is set
  }
  if (dn) {
    for (int k = g.rs; k < G.m; k += Geo<T>::RPS) {
      const int a = __ldg(G.f + k), b = __ldg(G.t + k);
      const int pa = __ldg(G.pre + a), pb = __ldg(G.pre + b);
      const double gk = __ldg(G.g + k), bk = __ldg(G.by + k), ir = __ldg(G.inv_rating + k);
      const double ck = __ldg(G.cf + k);  // 1 / turns ratio at a (1 for a line)
#pragma unroll 1
      for (int jp = 0; jp < LP; jp += 2) {
        if (!((dn >> jp) & 3)) continue;
        const double2* qa = reinterpret_cast<const double2*>(EF + ef_at<T>(a, g.lane + jp));
        const double2* qb = reinterpret_cast<const double2*>(EF + ef_at<T>(b, g.lane + jp));
        const double2 va[2] = {qa[0], qa[1]}, vb[2] = {qb[0], qb[1]};
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int j = jp + h, ln = g.lane + j;
          if (!((dn >> j) & 1)) continue;
          const int lo = L.lo[ln], cnt = L.cnt[ln];
          double Pab = 0.0;
          if (k != L.l[ln] && !in_island(pa, lo, cnt) && !in_island(pb, lo, cnt)) {
            // P_ab = c^2 g |V_a|^2 - c (g Re(V_a conj V_b) + b Im(V_a conj V_b)),
            // P_ba = g |V_b|^2 - c (g Re(V_a conj V_b) - b Im(V_a conj V_b)),
            // c = 1 / turns ratio at a (the pi-model sees V_a c)
            const double ea = va[h].x, fa = va[h].y, eb = vb[h].x, fb = vb[h].y;
            const double cr = ck * fma(ea, eb, fa * fb), sr = ck * fma(fa, eb, -ea * fb);
            const double gc = gk * cr;
            Pab = fma(gk * ck * ck, fma(ea, ea, fa * fa), -fma(bk, sr, gc));
            const double Pba = fma(gk, fma(eb, eb, fb * fb), fma(bk, sr, -gc));
            // loading max(|P_ab|, |P_ba|) / rating: the larger end picked on
            // the bit patterns, one multiplication
            const unsigned long long u = abs_bits(Pab), v = abs_bits(Pba);
            const double ld = __longlong_as_double((long long)(u > v ? u : v)) * ir;
            upd_max_bits(ml.v[j], ld);
            if (overloaded(ld)) {
              nov.v[j] += 1;
              if (P.out_ovmask)
                atomicOr(P.out_ovmask + (size_t)L.scen[ln] * nw + (k >> 5), 1u << (k & 31));
            }
          }
          if (P.out_flow) P.out_flow[(size_t)L.scen[ln] * G.m + k] = Pab;
        }
      }
    }
  }
  const Vec<unsigned long long, LP> mlb = lane_max_bits<T, RS_LOAD>(L, ml);
  // (the counts take the buffer of the solve's first reduction, which is
  // idle between solves)
  if (P.out_nover) nov = lane_sum<T, RS_BB>(L, nov);
  if (g.rs == 0) {
#pragma unroll
    for (int j = 0; j < LP; ++j) {
      const int ln = g.lane + j, s = L.scen[ln];
      if (!L.done[ln] || s < 0) continue;
      int st = L.status[ln];
      if (st == 0 && L.nogen[ln]) st = 3;
      if (P.out_status) P.out_status[s] = st;
      if (P.out_iters) {
        P.out_iters[(size_t)s * 3 + 0] = L.outer[ln];
        P.out_iters[(size_t)s * 3 + 1] = L.inP[ln];
        P.out_iters[(size_t)s * 3 + 2] = L.inQ[ln];
      }
      if (P.out_maxload) P.out_maxload[s] = from_bits(mlb.v[j]);
      if (P.out_nover) P.out_nover[s] = nov.v[j];
      if (P.phase_cycles) P.phase_cycles[8 + 2 * (size_t)s + 1] = global_ns();
      L.done[ln] = 0;
      L.scen[ln] = -1;
    }
  }
  __syncthreads();
}

// One persistent CTA = one slot of T scenario lanes.  Lanes draw scenarios
// from a device-side queue (in the order P.order gives); a lane whose
// scenario has converged, failed or diverged is retired at the next outer
// iteration and immediately refilled, so converged scenarios never hold a
// lane (the slot's lanes are compacted onto live work) and the kernel ends
// when the queue is drained and every lane has retired.
//
// ZS: the tile's z vector -- the one the substitutions and the SpMV gather
// from, level after level -- lives in the CTA's dynamic shared memory
// instead of global memory, so those dependent gathers wait on shared memory
// rather than on L2 or DRAM; the CTA then takes rows x T x sizeof(VT) bytes
// of shared memory (80 KB for FP32 tiles of two on a 10,000-bus grid), two
// CTAs fit an SM, and the register budget is set for two.
template <int T, typename VT, bool GEN, bool ZS = false>
__global__ void __launch_bounds__(NTHREADS, ZS ? 2 : FDPF_MIN_BLOCKS)
    fdpf_tiles_kernel(FdpfParams P_, DevMatT<VT> MP_, DevMatT<VT> MQ_) {
  __shared__ LaneState<T> L;
  // the parameter blocks in shared memory: the out-of-line passes take them
  // by reference, so their fields are read from shared memory rather than
  // from a per-thread local copy
  __shared__ __align__(16) unsigned char pbuf[sizeof(FdpfParams)];
  __shared__ __align__(16) unsigned char mbuf[2][sizeof(DevMatT<VT>)];
  const int tid = threadIdx.x;
  if (tid == 0) {
    memcpy(pbuf, &P_, sizeof(FdpfParams));
    memcpy(mbuf[0], &MP_, sizeof(DevMatT<VT>));
    memcpy(mbuf[1], &MQ_, sizeof(DevMatT<VT>));
  }
  // the extension rows' lane state, in the kernel with extension rows only
  SwitchState<T>* SW = nullptr;
  if constexpr (GEN) {
    __shared__ SwitchState<T> sw;
    SW = &sw;
  }
  __syncthreads();
  const FdpfParams& P = *reinterpret_cast<const FdpfParams*>(pbuf);
  const DevMatT<VT>& MP = *reinterpret_cast<const DevMatT<VT>*>(mbuf[0]);
  const DevMatT<VT>& MQ = *reinterpret_cast<const DevMatT<VT>*>(mbuf[1]);
  constexpr int LP = Geo<T>::LP;
  const Geo<T> g;
  VT* x = (VT*)P.wx + (size_t)blockIdx.x * P.vstride;
  VT* r = (VT*)P.wr + (size_t)blockIdx.x * P.vstride;
  VT* p = (VT*)P.wp + (size_t)blockIdx.x * P.vstride;
  VT* q = (VT*)P.wq + (size_t)blockIdx.x * P.vstride;
  extern __shared__ __align__(16) unsigned char zdyn[];
  VT* z = ZS ? reinterpret_cast<VT*>(zdyn) : (VT*)P.wz + (size_t)blockIdx.x * P.vstride;
  const size_t so = (size_t)blockIdx.x * P.sstride;
  // E and F regions of the slots taken together: [slot][bus][lane][e, f]
  double *th = P.wth + so, *EF = P.we + 2 * so;

  // optional per-phase cycle counters (thread 0's view of the CTA)
  const bool tim = P.phase_cycles != nullptr;
  long long t_prev = 0;
  if (tid == 0) {
    for (int k = 0; k < 8; ++k) L.tphase[k] = 0;
    t_prev = clock64();
    L.drained = 0;
  }
  if (tid < T) {
    // a lane the queue never fills keeps these: no outage, nothing islanded
    L.scen[tid] = -1;
    L.active[tid] = 0;
    L.done[tid] = 0;
    L.fresh[tid] = 0;
    L.l[tid] = L.fb[tid] = L.tb[tid] = -1;
    L.raP[tid] = L.rbP[tid] = L.raQ[tid] = L.rbQ[tid] = -1;
    L.wP[tid] = L.wQ[tid] = 0.0;
    L.cl[tid] = 1.0;
    L.gb[tid] = -1;
    if constexpr (GEN) {
      SW->nx[tid] = 0;
      SW->nc[tid] = 0;
      SW->bk[tid] = 0u;
      SW->skip[tid] = 0;
    }
    L.lo[tid] = L.cnt[tid] = 0;
  }
  __syncthreads();
#define GPCG_PHASE(k)                                  \
  if (tim && tid == 0) {                               \
    const long long t_ = clock64();                    \
    L.tphase[k] += (unsigned long long)(t_ - t_prev);  \
    t_prev = t_;                                       \
  }

  for (;;) {
    // retire finished lanes, then refill empty lanes from the queue
    if (any_lane<T>(L, L.done)) retire_pass<T>(P, L, th, EF);
    GPCG_PHASE(7);
    if (tid == 0 && !L.drained) {
      int need = 0;
      for (int s = 0; s < T; ++s) need += (L.scen[s] < 0);
      if (need) {
        const int base = atomicAdd(P.tile_counter, need);
        int j = 0;
        for (int s = 0; s < T; ++s) {
          if (L.scen[s] >= 0) continue;
          const int qi = base + j++;
          if (qi < P.S) {
            L.scen[s] = P.order ? P.order[qi] : qi;
            L.fresh[s] = 1;
          }
        }
        if (base + need >= P.S) L.drained = 1;
      }
    }
    __syncthreads();
    if (tid < T && L.fresh[tid]) {
      setup_lane<T, VT>(P, MP, MQ, L, tid, SW);
      if (tim) P.phase_cycles[8 + 2 * (size_t)L.scen[tid]] = global_ns();
    }
    __syncthreads();
    init_pass<T>(P, L, th, EF);
    __syncthreads();
    if (tid < T) L.fresh[tid] = 0;
    if constexpr (GEN) {
      // lanes that sat out the last outer iteration after a switch
      if (tid < T && SW->skip[tid]) {
        SW->skip[tid] = 0;
        L.active[tid] = 1;
      }
      __syncthreads();
    }
    GPCG_PHASE(0);
    if (!any_lane<T>(L, L.active)) {
      if (L.drained) break;
      continue;
    }
    // P half-step: mismatch + convergence test
    Vec<unsigned long long, LP> eP = vzero<unsigned long long, LP>(), eQ = eP;
    mismatch_pass<T, VT, true, GEN>(P, MP, MQ, L, EF, r, eP, eQ, SW);
    const Vec<unsigned long long, LP> bP = lane_max_bits<T, RS_ERRP>(L, eP);
    const Vec<unsigned long long, LP> bQ = lane_max_bits<T, RS_ERRQ>(L, eQ);
    if (g.rs == 0) {
#pragma unroll
      for (int j = 0; j < LP; ++j) {
        const int ln = g.lane + j;
        if (!L.active[ln]) continue;
        const double a = from_bits(bP.v[j]), b = from_bits(bQ.v[j]);
        const double e2 = (a != a || b != b) ? INFINITY : fmax(a, b);
        L.err[ln] = e2;
        int st = -1;
        // growth rule only for warm-started scenarios: a flat start may pass
        // through large mismatches on its way
        if (!(e2 <= DIVERGE_LIMIT) || (!P.flat_start && e2 > DIVERGE_GROWTH * L.best[ln])) st = 2;
        else if (e2 <= P.tol) st = 0;
        else if (L.outer[ln] >= P.max_outer) st = 1;
        L.best[ln] = fmin(L.best[ln], e2);
        if (GEN && st == 0 && (SW->nc[ln] > 0 || SW->bk[ln] != 0u)) {
          // converged with PV generators outside their reactive limits, or
          // held ones able to hold their set point again: the latter turn
          // back PV at the set point, the former PQ at the violated limit
          // (in bus order), and the lane sits out the rest of this outer
          // iteration, so the next starts from the mismatch of the new
          // state; the base case must be within its limits, and a lane
          // holds at most KX extension rows
          const int nc = SW->nc[ln];
          const unsigned bk = SW->bk[ln];
          if (P.flat_start || SW->nx[ln] - __popc(bk) + nc > KX) {
            st = 4;
          } else {
            int w = 0;
            for (int u = 0; u < SW->nx[ln]; ++u) {
              if ((bk >> u) & 1u) {
                // |V| back to the set point, the angle kept
                const int b = SW->xb[ln][u];
                double2* ef = reinterpret_cast<double2*>(EF + ef_at<T>(b, ln));
                const double2 v = ef[0];
                const double k = P.G.V_set[b] / sqrt(fma(v.x, v.x, v.y * v.y));
                ef[0] = make_double2(v.x * k, v.y * k);
                continue;
              }
              SW->xb[ln][w] = SW->xb[ln][u];
              SW->xq[ln][w] = SW->xq[ln][u];
              SW->xs[ln][w] = SW->xs[ln][u];
              ++w;
            }
            for (int u = 1; u < nc; ++u)
              for (int v = u; v > 0 && SW->cb[ln][v - 1] > SW->cb[ln][v]; --v) {
                const int tb = SW->cb[ln][v];
                SW->cb[ln][v] = SW->cb[ln][v - 1];
                SW->cb[ln][v - 1] = tb;
                const double tq = SW->cq[ln][v];
                SW->cq[ln][v] = SW->cq[ln][v - 1];
                SW->cq[ln][v - 1] = tq;
                const int ts = SW->cs[ln][v];
                SW->cs[ln][v] = SW->cs[ln][v - 1];
                SW->cs[ln][v - 1] = ts;
              }
            for (int u = 0; u < nc; ++u) {
              SW->xb[ln][w + u] = SW->cb[ln][u];
              SW->xq[ln][w + u] = SW->cq[ln][u];
              SW->xs[ln][w + u] = SW->cs[ln][u];
            }
            SW->nx[ln] = w + nc;
            L.best[ln] = INFINITY;  // the switch raises the mismatch on purpose
            SW->skip[ln] = 1;
            st = -1;
          }
        }
        if constexpr (GEN) {
          SW->nc[ln] = 0;
          SW->bk[ln] = 0u;
        }
        if (st >= 0) {
          L.status[ln] = st;
          L.active[ln] = 0;
          L.done[ln] = 1;
        } else if (GEN && SW->skip[ln]) {
          L.active[ln] = 0;  // back at the top of the next outer iteration
        }
        // a P mismatch already within the tolerance takes no P step
        L.hold[ln] = a <= P.tol;
      }
    }
    const bool more = any_lane<T>(L, L.active);
    GPCG_PHASE(1);
    if (!more) continue;
    if (any_stepping<T>(L)) {
      pcg_solve<T, VT, true, GEN>(P, MP, L, x, r, p, q, z, L.raP, L.rbP, L.wP, L.inP, nullptr,
                                  nullptr, L.hold);
      GPCG_PHASE(2);
      update_pass<T, VT, true, GEN>(MP, L, x, p, th, EF, SW);
    }
    __syncthreads();
    GPCG_PHASE(3);
    // Q half-step: the Q mismatch after the P step; a lane whose Q mismatch
    // is within the tolerance takes no Q step
    Vec<unsigned long long, LP> d0 = vzero<unsigned long long, LP>(), d1 = d0;
    mismatch_pass<T, VT, false, GEN>(P, MP, MQ, L, EF, r, d0, d1, SW);
    {
      const Vec<unsigned long long, LP> bQ2 = lane_max_bits<T, RS_ERRQ>(L, d1);
      if (g.rs == 0)
#pragma unroll
        for (int j = 0; j < LP; ++j) L.hold[g.lane + j] = from_bits(bQ2.v[j]) <= P.tol;
    }
    GPCG_PHASE(4);
    if (any_stepping<T>(L)) {
      pcg_solve<T, VT, true, GEN>(P, MQ, L, x, r, p, q, z, L.raQ, L.rbQ, L.wQ, L.inQ,
                                  MQ.c ? L.cl : nullptr, SW, L.hold);
      GPCG_PHASE(5);
      update_pass<T, VT, false, GEN>(MQ, L, x, p, th, EF, SW);
    }
    if (g.rs == 0)
#pragma unroll
      for (int j = 0; j < LP; ++j)
        if (L.active[g.lane + j]) L.outer[g.lane + j] += 1;
    __syncthreads();
    GPCG_PHASE(6);
  }
  if (tim && tid == 0)
    for (int k = 0; k < 8; ++k) atomicAdd(P.phase_cycles + k, L.tphase[k]);
#undef GPCG_PHASE
}


// ----------------------------------------------------------- launchers
// zbytes > 0: the variant with z in `zbytes` of dynamic shared memory (branch
// outages, tiles of 2 or 4); 0: z in global memory.
template <int T, typename VT, bool ZS>
cudaError_t set_zs_smem(size_t zbytes) {
  if constexpr (!ZS) return cudaSuccess;
  else return cudaFuncSetAttribute(fdpf_tiles_kernel<T, VT, false, true>,
                                   cudaFuncAttributeMaxDynamicSharedMemorySize, (int)zbytes);
}

template <bool GEN, typename VT>
cudaError_t launch_fdpf_g(cudaStream_t st, int T, int grid, const FdpfParams& P,
                          const DevMatT<VT>& MP, const DevMatT<VT>& MQ, size_t zbytes = 0) {
  if (zbytes) {
    if constexpr (GEN) return cudaErrorInvalidValue;
    else {
      cudaError_t ce = cudaErrorInvalidValue;
      if (T == 2 && (ce = set_zs_smem<2, VT, true>(zbytes)) == cudaSuccess)
        fdpf_tiles_kernel<2, VT, false, true><<<grid, NTHREADS, zbytes, st>>>(P, MP, MQ);
      else if (T == 4 && (ce = set_zs_smem<4, VT, true>(zbytes)) == cudaSuccess)
        fdpf_tiles_kernel<4, VT, false, true><<<grid, NTHREADS, zbytes, st>>>(P, MP, MQ);
      else
        return ce;
      return cudaGetLastError();
    }
  }
  switch (T) {
    case 2: fdpf_tiles_kernel<2, VT, GEN><<<grid, NTHREADS, 0, st>>>(P, MP, MQ); break;
    case 4: fdpf_tiles_kernel<4, VT, GEN><<<grid, NTHREADS, 0, st>>>(P, MP, MQ); break;
    case 8: fdpf_tiles_kernel<8, VT, GEN><<<grid, NTHREADS, 0, st>>>(P, MP, MQ); break;
    case 16:
      if constexpr (GEN) return cudaErrorInvalidValue;
      else fdpf_tiles_kernel<16, VT, GEN><<<grid, NTHREADS, 0, st>>>(P, MP, MQ);
      break;
    case 32:
      if constexpr (GEN) return cudaErrorInvalidValue;
      else fdpf_tiles_kernel<32, VT, GEN><<<grid, NTHREADS, 0, st>>>(P, MP, MQ);
      break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <bool GEN, typename VT>
int fdpf_blocks_g(int T, size_t zbytes = 0) {
  int nb = 0;
  cudaError_t ce = cudaErrorInvalidValue;
  if (zbytes) {
    if constexpr (!GEN) {
      if (T == 2 && set_zs_smem<2, VT, true>(zbytes) == cudaSuccess)
        ce = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &nb, fdpf_tiles_kernel<2, VT, false, true>, NTHREADS, zbytes);
      else if (T == 4 && set_zs_smem<4, VT, true>(zbytes) == cudaSuccess)
        ce = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &nb, fdpf_tiles_kernel<4, VT, false, true>, NTHREADS, zbytes);
    }
    return ce == cudaSuccess ? nb : 0;
  }
  switch (T) {
    case 2: ce = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fdpf_tiles_kernel<2, VT, GEN>, NTHREADS, 0); break;
    case 4: ce = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fdpf_tiles_kernel<4, VT, GEN>, NTHREADS, 0); break;
    case 8: ce = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fdpf_tiles_kernel<8, VT, GEN>, NTHREADS, 0); break;
    case 16:
      if constexpr (!GEN) ce = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fdpf_tiles_kernel<16, VT, GEN>, NTHREADS, 0);
      break;
    case 32:
      if constexpr (!GEN) ce = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fdpf_tiles_kernel<32, VT, GEN>, NTHREADS, 0);
      break;
  }
  return ce == cudaSuccess ? nb : 0;
}

}  // namespace gpcg
