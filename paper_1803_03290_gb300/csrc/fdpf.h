// Parameters and launchers of the persistent N-1 kernel (fdpf.cu).
#pragma once
#include "common.cuh"

namespace gpcg {

#ifndef FDPF_NTHREADS
#define FDPF_NTHREADS 256
#endif
constexpr int NTHREADS = FDPF_NTHREADS;  // threads per CTA of the persistent kernel
constexpr double DIVERGE_LIMIT = 1.0e4;   // p.u.: a larger mismatch is divergence
constexpr double DIVERGE_GROWTH = 10.0;   // as is growth to this multiple of the best
enum { PREC_IC0 = 0, PREC_JACOBI = 1, PREC_EXACT = 2 };

struct FdpfParams {
  DevGrid G;
  int S = 0, n_tiles = 0;
  ScenInfo sc;
  const double *th0 = nullptr, *V0 = nullptr;  // warm start (bus order)
  const double *c0 = nullptr, *s0 = nullptr;   // cos, sin of th0
  const double *r0P = nullptr, *r0Q = nullptr; // base-case mismatch per bus (null: not used)
  int flat_start = 0;
  double tol = 1e-4, inner_rtol = 3e-3;
  int max_outer = 50, max_inner = 500, precond = PREC_EXACT;
  int32_t* tile_counter = nullptr;     // scenario queue head
  const int32_t* order = nullptr;      // scenarios in processing order (null: 0..S-1)
  void *wx = nullptr, *wr = nullptr, *wp = nullptr, *wq = nullptr, *wz = nullptr;
  size_t vstride = 0;  // elements per slot of one vector
  // FP64 state per slot: theta, and e + jf interleaved over the we and wf
  // regions together ([slot][bus][lane][e, f], 2 sstride per slot); the
  // persistent N-1 kernel keeps no |V| (|e + jf|), so wV is scratch for the
  // DC and adjoint kernels only
  double *wth = nullptr, *wV = nullptr, *we = nullptr, *wf = nullptr;
  size_t sstride = 0;  // elements per slot of one state array
  double *out_theta = nullptr, *out_vm = nullptr, *out_flow = nullptr, *out_maxload = nullptr;
  // output column -> internal bus (null: identity): the outputs are written
  // column by column, so neighbouring threads store neighbouring columns
  const int32_t* out_bus_map = nullptr;
  int32_t *out_iters = nullptr, *out_status = nullptr;
  // overload screen: per scenario the number of branches loaded above their
  // rating, and those branches as a bit mask of mask_words words
  int32_t* out_nover = nullptr;
  uint32_t* out_ovmask = nullptr;
  // diagnostics, or null: [8] per-phase SM cycles summed over CTAs, then per
  // scenario the global timer (ns) when a lane took it and when it retired
  unsigned long long* phase_cycles = nullptr;
  const int32_t* mis_order = nullptr;   // non-slack buses sorted by degree
  const int32_t* misq_order = nullptr;  // B'' rows sorted by their bus's degree
};

// The persistent N-1 kernel for tiles of T scenarios (2 to 32; generator
// outages, P.sc.gen_bus set: 2, 4 or 8) on `grid` slots.  zbytes > 0 (branch
// outages without reactive limits, T = 2 or 4): each tile's z vector in
// zbytes of dynamic shared memory, P.wz unused.
template <typename VT>
cudaError_t launch_fdpf(cudaStream_t st, int T, int grid, const FdpfParams& P,
                        const DevMatT<VT>& MP, const DevMatT<VT>& MQ, size_t zbytes = 0);
template <typename VT>
int fdpf_max_blocks_per_sm(int T, bool gen = false, size_t zbytes = 0);
// the generator-outage kernel (fdpf_gen.cu)
template <typename VT>
cudaError_t launch_fdpf_gen(cudaStream_t st, int T, int grid, const FdpfParams& P,
                            const DevMatT<VT>& MP, const DevMatT<VT>& MQ);
template <typename VT>
int fdpf_blocks_gen(int T);
template <typename VT>
cudaError_t launch_apply(cudaStream_t st, int grid, const DevMatT<VT>& M, int op, int S,
                         const int32_t* outages, const int32_t* f, const int32_t* t,
                         const double* X, double* Y, VT* wbuf, size_t vstride, int precond);
cudaError_t launch_base_trig(cudaStream_t st, int n, const double* th, double* c, double* s);
cudaError_t launch_base_residual(cudaStream_t st, const DevGrid& G, const double* V0,
                                 const double* c0, const double* s0, double* r0P, double* r0Q);

// plain.cu: the unbatched FP64 path, one scenario per cooperative launch
// over the whole GPU.  Work buffers, device memory owned by the caller.
struct PlainBuffers {
  double* part = nullptr;          // [2 * 4 * grid]
  unsigned int* bar = nullptr;     // [2], zero before the first launch
  int* err = nullptr;              // [1], zero before the first launch
  unsigned wait_limit = 1u << 25;  // polls of a barrier wait (~64 ns each) before it gives up
  double *x = nullptr, *r = nullptr, *p = nullptr, *q = nullptr, *z = nullptr, *t = nullptr;
  double *th = nullptr, *V = nullptr, *ef = nullptr;  // [n], [n], [2 n]
};
cudaError_t launch_plain(cudaStream_t st, int grid, const FdpfParams& P,
                         const DevMatT<double>& MP, const DevMatT<double>& MQ,
                         const PlainBuffers& B, int s);
int plain_grid(int num_sms);  // CTAs of the cooperative launch (0: not available)

// adjoint.cu
struct AdjParamsView {
  const double* P;   // [n] injections, internal bus order
  const double* b;   // [m] branch susceptances
  double *gP, *gb, *loss;  // per-slot sums: [slots][n], [slots][m], [slots]
};
cudaError_t launch_adjoint(cudaStream_t st, int grid, const FdpfParams& P, const AdjParamsView& A,
                           const DevMatT<double>& M);
int adjoint_max_blocks_per_sm();

// Inputs and outputs of the DC (P-theta) quick screen.
struct DcParamsView {
  const double* P;              // [n] injections, internal bus order
  const int32_t* user_of_bus;   // internal bus -> caller's index
  double* theta;                // [S][n] caller's bus order, or null
  double* flow;                 // [S][m], or null
  double* maxload;              // [S], or null
  int32_t* iters;               // [S] PCG iterations, or null
  int32_t* status;              // [S], or null
  int32_t* nover;               // [S] branches loaded above their rating, or null
  uint32_t* ovmask;             // [S][(m + 31) / 32] those branches as bits, or null
};
template <typename VT>
cudaError_t launch_dc(cudaStream_t st, int grid, const FdpfParams& P, const DcParamsView& D,
                      const DevMatT<VT>& M, const DevMatT<double>& M64);
template <typename VT>
int dc_max_blocks_per_sm();
cudaError_t launch_slot_sum(cudaStream_t st, int n, int slots, const double* acc,
                            const int32_t* map, double* out);
cudaError_t launch_gather_perm(cudaStream_t st, int n, const int32_t* idx, const double* src,
                               double* dst);

}  // namespace gpcg
