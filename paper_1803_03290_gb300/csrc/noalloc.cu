// gpcg_n1_screen_noalloc: the N-1 screen with every scratch buffer taken
// from one fixed device array, for callers that cannot allocate GPU memory
// while they run (see include/gpcg.h).  This file only adds that entry
// point; it reuses the islanding and persistent-solve kernels unchanged.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstdarg>

#include "../../include/gpcg.h"
#include "common.cuh"
#include "ctx_view.h"
#include "fdpf.h"

namespace gpcg {
void set_last_error(const char* msg);
}  // namespace gpcg

using namespace gpcg;

// The scratch array.  It lives in device memory of every GPU that loads the
// library, for as long as the process runs.  In host code its name is only a
// stand-in: the device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[GPCG_NOALLOC_SCRATCH_BYTES];

namespace {

gpcg_status err(gpcg_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  std::vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  set_last_error(buf);
  return st;
}

// Device address of the scratch array in the calling thread's current CUDA
// context.  Each context that loads the library's device code has its own
// copy of the array at its own address (a second context on a device, or
// the primary context after cudaDeviceReset, gets a new one), so the address
// is looked up on every call rather than cached: the lookup is a table
// search in the runtime, small beside the call's own synchronisation.
gpcg_status scratch_address(unsigned char** out) {
  void* p = nullptr;
  const cudaError_t ce = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (ce != cudaSuccess || !p)
    return err(GPCG_ERR_CUDA, "cudaGetSymbolAddress(scratch): %s", cudaGetErrorString(ce));
  *out = (unsigned char*)p;
  return GPCG_OK;
}

size_t up256(size_t b) { return (b + 255) / 256 * 256; }

}  // namespace

extern "C" gpcg_status gpcg_n1_screen_noalloc(gpcg_ctx* ctx, const int32_t* outages,
                                              int32_t n_out, void* stream, double* theta,
                                              double* vm, double* flow, int32_t* island_label,
                                              int32_t* iters, int32_t* status,
                                              double* max_loading, int32_t* n_overload,
                                              uint32_t* overload) {
  CtxView c;
  if (!ctx_view(ctx, &c)) return err(GPCG_ERR_INVALID_ARG, "gpcg_n1_screen_noalloc: ctx is NULL");
  if (n_out < 0) return err(GPCG_ERR_INVALID_ARG, "n_out < 0");
  if (!c.base_ok) return err(GPCG_ERR_NOT_READY, "gpcg_base_solve has not succeeded");
  if (c.opt.precision != GPCG_BATCHED_FP32 && c.opt.precision != GPCG_BATCHED_FP64 &&
      c.opt.precision != GPCG_BATCHED_FP32_F16)
    return err(GPCG_ERR_INVALID_ARG,
               "gpcg_n1_screen_noalloc runs the batched solve only (precision 1, 2 or 3)");
  if (n_out == 0) { set_last_error(""); return GPCG_OK; }
  if (!outages) return err(GPCG_ERR_INVALID_ARG, "outages is NULL");
  cudaStream_t st = (cudaStream_t)stream;
  unsigned char* base = nullptr;
  gpcg_status s = scratch_address(&base);
  if (s != GPCG_OK) return s;

  // layout: [queue counter] [per-scenario island data] [solve slots]
  const size_t S = (size_t)n_out;
  // reactive limits take the kernel with extension rows (tiles of 2, 4, 8)
  const bool ext = c.G.qmax != nullptr;
  int T = c.opt.tile ? c.opt.tile : (c.tile ? c.tile : 2);
  if (ext) T = std::min(T, 8);
  const bool f32 = c.opt.precision != GPCG_BATCHED_FP64;
  const size_t vt = f32 ? 4 : 8;
  const size_t head = 256;
  const size_t scen = up256(S * 4) * 3 + up256(S * 8);
  const size_t vec_bytes = up256((size_t)(c.rows + 1) * T * vt);
  const size_t st_bytes = up256((size_t)c.n * T * 8);
  // five vectors; the state theta and e + jf (two arrays' worth)
  const size_t per_slot = 5 * vec_bytes + 3 * st_bytes;
  const size_t cap = GPCG_NOALLOC_SCRATCH_BYTES;
  if (head + scen + per_slot > cap)
    return err(GPCG_ERR_INVALID_ARG,
               "gpcg_n1_screen_noalloc: %zu scenarios of a %d-bus grid need %zu bytes of "
               "scratch, more than the %zu-byte limit",
               S, c.n, head + scen + per_slot, cap);
  const int n_tiles = (int)((S + T - 1) / T);
  const int occ =
      f32 ? fdpf_max_blocks_per_sm<float>(T, ext) : fdpf_max_blocks_per_sm<double>(T, ext);
  int per_sm = c.opt.ctas_per_sm ? c.opt.ctas_per_sm : std::min(c.per_sm, occ);
  if (per_sm <= 0) per_sm = occ;
  per_sm = std::max(per_sm, 1);
  const size_t fit = (cap - head - scen) / per_slot;
  const int slots = (int)std::max<size_t>(1, std::min<size_t>(
      fit, (size_t)std::min(n_tiles, c.num_sms * per_sm)));

  // validate the outage list through a fixed host buffer
  {
    int32_t buf[1024];
    for (size_t o = 0; o < S; o += 1024) {
      const size_t k = std::min<size_t>(1024, S - o);
      cudaError_t ce = cudaMemcpyAsync(buf, outages + o, k * 4, cudaMemcpyDeviceToHost, st);
      if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
      if (ce != cudaSuccess) return err(GPCG_ERR_CUDA, "outage copy: %s", cudaGetErrorString(ce));
      for (size_t j = 0; j < k; ++j)
        if (buf[j] < 0 || buf[j] >= c.m)
          return err(GPCG_ERR_INVALID_ARG, "outages[%zu] = %d is not a branch index", o + j, buf[j]);
    }
  }
  int32_t* counter = (int32_t*)base;
  unsigned char* q = base + head;
  int32_t* lo = (int32_t*)q;  q += up256(S * 4);
  int32_t* cnt = (int32_t*)q; q += up256(S * 4);
  int32_t* nogen = (int32_t*)q; q += up256(S * 4);
  double* coef = (double*)q;  q += up256(S * 8);
  unsigned char* work = q;

  cudaError_t ce = cudaMemsetAsync(base, 0, head, st);  // the queue head starts at 0
  if (ce != cudaSuccess) return err(GPCG_ERR_CUDA, "scratch reset: %s", cudaGetErrorString(ce));
  ce = launch_islands(st, (int)S, c.n, outages, c.isl, nullptr, nullptr, lo, cnt, coef, nogen,
                      island_label);
  if (ce != cudaSuccess) return err(GPCG_ERR_CUDA, "islands: %s", cudaGetErrorString(ce));

  FdpfParams P;
  P.G = c.G;
  P.mis_order = c.mis_order;
  P.misq_order = c.misq_order;
  P.r0P = c.r0P;
  P.r0Q = c.r0Q;
  P.tol = c.opt.tol;
  P.inner_rtol = c.opt.inner_rtol;
  P.max_outer = c.opt.max_outer;
  P.max_inner = c.opt.max_inner;
  P.precond = c.opt.precond;
  P.sc = ScenInfo{const_cast<int32_t*>(outages), lo, cnt, coef, nogen};
  P.th0 = c.th0; P.V0 = c.V0; P.c0 = c.c0; P.s0 = c.s0;
  P.out_theta = theta; P.out_vm = vm; P.out_flow = flow; P.out_maxload = max_loading;
  P.out_iters = iters; P.out_status = status;
  P.out_nover = n_overload; P.out_ovmask = overload;
  P.out_bus_map = c.bus_of_user;
  P.S = (int)S;
  P.n_tiles = n_tiles;
  P.tile_counter = counter;
  const size_t vb = (size_t)slots * vec_bytes, sb = (size_t)slots * st_bytes;
  P.wx = work; P.wr = work + vb; P.wp = work + 2 * vb; P.wq = work + 3 * vb; P.wz = work + 4 * vb;
  P.vstride = vec_bytes / vt;
  double* sbase = (double*)(work + 5 * vb);
  const size_t ss = st_bytes / 8;
  (void)sb;
  P.wth = sbase; P.we = sbase + slots * ss; P.wf = sbase + 2 * slots * ss;
  P.sstride = ss;
  ce = f32 ? launch_fdpf<float>(st, T, slots, P, c.MPf, c.MQf)
           : launch_fdpf<double>(st, T, slots, P, c.MPd, c.MQd);
  if (ce != cudaSuccess) return err(GPCG_ERR_CUDA, "solve: %s", cudaGetErrorString(ce));
  set_last_error("");
  return GPCG_OK;
}
