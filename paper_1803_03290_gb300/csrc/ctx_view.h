// Read-only view of a gpcg context for translation units other than the
// one that defines the context (abi.cu).
#pragma once
#include "../../include/gpcg.h"
#include "common.cuh"

namespace gpcg {

struct CtxView {
  DevGrid G;
  DevMatT<float> MPf, MQf;
  DevMatT<double> MPd, MQd;
  const double *th0 = nullptr, *V0 = nullptr, *c0 = nullptr, *s0 = nullptr;
  const int32_t *mis_order = nullptr, *misq_order = nullptr;
  const int32_t* bus_of_user = nullptr;  // caller's bus -> internal bus
  gpcg_options opt{};
  int num_sms = 0, n = 0, m = 0, slack = -1, rows = 0, tile = 0, slack_user = -1;
  int per_sm = 0;  // tiles per SM the autotuner chose (0: none yet)
  const int32_t *u_f = nullptr, *u_t = nullptr, *u_pre = nullptr;  // caller numbering
  const int8_t* u_bus_type = nullptr;
  const double *u_P_sched = nullptr, *u_P_gen = nullptr;
  IslandPlan isl;
  const double *r0P = nullptr, *r0Q = nullptr;
  bool base_ok = false;
};

bool ctx_view(const gpcg_ctx* c, CtxView* v);

}  // namespace gpcg
