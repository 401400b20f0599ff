// lym1_policies.h -- entry points of the per-policy translation units of the
// FMA-contracting policies (LYM1_FP64, LYM1_MIXED, LYM1_MIXED_FAST).  Each
// unit instantiates every kernel of one policy; kind 0 = transport,
// 1 = frequency step, 2 = step 2 under the substep acceptance rule.
#pragma once

#include "lym1_internal.h"

namespace lym1 {

#define LYM1_POLICY_API(NS)                                                            \
  namespace NS {                                                                       \
  int transport(const DeviceView& v, void* stream);                                    \
  int freq(const DeviceView& v, void* stream);                                         \
  int subcycle(const DeviceView& v, void* stream);                                     \
  int batched(int kind, int geometry, int pt, const DeviceView* views, const void* items, \
              int n, int grid, int nb_max, void* stream, int shape);                   \
  int resident(int kind, int geometry, int pt, int nb_max, int shape);                 \
  }

LYM1_POLICY_API(pol_f64)
LYM1_POLICY_API(pol_mix)
LYM1_POLICY_API(pol_mixf)

#undef LYM1_POLICY_API

}  // namespace lym1
