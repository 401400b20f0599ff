// lym1_pol_unit.cuh -- body of a per-policy translation unit: defines the
// entry points of lym1_policies.h for the policy LYM1_POL in namespace
// LYM1_POL_NS.
#include "lym1_kernels.cuh"
#include "lym1_policies.h"

namespace lym1 {
namespace LYM1_POL_NS {

using P = LYM1_POL;

int transport(const DeviceView& v, void* st) {
  return launch_transport_t<P>(v, static_cast<cudaStream_t>(st));
}

int freq(const DeviceView& v, void* st) {
  return launch_freq_t<P>(v, static_cast<cudaStream_t>(st));
}

int subcycle(const DeviceView& v, void* st) {
  return launch_subcycle_t<P>(v, static_cast<cudaStream_t>(st));
}

int batched(int kind, int geometry, int pt, const DeviceView* views, const void* items, int n,
            int grid, int nb_max, void* st, int shape) {
  const cudaStream_t s = static_cast<cudaStream_t>(st);
  const BatchItem* it = static_cast<const BatchItem*>(items);
  if (kind == 0)
    return launch_transport_batched_t<P>(geometry, pt, views, it, n, grid, nb_max, s, shape);
  if (kind == 1) return launch_freq_batched_t<P>(geometry, pt, views, it, n, grid, nb_max, s);
  return launch_subcycle_batched_t<P>(geometry, pt, views, it, n, grid, s);
}

int resident(int kind, int geometry, int pt, int nb_max, int shape) {
  if (kind == 0) return max_resident_transport<P>(geometry, pt, nb_max, shape);
  if (kind == 1) return max_resident_freq<P>(geometry, pt, nb_max);
  return max_resident_subcycle<P>(geometry, pt);
}

}  // namespace LYM1_POL_NS
}  // namespace lym1
