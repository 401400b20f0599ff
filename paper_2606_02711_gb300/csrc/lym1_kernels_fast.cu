// lym1_kernels_fast.cu -- kernels of the LYM1_FP64, LYM1_MIXED and
// LYM1_MIXED_FAST policies (FMA contraction allowed, hardware exp/expm1).
#include "lym1_kernels.cuh"

namespace lym1 {

using PolF64 = Policy<double, double, double, false>;
using PolMix = Policy<float, float, double, false>;
using PolMixFast = Policy<float, float, float, false>;

int launch_transport_fast(int precision, const DeviceView& v, void* st) {
  const cudaStream_t s = static_cast<cudaStream_t>(st);
  switch (precision) {
    case 1: return launch_transport_t<PolF64>(v, s);
    case 2: return launch_transport_t<PolMix>(v, s);
    case 3: return launch_transport_t<PolMixFast>(v, s);
    default: return static_cast<int>(cudaErrorInvalidValue);
  }
}

int launch_freq_fast(int precision, const DeviceView& v, void* st) {
  const cudaStream_t s = static_cast<cudaStream_t>(st);
  switch (precision) {
    case 1: return launch_freq_t<PolF64>(v, s);
    case 2: return launch_freq_t<PolMix>(v, s);
    case 3: return launch_freq_t<PolMixFast>(v, s);
    default: return static_cast<int>(cudaErrorInvalidValue);
  }
}

}  // namespace lym1
