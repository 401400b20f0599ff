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

int launch_batched_fast(int precision, int kind, int geometry, int pt, const DeviceView* views,
                        const void* items, int n, int grid, int nb_max, void* st) {
  const cudaStream_t s = static_cast<cudaStream_t>(st);
  const BatchItem* it = static_cast<const BatchItem*>(items);
  switch (precision * 2 + kind) {
    case 2: return launch_transport_batched_t<PolF64>(geometry, pt, views, it, n, grid, nb_max, s);
    case 3: return launch_freq_batched_t<PolF64>(geometry, pt, views, it, n, grid, nb_max, s);
    case 4: return launch_transport_batched_t<PolMix>(geometry, pt, views, it, n, grid, nb_max, s);
    case 5: return launch_freq_batched_t<PolMix>(geometry, pt, views, it, n, grid, nb_max, s);
    case 6: return launch_transport_batched_t<PolMixFast>(geometry, pt, views, it, n, grid, nb_max, s);
    case 7: return launch_freq_batched_t<PolMixFast>(geometry, pt, views, it, n, grid, nb_max, s);
    default: return static_cast<int>(cudaErrorInvalidValue);
  }
}

int resident_blocks_fast(int precision, int kind, int geometry, int pt, int nb_max) {
  switch (precision * 2 + kind) {
    case 2: return max_resident_transport<PolF64>(geometry, pt, nb_max);
    case 3: return max_resident_freq<PolF64>(geometry, pt, nb_max);
    case 4: return max_resident_transport<PolMix>(geometry, pt, nb_max);
    case 5: return max_resident_freq<PolMix>(geometry, pt, nb_max);
    case 6: return max_resident_transport<PolMixFast>(geometry, pt, nb_max);
    case 7: return max_resident_freq<PolMixFast>(geometry, pt, nb_max);
    default: return 1;
  }
}

__global__ void fp64_helpers_kernel(const float* xf, const double* xd, long long n, double* wide,
                                    float* narrow, double* rcp) {
  const long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  wide[i] = f2d_alu(xf[i]);
  narrow[i] = d2f_alu(xd[i]);
  rcp[i] = drcp_nr(xd[i]);
}

}  // namespace lym1

extern "C" int lym1_debug_fp64_helpers(const float* xf, const double* xd, long long n, double* wide,
                                       float* narrow, double* rcp) {
  if (!xf || !xd || !wide || !narrow || !rcp || n < 0) return LYM1_EINVAL;
  if (n == 0) return LYM1_OK;
  const long long blocks = (n + 255) / 256;
  if (blocks > 0x7fffffffLL) return LYM1_EINVAL;
  lym1::fp64_helpers_kernel<<<static_cast<unsigned>(blocks), 256>>>(xf, xd, n, wide, narrow, rcp);
  if (cudaGetLastError() != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) {
    cudaGetLastError();
    return LYM1_ECUDA;
  }
  return LYM1_OK;
}
