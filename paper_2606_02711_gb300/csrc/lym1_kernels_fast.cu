// lym1_kernels_fast.cu -- dispatch to the kernels of the LYM1_FP64,
// LYM1_MIXED and LYM1_MIXED_FAST policies (FMA contraction allowed, hardware
// exp/expm1).  Each policy is instantiated in a translation unit of its own
// (lym1_pol_f64.cu, lym1_pol_mix.cu, lym1_pol_mixf.cu), compiled in parallel.
#include "lym1_kernels.cuh"
#include "lym1_policies.h"

namespace lym1 {

int launch_transport_fast(int precision, const DeviceView& v, void* st) {
  switch (precision) {
    case 1: return pol_f64::transport(v, st);
    case 2: return pol_mix::transport(v, st);
    case 3: return pol_mixf::transport(v, st);
    default: return static_cast<int>(cudaErrorInvalidValue);
  }
}

int launch_freq_fast(int precision, const DeviceView& v, void* st) {
  switch (precision) {
    case 1: return pol_f64::freq(v, st);
    case 2: return pol_mix::freq(v, st);
    case 3: return pol_mixf::freq(v, st);
    default: return static_cast<int>(cudaErrorInvalidValue);
  }
}

int launch_subcycle_fast(int precision, const DeviceView& v, void* st) {
  switch (precision) {
    case 1: return pol_f64::subcycle(v, st);
    case 2: return pol_mix::subcycle(v, st);
    case 3: return pol_mixf::subcycle(v, st);
    default: return static_cast<int>(cudaErrorInvalidValue);
  }
}

int launch_batched_fast(int precision, int kind, int geometry, int pt, const DeviceView* views,
                        const void* items, int n, int grid, int nb_max, void* st, int shape) {
  switch (precision) {
    case 1: return pol_f64::batched(kind, geometry, pt, views, items, n, grid, nb_max, st, shape);
    case 2: return pol_mix::batched(kind, geometry, pt, views, items, n, grid, nb_max, st, shape);
    case 3: return pol_mixf::batched(kind, geometry, pt, views, items, n, grid, nb_max, st, shape);
    default: return static_cast<int>(cudaErrorInvalidValue);
  }
}

int resident_blocks_fast(int precision, int kind, int geometry, int pt, int nb_max, int shape) {
  switch (precision) {
    case 1: return pol_f64::resident(kind, geometry, pt, nb_max, shape);
    case 2: return pol_mix::resident(kind, geometry, pt, nb_max, shape);
    case 3: return pol_mixf::resident(kind, geometry, pt, nb_max, shape);
    default: return 1;
  }
}

__global__ void fp64_helpers_kernel(const float* xf, const double* xd, long long n, double* wide,
                                    float* narrow, double* rcp, double* rcp1, double* rcpf) {
  const long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  wide[i] = f2d_alu(xf[i]);
  narrow[i] = d2f_alu(xd[i]);
  rcp[i] = drcp_nr(xd[i]);
  rcp1[i] = drcp_nr1(xd[i]);
  rcpf[i] = drcp_fs(xd[i]);
}

}  // namespace lym1

extern "C" int lym1_debug_fp64_helpers(const float* xf, const double* xd, long long n, double* wide,
                                       float* narrow, double* rcp, double* rcp1, double* rcpf) {
  if (!xf || !xd || !wide || !narrow || !rcp || !rcp1 || !rcpf || n < 0) return LYM1_EINVAL;
  if (n == 0) return LYM1_OK;
  const long long blocks = (n + 255) / 256;
  if (blocks > 0x7fffffffLL) return LYM1_EINVAL;
  lym1::fp64_helpers_kernel<<<static_cast<unsigned>(blocks), 256>>>(xf, xd, n, wide, narrow, rcp,
                                                                     rcp1, rcpf);
  if (cudaGetLastError() != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) {
    cudaGetLastError();
    return LYM1_ECUDA;
  }
  return LYM1_OK;
}
