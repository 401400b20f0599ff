// lym1_noalloc.cu -- lym1_energy_noalloc: the domain Lya energy of a
// caller-owned state, computed without allocating any device memory.
//
// Some callers cannot call cudaMalloc at the moment they need this number: a
// host code whose device memory is owned by another runtime's allocator (a
// framework that preallocates most of HBM), or a real-time loop that forbids
// allocation.  This entry point runs the same two-stage reduction as the
// library's own energy bookkeeping, with its per-block partial sums in a
// file-scope device array of fixed size instead of a context's allocation.
#include <cuda_runtime.h>

#include <mutex>

#include "lym1.h"
#include "lym1_kernels.cuh"

namespace lym1 {
namespace {

constexpr int kNoAllocMaxBlocks = static_cast<int>(
    (static_cast<long long>(LYM1_NOALLOC_MAX_CELLS) + kFreqThreads - 1) / kFreqThreads);

// Shared scratch: one partial sum per block, then the result.  Every GPU that
// loads the library holds it (1 MiB + 8 B) until the process exits.  In host
// code this name is only a stand-in for the device array; kernels get its
// device address from cudaGetSymbolAddress.
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocMaxBlocks + 1];

struct NoAllocArgs {
  const double* J;
  long long nc;
  int nb;
  double unit;
  double dnu[LYM1_NOALLOC_MAX_BINS];
};

// Stage 1: per-thread sum_k dnu_k J_k, block sums in fixed order (the same
// partition and order as the library's energy kernel, whose translation unit
// is built without FMA contraction: the explicitly rounded product and sum
// keep the two bit-identical).
__global__ void __launch_bounds__(kFreqThreads) noalloc_energy_blocks(const NoAllocArgs a,
                                                                      double* scratch) {
  __shared__ double red[kFreqThreads / 32];
  const long long cell = static_cast<long long>(blockIdx.x) * kFreqThreads + threadIdx.x;
  double en = 0.0;
  if (cell < a.nc)
    for (int k = 0; k < a.nb; ++k)
      en = __dadd_rn(en, __dmul_rn(a.dnu[k], a.J[static_cast<long long>(k) * a.nc + cell]));
  const double s = block_sum<kFreqThreads>(en, red);
  if (threadIdx.x == 0) scratch[blockIdx.x] = s;
}

// Stage 2: one block sums the partials of this call (strided, then in warp
// order) and stores unit * total after them.  Only slots written by stage 1 of
// the same call are read, so nothing needs clearing between calls.
__global__ void __launch_bounds__(256) noalloc_energy_total(int nblocks, double unit,
                                                            double* scratch) {
  __shared__ double red[8];
  double v = 0.0;
  for (int b = threadIdx.x; b < nblocks; b += 256) v += scratch[b];
  const double t = block_sum<256>(v, red);
  if (threadIdx.x == 0) scratch[kNoAllocMaxBlocks] = unit * t;
}

std::mutex g_setup_mutex;
double* g_scratch_ptr[256] = {};

// Device address of the scratch array for the current device, looked up once
// per device with that device current.
int scratch_for_current_device(double** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) {
    cudaGetLastError();
    return LYM1_ENODEVICE;
  }
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return LYM1_ECUDA;
    }
    g_scratch_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_ptr[dev];
  return LYM1_OK;
}

// J must be device memory of the current device: the kernels dereference it
// directly, and the scratch address is the current device's.  The attribute
// query allocates nothing.
bool on_current_device(const void* p) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return false;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) return false;
  return (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) && at.device == dev;
}

}  // namespace
}  // namespace lym1

extern "C" int lym1_energy_noalloc(const double* J, const double* dnu, int nb, long long nc,
                                   double dx_cm, double* e_out, void* cuda_stream) {
  using namespace lym1;
  if (!J || !dnu || !e_out || !(dx_cm > 0.0)) return LYM1_EINVAL;
  if (nb < 1 || nc < 1) return LYM1_EINVAL;
  if (nb > LYM1_NOALLOC_MAX_BINS || nc > LYM1_NOALLOC_MAX_CELLS) return LYM1_ERANGE;
  // an error the caller left pending stays theirs: report it, do not clear it
  if (cudaPeekAtLastError() != cudaSuccess) return LYM1_ECUDA;
  // from here on any pending error comes from this call, which clears it
  if (!on_current_device(J)) {
    cudaGetLastError();
    return LYM1_EINVAL;
  }
  double* scratch = nullptr;
  const int rc = scratch_for_current_device(&scratch);
  if (rc != LYM1_OK) return rc;
  const cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  NoAllocArgs a;
  a.J = J;
  a.nc = nc;
  a.nb = nb;
  const double V = (dx_cm * dx_cm) * dx_cm;
  a.unit = ((4.0 * kPi) / kLight) * V;
  for (int k = 0; k < nb; ++k) a.dnu[k] = dnu[k];
  const int nblocks = static_cast<int>((nc + kFreqThreads - 1) / kFreqThreads);
  noalloc_energy_blocks<<<nblocks, kFreqThreads, 0, st>>>(a, scratch);
  noalloc_energy_total<<<1, 256, 0, st>>>(nblocks, a.unit, scratch);
  if (cudaGetLastError() != cudaSuccess) return LYM1_ECUDA;
  if (cudaMemcpyAsync(e_out, scratch + kNoAllocMaxBlocks, sizeof(double), cudaMemcpyDefault, st) !=
          cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess) {
    cudaGetLastError();
    return LYM1_ECUDA;
  }
  return LYM1_OK;
}
