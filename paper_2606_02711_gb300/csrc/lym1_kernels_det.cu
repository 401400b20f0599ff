// lym1_kernels_det.cu -- LYM1_FP64_DET kernels and the FP64 utility kernels.
// Built with -fmad=false: every FP64 operation is a separately rounded IEEE
// operation in the order written, which makes the substep reproducible to the
// last bit by any implementation that follows the same operation order.
#include "lym1_kernels.cuh"

namespace lym1 {

using PolDet = Policy<double, double, double, true>;

int launch_transport_det(const DeviceView& v, void* st) {
  return launch_transport_t<PolDet>(v, static_cast<cudaStream_t>(st));
}
int launch_freq_det(const DeviceView& v, void* st) {
  return launch_freq_t<PolDet>(v, static_cast<cudaStream_t>(st));
}

int launch_subcycle_det(const DeviceView& v, void* st) {
  return launch_subcycle_t<PolDet>(v, static_cast<cudaStream_t>(st));
}

int launch_batched_det(int kind, int geometry, int pt, const DeviceView* views, const void* items,
                       int n, int grid, int nb_max, void* st, int shape) {
  const cudaStream_t s = static_cast<cudaStream_t>(st);
  const BatchItem* it = static_cast<const BatchItem*>(items);
  if (kind == 0)
    return launch_transport_batched_t<PolDet>(geometry, pt, views, it, n, grid, nb_max, s, shape);
  if (kind == 1) return launch_freq_batched_t<PolDet>(geometry, pt, views, it, n, grid, nb_max, s);
  return launch_subcycle_batched_t<PolDet>(geometry, pt, views, it, n, grid, s);
}

int resident_blocks_det(int kind, int geometry, int pt, int nb_max, int shape) {
  if (kind == 0) return max_resident_transport<PolDet>(geometry, pt, nb_max, shape);
  if (kind == 1) return max_resident_freq<PolDet>(geometry, pt, nb_max);
  return max_resident_subcycle<PolDet>(geometry, pt);
}


// alpha = n_HI sigma0; velocity gradients by central differences over the
// two neighbours.  Geometry 0: ghosts = edge values (outflow boundaries).
// Geometry 1 (R = x, Z = y): the ghost across the axis (midplane) mirrors the
// first column (row) with u_R (u_Z) negated; <u_R / R> from the mean of the
// two R-face velocities over the mean face radius.
__global__ void setup_statics_kernel(const double* n_hi, const double* ux, const double* uy,
                                     double sigma0, const double* sigma0c, int nx, int ny,
                                     double dx, double* alpha, double* gxx, double* gyy,
                                     double* gsh, int geometry, double* gphi) {
  const long long id = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  const long long nc = static_cast<long long>(nx) * ny;
  if (id >= nc) return;
  const int i = static_cast<int>(id % nx), j = static_cast<int>(id / nx);
  const double h2 = 2.0 * dx;
  alpha[id] = n_hi[id] * (sigma0c ? sigma0c[id] : sigma0);
  if (geometry == 1) {
    bool fm, fp, gm, gp;
    const int im = ghost<1>(i - 1, nx, fm), ip = ghost<1>(i + 1, nx, fp);
    const int jm = ghost<1>(j - 1, ny, gm), jp = ghost<1>(j + 1, ny, gp);
    const long long row = static_cast<long long>(j) * nx;
    const double uRm = ux[row + im] * (fm ? -1.0 : 1.0);
    const double uRp = ux[row + ip];
    const double uZm = uy[static_cast<long long>(jm) * nx + i] * (gm ? -1.0 : 1.0);
    const double uZp = uy[static_cast<long long>(jp) * nx + i];
    const double uZl = uy[row + im], uZr = uy[row + ip];
    const double uRd = ux[static_cast<long long>(jm) * nx + i];
    const double uRu = ux[static_cast<long long>(jp) * nx + i];
    gxx[id] = (uRp - uRm) / h2;
    gyy[id] = (uZp - uZm) / h2;
    gsh[id] = (uRu - uRd) / h2 + (uZr - uZl) / h2;
    const double fL = 0.5 * (uRm + ux[id]), fR = 0.5 * (ux[id] + uRp);
    gphi[id] = (fR + fL) / ((i + 1) * dx + i * dx);
    return;
  }
  const long long xm = static_cast<long long>(j) * nx + clampi(i - 1, nx);
  const long long xp = static_cast<long long>(j) * nx + clampi(i + 1, nx);
  const long long ym = static_cast<long long>(clampi(j - 1, ny)) * nx + i;
  const long long yp = static_cast<long long>(clampi(j + 1, ny)) * nx + i;
  gxx[id] = (ux[xp] - ux[xm]) / h2;
  gyy[id] = (uy[yp] - uy[ym]) / h2;
  gsh[id] = (ux[yp] - ux[ym]) / h2 + (uy[xp] - uy[xm]) / h2;
}

int launch_setup_statics(const double* n_hi, const double* ux, const double* uy, double sigma0,
                         const double* sigma0c, int nx, int ny, double dx, double* alpha,
                         double* gxx, double* gyy, double* gsh, int geometry, double* gphi,
                         void* st) {
  const long long nc = static_cast<long long>(nx) * ny;
  const int blocks = static_cast<int>((nc + 255) / 256);
  setup_statics_kernel<<<blocks, 256, 0, static_cast<cudaStream_t>(st)>>>(
      n_hi, ux, uy, sigma0, sigma0c, nx, ny, dx, alpha, gxx, gyy, gsh, geometry, gphi);
  return static_cast<int>(cudaGetLastError());
}

__global__ void scale_columns_kernel(double* a, const double* w, int nx, long long nc) {
  for (long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; i < nc;
       i += static_cast<long long>(gridDim.x) * blockDim.x)
    a[i] = a[i] / w[i % nx];
}

template <class S>
__global__ void convert_out_kernel(const S* src, double* dst, long long n, double scale) {
  for (long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += static_cast<long long>(gridDim.x) * blockDim.x)
    dst[i] = scale * static_cast<double>(src[i]);
}
template <class S>
__global__ void convert_in_kernel(const double* src, S* dst, long long n) {
  for (long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += static_cast<long long>(gridDim.x) * blockDim.x)
    dst[i] = static_cast<S>(src[i]);
}

static int grid_for(long long n) {
  long long b = (n + 255) / 256;
  if (b > 152LL * 32) b = 152LL * 32;
  return static_cast<int>(b < 1 ? 1 : b);
}

int launch_scale_columns(double* lum, const double* V2pi, int nx, long long nc, void* st) {
  scale_columns_kernel<<<grid_for(nc), 256, 0, static_cast<cudaStream_t>(st)>>>(lum, V2pi, nx, nc);
  return static_cast<int>(cudaGetLastError());
}

int launch_convert_out(int precision, const void* src, double* dst, long long n, double scale,
                       void* st) {
  const cudaStream_t s = static_cast<cudaStream_t>(st);
  if (precision >= 2)
    convert_out_kernel<float><<<grid_for(n), 256, 0, s>>>(static_cast<const float*>(src), dst, n, scale);
  else
    convert_out_kernel<double><<<grid_for(n), 256, 0, s>>>(static_cast<const double*>(src), dst, n, scale);
  return static_cast<int>(cudaGetLastError());
}

int launch_convert_in(int precision, const double* src, void* dst, long long n, void* st) {
  const cudaStream_t s = static_cast<cudaStream_t>(st);
  if (precision >= 2)
    convert_in_kernel<float><<<grid_for(n), 256, 0, s>>>(src, static_cast<float*>(dst), n);
  else
    convert_in_kernel<double><<<grid_for(n), 256, 0, s>>>(src, static_cast<double*>(dst), n);
  return static_cast<int>(cudaGetLastError());
}

// energy of a state: per-block partials of sum_k dnu_k J_k (times the
// column weight on the axisymmetric grid)
template <class S>
__global__ void __launch_bounds__(kFreqThreads) energy_kernel(const S* J, const double* dnu, int nb,
                                                              long long nc, double* part,
                                                              const double* wcol, int nx) {
  __shared__ double red[kFreqThreads / 32];
  const long long cell = static_cast<long long>(blockIdx.x) * kFreqThreads + threadIdx.x;
  double en = 0.0;
  if (cell < nc) {
    for (int k = 0; k < nb; ++k) en += dnu[k] * static_cast<double>(J[static_cast<long long>(k) * nc + cell]);
    if (wcol) en *= wcol[cell % nx];
  }
  const double s = block_sum<kFreqThreads>(en, red);
  if (threadIdx.x == 0) part[static_cast<long long>(blockIdx.x) * kDiagSlots + kSlotEnergy] = s;
}

int launch_energy(int precision, const void* J, const double* dnu, int nb, long long nc,
                  double* part, const double* wcol, int nx, void* st) {
  const cudaStream_t s = static_cast<cudaStream_t>(st);
  if (precision >= 2)
    energy_kernel<float><<<freq_blocks(nc), kFreqThreads, 0, s>>>(static_cast<const float*>(J), dnu, nb, nc,
                                                                  part, wcol, nx);
  else
    energy_kernel<double><<<freq_blocks(nc), kFreqThreads, 0, s>>>(static_cast<const double*>(J), dnu, nb,
                                                                   nc, part, wcol, nx);
  return static_cast<int>(cudaGetLastError());
}

// Neumaier compensated accumulation a += v (a = {sum, compensation})
__device__ __forceinline__ void kahan_add(double* a, double v) {
  const double s = a[0], t = s + v;
  if (fabs(s) >= fabs(v))
    a[1] += (s - t) + v;
  else
    a[1] += (v - t) + s;
  a[0] = t;
}

// Fixed-order reduction of the per-block partials of one substep and
// accumulation into the context's running totals.
//   acc layout: [0..7] emitted, absorbed, outflow, work as (sum, comp) pairs,
//               [8] energy after the substep, [9] max f, [10] unrealisable count,
//               [11] substeps, [12] energy at the last reset, [13] energy unit
// mode 0: substep (flows from partT, energy/max f from partE);
// mode 1: reset (energy from partE; flows and counters zeroed);
// mode 2: substep whose step 2 ran in the subcycling kernel of the acceptance
//         rule (emitted and absorbed also from partE).
__device__ __forceinline__ void finalize_body(const double* partT, int nT, const double* partE,
                                              int nE, double* acc, int mode) {
  __shared__ double red[8];
  double v[kDiagSlots];
  for (int s = 0; s < kDiagSlots; ++s) v[s] = 0.0;
  const bool reset = (mode & 1) != 0;
  if (!reset)
    for (int b = threadIdx.x; b < nT; b += 256)
      for (int s = 0; s < 4; ++s) v[s] += partT[static_cast<long long>(b) * kDiagSlots + s];
  for (int b = threadIdx.x; b < nE; b += 256) {
    const double* p = partE + static_cast<long long>(b) * kDiagSlots;
    v[kSlotEnergy] += p[kSlotEnergy];
    if (!reset) {
      v[kSlotMaxF] = fmax(v[kSlotMaxF], p[kSlotMaxF]);
      v[kSlotBad] += p[kSlotBad];
      if (mode & 2) {  // step 2 ran in the subcycling kernel: its flows
        v[kSlotEmitted] += p[kSlotEmitted];
        v[kSlotAbsorbed] += p[kSlotAbsorbed];
      }
    }
  }
  double tot[kDiagSlots];
  for (int s = 0; s < kDiagSlots; ++s) {
    if (s == kSlotMaxF)
      tot[s] = block_max<256>(v[s], red);
    else
      tot[s] = block_sum<256>(v[s], red);
  }
  if (threadIdx.x == 0) {
    const double u = acc[13];
    if (reset) {
      for (int i = 0; i < 8; ++i) acc[i] = 0.0;
      acc[8] = u * tot[kSlotEnergy];
      acc[9] = 0.0;
      acc[10] = 0.0;
      acc[11] = 0.0;
      acc[12] = acc[8];
      acc[14] = 1e-8 * tot[kSlotEnergy];
    } else {
      kahan_add(acc + 0, u * tot[kSlotEmitted]);
      kahan_add(acc + 2, u * tot[kSlotAbsorbed]);
      kahan_add(acc + 4, u * tot[kSlotOutflow]);
      kahan_add(acc + 6, u * tot[kSlotWork]);
      acc[8] = u * tot[kSlotEnergy];
      acc[9] = tot[kSlotMaxF];
      acc[10] = tot[kSlotBad];
      acc[11] += 1.0;
      acc[14] = 1e-8 * tot[kSlotEnergy];  // FP32 realisability threshold on J dnu_k
    }
  }
}

__global__ void __launch_bounds__(256) finalize_kernel(const double* partT, int nT,
                                                       const double* partE, int nE,
                                                       double* acc, int mode) {
  finalize_body(partT, nT, partE, nE, acc, mode);
}

int launch_finalize(const double* partT, int nT, const double* partE, int nE, double* acc,
                    int mode, void* st) {
  finalize_kernel<<<1, 256, 0, static_cast<cudaStream_t>(st)>>>(partT, nT, partE, nE, acc, mode);
  return static_cast<int>(cudaGetLastError());
}

// force sums over cells: |f| dV and f . r_hat dV.  Geometry 0: r from the box
// centre, dV = dx^3.  Geometry 1: r from the origin (R, Z) = (0, 0), dV the
// ring volume 2 pi Vol of the cell.
__global__ void __launch_bounds__(256) force_reduce_kernel(const double* fx, const double* fy,
                                                           int nx, int ny, double dx,
                                                           int geometry, double* part) {
  __shared__ double red[8];
  const long long nc = static_cast<long long>(nx) * ny;
  double a = 0.0, r = 0.0;
  const double cx = geometry == 1 ? 0.0 : 0.5 * nx * dx, cy = geometry == 1 ? 0.0 : 0.5 * ny * dx;
  for (long long id = static_cast<long long>(blockIdx.x) * 256 + threadIdx.x; id < nc;
       id += static_cast<long long>(gridDim.x) * 256) {
    const int i = static_cast<int>(id % nx), j = static_cast<int>(id / nx);
    double V = (dx * dx) * dx;
    if (geometry == 1) {
      const double Rm = i * dx, Rp = (i + 1) * dx;
      V = (2.0 * kPi) * ((0.5 * (Rp * Rp - Rm * Rm)) * dx);
    }
    const double x = (i + 0.5) * dx - cx, y = (j + 0.5) * dx - cy, rr = sqrt(x * x + y * y);
    a += sqrt(fx[id] * fx[id] + fy[id] * fy[id]) * V;
    if (rr > 0.0) r += ((fx[id] * x + fy[id] * y) / rr) * V;
  }
  const double sa = block_sum<256>(a, red);
  const double sr = block_sum<256>(r, red);
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = sa;
    part[2 * blockIdx.x + 1] = sr;
  }
}

int launch_force_reduce(const double* fx, const double* fy, int nx, int ny, double dx,
                        int geometry, double* part, int nblocks, void* st) {
  force_reduce_kernel<<<nblocks, 256, 0, static_cast<cudaStream_t>(st)>>>(fx, fy, nx, ny, dx,
                                                                          geometry, part);
  return static_cast<int>(cudaGetLastError());
}

// Dynamic reduced speed of light (Sec. 2.1).  Per cell: tau_0 = alpha dx, the
// continuum absorption depth tau_c = rho_d kappa_abs dx, X = (a_v tau_0)^(1/3)
// with a_v at the cell's temperature, f_abs = 1 / (1 + X tau_c + 0.6 p_d tau_0)
// and the term max[1, X f_abs] max[|u|, c_s]; c_s from cs, else that of neutral
// atomic gas at T (gamma = 5/3, mu = 1.22).  The terms are >= 0, so the
// maximum over cells is a 64-bit atomicMax on their IEEE bit patterns (one
// per block); NaN terms are dropped by fmax.
__global__ void __launch_bounds__(256) ctilde_reduce_kernel(
    const double* alpha, const double* rho, const double* pd, const double* ux, const double* uy,
    const double* Tc, double T, const double* cs, double kabs, double dx, long long nc,
    unsigned long long* mx) {
  __shared__ double red[8];
  double m = 0.0;
  for (long long id = static_cast<long long>(blockIdx.x) * 256 + threadIdx.x; id < nc;
       id += static_cast<long long>(gridDim.x) * 256) {
    const double Tk = Tc ? Tc[id] : T;
    const double dnuD = (kNuLya * sqrt((2.0 * kBoltzmann * Tk) / kMassH)) / kLight;
    const double a_v = kEinsteinA / ((4.0 * kPi) * dnuD);
    const double tau0 = alpha[id] * dx;
    const double tauc = (rho[id] * kabs) * dx;
    const double X = cbrt(a_v * tau0);
    const double fa = 1.0 / ((1.0 + X * tauc) + (0.6 * pd[id]) * tau0);
    const double u = sqrt(ux[id] * ux[id] + uy[id] * uy[id]);
    const double s = cs ? cs[id] : sqrt(((5.0 / 3.0) * (kBoltzmann * Tk)) / (1.22 * kMassH));
    m = fmax(m, fmax(1.0, X * fa) * fmax(u, s));
  }
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < 8; ++w) m = fmax(m, red[w]);
    atomicMax(mx, static_cast<unsigned long long>(__double_as_longlong(m)));
  }
}

// c_tilde = min[max(c_min, eps_RSL max), c], then at most -25 % / x4 from prev
__global__ void ctilde_finalize_kernel(const unsigned long long* mx, double eps, double ct_min,
                                       double prev, double* out) {
  const double m = __longlong_as_double(static_cast<long long>(*mx));
  double ct = fmin(fmax(ct_min, eps * m), kLight);
  ct = fmin(fmax(ct, 0.75 * prev), 4.0 * prev);
  *out = ct;
}

int launch_dynamic_ctilde(const double* alpha, const double* rho, const double* pd,
                          const double* ux, const double* uy, const double* Tc, double T,
                          const double* cs, double kabs, double dx, long long nc, double eps,
                          double ct_min, double prev, unsigned long long* work, void* st) {
  const cudaStream_t s = static_cast<cudaStream_t>(st);
  cudaError_t e = cudaMemsetAsync(work, 0, sizeof(unsigned long long), s);
  if (e != cudaSuccess) return static_cast<int>(e);
  ctilde_reduce_kernel<<<grid_for(nc), 256, 0, s>>>(alpha, rho, pd, ux, uy, Tc, T, cs, kabs, dx,
                                                   nc, work);
  ctilde_finalize_kernel<<<1, 1, 0, s>>>(work, eps, ct_min, prev,
                                         reinterpret_cast<double*>(work + 1));
  return static_cast<int>(cudaGetLastError());
}

// ---------------------------------------------------------------------------
// Per-cell A0 on the device (App. A: <H>_k at each cell's temperature; Sec. 2.1
// step 2: emission fractions w_k = <H>_k dx_k / sum; Sec. 2.1: Doppler width,
// a_v, sigma0), for temperature fields that change between hydro steps.  The
// same steps, in the same order, as the host tables of lym1_tables.cpp, with
// CUDA's exp / erf / erfc in place of the host library's.

// Dawson's integral: Maclaurin series below 0.2, Rybicki's sampling sum with
// h = 0.2 below 10, the asymptotic series above
__device__ double dawson_dev(double x) {
  const double ax = fabs(x);
  double f;
  if (ax < 0.2) {
    const double x2 = ax * ax;
    double term = ax;
    f = ax;
    for (int n = 1; n <= 12; ++n) {
      term = (term * (-2.0 * x2)) / (2.0 * n + 1.0);
      f += term;
    }
  } else if (ax < 10.0) {
    const double h = 0.2;
    const int lo = static_cast<int>(ceil((ax - 8.0) / h));
    const int hi = static_cast<int>(floor((ax + 8.0) / h));
    double s = 0.0;
    for (int n = lo; n <= hi; ++n) {
      if ((n & 1) == 0) continue;
      const double d = ax - n * h;
      s += exp(-d * d) / n;
    }
    f = s / kSqrtPi;
  } else {
    const double y = 1.0 / (2.0 * ax * ax);
    double term = 1.0, s = 1.0;
    for (int n = 1; n <= 20; ++n) {
      term = term * ((2.0 * n - 1.0) * y);
      s += term;
    }
    f = s / (2.0 * ax);
  }
  return x < 0.0 ? -f : f;
}

// The a-dependent terms of I(x, a): -(2a/sqrt(pi)) F(x) + a^2 x exp(-x^2)
__device__ double voigt_rest_dev(double x, double a) {
  return -((2.0 * a) / kSqrtPi) * dawson_dev(x) + ((a * a) * x) * exp(-(x * x));
}

// One thread per cell.  Writes the per-[bin][cell] <H>_k and emission factors
// in the state type S (FP32: the factors over the cell's maximum, kept in
// gmaxc), sigma0, h/(k_B T) (0 without recoil or for a gray group),
// dnu_D^2 / 2, alpha = n_HI sigma0 and the temperature itself.  <H>_k goes
// straight into Hc; the normalisation sum always takes the FP64 value, and the
// emission factors are formed from Hc (exact for FP64 state, the stored FP32
// value otherwise).  A gray group (one table entry per cell) forms <H>_k twice.
template <class S>
__global__ void __launch_bounds__(128) cell_tables_kernel(
    const double* T, const double* nhi, const double* edges, int n, int gray, int recoil,
    int geometry, double dx, long long nc, S* Hc, S* Gc, double* gmaxc, double* Kcc,
    double* hkTc, double* sig0c, double* alpha, double* Tc) {
  const long long cell = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (cell >= nc) return;
  const double t = T[cell];
  const double dnuD = (kNuLya * sqrt((2.0 * kBoltzmann * t) / kMassH)) / kLight;
  const double a_v = kEinsteinA / ((4.0 * kPi) * dnuD);
  const double sigma0 = ((kSqrtPi * (kCharge * kCharge)) * kOscStrength) / ((kMassE * kLight) * dnuD);
  // <H> over [xa, xb] (Doppler units): the erf difference through erfc on the
  // side away from line centre, plus the a-dependent terms; each edge's erfc
  // and I-terms are formed once and carried to the next bin.  pass 0 sums the
  // emission weights (and stores <H>_k), pass 1 (gray group only) forms eta.
  double S_ = 0.0, eta = 0.0;
  for (int pass = 0; pass < (gray ? 2 : 1); ++pass) {
    double xa = edges[0] / dnuD;
    double ea = erfc(fabs(xa)), ra = voigt_rest_dev(xa, a_v);
    for (int k = 0; k < n; ++k) {
      const double dnu = edges[k + 1] - edges[k];
      const double xb = edges[k + 1] / dnuD;
      const double dxk = dnu / dnuD;
      const double eb = erfc(fabs(xb)), rb = voigt_rest_dev(xb, a_v);
      double derf;
      if (xa >= 0.0)
        derf = (kSqrtPi / 2.0) * (ea - eb);
      else if (xb <= 0.0)
        derf = (kSqrtPi / 2.0) * (eb - ea);
      else
        derf = (kSqrtPi / 2.0) * (erf(xb) - erf(xa));
      const double Hv = (derf + (rb - ra)) / dxk;
      if (pass == 0) {
        if (!gray) Hc[static_cast<long long>(k) * nc + cell] = S(Hv);
        S_ += Hv * dxk;
      } else {
        eta += ((Hv * dxk) / S_) * Hv;
      }
      xa = xb;
      ea = eb;
      ra = rb;
    }
  }
  const double V = geometry == 1 ? 1.0 : (dx * dx) * dx;
  const double fourpiV = (4.0 * kPi) * V;
  double gmax = 0.0;
  if (gray) {
    gmax = 1.0 / fourpiV;
    Hc[cell] = S(eta);
    Gc[cell] = sizeof(S) == 8 ? S(gmax) : S(1.0);
  } else {
    for (int k = 0; k < n; ++k) {
      const double dnu = edges[k + 1] - edges[k];
      const double Hv = double(Hc[static_cast<long long>(k) * nc + cell]);
      const double g = ((Hv * (dnu / dnuD)) / S_) / (fourpiV * dnu);
      gmax = fmax(gmax, g);
      if (sizeof(S) == 8) Gc[static_cast<long long>(k) * nc + cell] = S(g);
    }
    if (!(gmax > 0.0)) gmax = 1.0;
    if (sizeof(S) == 4)
      for (int k = 0; k < n; ++k) {
        const double dnu = edges[k + 1] - edges[k];
        const double Hv = double(Hc[static_cast<long long>(k) * nc + cell]);
        const double g = ((Hv * (dnu / dnuD)) / S_) / (fourpiV * dnu);
        Gc[static_cast<long long>(k) * nc + cell] = S(g / gmax);
      }
  }
  gmaxc[cell] = gmax;
  sig0c[cell] = sigma0;
  hkTc[cell] = (recoil && !gray) ? kPlanck / (kBoltzmann * t) : 0.0;
  Kcc[cell] = 0.5 * (dnuD * dnuD);
  alpha[cell] = nhi[cell] * sigma0;
  Tc[cell] = t;
}

int launch_cell_tables(int selem, const double* T, const double* nhi, const double* edges, int n,
                       int gray, int recoil, int geometry, double dx, long long nc, void* Hc,
                       void* Gc, double* gmaxc, double* Kcc, double* hkTc, double* sig0c,
                       double* alpha, double* Tc, void* st) {
  const cudaStream_t s = static_cast<cudaStream_t>(st);
  const int blocks = static_cast<int>((nc + 127) / 128);
  if (selem == 8)
    cell_tables_kernel<double><<<blocks, 128, 0, s>>>(T, nhi, edges, n, gray, recoil, geometry, dx,
                                                      nc, static_cast<double*>(Hc),
                                                      static_cast<double*>(Gc), gmaxc, Kcc, hkTc,
                                                      sig0c, alpha, Tc);
  else
    cell_tables_kernel<float><<<blocks, 128, 0, s>>>(T, nhi, edges, n, gray, recoil, geometry, dx,
                                                     nc, static_cast<float*>(Hc),
                                                     static_cast<float*>(Gc), gmaxc, Kcc, hkTc,
                                                     sig0c, alpha, Tc);
  return static_cast<int>(cudaGetLastError());
}

// Active-bin pruning (Sec. 2.2): the energy of each bin, dnu_k sum_cells w J_k
// with w the column weight of the axisymmetric grid (1 on the Cartesian one).
// Each bin plane is split into kBinChunks chunks, one block each; a block sums
// its chunk in a fixed order (FP32 state: per-thread compensated FP32 sums,
// accurate to ~1e-12, since GB300's FP64 pipe runs at ~1/60 of FP32; FP64
// state: FP64), then one thread adds the chunks in order, forms the total in
// bin order and makes the strict cut of the bins that step 1 advects.
constexpr int kBinChunks = 16;

template <class S>
__global__ void __launch_bounds__(256) bin_energy_kernel(const S* J, long long nc, int nx,
                                                         const double* wcol, double* part) {
  __shared__ double red[8];
  const int k = blockIdx.y, ch = blockIdx.x;
  const S* Jk = J + static_cast<long long>(k) * nc;
  const long long per = (nc + kBinChunks - 1) / kBinChunks;
  const long long lo = static_cast<long long>(ch) * per;
  const long long hi = lo + per < nc ? lo + per : nc;
  double v;
  if constexpr (sizeof(S) == 4) {
    float s = 0.0f, c = 0.0f;
    for (long long id = lo + threadIdx.x; id < hi; id += 256) {
      const float x = wcol ? Jk[id] * float(wcol[id % nx]) : Jk[id];
      const float t = s + x;
      if (fabsf(s) >= fabsf(x))
        c += (s - t) + x;
      else
        c += (x - t) + s;
      s = t;
    }
    v = double(s) + double(c);
  } else {
    v = 0.0;
    for (long long id = lo + threadIdx.x; id < hi; id += 256)
      v += wcol ? double(Jk[id]) * wcol[id % nx] : double(Jk[id]);
  }
  v = block_sum<256>(v, red);
  if (threadIdx.x == 0) part[static_cast<long long>(k) * kBinChunks + ch] = v;
}

__global__ void active_bins_kernel(const double* part, const double* dnu, int nb, double cut,
                                   double* E, unsigned char* active) {
  double tot = 0.0;
  for (int k = 0; k < nb; ++k) {
    double s = 0.0;
    for (int ch = 0; ch < kBinChunks; ++ch) s += part[k * kBinChunks + ch];
    E[k] = dnu[k] * s;
    tot += E[k];
  }
  const double c = cut * tot;
  for (int k = 0; k < nb; ++k) active[k] = E[k] > c ? 1 : 0;
}

int launch_active_bins(int selem, const void* J, int nb, long long nc, int nx, const double* wcol,
                       const double* dnu, double cut, double* E, unsigned char* active, void* st) {
  const cudaStream_t s = static_cast<cudaStream_t>(st);
  double* part = E + nb;  // E holds nb energies, then nb x kBinChunks partials
  const dim3 grid(kBinChunks, nb);
  if (selem == 8)
    bin_energy_kernel<double><<<grid, 256, 0, s>>>(static_cast<const double*>(J), nc, nx, wcol, part);
  else
    bin_energy_kernel<float><<<grid, 256, 0, s>>>(static_cast<const float*>(J), nc, nx, wcol, part);
  active_bins_kernel<<<1, 1, 0, s>>>(part, dnu, nb, cut, E, active);
  return static_cast<int>(cudaGetLastError());
}

// Sum of a per-cell array (the luminosity), in a fixed order: a fixed grid of
// grid-stride block partials, which the last block to finish adds in block order
// (the count returns to 0 for the next call).  Nothing waits on another block.
constexpr int kSumBlocks = 152;

__global__ void __launch_bounds__(256) sum_cells_kernel(const double* a, long long n, double* part,
                                                        unsigned* count, double* out) {
  __shared__ double red[8];
  __shared__ int last;
  double s = 0.0;
  for (long long id = static_cast<long long>(blockIdx.x) * 256 + threadIdx.x; id < n;
       id += static_cast<long long>(gridDim.x) * 256)
    s += a[id];
  s = block_sum<256>(s, red);
  if (threadIdx.x == 0) {
    part[blockIdx.x] = s;
    __threadfence();
    last = atomicAdd(count, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (last && threadIdx.x == 0) {
    __threadfence();
    double t = 0.0;
    for (int b = 0; b < static_cast<int>(gridDim.x); ++b) t += __ldcg(part + b);
    *out = t;
    *count = 0u;
  }
}

int launch_sum_cells(const double* a, long long n, double* work, void* st) {
  // work: kSumBlocks partials, the result, then the counter (in the next word)
  sum_cells_kernel<<<kSumBlocks, 256, 0, static_cast<cudaStream_t>(st)>>>(
      a, n, work, reinterpret_cast<unsigned*>(work + kSumBlocks + 1), work + kSumBlocks);
  return static_cast<int>(cudaGetLastError());
}

// one block per context: the per-substep reduction of finalize_kernel for a batch
__global__ void __launch_bounds__(256) finalize_batched_kernel(const FinalizeJob* jobs) {
  const FinalizeJob j = jobs[blockIdx.x];
  finalize_body(j.partT, j.nT, j.partE, j.nE, j.acc, j.mode);
}

int launch_finalize_batched(const FinalizeJob* jobs, int n, void* st) {
  finalize_batched_kernel<<<n, 256, 0, static_cast<cudaStream_t>(st)>>>(jobs);
  return static_cast<int>(cudaGetLastError());
}

}  // namespace lym1
