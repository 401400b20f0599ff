// lym1_kernels.cuh -- sm_103a kernels of one Lya M1 substep (arXiv 2606.02711).
//
// Included by two translation units: lym1_kernels_det.cu (built with
// -fmad=false; the LYM1_FP64_DET policy) and lym1_kernels_fast.cu (FMA on; the
// LYM1_FP64, LYM1_MIXED and LYM1_MIXED_FAST policies).  A policy fixes the
// storage type S of the state, the type F of the transport fluxes and closure,
// the type I of the implicit steps and whether the fixed-order FP64 recipe with
// this file's own exp/expm1 is used.
//
// Kernels of one substep (state ping-pong A -> B -> A):
//   transport_kernel  rows A1-A5: per 32x8 cell tile, loops over all bins; per
//                     bin the (tile + 2) halo of J, Hx, Hy goes to shared memory,
//                     every face flux is computed once, then the explicit update,
//                     the implicit source step and the force sum (bins in order).
//   freq_kernel       row A6: one thread per cell, forward sweep of the
//                     subtraction-free tridiagonal elimination over the bins
//                     (elimination factors kept in the output arrays), then the
//                     back substitution and H <- (J_new/J_old) H.
//   finalize_kernel   row A7: fixed-order sums of the per-block partials.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "lym1.h"
#include "lym1_internal.h"

namespace lym1 {

template <class S_, class F_, class I_, bool DET_>
struct Policy {
  using S = S_;  // state storage
  using F = F_;  // transport fluxes, closure, frequency-step coefficients
  using I = I_;  // implicit source step, elimination, force and energy sums
  static constexpr bool DET = DET_;
};

// ------------------------------------------------------------------ exp/expm1
// Own exp/expm1 for the deterministic policy: Cody-Waite reduction
// x = n ln2 + r (|r| <= ln2/2; ln2 split into a 32-bit head and the rounded
// tail), degree-13 Taylor polynomial of expm1(r), scaling by 2^n.
__device__ __forceinline__ double own_pow2i(int n) {
  return __longlong_as_double(static_cast<long long>(n + 1023) << 52);
}

__device__ __forceinline__ double own_expm1_poly(double r) {
  double q = 1.0 / 6227020800.0;
  q = q * r + 1.0 / 479001600.0;
  q = q * r + 1.0 / 39916800.0;
  q = q * r + 1.0 / 3628800.0;
  q = q * r + 1.0 / 362880.0;
  q = q * r + 1.0 / 40320.0;
  q = q * r + 1.0 / 5040.0;
  q = q * r + 1.0 / 720.0;
  q = q * r + 1.0 / 120.0;
  q = q * r + 1.0 / 24.0;
  q = q * r + 1.0 / 6.0;
  q = q * r + 1.0 / 2.0;
  return r + (r * r) * q;
}

__device__ __forceinline__ void own_reduce(double x, int& n, double& r) {
  const double kInvLn2 = 0x1.71547652b82fep+0;
  const double kLn2Hi = 0x1.62e42feep-1;
  const double kLn2Lo = 0x1.a39ef35793c76p-33;
  const double t = floor(x * kInvLn2 + 0.5);
  n = static_cast<int>(t);
  r = (x - t * kLn2Hi) - t * kLn2Lo;
}

__device__ inline double own_exp(double x) {
  if (x != x) return x;
  if (x > 709.782712893384) return __longlong_as_double(0x7ff0000000000000LL);
  if (x < -745.2) return 0.0;
  int n;
  double r;
  own_reduce(x, n, r);
  const double s = 1.0 + own_expm1_poly(r);
  if (n > 1023) return (s * 2.0) * own_pow2i(n - 1);
  if (n >= -1022) return s * own_pow2i(n);
  return (s * own_pow2i(n + 1022)) * own_pow2i(-1022);
}

__device__ inline double own_expm1(double x) {
  if (x != x) return x;
  if (x > 709.782712893384) return __longlong_as_double(0x7ff0000000000000LL);
  if (x < -745.2) return -1.0;
  int n;
  double r;
  own_reduce(x, n, r);
  const double p = own_expm1_poly(r);
  if (n == 0) return p;
  if (n < -1022) return -1.0;
  if (n > 1023) return (p + 1.0) * 2.0 * own_pow2i(n - 1);
  const double t = own_pow2i(n);
  return t * p + (t - 1.0);
}

template <bool DET>
__device__ __forceinline__ double m_exp(double x) {
  if constexpr (DET) return own_exp(x);
  else return exp(x);
}
template <bool DET>
__device__ __forceinline__ double m_expm1(double x) {
  if constexpr (DET) return own_expm1(x);
  else return expm1(x);
}
template <bool DET>
__device__ __forceinline__ float m_exp(float x) { return __expf(x); }
template <bool DET>
__device__ __forceinline__ float m_expm1(float x) { return expm1f(x); }

template <class F>
__device__ __forceinline__ F m_sqrt(F x) { return sqrt(x); }

// ------------------------------------------------------------ closure & flux
// Levermore M1 closure (Sec. 2.1): D = (1-chi)/2 I + (3chi-1)/2 h h with
// chi = (3 + 4f^2) / (5 + 2 sqrt(4 - 3f^2)); components for f = (fn, ft).
// FP64 evaluates the formula as written.  FP32 uses the exact rearrangement
// (with s = sqrt(4 - 3f^2))
//   (1-chi)/2 = (1 + s - 2f^2) / (5 + 2s),  (3chi-1)/(2f^2) = (6 + 3/(2+s)) / (5 + 2s),
// because 3chi - 1 ~ 1.5 f^2 cancels to noise in FP32 when f is small
// (optically thick cells, f ~ 1/tau).
// Dpp = (1-chi)/2 is the component along any direction normal to f (the
// azimuthal one on the axisymmetric grid).
template <class F>
__device__ __forceinline__ void closure(F fn, F ft, F& Dnn, F& Dnt, F& Dtt, F& Dpp) {
  const F f2 = fn * fn + ft * ft;
  if constexpr (sizeof(F) == 4) {
    const F s = sqrtf(F(4) - F(3) * f2);
    const F inv = F(1) / (F(5) + F(2) * s);
    const F dA = (F(1) + s - F(2) * f2) * inv;
    const F g = (F(6) + F(3) / (F(2) + s)) * inv;
    Dnn = dA + g * (fn * fn);
    Dnt = g * (fn * ft);
    Dtt = dA + g * (ft * ft);
    Dpp = dA;
  } else {
    const F chi = (F(3) + F(4) * f2) / (F(5) + F(2) * m_sqrt(F(4) - F(3) * f2));
    const F dA = (F(1) - chi) / F(2), dB = (F(3) * chi - F(1)) / F(2);
    Dpp = dA;
    if (f2 > F(0)) {
      Dnn = dA + (dB * (fn * fn)) / f2;
      Dnt = (dB * (fn * ft)) / f2;
      Dtt = dA + (dB * (ft * ft)) / f2;
    } else {
      Dnn = dA;
      Dnt = F(0);
      Dtt = dA;
    }
  }
}

template <class F>
__device__ __forceinline__ void closure(F fn, F ft, F& Dnn, F& Dnt, F& Dtt) {
  F Dpp;
  closure(fn, ft, Dnn, Dnt, Dtt, Dpp);
}

// FP64 closure for the tuned policy: with s = sqrt(4 - 3f^2) the printed chi is
// (5 - 2s)/3, so (1-chi)/2 = (s - 1)/3 and (3chi - 1)/(2f^2) = 3/(2 + s): one
// square root and one division instead of the printed form's three divisions
// (GB300's FP64 division is a multi-instruction sequence on a 1/64-rate pipe).
// LYM1_FP64_DET keeps the printed form and its operation order.
template <bool DET>
__device__ __forceinline__ void closure_d(double fn, double ft, double& Dnn, double& Dnt,
                                          double& Dtt, double& Dpp) {
  if constexpr (DET) {
    closure(fn, ft, Dnn, Dnt, Dtt, Dpp);
  } else {
    const double f2 = fn * fn + ft * ft;
    const double s = sqrt(4.0 - 3.0 * f2);
    const double dA = (s - 1.0) * (1.0 / 3.0);
    const double g = 3.0 / (2.0 + s);
    Dnn = dA + g * (fn * fn);
    Dnt = g * (fn * ft);
    Dtt = dA + g * (ft * ft);
    Dpp = dA;
  }
}

// Causality after the frequency step (Sec. 2.1 step 3: |H|/J <= 1 with H
// rescaled by J_new/J_old): an H longer than J is shortened to J along its
// direction; H = 0 where J <= 0.
// FP64: the square root is taken only when |H|^2 > J^2, which leaves the
// decision |H| > J unchanged (sqrt(fl(J J)) = J for a correctly rounded
// product and square root in binary arithmetic without under/overflow) and
// keeps the result bit-identical to the plain form.
template <class I>
__device__ __forceinline__ void causal(I J, I& Hx, I& Hy) {
  if constexpr (sizeof(I) == 8) {
    if (J > I(0)) {
      const I h2 = Hx * Hx + Hy * Hy;
      if (h2 > J * J) {
        const I hn = sqrt(h2);
        if (hn > J) {
          const I s = J / hn;
          Hx = Hx * s;
          Hy = Hy * s;
        }
      }
    } else {
      Hx = I(0);
      Hy = I(0);
    }
  } else {
    if (J > 0.0f) {
      const float h2 = Hx * Hx + Hy * Hy;
      if (h2 > J * J) {
        const float s = J * rsqrtf(h2);
        Hx *= s;
        Hy *= s;
      }
    } else {
      Hx = 0.0f;
      Hy = 0.0f;
    }
  }
}

// Running sum: plain in FP64, Neumaier-compensated in FP32.
template <class T>
struct RSum {
  T s = T(0), c = T(0);
  __device__ __forceinline__ void add(T v) {
    if constexpr (sizeof(T) == 8) {
      s += v;
    } else {
      const T t = s + v;
      if (fabsf(s) >= fabsf(v))
        c += (s - t) + v;
      else
        c += (v - t) + s;
      s = t;
    }
  }
  __device__ __forceinline__ double value() const { return double(s) + double(c); }
};

template <class F>
__device__ __forceinline__ F minmod(F a, F b) {
  if (a > F(0) && b > F(0)) return a < b ? a : b;
  if (a < F(0) && b < F(0)) return a > b ? a : b;
  return F(0);
}

// |f| > 1: scale the components down to the unit circle
template <class F>
__device__ __forceinline__ void cap_unit(F& fn, F& ft) {
  const F f2 = fn * fn + ft * ft;
  if (f2 > F(1)) {
    const F r = m_sqrt(f2);
    fn = fn / r;
    ft = ft / r;
  }
}

// Flux across the face between cells 0 and 1 along normal n (Sec. 2.1 step 1):
// MinMod reconstruction of J, f_n, f_t from cells -1, 0, +1, +2; interface
// rescale of |f| > 1; corrected GLF flux of J; modified GLF flux of K; upwind
// advection with the mean face velocity (reconstructed donor state).
template <class F, bool DET = true>
__device__ __forceinline__ void face_flux(F Jm, F nm, F tm, F J0, F n0, F t0, F J1, F n1, F t1,
                                          F J2, F n2, F t2, F aF0, F aF1, F un0, F un1,
                                          F dl0, F dl1, F& oJ, F& oN, F& oT) {
  const F sJ0 = minmod(J0 - Jm, J1 - J0), sJ1 = minmod(J1 - J0, J2 - J1);
  const F sn0 = minmod(n0 - nm, n1 - n0), sn1 = minmod(n1 - n0, n2 - n1);
  const F st0 = minmod(t0 - tm, t1 - t0), st1 = minmod(t1 - t0, t2 - t1);
  const F JL = J0 + F(0.5) * sJ0, JR = J1 - F(0.5) * sJ1;
  F nL = n0 + F(0.5) * sn0, tL = t0 + F(0.5) * st0;
  F nR = n1 - F(0.5) * sn1, tR = t1 - F(0.5) * st1;
  cap_unit(nL, tL);
  cap_unit(nR, tR);
  const F HnL = JL * nL, HtL = JL * tL, HnR = JR * nR, HtR = JR * tR;
  F DnnL, DntL, DttL, DnnR, DntR, DttR, DppL, DppR;
  closure_d<DET>(nL, tL, DnnL, DntL, DttL, DppL);
  closure_d<DET>(nR, tR, DnnR, DntR, DttR, DppR);
  const F KnnL = DnnL * JL, KntL = DntL * JL, KnnR = DnnR * JR, KntR = DntR * JR;
  // face optical depth from the two cells' centres (centroids) to the face
  const F tau = aF0 * dl0 + aF1 * dl1;
  F eps, dif;
  if constexpr (DET) {
    eps = (F(0.2) + tau) / ((F(0.2) + tau) + tau * tau);
    dif = (tau > F(0)) ? ((F(1) - eps) * (J1 - J0)) / (F(3) * tau) : F(0);
  } else {  // one division: (1 - eps)/(3 tau) = tau / (3 d), d = 0.2 + tau + tau^2
    const F rd = F(1) / ((F(0.2) + tau) + tau * tau);
    eps = (F(0.2) + tau) * rd;
    dif = (tau * rd) * (F(1) / F(3)) * (J1 - J0);
  }
  F fJ = (eps * (F(0.5) * (HnL + HnR)) - eps * (F(0.5) * (JR - JL))) - dif;
  F fN = F(0.5) * (KnnL + KnnR) - eps * (F(0.5) * (HnR - HnL));
  F fT = F(0.5) * (KntL + KntR) - eps * (F(0.5) * (HtR - HtL));
  const F uf = F(0.5) * (un0 + un1);
  const F cl = F(kLight);
  if constexpr (DET) {
    if (uf > F(0)) {
      fJ = fJ + (uf * JL) / cl;
      fN = fN + (uf * HnL) / cl;
      fT = fT + (uf * HtL) / cl;
    } else if (uf < F(0)) {
      fJ = fJ + (uf * JR) / cl;
      fN = fN + (uf * HnR) / cl;
      fT = fT + (uf * HtR) / cl;
    }
  } else {
    const F w = uf * (F(1) / cl);
    const bool up = uf > F(0);
    fJ = fJ + w * (up ? JL : JR);
    fN = fN + w * (up ? HnL : HnR);
    fT = fT + w * (up ? HtL : HtR);
  }
  oJ = fJ;
  oN = fN;
  oT = fT;
}

__device__ __forceinline__ int clampi(int i, int n) { return i < 0 ? 0 : (i >= n ? n - 1 : i); }

// Ghost cell index along one axis.  Geometry 0: outflow on both sides (copy
// of the edge cell).  Geometry 1: the low side (R = 0 axis, Z = 0 midplane)
// is a mirror, where the normal components of H and u change sign (flip =
// true); the high side is outflow.
template <int G>
__device__ __forceinline__ int ghost(int i, int n, bool& flip) {
  if constexpr (G == 1) {
    if (i < 0) {
      flip = true;
      const int m = -1 - i;
      return m >= n ? n - 1 : m;
    }
  }
  flip = false;
  return clampi(i, n);
}

// Ghost cell (x, y) outside an outflow side into vacuum (DeviceView::vac):
// its radiation state is zero.  The low sides of geometry 1 are mirrors.
template <int G>
__device__ __forceinline__ bool vac_ghost(int x, int y, int nx, int ny, int vac) {
  return (G == 0 && x < 0 && (vac & 1)) || (x >= nx && (vac & 2)) ||
         (G == 0 && y < 0 && (vac & 4)) || (y >= ny && (vac & 8));
}

// block-wide fixed-order reductions (warp shuffles, then warps in order)
template <int NT>
__device__ __forceinline__ double block_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x % 32 + 0, tid = threadIdx.y * blockDim.x + threadIdx.x;
  (void)lane;
  __syncthreads();
  if ((tid & 31) == 0) red[tid >> 5] = v;
  __syncthreads();
  double s = 0.0;
  if (tid == 0)
    for (int w = 0; w < NT / 32; ++w) s += red[w];
  return s;
}
// FP32 partials: the warp sums in FP32 (on the FP32 pipe), their total in FP64
// in warp order
template <int NT>
__device__ __forceinline__ double block_sum_f32(float v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  __syncthreads();
  if ((tid & 31) == 0) red[tid >> 5] = double(v);
  __syncthreads();
  double s = 0.0;
  if (tid == 0)
    for (int w = 0; w < NT / 32; ++w) s += red[w];
  return s;
}
template <int NT>
__device__ __forceinline__ double block_max(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  __syncthreads();
  if ((tid & 31) == 0) red[tid >> 5] = v;
  __syncthreads();
  double s = 0.0;
  if (tid == 0)
    for (int w = 0; w < NT / 32; ++w) s = fmax(s, red[w]);
  return s;
}

// The force of a cell from the sums over its bins sum_k dnu_k (H' - H'')
// (Sec. 2.3): written directly when one block holds all bins; a bin group
// of a split tile writes its raw sums to v.fpg, and the frequency step forms
// the force from the groups in group order (combine_force_groups).
__device__ __forceinline__ void store_force(const DeviceView& v, long long cell, int grp, double ax,
                                            double ay) {
  if (v.ngrp > 1) {
    v.fpg[(2LL * grp) * v.nc + cell] = ax;
    v.fpg[(2LL * grp + 1) * v.nc + cell] = ay;
  } else {
    v.fx[cell] = v.fcoef * ax;
    v.fy[cell] = v.fcoef * ay;
  }
}

__device__ __forceinline__ void combine_force_groups(const DeviceView& v, long long cell) {
  if (v.ngrp <= 1 || (v.pt & 8)) return;  // under the acceptance rule its kernel writes the force
  double ax = 0.0, ay = 0.0;
  for (int g = 0; g < v.ngrp; ++g) {
    ax += v.fpg[(2LL * g) * v.nc + cell];
    ay += v.fpg[(2LL * g + 1) * v.nc + cell];
  }
  v.fx[cell] = v.fcoef * ax;
  v.fy[cell] = v.fcoef * ay;
}

// ------------------------------------------------------------ transport kernel
// One tile, bins [k0, k1) (the whole range unless the bins of a small grid's
// tiles are split over several blocks: group grp of v.ngrp, see
// DeviceView::fpg).
template <class P, int G, int PT, int TS = 0>
__device__ __forceinline__ void transport_tile(const DeviceView& v, int x0, int y0, int blk, int k0,
                                               int k1, int grp) {
  // table mode (0 uniform T, 1 temperature field, 2 broad bands) and, in bit 4,
  // active-bin pruning: without it the tile compiles with no pruning code
  constexpr int TM = PT & 3;
  constexpr bool PR = (PT & 4) != 0;
  // bit 8: step 2 is left to the subcycling kernel of the acceptance rule;
  // the tile writes the post-transport state J', H'
  constexpr bool DF = (PT & 8) != 0;
  using S = typename P::S;
  using F = typename P::F;
  using I = typename P::I;
  constexpr int TX = TileShape<TS>::X, TY = TileShape<TS>::Y, SX = TX + 4, SY = TY + 4;
  constexpr int QX = TX + 2, QY = TY + 2;
  constexpr int NT = TX * TY;
  constexpr int NXF = (TX + 1) * TY, NYF = TX * (TY + 1);
  __shared__ F sJ[SY][SX], sHx[SY][SX], sHy[SY][SX], sfx[SY][SX], sfy[SY][SX];
  __shared__ F qA[QY][QX], qR[QY][QX], qUx[QY][QX], qUy[QY][QX];
  __shared__ F xJ[TY][TX + 1], xN[TY][TX + 1], xT[TY][TX + 1];
  __shared__ F yJ[TY + 1][TX], yN[TY + 1][TX], yT[TY + 1][TX];
  __shared__ F sdl[2][G == 1 ? TX + 1 : 1];  // axisymmetric: centroid distances per R face
  __shared__ F qH[TM ? QY : 1][TM ? QX : 1];  // temperature field: <H>_k of the one-cell halo
  const S* __restrict__ Hcs = static_cast<const S*>(v.Hc);
  const S* __restrict__ Gcs = static_cast<const S*>(v.Gc);
  const S* __restrict__ Kbs = static_cast<const S*>(v.Kb);  // bands: kappa per [band][cell]
  __shared__ double red[NT / 32];

  const S* __restrict__ Jin = static_cast<const S*>(v.J);
  const S* __restrict__ Hxin = static_cast<const S*>(v.Hx);
  const S* __restrict__ Hyin = static_cast<const S*>(v.Hy);
  S* __restrict__ Jout = static_cast<S*>(v.Jo);
  S* __restrict__ Hxout = static_cast<S*>(v.Hxo);
  S* __restrict__ Hyout = static_cast<S*>(v.Hyo);

  const int nx = v.nx, ny = v.ny;
  const long long nc = v.nc;
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TX + tx;
  const int gx = x0 + tx, gy = y0 + ty;
  const bool valid = gx < nx && gy < ny;
  const long long cell = valid ? static_cast<long long>(gy) * nx + gx : 0;

  for (int idx = tid; idx < QX * QY; idx += NT) {
    const int lx = idx % QX, ly = idx / QX;
    bool fxg, fyg;
    const int ix = ghost<G>(x0 + lx - 1, nx, fxg), iy = ghost<G>(y0 + ly - 1, ny, fyg);
    const long long c = static_cast<long long>(iy) * nx + ix;
    qA[ly][lx] = F(v.alpha[c]);
    qR[ly][lx] = F(v.rho[c]);
    qUx[ly][lx] = fxg ? -F(v.ux[c]) : F(v.ux[c]);
    qUy[ly][lx] = fyg ? -F(v.uy[c]) : F(v.uy[c]);
  }
  if constexpr (G == 1) {
    for (int f = tid; f <= TX; f += NT) {
      const int gf = x0 + f <= nx ? x0 + f : nx;
      sdl[0][f] = F(v.g_dlL[gf]);
      sdl[1][f] = F(v.g_dlR[gf]);
    }
  }
  I alpha_c = 0, rho_c = 0, pd_c = 0;
  F gxx = 0, gyy = 0, gsh = 0, gphi = 0;
  F ARm = 0, ARp = 0, AZc = 0, Volc = 0, invRc = 0;
  double wcell = 1.0;
  if (valid) {
    alpha_c = I(v.alpha[cell]);
    rho_c = I(v.rho[cell]);
    pd_c = I(v.pd[cell]);
    gxx = F(v.gxx[cell]);
    gyy = F(v.gyy[cell]);
    gsh = F(v.gsh[cell]);
    if constexpr (G == 1) {
      gphi = F(v.gphi[cell]);
      ARm = F(v.g_AR[gx]);
      ARp = F(v.g_AR[gx + 1]);
      AZc = F(v.g_AZ[gx]);
      Volc = F(v.g_Vol[gx]);
      invRc = F(v.g_invR[gx]);
      wcell = v.g_wv[gx];
    }
  }
  const F dx = F(v.dx), half_dx = F(0.5) * F(v.dx), kF_f = F(v.kF), cdt_f = F(v.cdt);
  const I cdt = I(v.cdt), kabs = I(v.kabs), kF = I(v.kF);
  const F cl = F(kLight);
  I ax = 0, ay = 0;
  RSum<I> em, ab, out, wk, en;
  I mxf = 0;
  double bad = 0;
  const double lum_d = valid ? v.lum[cell] : 0.0;

  for (int k = k0; k < k1; ++k) {
    const long long base = static_cast<long long>(k) * nc;
    const double Hk_d = v.t_H[k];
    const F Hk = F(Hk_d);
    // active-bin pruning: a bin left out this substep takes no step 1 (zero
    // face fluxes, J' = J, H' = H); the flag is the same for the whole block
    const bool on = !PR || !v.active || v.active[k];
    if constexpr (TM) {  // <H>_k of the one-cell halo at each cell's temperature
      for (int idx = tid; idx < QX * QY; idx += NT) {
        const int lx = idx % QX, ly = idx / QX;
        bool fxg, fyg;
        const int ix = ghost<G>(x0 + lx - 1, nx, fxg), iy = ghost<G>(y0 + ly - 1, ny, fyg);
        qH[ly][lx] = F(Hcs[base + static_cast<long long>(iy) * nx + ix]);
      }
    }
    // phase A: halo tile of the state and its primitives
    for (int idx = tid; idx < SX * SY; idx += NT) {
      const int lx = idx % SX, ly = idx / SX;
      bool fxg, fyg;
      const int xx = x0 + lx - 2, yy = y0 + ly - 2;
      const int ix = ghost<G>(xx, nx, fxg), iy = ghost<G>(yy, ny, fyg);
      const long long c = base + static_cast<long long>(iy) * nx + ix;
      const bool vz = vac_ghost<G>(xx, yy, nx, ny, v.vac);
      const F J = vz ? F(0) : F(Jin[c]);
      F Hx = vz ? F(0) : F(Hxin[c]);
      F Hy = vz ? F(0) : F(Hyin[c]);
      if (fxg) Hx = -Hx;
      if (fyg) Hy = -Hy;
      sJ[ly][lx] = J;
      sHx[ly][lx] = Hx;
      sHy[ly][lx] = Hy;
      if (J > F(0)) {
        if constexpr (P::DET) {
          sfx[ly][lx] = Hx / J;
          sfy[ly][lx] = Hy / J;
        } else {
          const F rJ = F(1) / J;
          sfx[ly][lx] = Hx * rJ;
          sfy[ly][lx] = Hy * rJ;
        }
      } else {
        sfx[ly][lx] = F(0);
        sfy[ly][lx] = F(0);
      }
    }
    __syncthreads();
    // phase B: every x and y face of the tile once
    for (int f = tid; f < NXF + NYF; f += NT) {
      if (!on) {
        if (f < NXF) {
          const int fi = f % (TX + 1), fj = f / (TX + 1);
          xJ[fj][fi] = xN[fj][fi] = xT[fj][fi] = F(0);
        } else {
          const int g = f - NXF;
          const int fi = g % TX, fj = g / TX;
          yJ[fj][fi] = yN[fj][fi] = yT[fj][fi] = F(0);
        }
        continue;
      }
      if (f < NXF) {
        const int fi = f % (TX + 1), fj = f / (TX + 1);
        const int r = fj + 2;
        const F aF0 = qA[fj + 1][fi] * (TM ? qH[fj + 1][fi] : Hk) + qR[fj + 1][fi] * kF_f;
        const F aF1 = qA[fj + 1][fi + 1] * (TM ? qH[fj + 1][fi + 1] : Hk) + qR[fj + 1][fi + 1] * kF_f;
        F dl0 = half_dx, dl1 = half_dx;
        if constexpr (G == 1) {
          dl0 = sdl[0][fi];
          dl1 = sdl[1][fi];
        }
        face_flux<F, P::DET>(sJ[r][fi], sfx[r][fi], sfy[r][fi], sJ[r][fi + 1], sfx[r][fi + 1],
                     sfy[r][fi + 1], sJ[r][fi + 2], sfx[r][fi + 2], sfy[r][fi + 2], sJ[r][fi + 3],
                     sfx[r][fi + 3], sfy[r][fi + 3], aF0, aF1, qUx[fj + 1][fi],
                     qUx[fj + 1][fi + 1], dl0, dl1, xJ[fj][fi], xN[fj][fi], xT[fj][fi]);
      } else {
        const int g = f - NXF;
        const int fi = g % TX, fj = g / TX;
        const int cc = fi + 2;
        const F aF0 = qA[fj][fi + 1] * (TM ? qH[fj][fi + 1] : Hk) + qR[fj][fi + 1] * kF_f;
        const F aF1 = qA[fj + 1][fi + 1] * (TM ? qH[fj + 1][fi + 1] : Hk) + qR[fj + 1][fi + 1] * kF_f;
        face_flux<F, P::DET>(sJ[fj][cc], sfy[fj][cc], sfx[fj][cc], sJ[fj + 1][cc], sfy[fj + 1][cc],
                     sfx[fj + 1][cc], sJ[fj + 2][cc], sfy[fj + 2][cc], sfx[fj + 2][cc],
                     sJ[fj + 3][cc], sfy[fj + 3][cc], sfx[fj + 3][cc], aF0, aF1, qUy[fj][fi + 1],
                     qUy[fj + 1][fi + 1], half_dx, half_dx, yJ[fj][fi], yN[fj][fi], yT[fj][fi]);
      }
    }
    __syncthreads();
    // phase C: explicit update (A3), implicit source (A4), force (A5)
    if (valid) {
      const F J = sJ[ty + 2][tx + 2], Hx = sHx[ty + 2][tx + 2], Hy = sHy[ty + 2][tx + 2];
      F fxc = sfx[ty + 2][tx + 2], fyc = sfy[ty + 2][tx + 2];
      cap_unit(fxc, fyc);
      F Dxx, Dxy, Dyy, Dpp;
      closure_d<P::DET>(fxc, fyc, Dxx, Dxy, Dyy, Dpp);
      F J1, Hx1, Hy1, W;
      if constexpr (G == 1) {
        // finite volumes per radian; hoop source K_phiphi <1/R> in the R equation
        W = (((Dxx * J) * gxx + (Dyy * J) * gyy) + (Dxy * J) * gsh) + (Dpp * J) * gphi;
        const F divJ = ((ARp * xJ[ty][tx + 1] - ARm * xJ[ty][tx]) + AZc * (yJ[ty + 1][tx] - yJ[ty][tx])) / Volc;
        const F divHx = ((ARp * xN[ty][tx + 1] - ARm * xN[ty][tx]) + AZc * (yT[ty + 1][tx] - yT[ty][tx])) / Volc -
                        (Dpp * J) * invRc;
        const F divHy = ((ARp * xT[ty][tx + 1] - ARm * xT[ty][tx]) + AZc * (yN[ty + 1][tx] - yN[ty][tx])) / Volc;
        J1 = J - cdt_f * (divJ + W / cl);
        Hx1 = Hx - cdt_f * divHx;
        Hy1 = Hy - cdt_f * divHy;
      } else {
        W = ((Dxx * J) * gxx + (Dyy * J) * gyy) + (Dxy * J) * gsh;
        const F divJ = (xJ[ty][tx + 1] - xJ[ty][tx]) + (yJ[ty + 1][tx] - yJ[ty][tx]);
        const F divHx = (xN[ty][tx + 1] - xN[ty][tx]) + (yT[ty + 1][tx] - yT[ty][tx]);
        const F divHy = (xT[ty][tx + 1] - xT[ty][tx]) + (yN[ty + 1][tx] - yN[ty][tx]);
        if constexpr (P::DET) {
          J1 = J - cdt_f * (divJ / dx + W / cl);
          Hx1 = Hx - cdt_f * (divHx / dx);
          Hy1 = Hy - cdt_f * (divHy / dx);
        } else {  // constant reciprocals instead of divisions
          const F cdx = cdt_f * (F(1) / dx);
          J1 = J - (cdx * divJ + cdt_f * (W * (F(1) / cl)));
          Hx1 = Hx - cdx * divHx;
          Hy1 = Hy - cdx * divHy;
        }
      }
      if (!on) {  // pruned bin: no step 1
        J1 = J;
        Hx1 = Hx;
        Hy1 = Hy;
        W = F(0);
      }
      if constexpr (DF) {  // step 2 follows in the subcycling kernel
        const long long o = base + cell;
        Jout[o] = S(J1);
        Hxout[o] = S(Hx1);
        Hyout[o] = S(Hy1);
      } else {
        const I aH = alpha_c * (TM ? I(Hcs[base + cell]) : I(Hk_d));
        const I kap = (TM == 2) ? I(Kbs[base + cell]) : rho_c * kabs + pd_c * aH;
        const I aF = aH + rho_c * kF;
        // j_k = L w_k / (4 pi V dnu_k): formed in FP64 (L ~ 1e39 erg/s and
        // w_k / (4 pi V dnu_k) ~ 1e-58 are both outside the FP32 range); on the
        // axisymmetric grid lum already holds L / (2 pi Vol) and gem_k has V = 1
        const I js = (lum_d != 0.0) ? I(lum_d * (TM ? double(Gcs[base + cell]) : v.t_gem[k])) : I(0);
        I J2, Hx2, Hy2;
        if constexpr (P::DET) {
          J2 = (I(J1) + cdt * js) / (I(1) + cdt * kap);
          Hx2 = I(Hx1) / (I(1) + cdt * aF);
          Hy2 = I(Hy1) / (I(1) + cdt * aF);
        } else {
          J2 = (I(J1) + cdt * js) / (I(1) + cdt * kap);
          const I ra = I(1) / (I(1) + cdt * aF);
          Hx2 = I(Hx1) * ra;
          Hy2 = I(Hy1) * ra;
        }
        const long long o = base + cell;
        Jout[o] = S(J2);
        Hxout[o] = S(Hx2);
        Hyout[o] = S(Hy2);
        const I dnu = I(v.t_dnu[k]);
        ax = ax + dnu * (I(Hx1) - Hx2);
        ay = ay + dnu * (I(Hy1) - Hy2);
        // A7 bookkeeping (energy units applied once per substep on the host side)
        if (lum_d != 0.0) em.add(dnu * (cdt * js));
        ab.add(dnu * (cdt * (kap * J2)));
        if (v.tdiag) {  // the frequency step recomputes these when it follows
          en.add(dnu * J2);
          const I hn = sqrt(Hx2 * Hx2 + Hy2 * Hy2);
          if (J2 > I(0)) mxf = fmax(mxf, hn / J2);
          if (hn > J2 * I(1.000001) && hn > I(0)) bad += 1.0;
        }
      }
      const I dnu = I(v.t_dnu[k]);
      wk.add(dnu * (cdt * (I(W) / I(kLight))));
      const I cdx = cdt / I(v.dx);
      if constexpr (G == 1) {  // outflow through the outer R and Z faces only
        if (gx == nx - 1) out.add(dnu * (cdx * (I(v.g_wR) * I(xJ[ty][tx + 1]))));
        if (gy == ny - 1) out.add(dnu * (cdx * (I(wcell) * I(yJ[ty + 1][tx]))));
      } else {
        if (gx == 0) out.add(dnu * (cdx * -I(xJ[ty][tx])));
        if (gx == nx - 1) out.add(dnu * (cdx * I(xJ[ty][tx + 1])));
        if (gy == 0) out.add(dnu * (cdx * -I(yJ[ty][tx])));
        if (gy == ny - 1) out.add(dnu * (cdx * I(yJ[ty + 1][tx])));
      }
      if (v.spec && (gx == nx - 1 || gy == ny - 1 || (G == 0 && (gx == 0 || gy == 0)))) {
        // emergent spectrum: the escaping energy of each outer face of this cell
        double* sp = v.spec + static_cast<long long>(k) * v.nf;
        const double cdt_d = v.cdt, dxd = v.dx, dnud = v.t_dnu[k];
        if constexpr (G == 1) {
          if (gx == nx - 1)
            sp[gy] += v.spec_unit * ((2.0 * kPi) * (v.g_AR[nx] * (dnud * (cdt_d * double(xJ[ty][tx + 1])))));
          if (gy == ny - 1)
            sp[ny + gx] += v.spec_unit * ((2.0 * kPi) * (v.g_AZ[gx] * (dnud * (cdt_d * double(yJ[ty + 1][tx])))));
        } else {
          const double eu = v.spec_unit * ((dxd * dxd) * dxd);  // erg per unit of the sums
          if (gx == 0) sp[gy] += eu * (dnud * (cdt_d * (-double(xJ[ty][tx]) / dxd)));
          if (gx == nx - 1) sp[ny + gy] += eu * (dnud * (cdt_d * (double(xJ[ty][tx + 1]) / dxd)));
          if (gy == 0) sp[2 * ny + gx] += eu * (dnud * (cdt_d * (-double(yJ[ty][tx]) / dxd)));
          if (gy == ny - 1) sp[2 * ny + nx + gx] += eu * (dnud * (cdt_d * (double(yJ[ty + 1][tx]) / dxd)));
        }
      }
    }
    __syncthreads();
  }
  if (valid && !DF) store_force(v, cell, grp, double(ax), double(ay));
  double* part = v.partT + static_cast<long long>(blk) * kDiagSlots;
  double s;
  s = block_sum<NT>(em.value() * wcell, red);
  if (tid == 0) part[kSlotEmitted] = s;
  s = block_sum<NT>(ab.value() * wcell, red);
  if (tid == 0) part[kSlotAbsorbed] = s;
  s = block_sum<NT>(out.value(), red);
  if (tid == 0) part[kSlotOutflow] = s;
  s = block_sum<NT>(wk.value() * wcell, red);
  if (tid == 0) part[kSlotWork] = s;
  if (v.tdiag && !DF) {
    s = block_sum<NT>(en.value() * wcell, red);
    if (tid == 0) part[kSlotEnergy] = s;
    s = block_max<NT>(double(mxf), red);
    if (tid == 0) part[kSlotMaxF] = s;
    s = block_sum<NT>(bad, red);
    if (tid == 0) part[kSlotBad] = s;
  }
}


template <class P, int G, int PT>
__global__ void __launch_bounds__(kTileX* kTileY) transport_kernel(DeviceView v) {
  transport_tile<P, G, PT>(v, blockIdx.x * kTileX, blockIdx.y * kTileY, blockIdx.y * gridDim.x + blockIdx.x,
                           0, v.nb, 0);
}

// ------------------------------------------------------- FP32 fast-path math
// The FP32 policies use the SFU reciprocal / reciprocal square root (a few ulp)
// and fold divisions by constants into multiplications; their results are
// checked against the FP64 oracle at the mixed-precision bar.
__device__ __forceinline__ float frcp(float b) { return __fdividef(1.0f, b); }
__device__ __forceinline__ float fdiv(float a, float b) { return __fdividef(a, b); }
// J below this is treated as zero when forming f = H/J in FP32: the SFU
// reciprocal flushes subnormal inputs, and such J are ~1e-30 of any field's
// scale (the far wings of the line far from the sources).
constexpr float kTinyJ = 1e-30f;
// share of the domain energy above which a (cell, bin) pair enters the FP32
// realisability diagnostics (the reduction of each substep stores
// kActiveShare E / unit for the next one)
constexpr double kActiveShare = 1e-8;

// ------------------------------------------- FP64 on GB300's narrow FP64 pipe
// GB300 issues FP64 arithmetic, and the FP32 <-> FP64 conversions, on a pipe
// of about 1/70 of the FP32 rate (measured: 0.53 T DFMA/s against 37 T FFMA/s
// per GPU; one conversion costs about one DFMA, an IEEE FP64 division about
// nine).  The LYM1_MIXED policy keeps its implicit steps and its sums in FP64
// and spends that pipe on them only:
//  - conversions run on the integer pipe.  binary32 -> binary64 widening is
//    exact: the exponent is rebiased by 1023 - 127 = 896 and the 23-bit
//    significand moves up by 29 bits.  binary64 -> binary32 narrowing drops 29
//    significand bits and rounds them to nearest, ties to even (a carry into
//    the exponent is the correct rounding, up to infinity).  Both flush
//    subnormal inputs and results to signed zero, like the -ftz FP32
//    arithmetic of these kernels; infinities and NaN map to infinities and
//    quiet NaN.
//  - reciprocals: the hardware approximation rcp.approx.ftz.f64 refined by
//    two Newton-Raphson steps y <- y + y (1 - x y), each of which squares the
//    relative error (within one ulp of 1/x for normal x).
__device__ __forceinline__ double f2d_alu(float x) {
  const unsigned u = __float_as_uint(x);
  const unsigned s = u & 0x80000000u, a = u & 0x7fffffffu;
  unsigned hi = s | ((a >> 3) + 0x38000000u);
  unsigned lo = u << 29;
  if (a < 0x00800000u) {  // zero or subnormal: signed zero
    hi = s;
    lo = 0u;
  } else if (a >= 0x7f800000u) {  // infinity, NaN
    hi = s | (a > 0x7f800000u ? 0x7ff80000u : 0x7ff00000u);
    lo = 0u;
  }
  return __hiloint2double(static_cast<int>(hi), static_cast<int>(lo));
}

__device__ __forceinline__ float d2f_alu(double x) {
  const unsigned hi = static_cast<unsigned>(__double2hiint(x));
  const unsigned lo = static_cast<unsigned>(__double2loint(x));
  const unsigned s = hi & 0x80000000u, a = hi & 0x7fffffffu;
  // biased binary64 exponent e = a >> 20; binary32 normals need 897 <= e <= 1150
  unsigned f = ((a - 0x38000000u) << 3) | (lo >> 29);
  const unsigned r = lo & 0x1fffffffu;  // the 29 dropped bits, half = 2^28
  f += (r > 0x10000000u || (r == 0x10000000u && (f & 1u))) ? 1u : 0u;
  if (a < 0x38100000u) f = 0u;  // below the binary32 normal range
  if (a >= 0x47f00000u)         // beyond the binary32 range, infinity, NaN
    f = (a > 0x7ff00000u || (a == 0x7ff00000u && lo != 0u)) ? 0x7fc00000u : 0x7f800000u;
  return __uint_as_float(s | f);
}

// The per-tile FP32 constants of the FP32 tile are narrowed from their FP64
// inputs on the integer pipe: under register pressure the compiler re-forms
// such values inside the bin loop, and a hardware FP64 -> FP32 conversion there
// costs GB300's narrow FP64 pipe an issue slot per cell-bin (measured: two
// slots per cell-bin, 6 % of LYM1_MIXED's transport).  Same result as the
// conversion for every FP32-normal value.
// x != 0 and x > 0 for a binary64 x, decided on its bits (integer pipe): a
// per-cell predicate that the compiler re-forms inside a bin loop from the
// double itself would otherwise be an FP64 compare there.  Same truth values
// as the comparisons, NaN included.
__device__ __forceinline__ bool nonzero_bits(double x) {
  return (static_cast<unsigned long long>(__double_as_longlong(x)) << 1) != 0ull;
}
__device__ __forceinline__ bool positive_bits(double x) {
  const long long b = __double_as_longlong(x);
  return b > 0 && b <= 0x7ff0000000000000LL;
}

template <class T>
__device__ __forceinline__ T narrow_to(double x) {
  if constexpr (sizeof(T) == 4)
    return d2f_alu(x);
  else
    return x;
}

__device__ __forceinline__ double drcp_nr(double x) {
  double y;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
  double e = fma(-x, y, 1.0);
  y = fma(y, e, y);
  e = fma(-x, y, 1.0);
  return fma(y, e, y);
}

// Seed of 1/x for a binary64 normal x > 0 below 2^1020, without the FP64 pipe:
// x = m 2^q with m in [1, 2); the top 23 bits of m's fraction form a binary32
// m' in [1, 2) (truncated, within 2^-23 of m), whose SFU reciprocal r lies in
// (1/2, 1] (XU pipe); r widened to binary64 and its exponent lowered by q is
// the seed, within ~2^-22 of 1/x.  Integer-pipe bit operations otherwise.
// Also returns q and r's bits, from which the binary32 seed follows.
__device__ __forceinline__ double rcp_seed(double x, int& q, unsigned& rb) {
  const unsigned hi = static_cast<unsigned>(__double2hiint(x));
  const unsigned lo = static_cast<unsigned>(__double2loint(x));
  const unsigned mb = 0x3f800000u | ((hi & 0x000fffffu) << 3) | (lo >> 29);
  rb = __float_as_uint(__fdividef(1.0f, __uint_as_float(mb)));
  q = static_cast<int>(hi >> 20) - 1023;
  const unsigned yhi = ((rb >> 3) + 0x38000000u) - (static_cast<unsigned>(q) << 20);
  return __hiloint2double(static_cast<int>(yhi), static_cast<int>(rb << 29));
}

__device__ __forceinline__ double rcp_seed(double x) {
  int q;
  unsigned rb;
  return rcp_seed(x, q, rb);
}

// binary64 -> binary32 by truncation, for small correction terms: |x| below
// 2^127; results below the binary32 normal range flush to signed zero
__device__ __forceinline__ float d2f_trunc(double x) {
  const unsigned hi = static_cast<unsigned>(__double2hiint(x));
  const unsigned lo = static_cast<unsigned>(__double2loint(x));
  const unsigned a = hi & 0x7fffffffu;
  const unsigned f = a < 0x38100000u ? 0u : (((a - 0x38000000u) << 3) | (lo >> 29));
  return __uint_as_float((hi & 0x80000000u) | f);
}

// Reciprocal of x > 0 from that seed and one FP64 Newton-Raphson step, which
// squares the error (2^-44; tested against IEEE division).
__device__ __forceinline__ double drcp_fs(double x) {
  const double y = rcp_seed(x);
  const double e = fma(-x, y, 1.0);
  return fma(y, e, y);
}

// One Newton-Raphson step: the relative error of the approximation squared
// (2^-40 measured over the normal range against IEEE division, 2^-38 the
// tested bound), for the FP64 steps of LYM1_MIXED whose results are rounded to
// the FP32 state (2^-24).
__device__ __forceinline__ double drcp_nr1(double x) {
  double y;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
  const double e = fma(-x, y, 1.0);
  return fma(y, e, y);
}

// Levermore closure for FP32 from f = (fn, ft) and f2 = |f|^2.  With
// s = sqrt(4 - 3 f2) (so f2 = (4 - s^2)/3) the printed chi reduces exactly to
// chi = (5 - 2s)/3, hence
//   (1 - chi)/2 = (s - 1)/3   and   (3 chi - 1)/(2 f2) = (2 - s)/f2 = 3/(2 + s),
// both free of cancellation at small f (where the printed 3 chi - 1 ~ 1.5 f2
// loses every digit in FP32).  Dpp = (1 - chi)/2.
//
// The face flux and the closure are evaluated by several inlined copies (the
// regular faces of each direction and the extra faces of a tile's edge), and a
// face shared by two tiles must have one value whichever copy computes it.  So
// every product and sum here is written with explicit rounding (fmaf for the
// fused steps, __fmul_rn / __fadd_rn / __fsub_rn for the rest): the compiler
// may not contract them, and each copy does the same operations.
__device__ __forceinline__ void closure_f32q(float fn, float ft, float f2, float& Dnn, float& Dnt,
                                             float& Dtt, float& Dpp) {
  const float y = fmaf(-3.0f, f2, 4.0f);
  const float s = __fmul_rn(y, rsqrtf(y));
  const float dA = __fmul_rn(__fsub_rn(s, 1.0f), 1.0f / 3.0f);
  const float g = __fmul_rn(3.0f, frcp(__fadd_rn(2.0f, s)));
  Dnn = fmaf(g, __fmul_rn(fn, fn), dA);
  Dnt = __fmul_rn(g, __fmul_rn(fn, ft));
  Dtt = fmaf(g, __fmul_rn(ft, ft), dA);
  Dpp = dA;
}

__device__ __forceinline__ void closure_f32(float fn, float ft, float& Dnn, float& Dnt, float& Dtt,
                                            float& Dpp) {
  closure_f32q(fn, ft, fmaf(fn, fn, __fmul_rn(ft, ft)), Dnn, Dnt, Dtt, Dpp);
}

__device__ __forceinline__ void closure_f32(float fn, float ft, float& Dnn, float& Dnt, float& Dtt) {
  float Dpp;
  closure_f32(fn, ft, Dnn, Dnt, Dtt, Dpp);
}

// |f| > 1: scale to the unit circle (without a branch: the factor is
// rsqrt(max(|f|^2, 1)), 1 for |f| <= 1); returns |f|^2 after the scaling
__device__ __forceinline__ float cap_unit_f32(float& fn, float& ft) {
  const float f2 = fmaf(fn, fn, __fmul_rn(ft, ft));
  const float r = rsqrtf(fmaxf(f2, 1.0f));
  fn = __fmul_rn(fn, r);
  ft = __fmul_rn(ft, r);
  return fminf(f2, 1.0f);
}

// MinMod as the median of (a, b, 0): the smaller magnitude when a and b share
// a sign, zero otherwise (pure selection, so tiny slopes are kept).
__device__ __forceinline__ float minmod_f32(float a, float b) {
  return fmaxf(fminf(a, b), fminf(fmaxf(a, b), 0.0f));
}

// Face flux (same scheme as face_flux) from packed primitives q = (J, f_n, f_t)
// of cells -1, 0, +1, +2, the face optical depth tau and the face velocity
// wf = (u_0 + u_1) / (2c); the interpolation factor and the diffusion
// coefficient share one reciprocal:
//   eps = (0.2 + tau) / d,  (1 - eps) / (3 tau) = tau / (3 d),  d = 0.2 + tau + tau^2.
__device__ __forceinline__ void face_flux_f32(float Jm, float nm, float tm, float J0, float n0,
                                              float t0, float J1, float n1, float t1, float J2,
                                              float n2, float t2, float tau, float wf, float& oJ,
                                              float& oN, float& oT) {
  const float d0 = __fsub_rn(J0, Jm), d1 = __fsub_rn(J1, J0), d2 = __fsub_rn(J2, J1);
  const float JL = fmaf(0.5f, minmod_f32(d0, d1), J0), JR = fmaf(-0.5f, minmod_f32(d1, d2), J1);
  const float e1 = __fsub_rn(n1, n0), g1 = __fsub_rn(t1, t0);
  float nL = fmaf(0.5f, minmod_f32(__fsub_rn(n0, nm), e1), n0);
  float tL = fmaf(0.5f, minmod_f32(__fsub_rn(t0, tm), g1), t0);
  float nR = fmaf(-0.5f, minmod_f32(e1, __fsub_rn(n2, n1)), n1);
  float tR = fmaf(-0.5f, minmod_f32(g1, __fsub_rn(t2, t1)), t1);
  const float f2L = cap_unit_f32(nL, tL);
  const float f2R = cap_unit_f32(nR, tR);
  const float HnL = __fmul_rn(JL, nL), HtL = __fmul_rn(JL, tL);
  const float HnR = __fmul_rn(JR, nR), HtR = __fmul_rn(JR, tR);
  float DnnL, DntL, DttL, DppL, DnnR, DntR, DttR, DppR;
  closure_f32q(nL, tL, f2L, DnnL, DntL, DttL, DppL);
  closure_f32q(nR, tR, f2R, DnnR, DntR, DttR, DppR);
  const float a = __fadd_rn(0.2f, tau);
  const float rden = frcp(fmaf(tau, tau, a));
  const float eps = __fmul_rn(a, rden);
  const float dcoef = __fmul_rn(__fmul_rn(tau, rden), 1.0f / 3.0f);
  const bool up = wf > 0.0f;  // upwind donor: reconstructed state on the upwind side
  const float Jd = up ? JL : JR, Hnd = up ? HnL : HnR, Htd = up ? HtL : HtR;
  const float he = __fmul_rn(0.5f, eps);
  oJ = fmaf(wf, Jd, fmaf(-dcoef, d1, __fmul_rn(he, __fsub_rn(__fadd_rn(HnL, HnR), __fsub_rn(JR, JL)))));
  oN = fmaf(wf, Hnd,
            __fmul_rn(0.5f, fmaf(-eps, __fsub_rn(HnR, HnL), fmaf(DnnL, JL, __fmul_rn(DnnR, JR)))));
  oT = fmaf(wf, Htd,
            __fmul_rn(0.5f, fmaf(-eps, __fsub_rn(HtR, HtL), fmaf(DntL, JL, __fmul_rn(DntR, JR)))));
}

// ------------------------------------------------ FP32 transport kernel
// Same rows A1-A5 as transport_kernel for FP32 state and fluxes.  The halo
// tile is double-buffered and packed as float4 (J, f_x, f_y, alpha_F,k) per
// cell; each thread owns at most two halo entries, keeps their opacities in
// registers and prefetches their state of bin k+1 while bin k is computed, so
// one bin needs two block barriers.  Faces are mapped to threads without
// division: every thread computes the left x-face and the bottom y-face of
// its cell, warp 0 the top row of y-faces and part of warp 1 the right column
// of x-faces; the face velocities (and on the axisymmetric grid the centroid
// distances) of a thread's faces do not depend on the bin and stay in
// registers.  The implicit source step runs in type I (FP64 for LYM1_MIXED,
// FP32 for LYM1_MIXED_FAST).
// The FP32 tile's static shared buffers, declared once per kernel (the tile
// body is instantiated twice under LYM1_MIXED, see transport_tile_f32_any)
template <int TS>
struct TileSmemF32 {
  static constexpr int TX = TileShape<TS>::X, TY = TileShape<TS>::Y, SX = TX + 4, SY = TY + 4;
  float4 sq[2][SY][SX];  // (J, f_x, f_y, alpha_F of the bin)
  float sHx[2][SY][SX], sHy[2][SY][SX];
  // face fluxes (J, normal K, tangential K, -): x faces (J, K_xx, K_xy), y faces
  // (J, K_yy, K_yx)
  float4 xF[TY][TX + 1];
  float4 yF[TY + 1][TX];
  double red[2 * (TX * TY / 32)];  // the last pair of reductions uses both halves
};

// SRC = false: no cell of the tile holds a source (LYM1_MIXED's step 2 then
// compiles without the emission term; decided per tile by the kernel wrapper)
template <class P, int G, int PT, int TS = 0, bool SRC = true>
__device__ __forceinline__ void transport_tile_f32(TileSmemF32<TS>& sm, const DeviceView& v, int x0,
                                                   int y0, int blk, int k0, int k1, int grp) {
  // table mode (0 uniform T, 1 temperature field, 2 broad bands) and, in bit 4,
  // active-bin pruning: without it the tile compiles with no pruning code
  constexpr int TM = PT & 3;
  constexpr bool PR = (PT & 4) != 0;
  // bit 8: step 2 is left to the subcycling kernel of the acceptance rule
  constexpr bool DF = (PT & 8) != 0;
  using I = typename P::I;
  constexpr int TX = TileShape<TS>::X, TY = TileShape<TS>::Y, SX = TX + 4, SY = TY + 4;
  constexpr int NT = TX * TY;
  static_assert(SX * SY <= 2 * NT, "two halo entries per thread at most");
  static_assert(TX + TY <= 64, "the extra faces are the first two warps' work at most");
  auto& sq = sm.sq;
  auto& sHx = sm.sHx;
  auto& sHy = sm.sHy;
  auto& xF = sm.xF;
  auto& yF = sm.yF;
  auto& red = sm.red;
  extern __shared__ float4 tab4[];  // per bin (<H>_k, dnu_k, gem_k / gem_max, J_act,k) as FP32

  const float* __restrict__ Jin = static_cast<const float*>(v.J);
  const float* __restrict__ Hxin = static_cast<const float*>(v.Hx);
  const float* __restrict__ Hyin = static_cast<const float*>(v.Hy);
  float* __restrict__ Jout = static_cast<float*>(v.Jo);
  float* __restrict__ Hxout = static_cast<float*>(v.Hxo);
  float* __restrict__ Hyout = static_cast<float*>(v.Hyo);
  // temperature field: <H>_k and gem_k / gmax per [k][cell]
  const float* __restrict__ Hcf = static_cast<const float*>(v.Hc);
  const float* __restrict__ Gcf = static_cast<const float*>(v.Gc);
  const float* __restrict__ Kbf = static_cast<const float*>(v.Kb);  // bands: kappa per [band][cell]

  const int nx = v.nx, ny = v.ny, nb = v.nb;
  const long long nc = v.nc;
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TX + tx;
  const int gx = x0 + tx, gy = y0 + ty;
  const bool valid = gx < nx && gy < ny;
  const long long cell = valid ? static_cast<long long>(gy) * nx + gx : 0;
  const float inv_c = 1.0f / float(kLight);
  const bool tdiag = v.tdiag != 0;

  // realisability is checked on (cell, bin) pairs holding at least kActiveShare
  // of the domain energy of the previous substep (FP32 rounding makes |H|/J
  // meaningless far below a bin plane's scale)
  // J dnu_k above thr = kActiveShare E_prev / unit (set by the previous substep's reduction)
  const float thr = float(v.acc[14]);
  for (int i = tid; i < nb; i += NT)
    tab4[i] = make_float4(v.f_H[i], v.f_dnu[i], v.f_G[i], fmaxf(thr, 1e-30f) / v.f_dnu[i]);
  // halo entries owned by this thread (plane offsets; sign of H_x, H_y;
  // opacity alpha and rho_d kappa_F of the ghost-mapped cell)
  const int e0 = tid, e1 = tid + NT;
  const bool has1 = e1 < SX * SY;
  const int ex0 = e0 % SX, ey0 = e0 / SX, ex1 = e1 % SX, ey1 = e1 / SX;
  bool fx0, fy0, fx1 = false, fy1 = false;
  // in-plane offsets fit in 32 bits (cells per plane <= 2^31, checked at creation)
  const int off0 = ghost<G>(y0 + ey0 - 2, ny, fy0) * nx + ghost<G>(x0 + ex0 - 2, nx, fx0);
  const int off1 = has1 ? ghost<G>(y0 + ey1 - 2, ny, fy1) * nx + ghost<G>(x0 + ex1 - 2, nx, fx1) : 0;
  const int cell32 = static_cast<int>(cell);
  const float sx0 = fx0 ? -1.0f : 1.0f, sy0 = fy0 ? -1.0f : 1.0f;
  const float sx1 = fx1 ? -1.0f : 1.0f, sy1 = fy1 ? -1.0f : 1.0f;
  // ghosts beyond an outflow side into vacuum hold no radiation
  const bool vz0 = vac_ghost<G>(x0 + ex0 - 2, y0 + ey0 - 2, nx, ny, v.vac);
  const bool vz1 = has1 && vac_ghost<G>(x0 + ex1 - 2, y0 + ey1 - 2, nx, ny, v.vac);
  const float kF_f = float(v.kF);
  const float al0 = float(v.alpha[off0]), rk0 = float(v.rho[off0]) * kF_f;
  const float al1 = has1 ? float(v.alpha[off1]) : 0.0f;
  const float rk1 = has1 ? float(v.rho[off1]) * kF_f : 0.0f;
  // this thread's faces: x-face (tx, ty), y-face (tx, ty) and the extra
  // ones; velocity u/c of each adjacent cell with the mirror flips
  auto wcell = [&](int x, int y, bool xdir) {
    bool fxg, fyg;
    const int ix = ghost<G>(x, nx, fxg), iy = ghost<G>(y, ny, fyg);
    const long long c = static_cast<long long>(iy) * nx + ix;
    const float w = __fmul_rn(float(xdir ? v.ux[c] : v.uy[c]), inv_c);
    return (xdir ? fxg : fyg) ? -w : w;
  };
  const float wfx = 0.5f * (wcell(gx - 1, gy, true) + wcell(gx, gy, true));
  const float wfy = 0.5f * (wcell(gx, gy - 1, false) + wcell(gx, gy, false));
  // the TX + TY extra faces are one evaluation by the first threads (warp 0
  // for 16 x 16): threads 0..TX-1 take the top row of y faces (fi = tid,
  // fj = TY), threads TX..TX+TY-1 the right column of x faces (fi = TX,
  // fj = tid - TX)
  const bool xtra = tid < TX + TY;
  const bool xisx = tid >= TX;
  const int xfi = xisx ? TX : tid, xfj = xisx ? tid - TX : TY;
  float wf2 = 0.0f;
  if (xtra)
    wf2 = xisx ? 0.5f * (wcell(x0 + TX - 1, y0 + xfj, true) + wcell(x0 + TX, y0 + xfj, true))
               : 0.5f * (wcell(x0 + xfi, y0 + TY - 1, false) + wcell(x0 + xfi, y0 + TY, false));
  // face optical depth = aF_0 dl_0 + aF_1 dl_1 (centroid distances, geometry
  // 1) or (aF_0 + aF_1) dx/2 (geometry 0)
  const float half_dx = 0.5f * d2f_alu(v.dx);
  float dlA0 = half_dx, dlA1 = half_dx, dlB0 = half_dx, dlB1 = half_dx;
  if constexpr (G == 1) {
    const int fa = gx <= nx ? gx : nx;
    dlA0 = v.gf_dlL[fa];
    dlA1 = v.gf_dlR[fa];
    if (xtra && xisx) {
      const int fb = x0 + TX <= nx ? x0 + TX : nx;
      dlB0 = v.gf_dlL[fb];
      dlB1 = v.gf_dlR[fb];
    }
  }

  I alpha_c = 0, rho_c = 0, pd_c = 0;
  float gxx = 0, gyy = 0, gsh = 0, gphi = 0;
  float r0c = 0, r1c = 0, hoopc = 0, wvf = 1.0f;
  double lum_d = 0.0;
  if (valid) {
    alpha_c = narrow_to<I>(v.alpha[cell]);
    rho_c = narrow_to<I>(v.rho[cell]);
    pd_c = narrow_to<I>(v.pd[cell]);
    lum_d = v.lum[cell];
    // velocity gradients times c_tilde dt / c: W below is then the step-1
    // change of J itself, (c_tilde dt / c) D : grad u J, which stays in the
    // FP32 range where J does (W / c alone is ~1e-20 J)
    gxx = d2f_alu(v.gxx[cell] * v.cdt_c);
    gyy = d2f_alu(v.gyy[cell] * v.cdt_c);
    gsh = d2f_alu(v.gsh[cell] * v.cdt_c);
    if constexpr (G == 1) {
      gphi = d2f_alu(v.gphi[cell] * v.cdt_c);
      r0c = v.gf_r0[gx];
      r1c = v.gf_r1[gx];
      hoopc = v.gf_hoop[gx];
      wvf = v.gf_wv[gx];
    }
  }
  const float cdt_dx = d2f_alu(v.cdt_dx);
  const I cdt = narrow_to<I>(v.cdt), kabs = narrow_to<I>(v.kabs), kF = narrow_to<I>(v.kF),
          cdx = narrow_to<I>(v.cdt_dx);
  const I wR = narrow_to<I>(v.g_wR), wcol = I(wvf);
  const float wRf = d2f_alu(v.g_wR);
  // LYM1_MIXED (FP64 implicit step): the per-cell factors with c_tilde dt
  // folded in, c dt kappa_k = cA + cB <H>_k and c dt alpha_F,k = cD + cC <H>_k
  // (bands: c dt kappa_k from their kappa table, alpha = 1, rho_d = 0)
  constexpr bool MIX = sizeof(I) == 8 && !DF;
  double cA = 0.0, cB = 0.0, cC = 0.0, cD = 0.0, cjs = 0.0;
  // 1 + cA and 1 + cD (the denominators of step 2 in one FMA each) and FP32
  // copies of cC, cD for the force weight
  double cA1 = 1.0, cD1 = 1.0;
  float cCf = 0.0f, cDf = 0.0f;
  // emission of a uniform-temperature cell over this block's bins k0..k1-1:
  // c dt L_cell sum_k dnu_k gem_k
  double sgk = 0.0;
  if constexpr (MIX) {
    const double cd = v.cdt;
    cA = cd * (double(rho_c) * v.kabs);
    cB = cd * (double(pd_c) * double(alpha_c));
    cC = cd * double(alpha_c);
    cD = cd * (double(rho_c) * v.kF);
    cjs = cd * lum_d;
    cA1 = 1.0 + cA;
    cD1 = 1.0 + cD;
    cCf = d2f_alu(cC);
    cDf = d2f_alu(cD);
    if constexpr (TM == 0)
      if (lum_d != 0.0)
        for (int k = k0; k < k1; ++k) sgk = fma(v.t_dnu[k], v.t_gem[k], sgk);
  }
  I ax = 0, ay = 0;
  // per-cell bookkeeping sums over the bins: FP64 (compensation-free, exact
  // enough at 194 terms) for LYM1_MIXED, plain FP32 for LYM1_MIXED_FAST; the
  // sums over cells are FP64 in both
  I em = 0, ab = 0, out = 0, wk = 0, en = 0;
  // LYM1_MIXED, Lya table modes: the absorbed energy sum_k dnu_k c dt kappa_k J''_k
  // as cA sum_k dnu_k J''_k + cB sum_k dnu_k <H>_k J''_k (c dt kappa_k = cA + cB <H>_k)
  double sJ = 0.0, sHJ = 0.0;
  float mxf2 = 0.0f;
  int bad = 0;
  // source term c_tilde dt j_k = (c_tilde dt L_cell gem_max) (gem_k / gem_max):
  // both factors lie in the FP32 range, unlike L_cell (~1e39 erg/s) and gem_k
  // (~1e-75) alone, or j_k itself in the far wings (~1e-38)
  const bool src = nonzero_bits(lum_d);
  const double gmax_c = TM ? (valid ? v.gmaxc[cell] : 1.0) : v.gem_max;
  const float cjsc = d2f_alu(v.cdt * (lum_d * gmax_c));
  const bool bnd = valid && (G == 1 ? (gx == nx - 1 || gy == ny - 1)
                                     : (gx == 0 || gx == nx - 1 || gy == 0 || gy == ny - 1));

  long long base = static_cast<long long>(k0) * nc;  // k * nc
  float pJ0 = Jin[base + off0], pX0 = Hxin[base + off0], pY0 = Hyin[base + off0];
  float pJ1 = 0.f, pX1 = 0.f, pY1 = 0.f;
  float pH0 = 0.f, pH1 = 0.f;  // <H>_k of the halo entries (temperature field)
  if (has1) {
    pJ1 = Jin[base + off1];
    pX1 = Hxin[base + off1];
    pY1 = Hyin[base + off1];
  }
  if constexpr (TM) {
    pH0 = Hcf[base + off0];
    if (has1) pH1 = Hcf[base + off1];
  }
  // LYM1_MIXED: the FP64 implicit step of bin k - 1 (Sec. 2.1 step 2) is
  // issued in the face phase of bin k, so that GB300's narrow FP64 pipe works
  // while the FP32 face fluxes are formed; pending values of the last bin are
  // finished after the loop.
  float dJ1 = 0.0f, dHx1 = 0.0f, dHy1 = 0.0f, dW = 0.0f;
  RSum<float> fxs, fys;  // LYM1_MIXED: sum_k dnu_k (H' - H'') per component
  auto step2_mix = [&](int kk, long long kbase) {
    if constexpr (MIX) {
      // d1 = 1 + c dt kappa_k and d2 = 1 + c dt alpha_F,k, each in one FMA
      const double Hd = TM ? f2d_alu(Hcf[kbase + cell]) : v.t_H[kk];
      const double dnud = v.t_dnu[kk];
      double ck = 0.0, d1;
      if constexpr (TM == 2) {
        ck = v.cdt * f2d_alu(Kbf[kbase + cell]);
        d1 = 1.0 + ck;
      } else {
        d1 = fma(cB, Hd, cA1);
      }
      const double d2 = fma(cC, Hd, cD1);
      double num = f2d_alu(dJ1);
      double gk = 0.0;
      if constexpr (SRC)
        if (src) {
          gk = TM ? gmax_c * f2d_alu(Gcf[kbase + cell]) : v.t_gem[kk];
          num = fma(cjs, gk, num);
        }
      // J'' = num / d1 in FP64: the FP32 seed y of 1/d1 (d1 >= 1) and one
      // Newton-Raphson step folded into the product, num y (1 + e) with the
      // FP64 residual e = 1 - d1 y (relative error e^2 ~ 2^-44)
      const double y1 = rcp_seed(d1);
      const double e1 = fma(-d1, y1, 1.0);
      const double t1 = num * y1;
      const double J2d = fma(t1, e1, t1);
      const float J2 = d2f_alu(J2d);
      // H'' = H' / d2 with the factor 1/d2 rounded to the FP32 of the state:
      // the FP32 seed corrected by its FP64 residual (the correction itself,
      // ~2^-22 of the seed, needs no more than FP32)
      int q2;
      unsigned rb2;
      const double y2d = rcp_seed(d2, q2, rb2);
      const double e2 = fma(-d2, y2d, 1.0);
      // the same seed in binary32 (d2 >= 1, so q2 >= 0; 1/d2 below the binary32
      // normal range flushes to zero, as the state's FP32 arithmetic would)
      const float y2 = q2 < 126 ? __uint_as_float(rb2 - (static_cast<unsigned>(q2) << 23)) : 0.0f;
      const float raf = fmaf(y2, d2f_trunc(e2), y2);
      const float Hx2 = dHx1 * raf, Hy2 = dHy1 * raf;
      if (valid) {
        (Jout + kbase)[cell32] = J2;
        (Hxout + kbase)[cell32] = Hx2;
        (Hyout + kbase)[cell32] = Hy2;
      }
      // the force term dnu_k (H' - H'') = dnu_k (c dt alpha_F / d2) H' has no
      // cancellation; its weight dnu_k c dt alpha_F / d2 is FP32 (the force is
      // summed in compensated FP32, off the FP64 pipe)
      const float caFf = fmaf(cCf, TM ? Hcf[kbase + cell] : tab4[kk].x, cDf);
      const float wq = tab4[kk].y * (caFf * raf);
      // A7 bookkeeping in FP64 (c_tilde dt is in the factors; 1/c and the
      // energy units once per substep)
      const double twk = f2d_alu(tab4[kk].y * dW);
      fxs.add(wq * dHx1);
      fys.add(wq * dHy1);
      if constexpr (TM == 2) {
        ab = fma(dnud * ck, J2d, ab);
      } else {
        sJ = fma(dnud, J2d, sJ);
        sHJ = fma(TM ? dnud * Hd : v.t_dH[kk], J2d, sHJ);
      }
      wk = wk + twk;
      if constexpr (TM != 0) em = fma(dnud, gk, em);
      if (tdiag) {  // the frequency step recomputes these when it follows
        if constexpr (TM == 2) en = fma(dnud, J2d, en);
        const float h2 = Hx2 * Hx2 + Hy2 * Hy2, jj = J2 * J2;
        if ((G == 1 ? J2 * wvf : J2) > tab4[kk].w) {
          mxf2 = fmaxf(mxf2, fdiv(h2, jj));
          bad += (h2 > jj * 1.000002f) ? 1 : 0;
        }
      }
    }
  };

  for (int k = k0; k < k1; ++k) {
    const int b = k & 1;
    const float4 tb = tab4[k];  // (<H>_k, dnu_k, gem_k / gem_max, J_act,k)
    const float Hk = tb.x;
    // active-bin pruning: a bin left out this substep takes no step 1 (zero
    // face fluxes, J' = J, H' = H); the flag is the same for the whole block
    const bool on = !PR || !v.active || v.active[k];
    {  // halo entries of bin k: registers -> shared, with primitives and alpha_F
      float J0 = pJ0, X0 = pX0, Y0 = pY0, J1 = pJ1, X1 = pX1, Y1 = pY1;
      if (vz0) J0 = X0 = Y0 = 0.0f;
      if (vz1) J1 = X1 = Y1 = 0.0f;
      if constexpr (G == 1) {
        X0 *= sx0;
        Y0 *= sy0;
        X1 *= sx1;
        Y1 *= sy1;
      }
      const float r0 = J0 > kTinyJ ? frcp(J0) : 0.0f;
      sq[b][ey0][ex0] = make_float4(J0, X0 * r0, Y0 * r0, al0 * (TM ? pH0 : Hk) + rk0);
      sHx[b][ey0][ex0] = X0;
      sHy[b][ey0][ex0] = Y0;
      if (has1) {
        const float r1 = J1 > kTinyJ ? frcp(J1) : 0.0f;
        sq[b][ey1][ex1] = make_float4(J1, X1 * r1, Y1 * r1, al1 * (TM ? pH1 : Hk) + rk1);
        sHx[b][ey1][ex1] = X1;
        sHy[b][ey1][ex1] = Y1;
      }
    }
    const long long nbase = base + nc;
    if (k + 1 < k1) {  // prefetch bin k+1
      const float* Jn = Jin + nbase;
      const float* Xn = Hxin + nbase;
      const float* Yn = Hyin + nbase;
      pJ0 = Jn[off0];
      pX0 = Xn[off0];
      pY0 = Yn[off0];
      if (has1) {
        pJ1 = Jn[off1];
        pX1 = Xn[off1];
        pY1 = Yn[off1];
      }
      if constexpr (TM) {
        pH0 = Hcf[nbase + off0];
        if (has1) pH1 = Hcf[nbase + off1];
      }
    }
    __syncthreads();
    if constexpr (MIX)
      if (k > k0) step2_mix(k - 1, base - nc);  // a block-uniform branch
    auto xface = [&](int fi, int fj, float wf, float dl0, float dl1) {
      // between tile cells (fi-1, fj) and (fi, fj)
      const int r = fj + 2;
      const float4 qm = sq[b][r][fi], q0 = sq[b][r][fi + 1], q1 = sq[b][r][fi + 2],
                   q2 = sq[b][r][fi + 3];
      const float tau = (G == 1) ? fmaf(q0.w, dl0, __fmul_rn(q1.w, dl1))
                                 : __fmul_rn(__fadd_rn(q0.w, q1.w), dl0);
      float oJ, oN, oT;
      face_flux_f32(qm.x, qm.y, qm.z, q0.x, q0.y, q0.z, q1.x, q1.y, q1.z, q2.x, q2.y, q2.z, tau,
                    wf, oJ, oN, oT);
      xF[fj][fi] = make_float4(oJ, oN, oT, 0.0f);
    };
    auto yface = [&](int fi, int fj, float wf) {  // between tile cells (fi, fj-1) and (fi, fj)
      const int cc = fi + 2;
      const float4 qm = sq[b][fj][cc], q0 = sq[b][fj + 1][cc], q1 = sq[b][fj + 2][cc],
                   q2 = sq[b][fj + 3][cc];
      float oJ, oN, oT;
      face_flux_f32(qm.x, qm.z, qm.y, q0.x, q0.z, q0.y, q1.x, q1.z, q1.y, q2.x, q2.z, q2.y,
                    __fmul_rn(__fadd_rn(q0.w, q1.w), half_dx), wf, oJ, oN, oT);
      yF[fj][fi] = make_float4(oJ, oN, oT, 0.0f);
    };
    if (on) {
      xface(tx, ty, wfx, dlA0, dlA1);
      yface(tx, ty, wfy);
      if (xtra) {  // one evaluation for both kinds of extra face
        const float4* q = xisx ? &sq[b][xfj + 2][xfi] : &sq[b][xfj][xfi + 2];
        const int st = xisx ? 1 : SX;
        const float4 qm = q[0], q0 = q[st], q1 = q[2 * st], q2 = q[3 * st];
        // the same expression as the regular faces, so that a face shared by
        // two tiles has one value whichever tile evaluates it
        const float tau = (G == 1 && xisx) ? fmaf(q0.w, dlB0, __fmul_rn(q1.w, dlB1))
                                           : __fmul_rn(__fadd_rn(q0.w, q1.w), half_dx);
        float oJ, oN, oT;
        face_flux_f32(qm.x, xisx ? qm.y : qm.z, xisx ? qm.z : qm.y, q0.x, xisx ? q0.y : q0.z,
                      xisx ? q0.z : q0.y, q1.x, xisx ? q1.y : q1.z, xisx ? q1.z : q1.y, q2.x,
                      xisx ? q2.y : q2.z, xisx ? q2.z : q2.y, tau, wf2, oJ, oN, oT);
        float4* dst = xisx ? &xF[xfj][TX] : &yF[TY][xfi];
        *dst = make_float4(oJ, oN, oT, 0.0f);
      }
    } else {  // pruned bin: zero fluxes on this thread's faces
      const float4 z4 = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
      xF[ty][tx] = z4;
      yF[ty][tx] = z4;
      if (xtra) *(xisx ? &xF[xfj][TX] : &yF[TY][xfi]) = z4;
    }
    __syncthreads();
    if (valid) {
      const float4 qs = sq[b][ty + 2][tx + 2];
      const float J = qs.x, Hx = sHx[b][ty + 2][tx + 2], Hy = sHy[b][ty + 2][tx + 2];
      float fxc = qs.y, fyc = qs.z;
      const float f2c = cap_unit_f32(fxc, fyc);
      float Dxx, Dxy, Dyy, Dpp;
      closure_f32q(fxc, fyc, f2c, Dxx, Dxy, Dyy, Dpp);
      const float4 xl = xF[ty][tx], xr = xF[ty][tx + 1], yb = yF[ty][tx], yt = yF[ty + 1][tx];
      float W, divJ, divHx, divHy;
      if constexpr (G == 1) {
        // per-radian finite volumes in units of dx (r0, r1 = R-face areas x dx /
        // Vol, hoop = dx^3 / Vol); hoop source K_phiphi <1/R> in the R equation
        W = J * (((Dxx * gxx + Dyy * gyy) + Dxy * gsh) + Dpp * gphi);
        divJ = (r1c * xr.x - r0c * xl.x) + (yt.x - yb.x);
        divHx = ((r1c * xr.y - r0c * xl.y) + (yt.z - yb.z)) - hoopc * (Dpp * J);
        divHy = (r1c * xr.z - r0c * xl.z) + (yt.y - yb.y);
      } else {
        W = J * ((Dxx * gxx + Dyy * gyy) + Dxy * gsh);
        divJ = (xr.x - xl.x) + (yt.x - yb.x);
        divHx = (xr.y - xl.y) + (yt.z - yb.z);
        divHy = (xr.z - xl.z) + (yt.y - yb.y);
      }
      if (!on) W = 0.0f;  // pruned bin: no step 1
      // c_tilde dt / dx folded into one factor: divJ / dx alone leaves the
      // FP32 range for J below ~1e-22
      const float J1 = on ? J - fmaf(cdt_dx, divJ, W) : J;
      const float Hx1 = on ? Hx - cdt_dx * divHx : Hx;
      const float Hy1 = on ? Hy - cdt_dx * divHy : Hy;
      if constexpr (DF) {  // step 2 follows in the subcycling kernel
        (Jout + base)[cell32] = J1;
        (Hxout + base)[cell32] = Hx1;
        (Hyout + base)[cell32] = Hy1;
        wk += I(tb.y * W);
      } else if constexpr (MIX) {
        // the FP64 step of this bin runs in the face phase of the next bin
        dJ1 = J1;
        dHx1 = Hx1;
        dHy1 = Hy1;
        dW = W;
      } else {
        const float aH = alpha_c * (TM ? Hcf[base + cell] : Hk);
        const float dnu = tb.y;
        const float kap = (TM == 2) ? Kbf[base + cell] : rho_c * kabs + pd_c * aH;
        const float aF = aH + rho_c * kF;
        const float cjk = src ? cjsc * (TM ? Gcf[base + cell] : tb.z) : 0.0f;
        const float ckap = cdt * kap;  // c_tilde dt kappa_k
        const float J2 = (J1 + cjk) * frcp(1.0f + ckap);
        const float caF = cdt * aF;
        const float ra = frcp(1.0f + caF);
        const float Hx2 = Hx1 * ra, Hy2 = Hy1 * ra;
        (Jout + base)[cell32] = J2;
        (Hxout + base)[cell32] = Hx2;
        (Hyout + base)[cell32] = Hy2;
        // H' - H'' = H' c dt alpha_F / (1 + c dt alpha_F): the product form,
        // free of the cancellation of the difference in thin bins
        const float wq = dnu * (caF * ra);
        ax += wq * Hx1;
        ay += wq * Hy1;
        // A7 bookkeeping (energy units applied once per substep; the factors
        // c_tilde dt and 1/c once per cell after the bin loop)
        if (src) em += dnu * cjk;
        ab += dnu * (ckap * J2);
        wk += dnu * W;
        if (tdiag) {  // the frequency step recomputes these when it follows
          en += dnu * J2;
          const float h2 = Hx2 * Hx2 + Hy2 * Hy2, jj = J2 * J2;
          if ((G == 1 ? J2 * wvf : J2) > tb.w) {
            mxf2 = fmaxf(mxf2, fdiv(h2, jj));
            bad += (h2 > jj * 1.000002f) ? 1 : 0;
          }
        }
      }
      if (bnd) {
        // the escaping flux of the cell's outer faces, formed in FP32 (the face
        // fluxes are FP32) and added to the outflow sum once per bin
        float o2 = 0.0f;
        if constexpr (G == 1) {
          if (gx == nx - 1) o2 += wRf * xr.x;
          if (gy == ny - 1) o2 += wvf * yt.x;
        } else {
          if (gx == 0) o2 -= xl.x;
          if (gx == nx - 1) o2 += xr.x;
          if (gy == 0) o2 -= yb.x;
          if (gy == ny - 1) o2 += yt.x;
        }
        const I dnu = sizeof(I) == 8 ? I(v.t_dnu[k]) : I(tb.y);
        if constexpr (sizeof(I) == 8)
          out = fma(dnu * cdx, f2d_alu(o2), out);
        else
          out += dnu * (cdx * o2);
        if (v.spec) {  // emergent spectrum: the escaping energy of each outer face
          double* sp = v.spec + static_cast<long long>(k) * v.nf;
          const double dxd = v.dx;
          const double u = (v.spec_unit * ((dxd * dxd) * dxd)) * double(dnu * cdx);
          if constexpr (G == 1) {
            if (gx == nx - 1) sp[gy] += u * double(wR * I(xr.x));
            if (gy == ny - 1) sp[ny + gx] += u * double(wcol * I(yt.x));
          } else {
            if (gx == 0) sp[gy] -= u * double(xl.x);
            if (gx == nx - 1) sp[ny + gy] += u * double(xr.x);
            if (gy == 0) sp[2 * ny + gx] -= u * double(yb.x);
            if (gy == ny - 1) sp[2 * ny + nx + gx] += u * double(yt.x);
          }
        }
      }
    }
    base = nbase;
  }
  if constexpr (MIX) {
    if (k1 > k0) step2_mix(k1 - 1, base - nc);
    if constexpr (TM != 2) {
      ab = fma(cA, sJ, cB * sHJ);
      en = sJ;
    }
  }
  if (valid && !DF) {
    if constexpr (MIX)
      store_force(v, cell, grp, fxs.value(), fys.value());
    else
      store_force(v, cell, grp, double(ax), double(ay));
  }
  double* part = v.partT + static_cast<long long>(blk) * kDiagSlots;
  double s;
  if constexpr (sizeof(I) == 4) {
    // FP32 accumulators: each tile's reductions stay off GB300's FP64 pipe
    // (~1/60 of the FP32 rate) except for the last eight-term sum
    const float wf = G == 1 ? wvf : 1.0f;
    s = block_sum_f32<NT>(em * wf, red);
    if (tid == 0) part[kSlotEmitted] = s;
    s = block_sum_f32<NT>(ab * wf, red);
    if (tid == 0) part[kSlotAbsorbed] = s;
    s = block_sum_f32<NT>(out, red);
    if (tid == 0) part[kSlotOutflow] = s;
    s = block_sum_f32<NT>(wk * wf, red);
    if (tid == 0) part[kSlotWork] = s;
    if (tdiag && !DF) {
      s = block_sum_f32<NT>(en * wf, red);
      if (tid == 0) part[kSlotEnergy] = s;
      int b = bad;
      for (int o = 16; o > 0; o >>= 1) b += __shfl_down_sync(0xffffffffu, b, o);
      float m = mxf2;
      for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_down_sync(0xffffffffu, m, o));
      __syncthreads();
      if ((tid & 31) == 0) {
        red[tid >> 5] = double(b);
        red[NT / 32 + (tid >> 5)] = double(m);
      }
      __syncthreads();
      if (tid == 0) {
        double sb = 0.0, sm = 0.0;
        for (int w = 0; w < NT / 32; ++w) {
          sb += red[w];
          sm = fmax(sm, red[NT / 32 + w]);
        }
        part[kSlotBad] = sb;
        part[kSlotMaxF] = sqrt(sm);
      }
    }
  } else {
    // FP64 sums (LYM1_MIXED): c_tilde dt is already in ab; the emission of a
    // uniform-temperature cell is c dt L_cell sum_k dnu_k gem_k
    const double wd = G == 1 ? double(wvf) : 1.0;
    s = block_sum<NT>((cjs * (TM ? double(em) : sgk)) * wd, red);
    if (tid == 0) part[kSlotEmitted] = s;
    s = block_sum<NT>(double(ab) * wd, red);
    if (tid == 0) part[kSlotAbsorbed] = s;
    s = block_sum<NT>(double(out), red);
    if (tid == 0) part[kSlotOutflow] = s;
    s = block_sum<NT>(double(wk) * wd, red);
    if (tid == 0) part[kSlotWork] = s;
    if (tdiag && !DF) {
      s = block_sum<NT>(double(en) * wd, red);
      if (tid == 0) part[kSlotEnergy] = s;
      s = block_max<NT>(sqrt(double(mxf2)), red);
      if (tid == 0) part[kSlotMaxF] = s;
      s = block_sum<NT>(double(bad), red);
      if (tid == 0) part[kSlotBad] = s;
    }
  }
}

// The FP32 tile for any tile: under LYM1_MIXED (FP64 step 2 in the tile) the
// tiles without a source cell, nearly all of them, take the variant without
// the emission term.  A per-cell branch inside step 2 costs GB300's narrow
// FP64 pipe two issue slots per cell-bin even where no cell takes it, and a
// per-tile branch inside the bin loop keeps the compiler from interleaving
// step 2 with the face fluxes; a whole-tile choice costs neither.
template <class P, int G, int PT, int TS>
__device__ __forceinline__ void transport_tile_f32_any(const DeviceView& v, int x0, int y0, int blk,
                                                       int k0, int k1, int grp) {
  __shared__ TileSmemF32<TS> sm;
  if constexpr (sizeof(typename P::I) == 8 && (PT & 8) == 0) {
    const int gx = x0 + static_cast<int>(threadIdx.x), gy = y0 + static_cast<int>(threadIdx.y);
    const bool s = gx < v.nx && gy < v.ny && v.lum[static_cast<long long>(gy) * v.nx + gx] != 0.0;
    if (__syncthreads_or(s ? 1 : 0)) {
      transport_tile_f32<P, G, PT, TS, true>(sm, v, x0, y0, blk, k0, k1, grp);
      return;
    }
    transport_tile_f32<P, G, PT, TS, false>(sm, v, x0, y0, blk, k0, k1, grp);
  } else {
    transport_tile_f32<P, G, PT, TS, true>(sm, v, x0, y0, blk, k0, k1, grp);
  }
}

// blocks per SM the FP32 tile is register-budgeted for: 3 (80 registers).
// LYM1_MIXED's FP64 step holds more live values: at 3 blocks it spills
// ~60 bytes a thread, yet the third block's warps hide enough of the FP64
// pipe's latency to win (512^2 x 194: 2.47 ms at 2 blocks of 128 registers,
// 2.19 ms at 3, 2.38 ms at 4 with 190 bytes of spills)
template <class P>
__host__ __device__ constexpr int tile_f32_min_blocks() {
  return 3;
}

template <class P, int G, int PT>
__global__ void __launch_bounds__(kTileX* kTileY, tile_f32_min_blocks<P>()) transport_kernel_f32(DeviceView v) {
  transport_tile_f32_any<P, G, PT, 0>(v, blockIdx.x * kTileX, blockIdx.y * kTileY,
                                      blockIdx.y * gridDim.x + blockIdx.x, 0, v.nb, 0);
}

// ------------------------------------------------------------ frequency kernel
// LYM1_MIXED (FP32 state and coefficients, FP64 elimination): the
// elimination's conversions run on the integer pipe and its reciprocals are
// Newton-refined hardware approximations; the H rescale, the causality cap and
// the realisability check stay in the FP32 of the state.
template <class P>
__host__ __device__ constexpr bool freq_mix() {
  return sizeof(typename P::S) == 4 && sizeof(typename P::I) == 8;
}
template <class P>
__device__ __forceinline__ typename P::I to_elim(typename P::F x) {
  if constexpr (freq_mix<P>()) return f2d_alu(x);
  else return typename P::I(x);
}
template <class P>
__device__ __forceinline__ typename P::S to_state(typename P::I x) {
  if constexpr (freq_mix<P>()) return d2f_alu(x);
  else return typename P::S(x);
}
template <class P>
__device__ __forceinline__ typename P::I rcp_elim(typename P::I x) {
  using I = typename P::I;
  if constexpr (sizeof(I) == 4) return frcp(x);
  else if constexpr (freq_mix<P>()) return drcp_fs(x);
  else return I(1) / x;
}
// Exponential of the frequency-step coefficients: the FP64 policies' own
// (LYM1_FP64_DET) or library exp; FP32 coefficients take the accurate expf
// under LYM1_MIXED, whose frequency kernel is bound by its FP64 elimination
// (the FP32 pipe has room), and the fast __expf under LYM1_MIXED_FAST.  The
// approximate exponential's error grows with |x|, and the Peclet numbers of
// the line wings reach |P| ~ 1e3-1e5.
template <class P>
__device__ __forceinline__ typename P::F fexp(typename P::F x) {
  if constexpr (sizeof(typename P::F) == 8) return m_exp<P::DET>(x);
  else if constexpr (sizeof(typename P::I) == 8) return expf(x);
  else return __expf(x);
}

// The causality cap and the FP32 realisability statistics (max |H|^2 / J^2
// and the count of |H| > J) of the (cell, bin) pairs whose weighted J is above thr
__device__ __forceinline__ void causal_stats_f32(float J, float& Hx, float& Hy, float wf, float thr,
                                                 float& mxf2, int& bad) {
  causal(J, Hx, Hy);
  if (J * wf > thr) {
    const float h2 = Hx * Hx + Hy * Hy, jj = J * J;
    mxf2 = fmaxf(mxf2, fdiv(h2, jj));
    bad += (h2 > jj * 1.000002f) ? 1 : 0;
  }
}

// Coefficients of bin k for one cell (App. A): Peclet number P_k, dlt_k/K_k and
// E(-|P_k|) = expm1(-|P_k|) / (-|P_k|), with D_k from the post-source state.
template <class P, int G, class T>
__device__ __forceinline__ void freq_coef(typename P::F Jc, typename P::F Hxc, typename P::F Hyc,
                                          typename P::F Kc, typename P::F gxx,
                                          typename P::F gyy, typename P::F gsh,
                                          typename P::F gphi, typename P::F Hk,
                                          typename P::F Rk, const T* tn, const T* th, int k,
                                          typename P::F& Pk, typename P::F& ak,
                                          typename P::F& ek) {
  using F = typename P::F;
  if constexpr (sizeof(F) == 4) {
    const float r = Jc > kTinyJ ? frcp(Jc) : 0.0f;
    float fx = Hxc * r, fy = Hyc * r;
    cap_unit_f32(fx, fy);
    float Dxx, Dxy, Dyy, Dpp;
    closure_f32(fx, fy, Dxx, Dxy, Dyy, Dpp);
    float DdU = (Dxx * gxx + Dyy * gyy) + Dxy * gsh;
    if constexpr (G == 1) DdU = DdU + Dpp * gphi;
    const float K = Kc * Hk;
    const float rK = frcp(K);
    const float C = K * Rk + tn[k] * DdU;
    const float half = th[k];
    ak = half * rK;
    Pk = C * ak;
    const float z = -fabsf(Pk);
    // E(z) = expm1(z)/z: its Taylor polynomial to z^6 on [-0.5, 0] (truncation
    // below 2e-7 relative), (e^z - 1)/z below, where the subtraction loses at
    // most a factor 2.5 of e^z's relative error
    const float poly =
        1.0f + z * (0.5f + z * (1.0f / 6 + z * (1.0f / 24 + z * (1.0f / 120 + z * (1.0f / 720 + z * (1.0f / 5040))))));
    ek = (z > -0.5f) ? poly : (fexp<P>(z) - 1.0f) * frcp(z);
  } else {
    F fx = F(0), fy = F(0);
    if (Jc > F(0)) {
      if constexpr (P::DET) {
        fx = Hxc / Jc;
        fy = Hyc / Jc;
      } else {
        const F rJ = F(1) / Jc;
        fx = Hxc * rJ;
        fy = Hyc * rJ;
      }
    }
    cap_unit(fx, fy);
    F Dxx, Dxy, Dyy, Dpp;
    closure_d<P::DET>(fx, fy, Dxx, Dxy, Dyy, Dpp);
    F DdU = (Dxx * gxx + Dyy * gyy) + Dxy * gsh;
    if constexpr (G == 1) DdU = DdU + Dpp * gphi;  // D_phiphi <u_R / R>
    const F K = Kc * Hk;
    const F C = K * Rk + F(tn[k]) * DdU;
    const F half = F(th[k]);
    if constexpr (P::DET) {
      Pk = (C * half) / K;
      ak = half / K;
    } else {
      ak = half / K;
      Pk = C * ak;
    }
    const F z = -fabs(Pk);
    ek = (z == F(0)) ? F(1) : m_expm1<P::DET>(z) / z;
  }
}

// shared memory of the frequency step's per-bin tables, per bin.  With an FP64
// elimination (LYM1_MIXED, FP64) the tables keep 56 bytes a bin whatever they
// hold: that caps the resident blocks where the FP64 pipe is the limit and more
// blocks only contend for it (2.5 % slower when packed).
template <class P>
constexpr size_t freq_smem_per_bin() {
  return sizeof(typename P::I) == 8 ? 7 * sizeof(double)
                                    : 2 * sizeof(typename P::I) + 5 * sizeof(typename P::F);
}

template <class P, int G, int PT>
__device__ __forceinline__ void freq_block(const DeviceView& v, int blk) {
  using S = typename P::S;
  using F = typename P::F;
  using I = typename P::I;
  using T = F;  // table type in shared memory
  constexpr int NT = kFreqThreads;
  extern __shared__ double tabs_raw[];
  __shared__ double red[NT / 32];
  const int nb = v.nb;
  // per-bin tables, freq_smem_per_bin<P>() bytes a bin: two in the elimination
  // type I, then five in the coefficient type T
  constexpr bool MIX = freq_mix<P>();
  I* tdi = reinterpret_cast<I*>(tabs_raw);  // dnu_k in the elimination type
  I* tact = tdi + nb;                       // J above which |H|/J is checked
  // LYM1_MIXED: the threshold in FP32, and dnu_k / (c dt) in FP64
  float* tactf = reinterpret_cast<float*>(tact);
  I* tsk = MIX ? tact + nb : nullptr;
  float* tskf = tactf + nb;  // LYM1_MIXED: s_k in FP32 (the spare half of tact)
  T* tabs = reinterpret_cast<T*>(MIX ? tsk + nb : tact + nb);
  T* tH = tabs;
  T* tR = tabs + nb;
  T* tn = tabs + 2 * nb;
  T* th = tabs + 3 * nb;
  T* td = tabs + 4 * nb;
  if constexpr (sizeof(F) == 4) {
    const float thr = float(v.acc[14]);
    for (int i = threadIdx.x; i < nb; i += NT) {
      if constexpr (MIX) {
        tactf[i] = fmaxf(thr, 1e-30f) / v.f_dnu[i];
        tsk[i] = v.t_dnu[i] * v.rcdt;
        tskf[i] = d2f_alu(tsk[i]);
      } else {
        tact[i] = I(fmaxf(thr, 1e-30f) / v.f_dnu[i]);
      }
      tH[i] = v.f_H[i];
      tR[i] = v.f_R[i];
      tn[i] = v.f_nbc[i];
      th[i] = v.f_half[i];
      td[i] = v.f_dnu[i];
      if constexpr (sizeof(I) == 4)
        tdi[i] = v.f_dnu[i];
      else
        tdi[i] = v.t_dnu[i];
    }
  } else {
    for (int i = threadIdx.x; i < nb; i += NT) {
      tact[i] = I(0);
      tH[i] = T(v.t_H[i]);
      tR[i] = T(v.t_R[i]);
      tn[i] = T(v.t_nbc[i]);
      th[i] = T(v.t_half[i]);
      td[i] = T(v.t_dnu[i]);
      tdi[i] = I(v.t_dnu[i]);
    }
  }
  __syncthreads();

  const S* __restrict__ Jin = static_cast<const S*>(v.J);
  const S* __restrict__ Hxin = static_cast<const S*>(v.Hx);
  const S* __restrict__ Hyin = static_cast<const S*>(v.Hy);
  S* __restrict__ Jout = static_cast<S*>(v.Jo);
  S* __restrict__ Hxout = static_cast<S*>(v.Hxo);
  S* __restrict__ Hyout = static_cast<S*>(v.Hyo);
  const long long nc = v.nc;
  const long long cell = static_cast<long long>(blk) * NT + threadIdx.x;
  RSum<I> en;
  I mxf = 0;
  float mxf2 = 0.0f;  // LYM1_MIXED: max |H|^2 / J^2
  int bad = 0;
  // axisymmetric grid: energy weight 2 pi Vol / dx^3 of the cell's column
  double wcell = 1.0;
  if constexpr (G == 1)
    if (cell < nc) wcell = v.g_wv[cell % v.nx];
  const I wI = I(wcell);
  const float wf = d2f_alu(wcell);
  if (cell < nc) {
    combine_force_groups(v, cell);
    const double alpha = v.alpha[cell];
    if (v.freq_step && alpha > 0.0) {
      const F Kc = narrow_to<F>(PT ? v.Kcc[cell] * alpha : v.Kc * alpha);
      const F gxx = narrow_to<F>(v.gxx[cell]), gyy = narrow_to<F>(v.gyy[cell]),
              gsh = narrow_to<F>(v.gsh[cell]);
      const F gphi = G == 1 ? narrow_to<F>(v.gphi[cell]) : F(0);
      // <H>_k and the recoil factor R_k of bin kk: per-bin tables, or the
      // cell's own under a temperature field
      const S* __restrict__ Hcs = static_cast<const S*>(v.Hc);
      const double hkT_c = PT ? v.hkTc[cell] : 0.0;
      const float hkT_f = d2f_alu(hkT_c);
      auto HR = [&](int kk, F& Hk, F& Rk) {
        if constexpr (PT) {
          Hk = F(Hcs[static_cast<long long>(kk) * nc + cell]);
          if constexpr (sizeof(F) == 8)
            Rk = F(hkT_c - v.t_2nu[kk]);
          else
            Rk = hkT_f - v.f_2nu[kk];
        } else {
          Hk = tH[kk];
          Rk = tR[kk];
        }
      };
      F H0, R0;
      HR(0, H0, R0);
      const I cdt = I(v.cdt);
      const float rcdt = float(1.0 / v.cdt);
      (void)rcdt;
      F P0, a0, e0, P1 = F(0), a1 = F(0), e1 = F(0);
      // LYM1_MIXED: Jin0, Jin1 hold s_k J_k formed in FP32 (as the bulk-copy sweep)
      I Jin0 = MIX ? f2d_alu(tskf[0] * float(Jin[cell])) : to_elim<P>(F(Jin[cell]));
      I Jin1 = 0;
      freq_coef<P, G>(F(Jin[cell]), F(Hxin[cell]), F(Hyin[cell]), Kc, gxx, gyy, gsh, gphi, H0, R0,
                      tn, th, 0, P0, a0, e0);
      // E_k = s_k + B_{k-1} q_{k-1}; outside FP64_DET as s_k + h_{k-1} E_{k-1}
      // (q_{k-1} = E_{k-1} / D'_{k-1}, h_{k-1} = B_{k-1} / D'_{k-1}): one product less
      I qprev = 0, gprev = 0, Bprev = 0, Aprev = 0, hprev = 0, Eprev = 0;
      // two-deep software pipeline: (nJ, nX, nY) hold bin k+1, loads for k+2 are in flight
      S nJ = S(0), nX = S(0), nY = S(0);
      if (nb > 1) {
        const long long o1 = nc + cell;
        nJ = Jin[o1];
        nX = Hxin[o1];
        nY = Hyin[o1];
      }
      for (int k = 0; k < nb; ++k) {
        I A = 0, B = 0;
        if (k + 1 < nb) {
          const S Jr = nJ, Xr = nX, Yr = nY;
          if (k + 2 < nb) {
            const long long o2 = static_cast<long long>(k + 2) * nc + cell;
            nJ = Jin[o2];
            nX = Hxin[o2];
            nY = Hyin[o2];
          }
          if constexpr (MIX)
            Jin1 = f2d_alu(tskf[k + 1] * float(Jr));
          else
            Jin1 = to_elim<P>(F(Jr));
          F H1, R1;
          HR(k + 1, H1, R1);
          freq_coef<P, G>(F(Jr), F(Xr), F(Yr), Kc, gxx, gyy, gsh, gphi, H1, R1, tn, th, k + 1, P1,
                          a1, e1);
          const F d1 = (-P0 > F(0)) ? -P0 : F(0);
          const F d2 = (P1 > F(0)) ? P1 : F(0);
          const F m = (d1 > d2) ? d1 : d2;
          const F den = fexp<P>(d1 - m) * (e0 * a0) + fexp<P>(d2 - m) * (e1 * a1);
          if constexpr (sizeof(F) == 4) {
            const float rden = frcp(den);
            A = to_elim<P>(fexp<P>(-P0 - m) * rden);
            B = to_elim<P>(fexp<P>(P1 - m) * rden);
          } else if constexpr (P::DET) {
            A = I(fexp<P>(-P0 - m) / den);
            B = I(fexp<P>(P1 - m) / den);
          } else {
            const F rden = F(1) / den;
            A = I(fexp<P>(-P0 - m) * rden);
            B = I(fexp<P>(P1 - m) * rden);
          }
        }
        I s;
        if constexpr (sizeof(I) == 4)
          s = tdi[k] * rcdt;
        else if constexpr (MIX)
          s = tsk[k];
        else if constexpr (P::DET)
          s = tdi[k] / cdt;
        else
          s = tdi[k] * (I(1) / cdt);
        I E, r;
        if constexpr (P::DET)
          E = (k == 0) ? s : s + Bprev * qprev;
        else if constexpr (MIX)
          E = (k == 0) ? s : fma(hprev, Eprev, s);
        else
          E = (k == 0) ? s : s + hprev * Eprev;
        if constexpr (MIX)
          r = (k == 0) ? Jin0 : fma(Aprev, gprev, Jin0);
        else
          r = (k == 0) ? s * Jin0 : s * Jin0 + Aprev * gprev;
        const I Dp = E + A;
        const I inv = rcp_elim<P>(Dp);
        const I g = r * inv;
        const I h = B * inv;
        if constexpr (P::DET)
          qprev = E * inv;
        hprev = h;
        Eprev = E;
        gprev = g;
        Bprev = B;
        Aprev = A;
        const long long o = static_cast<long long>(k) * nc + cell;
        Jout[o] = to_state<P>(g);
        Hxout[o] = to_state<P>(h);
        P0 = P1;
        a0 = a1;
        e0 = e1;
        Jin0 = Jin1;
      }
      I Jnext = 0;
      long long o = static_cast<long long>(nb - 1) * nc + cell;
      S cg = Jout[o], ch = Hxout[o], cJ = Jin[o], cX = Hxin[o], cY = Hyin[o];
      for (int k = nb - 1; k >= 0; --k) {
        const S gS = cg, hS = ch, JS = cJ, XS = cX, YS = cY;
        const long long oc = o;
        if (k > 0) {  // prefetch bin k-1
          o -= nc;
          cg = Jout[o];
          ch = Hxout[o];
          cJ = Jin[o];
          cX = Hxin[o];
          cY = Hyin[o];
        }
        if constexpr (MIX) {
          const double g = f2d_alu(gS), h = f2d_alu(hS);
          const double Jn = (k == nb - 1) ? g : fma(h, Jnext, g);
          Jnext = Jn;
          const float Jnf = d2f_alu(Jn);
          const float ratio = JS > kTinyJ ? fdiv(Jnf, JS) : 0.0f;
          float Hx2 = ratio * XS, Hy2 = ratio * YS;
          causal_stats_f32(Jnf, Hx2, Hy2, G == 1 ? wf : 1.0f, tactf[k], mxf2, bad);
          Jout[oc] = Jnf;
          Hxout[oc] = Hx2;
          Hyout[oc] = Hy2;
          en.s = fma(tdi[k], Jn, en.s);
          continue;
        }
        const I g = I(gS), h = I(hS);
        const I Jn = (k == nb - 1) ? g : g + h * Jnext;
        Jnext = Jn;
        const I Jo = I(JS);
        I ratio;
        if constexpr (sizeof(I) == 4)
          ratio = (Jo > kTinyJ) ? fdiv(Jn, Jo) : 0.0f;
        else
          ratio = (Jo > I(0)) ? Jn / Jo : I(0);
        I Hx2 = ratio * I(XS);
        I Hy2 = ratio * I(YS);
        causal(Jn, Hx2, Hy2);
        Jout[oc] = S(Jn);
        Hxout[oc] = S(Hx2);
        Hyout[oc] = S(Hy2);
        en.add(tdi[k] * Jn);
        if ((G == 1 ? Jn * wI : Jn) > tact[k]) {
          const I hn = sqrt(Hx2 * Hx2 + Hy2 * Hy2);
          mxf = fmax(mxf, hn / Jn);
          bad += (hn > Jn * I(1.000001)) ? 1 : 0;
        }
      }
    } else {
      for (int k = 0; k < nb; ++k) {
        const long long o = static_cast<long long>(k) * nc + cell;
        const S J = Jin[o];
        if constexpr (MIX) {
          float Hxi = Hxin[o], Hyi = Hyin[o];
          causal_stats_f32(J, Hxi, Hyi, G == 1 ? wf : 1.0f, tactf[k], mxf2, bad);
          Jout[o] = J;
          Hxout[o] = Hxi;
          Hyout[o] = Hyi;
          en.s = fma(tdi[k], f2d_alu(J), en.s);
          continue;
        }
        const I Ji = I(J);
        I Hxi = I(Hxin[o]), Hyi = I(Hyin[o]);
        causal(Ji, Hxi, Hyi);
        Jout[o] = J;
        Hxout[o] = S(Hxi);
        Hyout[o] = S(Hyi);
        en.add(tdi[k] * Ji);
        if ((G == 1 ? Ji * wI : Ji) > tact[k]) {
          const I hn = sqrt(Hxi * Hxi + Hyi * Hyi);
          mxf = fmax(mxf, hn / Ji);
          bad += (hn > Ji * I(1.000001)) ? 1 : 0;
        }
      }
    }
  }
  double* part = v.partF + static_cast<long long>(blk) * kDiagSlots;
  double s;
  s = block_sum<NT>(en.value() * wcell, red);
  if (threadIdx.x == 0) part[kSlotEnergy] = s;
  s = block_max<NT>(MIX ? double(sqrtf(mxf2)) : double(mxf), red);
  if (threadIdx.x == 0) part[kSlotMaxF] = s;
  s = block_sum<NT>(double(bad), red);
  if (threadIdx.x == 0) part[kSlotBad] = s;
}


// ------------------------------------------- bulk-copy pipeline (FP32 state)
// Shared-memory ring fed by cp.async.bulk (one thread issues, an mbarrier per
// stage counts the bytes).  Every wait is bounded: past kMaxSpins polls the
// block records LYM1_ETIMEOUT in the context's status word and gives up.
// ring depth of the bulk-copy pipeline: 6 bins for an FP32 elimination (the
// smaller ring lets 9 blocks share an SM), 8 for an FP64 one (FP64-pipe-bound,
// where the resident blocks are fewer and each needs more bytes in flight)
template <class I>
__host__ __device__ constexpr int bulk_depth() {
  return sizeof(I) == 4 ? 6 : 8;
}
constexpr long long kMaxSpins = 100000000;          // backstop on the number of polls
constexpr unsigned long long kWaitLimitNs = 2000000000ull;  // 2 s per wait

__device__ __forceinline__ unsigned smem_addr(const void* p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_load(void* dst, const void* src, unsigned bytes,
                                          unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long* bar, unsigned parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = global_ns();
  for (long long i = 0; i < kMaxSpins; ++i) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((i & 255) == 0 && global_ns() - t0 > kWaitLimitNs) return false;
  }
  return false;
}
__device__ __forceinline__ void fence_proxy_async_global() {
  asm volatile("fence.proxy.async.global;" ::: "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Frequency step of one block of kFreqThreads cells with every bin row
// streamed through the ring (cell count a multiple of 4, so that every row
// segment starts on a 16-byte boundary and is a whole number of 16 bytes).
// Same arithmetic, in the same order, as freq_block.
template <class P, int G, int PT>
__device__ __forceinline__ void freq_block_bulk(const DeviceView& v, int blk) {
  using F = typename P::F;
  using I = typename P::I;
  using T = F;
  constexpr int NT = kFreqThreads, D = bulk_depth<I>();
  __shared__ __align__(128) float ring[D][5][NT];
  __shared__ __align__(8) unsigned long long barF[D], barB[D];
  __shared__ double red[NT / 32];
  extern __shared__ double tabs_raw[];
  const int nb = v.nb;
  constexpr bool MIX = freq_mix<P>();
  I* tdi = reinterpret_cast<I*>(tabs_raw);  // same layout as freq_block
  I* tact = tdi + nb;
  float* tactf = reinterpret_cast<float*>(tact);
  I* tsk = MIX ? tact + nb : nullptr;
  // LYM1_MIXED: s_k in FP32 in the spare half of tact (the right-hand side s_k J_k
  // is formed in FP32, like the other coefficients)
  float* tskf = tactf + nb;
  T* tabs = reinterpret_cast<T*>(MIX ? tsk + nb : tact + nb);
  T* tH = tabs;
  T* tR = tabs + nb;
  T* tn = tabs + 2 * nb;
  T* th = tabs + 3 * nb;
  const int tid = threadIdx.x;
  const float thr = float(v.acc[14]);
  for (int i = tid; i < nb; i += NT) {
    tH[i] = v.f_H[i];
    tR[i] = v.f_R[i];
    tn[i] = v.f_nbc[i];
    th[i] = v.f_half[i];
    if constexpr (sizeof(I) == 4)
      tdi[i] = v.f_dnu[i];
    else
      tdi[i] = v.t_dnu[i];
    if constexpr (MIX) {
      tactf[i] = fmaxf(thr, 1e-30f) / v.f_dnu[i];
      tsk[i] = v.t_dnu[i] * v.rcdt;
      tskf[i] = d2f_alu(tsk[i]);
    } else {
      tact[i] = I(fmaxf(thr, 1e-30f) / v.f_dnu[i]);
    }
  }
  if (tid == 0) {
    for (int s = 0; s < D; ++s) {
      mbar_init(&barF[s], 1);
      mbar_init(&barB[s], 1);
    }
    fence_mbar_init();
  }
  __syncthreads();

  const float* __restrict__ Jin = static_cast<const float*>(v.J);
  const float* __restrict__ Hxin = static_cast<const float*>(v.Hx);
  const float* __restrict__ Hyin = static_cast<const float*>(v.Hy);
  float* __restrict__ Jout = static_cast<float*>(v.Jo);
  float* __restrict__ Hxout = static_cast<float*>(v.Hxo);
  float* __restrict__ Hyout = static_cast<float*>(v.Hyo);
  const long long nc = v.nc;
  const long long c0 = static_cast<long long>(blk) * NT;
  const int ncell = static_cast<int>(nc - c0 < NT ? nc - c0 : NT);
  const unsigned rowb = static_cast<unsigned>(ncell) * 4u;
  const long long cell = c0 + tid;
  const bool valid = tid < ncell;
  const double alpha = valid ? v.alpha[cell] : 0.0;
  const bool act = valid && positive_bits(alpha);
  const F Kc = narrow_to<F>(PT ? (valid ? v.Kcc[cell] : 0.0) * alpha : v.Kc * alpha);
  // temperature field: <H>_k rides the forward ring as a fourth row
  const float* __restrict__ Hcf = static_cast<const float*>(v.Hc);
  const float hkT_c = PT ? d2f_alu(valid ? v.hkTc[cell] : 0.0) : 0.0f;
  const F gxx = valid ? narrow_to<F>(v.gxx[cell]) : F(0), gyy = valid ? narrow_to<F>(v.gyy[cell]) : F(0),
          gsh = valid ? narrow_to<F>(v.gsh[cell]) : F(0);
  F gphi = F(0);
  double wcell = 1.0;  // axisymmetric grid: energy weight of the cell's column
  if constexpr (G == 1)
    if (valid) {
      gphi = narrow_to<F>(v.gphi[cell]);
      wcell = v.g_wv[cell % v.nx];
    }
  const I wI = I(wcell);
  const I cdt = I(v.cdt);
  const float rcdt = float(1.0 / v.cdt);
  (void)rcdt;
  if (valid) combine_force_groups(v, cell);

  auto issue_fwd = [&](int k) {
    const int s = k % D;
    const long long off = static_cast<long long>(k) * nc + c0;
    mbar_expect_tx(&barF[s], (PT ? 4u : 3u) * rowb);
    bulk_load(&ring[s][0][0], Jin + off, rowb, &barF[s]);
    bulk_load(&ring[s][1][0], Hxin + off, rowb, &barF[s]);
    bulk_load(&ring[s][2][0], Hyin + off, rowb, &barF[s]);
    if constexpr (PT) bulk_load(&ring[s][3][0], Hcf + off, rowb, &barF[s]);
  };
  auto issue_bwd = [&](int j) {  // j-th bin from the top
    const int s = j % D, k = nb - 1 - j;
    const long long off = static_cast<long long>(k) * nc + c0;
    mbar_expect_tx(&barB[s], 5u * rowb);
    bulk_load(&ring[s][0][0], Jout + off, rowb, &barB[s]);
    bulk_load(&ring[s][1][0], Hxout + off, rowb, &barB[s]);
    bulk_load(&ring[s][2][0], Jin + off, rowb, &barB[s]);
    bulk_load(&ring[s][3][0], Hxin + off, rowb, &barB[s]);
    bulk_load(&ring[s][4][0], Hyin + off, rowb, &barB[s]);
  };
  // bounded failure: record the status, let the copies in flight land, stop
  auto give_up = [&](unsigned long long* bars, int issued_upto, int consumed) {
    if (tid == 0) {
      atomicExch(v.status, 1);
      for (int j = consumed; j < issued_upto; ++j) mbar_wait_bounded(&bars[j % D], (j / D) & 1);
    }
  };

  // status[1] == 1 (set only by lym1_debug_expire_wait) arms stage 0 without
  // issuing its copies, so that its bounded wait runs out
  const bool expire = v.status[1] == 1;
  if (tid == 0)
    for (int k = 0; k < nb && k < D; ++k) {
      if (k == 0 && expire)
        mbar_expect_tx(&barF[0], 3u * rowb);
      else
        issue_fwd(k);
    }
  // forward sweep, one bin behind the data: iteration k forms the
  // coefficients of bin k and eliminates row k-1
  F Pp = F(0), ap = F(0), ep = F(0);
  I Jp = 0, qprev = 0, gprev = 0, Bprev = 0, Aprev = 0, hprev = 0, Eprev = 0;
  long long ofw = cell - nc;  // plane offset of row k - 1
  for (int k = 0; k < nb; ++k, ofw += nc) {
    const int s = k % D;
    // every thread waits for the stage itself (the completed phase makes the
    // copied rows visible to it); a wait that ran out is caught at the one
    // block barrier below, after which nobody reads the ring
    const bool okF = mbar_wait_bounded(&barF[s], (k / D) & 1);
    if (act && okF) {
      const F Jc = F(ring[s][0][tid]), Xc = F(ring[s][1][tid]), Yc = F(ring[s][2][tid]);
      F Pk, ak, ek;
      const F Hk = PT ? F(ring[s][3][tid]) : F(tH[k]);
      const F Rk = PT ? F(hkT_c - v.f_2nu[k]) : F(tR[k]);
      freq_coef<P, G>(Jc, Xc, Yc, Kc, gxx, gyy, gsh, gphi, Hk, Rk, tn, th, k, Pk, ak, ek);
      if (k > 0) {
        const F d1 = (-Pp > F(0)) ? -Pp : F(0);
        const F d2 = (Pk > F(0)) ? Pk : F(0);
        const F m = (d1 > d2) ? d1 : d2;
        const F den = fexp<P>(d1 - m) * (ep * ap) + fexp<P>(d2 - m) * (ek * ak);
        const float rden = frcp(den);
        const I A = to_elim<P>(fexp<P>(-Pp - m) * rden);
        const I B = to_elim<P>(fexp<P>(Pk - m) * rden);
        // row k-1
        I sk;
        if constexpr (sizeof(I) == 4)
          sk = tdi[k - 1] * rcdt;
        else if constexpr (MIX)
          sk = tsk[k - 1];
        else
          sk = tdi[k - 1] / cdt;
        I E;  // as in freq_block
        if constexpr (P::DET)
          E = (k == 1) ? sk : sk + Bprev * qprev;
        else if constexpr (MIX)
          E = (k == 1) ? sk : fma(hprev, Eprev, sk);
        else
          E = (k == 1) ? sk : sk + hprev * Eprev;
        I r;
        if constexpr (MIX)  // Jp holds s_{k-1} J_{k-1}
          r = (k == 1) ? Jp : fma(Aprev, gprev, Jp);
        else
          r = (k == 1) ? sk * Jp : sk * Jp + Aprev * gprev;
        const I Dp = E + A;
        const I inv = rcp_elim<P>(Dp);
        const I g = r * inv;
        const I h = B * inv;
        if constexpr (P::DET)
          qprev = E * inv;
        hprev = h;
        Eprev = E;
        gprev = g;
        Bprev = B;
        Aprev = A;
        const long long o = ofw;
        Jout[o] = to_state<P>(g);
        Hxout[o] = to_state<P>(h);
      }
      Pp = Pk;
      ap = ak;
      ep = ek;
      if constexpr (MIX)
        Jp = f2d_alu(tskf[k] * Jc);
      else
        Jp = to_elim<P>(Jc);
    }
    if (__syncthreads_or(okF ? 0 : 1)) {  // stage s consumed (or a wait ran out)
      give_up(barF, nb < k + D ? nb : k + D, k);
      return;
    }
    if (tid == 0 && k + D < nb) issue_fwd(k + D);
  }
  if (act) {  // last row: no interface above
    I sk;
    if constexpr (sizeof(I) == 4)
      sk = tdi[nb - 1] * rcdt;
    else if constexpr (MIX)
      sk = tsk[nb - 1];
    else
      sk = tdi[nb - 1] / cdt;
    I E;
    if constexpr (P::DET)
      E = (nb == 1) ? sk : sk + Bprev * qprev;
    else if constexpr (MIX)
      E = (nb == 1) ? sk : fma(hprev, Eprev, sk);
    else
      E = (nb == 1) ? sk : sk + hprev * Eprev;
    I r;
    if constexpr (MIX)
      r = (nb == 1) ? Jp : fma(Aprev, gprev, Jp);
    else
      r = (nb == 1) ? sk * Jp : sk * Jp + Aprev * gprev;
    const I inv = rcp_elim<P>(E);
    const long long o = static_cast<long long>(nb - 1) * nc + cell;
    Jout[o] = to_state<P>(r * inv);
    Hxout[o] = 0.0f;
  }
  // the elimination factors go back through the async proxy
  fence_proxy_async_global();
  __syncthreads();
  if (tid == 0)
    for (int j = 0; j < nb && j < D; ++j) issue_bwd(j);
  RSum<I> en;
  I mxf = 0;
  float mxf2 = 0.0f;  // LYM1_MIXED: max |H|^2 / J^2
  int bad = 0;
  I Jnext = 0;
  const float wf = G == 1 ? d2f_alu(wcell) : 1.0f;
  long long obw = static_cast<long long>(nb - 1) * nc + cell;  // plane offset of row k
  for (int j = 0; j < nb; ++j, obw -= nc) {
    const int s = j % D, k = nb - 1 - j;
    const bool okB = mbar_wait_bounded(&barB[s], (j / D) & 1);
    if (valid && okB) {
      const long long o = obw;
      const float Jo = ring[s][2][tid], Xo = ring[s][3][tid], Yo = ring[s][4][tid];
      if (MIX && act) {
        const double g = f2d_alu(ring[s][0][tid]), h = f2d_alu(ring[s][1][tid]);
        const double Jn = (j == 0) ? g : fma(h, double(Jnext), g);
        Jnext = I(Jn);
        const float Jnf = d2f_alu(Jn);
        const float ratio = Jo > kTinyJ ? fdiv(Jnf, Jo) : 0.0f;
        float Hx2 = ratio * Xo, Hy2 = ratio * Yo;
        causal_stats_f32(Jnf, Hx2, Hy2, wf, tactf[k], mxf2, bad);
        Jout[o] = Jnf;
        Hxout[o] = Hx2;
        Hyout[o] = Hy2;
        if constexpr (MIX) en.s = fma(tdi[k], Jn, en.s);
      } else if (MIX) {
        float Hxi = Xo, Hyi = Yo;
        causal_stats_f32(Jo, Hxi, Hyi, wf, tactf[k], mxf2, bad);
        Jout[o] = Jo;
        Hxout[o] = Hxi;
        Hyout[o] = Hyi;
        if constexpr (MIX) en.s = fma(tdi[k], f2d_alu(Jo), en.s);
      } else if (act) {
        const I g = I(ring[s][0][tid]), h = I(ring[s][1][tid]);
        const I Jn = (j == 0) ? g : g + h * Jnext;
        Jnext = Jn;
        I ratio;
        if constexpr (sizeof(I) == 4)
          ratio = (Jo > kTinyJ) ? fdiv(Jn, Jo) : 0.0f;
        else
          ratio = (I(Jo) > I(0)) ? Jn / I(Jo) : I(0);
        I Hx2 = ratio * I(Xo), Hy2 = ratio * I(Yo);
        causal(Jn, Hx2, Hy2);
        Jout[o] = float(Jn);
        Hxout[o] = float(Hx2);
        Hyout[o] = float(Hy2);
        en.add(tdi[k] * Jn);
        if ((G == 1 ? Jn * wI : Jn) > tact[k]) {
          const I hn = sqrt(Hx2 * Hx2 + Hy2 * Hy2);
          mxf = fmax(mxf, hn / Jn);
          bad += (hn > Jn * I(1.000001)) ? 1 : 0;
        }
      } else {
        const I Ji = I(Jo);
        I Hxi = I(Xo), Hyi = I(Yo);
        causal(Ji, Hxi, Hyi);
        Jout[o] = Jo;
        Hxout[o] = float(Hxi);
        Hyout[o] = float(Hyi);
        en.add(tdi[k] * Ji);
        if ((G == 1 ? Ji * wI : Ji) > tact[k]) {
          const I hn = sqrt(Hxi * Hxi + Hyi * Hyi);
          mxf = fmax(mxf, hn / Ji);
          bad += (hn > Ji * I(1.000001)) ? 1 : 0;
        }
      }
    }
    if (__syncthreads_or(okB ? 0 : 1)) {  // stage s consumed (or a wait ran out)
      give_up(barB, nb < j + D ? nb : j + D, j);
      return;
    }
    if (tid == 0 && j + D < nb) issue_bwd(j + D);
  }
  double* part = v.partF + static_cast<long long>(blk) * kDiagSlots;
  double sres;
  sres = block_sum<NT>(en.value() * wcell, red);
  if (tid == 0) part[kSlotEnergy] = sres;
  sres = block_max<NT>(MIX ? double(sqrtf(mxf2)) : double(mxf), red);
  if (tid == 0) part[kSlotMaxF] = sres;
  sres = block_sum<NT>(double(bad), red);
  if (tid == 0) part[kSlotBad] = sres;
}

// FP32 state with a cell count that is a multiple of 4 takes the bulk-copy
// pipeline; everything else the register-prefetch sweep
template <class P, int G, int PT>
__device__ __forceinline__ void freq_dispatch(const DeviceView& v, int blk) {
  if constexpr (sizeof(typename P::S) == 4) {
    if ((v.nc & 3) == 0) {
      freq_block_bulk<P, G, PT>(v, blk);
      return;
    }
  }
  freq_block<P, G, PT>(v, blk);
}

// FP32 state: at most 64 registers so that 8 blocks (32 warps) per SM keep
// enough loads in flight for the latency-bound bin sweeps
template <class P, int G, int PT>
__global__ void __launch_bounds__(kFreqThreads, sizeof(typename P::S) == 4 ? (sizeof(typename P::I) == 4 ? 9 : 8) : 1)
    freq_kernel(DeviceView v) {
  freq_dispatch<P, G, PT>(v, blockIdx.x);
}

// ---------------------------------------- step 2 under the acceptance rule
// Sec. 2.1 step 2 and its footnote: every cell subcycles its implicit
// emission/absorption update.  A trial substep is accepted when the cell's
// Lya energy density changes by |e'' - e'| / (e' + e_floor) < 0.1 (e_floor =
// 4 pi J_floor / c, J_floor = 1e-15 erg cm^-2 s^-1 sr^-1); otherwise it is
// halved and redone, until the accepted substeps fill the RT step.  Where the
// paper gives only the halving: every cell starts with the whole step, an
// accepted substep doubles the next trial (capped by what is left),
// substeps are whole multiples of dt / 2^kSubLevels, one of that size is
// accepted whatever the change, and once a cell has made kSubMaxTrials trials
// every further trial is accepted (a bound on the loop that finite inputs do
// not reach).  One thread per cell, in place on the post-transport state (the
// view's input arrays, which the frequency step then reads); the force, the
// emission and the absorption add up over the accepted substeps.  The
// decision is taken in FP64 for every policy, the updates in the policy's
// implicit type, with the operations in the order written (bit for bit the
// oracle's under LYM1_FP64_DET).  Partial sums go to the frequency-step
// partials of the same 128-cell block: emitted and absorbed, and, without a
// frequency step, the energy and realisability slots.
constexpr int kSubLevels = 40;
constexpr int kSubMaxTrials = 1 << 16;
constexpr double kJFloor = 1e-15;

template <class P, int G, int TM>
__device__ __forceinline__ void subcycle_block(const DeviceView& v, int blk) {
  using S = typename P::S;
  using I = typename P::I;
  constexpr int NT = kFreqThreads;
  __shared__ double red[NT / 32];
  S* __restrict__ Js = static_cast<S*>(const_cast<void*>(v.J));
  S* __restrict__ Hxs = static_cast<S*>(const_cast<void*>(v.Hx));
  S* __restrict__ Hys = static_cast<S*>(const_cast<void*>(v.Hy));
  const S* __restrict__ Hcs = static_cast<const S*>(v.Hc);
  const S* __restrict__ Gcs = static_cast<const S*>(v.Gc);
  const int nb = v.nb;
  const long long nc = v.nc;
  const long long cell = static_cast<long long>(blk) * NT + threadIdx.x;
  const bool valid = cell < nc;
  double wcell = 1.0;
  if constexpr (G == 1)
    if (valid) wcell = v.g_wv[cell % v.nx];
  I em = I(0), ab = I(0), ax = I(0), ay = I(0);
  double en = 0.0, mxf = 0.0, bad = 0.0;
  if (valid) {
    const I alpha = I(v.alpha[cell]), rho = I(v.rho[cell]), pd = I(v.pd[cell]);
    const I kabs = I(v.kabs), kF = I(v.kF);
    const double lum = v.lum[cell];
    // temperature field with FP32 state: the emission factors are stored over
    // the cell's maximum
    const double gmc = (TM && sizeof(S) == 4) ? v.gmaxc[cell] : 1.0;
    // FP32 implicit type: the source term c_tilde h j_k is formed in FP64 and
    // rounded once (j_k alone falls below the FP32 range in the far wings), and
    // the absorption sum takes c_tilde h kappa_k J'' (kappa_k J'' alone can)
    constexpr bool F32 = sizeof(I) == 4;
    auto coef = [&](int k, long long o, double chd, I& kap, I& aF, I& js) {
      const I Hk = TM ? I(Hcs[o]) : I(v.t_H[k]);
      const I aH = alpha * Hk;
      kap = rho * kabs + pd * aH;
      aF = aH + rho * kF;
      const double jd = lum != 0.0 ? lum * (TM ? gmc * double(Gcs[o]) : v.t_gem[k]) : 0.0;
      js = F32 ? I(chd * jd) : I(jd);
    };
    const long long full = 1LL << kSubLevels;
    long long done = 0, size = full;
    double e_cur = 0.0;
    for (int k = 0; k < nb; ++k)
      e_cur = e_cur + v.t_dnu[k] * double(Js[static_cast<long long>(k) * nc + cell]);
    int trials = 0;
    while (done < full) {
      if (size > full - done) size = full - done;
      const double h = v.dt * (double(size) / double(full));
      const double chd = v.ct * h;
      const I ch = I(chd);
      ++trials;
      double e_new = 0.0;
      for (int k = 0; k < nb; ++k) {
        const long long o = static_cast<long long>(k) * nc + cell;
        I kap, aF, js;
        coef(k, o, chd, kap, aF, js);
        const I Jt = F32 ? (I(Js[o]) + js) / (I(1) + ch * kap)
                         : (I(Js[o]) + ch * js) / (I(1) + ch * kap);
        e_new = e_new + v.t_dnu[k] * double(Jt);
      }
      const double change = fabs(e_new - e_cur) / (e_cur + kJFloor);
      if (!(change < 0.1) && size > 1 && trials <= kSubMaxTrials) {
        size = size / 2;
        continue;
      }
      for (int k = 0; k < nb; ++k) {
        const long long o = static_cast<long long>(k) * nc + cell;
        I kap, aF, js;
        coef(k, o, chd, kap, aF, js);
        const I J2 = F32 ? (I(Js[o]) + js) / (I(1) + ch * kap)
                         : (I(Js[o]) + ch * js) / (I(1) + ch * kap);
        const I hx = I(Hxs[o]), hy = I(Hys[o]);
        const I Hx2 = hx / (I(1) + ch * aF);
        const I Hy2 = hy / (I(1) + ch * aF);
        const I dnu = I(v.t_dnu[k]);
        if constexpr (F32) {  // the product form of H' - H'' (no cancellation in thin bins)
          const I w = dnu * ((ch * aF) / (I(1) + ch * aF));
          ax = ax + w * hx;
          ay = ay + w * hy;
        } else {
          ax = ax + dnu * (hx - Hx2);
          ay = ay + dnu * (hy - Hy2);
        }
        em = em + dnu * (F32 ? js : ch * js);
        ab = ab + dnu * (F32 ? (ch * kap) * J2 : ch * (kap * J2));
        Js[o] = S(J2);
        Hxs[o] = S(Hx2);
        Hys[o] = S(Hy2);
      }
      e_cur = e_new;
      done += size;
      size = size * 2;
    }
    v.fx[cell] = v.fcoef * double(ax);
    v.fy[cell] = v.fcoef * double(ay);
    if (v.tdiag) {  // no frequency step follows: the energy and realisability here
      for (int k = 0; k < nb; ++k) {
        const long long o = static_cast<long long>(k) * nc + cell;
        const double J = double(Js[o]), hx = double(Hxs[o]), hy = double(Hys[o]);
        en = en + v.t_dnu[k] * J;
        const double hn = sqrt(hx * hx + hy * hy);
        if (J > 0.0) mxf = fmax(mxf, hn / J);
        if (hn > J * 1.000001 && hn > 0.0) bad += 1.0;
      }
    }
  }
  double* part = v.partF + static_cast<long long>(blk) * kDiagSlots;
  double s;
  s = block_sum<NT>(double(em) * wcell, red);
  if (threadIdx.x == 0) part[kSlotEmitted] = s;
  s = block_sum<NT>(double(ab) * wcell, red);
  if (threadIdx.x == 0) part[kSlotAbsorbed] = s;
  if (v.tdiag) {
    s = block_sum<NT>(en * wcell, red);
    if (threadIdx.x == 0) part[kSlotEnergy] = s;
    s = block_max<NT>(mxf, red);
    if (threadIdx.x == 0) part[kSlotMaxF] = s;
    s = block_sum<NT>(bad, red);
    if (threadIdx.x == 0) part[kSlotBad] = s;
  }
}

template <class P, int G, int TM>
__global__ void __launch_bounds__(kFreqThreads) subcycle_kernel(DeviceView v) {
  subcycle_block<P, G, TM>(v, blockIdx.x);
}

// ------------------------------------------------------------ batched launches
// Persistent kernels over a work list that spans several contexts (clouds of
// different sizes, one geometry and temperature mode): each item names a
// context and a tile (transport) or a block of cells (frequency step); blocks
// walk the list with a grid stride.
struct BatchItem {
  int ctx, x0, y0, blk;
  int k0, k1, grp;  // transport: the bins of this item and its bin group
};

template <class P, int G, int PT, int TS>
__global__ void __launch_bounds__(TileShape<TS>::X* TileShape<TS>::Y) transport_batched(
    const DeviceView* views, const BatchItem* items, int n) {
  for (int i = blockIdx.x; i < n; i += gridDim.x) {
    const BatchItem it = items[i];
    const DeviceView v = views[it.ctx];
    transport_tile<P, G, PT, TS>(v, it.x0, it.y0, it.blk, it.k0, it.k1, it.grp);
    __syncthreads();
  }
}

template <class P, int G, int PT, int TS>
__global__ void __launch_bounds__(TileShape<TS>::X* TileShape<TS>::Y, tile_f32_min_blocks<P>())
    transport_batched_f32(const DeviceView* views, const BatchItem* items, int n) {
  for (int i = blockIdx.x; i < n; i += gridDim.x) {
    const BatchItem it = items[i];
    const DeviceView v = views[it.ctx];
    transport_tile_f32_any<P, G, PT, TS>(v, it.x0, it.y0, it.blk, it.k0, it.k1, it.grp);
    __syncthreads();
  }
}

template <class P, int G, int PT>
__global__ void __launch_bounds__(kFreqThreads, sizeof(typename P::S) == 4 ? (sizeof(typename P::I) == 4 ? 9 : 8) : 1)
    freq_batched(const DeviceView* views, const BatchItem* items, int n) {
  for (int i = blockIdx.x; i < n; i += gridDim.x) {
    const BatchItem it = items[i];
    const DeviceView v = views[it.ctx];
    freq_dispatch<P, G, PT>(v, it.blk);
    __syncthreads();
  }
}

template <class P, int G, int TM>
__global__ void __launch_bounds__(kFreqThreads) subcycle_batched(const DeviceView* views,
                                                                 const BatchItem* items, int n) {
  for (int i = blockIdx.x; i < n; i += gridDim.x) {
    const BatchItem it = items[i];
    const DeviceView v = views[it.ctx];
    subcycle_block<P, G, TM>(v, it.blk);
    __syncthreads();
  }
}

template <class P, int G, int PT, int TS>
int launch_transport_batched_s(const DeviceView* views, const BatchItem* items, int n, int grid,
                               int nb_max, cudaStream_t st) {
  const dim3 block(TileShape<TS>::X, TileShape<TS>::Y);
  if constexpr (sizeof(typename P::S) == 4) {
    const size_t smem = sizeof(float) * 4 * static_cast<size_t>(nb_max);
    transport_batched_f32<P, G, PT, TS><<<grid, block, smem, st>>>(views, items, n);
  } else {
    transport_batched<P, G, PT, TS><<<grid, block, 0, st>>>(views, items, n);
  }
  return static_cast<int>(cudaGetLastError());
}

// tile shape 1 is instantiated for the plain table modes only (0, 1)
template <class P, int G, int PT>
int launch_transport_batched_g(const DeviceView* views, const BatchItem* items, int n, int grid,
                               int nb_max, cudaStream_t st, int shape) {
  if constexpr (PT == 0 || PT == 1)
    if (shape == 1) return launch_transport_batched_s<P, G, PT, 1>(views, items, n, grid, nb_max, st);
  if (shape != 0) return static_cast<int>(cudaErrorInvalidValue);
  return launch_transport_batched_s<P, G, PT, 0>(views, items, n, grid, nb_max, st);
}

template <class P, int G, int PT>
int launch_freq_batched_g(const DeviceView* views, const BatchItem* items, int n, int grid,
                          int nb_max, cudaStream_t st) {
  const size_t smem = freq_smem_per_bin<P>() * static_cast<size_t>(nb_max);
  freq_batched<P, G, PT><<<grid, kFreqThreads, smem, st>>>(views, items, n);
  return static_cast<int>(cudaGetLastError());
}

// (geometry, temperature mode) -> template instance
// transport: pt & 3 = 0 uniform temperature, 1 temperature field, 2 broad
// bands; pt & 4 = active-bin pruning; pt & 8 = step 2 left to the subcycling
// kernel of the acceptance rule (Lya only: not with broad bands)
#define LYM1_PT_(F_, G_, ...)                                                   \
  (pt == 13  ? F_<P, G_, 13>(__VA_ARGS__)                                       \
   : pt == 12 ? F_<P, G_, 12>(__VA_ARGS__)                                      \
   : pt == 9 ? F_<P, G_, 9>(__VA_ARGS__)                                        \
   : pt == 8 ? F_<P, G_, 8>(__VA_ARGS__)                                        \
   : pt == 6 ? F_<P, G_, 6>(__VA_ARGS__)                                        \
   : pt == 5 ? F_<P, G_, 5>(__VA_ARGS__)                                        \
   : pt == 4 ? F_<P, G_, 4>(__VA_ARGS__)                                        \
   : pt == 2 ? F_<P, G_, 2>(__VA_ARGS__)                                        \
   : pt == 1 ? F_<P, G_, 1>(__VA_ARGS__)                                        \
             : F_<P, G_, 0>(__VA_ARGS__))
#define LYM1_GPT(F_, ...) \
  (geometry == 1 ? LYM1_PT_(F_, 1, __VA_ARGS__) : LYM1_PT_(F_, 0, __VA_ARGS__))
// frequency step: bands have none (pt 2 is refused before any launch)
#define LYM1_GPT_F(F_, ...)                                                        \
  (geometry == 1 ? (pt ? F_<P, 1, 1>(__VA_ARGS__) : F_<P, 1, 0>(__VA_ARGS__)) \
                 : (pt ? F_<P, 0, 1>(__VA_ARGS__) : F_<P, 0, 0>(__VA_ARGS__)))

template <class P>
int launch_transport_batched_t(int geometry, int pt, const DeviceView* views, const BatchItem* items,
                               int n, int grid, int nb_max, cudaStream_t st, int shape = 0) {
  return LYM1_GPT(launch_transport_batched_g, views, items, n, grid, nb_max, st, shape);
}

template <class P>
int launch_freq_batched_t(int geometry, int pt, const DeviceView* views, const BatchItem* items,
                          int n, int grid, int nb_max, cudaStream_t st) {
  pt &= 3;
  if (pt == 2) return static_cast<int>(cudaErrorInvalidValue);
  return LYM1_GPT_F(launch_freq_batched_g, views, items, n, grid, nb_max, st);
}

// The frequency step keeps its per-bin tables in dynamic shared memory, at most
// 7 doubles per bin (28 bytes for FP32 state); beside the static ring and
// reduction buffers that passes the 48 KB a launch may take by default for
// large bin counts.  The kernels are
// opted in to the size for LYM1_MAX_BINS bins once per device, outside any
// stream capture (at batch creation and before a direct launch), so that every
// bin count the ABI accepts launches.  The FP32 transport tables (4 floats per
// bin) stay under the default at LYM1_MAX_BINS.
constexpr size_t kFreqSmemMax = sizeof(double) * 7 * LYM1_MAX_BINS;

template <class P, int G, int PT, int TS>
int max_resident_transport_s(int nb_max) {
  int nblk = 0;
  constexpr int NT = TileShape<TS>::X * TileShape<TS>::Y;
  if constexpr (sizeof(typename P::S) == 4)
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nblk, transport_batched_f32<P, G, PT, TS>, NT,
                                                  sizeof(float) * 4 * static_cast<size_t>(nb_max));
  else
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nblk, transport_batched<P, G, PT, TS>, NT, 0);
  return nblk < 1 ? 1 : nblk;
}

template <class P, int G, int PT>
int max_resident_transport_g(int nb_max, int shape) {
  if constexpr (PT == 0 || PT == 1)
    if (shape == 1) return max_resident_transport_s<P, G, PT, 1>(nb_max);
  return max_resident_transport_s<P, G, PT, 0>(nb_max);
}

template <class P, int G, int PT>
int max_resident_freq_g(int nb_max) {
  cudaFuncSetAttribute(freq_batched<P, G, PT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       static_cast<int>(kFreqSmemMax));
  int nblk = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nblk, freq_batched<P, G, PT>, kFreqThreads,
                                                freq_smem_per_bin<P>() * static_cast<size_t>(nb_max));
  return nblk < 1 ? 1 : nblk;
}

template <class P>
int max_resident_transport(int geometry, int pt, int nb_max, int shape = 0) {
  return LYM1_GPT(max_resident_transport_g, nb_max, shape);
}

template <class P>
int max_resident_freq(int geometry, int pt, int nb_max) {
  pt &= 3;
  if (pt == 2) return 1;
  return LYM1_GPT_F(max_resident_freq_g, nb_max);
}

template <class P, int G, int PT>
int launch_transport_g(const DeviceView& v, cudaStream_t st) {
  dim3 grid((v.nx + kTileX - 1) / kTileX, (v.ny + kTileY - 1) / kTileY);
  if constexpr (sizeof(typename P::S) == 4) {
    const size_t smem = sizeof(float) * 4 * static_cast<size_t>(v.nb);
    transport_kernel_f32<P, G, PT><<<grid, dim3(kTileX, kTileY), smem, st>>>(v);
  } else {
    transport_kernel<P, G, PT><<<grid, dim3(kTileX, kTileY), 0, st>>>(v);
  }
  return static_cast<int>(cudaGetLastError());
}

template <class P, int G, int PT>
int launch_freq_g(const DeviceView& v, cudaStream_t st) {
  const size_t smem = freq_smem_per_bin<P>() * static_cast<size_t>(v.nb);
  cudaFuncSetAttribute(freq_kernel<P, G, PT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       static_cast<int>(kFreqSmemMax));
  freq_kernel<P, G, PT><<<freq_blocks(v.nc), kFreqThreads, smem, st>>>(v);
  return static_cast<int>(cudaGetLastError());
}

template <class P>
int launch_transport_t(const DeviceView& v, cudaStream_t st) {
  const int geometry = v.geometry, pt = v.pt;
  return LYM1_GPT(launch_transport_g, v, st);
}

template <class P>
int launch_freq_t(const DeviceView& v, cudaStream_t st) {
  const int geometry = v.geometry, pt = v.pt & 3;
  if (pt == 2) return static_cast<int>(cudaErrorInvalidValue);
  return LYM1_GPT_F(launch_freq_g, v, st);
}

// step 2 under the acceptance rule (Lya: uniform temperature or a
// temperature field; pt & 3 == 2, broad bands, is refused)
template <class P, int G, int TM>
int launch_subcycle_g(const DeviceView& v, cudaStream_t st) {
  subcycle_kernel<P, G, TM><<<freq_blocks(v.nc), kFreqThreads, 0, st>>>(v);
  return static_cast<int>(cudaGetLastError());
}

template <class P>
int launch_subcycle_t(const DeviceView& v, cudaStream_t st) {
  const int geometry = v.geometry, pt = v.pt & 3;
  if (pt == 2) return static_cast<int>(cudaErrorInvalidValue);
  return LYM1_GPT_F(launch_subcycle_g, v, st);
}

template <class P, int G, int TM>
int launch_subcycle_batched_g(const DeviceView* views, const BatchItem* items, int n, int grid,
                              cudaStream_t st) {
  subcycle_batched<P, G, TM><<<grid, kFreqThreads, 0, st>>>(views, items, n);
  return static_cast<int>(cudaGetLastError());
}

template <class P>
int launch_subcycle_batched_t(int geometry, int pt, const DeviceView* views, const BatchItem* items,
                              int n, int grid, cudaStream_t st) {
  pt &= 3;
  if (pt == 2) return static_cast<int>(cudaErrorInvalidValue);
  return LYM1_GPT_F(launch_subcycle_batched_g, views, items, n, grid, st);
}

template <class P, int G, int TM>
int max_resident_subcycle_g(int) {
  int nblk = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nblk, subcycle_batched<P, G, TM>, kFreqThreads, 0);
  return nblk < 1 ? 1 : nblk;
}

template <class P>
int max_resident_subcycle(int geometry, int pt) {
  pt &= 3;
  if (pt == 2) return 1;
  return LYM1_GPT_F(max_resident_subcycle_g, 0);
}

}  // namespace lym1
