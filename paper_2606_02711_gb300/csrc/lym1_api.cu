// lym1_api.cu -- host side of the C ABI declared in include/lym1.h: context
// lifetime, device memory, the substep driver and the diagnostics.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <utility>
#include <vector>

#include "lym1.h"
#include "lym1_internal.h"

using namespace lym1;

struct lym1_ctx {
  int nx = 0, ny = 0, nb = 0, precision = 0, gray = 0, freq_step = 0, recoil = 0, geometry = 0;
  int vac = 0;  // outflow sides into vacuum, bit 0 x-, 1 x+, 2 y-, 3 y+
  // temperature field: per [bin][cell] tables (state type) and per-cell constants
  int pt = 0;
  void *Hc = nullptr, *Gc = nullptr;
  double *gmaxc = nullptr, *Kcc = nullptr, *hkTc = nullptr, *t_2nu = nullptr, *sig0c = nullptr,
         *Tc = nullptr;
  // temperature field: n_HI and the grid edges, for lym1_set_temperature
  double* nhi = nullptr;
  std::vector<double> edges;
  float* f_2nu = nullptr;
  // broad bands (pt = 2): Hc = alpha_F, Gc = emissivity, Kb = kappa per [band][cell]
  int bands = 0;
  void* Kb = nullptr;
  // emergent spectrum accumulation (lym1_spectrum_enable)
  double* spec = nullptr;
  int spec_on = 0;
  long long nc = 0;
  double dx = 0, T = 0, c_tilde = 0, cfl = 0, kabs = 0, kF = 0, dt_cfl = 0, umax = 0;
  double L_tot = 0, device_bytes = 0, gem_max = 1;
  // bumped when a value baked into the device views changes (c_tilde): a
  // batch holding this context re-uploads its views before the next launch
  unsigned view_gen = 0;
  unsigned long long* ctw = nullptr;  // dynamic c_tilde: running max, result
  // luminosity sum on the device (lym1_set_sources), read back when needed
  double* lsum = nullptr;
  int L_pending = 0;
  // active-bin pruning (lym1_set_pruning): cut, per-bin energies and flags;
  // prune_gen changes whenever the cut changes
  double prune = 0.0;
  double* Ebin = nullptr;
  unsigned char* active = nullptr;
  unsigned prune_gen = 0;
  // substep acceptance rule of step 2 (lym1_set_accept); accept_gen changes
  // with it
  int accept = 0;
  unsigned accept_gen = 0;
  long long substeps_done = 0;
  cudaStream_t stream = nullptr;
  BinTables tab;
  size_t selem = 8;  // bytes per state element
  // device arrays
  void* A[3] = {nullptr, nullptr, nullptr};  // current state J, Hx, Hy
  void* B[3] = {nullptr, nullptr, nullptr};  // ping-pong partner
  double *alpha = nullptr, *rho = nullptr, *pd = nullptr, *ux = nullptr, *uy = nullptr;
  double *gxx = nullptr, *gyy = nullptr, *gsh = nullptr, *lum = nullptr;
  double *t_dH = nullptr;
  double *t_dnu = nullptr, *t_H = nullptr, *t_gem = nullptr, *t_half = nullptr, *t_R = nullptr,
         *t_nbc = nullptr;
  double *fx = nullptr, *fy = nullptr, *partT = nullptr, *partF = nullptr, *acc = nullptr;
  double* staging = nullptr;  // one bin plane of doubles
  double* fpart = nullptr;    // force-reduction partials
  int* status = nullptr;      // set by a kernel whose bounded wait expired
  float *f_H = nullptr, *f_dnu = nullptr, *f_G = nullptr, *f_R = nullptr, *f_nbc = nullptr,
        *f_half = nullptr;
  // axisymmetric grid (geometry 1): <u_R/R> per cell and the per-column tables
  double *gphi = nullptr, *g_AR = nullptr, *g_AZ = nullptr, *g_Vol = nullptr, *g_invR = nullptr,
         *g_dlL = nullptr, *g_dlR = nullptr, *g_wv = nullptr, *g_V2pi = nullptr;
  float *gf_r0 = nullptr, *gf_r1 = nullptr, *gf_hoop = nullptr, *gf_dlL = nullptr,
        *gf_dlR = nullptr, *gf_wv = nullptr;
  double g_wR = 0;
  std::vector<void*> allocs;
  // persistent graph-replayed path for CFL substeps (a batch of this context alone)
  lym1_batch* self_batch = nullptr;
  // kernel timing (lym1_profile_enable): event pairs per launch, kind 0..2
  bool profiling = false;
  std::vector<cudaEvent_t> ev_start, ev_stop;
  std::vector<int> ev_kind;
};

namespace {

constexpr int kForceBlocks = 152 * 4;

// host mirror of the kernels' BatchItem {ctx, x0, y0, blk, k0, k1, grp}
struct BatchItemHost {
  int ctx, x0, y0, blk;
  int k0, k1, grp;
};

int map_cuda(cudaError_t e) {
  if (e == cudaSuccess) return LYM1_OK;
  if (e == cudaErrorMemoryAllocation) return LYM1_ENOMEM;
  if (e == cudaErrorNoDevice || e == cudaErrorInsufficientDriver) return LYM1_ENODEVICE;
  return LYM1_ECUDA;
}

#define LYM1_TRY(expr)                                 \
  do {                                                 \
    const cudaError_t e_ = (expr);                     \
    if (e_ != cudaSuccess) return map_cuda(e_);        \
  } while (0)

#define LYM1_TRYK(expr)                                                  \
  do {                                                                   \
    const int e_ = (expr);                                               \
    if (e_ != 0) return map_cuda(static_cast<cudaError_t>(e_));          \
  } while (0)

int dalloc(lym1_ctx* c, void** p, size_t bytes) {
  if (bytes == 0) bytes = 16;
  const cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    *p = nullptr;
    cudaGetLastError();
    return LYM1_ENOMEM;
  }
  c->allocs.push_back(*p);
  c->device_bytes += static_cast<double>(bytes);
  return LYM1_OK;
}

template <class T>
int dalloc_t(lym1_ctx* c, T** p, size_t n) {
  void* q = nullptr;
  const int rc = dalloc(c, &q, n * sizeof(T));
  *p = static_cast<T*>(q);
  return rc;
}

bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

void free_all(lym1_ctx* c) {
  for (void* p : c->allocs) cudaFree(p);
  c->allocs.clear();
}

DeviceView make_view(const lym1_ctx* c, double dt) {
  DeviceView v;
  v.nx = c->nx;
  v.ny = c->ny;
  v.nb = c->nb;
  v.nc = c->nc;
  v.dx = c->dx;
  v.J = c->A[0];
  v.Hx = c->A[1];
  v.Hy = c->A[2];
  v.Jo = c->B[0];
  v.Hxo = c->B[1];
  v.Hyo = c->B[2];
  v.alpha = c->alpha;
  v.rho = c->rho;
  v.pd = c->pd;
  v.ux = c->ux;
  v.uy = c->uy;
  v.gxx = c->gxx;
  v.gyy = c->gyy;
  v.gsh = c->gsh;
  v.lum = c->lum;
  v.t_dnu = c->t_dnu;
  v.t_H = c->t_H;
  v.t_gem = c->t_gem;
  v.t_half = c->t_half;
  v.t_R = c->t_R;
  v.t_nbc = c->t_nbc;
  v.t_dH = c->t_dH;
  v.fx = c->fx;
  v.fy = c->fy;
  v.partT = c->partT;
  v.partF = c->partF;
  v.kabs = c->kabs;
  v.kF = c->kF;
  v.Kc = 0.5 * (c->tab.lc.dnu_D * c->tab.lc.dnu_D);
  v.cdt = c->c_tilde * dt;
  v.cdt_dx = v.cdt / c->dx;
  v.cdt_c = v.cdt / kLight;
  // Sec. 2.3: f = 4 pi / (c ct dt) sum_k dnu_k (H' - H'')
  v.fcoef = (4.0 * kPi) / ((kLight * c->c_tilde) * dt);
  v.freq_step = c->freq_step;
  v.tdiag = (!c->gray && c->freq_step) ? 0 : 1;
  v.gem_max = c->gem_max;
  v.rcdt = 1.0 / v.cdt;
  v.acc = c->acc;
  v.status = c->status;
  v.f_H = c->f_H;
  v.f_dnu = c->f_dnu;
  v.f_G = c->f_G;
  v.f_R = c->f_R;
  v.f_nbc = c->f_nbc;
  v.f_half = c->f_half;
  v.geometry = c->geometry;
  v.vac = c->vac;
  v.spec = c->spec_on ? c->spec : nullptr;
  v.spec_unit = (4.0 * kPi) / kLight;
  v.nf = c->geometry == 1 ? (c->nx + c->ny) : 2 * (c->nx + c->ny);
  // table mode, with bit 4 for the transport's active-bin pruning variant and
  // bit 8 for its variant that leaves step 2 to the acceptance rule's kernel
  v.pt = c->pt | (c->prune > 0.0 ? 4 : 0) | (c->accept ? 8 : 0);
  v.ct = c->c_tilde;
  v.dt = dt;
  v.Hc = c->Hc;
  v.Gc = c->Gc;
  v.Kb = c->Kb;
  v.active = c->prune > 0.0 ? c->active : nullptr;
  v.gmaxc = c->gmaxc;
  v.Kcc = c->Kcc;
  v.hkTc = c->hkTc;
  v.t_2nu = c->t_2nu;
  v.f_2nu = c->f_2nu;
  v.gphi = c->gphi;
  v.g_AR = c->g_AR;
  v.g_AZ = c->g_AZ;
  v.g_Vol = c->g_Vol;
  v.g_invR = c->g_invR;
  v.g_dlL = c->g_dlL;
  v.g_dlR = c->g_dlR;
  v.g_wv = c->g_wv;
  v.gf_r0 = c->gf_r0;
  v.gf_r1 = c->gf_r1;
  v.gf_hoop = c->gf_hoop;
  v.gf_dlL = c->gf_dlL;
  v.gf_dlR = c->gf_dlR;
  v.gf_wv = c->gf_wv;
  v.g_wR = c->g_wR;
  return v;
}

int reset_counters(lym1_ctx* c) {
  LYM1_TRYK(launch_energy(c->precision, c->A[0], c->t_dnu, c->nb, c->nc, c->partF,
                          c->geometry == 1 ? c->g_wv : nullptr, c->nx, c->stream));
  LYM1_TRYK(launch_finalize(c->partT, 0, c->partF, freq_blocks(c->nc), c->acc, 1, c->stream));
  return LYM1_OK;
}

// copy nb x nc doubles from a caller buffer into a state array of the context
int state_in(lym1_ctx* c, const double* src, void* dst) {
  const size_t plane = static_cast<size_t>(c->nc);
  if (c->selem == 8) {
    LYM1_TRY(cudaMemcpyAsync(dst, src, plane * c->nb * sizeof(double), cudaMemcpyDefault, c->stream));
    return LYM1_OK;
  }
  if (is_device_ptr(src)) {
    LYM1_TRYK(launch_convert_in(c->precision, src, dst, static_cast<long long>(plane) * c->nb, c->stream));
    return LYM1_OK;
  }
  for (int k = 0; k < c->nb; ++k) {
    LYM1_TRY(cudaMemcpyAsync(c->staging, src + k * plane, plane * sizeof(double), cudaMemcpyDefault,
                             c->stream));
    LYM1_TRYK(launch_convert_in(c->precision, c->staging,
                                static_cast<char*>(dst) + k * plane * c->selem,
                                static_cast<long long>(plane), c->stream));
  }
  return LYM1_OK;
}

// copy a state array out as FP64 (times scale) into a caller buffer
int state_out(lym1_ctx* c, const void* src, double* dst, double scale) {
  const size_t plane = static_cast<size_t>(c->nc);
  if (is_device_ptr(dst)) {
    LYM1_TRYK(launch_convert_out(c->precision, src, dst, static_cast<long long>(plane) * c->nb, scale,
                                 c->stream));
    return LYM1_OK;
  }
  for (int k = 0; k < c->nb; ++k) {
    LYM1_TRYK(launch_convert_out(c->precision, static_cast<const char*>(src) + k * plane * c->selem,
                                 c->staging, static_cast<long long>(plane), scale, c->stream));
    LYM1_TRY(cudaMemcpyAsync(dst + k * plane, c->staging, plane * sizeof(double), cudaMemcpyDefault,
                             c->stream));
  }
  return LYM1_OK;
}

// brackets one kernel launch with profiling events when enabled
struct KernelTimer {
  lym1_ctx* c;
  int kind;
  cudaEvent_t stop = nullptr;
  KernelTimer(lym1_ctx* ctx, int k) : c(ctx), kind(k) {
    if (!c->profiling) return;
    cudaEvent_t a, b;
    if (cudaEventCreate(&a) != cudaSuccess) return;
    if (cudaEventCreate(&b) != cudaSuccess) {
      cudaEventDestroy(a);
      return;
    }
    cudaEventRecord(a, c->stream);
    c->ev_start.push_back(a);
    c->ev_stop.push_back(b);
    c->ev_kind.push_back(kind);
    stop = b;
  }
  ~KernelTimer() {
    if (stop) cudaEventRecord(stop, c->stream);
  }
};

// active-bin pruning: the flags of this substep from the current state,
// enqueued before its transport
int prune_launch(lym1_ctx* c, cudaStream_t s) {
  if (!(c->prune > 0.0)) return LYM1_OK;
  LYM1_TRYK(launch_active_bins(static_cast<int>(c->selem), c->A[0], c->nb, c->nc, c->nx,
                               c->geometry == 1 ? c->g_wv : nullptr, c->t_dnu, c->prune, c->Ebin,
                               c->active, s));
  return LYM1_OK;
}

int one_substep(lym1_ctx* c, double dt) {
  {
    const int rc = prune_launch(c, c->stream);
    if (rc != LYM1_OK) return rc;
  }
  const DeviceView v = make_view(c, dt);
  {
    KernelTimer t(c, 0);
    if (c->precision == LYM1_FP64_DET)
      LYM1_TRYK(launch_transport_det(v, c->stream));
    else
      LYM1_TRYK(launch_transport_fast(c->precision, v, c->stream));
  }
  const bool freq = !c->gray && c->freq_step;
  DeviceView w = v;  // the frequency step and the acceptance rule read B
  w.J = c->B[0];
  w.Hx = c->B[1];
  w.Hy = c->B[2];
  w.Jo = c->A[0];
  w.Hxo = c->A[1];
  w.Hyo = c->A[2];
  if (c->accept) {  // step 2 subcycled per cell, in place on B
    KernelTimer t(c, 1);
    if (c->precision == LYM1_FP64_DET)
      LYM1_TRYK(launch_subcycle_det(w, c->stream));
    else
      LYM1_TRYK(launch_subcycle_fast(c->precision, w, c->stream));
  }
  const int fmode = c->accept ? 2 : 0;
  if (freq) {
    {
      KernelTimer t(c, 1);
      if (c->precision == LYM1_FP64_DET)
        LYM1_TRYK(launch_freq_det(w, c->stream));
      else
        LYM1_TRYK(launch_freq_fast(c->precision, w, c->stream));
    }
    KernelTimer t(c, 2);
    LYM1_TRYK(launch_finalize(c->partT, transport_blocks(c->nx, c->ny), c->partF,
                              freq_blocks(c->nc), c->acc, fmode, c->stream));
  } else {
    for (int i = 0; i < 3; ++i) std::swap(c->A[i], c->B[i]);
    KernelTimer t(c, 2);
    // without a frequency step the energy comes from the transport, or from
    // the acceptance rule's kernel when it ran
    if (c->accept)
      LYM1_TRYK(launch_finalize(c->partT, transport_blocks(c->nx, c->ny), c->partF,
                                freq_blocks(c->nc), c->acc, fmode, c->stream));
    else
      LYM1_TRYK(launch_finalize(c->partT, transport_blocks(c->nx, c->ny), c->partT,
                                transport_blocks(c->nx, c->ny), c->acc, 0, c->stream));
  }
  c->substeps_done += 1;
  return LYM1_OK;
}

// Validates and uploads the per-[band][cell] inputs of a band context (host or
// device pointers, FP64): flux opacity and absorption opacity into Hc and Kb,
// emissivity into Gc (FP32 policies: over its per-cell maximum, kept in gmaxc,
// so that the kernels' jsc = lum gmax with lum = 1 restores it).  Nothing is
// changed unless every value is finite and >= 0.
int bands_upload(lym1_ctx* c, const double* aF, const double* kap, const double* j) {
  if (!aF || !kap || !j) return LYM1_EINVAL;
  const size_t plane = static_cast<size_t>(c->nc), n = plane * c->nb;
  std::vector<double> ha(n), hk(n), hj(n);
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) return LYM1_ECUDA;
  if (cudaMemcpy(ha.data(), aF, n * sizeof(double), cudaMemcpyDefault) != cudaSuccess ||
      cudaMemcpy(hk.data(), kap, n * sizeof(double), cudaMemcpyDefault) != cudaSuccess ||
      cudaMemcpy(hj.data(), j, n * sizeof(double), cudaMemcpyDefault) != cudaSuccess) {
    cudaGetLastError();
    return LYM1_EINVAL;
  }
  for (size_t q = 0; q < n; ++q)
    if (!(ha[q] >= 0.0) || !(hk[q] >= 0.0) || !(hj[q] >= 0.0) || !std::isfinite(ha[q]) ||
        !std::isfinite(hk[q]) || !std::isfinite(hj[q]))
      return LYM1_EINVAL;
  // total emitted power over the cells (ring volumes pi (2i + 1) dx^3 of the
  // half-space Z > 0 on the axisymmetric grid), the M_F normaliser
  const double V = (c->dx * c->dx) * c->dx;
  double L = 0.0;
  for (size_t q = 0; q < n; ++q) {
    const double Vc = c->geometry == 1 ? kPi * (2.0 * static_cast<double>((q % plane) % c->nx) + 1.0) * V : V;
    L += (4.0 * kPi) * hj[q] * Vc;
  }
  if (c->selem == 8) {
    LYM1_TRY(cudaMemcpy(c->Hc, ha.data(), n * sizeof(double), cudaMemcpyHostToDevice));
    LYM1_TRY(cudaMemcpy(c->Kb, hk.data(), n * sizeof(double), cudaMemcpyHostToDevice));
    LYM1_TRY(cudaMemcpy(c->Gc, hj.data(), n * sizeof(double), cudaMemcpyHostToDevice));
  } else {
    std::vector<double> gmax(plane, 0.0);
    for (size_t q = 0; q < n; ++q) gmax[q % plane] = std::max(gmax[q % plane], hj[q]);
    for (double& g : gmax)
      if (!(g > 0.0)) g = 1.0;
    std::vector<float> fa(n), fk(n), fj(n);
    for (size_t q = 0; q < n; ++q) {
      fa[q] = static_cast<float>(ha[q]);
      fk[q] = static_cast<float>(hk[q]);
      fj[q] = static_cast<float>(hj[q] / gmax[q % plane]);
    }
    LYM1_TRY(cudaMemcpy(c->Hc, fa.data(), n * sizeof(float), cudaMemcpyHostToDevice));
    LYM1_TRY(cudaMemcpy(c->Kb, fk.data(), n * sizeof(float), cudaMemcpyHostToDevice));
    LYM1_TRY(cudaMemcpy(c->Gc, fj.data(), n * sizeof(float), cudaMemcpyHostToDevice));
    LYM1_TRY(cudaMemcpy(c->gmaxc, gmax.data(), plane * sizeof(double), cudaMemcpyHostToDevice));
  }
  c->L_tot = L;
  return LYM1_OK;
}

// Device bytes of a context's creation-time allocations, by the same list and
// the same rounding (an empty allocation takes 16 bytes) as create_impl:
// mode 0 uniform temperature, 1 temperature field, 2 broad bands.  Buffers
// made on demand later (spectrum, pruning, the persistent batch) are not in it.
double plan_context_bytes(long long nx, long long ny, long long nb, size_t selem, int mode,
                          int geometry) {
  auto a = [](double b) { return b > 0.0 ? b : 16.0; };
  const double plane = static_cast<double>(nx) * static_cast<double>(ny);
  const double nstate = plane * static_cast<double>(nb), ncol = static_cast<double>(nx);
  const double tb = static_cast<double>(transport_blocks(static_cast<int>(nx), static_cast<int>(ny)));
  const double fb = static_cast<double>(freq_blocks(static_cast<long long>(plane)));
  double t = 6.0 * a(nstate * selem) + 12.0 * a(plane * 8) + 7.0 * a(nb * 8.0);
  t += a(tb * kDiagSlots * 8) + a(fb * kDiagSlots * 8) + a(16 * 8) + a(2.0 * kForceBlocks * 8);
  t += a(4 * sizeof(int)) + a(2 * sizeof(unsigned long long)) + a(kSumWork * 8) + 6.0 * a(nb * 4.0);
  if (mode == 2) t += 3.0 * a(nstate * selem) + 2.0 * a(plane * 8);
  if (mode == 1) t += 2.0 * a(nstate * selem) + 6.0 * a(plane * 8) + a(nb * 8.0) + a(nb * 4.0);
  if (geometry == 1)
    t += a(plane * 8) + 3.0 * a((ncol + 1) * 8) + 5.0 * a(ncol * 8) + 2.0 * a((ncol + 1) * 4) +
         4.0 * a(ncol * 4);
  return t;
}

void drop_events(lym1_ctx* c) {
  for (cudaEvent_t e : c->ev_start) cudaEventDestroy(e);
  for (cudaEvent_t e : c->ev_stop) cudaEventDestroy(e);
  c->ev_start.clear();
  c->ev_stop.clear();
  c->ev_kind.clear();
}

}  // namespace

// One work layout of a batch's transport launch: the tile shape (TileShape)
// and the number of blocks the bins of each tile are split over, with its
// work items, the views that carry it and the finalize jobs.
struct BatchLayout {
  int shape = 0, groups = 1, nT = 0;
  void* itemsT = nullptr;
  DeviceView *viewsT = nullptr, *viewsF = nullptr;
  FinalizeJob* jobs = nullptr;
  int rT = 1;  // transport blocks resident per SM
};

struct lym1_batch {
  std::vector<lym1_ctx*> ctxs;
  int precision = 0, nb = 0, nF = 0, geometry = 0, pt = 0;
  int tpt = 0;  // the transport's mode: pt, with bit 4 if a context prunes, 8 under the acceptance rule
  int accept = 0;  // the contexts subcycle step 2 (acceptance rule)
  int gridS = 0;   // persistent grid of the acceptance rule's kernel
  int nsm = 1, dev = 0;
  cudaStream_t ctx_stream = nullptr, bs = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr, t0 = nullptr, t1 = nullptr;
  void* itemsF = nullptr;
  std::vector<BatchLayout> layouts;
  // batch-owned scratch of each context for split tiles: per-block partials
  // and per-group force sums (DeviceView::fpg), sized for scratch_groups
  std::vector<double*> partS, fpg;
  int scratch_groups = 0;
  std::vector<unsigned> gens;  // view_gen of each context at the last upload
  std::vector<unsigned> prune_gens;  // prune_gen of each context at creation
  std::vector<unsigned> accept_gens;  // accept_gen of each context at creation
  int gridF = 0;
  // tuning: candidate (layout, persistent transport grid) pairs, each timed
  // on one substep; cur is the one in use
  std::vector<std::pair<int, int>> cands;
  std::vector<float> ctime;
  int cur = 0;
  int tuned = 0;
  // class of this batch in the process-wide cache of tuned choices: device,
  // precision, geometry, transport mode, bins, log2 of the tile count
  std::vector<long long> tune_key;
  cudaGraphExec_t exec = nullptr;
  cudaGraph_t graph = nullptr;
};

namespace {

// Tuned persistent grids shared by every batch of the same class, so that a
// new batch (a new mix of clouds in the serving loop) skips the timed tuning
// substeps when a batch of its class was tuned before on this device.
std::mutex g_tune_mutex;
std::map<std::vector<long long>, std::vector<int>> g_tune_cache;  // {shape, groups, grid}

std::vector<int> tuned_lookup(const std::vector<long long>& key) {
  std::lock_guard<std::mutex> lock(g_tune_mutex);
  const auto it = g_tune_cache.find(key);
  return it == g_tune_cache.end() ? std::vector<int>() : it->second;
}

void tuned_store(const std::vector<long long>& key, const std::vector<int>& choice) {
  std::lock_guard<std::mutex> lock(g_tune_mutex);
  g_tune_cache[key] = choice;
}

// the two views of context i in a batch under a layout: the transport step
// reads A and writes B, the frequency step reads B and writes A; a layout
// other than one 16 x 16 block per tile keeps its partials in the batch's
// scratch and, with split tiles, its per-group force sums
void batch_views(const lym1_batch* b, size_t i, const BatchLayout& L, DeviceView* vT,
                 DeviceView* vF) {
  const lym1_ctx* c = b->ctxs[i];
  *vT = make_view(c, c->dt_cfl);
  if (L.shape != 0 || L.groups > 1) vT->partT = b->partS[i];
  if (L.groups > 1) {
    vT->ngrp = L.groups;
    vT->fpg = b->fpg[i];
  }
  *vF = *vT;
  vF->J = c->B[0];
  vF->Hx = c->B[1];
  vF->Hy = c->B[2];
  vF->Jo = c->A[0];
  vF->Hxo = c->A[1];
  vF->Hyo = c->A[2];
}

// uploads the views and finalize jobs of every context under one layout
int upload_layout(const lym1_batch* b, const BatchLayout& L, cudaStream_t s) {
  const size_t n = b->ctxs.size();
  std::vector<DeviceView> vT(n), vF(n);
  std::vector<FinalizeJob> jobs(n);
  for (size_t i = 0; i < n; ++i) {
    const lym1_ctx* c = b->ctxs[i];
    batch_views(b, i, L, &vT[i], &vF[i]);
    jobs[i] = {vT[i].partT, c->partF, c->acc,
               transport_blocks(c->nx, c->ny, L.shape) * L.groups, freq_blocks(c->nc),
               c->accept ? 2 : 0};
  }
  LYM1_TRY(cudaMemcpyAsync(L.viewsT, vT.data(), sizeof(DeviceView) * n, cudaMemcpyHostToDevice, s));
  LYM1_TRY(cudaMemcpyAsync(L.viewsF, vF.data(), sizeof(DeviceView) * n, cudaMemcpyHostToDevice, s));
  LYM1_TRY(cudaMemcpyAsync(L.jobs, jobs.data(), sizeof(FinalizeJob) * n, cudaMemcpyHostToDevice, s));
  LYM1_TRY(cudaStreamSynchronize(s));
  return LYM1_OK;
}

// re-upload, stream-ordered before the next launch, the views of contexts
// whose c_tilde changed since the last upload (the kernels and the captured
// graph read the views from device memory)
int refresh_views(lym1_batch* b, cudaStream_t s) {
  for (size_t i = 0; i < b->ctxs.size(); ++i) {
    const lym1_ctx* c = b->ctxs[i];
    if (c->view_gen == b->gens[i]) continue;
    for (const BatchLayout& L : b->layouts) {
      DeviceView v[2];
      batch_views(b, i, L, &v[0], &v[1]);
      LYM1_TRY(cudaMemcpyAsync(L.viewsT + i, &v[0], sizeof(DeviceView), cudaMemcpyHostToDevice, s));
      LYM1_TRY(cudaMemcpyAsync(L.viewsF + i, &v[1], sizeof(DeviceView), cudaMemcpyHostToDevice, s));
    }
    LYM1_TRY(cudaStreamSynchronize(s));
    b->gens[i] = c->view_gen;
  }
  return LYM1_OK;
}

// one launch of a batch kernel (kind 0 transport, 1 frequency step, 2 the
// acceptance rule's step 2) under the layout and grid in use
int batch_kernel(lym1_batch* b, int kind, cudaStream_t s) {
  const BatchLayout& L = b->layouts[b->cands[b->cur].first];
  const int gridT = b->cands[b->cur].second;
  const bool tr = kind == 0;
  const int pt = tr ? b->tpt : b->pt;
  const DeviceView* views = tr ? L.viewsT : L.viewsF;
  const void* items = tr ? L.itemsT : b->itemsF;
  const int n = tr ? L.nT : b->nF;
  const int grid = tr ? gridT : (kind == 2 ? b->gridS : b->gridF);
  if (b->precision == LYM1_FP64_DET)
    return launch_batched_det(kind, b->geometry, pt, views, items, n, grid, b->nb, s, L.shape);
  return launch_batched_fast(b->precision, kind, b->geometry, pt, views, items, n, grid, b->nb, s,
                             L.shape);
}

int batch_launch(lym1_batch* b, cudaStream_t s) {
  const int n = static_cast<int>(b->ctxs.size());
  for (lym1_ctx* c : b->ctxs) {
    const int rc = prune_launch(c, s);
    if (rc != LYM1_OK) return rc;
  }
  LYM1_TRYK(batch_kernel(b, 0, s));
  if (b->accept) LYM1_TRYK(batch_kernel(b, 2, s));
  LYM1_TRYK(batch_kernel(b, 1, s));
  LYM1_TRYK(launch_finalize_batched(b->layouts[b->cands[b->cur].first].jobs, n, s));
  return LYM1_OK;
}

// the persistent launches of one substep on the context's stream, each
// bracketed by profiling events (no graph)
int batch_launch_timed(lym1_batch* b, lym1_ctx* c) {
  const int n = static_cast<int>(b->ctxs.size());
  for (lym1_ctx* x : b->ctxs) {
    const int rc = prune_launch(x, c->stream);
    if (rc != LYM1_OK) return rc;
  }
  {
    KernelTimer t(c, 0);
    LYM1_TRYK(batch_kernel(b, 0, c->stream));
  }
  {
    KernelTimer t(c, 1);  // with the acceptance rule, its kernel counts here
    if (b->accept) LYM1_TRYK(batch_kernel(b, 2, c->stream));
    LYM1_TRYK(batch_kernel(b, 1, c->stream));
  }
  KernelTimer t(c, 2);
  LYM1_TRYK(launch_finalize_batched(b->layouts[b->cands[b->cur].first].jobs, n, c->stream));
  return LYM1_OK;
}

// reports an expired bounded wait once, then clears the status words
int device_status(lym1_ctx* c) {
  int st[2] = {0, 0};
  LYM1_TRY(cudaMemcpy(st, c->status, sizeof st, cudaMemcpyDeviceToHost));
  if (st[0] == 0 && st[1] == 0) return LYM1_OK;
  LYM1_TRY(cudaMemset(c->status, 0, 2 * sizeof(int)));
  return st[0] != 0 ? LYM1_ETIMEOUT : LYM1_OK;
}

void batch_free(lym1_batch* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  for (BatchLayout& L : b->layouts) {
    void* ptrs[] = {L.itemsT, L.viewsT, L.viewsF, L.jobs};
    for (void* p : ptrs)
      if (p) cudaFree(p);
  }
  for (double* p : b->partS)
    if (p) cudaFree(p);
  for (double* p : b->fpg)
    if (p) cudaFree(p);
  if (b->itemsF) cudaFree(b->itemsF);
  cudaEvent_t evs[] = {b->ev_in, b->ev_out, b->t0, b->t1};
  for (cudaEvent_t e : evs)
    if (e) cudaEventDestroy(e);
  if (b->bs) cudaStreamDestroy(b->bs);
}

// The batch's scratch for split tiles and other shapes, sized for up to
// `groups` bin groups (grown, never shrunk; outside any capture).
int ensure_scratch(lym1_batch* b, int groups) {
  if (groups <= b->scratch_groups) return LYM1_OK;
  for (size_t i = 0; i < b->ctxs.size(); ++i) {
    const lym1_ctx* c = b->ctxs[i];
    const int tiles = std::max(transport_blocks(c->nx, c->ny, 0), transport_blocks(c->nx, c->ny, 1));
    double* ps = nullptr;
    double* fg = nullptr;
    if (cudaMalloc(reinterpret_cast<void**>(&ps), sizeof(double) * kDiagSlots * tiles * groups) !=
        cudaSuccess) {
      cudaGetLastError();
      return LYM1_ENOMEM;
    }
    if (groups > 1 &&
        cudaMalloc(reinterpret_cast<void**>(&fg), sizeof(double) * 2 * groups * c->nc) != cudaSuccess) {
      cudaGetLastError();
      cudaFree(ps);
      return LYM1_ENOMEM;
    }
    if (b->partS[i]) cudaFree(b->partS[i]);
    if (b->fpg[i]) cudaFree(b->fpg[i]);
    b->partS[i] = ps;
    b->fpg[i] = fg;
  }
  b->scratch_groups = groups;
  return LYM1_OK;
}

// Index of the layout (shape, groups), made (items, views, jobs) if new.
// Every layout's views are re-uploaded, since the scratch may have moved.
int ensure_layout(lym1_batch* b, int shape, int groups, int* index) {
  for (size_t j = 0; j < b->layouts.size(); ++j)
    if (b->layouts[j].shape == shape && b->layouts[j].groups == groups) {
      *index = static_cast<int>(j);
      return LYM1_OK;
    }
  {
    const int rc = ensure_scratch(b, groups);
    if (rc != LYM1_OK) return rc;
  }
  BatchLayout L;
  L.shape = shape;
  L.groups = groups;
  std::vector<BatchItemHost> it;
  const int tx = tile_x(shape), ty = tile_y(shape);
  for (size_t i = 0; i < b->ctxs.size(); ++i) {
    const lym1_ctx* c = b->ctxs[i];
    const int gx = (c->nx + tx - 1) / tx, gy = (c->ny + ty - 1) / ty, tiles = gx * gy;
    for (int g = 0; g < groups; ++g) {
      const int k0 = static_cast<int>(static_cast<long long>(c->nb) * g / groups);
      const int k1 = static_cast<int>(static_cast<long long>(c->nb) * (g + 1) / groups);
      for (int by = 0; by < gy; ++by)
        for (int bx = 0; bx < gx; ++bx)
          it.push_back({static_cast<int>(i), bx * tx, by * ty, g * tiles + by * gx + bx, k0, k1, g});
    }
  }
  L.nT = static_cast<int>(it.size());
  const size_t n = b->ctxs.size();
  if (cudaMalloc(&L.itemsT, sizeof(BatchItemHost) * it.size()) != cudaSuccess ||
      cudaMalloc(reinterpret_cast<void**>(&L.viewsT), sizeof(DeviceView) * n) != cudaSuccess ||
      cudaMalloc(reinterpret_cast<void**>(&L.viewsF), sizeof(DeviceView) * n) != cudaSuccess ||
      cudaMalloc(reinterpret_cast<void**>(&L.jobs), sizeof(FinalizeJob) * n) != cudaSuccess) {
    cudaGetLastError();
    void* ptrs[] = {L.itemsT, L.viewsT, L.viewsF, L.jobs};
    for (void* p : ptrs)
      if (p) cudaFree(p);
    return LYM1_ENOMEM;
  }
  LYM1_TRY(cudaMemcpy(L.itemsT, it.data(), sizeof(BatchItemHost) * it.size(), cudaMemcpyHostToDevice));
  L.rT = b->precision == LYM1_FP64_DET
             ? resident_blocks_det(0, b->geometry, b->tpt, b->nb, shape)
             : resident_blocks_fast(b->precision, 0, b->geometry, b->tpt, b->nb, shape);
  b->layouts.push_back(L);
  for (const BatchLayout& M : b->layouts) {
    const int rc = upload_layout(b, M, b->bs);
    if (rc != LYM1_OK) return rc;
  }
  *index = static_cast<int>(b->layouts.size()) - 1;
  return LYM1_OK;
}

}  // namespace

extern "C" {

const char* lym1_strerror(int s) {
  switch (s) {
    case LYM1_OK: return "ok";
    case LYM1_EINVAL: return "invalid argument";
    case LYM1_ENOMEM: return "device memory allocation failed";
    case LYM1_ECUDA: return "CUDA runtime or kernel error";
    case LYM1_ENONFINITE: return "non-finite value in the diagnostics";
    case LYM1_ETIMEOUT: return "bounded device wait expired";
    case LYM1_ENOTCONVERGED: return "substep cap reached before steady state";
    case LYM1_ENODEVICE: return "no usable CUDA device";
    case LYM1_ERANGE: return "size beyond the fixed maximum of an allocation-free call";
    default: return "unknown status";
  }
}

static int create_impl(const lym1_grid* grid, const lym1_groups* groups, const lym1_opacities* op,
                       const lym1_bands* bands, lym1_ctx** out) {
  if (!out) return LYM1_EINVAL;
  *out = nullptr;
  if (!grid || !groups || !op) return LYM1_EINVAL;
  if (grid->nx < 1 || grid->ny < 1 || !(grid->dx_cm > 0.0)) return LYM1_EINVAL;
  if (grid->geometry != 0 && grid->geometry != 1) return LYM1_EINVAL;
  for (int i = 0; i < 4; ++i)
    if (grid->bc[i] != 0 && grid->bc[i] != 1) return LYM1_EINVAL;
  if (!(op->temp_K > 0.0) || op->precision < 0 || op->precision > 3) return LYM1_EINVAL;
  if (!op->n_hi || !op->rho_dust || !op->p_d || !op->ux || !op->uy) return LYM1_EINVAL;
  if (op->c_tilde < 0.0 || op->cfl < 0.0 || op->kappa_abs < 0.0 || op->kappa_F < 0.0) return LYM1_EINVAL;
  const long long nc = static_cast<long long>(grid->nx) * grid->ny;
  if (nc > (1LL << 31)) return LYM1_EINVAL;

  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) {
    cudaGetLastError();
    return LYM1_ENODEVICE;
  }

  std::vector<double> edges;
  if (groups->edges_dnu_hz) {
    if (groups->n_bins < 1 || groups->n_bins > LYM1_MAX_BINS) return LYM1_EINVAL;
    edges.assign(groups->edges_dnu_hz, groups->edges_dnu_hz + groups->n_bins + 1);
    for (int k = 0; k < groups->n_bins; ++k)
      if (!(edges[k + 1] > edges[k])) return LYM1_EINVAL;
  } else {
    const double q = groups->q > 0.0 ? groups->q : 1.1;
    const double Tm = groups->T_min > 0.0 ? groups->T_min : 30.0;
    if (!(q > 1.0)) return LYM1_EINVAL;
    const int n = paper_frequency_grid(Tm, q, &edges);
    if (n < 1 || n > LYM1_MAX_BINS) return LYM1_EINVAL;
  }

  lym1_ctx* c = new (std::nothrow) lym1_ctx();
  if (!c) return LYM1_ENOMEM;
  c->nx = grid->nx;
  c->ny = grid->ny;
  c->nc = nc;
  c->dx = grid->dx_cm;
  c->T = op->temp_K;
  c->c_tilde = op->c_tilde > 0.0 ? op->c_tilde : kLight;
  c->cfl = op->cfl > 0.0 ? op->cfl : 0.4;
  c->kabs = op->kappa_abs;
  c->kF = op->kappa_F;
  c->precision = op->precision;
  c->gray = groups->gray ? 1 : 0;
  c->recoil = op->recoil ? 1 : 0;
  c->freq_step = op->freq_step ? 1 : 0;
  c->stream = static_cast<cudaStream_t>(op->cuda_stream);
  c->selem = (c->precision >= LYM1_MIXED) ? 4 : 8;
  c->geometry = grid->geometry;
  for (int i = 0; i < 4; ++i)
    if (grid->bc[i] == 1 && !(c->geometry == 1 && (i == 0 || i == 2))) c->vac |= 1 << i;
  build_tables(edges, c->T, c->dx, c->gray, c->recoil, &c->tab, c->geometry);
  c->nb = c->tab.nb;
  c->gem_max = 0.0;
  for (double g : c->tab.gem) c->gem_max = std::max(c->gem_max, g);
  if (!(c->gem_max > 0.0)) c->gem_max = 1.0;

  int rc = LYM1_OK;
  const size_t plane = static_cast<size_t>(nc);
  const size_t nstate = plane * c->nb;
  for (int i = 0; i < 3 && rc == LYM1_OK; ++i) rc = dalloc(c, &c->A[i], nstate * c->selem);
  for (int i = 0; i < 3 && rc == LYM1_OK; ++i) rc = dalloc(c, &c->B[i], nstate * c->selem);
  double** cell_arrays[] = {&c->alpha, &c->rho, &c->pd, &c->ux, &c->uy, &c->gxx,
                            &c->gyy,   &c->gsh, &c->lum, &c->fx, &c->fy, &c->staging};
  for (double** p : cell_arrays)
    if (rc == LYM1_OK) rc = dalloc_t(c, p, plane);
  double** bin_arrays[] = {&c->t_dnu, &c->t_H, &c->t_gem, &c->t_half, &c->t_R, &c->t_nbc, &c->t_dH};
  for (double** p : bin_arrays)
    if (rc == LYM1_OK) rc = dalloc_t(c, p, static_cast<size_t>(c->nb));
  if (rc == LYM1_OK) rc = dalloc_t(c, &c->partT, static_cast<size_t>(transport_blocks(c->nx, c->ny)) * kDiagSlots);
  if (rc == LYM1_OK) rc = dalloc_t(c, &c->partF, static_cast<size_t>(freq_blocks(nc)) * kDiagSlots);
  if (rc == LYM1_OK) rc = dalloc_t(c, &c->acc, 16);
  if (rc == LYM1_OK) rc = dalloc_t(c, &c->fpart, 2 * kForceBlocks);
  if (rc == LYM1_OK) rc = dalloc_t(c, &c->status, 4);
  if (rc == LYM1_OK) rc = dalloc_t(c, &c->ctw, 2);
  if (rc == LYM1_OK) rc = dalloc_t(c, &c->lsum, kSumWork);
  float** ftabs[] = {&c->f_H, &c->f_dnu, &c->f_G, &c->f_R, &c->f_nbc, &c->f_half};
  for (float** p : ftabs)
    if (rc == LYM1_OK) rc = dalloc_t(c, p, static_cast<size_t>(c->nb));
  CellTables ct;
  if (bands) {
    // broad bands: per-[band][cell] tables in the state type; alpha = n_HI
    // sigma0c = 1 and rho_d = 0, so that the kernels' alpha_F = alpha Hc +
    // rho_d kappa_F is the band's own flux opacity
    c->pt = 2;
    c->bands = 1;
    if (rc == LYM1_OK) rc = dalloc(c, &c->Hc, nstate * c->selem);
    if (rc == LYM1_OK) rc = dalloc(c, &c->Gc, nstate * c->selem);
    if (rc == LYM1_OK) rc = dalloc(c, &c->Kb, nstate * c->selem);
    if (rc == LYM1_OK) rc = dalloc_t(c, &c->gmaxc, plane);
    if (rc == LYM1_OK) rc = dalloc_t(c, &c->sig0c, plane);
  } else if (op->temp_field) {
    // per-cell A0 on the host (the field may live on the device)
    std::vector<double> hT(plane);
    if (cudaMemcpy(hT.data(), op->temp_field, plane * sizeof(double), cudaMemcpyDefault) != cudaSuccess) {
      cudaGetLastError();
      rc = LYM1_EINVAL;
    }
    for (size_t i = 0; rc == LYM1_OK && i < plane; ++i)
      if (!(hT[i] > 0.0) || !std::isfinite(hT[i])) rc = LYM1_EINVAL;
    if (rc == LYM1_OK) {
      c->pt = 1;
      build_cell_tables(edges, hT.data(), nc, c->dx, c->gray, c->recoil, grid->geometry, &ct);
      if (rc == LYM1_OK) rc = dalloc(c, &c->Hc, nstate * c->selem);
      if (rc == LYM1_OK) rc = dalloc(c, &c->Gc, nstate * c->selem);
      double** pc[] = {&c->gmaxc, &c->Kcc, &c->hkTc, &c->sig0c, &c->Tc, &c->nhi};
      for (double** q : pc)
        if (rc == LYM1_OK) rc = dalloc_t(c, q, plane);
      if (rc == LYM1_OK) rc = dalloc_t(c, &c->t_2nu, static_cast<size_t>(c->nb));
      if (rc == LYM1_OK) rc = dalloc_t(c, &c->f_2nu, static_cast<size_t>(c->nb));
    }
  }
  CylTables cyl;
  const size_t ncol = static_cast<size_t>(c->nx);
  if (c->geometry == 1) {
    build_cyl_tables(c->nx, c->dx, &cyl);
    c->g_wR = cyl.wR;
    if (rc == LYM1_OK) rc = dalloc_t(c, &c->gphi, plane);
    double** cd[] = {&c->g_AR, &c->g_dlL, &c->g_dlR};
    for (double** p : cd)
      if (rc == LYM1_OK) rc = dalloc_t(c, p, ncol + 1);
    double** cc[] = {&c->g_AZ, &c->g_Vol, &c->g_invR, &c->g_wv, &c->g_V2pi};
    for (double** p : cc)
      if (rc == LYM1_OK) rc = dalloc_t(c, p, ncol);
    float** fd1[] = {&c->gf_dlL, &c->gf_dlR};
    for (float** p : fd1)
      if (rc == LYM1_OK) rc = dalloc_t(c, p, ncol + 1);
    float** fc[] = {&c->gf_r0, &c->gf_r1, &c->gf_hoop, &c->gf_wv};
    for (float** p : fc)
      if (rc == LYM1_OK) rc = dalloc_t(c, p, ncol);
  }
  if (rc != LYM1_OK) {
    free_all(c);
    delete c;
    return rc;
  }

  auto fail = [&](int r) {
    cudaStreamSynchronize(c->stream);
    cudaGetLastError();
    free_all(c);
    delete c;
    return r;
  };
  const cudaStream_t s = c->stream;
  const size_t pb = plane * sizeof(double);
  // per-cell inputs: n_HI and u go through the statics kernel via staging
  double* d_nhi = c->staging;
  if (cudaMemcpyAsync(d_nhi, op->n_hi, pb, cudaMemcpyDefault, s) != cudaSuccess ||
      cudaMemcpyAsync(c->ux, op->ux, pb, cudaMemcpyDefault, s) != cudaSuccess ||
      cudaMemcpyAsync(c->uy, op->uy, pb, cudaMemcpyDefault, s) != cudaSuccess ||
      cudaMemcpyAsync(c->rho, op->rho_dust, pb, cudaMemcpyDefault, s) != cudaSuccess ||
      cudaMemcpyAsync(c->pd, op->p_d, pb, cudaMemcpyDefault, s) != cudaSuccess)
    return fail(LYM1_ECUDA);
  if (c->pt == 2) {
    std::vector<double> ones(plane, 1.0);
    if (cudaMemcpy(c->sig0c, ones.data(), pb, cudaMemcpyHostToDevice) != cudaSuccess)
      return fail(LYM1_ECUDA);
  }
  if (c->pt == 1) {
    // per-[bin][cell] tables in the state type (FP32 policies: G / gmax)
    const size_t nsv = ct.H.size();
    if (c->selem == 8) {
      if (cudaMemcpy(c->Hc, ct.H.data(), nsv * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess ||
          cudaMemcpy(c->Gc, ct.G.data(), nsv * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess)
        return fail(LYM1_ECUDA);
    } else {
      std::vector<float> hf(nsv), gf(nsv);
      for (size_t q = 0; q < nsv; ++q) {
        hf[q] = static_cast<float>(ct.H[q]);
        gf[q] = static_cast<float>(ct.G[q] / ct.gmax[q % plane]);
      }
      if (cudaMemcpy(c->Hc, hf.data(), nsv * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess ||
          cudaMemcpy(c->Gc, gf.data(), nsv * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess)
        return fail(LYM1_ECUDA);
    }
    // the recoil factor R_k = h/(k_B T) - 2/nubar_k, zero without recoil
    std::vector<double> hk(ct.hkT), t2(c->nb, 0.0);
    std::vector<float> f2(c->nb, 0.0f);
    if (c->recoil && !c->gray)
      for (int k = 0; k < c->nb; ++k) {
        t2[k] = 2.0 / c->tab.nubar[k];
        f2[k] = static_cast<float>(t2[k]);
      }
    else
      std::fill(hk.begin(), hk.end(), 0.0);
    if (cudaMemcpy(c->gmaxc, ct.gmax.data(), pb, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(c->Kcc, ct.Kc.data(), pb, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(c->hkTc, hk.data(), pb, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(c->sig0c, ct.sigma0.data(), pb, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(c->Tc, op->temp_field, pb, cudaMemcpyDefault) != cudaSuccess ||
        cudaMemcpy(c->t_2nu, t2.data(), sizeof(double) * c->nb, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(c->f_2nu, f2.data(), sizeof(float) * c->nb, cudaMemcpyHostToDevice) != cudaSuccess)
      return fail(LYM1_ECUDA);
  }
  if (c->pt == 1) {
    c->edges = edges;
    if (cudaMemcpyAsync(c->nhi, d_nhi, pb, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
      return fail(LYM1_ECUDA);
  }
  if (launch_setup_statics(d_nhi, c->ux, c->uy, c->tab.lc.sigma0, c->pt ? c->sig0c : nullptr, c->nx,
                           c->ny, c->dx, c->alpha, c->gxx, c->gyy, c->gsh, c->geometry, c->gphi, s) != 0)
    return fail(LYM1_ECUDA);
  if (c->geometry == 1) {
    const std::pair<double*, const std::vector<double>*> dt[] = {
        {c->g_AR, &cyl.AR},     {c->g_dlL, &cyl.dlL}, {c->g_dlR, &cyl.dlR},   {c->g_AZ, &cyl.AZ},
        {c->g_Vol, &cyl.Vol},   {c->g_invR, &cyl.invR}, {c->g_wv, &cyl.wv}, {c->g_V2pi, &cyl.V2pi}};
    for (const auto& e : dt)
      if (cudaMemcpy(e.first, e.second->data(), sizeof(double) * e.second->size(),
                     cudaMemcpyHostToDevice) != cudaSuccess)
        return fail(LYM1_ECUDA);
    const std::pair<float*, const std::vector<float>*> ft[] = {
        {c->gf_dlL, &cyl.fdlL}, {c->gf_dlR, &cyl.fdlR}, {c->gf_r0, &cyl.r0},
        {c->gf_r1, &cyl.r1},    {c->gf_hoop, &cyl.hoop}, {c->gf_wv, &cyl.fwv}};
    for (const auto& e : ft)
      if (cudaMemcpy(e.first, e.second->data(), sizeof(float) * e.second->size(),
                     cudaMemcpyHostToDevice) != cudaSuccess)
        return fail(LYM1_ECUDA);
  }
  const std::vector<double>* tabs[] = {&c->tab.dnu, &c->tab.Havg, &c->tab.gem,
                                       &c->tab.half, &c->tab.Rk, &c->tab.nubar_c};
  double* dtabs[] = {c->t_dnu, c->t_H, c->t_gem, c->t_half, c->t_R, c->t_nbc};
  for (int i = 0; i < 6; ++i)
    if (cudaMemcpyAsync(dtabs[i], tabs[i]->data(), sizeof(double) * c->nb, cudaMemcpyHostToDevice, s) !=
        cudaSuccess)
      return fail(LYM1_ECUDA);
  {  // dnu_k <H>_k (the destruction part of the mixed step's absorbed energy)
    std::vector<double> dH(c->nb);
    for (int k = 0; k < c->nb; ++k) dH[k] = c->tab.dnu[k] * c->tab.Havg[k];
    if (cudaMemcpy(c->t_dH, dH.data(), sizeof(double) * c->nb, cudaMemcpyHostToDevice) != cudaSuccess)
      return fail(LYM1_ECUDA);
  }
  // FP32 table copies (the emissivity factor scaled by its maximum)
  std::vector<float> fh[6];
  for (int k = 0; k < c->nb; ++k) {
    fh[0].push_back(static_cast<float>(c->tab.Havg[k]));
    fh[1].push_back(static_cast<float>(c->tab.dnu[k]));
    fh[2].push_back(static_cast<float>(c->tab.gem[k] / c->gem_max));
    fh[3].push_back(static_cast<float>(c->tab.Rk[k]));
    fh[4].push_back(static_cast<float>(c->tab.nubar_c[k]));
    fh[5].push_back(static_cast<float>(c->tab.half[k]));
  }
  float* fd[] = {c->f_H, c->f_dnu, c->f_G, c->f_R, c->f_nbc, c->f_half};
  for (int i = 0; i < 6; ++i)
    if (cudaMemcpy(fd[i], fh[i].data(), sizeof(float) * c->nb, cudaMemcpyHostToDevice) != cudaSuccess)
      return fail(LYM1_ECUDA);
  for (int i = 0; i < 3; ++i)
    if (cudaMemsetAsync(c->A[i], 0, nstate * c->selem, s) != cudaSuccess) return fail(LYM1_ECUDA);
  if (cudaMemsetAsync(c->lum, 0, pb, s) != cudaSuccess || cudaMemsetAsync(c->fx, 0, pb, s) != cudaSuccess ||
      cudaMemsetAsync(c->fy, 0, pb, s) != cudaSuccess || cudaMemsetAsync(c->acc, 0, 16 * sizeof(double), s) != cudaSuccess ||
      cudaMemsetAsync(c->status, 0, 4 * sizeof(int), s) != cudaSuccess ||
      cudaMemsetAsync(c->lsum, 0, kSumWork * sizeof(double), s) != cudaSuccess)
    return fail(LYM1_ECUDA);
  // max |u| for the RT time step (Sec. 2.1, CFL condition with D = 2)
  std::vector<double> hux(plane), huy(plane);
  if (cudaMemcpyAsync(hux.data(), op->ux, pb, cudaMemcpyDefault, s) != cudaSuccess ||
      cudaMemcpyAsync(huy.data(), op->uy, pb, cudaMemcpyDefault, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return fail(LYM1_ECUDA);
  double umax = 0.0;
  for (size_t i = 0; i < plane; ++i) {
    const double um = std::sqrt(hux[i] * hux[i] + huy[i] * huy[i]);
    if (um > umax) umax = um;
  }
  c->umax = umax;
  c->dt_cfl = (c->cfl / 2.0) * (c->dx / (c->c_tilde + umax));
  const double V = (c->dx * c->dx) * c->dx;
  const double eunit = ((4.0 * kPi) / kLight) * V;
  if (cudaMemcpyAsync(c->acc + 13, &eunit, sizeof(double), cudaMemcpyHostToDevice, s) != cudaSuccess)
    return fail(LYM1_ECUDA);
  if (reset_counters(c) != LYM1_OK || cudaStreamSynchronize(s) != cudaSuccess) return fail(LYM1_ECUDA);
  if (bands) {
    // lum = 1 per cell: the kernels' j = lum Gc is then the band emissivity
    std::vector<double> ones(plane, 1.0);
    if (cudaMemcpy(c->lum, ones.data(), pb, cudaMemcpyHostToDevice) != cudaSuccess)
      return fail(LYM1_ECUDA);
    const int rb = bands_upload(c, bands->alpha_F, bands->kappa, bands->emissivity);
    if (rb != LYM1_OK) return fail(rb);
  }
  *out = c;
  return LYM1_OK;
}

int lym1_create(const lym1_grid* grid, const lym1_groups* groups, const lym1_opacities* op,
                lym1_ctx** out) {
  return create_impl(grid, groups, op, nullptr, out);
}

int lym1_create_bands(const lym1_grid* grid, const lym1_bands* bands, const double* ux,
                      const double* uy, double c_tilde, double cfl, int precision,
                      void* cuda_stream, lym1_ctx** out) {
  if (!out) return LYM1_EINVAL;
  *out = nullptr;
  if (!grid || !bands || !ux || !uy || !bands->alpha_F || !bands->kappa || !bands->emissivity)
    return LYM1_EINVAL;
  if (bands->n_bands < 1 || bands->n_bands > LYM1_MAX_BINS) return LYM1_EINVAL;
  if (grid->nx < 1 || grid->ny < 1) return LYM1_EINVAL;
  const long long nc = static_cast<long long>(grid->nx) * grid->ny;
  if (nc > (1LL << 31)) return LYM1_EINVAL;
  const size_t plane = static_cast<size_t>(nc);
  std::vector<double> ones(plane, 1.0), zeros(plane, 0.0), edges(bands->n_bands + 1);
  for (int k = 0; k <= bands->n_bands; ++k) edges[k] = static_cast<double>(k);
  lym1_groups g;
  std::memset(&g, 0, sizeof g);
  g.n_bins = bands->n_bands;
  g.edges_dnu_hz = edges.data();
  lym1_opacities o;
  std::memset(&o, 0, sizeof o);
  o.n_hi = ones.data();
  o.rho_dust = zeros.data();
  o.p_d = zeros.data();
  o.ux = ux;
  o.uy = uy;
  o.temp_K = 1.0e4;
  o.c_tilde = c_tilde;
  o.cfl = cfl;
  o.precision = precision;
  o.cuda_stream = cuda_stream;
  return create_impl(grid, &g, &o, bands, out);
}

int lym1_bands_update(lym1_ctx* c, const double* alpha_F, const double* kappa,
                      const double* emissivity) {
  if (!c || !c->bands) return LYM1_EINVAL;
  return bands_upload(c, alpha_F, kappa, emissivity);
}

void lym1_destroy(lym1_ctx* c) {
  if (!c) return;
  cudaStreamSynchronize(c->stream);
  if (c->self_batch) lym1_batch_destroy(c->self_batch);
  c->self_batch = nullptr;
  drop_events(c);
  free_all(c);
  delete c;
}

int lym1_set_sources(lym1_ctx* c, const double* lum) {
  if (!c || !lum || c->bands) return LYM1_EINVAL;
  const size_t n = static_cast<size_t>(c->nc);
  LYM1_TRY(cudaMemcpyAsync(c->lum, lum, n * sizeof(double), cudaMemcpyDefault, c->stream));
  // the total luminosity (M_F normaliser), summed on the device and read back
  // only by the diagnostics: the call does not wait for the GPU
  LYM1_TRYK(launch_sum_cells(c->lum, c->nc, c->lsum, c->stream));
  c->L_pending = 1;
  // axisymmetric grid: the kernels take the luminosity per unit ring volume
  if (c->geometry == 1)
    LYM1_TRYK(launch_scale_columns(c->lum, c->g_V2pi, c->nx, c->nc, c->stream));
  return LYM1_OK;
}

int lym1_set_state(lym1_ctx* c, const double* J, const double* Hx, const double* Hy) {
  if (!c || !J || !Hx || !Hy) return LYM1_EINVAL;
  int rc = state_in(c, J, c->A[0]);
  if (rc == LYM1_OK) rc = state_in(c, Hx, c->A[1]);
  if (rc == LYM1_OK) rc = state_in(c, Hy, c->A[2]);
  if (rc != LYM1_OK) return rc;
  return reset_counters(c);
}

int lym1_get_state(lym1_ctx* c, double* J, double* Hx, double* Hy) {
  if (!c || !J || !Hx || !Hy) return LYM1_EINVAL;
  int rc = state_out(c, c->A[0], J, 1.0);
  if (rc == LYM1_OK) rc = state_out(c, c->A[1], Hx, 1.0);
  if (rc == LYM1_OK) rc = state_out(c, c->A[2], Hy, 1.0);
  if (rc != LYM1_OK) return rc;
  LYM1_TRY(cudaStreamSynchronize(c->stream));
  return LYM1_OK;
}

int lym1_state_elem_size(lym1_ctx* c, int* bytes) {
  if (!c || !bytes) return LYM1_EINVAL;
  *bytes = static_cast<int>(c->selem);
  return LYM1_OK;
}

int lym1_get_rows(lym1_ctx* c, int y0, int n_rows, void* J, void* Hx, void* Hy) {
  if (!c || !J || !Hx || !Hy || y0 < 0 || n_rows < 0 || y0 > c->ny - n_rows) return LYM1_EINVAL;
  if (n_rows == 0) return LYM1_OK;
  // every bin's rows [y0, y0 + n_rows) are contiguous: one strided copy per array
  const size_t w = static_cast<size_t>(n_rows) * c->nx * c->selem;
  const size_t off = static_cast<size_t>(y0) * c->nx * c->selem;
  const size_t pitch = static_cast<size_t>(c->nc) * c->selem;
  void* dst[3] = {J, Hx, Hy};
  for (int i = 0; i < 3; ++i)
    LYM1_TRY(cudaMemcpy2DAsync(dst[i], w, static_cast<const char*>(c->A[i]) + off, pitch, w,
                               static_cast<size_t>(c->nb), cudaMemcpyDefault, c->stream));
  return LYM1_OK;
}

int lym1_set_rows(lym1_ctx* c, int y0, int n_rows, const void* J, const void* Hx, const void* Hy) {
  if (!c || !J || !Hx || !Hy || y0 < 0 || n_rows < 0 || y0 > c->ny - n_rows) return LYM1_EINVAL;
  if (n_rows == 0) return LYM1_OK;
  const size_t w = static_cast<size_t>(n_rows) * c->nx * c->selem;
  const size_t off = static_cast<size_t>(y0) * c->nx * c->selem;
  const size_t pitch = static_cast<size_t>(c->nc) * c->selem;
  const void* src[3] = {J, Hx, Hy};
  for (int i = 0; i < 3; ++i)
    LYM1_TRY(cudaMemcpy2DAsync(static_cast<char*>(c->A[i]) + off, pitch, src[i], w, w,
                               static_cast<size_t>(c->nb), cudaMemcpyDefault, c->stream));
  return LYM1_OK;
}

int lym1_substeps(lym1_ctx* c, int n, double dt) {
  if (!c || n < 0) return LYM1_EINVAL;
  if (!(dt > 0.0)) dt = c->dt_cfl;
  if (n > 0 && dt == c->dt_cfl && !c->gray && c->freq_step) {
    // CFL substeps: the persistent work-list kernels, graph-replayed
    if (!c->self_batch) {
      lym1_ctx* one[1] = {c};
      const int rc = lym1_batch_create(one, 1, &c->self_batch);
      if (rc != LYM1_OK) return rc;
    }
    if (!c->profiling) return lym1_batch_substeps(c->self_batch, n);
    lym1_batch* b = c->self_batch;
    {
      const int rc = refresh_views(b, c->stream);
      if (rc != LYM1_OK) return rc;
    }
    int done = 0;
    if (!b->tuned) {  // the tuning substeps (untimed) count toward n
      done = std::min(n, static_cast<int>(b->cands.size() - b->ctime.size()));
      const int rc = lym1_batch_substeps(b, done);
      if (rc != LYM1_OK) return rc;
    }
    for (; done < n; ++done) {
      const int rc = batch_launch_timed(b, c);
      if (rc != LYM1_OK) return rc;
      c->substeps_done += 1;
    }
    return LYM1_OK;
  }
  for (int i = 0; i < n; ++i) {
    const int rc = one_substep(c, dt);
    if (rc != LYM1_OK) return rc;
  }
  return LYM1_OK;
}

int lym1_step(lym1_ctx* c, double dt, int* n_out) {
  if (!c || !(dt > 0.0)) return LYM1_EINVAL;
  const double r = dt / c->dt_cfl;
  if (!(r < 2e9)) return LYM1_EINVAL;
  int n = static_cast<int>(std::ceil(r));
  if (n < 1) n = 1;
  if (n_out) *n_out = n;
  return lym1_substeps(c, n, dt / n);
}

int lym1_moments(lym1_ctx* c, double* E, double* Fx, double* Fy) {
  if (!c) return LYM1_EINVAL;
  int rc = LYM1_OK;
  if (E) rc = state_out(c, c->A[0], E, (4.0 * kPi) / kLight);
  if (rc == LYM1_OK && Fx) rc = state_out(c, c->A[1], Fx, 4.0 * kPi);
  if (rc == LYM1_OK && Fy) rc = state_out(c, c->A[2], Fy, 4.0 * kPi);
  if (rc != LYM1_OK) return rc;
  LYM1_TRY(cudaStreamSynchronize(c->stream));
  return LYM1_OK;
}

int lym1_force(lym1_ctx* c, double* fx, double* fy) {
  if (!c || !fx || !fy) return LYM1_EINVAL;
  const size_t pb = static_cast<size_t>(c->nc) * sizeof(double);
  LYM1_TRY(cudaMemcpyAsync(fx, c->fx, pb, cudaMemcpyDefault, c->stream));
  LYM1_TRY(cudaMemcpyAsync(fy, c->fy, pb, cudaMemcpyDefault, c->stream));
  LYM1_TRY(cudaStreamSynchronize(c->stream));
  return LYM1_OK;
}

int lym1_diagnostics(lym1_ctx* c, lym1_diag* d) {
  if (!c || !d) return LYM1_EINVAL;
  double acc[16];
  std::vector<double> fp(2 * kForceBlocks);
  LYM1_TRYK(launch_force_reduce(c->fx, c->fy, c->nx, c->ny, c->dx, c->geometry, c->fpart,
                                kForceBlocks, c->stream));
  LYM1_TRY(cudaMemcpyAsync(acc, c->acc, sizeof acc, cudaMemcpyDeviceToHost, c->stream));
  double Ldev = 0.0;
  if (c->L_pending)
    LYM1_TRY(cudaMemcpyAsync(&Ldev, c->lsum + kSumResult, sizeof Ldev, cudaMemcpyDeviceToHost, c->stream));
  LYM1_TRY(cudaMemcpyAsync(fp.data(), c->fpart, fp.size() * sizeof(double), cudaMemcpyDeviceToHost,
                           c->stream));
  LYM1_TRY(cudaStreamSynchronize(c->stream));
  if (c->L_pending) {
    c->L_tot = Ldev;
    c->L_pending = 0;
  }
  std::memset(d, 0, sizeof *d);
  d->emitted = acc[0] + acc[1];
  d->absorbed = acc[2] + acc[3];
  d->outflow = acc[4] + acc[5];
  d->work = acc[6] + acc[7];
  d->e_tot = acc[8];
  d->max_f = acc[9];
  d->n_unrealisable = acc[10];
  d->substeps = static_cast<long long>(acc[11]);
  d->e_start = acc[12];
  d->residual = (d->e_tot - d->e_start) - (((d->emitted - d->absorbed) - d->outflow) - d->work);
  double fa = 0.0, fr = 0.0;
  for (int b = 0; b < kForceBlocks; ++b) {
    fa += fp[2 * b];
    fr += fp[2 * b + 1];
  }
  d->force_abs = fa;
  d->force_radial = fr;
  d->L_tot = c->L_tot;
  if (c->L_tot > 0.0) {
    d->M_F = fa / (c->L_tot / kLight);
    d->M_F_radial = fr / (c->L_tot / kLight);
  }
  if (d->emitted > 0.0) d->f_esc = d->outflow / d->emitted;
  const double vals[] = {d->e_tot, d->emitted, d->absorbed, d->outflow, d->work, fa, fr};
  for (double x : vals)
    if (!std::isfinite(x)) return LYM1_ENONFINITE;
  return device_status(c);
}

int lym1_get_info(lym1_ctx* c, lym1_info* o) {
  if (!c || !o) return LYM1_EINVAL;
  std::memset(o, 0, sizeof *o);
  o->nb = c->nb;
  o->precision = c->precision;
  o->dt_cfl = c->dt_cfl;
  o->eta = c->tab.eta;
  o->dnu_D = c->tab.lc.dnu_D;
  o->a_v = c->tab.lc.a_v;
  o->sigma0 = c->tab.lc.sigma0;
  // state read + written once, six FP64 per-cell inputs, the FP64 force
  o->bytes_per_substep = static_cast<double>(c->nc) *
                         (6.0 * c->nb * static_cast<double>(c->selem) + 48.0 + 16.0);
  o->device_bytes = c->device_bytes;
  o->substeps_done = c->substeps_done;
  return LYM1_OK;
}

int lym1_plan_bytes(const lym1_grid* grid, const lym1_groups* groups, int precision,
                    int temp_field, double* bytes) {
  if (!grid || !groups || !bytes) return LYM1_EINVAL;
  if (grid->nx < 1 || grid->ny < 1 || (grid->geometry != 0 && grid->geometry != 1)) return LYM1_EINVAL;
  if (precision < 0 || precision > 3) return LYM1_EINVAL;
  if (static_cast<long long>(grid->nx) * grid->ny > (1LL << 31)) return LYM1_EINVAL;
  int nb = 0;
  if (groups->edges_dnu_hz) {
    if (groups->n_bins < 1 || groups->n_bins > LYM1_MAX_BINS) return LYM1_EINVAL;
    nb = groups->n_bins;
  } else {
    const double q = groups->q > 0.0 ? groups->q : 1.1;
    const double Tm = groups->T_min > 0.0 ? groups->T_min : 30.0;
    if (!(q > 1.0)) return LYM1_EINVAL;
    std::vector<double> edges;
    nb = paper_frequency_grid(Tm, q, &edges);
    if (nb < 1 || nb > LYM1_MAX_BINS) return LYM1_EINVAL;
  }
  if (groups->gray) nb = 1;
  *bytes = plan_context_bytes(grid->nx, grid->ny, nb, precision >= LYM1_MIXED ? 4 : 8,
                              temp_field ? 1 : 0, grid->geometry);
  return LYM1_OK;
}

int lym1_tables(lym1_ctx* c, double* dnu, double* nubar, double* Havg, double* gem) {
  if (!c) return LYM1_EINVAL;
  for (int k = 0; k < c->nb; ++k) {
    if (dnu) dnu[k] = c->tab.dnu[k];
    if (nubar) nubar[k] = c->tab.nubar[k];
    if (Havg) Havg[k] = c->tab.Havg[k];
    if (gem) gem[k] = c->tab.gem[k];
  }
  return LYM1_OK;
}

int lym1_synchronize(lym1_ctx* c) {
  if (!c) return LYM1_EINVAL;
  LYM1_TRY(cudaStreamSynchronize(c->stream));
  LYM1_TRY(cudaGetLastError());
  return device_status(c);
}

int lym1_run_to_steady(lym1_ctx* c, double tol, int check_every, int max_substeps, int* n_done) {
  if (!c || !(tol > 0.0) || check_every < 1 || max_substeps < 1) return LYM1_EINVAL;
  int done = 0;
  double prev = -1.0;
  while (done < max_substeps) {
    const int n = std::min(check_every, max_substeps - done);
    const int rc = lym1_substeps(c, n, 0.0);
    if (rc != LYM1_OK) return rc;
    done += n;
    double e = 0.0;
    LYM1_TRY(cudaMemcpyAsync(&e, c->acc + 8, sizeof e, cudaMemcpyDeviceToHost, c->stream));
    LYM1_TRY(cudaStreamSynchronize(c->stream));
    if (!std::isfinite(e)) {
      if (n_done) *n_done = done;
      return LYM1_ENONFINITE;
    }
    if (prev >= 0.0 && n == check_every && e > 0.0 &&
        std::fabs(e - prev) / e / static_cast<double>(check_every) < tol) {
      if (n_done) *n_done = done;
      return LYM1_OK;
    }
    prev = e;
  }
  if (n_done) *n_done = done;
  return LYM1_ENOTCONVERGED;
}

int lym1_substeps_batched(lym1_ctx** ctxs, int n_ctx, int n) {
  lym1_batch* b = nullptr;
  int rc = lym1_batch_create(ctxs, n_ctx, &b);
  if (rc != LYM1_OK) return rc;
  rc = lym1_batch_substeps(b, n);
  lym1_batch_destroy(b);
  return rc;
}

int lym1_batch_create(lym1_ctx* const* ctxs, int n_ctx, lym1_batch** out) {
  if (!out) return LYM1_EINVAL;
  *out = nullptr;
  if (!ctxs || n_ctx < 1) return LYM1_EINVAL;
  for (int i = 0; i < n_ctx; ++i) {
    if (!ctxs[i] || ctxs[i]->gray || !ctxs[i]->freq_step) return LYM1_EINVAL;
    if (ctxs[i]->precision != ctxs[0]->precision || ctxs[i]->nb != ctxs[0]->nb ||
        ctxs[i]->stream != ctxs[0]->stream || ctxs[i]->geometry != ctxs[0]->geometry ||
        ctxs[i]->pt != ctxs[0]->pt || ctxs[i]->accept != ctxs[0]->accept)
      return LYM1_EINVAL;
  }
  lym1_batch* b = new (std::nothrow) lym1_batch();
  if (!b) return LYM1_ENOMEM;
  b->ctxs.assign(ctxs, ctxs + n_ctx);
  b->precision = ctxs[0]->precision;
  b->geometry = ctxs[0]->geometry;
  b->pt = ctxs[0]->pt;
  b->tpt = b->pt;
  for (int i = 0; i < n_ctx; ++i)
    if (ctxs[i]->prune > 0.0) b->tpt = b->pt | 4;
  b->accept = ctxs[0]->accept;
  if (b->accept) b->tpt |= 8;
  b->nb = ctxs[0]->nb;
  b->ctx_stream = ctxs[0]->stream;
  b->partS.assign(n_ctx, nullptr);
  b->fpg.assign(n_ctx, nullptr);
  std::vector<BatchItemHost> iF;
  long long tiles0 = 0;
  for (int i = 0; i < n_ctx; ++i) {
    lym1_ctx* c = ctxs[i];
    b->gens.push_back(c->view_gen);
    b->prune_gens.push_back(c->prune_gen);
    b->accept_gens.push_back(c->accept_gen);
    const int fb = freq_blocks(c->nc);
    for (int k = 0; k < fb; ++k) iF.push_back({i, 0, 0, k, 0, 0, 0});
    tiles0 += transport_blocks(c->nx, c->ny, 0);
  }
  b->nF = static_cast<int>(iF.size());
  auto fail = [&](int rc) {
    batch_free(b);
    delete b;
    return rc;
  };
  if (cudaMalloc(&b->itemsF, sizeof(BatchItemHost) * iF.size()) != cudaSuccess) {
    cudaGetLastError();
    return fail(LYM1_ENOMEM);
  }
  if (cudaMemcpy(b->itemsF, iF.data(), sizeof(BatchItemHost) * iF.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaStreamCreateWithFlags(&b->bs, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreate(&b->t0) != cudaSuccess || cudaEventCreate(&b->t1) != cudaSuccess) {
    cudaGetLastError();
    return fail(LYM1_ECUDA);
  }
  cudaGetDevice(&b->dev);
  cudaDeviceGetAttribute(&b->nsm, cudaDevAttrMultiProcessorCount, b->dev);
  if (b->nsm < 1) b->nsm = 1;
  const int nsm = b->nsm;
  const int rF = b->precision == LYM1_FP64_DET
                     ? resident_blocks_det(1, b->geometry, b->pt, b->nb)
                     : resident_blocks_fast(b->precision, 1, b->geometry, b->pt, b->nb);
  b->gridF = std::min(b->nF, rF * nsm);
  if (b->accept) {
    const int rS = b->precision == LYM1_FP64_DET
                       ? resident_blocks_det(2, b->geometry, b->pt, b->nb)
                       : resident_blocks_fast(b->precision, 2, b->geometry, b->pt, b->nb);
    b->gridS = std::min(b->nF, rS * nsm);
  }
  // candidate layouts: one 16 x 16 block per tile always; for the policies
  // other than LYM1_FP64_DET (whose batches keep it, and so equal solo runs
  // bit for bit) also 32 x 8 tiles in the plain table modes, and the bins of
  // each tile split over 2, 4 or 8 blocks where the tiles alone do not fill
  // the GPU (at least 16 bins a group)
  int base = 0;
  {
    const int rc = ensure_layout(b, 0, 1, &base);
    if (rc != LYM1_OK) return fail(rc);
  }
  std::vector<int> lay = {base};
  if (b->precision != LYM1_FP64_DET) {
    const long long room = 2LL * nsm * b->layouts[base].rT;
    if (b->tpt == 0 || b->tpt == 1) {
      int j = 0;
      const int rc = ensure_layout(b, 1, 1, &j);
      if (rc != LYM1_OK) return fail(rc);
      lay.push_back(j);
    }
    for (int g = 2; g <= 8; g *= 2) {
      if (b->nb < 16 * g || tiles0 * g > room) break;
      int j = 0;
      const int rc = ensure_layout(b, 0, g, &j);
      if (rc != LYM1_OK) return fail(rc);
      lay.push_back(j);
    }
  }
  for (int j : lay) {
    const BatchLayout& L = b->layouts[j];
    int last = 0;
    for (int m = 1; m <= L.rT; ++m) {
      const int g = std::min(L.nT, m * nsm);
      if (g != last) b->cands.push_back({j, g});
      last = g;
    }
  }
  int lg = 0;
  while ((2LL << lg) <= tiles0) ++lg;
  b->tune_key = {b->dev, b->precision, b->geometry, b->tpt, b->nb, lg};
  const std::vector<int> known = tuned_lookup(b->tune_key);
  if (known.size() == 3) {  // {shape, groups, grid} of an earlier batch of this class
    int j = 0;
    const int rc = ensure_layout(b, known[0], known[1], &j);
    if (rc != LYM1_OK) return fail(rc);
    b->cands = {{j, std::min(known[2], b->layouts[j].nT)}};
    b->tuned = 1;
  }
  b->cur = static_cast<int>(b->cands.size()) - 1;
  *out = b;
  return LYM1_OK;
}

int lym1_batch_substeps(lym1_batch* b, int n) {
  if (!b || n < 0) return LYM1_EINVAL;
  // the captured launches include the pruning kernels of the contexts that
  // pruned at creation: switching pruning since then needs a new batch
  for (size_t i = 0; i < b->ctxs.size(); ++i)
    if (b->ctxs[i]->prune_gen != b->prune_gens[i] || b->ctxs[i]->accept_gen != b->accept_gens[i])
      return LYM1_EINVAL;
  if (n == 0) return LYM1_OK;
  LYM1_TRY(cudaEventRecord(b->ev_in, b->ctx_stream));
  LYM1_TRY(cudaStreamWaitEvent(b->bs, b->ev_in, 0));
  {
    const int rc = refresh_views(b, b->bs);
    if (rc != LYM1_OK) return rc;
  }
  int done = 0;
  // tuning: the first substeps run once with each candidate (layout, grid)
  while (!b->tuned && done < n) {
    b->cur = static_cast<int>(b->ctime.size());
    LYM1_TRY(cudaEventRecord(b->t0, b->bs));
    const int rc = batch_launch(b, b->bs);
    if (rc != LYM1_OK) return rc;
    LYM1_TRY(cudaEventRecord(b->t1, b->bs));
    LYM1_TRY(cudaEventSynchronize(b->t1));
    float ms = 0.0f;
    LYM1_TRY(cudaEventElapsedTime(&ms, b->t0, b->t1));
    b->ctime.push_back(ms);
    ++done;
    if (b->ctime.size() == b->cands.size()) {
      size_t best = 0;
      for (size_t k = 1; k < b->ctime.size(); ++k)
        if (b->ctime[k] < b->ctime[best]) best = k;
      b->cur = static_cast<int>(best);
      b->tuned = 1;
      const BatchLayout& L = b->layouts[b->cands[best].first];
      tuned_store(b->tune_key, {L.shape, L.groups, b->cands[best].second});
    }
  }
  if (done < n) {
    if (!b->exec) {
      LYM1_TRY(cudaStreamBeginCapture(b->bs, cudaStreamCaptureModeThreadLocal));
      const int rc = batch_launch(b, b->bs);
      cudaGraph_t g = nullptr;
      const cudaError_t e = cudaStreamEndCapture(b->bs, &g);
      if (rc != LYM1_OK) return rc;
      LYM1_TRY(e);
      b->graph = g;
      LYM1_TRY(cudaGraphInstantiate(&b->exec, b->graph, 0));
    }
    for (; done < n; ++done) LYM1_TRY(cudaGraphLaunch(b->exec, b->bs));
  }
  LYM1_TRY(cudaEventRecord(b->ev_out, b->bs));
  LYM1_TRY(cudaStreamWaitEvent(b->ctx_stream, b->ev_out, 0));
  for (lym1_ctx* c : b->ctxs) c->substeps_done += n;
  return LYM1_OK;
}

int lym1_batch_grid(lym1_batch* b, int* gt, int* gf) {
  if (!b) return LYM1_EINVAL;
  if (gt) *gt = b->tuned ? b->cands[b->cur].second : 0;
  if (gf) *gf = b->tuned ? b->gridF : 0;
  return LYM1_OK;
}

int lym1_batch_config(lym1_batch* b, int* tile_x_out, int* tile_y_out, int* groups, int* grid_t,
                      int* grid_f) {
  if (!b) return LYM1_EINVAL;
  const BatchLayout& L = b->layouts[b->cands[b->cur].first];
  if (tile_x_out) *tile_x_out = b->tuned ? tile_x(L.shape) : 0;
  if (tile_y_out) *tile_y_out = b->tuned ? tile_y(L.shape) : 0;
  if (groups) *groups = b->tuned ? L.groups : 0;
  if (grid_t) *grid_t = b->tuned ? b->cands[b->cur].second : 0;
  if (grid_f) *grid_f = b->tuned ? b->gridF : 0;
  return LYM1_OK;
}

int lym1_batch_configure(lym1_batch* b, int tile_shape, int bin_groups, int grid_t) {
  if (!b) return LYM1_EINVAL;
  if (tile_shape != 0 && tile_shape != 1) return LYM1_EINVAL;
  if (tile_shape == 1 && b->tpt != 0 && b->tpt != 1) return LYM1_EINVAL;
  if (bin_groups != 1 && bin_groups != 2 && bin_groups != 4 && bin_groups != 8) return LYM1_EINVAL;
  if (bin_groups > b->nb || grid_t < 0) return LYM1_EINVAL;
  LYM1_TRY(cudaStreamSynchronize(b->bs));
  int j = 0;
  {
    const int rc = ensure_layout(b, tile_shape, bin_groups, &j);
    if (rc != LYM1_OK) return rc;
  }
  const BatchLayout& L = b->layouts[j];
  const int g = grid_t > 0 ? grid_t : L.rT * b->nsm;
  b->cands = {{j, std::min(g, L.nT)}};
  b->ctime.clear();
  b->cur = 0;
  b->tuned = 1;
  // the captured launches hold the old layout
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
  return LYM1_OK;
}

void lym1_batch_destroy(lym1_batch* b) {
  if (!b) return;
  cudaStreamSynchronize(b->bs);
  batch_free(b);
  delete b;
}

int lym1_debug_expire_wait(lym1_ctx* c) {
  if (!c) return LYM1_EINVAL;
  if (c->precision < LYM1_MIXED || (c->nc & 3) != 0 || c->gray || !c->freq_step) return LYM1_EINVAL;
  const int one = 1;
  LYM1_TRY(cudaMemcpyAsync(c->status + 1, &one, sizeof one, cudaMemcpyHostToDevice, c->stream));
  LYM1_TRY(cudaStreamSynchronize(c->stream));
  return LYM1_OK;
}

int lym1_profile_enable(lym1_ctx* c, int on) {
  if (!c) return LYM1_EINVAL;
  c->profiling = on != 0;
  return LYM1_OK;
}

int lym1_profile_read(lym1_ctx* c, lym1_profile* out, int reset) {
  if (!c || !out) return LYM1_EINVAL;
  LYM1_TRY(cudaStreamSynchronize(c->stream));
  std::memset(out, 0, sizeof *out);
  for (size_t i = 0; i < c->ev_kind.size(); ++i) {
    float ms = 0.0f;
    LYM1_TRY(cudaEventElapsedTime(&ms, c->ev_start[i], c->ev_stop[i]));
    switch (c->ev_kind[i]) {
      case 0: out->transport_ms += ms; out->transport_launches += 1; break;
      case 1: out->freq_ms += ms; out->freq_launches += 1; break;
      default: out->finalize_ms += ms; out->finalize_launches += 1; break;
    }
  }
  if (reset) drop_events(c);
  return LYM1_OK;
}

}  // extern "C"

int lym1_spectrum_enable(lym1_ctx* c, int on) {
  if (!c) return LYM1_EINVAL;
  const int nf = c->geometry == 1 ? (c->nx + c->ny) : 2 * (c->nx + c->ny);
  const size_t bytes = sizeof(double) * static_cast<size_t>(nf) * c->nb;
  if (on) {
    if (!c->spec) {
      const int rc = dalloc_t(c, &c->spec, bytes / sizeof(double));
      if (rc != LYM1_OK) return rc;
    }
    LYM1_TRY(cudaMemsetAsync(c->spec, 0, bytes, c->stream));
  }
  c->spec_on = on ? 1 : 0;
  // the graph-replayed path holds device copies of the views: rebuild it
  if (c->self_batch) {
    LYM1_TRY(cudaStreamSynchronize(c->stream));
    lym1_batch_destroy(c->self_batch);
    c->self_batch = nullptr;
  }
  return LYM1_OK;
}

int lym1_spectrum_read(lym1_ctx* c, double* out, int* n_faces) {
  if (!c) return LYM1_EINVAL;
  const int nf = c->geometry == 1 ? (c->nx + c->ny) : 2 * (c->nx + c->ny);
  if (n_faces) *n_faces = nf;
  if (!out) return LYM1_OK;
  if (!c->spec) return LYM1_EINVAL;
  const size_t bytes = sizeof(double) * static_cast<size_t>(nf) * c->nb;
  LYM1_TRY(cudaMemcpyAsync(out, c->spec, bytes, cudaMemcpyDefault, c->stream));
  LYM1_TRY(cudaStreamSynchronize(c->stream));
  return LYM1_OK;
}

int lym1_set_ctilde(lym1_ctx* c, double c_tilde) {
  if (!c || !(c_tilde > 0.0) || !(c_tilde <= kLight)) return LYM1_EINVAL;
  c->c_tilde = c_tilde;
  c->dt_cfl = (c->cfl / 2.0) * (c->dx / (c_tilde + c->umax));
  c->view_gen += 1;
  return LYM1_OK;
}

int lym1_dynamic_ctilde(lym1_ctx* c, const double* cs, double eps_rsl, double ct_min,
                        double* c_tilde_out) {
  if (!c || c->bands || !(eps_rsl > 0.0) || !std::isfinite(eps_rsl) || !(ct_min >= 0.0) ||
      !(ct_min <= kLight))
    return LYM1_EINVAL;
  const double* dcs = nullptr;
  if (cs) {
    LYM1_TRY(cudaMemcpyAsync(c->staging, cs, static_cast<size_t>(c->nc) * sizeof(double),
                             cudaMemcpyDefault, c->stream));
    dcs = c->staging;
  }
  LYM1_TRYK(launch_dynamic_ctilde(c->alpha, c->rho, c->pd, c->ux, c->uy, c->Tc, c->T, dcs, c->kabs,
                                  c->dx, c->nc, eps_rsl, ct_min, c->c_tilde, c->ctw, c->stream));
  double ct = 0.0;
  LYM1_TRY(cudaMemcpyAsync(&ct, c->ctw + 1, sizeof ct, cudaMemcpyDeviceToHost, c->stream));
  LYM1_TRY(cudaStreamSynchronize(c->stream));
  if (!(ct > 0.0) || !(ct <= kLight)) return LYM1_ENONFINITE;
  const int rc = lym1_set_ctilde(c, ct);
  if (rc == LYM1_OK && c_tilde_out) *c_tilde_out = ct;
  return rc;
}

int lym1_set_temperature(lym1_ctx* c, const double* temp_field) {
  if (!c || !temp_field || c->pt != 1) return LYM1_EINVAL;
  const size_t plane = static_cast<size_t>(c->nc);
  const size_t pb = plane * sizeof(double);
  std::vector<double> hT(plane);
  LYM1_TRY(cudaStreamSynchronize(c->stream));
  if (cudaMemcpy(hT.data(), temp_field, pb, cudaMemcpyDefault) != cudaSuccess) {
    cudaGetLastError();
    return LYM1_EINVAL;
  }
  for (double t : hT)
    if (!(t > 0.0) || !std::isfinite(t)) return LYM1_EINVAL;
  const int n = static_cast<int>(c->edges.size()) - 1;
  // scratch: the temperatures and the edges
  double* scr = nullptr;
  const size_t words = plane + static_cast<size_t>(n + 1);
  if (cudaMalloc(&scr, words * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    return LYM1_ENOMEM;
  }
  double* dT = scr;
  double* de = scr + plane;
  int rc = LYM1_OK;
  if (cudaMemcpy(dT, hT.data(), pb, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(de, c->edges.data(), sizeof(double) * (n + 1), cudaMemcpyHostToDevice) != cudaSuccess)
    rc = LYM1_ECUDA;
  if (rc == LYM1_OK &&
      launch_cell_tables(static_cast<int>(c->selem), dT, c->nhi, de, n, c->gray, c->recoil,
                         c->geometry, c->dx, c->nc, c->Hc, c->Gc, c->gmaxc, c->Kcc, c->hkTc,
                         c->sig0c, c->alpha, c->Tc, c->stream) != 0)
    rc = LYM1_ECUDA;
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) rc = LYM1_ECUDA;
  cudaFree(scr);
  return rc;
}

int lym1_set_accept(lym1_ctx* c, int on) {
  if (!c || (on != 0 && on != 1)) return LYM1_EINVAL;
  if (on && c->bands) return LYM1_EINVAL;  // the rule watches the Lya energy density
  if (on == c->accept) return LYM1_OK;
  c->accept = on;
  c->accept_gen += 1;
  c->view_gen += 1;
  // the graph-replayed path captured its launches with the old setting
  if (c->self_batch) {
    LYM1_TRY(cudaStreamSynchronize(c->stream));
    lym1_batch_destroy(c->self_batch);
    c->self_batch = nullptr;
  }
  return LYM1_OK;
}

int lym1_set_pruning(lym1_ctx* c, double cut) {
  if (!c || !(cut >= 0.0) || !(cut < 1.0)) return LYM1_EINVAL;
  if (cut > 0.0) {  // each buffer once (a failed call leaves the other for the next)
    int rc = c->Ebin ? LYM1_OK : dalloc_t(c, &c->Ebin, static_cast<size_t>(c->nb) * 17);
    if (rc == LYM1_OK && !c->active) rc = dalloc_t(c, &c->active, static_cast<size_t>(c->nb));
    if (rc != LYM1_OK) return rc;
  }
  // the captured launches hold the cut by value: any change rebuilds them
  const bool changed = cut != c->prune;
  c->prune = cut;
  if (changed) {
    c->prune_gen += 1;
    c->view_gen += 1;
    // the graph-replayed path captured its launches with the old setting
    if (c->self_batch) {
      LYM1_TRY(cudaStreamSynchronize(c->stream));
      lym1_batch_destroy(c->self_batch);
      c->self_batch = nullptr;
    }
  }
  return LYM1_OK;
}
