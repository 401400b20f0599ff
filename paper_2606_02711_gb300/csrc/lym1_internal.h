// lym1_internal.h -- declarations shared by the host API (lym1_api.cu), the
// host table setup (lym1_tables.cpp) and the kernel translation units.
#pragma once

#include <cstddef>
#include <cstdint>
#include <vector>

namespace lym1 {

// physical constants, cgs (CODATA 2018)
constexpr double kPi = 3.14159265358979323846;
constexpr double kSqrtPi = 1.772453850905516;
constexpr double kLight = 2.99792458e10;        // cm/s
constexpr double kPlanck = 6.62607015e-27;      // erg s
constexpr double kBoltzmann = 1.380649e-16;     // erg/K
constexpr double kMassE = 9.1093837015e-28;     // g
constexpr double kCharge = 4.803204712570263e-10;  // esu
constexpr double kMassH = 1.67353284e-24;       // g, hydrogen atom
constexpr double kNuLya = kLight / 1215.67e-8;  // Hz, Lya line centre
constexpr double kNuLyc = 3.28805e15;           // Hz, H ionisation threshold
constexpr double kEinsteinA = 6.265e8;          // 1/s, Lya
constexpr double kOscStrength = 0.4162;         // Lya f_12

struct LineConstants {
  double dnu_D = 0, a_v = 0, sigma0 = 0;
};

struct BinTables {
  int nb = 0;
  LineConstants lc;
  double eta = 0, hkT = 0;
  std::vector<double> dnu, nubar, Havg, gem, Rk, half, nubar_c;
};

// Per-column tables of the axisymmetric (R, Z) grid, per radian: R-face areas
// AR[i] = R_i dZ (nx+1), Z-face areas AZ = (R+^2 - R-^2)/2, volumes Vol = AZ dZ,
// <1/R> = dR dZ / Vol, ring volumes 2 pi Vol, centroid-to-face distances on
// the two sides of each R face (nx+1; the axis face mirrors the first
// centroid, the outer face sits half a cell from a ghost at Rbar + dx), and
// the dimensionless factors the FP32 kernels use: AR[i] dx / Vol, AR[i+1] dx /
// Vol, dx^3 / Vol (the hoop factor), 2 pi Vol / dx^3 (energy weight).
struct CylTables {
  std::vector<double> AR, AZ, Vol, invR, V2pi, dlL, dlR, wv;
  std::vector<float> r0, r1, hoop, fdlL, fdlR, fwv;
  double wR = 0;  // 2 pi AR[nx] / dx^2: outflow weight of the outer R face
};

LineConstants line_constants(double T);
int paper_frequency_grid(double T_min, double q, std::vector<double>* edges);
// cell volume dx^3 in the emissivity factor gem_k for geometry 0; 1 for the
// axisymmetric grid, whose per-cell luminosity is divided by 2 pi Vol on the
// device
void build_tables(const std::vector<double>& edges, double T, double dx, int gray, int recoil,
                  BinTables* t, int geometry = 0);
void build_cyl_tables(int nx, double dx, CylTables* g);

// A0 at every cell's own temperature (per-cell gas temperature): <H>_k and the
// emission factor per [k][cell] and the per-cell line constants.  The same
// routine as build_tables runs once per distinct temperature value.
struct CellTables {
  std::vector<double> H, G;                // [nb][nc]
  std::vector<double> sigma0, hkT, Kc, gmax;  // [nc]; Kc = dnu_D^2 / 2, gmax = max_k G
};
void build_cell_tables(const std::vector<double>& edges, const double* T, long long nc, double dx,
                       int gray, int recoil, int geometry, CellTables* out);

// ---------------------------------------------------------------- kernel side
// transport tile: one thread per cell; 16 x 16 makes the 32 faces beyond
// the per-thread left and bottom faces (top row, right column) one warp's work.
// Persistent batched launches may take the other shape the tuner times,
// 32 x 8 (shape 1: rows of 128 bytes, 40 extra faces).
constexpr int kTileX = 16;
constexpr int kTileY = 16;
template <int TS>
struct TileShape {
  static constexpr int X = TS == 1 ? 32 : 16;
  static constexpr int Y = TS == 1 ? 8 : 16;
};
inline int tile_x(int shape) { return shape == 1 ? 32 : 16; }
inline int tile_y(int shape) { return shape == 1 ? 8 : 16; }
constexpr int kFreqThreads = 128;
constexpr int kDiagSlots = 8;  // per-block partial sums written by the kernels

// per-block partial sums (slot meaning)
enum DiagSlot {
  kSlotEmitted = 0,
  kSlotAbsorbed = 1,
  kSlotOutflow = 2,
  kSlotWork = 3,
  kSlotEnergy = 4,     // sum_k dnu_k J_k after the substep (Hz-weighted, per cell volume)
  kSlotMaxF = 5,       // max |H|/J
  kSlotBad = 6,        // count of |H| > J (1 + 1e-6)
  kSlotForceAbs = 7,   // filled by the force reduction
};

// Device pointers of one context's arrays, passed by value to the kernels.
struct DeviceView {
  int nx = 0, ny = 0, nb = 0;
  long long nc = 0;
  double dx = 0;
  // state ping-pong (element type depends on the precision; void here)
  const void* J = nullptr;
  const void* Hx = nullptr;
  const void* Hy = nullptr;
  void* Jo = nullptr;
  void* Hxo = nullptr;
  void* Hyo = nullptr;
  // per-cell statics (FP64)
  const double* alpha = nullptr;
  const double* rho = nullptr;
  const double* pd = nullptr;
  const double* ux = nullptr;
  const double* uy = nullptr;
  const double* gxx = nullptr;
  const double* gyy = nullptr;
  const double* gsh = nullptr;
  const double* lum = nullptr;
  // per-bin tables (FP64, nb each)
  const double* t_dnu = nullptr;
  const double* t_H = nullptr;
  const double* t_gem = nullptr;
  const double* t_half = nullptr;
  const double* t_R = nullptr;
  const double* t_nbc = nullptr;
  const double* t_dH = nullptr;  // dnu_k <H>_k
  // outputs
  double* fx = nullptr;
  double* fy = nullptr;
  double* partT = nullptr;  // transport-kernel block partials [blocks][kDiagSlots]
  double* partF = nullptr;  // frequency-kernel block partials [blocks][kDiagSlots]
  // scalars
  double kabs = 0, kF = 0, Kc = 0, cdt = 0, fcoef = 0;
  // c_tilde dt / dx and c_tilde dt / c, formed on the host (the FP32 tiles
  // would otherwise divide in FP64 on every thread of every tile)
  double cdt_dx = 0, cdt_c = 0;
  double gem_max = 1;  // max_k gem_k (FP32 emissivity scaling)
  double rcdt = 0;     // 1 / (c_tilde dt)
  double ct = 0, dt = 0;  // c_tilde and dt apart (substep lengths of the acceptance rule)
  // bins of a small grid's tiles split over ngrp blocks (the batch's tuned
  // choice): each group writes its raw force sums to fpg[(2 grp + c) nc +
  // cell], which the frequency step adds up in group order; 1 = one block
  // per tile writes the force itself
  double* fpg = nullptr;
  int ngrp = 1;
  const double* acc = nullptr;  // running totals: [8] energy of the last substep, [13] energy unit
  int* status = nullptr;        // device status word: nonzero after a bounded wait expired
  // FP32 copies of the per-bin tables for the FP32 policies: <H>_k, dnu_k,
  // gem_k / gem_max, R_k, nubar_k / c, half width
  const float* f_H = nullptr;
  const float* f_dnu = nullptr;
  const float* f_G = nullptr;
  const float* f_R = nullptr;
  const float* f_nbc = nullptr;
  const float* f_half = nullptr;
  int freq_step = 0;
  // 1: the transport kernel produces the energy and realisability partials
  // (no frequency step follows it in this substep)
  int tdiag = 1;
  // axisymmetric (R, Z) grid (geometry 1): per-cell <u_R / R> and the
  // per-column tables of CylTables (nullptr for geometry 0)
  int geometry = 0;
  // outflow sides into vacuum (bit 0 x-, 1 x+, 2 y-, 3 y+): ghost cells there
  // carry no radiation; the other outflow sides copy the edge cell
  int vac = 0;
  // per-cell gas temperature (pt = 1): <H>_k and the emission factor per
  // [k][cell] in the state type (FP32 policies hold G / gmax), and the
  // per-cell line constants; the per-bin tables above are then unused
  // emergent spectrum (nullptr: off): escaping energy (erg) accumulated per
  // [bin][outer face] (faces x-, x+, y-, y+ for geometry 0; R and Z outer for
  // geometry 1); spec_unit = 4 pi / c
  double* spec = nullptr;
  double spec_unit = 0;
  int nf = 0;
  int pt = 0;
  const void* Hc = nullptr;
  const void* Gc = nullptr;
  // broad bands (pt = 2): Hc holds alpha_F, Gc the emissivity (over gmaxc in
  // FP32) and Kb the absorption opacity kappa of each [band][cell]
  const void* Kb = nullptr;
  // active-bin pruning: 1 per bin that step 1 advects this substep, or
  // nullptr (every bin)
  const unsigned char* active = nullptr;
  const double* gmaxc = nullptr;
  const double* Kcc = nullptr;
  const double* hkTc = nullptr;
  const double* t_2nu = nullptr;  // 2 / nubar_k
  const float* f_2nu = nullptr;
  const double* gphi = nullptr;
  const double* g_AR = nullptr;
  const double* g_AZ = nullptr;
  const double* g_Vol = nullptr;
  const double* g_invR = nullptr;
  const double* g_dlL = nullptr;
  const double* g_dlR = nullptr;
  const double* g_wv = nullptr;
  const float* gf_r0 = nullptr;
  const float* gf_r1 = nullptr;
  const float* gf_hoop = nullptr;
  const float* gf_dlL = nullptr;
  const float* gf_dlR = nullptr;
  const float* gf_wv = nullptr;
  double g_wR = 0;
};

// Launchers (defined in the kernel translation units); each returns a
// cudaError_t cast to int.
int launch_transport_det(const DeviceView& v, void* stream);
int launch_freq_det(const DeviceView& v, void* stream);
int launch_transport_fast(int precision, const DeviceView& v, void* stream);
int launch_freq_fast(int precision, const DeviceView& v, void* stream);
// step 2 under the substep acceptance rule, in place on the view's input state
int launch_subcycle_det(const DeviceView& v, void* stream);
int launch_subcycle_fast(int precision, const DeviceView& v, void* stream);
// wcol: per-column energy weights (nullptr = 1), nx columns
int launch_energy(int precision, const void* J, const double* dnu, int nb, long long nc,
                  double* part, const double* wcol, int nx, void* stream);
int launch_finalize(const double* partT, int nT, const double* partE, int nE, double* acc,
                    int mode, void* stream);
// sigma0c: per-cell line-centre cross-sections (temperature field) or nullptr
int launch_setup_statics(const double* n_hi, const double* ux, const double* uy, double sigma0,
                         const double* sigma0c, int nx, int ny, double dx, double* alpha,
                         double* gxx, double* gyy, double* gsh, int geometry, double* gphi,
                         void* stream);
// lum[j][i] /= V2pi[i] (axisymmetric grid: per-volume luminosity density)
int launch_scale_columns(double* lum, const double* V2pi, int nx, long long nc, void* stream);
int launch_convert_out(int precision, const void* src, double* dst, long long n, double scale,
                       void* stream);
int launch_convert_in(int precision, const double* src, void* dst, long long n, void* stream);
int launch_force_reduce(const double* fx, const double* fy, int nx, int ny, double dx,
                        int geometry, double* part, int nblocks, void* stream);
// sum over cells of a[n] into work[152] (work: 152 partials, the sum, a zeroed
// counter word; kSumWork doubles)
constexpr int kSumWork = 154;
constexpr int kSumResult = 152;  // index of the sum in work
int launch_sum_cells(const double* a, long long n, double* work, void* stream);
// active-bin pruning: E[k] = dnu_k sum_cells w J_k (w = wcol[column], or 1),
// then active[k] = E[k] > cut sum_k E[k]; E holds nb x (1 + 16) doubles
// (the energies, then per-chunk partial sums)
int launch_active_bins(int selem, const void* J, int nb, long long nc, int nx, const double* wcol,
                       const double* dnu, double cut, double* E, unsigned char* active,
                       void* stream);
// per-cell A0 tables of a temperature field on the device (n = bins of the edges)
int launch_cell_tables(int selem, const double* T, const double* nhi, const double* edges, int n,
                       int gray, int recoil, int geometry, double dx, long long nc, void* Hc,
                       void* Gc, double* gmaxc, double* Kcc, double* hkTc, double* sig0c,
                       double* alpha, double* Tc, void* stream);
// dynamic reduced speed of light: work holds 2 words (the running maximum,
// then the new c_tilde as a double); Tc per-cell temperatures or nullptr (T),
// cs per-cell sound speeds or nullptr (neutral gas at T)
int launch_dynamic_ctilde(const double* alpha, const double* rho, const double* pd,
                          const double* ux, const double* uy, const double* Tc, double T,
                          const double* cs, double kabs, double dx, long long nc, double eps,
                          double ct_min, double prev, unsigned long long* work, void* stream);

// batched (multi-context) launches; kind 0 = transport, 1 = frequency step,
// 2 = step 2 under the acceptance rule (over the frequency step's items);
// items point to device arrays of {ctx, x0, y0, blk}
struct FinalizeJob {
  const double* partT;
  const double* partE;
  double* acc;
  int nT, nE;
  int mode;  // 0, or 2 when step 2 ran in the subcycling kernel
};
// every context of one batched launch has the same geometry
// every context of one batched launch has the same geometry and temperature mode
// shape: the transport tile shape (TileShape; 1 only with table modes 0 and 1)
int launch_batched_det(int kind, int geometry, int pt, const DeviceView* views, const void* items,
                       int n, int grid, int nb_max, void* stream, int shape = 0);
int launch_batched_fast(int precision, int kind, int geometry, int pt, const DeviceView* views,
                        const void* items, int n, int grid, int nb_max, void* stream, int shape = 0);
// blocks of one persistent launch resident per SM at nb_max bins (also opts
// the frequency kernels in to their shared-memory size; call outside capture)
int resident_blocks_det(int kind, int geometry, int pt, int nb_max, int shape = 0);
int resident_blocks_fast(int precision, int kind, int geometry, int pt, int nb_max, int shape = 0);
int launch_finalize_batched(const FinalizeJob* jobs, int n, void* stream);

inline int transport_blocks(int nx, int ny, int shape = 0) {
  const int tx = tile_x(shape), ty = tile_y(shape);
  return ((nx + tx - 1) / tx) * ((ny + ty - 1) / ty);
}
inline int freq_blocks(long long nc) {
  return static_cast<int>((nc + kFreqThreads - 1) / kFreqThreads);
}

}  // namespace lym1
