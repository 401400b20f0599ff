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

LineConstants line_constants(double T);
int paper_frequency_grid(double T_min, double q, std::vector<double>* edges);
void build_tables(const std::vector<double>& edges, double T, double dx, int gray, int recoil,
                  BinTables* t);

// ---------------------------------------------------------------- kernel side
constexpr int kTileX = 32;   // transport tile: one thread per cell
constexpr int kTileY = 8;
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
  // outputs
  double* fx = nullptr;
  double* fy = nullptr;
  double* partT = nullptr;  // transport-kernel block partials [blocks][kDiagSlots]
  double* partF = nullptr;  // frequency-kernel block partials [blocks][kDiagSlots]
  // scalars
  double kabs = 0, kF = 0, Kc = 0, cdt = 0, fcoef = 0;
  double gem_max = 1;  // max_k gem_k (FP32 emissivity scaling)
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
};

// Launchers (defined in the kernel translation units); each returns a
// cudaError_t cast to int.
int launch_transport_det(const DeviceView& v, void* stream);
int launch_freq_det(const DeviceView& v, void* stream);
int launch_transport_fast(int precision, const DeviceView& v, void* stream);
int launch_freq_fast(int precision, const DeviceView& v, void* stream);
int launch_energy(int precision, const void* J, const double* dnu, int nb, long long nc,
                  double* part, void* stream);
int launch_finalize(const double* partT, int nT, const double* partE, int nE, double* acc,
                    int mode, void* stream);
int launch_setup_statics(const double* n_hi, const double* ux, const double* uy, double sigma0,
                         int nx, int ny, double dx, double* alpha, double* gxx, double* gyy,
                         double* gsh, void* stream);
int launch_convert_out(int precision, const void* src, double* dst, long long n, double scale,
                       void* stream);
int launch_convert_in(int precision, const double* src, void* dst, long long n, void* stream);
int launch_force_reduce(const double* fx, const double* fy, int nx, int ny, double dx,
                        double* part, int nblocks, void* stream);

// batched (multi-context) launches; kind 0 = transport, 1 = frequency step;
// items point to device arrays of {ctx, x0, y0, blk}
struct FinalizeJob {
  const double* partT;
  const double* partE;
  double* acc;
  int nT, nE;
};
int launch_batched_det(int kind, const DeviceView* views, const void* items, int n, int grid,
                       int nb_max, void* stream);
int launch_batched_fast(int precision, int kind, const DeviceView* views, const void* items, int n,
                        int grid, int nb_max, void* stream);
int resident_blocks_det(int kind);
int resident_blocks_fast(int precision, int kind);
int launch_finalize_batched(const FinalizeJob* jobs, int n, void* stream);

inline int transport_blocks(int nx, int ny) {
  return ((nx + kTileX - 1) / kTileX) * ((ny + kTileY - 1) / kTileY);
}
inline int freq_blocks(long long nc) {
  return static_cast<int>((nc + kFreqThreads - 1) / kFreqThreads);
}

}  // namespace lym1
