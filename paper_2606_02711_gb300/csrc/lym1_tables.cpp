// lym1_tables.cpp -- host-side setup of the per-bin tables (row A0 of the
// substep): the paper's frequency grid, the line constants, the bin-averaged
// Voigt profile and the emission fractions.  Runs once per context on the host
// (a few hundred bins); compiled without FMA contraction so that the tables are
// reproducible to the last bit on any host.
//
// Sources (arXiv 2606.02711):
//   frequency grid ............ Sec. 2.1, grid paragraph (q = 1.1, T_min = 30 K,
//                               |dnu| <= min(1e5 dnu_D(T_min), 0.99 nu_Lya, nu_LyC - nu_Lya))
//   a_v, sigma0, dnu_D ........ Sec. 2.1 (a_v ~ 4.7e-4 T4^-1/2, sigma0 ~ 5.9e-14 T4^-1/2)
//   <H>_k, I(x, a) ............ App. A, bin-averaged Voigt profile and its integral
//   phi_nu = H / sqrt(pi) ..... Sec. 2.1 step 2 (emission profile)
//   bin centres = midpoints ... App. A footnote
#include <cstring>
#include <thread>
#include <unordered_map>
#include <cmath>
#include <cstring>
#include <vector>

#include "lym1_internal.h"

namespace lym1 {

namespace {

// Dawson's integral F(x) = exp(-x^2) int_0^x exp(t^2) dt:
//   |x| < 0.2  Maclaurin series sum_n (-2)^n x^(2n+1) / (2n+1)!!,
//   |x| < 10   Rybicki's (1989) sampling-theorem sum with step h = 0.2:
//              F(x) ~ pi^-1/2 sum over odd n of exp(-(x - n h)^2) / n,
//   otherwise  the asymptotic series (1/2x) sum_n (2n-1)!! / (2x^2)^n.
double dawson(double x) {
  const double ax = std::fabs(x);
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
    const int lo = static_cast<int>(std::ceil((ax - 8.0) / h));
    const int hi = static_cast<int>(std::floor((ax + 8.0) / h));
    double s = 0.0;
    for (int n = lo; n <= hi; ++n) {
      if ((n & 1) == 0) continue;
      const double d = ax - n * h;
      s += std::exp(-d * d) / n;
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

// I(x, a) without its erf term: -(2a/sqrt(pi)) F(x) + a^2 x exp(-x^2)
double voigt_integral_rest(double x, double a) {
  return -((2.0 * a) / kSqrtPi) * dawson(x) + ((a * a) * x) * std::exp(-(x * x));
}

// <H> over [xa, xb] (Doppler units).  The erf difference goes through erfc on
// the side of the bin away from line centre, which keeps the wing bins exact.
double bin_voigt(double xa, double xb, double a, double dxk) {
  double derf;
  if (xa >= 0.0)
    derf = (kSqrtPi / 2.0) * (std::erfc(xa) - std::erfc(xb));
  else if (xb <= 0.0)
    derf = (kSqrtPi / 2.0) * (std::erfc(-xb) - std::erfc(-xa));
  else
    derf = (kSqrtPi / 2.0) * (std::erf(xb) - std::erf(xa));
  return (derf + (voigt_integral_rest(xb, a) - voigt_integral_rest(xa, a))) / dxk;
}

}  // namespace

LineConstants line_constants(double T) {
  LineConstants lc;
  lc.dnu_D = (kNuLya * std::sqrt((2.0 * kBoltzmann * T) / kMassH)) / kLight;
  lc.a_v = kEinsteinA / ((4.0 * kPi) * lc.dnu_D);
  lc.sigma0 = ((kSqrtPi * (kCharge * kCharge)) * kOscStrength) / ((kMassE * kLight) * lc.dnu_D);
  return lc;
}

int paper_frequency_grid(double T_min, double q, std::vector<double>* edges) {
  const double w0 = line_constants(T_min).dnu_D;
  double lim = 1e5 * w0;
  if (0.99 * kNuLya < lim) lim = 0.99 * kNuLya;
  if (kNuLyc - kNuLya < lim) lim = kNuLyc - kNuLya;
  std::vector<double> side{0.0};
  double e = 0.0, w = w0;
  for (;;) {
    const double next = e + w;
    if (side.size() > 100000) return -1;
    if (next >= lim) {
      side.push_back(lim);
      break;
    }
    side.push_back(next);
    e = next;
    w = w * q;
  }
  const int M = static_cast<int>(side.size()) - 1;
  edges->assign(2 * M + 1, 0.0);
  for (int j = 0; j <= M; ++j) {
    (*edges)[M + j] = side[j];
    (*edges)[M - j] = -side[j];
  }
  (*edges)[M] = 0.0;
  return 2 * M;
}

// Fills the per-bin tables of a context.  For a gray group the single "bin"
// carries <H> = eta = sum_k w_k <H>_k over the given grid, width 1 (so J is the
// frequency-integrated mean intensity) and no frequency step.
void build_tables(const std::vector<double>& edges, double T, double dx, int gray, int recoil,
                  BinTables* t, int geometry) {
  const int n = static_cast<int>(edges.size()) - 1;
  const LineConstants lc = line_constants(T);
  std::vector<double> dnu(n), nubar(n), Hv(n), w(n);
  double S = 0.0;
  for (int k = 0; k < n; ++k) {
    dnu[k] = edges[k + 1] - edges[k];
    nubar[k] = kNuLya + 0.5 * (edges[k] + edges[k + 1]);
    const double xa = edges[k] / lc.dnu_D, xb = edges[k + 1] / lc.dnu_D;
    const double dxk = dnu[k] / lc.dnu_D;
    Hv[k] = bin_voigt(xa, xb, lc.a_v, dxk);
    w[k] = Hv[k] * dxk;
    S += w[k];
  }
  double eta = 0.0;
  for (int k = 0; k < n; ++k) {
    w[k] = w[k] / S;
    eta += w[k] * Hv[k];
  }
  t->lc = lc;
  t->eta = eta;
  t->hkT = kPlanck / (kBoltzmann * T);
  const double V = geometry == 1 ? 1.0 : (dx * dx) * dx;
  const double fourpiV = (4.0 * kPi) * V;
  const int nb = gray ? 1 : n;
  t->nb = nb;
  t->dnu.assign(nb, 0.0);
  t->nubar.assign(nb, 0.0);
  t->Havg.assign(nb, 0.0);
  t->gem.assign(nb, 0.0);
  t->Rk.assign(nb, 0.0);
  t->half.assign(nb, 0.0);
  t->nubar_c.assign(nb, 0.0);
  if (gray) {
    t->dnu[0] = 1.0;
    t->nubar[0] = kNuLya;
    t->Havg[0] = eta;
    t->gem[0] = 1.0 / fourpiV;
    t->half[0] = 0.5;
    t->nubar_c[0] = kNuLya / kLight;
    return;
  }
  for (int k = 0; k < n; ++k) {
    t->dnu[k] = dnu[k];
    t->nubar[k] = nubar[k];
    t->Havg[k] = Hv[k];
    t->gem[k] = w[k] / (fourpiV * dnu[k]);
    t->Rk[k] = recoil ? (t->hkT - 2.0 / nubar[k]) : 0.0;
    t->half[k] = 0.5 * dnu[k];
    t->nubar_c[k] = nubar[k] / kLight;
  }
}

}  // namespace lym1

namespace lym1 {

// Axisymmetric finite-volume geometry, per radian (cells [i dx, (i+1) dx] in R).
void build_cyl_tables(int nx, double dx, CylTables* g) {
  g->AR.assign(nx + 1, 0.0);
  g->dlL.assign(nx + 1, 0.0);
  g->dlR.assign(nx + 1, 0.0);
  g->AZ.assign(nx, 0.0);
  g->Vol.assign(nx, 0.0);
  g->invR.assign(nx, 0.0);
  g->V2pi.assign(nx, 0.0);
  g->wv.assign(nx, 0.0);
  std::vector<double> Rbar(nx);
  const double dx3 = (dx * dx) * dx;
  for (int i = 0; i < nx; ++i) {
    const double Rm = i * dx, Rp = (i + 1) * dx;
    g->AZ[i] = 0.5 * (Rp * Rp - Rm * Rm);
    g->Vol[i] = g->AZ[i] * dx;
    // centroid of the annulus: int R^2 dR / int R dR
    Rbar[i] = (2.0 / 3.0) * ((Rp * Rp * Rp - Rm * Rm * Rm) / (Rp * Rp - Rm * Rm));
    g->invR[i] = (dx * dx) / g->Vol[i];
    g->V2pi[i] = (2.0 * kPi) * g->Vol[i];
    g->wv[i] = g->V2pi[i] / dx3;
  }
  for (int i = 0; i <= nx; ++i) {
    const double Rf = i * dx;
    g->AR[i] = Rf * dx;
    const double left = (i == 0) ? -Rbar[0] : Rbar[i - 1];
    const double right = (i == nx) ? Rbar[nx - 1] + dx : Rbar[i];
    g->dlL[i] = Rf - left;
    g->dlR[i] = right - Rf;
  }
  g->wR = (2.0 * kPi) * g->AR[nx] / (dx * dx);
  g->r0.resize(nx);
  g->r1.resize(nx);
  g->hoop.resize(nx);
  g->fwv.resize(nx);
  g->fdlL.resize(nx + 1);
  g->fdlR.resize(nx + 1);
  for (int i = 0; i < nx; ++i) {
    g->r0[i] = static_cast<float>(g->AR[i] * dx / g->Vol[i]);
    g->r1[i] = static_cast<float>(g->AR[i + 1] * dx / g->Vol[i]);
    g->hoop[i] = static_cast<float>(g->invR[i] * dx);
    g->fwv[i] = static_cast<float>(g->wv[i]);
  }
  for (int i = 0; i <= nx; ++i) {
    g->fdlL[i] = static_cast<float>(g->dlL[i]);
    g->fdlR[i] = static_cast<float>(g->dlR[i]);
  }
}

}  // namespace lym1

namespace lym1 {

void build_cell_tables(const std::vector<double>& edges, const double* T, long long nc, double dx,
                       int gray, int recoil, int geometry, CellTables* out) {
  // distinct temperatures, by bit pattern
  std::unordered_map<unsigned long long, int> index;
  std::vector<double> uniq;
  std::vector<int> which(static_cast<size_t>(nc));
  for (long long i = 0; i < nc; ++i) {
    unsigned long long key;
    std::memcpy(&key, &T[i], sizeof key);
    auto it = index.find(key);
    if (it == index.end()) {
      it = index.emplace(key, static_cast<int>(uniq.size())).first;
      uniq.push_back(T[i]);
    }
    which[static_cast<size_t>(i)] = it->second;
  }
  std::vector<BinTables> tabs(uniq.size());
  unsigned nt = std::thread::hardware_concurrency();
  if (nt < 1) nt = 1;
  if (nt > uniq.size()) nt = static_cast<unsigned>(uniq.size());
  std::vector<std::thread> pool;
  for (unsigned t = 0; t < nt; ++t)
    pool.emplace_back([&, t]() {
      for (size_t u = t; u < uniq.size(); u += nt)
        build_tables(edges, uniq[u], dx, gray, recoil, &tabs[u], geometry);
    });
  for (auto& th : pool) th.join();
  const int nb = tabs.empty() ? 0 : tabs[0].nb;
  const size_t n = static_cast<size_t>(nc);
  out->H.assign(static_cast<size_t>(nb) * n, 0.0);
  out->G.assign(static_cast<size_t>(nb) * n, 0.0);
  out->sigma0.assign(n, 0.0);
  out->hkT.assign(n, 0.0);
  out->Kc.assign(n, 0.0);
  out->gmax.assign(n, 0.0);
  std::vector<double> gm(uniq.size(), 0.0);
  for (size_t u = 0; u < uniq.size(); ++u)
    for (double g : tabs[u].gem) gm[u] = std::max(gm[u], g);
  for (size_t i = 0; i < n; ++i) {
    const BinTables& t = tabs[static_cast<size_t>(which[i])];
    for (int k = 0; k < nb; ++k) {
      out->H[static_cast<size_t>(k) * n + i] = t.Havg[k];
      out->G[static_cast<size_t>(k) * n + i] = t.gem[k];
    }
    out->sigma0[i] = t.lc.sigma0;
    out->hkT[i] = t.hkT;
    out->Kc[i] = 0.5 * (t.lc.dnu_D * t.lc.dnu_D);
    out->gmax[i] = gm[static_cast<size_t>(which[i])] > 0.0 ? gm[static_cast<size_t>(which[i])] : 1.0;
  }
}

}  // namespace lym1
