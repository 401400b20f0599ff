"""Seeded synthetic inputs for the Lya M1 substep: clouds shaped like the paper's setups.

This module is shared by the GPU path's tests/bench and by the oracle's tests.
It only draws and lays out input fields (densities, dust, velocities, sources);
it holds none of the M1 method's arithmetic.  All randomness comes from
numpy's counter-based Philox generator with an explicit seed.

Physical setup readings (each cites the paper, arXiv 2606.02711):
  * dust-to-gas: D/D_sun = Z/Z_sun with D_sun = 1/162 (Sec. 5 cluster setup and the
    dust-to-gas normalisation), gas mass density rho = 1.333 m_H n_H;
  * Lya dust opacities: mass-fraction-weighted Table 1 Lya row with f_Sil =
    0.7264, f_C = 0.2517, f_PAH = 0.0218 (Table 1 caption);
  * all hydrogen neutral (n_HI = n_H), T = 1e4 K;
  * a point source is spread equally over the central 2x2 cells;
  * velocity u = v_edge (r / r_edge) r_hat about the box centre.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

L_SUN = 3.828e33          # erg/s
PC = 3.0857e18            # cm
M_H = 1.67353284e-24      # g
KM = 1.0e5                # cm
C_LIGHT = 2.99792458e10   # cm/s

# Table 1, Lya row (cm^2 per g of dust in the bin) and dust mass fractions
_F_BIN = (0.7264, 0.2517, 0.0218)
_KABS = (1.84e4, 2.48e4, 3.31e5)
_KF = (2.22e4, 2.84e4, 3.31e5)
KAPPA_ABS = sum(f * k for f, k in zip(_F_BIN, _KABS))
KAPPA_F = sum(f * k for f, k in zip(_F_BIN, _KF))
DUST_TO_GAS_SUN = 1.0 / 162.0


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(int(seed)))


def gaussian_field(nx: int, ny: int, seed: int, slope: float = -4.0) -> np.ndarray:
    """Unit-variance Gaussian random field with 2D power spectrum P(k) ~ |k|^slope
    (k != 0), built by filtering seeded white noise with numpy's FFT."""
    g = rng(seed)
    white = g.standard_normal((ny, nx))
    Wk = np.fft.rfft2(white)
    ky = np.fft.fftfreq(ny)[:, None]
    kx = np.fft.rfftfreq(nx)[None, :]
    k2 = kx * kx + ky * ky
    amp = np.zeros_like(k2)
    amp[k2 > 0] = k2[k2 > 0] ** (slope / 4.0)   # sqrt(P) = |k|^(slope/2)
    f = np.fft.irfft2(Wk * amp, s=(ny, nx))
    f -= f.mean()
    sd = f.std()
    return f / sd if sd > 0 else f


def lognormal_density(nx, ny, mean, sigma_ln, seed) -> np.ndarray:
    """n = mean * exp(sigma g - sigma^2/2), rescaled to sample mean `mean`."""
    g = gaussian_field(nx, ny, seed)
    n = np.exp(sigma_ln * g - 0.5 * sigma_ln * sigma_ln)
    return n * (mean / n.mean())


def radial_velocity(nx, ny, dx, v_edge=10 * KM, r_edge=1.0 * PC):
    x = (np.arange(nx) + 0.5) * dx - 0.5 * nx * dx
    y = (np.arange(ny) + 0.5) * dx - 0.5 * ny * dx
    X, Y = np.meshgrid(x, y)
    s = v_edge / r_edge
    return s * X, s * Y


def central_source(nx, ny, L) -> np.ndarray:
    lum = np.zeros((ny, nx))
    i0, j0 = nx // 2 - 1, ny // 2 - 1
    lum[j0:j0 + 2, i0:i0 + 2] = L / 4.0
    return lum


def dust_density(n_h, Z_over_Zsun) -> np.ndarray:
    return (Z_over_Zsun * DUST_TO_GAS_SUN) * (1.333 * M_H) * n_h


@dataclass
class Cloud:
    """Inputs of one solve: grid, groups, opacities and sources."""
    name: str
    nx: int
    ny: int
    dx: float
    n_hi: np.ndarray
    rho_d: np.ndarray
    p_d: np.ndarray
    ux: np.ndarray
    uy: np.ndarray
    lum: np.ndarray
    T: float = 1.0e4
    gray: bool = False
    recoil: bool = True
    freq_step: bool = True
    kappa_abs: float = KAPPA_ABS
    kappa_F: float = KAPPA_F
    c_tilde: float = C_LIGHT
    cfl: float = 0.4
    substeps: int = 1
    geometry: int = 0        # 0: 2D Cartesian slab; 1: axisymmetric (R = x, Z = y)
    bc: tuple = (0, 0, 0, 0)  # x-, x+, y-, y+: 0 = zero-gradient outflow, 1 = vacuum outflow
    temp: object = None       # [ny][nx] gas temperature (K) per cell, or None for the uniform T
    meta: dict = field(default_factory=dict)

    @property
    def L_total(self) -> float:
        return float(self.lum.sum())

    def kwargs(self) -> dict:
        """Keyword arguments common to the oracle and the GPU binding."""
        return dict(nx=self.nx, ny=self.ny, dx=self.dx, T=self.T, n_hi=self.n_hi,
                    rho_d=self.rho_d, p_d=self.p_d, ux=self.ux, uy=self.uy, lum=self.lum,
                    kappa_abs=self.kappa_abs, kappa_F=self.kappa_F, c_tilde=self.c_tilde,
                    cfl=self.cfl, gray=self.gray, recoil=self.recoil,
                    freq_step=self.freq_step, geometry=self.geometry, bc=self.bc,
                    temp=self.temp)


def uniform_gray(nx=64, ny=64, box_pc=2.0, n_h=1e3, L_sun=1e6, name="uniform-gray"):
    """Static uniform neutral cloud, one gray group, central point source, no
    dust, no velocity, p_d = 0 (64x64, 2 pc, n_H = 1e3, 1e6 L_sun at full size)."""
    dx = box_pc * PC / nx
    z = np.zeros((ny, nx))
    return Cloud(name, nx, ny, dx, np.full((ny, nx), float(n_h)), z.copy(), z.copy(), z.copy(),
                 z.copy(), central_source(nx, ny, L_sun * L_SUN), gray=True, substeps=2000)


def lognormal_cloud(nx=512, ny=512, box_pc=2.0, mean_nh=1e3, sigma_ln=1.0, Z=0.01, L_sun=1e6,
                    seed=1, p_d=1e-12, v_edge_kms=10.0, name="lognormal", substeps=500):
    """Lognormal n_H (k^-4 spectrum), dust at Z/Z_sun, v ~ r with v_edge at 1 pc,
    central source, 194 frequency bins at T = 1e4 K."""
    dx = box_pc * PC / nx
    n_h = lognormal_density(nx, ny, mean_nh, sigma_ln, seed)
    ux, uy = radial_velocity(nx, ny, dx, v_edge_kms * KM, 1.0 * PC)
    return Cloud(name, nx, ny, dx, n_h, dust_density(n_h, Z), np.full((ny, nx), float(p_d)), ux,
                 uy, central_source(nx, ny, L_sun * L_SUN), substeps=substeps,
                 meta={"seed": seed, "sigma_ln": sigma_ln, "mean_nh": mean_nh, "Z": Z})


# Broad bands (Sec. 3): IR, optical, FUV, LW, EUV1, EUV2, EUV3.  Dust opacities of
# the non-IR bands from the dust-opacity table of Sec. 3 (kappa_abs, kappa_F in cm^2
# per g of dust in the bin, for silicate, graphite and PAH grains), weighted with
# the bin mass fractions of its caption.
BAND_NAMES = ("IR", "opt", "FUV", "LW", "EUV1", "EUV2", "EUV3")
_BAND_DUST = {
    "opt": ((5.98e3, 1.69e4), (2.09e4, 2.61e4), (2.27e5, 2.27e5)),
    "FUV": ((1.71e4, 2.21e4), (2.29e4, 2.57e4), (2.86e5, 2.86e5)),
    "LW": ((1.80e4, 2.18e4), (3.88e4, 4.48e4), (5.92e5, 5.92e5)),
    "EUV1": ((1.53e4, 1.85e4), (5.60e4, 6.22e4), (1.08e6, 1.08e6)),
    "EUV2": ((1.37e4, 1.46e4), (1.90e4, 2.12e4), (2.83e5, 2.84e5)),
    "EUV3": ((1.30e4, 1.32e4), (1.04e4, 1.09e4), (8.81e4, 8.82e4)),
}
# stand-ins where the paper gives no number: the IR Planck-mean dust opacity
# (shown only as a figure) and the H I photoionisation cross-section of the EUV
# bands (hydrogenic 6.3e-18 cm^2 (E / 13.6 eV)^-3 at the band's mean energy)
KAPPA_IR = 5.0               # cm^2 per g of dust
_EUV_E = {"EUV1": 19.1, "EUV2": 39.5, "EUV3": 80.0}   # eV
SIGMA_SB = 5.670374419e-5    # erg cm^-2 s^-1 K^-4


def stellar_bands(cloud, T_dust=20.0, L_sun=None):
    """Per-[band][cell] flux opacity, absorption opacity (cm^-1) and emissivity
    (erg/s/cm^3/sr) of the seven bands for a cloud: dust in every band, neutral
    H I absorption in the EUV bands, the cloud's source luminosity split evenly
    over the six stellar bands, IR emission rho_d kappa_IR sigma T_d^4 / pi."""
    ny, nx = cloud.n_hi.shape
    rho, nh = cloud.rho_d, cloud.n_hi
    aF = np.zeros((7, ny, nx))
    ka = np.zeros((7, ny, nx))
    je = np.zeros((7, ny, nx))
    aF[0] = ka[0] = rho * KAPPA_IR
    V = cloud.dx ** 3
    lum = cloud.lum if L_sun is None else cloud.lum * (L_sun * L_SUN / cloud.lum.sum())
    for b, name in enumerate(BAND_NAMES[1:], start=1):
        kabs = sum(f * k[0] for f, k in zip(_F_BIN, _BAND_DUST[name]))
        kF = sum(f * k[1] for f, k in zip(_F_BIN, _BAND_DUST[name]))
        gas = 6.3e-18 * (13.6 / _EUV_E[name]) ** 3 * nh if name in _EUV_E else 0.0
        ka[b] = rho * kabs + gas
        aF[b] = rho * kF + gas
        je[b] = lum / 6.0 / (4.0 * math.pi * V)
    je[0] = rho * KAPPA_IR * SIGMA_SB * T_dust ** 4 / math.pi
    return aF, ka, je


def config_lognormal_512(seed=1):
    """512x512, 194 bins, sigma_ln = 1.0, mean n_H 1e3, Z = 0.01 Z_sun, 1e6 L_sun."""
    return lognormal_cloud(512, 512, mean_nh=1e3, sigma_ln=1.0, Z=0.01, L_sun=1e6, seed=seed,
                           name="lognormal-512", substeps=500)


def config_lognormal_2048(seed=1):
    """2048x2048, 194 bins, sigma_ln = 1.5, mean n_H 1e4, Z = 1e-3 Z_sun, 1e7 L_sun."""
    return lognormal_cloud(2048, 2048, mean_nh=1e4, sigma_ln=1.5, Z=1e-3, L_sun=1e7, seed=seed,
                           name="lognormal-2048", substeps=5000)


def batch_clouds(n=256, base_seed=1000, side_lo=64, side_hi=512, nh_lo=1e2, nh_hi=1e5,
                 bc=(0, 0, 0, 0)):
    """Independent clouds for a batched sweep: side log-uniform in
    [side_lo, side_hi] rounded to a multiple of 16, mean n_H log-uniform
    [nh_lo, nh_hi] (default [1e2, 1e5]), L log-uniform [1e4, 1e7] L_sun,
    Z in {0, 1e-3, 1e-2} Z_sun; bc: the outflow kind of the four sides
    (0 zero gradient, 1 into vacuum)."""
    g = rng(base_seed)
    out = []
    for i in range(n):
        side = int(round(math.exp(g.uniform(math.log(side_lo), math.log(side_hi))) / 16.0)) * 16
        side = max(16, side)
        mean = 10 ** g.uniform(math.log10(nh_lo), math.log10(nh_hi))
        L = 10 ** g.uniform(4, 7)
        Z = (0.0, 1e-3, 1e-2)[int(g.integers(0, 3))]
        c = lognormal_cloud(side, side, mean_nh=mean, sigma_ln=1.0, Z=Z, L_sun=L,
                            seed=base_seed + 1 + i, name=f"batch-{i}", substeps=1000)
        c.bc = tuple(bc)
        out.append(c)
    return out


def poisson_arrivals(n=1000, rate=50.0, seed=7):
    """Seeded Poisson arrival times (s) for a request stream."""
    g = rng(seed)
    return np.cumsum(g.exponential(1.0 / rate, size=n))


# Line-centre Lya cross-section at 1e4 K (cm^2), used only to turn a quoted
# optical depth into a density; it scales as T^-1/2 through the Doppler width.
SIGMA0_1E4K = 5.898e-14


def _sigma0(T: float) -> float:
    return SIGMA0_1E4K * math.sqrt(1.0e4 / T)


def _rz_grid(n, R_cl, extent=1.1):
    """Cell centres (R, Z) of an n x n axisymmetric grid covering [0, extent R_cl]^2."""
    dx = extent * R_cl / n
    c = (np.arange(n) + 0.5) * dx
    R, Z = np.meshgrid(c, c)          # [ny][nx]: Z rows, R columns
    vol = 2.0 * math.pi * 0.5 * (((np.arange(n) + 1) * dx) ** 2 - (np.arange(n) * dx) ** 2) * dx
    return dx, R, Z, np.broadcast_to(vol, (n, n))


def uniform_sphere(n=64, tau_cl=0.1, T=1.0e4, R_cl_pc=1.0, L_sun=1e6, gray=False, recoil=False,
                   freq_step=True, sigma0=None, name="uniform-sphere"):
    """Static dust-free uniform sphere in axisymmetric (R, Z) coordinates with
    the midplane mirrored (Sec. 4.1, Test 1): line-centre optical depth
    tau_cl = n_HI sigma0 R_cl inside r <= R_cl, vacuum outside, box 1.1 R_cl,
    emission uniform per unit volume inside the sphere (the upper half emits
    L/2 of a total L), c_tilde = c; vacuum outflow at the outer R and Z edges."""
    R_cl = R_cl_pc * PC
    dx, R, Z, vol = _rz_grid(n, R_cl)
    inside = np.sqrt(R * R + Z * Z) <= R_cl
    s0 = _sigma0(T) if sigma0 is None else sigma0
    n_hi = np.where(inside, tau_cl / (s0 * R_cl), 0.0)
    z = np.zeros((n, n))
    lum = np.where(inside, vol, 0.0)
    lum = lum * (0.5 * L_sun * L_SUN / lum.sum())
    return Cloud(name, n, n, dx, n_hi, z.copy(), z.copy(), z.copy(), z.copy(), lum, T=T, gray=gray,
                 recoil=recoil, freq_step=freq_step, kappa_abs=0.0, kappa_F=0.0, geometry=1,
                 bc=(0, 1, 0, 1), meta={"tau_cl": tau_cl, "R_cl": R_cl})


def cone_cloud(n=256, tau_cl=1e8, tau_cone=1e5, T=1.0e4, R_cl_pc=1.0, L_sun=1e6,
               mu_cone=1.0 / math.sqrt(2.0), dmu=0.025, eps_core=1e-4, sigma0=None,
               name="cone"):
    """Anisotropic escape test (Sec. 4.2, Test 6): a uniform sphere with a bipolar
    low-opacity cone about the Z axis.  n_H = n_cone + (n_cl - n_cone)/2
    [1 - tanh((mu - mu_cone)/dmu)], mu = |Z|/r; n_HI = eps n_H with eps = 1 in the
    shell 0.5 R_cl < r <= R_cl and eps_core inside 0.5 R_cl (the emission
    region, emitting uniformly per unit volume); vacuum outside R_cl; recoil
    on; no dust or destruction; static gas; 256^2 cells over 1.1 R_cl;
    n_cl, n_cone from tau = n sigma0 R_cl; vacuum outflow at the outer edges."""
    R_cl = R_cl_pc * PC
    dx, R, Z, vol = _rz_grid(n, R_cl)
    r = np.sqrt(R * R + Z * Z)
    mu = np.abs(Z) / r
    s0 = _sigma0(T) if sigma0 is None else sigma0
    n_cl, n_cn = tau_cl / (s0 * R_cl), tau_cone / (s0 * R_cl)
    n_h = n_cn + 0.5 * (n_cl - n_cn) * (1.0 - np.tanh((mu - mu_cone) / dmu))
    eps = np.where(r <= 0.5 * R_cl, eps_core, 1.0)
    n_hi = np.where(r <= R_cl, eps * n_h, 0.0)
    z = np.zeros((n, n))
    lum = np.where(r <= 0.5 * R_cl, vol, 0.0)
    lum = lum * (0.5 * L_sun * L_SUN / lum.sum())
    t_max = 4.0 * max((4.7e-4 * math.sqrt(1e4 / T) * tau_cl) ** (1.0 / 3.0), 3.0) * R_cl / C_LIGHT
    return Cloud(name, n, n, dx, n_hi, z.copy(), z.copy(), z.copy(), z.copy(), lum, T=T,
                 recoil=True, freq_step=True, kappa_abs=0.0, kappa_F=0.0, geometry=1,
                 bc=(0, 1, 0, 1), meta={"tau_cl": tau_cl, "tau_cone": tau_cone, "R_cl": R_cl, "t_max": t_max})


def two_phase_temperature(nx, ny, seed, T_cold=100.0, T_hot=1.0e4, frac_hot=0.5, smooth=True):
    """Seeded temperature field with warm and cold phases (K): a k^-4 Gaussian
    field thresholded at the quantile giving frac_hot of the cells the warm
    phase, with a log-linear transition of width ~0.3 sigma when smooth."""
    g = gaussian_field(nx, ny, seed)
    t = np.quantile(g, 1.0 - frac_hot)
    if smooth:
        s = 0.5 * (1.0 + np.tanh((g - t) / 0.3))
    else:
        s = (g > t).astype(float)
    return np.exp(np.log(T_cold) + s * (np.log(T_hot) - np.log(T_cold)))


def populated_state(cloud, nb, seed=11, ell_cells=24.0, f_out=0.4, x_peak=12.0, x_width=8.0,
                    J0=1e-12):
    """A smooth, realisable radiation state [nb][ny][nx] (J, Hx, Hy) shaped like the
    field around a central source, for tests that must not start from zero.

    Spectrum: a double peak in the bin index offset from line centre (the bins are
    ordered from the blue wing to the red wing, symmetric about nb/2), peaks at
    x_peak bins from the centre with width x_width, plus a 1e-6 floor.  Space: J
    falls as (1 + r/ell)^-2 from the box centre, modulated by 1 + 0.3 g with g a
    seeded smooth field in [-1, 1].  Flux: f = f_out tanh(r/ell) r_hat plus a
    seeded smooth perturbation of 0.2, capped at |f| = 0.95.  Only shapes are
    drawn here; no step of the method is computed."""
    nx, ny = cloud.nx, cloud.ny
    x = np.arange(nx) + 0.5 - 0.5 * nx
    y = np.arange(ny) + 0.5 - 0.5 * ny
    X, Y = np.meshgrid(x, y)
    r = np.sqrt(X * X + Y * Y)
    g = gaussian_field(nx, ny, seed)
    g = np.tanh(g)
    space = (1.0 + r / ell_cells) ** -2 * (1.0 + 0.3 * g)
    kk = np.arange(nb) + 0.5 - 0.5 * nb
    spec = np.exp(-((np.abs(kk) - x_peak) / x_width) ** 2) + 1e-6
    J = J0 * spec[:, None, None] * space[None, :, :]
    rs = np.maximum(r, 1e-12)
    fr = f_out * np.tanh(r / ell_cells)
    p1 = 0.2 * np.tanh(gaussian_field(nx, ny, seed + 1))
    p2 = 0.2 * np.tanh(gaussian_field(nx, ny, seed + 2))
    fx = fr * X / rs + p1
    fy = fr * Y / rs + p2
    fm = np.sqrt(fx * fx + fy * fy)
    sc = np.where(fm > 0.95, 0.95 / np.maximum(fm, 1e-300), 1.0)
    fx, fy = fx * sc, fy * sc
    return J, J * fx[None], J * fy[None]
