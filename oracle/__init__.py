"""Plain FP64 CPU oracle for the Lya M1 substep (arXiv 2606.02711, Sec. 2.1-2.3, App. A).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference arm of ``bench.py`` may import this package.  The
product path (``paper_2606_02711_gb300``) never imports it, and the two share
no code: this package wraps ``lym1_oracle.c`` (compiled with gcc,
``-ffp-contract=off``) through ctypes.

Every function here is argument marshalling; the arithmetic is in the C file,
which cites the paper passage each step follows.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import sys

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lym1_oracle.c")
_LIB = os.path.join(_HERE, "liblym1_oracle.so")


def build(force: bool = False) -> str:
    """Compile the oracle shared library with gcc (OpenMP if available)."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    base = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c11",
            "-shared", "-fPIC", _SRC, "-o", _LIB + ".tmp", "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True,
                       capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True)
    os.replace(_LIB + ".tmp", _LIB)
    return _LIB


_D = C.c_double
_PD = C.POINTER(C.c_double)


class Problem(C.Structure):
    """Mirror of ``lym1o_problem``."""
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nbins", C.c_int), ("gray", C.c_int),
                ("recoil", C.c_int), ("freq_step", C.c_int), ("dx", _D), ("T", _D),
                ("c_tilde", _D), ("cfl", _D), ("kappa_abs", _D), ("kappa_F", _D),
                ("edges", _PD), ("n_hi", _PD), ("rho_d", _PD), ("p_d", _PD),
                ("ux", _PD), ("uy", _PD), ("lum", _PD), ("geometry", C.c_int),
                ("bc", C.c_int * 4), ("temp", _PD), ("band_aF", _PD), ("band_kap", _PD),
                ("band_j", _PD), ("prune", C.c_double), ("accept", C.c_int)]


class Diag(C.Structure):
    """Mirror of ``lym1o_diag`` (energies in erg, force sums in dyn)."""
    _fields_ = [("e_before", _D), ("e_after", _D), ("emitted", _D), ("absorbed", _D),
                ("outflow", _D), ("work", _D), ("residual", _D), ("max_f", _D),
                ("n_unrealisable", _D), ("force_abs", _D), ("force_radial", _D)]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_}


_lib = None


def lib():
    global _lib
    if _lib is None:
        path = build()
        L = C.CDLL(path)
        L.lym1o_exp.restype = _D
        L.lym1o_exp.argtypes = [_D]
        L.lym1o_expm1.restype = _D
        L.lym1o_expm1.argtypes = [_D]
        L.lym1o_dawson.restype = _D
        L.lym1o_dawson.argtypes = [_D]
        L.lym1o_line.argtypes = [_D, _PD]
        L.lym1o_freq_grid.restype = C.c_int
        L.lym1o_freq_grid.argtypes = [_D, _D, _PD, C.c_int]
        L.lym1o_bin_tables.restype = _D
        L.lym1o_bin_tables.argtypes = [C.c_int, _PD, _D, _PD, _PD, _PD, _PD]
        L.lym1o_create.restype = C.c_void_p
        L.lym1o_create.argtypes = [C.POINTER(Problem)]
        L.lym1o_destroy.argtypes = [C.c_void_p]
        L.lym1o_dt_cfl.restype = _D
        L.lym1o_dt_cfl.argtypes = [C.c_void_p]
        L.lym1o_eta.restype = _D
        L.lym1o_eta.argtypes = [C.c_void_p]
        L.lym1o_nb.restype = C.c_int
        L.lym1o_nb.argtypes = [C.c_void_p]
        L.lym1o_tables.argtypes = [C.c_void_p, _PD, _PD, _PD, _PD]
        L.lym1o_closure.argtypes = [_D, _D, _PD]
        L.lym1o_eps.restype = _D
        L.lym1o_eps.argtypes = [_D]
        L.lym1o_face_flux.argtypes = [_PD, _PD, _PD, _D, _D, _D, _D, _D, _PD]
        L.lym1o_freq_solve.argtypes = [C.c_int, _PD, _D, _D, C.c_int, _PD, _D, _PD, _PD]
        L.lym1o_leakage.argtypes = [C.c_int, _PD, _D, _D, C.c_int, _PD, _PD, _PD]
        L.lym1o_energy.restype = _D
        L.lym1o_energy.argtypes = [C.c_void_p, _PD]
        L.lym1o_substep.restype = C.c_int
        L.lym1o_substep.argtypes = [C.c_void_p, _D, _PD, _PD, _PD, _PD, _PD, _PD, _PD, _PD,
                                    C.POINTER(Diag)]
        L.lym1o_set_threads.argtypes = [C.c_int]
        L.lym1o_set_spectrum.argtypes = [C.c_void_p, _PD]
        L.lym1o_set_subcycle_out.argtypes = [C.c_void_p, C.POINTER(C.c_int)]
        L.lym1o_set_ctilde.argtypes = [C.c_void_p, _D]
        L.lym1o_dynamic_ctilde.restype = _D
        L.lym1o_dynamic_ctilde.argtypes = [C.c_void_p, _PD, _D, _D]
        L.lym1o_get_threads.restype = C.c_int
        _lib = L
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(_PD)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


# ---------------------------------------------------------------- scalar helpers
def exp(x: float) -> float:
    return lib().lym1o_exp(float(x))


def expm1(x: float) -> float:
    return lib().lym1o_expm1(float(x))


def dawson(x: float) -> float:
    return lib().lym1o_dawson(float(x))


def line_constants(T: float) -> dict:
    out = np.zeros(3)
    lib().lym1o_line(float(T), _p(out))
    return {"dnu_D": out[0], "a_v": out[1], "sigma0": out[2]}


def freq_grid(T_min: float = 30.0, q: float = 1.1) -> np.ndarray:
    """Bin edges in dnu = nu - nu_Lya (Hz) of the paper's frequency grid."""
    buf = np.zeros(200001)
    n = lib().lym1o_freq_grid(float(T_min), float(q), _p(buf), buf.size)
    if n < 0:
        raise ValueError("frequency grid too large")
    return buf[: n + 1].copy()


def bin_tables(edges, T: float) -> dict:
    e = _f64(edges)
    n = e.size - 1
    dnu, nubar, Havg, w = (np.zeros(n) for _ in range(4))
    eta = lib().lym1o_bin_tables(n, _p(e), float(T), _p(dnu), _p(nubar), _p(Havg), _p(w))
    return {"dnu": dnu, "nubar": nubar, "Havg": Havg, "w": w, "eta": eta}


def closure(fx: float, fy: float) -> tuple:
    out = np.zeros(3)
    lib().lym1o_closure(float(fx), float(fy), _p(out))
    return tuple(out)


def eps(tau: float) -> float:
    return lib().lym1o_eps(float(tau))


def face_flux(J4, Hn4, Ht4, aF0, aF1, un0, un1, dx) -> np.ndarray:
    J4, Hn4, Ht4 = _f64(J4), _f64(Hn4), _f64(Ht4)
    out = np.zeros(3)
    lib().lym1o_face_flux(_p(J4), _p(Hn4), _p(Ht4), aF0, aF1, un0, un1, dx, _p(out))
    return out


def freq_solve(edges, T, alpha, recoil, DdU, cdt, Jin) -> np.ndarray:
    e = _f64(edges)
    n = e.size - 1
    d, j = _f64(np.broadcast_to(DdU, (n,))), _f64(Jin)
    out = np.zeros(n)
    lib().lym1o_freq_solve(n, _p(e), T, alpha, int(recoil), _p(d), cdt, _p(j), _p(out))
    return out


def leakage(edges, T, alpha, recoil, DdU) -> tuple:
    e = _f64(edges)
    n = e.size - 1
    d = _f64(np.broadcast_to(DdU, (n,)))
    A, B = np.zeros(n - 1), np.zeros(n - 1)
    lib().lym1o_leakage(n, _p(e), T, alpha, int(recoil), _p(d), _p(A), _p(B))
    return A, B


def set_threads(n: int) -> None:
    lib().lym1o_set_threads(int(n))


def get_threads() -> int:
    return lib().lym1o_get_threads()


# ---------------------------------------------------------------- full substeps
class Oracle:
    """One problem (grid, groups, opacities, sources) and its FP64 substep.

    Field arrays are [ny][nx]; state arrays are [nb][ny][nx] (J, Hx, Hy in
    erg cm^-2 s^-1 Hz^-1 sr^-1, or frequency-integrated for a gray group).
    """

    def __init__(self, *, nx, ny, dx, edges, T, n_hi, rho_d, p_d, ux, uy, lum,
                 kappa_abs=0.0, kappa_F=0.0, c_tilde=2.99792458e10, cfl=0.4,
                 gray=False, recoil=True, freq_step=True, geometry=0, bc=(0, 0, 0, 0),
                 temp=None, bands=None, prune=0.0, accept=False):
        bd = None
        if bands is not None:
            # (alpha_F, kappa, emissivity), each [n_bands][ny][nx]
            bd = [_f64(np.broadcast_to(a, np.shape(bands[0])[:1] + (ny, nx))) for a in bands]
            edges = np.arange(bd[0].shape[0] + 1, dtype=np.float64)
        self._keep = [_f64(edges)] + [_f64(np.broadcast_to(a, (ny, nx)))
                                      for a in (n_hi, rho_d, p_d, ux, uy, lum)]
        e, n_hi, rho_d, p_d, ux, uy, lum = self._keep
        tp = None
        if temp is not None:
            tp = _f64(np.broadcast_to(temp, (ny, nx)))
            self._keep.append(tp)
        if bd is not None:
            self._keep += bd
        self.nx, self.ny = int(nx), int(ny)
        self.prob = Problem(self.nx, self.ny, e.size - 1, int(gray), int(recoil), int(freq_step),
                            float(dx), float(T), float(c_tilde), float(cfl), float(kappa_abs),
                            float(kappa_F), _p(e), _p(n_hi), _p(rho_d), _p(p_d), _p(ux), _p(uy),
                            _p(lum), int(geometry), (C.c_int * 4)(*[int(b) for b in bc]),
                            _p(tp) if tp is not None else None,
                            *([_p(a) for a in bd] if bd is not None else [None, None, None]),
                            float(prune), int(bool(accept)))
        self.ctx = lib().lym1o_create(C.byref(self.prob))
        if not self.ctx:
            raise ValueError("invalid oracle problem")
        self.nb = lib().lym1o_nb(self.ctx)
        self.dt_cfl = lib().lym1o_dt_cfl(self.ctx)
        self.eta = lib().lym1o_eta(self.ctx)

    def __del__(self):
        ctx = getattr(self, "ctx", None)
        if ctx and lib is not None:
            try:
                lib().lym1o_destroy(ctx)
            except Exception:
                pass
            self.ctx = None

    def tables(self) -> dict:
        nb = self.nb
        dnu, nubar, Havg, gem = (np.zeros(nb) for _ in range(4))
        lib().lym1o_tables(self.ctx, _p(dnu), _p(nubar), _p(Havg), _p(gem))
        return {"dnu": dnu, "nubar": nubar, "Havg": Havg, "gem": gem}

    @classmethod
    def for_bands(cls, *, nx, ny, dx, alpha_F, kappa, emissivity, ux=0.0, uy=0.0,
                  c_tilde=2.99792458e10, cfl=0.4, geometry=0, bc=(0, 0, 0, 0)):
        """Broad-band problem (stellar / IR bands): per-[band][cell] flux
        opacity, absorption opacity (cm^-1) and emissivity (erg/s/cm^3/sr)."""
        z = np.zeros((ny, nx))
        return cls(nx=nx, ny=ny, dx=dx, edges=None, T=1e4, n_hi=z, rho_d=z, p_d=z, ux=ux, uy=uy,
                   lum=z, c_tilde=c_tilde, cfl=cfl, recoil=False, freq_step=False,
                   geometry=geometry, bc=bc, bands=(alpha_F, kappa, emissivity))

    def zero_state(self):
        s = (self.nb, self.ny, self.nx)
        return np.zeros(s), np.zeros(s), np.zeros(s)

    def energy(self, J) -> float:
        return lib().lym1o_energy(self.ctx, _p(_f64(J)))

    def n_faces(self) -> int:
        """Outer faces of the emergent spectrum (x-, x+, y-, y+; R and Z outer
        for the axisymmetric grid)."""
        g = self.prob.geometry
        return (self.nx + self.ny) if g == 1 else 2 * (self.nx + self.ny)

    def set_ctilde(self, ct: float):
        """Reduced speed of light (cm/s) and the RT time step with it."""
        lib().lym1o_set_ctilde(self.ctx, float(ct))
        self.dt_cfl = lib().lym1o_dt_cfl(self.ctx)

    def dynamic_ctilde(self, cs=None, eps_rsl=4.0, ct_min=1.0e7) -> float:
        """Apply the dynamic reduced speed of light; returns the new value."""
        buf = None
        if cs is not None:
            buf = _f64(np.broadcast_to(cs, (self.ny, self.nx)))
        ct = lib().lym1o_dynamic_ctilde(self.ctx, _p(buf) if buf is not None else None,
                                        float(eps_rsl), float(ct_min))
        self.dt_cfl = lib().lym1o_dt_cfl(self.ctx)
        return ct

    def spectrum_on(self, on: bool = True):
        """Record the emergent spectrum (erg per [bin][face]) of each substep
        in self.spectrum."""
        if on:
            self.spectrum = np.zeros((self.nb, self.n_faces()))
            lib().lym1o_set_spectrum(self.ctx, _p(self.spectrum))
        else:
            lib().lym1o_set_spectrum(self.ctx, None)
            self.spectrum = None

    def subcycle_on(self, on: bool = True):
        """Record, per cell, the accepted step-2 substeps of each substep in
        self.nsub (only with accept=True)."""
        if on:
            self.nsub = np.zeros((self.ny, self.nx), dtype=np.int32)
            lib().lym1o_set_subcycle_out(self.ctx, self.nsub.ctypes.data_as(C.POINTER(C.c_int)))
        else:
            lib().lym1o_set_subcycle_out(self.ctx, None)
            self.nsub = None

    def substep(self, J, Hx, Hy, dt=None):
        """Advance one substep; returns (J, Hx, Hy, fx, fy, diag dict)."""
        dt = self.dt_cfl if dt is None else float(dt)
        J, Hx, Hy = _f64(J), _f64(Hx), _f64(Hy)
        Jo, Hxo, Hyo = np.empty_like(J), np.empty_like(J), np.empty_like(J)
        fx, fy = np.zeros((self.ny, self.nx)), np.zeros((self.ny, self.nx))
        d = Diag()
        rc = lib().lym1o_substep(self.ctx, dt, _p(J), _p(Hx), _p(Hy), _p(Jo), _p(Hxo), _p(Hyo),
                                 _p(fx), _p(fy), C.byref(d))
        if rc != 0:
            raise RuntimeError(f"oracle substep failed ({rc})")
        return Jo, Hxo, Hyo, fx, fy, d.as_dict()

    def run(self, nsteps, state=None, dt=None):
        """Advance nsteps substeps from state (default zero); returns final
        (J, Hx, Hy, fx, fy) and the list of per-substep diagnostics."""
        J, Hx, Hy = state if state is not None else self.zero_state()
        fx = fy = None
        diags = []
        for _ in range(int(nsteps)):
            J, Hx, Hy, fx, fy, d = self.substep(J, Hx, Hy, dt)
            diags.append(d)
        return (J, Hx, Hy, fx, fy), diags


if __name__ == "__main__":
    build(force="--force" in sys.argv)
    print(_LIB)
