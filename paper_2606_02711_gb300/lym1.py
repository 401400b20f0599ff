"""Thin ctypes binding of ``include/lym1.h`` (argument marshalling only).

Every step of the substep runs in the CUDA library ``liblym1.so``; this module
only converts Python arguments into the C structs and pointers.  Host arrays
are numpy float64 arrays; device buffers are CUDA ``torch.Tensor``s (float64,
contiguous), whose data pointers are passed straight through.  Streams may be
given as ``torch.cuda.Stream`` objects.  The module raises if the library has
not been built; it has no other code path.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblym1.so")

OK, EINVAL, ENOMEM, ECUDA, ENONFINITE, ETIMEOUT, ENOTCONVERGED, ENODEVICE = 0, -1, -2, -3, -4, -5, -6, -7
ERANGE = -8
FP64_DET, FP64, MIXED, MIXED_FAST = 0, 1, 2, 3
PRECISIONS = {"fp64_det": FP64_DET, "fp64": FP64, "mixed": MIXED, "mixed_fast": MIXED_FAST}

_PD = C.POINTER(C.c_double)


class Lym1Error(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {strerror(status)} ({status})")


class lym1_grid(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("dx_cm", C.c_double), ("geometry", C.c_int),
                ("bc", C.c_int * 4)]


class lym1_groups(C.Structure):
    _fields_ = [("n_bins", C.c_int), ("edges_dnu_hz", _PD), ("q", C.c_double),
                ("T_min", C.c_double), ("gray", C.c_int)]


class lym1_opacities(C.Structure):
    _fields_ = [("n_hi", _PD), ("rho_dust", _PD), ("p_d", _PD), ("ux", _PD), ("uy", _PD),
                ("temp_K", C.c_double), ("kappa_abs", C.c_double), ("kappa_F", C.c_double),
                ("c_tilde", C.c_double), ("cfl", C.c_double), ("recoil", C.c_int),
                ("freq_step", C.c_int), ("precision", C.c_int), ("cuda_stream", C.c_void_p),
                ("temp_field", _PD)]


class lym1_info(C.Structure):
    _fields_ = [("nb", C.c_int), ("precision", C.c_int), ("dt_cfl", C.c_double),
                ("eta", C.c_double), ("dnu_D", C.c_double), ("a_v", C.c_double),
                ("sigma0", C.c_double), ("bytes_per_substep", C.c_double),
                ("device_bytes", C.c_double), ("substeps_done", C.c_longlong)]


class lym1_diag(C.Structure):
    _fields_ = [("e_tot", C.c_double), ("emitted", C.c_double), ("absorbed", C.c_double),
                ("outflow", C.c_double), ("work", C.c_double), ("residual", C.c_double),
                ("e_start", C.c_double), ("max_f", C.c_double), ("n_unrealisable", C.c_double),
                ("force_abs", C.c_double), ("force_radial", C.c_double), ("M_F", C.c_double),
                ("M_F_radial", C.c_double), ("f_esc", C.c_double), ("L_tot", C.c_double),
                ("substeps", C.c_longlong)]


class lym1_bands(C.Structure):
    _fields_ = [("n_bands", C.c_int), ("alpha_F", _PD), ("kappa", _PD), ("emissivity", _PD)]


class lym1_profile(C.Structure):
    _fields_ = [("transport_ms", C.c_double), ("freq_ms", C.c_double),
                ("finalize_ms", C.c_double), ("transport_launches", C.c_longlong),
                ("freq_launches", C.c_longlong), ("finalize_launches", C.c_longlong)]


_lib = None

# every symbol the header declares, with its ctypes signature
SIGNATURES = {
    "lym1_strerror": (C.c_char_p, [C.c_int]),
    "lym1_spectrum_enable": (C.c_int, [C.c_void_p, C.c_int]),
    "lym1_spectrum_read": (C.c_int, [C.c_void_p, _PD, C.POINTER(C.c_int)]),
    "lym1_set_ctilde": (C.c_int, [C.c_void_p, C.c_double]),
    "lym1_create_bands": (C.c_int, [C.POINTER(lym1_grid), C.POINTER(lym1_bands), _PD, _PD,
                                    C.c_double, C.c_double, C.c_int, C.c_void_p,
                                    C.POINTER(C.c_void_p)]),
    "lym1_bands_update": (C.c_int, [C.c_void_p, _PD, _PD, _PD]),
    "lym1_set_temperature": (C.c_int, [C.c_void_p, _PD]),
    "lym1_set_pruning": (C.c_int, [C.c_void_p, C.c_double]),
    "lym1_set_accept": (C.c_int, [C.c_void_p, C.c_int]),
    "lym1_dynamic_ctilde": (C.c_int, [C.c_void_p, _PD, C.c_double, C.c_double, _PD]),
    "lym1_create": (C.c_int, [C.POINTER(lym1_grid), C.POINTER(lym1_groups),
                              C.POINTER(lym1_opacities), C.POINTER(C.c_void_p)]),
    "lym1_destroy": (None, [C.c_void_p]),
    "lym1_set_sources": (C.c_int, [C.c_void_p, _PD]),
    "lym1_set_state": (C.c_int, [C.c_void_p, _PD, _PD, _PD]),
    "lym1_get_state": (C.c_int, [C.c_void_p, _PD, _PD, _PD]),
    "lym1_state_elem_size": (C.c_int, [C.c_void_p, C.POINTER(C.c_int)]),
    "lym1_get_rows": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p]),
    "lym1_set_rows": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p]),
    "lym1_substeps": (C.c_int, [C.c_void_p, C.c_int, C.c_double]),
    "lym1_step": (C.c_int, [C.c_void_p, C.c_double, C.POINTER(C.c_int)]),
    "lym1_moments": (C.c_int, [C.c_void_p, _PD, _PD, _PD]),
    "lym1_force": (C.c_int, [C.c_void_p, _PD, _PD]),
    "lym1_diagnostics": (C.c_int, [C.c_void_p, C.POINTER(lym1_diag)]),
    "lym1_get_info": (C.c_int, [C.c_void_p, C.POINTER(lym1_info)]),
    "lym1_plan_bytes": (C.c_int, [C.POINTER(lym1_grid), C.POINTER(lym1_groups), C.c_int, C.c_int,
                                  _PD]),
    "lym1_tables": (C.c_int, [C.c_void_p, _PD, _PD, _PD, _PD]),
    "lym1_synchronize": (C.c_int, [C.c_void_p]),
    "lym1_run_to_steady": (C.c_int, [C.c_void_p, C.c_double, C.c_int, C.c_int,
                                     C.POINTER(C.c_int)]),
    "lym1_substeps_batched": (C.c_int, [C.POINTER(C.c_void_p), C.c_int, C.c_int]),
    "lym1_profile_enable": (C.c_int, [C.c_void_p, C.c_int]),
    "lym1_profile_read": (C.c_int, [C.c_void_p, C.POINTER(lym1_profile), C.c_int]),
    "lym1_batch_create": (C.c_int, [C.POINTER(C.c_void_p), C.c_int, C.POINTER(C.c_void_p)]),
    "lym1_batch_substeps": (C.c_int, [C.c_void_p, C.c_int]),
    "lym1_batch_grid": (C.c_int, [C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    "lym1_batch_config": (C.c_int, [C.c_void_p] + [C.POINTER(C.c_int)] * 5),
    "lym1_batch_configure": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_int]),
    "lym1_batch_destroy": (None, [C.c_void_p]),
    "lym1_debug_expire_wait": (C.c_int, [C.c_void_p]),
    "lym1_debug_fp64_helpers": (C.c_int, [C.c_void_p, C.c_void_p, C.c_longlong, C.c_void_p,
                                          C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "lym1_energy_noalloc": (C.c_int, [_PD, _PD, C.c_int, C.c_longlong, C.c_double, _PD,
                                      C.c_void_p]),
}


def lib():
    """The loaded CUDA library; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "paper_2606_02711_gb300.build.build() (needs nvcc)")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def strerror(status: int) -> str:
    return lib().lym1_strerror(int(status)).decode()


def _check(status: int, where: str) -> int:
    if status != OK:
        raise Lym1Error(status, where)
    return status


def _ptr(a, keep: list):
    """Pointer to a float64 host array (numpy) or device tensor (torch)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):  # torch tensor, any device
        if str(a.dtype) != "torch.float64" or not a.is_contiguous():
            raise TypeError("tensor buffers must be contiguous float64")
        keep.append(a)
        return C.cast(C.c_void_p(a.data_ptr()), _PD)
    arr = np.ascontiguousarray(a, dtype=np.float64)
    keep.append(arr)
    return arr.ctypes.data_as(_PD)


def _out_ptr(a):
    if hasattr(a, "data_ptr"):
        if str(a.dtype) != "torch.float64" or not a.is_contiguous():
            raise TypeError("tensor buffers must be contiguous float64")
        return C.cast(C.c_void_p(a.data_ptr()), _PD)
    if not (isinstance(a, np.ndarray) and a.dtype == np.float64 and a.flags.c_contiguous
            and a.flags.writeable):
        raise TypeError("output arrays must be writable C-contiguous float64")
    return a.ctypes.data_as(_PD)


def _stream_handle(stream):
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return C.c_void_p(stream.cuda_stream)
    return C.c_void_p(int(stream))


class Context:
    """One lym1 context (``lym1_create`` ... ``lym1_destroy``)."""

    def __init__(self, *, nx, ny, dx, n_hi, rho_d, p_d, ux, uy, T=1e4, kappa_abs=0.0,
                 kappa_F=0.0, c_tilde=0.0, cfl=0.0, recoil=True, freq_step=True, gray=False,
                 edges=None, q=0.0, T_min=0.0, precision=FP64_DET, stream=None, lum=None,
                 geometry=0, bc=(0, 0, 0, 0), temp=None):
        keep = []
        if isinstance(precision, str):
            precision = PRECISIONS[precision]
        g = lym1_grid(int(nx), int(ny), float(dx), int(geometry),
                      (C.c_int * 4)(*[int(b) for b in bc]))
        if edges is not None:
            e = np.ascontiguousarray(edges, dtype=np.float64)
            keep.append(e)
            gr = lym1_groups(e.size - 1, e.ctypes.data_as(_PD), float(q), float(T_min), int(gray))
        else:
            gr = lym1_groups(0, None, float(q), float(T_min), int(gray))

        def field(a):
            if hasattr(a, "data_ptr"):
                return _ptr(a, keep)
            return _ptr(np.broadcast_to(np.asarray(a, dtype=np.float64), (ny, nx)), keep)

        op = lym1_opacities(field(n_hi), field(rho_d), field(p_d), field(ux), field(uy), float(T),
                            float(kappa_abs), float(kappa_F), float(c_tilde), float(cfl),
                            int(bool(recoil)), int(bool(freq_step)), int(precision),
                            _stream_handle(stream), field(temp) if temp is not None else None)
        h = C.c_void_p()
        _check(lib().lym1_create(C.byref(g), C.byref(gr), C.byref(op), C.byref(h)), "lym1_create")
        self.handle = h
        self.nx, self.ny = int(nx), int(ny)
        inf = self.info()
        self.nb = inf["nb"]
        self.dt_cfl = inf["dt_cfl"]
        self.precision = int(precision)
        if lum is not None:
            self.set_sources(lum)

    @classmethod
    def for_bands(cls, *, nx, ny, dx, alpha_F, kappa, emissivity, ux=0.0, uy=0.0, c_tilde=0.0,
                  cfl=0.0, precision=FP64_DET, stream=None, geometry=0, bc=(0, 0, 0, 0)):
        """``lym1_create_bands``: broad bands with per-[band][cell] flux opacity,
        absorption opacity (cm^-1) and emissivity (erg/s/cm^3/sr)."""
        keep = []
        if isinstance(precision, str):
            precision = PRECISIONS[precision]
        nb = int(np.shape(alpha_F)[0])
        g = lym1_grid(int(nx), int(ny), float(dx), int(geometry),
                      (C.c_int * 4)(*[int(b) for b in bc]))

        def arr(a, shape):
            if hasattr(a, "data_ptr"):
                return _ptr(a, keep)
            return _ptr(np.broadcast_to(np.asarray(a, dtype=np.float64), shape), keep)

        bs = (nb, int(ny), int(nx))
        b = lym1_bands(nb, arr(alpha_F, bs), arr(kappa, bs), arr(emissivity, bs))
        h = C.c_void_p()
        _check(lib().lym1_create_bands(C.byref(g), C.byref(b), arr(ux, bs[1:]), arr(uy, bs[1:]),
                                       float(c_tilde), float(cfl), int(precision),
                                       _stream_handle(stream), C.byref(h)), "lym1_create_bands")
        self = cls.__new__(cls)
        self.handle = h
        self.nx, self.ny = int(nx), int(ny)
        inf = self.info()
        self.nb = inf["nb"]
        self.dt_cfl = inf["dt_cfl"]
        self.precision = int(precision)
        return self

    def set_pruning(self, cut: float = 1e-10):
        """``lym1_set_pruning``: advect only bins above cut of the energy (0: all)."""
        _check(lib().lym1_set_pruning(self.handle, float(cut)), "lym1_set_pruning")

    def set_accept(self, on: bool = True):
        """``lym1_set_accept``: the substep acceptance rule of step 2 (Sec. 2.1)."""
        _check(lib().lym1_set_accept(self.handle, int(bool(on))), "lym1_set_accept")

    def set_temperature(self, temp):
        """``lym1_set_temperature``: per-cell tables for new gas temperatures."""
        keep = []
        if not hasattr(temp, "data_ptr"):
            temp = np.broadcast_to(np.asarray(temp, dtype=np.float64), (self.ny, self.nx))
        _check(lib().lym1_set_temperature(self.handle, _ptr(temp, keep)), "lym1_set_temperature")

    def bands_update(self, alpha_F, kappa, emissivity):
        """``lym1_bands_update``: new per-[band][cell] opacities and emissivity."""
        keep = []
        bs = (self.nb, self.ny, self.nx)

        def arr(a):
            if hasattr(a, "data_ptr"):
                return _ptr(a, keep)
            return _ptr(np.broadcast_to(np.asarray(a, dtype=np.float64), bs), keep)

        _check(lib().lym1_bands_update(self.handle, arr(alpha_F), arr(kappa), arr(emissivity)),
               "lym1_bands_update")

    # lifetime ------------------------------------------------------------
    def destroy(self):
        if getattr(self, "handle", None):
            lib().lym1_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.destroy()

    # calls ---------------------------------------------------------------
    def set_sources(self, lum):
        keep = []
        if not hasattr(lum, "data_ptr"):
            lum = np.broadcast_to(np.asarray(lum, dtype=np.float64), (self.ny, self.nx))
        _check(lib().lym1_set_sources(self.handle, _ptr(lum, keep)), "lym1_set_sources")

    def set_state(self, J, Hx, Hy):
        keep = []
        _check(lib().lym1_set_state(self.handle, _ptr(J, keep), _ptr(Hx, keep), _ptr(Hy, keep)),
               "lym1_set_state")

    def get_state(self, out=None):
        shape = (self.nb, self.ny, self.nx)
        J, Hx, Hy = out if out is not None else (np.empty(shape), np.empty(shape), np.empty(shape))
        _check(lib().lym1_get_state(self.handle, _out_ptr(J), _out_ptr(Hx), _out_ptr(Hy)),
               "lym1_get_state")
        return J, Hx, Hy

    def state_itemsize(self) -> int:
        """Bytes per state element: 4 under the mixed policies, 8 under the FP64 ones."""
        b = C.c_int()
        _check(lib().lym1_state_elem_size(self.handle, C.byref(b)), "lym1_state_elem_size")
        return b.value

    def _row_ptrs(self, arrays, n, writable):
        """Pointers to three [nb][n][nx] arrays (numpy) or tensors (torch, any
        device) of the state's element type, contiguous."""
        size = self.state_itemsize()
        want = np.float32 if size == 4 else np.float64
        ptrs = []
        for a in arrays:
            if hasattr(a, "data_ptr"):
                if a.element_size() != size or not a.is_floating_point() or not a.is_contiguous():
                    raise TypeError(f"row buffers must be contiguous {np.dtype(want).name} tensors")
                if a.numel() != self.nb * n * self.nx:
                    raise ValueError("row buffers must hold nb * n_rows * nx elements")
                ptrs.append(C.c_void_p(a.data_ptr()))
            else:
                if not (isinstance(a, np.ndarray) and a.dtype == want and a.flags.c_contiguous
                        and (a.flags.writeable or not writable)):
                    raise TypeError(f"row arrays must be C-contiguous {np.dtype(want).name}")
                if a.size != self.nb * n * self.nx:
                    raise ValueError("row arrays must hold nb * n_rows * nx elements")
                ptrs.append(C.c_void_p(a.ctypes.data))
        return ptrs

    def get_rows(self, y0, n, out=None):
        """Rows [y0, y0 + n) of J, Hx, Hy ([nb][n][nx] each) in the state's own
        element type, into ``out`` (three arrays or tensors, host or device) or
        new numpy arrays; the copies are complete when this returns."""
        if out is None:
            dt = np.float32 if self.state_itemsize() == 4 else np.float64
            out = tuple(np.empty((self.nb, int(n), self.nx), dtype=dt) for _ in range(3))
        p = self._row_ptrs(out, int(n), True)
        _check(lib().lym1_get_rows(self.handle, int(y0), int(n), *p), "lym1_get_rows")
        self.synchronize()
        return out

    def set_rows(self, y0, J, Hx, Hy):
        """Writes rows [y0, y0 + n) of the state from three [nb][n][nx] arrays or
        tensors of the state's element type; complete when this returns."""
        n = (J.numel() if hasattr(J, "numel") else J.size) // max(self.nb * self.nx, 1)
        p = self._row_ptrs((J, Hx, Hy), n, False)
        _check(lib().lym1_set_rows(self.handle, int(y0), int(n), *p), "lym1_set_rows")
        self.synchronize()

    def substeps(self, n, dt=0.0):
        _check(lib().lym1_substeps(self.handle, int(n), float(dt)), "lym1_substeps")

    def step(self, dt):
        n = C.c_int()
        _check(lib().lym1_step(self.handle, float(dt), C.byref(n)), "lym1_step")
        return n.value

    def moments(self, out=None):
        shape = (self.nb, self.ny, self.nx)
        E, Fx, Fy = out if out is not None else (np.empty(shape), np.empty(shape), np.empty(shape))
        _check(lib().lym1_moments(self.handle, _out_ptr(E), _out_ptr(Fx), _out_ptr(Fy)),
               "lym1_moments")
        return E, Fx, Fy

    def force(self, out=None):
        shape = (self.ny, self.nx)
        fx, fy = out if out is not None else (np.empty(shape), np.empty(shape))
        _check(lib().lym1_force(self.handle, _out_ptr(fx), _out_ptr(fy)), "lym1_force")
        return fx, fy

    def diagnostics(self, check=True) -> dict:
        d = lym1_diag()
        st = lib().lym1_diagnostics(self.handle, C.byref(d))
        if check:
            _check(st, "lym1_diagnostics")
        return {name: getattr(d, name) for name, _ in d._fields_}

    def spectrum_enable(self, on: bool = True):
        """Start (zeroed) or stop accumulating the emergent spectrum."""
        _check(lib().lym1_spectrum_enable(self.handle, int(bool(on))), "lym1_spectrum_enable")

    def spectrum(self) -> np.ndarray:
        """Escaping energy (erg) per [bin][outer face] since spectrum_enable."""
        nf = C.c_int()
        _check(lib().lym1_spectrum_read(self.handle, None, C.byref(nf)), "lym1_spectrum_read")
        out = np.empty((self.nb, nf.value))
        _check(lib().lym1_spectrum_read(self.handle, out.ctypes.data_as(_PD), C.byref(nf)),
               "lym1_spectrum_read")
        return out

    def set_ctilde(self, c_tilde: float):
        """Reduced speed of light (cm/s); the RT time step follows it."""
        _check(lib().lym1_set_ctilde(self.handle, float(c_tilde)), "lym1_set_ctilde")
        self.dt_cfl = self.info()["dt_cfl"]

    def dynamic_ctilde(self, cs=None, eps_rsl: float = 4.0, ct_min: float = 1.0e7) -> float:
        """Dynamic reduced speed of light (Sec. 2.1) from the context's fields;
        cs: per-cell sound speed (cm/s) or None for neutral gas at T.  Returns
        the new c_tilde."""
        keep = []
        p = None
        if cs is not None:
            if not hasattr(cs, "data_ptr"):
                cs = np.broadcast_to(np.asarray(cs, dtype=np.float64), (self.ny, self.nx))
            p = _ptr(cs, keep)
        out = C.c_double()
        _check(lib().lym1_dynamic_ctilde(self.handle, p, float(eps_rsl), float(ct_min),
                                         C.byref(out)), "lym1_dynamic_ctilde")
        self.dt_cfl = self.info()["dt_cfl"]
        return out.value

    def info(self) -> dict:
        i = lym1_info()
        _check(lib().lym1_get_info(self.handle, C.byref(i)), "lym1_get_info")
        return {name: getattr(i, name) for name, _ in i._fields_}

    def tables(self) -> dict:
        nb = self.info()["nb"]
        arrs = [np.empty(nb) for _ in range(4)]
        _check(lib().lym1_tables(self.handle, *[a.ctypes.data_as(_PD) for a in arrs]), "lym1_tables")
        return dict(zip(("dnu", "nubar", "Havg", "gem"), arrs))

    def synchronize(self):
        _check(lib().lym1_synchronize(self.handle), "lym1_synchronize")

    def synchronize_status(self) -> int:
        """``lym1_synchronize`` returning the status code instead of raising."""
        return lib().lym1_synchronize(self.handle)

    def debug_expire_wait(self):
        """Test hook: make the next frequency-step launch's bounded wait run out."""
        _check(lib().lym1_debug_expire_wait(self.handle), "lym1_debug_expire_wait")

    def profile_enable(self, on=True):
        _check(lib().lym1_profile_enable(self.handle, int(bool(on))), "lym1_profile_enable")

    def profile_read(self, reset=True) -> dict:
        p = lym1_profile()
        _check(lib().lym1_profile_read(self.handle, C.byref(p), int(bool(reset))),
               "lym1_profile_read")
        return {name: getattr(p, name) for name, _ in p._fields_}

    def run_to_steady(self, tol=1e-6, check_every=50, max_substeps=100000):
        """Returns (converged, substeps run)."""
        n = C.c_int()
        st = lib().lym1_run_to_steady(self.handle, float(tol), int(check_every),
                                      int(max_substeps), C.byref(n))
        if st == ENOTCONVERGED:
            return False, n.value
        _check(st, "lym1_run_to_steady")
        return True, n.value


def plan_bytes(nx, ny, precision, *, geometry=0, edges=None, q=0.0, T_min=0.0, gray=False,
               temp_field=False) -> float:
    """``lym1_plan_bytes``: device bytes a Lya context of this shape will
    allocate at creation (no CUDA call)."""
    if isinstance(precision, str):
        precision = PRECISIONS[precision]
    g = lym1_grid(int(nx), int(ny), 1.0, int(geometry), (C.c_int * 4)(0, 0, 0, 0))
    keep = None
    if edges is not None:
        keep = np.ascontiguousarray(edges, dtype=np.float64)
        gr = lym1_groups(keep.size - 1, keep.ctypes.data_as(_PD), float(q), float(T_min), int(gray))
    else:
        gr = lym1_groups(0, None, float(q), float(T_min), int(gray))
    out = C.c_double()
    _check(lib().lym1_plan_bytes(C.byref(g), C.byref(gr), int(precision), int(bool(temp_field)),
                                 C.byref(out)), "lym1_plan_bytes")
    del keep
    return out.value


def energy_noalloc(J, dnu, dx, stream=None) -> float:
    """``lym1_energy_noalloc``: Lya energy (erg) of a device state J[nb][ny][nx]
    (contiguous float64 CUDA tensor on the current device) with bin widths dnu
    (host), for callers that cannot allocate device memory at that point (their
    HBM is owned by another runtime's allocator, or their loop forbids
    allocation); the call itself allocates nothing."""
    d = np.ascontiguousarray(dnu, dtype=np.float64)
    nb = d.size
    if not getattr(J, "is_cuda", False):
        raise ValueError("energy_noalloc: J must be a CUDA tensor")
    import torch
    if J.device.index != torch.cuda.current_device():
        raise ValueError(f"energy_noalloc: J is on cuda:{J.device.index}, the current device "
                         f"is cuda:{torch.cuda.current_device()}")
    if J.dtype != torch.float64 or not J.is_contiguous():
        raise ValueError("energy_noalloc: J must be contiguous float64")
    if nb < 1 or J.numel() % nb != 0 or J.numel() == 0:
        raise ValueError(f"energy_noalloc: {J.numel()} values are not nb x nc with nb = {nb}")
    nc = J.numel() // nb
    out = np.zeros(1)
    _check(lib().lym1_energy_noalloc(_out_ptr(J), d.ctypes.data_as(_PD), nb, nc, float(dx),
                                     out.ctypes.data_as(_PD), _stream_handle(stream)),
           "lym1_energy_noalloc")
    return float(out[0])


class Batch:
    """``lym1_batch_*``: several contexts advanced by one graph-replayed set of
    persistent launches per substep.  Destroy it before its contexts."""

    def __init__(self, contexts):
        self.contexts = list(contexts)
        arr = (C.c_void_p * len(self.contexts))(*[c.handle.value for c in self.contexts])
        h = C.c_void_p()
        _check(lib().lym1_batch_create(arr, len(self.contexts), C.byref(h)), "lym1_batch_create")
        self.handle = h

    def substeps(self, n):
        _check(lib().lym1_batch_substeps(self.handle, int(n)), "lym1_batch_substeps")

    def grid(self):
        a, b = C.c_int(), C.c_int()
        _check(lib().lym1_batch_grid(self.handle, C.byref(a), C.byref(b)), "lym1_batch_grid")
        return a.value, b.value

    def config(self) -> dict:
        """``lym1_batch_config``: tile shape, bin groups and grids in use (0 until tuned)."""
        v = [C.c_int() for _ in range(5)]
        _check(lib().lym1_batch_config(self.handle, *[C.byref(x) for x in v]), "lym1_batch_config")
        return dict(zip(("tile_x", "tile_y", "bin_groups", "grid_t", "grid_f"), [x.value for x in v]))

    def configure(self, tile_shape=0, bin_groups=1, grid_t=0):
        """``lym1_batch_configure``: fix the transport layout instead of tuning it."""
        _check(lib().lym1_batch_configure(self.handle, int(tile_shape), int(bin_groups), int(grid_t)),
               "lym1_batch_configure")

    def destroy(self):
        if getattr(self, "handle", None):
            lib().lym1_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def substeps_batched(contexts, n):
    """``lym1_substeps_batched`` over a list of Context objects."""
    arr = (C.c_void_p * len(contexts))(*[c.handle.value for c in contexts])
    _check(lib().lym1_substeps_batched(arr, len(contexts), int(n)), "lym1_substeps_batched")


def from_cloud(cloud, precision=FP64_DET, stream=None, edges=None, q=0.0) -> Context:
    """A context for a ``workloads.Cloud`` with its sources set; edges None
    takes the paper grid with growth factor q (0: 1.1)."""
    return Context(nx=cloud.nx, ny=cloud.ny, dx=cloud.dx, n_hi=cloud.n_hi, rho_d=cloud.rho_d,
                   p_d=cloud.p_d, ux=cloud.ux, uy=cloud.uy, T=cloud.T, kappa_abs=cloud.kappa_abs,
                   kappa_F=cloud.kappa_F, c_tilde=cloud.c_tilde, cfl=cloud.cfl,
                   recoil=cloud.recoil, freq_step=cloud.freq_step, gray=cloud.gray, edges=edges,
                   precision=precision, stream=stream, lum=cloud.lum, q=q,
                   geometry=getattr(cloud, "geometry", 0), bc=getattr(cloud, "bc", (0, 0, 0, 0)),
                   temp=getattr(cloud, "temp", None))
