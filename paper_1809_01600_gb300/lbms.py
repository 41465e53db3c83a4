"""Python binding of the C ABI in ``include/lbms.h`` (ctypes, marshalling only).

Every step of the solver runs in the CUDA library ``_build/liblbms.so``;
this module only converts arguments.  PyTorch, when present, supplies the
device allocator (its caching allocator) and the current CUDA stream.
Loading fails loudly when the library is missing or cannot be built: there
is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

LBMS_OK, LBMS_EINVAL, LBMS_ENOMEM, LBMS_ECUDA, LBMS_ENOTCONVERGED, LBMS_EUNSTABLE, \
    LBMS_EDEPLETED, LBMS_ESTATE = range(8)
LBMS_FP64, LBMS_FP32, LBMS_FP16 = 0, 1, 2
LBMS_COUPLING_MS, LBMS_COUPLING_TAU_ONLY = 0, 1
LBMS_INIT_UNIFORM, LBMS_INIT_PROFILE_1D = 0, 1
UNET_MAX_VOXELS = 8000000
_INIT_MODES = {"uniform": LBMS_INIT_UNIFORM, "profile1d": LBMS_INIT_PROFILE_1D}
LBMS_OUTLET_FLUX, LBMS_OUTLET_EXTRAPOLATED = 0, 1
LBMS_GRAD_CENTRAL, LBMS_GRAD_FORWARD = 0, 1
_OUTLETS = {"flux": LBMS_OUTLET_FLUX, "extrapolated": LBMS_OUTLET_EXTRAPOLATED}
_STENCILS = {"central": LBMS_GRAD_CENTRAL, "forward": LBMS_GRAD_FORWARD}

STATUS_NAMES = {0: "LBMS_OK", 1: "LBMS_EINVAL", 2: "LBMS_ENOMEM", 3: "LBMS_ECUDA",
                4: "LBMS_ENOTCONVERGED", 5: "LBMS_EUNSTABLE", 6: "LBMS_EDEPLETED",
                7: "LBMS_ESTATE"}

EXPORTS = ("lbms_default_options", "lbms_create", "lbms_set_bc", "lbms_set_fields", "lbms_step",
           "lbms_residual", "lbms_run_to_residual", "lbms_get_fields", "lbms_overpotential",
           "lbms_boundary_flux", "lbms_get_info", "lbms_synchronize", "lbms_destroy",
           "lbms_last_error", "lbms_status_string", "lbms_residual_sums_noalloc",
           "lbms_create_batch", "lbms_batch_set_bc", "lbms_batch_set_fields", "lbms_batch_residuals",
           "lbms_batch_run_to_residual", "lbms_batch_get_fields", "lbms_batch_overpotentials")
NET_EXPORTS = ("lbms_net_create", "lbms_net_add_sample", "lbms_net_features", "lbms_net_train",
               "lbms_net_warm_start", "lbms_net_set_gemm", "lbms_net_gemm_calls",
               "lbms_net_forward", "lbms_net_train_batch", "lbms_net_get", "lbms_net_set", "lbms_net_info",
               "lbms_net_last_error", "lbms_net_destroy")
UNET_EXPORTS = ("lbms_unet_create", "lbms_unet_add_sample", "lbms_unet_add_volume", "lbms_unet_train",
                "lbms_unet_warm_start",
                "lbms_unet_forward", "lbms_unet_train_batch", "lbms_unet_get", "lbms_unet_set", "lbms_unet_info",
                "lbms_unet_gemm_calls", "lbms_unet_last_error", "lbms_unet_destroy")


class LbmsError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status
        self.message = message


class Geometry(C.Structure):
    _fields_ = [("dim", C.c_int), ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("solid", C.c_void_p), ("length_x_m", C.c_double), ("periodic_x", C.c_int)]


class Species(C.Structure):
    _fields_ = [("n", C.c_int), ("molar_mass", C.POINTER(C.c_double)),
                ("fuller_volume", C.POINTER(C.c_double)), ("stoich", C.POINTER(C.c_int)),
                ("electrons", C.c_int)]


class Diffusivities(C.Structure):
    _fields_ = [("D_binary_m2s", C.POINTER(C.c_double)), ("pore_diameter_m", C.c_double),
                ("eps_over_tau", C.c_double)]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)


class Options(C.Structure):
    _fields_ = [("precision", C.c_int), ("coupling", C.c_int), ("tau_min", C.c_double),
                ("tau_max", C.c_double), ("dt_s", C.c_double), ("check_every", C.c_int),
                ("extrapolate_every", C.c_int), ("step_variant", C.c_int),
                ("init_mode", C.c_int), ("outlet_bc", C.c_int), ("grad_stencil", C.c_int),
                ("stream", C.c_void_p), ("alloc", ALLOC_FN), ("free", FREE_FN),
                ("alloc_user", C.c_void_p), ("extrapolate_modes", C.c_int)]


class Info(C.Structure):
    _fields_ = [("n_cells", C.c_int64), ("n_fluid", C.c_int64), ("q", C.c_int),
                ("precision", C.c_int), ("dx_m", C.c_double), ("dt_s", C.c_double),
                ("C_t", C.c_double), ("D_eff_m2s", C.c_double * 9), ("D_lat", C.c_double * 9),
                ("q_lat", C.c_double * 3), ("x_in", C.c_double * 3),
                ("current_A_cm2", C.c_double), ("steps", C.c_int64),
                ("device_bytes", C.c_size_t), ("h2d_bytes", C.c_uint64),
                ("d2h_bytes", C.c_uint64), ("n_cases", C.c_int), ("tile_cells", C.c_int),
                ("tile_min_blocks", C.c_int), ("neighbour_bits", C.c_int),
                ("threads_per_cell", C.c_int)]


_lib = None


def load(build_if_needed: bool = True):
    """Loads (building if needed) the solver library and declares its ABI."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_needed:
        _build.build()
    if not os.path.exists(_build.LIB):
        raise RuntimeError(f"solver library {_build.LIB} is missing; run __graft_entry__.build()")
    lib = C.CDLL(_build.LIB)
    P, D, I64 = C.c_void_p, C.POINTER(C.c_double), C.c_int64
    st = C.c_int
    sig = {
        "lbms_default_options": (None, [C.POINTER(Options)]),
        "lbms_create": (st, [C.POINTER(Geometry), C.POINTER(Species), C.POINTER(Diffusivities),
                             C.c_double, C.c_double, C.POINTER(Options), C.POINTER(P)]),
        "lbms_set_bc": (st, [P, D, C.c_double]),
        "lbms_set_fields": (st, [P, D]),
        "lbms_step": (st, [P, I64]),
        "lbms_residual": (st, [P, C.c_int, D]),
        "lbms_run_to_residual": (st, [P, C.c_double, I64, C.POINTER(I64), D]),
        "lbms_get_fields": (st, [P, D, D, D]),
        "lbms_overpotential": (st, [P, D, D]),
        "lbms_boundary_flux": (st, [P, D, D]),
        "lbms_get_info": (st, [P, C.POINTER(Info)]),
        "lbms_synchronize": (st, [P]),
        "lbms_destroy": (None, [P]),
        "lbms_last_error": (C.c_char_p, [P]),
        "lbms_status_string": (C.c_char_p, [C.c_int]),
        "lbms_residual_sums_noalloc": (st, [P, P, I64, C.c_int, P, P]),
        "lbms_create_batch": (st, [C.c_int, C.POINTER(Geometry), C.POINTER(Species),
                                   C.POINTER(Diffusivities), C.c_double, C.c_double,
                                   C.POINTER(Options), C.POINTER(P)]),
        "lbms_batch_set_bc": (st, [P, C.c_int, D, C.c_double]),
        "lbms_batch_set_fields": (st, [P, C.c_int, D]),
        "lbms_batch_residuals": (st, [P, C.c_int, D]),
        "lbms_batch_run_to_residual": (st, [P, C.c_double, I64, C.POINTER(I64), C.POINTER(I64), D]),
        "lbms_batch_get_fields": (st, [P, C.c_int, D, D, D]),
        "lbms_batch_overpotentials": (st, [P, D, D]),
        "lbms_net_create": (st, [C.c_int, C.c_int, C.c_uint64, C.POINTER(P)]),
        "lbms_net_add_sample": (st, [P, P, C.c_int]),
        "lbms_net_features": (st, [P, P, C.c_int, P, I64]),
        "lbms_net_set_gemm": (st, [P, C.c_int]),
        "lbms_net_gemm_calls": (st, [P, C.POINTER(I64), C.POINTER(I64)]),
        "lbms_net_train": (st, [P, C.c_int, C.c_int, C.c_double, D]),
        "lbms_net_warm_start": (st, [P, P, C.c_int, D]),
        "lbms_net_forward": (st, [P, P, C.c_int, P]),
        "lbms_net_train_batch": (st, [P, P, P, C.c_int, C.c_double, D]),
        "lbms_net_get": (st, [P, C.c_int, P, I64]),
        "lbms_net_set": (st, [P, P, I64]),
        "lbms_net_info": (st, [P, C.POINTER(I64), C.POINTER(I64)]),
        "lbms_net_last_error": (C.c_char_p, [P]),
        "lbms_net_destroy": (None, [P]),
        "lbms_unet_create": (st, [C.c_int, I64, C.c_uint64, C.POINTER(P)]),
        "lbms_unet_add_sample": (st, [P, P, C.c_int]),
        "lbms_unet_add_volume": (st, [P, P, P, C.c_int, C.c_int, C.c_int]),
        "lbms_unet_train": (st, [P, C.c_int, C.c_int, C.c_double, D]),
        "lbms_unet_warm_start": (st, [P, P, C.c_int, D]),
        "lbms_unet_forward": (st, [P, P, C.c_int, C.c_int, C.c_int, C.c_int, P]),
        "lbms_unet_train_batch": (st, [P, P, P, C.c_int, C.c_int, C.c_int, C.c_int, C.c_double, D]),
        "lbms_unet_get": (st, [P, C.c_int, P, I64]),
        "lbms_unet_set": (st, [P, P, I64]),
        "lbms_unet_info": (st, [P, C.POINTER(I64), C.POINTER(I64)]),
        "lbms_unet_gemm_calls": (st, [P, C.POINTER(I64)]),
        "lbms_unet_last_error": (C.c_char_p, [P]),
        "lbms_unet_destroy": (None, [P]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _dptr(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


class _Handle:
    """Argument marshalling shared by Solver and Batch."""

    def _setup(self, molar_mass, fuller_volume, stoich, electrons, D_binary, pore_diameter,
               eps_over_tau, precision, coupling, tau_min, tau_max, dt, check_every, stream,
               torch_allocator, extrapolate_every=0, step_variant=0, init_mode="uniform",
               outlet_bc="flux", grad_stencil="central", extrapolate_modes=1):
        lib = load()
        self._lib = lib
        self._mm = np.ascontiguousarray(molar_mass, dtype=np.float64)
        self._fv = np.ascontiguousarray(fuller_volume, dtype=np.float64)
        self._nu = np.ascontiguousarray(stoich, dtype=np.int32)
        sp = Species(3, _dptr(self._mm), _dptr(self._fv),
                     self._nu.ctypes.data_as(C.POINTER(C.c_int)), int(electrons))
        if D_binary is not None:
            self._db = np.ascontiguousarray(D_binary, dtype=np.float64).reshape(9)
            dptr = _dptr(self._db)
        else:
            dptr = None
        df = Diffusivities(dptr, float(pore_diameter or 0.0), float(eps_over_tau))
        o = Options()
        lib.lbms_default_options(C.byref(o))
        o.precision = {"fp64": LBMS_FP64, "fp32": LBMS_FP32, "fp16": LBMS_FP16}[precision]
        o.coupling = {"ms": LBMS_COUPLING_MS, "tau_only": LBMS_COUPLING_TAU_ONLY}[coupling]
        o.tau_min = float(tau_min)
        o.tau_max = float(tau_max)
        o.dt_s = float(dt or 0.0)
        o.check_every = int(check_every)
        o.extrapolate_every = int(extrapolate_every)
        o.extrapolate_modes = int(extrapolate_modes)
        o.step_variant = int(step_variant)
        o.init_mode = _INIT_MODES[init_mode]
        o.outlet_bc = _OUTLETS[outlet_bc]
        o.grad_stencil = _STENCILS[grad_stencil]
        self._keep = []
        if stream is None or torch_allocator:
            try:
                import torch
                if torch.cuda.is_available():
                    if stream is None:
                        stream = torch.cuda.current_stream().cuda_stream
                    if torch_allocator:
                        dev = torch.cuda.current_device()

                        def _alloc(size, s, user):
                            return torch.cuda.caching_allocator_alloc(int(size), dev, int(s or 0))

                        def _free(ptr, size, s, user):
                            torch.cuda.caching_allocator_delete(int(ptr))

                        fa, ff = ALLOC_FN(_alloc), FREE_FN(_free)
                        self._keep += [fa, ff]
                        o.alloc, o.free = fa, ff
            except ImportError:
                pass
        o.stream = stream or None
        self.stream = stream or 0
        self._opts = o
        return sp, df, o

    @staticmethod
    def _geometry(solid, dim, length_x, periodic_x):
        solid = np.asarray(solid, dtype=bool)
        if solid.ndim == 2:
            solid = solid[None]
        nz, ny, nx = solid.shape
        if dim is None:
            dim = 2 if nz == 1 else 3
        mask = np.ascontiguousarray(solid.astype(np.uint8))
        g = Geometry(dim, nx, ny, nz, mask.ctypes.data, float(length_x), int(bool(periodic_x)))
        return g, mask, solid.shape, dim

    def _check(self, s):
        if s != LBMS_OK:
            raise LbmsError(s, self._lib.lbms_last_error(self._h).decode())

    def step(self, n=1):
        self._check(self._lib.lbms_step(self._h, int(n)))

    def info(self):
        i = Info()
        self._check(self._lib.lbms_get_info(self._h, C.byref(i)))
        return i

    def synchronize(self):
        self._check(self._lib.lbms_synchronize(self._h))

    def close(self):
        if getattr(self, "_h", None):
            self._lib.lbms_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


_GAS_DEFAULTS = dict(molar_mass=(2.016, 18.015, 39.948), fuller_volume=(6.12, 13.1, 16.2),
                     stoich=(-1, 1, 0), electrons=2, D_binary=None, pore_diameter=1e-6,
                     eps_over_tau=1.0)


def _case_gas(case):
    g = case.gas
    return dict(molar_mass=g.molar_mass, fuller_volume=g.fuller_volume, stoich=g.stoich,
                electrons=g.electrons, D_binary=g.D_binary, pore_diameter=g.pore_diameter,
                eps_over_tau=g.eps_over_tau, T=g.T, p=g.p)


class Batch(_Handle):
    """Several independent anodes stepped by one kernel launch per step.

    ``solids`` is a list of bool arrays [z, y, x] (all 2-D or all 3-D);
    ``length_x`` and ``periodic_x`` are scalars or per-case lists.
    """

    def __init__(self, solids, dim=None, length_x=2e-3, periodic_x=False, *, T=1073.0, p=101325.0,
                 precision="fp32", coupling="ms", tau_min=1.0, tau_max=5.0, dt=0.0, check_every=100,
                 stream=None, torch_allocator=True, extrapolate_every=0, step_variant=0,
                 init_mode="uniform", outlet_bc="flux", grad_stencil="central", extrapolate_modes=1,
                 **gas):
        g = dict(_GAS_DEFAULTS)
        g.update(gas)
        sp, df, o = self._setup(g["molar_mass"], g["fuller_volume"], g["stoich"], g["electrons"],
                                g["D_binary"], g["pore_diameter"], g["eps_over_tau"], precision,
                                coupling, tau_min, tau_max, dt, check_every, stream, torch_allocator,
                                extrapolate_every, step_variant, init_mode, outlet_bc, grad_stencil,
                                extrapolate_modes)
        n = len(solids)
        lx = list(length_x) if np.ndim(length_x) else [length_x] * n
        px = list(periodic_x) if np.ndim(periodic_x) else [periodic_x] * n
        geoms = (Geometry * n)()
        self._masks, self.shapes = [], []
        for k in range(n):
            gk, mask, shape, d = self._geometry(solids[k], dim, lx[k], px[k])
            geoms[k] = gk
            self._masks.append(mask)
            self.shapes.append(shape)
            self.dim = d
        self.n = n
        h = C.c_void_p()
        s = self._lib.lbms_create_batch(n, geoms, C.byref(sp), C.byref(df), float(T), float(p),
                                        C.byref(o), C.byref(h))
        if s != LBMS_OK:
            raise LbmsError(s, self._lib.lbms_last_error(None).decode())
        self._h = h

    @classmethod
    def from_cases(cls, cases, **kw):
        """Builds a batch from workload descriptions sharing the same gas."""
        args = dict(dim=cases[0].dim, length_x=[c.length_x for c in cases],
                    periodic_x=[c.periodic_x for c in cases])
        args.update(_case_gas(cases[0]))
        args.update(kw)
        b = cls([c.solid for c in cases], **args)
        return b

    def set_bc(self, x_in, current_A_cm2, case=None):
        x = np.ascontiguousarray(x_in, dtype=np.float64)
        if case is None:
            self._check(self._lib.lbms_set_bc(self._h, _dptr(x), float(current_A_cm2)))
        else:
            self._check(self._lib.lbms_batch_set_bc(self._h, int(case), _dptr(x), float(current_A_cm2)))

    def set_fields(self, case, X):
        n = int(np.prod(self.shapes[case]))
        X = np.ascontiguousarray(X, dtype=np.float64).reshape(3 * n)
        self._check(self._lib.lbms_batch_set_fields(self._h, int(case), _dptr(X)))

    def residuals(self, K):
        r = np.empty(self.n)
        self._check(self._lib.lbms_batch_residuals(self._h, int(K), _dptr(r)))
        return r

    def run_to_residual(self, tol, max_steps, raise_on_fail=True):
        n = C.c_int64()
        steps = np.empty(self.n, dtype=np.int64)
        r = np.empty(self.n)
        s = self._lib.lbms_batch_run_to_residual(self._h, float(tol), int(max_steps), C.byref(n),
                                                 steps.ctypes.data_as(C.POINTER(C.c_int64)), _dptr(r))
        if raise_on_fail:
            self._check(s)
        return n.value, steps, r, s

    def fields(self, case, u=False, tau=False):
        shape = self.shapes[case]
        X = np.empty((3,) + shape)
        U = np.empty((3, self.dim) + shape) if u else None
        T = np.empty((3,) + shape) if tau else None
        self._check(self._lib.lbms_batch_get_fields(self._h, int(case), _dptr(X),
                                                    _dptr(U) if u else None, _dptr(T) if tau else None))
        out = [X] + ([U] if u else []) + ([T] if tau else [])
        return out[0] if len(out) == 1 else tuple(out)

    def overpotentials(self, raise_on_fail=True):
        eta = np.empty(self.n)
        xo = np.empty((self.n, 3))
        s = self._lib.lbms_batch_overpotentials(self._h, _dptr(eta), _dptr(xo))
        if raise_on_fail:
            self._check(s)
        return eta, xo


class Solver(_Handle):
    """One solver instance on the current CUDA device (a handle of the C ABI).

    ``solid`` is a bool array [z, y, x] (or [y, x] in 2-D), True = solid.
    """

    def __init__(self, solid, dim=None, length_x=2e-3, periodic_x=False, *,
                 molar_mass=(2.016, 18.015, 39.948), fuller_volume=(6.12, 13.1, 16.2),
                 stoich=(-1, 1, 0), electrons=2, D_binary=None, pore_diameter=1e-6,
                 eps_over_tau=1.0, T=1073.0, p=101325.0, precision="fp32", coupling="ms",
                 tau_min=1.0, tau_max=5.0, dt=0.0, check_every=100, stream=None,
                 torch_allocator=True, extrapolate_every=0, step_variant=0, init_mode="uniform",
                 outlet_bc="flux", grad_stencil="central", extrapolate_modes=1):
        sp, df, o = self._setup(molar_mass, fuller_volume, stoich, electrons, D_binary,
                                pore_diameter, eps_over_tau, precision, coupling, tau_min, tau_max,
                                dt, check_every, stream, torch_allocator, extrapolate_every,
                                step_variant, init_mode, outlet_bc, grad_stencil, extrapolate_modes)
        g, mask, shape, dim = self._geometry(solid, dim, length_x, periodic_x)
        self._mask = mask
        self.shape = shape
        self.dim = dim
        self.N = int(np.prod(shape))
        h = C.c_void_p()
        s = self._lib.lbms_create(C.byref(g), C.byref(sp), C.byref(df), float(T), float(p),
                                  C.byref(o), C.byref(h))
        if s != LBMS_OK:
            raise LbmsError(s, self._lib.lbms_last_error(None).decode())
        self._h = h

    # -------------------------------------------------------------- helpers
    @classmethod
    def from_case(cls, case, **kw):
        """Builds a solver from a workload description (duck-typed)."""
        g = case.gas
        args = dict(dim=case.dim, length_x=case.length_x, periodic_x=case.periodic_x,
                    molar_mass=g.molar_mass, fuller_volume=g.fuller_volume, stoich=g.stoich,
                    electrons=g.electrons, D_binary=g.D_binary, pore_diameter=g.pore_diameter,
                    eps_over_tau=g.eps_over_tau, T=g.T, p=g.p)
        args.update(kw)
        return cls(case.solid, **args)

    # ------------------------------------------------------------------ ABI
    def set_bc(self, x_in, current_A_cm2):
        x = np.ascontiguousarray(x_in, dtype=np.float64)
        self._check(self._lib.lbms_set_bc(self._h, _dptr(x), float(current_A_cm2)))

    def set_fields(self, X):
        X = np.ascontiguousarray(X, dtype=np.float64).reshape(3 * self.N)
        self._check(self._lib.lbms_set_fields(self._h, _dptr(X)))

    def residual(self, K):
        r = C.c_double()
        self._check(self._lib.lbms_residual(self._h, int(K), C.byref(r)))
        return r.value

    def run_to_residual(self, tol, max_steps, raise_on_fail=True):
        n = C.c_int64()
        r = C.c_double()
        s = self._lib.lbms_run_to_residual(self._h, float(tol), int(max_steps), C.byref(n), C.byref(r))
        if raise_on_fail:
            self._check(s)
        return n.value, r.value, s

    def fields(self, u=False, tau=False):
        """Returns X [3, z, y, x] (and u [3, dim, z, y, x] in m/s, tau [3, z, y, x])."""
        X = np.empty((3,) + self.shape)
        U = np.empty((3, self.dim) + self.shape) if u else None
        T = np.empty((3,) + self.shape) if tau else None
        self._check(self._lib.lbms_get_fields(self._h, _dptr(X), _dptr(U) if u else None,
                                              _dptr(T) if tau else None))
        out = [X]
        if u:
            out.append(U)
        if tau:
            out.append(T)
        return out[0] if len(out) == 1 else tuple(out)

    def overpotential(self):
        eta = C.c_double()
        xo = np.empty(3)
        self._check(self._lib.lbms_overpotential(self._h, C.byref(eta), _dptr(xo)))
        return eta.value, xo

    def boundary_flux(self):
        fl = np.empty(3)
        tot = np.empty(3)
        self._check(self._lib.lbms_boundary_flux(self._h, _dptr(fl), _dptr(tot)))
        return fl, tot



def to_bf16_bits(a):
    """Float array -> BF16 bit patterns (uint16), round to nearest even."""
    u = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32)
    r = ((u >> 16) & 1) + 0x7FFF
    return ((u + r) >> 16).astype(np.uint16)


def from_bf16_bits(b):
    return (np.asarray(b, dtype=np.uint16).astype(np.uint32) << 16).view(np.float32)


class Net:
    """The warm-start network of include/lbms_net.h (argument marshalling only)."""

    FEATURES = 64

    def __init__(self, width=704, depth=3, seed=0):
        self._lib = load()
        h = C.c_void_p()
        s = self._lib.lbms_net_create(int(width), int(depth), int(seed), C.byref(h))
        if s != LBMS_OK:
            raise LbmsError(s, "lbms_net_create(width=%d, depth=%d)" % (width, depth))
        self._h = h
        self.width, self.depth = width, depth

    def _check(self, s):
        if s != LBMS_OK:
            raise LbmsError(s, self._lib.lbms_net_last_error(self._h).decode())

    def info(self):
        a, b = C.c_int64(), C.c_int64()
        self._check(self._lib.lbms_net_info(self._h, C.byref(a), C.byref(b)))
        return a.value, b.value

    def add_sample(self, handle, case=0):
        self._check(self._lib.lbms_net_add_sample(self._h, handle._h, int(case)))

    GEMM_KINDS = {"auto": 0, "tcgen05": 1, "mma_sync": 2}

    def set_gemm(self, kind):
        """Which kernel computes the matrix products: auto, tcgen05, mma_sync."""
        self._check(self._lib.lbms_net_set_gemm(self._h, self.GEMM_KINDS[kind]))

    def gemm_calls(self):
        """(tcgen05 products, mma.sync products) computed so far."""
        a, b = C.c_int64(), C.c_int64()
        self._check(self._lib.lbms_net_gemm_calls(self._h, C.byref(a), C.byref(b)))
        return a.value, b.value

    def features(self, handle, n_fluid, case=0):
        """The case's feature rows as float32 [n_fluid, FEATURES] (from BF16)."""
        bits = np.empty((int(n_fluid), self.FEATURES), dtype=np.uint16)
        self._check(self._lib.lbms_net_features(self._h, handle._h, int(case), bits.ctypes.data, int(n_fluid)))
        return from_bf16_bits(bits).reshape(int(n_fluid), self.FEATURES)

    def train(self, iters, batch=8192, lr=1e-3):
        loss = C.c_double()
        self._check(self._lib.lbms_net_train(self._h, int(iters), int(batch), float(lr), C.byref(loss)))
        return loss.value

    def warm_start(self, handle, case=0):
        shape = handle.shapes[case] if hasattr(handle, "shapes") else handle.shape
        X = np.empty((3,) + tuple(shape))
        self._check(self._lib.lbms_net_warm_start(self._h, handle._h, int(case), _dptr(X)))
        return X

    def forward(self, features):
        f = np.ascontiguousarray(features, dtype=np.uint16)
        rows = f.shape[0]
        out = np.empty((rows, 3), dtype=np.float32)
        self._check(self._lib.lbms_net_forward(self._h, f.ctypes.data, rows, out.ctypes.data))
        return out

    def train_batch(self, features, targets, lr=0.0):
        f = np.ascontiguousarray(features, dtype=np.uint16)
        t = np.ascontiguousarray(targets, dtype=np.float32)
        loss = C.c_double()
        self._check(self._lib.lbms_net_train_batch(self._h, f.ctypes.data, t.ctypes.data, f.shape[0],
                                                   float(lr), C.byref(loss)))
        return loss.value

    def _layers(self, flat):
        """Splits a flat parameter vector into [(W, b), ...] per layer."""
        out, off = [], 0
        dims = [self.FEATURES] + [self.width] * self.depth + [3]
        for l in range(self.depth + 1):
            i, o = dims[l], dims[l + 1]
            W = flat[off:off + o * i].reshape(o, i)
            off += o * i
            b = flat[off:off + o]
            off += o
            out.append((W, b))
        return out

    def get(self, what=0):
        n, _ = self.info()
        buf = np.empty(n, dtype=np.float32)
        self._check(self._lib.lbms_net_get(self._h, int(what), buf.ctypes.data, n))
        return self._layers(buf)

    def set(self, layers):
        flat = np.concatenate([np.concatenate([W.ravel(), b.ravel()]) for W, b in layers]).astype(np.float32)
        self._check(self._lib.lbms_net_set(self._h, flat.ctypes.data, flat.size))

    def close(self):
        if getattr(self, "_h", None):
            self._lib.lbms_net_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class UNet:
    """The convolutional warm start of include/lbms_net.h (argument marshalling only)."""

    IN_CHANNELS = 17

    def __init__(self, width=28, max_voxels=1 << 20, seed=0):
        self._lib = load()
        h = C.c_void_p()
        s = self._lib.lbms_unet_create(int(width), int(max_voxels), int(seed), C.byref(h))
        if s != LBMS_OK:
            raise LbmsError(s, "lbms_unet_create(width=%d, max_voxels=%d)" % (width, max_voxels))
        self._h = h
        self.width, self.max_voxels = width, max_voxels

    def _check(self, s):
        if s != LBMS_OK:
            raise LbmsError(s, self._lib.lbms_unet_last_error(self._h).decode())

    def info(self):
        a, b = C.c_int64(), C.c_int64()
        self._check(self._lib.lbms_unet_info(self._h, C.byref(a), C.byref(b)))
        return a.value, b.value

    def gemm_calls(self):
        a = C.c_int64()
        self._check(self._lib.lbms_unet_gemm_calls(self._h, C.byref(a)))
        return a.value

    def add_sample(self, handle, case=0):
        self._check(self._lib.lbms_unet_add_sample(self._h, handle._h, int(case)))

    def add_volume(self, x, targets):
        """A training volume x float32 [17, Z, Y, X] with targets [3, Z, Y, X]."""
        x = np.ascontiguousarray(x, dtype=np.float32)
        t = np.ascontiguousarray(targets, dtype=np.float32)
        _, Z, Y, X = x.shape
        self._check(self._lib.lbms_unet_add_volume(self._h, x.ctypes.data, t.ctypes.data, X, Y, Z))

    def train(self, iters, max_batch=8, lr=1e-3):
        loss = C.c_double()
        self._check(self._lib.lbms_unet_train(self._h, int(iters), int(max_batch), float(lr), C.byref(loss)))
        return loss.value

    def warm_start(self, handle, case=0):
        shape = handle.shapes[case] if hasattr(handle, "shapes") else handle.shape
        X = np.empty((3,) + tuple(shape))
        self._check(self._lib.lbms_unet_warm_start(self._h, handle._h, int(case), _dptr(X)))
        return X

    def forward(self, x):
        """x float32 [B, 17, Z, Y, X] -> [B, 3, Z, Y, X]."""
        x = np.ascontiguousarray(x, dtype=np.float32)
        B, _, Z, Y, X = x.shape
        out = np.empty((B, 3, Z, Y, X), dtype=np.float32)
        self._check(self._lib.lbms_unet_forward(self._h, x.ctypes.data, B, X, Y, Z, out.ctypes.data))
        return out

    def train_batch(self, x, targets, lr=0.0):
        x = np.ascontiguousarray(x, dtype=np.float32)
        t = np.ascontiguousarray(targets, dtype=np.float32)
        B, _, Z, Y, X = x.shape
        loss = C.c_double()
        self._check(self._lib.lbms_unet_train_batch(self._h, x.ctypes.data, t.ctypes.data, B, X, Y, Z, float(lr),
                                                    C.byref(loss)))
        return loss.value

    def shapes(self):
        """Parameter shapes in order (those of the equivalent PyTorch modules)."""
        w = self.width
        out = []
        for ci, co in ((17, w), (w, w), (w, 2 * w), (2 * w, 2 * w), (2 * w, 4 * w), (4 * w, 4 * w)):
            out += [(co, ci, 3, 3, 3), (co,)]
        out += [(4 * w, 2 * w, 2, 2, 2), (2 * w,)]
        out += [(2 * w, 4 * w, 3, 3, 3), (2 * w,), (2 * w, 2 * w, 3, 3, 3), (2 * w,)]
        out += [(2 * w, w, 2, 2, 2), (w,)]
        out += [(w, 2 * w, 3, 3, 3), (w,), (w, w, 3, 3, 3), (w,)]
        out += [(3, w, 1, 1, 1), (3,)]
        return out

    def get(self, what=0):
        """Parameters (0) or last gradients (1) as a list of arrays of shapes()."""
        n, _ = self.info()
        buf = np.empty(n, dtype=np.float32)
        self._check(self._lib.lbms_unet_get(self._h, int(what), buf.ctypes.data, n))
        out, off = [], 0
        for sh in self.shapes():
            k = int(np.prod(sh))
            out.append(buf[off:off + k].reshape(sh))
            off += k
        return out

    def set(self, params):
        flat = np.concatenate([np.asarray(p, dtype=np.float32).ravel() for p in params])
        self._check(self._lib.lbms_unet_set(self._h, flat.ctypes.data, flat.size))

    def close(self):
        if getattr(self, "_h", None):
            self._lib.lbms_unet_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
