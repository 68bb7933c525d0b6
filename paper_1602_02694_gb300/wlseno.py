"""Thin ctypes binding of libwlseno (include/wlseno.h).

Argument marshalling only: every step of the method runs in the library's
CUDA kernels (and its native host setup).  Arrays may be torch tensors on the
context's GPU (used in place, on torch's current stream) or host numpy
arrays / CPU tensors (copied by the library inside the call).  The binding
raises if the compiled library is missing; there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libwlseno.so")

ADVECTION, BURGERS, EULER = 0, 1, 2
FP64, FP32_BULK = 0, 1
_PDE = {"advection": ADVECTION, "burgers": BURGERS, "euler": EULER}
_PREC = {"fp64": FP64, "fp32_bulk": FP32_BULK, "fp32-bulk": FP32_BULK}


class WlsenoError(RuntimeError):
    def __init__(self, status, where, detail=""):
        self.status = status
        super().__init__(f"{where}: {status_string(status)} ({status}) {detail}".rstrip())


class wlseno_mesh(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("n_vertices", ctypes.c_int64), ("n_cells", ctypes.c_int64),
                ("vertices", ctypes.c_void_p), ("cells", ctypes.c_void_p), ("period", ctypes.c_void_p)]


class wlseno_stencil_opts(ctypes.Structure):
    _fields_ = [("order_p", ctypes.c_int), ("ring", ctypes.c_double), ("radius_cut", ctypes.c_double),
                ("min_rows", ctypes.c_int), ("lanes_per_cell", ctypes.c_int),
                ("rows_per_lane", ctypes.c_int), ("moments_mode", ctypes.c_int),
                ("reorder", ctypes.c_int), ("persistent", ctypes.c_int)]


class wlseno_scheme(ctypes.Structure):
    _fields_ = [("pde", ctypes.c_int), ("n_comp", ctypes.c_int), ("velocity", ctypes.c_double * 3),
                ("eps", ctypes.c_double), ("alpha_c", ctypes.c_double), ("rank_tol", ctypes.c_double),
                ("kappa_flag", ctypes.c_double), ("precision", ctypes.c_int), ("gamma", ctypes.c_double),
                ("characteristic", ctypes.c_int), ("balanced", ctypes.c_int),
                ("balance_margin", ctypes.c_double)]


class wlseno_info(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("order_p", ctypes.c_int), ("m", ctypes.c_int),
                ("n_comp", ctypes.c_int), ("n_meshes", ctypes.c_int), ("n_cells", ctypes.c_int64),
                ("stencil_nnz", ctypes.c_int64), ("max_stencil", ctypes.c_int),
                ("min_stencil", ctypes.c_int), ("quad_per_facet", ctypes.c_int),
                ("lanes_per_cell", ctypes.c_int), ("rows_per_lane", ctypes.c_int),
                ("moments_mode", ctypes.c_int), ("persistent", ctypes.c_int)]


KERNEL_KINDS = ("moments", "reconstruct", "flux", "dt", "adjoint", "fixup", "step")


class wlseno_diagnostics(ctypes.Structure):
    _fields_ = [("flagged_cells", ctypes.c_int64), ("rank_deficient", ctypes.c_int64),
                ("nonfinite", ctypes.c_int64), ("kernel_launches", ctypes.c_int64),
                ("last_dt", ctypes.c_double),
                ("launches_by_kind", ctypes.c_int64 * len(KERNEL_KINDS)),
                ("kernel_ms", ctypes.c_double * len(KERNEL_KINDS)),
                ("positivity_fallbacks", ctypes.c_int64), ("balanced_cells", ctypes.c_int64)]


# every symbol include/wlseno.h declares, with its C signature
_P = ctypes.c_void_p
_I = ctypes.c_int
_D = ctypes.c_double
SIGNATURES = {
    "wlseno_create": (_I, [ctypes.POINTER(_P), _I, ctypes.POINTER(wlseno_scheme)]),
    "wlseno_destroy": (None, [_P]),
    "wlseno_build_stencils": (_I, [_P, ctypes.POINTER(wlseno_mesh), _I,
                                   ctypes.POINTER(wlseno_stencil_opts), _P]),
    "wlseno_precompute_moments": (_I, [_P, _P]),
    "wlseno_reconstruct": (_I, [_P, _P, _P, _P, _P]),
    "wlseno_flux_residual": (_I, [_P, _P, _P, _P]),
    "wlseno_rk_step": (_I, [_P, _P, _D, _D, _I, _P, _P]),
    "wlseno_step_adjoint": (_I, [_P, _P, _D, _P, _P, _P]),
    "wlseno_get_info": (_I, [_P, ctypes.POINTER(wlseno_info)]),
    "wlseno_get_stencils": (_I, [_P, _P, _P]),
    "wlseno_get_geometry": (_I, [_P, _P, _P, _P, _P]),
    "wlseno_get_diagnostics": (_I, [_P, ctypes.POINTER(wlseno_diagnostics)]),
    "wlseno_set_timing": (_I, [_P, _I]),
    "wlseno_set_wait_limit": (_I, [_P, ctypes.c_int64]),
    "wlseno_autotune": (_I, [_P, _P, _I, _P, _P]),
    "wlseno_flux_residual_static": (_I, [_P, _P, _P, _P]),
    "wlseno_set_mesh_dt": (_I, [_P, _P]),
    "wlseno_measure_fma_peak": (_I, [_I, _I, ctypes.POINTER(_D)]),
    "wlseno_status_string": (ctypes.c_char_p, [_I]),
    "wlseno_last_error_message": (ctypes.c_char_p, [_P]),
}

_lib = None


def load_library(path: str = LIB_PATH):
    """Load libwlseno.so and declare every entry point; raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is not built; run `python -c 'import __graft_entry__ as g; g.build()'`")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def measure_fma_peak(device: int, precision: str) -> float:
    """wlseno_measure_fma_peak: measured FP32 ("fp32") or FP64 ("fp64") FMA
    throughput of the device in TFLOP/s."""
    lib = load_library()
    out = ctypes.c_double(0.0)
    st = lib.wlseno_measure_fma_peak(int(device), FP64 if precision == "fp64" else FP32_BULK, ctypes.byref(out))
    if st != 0:
        raise WlsenoError(st, "wlseno_measure_fma_peak")
    return out.value


def status_string(status: int) -> str:
    try:
        return load_library().wlseno_status_string(status).decode()
    except Exception:  # library missing: still format the number
        return "status"


# ----------------------------------------------------------------------------
# pointer marshalling
# ----------------------------------------------------------------------------

def _is_torch(x):
    return type(x).__module__.startswith("torch")


def _ptr(x, dtype=np.float64, writable=False):
    """(address, keep-alive) of a contiguous float64 array (torch or numpy)."""
    if x is None:
        return None, None
    if _is_torch(x):
        import torch
        if x.dtype != torch.float64 or not x.is_contiguous():
            raise TypeError("arrays must be contiguous float64 tensors")
        return x.data_ptr(), x
    if not isinstance(x, np.ndarray) or x.dtype != dtype or not x.flags.c_contiguous:
        raise TypeError("arrays must be C-contiguous float64 numpy arrays")
    if writable and not x.flags.writeable:
        raise TypeError("output array is read-only")
    return x.ctypes.data, x


def _numel(x):
    return x.numel() if _is_torch(x) else int(x.size)


def check_length(x, need, name):
    """Raise ValueError when array x (torch or numpy, may be None) holds
    fewer than `need` elements: the library takes plain pointers and would
    read or write past its end."""
    if x is None or not (_is_torch(x) or isinstance(x, np.ndarray)):
        return  # not an array: the pointer marshalling raises TypeError
    if _numel(x) < need:
        raise ValueError(f"{name} has {_numel(x)} elements; this context needs {need}")


def _stream_of(*arrays):
    for a in arrays:
        if a is not None and _is_torch(a) and a.is_cuda:
            import torch
            return torch.cuda.current_stream(a.device).cuda_stream
    return None


class Context:
    """One wlseno_ctx: a scheme, the meshes' stencils and moments on one GPU.

    The keyword arguments fill wlseno_scheme: pde ("advection", "burgers",
    "euler"), precision ("fp64" or "fp32_bulk"), n_comp (default 1, or 4 for
    Euler; 3 and 5 for 1-D and 3-D Euler), characteristic (Euler in 1-D and
    2-D), balanced and balance_margin (the balanced-stencil re-selection of
    scalar equations), eps, alpha_c, rank_tol, kappa_flag, gamma, velocity.
    Raises WlsenoError with the library's status and message."""

    def __init__(self, device: int = 0, pde="advection", velocity=(1.0, 1.0, 0.0), eps=1e-2,
                 alpha_c=1.5, rank_tol=1e-10, kappa_flag=1e3, precision="fp64", n_comp=None,
                 gamma=1.4, characteristic=False, balanced=False, balance_margin=0.02):
        self.lib = load_library()
        sch = wlseno_scheme()
        sch.pde = _PDE[pde] if isinstance(pde, str) else int(pde)
        sch.n_comp = n_comp if n_comp is not None else (4 if sch.pde == EULER else 1)
        sch.gamma = gamma
        sch.characteristic = 1 if characteristic else 0
        sch.balanced = 1 if balanced else 0
        sch.balance_margin = balance_margin
        for a in range(3):
            sch.velocity[a] = float(velocity[a]) if a < len(velocity) else 0.0
        sch.eps, sch.alpha_c, sch.rank_tol, sch.kappa_flag = eps, alpha_c, rank_tol, kappa_flag
        sch.precision = _PREC[precision] if isinstance(precision, str) else int(precision)
        self.scheme = sch
        self.device = device
        h = ctypes.c_void_p()
        self._check(self.lib.wlseno_create(ctypes.byref(h), device, ctypes.byref(sch)), "wlseno_create",
                    use_ctx=False)
        self.h = h

    # -- plumbing
    def _check(self, st, where, use_ctx=True):
        if st != 0:
            detail = ""
            if use_ctx and getattr(self, "h", None):
                detail = self.lib.wlseno_last_error_message(self.h).decode()
            raise WlsenoError(st, where, detail)

    def close(self):
        if getattr(self, "h", None):
            self.lib.wlseno_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- entry points
    def build_stencils(self, meshes, order_p, ring, radius_cut=0.0, min_rows=0,
                       lanes_per_cell=0, rows_per_lane=0, moments_mode=0, reorder=0, persistent=0):
        """wlseno_build_stencils over one mesh or a list of meshes (objects with
        .vertices [nv][d] float64, .cells [nc][d+1] int64 and .period [d]).
        lanes_per_cell, rows_per_lane: kernel shape ((0, 0): the default);
        moments_mode: FP32-bulk thread-per-cell only, 0 stored moment rows,
        1 rows formed on the fly; reorder: 1 renumbers each mesh's cells along
        the Hilbert curve of their centroids (self.perm then holds new -> old,
        so ubar_lib = ubar_caller[perm]); persistent: 1 runs each RK step as
        one persistent cooperative kernel.  Returns the context's info dict."""
        if not isinstance(meshes, (list, tuple)):
            meshes = [meshes]
        arr = (wlseno_mesh * len(meshes))()
        keep = []
        for k, m in enumerate(meshes):
            v = np.ascontiguousarray(m.vertices, dtype=np.float64)
            c = np.ascontiguousarray(m.cells, dtype=np.int64)
            p = np.ascontiguousarray(m.period, dtype=np.float64)
            keep += [v, c, p]
            arr[k].dim = v.shape[1]
            arr[k].n_vertices = v.shape[0]
            arr[k].n_cells = c.shape[0]
            arr[k].vertices = v.ctypes.data
            arr[k].cells = c.ctypes.data
            arr[k].period = p.ctypes.data
        opts = wlseno_stencil_opts(order_p, float(ring), float(radius_cut), min_rows,
                                   lanes_per_cell, rows_per_lane, moments_mode, reorder, persistent)
        self._info = None
        perm = np.zeros(sum(int(np.asarray(m.cells).shape[0]) for m in meshes), dtype=np.int64)
        self._check(self.lib.wlseno_build_stencils(self.h, arr, len(meshes), ctypes.byref(opts),
                                                   perm.ctypes.data), "wlseno_build_stencils")
        self.perm = perm
        self._info = self.info()
        return self._info

    def _lengths(self, per_cell, **arrays):
        """Check the arrays against the built context's sizes: n_comp x
        n_cells x per_cell[name] elements each (before any build the library
        itself reports the missing state)."""
        inf = getattr(self, "_info", None)
        if not inf:
            return
        base = inf["n_comp"] * inf["n_cells"]
        for name, x in arrays.items():
            check_length(x, base * per_cell.get(name, 1), name)

    def precompute_moments(self, stream=None):
        self._check(self.lib.wlseno_precompute_moments(self.h, stream), "wlseno_precompute_moments")

    def reconstruct(self, ubar, coeffs=None, facet_values=None, stream=None):
        inf = getattr(self, "_info", None) or {}
        self._lengths({"coeffs": inf.get("m", 1),
                       "facet_values": (inf.get("dim", 0) + 1) * inf.get("quad_per_facet", 1)},
                      ubar=ubar, coeffs=coeffs, facet_values=facet_values)
        pu, _ = _ptr(ubar)
        pc, _ = _ptr(coeffs, writable=True)
        pf, _ = _ptr(facet_values, writable=True)
        s = stream if stream is not None else _stream_of(ubar, coeffs, facet_values)
        self._check(self.lib.wlseno_reconstruct(self.h, pu, pc, pf, s), "wlseno_reconstruct")

    def flux_residual(self, ubar, residual, stream=None):
        self._lengths({}, ubar=ubar, residual=residual)
        pu, _ = _ptr(ubar)
        pr, _ = _ptr(residual, writable=True)
        s = stream if stream is not None else _stream_of(ubar, residual)
        self._check(self.lib.wlseno_flux_residual(self.h, pu, pr, s), "wlseno_flux_residual")

    def flux_residual_static(self, ubar, residual, stream=None):
        """wlseno_flux_residual_static: L(ubar) with no device allocation
        (fixed library scratch; device arrays only)."""
        self._lengths({}, ubar=ubar, residual=residual)
        pu, _ = _ptr(ubar)
        pr, _ = _ptr(residual, writable=True)
        s = stream if stream is not None else _stream_of(ubar, residual)
        self._check(self.lib.wlseno_flux_residual_static(self.h, pu, pr, s),
                    "wlseno_flux_residual_static")

    def rk_step(self, ubar, dt=0.0, cfl=0.0, n_steps=1, want_dt=False, stream=None):
        """TVD-RK3 steps in place; returns the last dt when want_dt."""
        self._lengths({}, ubar=ubar)
        pu, _ = _ptr(ubar, writable=True)
        out = ctypes.c_double(0.0)
        s = stream if stream is not None else _stream_of(ubar)
        self._check(self.lib.wlseno_rk_step(self.h, pu, float(dt), float(cfl), int(n_steps),
                                            ctypes.byref(out) if want_dt else None, s),
                    "wlseno_rk_step")
        return out.value if want_dt else None

    def autotune(self, ubar, reps=5, stream=None):
        """Pick the fastest reconstruction kernel shape on this data;
        returns (lanes_per_cell, rows_per_lane, mean launch microseconds)."""
        self._lengths({}, ubar=ubar)
        pu, _ = _ptr(ubar)
        best = ctypes.c_double(0.0)
        s = stream if stream is not None else _stream_of(ubar)
        self._check(self.lib.wlseno_autotune(self.h, pu, int(reps), s, ctypes.byref(best)),
                    "wlseno_autotune")
        inf = self.info()
        return inf["lanes_per_cell"], inf["rows_per_lane"], best.value

    def set_mesh_dt(self, dts):
        """Per-mesh fixed steps, used by rk_step / step_adjoint with dt < 0."""
        a = np.ascontiguousarray(dts, dtype=np.float64)
        inf = getattr(self, "_info", None)
        if inf:
            check_length(a, inf["n_meshes"], "dts")
        self._check(self.lib.wlseno_set_mesh_dt(self.h, a.ctypes.data), "wlseno_set_mesh_dt")

    def step_adjoint(self, ubar_n, dt, gbar_next, gbar_n, stream=None):
        self._lengths({}, ubar_n=ubar_n, gbar_next=gbar_next, gbar_n=gbar_n)
        pu, _ = _ptr(ubar_n)
        pg, _ = _ptr(gbar_next)
        po, _ = _ptr(gbar_n, writable=True)
        s = stream if stream is not None else _stream_of(ubar_n, gbar_next, gbar_n)
        self._check(self.lib.wlseno_step_adjoint(self.h, pu, float(dt), pg, po, s),
                    "wlseno_step_adjoint")

    # -- queries
    def info(self):
        inf = wlseno_info()
        self._check(self.lib.wlseno_get_info(self.h, ctypes.byref(inf)), "wlseno_get_info")
        return {f: getattr(inf, f) for f, _ in wlseno_info._fields_}

    def stencils(self):
        inf = self.info()
        ptr = np.zeros(inf["n_cells"] + 1, dtype=np.int64)
        cols = np.zeros(inf["stencil_nnz"], dtype=np.int64)
        self._check(self.lib.wlseno_get_stencils(self.h, ptr.ctypes.data, cols.ctypes.data),
                    "wlseno_get_stencils")
        return ptr, cols

    def geometry(self):
        inf = self.info()
        N, d = inf["n_cells"], inf["dim"]
        cen = np.zeros((N, d))
        vol = np.zeros(N)
        h = np.zeros(N)
        inr = np.zeros(N)
        self._check(self.lib.wlseno_get_geometry(self.h, cen.ctypes.data, vol.ctypes.data,
                                                 h.ctypes.data, inr.ctypes.data), "wlseno_get_geometry")
        return {"centroid": cen, "volume": vol, "h": h, "inradius": inr}

    def diagnostics(self):
        d = wlseno_diagnostics()
        self._check(self.lib.wlseno_get_diagnostics(self.h, ctypes.byref(d)), "wlseno_get_diagnostics")
        out = {f: getattr(d, f) for f, _ in wlseno_diagnostics._fields_[:5]}
        out["launches_by_kind"] = dict(zip(KERNEL_KINDS, list(d.launches_by_kind)))
        out["kernel_ms"] = dict(zip(KERNEL_KINDS, list(d.kernel_ms)))
        out["positivity_fallbacks"] = d.positivity_fallbacks
        out["balanced_cells"] = d.balanced_cells
        return out

    def set_wait_limit(self, max_polls=0):
        """Poll limit of the persistent step's bounded barrier waits (0: default)."""
        self._check(self.lib.wlseno_set_wait_limit(self.h, int(max_polls)), "wlseno_set_wait_limit")

    def set_timing(self, enable=True):
        self._check(self.lib.wlseno_set_timing(self.h, 1 if enable else 0), "wlseno_set_timing")
