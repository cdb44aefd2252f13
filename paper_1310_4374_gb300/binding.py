"""Thin Python binding of the C-ABI in ``include/psum.h`` (ctypes).

The functions here carry the C names and only marshal arguments: tensors are
passed as raw device pointers and the current torch CUDA stream as a
``cudaStream_t``.  Every step of the computation runs in ``libpsum.so``; if the
library cannot be built or loaded, ``load()`` raises.
"""
from __future__ import annotations

import ctypes
import os
import re

from . import build as _build

PSUM_OK = 0
PSUM_ERR_ARG = 1
PSUM_ERR_NONNEUTRAL = 2
PSUM_ERR_OUT_OF_BOX = 3
PSUM_ERR_RANK = 4
PSUM_ERR_CUDA = 5
PSUM_ERR_TIMEOUT = 6
PSUM_ERR_NOMEM = 7
PSUM_ERR_NONFINITE = 8
PSUM_ERR_INTERNAL = 9
PSUM_ERR_IO = 10

PSUM_FP64 = 0
PSUM_FP32C = 1
PSUM_MEAN_ZERO = 0
PSUM_MEAN_NONE = 1
PSUM_NUM_STAGES = 5
STAGE_NAMES = ("prepare", "near_charges", "near_checkpoints", "fit", "far_combine")

PSUM_FF = 2
PRECISIONS = {"fp64": PSUM_FP64, "fp32c": PSUM_FP32C, "ff": PSUM_FF}
POINTS = {"fibonacci": 0, "gauss": 1}
BASES = {"spherical": 0, "rbf": 1}
PAIR_KERNELS = {"auto": 0, "one-sided": 1, "symmetric": 2}
CHECK_FORMS = {"auto": 0, "points": 1, "layers": 2}
FP32_TERMS = {"fast": 0, "refined": 1}
MEAN_MODES = {"zero": PSUM_MEAN_ZERO, "none": PSUM_MEAN_NONE}


class psum_opts(ctypes.Structure):
    _fields_ = [("d", ctypes.c_double * 3), ("p", ctypes.c_int), ("M", ctypes.c_int),
                ("precision", ctypes.c_int), ("mean_mode", ctypes.c_int), ("K", ctypes.c_int * 3),
                ("points", ctypes.c_int), ("lambda_", ctypes.c_double), ("basis", ctypes.c_int),
                ("n_rbf", ctypes.c_int), ("rbf_radius", ctypes.c_double), ("pair_kernel", ctypes.c_int),
                ("check_form", ctypes.c_int), ("fp32_terms", ctypes.c_int)]


class psum_info(ctypes.Structure):
    _fields_ = [("d", ctypes.c_double * 3), ("R0", ctypes.c_double), ("lambda_eff", ctypes.c_double),
                ("cond_est", ctypes.c_double), ("rank", ctypes.c_int), ("p", ctypes.c_int),
                ("P", ctypes.c_int), ("M", ctypes.c_int), ("K", ctypes.c_int * 3),
                ("n_images", ctypes.c_int), ("precision", ctypes.c_int), ("mean_mode", ctypes.c_int)]

    def as_dict(self):
        return {"d": tuple(self.d), "R0": self.R0, "lambda_eff": self.lambda_eff, "cond_est": self.cond_est,
                "rank": self.rank, "p": self.p, "P": self.P, "M": self.M, "K": tuple(self.K),
                "n_images": self.n_images, "precision": self.precision, "mean_mode": self.mean_mode}


class psum_batch_info(ctypes.Structure):
    _fields_ = [("B", ctypes.c_int), ("N_total", ctypes.c_int64), ("units", ctypes.c_int64),
                ("pairs", ctypes.c_int64), ("ctas", ctypes.c_int), ("variant", ctypes.c_int),
                ("tuned_ms", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class PsumError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        super().__init__(f"{what}: {psum_strerror(status)} (status {status})" if what else psum_strerror(status))


_lib = None
_vp = ctypes.c_void_p
_dp = ctypes.POINTER(ctypes.c_double)


def load(build_if_needed: bool = True):
    """Load libpsum.so (building it first if its sources changed)."""
    global _lib
    if _lib is not None:
        return _lib
    path = os.environ.get("PSUM_LIB") or (_build.build() if build_if_needed else _build.LIB_PATH)
    if not os.path.exists(path):
        raise RuntimeError(f"libpsum.so not found at {path}")
    lib = ctypes.CDLL(path)
    lib.psum_opts_default.argtypes = [ctypes.POINTER(psum_opts)]
    lib.psum_opts_default.restype = None
    lib.psum_plan_create.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                     ctypes.POINTER(_vp)]
    lib.psum_plan_create_ex.argtypes = [ctypes.POINTER(psum_opts), ctypes.POINTER(_vp)]
    lib.psum_plan_save.argtypes = [_vp, ctypes.c_char_p]
    lib.psum_plan_load.argtypes = [ctypes.c_char_p, ctypes.POINTER(_vp)]
    lib.psum_eval.argtypes = [_vp, ctypes.c_int64, _vp, _vp, _vp, _vp, _vp]
    lib.psum_debug_inject_timeout.argtypes = [_vp, ctypes.c_int]
    lib.psum_eval_graph.argtypes = [_vp, ctypes.c_int64, _vp, _vp, _vp, _vp, _vp]
    lib.psum_eval_points.argtypes = [_vp, ctypes.c_int64, _vp, _vp, ctypes.c_int64, _vp, _vp, _vp, _vp]
    lib.psum_eval_host.argtypes = [_vp, ctypes.c_int64, _vp, _vp, _vp, _vp, _vp]
    lib.psum_eval_noalloc.argtypes = [_vp, ctypes.c_int64, _vp, _vp, _vp, _vp, _vp]
    lib.psum_sync.argtypes = [_vp, _vp]
    lib.psum_get_coeffs.argtypes = [_vp, _dp, _vp]
    lib.psum_plan_info.argtypes = [_vp, ctypes.POINTER(psum_info)]
    lib.psum_pair_kernel.argtypes = [_vp, ctypes.c_int64, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]
    lib.psum_check_form.argtypes = [_vp, ctypes.POINTER(ctypes.c_int)]
    lib.psum_scratch_bytes.argtypes = [_vp, ctypes.c_int64, ctypes.POINTER(ctypes.c_int64),
                                       ctypes.POINTER(ctypes.c_int)]
    lib.psum_debug_band_bytes.argtypes = [_vp, ctypes.c_int64]
    lib.psum_debug_fail_allocs.argtypes = [_vp, ctypes.c_int]
    lib.psum_debug_bounds_limit.argtypes = [_vp, ctypes.c_int64]
    lib.psum_debug_checks.argtypes = []
    lib.psum_profile.argtypes = [_vp, ctypes.c_int]
    lib.psum_last_timings.argtypes = [_vp, _dp, _vp]
    lib.psum_launch_count.argtypes = [_vp, ctypes.POINTER(ctypes.c_int64)]
    lib.psum_energy.argtypes = [_vp, ctypes.c_int64, _vp, _vp, _vp, _vp]
    lib.psum_energy_backward.argtypes = [_vp, ctypes.c_int64, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp]
    lib.psum_energy_backward_c.argtypes = [_vp, ctypes.c_int64, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp]
    lib.psum_coeffs_device.argtypes = [_vp, _vp, _vp]
    lib.psum_batch_create.argtypes = [ctypes.POINTER(_vp), ctypes.c_int, ctypes.POINTER(ctypes.c_int64),
                                      ctypes.POINTER(_vp)]
    lib.psum_batch_eval.argtypes = [_vp, _vp, _vp, _vp, _vp, ctypes.c_int, _vp]
    lib.psum_batch_sync.argtypes = [_vp, ctypes.POINTER(ctypes.c_int), _vp]
    lib.psum_batch_get_coeffs.argtypes = [_vp, ctypes.c_int, _dp, _vp]
    lib.psum_batch_get_info.argtypes = [_vp, ctypes.POINTER(psum_batch_info)]
    lib.psum_batch_destroy.argtypes = [_vp]
    lib.psum_batch_destroy.restype = None
    lib.psum_destroy.argtypes = [_vp]
    lib.psum_destroy.restype = None
    lib.psum_strerror.argtypes = [ctypes.c_int]
    lib.psum_strerror.restype = ctypes.c_char_p
    for name in ("psum_plan_create", "psum_plan_create_ex", "psum_plan_save", "psum_plan_load", "psum_eval", "psum_eval_host", "psum_eval_noalloc",
                 "psum_sync",
                 "psum_get_coeffs", "psum_plan_info", "psum_pair_kernel", "psum_check_form",
                 "psum_scratch_bytes", "psum_debug_band_bytes", "psum_debug_fail_allocs",
                 "psum_debug_bounds_limit", "psum_debug_checks", "psum_profile", "psum_last_timings", "psum_launch_count",
                 "psum_energy", "psum_energy_backward", "psum_energy_backward_c", "psum_coeffs_device",
                 "psum_eval_points", "psum_debug_inject_timeout", "psum_eval_graph", "psum_batch_create", "psum_batch_eval",
                 "psum_batch_sync", "psum_batch_get_coeffs", "psum_batch_get_info"):
        getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


def header_functions() -> list:
    """Names of the functions declared in include/psum.h."""
    path = os.path.join(_build.INCLUDE, "psum.h")
    with open(path) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(psum_[a-z_]+)\s*\(", text)))


def _stream_ptr(stream):
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)


def _check(status: int, what: str):
    if status != PSUM_OK:
        raise PsumError(status, what)


def psum_strerror(status: int) -> str:
    return load().psum_strerror(int(status)).decode()


def psum_opts_default() -> psum_opts:
    o = psum_opts()
    load().psum_opts_default(ctypes.byref(o))
    return o


def psum_plan_create(d1: float, d2: float, d3: float, p: int, M: int):
    h = _vp()
    _check(load().psum_plan_create(float(d1), float(d2), float(d3), int(p), int(M), ctypes.byref(h)),
           "psum_plan_create")
    return h


def psum_plan_create_ex(d, p: int, M: int, precision="fp64", mean="zero", K=(1, 1, 1), points="fibonacci",
                        lam: float = 0.0, basis="spherical", n_rbf: int = 256, rbf_radius: float = 0.0,
                        pairs="auto", checks="auto", terms="fast"):
    o = psum_opts_default()
    o.fp32_terms = FP32_TERMS[terms] if isinstance(terms, str) else int(terms)
    o.pair_kernel = PAIR_KERNELS[pairs] if isinstance(pairs, str) else int(pairs)
    o.check_form = CHECK_FORMS[checks] if isinstance(checks, str) else int(checks)
    o.lambda_ = float(lam)
    o.basis = BASES[basis] if isinstance(basis, str) else int(basis)
    o.n_rbf = int(n_rbf)
    o.rbf_radius = float(rbf_radius)
    o.points = POINTS[points] if isinstance(points, str) else int(points)
    for k in range(3):
        o.d[k] = float(d[k])
        o.K[k] = int(K[k])
    o.p, o.M = int(p), int(M)
    o.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    o.mean_mode = MEAN_MODES[mean] if isinstance(mean, str) else int(mean)
    h = _vp()
    _check(load().psum_plan_create_ex(ctypes.byref(o), ctypes.byref(h)), "psum_plan_create_ex")
    return h


def psum_plan_save(plan, path) -> None:
    """Write the plan's options and factorisation to a file (algorithm "set" kept, Sec. 2.1)."""
    _check(load().psum_plan_save(plan, os.fsencode(path)), "psum_plan_save")


def psum_plan_load(path):
    """A plan from a file of psum_plan_save, without factoring the fitting matrix again."""
    h = _vp()
    _check(load().psum_plan_load(os.fsencode(path), ctypes.byref(h)), "psum_plan_load")
    return h


def psum_eval(plan, x, q, phi, grad=None, stream=None, check: bool = False) -> int:
    """Queue algorithm "get" on device tensors (float64, contiguous). Returns the launch status."""
    for t in (x, q, phi) + ((grad,) if grad is not None else ()):
        if not (t.is_cuda and t.is_contiguous()):
            raise ValueError("psum_eval takes contiguous CUDA tensors")
    st = _stream_ptr(stream)
    s = load().psum_eval(plan, int(q.numel()), x.data_ptr(), q.data_ptr(), phi.data_ptr(),
                         grad.data_ptr() if grad is not None else None, st)
    _check(s, "psum_eval")
    if check:
        _check(psum_sync(plan, st), "psum_eval (device)")
    return s


def psum_eval_graph(plan, x, q, phi, grad=None, stream=None, check: bool = False) -> int:
    """psum_eval replayed from a CUDA graph captured on first use for these tensors."""
    for t in (x, q, phi) + ((grad,) if grad is not None else ()):
        if not (t.is_cuda and t.is_contiguous()):
            raise ValueError("psum_eval_graph takes contiguous CUDA tensors")
    st = _stream_ptr(stream)
    s = load().psum_eval_graph(plan, int(q.numel()), x.data_ptr(), q.data_ptr(), phi.data_ptr(),
                               grad.data_ptr() if grad is not None else None, st)
    _check(s, "psum_eval_graph")
    if check:
        _check(psum_sync(plan, st), "psum_eval_graph (device)")
    return s


def psum_eval_points(plan, x, q, y, phi, grad=None, stream=None, check: bool = False) -> int:
    """Queue algorithm "get" at separate evaluation points y (device tensors, float64)."""
    for t in (x, q, y, phi) + ((grad,) if grad is not None else ()):
        if not (t.is_cuda and t.is_contiguous()):
            raise ValueError("psum_eval_points takes contiguous CUDA tensors")
    st = _stream_ptr(stream)
    s = load().psum_eval_points(plan, int(q.numel()), x.data_ptr(), q.data_ptr(), int(y.shape[0]), y.data_ptr(),
                                phi.data_ptr(), grad.data_ptr() if grad is not None else None, st)
    _check(s, "psum_eval_points")
    if check:
        _check(psum_sync(plan, st), "psum_eval_points (device)")
    return s


def psum_debug_inject_timeout(plan, enable: bool) -> None:
    _check(load().psum_debug_inject_timeout(plan, 1 if enable else 0), "psum_debug_inject_timeout")


def psum_eval_noalloc(plan, x, q, phi, grad=None, stream=None, check: bool = False) -> int:
    """psum_eval with all scratch taken from the library's static device array (no allocation)."""
    for t in (x, q, phi) + ((grad,) if grad is not None else ()):
        if not (t.is_cuda and t.is_contiguous()):
            raise ValueError("psum_eval_noalloc takes contiguous CUDA tensors")
    st = _stream_ptr(stream)
    s = load().psum_eval_noalloc(plan, int(q.numel()), x.data_ptr(), q.data_ptr(), phi.data_ptr(),
                                 grad.data_ptr() if grad is not None else None, st)
    _check(s, "psum_eval_noalloc")
    if check:
        _check(psum_sync(plan, st), "psum_eval_noalloc (device)")
    return s


def psum_eval_host(plan, x, q, phi, grad=None, stream=None) -> int:
    """Host arrays (numpy float64, C-contiguous or pinned CPU tensors); copies both ways and waits."""
    def ptr(a):
        if a is None:
            return None
        if hasattr(a, "data_ptr"):
            return a.data_ptr()
        return a.ctypes.data
    n = int(q.numel() if hasattr(q, "numel") else q.size)
    s = load().psum_eval_host(plan, n, ptr(x), ptr(q), ptr(phi), ptr(grad), _stream_ptr(stream) if stream is not None else None)
    return s


def psum_sync(plan, stream=None) -> int:
    return load().psum_sync(plan, _stream_ptr(stream))


def psum_get_coeffs(plan, P: int, stream=None):
    import numpy as np
    out = np.zeros(P, dtype=np.float64)
    _check(load().psum_get_coeffs(plan, out.ctypes.data_as(_dp), _stream_ptr(stream)), "psum_get_coeffs")
    return out


def psum_plan_info(plan) -> dict:
    info = psum_info()
    _check(load().psum_plan_info(plan, ctypes.byref(info)), "psum_plan_info")
    return info.as_dict()


def psum_pair_kernel(plan, N: int):
    """(kernel, image_groups) psum_eval uses for N charges: kernel is "one-sided" or "symmetric"."""
    k, g = ctypes.c_int(0), ctypes.c_int(0)
    _check(load().psum_pair_kernel(plan, int(N), ctypes.byref(k), ctypes.byref(g)), "psum_pair_kernel")
    return ("symmetric" if k.value == 2 else "one-sided"), g.value


def psum_scratch_bytes(plan, N: int):
    """(scratch bytes of psum_eval for N charges, bands of the symmetric charge kernel)."""
    nb, bands = ctypes.c_int64(0), ctypes.c_int(0)
    _check(load().psum_scratch_bytes(plan, int(N), ctypes.byref(nb), ctypes.byref(bands)), "psum_scratch_bytes")
    return int(nb.value), int(bands.value)


def psum_debug_band_bytes(plan, nbytes: int) -> None:
    _check(load().psum_debug_band_bytes(plan, int(nbytes)), "psum_debug_band_bytes")


def psum_debug_bounds_limit(plan, doubles: int) -> None:
    _check(load().psum_debug_bounds_limit(plan, int(doubles)), "psum_debug_bounds_limit")


def psum_debug_checks() -> bool:
    return bool(load().psum_debug_checks())


def psum_debug_fail_allocs(plan, count: int) -> None:
    _check(load().psum_debug_fail_allocs(plan, int(count)), "psum_debug_fail_allocs")


def psum_check_form(plan) -> str:
    """The form of the check-point sums psum_eval runs: "points" or "layers"."""
    f = ctypes.c_int(0)
    _check(load().psum_check_form(plan, ctypes.byref(f)), "psum_check_form")
    return "layers" if f.value == 2 else "points"


def psum_profile(plan, enable: bool = True):
    _check(load().psum_profile(plan, 1 if enable else 0), "psum_profile")


def psum_last_timings(plan, stream=None) -> dict:
    arr = (ctypes.c_double * PSUM_NUM_STAGES)()
    _check(load().psum_last_timings(plan, arr, _stream_ptr(stream)), "psum_last_timings")
    return dict(zip(STAGE_NAMES, list(arr)))


def psum_energy(plan, q, phi, E, stream=None):
    """E (a one-element float64 device tensor) = 1/2 sum q phi."""
    _check(load().psum_energy(plan, int(q.numel()), q.data_ptr(), phi.data_ptr(), E.data_ptr(),
                              _stream_ptr(stream)), "psum_energy")


def psum_energy_backward(plan, x, q, phi, grad, gE=None, dEdq=None, dEdx=None, stream=None):
    """dE/dq and dE/dx (device tensors) of E = 1/2 q.phi for the last psum_eval of this plan."""
    def ptr(t):
        return t.data_ptr() if t is not None else None
    _check(load().psum_energy_backward(plan, int(q.numel()), x.data_ptr(), q.data_ptr(), phi.data_ptr(),
                                       grad.data_ptr(), ptr(gE), ptr(dEdq), ptr(dEdx), _stream_ptr(stream)),
           "psum_energy_backward")


def psum_coeffs_device(plan, C, stream=None):
    """Queue a copy of the last evaluation's P coefficients into the device tensor C."""
    if not (C.is_cuda and C.is_contiguous() and C.dtype.itemsize == 8):
        raise ValueError("psum_coeffs_device takes a contiguous float64 CUDA tensor")
    _check(load().psum_coeffs_device(plan, C.data_ptr(), _stream_ptr(stream)), "psum_coeffs_device")


def psum_energy_backward_c(plan, x, q, phi, grad, C, gE=None, dEdq=None, dEdx=None, stream=None):
    """psum_energy_backward with the forward evaluation's coefficients C (device tensor)."""
    def ptr(t):
        return t.data_ptr() if t is not None else None
    _check(load().psum_energy_backward_c(plan, int(q.numel()), x.data_ptr(), q.data_ptr(), phi.data_ptr(),
                                         grad.data_ptr(), C.data_ptr(), ptr(gE), ptr(dEdq), ptr(dEdx),
                                         _stream_ptr(stream)), "psum_energy_backward_c")


def psum_launch_count(plan) -> int:
    n = ctypes.c_int64()
    _check(load().psum_launch_count(plan, ctypes.byref(n)), "psum_launch_count")
    return int(n.value)


def psum_destroy(plan):
    if plan:
        load().psum_destroy(plan)


def psum_batch_create(plans, offsets):
    arr = (_vp * len(plans))(*[p.value if isinstance(p, _vp) else p for p in plans])
    off = (ctypes.c_int64 * len(offsets))(*[int(v) for v in offsets])
    h = _vp()
    _check(load().psum_batch_create(arr, len(plans), off, ctypes.byref(h)), "psum_batch_create")
    return h


def psum_batch_eval(batch, x, q, phi, grad=None, use_graph: bool = False, stream=None) -> int:
    for t in (x, q, phi) + ((grad,) if grad is not None else ()):
        if not (t.is_cuda and t.is_contiguous()):
            raise ValueError("psum_batch_eval takes contiguous CUDA tensors")
    s = load().psum_batch_eval(batch, x.data_ptr(), q.data_ptr(), phi.data_ptr(),
                               grad.data_ptr() if grad is not None else None, 1 if use_graph else 0,
                               _stream_ptr(stream))
    _check(s, "psum_batch_eval")
    return s


def psum_batch_sync(batch, B: int, stream=None):
    """(first status, per-system statuses)."""
    st = (ctypes.c_int * B)()
    first = load().psum_batch_sync(batch, st, _stream_ptr(stream))
    return first, list(st)


def psum_batch_get_coeffs(batch, b: int, P: int, stream=None):
    import numpy as np
    out = np.zeros(P, dtype=np.float64)
    _check(load().psum_batch_get_coeffs(batch, int(b), out.ctypes.data_as(_dp), _stream_ptr(stream)),
           "psum_batch_get_coeffs")
    return out


def psum_batch_get_info(batch) -> dict:
    info = psum_batch_info()
    _check(load().psum_batch_get_info(batch, ctypes.byref(info)), "psum_batch_get_info")
    return info.as_dict()


def psum_batch_destroy(batch):
    if batch:
        load().psum_batch_destroy(batch)


class PeriodicBatch:
    """Many independent systems (each with its own plan) evaluated together."""

    def __init__(self, systems, precision="fp32c", mean="zero", pairs="auto", checks="auto"):
        """checks: one check-sum form for every plan, or a list with one per system."""
        forms = checks if isinstance(checks, (list, tuple)) else [checks] * len(systems)
        self.plans = [psum_plan_create_ex(s.d, s.p, s.M, precision, mean, getattr(s, "K", (1, 1, 1)), pairs=pairs,
                                          checks=c)
                      for s, c in zip(systems, forms)]
        self.P = [psum_plan_info(p)["P"] for p in self.plans]
        self.offsets = [0]
        for s in systems:
            self.offsets.append(self.offsets[-1] + s.N)
        self.batch = psum_batch_create(self.plans, self.offsets)
        self.B = len(systems)

    def __call__(self, x, q, phi=None, grad=None, use_graph=False, stream=None, check=True):
        import torch
        N = self.offsets[-1]
        if phi is None:
            phi = torch.empty(N, dtype=torch.float64, device=x.device)
        if grad is None:
            grad = torch.empty((N, 3), dtype=torch.float64, device=x.device)
        psum_batch_eval(self.batch, x, q, phi, grad, use_graph, stream)
        if check:
            first, _ = psum_batch_sync(self.batch, self.B, stream)
            _check(first, "psum_batch_eval (device)")
        return phi, grad

    def close(self):
        if self.batch:
            psum_batch_destroy(self.batch)
            self.batch = None
        for p in self.plans:
            psum_destroy(p)
        self.plans = []

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class PeriodicCoulomb:
    """A plan plus tensor-returning evaluation (allocation through torch only)."""

    def __init__(self, d, p: int, M: int, precision="fp64", mean="zero", K=(1, 1, 1), points="fibonacci",
                 lam: float = 0.0, basis="spherical", n_rbf: int = 256, rbf_radius: float = 0.0, pairs="auto",
                 checks="auto", terms="fast"):
        self.plan = psum_plan_create_ex(d, p, M, precision, mean, K, points, lam, basis, n_rbf, rbf_radius,
                                        pairs, checks, terms)
        self.info = psum_plan_info(self.plan)

    def at(self, x, q, y, grad: bool = True, stream=None, check: bool = True):
        """phi (and grad phi) at the evaluation points y due to the charges (x, q)."""
        import torch
        phi = torch.empty(y.shape[0], dtype=torch.float64, device=y.device)
        g = torch.empty((y.shape[0], 3), dtype=torch.float64, device=y.device) if grad else None
        psum_eval_points(self.plan, x, q, y, phi, g, stream, check)
        return (phi, g) if grad else phi

    def __call__(self, x, q, grad: bool = True, stream=None, check: bool = True):
        import torch
        N = q.numel()
        phi = torch.empty(N, dtype=torch.float64, device=x.device)
        g = torch.empty((N, 3), dtype=torch.float64, device=x.device) if grad else None
        psum_eval(self.plan, x, q, phi, g, stream=stream, check=check)
        return phi, g

    def coefficients(self, stream=None):
        return psum_get_coeffs(self.plan, self.info["P"], stream)

    def close(self):
        if self.plan:
            psum_destroy(self.plan)
            self.plan = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
